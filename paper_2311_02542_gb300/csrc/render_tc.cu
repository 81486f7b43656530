// render_tc.cu -- tensor-core (tcgen05) MLP path. Placeholder until the
// kernel lands: reports "not supported" so callers fail loudly.
#include "field.h"

namespace vrn {

cudaError_t launch_render_tc(vrnerf_field *, const RaySource &, const RenderOut &, int, cudaStream_t) {
    return cudaErrorNotSupported;
}

cudaError_t launch_query_tc(vrnerf_field *, const float *, const float *, const float *, int, float *,
                            float *, float *, int, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace vrn
