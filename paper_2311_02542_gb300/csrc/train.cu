// train.cu -- backward pass and Adam. Placeholder until the kernels land.
#include "field.h"

using namespace vrn;

extern "C" {

int vrnerf_backward(vrnerf_field *, const float *, const float *, const float *, const float *, int32_t,
                    float *, void *) {
    return fail(VRNERF_EINVAL, "backward: not built yet");
}
int vrnerf_field_get_grads(vrnerf_field *, float *, float *) {
    return fail(VRNERF_EINVAL, "get_grads: not built yet");
}
int vrnerf_adam_step(vrnerf_field *, float, float, void *) { return fail(VRNERF_EINVAL, "adam: not built yet"); }
int vrnerf_train_step(vrnerf_field *, const float *, const float *, const float *, const float *, int32_t,
                      float, float, float *, void *) {
    return fail(VRNERF_EINVAL, "train_step: not built yet");
}
int vrnerf_field_set_grads(vrnerf_field *, const float *, const float *) {
    return fail(VRNERF_EINVAL, "set_grads: not built yet");
}
}
