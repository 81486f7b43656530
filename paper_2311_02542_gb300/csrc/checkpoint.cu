// checkpoint.cu -- vrnerf_field_save / vrnerf_field_load: one flat file with
// the description, parameters, occupancy and Adam state.
//
// Layout (little-endian, as written by the host): char[4] "VRNF", uint32
// version = 1, uint32 sizeof(vrnerf_field_desc), the description, uint64
// grid bytes, uint64 MLP floats, uint64 occupancy words, int32 Adam step
// (0 = no optimiser state), int32 reserved; then the grid, the MLP weights,
// the occupancy words and, when the Adam step is > 0, m and v of the grid,
// m and v of the MLP and (for an fp16 grid) the fp32 master grid.
#include <cstdio>
#include <cstring>
#include <vector>

#include "field.h"

namespace vrn {
int check_desc(const vrnerf_field_desc *d);
uint64_t occ_words(const vrnerf_field_desc &d);
}  // namespace vrn

using namespace vrn;

namespace {

struct Header {
    char magic[4];
    uint32_t version, desc_bytes;
    vrnerf_field_desc desc;
    uint64_t grid_bytes, mlp_floats, occ_words;
    int32_t adam_t, reserved;
};

bool put(FILE *f, const void *dev, size_t bytes, std::vector<unsigned char> &buf) {
    buf.resize(bytes);
    if (bytes && cudaMemcpy(buf.data(), dev, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    return fwrite(buf.data(), 1, bytes, f) == bytes;
}

bool get(FILE *f, void *dev, size_t bytes, std::vector<unsigned char> &buf) {
    buf.resize(bytes);
    if (fread(buf.data(), 1, bytes, f) != bytes) return false;
    return !bytes || cudaMemcpy(dev, buf.data(), bytes, cudaMemcpyHostToDevice) == cudaSuccess;
}

}  // namespace

extern "C" {

int vrnerf_field_save(vrnerf_field *F, const char *path) {
    if (!F || !path) return fail(VRNERF_EINVAL, "NULL argument");
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(VRNERF_ECUDA, "save: device error");
    Header h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, "VRNF", 4);
    h.version = 1;
    h.desc_bytes = sizeof(vrnerf_field_desc);
    h.desc = F->desc;
    h.grid_bytes = grid_bytes(F->desc);
    h.mlp_floats = (uint64_t)F->view.n_mlp;
    h.occ_words = occ_words(F->desc);
    h.adam_t = F->m_grid ? F->adam_t : 0;
    FILE *f = fopen(path, "wb");
    if (!f) return fail(VRNERF_EINVAL, "save: cannot open %s", path);
    std::vector<unsigned char> buf;
    bool ok = fwrite(&h, sizeof h, 1, f) == 1 && put(f, F->grid, h.grid_bytes, buf) &&
              put(f, F->mlp, h.mlp_floats * 4, buf) && put(f, F->occ, h.occ_words * 4, buf);
    if (ok && h.adam_t > 0) {
        const size_t ng = grid_entries(F->desc) * 4, nm = h.mlp_floats * 4;
        ok = put(f, F->m_grid, ng, buf) && put(f, F->v_grid, ng, buf) && put(f, F->m_mlp, nm, buf) &&
             put(f, F->v_mlp, nm, buf) && (!F->desc.feat_fp16 || put(f, F->grid_master, ng, buf));
    }
    ok = (fclose(f) == 0) && ok;
    if (!ok) return fail(VRNERF_EINVAL, "save: write to %s failed", path);
    return VRNERF_OK;
}

int vrnerf_field_load(const char *path, vrnerf_field **out) {
    if (!path || !out) return fail(VRNERF_EINVAL, "NULL argument");
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) return fail(VRNERF_EINVAL, "load: cannot open %s", path);
    Header h;
    if (fread(&h, sizeof h, 1, f) != 1 || memcmp(h.magic, "VRNF", 4) != 0 || h.version != 1 ||
        h.desc_bytes != sizeof(vrnerf_field_desc) || check_desc(&h.desc) != VRNERF_OK ||
        h.grid_bytes != grid_bytes(h.desc) || h.occ_words != occ_words(h.desc) || h.adam_t < 0) {
        fclose(f);
        return fail(VRNERF_EINVAL, "load: %s is not a field file of this version", path);
    }
    std::vector<unsigned char> grid(h.grid_bytes), occ(h.occ_words * 4);
    std::vector<float> mlp(h.mlp_floats);
    bool ok = fread(grid.data(), 1, grid.size(), f) == grid.size() &&
              fread(mlp.data(), 4, mlp.size(), f) == mlp.size() && fread(occ.data(), 1, occ.size(), f) == occ.size();
    vrnerf_field *F = nullptr;
    int rc = VRNERF_OK;
    if (ok) rc = vrnerf_field_create(&h.desc, grid.data(), mlp.data(), reinterpret_cast<const uint32_t *>(occ.data()),
                                     0, &F);
    if (ok && rc == VRNERF_OK && h.adam_t > 0) {
        const size_t ng = grid_entries(h.desc) * 4, nm = h.mlp_floats * 4;
        cudaError_t e = cudaSuccess;
        if ((e = cudaMalloc(&F->m_grid, ng)) != cudaSuccess || (e = cudaMalloc(&F->v_grid, ng)) != cudaSuccess ||
            (e = cudaMalloc(&F->m_mlp, nm)) != cudaSuccess || (e = cudaMalloc(&F->v_mlp, nm)) != cudaSuccess ||
            (h.desc.feat_fp16 && (e = cudaMalloc(&F->grid_master, ng)) != cudaSuccess))
            rc = fail(VRNERF_ENOMEM, "load: optimiser state: %s", cudaGetErrorString(e));
        std::vector<unsigned char> buf;
        if (rc == VRNERF_OK)
            ok = get(f, F->m_grid, ng, buf) && get(f, F->v_grid, ng, buf) && get(f, F->m_mlp, nm, buf) &&
                 get(f, F->v_mlp, nm, buf) && (!h.desc.feat_fp16 || get(f, F->grid_master, ng, buf));
        F->adam_t = h.adam_t;
    }
    fclose(f);
    if (!ok || rc != VRNERF_OK) {
        if (F) vrnerf_field_destroy(F);
        return rc != VRNERF_OK ? rc : fail(VRNERF_EINVAL, "load: %s is truncated", path);
    }
    *out = F;
    return VRNERF_OK;
}

}  // extern "C"
