// TMA tensor maps of a state on a structured mesh.
//
// For each of the two population buffers c, four maps (4c + 0 .. 3)
// describe the halo windows of one iteration of the march along y
// (felbm_march.cuh), over the slot arrays (ghost columns and rows included,
// coordinates in slots): the 4 h pairs as a 3-D tensor (x in 4-byte words,
// y, pair) with a box of 40 columns x 10 rows x 4 pairs; the h rest population
// as a 2-D tensor with a box of 40 x 8; the 4 g pairs as a 3-D tensor with a
// box of the g window (10 rows); the g rest population with a box of the
// strip's own 32 x 8 nodes.  Rows outside the slot rows load zeros (outside
// a walled domain).  The maps need the driver's encoder; without it the state
// keeps d_tmap null and every window is filled by cp.async.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "felbm_internal.h"
#include "felbm_kernels.cuh"
#include "felbm_lattice.cuh"
#include "felbm_march.cuh"

namespace felbm {

static PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// One map over 4-byte words: dims/strides/box in words (x), rows, planes.
static bool encode(PFN_cuTensorMapEncodeTiled_v12000 fn, TMap *out, void *base, int rank, uint64_t x,
                   uint64_t y, uint64_t z, uint64_t row_bytes, uint64_t plane_bytes, uint32_t bx, uint32_t by,
                   uint32_t bz) {
    static_assert(sizeof(TMap) == sizeof(CUtensorMap), "tensor map size");
    const cuuint64_t dims[3] = {x, y, z};
    const cuuint64_t strides[2] = {row_bytes, plane_bytes};
    const cuuint32_t box[3] = {bx, by, bz};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUtensorMap m;
    const CUresult r = fn(&m, CU_TENSOR_MAP_DATA_TYPE_UINT32, (cuuint32_t)rank, base, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    std::memcpy(out, &m, sizeof(m));
    return true;
}

template <typename T>
static bool encode_state(PFN_cuTensorMapEncodeTiled_v12000 fn, const felbm_state *s, TMap maps[8]) {
    using MS = MarchSmem<T>;
    // the tensors are the slot arrays: pitch slots per row (ghost columns and
    // padding included), rows slot rows (ghost rows included)
    const uint64_t pitch = (uint64_t)s->mesh->sinfo.pitch, rows = (uint64_t)s->mesh->sinfo.rows;
    const uint64_t nx = pitch, ny = rows;
    const uint64_t np = pad4(pop_slots(s->mesh));
    const uint64_t wpn = sizeof(T) * 2 / 4, spn = sizeof(T) / 4;  // words per pair, per scalar
    for (int c = 0; c < 2; ++c) {
        T *f = reinterpret_cast<T *>(s->f[c]);
        const uint64_t pair_rows = pitch * wpn * 4, pair_planes = 2 * np * sizeof(T);
        TMap *mm = maps + 4 * c;
        if (!encode(fn, &mm[0], f + np, 3, nx * wpn, ny, 4, pair_rows, pair_planes, (uint32_t)(kMX * wpn),
                    (uint32_t)kHWR, 4))
            return false;
        if (!encode(fn, &mm[1], f, 2, nx * spn, ny, 1, pitch * spn * 4, 0, (uint32_t)(kMX * spn), (uint32_t)kMR,
                    1))
            return false;
        if (!encode(fn, &mm[2], f + 10 * np, 3, nx * wpn, ny, 4, pair_rows, pair_planes,
                    (uint32_t)(MS::GW * wpn), (uint32_t)kGWR, 4))
            return false;
        if (!encode(fn, &mm[3], f + 9 * np, 2, nx * spn, ny, 1, pitch * spn * 4, 0, (uint32_t)(32 * spn),
                    (uint32_t)kMR, 1))
            return false;
    }
    return true;
}

void lattice_tmaps(felbm_state *s) {
    s->d_tmap = nullptr;
    const felbm_mesh *m = s->mesh;
    if (m->kind != 1 || m->sinfo.pitch % 4 != 0) return;
    PFN_cuTensorMapEncodeTiled_v12000 fn = encoder();
    if (!fn) return;
    TMap maps[8];
    const bool ok = s->esize == 8 ? encode_state<double>(fn, s, maps) : encode_state<float>(fn, s, maps);
    if (!ok) return;
    TMap *d = nullptr;
    if (cudaMalloc((void **)&d, sizeof(maps)) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (cudaMemcpy(d, maps, sizeof(maps), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d);
        return;
    }
    s->d_tmap = d;
}

}  // namespace felbm
