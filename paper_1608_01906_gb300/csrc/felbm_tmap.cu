// TMA tensor maps of a state on a structured mesh.
//
// For each of the two population buffers, three maps describe the halo
// windows a tile step loads (felbm_lattice.cuh):
//   0  the 4 h pairs: 3-D (x in 4-byte words, y, pair), box of the depth-4
//      pair tile;
//   1  the h rest population: 2-D (x in words, y), box of the rest tile;
//   2  the 4 g pairs: 3-D, box of the depth-1 pair tile.
// Coordinates outside the mesh load zeros (walls); tiles whose windows would
// wrap periodically use cp.async fills instead.  The maps need rows of a
// multiple of 16 bytes (the row pitch, a multiple of 4 slots) and the
// driver's encoder; without it the state keeps d_tmap null and every tile
// uses cp.async.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "felbm_internal.h"
#include "felbm_kernels.cuh"
#include "felbm_lattice.cuh"

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
static bool encode_state(PFN_cuTensorMapEncodeTiled_v12000 fn, const felbm_state *s, TMap maps[6]) {
    using PH = PairTile<T, kHD>;
    using PG = PairTile<T, 1>;
    const uint64_t nx = (uint64_t)s->mesh->sinfo.nx, ny = (uint64_t)s->mesh->sinfo.ny;
    const uint64_t pitch = (uint64_t)s->mesh->sinfo.pitch;
    const uint64_t np = pad4(pop_slots(s->mesh));
    const uint64_t wpn = sizeof(T) * 2 / 4, spn = sizeof(T) / 4;  // words per pair, per scalar
    for (int c = 0; c < 2; ++c) {
        T *f = reinterpret_cast<T *>(s->f[c]);
        const uint64_t pair_rows = pitch * wpn * 4, pair_planes = 2 * np * sizeof(T);
        if (!encode(fn, &maps[3 * c + 0], f + np, 3, nx * wpn, ny, 4, pair_rows, pair_planes,
                    (uint32_t)(PH::W * wpn), (uint32_t)PH::H, 4))
            return false;
        if (!encode(fn, &maps[3 * c + 1], f, 2, nx * spn, ny, 1, pitch * spn * 4, 0, (uint32_t)(kH0W * spn),
                    (uint32_t)kH0H, 1))
            return false;
        if (!encode(fn, &maps[3 * c + 2], f + 10 * np, 3, nx * wpn, ny, 4, pair_rows, pair_planes,
                    (uint32_t)(PG::W * wpn), (uint32_t)PG::H, 4))
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
    TMap maps[6];
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
