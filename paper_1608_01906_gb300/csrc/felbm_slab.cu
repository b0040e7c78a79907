// Halo-sharded structured lattices: a lattice too large for one device is
// cut into slabs of whole rows, one per device.  One time step of a node
// needs the populations of the previous step up to 4 rows away (h streamed
// on the depth-3 rho region, which is itself streamed from depth-1
// neighbours: rho -> grad rho -> lap rho, mu -> grad mu, Sec. 2.2.1 and
// Sec. 2.3), so each slab keeps 4 halo rows on both sides of its own rows,
// steps its own rows only, and after each step receives its halo rows from
// its neighbours' first and last 4 own rows.
//
// A halo message (one side) holds, for the 4 rows, the h_0 array's rows,
// the 4 h pair arrays' rows, the g_0 array's rows and the 4 g pair arrays'
// rows (population layout of pop_index), each 4 x pitch slots (pairs: 2
// values per slot): 72 x pitch values.
#include <algorithm>
#include <cstring>

#include "felbm_internal.h"
#include "felbm_kernels.cuh"

namespace felbm {

constexpr int kSlabHalo = 4;  // halo rows per side

// Values of one halo message.
inline size_t halo_values(const felbm_mesh *m) { return (size_t)72 * (size_t)m->sinfo.pitch; }

// Copy the 4 rows from storage row r0 (side 0) and r1 (side 1) of the 18
// population arrays to (PACK) or from the two messages, in 16-byte chunks
// (pitch and the array stride np are multiples of 4 slots).
template <typename T, bool PACK>
__global__ void k_slab_halo(T *f, size_t np, int pitch, int r0, int r1, T *m0, T *m1) {
    constexpr int CE = 16 / (int)sizeof(T);
    const size_t p4 = (size_t)kSlabHalo * pitch;  // slots of 4 rows
    const size_t chunks = 18 * p4 / CE;           // per message
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < 2 * chunks;
         c += (size_t)gridDim.x * blockDim.x) {
        const int side = c >= chunks;
        const size_t m = (c - side * chunks) * CE;  // value index in the message
        const size_t row = (size_t)(side ? r1 : r0) * pitch;
        size_t off;
        if (m < p4) {  // h_0
            off = row + m;
        } else if (m < 9 * p4) {  // h pairs: 2 values per slot
            const size_t q = (m - p4) / (2 * p4), k = (m - p4) - q * 2 * p4;
            off = np + 2 * np * q + 2 * row + k;
        } else if (m < 10 * p4) {  // g_0
            off = 9 * np + row + (m - 9 * p4);
        } else {  // g pairs
            const size_t q = (m - 10 * p4) / (2 * p4), k = (m - 10 * p4) - q * 2 * p4;
            off = 10 * np + 2 * np * q + 2 * row + k;
        }
        if (!chk_idx(off, 18 * np - CE + 1, 8u)) continue;
        uint4 *msg = reinterpret_cast<uint4 *>((side ? m1 : m0) + m);
        uint4 *pop = reinterpret_cast<uint4 *>(f + off);
        if (PACK)
            *msg = *pop;
        else
            *pop = *msg;
    }
}

static bool is_slab(const felbm_mesh *m) { return m && m->kind == 1 && m->sinfo.gny != m->sinfo.ny; }

// Halo messages of a slab state (allocated at first use).
// Messages start zeroed: the halo rows outside a walled lattice receive
// zeros (no neighbour sends them; the step never reads them).
static cudaError_t slab_halo_alloc(felbm_state *s) {
    if (s->halo) return cudaSuccess;
    const size_t b = 4 * halo_values(s->mesh) * s->esize;
    cudaError_t e = cudaMalloc(&s->halo, b);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->halo, 0, b, s->mesh->stream);
    return e;
}

template <typename T>
static void slab_copy(felbm_state *s, bool pack) {
    const felbm_mesh *m = s->mesh;
    const StructuredInfo &si = m->sinfo;
    const size_t np = pad4(pop_slots(m)), hv = halo_values(m);
    T *f = reinterpret_cast<T *>(s->f[s->cur]);
    T *msg = reinterpret_cast<T *>(s->halo);
    const unsigned blocks = (unsigned)std::min<size_t>((2 * hv * sizeof(T) / 16 + 255) / 256, 1024);
    if (pack)  // own rows [ylo, ylo + 4) and [yhi - 4, yhi) -> send lo, send hi
        k_slab_halo<T, true><<<blocks, 256, 0, m->stream>>>(f, np, si.pitch, si.ylo, si.yhi - kSlabHalo, msg,
                                                          msg + hv);
    else  // recv lo, recv hi -> halo rows [ylo - 4, ylo) and [yhi, yhi + 4)
        k_slab_halo<T, false><<<blocks, 256, 0, m->stream>>>(f, np, si.pitch, si.ylo - kSlabHalo, si.yhi,
                                                           msg + 2 * hv, msg + 3 * hv);
}

static int slab_pack_unpack(felbm_state *s, bool pack) {
    if (!s || !is_slab(s->mesh)) return FELBM_ERR_INVALID_ARG;
    cudaError_t e = slab_halo_alloc(s);
    if (e != cudaSuccess) return cuda_status(e);
    if (s->esize == 8)
        slab_copy<double>(s, pack);
    else
        slab_copy<float>(s, pack);
    return cuda_status(cudaGetLastError());
}

FELBM_CHECK_READER(check_bits_slab)

}  // namespace felbm

using namespace felbm;

extern "C" {

int felbm_mesh_slab(const felbm_mesh *mesh, int64_t y_begin, int64_t n_rows, void *stream, felbm_mesh **out) {
    if (!mesh || !out) return FELBM_ERR_INVALID_ARG;
    if (mesh->kind != 1 || is_slab(mesh)) return FELBM_ERR_UNSUPPORTED;
    const StructuredInfo &si = mesh->sinfo;
    if (n_rows < 2 * kSlabHalo || y_begin < 0 || y_begin + n_rows > si.ny) return FELBM_ERR_INVALID_ARG;
    felbm_mesh *m = new (std::nothrow) felbm_mesh();
    if (!m) return FELBM_ERR_OOM;
    m->flags = mesh->flags;
    m->stream = reinterpret_cast<cudaStream_t>(stream);
    m->kind = 1;
    m->sinfo = si;
    m->sinfo.ny = (int32_t)(n_rows + 2 * kSlabHalo);
    m->sinfo.row0 = (int32_t)(y_begin - kSlabHalo);
    m->sinfo.gny = si.ny;
    m->sinfo.ylo = kSlabHalo;
    m->sinfo.yhi = (int32_t)(kSlabHalo + n_rows);
    m->n_nodes = (int64_t)si.nx * m->sinfo.ny;
    m->n_tri = 2 * m->n_nodes;
    // lumped masses of the own rows; zero on the halo rows, so that the
    // slab's totals are its share of the lattice's
    const size_t nx = (size_t)si.nx;
    cudaError_t e = cudaMalloc((void **)&m->d_mass, (size_t)m->n_nodes * sizeof(double));
    if (e == cudaSuccess) m->device_bytes = m->n_nodes * (int64_t)sizeof(double);
    if (e == cudaSuccess) e = cudaMemset(m->d_mass, 0, (size_t)m->n_nodes * sizeof(double));
    if (e == cudaSuccess)
        e = cudaMemcpy(m->d_mass + kSlabHalo * nx, mesh->d_mass + (size_t)y_begin * nx,
                       (size_t)n_rows * nx * sizeof(double), cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) {
        const int rs = cuda_status(e);
        mesh_free(m);
        return rs;
    }
    *out = m;
    return FELBM_OK;
}

int felbm_slab_info(const felbm_mesh *mesh, int64_t *row0, int64_t *rows, int64_t *halo_bytes_fp32) {
    if (!is_slab(mesh)) return FELBM_ERR_INVALID_ARG;
    if (row0) *row0 = mesh->sinfo.row0 + kSlabHalo;
    if (rows) *rows = mesh->sinfo.yhi - mesh->sinfo.ylo;
    if (halo_bytes_fp32) *halo_bytes_fp32 = (int64_t)(halo_values(mesh) * sizeof(float));
    return FELBM_OK;
}

int felbm_slab_halo(felbm_state *s, void **send, void **recv, int64_t *bytes) {
    if (!s || !is_slab(s->mesh) || !send || !recv || !bytes) return FELBM_ERR_INVALID_ARG;
    const cudaError_t e = slab_halo_alloc(s);
    if (e != cudaSuccess) return cuda_status(e);
    const size_t b = halo_values(s->mesh) * s->esize;
    unsigned char *h = reinterpret_cast<unsigned char *>(s->halo);
    send[0] = h;
    send[1] = h + b;
    recv[0] = h + 2 * b;
    recv[1] = h + 3 * b;
    *bytes = (int64_t)b;
    return FELBM_OK;
}

int felbm_slab_pack(felbm_state *s) { return slab_pack_unpack(s, true); }

int felbm_slab_unpack(felbm_state *s) { return slab_pack_unpack(s, false); }

int felbm_slab_exchange(felbm_state *const *slabs, int32_t n_slabs) {
    felbm::NvtxRange nvtx_range("felbm_slab_exchange");
    if (!slabs || n_slabs < 1) return FELBM_ERR_INVALID_ARG;
    const felbm_state *s0 = slabs[0];
    if (!s0 || !is_slab(s0->mesh)) return FELBM_ERR_INVALID_ARG;
    const StructuredInfo &a = s0->mesh->sinfo;
    int64_t next = a.row0 + kSlabHalo;  // the chain must tile the lattice's rows in order
    for (int32_t k = 0; k < n_slabs; ++k) {
        const felbm_state *s = slabs[k];
        if (!s || !is_slab(s->mesh)) return FELBM_ERR_INVALID_ARG;
        const StructuredInfo &b = s->mesh->sinfo;
        if (b.nx != a.nx || b.gny != a.gny || b.walls != a.walls || s->esize != s0->esize ||
            s->mesh->stream != s0->mesh->stream || b.row0 + kSlabHalo != next)
            return FELBM_ERR_INVALID_ARG;
        next += b.yhi - b.ylo;
    }
    if (next != a.row0 + kSlabHalo + a.gny || a.row0 + kSlabHalo != 0) return FELBM_ERR_INVALID_ARG;
    for (int32_t k = 0; k < n_slabs; ++k) {
        const int st = felbm_slab_pack(slabs[k]);
        if (st != FELBM_OK) return st;
    }
    // slab k's recv lo <- slab k-1's send hi, its recv hi <- slab k+1's
    // send lo (periodic: around the ends; walled: the rows outside the
    // lattice are never read and get no message)
    const size_t b = halo_values(s0->mesh) * s0->esize;
    const cudaStream_t st = s0->mesh->stream;
    for (int32_t k = 0; k < n_slabs; ++k) {
        unsigned char *rk = reinterpret_cast<unsigned char *>(slabs[k]->halo);
        const bool lo_in = k > 0 || !a.walls, hi_in = k < n_slabs - 1 || !a.walls;
        const int32_t kl = (k + n_slabs - 1) % n_slabs, kh = (k + 1) % n_slabs;
        cudaError_t e = cudaSuccess;
        if (lo_in)
            e = cudaMemcpyAsync(rk + 2 * b, reinterpret_cast<unsigned char *>(slabs[kl]->halo) + b, b,
                                cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess && hi_in)
            e = cudaMemcpyAsync(rk + 3 * b, reinterpret_cast<unsigned char *>(slabs[kh]->halo), b,
                                cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_status(e);
    }
    for (int32_t k = 0; k < n_slabs; ++k) {
        const int st2 = felbm_slab_unpack(slabs[k]);
        if (st2 != FELBM_OK) return st2;
    }
    return FELBM_OK;
}

}  // extern "C"
