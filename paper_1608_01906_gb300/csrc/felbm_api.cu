// C ABI of the FE-LBM library: handle management, uploads, launches.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "felbm_internal.h"
#include "felbm_kernels.cuh"
#include "felbm_lattice.cuh"
#include "felbm_patch.cuh"

using namespace felbm;

namespace felbm {

__global__ void k_totals_final(int nparts, const double *__restrict__ part, double *__restrict__ out) {
    // single warp, fixed order over lanes then shuffle tree: deterministic
    double s0 = 0, s1 = 0, s2 = 0;
    for (int k = threadIdx.x; k < nparts; k += 32) {
        s0 += part[3 * k];
        s1 += part[3 * k + 1];
        s2 += part[3 * k + 2];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if (threadIdx.x == 0) {
        out[0] = s0;
        out[1] = s1;
        out[2] = s2;
    }
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return FELBM_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return FELBM_ERR_OOM;
    }
    return FELBM_ERR_CUDA;
}

#define FELBM_CK(x)                              \
    do {                                         \
        cudaError_t _e = (x);                    \
        if (_e != cudaSuccess) return cuda_status(_e); \
    } while (0)

template <typename T>
static DevCSR<T> dev_csr(const felbm_mesh *m) {
    DevCSR<T> d;
    d.n = (int32_t)m->n_nodes;
    d.rowptr = m->d_rowptr;
    d.col = m->d_col;
    const size_t nnz = m->host.col.size();
    const T *base;
    if (sizeof(T) == 8)
        base = reinterpret_cast<const T *>(m->d_coef64);
    else
        base = reinterpret_cast<const T *>(m->d_coef32);
    d.ax = base;
    d.ay = base + nnz;
    d.bxx = base + 2 * nnz;
    d.bxy = base + 3 * nnz;
    d.byy = base + 4 * nnz;
    d.tag = m->d_tag;
    return d;
}

template <typename T>
static Phys<T> phys_of(const felbm_params &p) {
    const double d = p.rho_l - p.rho_v;
    Phys<T> P;
    P.rho_l = (T)p.rho_l;
    P.rho_v = (T)p.rho_v;
    P.beta = (T)(12.0 * p.sigma / (p.xi * d * d * d * d));
    P.kappa = (T)(1.5 * p.xi * p.sigma / (d * d));
    P.inv_tau_l = (T)(1.0 / p.tau_l);
    P.inv_tau_v = (T)(1.0 / p.tau_v);
    P.dt = (T)p.dt;
    P.gx = (T)p.gravity[0];
    P.gy = (T)p.gravity[1];
    P.inv_drho = (T)(1.0 / (p.rho_l - p.rho_v));
    return P;
}

// Scratch: on general meshes the streamed h* (9 Np, population layout)
// first, then 6 N fields (rho, grad rho, mu, K).
static size_t hstar_elems(const felbm_mesh *m) { return m->kind == 0 ? 9 * pad4(pop_slots(m)) : 0; }

template <typename T>
static Fields<T> fields_of(felbm_state *s) {
    const size_t n = (size_t)s->mesh->n_nodes;
    T *base = reinterpret_cast<T *>(s->scratch);
    const size_t nh = hstar_elems(s->mesh);
    T *b = base + nh;
    Fields<T> F;
    F.hs = nh ? base : nullptr;
    F.rho = b;
    F.drx = b + n;
    F.dry = b + 2 * n;
    F.mu = b + 3 * n;
    F.kx = b + 4 * n;
    F.ky = b + 5 * n;
    return F;
}

static inline unsigned nblocks(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

static constexpr size_t kProfMaxLaunches = 4096;

int prof_begin(felbm_state *s, int kind) {
    s->launches[kind]++;
    if (!s->prof_on || (s->prof_seen[kind]++ % s->prof_stride) != 0 || s->prof_used >= kProfMaxLaunches)
        return -1;
    const size_t slot = s->prof_used++;
    s->prof_kind[slot] = kind;
    cudaEventRecord(s->prof_ev[2 * slot], s->mesh->stream);
    return (int)slot;
}

void prof_end(felbm_state *s, int slot) {
    if (slot >= 0) cudaEventRecord(s->prof_ev[2 * slot + 1], s->mesh->stream);
}

template <typename T>
static DevLattice<T> dev_lattice(const felbm_mesh *m) {
    DevLattice<T> d;
    d.n = (int32_t)m->n_nodes;
    d.nx = m->sinfo.nx;
    d.ny = m->sinfo.ny;
    d.walls = m->sinfo.walls ? 1 : 0;
    d.pitch = m->sinfo.pitch;
    d.row0 = m->sinfo.row0;
    d.gny = m->sinfo.gny;
    for (int k = 0; k < 3; ++k)
        for (int o = 0; o < 6; ++o) {
            d.c[k][o][0] = (T)m->sinfo.a[k][o][0];
            d.c[k][o][1] = (T)m->sinfo.a[k][o][1];
            for (int q = 0; q < 3; ++q) d.c[k][o][2 + q] = (T)m->sinfo.b[k][o][q];
        }
    return d;
}

// Derivative chain shared by init and step: rho (already in F.rho) ->
// grad rho -> lap rho, K, mu.
// Threads per block of the general path's node kernels (one node per
// thread).  On the 256 x 256 Delaunay mesh (65,536 nodes, fewer blocks than
// two per SM) blocks of 128 and 64 threads spread the mesh more evenly but
// ran 3-7% slower than 256.
constexpr int kGenBlock = 256;

// kappa in FP64 (the FP64 kappa lap rho term of FELBM_PARAM_LAP_FP64)
static double kappa64(const felbm_params &p) {
    const double d = p.rho_l - p.rho_v;
    return 1.5 * p.xi * p.sigma / (d * d);
}

static bool lap_fp64(const felbm_state *s) { return s->esize == 4 && (s->params.flags & FELBM_PARAM_LAP_FP64); }

// The mesh's operators with FP64 coefficients, for the FP64 Laplacian.
static DevCSR<double> topo64(const felbm_mesh *m, const DevCSR<float> &) { return dev_csr<double>(m); }
static DevLattice<double> topo64(const felbm_mesh *m, const DevLattice<float> &) { return dev_lattice<double>(m); }

template <typename T, typename Topo>
static void launch_chain(felbm_state *s, const Topo &d) {
    const felbm_mesh *m = s->mesh;
    const Fields<T> F = fields_of<T>(s);
    const Phys<T> P = phys_of<T>(s->params);
    const unsigned g = nblocks(m->n_nodes, kGenBlock);
    int sl = prof_begin(s, 1);
    k_grad<T, Topo><<<g, kGenBlock, 0, m->stream>>>(d, F);
    prof_end(s, sl);
    sl = prof_begin(s, 2);
    if constexpr (sizeof(T) == 4) {
        if (lap_fp64(s)) {
            const auto d64 = topo64(m, d);
            k_mu_lap64<decltype(d64)><<<g, kGenBlock, 0, m->stream>>>(d64, F, P, kappa64(s->params));
        } else {
            k_mu<T, Topo><<<g, kGenBlock, 0, m->stream>>>(d, F, P);
        }
    } else {
        k_mu<T, Topo><<<g, kGenBlock, 0, m->stream>>>(d, F, P);
    }
    prof_end(s, sl);
}

template <typename T, typename Topo>
static void step_topo(felbm_state *s, const Topo &d, bool write_mom) {
    const felbm_mesh *m = s->mesh;
    const Fields<T> F = fields_of<T>(s);
    const Phys<T> P = phys_of<T>(s->params);
    const unsigned g = nblocks(m->n_nodes, kGenBlock);
    const T *fin = reinterpret_cast<const T *>(s->f[s->cur]);
    T *fout = reinterpret_cast<T *>(s->f[s->cur ^ 1]);
    int sl = prof_begin(s, 0);
    k_rho<T, Topo><<<g, kGenBlock, 0, m->stream>>>(d, fin, P.dt, F.rho, F.hs);
    prof_end(s, sl);
    launch_chain<T, Topo>(s, d);
    CollideArgs<T, Topo> A;
    A.m = d;
    A.fin = fin;
    A.fout = fout;
    A.F = F;
    A.P = P;
    A.mom = write_mom ? reinterpret_cast<T *>(s->mom) : nullptr;
    A.flag = s->d_flag;
    sl = prof_begin(s, 3);
    k_collide<T, Topo><<<g, kGenBlock, 0, m->stream>>>(A);
    prof_end(s, sl);
    s->cur ^= 1;
}

template <typename T, typename Topo>
static void init_topo(felbm_state *s, const Topo &d) {
    const felbm_mesh *m = s->mesh;
    const Fields<T> F = fields_of<T>(s);
    const Phys<T> P = phys_of<T>(s->params);
    // F.rho <- rho0 (first quarter of the moments buffer)
    cudaMemcpyAsync(F.rho, s->mom, (size_t)m->n_nodes * sizeof(T), cudaMemcpyDeviceToDevice,
                    m->stream);
    launch_chain<T, Topo>(s, d);
    const unsigned g = nblocks(m->n_nodes, kGenBlock);
    k_init<T, Topo><<<g, kGenBlock, 0, m->stream>>>(d, reinterpret_cast<T *>(s->f[s->cur]), F, P,
                                              reinterpret_cast<const T *>(s->mom));
}

// Constant coefficient tables of a structured mesh for the state's dt.
template <typename T>
static LatCoef<T> lat_coef(const felbm_mesh *m, double dt) {
    LatCoef<T> c;
    for (int k = 0; k < 3; ++k)
        for (int o = 0; o < 6; ++o) {
            const double ax = m->sinfo.a[k][o][0], ay = m->sinfo.a[k][o][1];
            const double bxx = m->sinfo.b[k][o][0], bxy = m->sinfo.b[k][o][1],
                         byy = m->sinfo.b[k][o][2];
            c.r[k][o][0] = (T)ax;
            c.r[k][o][1] = (T)ay;
            T sv[9];
            for (int a = 1; a < 9; ++a) {
                const double ex = kEx(a), ey = kEy(a);
                sv[a] = (T)(ex * ax + ey * ay +
                            0.5 * dt * (ex * ex * bxx + 2.0 * ex * ey * bxy + ey * ey * byy));
            }
            for (int q = 0; q < 4; ++q) {
                c.s[k][o][q].x = sv[pair_dir(q, 0)];
                c.s[k][o][q].y = sv[pair_dir(q, 1)];
            }
        }
    return c;
}

template <typename T, bool LAP64>
static void step_lattice(felbm_state *s, LatArgs<T> &A, bool write_mom) {
    const felbm_mesh *m = s->mesh;
    A.fin = reinterpret_cast<const T *>(s->f[s->cur]);
    A.fout = reinterpret_cast<T *>(s->f[s->cur ^ 1]);
    A.mom = write_mom ? reinterpret_cast<T *>(s->mom) : nullptr;
    A.tmap = s->d_tmap ? s->d_tmap + 3 * s->cur : nullptr;
    const dim3 grd((A.nx + kLTX - 1) / kLTX, (A.yhi - A.ylo + kLTY - 1) / kLTY);
    const int sl = prof_begin(s, 4);
    k_lat_step<T, LAP64><<<grd, dim3(kLTX, kLTY), lat_smem<T>(), m->stream>>>(A);
    prof_end(s, sl);
    s->cur ^= 1;
}

// The dynamic shared memory of k_lat_step is above the default limit: set
// the function attribute once per device (bit d of done, set only once the
// call succeeded; devices from 64 on set it at every call).  A refusal is
// returned to the caller of felbm_step.
template <typename T, bool LAP64>
static cudaError_t lat_smem_attr() {
    static std::atomic<uint64_t> done{0};
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = -1;
    }
    const uint64_t bit = (dev >= 0 && dev < 64) ? (uint64_t(1) << dev) : 0;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    const cudaError_t e =
        cudaFuncSetAttribute(k_lat_step<T, LAP64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lat_smem<T>());
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e;
    }
    if (bit) done.fetch_or(bit, std::memory_order_release);
    return cudaSuccess;
}

// One launch per step over the patches of a general triangle mesh; false
// when its shared memory exceeds what a block can have (the four-launch
// step then runs).
template <typename T, bool LAP64>
static bool patch_steps(felbm_state *s, int64_t n, cudaError_t &err) {
    const felbm_mesh *m = s->mesh;
    const HostCSR &H = m->host;
    const size_t smem = patch_smem<T>(H.rmax, H.r1max, H.r2max, H.r3max);
    if (smem > 227 * 1024) return false;
    err = cudaFuncSetAttribute(k_patch_step<T, LAP64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    PatchArgs<T> A;
    A.m = dev_csr<T>(m);
    A.nbase = m->d_pnbase;
    A.count = m->d_pcount;
    A.node = m->d_pnode;
    A.rowbase = m->d_prowbase;
    A.lcol = m->d_plcol;
    A.rmax = H.rmax;
    A.r1max = H.r1max;
    A.r2max = H.r2max;
    A.r3max = H.r3max;
    A.P = phys_of<T>(s->params);
    A.flag = s->d_flag;
    A.ax64 = m->d_coef64;  // SoA: a_x, a_y, b_xx, b_xy, b_yy
    A.ay64 = m->d_coef64 + m->host.col.size();
    A.kappa64 = kappa64(s->params);
    const unsigned blocks = (unsigned)(H.pnbase.size() - 1);
    for (int64_t k = 0; k < n; ++k) {
        A.fin = reinterpret_cast<const T *>(s->f[s->cur]);
        A.fout = reinterpret_cast<T *>(s->f[s->cur ^ 1]);
        A.mom = k == n - 1 ? reinterpret_cast<T *>(s->mom) : nullptr;
        const int sl = prof_begin(s, 5);
        k_patch_step<T, LAP64><<<blocks, kPatch, smem, m->stream>>>(A);
        prof_end(s, sl);
        s->cur ^= 1;
    }
    return true;
}

template <typename T>
static int do_steps(felbm_state *s, int64_t n) {
    const felbm_mesh *m = s->mesh;
    if (m->kind == 0 && m->patch_step) {
        cudaError_t err = cudaSuccess;
        bool done;
        if constexpr (sizeof(T) == 4)
            done = lap_fp64(s) ? patch_steps<T, true>(s, n, err) : patch_steps<T, false>(s, n, err);
        else
            done = patch_steps<T, false>(s, n, err);
        if (done) return cuda_status(err);
    }
    if (m->kind == 1) {
        const bool l64 = lap_fp64(s);
        cudaError_t ea;
        if constexpr (sizeof(T) == 4)
            ea = l64 ? lat_smem_attr<T, true>() : lat_smem_attr<T, false>();
        else
            ea = lat_smem_attr<T, false>();
        if (ea != cudaSuccess) return cuda_status(ea);
        LatArgs<T> A;
        A.nx = m->sinfo.nx;
        A.ny = m->sinfo.ny;
        A.pitch = m->sinfo.pitch;
        A.walls = m->sinfo.walls ? 1 : 0;
        A.row0 = m->sinfo.row0;
        A.gny = m->sinfo.gny;
        A.ylo = m->sinfo.ylo;
        A.yhi = m->sinfo.yhi;
        A.c = lat_coef<T>(m, s->params.dt);
        lat_uniform_consts<T>(m->sinfo, s->params.dt, A);
        A.P = phys_of<T>(s->params);
        A.rho = fields_of<T>(s).rho;
        A.flag = s->d_flag;
        A.al64 = 1.0 / (6.0 * m->sinfo.h);
        A.kappa64 = kappa64(s->params);
        for (int k = 0; k < 3; ++k)
            for (int o = 0; o < 6; ++o)
                for (int c = 0; c < 2; ++c) A.r64[k][o][c] = m->sinfo.a[k][o][c];
        for (int64_t k = 0; k < n; ++k) {
            if constexpr (sizeof(T) == 4) {
                if (l64) {
                    step_lattice<T, true>(s, A, k == n - 1);
                    continue;
                }
            }
            step_lattice<T, false>(s, A, k == n - 1);
        }
    } else {
        const DevCSR<T> d = dev_csr<T>(m);
        for (int64_t k = 0; k < n; ++k) step_topo<T>(s, d, k == n - 1);
    }
    return FELBM_OK;
}

template <typename T>
static void init_any(felbm_state *s) {
    if (s->mesh->kind == 1)
        init_topo<T>(s, dev_lattice<T>(s->mesh));
    else
        init_topo<T>(s, dev_csr<T>(s->mesh));
}

template <typename T>
static void launch_moments(felbm_state *s) {
    const felbm_mesh *m = s->mesh;
    const int32_t n = (int32_t)m->n_nodes;
    const int32_t *iperm = m->kind == 1 ? nullptr : m->d_perm + n;  // d_perm holds perm | iperm
    k_gather_moments<T><<<nblocks(n, 256), 256, 0, m->stream>>>(
        n, reinterpret_cast<const T *>(s->mom), iperm, s->params.rho_l, s->params.rho_v, s->d_out);
    double *part = s->d_out + 5 * (size_t)n;
    k_totals_partial<T><<<kTotalsBlocks, 256, 0, m->stream>>>(
        n, reinterpret_cast<const T *>(s->mom), m->d_mass, part);
    k_totals_final<<<1, 32, 0, m->stream>>>(kTotalsBlocks, part, part + 3 * kTotalsBlocks);
}

void mesh_free(felbm_mesh *m) {
    if (!m) return;
    cudaFree(m->d_rowptr);
    cudaFree(m->d_col);
    cudaFree(m->d_perm);
    cudaFree(m->d_coef64);
    cudaFree(m->d_coef32);
    cudaFree(m->d_mass);
    cudaFree(m->d_tag);
    cudaFree(m->d_pnbase);
    cudaFree(m->d_pcount);
    cudaFree(m->d_pnode);
    cudaFree(m->d_prowbase);
    cudaFree(m->d_plcol);
    delete m;
}

void state_free(felbm_state *s) {
    if (!s) return;
    for (auto &e : s->prof_ev)
        if (e) cudaEventDestroy(e);
    cudaFree(s->f[0]);
    cudaFree(s->f[1]);
    cudaFree(s->scratch);
    cudaFree(s->mom);
    cudaFree(s->d_out);
    cudaFree(s->d_flag);
    cudaFree(s->d_tmap);
    cudaFree(s->halo);
    delete s;
}

bool params_ok(const felbm_params *p) {
    const double v[] = {p->rho_l, p->rho_v, p->sigma, p->xi, p->tau_l, p->tau_v, p->dt,
                        p->gravity[0], p->gravity[1], p->gravity[2]};
    for (double x : v)
        if (!std::isfinite(x)) return false;
    return p->rho_l > p->rho_v && p->rho_v > 0.0 && p->sigma >= 0.0 && p->xi > 0.0 &&
           p->tau_l > 0.0 && p->tau_v > 0.0 && p->dt > 0.0 &&
           (p->precision == FELBM_FP64 || p->precision == FELBM_FP32) && (p->flags & ~FELBM_PARAM_LAP_FP64) == 0;
}

// One block waits on an mbarrier that nothing arrives on (phase 0 never
// completes), through the same bounded wait the tiles use for their TMA
// loads, and records the give-up in the flag as a tile does.
__global__ void k_wait_selftest(int *flag, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    const bool ok = threadIdx.x != 0 || mbar_wait(&bar, 0u, limit_ns);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(flag, 4);
}

FELBM_CHECK_READER(check_bits_api)

}  // namespace felbm

// ============================================================================
extern "C" {

int felbm_check_status(int32_t *checked_build, int32_t *bits) {
    if (!checked_build || !bits) return FELBM_ERR_INVALID_ARG;
#ifdef FELBM_CHECKED
    *checked_build = 1;
#else
    *checked_build = 0;
#endif
    *bits = (int32_t)(check_bits_api() | check_bits_api3() | check_bits_batch() | check_bits_slab());
    return FELBM_OK;
}

int felbm_wait_selftest(felbm_state *s, int64_t limit_ns) {
    if (!s || limit_ns < 1 || limit_ns > 2000000000LL) return FELBM_ERR_INVALID_ARG;
    k_wait_selftest<<<1, 32, 0, s->mesh->stream>>>(s->d_flag, (uint64_t)limit_ns);
    return cuda_status(cudaGetLastError());
}

const char *felbm_status_string(int st) {
    switch (st) {
        case FELBM_OK: return "ok";
        case FELBM_ERR_INVALID_ARG: return "invalid argument";
        case FELBM_ERR_INVALID_MESH: return "invalid mesh";
        case FELBM_ERR_OOM: return "out of memory";
        case FELBM_ERR_NONFINITE: return "non-finite value produced";
        case FELBM_ERR_TIMEOUT: return "bounded device wait gave up";
        case FELBM_ERR_CUDA: return "CUDA error";
        case FELBM_ERR_UNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}


int felbm_mesh_create(const double *xy, int64_t n_nodes, const int32_t *tri, int64_t n_tri,
                      const double box[2], uint32_t flags, const uint8_t *node_tag, void *stream,
                      felbm_mesh **out) {
    if (!xy || !tri || !box || !out) return FELBM_ERR_INVALID_ARG;
    if (n_nodes < 3 || n_tri < 1 || n_nodes > 0x7fffffffLL || n_tri > 0x7fffffffLL / 3)
        return FELBM_ERR_INVALID_ARG;
    if ((flags & ~(FELBM_PERIODIC_X | FELBM_PERIODIC_Y | FELBM_MESH_GENERAL | FELBM_MESH_SPLIT_STEP |
                   FELBM_MESH_PATCH_STEP)) ||
        ((flags & FELBM_MESH_SPLIT_STEP) && (flags & FELBM_MESH_PATCH_STEP)))
        return FELBM_ERR_INVALID_ARG;
    felbm_mesh *m = new (std::nothrow) felbm_mesh();
    if (!m) return FELBM_ERR_OOM;
    m->n_nodes = n_nodes;
    m->n_tri = n_tri;
    m->flags = flags;
    m->stream = reinterpret_cast<cudaStream_t>(stream);
    // cheap checks every path relies on
    if (((flags & FELBM_PERIODIC_X) && !(box[0] > 0.0)) ||
        ((flags & FELBM_PERIODIC_Y) && !(box[1] > 0.0))) {
        delete m;
        return FELBM_ERR_INVALID_ARG;
    }
    for (int64_t t = 0; t < 3 * n_tri; ++t)
        if (tri[t] < 0 || tri[t] >= n_nodes) {
            delete m;
            return FELBM_ERR_INVALID_MESH;
        }
    int st = FELBM_OK;
    std::vector<double> lattice_mass;
    try {
        // a structured lattice needs no assembled CSR: its three row kinds'
        // coefficients come from the triangles around representative nodes
        if (!(flags & FELBM_MESH_GENERAL))
            detect_structured(xy, n_nodes, tri, n_tri, box, flags, node_tag, m->sinfo, lattice_mass);
        if (!m->sinfo.ok) st = build_csr(xy, n_nodes, tri, n_tri, box, flags, node_tag, m->host);
    } catch (const std::bad_alloc &) {
        st = FELBM_ERR_OOM;
    }
    if (st != FELBM_OK) {
        delete m;
        return st;
    }
    m->kind = m->sinfo.ok ? 1 : 0;
    const HostCSR &H = m->host;
    const size_t N = (size_t)n_nodes, nnz = H.col.size();
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) {
            e = cudaMalloc(p, bytes);
            if (e == cudaSuccess) m->device_bytes += (int64_t)bytes;
        }
    };
    alloc((void **)&m->d_mass, N * sizeof(double));
    if (m->kind == 0) {
        alloc((void **)&m->d_rowptr, (N + 1) * sizeof(int32_t));
        alloc((void **)&m->d_col, nnz * sizeof(int32_t));
        alloc((void **)&m->d_perm, 2 * N * sizeof(int32_t));
        alloc((void **)&m->d_coef64, 5 * nnz * sizeof(double));
        alloc((void **)&m->d_coef32, 5 * nnz * sizeof(float));
        if (!H.tag.empty()) alloc((void **)&m->d_tag, N);
        // the patch step by default up to kPatchStepMaxNodes (measured: 1.48x
        // faster on 65,536 nodes, even on 262,144, 1.27x slower on 1,048,576,
        // where its dependent coefficient loads leave it latency-bound)
        m->patch_step = !H.pnbase.empty() && ((flags & FELBM_MESH_PATCH_STEP) ||
                                              (!(flags & FELBM_MESH_SPLIT_STEP) && n_nodes <= kPatchStepMaxNodes));
        if (m->patch_step) {
            alloc((void **)&m->d_pnbase, H.pnbase.size() * sizeof(int32_t));
            alloc((void **)&m->d_pcount, H.pcount.size() * sizeof(int32_t));
            alloc((void **)&m->d_pnode, H.pnode.size() * sizeof(int32_t));
            alloc((void **)&m->d_prowbase, H.prowbase.size() * sizeof(int32_t));
            alloc((void **)&m->d_plcol, std::max<size_t>(H.plcol.size(), 1) * sizeof(uint16_t));
        }
    }
    if (e != cudaSuccess) {
        int rs = cuda_status(e);
        mesh_free(m);
        return rs;
    }
    // uploads (synchronous: host vectors are temporaries of this call)
    if (m->kind == 1) {
        // structured kernels use the caller's (lattice) order
        e = cudaMemcpy(m->d_mass, lattice_mass.data(), N * sizeof(double), cudaMemcpyHostToDevice);
    } else {
        e = cudaMemcpy(m->d_mass, H.mass.data(), N * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(m->d_rowptr, H.rowptr.data(), (N + 1) * sizeof(int32_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(m->d_col, H.col.data(), nnz * sizeof(int32_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(m->d_perm, H.perm.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(m->d_perm + N, H.iperm.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice);
        std::vector<double> c64(5 * nnz);
        std::vector<float> c32(5 * nnz);
        const std::vector<double> *src[5] = {&H.ax, &H.ay, &H.bxx, &H.bxy, &H.byy};
        for (int k = 0; k < 5; ++k)
            for (size_t q = 0; q < nnz; ++q) {
                c64[k * nnz + q] = (*src[k])[q];
                c32[k * nnz + q] = (float)(*src[k])[q];
            }
        if (e == cudaSuccess)
            e = cudaMemcpy(m->d_coef64, c64.data(), 5 * nnz * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(m->d_coef32, c32.data(), 5 * nnz * sizeof(float), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && m->d_tag)
            e = cudaMemcpy(m->d_tag, H.tag.data(), N, cudaMemcpyHostToDevice);
        if (m->patch_step) {
            auto up = [&](void *d, const void *h, size_t b) {
                if (e == cudaSuccess && b) e = cudaMemcpy(d, h, b, cudaMemcpyHostToDevice);
            };
            up(m->d_pnbase, H.pnbase.data(), H.pnbase.size() * sizeof(int32_t));
            up(m->d_pcount, H.pcount.data(), H.pcount.size() * sizeof(int32_t));
            up(m->d_pnode, H.pnode.data(), H.pnode.size() * sizeof(int32_t));
            up(m->d_prowbase, H.prowbase.data(), H.prowbase.size() * sizeof(int32_t));
            up(m->d_plcol, H.plcol.data(), H.plcol.size() * sizeof(uint16_t));
        }
    }
    if (e != cudaSuccess) {
        int rs = cuda_status(e);
        mesh_free(m);
        return rs;
    }
    *out = m;
    return FELBM_OK;
}

int felbm_mesh_info(const felbm_mesh *m, int64_t *n_nodes, int64_t *n_tri, int32_t *kind,
                    int64_t *device_bytes) {
    if (!m) return FELBM_ERR_INVALID_ARG;
    if (n_nodes) *n_nodes = m->n_nodes;
    if (n_tri) *n_tri = m->n_tri;
    if (kind) *kind = m->kind;
    if (device_bytes) *device_bytes = m->device_bytes;
    return FELBM_OK;
}

void felbm_mesh_destroy(felbm_mesh *m) { mesh_free(m); }



int felbm_state_init(const felbm_mesh *mesh, const felbm_params *params, const double *rho0,
                     const double *u0, const double *p0, felbm_state **out) {
    felbm::NvtxRange nvtx_range("felbm_state_init");
    if (!mesh || !params || !rho0 || !out) return FELBM_ERR_INVALID_ARG;
    if (!params_ok(params)) return FELBM_ERR_INVALID_ARG;
    if (mesh->kind >= 2) return state_init3(mesh, params, rho0, u0, p0, out);
    const size_t N = (size_t)mesh->n_nodes;
    for (size_t i = 0; i < N; ++i)
        if (!(rho0[i] > 0.0) || !std::isfinite(rho0[i])) return FELBM_ERR_INVALID_ARG;
    felbm_state *s = new (std::nothrow) felbm_state();
    if (!s) return FELBM_ERR_OOM;
    s->mesh = mesh;
    s->params = *params;
    s->precision = params->precision;
    s->esize = params->precision == FELBM_FP64 ? 8 : 4;
    const size_t es = s->esize;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    alloc(&s->f[0], 18 * pad4(pop_slots(mesh)) * es);
    alloc(&s->f[1], 18 * pad4(pop_slots(mesh)) * es);
    alloc(&s->scratch, (hstar_elems(mesh) + 6 * N) * es);
    alloc(&s->mom, 4 * N * es);
    alloc((void **)&s->d_out, (5 * N + 3 * (kTotalsBlocks + 1)) * sizeof(double));
    alloc((void **)&s->d_flag, sizeof(int));
    if (e != cudaSuccess) {
        int rs = cuda_status(e);
        state_free(s);
        return rs;
    }
    // initial moments in the kernels' node order and precision
    const bool perm = mesh->kind == 0;
    std::vector<unsigned char> hm(4 * N * es);
    for (size_t k = 0; k < N; ++k) {
        const size_t c = perm ? (size_t)mesh->host.perm[k] : k;
        const double v[4] = {rho0[c], u0 ? u0[2 * c] : 0.0, u0 ? u0[2 * c + 1] : 0.0,
                             p0 ? p0[c] : 0.0};
        for (int q = 0; q < 4; ++q) {
            if (!std::isfinite(v[q])) {
                state_free(s);
                return FELBM_ERR_INVALID_ARG;
            }
            if (es == 8)
                reinterpret_cast<double *>(hm.data())[q * N + k] = v[q];
            else
                reinterpret_cast<float *>(hm.data())[q * N + k] = (float)v[q];
        }
    }
    e = cudaMemcpyAsync(s->mom, hm.data(), hm.size(), cudaMemcpyHostToDevice, mesh->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_flag, 0, sizeof(int), mesh->stream);
    // padding slots of structured rows are never read; zeroed all the same
    for (int c = 0; c < 2 && e == cudaSuccess; ++c)
        e = cudaMemsetAsync(s->f[c], 0, 18 * pad4(pop_slots(mesh)) * es, mesh->stream);
    if (e == cudaSuccess) {
        if (es == 8)
            init_any<double>(s);
        else
            init_any<float>(s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(mesh->stream);  // hm is a temporary
    if (e != cudaSuccess) {
        int rs = cuda_status(e);
        state_free(s);
        return rs;
    }
    lattice_tmaps(s);  // optional: tiles fall back to cp.async fills without maps
    s->have_moments = true;
    *out = s;
    return FELBM_OK;
}

int felbm_step(felbm_state *s, int64_t n_steps) {
    felbm::NvtxRange nvtx_range("felbm_step");
    if (!s || n_steps < 0) return FELBM_ERR_INVALID_ARG;
    if (n_steps == 0) return FELBM_OK;
    if (s->mesh->kind >= 2) {
        steps3(s, n_steps);
    } else {
        const int st = s->esize == 8 ? do_steps<double>(s, n_steps) : do_steps<float>(s, n_steps);
        if (st != FELBM_OK) return st;
    }
    s->steps_done += n_steps;
    s->have_moments = true;
    return cuda_status(cudaGetLastError());
}

static int check_flag(felbm_state *s) {
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, s->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s->mesh->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->mesh->stream);
    if (e != cudaSuccess) return cuda_status(e);
    return (h & 1) ? FELBM_ERR_NONFINITE : (h & 4) ? FELBM_ERR_TIMEOUT : FELBM_OK;
}

int felbm_state_sync(felbm_state *s) {
    if (!s) return FELBM_ERR_INVALID_ARG;
    return check_flag(s);
}

int felbm_moments_get(felbm_state *s, double *rho, double *C, double *u, double *p, double totals[3]) {
    felbm::NvtxRange nvtx_range("felbm_moments_get");
    if (!s) return FELBM_ERR_INVALID_ARG;
    if (!s->have_moments) return FELBM_ERR_INVALID_ARG;
    if (s->mesh->kind >= 2) {
        const int st3 = moments3(s, rho, C, u, p, totals);
        return st3 != FELBM_OK ? st3 : check_flag(s);
    }
    const size_t N = (size_t)s->mesh->n_nodes;
    const cudaStream_t st = s->mesh->stream;
    if (s->esize == 8)
        launch_moments<double>(s);
    else
        launch_moments<float>(s);
    cudaError_t e = cudaGetLastError();
    double *o = s->d_out;
    if (e == cudaSuccess && rho) e = cudaMemcpyAsync(rho, o, N * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && C) e = cudaMemcpyAsync(C, o + N, N * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && u) e = cudaMemcpyAsync(u, o + 2 * N, 2 * N * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && p) e = cudaMemcpyAsync(p, o + 4 * N, N * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && totals)
        e = cudaMemcpyAsync(totals, o + 5 * N + 3 * kTotalsBlocks, 3 * 8, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_status(e);
    return check_flag(s);
}

int felbm_state_export(felbm_state *s, double *hbar, double *gbar) {
    if (!s || !hbar || !gbar) return FELBM_ERR_INVALID_ARG;
    if (s->mesh->kind >= 2) {
        const int st3 = export3(s, hbar, gbar);
        return st3 != FELBM_OK ? st3 : check_flag(s);
    }
    const size_t N = (size_t)s->mesh->n_nodes, es = s->esize, S = pop_slots(s->mesh);
    std::vector<unsigned char> buf(18 * pad4(S) * es);
    cudaError_t e = cudaMemcpyAsync(buf.data(), s->f[s->cur], buf.size(), cudaMemcpyDeviceToHost,
                                    s->mesh->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->mesh->stream);
    if (e != cudaSuccess) return cuda_status(e);
    const bool perm = s->mesh->kind == 0;
    for (int a = 0; a < 18; ++a)
        for (size_t k = 0; k < N; ++k) {
            const size_t c = perm ? (size_t)s->mesh->host.perm[k] : k;
            const size_t q = pop_index(a, pop_slot(s->mesh, k), S);
            const double v = es == 8 ? reinterpret_cast<double *>(buf.data())[q]
                                     : (double)reinterpret_cast<float *>(buf.data())[q];
            (a < 9 ? hbar : gbar)[(a % 9) * N + c] = v;
        }
    return check_flag(s);
}

int felbm_state_import(felbm_state *s, const double *hbar, const double *gbar) {
    if (!s || !hbar || !gbar) return FELBM_ERR_INVALID_ARG;
    if (s->mesh->kind >= 2) return import3(s, hbar, gbar);
    const size_t N = (size_t)s->mesh->n_nodes, es = s->esize, S = pop_slots(s->mesh);
    std::vector<unsigned char> buf(18 * pad4(S) * es, 0);
    const bool perm = s->mesh->kind == 0;
    for (int a = 0; a < 18; ++a)
        for (size_t k = 0; k < N; ++k) {
            const size_t c = perm ? (size_t)s->mesh->host.perm[k] : k;
            const double v = (a < 9 ? hbar : gbar)[(a % 9) * N + c];
            if (!std::isfinite(v)) return FELBM_ERR_INVALID_ARG;
            const size_t q = pop_index(a, pop_slot(s->mesh, k), S);
            if (es == 8)
                reinterpret_cast<double *>(buf.data())[q] = v;
            else
                reinterpret_cast<float *>(buf.data())[q] = (float)v;
        }
    cudaError_t e = cudaMemcpyAsync(s->f[s->cur], buf.data(), buf.size(), cudaMemcpyHostToDevice,
                                    s->mesh->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_flag, 0, sizeof(int), s->mesh->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->mesh->stream);
    if (e != cudaSuccess) return cuda_status(e);
    s->have_moments = false;
    return FELBM_OK;
}

void felbm_state_destroy(felbm_state *s) {
    if (!s) return;
    cudaStreamSynchronize(s->mesh->stream);
    state_free(s);
}

int felbm_profile_enable(felbm_state *s, int on) {
    if (!s || on < 0) return FELBM_ERR_INVALID_ARG;
    if (on && s->prof_ev.empty()) {
        try {
            s->prof_ev.assign(2 * kProfMaxLaunches, nullptr);
            s->prof_kind.assign(kProfMaxLaunches, 0);
        } catch (const std::bad_alloc &) {
            return FELBM_ERR_OOM;
        }
        for (auto &e : s->prof_ev) {
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return cuda_status(r);
        }
    }
    s->prof_on = on != 0;
    s->prof_stride = on > 0 ? on : 1;
    s->prof_used = 0;
    for (auto &c : s->launches) c = 0;
    for (auto &c : s->prof_seen) c = 0;
    return FELBM_OK;
}

int felbm_profile_read(felbm_state *s, double *ms, int64_t *timed, int64_t *launches) {
    if (!s) return FELBM_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(s->mesh->stream);
    if (e != cudaSuccess) return cuda_status(e);
    double acc[8] = {0};
    int64_t cnt[8] = {0};
    for (size_t k = 0; k < s->prof_used; ++k) {
        float t = 0.f;
        e = cudaEventElapsedTime(&t, s->prof_ev[2 * k], s->prof_ev[2 * k + 1]);
        if (e != cudaSuccess) return cuda_status(e);
        acc[s->prof_kind[k]] += t;
        cnt[s->prof_kind[k]]++;
    }
    for (int k = 0; k < FELBM_PROFILE_KINDS; ++k) {
        if (ms) ms[k] = acc[k];
        if (timed) timed[k] = cnt[k];
        if (launches) launches[k] = s->launches[k];
        s->launches[k] = 0;
    }
    s->prof_used = 0;
    return FELBM_OK;
}

const char *felbm_profile_kind_name(int k) {
    static const char *names[FELBM_PROFILE_KINDS] = {
        "k_rho", "k_grad", "k_mu", "k_collide", "k_lattice_step", "k_patch_step", "unused6",
        "unused7"};
    return (k >= 0 && k < FELBM_PROFILE_KINDS) ? names[k] : nullptr;
}

}  // extern "C"
