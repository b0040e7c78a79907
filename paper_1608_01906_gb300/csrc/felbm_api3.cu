// C ABI on tetrahedral meshes (D3Q19; kind 2 general CSR, kind 3 Kuhn
// lattice): mesh creation and the per-state work the common entry points of
// felbm_api.cu hand over here.
#include <cmath>
#include <new>
#include <type_traits>
#include <vector>

#include "felbm_internal.h"
#include "felbm_kernels.cuh"
#include "felbm_kernels3.cuh"

namespace felbm {

static inline unsigned nblocks3(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// Storage index of population a (D3Q19 order) of node i: rest at [0, S),
// pair q = (2q+1, 2q+2) at Np + 2 Np q + 2 i + slot; g from 19 Np.
static size_t pop_index3(int a, size_t i, size_t n) {
    const size_t np = pad4(n);
    const size_t base = a < 19 ? 0 : 19 * np;
    const int d = a % 19;
    if (d == 0) return base + i;
    const int q = (d - 1) / 2, slot = (d - 1) % 2;
    return base + np + 2 * np * (size_t)q + 2 * i + (size_t)slot;
}

template <typename T>
static DevCSR3<T> dev_csr3(const felbm_mesh *m) {
    DevCSR3<T> d;
    d.n = (int32_t)m->n_nodes;
    d.rowptr = m->d_rowptr;
    d.col = m->d_col;
    const size_t nnz = m->host3.col.size();
    const T *base = sizeof(T) == 8 ? reinterpret_cast<const T *>(m->d_coef64)
                                   : reinterpret_cast<const T *>(m->d_coef32);
    for (int k = 0; k < 9; ++k) d.c[k] = base + (size_t)k * nnz;
    d.tag = m->d_tag;
    return d;
}

template <typename T>
static DevLattice3<T> dev_lat3(const felbm_mesh *m, double dt) {
    const Lattice3Info &L = m->linfo3;
    DevLattice3<T> d;
    d.n = (int32_t)m->n_nodes;
    d.nx = L.nx;
    d.ny = L.ny;
    d.nz = L.nz;
    d.walls = L.walls ? 1 : 0;
    const double hdt = 0.5 * dt;
    for (int k = 0; k < 3; ++k)
        for (int o = 0; o < 14; ++o) {
            const double *cf = L.c[k][o];
            for (int q = 0; q < 9; ++q) {
                const int a = 2 * q + 1;
                const double ex = e3x(a), ey = e3y(a), ez = e3z(a);
                const double odd = ex * cf[0] + ey * cf[1] + ez * cf[2];
                const double even = hdt * ((ex * ex * cf[3] + ey * ey * cf[6] + ez * ez * cf[8]) +
                                           2.0 * (ex * ey * cf[4] + ex * ez * cf[5] + ey * ez * cf[7]));
                d.k.pc[k][o][q].x = (T)(even + odd);
                d.k.pc[k][o][q].y = (T)(even - odd);
            }
            for (int c = 0; c < 3; ++c) d.k.a[k][o][c] = (T)cf[c];
        }
    return d;
}

template <typename T>
static Phys3<T> phys3_of(const felbm_params &p) {
    const double dd = p.rho_l - p.rho_v;
    Phys3<T> P;
    P.rho_l = (T)p.rho_l;
    P.rho_v = (T)p.rho_v;
    P.beta = (T)(12.0 * p.sigma / (p.xi * dd * dd * dd * dd));
    P.kappa = (T)(1.5 * p.xi * p.sigma / (dd * dd));
    P.inv_tau_l = (T)(1.0 / p.tau_l);
    P.inv_tau_v = (T)(1.0 / p.tau_v);
    P.dt = (T)p.dt;
    for (int k = 0; k < 3; ++k) P.g[k] = (T)p.gravity[k];
    P.inv_drho = (T)(1.0 / dd);
    return P;
}

// Scratch layout (19 Np + 9 N): streamed h*, grad rho (4 N interleaved,
// 16-byte aligned since Np is a multiple of 4), rho, mu, K (3).
template <typename T>
static Fields3<T> fields3_of(felbm_state *s) {
    const size_t n = (size_t)s->mesh->n_nodes;
    Fields3<T> F;
    F.hs = reinterpret_cast<T *>(s->scratch);
    F.dr4 = F.hs + 19 * pad4(n);
    T *b = F.dr4 + 4 * n;
    F.rho = b;
    F.mu = b + n;
    for (int k = 0; k < 3; ++k) F.k[k] = b + (2 + k) * n;
    return F;
}

// grad rho, then lap rho, K and mu, from F.rho.
template <typename T, typename Topo>
static void chain3(felbm_state *s, const Topo &d, const Fields3<T> &F, const Phys3<T> &P) {
    const felbm_mesh *m = s->mesh;
    const unsigned g = nblocks3(m->n_nodes, 256);
    int sl = prof_begin(s, 1);
    k_grad3<T, Topo><<<g, 256, 0, m->stream>>>(d, F);
    prof_end(s, sl);
    sl = prof_begin(s, 2);
    k_mu3<T, Topo><<<g, 256, 0, m->stream>>>(d, F, P);
    prof_end(s, sl);
}

// Calls fn(topology) with the device view of the state's mesh.
template <typename T, typename Fn>
static void with_topo(felbm_state *s, Fn &&fn) {
    if (s->mesh->kind == 3)
        fn(dev_lat3<T>(s->mesh, s->params.dt));
    else
        fn(dev_csr3<T>(s->mesh));
}

template <typename T>
static void init3(felbm_state *s) {
    with_topo<T>(s, [&](const auto &d) {
        using Topo = std::decay_t<decltype(d)>;
        const felbm_mesh *m = s->mesh;
        const Fields3<T> F = fields3_of<T>(s);
        const Phys3<T> P = phys3_of<T>(s->params);
        cudaMemcpyAsync(F.rho, s->mom, (size_t)m->n_nodes * sizeof(T), cudaMemcpyDeviceToDevice, m->stream);
        chain3<T>(s, d, F, P);
        k_init3<T, Topo><<<nblocks3(m->n_nodes, 128), 128, 0, m->stream>>>(
            d, reinterpret_cast<T *>(s->f[s->cur]), F, P, reinterpret_cast<const T *>(s->mom));
    });
}

template <typename T, typename Topo>
static void step3(felbm_state *s, const Topo &d, const Fields3<T> &F, const Phys3<T> &P, bool write_mom) {
    const felbm_mesh *m = s->mesh;
    const T *fin = reinterpret_cast<const T *>(s->f[s->cur]);
    T *fout = reinterpret_cast<T *>(s->f[s->cur ^ 1]);
    int sl = prof_begin(s, 0);
    k_rho3<T, Topo><<<nblocks3(m->n_nodes, 256), 256, 0, m->stream>>>(d, fin, P.dt, F.rho, F.hs);
    prof_end(s, sl);
    chain3<T>(s, d, F, P);
    Collide3Args<T, Topo> A;
    A.m = d;
    A.fin = fin;
    A.fout = fout;
    A.F = F;
    A.P = P;
    A.mom = write_mom ? reinterpret_cast<T *>(s->mom) : nullptr;
    A.flag = s->d_flag;
    sl = prof_begin(s, 3);
    k_collide3<T, Topo><<<nblocks3(m->n_nodes, 128), 128, 0, m->stream>>>(A);
    prof_end(s, sl);
    s->cur ^= 1;
}

template <typename T>
static void steps3_t(felbm_state *s, int64_t n) {
    with_topo<T>(s, [&](const auto &d) {
        const Fields3<T> F = fields3_of<T>(s);
        const Phys3<T> P = phys3_of<T>(s->params);
        for (int64_t k = 0; k < n; ++k) step3<T>(s, d, F, P, k == n - 1);
    });
}

void steps3(felbm_state *s, int64_t n) {
    if (s->esize == 8)
        steps3_t<double>(s, n);
    else
        steps3_t<float>(s, n);
}

int state_init3(const felbm_mesh *mesh, const felbm_params *params, const double *rho0,
                const double *u0, const double *p0, felbm_state **out) {
    if (params->flags & FELBM_PARAM_LAP_FP64) return FELBM_ERR_UNSUPPORTED;
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
    alloc(&s->f[0], 38 * pad4(N) * es);
    alloc(&s->f[1], 38 * pad4(N) * es);
    alloc(&s->scratch, (19 * pad4(N) + 9 * N) * es);
    alloc(&s->mom, 5 * N * es);
    alloc((void **)&s->d_out, (6 * N + 4 * (kTotalsBlocks + 1)) * sizeof(double));
    alloc((void **)&s->d_flag, sizeof(int));
    if (e != cudaSuccess) {
        const int rs = cuda_status(e);
        state_free(s);
        return rs;
    }
    // initial moments (rho, ux, uy, uz, p) in internal order and precision
    std::vector<unsigned char> hm(5 * N * es);
    for (size_t k = 0; k < N; ++k) {
        const size_t c = (size_t)mesh->host3.perm[k];
        const double v[5] = {rho0[c], u0 ? u0[3 * c] : 0.0, u0 ? u0[3 * c + 1] : 0.0,
                             u0 ? u0[3 * c + 2] : 0.0, p0 ? p0[c] : 0.0};
        for (int q = 0; q < 5; ++q) {
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
    for (int c = 0; c < 2 && e == cudaSuccess; ++c)
        e = cudaMemsetAsync(s->f[c], 0, 38 * pad4(N) * es, mesh->stream);
    if (e == cudaSuccess) {
        if (es == 8)
            init3<double>(s);
        else
            init3<float>(s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(mesh->stream);  // hm is a temporary
    if (e != cudaSuccess) {
        const int rs = cuda_status(e);
        state_free(s);
        return rs;
    }
    s->have_moments = true;
    *out = s;
    return FELBM_OK;
}

template <typename T>
static void launch_moments3(felbm_state *s) {
    const felbm_mesh *m = s->mesh;
    const int32_t n = (int32_t)m->n_nodes;
    k_gather_moments3<T><<<nblocks3(n, 256), 256, 0, m->stream>>>(
        n, reinterpret_cast<const T *>(s->mom), m->d_perm + n, s->params.rho_l, s->params.rho_v, s->d_out);
    double *part = s->d_out + 6 * (size_t)n;
    k_totals3_partial<T><<<kTotalsBlocks, 256, 0, m->stream>>>(n, reinterpret_cast<const T *>(s->mom),
                                                               m->d_mass, part);
    k_totals3_final<<<1, 32, 0, m->stream>>>(kTotalsBlocks, part, part + 4 * kTotalsBlocks);
}

int moments3(felbm_state *s, double *rho, double *C, double *u, double *p, double *totals) {
    const size_t N = (size_t)s->mesh->n_nodes;
    const cudaStream_t st = s->mesh->stream;
    if (s->esize == 8)
        launch_moments3<double>(s);
    else
        launch_moments3<float>(s);
    cudaError_t e = cudaGetLastError();
    const double *o = s->d_out;
    if (e == cudaSuccess && rho) e = cudaMemcpyAsync(rho, o, N * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && C) e = cudaMemcpyAsync(C, o + N, N * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && u) e = cudaMemcpyAsync(u, o + 2 * N, 3 * N * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && p) e = cudaMemcpyAsync(p, o + 5 * N, N * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && totals)
        e = cudaMemcpyAsync(totals, o + 6 * N + 4 * kTotalsBlocks, 4 * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return cuda_status(e);
}

int export3(felbm_state *s, double *hbar, double *gbar) {
    const size_t N = (size_t)s->mesh->n_nodes, es = s->esize;
    std::vector<unsigned char> buf(38 * pad4(N) * es);
    cudaError_t e = cudaMemcpyAsync(buf.data(), s->f[s->cur], buf.size(), cudaMemcpyDeviceToHost,
                                    s->mesh->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->mesh->stream);
    if (e != cudaSuccess) return cuda_status(e);
    for (int a = 0; a < 38; ++a)
        for (size_t k = 0; k < N; ++k) {
            const size_t c = (size_t)s->mesh->host3.perm[k];
            const size_t q = pop_index3(a, k, N);
            const double v = es == 8 ? reinterpret_cast<double *>(buf.data())[q]
                                     : (double)reinterpret_cast<float *>(buf.data())[q];
            (a < 19 ? hbar : gbar)[(a % 19) * N + c] = v;
        }
    return FELBM_OK;
}

int import3(felbm_state *s, const double *hbar, const double *gbar) {
    const size_t N = (size_t)s->mesh->n_nodes, es = s->esize;
    std::vector<unsigned char> buf(38 * pad4(N) * es, 0);
    for (int a = 0; a < 38; ++a)
        for (size_t k = 0; k < N; ++k) {
            const size_t c = (size_t)s->mesh->host3.perm[k];
            const double v = (a < 19 ? hbar : gbar)[(a % 19) * N + c];
            if (!std::isfinite(v)) return FELBM_ERR_INVALID_ARG;
            const size_t q = pop_index3(a, k, N);
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

FELBM_CHECK_READER(check_bits_api3)

}  // namespace felbm

using namespace felbm;

extern "C" int felbm_mesh_create_tet(const double *xyz, int64_t n_nodes, const int32_t *tet, int64_t n_tet,
                                     const double box[3], uint32_t flags, const uint8_t *node_tag,
                                     void *stream, felbm_mesh **out) {
    if (!xyz || !tet || !box || !out) return FELBM_ERR_INVALID_ARG;
    if (n_nodes < 4 || n_tet < 1 || n_nodes > 0x7fffffffLL || n_tet > 0x7fffffffLL / 4)
        return FELBM_ERR_INVALID_ARG;
    if (flags & ~(FELBM_PERIODIC_X | FELBM_PERIODIC_Y | FELBM_PERIODIC_Z | FELBM_MESH_GENERAL))
        return FELBM_ERR_INVALID_ARG;
    felbm_mesh *m = new (std::nothrow) felbm_mesh();
    if (!m) return FELBM_ERR_OOM;
    m->n_nodes = n_nodes;
    m->n_tri = n_tet;
    m->flags = flags;
    m->stream = reinterpret_cast<cudaStream_t>(stream);
    m->kind = 2;
    int st = FELBM_OK;
    try {
        st = build_csr3(xyz, n_nodes, tet, n_tet, box, flags, node_tag, m->host3);
    } catch (const std::bad_alloc &) {
        st = FELBM_ERR_OOM;
    }
    if (st != FELBM_OK) {
        delete m;
        return st;
    }
    HostCSR3 &H = m->host3;
    if (!(flags & FELBM_MESH_GENERAL)) detect_lattice3(xyz, n_nodes, box, flags, node_tag, H, m->linfo3);
    if (m->linfo3.ok) {
        // the lattice kernels take neighbours and coefficients from the node
        // position: natural order, no assembled arrays on the device
        m->kind = 3;
        std::vector<double> mass(H.n);
        for (int32_t c = 0; c < H.n; ++c) {
            mass[c] = H.mass[H.iperm[c]];
            H.perm[c] = H.iperm[c] = c;
        }
        H.mass.swap(mass);
        std::vector<int32_t>().swap(H.col);
        std::vector<double>().swap(H.coef);
        std::vector<uint8_t>().swap(H.tag);
    }
    const size_t N = (size_t)n_nodes, nnz = H.col.size();
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) {
            e = cudaMalloc(p, bytes);
            if (e == cudaSuccess) m->device_bytes += (int64_t)bytes;
        }
    };
    const bool csr = m->kind == 2;
    alloc((void **)&m->d_mass, N * sizeof(double));
    alloc((void **)&m->d_perm, 2 * N * sizeof(int32_t));
    if (csr) {
        alloc((void **)&m->d_rowptr, (N + 1) * sizeof(int32_t));
        alloc((void **)&m->d_col, nnz * sizeof(int32_t));
        alloc((void **)&m->d_coef64, 9 * nnz * sizeof(double));
        alloc((void **)&m->d_coef32, 9 * nnz * sizeof(float));
        if (!H.tag.empty()) alloc((void **)&m->d_tag, N);
    }
    std::vector<float> c32;
    try {
        c32.resize(9 * nnz);
    } catch (const std::bad_alloc &) {
        e = cudaErrorMemoryAllocation;
    }
    for (size_t q = 0; q < c32.size(); ++q) c32[q] = (float)H.coef[q];
    if (e == cudaSuccess) e = cudaMemcpy(m->d_mass, H.mass.data(), N * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && csr)
        e = cudaMemcpy(m->d_rowptr, H.rowptr.data(), (N + 1) * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && csr)
        e = cudaMemcpy(m->d_col, H.col.data(), nnz * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_perm, H.perm.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(m->d_perm + N, H.iperm.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && csr)
        e = cudaMemcpy(m->d_coef64, H.coef.data(), 9 * nnz * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && csr)
        e = cudaMemcpy(m->d_coef32, c32.data(), 9 * nnz * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && m->d_tag) e = cudaMemcpy(m->d_tag, H.tag.data(), N, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        const int rs = cuda_status(e);
        mesh_free(m);
        return rs;
    }
    *out = m;
    return FELBM_OK;
}
