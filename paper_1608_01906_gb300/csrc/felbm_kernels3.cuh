// Device kernels of one FE-LBM time step on tetrahedral meshes (D3Q19, the
// paper's own setting), on two topologies: the general CSR (DevCSR3) and the
// Kuhn-split cube lattice (DevLattice3).  Same four dependent passes as the
// two-dimensional general path (felbm_kernels.cuh):
//   k_rho3      Taylor-Galerkin streaming of the 19 h populations (Sec.
//               2.2.1, lumped mass), wall bounce-back, rho = sum_a h_a; the
//               streamed h* is kept for the collision;
//   k_grad3     recovered grad rho (Sec. 2.3);
//   k_mu3       Laplacian of rho, the stress force
//               K_i = kappa [d_i |grad rho|^2 - d_j (d_i rho d_j rho)] and
//               mu = mu_phi(rho) - kappa lap rho (Sec. 2.1);
//   k_collide3  recovered grad mu, streaming of the 19 g populations,
//               bounce-back, moments (Eqs. velocity, pressure) and the
//               post- and next pre-streaming collision (Sec. 2.2).
// D3Q19 directions are ordered so that 2q+1 and 2q+2 are opposite (q =
// 0..8); the populations are stored as the rest value plus 9 interleaved
// opposite pairs (pop layout of felbm_internal.h with 19 per distribution).
#pragma once

#include <type_traits>

#include "felbm_internal.h"
#include "felbm_kernels.cuh"

namespace felbm {

// D3Q19: rest, +-x, +-y, +-z, then the 12 edge directions in opposite pairs.
__host__ __device__ constexpr int e3x(int a) {
    return (a == 1 || a == 7 || a == 9 || a == 11 || a == 13) ? 1
           : (a == 2 || a == 8 || a == 10 || a == 12 || a == 14) ? -1 : 0;
}
__host__ __device__ constexpr int e3y(int a) {
    return (a == 3 || a == 7 || a == 10 || a == 15 || a == 17) ? 1
           : (a == 4 || a == 8 || a == 9 || a == 16 || a == 18) ? -1 : 0;
}
__host__ __device__ constexpr int e3z(int a) {
    return (a == 5 || a == 11 || a == 14 || a == 15 || a == 18) ? 1
           : (a == 6 || a == 12 || a == 13 || a == 16 || a == 17) ? -1 : 0;
}
template <typename T>
__host__ __device__ constexpr T w3(int a) {
    return a == 0 ? T(1) / T(3) : (a <= 6 ? T(1) / T(18) : T(1) / T(36));
}

// 3 w_a of D3Q19 in the working precision with the moment identities exact
// in T (see kW3): sum_a 3 w_a = 3 (w3_0 + 6 w3_1 + 12 w3_7) and
// sum_a 3 w_a e_ax^2 = 1 (2 w3_1 + 8 w3_7), from e ~ 1/12 (kTwelfth):
// w3_7 = e, w3_1 = (1 - 8 e)/2, w3_0 = 12 e.
template <typename T>
__host__ __device__ constexpr T w3x3(int a) {
    return a == 0 ? T(12) * kTwelfth<T>() : (a <= 6 ? (T(1) - T(8) * kTwelfth<T>()) / T(2) : kTwelfth<T>());
}

// Model constants of one state (Sec. 2.1) with three-component gravity.
template <typename T>
struct Phys3 {
    T rho_l, rho_v, beta, kappa, inv_tau_l, inv_tau_v, dt, g[3];
    T inv_drho;  // 1 / (rho_l - rho_v)
};

template <typename T>
__device__ __forceinline__ T mu_bulk3(const Phys3<T> &P, T r) {
    return T(4) * P.beta * (r - P.rho_v) * (r - P.rho_l) * (r - T(0.5) * (P.rho_v + P.rho_l));
}

// General tetrahedral mesh: CSR in reverse Cuthill-McKee order with the
// coefficient arrays of HostCSR3 (a: 3, b: 6 symmetric components).
// Both topologies give, for node i, the neighbours j with their
// coefficients: for_each<K>(i, fn(j, a)) with a = (a_x, a_y, a_z) at least,
// for_each_pair<K>(i, dt/2, fn(j, c)) with c[q] = (e.a + dt/2 e.b.e) for the
// pair q = (2q+1, 2q+2) as (first, second) = (even + odd, even - odd) parts.
// K >= 0 promises that node i is of z-layer kind K (lattice only; -1 = any).
template <typename T>
struct DevCSR3 {
    static constexpr bool kLattice = false;
    int32_t n;
    const int32_t *rowptr;
    const int32_t *col;
    const T *c[9];       // ax, ay, az, bxx, bxy, bxz, byy, byz, bzz (nnz each)
    const uint8_t *tag;  // nullptr if no walls
#ifdef __CUDACC__
    template <int K, typename Fn>
    __device__ __forceinline__ void for_each(int32_t i, Fn &&fn) const {
        const int32_t p1 = __ldg(rowptr + i + 1);
        for (int32_t p = __ldg(rowptr + i); p < p1; ++p) {
            const int32_t j = __ldg(col + p);
            if (!chk_idx(j, n, 1u)) continue;
            T cf[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) cf[k] = __ldg(c[k] + p);
            fn(j, cf);
        }
    }
    template <int K, typename Fn>
    __device__ __forceinline__ void for_each_pair(int32_t i, T hdt, Fn &&fn) const {
        for_each<K>(i, [&](int32_t j, const T *cf) {
            V2<T> c[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const int a = 2 * q + 1;
                const T ex = T(e3x(a)), ey = T(e3y(a)), ez = T(e3z(a));
                const T odd = ex * cf[0] + ey * cf[1] + ez * cf[2];
                const T even = hdt * ((ex * ex * cf[3] + ey * ey * cf[6] + ez * ez * cf[8]) +
                                      T(2) * (ex * ey * cf[4] + ex * ez * cf[5] + ey * ez * cf[7]));
                c[q] = vset(even + odd, even - odd);
            }
            fn(j, c);
        });
    }
    __device__ __forceinline__ int kind_of(int32_t) const { return -1; }
    __device__ __forceinline__ int tag_of(int32_t i) const { return tag ? (int)tag[i] : 0; }
#endif
};

// Coefficients of the Kuhn lattice per z-layer kind (0 interior, 1 bottom
// wall layer, 2 top wall layer) and neighbour offset o (lat3_d*(o)), passed
// as kernel parameters: the pair form of the streaming coefficients with
// dt/2 folded in, and the recovery coefficients a_ij.
template <typename T>
struct Lat3Coef {
    V2<T> pc[3][14][9];
    T a[3][14][3];
};

// Kuhn-split cube lattice in natural order (i = x + nx (y + ny z)): the 14
// neighbour ids follow from the node's position; a walled z direction has
// tags 5 (bottom layer, inward normal +z) and 6 (top layer).
template <typename T>
struct DevLattice3 {
    static constexpr bool kLattice = true;
    int32_t n, nx, ny, nz;
    int32_t walls;
    Lat3Coef<T> k;
#ifdef __CUDACC__
    __device__ __forceinline__ int kind_of(int32_t i) const {
        if (!walls) return 0;
        const int32_t z = i / (nx * ny);
        return z == 0 ? 1 : (z == nz - 1 ? 2 : 0);
    }
    __device__ __forceinline__ int tag_of(int32_t i) const {
        const int kd = kind_of(i);
        return kd == 0 ? 0 : 4 + kd;
    }
    // Where an offset leaves a walled domain its coefficients are zero and
    // the id is an in-range stand-in (the wrapped x-y neighbour in-layer).
    __device__ __forceinline__ void nbrs(int32_t i, int32_t *j) const {
        const int32_t L = nx * ny;
        const int32_t z = i / L, r = i - z * L, y = r / nx, x = r - y * nx;
        const int32_t xp = x == nx - 1 ? 1 - nx : 1, xm = x == 0 ? nx - 1 : -1;
        const int32_t yp = (y == ny - 1 ? 1 - ny : 1) * nx, ym = (y == 0 ? ny - 1 : -1) * nx;
        int32_t zp, zm;
        if (walls) {
            zp = z == nz - 1 ? 0 : L;
            zm = z == 0 ? 0 : -L;
        } else {
            zp = (z == nz - 1 ? 1 - nz : 1) * L;
            zm = (z == 0 ? nz - 1 : -1) * L;
        }
#pragma unroll
        for (int o = 0; o < 14; ++o)
            j[o] = i + (lat3_dx(o) > 0 ? xp : (lat3_dx(o) < 0 ? xm : 0)) +
                   (lat3_dy(o) > 0 ? yp : (lat3_dy(o) < 0 ? ym : 0)) +
                   (lat3_dz(o) > 0 ? zp : (lat3_dz(o) < 0 ? zm : 0));
    }
    template <int K, typename Fn>
    __device__ __forceinline__ void for_each(int32_t i, Fn &&fn) const {
        int32_t j[14];
        nbrs(i, j);
        const int kd = K >= 0 ? K : kind_of(i);
#pragma unroll
        for (int o = 0; o < 14; ++o)
            if (chk_idx(j[o], n, 1u)) fn(j[o], k.a[kd][o]);
    }
    template <int K, typename Fn>
    __device__ __forceinline__ void for_each_pair(int32_t i, T, Fn &&fn) const {
        int32_t j[14];
        nbrs(i, j);
        const int kd = K >= 0 ? K : kind_of(i);
#pragma unroll
        for (int o = 0; o < 14; ++o)
            if (chk_idx(j[o], n, 1u)) fn(j[o], k.pc[kd][o]);
    }
#endif
};

#ifdef __CUDACC__
// Runs fn(integral_constant<K>) with K = 0 for interior lattice nodes (the
// coefficients are then compile-time parameter offsets) and K = -1 otherwise.
template <typename Topo, typename Fn>
__device__ __forceinline__ void by_kind(const Topo &m, int32_t i, Fn &&fn) {
    if constexpr (Topo::kLattice) {
        if (m.kind_of(i) == 0) {
            fn(std::integral_constant<int, 0>());
            return;
        }
    }
    fn(std::integral_constant<int, -1>());
}
#endif

// Fields of one time level: rho, mu, K (N each); grad rho interleaved as
// (x, y, z, unused) per node (4 N, 16-byte aligned), so that one gather
// reads a neighbour's gradient; and the streamed, bounced-back h* of k_rho3
// (19 values per node, population layout: rest at [0, Np), pair q at
// Np + 2 Np q).
template <typename T>
struct Fields3 {
    T *rho, *dr4, *mu, *k[3];
    T *hs;
};

#ifdef __CUDACC__
template <typename T>
__device__ __forceinline__ void load_grad3(const T *__restrict__ dr4, int32_t j, T *g) {
    if constexpr (sizeof(T) == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(dr4) + j);
        g[0] = v.x;
        g[1] = v.y;
        g[2] = v.z;
    } else {
        const double2 *p = reinterpret_cast<const double2 *>(dr4) + 2 * (size_t)j;
        const double2 a = __ldg(p), b = __ldg(p + 1);
        g[0] = a.x;
        g[1] = a.y;
        g[2] = b.x;
    }
}

template <typename T>
__device__ __forceinline__ void store_grad3(T *__restrict__ dr4, int32_t i, const T *g) {
    if constexpr (sizeof(T) == 4) {
        reinterpret_cast<float4 *>(dr4)[i] = make_float4(g[0], g[1], g[2], 0.0f);
    } else {
        double2 *p = reinterpret_cast<double2 *>(dr4) + 2 * (size_t)i;
        p[0] = make_double2(g[0], g[1]);
        p[1] = make_double2(g[2], 0.0);
    }
}
#endif

// Streamed values of pairs Q0 .. Q0+NQ-1 of one distribution of node i
// (base: its rest values; pair q at base + Np + 2 Np q):
// psi* = psi - dt sum_j (e.a_ij + dt/2 e.b_ij.e) (psi_j - psi_i).
template <typename T, int Q0, int NQ, int K, typename Topo>
__device__ __forceinline__ void stream_range3(const Topo &m, const T *__restrict__ base, size_t np, int32_t i,
                                              T dt, V2<T> *out) {
    const V2<T> *pb = reinterpret_cast<const V2<T> *>(base + np);
    const V2<T> m1 = vset(T(-1), T(-1));
    V2<T> own[NQ], acc[NQ];
#pragma unroll
    for (int r = 0; r < NQ; ++r) {
        own[r] = pb[(Q0 + r) * np + i];
        acc[r] = vset(T(0), T(0));
    }
    m.template for_each_pair<K>(i, T(0.5) * dt, [&](int32_t j, const V2<T> *c) {
#pragma unroll
        for (int r = 0; r < NQ; ++r)
            acc[r] = vfma(c[Q0 + r], vfma(own[r], m1, __ldg(pb + (Q0 + r) * np + j)), acc[r]);
    });
    const V2<T> mdt = vset(-dt, -dt);
#pragma unroll
    for (int r = 0; r < NQ; ++r) out[r] = vfma(mdt, acc[r], own[r]);
}

// The 9 streamed pairs in two passes over the neighbours (5 + 4 pairs):
// fewer live registers per thread, more threads per SM.
template <typename T, int K, typename Topo>
__device__ __forceinline__ void stream_all3(const Topo &m, const T *__restrict__ base, size_t np, int32_t i,
                                            T dt, V2<T> *out) {
    stream_range3<T, 0, 5, K>(m, base, np, i, dt, out);
    stream_range3<T, 5, 4, K>(m, base, np, i, dt, out + 5);
}

template <typename T>
__device__ __forceinline__ void unpack3(T rest, const V2<T> *p, T *psi) {
    psi[0] = rest;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        psi[2 * q + 1] = p[q].x;
        psi[2 * q + 2] = p[q].y;
    }
}

// Bounce-back at a wall node with inward normal e_k: every population with
// e_a . e_k > 0 takes the value of its opposite.
template <typename T>
__device__ __forceinline__ void bounce_back3(int k, T *psi) {
    const int kx = e3x(k), ky = e3y(k), kz = e3z(k);
#pragma unroll
    for (int a = 1; a < 19; ++a)
        if (e3x(a) * kx + e3y(a) * ky + e3z(a) * kz > 0) psi[a] = psi[a % 2 ? a + 1 : a - 1];
}

// Bounce-back of pair q = (a, a+1), a = 2q+1, at a wall node with inward
// normal e_k: the member with e . e_k > 0 takes the value of the other
// (bounce_back3 on one pair).
template <typename T>
__device__ __forceinline__ void bounce_pair3(int k, int q, V2<T> &p) {
    const int a = 2 * q + 1;
    const int d = e3x(a) * e3x(k) + e3y(a) * e3y(k) + e3z(a) * e3z(k);
    if (d > 0)
        p.x = p.y;
    else if (d < 0)
        p.y = p.x;
}

template <typename T, typename Topo>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 1) k_rho3(const __grid_constant__ Topo m, const T *__restrict__ f, T dt,
                                              T *__restrict__ rho, T *__restrict__ hs) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.n) return;
    const size_t np = pad4((size_t)m.n);
    V2<T> hp[9];
    by_kind(m, i, [&](auto K) { stream_all3<T, decltype(K)::value>(m, f, np, i, dt, hp); });
    T h[19];
    unpack3<T>(f[i], hp, h);
    const int k = m.tag_of(i);
    if (k) bounce_back3<T>(k, h);
    T r = T(0);
#pragma unroll
    for (int a = 0; a < 19; ++a) r += h[a];
    rho[i] = r;
    V2<T> *hb = reinterpret_cast<V2<T> *>(hs + np);
#pragma unroll
    for (int q = 0; q < 9; ++q) hb[q * np + i] = vset(h[2 * q + 1], h[2 * q + 2]);
    hs[i] = h[0];
}

// Recovered gradient of a scalar field (3 components).
template <typename T, int K, typename Topo>
__device__ __forceinline__ void recover3(const Topo &m, const T *__restrict__ f, int32_t i, T *g) {
    const T fi = f[i];
    T s0 = T(0), s1 = T(0), s2 = T(0);
    m.template for_each<K>(i, [&](int32_t j, const T *cf) {
        const T d = __ldg(f + j) - fi;
        s0 += cf[0] * d;
        s1 += cf[1] * d;
        s2 += cf[2] * d;
    });
    g[0] = s0;
    g[1] = s1;
    g[2] = s2;
}

template <typename T, typename Topo>
__global__ void __launch_bounds__(256) k_grad3(const __grid_constant__ Topo m, Fields3<T> F) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.n) return;
    T g[3];
    by_kind(m, i, [&](auto K) { recover3<T, decltype(K)::value>(m, F.rho, i, g); });
    store_grad3<T>(F.dr4, i, g);
}

// lap rho = sum_c R_c(d_c rho);
// K_i = kappa [sum_{k != i} R_i((d_k rho)^2) - sum_{j != i} R_j(d_i rho d_j rho)]
// (the printed form with the identical (d_i rho)^2 contributions cancelled);
// differences of the products in product form.
template <typename T, int K, typename Topo>
__device__ __forceinline__ void mu_sums3(const Topo &m, const Fields3<T> &F, int32_t i, const T *gi, T &lap,
                                         T *K3) {
    m.template for_each<K>(i, [&](int32_t j, const T *cf) {
        T gj[3], d[3];
        load_grad3<T>(F.dr4, j, gj);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            d[c] = gj[c] - gi[c];
            lap += cf[c] * d[c];
        }
        T sq[3];  // differences of (d_c rho)^2
#pragma unroll
        for (int c = 0; c < 3; ++c) sq[c] = d[c] * (gj[c] + gi[c]);
        // differences of d_a rho d_b rho (a < b), each formed once
        const T pxy = gj[0] * d[1] + gi[1] * d[0];
        const T pxz = gj[0] * d[2] + gi[2] * d[0];
        const T pyz = gj[1] * d[2] + gi[2] * d[1];
        K3[0] += cf[0] * (sq[1] + sq[2]) - (cf[1] * pxy + cf[2] * pxz);
        K3[1] += cf[1] * (sq[0] + sq[2]) - (cf[0] * pxy + cf[2] * pyz);
        K3[2] += cf[2] * (sq[0] + sq[1]) - (cf[0] * pxz + cf[1] * pyz);
    });
}

template <typename T, typename Topo>
__global__ void __launch_bounds__(256) k_mu3(const __grid_constant__ Topo m, Fields3<T> F, Phys3<T> P) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.n) return;
    T gi[3];
    load_grad3<T>(F.dr4, i, gi);
    T lap = T(0), K[3] = {T(0), T(0), T(0)};
    by_kind(m, i, [&](auto KD) { mu_sums3<T, decltype(KD)::value>(m, F, i, gi, lap, K); });
    F.mu[i] = mu_bulk3<T>(P, F.rho[i]) - P.kappa * lap;
#pragma unroll
    for (int c = 0; c < 3; ++c) F.k[c][i] = P.kappa * K[c];
}

// Per-node scalars of the collision (3-D form of CollidePrep).
template <typename T>
struct Prep3 {
    T r, u[3], p, omw, opw, hdt, X[3], dr[3], K[3], du[3], uX, uD, uK, uu, udu;
};

template <typename T>
__device__ __forceinline__ Prep3<T> prep3(const Phys3<T> &P, T sg, const T *mg, T r, const T *dr,
                                          const T *dm, const T *K) {
    constexpr T cs2 = T(1) / T(3);
    Prep3<T> c;
    c.hdt = T(0.5) * P.dt;
    c.r = r;
    const T inv_r = recip_rn(r);
    T ud = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        c.u[k] = (mg[k] + c.hdt * K[k] + c.hdt * r * P.g[k]) * inv_r;
        ud += c.u[k] * dr[k];
    }
    c.p = div3(sg + c.hdt * ud);  // correctly rounded: a rounded 1/3 is a gain on p (see kW3)
    T C = (r - P.rho_v) * P.inv_drho;
    C = C < T(0) ? T(0) : (C > T(1) ? T(1) : C);
    const T s = C * P.inv_tau_l + (T(1) - C) * P.inv_tau_v;  // 1/tau
    const T d = recip_rn(T(2) + s);
    c.omw = T(2) * s * d;  // 1 - w
    c.opw = T(4) * d;      // 1 + w
    c.uX = c.uD = c.uK = c.uu = c.udu = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        c.X[k] = cs2 * dr[k] - r * dm[k];
        c.dr[k] = dr[k];
        c.K[k] = K[k];
        c.du[k] = P.g[k] * P.dt;
        c.uX += c.u[k] * c.X[k];
        c.uD += c.u[k] * dr[k];
        c.uK += c.u[k] * K[k];
        c.uu += c.u[k] * c.u[k];
        c.udu += c.du[k] * (T(2) * c.u[k] + c.du[k]);
    }
    return c;
}

// Update of population a (same increment form as collide_pop).
template <typename T>
__device__ __forceinline__ void collide_pop3(const Prep3<T> &c, int a, T hs, T gs, T &hout, T &gout) {
    const T ex = T(e3x(a)), ey = T(e3y(a)), ez = T(e3z(a));
    const T wa = w3<T>(a), w3a = w3x3<T>(a);
    const T eu = ex * c.u[0] + ey * c.u[1] + ez * c.u[2];
    const T gmw = w3a * (eu + T(1.5) * eu * eu - T(0.5) * c.uu);  // Gamma - w
    const T gam3 = w3a + T(3) * gmw;                             // 3 Gamma
    const T eX = ex * c.X[0] + ey * c.X[1] + ez * c.X[2];
    const T eD = ex * c.dr[0] + ey * c.dr[1] + ez * c.dr[2];
    const T eK = ex * c.K[0] + ey * c.K[1] + ez * c.K[2];
    const T edu = ex * c.du[0] + ey * c.du[1] + ez * c.du[2];
    const T Fa = c.hdt * (eX - c.uX) * gam3;
    const T Ga = c.hdt * (eD - c.uD) * gmw + c.hdt * (eK - c.uK) * gam3;
    const T Ba = T(0.5) * c.r * w3a * (edu + T(1.5) * edu * (T(2) * eu + edu) - T(0.5) * c.udu);
    const T dh = fma(c.r, wa, -hs) + c.r * gmw;
    const T dg = fma(w3a, c.p, -gs) + c.r * gmw;
    hout = hs + (c.omw * dh + c.opw * Fa);
    gout = gs + (c.omw * dg + c.opw * (Ga + Ba));
}

// Collision of the opposite pair q = (a, a+1), a = 2q+1, in packed
// two-wide arithmetic: e_(a+1) = -e_a and equal weights, so the odd parts
// (e.u, e.X, e.grad rho, e.K, e.du) flip sign between the lanes and the even
// parts are shared (collide_pop3 on both members).
template <typename T>
__device__ __forceinline__ void collide_pair3(const Prep3<T> &c, int q, V2<T> hs, V2<T> gs, V2<T> &ho,
                                              V2<T> &go) {
    const int a = 2 * q + 1;
    const T ex = T(e3x(a)), ey = T(e3y(a)), ez = T(e3z(a));
    const T wa = w3<T>(a), w3a = w3x3<T>(a);
    const T eu = ex * c.u[0] + ey * c.u[1] + ez * c.u[2];
    const T eX = ex * c.X[0] + ey * c.X[1] + ez * c.X[2];
    const T eD = ex * c.dr[0] + ey * c.dr[1] + ez * c.dr[2];
    const T eK = ex * c.K[0] + ey * c.K[1] + ez * c.K[2];
    const T edu = ex * c.du[0] + ey * c.du[1] + ez * c.du[2];
    const T even = T(1.5) * eu * eu - T(0.5) * c.uu;
    const V2<T> gmw = vfma(vset(w3a, w3a), vset(eu, -eu), vset(w3a * even, w3a * even));  // Gamma - w
    const V2<T> gam3 = vfma(vset(T(3), T(3)), gmw, vset(w3a, w3a));                       // 3 Gamma
    const V2<T> Fa = vmul(vset(c.hdt * (eX - c.uX), c.hdt * (-eX - c.uX)), gam3);
    const V2<T> Ga = vfma(vset(c.hdt * (eD - c.uD), c.hdt * (-eD - c.uD)), gmw,
                          vmul(vset(c.hdt * (eK - c.uK), c.hdt * (-eK - c.uK)), gam3));
    const T bev = T(1.5) * edu * (T(2) * eu + edu) - T(0.5) * c.udu;
    const T hrw = T(0.5) * c.r * w3a;
    const V2<T> Sg = vfma(vset(hrw, hrw), vset(edu + bev, bev - edu), Ga);  // G + B
    const V2<T> rg = vmul(vset(c.r, c.r), gmw);
    const V2<T> dh = vadd(vfma(vset(c.r, c.r), vset(wa, wa), vset(-hs.x, -hs.y)), rg);   // h_eq - h*
    const V2<T> dg = vadd(vfma(vset(w3a, w3a), vset(c.p, c.p), vset(-gs.x, -gs.y)), rg);  // g_eq - g*
    ho = vadd(hs, vfma(vset(c.omw, c.omw), dh, vmul(vset(c.opw, c.opw), Fa)));
    go = vadd(gs, vfma(vset(c.omw, c.omw), dg, vmul(vset(c.opw, c.opw), Sg)));
}

template <typename T, typename Topo>
struct Collide3Args {
    Topo m;
    const T *fin;
    T *fout;
    Fields3<T> F;
    Phys3<T> P;
    T *mom;  // 5N (rho, ux, uy, uz, p) or nullptr
    int *flag;
};

template <typename T, typename Topo>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 5 : 1) k_collide3(const __grid_constant__ Collide3Args<T, Topo> A) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const Topo &m = A.m;
    if (i >= m.n) return;
    const size_t n = (size_t)m.n, np = pad4(n);
    T dm[3];
    V2<T> hp[9], gp[9];  // h* (from k_rho3) and the streamed g, as opposite pairs
    // g: streamed here (the h code on the g half of the state)
    by_kind(m, i, [&](auto K) {
        recover3<T, decltype(K)::value>(m, A.F.mu, i, dm);
        stream_all3<T, decltype(K)::value>(m, A.fin + 19 * np, np, i, A.P.dt, gp);
    });
    const T g0 = A.fin[19 * np + i];
    {
        // h: streamed and bounced back by k_rho3
        const V2<T> *hb = reinterpret_cast<const V2<T> *>(A.F.hs + np);
#pragma unroll
        for (int q = 0; q < 9; ++q) hp[q] = hb[q * np + i];
    }
    const T h0 = A.F.hs[i];
    const int k = m.tag_of(i);
    if (k) {
#pragma unroll
        for (int q = 0; q < 9; ++q) bounce_pair3<T>(k, q, gp[q]);
    }
    // moments of g: first moments from the differences of opposite pairs
    T sg = g0, mg[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const int a = 2 * q + 1;
        const T d = gp[q].x - gp[q].y;
        sg += gp[q].x + gp[q].y;
        mg[0] += T(e3x(a)) * d;
        mg[1] += T(e3y(a)) * d;
        mg[2] += T(e3z(a)) * d;
    }
    const T r = A.F.rho[i];
    T dr[3], K[3];
    load_grad3<T>(A.F.dr4, i, dr);
#pragma unroll
    for (int c = 0; c < 3; ++c) K[c] = A.F.k[c][i];
    const Prep3<T> c = prep3<T>(A.P, sg, mg, r, dr, dm, K);
    V2<T> *hb = reinterpret_cast<V2<T> *>(A.fout + np);
    V2<T> *gb = reinterpret_cast<V2<T> *>(A.fout + 20 * np);
    T dsum = T(0);
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        V2<T> ho, go;
        collide_pair3<T>(c, q, hp[q], gp[q], ho, go);
        dsum += (ho.x - hp[q].x) + (ho.y - hp[q].y);
        hb[q * np + i] = ho;
        gb[q * np + i] = go;
    }
    T hout0, gout0;
    collide_pop3<T>(c, 0, h0, g0, hout0, gout0);
    dsum += hout0 - h0;
    A.fout[i] = hout0 - dsum;  // local mass: sum_a hbar_a = sum_a h*_a up to one rounding
    A.fout[19 * np + i] = gout0;
    if (!(finite_val(r) && finite_val(c.u[0]) && finite_val(c.u[1]) && finite_val(c.u[2]) &&
          finite_val(c.p)))
        atomicOr(A.flag, 1);
    if (A.mom) {
        A.mom[i] = r;
        A.mom[n + i] = c.u[0];
        A.mom[2 * n + i] = c.u[1];
        A.mom[3 * n + i] = c.u[2];
        A.mom[4 * n + i] = c.p;
    }
}

// Initial pre-collided state psibar = eq + S of (rho, u, p) in mom.
template <typename T, typename Topo>
__global__ void __launch_bounds__(128) k_init3(const __grid_constant__ Topo m, T *__restrict__ fout,
                                               Fields3<T> F, Phys3<T> P, const T *__restrict__ mom) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.n) return;
    const size_t n = (size_t)m.n, np = pad4(n);
    T dm[3], dr[3], K[3];
    by_kind(m, i, [&](auto KD) { recover3<T, decltype(KD)::value>(m, F.mu, i, dm); });
    load_grad3<T>(F.dr4, i, dr);
#pragma unroll
    for (int c = 0; c < 3; ++c) K[c] = F.k[c][i];
    const T r = mom[i];
    Prep3<T> c;
    constexpr T cs2 = T(1) / T(3);
    c.hdt = T(0.5) * P.dt;
    c.r = r;
    c.p = mom[4 * n + i];
    c.uX = c.uD = c.uK = c.uu = c.udu = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        c.u[k] = mom[(1 + k) * n + i];
        c.X[k] = cs2 * dr[k] - r * dm[k];
        c.dr[k] = dr[k];
        c.K[k] = K[k];
        c.du[k] = P.g[k] * P.dt;
        c.uX += c.u[k] * c.X[k];
        c.uD += c.u[k] * dr[k];
        c.uK += c.u[k] * K[k];
        c.uu += c.u[k] * c.u[k];
        c.udu += c.du[k] * (T(2) * c.u[k] + c.du[k]);
    }
    // eq + S: the collision increment form with 1 - w = 1 and 1 + w = 1
    // applied to psi* = 0 gives eq + F (h) and eq + G + B (g)
    c.omw = T(1);
    c.opw = T(1);
    T h[19], g[19];
#pragma unroll
    for (int a = 0; a < 19; ++a) collide_pop3<T>(c, a, T(0), T(0), h[a], g[a]);
    V2<T> *hb = reinterpret_cast<V2<T> *>(fout + np);
    V2<T> *gb = reinterpret_cast<V2<T> *>(fout + 20 * np);
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        hb[q * np + i] = vset(h[2 * q + 1], h[2 * q + 2]);
        gb[q * np + i] = vset(g[2 * q + 1], g[2 * q + 2]);
    }
    fout[i] = h[0];
    fout[19 * np + i] = g[0];
}

// Moments in caller order, FP64: out[0..N) rho, [N..2N) C, [2N..5N) u
// interleaved (ux, uy, uz), [5N..6N) p.
template <typename T>
__global__ void k_gather_moments3(int32_t n, const T *__restrict__ mom, const int32_t *__restrict__ iperm,
                                  double rho_l, double rho_v, double *__restrict__ out) {
    const int32_t c = blockIdx.x * blockDim.x + threadIdx.x;  // caller id
    if (c >= n) return;
    const int32_t i = iperm[c];
    const size_t N = (size_t)n;
    const double r = (double)mom[i];
    out[c] = r;
    out[N + c] = (r - rho_v) / (rho_l - rho_v);
    for (int k = 0; k < 3; ++k) out[2 * N + 3 * (size_t)c + k] = (double)mom[(1 + k) * N + i];
    out[5 * N + c] = (double)mom[4 * N + i];
}

// FP64 totals: per-block partials of sum m rho and sum m rho u (4 values,
// [4][blocks]), then one warp reduces them in a fixed order.
template <typename T>
__global__ void __launch_bounds__(256) k_totals3_partial(int32_t n, const T *__restrict__ mom,
                                                         const double *__restrict__ mass,
                                                         double *__restrict__ part) {
    __shared__ double s[4][256];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const size_t N = (size_t)n;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double mr = mass[i] * (double)mom[i];
        acc[0] += mr;
        for (int k = 0; k < 3; ++k) acc[1 + k] += mr * (double)mom[(1 + k) * N + i];
    }
    for (int k = 0; k < 4; ++k) s[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 4; ++k) s[k][threadIdx.x] += s[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) part[(size_t)k * gridDim.x + blockIdx.x] = s[k][0];
}

__global__ void k_totals3_final(int nparts, const double *__restrict__ part, double *__restrict__ out) {
    const int l = threadIdx.x;
    for (int k = 0; k < 4; ++k) {
        double v = 0.0;
        for (int b = l; b < nparts; b += 32) v += part[(size_t)k * nparts + b];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (l == 0) out[k] = v;
    }
}

}  // namespace felbm
