// Device kernels of one FE-LBM time step, general (unstructured CSR) path.
//
// One step = four dependent neighbour passes, each a gather over the
// assembled per-node operators (HostCSR in felbm_internal.h):
//   k_rho      Taylor-Galerkin streaming of the 9 h populations (Sec. 2.2.1,
//              Eq. galerkin_lbm with the lumped mass), wall bounce-back,
//              rho = sum_a h_a.
//   k_grad     recovered grad rho (Sec. 2.3).
//   k_mu       Laplacian of rho (recovery of the recovered gradient), the
//              stress force K = kappa [d_i |grad rho|^2 - d_j (d_i rho d_j rho)]
//              and mu = mu_phi(rho) - kappa lap rho (Sec. 2.1).
//   k_collide  recovered grad mu; streaming of all 18 populations; bounce-back;
//              moments (Eqs. velocity, pressure); post-streaming collision and
//              the next pre-streaming collision (Sec. 2.2) in one update.
// Operators use the difference form sum_{j != i} c_ij (f_j - f_i), exact for
// constant fields in any precision.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "felbm_internal.h"

namespace felbm {

// D2Q9 velocity components, weights, opposite directions.
__host__ __device__ constexpr int kEx(int a) { return a == 1 || a == 5 || a == 8 ? 1 : (a == 3 || a == 6 || a == 7 ? -1 : 0); }
__host__ __device__ constexpr int kEy(int a) { return a == 2 || a == 5 || a == 6 ? 1 : (a == 4 || a == 7 || a == 8 ? -1 : 0); }
__host__ __device__ constexpr int kOpp(int a) { return a == 0 ? 0 : (a <= 4 ? ((a + 1) % 4) + 1 : ((a - 5 + 2) % 4) + 5); }
template <typename T>
__host__ __device__ constexpr T kW(int a) { return a == 0 ? T(4) / T(9) : (a <= 4 ? T(1) / T(9) : T(1) / T(36)); }

// 1/12 rounded to a multiple of 2^-25 (FP32) or 2^-54 (FP64): the base of the
// 3 w_a constants below, chosen so that they are exact in T.
template <typename T>
__host__ __device__ constexpr T kTwelfth() {
    return sizeof(T) == 4 ? T(2796203.0 / 33554432.0) : T(1501199875790165.0 / 18014398509481984.0);
}

// 3 w_a in the working precision, with the moment identities of the
// equilibria exact in T: sum_a 3 w_a = 3 (w3_0 + 4 w3_1 + 4 w3_5) and
// sum_a 3 w_a e_ax^2 = 1 (2 w3_1 + 4 w3_5), from e ~ 1/12: w3_5 = e,
// w3_1 = (1 - 4 e)/2, w3_0 = 1 + 4 e.  The nearest values to 4/3, 1/3, 1/12
// miss both identities by about one rounding; through the pressure and the
// momentum of g that bias is a gain on p and u applied every step, which a
// near-steady FP32 run accumulates (1.3e-5 in u after 1000 steps of a
// droplet, against 1.3e-6 with these constants).
template <typename T>
__host__ __device__ constexpr T kW3(int a) {
    return a == 0 ? T(1) + T(4) * kTwelfth<T>() : (a <= 4 ? (T(1) - T(4) * kTwelfth<T>()) / T(2) : kTwelfth<T>());
}

template <typename T>
__device__ __forceinline__ bool finite_val(T v) { return isfinite(v); }

// ---- packed two-wide arithmetic on a pair of opposite populations ----

template <typename T>
struct V2T;
template <>
struct V2T<float> {
    using type = float2;
};
template <>
struct V2T<double> {
    using type = double2;
};
template <typename T>
using V2 = typename V2T<T>::type;

// packed two-wide arithmetic (one instruction per operation in FP32)
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 vfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 vset(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 vset(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 vadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double2 vmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }


// Streaming coefficient of direction a from the assembled tensors:
//   c = e.a_ij + (dt/2) e.b_ij.e
template <typename T, int A>
__device__ __forceinline__ T stream_coef(T ax, T ay, T hbxx, T hbxy, T hbyy) {
    constexpr int ex = kEx(A), ey = kEy(A);
    T c = T(0);
    if (ex) c += T(ex) * ax + hbxx;
    if (ey) c += T(ey) * ay + hbyy;
    if (ex && ey) c += T(2 * ex * ey) * hbxy;
    return c;
}

// Streaming coefficients of pair q (directions pair_dir(q, 0), its opposite):
// c = e.a_ij + (dt/2) e.b_ij.e, the odd part e.a flipping sign between the
// two; the slot-0 directions are (1,0), (0,1), (1,1), (-1,1).
template <typename T>
__device__ __forceinline__ V2<T> pair_coef(int q, T ax, T ay, T hbxx, T hbxy, T hbyy) {
    T odd, even;
    if (q == 0) {
        odd = ax;
        even = hbxx;
    } else if (q == 1) {
        odd = ay;
        even = hbyy;
    } else if (q == 2) {
        odd = ax + ay;
        even = (hbxx + hbyy) + T(2) * hbxy;
    } else {
        odd = ay - ax;
        even = (hbxx + hbyy) - T(2) * hbxy;
    }
    return vset(even + odd, even - odd);
}

// Streamed pairs of node i from the state f (pair layout, np = padded slot
// count): psi* = psi - dt sum_{j != i} c_ij (psi_j - psi_i) for the 4 h
// pairs and, with G, the 4 g pairs, one 8-byte load per pair and neighbour
// and the neighbour's coefficients loaded once.
template <typename T, bool G, typename Topo>
__device__ __forceinline__ void stream_pairs(const Topo &m, const T *__restrict__ f, size_t np, int32_t i,
                                             T dt, V2<T> *hp, V2<T> *gp) {
    const V2<T> *hb = reinterpret_cast<const V2<T> *>(f + np);
    const V2<T> *gb = reinterpret_cast<const V2<T> *>(f + 10 * np);
    const size_t si = m.slot(i);
    const V2<T> m1 = vset(T(-1), T(-1));
    V2<T> hs[4], ha[4], gs[4], ga[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        hs[q] = hb[q * np + si];
        ha[q] = vset(T(0), T(0));
        if (G) {
            gs[q] = gb[q * np + si];
            ga[q] = vset(T(0), T(0));
        }
    }
    const T hdt = T(0.5) * dt;
    m.for_each(i, [&](int32_t j, T ax, T ay, T bxx, T bxy, T byy) {
        const size_t sj = m.slot(j);
        const T hbxx = hdt * bxx, hbxy = hdt * bxy, hbyy = hdt * byy;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const V2<T> c = pair_coef<T>(q, ax, ay, hbxx, hbxy, hbyy);
            ha[q] = vfma(c, vfma(hs[q], m1, __ldg(hb + q * np + sj)), ha[q]);
            if (G) ga[q] = vfma(c, vfma(gs[q], m1, __ldg(gb + q * np + sj)), ga[q]);
        }
    });
    const V2<T> mdt = vset(-dt, -dt);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        hp[q] = vfma(mdt, ha[q], hs[q]);
        if (G) gp[q] = vfma(mdt, ga[q], gs[q]);
    }
}

// Populations of a node by direction from its rest value and 4 pairs.
template <typename T>
__device__ __forceinline__ void unpack_pairs(T rest, const V2<T> *p, T *psi) {
    psi[0] = rest;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        psi[pair_dir(q, 0)] = p[q].x;
        psi[pair_dir(q, 1)] = p[q].y;
    }
}

// Bounce-back at a wall node with inward normal e_k: every population with
// e_a . e_k > 0 takes the value of its opposite.  psi holds 9 populations.
template <typename T>
__device__ __forceinline__ void bounce_back(int k, T *psi) {
    const int nx = kEx(k), ny = kEy(k);
#pragma unroll
    for (int a = 1; a < 9; ++a)
        if (kEx(a) * nx + kEy(a) * ny > 0) psi[a] = psi[kOpp(a)];
}

template <typename T, typename Topo>
__global__ void __launch_bounds__(256) k_rho(Topo m, const T *__restrict__ f, T dt,
                                             T *__restrict__ rho, T *__restrict__ hs) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.n) return;
    const size_t np = pad4(m.slots());
    V2<T> hp[4];
    stream_pairs<T, false>(m, f, np, i, dt, hp, hp);
    T h[9];
    unpack_pairs<T>(f[m.slot(i)], hp, h);
    {
        const int k = m.tag_of(i);
        if (k) bounce_back<T>(k, h);
    }
    T r = T(0);
#pragma unroll
    for (int a = 0; a < 9; ++a) r += h[a];
    rho[i] = r;
    const size_t si = m.slot(i);
    V2<T> *hb = reinterpret_cast<V2<T> *>(hs + np);
#pragma unroll
    for (int q = 0; q < 4; ++q) hb[q * np + si] = vset(h[pair_dir(q, 0)], h[pair_dir(q, 1)]);
    hs[si] = h[0];
}

// Recovered gradient of a scalar field.
template <typename T, typename Topo>
__device__ __forceinline__ void recover(const Topo &m, const T *__restrict__ f, int32_t i,
                                        T &gx, T &gy) {
    const T fi = f[i];
    T sx = T(0), sy = T(0);
    m.for_each(i, [&](int32_t j, T ax, T ay, T, T, T) {
        const T d = __ldg(f + j) - fi;
        sx += ax * d;
        sy += ay * d;
    });
    gx = sx;
    gy = sy;
}

template <typename T, typename Topo>
__global__ void __launch_bounds__(256) k_grad(Topo m, Fields<T> F) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.n) return;
    T gx, gy;
    recover(m, F.rho, i, gx, gy);
    F.drx[i] = gx;
    F.dry[i] = gy;
}

// mu_phi = 4 beta (rho - rho_v)(rho - rho_l)(rho - (rho_v + rho_l)/2).
template <typename T>
__device__ __forceinline__ T mu_bulk(const Phys<T> &P, T r) {
    return T(4) * P.beta * (r - P.rho_v) * (r - P.rho_l) * (r - T(0.5) * (P.rho_v + P.rho_l));
}

// lap rho = R_x(d_x rho) + R_y(d_y rho);
// K_x = kappa [R_x((d_y rho)^2) - R_y(d_x rho d_y rho)],
// K_y = kappa [R_y((d_x rho)^2) - R_x(d_x rho d_y rho)]
// (the printed form d_i(|grad rho|^2) - d_j(d_i rho d_j rho) with the
// identical (d_i rho)^2 contributions cancelled, R linear);
// mu = 4 beta (rho - rho_v)(rho - rho_l)(rho - (rho_v + rho_l)/2) - kappa lap rho.
template <typename T, typename Topo>
__global__ void __launch_bounds__(256) k_mu(Topo m, Fields<T> F, Phys<T> P) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.n) return;
    const T gxi = F.drx[i], gyi = F.dry[i];
    T lap = T(0), kx = T(0), ky = T(0);
    m.for_each(i, [&](int32_t j, T ax, T ay, T, T, T) {
        const T gxj = __ldg(F.drx + j), gyj = __ldg(F.dry + j);
        lap += ax * (gxj - gxi) + ay * (gyj - gyi);
        // differences of the gradient products in product form (no
        // cancellation between two squares of nearly equal size)
        const T ddx = gxj - gxi, ddy = gyj - gyi;
        const T dxx = ddx * (gxj + gxi), dxy = gxj * ddy + gyi * ddx, dyy = ddy * (gyj + gyi);
        kx += ax * dyy - ay * dxy;
        ky += ay * dxx - ax * dxy;
    });
    F.mu[i] = mu_bulk<T>(P, F.rho[i]) - P.kappa * lap;
    F.kx[i] = P.kappa * kx;
    F.ky[i] = P.kappa * ky;
}

// k_mu for FP32 fields with the kappa lap rho term of mu in FP64
// (FELBM_PARAM_LAP_FP64): Topo64 carries the mesh's FP64 coefficients; the
// Laplacian of the FP32 gradient and its product with kappa are formed in
// FP64 and subtracted from the bulk term in FP64, rounded once.  K is formed
// as in k_mu, from the same coefficients rounded to FP32.
template <typename Topo64>
__global__ void __launch_bounds__(256) k_mu_lap64(Topo64 m, Fields<float> F, Phys<float> P, double kappa) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.n) return;
    const float gxi = F.drx[i], gyi = F.dry[i];
    double lap = 0.0;
    float kx = 0.f, ky = 0.f;
    m.for_each(i, [&](int32_t j, double ax, double ay, double, double, double) {
        const float gxj = __ldg(F.drx + j), gyj = __ldg(F.dry + j);
        lap += ax * ((double)gxj - (double)gxi) + ay * ((double)gyj - (double)gyi);
        const float fax = (float)ax, fay = (float)ay;
        const float ddx = gxj - gxi, ddy = gyj - gyi;
        const float dxx = ddx * (gxj + gxi), dxy = gxj * ddy + gyi * ddx, dyy = ddy * (gyj + gyi);
        kx += fax * dyy - fay * dxy;
        ky += fay * dxx - fax * dxy;
    });
    F.mu[i] = (float)((double)mu_bulk<float>(P, F.rho[i]) - kappa * lap);
    F.kx[i] = P.kappa * kx;
    F.ky[i] = P.kappa * ky;
}

// Local collision of one node (Sec. 2.2), split in two so that callers can
// keep the streamed populations outside registers:
//   collide_prep  moments (Eqs. velocity, pressure), tau, and the per-node
//                 scalars of the equilibria and sources;
//   collide_pop   the update of population a.
// With eq and source S of the node, the post-streaming collision
//   psi = psi* + 2tau/(2tau+1) (-(psi* - eq)/(2tau) + S)
// followed by the pre-streaming collision of the next step
//   psibar = psi + (-(psi - eq)/(2tau) + S)
// equals psibar = eq + S + w (psi* - eq + S), w = (2tau - 1)/(2tau + 1),
// evaluated as psibar = psi* + (1 - w)(eq - psi*) + (1 + w) S with
// eq - psi* = fma(rho, w_a, -psi*) + rho (Gamma - w_a): every rounding then
// falls on the small collision increment instead of on O(w_a rho) terms
// (in FP32 the other order repeats the same O(ulp(rho)) error every step).
template <typename T>
struct CollidePrep {
    T r, ux, uy, p, omw, opw, hdt, Xx, Xy, uX, uD, uK, uu, dux, duy, udu, drx, dry, kx, ky;
};

// Correctly rounded reciprocal (the same value as T(1) / x).
__device__ __forceinline__ float recip_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip_rn(double x) { return __drcp_rn(x); }

// x / 3 correctly rounded, by a product with the rounded 1/3 and one
// correction with the exact remainder x - 3 q (the FMA form of
// division by a constant of Markstein, IBM J. Res. Dev. 34 (1990)).  It
// equals the rounded quotient for every normal FP32 mantissa and for all
// FP64 operands sampled (checked with exact rational arithmetic).
template <typename T>
__device__ __forceinline__ T div3(T x) {
    constexpr T c = T(1) / T(3);
    const T q = x * c;
    const T r = fma(T(-3), q, x);
    return fma(r, c, q);
}

// sg = sum_a g*_a, mx, my = sum_a e_a g*_a of the streamed (and bounced) g.
template <typename T>
__device__ __forceinline__ CollidePrep<T> collide_prep(const Phys<T> &P, T sg, T mx, T my, T r,
                                                       T drx, T dry, T dmx, T dmy, T kx, T ky) {
    constexpr T cs2 = T(1) / T(3);
    CollidePrep<T> c;
    c.hdt = T(0.5) * P.dt;
    const T inv_r = recip_rn(r);
    c.r = r;
    c.ux = (mx + c.hdt * kx + c.hdt * r * P.gx) * inv_r;
    c.uy = (my + c.hdt * ky + c.hdt * r * P.gy) * inv_r;
    // p = c_s^2 (...) as a division by 3: a rounded 1/3 would be a gain on p
    // every step (see kW3)
    c.p = div3(sg + c.hdt * (c.ux * drx + c.uy * dry));
    T C = (r - P.rho_v) * P.inv_drho;
    C = C < T(0) ? T(0) : (C > T(1) ? T(1) : C);
    // 1/tau = C/tau_l + (1-C)/tau_v; w = (2 tau - 1)/(2 tau + 1) gives, with
    // s = 1/tau, 1 - w = 2 s/(2 + s) and 1 + w = 4/(2 + s): one reciprocal
    const T s = C * P.inv_tau_l + (T(1) - C) * P.inv_tau_v;
    const T d = recip_rn(T(2) + s);
    c.omw = T(2) * s * d;  // 1 - w
    c.opw = T(4) * d;      // 1 + w
    c.Xx = cs2 * drx - r * dmx;  // F: c_s^2 grad rho - rho grad mu
    c.Xy = cs2 * dry - r * dmy;
    c.uX = c.ux * c.Xx + c.uy * c.Xy;
    c.uD = c.ux * drx + c.uy * dry;
    c.uK = c.ux * kx + c.uy * ky;
    c.uu = c.ux * c.ux + c.uy * c.uy;
    c.dux = P.gx * P.dt;  // exact-difference du = g dt
    c.duy = P.gy * P.dt;
    c.udu = c.dux * (T(2) * c.ux + c.dux) + c.duy * (T(2) * c.uy + c.duy);
    c.drx = drx;
    c.dry = dry;
    c.kx = kx;
    c.ky = ky;
    return c;
}

template <typename T, int A>
__device__ __forceinline__ void collide_pop(const CollidePrep<T> &c, T hs, T gs, T &hout, T &gout) {
    constexpr int ex = kEx(A), ey = kEy(A);
    constexpr T wa = kW<T>(A), w3 = kW3<T>(A);
    const T eu = T(ex) * c.ux + T(ey) * c.uy;
    // Gamma - w formed directly: forming Gamma ~ w first and subtracting w
    // would cancel away the momentum part rho w 3 e.u in FP32.
    const T gmw = w3 * (eu + T(1.5) * eu * eu - T(0.5) * c.uu);
    const T gam3 = w3 + T(3) * gmw;  // 3 Gamma
    const T eX = T(ex) * c.Xx + T(ey) * c.Xy;
    const T eD = T(ex) * c.drx + T(ey) * c.dry;
    const T eK = T(ex) * c.kx + T(ey) * c.ky;
    const T edu = T(ex) * c.dux + T(ey) * c.duy;
    const T Fa = c.hdt * (eX - c.uX) * gam3;
    const T Ga = c.hdt * (eD - c.uD) * gmw + c.hdt * (eK - c.uK) * gam3;
    // 1/2 [g_eq(u + du) - g_eq(u)] = rho/2 [Gamma(u + du) - Gamma(u)]
    const T Ba = T(0.5) * c.r * w3 * (edu + T(1.5) * edu * (T(2) * eu + edu) - T(0.5) * c.udu);
    const T Sg = Ga + Ba;
    const T dh = fma(c.r, wa, -hs) + c.r * gmw;  // h_eq - h*
    const T dg = fma(w3, c.p, -gs) + c.r * gmw;  // g_eq - g*
    hout = hs + (c.omw * dh + c.opw * Fa);
    gout = gs + (c.omw * dg + c.opw * Sg);
}

template <typename T>
__device__ __forceinline__ void collide_pop_rt(const CollidePrep<T> &c, int a, T hs, T gs, T &ho,
                                               T &go) {
    switch (a) {
        case 0: collide_pop<T, 0>(c, hs, gs, ho, go); break;
        case 1: collide_pop<T, 1>(c, hs, gs, ho, go); break;
        case 2: collide_pop<T, 2>(c, hs, gs, ho, go); break;
        case 3: collide_pop<T, 3>(c, hs, gs, ho, go); break;
        case 4: collide_pop<T, 4>(c, hs, gs, ho, go); break;
        case 5: collide_pop<T, 5>(c, hs, gs, ho, go); break;
        case 6: collide_pop<T, 6>(c, hs, gs, ho, go); break;
        case 7: collide_pop<T, 7>(c, hs, gs, ho, go); break;
        default: collide_pop<T, 8>(c, hs, gs, ho, go); break;
    }
}

// Zeroth and first moments of the streamed g.  The first moments are summed
// as differences of opposite populations: each difference is exact in
// floating point when the two are close (they share the pressure part
// w_a 3p), so only the small momentum-carrying parts are rounded.
template <typename T>
__device__ __forceinline__ void g_moments(T g0, T g1, T g2, T g3, T g4, T g5, T g6, T g7, T g8,
                                          T &sg, T &mx, T &my) {
    const T d13 = g1 - g3, d24 = g2 - g4, d57 = g5 - g7, d68 = g6 - g8;
    mx = d13 + (d57 - d68);  // e_x: +1, 3: -1, 5: +1, 6: -1, 7: -1, 8: +1
    my = d24 + (d57 + d68);  // e_y: +2, 4: -1, 5: +1, 6: +1, 7: -1, 8: -1
    sg = ((g0 + (g1 + g3)) + (g2 + g4)) + ((g5 + g7) + (g6 + g8));
}

template <typename T>
__device__ __forceinline__ void collide_node(const Phys<T> &P, const T *hs, const T *gs, T r,
                                             T drx, T dry, T dmx, T dmy, T kx, T ky, T *hout,
                                             T *gout, T &ux, T &uy, T &p) {
    T sg, mx, my;
    g_moments<T>(gs[0], gs[1], gs[2], gs[3], gs[4], gs[5], gs[6], gs[7], gs[8], sg, mx, my);
    const CollidePrep<T> c = collide_prep<T>(P, sg, mx, my, r, drx, dry, dmx, dmy, kx, ky);
    T dsum = T(0);  // sum of the h increments: zero in exact arithmetic
#pragma unroll
    for (int a = 1; a < 9; ++a) {
        collide_pop_rt<T>(c, a, hs[a], gs[a], hout[a], gout[a]);
        dsum += hout[a] - hs[a];
    }
    collide_pop_rt<T>(c, 0, hs[0], gs[0], hout[0], gout[0]);
    dsum += hout[0] - hs[0];
    hout[0] -= dsum;  // local mass: sum_a hbar_a = sum_a h*_a up to one rounding
    ux = c.ux;
    uy = c.uy;
    p = c.p;
}

template <typename T, typename Topo>
struct CollideArgs {
    Topo m;
    const T *fin;
    T *fout;
    Fields<T> F;
    Phys<T> P;
    T *mom;  // 4N or nullptr
    int *flag;
};

template <typename T, typename Topo>
__global__ void __launch_bounds__(256) k_collide(CollideArgs<T, Topo> A) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const Topo &m = A.m;
    if (i >= m.n) return;
    const size_t n = (size_t)m.n;
    T dmx, dmy;
    recover(m, A.F.mu, i, dmx, dmy);
    const size_t np = pad4(m.slots()), si = m.slot(i);
    T hs[9], gs[9];
    {
        // g streamed here (the h code on the g half of the state); h* was
        // streamed and bounced back by k_rho
        V2<T> gp[4], hp[4];
        stream_pairs<T, false>(m, A.fin + 9 * np, np, i, A.P.dt, gp, gp);
        unpack_pairs<T>(A.fin[9 * np + si], gp, gs);
        const V2<T> *hsb = reinterpret_cast<const V2<T> *>(A.F.hs + np);
#pragma unroll
        for (int q = 0; q < 4; ++q) hp[q] = hsb[q * np + si];
        unpack_pairs<T>(A.F.hs[si], hp, hs);
    }
    {
        const int k = m.tag_of(i);
        if (k) bounce_back<T>(k, gs);
    }
    const T r = A.F.rho[i];
    T hout[9], gout[9], ux, uy, p;
    collide_node<T>(A.P, hs, gs, r, A.F.drx[i], A.F.dry[i], dmx, dmy, A.F.kx[i], A.F.ky[i], hout,
                    gout, ux, uy, p);
    V2<T> *hb = reinterpret_cast<V2<T> *>(A.fout + np);
    V2<T> *gb = reinterpret_cast<V2<T> *>(A.fout + 10 * np);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        hb[q * np + si] = vset(hout[pair_dir(q, 0)], hout[pair_dir(q, 1)]);
        gb[q * np + si] = vset(gout[pair_dir(q, 0)], gout[pair_dir(q, 1)]);
    }
    A.fout[si] = hout[0];
    A.fout[9 * np + si] = gout[0];
    if (!(finite_val(r) && finite_val(ux) && finite_val(uy) && finite_val(p))) atomicOr(A.flag, 1);
    if (A.mom) {
        A.mom[i] = r;
        A.mom[n + i] = ux;
        A.mom[2 * n + i] = uy;
        A.mom[3 * n + i] = p;
    }
}

// Initial state: post-collision distributions are the equilibria of
// (rho0, u0, p0); stored value psibar = eq + S (Omega(eq) = 0).
template <typename T, typename Topo>
__global__ void __launch_bounds__(256) k_init(Topo m, T *__restrict__ fout, Fields<T> F,
                                              Phys<T> P, const T *__restrict__ mom) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.n) return;
    const size_t n = (size_t)m.n;
    T dmx, dmy;
    recover(m, F.mu, i, dmx, dmy);
    const T r = mom[i], ux = mom[n + i], uy = mom[2 * n + i], p = mom[3 * n + i];
    const T drx = F.drx[i], dry = F.dry[i], kx = F.kx[i], ky = F.ky[i];
    const T hdt = T(0.5) * P.dt;
    const T Xx = T(1) / T(3) * drx - r * dmx, Xy = T(1) / T(3) * dry - r * dmy;
    const T uX = ux * Xx + uy * Xy, uD = ux * drx + uy * dry, uK = ux * kx + uy * ky;
    const T uu = ux * ux + uy * uy;
    const T dux = P.gx * P.dt, duy = P.gy * P.dt;
    const T udu = dux * (T(2) * ux + dux) + duy * (T(2) * uy + duy);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const int ex = kEx(a), ey = kEy(a);
        const T wa = kW<T>(a), w3 = kW3<T>(a);
        const T eu = T(ex) * ux + T(ey) * uy;
        const T gmw = w3 * (eu + T(1.5) * eu * eu - T(0.5) * uu);  // Gamma - w
        const T gam3 = w3 + T(3) * gmw;                             // 3 Gamma
        const T eX = T(ex) * Xx + T(ey) * Xy;
        const T eD = T(ex) * drx + T(ey) * dry;
        const T eK = T(ex) * kx + T(ey) * ky;
        const T edu = T(ex) * dux + T(ey) * duy;
        const T Fa = hdt * (eX - uX) * gam3;
        const T Ga = hdt * (eD - uD) * gmw + hdt * (eK - uK) * gam3;
        const T Ba = T(0.5) * r * w3 * (edu + T(1.5) * edu * (T(2) * eu + edu) - T(0.5) * udu);
        fout[pop_index(a, m.slot(i), m.slots())] = (r * wa + r * gmw) + Fa;
        fout[pop_index(9 + a, m.slot(i), m.slots())] = w3 * p + r * gmw + Ga + Ba;
    }
}

// Moments in caller order, FP64: out[0..N) rho, [N..2N) C, [2N..4N) u
// interleaved (ux, uy), [4N..5N) p.
template <typename T>
__global__ void k_gather_moments(int32_t n, const T *__restrict__ mom, const int32_t *__restrict__ iperm,
                                 double rho_l, double rho_v, double *__restrict__ out) {
    const int32_t c = blockIdx.x * blockDim.x + threadIdx.x;  // caller id
    if (c >= n) return;
    const int32_t k = iperm ? iperm[c] : c;
    const double r = (double)mom[k];
    out[c] = r;
    out[(size_t)n + c] = (r - rho_v) / (rho_l - rho_v);
    out[2 * (size_t)n + 2 * (size_t)c] = (double)mom[(size_t)n + k];
    out[2 * (size_t)n + 2 * (size_t)c + 1] = (double)mom[2 * (size_t)n + k];
    out[4 * (size_t)n + c] = (double)mom[3 * (size_t)n + k];
}

// FP64 totals: sum m rho, sum m rho ux, sum m rho uy.  Deterministic two-pass
// reduction: block partials (warp shuffles + shared memory), then one block.
template <typename T>
__global__ void __launch_bounds__(256) k_totals_partial(int32_t n, const T *__restrict__ mom,
                                                        const double *__restrict__ mass,
                                                        double *__restrict__ part) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double mr = mass[i] * (double)mom[i];
        s0 += mr;
        s1 += mr * (double)mom[(size_t)n + i];
        s2 += mr * (double)mom[2 * (size_t)n + i];
    }
    __shared__ double sh[3][8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sh[0][wid] = s0;
        sh[1][wid] = s1;
        sh[2][wid] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0, t1 = 0, t2 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t0 += sh[0][w];
            t1 += sh[1][w];
            t2 += sh[2][w];
        }
        part[3 * blockIdx.x] = t0;
        part[3 * blockIdx.x + 1] = t1;
        part[3 * blockIdx.x + 2] = t2;
    }
}

__global__ void k_totals_final(int nparts, const double *__restrict__ part, double *__restrict__ out);

}  // namespace felbm
