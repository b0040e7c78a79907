// One-launch step of a general triangle mesh (k_patch_step): one block per
// patch of kPatch nodes (a compact piece of the mesh along a Hilbert curve,
// internal order patch-major).  A node's next state depends on the present
// populations up to 4 edges away (h streamed on the rings <= 3 around the
// patch, whose own values are streamed from one ring further out; rho ->
// grad rho -> lap rho, mu -> grad mu, Sec. 2.2.1 and Sec. 2.3), so the block
//   0. gathers the h pairs and h_0 of its region (own nodes and rings 1..4)
//      and the g pairs of rings <= 1 into shared memory;
//   1. streams h and bounces it back on rings <= 3 and forms rho there; each
//      thread keeps its own node's streamed h in registers;
//   2. recovers grad rho on rings <= 2, then
//   3. lap rho and mu on rings <= 1 (and the stress force at its own node);
//   4. at its own node: grad mu, the g streaming, the moments and the
//      collision, and one write of the 18 populations.
// The neighbours of a region node are read through the mesh's CSR (rows in
// internal order, coefficients in the state's precision) with their region
// indices (16-bit) in place of the column ids.  Every stage is the
// four-launch path's per-node arithmetic in the same order (k_rho, k_grad,
// k_mu, k_collide), so both give the same results bit for bit.
#pragma once

#include "felbm_internal.h"
#include "felbm_kernels.cuh"

namespace felbm {

template <typename T>
struct PatchArgs {
    DevCSR<T> m;
    const int32_t *nbase;    // region list offsets, one per patch + 1
    const int32_t *count;    // per patch: nodes of rings <= 0, 1, 2, 3
    const int32_t *node;     // region nodes (internal ids), own first
    const int32_t *rowbase;  // rings <= 3: offset of the row's region columns in lcol
    const uint16_t *lcol;    // region index of every CSR column of those rows
    int32_t rmax, r1max, r2max, r3max;
    const T *fin;
    T *fout;
    Phys<T> P;
    T *mom;  // 4N or nullptr
    int *flag;
    // FP64 kappa lap rho term (FELBM_PARAM_LAP_FP64, LAP64 kernels only): the
    // CSR's a coefficients in FP64 and kappa
    const double *ax64, *ay64;
    double kappa64;
};

// Shared-memory bytes of one block (layout of k_patch_step).
template <typename T>
inline size_t patch_smem(int32_t rmax, int32_t r1max, int32_t r2max, int32_t r3max) {
    return (size_t)(4 * rmax + 4 * r1max + r2max) * sizeof(V2<T>) + (size_t)(rmax + r3max + r1max) * sizeof(T) +
           (size_t)r3max;
}

// LAP64: the kappa lap rho term of mu in FP64, as k_mu_lap64 forms it.
template <typename T, bool LAP64>
__global__ void __launch_bounds__(kPatch, sizeof(T) == 4 ? 3 : 1) k_patch_step(const __grid_constant__ PatchArgs<T> A) {
    extern __shared__ __align__(16) unsigned char psm[];
    const DevCSR<T> &m = A.m;
    const int p = blockIdx.x, tid = threadIdx.x;
    const int32_t base = A.nbase[p], nreg = A.nbase[p + 1] - base;
    const int32_t n0 = A.count[4 * p], n1 = A.count[4 * p + 1], n2 = A.count[4 * p + 2], n3 = A.count[4 * p + 3];
    const int32_t rmax = A.rmax, r1max = A.r1max;
    V2<T> *hP = reinterpret_cast<V2<T> *>(psm);  // [4][rmax]
    V2<T> *gP = hP + 4 * rmax;                   // [4][r1max]
    V2<T> *grd = gP + 4 * r1max;                 // [r2max]
    T *h0 = reinterpret_cast<T *>(grd + A.r2max);  // [rmax]
    T *rho = h0 + rmax;                            // [r3max]
    T *mu = rho + A.r3max;                         // [r1max]
    uint8_t *tg = reinterpret_cast<uint8_t *>(mu + r1max);  // [r3max]
    const size_t n = (size_t)m.n, np = pad4((size_t)m.n);
    const V2<T> *hb = reinterpret_cast<const V2<T> *>(A.fin + np);
    const V2<T> *gb = reinterpret_cast<const V2<T> *>(A.fin + 10 * np);
    const Phys<T> &P = A.P;

    // 0. the region's populations (own nodes first: contiguous)
    for (int32_t r = tid; r < nreg; r += kPatch) {
        const int32_t g = A.node[base + r];
        if (!chk_idx(g, m.n, 1u) || !chk_idx(r, rmax, 2u)) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) hP[q * rmax + r] = hb[q * np + g];
        h0[r] = A.fin[g];
        if (r < n1) {
#pragma unroll
            for (int q = 0; q < 4; ++q) gP[q * r1max + r] = gb[q * np + g];
        }
        if (r < n3) tg[r] = m.tag ? m.tag[g] : uint8_t(0);
    }
    __syncthreads();

    // 1. streamed, bounced-back h and rho on rings <= 3 (k_rho)
    const T dt = P.dt, hdt = T(0.5) * dt;
    const V2<T> m1 = vset(T(-1), T(-1)), mdt = vset(-dt, -dt);
    T hown[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) hown[a] = T(0);
    for (int32_t r = tid; r < n3; r += kPatch) {
        const int32_t g = A.node[base + r];
        const int32_t e0 = __ldg(m.rowptr + g), e1 = __ldg(m.rowptr + g + 1);
        const uint16_t *lc = A.lcol + A.rowbase[base + r];  // columns of e0 .. e1
        V2<T> hs[4], ha[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            hs[q] = hP[q * rmax + r];
            ha[q] = vset(T(0), T(0));
        }
#pragma unroll 4
        for (int32_t e = e0; e < e1; ++e) {
            const int j = lc[e - e0];
            if (!chk_idx(j, nreg, 2u)) continue;
            const T ax = __ldg(m.ax + e), ay = __ldg(m.ay + e);
            const T hbxx = hdt * __ldg(m.bxx + e), hbxy = hdt * __ldg(m.bxy + e), hbyy = hdt * __ldg(m.byy + e);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const V2<T> c = pair_coef<T>(q, ax, ay, hbxx, hbxy, hbyy);
                ha[q] = vfma(c, vfma(hs[q], m1, hP[q * rmax + j]), ha[q]);
            }
        }
        V2<T> hp[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) hp[q] = vfma(mdt, ha[q], hs[q]);
        T h[9];
        unpack_pairs<T>(h0[r], hp, h);
        {
            const int k = tg[r];
            if (k) bounce_back<T>(k, h);
        }
        T s = T(0);
#pragma unroll
        for (int a = 0; a < 9; ++a) s += h[a];
        rho[r] = s;
        if (r < n0) {
#pragma unroll
            for (int a = 0; a < 9; ++a) hown[a] = h[a];
        }
    }
    __syncthreads();

    // 2. recovered grad rho on rings <= 2 (k_grad)
    for (int32_t r = tid; r < n2; r += kPatch) {
        const int32_t g = A.node[base + r];
        const int32_t e0 = __ldg(m.rowptr + g), e1 = __ldg(m.rowptr + g + 1);
        const uint16_t *lc = A.lcol + A.rowbase[base + r];  // columns of e0 .. e1
        const T fi = rho[r];
        T sx = T(0), sy = T(0);
#pragma unroll 4
        for (int32_t e = e0; e < e1; ++e) {
            const int j = lc[e - e0];
            if (!chk_idx(j, n3, 2u)) continue;
            const T d = rho[j] - fi;
            sx += __ldg(m.ax + e) * d;
            sy += __ldg(m.ay + e) * d;
        }
        grd[r] = vset(sx, sy);
    }
    __syncthreads();

    // 3. lap rho and mu on rings <= 1, the stress force at the own node (k_mu)
    T kx_own = T(0), ky_own = T(0);
    for (int32_t r = tid; r < n1; r += kPatch) {
        const int32_t g = A.node[base + r];
        const int32_t e0 = __ldg(m.rowptr + g), e1 = __ldg(m.rowptr + g + 1);
        const uint16_t *lc = A.lcol + A.rowbase[base + r];  // columns of e0 .. e1
        const V2<T> gi = grd[r];
        const T gxi = gi.x, gyi = gi.y;
        T lap = T(0), kx = T(0), ky = T(0);
        double lap64 = 0.0;
#pragma unroll 4
        for (int32_t e = e0; e < e1; ++e) {
            const int j = lc[e - e0];
            if (!chk_idx(j, n2, 2u)) continue;
            const V2<T> gj = grd[j];
            const T gxj = gj.x, gyj = gj.y;
            T ax, ay;
            if (LAP64) {
                const double ax_ = __ldg(A.ax64 + e), ay_ = __ldg(A.ay64 + e);
                lap64 += ax_ * ((double)gxj - (double)gxi) + ay_ * ((double)gyj - (double)gyi);
                ax = (T)ax_;
                ay = (T)ay_;
            } else {
                ax = __ldg(m.ax + e);
                ay = __ldg(m.ay + e);
                lap += ax * (gxj - gxi) + ay * (gyj - gyi);
            }
            const T ddx = gxj - gxi, ddy = gyj - gyi;
            const T dxx = ddx * (gxj + gxi), dxy = gxj * ddy + gyi * ddx, dyy = ddy * (gyj + gyi);
            kx += ax * dyy - ay * dxy;
            ky += ay * dxx - ax * dxy;
        }
        if (LAP64)
            mu[r] = (T)((double)mu_bulk<T>(P, rho[r]) - A.kappa64 * lap64);
        else
            mu[r] = mu_bulk<T>(P, rho[r]) - P.kappa * lap;
        if (r < n0) {
            kx_own = P.kappa * kx;
            ky_own = P.kappa * ky;
        }
    }
    __syncthreads();

    // 4. own node: grad mu, g streamed and bounced back, collision (k_collide)
    if (tid >= n0) return;
    const int32_t r = tid, g = A.node[base + r];
    const int32_t e0 = __ldg(m.rowptr + g), e1 = __ldg(m.rowptr + g + 1);
    const uint16_t *lc = A.lcol + A.rowbase[base + r];  // columns of e0 .. e1
    T dmx, dmy;
    {
        const T fi = mu[r];
        T sx = T(0), sy = T(0);
#pragma unroll 4
        for (int32_t e = e0; e < e1; ++e) {
            const int j = lc[e - e0];
            if (!chk_idx(j, n1, 2u)) continue;
            const T d = mu[j] - fi;
            sx += __ldg(m.ax + e) * d;
            sy += __ldg(m.ay + e) * d;
        }
        dmx = sx;
        dmy = sy;
    }
    T gs[9];
    {
        V2<T> gsv[4], ga[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            gsv[q] = gP[q * r1max + r];
            ga[q] = vset(T(0), T(0));
        }
#pragma unroll 4
        for (int32_t e = e0; e < e1; ++e) {
            const int j = lc[e - e0];
            if (!chk_idx(j, n1, 2u)) continue;
            const T ax = __ldg(m.ax + e), ay = __ldg(m.ay + e);
            const T hbxx = hdt * __ldg(m.bxx + e), hbxy = hdt * __ldg(m.bxy + e), hbyy = hdt * __ldg(m.byy + e);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const V2<T> c = pair_coef<T>(q, ax, ay, hbxx, hbxy, hbyy);
                ga[q] = vfma(c, vfma(gsv[q], m1, gP[q * r1max + j]), ga[q]);
            }
        }
        V2<T> gp[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) gp[q] = vfma(mdt, ga[q], gsv[q]);
        unpack_pairs<T>(A.fin[9 * np + g], gp, gs);
    }
    {
        const int k = tg[r];
        if (k) bounce_back<T>(k, gs);
    }
    const V2<T> gr = grd[r];
    const T rr = rho[r];
    T hout[9], gout[9], ux, uy, pp;
    collide_node<T>(P, hown, gs, rr, gr.x, gr.y, dmx, dmy, kx_own, ky_own, hout, gout, ux, uy, pp);
    V2<T> *ho = reinterpret_cast<V2<T> *>(A.fout + np);
    V2<T> *go = reinterpret_cast<V2<T> *>(A.fout + 10 * np);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        ho[q * np + g] = vset(hout[pair_dir(q, 0)], hout[pair_dir(q, 1)]);
        go[q * np + g] = vset(gout[pair_dir(q, 0)], gout[pair_dir(q, 1)]);
    }
    A.fout[g] = hout[0];
    A.fout[9 * np + g] = gout[0];
    if (!(finite_val(rr) && finite_val(ux) && finite_val(uy) && finite_val(pp))) atomicOr(A.flag, 1);
    if (A.mom) {
        A.mom[g] = rr;
        A.mom[n + g] = ux;
        A.mom[2 * n + g] = uy;
        A.mom[3 * n + g] = pp;
    }
}

}  // namespace felbm
