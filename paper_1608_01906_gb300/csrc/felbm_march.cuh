// Structured-lattice step as a march along y: one launch per time step, each
// block owns a strip of 32 columns and sweeps a segment of rows upward, 8
// rows per iteration (k_lat_march).
//
// Per iteration with base row Y (rows are absolute mesh rows):
//   D  rows Y+3 .. Y+10: the h populations are streamed (Taylor-Galerkin,
//      Sec. 2.2.1) and bounced back at walls, rho = sum_a h_a; the streamed
//      h of the strip's own columns are kept for the collision;
//   G  rows Y+2 .. Y+9: recovered grad rho (Sec. 2.3);
//   M  rows Y+1 .. Y+8: lap rho and mu = mu_phi - kappa lap rho (Sec. 2.1);
//   F  rows Y .. Y+7: grad mu and the stress force, the g populations
//      streamed, the moments (Eqs. velocity, pressure) and the collision of
//      all 18 populations (Sec. 2.2), one write of each.
// Each stage reads the previous one's rows and the rows it kept from the
// iteration before: rho, grad rho, mu and the streamed h live in rings of 16
// rows in shared memory.  Only the x halo of the scalar chain (3 columns on
// each side) is computed twice, by the two strips that share it; the y halo
// is computed once per segment (a short prologue).  The tile step of
// felbm_lattice.cuh recomputes a depth-3 halo on all four sides of every
// 32 x 8 tile (2.08 times the tile for rho).
//
// Item layout: stages D, G and M map thread t to row t / 40 and column
// t % 40 of a 40-column window (columns x0-4 .. x0+35, the same for the h
// window and the rings), so that the 32 lanes of a warp read 32 consecutive
// shared-memory words (no bank conflicts); lanes outside a stage's columns
// idle.  F maps thread t < 256 to row t / 32 and column t % 32.
//
// Halo windows: the h window (4 pairs, rows Y+2 .. Y+11) and the h rest
// window (rows Y+3 .. Y+10) are requested as soon as stage D of the previous
// iteration is done, the g window (rows Y-1 .. Y+8) as soon as stage F of
// the previous iteration is done, by TMA (cp.async.bulk.tensor) on strips
// whose windows never wrap periodically, else by cp.async (zero-fill outside
// a walled domain, in both modes).  Waits for TMA are bounded; a wait that
// gives up sets flag bit 2 and the block stops after its pending loads.
#pragma once

#include "felbm_lattice.cuh"

namespace felbm {

constexpr int kMR = 8;                // rows per iteration
constexpr int kMX = 40;               // window / ring row width
constexpr int kMT = kMR * kMX;        // threads per block (320)
constexpr int kRing = 16;             // rows held by each ring
constexpr int kHWR = kMR + 2;         // rows of the h pair window
constexpr int kGWR = kMR + 2;         // rows of the g pair window

// Dynamic shared memory of one block (regions 128-byte aligned: TMA
// destinations first).
template <typename T>
struct MarchSmem {
    using PG = PairTile<T, 1>;
    static constexpr int GW = PG::W;    // g window columns: x0 - GXH ..
    static constexpr int GXH = PG::XH;
    static constexpr unsigned hW_bytes = 4 * kHWR * kMX * sizeof(V2<T>);
    static constexpr unsigned h0_bytes = kMR * kMX * sizeof(T);
    static constexpr unsigned gW_bytes = 4 * kGWR * GW * sizeof(V2<T>);
    static constexpr size_t hW = 0;
    static constexpr size_t h0 = align128(hW + hW_bytes);
    static constexpr size_t gW = align128(h0 + h0_bytes);
    static constexpr size_t rho = align128(gW + gW_bytes);                    // [16][40] T
    static constexpr size_t grad = align128(rho + kRing * kMX * sizeof(T));   // [16][40] V2
    static constexpr size_t mu = align128(grad + kRing * kMX * sizeof(V2<T>));  // [16][40] T
    static constexpr size_t psi = align128(mu + kRing * kMX * sizeof(T));     // [16][4][32] V2
    static constexpr size_t psi0 = align128(psi + kRing * 4 * 32 * sizeof(V2<T>));  // [16][32] T
    static constexpr size_t bytes = psi0 + kRing * 32 * sizeof(T);
};

template <typename T>
constexpr size_t march_smem() {
    return MarchSmem<T>::bytes;
}

// Arguments of the march (the tile step's, plus the segment length and the
// march's own tensor maps {h pairs, h rest, g pairs} of fin).
template <typename T>
struct MarchArgs {
    LatArgs<T> a;
    int32_t seg;        // rows per segment (a multiple of kMR); grid.y = ceil(ny / seg)
    int32_t uni;        // interior rows use the integer-weight operators below
    T al;               // 1 / (6 h)
    V2<T> ka;           // (-dt/(6h), dt/(6h)): odd part of the streaming weights
    V2<T> kb;           // (dt^2/(2h^2), dt^2/(2h^2)): even part
    const TMap *tmap;   // or nullptr
};

// ---- interior operators of the structured split --------------------------
// On a split of a lattice of spacing h, every node whose six neighbours are
// inside the mesh has the same assembled weights (felbm_mesh.cu reads them
// off the assembled operators, a_ij = sum |T| grad N_j / (3 m_i) and the
// symmetric part of b_ij = sum |T| / m_i grad N_i (x) grad N_j).  For the
// offsets o = (1,0), (1,1), (0,1), (-1,0), (-1,-1), (0,-1):
//   6h a_o = (2,-1), (1,1), (-1,2), (-2,1), (-1,-1), (1,-2)   (a_{o+3} = -a_o)
//   h^2 b_o (xx, xy, yy) = (-1,1/2,0), (0,-1/2,0), (0,1/2,-1), the same for o+3.
// With E_k = f(o_k) - f(o_{k+3}) and S_k = (f(o_k) - f) + (f(o_{k+3}) - f):
//   recovered gradient  R_x f = (2 E_0 + E_1 - E_2) / (6h),
//                       R_y f = (-E_0 + E_1 + 2 E_2) / (6h);
//   streaming of the pair q (directions e, -e):
//     psi* = psi + (-dt/(6h), dt/(6h)) (.) SA_q + dt^2/(2h^2) SB_q
//   with SA = e.(2E_0 + E_1 - E_2, -E_0 + E_1 + 2E_2) and SB = -sum_o
//   (e.(h^2 b_o).e) d_o:  q0 e = (1,0): SA = 2E_0 + E_1 - E_2, SB = S_0;
//   q1 (0,1): -E_0 + E_1 + 2E_2, S_2;  q2 (1,1): E_0 + 2E_1 + E_2, S_1;
//   q3 (-1,1): 3(E_2 - E_0), 2(S_0 + S_2) - S_1.
// Only differences of neighbouring values are rounded, as in the weighted
// difference form of the tables (exact for constant fields); no weight is
// loaded.  The host checks that the mesh's interior weights are these.

template <typename T>
__device__ __forceinline__ V2<T> vsub(V2<T> a, V2<T> b) {
    return vfma(b, vset(T(-1), T(-1)), a);
}

// streamed pair Q of the node at index c of a window with rows of W pairs
template <typename T, int W, int Q>
__device__ __forceinline__ V2<T> stream_uni(const V2<T> *b, int c, V2<T> ka, V2<T> kb) {
    const V2<T> s = b[c];
    const V2<T> n0 = b[c + 1], n1 = b[c + W + 1], n2 = b[c + W];
    const V2<T> n3 = b[c - 1], n4 = b[c - W - 1], n5 = b[c - W];
    const V2<T> two = vset(T(2), T(2));
    if (Q == 0) {
        const V2<T> SA = vfma(vsub<T>(n0, n3), two, vsub<T>(vsub<T>(n1, n4), vsub<T>(n2, n5)));
        const V2<T> SB = vadd(vsub<T>(n0, s), vsub<T>(n3, s));
        return vfma(ka, SA, vfma(kb, SB, s));
    } else if (Q == 1) {
        const V2<T> SA = vfma(vsub<T>(n2, n5), two, vsub<T>(vsub<T>(n1, n4), vsub<T>(n0, n3)));
        const V2<T> SB = vadd(vsub<T>(n2, s), vsub<T>(n5, s));
        return vfma(ka, SA, vfma(kb, SB, s));
    } else if (Q == 2) {
        const V2<T> SA = vfma(vsub<T>(n1, n4), two, vadd(vsub<T>(n0, n3), vsub<T>(n2, n5)));
        const V2<T> SB = vadd(vsub<T>(n1, s), vsub<T>(n4, s));
        return vfma(ka, SA, vfma(kb, SB, s));
    } else {
        const V2<T> d0 = vsub<T>(n0, s), d1 = vsub<T>(n1, s), d2 = vsub<T>(n2, s);
        const V2<T> d3 = vsub<T>(n3, s), d4 = vsub<T>(n4, s), d5 = vsub<T>(n5, s);
        const V2<T> S02 = vadd(vadd(d0, d3), vadd(d2, d5));
        const V2<T> SB = vsub<T>(vadd(S02, S02), vadd(d1, d4));
        const V2<T> SA = vsub<T>(vadd(d2, d3), vadd(d0, d5));  // E_2 - E_0
        return vfma(vmul(ka, vset(T(3), T(3))), SA, vfma(kb, SB, s));
    }
}

// (6h R_x f, 6h R_y f) from the six neighbour values
template <typename T>
__device__ __forceinline__ void rec_uni(T f0, T f1, T f2, T f3, T f4, T f5, T &rx, T &ry) {
    const T E0 = f0 - f3, E1 = f1 - f4, E2 = f2 - f5;
    rx = fma(T(2), E0, E1 - E2);
    ry = fma(T(2), E2, E1 - E0);
}

// Whether the interior weights of a structured mesh are those of the split
// of a lattice of spacing h that the integer-weight operators assume (a_o
// 6h and b_o h^2 to 1e-12 of their size); else every row uses the tables.
inline bool lattice_uniform(const StructuredInfo &si) {
    static const double A[6][2] = {{2, -1}, {1, 1}, {-1, 2}, {-2, 1}, {-1, -1}, {1, -2}};
    static const double B[6][3] = {{-1, 0.5, 0}, {0, -0.5, 0}, {0, 0.5, -1},
                                   {-1, 0.5, 0}, {0, -0.5, 0}, {0, 0.5, -1}};
    const double h = si.h;
    if (!(h > 0.0)) return false;
    for (int o = 0; o < 6; ++o) {
        for (int c = 0; c < 2; ++c) {
            const double d = si.a[0][o][c] * 6.0 * h - A[o][c];
            if (d > 1e-12 || d < -1e-12) return false;
        }
        for (int c = 0; c < 3; ++c) {
            const double d = si.b[0][o][c] * h * h - B[o][c];
            if (d > 1e-12 || d < -1e-12) return false;
        }
    }
    return true;
}

// The interior-operator constants of a mesh for time step dt.
template <typename T>
inline void march_consts(const StructuredInfo &si, double dt, MarchArgs<T> &M) {
    const double h = si.h;
    M.uni = lattice_uniform(si) ? 1 : 0;
    M.al = (T)(1.0 / (6.0 * h));
    const double ka = dt / (6.0 * h), kb = dt * dt / (2.0 * h * h);
    M.ka.x = (T)-ka;
    M.ka.y = (T)ka;
    M.kb.x = (T)kb;
    M.kb.y = (T)kb;
}

// Block state carried from iteration to iteration.
struct MarchPipe {
    unsigned ph_h = 0, ph_g = 0;  // parities of the next TMA phases
};

// cp.async fills of the h windows of the iteration with base row Y (out of
// line: the fill plans would otherwise stay live beside the stage values).
template <typename T>
__device__ __noinline__ void march_fill_h(const LatArgs<T> &A, int x0, int Y, unsigned char *dsm) {
    using L = MarchSmem<T>;
    using E = V2<T>;
    const int tid = threadIdx.x;
    const size_t np = pad4((size_t)A.pitch * A.ny);
    const E *src = reinterpret_cast<const E *>(A.fin + np);
    E *hW = reinterpret_cast<E *>(dsm + L::hW);
    T *h0 = reinterpret_cast<T *>(dsm + L::h0);
    if (vec_fills(x0, A.nx)) {
        fill_issue<E, true, 4>(
            fill_plan<E, kMX, kHWR, true>(tid, kMT, x0 - 4, Y + 2, A.nx, A.pitch, A.ny, A.walls), src, np, hW,
            kHWR * kMX);
        fill_issue<T, true, 1>(
            fill_plan<T, kMX, kMR, true>(tid, kMT, x0 - 4, Y + 3, A.nx, A.pitch, A.ny, A.walls), A.fin, 0, h0, 0);
    } else {
        fill_issue<E, false, 4>(
            fill_plan<E, kMX, kHWR, false>(tid, kMT, x0 - 4, Y + 2, A.nx, A.pitch, A.ny, A.walls), src, np, hW,
            kHWR * kMX);
        fill_issue<T, false, 1>(
            fill_plan<T, kMX, kMR, false>(tid, kMT, x0 - 4, Y + 3, A.nx, A.pitch, A.ny, A.walls), A.fin, 0, h0,
            0);
    }
    cp_async_commit();
}

// cp.async fills of the g window of the iteration with base row Y.
template <typename T>
__device__ __noinline__ void march_fill_g(const LatArgs<T> &A, int x0, int Y, unsigned char *dsm) {
    using L = MarchSmem<T>;
    using E = V2<T>;
    const int tid = threadIdx.x;
    const size_t np = pad4((size_t)A.pitch * A.ny);
    const E *src = reinterpret_cast<const E *>(A.fin + 10 * np);
    E *gW = reinterpret_cast<E *>(dsm + L::gW);
    if (vec_fills(x0, A.nx))
        fill_issue<E, true, 4>(
            fill_plan<E, L::GW, kGWR, true>(tid, kMT, x0 - L::GXH, Y - 1, A.nx, A.pitch, A.ny, A.walls), src, np,
            gW, kGWR * L::GW);
    else
        fill_issue<E, false, 4>(
            fill_plan<E, L::GW, kGWR, false>(tid, kMT, x0 - L::GXH, Y - 1, A.nx, A.pitch, A.ny, A.walls), src,
            np, gW, kGWR * L::GW);
    cp_async_commit();
}

// Request the h windows (4 pairs, rows Y+2 .. Y+11; rest, rows Y+3 .. Y+10)
// of the iteration with base row Y.
template <typename T, bool TMA>
__device__ __forceinline__ void march_issue_h(const MarchArgs<T> &M, int x0, int Y, unsigned char *dsm,
                                              uint64_t *bar) {
    using L = MarchSmem<T>;
    if (TMA) {
        if (threadIdx.x == 0) {
            constexpr int WPN = (int)sizeof(V2<T>) / 4, SPN = (int)sizeof(T) / 4;
            fence_proxy_async();
            mbar_expect_tx(bar, L::hW_bytes + L::h0_bytes);
            tma_load_3d(dsm + L::hW, M.tmap + 0, (x0 - 4) * WPN, Y + 2, 0, bar);
            tma_load_2d(dsm + L::h0, M.tmap + 1, (x0 - 4) * SPN, Y + 3, bar);
        }
    } else {
        march_fill_h<T>(M.a, x0, Y, dsm);
    }
}

// Request the g window (4 pairs, rows Y-1 .. Y+8) of the iteration with
// base row Y.
template <typename T, bool TMA>
__device__ __forceinline__ void march_issue_g(const MarchArgs<T> &M, int x0, int Y, unsigned char *dsm,
                                              uint64_t *bar) {
    using L = MarchSmem<T>;
    if (TMA) {
        if (threadIdx.x == 0) {
            constexpr int WPN = (int)sizeof(V2<T>) / 4;
            fence_proxy_async();
            mbar_expect_tx(bar, L::gW_bytes);
            tma_load_3d(dsm + L::gW, M.tmap + 2, (x0 - L::GXH) * WPN, Y - 1, 0, bar);
        }
    } else {
        march_fill_g<T>(M.a, x0, Y, dsm);
    }
}

// Bounded wait of this thread for a TMA phase; false when it gave up.
__device__ __forceinline__ bool march_wait(uint64_t *bar, unsigned parity) { return mbar_wait(bar, parity); }

// A bounded wait for a TMA load gave up (in some thread): record it, give
// each load still in flight (hpar / gpar: parity of the phase it completes,
// or -1) one more bounded wait, and stop the block (all threads alike).
template <typename T>
__device__ __noinline__ bool march_stop(const LatArgs<T> &A, uint64_t *bars, int hpar, int gpar) {
    if (threadIdx.x == 0) {
        atomicOr(A.flag, 4);
        if (hpar >= 0) mbar_wait(&bars[0], (unsigned)hpar);
        if (gpar >= 0) mbar_wait(&bars[1], (unsigned)gpar);
    }
    __syncthreads();
    return false;
}

// One iteration of the march with base row Y.  UNI: every row the stages
// compute is an interior row (kind 0; no wall row, none outside a walled
// domain) and the interior operators of the uniform split apply; otherwise
// the weights come from the tables of the row kinds.  PRO: the prologue
// before the first iteration of a segment starting at ya = Y + 8 (rho rows
// ya-3 .. ya+2, grad rows ya-2 .. ya+1, mu rows ya-1 .. ya; no collision).
// Returns false (all threads alike) when a bounded TMA wait gave up.
template <typename T, bool TMA, bool UNI, bool PRO>
__device__ __forceinline__ bool march_iter(const MarchArgs<T> &M, const LatCoef<T> &C, int x0, int Y, int yend,
                                           bool more, unsigned char *dsm, uint64_t *bars, MarchPipe &pp) {
    using L = MarchSmem<T>;
    const LatArgs<T> &A = M.a;
    const int tid = threadIdx.x;
    const int nx = A.nx, ny = A.ny, walls = A.walls;
    const T dt = A.P.dt;
    const V2<T> *hW = reinterpret_cast<const V2<T> *>(dsm + L::hW);
    const T *hR = reinterpret_cast<const T *>(dsm + L::h0);
    const V2<T> *gW = reinterpret_cast<const V2<T> *>(dsm + L::gW);
    T *rhoR = reinterpret_cast<T *>(dsm + L::rho);
    V2<T> *gradR = reinterpret_cast<V2<T> *>(dsm + L::grad);
    T *muR = reinterpret_cast<T *>(dsm + L::mu);
    V2<T> *psiR = reinterpret_cast<V2<T> *>(dsm + L::psi);
    T *psi0R = reinterpret_cast<T *>(dsm + L::psi0);
    const int sr = tid / kMX, sc = tid - (tid / kMX) * kMX;  // D, G, M item
    const size_t np = pad4((size_t)A.pitch * ny);
    // F item: row Y + fr, column x0 + fc; its g rest population is requested
    // now so that the load overlaps stages D, G and M
    const int fr = tid >> 5, fc = tid & 31;
    const int fx = x0 + fc, fy = Y + fr;
    const bool fvalid = !PRO && tid < 256 && fx < nx && fy < yend;
    const size_t fip = fvalid ? (size_t)fx + (size_t)A.pitch * fy : 0;
    T g0 = T(0);
    if (fvalid) g0 = __ldg(A.fin + 9 * np + fip);
    constexpr int RM = kRing - 1;
    // rows of kind 0 take the interior operators when the mesh has the
    // uniform weights (the choice depends on the row alone, never on the
    // segment or the iteration: results do not depend on the launch shape)
    const bool uni = M.uni != 0;

    // ---- D: rho rows Y+3 .. Y+10 -------------------------------------
    bool ok = true;
    if (TMA) {
        ok = march_wait(&bars[0], pp.ph_h);
        pp.ph_h ^= 1u;
    }
    {
        const int r = sr, c = sc;
        const int y = Y + 3 + r;
        if (c >= 1 && c < kMX - 1 && (!PRO || r >= 2)) {
            T rho = T(0);
            if (UNI || !walls || (y >= 0 && y < ny)) {
                const int cw = (r + 1) * kMX + c;
                const T rest = hR[r * kMX + c];
                const bool own = c >= 4 && c < 36;
                const int slot = y & RM;
                V2<T> v[4];
                const int k = UNI ? 0 : lat_kind(walls, y, ny);
                if (UNI || (uni && k == 0)) {
                    v[0] = stream_uni<T, kMX, 0>(hW + 0 * kHWR * kMX, cw, M.ka, M.kb);
                    v[1] = stream_uni<T, kMX, 1>(hW + 1 * kHWR * kMX, cw, M.ka, M.kb);
                    v[2] = stream_uni<T, kMX, 2>(hW + 2 * kHWR * kMX, cw, M.ka, M.kb);
                    v[3] = stream_uni<T, kMX, 3>(hW + 3 * kHWR * kMX, cw, M.ka, M.kb);
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        v[q] = bounce_pair<T>(k, q, stream_pair<T, kMX>(C, k, q, hW + q * kHWR * kMX, cw, dt));
                }
                rho = rest + ((v[0].x + v[0].y) + (v[1].x + v[1].y)) + ((v[2].x + v[2].y) + (v[3].x + v[3].y));
                if (own) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) psiR[(slot * 4 + q) * 32 + (c - 4)] = v[q];
                    psi0R[slot * 32 + (c - 4)] = rest;
                }
            }
            rhoR[(y & RM) * kMX + c] = rho;
        }
    }
    // the h load waited for may still be in flight, and so is the g load of
    // this iteration
    if (__syncthreads_or(!ok)) return march_stop<T>(A, bars, (int)(pp.ph_h ^ 1u), (int)pp.ph_g);
    // the h windows are dead: request the next iteration's
    if (more) march_issue_h<T, TMA>(M, x0, Y + kMR, dsm, &bars[0]);

    const auto &rc = C.r;
    const T al = M.al;
    // ---- G: grad rho rows Y+2 .. Y+9 ---------------------------------
    {
        const int r = sr, c = sc;
        const int y = Y + 2 + r;
        if (c >= 2 && c < kMX - 2 && (!PRO || r >= 4)) {
            const int b0 = (y & RM) * kMX + c;
            const int bm = ((y - 1) & RM) * kMX + c, bp = ((y + 1) & RM) * kMX + c;
            T sx, sy;
            const int k = (!UNI && walls && (y == 0 || y == ny - 1)) ? (y == 0 ? 1 : 2) : 0;
            if (UNI || (uni && k == 0)) {
                rec_uni<T>(rhoR[b0 + 1], rhoR[bp + 1], rhoR[bp], rhoR[b0 - 1], rhoR[bm - 1], rhoR[bm], sx, sy);
                sx *= al;
                sy *= al;
            } else {
                const T c0 = rhoR[b0];
                sx = T(0);
                sy = T(0);
#pragma unroll
                for (int o = 0; o < 6; ++o) {
                    const int b = lat_dy(o) < 0 ? bm : (lat_dy(o) > 0 ? bp : b0);
                    const T d = rhoR[b + lat_dx(o)] - c0;
                    sx += rc[k][o][0] * d;
                    sy += rc[k][o][1] * d;
                }
            }
            gradR[b0] = vset(sx, sy);
        }
    }
    __syncthreads();
    // ---- M: lap rho and mu rows Y+1 .. Y+8 ---------------------------
    const Phys<T> &P = A.P;
    {
        const int r = sr, c = sc;
        const int y = Y + 1 + r;
        if (c >= 3 && c < kMX - 3 && (!PRO || r >= 6)) {
            const int b0 = (y & RM) * kMX + c;
            const int bm = ((y - 1) & RM) * kMX + c, bp = ((y + 1) & RM) * kMX + c;
            T lap;
            const int k = (!UNI && walls && (y == 0 || y == ny - 1)) ? (y == 0 ? 1 : 2) : 0;
            if (UNI || (uni && k == 0)) {
                const V2<T> E0 = vsub<T>(gradR[b0 + 1], gradR[b0 - 1]);
                const V2<T> E1 = vsub<T>(gradR[bp + 1], gradR[bm - 1]);
                const V2<T> E2 = vsub<T>(gradR[bp], gradR[bm]);
                // R_x(d_x rho) + R_y(d_y rho)
                lap = al * (fma(T(2), E0.x, E1.x - E2.x) + fma(T(2), E2.y, E1.y - E0.y));
            } else {
                const V2<T> gc = gradR[b0];
                lap = T(0);
#pragma unroll
                for (int o = 0; o < 6; ++o) {
                    const int b = lat_dy(o) < 0 ? bm : (lat_dy(o) > 0 ? bp : b0);
                    const V2<T> gj = gradR[b + lat_dx(o)];
                    lap += rc[k][o][0] * (gj.x - gc.x) + rc[k][o][1] * (gj.y - gc.y);
                }
            }
            muR[b0] = mu_bulk<T>(P, rhoR[b0]) - P.kappa * lap;
        }
    }
    if (PRO) {
        // cp.async: the first iteration's g window and h window complete
        if (!TMA) cp_async_wait_group<0>();
        __syncthreads();
        return true;
    }
    if (!TMA) {
        // the g window of this iteration: every group but the h window
        // requested after stage D
        if (more)
            cp_async_wait_group<1>();
        else
            cp_async_wait_group<0>();
    }
    __syncthreads();
    // ---- F: grad mu, stress force, g streaming, collision rows Y .. Y+7 --
    if (TMA) {
        ok = march_wait(&bars[1], pp.ph_g);
        pp.ph_g ^= 1u;
    }
    if (tid < 256) {
        const int c = fc + 4;
        const int y = fy;
        const int b0 = (y & RM) * kMX + c;
        const int bm = ((y - 1) & RM) * kMX + c, bp = ((y + 1) & RM) * kMX + c;
        const int k = (UNI || !fvalid) ? 0 : lat_kind(walls, y, ny);
        T dmx, dmy, kx, ky;
        const bool urow = UNI || (uni && k == 0);
        if (urow) {
            rec_uni<T>(muR[b0 + 1], muR[bp + 1], muR[bp], muR[b0 - 1], muR[bm - 1], muR[bm], dmx, dmy);
            dmx *= al;
            dmy *= al;
            // differences of the gradient products across opposite
            // neighbours, in product form: (P.x, P.y) = E(d_x rho^2),
            // E(d_y rho^2); Q = E(d_x rho d_y rho)
            V2<T> Pk[3];
            T Qk[3];
            auto prod = [&](int j, V2<T> a, V2<T> b) {
                const V2<T> D = vsub<T>(a, b);
                Pk[j] = vmul(D, vadd(a, b));
                Qk[j] = fma(a.x, D.y, b.y * D.x);
            };
            prod(0, gradR[b0 + 1], gradR[b0 - 1]);
            prod(1, gradR[bp + 1], gradR[bm - 1]);
            prod(2, gradR[bp], gradR[bm]);
            // K_x = kappa [R_x(d_y rho^2) - R_y(d_x rho d_y rho)],
            // K_y = kappa [R_y(d_x rho^2) - R_x(d_x rho d_y rho)]
            const T rxy = fma(T(2), Pk[0].y, Pk[1].y - Pk[2].y), ryq = fma(T(2), Qk[2], Qk[1] - Qk[0]);
            const T ryx = fma(T(2), Pk[2].x, Pk[1].x - Pk[0].x), rxq = fma(T(2), Qk[0], Qk[1] - Qk[2]);
            const T ka = P.kappa * al;
            kx = ka * (rxy - ryq);
            ky = ka * (ryx - rxq);
        } else {
            T smx = T(0), smy = T(0), skx = T(0), sky = T(0);
            const T mc = muR[b0];
            const V2<T> gc = gradR[b0];
#pragma unroll
            for (int o = 0; o < 6; ++o) {
                const int b = (lat_dy(o) < 0 ? bm : (lat_dy(o) > 0 ? bp : b0)) + lat_dx(o);
                const T ax = rc[k][o][0], ay = rc[k][o][1];
                const T dm = muR[b] - mc;
                smx += ax * dm;
                smy += ay * dm;
                const V2<T> gj = gradR[b];
                const T ddx = gj.x - gc.x, ddy = gj.y - gc.y;  // product form, see k_mu
                const T dxx = ddx * (gj.x + gc.x), dxy = gj.x * ddy + gc.y * ddx, dyy = ddy * (gj.y + gc.y);
                skx += ax * dyy - ay * dxy;
                sky += ay * dxx - ax * dxy;
            }
            dmx = smx;
            dmy = smy;
            kx = P.kappa * skx;
            ky = P.kappa * sky;
        }
        const T r0 = rhoR[b0];
        const V2<T> dr = gradR[b0];
        if (fvalid) {
            const int slot = y & RM;
            const int cg = (fr + 1) * L::GW + fc + L::GXH;
            V2<T> gq[4];
            if (urow) {
                gq[0] = stream_uni<T, L::GW, 0>(gW + 0 * kGWR * L::GW, cg, M.ka, M.kb);
                gq[1] = stream_uni<T, L::GW, 1>(gW + 1 * kGWR * L::GW, cg, M.ka, M.kb);
                gq[2] = stream_uni<T, L::GW, 2>(gW + 2 * kGWR * L::GW, cg, M.ka, M.kb);
                gq[3] = stream_uni<T, L::GW, 3>(gW + 3 * kGWR * L::GW, cg, M.ka, M.kb);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    gq[q] = bounce_pair<T>(k, q, stream_pair<T, L::GW>(C, k, q, gW + q * kGWR * L::GW, cg, dt));
            }
            T sg, mx, my;
            g_moments<T>(g0, gq[0].x, gq[1].x, gq[0].y, gq[1].y, gq[2].x, gq[3].x, gq[2].y, gq[3].y, sg, mx, my);
            const CollidePrep<T> cp = collide_prep<T>(P, sg, mx, my, r0, dr.x, dr.y, dmx, dmy, kx, ky);
            const T h0 = psi0R[slot * 32 + fc];
            T dsum = T(0);
            V2<T> *hout = reinterpret_cast<V2<T> *>(A.fout + np);
            V2<T> *gout = reinterpret_cast<V2<T> *>(A.fout + 10 * np);
            auto pair_update = [&](auto qc) {
                constexpr int q = decltype(qc)::value;
                const V2<T> hs = psiR[(slot * 4 + q) * 32 + fc];
                V2<T> ho, go;
                collide_pair<T, q>(cp, hs, gq[q], ho, go);
                dsum += (ho.x - hs.x) + (ho.y - hs.y);
                hout[(size_t)q * np + fip] = ho;
                gout[(size_t)q * np + fip] = go;
            };
            pair_update(IntC<0>{});
            pair_update(IntC<1>{});
            pair_update(IntC<2>{});
            pair_update(IntC<3>{});
            {
                T ho, go;
                collide_pop_rt<T>(cp, 0, h0, g0, ho, go);
                dsum += ho - h0;
                A.fout[fip] = ho - dsum;
                A.fout[9 * np + fip] = go;
            }
            if (!(finite_val(cp.r) && finite_val(cp.ux) && finite_val(cp.uy) && finite_val(cp.p)))
                atomicOr(A.flag, 1);
            if (A.mom) {
                const size_t n = (size_t)nx * ny;
                const size_t i = (size_t)fx + (size_t)nx * y;
                A.mom[i] = cp.r;
                A.mom[n + i] = cp.ux;
                A.mom[2 * n + i] = cp.uy;
                A.mom[3 * n + i] = cp.p;
            }
        }
    }
    if (!TMA && more) {
        // the next h window (requested after stage D) is complete before
        // the barrier
        cp_async_wait_group<0>();
    }
    if (__syncthreads_or(!ok)) return march_stop<T>(A, bars, more ? (int)pp.ph_h : -1, (int)(pp.ph_g ^ 1u));
    // the g window is dead: request the next iteration's
    if (more) march_issue_g<T, TMA>(M, x0, Y + kMR, dsm, &bars[1]);
    return true;
}

// Whether a block's windows load by TMA: the strip's windows need no
// periodic wrap in x, and in y either the domain is walled (rows outside
// load as zeros) or no window of the segment (rows ya-6 .. ylast+11) wraps.
__device__ __forceinline__ bool march_tma_rows(int x0, int ya, int ylast, int nx, int ny, int walls) {
    return x0 >= 4 && x0 + 36 <= nx && (walls || (ya - 6 >= 0 && ylast + 11 <= ny - 1));
}

template <typename T, bool TMA>
__device__ __forceinline__ void march_block(const MarchArgs<T> &M, const LatCoef<T> &C, int x0, int ya, int yend,
                                            int niter, unsigned char *dsm, uint64_t *bars) {
    const LatArgs<T> &A = M.a;
    MarchPipe pp;
    // the prologue's h window and the first iteration's g window
    march_issue_h<T, TMA>(M, x0, ya - kMR, dsm, &bars[0]);
    march_issue_g<T, TMA>(M, x0, ya, dsm, &bars[1]);
    if (!TMA) {
        cp_async_wait_group<1>();
        __syncthreads();
    }
    if (!march_iter<T, TMA, false, true>(M, C, x0, ya - kMR, yend, true, dsm, bars, pp)) return;
    for (int j = 0; j < niter; ++j) {
        const int Y = ya + j * kMR;
        const bool more = j + 1 < niter;
        // every row computed (Y .. Y+10) of kind 0, with the uniform weights
        const bool uni = M.uni && (!A.walls || (Y >= 1 && Y + kMR + 2 <= A.ny - 2));
        const bool ok = uni ? march_iter<T, TMA, true, false>(M, C, x0, Y, yend, more, dsm, bars, pp)
                            : march_iter<T, TMA, false, false>(M, C, x0, Y, yend, more, dsm, bars, pp);
        if (!ok) return;
    }
}

// One time step: grid (ceil(nx / 32), ceil(ny / seg)), kMT threads, the
// dynamic shared memory of march_smem.
template <typename T>
__global__ void __launch_bounds__(kMT, sizeof(T) == 4 ? 3 : 2) k_lat_march(MarchArgs<T> M) {
    __shared__ __align__(8) uint64_t bars[2];
    extern __shared__ __align__(128) unsigned char march_dsm[];
    const LatArgs<T> &A = M.a;
    const int x0 = blockIdx.x * 32;
    const int ya = blockIdx.y * M.seg;
    const int yend = min(ya + M.seg, A.ny);
    const int niter = (yend - ya + kMR - 1) / kMR;
    const bool tma = M.tmap && march_tma_rows(x0, ya, ya + (niter - 1) * kMR, A.nx, A.ny, A.walls) &&
                     (smem_u32(march_dsm) & 127u) == 0;
    if (tma) {
        if (threadIdx.x == 0) {
            mbar_init(&bars[0], 1);
            mbar_init(&bars[1], 1);
            mbar_fence_init();
        }
        __syncthreads();
        march_block<T, true>(M, A.c, x0, ya, yend, niter, march_dsm, bars);
    } else {
        march_block<T, false>(M, A.c, x0, ya, yend, niter, march_dsm, bars);
    }
}

}  // namespace felbm
