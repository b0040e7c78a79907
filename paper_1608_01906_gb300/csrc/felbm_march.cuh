// Structured-lattice step as a march along y: one launch per time step, each
// block owns a strip of 32 columns and sweeps a segment of rows upward, 8
// rows per iteration (k_lat_march; k_batch_march runs the same march over
// the strips and segments of many meshes).
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
// rho, grad rho, mu and the streamed h live in rings of 32 rows in shared
// memory.  Only the x halo of the scalar chain (3 columns on each side) is
// computed twice, by the two strips that share it; the y halo once per
// segment (a short prologue).
//
// Warp specialisation: 5 producer warps run D, G and M (two items per
// thread: rows r and r + 4 of a 40-column window, columns x0-4 .. x0+35, so
// that a warp reads consecutive shared-memory words), 8 consumer warps run
// F (one node per thread).  The producers run up to two iterations ahead:
// mbarriers carry "rows of iteration j ready" (producer to consumer) and
// "iteration j collided" (consumer to producer, before the producers
// overwrite ring rows that iteration still reads).  Producer and consumer
// each synchronise among themselves with named barriers.
//
// Halo windows: the h window (4 pairs, rows Y+2 .. Y+11, and the rest
// population, rows Y+3 .. Y+10) is requested by the producers as soon as
// stage D of the previous iteration is done; the g window (rows Y-1 .. Y+8)
// is double-buffered and requested by the consumers two iterations ahead.
// Strips whose windows never wrap periodically load them by TMA
// (cp.async.bulk.tensor), the others by cp.async (zero-fill outside a walled
// domain in both modes).  Every wait is bounded; a wait that gives up sets
// flag bit 2 and the group stops after its pending loads.
#pragma once

#include "felbm_lattice.cuh"

namespace felbm {

constexpr int kMR = 8;                // rows per iteration
constexpr int kMX = 40;               // window / ring row width
constexpr int kRing = 32;             // rows held by each ring
constexpr int kHWR = kMR + 2;         // rows of the h pair window
constexpr int kGWR = kMR + 2;         // rows of the g pair window
constexpr int kPT = 160;              // producer threads: D, G, M
constexpr int kCT = 256;              // consumer threads: F
constexpr int kMT = kPT + kCT;        // threads per block
constexpr int kBarP = 1, kBarC = 2;   // named barriers of the two groups

// Dynamic shared memory of one block (regions 128-byte aligned: TMA
// destinations first).  The h window (4 pairs and the rest population) and
// the g window (4 pairs and the rest population of the own nodes) are each
// double-buffered.
template <typename T>
struct MarchSmem {
    using PG = PairTile<T, 1>;
    static constexpr int GW = PG::W;    // g window columns: x0 - GXH ..
    static constexpr int GXH = PG::XH;
    static constexpr unsigned hW_bytes = 4 * kHWR * kMX * sizeof(V2<T>);
    static constexpr unsigned h0_bytes = kMR * kMX * sizeof(T);
    static constexpr unsigned gW_bytes = 4 * kGWR * GW * sizeof(V2<T>);
    static constexpr unsigned g0_bytes = kMR * 32 * sizeof(T);
    // one h buffer: pairs, then the rest window
    static constexpr size_t hb_h0 = align128(hW_bytes);
    static constexpr size_t hb_stride = align128(hb_h0 + h0_bytes);
    // one g buffer: pairs, then the rest of the own nodes
    static constexpr size_t gb_g0 = align128(gW_bytes);
    static constexpr size_t gb_stride = align128(gb_g0 + g0_bytes);
    static constexpr size_t hW = 0;                                           // 2 h buffers
    static constexpr size_t gW = hW + 2 * hb_stride;                          // 2 g buffers
    static constexpr size_t rho = gW + 2 * gb_stride;                         // [32][40] T
    static constexpr size_t grad = align128(rho + kRing * kMX * sizeof(T));   // [32][40] V2
    static constexpr size_t mu = align128(grad + kRing * kMX * sizeof(V2<T>));  // [32][40] T
    static constexpr size_t psi = align128(mu + kRing * kMX * sizeof(T));     // [32][4][32] V2
    static constexpr size_t psi0 = align128(psi + kRing * 4 * 32 * sizeof(V2<T>));  // [32][32] T
    static constexpr size_t bytes = psi0 + kRing * 32 * sizeof(T);
};

template <typename T>
constexpr size_t march_smem() {
    return MarchSmem<T>::bytes;
}

// mbarriers of a block (static shared memory)
struct MarchBars {
    uint64_t h[2];      // h window buffers loaded (TMA)
    uint64_t g[2];      // g window buffers loaded (TMA)
    uint64_t ready[2];  // producer: rows of an iteration written (kPT arrivals)
    uint64_t done[2];   // consumer: an iteration collided (kCT arrivals)
};

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


// ---- synchronisation --------------------------------------------------

__device__ __forceinline__ void named_bar(int id, int n) {
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory");
}
// barrier of a group that also ORs a flag over it
__device__ __forceinline__ bool named_bar_or(int id, int n, bool v) {
    unsigned r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n"
        " selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((unsigned)v), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// ---- halo windows -----------------------------------------------------

// cp.async fills of the h windows of the iteration with base row Y into
// buffer b, by the producers (out of line: the fill plans would otherwise
// stay live beside the stage values).  Used when the state has no tensor
// maps; the windows are rectangles of slots (ghost columns and rows), in
// 16-byte chunks.
template <typename T>
__device__ __noinline__ void march_fill_h(const LatArgs<T> &A, int x0, int Y, unsigned char *dsm, int b, int t) {
    using L = MarchSmem<T>;
    using E = V2<T>;
    const size_t np = pad4((size_t)A.pitch * A.rows);
    const E *src = reinterpret_cast<const E *>(A.fin + np);
    E *hW = reinterpret_cast<E *>(dsm + L::hW + b * L::hb_stride);
    T *h0 = reinterpret_cast<T *>(dsm + L::hW + b * L::hb_stride + L::hb_h0);
    fill_issue<E, true, 4>(fill_plan_slots<E, kMX, kHWR, true>(t, kPT, x0, Y + 2 + A.gy, A.pitch, A.rows), src, np,
                           hW, kHWR * kMX);
    fill_issue<T, true, 1>(fill_plan_slots<T, kMX, kMR, true>(t, kPT, x0, Y + 3 + A.gy, A.pitch, A.rows), A.fin, 0,
                           h0, 0);
    cp_async_commit();
}

// cp.async fills of the g window of the iteration with base row Y into
// buffer b, by the consumers.
template <typename T>
__device__ __noinline__ void march_fill_g(const LatArgs<T> &A, int x0, int Y, unsigned char *dsm, int b, int t) {
    using L = MarchSmem<T>;
    using E = V2<T>;
    const size_t np = pad4((size_t)A.pitch * A.rows);
    const E *src = reinterpret_cast<const E *>(A.fin + 10 * np);
    E *gW = reinterpret_cast<E *>(dsm + L::gW + b * L::gb_stride);
    T *g0 = reinterpret_cast<T *>(dsm + L::gW + b * L::gb_stride + L::gb_g0);
    fill_issue<E, true, 4>(
        fill_plan_slots<E, L::GW, kGWR, true>(t, kCT, x0 + kGX - L::GXH, Y - 1 + A.gy, A.pitch, A.rows), src, np,
        gW, kGWR * L::GW);
    fill_issue<T, true, 1>(fill_plan_slots<T, 32, kMR, true>(t, kCT, x0 + kGX, Y + A.gy, A.pitch, A.rows),
                           A.fin + 9 * np, 0, g0, 0);
    cp_async_commit();
}

// Request the h windows of the iteration with base row Y into buffer b
// (producers; the caller has made sure that no producer reads buffer b).
template <typename T, bool TMA>
__device__ __forceinline__ void march_issue_h(const MarchArgs<T> &M, int x0, int Y, unsigned char *dsm,
                                              MarchBars &B, int b, int t) {
    using L = MarchSmem<T>;
    if (TMA) {
        if (t == 0) {
            constexpr int WPN = (int)sizeof(V2<T>) / 4, SPN = (int)sizeof(T) / 4;
            unsigned char *dst = dsm + L::hW + b * L::hb_stride;
            fence_proxy_async();
            mbar_expect_tx(&B.h[b], L::hW_bytes + L::h0_bytes);
            tma_load_3d(dst, M.tmap + 0, x0 * WPN, Y + 2 + M.a.gy, 0, &B.h[b]);
            tma_load_2d(dst + L::hb_h0, M.tmap + 1, x0 * SPN, Y + 3 + M.a.gy, &B.h[b]);
        }
    } else {
        march_fill_h<T>(M.a, x0, Y, dsm, b, t);
    }
}

// Request the g window of the iteration with base row Y into buffer b
// (consumers; the caller has made sure that no consumer reads buffer b).
template <typename T, bool TMA>
__device__ __forceinline__ void march_issue_g(const MarchArgs<T> &M, int x0, int Y, unsigned char *dsm,
                                              MarchBars &B, int b, int t) {
    using L = MarchSmem<T>;
    if (TMA) {
        if (t == 0) {
            constexpr int WPN = (int)sizeof(V2<T>) / 4, SPN = (int)sizeof(T) / 4;
            unsigned char *dst = dsm + L::gW + b * L::gb_stride;
            fence_proxy_async();
            mbar_expect_tx(&B.g[b], L::gW_bytes + L::g0_bytes);
            tma_load_3d(dst, M.tmap + 2, (x0 + kGX - L::GXH) * WPN, Y - 1 + M.a.gy, 0, &B.g[b]);
            tma_load_2d(dst + L::gb_g0, M.tmap + 3, (x0 + kGX) * SPN, Y + M.a.gy, &B.g[b]);
        }
    } else {
        march_fill_g<T>(M.a, x0, Y, dsm, b, t);
    }
}

// Iterations ahead of its use that a window is brought into L2: the loads
// into shared memory (two iterations ahead) then find it there.  Without
// it the two buffers of each window keep too few bytes in flight per SM to
// cover the latency of HBM.
constexpr int kPrefetch = 4;

// Bring the h and g windows of the iteration with base row Y into L2
// (TMA strips; one thread).
template <typename T>
__device__ __forceinline__ void march_prefetch(const MarchArgs<T> &M, int x0, int Y) {
    using L = MarchSmem<T>;
    constexpr int WPN = (int)sizeof(V2<T>) / 4, SPN = (int)sizeof(T) / 4;
    const int gy = M.a.gy;
    tma_prefetch_3d(M.tmap + 0, x0 * WPN, Y + 2 + gy, 0);
    tma_prefetch_2d(M.tmap + 1, x0 * SPN, Y + 3 + gy);
    tma_prefetch_3d(M.tmap + 2, (x0 + kGX - L::GXH) * WPN, Y - 1 + gy, 0);
    tma_prefetch_2d(M.tmap + 3, (x0 + kGX) * SPN, Y + gy);
}

// ---- stages -------------------------------------------------------------

// Whether every row an iteration with base row Y computes (Y .. Y+10) is an
// interior row with the uniform weights.
template <typename T>
__device__ __forceinline__ bool march_uni_rows(const MarchArgs<T> &M, int Y) {
    return M.uni && (!M.a.walls || (Y >= 1 && Y + kMR + 2 <= M.a.ny - 2));
}

// D: rho of row Y+3+r, column x0-4+c, and the streamed h of the own columns.
// UNI: the row is interior with the uniform weights; otherwise the row's kind
// decides (interior rows still take the interior operators when the mesh has
// the uniform weights, so a node's arithmetic never depends on the iteration
// that computes it).
template <typename T, bool UNI>
__device__ __forceinline__ void stage_d(const MarchArgs<T> &M, const LatCoef<T> &C, unsigned char *dsm,
                                        const unsigned char *hbuf, int Y, int r, int c) {
    using L = MarchSmem<T>;
    const LatArgs<T> &A = M.a;
    const int ny = A.ny, walls = A.walls;
    const int y = Y + 3 + r;
    if (c < 1 || c >= kMX - 1) return;
    const V2<T> *hW = reinterpret_cast<const V2<T> *>(hbuf);
    const T *hR = reinterpret_cast<const T *>(hbuf + L::hb_h0);
    T *rhoR = reinterpret_cast<T *>(dsm + L::rho);
    V2<T> *psiR = reinterpret_cast<V2<T> *>(dsm + L::psi);
    T *psi0R = reinterpret_cast<T *>(dsm + L::psi0);
    constexpr int RM = kRing - 1;
    T rho = T(0);
    if (UNI || !walls || (y >= 0 && y < ny)) {
        const int cw = (r + 1) * kMX + c;
        const T rest = hR[r * kMX + c];
        const bool own = c >= 4 && c < 36;
        const int slot = y & RM;
        V2<T> v[4];
        const int k = UNI ? 0 : lat_kind(walls, y, ny);
        if (UNI || (M.uni && k == 0)) {
            v[0] = stream_uni<T, kMX, 0>(hW + 0 * kHWR * kMX, cw, M.ka, M.kb);
            v[1] = stream_uni<T, kMX, 1>(hW + 1 * kHWR * kMX, cw, M.ka, M.kb);
            v[2] = stream_uni<T, kMX, 2>(hW + 2 * kHWR * kMX, cw, M.ka, M.kb);
            v[3] = stream_uni<T, kMX, 3>(hW + 3 * kHWR * kMX, cw, M.ka, M.kb);
        } else {
            const T dt = A.P.dt;
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

// G: grad rho of row Y+2+r, column x0-4+c.
template <typename T, bool UNI>
__device__ __forceinline__ void stage_g(const MarchArgs<T> &M, const LatCoef<T> &C, unsigned char *dsm, int Y,
                                        int r, int c) {
    using L = MarchSmem<T>;
    if (c < 2 || c >= kMX - 2) return;
    const int ny = M.a.ny, walls = M.a.walls;
    const int y = Y + 2 + r;
    const T *rhoR = reinterpret_cast<const T *>(dsm + L::rho);
    V2<T> *gradR = reinterpret_cast<V2<T> *>(dsm + L::grad);
    constexpr int RM = kRing - 1;
    const int b0 = (y & RM) * kMX + c;
    const int bm = ((y - 1) & RM) * kMX + c, bp = ((y + 1) & RM) * kMX + c;
    T sx, sy;
    const int k = (!UNI && walls && (y == 0 || y == ny - 1)) ? (y == 0 ? 1 : 2) : 0;
    if (UNI || (M.uni && k == 0)) {
        rec_uni<T>(rhoR[b0 + 1], rhoR[bp + 1], rhoR[bp], rhoR[b0 - 1], rhoR[bm - 1], rhoR[bm], sx, sy);
        sx *= M.al;
        sy *= M.al;
    } else {
        const auto &rc = C.r;
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

// M: lap rho and mu of row Y+1+r, column x0-4+c.
template <typename T, bool UNI>
__device__ __forceinline__ void stage_m(const MarchArgs<T> &M, const LatCoef<T> &C, unsigned char *dsm, int Y,
                                        int r, int c) {
    using L = MarchSmem<T>;
    if (c < 3 || c >= kMX - 3) return;
    const int ny = M.a.ny, walls = M.a.walls;
    const int y = Y + 1 + r;
    const T *rhoR = reinterpret_cast<const T *>(dsm + L::rho);
    const V2<T> *gradR = reinterpret_cast<const V2<T> *>(dsm + L::grad);
    T *muR = reinterpret_cast<T *>(dsm + L::mu);
    constexpr int RM = kRing - 1;
    const int b0 = (y & RM) * kMX + c;
    const int bm = ((y - 1) & RM) * kMX + c, bp = ((y + 1) & RM) * kMX + c;
    T lap;
    const int k = (!UNI && walls && (y == 0 || y == ny - 1)) ? (y == 0 ? 1 : 2) : 0;
    if (UNI || (M.uni && k == 0)) {
        const V2<T> E0 = vsub<T>(gradR[b0 + 1], gradR[b0 - 1]);
        const V2<T> E1 = vsub<T>(gradR[bp + 1], gradR[bm - 1]);
        const V2<T> E2 = vsub<T>(gradR[bp], gradR[bm]);
        // R_x(d_x rho) + R_y(d_y rho)
        lap = M.al * (fma(T(2), E0.x, E1.x - E2.x) + fma(T(2), E2.y, E1.y - E0.y));
    } else {
        const auto &rc = C.r;
        const V2<T> gc = gradR[b0];
        lap = T(0);
#pragma unroll
        for (int o = 0; o < 6; ++o) {
            const int b = lat_dy(o) < 0 ? bm : (lat_dy(o) > 0 ? bp : b0);
            const V2<T> gj = gradR[b + lat_dx(o)];
            lap += rc[k][o][0] * (gj.x - gc.x) + rc[k][o][1] * (gj.y - gc.y);
        }
    }
    muR[b0] = mu_bulk<T>(M.a.P, rhoR[b0]) - M.a.P.kappa * lap;
}

// Slot of ghost copy k (1 .. 8) of node (x, y), or -1: copy k takes the
// x image k % 3 (0 the node's own x; 1 x + nx if gmask bit 0, x < kGX; 2
// x - nx if bit 1, x >= nx - kGX) and the y image k / 3 (bits 2 and 3 the
// same in y, with ghost rows only).
template <typename T>
__device__ __forceinline__ long long ghost_slot(const LatArgs<T> &A, unsigned gmask, int x, int y, int k) {
    const int a = k % 3, b = k / 3;
    if ((a == 1 && !(gmask & 1u)) || (a == 2 && !(gmask & 2u)) || (b == 1 && !(gmask & 4u)) ||
        (b == 2 && !(gmask & 8u)))
        return -1;
    const int xx = a == 0 ? x : (a == 1 ? x + A.nx : x - A.nx);
    const int yy = b == 0 ? y : (b == 1 ? y + A.ny : y - A.ny);
    return (long long)(xx + kGX) + (long long)A.pitch * (yy + A.gy);
}

// F: node (x0 + fc, Y + fr): grad mu, stress force, g streaming from window
// buffer gWb, moments and collision, one write of its 18 populations.
template <typename T, bool UNI>
__device__ __forceinline__ void stage_f(const MarchArgs<T> &M, const LatCoef<T> &C, unsigned char *dsm,
                                        const unsigned char *gbuf, int x0, int Y, int yend, int fr, int fc) {
    using L = MarchSmem<T>;
    const LatArgs<T> &A = M.a;
    const int nx = A.nx, ny = A.ny, walls = A.walls;
    const int fx = x0 + fc, y = Y + fr;
    const bool fvalid = fx < nx && y < yend;
    const T *rhoR = reinterpret_cast<const T *>(dsm + L::rho);
    const V2<T> *gradR = reinterpret_cast<const V2<T> *>(dsm + L::grad);
    const T *muR = reinterpret_cast<const T *>(dsm + L::mu);
    const V2<T> *psiR = reinterpret_cast<const V2<T> *>(dsm + L::psi);
    const T *psi0R = reinterpret_cast<const T *>(dsm + L::psi0);
    constexpr int RM = kRing - 1;
    const Phys<T> &P = A.P;
    const int c = fc + 4;
    const int b0 = (y & RM) * kMX + c;
    const int bm = ((y - 1) & RM) * kMX + c, bp = ((y + 1) & RM) * kMX + c;
    const int k = (UNI || !fvalid) ? 0 : lat_kind(walls, y, ny);
    const bool urow = UNI || (M.uni && k == 0);
    T dmx, dmy, kx, ky;
    if (urow) {
        const T al = M.al;
        rec_uni<T>(muR[b0 + 1], muR[bp + 1], muR[bp], muR[b0 - 1], muR[bm - 1], muR[bm], dmx, dmy);
        dmx *= al;
        dmy *= al;
        // differences of the gradient products across opposite neighbours,
        // in product form: (P.x, P.y) = E(d_x rho^2), E(d_y rho^2);
        // Q = E(d_x rho d_y rho)
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
        const auto &rc = C.r;
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
    if (!fvalid) return;
    const V2<T> *gWb = reinterpret_cast<const V2<T> *>(gbuf);
    const T g0 = reinterpret_cast<const T *>(gbuf + L::gb_g0)[fr * 32 + fc];
    const T r0 = rhoR[b0];
    const V2<T> dr = gradR[b0];
    const size_t np = pad4((size_t)A.pitch * A.rows);
    const size_t fip = (size_t)(fx + kGX) + (size_t)A.pitch * (y + A.gy);
    // copies kept in ghost slots (nodes within kGX of a periodic edge): the
    // x image, the y image and the corner, as offsets from the node's slot;
    // on meshes narrower than 2 kGX a node can have two images in one
    // direction (rare: the general loop below)
    const unsigned gmask = (fx < kGX ? 1u : 0u) | (fx >= nx - kGX ? 2u : 0u) |
                           (A.gy && y < kGX ? 4u : 0u) | (A.gy && y >= ny - kGX ? 8u : 0u);
    const bool grare = (gmask & 3u) == 3u || (gmask & 12u) == 12u;
    long long go1 = 0, go2 = 0, go3 = 0;
    if (gmask && !grare) {
        const long long dxg = (gmask & 1u) ? nx : ((gmask & 2u) ? -nx : 0);
        const long long dyg = ((gmask & 4u) ? ny : ((gmask & 8u) ? -ny : 0)) * (long long)A.pitch;
        go1 = dxg;
        go2 = dyg;
        go3 = (dxg && dyg) ? dxg + dyg : 0;
    }
    const int slot = y & RM;
    const int cg = (fr + 1) * L::GW + fc + L::GXH;
    V2<T> gq[4];
    if (urow) {
        gq[0] = stream_uni<T, L::GW, 0>(gWb + 0 * kGWR * L::GW, cg, M.ka, M.kb);
        gq[1] = stream_uni<T, L::GW, 1>(gWb + 1 * kGWR * L::GW, cg, M.ka, M.kb);
        gq[2] = stream_uni<T, L::GW, 2>(gWb + 2 * kGWR * L::GW, cg, M.ka, M.kb);
        gq[3] = stream_uni<T, L::GW, 3>(gWb + 3 * kGWR * L::GW, cg, M.ka, M.kb);
    } else {
        const T dt = P.dt;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            gq[q] = bounce_pair<T>(k, q, stream_pair<T, L::GW>(C, k, q, gWb + q * kGWR * L::GW, cg, dt));
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
        if (gmask) {
            // ghost copies (edge nodes only)
            const size_t b = (size_t)q * np + fip;
            if (go1) {
                hout[b + go1] = ho;
                gout[b + go1] = go;
            }
            if (go2) {
                hout[b + go2] = ho;
                gout[b + go2] = go;
            }
            if (go3) {
                hout[b + go3] = ho;
                gout[b + go3] = go;
            }
            if (grare) {
#pragma unroll 1
                for (int k = 1; k < 9; ++k) {
                    const long long sl = ghost_slot<T>(A, gmask, fx, y, k);
                    if (sl < 0) continue;
                    hout[(size_t)q * np + (size_t)sl] = ho;
                    gout[(size_t)q * np + (size_t)sl] = go;
                }
            }
        }
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
        if (gmask) {
            const T hr = ho - dsum;
            if (go1) {
                A.fout[fip + go1] = hr;
                A.fout[9 * np + fip + go1] = go;
            }
            if (go2) {
                A.fout[fip + go2] = hr;
                A.fout[9 * np + fip + go2] = go;
            }
            if (go3) {
                A.fout[fip + go3] = hr;
                A.fout[9 * np + fip + go3] = go;
            }
            if (grare) {
#pragma unroll 1
                for (int k = 1; k < 9; ++k) {
                    const long long sl = ghost_slot<T>(A, gmask, fx, y, k);
                    if (sl < 0) continue;
                    A.fout[(size_t)sl] = hr;
                    A.fout[9 * np + (size_t)sl] = go;
                }
            }
        }
    }
    if (!(finite_val(cp.r) && finite_val(cp.ux) && finite_val(cp.uy) && finite_val(cp.p))) atomicOr(A.flag, 1);
    if (A.mom) {
        const size_t n = (size_t)nx * ny;
        const size_t i = (size_t)fx + (size_t)nx * y;
        A.mom[i] = cp.r;
        A.mom[n + i] = cp.ux;
        A.mom[2 * n + i] = cp.uy;
        A.mom[3 * n + i] = cp.p;
    }
}

// ---- the two groups -----------------------------------------------------

// A wait of the group gave up: record it, give the group's loads still in
// flight one more bounded wait (TMA), and stop the group.
template <typename T>
__device__ __noinline__ void march_give_up(const LatArgs<T> &A, uint64_t *bar0, int par0, uint64_t *bar1,
                                           int par1, bool lead) {
    if (lead) {
        atomicOr(A.flag, 4);
        if (bar0) mbar_wait(bar0, (unsigned)par0);
        if (bar1) mbar_wait(bar1, (unsigned)par1);
    }
}

// Producers (threads 0 .. kPT-1): prologue, then D, G, M of every
// iteration, up to two iterations ahead of the consumers.  h window loads:
// number 0 for the prologue, j + 1 for iteration j, into buffer (number & 1),
// each requested two loads ahead.
template <typename T, bool TMA>
__device__ __forceinline__ void march_producer(const MarchArgs<T> &M, const LatCoef<T> &C, int x0, int ya,
                                               int niter, unsigned char *dsm, MarchBars &B) {
    using L = MarchSmem<T>;
    const int t = threadIdx.x;
    const int r = t / kMX, c = t - (t / kMX) * kMX;  // items (r, c) and (r + 4, c)
    // the prologue's h window (rows ya-6 .. ya+3) and the first iteration's
    march_issue_h<T, TMA>(M, x0, ya - kMR, dsm, B, 0, t);
    march_issue_h<T, TMA>(M, x0, ya, dsm, B, 1, t);
    if (TMA && t == 0)
        for (int q = 2; q < 2 + kPrefetch && q < niter; ++q) march_prefetch<T>(M, x0, ya + q * kMR);
    bool ok = true;
    // prologue: rho rows ya-3 .. ya+2, grad rows ya-2 .. ya+1, mu rows ya-1 .. ya
    {
        const int Y = ya - kMR;
        if (TMA) {
            ok = mbar_wait(&B.h[0], 0u);
        } else {
            cp_async_wait_group<1>();
            named_bar(kBarP, kPT);
        }
        const unsigned char *hb = dsm + L::hW;
        if (r >= 2) stage_d<T, false>(M, C, dsm, hb, Y, r, c);
        stage_d<T, false>(M, C, dsm, hb, Y, r + 4, c);
        if (named_bar_or(kBarP, kPT, !ok)) {
            march_give_up<T>(M.a, TMA ? &B.h[0] : nullptr, 0, TMA ? &B.h[1] : nullptr, 0, t == 0);
            return;
        }
        if (niter > 1) march_issue_h<T, TMA>(M, x0, ya + kMR, dsm, B, 0, t);
        stage_g<T, false>(M, C, dsm, Y, r + 4, c);
        named_bar(kBarP, kPT);
        if (r >= 2) stage_m<T, false>(M, C, dsm, Y, r + 4, c);
    }
    for (int j = 0; j < niter; ++j) {
        const int Y = ya + j * kMR;
        const int b = (j + 1) & 1;                        // buffer of load j + 1
        const unsigned ph = (unsigned)(((j + 1) >> 1) & 1);
        // ring rows of iteration j - 2 are overwritten from here on
        if (j >= 2) ok = mbar_wait(&B.done[j & 1], (unsigned)(((j - 2) >> 1) & 1));
        if (TMA) {
            ok = mbar_wait(&B.h[b], ph) && ok;
        } else {
            // pending: this window and, unless last, the next one
            if (j + 1 < niter)
                cp_async_wait_group<1>();
            else
                cp_async_wait_group<0>();
            named_bar(kBarP, kPT);
        }
        const unsigned char *hb = dsm + L::hW + b * L::hb_stride;
        const bool uni = march_uni_rows(M, Y);
        if (uni) {
            stage_d<T, true>(M, C, dsm, hb, Y, r, c);
            stage_d<T, true>(M, C, dsm, hb, Y, r + 4, c);
        } else {
            stage_d<T, false>(M, C, dsm, hb, Y, r, c);
            stage_d<T, false>(M, C, dsm, hb, Y, r + 4, c);
        }
        if (named_bar_or(kBarP, kPT, !ok)) {
            march_give_up<T>(M.a, TMA ? &B.h[b] : nullptr, (int)ph, (TMA && j + 1 < niter) ? &B.h[b ^ 1] : nullptr,
                             (int)(((j + 2) >> 1) & 1), t == 0);
            return;
        }
        // buffer b is free: the window of iteration j + 2
        if (j + 2 < niter) march_issue_h<T, TMA>(M, x0, Y + 2 * kMR, dsm, B, b, t);
        if (TMA && t == 0 && j + 2 + kPrefetch < niter) march_prefetch<T>(M, x0, Y + (2 + kPrefetch) * kMR);
        if (uni) {
            stage_g<T, true>(M, C, dsm, Y, r, c);
            stage_g<T, true>(M, C, dsm, Y, r + 4, c);
        } else {
            stage_g<T, false>(M, C, dsm, Y, r, c);
            stage_g<T, false>(M, C, dsm, Y, r + 4, c);
        }
        named_bar(kBarP, kPT);
        if (uni) {
            stage_m<T, true>(M, C, dsm, Y, r, c);
            stage_m<T, true>(M, C, dsm, Y, r + 4, c);
        } else {
            stage_m<T, false>(M, C, dsm, Y, r, c);
            stage_m<T, false>(M, C, dsm, Y, r + 4, c);
        }
        // rows of iteration j in the rings (each thread releases its own writes)
        mbar_arrive(&B.ready[j & 1]);
    }
}

// Consumers (threads kPT .. kMT-1): F of every iteration, the g windows two
// iterations ahead.
template <typename T, bool TMA>
__device__ __forceinline__ void march_consumer(const MarchArgs<T> &M, const LatCoef<T> &C, int x0, int ya,
                                               int yend, int niter, unsigned char *dsm, MarchBars &B) {
    using L = MarchSmem<T>;
    const LatArgs<T> &A = M.a;
    const int t = threadIdx.x - kPT;
    const int fr = t >> 5, fc = t & 31;
    march_issue_g<T, TMA>(M, x0, ya, dsm, B, 0, t);
    if (niter > 1) march_issue_g<T, TMA>(M, x0, ya + kMR, dsm, B, 1, t);
    for (int j = 0; j < niter; ++j) {
        const int Y = ya + j * kMR;
        const int b = j & 1;
        const unsigned ph = (unsigned)((j >> 1) & 1);
        bool ok = mbar_wait(&B.ready[b], ph);
        if (TMA) {
            ok = mbar_wait(&B.g[b], ph) && ok;
        } else {
            // pending: this window and, unless last, the next one
            if (j + 1 < niter)
                cp_async_wait_group<1>();
            else
                cp_async_wait_group<0>();
        }
        if (named_bar_or(kBarC, kCT, !ok)) {
            march_give_up<T>(A, TMA ? &B.g[b] : nullptr, (int)ph, (TMA && j + 1 < niter) ? &B.g[b ^ 1] : nullptr,
                             (int)(((j + 1) >> 1) & 1), t == 0);
            return;
        }
        const unsigned char *gb = dsm + L::gW + b * L::gb_stride;
        if (march_uni_rows(M, Y))
            stage_f<T, true>(M, C, dsm, gb, x0, Y, yend, fr, fc);
        else
            stage_f<T, false>(M, C, dsm, gb, x0, Y, yend, fr, fc);
        // iteration j collided (each thread releases its reads of the rings)
        mbar_arrive(&B.done[b]);
        if (j + 2 < niter) {
            // buffer b is free once every consumer is done with it
            if (TMA) {
                // (a wait that gives up leaves the window unrequested: every
                // consumer then gives up at its next bounded wait, together)
                if (t == 0) {
                    if (mbar_wait(&B.done[b], ph))
                        march_issue_g<T, TMA>(M, x0, Y + 2 * kMR, dsm, B, b, t);
                    else
                        atomicOr(A.flag, 4);
                }
            } else {
                named_bar(kBarC, kCT);
                march_issue_g<T, TMA>(M, x0, Y + 2 * kMR, dsm, B, b, t);
            }
        }
    }
}


// Initialise the block's mbarriers (thread 0; the caller synchronises).
__device__ __forceinline__ void march_bars_init(MarchBars &B) {
    mbar_init(&B.h[0], 1);
    mbar_init(&B.h[1], 1);
    mbar_init(&B.g[0], 1);
    mbar_init(&B.g[1], 1);
    mbar_init(&B.ready[0], kPT);
    mbar_init(&B.ready[1], kPT);
    mbar_init(&B.done[0], kCT);
    mbar_init(&B.done[1], kCT);
    mbar_fence_init();
}

// One block's march over rows ya .. yend-1 of the strip at x0 (after the
// barriers are initialised and visible to every thread).
template <typename T>
__device__ __forceinline__ void march_block(const MarchArgs<T> &M, const LatCoef<T> &C, int x0, int ya, int yend,
                                            unsigned char *dsm, MarchBars &B) {
    const int niter = (yend - ya + kMR - 1) / kMR;
    // every window is a rectangle of slots (ghost columns and rows): TMA
    // boxes whenever the state has tensor maps
    const bool tma = M.tmap && (smem_u32(dsm) & 127u) == 0;
    if (threadIdx.x < kPT) {
        if (tma)
            march_producer<T, true>(M, C, x0, ya, niter, dsm, B);
        else
            march_producer<T, false>(M, C, x0, ya, niter, dsm, B);
    } else {
        if (tma)
            march_consumer<T, true>(M, C, x0, ya, yend, niter, dsm, B);
        else
            march_consumer<T, false>(M, C, x0, ya, yend, niter, dsm, B);
    }
}

// One time step: grid (ceil(nx / 32), ceil(ny / seg)), kMT threads, the
// dynamic shared memory of march_smem.
template <typename T>
__global__ void __launch_bounds__(kMT, sizeof(T) == 4 ? 2 : 1) k_lat_march(MarchArgs<T> M) {
    __shared__ MarchBars B;
    extern __shared__ __align__(128) unsigned char march_dsm[];
    if (threadIdx.x == 0) march_bars_init(B);
    __syncthreads();
    const int x0 = blockIdx.x * 32;
    const int ya = blockIdx.y * M.seg;
    const int yend = min(ya + M.seg, M.a.ny);
    march_block<T>(M, M.a.c, x0, ya, yend, march_dsm, B);
}

}  // namespace felbm
