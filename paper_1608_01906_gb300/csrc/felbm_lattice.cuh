// Structured-lattice step: one launch per time step, one 32 x 8 tile of
// nodes per block (k_lat_step).
//
//   1. the 4 h pair tiles (halo depth 4) and the h rest tile are staged in
//      shared memory; the h populations are streamed (Taylor-Galerkin,
//      Sec. 2.2.1) and bounced back at walls on the tile's depth-3 halo, and
//      rho = sum_a h_a there; the tile's own streamed h pairs are kept;
//   2. grad rho (depth 2), lap rho and mu (depth 1), then grad mu and the
//      stress force at the tile's nodes (Sec. 2.3 recovery, Sec. 2.1 mu,
//      stress form);
//   3. the g pairs are streamed from depth-1 tiles, the moments formed and
//      all populations collided (Sec. 2.2); one write of the 18 populations.
//
// The density stage recomputes the streaming of h on the halo instead of a
// separate density launch: neighbouring tiles share no data within a step.
// Opposite directions (a, abar) are stored interleaved (pop_index): the
// stencil of a pair reads one 8-byte (FP32) word per neighbour and runs in
// packed two-wide arithmetic (FFMA2 on sm_103a), each lane with its own
// coefficient.  Population rows are stored with a pitch of nx rounded up to
// a multiple of 4 slots, so every row starts 16-byte aligned.  Halo windows
// that need no periodic wrap arrive as TMA boxes, the others by cp.async
// (16-byte chunks unless a chunk would straddle the wrap of a row whose
// length is not a multiple of 4); all are requested when the block starts,
// and the g tiles arrive while rho and the scalar chain are computed.
//
// Coefficient tables: for each row kind (interior, bottom wall row, top wall
// row), offset o and pair q, the streaming coefficients of the pair's two
// directions
//   s[k][o][q] = (e_a . a_o + dt/2 e_a . b_o . e_a,  same for abar)
// and the recovery coefficients r[k][o] = a_o, read off the assembled
// operators of the mesh (zero for offsets outside a walled domain).
#pragma once

#include "felbm_internal.h"
#include "felbm_kernels.cuh"

namespace felbm {

constexpr int kLTX = 32, kLTY = 8;  // tile of nodes per block

template <int V>
struct IntC {
    static constexpr int value = V;
};

template <typename T>
struct LatCoef {
    V2<T> s[3][6][4];  // streaming coefficients per kind, offset, pair
    T r[3][6][2];      // recovery coefficients
};

template <typename T>
struct LatArgs {
    int32_t nx, ny, walls;
    int32_t pitch;  // population row pitch (slots), nx rounded up to a multiple of 4
    // storage row r is row r + row0 of the whole lattice of gny rows (wall
    // rows and the outside of a walled domain are decided on those rows);
    // the tiles cover the storage rows [ylo, yhi).  A whole lattice has
    // row0 = ylo = 0 and gny = yhi = ny; a slab of a sharded lattice keeps
    // depth-4 halo rows on both sides of its rows.
    int32_t row0, gny, ylo, yhi;
    LatCoef<T> c;
    Phys<T> P;
    const T *fin;
    T *fout;
    T *rho;  // unused by the lattice step (rho is formed per tile)
    T *mom;  // 4N or nullptr
    int *flag;
    const TMap *tmap;  // {h pairs, h rest, g pairs} of fin, or nullptr
    // interior operators of the uniform split (below): used on interior
    // tiles when uni is set (the host checked the mesh's interior weights)
    int32_t uni;
    T al;        // 1 / (6 h)
    V2<T> ka;    // (-dt/(6h), dt/(6h)): odd part of the streaming weights
    V2<T> kb;    // (dt^2/(2h^2), dt^2/(2h^2)): even part
    // FP64 kappa lap rho term of mu (FELBM_PARAM_LAP_FP64; read only by the
    // kernel built for it): 1/(6h), kappa and the recovery coefficients
    double al64, kappa64;
    double r64[3][6][2];
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
// loaded.  Opposite offsets carry opposite recovery weights, so a recovered
// derivative needs three differences instead of six.

template <typename T>
__device__ __forceinline__ V2<T> vsub(V2<T> a, V2<T> b) {
    return vfma(b, vset(T(-1), T(-1)), a);
}

// streamed pair Q of a node from its own value s and its neighbours n_o at
// the offsets o = (1,0), (1,1), (0,1), (-1,0), (-1,-1), (0,-1)
template <typename T, int Q>
__device__ __forceinline__ V2<T> stream_uni_v(V2<T> s, V2<T> n0, V2<T> n1, V2<T> n2, V2<T> n3, V2<T> n4,
                                              V2<T> n5, V2<T> ka, V2<T> kb) {
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

// streamed pair Q of the node at index c of a window with rows of W pairs
template <typename T, int W, int Q>
__device__ __forceinline__ V2<T> stream_uni(const V2<T> *b, int c, V2<T> ka, V2<T> kb) {
    return stream_uni_v<T, Q>(b[c], b[c + 1], b[c + W + 1], b[c + W], b[c - 1], b[c - W - 1], b[c - W], ka, kb);
}

// The same for three nodes stacked in one column, from 13 loads instead of
// 21: rb[j] is the offset of the window row holding y - 1 + j (j = 0 .. 4,
// y the first node's row), c the column.
template <typename T, int Q>
__device__ __forceinline__ void stream_uni3(const V2<T> *b, const int *rb, int c, V2<T> ka, V2<T> kb, V2<T> *out) {
    V2<T> cx[5], cl[4], cr[4];
#pragma unroll
    for (int j = 0; j < 5; ++j) cx[j] = b[rb[j] + c];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        cl[j] = b[rb[j] + c - 1];
        cr[j] = b[rb[j + 1] + c + 1];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
        out[i] = stream_uni_v<T, Q>(cx[i + 1], cr[i], cr[i + 1], cx[i + 2], cl[i + 1], cl[i], cx[i], ka, kb);
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
// 6h and b_o h^2 to 1e-12 of their size); else every tile uses the tables.
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
inline void lat_uniform_consts(const StructuredInfo &si, double dt, LatArgs<T> &A) {
    const double h = si.h;
    A.uni = lattice_uniform(si) ? 1 : 0;
    A.al = (T)(1.0 / (6.0 * h));
    const double ka = dt / (6.0 * h), kb = dt * dt / (2.0 * h * h);
    A.ka.x = (T)-ka;
    A.ka.y = (T)ka;
    A.kb.x = (T)kb;
    A.kb.y = (T)kb;
}

__device__ __forceinline__ int lat_kind(int walls, int y, int ny) {
    return walls ? (y == 0 ? 1 : (y == ny - 1 ? 2 : 0)) : 0;
}

// ---- halo windows filled with cp.async ---------------------------------

// Window of H rows x W elements of type E (a population pair, or a scalar)
// around the block's tile.  Fill plan of one thread: up to kMaxSlots slots,
// each a global element offset and a shared element offset; a slot outside
// a walled domain copies zero bytes (cp.async zero-fills it).  VEC: the
// slots are 16-byte chunks (window without x wrap, rows 16-byte aligned).
constexpr int kMaxSlots = 3;
struct FillPlan {
    int32_t src[kMaxSlots];
    int32_t dst[kMaxSlots];
    int8_t ok[kMaxSlots];
    int n;
};

template <typename E, int W, int H, bool VEC>
__device__ __forceinline__ FillPlan fill_plan(int tid, int nthreads, int gx0, int gy0, int nx, int pitch, int ny,
                                              int walls, int row0, int gny) {
    constexpr int CE = 16 / (int)sizeof(E);
    constexpr int PER_ROW = VEC ? W / CE : W;
    constexpr int TOTAL = PER_ROW * H;
    FillPlan f;
    f.n = 0;
#pragma unroll
    for (int t = 0; t < kMaxSlots; ++t) {
        const int q = tid + t * nthreads;
        f.src[t] = 0;
        f.dst[t] = 0;
        f.ok[t] = 0;
        if (q < TOTAL) {
            const int r = q / PER_ROW, c = q - r * PER_ROW;
            const int col = VEC ? c * CE : c;
            int gx = gx0 + col, gy = gy0 + r;
            while (gx < 0) gx += nx;  // a halo may span more than one period
            while (gx >= nx) gx -= nx;
            bool inside = true;
            if (walls) {
                // (a storage row past a slab's halo only feeds nodes outside
                // the slab's rows: zero-filled like the outside)
                inside = gy + row0 >= 0 && gy + row0 < gny && gy >= 0 && gy < ny;
            } else {
                while (gy < 0) gy += ny;
                while (gy >= ny) gy -= ny;
            }
            f.src[t] = inside ? gx + pitch * gy : 0;
            f.ok[t] = inside;
            f.dst[t] = r * W + col;
            // (checked build: a slot outside the window or the arrays copies
            // nothing and zero-fills the window's first element)
            if (!chk_idx(f.src[t], (long long)pitch * ny, 1u) || !chk_idx(f.dst[t], W * H, 2u)) {
                f.src[t] = 0;
                f.dst[t] = 0;
                f.ok[t] = 0;
            }
            f.n = t + 1;
        }
    }
    return f;
}

// cp.async of one slot; a zero source size fills the destination with zeros.
template <typename E, bool VEC>
__device__ __forceinline__ void cp_async_zfill(E *smem, const E *gmem, bool ok) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    constexpr int BYTES = VEC ? 16 : (int)sizeof(E);
    const int ssz = ok ? BYTES : 0;
    if (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(ssz)
                     : "memory");
    else if (BYTES == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(ssz)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(ssz)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N committed groups of this thread are still pending
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---- halo windows loaded by TMA -----------------------------------------

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make barrier initialisation visible to the async proxy
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// Wait for the phase of the given parity to complete; each try_wait is
// itself time-limited, and the wait gives up after kMbarTries tries or
// limit_ns nanoseconds of the global timer, whichever comes first: false
// when it gave up.
constexpr unsigned kMbarTries = 1u << 20;
constexpr uint64_t kMbarLimitNs = 2000000000ull;  // 2 s
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_try(unsigned a, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    return done != 0;
}
static __device__ __noinline__ bool mbar_wait_slow(unsigned a, unsigned parity, uint64_t limit_ns) {
    const uint64_t t0 = global_ns();
    for (unsigned it = 0; it < kMbarTries; ++it) {
        if (mbar_try(a, parity)) return true;
        if ((it & 63u) == 63u && global_ns() - t0 > limit_ns) return false;
    }
    return false;
}
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, uint64_t limit_ns = kMbarLimitNs) {
    const unsigned a = smem_u32(bar);
    if (mbar_try(a, parity)) return true;
    return mbar_wait_slow(a, parity, limit_ns);
}
// Block-wide wait for a TMA load group: the first warp polls the barrier,
// the others wait at the block barrier (no issue slots spent polling).
// True when the phase completed, the same in every thread.
__device__ __forceinline__ bool block_mbar_wait(uint64_t *bar, unsigned parity) {
    const bool ok = threadIdx.y != 0 || mbar_wait(bar, parity);
    return !__syncthreads_or(!ok);
}

// order this thread's earlier generic-proxy shared accesses (as released to
// it by a barrier) before later async-proxy writes
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void tma_load_2d(void *dst, const TMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const TMap *map, int x, int y, int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Request NF windows (src + f * src_stride -> dst + f * dst_stride).
template <typename E, bool VEC, int NF>
__device__ __forceinline__ void fill_issue(const FillPlan &f, const E *__restrict__ src, size_t src_stride,
                                           E *dst, int dst_stride) {
#pragma unroll
    for (int t = 0; t < kMaxSlots; ++t) {
        if (t < f.n) {
            const E *s = src + f.src[t];
            E *d = dst + f.dst[t];
            const bool ok = f.ok[t];
#pragma unroll
            for (int q = 0; q < NF; ++q) cp_async_zfill<E, VEC>(d + q * dst_stride, s + q * src_stride, ok);
        }
    }
}

// Halo tile of one population pair with D rows of halo above and below and
// XH >= D columns left and right; XH is D rounded up to whole 16-byte chunks
// of pairs, so rows start 16-byte aligned.
template <typename T, int D>
struct PairTile {
    static constexpr int CE = 16 / (int)sizeof(V2<T>);
    static constexpr int XH = (D + CE - 1) / CE * CE;
    static constexpr int W = kLTX + 2 * XH;
    static constexpr int H = kLTY + 2 * D;
    static constexpr int N = W * H;
};

// Request the depth-D halo tiles of the 4 pairs of h (G = 0) or g (G = 1).
// VEC: 16-byte chunks (needs a window without x wrap, or nx % 4 == 0, so
// that no chunk straddles the wrap).
template <typename T, int G, int D, bool VEC>
__device__ __forceinline__ void issue_pair_tiles(const LatArgs<T> &A, int tid, int x0, int y0,
                                                 V2<T> *tiles, size_t np) {
    using E = V2<T>;
    using PT = PairTile<T, D>;
    const E *src = reinterpret_cast<const E *>(A.fin + (G ? 10 : 1) * np);  // pair 0; pair q at + q np
    const FillPlan f =
        fill_plan<E, PT::W, PT::H, VEC>(tid, kLTX * kLTY, x0 - PT::XH, y0 - D, A.nx, A.pitch, A.ny, A.walls,
                                        A.row0, A.gny);
    fill_issue<E, VEC, 4>(f, src, np, tiles, PT::N);
}

// Streamed values of pair q of the node whose element in the halo tile buf
// (rows of W elements) is c, at row kind k:
// psi* = psi - dt sum_o s_o (psi(node + o) - psi(node)), both directions in
// one packed operation per offset.
template <typename T, int W>
__device__ __forceinline__ V2<T> stream_pair(const LatCoef<T> &cf, int k, int q, const V2<T> *buf, int c,
                                             T dt) {
    const V2<T> self = buf[c];
    const V2<T> m1 = vset(T(-1), T(-1));
    V2<T> acc = vset(T(0), T(0));
#pragma unroll
    for (int o = 0; o < 6; ++o) {
        const V2<T> nb = buf[c + lat_dy(o) * W + lat_dx(o)];
        const V2<T> d = vfma(self, m1, nb);  // nb - self, exact negation
        acc = vfma(cf.s[k][o][q], d, acc);
    }
    return vfma(vset(-dt, -dt), acc, self);
}

// Collision of the opposite pair q = (a, abar) of one node (see
// collide_pop): e_abar = -e_a and w_abar = w_a, so the odd parts (e.u, e.X,
// e.grad rho, e.K, e.du) flip sign between the two lanes and the even parts
// are shared; the two lanes run in packed two-wide arithmetic.
template <typename T, int Q>
__device__ __forceinline__ void collide_pair(const CollidePrep<T> &c, V2<T> hs, V2<T> gs, V2<T> &ho,
                                             V2<T> &go) {
    constexpr int A = pair_dir(Q, 0);
    constexpr int ex = kEx(A), ey = kEy(A);
    constexpr T wa = kW<T>(A), w3 = kW3<T>(A);
    const T eu = T(ex) * c.ux + T(ey) * c.uy;
    const T eX = T(ex) * c.Xx + T(ey) * c.Xy;
    const T eD = T(ex) * c.drx + T(ey) * c.dry;
    const T eK = T(ex) * c.kx + T(ey) * c.ky;
    const T edu = T(ex) * c.dux + T(ey) * c.duy;
    // Gamma - w = 3w (e.u + 1.5 (e.u)^2 - 0.5 u.u), formed without the w
    // offset (FP32: keeps the momentum part); 3w from kW3
    const T even = T(1.5) * eu * eu - T(0.5) * c.uu;
    const V2<T> gmw = vfma(vset(w3, w3), vset(eu, -eu), vset(w3 * even, w3 * even));
    const V2<T> gam3 = vfma(vset(T(3), T(3)), gmw, vset(w3, w3));  // 3 Gamma
    const V2<T> Fa = vmul(vset(c.hdt * (eX - c.uX), c.hdt * (-eX - c.uX)), gam3);
    const V2<T> Ga = vfma(vset(c.hdt * (eD - c.uD), c.hdt * (-eD - c.uD)), gmw,
                          vmul(vset(c.hdt * (eK - c.uK), c.hdt * (-eK - c.uK)), gam3));
    // 1/2 [g_eq(u + du) - g_eq(u)] = rho/2 [Gamma(u + du) - Gamma(u)]
    const T bev = T(1.5) * edu * (T(2) * eu + edu) - T(0.5) * c.udu;
    const T hrw = T(0.5) * c.r * w3;
    const V2<T> Sg = vfma(vset(hrw, hrw), vset(edu + bev, bev - edu), Ga);
    const V2<T> rg = vmul(vset(c.r, c.r), gmw);
    const V2<T> dh = vadd(vfma(vset(c.r, c.r), vset(wa, wa), vset(-hs.x, -hs.y)), rg);  // h_eq - h*
    const V2<T> dg = vadd(vfma(vset(w3, w3), vset(c.p, c.p), vset(-gs.x, -gs.y)), rg);  // g_eq - g*
    ho = vadd(hs, vfma(vset(c.omw, c.omw), dh, vmul(vset(c.opw, c.opw), Fa)));
    go = vadd(gs, vfma(vset(c.omw, c.omw), dg, vmul(vset(c.opw, c.opw), Sg)));
}

// Bounce-back of a pair at a wall row of kind k (1: inward normal +y, the
// slot-0 directions 2, 5, 6 of pairs 1..3 take their opposites; 2: normal
// -y, the slot-1 directions 4, 7, 8 take theirs).
template <typename T>
__device__ __forceinline__ V2<T> bounce_pair(int k, int q, V2<T> v) {
    if (k == 0 || q == 0) return v;
    return k == 1 ? vset(v.y, v.y) : vset(v.x, v.x);
}

// ---- one step of a tile ---------------------------------------------------

constexpr int kHD = 4;                            // depth of the h pair tiles
constexpr int kH0W = kLTX + 8, kH0H = kLTY + 6;   // h rest tile: from (x0 - 4, y0 - 3)
constexpr int kQW = kLTX + 6, kQH = kLTY + 6;     // rho region: halo 3
constexpr int kRW = kLTX + 8, kRH = kLTY + 6;     // rho: rows from x0 - 4 (column 0, 39 unused)
constexpr int kGW = kLTX + 4, kGH = kLTY + 4;     // grad rho: halo 2
constexpr int kMW = kLTX + 2, kMH = kLTY + 2;     // mu: halo 1
constexpr int kNT = kLTX * kLTY;
// row groups of three of the blocked stages on interior tiles (one pass each)
// (rows per thread: kGR in the gradient stage, kMR in the mu stage)
constexpr int kGR = 3, kMR = 3;
constexpr int kDG = (kQH + 2) / 3, kGG = (kGH + kGR - 1) / kGR, kMG = (kMH + kMR - 1) / kMR;
static_assert(kRW * kDG <= kNT && kRW * kGG <= kNT && kRW * kMG <= kNT, "one pass per blocked stage");

// Shared memory of one tile: the scalar chain (static) and the population
// tiles (dynamic, lat_smem bytes).  The streamed g pairs stay in registers.
template <typename T>
struct __align__(16) StepSmem {
    uint64_t bar[2];  // TMA completion: h tiles, g tiles
    int nt[4];        // the block's next tile as claimed by thread 0: index, bx, by, flags
    T s_rho[kRH][kRW];
    V2<T> s_g[kGH][kGW];  // recovered grad rho, (x, y) interleaved
    T s_mu[kMH][kMW];
};

constexpr size_t align128(size_t b) { return (b + 127) / 128 * 128; }

// Regions of the dynamic shared memory, each 128-byte aligned (TMA
// destinations).  The byte sizes of the h tiles (pairs + rest) and of the g
// tiles are what one TMA load group delivers.
template <typename T>
struct LatSmem {
    using PH = PairTile<T, kHD>;
    using PG = PairTile<T, 1>;
    static constexpr unsigned hT_bytes = 4 * PH::N * sizeof(V2<T>);
    static constexpr unsigned h0_bytes = kH0W * kH0H * sizeof(T);
    static constexpr unsigned gT_bytes = 4 * PG::N * sizeof(V2<T>);
    static constexpr size_t hT = 0;                             // 4 h pair tiles
    static constexpr size_t h0 = align128(hT + hT_bytes);      // h rest tile
    static constexpr size_t gT = align128(h0 + h0_bytes);      // 4 g pair tiles
    static constexpr size_t psi = align128(gT + gT_bytes);     // streamed h pairs
    static constexpr size_t bytes = psi + 4 * (size_t)kNT * sizeof(V2<T>);
};

template <typename T>
constexpr size_t lat_smem() {
    return LatSmem<T>::bytes;
}

// Whether the halo windows of a tile at x0 may be filled in 16-byte chunks:
// rows are 16-byte aligned (pitch), so unless a window wraps around a row
// whose length is not a multiple of 4.
__device__ __forceinline__ bool vec_fills(int x0, int nx) {
    return (nx % 4) == 0 || (x0 >= kHD && x0 + kLTX + kHD <= nx);
}

// Whether tile (x0, y0) is whole (no node outside the mesh), its rho region
// and h tiles hold no wall row nor a row outside a walled domain, and rows
// are 16-byte aligned: such tiles run with the row kind fixed at compile
// time and vector fills only.
template <typename T>
__device__ __forceinline__ bool tile_interior(const LatArgs<T> &A, int x0, int y0) {
    const int g0 = y0 + A.row0;  // the tile's first row in the whole lattice
    const bool yin = y0 + kLTY <= A.yhi && (!A.walls || (g0 >= kHD && g0 + kLTY + kHD <= A.gny));
    return A.uni && yin && x0 + kLTX <= A.nx && vec_fills(x0, A.nx);
}

// Whether the halo windows of tile (x0, y0) lie inside the mesh without a
// periodic wrap: a TMA box then covers each of them.
__device__ __forceinline__ bool tile_unwrapped(int x0, int y0, int nx, int ny) {
    return x0 >= kHD && x0 + kLTX + kHD <= nx && y0 >= kHD && y0 + kLTY + kHD <= ny;
}

// Collision of one node: the g pairs are streamed here from their depth-1
// tiles, the h pairs were streamed by the density stage.
template <typename T, bool UNI>
__device__ __forceinline__ void lat_node(const LatArgs<T> &A, const LatCoef<T> &C, int k, int lx, int ly,
                                         int tid, int32_t i,
                                         size_t ip, size_t n, size_t np, T h0, T g0, T r0, T drx, T dry,
                                         T dmx, T dmy, T kx, T ky, const V2<T> *gT,
                                         const V2<T> (*s_psi)[kNT]) {
    using PG = PairTile<T, 1>;
    const Phys<T> &P = A.P;
    const int c = (ly + 1) * PG::W + lx + PG::XH;
    V2<T> gq[4];
    if (UNI) {
        gq[0] = stream_uni<T, PG::W, 0>(gT + 0 * PG::N, c, A.ka, A.kb);
        gq[1] = stream_uni<T, PG::W, 1>(gT + 1 * PG::N, c, A.ka, A.kb);
        gq[2] = stream_uni<T, PG::W, 2>(gT + 2 * PG::N, c, A.ka, A.kb);
        gq[3] = stream_uni<T, PG::W, 3>(gT + 3 * PG::N, c, A.ka, A.kb);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            gq[q] = bounce_pair<T>(k, q, stream_pair<T, PG::W>(C, k, q, gT + q * PG::N, c, P.dt));
    }
    T sg, mx, my;
    // g_1 = q0.x, g_3 = q0.y, g_2 = q1.x, g_4 = q1.y, g_5 = q2.x, g_7 = q2.y, g_6 = q3.x, g_8 = q3.y
    g_moments<T>(g0, gq[0].x, gq[1].x, gq[0].y, gq[1].y, gq[2].x, gq[3].x, gq[2].y, gq[3].y, sg, mx, my);
    const CollidePrep<T> cp = collide_prep<T>(P, sg, mx, my, r0, drx, dry, dmx, dmy, kx, ky);
    const T r = cp.r, ux = cp.ux, uy = cp.uy, p = cp.p;
    // pairs, then the rest population, which also takes the sum of the h
    // increments (zero in exact arithmetic): the collision then keeps the
    // node's mass to one rounding instead of accumulating the rounding of the
    // nine source terms every step
    T dsum = T(0);
    V2<T> *hout = reinterpret_cast<V2<T> *>(A.fout + np);
    V2<T> *gout = reinterpret_cast<V2<T> *>(A.fout + 10 * np);
    auto pair_update = [&](auto qc) {
        constexpr int q = decltype(qc)::value;
        const V2<T> hs = s_psi[q][tid];
        V2<T> ho, go;
        collide_pair<T, q>(cp, hs, gq[q], ho, go);
        dsum += (ho.x - hs.x) + (ho.y - hs.y);
        hout[(size_t)q * np + ip] = ho;
        gout[(size_t)q * np + ip] = go;
    };
    pair_update(IntC<0>{});
    pair_update(IntC<1>{});
    pair_update(IntC<2>{});
    pair_update(IntC<3>{});
    {
        T ho, go;
        collide_pop_rt<T>(cp, 0, h0, g0, ho, go);
        dsum += ho - h0;
        A.fout[ip] = ho - dsum;
        A.fout[9 * np + ip] = go;
    }
    if (!(finite_val(r) && finite_val(ux) && finite_val(uy) && finite_val(p))) atomicOr(A.flag, 1);
    if (A.mom) {
        A.mom[i] = r;
        A.mom[n + i] = ux;
        A.mom[2 * n + i] = uy;
        A.mom[3 * n + i] = p;
    }
}

// TMA state of a block walking its tiles (same value in every thread).
struct TilePipe {
    unsigned ph[2] = {0u, 0u};  // parity of the next phase of bar[0] (h group), bar[1] (g group)
    bool h_issued = false;      // the current tile's h group was requested during the previous tile
};

// The block's next tile (known to thread 0 only): its h group is requested
// as soon as the current tile has formed rho (tma: it loads by TMA, from
// the same mesh).  Thread 0 publishes it in S.nt (flags: bit 0 valid, bit 1
// h group requested) for the whole block after the tile.
struct NextTile {
    int t, bx, by;
    bool valid, tma;
};

// Request the h group (4 h pair tiles + the rest tile) of tile (x0, y0).
template <typename T>
__device__ __forceinline__ void issue_h_group(const LatArgs<T> &A, int x0, int y0, StepSmem<T> &S,
                                              unsigned char *dsm) {
    using L = LatSmem<T>;
    using PH = PairTile<T, kHD>;
    constexpr int WPN = (int)sizeof(V2<T>) / 4, SPN = (int)sizeof(T) / 4;  // 4-byte words per element
    fence_proxy_async();
    mbar_expect_tx(&S.bar[0], L::hT_bytes + L::h0_bytes);
    tma_load_3d(dsm + L::hT, A.tmap + 0, (x0 - PH::XH) * WPN, y0 - kHD, 0, &S.bar[0]);
    tma_load_2d(dsm + L::h0, A.tmap + 1, (x0 - 4) * SPN, y0 - 3, &S.bar[0]);
}

// Request the g group (4 g pair tiles) of tile (x0, y0).
template <typename T>
__device__ __forceinline__ void issue_g_group(const LatArgs<T> &A, int x0, int y0, StepSmem<T> &S,
                                              unsigned char *dsm) {
    using L = LatSmem<T>;
    using PG = PairTile<T, 1>;
    constexpr int WPN = (int)sizeof(V2<T>) / 4;
    fence_proxy_async();
    mbar_expect_tx(&S.bar[1], L::gT_bytes);
    tma_load_3d(dsm + L::gT, A.tmap + 2, (x0 - PG::XH) * WPN, y0 - 1, 0, &S.bar[1]);
}

// A bounded wait for a TMA load ran out: record it, give the loads still in
// flight one more bounded wait each, and stop (all threads alike).
template <typename T>
__device__ __noinline__ bool tma_gave_up(const LatArgs<T> &A, StepSmem<T> &S, const TilePipe &pp) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        atomicOr(A.flag, 4);
        mbar_wait(&S.bar[0], pp.ph[0]);
        mbar_wait(&S.bar[1], pp.ph[1]);
    }
    __syncthreads();
    return false;
}

// One time step of tile (bx, by).  TMA: the halo windows come as TMA boxes
// (tile_unwrapped, interior tiles) completing on S.bar, else as cp.async
// fills.  C: the mesh's coefficient tables (kernel parameters where they
// can be, so that interior tiles read them as constant operands).  Returns
// false (all threads alike) when a bounded wait for a TMA load gave up; the
// flag then carries bit 2.
template <typename T, bool INTERIOR, bool TMA, bool LAP64>
__device__ __forceinline__ bool lat_tile_impl(const LatArgs<T> &A, const LatCoef<T> &C, int bx, int by,
                                              StepSmem<T> &S, unsigned char *dsm, TilePipe &pp,
                                              const NextTile &next) {
    using L = LatSmem<T>;
    using PH = PairTile<T, kHD>;
    auto &s_rho = S.s_rho;
    auto &s_g = S.s_g;
    auto &s_mu = S.s_mu;
    V2<T> *hT = reinterpret_cast<V2<T> *>(dsm + L::hT);
    T(*s_h0)[kH0W] = reinterpret_cast<T(*)[kH0W]>(dsm + L::h0);
    V2<T> *gT = reinterpret_cast<V2<T> *>(dsm + L::gT);
    V2<T>(*s_psi)[kNT] = reinterpret_cast<V2<T>(*)[kNT]>(dsm + L::psi);
    const int nx = A.nx, ny = A.ny, walls = A.walls;
    const int x0 = bx * kLTX, y0 = A.ylo + by * kLTY;
    const int tid = threadIdx.y * kLTX + threadIdx.x;
    const size_t n = (size_t)nx * ny, np = pad4((size_t)A.pitch * ny);
    const T dt = A.P.dt;
    // 0. request the h pair tiles (depth 4) and the h rest tile (depth 3) as
    //    group 1, the g pair tiles (depth 1) as group 2; the g tiles arrive
    //    while rho and the scalar chain are computed
    if (TMA) {
        if (tid == 0) {
            if (!pp.h_issued) issue_h_group<T>(A, x0, y0, S, dsm);
            issue_g_group<T>(A, x0, y0, S, dsm);
        }
    } else if (INTERIOR || vec_fills(x0, nx)) {
        issue_pair_tiles<T, 0, kHD, true>(A, tid, x0, y0, hT, np);
        fill_issue<T, true, 1>(fill_plan<T, kH0W, kH0H, true>(tid, kNT, x0 - 4, y0 - 3, nx, A.pitch, ny, walls,
                                                              A.row0, A.gny),
                               A.fin, 0, &s_h0[0][0], 0);
        cp_async_commit();
        issue_pair_tiles<T, 1, 1, true>(A, tid, x0, y0, gT, np);
    } else {
        issue_pair_tiles<T, 0, kHD, false>(A, tid, x0, y0, hT, np);
        fill_issue<T, false, 1>(fill_plan<T, kH0W, kH0H, false>(tid, kNT, x0 - 4, y0 - 3, nx, A.pitch, ny, walls,
                                                                A.row0, A.gny),
                                A.fin, 0, &s_h0[0][0], 0);
        cp_async_commit();
        issue_pair_tiles<T, 1, 1, false>(A, tid, x0, y0, gT, np);
    }
    if (!TMA) cp_async_commit();
    // the node's g rest population (not moved by streaming): requested now so
    // that its latency overlaps the density stage and the scalar chain
    const int x = x0 + (int)threadIdx.x, y = y0 + (int)threadIdx.y;
    const bool valid = INTERIOR || (x < nx && y < A.yhi);
    const int32_t i = valid ? x + nx * y : 0;                        // node (moments)
    const size_t ip = valid ? (size_t)x + (size_t)A.pitch * y : 0;  // population slot
    const T g0 = valid ? __ldg(A.fin + 9 * np + ip) : T(0);
    // rows of the rho region (y0 - 3 .. y0 + 10) all of kind 0 and inside
    // (decided on the whole lattice's rows: row y0 + row0 of gny)
    const bool rows_in = INTERIOR || !walls || (y0 + A.row0 >= kHD && y0 + A.row0 + kLTY + kHD <= A.gny);
    if (TMA) {
        if (!block_mbar_wait(&S.bar[0], pp.ph[0])) return tma_gave_up(A, S, pp);
        pp.ph[0] ^= 1u;
    } else {
        cp_async_wait_group<1>();
        __syncthreads();
    }
    // the node's own rest population, read before the h tiles are reused
    const T h0 = s_h0[threadIdx.y + 3][threadIdx.x + 4];
    // 1. rho = sum of the streamed, bounced-back h on the depth-3 region
    //    (s_rho[r][c] = global (x0 - 4 + c, y0 - 3 + r); zero outside a walled
    //    domain, where only zero coefficients meet it); the tile's own
    //    streamed h pairs are kept for the collision
    // (items over whole 40-slot rows of the windows, so that the lanes of a
    // warp read consecutive shared-memory words; slots 0 and 39 idle)
    if (INTERIOR) {
        // interior tile, integer-weight operators: three rows of one column
        // per thread (neighbour loads shared), one pass over the row groups
        if (tid < kRW * kDG) {
            const int g = tid / kRW, rw = tid - g * kRW;
            if (rw >= 1 && rw <= kQW) {
                const int rx = rw - 1, ry0 = 3 * g;
                const int c = rx + (PH::XH - 3);
                // window rows of y - 1 .. y + 3 (row ry sits at window row
                // ry + 1); the last group's third row is not in the region,
                // its rows are clamped to the window and its value dropped
                int rb[5];
#pragma unroll
                for (int j = 0; j < 5; ++j) rb[j] = min(ry0 + j, PH::H - 1) * PH::W;
                T ra[3], rb2[3];
                auto pair = [&](auto qc) {
                    constexpr int p = decltype(qc)::value;
                    V2<T> v[3];
                    stream_uni3<T, p>(hT + p * PH::N, rb, c, A.ka, A.kb, v);
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        const T t = v[i].x + v[i].y;
                        if (p == 0) ra[i] = t;
                        if (p == 1) ra[i] += t;
                        if (p == 2) rb2[i] = t;
                        if (p == 3) rb2[i] += t;
                        const int ry = ry0 + i;
                        if ((unsigned)(rx - 3) < (unsigned)kLTX && (unsigned)(ry - 3) < (unsigned)kLTY)
                            s_psi[p][(ry - 3) * kLTX + (rx - 3)] = v[i];
                    }
                };
                pair(IntC<0>{});
                pair(IntC<1>{});
                pair(IntC<2>{});
                pair(IntC<3>{});
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const int ry = ry0 + i;
                    if (ry < kQH) s_rho[ry][rw] = s_h0[ry][rw] + ra[i] + rb2[i];
                }
            }
        }
    } else {
        for (int q = tid; q < kRW * kQH; q += kNT) {
            const int ry = q / kRW, rw = q - ry * kRW;
            if (rw < 1 || rw > kQW) continue;
            const int rx = rw - 1;
            const int gy = y0 + A.row0 + ry - 3;
            T r = T(0);
            if (rows_in || (gy >= 0 && gy < A.gny && y0 + ry - 3 >= 0 && y0 + ry - 3 < ny)) {
                const int k = rows_in ? 0 : lat_kind(walls, gy, A.gny);
                const int c = (ry + 1) * PH::W + rx + (PH::XH - 3);
                const bool own = (unsigned)(rx - 3) < (unsigned)kLTX && (unsigned)(ry - 3) < (unsigned)kLTY;
                const int o = (ry - 3) * kLTX + (rx - 3);
                V2<T> v[4];
#pragma unroll
                for (int p = 0; p < 4; ++p)
                    v[p] = bounce_pair<T>(k, p, stream_pair<T, PH::W>(C, k, p, hT + p * PH::N, c, dt));
                r = s_h0[ry][rx + 1] + ((v[0].x + v[0].y) + (v[1].x + v[1].y)) +
                    ((v[2].x + v[2].y) + (v[3].x + v[3].y));
                if (own) {
#pragma unroll
                    for (int p = 0; p < 4; ++p) s_psi[p][o] = v[p];
                }
            }
            s_rho[ry][rx + 1] = r;
        }
    }
    __syncthreads();
    // the h pair tiles and the rest tile are dead (nothing below reads them):
    // request the next tile's h group now, so that it arrives while this
    // tile finishes
    if (tid == 0) {
        if (next.tma) issue_h_group<T>(A, next.bx * kLTX, next.by * kLTY, S, dsm);
        S.nt[0] = next.t;
        S.nt[1] = next.bx;
        S.nt[2] = next.by;
        S.nt[3] = (next.valid ? 1 : 0) | (next.tma ? 2 : 0);
    }
    const auto &rc = C.r;  // recovery coefficients
    // 2. recovered grad rho on the depth-2 region
    if (INTERIOR) {
        // three rows of one column per thread (s_rho column lw = lx + 2),
        // one pass over the row groups (the last group's loads are clamped to
        // the region, values of rows past it dropped)
        if (tid < kRW * kGG) {
            const int g = tid / kRW, lw = tid - g * kRW;
            if (lw >= 2 && lw < kGW + 2) {
                const int lx = lw - 2, ly0 = kGR * g;
                // s_rho rows ly0 .. ly0 + kGR + 1 (rows a - 1 .. a + 1 of a = ly + 1)
                T cx[kGR + 2], cl[kGR + 1], cr[kGR + 1];
#pragma unroll
                for (int j = 0; j < kGR + 2; ++j) cx[j] = s_rho[min(ly0 + j, kRH - 1)][lw];
#pragma unroll
                for (int j = 0; j < kGR + 1; ++j) {
                    cl[j] = s_rho[min(ly0 + j, kRH - 1)][lw - 1];
                    cr[j] = s_rho[min(ly0 + 1 + j, kRH - 1)][lw + 1];
                }
#pragma unroll
                for (int i = 0; i < kGR; ++i) {
                    if (ly0 + i < kGH) {
                        T sx, sy;
                        rec_uni<T>(cr[i], cr[i + 1], cx[i + 2], cl[i + 1], cl[i], cx[i], sx, sy);
                        s_g[ly0 + i][lx] = vset(sx * A.al, sy * A.al);
                    }
                }
            }
        }
    } else {
        for (int q = tid; q < kGW * kGH; q += kNT) {
            const int ly = q / kGW, lx = q - ly * kGW;
            const int gy = y0 + A.row0 + ly - 2;
            const int k = (walls && (gy == 0 || gy == A.gny - 1)) ? (gy == 0 ? 1 : 2) : 0;
            T sx = T(0), sy = T(0);
            const T c0 = s_rho[ly + 1][lx + 2];
#pragma unroll
            for (int o = 0; o < 6; ++o) {
                const T d = s_rho[ly + 1 + lat_dy(o)][lx + 2 + lat_dx(o)] - c0;
                sx += rc[k][o][0] * d;
                sy += rc[k][o][1] * d;
            }
            s_g[ly][lx] = vset(sx, sy);
        }
    }
    __syncthreads();
    // 3. lap rho and mu on the depth-1 region
    const Phys<T> &P = A.P;
    if (INTERIOR) {
        // three rows of one column per thread (s_g column lw = lx + 1), one
        // pass over the row groups (loads clamped to the region, values of
        // rows past it dropped)
        if (tid < kRW * kMG) {
            const int g = tid / kRW, lw = tid - g * kRW;
            if (lw >= 1 && lw < kMW + 1) {
                const int lx = lw - 1, ly0 = kMR * g;
                V2<T> cx[kMR + 2], cl[kMR + 1], cr[kMR + 1];
#pragma unroll
                for (int j = 0; j < kMR + 2; ++j) cx[j] = s_g[min(ly0 + j, kGH - 1)][lw];
#pragma unroll
                for (int j = 0; j < kMR + 1; ++j) {
                    cl[j] = s_g[min(ly0 + j, kGH - 1)][lw - 1];
                    cr[j] = s_g[min(ly0 + 1 + j, kGH - 1)][lw + 1];
                }
#pragma unroll
                for (int i = 0; i < kMR; ++i) {
                    const int ly = ly0 + i;
                    if (ly < kMH) {
                        const V2<T> E0 = vsub<T>(cr[i], cl[i + 1]);
                        const V2<T> E1 = vsub<T>(cr[i + 1], cl[i]);
                        const V2<T> E2 = vsub<T>(cx[i + 2], cx[i]);
                        // R_x(d_x rho) + R_y(d_y rho)
                        if (LAP64) {
                            // the same differences and weights in FP64
                            const double e0x = (double)cr[i].x - (double)cl[i + 1].x;
                            const double e0y = (double)cr[i].y - (double)cl[i + 1].y;
                            const double e1x = (double)cr[i + 1].x - (double)cl[i].x;
                            const double e1y = (double)cr[i + 1].y - (double)cl[i].y;
                            const double e2x = (double)cx[i + 2].x - (double)cx[i].x;
                            const double e2y = (double)cx[i + 2].y - (double)cx[i].y;
                            const double lap = A.al64 * (fma(2.0, e0x, e1x - e2x) + fma(2.0, e2y, e1y - e0y));
                            s_mu[ly][lx] =
                                (T)((double)mu_bulk<T>(P, s_rho[ly + 2][lx + 3]) - A.kappa64 * lap);
                        } else {
                            const T lap = A.al * (fma(T(2), E0.x, E1.x - E2.x) + fma(T(2), E2.y, E1.y - E0.y));
                            s_mu[ly][lx] = mu_bulk<T>(P, s_rho[ly + 2][lx + 3]) - P.kappa * lap;
                        }
                    }
                }
            }
        }
    } else {
        for (int q = tid; q < kMW * kMH; q += kNT) {
            const int ly = q / kMW, lx = q - ly * kMW;
            const int gy = y0 + A.row0 + ly - 1;
            const int k = (walls && (gy == 0 || gy == A.gny - 1)) ? (gy == 0 ? 1 : 2) : 0;
            const V2<T> gc = s_g[ly + 1][lx + 1];
            if (LAP64) {
                double lap = 0.0;
#pragma unroll
                for (int o = 0; o < 6; ++o) {
                    const V2<T> gj = s_g[ly + 1 + lat_dy(o)][lx + 1 + lat_dx(o)];
                    lap += A.r64[k][o][0] * ((double)gj.x - (double)gc.x) +
                           A.r64[k][o][1] * ((double)gj.y - (double)gc.y);
                }
                s_mu[ly][lx] = (T)((double)mu_bulk<T>(P, s_rho[ly + 2][lx + 3]) - A.kappa64 * lap);
            } else {
                T lap = T(0);
#pragma unroll
                for (int o = 0; o < 6; ++o) {
                    const V2<T> gj = s_g[ly + 1 + lat_dy(o)][lx + 1 + lat_dx(o)];
                    lap += rc[k][o][0] * (gj.x - gc.x) + rc[k][o][1] * (gj.y - gc.y);
                }
                s_mu[ly][lx] = mu_bulk<T>(P, s_rho[ly + 2][lx + 3]) - P.kappa * lap;
            }
        }
    }
    __syncthreads();
    // 4. per node: grad mu, stress force, then the collision.  Threads of a
    //    ragged tile outside the mesh take part in every barrier.
    const int lx = threadIdx.x, ly = threadIdx.y;
    const int k = (rows_in || !valid) ? 0 : lat_kind(walls, y + A.row0, A.gny);
    T dmx, dmy, kx, ky;
    if (INTERIOR) {
        const int a = ly + 1, b = lx + 1, a2 = ly + 2, b2 = lx + 2;
        rec_uni<T>(s_mu[a][b + 1], s_mu[a + 1][b + 1], s_mu[a + 1][b], s_mu[a][b - 1], s_mu[a - 1][b - 1], s_mu[a - 1][b],
                   dmx, dmy);
        dmx *= A.al;
        dmy *= A.al;
        // differences of the gradient products across opposite neighbours,
        // in product form: (P.x, P.y) = E(d_x rho^2), E(d_y rho^2);
        // Q = E(d_x rho d_y rho); then
        // K_x = kappa [R_x(d_y rho^2) - R_y(d_x rho d_y rho)],
        // K_y = kappa [R_y(d_x rho^2) - R_x(d_x rho d_y rho)]
        V2<T> Pk[3];
        T Qk[3];
        auto prod = [&](int j, V2<T> u, V2<T> w) {
            const V2<T> D = vsub<T>(u, w);
            Pk[j] = vmul(D, vadd(u, w));
            Qk[j] = fma(u.x, D.y, w.y * D.x);
        };
        prod(0, s_g[a2][b2 + 1], s_g[a2][b2 - 1]);
        prod(1, s_g[a2 + 1][b2 + 1], s_g[a2 - 1][b2 - 1]);
        prod(2, s_g[a2 + 1][b2], s_g[a2 - 1][b2]);
        const T rxy = fma(T(2), Pk[0].y, Pk[1].y - Pk[2].y), ryq = fma(T(2), Qk[2], Qk[1] - Qk[0]);
        const T ryx = fma(T(2), Pk[2].x, Pk[1].x - Pk[0].x), rxq = fma(T(2), Qk[0], Qk[1] - Qk[2]);
        const T kka = P.kappa * A.al;
        kx = kka * (rxy - ryq);
        ky = kka * (ryx - rxq);
    } else {
        T smx = T(0), smy = T(0), skx = T(0), sky = T(0);
        const T mc = s_mu[ly + 1][lx + 1];
        const V2<T> gcv = s_g[ly + 2][lx + 2];
        const T gxc = gcv.x, gyc = gcv.y;
#pragma unroll
        for (int o = 0; o < 6; ++o) {
            const T ax = rc[k][o][0], ay = rc[k][o][1];
            const T dm = s_mu[ly + 1 + lat_dy(o)][lx + 1 + lat_dx(o)] - mc;
            smx += ax * dm;
            smy += ay * dm;
            const V2<T> gjv = s_g[ly + 2 + lat_dy(o)][lx + 2 + lat_dx(o)];
            const T gxj = gjv.x, gyj = gjv.y;
            const T ddx = gxj - gxc, ddy = gyj - gyc;  // product form, see k_mu
            const T dxx = ddx * (gxj + gxc), dxy = gxj * ddy + gyc * ddx, dyy = ddy * (gyj + gyc);
            skx += ax * dyy - ay * dxy;
            sky += ay * dxx - ax * dxy;
        }
        dmx = smx;
        dmy = smy;
        kx = P.kappa * skx;
        ky = P.kappa * sky;
    }
    const T r0 = s_rho[ly + 3][lx + 4];
    const V2<T> drv = s_g[ly + 2][lx + 2];
    const T drx = drv.x, dry = drv.y;
    if (TMA) {
        if (!block_mbar_wait(&S.bar[1], pp.ph[1])) return tma_gave_up(A, S, pp);
        pp.ph[1] ^= 1u;
    } else {
        cp_async_wait_group<0>();
        __syncthreads();
    }
    if (valid)
        lat_node<T, INTERIOR>(A, C, k, lx, ly, tid, i, ip, n, np, h0, g0, r0, drx, dry, dmx, dmy, kx, ky, gT, s_psi);
    __syncthreads();  // the caller may reuse shared memory for the next tile
    return true;
}

// Barriers of the TMA loads; once per block before its first tile.
template <typename T>
__device__ __forceinline__ void lat_block_init(StepSmem<T> &S) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
}

// Whether tile (bx, by) loads its halo windows by TMA.
template <typename T>
__device__ __forceinline__ bool tile_tma(const LatArgs<T> &A, int bx, int by, const unsigned char *dsm) {
    const int x0 = bx * kLTX, y0 = A.ylo + by * kLTY;
    // the boxes' x coordinates (4-byte words) on 16-byte boundaries (by
    // construction; the checked build verifies it and falls back to cp.async)
    constexpr int WPN = (int)sizeof(V2<T>) / 4, SPN = (int)sizeof(T) / 4;
    const bool aligned = ((x0 - PairTile<T, kHD>::XH) * WPN) % 4 == 0 && ((x0 - 4) * SPN) % 4 == 0 &&
                         ((x0 - PairTile<T, 1>::XH) * WPN) % 4 == 0;
    return A.tmap && tile_interior(A, x0, y0) && tile_unwrapped(x0, y0, A.nx, A.ny) &&
           (smem_u32(dsm) & 127u) == 0 && chk_idx(aligned ? 0 : -1, 1, 4u);
}

// One tile of a block's walk (pp carries the TMA barrier phases and whether
// this tile's h group was already requested; next is the block's next tile).
// False when a bounded wait gave up.
template <typename T, bool LAP64 = false>
__device__ __forceinline__ bool lat_tile(const LatArgs<T> &A, const LatCoef<T> &C, int bx, int by, StepSmem<T> &S,
                                         unsigned char *dsm, TilePipe &pp, const NextTile &next) {
    if (tile_tma(A, bx, by, dsm)) return lat_tile_impl<T, true, true, LAP64>(A, C, bx, by, S, dsm, pp, next);
    if (tile_interior(A, bx * kLTX, A.ylo + by * kLTY))
        return lat_tile_impl<T, true, false, LAP64>(A, C, bx, by, S, dsm, pp, next);
    return lat_tile_impl<T, false, false, LAP64>(A, C, bx, by, S, dsm, pp, next);
}

// After a tile: the published next tile (false: none), and whether its h
// group was requested.
template <typename T>
__device__ __forceinline__ bool take_next(const StepSmem<T> &S, TilePipe &pp) {
    const int f = S.nt[3];
    pp.h_issued = (f & 2) != 0;
    return (f & 1) != 0;
}

// One tile per block (grid ntx x nty).  Halo windows of interior tiles come
// by TMA; walking several tiles per block with the next tile's h group
// requested early measured slower for a single mesh (more instructions per
// node, no better issue rate), so that walk is left to the batched kernel.
// LAP64: the kappa lap rho term of mu in FP64 (FELBM_PARAM_LAP_FP64).
template <typename T, bool LAP64 = false>
__global__ void __launch_bounds__(kNT, (sizeof(T) == 4 ? 1024 : 512) / kNT) k_lat_step(LatArgs<T> A) {
    __shared__ StepSmem<T> S;
    extern __shared__ __align__(128) unsigned char lat_dsm[];
    lat_block_init<T>(S);
    TilePipe pp;
    const NextTile none{0, 0, 0, false, false};
    lat_tile<T, LAP64>(A, A.c, blockIdx.x, blockIdx.y, S, lat_dsm, pp, none);
}

}  // namespace felbm
