// Structured-lattice step: two launches per time step.
//
//   k_lat_rho   Taylor-Galerkin streaming of the 9 h populations (Sec. 2.2.1)
//               with per-state constant coefficient tables, wall bounce-back,
//               rho = sum_a h_a.
//   k_lat_step  one 32 x 8 tile per block: rho with a depth-3 halo is staged in
//               shared memory; grad rho (depth 2), lap rho and mu (depth 1),
//               then grad mu and the stress force at the tile's nodes are all
//               recomputed there (Sec. 2.3 recovery, Sec. 2.1 mu, stress form);
//               the populations are streamed from shared-memory halo tiles,
//               bounced back at walls, and collided (Sec. 2.2); one write of
//               the 18 populations.
//
// Opposite directions (a, abar) are stored interleaved (pop_index): the
// stencil of a pair reads one 8-byte (FP32) word per neighbour and runs in
// packed two-wide arithmetic (FFMA2 on sm_103a), each lane with its own
// coefficient.  The halo tiles of all pairs are requested with cp.async
// (16-byte chunks away from the x wrap) when the block starts, so their
// latency overlaps the scalar chain.
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

template <typename T>
struct LatCoef {
    V2<T> s[3][6][4];  // streaming coefficients per kind, offset, pair
    T r[3][6][2];      // recovery coefficients
};

template <typename T>
struct LatArgs {
    int32_t nx, ny, walls;
    LatCoef<T> c;
    Phys<T> P;
    const T *fin;
    T *fout;
    T *rho;
    T *mom;  // 4N or nullptr
    int *flag;
};

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
__device__ __forceinline__ FillPlan fill_plan(int tid, int nthreads, int gx0, int gy0, int nx, int ny,
                                              int walls) {
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
                inside = gy >= 0 && gy < ny;
            } else {
                while (gy < 0) gy += ny;
                while (gy >= ny) gy -= ny;
            }
            f.src[t] = inside ? gx + nx * gy : 0;
            f.ok[t] = inside;
            f.dst[t] = r * W + col;
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

// Halo tile of one population pair: kLTY + 2 rows of W elements; rows start
// CE = 16 / sizeof(pair) elements left of the tile (16-byte aligned chunks);
// the stencil reads the kLTX + 2 central elements.
template <typename T>
struct PairTile {
    static constexpr int CE = 16 / (int)sizeof(V2<T>);
    static constexpr int W = kLTX + 2 * CE;
    static constexpr int H = kLTY + 2;
    static constexpr int N = W * H;
};

// Request the halo tiles of the 4 pairs of h (G = 0) or g (G = 1).
template <typename T, int G, bool INTERIOR = false>
__device__ __forceinline__ void issue_pair_tiles(const LatArgs<T> &A, int tid, int x0, int y0,
                                                 V2<T> *tiles, size_t n) {
    using E = V2<T>;
    constexpr int CE = PairTile<T>::CE, W = PairTile<T>::W, H = PairTile<T>::H;
    const int nx = A.nx, ny = A.ny, walls = A.walls;
    const size_t np = pad4(n);
    const E *src = reinterpret_cast<const E *>(A.fin + (G ? 10 : 1) * np);  // pair 0; pair q at + q np
    if (INTERIOR || ((nx % CE) == 0 && x0 - CE >= 0 && x0 + kLTX + CE <= nx)) {
        const FillPlan f = fill_plan<E, W, H, true>(tid, kLTX * kLTY, x0 - CE, y0 - 1, nx, ny, walls);
        fill_issue<E, true, 4>(f, src, np, tiles, PairTile<T>::N);
    } else {
        const FillPlan f = fill_plan<E, W, H, false>(tid, kLTX * kLTY, x0 - CE, y0 - 1, nx, ny, walls);
        fill_issue<E, false, 4>(f, src, np, tiles, PairTile<T>::N);
    }
}

// Streamed values of pair q of the node at (lx, ly) of the block's tile:
// psi* = psi - dt sum_o s_o (psi(node + o) - psi(node)), both directions in
// one packed operation per step; row kind 0 is compile-time on interior
// tiles.
template <typename T>
__device__ __forceinline__ V2<T> streamed2(const LatCoef<T> &c, int k, bool interior, int q,
                                           const V2<T> *buf, int lx, int ly, T dt) {
    constexpr int W = PairTile<T>::W, CE = PairTile<T>::CE;
    const V2<T> self = buf[(ly + 1) * W + lx + CE];
    const V2<T> m1 = vset(T(-1), T(-1));
    V2<T> acc = vset(T(0), T(0));
#pragma unroll
    for (int o = 0; o < 6; ++o) {
        const V2<T> nb = buf[(ly + 1 + lat_dy(o)) * W + lx + CE + lat_dx(o)];
        const V2<T> d = vfma(self, m1, nb);  // nb - self, exact negation
        acc = vfma(interior ? c.s[0][o][q] : c.s[k][o][q], d, acc);
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
    constexpr T wa = kW<T>(A);
    const T eu = T(ex) * c.ux + T(ey) * c.uy;
    const T eX = T(ex) * c.Xx + T(ey) * c.Xy;
    const T eD = T(ex) * c.drx + T(ey) * c.dry;
    const T eK = T(ex) * c.kx + T(ey) * c.ky;
    const T edu = T(ex) * c.dux + T(ey) * c.duy;
    // Gamma - w = w (3 e.u + 4.5 (e.u)^2 - 1.5 u.u), formed without the w
    // offset (FP32: keeps the momentum part)
    const T even = T(4.5) * eu * eu - T(1.5) * c.uu;
    const V2<T> gmw = vfma(vset(T(3) * wa, T(3) * wa), vset(eu, -eu), vset(wa * even, wa * even));
    const V2<T> gam = vadd(gmw, vset(wa, wa));
    const T h3 = c.hdt * T(3);
    const V2<T> Fa = vmul(vset(h3 * (eX - c.uX), h3 * (-eX - c.uX)), gam);
    const V2<T> Ga = vfma(vset(c.hdt * (eD - c.uD), c.hdt * (-eD - c.uD)), gmw,
                          vmul(vset(h3 * (eK - c.uK), h3 * (-eK - c.uK)), gam));
    // 1/2 [g_eq(u + du) - g_eq(u)] = rho/2 [Gamma(u + du) - Gamma(u)]
    const T bev = T(4.5) * edu * (T(2) * eu + edu) - T(1.5) * c.udu;
    const T hrw = T(0.5) * c.r * wa;
    const V2<T> Sg = vfma(vset(hrw, hrw), vset(T(3) * edu + bev, bev - T(3) * edu), Ga);
    const V2<T> rg = vmul(vset(c.r, c.r), gmw);
    const V2<T> dh = vadd(vfma(vset(c.r, c.r), vset(wa, wa), vset(-hs.x, -hs.y)), rg);  // h_eq - h*
    const T p3 = wa * T(3) * c.p;
    const V2<T> dg = vadd(vset(p3 - gs.x, p3 - gs.y), rg);  // g_eq - g*
    ho = vadd(hs, vfma(vset(c.omw, c.omw), dh, vmul(vset(c.opw, c.opw), Fa)));
    go = vadd(gs, vfma(vset(c.omw, c.omw), dg, vmul(vset(c.opw, c.opw), Sg)));
}

// Weight of streamed h_a in rho at a wall row of kind k (bounce-back replaces
// each population entering the fluid by its opposite).
__device__ __forceinline__ int bb_mult(int k, int a) {
    if (!k) return 1;
    const int nk = k == 1 ? 2 : 4;
    const int in_a = kEx(a) * kEx(nk) + kEy(a) * kEy(nk) > 0;
    const int ao = kOpp(a);
    const int in_opp = kEx(ao) * kEx(nk) + kEy(ao) * kEy(nk) > 0;
    return in_a ? 0 : (in_opp ? 2 : 1);
}

// Bounce-back of a pair at a wall row of kind k (1: inward normal +y, the
// slot-0 directions 2, 5, 6 of pairs 1..3 take their opposites; 2: normal
// -y, the slot-1 directions 4, 7, 8 take theirs).
template <typename T>
__device__ __forceinline__ V2<T> bounce_pair(int k, int q, V2<T> v) {
    if (k == 0 || q == 0) return v;
    return k == 1 ? vset(v.y, v.y) : vset(v.x, v.x);
}

// ---- density pass -------------------------------------------------------

template <typename T>
constexpr size_t lat_rho_smem() {
    return 4 * (size_t)PairTile<T>::N * sizeof(V2<T>);
}

// Whether every node and halo of tile (x0, y0) is an interior-row node away
// from the x wrap, with 16-byte aligned rows: such tiles run with the row
// kind fixed at compile time and vector fills only.
template <typename T>
__device__ __forceinline__ bool tile_interior(int x0, int y0, int nx, int ny, int walls) {
    const bool yin = !walls || (y0 > 0 && y0 + kLTY < ny);
    const bool xin = (nx % 4) == 0 && x0 - 4 >= 0 && x0 + kLTX + 4 <= nx;
    return yin && xin;
}

// Density pass of tile (bx, by); tiles: shared memory of lat_rho_smem bytes.
template <typename T, bool INTERIOR>
__device__ __forceinline__ void lat_rho_tile_impl(const LatArgs<T> &A, int bx, int by, V2<T> *tiles) {
    const int x0 = bx * kLTX, y0 = by * kLTY;
    const int lx = threadIdx.x, ly = threadIdx.y, tid = ly * kLTX + lx;
    const int x = x0 + lx, y = y0 + ly;
    const bool valid = x < A.nx && y < A.ny;
    const size_t n = (size_t)A.nx * A.ny;
    issue_pair_tiles<T, 0, INTERIOR>(A, tid, x0, y0, tiles, n);
    cp_async_commit();
    const int k = (INTERIOR || !valid) ? 0 : lat_kind(A.walls, y, A.ny);
    const bool interior = INTERIOR || !A.walls || (y0 > 0 && y0 + kLTY < A.ny);
    const int32_t i = x + A.nx * y;
    T r = valid ? __ldg(A.fin + i) : T(0);  // rest population is not moved
    cp_async_wait_group<0>();
    __syncthreads();
    if (valid) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const V2<T> v = streamed2<T>(A.c, k, interior, q, tiles + q * PairTile<T>::N, lx, ly, A.P.dt);
            if (!INTERIOR && k)
                r += T(bb_mult(k, pair_dir(q, 0))) * v.x + T(bb_mult(k, pair_dir(q, 1))) * v.y;
            else
                r += v.x + v.y;
        }
        A.rho[i] = r;
    }
    __syncthreads();  // the caller may reuse the tiles for the next tile
}

template <typename T>
__device__ __forceinline__ void lat_rho_tile(const LatArgs<T> &A, int bx, int by, V2<T> *tiles) {
    if (tile_interior<T>(bx * kLTX, by * kLTY, A.nx, A.ny, A.walls))
        lat_rho_tile_impl<T, true>(A, bx, by, tiles);
    else
        lat_rho_tile_impl<T, false>(A, bx, by, tiles);
}

template <typename T>
__global__ void __launch_bounds__(kLTX *kLTY, 6) k_lat_rho(LatArgs<T> A) {
    __shared__ __align__(16) V2<T> tiles[4 * PairTile<T>::N];
    lat_rho_tile<T>(A, blockIdx.x, blockIdx.y, tiles);
}

// ---- step pass ----------------------------------------------------------

constexpr int kRW = kLTX + 8, kRH = kLTY + 6;  // rho: halo 3, rows from x0 - 4 (16-byte aligned)
constexpr int kGW = kLTX + 4, kGH = kLTY + 4;  // grad rho: halo 2
constexpr int kMW = kLTX + 2, kMH = kLTY + 2;  // mu: halo 1

// Shared memory of one step tile: the scalar chain (static) and, in the
// dynamic part (lat_step_smem bytes), the 8 pair halo tiles then the 8 rows
// of streamed pairs.
template <typename T>
struct __align__(16) StepSmem {
    T s_rho[kRH][kRW];
    T s_gx[kGH][kGW], s_gy[kGH][kGW];
    T s_mu[kMH][kMW];
};

template <typename T>
constexpr size_t lat_step_smem() {
    return (8 * (size_t)PairTile<T>::N + 8 * (size_t)kLTX * kLTY) * sizeof(V2<T>);
}

// Streaming from the pair tiles, bounce-back, collision and the write of one
// node of a step tile.
template <typename T>
__device__ __forceinline__ void lat_step_node(const LatArgs<T> &A, int k, bool interior, int lx, int ly,
                                              int tid, int32_t i, size_t n, T r0, T drx, T dry,
                                              T dmx, T dmy, T kx, T ky, const V2<T> *tiles,
                                              V2<T> (*s_psi)[kLTX * kLTY]) {
    const Phys<T> &P = A.P;
    const size_t np = pad4(n);
    const T dt = P.dt;
    const T h0 = __ldg(A.fin + i), g0 = __ldg(A.fin + 9 * np + i);
    // streamed pairs (bounced back at wall rows) go to shared memory: keeps
    // them out of registers
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        s_psi[q][tid] = bounce_pair<T>(k, q, streamed2<T>(A.c, k, interior, q,
                                                          tiles + q * PairTile<T>::N, lx, ly, dt));
        s_psi[4 + q][tid] = bounce_pair<T>(k, q, streamed2<T>(A.c, k, interior, q,
                                                              tiles + (4 + q) * PairTile<T>::N, lx, ly, dt));
    }
    const V2<T> gq0 = s_psi[4][tid], gq1 = s_psi[5][tid], gq2 = s_psi[6][tid], gq3 = s_psi[7][tid];
    T sg, mx, my;
    // g_1 = q0.x, g_3 = q0.y, g_2 = q1.x, g_4 = q1.y, g_5 = q2.x, g_7 = q2.y, g_6 = q3.x, g_8 = q3.y
    g_moments<T>(g0, gq0.x, gq1.x, gq0.y, gq1.y, gq2.x, gq3.x, gq2.y, gq3.y, sg, mx, my);
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
        const V2<T> hs = s_psi[q][tid], gs = s_psi[4 + q][tid];
        V2<T> ho, go;
        collide_pair<T, q>(cp, hs, gs, ho, go);
        dsum += (ho.x - hs.x) + (ho.y - hs.y);
        hout[(size_t)q * np + i] = ho;
        gout[(size_t)q * np + i] = go;
    };
    pair_update(IntC<0>{});
    pair_update(IntC<1>{});
    pair_update(IntC<2>{});
    pair_update(IntC<3>{});
    {
        T ho, go;
        collide_pop_rt<T>(cp, 0, h0, g0, ho, go);
        dsum += ho - h0;
        A.fout[i] = ho - dsum;
        A.fout[9 * np + i] = go;
    }
    if (!(finite_val(r) && finite_val(ux) && finite_val(uy) && finite_val(p))) atomicOr(A.flag, 1);
    if (A.mom) {
        A.mom[i] = r;
        A.mom[n + i] = ux;
        A.mom[2 * n + i] = uy;
        A.mom[3 * n + i] = p;
    }
}

// Step pass of tile (bx, by).
template <typename T, bool INTERIOR>
__device__ __forceinline__ void lat_step_tile_impl(const LatArgs<T> &A, int bx, int by, StepSmem<T> &S,
                                                   unsigned char *lat_dsm) {
    constexpr int RW = kRW, RH = kRH, GW = kGW, GH = kGH, MW = kMW, MH = kMH;
    auto &s_rho = S.s_rho;
    auto &s_gx = S.s_gx;
    auto &s_gy = S.s_gy;
    auto &s_mu = S.s_mu;
    V2<T> *tiles = reinterpret_cast<V2<T> *>(lat_dsm);
    V2<T>(*s_psi)[kLTX * kLTY] =
        reinterpret_cast<V2<T>(*)[kLTX * kLTY]>(lat_dsm + 8 * PairTile<T>::N * sizeof(V2<T>));
    const int nx = A.nx, ny = A.ny, walls = A.walls;
    const int x0 = bx * kLTX, y0 = by * kLTY;
    const int tid = threadIdx.y * kLTX + threadIdx.x;
    constexpr int NT = kLTX * kLTY;
    const size_t n = (size_t)nx * ny;
    // 0. request rho with a depth-3 halo (group 1), then the halo tiles of the
    //    8 pairs (group 2); the populations arrive while the scalar chain is
    //    computed
    {
        constexpr int CE = 16 / (int)sizeof(T);
        if (INTERIOR || ((nx % CE) == 0 && x0 - 4 >= 0 && x0 + kLTX + 4 <= nx)) {
            const FillPlan fr = fill_plan<T, RW, RH, true>(tid, NT, x0 - 4, y0 - 3, nx, ny, walls);
            fill_issue<T, true, 1>(fr, A.rho, 0, &s_rho[0][0], 0);
        } else {
            const FillPlan fr = fill_plan<T, RW, RH, false>(tid, NT, x0 - 4, y0 - 3, nx, ny, walls);
            fill_issue<T, false, 1>(fr, A.rho, 0, &s_rho[0][0], 0);
        }
        cp_async_commit();
    }
    issue_pair_tiles<T, 0, INTERIOR>(A, tid, x0, y0, tiles, n);
    issue_pair_tiles<T, 1, INTERIOR>(A, tid, x0, y0, tiles + 4 * PairTile<T>::N, n);
    cp_async_commit();
    const auto &rc = A.c.r;  // recovery coefficients
    // 1. rho (s_rho[r][c] = global (x0 - 4 + c, y0 - 3 + r); zero outside a
    //    walled domain, where only zero coefficients meet it)
    cp_async_wait_group<1>();
    __syncthreads();
    // 2. recovered grad rho on the depth-2 region
    for (int q = tid; q < GW * GH; q += NT) {
        const int ly = q / GW, lx = q - ly * GW;
        const int gy = y0 + ly - 2;
        const int k = (!INTERIOR && walls && (gy == 0 || gy == ny - 1)) ? (gy == 0 ? 1 : 2) : 0;
        const T c0 = s_rho[ly + 1][lx + 2];
        T sx = T(0), sy = T(0);
#pragma unroll
        for (int o = 0; o < 6; ++o) {
            const T d = s_rho[ly + 1 + lat_dy(o)][lx + 2 + lat_dx(o)] - c0;
            sx += rc[k][o][0] * d;
            sy += rc[k][o][1] * d;
        }
        s_gx[ly][lx] = sx;
        s_gy[ly][lx] = sy;
    }
    __syncthreads();
    // 3. lap rho and mu on the depth-1 region
    const Phys<T> &P = A.P;
    for (int q = tid; q < MW * MH; q += NT) {
        const int ly = q / MW, lx = q - ly * MW;
        const int gy = y0 + ly - 1;
        const int k = (!INTERIOR && walls && (gy == 0 || gy == ny - 1)) ? (gy == 0 ? 1 : 2) : 0;
        const T gxc = s_gx[ly + 1][lx + 1], gyc = s_gy[ly + 1][lx + 1];
        T lap = T(0);
#pragma unroll
        for (int o = 0; o < 6; ++o) {
            lap += rc[k][o][0] * (s_gx[ly + 1 + lat_dy(o)][lx + 1 + lat_dx(o)] - gxc) +
                   rc[k][o][1] * (s_gy[ly + 1 + lat_dy(o)][lx + 1 + lat_dx(o)] - gyc);
        }
        s_mu[ly][lx] = mu_bulk<T>(P, s_rho[ly + 2][lx + 3]) - P.kappa * lap;
    }
    __syncthreads();
    // 4. per node: grad mu, stress force, streaming, collision.  Threads of
    //    a ragged tile outside the mesh take part in every barrier.
    const int lx = threadIdx.x, ly = threadIdx.y;
    const int x = x0 + lx, y = y0 + ly;
    const bool valid = x < nx && y < ny;
    const int k = (INTERIOR || !valid) ? 0 : lat_kind(walls, y, ny);
    const bool interior = INTERIOR || !walls || (y0 > 0 && y0 + kLTY < ny);
    T dmx, dmy, kx, ky;
    {
        T smx = T(0), smy = T(0), skx = T(0), sky = T(0);
        const T mc = s_mu[ly + 1][lx + 1];
        const T gxc = s_gx[ly + 2][lx + 2], gyc = s_gy[ly + 2][lx + 2];
#pragma unroll
        for (int o = 0; o < 6; ++o) {
            const T ax = rc[k][o][0], ay = rc[k][o][1];
            const T dm = s_mu[ly + 1 + lat_dy(o)][lx + 1 + lat_dx(o)] - mc;
            smx += ax * dm;
            smy += ay * dm;
            const T gxj = s_gx[ly + 2 + lat_dy(o)][lx + 2 + lat_dx(o)];
            const T gyj = s_gy[ly + 2 + lat_dy(o)][lx + 2 + lat_dx(o)];
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
    const T drx = s_gx[ly + 2][lx + 2], dry = s_gy[ly + 2][lx + 2];
    const int32_t i = valid ? x + nx * y : 0;
    cp_async_wait_group<0>();
    __syncthreads();
    if (valid) lat_step_node<T>(A, k, interior, lx, ly, tid, i, n, r0, drx, dry, dmx, dmy, kx, ky,
                                tiles, s_psi);
    __syncthreads();  // the caller may reuse shared memory for the next tile
}

template <typename T>
__device__ __forceinline__ void lat_step_tile(const LatArgs<T> &A, int bx, int by, StepSmem<T> &S,
                                              unsigned char *lat_dsm) {
    if (tile_interior<T>(bx * kLTX, by * kLTY, A.nx, A.ny, A.walls))
        lat_step_tile_impl<T, true>(A, bx, by, S, lat_dsm);
    else
        lat_step_tile_impl<T, false>(A, bx, by, S, lat_dsm);
}

template <typename T>
__global__ void __launch_bounds__(kLTX *kLTY, 4) k_lat_step(LatArgs<T> A) {
    __shared__ StepSmem<T> S;
    extern __shared__ __align__(16) unsigned char lat_dsm[];
    lat_step_tile<T>(A, blockIdx.x, blockIdx.y, S, lat_dsm);
}

}  // namespace felbm
