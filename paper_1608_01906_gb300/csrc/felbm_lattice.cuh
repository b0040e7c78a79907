// Building blocks of the structured-lattice step (felbm_march.cuh): the
// coefficient tables and arguments of a lattice, halo windows filled with
// cp.async or loaded by TMA (cp.async.bulk.tensor with mbarrier waits that
// are bounded), the Taylor-Galerkin streaming of a pair of opposite
// populations from a shared-memory window (Sec. 2.2.1), bounce-back at wall
// rows (Sec. 3.3) and the collision of a pair (Sec. 2.2).
//
// Opposite directions (a, abar) are stored interleaved (pop_index): the
// stencil of a pair reads one 8-byte (FP32) word per neighbour and runs in
// packed two-wide arithmetic (FFMA2 on sm_103a), each lane with its own
// coefficient.  Population rows are stored with a pitch of nx rounded up to
// a multiple of 4 slots, so every row starts 16-byte aligned.
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

constexpr int kLTX = 32, kLTY = 8;  // strip width and rows per iteration of the march

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
    int32_t pitch;  // population row pitch (slots)
    int32_t gy;     // ghost rows on each side (slot row of mesh row y: y + gy)
    int32_t rows;   // slot rows: ny + 2 gy
    LatCoef<T> c;
    Phys<T> P;
    const T *fin;
    T *fout;
    T *rho;  // unused by the lattice step (rho is formed per tile)
    T *mom;  // 4N or nullptr
    int *flag;
    const TMap *tmap;  // {h pairs, h rest, g pairs} of fin, or nullptr
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
__device__ __forceinline__ FillPlan fill_plan(int tid, int nthreads, int gx0, int gy0, int nx, int pitch, int ny,
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
            f.src[t] = inside ? gx + pitch * gy : 0;
            f.ok[t] = inside;
            f.dst[t] = r * W + col;
            f.n = t + 1;
        }
    }
    return f;
}

// Fill plan of a window of H rows x W elements whose top-left element is
// slot (sx0, sy0) of a storage with rows of `pitch` slots and `rows` slot
// rows: the columns are inside by construction (ghost columns), rows outside
// [0, rows) fill with zeros.
template <typename E, int W, int H, bool VEC>
__device__ __forceinline__ FillPlan fill_plan_slots(int tid, int nthreads, int sx0, int sy0, int pitch,
                                                    int rows) {
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
            const int sy = sy0 + r;
            const bool inside = sy >= 0 && sy < rows;
            f.src[t] = inside ? sx0 + col + pitch * sy : 0;
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

// Bring a TMA box into L2 (no shared memory, no completion to wait for).
__device__ __forceinline__ void tma_prefetch_2d(const TMap *map, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];\n" ::"l"(map), "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void tma_prefetch_3d(const TMap *map, int x, int y, int z) {
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];\n" ::"l"(map), "r"(x), "r"(y),
                 "r"(z)
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

// ---- windows of the march ------------------------------------------

constexpr int kHD = 4;  // depth of the h windows in x (columns x0-4 .. x0+35)

constexpr size_t align128(size_t b) { return (b + 127) / 128 * 128; }

// Whether the halo windows of a strip at x0 may be filled in 16-byte
// chunks: rows are 16-byte aligned (pitch), so unless a window wraps around
// a row whose length is not a multiple of 4.
__device__ __forceinline__ bool vec_fills(int x0, int nx) {
    return (nx % 4) == 0 || (x0 >= kHD && x0 + kLTX + kHD <= nx);
}

}  // namespace felbm
