// Structured-lattice step: two launches per time step.
//
//   k_lat_rho   Taylor-Galerkin streaming of the 9 h populations (Sec. 2.2.1)
//               with per-state constant coefficient tables, wall bounce-back,
//               rho = sum_a h_a.  32 x 8 node tiles, neighbour rows shared
//               through L1.
//   k_lat_step  one 32 x 8 tile per block: rho with a depth-3 halo is staged in
//               shared memory; grad rho (depth 2), lap rho and mu (depth 1),
//               then grad mu and the stress force at the tile's nodes are all
//               recomputed there (Sec. 2.3 recovery, Sec. 2.1 mu, stress form);
//               the 18 populations are streamed from global memory (neighbour
//               rows through L1), bounced back at walls, and collided
//               (Sec. 2.2) in registers; one write of the 18 populations.
//
// Coefficient tables: for each row kind (interior, bottom wall row, top wall
// row), offset o and moving population a, the streaming coefficient
//   s[k][o][a] = e_a . a_o + dt/2 e_a . b_o . e_a
// and the recovery coefficients r[k][o] = a_o, read off the assembled
// operators of the mesh (zero for offsets outside a walled domain).
#pragma once

#include "felbm_internal.h"
#include "felbm_kernels.cuh"

namespace felbm {

constexpr int kLTX = 32, kLTY = 8;  // tile of nodes per block

template <typename T>
struct LatCoef {
    T s[3][6][9];  // streaming coefficient per kind, offset, population (a = 0 unused)
    T r[3][6][2];  // recovery coefficients
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

// Neighbour node ids of (x, y) for the six lattice offsets; for a walled
// domain an out-of-range row maps to the node itself (its coefficient is 0).
__device__ __forceinline__ void lat_neighbours(int x, int y, int nx, int ny, int walls,
                                               int32_t *j) {
#pragma unroll
    for (int o = 0; o < 6; ++o) {
        int xx = x + lat_dx(o), yy = y + lat_dy(o);
        xx = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
        if (walls) {
            if (yy < 0 || yy >= ny) {
                xx = x;
                yy = y;
            }
        } else {
            yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
        }
        j[o] = xx + nx * yy;
    }
}

// Halo tile of one population: kPH = kLTY + 2 rows of kPW<T> values around
// the block's tile.  Rows start CE = 16 / sizeof(T) columns left of the tile
// so that a tile away from the x wrap is filled with 16-byte copies (the
// stencil reads the kLTX + 2 central columns).  Tiles at the x wrap, and
// meshes whose row length is not a multiple of CE, are filled element by
// element with the periodic wrap applied per element.
template <typename T>
struct PopTile {
    static constexpr int CE = 16 / (int)sizeof(T);
    static constexpr int W = kLTX + 2 * CE;
    static constexpr int H = kLTY + 2;
    static constexpr int N = W * H;
    static constexpr int CHUNKS = N / CE;  // 16-byte chunks of a tile
};
constexpr int kPH = kLTY + 2;
template <typename T>
constexpr int kPN = PopTile<T>::N;

// Fill plan of one thread for one halo window (the same for every
// population): up to kMaxSlots slots, each a global element offset and a
// shared-memory element offset; a slot outside a walled domain copies zero
// bytes (cp.async zero-fills it).  VEC: the slots are 16-byte chunks.
constexpr int kMaxSlots = 3;
struct FillPlan {
    int32_t src[kMaxSlots];
    int32_t dst[kMaxSlots];
    int8_t ok[kMaxSlots];  // inside the domain
    int n;
};

// Plan for a window of H rows x W columns whose top-left element is global
// (gx0, gy0).  VEC requires a window without x wrap and 16-byte aligned rows
// (the caller checks).
template <typename T, int W, int H, bool VEC>
__device__ __forceinline__ FillPlan fill_plan(int tid, int nthreads, int gx0, int gy0, int nx, int ny,
                                              int walls) {
    constexpr int CE = 16 / (int)sizeof(T);
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
            while (gx < 0) gx += nx;
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

// Asynchronous global -> shared copies (cp.async) with a source size: a
// zero source size fills the destination with zeros.  The halo tiles of all
// moving populations are requested at once so that their latency overlaps
// the other work of the block.
template <typename T, bool VEC>
__device__ __forceinline__ void cp_async_zfill(T *smem, const T *gmem, bool ok) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if (VEC) {
        const int ssz = ok ? 16 : 0;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(ssz)
                     : "memory");
    } else if (sizeof(T) == 4) {
        const int ssz = ok ? 4 : 0;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(ssz)
                     : "memory");
    } else {
        const int ssz = ok ? 8 : 0;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(ssz)
                     : "memory");
    }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N committed groups of this thread are still pending
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Request NF fields (src + f_i * src_stride -> dst + f_i * dst_stride) of
// one window following plan f.
template <typename T, bool VEC, int NF>
__device__ __forceinline__ void fill_issue(const FillPlan &f, const T *__restrict__ src, size_t src_stride,
                                           T *dst, int dst_stride) {
#pragma unroll
    for (int t = 0; t < kMaxSlots; ++t) {
        if (t < f.n) {
            const T *s = src + f.src[t];
            T *d = dst + f.dst[t];
            const bool ok = f.ok[t];
#pragma unroll
            for (int q = 0; q < NF; ++q) cp_async_zfill<T, VEC>(d + q * dst_stride, s + q * src_stride, ok);
        }
    }
}

// Request the halo tiles of populations A0 + 1 .. A0 + 8 of block tile
// (x0, y0) into tiles[0..8) (tile stride kPN).
template <typename T, int A0>
__device__ __forceinline__ void issue_pop_tiles(const LatArgs<T> &A, int tid, int x0, int y0, T *tiles,
                                                size_t n) {
    constexpr int CE = PopTile<T>::CE, W = PopTile<T>::W, H = PopTile<T>::H;
    const int nx = A.nx, ny = A.ny, walls = A.walls;
    const T *src = A.fin + (size_t)(A0 + 1) * n;
    if ((nx % CE) == 0 && x0 - CE >= 0 && x0 + kLTX + CE <= nx) {
        const FillPlan f = fill_plan<T, W, H, true>(tid, kLTX * kLTY, x0 - CE, y0 - 1, nx, ny, walls);
        fill_issue<T, true, 8>(f, src, n, tiles, kPN<T>);
    } else {
        const FillPlan f = fill_plan<T, W, H, false>(tid, kLTX * kLTY, x0 - CE, y0 - 1, nx, ny, walls);
        fill_issue<T, false, 8>(f, src, n, tiles, kPN<T>);
    }
}

// sum_o s[k][o][d] (psi(node + o) - psi(node)) from a halo tile, node at
// (lx, ly) of the block's tile.
template <typename T>
__device__ __forceinline__ T stencil(const LatCoef<T> &c, int k, int d, const T *buf, int lx, int ly) {
    constexpr int W = PopTile<T>::W, CE = PopTile<T>::CE;
    const T self = buf[(ly + 1) * W + lx + CE];
    T acc = T(0);
#pragma unroll
    for (int o = 0; o < 6; ++o)
        acc += c.s[k][o][d] * (buf[(ly + 1 + lat_dy(o)) * W + lx + CE + lat_dx(o)] - self);
    return acc;
}

// Streamed value of moving population d (1..8) from its halo tile; row kind
// 0 is compile-time on interior tiles.
template <typename T>
__device__ __forceinline__ T streamed(const LatCoef<T> &c, int k, bool interior, int d, const T *buf,
                                      int lx, int ly, T dt) {
    constexpr int W = PopTile<T>::W, CE = PopTile<T>::CE;
    const T self = buf[(ly + 1) * W + lx + CE];
    const T acc = interior ? stencil<T>(c, 0, d, buf, lx, ly) : stencil<T>(c, k, d, buf, lx, ly);
    return self - dt * acc;
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

// Density pass of tile (bx, by); tiles: shared memory for 8 halo tiles.
template <typename T>
__device__ __forceinline__ void lat_rho_tile(const LatArgs<T> &A, int bx, int by, T *tiles) {
    const int x0 = bx * kLTX, y0 = by * kLTY;
    const int lx = threadIdx.x, ly = threadIdx.y, tid = ly * kLTX + lx;
    const int x = x0 + lx, y = y0 + ly;
    const bool valid = x < A.nx && y < A.ny;
    const size_t n = (size_t)A.nx * A.ny;
    issue_pop_tiles<T, 0>(A, tid, x0, y0, tiles, n);
    cp_async_commit();
    const int k = valid ? lat_kind(A.walls, y, A.ny) : 0;
    const bool interior = !A.walls || (y0 > 0 && y0 + kLTY < A.ny);
    const int32_t i = x + A.nx * y;
    T r = valid ? __ldg(A.fin + i) : T(0);  // rest population is not moved
    cp_async_wait_all();
    __syncthreads();
    if (valid) {
#pragma unroll
        for (int d = 1; d < 9; ++d) {
            const T v = streamed<T>(A.c, k, interior, d, tiles + (d - 1) * kPN<T>, lx, ly, A.P.dt);
            r += k ? T(bb_mult(k, d)) * v : v;
        }
        A.rho[i] = r;
    }
    __syncthreads();  // the caller may reuse the tiles for the next tile
}

template <typename T>
__global__ void __launch_bounds__(kLTX *kLTY, 4) k_lat_rho(LatArgs<T> A) {
    __shared__ __align__(16) T tiles[8 * kPN<T>];
    lat_rho_tile<T>(A, blockIdx.x, blockIdx.y, tiles);
}

template <typename T>
constexpr size_t lat_step_smem() {
    return (16 * (size_t)kPN<T> + 18 * (size_t)kLTX * kLTY) * sizeof(T);
}

// Streaming from the halo tiles, bounce-back, collision and the write of one
// node of a step tile.
template <typename T>
__device__ __forceinline__ void lat_step_node(const LatArgs<T> &A, int k, bool interior, int lx, int ly,
                                              int tid, int32_t i, size_t n, T r0, T drx, T dry,
                                              T dmx, T dmy, T kx, T ky, const T *tiles,
                                              T (*s_psi)[kLTX * kLTY]) {
    const Phys<T> &P = A.P;
    // streamed populations of this node go to shared memory (slot tid of
    // row a): keeps the 18 values out of registers
    const T dt = P.dt;
    s_psi[0][tid] = __ldg(A.fin + i);
    s_psi[9][tid] = __ldg(A.fin + 9 * n + i);
#pragma unroll
    for (int d = 1; d < 9; ++d) {
        s_psi[d][tid] = streamed<T>(A.c, k, interior, d, tiles + (d - 1) * kPN<T>, lx, ly, dt);
        s_psi[9 + d][tid] = streamed<T>(A.c, k, interior, d, tiles + (7 + d) * kPN<T>, lx, ly, dt);
    }
    if (k) {  // wall row: bounce-back of the populations entering the fluid
        const int nk = k == 1 ? 2 : 4;
#pragma unroll
        for (int a = 1; a < 9; ++a)
            if (kEx(a) * kEx(nk) + kEy(a) * kEy(nk) > 0) {
                s_psi[a][tid] = s_psi[kOpp(a)][tid];
                s_psi[9 + a][tid] = s_psi[9 + kOpp(a)][tid];
            }
    }
    T sg, mx, my;
    g_moments<T>(s_psi[9][tid], s_psi[10][tid], s_psi[11][tid], s_psi[12][tid], s_psi[13][tid],
                 s_psi[14][tid], s_psi[15][tid], s_psi[16][tid], s_psi[17][tid], sg, mx, my);
    const CollidePrep<T> cp = collide_prep<T>(P, sg, mx, my, r0, drx, dry, dmx, dmy, kx, ky);
    const T r = cp.r, ux = cp.ux, uy = cp.uy, p = cp.p;
    // populations 1..8, then the rest population, which also takes the sum of
    // the h increments (zero in exact arithmetic): the collision then keeps
    // the node's mass to one rounding instead of accumulating the rounding
    // of the nine source terms every step
    T dsum = T(0);
#pragma unroll
    for (int a = 1; a < 9; ++a) {
        T ho, go;
        const T hs = s_psi[a][tid];
        collide_pop_rt<T>(cp, a, hs, s_psi[9 + a][tid], ho, go);
        dsum += ho - hs;
        A.fout[(size_t)a * n + i] = ho;
        A.fout[(size_t)(9 + a) * n + i] = go;
    }
    {
        T ho, go;
        const T hs = s_psi[0][tid];
        collide_pop_rt<T>(cp, 0, hs, s_psi[9][tid], ho, go);
        dsum += ho - hs;
        A.fout[i] = ho - dsum;
        A.fout[(size_t)9 * n + i] = go;
    }
    if (!(finite_val(r) && finite_val(ux) && finite_val(uy) && finite_val(p))) atomicOr(A.flag, 1);
    if (A.mom) {
        A.mom[i] = r;
        A.mom[n + i] = ux;
        A.mom[2 * n + i] = uy;
        A.mom[3 * n + i] = p;
    }
}

constexpr int kRW = kLTX + 8, kRH = kLTY + 6;  // rho: halo 3, rows from x0 - 4 (16-byte aligned)
constexpr int kGW = kLTX + 4, kGH = kLTY + 4;  // grad rho: halo 2
constexpr int kMW = kLTX + 2, kMH = kLTY + 2;  // mu: halo 1

// Shared memory of one step tile: the scalar chain and, in lat_dsm (dynamic,
// lat_step_smem bytes), 16 halo tiles then 18 rows of streamed values.
template <typename T>
struct __align__(16) StepSmem {
    T s_rho[kRH][kRW];
    T s_gx[kGH][kGW], s_gy[kGH][kGW];
    T s_mu[kMH][kMW];
};

// Step pass of tile (bx, by).
template <typename T>
__device__ __forceinline__ void lat_step_tile(const LatArgs<T> &A, int bx, int by, StepSmem<T> &S,
                                              unsigned char *lat_dsm) {
    constexpr int RW = kRW, RH = kRH, GW = kGW, GH = kGH, MW = kMW, MH = kMH;
    auto &s_rho = S.s_rho;
    auto &s_gx = S.s_gx;
    auto &s_gy = S.s_gy;
    auto &s_mu = S.s_mu;
    T *tiles = reinterpret_cast<T *>(lat_dsm);
    T (*s_psi)[kLTX * kLTY] = reinterpret_cast<T (*)[kLTX * kLTY]>(lat_dsm + 16 * kPN<T> * sizeof(T));
    const int nx = A.nx, ny = A.ny, walls = A.walls;
    const int x0 = bx * kLTX, y0 = by * kLTY;
    const int tid = threadIdx.y * kLTX + threadIdx.x;
    constexpr int NT = kLTX * kLTY;
    const size_t n = (size_t)nx * ny;
    // 0. request rho with a depth-3 halo (group 1), then the halo tiles of the
    //    16 moving populations (group 2); the populations arrive while the
    //    scalar chain is computed
    {
        constexpr int CE = 16 / (int)sizeof(T);
        if ((nx % CE) == 0 && x0 - 4 >= 0 && x0 + kLTX + 4 <= nx) {
            const FillPlan fr = fill_plan<T, RW, RH, true>(tid, NT, x0 - 4, y0 - 3, nx, ny, walls);
            fill_issue<T, true, 1>(fr, A.rho, 0, &s_rho[0][0], 0);
        } else {
            const FillPlan fr = fill_plan<T, RW, RH, false>(tid, NT, x0 - 4, y0 - 3, nx, ny, walls);
            fill_issue<T, false, 1>(fr, A.rho, 0, &s_rho[0][0], 0);
        }
        cp_async_commit();
    }
    issue_pop_tiles<T, 0>(A, tid, x0, y0, tiles, n);
    issue_pop_tiles<T, 9>(A, tid, x0, y0, tiles + 8 * kPN<T>, n);
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
        const int k = (walls && (gy == 0 || gy == ny - 1)) ? (gy == 0 ? 1 : 2) : 0;
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
        const int k = (walls && (gy == 0 || gy == ny - 1)) ? (gy == 0 ? 1 : 2) : 0;
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
    const int k = valid ? lat_kind(walls, y, ny) : 0;
    const bool interior = !walls || (y0 > 0 && y0 + kLTY < ny);
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
    cp_async_wait_all();
    __syncthreads();
    if (valid) lat_step_node<T>(A, k, interior, lx, ly, tid, i, n, r0, drx, dry, dmx, dmy, kx, ky,
                                tiles, s_psi);
    __syncthreads();  // the caller may reuse shared memory for the next tile
}

template <typename T>
__global__ void __launch_bounds__(kLTX *kLTY, 3) k_lat_step(LatArgs<T> A) {
    __shared__ StepSmem<T> S;
    extern __shared__ __align__(16) unsigned char lat_dsm[];
    lat_step_tile<T>(A, blockIdx.x, blockIdx.y, S, lat_dsm);
}

}  // namespace felbm
