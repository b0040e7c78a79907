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

// Halo tile of one population: (kLTY + 2) x (kLTX + 2) values around the
// block's tile, filled by the block's threads (each fills at most 2 slots;
// the global offsets of those slots are the same for every population).
constexpr int kPW = kLTX + 2, kPH = kLTY + 2, kPN = kPW * kPH;
static_assert(kPN <= 2 * kLTX * kLTY, "two fill slots per thread");

struct FillSlots {
    int32_t off[2];  // global node id of the slot, -1 = outside a walled domain
    int n;           // number of slots this thread fills
};

__device__ __forceinline__ FillSlots fill_slots(int tid, int x0, int y0, int nx, int ny, int walls) {
    FillSlots f;
    f.n = 0;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int q = tid + t * kLTX * kLTY;
        f.off[t] = -1;
        if (q < kPN) {
            const int ly = q / kPW, lx = q - ly * kPW;
            int gx = x0 + lx - 1, gy = y0 + ly - 1;
            while (gx < 0) gx += nx;
            while (gx >= nx) gx -= nx;
            if (walls) {
                if (gy >= 0 && gy < ny) f.off[t] = gx + nx * gy;
            } else {
                while (gy < 0) gy += ny;
                while (gy >= ny) gy -= ny;
                f.off[t] = gx + nx * gy;
            }
            f.n = t + 1;
        }
    }
    return f;
}

// Asynchronous global -> shared copies (cp.async, one element each): the
// halo tiles of all moving populations are requested at once so that their
// latency overlaps the other work of the block.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *smem, const T *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Request the halo tiles of populations A0 + 1 .. A0 + 8 into tiles[0..8).
// Slots outside a walled domain are set to zero.
template <typename T, int A0>
__device__ __forceinline__ void issue_tiles(const LatArgs<T> &A, const FillSlots &f, T (*tiles)[kPN],
                                            int tid, size_t n) {
#pragma unroll
    for (int d = 1; d < 9; ++d) {
        const T *src = A.fin + (size_t)(A0 + d) * n;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            if (t < f.n) {
                T *dst = &tiles[d - 1][tid + t * kLTX * kLTY];
                if (f.off[t] >= 0)
                    cp_async_elem<T>(dst, src + f.off[t]);
                else
                    *dst = T(0);
            }
        }
    }
}

// sum_o s[k][o][d] (psi(node + o) - psi(node)) from a halo tile, node at
// (lx, ly) of the block's tile.
template <typename T>
__device__ __forceinline__ T stencil(const LatCoef<T> &c, int k, int d, const T *buf, int lx, int ly) {
    const T self = buf[(ly + 1) * kPW + lx + 1];
    T acc = T(0);
#pragma unroll
    for (int o = 0; o < 6; ++o)
        acc += c.s[k][o][d] * (buf[(ly + 1 + lat_dy(o)) * kPW + lx + 1 + lat_dx(o)] - self);
    return acc;
}

// Streamed value of moving population d (1..8) from its halo tile; row kind
// 0 is compile-time on interior tiles.
template <typename T>
__device__ __forceinline__ T streamed(const LatCoef<T> &c, int k, bool interior, int d, const T *buf,
                                      int lx, int ly, T dt) {
    const T self = buf[(ly + 1) * kPW + lx + 1];
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
__device__ __forceinline__ void lat_rho_tile(const LatArgs<T> &A, int bx, int by, T (*tiles)[kPN]) {
    const int x0 = bx * kLTX, y0 = by * kLTY;
    const int lx = threadIdx.x, ly = threadIdx.y, tid = ly * kLTX + lx;
    const int x = x0 + lx, y = y0 + ly;
    const bool valid = x < A.nx && y < A.ny;
    const size_t n = (size_t)A.nx * A.ny;
    const FillSlots f = fill_slots(tid, x0, y0, A.nx, A.ny, A.walls);
    issue_tiles<T, 0>(A, f, tiles, tid, n);
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
            const T v = streamed<T>(A.c, k, interior, d, tiles[d - 1], lx, ly, A.P.dt);
            r += k ? T(bb_mult(k, d)) * v : v;
        }
        A.rho[i] = r;
    }
    __syncthreads();  // the caller may reuse the tiles for the next tile
}

template <typename T>
__global__ void __launch_bounds__(kLTX *kLTY, 4) k_lat_rho(LatArgs<T> A) {
    __shared__ T tiles[8][kPN];
    lat_rho_tile<T>(A, blockIdx.x, blockIdx.y, tiles);
}

template <typename T>
constexpr size_t lat_step_smem() {
    return (16 * (size_t)kPN + 18 * (size_t)kLTX * kLTY) * sizeof(T);
}

// Streaming from the halo tiles, bounce-back, collision and the write of one
// node of a step tile.
template <typename T>
__device__ __forceinline__ void lat_step_node(const LatArgs<T> &A, int k, bool interior, int lx, int ly,
                                              int tid, int32_t i, size_t n, T r0, T drx, T dry,
                                              T dmx, T dmy, T kx, T ky, T (*tiles)[kPN],
                                              T (*s_psi)[kLTX * kLTY]) {
    const Phys<T> &P = A.P;
    // streamed populations of this node go to shared memory (slot tid of
    // row a): keeps the 18 values out of registers
    const T dt = P.dt;
    s_psi[0][tid] = __ldg(A.fin + i);
    s_psi[9][tid] = __ldg(A.fin + 9 * n + i);
#pragma unroll
    for (int d = 1; d < 9; ++d) {
        s_psi[d][tid] = streamed<T>(A.c, k, interior, d, tiles[d - 1], lx, ly, dt);
        s_psi[9 + d][tid] = streamed<T>(A.c, k, interior, d, tiles[7 + d], lx, ly, dt);
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
    T sg = T(0), mx = T(0), my = T(0);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const T g = s_psi[9 + a][tid];
        sg += g;
        if (kEx(a)) mx += T(kEx(a)) * g;
        if (kEy(a)) my += T(kEy(a)) * g;
    }
    const CollidePrep<T> cp = collide_prep<T>(P, sg, mx, my, r0, drx, dry, dmx, dmy, kx, ky);
    const T r = cp.r, ux = cp.ux, uy = cp.uy, p = cp.p;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        T ho, go;
        collide_pop_rt<T>(cp, a, s_psi[a][tid], s_psi[9 + a][tid], ho, go);
        A.fout[(size_t)a * n + i] = ho;
        A.fout[(size_t)(9 + a) * n + i] = go;
    }
    if (!(finite_val(r) && finite_val(ux) && finite_val(uy) && finite_val(p))) atomicOr(A.flag, 1);
    if (A.mom) {
        A.mom[i] = r;
        A.mom[n + i] = ux;
        A.mom[2 * n + i] = uy;
        A.mom[3 * n + i] = p;
    }
}

constexpr int kRW = kLTX + 6, kRH = kLTY + 6;  // rho: halo 3
constexpr int kGW = kLTX + 4, kGH = kLTY + 4;  // grad rho: halo 2
constexpr int kMW = kLTX + 2, kMH = kLTY + 2;  // mu: halo 1

// Shared memory of one step tile: the scalar chain and, in lat_dsm (dynamic,
// lat_step_smem bytes), 16 halo tiles then 18 rows of streamed values.
template <typename T>
struct StepSmem {
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
    T (*tiles)[kPN] = reinterpret_cast<T (*)[kPN]>(lat_dsm);
    T (*s_psi)[kLTX * kLTY] = reinterpret_cast<T (*)[kLTX * kLTY]>(lat_dsm + 16 * kPN * sizeof(T));
    const int nx = A.nx, ny = A.ny, walls = A.walls;
    const int x0 = bx * kLTX, y0 = by * kLTY;
    const int tid = threadIdx.y * kLTX + threadIdx.x;
    constexpr int NT = kLTX * kLTY;
    const size_t n = (size_t)nx * ny;
    // 0. request the halo tiles of the 16 moving populations (h then g)
    const FillSlots f = fill_slots(tid, x0, y0, nx, ny, walls);
    issue_tiles<T, 0>(A, f, tiles, tid, n);
    issue_tiles<T, 9>(A, f, tiles + 8, tid, n);
    cp_async_commit();
    const auto &rc = A.c.r;  // recovery coefficients
    // 1. rho on the tile with a depth-3 halo (periodic wrap in x; in y wrap or,
    //    for walls, zero outside the domain: those entries meet only zero
    //    coefficients)
    for (int q = tid; q < RW * RH; q += NT) {
        const int ly = q / RW, lx = q - ly * RW;
        int gx = x0 + lx - 3, gy = y0 + ly - 3;
        while (gx < 0) gx += nx;  // the halo may span more than one period
        while (gx >= nx) gx -= nx;
        T v = T(0);
        if (walls) {
            if (gy >= 0 && gy < ny) v = __ldg(A.rho + gx + nx * gy);
        } else {
            while (gy < 0) gy += ny;
            while (gy >= ny) gy -= ny;
            v = __ldg(A.rho + gx + nx * gy);
        }
        s_rho[ly][lx] = v;
    }
    __syncthreads();
    // 2. recovered grad rho on the depth-2 region
    for (int q = tid; q < GW * GH; q += NT) {
        const int ly = q / GW, lx = q - ly * GW;
        const int gy = y0 + ly - 2;
        const int k = (walls && (gy == 0 || gy == ny - 1)) ? (gy == 0 ? 1 : 2) : 0;
        const T c0 = s_rho[ly + 1][lx + 1];
        T sx = T(0), sy = T(0);
#pragma unroll
        for (int o = 0; o < 6; ++o) {
            const T d = s_rho[ly + 1 + lat_dy(o)][lx + 1 + lat_dx(o)] - c0;
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
        s_mu[ly][lx] = mu_bulk<T>(P, s_rho[ly + 2][lx + 2]) - P.kappa * lap;
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
    const T r0 = s_rho[ly + 3][lx + 3];
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
