// Batched time step: many structured-lattice states of uneven size advance
// in one launch per time step.
//
// The launch walks a global list of the 32 x 8 tiles of all meshes and runs
// the single-mesh tile step on each (so a state's results do not depend on
// which other states share the launch).  A tile step reads only the previous
// step's populations, so no tile waits for another within a launch.  The
// grid is either persistent (blocks per SM x SMs) or one block per tile.
// Block b starts with tile b and claims each further tile from the launch's
// counter at the start of its current tile; when the claimed tile is on the
// same mesh and loads by TMA, its h halo is requested as soon as the current
// tile has formed rho.  Launches of whole step pairs are captured in a CUDA
// graph.  An autotuner picks the grid and the tile order by timing real
// steps (all candidates compute identical values, so tuning steps are
// ordinary steps of the runs).
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "felbm_internal.h"
#include "felbm_kernels.cuh"
#include "felbm_lattice.cuh"

namespace felbm {

struct TileRef {
    uint16_t mesh, bx, by, pad;
};

template <typename T>
struct BatchMesh {
    LatArgs<T> a;  // fin / fout / mom / tmap are set per launch from f[], c0
    T *f[2];
    T *mom;
    const TMap *tmap;  // the state's 2 x 3 tensor maps, or nullptr
    int32_t c0;
};

template <typename T>
struct BatchArgs {
    const BatchMesh<T> *meshes;
    const TileRef *tiles;
    int32_t ntiles;
    unsigned *ctr;  // 2 tile counters, by parity
    int parity;
    int write_mom;
    // the coefficient tables of every mesh when they are all the same (same
    // lattice spacing and dt): read as kernel parameters by the SC kernels
    LatCoef<T> c;
};

template <typename T>
__device__ __forceinline__ void load_mesh(const BatchArgs<T> &B, int m, LatArgs<T> &sA, int &cur) {
    if (m == cur) return;
    const BatchMesh<T> &bm = B.meshes[m];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    static_assert(sizeof(LatArgs<T>) % 4 == 0, "word copy");
    const uint32_t *src = reinterpret_cast<const uint32_t *>(&bm.a);
    uint32_t *dst = reinterpret_cast<uint32_t *>(&sA);
    for (int w = tid; w < (int)(sizeof(LatArgs<T>) / 4); w += blockDim.x * blockDim.y) dst[w] = src[w];
    __syncthreads();
    if (tid == 0) {
        const int c = bm.c0 ^ B.parity;
        sA.fin = bm.f[c];
        sA.fout = bm.f[c ^ 1];
        sA.mom = B.write_mom ? bm.mom : nullptr;
        sA.tmap = bm.tmap ? bm.tmap + 3 * c : nullptr;
    }
    __syncthreads();
    cur = m;
}

// SC: all meshes share B.c (interior tiles then read the coefficients as
// constant operands, as the single-mesh step does), else each mesh's own
// tables from its shared-memory descriptor.
template <typename T, bool SC>
__device__ __forceinline__ const LatCoef<T> &batch_coef(const BatchArgs<T> &B, const LatArgs<T> &sA) {
    if constexpr (SC)
        return B.c;
    else
        return sA.c;
}

template <typename T, bool SC>
__global__ void __launch_bounds__(kNT, (sizeof(T) == 4 ? 768 : 512) / kNT) k_batch_step(const __grid_constant__ BatchArgs<T> B) {
    __shared__ StepSmem<T> S;
    __shared__ __align__(16) LatArgs<T> sA;
    extern __shared__ __align__(128) unsigned char bdsm[];
    const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
    if (lead && blockIdx.x == 0) B.ctr[B.parity ^ 1] = 0u;
    if ((int)blockIdx.x >= B.ntiles) return;
    lat_block_init<T>(S);
    TilePipe pp;
    int cur = -1;
    // block b starts with tile b and claims the following ones from
    // ctr[parity]; a claimed tile's h group is requested early only when it
    // is on the same mesh
    int t = blockIdx.x;
    for (;;) {
        const TileRef r = B.tiles[t];
        load_mesh<T>(B, r.mesh, sA, cur);
        NextTile next{0, 0, 0, false, false};
        if (lead) {
            next.t = (int)gridDim.x + (int)atomicAdd(&B.ctr[B.parity], 1u);
            next.valid = next.t < B.ntiles;
            if (next.valid) {
                const TileRef rn = B.tiles[next.t];
                next.bx = rn.bx;
                next.by = rn.by;
                next.tma = rn.mesh == r.mesh && tile_tma(sA, rn.bx, rn.by, bdsm);
            }
        }
        if (!lat_tile<T>(sA, batch_coef<T, SC>(B, sA), r.bx, r.by, S, bdsm, pp, next)) return;
        if (!take_next(S, pp)) return;
        t = S.nt[0];
    }
}

// One block per tile of the batch's tile list, at the register budget of
// the single-mesh step (4 blocks per SM in FP32).  Zeroes both tile counters,
// so that a walking launch after it starts from zero.
template <typename T, bool SC>
__global__ void __launch_bounds__(kNT, (sizeof(T) == 4 ? 1024 : 512) / kNT) k_batch_tile(const __grid_constant__ BatchArgs<T> B) {
    __shared__ StepSmem<T> S;
    __shared__ __align__(16) LatArgs<T> sA;
    extern __shared__ __align__(128) unsigned char bdsm[];
    if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        B.ctr[0] = 0u;
        B.ctr[1] = 0u;
    }
    lat_block_init<T>(S);
    const TileRef r = B.tiles[blockIdx.x];
    int cur = -1;
    load_mesh<T>(B, r.mesh, sA, cur);
    TilePipe pp;
    const NextTile none{0, 0, 0, false, false};
    lat_tile<T>(sA, batch_coef<T, SC>(B, sA), r.bx, r.by, S, bdsm, pp, none);
}

template <typename T>
static LatCoef<T> lat_coef_b(const felbm_mesh *m, double dt) {
    LatCoef<T> c;
    for (int k = 0; k < 3; ++k)
        for (int o = 0; o < 6; ++o) {
            const double ax = m->sinfo.a[k][o][0], ay = m->sinfo.a[k][o][1];
            const double bxx = m->sinfo.b[k][o][0], bxy = m->sinfo.b[k][o][1],
                         byy = m->sinfo.b[k][o][2];
            c.r[k][o][0] = (T)ax;
            c.r[k][o][1] = (T)ay;
            T sv[9];
            for (int a = 1; a < 9; ++a) {
                const double ex = kEx(a), ey = kEy(a);
                sv[a] = (T)(ex * ax + ey * ay +
                            0.5 * dt * (ex * ex * bxx + 2.0 * ex * ey * bxy + ey * ey * byy));
            }
            for (int q = 0; q < 4; ++q) {
                c.s[k][o][q].x = sv[pair_dir(q, 0)];
                c.s[k][o][q].y = sv[pair_dir(q, 1)];
            }
        }
    return c;
}

template <typename T>
static Phys<T> phys_b(const felbm_params &p) {
    const double d = p.rho_l - p.rho_v;
    Phys<T> P;
    P.rho_l = (T)p.rho_l;
    P.rho_v = (T)p.rho_v;
    P.beta = (T)(12.0 * p.sigma / (p.xi * d * d * d * d));
    P.kappa = (T)(1.5 * p.xi * p.sigma / (d * d));
    P.inv_tau_l = (T)(1.0 / p.tau_l);
    P.inv_tau_v = (T)(1.0 / p.tau_v);
    P.dt = (T)p.dt;
    P.gx = (T)p.gravity[0];
    P.gy = (T)p.gravity[1];
    P.inv_drho = (T)(1.0 / (p.rho_l - p.rho_v));
    return P;
}

FELBM_CHECK_READER(check_bits_batch)

}  // namespace felbm

using namespace felbm;

struct felbm_batch {
    std::vector<felbm_state *> states;
    int esize = 4;
    cudaStream_t stream = nullptr;
    void *d_meshes = nullptr;
    TileRef *d_tiles = nullptr;
    unsigned *d_ctr = nullptr;  // tile counters of the launches, by parity
    int32_t ntiles = 0;
    int parity = 0;
    int sm_count = 0, max_bps = 1;
    int bps = 1, order = 0;  // chosen configuration (bps 0: one block per tile)
    bool autotune = false, tuned = false;
    double tuned_ms = 0.0;
    cudaGraphExec_t graph = nullptr;
    bool graph_failed = false;
    int64_t launches = 0;
    std::vector<TileRef> tiles_mesh_major, tiles_interleaved;
    std::vector<int> c0;  // each state's current buffer when descriptors were built
    bool shared_coef = false;          // every mesh has the same coefficient tables
    std::vector<unsigned char> coef;   // those tables (LatCoef of the batch's precision)
};

static int b_status(cudaError_t e) {
    if (e == cudaSuccess) return FELBM_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return FELBM_ERR_OOM;
    }
    return FELBM_ERR_CUDA;
}

static size_t batch_smem(int esize) {
    return esize == 8 ? lat_smem<double>() : lat_smem<float>();
}

template <typename T>
static cudaError_t batch_launch(felbm_batch *b, int parity, int write_mom) {
    BatchArgs<T> B;
    B.meshes = reinterpret_cast<const BatchMesh<T> *>(b->d_meshes);
    B.tiles = b->d_tiles;
    B.ntiles = b->ntiles;
    B.ctr = b->d_ctr;
    B.parity = parity;
    B.write_mom = write_mom;
    std::memset(&B.c, 0, sizeof(B.c));
    if (b->shared_coef) std::memcpy(&B.c, b->coef.data(), sizeof(B.c));
    b->launches++;
    const dim3 blk(kLTX, kLTY);
    const size_t sm = batch_smem(sizeof(T));
    if (b->bps > 0) {
        const unsigned grid = (unsigned)(b->bps * b->sm_count);
        if (b->shared_coef)
            k_batch_step<T, true><<<grid, blk, sm, b->stream>>>(B);
        else
            k_batch_step<T, false><<<grid, blk, sm, b->stream>>>(B);
    } else if (b->shared_coef) {
        k_batch_tile<T, true><<<(unsigned)b->ntiles, blk, sm, b->stream>>>(B);
    } else {
        k_batch_tile<T, false><<<(unsigned)b->ntiles, blk, sm, b->stream>>>(B);
    }
    return cudaGetLastError();
}

static cudaError_t launch_any(felbm_batch *b, int parity, int write_mom) {
    return b->esize == 8 ? batch_launch<double>(b, parity, write_mom)
                         : batch_launch<float>(b, parity, write_mom);
}

static cudaError_t upload_tiles(felbm_batch *b) {
    const std::vector<TileRef> &src = b->order ? b->tiles_interleaved : b->tiles_mesh_major;
    return cudaMemcpy(b->d_tiles, src.data(), src.size() * sizeof(TileRef), cudaMemcpyHostToDevice);
}

static void drop_graph(felbm_batch *b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

// Graph of two steps starting at parity 0, without moments.
static void build_graph(felbm_batch *b) {
    drop_graph(b);
    if (b->graph_failed) return;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        b->graph_failed = true;
        return;
    }
    const int64_t l0 = b->launches;
    cudaError_t e1 = launch_any(b, 0, 0);
    cudaError_t e2 = launch_any(b, 1, 0);
    b->launches = l0;
    cudaError_t e3 = cudaStreamEndCapture(b->stream, &g);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess ||
        cudaGraphInstantiate(&b->graph, g, 0) != cudaSuccess) {
        cudaGetLastError();
        b->graph = nullptr;
        b->graph_failed = true;
    }
    if (g) cudaGraphDestroy(g);
}

template <typename T>
static int setup_meshes(felbm_batch *b) {
    const size_t n = b->states.size();
    std::vector<BatchMesh<T>> hm(n);
    for (size_t k = 0; k < n; ++k) {
        felbm_state *s = b->states[k];
        const felbm_mesh *m = s->mesh;
        BatchMesh<T> &bm = hm[k];
        std::memset(&bm, 0, sizeof(bm));
        bm.a.nx = m->sinfo.nx;
        bm.a.ny = m->sinfo.ny;
        bm.a.pitch = m->sinfo.pitch;
        bm.a.walls = m->sinfo.walls ? 1 : 0;
        bm.a.row0 = 0;  // whole lattices only (slabs are refused)
        bm.a.gny = bm.a.yhi = m->sinfo.ny;
        bm.a.ylo = 0;
        bm.a.c = lat_coef_b<T>(m, s->params.dt);
        bm.a.P = phys_b<T>(s->params);
        bm.a.rho = reinterpret_cast<T *>(s->scratch);  // first scratch field
        bm.a.flag = s->d_flag;
        lat_uniform_consts<T>(m->sinfo, s->params.dt, bm.a);
        bm.f[0] = reinterpret_cast<T *>(s->f[0]);
        bm.f[1] = reinterpret_cast<T *>(s->f[1]);
        bm.mom = reinterpret_cast<T *>(s->mom);
        bm.tmap = s->d_tmap;
        bm.c0 = s->cur;
        b->c0[k] = s->cur;
    }
    b->shared_coef = true;
    for (size_t k = 1; k < n; ++k)
        if (std::memcmp(&hm[k].a.c, &hm[0].a.c, sizeof(LatCoef<T>)) != 0) b->shared_coef = false;
    if (n) {
        const unsigned char *c = reinterpret_cast<const unsigned char *>(&hm[0].a.c);
        b->coef.assign(c, c + sizeof(LatCoef<T>));
    }
    return b_status(cudaMemcpy(b->d_meshes, hm.data(), n * sizeof(BatchMesh<T>), cudaMemcpyHostToDevice));
}

template <typename T>
static int occupancy(felbm_batch *b) {
    int bps = 0;
    const int sm = (int)batch_smem(sizeof(T));
    cudaError_t e = cudaFuncSetAttribute(k_batch_tile<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch_tile<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch_step<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch_step<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_batch_step<T, false>, kLTX * kLTY,
                                                          batch_smem(sizeof(T)));
    if (e != cudaSuccess) return b_status(e);
    b->max_bps = std::max(1, bps);
    return FELBM_OK;
}

// A state stepped on its own since the descriptors were built no longer
// matches them: wait for the stream (no launch may still read the
// descriptors) and rebuild them from the states' current buffers.
static int sync_descriptors(felbm_batch *b) {
    bool stale = false;
    for (size_t k = 0; k < b->states.size(); ++k)
        stale |= b->states[k]->cur != (b->c0[k] ^ b->parity);
    if (!stale) return FELBM_OK;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return b_status(e);
    b->parity = 0;
    return b->esize == 8 ? setup_meshes<double>(b) : setup_meshes<float>(b);
}

extern "C" {

int felbm_batch_create(felbm_state *const *states, int32_t n_states, uint32_t flags,
                       felbm_batch **out) {
    if (!states || n_states < 1 || n_states > 65535 || !out) return FELBM_ERR_INVALID_ARG;
    if (flags & ~FELBM_BATCH_AUTOTUNE) return FELBM_ERR_INVALID_ARG;
    felbm_batch *b = new (std::nothrow) felbm_batch();
    if (!b) return FELBM_ERR_OOM;
    try {
        b->states.assign(states, states + n_states);
    } catch (const std::bad_alloc &) {
        delete b;
        return FELBM_ERR_OOM;
    }
    for (int32_t k = 0; k < n_states; ++k) {
        felbm_state *s = states[k];
        const bool slab = s && s->mesh->kind == 1 && (s->mesh->sinfo.gny != s->mesh->sinfo.ny ||
                                                      (s->params.flags & FELBM_PARAM_LAP_FP64));
        if (!s || s->mesh->kind != 1 || slab || (int)s->esize != (int)states[0]->esize ||
            s->mesh->stream != states[0]->mesh->stream || s->mesh->sinfo.nx > 65535 * kLTX ||
            s->mesh->sinfo.ny > 65535 * kLTY) {
            delete b;
            return (s && (s->mesh->kind != 1 || slab)) ? FELBM_ERR_UNSUPPORTED : FELBM_ERR_INVALID_ARG;
        }
        for (int32_t q = 0; q < k; ++q)
            if (states[q] == s) {
                delete b;
                return FELBM_ERR_INVALID_ARG;
            }
    }
    b->esize = (int)states[0]->esize;
    b->c0.assign(n_states, 0);
    b->stream = states[0]->mesh->stream;
    b->autotune = (flags & FELBM_BATCH_AUTOTUNE) != 0;
    // tile lists: mesh-major and round-robin over meshes (largest first)
    std::vector<std::vector<TileRef>> per(n_states);
    for (int32_t k = 0; k < n_states; ++k) {
        const int tx = (states[k]->mesh->sinfo.nx + kLTX - 1) / kLTX;
        const int ty = (states[k]->mesh->sinfo.ny + kLTY - 1) / kLTY;
        for (int by = 0; by < ty; ++by)
            for (int bx = 0; bx < tx; ++bx)
                per[k].push_back(TileRef{(uint16_t)k, (uint16_t)bx, (uint16_t)by, 0});
        b->tiles_mesh_major.insert(b->tiles_mesh_major.end(), per[k].begin(), per[k].end());
    }
    {
        std::vector<size_t> pos(n_states, 0);
        bool any = true;
        while (any) {
            any = false;
            for (int32_t k = 0; k < n_states; ++k)
                if (pos[k] < per[k].size()) {
                    b->tiles_interleaved.push_back(per[k][pos[k]++]);
                    any = true;
                }
        }
    }
    b->ntiles = (int32_t)b->tiles_mesh_major.size();
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
    const size_t mesh_bytes = (size_t)n_states * (b->esize == 8 ? sizeof(BatchMesh<double>)
                                                                : sizeof(BatchMesh<float>));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_meshes, mesh_bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_tiles, (size_t)b->ntiles * sizeof(TileRef));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_ctr, 2 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(b->d_ctr, 0, 2 * sizeof(unsigned));
    int st = b_status(e);
    if (st == FELBM_OK) st = b->esize == 8 ? occupancy<double>(b) : occupancy<float>(b);
    if (st == FELBM_OK) {
        b->bps = b->max_bps;
        b->order = 0;
        st = b_status(upload_tiles(b));
    }
    if (st == FELBM_OK) st = b->esize == 8 ? setup_meshes<double>(b) : setup_meshes<float>(b);
    if (st != FELBM_OK) {
        felbm_batch_destroy(b);
        return st;
    }
    *out = b;
    return FELBM_OK;
}

// Time `trial` direct steps under each candidate (blocks per SM, or one
// block per tile, x tile order) and keep the fastest.  Steps taken here are ordinary steps.
static int autotune(felbm_batch *b, int trial, int64_t *used) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return FELBM_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return FELBM_ERR_CUDA;
    }
    double best = 1e30;
    int best_bps = b->bps, best_order = b->order;
    int st = FELBM_OK;
    for (int order = 0; order < 2 && st == FELBM_OK; ++order) {
        b->order = order;
        st = b_status(upload_tiles(b));
        for (int bps = 0; bps <= b->max_bps && st == FELBM_OK; ++bps) {
            b->bps = bps;
            // one untimed step, then `trial` timed steps
            cudaError_t e = launch_any(b, b->parity, 0);
            b->parity ^= 1;
            *used += 1;
            if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
            for (int k = 0; k < trial && e == cudaSuccess; ++k) {
                e = launch_any(b, b->parity, 0);
                b->parity ^= 1;
                *used += 1;
            }
            if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            st = b_status(e);
            if (st == FELBM_OK && ms / trial < best) {
                best = ms / trial;
                best_bps = bps;
                best_order = order;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != FELBM_OK) return st;
    b->bps = best_bps;
    b->order = best_order;
    b->tuned = true;
    b->tuned_ms = best;
    return b_status(upload_tiles(b));
}

int felbm_batch_step(felbm_batch *b, int64_t n_steps) {
    felbm::NvtxRange nvtx_range("felbm_batch_step");
    if (!b || n_steps < 0) return FELBM_ERR_INVALID_ARG;
    if (n_steps == 0) return FELBM_OK;
    int st0 = sync_descriptors(b);
    if (st0 != FELBM_OK) return st0;
    int64_t left = n_steps;
    cudaError_t e = cudaSuccess;
    if (b->autotune && !b->tuned) {
        const int trial = 3;
        const int64_t need = 2LL * (b->max_bps + 1) * (trial + 1) + 1;
        if (left > need) {
            int64_t used = 0;
            int st = autotune(b, trial, &used);
            left -= used;
            if (st != FELBM_OK) return st;
            drop_graph(b);
        }
    }
    // steps before an even parity, then graph pairs, then the last step
    // with the moments written
    while (left > 1 && b->parity != 0 && e == cudaSuccess) {
        e = launch_any(b, b->parity, 0);
        b->parity ^= 1;
        --left;
    }
    if (e == cudaSuccess && left > 2) {
        if (!b->graph && !b->graph_failed) build_graph(b);
        const int64_t pairs = (left - 1) / 2;
        for (int64_t p = 0; p < pairs && e == cudaSuccess; ++p) {
            if (b->graph) {
                e = cudaGraphLaunch(b->graph, b->stream);
                b->launches += 2;
            } else {
                e = launch_any(b, 0, 0);
                if (e == cudaSuccess) e = launch_any(b, 1, 0);
            }
        }
        left -= 2 * pairs;
    }
    while (left > 1 && e == cudaSuccess) {
        e = launch_any(b, b->parity, 0);
        b->parity ^= 1;
        --left;
    }
    if (e == cudaSuccess) {
        e = launch_any(b, b->parity, 1);
        b->parity ^= 1;
    }
    if (e != cudaSuccess) return b_status(e);
    // each state's current buffer follows the batch parity (host bookkeeping
    // only; the descriptors stay valid)
    for (size_t k = 0; k < b->states.size(); ++k) {
        felbm_state *s = b->states[k];
        s->cur = b->c0[k] ^ b->parity;
        s->have_moments = true;
        s->steps_done += n_steps;
    }
    return FELBM_OK;
}

int felbm_batch_sync(felbm_batch *b) {
    if (!b) return FELBM_ERR_INVALID_ARG;
    const cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return b_status(e);
    for (felbm_state *s : b->states) {
        const int st = felbm_state_sync(s);
        if (st != FELBM_OK) return st;
    }
    return FELBM_OK;
}

int felbm_batch_info(const felbm_batch *b, int32_t *blocks_per_sm, int32_t *tile_order,
                     int32_t *n_tiles, int64_t *launches, double *tuned_ms_per_step) {
    if (!b) return FELBM_ERR_INVALID_ARG;
    if (blocks_per_sm) *blocks_per_sm = b->bps;
    if (tile_order) *tile_order = b->order;
    if (n_tiles) *n_tiles = b->ntiles;
    if (launches) *launches = b->launches;
    if (tuned_ms_per_step) *tuned_ms_per_step = b->tuned ? b->tuned_ms : 0.0;
    return FELBM_OK;
}

void felbm_batch_destroy(felbm_batch *b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    drop_graph(b);
    cudaFree(b->d_meshes);
    cudaFree(b->d_tiles);
    cudaFree(b->d_ctr);
    delete b;
}

}  // extern "C"
