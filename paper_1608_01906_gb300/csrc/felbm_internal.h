// Internal declarations of the FE-LBM library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <vector>

#include "../../include/felbm.h"

namespace felbm {

// ---- checked build (FELBM_CHECKED) -----------------------------------------
// Kernels bounds-check the indices they gather with and record a violation
// as a bit of a device status word (no assert, no trap: the access is
// skipped); felbm_check_status reads and clears it.  Bits: 1 a gathered node
// or slot index out of range, 2 a shared-memory (region) index out of range,
// 4 a TMA box coordinate off its 16-byte rule (the tile then loads by
// cp.async), 8 a slab halo copy out of range.  Without FELBM_CHECKED every
// check is the constant true.  Each translation unit holds its own status
// word (no relocatable device code) and a reader, check_bits_<unit>().
#ifdef __CUDACC__
#ifdef FELBM_CHECKED
static __device__ unsigned g_check_bits;
__device__ __forceinline__ bool chk_idx(long long i, long long n, unsigned bit) {
    if (i >= 0 && i < n) return true;
    atomicOr(&g_check_bits, bit);
    return false;
}
#define FELBM_CHECK_READER(name)                                                  \
    unsigned name() {                                                             \
        unsigned v = 0, z = 0;                                                    \
        cudaDeviceSynchronize();                                                  \
        if (cudaMemcpyFromSymbol(&v, g_check_bits, sizeof v) != cudaSuccess) v = ~0u; \
        cudaMemcpyToSymbol(g_check_bits, &z, sizeof z);                           \
        return v;                                                                 \
    }
#else
__device__ __forceinline__ constexpr bool chk_idx(long long, long long, unsigned) { return true; }
#define FELBM_CHECK_READER(name) \
    unsigned name() { return 0u; }
#endif
#endif
// NVTX range around an entry point (seen by nsys / ncu; a no-op otherwise).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

unsigned check_bits_api();
unsigned check_bits_api3();
unsigned check_bits_batch();
unsigned check_bits_slab();

// ---- host-side mesh preprocessing (felbm_mesh.cu) -------------------------

// Assembled per-node operators in the internal (reverse Cuthill-McKee) order.
// For node i and each neighbour j != i sharing a triangle:
//   a_ij = sum_{T∋i,j} |T| grad N_j^T / (3 m_i)                 (2-vector)
//   b_ij = sum_{T∋i,j} |T| / m_i * sym(grad N_i^T (x) grad N_j^T)  (2x2, symmetric part)
// so that, with sum_j a_ij = 0 and sum_j b_ij = 0 (P1 partition of unity),
//   recovered gradient  (R f)_i   = sum_{j!=i} a_ij (f_j - f_i)
//   lumped TG streaming psi*_i    = psi_i - dt sum_{j!=i} (e.a_ij + dt/2 e.b_ij.e)(psi_j - psi_i)
struct HostCSR {
    int32_t n = 0;
    std::vector<int32_t> rowptr, col;
    std::vector<double> ax, ay, bxx, bxy, byy;
    std::vector<double> mass;      // lumped mass, internal order
    std::vector<uint8_t> tag;      // internal order, empty if no walls
    std::vector<int32_t> perm;     // perm[internal] = caller id
    std::vector<int32_t> iperm;    // iperm[caller] = internal id
    // Patches of the one-launch step (internal order is patch-major: patch p
    // owns the nodes [p kPatch, min(n, (p + 1) kPatch))).  Per patch its
    // region: its own nodes, then the nodes 1, 2, 3 and 4 edges away, as
    // internal ids in pnode[pnbase[p] ..); pcount[4 p ..] the cumulative
    // counts of rings <= 0, 1, 2, 3.  For the region nodes of rings <= 3,
    // prowbase gives the offset in plcol of the region indices of their CSR
    // columns (in CSR order).
    std::vector<int32_t> pnbase, pcount, pnode, prowbase;
    std::vector<uint16_t> plcol;
    int32_t rmax = 0, r1max = 0, r2max = 0, r3max = 0;  // largest region / ring <= 1, 2, 3 sizes
};

constexpr int kPatch = 256;  // nodes per patch of the general one-launch step
constexpr int64_t kPatchStepMaxNodes = 1 << 18;  // default patch step up to this size

// General tetrahedral mesh (3-D), same conventions: for each neighbour j != i
// a_ij = sum_{T∋i,j} |T| grad N_j / (4 m_i) (3 components) and the symmetric
// part of b_ij = sum |T|/m_i grad N_i (x) grad N_j (6 components: xx, xy, xz,
// yy, yz, zz).
struct HostCSR3 {
    int32_t n = 0;
    std::vector<int32_t> rowptr, col;
    std::vector<double> coef;      // 9 * nnz, SoA: ax, ay, az, bxx, bxy, bxz, byy, byz, bzz
    std::vector<double> mass;      // lumped mass m_i = sum |T|/4, internal order
    std::vector<uint8_t> tag;      // internal order, empty if no walls (1..18: inward e_k)
    std::vector<int32_t> perm;     // perm[internal] = caller id
    std::vector<int32_t> iperm;    // iperm[caller] = internal id
};

// Kuhn-split cube lattice (3-D): node i = x + nx (y + ny z) at (x, y, z) h,
// every cube cut into the six tetrahedra around its (0,0,0)-(1,1,1)
// diagonal, periodic in x and y, periodic in z or walled (tags 5 on z = 0,
// 6 on z = nz - 1).  The 14 neighbour offsets are lat3_d*(o); c holds the
// assembled coefficients (HostCSR3 order) per z-layer kind (0 interior, 1
// bottom wall layer, 2 top wall layer) and offset, zero where the offset
// leaves a walled domain.
struct Lattice3Info {
    bool ok = false;
    int32_t nx = 0, ny = 0, nz = 0;
    bool walls = false;
    double c[3][14][9];
};

#ifdef __CUDACC__
__host__ __device__
#endif
constexpr int lat3_dx(int o) {
    return (o == 0 || o == 6 || o == 8 || o == 12) ? 1 : (o == 1 || o == 7 || o == 9 || o == 13) ? -1 : 0;
}
#ifdef __CUDACC__
__host__ __device__
#endif
constexpr int lat3_dy(int o) {
    return (o == 2 || o == 6 || o == 10 || o == 12) ? 1 : (o == 3 || o == 7 || o == 11 || o == 13) ? -1 : 0;
}
#ifdef __CUDACC__
__host__ __device__
#endif
constexpr int lat3_dz(int o) {
    return (o == 4 || o == 8 || o == 10 || o == 12) ? 1 : (o == 5 || o == 9 || o == 11 || o == 13) ? -1 : 0;
}

struct StructuredInfo {
    bool ok = false;
    int32_t nx = 0, ny = 0;
    int32_t pitch = 0;   // population row pitch: nx rounded up to a multiple of 4
    bool walls = false;  // non-periodic y with walls on the first and last row
    double h = 1.0;
    // A slab of a sharded lattice (felbm_mesh_slab): storage row r is row
    // r + row0 of the whole lattice of gny rows, the slab's own rows are the
    // storage rows [ylo, yhi), with 4 halo rows below and above.  A whole
    // lattice: row0 = ylo = 0, gny = yhi = ny.
    int32_t row0 = 0, gny = 0, ylo = 0, yhi = 0;
    // 6 neighbour offsets (dx, dy) and their assembled a/b coefficients of an
    // interior node; wall rows get their own sets (bottom, top).
    double a[3][6][2];
    double b[3][6][3];
};

int build_csr(const double *xy, int64_t n_nodes, const int32_t *tri, int64_t n_tri,
              const double box[2], uint32_t flags, const uint8_t *tag, HostCSR &out);
// Tetrahedral mesh: validation, geometry, assembly, RCM (felbm_mesh3.cu).
int build_csr3(const double *xyz, int64_t n_nodes, const int32_t *tet, int64_t n_tet,
               const double box[3], uint32_t flags, const uint8_t *tag, HostCSR3 &out);
// Recognise the Kuhn lattice in an assembled tetrahedral mesh (H in RCM
// order); on success fills info (felbm_mesh3.cu).
void detect_lattice3(const double *xyz, int64_t n_nodes, const double box[3], uint32_t flags,
                     const uint8_t *tag, const HostCSR3 &H, Lattice3Info &info);
// Reverse Cuthill-McKee order of a node graph given as CSR without self loops.
std::vector<int32_t> rcm_order(int32_t n, const std::vector<int32_t> &rp,
                               const std::vector<int32_t> &cl);
// Recognise the structured lattice split; on success fills info (sizes and
// the coefficients of the three row kinds) and the lumped mass (lattice order).
void detect_structured(const double *xy, int64_t n_nodes, const int32_t *tri, int64_t n_tri,
                       const double box[2], uint32_t flags, const uint8_t *tag,
                       StructuredInfo &info, std::vector<double> &mass);

// ---- device-side views --------------------------------------------------

// Neighbour topologies.  for_each(i, fn) calls fn(j, ax, ay, bxx, bxy, byy)
// for every neighbour j != i of node i with the assembled coefficients a_ij,
// b_ij; tag_of(i) is the wall tag (0 = fluid).

// General mesh: CSR in reverse Cuthill-McKee order.
template <typename T>
struct DevCSR {
    int32_t n;
    const int32_t *rowptr;
    const int32_t *col;
    const T *ax, *ay, *bxx, *bxy, *byy;
    const uint8_t *tag;  // nullptr if no walls
#ifdef __CUDACC__
    template <typename Fn>
    __device__ __forceinline__ void for_each(int32_t i, Fn &&fn) const {
        const int32_t p1 = __ldg(rowptr + i + 1);
        for (int32_t p = __ldg(rowptr + i); p < p1; ++p) {
            const int32_t j = __ldg(col + p);
            if (!chk_idx(j, n, 1u)) continue;
            fn(j, __ldg(ax + p), __ldg(ay + p), __ldg(bxx + p), __ldg(bxy + p), __ldg(byy + p));
        }
    }
    __device__ __forceinline__ int tag_of(int32_t i) const { return tag ? (int)tag[i] : 0; }
    // population storage: slot of node i, slots per population array
    __device__ __forceinline__ size_t slot(int32_t i) const { return (size_t)i; }
    __device__ __forceinline__ size_t slots() const { return (size_t)n; }
#endif
};

// Structured lattice split (node i = x + nx*y): six neighbours at fixed
// offsets, coefficients of three row kinds (0 interior, 1 bottom wall row,
// 2 top wall row) held in the kernel parameters.  Populations are stored in
// rows of `pitch` slots (x + pitch*y), pitch = nx rounded up to a multiple
// of 4, so that every row starts 16-byte aligned.
// offsets o = 0..5: (1,0), (1,1), (0,1), (-1,0), (-1,-1), (0,-1)
#ifdef __CUDACC__
__host__ __device__
#endif
constexpr int lat_dx(int o) { return o == 0 || o == 1 ? 1 : (o == 3 || o == 4 ? -1 : 0); }
#ifdef __CUDACC__
__host__ __device__
#endif
constexpr int lat_dy(int o) { return o == 1 || o == 2 ? 1 : (o == 4 || o == 5 ? -1 : 0); }

template <typename T>
struct DevLattice {
    int32_t n, nx, ny, walls, pitch;
    int32_t row0, gny;  // storage row y is row y + row0 of a lattice of gny rows
    T c[3][6][5];  // ax, ay, bxx, bxy, byy
#ifdef __CUDACC__
    template <typename Fn>
    __device__ __forceinline__ void for_each(int32_t i, Fn &&fn) const {
        const int32_t y = i / nx, x = i - y * nx, gy = y + row0;
        const int kind = walls ? (gy == 0 ? 1 : (gy == gny - 1 ? 2 : 0)) : 0;
#pragma unroll
        for (int o = 0; o < 6; ++o) {
            int32_t yy = y + lat_dy(o);
            if (walls && (yy + row0 < 0 || yy + row0 >= gny)) continue;
            // (a slab's halo rows at the ends of its storage wrap onto its
            // own rows: their values feed only halo rows, which the halo
            // exchange replaces)
            yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
            int32_t xx = x + lat_dx(o);
            xx = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
            if (!chk_idx(xx + nx * yy, n, 1u)) continue;
            fn(xx + nx * yy, c[kind][o][0], c[kind][o][1], c[kind][o][2], c[kind][o][3],
               c[kind][o][4]);
        }
    }
    __device__ __forceinline__ int tag_of(int32_t i) const {
        if (!walls) return 0;
        const int32_t gy = i / nx + row0;
        return gy == 0 ? 2 : (gy == gny - 1 ? 4 : 0);
    }
    __device__ __forceinline__ size_t slot(int32_t i) const {
        const int32_t y = i / nx;
        return (size_t)(i - y * nx) + (size_t)pitch * (size_t)y;
    }
    __device__ __forceinline__ size_t slots() const { return (size_t)pitch * (size_t)ny; }
#endif
};

// Model constants of one state (Sec. 2.1), in the state's precision.
template <typename T>
struct Phys {
    T rho_l, rho_v, beta, kappa, inv_tau_l, inv_tau_v, dt, gx, gy;
    T inv_drho;  // 1 / (rho_l - rho_v)
};

// Storage of the 18 populations of a state: direction pairs interleaved.
// Each population array has S slots (S = N on general meshes, pitch * ny on
// structured ones; slot i of node i, or x + pitch*y).  With Np = S rounded up
// to a multiple of 4 (keeps every pair array 16-byte aligned): h_0 at
// [0, S); the h pairs q = 0..3 of opposite directions (1,3), (2,4), (5,7),
// (6,8) at Np + 2 Np q + 2 i + s, slot s = 0 for 1, 2, 5, 6 and s = 1 for 3,
// 4, 7, 8; g the same from offset 9 Np.  A state buffer holds 18 Np values.
// A pair is one 8-byte (FP32) or 16-byte (FP64) word per node, read and
// streamed together with packed two-wide arithmetic.
#ifdef __CUDACC__
__host__ __device__
#endif
constexpr int pair_of(int d) { return d == 1 || d == 3 ? 0 : (d == 2 || d == 4 ? 1 : (d == 5 || d == 7 ? 2 : 3)); }
#ifdef __CUDACC__
__host__ __device__
#endif
constexpr int slot_of(int d) { return d == 3 || d == 4 || d == 7 || d == 8 ? 1 : 0; }
// first direction of pair q (slot 0): 1, 2, 5, 6
#ifdef __CUDACC__
__host__ __device__
#endif
constexpr int pair_dir(int q, int s) { return s == 0 ? (q == 0 ? 1 : (q == 1 ? 2 : (q == 2 ? 5 : 6)))
                                                     : (q == 0 ? 3 : (q == 1 ? 4 : (q == 2 ? 7 : 8))); }
#ifdef __CUDACC__
__host__ __device__
#endif
#ifdef __CUDACC__
__host__ __device__
#endif
inline size_t pad4(size_t n) { return (n + 3) & ~(size_t)3; }
#ifdef __CUDACC__
__host__ __device__
#endif
inline size_t pop_index(int a, size_t i, size_t n) {
    const size_t np = pad4(n);
    const size_t base = a < 9 ? 0 : 9 * np;
    const int d = a % 9;
    return d == 0 ? base + i : base + np + 2 * np * (size_t)pair_of(d) + 2 * i + (size_t)slot_of(d);
}

template <typename T>
struct Fields {
    T *rho, *drx, *dry, *mu, *kx, *ky;  // N each
    // general meshes: the streamed, bounced-back h* of k_rho (population
    // layout: rest at [0, Np), pair q at Np + 2 Np q); nullptr otherwise
    T *hs;
};

}  // namespace felbm

// ---- opaque handles ---------------------------------------------------------

// Opaque storage of one TMA tensor map (CUtensorMap: 128 bytes, 64-byte
// aligned), encoded on the host and read by cp.async.bulk.tensor from
// global memory.
struct alignas(64) TMap {
    unsigned char bytes[128];
};

struct felbm_mesh {
    int64_t n_nodes = 0, n_tri = 0;
    uint32_t flags = 0;
    cudaStream_t stream = nullptr;
    int kind = 0;  // 0 general triangles, 1 structured triangles, 2 general tetrahedra, 3 tet lattice
    felbm::HostCSR host;
    felbm::HostCSR3 host3;
    felbm::Lattice3Info linfo3;
    felbm::StructuredInfo sinfo;
    // device arrays
    int32_t *d_rowptr = nullptr, *d_col = nullptr, *d_perm = nullptr;
    double *d_coef64 = nullptr;  // 5 * nnz, SoA: ax, ay, bxx, bxy, byy (kind 2: 9 * nnz, HostCSR3)
    float *d_coef32 = nullptr;
    double *d_mass = nullptr;
    uint8_t *d_tag = nullptr;
    // patches of the one-launch step of general triangle meshes (HostCSR)
    int32_t *d_pnbase = nullptr, *d_pcount = nullptr, *d_pnode = nullptr, *d_prowbase = nullptr;
    uint16_t *d_plcol = nullptr;
    bool patch_step = false;
    int64_t device_bytes = 0;
};

// Population slots per array of a state on mesh m, and the slot of node i
// (internal order).
inline int mesh_dim(const felbm_mesh *m) { return m->kind >= 2 ? 3 : 2; }
inline int mesh_q(const felbm_mesh *m) { return m->kind >= 2 ? 19 : 9; }
inline size_t pop_slots(const felbm_mesh *m) {
    return m->kind == 1 ? (size_t)m->sinfo.pitch * (size_t)m->sinfo.ny : (size_t)m->n_nodes;
}
inline size_t pop_slot(const felbm_mesh *m, size_t i) {
    if (m->kind != 1) return i;
    const size_t nx = (size_t)m->sinfo.nx;
    return i % nx + (size_t)m->sinfo.pitch * (i / nx);
}

struct felbm_state {
    const felbm_mesh *mesh = nullptr;
    felbm_params params{};
    int precision = FELBM_FP64;
    size_t esize = 8;
    void *f[2] = {nullptr, nullptr};  // 18 pad4(N) each, layout of pop_index
    int cur = 0;
    void *scratch = nullptr;          // 6 N: rho, drx, dry, mu, kx, ky
    void *mom = nullptr;              // 4 N: rho, ux, uy, p (internal order)
    double *d_out = nullptr;          // 5 N staging in caller order + reduction partials
    int *d_flag = nullptr;            // bit 0: non-finite field, bit 2: bounded wait gave up
    TMap *d_tmap = nullptr;           // structured meshes: 2 buffers x {h pairs, h rest, g pairs}
    void *halo = nullptr;             // slabs: halo messages send lo, send hi, recv lo, recv hi
    bool have_moments = false;
    int64_t steps_done = 0;
    // profiling: event pairs around launches (felbm_profile_enable)
    bool prof_on = false;
    int prof_stride = 1;                  // time every prof_stride-th launch of a kind
    int64_t prof_seen[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    std::vector<cudaEvent_t> prof_ev;     // 2 per timed launch
    std::vector<int> prof_kind;           // kind of each timed launch
    size_t prof_used = 0;
    int64_t launches[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

namespace felbm {
// Record the launch of a kernel of the given kind; when profiling, the
// returned event index brackets it (-1: not timed).
int prof_begin(felbm_state *s, int kind);
// Shared helpers of the C ABI (felbm_api.cu) and its 3-D part (felbm_api3.cu).
constexpr int kTotalsBlocks = 304;  // 2 x 152 SMs
int cuda_status(cudaError_t e);
bool params_ok(const felbm_params *p);
void mesh_free(felbm_mesh *m);
void state_free(felbm_state *s);
// Tetrahedral meshes (felbm_api3.cu): the state entry points of mesh kind 2.
int state_init3(const felbm_mesh *mesh, const felbm_params *params, const double *rho0,
                const double *u0, const double *p0, felbm_state **out);
void steps3(felbm_state *s, int64_t n);
int moments3(felbm_state *s, double *rho, double *C, double *u, double *p, double *totals);
int export3(felbm_state *s, double *hbar, double *gbar);
int import3(felbm_state *s, const double *hbar, const double *gbar);
// Encode and upload the tensor maps of a state on a structured mesh
// (felbm_tmap.cu); leaves d_tmap null where TMA is not usable.
void lattice_tmaps(felbm_state *s);
void prof_end(felbm_state *s, int slot);
}  // namespace felbm
