/*
 * felbm.h -- C ABI of the GB300 finite-element lattice Boltzmann library for
 * binary fluids (Lee-Lin free-energy model, D2Q9 populations on a 2-D P1
 * triangle mesh).
 *
 * One time step (felbm_step) is the scheme of Sec. 2.2 of Matin, Misztal,
 * Hernandez-Garcia, Mathiesen, "Evaluation of the Finite Element Lattice
 * Boltzmann Method for Binary Fluid Flows":
 *   1. Taylor-Galerkin streaming of the stored pre-collided distributions h
 *      (the paper's f, zeroth moment rho) and g (pressure/momentum), P1
 *      Bubnov-Galerkin with the lumped mass matrix (Sec. 2.2.1, Eqs.
 *      local_formulation, galerkin_lbm, fem_matrices);
 *   2. bounce-back at wall nodes (Sec. 3.3, no-slip by bounce-back);
 *   3. rho, recovered grad rho, Laplacian of rho, stress force, chemical
 *      potential mu = mu_phi - kappa lap rho and its recovered gradient
 *      (Sec. 2.1 and Sec. 2.3);
 *   4. velocity and pressure moments (Eqs. velocity, pressure);
 *   5. post-streaming collision (Eqs. lbmf_post, lbmg_post) followed by the
 *      pre-streaming collision of the next step (Eqs. lbmf_pre, lbmg_pre)
 *      with forcing F (Eq. F), G (Eq. G) and the exact-difference body force.
 *
 * Conventions shared by every entry point
 *   - All host arrays are C-contiguous, in the caller's node numbering.  The
 *     library copies every input it needs; the caller keeps ownership of all
 *     arrays it passes and may free them after the call returns.
 *   - Handles are opaque, owned by the library, and released only by the
 *     matching *_destroy call.  A state borrows its mesh: the mesh must
 *     outlive every state created on it.
 *   - Every int-returning call returns FELBM_OK (0) or a negative
 *     felbm_status code; no call aborts, traps or exits.  A failed call leaves
 *     its output handle untouched.
 *   - D2Q9 population order: e_0 = (0,0), e_1 = (1,0), e_2 = (0,1),
 *     e_3 = (-1,0), e_4 = (0,-1), e_5 = (1,1), e_6 = (-1,1), e_7 = (-1,-1),
 *     e_8 = (1,-1); weights 4/9, 1/9 (1..4), 1/36 (5..8); c_s^2 = 1/3.
 *   - Work is issued on the CUDA stream given at mesh creation (NULL = the
 *     legacy default stream).  felbm_step returns after enqueueing; errors
 *     detected on the device (non-finite values) are reported by the next
 *     synchronising call (felbm_state_sync, felbm_moments_get,
 *     felbm_state_export).
 */
#ifndef FELBM_H
#define FELBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum felbm_status {
    FELBM_OK = 0,
    FELBM_ERR_INVALID_ARG = -1,  /* NULL handle/pointer, size out of range, bad flag */
    FELBM_ERR_INVALID_MESH = -2, /* index out of range, non-positive area, isolated node, bad tag */
    FELBM_ERR_OOM = -3,          /* device or host allocation refused */
    FELBM_ERR_NONFINITE = -4,    /* a NaN/Inf moment was produced by an earlier step */
    FELBM_ERR_TIMEOUT = -5,      /* a bounded device-side wait gave up */
    FELBM_ERR_CUDA = -6,         /* any other CUDA runtime error */
    FELBM_ERR_UNSUPPORTED = -7   /* valid request this build does not serve */
} felbm_status;

/* mesh flags */
#define FELBM_PERIODIC_X 0x1u   /* box[0] > 0 is the period in x */
#define FELBM_PERIODIC_Y 0x2u   /* box[1] > 0 is the period in y */
#define FELBM_MESH_GENERAL 0x4u /* never use the structured-lattice kernels */
#define FELBM_PERIODIC_Z 0x8u   /* tetrahedral meshes: box[2] > 0 is the period in z */
#define FELBM_MESH_SPLIT_STEP 0x10u /* general triangle meshes: always four launches per step */
#define FELBM_MESH_PATCH_STEP 0x20u /* general triangle meshes: always the one-launch patch step */

/* precision of the stored distributions and of the bulk arithmetic */
#define FELBM_FP64 0
#define FELBM_FP32 1

typedef struct felbm_mesh felbm_mesh;
typedef struct felbm_state felbm_state;
typedef struct felbm_batch felbm_batch;

/* Physical parameters (Sec. 2.1).  beta = 12 sigma / (xi drho^4) and
 * kappa = 3 xi sigma / (2 drho^2) with drho = rho_l - rho_v; the relaxation
 * parameter is the C-weighted harmonic mean of tau_l and tau_v; the kinematic
 * viscosity is nu = c_s^2 tau dt.  dt is in the mesh's length unit per unit
 * lattice speed (|e| = 1).  gravity is the body-force acceleration applied by
 * the exact-difference method with du = g dt (gravity[2], the z component, is
 * read on tetrahedral meshes only).  Requirements: rho_l > rho_v > 0,
 * sigma >= 0, xi > 0, tau_l > 0, tau_v > 0, dt > 0, all finite. */
typedef struct felbm_params {
    double rho_l, rho_v;
    double sigma, xi;
    double tau_l, tau_v;
    double dt;
    double gravity[3];
    int32_t precision; /* FELBM_FP64 or FELBM_FP32 */
    int32_t flags;     /* 0, or FELBM_PARAM_LAP_FP64 */
} felbm_params;

/* felbm_params.flags: FP32 states on triangle meshes form the kappa lap rho
 * term of mu (Sec. 2.1, Eq. F) in FP64: the Laplacian of rho (recovery of
 * the recovered FP32 gradient, with the mesh's FP64 coefficients) and its
 * product with kappa in FP64, subtracted from the FP32 bulk term in FP64 and
 * rounded once (for large density ratios, where kappa is large).
 * Everything else stays FP32.  No effect on FP64 states.  Tetrahedral
 * meshes and batches refuse it (UNSUPPORTED). */
#define FELBM_PARAM_LAP_FP64 0x1

/* Create a device-resident mesh (Sec. 2.2.1 P1 elements, Sec. 2.3 recovery).
 *   xy        host, n_nodes x 2 doubles (x, y), node coordinates.
 *   tri       host, n_tri x 3 int32 node ids, counter-clockwise: every
 *             triangle must have positive area once its second and third
 *             vertex are mapped to the minimum image of the first.
 *   box       host, 2 doubles: period in x and y; read only for the
 *             directions flagged periodic.  Every element edge must be shorter
 *             than half the period.
 *   flags     FELBM_PERIODIC_X | FELBM_PERIODIC_Y | FELBM_MESH_GENERAL |
 *             FELBM_MESH_SPLIT_STEP or FELBM_MESH_PATCH_STEP.
 *   node_tag  host, n_nodes uint8 or NULL: 0 = fluid; k in 1..8 = no-slip
 *             wall node whose inward normal is e_k.
 *   stream    cudaStream_t (as void*) all work of this mesh and its states is
 *             issued on; NULL = legacy default stream.
 * The library computes element geometry, the lumped mass, the assembled
 * streaming/recovery coefficients and an internal node order: patches of
 * 256 nodes along a Hilbert curve over the domain, reverse Cuthill-McKee
 * order within a patch.  A general mesh of up to 2^18 nodes steps in one
 * launch per step, one block per patch with the patch's nodes up to 4 edges
 * away staged in shared memory; larger ones in four launches per step over
 * global fields (measured faster there).  FELBM_MESH_SPLIT_STEP and
 * FELBM_MESH_PATCH_STEP force one of the two; both give the same results bit
 * for bit.  A mesh that is the structured split of a unit lattice
 * (node i at ((i mod nx) h, (i div nx) h), each square cut along its
 * (i,j)-(i+1,j+1) diagonal, periodic in x, periodic or walled in y) is served
 * by the structured-lattice kernels unless FELBM_MESH_GENERAL is set.
 * Errors: INVALID_ARG (NULL pointers, n_nodes < 3, n_tri < 1, sizes above
 * 2^31-1), INVALID_MESH, OOM, CUDA. */
int felbm_mesh_create(const double *xy, int64_t n_nodes, const int32_t *tri, int64_t n_tri,
                      const double box[2], uint32_t flags, const uint8_t *node_tag,
                      void *stream, felbm_mesh **out);

/* Create a device-resident tetrahedral mesh: the paper's own
 * three-dimensional setting (Sec. 2.2.1 linear tetrahedra with the lumped
 * mass m_i = sum |T|/4, Sec. 2.3 volume-weighted recovery; D3Q19).
 *   xyz       host, n_nodes x 3 doubles.
 *   tet       host, n_tet x 4 int32 node ids, positively oriented: the edge
 *             vectors from the first vertex to the others, at the minimum
 *             image of the periodic box, have a positive determinant.
 *   box       host, 3 doubles: periods, read for the flagged directions
 *             (every element edge shorter than half the period).
 *   flags     FELBM_PERIODIC_X | FELBM_PERIODIC_Y | FELBM_PERIODIC_Z |
 *             FELBM_MESH_GENERAL.
 *   node_tag  host, n_nodes uint8 or NULL: 0 = fluid; k in 1..18 = no-slip
 *             wall node whose inward normal is the D3Q19 direction e_k of
 *             the order (0,0,0), (+-1,0,0), (0,+-1,0), (0,0,+-1), (1,1,0),
 *             (-1,-1,0), (1,-1,0), (-1,1,0), (1,0,1), (-1,0,-1), (1,0,-1),
 *             (-1,0,1), (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1) (opposite
 *             directions are neighbours).
 *   stream    as for felbm_mesh_create.
 * The mesh has kind 2 (felbm_mesh_info) and is stepped by the general
 * kernels in D3Q19, except the Kuhn-split cube lattice: node i at
 * (i mod nx, (i div nx) mod ny, i div (nx ny)) h, each cube cut into the six
 * tetrahedra around its (0,0,0)-(1,1,1) diagonal, periodic in x and y,
 * periodic in z or walled with tags 5 on the bottom layer and 6 on the top
 * layer (nx, ny, nz >= 3).  Unless FELBM_MESH_GENERAL is set, that lattice
 * has kind 3: the kernels compute its neighbours from the node position and
 * take its coefficients from the kernel parameters (no assembled arrays on
 * the device); the results agree with kind 2 to rounding.
 * On states of tetrahedral meshes u has 3 components (u0 and u
 * are n_nodes x 3 doubles), totals has 4 entries (mass and the three
 * momentum components), and the checkpoint arrays hold 19 x n_nodes
 * doubles each.  Errors: as felbm_mesh_create (n_nodes < 4, n_tet < 1). */
int felbm_mesh_create_tet(const double *xyz, int64_t n_nodes, const int32_t *tet, int64_t n_tet,
                          const double box[3], uint32_t flags, const uint8_t *node_tag,
                          void *stream, felbm_mesh **out);

/* Mesh facts.  Any output pointer may be NULL.  kind: 0 = general
 * (unstructured CSR kernels), 1 = structured lattice, 2 = tetrahedral,
 * 3 = Kuhn tetrahedral lattice (n_tri then counts tetrahedra).  device_bytes: device memory held by the
 * mesh. */
int felbm_mesh_info(const felbm_mesh *mesh, int64_t *n_nodes, int64_t *n_tri, int32_t *kind,
                    int64_t *device_bytes);

void felbm_mesh_destroy(felbm_mesh *mesh);

/* Create a state and initialise it (Sec. 2.2): from rho0, u0, p0 the library
 * computes grad rho, the stress force and grad mu, takes the post-collision
 * distributions to be the equilibria h_eq = rho Gamma(u), g_eq (Eqs. f_eq,
 * g_eq), and stores the pre-collided values psi_eq + source.
 *   rho0  host, n_nodes doubles, > 0.
 *   u0    host, n_nodes x 2 doubles (ux, uy) or NULL for rest (x 3 on
 *         tetrahedral meshes).
 *   p0    host, n_nodes doubles or NULL for zero pressure.
 * Device memory: 2 x 18 n_nodes values of the chosen precision plus scratch
 * (2 x 38 n_nodes on tetrahedral meshes)
 * (structured meshes: also 768 bytes of TMA tensor maps; rows are padded to
 * a multiple of 4 slots, so every width qualifies).
 * Errors: INVALID_ARG, OOM, CUDA. */
int felbm_state_init(const felbm_mesh *mesh, const felbm_params *params, const double *rho0,
                     const double *u0, const double *p0, felbm_state **out);

/* Advance n_steps >= 0 time steps (asynchronous, on the mesh's stream).
 * The moments of the last step are kept for felbm_moments_get. */
int felbm_step(felbm_state *state, int64_t n_steps);

/* Wait for the state's work and report FELBM_ERR_NONFINITE if any step
 * produced a non-finite density, velocity or pressure, else
 * FELBM_ERR_TIMEOUT if a bounded device wait for a tile's TMA halo load gave
 * up (that step's tile was not updated). */
int felbm_state_sync(felbm_state *state);

/* Self-test of the failure detection of the bounded device waits (no GPU
 * fault involved): enqueues on the state's stream one block that waits, as a
 * tile waits for its TMA halo loads, on a shared-memory mbarrier that nothing
 * arrives on, with the time limit limit_ns (1 .. 2e9 nanoseconds) in place of
 * the step's 2 s.  When the limit runs out the block records the give-up in
 * the state's device flag exactly as a tile does, then returns, so the
 * context stays usable.  The next synchronising call on the state
 * (felbm_state_sync, felbm_moments_get, felbm_state_export) reports
 * FELBM_ERR_TIMEOUT, and keeps reporting it until felbm_state_import loads
 * new distributions.  Errors: INVALID_ARG (NULL state, limit out of range),
 * CUDA (launch failure). */
int felbm_wait_selftest(felbm_state *state, int64_t limit_ns);

/* Moments of the latest step (or of the initial fields before any step):
 *   rho  n_nodes doubles, C n_nodes doubles ((rho - rho_v)/(rho_l - rho_v)),
 *   u    n_nodes x 2 doubles (x 3 on tetrahedral meshes), p n_nodes doubles,
 *   totals 3 doubles: sum_i m_i rho_i, sum_i m_i rho_i ux_i, sum_i m_i rho_i uy_i
 *   (4 on tetrahedral meshes, with sum_i m_i rho_i uz_i)
 *   with m_i the lumped mass, accumulated in FP64 on the device.
 * Host buffers, any may be NULL.  Synchronises the stream. */
int felbm_moments_get(felbm_state *state, double *rho, double *C, double *u, double *p,
                      double totals[3]);

/* Checkpoint / restart of the stored pre-collided distributions: hbar and
 * gbar are host arrays of 9 x n_nodes doubles (19 x n_nodes on tetrahedral
 * meshes, D3Q19 order of felbm_mesh_create_tet), population-major
 * (hbar[a * n_nodes + i]), FP64 on the host whatever the state's precision.
 * Export synchronises the stream.  Import converts to the state's precision,
 * clears the non-finite flag, and leaves the state without moments:
 * felbm_moments_get returns FELBM_ERR_INVALID_ARG until the next felbm_step.
 * Errors: INVALID_ARG (NULL pointers, non-finite imported value), CUDA. */
int felbm_state_export(felbm_state *state, double *hbar, double *gbar);
int felbm_state_import(felbm_state *state, const double *hbar, const double *gbar);

void felbm_state_destroy(felbm_state *state);

/* ---- batched launch (many runs per launch; the paper has a single run) ---
 * A batch advances many states on structured meshes (felbm_mesh_info kind
 * 1) of any sizes in one launch per time step over every 32 x 8 tile of every
 * mesh.  Each state's results are the same as from felbm_step alone (same
 * per-tile code).  Step pairs are replayed from a CUDA graph.  With
 * FELBM_BATCH_AUTOTUNE the first felbm_batch_step long enough to afford it
 * times real steps under each candidate (a persistent grid of 1 to the
 * co-resident maximum blocks per SM, or one block per tile, reported as 0;
 * tile order mesh-major or interleaved) and keeps the fastest; those steps
 * count toward n_steps.  When every member has the same coefficient tables
 * (same lattice spacing and dt, and the same walls), the launch carries them
 * once as kernel parameters; otherwise each tile reads its mesh's tables.
 * Results are the same either way.
 *   states   n_states distinct states, same precision, meshes on the same
 *            stream; the batch borrows them (they must outlive it).
 * Stepping a member state on its own between batch steps is allowed; the
 * next felbm_batch_step then waits for the stream and rebuilds its tables.
 * Errors: INVALID_ARG, UNSUPPORTED (a general or tetrahedral mesh), OOM, CUDA; NONFINITE
 * (or TIMEOUT) from felbm_batch_sync as a member's felbm_state_sync reports
 * it. */
#define FELBM_BATCH_AUTOTUNE 0x1u
int felbm_batch_create(felbm_state *const *states, int32_t n_states, uint32_t flags,
                       felbm_batch **out);
int felbm_batch_step(felbm_batch *batch, int64_t n_steps);
int felbm_batch_sync(felbm_batch *batch);
/* Chosen configuration and counters; any output pointer may be NULL.
 * tile_order: 0 mesh-major, 1 interleaved across meshes. */
int felbm_batch_info(const felbm_batch *batch, int32_t *blocks_per_sm, int32_t *tile_order,
                     int32_t *n_tiles, int64_t *launches, double *tuned_ms_per_step);
void felbm_batch_destroy(felbm_batch *batch);

/* ---- profiling aid (no counterpart in the paper) ------------------------
 * Kernel kinds issued by felbm_step, reported by felbm_profile_read:
 *   0 stream h + rho, 1 grad rho, 2 lap rho / stress / mu,
 *   3 grad mu + stream + collide (the general four-pass step),
 *   4 lattice step (one launch per step on structured meshes),
 *   5 patch step (one launch per step on general triangle meshes),
 *   6-7 unused. */
#define FELBM_PROFILE_KINDS 8

/* on >= 1: every on-th launch of each kernel kind issued by later
 * felbm_step calls (the first, the (on+1)-th, ...) is bracketed by a pair of
 * CUDA events on the state's stream, up to 4096 timed launches after the
 * call; the others are counted, not timed (a stride spreads the timed
 * launches over a long run and keeps the event records out of most
 * launches).  on == 0 stops recording.  Errors: INVALID_ARG (NULL, on < 0),
 * OOM (event creation), CUDA. */
int felbm_profile_enable(felbm_state *state, int on);

/* Synchronise, then report per kernel kind the summed device milliseconds of
 * the timed launches (ms), how many launches were timed (timed) and how many
 * were issued in total since the last read or enable (launches); arrays of
 * FELBM_PROFILE_KINDS entries, any may be NULL.  Resets the counters. */
int felbm_profile_read(felbm_state *state, double *ms, int64_t *timed, int64_t *launches);

/* Static name of kernel kind k (NULL when out of range). */
const char *felbm_profile_kind_name(int k);

/* ---- allocation-free reduction (no counterpart in the paper) ------------
 * The same FP64 totals as felbm_moments_get -- sum_i w_i rho_i,
 * sum_i w_i rho_i ux_i, sum_i w_i rho_i uy_i -- over device arrays the
 * caller owns, for callers whose device memory belongs to another allocator
 * (a framework's caching allocator, an arena sized once at start-up) and who
 * therefore cannot let this library call cudaMalloc.  This entry point
 * allocates nothing: its scratch, 1024 x 3 partial sums (24 KiB), is a
 * fixed array in the library's device image that every GPU which loads the
 * library holds until the process exits.
 *   rho, ux, uy  device arrays of n values, double (FELBM_FP64) or float
 *                (FELBM_FP32) as precision says.
 *   weight       device array of n doubles (e.g. the lumped nodal mass), or
 *                NULL for unit weights.
 *   n            1 .. FELBM_NALLOC_MAX_NODES; larger n returns
 *                FELBM_ERR_INVALID_ARG.
 *   totals       device array of 3 doubles, written by the call.
 *   stream       cudaStream_t (as void*) the work is issued on; NULL = the
 *                legacy default stream.  The call returns after enqueueing.
 * The first call on a device, with that device current, looks up the device
 * address of the scratch array and keeps it for the life of the process;
 * make that first call before any stream capture, and do not use this entry
 * point on a device after cudaDeviceReset (the device image is reloaded and
 * the kept address no longer names the array).  All calls on a device share the one scratch array and leave
 * their partial sums in it (each call writes every slot it reads, so nothing
 * needs clearing); calls whose work overlaps on the GPU -- on different
 * streams, or from different host threads without ordering -- race on it.
 * Errors: INVALID_ARG (NULL pointer, n out of range, bad precision),
 * UNSUPPORTED (device ordinal >= 64), CUDA. */
#define FELBM_NALLOC_MAX_NODES (1LL << 30)
int felbm_totals_nalloc(const void *rho, const void *ux, const void *uy, const double *weight,
                        int64_t n, int32_t precision, double *totals, void *stream);

/* Measured arithmetic peak of the current device, in flop/s (an FMA counts
 * as 2): one full-occupancy launch of independent FMA chains per thread,
 * timed with CUDA events on the legacy default stream (best of three after a
 * warm-up launch).  kind: 0 = FP32 FMA, 1 = FP32 packed two-wide FMA
 * (FFMA2), 2 = FP64 FMA.  These are the ALU ceilings of the step kernels.
 * Synchronises the default stream; allocates 16 bytes of device memory for
 * the call.  Errors: INVALID_ARG (NULL pointer, kind out of range), CUDA. */
int felbm_alu_peak(int kind, double *flops_per_s);

/* ---- Halo-sharded structured lattices ----------------------------------
 * A structured lattice (felbm_mesh_create's split lattice) too large for one
 * device is cut into slabs of whole rows, one per device (the paper's large
 * single meshes, Sec. 3.4, split spatially).  A node's next state depends on
 * the present populations up to 4 rows away (h streamed on the depth-3
 * density region, whose rows are streamed from their depth-1 neighbours;
 * rho -> grad rho -> lap rho and mu -> grad mu, Sec. 2.2.1 and Sec. 2.3), so
 * a slab holds its own rows plus 4 halo rows below and above, steps its own
 * rows, and after every step (and once after felbm_state_init) its halo
 * rows are replaced by its neighbours' first and last 4 own rows.  The
 * slabs of a run then reproduce the whole lattice's run bitwise when every
 * cut (y_begin) is a multiple of 8 rows (the step's tile height: every node
 * is then updated by the same code path as in the whole lattice).
 *
 * felbm_mesh_slab: the slab of rows [y_begin, y_begin + n_rows) of the
 * whole structured lattice `mesh` (made by felbm_mesh_create; the slab
 * copies what it needs, so `mesh` may be destroyed after the call), with its
 * work on cuda_stream.
 * Its nodes are the n_rows + 8 storage rows in lattice order, row r being
 * row y_begin - 4 + r of the lattice (modulo its rows when y is periodic;
 * rows outside a walled lattice are kept but never read): states on it take
 * and return fields of nx * (n_rows + 8) nodes.  The lumped masses of the
 * halo rows are zero, so a slab state's totals are its own rows' share.
 * n_rows >= 8 and the slab inside the lattice; batches refuse slab states.
 * Errors: INVALID_ARG, UNSUPPORTED (not a structured lattice, or a slab),
 * OOM, CUDA. */
int felbm_mesh_slab(const felbm_mesh *mesh, int64_t y_begin, int64_t n_rows, void *cuda_stream,
                    felbm_mesh **out);

/* The slab's first own row in the lattice, its own row count, and the bytes
 * of one FP32 halo message (twice that in FP64).  INVALID_ARG if mesh is
 * not a slab. */
int felbm_slab_info(const felbm_mesh *mesh, int64_t *y_begin, int64_t *n_rows, int64_t *halo_bytes_fp32);

/* The state's four halo messages (device memory owned by the state, 16-byte
 * aligned, zeroed at first use): send[0] (its first 4 own rows, for the slab
 * below), send[1] (its last 4 own rows, for the slab above), recv[0] (for
 * its 4 halo rows below), recv[1] (above); *bytes per message.  A transport
 * between devices (NCCL send/recv, peer copies) carries send[1] of slab k to
 * recv[0] of slab k+1 and send[0] of slab k+1 to recv[1] of slab k, on the
 * states' streams, between felbm_slab_pack and felbm_slab_unpack.
 * Layout: per message, 4 rows (pitch = nx rounded up to 4 slots) of h_0, of
 * the 4 h direction-pair arrays (2 values per slot), of g_0 and of the 4 g
 * pair arrays: 72 x pitch values of the state's precision. */
int felbm_slab_halo(felbm_state *state, void **send, void **recv, int64_t *bytes);

/* Enqueue (one launch each, on the state's stream): pack the current
 * populations' first and last 4 own rows into send[0], send[1]; unpack
 * recv[0], recv[1] into the 4 halo rows below and above.  INVALID_ARG if the
 * state is not on a slab. */
int felbm_slab_pack(felbm_state *state);
int felbm_slab_unpack(felbm_state *state);

/* The exchange of one device's chain of slab states that together tile the
 * lattice's rows in order (slabs[0] starting at row 0, all of one
 * precision and on one stream): pack all, copy each message to its
 * neighbour (periodic y: around the ends; walled: nothing across the
 * walls), unpack all.  Asynchronous.  Errors: INVALID_ARG (not such a
 * chain), CUDA. */
int felbm_slab_exchange(felbm_state *const *slabs, int32_t n_slabs);

/* Checked build (library compiled with FELBM_CHECKED, libfelbm_checked.so):
 * the kernels bounds-check the indices they gather with -- node and slot
 * indices of the CSR, lattice and patch neighbours, shared-memory region
 * indices, the cp.async fill plans, the TMA boxes' 16-byte x rule, the slab
 * halo copies -- and, instead of an out-of-range access, skip it and record
 * a bit of a device status word (no assert, no trap).  This call waits for
 * the device, reads and clears that word: *bits = 1 a node or slot index out
 * of range, 2 a shared-memory index out of range, 4 a TMA coordinate off its
 * rule (that tile loaded by cp.async), 8 a slab copy out of range;
 * *checked_build = 1 in the checked build.  The regular build returns 0 for
 * both (its checks compile away).  Errors: INVALID_ARG (NULL pointer). */
int felbm_check_status(int32_t *checked_build, int32_t *bits);

/* Short static description of a status code. */
const char *felbm_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* FELBM_H */
