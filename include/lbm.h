/*
 * lbm.h - C ABI of the GB300 (sm_103a) two-component D2Q9 Shan-Chen lattice
 * Boltzmann solver for 2D Rayleigh-Taylor turbulence.
 *
 * The method is the one of Tavares, Biferale, Sbragaglia and Mailybaev,
 * "Validation and application of the lattice Boltzmann algorithm for a
 * turbulent immiscible Rayleigh-Taylor system" (arXiv 2101.04847):
 *   - densities and common velocity: Section 2, Eq. (1);
 *   - forced BGK kinetic equation: Section 2, Eq. "Kinetic equation";
 *   - shifted-velocity equilibrium: Section 2, Eq. "Equilibrium distribution";
 *   - Shan-Chen fluid-fluid force (psi = rho, no self-interaction):
 *     Section 2, Eq. "Shan-Chen forcing term";
 *   - fluid-boundary force: Section 2, Eq. after the Shan-Chen force;
 *   - Boussinesq buoyancy: Section 2, Eq. (3_Fex);
 *   - periodic x, solid bottom/top with bounce-back: Section 2, last paragraph;
 *   - energies, energy budget, stress split, interface length and enstrophy:
 *     Section 3 (Eqs. "Kinetic energy balance", "Three parts of the pressure
 *     tensor", "Korteweg stress and total length", "Dissipation function").
 *
 * Conventions for every entry point:
 *   - Every call returns an lbm_status; nothing throws across the ABI.
 *     lbm_last_error() gives a human-readable message for the calling thread.
 *   - Grids are nx (periodic, x) by ny (walls, y); y = 0 is the bottom wall row
 *     and y = ny-1 the top wall row.  Component A (index 0) is the heavy fluid
 *     on top, B (index 1) the light fluid below.  Directions:
 *     0 (0,0) 1 (1,0) 2 (0,1) 3 (-1,0) 4 (0,-1) 5 (1,1) 6 (-1,1) 7 (-1,-1) 8 (1,-1).
 *   - Host arrays are C-contiguous double arrays, row-major [y][x]; population
 *     arrays are [component][direction][y][x] and hold the post-streaming
 *     populations f_i^s(x, t) of the kinetic equation (the values whose sums are
 *     the densities of Eq. (1)).
 *   - Ownership: a device workspace or stream passed in is borrowed; the caller
 *     keeps it alive until lbm_destroy.  With a NULL workspace the library
 *     allocates (cudaMalloc) and frees its own.
 *   - Threads: one handle is used by one host thread at a time.
 *   - Work is queued asynchronously on the handle's stream; the calls that return
 *     data to the host (diagnostics, fields, populations, save) synchronise it.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,     /* invalid argument or parameter set */
    LBM_ENOMEM = 2,     /* allocation failed or workspace too small */
    LBM_ECUDA = 3,      /* a CUDA runtime call failed (message in lbm_last_error) */
    LBM_EUNSTABLE = 4,  /* sticky: a non-finite density, or one below -5 % of rho0_s =
                         * mass_s (1 + minority) / 2, was seen by the step (small transient
                         * negative values of a nearly absent component are part of the
                         * over-relaxed update near tau = 1/2, not a blow-up) */
    LBM_ETIMEOUT = 5,   /* sticky: a bounded device-side wait gave up */
    LBM_ESTATE = 6,     /* call not valid in the handle's current state */
    LBM_EIO = 7         /* file I/O error (save/load) */
} lbm_status;

typedef enum {
    LBM_STORE_F32 = 0,   /* populations stored as float */
    LBM_STORE_F16 = 1,   /* stored as half, shifted: h = f - w_i rho0_s */
    LBM_STORE_BF16 = 2   /* stored as bfloat16, shifted: h = f - w_i rho0_s */
} lbm_storage;

typedef enum {
    LBM_KERNEL_FUSED = 0,    /* one fused pull stream-collide kernel per step (global-memory pulls) */
    LBM_KERNEL_TWO_PASS = 1, /* density kernel + stream-collide kernel per step */
    LBM_KERNEL_STAGED = 2,   /* fused kernel, rows staged in shared memory by bulk async copies,
                              * block-wide sweep (the default: the fastest; the ensemble's tile code) */
    LBM_KERNEL_WARP = 3,     /* as STAGED, one independent sweep per warp */
    LBM_KERNEL_PIPE = 4,     /* as STAGED, warps sweep independently over shared stages (no block barrier) */
    LBM_KERNEL_DECOUPLED = 5,/* as STAGED (same tiles and row stages), but no block barrier per row: each warp
                              * keeps its own density ring, stages are handed back through per-stage barriers */
    LBM_KERNEL_PAIRED = 6    /* 16-bit storage only: as STAGED with 256-column tiles, each thread owning two
                              * neighbouring columns (per-row work shared by two sites, paired 32-bit stores);
                              * what STAGED runs for 16-bit storage when tile_x is 0 */
} lbm_kernel;

/* Parameters (lattice units, dx = dt = 1).  lbm_params_default() fills them. */
typedef struct {
    int32_t nx, ny;          /* grid; nx >= 4, ny >= 8 */
    double tau_A, tau_B;     /* BGK relaxation times, > 0.5 (kinematic viscosity cs^2 (tau - 1/2)) */
    double G;                /* G_AB of the Shan-Chen force */
    double G_wall_A;         /* G_Ab of the fluid-boundary force (0 = neutral wetting) */
    double G_wall_B;         /* G_Bb */
    double mass_A, mass_B;   /* bulk density of pure A (top) and pure B (bottom), > 0 */
    double g;                /* g~ of Eq. (3_Fex) */
    int32_t gravity_mode;    /* 0: F_A = -rho_A g e_y, F_B = +rho_B g e_y (Eq. 3_Fex); 1: -rho_s g e_y for both */
    double gx;               /* uniform body acceleration along x (validation cases) */
    uint64_t seed;           /* interface perturbation seed (splitmix64) */
    int32_t n_modes;         /* number of sinusoidal modes of the interface perturbation, 0..64 */
    double amp;              /* perturbation amplitude in cells */
    double width;            /* tanh half-width of the initial interface, > 0 */
    double minority;         /* fraction of the other component in each bulk, [0, 1) */
    double y0;               /* mean interface height; < 0 means ny / 2 */
    int32_t crop_rows;       /* rows cut at top and bottom for averages, >= 3, 2*crop_rows < ny */
    int32_t storage;         /* lbm_storage */
    int32_t kernel;          /* lbm_kernel */
    int32_t tile_y;          /* at most this many rows per block tile of the step kernel (the
                              * rows are split evenly over the tiles); 0 = the kernel's default
                              * (block-staged: one wave of tiles filling every SM) */
    double shift_A, shift_B; /* rho0_s of the shifted storage; <= 0 means (mass_s (1 + minority)) / 2 */
    int32_t tile_x;          /* columns per block tile of the block-staged kernel: 128 or 256
                              * (one column per thread); 0 = chosen per grid: for 16-bit storage
                              * the paired-column tile (256 columns, two per thread, the
                              * LBM_KERNEL_PAIRED kernel), for FP32 256 when the 256-column tiles
                              * are at least 64 rows tall, else 128.  Other kernels ignore it.
                              * Ensembles (the first member's value): 128 or 256 columns, one
                              * per thread, for every member; 0 = blocks of 128 threads, FP32
                              * members in 128-column tiles and 16-bit members in paired
                              * 256-column tiles (lbm_ens_tune picks among the three). */
    int32_t wall_mode;       /* pseudopotential beyond the walls in the Shan-Chen force (Section 2
                              * leaves it open): 0 = none (psi = 0 on the virtual rows y = -1 and
                              * y = ny); 1 = mirror (those rows hold the wall rows' own psi: a
                              * neutral wall that exerts no force on a uniform fluid) */
    int32_t x_offset;        /* the grid is columns [x_offset, x_offset + nx) of a whole grid of */
    int32_t nx_total;        /* nx_total columns (domain decomposition along x): the initial
                              * interface follows the whole grid; nx_total 0 = nx (x_offset 0) */
} lbm_params;

/* Diagnostics of one state (Section 3).  Averages <.> run over the sub-domain
 * without crop_rows rows at each wall; u is the physical velocity
 * (sum_{s,i} f c + (F_A + F_B)/2) / rho. */
typedef struct {
    int64_t step;        /* time step of the state */
    double mass_A;       /* sum of rho_A over the whole grid */
    double mass_B;       /* sum of rho_B over the whole grid */
    double E_k;          /* <rho |u|^2 / 2> */
    double E_p;          /* g <y phi>, phi = rho_A - rho_B */
    double buoyancy;     /* g <u_y phi> */
    double flux_pb;      /* <u . grad p_b>, p_b = cs^2 rho + G cs^2 (rho^2 - phi^2) / 4 */
    double flux_K;       /* <u . div P^K> (Korteweg stress, kappa = cs^4 G / 4) */
    double flux_tau;     /* <u . div K^(tau)> (spurious tau-dependent stress) */
    double viscous;      /* <u . div(eta grad u + eta grad u^T)>, eta = rho_bar cs^2 (tau - 1/2) */
    double enstrophy;    /* (1/2) sum omega^2 over the sub-domain */
    double rho_bar;      /* <rho> */
    double h;            /* mixing-layer width 6 sum_y c (1 - c), c the row mean of the mass
                          * fraction rho_A / (rho_A + rho_B) normalised by its two bulk values */
    double L_int;        /* interface length, 4-direction Cauchy-Crofton estimate */
    int64_t cc[4];       /* sign changes of (phi > 0) along 0, 90, 45, 135 degrees */
    int32_t status;      /* LBM_OK or LBM_EUNSTABLE */
} lbm_diag;

typedef struct lbm_handle lbm_handle;

/* Library version string. */
const char* lbm_version(void);

/* Text of a status code; never NULL. */
const char* lbm_status_str(lbm_status st);

/* Message of the last failing call on this thread; "" if none. */
const char* lbm_last_error(void);

/* Fill *p with the defaults: 128 x 256, tau 1, G 1.4, masses 1.0 / 0.9,
 * g 1e-5, Boussinesq gravity, 8 modes of amplitude 2, width 1.5, minority 0.08,
 * crop 10, FP32 fused.  Returns LBM_EINVAL if p is NULL. */
lbm_status lbm_params_default(lbm_params* p);

/* Bytes of device workspace lbm_create_ex needs for *p. */
lbm_status lbm_workspace_bytes(const lbm_params* p, size_t* bytes);

/* Create a solver with the defaults overridden by the arguments, on the current
 * device, with its own workspace and stream, initialised to the perturbed
 * interface (Section 2, last paragraph).  LBM_EINVAL on an invalid parameter. */
lbm_status lbm_create(int32_t nx, int32_t ny, double tau, double G, double mass_A,
                      double mass_B, double g, uint64_t seed, lbm_handle** out);

/* Create a solver from a full parameter set.  dev_workspace: NULL, or a device
 * buffer of at least lbm_workspace_bytes(p) bytes, 256-byte aligned, borrowed.
 * cuda_stream: a cudaStream_t to queue work on, or NULL for a stream owned by
 * the handle.  The state is initialised as in lbm_create. */
lbm_status lbm_create_ex(const lbm_params* p, void* dev_workspace, size_t ws_bytes,
                         void* cuda_stream, lbm_handle** out);

/* Re-initialise the state to step 0 (the initial condition of the parameters). */
lbm_status lbm_reset(lbm_handle* h);

/* Advance nsteps >= 0 time steps of the kinetic equation (Section 2): pull
 * streaming with periodic x and half-way bounce-back walls, densities and common
 * velocity (Eq. 1), Shan-Chen + wall + buoyancy forces, forced BGK collision.
 * Asynchronous; returns LBM_EUNSTABLE only if an earlier sync saw it. */
lbm_status lbm_step(lbm_handle* h, int64_t nsteps);

/* Wait for the queued work; LBM_EUNSTABLE if a NaN / negative density was seen. */
lbm_status lbm_sync(lbm_handle* h);

/* Current time step of the state. */
lbm_status lbm_step_count(lbm_handle* h, int64_t* step);

/* Test of the step kernels' timeout path (no counterpart in the paper): one launch of
 * the block-staged FP32 step with its bulk row copies withheld and its waits limited
 * to a few thousand polls, so that every wait gives up and raises the guard's timeout
 * bit with nothing in flight.  It writes garbage to the buffer the next step writes
 * and leaves the current state and the step count unchanged; the next lbm_sync or
 * lbm_diagnostics returns LBM_ETIMEOUT, which stays raised until lbm_reset.
 * FP32 storage only (else LBM_EINVAL); asynchronous. */
lbm_status lbm_step_test_timeout(lbm_handle* h);

/* Domain decomposition along x (an extension of the paper's single-grid runs): a
 * grid split into sub-grids of consecutive columns, one solver each (x_offset and
 * nx_total of lbm_params place a sub-grid in the whole grid), advances one step at
 * a time, and between steps every sub-grid's ghost columns take its neighbours' edge
 * columns.  The block-staged and decoupled kernels read the stored populations of
 * the two columns beside the grid from those ghost columns, so the split run equals
 * the whole-grid run bit for bit; the other kernels wrap x inside each solver and
 * cannot be split.  lbm_halo_pack copies the two edge columns of the current state
 * (side 0: columns 0, 1; side 1: nx - 2, nx - 1) to dev_buf, lbm_halo_unpack copies
 * dev_buf into the ghost columns (side 0: -2, -1 from the left neighbour's side-1
 * pack; side 1: nx, nx + 1 from the right neighbour's side-0 pack).  dev_buf: device
 * memory of lbm_halo_bytes bytes (36 * ny stored values, [plane][row][column]),
 * owned by the caller.  Both are queued on the solver's stream; side other than 0
 * or 1 gives LBM_EINVAL.  The diagnostics of a sub-grid treat it as periodic in x
 * (their derivatives at its two edges wrap inside it). */
lbm_status lbm_halo_bytes(lbm_handle* h, size_t* bytes);
lbm_status lbm_halo_pack(lbm_handle* h, int32_t side, void* dev_buf);
lbm_status lbm_halo_unpack(lbm_handle* h, int32_t side, const void* dev_buf);

/* Diagnostics of the current state (Section 3); synchronises.  *out is filled
 * even when the returned status is LBM_EUNSTABLE. */
lbm_status lbm_diagnostics(lbm_handle* h, lbm_diag* out);

/* The same evaluation without waiting: lbm_diagnostics_async launches the kernels
 * and the copies of their results (and of the guard flag) to pinned host memory on
 * the handle's stream and returns; lbm_diagnostics_wait blocks until those copies
 * are done (not later work on the stream) and fills *out, with the status
 * lbm_diagnostics would return.  One evaluation may be pending at a time
 * (LBM_ESTATE otherwise, and for a wait with none pending).  Lets a caller queue
 * the next steps before reading this step's result. */
lbm_status lbm_diagnostics_async(lbm_handle* h);
lbm_status lbm_diagnostics_wait(lbm_handle* h, lbm_diag* out);

/* Row means of phi = rho_A - rho_B over rows [crop_rows, ny - crop_rows) from
 * the last evaluation read (lbm_diagnostics or lbm_diagnostics_wait):
 * ny - 2 crop_rows doubles written to host_rows. */
lbm_status lbm_profile(lbm_handle* h, double* host_rows);

/* rho_A, rho_B and the physical velocity components on the whole grid, nx*ny
 * doubles each, host pointers ([y][x]); any of them may be NULL. */
lbm_status lbm_get_fields(lbm_handle* h, double* rhoA, double* rhoB, double* ux, double* uy);

/* Post-streaming populations, 2*9*ny*nx doubles, host pointer. */
lbm_status lbm_get_populations(lbm_handle* h, double* host);

/* Replace the state by the given post-streaming populations (2*9*ny*nx doubles,
 * host pointer), rounded to the storage type.  The step counter is kept. */
lbm_status lbm_set_populations(lbm_handle* h, const double* host);

/* The same two calls with FP32 host values (2*9*ny*nx floats, same layout): half
 * the bytes over the host link, exact for FP32 storage (for 16-bit storage the
 * values are rounded to it as above). */
lbm_status lbm_get_populations_f32(lbm_handle* h, float* host);
lbm_status lbm_set_populations_f32(lbm_handle* h, const float* host);

/* Asynchronous form of lbm_set_populations_f32: the host-to-device copy runs on a
 * copy stream of the handle into a staging buffer (72 bytes per site, allocated on
 * the first call; LBM_ENOMEM if that fails), so it overlaps work already queued on
 * the handle's stream; the state is replaced at this point of the handle's stream.
 * The host buffer must stay unchanged until the copy is done: lbm_sync returns,
 * or a result queued after this call is read (lbm_diagnostics_wait, or any
 * synchronising call); pinned memory makes the copy asynchronous. */
lbm_status lbm_set_populations_f32_async(lbm_handle* h, const float* host);

/* Write the raw stored state (header + populations) to a file / read it back
 * into a handle created with the same nx, ny and storage.  Bitwise round trip. */
lbm_status lbm_save(lbm_handle* h, const char* path);
lbm_status lbm_load(lbm_handle* h, const char* path);

/* Release the handle (and its own workspace / stream if it allocated them). */
void lbm_destroy(lbm_handle* h);

/* Pick the rows per tile (tile_y) of the handle's step kernel, and for the
 * block-staged kernel the columns per tile (tile_x: 128 or 256, and for 16-bit
 * storage also 0, the paired-column tile), by timing candidate
 * values (0 = the default among them) on the handle's own grid, then use the
 * fastest; lbm_get_params reports both.  The state and the step counter are left as
 * they were.  cache_path: NULL, or a text file of
 * "<gpu>|<kernel>|<storage>|<nx>x<ny> <tile_x> <tile_y> <ms>" lines; a matching line
 * is used without timing, a new result is appended (lines of another form are
 * skipped).  Outputs may be NULL. */
lbm_status lbm_tune(lbm_handle* h, const char* cache_path, int32_t* tile_y, double* ms_per_step);

/* The handle's parameters as in use (tile_x / tile_y after lbm_tune). */
lbm_status lbm_get_params(lbm_handle* h, lbm_params* out);

/* ---- Ensembles of independent realisations (Section 2: at least 10 runs per
 * experiment).  One kernel launch per time step advances every member; chunks
 * of steps are replayed as CUDA graphs.  Members may differ in grid, physics and
 * storage; each uses the staged kernel and its own workspace. ---- */
typedef struct lbm_ensemble lbm_ensemble;

/* n parameter sets (1..256); tile_y of members[0] is the rows per tile of every
 * member (0: chosen so that the tiles fill the device's block slots in whole waves).  cuda_stream: a cudaStream_t shared by all members, or NULL for one owned
 * by the ensemble. */
lbm_status lbm_ens_create(int32_t n, const lbm_params* members, void* cuda_stream, lbm_ensemble** out);

/* Advance every member by nsteps (asynchronous). */
lbm_status lbm_ens_step(lbm_ensemble* e, int64_t nsteps);

/* Wait; the first non-OK member status (LBM_EUNSTABLE / LBM_ETIMEOUT) if any. */
lbm_status lbm_ens_sync(lbm_ensemble* e);

/* Borrowed handle of member i, for diagnostics, fields, populations and
 * checkpoints; valid until lbm_ens_destroy.  lbm_step on it returns LBM_ESTATE. */
lbm_status lbm_ens_member(lbm_ensemble* e, int32_t i, lbm_handle** out);

/* Diagnostics of every member into out[0..n-1]; synchronises. */
lbm_status lbm_ens_diagnostics(lbm_ensemble* e, lbm_diag* out);

/* Pick the tile shape for the whole ensemble by timing candidates: the three tile
 * widths of lbm_params.tile_x (128, 256, 0 = paired 16-bit tiles) times tile heights
 * (0, the slot-filling default, among them); states are kept.  tile_y receives the
 * rows per tile in use.  The initial width is the first member's tile_x when it is
 * 128 or 256, else 0. */
lbm_status lbm_ens_tune(lbm_ensemble* e, int32_t* tile_y, double* ms_per_step);

/* Tile width of the ensemble's launch: 128, 256 or 0 (see lbm_params.tile_x). */
lbm_status lbm_ens_tile_width(lbm_ensemble* e, int32_t* tile_x);

void lbm_ens_destroy(lbm_ensemble* e);

/* ---- Learned closure of a 2x-coarsened run (an extension built on the solver;
 * the paper has none).  CNN: conv3x3 4->32, ReLU, conv3x3 32->32, ReLU,
 * conv3x3 32->4 on fields [4][ny][nx] = (rho_A, rho_B, u_x, u_y), x periodic and
 * zero padding beyond the walls; BF16 weights, FP32 accumulation; FP32 activations in
 * lbm_cnn_forward and the training kernels, BF16 activations in lbm_cnn_infer.
 * Parameters: one FP32 vector of LBM_CNN_PARAMS values, w1[32][4][3][3], b1[32],
 * w2[32][32][3][3], b2[32], w3[4][32][3][3], b3[4]. ---- */
#define LBM_CNN_PARAMS 11588

/* Device workspace for the CNN calls on an nx x ny image. */
lbm_status lbm_cnn_workspace_bytes(int32_t nx, int32_t ny, size_t* bytes);

/* y = CNN(x); all pointers device (x, y: 4*ny*nx floats). Asynchronous. */
lbm_status lbm_cnn_forward(const float* params, const float* x, int32_t nx, int32_t ny, void* workspace,
                           size_t ws_bytes, void* cuda_stream, float* y);

/* y = CNN(x) on the tensor cores (tcgen05): x and both hidden layers rounded to
 * BF16 (nearest even), FP32 accumulation; same parameters, layouts and workspace
 * as lbm_cnn_forward.  The learned closure corrects with this path.
 * Asynchronous; a bounded wait inside the kernels that gave up is reported by
 * lbm_cnn_infer_status. */
lbm_status lbm_cnn_infer(const float* params, const float* x, int32_t nx, int32_t ny, void* workspace,
                         size_t ws_bytes, void* cuda_stream, float* y);

/* Synchronises the stream; LBM_ETIMEOUT if a wait of the last lbm_cnn_infer on
 * this workspace gave up (its output is then incomplete), else LBM_OK. */
lbm_status lbm_cnn_infer_status(void* workspace, int32_t nx, int32_t ny, void* cuda_stream);

/* Test of the timeout path (no counterpart in the paper): lbm_cnn_infer with the
 * kernels' bulk copies withheld and their waits limited to a few thousand polls,
 * so every wait gives up, raises the status word and the kernels return (y is
 * left incomplete).  lbm_cnn_infer_status then reports LBM_ETIMEOUT; the next
 * lbm_cnn_infer clears the status. */
lbm_status lbm_cnn_infer_test_timeout(const float* params, const float* x, int32_t nx, int32_t ny, void* workspace,
                                      size_t ws_bytes, void* cuda_stream, float* y);

/* loss = mean((CNN(x) - t)^2) over the 4*ny*nx outputs (host), grad = dloss/dparams
 * (device, LBM_CNN_PARAMS floats).  Synchronises the stream. */
lbm_status lbm_cnn_loss_grad(const float* params, const float* x, const float* t, int32_t nx, int32_t ny,
                             void* workspace, size_t ws_bytes, void* cuda_stream, double* loss, float* grad);

typedef struct lbm_closure lbm_closure;

/* Parameters of the coarse run for a fine parameter set (diffusive scaling: nx/2,
 * ny/2, the same tau and G, g_c = 8 g; one coarse step = four fine steps, coarse
 * lattice velocities are twice the fine ones). */
lbm_status lbm_closure_coarse_params(const lbm_params* fine, lbm_params* coarse);

/* A fine and a coarse solver plus the network (He-initialised from seed); the
 * correction is applied every `interval` coarse steps. */
lbm_status lbm_closure_create(const lbm_params* fine, int32_t interval, uint64_t seed, void* cuda_stream,
                              lbm_closure** out);

/* Training data from the plain solver: for runs seeded seed0 .. seed0 + n_runs - 1,
 * after warmup fine steps, each interval restarts the coarse run from the restricted
 * fine fields, advances both, and keeps (coarse fields, restricted fine fields). */
lbm_status lbm_closure_generate(lbm_closure* c, int32_t n_runs, uint64_t seed0, int32_t warmup_fine_steps,
                                int32_t intervals_per_run);

/* Adam (lr) over the samples, one sample per update, shuffled per epoch; the mean
 * loss of the last epoch (normalised units) in *final_loss. */
lbm_status lbm_closure_train(lbm_closure* c, int32_t epochs, double lr, uint64_t shuffle_seed, double* final_loss);

/* Held-out run: fine run seeded `seed` (after warmup), coarse run started from its
 * restriction and corrected every interval by the network: use_net 0 = no
 * correction, 1 = densities and velocity, 2 = order parameter only (rho_A and rho_B
 * move by opposite amounts, velocity kept), 3 = order parameter and a quarter of the
 * velocity correction, 4 = as 3 with the order-parameter correction (and the mass
 * restoring offset) weighted by 4 c (1 - c) of the normalised mass fraction c, i.e.
 * applied on the interface and not in either bulk.  Corrections keep each component's
 * mass and never halve a density.  Diagnostics of both runs at intervals + 1 times
 * into coarse_out / fine_out (the fine run is the reference and the fallback: if the
 * coarse run turns unstable its status is returned, fine_out stays valid).  Each call
 * starts both runs afresh, their density guards cleared. */
lbm_status lbm_closure_evaluate(lbm_closure* c, uint64_t seed, int32_t warmup_fine_steps, int32_t intervals,
                                int32_t use_net, lbm_diag* coarse_out, lbm_diag* fine_out);

/* Production use of the closure: advance the coarse run by `intervals` intervals
 * of `interval` coarse steps, correcting it after each with mode use_net (0 = no
 * correction, 1-4 as in lbm_closure_evaluate), without running the fine solver.
 * Needs trained (or set) parameters for use_net > 0 (else LBM_ESTATE).  Queued on
 * the closure's stream; with use_net > 0 it then synchronises once to read the
 * tensor-core kernels' status: LBM_ETIMEOUT if a bounded wait of theirs gave up in
 * any interval (the coarse state is then unreliable).
 *
 * One correction, per site of the coarse grid (f the populations after streaming,
 * rho_s = sum_i f_i^s, rho = rho_A + rho_B, u_b = sum_{s,i} f_i^s c_i / rho):
 *   network input x = ((rho_A, rho_B, u_x, u_y) - in_mean) / in_scale with u the
 *     physical velocity (sum_{s,i} f_i^s c_i + F / 2) / rho, F the total force;
 *   p = CNN(x) * out_scale (lbm_cnn_infer), p = (dA, dB, du_x, du_y);
 *   d_s: mode 1 max(p_s, -rho_s / 2) minus its grid mean; modes 2, 3
 *     h = clamp((dA - dB) / 2, -rho_A / 2, rho_B / 2), d_A = h - mean(h), d_B = -d_A;
 *     mode 4 h = clamp(w (dA - dB) / 2, ...) with w = 4 c (1 - c), c the mass fraction
 *     rho_A / rho normalised by its bulk values (lbm_closure_evaluate) and clamped to
 *     [0, 1], d_A = h - w sum(h) / sum(w), d_B = -d_A;
 *   u' = u_b + a du, a = 1 (mode 1), 0 (mode 2), 1/4 (modes 3, 4);
 *   rho'_s = max(rho_s + d_s, 0),
 *   f_i^s <- f_i^eq(rho'_s, u') + (rho'_s / rho_s) (f_i^s - f_i^eq(rho_s, u_b)).
 * Arithmetic in FP32 per site; the grid sums are compensated FP32 sums per thread,
 * added in FP64 across threads. */
lbm_status lbm_closure_advance(lbm_closure* c, int32_t intervals, int32_t use_net);

/* One correction (mode use_net, as above) of the coarse run's current state, with
 * no time steps: lbm_closure_advance is lbm_step(coarse, interval) followed by this
 * call, interval after interval.  use_net 0 does nothing.  LBM_ESTATE without
 * trained or set parameters; synchronises the closure's stream and returns
 * LBM_ETIMEOUT as lbm_closure_advance does. */
lbm_status lbm_closure_correct(lbm_closure* c, int32_t use_net);

/* The closure in production, the call the method's workload makes (an extension:
 * the paper has no learned closure): advance the coarse run by coarse_steps coarse
 * steps (each worth four fine steps), correcting it with mode 4 (lbm_closure_advance)
 * after every full interval, then write the coarse run's diagnostics to *out.
 * Needs trained or set parameters (else LBM_ESTATE).  Synchronises the closure's
 * stream.
 *
 * The fine plain solver is the fallback.  The call first saves the coarse fields
 * (rho_A, rho_B, u).  If at the end the coarse run's guard reports a NaN or a
 * negative density, or a bounded wait of the tensor-core kernels gave up, the fine
 * solver restarts from those fields, prolonged bilinearly to the fine grid (mass of
 * each component kept, velocities halved to fine lattice units) at equilibrium, runs
 * 4 * coarse_steps fine steps, and the coarse run restarts from the restriction of
 * the result (2 x 2 block means, the velocity momentum-weighted); the call then
 * returns LBM_OK with the diagnostics of that state and lbm_closure_fallbacks counts
 * one more.  The first fallback allocates the fine buffers it needs: 16 floats of
 * fields and 72 doubles of populations per coarse site.
 * An instability of the fine run itself is returned (LBM_EUNSTABLE).  Shorter calls
 * lose less work to a fallback. */
lbm_status lbm_closure_run(lbm_closure* c, int64_t coarse_steps, lbm_diag* out);

/* How many lbm_closure_run calls fell back to the fine solver. */
lbm_status lbm_closure_fallbacks(lbm_closure* c, int64_t* count);

/* Copy the network parameters to (set = 0) or from (set = 1) host memory. */
lbm_status lbm_closure_params(lbm_closure* c, float* host, int32_t set);

/* Borrowed handles of the closure's fine and coarse solvers (either may be NULL). */
lbm_status lbm_closure_solvers(lbm_closure* c, lbm_handle** fine, lbm_handle** coarse);

/* Input means, input scales and output scales (12 floats) used by the network. */
lbm_status lbm_closure_normalisation(lbm_closure* c, float* host12);

/* Set them (host12 as above), e.g. with parameters saved from an earlier training:
 * LBM_EINVAL unless all 12 are finite and the 8 scales positive;
 * lbm_closure_train overwrites them with the statistics of its samples. */
lbm_status lbm_closure_set_normalisation(lbm_closure* c, const float* host12);

void lbm_closure_destroy(lbm_closure* c);

/* One time step that allocates nothing, for callers that cannot allocate device
 * memory: code running inside a host application or framework that owns the GPU
 * memory budget and forbids allocations outside it, or a loop that cannot take
 * the device-wide synchronisation a cudaMalloc / cudaFree can cause.  The paper
 * has no counterpart; this is an embedding interface.
 *
 * Same physics and FP32 arithmetic as lbm_step (the two-pass form: a density pass,
 * then collision and streaming).  pops_in and pops_out are device arrays of
 * 2*9*ny*nx floats, [component][direction][y][x], holding post-streaming
 * populations (the layout of lbm_get_populations, in FP32); they must not overlap
 * at all (LBM_EINVAL if they do).  pops_out receives the populations one step
 * later.  Only nx, ny, tau_A, tau_B, G, G_wall_A, G_wall_B, g, gravity_mode, gx
 * and wall_mode of *p are used; storage must be LBM_STORE_F32; 4 <= nx, 8 <= ny <= 65535.
 * cuda_stream: a cudaStream_t, or NULL for the default stream.  Asynchronous.
 * A CUDA error already pending when the call is made is returned as LBM_ECUDA
 * (and left pending); a launch failure is returned as LBM_ECUDA naming the kernel.
 *
 * Scratch: the densities go to a fixed device array inside the library of
 * 2 * 2^20 floats (8 MiB), held by every GPU that loads the library until the
 * process exits; grids with nx * ny > 2^20 are rejected with LBM_EINVAL.  A call
 * made outside a stream capture looks up that array's device address in the
 * current context (cudaGetSymbolAddress) and remembers it for the device; a call
 * made while cuda_stream is capturing uses the remembered address, so make one
 * call on each device before any stream capture, and again after a device reset
 * (cudaDeviceReset) or a switch to another context on that device, which
 * invalidate it (LBM_ESTATE if no address is remembered).  All calls share the
 * array: calls whose kernels overlap on the GPU (different streams, or threads)
 * race and give wrong results; serialise them.  No NaN / negative-density report:
 * use lbm_step on a handle for that. */
lbm_status lbm_step_noalloc(const lbm_params* p, const float* pops_in, float* pops_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
