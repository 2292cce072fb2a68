// Internal declarations shared by the CUDA translation units of liblbm.
// Not part of the public ABI (include/lbm.h is).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

#include <string>

#include "../../include/lbm.h"

namespace lbm {

// ---------------------------------------------------------------------------
// D2Q9 lattice (Section 2): c_i, weights from the isotropy conditions,
// opposite directions.  Direction order matches include/lbm.h.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int cx(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 5 + 2) & 3) + 5);
}
__host__ __device__ constexpr float wf(int i) {
    return i == 0 ? 4.0f / 9.0f : (i <= 4 ? 1.0f / 9.0f : 1.0f / 36.0f);
}
__host__ __device__ constexpr double wd(int i) {
    return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}

constexpr int kThreadsX = 128;  // columns per block of the step kernels

// Physical constants of one solver, in the form the kernels use.
struct Physics {
    float om[2];       // 1 / tau_s
    float tau[2];      // tau_s
    float G;           // G_AB
    float ay_wall_bottom[2];  // wall-force acceleration on row 0 (per component)
    float ay_wall_top[2];     // wall-force acceleration on row ny-1
    float ay_ext[2];   // buoyancy acceleration along y (per component)
    float ax_ext;      // body acceleration along x
    float shift[2];    // rho0_s of the shifted storage (0 for FP32)
    float rho_floor[2];  // smallest density the instability guard accepts (see lbm_create)
    int wall_mirror;   // 1: the pseudopotential beyond a wall mirrors the wall row (wall_mode 1)
    // Time-step counter of the stochastic rounding: a launch reads *step_in and one of
    // its threads writes *step_in + 1 to *step_out, the counter the next launch reads
    // (two counters alternating with the buffers).  Null: no counter (seed 0).
    const uint32_t* step_in;
    uint32_t* step_out;
};

// Geometry of one population array set.
struct Grid {
    int nx, ny;
    int pitch;          // elements per stored row
    int origin;         // element offset of column 0 in a row (128 bytes); columns
                        // -2, -1, nx, nx+1 hold periodic copies of nx-2, nx-1, 0, 1
    size_t plane;       // elements per (component, direction) plane = ny * pitch
    int x_offset = 0;   // column 0 is column x_offset of a whole grid of nx_total columns
    int nx_total = 0;   // (domain decomposition; 0 = nx): the stochastic rounding's site index
};

// Columns of one block tile of the block-staged kernel (one thread per column): the
// ensemble kernel's and the narrow single-grid tile, and the wide single-grid tile.
constexpr int kBlockTileW = 128;
constexpr int kWideTileW = 256;
// Ensemble tile width 0: blocks of 128 threads, FP32 members in tiles of 128 columns
// (one per thread), 16-bit members in paired-column tiles of 256 (two per thread).
constexpr int kEnsPaired = 0;

struct StepLaunch {
    const void* fin;
    void* fout;
    float* psi;          // two-pass only: [2][ny][pitch]
    int* flag;           // guard flag (NaN / negative density)
    Grid grid;
    Physics phys;
    int storage;         // lbm_storage
    int tile_x;          // block-staged kernel: 128 or 256 columns per tile, 0 = chosen per grid
    int tile_y;
};

// One member of an ensemble launch (device-side table entry).
struct EnsMember {
    Grid grid;
    Physics phys;
    void* buf[2];        // the two population buffers (input = buf[parity])
    int* flag;           // the member's guard flag
    int storage;         // lbm_storage
    uint32_t* step_ctr;  // the member's two time-step counters (see Physics)
    int tiles_x;         // block tiles along x (ensemble_tile_cols columns each)
    int tiles_y;         // block tiles along y (rows split evenly)
    int tile_begin;      // index of the member's first tile in the flat list
};

// ensemble / tiling helpers (step_kernels.cu)
int warp_tiles(const Grid& g, int tile_y, int* tiles_x);
int default_tile_y();
// columns of one ensemble tile of a member with this storage (tile_x 128, 256 or kEnsPaired)
int ensemble_tile_cols(int storage, int tile_x);
// dynamic shared memory of one block tile for a storage type
size_t block_tile_smem_bytes(int storage, int tile_x);
// resident blocks of the ensemble kernel on the current device with `smem` bytes each
int ensemble_slots(size_t smem, int tile_x, cudaError_t* err);
cudaError_t launch_ensemble_step(const EnsMember* d_members, int n, int total_tiles, int parity, size_t smem,
                                 int tile_x, cudaStream_t st);

// handle accessors for the ensemble (lbm_api.cu)
void* handle_buffer(lbm_handle* h, int k);
int handle_parity(lbm_handle* h);
Grid handle_grid(lbm_handle* h);
Physics handle_phys(lbm_handle* h);
int* handle_flag(lbm_handle* h);
uint32_t* handle_step_counters(lbm_handle* h);
const lbm_params& handle_params(lbm_handle* h);
void handle_set_ensemble(lbm_handle* h, bool on);
void handle_advance(lbm_handle* h, int64_t n);
lbm_status handle_check(lbm_handle* h);
cudaError_t handle_save_state(lbm_handle* h);
cudaError_t handle_restore_state(lbm_handle* h);
cudaError_t handle_fields(lbm_handle* h, const double** rA, const double** rB, const double** ux, const double** uy);
cudaError_t handle_push_S(lbm_handle* h, const double* S);
// A handle's current population buffer, which the closure's correction reads and
// rewrites in place.
struct PopView {
    void* pops;
    Grid grid;
    int storage;
    float shift[2];
    cudaStream_t stream;
};
PopView handle_pops(lbm_handle* h);
lbm_status handle_reseed(lbm_handle* h, uint64_t seed);
// clear the guard flag (device word and the sticky host copies) after the state
// has been replaced, queued on the handle's stream
cudaError_t handle_clear_guard(lbm_handle* h);

// message returned by lbm_last_error() on this thread (lbm_api.cu)
void set_last_error(const std::string& msg);

// step kernels (step_kernels.cu)
cudaError_t launch_step(const StepLaunch& L, int kernel, cudaStream_t st);
// the block-staged FP32 step with its row copies withheld (tests of the timeout path)
cudaError_t launch_step_test_timeout(const StepLaunch& L, cudaStream_t st);
cudaError_t launch_init(void* fout, const Grid& g, int storage, const float shift[2],
                        const double* y0, double mass_A, double mass_B, double minority,
                        double width, cudaStream_t st);
// S (double, [2][9][ny][nx]) from the stored state
cudaError_t launch_pull_to_double(const void* fin, const Grid& g, int storage,
                                  const float shift[2], double* S, cudaStream_t st);
// stored state from S (double, [2][9][ny][nx])
cudaError_t launch_push_from_double(const double* S, const Grid& g, int storage,
                                    const float shift[2], void* fout, cudaStream_t st);
// the same with FP32 host-side values
cudaError_t launch_pull_to_float(const void* fin, const Grid& g, int storage, const float shift[2], float* S,
                                 cudaStream_t st);
cudaError_t launch_push_from_float(const float* S, const Grid& g, int storage, const float shift[2], void* fout,
                                   cudaStream_t st);

// diagnostics (diag_kernels.cu)
constexpr int kDiagTerms = 15;
enum DiagTerm {
    T_MASS_A = 0, T_MASS_B, T_EK, T_EP, T_BUOY, T_RHO, T_FLUX_PB, T_OMEGA2,
    T_FLUX_K, T_FLUX_TAU, T_VISC, T_N0, T_N90, T_N45, T_N135
};
struct DiagLaunch {
    const void* fin;
    Grid grid;
    int storage;
    float shift[2];
    double G, G_wall[2], g_ext[2], gx, tau_bar;
    int crop;
    int wall_mirror;     // pseudopotential beyond the walls: 0 none, 1 the wall rows' (wall_mode)
    double* scratch;     // 15 doubles per site
    double* partials;    // kDiagTerms * nblocks + 2 * ny * nbx
    double* out;         // kDiagTerms + 2 * ny doubles (terms, row sums of phi, of the mass fraction)
};
size_t diag_scratch_doubles(int nx, int ny);
size_t diag_partials_doubles(int nx, int ny);
// offset (in doubles) of the rho_A, rho_B, ux, uy fields (double [ny][nx] each) that
// launch_fields leaves in the scratch region
size_t diag_fields_offset(int nx, int ny);
cudaError_t launch_diagnostics(const DiagLaunch& D, cudaStream_t st);
// rho_A, rho_B, ux, uy (double [ny][nx] each) into the scratch region at
// diag_fields_offset (uses the whole scratch: 15 doubles per site)
cudaError_t launch_fields(const DiagLaunch& D, double* fields, cudaStream_t st);
// The closure network's input in FP32: rho_A, rho_B from rho2 [2][n] and the
// physical velocity (j + F/2) / rho from the momenta j2 [2][n] (the force from the
// neighbours' densities, as in the diagnostics), each as (v - mean[c]) / scale[c],
// into x [4][n].
cudaError_t launch_closure_features(const DiagLaunch& D, const float* rho2, const float* j2, const float mean[4],
                                    const float scale[4], float* x, cudaStream_t st);
cudaError_t handle_closure_features(lbm_handle* h, const float* rho2, const float* j2, const float mean[4],
                                    const float scale[4], float* x);

}  // namespace lbm
