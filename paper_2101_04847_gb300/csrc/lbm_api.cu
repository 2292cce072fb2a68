// Host side of the C ABI declared in include/lbm.h: parameter validation,
// workspace layout, stream and CUDA-graph management, diagnostics assembly,
// host transfers and checkpoints.  All compute runs in the kernels of
// step_kernels.cu and diag_kernels.cu.
#include "lbm_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

namespace {

thread_local std::string g_last_error;

lbm_status fail(lbm_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

lbm_status cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return LBM_ECUDA;
}

#define LBM_TRY(call, what)                                \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

constexpr int kGraphChunk = 50;   // steps per captured CUDA graph
constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

size_t elem_size(int storage) { return storage == LBM_STORE_F32 ? 4 : 2; }

// ---------------------------------------------------------------------------
// splitmix64 (Steele, Lea, Flood, OOPSLA 2014) for the interface perturbation
// ---------------------------------------------------------------------------
uint64_t splitmix64_next(uint64_t& state) {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double unit_double(uint64_t v) { return (double)(v >> 11) * (1.0 / 9007199254740992.0); }

// Interface height y0(x) = base + amp * eta(x) / max|eta|,
// eta(x) = sum_{m=1..M} a_m sin(2 pi m x / nx + theta_m), draws a_1, theta_1, a_2, ...
// Interface heights y0(x) for the handle's columns x = -1 .. nx (index x + 1): the
// columns beside the grid too, which the initial state's streamed-in populations come
// from.  Column x is column x_offset + x of the whole grid of nx_total columns
// (periodic), so the sub-grids of a split grid start from the whole grid's state;
// the normalisation uses the whole grid's largest deflection.
std::vector<double> interface_height(const lbm_params& p) {
    const double two_pi = 6.283185307179586476925286766559;
    const int total = p.nx_total > 0 ? p.nx_total : p.nx;
    std::vector<double> a(p.n_modes), th(p.n_modes);
    uint64_t st = p.seed;
    for (int m = 0; m < p.n_modes; ++m) {
        a[m] = unit_double(splitmix64_next(st));
        th[m] = two_pi * unit_double(splitmix64_next(st));
    }
    auto eta_at = [&](int xg) {
        double e = 0.0;
        for (int m = 0; m < p.n_modes; ++m) e += a[m] * std::sin(two_pi * (m + 1) * xg / total + th[m]);
        return e;
    };
    double peak = 0.0;
    for (int xg = 0; xg < total; ++xg) peak = std::fmax(peak, std::fabs(eta_at(xg)));
    const double base = p.y0 < 0.0 ? p.ny / 2.0 : p.y0;
    std::vector<double> y0(p.nx + 2);
    for (int x = -1; x <= p.nx; ++x) {
        const int xg = ((x + p.x_offset) % total + total) % total;
        y0[x + 1] = peak > 0.0 ? base + p.amp * eta_at(xg) / peak : base;
    }
    return y0;
}

struct Layout {
    size_t pops[2], psi, scratch, partials, out, flag, y0, total;
    size_t pop_bytes, plane;
    int pitch, origin;
};

Layout make_layout(const lbm_params& p) {
    Layout L;
    // column 0 sits 128 bytes into each row; the row leaves room for the staged
    // kernels' windows (up to 144 columns from x0 - 10, x0 < nx; the 256-column tile's
    // up to 8 columns past nx rounded up to 256) and the ghost copies.  No wider: at
    // 1024 x 2048 a row of 1344 floats instead of 1216 measured 0.5 % slower.
    L.origin = (int)(128 / elem_size(p.storage));
    const int wide_end = (p.nx + lbm::kWideTileW - 1) / lbm::kWideTileW * lbm::kWideTileW + 8;
    L.pitch = (L.origin + std::max(p.nx + lbm::kBlockTileW + 32, wide_end) + 63) / 64 * 64;
    L.plane = (size_t)p.ny * L.pitch;
    L.pop_bytes = 18 * L.plane * elem_size(p.storage);
    const size_t n = (size_t)p.nx * p.ny;
    size_t off = 0;
    L.pops[0] = off; off = align_up(off + L.pop_bytes);
    L.pops[1] = off; off = align_up(off + L.pop_bytes);
    L.psi = off; off = align_up(off + 2 * L.plane * sizeof(float));
    // scratch: diagnostics fields, host staging (18 doubles per site), or a saved copy
    // of one population buffer (tuning)
    const size_t scratch_b = std::max({lbm::diag_scratch_doubles(p.nx, p.ny) * sizeof(double),
                                       (size_t)18 * n * sizeof(double), L.pop_bytes});
    L.scratch = off; off = align_up(off + scratch_b);
    L.partials = off; off = align_up(off + lbm::diag_partials_doubles(p.nx, p.ny) * sizeof(double));
    L.out = off; off = align_up(off + (lbm::kDiagTerms + 2 * (size_t)p.ny) * sizeof(double));
    L.flag = off; off = align_up(off + 16);
    L.y0 = off; off = align_up(off + (size_t)(p.nx + 2) * sizeof(double));
    L.total = off;
    return L;
}

lbm_status validate(const lbm_params* p) {
    if (!p) return fail(LBM_EINVAL, "params is NULL");
    if (p->nx < 4 || p->ny < 8) return fail(LBM_EINVAL, "nx must be >= 4 and ny >= 8");
    if ((int64_t)p->nx * p->ny > (int64_t)1 << 31) return fail(LBM_EINVAL, "nx*ny must be < 2^31");
    if (!(p->tau_A > 0.5) || !(p->tau_B > 0.5)) return fail(LBM_EINVAL, "tau must be > 0.5");
    if (!(p->mass_A > 0.0) || !(p->mass_B > 0.0)) return fail(LBM_EINVAL, "masses must be > 0");
    if (!(p->width > 0.0)) return fail(LBM_EINVAL, "width must be > 0");
    if (!(p->minority >= 0.0 && p->minority < 1.0)) return fail(LBM_EINVAL, "minority must be in [0, 1)");
    if (p->n_modes < 0 || p->n_modes > 64) return fail(LBM_EINVAL, "n_modes must be in [0, 64]");
    if (p->crop_rows < 3 || 2 * p->crop_rows >= p->ny) return fail(LBM_EINVAL, "crop_rows must be >= 3 and 2*crop_rows < ny");
    if (p->storage < LBM_STORE_F32 || p->storage > LBM_STORE_BF16) return fail(LBM_EINVAL, "unknown storage");
    if (p->kernel < LBM_KERNEL_FUSED || p->kernel > LBM_KERNEL_PAIRED) return fail(LBM_EINVAL, "unknown kernel");
    if (p->kernel == LBM_KERNEL_PAIRED && p->storage == LBM_STORE_F32)
        return fail(LBM_EINVAL, "the paired-column kernel is for 16-bit storage");
    if (p->tile_y < 0 || p->tile_y > 4096) return fail(LBM_EINVAL, "tile_y must be in [0, 4096]");
    if (p->tile_x != 0 && p->tile_x != 128 && p->tile_x != 256) return fail(LBM_EINVAL, "tile_x must be 0, 128 or 256");
    if (p->gravity_mode < 0 || p->gravity_mode > 1) return fail(LBM_EINVAL, "gravity_mode must be 0 or 1");
    if (p->wall_mode < 0 || p->wall_mode > 1) return fail(LBM_EINVAL, "wall_mode must be 0 or 1");
    if (p->x_offset < 0 || p->nx_total < 0 || (p->nx_total > 0 && (int64_t)p->x_offset + p->nx > p->nx_total) ||
        (p->nx_total == 0 && p->x_offset != 0))
        return fail(LBM_EINVAL, "x_offset and nx_total must place the grid inside a whole grid of nx_total columns");
    const double vals[] = {p->tau_A, p->tau_B, p->G, p->G_wall_A, p->G_wall_B, p->mass_A, p->mass_B,
                           p->g, p->gx, p->amp, p->width, p->minority, p->y0, p->shift_A, p->shift_B};
    for (double v : vals)
        if (!std::isfinite(v)) return fail(LBM_EINVAL, "parameters must be finite");
    return LBM_OK;
}

}  // namespace

void lbm::set_last_error(const std::string& msg) { g_last_error = msg; }

struct lbm_handle {
    lbm_params p;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    char* ws = nullptr;
    bool own_ws = false;
    Layout L;
    lbm::Grid grid;
    lbm::Physics phys;
    float shift[2];
    int cur = 0;
    int64_t step = 0;
    bool unstable = false;
    bool timed_out = false;
    bool in_ensemble = false;     // stepped by its ensemble only
    double* host_out = nullptr;   // pinned, kDiagTerms + 2 ny doubles, then the guard flag
    std::vector<double> last_rows;
    cudaEvent_t ev_diag = nullptr;      // after the last diagnostics' copies to host_out
    bool diag_pending = false;          // lbm_diagnostics_async issued, not yet collected
    // asynchronous uploads: a staging buffer filled on a copy stream (created on first use)
    cudaStream_t copy_stream = nullptr;
    float* staging = nullptr;
    cudaEvent_t ev_staged = nullptr, ev_free = nullptr;
    bool staging_used = false;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};

    void* pops(int k) { return ws + L.pops[k]; }
    double* scratch() { return (double*)(ws + L.scratch); }
    int* flag() { return (int*)(ws + L.flag); }
    int* host_flag() { return (int*)(host_out + lbm::kDiagTerms + 2 * (size_t)p.ny); }
    // the two time-step counters of the stochastic rounding (after the flag, same region)
    uint32_t* step_ctr() { return (uint32_t*)(ws + L.flag) + 2; }
    uint32_t saved_ctr[2] = {0, 0};   // counters kept with a saved state (tuning)
};

namespace {

lbm::StepLaunch step_launch(lbm_handle* h, int from) {
    lbm::StepLaunch S;
    S.fin = h->pops(from);
    S.fout = h->pops(from ^ 1);
    S.psi = (float*)(h->ws + h->L.psi);
    S.flag = h->flag();
    S.grid = h->grid;
    S.phys = h->phys;
    S.phys.step_in = h->step_ctr() + from;
    S.phys.step_out = h->step_ctr() + (from ^ 1);
    S.storage = h->p.storage;
    S.tile_x = h->p.tile_x;
    S.tile_y = h->p.tile_y;
    return S;
}

lbm::DiagLaunch diag_launch(lbm_handle* h) {
    const lbm_params& p = h->p;
    lbm::DiagLaunch D;
    D.fin = h->pops(h->cur);
    D.grid = h->grid;
    D.storage = p.storage;
    D.shift[0] = h->shift[0];
    D.shift[1] = h->shift[1];
    D.G = p.G;
    D.G_wall[0] = p.G_wall_A;
    D.G_wall[1] = p.G_wall_B;
    D.g_ext[0] = -p.g;
    D.g_ext[1] = p.gravity_mode == 0 ? p.g : -p.g;
    D.gx = p.gx;
    D.tau_bar = 0.5 * (p.tau_A + p.tau_B);
    D.crop = p.crop_rows;
    D.wall_mirror = p.wall_mode == 1 ? 1 : 0;
    D.scratch = h->scratch();
    D.partials = (double*)(h->ws + h->L.partials);
    D.out = (double*)(h->ws + h->L.out);
    return D;
}

void destroy_graphs(lbm_handle* h) {
    for (auto& g : h->graph) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

lbm_status run_init(lbm_handle* h) {
    std::vector<double> y0 = interface_height(h->p);
    double* dy0 = (double*)(h->ws + h->L.y0);
    LBM_TRY(cudaMemcpyAsync(dy0, y0.data(), y0.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy y0");
    LBM_TRY(cudaMemsetAsync(h->flag(), 0, 16, h->stream), "clear flag");
    // padding and unused window columns of both buffers start at zero
    LBM_TRY(cudaMemsetAsync(h->pops(0), 0, h->L.pop_bytes, h->stream), "clear populations");
    LBM_TRY(cudaMemsetAsync(h->pops(1), 0, h->L.pop_bytes, h->stream), "clear populations");
    LBM_TRY(lbm::launch_init(h->pops(0), h->grid, h->p.storage, h->shift, dy0, h->p.mass_A, h->p.mass_B,
                             h->p.minority, h->p.width, h->stream), "init kernel");
    // the copy reads y0 from pageable host memory: finish before the vector dies
    LBM_TRY(cudaStreamSynchronize(h->stream), "init sync");
    h->cur = 0;
    h->step = 0;
    h->unstable = false;
    h->timed_out = false;
    return LBM_OK;
}

lbm_status check_flag(lbm_handle* h) {
    int flag = 0;
    LBM_TRY(cudaMemcpyAsync(&flag, h->flag(), sizeof(int), cudaMemcpyDeviceToHost, h->stream), "read flag");
    LBM_TRY(cudaStreamSynchronize(h->stream), "sync");
    if (flag & 1) h->unstable = true;
    if (flag & 2) h->timed_out = true;
    if (h->timed_out) return fail(LBM_ETIMEOUT, "a bounded wait for a staged row copy gave up");
    return h->unstable ? fail(LBM_EUNSTABLE, "NaN or negative density seen by the step") : LBM_OK;
}

lbm_status launch_steps(lbm_handle* h, int64_t n) {
    for (int64_t k = 0; k < n; ++k) {
        LBM_TRY(lbm::launch_step(step_launch(h, h->cur), h->p.kernel, h->stream), "step kernel");
        h->cur ^= 1;
    }
    return LBM_OK;
}

lbm_status get_graph(lbm_handle* h, int parity, cudaGraphExec_t* out) {
    if (h->graph[parity]) {
        *out = h->graph[parity];
        return LBM_OK;
    }
    cudaGraph_t g = nullptr;
    LBM_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    int cur = parity;
    for (int k = 0; k < kGraphChunk; ++k) {
        cudaError_t e = lbm::launch_step(step_launch(h, cur), h->p.kernel, h->stream);
        if (e != cudaSuccess) {
            cudaStreamEndCapture(h->stream, &g);
            if (g) cudaGraphDestroy(g);
            return cuda_fail(e, "capture step");
        }
        cur ^= 1;
    }
    LBM_TRY(cudaStreamEndCapture(h->stream, &g), "end capture");
    cudaError_t e = cudaGraphInstantiate(&h->graph[parity], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "instantiate graph");
    *out = h->graph[parity];
    return LBM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// internal accessors (ensemble.cu) and the tile tuner
// ---------------------------------------------------------------------------
namespace lbm {
void* handle_buffer(lbm_handle* h, int k) { return h->pops(k); }
int handle_parity(lbm_handle* h) { return h->cur; }
Grid handle_grid(lbm_handle* h) { return h->grid; }
Physics handle_phys(lbm_handle* h) { return h->phys; }
int* handle_flag(lbm_handle* h) { return h->flag(); }
uint32_t* handle_step_counters(lbm_handle* h) { return h->step_ctr(); }
const lbm_params& handle_params(lbm_handle* h) { return h->p; }
void handle_set_ensemble(lbm_handle* h, bool on) { h->in_ensemble = on; }
void handle_advance(lbm_handle* h, int64_t n) {
    h->step += n;
    h->cur ^= (int)(n & 1);
}
lbm_status handle_check(lbm_handle* h) { return check_flag(h); }
// copy the current population buffer to the scratch region / back (state kept while tuning)
cudaError_t handle_save_state(lbm_handle* h) {
    cudaError_t e = cudaMemcpyAsync(h->saved_ctr, h->step_ctr(), sizeof(h->saved_ctr), cudaMemcpyDeviceToHost,
                                    h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(h->scratch(), h->pops(h->cur), h->L.pop_bytes, cudaMemcpyDeviceToDevice, h->stream);
}
cudaError_t handle_restore_state(lbm_handle* h) {
    cudaError_t e = cudaMemcpyAsync(h->step_ctr(), h->saved_ctr, sizeof(h->saved_ctr), cudaMemcpyHostToDevice,
                                    h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(h->pops(h->cur), h->scratch(), h->L.pop_bytes, cudaMemcpyDeviceToDevice, h->stream);
}
// rho_A, rho_B and the physical velocity on the whole grid (doubles in the scratch
// region, valid until the next call that uses the scratch)
cudaError_t handle_fields(lbm_handle* h, const double** rA, const double** rB, const double** ux, const double** uy) {
    cudaError_t e = launch_fields(diag_launch(h), nullptr, h->stream);
    const size_t n = (size_t)h->p.nx * h->p.ny;
    const double* F = h->scratch() + diag_fields_offset(h->p.nx, h->p.ny);
    *rA = F;
    *rB = F + n;
    *ux = F + 2 * n;
    *uy = F + 3 * n;
    return e;
}
cudaError_t handle_push_S(lbm_handle* h, const double* S) {
    return launch_push_from_double(S, h->grid, h->p.storage, h->shift, h->pops(h->cur), h->stream);
}
PopView handle_pops(lbm_handle* h) {
    PopView v;
    v.pops = h->pops(h->cur);
    v.grid = h->grid;
    v.storage = h->p.storage;
    v.shift[0] = h->shift[0];
    v.shift[1] = h->shift[1];
    v.stream = h->stream;
    return v;
}
cudaError_t handle_closure_features(lbm_handle* h, const float* rho2, const float* j2, const float mean[4],
                                    const float scale[4], float* x) {
    return launch_closure_features(diag_launch(h), rho2, j2, mean, scale, x, h->stream);
}
lbm_status handle_reseed(lbm_handle* h, uint64_t seed) {
    h->p.seed = seed;
    destroy_graphs(h);
    return run_init(h);
}
cudaError_t handle_clear_guard(lbm_handle* h) {
    h->unstable = false;
    h->timed_out = false;
    return cudaMemsetAsync(h->flag(), 0, sizeof(int), h->stream);
}
}  // namespace lbm

namespace {

std::string tune_key(const lbm_handle* h) {
    cudaDeviceProp prop;
    std::string dev = cudaGetDeviceProperties(&prop, h->device) == cudaSuccess ? prop.name : "unknown";
    for (char& c : dev)
        if (c == ' ') c = '_';
    return dev + "|" + std::to_string(h->p.kernel) + "|" + std::to_string(h->p.storage) + "|" +
           std::to_string(h->p.nx) + "x" + std::to_string(h->p.ny);
}

// "<key> <tile_x> <tile_y> <ms>" lines; the last match wins, lines of another form
// (or with a tile_x the library does not have) are skipped
bool cache_lookup(const char* path, const std::string& key, int* tile_x, int* tile_y, double* ms) {
    if (!path) return false;
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[1024], k[512];
    bool found = false;
    while (std::fgets(line, sizeof line, f)) {
        int tx = 0, ty = 0;
        double t = 0.0;
        if (std::sscanf(line, "%511s %d %d %lf", k, &tx, &ty, &t) != 4) continue;
        if (key != k || (tx != 0 && tx != lbm::kBlockTileW && tx != lbm::kWideTileW) || ty < 0 || ty > 4096) continue;
        *tile_x = tx;
        *tile_y = ty;
        *ms = t;
        found = true;
    }
    std::fclose(f);
    return found;
}

void cache_store(const char* path, const std::string& key, int tile_x, int tile_y, double ms) {
    if (!path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d %d %.6f\n", key.c_str(), tile_x, tile_y, ms);
    std::fclose(f);
}

}  // namespace

extern "C" lbm_status lbm_tune(lbm_handle* h, const char* cache_path, int32_t* tile_y_out, double* ms_out) {
    if (!h) return fail(LBM_EINVAL, "handle is NULL");
    if (h->in_ensemble) return fail(LBM_ESTATE, "tune the ensemble with lbm_ens_tune");
    const std::string key = tune_key(h);
    int best_tx = 0, best_ty = 0;
    double best_ms = 0.0;
    if (cache_lookup(cache_path, key, &best_tx, &best_ty, &best_ms)) {
        h->p.tile_x = best_tx;
        h->p.tile_y = best_ty;
        destroy_graphs(h);
    } else {
        const int cand[] = {0, 8, 12, 16, 24, 32, 48, 64, 96, 128};   // 0: the kernel's own default
        // tile widths: the block-staged kernel has two, and for 16-bit storage also
        // the paired-column tile (tile_x 0); the others ignore tile_x
        const int xs_staged[] = {lbm::kBlockTileW, lbm::kWideTileW, 0}, xs_other[] = {0};
        const bool staged = h->p.kernel == LBM_KERNEL_STAGED || h->p.kernel == LBM_KERNEL_DECOUPLED;
        const bool paired_too = h->p.kernel == LBM_KERNEL_STAGED && h->p.storage != LBM_STORE_F32;
        const int* xs = staged ? xs_staged : xs_other;
        const int nxs = staged ? (paired_too ? 3 : 2) : 1;
        cudaEvent_t a, b;
        LBM_TRY(cudaEventCreate(&a), "event");
        LBM_TRY(cudaEventCreate(&b), "event");
        LBM_TRY(lbm::handle_save_state(h), "save state");
        const int cur0 = h->cur;
        best_ms = 1e30;
        for (int ix = 0; ix < nxs; ++ix)
        for (int ty : cand) {
            if (ty > h->p.ny && ty != cand[0]) break;
            h->p.tile_x = xs[ix];
            h->p.tile_y = ty;
            // 30 steps per candidate: the two tile widths can differ by well under 1 %
            const int reps = 30;
            lbm_status st = launch_steps(h, 2);
            if (st == LBM_OK) {
                cudaEventRecord(a, h->stream);
                st = launch_steps(h, reps);
                cudaEventRecord(b, h->stream);
            }
            if (st != LBM_OK) {
                cudaEventDestroy(a);
                cudaEventDestroy(b);
                return st;
            }
            LBM_TRY(cudaEventSynchronize(b), "sync");
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, a, b);
            // back to the saved state
            h->cur = cur0;
            LBM_TRY(lbm::handle_restore_state(h), "restore state");
            if (ms / reps < best_ms) {
                best_ms = ms / reps;
                best_tx = xs[ix];
                best_ty = ty;
            }
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        LBM_TRY(cudaStreamSynchronize(h->stream), "sync");
        h->p.tile_x = best_tx;
        h->p.tile_y = best_ty;
        destroy_graphs(h);
        cache_store(cache_path, key, best_tx, best_ty, best_ms);
    }
    if (tile_y_out) *tile_y_out = best_ty;
    if (ms_out) *ms_out = best_ms;
    return LBM_OK;
}

extern "C" lbm_status lbm_get_params(lbm_handle* h, lbm_params* out) {
    if (!h || !out) return fail(LBM_EINVAL, "NULL argument");
    *out = h->p;
    return LBM_OK;
}

extern "C" {

const char* lbm_version(void) { return "lbm-gb300 0.1 (sm_103a)"; }

const char* lbm_status_str(lbm_status st) {
    switch (st) {
        case LBM_OK: return "ok";
        case LBM_EINVAL: return "invalid argument";
        case LBM_ENOMEM: return "out of memory";
        case LBM_ECUDA: return "CUDA error";
        case LBM_EUNSTABLE: return "unstable (NaN or negative density)";
        case LBM_ETIMEOUT: return "device wait timed out";
        case LBM_ESTATE: return "invalid state";
        case LBM_EIO: return "I/O error";
    }
    return "unknown status";
}

const char* lbm_last_error(void) { return g_last_error.c_str(); }

lbm_status lbm_params_default(lbm_params* p) {
    if (!p) return fail(LBM_EINVAL, "params is NULL");
    std::memset(p, 0, sizeof(*p));
    p->nx = 128;
    p->ny = 256;
    p->tau_A = p->tau_B = 1.0;
    p->G = 1.4;
    p->mass_A = 1.0;
    p->mass_B = 0.9;
    p->g = 1e-5;
    p->gravity_mode = 0;
    p->seed = 1;
    p->n_modes = 8;
    p->amp = 2.0;
    p->width = 1.5;
    p->minority = 0.08;
    p->y0 = -1.0;
    p->crop_rows = 10;
    p->storage = LBM_STORE_F32;
    p->kernel = LBM_KERNEL_STAGED;
    p->tile_y = 0;
    p->tile_x = 0;
    return LBM_OK;
}

lbm_status lbm_workspace_bytes(const lbm_params* p, size_t* bytes) {
    lbm_status st = validate(p);
    if (st != LBM_OK) return st;
    if (!bytes) return fail(LBM_EINVAL, "bytes is NULL");
    *bytes = make_layout(*p).total;
    return LBM_OK;
}

lbm_status lbm_create_ex(const lbm_params* p, void* dev_workspace, size_t ws_bytes, void* cuda_stream,
                         lbm_handle** out) {
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    lbm_status st = validate(p);
    if (st != LBM_OK) return st;
    Layout L = make_layout(*p);
    if (dev_workspace && ws_bytes < L.total) return fail(LBM_ENOMEM, "workspace smaller than lbm_workspace_bytes");
    if (dev_workspace && ((uintptr_t)dev_workspace % kAlign) != 0) return fail(LBM_EINVAL, "workspace must be 256-byte aligned");
    lbm_handle* h = new lbm_handle();
    h->p = *p;
    h->L = L;
    cudaGetDevice(&h->device);
    if (dev_workspace) {
        h->ws = (char*)dev_workspace;
    } else {
        cudaError_t e = cudaMalloc((void**)&h->ws, L.total);
        if (e != cudaSuccess) {
            delete h;
            cudaGetLastError();
            return fail(LBM_ENOMEM, std::string("cudaMalloc workspace: ") + cudaGetErrorString(e));
        }
        h->own_ws = true;
    }
    if (cuda_stream) {
        h->stream = (cudaStream_t)cuda_stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            lbm_destroy(h);
            return cuda_fail(e, "create stream");
        }
        h->own_stream = true;
    }
    cudaError_t e = cudaMallocHost((void**)&h->host_out, (lbm::kDiagTerms + 2 * (size_t)p->ny + 1) * sizeof(double));
    if (e != cudaSuccess) {
        h->host_out = nullptr;
        lbm_destroy(h);
        return cuda_fail(e, "pinned host buffer");
    }
    // work queued on other streams (e.g. whoever produced the workspace) is done
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        lbm_destroy(h);
        return cuda_fail(e, "synchronize");
    }
    h->grid.nx = p->nx;
    h->grid.ny = p->ny;
    h->grid.pitch = L.pitch;
    h->grid.origin = L.origin;
    h->grid.plane = L.plane;
    h->grid.x_offset = p->x_offset;
    h->grid.nx_total = p->nx_total;
    const bool shifted = p->storage != LBM_STORE_F32;
    const double sA = p->shift_A > 0.0 ? p->shift_A : 0.5 * p->mass_A * (1.0 + p->minority);
    const double sB = p->shift_B > 0.0 ? p->shift_B : 0.5 * p->mass_B * (1.0 + p->minority);
    h->shift[0] = shifted ? (float)sA : 0.0f;
    h->shift[1] = shifted ? (float)sB : 0.0f;
    lbm::Physics& ph = h->phys;
    ph.tau[0] = (float)p->tau_A;
    ph.tau[1] = (float)p->tau_B;
    ph.om[0] = (float)(1.0 / p->tau_A);
    ph.om[1] = (float)(1.0 / p->tau_B);
    ph.G = (float)p->G;
    // wall force: sum_i w_i S(x + c_i) c_i = (0, -1/6) on row 0 and (0, +1/6) on row ny-1
    ph.ay_wall_bottom[0] = (float)(p->G_wall_A / 6.0);
    ph.ay_wall_bottom[1] = (float)(p->G_wall_B / 6.0);
    ph.ay_wall_top[0] = (float)(-p->G_wall_A / 6.0);
    ph.ay_wall_top[1] = (float)(-p->G_wall_B / 6.0);
    ph.ay_ext[0] = (float)(-p->g);
    ph.ay_ext[1] = (float)(p->gravity_mode == 0 ? p->g : -p->g);
    ph.ax_ext = (float)p->gx;
    ph.wall_mirror = p->wall_mode == 1 ? 1 : 0;
    ph.shift[0] = h->shift[0];
    ph.shift[1] = h->shift[1];
    // The instability guard rejects densities below -5 % of rho0_s = mass_s (1 + minority)
    // / 2, and non-finite ones.  Zero is not the floor: near tau = 1/2 the over-relaxed
    // BGK update sends the density of a component that is nearly absent at a site below
    // zero for a while (the minority component in the thin filaments of the paper's
    // turbulent mixing layer at tau = 0.53, measured on the 10000 x 5000 grid after
    // ~29 000 steps; an absent component a few rounding units below zero near a front;
    // the 16-bit storage's rounding noise around zero), without any blow-up, which
    // grows past any such floor within a few steps or turns a density non-finite.
    const float floor_frac = 0.05f;
    ph.rho_floor[0] = (float)(-floor_frac * sA);
    ph.rho_floor[1] = (float)(-floor_frac * sB);
    ph.step_in = nullptr;    // set per launch (step_launch)
    ph.step_out = nullptr;
    st = run_init(h);
    if (st != LBM_OK) {
        std::string msg = g_last_error;
        lbm_destroy(h);
        return fail(st, msg);
    }
    *out = h;
    return LBM_OK;
}

lbm_status lbm_create(int32_t nx, int32_t ny, double tau, double G, double mass_A, double mass_B, double g,
                      uint64_t seed, lbm_handle** out) {
    lbm_params p;
    lbm_params_default(&p);
    p.nx = nx;
    p.ny = ny;
    p.tau_A = p.tau_B = tau;
    p.G = G;
    p.mass_A = mass_A;
    p.mass_B = mass_B;
    p.g = g;
    p.seed = seed;
    return lbm_create_ex(&p, nullptr, 0, nullptr, out);
}

lbm_status lbm_reset(lbm_handle* h) {
    if (!h) return fail(LBM_EINVAL, "handle is NULL");
    return run_init(h);
}

lbm_status lbm_step(lbm_handle* h, int64_t nsteps) {
    if (!h) return fail(LBM_EINVAL, "handle is NULL");
    if (nsteps < 0) return fail(LBM_EINVAL, "nsteps must be >= 0");
    if (h->in_ensemble) return fail(LBM_ESTATE, "this handle is an ensemble member: step it with lbm_ens_step");
    if (h->timed_out) return fail(LBM_ETIMEOUT, "an earlier step timed out");
    if (h->unstable) return fail(LBM_EUNSTABLE, "state is unstable");
    int64_t left = nsteps;
    while (left >= kGraphChunk) {
        cudaGraphExec_t g = nullptr;
        lbm_status st = get_graph(h, h->cur, &g);
        if (st != LBM_OK) return st;
        LBM_TRY(cudaGraphLaunch(g, h->stream), "graph launch");
        h->cur ^= (kGraphChunk & 1);
        h->step += kGraphChunk;
        left -= kGraphChunk;
    }
    lbm_status st = launch_steps(h, left);
    if (st != LBM_OK) return st;
    h->step += left;
    return LBM_OK;
}

lbm_status lbm_sync(lbm_handle* h) {
    if (!h) return fail(LBM_EINVAL, "handle is NULL");
    return check_flag(h);
}

lbm_status lbm_step_test_timeout(lbm_handle* h) {
    if (!h) return fail(LBM_EINVAL, "handle is NULL");
    if (h->in_ensemble) return fail(LBM_ESTATE, "ensemble members are stepped by their ensemble");
    if (h->p.storage != LBM_STORE_F32) return fail(LBM_EINVAL, "the timeout test runs on FP32 storage");
    LBM_TRY(lbm::launch_step_test_timeout(step_launch(h, h->cur), h->stream), "timeout test kernel");
    return LBM_OK;
}

lbm_status lbm_step_count(lbm_handle* h, int64_t* step) {
    if (!h || !step) return fail(LBM_EINVAL, "NULL argument");
    *step = h->step;
    return LBM_OK;
}

}  // extern "C"

namespace {

// The diagnostics kernels, their results and the guard flag copied to the pinned
// host buffer, and an event after them; nothing waits.
lbm_status diag_issue(lbm_handle* h) {
    const lbm_params& p = h->p;
    lbm::DiagLaunch D = diag_launch(h);
    LBM_TRY(lbm::launch_diagnostics(D, h->stream), "diagnostics kernels");
    const int nrows = p.ny - 2 * p.crop_rows;
    LBM_TRY(cudaMemcpyAsync(h->host_out, D.out, (lbm::kDiagTerms + 2 * (size_t)nrows) * sizeof(double),
                            cudaMemcpyDeviceToHost, h->stream), "copy diagnostics");
    LBM_TRY(cudaMemcpyAsync(h->host_flag(), h->flag(), sizeof(int), cudaMemcpyDeviceToHost, h->stream), "read flag");
    if (!h->ev_diag) LBM_TRY(cudaEventCreateWithFlags(&h->ev_diag, cudaEventDisableTiming), "diagnostics event");
    LBM_TRY(cudaEventRecord(h->ev_diag, h->stream), "record diagnostics event");
    return LBM_OK;
}

// Waits for the event of diag_issue (not for later work on the stream) and fills *out.
lbm_status diag_collect(lbm_handle* h, lbm_diag* out) {
    LBM_TRY(cudaEventSynchronize(h->ev_diag), "wait for diagnostics");
    const int flag = *h->host_flag();
    if (flag & 1) h->unstable = true;
    if (flag & 2) h->timed_out = true;
    if (h->timed_out) return fail(LBM_ETIMEOUT, "a bounded wait for a staged row copy gave up");
    const lbm_status st = h->unstable ? fail(LBM_EUNSTABLE, "NaN or negative density seen by the step") : LBM_OK;
    const lbm_params& p = h->p;
    const int nrows = p.ny - 2 * p.crop_rows;
    const double* o = h->host_out;
    const double Dn = (double)p.nx * nrows;
    const double cs2 = 1.0 / 3.0;
    const double tau_bar = 0.5 * (p.tau_A + p.tau_B);
    std::memset(out, 0, sizeof(*out));
    out->step = h->step;
    out->mass_A = o[lbm::T_MASS_A];
    out->mass_B = o[lbm::T_MASS_B];
    out->E_k = o[lbm::T_EK] / Dn;
    out->E_p = p.g * o[lbm::T_EP] / Dn;
    out->buoyancy = p.g * o[lbm::T_BUOY] / Dn;
    out->flux_pb = o[lbm::T_FLUX_PB] / Dn;
    out->flux_K = o[lbm::T_FLUX_K] / Dn;
    out->flux_tau = o[lbm::T_FLUX_TAU] / Dn;
    out->rho_bar = o[lbm::T_RHO] / Dn;
    const double eta = out->rho_bar * cs2 * (tau_bar - 0.5);
    out->viscous = eta * o[lbm::T_VISC] / Dn;
    out->enstrophy = 0.5 * o[lbm::T_OMEGA2];
    for (int k = 0; k < 4; ++k) out->cc[k] = (int64_t)std::llround(o[lbm::T_N0 + k]);
    out->L_int = (M_PI / 8.0) * ((double)out->cc[0] + (double)out->cc[1] +
                                 ((double)out->cc[2] + (double)out->cc[3]) / std::sqrt(2.0));
    // row means of phi (the profile) and the mixing-layer width from the normalised
    // row means of the mass fraction rho_A / (rho_A + rho_B)
    const double eps = p.minority;
    const double top = p.mass_A / (p.mass_A + eps * p.mass_B);
    const double bot = eps * p.mass_A / (eps * p.mass_A + p.mass_B);
    h->last_rows.assign(nrows, 0.0);
    double hw = 0.0;
    for (int r = 0; r < nrows; ++r) {
        h->last_rows[r] = o[lbm::kDiagTerms + r] / p.nx;
        double c = (o[lbm::kDiagTerms + nrows + r] / p.nx - bot) / (top - bot);
        c = c < 0.0 ? 0.0 : (c > 1.0 ? 1.0 : c);
        hw += c * (1.0 - c);
    }
    out->h = 6.0 * hw;
    out->status = h->unstable ? LBM_EUNSTABLE : LBM_OK;
    return st;
}

}  // namespace

extern "C" {

lbm_status lbm_diagnostics(lbm_handle* h, lbm_diag* out) {
    if (!h || !out) return fail(LBM_EINVAL, "NULL argument");
    if (h->diag_pending) return fail(LBM_ESTATE, "collect the pending lbm_diagnostics_async first");
    lbm_status st = diag_issue(h);
    if (st != LBM_OK) return st;
    return diag_collect(h, out);
}

lbm_status lbm_diagnostics_async(lbm_handle* h) {
    if (!h) return fail(LBM_EINVAL, "handle is NULL");
    if (h->diag_pending) return fail(LBM_ESTATE, "collect the pending lbm_diagnostics_async first");
    lbm_status st = diag_issue(h);
    if (st == LBM_OK) h->diag_pending = true;
    return st;
}

lbm_status lbm_diagnostics_wait(lbm_handle* h, lbm_diag* out) {
    if (!h || !out) return fail(LBM_EINVAL, "NULL argument");
    if (!h->diag_pending) return fail(LBM_ESTATE, "no lbm_diagnostics_async pending");
    h->diag_pending = false;
    return diag_collect(h, out);
}

lbm_status lbm_profile(lbm_handle* h, double* host_rows) {
    if (!h || !host_rows) return fail(LBM_EINVAL, "NULL argument");
    if (h->last_rows.empty()) return fail(LBM_ESTATE, "no diagnostics computed yet");
    std::memcpy(host_rows, h->last_rows.data(), h->last_rows.size() * sizeof(double));
    return LBM_OK;
}

lbm_status lbm_get_fields(lbm_handle* h, double* rhoA, double* rhoB, double* ux, double* uy) {
    if (!h) return fail(LBM_EINVAL, "handle is NULL");
    lbm::DiagLaunch D = diag_launch(h);
    LBM_TRY(lbm::launch_fields(D, nullptr, h->stream), "fields kernels");
    const size_t n = (size_t)h->p.nx * h->p.ny;
    const double* F = h->scratch() + lbm::diag_fields_offset(h->p.nx, h->p.ny);
    double* dst[4] = {rhoA, rhoB, ux, uy};
    for (int k = 0; k < 4; ++k)
        if (dst[k])
            LBM_TRY(cudaMemcpyAsync(dst[k], F + k * n, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
                    "copy fields");
    LBM_TRY(cudaStreamSynchronize(h->stream), "sync");
    return LBM_OK;
}

lbm_status lbm_get_populations(lbm_handle* h, double* host) {
    if (!h || !host) return fail(LBM_EINVAL, "NULL argument");
    double* S = h->scratch();
    LBM_TRY(lbm::launch_pull_to_double(h->pops(h->cur), h->grid, h->p.storage, h->shift, S, h->stream), "pull kernel");
    const size_t n = (size_t)18 * h->p.nx * h->p.ny;
    LBM_TRY(cudaMemcpyAsync(host, S, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy populations");
    LBM_TRY(cudaStreamSynchronize(h->stream), "sync");
    return LBM_OK;
}

lbm_status lbm_set_populations(lbm_handle* h, const double* host) {
    if (!h || !host) return fail(LBM_EINVAL, "NULL argument");
    double* S = h->scratch();
    const size_t n = (size_t)18 * h->p.nx * h->p.ny;
    LBM_TRY(cudaMemcpyAsync(S, host, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy populations");
    LBM_TRY(lbm::launch_push_from_double(S, h->grid, h->p.storage, h->shift, h->pops(h->cur), h->stream), "push kernel");
    LBM_TRY(cudaStreamSynchronize(h->stream), "sync");
    return LBM_OK;
}

lbm_status lbm_get_populations_f32(lbm_handle* h, float* host) {
    if (!h || !host) return fail(LBM_EINVAL, "NULL argument");
    float* S = reinterpret_cast<float*>(h->scratch());
    LBM_TRY(lbm::launch_pull_to_float(h->pops(h->cur), h->grid, h->p.storage, h->shift, S, h->stream), "pull kernel");
    const size_t n = (size_t)18 * h->p.nx * h->p.ny;
    LBM_TRY(cudaMemcpyAsync(host, S, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream), "copy populations");
    LBM_TRY(cudaStreamSynchronize(h->stream), "sync");
    return LBM_OK;
}

lbm_status lbm_set_populations_f32_async(lbm_handle* h, const float* host) {
    if (!h || !host) return fail(LBM_EINVAL, "NULL argument");
    const size_t n = (size_t)18 * h->p.nx * h->p.ny;
    if (!h->staging) {
        LBM_TRY(cudaSetDevice(h->device), "set device");
        if (cudaMalloc((void**)&h->staging, n * sizeof(float)) != cudaSuccess) {
            (void)cudaGetLastError();
            h->staging = nullptr;
            return fail(LBM_ENOMEM, "staging buffer of the asynchronous upload");
        }
        LBM_TRY(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking), "copy stream");
        LBM_TRY(cudaEventCreateWithFlags(&h->ev_staged, cudaEventDisableTiming), "upload event");
        LBM_TRY(cudaEventCreateWithFlags(&h->ev_free, cudaEventDisableTiming), "upload event");
    }
    // the previous upload's push has read the staging buffer before it is refilled
    if (h->staging_used) LBM_TRY(cudaStreamWaitEvent(h->copy_stream, h->ev_free, 0), "wait for staging");
    LBM_TRY(cudaMemcpyAsync(h->staging, host, n * sizeof(float), cudaMemcpyHostToDevice, h->copy_stream),
            "copy populations");
    LBM_TRY(cudaEventRecord(h->ev_staged, h->copy_stream), "record upload");
    LBM_TRY(cudaStreamWaitEvent(h->stream, h->ev_staged, 0), "order upload");
    LBM_TRY(lbm::launch_push_from_float(h->staging, h->grid, h->p.storage, h->shift, h->pops(h->cur), h->stream),
            "push kernel");
    LBM_TRY(cudaEventRecord(h->ev_free, h->stream), "record push");
    h->staging_used = true;
    return LBM_OK;
}

lbm_status lbm_set_populations_f32(lbm_handle* h, const float* host) {
    if (!h || !host) return fail(LBM_EINVAL, "NULL argument");
    float* S = reinterpret_cast<float*>(h->scratch());
    const size_t n = (size_t)18 * h->p.nx * h->p.ny;
    LBM_TRY(cudaMemcpyAsync(S, host, n * sizeof(float), cudaMemcpyHostToDevice, h->stream), "copy populations");
    LBM_TRY(lbm::launch_push_from_float(S, h->grid, h->p.storage, h->shift, h->pops(h->cur), h->stream), "push kernel");
    LBM_TRY(cudaStreamSynchronize(h->stream), "sync");
    return LBM_OK;
}

struct SaveHeader {
    char magic[8];
    int32_t version, nx, ny, storage, pitch, cur;
    int64_t step;
    uint64_t bytes;
    lbm_params params;
};

lbm_status lbm_save(lbm_handle* h, const char* path) {
    if (!h || !path) return fail(LBM_EINVAL, "NULL argument");
    std::vector<char> buf(h->L.pop_bytes);
    LBM_TRY(cudaMemcpyAsync(buf.data(), h->pops(h->cur), buf.size(), cudaMemcpyDeviceToHost, h->stream), "copy state");
    LBM_TRY(cudaStreamSynchronize(h->stream), "sync");
    SaveHeader hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, "LBMSTAT1", 8);
    hd.version = 1;
    hd.nx = h->p.nx;
    hd.ny = h->p.ny;
    hd.storage = h->p.storage;
    hd.pitch = h->L.pitch;
    hd.step = h->step;
    hd.bytes = buf.size();
    hd.params = h->p;
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(LBM_EIO, std::string("cannot open ") + path);
    const bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1 && std::fwrite(buf.data(), 1, buf.size(), f) == buf.size();
    const bool closed = std::fclose(f) == 0;
    if (!ok || !closed) return fail(LBM_EIO, std::string("write failed: ") + path);
    return LBM_OK;
}

lbm_status lbm_load(lbm_handle* h, const char* path) {
    if (!h || !path) return fail(LBM_EINVAL, "NULL argument");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(LBM_EIO, std::string("cannot open ") + path);
    SaveHeader hd;
    if (std::fread(&hd, sizeof(hd), 1, f) != 1 || std::memcmp(hd.magic, "LBMSTAT1", 8) != 0) {
        std::fclose(f);
        return fail(LBM_EIO, "not a state file");
    }
    if (hd.nx != h->p.nx || hd.ny != h->p.ny || hd.storage != h->p.storage || hd.pitch != h->L.pitch ||
        hd.bytes != h->L.pop_bytes) {
        std::fclose(f);
        return fail(LBM_EINVAL, "state file does not match the handle (nx, ny, storage)");
    }
    std::vector<char> buf(hd.bytes);
    const bool ok = std::fread(buf.data(), 1, buf.size(), f) == buf.size();
    std::fclose(f);
    if (!ok) return fail(LBM_EIO, "truncated state file");
    LBM_TRY(cudaMemcpyAsync(h->pops(h->cur), buf.data(), buf.size(), cudaMemcpyHostToDevice, h->stream), "copy state");
    // the rounding counter continues from the saved step, as in the run that saved it
    h->saved_ctr[0] = h->saved_ctr[1] = (uint32_t)hd.step;
    LBM_TRY(cudaMemcpyAsync(h->step_ctr(), h->saved_ctr, sizeof(h->saved_ctr), cudaMemcpyHostToDevice, h->stream),
            "set step counter");
    LBM_TRY(cudaStreamSynchronize(h->stream), "sync");
    h->step = hd.step;
    return LBM_OK;
}

void lbm_destroy(lbm_handle* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    destroy_graphs(h);
    if (h->copy_stream) cudaStreamSynchronize(h->copy_stream);
    if (h->host_out) cudaFreeHost(h->host_out);
    if (h->ev_diag) cudaEventDestroy(h->ev_diag);
    if (h->ev_staged) cudaEventDestroy(h->ev_staged);
    if (h->ev_free) cudaEventDestroy(h->ev_free);
    if (h->staging) cudaFree(h->staging);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    if (h->own_ws && h->ws) cudaFree(h->ws);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

}  // extern "C"
