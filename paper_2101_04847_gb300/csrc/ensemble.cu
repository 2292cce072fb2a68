// Ensembles of independent realisations (the paper runs at least 10 per
// experiment, Section 2): one kernel launch per time step advances every member
// (ensemble_step_kernel, step_kernels.cu: the block-staged tile code over a flat
// list of every member's tiles), and chunks of steps are captured in CUDA graphs.  Members may differ in grid size, physics and storage type; each
// member is a full lbm_handle (init, diagnostics, fields, checkpoints) that only
// the ensemble steps.
#include "lbm_internal.cuh"

#include <algorithm>
#include <string>
#include <vector>

namespace {

constexpr int kEnsGraphChunk = 50;
constexpr int kEnsMaxMembers = 256;

lbm_status ens_fail(lbm_status st, const std::string& msg) {
    lbm::set_last_error(msg);
    return st;
}

#define ENS_TRY(call, what)                                                                       \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return ens_fail(LBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

struct lbm_ensemble {
    std::vector<lbm_handle*> members;
    std::vector<lbm::EnsMember> table;
    lbm::EnsMember* d_table = nullptr;
    int total_tiles = 0;
    int tile_x = lbm::kEnsPaired;    // 128 or 256 columns per tile (one per thread), or
                                     // kEnsPaired (FP32 128 columns, 16-bit paired 256)
    int tile_y = 0;       // requested rows per tile; 0: chosen from the device's block slots
    int rows = 0;         // rows per tile in use
    size_t smem = 0;      // dynamic shared memory per block (largest storage type present)
    int parity = 0;
    int64_t step = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
};

namespace {

void ens_drop_graphs(lbm_ensemble* e) {
    for (auto& g : e->graph) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

int tiles_of(const lbm::Grid& g, int tile_x, int rows, int* tx, int* ty) {
    *tx = (g.nx + tile_x - 1) / tile_x;
    *ty = std::min(g.ny, std::max(1, (g.ny + rows - 1) / rows));
    return *tx * *ty;
}

// Rows per tile when none is requested: the height whose tile count fills the
// resident block slots in whole waves best, weighted by the share of rows that
// are not halo (3 halo rows per tile).
int auto_rows(const lbm_ensemble* e, int slots) {
    int best = 32;
    double best_score = -1.0;
    for (int rows = 12; rows <= 256; ++rows) {
        long long tiles = 0;
        for (lbm_handle* h : e->members) {
            int tx, ty;
            tiles += tiles_of(lbm::handle_grid(h), lbm::ensemble_tile_cols(lbm::handle_params(h).storage, e->tile_x),
                              rows, &tx, &ty);
        }
        const long long waves = (tiles + slots - 1) / slots;
        const double score = (double)tiles / (double)(waves * slots) * rows / (rows + 3.0);
        if (score > best_score + 1e-9) {
            best_score = score;
            best = rows;
        }
    }
    return best;
}

// (Re)build the member table for the current tile height and upload it.
lbm_status ens_build_table(lbm_ensemble* e) {
    e->table.clear();
    e->smem = 0;
    for (lbm_handle* h : e->members)
        e->smem = std::max(e->smem, lbm::block_tile_smem_bytes(lbm::handle_params(h).storage, e->tile_x));
    if (e->tile_y > 0) {
        e->rows = e->tile_y;
    } else {
        cudaError_t err = cudaSuccess;
        const int slots = lbm::ensemble_slots(e->smem, e->tile_x, &err);
        ENS_TRY(err, "ensemble occupancy");
        e->rows = auto_rows(e, slots);
    }
    // Tiles of one storage type are contiguous in the flat list, so that the blocks
    // resident at one time mostly run one instantiation of the tile code (mixing
    // them on an SM thrashes its instruction cache).
    std::vector<lbm_handle*> order;
    for (int st : {LBM_STORE_F32, LBM_STORE_F16, LBM_STORE_BF16})
        for (lbm_handle* h : e->members)
            if (lbm::handle_params(h).storage == st) order.push_back(h);
    int begin = 0;
    for (lbm_handle* h : order) {
        lbm::EnsMember m;
        m.grid = lbm::handle_grid(h);
        m.phys = lbm::handle_phys(h);
        m.buf[0] = lbm::handle_buffer(h, 0);
        m.buf[1] = lbm::handle_buffer(h, 1);
        m.flag = lbm::handle_flag(h);
        m.storage = lbm::handle_params(h).storage;
        m.step_ctr = lbm::handle_step_counters(h);
        const int tiles = tiles_of(m.grid, lbm::ensemble_tile_cols(m.storage, e->tile_x), e->rows, &m.tiles_x,
                                   &m.tiles_y);
        m.tile_begin = begin;
        begin += tiles;
        e->table.push_back(m);
    }
    e->total_tiles = begin;
    ENS_TRY(cudaMemcpyAsync(e->d_table, e->table.data(), e->table.size() * sizeof(lbm::EnsMember),
                            cudaMemcpyHostToDevice, e->stream), "upload member table");
    ENS_TRY(cudaStreamSynchronize(e->stream), "sync");
    ens_drop_graphs(e);
    return LBM_OK;
}

lbm_status ens_launch(lbm_ensemble* e, int64_t n) {
    for (int64_t k = 0; k < n; ++k) {
        ENS_TRY(lbm::launch_ensemble_step(e->d_table, (int)e->members.size(), e->total_tiles, e->parity, e->smem,
                                          e->tile_x, e->stream),
                "ensemble step");
        e->parity ^= 1;
    }
    return LBM_OK;
}

lbm_status ens_graph(lbm_ensemble* e, cudaGraphExec_t* out) {
    const int par = e->parity;
    if (!e->graph[par]) {
        cudaGraph_t g = nullptr;
        ENS_TRY(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        for (int k = 0; k < kEnsGraphChunk; ++k) {
            cudaError_t err = lbm::launch_ensemble_step(e->d_table, (int)e->members.size(), e->total_tiles,
                                                        (par + k) & 1, e->smem, e->tile_x, e->stream);
            if (err != cudaSuccess) {
                cudaStreamEndCapture(e->stream, &g);
                if (g) cudaGraphDestroy(g);
                return ens_fail(LBM_ECUDA, std::string("capture ensemble step: ") + cudaGetErrorString(err));
            }
        }
        ENS_TRY(cudaStreamEndCapture(e->stream, &g), "end capture");
        cudaError_t err = cudaGraphInstantiate(&e->graph[par], g, 0);
        cudaGraphDestroy(g);
        if (err != cudaSuccess) return ens_fail(LBM_ECUDA, std::string("instantiate: ") + cudaGetErrorString(err));
    }
    *out = e->graph[par];
    return LBM_OK;
}

}  // namespace

extern "C" {

void lbm_ens_destroy(lbm_ensemble* e) {
    if (!e) return;
    if (e->stream) cudaStreamSynchronize(e->stream);
    ens_drop_graphs(e);
    for (lbm_handle* h : e->members) {
        lbm::handle_set_ensemble(h, false);
        lbm_destroy(h);
    }
    if (e->d_table) cudaFree(e->d_table);
    if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
    delete e;
}

lbm_status lbm_ens_create(int32_t n, const lbm_params* params, void* cuda_stream, lbm_ensemble** out) {
    if (!out) return ens_fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!params || n < 1 || n > kEnsMaxMembers) return ens_fail(LBM_EINVAL, "need 1..256 member parameter sets");
    lbm_ensemble* e = new lbm_ensemble();
    if (cuda_stream) {
        e->stream = (cudaStream_t)cuda_stream;
    } else {
        cudaError_t err = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking);
        if (err != cudaSuccess) {
            delete e;
            return ens_fail(LBM_ECUDA, std::string("create stream: ") + cudaGetErrorString(err));
        }
        e->own_stream = true;
    }
    e->tile_y = params[0].tile_y > 0 ? params[0].tile_y : 0;
    e->tile_x = params[0].tile_x == lbm::kWideTileW || params[0].tile_x == lbm::kBlockTileW ? params[0].tile_x
                                                                                             : lbm::kEnsPaired;
    for (int i = 0; i < n; ++i) {
        lbm_params p = params[i];
        p.kernel = LBM_KERNEL_STAGED;
        lbm_handle* h = nullptr;
        lbm_status st = lbm_create_ex(&p, nullptr, 0, e->stream, &h);
        if (st != LBM_OK) {
            const std::string msg = std::string("member ") + std::to_string(i) + ": " + lbm_last_error();
            lbm_ens_destroy(e);
            return ens_fail(st, msg);
        }
        lbm::handle_set_ensemble(h, true);
        e->members.push_back(h);
    }
    cudaError_t err = cudaMalloc((void**)&e->d_table, (size_t)n * sizeof(lbm::EnsMember));
    if (err != cudaSuccess) {
        e->d_table = nullptr;
        lbm_ens_destroy(e);
        return ens_fail(LBM_ENOMEM, "member table");
    }
    lbm_status st = ens_build_table(e);
    if (st != LBM_OK) {
        const std::string msg = lbm_last_error();
        lbm_ens_destroy(e);
        return ens_fail(st, msg);
    }
    *out = e;
    return LBM_OK;
}

lbm_status lbm_ens_step(lbm_ensemble* e, int64_t nsteps) {
    if (!e) return ens_fail(LBM_EINVAL, "ensemble is NULL");
    if (nsteps < 0) return ens_fail(LBM_EINVAL, "nsteps must be >= 0");
    int64_t left = nsteps;
    while (left >= kEnsGraphChunk) {
        cudaGraphExec_t g = nullptr;
        lbm_status st = ens_graph(e, &g);
        if (st != LBM_OK) return st;
        ENS_TRY(cudaGraphLaunch(g, e->stream), "graph launch");
        e->parity ^= (kEnsGraphChunk & 1);
        left -= kEnsGraphChunk;
    }
    lbm_status st = ens_launch(e, left);
    if (st != LBM_OK) return st;
    e->step += nsteps;
    for (lbm_handle* h : e->members) lbm::handle_advance(h, nsteps);
    return LBM_OK;
}

lbm_status lbm_ens_sync(lbm_ensemble* e) {
    if (!e) return ens_fail(LBM_EINVAL, "ensemble is NULL");
    lbm_status worst = LBM_OK;
    for (lbm_handle* h : e->members) {
        lbm_status st = lbm::handle_check(h);
        if (st != LBM_OK && worst == LBM_OK) worst = st;
    }
    return worst;
}

lbm_status lbm_ens_member(lbm_ensemble* e, int32_t i, lbm_handle** out) {
    if (!e || !out) return ens_fail(LBM_EINVAL, "NULL argument");
    if (i < 0 || i >= (int)e->members.size()) return ens_fail(LBM_EINVAL, "member index out of range");
    *out = e->members[i];
    return LBM_OK;
}

lbm_status lbm_ens_diagnostics(lbm_ensemble* e, lbm_diag* out) {
    if (!e || !out) return ens_fail(LBM_EINVAL, "NULL argument");
    lbm_status worst = LBM_OK;
    for (size_t i = 0; i < e->members.size(); ++i) {
        lbm_status st = lbm_diagnostics(e->members[i], &out[i]);
        if (st != LBM_OK && worst == LBM_OK) worst = st;
    }
    return worst;
}

lbm_status lbm_ens_tune(lbm_ensemble* e, int32_t* tile_y_out, double* ms_out) {
    if (!e) return ens_fail(LBM_EINVAL, "ensemble is NULL");
    const int cand[] = {0, 12, 16, 20, 24, 32, 48, 64, 96};   // 0: the slot-filling default
    const int widths[] = {lbm::kEnsPaired, lbm::kBlockTileW, lbm::kWideTileW};
    cudaEvent_t a, b;
    ENS_TRY(cudaEventCreate(&a), "event");
    ENS_TRY(cudaEventCreate(&b), "event");
    for (lbm_handle* h : e->members) ENS_TRY(lbm::handle_save_state(h), "save state");
    const int par0 = e->parity;
    double best_ms = 1e30;
    int best_ty = e->tile_y, best_tx = e->tile_x;
    for (int tx : widths)
    for (int ty : cand) {
        e->tile_x = tx;
        e->tile_y = ty;
        lbm_status st = ens_build_table(e);
        const int reps = 6;
        if (st == LBM_OK) st = ens_launch(e, 2);
        if (st == LBM_OK) {
            cudaEventRecord(a, e->stream);
            st = ens_launch(e, reps);
            cudaEventRecord(b, e->stream);
        }
        if (st != LBM_OK) {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            return st;
        }
        ENS_TRY(cudaEventSynchronize(b), "sync");
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        e->parity = par0;   // 8 steps: back on the same buffer; restore its contents
        for (lbm_handle* h : e->members) ENS_TRY(lbm::handle_restore_state(h), "restore state");
        if (ms / reps < best_ms) {
            best_ms = ms / reps;
            best_ty = ty;
            best_tx = tx;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    e->tile_x = best_tx;
    e->tile_y = best_ty;
    lbm_status st = ens_build_table(e);
    if (st != LBM_OK) return st;
    if (tile_y_out) *tile_y_out = e->rows;
    if (ms_out) *ms_out = best_ms;
    return LBM_OK;
}

lbm_status lbm_ens_tile_width(lbm_ensemble* e, int32_t* tile_x) {
    if (!e || !tile_x) return ens_fail(LBM_EINVAL, "NULL argument");
    *tile_x = e->tile_x;
    return LBM_OK;
}

}  // extern "C"
