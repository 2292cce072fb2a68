// Halo exchange of a grid split along x over several solvers (domain decomposition):
// the step kernels that stage row windows (block-staged, decoupled) read the stored
// populations of the two columns beside the grid from ghost columns -2, -1, nx and
// nx + 1.  An undivided grid fills them with its own periodic copies; a sub-grid
// takes them from its neighbours: its left ghosts are the left neighbour's last two
// columns, its right ghosts the right neighbour's first two.  These kernels copy the
// two edge columns of the current buffer into a contiguous buffer and back into the
// ghost columns, so that any transport (a device copy, NCCL, a host round trip) can
// carry them.  The pull of Section 2 (S_i(x) = B_i(x - c_i)) then reads across the
// seam exactly as inside one grid.
#include "lbm_internal.cuh"

#include <string>

namespace lbm {
namespace {

// buf layout: [plane 18][row ny][column 2], element type of the storage
template <typename T>
__global__ void halo_pack_kernel(const T* __restrict__ pops, Grid g, int col0, T* __restrict__ buf) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = 36 * g.ny;
    if (idx >= n) return;
    const int c = idx & 1, r = (idx >> 1) % g.ny, pl = (idx >> 1) / g.ny;
    buf[idx] = pops[(size_t)pl * g.plane + (size_t)r * g.pitch + g.origin + col0 + c];
}

template <typename T>
__global__ void halo_unpack_kernel(T* __restrict__ pops, Grid g, int col0, const T* __restrict__ buf) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = 36 * g.ny;
    if (idx >= n) return;
    const int c = idx & 1, r = (idx >> 1) % g.ny, pl = (idx >> 1) / g.ny;
    pops[(size_t)pl * g.plane + (size_t)r * g.pitch + g.origin + col0 + c] = buf[idx];
}

size_t elem_bytes(int storage) { return storage == LBM_STORE_F32 ? 4 : 2; }

template <typename T>
cudaError_t launch_halo(const PopView& v, int side, void* buf, bool pack) {
    const int n = 36 * v.grid.ny;
    const int threads = 256, blocks = (n + threads - 1) / threads;
    if (pack) {
        const int col0 = side == 0 ? 0 : v.grid.nx - 2;
        halo_pack_kernel<T><<<blocks, threads, 0, v.stream>>>((const T*)v.pops, v.grid, col0, (T*)buf);
    } else {
        const int col0 = side == 0 ? -2 : v.grid.nx;
        halo_unpack_kernel<T><<<blocks, threads, 0, v.stream>>>((T*)v.pops, v.grid, col0, (const T*)buf);
    }
    return cudaGetLastError();
}

lbm_status halo_call(lbm_handle* h, int side, void* buf, bool pack, const char* what) {
    if (!h || !buf) {
        set_last_error(std::string(what) + ": NULL argument");
        return LBM_EINVAL;
    }
    if (side != 0 && side != 1) {
        set_last_error(std::string(what) + ": side must be 0 (left) or 1 (right)");
        return LBM_EINVAL;
    }
    const PopView v = handle_pops(h);
    if (v.grid.nx < 2) {
        set_last_error(std::string(what) + ": the grid needs two columns");
        return LBM_EINVAL;
    }
    (void)cudaGetLastError();
    cudaError_t e;
    switch (v.storage) {
        case LBM_STORE_F32: e = launch_halo<float>(v, side, buf, pack); break;
        default: e = launch_halo<uint16_t>(v, side, buf, pack); break;   // FP16 / BF16 bit patterns
    }
    if (e != cudaSuccess) {
        set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
        return LBM_ECUDA;
    }
    return LBM_OK;
}

}  // namespace
}  // namespace lbm

extern "C" {

lbm_status lbm_halo_bytes(lbm_handle* h, size_t* bytes) {
    if (!h || !bytes) {
        lbm::set_last_error("lbm_halo_bytes: NULL argument");
        return LBM_EINVAL;
    }
    const lbm::PopView v = lbm::handle_pops(h);
    *bytes = (size_t)36 * v.grid.ny * lbm::elem_bytes(v.storage);
    return LBM_OK;
}

lbm_status lbm_halo_pack(lbm_handle* h, int32_t side, void* dev_buf) {
    return lbm::halo_call(h, side, dev_buf, true, "lbm_halo_pack");
}

lbm_status lbm_halo_unpack(lbm_handle* h, int32_t side, const void* dev_buf) {
    return lbm::halo_call(h, side, const_cast<void*>(dev_buf), false, "lbm_halo_unpack");
}

}  // extern "C"
