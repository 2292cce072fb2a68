// lbm_step_noalloc: one time step that allocates no memory, for callers that
// cannot allocate device memory themselves.  It is the two-pass step (a density
// pass into scratch, then collision and streaming) working on dense FP32
// population arrays that the caller owns; the density scratch is a file-scope
// device array of fixed size instead of a workspace.
//
// The paper has no counterpart: this is an interface for embedding, not part of
// the method.  Same arithmetic as the other FP32 steps (collide.cuh).
#include "collide.cuh"

#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

namespace lbm {
namespace {

constexpr int kNoAllocMaxSites = 1 << 20;     // largest nx * ny accepted
constexpr int kNoAllocMaxRows = 65535;          // gridDim.y limit: the kernels run one block row per grid row
constexpr int kNoAllocMaxDevices = 64;

// Density scratch: rho_A at [0, n), rho_B at [n, 2n); the int after the densities is
// where the collision's guard writes its status (nothing reads it: this entry point
// makes no NaN / negative-density report).  Every GPU that loads the library holds
// these 8 MiB until the process exits.
static __device__ __align__(256) float g_noalloc_scratch[2 * kNoAllocMaxSites + 64];

std::mutex g_noalloc_mu;
float* g_noalloc_ptr[kNoAllocMaxDevices] = {};

__global__ void __launch_bounds__(kThreadsX)
noalloc_density_kernel(const float* __restrict__ S, int nx, int ny, float* __restrict__ rho) {
    const int x = blockIdx.x * kThreadsX + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= nx) return;
    const size_t n = (size_t)nx * ny;
    const size_t k = (size_t)y * nx + x;
    for (int s = 0; s < 2; ++s) {
        float f[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = __ldg(S + (size_t)(s * 9 + i) * n + k);
        rho[(size_t)s * n + k] = sum9(f);
    }
}

// Collide the post-streaming populations of each site and push them to their
// destinations (periodic x, half-way bounce-back at the walls).
__global__ void __launch_bounds__(kThreadsX)
noalloc_collide_push_kernel(const float* __restrict__ S, float* __restrict__ out, const float* __restrict__ rho,
                            Physics ph, int nx, int ny, int* flag) {
    const int x = blockIdx.x * kThreadsX + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= nx) return;
    const size_t n = (size_t)nx * ny;
    const size_t k = (size_t)y * nx + x;
    float f[2][9];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int i = 0; i < 9; ++i) f[s][i] = __ldg(S + (size_t)(s * 9 + i) * n + k);
    const int xm = x == 0 ? nx - 1 : x - 1;
    const int xp = x == nx - 1 ? 0 : x + 1;
    Nbr p[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const float* r = rho + (size_t)s * n;
        p[s].E = __ldg(r + (size_t)y * nx + xp);
        p[s].W = __ldg(r + (size_t)y * nx + xm);
        if (y + 1 < ny) {
            p[s].N = __ldg(r + (size_t)(y + 1) * nx + x);
            p[s].NE = __ldg(r + (size_t)(y + 1) * nx + xp);
            p[s].NW = __ldg(r + (size_t)(y + 1) * nx + xm);
        } else {
            p[s].N = p[s].NE = p[s].NW = 0.0f;
        }
        if (y > 0) {
            p[s].S = __ldg(r + (size_t)(y - 1) * nx + x);
            p[s].SE = __ldg(r + (size_t)(y - 1) * nx + xp);
            p[s].SW = __ldg(r + (size_t)(y - 1) * nx + xm);
        } else {
            p[s].S = p[s].SE = p[s].SW = 0.0f;
        }
    }
    collide_site<true>(f, p[0], p[1], ph, y, ny, flag);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int ty = y + cy(i);
            if (ty >= 0 && ty < ny) {
                const int tx = cx(i) == 0 ? x : (cx(i) == 1 ? xp : xm);
                out[(size_t)(s * 9 + i) * n + (size_t)ty * nx + tx] = f[s][i];
            } else {
                out[(size_t)(s * 9 + opp(i)) * n + k] = f[s][i];
            }
        }
    }
}

lbm_status noalloc_fail(lbm_status st, const std::string& msg) {
    set_last_error(msg);
    return st;
}

}  // namespace
}  // namespace lbm

extern "C" lbm_status lbm_step_noalloc(const lbm_params* p, const float* pops_in, float* pops_out,
                                       void* cuda_stream) {
    using namespace lbm;
    if (!p || !pops_in || !pops_out) return noalloc_fail(LBM_EINVAL, "lbm_step_noalloc: NULL argument");
    if (pops_in == pops_out) return noalloc_fail(LBM_EINVAL, "lbm_step_noalloc: pops_in and pops_out must differ");
    if (p->nx < 4 || p->ny < 8) return noalloc_fail(LBM_EINVAL, "lbm_step_noalloc: nx must be >= 4 and ny >= 8");
    if (p->ny > kNoAllocMaxRows)
        return noalloc_fail(LBM_EINVAL, "lbm_step_noalloc: ny = " + std::to_string(p->ny) + " exceeds " +
                                            std::to_string(kNoAllocMaxRows) + " rows (one grid row per launch row)");
    if ((int64_t)p->nx * p->ny > kNoAllocMaxSites)
        return noalloc_fail(LBM_EINVAL, "lbm_step_noalloc: nx * ny = " + std::to_string((int64_t)p->nx * p->ny) +
                                            " exceeds the fixed scratch of " + std::to_string(kNoAllocMaxSites) +
                                            " sites; use lbm_step on a handle");
    if (p->storage != LBM_STORE_F32) return noalloc_fail(LBM_EINVAL, "lbm_step_noalloc: FP32 populations only");
    {
        const uintptr_t bytes = (uintptr_t)18 * (uintptr_t)p->nx * (uintptr_t)p->ny * sizeof(float);
        const uintptr_t a = (uintptr_t)pops_in, b = (uintptr_t)pops_out;
        if (a < b + bytes && b < a + bytes)
            return noalloc_fail(LBM_EINVAL, "lbm_step_noalloc: pops_in and pops_out overlap");
    }
    if (!(p->tau_A > 0.5) || !(p->tau_B > 0.5)) return noalloc_fail(LBM_EINVAL, "lbm_step_noalloc: tau must be > 0.5");
    if (p->gravity_mode < 0 || p->gravity_mode > 1)
        return noalloc_fail(LBM_EINVAL, "lbm_step_noalloc: gravity_mode must be 0 or 1");
    if (p->wall_mode < 0 || p->wall_mode > 1)
        return noalloc_fail(LBM_EINVAL, "lbm_step_noalloc: wall_mode must be 0 or 1");
    const double vals[] = {p->G, p->G_wall_A, p->G_wall_B, p->g, p->gx};
    for (double v : vals)
        if (!std::isfinite(v)) return noalloc_fail(LBM_EINVAL, "lbm_step_noalloc: parameters must be finite");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(LBM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return noalloc_fail(LBM_EINVAL, "lbm_step_noalloc: device index too large");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // an error left by the caller's earlier work is reported, not cleared or taken as ours
    e = cudaPeekAtLastError();
    if (e != cudaSuccess)
        return noalloc_fail(LBM_ECUDA, std::string("lbm_step_noalloc: a CUDA error was pending before the call: ") +
                                           cudaGetErrorString(e));
    cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &capture);
    if (e != cudaSuccess) return noalloc_fail(LBM_ECUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
    float* scratch = nullptr;
    {
        // The host-side name of the scratch array is only a stand-in: its device address
        // belongs to the context that is current.  Outside a stream capture every call looks
        // it up again, so a device reset or another context on the same device gets the
        // address that is valid there; inside a capture the address of the last call made
        // outside one on this device is used.
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (capture == cudaStreamCaptureStatusNone) {
            float* addr = nullptr;
            e = cudaGetSymbolAddress((void**)&addr, g_noalloc_scratch);
            if (e != cudaSuccess) return noalloc_fail(LBM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_noalloc_ptr[dev] = addr;
        } else if (!g_noalloc_ptr[dev]) {
            return noalloc_fail(LBM_ESTATE, "lbm_step_noalloc: the first call on a device must come before any stream capture");
        }
        scratch = g_noalloc_ptr[dev];
    }
    const int nx = p->nx, ny = p->ny;
    float* rho = scratch;
    int* flag = reinterpret_cast<int*>(scratch + 2 * (size_t)kNoAllocMaxSites);

    Physics ph;
    ph.tau[0] = (float)p->tau_A;
    ph.tau[1] = (float)p->tau_B;
    ph.om[0] = (float)(1.0 / p->tau_A);
    ph.om[1] = (float)(1.0 / p->tau_B);
    ph.G = (float)p->G;
    ph.ay_wall_bottom[0] = (float)(p->G_wall_A / 6.0);
    ph.ay_wall_bottom[1] = (float)(p->G_wall_B / 6.0);
    ph.ay_wall_top[0] = (float)(-p->G_wall_A / 6.0);
    ph.ay_wall_top[1] = (float)(-p->G_wall_B / 6.0);
    ph.ay_ext[0] = (float)(-p->g);
    ph.ay_ext[1] = (float)(p->gravity_mode == 0 ? p->g : -p->g);
    ph.ax_ext = (float)p->gx;
    ph.wall_mirror = p->wall_mode == 1 ? 1 : 0;
    ph.shift[0] = ph.shift[1] = 0.0f;
    ph.rho_floor[0] = ph.rho_floor[1] = 0.0f;
    ph.step_in = nullptr;
    ph.step_out = nullptr;

    dim3 grid((nx + kThreadsX - 1) / kThreadsX, ny);
    noalloc_density_kernel<<<grid, kThreadsX, 0, st>>>(pops_in, nx, ny, rho);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(LBM_ECUDA, std::string("lbm_step_noalloc: density kernel launch: ") + cudaGetErrorString(e));
    noalloc_collide_push_kernel<<<grid, kThreadsX, 0, st>>>(pops_in, pops_out, rho, ph, nx, ny, flag);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(LBM_ECUDA, std::string("lbm_step_noalloc: collide/push kernel launch: ") + cudaGetErrorString(e));
    return LBM_OK;
}
