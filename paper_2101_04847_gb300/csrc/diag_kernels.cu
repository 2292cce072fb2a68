// Diagnostics of one state (Section 3 of arXiv 2101.04847): energies, the terms
// of the kinetic-energy budget, the split of the momentum-flux term into bulk
// pressure, Korteweg and tau-dependent parts, enstrophy, row means of the order
// parameter (mixing-layer width) and Cauchy-Crofton crossing counts (interface
// length).
//
// Per-site arithmetic is FP64: the budget terms are centred differences of
// fields whose gradients are ~1e-5 of their values, so FP32 would lose most of
// their digits to cancellation.  Sums are deterministic: warp shuffles, then a
// fixed-order block reduction into per-block partials, then a fixed-order final
// reduction.  Work is split into passes over a 32x8-thread block grid:
//   D1 moments   : rho_A, rho_B, j (sum over components) per site; masses
//   D2 velocity  : physical velocity u = (j + F/2) / rho; E_k, E_p, buoyancy,
//                  row sums of phi, crossing counts
//   D3 tensors   : P^K, K^(tau), grad u + grad u^T per site; <u.grad p_b>, omega^2
//   D4 divergence: <u . div P^K>, <u . div K^(tau)>, <u . div(grad u + grad u^T)>
//   D5 reduce    : per-term and per-row sums of the block partials
// Scratch: 15 doubles per site (M[4], U[2], T[9]).
#include "lattice.cuh"

namespace lbm {

namespace {

constexpr int DX = 32, DY = 8;
constexpr double kCs2 = 1.0 / 3.0;

struct DiagArgs {
    Grid g;
    int nx, ny;
    size_t n;           // nx * ny
    int r0, r1;         // averaged rows [r0, r1)
    double G, gwall[2], gext[2], gx, tau_bar;
    double* M;          // [4][ny][nx]: rho_A, rho_B, jx, jy
    double* U;          // [2][ny][nx]: ux, uy
    double* T;          // [9][ny][nx]: Pxx Pxy Pyy Kxx Kxy Kyy Sxx Sxy Syy
    double* partials;   // [kDiagTerms][nblocks]
    double* rowpart;    // [ny][nbx]
    int nblocks, nbx;   // blocks in total / along x
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block sums of N per-thread values into partials[(term0 + k) * nblocks + block].
template <int N>
__device__ __forceinline__ void block_sums(double (&v)[N], const DiagArgs& a, int term0) {
    __shared__ double sm[N][DY];
    const int lane = threadIdx.x, warp = threadIdx.y;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const double s = warp_sum(v[k]);
        if (lane == 0) sm[k][warp] = s;
    }
    __syncthreads();
    if (warp == 0 && lane < N) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < DY; ++w) s += sm[lane][w];
        a.partials[(size_t)(term0 + lane) * a.nblocks + blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

__device__ __forceinline__ double at(const double* f, const DiagArgs& a, int x, int y) {
    return f[(size_t)y * a.nx + x];
}
__device__ __forceinline__ double at0(const double* f, const DiagArgs& a, int x, int y) {
    return (y < 0 || y >= a.ny) ? 0.0 : f[(size_t)y * a.nx + x];
}

template <typename T>
__global__ void __launch_bounds__(DX * DY) moments_kernel(const T* __restrict__ fin, DiagArgs a, float sA, float sB) {
    const int x = blockIdx.x * DX + threadIdx.x;
    const int y = blockIdx.y * DY + threadIdx.y;
    double v[2] = {0.0, 0.0};
    if (x < a.nx && y < a.ny) {
        const float shift[2] = {sA, sB};
        const int xm = x == 0 ? a.nx - 1 : x - 1;
        const int xp = x == a.nx - 1 ? 0 : x + 1;
        float f[2][9];
        pull_site<T>(fin, a.g, shift, y, x, xm, xp, f);
        double r[2] = {0.0, 0.0}, jx = 0.0, jy = 0.0;
        for (int s = 0; s < 2; ++s) {
            for (int i = 0; i < 9; ++i) {
                const double fi = (double)f[s][i];
                r[s] += fi;
                jx += cx(i) * fi;
                jy += cy(i) * fi;
            }
        }
        const size_t k = (size_t)y * a.nx + x;
        a.M[k] = r[0];
        a.M[a.n + k] = r[1];
        a.M[2 * a.n + k] = jx;
        a.M[3 * a.n + k] = jy;
        v[0] = r[0];
        v[1] = r[1];
    }
    block_sums<2>(v, a, T_MASS_A);
}

// sum_i w_i psi(x + c_i) c_i of a density field (zero on the virtual wall rows)
__device__ __forceinline__ void nbr_sum_d(const double* f, const DiagArgs& a, int x, int y, double& sx, double& sy) {
    const int xm = x == 0 ? a.nx - 1 : x - 1;
    const int xp = x == a.nx - 1 ? 0 : x + 1;
    const double E = at0(f, a, xp, y), W = at0(f, a, xm, y);
    const double N = at0(f, a, x, y + 1), S = at0(f, a, x, y - 1);
    const double NE = at0(f, a, xp, y + 1), NW = at0(f, a, xm, y + 1);
    const double SE = at0(f, a, xp, y - 1), SW = at0(f, a, xm, y - 1);
    sx = (E - W) / 9.0 + (NE - NW - SW + SE) / 36.0;
    sy = (N - S) / 9.0 + (NE + NW - SW - SE) / 36.0;
}

__global__ void __launch_bounds__(DX * DY) velocity_kernel(DiagArgs a, int lo, int hi, int accumulate) {
    const int x = blockIdx.x * DX + threadIdx.x;
    const int y = blockIdx.y * DY + threadIdx.y;
    const bool valid = x < a.nx && y >= lo && y < hi && y < a.ny;
    const bool avg = valid && y >= a.r0 && y < a.r1;
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double phi = 0.0;
    if (valid) {
        const size_t k = (size_t)y * a.nx + x;
        const double rA = a.M[k], rB = a.M[a.n + k], jx = a.M[2 * a.n + k], jy = a.M[3 * a.n + k];
        double nAx, nAy, nBx, nBy;
        nbr_sum_d(a.M, a, x, y, nAx, nAy);
        nbr_sum_d(a.M + a.n, a, x, y, nBx, nBy);
        double wA = 0.0, wB = 0.0;  // wall force: sum_i w_i S(x + c_i) c_i = (0, -1/6) on row 0, (0, 1/6) on row ny-1
        if (y == 0) { wA += a.gwall[0] / 6.0; wB += a.gwall[1] / 6.0; }
        if (y == a.ny - 1) { wA -= a.gwall[0] / 6.0; wB -= a.gwall[1] / 6.0; }
        const double aAx = -a.G * nBx + a.gx, aAy = -a.G * nBy + wA + a.gext[0];
        const double aBx = -a.G * nAx + a.gx, aBy = -a.G * nAy + wB + a.gext[1];
        const double Fx = rA * aAx + rB * aBx, Fy = rA * aAy + rB * aBy;
        const double rho = rA + rB;
        const double ux = (jx + 0.5 * Fx) / rho, uy = (jy + 0.5 * Fy) / rho;
        a.U[k] = ux;
        a.U[a.n + k] = uy;
        phi = rA - rB;
        if (avg) {
            v[0] = 0.5 * rho * (ux * ux + uy * uy);
            v[1] = (double)y * phi;
            v[2] = uy * phi;
            v[3] = rho;
            // crossing counts of (phi > 0) for pairs starting at (x, y)
            const int xm = x == 0 ? a.nx - 1 : x - 1;
            const int xp = x == a.nx - 1 ? 0 : x + 1;
            const bool b = phi > 0.0;
            const bool bE = (a.M[(size_t)y * a.nx + xp] - a.M[a.n + (size_t)y * a.nx + xp]) > 0.0;
            v[4] = (b != bE) ? 1.0 : 0.0;
            if (y + 1 < a.r1) {
                const size_t up = (size_t)(y + 1) * a.nx;
                const bool bN = (a.M[up + x] - a.M[a.n + up + x]) > 0.0;
                const bool bNE = (a.M[up + xp] - a.M[a.n + up + xp]) > 0.0;
                const bool bNW = (a.M[up + xm] - a.M[a.n + up + xm]) > 0.0;
                v[5] = (b != bN) ? 1.0 : 0.0;
                v[6] = (b != bNE) ? 1.0 : 0.0;
                v[7] = (b != bNW) ? 1.0 : 0.0;
            }
        }
    }
    if (!accumulate) return;  // uniform over the launch
    // row partial of phi: one warp is one row of 32 columns
    const double rs = warp_sum(avg ? phi : 0.0);
    if (threadIdx.x == 0 && y < a.ny && y >= a.r0 && y < a.r1) a.rowpart[(size_t)y * a.nbx + blockIdx.x] = rs;
    double e[4] = {v[0], v[1], v[2], v[3]};
    block_sums<4>(e, a, T_EK);
    __syncthreads();
    double c[4] = {v[4], v[5], v[6], v[7]};
    block_sums<4>(c, a, T_N0);
}

__global__ void __launch_bounds__(DX * DY) tensor_kernel(DiagArgs a) {
    const int x = blockIdx.x * DX + threadIdx.x;
    const int y = blockIdx.y * DY + threadIdx.y;
    const bool valid = x < a.nx && y >= a.r0 - 1 && y < a.r1 + 1;
    const bool avg = valid && y >= a.r0 && y < a.r1;
    double v[2] = {0.0, 0.0};
    if (valid) {
        const int xm = x == 0 ? a.nx - 1 : x - 1;
        const int xp = x == a.nx - 1 ? 0 : x + 1;
        const double* A = a.M;
        const double* B = a.M + a.n;
        const double rA = at(A, a, x, y), rB = at(B, a, x, y);
        const double rAE = at(A, a, xp, y), rAW = at(A, a, xm, y), rAN = at(A, a, x, y + 1), rAS = at(A, a, x, y - 1);
        const double rBE = at(B, a, xp, y), rBW = at(B, a, xm, y), rBN = at(B, a, x, y + 1), rBS = at(B, a, x, y - 1);
        const double phi = rA - rB;
        const double phE = rAE - rBE, phW = rAW - rBW, phN = rAN - rBN, phS = rAS - rBS;
        const double kappa = kCs2 * kCs2 * a.G / 4.0;
        // Korteweg stress (Section 2, Eq. "Korteweg stress tensor")
        const double px = 0.5 * (phE - phW), py = 0.5 * (phN - phS);
        const double lap = phE + phW + phN + phS - 4.0 * phi;
        const double iso = -kappa * phi * lap - 0.5 * kappa * (px * px + py * py);
        // tau-dependent stress (Section 2, Eq. "Spurious contribution")
        const double dAx = 0.5 * (rAE - rAW), dAy = 0.5 * (rAN - rAS);
        const double dBx = 0.5 * (rBE - rBW), dBy = 0.5 * (rBN - rBS);
        const double vx = rB * dAx - rA * dBx, vy = rB * dAy - rA * dBy;
        const double prod = fmax(rA * rB, 1e-12);
        const double tm = a.tau_bar - 0.5;
        const double coef = kCs2 * kCs2 * tm * tm / (prod * (rA + rB));
        // velocity gradient (symmetrised)
        const double* UX = a.U;
        const double* UY = a.U + a.n;
        const double uxE = at(UX, a, xp, y), uxW = at(UX, a, xm, y), uxN = at(UX, a, x, y + 1), uxS = at(UX, a, x, y - 1);
        const double uyE = at(UY, a, xp, y), uyW = at(UY, a, xm, y), uyN = at(UY, a, x, y + 1), uyS = at(UY, a, x, y - 1);
        const double dxux = 0.5 * (uxE - uxW), dyux = 0.5 * (uxN - uxS);
        const double dxuy = 0.5 * (uyE - uyW), dyuy = 0.5 * (uyN - uyS);
        const size_t k = (size_t)y * a.nx + x;
        const size_t n = a.n;
        a.T[k] = iso + kappa * px * px;
        a.T[n + k] = kappa * px * py;
        a.T[2 * n + k] = iso + kappa * py * py;
        a.T[3 * n + k] = coef * vx * vx;
        a.T[4 * n + k] = coef * vx * vy;
        a.T[5 * n + k] = coef * vy * vy;
        a.T[6 * n + k] = 2.0 * dxux;
        a.T[7 * n + k] = dxuy + dyux;
        a.T[8 * n + k] = 2.0 * dyuy;
        if (avg) {
            const double G4 = a.G * kCs2 / 4.0;
            const double pE = kCs2 * (rAE + rBE) + G4 * ((rAE + rBE) * (rAE + rBE) - phE * phE);
            const double pW = kCs2 * (rAW + rBW) + G4 * ((rAW + rBW) * (rAW + rBW) - phW * phW);
            const double pN = kCs2 * (rAN + rBN) + G4 * ((rAN + rBN) * (rAN + rBN) - phN * phN);
            const double pS = kCs2 * (rAS + rBS) + G4 * ((rAS + rBS) * (rAS + rBS) - phS * phS);
            const double ux = at(UX, a, x, y), uy = at(UY, a, x, y);
            v[0] = ux * 0.5 * (pE - pW) + uy * 0.5 * (pN - pS);
            const double om = dxuy - dyux;
            v[1] = om * om;
        }
    }
    block_sums<2>(v, a, T_FLUX_PB);
}

__device__ __forceinline__ void div_at(const double* Txx, const double* Txy, const double* Tyy, const DiagArgs& a,
                                       int x, int y, int xm, int xp, double& dx, double& dy) {
    dx = 0.5 * (at(Txx, a, xp, y) - at(Txx, a, xm, y)) + 0.5 * (at(Txy, a, x, y + 1) - at(Txy, a, x, y - 1));
    dy = 0.5 * (at(Txy, a, xp, y) - at(Txy, a, xm, y)) + 0.5 * (at(Tyy, a, x, y + 1) - at(Tyy, a, x, y - 1));
}

__global__ void __launch_bounds__(DX * DY) divergence_kernel(DiagArgs a) {
    const int x = blockIdx.x * DX + threadIdx.x;
    const int y = blockIdx.y * DY + threadIdx.y;
    double v[3] = {0.0, 0.0, 0.0};
    if (x < a.nx && y >= a.r0 && y < a.r1) {
        const int xm = x == 0 ? a.nx - 1 : x - 1;
        const int xp = x == a.nx - 1 ? 0 : x + 1;
        const size_t n = a.n;
        const double ux = at(a.U, a, x, y), uy = at(a.U + n, a, x, y);
        double dx, dy;
        div_at(a.T, a.T + n, a.T + 2 * n, a, x, y, xm, xp, dx, dy);
        v[0] = ux * dx + uy * dy;
        div_at(a.T + 3 * n, a.T + 4 * n, a.T + 5 * n, a, x, y, xm, xp, dx, dy);
        v[1] = ux * dx + uy * dy;
        div_at(a.T + 6 * n, a.T + 7 * n, a.T + 8 * n, a, x, y, xm, xp, dx, dy);
        v[2] = ux * dx + uy * dy;
    }
    block_sums<3>(v, a, T_FLUX_K);
}

// blocks [0, kDiagTerms): term sums over the block partials; the next blocks: row sums.
__global__ void __launch_bounds__(256) reduce_kernel(DiagArgs a, double* out) {
    __shared__ double sm[256];
    const int tid = threadIdx.x;
    double s = 0.0;
    if (blockIdx.x < kDiagTerms) {
        const double* p = a.partials + (size_t)blockIdx.x * a.nblocks;
        for (int b = tid; b < a.nblocks; b += 256) s += p[b];
    } else {
        const int y = a.r0 + (blockIdx.x - kDiagTerms);
        const double* p = a.rowpart + (size_t)y * a.nbx;
        for (int b = tid; b < a.nbx; b += 256) s += p[b];
    }
    sm[tid] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (tid < o) sm[tid] += sm[tid + o];
        __syncthreads();
    }
    if (tid == 0) out[blockIdx.x] = sm[0];
}

DiagArgs make_args(const DiagLaunch& D) {
    DiagArgs a;
    a.g = D.grid;
    a.nx = D.grid.nx;
    a.ny = D.grid.ny;
    a.n = (size_t)a.nx * a.ny;
    a.r0 = D.crop;
    a.r1 = a.ny - D.crop;
    a.G = D.G;
    a.gwall[0] = D.G_wall[0];
    a.gwall[1] = D.G_wall[1];
    a.gext[0] = D.g_ext[0];
    a.gext[1] = D.g_ext[1];
    a.gx = D.gx;
    a.tau_bar = D.tau_bar;
    a.M = D.scratch;
    a.U = D.scratch + 4 * a.n;
    a.T = D.scratch + 6 * a.n;
    a.nbx = (a.nx + DX - 1) / DX;
    a.nblocks = a.nbx * ((a.ny + DY - 1) / DY);
    a.partials = D.partials;
    a.rowpart = D.partials + (size_t)kDiagTerms * a.nblocks;
    return a;
}

template <typename T>
cudaError_t launch_moments(const DiagLaunch& D, const DiagArgs& a, cudaStream_t st) {
    dim3 grid(a.nbx, (a.ny + DY - 1) / DY), block(DX, DY);
    moments_kernel<T><<<grid, block, 0, st>>>((const T*)D.fin, a, D.shift[0], D.shift[1]);
    return cudaGetLastError();
}

cudaError_t moments(const DiagLaunch& D, const DiagArgs& a, cudaStream_t st) {
    switch (D.storage) {
        case LBM_STORE_F16: return launch_moments<__half>(D, a, st);
        case LBM_STORE_BF16: return launch_moments<__nv_bfloat16>(D, a, st);
        default: return launch_moments<float>(D, a, st);
    }
}

}  // namespace

size_t diag_scratch_doubles(int nx, int ny) { return (size_t)15 * nx * ny; }

size_t diag_partials_doubles(int nx, int ny) {
    const size_t gx = (nx + DX - 1) / DX, gy = (ny + DY - 1) / DY;
    return (size_t)kDiagTerms * gx * gy + (size_t)ny * gx;
}

cudaError_t launch_diagnostics(const DiagLaunch& D, cudaStream_t st) {
    (void)cudaGetLastError();   // a launch reports only its own error
    DiagArgs a = make_args(D);
    // The velocity gradient terms of D3/D4 need u two rows outside the averaged rows and
    // u needs rho one row further out; crop >= 3 keeps all of them inside the grid.
    cudaError_t e = moments(D, a, st);
    if (e != cudaSuccess) return e;
    dim3 grid(a.nbx, (a.ny + DY - 1) / DY), block(DX, DY);
    velocity_kernel<<<grid, block, 0, st>>>(a, a.r0 - 2, a.r1 + 2, 1);
    tensor_kernel<<<grid, block, 0, st>>>(a);
    divergence_kernel<<<grid, block, 0, st>>>(a);
    reduce_kernel<<<kDiagTerms + (a.r1 - a.r0), 256, 0, st>>>(a, D.out);
    return cudaGetLastError();
}

cudaError_t launch_fields(const DiagLaunch& D, double* /*unused*/, cudaStream_t st) {
    (void)cudaGetLastError();
    DiagArgs a = make_args(D);
    cudaError_t e = moments(D, a, st);
    if (e != cudaSuccess) return e;
    dim3 grid(a.nbx, (a.ny + DY - 1) / DY), block(DX, DY);
    velocity_kernel<<<grid, block, 0, st>>>(a, 0, a.ny, 0);
    return cudaGetLastError();
}

}  // namespace lbm
