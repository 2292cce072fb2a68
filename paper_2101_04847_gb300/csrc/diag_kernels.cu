// Diagnostics of one state (Section 3 of arXiv 2101.04847): energies, the terms
// of the kinetic-energy budget, the split of the momentum-flux term into bulk
// pressure, Korteweg and tau-dependent parts, enstrophy, row means of the order
// parameter (mixing-layer width) and Cauchy-Crofton crossing counts (interface
// length).
//
// Precision.  The budget terms are centred differences of fields whose gradients
// are ~1e-5 of their values, so plain FP32 would lose most of their digits to
// cancellation; FP64, on the other hand, runs at a small fraction of the FP32
// rate on this GPU.  All per-site arithmetic is therefore double-float ("dfl":
// an unevaluated sum hi + lo of two floats, ~44 significant bits) built from the
// error-free transformations TwoSum (Knuth), Fast2Sum (Dekker) and the FMA
// product error (Ogita, Rump and Oishi, "Accurate sum and dot product", 2005).
// The moments are exact sums of the FP32 populations.  Block partials and the
// final sums are FP64, in a fixed order, so the results are deterministic.
//
// Passes over a grid of 32x8-thread blocks, each covering 32 columns x 64 rows
// (a thread takes 8 rows):
//   D1 moments   : rho_A, rho_B, j (sum over components) per site; masses
//   D2 velocity  : physical velocity u = (j + F/2) / rho; E_k, E_p, buoyancy,
//                  row sums of phi and of the mass fraction, crossing counts
//   D3 tensors   : P^K, K^(tau), grad u + grad u^T per site; <u.grad p_b>, omega^2
//   D4 divergence: <u . div P^K>, <u . div K^(tau)>, <u . div(grad u + grad u^T)>
//   D5 reduce    : per-term and per-row sums of the block partials
// Scratch (8-byte units per site): M[4] (rho_A, rho_B, jx, jy), U[2] (ux, uy),
// T[9] (Pxx Pxy Pyy Kxx Kxy Kyy Sxx Sxy Syy), all dfl; the field extraction
// reuses T[0..3] for rho_A, rho_B, ux, uy as doubles.
#include "lattice.cuh"

#include <algorithm>

namespace lbm {

namespace {

constexpr int DX = 32, DY = 8, RY = 8;   // a thread takes rows y0 + threadIdx.y + r DY, r < RY
constexpr int BY = DY * RY;               // rows per block
constexpr double kCs2 = 1.0 / 3.0;

// ---------------------------------------------------------------------------
// double-float arithmetic
// ---------------------------------------------------------------------------
struct dfl { float hi, lo; };   // value hi + lo with |lo| <= ulp(hi) / 2

__device__ __forceinline__ dfl two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {   // |a| >= |b| or a == 0
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
    dfl s = two_sum(a.hi, b.hi);
    const dfl t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dfl operator-(dfl a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    return fast_two_sum(p, e);
}
__device__ __forceinline__ dfl operator*(dfl a, float b) {   // exact for b a power of two
    const float p = a.hi * b;
    const float e = fmaf(a.lo, b, fmaf(a.hi, b, -p));
    return fast_two_sum(p, e);
}
// a / b by one correction step of the FP32 quotient (remainder a - b q1 in dfl)
__device__ __forceinline__ dfl dfl_div(dfl a, dfl b) {
    const float q1 = a.hi / b.hi;
    const dfl r = a - b * q1;
    return fast_two_sum(q1, r.hi / b.hi);
}
__device__ __forceinline__ double to_d(dfl a) { return (double)a.hi + (double)a.lo; }
dfl dfl_of(double v) {   // host: nearest dfl of a double
    const float hi = (float)v;
    return {hi, (float)(v - (double)hi)};
}

struct DiagArgs {
    Grid g;
    int nx, ny;
    size_t n;           // nx * ny
    int r0, r1;         // averaged rows [r0, r1)
    // physics constants as dfl: G, body force, wall forces (G_wall / 6), external accelerations
    dfl G, gx, gw6[2], gext[2];
    dfl cs2, w1, w2, kappa, G4, cK, floor_prod;
    dfl* M;             // [4][ny][nx]: rho_A, rho_B, jx, jy
    dfl* U;             // [2][ny][nx]: ux, uy
    dfl* T;             // [9][ny][nx]
    double* F;          // [4][ny][nx] doubles (field extraction; aliases T)
    double* partials;   // [kDiagTerms][nblocks]
    double* rowpart;    // [ny][nbx]: row partials of phi
    double* rowpart_c;  // [ny][nbx]: row partials of the mass fraction rho_A / (rho_A + rho_B)
    int nblocks, nbx;   // blocks in total / along x
    int mirror;         // 1: the pseudopotential beyond a wall is the wall row's (wall_mode 1)
};

__device__ __forceinline__ int row_of(int r) { return blockIdx.y * BY + threadIdx.y + r * DY; }

__device__ __forceinline__ dfl warp_sum(dfl v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const dfl w = {__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
        v = v + w;
    }
    return v;
}

// Block sums of N per-thread values into partials[(term0 + k) * nblocks + block].
template <int N>
__device__ __forceinline__ void block_sums(const dfl (&v)[N], const DiagArgs& a, int term0) {
    __shared__ double sm[N][DY];
    const int lane = threadIdx.x, warp = threadIdx.y;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const dfl s = warp_sum(v[k]);
        if (lane == 0) sm[k][warp] = to_d(s);
    }
    __syncthreads();
    if (warp == 0 && lane < N) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < DY; ++w) s += sm[lane][w];
        a.partials[(size_t)(term0 + lane) * a.nblocks + blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

__device__ __forceinline__ dfl at(const dfl* f, const DiagArgs& a, int x, int y) {
    return f[(size_t)y * a.nx + x];
}
// a density field's value as the Shan-Chen force sees it: beyond a wall 0, or with
// the mirror the wall row's own value
__device__ __forceinline__ dfl at0(const dfl* f, const DiagArgs& a, int x, int y) {
    if (y < 0 || y >= a.ny) {
        if (!a.mirror) return dfl{0.0f, 0.0f};
        y = y < 0 ? 0 : a.ny - 1;
    }
    return f[(size_t)y * a.nx + x];
}

// Exact sum of FP32 terms: every TwoSum error is kept in lo (its own rounding is
// ~2^-48 of the largest term), normalised at the end.
struct Acc {
    float hi, lo;
    __device__ __forceinline__ void add(float v) {
        const dfl s = two_sum(hi, v);
        hi = s.hi;
        lo += s.lo;
    }
    __device__ __forceinline__ dfl value() const { return fast_two_sum(hi, lo); }
};

template <typename T>
__global__ void __launch_bounds__(DX * DY) moments_kernel(const T* __restrict__ fin, DiagArgs a, float sA, float sB) {
    const int x = blockIdx.x * DX + threadIdx.x;
    dfl v[2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
#pragma unroll 1
    for (int r = 0; r < RY; ++r) {
        const int y = row_of(r);
        if (x >= a.nx || y >= a.ny) break;
        const float shift[2] = {sA, sB};
        // the columns beside the grid from the ghost columns (periodic copies, or a
        // split grid's neighbours)
        float f[2][9];
        pull_site<T>(fin, a.g, shift, y, x, x - 1, x + 1, f);
        dfl rho[2], jx[2], jy[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            Acc m = {f[s][0], 0.0f}, qx = {f[s][1], 0.0f}, qy = {f[s][2], 0.0f};
#pragma unroll
            for (int i = 1; i < 9; ++i) m.add(f[s][i]);
            qx.add(-f[s][3]); qx.add(f[s][5]); qx.add(-f[s][7]); qx.add(f[s][8]); qx.add(-f[s][6]);
            qy.add(-f[s][4]); qy.add(f[s][5]); qy.add(-f[s][7]); qy.add(f[s][6]); qy.add(-f[s][8]);
            rho[s] = m.value();
            jx[s] = qx.value();
            jy[s] = qy.value();
        }
        const size_t k = (size_t)y * a.nx + x;
        a.M[k] = rho[0];
        a.M[a.n + k] = rho[1];
        a.M[2 * a.n + k] = jx[0] + jx[1];
        a.M[3 * a.n + k] = jy[0] + jy[1];
        v[0] = v[0] + rho[0];
        v[1] = v[1] + rho[1];
    }
    block_sums<2>(v, a, T_MASS_A);
}

// sum_i w_i psi(x + c_i) c_i of a density field (the virtual wall rows as at0 gives them)
__device__ __forceinline__ void nbr_sum_d(const dfl* f, const DiagArgs& a, int x, int y, dfl& sx, dfl& sy) {
    const int xm = x == 0 ? a.nx - 1 : x - 1;
    const int xp = x == a.nx - 1 ? 0 : x + 1;
    const dfl E = at0(f, a, xp, y), W = at0(f, a, xm, y);
    const dfl N = at0(f, a, x, y + 1), S = at0(f, a, x, y - 1);
    const dfl NE = at0(f, a, xp, y + 1), NW = at0(f, a, xm, y + 1);
    const dfl SE = at0(f, a, xp, y - 1), SW = at0(f, a, xm, y - 1);
    const dfl d = NE - SW;
    sx = (E - W) * a.w1 + (d + (SE - NW)) * a.w2;
    sy = (N - S) * a.w1 + (d + (NW - SE)) * a.w2;
}

// accumulate = 0: fields only (rho_A, rho_B, ux, uy as doubles into F)
__global__ void __launch_bounds__(DX * DY) velocity_kernel(DiagArgs a, int lo, int hi, int accumulate) {
    const int x = blockIdx.x * DX + threadIdx.x;
    dfl v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = {0.0f, 0.0f};
#pragma unroll 1
    for (int r = 0; r < RY; ++r) {
        const int y = row_of(r);
        const bool valid = x < a.nx && y >= lo && y < hi && y < a.ny;
        const bool avg = valid && y >= a.r0 && y < a.r1;
        dfl phi = {0.0f, 0.0f}, cA = {0.0f, 0.0f};
        if (valid) {
            const size_t k = (size_t)y * a.nx + x;
            const dfl rA = a.M[k], rB = a.M[a.n + k], jx = a.M[2 * a.n + k], jy = a.M[3 * a.n + k];
            dfl nAx, nAy, nBx, nBy;
            nbr_sum_d(a.M, a, x, y, nAx, nAy);
            nbr_sum_d(a.M + a.n, a, x, y, nBx, nBy);
            // wall force: sum_i w_i S(x + c_i) c_i = (0, -1/6) on row 0, (0, 1/6) on row ny-1
            dfl wA = {0.0f, 0.0f}, wB = {0.0f, 0.0f};
            if (y == 0) { wA = wA + a.gw6[0]; wB = wB + a.gw6[1]; }
            if (y == a.ny - 1) { wA = wA - a.gw6[0]; wB = wB - a.gw6[1]; }
            const dfl aAx = a.gx - a.G * nBx, aAy = (wA + a.gext[0]) - a.G * nBy;
            const dfl aBx = a.gx - a.G * nAx, aBy = (wB + a.gext[1]) - a.G * nAy;
            const dfl Fx = rA * aAx + rB * aBx, Fy = rA * aAy + rB * aBy;
            const dfl rho = rA + rB;
            const dfl ux = dfl_div(jx + Fx * 0.5f, rho), uy = dfl_div(jy + Fy * 0.5f, rho);
            a.U[k] = ux;
            a.U[a.n + k] = uy;
            if (!accumulate) {
                a.F[k] = to_d(rA);
                a.F[a.n + k] = to_d(rB);
                a.F[2 * a.n + k] = to_d(ux);
                a.F[3 * a.n + k] = to_d(uy);
            }
            phi = rA - rB;
            if (rho.hi > 0.0f) cA = dfl_div(rA, rho);
            if (avg) {
                v[0] = v[0] + rho * (ux * ux + uy * uy) * 0.5f;
                v[1] = v[1] + phi * (float)y;
                v[2] = v[2] + uy * phi;
                v[3] = v[3] + rho;
                // crossing counts of (phi > 0) for pairs starting at (x, y); the sign
                // of hi is the sign of the exact difference
                const int xm = x == 0 ? a.nx - 1 : x - 1;
                const int xp = x == a.nx - 1 ? 0 : x + 1;
                auto positive = [&](size_t kk) { return (a.M[kk] - a.M[a.n + kk]).hi > 0.0f; };
                const bool b = phi.hi > 0.0f;
                if (b != positive((size_t)y * a.nx + xp)) v[4].hi += 1.0f;
                if (y + 1 < a.r1) {
                    const size_t up = (size_t)(y + 1) * a.nx;
                    if (b != positive(up + x)) v[5].hi += 1.0f;
                    if (b != positive(up + xp)) v[6].hi += 1.0f;
                    if (b != positive(up + xm)) v[7].hi += 1.0f;
                }
            }
        }
        if (accumulate) {   // uniform over the launch
            // row partial of phi: one warp is one row of 32 columns
            const dfl rs = warp_sum(avg ? phi : dfl{0.0f, 0.0f});
            const dfl rc = warp_sum(avg ? cA : dfl{0.0f, 0.0f});
            if (threadIdx.x == 0 && y < a.ny && y >= a.r0 && y < a.r1) {
                a.rowpart[(size_t)y * a.nbx + blockIdx.x] = to_d(rs);
                a.rowpart_c[(size_t)y * a.nbx + blockIdx.x] = to_d(rc);
            }
        }
    }
    if (!accumulate) return;
    const dfl e[4] = {v[0], v[1], v[2], v[3]};
    block_sums<4>(e, a, T_EK);
    __syncthreads();
    const dfl c[4] = {v[4], v[5], v[6], v[7]};
    block_sums<4>(c, a, T_N0);
}

__global__ void __launch_bounds__(DX * DY) tensor_kernel(DiagArgs a) {
    const int x = blockIdx.x * DX + threadIdx.x;
    dfl v[2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
#pragma unroll 1
    for (int r = 0; r < RY; ++r) {
        const int y = row_of(r);
        const bool valid = x < a.nx && y >= a.r0 - 1 && y < a.r1 + 1;
        const bool avg = valid && y >= a.r0 && y < a.r1;
        if (!valid) continue;
        const int xm = x == 0 ? a.nx - 1 : x - 1;
        const int xp = x == a.nx - 1 ? 0 : x + 1;
        const dfl* A = a.M;
        const dfl* B = a.M + a.n;
        const dfl rA = at(A, a, x, y), rB = at(B, a, x, y);
        const dfl rAE = at(A, a, xp, y), rAW = at(A, a, xm, y), rAN = at(A, a, x, y + 1), rAS = at(A, a, x, y - 1);
        const dfl rBE = at(B, a, xp, y), rBW = at(B, a, xm, y), rBN = at(B, a, x, y + 1), rBS = at(B, a, x, y - 1);
        const dfl phi = rA - rB;
        const dfl phE = rAE - rBE, phW = rAW - rBW, phN = rAN - rBN, phS = rAS - rBS;
        // Korteweg stress (Section 2, Eq. "Korteweg stress tensor")
        const dfl px = (phE - phW) * 0.5f, py = (phN - phS) * 0.5f;
        const dfl lap = ((phE + phW) + (phN + phS)) - phi * 4.0f;
        const dfl iso = -(a.kappa * phi * lap) - (a.kappa * (px * px + py * py)) * 0.5f;
        // tau-dependent stress (Section 2, Eq. "Spurious contribution")
        const dfl dAx = (rAE - rAW) * 0.5f, dAy = (rAN - rAS) * 0.5f;
        const dfl dBx = (rBE - rBW) * 0.5f, dBy = (rBN - rBS) * 0.5f;
        const dfl vx = rB * dAx - rA * dBx, vy = rB * dAy - rA * dBy;
        dfl prod = rA * rB;
        if (prod.hi < a.floor_prod.hi || (prod.hi == a.floor_prod.hi && prod.lo < a.floor_prod.lo)) prod = a.floor_prod;
        const dfl coef = dfl_div(a.cK, prod * (rA + rB));
        // velocity gradient (symmetrised)
        const dfl* UX = a.U;
        const dfl* UY = a.U + a.n;
        const dfl uxE = at(UX, a, xp, y), uxW = at(UX, a, xm, y), uxN = at(UX, a, x, y + 1), uxS = at(UX, a, x, y - 1);
        const dfl uyE = at(UY, a, xp, y), uyW = at(UY, a, xm, y), uyN = at(UY, a, x, y + 1), uyS = at(UY, a, x, y - 1);
        const dfl dxux = (uxE - uxW) * 0.5f, dyux = (uxN - uxS) * 0.5f;
        const dfl dxuy = (uyE - uyW) * 0.5f, dyuy = (uyN - uyS) * 0.5f;
        const size_t k = (size_t)y * a.nx + x;
        const size_t n = a.n;
        const dfl kpx = a.kappa * px;
        a.T[k] = iso + kpx * px;
        a.T[n + k] = kpx * py;
        a.T[2 * n + k] = iso + a.kappa * py * py;
        const dfl cvx = coef * vx;
        a.T[3 * n + k] = cvx * vx;
        a.T[4 * n + k] = cvx * vy;
        a.T[5 * n + k] = coef * vy * vy;
        a.T[6 * n + k] = dxux * 2.0f;
        a.T[7 * n + k] = dxuy + dyux;
        a.T[8 * n + k] = dyuy * 2.0f;
        if (avg) {
            // bulk pressure p_b = cs2 (rho_A + rho_B) + G cs2 / 4 ((rho_A + rho_B)^2 - phi^2)
            auto pb = [&](dfl sA, dfl sB, dfl ph) {
                const dfl sum = sA + sB;
                return a.cs2 * sum + a.G4 * (sum * sum - ph * ph);
            };
            const dfl pE = pb(rAE, rBE, phE), pW = pb(rAW, rBW, phW);
            const dfl pN = pb(rAN, rBN, phN), pS = pb(rAS, rBS, phS);
            const dfl ux = at(UX, a, x, y), uy = at(UY, a, x, y);
            v[0] = v[0] + (ux * (pE - pW) + uy * (pN - pS)) * 0.5f;
            const dfl om = dxuy - dyux;
            v[1] = v[1] + om * om;
        }
    }
    block_sums<2>(v, a, T_FLUX_PB);
}

__device__ __forceinline__ void div_at(const dfl* Txx, const dfl* Txy, const dfl* Tyy, const DiagArgs& a,
                                       int x, int y, int xm, int xp, dfl& dx, dfl& dy) {
    dx = ((at(Txx, a, xp, y) - at(Txx, a, xm, y)) + (at(Txy, a, x, y + 1) - at(Txy, a, x, y - 1))) * 0.5f;
    dy = ((at(Txy, a, xp, y) - at(Txy, a, xm, y)) + (at(Tyy, a, x, y + 1) - at(Tyy, a, x, y - 1))) * 0.5f;
}

__global__ void __launch_bounds__(DX * DY) divergence_kernel(DiagArgs a) {
    const int x = blockIdx.x * DX + threadIdx.x;
    dfl v[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
#pragma unroll 1
    for (int r = 0; r < RY; ++r) {
        const int y = row_of(r);
        if (x >= a.nx || y < a.r0 || y >= a.r1) continue;
        const int xm = x == 0 ? a.nx - 1 : x - 1;
        const int xp = x == a.nx - 1 ? 0 : x + 1;
        const size_t n = a.n;
        const dfl ux = at(a.U, a, x, y), uy = at(a.U + n, a, x, y);
        dfl dx, dy;
        div_at(a.T, a.T + n, a.T + 2 * n, a, x, y, xm, xp, dx, dy);
        v[0] = v[0] + (ux * dx + uy * dy);
        div_at(a.T + 3 * n, a.T + 4 * n, a.T + 5 * n, a, x, y, xm, xp, dx, dy);
        v[1] = v[1] + (ux * dx + uy * dy);
        div_at(a.T + 6 * n, a.T + 7 * n, a.T + 8 * n, a, x, y, xm, xp, dx, dy);
        v[2] = v[2] + (ux * dx + uy * dy);
    }
    block_sums<3>(v, a, T_FLUX_K);
}

// blocks [0, kDiagTerms): term sums over the block partials; the next r1 - r0 blocks:
// row sums of phi; the last r1 - r0 blocks: row sums of the mass fraction.
__global__ void __launch_bounds__(256) reduce_kernel(DiagArgs a, double* out) {
    __shared__ double sm[256];
    const int tid = threadIdx.x;
    double s = 0.0;
    if (blockIdx.x < kDiagTerms) {
        const double* p = a.partials + (size_t)blockIdx.x * a.nblocks;
        for (int b = tid; b < a.nblocks; b += 256) s += p[b];
    } else {
        const int nrows = a.r1 - a.r0;
        const int k = blockIdx.x - kDiagTerms;
        const int y = a.r0 + (k < nrows ? k : k - nrows);
        const double* p = (k < nrows ? a.rowpart : a.rowpart_c) + (size_t)y * a.nbx;
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
    a.G = dfl_of(D.G);
    a.gx = dfl_of(D.gx);
    a.gw6[0] = dfl_of(D.G_wall[0] / 6.0);
    a.gw6[1] = dfl_of(D.G_wall[1] / 6.0);
    a.gext[0] = dfl_of(D.g_ext[0]);
    a.gext[1] = dfl_of(D.g_ext[1]);
    a.cs2 = dfl_of(kCs2);
    a.w1 = dfl_of(1.0 / 9.0);
    a.w2 = dfl_of(1.0 / 36.0);
    a.kappa = dfl_of(kCs2 * kCs2 * D.G / 4.0);
    a.G4 = dfl_of(D.G * kCs2 / 4.0);
    const double tm = D.tau_bar - 0.5;
    a.cK = dfl_of(kCs2 * kCs2 * tm * tm);
    a.floor_prod = dfl_of(1e-12);
    a.mirror = D.wall_mirror;
    a.M = reinterpret_cast<dfl*>(D.scratch);
    a.U = reinterpret_cast<dfl*>(D.scratch + 4 * a.n);
    a.T = reinterpret_cast<dfl*>(D.scratch + 6 * a.n);
    a.F = D.scratch + diag_fields_offset(a.nx, a.ny);
    a.nbx = (a.nx + DX - 1) / DX;
    a.nblocks = a.nbx * ((a.ny + BY - 1) / BY);
    a.partials = D.partials;
    a.rowpart = D.partials + (size_t)kDiagTerms * a.nblocks;
    a.rowpart_c = a.rowpart + (size_t)a.ny * a.nbx;
    return a;
}

template <typename T>
cudaError_t launch_moments(const DiagLaunch& D, const DiagArgs& a, cudaStream_t st) {
    dim3 grid(a.nbx, (a.ny + BY - 1) / BY), block(DX, DY);
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

// ---------------------------------------------------------------------------
// closure network input (FP32)
// ---------------------------------------------------------------------------
struct FeatArgs {
    int nx, ny;
    size_t n;
    float G, gx, gw6[2], gext[2];
    float mean[4], scale[4];
    int mirror;
};

// sum_i w_i rho(x + c_i) c_i of one density field, zero beyond the walls (or the wall
// rows' values with the mirror)
__device__ __forceinline__ void nbr_sum_f(const float* __restrict__ r, const FeatArgs& a, int x, int y, float& sx,
                                          float& sy) {
    const int xm = x == 0 ? a.nx - 1 : x - 1;
    const int xp = x == a.nx - 1 ? 0 : x + 1;
    auto at = [&](int xx, int yy) {
        if (yy < 0 || yy >= a.ny) {
            if (!a.mirror) return 0.0f;
            yy = yy < 0 ? 0 : a.ny - 1;
        }
        return r[(size_t)yy * a.nx + xx];
    };
    const float E = at(xp, y), W = at(xm, y), N = at(x, y + 1), S = at(x, y - 1);
    const float d = at(xp, y + 1) - at(xm, y - 1);
    const float SE = at(xp, y - 1), NW = at(xm, y + 1);
    sx = (E - W) * (1.0f / 9.0f) + (d + (SE - NW)) * (1.0f / 36.0f);
    sy = (N - S) * (1.0f / 9.0f) + (d + (NW - SE)) * (1.0f / 36.0f);
}

// the same force and physical velocity as the diagnostics' velocity pass, in FP32;
// one thread per column, rows y = blockIdx.y, blockIdx.y + gridDim.y, ...
__global__ void __launch_bounds__(128) closure_features_kernel(FeatArgs a, const float* __restrict__ rho2,
                                                                const float* __restrict__ j2, float* __restrict__ xo) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= a.nx) return;
    for (int y = blockIdx.y; y < a.ny; y += gridDim.y) {
        const size_t k = (size_t)y * a.nx + x;
        const float jx = j2[k], jy = j2[a.n + k];
        const float rA = rho2[k], rB = rho2[a.n + k];
        float nAx, nAy, nBx, nBy;
        nbr_sum_f(rho2, a, x, y, nAx, nAy);
        nbr_sum_f(rho2 + a.n, a, x, y, nBx, nBy);
        float wA = 0.0f, wB = 0.0f;
        if (y == 0) { wA += a.gw6[0]; wB += a.gw6[1]; }
        if (y == a.ny - 1) { wA -= a.gw6[0]; wB -= a.gw6[1]; }
        const float aAx = a.gx - a.G * nBx, aAy = (wA + a.gext[0]) - a.G * nBy;
        const float aBx = a.gx - a.G * nAx, aBy = (wB + a.gext[1]) - a.G * nAy;
        const float Fx = rA * aAx + rB * aBx, Fy = rA * aAy + rB * aBy;
        const float rho = rA + rB;
        const float ux = (jx + 0.5f * Fx) / rho, uy = (jy + 0.5f * Fy) / rho;
        const float v[4] = {rA, rB, ux, uy};
#pragma unroll
        for (int c = 0; c < 4; ++c) xo[(size_t)c * a.n + k] = (v[c] - a.mean[c]) / a.scale[c];
    }
}

}  // namespace

cudaError_t launch_closure_features(const DiagLaunch& D, const float* rho2, const float* j2, const float mean[4],
                                    const float scale[4], float* x, cudaStream_t st) {
    FeatArgs a;
    a.nx = D.grid.nx;
    a.ny = D.grid.ny;
    a.n = (size_t)a.nx * a.ny;
    a.G = (float)D.G;
    a.gx = (float)D.gx;
    a.mirror = D.wall_mirror;
    for (int s = 0; s < 2; ++s) {
        a.gw6[s] = (float)(D.G_wall[s] / 6.0);
        a.gext[s] = (float)D.g_ext[s];
    }
    for (int c = 0; c < 4; ++c) {
        a.mean[c] = mean[c];
        a.scale[c] = scale[c];
    }
    const dim3 grid((a.nx + 127) / 128, std::min(a.ny, 65535));
    closure_features_kernel<<<grid, 128, 0, st>>>(a, rho2, j2, x);
    return cudaGetLastError();
}

size_t diag_scratch_doubles(int nx, int ny) { return (size_t)15 * nx * ny; }

size_t diag_partials_doubles(int nx, int ny) {
    const size_t gx = (nx + DX - 1) / DX, gy = (ny + BY - 1) / BY;
    return (size_t)kDiagTerms * gx * gy + (size_t)2 * ny * gx;
}

size_t diag_fields_offset(int nx, int ny) { return (size_t)6 * nx * ny; }

cudaError_t launch_diagnostics(const DiagLaunch& D, cudaStream_t st) {
    (void)cudaGetLastError();   // a launch reports only its own error
    DiagArgs a = make_args(D);
    // The velocity gradient terms of D3/D4 need u two rows outside the averaged rows and
    // u needs rho one row further out; crop >= 3 keeps all of them inside the grid.
    cudaError_t e = moments(D, a, st);
    if (e != cudaSuccess) return e;
    dim3 grid(a.nbx, (a.ny + BY - 1) / BY), block(DX, DY);
    velocity_kernel<<<grid, block, 0, st>>>(a, a.r0 - 2, a.r1 + 2, 1);
    tensor_kernel<<<grid, block, 0, st>>>(a);
    divergence_kernel<<<grid, block, 0, st>>>(a);
    reduce_kernel<<<kDiagTerms + 2 * (a.r1 - a.r0), 256, 0, st>>>(a, D.out);
    return cudaGetLastError();
}

cudaError_t launch_fields(const DiagLaunch& D, double* /*unused*/, cudaStream_t st) {
    (void)cudaGetLastError();
    DiagArgs a = make_args(D);
    cudaError_t e = moments(D, a, st);
    if (e != cudaSuccess) return e;
    dim3 grid(a.nbx, (a.ny + BY - 1) / BY), block(DX, DY);
    velocity_kernel<<<grid, block, 0, st>>>(a, 0, a.ny, 0);
    return cudaGetLastError();
}

}  // namespace lbm
