// Collision of one site (Section 2 of arXiv 2101.04847: Eq. 1 moments,
// Shan-Chen + wall + buoyancy accelerations, forced BGK with the
// shifted-velocity equilibrium), shared by the step kernels.
#pragma once
#include "lattice.cuh"

namespace lbm {

// Neighbour sums of the pseudopotential of one component:
// (nx, ny) = sum_i w_i psi(x + c_i) c_i.
struct Nbr { float E, W, N, S, NE, NW, SE, SW; };
__device__ __forceinline__ void nbr_sum(const Nbr& r, float& sx, float& sy) {
    sx = (1.0f / 9.0f) * (r.E - r.W) + (1.0f / 36.0f) * ((r.NE - r.SW) + (r.SE - r.NW));
    sy = (1.0f / 9.0f) * (r.N - r.S) + (1.0f / 36.0f) * ((r.NE - r.SW) + (r.NW - r.SE));
}

// Common velocity u = sum_s j_s / tau_s / sum_s rho_s / tau_s (Eq. 1) and the
// accelerations a_s = F_s / rho_s: Shan-Chen coupling to the other component's
// pseudopotential, the external (buoyancy, body) accelerations and, on the wall
// rows, the fluid-boundary force.  Raises bit 0 of the guard flag for a density
// below ph.rho_floor (0 for FP32 storage) or a non-finite one.
__device__ __forceinline__ void velocity_and_accel(const float rho[2], const float jx[2], const float jy[2],
                                                   const Nbr& psiA, const Nbr& psiB, const Physics& ph, int y,
                                                   int ny, int* flag, float& ux, float& uy, float ax[2],
                                                   float ay[2]) {
    const float rA = rho[0];
    const float rB = rho[1];
    if (!(rA >= ph.rho_floor[0] && rB >= ph.rho_floor[1] && rA < 1e30f && rB < 1e30f)) atomicOr(flag, 1);
    const float inv = 1.0f / (rA * ph.om[0] + rB * ph.om[1]);
    ux = (jx[0] * ph.om[0] + jx[1] * ph.om[1]) * inv;
    uy = (jy[0] * ph.om[0] + jy[1] * ph.om[1]) * inv;
    float nAx, nAy, nBx, nBy;
    nbr_sum(psiA, nAx, nAy);
    nbr_sum(psiB, nBx, nBy);
    ax[0] = -ph.G * nBx + ph.ax_ext;
    ay[0] = -ph.G * nBy + ph.ay_ext[0];
    ax[1] = -ph.G * nAx + ph.ax_ext;
    ay[1] = -ph.G * nAy + ph.ay_ext[1];
    if (y == 0) { ay[0] += ph.ay_wall_bottom[0]; ay[1] += ph.ay_wall_bottom[1]; }
    if (y == ny - 1) { ay[0] += ph.ay_wall_top[0]; ay[1] += ph.ay_wall_top[1]; }
}

// Forced BGK collision of one site (Section 2, Eqs. "Kinetic equation" and
// "Equilibrium distribution"): f <- f + (f^eq(rho_s, u + tau_s a_s) - f) / tau_s with
// a_s = F_s / rho_s computed directly (no division by rho_s).  The equilibrium is
// evaluated per pair of opposite directions: f^eq_i + f^eq_ibar = 2 w rho (1 + 9/2 (c.u')^2
// - 3/2 u'^2) and f^eq_i - f^eq_ibar = 6 w rho c.u'.
//
// kExact (FP32 storage) works with the increments d_i = f*_i - f_i that the stored
// values really received (d_i is recomputed from the rounded f*_i; the subtraction
// is exact while |d_i| <= |f_i|, as in Dekker's Fast2Sum).  The BGK update changes a
// component's momentum by omega (rho_s u'_s - j_s) and its mass by nothing; the
// pairs 1/3 and 2/4 take half of the momentum defect each way, and the rest
// population takes minus the sum of the other eight increments.  The defects are
// sums of small increments, so their rounding is far below one unit in the last
// place of a population: mass is kept up to one rounding of f*_0 and the large,
// nearly cancelling inter-component Shan-Chen momenta do not random-walk the
// interface (plain FP32 moves rho by ~1e-5 of its range in 1000 steps at tau = 1).
template <bool kExact>
__device__ __forceinline__ void collide_site(float f[2][9], const Nbr& psiA, const Nbr& psiB,
                                             const Physics& ph, int y, int ny, int* flag) {
    float rho[2], jx[2], jy[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        rho[s] = sum9(f[s]);
        jx[s] = (f[s][1] - f[s][3]) + (f[s][5] - f[s][7]) + (f[s][8] - f[s][6]);
        jy[s] = (f[s][2] - f[s][4]) + (f[s][5] - f[s][7]) + (f[s][6] - f[s][8]);
    }
    float ux, uy, ax[2], ay[2];
    velocity_and_accel(rho, jx, jy, psiA, psiB, ph, y, ny, flag, ux, uy, ax, ay);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const float vx = ux + ph.tau[s] * ax[s];
        const float vy = uy + ph.tau[s] * ay[s];
        const float om = ph.om[s];
        const float one_minus_usq = 1.0f - 1.5f * (vx * vx + vy * vy);
        const float r9 = rho[s] * (1.0f / 9.0f);
        const float r36 = rho[s] * (1.0f / 36.0f);
        float feq[9];
        feq[0] = rho[s] * (4.0f / 9.0f) * one_minus_usq;
        {   // pairs (1,3), (2,4), (5,7), (6,8)
            const float c[4] = {vx, vy, vx + vy, vy - vx};
            const float r[4] = {r9, r9, r36, r36};
            const int a[4] = {1, 2, 5, 6}, b[4] = {3, 4, 7, 8};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float sym = r[q] * fmaf(4.5f * c[q], c[q], one_minus_usq);
                const float anti = r[q] * (3.0f * c[q]);
                feq[a[q]] = sym + anti;
                feq[b[q]] = sym - anti;
            }
        }
        if (!kExact) {
#pragma unroll
            for (int i = 0; i < 9; ++i) f[s][i] = fmaf(om, feq[i] - f[s][i], f[s][i]);
            continue;
        }
        float in[5], d[9];
#pragma unroll
        for (int i = 1; i < 5; ++i) in[i] = f[s][i];
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const float o = fmaf(om, feq[i] - f[s][i], f[s][i]);
            d[i] = o - f[s][i];
            f[s][i] = o;
        }
        const float Jx = (d[1] - d[3]) + (d[5] - d[7]) + (d[8] - d[6]);
        const float Jy = (d[2] - d[4]) + (d[5] - d[7]) + (d[6] - d[8]);
        const float hx = 0.5f * (om * fmaf(rho[s], vx, -jx[s]) - Jx);
        const float hy = 0.5f * (om * fmaf(rho[s], vy, -jy[s]) - Jy);
        f[s][1] += hx;
        f[s][3] -= hx;
        f[s][2] += hy;
        f[s][4] -= hy;
#pragma unroll
        for (int i = 1; i < 5; ++i) d[i] = f[s][i] - in[i];
        const float m = ((d[1] + d[2]) + (d[3] + d[4])) + ((d[5] + d[6]) + (d[7] + d[8]));
        f[s][0] -= m;
    }
}

// The same collision on shifted populations h_i = f_i - w_i rho0_s (16-bit
// storage), without forming f: rho_s = rho0_s + sum_i h_i, j_s = sum_i c_i h_i
// (the shift carries no momentum), and
//   f^eq_i - w_i rho0_s = w_i (rho_s - rho0_s) + w_i rho_s (9/2 (c_i.u')^2 - 3/2 u'^2 + 3 c_i.u'),
// so h_i <- h_i + (f^eq_i - w_i rho0_s - h_i) / tau_s.
__device__ __forceinline__ void collide_shifted(float h[2][9], const Nbr& psiA, const Nbr& psiB,
                                                const Physics& ph, int y, int ny, int* flag) {
    float dr[2], rho[2], jx[2], jy[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        dr[s] = sum9(h[s]);
        rho[s] = ph.shift[s] + dr[s];
        jx[s] = (h[s][1] - h[s][3]) + (h[s][5] - h[s][7]) + (h[s][8] - h[s][6]);
        jy[s] = (h[s][2] - h[s][4]) + (h[s][5] - h[s][7]) + (h[s][6] - h[s][8]);
    }
    float ux, uy, ax[2], ay[2];
    velocity_and_accel(rho, jx, jy, psiA, psiB, ph, y, ny, flag, ux, uy, ax, ay);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const float vx = ux + ph.tau[s] * ax[s];
        const float vy = uy + ph.tau[s] * ay[s];
        const float om = ph.om[s];
        const float usq = 1.5f * (vx * vx + vy * vy);
        float feq[9];
        feq[0] = (4.0f / 9.0f) * fmaf(-rho[s], usq, dr[s]);
        {   // pairs (1,3), (2,4), (5,7), (6,8)
            const float c[4] = {vx, vy, vx + vy, vy - vx};
            const float w[4] = {1.0f / 9.0f, 1.0f / 9.0f, 1.0f / 36.0f, 1.0f / 36.0f};
            const int a[4] = {1, 2, 5, 6}, b[4] = {3, 4, 7, 8};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float sym = w[q] * fmaf(rho[s], fmaf(4.5f * c[q], c[q], -usq), dr[s]);
                const float anti = (w[q] * rho[s]) * (3.0f * c[q]);
                feq[a[q]] = sym + anti;
                feq[b[q]] = sym - anti;
            }
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) h[s][i] = fmaf(om, feq[i] - h[s][i], h[s][i]);
    }
}

}  // namespace lbm
