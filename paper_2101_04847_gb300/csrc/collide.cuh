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

// Error-free transformations used to repair the FP32 rounding of mass and
// momentum: Knuth's TwoSum (any operands) and Dekker's Fast2Sum (exact when the
// running sum is at least as large as the addend, as for sums of non-negative
// populations started from the largest term).
struct DF { float hi, lo; };
__device__ __forceinline__ DF df_two(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ void df_fast_add(DF& d, float v) {
    const float s = d.hi + v;
    d.lo += v - (s - d.hi);
    d.hi = s;
}
// a - b for two double-float values
__device__ __forceinline__ DF df_sub(DF a, DF b) {
    DF s = df_two(a.hi, -b.hi);
    s.lo += a.lo - b.lo;
    return s;
}
// f[a] + f[b] + f[c] (non-negative, |f[a]| largest) in double-float
__device__ __forceinline__ DF df_sum3(float a, float b, float c) {
    DF d = {a, 0.0f};
    df_fast_add(d, b);
    df_fast_add(d, c);
    return d;
}

// Forced BGK collision of one site (Section 2, Eqs. "Kinetic equation" and
// "Equilibrium distribution"): f <- f + (f^eq(rho_s, u + tau_s a_s) - f) / tau_s with
// a_s = F_s / rho_s computed directly (no division by rho_s).  The equilibrium is
// evaluated per pair of opposite directions: f^eq_i + f^eq_ibar = 2 w rho (1 + 9/2 (c.u')^2
// - 3/2 u'^2) and f^eq_i - f^eq_ibar = 6 w rho c.u'.
//
// kExact (FP32 storage): each component's momentum after the update is summed in
// double-float (positive and negative directions separately, then their
// difference) and nudged, on the pairs 1/3 and 2/4, to (1 - w) j_s + w rho_s u'_s;
// the rest population is then set to rho_s - sum_{i>0} f*_i with both sums in
// double-float.  Both are identities of the exact BGK update (it keeps rho_s and gives
// that momentum); in FP32 they remove the per-site rounding of mass and of the
// large, nearly cancelling inter-component Shan-Chen momenta, which otherwise
// random-walks the interface (~1e-5 of rho after 1000 steps at tau = 1).
template <bool kExact>
__device__ __forceinline__ void collide_site(float f[2][9], const Nbr& psiA, const Nbr& psiB,
                                             const Physics& ph, int y, int ny, int* flag) {
    DF rr[2];
    float jx[2], jy[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        if (kExact) {
            rr[s] = {f[s][0], 0.0f};   // rest population first: the largest term
#pragma unroll
            for (int i = 1; i < 9; ++i) df_fast_add(rr[s], f[s][i]);
        } else {
            rr[s] = {sum9(f[s]), 0.0f};
        }
        jx[s] = (f[s][1] - f[s][3]) + (f[s][5] - f[s][7]) + (f[s][8] - f[s][6]);
        jy[s] = (f[s][2] - f[s][4]) + (f[s][5] - f[s][7]) + (f[s][6] - f[s][8]);
    }
    const float rA = rr[0].hi + rr[0].lo;
    const float rB = rr[1].hi + rr[1].lo;
    if (!(rA >= 0.0f && rB >= 0.0f && rA < 1e30f && rB < 1e30f)) atomicOr(flag, 1);
    const float inv = 1.0f / (rA * ph.om[0] + rB * ph.om[1]);
    const float ux = (jx[0] * ph.om[0] + jx[1] * ph.om[1]) * inv;
    const float uy = (jy[0] * ph.om[0] + jy[1] * ph.om[1]) * inv;
    float nAx, nAy, nBx, nBy;
    nbr_sum(psiA, nAx, nAy);
    nbr_sum(psiB, nBx, nBy);
    float ax[2], ay[2];
    ax[0] = -ph.G * nBx + ph.ax_ext;
    ay[0] = -ph.G * nBy + ph.ay_ext[0];
    ax[1] = -ph.G * nAx + ph.ax_ext;
    ay[1] = -ph.G * nAy + ph.ay_ext[1];
    if (y == 0) { ay[0] += ph.ay_wall_bottom[0]; ay[1] += ph.ay_wall_bottom[1]; }
    if (y == ny - 1) { ay[0] += ph.ay_wall_top[0]; ay[1] += ph.ay_wall_top[1]; }
    const float rho[2] = {rA, rB};
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
#pragma unroll
        for (int i = kExact ? 1 : 0; i < 9; ++i) f[s][i] = fmaf(om, feq[i] - f[s][i], f[s][i]);
        if (kExact) {
            const float om1 = 1.0f - om;
            // x: target (1 - w) jx + w rho vx, repaired on the pair 1 / 3
            {
                const float t = fmaf(om1, jx[s], om * (rho[s] * vx));
                const DF o = df_sub(df_sum3(f[s][1], f[s][5], f[s][8]), df_sum3(f[s][3], f[s][7], f[s][6]));
                const float half = 0.5f * ((t - o.hi) - o.lo);
                f[s][1] += half;
                f[s][3] -= half;
            }
            // y: pair 2 / 4
            {
                const float t = fmaf(om1, jy[s], om * (rho[s] * vy));
                const DF o = df_sub(df_sum3(f[s][2], f[s][5], f[s][6]), df_sum3(f[s][4], f[s][7], f[s][8]));
                const float half = 0.5f * ((t - o.hi) - o.lo);
                f[s][2] += half;
                f[s][4] -= half;
            }
            DF m = {f[s][1], 0.0f};    // axis directions (weight 1/9) before the diagonals
#pragma unroll
            for (int i = 2; i < 9; ++i) df_fast_add(m, f[s][i]);
            f[s][0] = (rr[s].hi - m.hi) + (rr[s].lo - m.lo);
        }
    }
}

}  // namespace lbm
