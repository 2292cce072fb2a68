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

// Double-float helpers (error-free transformations, Knuth's TwoSum and the
// FMA-based TwoProduct) used to repair the FP32 rounding of mass and momentum.
struct DF { float hi, lo; };
__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ void df_add(DF& d, float v) {
    const DF t = two_sum(d.hi, v);
    d.hi = t.hi;
    d.lo += t.lo;
}
// a * b with a double-float: (a.hi*b, err) as double-float
__device__ __forceinline__ DF df_mul(DF a, float b) {
    const float p = a.hi * b;
    return {p, fmaf(a.hi, b, -p) + a.lo * b};
}

// Forced BGK collision of one site (Section 2, Eqs. "Kinetic equation" and
// "Equilibrium distribution"): f <- f + (f^eq(rho_s, u + tau_s a_s) - f) / tau_s with
// a_s = F_s / rho_s computed directly (no division by rho_s).
//
// kExact (FP32 storage): after the BGK update, the moving populations 1..4 are
// nudged so that each component's momentum equals (1 - w) j_s + w rho_s u'_s to
// double-float accuracy, and the rest population is set to rho_s - sum_{i>0} f*_i
// (double-float).  Both are identities of the exact BGK update (it keeps rho_s and
// gives that momentum); in FP32 they remove the per-site rounding of mass and of
// the large, nearly cancelling inter-component Shan-Chen momenta, which otherwise
// random-walks the interface position (~1e-5 of rho after 1000 steps at tau = 1).
template <bool kExact>
__device__ __forceinline__ void collide_site(float f[2][9], const Nbr& psiA, const Nbr& psiB,
                                             const Physics& ph, int y, int ny, int* flag) {
    DF rr[2], jxd[2], jyd[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        if (kExact) {
            rr[s] = {f[s][0], 0.0f};
#pragma unroll
            for (int i = 1; i < 9; ++i) df_add(rr[s], f[s][i]);
            jxd[s] = {f[s][1], 0.0f};
            df_add(jxd[s], -f[s][3]); df_add(jxd[s], f[s][5]); df_add(jxd[s], -f[s][6]);
            df_add(jxd[s], f[s][8]); df_add(jxd[s], -f[s][7]);
            jyd[s] = {f[s][2], 0.0f};
            df_add(jyd[s], -f[s][4]); df_add(jyd[s], f[s][5]); df_add(jyd[s], -f[s][8]);
            df_add(jyd[s], f[s][6]); df_add(jyd[s], -f[s][7]);
        } else {
            rr[s] = {sum9(f[s]), 0.0f};
            jxd[s] = {(f[s][1] - f[s][3]) + (f[s][5] - f[s][6]) + (f[s][8] - f[s][7]), 0.0f};
            jyd[s] = {(f[s][2] - f[s][4]) + (f[s][5] - f[s][8]) + (f[s][6] - f[s][7]), 0.0f};
        }
    }
    const float rA = rr[0].hi + rr[0].lo;
    const float rB = rr[1].hi + rr[1].lo;
    if (!(rA >= 0.0f && rB >= 0.0f && rA < 1e30f && rB < 1e30f)) atomicOr(flag, 1);
    const float jx[2] = {jxd[0].hi + jxd[0].lo, jxd[1].hi + jxd[1].lo};
    const float jy[2] = {jyd[0].hi + jyd[0].lo, jyd[1].hi + jyd[1].lo};
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
        const float usq = 1.5f * (vx * vx + vy * vy);
        const float om = ph.om[s];
#pragma unroll
        for (int i = kExact ? 1 : 0; i < 9; ++i) {
            const float cu = (float)cx(i) * vx + (float)cy(i) * vy;
            const float feq = rho[s] * wf(i) * (1.0f + 3.0f * cu + 4.5f * cu * cu - usq);
            f[s][i] = f[s][i] + om * (feq - f[s][i]);
        }
        if (kExact) {
            const float om1 = 1.0f - om;
            // x: target (1 - w) jx + w rho vx, repaired on the pair 1 / 3
            {
                const DF rv = df_mul(rr[s], vx);
                const DF a = df_mul(jxd[s], om1);
                const DF b = df_mul(rv, om);
                DF t = two_sum(a.hi, b.hi);
                t.lo += a.lo + b.lo;
                DF o = {f[s][1], 0.0f};
                df_add(o, -f[s][3]); df_add(o, f[s][5]); df_add(o, -f[s][6]);
                df_add(o, f[s][8]); df_add(o, -f[s][7]);
                const float half = 0.5f * ((t.hi - o.hi) + (t.lo - o.lo));
                f[s][1] += half;
                f[s][3] -= half;
            }
            // y: pair 2 / 4
            {
                const DF rv = df_mul(rr[s], vy);
                const DF a = df_mul(jyd[s], om1);
                const DF b = df_mul(rv, om);
                DF t = two_sum(a.hi, b.hi);
                t.lo += a.lo + b.lo;
                DF o = {f[s][2], 0.0f};
                df_add(o, -f[s][4]); df_add(o, f[s][5]); df_add(o, -f[s][8]);
                df_add(o, f[s][6]); df_add(o, -f[s][7]);
                const float half = 0.5f * ((t.hi - o.hi) + (t.lo - o.lo));
                f[s][2] += half;
                f[s][4] -= half;
            }
            DF m = {f[s][1], 0.0f};
#pragma unroll
            for (int i = 2; i < 9; ++i) df_add(m, f[s][i]);
            f[s][0] = (rr[s].hi - m.hi) + (rr[s].lo - m.lo);
        }
    }
}

}  // namespace lbm
