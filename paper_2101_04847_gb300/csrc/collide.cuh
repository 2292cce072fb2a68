// Collision of one site (Section 2 of arXiv 2101.04847: Eq. 1 moments,
// Shan-Chen + wall + buoyancy accelerations, forced BGK with the
// shifted-velocity equilibrium), shared by the step kernels.
//
// The two components are processed as the two lanes of float2 values with the
// packed FP32 instructions of this architecture (FADD2 / FMUL2 / FFMA2: two IEEE
// round-to-nearest operations in one instruction): the collision is the same
// arithmetic for component A (lane x) and component B (lane y).  A difference
// a - b is one FFMA2, b * (-1) + a, which rounds like the subtraction.
#pragma once
#include "lattice.cuh"

namespace lbm {

__device__ __forceinline__ float2 splat(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Neighbour sums of the pseudopotential of one component:
// (nx, ny) = sum_i w_i psi(x + c_i) c_i.
struct Nbr { float E, W, N, S, NE, NW, SE, SW; };

// Both components' neighbour sums, lane x from a, lane y from b.
__device__ __forceinline__ void nbr_sum2(const Nbr& a, const Nbr& b, float2& sx, float2& sy) {
    const float2 E = make_float2(a.E, b.E), W = make_float2(a.W, b.W);
    const float2 N = make_float2(a.N, b.N), S = make_float2(a.S, b.S);
    const float2 NE = make_float2(a.NE, b.NE), NW = make_float2(a.NW, b.NW);
    const float2 SE = make_float2(a.SE, b.SE), SW = make_float2(a.SW, b.SW);
    const float2 d = sub2(NE, SW);
    sx = fma2(splat(1.0f / 9.0f), sub2(E, W), mul2(splat(1.0f / 36.0f), add2(d, sub2(SE, NW))));
    sy = fma2(splat(1.0f / 9.0f), sub2(N, S), mul2(splat(1.0f / 36.0f), add2(d, sub2(NW, SE))));
}

// Common velocity u = sum_s j_s / tau_s / sum_s rho_s / tau_s (Eq. 1) and the
// accelerations a_s = F_s / rho_s: Shan-Chen coupling to the other component's
// pseudopotential, the external (buoyancy, body) accelerations and, on the wall
// rows, the fluid-boundary force.  Raises bit 0 of the guard flag for a density
// below ph.rho_floor (0 for FP32 storage) or a non-finite one.
__device__ __forceinline__ void velocity_and_accel(float2 rho, float2 jx, float2 jy, const Nbr& psiA,
                                                   const Nbr& psiB, const Physics& ph, int y, int ny, int* flag,
                                                   float& ux, float& uy, float2& ax, float2& ay) {
    if (!(rho.x >= ph.rho_floor[0] && rho.y >= ph.rho_floor[1] && rho.x < 1e30f && rho.y < 1e30f))
        atomicOr(flag, 1);
    const float inv = 1.0f / (rho.x * ph.om[0] + rho.y * ph.om[1]);
    ux = (jx.x * ph.om[0] + jx.y * ph.om[1]) * inv;
    uy = (jy.x * ph.om[0] + jy.y * ph.om[1]) * inv;
    // lane x of the sums: A's neighbours, which act on B (and the other way round)
    float2 sx, sy;
    nbr_sum2(psiB, psiA, sx, sy);
    ax = fma2(splat(-ph.G), sx, splat(ph.ax_ext));
    ay = fma2(splat(-ph.G), sy, make_float2(ph.ay_ext[0], ph.ay_ext[1]));
    if (y == 0) ay = add2(ay, make_float2(ph.ay_wall_bottom[0], ph.ay_wall_bottom[1]));
    if (y == ny - 1) ay = add2(ay, make_float2(ph.ay_wall_top[0], ph.ay_wall_top[1]));
    if (ph.wall_mirror && (y == 0 || y == ny - 1)) {
        // wall_mode 1: the virtual row beyond the wall holds this row's pseudopotentials
        // (the kernels passed zeros for it).  Its three neighbours add w c psi: the
        // straight one the other component's density here, the diagonals those at x + 1
        // and x - 1, i.e. (1/9) psi' + (1/36)(E' + W') along the outward normal and
        // (1/36)(E' - W') along x.
        const float2 own = make_float2(rho.y, rho.x);
        const float2 E = make_float2(psiB.E, psiA.E), W = make_float2(psiB.W, psiA.W);
        const float2 dn = fma2(splat(1.0f / 9.0f), own, mul2(splat(1.0f / 36.0f), add2(E, W)));
        const float2 dx = mul2(splat(1.0f / 36.0f), sub2(E, W));
        ax = fma2(splat(-ph.G), dx, ax);
        ay = fma2(splat(y == 0 ? ph.G : -ph.G), dn, ay);
    }
}

// sum of nine values, associated as ((0+1)+(2+3)) + ((4+5)+(6+7)) + 8
__device__ __forceinline__ float2 sum9_2(const float2* f) {
    const float2 lo = add2(add2(f[0], f[1]), add2(f[2], f[3]));
    const float2 hi = add2(add2(f[4], f[5]), add2(f[6], f[7]));
    return add2(add2(lo, hi), f[8]);
}
// momenta (1 - 3) + (5 - 7) + (8 - 6) and (2 - 4) + (5 - 7) + (6 - 8)
__device__ __forceinline__ float2 momx2(const float2* f) {
    return add2(add2(sub2(f[1], f[3]), sub2(f[5], f[7])), sub2(f[8], f[6]));
}
__device__ __forceinline__ float2 momy2(const float2* f) {
    return add2(add2(sub2(f[2], f[4]), sub2(f[5], f[7])), sub2(f[6], f[8]));
}

// Equilibrium part shared by both collisions: feq_i = base_i + w_i rho u-terms,
// evaluated per pair of opposite directions (1,3), (2,4), (5,7), (6,8):
// f^eq_i + f^eq_ibar = 2 w (base + rho (9/2 (c.u')^2 - 3/2 u'^2)) and
// f^eq_i - f^eq_ibar = 6 w rho c.u'.  `k0` is the rest term, `sym(q, c)` the
// symmetric part of pair q.
template <typename Sym>
__device__ __forceinline__ void pairs2(float2 vx, float2 vy, float2 rho, Sym sym, float2 feq[9]) {
    const float2 c[4] = {vx, vy, add2(vx, vy), sub2(vy, vx)};
    const float w[4] = {1.0f / 9.0f, 1.0f / 9.0f, 1.0f / 36.0f, 1.0f / 36.0f};
    const int a[4] = {1, 2, 5, 6}, b[4] = {3, 4, 7, 8};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float2 s = sym(q, c[q]);
        const float2 anti = mul2(mul2(splat(w[q]), rho), mul2(splat(3.0f), c[q]));
        feq[a[q]] = add2(s, anti);
        feq[b[q]] = sub2(s, anti);
    }
}

// Forced BGK collision of one site (Section 2, Eqs. "Kinetic equation" and
// "Equilibrium distribution"): f <- f + (f^eq(rho_s, u + tau_s a_s) - f) / tau_s with
// a_s = F_s / rho_s computed directly (no division by rho_s).
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
    float2 F[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) F[i] = make_float2(f[0][i], f[1][i]);
    const float2 rho = sum9_2(F);
    const float2 jx = momx2(F), jy = momy2(F);
    float ux, uy;
    float2 ax, ay;
    velocity_and_accel(rho, jx, jy, psiA, psiB, ph, y, ny, flag, ux, uy, ax, ay);
    const float2 tau = make_float2(ph.tau[0], ph.tau[1]);
    const float2 om = make_float2(ph.om[0], ph.om[1]);
    const float2 vx = fma2(tau, ax, splat(ux));
    const float2 vy = fma2(tau, ay, splat(uy));
    // 1 - 3/2 u'^2
    const float2 omu = fma2(splat(-1.5f), fma2(vx, vx, mul2(vy, vy)), splat(1.0f));
    float2 feq[9];
    feq[0] = mul2(mul2(rho, splat(4.0f / 9.0f)), omu);
    const float2 r9 = mul2(rho, splat(1.0f / 9.0f)), r36 = mul2(rho, splat(1.0f / 36.0f));
    pairs2(vx, vy, rho,
           [&](int q, float2 c) { return mul2(q < 2 ? r9 : r36, fma2(mul2(splat(4.5f), c), c, omu)); }, feq);
    if (!kExact) {
#pragma unroll
        for (int i = 0; i < 9; ++i) F[i] = fma2(om, sub2(feq[i], F[i]), F[i]);
    } else {
        float2 in[5], d[9];
#pragma unroll
        for (int i = 1; i < 5; ++i) in[i] = F[i];
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const float2 o = fma2(om, sub2(feq[i], F[i]), F[i]);
            d[i] = sub2(o, F[i]);
            F[i] = o;
        }
        const float2 Jx = momx2(d), Jy = momy2(d);
        // (om (rho u' - j) - J) / 2, with om / 2 and -J / 2 exact scalings
        const float2 omh = mul2(om, splat(0.5f));
        const float2 hx = fma2(omh, fma2(rho, vx, mul2(jx, splat(-1.0f))), mul2(Jx, splat(-0.5f)));
        const float2 hy = fma2(omh, fma2(rho, vy, mul2(jy, splat(-1.0f))), mul2(Jy, splat(-0.5f)));
        F[1] = add2(F[1], hx);
        F[3] = sub2(F[3], hx);
        F[2] = add2(F[2], hy);
        F[4] = sub2(F[4], hy);
#pragma unroll
        for (int i = 1; i < 5; ++i) d[i] = sub2(F[i], in[i]);
        const float2 m = add2(add2(add2(d[1], d[2]), add2(d[3], d[4])), add2(add2(d[5], d[6]), add2(d[7], d[8])));
        F[0] = sub2(F[0], m);
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        f[0][i] = F[i].x;
        f[1][i] = F[i].y;
    }
}

// The same collision on shifted populations h_i = f_i - w_i rho0_s (16-bit
// storage), without forming f: rho_s = rho0_s + sum_i h_i, j_s = sum_i c_i h_i
// (the shift carries no momentum), and
//   f^eq_i - w_i rho0_s = w_i (rho_s - rho0_s) + w_i rho_s (9/2 (c_i.u')^2 - 3/2 u'^2 + 3 c_i.u'),
// so h_i <- h_i + (f^eq_i - w_i rho0_s - h_i) / tau_s.
__device__ __forceinline__ void collide_shifted(float h[2][9], const Nbr& psiA, const Nbr& psiB,
                                                const Physics& ph, int y, int ny, int* flag) {
    float2 H[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) H[i] = make_float2(h[0][i], h[1][i]);
    const float2 dr = sum9_2(H);
    const float2 rho = add2(make_float2(ph.shift[0], ph.shift[1]), dr);
    const float2 jx = momx2(H), jy = momy2(H);
    float ux, uy;
    float2 ax, ay;
    velocity_and_accel(rho, jx, jy, psiA, psiB, ph, y, ny, flag, ux, uy, ax, ay);
    const float2 tau = make_float2(ph.tau[0], ph.tau[1]);
    const float2 om = make_float2(ph.om[0], ph.om[1]);
    const float2 vx = fma2(tau, ax, splat(ux));
    const float2 vy = fma2(tau, ay, splat(uy));
    const float2 usq = mul2(splat(1.5f), fma2(vx, vx, mul2(vy, vy)));
    const float2 mrho = mul2(rho, splat(-1.0f));
    float2 feq[9];
    feq[0] = mul2(splat(4.0f / 9.0f), fma2(mrho, usq, dr));
    pairs2(vx, vy, rho,
           [&](int q, float2 c) {
               const float w = q < 2 ? 1.0f / 9.0f : 1.0f / 36.0f;
               return mul2(splat(w), fma2(rho, fma2(mul2(splat(4.5f), c), c, mul2(usq, splat(-1.0f))), dr));
           },
           feq);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        H[i] = fma2(om, sub2(feq[i], H[i]), H[i]);
        h[0][i] = H[i].x;
        h[1][i] = H[i].y;
    }
}

}  // namespace lbm
