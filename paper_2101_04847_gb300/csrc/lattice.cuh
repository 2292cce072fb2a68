// Device helpers shared by the kernels of liblbm: storage conversion of the
// populations and the pull of the post-streaming populations of one site.
// A buffer B holds post-collision populations in structure-of-arrays layout
// [component][direction][y][pitch]; the post-streaming population of the kinetic
// equation (Section 2 of arXiv 2101.04847) is
//     S_i(x, y) = B_i(x - c_ix, y - c_iy)   if 0 <= y - c_iy < ny  (x periodic)
//     S_i(x, y) = B_opp(i)(x, y)            otherwise (half-way bounce-back)
#pragma once
#include "lbm_internal.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// storage types: float, or half / bfloat16 holding f - w_i rho0_s
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

template <typename T> struct IsShifted { static constexpr bool value = true; };
template <> struct IsShifted<float> { static constexpr bool value = false; };

template <typename T>
__device__ __forceinline__ float load_pop(const T* p, int i, float shift_s) {
    float v = to_f<T>(__ldg(p));
    if (IsShifted<T>::value) v += wf(i) * shift_s;
    return v;
}

// Pull the 18 post-streaming populations of column xc (neighbours xm, xp) on row y.
template <typename T>
__device__ __forceinline__ void pull_site(const T* __restrict__ fin, const Grid& g, const float shift[2],
                                          int y, int xc, int xm, int xp, float f[2][9]) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int sy = y - cy(i);
            const int sx = cx(i) == 0 ? xc : (cx(i) == 1 ? xm : xp);
            const bool inside = (cy(i) == 0) || (sy >= 0 && sy < g.ny);
            const size_t idx = inside
                ? (size_t)(s * 9 + i) * g.plane + (size_t)sy * g.pitch + g.origin + sx
                : (size_t)(s * 9 + opp(i)) * g.plane + (size_t)y * g.pitch + g.origin + xc;
            f[s][i] = load_pop<T>(fin + idx, i, shift[s]);
        }
    }
}

// Store the 18 post-collision values of column x on row y, plus the periodic ghost
// copy of the two first / last columns (read by the staged kernels' row windows).
// The ghost copies take a separate branch, taken only by threads of edge columns.
template <typename T>
__device__ __forceinline__ void store_site(T* __restrict__ fout, const Grid& g, int y, int x,
                                           const float f[2][9], const float shift[2]) {
    T* q = fout + (size_t)y * g.pitch + g.origin + x;
    T tv[2][9];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            float v = f[s][i];
            if (IsShifted<T>::value) v -= wf(i) * shift[s];
            tv[s][i] = from_f<T>(v);
            q[(size_t)(s * 9 + i) * g.plane] = tv[s][i];
        }
    }
    if (x < 2 || x >= g.nx - 2) {
        T* qg = q + (x < 2 ? g.nx : -g.nx);
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int i = 0; i < 9; ++i) qg[(size_t)(s * 9 + i) * g.plane] = tv[s][i];
    }
}

// ---------------------------------------------------------------------------
// Stochastic rounding of the 16-bit stores.  Rounding to nearest lets slowly
// varying populations round the same way step after step, which drifts the
// masses by several per cent over 10^4 steps.  A value is instead rounded up in
// magnitude with probability equal to its distance from the lower neighbour, in
// units of the spacing: uniform random bits are added below the kept mantissa of
// the FP32 pattern and the sum is truncated.  The random bits are a hash of the
// site, the component and the time step (lowbias32 of C. Wellons' hash
// prospector; a counter-based generator, so results are reproducible), stepped
// by the PCG multiplier of M. E. O'Neill per value.  The time step matters: a
// hash of the values alone repeats its decisions in slowly varying regions and
// drifts the masses by ~1e-4 per 5000 steps.  FP16 subnormals (|h| < 2^-14) keep
// a truncation bias below 2^-24.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t hash_lowbias32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}
// Seed of a launch's stochastic rounding: a hash of its time step (0 without a counter).
__device__ __forceinline__ uint32_t launch_seed(const Physics& ph) {
    return ph.step_in ? hash_lowbias32(*ph.step_in * 0x9E3779B9u + 0x7F4A7C15u) : 0u;
}
// The one thread `leader` of a launch passes the time step on to the next launch.
__device__ __forceinline__ void advance_step(const Physics& ph, bool leader) {
    if (leader && ph.step_out) *ph.step_out = *ph.step_in + 1u;
}

template <typename T> __device__ __forceinline__ T round_stochastic(float v, uint32_t r);
template <> __device__ __forceinline__ __half round_stochastic<__half>(float v, uint32_t r) {
    return __float2half_rz(__uint_as_float(__float_as_uint(v) + (r >> 19)));   // 13 bits dropped
}
template <> __device__ __forceinline__ __nv_bfloat16 round_stochastic<__nv_bfloat16>(float v, uint32_t r) {
    return __float2bfloat16_rz(__uint_as_float(__float_as_uint(v) + (r >> 16)));   // 16 bits dropped
}

// Store the 18 shifted values h of column x on row y (16-bit storage: h is what is
// stored, no shift applied here), stochastically rounded, plus the periodic ghost
// copy of the two first / last columns.
template <typename T>
__device__ __forceinline__ void store_site_sr(T* __restrict__ fout, const Grid& g, int y, int x,
                                              const float h[2][9], uint32_t seed) {
    T* q = fout + (size_t)y * g.pitch + g.origin + x;
    T tv[2][9];
    // the site's index in the whole grid, so that a split grid draws the same bits
    const uint32_t site = g.nx_total > 0 ? (uint32_t)y * (uint32_t)g.nx_total + (uint32_t)(g.x_offset + x)
                                         : (uint32_t)y * (uint32_t)g.nx + (uint32_t)x;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        uint32_t r = hash_lowbias32((site * 2u + (uint32_t)s) ^ seed);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            r = r * 747796405u + 2891336453u;
            tv[s][i] = round_stochastic<T>(h[s][i], r);
            q[(size_t)(s * 9 + i) * g.plane] = tv[s][i];
        }
    }
    if (x < 2 || x >= g.nx - 2) {
        T* qg = q + (x < 2 ? g.nx : -g.nx);
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int i = 0; i < 9; ++i) qg[(size_t)(s * 9 + i) * g.plane] = tv[s][i];
    }
}

// Store of a time step's result f: FP32 storage as it is; 16-bit storage as
// h = f - w_i rho0_s with the stochastic rounding above.
template <typename T>
__device__ __forceinline__ void store_step(T* __restrict__ fout, const Grid& g, int y, int x, const float f[2][9],
                                           const float shift[2], uint32_t seed) {
    if constexpr (IsShifted<T>::value) {
        float h[2][9];
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int i = 0; i < 9; ++i) h[s][i] = f[s][i] - wf(i) * shift[s];
        store_site_sr<T>(fout, g, y, x, h, seed);
    } else {
        store_site<T>(fout, g, y, x, f, shift);
    }
}

__device__ __forceinline__ float sum9(const float* f) {
    return ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
}

}  // namespace lbm
