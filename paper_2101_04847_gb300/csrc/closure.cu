// Learned closure for a 2x-coarsened run.  The paper has no such component;
// it is built on the plain solver as an extension: a small CNN (conv3x3 4->32,
// ReLU, conv3x3 32->32, ReLU, conv3x3 32->4; x periodic, zero padding beyond the
// walls) reads the coarse fields (rho_A, rho_B, u_x, u_y) every `interval` coarse
// steps and predicts their correction toward the restricted fields of a run on
// the 2x finer grid.  Weights are BF16 in the convolutions, activations and
// accumulation FP32; training (forward, backward, Adam) runs in the kernels below.
//
// Coarse parameters (diffusive scaling: dx_c = 2 dx, dt_c = 4 dt): nx/2, ny/2,
// the same tau (hence the same kinematic viscosity and, since the Shan-Chen phase
// behaviour depends on tau, the same miscibility), same G, masses and wall
// coupling, g_c = 8 g; lattice velocities double (u_c = 2 u).  Acoustic scaling
// (tau_c = 1/2 + (tau - 1/2)/2) would move the coarse mixture deeper into the
// immiscible regime and drive its minority densities negative.
#include "lattice.cuh"
#include "cnn_tc.cuh"

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

namespace lbm {
namespace cnn {

constexpr int kHid = 32, kIn = 4, kOut = 4;
constexpr int kW1 = 0, kB1 = kW1 + kHid * kIn * 9;
constexpr int kW2 = kB1 + kHid, kB2 = kW2 + kHid * kHid * 9;
constexpr int kW3 = kB2 + kHid, kB3 = kW3 + kOut * kHid * 9;
constexpr int kParams = kB3 + kOut;   // 11588
constexpr int kTile = 16;
constexpr int kChunk = 2048;          // pixels per weight-gradient block

static_assert(kParams == 11588, "parameter count");

__device__ __forceinline__ int wrapx(int x, int nx) { return x < 0 ? x + nx : (x >= nx ? x - nx : x); }

// Load a (kTile+2)^2 tile of CH channels starting at channel c0 into smem
// (periodic in x, zeros beyond the walls in y).
template <int CH>
__device__ __forceinline__ void load_tile(float (*s)[kTile + 2][kTile + 2], const float* __restrict__ a, int c0, int cmax,
                                          int nx, int ny) {
    const int tid = threadIdx.y * kTile + threadIdx.x;
    const size_t n = (size_t)nx * ny;
    for (int i = tid; i < CH * (kTile + 2) * (kTile + 2); i += kTile * kTile) {
        const int c = i / ((kTile + 2) * (kTile + 2));
        const int r = i % ((kTile + 2) * (kTile + 2));
        const int yy = r / (kTile + 2), xx = r % (kTile + 2);
        const int gy = blockIdx.y * kTile + yy - 1;
        const int gx = wrapx((int)(blockIdx.x * kTile) + xx - 1, nx);
        float v = 0.0f;
        if (c0 + c < cmax && gy >= 0 && gy < ny && gx < nx) v = a[(size_t)(c0 + c) * n + (size_t)gy * nx + gx];
        s[c][yy][xx] = v;
    }
}

// out[o, y, x] = b[o] + sum_{c, dy, dx} w[o, c, dy+1, dx+1] in[c, y+dy, x+dx]  (optional ReLU)
template <int CIN, int COUT, bool RELU>
__global__ void __launch_bounds__(kTile * kTile)
conv_fwd_kernel(const float* __restrict__ in, const __nv_bfloat16* __restrict__ w, const float* __restrict__ b,
                float* __restrict__ out, int nx, int ny) {
    constexpr int CH = CIN < 8 ? CIN : 8;
    __shared__ float sw[COUT * CIN * 9];
    __shared__ float st[CH][kTile + 2][kTile + 2];
    const int tid = threadIdx.y * kTile + threadIdx.x;
    for (int i = tid; i < COUT * CIN * 9; i += kTile * kTile) sw[i] = __bfloat162float(w[i]);
    const int x = blockIdx.x * kTile + threadIdx.x, y = blockIdx.y * kTile + threadIdx.y;
    float acc[COUT];
#pragma unroll
    for (int o = 0; o < COUT; ++o) acc[o] = b[o];
    for (int c0 = 0; c0 < CIN; c0 += CH) {
        __syncthreads();
        load_tile<CH>(st, in, c0, CIN, nx, ny);
        __syncthreads();
#pragma unroll
        for (int c = 0; c < CH; ++c)
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const float v = st[c][threadIdx.y + k / 3][threadIdx.x + k % 3];
#pragma unroll
                for (int o = 0; o < COUT; ++o) acc[o] = fmaf(sw[(o * CIN + c0 + c) * 9 + k], v, acc[o]);
            }
    }
    if (x < nx && y < ny) {
        const size_t n = (size_t)nx * ny;
#pragma unroll
        for (int o = 0; o < COUT; ++o) out[(size_t)o * n + (size_t)y * nx + x] = RELU ? fmaxf(acc[o], 0.0f) : acc[o];
    }
}

// din[c, y, x] = sum_{o, dy, dx} w[o, c, dy+1, dx+1] dout[o, y-dy, x-dx]; times (act[c] > 0) if MASK
template <int CIN, int COUT, bool MASK>
__global__ void __launch_bounds__(kTile * kTile)
conv_bwd_data_kernel(const float* __restrict__ dout, const __nv_bfloat16* __restrict__ w, const float* __restrict__ act,
                     float* __restrict__ din, int nx, int ny) {
    constexpr int CH = COUT < 8 ? COUT : 8;
    __shared__ float sw[COUT * CIN * 9];
    __shared__ float st[CH][kTile + 2][kTile + 2];
    const int tid = threadIdx.y * kTile + threadIdx.x;
    for (int i = tid; i < COUT * CIN * 9; i += kTile * kTile) sw[i] = __bfloat162float(w[i]);
    const int x = blockIdx.x * kTile + threadIdx.x, y = blockIdx.y * kTile + threadIdx.y;
    float acc[CIN];
#pragma unroll
    for (int c = 0; c < CIN; ++c) acc[c] = 0.0f;
    for (int o0 = 0; o0 < COUT; o0 += CH) {
        __syncthreads();
        load_tile<CH>(st, dout, o0, COUT, nx, ny);
        __syncthreads();
#pragma unroll 1
        for (int o = 0; o < CH; ++o)
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                // dout at (y - dy, x - dx) with dy = k/3 - 1, dx = k%3 - 1
                const float g = st[o][threadIdx.y + 2 - k / 3][threadIdx.x + 2 - k % 3];
#pragma unroll
                for (int c = 0; c < CIN; ++c) acc[c] = fmaf(sw[((o0 + o) * CIN + c) * 9 + k], g, acc[c]);
            }
    }
    if (x < nx && y < ny) {
        const size_t n = (size_t)nx * ny;
#pragma unroll
        for (int c = 0; c < CIN; ++c) {
            const size_t k = (size_t)c * n + (size_t)y * nx + x;
            din[k] = MASK ? (act[k] > 0.0f ? acc[c] : 0.0f) : acc[c];
        }
    }
}

// Partial weight / bias gradients of one (o, c) pair over one chunk of pixels:
// part[((p * COUT + o) * CIN + c) * 10 + k] (k < 9: weight tap, 9: bias when c == 0)
template <int CIN, int COUT>
__global__ void __launch_bounds__(256)
conv_bwd_weight_kernel(const float* __restrict__ in, const float* __restrict__ dout, float* __restrict__ part, int nx,
                       int ny) {
    const int o = blockIdx.x / CIN, c = blockIdx.x % CIN, p = blockIdx.y;
    const size_t n = (size_t)nx * ny;
    const size_t p0 = (size_t)p * kChunk, p1 = min(n, p0 + kChunk);
    float s[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) s[k] = 0.0f;
    const float* a = in + (size_t)c * n;
    const float* g = dout + (size_t)o * n;
    for (size_t q = p0 + threadIdx.x; q < p1; q += 256) {
        const int y = (int)(q / nx), x = (int)(q % nx);
        const float gv = g[q];
        s[9] += gv;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int yy = y + k / 3 - 1;
            const int xx = wrapx(x + k % 3 - 1, nx);
            const float v = (yy >= 0 && yy < ny) ? a[(size_t)yy * nx + xx] : 0.0f;
            s[k] = fmaf(gv, v, s[k]);
        }
    }
    __shared__ float red[8][10];
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        float v = s[k];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 10) {
        float v = 0.0f;
        for (int wdx = 0; wdx < 8; ++wdx) v += red[wdx][threadIdx.x];
        part[(((size_t)p * COUT + o) * CIN + c) * 10 + threadIdx.x] = v;
    }
}

// Sum the chunk partials into the gradient vector (fixed order).
template <int CIN, int COUT>
__global__ void reduce_weight_kernel(const float* __restrict__ part, int P, float* __restrict__ gw, float* __restrict__ gb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < COUT * CIN * 9) {
        const int o = i / (CIN * 9), c = (i / 9) % CIN, k = i % 9;
        float v = 0.0f;
        for (int p = 0; p < P; ++p) v += part[(((size_t)p * COUT + o) * CIN + c) * 10 + k];
        gw[i] = v;
    } else if (i < COUT * CIN * 9 + COUT) {
        const int o = i - COUT * CIN * 9;
        float v = 0.0f;
        for (int p = 0; p < P; ++p) v += part[(((size_t)p * COUT + o) * CIN + 0) * 10 + 9];
        gb[o] = v;
    }
}

// d = 2 (y - t) / m and per-block partial sums of (y - t)^2 (double)
__global__ void loss_grad_kernel(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ d,
                                 double* __restrict__ part, size_t m) {
    __shared__ double red[8];
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x) {
        const float e = y[i] - t[i];
        d[i] = 2.0f * e / (float)m;
        s += (double)e * e;
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v += red[k];
        part[blockIdx.x] = v;
    }
}

__global__ void to_bf16_kernel(const float* __restrict__ p, __nv_bfloat16* __restrict__ q, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) q[i] = __float2bfloat16_rn(p[i]);
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1t, float b2t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.0f - b1t), vh = vi / (1.0f - b2t);
    p[i] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

// ------------------------------------------------------------------ workspace
struct Net {
    int nx, ny;
    size_t n;
    __nv_bfloat16* wb;
    float *a1, *a2, *y, *dy, *dz2, *dz1, *part;
    double* lpart;
    int P;
    cnn_tc::Bufs tc;   // tensor-core inference
};

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// FP32 forward/backward buffers, then the tensor-core inference planes
size_t training_bytes(int nx, int ny) {
    const size_t n = (size_t)nx * ny;
    const size_t P = (n + kChunk - 1) / kChunk;
    size_t b = align256(kParams * sizeof(__nv_bfloat16));
    b += align256(kHid * n * 4) * 2 + align256(kOut * n * 4) * 2 + align256(kHid * n * 4) * 2;
    b += align256(P * kHid * kHid * 10 * 4);
    b += align256(1024 * sizeof(double));
    return b;
}

size_t workspace_bytes(int nx, int ny) { return training_bytes(nx, ny) + cnn_tc::bytes(nx, ny); }

Net carve(void* ws, int nx, int ny) {
    Net N;
    N.nx = nx;
    N.ny = ny;
    N.n = (size_t)nx * ny;
    N.P = (int)((N.n + kChunk - 1) / kChunk);
    char* p = (char*)ws;
    N.wb = (__nv_bfloat16*)p; p += align256(kParams * sizeof(__nv_bfloat16));
    N.a1 = (float*)p; p += align256(kHid * N.n * 4);
    N.a2 = (float*)p; p += align256(kHid * N.n * 4);
    N.y = (float*)p; p += align256(kOut * N.n * 4);
    N.dy = (float*)p; p += align256(kOut * N.n * 4);
    N.dz2 = (float*)p; p += align256(kHid * N.n * 4);
    N.dz1 = (float*)p; p += align256(kHid * N.n * 4);
    N.part = (float*)p; p += align256((size_t)N.P * kHid * kHid * 10 * 4);
    N.lpart = (double*)p;
    N.tc = cnn_tc::carve((char*)ws + training_bytes(nx, ny), nx, ny);
    return N;
}

cudaError_t forward(const Net& N, const float* params, const float* x, float* y, cudaStream_t st) {
    to_bf16_kernel<<<(kParams + 255) / 256, 256, 0, st>>>(params, N.wb, kParams);
    dim3 grid((N.nx + kTile - 1) / kTile, (N.ny + kTile - 1) / kTile), blk(kTile, kTile);
    conv_fwd_kernel<kIn, kHid, true><<<grid, blk, 0, st>>>(x, N.wb + kW1, params + kB1, N.a1, N.nx, N.ny);
    conv_fwd_kernel<kHid, kHid, true><<<grid, blk, 0, st>>>(N.a1, N.wb + kW2, params + kB2, N.a2, N.nx, N.ny);
    conv_fwd_kernel<kHid, kOut, false><<<grid, blk, 0, st>>>(N.a2, N.wb + kW3, params + kB3, y, N.nx, N.ny);
    return cudaGetLastError();
}

// forward + loss + backward; grad gets dL/dparams, lpart[0..nb) the loss partials
cudaError_t loss_grad(const Net& N, const float* params, const float* x, const float* t, float* grad, int* nb_out,
                      cudaStream_t st) {
    cudaError_t e = forward(N, params, x, N.y, st);
    if (e != cudaSuccess) return e;
    const size_t m = kOut * N.n;
    const int nb = (int)std::min<size_t>(1024, (m + 255) / 256);
    loss_grad_kernel<<<nb, 256, 0, st>>>(N.y, t, N.dy, N.lpart, m);
    *nb_out = nb;
    dim3 grid((N.nx + kTile - 1) / kTile, (N.ny + kTile - 1) / kTile), blk(kTile, kTile);
    // layer 3
    conv_bwd_weight_kernel<kHid, kOut><<<dim3(kOut * kHid, N.P), 256, 0, st>>>(N.a2, N.dy, N.part, N.nx, N.ny);
    reduce_weight_kernel<kHid, kOut><<<(kOut * kHid * 9 + kOut + 255) / 256, 256, 0, st>>>(N.part, N.P, grad + kW3, grad + kB3);
    conv_bwd_data_kernel<kHid, kOut, true><<<grid, blk, 0, st>>>(N.dy, N.wb + kW3, N.a2, N.dz2, N.nx, N.ny);
    // layer 2
    conv_bwd_weight_kernel<kHid, kHid><<<dim3(kHid * kHid, N.P), 256, 0, st>>>(N.a1, N.dz2, N.part, N.nx, N.ny);
    reduce_weight_kernel<kHid, kHid><<<(kHid * kHid * 9 + kHid + 255) / 256, 256, 0, st>>>(N.part, N.P, grad + kW2, grad + kB2);
    conv_bwd_data_kernel<kHid, kHid, true><<<grid, blk, 0, st>>>(N.dz2, N.wb + kW2, N.a1, N.dz1, N.nx, N.ny);
    // layer 1
    conv_bwd_weight_kernel<kIn, kHid><<<dim3(kHid * kIn, N.P), 256, 0, st>>>(x, N.dz1, N.part, N.nx, N.ny);
    reduce_weight_kernel<kIn, kHid><<<(kHid * kIn * 9 + kHid + 255) / 256, 256, 0, st>>>(N.part, N.P, grad + kW1, grad + kB1);
    return cudaGetLastError();
}

}  // namespace cnn

// ------------------------------------------------------------------ field kernels
namespace {

// 2x2 block means of the fine fields: densities averaged, velocity momentum-weighted
// and expressed in coarse lattice units
__global__ void restrict_kernel(const double* __restrict__ rA, const double* __restrict__ rB,
                                const double* __restrict__ ux, const double* __restrict__ uy, int nxf,
                                float* __restrict__ out, int ncx, int ncy) {
    const int X = blockIdx.x * blockDim.x + threadIdx.x, Y = blockIdx.y;
    if (X >= ncx || Y >= ncy) return;
    double sA = 0, sB = 0, jx = 0, jy = 0;
    for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
            const size_t k = (size_t)(2 * Y + dy) * nxf + 2 * X + dx;
            const double r = rA[k] + rB[k];
            sA += rA[k];
            sB += rB[k];
            jx += r * ux[k];
            jy += r * uy[k];
        }
    const size_t nc = (size_t)ncx * ncy, k = (size_t)Y * ncx + X;
    out[k] = (float)(0.25 * sA);
    out[nc + k] = (float)(0.25 * sB);
    out[2 * nc + k] = (float)(2.0 * jx / (sA + sB));   // coarse lattice velocity = 2 x fine
    out[3 * nc + k] = (float)(2.0 * jy / (sA + sB));
}

// the coarse fields of a handle (doubles in its scratch) as floats
__global__ void fields_to_float_kernel(const double* __restrict__ rA, const double* __restrict__ rB,
                                       const double* __restrict__ ux, const double* __restrict__ uy, size_t n,
                                       float* __restrict__ out) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        out[k] = (float)rA[k];
        out[n + k] = (float)rB[k];
        out[2 * n + k] = (float)ux[k];
        out[3 * n + k] = (float)uy[k];
    }
}

// populations at rest relative to u: S_i^s = w_i rho_s (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u^2)
__global__ void fields_to_populations_kernel(const float* __restrict__ fld, size_t n, double* __restrict__ S) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const double ux = fld[2 * n + k], uy = fld[3 * n + k];
        const double usq = ux * ux + uy * uy;
        for (int s = 0; s < 2; ++s) {
            const double r = fld[(size_t)s * n + k];
            for (int i = 0; i < 9; ++i) {
                const double cu = cx(i) * ux + cy(i) * uy;
                S[(size_t)(s * 9 + i) * n + k] = wd(i) * r * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
            }
        }
    }
}

// Fine fields from coarse fields (the fallback's restart): bilinear in the cell
// centres (coarse cell X covers fine columns 2X and 2X + 1, so fine column x sits at
// coarse coordinate (x - 1/2) / 2), periodic in x, the wall rows' values held at the
// walls; densities as they are, velocities halved (a coarse lattice velocity is twice
// the fine one).  Each component keeps its mass: four times the coarse sum.
__global__ void prolong_kernel(const float* __restrict__ cf, int ncx, int ncy, float* __restrict__ ff) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    const int nxf = 2 * ncx, nyf = 2 * ncy;
    if (x >= nxf || y >= nyf) return;
    // (x - 1/2) / 2 = X0 + t with t = 3/4 for even x, 1/4 for odd x
    const int X0 = (x >> 1) - ((x & 1) ? 0 : 1), Y0 = (y >> 1) - ((y & 1) ? 0 : 1);
    const float tx = (x & 1) ? 0.25f : 0.75f, ty = (y & 1) ? 0.25f : 0.75f;
    const int xa = (X0 + ncx) % ncx, xb = (X0 + 1) % ncx;
    const int ya = max(Y0, 0), yb = min(Y0 + 1, ncy - 1);
    const size_t nc = (size_t)ncx * ncy, nf = (size_t)nxf * nyf;
    for (int ch = 0; ch < 4; ++ch) {
        const float* c = cf + (size_t)ch * nc;
        const float v = (1.0f - ty) * ((1.0f - tx) * c[(size_t)ya * ncx + xa] + tx * c[(size_t)ya * ncx + xb]) +
                        ty * ((1.0f - tx) * c[(size_t)yb * ncx + xa] + tx * c[(size_t)yb * ncx + xb]);
        ff[(size_t)ch * nf + (size_t)y * nxf + x] = ch < 2 ? v : 0.5f * v;
    }
}

// x = (raw - mean) / scale (network input); t = (target - raw) / out_scale (training target)
__global__ void normalize_kernel(const float* __restrict__ raw, const float* __restrict__ target, size_t n,
                                 float4 mean, float4 scale, float4 oscale, float* __restrict__ x, float* __restrict__ t) {
    const float mu[4] = {mean.x, mean.y, mean.z, mean.w}, sc[4] = {scale.x, scale.y, scale.z, scale.w};
    const float os[4] = {oscale.x, oscale.y, oscale.z, oscale.w};
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        for (int c = 0; c < 4; ++c) {
            const float r = raw[(size_t)c * n + k];
            x[(size_t)c * n + k] = (r - mu[c]) / sc[c];
            if (target) t[(size_t)c * n + k] = (target[(size_t)c * n + k] - r) / os[c];
        }
}

// The density corrections of one site from the network output (drho_A, drho_B in
// physical units), limited so that no density drops below half its value.
// mode 1: drho_A and drho_B as predicted; modes 2 and 3: only the order parameter,
// drho_A = -drho_B = (drho_A - drho_B) / 2, so the total density is unchanged;
// mode 4: the order parameter times the interface weight w (below).
__device__ __forceinline__ void limited_drho(int mode, const float rho[2], float pA, float pB, float w, float d[2]) {
    if (mode >= 2) {
        const float s = mode == 4 ? w : 1.0f;
        const float h = fminf(fmaxf(0.5f * s * (pA - pB), -0.5f * rho[0]), 0.5f * rho[1]);
        d[0] = h;
        d[1] = -h;
    } else {
        d[0] = fmaxf(pA, -0.5f * rho[0]);
        d[1] = fmaxf(pB, -0.5f * rho[1]);
    }
}

// Interface weight w = 4 c (1 - c) of the normalised mass fraction
// c = (rho_A / rho - c_bot) / (c_top - c_bot), clamped to [0, 1]: 1 on the interface,
// 0 in either bulk, so that mode 4 leaves the bulk composition alone.
__device__ __forceinline__ float interface_weight(const float rho[2], float2 cbulk) {
    const float r = rho[0] + rho[1];
    if (!(r > 0.0f)) return 0.0f;
    const float c = fminf(fmaxf((rho[0] / r - cbulk.y) / (cbulk.x - cbulk.y), 0.0f), 1.0f);
    return 4.0f * c * (1.0f - c);
}

// Densities and total momentum of one site's gathered populations, summed in one
// fixed order (the mass sums and the correction must see the same values).
__device__ __forceinline__ void site_moments(const float f[2][9], float rho[2], float& jx, float& jy) {
    jx = 0.0f;
    jy = 0.0f;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        float r = 0.0f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            r += f[s][i];
            jx += cx(i) * f[s][i];
            jy += cy(i) * f[s][i];
        }
        rho[s] = r;
    }
}

// Pass 1 of a correction: the densities rho2 [2][n] and total momenta j2 [2][n] of the
// coarse run's populations after streaming (FP32 storage), gathered as the step
// kernels pull them.
__global__ void __launch_bounds__(128) closure_moments_kernel(const float* __restrict__ fin, Grid g,
                                                              float* __restrict__ rho2, float* __restrict__ j2) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= g.nx) return;
    const float zero[2] = {0.0f, 0.0f};
    const int xm = x == 0 ? g.nx - 1 : x - 1;
    const int xp = x == g.nx - 1 ? 0 : x + 1;
    float f[2][9], rho[2], jx, jy;
    pull_site<float>(fin, g, zero, y, x, xm, xp, f);
    site_moments(f, rho, jx, jy);
    const size_t n = (size_t)g.nx * g.ny, k = (size_t)y * g.nx + x;
    rho2[k] = rho[0];
    rho2[n + k] = rho[1];
    j2[k] = jx;
    j2[n + k] = jy;
}

// Per-block sums (FP64) of the limited density corrections, from the densities
// rho2 ([2][n], the sums of the FP32 populations); mode 4: the sum of the
// order-parameter corrections and the sum of the weights.
__global__ void __launch_bounds__(256) drho_sum_kernel(const float* __restrict__ rho2, const float* __restrict__ y,
                                                       size_t n, float4 oscale, int mode, float2 cbulk,
                                                       double* __restrict__ part) {
    __shared__ double red[2][8];
    // per thread: compensated FP32 sums (Kahan) of its ~n / (blocks x 256) sites;
    // FP64 from the warp reduction on (this GPU's FP64 rate is a small fraction of FP32)
    float sa = 0.0f, ca = 0.0f, sb = 0.0f, cb = 0.0f;
#pragma unroll 4
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const float rho[2] = {rho2[k], rho2[n + k]};
        const float w = interface_weight(rho, cbulk);
        float d[2];
        limited_drho(mode, rho, y[k] * oscale.x, y[n + k] * oscale.y, w, d);
        const float va = d[0] - ca, ta = sa + va;
        ca = (ta - sa) - va;
        sa = ta;
        const float vb = (mode == 4 ? w : d[1]) - cb, tb = sb + vb;
        cb = (tb - sb) - vb;
        sb = tb;
    }
    double a = (double)sa - (double)ca, b = (double)sb - (double)cb;
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b += __shfl_down_sync(0xffffffffu, b, off);
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = a; red[1][threadIdx.x >> 5] = b; }
    __syncthreads();
    if (threadIdx.x < 2) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
        part[2 * blockIdx.x + threadIdx.x] = v;
    }
}

// The block partials summed into part[2 nparts], part[2 nparts + 1] by one block of
// 256 threads: strided per-thread sums, then a tree in shared memory (fixed order);
// n sites.
__global__ void __launch_bounds__(256) drho_total_kernel(double* __restrict__ part, int nparts, size_t n) {
    __shared__ double red[2][256];
    double a = 0.0, b = 0.0;
    for (int p = threadIdx.x; p < nparts; p += 256) {
        a += part[2 * p];
        b += part[2 * p + 1];
    }
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = b;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            red[0][threadIdx.x] += red[0][threadIdx.x + h];
            red[1][threadIdx.x] += red[1][threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // the per-site scalars of correct_inplace_kernel, once: sum(h) / sum(w) (mode 4) and
        // the mean corrections (modes 1-3), as FP32 after part[2 nparts + 1]
        const double sA = red[0][0], sB = red[1][0];
        part[2 * nparts] = sA;
        part[2 * nparts + 1] = sB;
        float* sc = reinterpret_cast<float*>(part + 2 * nparts + 2);
        sc[0] = sB > 0.0 ? (float)(sA / sB) : 0.0f;
        sc[1] = (float)(sA / (double)n);
        sc[2] = (float)(sB / (double)n);
    }
}

// Re-equilibration with the corrected moments: with rho'_s = rho_s + drho_s - mean
// (drho limited as above, the mean over the grid removed so that each component's
// mass is unchanged; mode 4 removes it in proportion to the interface weight,
// drho_A = -drho_B = h - w sum(h) / sum(w)) and u' = u_b + du in mode 1, u_b in
// mode 2 and u_b + du / 4 in modes 3 and 4 (u_b = j / rho of f itself),
//   f <- f^eq(rho'_s, u') + (rho'_s / rho_s) (f - f^eq(rho_s, u_b)),
// i.e. the non-equilibrium part is kept in proportion to the density.  With
// q = rho'_s / rho_s, so that q rho_s = rho'_s, the two equilibria combine into
//   f <- q f + w_i rho'_s (3 dc + 9/2 dc (c1 + c0) - 3/2 (u'.u' - u_b.u_b)),
// c0 = c_i.u_b, c1 = c_i.u', dc = c1 - c0 (a few operations per population instead
// of two equilibria).  p: the network output of the site in physical units (dA, dB,
// du_x, du_y); hw = sum(h) / sum(w) (mode 4), mA / mB the mean corrections (modes
// 1-3).  FP32: the corrections are small next to the populations, and the mass sums
// are FP64.
__device__ __forceinline__ void correct_site(float f[2][9], float4 p, int mode, float2 cbulk, float hw, float mA,
                                             float mB) {
    // mode 2 keeps the velocity; modes 3 and 4 relax it a quarter of the way (the
    // full correction of mode 1 feeds back into the growing coarse modes)
    const float du = mode == 1 ? 1.0f : (mode >= 3 ? 0.25f : 0.0f);
    float rho[2], jx, jy;
    site_moments(f, rho, jx, jy);
    const float r = rho[0] + rho[1];
    if (!(r > 0.0f)) return;
    const float ux = jx / r, uy = jy / r;
    const float vx = ux + du * p.z, vy = uy + du * p.w;
    const float w = interface_weight(rho, cbulk);
    float d[2];
    limited_drho(mode, rho, p.x, p.y, w, d);
    if (mode == 4) {
        d[0] -= w * hw;
        d[1] = -d[0];
    } else {
        d[0] -= mA;
        d[1] -= mB;
    }
    const float du2 = 1.5f * ((vx * vx + vy * vy) - (ux * ux + uy * uy));
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const float r0 = rho[s];
        if (!(r0 > 0.0f)) continue;
        const float r1 = fmaxf(r0 + d[s], 0.0f);
        const float q = r1 / r0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const float c0 = cx(i) * ux + cy(i) * uy, c1 = cx(i) * vx + cy(i) * vy;
            const float dc = c1 - c0;
            f[s][i] = q * f[s][i] + wf(i) * r1 * (3.0f * dc + 4.5f * dc * (c1 + c0) - du2);
        }
    }
}

// Pass 2 of a correction, in place on the coarse run's stored FP32 populations: each
// site gathers its 18 populations after streaming from the slots pull_site reads
// (addressed from one site pointer: slot = site + plane offset - c_iy pitch + the
// periodic column offset, or the site's own slot of the opposite direction on a
// wall row), corrects them (correct_site) and writes them back to the same slots,
// with the periodic ghost copy of columns 0, 1, nx - 2, nx - 1 that the staged
// kernels' row windows read.  Every stored slot belongs to exactly one (site,
// direction) pair, so no two threads touch the same slot; a thread's 18 loads
// precede its stores through one pointer.  scalars: sum(h) / sum(w) (mode 4) and the
// mean corrections (modes 1-3), from drho_total_kernel.
__global__ void __launch_bounds__(128, 7) correct_inplace_kernel(float* pops, Grid g, const float* __restrict__ y,
                                                              float4 oscale, int mode, float2 cbulk,
                                                              const float* __restrict__ scalars) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int row = blockIdx.y;
    if (x >= g.nx) return;
    // column offsets of the west and east neighbours (periodic)
    const int dxw = x == 0 ? g.nx - 1 : -1;
    const int dxe = x == g.nx - 1 ? 1 - g.nx : 1;
    const bool bottom = row == 0, top = row == g.ny - 1;
    const ptrdiff_t plane = (ptrdiff_t)g.plane, pitch = g.pitch;
    float* const site = pops + (ptrdiff_t)row * pitch + g.origin + x;
    // slot of direction i of component s, and the slot's column offset from x
    auto slot = [&](int s, int i, int* dcol) -> float* {
        if ((cy(i) == 1 && bottom) || (cy(i) == -1 && top)) {
            *dcol = 0;
            return site + (s * 9 + opp(i)) * plane;
        }
        *dcol = cx(i) == 0 ? 0 : (cx(i) == 1 ? dxw : dxe);
        return site + (s * 9 + i) * plane - cy(i) * pitch + *dcol;
    };
    float f[2][9];
    int dcol;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int i = 0; i < 9; ++i) f[s][i] = *slot(s, i, &dcol);
    const size_t n = (size_t)g.nx * g.ny, k = (size_t)row * g.nx + x;
    const float4 p = make_float4(y[k] * oscale.x, y[n + k] * oscale.y, y[2 * n + k] * oscale.z,
                                 y[3 * n + k] * oscale.w);
    correct_site(f, p, mode, cbulk, mode == 4 ? scalars[0] : 0.0f, scalars[1], scalars[2]);
    // ghost copies: only the threads of the first / last three columns can write a
    // slot in columns 0, 1, nx - 2, nx - 1
    const bool edge = x < 3 || x >= g.nx - 3;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            float* q = slot(s, i, &dcol);
            *q = f[s][i];
            if (edge) {
                const int col = x + dcol;
                if (col < 2) q[g.nx] = f[s][i];
                else if (col >= g.nx - 2) q[-g.nx] = f[s][i];
            }
        }
}

}  // namespace
}  // namespace lbm

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

lbm_status cl_fail(lbm_status st, const std::string& msg) {
    lbm::set_last_error(msg);
    return st;
}

#define CL_TRY(call, what)                                                                              \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) return cl_fail(LBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define CL_STATUS(call)                       \
    do {                                      \
        lbm_status s_ = (call);               \
        if (s_ != LBM_OK) return s_;          \
    } while (0)

constexpr int kFineStepsPerCoarse = 4;   // diffusive scaling: dt_c = 4 dt

uint64_t sm64(uint64_t& s) {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double unit(uint64_t& s) { return (double)(sm64(s) >> 11) * (1.0 / 9007199254740992.0); }

}  // namespace

struct lbm_closure {
    lbm_params fine_p, coarse_p;
    lbm_handle* fine = nullptr;
    lbm_handle* coarse = nullptr;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int interval = 10;
    int ncx = 0, ncy = 0;
    size_t nc = 0;
    float *params = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    int64_t adam_t = 0;
    void* cnn_ws = nullptr;
    lbm::cnn::Net net;
    float *raw = nullptr, *xin = nullptr, *yout = nullptr;   // [4 nc] each
    double* S = nullptr;                                       // [18 nc]
    double* part = nullptr;                                    // reduction partials
    std::vector<float*> samp_raw, samp_tgt;                    // raw coarse / restricted fine after an interval
    float *train_x = nullptr, *train_t = nullptr;
    int ntrain = 0;
    bool have_params = false;                                  // trained or set by the caller
    float* snap = nullptr;                                     // [4 nc] coarse fields at the start of lbm_closure_run
    float* fine_fld = nullptr;                                 // [4 nf] prolonged fields (fallback)
    double* S_fine = nullptr;                                  // [18 nf] fine populations (fallback)
    int64_t fallbacks = 0;                                     // intervals re-run on the fine solver
    float in_mean[4] = {0, 0, 0, 0}, in_scale[4] = {1, 1, 1, 1}, out_scale[4] = {1, 1, 1, 1};
};

namespace {

float4 f4(const float* a) { return make_float4(a[0], a[1], a[2], a[3]); }

// blocks of the correction's mass sums (enough for the loads in flight to cover
// the memory latency): 2 partials each, then 2 totals and 3 FP32 scalars (2 doubles)
constexpr int kCorrBlocks = 4096;
constexpr size_t kPartDoubles = 2 * kCorrBlocks + 4;

// restricted fields of the fine run into c->raw (or `dst`)
lbm_status restrict_fine(lbm_closure* c, float* dst) {
    const double *rA, *rB, *ux, *uy;
    CL_TRY(lbm::handle_fields(c->fine, &rA, &rB, &ux, &uy), "fine fields");
    dim3 grid((c->ncx + 127) / 128, c->ncy);
    lbm::restrict_kernel<<<grid, 128, 0, c->stream>>>(rA, rB, ux, uy, c->fine_p.nx, dst, c->ncx, c->ncy);
    CL_TRY(cudaGetLastError(), "restrict");
    return LBM_OK;
}

lbm_status coarse_fields(lbm_closure* c, float* dst) {
    const double *rA, *rB, *ux, *uy;
    CL_TRY(lbm::handle_fields(c->coarse, &rA, &rB, &ux, &uy), "coarse fields");
    lbm::fields_to_float_kernel<<<512, 256, 0, c->stream>>>(rA, rB, ux, uy, c->nc, dst);
    CL_TRY(cudaGetLastError(), "fields to float");
    return LBM_OK;
}

// replace the coarse state by populations built from the fields in `fld`
lbm_status set_coarse(lbm_closure* c, const float* fld) {
    lbm::fields_to_populations_kernel<<<512, 256, 0, c->stream>>>(fld, c->nc, c->S);
    CL_TRY(cudaGetLastError(), "fields to populations");
    CL_TRY(lbm::handle_push_S(c->coarse, c->S), "push coarse state");
    return LBM_OK;
}

// apply the network's correction to the coarse run (mode 1: densities and velocity,
// mode 2: order parameter only, mode 3: order parameter and a quarter of the velocity,
// mode 4: as mode 3 with the order parameter corrected on the interface only): the
// moments, the network input and output, the mass sums, then the correction in
// place on the stored populations.  clear_status: start the tensor-core kernels' status word from 0 (the first
// correction of a call); later ones keep an earlier failure raised for the check
// at the end of the call
lbm_status correct(lbm_closure* c, int mode, bool clear_status) {
    // bulk mass fractions of the coarse run's initial state (pure A on top, pure B below)
    const lbm_params& q = c->coarse_p;
    const double2 cbulk = make_double2(q.mass_A / (q.mass_A + q.minority * q.mass_B),
                                       q.minority * q.mass_A / (q.minority * q.mass_A + q.mass_B));
    const lbm::PopView v = lbm::handle_pops(c->coarse);
    if (v.storage != LBM_STORE_F32) return cl_fail(LBM_ESTATE, "the closure's coarse run must store FP32");
    float* pops = static_cast<float*>(v.pops);
    // raw holds the densities (first half) and the momenta (second half)
    float* rho2 = c->raw;
    float* j2 = c->raw + 2 * c->nc;
    const dim3 grid((v.grid.nx + 127) / 128, v.grid.ny);
    lbm::closure_moments_kernel<<<grid, 128, 0, v.stream>>>(pops, v.grid, rho2, j2);
    CL_TRY(cudaGetLastError(), "coarse moments");
    CL_TRY(lbm::handle_closure_features(c->coarse, rho2, j2, c->in_mean, c->in_scale, c->xin), "network input");
    CL_TRY(lbm::cnn_tc::infer(c->net.tc, c->params, c->xin, c->yout, c->stream, false, clear_status), "cnn inference");
    const float2 cb = make_float2((float)cbulk.x, (float)cbulk.y);
    lbm::drho_sum_kernel<<<kCorrBlocks, 256, 0, c->stream>>>(rho2, c->yout, c->nc, f4(c->out_scale), mode, cb, c->part);
    CL_TRY(cudaGetLastError(), "mass sums");
    lbm::drho_total_kernel<<<1, 256, 0, c->stream>>>(c->part, kCorrBlocks, c->nc);
    lbm::correct_inplace_kernel<<<grid, 128, 0, v.stream>>>(pops, v.grid, c->yout, f4(c->out_scale), mode, cb,
                                                           reinterpret_cast<const float*>(c->part + 2 * kCorrBlocks + 2));
    CL_TRY(cudaGetLastError(), "correct");
    return LBM_OK;
}

// Synchronises the closure's stream and reads the tensor-core kernels' status word:
// LBM_ETIMEOUT if one of their waits gave up since the word was last cleared.
lbm_status cnn_check(lbm_closure* c) {
    int st = 0;
    CL_TRY(lbm::cnn_tc::status(c->net.tc, c->stream, &st), "cnn inference status");
    if (st != 0)
        return cl_fail(LBM_ETIMEOUT, "a wait of the tensor-core CNN kernels gave up (status " + std::to_string(st) +
                                         "): the corrected state is unreliable");
    return LBM_OK;
}

// The fallback: the fine plain solver re-runs `coarse_steps` coarse steps' worth of
// time (four fine steps each) from the coarse fields saved in c->snap, prolonged to the
// fine grid, and the coarse run restarts from the restriction of the result.
lbm_status fine_fallback(lbm_closure* c, int64_t coarse_steps) {
    const size_t nf = 4 * c->nc;
    if (!c->fine_fld) {
        if (cudaMalloc((void**)&c->fine_fld, 4 * nf * 4) != cudaSuccess) return cl_fail(LBM_ENOMEM, "fallback fields");
        if (cudaMalloc((void**)&c->S_fine, 18 * nf * 8) != cudaSuccess) return cl_fail(LBM_ENOMEM, "fallback populations");
    }
    const dim3 grid((2 * c->ncx + 127) / 128, 2 * c->ncy);
    lbm::prolong_kernel<<<grid, 128, 0, c->stream>>>(c->snap, c->ncx, c->ncy, c->fine_fld);
    CL_TRY(cudaGetLastError(), "prolong");
    lbm::fields_to_populations_kernel<<<512, 256, 0, c->stream>>>(c->fine_fld, nf, c->S_fine);
    CL_TRY(cudaGetLastError(), "fine populations");
    CL_TRY(lbm::handle_push_S(c->fine, c->S_fine), "push fine state");
    CL_TRY(lbm::handle_clear_guard(c->fine), "clear fine guard");
    CL_STATUS(lbm_step(c->fine, kFineStepsPerCoarse * coarse_steps));
    CL_STATUS(lbm_sync(c->fine));
    CL_STATUS(restrict_fine(c, c->raw));
    CL_STATUS(set_coarse(c, c->raw));
    CL_TRY(lbm::handle_clear_guard(c->coarse), "clear coarse guard");
    ++c->fallbacks;
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_cnn_workspace_bytes(int32_t nx, int32_t ny, size_t* bytes) {
    if (!bytes || nx < 1 || ny < 1) return cl_fail(LBM_EINVAL, "invalid CNN grid");
    *bytes = lbm::cnn::workspace_bytes(nx, ny);
    return LBM_OK;
}

lbm_status lbm_cnn_forward(const float* params, const float* x, int32_t nx, int32_t ny, void* ws, size_t ws_bytes,
                           void* stream, float* y) {
    if (!params || !x || !ws || !y || nx < 1 || ny < 1) return cl_fail(LBM_EINVAL, "NULL argument or empty grid");
    if (ws_bytes < lbm::cnn::workspace_bytes(nx, ny)) return cl_fail(LBM_ENOMEM, "CNN workspace too small");
    lbm::cnn::Net N = lbm::cnn::carve(ws, nx, ny);
    CL_TRY(lbm::cnn::forward(N, params, x, y, (cudaStream_t)stream), "cnn forward");
    return LBM_OK;
}

lbm_status lbm_cnn_infer(const float* params, const float* x, int32_t nx, int32_t ny, void* ws, size_t ws_bytes,
                         void* stream, float* y) {
    if (!params || !x || !ws || !y || nx < 1 || ny < 1) return cl_fail(LBM_EINVAL, "NULL argument or empty grid");
    if (ws_bytes < lbm::cnn::workspace_bytes(nx, ny)) return cl_fail(LBM_ENOMEM, "CNN workspace too small");
    lbm::cnn::Net N = lbm::cnn::carve(ws, nx, ny);
    CL_TRY(lbm::cnn_tc::infer(N.tc, params, x, y, (cudaStream_t)stream), "cnn inference");
    return LBM_OK;
}

lbm_status lbm_cnn_infer_test_timeout(const float* params, const float* x, int32_t nx, int32_t ny, void* ws,
                                      size_t ws_bytes, void* stream, float* y) {
    if (!params || !x || !ws || !y || nx < 1 || ny < 1) return cl_fail(LBM_EINVAL, "NULL argument or empty grid");
    if (ws_bytes < lbm::cnn::workspace_bytes(nx, ny)) return cl_fail(LBM_ENOMEM, "CNN workspace too small");
    lbm::cnn::Net N = lbm::cnn::carve(ws, nx, ny);
    CL_TRY(lbm::cnn_tc::infer(N.tc, params, x, y, (cudaStream_t)stream, true), "cnn inference (copies withheld)");
    return LBM_OK;
}

lbm_status lbm_cnn_infer_status(void* ws, int32_t nx, int32_t ny, void* stream) {
    if (!ws || nx < 1 || ny < 1) return cl_fail(LBM_EINVAL, "NULL workspace or empty grid");
    lbm::cnn::Net N = lbm::cnn::carve(ws, nx, ny);
    int st = 0;
    CL_TRY(lbm::cnn_tc::status(N.tc, (cudaStream_t)stream, &st), "cnn inference status");
    if (st != 0) return cl_fail(LBM_ETIMEOUT, "a wait of the tensor-core CNN kernels gave up (status " + std::to_string(st) + ")");
    return LBM_OK;
}

lbm_status lbm_cnn_loss_grad(const float* params, const float* x, const float* t, int32_t nx, int32_t ny, void* ws,
                             size_t ws_bytes, void* stream, double* loss, float* grad) {
    if (!params || !x || !t || !ws || !grad || !loss || nx < 1 || ny < 1)
        return cl_fail(LBM_EINVAL, "NULL argument or empty grid");
    if (ws_bytes < lbm::cnn::workspace_bytes(nx, ny)) return cl_fail(LBM_ENOMEM, "CNN workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    lbm::cnn::Net N = lbm::cnn::carve(ws, nx, ny);
    int nb = 0;
    CL_TRY(lbm::cnn::loss_grad(N, params, x, t, grad, &nb, st), "cnn loss/grad");
    std::vector<double> part(nb);
    CL_TRY(cudaMemcpyAsync(part.data(), N.lpart, nb * sizeof(double), cudaMemcpyDeviceToHost, st), "copy loss");
    CL_TRY(cudaStreamSynchronize(st), "sync");
    double s = 0.0;
    for (double p : part) s += p;
    *loss = s / (double)(lbm::cnn::kOut * (size_t)nx * ny);
    return LBM_OK;
}

void lbm_closure_destroy(lbm_closure* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->fine) lbm_destroy(c->fine);
    if (c->coarse) lbm_destroy(c->coarse);
    for (float* p : c->samp_raw) cudaFree(p);
    for (float* p : c->samp_tgt) cudaFree(p);
    void* bufs[] = {c->params, c->grad, c->m, c->v, c->cnn_ws, c->raw, c->xin, c->yout, c->S, c->part, c->train_x, c->train_t,
                    c->snap, c->fine_fld, c->S_fine};
    for (void* p : bufs)
        if (p) cudaFree(p);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

lbm_status lbm_closure_coarse_params(const lbm_params* fine, lbm_params* out) {
    if (!fine || !out) return cl_fail(LBM_EINVAL, "NULL argument");
    if (fine->nx % 2 || fine->ny % 2 || fine->x_offset % 2 || fine->nx_total % 2)
        return cl_fail(LBM_EINVAL, "the fine grid must have even nx, ny, x_offset and nx_total");
    lbm_params p = *fine;
    p.nx = fine->nx / 2;
    p.ny = fine->ny / 2;
    p.g = 8.0 * fine->g;
    p.gx = 8.0 * fine->gx;
    p.amp = fine->amp / 2.0;
    p.width = std::max(0.5, fine->width / 2.0);
    p.y0 = fine->y0 < 0.0 ? -1.0 : fine->y0 / 2.0;
    p.crop_rows = std::max(3, fine->crop_rows / 2);
    p.x_offset = fine->x_offset / 2;
    p.nx_total = fine->nx_total / 2;
    p.storage = LBM_STORE_F32;
    p.kernel = LBM_KERNEL_STAGED;
    p.tile_y = 0;
    p.tile_x = 0;
    *out = p;
    return LBM_OK;
}

lbm_status lbm_closure_create(const lbm_params* fine, int32_t interval, uint64_t seed, void* cuda_stream,
                              lbm_closure** out) {
    if (!out) return cl_fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!fine || interval < 1) return cl_fail(LBM_EINVAL, "invalid arguments");
    lbm_closure* c = new lbm_closure();
    c->interval = interval;
    c->fine_p = *fine;
    c->fine_p.storage = LBM_STORE_F32;
    c->fine_p.kernel = LBM_KERNEL_STAGED;
    lbm_status st = lbm_closure_coarse_params(&c->fine_p, &c->coarse_p);
    if (st != LBM_OK) {
        delete c;
        return st;
    }
    auto bail = [&](lbm_status s, const std::string& msg) {
        lbm_closure_destroy(c);
        return cl_fail(s, msg);
    };
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(LBM_ECUDA, "stream");
        c->own_stream = true;
    }
    if ((st = lbm_create_ex(&c->fine_p, nullptr, 0, c->stream, &c->fine)) != LBM_OK)
        return bail(st, std::string("fine solver: ") + lbm_last_error());
    if ((st = lbm_create_ex(&c->coarse_p, nullptr, 0, c->stream, &c->coarse)) != LBM_OK)
        return bail(st, std::string("coarse solver: ") + lbm_last_error());
    c->ncx = c->coarse_p.nx;
    c->ncy = c->coarse_p.ny;
    c->nc = (size_t)c->ncx * c->ncy;
    const size_t P = lbm::cnn::kParams;
    bool ok = cudaMalloc((void**)&c->params, P * 4) == cudaSuccess && cudaMalloc((void**)&c->grad, P * 4) == cudaSuccess &&
              cudaMalloc((void**)&c->m, P * 4) == cudaSuccess && cudaMalloc((void**)&c->v, P * 4) == cudaSuccess &&
              cudaMalloc(&c->cnn_ws, lbm::cnn::workspace_bytes(c->ncx, c->ncy)) == cudaSuccess &&
              cudaMalloc((void**)&c->raw, 4 * c->nc * 4) == cudaSuccess &&
              cudaMalloc((void**)&c->xin, 4 * c->nc * 4) == cudaSuccess &&
              cudaMalloc((void**)&c->yout, 4 * c->nc * 4) == cudaSuccess &&
              cudaMalloc((void**)&c->S, 18 * c->nc * 8) == cudaSuccess &&
              cudaMalloc((void**)&c->snap, 4 * c->nc * 4) == cudaSuccess &&
              cudaMalloc((void**)&c->part, kPartDoubles * 8) == cudaSuccess;
    if (!ok) return bail(LBM_ENOMEM, "closure buffers");
    c->net = lbm::cnn::carve(c->cnn_ws, c->ncx, c->ncy);
    // He-normal weights (Box-Muller on splitmix64), zero biases
    std::vector<float> h(P, 0.0f);
    uint64_t s = seed;
    auto fill = [&](int off, int count, int fan_in) {
        const double sd = std::sqrt(2.0 / fan_in);
        for (int i = 0; i < count; ++i) {
            const double u1 = std::max(unit(s), 1e-300), u2 = unit(s);
            h[off + i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
        }
    };
    fill(lbm::cnn::kW1, lbm::cnn::kHid * lbm::cnn::kIn * 9, lbm::cnn::kIn * 9);
    fill(lbm::cnn::kW2, lbm::cnn::kHid * lbm::cnn::kHid * 9, lbm::cnn::kHid * 9);
    fill(lbm::cnn::kW3, lbm::cnn::kOut * lbm::cnn::kHid * 9, lbm::cnn::kHid * 9);
    // the last layer starts small, so the untrained closure is close to no correction
    for (int i = 0; i < lbm::cnn::kOut * lbm::cnn::kHid * 9; ++i) h[lbm::cnn::kW3 + i] *= 0.01f;
    if (cudaMemcpy(c->params, h.data(), P * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(c->m, 0, P * 4) != cudaSuccess || cudaMemset(c->v, 0, P * 4) != cudaSuccess)
        return bail(LBM_ECUDA, "upload parameters");
    *out = c;
    return LBM_OK;
}

lbm_status lbm_closure_generate(lbm_closure* c, int32_t n_runs, uint64_t seed0, int32_t warmup_fine_steps,
                                int32_t intervals_per_run) {
    if (!c || n_runs < 1 || intervals_per_run < 1 || warmup_fine_steps < 0) return cl_fail(LBM_EINVAL, "invalid arguments");
    const size_t bytes = 4 * c->nc * 4;
    for (int r = 0; r < n_runs; ++r) {
        CL_STATUS(lbm::handle_reseed(c->fine, seed0 + (uint64_t)r));
        CL_STATUS(lbm_step(c->fine, warmup_fine_steps));
        for (int k = 0; k < intervals_per_run; ++k) {
            CL_STATUS(restrict_fine(c, c->raw));
            CL_STATUS(set_coarse(c, c->raw));
            CL_STATUS(lbm_step(c->coarse, c->interval));
            CL_STATUS(lbm_step(c->fine, kFineStepsPerCoarse * c->interval));
            float *sr = nullptr, *sg = nullptr;
            if (cudaMalloc((void**)&sr, bytes) != cudaSuccess) return cl_fail(LBM_ENOMEM, "sample buffer");
            c->samp_raw.push_back(sr);
            if (cudaMalloc((void**)&sg, bytes) != cudaSuccess) return cl_fail(LBM_ENOMEM, "sample buffer");
            c->samp_tgt.push_back(sg);
            CL_STATUS(coarse_fields(c, sr));
            CL_STATUS(restrict_fine(c, sg));
        }
    }
    CL_STATUS(lbm_sync(c->fine));
    CL_STATUS(lbm_sync(c->coarse));
    return LBM_OK;
}

lbm_status lbm_closure_train(lbm_closure* c, int32_t epochs, double lr, uint64_t shuffle_seed, double* final_loss) {
    if (!c || epochs < 0 || !(lr > 0.0)) return cl_fail(LBM_EINVAL, "invalid arguments");
    const int ns = (int)c->samp_raw.size();
    if (ns == 0) return cl_fail(LBM_ESTATE, "no training samples: call lbm_closure_generate first");
    const size_t n = c->nc;
    // normalisation constants from the samples (host statistics)
    {
        std::vector<float> a(4 * n), b(4 * n);
        double s1[4] = {0}, s2[4] = {0}, d2[4] = {0};
        for (int i = 0; i < ns; ++i) {
            CL_TRY(cudaMemcpy(a.data(), c->samp_raw[i], 4 * n * 4, cudaMemcpyDeviceToHost), "copy sample");
            CL_TRY(cudaMemcpy(b.data(), c->samp_tgt[i], 4 * n * 4, cudaMemcpyDeviceToHost), "copy sample");
            for (int ch = 0; ch < 4; ++ch)
                for (size_t k = 0; k < n; ++k) {
                    const double r = a[ch * n + k], d = (double)b[ch * n + k] - r;
                    s1[ch] += r;
                    s2[ch] += r * r;
                    d2[ch] += d * d;
                }
        }
        const double cnt = (double)ns * n;
        for (int ch = 0; ch < 4; ++ch) {
            c->in_mean[ch] = (float)(s1[ch] / cnt);
            c->in_scale[ch] = (float)std::max(std::sqrt(std::max(s2[ch] / cnt - (s1[ch] / cnt) * (s1[ch] / cnt), 0.0)), 1e-12);
            c->out_scale[ch] = (float)std::max(std::sqrt(d2[ch] / cnt), 1e-12);
        }
    }
    if (c->ntrain != ns) {
        if (c->train_x) cudaFree(c->train_x);
        if (c->train_t) cudaFree(c->train_t);
        c->train_x = c->train_t = nullptr;
        if (cudaMalloc((void**)&c->train_x, (size_t)ns * 4 * n * 4) != cudaSuccess ||
            cudaMalloc((void**)&c->train_t, (size_t)ns * 4 * n * 4) != cudaSuccess)
            return cl_fail(LBM_ENOMEM, "training set");
        c->ntrain = ns;
    }
    for (int i = 0; i < ns; ++i) {
        lbm::normalize_kernel<<<512, 256, 0, c->stream>>>(c->samp_raw[i], c->samp_tgt[i], n, f4(c->in_mean),
                                                          f4(c->in_scale), f4(c->out_scale), c->train_x + (size_t)i * 4 * n,
                                                          c->train_t + (size_t)i * 4 * n);
    }
    CL_TRY(cudaGetLastError(), "normalize samples");
    std::vector<int> order(ns);
    for (int i = 0; i < ns; ++i) order[i] = i;
    uint64_t rs = shuffle_seed;
    double last = 0.0;
    const size_t P = lbm::cnn::kParams;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int i = ns - 1; i > 0; --i) std::swap(order[i], order[sm64(rs) % (uint64_t)(i + 1)]);
        double sum = 0.0;
        for (int idx : order) {
            int nb = 0;
            CL_TRY(lbm::cnn::loss_grad(c->net, c->params, c->train_x + (size_t)idx * 4 * n,
                                       c->train_t + (size_t)idx * 4 * n, c->grad, &nb, c->stream), "loss/grad");
            ++c->adam_t;
            const float b1t = (float)std::pow(0.9, (double)c->adam_t), b2t = (float)std::pow(0.999, (double)c->adam_t);
            lbm::cnn::adam_kernel<<<(int)((P + 255) / 256), 256, 0, c->stream>>>(c->params, c->grad, c->m, c->v, (int)P,
                                                                                 (float)lr, b1t, b2t);
            CL_TRY(cudaGetLastError(), "adam");
            std::vector<double> part(nb);
            CL_TRY(cudaMemcpyAsync(part.data(), c->net.lpart, nb * 8, cudaMemcpyDeviceToHost, c->stream), "loss");
            CL_TRY(cudaStreamSynchronize(c->stream), "sync");
            for (double p : part) sum += p;
        }
        last = sum / ((double)ns * 4 * n);
    }
    c->have_params = true;
    if (final_loss) *final_loss = last;
    return LBM_OK;
}

lbm_status lbm_closure_evaluate(lbm_closure* c, uint64_t seed, int32_t warmup_fine_steps, int32_t intervals,
                                int32_t use_net, lbm_diag* coarse_out, lbm_diag* fine_out) {
    if (!c || intervals < 0 || warmup_fine_steps < 0 || !coarse_out || !fine_out) return cl_fail(LBM_EINVAL, "invalid arguments");
    if (use_net < 0 || use_net > 4) return cl_fail(LBM_EINVAL, "use_net must be 0 to 4");
    if (use_net && !c->have_params) return cl_fail(LBM_ESTATE, "the network has not been trained");
    CL_STATUS(lbm::handle_reseed(c->fine, seed));
    CL_STATUS(lbm_step(c->fine, warmup_fine_steps));
    CL_STATUS(restrict_fine(c, c->raw));
    CL_STATUS(set_coarse(c, c->raw));
    // a new coarse run: an earlier evaluation that tripped the guard leaves it raised
    CL_TRY(lbm::handle_clear_guard(c->coarse), "clear coarse guard");
    CL_STATUS(lbm_diagnostics(c->coarse, &coarse_out[0]));
    CL_STATUS(lbm_diagnostics(c->fine, &fine_out[0]));
    for (int k = 1; k <= intervals; ++k) {
        CL_STATUS(lbm_step(c->coarse, c->interval));
        if (use_net) CL_STATUS(correct(c, use_net, k == 1));
        CL_STATUS(lbm_step(c->fine, kFineStepsPerCoarse * c->interval));
        lbm_status st = lbm_diagnostics(c->coarse, &coarse_out[k]);
        if (st != LBM_OK) return st;   // the caller falls back to the fine run (fine_out stays valid)
        CL_STATUS(lbm_diagnostics(c->fine, &fine_out[k]));
    }
    if (use_net && intervals > 0) CL_STATUS(cnn_check(c));
    return LBM_OK;
}

lbm_status lbm_closure_advance(lbm_closure* c, int32_t intervals, int32_t use_net) {
    if (!c || intervals < 0) return cl_fail(LBM_EINVAL, "invalid arguments");
    if (use_net < 0 || use_net > 4) return cl_fail(LBM_EINVAL, "use_net must be 0 to 4");
    if (use_net && !c->have_params) return cl_fail(LBM_ESTATE, "the network has not been trained");
    for (int k = 0; k < intervals; ++k) {
        CL_STATUS(lbm_step(c->coarse, c->interval));
        if (use_net) CL_STATUS(correct(c, use_net, k == 0));
    }
    if (use_net && intervals > 0) CL_STATUS(cnn_check(c));
    return LBM_OK;
}

lbm_status lbm_closure_correct(lbm_closure* c, int32_t use_net) {
    if (!c) return cl_fail(LBM_EINVAL, "NULL closure");
    if (use_net < 0 || use_net > 4) return cl_fail(LBM_EINVAL, "use_net must be 0 to 4");
    if (use_net == 0) return LBM_OK;
    if (!c->have_params) return cl_fail(LBM_ESTATE, "the network has not been trained");
    CL_STATUS(correct(c, use_net, true));
    return cnn_check(c);
}

lbm_status lbm_closure_run(lbm_closure* c, int64_t coarse_steps, lbm_diag* out) {
    if (!c || coarse_steps < 0 || !out) return cl_fail(LBM_EINVAL, "invalid arguments");
    if (!c->have_params) return cl_fail(LBM_ESTATE, "the network has not been trained");
    constexpr int kRunMode = 4;
    CL_STATUS(coarse_fields(c, c->snap));          // the state the fallback restarts from
    const int64_t full = coarse_steps / c->interval, rest = coarse_steps % c->interval;
    for (int64_t k = 0; k < full; ++k) {
        CL_STATUS(lbm_step(c->coarse, c->interval));
        CL_STATUS(correct(c, kRunMode, k == 0));
    }
    if (rest) CL_STATUS(lbm_step(c->coarse, rest));
    // the indicators: the step kernels' guard (a NaN or negative density) and the
    // tensor-core kernels' status (a wait that gave up)
    lbm_status st = lbm_sync(c->coarse);
    if (st == LBM_OK && full > 0) st = cnn_check(c);
    if (st == LBM_EUNSTABLE || st == LBM_ETIMEOUT) {
        CL_STATUS(fine_fallback(c, coarse_steps));
    } else if (st != LBM_OK) {
        return st;
    }
    return lbm_diagnostics(c->coarse, out);
}

lbm_status lbm_closure_fallbacks(lbm_closure* c, int64_t* count) {
    if (!c || !count) return cl_fail(LBM_EINVAL, "NULL argument");
    *count = c->fallbacks;
    return LBM_OK;
}

lbm_status lbm_closure_params(lbm_closure* c, float* host, int32_t set) {
    if (!c || !host) return cl_fail(LBM_EINVAL, "NULL argument");
    const size_t bytes = lbm::cnn::kParams * 4;
    if (set) {
        CL_TRY(cudaMemcpy(c->params, host, bytes, cudaMemcpyHostToDevice), "set parameters");
        c->have_params = true;
    } else
        CL_TRY(cudaMemcpy(host, c->params, bytes, cudaMemcpyDeviceToHost), "get parameters");
    return LBM_OK;
}

lbm_status lbm_closure_solvers(lbm_closure* c, lbm_handle** fine, lbm_handle** coarse) {
    if (!c) return cl_fail(LBM_EINVAL, "NULL argument");
    if (fine) *fine = c->fine;
    if (coarse) *coarse = c->coarse;
    return LBM_OK;
}

lbm_status lbm_closure_normalisation(lbm_closure* c, float* host12) {
    if (!c || !host12) return cl_fail(LBM_EINVAL, "NULL argument");
    for (int i = 0; i < 4; ++i) {
        host12[i] = c->in_mean[i];
        host12[4 + i] = c->in_scale[i];
        host12[8 + i] = c->out_scale[i];
    }
    return LBM_OK;
}

lbm_status lbm_closure_set_normalisation(lbm_closure* c, const float* host12) {
    if (!c || !host12) return cl_fail(LBM_EINVAL, "NULL argument");
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(host12[i]) || (i >= 4 && !(host12[i] > 0.0f)))
            return cl_fail(LBM_EINVAL, "normalisation: values must be finite and the scales positive");
    for (int i = 0; i < 4; ++i) {
        c->in_mean[i] = host12[i];
        c->in_scale[i] = host12[4 + i];
        c->out_scale[i] = host12[8 + i];
    }
    return LBM_OK;
}

}  // extern "C"
