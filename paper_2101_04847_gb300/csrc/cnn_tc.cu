// Tensor-core inference of the closure CNN on sm_103a (tcgen05 MMA, operands in
// shared memory staged by bulk asynchronous copies, FP32 accumulators in tensor
// memory).
//
// One 3x3 convolution is an implicit GEMM over row segments of 128 pixels.  The
// three row taps are folded into N: for each staged input row r and x shift kx,
//   D_r[m][ky W + n] += sum_c in[r][x0 + m + kx - 1][c] * w[n][c][ky][kx]
// (M = 128 pixels, N = 3 W, W = 32 output channels, or 4 for the last layer with N
// padded to 16; K = 16 channels per MMA instruction), and output row y is
// D_(y-1)[., 0..W) + D_y[., W..2W) + D_(y+1)[., 2W..3W), summed in registers by the
// epilogue as the rows stream past.  Each staged row is thus read by 3 x shifts x
// (channels / 16) MMAs instead of 9 x (channels / 16): the tensor cores' reads of
// shared memory, not DRAM, were the busiest unit with one tap per MMA.
//
// A CTA owns a 128-pixel column strip and a band of rows.  It streams the input
// rows of its band (plus one above and below) through a ring of shared-memory
// slots, one row per slot with the channel groups of 8 as separate planes of 136
// pixels x 16 bytes, which is the tensor cores' K-major layout without swizzle: 8
// consecutive pixels form one 8x16-byte core matrix, the next 8 pixels follow at
// 128 bytes (SBO) and the next 8 channels one plane further (LBO).  The x shift of
// a tap is then just a 16-byte shift of the operand's start address.  Weights are
// staged once per CTA in the same layout (N rows of 16 bytes per channel group).
//
// Roles (6 warps): warp 0 lane 0 issues the bulk copies; warp 1 owns the tensor
// memory (two accumulators of N columns, alternating between input rows) and lane
// 0 issues the MMAs; warps 2-5 read the accumulators (warp w reads lanes
// 32 (w mod 4) ... of tensor memory, i.e. pixels 32 (w mod 4) ...), complete one
// output row per input row, add the bias, apply ReLU, round to BF16 and store.
// mbarriers: full[s] (copies landed), empty[s] (MMAs reading slot s done, by
// tcgen05.commit), accf[b] (accumulator b complete), acce[b] (accumulator b read).
// Every wait is bounded: a wait that gives up raises the status word, tells the
// other roles to stop, and the CTA waits (again bounded) for its copies and MMAs in
// flight before freeing its tensor memory.
#include "cnn_tc.cuh"

#include <cuda_bf16.h>

#include <algorithm>

namespace lbm {
namespace cnn_tc {
namespace {

constexpr int kHid = 32, kIn = 4, kOut = 4;
constexpr int kW1 = 0, kB1 = kW1 + kHid * kIn * 9;
constexpr int kW2 = kB1 + kHid, kB2 = kW2 + kHid * kHid * 9;
constexpr int kW3 = kB2 + kHid, kB3 = kW3 + kOut * kHid * 9;

constexpr int kM = 128;                 // pixels per MMA (rows of D)
constexpr int kSlotPx = 136;            // pixels per shared-memory plane (130 used, rest zero)
constexpr int kPlane = kSlotPx * 16;    // bytes per plane (LBO of the A operand)
constexpr int kCopy = (kM + 2) * 16;    // bytes copied per plane and row
constexpr int kStages = 6;              // ring slots: 3 rows in use + 3 in flight
constexpr int kThreads = 192;
constexpr uint32_t kWaitLimit = 1u << 22;

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Operand bytes of one layer's weights: 3 x shifts x (KG/2) K-steps x 2 groups x NF rows x 16 B.
__host__ __device__ constexpr int wbytes(int KG, int NF) { return 3 * (KG / 2) * 2 * NF * 16; }
// MMA width for W output channels per row tap: 3 W rounded up to a multiple of 16
__host__ __device__ constexpr int nfold(int W) { return (3 * W + 15) / 16 * 16; }
// tensor-memory columns of two accumulators (a power of two, at least 32)
__host__ __device__ constexpr uint32_t tmem_cols(int NF) {
    return 2 * NF <= 32 ? 32u : (2 * NF <= 64 ? 64u : (2 * NF <= 128 ? 128u : 256u));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the completion of the phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit = kWaitLimit) {
    for (uint32_t it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major without swizzle: start address, LBO
// (distance of the next 8 K-elements), SBO (distance of the next 8 M/N rows), all
// in 16-byte units; bit 46 is the descriptor version of this architecture.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 lanes x N consecutive 32-bit columns of tensor memory into v (one lane's row per thread).
template <int N> __device__ __forceinline__ void tmem_load(uint32_t taddr, float* v);
template <> __device__ __forceinline__ void tmem_load<32>(uint32_t t, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(t));
    // the registers pass through the wait, so that no use is scheduled before it
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
          "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),
          "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
          "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
template <> __device__ __forceinline__ void tmem_load<16>(uint32_t t, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(t));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
          "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                 :
                 : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <> __device__ __forceinline__ void tmem_load<4>(uint32_t t, float* v) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(t));
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]) : : "memory");
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

template <int KG, int NF> constexpr int smem_bytes() { return 256 + wbytes(KG, NF) + kStages * KG * kPlane; }

// One 3x3 convolution layer.  KGG channel groups of 8 are read per input row
// (KG >= KGG groups in shared memory, the extra ones zero: the first layer has 4
// channels, padded to one group of 8 in memory and to K = 16 in the MMA).  W
// output channels per row tap.  HIDDEN: bias + ReLU, BF16 activation planes out;
// else bias, 4 channels as FP32 planes y[4][ny][nx].
template <int KGG, int KG, int W, bool HIDDEN>
__global__ void __launch_bounds__(kThreads, 1)
conv_tc_kernel(const uint8_t* __restrict__ in, const uint8_t* __restrict__ wop, const float* __restrict__ bias,
               uint8_t* __restrict__ hout, float* __restrict__ yout, int nx, int ny, int pitch, int rows_per_cta,
               int* __restrict__ status, int withhold) {
    // withhold != 0 (tests of the timeout path only): no copies are issued and every
    // wait polls 4096 times, so the waits of the MMA issuer and of the epilogue give
    // up, raise the status word and the CTA returns
    const uint32_t lim = withhold ? 4096u : kWaitLimit;
    constexpr int KSTEPS = KG / 2;
    constexpr int NF = nfold(W);
    constexpr int WB = wbytes(KG, NF);
    constexpr int SLOT = KG * kPlane;
    constexpr uint32_t NCOL = tmem_cols(NF);
    constexpr uint32_t ID = idesc(kM, NF);
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + kStages;
    uint64_t* accf = empty + kStages;
    uint64_t* acce = accf + 2;
    uint64_t* wbar = acce + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(wbar + 1);
    volatile int* stop = reinterpret_cast<volatile int*>(tslot + 1);
    uint8_t* wsm = smem + 256;
    uint8_t* ring = wsm + WB;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x0 = blockIdx.x * kM;
    const int y0 = blockIdx.y * rows_per_cta;
    const int R = min(rows_per_cta, ny - y0);
    const int rows_in = R + 2;   // input rows y0 - 1 ... y0 + R

    for (int i = threadIdx.x; i < kStages * SLOT / 16; i += kThreads)
        reinterpret_cast<uint4*>(ring)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 4);
        }
        mbar_init(wbar, 1);
        *stop = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // zeros visible to the tensor cores
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(NCOL)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0 && lane == 0 && R > 0 && !withhold) {
        // ---- producer: weights once, then the input rows of the band
        mbar_expect_tx(wbar, WB);
        bulk_g2s(wsm, wop, WB, wbar);
        int j = 0;
        for (; j < rows_in; ++j) {
            const int s = j % kStages;
            if (j >= kStages && !mbar_wait(&empty[s], (uint32_t)((j / kStages) - 1) & 1u)) {
                *stop = 1;
                atomicOr(status, 1);
                break;
            }
            if (*stop) break;
            mbar_expect_tx(&full[s], KGG * kCopy);
            const uint8_t* src = in + (((size_t)(y0 + j) * KGG) * pitch + x0) * 16;
#pragma unroll
            for (int g = 0; g < KGG; ++g) bulk_g2s(ring + s * SLOT + g * kPlane, src + (size_t)g * pitch * 16, kCopy, &full[s]);
        }
        // copies still in flight land before the CTA exits (completed phases pass at once)
        for (int q = j > kStages ? j - kStages : 0; q < j; ++q)
            if (!mbar_wait(&full[q % kStages], (uint32_t)(q / kStages) & 1u)) atomicOr(status, 2);
        mbar_wait(wbar, 0);
    } else if (warp == 1 && lane == 0 && R > 0) {
        // ---- MMA issuer: one accumulator per input row
        bool ok = mbar_wait(wbar, 0, lim);
        int j = 0;
        for (; ok && j < rows_in; ++j) {
            ok = mbar_wait(&full[j % kStages], (uint32_t)(j / kStages) & 1u, lim);
            if (ok && j >= 2) ok = mbar_wait(&acce[j & 1], (uint32_t)((j >> 1) - 1) & 1u, lim);
            if (!ok || *stop) break;
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)((j & 1) * NF);
            const uint32_t slot = smem_u32(ring + (j % kStages) * SLOT);
            uint32_t acc = 0;
#pragma unroll
            for (int kx = 0; kx < 3; ++kx)
#pragma unroll
                for (int s = 0; s < KSTEPS; ++s) {
                    const uint64_t a = sdesc(slot + (uint32_t)(2 * s * kPlane + kx * 16), kPlane, 128);
                    const uint64_t b = sdesc(smem_u32(wsm) + (uint32_t)(((kx * KSTEPS + s) * 2 * NF) * 16), NF * 16, 128);
                    mma_bf16(d, a, b, ID, acc);
                    acc = 1;
                }
            mma_commit(&accf[j & 1]);
            mma_commit(&empty[j % kStages]);
        }
        if (!ok) {
            *stop = 1;
            atomicOr(status, 4);
        }
        // the MMAs issued last are done before anyone frees the tensor memory
        if (j > 0 && !mbar_wait(&accf[(j - 1) & 1], (uint32_t)((j - 1) >> 1) & 1u, lim)) atomicOr(status, 8);
    } else if (warp >= 2 && R > 0) {
        // ---- epilogue: pixel m of the strip = TMEM lane 32 (warp mod 4) + lane.
        // Before input row j: T1 = output row j - 2 without its last tap row,
        // T2 = output row j - 1 with its first only (band indices).
        constexpr int L = HIDDEN ? W : kOut;   // channels read back per row tap
        const int q = warp & 3;
        const int m = q * 32 + lane;
        const int x = x0 + m;
        float T1[L], T2[L], O[L];
#pragma unroll
        for (int n = 0; n < L; ++n) T1[n] = T2[n] = 0.0f;
        for (int j = 0; j < rows_in; ++j) {
            if (__any_sync(0xffffffffu, *stop != 0)) break;
            const bool mine = mbar_wait(&accf[j & 1], (uint32_t)(j >> 1) & 1u, lim);
            if (!__all_sync(0xffffffffu, mine)) {
                if (lane == 0) {
                    *stop = 1;
                    atomicOr(status, 16);
                }
                break;
            }
            tc_fence_after();
            const uint32_t t = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((j & 1) * NF);
            tmem_load<L>(t + 2 * W, O);        // third row tap: output row j - 2 is complete
#pragma unroll
            for (int n = 0; n < L; ++n) O[n] += T1[n];
            tmem_load<L>(t + W, T1);           // second row tap of output row j - 1
#pragma unroll
            for (int n = 0; n < L; ++n) T1[n] += T2[n];
            tmem_load<L>(t, T2);               // first row tap of output row j
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[j & 1]);
            const int y = y0 + j - 2;
            if (j >= 2 && x < nx) {
                if constexpr (HIDDEN) {
                    uint32_t pk[W / 2];
#pragma unroll
                    for (int n = 0; n < W / 2; ++n)
                        pk[n] = pack_bf16(fmaxf(O[2 * n] + __ldg(bias + 2 * n), 0.0f),
                                          fmaxf(O[2 * n + 1] + __ldg(bias + 2 * n + 1), 0.0f));
                    const size_t row = (size_t)(y + 1) * 4 * pitch;
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        const uint4 val = make_uint4(pk[4 * g], pk[4 * g + 1], pk[4 * g + 2], pk[4 * g + 3]);
                        uint8_t* plane = hout + (row + (size_t)g * pitch) * 16;
                        *reinterpret_cast<uint4*>(plane + (size_t)(x + 1) * 16) = val;
                        if (x == 0) *reinterpret_cast<uint4*>(plane + (size_t)(nx + 1) * 16) = val;
                        if (x == nx - 1) *reinterpret_cast<uint4*>(plane) = val;
                    }
                } else {
                    const size_t n = (size_t)nx * ny;
#pragma unroll
                    for (int c = 0; c < kOut; ++c) yout[(size_t)c * n + (size_t)y * nx + x] = O[c] + __ldg(bias + c);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL) : "memory");
    }
}

// Weights of one layer into the operand layout: [kx][K-step][group j][row n'][8]
// with row n' = ky W + n (the three row taps side by side) and channel
// c = (2 K-step + j) * 8 + e; zero for c >= cin, n >= cout or n' >= 3 W.
__global__ void weights_kernel(const float* __restrict__ w, int cin, int cout, int ksteps, int W, int NF,
                               __nv_bfloat16* __restrict__ out) {
    const int total = 3 * ksteps * 2 * NF * 8;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int e = i & 7;
        const int np = (i >> 3) % NF;
        const int j = (i / (8 * NF)) & 1;
        const int s = (i / (16 * NF)) % ksteps;
        const int kx = i / (16 * NF * ksteps);
        const int ky = np / W, n = np % W;
        const int c = (2 * s + j) * 8 + e;
        const float v = (c < cin && n < cout && ky < 3) ? w[(n * cin + c) * 9 + ky * 3 + kx] : 0.0f;
        out[i] = __float2bfloat16_rn(v);
    }
}

// Input planes (4 channels + 4 zeros, ghost columns, zero wall rows), the wall
// rows of the hidden planes, and (clear != 0) the status word.
__global__ void prep_kernel(const float* __restrict__ x, int nx, int ny, int pitch, uint8_t* __restrict__ xin,
                            uint8_t* __restrict__ h1, uint8_t* __restrict__ h2, int* __restrict__ status, int clear) {
    const size_t n = (size_t)nx * ny;
    const size_t total = (size_t)(ny + 2) * pitch;
    if (clear && blockIdx.x == 0 && threadIdx.x == 0) *status = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / pitch), p = (int)(i % pitch);
        uint4 val = make_uint4(0u, 0u, 0u, 0u);
        if (r >= 1 && r <= ny && p <= nx + 1) {
            const int xa = p == 0 ? nx - 1 : (p == nx + 1 ? 0 : p - 1);
            const size_t k = (size_t)(r - 1) * nx + xa;
            val.x = pack_bf16(x[k], x[n + k]);
            val.y = pack_bf16(x[2 * n + k], x[3 * n + k]);
        }
        reinterpret_cast<uint4*>(xin)[i] = val;
        if (r == 0 || r == ny + 1) {
            const uint4 z = make_uint4(0u, 0u, 0u, 0u);
            for (int g = 0; g < 4; ++g) {
                const size_t o = ((size_t)r * 4 + g) * pitch + p;
                reinterpret_cast<uint4*>(h1)[o] = z;
                reinterpret_cast<uint4*>(h2)[o] = z;
            }
        }
    }
}

struct Launch {
    int groups = 1, rows = 1;
};

// Bands of rows so that all CTAs of a layer are resident at once.
template <int KGG, int KG, int W, bool HIDDEN>
cudaError_t launch_conv(const Bufs& B, const uint8_t* in, const uint8_t* w, const float* bias, uint8_t* hout,
                        float* yout, cudaStream_t st, int withhold) {
    constexpr int SM = smem_bytes<KG, nfold(W)>();
    auto kern = conv_tc_kernel<KGG, KG, W, HIDDEN>;
    static bool configured = false;
    static int per_sm = 1, sms = 1;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        // resident CTAs per SM from the device limits: shared memory (1 KB of it
        // reserved per CTA), registers, threads, and the 512 tensor-memory columns
        int dev = 0, smem_sm = 0, regs_sm = 0, thr_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
        cudaFuncAttributes fa{};
        e = cudaFuncGetAttributes(&fa, kern);
        if (e != cudaSuccess) return e;
        const int regs = (std::max(fa.numRegs, 1) + 7) / 8 * 8 * kThreads;
        per_sm = std::min({smem_sm / (SM + 1024), regs_sm / regs, thr_sm / kThreads, 512 / (int)tmem_cols(nfold(W))});
        per_sm = std::max(1, per_sm);
        configured = true;
    }
    const int slots = sms * per_sm;
    int groups = std::max(1, slots / B.tiles_x);
    int rows = std::max(1, (B.ny + groups - 1) / groups);
    groups = (B.ny + rows - 1) / rows;
    conv_tc_kernel<KGG, KG, W, HIDDEN><<<dim3(B.tiles_x, groups), kThreads, SM, st>>>(in, w, bias, hout, yout, B.nx,
                                                                                      B.ny, B.pitch, rows, B.status,
                                                                                      withhold);
    return cudaGetLastError();
}

}  // namespace

size_t bytes(int nx, int ny) {
    const int tiles = (nx + kM - 1) / kM;
    const size_t pitch = (size_t)tiles * kM + 2;
    const size_t rows = (size_t)ny + 2;
    return align256(rows * pitch * 16) + 2 * align256(rows * 4 * pitch * 16) + align256(wbytes(2, nfold(32))) +
           align256(wbytes(4, nfold(32))) + align256(wbytes(4, nfold(kOut))) + 256;
}

Bufs carve(void* base, int nx, int ny) {
    Bufs B;
    B.nx = nx;
    B.ny = ny;
    B.tiles_x = (nx + kM - 1) / kM;
    B.pitch = B.tiles_x * kM + 2;
    const size_t rows = (size_t)ny + 2;
    uint8_t* p = static_cast<uint8_t*>(base);
    B.xin = p; p += align256(rows * B.pitch * 16);
    B.h1 = p; p += align256(rows * 4 * B.pitch * 16);
    B.h2 = p; p += align256(rows * 4 * B.pitch * 16);
    B.w1 = p; p += align256(wbytes(2, nfold(32)));
    B.w2 = p; p += align256(wbytes(4, nfold(32)));
    B.w3 = p; p += align256(wbytes(4, nfold(kOut)));
    B.status = reinterpret_cast<int*>(p);
    return B;
}

cudaError_t infer(const Bufs& B, const float* params, const float* x, float* y, cudaStream_t st, bool withhold,
                  bool clear_status) {
    const int wh = withhold ? 1 : 0;
    weights_kernel<<<8, 256, 0, st>>>(params + kW1, kIn, kHid, 1, kHid, nfold(kHid), reinterpret_cast<__nv_bfloat16*>(B.w1));
    weights_kernel<<<16, 256, 0, st>>>(params + kW2, kHid, kHid, 2, kHid, nfold(kHid), reinterpret_cast<__nv_bfloat16*>(B.w2));
    weights_kernel<<<4, 256, 0, st>>>(params + kW3, kHid, kOut, 2, kOut, nfold(kOut), reinterpret_cast<__nv_bfloat16*>(B.w3));
    const size_t px = (size_t)(B.ny + 2) * B.pitch;
    const int blocks = (int)std::min<size_t>(4096, (px + 255) / 256);
    prep_kernel<<<blocks, 256, 0, st>>>(x, B.nx, B.ny, B.pitch, B.xin, B.h1, B.h2, B.status,
                                                clear_status ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_conv<1, 2, 32, true>(B, B.xin, B.w1, params + kB1, B.h1, nullptr, st, wh);
    if (e != cudaSuccess) return e;
    e = launch_conv<4, 4, 32, true>(B, B.h1, B.w2, params + kB2, B.h2, nullptr, st, wh);
    if (e != cudaSuccess) return e;
    return launch_conv<4, 4, kOut, false>(B, B.h2, B.w3, params + kB3, nullptr, y, st, wh);
}

cudaError_t status(const Bufs& B, cudaStream_t st, int* out) {
    cudaError_t e = cudaMemcpyAsync(out, B.status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

}  // namespace cnn_tc
}  // namespace lbm
