// Tensor-core (tcgen05) inference path of the closure CNN: conv3x3 4->32, ReLU,
// conv3x3 32->32, ReLU, conv3x3 32->4 with BF16 weights and activations and FP32
// accumulation in tensor memory.  Host-side interface; kernels in cnn_tc.cu.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace lbm {
namespace cnn_tc {

// Activation planes: rows 0 and ny + 1 are zero (the walls), columns 0 and
// nx + 1 repeat columns nx - 1 and 0 (periodic x); pixel (y, x) sits at padded
// row y + 1, column x + 1.  A plane row holds `pitch` pixels of 8 BF16 channels
// (16 bytes), the channel groups of one row follow each other:
//   byte offset of (padded row r, group g, padded column p) = ((r * G + g) * pitch + p) * 16.
struct Bufs {
    int nx = 0, ny = 0, tiles_x = 0, pitch = 0;
    uint8_t* xin = nullptr;   // G = 1: the 4 input channels + 4 zero channels
    uint8_t* h1 = nullptr;    // G = 4: 32 hidden channels after the first ReLU
    uint8_t* h2 = nullptr;    // G = 4: after the second ReLU
    uint8_t* w1 = nullptr;    // weights in the tensor cores' shared-memory operand layout
    uint8_t* w2 = nullptr;
    uint8_t* w3 = nullptr;
    int* status = nullptr;    // nonzero after a bounded wait gave up
};

size_t bytes(int nx, int ny);
Bufs carve(void* base, int nx, int ny);
// y[4][ny][nx] = CNN(x[4][ny][nx]); params as in the FP32 path.  Asynchronous.
// withhold (tests of the timeout path only): the kernels issue no copies and poll
// briefly, so their waits give up and raise the status word.  clear_status: the
// status word starts from 0; without it a failure of an earlier call stays raised.
cudaError_t infer(const Bufs& B, const float* params, const float* x, float* y, cudaStream_t st,
                  bool withhold = false, bool clear_status = true);
// Reads the status word (synchronises the stream): 0 if every wait completed.
cudaError_t status(const Bufs& B, cudaStream_t st, int* out);

}  // namespace cnn_tc
}  // namespace lbm
