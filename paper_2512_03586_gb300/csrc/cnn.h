// cnn.h -- learned regime switch: network layout and host launchers
// (internal to the library; the C ABI is in include/esbgk.h).
//
// Network (3 layers, receptive field 5 x 5 cells, 'same' zero padding):
//   x  : features [img][H][W][16] bf16 (channels 0..4 used, 5..15 zero)
//   a1 = relu(b1 + conv3x3(x, W1))   [img][H][W][32] bf16
//   a2 = relu(b2 + conv3x3(a1, W2))  [img][H][W][32] bf16
//   z  = b3 + a2 . w3                [img][H][W] float32 (logit)
// Parameters (float32 master copy, this order): W1 [32][3][3][5], b1[32],
// W2 [32][3][3][32], b2[32], w3[32], b3[1].
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace esbgk {
namespace cnn {

constexpr int kCin = 5, kCinPad = 16, kHid = 32;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kHid * 9 * kCin;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid * 9 * kHid;
constexpr int kOffW3 = kOffB2 + kHid;
constexpr int kOffB3 = kOffW3 + kHid;
constexpr int kParams = kOffB3 + 1;  // 10753
constexpr int kK1 = 9 * kCinPad;     // GEMM depth of layer 1 (taps x padded channels)
constexpr int kK2 = 9 * kHid;        // GEMM depth of layer 2
// reference cell size of the features (the 128 x 128 grid of the unit square)
constexpr double kDxRef = 1.0 / 128.0;

// Device weights of one network: float32 parameters and the bf16 GEMM
// operands (W1f [32][144], W2f [32][288] for the forward convolutions;
// W2d [32][288] = the flipped, transposed W2 of the input-gradient pass).
struct Weights {
  float* theta;
  __nv_bfloat16 *w1f, *w2f, *w2d;
};

size_t weights_bytes();
// Carve the weights out of `p` (256-byte aligned); returns bytes used.
size_t carve_weights(unsigned char* p, Weights& w);

// Launchers (all asynchronous on stream s).
void launch_pack(const Weights& w, cudaStream_t s);  // bf16 operands from theta
void launch_features(const double* U, const double* eps, int nc, double dx, __nv_bfloat16* x, cudaStream_t s);
// logits of n images of H x W cells (a1, a2: scratch activations); err:
// device error word (first int: code), set to 2 when a bounded wait for the
// tensor cores expired
void launch_forward(const Weights& w, const __nv_bfloat16* x, int n, int H, int W, __nv_bfloat16* a1,
                    __nv_bfloat16* a2, float* logits, int* err, cudaStream_t s);
// judge of the learned switch: flags (the criterion's map q) becomes
// q | (logit > 0); counters[0..3] += judged cells' (predicted, missed,
// extra, cells) against the previous prediction pred (when have_prev);
// pred := (logit > 0).
void launch_judge(uint8_t* flags, uint8_t* pred, const float* logits, int nc, int have_prev,
                  unsigned long long* counters, cudaStream_t s);

}  // namespace cnn
}  // namespace esbgk
