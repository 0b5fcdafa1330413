// Learned proposal: a small 1-D convolutional encoder whose embeddings rank
// the database series for one query, so that the series most likely to be
// near are scored exactly first (their k-th best distance becomes the
// threshold of the exact scan; the result never depends on the encoder).
//
// Network (fixed): input [len][16] (coordinates beyond d are zero)
//   conv1 (kernel 5, same padding, 16 -> 64) + bias, ReLU
//   conv2 (kernel 5, 64 -> 64) + bias, ReLU
//   conv3 (kernel 5, 64 -> 64) + bias, ReLU
//   mean over the series' positions -> h [64]
//   linear 64 -> 64 -> embedding e [64]
// Predicted distance of two series: ||e_a - e_b||^2.
//
// Arithmetic: BF16 operands on the tensor cores with FP32 accumulation: the
// convolutions and their gradients (mma.sync m16n8k16), the query x series
// scores of a scan (tcgen05.mma with the accumulator in tensor memory,
// score_tc.cu); the input and every convolution output are rounded to BF16
// once; pooling, the linear layer, the loss and Adam are FP32.  FP32 master
// weights.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace knn {

constexpr int ENC_CIN = 16;   // padded input coordinates
constexpr int ENC_C = 64;     // channels
constexpr int ENC_E = 64;     // embedding size
constexpr int ENC_K = 5;      // kernel taps

// Flat parameter layout (FP32 masters, gradients and Adam moments alike).
constexpr int ENC_OFF_W1 = 0;                                   // [5][16][64]
constexpr int ENC_OFF_B1 = ENC_OFF_W1 + ENC_K * ENC_CIN * ENC_C;
constexpr int ENC_OFF_W2 = ENC_OFF_B1 + ENC_C;                  // [5][64][64]
constexpr int ENC_OFF_B2 = ENC_OFF_W2 + ENC_K * ENC_C * ENC_C;
constexpr int ENC_OFF_W3 = ENC_OFF_B2 + ENC_C;                  // [5][64][64]
constexpr int ENC_OFF_B3 = ENC_OFF_W3 + ENC_K * ENC_C * ENC_C;
constexpr int ENC_OFF_WL = ENC_OFF_B3 + ENC_C;                  // [64 in][64 out]
constexpr int ENC_OFF_BL = ENC_OFF_WL + ENC_C * ENC_E;
constexpr int ENC_NPARAM = ENC_OFF_BL + ENC_E;

// Lowest predicted distance of each 64-series tile per query and its series
// ([nq][stride] each), on the tcgen05 tensor cores (score_tc.cu).
void launch_score_tc(const __nv_bfloat16 *eq, const float *nq2, int nq, const __nv_bfloat16 *ec,
                     const float *nc2, int n, float *score, int *tile_idx, int64_t stride,
                     int *status, cudaStream_t st);

}  // namespace knn
