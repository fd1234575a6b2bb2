// Internal state of the warm-start network (mlp.cu) shared with warm.cu.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

struct kps_mlp {
    int din = 0, width = 0, dout = 0;
    // parameters: W1 [din x width], b1, W2 [width x width], b2, W3 [width x dout], b3
    long long off[7] = {};          // offsets of the six blocks in the flat arrays, total
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *ph = nullptr;
    int step = 0;
    // activations, sized for `cap` rows
    int cap = 0;
    float *H1 = nullptr, *H2 = nullptr, *Z = nullptr, *dZ = nullptr, *dH1 = nullptr, *dH2 = nullptr;
    float *row_loss = nullptr, *wsum = nullptr;
};

namespace kps_abi {

// C [M x N] = A [M x K] (FP32, row stride lda) * W [K x N] (BF16, row
// stride ldw), FP32 accumulation, C row stride ldc.
cudaError_t mlp_gemm_xw(int M, int N, int K, const float *A, long long lda, const __nv_bfloat16 *W, long long ldw,
                        float *C, long long ldc, cudaStream_t st);

}  // namespace kps_abi
