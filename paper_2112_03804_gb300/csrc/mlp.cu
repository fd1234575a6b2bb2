// Warm-start network: a 3-layer perceptron with BF16 weights and FP32
// accumulation, trained and evaluated by the kernels in this file.
//
//   H1 = relu(X W1 + b1),  H2 = relu(H1 W2 + b2),  Z = H2 W3 + b3,
//   P[q, a] = softmax over the node's actions a < nact[q] of Z[q, :]
//
// Loss: weighted cross-entropy against target strategies T,
//   L = - sum_q w_q sum_{a < nact_q} T[q,a] log P[q,a] / sum_q w_q,
// whose gradient at the logits is dZ = w_q (P - T) / sum w (zero for a >= nact).
// Weights live in FP32 (master copy, Adam moments) and BF16 (what the
// forward and backward products read); activations and gradients are FP32.
// The products are one tiled SIMT kernel (64x64 tile, 16-deep k slices in
// shared memory, 4x4 outputs per thread) with generic strides, so the same
// code computes X W, dZ W^T and X^T dH.  Not in the paper: a service for
// warm-starting the solver (Sec. 2's first-order methods start from a given
// strategy).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "abi_internal.h"
#include "mlp_internal.h"

using namespace kps_abi;

namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16;

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// C(m,n) = sum_k A(m,k) B(k,n) [+ bias(n)] [relu] [* (gate(m,n) > 0)]
// A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn], C row-major ldc.
template <typename TA, typename TB>
__global__ void __launch_bounds__(256)
gemm_kernel(int M, int N, int K, const TA *__restrict__ A, long long sam, long long sak, const TB *__restrict__ B,
            long long sbk, long long sbn, float *__restrict__ C, long long ldc, const float *__restrict__ bias,
            int relu, const float *__restrict__ gate, long long ldg) {
    __shared__ float As[kBK][kBM + 4];
    __shared__ float Bs[kBK][kBN + 4];
    const int tid = threadIdx.x;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    const int tr = tid / 16, tc = tid % 16;   // 16 x 16 threads, 4 x 4 outputs each
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += kBK) {
        // 64 x 16 elements of each operand, 4 per thread
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int e = tid + 256 * i;
            // A tile: consecutive threads walk k when A is k-contiguous, else m
            int am, ak;
            if (sak == 1) { am = e / kBK; ak = e % kBK; } else { am = e % kBM; ak = e / kBM; }
            const int gm = m0 + am, gk = k0 + ak;
            As[ak][am] = (gm < M && gk < K) ? to_f<TA>(A[gm * sam + gk * sak]) : 0.f;
            int bk, bn;
            if (sbn == 1) { bk = e / kBN; bn = e % kBN; } else { bk = e % kBK; bn = e / kBK; }
            const int gk2 = k0 + bk, gn = n0 + bn;
            Bs[bk][bn] = (gk2 < K && gn < N) ? to_f<TB>(B[gk2 * sbk + gn * sbn]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tr + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tc + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + tr + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tc + 16 * j;
            if (n >= N) continue;
            float v = acc[i][j];
            if (bias) v += bias[n];
            if (relu) v = fmaxf(v, 0.f);
            if (gate && !(gate[(long long)m * ldg + n] > 0.f)) v = 0.f;
            C[(long long)m * ldc + n] = v;
        }
    }
}

// Column sums of G [M x N] (bias gradients): out[n] = sum_m G[m, n].
__global__ void colsum_kernel(int M, int N, const float *__restrict__ G, float *__restrict__ out) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int m = 0; m < M; ++m) s += G[(long long)m * N + n];
    out[n] = s;
}

// Masked softmax of each row; with targets: per-row loss terms and dZ.
// One thread per row (rows have at most 32 outputs).
__global__ void softmax_kernel(int Q, int D, const float *__restrict__ Z, const int *__restrict__ nact,
                               float *__restrict__ P, const float *__restrict__ T, const float *__restrict__ w,
                               float inv_wsum, float *__restrict__ dZ, float *__restrict__ row_loss) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q) return;
    const int na = nact[q];
    const float *z = Z + (long long)q * D;
    float mx = -INFINITY;
    for (int a = 0; a < na; ++a) mx = fmaxf(mx, z[a]);
    float s = 0.f;
    for (int a = 0; a < na; ++a) s += expf(z[a] - mx);
    const float ls = logf(s);
    float loss = 0.f;
    for (int a = 0; a < D; ++a) {
        const float p = a < na ? expf(z[a] - mx - ls) : 0.f;
        if (P) P[(long long)q * D + a] = p;
        if (T) {
            const float t = a < na ? T[(long long)q * D + a] : 0.f;
            if (a < na && t > 0.f) loss -= t * (z[a] - mx - ls);
            dZ[(long long)q * D + a] = a < na ? w[q] * inv_wsum * (p - t) : 0.f;
        }
    }
    if (T) row_loss[q] = w[q] * inv_wsum * loss;
}

__global__ void sum_kernel(int n, const float *__restrict__ v, float *__restrict__ out) {
    __shared__ float red[256];
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += 256) s += v[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// Adam on the FP32 master weights, then the BF16 copy.
__global__ void adam_kernel(long long n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, __nv_bfloat16 *__restrict__ ph, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (ph) ph[i] = __float2bfloat16_rn(pi);
}

__global__ void to_bf16_kernel(long long n, const float *__restrict__ p, __nv_bfloat16 *__restrict__ ph) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) ph[i] = __float2bfloat16_rn(p[i]);
}

template <typename TA, typename TB>
cudaError_t gemm(int M, int N, int K, const TA *A, long long sam, long long sak, const TB *B, long long sbk,
                 long long sbn, float *C, long long ldc, const float *bias, bool relu, const float *gate,
                 long long ldg, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM);
    if (grid.y > 65535) return cudaErrorInvalidValue;
    gemm_kernel<TA, TB><<<grid, 256, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, relu ? 1 : 0, gate,
                                               ldg);
    return cudaGetLastError();
}

}  // namespace

namespace kps_abi {

cudaError_t mlp_gemm_xw(int M, int N, int K, const float *A, long long lda, const __nv_bfloat16 *W, long long ldw,
                        float *C, long long ldc, cudaStream_t st) {
    return gemm<float, __nv_bfloat16>(M, N, K, A, lda, 1, W, ldw, 1, C, ldc, nullptr, false, nullptr, 0, st);
}

}  // namespace kps_abi

namespace {

kps_status ensure_cap(kps_mlp *m, int rows) {
    if (rows <= m->cap) return KPS_OK;
    cudaFree(m->H1);
    cudaFree(m->H2);
    cudaFree(m->Z);
    cudaFree(m->dZ);
    cudaFree(m->dH1);
    cudaFree(m->dH2);
    cudaFree(m->row_loss);
    m->H1 = m->H2 = m->Z = m->dZ = m->dH1 = m->dH2 = m->row_loss = nullptr;
    m->cap = 0;
    const size_t r = (size_t)rows;
    cudaError_t e = cudaMalloc(&m->H1, r * m->width * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->H2, r * m->width * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->Z, r * m->dout * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->dZ, r * m->dout * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->dH1, r * m->width * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->dH2, r * m->width * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->row_loss, r * 4);
    if (e != cudaSuccess) return fail(KPS_ENOMEM, "network activations");
    m->cap = rows;
    return KPS_OK;
}

const __nv_bfloat16 *Wh(const kps_mlp *m, int l) { return m->ph + m->off[2 * l]; }
const float *Bf(const kps_mlp *m, int l) { return m->p + m->off[2 * l + 1]; }

// Forward pass into H1, H2, Z (and P if given).
kps_status forward(kps_mlp *m, const float *X, int Q, const int *nact, float *P, cudaStream_t st) {
    const int D = m->din, W = m->width, O = m->dout;
    cudaError_t e = gemm<float, __nv_bfloat16>(Q, W, D, X, D, 1, Wh(m, 0), W, 1, m->H1, W, Bf(m, 0), true, nullptr, 0, st);
    if (e == cudaSuccess)
        e = gemm<float, __nv_bfloat16>(Q, W, W, m->H1, W, 1, Wh(m, 1), W, 1, m->H2, W, Bf(m, 1), true, nullptr, 0, st);
    if (e == cudaSuccess)
        e = gemm<float, __nv_bfloat16>(Q, O, W, m->H2, W, 1, Wh(m, 2), O, 1, m->Z, O, Bf(m, 2), false, nullptr, 0, st);
    if (e == cudaSuccess && P) {
        softmax_kernel<<<(Q + 127) / 128, 128, 0, st>>>(Q, O, m->Z, nact, P, nullptr, nullptr, 0.f, nullptr, nullptr);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(e, "network forward");
    return KPS_OK;
}

kps_status backward(kps_mlp *m, const float *X, int Q, const int *nact, const float *T, const float *w,
                    float inv_wsum, float *loss, cudaStream_t st) {
    const int D = m->din, W = m->width, O = m->dout;
    softmax_kernel<<<(Q + 127) / 128, 128, 0, st>>>(Q, O, m->Z, nact, nullptr, T, w, inv_wsum, m->dZ, m->row_loss);
    cudaError_t e = cudaGetLastError();
    float *g = m->g;
    // layer 3: dW3 = H2^T dZ, db3 = colsum dZ, dH2 = (dZ W3^T) * [H2 > 0]
    if (e == cudaSuccess)
        e = gemm<float, float>(W, O, Q, m->H2, 1, W, m->dZ, O, 1, g + m->off[4], O, nullptr, false, nullptr, 0, st);
    if (e == cudaSuccess) {
        colsum_kernel<<<(O + 127) / 128, 128, 0, st>>>(Q, O, m->dZ, g + m->off[5]);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = gemm<float, __nv_bfloat16>(Q, W, O, m->dZ, O, 1, Wh(m, 2), 1, O, m->dH2, W, nullptr, false, m->H2, W, st);
    // layer 2
    if (e == cudaSuccess)
        e = gemm<float, float>(W, W, Q, m->H1, 1, W, m->dH2, W, 1, g + m->off[2], W, nullptr, false, nullptr, 0, st);
    if (e == cudaSuccess) {
        colsum_kernel<<<(W + 127) / 128, 128, 0, st>>>(Q, W, m->dH2, g + m->off[3]);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = gemm<float, __nv_bfloat16>(Q, W, W, m->dH2, W, 1, Wh(m, 1), 1, W, m->dH1, W, nullptr, false, m->H1, W, st);
    // layer 1
    if (e == cudaSuccess)
        e = gemm<float, float>(D, W, Q, X, 1, D, m->dH1, W, 1, g + m->off[0], W, nullptr, false, nullptr, 0, st);
    if (e == cudaSuccess) {
        colsum_kernel<<<(W + 127) / 128, 128, 0, st>>>(Q, W, m->dH1, g + m->off[1]);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && loss) {
        sum_kernel<<<1, 256, 0, st>>>(Q, m->row_loss, loss);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(e, "network backward");
    return KPS_OK;
}

kps_status check_rows(const kps_mlp *m, const void *X, int Q) {
    if (!m) return fail(KPS_EINVAL, "network is NULL");
    if (Q < 0) return fail(KPS_EINVAL, "rows must be >= 0");
    if (Q > 0 && !X) return fail(KPS_EINVAL, "input is NULL");
    if ((long long)Q > 65535LL * kBM) return fail(KPS_ENOTSUP, "too many rows in one call (split the batch)");
    return KPS_OK;
}

}  // namespace

extern "C" {

kps_status kps_mlp_create(int32_t din, int32_t width, int32_t dout, uint64_t seed, kps_mlp **out) {
    if (!out) return fail(KPS_EINVAL, "out is NULL");
    *out = nullptr;
    if (din < 1 || width < 1 || dout < 1 || dout > 32) return fail(KPS_EINVAL, "bad layer sizes (dout <= 32)");
    kps_mlp *m = new (std::nothrow) kps_mlp;
    if (!m) return fail(KPS_ENOMEM, "network object");
    m->din = din;
    m->width = width;
    m->dout = dout;
    const long long sz[6] = {(long long)din * width, width, (long long)width * width, width, (long long)width * dout,
                             dout};
    for (int i = 0; i < 6; ++i) m->off[i + 1] = m->off[i] + sz[i];
    const long long n = m->off[6];
    // He initialisation (normal, std sqrt(2 / fan_in)), zero biases
    std::vector<float> host(n, 0.f);
    std::mt19937_64 rng(seed);
    const int fan[3] = {din, width, width};
    for (int l = 0; l < 3; ++l) {
        std::normal_distribution<float> nd(0.f, std::sqrt(2.f / fan[l]));
        for (long long i = m->off[2 * l]; i < m->off[2 * l + 1]; ++i) host[i] = nd(rng);
    }
    cudaError_t e = cudaMalloc(&m->p, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->g, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->m, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->v, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->ph, n * 2);
    if (e == cudaSuccess) e = cudaMalloc(&m->wsum, 4);
    if (e != cudaSuccess) {
        kps_mlp_destroy(m);
        return fail(KPS_ENOMEM, "network parameters");
    }
    e = cudaMemcpy(m->p, host.data(), n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->m, 0, n * 4);
    if (e == cudaSuccess) e = cudaMemset(m->v, 0, n * 4);
    if (e == cudaSuccess) e = cudaMemset(m->g, 0, n * 4);
    if (e == cudaSuccess) {
        to_bf16_kernel<<<(unsigned)((n + 255) / 256), 256>>>(n, m->p, m->ph);
        e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        kps_mlp_destroy(m);
        return cuda_fail(e, "initialising the network");
    }
    *out = m;
    return KPS_OK;
}

kps_status kps_mlp_destroy(kps_mlp *m) {
    if (!m) return KPS_OK;
    for (void *q : {(void *)m->p, (void *)m->g, (void *)m->m, (void *)m->v, (void *)m->ph, (void *)m->wsum,
                    (void *)m->H1, (void *)m->H2, (void *)m->Z, (void *)m->dZ, (void *)m->dH1, (void *)m->dH2,
                    (void *)m->row_loss})
        if (q) cudaFree(q);
    delete m;
    return KPS_OK;
}

kps_status kps_mlp_num_params(const kps_mlp *m, int64_t *n) {
    if (!m || !n) return fail(KPS_EINVAL, "bad argument");
    *n = m->off[6];
    return KPS_OK;
}

kps_status kps_mlp_get(const kps_mlp *m, int32_t which, float *host) {
    if (!m || !host || which < 0 || which > 1) return fail(KPS_EINVAL, "bad argument");
    cudaError_t e = cudaMemcpy(host, which == 0 ? m->p : m->g, m->off[6] * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the network");
    return KPS_OK;
}

kps_status kps_mlp_set(kps_mlp *m, const float *host) {
    if (!m || !host) return fail(KPS_EINVAL, "bad argument");
    cudaError_t e = cudaMemcpy(m->p, host, m->off[6] * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        to_bf16_kernel<<<(unsigned)((m->off[6] + 255) / 256), 256>>>(m->off[6], m->p, m->ph);
        e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) return cuda_fail(e, "writing the network");
    return KPS_OK;
}

// Checkpoint of a network (kps_mlp_save / kps_mlp_load): this header, then
// the FP32 parameters and Adam's first and second moments.
struct MlpCkpt {
    char magic[8];
    int32_t version, din, width, dout;
    int64_t step, n;
};
static const char kMlpMagic[8] = {'K', 'P', 'S', 'M', 'L', 'P', '0', '1'};

kps_status kps_mlp_state_bytes(const kps_mlp *m, int64_t *bytes) {
    if (!m || !bytes) return fail(KPS_EINVAL, "NULL argument");
    *bytes = (int64_t)sizeof(MlpCkpt) + 3 * 4 * m->off[6];
    return KPS_OK;
}

kps_status kps_mlp_save(const kps_mlp *m, void *host, int64_t bytes) {
    if (!m || !host) return fail(KPS_EINVAL, "NULL argument");
    const long long n = m->off[6];
    if (bytes < (int64_t)sizeof(MlpCkpt) + 12 * n) return fail(KPS_EINVAL, "buffer smaller than kps_mlp_state_bytes");
    MlpCkpt h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kMlpMagic, 8);
    h.version = 1;
    h.din = m->din;
    h.width = m->width;
    h.dout = m->dout;
    h.step = m->step;
    h.n = n;
    unsigned char *dst = static_cast<unsigned char *>(host);
    std::memcpy(dst, &h, sizeof(h));
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(dst + sizeof(h), m->p, 4 * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(dst + sizeof(h) + 4 * n, m->m, 4 * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(dst + sizeof(h) + 8 * n, m->v, 4 * n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "saving the network");
    return KPS_OK;
}

kps_status kps_mlp_load(kps_mlp *m, const void *host, int64_t bytes) {
    if (!m || !host) return fail(KPS_EINVAL, "NULL argument");
    if (bytes < (int64_t)sizeof(MlpCkpt)) return fail(KPS_EINVAL, "buffer too small for a checkpoint");
    MlpCkpt h;
    std::memcpy(&h, host, sizeof(h));
    if (std::memcmp(h.magic, kMlpMagic, 8) != 0 || h.version != 1) return fail(KPS_EINVAL, "not a network checkpoint");
    if (h.din != m->din || h.width != m->width || h.dout != m->dout || h.n != m->off[6])
        return fail(KPS_EINVAL, "checkpoint of a network with other layer sizes");
    const long long n = m->off[6];
    if (bytes < (int64_t)sizeof(MlpCkpt) + 12 * n) return fail(KPS_EINVAL, "checkpoint truncated");
    if (h.step < 0 || h.step > 0x7fffffffLL) return fail(KPS_EINVAL, "bad step count in the checkpoint");
    const unsigned char *src = static_cast<const unsigned char *>(host) + sizeof(h);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(m->p, src, 4 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->m, src + 4 * n, 4 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->v, src + 8 * n, 4 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        to_bf16_kernel<<<(unsigned)((n + 255) / 256), 256>>>(n, m->p, m->ph);
        e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) return cuda_fail(e, "loading the network");
    m->step = (int)h.step;
    return KPS_OK;
}

kps_status kps_mlp_forward(kps_mlp *m, const float *X, int32_t Q, const int32_t *nact, float *P, void *stream) {
    kps_status st = check_rows(m, X, Q);
    if (st != KPS_OK) return st;
    if (Q == 0) return KPS_OK;
    if (!nact || !P) return fail(KPS_EINVAL, "nact and P are required");
    st = ensure_cap(m, Q);
    if (st != KPS_OK) return st;
    return forward(m, X, Q, nact, P, static_cast<cudaStream_t>(stream));
}

kps_status kps_mlp_gradients(kps_mlp *m, const float *X, int32_t Q, const int32_t *nact, const float *T,
                             const float *w, float wsum, float *loss, void *stream) {
    kps_status st = check_rows(m, X, Q);
    if (st != KPS_OK) return st;
    if (Q == 0) return KPS_OK;
    if (!nact || !T || !w || !(wsum > 0.f)) return fail(KPS_EINVAL, "nact, T, w and wsum > 0 are required");
    st = ensure_cap(m, Q);
    if (st != KPS_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = forward(m, X, Q, nact, nullptr, s);
    if (st != KPS_OK) return st;
    return backward(m, X, Q, nact, T, w, 1.f / wsum, loss, s);
}

kps_status kps_mlp_adam(kps_mlp *m, float lr, float beta1, float beta2, float eps, void *stream) {
    if (!m) return fail(KPS_EINVAL, "network is NULL");
    m->step += 1;
    const float c1 = 1.f - std::pow(beta1, (float)m->step), c2 = 1.f - std::pow(beta2, (float)m->step);
    const long long n = m->off[6];
    adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        n, m->p, m->g, m->m, m->v, m->ph, lr, beta1, beta2, eps, c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "Adam step");
    return KPS_OK;
}

}  // extern "C"
