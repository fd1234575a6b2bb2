// Technique B's explicit-factor route (Sec. 4): A y = Ahat y + U M^-1 V^T y
// with Ahat, U, M and V^T materialised in CSR (built on the host by
// kps::technique_b_factors) and applied to a batch of vectors in the
// library's [batch][sequence][hs] layout, which is a column-major dense
// matrix with one column per vector.  Two backends:
//   0: this library's kernels: a CSR times dense-matrix product (one group
//      of lanes per sparse row and block of vectors) and, for M^-1, the
//      prefix sum over the hands of every player-1 sequence (M's first
//      block is I (x) D with D lower bidiagonal (1, -1); its inverse sums);
//   1: cuSPARSE: SpMM for V^T, Ahat and U, SpSM (sparse triangular solve
//      with many right-hand sides) for M, as the paper's GPU route does.
// The fused kernels of kernels_tmem.cu compute the same product without
// materialising anything; this path exists to compare against.
#include <cuda_runtime.h>
#include <cusparse.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "abi_internal.h"
#include "game.h"

using kps_abi::cuda_fail;
using kps_abi::fail;

namespace {

constexpr int kFactors = 4;   // Ahat, U, M, V^T (the order of kps_tb_export)

struct DevCsr {
    int *rowptr = nullptr, *col = nullptr;
    float *vf = nullptr;
    double *vd = nullptr;
};

}  // namespace

struct kps_tb {
    const kps_game *game = nullptr;
    kps::TechniqueB f;
    int64_t sizes[7] = {0};
    int device = -1;
    void *blob = nullptr;
    DevCsr d[kFactors];
    // V^T y and M^-1 V^T y for the current batch
    void *tmp = nullptr, *tmp2 = nullptr;
    size_t tmp_bytes = 0;
    // cuSPARSE state for the current (dtype, batch)
    cusparseHandle_t handle = nullptr;
    cusparseSpMatDescr_t sp[kFactors] = {nullptr, nullptr, nullptr, nullptr};
    cusparseDnMatDescr_t dy = nullptr, dout = nullptr, dt1 = nullptr, dt2 = nullptr;
    cusparseSpSMDescr_t spsm = nullptr;
    void *cbuf = nullptr;
    size_t cbuf_bytes = 0;
    int plan_batch = -1;
    kps_dtype plan_dt = KPS_F32;
};

namespace {

const kps::Csr &factor(const kps_tb *tb, int which) {
    switch (which) {
        case 0: return tb->f.ahat;
        case 1: return tb->f.u;
        case 2: return tb->f.m;
        default: return tb->f.vt;
    }
}

// ---- kernels -----------------------------------------------------------

// Y[b][row] (+)= sum_k val[k] X[b][col[k]] for every row and vector b.  A
// group of LPR lanes takes one (block of VB vectors, row); consecutive
// groups take consecutive rows, so the gathered entries of X stay in L1.
// Every lane of a warp reaches the shuffles (no early exit).
template <typename T, int LPR, int VB>
__global__ void __launch_bounds__(256) tb_spmm_kernel(int rows, const int *__restrict__ rowptr,
                                                      const int *__restrict__ col, const T *__restrict__ val,
                                                      const T *__restrict__ X, long long ldx, T *__restrict__ Y,
                                                      long long ldy, int batch, int accumulate) {
    const int lg = threadIdx.x % LPR;
    const long long gid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / LPR;
    const long long nvb = (batch + VB - 1) / VB;
    const bool active = gid < (long long)rows * nvb;
    const int row = active ? (int)(gid % rows) : 0;
    const int b0 = active ? (int)(gid / rows) * VB : 0;
    T acc[VB];
#pragma unroll
    for (int i = 0; i < VB; ++i) acc[i] = T(0);
    if (active) {
        const int ke = rowptr[row + 1];
        for (int k = rowptr[row] + lg; k < ke; k += LPR) {
            const long long c = col[k];
            const T v = val[k];
#pragma unroll
            for (int i = 0; i < VB; ++i)
                if (b0 + i < batch) acc[i] += v * X[(long long)(b0 + i) * ldx + c];
        }
    }
#pragma unroll
    for (int off = LPR / 2; off > 0; off >>= 1)
#pragma unroll
        for (int i = 0; i < VB; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], off, LPR);
    if (active && lg == 0) {
#pragma unroll
        for (int i = 0; i < VB; ++i) {
            if (b0 + i >= batch) break;
            T *y = Y + (long long)(b0 + i) * ldy + row;
            *y = accumulate ? *y + acc[i] : acc[i];
        }
    }
}

// In place: Z[b][s*hs + h] <- sum_{h' <= h} Z[b][s*hs + h'] for h < H (the
// inverse of I (x) D); one warp per (vector, player-1 sequence).
template <typename T>
__global__ void __launch_bounds__(256) tb_prefix_kernel(T *Z, long long ldz, int n1, int hs, int H, int batch) {
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= (long long)batch * n1) return;          // the whole warp leaves together
    T *z = Z + (w / n1) * ldz + (long long)(w % n1) * hs;
    T carry = T(0);
    for (int h0 = 0; h0 < H; h0 += 32) {
        const int h = h0 + lane;
        T v = h < H ? z[h] : T(0);
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const T t = __shfl_up_sync(0xffffffffu, v, off);
            if (lane >= off) v += t;
        }
        v += carry;
        if (h < H) z[h] = v;
        carry = __shfl_sync(0xffffffffu, v, 31);
    }
}

template <typename T, int LPR>
cudaError_t spmm(const kps::Csr &h, const DevCsr &d, const T *vals, const T *X, long long ldx, T *Y, long long ldy,
                 int batch, bool accumulate, cudaStream_t stream) {
    constexpr int VB = 8;
    const long long groups = (long long)h.rows * ((batch + VB - 1) / VB);
    const long long blocks = (groups * LPR + 255) / 256;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > INT_MAX) return cudaErrorInvalidValue;
    tb_spmm_kernel<T, LPR, VB><<<(unsigned)blocks, 256, 0, stream>>>(h.rows, d.rowptr, d.col, vals, X, ldx, Y, ldy,
                                                                        batch, accumulate ? 1 : 0);
    return cudaGetLastError();
}

template <typename T>
const T *dev_vals(const DevCsr &d);
template <>
const float *dev_vals<float>(const DevCsr &d) { return d.vf; }
template <>
const double *dev_vals<double>(const DevCsr &d) { return d.vd; }

template <typename T>
kps_status own_matvec(kps_tb *tb, const T *y, T *out, int batch, cudaStream_t stream) {
    const kps::HostGame &g = tb->game->host;
    const long long R = tb->f.ahat.rows, C = tb->f.ahat.cols, m = tb->f.vt.rows;
    T *t = static_cast<T *>(tb->tmp);
    cudaError_t e = spmm<T, 32>(tb->f.vt, tb->d[3], dev_vals<T>(tb->d[3]), y, C, t, m, batch, false, stream);
    if (e == cudaSuccess) {
        const long long warps = (long long)batch * g.n[0];
        const long long blocks = (warps * 32 + 255) / 256;
        if (blocks > INT_MAX) return fail(KPS_ENOTSUP, "batch too large");
        if (blocks > 0) tb_prefix_kernel<T><<<(unsigned)blocks, 256, 0, stream>>>(t, m, g.n[0], g.hs, g.H, batch);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = spmm<T, 32>(tb->f.ahat, tb->d[0], dev_vals<T>(tb->d[0]), y, C, out, R, batch, false, stream);
    if (e == cudaSuccess) e = spmm<T, 2>(tb->f.u, tb->d[1], dev_vals<T>(tb->d[1]), t, m, out, R, batch, true, stream);
    return e == cudaSuccess ? KPS_OK : cuda_fail(e, "Technique B product");
}

kps_status sp_fail(cusparseStatus_t s, const char *what) {
    return fail(KPS_ECUDA, std::string("cuSPARSE ") + what + ": " + cusparseGetErrorString(s));
}

void drop_plan(kps_tb *tb) {
    for (auto &s : tb->sp)
        if (s) cusparseDestroySpMat(s), s = nullptr;
    for (auto *dn : {&tb->dy, &tb->dout, &tb->dt1, &tb->dt2})
        if (*dn) cusparseDestroyDnMat(*dn), *dn = nullptr;
    if (tb->spsm) cusparseSpSM_destroyDescr(tb->spsm), tb->spsm = nullptr;
    tb->plan_batch = -1;
}

// cuSPARSE descriptors, buffers and the triangular-solve analysis for one
// (dtype, batch); the dense descriptors' pointers are reset every call.
kps_status cusparse_plan(kps_tb *tb, int batch, kps_dtype dt, const void *y, void *out) {
    if (tb->plan_batch == batch && tb->plan_dt == dt) return KPS_OK;
    drop_plan(tb);
    cusparseStatus_t s = CUSPARSE_STATUS_SUCCESS;
    if (!tb->handle && (s = cusparseCreate(&tb->handle)) != CUSPARSE_STATUS_SUCCESS) return sp_fail(s, "create");
    const cudaDataType ty = dt == KPS_F64 ? CUDA_R_64F : CUDA_R_32F;
    for (int w = 0; w < kFactors; ++w) {
        const kps::Csr &h = factor(tb, w);
        void *vals = dt == KPS_F64 ? static_cast<void *>(tb->d[w].vd) : static_cast<void *>(tb->d[w].vf);
        s = cusparseCreateCsr(&tb->sp[w], h.rows, h.cols, (int64_t)h.col.size(), tb->d[w].rowptr, tb->d[w].col, vals,
                              CUSPARSE_INDEX_32I, CUSPARSE_INDEX_32I, CUSPARSE_INDEX_BASE_ZERO, ty);
        if (s != CUSPARSE_STATUS_SUCCESS) return sp_fail(s, "CSR descriptor");
    }
    const int64_t R = tb->f.ahat.rows, C = tb->f.ahat.cols, m = tb->f.vt.rows;
    struct DnSpec { cusparseDnMatDescr_t *d; int64_t rows; void *p; } dns[] = {
        {&tb->dy, C, const_cast<void *>(y)}, {&tb->dout, R, out}, {&tb->dt1, m, tb->tmp}, {&tb->dt2, m, tb->tmp2}};
    for (const DnSpec &q : dns) {
        s = cusparseCreateDnMat(q.d, q.rows, batch, q.rows, q.p, ty, CUSPARSE_ORDER_COL);
        if (s != CUSPARSE_STATUS_SUCCESS) return sp_fail(s, "dense descriptor");
    }
    cusparseFillMode_t fill = CUSPARSE_FILL_MODE_LOWER;
    cusparseDiagType_t diag = CUSPARSE_DIAG_TYPE_NON_UNIT;
    if ((s = cusparseSpMatSetAttribute(tb->sp[2], CUSPARSE_SPMAT_FILL_MODE, &fill, sizeof(fill))) != CUSPARSE_STATUS_SUCCESS ||
        (s = cusparseSpMatSetAttribute(tb->sp[2], CUSPARSE_SPMAT_DIAG_TYPE, &diag, sizeof(diag))) != CUSPARSE_STATUS_SUCCESS)
        return sp_fail(s, "triangular attributes");
    const double one_d = 1.0, zero_d = 0.0;
    const float one_f = 1.0f, zero_f = 0.0f;
    const void *one = dt == KPS_F64 ? static_cast<const void *>(&one_d) : static_cast<const void *>(&one_f);
    const void *zero = dt == KPS_F64 ? static_cast<const void *>(&zero_d) : static_cast<const void *>(&zero_f);
    const cusparseOperation_t N = CUSPARSE_OPERATION_NON_TRANSPOSE;
    size_t need = 0, b = 0;
    struct Mm { int w; cusparseDnMatDescr_t in, o; } mms[] = {{3, tb->dy, tb->dt1}, {0, tb->dy, tb->dout}, {1, tb->dt2, tb->dout}};
    for (const Mm &q : mms) {
        s = cusparseSpMM_bufferSize(tb->handle, N, N, one, tb->sp[q.w], q.in, zero, q.o, ty, CUSPARSE_SPMM_ALG_DEFAULT, &b);
        if (s != CUSPARSE_STATUS_SUCCESS) return sp_fail(s, "SpMM buffer size");
        need = std::max(need, b);
    }
    if ((s = cusparseSpSM_createDescr(&tb->spsm)) != CUSPARSE_STATUS_SUCCESS) return sp_fail(s, "SpSM descriptor");
    s = cusparseSpSM_bufferSize(tb->handle, N, N, one, tb->sp[2], tb->dt1, tb->dt2, ty, CUSPARSE_SPSM_ALG_DEFAULT, tb->spsm, &b);
    if (s != CUSPARSE_STATUS_SUCCESS) return sp_fail(s, "SpSM buffer size");
    // the SpSM buffer must stay untouched between analysis and solve: it
    // goes after the SpMM region
    const size_t spmm_bytes = (need + 255) / 256 * 256;
    need = spmm_bytes + b;
    if (need > tb->cbuf_bytes) {
        if (tb->cbuf) cudaFree(tb->cbuf);
        tb->cbuf = nullptr;
        tb->cbuf_bytes = 0;
        cudaError_t e = cudaMalloc(&tb->cbuf, need > 0 ? need : 1);
        if (e != cudaSuccess) return fail(KPS_ENOMEM, "cuSPARSE workspace");
        tb->cbuf_bytes = need;
    }
    s = cusparseSpSM_analysis(tb->handle, N, N, one, tb->sp[2], tb->dt1, tb->dt2, ty, CUSPARSE_SPSM_ALG_DEFAULT, tb->spsm,
                              static_cast<char *>(tb->cbuf) + spmm_bytes);
    if (s != CUSPARSE_STATUS_SUCCESS) return sp_fail(s, "SpSM analysis");
    tb->plan_batch = batch;
    tb->plan_dt = dt;
    return KPS_OK;
}

kps_status cusparse_matvec(kps_tb *tb, const void *y, void *out, int batch, kps_dtype dt, cudaStream_t stream) {
    kps_status st = cusparse_plan(tb, batch, dt, y, out);
    if (st != KPS_OK) return st;
    cusparseStatus_t s = cusparseSetStream(tb->handle, stream);
    if (s != CUSPARSE_STATUS_SUCCESS) return sp_fail(s, "set stream");
    if ((s = cusparseDnMatSetValues(tb->dy, const_cast<void *>(y))) != CUSPARSE_STATUS_SUCCESS ||
        (s = cusparseDnMatSetValues(tb->dout, out)) != CUSPARSE_STATUS_SUCCESS)
        return sp_fail(s, "dense pointers");
    const cudaDataType ty = dt == KPS_F64 ? CUDA_R_64F : CUDA_R_32F;
    const double one_d = 1.0, zero_d = 0.0;
    const float one_f = 1.0f, zero_f = 0.0f;
    const void *one = dt == KPS_F64 ? static_cast<const void *>(&one_d) : static_cast<const void *>(&one_f);
    const void *zero = dt == KPS_F64 ? static_cast<const void *>(&zero_d) : static_cast<const void *>(&zero_f);
    const cusparseOperation_t N = CUSPARSE_OPERATION_NON_TRANSPOSE;
    const cusparseSpMMAlg_t alg = CUSPARSE_SPMM_ALG_DEFAULT;
    if ((s = cusparseSpMM(tb->handle, N, N, one, tb->sp[3], tb->dy, zero, tb->dt1, ty, alg, tb->cbuf)) != CUSPARSE_STATUS_SUCCESS)
        return sp_fail(s, "SpMM V^T");
    if ((s = cusparseSpSM_solve(tb->handle, N, N, one, tb->sp[2], tb->dt1, tb->dt2, ty, CUSPARSE_SPSM_ALG_DEFAULT,
                                tb->spsm)) != CUSPARSE_STATUS_SUCCESS)
        return sp_fail(s, "SpSM M");
    if ((s = cusparseSpMM(tb->handle, N, N, one, tb->sp[0], tb->dy, zero, tb->dout, ty, alg, tb->cbuf)) != CUSPARSE_STATUS_SUCCESS)
        return sp_fail(s, "SpMM Ahat");
    if ((s = cusparseSpMM(tb->handle, N, N, one, tb->sp[1], tb->dt2, one, tb->dout, ty, alg, tb->cbuf)) != CUSPARSE_STATUS_SUCCESS)
        return sp_fail(s, "SpMM U");
    return KPS_OK;
}

// Device copies of the four factors (FP32 and FP64 values), one allocation.
kps_status tb_upload(kps_tb *tb, cudaStream_t stream) {
    int dev = -1;
    cudaGetDevice(&dev);
    if (tb->blob) return dev == tb->device ? KPS_OK : fail(KPS_EINVAL, "factors live on another device");
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    size_t off = 0, o[kFactors][4];
    for (int w = 0; w < kFactors; ++w) {
        const kps::Csr &h = factor(tb, w);
        const size_t nnz = h.col.size();
        o[w][0] = off; off = al(off + 4 * (h.rowptr.size()));
        o[w][1] = off; off = al(off + 4 * nnz);
        o[w][2] = off; off = al(off + 4 * nnz);
        o[w][3] = off; off = al(off + 8 * nnz);
    }
    std::vector<unsigned char> host(off, 0);
    for (int w = 0; w < kFactors; ++w) {
        const kps::Csr &h = factor(tb, w);
        const size_t nnz = h.col.size();
        std::memcpy(host.data() + o[w][0], h.rowptr.data(), 4 * h.rowptr.size());
        if (nnz) std::memcpy(host.data() + o[w][1], h.col.data(), 4 * nnz);
        float *vf = reinterpret_cast<float *>(host.data() + o[w][2]);
        for (size_t i = 0; i < nnz; ++i) vf[i] = (float)h.val[i];
        if (nnz) std::memcpy(host.data() + o[w][3], h.val.data(), 8 * nnz);
    }
    void *blob = nullptr;
    cudaError_t e = cudaMalloc(&blob, off);
    if (e != cudaSuccess) return fail(KPS_ENOMEM, "Technique B factors");
    e = cudaMemcpyAsync(blob, host.data(), off, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        cudaFree(blob);
        return cuda_fail(e, "uploading Technique B factors");
    }
    unsigned char *b = static_cast<unsigned char *>(blob);
    for (int w = 0; w < kFactors; ++w) {
        tb->d[w].rowptr = reinterpret_cast<int *>(b + o[w][0]);
        tb->d[w].col = reinterpret_cast<int *>(b + o[w][1]);
        tb->d[w].vf = reinterpret_cast<float *>(b + o[w][2]);
        tb->d[w].vd = reinterpret_cast<double *>(b + o[w][3]);
    }
    tb->blob = blob;
    tb->device = dev;
    return KPS_OK;
}

}  // namespace

extern "C" {

kps_status kps_tb_create(const kps_game *game, kps_tb **out) {
    if (!game || !out) return fail(KPS_EINVAL, "NULL argument");
    *out = nullptr;
    try {
        std::unique_ptr<kps_tb> owner(new kps_tb());
        kps_tb *tb = owner.get();
        tb->game = game;
        kps::technique_b_factors(game->host, tb->f);
        const kps::HostGame &g = game->host;
        for (int w = 0; w < kFactors; ++w)
            if (factor(tb, w).col.size() > (size_t)INT_MAX) return fail(KPS_ENOTSUP, "factor with more than 2^31 nonzeros");
        const int64_t pad = (int64_t)g.n[0] * (g.hs - g.H);    // M's diagonal on padding rows
        tb->sizes[0] = tb->f.ahat.rows;
        tb->sizes[1] = tb->f.ahat.cols;
        tb->sizes[2] = tb->f.vt.rows;
        tb->sizes[3] = (int64_t)tb->f.ahat.col.size();
        tb->sizes[4] = (int64_t)tb->f.u.col.size();
        tb->sizes[5] = (int64_t)tb->f.m.col.size() - pad;
        tb->sizes[6] = (int64_t)tb->f.vt.col.size();
        *out = owner.release();
        return KPS_OK;
    } catch (const std::bad_alloc &) {
        return fail(KPS_ENOMEM, "Technique B factors");
    }
}

kps_status kps_tb_destroy(kps_tb *tb) {
    if (!tb) return KPS_OK;
    drop_plan(tb);
    if (tb->handle) cusparseDestroy(tb->handle);
    if (tb->cbuf) cudaFree(tb->cbuf);
    if (tb->tmp) cudaFree(tb->tmp);
    if (tb->blob) cudaFree(tb->blob);
    delete tb;
    return KPS_OK;
}

kps_status kps_tb_sizes(const kps_tb *tb, int64_t *sizes) {
    if (!tb || !sizes) return fail(KPS_EINVAL, "NULL argument");
    std::memcpy(sizes, tb->sizes, sizeof(tb->sizes));
    return KPS_OK;
}

kps_status kps_tb_export(const kps_tb *tb, int which, int64_t *shape, int32_t *rowptr, int32_t *col, double *val) {
    if (!tb || which < 0 || which >= kFactors) return fail(KPS_EINVAL, "bad factor");
    const kps::Csr &h = factor(tb, which);
    if (shape) {
        shape[0] = h.rows;
        shape[1] = h.cols;
        shape[2] = (int64_t)h.col.size();
    }
    if (rowptr) std::memcpy(rowptr, h.rowptr.data(), 4 * h.rowptr.size());
    if (col && !h.col.empty()) std::memcpy(col, h.col.data(), 4 * h.col.size());
    if (val && !h.val.empty()) std::memcpy(val, h.val.data(), 8 * h.val.size());
    return KPS_OK;
}

kps_status kps_tb_matvec(kps_tb *tb, const void *y, void *out, int32_t batch, kps_dtype dt, int32_t backend,
                         void *stream_ptr) {
    if (!tb || !y || !out) return fail(KPS_EINVAL, "NULL argument");
    if (batch < 0) return fail(KPS_EINVAL, "negative batch");
    if (dt != KPS_F32 && dt != KPS_F64) return fail(KPS_ENOTSUP, "Technique B product: FP32 or FP64 only");
    if (backend != 0 && backend != 1) return fail(KPS_EINVAL, "backend is 0 (own kernels) or 1 (cuSPARSE)");
    if (batch == 0) return KPS_OK;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    kps_status st = tb_upload(tb, stream);
    if (st != KPS_OK) return st;
    const size_t es = dt == KPS_F64 ? 8 : 4;
    const size_t one = (size_t)batch * tb->f.vt.rows * es;
    if (2 * one > tb->tmp_bytes) {
        if (tb->plan_batch >= 0) drop_plan(tb);        // its dense descriptors point at the old buffers
        if (tb->tmp) cudaFree(tb->tmp);
        tb->tmp = tb->tmp2 = nullptr;
        tb->tmp_bytes = 0;
        if (cudaMalloc(&tb->tmp, 2 * one) != cudaSuccess) return fail(KPS_ENOMEM, "Technique B workspace");
        tb->tmp_bytes = 2 * one;
    }
    tb->tmp2 = static_cast<char *>(tb->tmp) + one;
    if (backend == 1) return cusparse_matvec(tb, y, out, batch, dt, stream);
    return dt == KPS_F64 ? own_matvec<double>(tb, static_cast<const double *>(y), static_cast<double *>(out), batch, stream)
                         : own_matvec<float>(tb, static_cast<const float *>(y), static_cast<float *>(out), batch, stream);
}

}  // extern "C"
