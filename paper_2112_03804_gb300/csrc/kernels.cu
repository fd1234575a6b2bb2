// Kronecker-form payoff products for GB300 (sm_103a).
//
// For one output column (output sequence sigma, batch vector b) the product
// of Prop. 1 reads, in the library's strength order of hands,
//
//   u = lambda_in * F_sigma * x[fcol]     (fold terminal of sigma, if any)
//   v = lambda_in * S_sigma * x[scol]     (showdown terminal of sigma, if any)
//   out = lambda_out * ( K_F(u) + K_W(v) )
//
// where K_F(u)[h] = sum of u over hands compatible with h (card removal, the
// sparsified fold term "cf" of Sec. 4: all hands, minus the hands holding a
// card of h, plus h itself for two-card hands) and K_W(v)[h] = sum of v over
// compatible hands that h beats minus over those that beat h (the strength
// sign W of Sec. 3 applied through prefix sums, i.e. the inverse of the
// bidiagonal D of Technique B, Sec. 4).  With Lo[h] = compatible strictly
// weaker mass and TieC[h] = compatible equal-strength mass,
//   K_W(v) = 2 Lo(v) - K_F(v) + TieC(v),
// so out/lambda_out = K_F(u - v) + 2 Lo(v) + TieC(v): one fold operator
// (needs per-card totals) and one strength-ordered scan (needs per-card
// running sums).
//
// Work decomposition ("lane = column"): each CTA owns 32 output columns, one
// per lane; all lanes walk the same hand order, so the card indices of a step
// are warp-uniform and every per-card table access Table[card][lane] is
// bank-conflict free.  The hand range is split into `nw` tie-aligned chunks,
// one per warp.  Phase 1 scans a chunk with chunk-local per-card sums and
// keeps a partial result per (hand, column) in shared memory; phase 2
// combines the chunk sums across warps; phase 3 adds the cross-chunk and fold
// terms; phase 4 writes the columns out coalesced.  Inputs are staged per
// 32-hand tile with coalesced loads (lane = hand) and transposed through
// shared memory.  No atomics: results are bit-reproducible.
#include "kernels.h"

#include <map>
#include <mutex>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

namespace kps {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kPad = 33;   // row pitch of [hand][column] buffers

template <typename S> struct Store;
template <> struct Store<float> {
    using C = float;
    __device__ static C load(const float *p) { return __ldg(p); }
    __device__ static float conv(C x) { return x; }
};
template <> struct Store<double> {
    using C = double;
    __device__ static C load(const double *p) { return __ldg(p); }
    __device__ static double conv(C x) { return x; }
};
template <> struct Store<__nv_bfloat16> {
    using C = float;
    __device__ static C load(const __nv_bfloat16 *p) {
        return __bfloat162float(__ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short *>(p))));
    }
    __device__ static __nv_bfloat16 conv(C x) { return __float2bfloat16_rn(x); }
};
template <> struct Store<__half> {
    using C = float;
    __device__ static C load(const __half *p) {
        return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short *>(p))));
    }
    __device__ static __half conv(C x) { return __float2half_rn(x); }
};

struct ColInfo {
    long long in_off;    // element offset of the column's input vector
    long long out_off;   // element offset of the output row, -1 = no column
    int foff, soff;      // input row offsets (sequence * hs), -1 = no term
};

template <typename C>
struct Layout {
    ColInfo *ci;
    C *fco, *sco;    // [32] terminal payoffs per column
    C *sums;         // [nw][3][32]: chunk mass of v, of w, then the base term
    C *tables;       // nw blocks of: Rv, Rw, Pc [nc][32], stf, sts [32][kPad]
    C *partial;      // [H][kPad] (when kept in shared memory)
    size_t per_warp;
};

template <typename C>
__device__ Layout<C> carve(unsigned char *raw, int nc, int nw, int H, bool pin) {
    Layout<C> L;
    L.ci = reinterpret_cast<ColInfo *>(raw);
    L.fco = reinterpret_cast<C *>(raw + 32 * sizeof(ColInfo));
    L.sco = L.fco + 32;
    L.sums = L.sco + 32;
    L.tables = L.sums + (size_t)nw * 3 * 32;
    L.per_warp = 3 * (size_t)nc * 32 + 2 * 32 * kPad;
    L.partial = pin ? L.tables + nw * L.per_warp : nullptr;
    (void)H;
    return L;
}

template <typename S, int K2, bool PIN>
__global__ void __launch_bounds__(32 * kMaxWarps)
pair_scan_kernel(const ScanParams p) {
    using C = typename Store<S>::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = p.nw, nc = p.nc;
    const int H = p.H;
    Layout<C> L = carve<C>(smem_raw, nc, nw, H, PIN);
    const S *vin = static_cast<const S *>(p.vin);
    S *vout = static_cast<S *>(p.vout);
    const C *lam_in = static_cast<const C *>(p.lam_in);
    const C *lam_out = static_cast<const C *>(p.lam_out);

    // ---- column set-up (warp 0): which terminal pairs feed each column
    int kinds = 0;
    if (threadIdx.x < 32) {
        const long long col = (long long)blockIdx.x * 32 + threadIdx.x;
        ColInfo c;
        C f = C(0), s = C(0);
        if (col < (long long)p.n_out * p.batch) {
            const int sg = (int)(col / p.batch), b = (int)(col % p.batch);
            const int fc = p.fcol[sg], sc = p.scol[sg];
            c.in_off = (long long)b * p.n_in * p.hs;
            c.out_off = ((long long)b * p.n_out + sg) * p.hs;
            c.foff = fc >= 0 ? fc * p.hs : -1;
            c.soff = sc >= 0 ? sc * p.hs : -1;
            if (fc >= 0) f = static_cast<const C *>(p.fcoef)[sg];
            if (sc >= 0) s = static_cast<const C *>(p.scoef)[sg];
        } else {
            c.in_off = 0;
            c.out_off = -1;
            c.foff = c.soff = -1;
        }
        L.ci[threadIdx.x] = c;
        L.fco[threadIdx.x] = f;
        L.sco[threadIdx.x] = s;
        kinds = (c.foff >= 0 ? 1 : 0) | (c.soff >= 0 ? 2 : 0);
    }
    const bool has_f = __syncthreads_or(kinds & 1) != 0;   // also publishes L.ci
    const bool has_s = __syncthreads_or(kinds & 2) != 0;
    // Common case: the CTA's valid columns share one output sequence and
    // take consecutive batch vectors, so input addresses are arithmetic.
    const ColInfo c0i = L.ci[0];
    int same = 1, nvalid_l = 0;
    if (threadIdx.x < 32) {
        const ColInfo c = L.ci[threadIdx.x];
        if (c.out_off >= 0) {
            nvalid_l = 1;
            same = c.foff == c0i.foff && c.soff == c0i.soff &&
                   c.in_off == c0i.in_off + (long long)threadIdx.x * p.n_in * p.hs;
        }
    }
    const bool uni = __syncthreads_and(same) != 0;
    const int nvalid = __syncthreads_count(nvalid_l);
    const long long ustride = (long long)p.n_in * p.hs;

    C *Rv = L.tables + warp * L.per_warp;     // running per-card mass of v
    C *Rw = Rv + (size_t)nc * 32;             // per-card totals of w = u - v
    C *Pc = Rw + (size_t)nc * 32;             // pending per-card mass of a tie group
    C *stf = Pc + (size_t)nc * 32;            // staged lambda_in * x[fcol]
    C *sts = stf + 32 * kPad;                 // staged lambda_in * x[scol]
    for (int c = 0; c < nc; ++c) {
        Rv[c * 32 + lane] = C(0);
        Rw[c * 32 + lane] = C(0);
        Pc[c * 32 + lane] = C(0);
    }
    const ColInfo mine = L.ci[lane];
    const C fco = L.fco[lane], sco = L.sco[lane];
    // partial results: shared memory, or (wide FP64 games) the output row itself
    S *prow = (!PIN && mine.out_off >= 0) ? vout + mine.out_off : nullptr;
    C dummy_slot = C(0);
    C *const dummy = &dummy_slot;   // target of writes for columns past the end
    auto Pref = [&](int q) -> C & {
        if constexpr (PIN) {
            return L.partial[(size_t)q * kPad + lane];
        } else {
            static_assert(std::is_same<S, C>::value, "in-place partials need S == C");
            if (prow) return *reinterpret_cast<C *>(prow + q);
            return *dummy;
        }
    };

    // ---- phase 1: chunk-local scan
    const int c0 = p.chunk[warp], c1 = p.chunk[warp + 1];
    C Gv = C(0), Gw = C(0), Pg = C(0);
    // Inputs of the next 32-hand tile, lane = hand, one register per column:
    // issued before the current tile is scanned so that DRAM latency overlaps
    // the scan.
    C xf[32], xs[32];
    C lin_next = C(0);
    uint32_t h_next = 0u;
    auto fetch = [&](int t0) {
        const int pos = t0 + lane;
        const bool pin = pos < c1;
        lin_next = pin ? lam_in[pos] : C(0);
        h_next = pin ? __ldg(&p.hinfo[pos]) : 0u;
        if (uni) {
            const S *fb = vin + c0i.in_off + pos + c0i.foff;
            const S *sb = vin + c0i.in_off + pos + c0i.soff;
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
                const bool ok = pin && jj < nvalid;
                xf[jj] = (ok && c0i.foff >= 0) ? Store<S>::load(fb + jj * ustride) : C(0);
                xs[jj] = (ok && c0i.soff >= 0) ? Store<S>::load(sb + jj * ustride) : C(0);
            }
        } else {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
                const ColInfo cj = L.ci[jj];
                const S *base = vin + cj.in_off + pos;
                xf[jj] = (pin && cj.foff >= 0) ? Store<S>::load(base + cj.foff) : C(0);
                xs[jj] = (pin && cj.soff >= 0) ? Store<S>::load(base + cj.soff) : C(0);
            }
        }
    };
    // One hand of the scan (single step, ties deferred to the group end).
    auto step1 = [&](int i, uint32_t hi, int q) {
        const int ca = hi & 63, cb = (hi >> 6) & 63;
        const C u = fco * stf[i * kPad + lane];
        const C v = sco * sts[i * kPad + lane];
        const C w = u - v;
        if (has_s) {
            const C ra = Rv[ca * 32 + lane];
            const C rb = K2 == 2 ? Rv[cb * 32 + lane] : C(0);
            const C lo = Gv - ra - rb;                  // compatible, strictly weaker
            if (!(hi & (1u << 12))) {
                Pref(q) = (K2 == 2 ? w : C(0)) + C(2) * lo;
                Rv[ca * 32 + lane] = ra + v;
                if (K2 == 2) Rv[cb * 32 + lane] = rb + v;
                Gv += v;
            } else {
                // tie group: updates wait until its last member
                Pref(q) = (K2 == 2 ? w + v : C(0)) + C(2) * lo;
                Pc[ca * 32 + lane] += v;
                if (K2 == 2) Pc[cb * 32 + lane] += v;
                Pg += v;
                if (hi & (1u << 13)) {
                    const int q0 = q - (int)(hi >> 16);
                    // compatible equal-strength mass, by inclusion-exclusion
                    for (int r = q0; r <= q; ++r) {
                        const uint32_t hr = __ldg(&p.hinfo[r]);
                        C t = Pg - Pc[(hr & 63) * 32 + lane];
                        if (K2 == 2) t -= Pc[((hr >> 6) & 63) * 32 + lane];
                        Pref(r) += t;
                    }
                    for (int r = q0; r <= q; ++r) {
                        const uint32_t hr = __ldg(&p.hinfo[r]);
                        const int a = hr & 63;
                        Rv[a * 32 + lane] += Pc[a * 32 + lane];
                        Pc[a * 32 + lane] = C(0);
                        if (K2 == 2) {
                            const int b = (hr >> 6) & 63;
                            Rv[b * 32 + lane] += Pc[b * 32 + lane];
                            Pc[b * 32 + lane] = C(0);
                        }
                    }
                    Gv += Pg;
                    Pg = C(0);
                }
            }
        } else {
            Pref(q) = K2 == 2 ? w : C(0);
        }
        if (has_f) {
            Rw[ca * 32 + lane] += w;
            if (K2 == 2) Rw[cb * 32 + lane] += w;
            Gw += w;
        }
    };
    // Two consecutive untied hands with disjoint cards: all per-card loads
    // are independent, so they are issued together (same result as two
    // single steps).
    auto step2 = [&](int i, uint32_t h1, uint32_t h2, int q) {
        const int a1 = h1 & 63, b1 = (h1 >> 6) & 63, a2 = h2 & 63, b2 = (h2 >> 6) & 63;
        const C u1 = fco * stf[i * kPad + lane], v1 = sco * sts[i * kPad + lane];
        const C u2 = fco * stf[(i + 1) * kPad + lane], v2 = sco * sts[(i + 1) * kPad + lane];
        const C w1 = u1 - v1, w2 = u2 - v2;
        if (has_s) {
            const C ra1 = Rv[a1 * 32 + lane], ra2 = Rv[a2 * 32 + lane];
            const C rb1 = K2 == 2 ? Rv[b1 * 32 + lane] : C(0);
            const C rb2 = K2 == 2 ? Rv[b2 * 32 + lane] : C(0);
            const C lo1 = Gv - ra1 - rb1;
            const C g1 = Gv + v1;
            const C lo2 = g1 - ra2 - rb2;
            Pref(q) = (K2 == 2 ? w1 : C(0)) + C(2) * lo1;
            Pref(q + 1) = (K2 == 2 ? w2 : C(0)) + C(2) * lo2;
            Rv[a1 * 32 + lane] = ra1 + v1;
            Rv[a2 * 32 + lane] = ra2 + v2;
            if (K2 == 2) {
                Rv[b1 * 32 + lane] = rb1 + v1;
                Rv[b2 * 32 + lane] = rb2 + v2;
            }
            Gv = g1 + v2;
        } else {
            Pref(q) = K2 == 2 ? w1 : C(0);
            Pref(q + 1) = K2 == 2 ? w2 : C(0);
        }
        if (has_f) {
            const C fa1 = Rw[a1 * 32 + lane], fa2 = Rw[a2 * 32 + lane];
            const C fb1 = K2 == 2 ? Rw[b1 * 32 + lane] : C(0);
            const C fb2 = K2 == 2 ? Rw[b2 * 32 + lane] : C(0);
            Rw[a1 * 32 + lane] = fa1 + w1;
            Rw[a2 * 32 + lane] = fa2 + w2;
            if (K2 == 2) {
                Rw[b1 * 32 + lane] = fb1 + w1;
                Rw[b2 * 32 + lane] = fb2 + w2;
            }
            Gw = (Gw + w1) + w2;
        }
    };
    if (c0 < c1) fetch(c0);
    for (int t0 = c0; t0 < c1; t0 += 32) {
        const int len = min(32, c1 - t0);
        const C lin = lin_next;
        const uint32_t hreg = h_next;
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
            stf[lane * kPad + jj] = lin * xf[jj];
            sts[lane * kPad + jj] = lin * xs[jj];
        }
        __syncwarp();
        if (t0 + 32 < c1) fetch(t0 + 32);
        for (int i = 0; i < len;) {
            const uint32_t h1 = __shfl_sync(kFull, hreg, i);
            const uint32_t h2 = __shfl_sync(kFull, hreg, min(i + 1, 31));
            if ((h1 & (1u << 14)) && i + 1 < len) {
                step2(i, h1, h2, t0 + i);
                i += 2;
            } else {
                step1(i, h1, t0 + i);
                i += 1;
            }
        }
        __syncwarp();
    }
    L.sums[(warp * 3 + 0) * 32 + lane] = Gv;
    L.sums[(warp * 3 + 1) * 32 + lane] = Gw;
    __syncthreads();

    // ---- phase 2: chunk offsets.  Z[k][c] = Pw[c] + 2 Xv[k][c] replaces Rv_k, where
    // Xv[k][c] is the mass of card c in earlier chunks (removed from Lo).
    for (int c = warp; c < nc; c += nw) {
        C pw = C(0);
        for (int k = 0; k < nw; ++k) {
            const C *Tk = L.tables + k * L.per_warp;
            pw += has_f ? Tk[(size_t)nc * 32 + c * 32 + lane] : -Tk[c * 32 + lane];
        }
        C xv = C(0);
        for (int k = 0; k < nw; ++k) {
            C *Tk = L.tables + k * L.per_warp;
            const C r = Tk[c * 32 + lane];
            Tk[c * 32 + lane] = pw + C(2) * xv;
            xv += r;
        }
    }
    if (warp == 0) {
        C tw = C(0);
        for (int k = 0; k < nw; ++k)
            tw += has_f ? L.sums[(k * 3 + 1) * 32 + lane] : -L.sums[(k * 3 + 0) * 32 + lane];
        C xg = C(0);
        for (int k = 0; k < nw; ++k) {
            L.sums[(k * 3 + 2) * 32 + lane] = tw + C(2) * xg;
            xg += L.sums[(k * 3 + 0) * 32 + lane];
        }
    }
    __syncthreads();

    // ---- phase 3: fold totals and cross-chunk scan terms (4 hands per round:
    // every load of the round is issued before its stores)
    {
        const C base = L.sums[(warp * 3 + 2) * 32 + lane];
        const C *Z = Rv;
        int q = c0;
        for (; q + 4 <= c1; q += 4) {
            uint32_t hq[4];
            C pv[4], za[4], zb[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) hq[j] = __ldg(&p.hinfo[q + j]);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                pv[j] = Pref(q + j);
                za[j] = Z[(hq[j] & 63) * 32 + lane];
                zb[j] = K2 == 2 ? Z[((hq[j] >> 6) & 63) * 32 + lane] : C(0);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) Pref(q + j) = pv[j] + base - za[j] - zb[j];
        }
        for (; q < c1; ++q) {
            const uint32_t hq = __ldg(&p.hinfo[q]);
            C val = Pref(q) + base - Z[(hq & 63) * 32 + lane];
            if (K2 == 2) val -= Z[((hq >> 6) & 63) * 32 + lane];
            Pref(q) = val;
        }
    }
    __syncthreads();

    // ---- phase 4: scale by lambda_out, write out (padding zeroed)
    if (PIN) {
        for (int jj = warp; jj < 32; jj += nw) {
            const ColInfo cj = L.ci[jj];
            if (cj.out_off < 0) continue;
            S *dst = vout + cj.out_off;
            for (int q = lane; q < p.hs; q += 32) {
                C val = C(0);
                if (q < H) val = lam_out[q] * L.partial[(size_t)q * kPad + jj];
                dst[q] = Store<S>::conv(val);
            }
        }
    } else if (prow) {
        // each warp scales its own chunk of the lane's row; the last one pads
        for (int q = c0; q < c1; ++q) prow[q] = Store<S>::conv(lam_out[q] * Pref(q));
        if (warp == nw - 1)
            for (int q = H; q < p.hs; ++q) prow[q] = Store<S>::conv(C(0));
    }
}

template <typename S, int K2, bool PIN>
cudaError_t launch_t(const ScanParams &p, size_t smem, cudaStream_t stream) {
    auto fn = pair_scan_kernel<S, K2, PIN>;
    cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void *>(fn), smem);
    if (e != cudaSuccess) return e;
    const long long ncols = (long long)p.n_out * p.batch;
    const long long blocks = (ncols + kColsPerCta - 1) / kColsPerCta;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    fn<<<(unsigned)blocks, 32 * p.nw, smem, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace

size_t scan_smem_bytes(int storage, int H, int nc, int nw, bool pin) {
    const size_t cs = storage == kStoreF64 ? 8 : 4;
    size_t bytes = 32 * sizeof(ColInfo) + 2 * 32 * cs + (size_t)nw * 3 * 32 * cs;
    bytes += (size_t)nw * (3 * (size_t)nc * 32 + 2 * 32 * kPad) * cs;
    if (pin) bytes += (size_t)H * kPad * cs;
    return bytes;
}

cudaError_t ensure_dyn_smem(const void *fn, size_t smem) {
    // the limit is a per-device property of the kernel: remember, per
    // (kernel, device), the largest size already set
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t &have = done[std::make_pair(fn, dev)];
    if (have >= smem) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    have = smem;
    return cudaSuccess;
}

int max_dyn_smem() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    return v;
}

cudaError_t launch_pair_scan(const ScanParams &p, int storage, int k, bool pin, cudaStream_t stream) {
    const size_t smem = scan_smem_bytes(storage, p.H, p.nc, p.nw, pin);
#define KPS_DISPATCH(S)                                                          \
    if (k == 1) return pin ? launch_t<S, 1, true>(p, smem, stream)               \
                           : launch_t<S, 1, false>(p, smem, stream);             \
    return pin ? launch_t<S, 2, true>(p, smem, stream) : launch_t<S, 2, false>(p, smem, stream);
    switch (storage) {
        case kStoreF32: { KPS_DISPATCH(float) }
        case kStoreF64: { KPS_DISPATCH(double) }
        case kStoreBF16: {
            if (!pin) return cudaErrorInvalidValue;
            if (k == 1) return launch_t<__nv_bfloat16, 1, true>(p, smem, stream);
            return launch_t<__nv_bfloat16, 2, true>(p, smem, stream);
        }
        case kStoreF16: {
            if (!pin) return cudaErrorInvalidValue;
            if (k == 1) return launch_t<__half, 1, true>(p, smem, stream);
            return launch_t<__half, 2, true>(p, smem, stream);
        }
        default: return cudaErrorInvalidValue;
    }
#undef KPS_DISPATCH
}

}  // namespace kps
