// Fast path of the Kronecker-form payoff products (sm_103a).
//
// Same mathematics as the general kernel (see kernels.cu):
//   out / lambda_out = K_F(u - v) + 2 Lo(v) + TieC(v)
// with u, v the lambda-weighted fold and showdown inputs of an output
// column, K_F the card-removal fold operator and Lo the compatible
// strictly-weaker mass of the strength-ordered scan.
//
// Differences from the general kernel, for occupancy and instruction count:
//   * per-card state is one float2 {running mass of v, total of w} per
//     (card, column), so one 64-bit shared access serves both sums;
//   * hands are scanned with immediate updates; a tie group (never split
//     across a tile) then gets the exact correction
//       TieC - 2 B = F - B,  B/F = compatible mass of the group members
//     before/after the hand, from the inputs still staged for the tile;
//   * partial results leave the SM through a staging tile as coalesced
//     stores into `scratch` (L2-resident until the CTA rereads them), so
//     shared memory holds only the per-warp state and 8 warps fit per SM;
//   * the final pass runs with lane = hand: the per-column card terms come
//     from a [column][card] table (odd pitch, at most 2-way bank conflicts),
//     loads and stores are coalesced.
// No atomics: results are bit-reproducible.
#include "kernels.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <mutex>
#include <type_traits>

namespace kps {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kPitch = 33;

template <typename S> struct Num;
template <> struct Num<float> {
    using C = float;
    using C2 = float2;
    __device__ static C load(const float *p) { return __ldg(p); }
    __device__ static float conv(C x) { return x; }
};
template <> struct Num<double> {
    using C = double;
    using C2 = double2;
    __device__ static C load(const double *p) { return __ldg(p); }
    __device__ static double conv(C x) { return x; }
};
template <> struct Num<__nv_bfloat16> {
    using C = float;
    using C2 = float2;
    __device__ static C load(const __nv_bfloat16 *p) {
        return __bfloat162float(__ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short *>(p))));
    }
    __device__ static __nv_bfloat16 conv(C x) { return __float2bfloat16_rn(x); }
};
template <> struct Num<__half> {
    using C = float;
    using C2 = float2;
    __device__ static C load(const __half *p) {
        return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short *>(p))));
    }
    __device__ static __half conv(C x) { return __float2half_rn(x); }
};

struct Col {
    long long in_off;    // element offset of the column's input vector
    long long out_off;   // element offset of the output row, -1 = no column
    int foff, soff;      // input row offsets (sequence * hs), -1 = no term
};

__host__ __device__ inline int zpitch(int nc) { return nc | 1; }

template <typename C>
__host__ __device__ inline size_t per_warp_elems(int nc) {
    // state [nc][32] C2 + stage [32][kPitch] C2 + partial tile [32][kPitch] C
    return 2 * (size_t)nc * 32 + 2 * 32 * kPitch + 32 * kPitch;
}

template <typename S, int K2>
__global__ void __launch_bounds__(32 * kMaxWarps)
fast_scan_kernel(const FastParams p) {
    using C = typename Num<S>::C;
    using C2 = typename Num<S>::C2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = p.nw, nc = p.nc;
    const int H = p.H, hs = p.hs;
    Col *ci = reinterpret_cast<Col *>(smem_raw);
    C *fco_s = reinterpret_cast<C *>(smem_raw + 32 * sizeof(Col));
    C *sco_s = fco_s + 32;
    C *sums = sco_s + 32;                                  // [nw][3][32]
    C *wbase = sums + (size_t)nw * 3 * 32;
    C *mine = wbase + (size_t)warp * per_warp_elems<C>(nc);
    C2 *R = reinterpret_cast<C2 *>(mine);                  // [nc][32]
    C2 *stage = R + (size_t)nc * 32;                       // [32][kPitch]
    C *ptile = reinterpret_cast<C *>(stage + 32 * kPitch); // [32][kPitch]
    const S *vin = static_cast<const S *>(p.vin);
    S *vout = static_cast<S *>(p.vout);
    C *scr = static_cast<C *>(p.scratch);
    const C *lam_in = static_cast<const C *>(p.lam_in);
    const C *lam_out = static_cast<const C *>(p.lam_out);

    // ---- columns of this CTA
    if (threadIdx.x < 32) {
        const long long col = (long long)blockIdx.x * 32 + threadIdx.x;
        Col c;
        C f = C(0), s = C(0);
        if (col < (long long)p.n_out * p.batch) {
            const int sg = (int)(col / p.batch), b = (int)(col % p.batch);
            const int fc = p.fcol[sg], sc = p.scol[sg];
            c.in_off = (long long)b * p.n_in * hs;
            c.out_off = ((long long)b * p.n_out + sg) * hs;
            c.foff = fc >= 0 ? fc * hs : -1;
            c.soff = sc >= 0 ? sc * hs : -1;
            if (fc >= 0) f = static_cast<const C *>(p.fcoef)[sg];
            if (sc >= 0) s = static_cast<const C *>(p.scoef)[sg];
        } else {
            c.in_off = 0;
            c.out_off = -1;
            c.foff = c.soff = -1;
        }
        ci[threadIdx.x] = c;
        fco_s[threadIdx.x] = f;
        sco_s[threadIdx.x] = s;
    }
    __syncthreads();
    const Col c0i = ci[0];
    int same = 1, valid = 0;
    if (threadIdx.x < 32) {
        const Col c = ci[threadIdx.x];
        if (c.out_off >= 0) {
            valid = 1;
            same = c.foff == c0i.foff && c.soff == c0i.soff &&
                   c.in_off == c0i.in_off + (long long)threadIdx.x * p.n_in * hs &&
                   c.out_off == c0i.out_off + (long long)threadIdx.x * p.n_out * hs;
        }
    }
    const bool uni = __syncthreads_and(same) != 0;
    const int nvalid = __syncthreads_count(valid);
    const long long istride = (long long)p.n_in * hs, ostride = (long long)p.n_out * hs;
    const C fco = fco_s[lane], sco = sco_s[lane];

    for (int c = 0; c < nc; ++c) R[c * 32 + lane] = C2{C(0), C(0)};

    // ---- phase 1: scan the chunk's tiles (lane = column)
    const int tb = p.tchunk[warp], te = p.tchunk[warp + 1];
    C Gv = C(0), Gw = C(0);
    C xf[32], xs[32];
    C lin_n = C(0);
    uint32_t h_n = 0u;
    auto fetch = [&](int t) {
        const int2 tl = p.tiles[t];
        const int pos = tl.x + lane;
        const bool pin = lane < tl.y;
        lin_n = pin ? lam_in[pos] : C(0);
        h_n = pin ? __ldg(&p.hinfo[pos]) : 0u;
        if (uni) {
            const S *fb = vin + c0i.in_off + pos + c0i.foff;
            const S *sb = vin + c0i.in_off + pos + c0i.soff;
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
                const bool ok = pin && jj < nvalid;
                xf[jj] = (ok && c0i.foff >= 0) ? Num<S>::load(fb + jj * istride) : C(0);
                xs[jj] = (ok && c0i.soff >= 0) ? Num<S>::load(sb + jj * istride) : C(0);
            }
        } else {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
                const Col cj = ci[jj];
                const S *base = vin + cj.in_off + pos;
                xf[jj] = (pin && cj.foff >= 0) ? Num<S>::load(base + cj.foff) : C(0);
                xs[jj] = (pin && cj.soff >= 0) ? Num<S>::load(base + cj.soff) : C(0);
            }
        }
    };
    if (tb < te) fetch(tb);
    for (int t = tb; t < te; ++t) {
        const int2 tl = p.tiles[t];
        const int t0 = tl.x, len = tl.y;
        const C lin = lin_n;
        const uint32_t hreg = h_n;
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) stage[lane * kPitch + jj] = C2{lin * xf[jj], lin * xs[jj]};
        __syncwarp();
        if (t + 1 < te) fetch(t + 1);
        for (int i = 0; i < len;) {
            const uint32_t h1 = __shfl_sync(kFull, hreg, i);
            const uint32_t h2 = __shfl_sync(kFull, hreg, min(i + 1, 31));
            const int a1 = h1 & 63, b1 = (h1 >> 6) & 63;
            const C2 x1 = stage[i * kPitch + lane];
            const C u1 = fco * x1.x, v1 = sco * x1.y, w1 = u1 - v1;
            if ((h1 & (1u << 15)) && i + 1 < len) {
                // next hand shares no card: both steps' loads are independent
                const int a2 = h2 & 63, b2 = (h2 >> 6) & 63;
                const C2 x2 = stage[(i + 1) * kPitch + lane];
                const C u2 = fco * x2.x, v2 = sco * x2.y, w2 = u2 - v2;
                const C2 ra1 = R[a1 * 32 + lane], ra2 = R[a2 * 32 + lane];
                C2 rb1 = C2{C(0), C(0)}, rb2 = C2{C(0), C(0)};
                if (K2 == 2) {
                    rb1 = R[b1 * 32 + lane];
                    rb2 = R[b2 * 32 + lane];
                }
                const C g1 = Gv + v1;
                ptile[i * kPitch + lane] = (K2 == 2 ? w1 : C(0)) + C(2) * (Gv - ra1.x - rb1.x);
                ptile[(i + 1) * kPitch + lane] = (K2 == 2 ? w2 : C(0)) + C(2) * (g1 - ra2.x - rb2.x);
                R[a1 * 32 + lane] = C2{ra1.x + v1, ra1.y + w1};
                R[a2 * 32 + lane] = C2{ra2.x + v2, ra2.y + w2};
                if (K2 == 2) {
                    R[b1 * 32 + lane] = C2{rb1.x + v1, rb1.y + w1};
                    R[b2 * 32 + lane] = C2{rb2.x + v2, rb2.y + w2};
                }
                Gv = g1 + v2;
                Gw = (Gw + w1) + w2;
                i += 2;
            } else {
                const C2 ra1 = R[a1 * 32 + lane];
                const C2 rb1 = K2 == 2 ? R[b1 * 32 + lane] : C2{C(0), C(0)};
                ptile[i * kPitch + lane] = (K2 == 2 ? w1 : C(0)) + C(2) * (Gv - ra1.x - rb1.x);
                R[a1 * 32 + lane] = C2{ra1.x + v1, ra1.y + w1};
                if (K2 == 2) R[b1 * 32 + lane] = C2{rb1.x + v1, rb1.y + w1};
                Gv += v1;
                Gw += w1;
                i += 1;
            }
        }
        // tie groups of this tile: the scan counted earlier members as
        // weaker; the exact term adds later members and removes earlier ones
        if (__any_sync(kFull, (lane < len) && (hreg & (1u << 12)))) {
            for (int i = 0; i < len; ++i) {
                const uint32_t hi = __shfl_sync(kFull, hreg, i);
                if (!(hi & (1u << 13))) continue;          // act at the group's last member
                const int g0 = i - (int)(hi >> 16);
                for (int q = g0; q <= i; ++q) {
                    const uint32_t hq = __shfl_sync(kFull, hreg, q);
                    C corr = C(0);
                    for (int r = g0; r <= i; ++r) {
                        if (r == q) continue;
                        const uint32_t hr = __shfl_sync(kFull, hreg, r);
                        const int qa = hq & 63, qb = (hq >> 6) & 63, ra = hr & 63, rb = (hr >> 6) & 63;
                        bool share = qa == ra;
                        if (K2 == 2) share = share || qa == rb || qb == ra || qb == rb;
                        if (share) continue;
                        const C vr = sco * stage[r * kPitch + lane].y;
                        corr += r > q ? vr : -vr;
                    }
                    ptile[q * kPitch + lane] += corr;
                }
            }
        }
        __syncwarp();
        // partial results out, lane = hand (coalesced rows)
        if (lane < len) {
            if (uni) {
                C *dst = scr + c0i.out_off + t0 + lane;
                for (int jj = 0; jj < nvalid; ++jj) dst[jj * ostride] = ptile[lane * kPitch + jj];
            } else {
                for (int jj = 0; jj < 32; ++jj) {
                    const long long o = ci[jj].out_off;
                    if (o >= 0) scr[o + t0 + lane] = ptile[lane * kPitch + jj];
                }
            }
        }
        __syncwarp();
    }
    sums[(warp * 3 + 0) * 32 + lane] = Gv;
    sums[(warp * 3 + 1) * 32 + lane] = Gw;
    __syncthreads();

    // ---- phase 2: per (card, column): fold totals Pw and the mass Xv of
    // the card in earlier chunks.  Z_k[column][card] = Pw + 2 Xv_k goes to
    // warp k's (now free) staging area.
    const int zp = zpitch(nc);
    for (int c = warp; c < nc; c += nw) {
        C pw = C(0);
        for (int k = 0; k < nw; ++k) {
            const C2 *Rk = reinterpret_cast<const C2 *>(wbase + (size_t)k * per_warp_elems<C>(nc));
            pw += Rk[c * 32 + lane].y;
        }
        C xv = C(0);
        for (int k = 0; k < nw; ++k) {
            C *base_k = wbase + (size_t)k * per_warp_elems<C>(nc);
            const C2 *Rk = reinterpret_cast<const C2 *>(base_k);
            C *Zk = base_k + 2 * (size_t)nc * 32;          // staging area of warp k
            const C r = Rk[c * 32 + lane].x;
            Zk[lane * zp + c] = pw + C(2) * xv;
            xv += r;
        }
    }
    if (warp == 0) {
        C tw = C(0);
        for (int k = 0; k < nw; ++k) tw += sums[(k * 3 + 1) * 32 + lane];
        C xg = C(0);
        for (int k = 0; k < nw; ++k) {
            sums[(k * 3 + 2) * 32 + lane] = tw + C(2) * xg;
            xg += sums[(k * 3 + 0) * 32 + lane];
        }
    }
    __syncthreads();

    // ---- phase 3: finish and write out, lane = hand
    const C *Z = mine + 2 * (size_t)nc * 32;
    const C basev = sums[(warp * 3 + 2) * 32 + lane];     // lane = column here
    for (int t = tb; t < te; ++t) {
        const int2 tl = p.tiles[t];
        const int pos = tl.x + lane;
        const bool pin = lane < tl.y;
        if (!__any_sync(kFull, pin)) continue;
        const uint32_t hq = pin ? __ldg(&p.hinfo[pos]) : 0u;
        const C lo = pin ? lam_out[pos] : C(0);
        const int a = hq & 63, b = (hq >> 6) & 63;
        C part[32];
        if (uni) {
            const C *src = scr + c0i.out_off + pos;
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) part[jj] = (pin && jj < nvalid) ? src[jj * ostride] : C(0);
        } else {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
                const long long o = ci[jj].out_off;
                part[jj] = (pin && o >= 0) ? scr[o + pos] : C(0);
            }
        }
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
            const C bj = __shfl_sync(kFull, basev, jj);
            C val = part[jj] + bj - Z[jj * zp + a];
            if (K2 == 2) val -= Z[jj * zp + b];
            part[jj] = lo * val;
        }
        if (pin) {
            if (uni) {
                S *dst = vout + c0i.out_off + pos;
#pragma unroll
                for (int jj = 0; jj < 32; ++jj)
                    if (jj < nvalid) dst[jj * ostride] = Num<S>::conv(part[jj]);
            } else {
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
                    const long long o = ci[jj].out_off;
                    if (o >= 0) vout[o + pos] = Num<S>::conv(part[jj]);
                }
            }
        }
    }
    // padding of every row
    if (warp == nw - 1 && H + lane < hs) {
        for (int jj = 0; jj < 32; ++jj) {
            const long long o = ci[jj].out_off;
            if (o >= 0) vout[o + H + lane] = Num<S>::conv(C(0));
        }
    }
}

template <typename S, int K2>
cudaError_t launch_t(const FastParams &p, size_t smem, cudaStream_t stream) {
    auto fn = fast_scan_kernel<S, K2>;
    {
        const cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void *>(fn), smem);
        if (e != cudaSuccess) return e;
    }
    const long long ncols = (long long)p.n_out * p.batch;
    const long long blocks = (ncols + 31) / 32;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    fn<<<(unsigned)blocks, 32 * p.nw, smem, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace

size_t fast_smem_bytes(int storage, int nc, int nw) {
    const size_t cs = storage == kStoreF64 ? 8 : 4;
    size_t bytes = 32 * sizeof(Col) + 2 * 32 * cs + (size_t)nw * 3 * 32 * cs;
    bytes += (size_t)nw * (2 * (size_t)nc * 32 + 3 * 32 * kPitch) * cs;
    return bytes;
}

cudaError_t launch_fast_scan(const FastParams &p, int storage, int k, cudaStream_t stream) {
    const size_t smem = fast_smem_bytes(storage, p.nc, p.nw);
    switch (storage) {
        case kStoreF32: return k == 1 ? launch_t<float, 1>(p, smem, stream) : launch_t<float, 2>(p, smem, stream);
        case kStoreF64: return k == 1 ? launch_t<double, 1>(p, smem, stream) : launch_t<double, 2>(p, smem, stream);
        case kStoreBF16:
            return k == 1 ? launch_t<__nv_bfloat16, 1>(p, smem, stream) : launch_t<__nv_bfloat16, 2>(p, smem, stream);
        case kStoreF16: return k == 1 ? launch_t<__half, 1>(p, smem, stream) : launch_t<__half, 2>(p, smem, stream);
        default: return cudaErrorInvalidValue;
    }
}

// ---- statically reserved scratch (see kps_matvec_A_static_scratch) --------
// One file-scope array per device that loads the library: the tile list of
// a launch followed by its FP32 partial results.  Every launch overwrites the
// parts it reads, so nothing has to start at zero.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticTileBytes + (size_t)kStaticScratchFloats * 4];

cudaError_t static_scratch_address(void **ptr) {
    // The array's name is a host-side stand-in; the device address is looked
    // up once per device, with that device current.
    static std::mutex mu;
    static void *addr[kMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = p;
    }
    *ptr = addr[dev];
    return cudaSuccess;
}

}  // namespace kps
