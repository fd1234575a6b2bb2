// Kronecker-form payoff products with partial results held in tensor memory
// (sm_103a).  FP32 arithmetic; FP32, BF16 or FP16 storage.
//
// Mathematics as in kernels.cu:
//   out / lambda_out = K_F(u - v) + 2 Lo(v) + TieC(v)
// with u, v the lambda-weighted fold and showdown inputs of an output column
// (its fold terminal and its showdown terminal, Sec. 3 / Prop. 1), K_F the
// card-removal fold operator and Lo the compatible strictly-weaker mass of
// the strength-ordered scan (the inverse of Technique B's bidiagonal D).
//
// Organisation (one CTA = 32 output columns, one per lane, up to 8 warps):
//   * each warp scans one tie-aligned chunk of the hand order; its inputs are
//     prefetched tile by tile (32 hands) into registers with coalesced loads
//     (lane = hand) and transposed through shared memory, while the previous
//     tile is scanned (lane = column; per-card state [card][lane] in shared
//     memory, conflict free, two hands per step when they share no card);
//   * the partial result of every (hand, column) stays on chip: the chunk's
//     last tile in the warp's partial tile in shared memory, the other
//     tiles in tensor memory (the warp's 32 lanes are the 32 columns, a
//     tensor-memory column is a hand, so a half tile leaves in one
//     tcgen05.st and comes back in one tcgen05.ld), and, for chunks longer
//     than the warp's 256 columns allow (the SP instantiation), the columns
//     past the region in spill rows of the partial tile.  Shared memory
//     keeps only per-warp state (about 27 KB); the partial results never
//     travel to global memory.  With 4 warps a CTA takes 256 tensor-memory
//     columns and ~110 KB of shared memory, so two CTAs share an SM and one
//     CTA's scan overlaps the other's combination and finishing pass;
//   * after the chunks' per-card sums are combined (fold totals and the mass
//     of earlier chunks), each warp finishes its hands, the last tile first,
//     and writes the output with coalesced stores (lane = hand).
// Scans are specialised by column kind: fold only, showdown only, or both.
// No atomics: results are bit-reproducible.
#include "kernels.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdint>

namespace kps {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kPitch = 33;         // row pitch of [hand][column] tiles
constexpr int kRegion = kTmemRegion;   // tensor-memory columns owned by one warp

template <typename S> struct Num;
template <> struct Num<float> {
    __device__ static float load(const float *p) { return __ldg(p); }
    __device__ static float conv(float x) { return x; }
};
template <> struct Num<__nv_bfloat16> {
    __device__ static float load(const __nv_bfloat16 *p) {
        return __bfloat162float(__ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short *>(p))));
    }
    __device__ static __nv_bfloat16 conv(float x) { return __float2bfloat16_rn(x); }
};
template <> struct Num<__half> {
    __device__ static float load(const __half *p) {
        return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short *>(p))));
    }
    __device__ static __half conv(float x) { return __float2half_rn(x); }
};

struct Col {
    long long in_off;
    long long out_off;   // -1 = no column
    int foff, soff;      // -1 = no such terminal
};

enum Kind { kKindF = 1, kKindS = 2, kKindFS = 3 };

// ---- tensor memory (tcgen05) ---------------------------------------------
__device__ __forceinline__ void tm_alloc(uint32_t *dst_smem, uint32_t ncols) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(dst_smem);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tm_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void tm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void tm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;"); }
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;"); }
// waits for this thread's tensor-memory loads; names the 16 destination
// registers so that no use of them is scheduled before the data arrive
__device__ __forceinline__ void tm_wait_ld16(float *r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+f"(r[0]), "+f"(r[1]), "+f"(r[2]), "+f"(r[3]), "+f"(r[4]), "+f"(r[5]), "+f"(r[6]), "+f"(r[7]),
                   "+f"(r[8]), "+f"(r[9]), "+f"(r[10]), "+f"(r[11]), "+f"(r[12]), "+f"(r[13]), "+f"(r[14]), "+f"(r[15])::"memory");
}

// one column of this warp's lanes <-> v
__device__ __forceinline__ void tm_st1(uint32_t taddr, float v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(taddr), "f"(v));
}
__device__ __forceinline__ void tm_ld1(uint32_t taddr, float &v) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=f"(v) : "r"(taddr));
}

// 16 consecutive tensor-memory columns of this warp's lanes <-> r[0..15]
__device__ __forceinline__ void tm_st16(uint32_t taddr, const float *r) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "f"(r[0]), "f"(r[1]), "f"(r[2]), "f"(r[3]), "f"(r[4]), "f"(r[5]), "f"(r[6]), "f"(r[7]), "f"(r[8]), "f"(r[9]),
        "f"(r[10]), "f"(r[11]), "f"(r[12]), "f"(r[13]), "f"(r[14]), "f"(r[15]));
}
__device__ __forceinline__ void tm_ld16(uint32_t taddr, float *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7]), "=f"(r[8]),
          "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15])
        : "r"(taddr));
}

// Shared memory: header (columns, coefficients, per-warp sums, the tensor-
// memory slot, per-warp tile descriptors) then, per warp, state [nc][32]
// float2, stage [32][kPitch] float2 and a [32 + kTmemSpill][kPitch] float
// tile (rows 32.. hold the columns kTmemRegion.. of the tensor-memory tiles).
constexpr int kTlCache = 16;       // tile descriptors of a chunk kept in shared memory
__host__ __device__ inline size_t tm_tls_offset(int nw) {
    return (32 * sizeof(Col) + (2 * 32 + (size_t)nw * 3 * 32) * sizeof(float) + 16 + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t tm_header_bytes(int nw) { return tm_tls_offset(nw) + (size_t)nw * kTlCache * 8; }
__host__ __device__ inline size_t tm_warp_floats(int nc) {
    return 2 * (size_t)nc * 32 + (3 * 32 + kTmemSpill) * kPitch;
}

struct Cta {
    const Col *ci;
    float *sums;      // [nw][3][32]
    bool uni;         // columns share a sequence and take consecutive vectors
    int nvalid;
    uint32_t tmem;    // tensor-memory base address of the CTA
};

template <typename S, int K2, int KIND, bool SP>
__device__ __forceinline__ void tm_body(const FastParams &p, unsigned char *smem, const Cta &cta,
                                        const float *fco_s, const float *sco_s) {
    constexpr bool HF = (KIND & kKindF) != 0, HS = (KIND & kKindS) != 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = p.nw, nc = p.nc;
    const int H = p.H, hs = p.hs;
    const Col *ci = cta.ci;
    float *sums = cta.sums;
    const bool uni = cta.uni;
    const int nvalid = cta.nvalid;
    float *wbase = reinterpret_cast<float *>(smem + tm_header_bytes(nw));
    float *mine = wbase + (size_t)warp * tm_warp_floats(nc);
    float2 *R = reinterpret_cast<float2 *>(mine);            // [card][32]: {v running, w total}
    float2 *stage = R + (size_t)nc * 32;                     // [hand][kPitch]: lambda_in * {x_f, x_s}
    float *ptile = reinterpret_cast<float *>(stage + 32 * kPitch);   // [hand][kPitch]
    const float *st1v = reinterpret_cast<const float *>(stage);      // single-width stage
    const S *vin = static_cast<const S *>(p.vin);
    S *vout = static_cast<S *>(p.vout);
    const float *lam_in = static_cast<const float *>(p.lam_in);
    const float *lam_out = static_cast<const float *>(p.lam_out);
    const long long istride = (long long)p.n_in * hs, ostride = (long long)p.n_out * hs;
    const float fco = fco_s[lane], sco = sco_s[lane];
    const Col c0i = ci[0];
    int2 *tls = reinterpret_cast<int2 *>(smem + tm_tls_offset(nw)) + warp * kTlCache;
    // this warp's tensor-memory lanes (= its 32 columns) and column region
    const uint32_t treg = cta.tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * kRegion);

    for (int c = 0; c < nc; ++c) R[c * 32 + lane] = make_float2(0.f, 0.f);

    // ---- phase 1: scan the chunk's tiles (lane = column)
    const int tb = p.tchunk[warp], te = p.tchunk[warp + 1];
    const int cstart = tb < te ? p.tiles[tb].x : 0;
    float Gv = 0.f, Gw = 0.f;
    float xf[32], xs[32];
    float lin_n = 0.f;
    uint32_t h_n = 0u;
    int2 tw_n = make_int2(0, 0);
    // next tile's inputs, lane = hand, one register per column
    auto fetch = [&](int t) {
        const int2 tl = p.tiles[t];
        const int pos = tl.x + lane;
        const bool pin = lane < tl.y;
        lin_n = pin ? lam_in[pos] : 0.f;
        h_n = pin ? __ldg(&p.hinfo[pos]) : 0u;
        if (HS) tw_n = p.tie_work[t];
        if (uni) {
            // lanes past the tile's end read its last hand (their staged
            // value is lin = 0 times a finite input)
            const int pc = min(pos, tl.x + tl.y - 1);
            const S *fb = vin + c0i.in_off + pc + (HF ? c0i.foff : 0);
            const S *sb = vin + c0i.in_off + pc + (HS ? c0i.soff : 0);
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
                xf[jj] = (HF && jj < nvalid) ? Num<S>::load(fb) : 0.f;
                xs[jj] = (HS && jj < nvalid) ? Num<S>::load(sb) : 0.f;
                fb += istride;
                sb += istride;
            }
        } else {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
                const Col cj = ci[jj];
                const S *base = vin + cj.in_off + pos;
                xf[jj] = (HF && pin && cj.foff >= 0) ? Num<S>::load(base + cj.foff) : 0.f;
                xs[jj] = (HS && pin && cj.soff >= 0) ? Num<S>::load(base + cj.soff) : 0.f;
            }
        }
    };
    if (tb < te) fetch(tb);
    for (int t = tb; t < te; ++t) {
        const int2 tl = p.tiles[t];
        const int t0 = tl.x, len = tl.y;
        const float lin = lin_n;
        const uint32_t hreg = h_n;
        const int2 tw = tw_n;
        if (lane == 0 && t - tb < kTlCache) tls[t - tb] = tl;
        // stage the tile (lane = hand), then prefetch the next one
        float *st1w = reinterpret_cast<float *>(stage);
        if constexpr (KIND == kKindFS) {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) stage[lane * kPitch + jj] = make_float2(lin * xf[jj], lin * xs[jj]);
        } else {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) st1w[lane * kPitch + jj] = lin * (HF ? xf[jj] : xs[jj]);
        }
        __syncwarp();
        if (t + 1 < te) fetch(t + 1);
        // Tie groups (never split across a tile): the scan counts earlier
        // members as weaker; the exact equal-strength term adds the later
        // compatible members and removes the earlier ones.  The tile's
        // compatible tied pairs come from a table; their terms (inputs only)
        // are summed per hand in the idle partial tile and added after the
        // scan of each half.
        const bool ties = HS && tw.y > 0;
        if (ties) {
#pragma unroll
            for (int k = 0; k < 32; ++k) ptile[k * kPitch + lane] = 0.f;
            for (int e = 0; e < tw.y; ++e) {
                const uint32_t tr = __ldg(&p.tie_trip[tw.x + e]);
                const int q = tr & 31, rr = (tr >> 5) & 31;
                const float vr = sco * (KIND == kKindFS ? stage[rr * kPitch + lane].y : st1v[rr * kPitch + lane]);
                ptile[q * kPitch + lane] += (tr >> 10) & 1u ? vr : -vr;
            }
        }
        // The scan, one half tile (16 hands, 8 steps of two hands) at a
        // time.  Hands past the tile's end have zero input and add nothing.
        // The half's inputs and hand records are read into registers first
        // (no staged value waits behind a per-card store); all four per-card
        // loads of a step are issued together; when the second hand holds a
        // card of the first, its loaded sums get the first hand's update in
        // registers, and its store (the later one) leaves the combined value.
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            if (16 * half >= len) break;   // a short tile's second half is all padding
            float r[16];
            uint32_t hh[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) hh[k] = __shfl_sync(kFull, hreg, 16 * half + k);
            if constexpr (KIND == kKindFS) {
                float2 xh[16];
                const float2 *st_l = stage + lane + 16 * half * kPitch;
#pragma unroll
                for (int k = 0; k < 16; ++k) xh[k] = st_l[k * kPitch];
#pragma unroll
                for (int k = 0; k < 16; k += 2) {
                    const uint32_t h1 = hh[k], h2 = hh[k + 1];
                    const int a1 = h1 & 63, b1 = (h1 >> 6) & 63, a2 = h2 & 63, b2 = (h2 >> 6) & 63;
                    const float2 x1 = xh[k], x2 = xh[k + 1];
                    const float u1 = fco * x1.x, v1 = sco * x1.y, w1 = u1 - v1;
                    const float u2 = fco * x2.x, v2 = sco * x2.y, w2 = u2 - v2;
                    float2 ra1 = R[a1 * 32 + lane], ra2 = R[a2 * 32 + lane];
                    float2 rb1 = make_float2(0.f, 0.f), rb2 = make_float2(0.f, 0.f);
                    if (K2 == 2) {
                        rb1 = R[b1 * 32 + lane];
                        rb2 = R[b2 * 32 + lane];
                        const bool sa = a2 == a1 || a2 == b1, sb = b2 == a1 || b2 == b1;
                        ra2.x += sa ? v1 : 0.f;
                        ra2.y += sa ? w1 : 0.f;
                        rb2.x += sb ? v1 : 0.f;
                        rb2.y += sb ? w1 : 0.f;
                    } else {
                        const bool sa = a2 == a1;
                        ra2.x += sa ? v1 : 0.f;
                        ra2.y += sa ? w1 : 0.f;
                    }
                    const float g1 = Gv + v1;
                    r[k] = (K2 == 2 ? w1 : 0.f) + 2.f * (Gv - ra1.x - rb1.x);
                    r[k + 1] = (K2 == 2 ? w2 : 0.f) + 2.f * (g1 - ra2.x - rb2.x);
                    R[a1 * 32 + lane] = make_float2(ra1.x + v1, ra1.y + w1);
                    if (K2 == 2) R[b1 * 32 + lane] = make_float2(rb1.x + v1, rb1.y + w1);
                    R[a2 * 32 + lane] = make_float2(ra2.x + v2, ra2.y + w2);
                    if (K2 == 2) R[b2 * 32 + lane] = make_float2(rb2.x + v2, rb2.y + w2);
                    Gv = g1 + v2;
                    Gw = (Gw + w1) + w2;
                }
            } else {
                // One running value per card (the fold total of fold-only
                // columns, the showdown mass of showdown-only ones, whose fold
                // total is its negative): half the shared-memory traffic.
                float *R1 = reinterpret_cast<float *>(mine);
                const float cof = HF ? fco : sco;
                float xh[16];
                const float *sl = st1v + lane + 16 * half * kPitch;
#pragma unroll
                for (int k = 0; k < 16; ++k) xh[k] = sl[k * kPitch];
#pragma unroll
                for (int k = 0; k < 16; k += 2) {
                    const uint32_t h1 = hh[k], h2 = hh[k + 1];
                    const int a1 = h1 & 63, b1 = (h1 >> 6) & 63, a2 = h2 & 63, b2 = (h2 >> 6) & 63;
                    const float c1 = cof * xh[k], c2 = cof * xh[k + 1];
                    float ra1 = R1[a1 * 32 + lane], ra2 = R1[a2 * 32 + lane], rb1 = 0.f, rb2 = 0.f;
                    if (K2 == 2) {
                        rb1 = R1[b1 * 32 + lane];
                        rb2 = R1[b2 * 32 + lane];
                        ra2 += (a2 == a1 || a2 == b1) ? c1 : 0.f;
                        rb2 += (b2 == a1 || b2 == b1) ? c1 : 0.f;
                    } else {
                        ra2 += a2 == a1 ? c1 : 0.f;
                    }
                    if (HS) {
                        // w = -v for a showdown-only column
                        const float g1 = Gv + c1;
                        r[k] = (K2 == 2 ? -c1 : 0.f) + 2.f * (Gv - ra1 - rb1);
                        r[k + 1] = (K2 == 2 ? -c2 : 0.f) + 2.f * (g1 - ra2 - rb2);
                        Gv = g1 + c2;
                    } else {
                        r[k] = K2 == 2 ? c1 : 0.f;
                        r[k + 1] = K2 == 2 ? c2 : 0.f;
                        Gw = (Gw + c1) + c2;
                    }
                    R1[a1 * 32 + lane] = ra1 + c1;
                    if (K2 == 2) R1[b1 * 32 + lane] = rb1 + c1;
                    R1[a2 * 32 + lane] = ra2 + c2;
                    if (K2 == 2) R1[b2 * 32 + lane] = rb2 + c2;
                }
            }
            if (ties) {
#pragma unroll
                for (int k = 0; k < 16; ++k) r[k] += ptile[(16 * half + k) * kPitch + lane];
            }
            // the half's partial results to tensor memory (lane = column;
            // columns past the tile's end are rewritten by the next tile),
            // the last tile's to the partial tile, where the finishing pass
            // takes them first
            const int c0 = t0 - cstart + 16 * half;
            if (t + 1 < te && (!SP || c0 + 16 <= kRegion)) {
                tm_st16(treg + (uint32_t)c0, r);
            } else if (SP && t + 1 < te) {
                // a half crossing the end of the tensor-memory region: its
                // columns past the end go to the spill rows
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    if (c0 + k < kRegion) tm_st1(treg + (uint32_t)(c0 + k), r[k]);
                    else ptile[(32 + c0 + k - kRegion) * kPitch + lane] = r[k];
                }
            } else {
#pragma unroll
                for (int k = 0; k < 16; ++k) ptile[(16 * half + k) * kPitch + lane] = r[k];
            }
        }
        __syncwarp();
    }
    tm_wait_st();
    sums[(warp * 3 + 0) * 32 + lane] = Gv;
    sums[(warp * 3 + 1) * 32 + lane] = Gw;
    __syncthreads();

    // ---- phase 2: per (card, column): fold total Pw and the card's mass Xv_k
    // in earlier chunks; Z_k[card][column] = Pw + 2 Xv_k goes to warp k's
    // (now free) staging area.  base_k = Tw + 2 Xg_k.
    for (int c = warp; c < nc; c += nw) {
        float tot[kMaxWarps], run[kMaxWarps];
#pragma unroll
        for (int k = 0; k < kMaxWarps; ++k) {
            tot[k] = run[k] = 0.f;
            if (k < nw) {
                const float *Rk = wbase + (size_t)k * tm_warp_floats(nc);
                if (KIND == kKindFS) {
                    const float2 s2 = reinterpret_cast<const float2 *>(Rk)[c * 32 + lane];
                    run[k] = s2.x;
                    tot[k] = s2.y;
                } else {
                    const float s1 = Rk[c * 32 + lane];
                    run[k] = HS ? s1 : 0.f;
                    tot[k] = HF ? s1 : -s1;
                }
            }
        }
        float pw = 0.f;
#pragma unroll
        for (int k = 0; k < kMaxWarps; ++k) pw += tot[k];
        float xv = 0.f;
#pragma unroll
        for (int k = 0; k < kMaxWarps; ++k) {
            if (k < nw) {
                float *Zk = wbase + (size_t)k * tm_warp_floats(nc) + 2 * (size_t)nc * 32;
                Zk[c * 32 + lane] = pw + 2.f * xv;
                xv += run[k];
            }
        }
    }
    if (warp == 0) {
        float tw = 0.f;
        for (int k = 0; k < nw; ++k) tw += HF ? sums[(k * 3 + 1) * 32 + lane] : -sums[(k * 3 + 0) * 32 + lane];
        float xg = 0.f;
        for (int k = 0; k < nw; ++k) {
            sums[(k * 3 + 2) * 32 + lane] = tw + 2.f * xg;
            xg += sums[(k * 3 + 0) * 32 + lane];
        }
    }
    __syncthreads();

    // ---- phase 3: finish each tile from tensor memory (the last tile from
    // the partial tile, first; lane = column), then write it out with
    // coalesced stores (lane = hand)
    const float *Z = mine + 2 * (size_t)nc * 32 + lane;
    const float base = sums[(warp * 3 + 2) * 32 + lane];
    // the next tile's descriptor (shared memory for the first kTlCache tiles
    // of the chunk), hand records and output weights are loaded while the
    // current tile is finished
    int2 tl_n = make_int2(0, 0);
    uint32_t hq_n = 0u;
    float lo_n = 0.f;
    auto pre3 = [&](int t) {
        tl_n = t - tb < kTlCache ? tls[t - tb] : p.tiles[t];
        const int pos = tl_n.x + lane;
        const bool pin = lane < tl_n.y;
        hq_n = pin ? __ldg(&p.hinfo[pos]) : 0u;
        lo_n = pin ? lam_out[pos] : 0.f;
    };
    const int nt = te - tb;
    if (nt > 0) pre3(te - 1);
    for (int i = 0; i < nt; ++i) {
        const int2 tl = tl_n;
        const uint32_t hq = hq_n;
        const float lo = lo_n;
        const int t0 = tl.x, len = tl.y;
        const int pos = t0 + lane;
        const bool pin = lane < len;
        if (i + 1 < nt) pre3(tb + i);
        // per half tile: partial results from tensor memory, every hand's
        // per-card terms (loaded before any store of the partial tile), the
        // finished values into the partial tile
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            if (16 * half >= len) break;
            float r[16], za[16], zb[16];
            const int c0 = t0 - cstart + 16 * half;
            if (i > 0 && (!SP || c0 + 16 <= kRegion)) {
                tm_ld16(treg + (uint32_t)c0, r);
            } else if (SP && i > 0) {
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    if (c0 + k < kRegion) tm_ld1(treg + (uint32_t)(c0 + k), r[k]);
                    else r[k] = ptile[(32 + c0 + k - kRegion) * kPitch + lane];
                }
            } else {
#pragma unroll
                for (int k = 0; k < 16; ++k) r[k] = ptile[(16 * half + k) * kPitch + lane];
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const uint32_t h = __shfl_sync(kFull, hq, 16 * half + k);
                za[k] = Z[(h & 63) * 32];
                zb[k] = K2 == 2 ? Z[((h >> 6) & 63) * 32] : 0.f;
            }
            tm_wait_ld16(r);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                float val = r[k] + base - za[k];
                if (K2 == 2) val -= zb[k];
                ptile[(16 * half + k) * kPitch + lane] = val;
            }
        }
        __syncwarp();
        // lane = hand: the hand's output weight, then coalesced stores
        if (pin) {
            if (uni) {
                S *dst = vout + c0i.out_off + pos;
                if (nvalid == 32) {
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) {
                        *dst = Num<S>::conv(lo * ptile[lane * kPitch + jj]);
                        dst += ostride;
                    }
                } else {
                    for (int jj = 0; jj < nvalid; ++jj) dst[jj * ostride] = Num<S>::conv(lo * ptile[lane * kPitch + jj]);
                }
            } else {
                for (int jj = 0; jj < 32; ++jj) {
                    const long long o = ci[jj].out_off;
                    if (o >= 0) vout[o + pos] = Num<S>::conv(lo * ptile[lane * kPitch + jj]);
                }
            }
        }
        __syncwarp();
    }
    // padding of every row
    if (warp == nw - 1 && H + lane < hs) {
        for (int jj = 0; jj < 32; ++jj) {
            const long long o = ci[jj].out_off;
            if (o >= 0) vout[o + H + lane] = Num<S>::conv(0.f);
        }
    }
}

// Shared-memory slot of the CTA's tensor-memory base address.
__device__ __forceinline__ uint32_t *tm_slot(unsigned char *smem_raw, int nw) {
    float *sums = reinterpret_cast<float *>(smem_raw + 32 * sizeof(Col)) + 2 * 32;
    return reinterpret_cast<uint32_t *>(sums + (size_t)nw * 3 * 32);
}

// One tile of 32 output columns (col = ctile * 32 + lane) of game p.  Ends
// with every tensor-memory access of the tile complete.
template <typename S, int K2, bool SP>
__device__ __forceinline__ void tm_tile(const FastParams &p, long long ctile, unsigned char *smem_raw,
                                        uint32_t tmem) {
    const int hs = p.hs;
    Col *ci = reinterpret_cast<Col *>(smem_raw);
    float *fco_s = reinterpret_cast<float *>(smem_raw + 32 * sizeof(Col));
    float *sco_s = fco_s + 32;
    float *sums = sco_s + 32;
    int kinds = 0;
    if (threadIdx.x < 32) {
        const long long col = ctile * 32 + threadIdx.x;
        Col c;
        float f = 0.f, s = 0.f;
        if (col < (long long)p.n_out * p.batch) {
            const int sg = (int)(col / p.batch), b = (int)(col % p.batch);
            const int fc = p.fcol[sg], sc = p.scol[sg];
            c.in_off = (long long)b * p.n_in * hs;
            c.out_off = ((long long)b * p.n_out + sg) * hs;
            c.foff = fc >= 0 ? fc * hs : -1;
            c.soff = sc >= 0 ? sc * hs : -1;
            if (fc >= 0) f = static_cast<const float *>(p.fcoef)[sg];
            if (sc >= 0) s = static_cast<const float *>(p.scoef)[sg];
        } else {
            c.in_off = 0;
            c.out_off = -1;
            c.foff = c.soff = -1;
        }
        ci[threadIdx.x] = c;
        fco_s[threadIdx.x] = f;
        sco_s[threadIdx.x] = s;
        kinds = (c.foff >= 0 ? 1 : 0) | (c.soff >= 0 ? 2 : 0);
    }
    tm_fence_before();
    const bool has_f = __syncthreads_or(kinds & 1) != 0;
    tm_fence_after();
    const bool has_s = __syncthreads_or(kinds & 2) != 0;
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
    Cta cta;
    cta.ci = ci;
    cta.sums = sums;
    cta.uni = __syncthreads_and(same) != 0;
    cta.nvalid = __syncthreads_count(valid);
    cta.tmem = tmem;
    if (has_f && has_s) tm_body<S, K2, kKindFS, SP>(p, smem_raw, cta, fco_s, sco_s);
    else if (has_s) tm_body<S, K2, kKindS, SP>(p, smem_raw, cta, fco_s, sco_s);
    else tm_body<S, K2, kKindF, SP>(p, smem_raw, cta, fco_s, sco_s);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
}

template <typename S, int K2, bool SP>
__global__ void __launch_bounds__(32 * kMaxWarps)
tmem_scan_kernel(const FastParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *tmem_slot = tm_slot(smem_raw, p.nw);
    // two warps share a lane quadrant when more than four run: 512 columns
    const uint32_t ncols = p.nw > 4 ? 2 * kRegion : kRegion;
    if (threadIdx.x < 32) tm_alloc(tmem_slot, ncols);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t tmem = *tmem_slot;
    tm_tile<S, K2, SP>(p, blockIdx.x, smem_raw, tmem);
    if (threadIdx.x < 32) tm_dealloc(tmem, ncols);
}

// Persistent launch over the column tiles of several games.
template <typename S, int K2, bool SP>
__global__ void __launch_bounds__(32 * kMaxWarps)
tmem_multi_kernel(const MultiParams m) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ FastParams sp;
    __shared__ long long s_tile;
    __shared__ int s_game;
    uint32_t *tmem_slot = tm_slot(smem_raw, m.nw);
    const uint32_t ncols = m.nw > 4 ? 2 * kRegion : kRegion;
    if (threadIdx.x < 32) tm_alloc(tmem_slot, ncols);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t tmem = *tmem_slot;
    int next = blockIdx.x;
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = m.schedule == 0 ? atomicAdd(m.ticket, 1) : next;
            next += gridDim.x;
            int g = -1;
            if (t < m.total_tiles) {
                g = m.tile_game[t];
                sp = m.games[g];
                sp.vin = static_cast<const S *>(m.vin) + m.in_off[g];
                sp.vout = static_cast<S *>(m.vout) + m.out_off[g];
                s_tile = t - m.tile_start[g];
            }
            s_game = g;
        }
        __syncthreads();
        if (s_game < 0) break;
        tm_tile<S, K2, SP>(sp, s_tile, smem_raw, tmem);
    }
    if (threadIdx.x < 32) tm_dealloc(tmem, ncols);
}

template <typename S, int K2, bool SP = false>
cudaError_t launch_t(const FastParams &p, size_t smem, cudaStream_t stream) {
    auto fn = tmem_scan_kernel<S, K2, SP>;
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

template <typename S, int K2, bool SP = false>
cudaError_t launch_multi_t(const MultiParams &m, size_t smem, int grid, cudaStream_t stream) {
    auto fn = tmem_multi_kernel<S, K2, SP>;
    {
        const cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void *>(fn), smem);
        if (e != cudaSuccess) return e;
    }
    if (m.total_tiles <= 0) return cudaSuccess;
    fn<<<grid, 32 * m.nw, smem, stream>>>(m);
    return cudaGetLastError();
}

template <typename S, int K2, bool SP = false>
int ctas_t(size_t smem, int nw) {
    // Resident CTAs per SM from the SM's limits: shared memory (1 KB
    // reserved per CTA), registers (allocated per warp in units of 256) and
    // thread slots.  The runtime's occupancy query reports one CTA per SM for
    // this kernel at every size, while two 4-warp CTAs do run side by side
    // (measured), so it is not used.
    auto fn = tmem_multi_kernel<S, K2, SP>;
    // raise the kernel's limit if needed (never lower it: another launch may need more)
    if (ensure_dyn_smem(reinterpret_cast<const void *>(fn), smem) != cudaSuccess) return 0;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return 0;
    int dev = 0, sm_smem = 0, sm_regs = 0, sm_threads = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sm_regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sm_threads, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess)
        return 0;
    const size_t per_cta_smem = smem + fa.sharedSizeBytes + 1024;
    const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;
    int n = (int)((size_t)sm_smem / per_cta_smem);
    n = std::min(n, sm_regs / (warp_regs * nw));
    n = std::min(n, sm_threads / (32 * nw));
    return n;
}

}  // namespace

size_t tmem_smem_bytes(int nc, int nw) { return tm_header_bytes(nw) + (size_t)nw * tm_warp_floats(nc) * 4; }

cudaError_t launch_tmem_scan(const FastParams &p, int storage, int k, cudaStream_t stream) {
    if (p.nc > 66 || p.nw < 1 || p.nw > kMaxWarps) return cudaErrorInvalidValue;
    const size_t smem = tmem_smem_bytes(p.nc, p.nw);
    switch (storage) {
        case kStoreF32:
            return k == 1 ? launch_t<float, 1>(p, smem, stream)
                          : p.spill ? launch_t<float, 2, true>(p, smem, stream) : launch_t<float, 2>(p, smem, stream);
        case kStoreBF16:
            return k == 1 ? launch_t<__nv_bfloat16, 1>(p, smem, stream)
                          : p.spill ? launch_t<__nv_bfloat16, 2, true>(p, smem, stream)
                                    : launch_t<__nv_bfloat16, 2>(p, smem, stream);
        case kStoreF16:
            return k == 1 ? launch_t<__half, 1>(p, smem, stream)
                          : p.spill ? launch_t<__half, 2, true>(p, smem, stream) : launch_t<__half, 2>(p, smem, stream);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_tmem_multi(const MultiParams &m, int storage, int k, int grid, cudaStream_t stream) {
    if (m.nc > 66 || m.nw < 1 || m.nw > kMaxWarps || grid < 1) return cudaErrorInvalidValue;
    const size_t smem = tmem_smem_bytes(m.nc, m.nw);
    switch (storage) {
        case kStoreF32:
            return k == 1 ? launch_multi_t<float, 1>(m, smem, grid, stream)
                          : m.spill ? launch_multi_t<float, 2, true>(m, smem, grid, stream)
                                    : launch_multi_t<float, 2>(m, smem, grid, stream);
        case kStoreBF16:
            return k == 1   ? launch_multi_t<__nv_bfloat16, 1>(m, smem, grid, stream)
                   : m.spill ? launch_multi_t<__nv_bfloat16, 2, true>(m, smem, grid, stream)
                             : launch_multi_t<__nv_bfloat16, 2>(m, smem, grid, stream);
        case kStoreF16:
            return k == 1   ? launch_multi_t<__half, 1>(m, smem, grid, stream)
                   : m.spill ? launch_multi_t<__half, 2, true>(m, smem, grid, stream)
                             : launch_multi_t<__half, 2>(m, smem, grid, stream);
        default: return cudaErrorInvalidValue;
    }
}

int tmem_multi_ctas_per_sm(int storage, int k, int nc, int nw) {
    const size_t smem = tmem_smem_bytes(nc, nw);
    int n = 0;
    switch (storage) {
        case kStoreF32: n = k == 1 ? ctas_t<float, 1>(smem, nw) : ctas_t<float, 2>(smem, nw); break;
        case kStoreBF16: n = k == 1 ? ctas_t<__nv_bfloat16, 1>(smem, nw) : ctas_t<__nv_bfloat16, 2>(smem, nw); break;
        case kStoreF16: n = k == 1 ? ctas_t<__half, 1>(smem, nw) : ctas_t<__half, 2>(smem, nw); break;
        default: return 0;
    }
    // tensor memory: 512 columns per SM
    const int by_tmem = nw > 4 ? 1 : 2;
    return n < by_tmem ? n : by_tmem;
}

}  // namespace kps
