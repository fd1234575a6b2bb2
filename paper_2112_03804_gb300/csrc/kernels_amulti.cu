// Kronecker-form payoff products of many games in one persistent launch
// (sm_103a), one vector per game and player, FP32 / BF16 / FP16 storage with
// FP32 arithmetic.
//
// Mathematics as in kernels_tma.cu (Prop. 1, Sec. 3):
//   out / lambda_out = K_F(w) + S (2 Lo_ord(b) - TB(b) + TA(b)),
//   a = lambda_in * y_f,  b = lambda_in * y_s,  w = F a - S b,
// K_F(w)[h] = Tot - P[c1] - P[c2] + w[h] (one-card hands: Tot - P[c1]).
//
// Organisation.  A work item is one game and up to 32 of its output
// sequences: lane j owns sequence sigma0 + j, with its own fold and
// showdown input rows and payoffs (a sequence without a fold or a
// showdown terminal reads a zero row and has a zero payoff for it).  The
// four warps of a CTA scan four chunks of the game's hand order in boxes
// of 16 hands (the chunks and per-box hand records of scan_records.h,
// built once per game and direction).  For each box every lane copies its
// own two 64-byte row segments with cp.async into its own 16-byte slots of
// the warp's ring ([chunk of 4 hands][lane]: conflict-free reads), and
// lanes 0-16 copy the box's 272-byte record block; a ring of three boxes
// keeps two in flight while one is scanned, and each lane waits only for
// its own copy groups (plus a warp barrier before reading the records and
// before a slot is refilled).  Per-card sums are float2 [card][lane]
// tables, one per warp.  Partial results of the first 16 boxes of a chunk
// stay in tensor memory (lane = column, a column per hand); later boxes go
// to a per-CTA scratch area in global memory (L2-resident).  The four
// chunks are combined in shared memory exactly as in the single-game
// kernel; the finishing pass reads each box's finishing records from the
// record ring (copied one box ahead with cp.async, 256 bytes per half-warp),
// and each lane writes its finished row segments with 16-byte stores.  CTAs are persistent: they take work items from an atomic ticket
// or a static stride.  No spin-waits (cp.async groups complete in
// hardware), no atomics on results: bit-reproducible.
#include "kernels.h"
#include "game.h"
#include "scan_records.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

namespace kps {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kNS = 3;                     // ring slots per warp
constexpr int kSlot = 4096;                // bytes per slot: fold rows, then showdown rows
constexpr int kRing = kNS * kSlot;         // per warp
constexpr int kRecRing = 2 * kNS * kScanBlock; // per warp: two record blocks per slot (split items)
constexpr int kTmemCols = 256;             // per CTA (two CTAs per SM)
constexpr int kMaxExtra = 8;               // chunk boxes past tensor memory (scratch)

// One game in one direction (device).
struct alignas(16) AmGame {
    int H, hs, nc, n_out;
    int nbox, pad0, pad1, pad2;
    int bchunk[kTmaWarps + 1];
    int pad3[3];
    int bchunk8[2 * kTmaWarps + 1];   // split items: each chunk cut in two at a tie-free box boundary
    int pad4[3];
    long long in_off, out_off;     // element offsets of the game's input / output vectors
    const int *fcol, *scol;        // per output sequence: its fold / showdown input sequence or -1
    const float *fcoef, *scoef;    // and the payoffs
    const unsigned char *rscan;    // [nbox][kScanBlock]
    const TmaFinRec *rfin;         // [nbox * 8]
};

struct AmArgs {
    const AmGame *games;
    const int4 *items;             // (game, first output sequence, split, 0)
    int nitems, nc, schedule;
    const void *vin;               // element type: the kernel's storage type
    void *vout;
    float *scratch;                // [grid][4 warps][kMaxExtra][16][32]
    int *ticket;
};

// Shared memory: the four rings, the four record rings, the four per-card
// tables (nc rows of 256 bytes), then the header (tensor-memory slot at
// +0, work item at +4, per-warp sums [2][4][32] floats at +16).
__host__ __device__ inline size_t am_ring_off(int w) { return (size_t)w * kRing; }
__host__ __device__ inline size_t am_rec_off(int w) { return (size_t)kTmaWarps * kRing + (size_t)w * kRecRing; }
__host__ __device__ inline size_t am_state_off(int w, int nc) { return am_rec_off(kTmaWarps) + (size_t)w * nc * 256; }
__host__ __device__ inline size_t am_hdr_off(int nc) { return am_state_off(kTmaWarps, nc); }
inline size_t am_smem_bytes(int nc) { return am_hdr_off(nc) + 16 + 2 * kTmaWarps * 32 * 4; }

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
// 16 bytes from global memory; the bytes past `src_bytes` (0 or 16) are zero
__device__ __forceinline__ void cp16(uint32_t dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void tm_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tm_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void tm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_st16(uint32_t taddr, const float *r) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "f"(r[0]), "f"(r[1]), "f"(r[2]), "f"(r[3]), "f"(r[4]), "f"(r[5]), "f"(r[6]), "f"(r[7]), "f"(r[8]), "f"(r[9]),
        "f"(r[10]), "f"(r[11]), "f"(r[12]), "f"(r[13]), "f"(r[14]), "f"(r[15])
        : "memory");
}
__device__ __forceinline__ void tm_ld16(uint32_t taddr, float *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7]), "=f"(r[8]),
          "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tm_wait_ld16(float *r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+f"(r[0]), "+f"(r[1]), "+f"(r[2]), "+f"(r[3]), "+f"(r[4]), "+f"(r[5]), "+f"(r[6]), "+f"(r[7]),
                   "+f"(r[8]), "+f"(r[9]), "+f"(r[10]), "+f"(r[11]), "+f"(r[12]), "+f"(r[13]), "+f"(r[14]), "+f"(r[15])::"memory");
}

// Storage types: a 16-byte chunk holds 4 FP32 or 8 BF16 / FP16 values.
template <typename T> struct Store;
template <> struct Store<float> {
    static constexpr int kPer = 4;
    __device__ static void load(const unsigned char *p, float *v) {
        const float4 u = *reinterpret_cast<const float4 *>(p);
        v[0] = u.x; v[1] = u.y; v[2] = u.z; v[3] = u.w;
    }
    __device__ static uint4 pack(const float *v) {
        return make_uint4(__float_as_uint(v[0]), __float_as_uint(v[1]), __float_as_uint(v[2]), __float_as_uint(v[3]));
    }
};
template <> struct Store<__nv_bfloat16> {
    static constexpr int kPer = 8;
    __device__ static void load(const unsigned char *p, float *v) {
        const uint4 u = *reinterpret_cast<const uint4 *>(p);
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            v[2 * i] = __uint_as_float(w[i] << 16);
            v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
        }
    }
    __device__ static uint4 pack(const float *v) {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
            w[i] = *reinterpret_cast<uint32_t *>(&h);
        }
        return make_uint4(w[0], w[1], w[2], w[3]);
    }
};
template <> struct Store<__half> {
    static constexpr int kPer = 8;
    __device__ static void load(const unsigned char *p, float *v) {
        const uint4 u = *reinterpret_cast<const uint4 *>(p);
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w[i]));
            v[2 * i] = f.x;
            v[2 * i + 1] = f.y;
        }
    }
    __device__ static uint4 pack(const float *v) {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __half2 h = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
            w[i] = *reinterpret_cast<uint32_t *>(&h);
        }
        return make_uint4(w[0], w[1], w[2], w[3]);
    }
};

// One work item, one warp: scan of the warp's chunk, combination of the
// four chunks (two CTA barriers), finishing pass.  A split item has at most
// 16 output sequences: lanes 16-31 take the same sequences as lanes 0-15 over
// the second half of the warp's chunk (eight sub-chunks in all), and the half
// with fewer boxes runs zero-filled boxes to the other's count, so that the
// warp's tensor-memory operations stay uniform.
template <typename T, int K2>
__device__ __forceinline__ void am_item(const AmArgs &P, const AmGame &G, int sigma0, int split, unsigned char *sm,
                                        uint32_t tmem, float *xs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nc = P.nc, hs = G.hs;
    const int half = split ? lane >> 4 : 0, col = split ? lane & 15 : lane;
    const int sub = split ? 2 * warp + half : warp;   // this lane's (sub-)chunk
    const int b0 = split ? G.bchunk8[sub] : G.bchunk[warp];
    const int nbl = (split ? G.bchunk8[sub + 1] : G.bchunk[warp + 1]) - b0;   // this lane's boxes
    const int b0h0 = __shfl_sync(kFull, b0, 0), b0h1 = __shfl_sync(kFull, b0, 16);
    const int nbh0 = __shfl_sync(kFull, nbl, 0), nbh1 = __shfl_sync(kFull, nbl, 16);
    const int nb = split ? max(nbh0, nbh1) : nbl;   // the warp's box count
    const int sigma = sigma0 + col;
    const bool act = sigma < G.n_out;
    const int rf = act ? G.fcol[sigma] : -1, rs = act ? G.scol[sigma] : -1;
    const float F = rf >= 0 ? G.fcoef[sigma] : 0.f;
    const float S = rs >= 0 ? G.scoef[sigma] : 0.f;
    const float S2 = 2.f * S;
    constexpr int NQ = 16 / Store<T>::kPer;   // 16-byte chunks per 16-hand row segment
    const T *vin = static_cast<const T *>(P.vin) + G.in_off;
    const T *pa = vin + (size_t)(rf >= 0 ? rf : 0) * hs;
    const T *pb = vin + (size_t)(rs >= 0 ? rs : 0) * hs;
    const uint32_t na = rf >= 0 ? 16u : 0u, nbytes_b = rs >= 0 ? 16u : 0u;
    unsigned char *ring = sm + am_ring_off(warp);
    const uint32_t ring_s = smem_u32(ring);
    unsigned char *rring = sm + am_rec_off(warp);
    const uint32_t rring_s = smem_u32(rring);
    unsigned char *stb = sm + am_state_off(warp, nc);
    unsigned char *lb = stb + 8 * lane;
    float *sums = reinterpret_cast<float *>(sm + am_hdr_off(nc) + 16);
    auto row = [&](uint32_t off) -> unsigned char * { return lb + 2 * off; };

    for (int q = lane; q < nc * 64; q += 32) reinterpret_cast<float *>(stb)[q] = 0.f;

    // copies of box m into slot m % kNS (an empty group past the chunk)
    auto issue = [&](int m) {
        if (m < nb) {
            const int sl = m % kNS;
            const bool real = m < nbl;   // past its half's boxes a lane copies zeros
            const int x = kTmaBox * (b0 + (real ? m : 0));
            const uint32_t dst = ring_s + (uint32_t)(sl * kSlot) + 16u * (uint32_t)lane;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int h0 = x + Store<T>::kPer * q;
                const bool in = real && h0 < hs;   // hs is a multiple of 8: a chunk is all in or all out
                cp16(dst + 512u * q, in ? pa + h0 : pa, in ? na : 0u);
                cp16(dst + 2048u + 512u * q, in ? pb + h0 : pb, in ? nbytes_b : 0u);
            }
            // the record block of each half's box (zeros for a zero-filled box)
            if (lane < kScanBlock / 16) {
                const bool r0 = m < nbh0;
                cp16(rring_s + (uint32_t)(2 * sl * kScanBlock) + 16u * (uint32_t)lane,
                     G.rscan + (size_t)(b0h0 + (r0 ? m : 0)) * kScanBlock + 16 * lane, r0 ? 16u : 0u);
                if (split) {
                    const bool r1 = m < nbh1;
                    cp16(rring_s + (uint32_t)((2 * sl + 1) * kScanBlock) + 16u * (uint32_t)lane,
                         G.rscan + (size_t)(b0h1 + (r1 ? m : 0)) * kScanBlock + 16 * lane, r1 ? 16u : 0u);
                }
            }
        }
        cp_commit();
    };
    for (int m = 0; m < kNS; ++m) issue(m);
    __syncwarp();

    float Gm = 0.f;
    float pp[16];
    float bq1 = 0.f, bq2 = 0.f, bq3 = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) pp[i] = 0.f;
    auto store_box = [&](int m, const float *r) {
        if (m < 16) {
            tm_st16(tmem + (uint32_t)(16 * m), r);
        } else {
            float *xp = xs + (m - 16) * (kTmaBox * 32);
#pragma unroll
            for (int i = 0; i < 16; ++i) xp[i * 32 + lane] = r[i];
        }
    };
    for (int m = 0; m < nb; ++m) {
        const int sl = m % kNS;
        cp_wait<kNS - 1>();
        __syncwarp();
        const unsigned char *slot = ring + sl * kSlot + 16 * lane;
        float yf[16], ys[16];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            Store<T>::load(slot + 512 * q, yf + Store<T>::kPer * q);
            Store<T>::load(slot + 2048 + 512 * q, ys + Store<T>::kPer * q);
        }
        const unsigned char *rsb = rring + (2 * sl + half) * kScanBlock;
        const uint32_t tw0 = reinterpret_cast<const uint32_t *>(rsb + 256)[0];
        const uint32_t tw1 = reinterpret_cast<const uint32_t *>(rsb + 256)[1];
        TmaScanRec rn = *reinterpret_cast<const TmaScanRec *>(rsb);
        float p[16], bv[16];
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
            const TmaScanRec r = rn;
            if (i + 2 < 16) rn = reinterpret_cast<const TmaScanRec *>(rsb)[i / 2 + 1];
            unsigned char *A1 = row(r.oa1), *A2 = row(r.oa2), *B1 = row(r.ob1), *B2 = row(r.ob2);
            float2 sa1 = *reinterpret_cast<const float2 *>(A1);
            float2 sa2 = *reinterpret_cast<const float2 *>(A2);
            float2 sb1 = make_float2(0.f, 0.f), sb2 = make_float2(0.f, 0.f);
            if (K2 == 2) {
                sb1 = *reinterpret_cast<const float2 *>(B1);
                sb2 = *reinterpret_cast<const float2 *>(B2);
            }
            const float b1 = r.lin1 * ys[i], b2 = r.lin2 * ys[i + 1];
            bv[i] = b1;
            bv[i + 1] = b2;
            const float w1 = fmaf(F, r.lin1 * yf[i], -(S * b1));
            const float w2 = fmaf(F, r.lin2 * yf[i + 1], -(S * b2));
            // the first hand's update, seen by the second hand's sums when
            // they share a card (ma, mb are 0 or 1)
            sa2.x = fmaf(r.ma, b1, sa2.x);
            sa2.y = fmaf(r.ma, w1, sa2.y);
            if (K2 == 2) {
                sb2.x = fmaf(r.mb, b1, sb2.x);
                sb2.y = fmaf(r.mb, w1, sb2.y);
            }
            // partial = w + S (2 Lo_ord - TB), the w only for two-card hands
            const float t1 = 2.f * (Gm - (sa1.x + sb1.x));
            const float g1 = Gm + b1;
            const float t2 = 2.f * (g1 - (sa2.x + sb2.x));
            Gm = g1 + b2;
            p[i] = fmaf(S, t1, K2 == 2 ? w1 : 0.f);
            p[i + 1] = fmaf(S, t2, K2 == 2 ? w2 : 0.f);
            *reinterpret_cast<float2 *>(A1) = make_float2(sa1.x + b1, sa1.y + w1);
            if (K2 == 2) *reinterpret_cast<float2 *>(B1) = make_float2(sb1.x + b1, sb1.y + w1);
            *reinterpret_cast<float2 *>(A2) = make_float2(sa2.x + b2, sa2.y + w2);
            if (K2 == 2) *reinterpret_cast<float2 *>(B2) = make_float2(sb2.x + b2, sb2.y + w2);
        }
        // tie corrections of the box (TB leaves each tied hand's partial,
        // TA enters the earlier partner's; partners before the box are the
        // previous box's last three hands, stored one box late)
        if (tw0 | tw1) {
            auto bat = [&](int j) { return j >= 0 ? bv[j] : (j == -1 ? bq1 : j == -2 ? bq2 : bq3); };
            auto pat = [&](int j) -> float & { return j >= 0 ? p[j] : pp[16 + j]; };
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint32_t tb = ((k < 4 ? tw0 : tw1) >> (8 * (k & 3))) & 0xfcu;
                if (tb) {
                    const int i = 2 * k;
#pragma unroll
                    for (int d = 1; d <= 3; ++d)
                        if (tb & (1u << (1 + d))) {
                            p[i] = fmaf(-S, bat(i - d), p[i]);
                            pat(i - d) = fmaf(S, bv[i], pat(i - d));
                        }
#pragma unroll
                    for (int d = 1; d <= 3; ++d)
                        if (tb & (1u << (4 + d))) {
                            p[i + 1] = fmaf(-S, bat(i + 1 - d), p[i + 1]);
                            pat(i + 1 - d) = fmaf(S, bv[i + 1], pat(i + 1 - d));
                        }
                }
            }
        }
        // every lane has read the slot's records: refill it
        __syncwarp();
        issue(m + kNS);
        if (m > 0) store_box(m - 1, pp);
#pragma unroll
        for (int i = 0; i < 16; ++i) pp[i] = p[i];
        bq1 = bv[15];
        bq2 = bv[14];
        bq3 = bv[13];
    }
    if (nb > 0) store_box(nb - 1, pp);
    cp_wait<0>();
    tm_wait_st();
    __syncwarp();

    // per-warp totals: b mass and K_F's Tot (every two-card hand is in two rows)
    float tot = 0.f;
    for (int q = 0; q < nc; ++q) tot += reinterpret_cast<const float2 *>(stb)[q * 32 + lane].y;
    if (K2 == 2) tot *= 0.5f;
    sums[(0 * kTmaWarps + warp) * 32 + lane] = Gm;
    sums[(1 * kTmaWarps + warp) * 32 + lane] = tot;
    __syncthreads();

    // combination: Q_k[c] = Pall[c] + 2 S (mass of card c in chunks < k),
    // [card][lane] floats at the start of warp k's ring; a split item's
    // sub-chunk k lives in warp k / 2, lanes 16 (k & 1) + column
    if (!split) {
        for (int q = warp; q < nc; q += kTmaWarps) {
            float rr[kTmaWarps], pw[kTmaWarps];
#pragma unroll
            for (int k = 0; k < kTmaWarps; ++k) {
                const float2 v = reinterpret_cast<const float2 *>(sm + am_state_off(k, nc))[q * 32 + lane];
                rr[k] = v.x;
                pw[k] = v.y;
            }
            const float pall = (pw[0] + pw[1]) + (pw[2] + pw[3]);
            float run = 0.f;
#pragma unroll
            for (int k = 0; k < kTmaWarps; ++k) {
                reinterpret_cast<float *>(sm + am_ring_off(k))[q * 32 + lane] = pall + S2 * run;
                run += rr[k];
            }
        }
    } else if (lane < 16) {
        for (int q = warp; q < nc; q += kTmaWarps) {
            float rr[2 * kTmaWarps], pw[2 * kTmaWarps];
#pragma unroll
            for (int k = 0; k < 2 * kTmaWarps; ++k) {
                const float2 v =
                    reinterpret_cast<const float2 *>(sm + am_state_off(k >> 1, nc))[q * 32 + lane + 16 * (k & 1)];
                rr[k] = v.x;
                pw[k] = v.y;
            }
            const float pall = ((pw[0] + pw[1]) + (pw[2] + pw[3])) + ((pw[4] + pw[5]) + (pw[6] + pw[7]));
            float run = 0.f;
#pragma unroll
            for (int k = 0; k < 2 * kTmaWarps; ++k) {
                reinterpret_cast<float *>(sm + am_ring_off(k >> 1))[q * 32 + lane + 16 * (k & 1)] = pall + S2 * run;
                run += rr[k];
            }
        }
    }
    float Cw;
    {
        float tall = 0.f, gb = 0.f;
        if (!split) {
#pragma unroll
            for (int k = 0; k < kTmaWarps; ++k) {
                tall += sums[(1 * kTmaWarps + k) * 32 + lane];
                if (k < warp) gb += sums[(0 * kTmaWarps + k) * 32 + lane];
            }
        } else {
#pragma unroll
            for (int k = 0; k < 2 * kTmaWarps; ++k) {
                const int at = (k >> 1) * 32 + col + 16 * (k & 1);
                tall += sums[1 * kTmaWarps * 32 + at];
                if (k < sub) gb += sums[at];
            }
        }
        Cw = tall + S2 * gb;
    }
    __syncthreads();

    // finishing: out = lambda_out (partial + C - Q[c1] - Q[c2])
    const unsigned char *qb = ring + 4 * lane;
    T *orow = static_cast<T *>(P.vout) + G.out_off + (size_t)(act ? sigma : 0) * hs;
    float cur[16], nxt[16];
    auto load_box = [&](int m, float *r) {
        if (m < 16) {
            tm_ld16(tmem + (uint32_t)(16 * m), r);
        } else {
            const float *xp = xs + (m - 16) * (kTmaBox * 32);
#pragma unroll
            for (int i = 0; i < 16; ++i) r[i] = xp[i * 32 + lane];
        }
    };
    // each half's finishing records of box m (256 bytes) are copied one box
    // ahead by its 16 lanes into two buffers in the record ring (idle after
    // the scan): [m & 1][half]
    const uint32_t frb_s = smem_u32(rring);
    auto fetch_fin = [&](int m) {
        if (m < nb && (split || lane < 16)) {
            const int bm = b0 + (m < nbl ? m : 0);   // a zero-filled box reads its half's first records
            cp16(frb_s + (uint32_t)((((m & 1) * 2 + half) * 256) + 16 * (lane & 15)),
                 reinterpret_cast<const unsigned char *>(G.rfin + (size_t)kTmaBox / 2 * bm) + 16 * (lane & 15), 16u);
        }
        cp_commit();
    };
    // box m: its partials in pc, box m + 1's loaded into pn (the two arrays
    // alternate, so no copy between boxes)
    auto box = [&](int m, const float *pc, float *pn) {
        if (m + 1 < nb) load_box(m + 1, pn);
        const bool real = m < nbl;   // a zero-filled box of the shorter half writes nothing
        __syncwarp();   // every lane has read box m - 1's records: refill their buffer
        fetch_fin(m + 1);
        cp_wait<1>();   // this lane's copy of box m's records
        __syncwarp();
        const TmaFinRec *fr = reinterpret_cast<const TmaFinRec *>(rring + ((m & 1) * 2 + half) * 256);
        float o[16];
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
            const TmaFinRec r = fr[i / 2];
            float q1 = *reinterpret_cast<const float *>(qb + r.oa1);
            float q2 = *reinterpret_cast<const float *>(qb + r.oa2);
            if (K2 == 2) {
                q1 += *reinterpret_cast<const float *>(qb + r.ob1);
                q2 += *reinterpret_cast<const float *>(qb + r.ob2);
            }
            o[i] = r.lout1 * ((pc[i] + Cw) - q1);
            o[i + 1] = r.lout2 * ((pc[i + 1] + Cw) - q2);
        }
        if (act && real) {
            const int x = kTmaBox * (b0 + m);
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (x + Store<T>::kPer * q < hs)
                    *reinterpret_cast<uint4 *>(orow + x + Store<T>::kPer * q) = Store<T>::pack(o + Store<T>::kPer * q);
        }
        if (m + 1 < nb) tm_wait_ld16(pn);
    };
    fetch_fin(0);
    if (nb > 0) {
        load_box(0, cur);
        tm_wait_ld16(cur);
    }
    for (int m = 0; m < nb; m += 2) {
        box(m, cur, nxt);
        if (m + 1 < nb) box(m + 1, nxt, cur);
    }
    cp_wait<0>();
    __syncwarp();
}

template <typename T, int K2>
__global__ void __launch_bounds__(128, 2) async_multi_kernel(const __grid_constant__ AmArgs P) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int warp = threadIdx.x >> 5;
    unsigned char *hdr = sm + am_hdr_off(P.nc);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(hdr);
    int *sitem = reinterpret_cast<int *>(hdr + 4);
    if (warp == 0) tm_alloc(smem_u32(tslot), kTmemCols);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t tmem = tbase + ((uint32_t)(32 * warp) << 16);
    float *xs = P.scratch + ((size_t)blockIdx.x * kTmaWarps + warp) * kMaxExtra * (kTmaBox * 32);
    int next = blockIdx.x;
    for (;;) {
        int item;
        if (P.schedule == 0) {
            if (threadIdx.x == 0) *sitem = atomicAdd(P.ticket, 1);
            __syncthreads();
            item = *sitem;
        } else {
            item = next;
            next += gridDim.x;
        }
        if (item >= P.nitems) break;
        const int4 it = P.items[item];
        am_item<T, K2>(P, P.games[it.x], it.y, it.z, sm, tmem, xs);
        // the next ticket is written only after every thread has read this one
        // (am_item ends its combination with a CTA barrier)
    }
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    if (warp == 0) tm_dealloc(tbase, kTmemCols);
}

}  // namespace

struct AmPlan {
    AmArgs a{};
    void *blob = nullptr;          // games, items, records
    float *scratch = nullptr;
    int grid_cap = 0;              // CTAs the scratch area holds
    int k = 2;
    int device = -1;
};

AmPlan *am_create(const std::vector<AmGameDesc> &games, int grid_cap, cudaStream_t stream, std::vector<char> *taken,
                  std::string *why) {
    if (games.empty() || grid_cap < 1) {
        *why = "no games";
        return nullptr;
    }
    const int ng = (int)games.size();
    std::vector<ScanRecords> rec(ng);
    taken->assign(ng, 0);
    int nc = 0, ntaken = 0;
    size_t rbytes = 0;
    long long nitems = 0;
    const int k = games[0].h->k;
    for (int i = 0; i < ng; ++i) {
        const AmGameDesc &d = games[i];
        if (d.h->k != k) {
            *why = "games with different hand sizes";
            return nullptr;
        }
        std::string w;
        try {
            w = build_scan_records(*d.h, d.lam_in, d.lam_out, kMaxExtra, &rec[i]);
        } catch (const std::bad_alloc &) {
            *why = "host allocation";
            return nullptr;
        }
        if (w.empty() && rec[i].hs % 8 != 0) w = "hand stride not a multiple of 8";
        if (!w.empty()) {
            // left to another kernel
            if (why->empty()) *why = "game " + std::to_string(i) + ": " + w;
            rec[i] = ScanRecords();
            continue;
        }
        (*taken)[i] = 1;
        ++ntaken;
        nc = std::max(nc, rec[i].nc);
        rbytes += (rec[i].bytes.size() + 255) / 256 * 256;
        nitems += (d.n_out + 31) / 32;
    }
    if (ntaken == 0) return nullptr;
    if (nitems > 0x7fffffffLL) {
        *why = "too many work items";
        return nullptr;
    }
    if (std::max<size_t>(am_smem_bytes(nc), 80 * 1024) > (size_t)max_dyn_smem()) {
        *why = "shared memory";
        return nullptr;
    }
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t o_games = 0, o_items = al(sizeof(AmGame) * ng), o_rec = o_items + al(sizeof(int4) * (size_t)nitems);
    const size_t total = o_rec + rbytes;
    AmPlan *p = new (std::nothrow) AmPlan();
    if (!p) {
        *why = "host allocation";
        return nullptr;
    }
    cudaError_t e = cudaMalloc(&p->blob, total);
    if (e == cudaSuccess)
        e = cudaMalloc(&p->scratch, (size_t)grid_cap * kTmaWarps * kMaxExtra * kTmaBox * 32 * sizeof(float));
    if (e != cudaSuccess) {
        if (p->blob) cudaFree(p->blob);
        delete p;
        *why = "device memory for the launch tables";
        return nullptr;
    }
    p->grid_cap = grid_cap;
    unsigned char *dev = static_cast<unsigned char *>(p->blob);
    std::vector<unsigned char> host(total, 0);
    std::vector<AmGame> g(ng);
    std::vector<int4> items;
    items.reserve((size_t)nitems);
    size_t ro = o_rec;
    for (int i = 0; i < ng; ++i) {
        const AmGameDesc &d = games[i];
        const ScanRecords &r = rec[i];
        AmGame &x = g[i];
        std::memset(&x, 0, sizeof(x));
        if (!(*taken)[i]) continue;
        x.H = r.H;
        x.hs = r.hs;
        x.nc = r.nc;
        x.n_out = d.n_out;
        x.nbox = r.nbox;
        for (int w = 0; w <= kTmaWarps; ++w) x.bchunk[w] = r.bchunk[w];
        x.in_off = d.in_off;
        x.out_off = d.out_off;
        x.fcol = d.fcol;
        x.scol = d.scol;
        x.fcoef = d.fcoef;
        x.scoef = d.scoef;
        std::memcpy(host.data() + ro, r.bytes.data(), r.bytes.size());
        x.rscan = dev + ro;
        x.rfin = reinterpret_cast<const TmaFinRec *>(dev + ro + (size_t)r.nbox * kScanBlock);
        ro += al(r.bytes.size());
        // sub-chunks of split items: each chunk cut at the tie-free box
        // boundary nearest its middle (an empty second half if there is none)
        const HostGame &h = *d.h;
        auto clean = [&](int bx) {
            return bx <= 0 || bx >= r.nbox || 16 * bx >= r.H || h.group_lo[16 * bx] == 16 * bx;
        };
        bool split_ok = true;
        for (int w = 0; w < kTmaWarps; ++w) {
            const int lo = r.bchunk[w], hi = r.bchunk[w + 1], ideal = (lo + hi) / 2;
            int mid = hi;
            for (int dd = 0; dd <= hi - lo && mid == hi; ++dd) {
                if (ideal - dd >= lo && clean(ideal - dd)) mid = ideal - dd;
                else if (ideal + dd <= hi && clean(ideal + dd)) mid = ideal + dd;
            }
            x.bchunk8[2 * w] = lo;
            x.bchunk8[2 * w + 1] = mid;
            split_ok = split_ok && mid - lo <= 16 && hi - mid <= 16;
        }
        x.bchunk8[2 * kTmaWarps] = r.nbox;
        // full items of 32 sequences; a tail of at most 16 as a split item
        const int nfull = d.n_out / 32, tail = d.n_out - 32 * nfull;
        for (int t = 0; t < nfull; ++t) items.push_back(make_int4(i, 32 * t, 0, 0));
        if (tail > 0) items.push_back(make_int4(i, 32 * nfull, tail <= 16 && split_ok ? 1 : 0, 0));
    }
    std::memcpy(host.data() + o_games, g.data(), sizeof(AmGame) * ng);
    if (!items.empty()) std::memcpy(host.data() + o_items, items.data(), sizeof(int4) * items.size());
    e = cudaMemcpyAsync(p->blob, host.data(), total, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        cudaFree(p->blob);
        cudaFree(p->scratch);
        delete p;
        *why = "uploading the launch tables";
        return nullptr;
    }
    p->a.games = reinterpret_cast<const AmGame *>(dev + o_games);
    p->a.items = reinterpret_cast<const int4 *>(dev + o_items);
    p->a.nitems = (int)nitems;
    p->a.nc = nc;
    p->k = k;
    cudaGetDevice(&p->device);
    return p;
}

void am_destroy(AmPlan *p) {
    if (!p) return;
    if (p->blob) cudaFree(p->blob);
    if (p->scratch) cudaFree(p->scratch);
    delete p;
}

// At least 80 KB of shared memory per CTA: never more than two CTAs per SM,
// so that their tensor memory (256 columns each) always fits.
static size_t am_launch_smem(int nc) { return std::max<size_t>(am_smem_bytes(nc), 80 * 1024); }

int am_grid_cap(const AmPlan *p) { return p->grid_cap; }

int am_ctas_per_sm(const AmPlan *p) {
    const size_t smem = am_launch_smem(p->a.nc);
    int dev = 0, per_sm = 0, reserved = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    const int by_smem = (int)((size_t)per_sm / (smem + (size_t)reserved));
    return std::max(0, std::min(2, by_smem));
}

cudaError_t launch_async_multi(AmPlan *p, int storage, const void *vin, void *vout, int *ticket, int schedule,
                               int grid, cudaStream_t stream) {
    // the scratch area holds the chunk boxes past tensor memory of grid_cap CTAs
    if (grid <= 0 || grid > p->grid_cap) return cudaErrorInvalidValue;
    AmArgs a = p->a;
    a.vin = vin;
    a.vout = vout;
    a.scratch = p->scratch;
    a.ticket = ticket;
    a.schedule = schedule;
    if (a.nitems == 0) return cudaSuccess;
    const size_t smem = am_launch_smem(a.nc);
    void (*fn)(AmArgs);
    switch (storage) {
        case kStoreF32: fn = p->k == 1 ? async_multi_kernel<float, 1> : async_multi_kernel<float, 2>; break;
        case kStoreBF16:
            fn = p->k == 1 ? async_multi_kernel<__nv_bfloat16, 1> : async_multi_kernel<__nv_bfloat16, 2>;
            break;
        case kStoreF16: fn = p->k == 1 ? async_multi_kernel<__half, 1> : async_multi_kernel<__half, 2>; break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void *>(fn), smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, 32 * kTmaWarps, smem, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace kps
