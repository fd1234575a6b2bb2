// Kronecker-form payoff products, TMA-staged (sm_103a): single game, FP32.
//
// Mathematics (Prop. 1, Sec. 3; the fold block is the card-removal
// compatibility of Sec. 4's eq. for C, the showdown block the strength sign
// times compatibility, whose inverse-D prefix sums are Technique B's):
//   out / lambda_out = K_F(w) + S (2 Lo(b) + TieC(b)),
//   a = lambda_in * y_f,  b = lambda_in * y_s,  w = F a - S b,
// with y_f / y_s the input rows of the output sequence's fold and showdown
// terminals (payoffs F and S), K_F(w)[h] = Tot - P[c1] - P[c2] + w[h]
// (P[c] the per-card totals; one-card hands: Tot - P[c1]), Lo the
// compatible strictly weaker mass and TieC the compatible tied mass.
//
// Ties without tie-aligned tiles.  The scan walks hands in library order
// (strength, then canonical index) and accumulates the compatible mass of
// every hand *before* the current one, Lo_ord.  With TB / TA the compatible
// tied mass before / after a hand in that order, Lo = Lo_ord - TB and
// TieC = TB + TA, so
//   2 Lo + TieC = 2 Lo_ord - TB + TA.
// Every tie group has at most 4 hands (the host checks it): a hand's tied
// partners are at most 3 positions away, and the two corrections are made in
// registers (the current 16-hand box and the previous one are held there).
//
// Organisation.  A CTA = one output sequence sigma and 32 consecutive
// vectors (lane j = vector b0 + j): all its columns share their input rows,
// payoffs and column kind (fold only, showdown only, both).  Four warps scan
// four chunks of the hand order (chunk boundaries at 16-hand boxes that cut
// no tie group).  For each box one lane issues cp.async.bulk.tensor copies
// of the box's [32 vectors][16 hands] from each input row into a 64-byte
// swizzled slot of the warp's ring (an mbarrier per slot); lanes read their
// row four hands at a time (conflict free under the swizzle).  Per-card sums
// live in shared memory [card][lane] (float2: mass of b for Lo, total of w
// for K_F), addressed by per-hand byte offsets from the box's hand records
// (copied by cp.async.bulk with the box into a record ring).  Two hands per
// step: all four per-card loads are issued together; when the second hand
// holds a card of the first, its loaded sums get the first hand's update in
// registers; the two hands' arithmetic (and the two halves of a float2 sum)
// runs as packed FP32x2 instructions.  Partial results stay on chip: the
// first 16 boxes of a chunk in tensor memory (lane = column, a column per
// hand, one tcgen05.st per box), later boxes in shared memory.  After a
// barrier the four chunks' per-card sums are combined into
// -Q[c] = -(Pall[c] + 2 S R_before[c]) at the start of each warp's ring, and
// each warp finishes its boxes: out = lambda_out ((partial + C) - (Q[c1] +
// Q[c2])) with C = Tot + 2 S G_before, the finishing records read from the
// record ring (copied one box ahead by cp.async), written into a swizzled
// box and stored with one cp.async.bulk.tensor per box.  No atomics:
// results are bit-reproducible.
//
// Waits are bounded: a wait that gives up sets *err; the warp scans no
// further box and finishes nothing, the CTA runs to its end without waiting
// again (its results are not valid), waits (bounded) for its copies still in
// flight and frees its tensor memory.
#include "kernels.h"
#include "game.h"
#include "scan_records.h"

#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

namespace kps {

constexpr int kTmaMaxExtra = 2;    // boxes of a chunk past the 256 tensor-memory columns

// Kernel arguments (__grid_constant__).
struct alignas(128) TmaArgs {
    CUtensorMap tin;               // input  [batch][n_in][H]  fp32, box 16 x 1 x 32, 64-byte swizzle
    CUtensorMap tout;              // output [batch][n_out][hs] fp32, same box
    int H, hs, nc, k, n_out, n_in, batch, nbb, nbox, extra;
    int stall_test;                // test hook: warp 0's first box expects 16 bytes that never come
    int bchunk[kTmaWarps + 1];     // warp k scans boxes [bchunk[k], bchunk[k+1])
    const int *fcol, *scol;        // per output sequence: its fold / showdown input sequence or -1
    const float *fcoef, *scoef;    // and the payoffs
    const unsigned char *rscan;    // [nbox][kScanBlock]
    const TmaFinRec *rfin;         // [nbox * 8]
    unsigned int *err;             // set to 1 when a wait gives up
};

// Host side of one direction: the arguments and the record tables.
struct TmaParams {
    TmaArgs a;
    void *dev = nullptr;           // device copy of the records (scan blocks, then finishing records)
    std::vector<unsigned char> host;
    int device = -1;
};

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kRingBytes = 12288;          // per warp: 3 slots of 4 KB or 6 of 2 KB
constexpr int kRecRing = 6 * kScanBlock;   // per warp: one scan block per slot
constexpr int kTmemCols = 256;             // per CTA (two CTAs per SM)
constexpr int kHdrBytes = 1536;            // tensor-memory slot, barriers, per-warp sums
constexpr unsigned long long kWaitNs = 2000000000ull;   // give up after 2 s

enum Kind { kKindF = 1, kKindS = 2, kKindFS = 3 };

// Shared memory (from a 1 KB aligned base): the four warps' rings, their
// per-card tables (nc rows of 256 bytes), their overflow boxes of partial
// results, their record rings, then the header (tensor-memory slot at +0,
// 4 x 8 mbarriers at +16, per-warp sums [2][4][32] floats at +272).
__host__ __device__ inline size_t ring_off(int w) { return (size_t)w * kRingBytes; }
__host__ __device__ inline size_t state_off(int w, int nc) { return (size_t)kTmaWarps * kRingBytes + (size_t)w * nc * 256; }
__host__ __device__ inline size_t extra_off(int w, int nc, int extra) {
    return state_off(kTmaWarps, nc) + (size_t)w * extra * kTmaBox * 32 * 4;
}
__host__ __device__ inline size_t rec_off(int w, int nc, int extra) {
    return extra_off(kTmaWarps, nc, extra) + (size_t)w * kRecRing;
}
__host__ __device__ inline size_t hdr_off(int nc, int extra) { return rec_off(kTmaWarps, nc, extra); }

// ---- PTX wrappers ------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait for phase `parity` of a barrier; false when it gave up.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = gtime();
    for (int i = 0; i < (1 << 26); ++i) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 63) == 63 && gtime() - t0 > kWaitNs) break;
    }
    return false;
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tma_load3(uint32_t dst, const CUtensorMap *map, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
                 : "memory");
}
// 16-byte copy global -> shared by this thread (cp.async, L2 only)
__device__ __forceinline__ void cp16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void tma_store3(const CUtensorMap *map, int x, int y, int z, uint32_t src) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(z), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
// the same with a run-time count of at most 5 groups still reading
__device__ __forceinline__ void bulk_wait_read_n(int n) {
    if (n <= 0) bulk_wait_read<0>();
    else if (n == 1) bulk_wait_read<1>();
    else if (n == 2) bulk_wait_read<2>();
    else if (n == 3) bulk_wait_read<3>();
    else if (n == 4) bulk_wait_read<4>();
    else bulk_wait_read<5>();
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
// waits for this thread's tensor-memory loads; names the 16 destination
// registers so that no use of them is scheduled before the data arrive
__device__ __forceinline__ void tm_wait_ld16(float *r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+f"(r[0]), "+f"(r[1]), "+f"(r[2]), "+f"(r[3]), "+f"(r[4]), "+f"(r[5]), "+f"(r[6]), "+f"(r[7]),
                   "+f"(r[8]), "+f"(r[9]), "+f"(r[10]), "+f"(r[11]), "+f"(r[12]), "+f"(r[13]), "+f"(r[14]), "+f"(r[15])::"memory");
}

// Packed FP32x2 arithmetic (each component rounded to nearest, as the
// scalar instruction would be).
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Byte offset of lane `row`'s 16-byte chunk q (hands 4q..4q+3) in a
// [32][16] fp32 box written by the 64-byte swizzle: chunk bits 4-5 are
// XORed with address bits 7-8 (the row pair).
__device__ __forceinline__ uint32_t swz(int row, int q) {
    return (uint32_t)(row * 64 + ((q ^ ((row >> 1) & 3)) << 4));
}

// The CTA's column set, its warp's chunk and its shared-memory regions.
struct Ctx {
    unsigned char *sm;
    int lane, warp;
    int bb, sigma, rf, rs;
    float F, S;
    int b0, nb;                // first box of the chunk, boxes in it
    uint32_t tmem;             // the warp's tensor-memory lanes, column 0
    bool ok;                   // no wait gave up
};

// Scan and combination of one column kind; returns this warp's C.
template <int KIND, int K2>
__device__ __forceinline__ float tma_scan(const TmaArgs &P, Ctx &c) {
    constexpr bool HF = (KIND & kKindF) != 0, HS = (KIND & kKindS) != 0, FS = KIND == kKindFS;
    constexpr int NS = FS ? 3 : 6;                    // ring slots
    constexpr int SLOT = FS ? 4096 : 2048;            // bytes per slot
    const int lane = c.lane, warp = c.warp, nc = P.nc;
    unsigned char *ring = c.sm + ring_off(warp);
    const uint32_t ring_s = smem_u32(ring);
    unsigned char *hdr = c.sm + hdr_off(nc, P.extra);
    const uint32_t bar0 = smem_u32(hdr + 16) + 8u * 8u * (uint32_t)warp;
    unsigned char *rring = c.sm + rec_off(warp, nc, P.extra);
    const uint32_t rring_s = smem_u32(rring);
    // per-card table of the chunk, [card][lane]: float2 {b mass, w total}
    // for columns of both kinds (rows of 256 bytes, row offset 2 * off),
    // one float otherwise (rows of 128 bytes, offset off)
    unsigned char *stb = c.sm + state_off(warp, nc);
    unsigned char *lb = stb + (FS ? 8 : 4) * lane;
    float *xpart = reinterpret_cast<float *>(c.sm + extra_off(warp, nc, P.extra));
    float *sums = reinterpret_cast<float *>(hdr + 272);
    const float F = c.F, S = c.S, S2 = 2.f * c.S;
    const int nb = c.nb;
    const int z0 = 32 * c.bb;
    auto row = [&](uint32_t off) -> unsigned char * { return lb + (FS ? 2 * off : off); };

    for (int q = lane; q < nc * (FS ? 64 : 32); q += 32) reinterpret_cast<float *>(stb)[q] = 0.f;

    auto issue = [&](int m) {
        const int sl = m % NS;
        const uint32_t bar = bar0 + 8u * (uint32_t)sl;
        const uint32_t dst = ring_s + (uint32_t)(sl * SLOT);
        const int x = kTmaBox * (c.b0 + m);
        mbar_expect_tx(bar, (uint32_t)(SLOT + kScanBlock) + (P.stall_test && m == 0 && warp == 0 ? 16u : 0u));
        if (HF) tma_load3(dst, &P.tin, x, c.rf, z0, bar);
        if (HS) tma_load3(dst + (HF ? 2048u : 0u), &P.tin, x, c.rs, z0, bar);
        bulk_load(rring_s + (uint32_t)(sl * kScanBlock), P.rscan + (size_t)(c.b0 + m) * kScanBlock, kScanBlock, bar);
    };
    if (lane == 0) {
        for (int sl = 0; sl < NS; ++sl) mbar_init(bar0 + 8u * (uint32_t)sl, 1);
        fence_barrier_init();
        for (int m = 0; m < NS && m < nb; ++m) issue(m);
    }
    __syncwarp();
    int nissued = min(NS, nb), nwaited = 0;   // boxes copied in / waited for (warp-uniform)

    // ---- scan (lane = column)
    float G2 = 0.f;               // twice the b mass before the current hand
    float2 pp[8];                 // the previous box's partial results (stored one box late)
    float bq1 = 0.f, bq2 = 0.f, bq3 = 0.f;   // b of the previous box's hands 15, 14, 13
    const float2 F2 = make_float2(F, F), S2v = make_float2(S, S), nS2 = make_float2(-S, -S);
#pragma unroll
    for (int k = 0; k < 8; ++k) pp[k] = make_float2(0.f, 0.f);
    auto store_box = [&](int m, const float2 *r) {
        if (m < 16) {
            tm_st16(c.tmem + (uint32_t)(16 * m), reinterpret_cast<const float *>(r));
        } else {
            float *xp = xpart + (m - 16) * (kTmaBox * 32);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                xp[(2 * k) * 32 + lane] = r[k].x;
                xp[(2 * k + 1) * 32 + lane] = r[k].y;
            }
        }
    };
    for (int m = 0; m < nb; ++m) {
        const int sl = m % NS;
        if (c.ok) {
            // the first try inline (the box is usually there), then the
            // bounded loop
            const uint32_t bar = bar0 + 8u * (uint32_t)sl, par = (uint32_t)((m / NS) & 1);
            const bool got = mbar_try(bar, par) || mbar_wait(bar, par);
            c.ok = __all_sync(kFull, got);
            if (c.ok) nwaited = m + 1;
        }
        // after a wait gave up, the slot's records (shared-memory offsets)
        // may never have arrived: scan no further
        if (!c.ok) break;
        const unsigned char *slot = ring + sl * SLOT;
        // the box's inputs as hand pairs (2i, 2i+1)
        float2 yf[8], ys[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (HF) {
                const float4 v = *reinterpret_cast<const float4 *>(slot + swz(lane, q));
                yf[2 * q] = make_float2(v.x, v.y);
                yf[2 * q + 1] = make_float2(v.z, v.w);
            } else {
                yf[2 * q] = yf[2 * q + 1] = make_float2(0.f, 0.f);
            }
            if (HS) {
                const float4 v = *reinterpret_cast<const float4 *>(slot + (HF ? 2048 : 0) + swz(lane, q));
                ys[2 * q] = make_float2(v.x, v.y);
                ys[2 * q + 1] = make_float2(v.z, v.w);
            } else {
                ys[2 * q] = ys[2 * q + 1] = make_float2(0.f, 0.f);
            }
        }
        // the box's records: the next pair's are read before this pair's
        // per-card stores (program order keeps them ahead)
        const unsigned char *rs = rring + sl * kScanBlock;
        const uint32_t tw0 = reinterpret_cast<const uint32_t *>(rs + 256)[0];
        const uint32_t tw1 = reinterpret_cast<const uint32_t *>(rs + 256)[1];
        TmaScanRec rn = *reinterpret_cast<const TmaScanRec *>(rs);
        // two hands per step; the arithmetic of the two hands (or of the two
        // halves of a per-card float2) runs as packed FP32x2 instructions,
        // each component rounded as the scalar operation would be
        float2 p[8], bv[8];
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
            const int k = i / 2;
            const TmaScanRec r = rn;
            if (i + 2 < 16) rn = reinterpret_cast<const TmaScanRec *>(rs)[k + 1];
            unsigned char *A1 = row(r.oa1), *A2 = row(r.oa2), *B1 = row(r.ob1), *B2 = row(r.ob2);
            const float2 lin = make_float2(r.lin1, r.lin2);
            // the two hands' inputs: a (fold side), b (showdown side), w
            const float2 bb = HS ? mul2(lin, ys[k]) : make_float2(0.f, 0.f);
            bv[k] = bb;
            float2 ww;
            if (FS) ww = fma2(F2, mul2(lin, yf[k]), mul2(nS2, bb));   // F a - S b
            else if (HF) ww = mul2(F2, mul2(lin, yf[k]));
            else ww = make_float2(0.f, 0.f);   // a showdown-only column tracks b alone
            float cs1, cs2;   // b mass of the hands' cards before them
            if (FS) {
                // per-card rows {b mass, w total}
                float2 sa1 = *reinterpret_cast<const float2 *>(A1);
                float2 sa2 = *reinterpret_cast<const float2 *>(A2);
                float2 sb1 = make_float2(0.f, 0.f), sb2 = make_float2(0.f, 0.f);
                if (K2 == 2) {
                    sb1 = *reinterpret_cast<const float2 *>(B1);
                    sb2 = *reinterpret_cast<const float2 *>(B2);
                }
                const float2 h1 = make_float2(bb.x, ww.x), h2 = make_float2(bb.y, ww.y);
                // the first hand's update, seen by the second hand's sums
                // when they share a card (ma, mb are 0 or 1)
                sa2 = fma2(make_float2(r.ma, r.ma), h1, sa2);
                if (K2 == 2) sb2 = fma2(make_float2(r.mb, r.mb), h1, sb2);
                cs1 = sa1.x + sb1.x;
                cs2 = sa2.x + sb2.x;
                *reinterpret_cast<float2 *>(A1) = add2(sa1, h1);
                if (K2 == 2) *reinterpret_cast<float2 *>(B1) = add2(sb1, h1);
                *reinterpret_cast<float2 *>(A2) = add2(sa2, h2);
                if (K2 == 2) *reinterpret_cast<float2 *>(B2) = add2(sb2, h2);
            } else {
                // one float per card: {first card, second card} of each hand
                float2 s1 = make_float2(*reinterpret_cast<const float *>(A1), 0.f);
                float2 s2 = make_float2(*reinterpret_cast<const float *>(A2), 0.f);
                if (K2 == 2) {
                    s1.y = *reinterpret_cast<const float *>(B1);
                    s2.y = *reinterpret_cast<const float *>(B2);
                }
                const float d1 = HS ? bb.x : ww.x, d2 = HS ? bb.y : ww.y;
                s2 = fma2(make_float2(r.ma, r.mb), make_float2(d1, d1), s2);
                cs1 = s1.x + s1.y;
                cs2 = s2.x + s2.y;
                const float2 u1 = add2(s1, make_float2(d1, d1)), u2 = add2(s2, make_float2(d2, d2));
                *reinterpret_cast<float *>(A1) = u1.x;
                if (K2 == 2) *reinterpret_cast<float *>(B1) = u1.y;
                *reinterpret_cast<float *>(A2) = u2.x;
                if (K2 == 2) *reinterpret_cast<float *>(B2) = u2.y;
            }
            if (HS) {
                // t = 2 Lo_ord - TB (b units), from the running 2G;
                // partial = w + S t, the w only for two-card hands (see K_F)
                const float gA = G2, gB = fmaf(2.f, bb.x, G2);
                G2 = fmaf(2.f, bb.y, gB);
                const float2 t = fma2(make_float2(-2.f, -2.f), make_float2(cs1, cs2), make_float2(gA, gB));
                p[k] = fma2(S2v, t, K2 == 2 ? ww : make_float2(0.f, 0.f));
                if (!HF && K2 == 2) p[k] = fma2(nS2, bb, p[k]);   // showdown only: w = -S b
            } else {
                p[k] = K2 == 2 ? ww : make_float2(0.f, 0.f);
            }
        }
        // tie corrections of the box (partial = w + S (2 Lo_ord - TB + TA)):
        // TB leaves each tied hand's partial, TA enters the earlier
        // partner's; partners before the box are the previous box's last
        // three hands (their partials are stored one box late)
        if (HS && (tw0 | tw1)) {
            auto hb = [&](int j) -> float { return (j & 1) ? bv[j >> 1].y : bv[j >> 1].x; };
            auto bat = [&](int j) { return j >= 0 ? hb(j) : (j == -1 ? bq1 : j == -2 ? bq2 : bq3); };
            auto pat = [&](int j) -> float & {
                float2 &v = j >= 0 ? p[j >> 1] : pp[(16 + j) >> 1];
                return (j & 1) ? v.y : v.x;
            };
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint32_t tb = ((k < 4 ? tw0 : tw1) >> (8 * (k & 3))) & 0xfcu;
                if (tb) {
                    const int i = 2 * k;
#pragma unroll
                    for (int d = 1; d <= 3; ++d)
                        if (tb & (1u << (1 + d))) {
                            p[k].x = fmaf(-S, bat(i - d), p[k].x);
                            pat(i - d) = fmaf(S, bv[k].x, pat(i - d));
                        }
#pragma unroll
                    for (int d = 1; d <= 3; ++d)
                        if (tb & (1u << (4 + d))) {
                            p[k].y = fmaf(-S, bat(i + 1 - d), p[k].y);
                            pat(i + 1 - d) = fmaf(S, bv[k].y, pat(i + 1 - d));
                        }
                }
            }
        }
        // every lane has used the slot's values: refill it
        __syncwarp();
        if (c.ok && m + NS < nb) {
            if (lane == 0) {
                fence_proxy_async();
                issue(m + NS);
            }
            nissued = m + NS + 1;
        }
        if (m > 0) store_box(m - 1, pp);
#pragma unroll
        for (int k = 0; k < 8; ++k) pp[k] = p[k];
        bq1 = bv[7].y;
        bq2 = bv[7].x;
        bq3 = bv[6].y;
    }
    if (nb > 0) store_box(nb - 1, pp);
    tm_wait_st();
    if (!c.ok && lane == 0) {
        // a wait gave up: wait (bounded) for the copies still in flight
        // before the ring is reused or the CTA exits
        for (int m = nwaited; m < nissued; ++m)
            if (!mbar_wait(bar0 + 8u * (uint32_t)(m % NS), (uint32_t)((m / NS) & 1))) break;
    }
    __syncwarp();

    // per-warp totals: G (b mass) and Tot (w total; K_F's Tot)
    float tot = 0.f;
    if (HF) {
        for (int q = 0; q < nc; ++q)
            tot += FS ? reinterpret_cast<const float2 *>(stb)[q * 32 + lane].y
                      : reinterpret_cast<const float *>(stb)[q * 32 + lane];
        if (K2 == 2) tot *= 0.5f;
    } else {
        tot = -S * (0.5f * G2);
    }
    sums[(0 * kTmaWarps + warp) * 32 + lane] = 0.5f * G2;
    sums[(1 * kTmaWarps + warp) * 32 + lane] = tot;
    __syncthreads();

    // ---- combination: -Q_k[c] with Q_k[c] = Pall[c] + 2 S (mass of card c
    // in chunks < k), [card][lane] floats at the start of warp k's ring (free
    // now: every copy in has been consumed)
    for (int q = warp; q < nc; q += kTmaWarps) {
        float rr[kTmaWarps], pw[kTmaWarps];
#pragma unroll
        for (int k = 0; k < kTmaWarps; ++k) {
            const unsigned char *sk = c.sm + state_off(k, nc);
            if (FS) {
                const float2 v = reinterpret_cast<const float2 *>(sk)[q * 32 + lane];
                rr[k] = v.x;
                pw[k] = v.y;
            } else {
                const float v = reinterpret_cast<const float *>(sk)[q * 32 + lane];
                rr[k] = HS ? v : 0.f;
                pw[k] = HS ? -S * v : v;
            }
        }
        const float pall = (pw[0] + pw[1]) + (pw[2] + pw[3]);
        float run = 0.f;
#pragma unroll
        for (int k = 0; k < kTmaWarps; ++k) {
            reinterpret_cast<float *>(c.sm + ring_off(k))[q * 32 + lane] = -(pall + S2 * run);
            run += rr[k];
        }
    }
    float Cw;
    {
        float T = 0.f, gb = 0.f;
#pragma unroll
        for (int k = 0; k < kTmaWarps; ++k) {
            T += sums[(1 * kTmaWarps + k) * 32 + lane];
            if (k < warp) gb += sums[(0 * kTmaWarps + k) * 32 + lane];
        }
        Cw = T + S2 * gb;
    }
    __syncthreads();

    return Cw;
}

// Finishing pass (the same for every column kind): out = lambda_out
// ((partial + C) - (Q[c1] + Q[c2])), staged in swizzled boxes (the rest of the
// ring, 2 KB each) and stored by TMA.  A box's finishing records (256 bytes)
// are copied one box ahead by cp.async into two buffers in the warp's record
// ring (idle after the scan).  A warp whose scan gave up finishes nothing: a
// copy into its ring may still be in flight.
template <int K2>
__device__ __forceinline__ void tma_finish(const TmaArgs &P, const Ctx &c, float Cw) {
    if (!c.ok) return;
    const int lane = c.lane, nc = P.nc, nb = c.nb, z0 = 32 * c.bb;
    unsigned char *ring = c.sm + ring_off(c.warp);
    const float *xpart = reinterpret_cast<const float *>(c.sm + extra_off(c.warp, nc, P.extra));
    const unsigned char *qb = ring + 4 * lane;
    const int qbytes = (nc * 128 + 1023) & ~1023;
    const int nbuf = (kRingBytes - qbytes) / 2048;
    unsigned char *frb = c.sm + rec_off(c.warp, nc, P.extra);
    const uint32_t frb_s = smem_u32(frb);
    auto fetch_fin = [&](int m) {
        if (m < nb && lane < 16)
            cp16(frb_s + (uint32_t)((m & 1) * 256 + 16 * lane),
                 reinterpret_cast<const unsigned char *>(P.rfin + (size_t)kTmaBox / 2 * (c.b0 + m)) + 16 * lane);
        cp_commit();
    };
    float cur[16], nxt[16];
    auto load_box = [&](int m, float *r) {
        if (m < 16) {
            tm_ld16(c.tmem + (uint32_t)(16 * m), r);
        } else {
            const float *xp = xpart + (m - 16) * (kTmaBox * 32);
#pragma unroll
            for (int i = 0; i < 16; ++i) r[i] = xp[i * 32 + lane];
        }
    };
    // box m of the chunk: its partials in pc, box m + 1's loaded into pn
    // (the two arrays alternate, so no copy between boxes)
    auto box = [&](int m, const float *pc, float *pn) {
        if (m + 1 < nb) load_box(m + 1, pn);
        fetch_fin(m + 1);
        cp_wait<1>();   // this lane's copy of box m's records
        __syncwarp();
        const TmaFinRec *fr = reinterpret_cast<const TmaFinRec *>(frb + (m & 1) * 256);
        float2 o[8];
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
            const TmaFinRec r = fr[i / 2];
            // the table holds -Q: nq = -(Q[c1] + Q[c2]) for both hands
            float2 nq = make_float2(*reinterpret_cast<const float *>(qb + r.oa1),
                                    *reinterpret_cast<const float *>(qb + r.oa2));
            if (K2 == 2)
                nq = add2(nq, make_float2(*reinterpret_cast<const float *>(qb + r.ob1),
                                          *reinterpret_cast<const float *>(qb + r.ob2)));
            o[i / 2] = mul2(make_float2(r.lout1, r.lout2),
                            add2(add2(make_float2(pc[i], pc[i + 1]), make_float2(Cw, Cw)), nq));
        }
        const int ob = m % nbuf;
        unsigned char *buf = ring + qbytes + ob * 2048;
        if (m >= nbuf) {
            if (lane == 0) bulk_wait_read_n(nbuf - 1);
            __syncwarp();
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<float4 *>(buf + swz(lane, q)) =
                make_float4(o[2 * q].x, o[2 * q].y, o[2 * q + 1].x, o[2 * q + 1].y);
        fence_proxy_async();
        // every lane has read box m's records (their buffer is refilled
        // with box m + 2 in the next box) and staged its outputs
        __syncwarp();
        if (lane == 0) {
            tma_store3(&P.tout, kTmaBox * (c.b0 + m), c.sigma, z0, smem_u32(buf));
            bulk_commit();
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
    if (lane == 0) bulk_wait_read<0>();
    __syncwarp();
}

template <int K2>
__global__ void __launch_bounds__(128, 2) tma_scan_kernel(const __grid_constant__ TmaArgs P) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // the swizzled boxes need 1 KB alignment (one KB of slack is allocated)
    unsigned char *sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    Ctx c;
    c.sm = sm;
    c.lane = threadIdx.x & 31;
    c.warp = threadIdx.x >> 5;
    c.bb = blockIdx.x / P.n_out;
    c.sigma = blockIdx.x - c.bb * P.n_out;
    c.rf = P.fcol[c.sigma];
    c.rs = P.scol[c.sigma];
    c.F = c.rf >= 0 ? P.fcoef[c.sigma] : 0.f;
    c.S = c.rs >= 0 ? P.scoef[c.sigma] : 0.f;
    c.b0 = P.bchunk[c.warp];
    c.nb = P.bchunk[c.warp + 1] - c.b0;
    c.ok = true;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + hdr_off(P.nc, P.extra));
    if (c.warp == 0) tm_alloc(smem_u32(tslot), kTmemCols);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t tbase = *tslot;
    c.tmem = tbase + ((uint32_t)(32 * c.warp) << 16);
    const int kind = (c.rf >= 0 ? kKindF : 0) | (c.rs >= 0 ? kKindS : 0);
    float Cw;
    if (kind == kKindFS) Cw = tma_scan<kKindFS, K2>(P, c);
    else if (kind == kKindF) Cw = tma_scan<kKindF, K2>(P, c);
    else Cw = tma_scan<kKindS, K2>(P, c);
    tma_finish<K2>(P, c, Cw);
    if (!c.ok && c.lane == 0) atomicExch(P.err, 1u);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    if (c.warp == 0) tm_dealloc(tbase, kTmemCols);
}

// ---- host ------------------------------------------------------------------
using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn(cudaError_t *err) {
    static std::once_flag once;
    static EncodeFn fn = nullptr;
    static cudaError_t status = cudaSuccess;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        status = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (status == cudaSuccess && (q != cudaDriverEntryPointSuccess || !p)) status = cudaErrorSymbolNotFound;
        if (status == cudaSuccess) fn = reinterpret_cast<EncodeFn>(p);
    });
    *err = status;
    return fn;
}

cudaError_t encode3(CUtensorMap *map, const void *base, int x, int y, int z, int pitch) {
    cudaError_t e;
    EncodeFn fn = encode_fn(&e);
    if (!fn) return e;
    const cuuint64_t dims[3] = {(cuuint64_t)x, (cuuint64_t)y, (cuuint64_t)z};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * 4, (cuuint64_t)pitch * 4 * (cuuint64_t)y};
    const cuuint32_t box[3] = {(cuuint32_t)kTmaBox, 1, 32};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

__device__ unsigned int g_tma_err;

}  // namespace

static size_t tma_smem_bytes(int nc, int extra) { return hdr_off(nc, extra) + kHdrBytes + 1024; }

// Chunks, records and eligibility of one direction; fills p.a (but the
// tensor maps, pointers and batch) and p.host.  Empty string on success.
static std::string tma_prepare(const HostGame &h, const double *lam_in, const double *lam_out, TmaParams &p) {
    ScanRecords r;
    const std::string why = build_scan_records(h, lam_in, lam_out, kTmaMaxExtra, &r);
    if (!why.empty()) return why;
    TmaArgs &A = p.a;
    A.H = r.H;
    A.hs = r.hs;
    A.nc = r.nc;
    A.k = r.k;
    A.nbox = r.nbox;
    A.extra = r.extra;
    for (int k = 0; k <= kTmaWarps; ++k) A.bchunk[k] = r.bchunk[k];
    p.host = std::move(r.bytes);
    return "";
}

}  // namespace kps

namespace kps {

TmaParams *tma_create(const HostGame &h, const double *lam_in, const double *lam_out, int n_out, int n_in,
                      const int *fcol, const int *scol, const float *fcoef, const float *scoef,
                      const int *hfcol, const int *hscol, std::string *why) {
    TmaParams *p = new (std::nothrow) TmaParams();
    if (!p) {
        *why = "host allocation";
        return nullptr;
    }
    std::string w;
    try {
        w = tma_prepare(h, lam_in, lam_out, *p);
    } catch (const std::bad_alloc &) {
        w = "host allocation";
    }
    for (int r = 0; r < n_out && w.empty(); ++r)
        if (hfcol[r] < 0 && hscol[r] < 0) w = "an output sequence without terminals";
    if (w.empty() && std::max<size_t>(tma_smem_bytes(p->a.nc, p->a.extra), 80 * 1024) > (size_t)max_dyn_smem())
        w = "shared memory";
    if (!w.empty()) {
        delete p;
        *why = w;
        return nullptr;
    }
    p->a.n_out = n_out;
    p->a.n_in = n_in;
    p->a.fcol = fcol;
    p->a.scol = scol;
    p->a.fcoef = fcoef;
    p->a.scoef = scoef;
    p->a.err = nullptr;
    return p;
}

cudaError_t tma_take_error(bool *set) {
    unsigned int v = 0, zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_tma_err, sizeof(v));
    if (e == cudaSuccess && v) e = cudaMemcpyToSymbol(g_tma_err, &zero, sizeof(zero));
    *set = v != 0;
    return e;
}

void tma_destroy(TmaParams *p) {
    if (!p) return;
    if (p->dev) cudaFree(p->dev);
    delete p;
}

cudaError_t launch_tma_scan(TmaParams *pp, const float *vin, float *vout, int batch, cudaStream_t stream) {
    TmaParams &p = *pp;
    TmaArgs &A = p.a;
    cudaError_t e;
    if (!p.dev) {
        // the record tables go to the device on the first product
        e = cudaMalloc(&p.dev, p.host.size());
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(p.dev, p.host.data(), p.host.size(), cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) {
            cudaFree(p.dev);
            p.dev = nullptr;
            return e;
        }
        A.rscan = static_cast<const unsigned char *>(p.dev);
        A.rfin = reinterpret_cast<const TmaFinRec *>(static_cast<const unsigned char *>(p.dev) +
                                                     (size_t)A.nbox * kScanBlock);
        cudaGetDevice(&p.device);
        e = cudaGetSymbolAddress(reinterpret_cast<void **>(&A.err), g_tma_err);
        if (e != cudaSuccess) return e;
    }
    A.batch = batch;
    A.nbb = (batch + 31) / 32;
    // test hook (KPS_TEST_STALL_WAIT=1): one barrier per CTA never completes,
    // so that its bounded wait gives up and sets the error flag
    const char *st = std::getenv("KPS_TEST_STALL_WAIT");
    A.stall_test = st && std::atoi(st) > 0 ? 1 : 0;
    e = encode3(&A.tin, vin, A.H, A.n_in, batch, A.hs);
    if (e == cudaSuccess) e = encode3(&A.tout, vout, A.hs, A.n_out, batch, A.hs);
    if (e != cudaSuccess) return e;
    // at least 80 KB: never more than two CTAs per SM, so that their tensor
    // memory (256 columns each) always fits
    const size_t smem = std::max<size_t>(tma_smem_bytes(A.nc, A.extra), 80 * 1024);
    const long long blocks = (long long)A.n_out * A.nbb;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    auto fn = A.k == 1 ? tma_scan_kernel<1> : tma_scan_kernel<2>;
    e = ensure_dyn_smem(reinterpret_cast<const void *>(fn), smem);
    if (e != cudaSuccess) return e;
    fn<<<(unsigned)blocks, 32 * kTmaWarps, smem, stream>>>(A);
    return cudaGetLastError();
}

}  // namespace kps
