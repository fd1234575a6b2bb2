// Inputs and outputs of the warm-start network for the games of a batch.
//
// A query is (game, player p, decision node k of p, hand h); the queries of
// a batch are enumerated game by game, then player 1's nodes, then player
// 2's, then hands in library order.  Its feature row (KPS_WARM_DIN floats):
//   [0, 52)       board one-hot (card ids)
//   [52, 1133)    1081-bin strength histogram of the opponent's range: bin
//                 floor(pos * 1081 / H) of the opponent hand at strength
//                 position pos gets mu_q(pos) / sum mu_q
//   [1133, 1173)  node: one-hot of k (first 32 nodes), player, actions / 12,
//                 depth (player-p ancestors) / 8
//   [1173, 1229)  hand: strength position / (H - 1), tie-group size / 32,
//                 mu_p(h) * H / sum mu_p, 0, two-hot of the hand's cards
//   [1229, 1232)  zero
// Targets are a solver's average behavioural strategy at (k, h) and the
// weight reach_p(parent sequence) * mu_p(h) * H / sum mu_p; predictions are
// scattered back into behavioural strategies in the batch layout.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "abi_internal.h"
#include "kernels.h"
#include "batch_internal.h"
#include "mlp_internal.h"

#include <cuda_bf16.h>

using namespace kps_abi;

namespace {

constexpr int kDin = KPS_WARM_DIN, kDout = KPS_WARM_DOUT;
// board at offset 0; node features are 40 wide
constexpr int kOffHist = 52, kOffNode = 1133, kOffHand = 1173;
constexpr int kHist = 1081, kHandF = 56;
static_assert(kOffHand + kHandF + 3 == kDin, "feature row layout");

struct WarmGame {
    int H, hs;
    long long qstart;          // first query of the game
    int nodes[2];
    int node_off[2];           // into the node arrays
    long long hist_off[2];     // into the histogram array
    long long hand_off;        // into the per-hand arrays
    long long voff[2];         // batch vector offsets
    unsigned long long board_lo; // board cards as a 64-bit mask
};

struct WarmDev {
    const WarmGame *games;
    const long long *qstart;   // [ngames + 1]
    int ngames;
    const float *hist;         // [game][player][1081]
    const int4 *node;          // {first sequence, actions, parent sequence, depth}
    const int2 *cards;         // per hand: card ids (b = -1 for one-card hands)
    const float *hand;         // per hand: {pos/(H-1), tie/32, mu1 norm, mu2 norm}
    const float *node_feat;    // per node: its 40 node features
    int total_nodes;
};

struct Query {
    int game, player, node, hand;
};

__device__ __forceinline__ Query decode(const WarmDev &d, long long q) {
    int lo = 0, hi = d.ngames - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d.qstart[mid] <= q) lo = mid; else hi = mid - 1;
    }
    const WarmGame &G = d.games[lo];
    long long r = q - G.qstart;
    Query Q;
    Q.game = lo;
    const long long n1 = (long long)G.nodes[0] * G.H;
    Q.player = r < n1 ? 0 : 1;
    if (Q.player) r -= n1;
    Q.node = (int)(r / G.H);
    Q.hand = (int)(r % G.H);
    return Q;
}

// One block per row: thread 0 decodes the query, the block writes the row.
__global__ void __launch_bounds__(256) features_kernel(const WarmDev d, const long long *qidx, long long q0,
                                                         float *X, int *nact) {
    __shared__ Query sq;
    const long long row = blockIdx.x;
    if (threadIdx.x == 0) sq = decode(d, qidx ? qidx[row] : q0 + row);
    __syncthreads();
    const Query Q = sq;
    const WarmGame &G = d.games[Q.game];
    const int4 nd = d.node[G.node_off[Q.player] + Q.node];
    const int2 cd = d.cards[G.hand_off + Q.hand];
    const float4 hf = reinterpret_cast<const float4 *>(d.hand)[G.hand_off + Q.hand];
    const float *hist = d.hist + G.hist_off[Q.player];
    float *x = X + row * kDin;
    for (int j = threadIdx.x; j < kDin; j += blockDim.x) {
        float v = 0.f;
        if (j < kOffHist) {
            v = (G.board_lo >> j) & 1ull ? 1.f : 0.f;
        } else if (j < kOffNode) {
            v = hist[j - kOffHist];
        } else if (j < kOffHand) {
            const int f = j - kOffNode;
            if (f < 32) v = f == Q.node ? 1.f : 0.f;
            else if (f == 32) v = (float)Q.player;
            else if (f == 33) v = nd.y / 12.f;
            else if (f == 34) v = nd.w / 8.f;
        } else if (j < kOffHand + kHandF) {
            const int f = j - kOffHand;
            if (f == 0) v = hf.x;
            else if (f == 1) v = hf.y;
            else if (f == 2) v = Q.player == 0 ? hf.z : hf.w;
            else if (f >= 4) v = (f - 4 == cd.x || f - 4 == cd.y) ? 1.f : 0.f;
        }
        x[j] = v;
    }
    if (threadIdx.x == 0 && nact) nact[row] = nd.y;
}

__global__ void targets_kernel(const WarmDev d, const double *beh1, const double *beh2, const double *x1,
                               const double *x2, const long long *qidx, long long q0, int nq, float *T, float *w) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= nq) return;
    const Query Q = decode(d, qidx ? qidx[row] : q0 + row);
    const WarmGame &G = d.games[Q.game];
    const int4 nd = d.node[G.node_off[Q.player] + Q.node];
    const double *beh = Q.player == 0 ? beh1 : beh2;
    const double *xs = Q.player == 0 ? x1 : x2;
    const long long base = G.voff[Q.player] + Q.hand;
    for (int a = 0; a < kDout; ++a)
        T[(long long)row * kDout + a] = a < nd.y ? (float)beh[base + (long long)(nd.x + a) * G.hs] : 0.f;
    const float4 hf = reinterpret_cast<const float4 *>(d.hand)[G.hand_off + Q.hand];
    const double reach = (xs && nd.z >= 0) ? xs[base + (long long)nd.z * G.hs] : 1.0;
    w[row] = (float)reach * (Q.player == 0 ? hf.z : hf.w);
}

__global__ void scatter_kernel(const WarmDev d, const float *P, const long long *qidx, long long q0, int nq,
                               float *beh1, float *beh2) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= nq) return;
    const Query Q = decode(d, qidx ? qidx[row] : q0 + row);
    const WarmGame &G = d.games[Q.game];
    const int4 nd = d.node[G.node_off[Q.player] + Q.node];
    float *beh = Q.player == 0 ? beh1 : beh2;
    const long long base = G.voff[Q.player] + Q.hand;
    for (int a = 0; a < nd.y; ++a) beh[base + (long long)(nd.x + a) * G.hs] = P[(long long)row * kDout + a];
}

// Game part of the feature rows, one row per (game, player): board one-hot
// and the opponent's strength histogram (feature columns [0, 1133)).
__global__ void game_part_kernel(const WarmDev d, float *Gf) {
    const int r = blockIdx.x, g = r >> 1, p = r & 1;
    const WarmGame &G = d.games[g];
    const float *hist = d.hist + G.hist_off[p];
    float *x = Gf + (long long)r * kOffNode;
    for (int j = threadIdx.x; j < kOffNode; j += blockDim.x)
        x[j] = j < kOffHist ? ((G.board_lo >> j) & 1ull ? 1.f : 0.f) : hist[j - kOffHist];
}

// ---- fused inference ---------------------------------------------------
// Layer 1 from its three parts (game and node parts precomputed, the hand
// part from five rows of W1), layers 2 and 3 on the fifth-generation tensor
// cores: tcgen05.mma (kind::f16, BF16 operands, FP32 accumulation in tensor
// memory) for a tile of 128 queries, M = 128, N = 256 (layer 2) and N = 16
// (layer 3, logits padded), K = 256 in 16 steps of 16.  Both operands are
// K-major in shared memory without swizzle, in 8-row x 16-byte core
// matrices: element (r, k) of an operand with K = 256 sits at byte
//   (r / 8) * 4096 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,
// so core matrices adjacent in K are 128 bytes apart and 8-row groups 4096
// bytes apart (the descriptors' leading and stride byte offsets).  W2 and W3
// stay resident in shared memory; the activations of layer 1 are written in
// that layout, read back from tensor memory after layer 2 (bias, ReLU,
// BF16) into the same buffer for layer 3, whose 16 logits per row go to the
// masked softmax, written straight into the behavioural strategies.  One
// thread issues the MMAs; tcgen05.commit arrives on an mbarrier that the
// others wait on (bounded: 2 s, then the error flag read by
// kps_device_status).
constexpr int kPR = 128;            // queries per tile (M)
constexpr int kWidth = 256;
constexpr int kOpRow = 4096;        // bytes between 8-row groups of an operand (K = 256)
constexpr int kTmemPred = 512;      // columns: layer 2 at 0..255, layer 3 at 256..271

struct RowInfo {
    long long base;                  // batch-vector offset of (player, hand)
    int gp, node, ca, cb, nact, s0, hs, player;
    float pos, tie, mu;
};

// Shared memory: W2 [256 rows][K] (128 KB), the activations [128][K]
// (64 KB), W3 [16][K] (8 KB), the row records, then the barrier and the
// tensor-memory slot.
constexpr size_t kOffW2 = 0, kOffH = kOffW2 + (size_t)kWidth / 8 * kOpRow, kOffW3 = kOffH + (size_t)kPR / 8 * kOpRow,
                 kOffRows = kOffW3 + 2 * (size_t)kOpRow, kOffBar = kOffRows + kPR * sizeof(RowInfo);
__host__ __device__ constexpr size_t predict_smem_bytes() { return kOffBar + 16 + 128; }
// (barrier at kOffBar, tensor-memory slot at +8, the tile's first game at +12)

__device__ __forceinline__ uint32_t op_off(int r, int k) {
    return (uint32_t)((r >> 3) * kOpRow + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
// Shared-memory matrix descriptor: start address, leading (K) and stride
// (8-row) byte offsets, the fixed version bits 46-48 = 0b001, no swizzle.
__device__ __forceinline__ uint64_t op_desc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(kOpRow >> 4) << 32) |
           (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void pmbar_init(uint32_t bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool pmbar_try(uint32_t bar, uint32_t parity) {
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
// Bounded wait (2 s of %globaltimer); false when it gave up.
__device__ __noinline__ bool pmbar_wait(uint32_t bar, uint32_t parity) {
    if (pmbar_try(bar, parity)) return true;
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (int i = 0; i < (1 << 26); ++i) {
        if (pmbar_try(bar, parity)) return true;
        if ((i & 63) == 63) {
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (t - t0 > 2000000000ull) break;
        }
    }
    return false;
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7]), "=f"(r[8]),
          "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+f"(r[0]), "+f"(r[1]), "+f"(r[2]), "+f"(r[3]), "+f"(r[4]), "+f"(r[5]), "+f"(r[6]), "+f"(r[7]),
                   "+f"(r[8]), "+f"(r[9]), "+f"(r[10]), "+f"(r[11]), "+f"(r[12]), "+f"(r[13]), "+f"(r[14]), "+f"(r[15])::"memory");
}

struct PredictArgs {
    WarmDev d;
    const float *G1;                 // [2 ngames][256]
    const float *N1;                 // [total nodes][256]
    const __nv_bfloat16 *W1h;        // rows 1173.. of W1: [59][256]
    const float *b1, *b2, *b3;
    const __nv_bfloat16 *W2;         // [256][256]
    const __nv_bfloat16 *W3;         // [256][dout]
    int dout;
    long long nq;
    float *beh1, *beh2;
    unsigned int *err;               // set when a wait gives up
};

__device__ unsigned int g_predict_err;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__global__ void __launch_bounds__(256, 1) predict_kernel(const PredictArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *W2s = smem_raw + kOffW2, *Hs = smem_raw + kOffH, *W3s = smem_raw + kOffW3;
    RowInfo *rows = reinterpret_cast<RowInfo *>(smem_raw + kOffRows);
    const uint32_t bar = smem_addr(smem_raw + kOffBar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem_raw + kOffBar + 8);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // W2 and W3 as B operands: row n of B is output column n, K contiguous
    for (int i = tid; i < kWidth * kWidth; i += blockDim.x) {
        const int k = i / kWidth, n = i % kWidth;
        *reinterpret_cast<__nv_bfloat16 *>(W2s + op_off(n, k)) = a.W2[i];
    }
    for (int i = tid; i < kWidth * 16; i += blockDim.x) {
        const int k = i / 16, n = i % 16;
        *reinterpret_cast<__nv_bfloat16 *>(W3s + op_off(n, k)) =
            n < a.dout ? a.W3[k * a.dout + n] : __float2bfloat16_rn(0.f);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                     "r"(kTmemPred));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) pmbar_init(bar);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t tlane = (uint32_t)(32 * (warp & 3)) << 16;   // this warp's tensor-memory lanes
    // this thread's column of the hand part of layer 1
    const int j = tid;
    const float wpos = __bfloat162float(a.W1h[0 * kWidth + j]), wtie = __bfloat162float(a.W1h[1 * kWidth + j]),
                wmu = __bfloat162float(a.W1h[2 * kWidth + j]), bias1 = a.b1[j];
    const __nv_bfloat16 *Wc = a.W1h + 4 * kWidth;
    uint32_t phase = 0;
    bool ok = true;
    const long long ntiles = (a.nq + kPR - 1) / kPR;
    int *tile_game = reinterpret_cast<int *>(smem_raw + kOffBar + 12);
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        // the tile's queries are consecutive: one search for the game of its
        // first query, then every row steps forward from it
        if (tid == 0) *tile_game = decode(a.d, tile * kPR).game;
        __syncthreads();
        if (tid < kPR) {
            const long long q = tile * kPR + tid;
            RowInfo ri;
            ri.nact = 0;
            if (q < a.nq) {
                int gq = *tile_game;
                while (a.d.qstart[gq + 1] <= q) ++gq;
                const WarmGame &GQ = a.d.games[gq];
                Query Q;
                Q.game = gq;
                int r = (int)(q - GQ.qstart);
                const int n1 = GQ.nodes[0] * GQ.H;
                Q.player = r < n1 ? 0 : 1;
                if (Q.player) r -= n1;
                Q.node = r / GQ.H;
                Q.hand = r - Q.node * GQ.H;
                const WarmGame &G = a.d.games[Q.game];
                const int4 nd = a.d.node[G.node_off[Q.player] + Q.node];
                const int2 cd = a.d.cards[G.hand_off + Q.hand];
                const float4 hf = reinterpret_cast<const float4 *>(a.d.hand)[G.hand_off + Q.hand];
                ri.base = G.voff[Q.player] + Q.hand;
                ri.gp = 2 * Q.game + Q.player;
                ri.node = G.node_off[Q.player] + Q.node;
                ri.ca = cd.x;
                ri.cb = cd.y;
                ri.nact = nd.y;
                ri.s0 = nd.x;
                ri.hs = G.hs;
                ri.player = Q.player;
                ri.pos = hf.x;
                ri.tie = hf.y;
                ri.mu = Q.player == 0 ? hf.z : hf.w;
            }
            rows[tid] = ri;
        }
        __syncthreads();
        // layer 1: column j of every row, written as BF16 in the A layout.
        // Eight rows at a time: their records and all their gathers are
        // issued before any sum or store, so the loads overlap (the sum order
        // is the definition's: game part, node part, hand features, cards).
        for (int r0 = 0; r0 < kPR; r0 += 8) {
            float g[8], nd[8], wa[8], wb[8], pos[8], tie[8], mu[8];
            bool live[8], two[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const RowInfo &ri = rows[r0 + u];
                live[u] = ri.nact > 0;
                two[u] = ri.cb >= 0;
                const int gp = live[u] ? ri.gp : 0, node = live[u] ? ri.node : 0;
                const int ca = live[u] ? ri.ca : 0, cb = live[u] && two[u] ? ri.cb : 0;
                g[u] = a.G1[(long long)gp * kWidth + j];
                nd[u] = a.N1[(long long)node * kWidth + j];
                wa[u] = __bfloat162float(Wc[ca * kWidth + j]);
                wb[u] = __bfloat162float(Wc[cb * kWidth + j]);
                pos[u] = ri.pos;
                tie[u] = ri.tie;
                mu[u] = ri.mu;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                float z = 0.f;
                if (live[u]) {
                    z = g[u] + nd[u] + pos[u] * wpos + tie[u] * wtie + mu[u] * wmu + wa[u] + bias1;
                    if (two[u]) z += wb[u];
                    z = fmaxf(z, 0.f);
                }
                *reinterpret_cast<__nv_bfloat16 *>(Hs + op_off(r0 + u, j)) = __float2bfloat16_rn(z);
            }
        }
        // the activations (generic writes) before the tensor cores read them;
        // the previous tile's tensor-memory loads before this tile's MMAs
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // layer 2: D[0..255] = H (128 x 256) x W2 (256 x 256)
        if (tid == 0) {
            const uint32_t ha = smem_addr(Hs), wa = smem_addr(W2s);
            for (int s = 0; s < kWidth / 16; ++s)
                mma_f16(tbase, op_desc(ha + 256u * s), op_desc(wa + 256u * s), mma_idesc(kPR, kWidth), s > 0);
            mma_commit(bar);
        }
        if (ok) ok = pmbar_wait(bar, phase);
        phase ^= 1u;
        if (!__syncthreads_and(ok)) break;
        tc_fence_after();
        // bias, ReLU, BF16, back into the A layout: warp w has rows 32 (w & 3)
        // .. + 31 and columns 128 (w >> 2) .. + 127
        {
            const int r = 32 * (warp & 3) + lane, c0 = 128 * (warp >> 2);
#pragma unroll 1
            for (int cb = 0; cb < 8; ++cb) {
                const int c = c0 + 16 * cb;
                float v[16];
                tc_ld16(tbase + tlane + (uint32_t)c, v);
                uint32_t w[8];
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    w[i] = pack_bf16(fmaxf(v[2 * i] + a.b2[c + 2 * i], 0.f), fmaxf(v[2 * i + 1] + a.b2[c + 2 * i + 1], 0.f));
                *reinterpret_cast<uint4 *>(Hs + op_off(r, c)) = make_uint4(w[0], w[1], w[2], w[3]);
                *reinterpret_cast<uint4 *>(Hs + op_off(r, c + 8)) = make_uint4(w[4], w[5], w[6], w[7]);
            }
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // layer 3: D[256..271] = H2 (128 x 256) x W3 (256 x 16)
        if (tid == 0) {
            const uint32_t ha = smem_addr(Hs), wa = smem_addr(W3s);
            for (int s = 0; s < kWidth / 16; ++s)
                mma_f16(tbase + 256u, op_desc(ha + 256u * s), op_desc(wa + 256u * s), mma_idesc(kPR, 16), s > 0);
            mma_commit(bar);
        }
        if (ok) ok = pmbar_wait(bar, phase);
        phase ^= 1u;
        if (!__syncthreads_and(ok)) break;
        tc_fence_after();
        // masked softmax of row 32 w + lane over its first nact logits
        if (warp < 4) {
            const int r = 32 * warp + lane;
            float z[16];
            tc_ld16(tbase + tlane + 256u, z);
            const RowInfo &ri = rows[r];
            if (ri.nact > 0) {
                float mx = -INFINITY;
#pragma unroll
                for (int n = 0; n < 16; ++n) {
                    z[n] += n < a.dout ? a.b3[n] : 0.f;
                    if (n < ri.nact) mx = fmaxf(mx, z[n]);
                }
                float e[16], s = 0.f;
#pragma unroll
                for (int n = 0; n < 16; ++n) {
                    e[n] = n < ri.nact ? __expf(z[n] - mx) : 0.f;
                    s += e[n];
                }
                float *beh = ri.player == 0 ? a.beh1 : a.beh2;
#pragma unroll
                for (int n = 0; n < 16; ++n)
                    if (n < ri.nact) beh[ri.base + (long long)(ri.s0 + n) * ri.hs] = e[n] / s;
            }
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    if (!ok && tid == 0) atomicExch(a.err, 1u);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kTmemPred));
}
}  // namespace

// Device tables of a batch's warm-start features (built on first use).
struct WarmTables {
    void *blob = nullptr;
    WarmDev d{};
    long long nq = 0;
};

namespace kps_abi {

cudaError_t predict_take_error(bool *set) {
    unsigned int v = 0, zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_predict_err, sizeof(v));
    if (e == cudaSuccess && v) e = cudaMemcpyToSymbol(g_predict_err, &zero, sizeof(zero));
    *set = v != 0;
    return e;
}

void warm_free(kps_batch *b) {
    if (b->warm) {
        cudaFree(static_cast<WarmTables *>(b->warm)->blob);
        delete static_cast<WarmTables *>(b->warm);
        b->warm = nullptr;
    }
}

}  // namespace kps_abi

namespace {

kps_status warm_tables(kps_batch *b, const WarmTables **out) {
    if (b->warm) {
        *out = static_cast<WarmTables *>(b->warm);
        return KPS_OK;
    }
    const int ng = (int)b->games.size();
    std::vector<WarmGame> games(ng);
    std::vector<long long> qstart(ng + 1, 0);
    std::vector<float> hist, hand, node_feat;
    std::vector<int4> node;
    std::vector<int2> cards;
    for (int i = 0; i < ng; ++i) {
        const kps::HostGame &h = b->games[i]->host;
        if (h.nodes[0] > 32 || h.nodes[1] > 32) return fail(KPS_ENOTSUP, "more than 32 decision nodes per player");
        WarmGame &G = games[i];
        G.H = h.H;
        G.hs = h.hs;
        G.qstart = qstart[i];
        qstart[i + 1] = qstart[i] + (long long)(h.nodes[0] + h.nodes[1]) * h.H;
        G.hand_off = (long long)cards.size();
        unsigned long long left = 0;
        for (int c : h.slot_card) left |= 1ull << c;
        const int deck = h.spec.ranks * h.spec.suits;
        const unsigned long long all = deck >= 64 ? ~0ull : ((1ull << deck) - 1);
        G.board_lo = all & ~left;
        double msum[2] = {0.0, 0.0};
        for (int q = 0; q < h.H; ++q) {
            msum[0] += h.mu1[q];
            msum[1] += h.mu2[q];
        }
        for (int p = 0; p < 2; ++p) {
            G.voff[p] = b->off[p][i];
            G.nodes[p] = h.nodes[p];
            G.node_off[p] = (int)node.size();
            G.hist_off[p] = (long long)hist.size();
            // the opponent's range over the strength order
            const std::vector<double> &mq = p == 0 ? h.mu2 : h.mu1;
            std::vector<float> hb(kHist, 0.f);
            for (int q = 0; q < h.H; ++q) {
                const int bin = (int)((long long)q * kHist / h.H);
                hb[bin] += msum[1 - p] > 0.0 ? (float)(mq[q] / msum[1 - p]) : 0.f;
            }
            hist.insert(hist.end(), hb.begin(), hb.end());
            std::vector<int> first(h.nodes[p], -1);
            for (int q = 0; q < h.n[p]; ++q)
                if (first[h.seqs[p][q].node] < 0) first[h.seqs[p][q].node] = q;
            std::vector<int> depth(h.nodes[p], 0);
            for (int k = 0; k < h.nodes[p]; ++k) {
                const int par = h.seqs[p][first[k]].parent;
                depth[k] = par < 0 ? 0 : depth[h.seqs[p][par].node] + 1;
                node.push_back(make_int4(first[k], h.nodes_nact[p][k], par, depth[k]));
                float nf[40] = {};
                nf[k] = 1.f;
                nf[32] = (float)p;
                nf[33] = h.nodes_nact[p][k] / 12.f;
                nf[34] = depth[k] / 8.f;
                node_feat.insert(node_feat.end(), nf, nf + 40);
            }
        }
        for (int q = 0; q < h.H; ++q) {
            const int a = h.slot_card[h.hand_slots[2 * q]];
            const int s2 = h.hand_slots[2 * q + 1];
            const int c2 = s2 < h.ncards ? h.slot_card[s2] : -1;
            cards.push_back(make_int2(a, c2));
            hand.push_back(h.H > 1 ? (float)q / (float)(h.H - 1) : 0.f);
            hand.push_back((float)(h.group_hi[q] - h.group_lo[q] + 1) / 32.f);
            hand.push_back(msum[0] > 0.0 ? (float)(h.mu1[q] * h.H / msum[0]) : 0.f);
            hand.push_back(msum[1] > 0.0 ? (float)(h.mu2[q] * h.H / msum[1]) : 0.f);
        }
    }
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t o_g = 0, o_q = al(sizeof(WarmGame) * ng), o_h = al(o_q + 8 * (size_t)(ng + 1)),
                 o_n = al(o_h + 4 * hist.size()), o_c = al(o_n + sizeof(int4) * node.size()),
                 o_f = al(o_c + sizeof(int2) * cards.size()), o_nf = al(o_f + 4 * hand.size()),
                 total = al(o_nf + 4 * node_feat.size());
    std::vector<unsigned char> host(total, 0);
    std::memcpy(host.data() + o_g, games.data(), sizeof(WarmGame) * ng);
    std::memcpy(host.data() + o_q, qstart.data(), 8 * (size_t)(ng + 1));
    std::memcpy(host.data() + o_h, hist.data(), 4 * hist.size());
    std::memcpy(host.data() + o_n, node.data(), sizeof(int4) * node.size());
    std::memcpy(host.data() + o_c, cards.data(), sizeof(int2) * cards.size());
    std::memcpy(host.data() + o_f, hand.data(), 4 * hand.size());
    std::memcpy(host.data() + o_nf, node_feat.data(), 4 * node_feat.size());
    WarmTables *t = new (std::nothrow) WarmTables;
    if (!t) return fail(KPS_ENOMEM, "warm-start tables");
    if (cudaMalloc(&t->blob, total) != cudaSuccess) {
        delete t;
        return fail(KPS_ENOMEM, "warm-start tables");
    }
    cudaError_t e = cudaMemcpy(t->blob, host.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(t->blob);
        delete t;
        return cuda_fail(e, "uploading warm-start tables");
    }
    unsigned char *bl = static_cast<unsigned char *>(t->blob);
    t->d.games = reinterpret_cast<const WarmGame *>(bl + o_g);
    t->d.qstart = reinterpret_cast<const long long *>(bl + o_q);
    t->d.ngames = ng;
    t->d.hist = reinterpret_cast<const float *>(bl + o_h);
    t->d.node = reinterpret_cast<const int4 *>(bl + o_n);
    t->d.cards = reinterpret_cast<const int2 *>(bl + o_c);
    t->d.hand = reinterpret_cast<const float *>(bl + o_f);
    t->d.node_feat = reinterpret_cast<const float *>(bl + o_nf);
    t->d.total_nodes = (int)node.size();
    t->nq = qstart[ng];
    b->warm = t;
    *out = t;
    return KPS_OK;
}

kps_status check_range(const WarmTables *t, const int64_t *qidx, int64_t q0, int32_t nq) {
    if (nq < 0) return fail(KPS_EINVAL, "nq must be >= 0");
    if (!qidx && (q0 < 0 || q0 + nq > t->nq)) return fail(KPS_EINVAL, "query range outside the batch");
    return KPS_OK;
}

}  // namespace

extern "C" {

kps_status kps_warm_num_queries(kps_batch *b, int64_t *n) {
    if (!b || !n) return fail(KPS_EINVAL, "bad argument");
    const WarmTables *t = nullptr;
    kps_status st = warm_tables(b, &t);
    if (st != KPS_OK) return st;
    *n = t->nq;
    return KPS_OK;
}

kps_status kps_warm_features(kps_batch *b, const int64_t *qidx, int64_t q0, int32_t nq, float *X, int32_t *nact,
                             void *stream) {
    if (!b || (nq > 0 && !X)) return fail(KPS_EINVAL, "bad argument");
    const WarmTables *t = nullptr;
    kps_status st = warm_tables(b, &t);
    if (st == KPS_OK) st = check_range(t, qidx, q0, nq);
    if (st != KPS_OK || nq == 0) return st;
    features_kernel<<<nq, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        t->d, reinterpret_cast<const long long *>(qidx), q0, X, nact);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "warm-start features");
    return KPS_OK;
}

kps_status kps_warm_targets(kps_batch *b, const double *beh1, const double *beh2, const double *x1, const double *x2,
                            const int64_t *qidx, int64_t q0, int32_t nq, float *T, float *w, void *stream) {
    if (!b || (nq > 0 && (!beh1 || !beh2 || !T || !w))) return fail(KPS_EINVAL, "bad argument");
    const WarmTables *t = nullptr;
    kps_status st = warm_tables(b, &t);
    if (st == KPS_OK) st = check_range(t, qidx, q0, nq);
    if (st != KPS_OK || nq == 0) return st;
    targets_kernel<<<(nq + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(
        t->d, beh1, beh2, x1, x2, reinterpret_cast<const long long *>(qidx), q0, nq, T, w);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "warm-start targets");
    return KPS_OK;
}

kps_status kps_warm_scatter(kps_batch *b, const float *P, const int64_t *qidx, int64_t q0, int32_t nq, float *beh1,
                            float *beh2, void *stream) {
    if (!b || (nq > 0 && (!P || !beh1 || !beh2))) return fail(KPS_EINVAL, "bad argument");
    const WarmTables *t = nullptr;
    kps_status st = warm_tables(b, &t);
    if (st == KPS_OK) st = check_range(t, qidx, q0, nq);
    if (st != KPS_OK || nq == 0) return st;
    scatter_kernel<<<(nq + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(
        t->d, P, reinterpret_cast<const long long *>(qidx), q0, nq, beh1, beh2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "warm-start scatter");
    return KPS_OK;
}

kps_status kps_warm_predict(kps_batch *b, kps_mlp *m, float *beh1, float *beh2, void *stream) {
    if (!b || !m || !beh1 || !beh2) return fail(KPS_EINVAL, "bad argument");
    if (m->din != kDin || m->width != kWidth || m->dout > 16)
        return fail(KPS_ENOTSUP, "the fused predictor needs din = KPS_WARM_DIN, width 256, dout <= 16");
    const WarmTables *t = nullptr;
    kps_status st = warm_tables(b, &t);
    if (st != KPS_OK) return st;
    if (t->nq == 0) return KPS_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int ng = t->d.ngames, nn = t->d.total_nodes;
    float *Gf = nullptr, *G1 = nullptr, *N1 = nullptr;
    cudaError_t e = cudaMalloc(&Gf, (size_t)2 * ng * kOffNode * 4);
    if (e == cudaSuccess) e = cudaMalloc(&G1, (size_t)2 * ng * kWidth * 4);
    if (e == cudaSuccess) e = cudaMalloc(&N1, (size_t)std::max(nn, 1) * kWidth * 4);
    if (e != cudaSuccess) {
        cudaFree(Gf);
        cudaFree(G1);
        return fail(KPS_ENOMEM, "predictor tables");
    }
    const __nv_bfloat16 *W1 = m->ph + m->off[0];
    game_part_kernel<<<2 * ng, 256, 0, s>>>(t->d, Gf);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = mlp_gemm_xw(2 * ng, kWidth, kOffNode, Gf, kOffNode, W1, kWidth, G1, kWidth, s);
    if (e == cudaSuccess)
        e = mlp_gemm_xw(nn, kWidth, kOffHand - kOffNode, t->d.node_feat, kOffHand - kOffNode,
                        W1 + (size_t)kOffNode * kWidth, kWidth, N1, kWidth, s);
    if (e == cudaSuccess) {
        e = kps::ensure_dyn_smem(reinterpret_cast<const void *>(predict_kernel), predict_smem_bytes());
    }
    if (e == cudaSuccess) {
        PredictArgs a;
        a.d = t->d;
        a.G1 = G1;
        a.N1 = N1;
        a.W1h = W1 + (size_t)kOffHand * kWidth;
        a.b1 = m->p + m->off[1];
        a.b2 = m->p + m->off[3];
        a.b3 = m->p + m->off[5];
        a.W2 = m->ph + m->off[2];
        a.W3 = m->ph + m->off[4];
        a.dout = m->dout;
        a.nq = t->nq;
        a.beh1 = beh1;
        a.beh2 = beh2;
        e = cudaGetSymbolAddress(reinterpret_cast<void **>(&a.err), g_predict_err);
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const long long ntiles = (t->nq + kPR - 1) / kPR;
        const int grid = (int)std::min<long long>(ntiles, sms);
        if (e == cudaSuccess) {
            predict_kernel<<<grid, 256, predict_smem_bytes(), s>>>(a);
            e = cudaGetLastError();
        }
    }
    // the temporaries are released after the work that reads them
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(Gf);
    cudaFree(G1);
    cudaFree(N1);
    if (e != cudaSuccess) return cuda_fail(e, "warm-start prediction");
    return KPS_OK;
}

}  // extern "C"
