// First-order equilibrium solver on a batch of games (C ABI in include/kps.h).
//
// Every iteration of a first-order method needs the gradients A y and
// -A^T x (Sec. 2, "First-order methods"); everything else is local to one
// hand of one player.  The solver is regret matching plus (RM+) with
// alternating updates and linearly weighted averages:
//   t <- t + 1
//   player 1: xsum += t x;  g = A y;  bottom-up over player 1's decision
//     nodes (children first): q(I,a) = g[sigma(I,a)] + sum of the values of
//     player 1's next decisions under (I,a), v(I) = sum_a b(I,a) q(I,a),
//     R(I,a) <- max(0, R(I,a) + q(I,a) - v(I));  b <- R / sum_a R
//     (uniform when the sum is at most the noise floor theta_p);
//     x <- sequence form of b (x[sigma(I,a)] = x[parent(I)] b(I,a));
//   player 2: the same against the new x with g = -A^T x.
// The noise floor: a value that is exactly zero (the opponent's compatible
// hands all have zero reach while hands sharing a card do not) leaves the
// product, which subtracts card-overlap masses, as rounding noise, and
// regret matching would follow the noise.  theta_p = eps * V_p with V_p =
// max |payoff| * max_h mu_p(h) * sum_h mu_q(h) / beta, a bound on p's
// counterfactual values, and eps = 2^-40 (FP64) or 2^-16 (FP32 arithmetic)
// treats regret sums at the noise level as zero.
// The exploitability of the averages xbar = xsum / sum t, ybar (FP64) is
// (BR1(ybar) + BR2(xbar)) / 2 / pot0, the best responses taking the max
// over actions in the same bottom-up walk (Sec. 5 measures average
// exploitability in units of the initial pot).
//
// One thread owns one hand of one game: regrets, values and strategies of
// a player are [sequence][hand] rows of that game, so a warp's loads and
// stores of one sequence are coalesced.  Per-thread running values (child
// values bottom-up, then new sequence-form entries top-down) live in shared
// memory, [sequence][thread].  Strategies and values are stored in the
// solver's storage type (FP32, FP64, BF16 or FP16); regrets, averages and
// all arithmetic are FP32 (FP64 for FP64 storage); the exploitability path
// is FP64 throughout.  The iteration count lives on the device so that a
// captured CUDA graph of k iterations can be replayed.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "abi_internal.h"
#include "batch_internal.h"
#include "kernels.h"

using namespace kps_abi;

namespace {

constexpr int kThreads = 64;     // hands per block (32 for trees whose sequences need more shared memory)
constexpr int kMaxActions = 12;  // fold, check/call, up to 8 bets, all-in

struct SolverGame {
    int H, hs;
    int n[2];
    int node_off[2], nnodes[2];
    long long off[2];
    int block0;       // first block of the game
    double pot0;
    double V[2];      // bound on each player's counterfactual values
    double theta[2];  // regret-matching noise floor of each player
};

template <typename S> struct Cv;
template <> struct Cv<float> {
    __device__ static float ld(const float *p) { return *p; }
    __device__ static float st(float x) { return x; }
};
template <> struct Cv<double> {
    __device__ static double ld(const double *p) { return *p; }
    __device__ static double st(double x) { return x; }
};
template <> struct Cv<__nv_bfloat16> {
    __device__ static float ld(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    __device__ static __nv_bfloat16 st(float x) { return __float2bfloat16_rn(x); }
};
template <> struct Cv<__half> {
    __device__ static float ld(const __half *p) { return __half2float(*p); }
    __device__ static __half st(float x) { return __float2half_rn(x); }
};

struct Where {
    int game, h;
};

template <int BW>
__device__ __forceinline__ Where locate(const SolverGame *games, const int *block_game) {
    Where w;
    w.game = block_game[blockIdx.x];
    w.h = (blockIdx.x - games[w.game].block0) * BW + threadIdx.x;
    return w;
}

// Regret matching of one node: b[a] = R+[a] / sum, uniform if the sum is
// at most the noise floor theta.
template <typename C>
__device__ __forceinline__ void regret_match(const C *r, int na, C *b, C theta) {
    // positive parts (RM+ regrets are never negative; DCFR's may be)
    C sum = C(0);
#pragma unroll
    for (int a = 0; a < kMaxActions; ++a)
        if (a < na) sum += r[a] > C(0) ? r[a] : C(0);
#pragma unroll
    for (int a = 0; a < kMaxActions; ++a)
        if (a < na) b[a] = sum > theta ? (r[a] > C(0) ? r[a] : C(0)) / sum : C(1) / C(na);
}

// Weight of iteration t in the average: t (RM+) or t^gamma (DCFR, from the
// host-computed table).
__device__ __forceinline__ double avg_weight(long long t, int method, const double *dtab) {
    return method == 0 ? (double)t : dtab[3 * t + 2];
}

template <typename S, typename C>
struct UpdateArgs {
    const SolverGame *games;
    const int *block_game;
    const int4 *nodes;       // {first sequence, actions, parent sequence, 0}
    int player;
    C sign;                  // +1: g = A y; -1: g = A^T x (the value is -g)
    const S *g;              // values, player layout
    C *regret;
    S *x;                    // sequence-form strategy (read: played; write: next)
    C *xsum;                 // sum over iterations of t * x
    const float *beh0;       // initial behavioural strategy
    const long long *iter;   // completed iterations
    const long long *init_iter;  // the iteration that plays beh0 (0 = none)
    const double *wsum;      // sum of the average weights so far
    C kappa;                 // warm start: regrets kappa * V_p * beh0
    C w0;                    // warm start: weight of the initial strategy in the average
    int method;              // 0 RM+, 1 DCFR
    const double *dtab;      // DCFR: per iteration t, {t^a/(t^a+1), t^b/(t^b+1), t^g} at 3t
    int nmax;                // largest sequence count (shared-memory rows)
};

// One node of the bottom-up walk with NA actions (exactly unrolled; NA = 0:
// the node's own count na, up to kMaxActions, predicated): regrets updated
// from the action values, the node's value added into its parent's slot.
template <int NA, typename C, int BW>
__device__ __forceinline__ void up_node(C *qv, C *rg, int s0, int na, int par, bool init, const float *beh0,
                                        long long hs, C theta, int method, C dpos, C dneg) {
    constexpr int M = NA > 0 ? NA : kMaxActions;
    if (NA > 0) na = NA;
    C r[M], b[M], q[M];
#pragma unroll
    for (int a = 0; a < M; ++a)
        if (a < na) {
            r[a] = rg[(s0 + a) * BW];
            q[a] = qv[(s0 + a) * BW];
        }
    if (init) {
#pragma unroll
        for (int a = 0; a < M; ++a)
            if (a < na) b[a] = C(beh0[(long long)(s0 + a) * hs]);
    } else {
        C sum = C(0);
#pragma unroll
        for (int a = 0; a < M; ++a)
            if (a < na) sum += r[a] > C(0) ? r[a] : C(0);
#pragma unroll
        for (int a = 0; a < M; ++a)
            if (a < na) b[a] = sum > theta ? (r[a] > C(0) ? r[a] : C(0)) / sum : C(1) / C(na);
    }
    C v = C(0);
#pragma unroll
    for (int a = 0; a < M; ++a)
        if (a < na) v += b[a] * q[a];
#pragma unroll
    for (int a = 0; a < M; ++a)
        if (a < na) {
            const C rn = r[a] + q[a] - v;
            rg[(s0 + a) * BW] = method == 0 ? (rn > C(0) ? rn : C(0)) : rn * (rn > C(0) ? dpos : dneg);
        }
    if (par >= 0) qv[par * BW] += v;
}

// One node of the top-down walk: the next behavioural strategy by regret
// matching and its sequence form from the parent's.
template <int NA, typename C, int BW>
__device__ __forceinline__ void down_node(C *qv, const C *rg, int s0, int na, int par, C theta) {
    constexpr int M = NA > 0 ? NA : kMaxActions;
    if (NA > 0) na = NA;
    C r[M], b[M];
#pragma unroll
    for (int a = 0; a < M; ++a)
        if (a < na) r[a] = rg[(s0 + a) * BW];
    C sum = C(0);
#pragma unroll
    for (int a = 0; a < M; ++a)
        if (a < na) sum += r[a] > C(0) ? r[a] : C(0);
#pragma unroll
    for (int a = 0; a < M; ++a)
        if (a < na) b[a] = sum > theta ? (r[a] > C(0) ? r[a] : C(0)) / sum : C(1) / C(na);
    const C xpar = par >= 0 ? qv[par * BW] : C(1);
#pragma unroll
    for (int a = 0; a < M; ++a)
        if (a < na) qv[(s0 + a) * BW] = xpar * b[a];
}

// One half-iteration of one player (see the file comment).  Everything the
// thread reads is loaded first, with independent loads, into shared memory
// ([sequence][thread]: values, then regrets); the bottom-up and top-down
// walks run in shared memory (child values are added into the parent's
// value slot, which the walk reads after all children; the slots then take
// the new sequence form), and regrets and strategy are written back last.
// At least 10 resident 64-thread blocks per SM for 16- and 32-bit
// accumulators (the kernel is latency bound); FP64 keeps its registers.
template <typename S, typename C, int BW>
__global__ void __launch_bounds__(BW, sizeof(C) == 8 ? 1 : 640 / BW) rm_update_kernel(const UpdateArgs<S, C> u) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Where w = locate<BW>(u.games, u.block_game);
    const SolverGame &G = u.games[w.game];
    if (w.h >= G.H) return;
    const int p = u.player, n = G.n[p], hs = G.hs;
    C *qv = reinterpret_cast<C *>(smem_raw) + threadIdx.x;      // [s * BW]
    C *rg = qv + (size_t)u.nmax * BW;
    const long long base = G.off[p] + w.h;
    const S *__restrict__ gp = u.g + base;
    C *__restrict__ Rp = u.regret + base;
    S *__restrict__ xp = u.x + base;
    C *__restrict__ xsp = u.xsum + base;
    const long long t = *u.iter + 1;
    const bool init = t == *u.init_iter;
    const C wt = C(avg_weight(t, u.method, u.dtab));
    // DCFR: positive cumulative regrets times t^a / (t^a + 1), others t^b / (t^b + 1)
    C dpos = C(1), dneg = C(0);
    if (u.method == 1) {
        dpos = C(u.dtab[3 * t]);
        dneg = C(u.dtab[3 * t + 1]);
    }
    const int4 *nodes = u.nodes + G.node_off[p];
    const int nn = G.nnodes[p];
    const C theta = C(G.theta[p]);
    // values, regrets, and the strategy played added to the average
#pragma unroll 4
    for (int s = 0; s < n; ++s) {
        const long long i = (long long)s * hs;
        qv[s * BW] = u.sign * C(Cv<S>::ld(gp + i));
        rg[s * BW] = Rp[i];
        xsp[i] += wt * C(Cv<S>::ld(xp + i));
    }
    // bottom-up: values and regrets; top-down: next strategy (a node's
    // action count picks an exactly unrolled step; the branch is uniform
    // over the block, whose threads are hands of one game)
    const float *beh0 = u.beh0 ? u.beh0 + base : nullptr;
    for (int k = nn - 1; k >= 0; --k) {
        const int4 nd = nodes[k];
        const int s0 = nd.x, na = nd.y, par = nd.z;
        switch (na) {
            case 2: up_node<2, C, BW>(qv, rg, s0, na, par, init, beh0, hs, theta, u.method, dpos, dneg); break;
            case 3: up_node<3, C, BW>(qv, rg, s0, na, par, init, beh0, hs, theta, u.method, dpos, dneg); break;
            case 4: up_node<4, C, BW>(qv, rg, s0, na, par, init, beh0, hs, theta, u.method, dpos, dneg); break;
            case 5: up_node<5, C, BW>(qv, rg, s0, na, par, init, beh0, hs, theta, u.method, dpos, dneg); break;
            case 6: up_node<6, C, BW>(qv, rg, s0, na, par, init, beh0, hs, theta, u.method, dpos, dneg); break;
            default: up_node<0, C, BW>(qv, rg, s0, na, par, init, beh0, hs, theta, u.method, dpos, dneg); break;
        }
    }
    for (int k = 0; k < nn; ++k) {
        const int4 nd = nodes[k];
        const int s0 = nd.x, na = nd.y, par = nd.z;
        switch (na) {
            case 2: down_node<2, C, BW>(qv, rg, s0, na, par, theta); break;
            case 3: down_node<3, C, BW>(qv, rg, s0, na, par, theta); break;
            case 4: down_node<4, C, BW>(qv, rg, s0, na, par, theta); break;
            case 5: down_node<5, C, BW>(qv, rg, s0, na, par, theta); break;
            case 6: down_node<6, C, BW>(qv, rg, s0, na, par, theta); break;
            default: down_node<0, C, BW>(qv, rg, s0, na, par, theta); break;
        }
    }
    // regrets and strategy back
#pragma unroll 4
    for (int s = 0; s < n; ++s) {
        const long long i = (long long)s * hs;
        Rp[i] = rg[s * BW];
        xp[i] = Cv<S>::st(qv[s * BW]);
    }
}

// Start of a run: x <- sequence form of the initial behavioural strategy
// beh0 (uniform if none); with a warm start also R <- kappa V_p beh0 (so that
// regret matching returns beh0) and xsum <- w0 x.
template <typename S, typename C, int BW>
__global__ void __launch_bounds__(BW) seqform_kernel(const UpdateArgs<S, C> u, int has_beh) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const Where w = locate<BW>(u.games, u.block_game);
    const SolverGame &G = u.games[w.game];
    if (w.h >= G.H) return;
    const int p = u.player, hs = G.hs, tid = threadIdx.x;
    const long long base = G.off[p] + w.h;
    const int4 *nodes = u.nodes + G.node_off[p];
    const C rscale = u.kappa * C(G.V[p]);
    for (int k = 0; k < G.nnodes[p]; ++k) {
        const int4 nd = nodes[k];
        const int s0 = nd.x, na = nd.y, par = nd.z;
        const C xp = par >= 0 ? buf[par * BW + tid] : C(1);
        for (int a = 0; a < na; ++a) {
            const long long i = base + (long long)(s0 + a) * hs;
            const C b = has_beh ? C(u.beh0[i]) : C(1) / C(na);
            buf[(s0 + a) * BW + tid] = xp * b;
            u.x[i] = Cv<S>::st(xp * b);
            u.regret[i] = rscale * b;
            u.xsum[i] = u.w0 * C(Cv<S>::ld(u.x + i));
        }
    }
}

__global__ void bump_kernel(long long *iter, double *wsum, int method, const double *dtab) {
    const long long t = *iter + 1;
    *wsum += avg_weight(t, method, dtab);
    *iter = t;
}

// FP64 averages: sequence form xsum / sum_t t (the current strategy before
// any iteration), or behavioural (x[sigma] / x[parent], uniform where the
// parent is never reached).
template <typename S, typename C, typename O, int BW>
__global__ void __launch_bounds__(BW) average_kernel(const UpdateArgs<S, C> u, O *out, int behavioural) {
    const Where w = locate<BW>(u.games, u.block_game);
    const SolverGame &G = u.games[w.game];
    if (w.h >= G.H) return;
    const int p = u.player, hs = G.hs;
    const long long base = G.off[p] + w.h;
    const double wsum = *u.wsum;
    auto avg = [&](int s) -> double {
        const long long i = base + (long long)s * hs;
        return wsum > 0.0 ? (double)u.xsum[i] / wsum : (double)Cv<S>::ld(u.x + i);
    };
    const int4 *nodes = u.nodes + G.node_off[p];
    for (int k = 0; k < G.nnodes[p]; ++k) {
        const int4 nd = nodes[k];
        const int s0 = nd.x, na = nd.y, par = nd.z;
        const double xp = par >= 0 ? avg(par) : 1.0;
        for (int a = 0; a < na; ++a) {
            const double xa = avg(s0 + a);
            double v = xa;
            if (behavioural) v = xp > 0.0 ? xa / xp : 1.0 / na;
            out[base + (long long)(s0 + a) * hs] = O(v);
        }
    }
}

struct BrArgs {
    const SolverGame *games;
    const int *block_game;
    const int4 *nodes;
    int player;
    double sign;
    const void *g;      // values (FP64, or FP32 for the estimate), player layout
    double *partial;    // [blocks]
};

// Best response value of every hand: bottom-up max over the player's
// actions on the values loaded into shared memory ([sequence][thread]; a
// child's value is added into its parent's slot, read after all children);
// the sum over the block's hands goes to partial[block].
template <typename V, int BW>
__global__ void __launch_bounds__(BW) best_response_kernel(const BrArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[BW];
    const Where w = locate<BW>(a.games, a.block_game);
    const SolverGame &G = a.games[w.game];
    double root = 0.0;
    if (w.h < G.H) {
        const int p = a.player, hs = G.hs, n = G.n[p];
        const V *__restrict__ gp = static_cast<const V *>(a.g) + G.off[p] + w.h;
        double *qv = reinterpret_cast<double *>(smem_raw) + threadIdx.x;
#pragma unroll 4
        for (int s = 0; s < n; ++s) qv[s * BW] = a.sign * (double)gp[(long long)s * hs];
        const int4 *nodes = a.nodes + G.node_off[p];
        for (int k = G.nnodes[p] - 1; k >= 0; --k) {
            const int4 nd = nodes[k];
            const int s0 = nd.x, na = nd.y, par = nd.z;
            double v = -1e300;
            for (int q = 0; q < na; ++q) {
                const double val = qv[(s0 + q) * BW];
                v = val > v ? val : v;
            }
            if (par >= 0) qv[par * BW] += v;
            else root += v;
        }
    }
    red[threadIdx.x] = root;
    __syncthreads();
    for (int st = BW / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) a.partial[blockIdx.x] = red[0];
}

// expl[g] = (BR1 + BR2) / 2 / pot0, sums over each game's blocks in order.
__global__ void expl_kernel(const SolverGame *games, int ngames, const int *nblocks, const double *part1,
                            const double *part2, double *expl, double *br1, double *br2) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ngames) return;
    const int b0 = games[g].block0, nb = nblocks[g];
    double s1 = 0.0, s2 = 0.0;
    for (int b = b0; b < b0 + nb; ++b) {
        s1 += part1[b];
        s2 += part2[b];
    }
    if (br1) br1[g] = s1;
    if (br2) br2[g] = s2;
    expl[g] = 0.5 * (s1 + s2) / games[g].pot0;
}

}  // namespace

struct kps_solver {
    kps_batch *batch = nullptr;
    kps_dtype dt = KPS_F32;
    int nblocks = 0, nmax = 0;
    int bw = kThreads;              // hands per block of the node kernels
    void *blob = nullptr;           // games, block_game, nblocks, nodes
    SolverGame *games = nullptr;
    int *block_game = nullptr, *game_blocks = nullptr;
    int4 *nodes = nullptr;
    // state, per player (concatenated layouts)
    void *g[2] = {nullptr, nullptr}, *x[2] = {nullptr, nullptr};
    void *regret[2] = {nullptr, nullptr}, *xsum[2] = {nullptr, nullptr};
    float *beh0[2] = {nullptr, nullptr};
    double *xa[2] = {nullptr, nullptr}, *g64[2] = {nullptr, nullptr};
    double *partial[2] = {nullptr, nullptr};
    long long *iter = nullptr;      // completed iterations (device)
    long long *init_iter = nullptr; // iteration that plays the initial strategy (device)
    double *wsum = nullptr;         // sum of the average weights (device)
    int has_beh = 0;
    double kappa = 0.0, w0 = 0.0;
    int method = 0;                 // 0 RM+, 1 DCFR
    double alpha = 1.5, beta = 0.0, gamma = 2.0;
    double *dtab = nullptr;         // DCFR factors per iteration (device), 3 per t
    long long dtab_cap = 0;         // iterations covered
    long long iters_host = 0;
    cudaStream_t cap = nullptr;     // capture stream
    std::map<int, cudaGraphExec_t> graphs;
    std::vector<void *> allocs;
    // non-finite check after every kps_solver_step: device flag, its pinned
    // host copy and the event that tells when the copy has landed
    unsigned int *bad = nullptr;
    unsigned int *bad_host = nullptr;
    cudaEvent_t bad_ev = nullptr;
    bool check_pending = false;
};

namespace {

size_t elem_size(kps_dtype dt) { return dtype_size(dt); }
size_t compute_size(kps_dtype dt) { return dt == KPS_F64 ? 8 : 4; }

template <typename S, typename C>
UpdateArgs<S, C> make_args(kps_solver *s, int p) {
    UpdateArgs<S, C> u;
    u.games = s->games;
    u.block_game = s->block_game;
    u.nodes = s->nodes;
    u.player = p;
    u.sign = p == 0 ? C(1) : C(-1);
    u.g = static_cast<const S *>(s->g[p]);
    u.regret = static_cast<C *>(s->regret[p]);
    u.x = static_cast<S *>(s->x[p]);
    u.xsum = static_cast<C *>(s->xsum[p]);
    u.beh0 = s->beh0[p];
    u.iter = s->iter;
    u.init_iter = s->init_iter;
    u.wsum = s->wsum;
    u.kappa = C(s->kappa);
    u.w0 = C(s->w0);
    u.method = s->method;
    u.dtab = s->dtab;
    u.nmax = s->nmax;
    return u;
}

// Raises a kernel's dynamic shared-memory limit once per size (never
// inside a stream capture: the solver warms every kernel up first).
cudaError_t smem_limit(const void *kernel, size_t smem) {
    if (smem <= 48 * 1024) return cudaSuccess;
    return kps::ensure_dyn_smem(kernel, smem);
}

template <typename S, typename C, typename K>
cudaError_t launch_node_kernel(kps_solver *s, K kernel, const UpdateArgs<S, C> &u, size_t smem, cudaStream_t st) {
    cudaError_t e = smem_limit(reinterpret_cast<const void *>(kernel), smem);
    if (e != cudaSuccess) return e;
    kernel<<<s->nblocks, s->bw, smem, st>>>(u);
    return cudaGetLastError();
}

template <typename S, typename C>
cudaError_t update_t(kps_solver *s, int p, cudaStream_t st) {
    const size_t smem = 2 * (size_t)s->nmax * s->bw * sizeof(C);
    return launch_node_kernel(s, s->bw == kThreads ? rm_update_kernel<S, C, kThreads> : rm_update_kernel<S, C, kThreads / 2>,
                              make_args<S, C>(s, p), smem, st);
}

template <typename S, typename C>
cudaError_t seqform_t(kps_solver *s, int p, cudaStream_t st) {
    const size_t smem = (size_t)s->nmax * s->bw * sizeof(C);
    auto kern = s->bw == kThreads ? seqform_kernel<S, C, kThreads> : seqform_kernel<S, C, kThreads / 2>;
    cudaError_t e = smem_limit(reinterpret_cast<const void *>(kern), smem);
    if (e != cudaSuccess) return e;
    kern<<<s->nblocks, s->bw, smem, st>>>(make_args<S, C>(s, p), s->has_beh);
    return cudaGetLastError();
}

template <typename S, typename C>
cudaError_t average_t(kps_solver *s, int p, double *out, int behavioural, cudaStream_t st) {
    auto kern = s->bw == kThreads ? average_kernel<S, C, double, kThreads> : average_kernel<S, C, double, kThreads / 2>;
    kern<<<s->nblocks, s->bw, 0, st>>>(make_args<S, C>(s, p), out, behavioural);
    return cudaGetLastError();
}

template <typename S, typename C>
cudaError_t average32_t(kps_solver *s, int p, float *out, cudaStream_t st) {
    auto kern = s->bw == kThreads ? average_kernel<S, C, float, kThreads> : average_kernel<S, C, float, kThreads / 2>;
    kern<<<s->nblocks, s->bw, 0, st>>>(make_args<S, C>(s, p), out, 0);
    return cudaGetLastError();
}

// Dispatch on the storage type.
#define KPS_DISPATCH(dt, F, ...)                                                        \
    ((dt) == KPS_F32    ? F<float, float>(__VA_ARGS__)                                  \
     : (dt) == KPS_F64  ? F<double, double>(__VA_ARGS__)                                \
     : (dt) == KPS_BF16 ? F<__nv_bfloat16, float>(__VA_ARGS__)                          \
                        : F<__half, float>(__VA_ARGS__))

kps_status one_iteration(kps_solver *s, cudaStream_t st) {
    kps_status r = batch_matvec(s->batch, 0, s->x[1], s->g[0], s->dt, st);
    if (r != KPS_OK) return r;
    cudaError_t e = KPS_DISPATCH(s->dt, update_t, s, 0, st);
    if (e != cudaSuccess) return cuda_fail(e, "player-1 update");
    r = batch_matvec(s->batch, 1, s->x[0], s->g[1], s->dt, st);
    if (r != KPS_OK) return r;
    e = KPS_DISPATCH(s->dt, update_t, s, 1, st);
    if (e != cudaSuccess) return cuda_fail(e, "player-2 update");
    bump_kernel<<<1, 1, 0, st>>>(s->iter, s->wsum, s->method, s->dtab);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "iteration counter");
    return KPS_OK;
}

// Sets *bad when a regret, a weighted strategy sum or a current strategy
// entry of a player is not finite (NaN or infinite): a product or an update
// has gone wrong, and the averages and exploitability carry it from then on
// (RM+'s max(0, .) turns a NaN regret into 0, so the regrets alone can look
// clean while the averages are not).
template <typename S, typename C>
__global__ void nonfinite_kernel(const C *regret, const C *xsum, const S *x, long long n, unsigned int *bad) {
    bool ok = true;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        ok = ok && isfinite((double)regret[i]) && isfinite((double)xsum[i]) && isfinite((double)Cv<S>::ld(x + i));
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(bad, 1u);
}

template <typename S, typename C>
cudaError_t nonfinite_t(kps_solver *s, int p, cudaStream_t st) {
    const long long n = s->batch->off[p].back();
    const int blocks = (int)std::min<long long>(1024, (n + 255) / 256);
    if (blocks <= 0) return cudaSuccess;
    nonfinite_kernel<S, C><<<blocks, 256, 0, st>>>(static_cast<const C *>(s->regret[p]),
                                                    static_cast<const C *>(s->xsum[p]),
                                                    static_cast<const S *>(s->x[p]), n, s->bad);
    return cudaGetLastError();
}

// Checkpoint of a solver (kps_solver_save / kps_solver_load): this header,
// then per player its regrets and its weighted strategy sums (compute
// type), its current strategy (storage type) and its initial behavioural
// strategy (FP32).
struct SolverCkpt {
    char magic[8];
    int32_t version, dtype, method, has_beh;
    double alpha, beta, gamma, kappa, w0, wsum;
    int64_t iter, init_iter;
    int64_t len[2];
    int64_t ngames;
    uint64_t signature;
};
constexpr char kCkptMagic[8] = {'K', 'P', 'S', 'S', 'O', 'L', 'V', '1'};

// Shape signature of a batch: games, hands and sequences (FNV-1a).
uint64_t batch_signature(const kps_batch *b) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](int64_t v) {
        for (int i = 0; i < 8; ++i) {
            h ^= (uint64_t)((v >> (8 * i)) & 0xff);
            h *= 1099511628211ull;
        }
    };
    mix((int64_t)b->games.size());
    for (const kps_game *g : b->games) {
        mix(g->host.H);
        mix(g->host.n[0]);
        mix(g->host.n[1]);
        mix(g->host.nodes[0]);
        mix(g->host.nodes[1]);
    }
    return h;
}

size_t ckpt_bytes(const kps_solver *s) {
    const size_t es = elem_size(s->dt), csz = compute_size(s->dt);
    size_t n = sizeof(SolverCkpt);
    for (int p = 0; p < 2; ++p) n += (size_t)s->batch->off[p].back() * (2 * csz + es + 4);
    return n;
}

void free_solver(kps_solver *s) {
    if (s->bad_ev) cudaEventDestroy(s->bad_ev);
    if (s->bad_host) cudaFreeHost(s->bad_host);
    for (auto &kv : s->graphs) cudaGraphExecDestroy(kv.second);
    if (s->dtab) cudaFree(s->dtab);
    for (void *p : s->allocs) cudaFree(p);
    if (s->cap) cudaStreamDestroy(s->cap);
    delete s;
}

// DCFR factors for every iteration up to `last` (host std::pow, the same
// values on every run); a reallocated table invalidates captured graphs.
kps_status ensure_dtab(kps_solver *s, long long last, cudaStream_t st) {
    if (s->method != 1 || last < s->dtab_cap) return KPS_OK;
    long long cap = std::max<long long>(1024, s->dtab_cap);
    while (cap <= last) cap *= 2;
    std::vector<double> h(3 * (size_t)cap, 0.0);
    for (long long t = 1; t < cap; ++t) {
        const double ta = std::pow((double)t, s->alpha), tb = std::pow((double)t, s->beta);
        h[3 * t] = ta / (ta + 1.0);
        h[3 * t + 1] = tb / (tb + 1.0);
        h[3 * t + 2] = std::pow((double)t, s->gamma);
    }
    double *d = nullptr;
    if (cudaMalloc(&d, h.size() * sizeof(double)) != cudaSuccess) return fail(KPS_ENOMEM, "DCFR table");
    cudaError_t e = cudaMemcpy(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "uploading the DCFR table");
    }
    (void)st;
    cudaDeviceSynchronize();   // work using the old table has finished
    if (s->dtab) cudaFree(s->dtab);
    s->dtab = d;
    s->dtab_cap = cap;
    for (auto &kv : s->graphs) cudaGraphExecDestroy(kv.second);
    s->graphs.clear();
    return KPS_OK;
}

}  // namespace

extern "C" {

kps_status kps_solver_create(kps_batch *b, kps_dtype dt, kps_solver **out) {
    if (!out) return fail(KPS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!b) return fail(KPS_EINVAL, "batch is NULL");
    if (dtype_size(dt) == 0) return fail(KPS_EINVAL, "unknown dtype");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != b->device) return fail(KPS_EINVAL, "batch tables live on another device");
    kps_solver *s = new (std::nothrow) kps_solver;
    if (!s) return fail(KPS_ENOMEM, "solver object");
    s->batch = b;
    s->dt = dt;
    const int ng = (int)b->games.size();
    // hands per block: 64, or 32 when the values and regrets of every
    // sequence of 64 hands do not fit in shared memory
    {
        int nm = 0;
        for (kps_game *g : b->games) nm = std::max(nm, std::max(g->host.n[0], g->host.n[1]));
        const size_t per = 2 * (size_t)nm * std::max<size_t>(compute_size(dt), 8);
        if (per * kThreads > (size_t)kps::max_dyn_smem()) s->bw = kThreads / 2;
    }
    std::vector<SolverGame> games(ng);
    std::vector<int> block_game, game_blocks(ng);
    std::vector<int4> nodes;
    for (int i = 0; i < ng; ++i) {
        const kps::HostGame &h = b->games[i]->host;
        SolverGame &G = games[i];
        G.H = h.H;
        G.hs = h.hs;
        G.pot0 = h.pot0;
        G.block0 = (int)block_game.size();
        {
            double cmax = 0.0;
            for (const kps::Terminal &z : h.terms) cmax = std::max(cmax, std::max(z.c1, z.c2));
            const double eps = dt == KPS_F64 ? 1.0 / 1099511627776.0 : 1.0 / 65536.0;
            for (int p = 0; p < 2; ++p) {
                const std::vector<double> &mp = p == 0 ? h.mu1 : h.mu2, &mq = p == 0 ? h.mu2 : h.mu1;
                double mmax = 0.0, msum = 0.0;
                for (double v : mp) mmax = std::max(mmax, v);
                for (double v : mq) msum += v;
                G.V[p] = cmax * mmax * msum / h.beta;
                G.theta[p] = eps * G.V[p];
            }
        }
        const int nb = (h.H + s->bw - 1) / s->bw;
        game_blocks[i] = nb;
        for (int k = 0; k < nb; ++k) block_game.push_back(i);
        for (int p = 0; p < 2; ++p) {
            G.n[p] = h.n[p];
            G.off[p] = b->off[p][i];
            G.node_off[p] = (int)nodes.size();
            G.nnodes[p] = h.nodes[p];
            s->nmax = std::max(s->nmax, h.n[p]);
            // first sequence of every node (sequences of a node are consecutive)
            std::vector<int> first(h.nodes[p], -1);
            for (int q = 0; q < h.n[p]; ++q)
                if (first[h.seqs[p][q].node] < 0) first[h.seqs[p][q].node] = q;
            for (int k = 0; k < h.nodes[p]; ++k) {
                const int na = h.nodes_nact[p][k];
                if (na > kMaxActions || first[k] < 0) {
                    free_solver(s);
                    return fail(KPS_ENOTSUP, "a decision node has more than 12 actions");
                }
                nodes.push_back(make_int4(first[k], na, h.seqs[p][first[k]].parent, 0));
            }
        }
    }
    s->nblocks = (int)block_game.size();
    const size_t csz = compute_size(dt);
    if (2 * (size_t)s->nmax * s->bw * std::max<size_t>(csz, 8) > (size_t)kps::max_dyn_smem()) {
        free_solver(s);
        return fail(KPS_ENOTSUP, "too many sequences per player for the solver's shared memory");
    }
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t o_g = 0, o_bg = al(sizeof(SolverGame) * ng), o_gb = al(o_bg + 4 * block_game.size()),
                 o_nd = al(o_gb + 4 * (size_t)ng), o_it = al(o_nd + sizeof(int4) * std::max<size_t>(1, nodes.size())),
                 total = al(o_it + 24);
    std::vector<unsigned char> host(total, 0);
    std::memcpy(host.data() + o_g, games.data(), sizeof(SolverGame) * ng);
    std::memcpy(host.data() + o_bg, block_game.data(), 4 * block_game.size());
    std::memcpy(host.data() + o_gb, game_blocks.data(), 4 * (size_t)ng);
    if (!nodes.empty()) std::memcpy(host.data() + o_nd, nodes.data(), sizeof(int4) * nodes.size());
    auto alloc = [&](size_t bytes, void **p) -> bool {
        if (cudaMalloc(p, std::max<size_t>(bytes, 256)) != cudaSuccess) return false;
        s->allocs.push_back(*p);
        return true;
    };
    if (!alloc(total, &s->blob)) { free_solver(s); return fail(KPS_ENOMEM, "solver tables"); }
    cudaError_t e = cudaMemcpy(s->blob, host.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { free_solver(s); return cuda_fail(e, "uploading solver tables"); }
    unsigned char *bl = static_cast<unsigned char *>(s->blob);
    s->games = reinterpret_cast<SolverGame *>(bl + o_g);
    s->block_game = reinterpret_cast<int *>(bl + o_bg);
    s->game_blocks = reinterpret_cast<int *>(bl + o_gb);
    s->nodes = reinterpret_cast<int4 *>(bl + o_nd);
    s->iter = reinterpret_cast<long long *>(bl + o_it);
    s->init_iter = reinterpret_cast<long long *>(bl + o_it + 8);
    s->wsum = reinterpret_cast<double *>(bl + o_it + 16);
    const size_t es = elem_size(dt);
    for (int p = 0; p < 2; ++p) {
        const size_t len = (size_t)b->off[p].back();
        bool ok = alloc(len * es, &s->g[p]) && alloc(len * es, &s->x[p]) && alloc(len * csz, &s->regret[p]) &&
                  alloc(len * csz, &s->xsum[p]) && alloc(len * 4, reinterpret_cast<void **>(&s->beh0[p])) &&
                  alloc(len * 8, reinterpret_cast<void **>(&s->xa[p])) &&
                  alloc(len * 8, reinterpret_cast<void **>(&s->g64[p])) &&
                  alloc((size_t)s->nblocks * 8, reinterpret_cast<void **>(&s->partial[p]));
        if (!ok) { free_solver(s); return fail(KPS_ENOMEM, "solver state"); }
    }
    e = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) { free_solver(s); return cuda_fail(e, "capture stream"); }
    if (!alloc(4, reinterpret_cast<void **>(&s->bad)) ||
        cudaMallocHost(reinterpret_cast<void **>(&s->bad_host), 4) != cudaSuccess) {
        free_solver(s);
        return fail(KPS_ENOMEM, "non-finite flag");
    }
    *s->bad_host = 0;
    e = cudaEventCreateWithFlags(&s->bad_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) { free_solver(s); return cuda_fail(e, "non-finite event"); }
    // launch tables of the products the solver uses, built before any capture
    for (kps_dtype d : {dt, KPS_F64}) {
        BatchShape sh;
        kps_status st = batch_default_shape(b, d, nullptr, &sh);
        for (int dir = 0; dir < 2 && st == KPS_OK && sh.kernel == KPS_BATCH_TMEM; ++dir) {
            const BatchTable *t = nullptr;
            st = batch_table(b, dir, d == KPS_F64, sh.nw, nullptr, &t);
        }
        if (st != KPS_OK) { free_solver(s); return st; }
    }
    // one iteration outside any capture sets every kernel attribute; then start over
    kps_status st = kps_solver_reset(s, nullptr, nullptr, nullptr);
    if (st == KPS_OK) st = one_iteration(s, nullptr);
    if (st == KPS_OK) st = kps_solver_reset(s, nullptr, nullptr, nullptr);
    if (st != KPS_OK) { free_solver(s); return st; }
    *out = s;
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_solver(s);
        *out = nullptr;
        return cuda_fail(e, "solver set-up");
    }
    return KPS_OK;
}

kps_status kps_solver_destroy(kps_solver *s) {
    if (s) free_solver(s);
    return KPS_OK;
}

kps_status kps_solver_warm_start(kps_solver *s, const float *beh1, const float *beh2, double kappa, int32_t t0,
                                 void *stream_ptr) {
    if (!s) return fail(KPS_EINVAL, "solver is NULL");
    if ((beh1 == nullptr) != (beh2 == nullptr)) return fail(KPS_EINVAL, "give both initial strategies or neither");
    if (!(kappa >= 0.0) || t0 < 0) return fail(KPS_EINVAL, "kappa and t0 must be >= 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream_ptr);
    const size_t es = elem_size(s->dt);
    // a fresh start clears the non-finite report (after any check in flight)
    if (s->check_pending) cudaEventSynchronize(s->bad_ev);
    s->check_pending = false;
    if (s->bad_host) *s->bad_host = 0;
    s->has_beh = beh1 ? 1 : 0;
    s->kappa = kappa;
    double w0 = 0.0;
    for (int k = 1; k <= t0; ++k) w0 += s->method == 0 ? (double)k : std::pow((double)k, s->gamma);
    {
        kps_status r0 = ensure_dtab(s, (long long)t0 + 1, st);
        if (r0 != KPS_OK) return r0;
    }
    s->w0 = w0;
    const long long iter0 = t0, init_iter = beh1 ? (long long)t0 + 1 : 0;
    cudaError_t e = cudaSuccess;
    for (int p = 0; p < 2 && e == cudaSuccess; ++p) {
        const size_t len = (size_t)s->batch->off[p].back();
        // padding entries stay zero; the start kernel writes every hand entry
        e = cudaMemsetAsync(s->regret[p], 0, len * compute_size(s->dt), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(s->xsum[p], 0, len * compute_size(s->dt), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(s->x[p], 0, len * es, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(s->g[p], 0, len * es, st);
        if (e == cudaSuccess && beh1)
            e = cudaMemcpyAsync(s->beh0[p], p == 0 ? beh1 : beh2, len * 4, cudaMemcpyDeviceToDevice, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->iter, &iter0, 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->init_iter, &init_iter, 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->wsum, &s->w0, 8, cudaMemcpyHostToDevice, st);
    // the pageable copies above are staged before they return
    for (int p = 0; p < 2 && e == cudaSuccess; ++p) e = KPS_DISPATCH(s->dt, seqform_t, s, p, st);
    if (e != cudaSuccess) return cuda_fail(e, "starting the solver");
    s->iters_host = t0;
    return KPS_OK;
}

kps_status kps_solver_reset(kps_solver *s, const float *beh1, const float *beh2, void *stream_ptr) {
    return kps_solver_warm_start(s, beh1, beh2, 0.0, 0, stream_ptr);
}

kps_status kps_solver_set_method(kps_solver *s, int32_t method, double alpha, double beta, double gamma) {
    if (!s) return fail(KPS_EINVAL, "solver is NULL");
    if (method != 0 && method != 1) return fail(KPS_EINVAL, "method must be 0 (RM+) or 1 (DCFR)");
    if (method == 1 && !(std::isfinite(alpha) && std::isfinite(beta) && std::isfinite(gamma) && gamma >= 0.0))
        return fail(KPS_EINVAL, "DCFR needs finite alpha, beta and gamma >= 0");
    s->method = method;
    if (method == 1) {
        s->alpha = alpha;
        s->beta = beta;
        s->gamma = gamma;
    }
    if (s->dtab) {
        cudaDeviceSynchronize();
        cudaFree(s->dtab);
    }
    s->dtab = nullptr;
    s->dtab_cap = 0;
    // captured iteration graphs hold the old parameters
    for (auto &kv : s->graphs) cudaGraphExecDestroy(kv.second);
    s->graphs.clear();
    return KPS_OK;
}

kps_status kps_solver_step(kps_solver *s, int32_t iters, void *stream_ptr) {
    if (!s) return fail(KPS_EINVAL, "solver is NULL");
    if (iters < 0) return fail(KPS_EINVAL, "iters must be >= 0");
    if (iters == 0) return KPS_OK;
    // the check queued by an earlier call, if its result has landed
    if (s->check_pending && cudaEventQuery(s->bad_ev) == cudaSuccess) {
        s->check_pending = false;
        if (*s->bad_host) return fail(KPS_ENUMERIC, "a regret or strategy entry is not finite (NaN or infinite)");
    } else if (!s->check_pending && *s->bad_host) {
        return fail(KPS_ENUMERIC, "a regret or strategy entry is not finite (NaN or infinite)");
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream_ptr);
    kps_status r0 = ensure_dtab(s, s->iters_host + iters, st);
    if (r0 != KPS_OK) return r0;
    auto it = s->graphs.find(iters);
    if (it == s->graphs.end()) {
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "beginning graph capture");
        kps_status r = KPS_OK;
        for (int k = 0; k < iters && r == KPS_OK; ++k) r = one_iteration(s, s->cap);
        e = cudaStreamEndCapture(s->cap, &graph);
        if (r != KPS_OK) {
            if (graph) cudaGraphDestroy(graph);
            return r;
        }
        if (e != cudaSuccess) return cuda_fail(e, "ending graph capture");
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "instantiating the iteration graph");
        it = s->graphs.emplace(iters, exec).first;
    }
    cudaError_t e = cudaGraphLaunch(it->second, st);
    if (e != cudaSuccess) return cuda_fail(e, "launching the iteration graph");
    s->iters_host += iters;
    // non-finite check of the state the iterations left (read back
    // asynchronously; reported by the next step or by kps_solver_status)
    e = cudaMemsetAsync(s->bad, 0, 4, st);
    for (int p = 0; p < 2 && e == cudaSuccess; ++p) e = KPS_DISPATCH(s->dt, nonfinite_t, s, p, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->bad_host, s->bad, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(s->bad_ev, st);
    if (e != cudaSuccess) return cuda_fail(e, "non-finite check");
    s->check_pending = true;
    return KPS_OK;
}

kps_status kps_solver_status(kps_solver *s) {
    if (!s) return fail(KPS_EINVAL, "solver is NULL");
    if (s->check_pending) {
        cudaError_t e = cudaEventSynchronize(s->bad_ev);
        if (e != cudaSuccess) return cuda_fail(e, "waiting for the non-finite check");
        s->check_pending = false;
    }
    if (*s->bad_host) return fail(KPS_ENUMERIC, "a regret or strategy entry is not finite (NaN or infinite)");
    return KPS_OK;
}

kps_status kps_solver_state_bytes(const kps_solver *s, int64_t *bytes) {
    if (!s || !bytes) return fail(KPS_EINVAL, "NULL argument");
    *bytes = (int64_t)ckpt_bytes(s);
    return KPS_OK;
}

kps_status kps_solver_save(kps_solver *s, void *host, int64_t bytes, void *stream_ptr) {
    if (!s || !host) return fail(KPS_EINVAL, "NULL argument");
    if (bytes < (int64_t)ckpt_bytes(s)) return fail(KPS_EINVAL, "buffer smaller than kps_solver_state_bytes");
    cudaStream_t st = static_cast<cudaStream_t>(stream_ptr);
    SolverCkpt h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kCkptMagic, 8);
    h.version = 1;
    h.dtype = (int32_t)s->dt;
    h.method = s->method;
    h.has_beh = s->has_beh;
    h.alpha = s->alpha;
    h.beta = s->beta;
    h.gamma = s->gamma;
    h.kappa = s->kappa;
    h.w0 = s->w0;
    h.ngames = (int64_t)s->batch->games.size();
    h.signature = batch_signature(s->batch);
    long long it = 0, ii = 0;
    double ws = 0.0;
    cudaError_t e = cudaMemcpyAsync(&it, s->iter, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ii, s->init_iter, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ws, s->wsum, 8, cudaMemcpyDeviceToHost, st);
    unsigned char *dst = static_cast<unsigned char *>(host) + sizeof(SolverCkpt);
    const size_t es = elem_size(s->dt), csz = compute_size(s->dt);
    for (int p = 0; p < 2 && e == cudaSuccess; ++p) {
        const size_t len = (size_t)s->batch->off[p].back();
        h.len[p] = (int64_t)len;
        const void *src[4] = {s->regret[p], s->xsum[p], s->x[p], s->beh0[p]};
        const size_t sz[4] = {len * csz, len * csz, len * es, len * 4};
        for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
            e = cudaMemcpyAsync(dst, src[k], sz[k], cudaMemcpyDeviceToHost, st);
            dst += sz[k];
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "saving the solver state");
    h.iter = it;
    h.init_iter = ii;
    h.wsum = ws;
    std::memcpy(host, &h, sizeof(h));
    return KPS_OK;
}

kps_status kps_solver_load(kps_solver *s, const void *host, int64_t bytes, void *stream_ptr) {
    if (!s || !host) return fail(KPS_EINVAL, "NULL argument");
    if (bytes < (int64_t)sizeof(SolverCkpt)) return fail(KPS_EINVAL, "buffer too small for a checkpoint");
    SolverCkpt h;
    std::memcpy(&h, host, sizeof(h));
    if (std::memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != 1) return fail(KPS_EINVAL, "not a solver checkpoint");
    if (h.dtype != (int32_t)s->dt) return fail(KPS_EINVAL, "checkpoint of a solver with another storage type");
    if (h.ngames != (int64_t)s->batch->games.size() || h.signature != batch_signature(s->batch) ||
        h.len[0] != s->batch->off[0].back() || h.len[1] != s->batch->off[1].back())
        return fail(KPS_EINVAL, "checkpoint of another batch of games");
    if (bytes < (int64_t)ckpt_bytes(s)) return fail(KPS_EINVAL, "checkpoint truncated");
    if (h.method != 0 && h.method != 1) return fail(KPS_EINVAL, "bad method in the checkpoint");
    if (h.iter < 0 || h.init_iter < 0) return fail(KPS_EINVAL, "bad iteration count in the checkpoint");
    cudaStream_t st = static_cast<cudaStream_t>(stream_ptr);
    // method and discount parameters as saved (captured graphs and the DCFR
    // table are rebuilt for them)
    if (h.method != s->method || (h.method == 1 && (h.alpha != s->alpha || h.beta != s->beta || h.gamma != s->gamma))) {
        kps_status r = kps_solver_set_method(s, h.method, h.alpha, h.beta, h.gamma);
        if (r != KPS_OK) return r;
    }
    cudaError_t e = cudaStreamSynchronize(st);   // work queued on the state has finished
    const unsigned char *src = static_cast<const unsigned char *>(host) + sizeof(SolverCkpt);
    const size_t es = elem_size(s->dt), csz = compute_size(s->dt);
    for (int p = 0; p < 2 && e == cudaSuccess; ++p) {
        const size_t len = (size_t)h.len[p];
        void *dst[4] = {s->regret[p], s->xsum[p], s->x[p], s->beh0[p]};
        const size_t sz[4] = {len * csz, len * csz, len * es, len * 4};
        for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
            e = cudaMemcpyAsync(dst[k], src, sz[k], cudaMemcpyHostToDevice, st);
            src += sz[k];
        }
    }
    const long long it = h.iter, ii = h.init_iter;
    const double ws = h.wsum;
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->iter, &it, 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->init_iter, &ii, 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->wsum, &ws, 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "loading the solver state");
    s->has_beh = h.has_beh;
    s->kappa = h.kappa;
    s->w0 = h.w0;
    s->iters_host = h.iter;
    s->check_pending = false;
    *s->bad_host = 0;
    return KPS_OK;
}

kps_status kps_solver_iterations(const kps_solver *s, int64_t *t) {
    if (!s || !t) return fail(KPS_EINVAL, "bad argument");
    *t = s->iters_host;
    return KPS_OK;
}

kps_status kps_solver_average(kps_solver *s, int32_t behavioural, double *x, double *y, void *stream_ptr) {
    if (!s) return fail(KPS_EINVAL, "solver is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream_ptr);
    for (int p = 0; p < 2; ++p) {
        double *dst = p == 0 ? x : y;
        if (!dst) continue;
        cudaError_t e = KPS_DISPATCH(s->dt, average_t, s, p, dst, behavioural ? 1 : 0, st);
        if (e != cudaSuccess) return cuda_fail(e, "averaging");
    }
    return KPS_OK;
}

kps_status kps_solver_strategy(kps_solver *s, void *x, void *y, void *stream_ptr) {
    if (!s) return fail(KPS_EINVAL, "solver is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream_ptr);
    const size_t es = elem_size(s->dt);
    for (int p = 0; p < 2; ++p) {
        void *dst = p == 0 ? x : y;
        if (!dst) continue;
        cudaError_t e = cudaMemcpyAsync(dst, s->x[p], (size_t)s->batch->off[p].back() * es, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "copying the strategy");
    }
    return KPS_OK;
}

}  // extern "C"

namespace {

// Averages, products of the averages (FP64, or FP32 for the estimate),
// best responses (FP64 sums), exploitability per game.
kps_status exploitability_impl(kps_solver *s, bool f32, double *expl, double *br1, double *br2, cudaStream_t st) {
    if (!s || !expl) return fail(KPS_EINVAL, "bad argument");
    for (int p = 0; p < 2; ++p) {
        cudaError_t e = f32 ? KPS_DISPATCH(s->dt, average32_t, s, p, reinterpret_cast<float *>(s->xa[p]), st)
                            : KPS_DISPATCH(s->dt, average_t, s, p, s->xa[p], 0, st);
        if (e != cudaSuccess) return cuda_fail(e, "averaging");
    }
    const kps_dtype pd = f32 ? KPS_F32 : KPS_F64;
    kps_status r = batch_matvec(s->batch, 0, s->xa[1], s->g64[0], pd, st);
    if (r == KPS_OK) r = batch_matvec(s->batch, 1, s->xa[0], s->g64[1], pd, st);
    if (r != KPS_OK) return r;
    const size_t smem = (size_t)s->nmax * s->bw * sizeof(double);
    const bool wide = s->bw == kThreads;
    auto kf = wide ? best_response_kernel<float, kThreads> : best_response_kernel<float, kThreads / 2>;
    auto kd = wide ? best_response_kernel<double, kThreads> : best_response_kernel<double, kThreads / 2>;
    const void *kern = f32 ? reinterpret_cast<const void *>(kf) : reinterpret_cast<const void *>(kd);
    cudaError_t e = smem_limit(kern, smem);
    if (e != cudaSuccess) return cuda_fail(e, "best response");
    for (int p = 0; p < 2; ++p) {
        BrArgs a;
        a.games = s->games;
        a.block_game = s->block_game;
        a.nodes = s->nodes;
        a.player = p;
        a.sign = p == 0 ? 1.0 : -1.0;
        a.g = s->g64[p];
        a.partial = s->partial[p];
        if (f32) kf<<<s->nblocks, s->bw, smem, st>>>(a);
        else kd<<<s->nblocks, s->bw, smem, st>>>(a);
    }
    const int ng = (int)s->batch->games.size();
    expl_kernel<<<(ng + 127) / 128, 128, 0, st>>>(s->games, ng, s->game_blocks, s->partial[0], s->partial[1], expl, br1,
                                                  br2);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "best response");
    return KPS_OK;
}

}  // namespace

extern "C" {

kps_status kps_solver_exploitability(kps_solver *s, double *expl, double *br1, double *br2, void *stream_ptr) {
    return exploitability_impl(s, false, expl, br1, br2, static_cast<cudaStream_t>(stream_ptr));
}

kps_status kps_solver_exploitability_estimate(kps_solver *s, double *expl, void *stream_ptr) {
    return exploitability_impl(s, true, expl, nullptr, nullptr, static_cast<cudaStream_t>(stream_ptr));
}

}  // extern "C"
