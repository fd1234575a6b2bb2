/*
 * kps.h -- C ABI of the Kronecker payoff-product library for GB300 (sm_103a).
 *
 * The library evaluates the payoff-matrix products A*y and A^T*x of a
 * two-player poker river endgame directly in the Kronecker form of
 * Farina & Sandholm, "Fast Payoff Matrix Sparsification Techniques for
 * Structured Extensive-Form Games" (AAAI-22), Prop. 1:
 *
 *     A = C (x) F + (Lambda1 W Lambda2) (x) S,
 *     C[h1,h2] = lambda1[h1] lambda2[h2] (1 - Hx[h1,h2]),
 *     lambda_i = mu_i / sqrt(beta),
 *
 * with F and S the fold and showdown payoffs of the betting skeleton
 * (Sec. 3), Hx the card-overlap indicator and W the win/lose sign.  The
 * card blocks are applied in O(hands + cards): the fold block by
 * inclusion-exclusion over the cards of a hand (the sparsified fold term of
 * Sec. 4, eq. "cf"), the showdown block by strength-ordered prefix sums with
 * per-card corrections (the prefix sum is the inverse of the bidiagonal D of
 * Technique B, Sec. 4).
 *
 * Conventions shared by every call
 * --------------------------------
 * Ownership: the caller owns every vector buffer (device pointers, e.g. a
 *   torch tensor's data_ptr()).  The library owns the opaque kps_game object
 *   and the device tables it uploads; kps_game_destroy frees both.
 * Errors: no C++ exception crosses the ABI.  Every call returns a
 *   kps_status; kps_last_error() returns a thread-local message describing
 *   the most recent failure of the calling thread.
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *   default stream).  GPU calls are asynchronous on that stream.
 * Hand order ("library order"): hands sorted by ascending strength, ties
 *   broken by canonical index.  The canonical order is the deck minus the
 *   board in increasing card id (card id = rank*suits + suit); one-card hands
 *   are single cards, two-card hands the pairs (a < b) in lexicographic
 *   order.  kps_game_hands() returns the cards and canonical index of every
 *   library-order hand.
 * Sequence order: depth-first pre-order of the skeleton; when a decision
 *   node is first reached, its actions receive consecutive sequence ids of
 *   the acting player in action order: fold, check/call, then aggressive
 *   actions by increasing amount.  The empty sequence is not stored.
 * Vector layout: [batch][sequence][hs], hs = H rounded up to a multiple of 8
 *   (kps_info.hs).  Entries h >= H are ignored on input and written as zero
 *   on output.  Player-1 vectors have n1 sequences, player-2 vectors n2.
 */
#ifndef KPS_H
#define KPS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KPS_OK = 0,
    KPS_EINVAL = 1,     /* invalid argument or game spec                      */
    KPS_ENOMEM = 2,     /* host or device allocation failed                   */
    KPS_ECUDA = 3,      /* a CUDA runtime call failed                         */
    KPS_ETIMEOUT = 4,   /* a bounded device wait gave up                      */
    KPS_ENOTSUP = 5,    /* valid input outside what this build supports       */
    KPS_ENUMERIC = 6    /* NaN/Inf detected                                   */
} kps_status;

typedef enum {
    KPS_F32 = 0,        /* storage f32, arithmetic f32                        */
    KPS_F64 = 1,        /* storage f64, arithmetic f64                        */
    KPS_BF16 = 2,       /* storage bf16, arithmetic f32                       */
    KPS_F16 = 3         /* storage f16, arithmetic f32                        */
} kps_dtype;

#define KPS_MAX_BETS 8
#define KPS_MAX_BOARD 8
#define KPS_SITUATIONS 5

/* Optional betting menu: the bet/raise pot fractions of each player in
 * each situation of the round (the shape of the Libratus abstraction the
 * paper's experiments use, appendix "Libratus' betting abstraction"):
 *   situation 0: first action of the round,
 *             1: after a check,
 *             2: facing the first bet,
 *             3: facing one raise,
 *             4: facing two or more raises.
 * nbet[p][s] fractions bet_frac[p][s][0..nbet-1] (> 0, finite) for player p
 * (0 = player 1).  Fractions are applied as the spec's bet_frac are. */
typedef struct {
    int32_t nbet[2][KPS_SITUATIONS];
    double bet_frac[2][KPS_SITUATIONS][KPS_MAX_BETS];
} kps_bet_menu;

/* River endgame (Sec. 3): board B, stacks, initial pot contributions,
 * beliefs mu1, mu2 and a fixed betting abstraction (appendix "Betting
 * abstraction").  Betting rules (appendix "Betting rounds", Fig. 1 caption):
 *   - player 1 acts first; with equal contributions a player may check or
 *     bet, facing a larger contribution it may fold, call or raise;
 *   - a bet/raise of fraction f first matches the opponent and then adds
 *     f times the pot after matching;
 *   - an amount at or above the effective stack min(contrib0+stack) is the
 *     all-in amount and merges with the all-in action;
 *   - raise_cap limits the aggressive actions of the round (bets, raises
 *     and all-ins counted together; < 0 = no cap);
 *   - with a menu (kps_bet_menu), the fractions of the acting player in the
 *     current situation replace bet_frac;
 *   - a call, or a check after a check, ends the round in a showdown.
 * The payoff of player 1 is +c2 when player 2 folds, -c1 when player 1
 * folds, and gamma(h1,h2) * min(c1,c2) at a showdown. */
typedef struct {
    int32_t ranks, suits;               /* deck = ranks*suits <= 63 cards      */
    int32_t cards_per_hand;             /* 1 or 2                              */
    int32_t nboard;
    int32_t board[KPS_MAX_BOARD];       /* card ids                            */
    double stack[2];                    /* chips behind at the start           */
    double contrib0[2];                 /* pot contributions at the start (>0) */
    int32_t nbet;
    double bet_frac[KPS_MAX_BETS];      /* > 0                                 */
    int32_t raise_cap;
    int32_t allow_allin;
    const double *mu1, *mu2;            /* beliefs per CANONICAL hand; NULL = 1 */
    const int32_t *strength;            /* per CANONICAL hand, higher wins     */
    const kps_bet_menu *menu;           /* NULL = bet_frac in every situation  */
} kps_game_spec;

typedef struct {
    int32_t H;            /* hands per player (same set for both players)     */
    int32_t hs;           /* hand stride of the vector layout                 */
    int32_t n1, n2;       /* sequences of player 1 / player 2                 */
    int32_t T, T_fold, T_showdown;
    int32_t ncards;       /* cards left after the board                       */
    int32_t cards_per_hand;
    int32_t nodes1, nodes2;       /* decision nodes of each player            */
    int32_t max_tie;      /* longest run of equal strengths                    */
    double beta;          /* normalisation of the chance deal pi (Sec. 3)     */
    double pot0;          /* contrib0[0] + contrib0[1]                        */
    /* Technique B (Sec. 4) sizes: nnz of A, then Ahat, U, M, V before and
     * after the postprocessing of Sec. 4. */
    int64_t nnz_A;
    int64_t nnz_Ahat, nnz_U, nnz_M, nnz_V;
    int64_t pp_nnz_Ahat, pp_nnz_U, pp_nnz_M, pp_nnz_V;
} kps_info;

typedef struct kps_game kps_game;

/* Build a game from its spec on the host (Sec. 3 skeleton, Prop. 1 factor
 * tables, Technique B counts).  Device tables are uploaded on the first GPU
 * call (or by kps_game_upload).  *out receives a new object on KPS_OK.
 * Errors: KPS_EINVAL (bad spec), KPS_ENOMEM, KPS_ENOTSUP (deck > 63 cards). */
kps_status kps_sparsify(const kps_game_spec *spec, kps_game **out);

/* Free the game and its device tables.  NULL is accepted. */
kps_status kps_game_destroy(kps_game *game);

/* Sizes and Technique B counts.  Host only. */
kps_status kps_game_info(const kps_game *game, kps_info *info);

/* Library-order hands: cards[i*k + j] (card ids), canon[i] = canonical
 * index.  Either pointer may be NULL.  Host only. */
kps_status kps_game_hands(const kps_game *game, int32_t *cards, int32_t *canon);

/* Sequences of player p (0 or 1): decision-node index, parent sequence of
 * that node (-1 = empty), action code (0 fold, 1 check/call, 2 aggressive),
 * contribution after the action; nodes_nact[i] = actions of node i.  Any
 * pointer may be NULL.  Host only. */
kps_status kps_game_sequences(const kps_game *game, int32_t player, int32_t *seq_node,
                              int32_t *seq_parent, int32_t *seq_action,
                              double *seq_amount, int32_t *nodes_nact);

/* Terminals in depth-first order: last sequence of each player, kind
 * (0 fold, 1 showdown), folder (-1 for showdowns), contributions.  Any
 * pointer may be NULL.  Host only. */
kps_status kps_game_terminals(const kps_game *game, int32_t *s1, int32_t *s2,
                              int32_t *kind, int32_t *folder, double *c1, double *c2);

/* Upload the device tables now (otherwise done by the first GPU call).
 * Call it before capturing GPU calls into a CUDA graph. */
kps_status kps_game_upload(kps_game *game, void *stream);

/* Which kernel ran the last product of a direction (dir 0 = A * y,
 * 1 = A^T * x) on this game: one of the KPS_KERNEL_* codes, 0 before the
 * first product.  The library picks the kernel from the dtype, the
 * vectors' alignment and the game's shape (tie groups, hand and card
 * counts); the environment variable KPS_KERNEL = tma | tmem | vec | fast
 * forces one where it applies.  Diagnostics only: results agree within the
 * stated tolerances whichever kernel runs. */
#define KPS_KERNEL_TMA 1      /* TMA-staged boxes, tensor-memory partials (FP32) */
#define KPS_KERNEL_TMEM 2     /* register staging, tensor-memory partials */
#define KPS_KERNEL_VEC 3      /* 16-byte asynchronous copies, partials through L2 */
#define KPS_KERNEL_SCALAR 4   /* scalar staging, partials through L2 */
#define KPS_KERNEL_GENERAL 5  /* tie groups longer than a tile */
kps_status kps_game_kernel(const kps_game *game, int32_t dir, int32_t *kernel);

/* out_b = A * y_b for b < batch (Prop. 1; the gradient of Sec. 2, "First-
 * order methods").  y: device [batch][n2][hs], out: device [batch][n1][hs],
 * both of type dt, non-overlapping.  batch >= 0 (0 is a no-op).
 * Errors: KPS_EINVAL (NULL/size/dtype), KPS_ECUDA (launch failure). */
kps_status kps_matvec_A(kps_game *game, const void *y, void *out, int32_t batch,
                        kps_dtype dt, void *stream);

/* out_b = A^T * x_b.  x: device [batch][n1][hs], out: device [batch][n2][hs]. */
kps_status kps_matvec_AT(kps_game *game, const void *x, void *out, int32_t batch,
                         kps_dtype dt, void *stream);

/* The same products through host buffers: copies in, computes on the
 * device, copies out, synchronises `stream`.  Uses library-owned device
 * staging buffers that grow as needed. */
kps_status kps_matvec_A_host(kps_game *game, const void *y, void *out, int32_t batch,
                             kps_dtype dt, void *stream);
kps_status kps_matvec_AT_host(kps_game *game, const void *x, void *out, int32_t batch,
                              kps_dtype dt, void *stream);

/* ---- Batches of games in one launch -------------------------------------
 * A batch holds several games (uneven hand counts and betting trees) whose
 * products run as ONE persistent kernel launch: CTAs take (game, 32-column
 * tile) tickets from an atomic counter (or a static stride) until every
 * tile of every game is done.  Not in the paper, whose products are per
 * game (Prop. 1); the per-game arithmetic is that of kps_matvec_A/AT.
 * Layout: one vector per game and player, concatenated in game order; game
 * g's player-p vector ([n_p(g)][hs(g)], same conventions as above) starts
 * at element off_p[g] (kps_batch_offsets).  Batch vectors must be 16-byte
 * aligned.  The games must outlive the batch, share cards_per_hand and have
 * no tie group longer than 32 hands.  Calls on one batch must not overlap
 * on the GPU (they share a ticket counter); they are asynchronous on
 * `stream`, and capturable in a CUDA graph once the batch has run (or been
 * tuned) for that dtype. */
typedef struct kps_batch kps_batch;

/* Multi-game kernels (kps_batch_shape.kernel):
 *   KPS_BATCH_TMEM    tensor-memory scan, 32-column tiles, 1-8 warps (every
 *                     storage type; FP64 runs its vector-register variant);
 *   KPS_BATCH_STAGED  FP32, BF16 or FP16 storage (FP32 arithmetic): 4 warps
 *                     per CTA scan chunks of a game's hand order in 16-hand
 *                     boxes staged by cp.async, with per-box hand records
 *                     (games whose tie groups have at most 4 hands and whose
 *                     chunks fit 24 boxes; the others run on the
 *                     tensor-memory kernel in a second launch). */
#define KPS_BATCH_TMEM 0
#define KPS_BATCH_STAGED 1

typedef struct {
    int32_t warps;        /* warps per CTA                                  */
    int32_t grid;         /* CTAs of the persistent launch                  */
    int32_t schedule;     /* 0 atomic ticket counter, 1 static stride       */
    int32_t kernel;       /* KPS_BATCH_TMEM or KPS_BATCH_STAGED             */
    double ms_per_pair;   /* tuned time of one A and one A^T launch, or 0   */
} kps_batch_shape;

/* Uploads every game.  Errors: KPS_EINVAL (NULL, mixed cards_per_hand),
 * KPS_ENOTSUP (tie group > 32 hands), KPS_ENOMEM. */
kps_status kps_batch_create(kps_game *const *games, int32_t n, kps_batch **out);
kps_status kps_batch_destroy(kps_batch *batch);
/* off[0..n]: element offsets of each game's player-`player` vector; off[n]
 * is the length of the batch vector.  Host only. */
kps_status kps_batch_offsets(const kps_batch *batch, int32_t player, int64_t *off);
/* out = A y per game (y: player-2 layout, out: player-1 layout) / A^T x. */
kps_status kps_batch_matvec_A(kps_batch *batch, const void *y, void *out, kps_dtype dt, void *stream);
kps_status kps_batch_matvec_AT(kps_batch *batch, const void *x, void *out, kps_dtype dt, void *stream);
/* Autotuner: times every admissible launch shape (kernel, warps per CTA,
 * CTAs per SM, schedule) of an A and an A^T launch with CUDA events on `stream`,
 * keeps the fastest for `dt` and reports it in *chosen (may be NULL).
 * Allocates temporary buffers; synchronises `stream`. */
kps_status kps_batch_tune(kps_batch *batch, kps_dtype dt, void *stream, kps_batch_shape *chosen);
/* The launch shape in use for `dt` (the default one if never tuned). */
kps_status kps_batch_shape_get(kps_batch *batch, kps_dtype dt, kps_batch_shape *shape);
/* Sets the launch shape for `dt` (ms_per_pair ignored).  Errors: KPS_EINVAL
 * (out of range), KPS_ENOTSUP (warp count the games do not fit; the staged
 * kernel for FP64, with other than 4 warps, more than 2
 * CTAs per SM, or for games it does not take). */
kps_status kps_batch_shape_set(kps_batch *batch, kps_dtype dt, const kps_batch_shape *shape);

/* Splits items 0..n-1 (games, in order) into `parts` contiguous ranges
 * [bounds[k], bounds[k+1]) whose weight sums (e.g. H * (n1 + n2) bytes per
 * game) are as even as a prefix split allows: cut k falls where the prefix
 * sum is closest to k/parts of the total.  bounds has parts + 1 entries.
 * Host only; used to shard a batch of games over GPUs, one rank each (the
 * games need no communication; only per-game scalars are gathered). */
kps_status kps_partition(const int64_t *weights, int32_t n, int32_t parts, int32_t *bounds);

/* ---- Turn endgames (end of Sec. 3) -----------------------------------------
 * A turn endgame: the turn betting round, then at every ending of that
 * round that is not a fold the river card (public; uniform over the cards
 * in neither hand nor on the board) and the river betting round.  The river
 * card being public, the payoff matrix is block diagonal with one river
 * block per (turn ending, river card), each a river game of Prop. 1 (the
 * paper's remark after Prop. 1).  The library builds the turn round (its
 * folds) and every block as Kronecker-form games and runs the products of
 * all of them in one batched persistent launch.
 *   - Hands: 1- or 2-card hands over the deck minus the turn board
 *     (canonical order as for kps_game_spec), the same hand set in every
 *     block; beliefs mu1, mu2 per canonical hand (NULL = 1).
 *   - strength[r * H + h]: showdown strength of canonical hand h when the
 *     river card is r (card id); higher wins; entries for cards on the
 *     board or in the hand are not read.
 *   - Betting in each round as for kps_game_spec, player 1 first in both;
 *     the river starts from the turn ending's contributions with the chips
 *     left behind.  An ending that leaves a player all in (no river betting)
 *     is refused (KPS_ENOTSUP).
 *   - Chance: pi(h1,h2) = mu1 mu2 / beta over disjoint hands (Sec. 3), the
 *     river card with probability 1 / (N - 2k) (N cards left after the
 *     board, k cards per hand); inside a block both factors are folded into
 *     lambda = mu / sqrt(beta (N - 2k)).
 * Vector layout: game after game as a kps_batch (kps_turn_offsets): game 0
 * is the turn round (its sequences), games 1.. the blocks, endings in
 * depth-first order of the turn round, river cards ascending; within a game
 * [sequence][hs], hands in that game's library order (kps_turn_block gives
 * the canonical index of every position: a block's order is its river
 * strength order).  One vector per call.
 * Errors: KPS_EINVAL (bad spec), KPS_ENOTSUP, KPS_ENOMEM, KPS_ECUDA. */
typedef struct {
    int32_t ranks, suits;              /* deck = ranks*suits <= 63 cards      */
    int32_t cards_per_hand;            /* 1 or 2                              */
    int32_t nboard;
    int32_t board[KPS_MAX_BOARD];      /* the turn board                      */
    double stack[2], contrib0[2];      /* at the start of the turn round      */
    int32_t nbet_turn;
    double bet_frac_turn[KPS_MAX_BETS];
    int32_t raise_cap_turn, allow_allin_turn;
    int32_t nbet_river;
    double bet_frac_river[KPS_MAX_BETS];
    int32_t raise_cap_river, allow_allin_river;
    const double *mu1, *mu2;           /* per canonical hand; NULL = 1        */
    const int32_t *strength;           /* [ranks*suits][H]                    */
} kps_turn_spec;

typedef struct kps_turn kps_turn;

kps_status kps_turn_create(const kps_turn_spec *spec, kps_turn **out);
kps_status kps_turn_destroy(kps_turn *turn);
/* info[0..8] = H, hs, n1, n2 (all sequences of the layout), turn endings
 * that are not folds, river blocks, games (blocks + 1), turn-round
 * sequences of player 1 and of player 2. */
kps_status kps_turn_info(const kps_turn *turn, int64_t *info);
/* Element offsets of every game's part of a player's vector (games + 1). */
kps_status kps_turn_offsets(const kps_turn *turn, int32_t player, int64_t *off);
/* Game `block` (0 = the turn round): its turn ending and river card (-1 for
 * the turn round) and the canonical index of each of its hand positions
 * (any pointer may be NULL). */
kps_status kps_turn_block(const kps_turn *turn, int32_t block, int32_t *ending, int32_t *river_card,
                          int32_t *canon);
/* out = A y (player-2 vector y, player-1 vector out) and out = A^T x, one
 * vector each, device, 16-byte aligned; dtypes as kps_batch_matvec_A. */
kps_status kps_turn_matvec_A(kps_turn *turn, const void *y, void *out, kps_dtype dt, void *stream);
kps_status kps_turn_matvec_AT(kps_turn *turn, const void *x, void *out, kps_dtype dt, void *stream);
/* The batch of games behind the turn endgame (owned by the turn object):
 * launch shapes (kps_batch_tune / kps_batch_shape_set) apply to it. */
kps_status kps_turn_batch(kps_turn *turn, kps_batch **batch);

/* ---- First-order solver ---------------------------------------------------
 * Regret matching plus with alternating updates and linearly weighted
 * averages on every game of a batch, the gradients A y and -A^T x coming
 * from the batched products (Sec. 2, "First-order methods", whose gradient
 * is the per-iteration cost that the sparsification of Prop. 1 makes cheap;
 * Sec. 5 runs such a solver).  One iteration t:
 *   xsum += t x;  R1 <- max(0, R1 + q - v) bottom-up against g = A y;
 *   x <- sequence form of R1 / sum R1 (uniform where the sum is at most
 *        a noise floor theta_p = eps * V_p, V_p a bound on player p's
 *        counterfactual values: eps = 2^-40 for KPS_F64 storage, 2^-16
 *        otherwise);
 *   ysum += t y;  the same for player 2 against g = -A^T x (the new x).
 * `dt` is the storage type of strategies and values (KPS_F32, KPS_F64,
 * KPS_BF16, KPS_F16); regrets, averages and arithmetic are FP32 (FP64 for
 * KPS_F64); averages, best responses and exploitability are FP64.  The
 * solver keeps a reference to the batch, which must outlive it. */
typedef struct kps_solver kps_solver;

/* Errors: KPS_ENOTSUP (a node with > 12 actions, too many sequences),
 * KPS_ENOMEM.  Starts from uniform strategies (kps_solver_reset). */
kps_status kps_solver_create(kps_batch *batch, kps_dtype dt, kps_solver **out);
kps_status kps_solver_destroy(kps_solver *solver);
/* Clears regrets, averages and the iteration count; the first iteration
 * plays the behavioural strategies beh1 / beh2 (device FP32, batch player
 * layouts: entry [sigma][h] = probability of sigma's last action at its
 * node), or uniform strategies if both are NULL. */
kps_status kps_solver_reset(kps_solver *solver, const float *beh1, const float *beh2, void *stream);
/* Warm start (not in the paper; the learned warm start of this library):
 * like kps_solver_reset, and in addition the regrets start at
 * kappa * V_p * beh_p (V_p = max|payoff| * max mu_p * sum mu_q / beta, a
 * bound on player p's counterfactual values; regret matching then returns
 * beh_p) and the initial strategies count as played at iterations 1..t0 of
 * the linear average; the next iteration is t0 + 1.  kappa = 0, t0 = 0 is
 * kps_solver_reset.  Errors: KPS_EINVAL (kappa < 0, t0 < 0, one of beh1 /
 * beh2 NULL). */
kps_status kps_solver_warm_start(kps_solver *solver, const float *beh1, const float *beh2, double kappa,
                                 int32_t t0, void *stream);
/* Selects the regret update: method 0 = RM+ (the default), method 1 =
 * Discounted CFR, the solver the paper runs (Sec. 5): on iteration t the
 * instantaneous regret is added, a cumulative regret is multiplied by
 * t^alpha/(t^alpha+1) when positive and t^beta/(t^beta+1) otherwise,
 * regret matching uses positive parts, iteration t enters the average with
 * weight t^gamma (1.5, 0, 2 are the usual values).  Takes effect at the next
 * reset / warm start.  Errors: KPS_EINVAL. */
kps_status kps_solver_set_method(kps_solver *solver, int32_t method, double alpha, double beta, double gamma);
/* Runs `iters` iterations as one CUDA graph (captured on first use of each
 * count), asynchronous on `stream`, then queues a check of the state those
 * iterations leave: every regret, weighted strategy sum and current
 * strategy entry of both players must be finite.  The check's result is read back asynchronously; a call
 * finds it once it has landed (KPS_ENUMERIC from that call on, and from
 * every later step, until kps_solver_reset, kps_solver_warm_start or
 * kps_solver_load), and kps_solver_status waits for it.  A NaN or an
 * infinity in the state (a non-finite input strategy, belief or payoff)
 * would otherwise be carried into the averages and the exploitability. */
kps_status kps_solver_step(kps_solver *solver, int32_t iters, void *stream);
/* Waits for the last step's non-finite check: KPS_OK, or KPS_ENUMERIC when
 * a regret, strategy-sum or strategy entry is NaN or infinite. */
kps_status kps_solver_status(kps_solver *solver);

/* ---- Checkpoint and resume ----------------------------------------------
 * A solver's whole iteration state goes to / comes from a caller-owned host
 * buffer of kps_solver_state_bytes bytes: a header (format version, storage
 * type, method and DCFR parameters, warm-start parameters, iteration count,
 * weight sum, a signature of the batch's games) followed, per player, by
 * the regrets and the weighted strategy sums (FP32, FP64 for KPS_F64), the
 * current sequence-form strategy (storage type) and the initial behavioural
 * strategy (FP32).  Iterations run after kps_solver_load are the ones an
 * uninterrupted solver would have run, bit for bit (Sec. 5's solver is a
 * long iterative run; this is how it survives a restart).
 *   kps_solver_save synchronises `stream` and fills `host`;
 *   kps_solver_load needs a solver created on a batch of the same games
 *   (same hands and trees) with the same storage type, synchronises
 *   `stream`, restores the method saved (kps_solver_set_method) and clears
 *   the non-finite report.
 * Errors: KPS_EINVAL (NULL, buffer too small, not a checkpoint, another
 * storage type or batch), KPS_ECUDA. */
kps_status kps_solver_state_bytes(const kps_solver *solver, int64_t *bytes);
kps_status kps_solver_save(kps_solver *solver, void *host, int64_t bytes, void *stream);
kps_status kps_solver_load(kps_solver *solver, const void *host, int64_t bytes, void *stream);
/* Iterations run since the last reset (host count). */
kps_status kps_solver_iterations(const kps_solver *solver, int64_t *iters);
/* FP64 average strategies (device, batch player layouts; either may be
 * NULL): sequence form xsum / sum_t t, or with `behavioural` != 0 the
 * behavioural strategy x[sigma] / x[parent] (uniform at unreached nodes).
 * Before any iteration: the current strategies. */
kps_status kps_solver_average(kps_solver *solver, int32_t behavioural, double *x, double *y, void *stream);
/* The current (last) sequence-form strategies x, y in the storage type
 * (device, batch player layouts; either may be NULL). */
kps_status kps_solver_strategy(kps_solver *solver, void *x, void *y, void *stream);
/* Per game (device arrays of n doubles): exploitability of the averages
 * (BR1(ybar) + BR2(xbar)) / 2 / pot0, in units of the initial pot (Sec. 5),
 * and the best-response values BR1, BR2 (may be NULL).  FP64 products and
 * best responses.  Asynchronous on `stream`. */
kps_status kps_solver_exploitability(kps_solver *solver, double *expl, double *br1, double *br2, void *stream);
/* The same quantity estimated cheaply for stopping tests: averages and
 * products in FP32 (tensor-memory kernels), best-response sums in FP64.
 * Differs from kps_solver_exploitability by the FP32 rounding of the
 * products (about 1e-6 of the values); confirm a stop with the FP64 call. */
kps_status kps_solver_exploitability_estimate(kps_solver *solver, double *expl, void *stream);

/* ---- Learned warm start ----------------------------------------------------
 * Not in the paper.  A 3-layer perceptron (BF16 weights, FP32 master copy,
 * activations and accumulation) maps a query (game, player, decision node,
 * hand) of a batch to a behavioural strategy at that node; a solver started
 * from its predictions (kps_solver_warm_start) needs fewer iterations.
 * Queries of a batch are numbered game by game, player 1's nodes then
 * player 2's, hands in library order within a node. */
#define KPS_WARM_DIN 1232   /* feature row length                            */
#define KPS_WARM_DOUT 12    /* outputs per row: actions of a node (masked)   */

/* Number of queries of the batch (builds its feature tables on first use).
 * KPS_ENOTSUP if a player has more than 32 decision nodes. */
kps_status kps_warm_num_queries(kps_batch *batch, int64_t *n);
/* Feature rows X [nq][KPS_WARM_DIN] (device FP32) and action counts nact
 * [nq] (device, may be NULL) of queries qidx[0..nq) (device int64), or of
 * q0 .. q0+nq-1 when qidx is NULL.  Row layout: board one-hot (52), the
 * opponent's belief mass over 1081 strength bins, node one-hot / player /
 * actions / depth (40), hand strength position / tie size / own belief /
 * card two-hot (56), padding (3). */
kps_status kps_warm_features(kps_batch *batch, const int64_t *qidx, int64_t q0, int32_t nq, float *X,
                             int32_t *nact, void *stream);
/* Training targets from a solver's FP64 average strategies (batch layouts,
 * kps_solver_average): T [nq][KPS_WARM_DOUT] the behavioural strategy at
 * the query's node, w [nq] = reach of the node's parent sequence in the
 * sequence-form average x1/x2 (1 at a root; 1 everywhere if x1/x2 are NULL)
 * times the hand's normalised belief. */
kps_status kps_warm_targets(kps_batch *batch, const double *beh1, const double *beh2, const double *x1,
                            const double *x2, const int64_t *qidx, int64_t q0, int32_t nq, float *T, float *w,
                            void *stream);
/* Writes predictions P [nq][KPS_WARM_DOUT] into behavioural strategies
 * beh1 / beh2 (device FP32, batch layouts) at the queries' nodes and hands. */
kps_status kps_warm_scatter(kps_batch *batch, const float *P, const int64_t *qidx, int64_t q0, int32_t nq,
                            float *beh1, float *beh2, void *stream);

typedef struct kps_mlp kps_mlp;

/* The network's behavioural strategy at EVERY query of the batch, written
 * into beh1 / beh2 (device FP32, batch layouts) in one fused pass: the first
 * layer from its game, node and hand parts (the game and node parts computed
 * once per game / node), layers 2 and 3 on the tensor cores (tcgen05.mma,
 * BF16 operands, FP32 accumulators in tensor memory) with BF16
 * activations, the masked softmax, the scatter.  Needs din = KPS_WARM_DIN,
 * width 256, dout <= 16 (KPS_ENOTSUP otherwise).  Allocates temporaries and
 * synchronises `stream`.  Agrees with kps_warm_features + kps_mlp_forward +
 * kps_warm_scatter up to the BF16 rounding of the activations. */
kps_status kps_warm_predict(kps_batch *batch, kps_mlp *mlp, float *beh1, float *beh2, void *stream);
/* Layers din -> width -> width -> dout (dout <= 32), ReLU, He-normal
 * weights from `seed`, zero biases. */
kps_status kps_mlp_create(int32_t din, int32_t width, int32_t dout, uint64_t seed, kps_mlp **out);
kps_status kps_mlp_destroy(kps_mlp *mlp);
/* Parameter count: W1 [din][width], b1, W2 [width][width], b2,
 * W3 [width][dout], b3, in this order in every flat array below. */
kps_status kps_mlp_num_params(const kps_mlp *mlp, int64_t *n);
/* Host copy of the FP32 parameters (which = 0) or of the last gradients
 * (which = 1); kps_mlp_set writes the parameters (and their BF16 copy). */
kps_status kps_mlp_get(const kps_mlp *mlp, int32_t which, float *host);
kps_status kps_mlp_set(kps_mlp *mlp, const float *host);
/* P [rows][dout] = softmax over the first nact[r] outputs of row r
 * (device).  Products read the BF16 weights, accumulate in FP32. */
kps_status kps_mlp_forward(kps_mlp *mlp, const float *X, int32_t rows, const int32_t *nact, float *P,
                           void *stream);
/* Gradients of L = -sum_r w_r sum_{a < nact_r} T[r][a] log P[r][a] / wsum
 * into the network's gradient buffer; *loss (device float, may be NULL)
 * receives L. */
kps_status kps_mlp_gradients(kps_mlp *mlp, const float *X, int32_t rows, const int32_t *nact, const float *T,
                             const float *w, float wsum, float *loss, void *stream);
/* One Adam step with the last gradients (FP32 master weights, then BF16). */
kps_status kps_mlp_adam(kps_mlp *mlp, float lr, float beta1, float beta2, float eps, void *stream);
/* Checkpoint of a network in a caller-owned host buffer of
 * kps_mlp_state_bytes bytes: a header (format version, layer sizes, Adam's
 * step count) then the FP32 parameters and Adam's first and second moments,
 * so that training resumed after kps_mlp_load takes the same steps, bit for
 * bit, as training that never stopped.  Both calls synchronise the device.
 * kps_mlp_load needs a network of the same layer sizes and rebuilds the
 * BF16 weight copy.  Errors: KPS_EINVAL (NULL, buffer too small, not a
 * checkpoint, other layer sizes), KPS_ECUDA. */
kps_status kps_mlp_state_bytes(const kps_mlp *mlp, int64_t *bytes);
kps_status kps_mlp_save(const kps_mlp *mlp, void *host, int64_t bytes);
kps_status kps_mlp_load(kps_mlp *mlp, const void *host, int64_t bytes);

/* A * y for BF16 or FP16 vectors without any device allocation.  The paper
 * has no counterpart: this is a service for callers that must not allocate
 * device memory while they run, such as serving loops that reserve all of
 * the GPU's memory up front for their own pool, real-time loops that cannot
 * afford cudaMalloc's implicit device synchronisation, or code that shares
 * a memory budget with other tenants and must not grow it.  kps_matvec_A
 * with BF16/FP16 storage allocates an FP32 partial-result buffer (and a tile
 * list) on first use; this variant uses instead a statically reserved device
 * array of KPS_STATIC_SCRATCH_FLOATS floats plus 64 KiB, which every device
 * that loads the library holds until the process exits.
 *   - Requires the game's tables on the current device (kps_game_upload or
 *     any earlier product call); KPS_EINVAL otherwise.
 *   - batch * n1 * hs must not exceed KPS_STATIC_SCRATCH_FLOATS; larger
 *     requests fail with KPS_EINVAL and a message giving both numbers.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress).
 *   - The call cannot be recorded into a CUDA graph: on a stream that is
 *     capturing it returns KPS_EINVAL and queues nothing.
 *   - All calls share the array: calls that overlap on the GPU (other
 *     streams, other threads) race and produce wrong results.  Every element
 *     the kernel reads is written by the same call first, so nothing needs to
 *     be cleared between calls.
 * Layouts, dtypes and results as kps_matvec_A (dt must be KPS_BF16 or
 * KPS_F16).  Calls no cudaMalloc, cudaFree or allocating library routine. */
#define KPS_STATIC_SCRATCH_FLOATS 4194304
kps_status kps_matvec_A_static_scratch(kps_game *game, const void *y, void *out, int32_t batch,
                                       kps_dtype dt, void *stream);

/* ---- Technique B's explicit factors (Sec. 4) ----------------------------
 * The paper's own route to A*y: A = Ahat + U M^-1 V^T (Technique B
 * proposition, before the postprocessing step), the four factors
 * materialised as sparse matrices and applied with sparse products and a
 * triangular solve.  The library's kps_matvec_A computes the same product
 * without materialising anything; these calls exist to compare the two.
 *
 * Layout of the factors (the vector layout above; hands in library order):
 *   rows of A (and of Ahat, U)    s1 * hs + h1       R = n1 * hs
 *   columns of A (and of V^T)     s2 * hs + h2       C = n2 * hs
 *   inner dimension (U, M, V^T)   s1 * hs + h  for the I (x) D block,
 *                                 n1 * hs + s1 for the identity block,
 *                                 m = n1 * hs + n1
 *   Ahat = -F (x) (Lambda1 Hx Lambda2)
 *   U    = [I (x) Lambda1 | I (x) lambda1]
 *   M    = diag(I (x) D, I), D lower bidiagonal with 1 on the diagonal and
 *          -1 below it (stored with its unit diagonal; rows of padding
 *          hands hold the diagonal alone)
 *   V^T  = [S (x) (Y Lambda2) ; F (x) lambda2^T],  Y = D W
 * with F, S the fold and showdown payoff matrices of the skeleton, W the
 * win/lose sign with zeros on card overlaps, Hx the card-overlap indicator
 * and lambda = mu / sqrt(beta) (the paper's hand-major D (x) I and
 * (Lambda2 Y^T) (x) S^T in this sequence-major order).
 *
 * kps_tb_create builds the factors on the host (no GPU needed); *out
 * receives a new object that refers to `game` (which must outlive it).
 * Errors: KPS_EINVAL (NULL), KPS_ENOMEM, KPS_ENOTSUP (a factor with more
 * than 2^31 nonzeros). */
typedef struct kps_tb kps_tb;
kps_status kps_tb_create(const kps_game *game, kps_tb **out);
kps_status kps_tb_destroy(kps_tb *tb);

/* sizes[0..6] = R, C, m, nnz(Ahat), nnz(U), nnz(M), nnz(V).  nnz(M)
 * excludes the diagonal of padding rows, so the four nonzero counts equal
 * kps_info's Technique B counts before postprocessing. */
kps_status kps_tb_sizes(const kps_tb *tb, int64_t *sizes);

/* Host copy of one factor in CSR (columns ascending within a row, FP64
 * values): which = 0 Ahat, 1 U, 2 M, 3 V^T.  shape[0..2] = rows, columns,
 * stored nonzeros; rowptr[rows + 1], col[nnz], val[nnz] (caller-owned; any
 * of the four pointers may be NULL to skip it). */
kps_status kps_tb_export(const kps_tb *tb, int which, int64_t *shape, int32_t *rowptr, int32_t *col, double *val);

/* out = (Ahat + U M^-1 V^T) y on the GPU for `batch` player-2 vectors y
 * (device, [batch][n2][hs]) into player-1 vectors out (device,
 * [batch][n1][hs]); dt = KPS_F32 or KPS_F64 (values and arithmetic).
 * backend 0: this library's kernels (a CSR times dense-matrix product and,
 *   for M^-1, prefix sums over the hands of each player-1 sequence);
 * backend 1: cuSPARSE (SpMM for V^T, Ahat and U; SpSM for M).
 * The factors are uploaded on the first call; a workspace of
 * 2 * batch * m values is kept between calls.  Errors: KPS_EINVAL,
 * KPS_ENOTSUP (other dtypes), KPS_ENOMEM, KPS_ECUDA (CUDA or cuSPARSE
 * failure, with the library's message). */
kps_status kps_tb_matvec(kps_tb *tb, const void *y, void *out, int32_t batch, kps_dtype dt, int32_t backend,
                         void *stream);

/* Thread-local description of the last failure ("" if none). */
const char *kps_last_error(void);

/* Synchronises `stream` and reports device-side failures of the launches
 * since the previous call: KPS_ETIMEOUT when a bounded wait of the
 * TMA-staged kernel (an mbarrier its copies complete; limit 2 s) gave up,
 * in which case the products of those launches are not valid (the flag is
 * then cleared and the context stays usable); KPS_ECUDA on a CUDA error.
 * The wait limit turns a copy that never completes into this status
 * instead of a hang.  Test hook: with the environment variable
 * KPS_TEST_STALL_WAIT=1 at launch, one barrier per CTA of that kernel
 * expects 16 bytes more than its copies bring, so its wait runs out. */
kps_status kps_device_status(void *stream);

/* Library version string. */
const char *kps_version(void);

#ifdef __cplusplus
}
#endif
#endif /* KPS_H */
