/*
 * kps_oracle.h -- plain CPU oracle for the Kronecker-structured payoff
 * matrix of a poker river endgame (Farina & Sandholm, "Fast Payoff Matrix
 * Sparsification Techniques for Structured Extensive-Form Games", AAAI-22).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header, table or helper with the CUDA product path.
 *
 * Everything is FP64 and written for clarity, not speed: the payoff matrix is
 * built from its definition (Sec. 2: A[s1,s2] = sum over terminals z of
 * u(z) * c(z)), the chance distribution pi(h1,h2) of Sec. 3 and the
 * skeleton betting tree of Fig. 1.
 *
 * Layout conventions used by this oracle (its own, independent of the
 * library's):
 *   - hands are in CANONICAL order: the deck minus the board in increasing
 *     card id (card id = rank*suits + suit); 1-card hands are single cards,
 *     2-card hands are the pairs (a<b) in lexicographic order;
 *   - strategy and gradient vectors are [sequence][hand] (hand fastest);
 *   - the dense payoff matrix follows the paper's block layout: row index
 *     h1*n1 + s1, column index h2*n2 + s2 (Sec. 3, block A_{h1,h2}).
 */
#ifndef KPS_ORACLE_H
#define KPS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_BETS 8
#define ORC_MAX_BOARD 8

typedef struct {
    int ranks, suits;          /* deck = ranks*suits cards                    */
    int cards_per_hand;        /* 1 or 2                                      */
    int nboard;                /* number of public cards                      */
    int board[ORC_MAX_BOARD];  /* card ids                                    */
    double stack[2];           /* chips behind at the start of the endgame    */
    double contrib0[2];        /* pot contribution at the start               */
    int nbet;                  /* number of bet/raise pot fractions           */
    double bet_frac[ORC_MAX_BETS];
    int raise_cap;             /* max aggressive actions in the round; <0 = none */
    int allow_allin;           /* explicit all-in action                      */
    const double *mu1, *mu2;   /* beliefs per canonical hand; NULL = uniform  */
    const int *strength;       /* per canonical hand, higher = stronger       */
    /* Optional per-player menu (appendix "Libratus' betting abstraction"):
     * when use_menu, player p in situation k bets the fractions
     * menu_frac[p][k][0..menu_nbet[p][k]-1] instead of bet_frac.  Situations:
     * 0 first action of the round, 1 after a check, 2 facing the first bet,
     * 3 facing one raise, 4 facing two or more raises. */
    int use_menu;
    int menu_nbet[2][5];
    double menu_frac[2][5][ORC_MAX_BETS];
} orc_spec;

typedef struct orc_game orc_game;

/* Build the skeleton, the hand list and pi.  Returns NULL on invalid input. */
orc_game *orc_build(const orc_spec *spec);
void orc_free(orc_game *g);

/* info[0..9] = H, n1, n2, T, T_fold, T_showdown, nnodes, ncards_left,
 *              nplayer_nodes1, nplayer_nodes2 */
void orc_info(const orc_game *g, int *info);
double orc_beta(const orc_game *g);
double orc_pot0(const orc_game *g);

/* Canonical hand list: cards[h*k + j]. */
void orc_hands(const orc_game *g, int *cards);

/* Terminal list in depth-first order.  kind: 0 fold, 1 showdown.
 * folder: 0/1 for fold terminals, -1 otherwise.  s1, s2: the last sequence
 * of each player on the path (-1 = empty sequence).  c1, c2: contributions. */
void orc_terminals(const orc_game *g, int *s1, int *s2, int *kind, int *folder,
                   double *c1, double *c2);

/* Per player p: for each of its sequences, the player node it belongs to,
 * the parent sequence of that node (-1 = empty) and the action code
 * (0 fold, 1 check/call, 2 aggressive).  nodes_nact[i] = actions of node i. */
void orc_sequences(const orc_game *g, int p, int *seq_node, int *seq_parent,
                   int *seq_action, double *seq_amount, int *nodes_nact);

/* Terminal reached by an action path; path tokens: 'f' fold, 'c' check/call,
 * 'b' the k-th smallest aggressive amount is given as a digit after 'b'
 * ("b0", "b1", ...), 'a' the largest aggressive amount (all-in).  Tokens are
 * separated by spaces.  Returns the terminal index or -1. */
int orc_find_terminal(const orc_game *g, const char *path);

/* Dense payoff matrix for player 1 (Sec. 2 definition), paper block layout,
 * (H*n1) x (H*n2) doubles, row-major. */
int orc_dense_A(const orc_game *g, double *A);

/* Direct products by summation over terminals and hand pairs.
 * y: [batch][n2][H], out: [batch][n1][H]  (A y)
 * x: [batch][n1][H], out: [batch][n2][H]  (A^T x) */
void orc_matvec_A(const orc_game *g, const double *y, double *out, int batch,
                  int nthreads);
void orc_matvec_AT(const orc_game *g, const double *x, double *out, int batch,
                   int nthreads);
/* Selected entries of A y_b: for each k, out[k] = (A y_{b[k]})[s[k]][h[k]]. */
void orc_matvec_A_entries(const orc_game *g, const double *y, int nent,
                          const int *b, const int *s, const int *h, double *out);
void orc_matvec_AT_entries(const orc_game *g, const double *x, int nent,
                           const int *b, const int *s, const int *h, double *out);

/* Brute-force expected payoff of player 1 by walking the full game tree
 * (chance deal, then the skeleton) with behavioural strategies beh1 [n1][H]
 * and beh2 [n2][H] (probability of each sequence's action at its node). */
double orc_bruteforce_value(const orc_game *g, const double *beh1,
                            const double *beh2);

/* Behavioural -> sequence form for player p: [n_p][H] -> [n_p][H]. */
void orc_seqform(const orc_game *g, int p, const double *beh, double *x);

/* Technique B (Sec. 4): dense explicit factors in the strength-sorted hand
 * order for small games.  Writes nnz counts:
 * cnt[0..4]  = nnz(A), nnz(Ahat), nnz(U), nnz(M), nnz(V)   before postprocessing
 * cnt[5..8]  = nnz(Ahat), nnz(U), nnz(M), nnz(V)           after postprocessing
 * and returns max |A - (Ahat + U M^-1 V^T)| (entrywise), both sides in the
 * sorted order, or -1 if the game is too large (H*max(n1,n2) > 4096). */
double orc_technique_b(const orc_game *g, long long *cnt);

/* Counts only (no dense matrices); valid for any size. Same cnt layout. */
void orc_technique_b_counts(const orc_game *g, long long *cnt);

/* Noise floor of regret matching for player p: eps * V_p, V_p a bound on
 * the magnitude of p's counterfactual values (see kps_oracle.c). */
#define ORC_REGRET_EPS (1.0 / 1099511627776.0)   /* 2^-40 */
double orc_regret_floor(const orc_game *g, int p, double eps);

/* RM+ (CFR+-style) alternating self-play with linearly weighted averages.
 * Regret matching plays uniformly at a node whose regret sum is at most
 * orc_regret_floor(g, p, ORC_REGRET_EPS) (exact zero in textbook RM+).
 * x0, y0: initial behavioural strategies [n][H] (NULL = uniform).
 * Runs iters iterations; writes average behavioural strategies (optional,
 * may be NULL) and returns the exploitability of the average in units of
 * the initial pot.  trace (optional, length iters) gets the exploitability
 * of the average after every iteration when trace_every > 0 and
 * (t % trace_every == 0), else 0. */
double orc_rmplus(const orc_game *g, int iters, const double *beh1_0,
                  const double *beh2_0, double *avg_beh1, double *avg_beh2,
                  double *trace, int trace_every);

/* The same loop started warm: regrets R_p = kappa * V_p * b_p (V_p =
 * orc_regret_floor(g, p, 1.0), so regret matching returns b_p), the initial
 * strategy counted as played at iterations 1..t0 (weight t0 (t0 + 1) / 2 in
 * the linear average), then iterations t0 + 1 .. t0 + iters.  kappa = 0,
 * t0 = 0 is orc_rmplus.  trace[k] belongs to iteration t0 + k + 1. */
double orc_rmplus_warm(const orc_game *g, int iters, const double *beh1_0, const double *beh2_0,
                       double kappa, int t0, double *avg_beh1, double *avg_beh2, double *trace,
                       int trace_every);

/* orc_rmplus from uniform strategies with the noise floor eps * V_p of
 * regret matching given explicitly (eps = 0: textbook RM+, uniform only at
 * an exact zero regret sum). */
double orc_rmplus_eps(const orc_game *g, int iters, double eps, double *avg_beh1, double *avg_beh2);

/* Discounted CFR (the solver the paper runs, Sec. 5; Brown & Sandholm's
 * DCFR): alternating updates from uniform strategies; on iteration t the
 * instantaneous regret q - v is added and a cumulative regret is multiplied
 * by t^alpha / (t^alpha + 1) when positive, t^beta / (t^beta + 1) otherwise;
 * regret matching on the positive parts (uniform at or below the noise
 * floor); iteration t's strategy enters the average with weight t^gamma. */
double orc_dcfr(const orc_game *g, int iters, double alpha, double beta, double gamma,
                double *avg_beh1, double *avg_beh2, double *trace, int trace_every);

/* Best-response values: br1 = max_x x^T A y, br2 = max_y -x^T A y for
 * sequence-form x [n1][H], y [n2][H].  Returns (br1 + br2)/2/pot0. */
double orc_exploitability(const orc_game *g, const double *x, const double *y,
                          double *br1, double *br2);

/* x^T A y for sequence-form vectors. */
double orc_value(const orc_game *g, const double *x, const double *y);

/* ---- Turn endgames (kps_turn_oracle.c; end of Sec. 3) --------------------
 * The turn betting round, then at every ending that is not a fold a chance
 * node over the river card and the river betting round.  Hands over the
 * deck minus the board (canonical order); strength[r * H + h] is hand h's
 * showdown strength with river card r (higher is stronger; entries for
 * cards on the board or in the hand are not read).  Vectors are
 * [sequence][hand]: the turn round's sequences, then one block per
 * (ending, river card), endings in depth-first order, cards ascending. */
typedef struct {
    int ranks, suits, cards_per_hand;
    int nboard;
    int board[ORC_MAX_BOARD];
    double stack[2], contrib0[2];
    int nbet_t;                      /* turn round */
    double bet_frac_t[ORC_MAX_BETS];
    int raise_cap_t, allow_allin_t;
    int nbet_r;                      /* river round */
    double bet_frac_r[ORC_MAX_BETS];
    int raise_cap_r, allow_allin_r;
    const double *mu1, *mu2;         /* per hand; NULL = uniform */
    const int *strength;             /* [ranks*suits][H] */
} orc_turn_spec;

typedef struct orc_turn orc_turn;

/* NULL on invalid input or when a non-fold ending of the turn leaves a
 * player all in (no river betting). */
orc_turn *orc_turn_build(const orc_turn_spec *spec);
void orc_turn_free(orc_turn *g);
/* info[0..8] = H, n1, n2, T, turn endings, river blocks, turn sequences of
 * player 1 and 2, cards left after the board. */
void orc_turn_info(const orc_turn *g, int *info);
double orc_turn_beta(const orc_turn *g);
int orc_turn_disjoint(const orc_turn *g, int h1, int h2);
/* Direct products: transpose 0: out = A v (v [batch][n2][H], out
 * [batch][n1][H]); 1: out = A^T v. */
void orc_turn_matvec(const orc_turn *g, const double *v, double *out, int batch, int transpose, int nthreads);
/* Selected entries of the product (out[k] = entry (s[k], h[k]) of vector b[k]). */
void orc_turn_entries(const orc_turn *g, const double *v, int nent, const int *b, const int *s, const int *h,
                      int transpose, double *out);
/* Expected payoff of player 1 by walking the whole tree (deal, turn round,
 * river card, river round) with behavioural strategies [n_p][H]. */
double orc_turn_bruteforce(const orc_turn *g, const double *beh1, const double *beh2);
/* parent[s]; for every sequence the id of its node's first sequence and the
 * node's action count (either array may be NULL). */
void orc_turn_sequences(const orc_turn *g, int p, int *parent, int *node_of_seq, int *nact_of_seq);
void orc_turn_seqform(const orc_turn *g, int p, const double *beh, double *x);

#ifdef __cplusplus
}
#endif
#endif
