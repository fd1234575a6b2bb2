/*
 * kps_turn_oracle.c -- plain CPU oracle for turn endgames (Farina &
 * Sandholm, AAAI-22, end of Sec. 3): the turn betting round, then, at every
 * ending of that round that is not a fold, a chance node over the river card
 * and the river betting round.  Because the river card is public, the payoff
 * matrix is block diagonal with one river block per (ending, river card).
 *
 * TEST INFRASTRUCTURE ONLY (see kps_oracle.h).  FP64, written for clarity.
 * This file builds the two-round game tree itself; it shares nothing with the
 * library and, inside the oracle, nothing with the river builder of
 * kps_oracle.c (the tests compare the two).
 *
 * Definitions (readings T1-T5 of the design notes):
 *   - hands: 1- or 2-card hands from the deck minus the 4-card turn board,
 *     canonical order as in kps_oracle.h; beliefs mu_p per hand;
 *   - chance deal pi(h1,h2) = mu1(h1) mu2(h2) / beta for disjoint hands,
 *     beta = sum of mu1 mu2 over disjoint pairs (Sec. 3); river card r
 *     uniform over the cards in neither hand nor on the board: probability
 *     1 / (N - 2k) with N the cards left after the board (T1);
 *   - betting: each round as the river skeleton (kps_oracle.h), player 1
 *     first in both rounds, the river starting from the turn ending's
 *     contributions with the chips left behind (T2); an ending where a
 *     player has no chips left behind is rejected (no river betting; T3);
 *   - payoffs: a fold pays the folder's contribution; a river showdown pays
 *     the sign of strength[r][h1] - strength[r][h2] times the matched
 *     contribution (higher is stronger, ties pay 0);
 *   - sequences (the layout of every vector, T4): the turn round's sequences
 *     in depth-first pre-order (a node's actions numbered when it is first
 *     reached), then one block per (ending, river card): endings in
 *     depth-first order of the turn round, river cards ascending, each
 *     block's sequences in depth-first pre-order; vectors are
 *     [sequence][hand], hands in canonical order.
 *
 * A[(h1,s1),(h2,s2)] = sum over terminals t whose last sequences are
 * (s1,s2) of pi(h1,h2) P(r_t | h1,h2) u_t(h1,h2), P = 1 for turn folds.
 */
#include "kps_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TMAXA (ORC_MAX_BETS + 3)

typedef struct {
    int player;            /* 0/1 acting; -1 terminal; -2 continuation (turn ending) */
    double c[2];
    int naggr, prev_check;
    int nact;
    int child[TMAXA];
    int act_code[TMAXA];
    int seq[TMAXA];
    int last_seq[2];
    int river;             /* river card on the path, -1 in the turn round    */
    int tkind, folder;
    int kid0;              /* continuation node: its chance children kids[kid0 .. kid0 + nact) */
} tnode;

struct orc_turn {
    orc_turn_spec sp;
    int H, k, N;               /* hands, cards per hand, cards left after the board */
    int ncard;
    int *cards;                /* H*k */
    double *mu[2];
    int *strength;             /* [ncard][H] */
    double beta;
    tnode *nodes;
    int nn, cap;
    int n[2];
    int *seq_parent[2], *seq_node_nact[2];
    int T;
    int *term;                 /* tree node of each terminal */
    int nend;                  /* turn endings that are not folds */
    int nturn[2];              /* sequences of the turn round */
    int nblocks;
    int *kids;                 /* chance children of the continuation nodes */
    int err;
};

static int tnew(orc_turn *g)
{
    if (g->nn == g->cap) {
        g->cap = g->cap ? 2 * g->cap : 256;
        g->nodes = (tnode *)realloc(g->nodes, (size_t)g->cap * sizeof(tnode));
    }
    memset(&g->nodes[g->nn], 0, sizeof(tnode));
    return g->nn++;
}

static double tmin(double a, double b) { return a < b ? a : b; }

/* The betting rules of one round (same rules as the river skeleton):
 * facing a larger contribution fold, call, raise; otherwise check or bet; a
 * bet of fraction f matches first and then adds f times the pot; amounts at
 * or above the effective stack are all-in (merged with an explicit all-in). */
static int round_actions(const orc_turn *g, const tnode *nd, int river, int *code, double *amt)
{
    const int nbet = river ? g->sp.nbet_r : g->sp.nbet_t;
    const double *frac = river ? g->sp.bet_frac_r : g->sp.bet_frac_t;
    const int cap = river ? g->sp.raise_cap_r : g->sp.raise_cap_t;
    const int allin = river ? g->sp.allow_allin_r : g->sp.allow_allin_t;
    int p = nd->player, o = 1 - p, na = 0, nag = 0;
    double maxp = g->sp.contrib0[p] + g->sp.stack[p], maxo = g->sp.contrib0[o] + g->sp.stack[o];
    double eff = tmin(maxp, maxo), ag[TMAXA];
    int can = cap < 0 || nd->naggr < cap;
    if (nd->c[p] < nd->c[o]) {
        code[na] = 0; amt[na++] = nd->c[p];
        code[na] = 1; amt[na++] = tmin(nd->c[o], maxp);
        if (can && eff > nd->c[o]) {
            for (int i = 0; i < nbet; i++) {
                double a = nd->c[o] + frac[i] * 2.0 * nd->c[o];
                ag[nag++] = a >= eff ? eff : a;
            }
            if (allin) ag[nag++] = eff;
        }
    } else {
        code[na] = 1; amt[na++] = nd->c[p];
        if (can && eff > nd->c[p]) {
            double pot = nd->c[0] + nd->c[1];
            for (int i = 0; i < nbet; i++) {
                double a = nd->c[p] + frac[i] * pot;
                ag[nag++] = a >= eff ? eff : a;
            }
            if (allin) ag[nag++] = eff;
        }
    }
    for (int i = 1; i < nag; i++)
        for (int j = i; j > 0 && ag[j] < ag[j - 1]; j--) { double t = ag[j]; ag[j] = ag[j - 1]; ag[j - 1] = t; }
    for (int i = 0; i < nag; i++) {
        if (i > 0 && ag[i] == ag[i - 1]) continue;
        code[na] = 2; amt[na++] = ag[i];
    }
    return na;
}

/* Depth-first construction of one betting round below node id.  Ends of the
 * turn round that are not folds become continuation nodes (player -2). */
static void grow(orc_turn *g, int id, int river)
{
    tnode *nd = &g->nodes[id];
    if (nd->player < 0) return;
    int code[TMAXA];
    double amt[TMAXA];
    int na = round_actions(g, nd, river, code, amt);
    int p = nd->player, o = 1 - p;
    nd->nact = na;
    for (int a = 0; a < na; a++) {
        g->nodes[id].act_code[a] = code[a];
        g->nodes[id].seq[a] = g->n[p]++;
    }
    for (int a = 0; a < na; a++) {
        int c = tnew(g);
        tnode *pa = &g->nodes[id], *ch = &g->nodes[c];
        pa->child[a] = c;
        ch->c[0] = pa->c[0];
        ch->c[1] = pa->c[1];
        ch->c[p] = amt[a];
        ch->last_seq[0] = pa->last_seq[0];
        ch->last_seq[1] = pa->last_seq[1];
        ch->last_seq[p] = pa->seq[a];
        ch->naggr = pa->naggr;
        ch->river = pa->river;
        if (code[a] == 0) {
            ch->player = -1; ch->tkind = 0; ch->folder = p;
        } else if (code[a] == 1) {
            if (pa->c[p] < pa->c[o] || pa->prev_check) {
                ch->player = river ? -1 : -2; ch->tkind = 1; ch->folder = -1;
            } else {
                ch->player = o; ch->prev_check = 1;
            }
        } else {
            ch->player = o; ch->naggr = pa->naggr + 1;
        }
        grow(g, c, river);
    }
}

/* Continuation nodes of the turn round, depth-first order. */
static void collect_ends(const orc_turn *g, int id, int *out, int *n)
{
    const tnode *nd = &g->nodes[id];
    if (nd->player == -2) { out[(*n)++] = id; return; }
    for (int a = 0; a < nd->nact; a++) collect_ends(g, nd->child[a], out, n);
}

orc_turn *orc_turn_build(const orc_turn_spec *sp)
{
    if (!sp || (sp->cards_per_hand != 1 && sp->cards_per_hand != 2)) return NULL;
    if (sp->nboard < 1 || sp->nboard > ORC_MAX_BOARD || !sp->strength) return NULL;
    if (sp->nbet_t < 0 || sp->nbet_t > ORC_MAX_BETS || sp->nbet_r < 0 || sp->nbet_r > ORC_MAX_BETS) return NULL;
    orc_turn *g = (orc_turn *)calloc(1, sizeof(orc_turn));
    g->sp = *sp;
    g->k = sp->cards_per_hand;
    g->ncard = sp->ranks * sp->suits;
    int *on = (int *)calloc((size_t)g->ncard, sizeof(int));
    for (int i = 0; i < sp->nboard; i++) {
        if (sp->board[i] < 0 || sp->board[i] >= g->ncard || on[sp->board[i]]) { free(on); free(g); return NULL; }
        on[sp->board[i]] = 1;
    }
    int *left = (int *)malloc((size_t)g->ncard * sizeof(int)), nl = 0;
    for (int c = 0; c < g->ncard; c++) if (!on[c]) left[nl++] = c;
    g->N = nl;
    g->H = g->k == 1 ? nl : nl * (nl - 1) / 2;
    g->cards = (int *)malloc((size_t)g->H * g->k * sizeof(int));
    for (int i = 0, h = 0; i < nl; i++) {
        if (g->k == 1) { g->cards[h++] = left[i]; continue; }
        for (int j = i + 1; j < nl; j++) { g->cards[2 * h] = left[i]; g->cards[2 * h + 1] = left[j]; h++; }
    }
    free(left);
    free(on);
    if (g->N - 2 * g->k < 1) { orc_turn_free(g); return NULL; }
    for (int p = 0; p < 2; p++) {
        g->mu[p] = (double *)malloc((size_t)g->H * sizeof(double));
        const double *src = p == 0 ? sp->mu1 : sp->mu2;
        for (int h = 0; h < g->H; h++) g->mu[p][h] = src ? src[h] : 1.0;
    }
    g->strength = (int *)malloc((size_t)g->ncard * g->H * sizeof(int));
    memcpy(g->strength, sp->strength, (size_t)g->ncard * g->H * sizeof(int));
    g->sp.mu1 = g->sp.mu2 = NULL;
    g->sp.strength = NULL;
    g->beta = 0.0;
    for (int h1 = 0; h1 < g->H; h1++)
        for (int h2 = 0; h2 < g->H; h2++)
            if (orc_turn_disjoint(g, h1, h2)) g->beta += g->mu[0][h1] * g->mu[1][h2];
    if (!(g->beta > 0.0)) { orc_turn_free(g); return NULL; }

    /* turn round */
    int root = tnew(g);
    g->nodes[root].player = 0;
    g->nodes[root].c[0] = sp->contrib0[0];
    g->nodes[root].c[1] = sp->contrib0[1];
    g->nodes[root].last_seq[0] = g->nodes[root].last_seq[1] = -1;
    g->nodes[root].river = -1;
    grow(g, root, 0);
    g->nturn[0] = g->n[0];
    g->nturn[1] = g->n[1];
    int *ends = (int *)malloc((size_t)g->nn * sizeof(int));
    collect_ends(g, root, ends, &g->nend);
    /* river rounds: ending by ending, river card by river card */
    g->kids = (int *)malloc((size_t)(g->nend > 0 ? g->nend : 1) * g->ncard * sizeof(int));
    for (int e = 0; e < g->nend; e++) {
        const tnode z = g->nodes[ends[e]];
        for (int p = 0; p < 2; p++)
            if (!(g->sp.contrib0[p] + g->sp.stack[p] > z.c[p])) g->err = 1;   /* all-in ending (T3) */
        g->nodes[ends[e]].kid0 = e * g->ncard;
        g->nodes[ends[e]].nact = 0;
        for (int r = 0; r < g->ncard; r++) {
            int onb = 0;
            for (int i = 0; i < sp->nboard; i++) onb |= sp->board[i] == r;
            if (onb) continue;
            int c = tnew(g);
            tnode *en = &g->nodes[ends[e]];
            g->kids[en->kid0 + en->nact++] = c;   /* chance children, card order */
            tnode *rt = &g->nodes[c];
            rt->player = 0;
            rt->c[0] = z.c[0];
            rt->c[1] = z.c[1];
            rt->last_seq[0] = z.last_seq[0];
            rt->last_seq[1] = z.last_seq[1];
            rt->river = r;
            grow(g, c, 1);
            g->nblocks++;
        }
    }
    free(ends);
    if (g->err) { orc_turn_free(g); return NULL; }
    /* terminals and sequence parents */
    g->term = (int *)malloc((size_t)g->nn * sizeof(int));
    for (int p = 0; p < 2; p++) g->seq_parent[p] = (int *)malloc((size_t)(g->n[p] + 1) * sizeof(int));
    for (int i = 0; i < g->nn; i++) {
        tnode *nd = &g->nodes[i];
        if (nd->player == -1) {
            if (nd->last_seq[0] < 0 || nd->last_seq[1] < 0) { orc_turn_free(g); return NULL; }
            g->term[g->T++] = i;
        } else if (nd->player >= 0) {
            for (int a = 0; a < nd->nact; a++) g->seq_parent[nd->player][nd->seq[a]] = nd->last_seq[nd->player];
        }
    }
    return g;
}

void orc_turn_free(orc_turn *g)
{
    if (!g) return;
    free(g->cards);
    free(g->mu[0]); free(g->mu[1]);
    free(g->strength);
    free(g->nodes);
    free(g->seq_parent[0]); free(g->seq_parent[1]);
    free(g->term);
    free(g->kids);
    free(g);
}

int orc_turn_disjoint(const orc_turn *g, int h1, int h2)
{
    for (int i = 0; i < g->k; i++)
        for (int j = 0; j < g->k; j++)
            if (g->cards[h1 * g->k + i] == g->cards[h2 * g->k + j]) return 0;
    return 1;
}

static int holds(const orc_turn *g, int h, int card)
{
    for (int i = 0; i < g->k; i++) if (g->cards[h * g->k + i] == card) return 1;
    return 0;
}

void orc_turn_info(const orc_turn *g, int *info)
{
    info[0] = g->H; info[1] = g->n[0]; info[2] = g->n[1]; info[3] = g->T;
    info[4] = g->nend; info[5] = g->nblocks; info[6] = g->nturn[0]; info[7] = g->nturn[1];
    info[8] = g->N;
}

double orc_turn_beta(const orc_turn *g) { return g->beta; }

/* Chance weight of terminal t for the deal (h1,h2): pi, times 1/(N - 2k)
 * for a river terminal when the river card is in neither hand. */
static double tweight(const orc_turn *g, const tnode *z, int h1, int h2)
{
    if (!orc_turn_disjoint(g, h1, h2)) return 0.0;
    double w = g->mu[0][h1] * g->mu[1][h2] / g->beta;
    if (z->river >= 0) {
        if (holds(g, h1, z->river) || holds(g, h2, z->river)) return 0.0;
        w /= (double)(g->N - 2 * g->k);
    }
    return w;
}

static double tpayoff(const orc_turn *g, const tnode *z, int h1, int h2)
{
    if (z->tkind == 0) return z->folder == 0 ? -z->c[0] : z->c[1];
    int s1 = g->strength[(size_t)z->river * g->H + h1], s2 = g->strength[(size_t)z->river * g->H + h2];
    return ((s1 > s2) - (s1 < s2)) * tmin(z->c[0], z->c[1]);
}

static void tmatvec(const orc_turn *g, const double *v, double *out, int transpose)
{
    int H = g->H, po = transpose ? 1 : 0;
    memset(out, 0, (size_t)g->n[po] * H * sizeof(double));
    for (int t = 0; t < g->T; t++) {
        const tnode *z = &g->nodes[g->term[t]];
        int so = z->last_seq[po], si = z->last_seq[1 - po];
        for (int ho = 0; ho < H; ho++) {
            double acc = 0.0;
            for (int hi = 0; hi < H; hi++) {
                int h1 = transpose ? hi : ho, h2 = transpose ? ho : hi;
                double w = tweight(g, z, h1, h2);
                if (w == 0.0) continue;
                acc += w * tpayoff(g, z, h1, h2) * v[(size_t)si * H + hi];
            }
            out[(size_t)so * H + ho] += acc;
        }
    }
}

void orc_turn_matvec(const orc_turn *g, const double *v, double *out, int batch, int transpose, int nthreads)
{
    size_t in = (size_t)g->n[transpose ? 0 : 1] * g->H, on = (size_t)g->n[transpose ? 1 : 0] * g->H;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = omp_get_max_threads();
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1)
#endif
    for (int b = 0; b < batch; b++) tmatvec(g, v + b * in, out + b * on, transpose);
    (void)nthreads;
}

void orc_turn_entries(const orc_turn *g, const double *v, int nent, const int *b, const int *s, const int *h,
                      int transpose, double *out)
{
    int H = g->H, po = transpose ? 1 : 0;
    size_t in = (size_t)g->n[1 - po] * H;
    for (int e = 0; e < nent; e++) {
        double acc = 0.0;
        const double *vb = v + (size_t)b[e] * in;
        for (int t = 0; t < g->T; t++) {
            const tnode *z = &g->nodes[g->term[t]];
            if (z->last_seq[po] != s[e]) continue;
            int si = z->last_seq[1 - po];
            for (int hi = 0; hi < H; hi++) {
                int h1 = transpose ? hi : h[e], h2 = transpose ? h[e] : hi;
                double w = tweight(g, z, h1, h2);
                if (w == 0.0) continue;
                acc += w * tpayoff(g, z, h1, h2) * vb[(size_t)si * H + hi];
            }
        }
        out[e] = acc;
    }
}

/* Brute force: walk the whole tree for every deal, with the chance node of
 * the river drawn card by card (the probability of a card held by a player
 * is 0, of any other 1/(N - 2k)). */
static double twalk(const orc_turn *g, int id, int h1, int h2, const double *b1, const double *b2)
{
    const tnode *nd = &g->nodes[id];
    if (nd->player == -1) return tpayoff(g, nd, h1, h2);
    if (nd->player == -2) {
        double v = 0.0;
        for (int a = 0; a < nd->nact; a++) {
            const int c = g->kids[nd->kid0 + a];
            const int r = g->nodes[c].river;
            if (holds(g, h1, r) || holds(g, h2, r)) continue;
            v += twalk(g, c, h1, h2, b1, b2) / (double)(g->N - 2 * g->k);
        }
        return v;
    }
    int hp = nd->player == 0 ? h1 : h2;
    const double *beh = nd->player == 0 ? b1 : b2;
    double v = 0.0;
    for (int a = 0; a < nd->nact; a++) {
        double pr = beh[(size_t)nd->seq[a] * g->H + hp];
        if (pr != 0.0) v += pr * twalk(g, nd->child[a], h1, h2, b1, b2);
    }
    return v;
}

double orc_turn_bruteforce(const orc_turn *g, const double *beh1, const double *beh2)
{
    double v = 0.0;
    for (int h1 = 0; h1 < g->H; h1++)
        for (int h2 = 0; h2 < g->H; h2++) {
            if (!orc_turn_disjoint(g, h1, h2)) continue;
            v += g->mu[0][h1] * g->mu[1][h2] / g->beta * twalk(g, 0, h1, h2, beh1, beh2);
        }
    return v;
}

void orc_turn_sequences(const orc_turn *g, int p, int *parent, int *node_of_seq, int *nact_of_seq)
{
    for (int s = 0; s < g->n[p]; s++) parent[s] = g->seq_parent[p][s];
    for (int i = 0; i < g->nn; i++) {
        const tnode *nd = &g->nodes[i];
        if (nd->player != p) continue;
        for (int a = 0; a < nd->nact; a++) {
            if (node_of_seq) node_of_seq[nd->seq[a]] = nd->seq[0];
            if (nact_of_seq) nact_of_seq[nd->seq[a]] = nd->nact;
        }
    }
}

void orc_turn_seqform(const orc_turn *g, int p, const double *beh, double *x)
{
    int H = g->H;
    for (int s = 0; s < g->n[p]; s++) {
        int par = g->seq_parent[p][s];
        for (int h = 0; h < H; h++)
            x[(size_t)s * H + h] = beh[(size_t)s * H + h] * (par < 0 ? 1.0 : x[(size_t)par * H + h]);
    }
}
