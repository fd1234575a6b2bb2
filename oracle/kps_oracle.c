/*
 * kps_oracle.c -- plain, slow, obviously-correct CPU oracle (FP64).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test-suite, the smoke check and
 * the benchmark's CPU-baseline leg, never by the product path.  It shares no
 * code with the CUDA library.  Every function follows the paper's statement
 * of the problem directly:
 *
 *   - the skeleton betting tree of a river endgame (Sec. 3, Fig. 1; betting
 *     rules in the appendix "Poker games"; pot arithmetic of the appendix
 *     worked example "Computation of pot contributions and stack amounts");
 *   - the chance deal pi(h1,h2) (Sec. 3): mu1*mu2/beta on compatible pairs;
 *   - the payoff matrix (Sec. 2): A[s1,s2] += u(z)*c(z) over terminals z;
 *   - Technique B (Sec. 4 and its appendix) and its postprocessing (Sec. 4,
 *     "Postprocessing");
 *   - a regret-matching-plus self-play loop and the exploitability measure
 *     of Sec. 5 ("First-order methods": half the saddle-point gap over the
 *     initial pot).
 *
 * Readings of the paper taken here (each is also listed with the design
 * notes): the rank-one term of C uses lambda_i = mu_i/sqrt(beta) rather than
 * mu_i; a bet or raise whose amount reaches the effective stack becomes the
 * all-in action and merges with it; the raise cap counts every aggressive
 * action of the round (bets, raises, all-ins); showdown payoff is
 * gamma * min(c1, c2); the postprocessing substitutes y_j = -sum a_i y_i
 * (so a column of U is added with factor -a_i).
 */
#include "kps_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXA (ORC_MAX_BETS + 3)

enum { ACT_FOLD = 0, ACT_CHECKCALL = 1, ACT_AGGR = 2 };

typedef struct {
    int player;            /* 0 or 1 acting player; -1 terminal               */
    double c[2];           /* pot contributions at this node                  */
    int naggr;             /* aggressive actions taken so far                 */
    int prev_check;        /* the previous action was a check                 */
    int nact;
    int child[MAXA];
    int act_code[MAXA];
    double act_amt[MAXA];  /* contribution of the actor after the action      */
    int seq[MAXA];         /* owner's sequence id of each action              */
    int last_seq[2];       /* last sequence of each player on the path        */
    int pnode;             /* index among the owner's nodes (pre-order)       */
    int tkind;             /* terminal: 0 fold, 1 showdown                    */
    int folder;            /* terminal fold: who folded                       */
    int tidx;              /* terminal index                                  */
} onode;

struct orc_game {
    orc_spec sp;
    int H, k, nleft;
    int *cards;            /* H*k                                             */
    double *mu[2];
    int *strength;
    double beta;
    int nn, cap_nodes;
    onode *nodes;
    int n[2];              /* number of sequences per player                  */
    int *seq_node[2];      /* owner node (index among the player's nodes)     */
    int *seq_parent[2];    /* parent sequence of that node (-1 = empty)       */
    int *seq_action[2];
    double *seq_amount[2];
    int np[2];             /* player nodes                                    */
    int *pn_tree[2];       /* tree node id of each player node                */
    int T, TF, TS;
    int *term_node;        /* tree node id of each terminal                   */
};

/* ------------------------------------------------------------------ tree */

static int new_node(orc_game *g)
{
    if (g->nn == g->cap_nodes) {
        g->cap_nodes = g->cap_nodes ? 2 * g->cap_nodes : 64;
        g->nodes = (onode *)realloc(g->nodes, (size_t)g->cap_nodes * sizeof(onode));
    }
    memset(&g->nodes[g->nn], 0, sizeof(onode));
    return g->nn++;
}

static double dmin(double a, double b) { return a < b ? a : b; }

/* Actions available at a decision node, following the appendix rules:
 * facing a larger contribution the player may fold, call or raise; with equal
 * contributions the player may check or bet.  A bet/raise of fraction f first
 * matches the opponent and then adds f times the pot after matching
 * (Fig. 1 caption).  Amounts at or above the effective stack become all-in. */
static int list_actions(const orc_game *g, const onode *nd, int *code, double *amt)
{
    int p = nd->player, o = 1 - p, na = 0;
    /* the bet sizes on offer: one list, or the menu entry of this player in
     * this situation (how many bets and raises came before, and whether the
     * opponent just checked) */
    int nbet = g->sp.nbet;
    const double *frac = g->sp.bet_frac;
    if (g->sp.use_menu) {
        int k;
        if (nd->naggr == 0) k = nd->prev_check ? 1 : 0;
        else if (nd->naggr == 1) k = 2;
        else if (nd->naggr == 2) k = 3;
        else k = 4;
        nbet = g->sp.menu_nbet[p][k];
        frac = g->sp.menu_frac[p][k];
    }
    double maxp = g->sp.contrib0[p] + g->sp.stack[p];
    double maxo = g->sp.contrib0[o] + g->sp.stack[o];
    double eff = dmin(maxp, maxo);
    int can_aggr = (g->sp.raise_cap < 0 || nd->naggr < g->sp.raise_cap);
    double aggr[MAXA];
    int nag = 0;
    if (nd->c[p] < nd->c[o]) {
        code[na] = ACT_FOLD; amt[na] = nd->c[p]; na++;
        code[na] = ACT_CHECKCALL; amt[na] = dmin(nd->c[o], maxp); na++;
        if (can_aggr && eff > nd->c[o]) {
            double matched = nd->c[o];
            double pot_after = 2.0 * matched;
            for (int i = 0; i < nbet; i++) {
                double a = matched + frac[i] * pot_after;
                aggr[nag++] = a >= eff ? eff : a;
            }
            if (g->sp.allow_allin) aggr[nag++] = eff;
        }
    } else {
        code[na] = ACT_CHECKCALL; amt[na] = nd->c[p]; na++;
        if (can_aggr && eff > nd->c[p]) {
            double pot = nd->c[0] + nd->c[1];
            for (int i = 0; i < nbet; i++) {
                double a = nd->c[p] + frac[i] * pot;
                aggr[nag++] = a >= eff ? eff : a;
            }
            if (g->sp.allow_allin) aggr[nag++] = eff;
        }
    }
    /* ascending, duplicates merged (a capped bet is the all-in action) */
    for (int i = 1; i < nag; i++)
        for (int j = i; j > 0 && aggr[j] < aggr[j - 1]; j--) {
            double t = aggr[j]; aggr[j] = aggr[j - 1]; aggr[j - 1] = t;
        }
    for (int i = 0; i < nag; i++) {
        if (i > 0 && aggr[i] == aggr[i - 1]) continue;
        code[na] = ACT_AGGR; amt[na] = aggr[i]; na++;
    }
    return na;
}

/* Depth-first construction.  Sequence ids of a node's actions are assigned
 * when the node is first visited (pre-order), consecutively in action order. */
static void expand(orc_game *g, int id)
{
    if (g->nodes[id].player < 0) {
        g->nodes[id].tidx = g->T++;
        return;
    }
    int code[MAXA];
    double amt[MAXA];
    int na = list_actions(g, &g->nodes[id], code, amt);
    int p = g->nodes[id].player, o = 1 - p;
    g->nodes[id].nact = na;
    g->nodes[id].pnode = g->np[p]++;
    for (int a = 0; a < na; a++) {
        g->nodes[id].act_code[a] = code[a];
        g->nodes[id].act_amt[a] = amt[a];
        g->nodes[id].seq[a] = g->n[p]++;
    }
    for (int a = 0; a < na; a++) {
        int c = new_node(g);
        onode *nd = &g->nodes[id];          /* realloc may move the array */
        onode *ch = &g->nodes[c];
        nd->child[a] = c;
        ch->c[0] = nd->c[0];
        ch->c[1] = nd->c[1];
        ch->last_seq[0] = nd->last_seq[0];
        ch->last_seq[1] = nd->last_seq[1];
        ch->last_seq[p] = nd->seq[a];
        ch->naggr = nd->naggr;
        ch->c[p] = amt[a];
        if (code[a] == ACT_FOLD) {
            ch->player = -1; ch->tkind = 0; ch->folder = p;
        } else if (code[a] == ACT_CHECKCALL) {
            if (nd->c[p] < nd->c[o] || nd->prev_check) {
                ch->player = -1; ch->tkind = 1; ch->folder = -1;
            } else {
                ch->player = o; ch->prev_check = 1;
            }
        } else {
            ch->player = o; ch->naggr = nd->naggr + 1;
        }
        expand(g, c);
    }
}

/* ----------------------------------------------------------------- hands */

static int hands_compatible(const orc_game *g, int h1, int h2)
{
    for (int i = 0; i < g->k; i++)
        for (int j = 0; j < g->k; j++)
            if (g->cards[h1 * g->k + i] == g->cards[h2 * g->k + j]) return 0;
    return 1;
}

/* gamma(h1,h2) of Sec. 3: +1 if h1 beats h2, -1 if beaten, 0 on a tie or
 * when the hands are incompatible. */
static int gamma_sign(const orc_game *g, int h1, int h2)
{
    if (!hands_compatible(g, h1, h2)) return 0;
    int s1 = g->strength[h1], s2 = g->strength[h2];
    return (s1 > s2) - (s1 < s2);
}

/* pi(h1,h2) of Sec. 3. */
static double chance(const orc_game *g, int h1, int h2)
{
    if (!hands_compatible(g, h1, h2)) return 0.0;
    return g->mu[0][h1] * g->mu[1][h2] / g->beta;
}

/* Player-1 payoff at terminal t for hands (h1,h2), before the chance weight:
 * fold terminals pay the folder's loss of its contribution; showdown
 * terminals pay gamma times the matched contribution. */
static double payoff(const orc_game *g, int t, int h1, int h2)
{
    const onode *z = &g->nodes[g->term_node[t]];
    if (z->tkind == 0) return z->folder == 0 ? -z->c[0] : z->c[1];
    return gamma_sign(g, h1, h2) * dmin(z->c[0], z->c[1]);
}

/* --------------------------------------------------------------- builder */

orc_game *orc_build(const orc_spec *sp)
{
    if (!sp || sp->cards_per_hand < 1 || sp->cards_per_hand > 2) return NULL;
    if (sp->ranks < 1 || sp->suits < 1 || sp->nbet < 0 || sp->nbet > ORC_MAX_BETS) return NULL;
    if (sp->use_menu)
        for (int p = 0; p < 2; p++)
            for (int k = 0; k < 5; k++)
                if (sp->menu_nbet[p][k] < 0 || sp->menu_nbet[p][k] > ORC_MAX_BETS) return NULL;
    if (sp->nboard < 0 || sp->nboard > ORC_MAX_BOARD) return NULL;
    if (!sp->strength) return NULL;
    int ncard = sp->ranks * sp->suits;
    orc_game *g = (orc_game *)calloc(1, sizeof(orc_game));
    g->sp = *sp;
    g->k = sp->cards_per_hand;
    int *onb = (int *)calloc((size_t)ncard, sizeof(int));
    for (int i = 0; i < sp->nboard; i++) {
        if (sp->board[i] < 0 || sp->board[i] >= ncard || onb[sp->board[i]]) {
            free(onb); free(g); return NULL;
        }
        onb[sp->board[i]] = 1;
    }
    int *left = (int *)malloc((size_t)ncard * sizeof(int));
    int nl = 0;
    for (int c = 0; c < ncard; c++) if (!onb[c]) left[nl++] = c;
    g->nleft = nl;
    if (g->k == 1) {
        g->H = nl;
        g->cards = (int *)malloc((size_t)nl * sizeof(int));
        for (int i = 0; i < nl; i++) g->cards[i] = left[i];
    } else {
        g->H = nl * (nl - 1) / 2;
        g->cards = (int *)malloc((size_t)g->H * 2 * sizeof(int));
        int h = 0;
        for (int i = 0; i < nl; i++)
            for (int j = i + 1; j < nl; j++) {
                g->cards[2 * h] = left[i];
                g->cards[2 * h + 1] = left[j];
                h++;
            }
    }
    free(left);
    free(onb);
    int H = g->H;
    for (int p = 0; p < 2; p++) {
        g->mu[p] = (double *)malloc((size_t)H * sizeof(double));
        const double *src = p == 0 ? sp->mu1 : sp->mu2;
        for (int h = 0; h < H; h++) g->mu[p][h] = src ? src[h] : 1.0;
    }
    g->strength = (int *)malloc((size_t)H * sizeof(int));
    memcpy(g->strength, sp->strength, (size_t)H * sizeof(int));
    g->sp.mu1 = g->sp.mu2 = NULL;
    g->sp.strength = NULL;
    g->beta = 0.0;
    for (int h1 = 0; h1 < H; h1++)
        for (int h2 = 0; h2 < H; h2++)
            if (hands_compatible(g, h1, h2)) g->beta += g->mu[0][h1] * g->mu[1][h2];
    if (!(g->beta > 0.0)) { orc_free(g); return NULL; }

    int root = new_node(g);
    g->nodes[root].player = 0;
    g->nodes[root].c[0] = sp->contrib0[0];
    g->nodes[root].c[1] = sp->contrib0[1];
    g->nodes[root].last_seq[0] = g->nodes[root].last_seq[1] = -1;
    expand(g, root);

    g->term_node = (int *)malloc((size_t)g->T * sizeof(int));
    for (int p = 0; p < 2; p++) {
        g->seq_node[p] = (int *)malloc((size_t)(g->n[p] + 1) * sizeof(int));
        g->seq_parent[p] = (int *)malloc((size_t)(g->n[p] + 1) * sizeof(int));
        g->seq_action[p] = (int *)malloc((size_t)(g->n[p] + 1) * sizeof(int));
        g->seq_amount[p] = (double *)malloc((size_t)(g->n[p] + 1) * sizeof(double));
        g->pn_tree[p] = (int *)malloc((size_t)(g->np[p] + 1) * sizeof(int));
    }
    g->TF = g->TS = 0;
    for (int i = 0; i < g->nn; i++) {
        onode *nd = &g->nodes[i];
        if (nd->player < 0) {
            g->term_node[nd->tidx] = i;
            if (nd->tkind == 0) g->TF++; else g->TS++;
            /* every terminal follows at least one action of each player */
            if (nd->last_seq[0] < 0 || nd->last_seq[1] < 0) { orc_free(g); return NULL; }
            continue;
        }
        int p = nd->player;
        g->pn_tree[p][nd->pnode] = i;
        for (int a = 0; a < nd->nact; a++) {
            int s = nd->seq[a];
            g->seq_node[p][s] = nd->pnode;
            g->seq_parent[p][s] = nd->last_seq[p];
            g->seq_action[p][s] = nd->act_code[a];
            g->seq_amount[p][s] = nd->act_amt[a];
        }
    }
    return g;
}

void orc_free(orc_game *g)
{
    if (!g) return;
    free(g->cards);
    free(g->mu[0]); free(g->mu[1]);
    free(g->strength);
    free(g->nodes);
    for (int p = 0; p < 2; p++) {
        free(g->seq_node[p]); free(g->seq_parent[p]); free(g->seq_action[p]);
        free(g->seq_amount[p]); free(g->pn_tree[p]);
    }
    free(g->term_node);
    free(g);
}

void orc_info(const orc_game *g, int *info)
{
    info[0] = g->H; info[1] = g->n[0]; info[2] = g->n[1]; info[3] = g->T;
    info[4] = g->TF; info[5] = g->TS; info[6] = g->nn; info[7] = g->nleft;
    info[8] = g->np[0]; info[9] = g->np[1];
}

double orc_beta(const orc_game *g) { return g->beta; }
double orc_pot0(const orc_game *g) { return g->sp.contrib0[0] + g->sp.contrib0[1]; }

void orc_hands(const orc_game *g, int *cards)
{
    memcpy(cards, g->cards, (size_t)g->H * g->k * sizeof(int));
}

void orc_terminals(const orc_game *g, int *s1, int *s2, int *kind, int *folder,
                   double *c1, double *c2)
{
    for (int t = 0; t < g->T; t++) {
        const onode *z = &g->nodes[g->term_node[t]];
        if (s1) s1[t] = z->last_seq[0];
        if (s2) s2[t] = z->last_seq[1];
        if (kind) kind[t] = z->tkind;
        if (folder) folder[t] = z->tkind == 0 ? z->folder : -1;
        if (c1) c1[t] = z->c[0];
        if (c2) c2[t] = z->c[1];
    }
}

void orc_sequences(const orc_game *g, int p, int *seq_node, int *seq_parent,
                   int *seq_action, double *seq_amount, int *nodes_nact)
{
    for (int s = 0; s < g->n[p]; s++) {
        if (seq_node) seq_node[s] = g->seq_node[p][s];
        if (seq_parent) seq_parent[s] = g->seq_parent[p][s];
        if (seq_action) seq_action[s] = g->seq_action[p][s];
        if (seq_amount) seq_amount[s] = g->seq_amount[p][s];
    }
    if (nodes_nact)
        for (int i = 0; i < g->np[p]; i++) nodes_nact[i] = g->nodes[g->pn_tree[p][i]].nact;
}

int orc_find_terminal(const orc_game *g, const char *path)
{
    int id = 0;
    const char *s = path;
    while (*s) {
        while (*s == ' ') s++;
        if (!*s) break;
        const onode *nd = &g->nodes[id];
        if (nd->player < 0) return -1;
        int want = -1;
        if (*s == 'f' || *s == 'c') {
            int code = *s == 'f' ? ACT_FOLD : ACT_CHECKCALL;
            for (int a = 0; a < nd->nact; a++) if (nd->act_code[a] == code) want = a;
            s++;
        } else if (*s == 'b') {
            s++;
            int idx = 0;
            while (*s >= '0' && *s <= '9') idx = idx * 10 + (*s++ - '0');
            int seen = 0;
            for (int a = 0; a < nd->nact; a++)
                if (nd->act_code[a] == ACT_AGGR) { if (seen == idx) { want = a; break; } seen++; }
        } else if (*s == 'a') {
            for (int a = 0; a < nd->nact; a++) if (nd->act_code[a] == ACT_AGGR) want = a;
            s++;
        } else {
            return -1;
        }
        if (want < 0) return -1;
        id = nd->child[want];
    }
    return g->nodes[id].player < 0 ? g->nodes[id].tidx : -1;
}

/* ------------------------------------------------------ payoff matrix A */

int orc_dense_A(const orc_game *g, double *A)
{
    int H = g->H, n1 = g->n[0], n2 = g->n[1];
    size_t ncol = (size_t)H * n2;
    memset(A, 0, (size_t)H * n1 * ncol * sizeof(double));
    for (int t = 0; t < g->T; t++) {
        const onode *z = &g->nodes[g->term_node[t]];
        int s1 = z->last_seq[0], s2 = z->last_seq[1];
        for (int h1 = 0; h1 < H; h1++)
            for (int h2 = 0; h2 < H; h2++) {
                double pi = chance(g, h1, h2);
                if (pi == 0.0) continue;
                A[((size_t)h1 * n1 + s1) * ncol + (size_t)h2 * n2 + s2] += pi * payoff(g, t, h1, h2);
            }
    }
    return 0;
}

static void matvec_one(const orc_game *g, const double *y, double *out)
{
    int H = g->H;
    memset(out, 0, (size_t)g->n[0] * H * sizeof(double));
    for (int t = 0; t < g->T; t++) {
        const onode *z = &g->nodes[g->term_node[t]];
        int s1 = z->last_seq[0], s2 = z->last_seq[1];
        for (int h1 = 0; h1 < H; h1++) {
            double acc = 0.0;
            for (int h2 = 0; h2 < H; h2++) {
                double pi = chance(g, h1, h2);
                if (pi == 0.0) continue;
                acc += pi * payoff(g, t, h1, h2) * y[(size_t)s2 * H + h2];
            }
            out[(size_t)s1 * H + h1] += acc;
        }
    }
}

static void matvec_t_one(const orc_game *g, const double *x, double *out)
{
    int H = g->H;
    memset(out, 0, (size_t)g->n[1] * H * sizeof(double));
    for (int t = 0; t < g->T; t++) {
        const onode *z = &g->nodes[g->term_node[t]];
        int s1 = z->last_seq[0], s2 = z->last_seq[1];
        for (int h2 = 0; h2 < H; h2++) {
            double acc = 0.0;
            for (int h1 = 0; h1 < H; h1++) {
                double pi = chance(g, h1, h2);
                if (pi == 0.0) continue;
                acc += pi * payoff(g, t, h1, h2) * x[(size_t)s1 * H + h1];
            }
            out[(size_t)s2 * H + h2] += acc;
        }
    }
}

void orc_matvec_A(const orc_game *g, const double *y, double *out, int batch, int nthreads)
{
    size_t in = (size_t)g->n[1] * g->H, on = (size_t)g->n[0] * g->H;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = omp_get_max_threads();
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1)
#endif
    for (int b = 0; b < batch; b++) matvec_one(g, y + b * in, out + b * on);
    (void)nthreads;
}

void orc_matvec_AT(const orc_game *g, const double *x, double *out, int batch, int nthreads)
{
    size_t in = (size_t)g->n[0] * g->H, on = (size_t)g->n[1] * g->H;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = omp_get_max_threads();
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1)
#endif
    for (int b = 0; b < batch; b++) matvec_t_one(g, x + b * in, out + b * on);
    (void)nthreads;
}

void orc_matvec_A_entries(const orc_game *g, const double *y, int nent,
                          const int *b, const int *s, const int *h, double *out)
{
    int H = g->H;
    size_t in = (size_t)g->n[1] * H;
    for (int e = 0; e < nent; e++) {
        double acc = 0.0;
        const double *yb = y + (size_t)b[e] * in;
        for (int t = 0; t < g->T; t++) {
            const onode *z = &g->nodes[g->term_node[t]];
            if (z->last_seq[0] != s[e]) continue;
            int s2 = z->last_seq[1];
            for (int h2 = 0; h2 < H; h2++) {
                double pi = chance(g, h[e], h2);
                if (pi == 0.0) continue;
                acc += pi * payoff(g, t, h[e], h2) * yb[(size_t)s2 * H + h2];
            }
        }
        out[e] = acc;
    }
}

void orc_matvec_AT_entries(const orc_game *g, const double *x, int nent,
                           const int *b, const int *s, const int *h, double *out)
{
    int H = g->H;
    size_t in = (size_t)g->n[0] * H;
    for (int e = 0; e < nent; e++) {
        double acc = 0.0;
        const double *xb = x + (size_t)b[e] * in;
        for (int t = 0; t < g->T; t++) {
            const onode *z = &g->nodes[g->term_node[t]];
            if (z->last_seq[1] != s[e]) continue;
            int s1 = z->last_seq[0];
            for (int h1 = 0; h1 < H; h1++) {
                double pi = chance(g, h1, h[e]);
                if (pi == 0.0) continue;
                acc += pi * payoff(g, t, h1, h[e]) * xb[(size_t)s1 * H + h1];
            }
        }
        out[e] = acc;
    }
}

/* ------------------------------------------------------------ brute force */

static double walk(const orc_game *g, int id, int h1, int h2, const double *b1,
                   const double *b2, double reach)
{
    const onode *nd = &g->nodes[id];
    if (nd->player < 0) return reach * payoff(g, nd->tidx, h1, h2);
    int H = g->H, hp = nd->player == 0 ? h1 : h2;
    const double *beh = nd->player == 0 ? b1 : b2;
    double v = 0.0;
    for (int a = 0; a < nd->nact; a++) {
        double pr = beh[(size_t)nd->seq[a] * H + hp];
        if (pr == 0.0) continue;
        v += walk(g, nd->child[a], h1, h2, b1, b2, reach * pr);
    }
    return v;
}

double orc_bruteforce_value(const orc_game *g, const double *beh1, const double *beh2)
{
    double v = 0.0;
    for (int h1 = 0; h1 < g->H; h1++)
        for (int h2 = 0; h2 < g->H; h2++) {
            double pi = chance(g, h1, h2);
            if (pi == 0.0) continue;
            v += pi * walk(g, 0, h1, h2, beh1, beh2, 1.0);
        }
    return v;
}

void orc_seqform(const orc_game *g, int p, const double *beh, double *x)
{
    int H = g->H;
    for (int s = 0; s < g->n[p]; s++) {
        int par = g->seq_parent[p][s];
        for (int h = 0; h < H; h++)
            x[(size_t)s * H + h] = beh[(size_t)s * H + h] * (par < 0 ? 1.0 : x[(size_t)par * H + h]);
    }
}

double orc_value(const orc_game *g, const double *x, const double *y)
{
    int H = g->H;
    double *ay = (double *)malloc((size_t)g->n[0] * H * sizeof(double));
    matvec_one(g, y, ay);
    double v = 0.0;
    for (size_t i = 0; i < (size_t)g->n[0] * H; i++) v += x[i] * ay[i];
    free(ay);
    return v;
}

/* ------------------------------------------------------------ Technique B */

/* Hands in strength order (ascending strength, ties by canonical index):
 * the order in which the rows of W read -1 ... 0 ... +1 (Sec. 4). */
static int *strength_order(const orc_game *g)
{
    int H = g->H;
    int *ord = (int *)malloc((size_t)H * sizeof(int));
    for (int i = 0; i < H; i++) ord[i] = i;
    for (int i = 1; i < H; i++)        /* insertion sort: stable, obvious */
        for (int j = i; j > 0; j--) {
            int a = ord[j - 1], b = ord[j];
            if (g->strength[a] > g->strength[b]) { ord[j - 1] = b; ord[j] = a; }
            else break;
        }
    return ord;
}

/* F and S of Sec. 3 as dense n1 x n2 matrices. */
static void fold_showdown(const orc_game *g, double *F, double *S)
{
    int n1 = g->n[0], n2 = g->n[1];
    memset(F, 0, (size_t)n1 * n2 * sizeof(double));
    memset(S, 0, (size_t)n1 * n2 * sizeof(double));
    for (int t = 0; t < g->T; t++) {
        const onode *z = &g->nodes[g->term_node[t]];
        size_t idx = (size_t)z->last_seq[0] * n2 + z->last_seq[1];
        if (z->tkind == 0) F[idx] = z->folder == 0 ? -z->c[0] : z->c[1];
        else S[idx] = dmin(z->c[0], z->c[1]);
    }
}

static long long count_nz(const double *a, size_t n)
{
    long long c = 0;
    for (size_t i = 0; i < n; i++) c += a[i] != 0.0;
    return c;
}

/* x = M^{-1} b for a unit lower-triangular dense M (forward substitution). */
static void lower_solve(const double *M, int m, double *b)
{
    for (int i = 0; i < m; i++) {
        double s = b[i];
        for (int j = 0; j < i; j++) s -= M[(size_t)i * m + j] * b[j];
        b[i] = s / M[(size_t)i * m + i];
    }
}

/* max |Adef - (Ahat + U M^{-1} V^T)| with U (R x m), M (m x m), V (C x m). */
static double identity_error(const double *Adef, const double *Ahat, const double *U,
                             const double *M, const double *V, int R, int C, int m)
{
    double err = 0.0;
    double *col = (double *)malloc((size_t)m * sizeof(double));
    for (int c = 0; c < C; c++) {
        for (int j = 0; j < m; j++) col[j] = V[(size_t)c * m + j];   /* (V^T)[:,c] */
        lower_solve(M, m, col);
        for (int r = 0; r < R; r++) {
            double s = Ahat[(size_t)r * C + c];
            for (int j = 0; j < m; j++) s += U[(size_t)r * m + j] * col[j];
            double e = fabs(s - Adef[(size_t)r * C + c]);
            if (e > err) err = e;
        }
    }
    free(col);
    return err;
}

double orc_technique_b(const orc_game *g, long long *cnt)
{
    int H = g->H, n1 = g->n[0], n2 = g->n[1];
    int R = H * n1, C = H * n2, m = H * n1 + n1;
    if ((long long)m > 2048 || (long long)C > 2048) return -1.0;
    int *ord = strength_order(g);
    double sb = sqrt(g->beta);
    double *lam1 = (double *)malloc((size_t)H * sizeof(double));
    double *lam2 = (double *)malloc((size_t)H * sizeof(double));
    for (int i = 0; i < H; i++) {
        lam1[i] = g->mu[0][ord[i]] / sb;
        lam2[i] = g->mu[1][ord[i]] / sb;
    }
    double *F = (double *)malloc((size_t)n1 * n2 * sizeof(double));
    double *S = (double *)malloc((size_t)n1 * n2 * sizeof(double));
    fold_showdown(g, F, S);
    double *W = (double *)calloc((size_t)H * H, sizeof(double));
    double *Hx = (double *)calloc((size_t)H * H, sizeof(double));
    for (int i = 0; i < H; i++)
        for (int j = 0; j < H; j++) {
            W[(size_t)i * H + j] = gamma_sign(g, ord[i], ord[j]);
            Hx[(size_t)i * H + j] = hands_compatible(g, ord[i], ord[j]) ? 0.0 : 1.0;
        }
    /* Y = D W, D lower bidiagonal with 1 on the diagonal, -1 below it. */
    double *Y = (double *)malloc((size_t)H * H * sizeof(double));
    for (int i = 0; i < H; i++)
        for (int j = 0; j < H; j++)
            Y[(size_t)i * H + j] = W[(size_t)i * H + j] - (i > 0 ? W[(size_t)(i - 1) * H + j] : 0.0);

    /* A from the definition, rows/cols in (sorted hand, sequence) paper order */
    double *Adef = (double *)calloc((size_t)R * C, sizeof(double));
    for (int t = 0; t < g->T; t++) {
        const onode *z = &g->nodes[g->term_node[t]];
        int s1 = z->last_seq[0], s2 = z->last_seq[1];
        for (int i = 0; i < H; i++)
            for (int j = 0; j < H; j++) {
                double pi = chance(g, ord[i], ord[j]);
                if (pi == 0.0) continue;
                Adef[((size_t)i * n1 + s1) * C + (size_t)j * n2 + s2] += pi * payoff(g, t, ord[i], ord[j]);
            }
    }
    /* Ahat = -(Lambda1 Hx Lambda2) (x) F */
    double *Ahat = (double *)calloc((size_t)R * C, sizeof(double));
    for (int i = 0; i < H; i++)
        for (int j = 0; j < H; j++) {
            double w = lam1[i] * Hx[(size_t)i * H + j] * lam2[j];
            if (w == 0.0) continue;
            for (int a = 0; a < n1; a++)
                for (int b = 0; b < n2; b++)
                    Ahat[((size_t)i * n1 + a) * C + (size_t)j * n2 + b] = -w * F[(size_t)a * n2 + b];
        }
    /* U = [Lambda1 (x) I | lambda1 (x) I]   (R x m) */
    double *U = (double *)calloc((size_t)R * m, sizeof(double));
    for (int i = 0; i < H; i++)
        for (int a = 0; a < n1; a++) {
            U[((size_t)i * n1 + a) * m + (size_t)i * n1 + a] = lam1[i];
            U[((size_t)i * n1 + a) * m + (size_t)H * n1 + a] = lam1[i];
        }
    /* M = diag(D (x) I, I)   (m x m) */
    double *M = (double *)calloc((size_t)m * m, sizeof(double));
    for (int i = 0; i < H; i++)
        for (int a = 0; a < n1; a++) {
            size_t r = (size_t)i * n1 + a;
            M[r * m + r] = 1.0;
            if (i > 0) M[r * m + (size_t)(i - 1) * n1 + a] = -1.0;
        }
    for (int a = 0; a < n1; a++) M[((size_t)H * n1 + a) * m + (size_t)H * n1 + a] = 1.0;
    /* V = [(Lambda2 Y^T) (x) S^T | lambda2 (x) F^T]   (C x m) */
    double *V = (double *)calloc((size_t)C * m, sizeof(double));
    for (int j = 0; j < H; j++)
        for (int b = 0; b < n2; b++) {
            size_t r = (size_t)j * n2 + b;
            for (int i = 0; i < H; i++) {
                double yv = lam2[j] * Y[(size_t)i * H + j];     /* (Lambda2 Y^T)[j][i] */
                if (yv == 0.0) continue;
                for (int a = 0; a < n1; a++) V[r * m + (size_t)i * n1 + a] = yv * S[(size_t)a * n2 + b];
            }
            for (int a = 0; a < n1; a++) V[r * m + (size_t)H * n1 + a] = lam2[j] * F[(size_t)a * n2 + b];
        }
    cnt[0] = count_nz(Adef, (size_t)R * C);
    cnt[1] = count_nz(Ahat, (size_t)R * C);
    cnt[2] = count_nz(U, (size_t)R * m);
    cnt[3] = count_nz(M, (size_t)m * m);
    cnt[4] = count_nz(V, (size_t)C * m);
    double err = identity_error(Adef, Ahat, U, M, V, R, C, m);

    /* Postprocessing (Sec. 4): for every zero column j of V (ascending),
     * y_j = -sum_i a_i y_i with a_i the off-diagonal entries of row j of M;
     * substitute y_j wherever it appears and drop row/column j of M and
     * column j of U and V. */
    int *alive = (int *)malloc((size_t)m * sizeof(int));
    for (int j = 0; j < m; j++) alive[j] = 1;
    for (int j = 0; j < m; j++) {
        int zero = 1;
        for (int c = 0; c < C && zero; c++) if (V[(size_t)c * m + j] != 0.0) zero = 0;
        if (!zero) continue;
        for (int i = 0; i < j; i++) {
            double ai = M[(size_t)j * m + i];
            if (!alive[i] || ai == 0.0) continue;
            for (int r = 0; r < R; r++) U[(size_t)r * m + i] += -ai * U[(size_t)r * m + j];
            for (int r = j + 1; r < m; r++) M[(size_t)r * m + i] += -ai * M[(size_t)r * m + j];
        }
        alive[j] = 0;
        for (int r = 0; r < R; r++) U[(size_t)r * m + j] = 0.0;
        for (int r = 0; r < m; r++) { M[(size_t)r * m + j] = 0.0; M[(size_t)j * m + r] = 0.0; }
    }
    /* compact the surviving indices and re-check the identity */
    int mm = 0;
    for (int j = 0; j < m; j++) mm += alive[j];
    double *U2 = (double *)calloc((size_t)R * (mm ? mm : 1), sizeof(double));
    double *M2 = (double *)calloc((size_t)(mm ? mm : 1) * (mm ? mm : 1), sizeof(double));
    double *V2 = (double *)calloc((size_t)C * (mm ? mm : 1), sizeof(double));
    for (int j = 0, jj = 0; j < m; j++) {
        if (!alive[j]) continue;
        for (int r = 0; r < R; r++) U2[(size_t)r * mm + jj] = U[(size_t)r * m + j];
        for (int c = 0; c < C; c++) V2[(size_t)c * mm + jj] = V[(size_t)c * m + j];
        for (int i = 0, ii = 0; i < m; i++) {
            if (!alive[i]) continue;
            M2[(size_t)jj * mm + ii] = M[(size_t)j * m + i];
            ii++;
        }
        jj++;
    }
    cnt[5] = cnt[1];
    cnt[6] = count_nz(U2, (size_t)R * mm);
    cnt[7] = count_nz(M2, (size_t)mm * mm);
    cnt[8] = count_nz(V2, (size_t)C * mm);
    double err2 = identity_error(Adef, Ahat, U2, M2, V2, R, C, mm);
    if (err2 > err) err = err2;

    free(alive); free(U2); free(M2); free(V2);
    free(ord); free(lam1); free(lam2); free(F); free(S); free(W); free(Hx); free(Y);
    free(Adef); free(Ahat); free(U); free(M); free(V);
    return err;
}

/* The same counts from the structure of the factors, for games of any size.
 * Follows the dense procedure above step by step on the chains of D (x) I. */
void orc_technique_b_counts(const orc_game *g, long long *cnt)
{
    int H = g->H, n1 = g->n[0];
    int *ord = strength_order(g);
    long long nz1 = 0, nz2 = 0, inc = 0, pairs_f = 0, pairs_s = 0;
    for (int h = 0; h < H; h++) { nz1 += g->mu[0][h] != 0.0; nz2 += g->mu[1][h] != 0.0; }
    for (int i = 0; i < H; i++)
        for (int j = 0; j < H; j++) {
            if (g->mu[0][i] == 0.0 || g->mu[1][j] == 0.0) continue;
            if (!hands_compatible(g, i, j)) { inc++; continue; }
            pairs_f++;
            if (g->strength[i] != g->strength[j]) pairs_s++;
        }
    /* rows of Y = D W in sorted order, columns restricted to mu2 != 0 */
    int *Wprev = (int *)calloc((size_t)H, sizeof(int));
    int *Wcur = (int *)calloc((size_t)H, sizeof(int));
    int *yzero = (int *)malloc((size_t)H * sizeof(int));
    long long nnzY = 0;
    for (int i = 0; i < H; i++) {
        int nzr = 0;
        for (int j = 0; j < H; j++) {
            Wcur[j] = gamma_sign(g, ord[i], ord[j]);
            if (Wcur[j] != Wprev[j] && g->mu[1][ord[j]] != 0.0) nzr++;
        }
        nnzY += nzr;
        yzero[i] = nzr == 0;
        int *t = Wprev; Wprev = Wcur; Wcur = t;
    }
    int *hasF = (int *)calloc((size_t)n1, sizeof(int));
    int *hasS = (int *)calloc((size_t)n1, sizeof(int));
    for (int t = 0; t < g->T; t++) {
        const onode *z = &g->nodes[g->term_node[t]];
        if (z->tkind == 0) hasF[z->last_seq[0]] = 1; else hasS[z->last_seq[0]] = 1;
    }
    cnt[0] = pairs_f * g->TF + pairs_s * g->TS;
    cnt[1] = inc * g->TF;
    cnt[2] = 2 * nz1 * n1;
    cnt[3] = (long long)(2 * H - 1) * n1 + n1;
    cnt[4] = nnzY * g->TS + nz2 * g->TF;
    long long U = cnt[2], M = cnt[3];
    for (int a = 0; a < n1; a++) {
        int pred_alive = 0;           /* row h references a surviving y       */
        for (int i = 0; i < H; i++) {
            int zero = !hasS[a] || yzero[i] || nz2 == 0;
            int has_off = i > 0 && pred_alive;
            if (!zero) { pred_alive = 1; continue; }
            M -= 1 + has_off;         /* row i of M removed                   */
            if (!has_off) {           /* y_i == 0: its column of U disappears */
                U -= g->mu[0][ord[i]] != 0.0;
                if (i + 1 < H) M -= 1;  /* row i+1 loses its reference        */
                pred_alive = 0;
            }
            /* else column i of U merges into its predecessor; row i+1 is
             * re-pointed, its nnz unchanged */
        }
        if (!hasF[a] || nz2 == 0) { M -= 1; U -= nz1; }
    }
    cnt[5] = cnt[1];
    cnt[6] = U;
    cnt[7] = M;
    cnt[8] = cnt[4];
    free(ord); free(Wprev); free(Wcur); free(yzero); free(hasF); free(hasS);
}

/* ---------------------------------------------------------------- solver */

/* Bottom-up over player p's nodes (reverse pre-order): q(I,a) = g(I,a) plus
 * the values of p's next decisions under (I,a); v(I) = sum_a b q (mode 0) or
 * max_a q (mode 1, best response).  With regrets != NULL (mode 0) the RM+
 * update R <- max(0, R + q - v) is applied.  Returns sum over hands of the
 * values of p's first decisions. */
static double bottom_up(const orc_game *g, int p, const double *gv, const double *beh,
                        double *regret, int mode)
{
    int H = g->H, n = g->n[p];
    double *cv = (double *)calloc((size_t)n * H, sizeof(double));
    double *q = (double *)malloc((size_t)MAXA * H * sizeof(double));
    double total = 0.0;
    for (int i = g->np[p] - 1; i >= 0; i--) {
        const onode *nd = &g->nodes[g->pn_tree[p][i]];
        int s0 = nd->seq[0], na = nd->nact;
        for (int a = 0; a < na; a++)
            for (int h = 0; h < H; h++)
                q[a * H + h] = gv[(size_t)(s0 + a) * H + h] + cv[(size_t)(s0 + a) * H + h];
        int par = nd->last_seq[p];
        for (int h = 0; h < H; h++) {
            double v;
            if (mode == 1) {
                v = q[h];
                for (int a = 1; a < na; a++) if (q[a * H + h] > v) v = q[a * H + h];
            } else {
                v = 0.0;
                for (int a = 0; a < na; a++) v += beh[(size_t)(s0 + a) * H + h] * q[a * H + h];
                if (regret)
                    for (int a = 0; a < na; a++) {
                        double r = regret[(size_t)(s0 + a) * H + h] + q[a * H + h] - v;
                        regret[(size_t)(s0 + a) * H + h] = r > 0.0 ? r : 0.0;
                    }
            }
            if (par >= 0) cv[(size_t)par * H + h] += v;
            else total += v;
        }
    }
    free(cv);
    free(q);
    return total;
}

/* Regret matching: b(I,a) = R+(I,a)/sum_a R+, uniform when the sum is at
 * most theta (the noise floor of orc_rmplus; 0 gives textbook RM+). */
static void regret_match(const orc_game *g, int p, const double *regret, double *beh, double theta)
{
    int H = g->H;
    for (int i = 0; i < g->np[p]; i++) {
        const onode *nd = &g->nodes[g->pn_tree[p][i]];
        int s0 = nd->seq[0], na = nd->nact;
        for (int h = 0; h < H; h++) {
            double s = 0.0;
            for (int a = 0; a < na; a++) s += regret[(size_t)(s0 + a) * H + h];
            for (int a = 0; a < na; a++)
                beh[(size_t)(s0 + a) * H + h] = s > theta ? regret[(size_t)(s0 + a) * H + h] / s : 1.0 / na;
        }
    }
}

/* Bound on |counterfactual value| of player p: max |payoff| times the
 * largest chance weight mass a hand of p can see,
 *   V_p = max_t max(c1, c2) * max_h mu_p(h) * sum_h mu_q(h) / beta.
 * A player's regret sum at or below eps * V_p is treated as zero: values
 * that are exactly zero (an opponent whose every compatible hand has zero
 * reach) come out of a product that subtracts card-overlap masses as
 * rounding noise instead, and regret matching would otherwise follow that
 * noise.  eps = 2^-40 keeps the floor far above FP64 noise and far below
 * any regret that moves a strategy. */
double orc_regret_floor(const orc_game *g, int p, double eps)
{
    double cmax = 0.0, mmax = 0.0, msum = 0.0;
    for (int t = 0; t < g->T; t++) {
        const onode *z = &g->nodes[g->term_node[t]];
        if (z->c[0] > cmax) cmax = z->c[0];
        if (z->c[1] > cmax) cmax = z->c[1];
    }
    for (int h = 0; h < g->H; h++) {
        if (g->mu[p][h] > mmax) mmax = g->mu[p][h];
        msum += g->mu[1 - p][h];
    }
    return eps * cmax * mmax * msum / g->beta;
}

static void uniform_beh(const orc_game *g, int p, double *beh)
{
    int H = g->H;
    for (int i = 0; i < g->np[p]; i++) {
        const onode *nd = &g->nodes[g->pn_tree[p][i]];
        for (int a = 0; a < nd->nact; a++)
            for (int h = 0; h < H; h++) beh[(size_t)(nd->seq[a]) * H + h] = 1.0 / nd->nact;
    }
}

/* DCFR's regret step for player p, bottom-up like bottom_up: with the
 * instantaneous regret q - v added, a cumulative regret is multiplied by
 * dpos when positive and by dneg otherwise. */
static void bottom_up_dcfr(const orc_game *g, int p, const double *gv, const double *beh, double *regret,
                           double dpos, double dneg)
{
    int H = g->H, n = g->n[p];
    double *cv = (double *)calloc((size_t)n * H, sizeof(double));
    double *q = (double *)malloc((size_t)MAXA * H * sizeof(double));
    for (int i = g->np[p] - 1; i >= 0; i--) {
        const onode *nd = &g->nodes[g->pn_tree[p][i]];
        int s0 = nd->seq[0], na = nd->nact;
        for (int a = 0; a < na; a++)
            for (int h = 0; h < H; h++)
                q[a * H + h] = gv[(size_t)(s0 + a) * H + h] + cv[(size_t)(s0 + a) * H + h];
        int par = nd->last_seq[p];
        for (int h = 0; h < H; h++) {
            double v = 0.0;
            for (int a = 0; a < na; a++) v += beh[(size_t)(s0 + a) * H + h] * q[a * H + h];
            for (int a = 0; a < na; a++) {
                double r = regret[(size_t)(s0 + a) * H + h] + q[a * H + h] - v;
                regret[(size_t)(s0 + a) * H + h] = r * (r > 0.0 ? dpos : dneg);
            }
            if (par >= 0) cv[(size_t)par * H + h] += v;
        }
    }
    free(cv);
    free(q);
}

/* Regret matching on the positive parts of possibly negative regrets. */
static void regret_match_pos(const orc_game *g, int p, const double *regret, double *beh, double theta)
{
    int H = g->H;
    for (int i = 0; i < g->np[p]; i++) {
        const onode *nd = &g->nodes[g->pn_tree[p][i]];
        int s0 = nd->seq[0], na = nd->nact;
        for (int h = 0; h < H; h++) {
            double s = 0.0;
            for (int a = 0; a < na; a++) {
                double r = regret[(size_t)(s0 + a) * H + h];
                s += r > 0.0 ? r : 0.0;
            }
            for (int a = 0; a < na; a++) {
                double r = regret[(size_t)(s0 + a) * H + h];
                beh[(size_t)(s0 + a) * H + h] = s > theta ? (r > 0.0 ? r : 0.0) / s : 1.0 / na;
            }
        }
    }
}

double orc_dcfr(const orc_game *g, int iters, double alpha, double beta, double gamma,
                double *avg_beh1, double *avg_beh2, double *trace, int trace_every)
{
    int H = g->H, n1 = g->n[0], n2 = g->n[1];
    size_t N1 = (size_t)n1 * H, N2 = (size_t)n2 * H;
    double *b1 = (double *)malloc(N1 * sizeof(double)), *b2 = (double *)malloc(N2 * sizeof(double));
    double *x = (double *)malloc(N1 * sizeof(double)), *y = (double *)malloc(N2 * sizeof(double));
    double *R1 = (double *)calloc(N1, sizeof(double)), *R2 = (double *)calloc(N2, sizeof(double));
    double *xs = (double *)calloc(N1, sizeof(double)), *ys = (double *)calloc(N2, sizeof(double));
    double *g1 = (double *)malloc(N1 * sizeof(double)), *g2 = (double *)malloc(N2 * sizeof(double));
    double *xa = (double *)malloc(N1 * sizeof(double)), *ya = (double *)malloc(N2 * sizeof(double));
    uniform_beh(g, 0, b1);
    uniform_beh(g, 1, b2);
    orc_seqform(g, 0, b1, x);
    orc_seqform(g, 1, b2, y);
    const double th1 = orc_regret_floor(g, 0, ORC_REGRET_EPS), th2 = orc_regret_floor(g, 1, ORC_REGRET_EPS);
    double wsum = 0.0, expl = 0.0;
    for (int t = 1; t <= iters; t++) {
        const double ta = pow((double)t, alpha), tb = pow((double)t, beta), wt = pow((double)t, gamma);
        const double dpos = ta / (ta + 1.0), dneg = tb / (tb + 1.0);
        for (size_t i = 0; i < N1; i++) xs[i] += wt * x[i];
        matvec_one(g, y, g1);
        bottom_up_dcfr(g, 0, g1, b1, R1, dpos, dneg);
        regret_match_pos(g, 0, R1, b1, th1);
        orc_seqform(g, 0, b1, x);
        for (size_t i = 0; i < N2; i++) ys[i] += wt * y[i];
        matvec_t_one(g, x, g2);
        for (size_t i = 0; i < N2; i++) g2[i] = -g2[i];
        bottom_up_dcfr(g, 1, g2, b2, R2, dpos, dneg);
        regret_match_pos(g, 1, R2, b2, th2);
        orc_seqform(g, 1, b2, y);
        wsum += wt;
        if (trace) {
            trace[t - 1] = 0.0;
            if (trace_every > 0 && t % trace_every == 0) {
                for (size_t i = 0; i < N1; i++) xa[i] = xs[i] / wsum;
                for (size_t i = 0; i < N2; i++) ya[i] = ys[i] / wsum;
                trace[t - 1] = orc_exploitability(g, xa, ya, NULL, NULL);
            }
        }
    }
    for (size_t i = 0; i < N1; i++) xa[i] = wsum > 0 ? xs[i] / wsum : x[i];
    for (size_t i = 0; i < N2; i++) ya[i] = wsum > 0 ? ys[i] / wsum : y[i];
    expl = orc_exploitability(g, xa, ya, NULL, NULL);
    for (int p = 0; p < 2; p++) {
        double *dst = p == 0 ? avg_beh1 : avg_beh2;
        double *src = p == 0 ? xa : ya;
        if (!dst) continue;
        for (int s = 0; s < g->n[p]; s++) {
            int par = g->seq_parent[p][s];
            for (int h = 0; h < H; h++) {
                double den = par < 0 ? 1.0 : src[(size_t)par * H + h];
                dst[(size_t)s * H + h] = den > 0.0 ? src[(size_t)s * H + h] / den : -1.0;
            }
        }
        for (int i = 0; i < g->np[p]; i++) {
            const onode *nd = &g->nodes[g->pn_tree[p][i]];
            for (int h = 0; h < H; h++)
                if (dst[(size_t)nd->seq[0] * H + h] < 0.0)
                    for (int a = 0; a < nd->nact; a++) dst[(size_t)nd->seq[a] * H + h] = 1.0 / nd->nact;
        }
    }
    free(b1); free(b2); free(x); free(y); free(R1); free(R2); free(xs); free(ys);
    free(g1); free(g2); free(xa); free(ya);
    return expl;
}

double orc_exploitability(const orc_game *g, const double *x, const double *y,
                          double *br1, double *br2)
{
    int H = g->H, n1 = g->n[0], n2 = g->n[1];
    double *g1 = (double *)malloc((size_t)n1 * H * sizeof(double));
    double *g2 = (double *)malloc((size_t)n2 * H * sizeof(double));
    matvec_one(g, y, g1);
    matvec_t_one(g, x, g2);
    for (size_t i = 0; i < (size_t)n2 * H; i++) g2[i] = -g2[i];
    double b1 = bottom_up(g, 0, g1, NULL, NULL, 1);
    double b2 = bottom_up(g, 1, g2, NULL, NULL, 1);
    if (br1) *br1 = b1;
    if (br2) *br2 = b2;
    free(g1);
    free(g2);
    return (b1 + b2) / 2.0 / orc_pot0(g);
}

double orc_rmplus(const orc_game *g, int iters, const double *beh1_0, const double *beh2_0,
                  double *avg_beh1, double *avg_beh2, double *trace, int trace_every)
{
    return orc_rmplus_warm(g, iters, beh1_0, beh2_0, 0.0, 0, avg_beh1, avg_beh2, trace, trace_every);
}

static double rmplus_loop(const orc_game *g, int iters, const double *beh1_0, const double *beh2_0,
                          double kappa, int t0, double eps, double *avg_beh1, double *avg_beh2,
                          double *trace, int trace_every);

double orc_rmplus_warm(const orc_game *g, int iters, const double *beh1_0, const double *beh2_0,
                       double kappa, int t0, double *avg_beh1, double *avg_beh2, double *trace,
                       int trace_every)
{
    return rmplus_loop(g, iters, beh1_0, beh2_0, kappa, t0, ORC_REGRET_EPS, avg_beh1, avg_beh2, trace,
                       trace_every);
}

double orc_rmplus_eps(const orc_game *g, int iters, double eps, double *avg_beh1, double *avg_beh2)
{
    return rmplus_loop(g, iters, NULL, NULL, 0.0, 0, eps, avg_beh1, avg_beh2, NULL, 0);
}

static double rmplus_loop(const orc_game *g, int iters, const double *beh1_0, const double *beh2_0,
                          double kappa, int t0, double eps, double *avg_beh1, double *avg_beh2,
                          double *trace, int trace_every)
{
    int H = g->H, n1 = g->n[0], n2 = g->n[1];
    size_t N1 = (size_t)n1 * H, N2 = (size_t)n2 * H;
    double *b1 = (double *)malloc(N1 * sizeof(double)), *b2 = (double *)malloc(N2 * sizeof(double));
    double *x = (double *)malloc(N1 * sizeof(double)), *y = (double *)malloc(N2 * sizeof(double));
    double *R1 = (double *)calloc(N1, sizeof(double)), *R2 = (double *)calloc(N2, sizeof(double));
    double *xs = (double *)calloc(N1, sizeof(double)), *ys = (double *)calloc(N2, sizeof(double));
    double *g1 = (double *)malloc(N1 * sizeof(double)), *g2 = (double *)malloc(N2 * sizeof(double));
    double *xa = (double *)malloc(N1 * sizeof(double)), *ya = (double *)malloc(N2 * sizeof(double));
    if (beh1_0) memcpy(b1, beh1_0, N1 * sizeof(double)); else uniform_beh(g, 0, b1);
    if (beh2_0) memcpy(b2, beh2_0, N2 * sizeof(double)); else uniform_beh(g, 1, b2);
    orc_seqform(g, 0, b1, x);
    orc_seqform(g, 1, b2, y);
    const double th1 = orc_regret_floor(g, 0, eps), th2 = orc_regret_floor(g, 1, eps);
    /* warm start: regrets proportional to the initial strategy, which then
     * counts as played for iterations 1..t0 in the linear average */
    const double r1 = kappa * orc_regret_floor(g, 0, 1.0), r2 = kappa * orc_regret_floor(g, 1, 1.0);
    const double w0 = 0.5 * (double)t0 * (double)(t0 + 1);
    for (size_t i = 0; i < N1; i++) { R1[i] = r1 * b1[i]; xs[i] = w0 * x[i]; }
    for (size_t i = 0; i < N2; i++) { R2[i] = r2 * b2[i]; ys[i] = w0 * y[i]; }
    double wsum = w0, expl = 0.0;
    for (int t = t0 + 1; t <= t0 + iters; t++) {
        /* player 1: accumulate the strategy played, then update against y */
        for (size_t i = 0; i < N1; i++) xs[i] += t * x[i];
        matvec_one(g, y, g1);
        bottom_up(g, 0, g1, b1, R1, 0);
        regret_match(g, 0, R1, b1, th1);
        orc_seqform(g, 0, b1, x);
        /* player 2 (alternating): against the updated x, gradient -A^T x */
        for (size_t i = 0; i < N2; i++) ys[i] += t * y[i];
        matvec_t_one(g, x, g2);
        for (size_t i = 0; i < N2; i++) g2[i] = -g2[i];
        bottom_up(g, 1, g2, b2, R2, 0);
        regret_match(g, 1, R2, b2, th2);
        orc_seqform(g, 1, b2, y);
        wsum += t;
        if (trace) {
            trace[t - t0 - 1] = 0.0;
            if (trace_every > 0 && (t - t0) % trace_every == 0) {
                for (size_t i = 0; i < N1; i++) xa[i] = xs[i] / wsum;
                for (size_t i = 0; i < N2; i++) ya[i] = ys[i] / wsum;
                trace[t - t0 - 1] = orc_exploitability(g, xa, ya, NULL, NULL);
            }
        }
    }
    for (size_t i = 0; i < N1; i++) xa[i] = wsum > 0 ? xs[i] / wsum : x[i];
    for (size_t i = 0; i < N2; i++) ya[i] = wsum > 0 ? ys[i] / wsum : y[i];
    expl = orc_exploitability(g, xa, ya, NULL, NULL);
    /* sequence form -> behavioural for the average */
    if (avg_beh1 || avg_beh2) {
        for (int p = 0; p < 2; p++) {
            double *dst = p == 0 ? avg_beh1 : avg_beh2;
            double *src = p == 0 ? xa : ya;
            if (!dst) continue;
            int n = g->n[p];
            for (int s = 0; s < n; s++) {
                int par = g->seq_parent[p][s];
                for (int h = 0; h < H; h++) {
                    double den = par < 0 ? 1.0 : src[(size_t)par * H + h];
                    dst[(size_t)s * H + h] = den > 0.0 ? src[(size_t)s * H + h] / den : -1.0;
                }
            }
            /* unreached infosets: uniform */
            for (int i = 0; i < g->np[p]; i++) {
                const onode *nd = &g->nodes[g->pn_tree[p][i]];
                for (int h = 0; h < H; h++)
                    if (dst[(size_t)nd->seq[0] * H + h] < 0.0)
                        for (int a = 0; a < nd->nact; a++) dst[(size_t)nd->seq[a] * H + h] = 1.0 / nd->nact;
            }
        }
    }
    free(b1); free(b2); free(x); free(y); free(R1); free(R2); free(xs); free(ys);
    free(g1); free(g2); free(xa); free(ya);
    return expl;
}
