// Turn endgames (end of Sec. 3): the turn betting round, then at every
// ending of that round that is not a fold the river card (public, drawn
// uniformly from the cards in neither hand nor on the board) and the river
// betting round.  Because the river card is public the payoff matrix is
// block diagonal: one block for the turn round's folds and one river block
// per (ending, river card), each a Kronecker-form river game of its own
// (Prop. 1).  This object builds those games and runs their products as
// members of one batched persistent launch (batch.cu):
//   - the turn round: the turn skeleton on the turn board, its showdowns
//     paying nothing (the game continues), the deal's normalisation beta;
//   - block (ending z, river card r): the river skeleton from z's
//     contributions with the chips left behind, over the turn board's hands,
//     beliefs zero for the hands holding r, strengths with r on the board,
//     and the normalisation beta (N - 2k) in place of its own: the river
//     card's probability 1 / (N - 2k) (N cards left after the turn board, k
//     cards per hand) times the deal's pi folded into lambda.
// Vectors: the batch layout, game after game (turn round first, then the
// blocks, endings in depth-first order of the turn round, river cards
// ascending); within a game [sequence][hs] in that game's hand order
// (kps_turn_hands).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/kps.h"
#include "abi_internal.h"
#include "batch_internal.h"
#include "game.h"

using namespace kps_abi;

struct kps_turn {
    std::vector<kps_game *> games;   // owned: turn round, then the blocks
    std::vector<int> block_end, block_card;
    kps_batch *batch = nullptr;
    int H = 0, hs = 0, nend = 0;
    double beta = 0.0;
};

namespace {

void free_turn(kps_turn *t) {
    if (t->batch) kps_batch_destroy(t->batch);
    for (kps_game *g : t->games) kps_game_destroy(g);
    delete t;
}

}  // namespace

extern "C" {

kps_status kps_turn_create(const kps_turn_spec *sp, kps_turn **out) {
    if (!out) return fail(KPS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!sp || !sp->strength) return fail(KPS_EINVAL, "spec or strength is NULL");
    if (sp->cards_per_hand != 1 && sp->cards_per_hand != 2) return fail(KPS_EINVAL, "cards_per_hand must be 1 or 2");
    if (sp->ranks < 1 || sp->suits < 1 || sp->ranks * sp->suits > 63) return fail(KPS_EINVAL, "deck of 1..63 cards");
    if (sp->nboard < 1 || sp->nboard > KPS_MAX_BOARD) return fail(KPS_EINVAL, "board of 1..8 cards");
    const int deck = sp->ranks * sp->suits, k = sp->cards_per_hand;
    const int N = deck - sp->nboard;
    if (N - 2 * k < 1) return fail(KPS_EINVAL, "no river card left once both hands are dealt");
    kps_turn *t = new (std::nothrow) kps_turn;
    if (!t) return fail(KPS_ENOMEM, "turn object");
    const int H = k == 1 ? N : N * (N - 1) / 2;
    t->H = H;
    // canonical hands (deck minus board, ascending; pairs a < b) by cards
    std::vector<char> on(deck, 0);
    for (int i = 0; i < sp->nboard; ++i) {
        if (sp->board[i] < 0 || sp->board[i] >= deck || on[sp->board[i]]) {
            free_turn(t);
            return fail(KPS_EINVAL, "bad board");
        }
        on[sp->board[i]] = 1;
    }
    std::vector<int> left;
    for (int c = 0; c < deck; ++c)
        if (!on[c]) left.push_back(c);
    std::vector<int> ca, cb;
    for (int i = 0; i < N; ++i) {
        if (k == 1) { ca.push_back(left[i]); cb.push_back(-1); continue; }
        for (int j = i + 1; j < N; ++j) { ca.push_back(left[i]); cb.push_back(left[j]); }
    }
    // the turn round: showdowns pay nothing, strengths distinct (they are
    // not read), the deal's own normalisation
    std::vector<int32_t> idx(H);
    for (int h = 0; h < H; ++h) idx[h] = h;
    kps_game_spec base{};
    base.ranks = sp->ranks;
    base.suits = sp->suits;
    base.cards_per_hand = k;
    base.nboard = sp->nboard;
    for (int i = 0; i < sp->nboard; ++i) base.board[i] = sp->board[i];
    kps_game_spec s0 = base;
    s0.stack[0] = sp->stack[0];
    s0.stack[1] = sp->stack[1];
    s0.contrib0[0] = sp->contrib0[0];
    s0.contrib0[1] = sp->contrib0[1];
    s0.nbet = sp->nbet_turn;
    for (int i = 0; i < sp->nbet_turn && i < KPS_MAX_BETS; ++i) s0.bet_frac[i] = sp->bet_frac_turn[i];
    s0.raise_cap = sp->raise_cap_turn;
    s0.allow_allin = sp->allow_allin_turn;
    s0.mu1 = sp->mu1;
    s0.mu2 = sp->mu2;
    s0.strength = idx.data();
    kps::BuildOptions o0;
    o0.showdown_pays_zero = true;
    kps_game *g0 = nullptr;
    kps_status st = create_game(&s0, &o0, &g0);
    if (st != KPS_OK) { free_turn(t); return st; }
    t->games.push_back(g0);
    t->beta = g0->host.beta;
    t->hs = g0->host.hs;
    const double beta_block = t->beta * (double)(N - 2 * k);
    // the river blocks
    std::vector<double> m1(H), m2(H);
    std::vector<int32_t> str(H);
    for (size_t ti = 0; ti < g0->host.terms.size(); ++ti) {
        const kps::Terminal &z = g0->host.terms[ti];
        if (z.kind != 1) continue;
        const double c = z.c1;
        double behind[2];
        for (int p = 0; p < 2; ++p) {
            behind[p] = sp->contrib0[p] + sp->stack[p] - c;
            if (!(behind[p] > 0.0)) {
                free_turn(t);
                return fail(KPS_ENOTSUP, "an ending of the turn round leaves a player all in (no river betting)");
            }
        }
        for (int r = 0; r < deck; ++r) {
            if (on[r]) continue;
            for (int h = 0; h < H; ++h) {
                const bool holds = ca[h] == r || cb[h] == r;
                m1[h] = holds ? 0.0 : (sp->mu1 ? sp->mu1[h] : 1.0);
                m2[h] = holds ? 0.0 : (sp->mu2 ? sp->mu2[h] : 1.0);
                // hands holding the river card: distinct strengths below the
                // others (zero beliefs; no tie group forms)
                str[h] = holds ? -1 - h : sp->strength[(size_t)r * H + h];
            }
            kps_game_spec sr = base;
            sr.stack[0] = behind[0];
            sr.stack[1] = behind[1];
            sr.contrib0[0] = c;
            sr.contrib0[1] = c;
            sr.nbet = sp->nbet_river;
            for (int i = 0; i < sp->nbet_river && i < KPS_MAX_BETS; ++i) sr.bet_frac[i] = sp->bet_frac_river[i];
            sr.raise_cap = sp->raise_cap_river;
            sr.allow_allin = sp->allow_allin_river;
            sr.mu1 = m1.data();
            sr.mu2 = m2.data();
            sr.strength = str.data();
            kps::BuildOptions orr;
            orr.beta = beta_block;
            kps_game *gb = nullptr;
            st = create_game(&sr, &orr, &gb);
            if (st != KPS_OK) { free_turn(t); return st; }
            t->games.push_back(gb);
            t->block_end.push_back(t->nend);
            t->block_card.push_back(r);
        }
        ++t->nend;
    }
    st = kps_batch_create(t->games.data(), (int32_t)t->games.size(), &t->batch);
    if (st != KPS_OK) { free_turn(t); return st; }
    *out = t;
    return KPS_OK;
}

kps_status kps_turn_destroy(kps_turn *t) {
    if (t) free_turn(t);
    return KPS_OK;
}

kps_status kps_turn_info(const kps_turn *t, int64_t *info) {
    if (!t || !info) return fail(KPS_EINVAL, "NULL argument");
    info[0] = t->H;
    info[1] = t->hs;
    int64_t n[2] = {0, 0};
    for (const kps_game *g : t->games)
        for (int p = 0; p < 2; ++p) n[p] += g->host.n[p];
    info[2] = n[0];
    info[3] = n[1];
    info[4] = t->nend;
    info[5] = (int64_t)t->block_card.size();
    info[6] = (int64_t)t->games.size();
    info[7] = t->games.empty() ? 0 : t->games[0]->host.n[0];
    info[8] = t->games.empty() ? 0 : t->games[0]->host.n[1];
    return KPS_OK;
}

kps_status kps_turn_offsets(const kps_turn *t, int32_t player, int64_t *off) {
    if (!t) return fail(KPS_EINVAL, "turn is NULL");
    return kps_batch_offsets(t->batch, player, off);
}

kps_status kps_turn_block(const kps_turn *t, int32_t block, int32_t *ending, int32_t *river_card, int32_t *canon) {
    if (!t || block < 0 || block >= (int32_t)t->games.size()) return fail(KPS_EINVAL, "bad block");
    if (ending) *ending = block == 0 ? -1 : t->block_end[block - 1];
    if (river_card) *river_card = block == 0 ? -1 : t->block_card[block - 1];
    if (canon) return kps_game_hands(t->games[block], nullptr, canon);
    return KPS_OK;
}

kps_status kps_turn_matvec_A(kps_turn *t, const void *y, void *out, kps_dtype dt, void *stream) {
    if (!t) return fail(KPS_EINVAL, "turn is NULL");
    return kps_batch_matvec_A(t->batch, y, out, dt, stream);
}

kps_status kps_turn_matvec_AT(kps_turn *t, const void *x, void *out, kps_dtype dt, void *stream) {
    if (!t) return fail(KPS_EINVAL, "turn is NULL");
    return kps_batch_matvec_AT(t->batch, x, out, dt, stream);
}

kps_status kps_turn_batch(kps_turn *t, kps_batch **batch) {
    if (!t || !batch) return fail(KPS_EINVAL, "NULL argument");
    *batch = t->batch;
    return KPS_OK;
}

}  // extern "C"
