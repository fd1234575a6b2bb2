// Host-side game and factor builder (runs once per game).
//
// Builds, from a kps_game_spec:
//   * the skeleton betting tree of the river endgame (Sec. 3, Fig. 1; the
//     betting rules of the appendix and the pot arithmetic of its worked
//     example), its sequences and terminal list;
//   * the hand list, the strength order (the order in which the rows of W
//     read -1 ... 0 ... +1, Sec. 4) and its tie groups;
//   * lambda_i = mu_i / sqrt(beta) of Prop. 1, with beta obtained by
//     inclusion-exclusion over cards instead of a sum over hand pairs;
//   * the terminal-pair lists grouped by output sequence, which carry the
//     entries of F and S (Sec. 3);
//   * the Technique B sizes of Sec. 4 (lazily, see technique_b_counts).
#include "game.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace kps {

namespace {

constexpr int kMaxActions = KPS_MAX_BETS + 3;
constexpr int kMaxTreeNodes = 1 << 22;

// A node waiting on the explicit depth-first stack.
struct Pending {
    int who;           // 0/1 decision of that player, 2 fold terminal, 3 showdown
    int folder;
    double c[2];
    int aggressive;    // aggressive actions so far in the round
    bool after_check;  // previous action was a check
    int last[2];       // last sequence of each player so far
};

struct Choice {
    int code;
    double contrib;    // actor's contribution after the action
};

// Actions of a decision node, in the library's action order.
// Situation of the acting player for the betting menu (kps_bet_menu).
int situation(const Pending &nd) {
    if (nd.aggressive == 0) return nd.after_check ? 1 : 0;
    return std::min(nd.aggressive + 1, KPS_SITUATIONS - 1);
}

int legal_actions(const kps_game_spec &s, const kps_bet_menu *menu, const Pending &nd, Choice *out) {
    const int me = nd.who, opp = 1 - nd.who;
    const double my_max = s.contrib0[me] + s.stack[me];
    const double opp_max = s.contrib0[opp] + s.stack[opp];
    const double all_in = std::min(my_max, opp_max);
    const bool facing = nd.c[me] < nd.c[opp];
    const bool may_raise = s.raise_cap < 0 || nd.aggressive < s.raise_cap;
    int n = 0;
    if (facing) {
        out[n++] = {kFold, nd.c[me]};
        out[n++] = {kCheckCall, std::min(nd.c[opp], my_max)};
    } else {
        out[n++] = {kCheckCall, nd.c[me]};
    }
    double raise_to[kMaxActions];
    int nr = 0;
    const double level = facing ? nd.c[opp] : nd.c[me];
    if (may_raise && all_in > level) {
        const int sit = situation(nd);
        const int nbet = menu ? menu->nbet[me][sit] : s.nbet;
        const double *frac = menu ? menu->bet_frac[me][sit] : s.bet_frac;
        for (int i = 0; i < nbet; ++i) {
            // match the opponent, then add the fraction of the matched pot
            double target = facing ? nd.c[opp] + frac[i] * (2.0 * nd.c[opp])
                                   : nd.c[me] + frac[i] * (nd.c[me] + nd.c[opp]);
            raise_to[nr++] = target >= all_in ? all_in : target;
        }
        if (s.allow_allin) raise_to[nr++] = all_in;
    }
    for (int i = 1; i < nr; ++i)   // ascending amounts
        for (int j = i; j > 0 && raise_to[j] < raise_to[j - 1]; --j) std::swap(raise_to[j], raise_to[j - 1]);
    for (int i = 0; i < nr; ++i)
        if (i == 0 || raise_to[i] != raise_to[i - 1]) out[n++] = {kAggressive, raise_to[i]};
    return n;
}

std::string validate(const kps_game_spec *s, kps_status *code) {
    *code = KPS_EINVAL;
    if (!s) return "spec is NULL";
    if (s->cards_per_hand != 1 && s->cards_per_hand != 2) return "cards_per_hand must be 1 or 2";
    if (s->ranks < 1 || s->suits < 1) return "ranks and suits must be positive";
    if (s->nboard < 0 || s->nboard > KPS_MAX_BOARD) return "nboard out of range";
    if (s->nbet < 0 || s->nbet > KPS_MAX_BETS) return "nbet out of range";
    if (!s->strength) return "strength is NULL";
    for (int p = 0; p < 2; ++p) {
        if (!(s->contrib0[p] > 0.0) || !std::isfinite(s->contrib0[p]))
            return "contrib0 must be positive and finite";
        if (!(s->stack[p] >= 0.0) || !std::isfinite(s->stack[p]))
            return "stack must be non-negative and finite";
    }
    for (int i = 0; i < s->nbet; ++i)
        if (!(s->bet_frac[i] > 0.0) || !std::isfinite(s->bet_frac[i]))
            return "bet fractions must be positive and finite";
    if (s->menu)
        for (int p = 0; p < 2; ++p)
            for (int k = 0; k < KPS_SITUATIONS; ++k) {
                const int n = s->menu->nbet[p][k];
                if (n < 0 || n > KPS_MAX_BETS) return "menu nbet out of range";
                for (int i = 0; i < n; ++i)
                    if (!(s->menu->bet_frac[p][k][i] > 0.0) || !std::isfinite(s->menu->bet_frac[p][k][i]))
                        return "menu bet fractions must be positive and finite";
            }
    const int deck = s->ranks * s->suits;
    if (deck > 63) {
        *code = KPS_ENOTSUP;
        return "decks above 63 cards are not supported";
    }
    std::vector<char> used(deck, 0);
    for (int i = 0; i < s->nboard; ++i) {
        int c = s->board[i];
        if (c < 0 || c >= deck) return "board card out of range";
        if (used[c]) return "board card repeated";
        used[c] = 1;
    }
    if (deck - s->nboard < 2 * s->cards_per_hand) return "not enough cards left to deal two hands";
    return "";
}

std::string build_tree(HostGame &g) {
    const kps_game_spec &s = g.spec;
    std::vector<Pending> stack;
    Pending root{};
    root.who = 0;
    root.folder = -1;
    root.c[0] = s.contrib0[0];
    root.c[1] = s.contrib0[1];
    root.last[0] = root.last[1] = -1;
    stack.push_back(root);
    long visited = 0;
    Choice acts[kMaxActions];
    while (!stack.empty()) {
        Pending nd = stack.back();
        stack.pop_back();
        if (++visited > kMaxTreeNodes) return "betting tree too large";
        if (nd.who >= 2) {
            if (nd.last[0] < 0 || nd.last[1] < 0) return "a terminal follows no action of some player";
            Terminal t{nd.last[0], nd.last[1], nd.who == 2 ? 0 : 1, nd.who == 2 ? nd.folder : -1,
                       nd.c[0], nd.c[1]};
            g.terms.push_back(t);
            continue;
        }
        const int me = nd.who;
        const int na = legal_actions(s, g.has_menu ? &g.menu : nullptr, nd, acts);
        const int node_id = g.nodes[me]++;
        g.nodes_nact[me].push_back(na);
        const int first = g.n[me];
        for (int a = 0; a < na; ++a) {
            g.seqs[me].push_back(Sequence{node_id, nd.last[me], acts[a].code, acts[a].contrib});
            g.n[me]++;
        }
        // children, pushed in reverse so that action 0 is expanded first
        for (int a = na - 1; a >= 0; --a) {
            Pending ch = nd;
            ch.c[me] = acts[a].contrib;
            ch.last[me] = first + a;
            ch.after_check = false;
            if (acts[a].code == kFold) {
                ch.who = 2;
                ch.folder = me;
            } else if (acts[a].code == kCheckCall) {
                const bool is_call = nd.c[me] < nd.c[1 - me];
                if (is_call || nd.after_check) {
                    ch.who = 3;
                } else {
                    ch.who = 1 - me;
                    ch.after_check = true;
                }
            } else {
                ch.who = 1 - me;
                ch.aggressive = nd.aggressive + 1;
            }
            stack.push_back(ch);
        }
    }
    g.T = (int)g.terms.size();
    for (const Terminal &t : g.terms) (t.kind == 0 ? g.TF : g.TS)++;
    return "";
}

void build_pairs(HostGame &g) {
    auto fill = [&](PairCsr &csr, bool transpose) {
        const int rows = transpose ? g.n[1] : g.n[0];
        csr.rowptr.assign(rows + 1, 0);
        for (const Terminal &t : g.terms) csr.rowptr[(transpose ? t.s2 : t.s1) + 1]++;
        for (int r = 0; r < rows; ++r) csr.rowptr[r + 1] += csr.rowptr[r];
        csr.col.assign(g.T, 0);
        csr.kind.assign(g.T, 0);
        csr.coef.assign(g.T, 0.0);
        std::vector<int> fillp(csr.rowptr.begin(), csr.rowptr.end() - 1);
        for (const Terminal &t : g.terms) {
            const int r = transpose ? t.s2 : t.s1;
            const int at = fillp[r]++;
            csr.col[at] = transpose ? t.s1 : t.s2;
            csr.kind[at] = t.kind;
            if (t.kind == 0) {
                csr.coef[at] = t.folder == 0 ? -t.c1 : t.c2;   // entry of F
            } else {
                const double pot = std::min(t.c1, t.c2);       // entry of S
                // W is antisymmetric, so the transposed product flips the sign
                csr.coef[at] = transpose ? -pot : pot;
            }
        }
    };
    fill(g.csr_A, false);
    fill(g.csr_AT, true);
}

std::string build_hands(HostGame &g, const double *mu1_canon, const double *mu2_canon,
                        const int32_t *strength_canon) {
    const kps_game_spec &s = g.spec;
    const int deck = s.ranks * s.suits;
    std::vector<char> on_board(deck, 0);
    for (int i = 0; i < s.nboard; ++i) on_board[s.board[i]] = 1;
    for (int c = 0; c < deck; ++c)
        if (!on_board[c]) g.slot_card.push_back(c);
    g.ncards = (int)g.slot_card.size();
    g.k = s.cards_per_hand;
    // canonical hands as slot pairs
    std::vector<int> ca, cb;
    if (g.k == 1) {
        for (int i = 0; i < g.ncards; ++i) { ca.push_back(i); cb.push_back(g.ncards); }
    } else {
        for (int i = 0; i < g.ncards; ++i)
            for (int j = i + 1; j < g.ncards; ++j) { ca.push_back(i); cb.push_back(j); }
    }
    g.H = (int)ca.size();
    g.hs = (g.H + 7) / 8 * 8;
    // library order: ascending strength, ties by canonical index
    g.canon.resize(g.H);
    std::iota(g.canon.begin(), g.canon.end(), 0);
    std::stable_sort(g.canon.begin(), g.canon.end(),
                     [&](int x, int y) { return strength_canon[x] < strength_canon[y]; });
    g.strength.resize(g.H);
    g.hand_slots.resize(2 * (size_t)g.H);
    g.mu1.resize(g.H);
    g.mu2.resize(g.H);
    for (int p = 0; p < g.H; ++p) {
        const int h = g.canon[p];
        g.strength[p] = strength_canon[h];
        g.hand_slots[2 * p] = ca[h];
        g.hand_slots[2 * p + 1] = cb[h];
        g.mu1[p] = mu1_canon ? mu1_canon[h] : 1.0;
        g.mu2[p] = mu2_canon ? mu2_canon[h] : 1.0;
        if (!(g.mu1[p] >= 0.0) || !std::isfinite(g.mu1[p]) || !(g.mu2[p] >= 0.0) ||
            !std::isfinite(g.mu2[p]))
            return "beliefs must be finite and non-negative";
    }
    // beta = sum over compatible pairs of mu1 mu2, by inclusion-exclusion:
    // all pairs, minus pairs sharing a card, plus pairs sharing both cards
    // (only a hand with itself shares both).
    double s1 = 0.0, s2 = 0.0, same = 0.0;
    std::vector<double> per1(g.ncards + 1, 0.0), per2(g.ncards + 1, 0.0);
    for (int p = 0; p < g.H; ++p) {
        s1 += g.mu1[p];
        s2 += g.mu2[p];
        same += g.mu1[p] * g.mu2[p];
        for (int j = 0; j < g.k; ++j) {
            per1[g.hand_slots[2 * p + j]] += g.mu1[p];
            per2[g.hand_slots[2 * p + j]] += g.mu2[p];
        }
    }
    double shared = 0.0;
    for (int c = 0; c < g.ncards; ++c) shared += per1[c] * per2[c];
    g.beta = g.k == 1 ? s1 * s2 - same : s1 * s2 - shared + same;
    if (!(g.beta > 0.0) || !std::isfinite(g.beta)) return "beliefs give no compatible deal";
    const double rs = 1.0 / std::sqrt(g.beta);
    g.lam1.resize(g.H);
    g.lam2.resize(g.H);
    for (int p = 0; p < g.H; ++p) {
        g.lam1[p] = g.mu1[p] * rs;
        g.lam2[p] = g.mu2[p] * rs;
    }
    // tie groups and the packed per-hand records
    g.group_lo.resize(g.H);
    g.group_hi.resize(g.H);
    g.hinfo.resize(g.H);
    g.max_tie = 0;
    for (int lo = 0; lo < g.H;) {
        int hi = lo;
        while (hi + 1 < g.H && g.strength[hi + 1] == g.strength[lo]) ++hi;
        const int len = hi - lo + 1;
        g.max_tie = std::max(g.max_tie, len);
        for (int p = lo; p <= hi; ++p) {
            g.group_lo[p] = lo;
            g.group_hi[p] = hi;
            g.hinfo[p] = pack_hinfo(g.hand_slots[2 * p], g.hand_slots[2 * p + 1], len > 1,
                                    len > 1 && p == hi, p - lo);
        }
        lo = hi + 1;
    }
    for (int p = 0; p + 1 < g.H; ++p) {
        const bool untied = g.group_lo[p] == g.group_hi[p] && g.group_lo[p + 1] == g.group_hi[p + 1];
        bool disjoint = true;
        for (int i = 0; i < g.k; ++i)
            for (int j = 0; j < g.k; ++j)
                if (g.hand_slots[2 * p + i] == g.hand_slots[2 * (p + 1) + j]) disjoint = false;
        if (untied && disjoint) g.hinfo[p] |= 1u << 14;
        if (disjoint) g.hinfo[p] |= 1u << 15;
    }
    if (g.max_tie > 65535) return "tie group too long";
    return "";
}

}  // namespace

std::string build_game(const kps_game_spec *spec, HostGame &g, kps_status *code, const BuildOptions *opt) {
    std::string err = validate(spec, code);
    if (!err.empty()) return err;
    g.spec = *spec;
    g.spec.mu1 = g.spec.mu2 = nullptr;
    g.spec.strength = nullptr;
    g.spec.menu = nullptr;
    if (spec->menu) {
        g.menu = *spec->menu;
        g.has_menu = true;
    }
    g.pot0 = spec->contrib0[0] + spec->contrib0[1];
    *code = KPS_EINVAL;
    err = build_hands(g, spec->mu1, spec->mu2, spec->strength);
    if (!err.empty()) return err;
    if (opt && opt->beta > 0.0) {
        if (!std::isfinite(opt->beta)) return "beta must be finite";
        g.beta = opt->beta;
        const double rs = 1.0 / std::sqrt(g.beta);
        for (int p = 0; p < g.H; ++p) {
            g.lam1[p] = g.mu1[p] * rs;
            g.lam2[p] = g.mu2[p] * rs;
        }
    }
    err = build_tree(g);
    if (!err.empty()) {
        if (err == "betting tree too large") *code = KPS_ENOTSUP;
        return err;
    }
    build_pairs(g);
    if (opt && opt->showdown_pays_zero)
        for (PairCsr *csr : {&g.csr_A, &g.csr_AT})
            for (size_t e = 0; e < csr->kind.size(); ++e)
                if (csr->kind[e] == 1) csr->coef[e] = 0.0;
    *code = KPS_OK;
    return "";
}

std::vector<int> chunk_bounds(const HostGame &g, int parts) {
    std::vector<int> b(parts + 1, g.H);
    b[0] = 0;
    for (int i = 1; i < parts; ++i) {
        int at = (int)((int64_t)g.H * i / parts);
        if (at < b[i - 1]) at = b[i - 1];
        if (at < g.H) at = g.group_lo[at] > b[i - 1] ? g.group_lo[at] : g.group_hi[at] + 1;
        if (at > g.H) at = g.H;
        b[i] = std::max(at, b[i - 1]);
    }
    b[parts] = g.H;
    return b;
}

std::vector<std::pair<int, int>> tie_tiles(const HostGame &g, int parts, int tile,
                                           std::vector<int> &tchunk, bool from_end) {
    std::vector<int> cb = chunk_bounds(g, parts);
    std::vector<std::pair<int, int>> tiles;
    tchunk.assign(parts + 1, 0);
    std::vector<std::pair<int, int>> rev;
    for (int k = 0; k < parts; ++k) {
        tchunk[k] = (int)tiles.size();
        if (!from_end) {
            int s = cb[k];
            while (s < cb[k + 1]) {
                int e = std::min(s + tile, cb[k + 1]);
                // back off to a tie-group boundary unless the tile ends the chunk
                if (e < cb[k + 1] && g.group_lo[e] > s) e = g.group_lo[e];
                tiles.emplace_back(s, e - s);
                s = e;
            }
            continue;
        }
        rev.clear();
        int e = cb[k + 1];
        while (e > cb[k]) {
            int s = std::max(e - tile, cb[k]);
            // move up to a tie-group boundary unless the tile starts the chunk
            if (s > cb[k] && g.group_lo[s] < s && g.group_hi[s] + 1 < e) s = g.group_hi[s] + 1;
            rev.emplace_back(s, e - s);
            e = s;
        }
        tiles.insert(tiles.end(), rev.rbegin(), rev.rend());
    }
    tchunk[parts] = (int)tiles.size();
    return tiles;
}

void tie_work(const HostGame &g, const std::vector<std::pair<int, int>> &tiles, std::vector<std::pair<int, int>> &work,
              std::vector<uint32_t> &trip) {
    work.assign(tiles.size(), std::make_pair(0, 0));
    trip.clear();
    for (size_t t = 0; t < tiles.size(); ++t) {
        const int s0 = tiles[t].first, len = tiles[t].second;
        const int first = (int)trip.size();
        for (int q = s0; q < s0 + len; ++q) {
            if (g.group_hi[q] == g.group_lo[q]) continue;
            const int qa = g.hand_slots[2 * q], qb = g.hand_slots[2 * q + 1];
            for (int r = g.group_lo[q]; r <= g.group_hi[q]; ++r) {
                if (r == q) continue;
                const int ra = g.hand_slots[2 * r], rb = g.hand_slots[2 * r + 1];
                bool share = qa == ra;
                if (g.k == 2) share = share || qa == rb || qb == ra || qb == rb;
                if (share) continue;
                trip.push_back((uint32_t)(q - s0) | ((uint32_t)(r - s0) << 5) | ((uint32_t)(r > q) << 10));
            }
        }
        work[t] = std::make_pair(first, (int)trip.size() - first);
    }
}

// Sizes of Technique B, counted from the structure of its factors:
//   Ahat = -(Lambda1 Hx Lambda2) (x) F,  U = [Lambda1 (x) I | lambda1 (x) I],
//   M = diag(D (x) I, I),  V = [(Lambda2 Y^T) (x) S^T | lambda2 (x) F^T],
//   Y = D W with D lower bidiagonal (1, -1) in the strength order.
// Postprocessing (Sec. 4): a zero column j of V makes y_j a copy of the
// variable it is chained to by D (or zero at the head of a chain); its row
// of M disappears and its column of U merges into that variable's column.
void technique_b_counts(HostGame &g) {
    if (g.counts_done) return;
    const int H = g.H, n1 = g.n[0], N = g.ncards, k = g.k;
    // hands with nonzero beliefs
    std::vector<char> nz1(H), nz2(H);
    int64_t N1 = 0, N2 = 0, both = 0;
    std::vector<int64_t> card1(N + 1, 0), card2(N + 1, 0);
    for (int p = 0; p < H; ++p) {
        nz1[p] = g.mu1[p] != 0.0;
        nz2[p] = g.mu2[p] != 0.0;
        N1 += nz1[p];
        N2 += nz2[p];
        both += nz1[p] && nz2[p];
        for (int j = 0; j < k; ++j) {
            card1[g.hand_slots[2 * p + j]] += nz1[p];
            card2[g.hand_slots[2 * p + j]] += nz2[p];
        }
    }
    int64_t sharing = 0;
    for (int c = 0; c < N; ++c) sharing += card1[c] * card2[c];
    const int64_t compat = k == 1 ? N1 * N2 - both : N1 * N2 - sharing + both;
    const int64_t incompat = N1 * N2 - compat;
    // compatible pairs with equal strength, group by group
    int64_t tied = 0;
    auto share = [&](int x, int y) {
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j)
                if (g.hand_slots[2 * x + i] == g.hand_slots[2 * y + j]) return true;
        return false;
    };
    for (int lo = 0; lo < H; lo = g.group_hi[lo] + 1)
        for (int x = lo; x <= g.group_hi[lo]; ++x)
            for (int y = lo; y <= g.group_hi[lo]; ++y)
                if (nz1[x] && nz2[y] && !share(x, y)) ++tied;
    // rows of Y: W[i][.] - W[i-1][.] differs only where a card is shared with
    // hand i or i-1, or where the strength lies between theirs
    std::vector<std::vector<int>> by_card(N + 1);
    for (int p = 0; p < H; ++p)
        for (int j = 0; j < k; ++j) by_card[g.hand_slots[2 * p + j]].push_back(p);
    auto wval = [&](int i, int j) -> int {
        if (i < 0 || share(i, j)) return 0;
        return (g.strength[i] > g.strength[j]) - (g.strength[i] < g.strength[j]);
    };
    std::vector<int> mark(H, -1);
    std::vector<char> yzero(H);
    int64_t nnzY = 0;
    for (int i = 0; i < H; ++i) {
        int cnt = 0;
        auto visit = [&](int j) {
            if (mark[j] == i) return;
            mark[j] = i;
            if (nz2[j] && wval(i, j) != wval(i - 1, j)) ++cnt;
        };
        const int lo = i > 0 ? g.group_lo[i - 1] : 0;
        for (int j = lo; j <= g.group_hi[i]; ++j) visit(j);
        if (i == 0)
            for (int j = 0; j < H; ++j) visit(j);
        for (int side = 0; side < 2; ++side) {
            const int h = i - side;
            if (h < 0) continue;
            for (int j = 0; j < k; ++j)
                for (int q : by_card[g.hand_slots[2 * h + j]]) visit(q);
        }
        nnzY += cnt;
        yzero[i] = cnt == 0;
    }
    std::vector<char> has_f(n1, 0), has_s(n1, 0);
    for (const Terminal &t : g.terms) (t.kind == 0 ? has_f : has_s)[t.s1] = 1;
    int64_t *c = g.counts;
    c[0] = compat * g.TF + (compat - tied) * g.TS;
    c[1] = incompat * g.TF;
    c[2] = 2 * N1 * n1;
    c[3] = (int64_t)(2 * H - 1) * n1 + n1;
    c[4] = nnzY * g.TS + N2 * g.TF;
    int64_t U = c[2], M = c[3];
    for (int a = 0; a < n1; ++a) {
        bool chained = false;            // row i still points at a live variable
        for (int i = 0; i < H; ++i) {
            const bool zero_col = !has_s[a] || yzero[i];
            if (!zero_col) {
                chained = true;
                continue;
            }
            const bool off = i > 0 && chained;
            M -= 1 + (off ? 1 : 0);
            if (!off) {
                U -= nz1[i] ? 1 : 0;
                if (i + 1 < H) M -= 1;
                chained = false;
            }
        }
        if (!has_f[a] || N2 == 0) {
            M -= 1;
            U -= N1;
        }
    }
    c[5] = c[1];
    c[6] = U;
    c[7] = M;
    c[8] = c[4];
    g.counts_done = true;
}

namespace {

// Appends row r of a CSR under construction from (column, value) pairs:
// sorted by column, equal columns summed, zeros dropped.
void csr_push_row(Csr &c, std::vector<std::pair<int, double>> &e) {
    std::sort(e.begin(), e.end(), [](const auto &x, const auto &y) { return x.first < y.first; });
    for (size_t i = 0; i < e.size();) {
        size_t j = i;
        double v = 0.0;
        for (; j < e.size() && e[j].first == e[i].first; ++j) v += e[j].second;
        if (v != 0.0) {
            c.col.push_back(e[i].first);
            c.val.push_back(v);
        }
        i = j;
    }
    c.rowptr.push_back((int)c.col.size());
    e.clear();
}

}  // namespace

void technique_b_factors(const HostGame &g, TechniqueB &f) {
    const int H = g.H, hs = g.hs, n1 = g.n[0], n2 = g.n[1], N = g.ncards, k = g.k;
    const int R = n1 * hs, C = n2 * hs, m = n1 * hs + n1;
    auto share = [&](int x, int y) {
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j)
                if (g.hand_slots[2 * x + i] == g.hand_slots[2 * y + j]) return true;
        return false;
    };
    std::vector<std::vector<int>> by_card(N + 1);
    for (int p = 0; p < H; ++p)
        for (int j = 0; j < k; ++j) by_card[g.hand_slots[2 * p + j]].push_back(p);
    // W[i][j]: +1 if hand i beats a compatible hand j, -1 if it loses, 0 for
    // ties and card overlaps (library order is the strength order).
    auto wval = [&](int i, int j) -> int {
        if (i < 0 || share(i, j)) return 0;
        return (g.strength[i] > g.strength[j]) - (g.strength[i] < g.strength[j]);
    };
    // Y = D W row by row.  Row i differs from row i-1 only in the columns of
    // strength between theirs (positions group_lo[i-1] .. group_hi[i]) and
    // in the hands sharing a card with i or i-1; row 0 is W's first row.
    std::vector<std::vector<std::pair<int, int>>> Y(H);
    std::vector<int> mark(H, -1), cand;
    for (int i = 0; i < H; ++i) {
        cand.clear();
        auto visit = [&](int j) {
            if (mark[j] != i) {
                mark[j] = i;
                cand.push_back(j);
            }
        };
        for (int j = i > 0 ? g.group_lo[i - 1] : 0; j <= g.group_hi[i]; ++j) visit(j);
        if (i == 0)
            for (int j = 0; j < H; ++j) visit(j);
        for (int side = 0; side < 2; ++side) {
            const int h = i - side;
            if (h < 0) continue;
            for (int j = 0; j < k; ++j)
                for (int q : by_card[g.hand_slots[2 * h + j]]) visit(q);
        }
        std::sort(cand.begin(), cand.end());
        for (int j : cand) {
            if (g.mu2[j] == 0.0) continue;
            const int y = wval(i, j) - wval(i - 1, j);
            if (y != 0) Y[i].emplace_back(j, y);
        }
    }
    const PairCsr &pc = g.csr_A;          // terminals by player-1 sequence
    std::vector<std::pair<int, double>> e;
    auto start = [](Csr &c, int rows, int cols) {
        c = Csr();
        c.rows = rows;
        c.cols = cols;
        c.rowptr.push_back(0);
    };
    // Ahat: card-overlapping pairs of every fold terminal
    start(f.ahat, R, C);
    for (int s1 = 0; s1 < n1; ++s1)
        for (int h1 = 0; h1 < hs; ++h1) {
            if (h1 < H && g.lam1[h1] != 0.0)
                for (int t = pc.rowptr[s1]; t < pc.rowptr[s1 + 1]; ++t) {
                    if (pc.kind[t] != 0) continue;
                    for (int j = 0; j < k; ++j)
                        for (int h2 : by_card[g.hand_slots[2 * h1 + j]]) {
                            // a hand sharing both cards with h1 is h1 itself:
                            // list it once
                            if (j == 1 && h2 == h1) continue;
                            if (g.lam2[h2] != 0.0)
                                e.emplace_back(pc.col[t] * hs + h2, -pc.coef[t] * g.lam1[h1] * g.lam2[h2]);
                        }
                }
            csr_push_row(f.ahat, e);
        }
    // U = [I (x) Lambda1 | I (x) lambda1]
    start(f.u, R, m);
    for (int s1 = 0; s1 < n1; ++s1)
        for (int h1 = 0; h1 < hs; ++h1) {
            if (h1 < H && g.lam1[h1] != 0.0) {
                e.emplace_back(s1 * hs + h1, g.lam1[h1]);
                e.emplace_back(n1 * hs + s1, g.lam1[h1]);
            }
            csr_push_row(f.u, e);
        }
    // M = diag(I (x) D, I)
    start(f.m, m, m);
    for (int s1 = 0; s1 < n1; ++s1)
        for (int h = 0; h < hs; ++h) {
            if (h > 0 && h < H) e.emplace_back(s1 * hs + h - 1, -1.0);
            e.emplace_back(s1 * hs + h, 1.0);
            csr_push_row(f.m, e);
        }
    for (int s1 = 0; s1 < n1; ++s1) {
        e.emplace_back(n1 * hs + s1, 1.0);
        csr_push_row(f.m, e);
    }
    // V^T = [S (x) (Y Lambda2) ; F (x) lambda2^T]
    start(f.vt, m, C);
    for (int s1 = 0; s1 < n1; ++s1)
        for (int h = 0; h < hs; ++h) {
            if (h < H)
                for (int t = pc.rowptr[s1]; t < pc.rowptr[s1 + 1]; ++t) {
                    if (pc.kind[t] != 1) continue;
                    for (const auto &yj : Y[h]) e.emplace_back(pc.col[t] * hs + yj.first, pc.coef[t] * yj.second * g.lam2[yj.first]);
                }
            csr_push_row(f.vt, e);
        }
    for (int s1 = 0; s1 < n1; ++s1) {
        for (int t = pc.rowptr[s1]; t < pc.rowptr[s1 + 1]; ++t) {
            if (pc.kind[t] != 0) continue;
            for (int h2 = 0; h2 < H; ++h2)
                if (g.lam2[h2] != 0.0) e.emplace_back(pc.col[t] * hs + h2, pc.coef[t] * g.lam2[h2]);
        }
        csr_push_row(f.vt, e);
    }
}

}  // namespace kps
