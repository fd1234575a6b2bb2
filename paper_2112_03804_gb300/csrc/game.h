// Internal host-side game representation of the Kronecker payoff library.
#pragma once

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "../../include/kps.h"

namespace kps {

enum ActionCode { kFold = 0, kCheckCall = 1, kAggressive = 2 };

struct Terminal {
    int s1, s2;        // last sequence of each player on the path
    int kind;          // 0 fold, 1 showdown
    int folder;        // player who folded, -1 at a showdown
    double c1, c2;     // pot contributions
};

struct Sequence {
    int node;          // decision node (index among the owner's nodes)
    int parent;        // parent sequence of that node, -1 = empty sequence
    int action;        // ActionCode
    double amount;     // owner's contribution after the action
};

// Terminal pairs grouped by output sequence: row r lists the terminals whose
// output-side sequence is r; `col` is the input-side sequence.
struct PairCsr {
    std::vector<int> rowptr;
    std::vector<int> col;
    std::vector<int> kind;         // 0 fold, 1 showdown
    std::vector<double> coef;      // F_t for folds, +-S_t for showdowns
};

// Per-hand record used by the kernels, library (strength) order:
//   bits 0-5   slot of the first card  (index into the cards left after the board)
//   bits 6-11  slot of the second card (== ncards for one-card hands)
//   bit  12    member of a tie group of length >= 2
//   bit  13    last member of such a group
//   bit  14    this hand and the next are both untied and share no card, so
//              a scan may update their per-card sums together
//   bit  15    this hand and the next share no card (ties allowed)
//   bits 16-31 offset of the hand inside its tie group
inline uint32_t pack_hinfo(int a, int b, bool tied, bool last, int off) {
    return (uint32_t)a | ((uint32_t)b << 6) | ((uint32_t)tied << 12) | ((uint32_t)last << 13) |
           ((uint32_t)off << 16);
}

struct HostGame {
    kps_game_spec spec{};          // copy; the pointer fields are cleared
    kps_bet_menu menu{};           // copy of *spec.menu when has_menu
    bool has_menu = false;
    int H = 0, hs = 0, k = 0, ncards = 0;
    int n[2] = {0, 0};
    int nodes[2] = {0, 0};
    int T = 0, TF = 0, TS = 0, max_tie = 0;
    double beta = 0.0, pot0 = 0.0;

    std::vector<int> slot_card;     // slot -> card id (cards left, increasing id)
    std::vector<int> hand_slots;    // library order, 2 per hand (second = ncards for k = 1)
    std::vector<int> canon;         // library order -> canonical index
    std::vector<int> strength;      // library order
    std::vector<double> mu1, mu2;   // library order
    std::vector<double> lam1, lam2; // library order, mu / sqrt(beta)
    std::vector<uint32_t> hinfo;    // library order, see pack_hinfo
    std::vector<int> group_lo, group_hi;  // tie group [lo, hi] of every position

    std::vector<Terminal> terms;
    std::vector<Sequence> seqs[2];
    std::vector<int> nodes_nact[2];
    PairCsr csr_A;                  // rows = player-1 sequences (A * y)
    PairCsr csr_AT;                 // rows = player-2 sequences (A^T * x)

    bool counts_done = false;
    int64_t counts[9] = {0};        // nnz A, Ahat, U, M, V, pp Ahat, U, M, V
};

// Internal build options for games that are parts of a larger game (the
// river blocks of a turn endgame, its turn round): a chance normalisation
// given from outside (lambda_i = mu_i / sqrt(beta)) instead of the game's
// own, and showdowns that pay nothing (the round continues elsewhere).
struct BuildOptions {
    double beta = 0.0;             // > 0: use this beta
    bool showdown_pays_zero = false;
};

// Builds the game; returns an empty string on success, else a message.
// `code` receives KPS_EINVAL or KPS_ENOTSUP on failure.
std::string build_game(const kps_game_spec *spec, HostGame &g, kps_status *code,
                       const BuildOptions *opt = nullptr);

// Technique B sizes (Sec. 4) from the structure of the factors.
void technique_b_counts(HostGame &g);

// A sparse matrix in CSR form (FP64 values, columns ascending in a row).
struct Csr {
    int rows = 0, cols = 0;
    std::vector<int> rowptr, col;
    std::vector<double> val;
};

// Technique B factors (Sec. 4), A = Ahat + U M^-1 V^T, before the
// postprocessing step, in the vector layout: rows of A are s1 * hs + h1,
// columns s2 * hs + h2 (library hand order, padding rows and columns
// empty).  The inner dimension lists one entry per (player-1 sequence,
// hand), s1 * hs + h (the I (x) D block; the paper's D (x) I in its
// hand-major order), then one per player-1 sequence, n1 * hs + s1.
//   Ahat = -F (x) (Lambda1 Hx Lambda2)
//   U    = [I (x) Lambda1 | I (x) lambda1]
//   M    = diag(I (x) D, I), D lower bidiagonal (1, -1), stored with its
//          unit diagonal (padding rows: the diagonal alone)
//   V^T  = [S (x) (Y Lambda2) ; F (x) lambda2^T],  Y = D W
// with lambda in the rank-one blocks (the chance deal of Sec. 3).
struct TechniqueB {
    Csr ahat, u, m, vt;
};
void technique_b_factors(const HostGame &g, TechniqueB &f);

// Split [0, H) into `parts` contiguous chunks whose boundaries fall on tie
// group boundaries.  Returns parts+1 offsets (some chunks may be empty).
std::vector<int> chunk_bounds(const HostGame &g, int parts);

// Tiles of at most `tile` hands inside each chunk, never splitting a tie
// group (requires max_tie <= tile), cut from the chunk's start (the last
// tile takes the remainder) or, with from_end, from its end (the first tile
// takes the remainder).  Returns (start, length) pairs; tchunk receives
// parts+1 offsets into the tile list.
std::vector<std::pair<int, int>> tie_tiles(const HostGame &g, int parts, int tile,
                                           std::vector<int> &tchunk, bool from_end = false);

// Tie work of a tile list: for every tile, the ordered pairs (q, r), q != r,
// of compatible hands (no shared card) in one tie group, packed as
// q | r << 5 | (r > q) << 10 with q, r offsets in the tile (groups never
// straddle a tile).  work[t] = (first entry, count).
void tie_work(const HostGame &g, const std::vector<std::pair<int, int>> &tiles, std::vector<std::pair<int, int>> &work,
              std::vector<uint32_t> &trip);

}  // namespace kps
