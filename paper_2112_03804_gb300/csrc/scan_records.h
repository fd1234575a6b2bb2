// Per-box hand records of the staged scan kernels (kernels_tma.cu for one
// game and many vectors, kernels_amulti.cu for many games), built on the
// host once per game and direction (scan_records.cpp).
//
// The scan walks hands in library order (strength, then canonical index) in
// boxes of 16 hands; a chunk of consecutive boxes goes to each of four warps.
// For every pair of hands (2i, 2i+1) the scan reads a TmaScanRec and the
// finishing pass a TmaFinRec:
//   oa*, ob*  byte offsets of the hands' card rows in a warp's per-card table
//             (card * 128; the spare row ncards * 128 for padding hands and
//             for the second card of one-card hands),
//   lin*      input weights lambda_in (0 for padding hands),
//   ma, mb    1 when the first / second card of hand 2i+1 is a card of hand
//             2i, else 0,
//   lout*     output weights lambda_out.
// A box's scan block is its 8 pair records followed by two tie words: byte
// 8j + (k - 4j) of word j (pair k) has
//   bits 2-4  hand 2k has a compatible tied hand 1, 2, 3 positions before it
//   bits 5-7  the same for hand 2k+1.
// Tie groups of at most 4 hands are accepted, and chunk boundaries fall on
// box boundaries that cut no tie group.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "game.h"

namespace kps {

constexpr int kTmaBox = 16;        // hands per box
constexpr int kTmaWarps = 4;       // chunks per CTA

struct alignas(16) TmaScanRec {
    uint32_t oa1, ob1, oa2, ob2;
    float lin1, lin2, ma, mb;
};
constexpr int kScanBlock = 8 * 32 + 16;   // bytes per box
struct alignas(16) TmaFinRec {
    uint32_t oa1, ob1, oa2, ob2;
    float lout1, lout2, pad0, pad1;
};

// Records of one game and direction.  bytes = nbox scan blocks, then
// nbox * 8 finishing records.
struct ScanRecords {
    int H = 0, hs = 0, nc = 0, k = 0, nbox = 0;
    int extra = 0;                 // boxes of the longest chunk past 16
    int bchunk[kTmaWarps + 1] = {0, 0, 0, 0, 0};
    std::vector<unsigned char> bytes;
};

// Empty string on success, else why the game does not fit these kernels
// (tie group over 4 hands, more than 64 card rows, a chunk longer than
// 16 + max_extra boxes).
std::string build_scan_records(const HostGame &h, const double *lam_in, const double *lam_out, int max_extra,
                               ScanRecords *out);

}  // namespace kps
