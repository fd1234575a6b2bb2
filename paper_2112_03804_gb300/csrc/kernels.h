// Device-side entry points of the Kronecker payoff library (internal).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>
#include <utility>

namespace kps {

constexpr int kMaxWarps = 8;     // warps (= hand chunks) per CTA
constexpr int kColsPerCta = 32;  // one output column per lane

// One direction (A or A^T) of the product for one game.
//
// Output column j of the CTA (lane j) is (sigma, b) with
//   sigma = col / batch, b = col % batch, col = blockIdx.x * 32 + j.
// Its terminal pairs are at most one fold terminal (input sequence fcol,
// payoff fcoef) and one showdown terminal (scol, scoef); -1 = absent.
struct ScanParams {
    const void *vin;             // [batch][n_in][hs]
    void *vout;                  // [batch][n_out][hs]
    int H, hs, nc;               // nc = per-card table rows (cards left + 1)
    int n_out, n_in, batch;
    const int *fcol, *scol;      // [n_out]
    const void *fcoef, *scoef;   // [n_out], compute type
    const uint32_t *hinfo;       // [H]
    const void *lam_in, *lam_out;  // [H], compute type
    int nw;                      // warps per CTA = hand chunks
    int chunk[kMaxWarps + 1];    // chunk boundaries (tie-group aligned)
};

enum StorageType { kStoreF32 = 0, kStoreF64 = 1, kStoreBF16 = 2, kStoreF16 = 3 };

// Bytes of dynamic shared memory the scan kernel needs.
size_t scan_smem_bytes(int storage, int H, int nc, int nw, bool partial_in_smem);

// Largest dynamic shared memory per block on the current device.
int max_dyn_smem();

// Raises kernel `fn`'s dynamic shared-memory limit to at least `smem` bytes
// on the current device (set once per kernel, device and size; thread safe).
cudaError_t ensure_dyn_smem(const void *fn, size_t smem);

cudaError_t launch_pair_scan(const ScanParams &p, int storage, int cards_per_hand,
                             bool partial_in_smem, cudaStream_t stream);

}  // namespace kps

namespace kps {

constexpr int kTile = 32;        // hands per staging tile (tie-aligned tiles are shorter)

// Fast path: partial results pass through `scratch` (the output buffer for
// FP32/FP64, an FP32 buffer for half-precision outputs) instead of shared
// memory, tie groups are corrected inside tie-aligned tiles (needs every tie
// group to fit in one tile).
struct FastParams {
    const void *vin;             // [batch][n_in][hs] storage type
    void *vout;                  // [batch][n_out][hs] storage type
    void *scratch;               // [batch][n_out][hs] compute type (may alias vout)
    int H, hs, nc;
    int n_out, n_in, batch;
    const int *fcol, *scol;
    const void *fcoef, *scoef;   // compute type
    const uint32_t *hinfo;
    const void *lam_in, *lam_out;  // compute type
    const int2 *tiles;           // (start, length) of every tile, chunk after chunk
    int nw;
    int tchunk[kMaxWarps + 1];   // chunk k owns tiles [tchunk[k], tchunk[k+1])
    // Tie work of every tile (tensor-memory kernels): tie_work[t] = (first,
    // count) of its entries in tie_trip, one per ordered pair (q, r) of
    // compatible hands of one tie group: q | r << 5 | (r > q) << 10, with q,
    // r offsets in the tile.
    const int2 *tie_work;
    const uint32_t *tie_trip;
    int spill;                   // the tile list uses the tensor-memory spill rows
};

size_t fast_smem_bytes(int storage, int nc, int nw);
cudaError_t launch_fast_scan(const FastParams &p, int storage, int cards_per_hand, cudaStream_t stream);

}  // namespace kps

namespace kps {

// Vectorised fast path for FP32/FP64 storage (16-byte async copies); same
// parameters as the fast path.  Column kinds (fold only, showdown only,
// both) get their own specialised scan.
size_t vec_smem_bytes(int storage, int nc, int nw);
cudaError_t launch_vec_scan(const FastParams &p, int storage, int cards_per_hand, cudaStream_t stream);

}  // namespace kps

namespace kps {

// Tensor-memory path (FP32 arithmetic; FP32/BF16/FP16 storage): partial
// results stay on chip.  A warp keeps one column per hand (written 16 hands
// at a time from a tile's offset in the chunk) for every tile of its chunk
// but the last: columns below kTmemRegion in tensor memory, the next
// kTmemSpill in spill rows of its shared-memory partial tile; the last
// tile's partial results stay in the partial tile.  `scratch` is unused.
constexpr int kTmemRegion = 256;
constexpr int kTmemSpill = 16;

// Does a chunk fit `limit` columns (kTmemRegion, or kTmemRegion +
// kTmemSpill with the spill rows)?  `tile(i)` gives the (start, length) of
// its i-th of n tiles.
template <typename TileAt>
inline bool tmem_chunk_fits(int n, TileAt tile, int limit) {
    if (n <= 1) return true;
    const int cs = tile(0).first;
    for (int i = 0; i + 1 < n; ++i) {
        const auto t = tile(i);
        if (t.first - cs + (t.second + 15) / 16 * 16 > limit) return false;
    }
    return true;
}
size_t tmem_smem_bytes(int nc, int nw);
cudaError_t launch_tmem_scan(const FastParams &p, int storage, int cards_per_hand, cudaStream_t stream);

}  // namespace kps

namespace kps {

// Statically reserved device memory for kps_matvec_A_static_scratch: a tile
// list (up to kStaticTileBytes) and kStaticScratchFloats FP32 partial results.
constexpr size_t kStaticTileBytes = 64 * 1024;
constexpr size_t kStaticScratchFloats = 4u * 1024u * 1024u;   // 16 MiB
constexpr int kMaxDevices = 64;
// Device address of the reserved array on the current device.
cudaError_t static_scratch_address(void **ptr);

}  // namespace kps

namespace kps {

// Several games in one persistent launch (uneven hand counts and trees).
// games[g] holds game g's parameters built for `nw` warps, with vin/vout
// unused: its vectors start in_off[g] / out_off[g] elements after vin /
// vout.  Column tile j of the launch belongs to game tile_game[j] and is
// that game's tile j - tile_start[game].  With schedule 0 the CTAs take
// tiles from the ticket counter *ticket (zeroed before the launch), with
// schedule 1 CTA b takes tiles b, b + grid, b + 2 grid, ...
struct MultiParams {
    const FastParams *games;        // [ngames]
    const long long *tile_start;    // [ngames + 1]
    const int *tile_game;           // [total_tiles]
    const long long *in_off, *out_off;  // [ngames]
    const void *vin;
    void *vout;
    int *ticket;
    int ngames;
    int total_tiles;
    int spill;                      // some game's tiles use the spill rows
    int nw;                         // warps per CTA
    int nc;                         // largest per-card row count of the games
    int schedule;
};

cudaError_t launch_tmem_multi(const MultiParams &m, int storage, int cards_per_hand, int grid, cudaStream_t stream);
cudaError_t launch_vec_multi(const MultiParams &m, int storage, int cards_per_hand, int grid, cudaStream_t stream);
// Resident CTAs per SM of the multi-game kernels for the given shape.
int tmem_multi_ctas_per_sm(int storage, int cards_per_hand, int nc, int nw);
int vec_multi_ctas_per_sm(int storage, int cards_per_hand, int nc, int nw);

}  // namespace kps

namespace kps {

// TMA-staged single-game path (FP32 storage, kernels_tma.cu).  A CTA owns
// one output sequence and 32 consecutive vectors of the batch (one per
// lane); its warps scan chunks of the hand order, each a run of 16-hand
// boxes that the tensor memory accelerator copies into shared memory.  The
// parameter block is opaque here: built once per game and direction.
struct TmaParams;
struct HostGame;

// Builds the parameter block for one direction (lam_in / lam_out: library
// order; fcol, scol, fcoef, scoef: the device tables of that direction;
// hfcol / hscol: their host copies).  Returns nullptr with *why set when
// the game cannot take this path.
TmaParams *tma_create(const HostGame &h, const double *lam_in, const double *lam_out, int n_out, int n_in,
                      const int *fcol, const int *scol, const float *fcoef, const float *scoef,
                      const int *hfcol, const int *hscol, std::string *why);
void tma_destroy(TmaParams *p);
// One product: out (device, [batch][n_out][hs]) from vin ([batch][n_in][hs]),
// both 16-byte aligned.
cudaError_t launch_tma_scan(TmaParams *p, const float *vin, float *vout, int batch, cudaStream_t stream);
// Reads and clears the flag the TMA-staged kernel sets when a bounded wait
// gives up (synchronises the device).
cudaError_t tma_take_error(bool *set);

// Staged multi-game path (FP32, BF16 or FP16 storage, kStore*; FP32
// arithmetic; kernels_amulti.cu): one persistent
// launch over (game, 32 output sequences) work items of a batch, one vector
// per game; the warps of a CTA scan chunks of the game's hand order in
// 16-hand boxes copied by cp.async.  One plan per direction.
struct AmGameDesc {
    const HostGame *h;
    const double *lam_in, *lam_out;   // host, library order
    int n_out;
    const int *fcol, *scol;           // device tables of the direction
    const float *fcoef, *scoef;
    long long in_off, out_off;        // element offsets in the batch vectors
};
struct AmPlan;
// Builds and uploads the plan (synchronises `stream`) for the games this
// path takes ((*taken)[i] = 1; the others, e.g. with a tie group longer than
// 4 hands, get no work items); nullptr when it takes none or on a failure,
// *why set.  Scratch for `grid_cap` CTAs.
AmPlan *am_create(const std::vector<AmGameDesc> &games, int grid_cap, cudaStream_t stream, std::vector<char> *taken,
                  std::string *why);
void am_destroy(AmPlan *p);
int am_ctas_per_sm(const AmPlan *p);
int am_grid_cap(const AmPlan *p);
// One product over every game; ticket: a device counter cleared before the
// launch when schedule == 0 (ticket), unused when 1 (static stride).
cudaError_t launch_async_multi(AmPlan *p, int storage, const void *vin, void *vout, int *ticket, int schedule,
                               int grid, cudaStream_t stream);

}  // namespace kps
