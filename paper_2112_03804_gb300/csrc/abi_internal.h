// Internal state shared by the C ABI's translation units (abi.cu, batch.cu,
// solver.cu): the game object, its device tables and the error helpers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "../../include/kps.h"
#include "game.h"
#include "kernels.h"

#include <memory>

namespace kps_abi {

// Records `msg` as the calling thread's last error and returns `s`.
kps_status fail(kps_status s, const std::string &msg);
kps_status cuda_fail(cudaError_t e, const char *what);

// Device copies of the per-game tables, one allocation.
struct DeviceTables {
    void *blob = nullptr;
    uint32_t *hinfo = nullptr;
    float *lam1_f = nullptr, *lam2_f = nullptr;
    double *lam1_d = nullptr, *lam2_d = nullptr;
    // per output row: fold / showdown terminal (input sequence, payoff)
    int *fcol[2] = {nullptr, nullptr}, *scol[2] = {nullptr, nullptr};
    float *fcoef_f[2] = {nullptr, nullptr}, *scoef_f[2] = {nullptr, nullptr};
    double *fcoef_d[2] = {nullptr, nullptr}, *scoef_d[2] = {nullptr, nullptr};
};

size_t dtype_size(kps_dtype dt);

}  // namespace kps_abi

struct kps_game {
    kps::HostGame host;
    // per output row of each direction (0 = A, 1 = A^T): terminal pairs
    std::vector<int> fcol[2], scol[2];
    std::vector<double> fcoef[2], scoef[2];
    bool uploaded = false;
    int device = -1;
    kps_abi::DeviceTables dev;
    void *stage_in = nullptr, *stage_out = nullptr;
    size_t stage_in_bytes = 0, stage_out_bytes = 0;
    // host-buffer products: streams for copies in, products and copies out,
    // and one event per chunk and stage (created on first use)
    static constexpr int kHostChunks = 8;
    bool host_streams = false;
    cudaStream_t hstream[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t hentry = nullptr, hin[kHostChunks] = {}, hdone[kHostChunks] = {};
    // tie-aligned tile lists on the device, per warp count
    struct Tiles {
        int2 *dev = nullptr;          // tile list, then tie work, then tie entries (one allocation)
        int2 *tie_work = nullptr;
        uint32_t *tie_trip = nullptr;
        std::vector<int2> host;
        std::vector<int> tchunk;
        bool spill = false;           // cut from the chunk ends, spill rows in use
    };
    std::map<int, Tiles> tiles;
    // warps per CTA of the tensor-memory path (0 = not chosen yet)
    int tmem_nw = 0;
    // FP32 partial results for half-precision outputs
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    // parameter blocks of the TMA-staged FP32 path per direction, built on
    // first use (state 1), or -1 when the game cannot take that path
    struct TmaDel {
        void operator()(kps::TmaParams *p) const { kps::tma_destroy(p); }
    };
    std::unique_ptr<kps::TmaParams, TmaDel> tma[2];
    int tma_state[2] = {0, 0};
    // kernel of the last product per direction (KPS_KERNEL_* of kps.h)
    int last_kernel[2] = {0, 0};
};

namespace kps_abi {

// kps_sparsify with internal build options (NULL = none).
kps_status create_game(const kps_game_spec *spec, const kps::BuildOptions *opt, kps_game **out);

// Uploads the game's tables to the current device on first use.
kps_status upload(kps_game *g, cudaStream_t stream);

// The tie-aligned tile list of the game for `nw` warps (created and
// uploaded on first use; synchronises `stream` then).
kps_status tiles_for(kps_game *g, int nw, cudaStream_t stream, const kps_game::Tiles **out);

// Do the chunks of the `nw`-warp tile list fit the tensor-memory layout
// (kps::tmem_chunk_fits)?  The first form checks an uploaded list, the
// second builds the list on the host.
bool tmem_chunks_fit(const kps_game::Tiles &t, int nw);
bool tmem_split_fits(const kps::HostGame &h, int nw);

// Tile list of `nw` chunks: cut from each chunk's start when every chunk
// then fits the tensor-memory region, else from each chunk's end (a full
// last tile) with the spill rows (*spill).
std::vector<std::pair<int, int>> layout_tiles(const kps::HostGame &h, int nw, std::vector<int> &tchunk, bool *spill);

// Warps per CTA of the tensor-memory path for a game with `nc` cards left:
// four (two CTAs per SM, whose phases overlap) when the four-way split fits
// and two CTAs fit an SM's shared memory, else the fewest warps from one
// per 32 hands (at most kMaxWarps) whose split fits; -1 if none does.
// KPS_WARPS overrides the choice when that split fits.  Cached per game.
int tmem_warps(kps_game *g, int nc);

}  // namespace kps_abi
