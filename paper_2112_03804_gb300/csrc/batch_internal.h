// Internal state of a batch of games (batch.cu) shared with the solver.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <tuple>
#include <vector>

#include "abi_internal.h"
#include "kernels.h"

namespace kps_abi {

// Launch shape of the multi-game kernel for one dtype.
struct BatchShape {
    int nw = 8;         // warps per CTA
    int per_sm = 1;     // CTAs per SM
    int grid = 0;       // CTAs of the persistent launch
    int schedule = 0;   // 0 ticket counter, 1 static stride
    int kernel = 0;     // KPS_BATCH_TMEM or KPS_BATCH_STAGED
    double ms = 0.0;    // tuned time of one A and one A^T launch (0 = untuned)
};

// Device launch table of one (direction, FP64 or not, warp count).
struct BatchTable {
    void *blob = nullptr;
    kps::MultiParams m{};
};

}  // namespace kps_abi

struct kps_batch {
    std::vector<kps_game *> games;   // not owned
    int k = 0;                       // cards per hand (shared)
    int device = -1;
    std::vector<long long> off[2];   // element offsets of each game's vector, [ngames + 1]
    int *ticket = nullptr;           // tile ticket counter (device)
    std::map<std::tuple<int, bool, int>, kps_abi::BatchTable> tables;
    std::map<int, kps_abi::BatchShape> shape;   // per dtype
    void *warm = nullptr;            // warm-start feature tables (warm.cu)
    kps::AmPlan *am[2] = {nullptr, nullptr};   // staged FP32 kernel, per direction
    int am_state = 0;                // 0 not tried, 1 built, -1 it takes no game
    std::vector<char> am_rest;       // per game: 1 when the staged kernel leaves it to the tensor-memory one
    int am_nrest = 0;
    int rest_nw = 0;                 // warps of the tensor-memory launch over those games
    std::map<int, kps_abi::BatchTable> rest_tables;   // per direction
};

namespace kps_abi {

kps_status batch_table(kps_batch *b, int dir, bool f64, int nw, cudaStream_t stream, const BatchTable **out);
// FP32 launch table of the tensor-memory kernel over the games the staged
// kernel leaves (b->am_rest), b->rest_nw warps.
kps_status batch_rest_table(kps_batch *b, int dir, cudaStream_t stream, const BatchTable **out);
kps_status batch_default_shape(kps_batch *b, kps_dtype dt, cudaStream_t stream, BatchShape *out);
// dir 0: out = A y per game (y player-2 layout, out player-1 layout); dir 1: A^T.
kps_status batch_matvec(kps_batch *b, int dir, const void *vin, void *vout, kps_dtype dt, cudaStream_t stream);
// Builds the staged kernel's plans on first use (host work, synchronises
// `stream`); true when every game fits that kernel.
bool batch_staged_ready(kps_batch *b, cudaStream_t stream);
// Reads and clears the flag the warm-start predictor sets when a bounded
// wait gives up (warm.cu; synchronises the device).
cudaError_t predict_take_error(bool *set);
// Frees the warm-start tables of the batch (warm.cu).
void warm_free(kps_batch *b);

}  // namespace kps_abi
