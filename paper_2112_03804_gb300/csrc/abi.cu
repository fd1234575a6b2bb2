// C ABI of the Kronecker payoff library (declared in include/kps.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/kps.h"
#include "abi_internal.h"
#include "batch_internal.h"
#include "game.h"
#include "kernels.h"

namespace kps_abi {

thread_local std::string g_last_error;

kps_status fail(kps_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

kps_status cuda_fail(cudaError_t e, const char *what) {
    return fail(KPS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace kps_abi

using namespace kps_abi;

namespace kps_abi {

size_t dtype_size(kps_dtype dt) {
    switch (dt) {
        case KPS_F32: return 4;
        case KPS_F64: return 8;
        case KPS_BF16: return 2;
        case KPS_F16: return 2;
        default: return 0;
    }
}

// Each output sequence has at most one fold terminal and one showdown
// terminal as its last action (its own terminating action, or the opponent's
// fold/call responses to it); split the terminal pair lists accordingly.
std::string split_rows(kps_game *g) {
    for (int dir = 0; dir < 2; ++dir) {
        const kps::PairCsr &csr = dir == 0 ? g->host.csr_A : g->host.csr_AT;
        const int rows = (int)csr.rowptr.size() - 1;
        g->fcol[dir].assign(rows, -1);
        g->scol[dir].assign(rows, -1);
        g->fcoef[dir].assign(rows, 0.0);
        g->scoef[dir].assign(rows, 0.0);
        for (int r = 0; r < rows; ++r)
            for (int e = csr.rowptr[r]; e < csr.rowptr[r + 1]; ++e) {
                auto &col = csr.kind[e] == 0 ? g->fcol[dir] : g->scol[dir];
                auto &coef = csr.kind[e] == 0 ? g->fcoef[dir] : g->scoef[dir];
                if (col[r] >= 0) return "a sequence ends two terminals of the same kind";
                col[r] = csr.col[e];
                coef[r] = csr.coef[e];
            }
    }
    return "";
}

kps_status upload(kps_game *g, cudaStream_t stream) {
    if (g->uploaded) {
        int dev = -1;
        cudaGetDevice(&dev);
        if (dev != g->device) return fail(KPS_EINVAL, "game tables live on another device");
        return KPS_OK;
    }
    const kps::HostGame &h = g->host;
    const int H = h.H;
    // layout of the blob (8-byte aligned pieces)
    auto al = [](size_t x) { return (x + 15) / 16 * 16; };
    size_t off = 0;
    // per-hand tables are padded by 16 entries: vector loads may round the
    // end of a hand range up to a multiple of 4
    const size_t Hp = (size_t)H + 16;
    const size_t o_hinfo = off; off = al(off + 4 * Hp);
    const size_t o_l1f = off; off = al(off + 4 * Hp);
    const size_t o_l2f = off; off = al(off + 4 * Hp);
    const size_t o_l1d = off; off = al(off + 8 * Hp);
    const size_t o_l2d = off; off = al(off + 8 * Hp);
    size_t o_fcol[2], o_scol[2], o_ff[2], o_sf[2], o_fd[2], o_sd[2];
    for (int d = 0; d < 2; ++d) {
        const size_t r = g->fcol[d].size();
        o_fcol[d] = off; off = al(off + 4 * r);
        o_scol[d] = off; off = al(off + 4 * r);
        o_ff[d] = off; off = al(off + 4 * r);
        o_sf[d] = off; off = al(off + 4 * r);
        o_fd[d] = off; off = al(off + 8 * r);
        o_sd[d] = off; off = al(off + 8 * r);
    }
    std::vector<unsigned char> hostblob(off, 0);
    auto put = [&](size_t o, const void *src, size_t bytes) { if (bytes) std::memcpy(hostblob.data() + o, src, bytes); };
    put(o_hinfo, h.hinfo.data(), 4 * (size_t)H);
    std::vector<float> tmp(H);
    for (int i = 0; i < H; ++i) tmp[i] = (float)h.lam1[i];
    put(o_l1f, tmp.data(), 4 * (size_t)H);
    for (int i = 0; i < H; ++i) tmp[i] = (float)h.lam2[i];
    put(o_l2f, tmp.data(), 4 * (size_t)H);
    put(o_l1d, h.lam1.data(), 8 * (size_t)H);
    put(o_l2d, h.lam2.data(), 8 * (size_t)H);
    for (int d = 0; d < 2; ++d) {
        const size_t r = g->fcol[d].size();
        put(o_fcol[d], g->fcol[d].data(), 4 * r);
        put(o_scol[d], g->scol[d].data(), 4 * r);
        std::vector<float> f(r), s(r);
        for (size_t i = 0; i < r; ++i) { f[i] = (float)g->fcoef[d][i]; s[i] = (float)g->scoef[d][i]; }
        put(o_ff[d], f.data(), 4 * r);
        put(o_sf[d], s.data(), 4 * r);
        put(o_fd[d], g->fcoef[d].data(), 8 * r);
        put(o_sd[d], g->scoef[d].data(), 8 * r);
    }
    void *blob = nullptr;
    cudaError_t e = cudaMalloc(&blob, off);
    if (e != cudaSuccess) return fail(KPS_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    e = cudaMemcpyAsync(blob, hostblob.data(), off, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        cudaFree(blob);
        return cuda_fail(e, "uploading game tables");
    }
    unsigned char *b = static_cast<unsigned char *>(blob);
    DeviceTables &t = g->dev;
    t.blob = blob;
    t.hinfo = reinterpret_cast<uint32_t *>(b + o_hinfo);
    t.lam1_f = reinterpret_cast<float *>(b + o_l1f);
    t.lam2_f = reinterpret_cast<float *>(b + o_l2f);
    t.lam1_d = reinterpret_cast<double *>(b + o_l1d);
    t.lam2_d = reinterpret_cast<double *>(b + o_l2d);
    for (int d = 0; d < 2; ++d) {
        t.fcol[d] = reinterpret_cast<int *>(b + o_fcol[d]);
        t.scol[d] = reinterpret_cast<int *>(b + o_scol[d]);
        t.fcoef_f[d] = reinterpret_cast<float *>(b + o_ff[d]);
        t.scoef_f[d] = reinterpret_cast<float *>(b + o_sf[d]);
        t.fcoef_d[d] = reinterpret_cast<double *>(b + o_fd[d]);
        t.scoef_d[d] = reinterpret_cast<double *>(b + o_sd[d]);
    }
    cudaGetDevice(&g->device);
    g->uploaded = true;
    return KPS_OK;
}

kps_status tiles_for(kps_game *g, int nw, cudaStream_t stream, const kps_game::Tiles **out) {
    auto it = g->tiles.find(nw);
    if (it == g->tiles.end()) {
        kps_game::Tiles t;
        std::vector<std::pair<int, int>> tl = layout_tiles(g->host, nw, t.tchunk, &t.spill);
        std::vector<int2> host(tl.size());
        for (size_t i = 0; i < tl.size(); ++i) host[i] = make_int2(tl[i].first, tl[i].second);
        t.host = host;
        std::vector<std::pair<int, int>> work;
        std::vector<uint32_t> trip;
        if (g->host.max_tie <= kps::kTile) kps::tie_work(g->host, tl, work, trip);
        else work.assign(tl.size(), std::make_pair(0, 0));
        // one allocation: tiles, tie work, tie entries
        const size_t n = host.size();
        const size_t bytes = (2 * n + 1) * sizeof(int2) + std::max<size_t>(1, trip.size()) * sizeof(uint32_t);
        std::vector<unsigned char> blob(bytes, 0);
        std::vector<int2> w2(n);
        for (size_t i = 0; i < n; ++i) w2[i] = make_int2(work[i].first, work[i].second);
        if (n) {
            std::memcpy(blob.data(), host.data(), n * sizeof(int2));
            std::memcpy(blob.data() + n * sizeof(int2), w2.data(), n * sizeof(int2));
        }
        if (!trip.empty()) std::memcpy(blob.data() + 2 * n * sizeof(int2), trip.data(), trip.size() * sizeof(uint32_t));
        cudaError_t e = cudaMalloc(&t.dev, bytes);
        if (e != cudaSuccess) return fail(KPS_ENOMEM, "tile table");
        t.tie_work = t.dev + n;
        t.tie_trip = reinterpret_cast<uint32_t *>(t.dev + 2 * n);
        e = cudaMemcpyAsync(t.dev, blob.data(), bytes, cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) {
            cudaFree(t.dev);
            return cuda_fail(e, "uploading the tile table");
        }
        it = g->tiles.emplace(nw, std::move(t)).first;
    }
    *out = &it->second;
    return KPS_OK;
}

namespace {
bool list_fits(const std::vector<std::pair<int, int>> &tl, const std::vector<int> &tchunk, int nw, int limit) {
    for (int k = 0; k < nw; ++k) {
        const int a = tchunk[k];
        if (!kps::tmem_chunk_fits(tchunk[k + 1] - a, [&](int i) { return tl[a + i]; }, limit)) return false;
    }
    return true;
}
}  // namespace

std::vector<std::pair<int, int>> layout_tiles(const kps::HostGame &h, int nw, std::vector<int> &tchunk, bool *spill) {
    *spill = false;
    std::vector<std::pair<int, int>> tl = kps::tie_tiles(h, nw, kps::kTile, tchunk);
    if (list_fits(tl, tchunk, nw, kps::kTmemRegion)) return tl;
    std::vector<int> tc2;
    std::vector<std::pair<int, int>> tl2 = kps::tie_tiles(h, nw, kps::kTile, tc2, true);
    if (h.k == 2 && list_fits(tl2, tc2, nw, kps::kTmemRegion + kps::kTmemSpill)) {
        tchunk = tc2;
        *spill = true;
        return tl2;
    }
    return tl;
}

bool tmem_chunks_fit(const kps_game::Tiles &t, int nw) {
    const int limit = kps::kTmemRegion + (t.spill ? kps::kTmemSpill : 0);
    for (int k = 0; k < nw; ++k) {
        const int a = t.tchunk[k];
        auto at = [&](int i) { return std::make_pair(t.host[a + i].x, t.host[a + i].y); };
        if (!kps::tmem_chunk_fits(t.tchunk[k + 1] - a, at, limit)) return false;
    }
    return true;
}

bool tmem_split_fits(const kps::HostGame &h, int nw) {
    std::vector<int> tchunk;
    bool spill = false;
    const std::vector<std::pair<int, int>> tl = layout_tiles(h, nw, tchunk, &spill);
    return list_fits(tl, tchunk, nw, kps::kTmemRegion + (spill ? kps::kTmemSpill : 0));
}

int tmem_warps(kps_game *g, int nc) {
    const kps::HostGame &h = g->host;
    if (const char *env = std::getenv("KPS_WARPS")) {
        const int w = std::atoi(env);
        if (w >= 1 && w <= kps::kMaxWarps && tmem_split_fits(h, w)) return w;
    }
    if (g->tmem_nw != 0) return g->tmem_nw;
    int nw = std::min(kps::kMaxWarps, (h.H + kps::kTile - 1) / kps::kTile);
    const int smem_max = kps::max_dyn_smem();
    if (nw > 4 && 2 * (kps::tmem_smem_bytes(nc, 4) + 1024) <= (size_t)smem_max + 1024 && tmem_split_fits(h, 4)) {
        nw = 4;
    } else {
        while (nw <= kps::kMaxWarps && !tmem_split_fits(h, nw)) ++nw;
        if (nw > kps::kMaxWarps) nw = -1;
    }
    g->tmem_nw = nw;
    return nw;
}

// Warps per CTA of the fast path: two CTAs of 4 warps per SM when they fit
// (smaller CTAs shorten the tail of the last wave), else the largest count
// that fits.  KPS_WARPS overrides the choice (1..8).
int fast_warps(int storage, int nc, int H, bool vec) {
    const int smem_max = kps::max_dyn_smem();
    auto bytes = [&](int w) { return vec ? kps::vec_smem_bytes(storage, nc, w) : kps::fast_smem_bytes(storage, nc, w); };
    int nw = 0;
    if (const char *env = std::getenv("KPS_WARPS")) nw = std::atoi(env);
    if (nw < 1 || nw > kps::kMaxWarps || bytes(nw) > (size_t)smem_max) {
        nw = 0;
        // prefer two CTAs per SM (227 KB per SM, 1 KB reserved per CTA)
        for (int w = 4; w >= 2 && nw == 0; --w)
            if (2 * (bytes(w) + 1024) <= (size_t)smem_max + 1024) nw = w;
        if (nw == 0)
            for (int w = kps::kMaxWarps; w >= 1; --w)
                if (bytes(w) <= (size_t)smem_max) { nw = w; break; }
    }
    return std::max(1, std::min(nw, (H + kps::kTile - 1) / kps::kTile));
}

kps_status matvec_fast(kps_game *g, int dir, const kps::ScanParams &sp, int storage, kps_dtype dt,
                       cudaStream_t stream) {
    const kps::HostGame &h = g->host;
    // Kernel choice: tensor-memory partials (FP32 arithmetic storages), else
    // the vectorised path (16-byte aligned FP32/FP64), else scalar staging.
    // KPS_KERNEL=tmem|vec|fast forces one where it applies.
    const char *force = std::getenv("KPS_KERNEL");
    const bool aligned = ((reinterpret_cast<uintptr_t>(sp.vin) | reinterpret_cast<uintptr_t>(sp.vout)) & 15) == 0;
    const bool vec_ok = aligned && (storage == kps::kStoreF32 || storage == kps::kStoreF64) && sp.nc <= 64 &&
                        std::getenv("KPS_NO_VEC") == nullptr;
    const bool tmem_ok = storage != kps::kStoreF64 && sp.nc <= 66;
    enum { kTmem, kVec, kScalar } path = tmem_ok ? kTmem : vec_ok ? kVec : kScalar;
    if (force) {
        if (!std::strcmp(force, "vec") && vec_ok) path = kVec;
        else if (!std::strcmp(force, "fast")) path = kScalar;
        else if (!std::strcmp(force, "tmem") && tmem_ok) path = kTmem;
    }
    int nw;
    if (path == kTmem) {
        nw = tmem_warps(g, sp.nc);
        if (nw < 1 || kps::tmem_smem_bytes(sp.nc, nw) > (size_t)kps::max_dyn_smem()) path = kScalar;
    }
    const bool vec = path == kVec;
    if (path != kTmem) nw = fast_warps(storage, sp.nc, h.H, vec);
    const size_t need = path == kTmem ? kps::tmem_smem_bytes(sp.nc, nw)
                        : vec ? kps::vec_smem_bytes(storage, sp.nc, nw) : kps::fast_smem_bytes(storage, sp.nc, nw);
    if (need > (size_t)kps::max_dyn_smem())
        return fail(KPS_ENOTSUP, "card count too large for shared memory");
    const kps_game::Tiles *tiles = nullptr;
    kps_status st = tiles_for(g, nw, stream, &tiles);
    if (st != KPS_OK) return st;
    if (path == kTmem && !tmem_chunks_fit(*tiles, nw)) return fail(KPS_ENOTSUP, "hand chunk too long for tensor memory");
    void *scratch = sp.vout;
    if (path != kTmem && (storage == kps::kStoreBF16 || storage == kps::kStoreF16)) {
        const size_t need = (size_t)sp.batch * sp.n_out * h.hs * sizeof(float);
        if (g->scratch_bytes < need) {
            if (g->scratch) cudaFree(g->scratch);
            g->scratch = nullptr;
            g->scratch_bytes = 0;
            cudaError_t e = cudaMalloc(&g->scratch, need);
            if (e != cudaSuccess) return fail(KPS_ENOMEM, "partial-result buffer");
            g->scratch_bytes = need;
        }
        scratch = g->scratch;
    }
    kps::FastParams p{};
    p.vin = sp.vin;
    p.vout = sp.vout;
    p.scratch = scratch;
    p.H = sp.H;
    p.hs = sp.hs;
    p.nc = sp.nc;
    p.n_out = sp.n_out;
    p.n_in = sp.n_in;
    p.batch = sp.batch;
    p.fcol = sp.fcol;
    p.scol = sp.scol;
    p.fcoef = sp.fcoef;
    p.scoef = sp.scoef;
    p.hinfo = sp.hinfo;
    p.lam_in = sp.lam_in;
    p.lam_out = sp.lam_out;
    p.tiles = tiles->dev;
    p.tie_work = tiles->tie_work;
    p.tie_trip = tiles->tie_trip;
    p.spill = tiles->spill ? 1 : 0;
    p.nw = nw;
    for (int i = 0; i <= nw; ++i) p.tchunk[i] = tiles->tchunk[i];
    (void)dir;
    (void)dt;
    cudaError_t e;
    g->last_kernel[dir] = path == kTmem ? KPS_KERNEL_TMEM : vec ? KPS_KERNEL_VEC : KPS_KERNEL_SCALAR;
    if (path == kTmem) e = kps::launch_tmem_scan(p, storage, h.k, stream);
    else if (vec) e = kps::launch_vec_scan(p, storage, h.k, stream);
    else e = kps::launch_fast_scan(p, storage, h.k, stream);
    if (e != cudaSuccess) return cuda_fail(e, "launching the payoff scan");
    return KPS_OK;
}

// The TMA-staged FP32 path (kernels_tma.cu) when the game and the vectors
// allow it; *taken tells whether it ran.  KPS_KERNEL=tma|tmem|vec|fast
// forces a path where it applies (any value other than tma disables this
// one).
kps_status matvec_tma(kps_game *g, int dir, const void *vin, void *vout, int32_t batch, cudaStream_t stream,
                      bool *taken) {
    *taken = false;
    const char *force = std::getenv("KPS_KERNEL");
    if (force && std::strcmp(force, "tma") != 0) return KPS_OK;
    if (((reinterpret_cast<uintptr_t>(vin) | reinterpret_cast<uintptr_t>(vout)) & 15) != 0) return KPS_OK;
    if (g->tma_state[dir] == 0) {
        const kps::HostGame &h = g->host;
        const double *lin = dir == 0 ? h.lam2.data() : h.lam1.data();
        const double *lout = dir == 0 ? h.lam1.data() : h.lam2.data();
        std::string why;
        kps::TmaParams *p = kps::tma_create(h, lin, lout, dir == 0 ? h.n[0] : h.n[1], dir == 0 ? h.n[1] : h.n[0],
                                            g->dev.fcol[dir], g->dev.scol[dir], g->dev.fcoef_f[dir],
                                            g->dev.scoef_f[dir], g->fcol[dir].data(), g->scol[dir].data(), &why);
        g->tma[dir].reset(p);
        g->tma_state[dir] = p ? 1 : -1;
    }
    if (g->tma_state[dir] != 1) return KPS_OK;
    *taken = true;
    g->last_kernel[dir] = KPS_KERNEL_TMA;
    cudaError_t e = kps::launch_tma_scan(g->tma[dir].get(), static_cast<const float *>(vin),
                                         static_cast<float *>(vout), batch, stream);
    if (e != cudaSuccess) return cuda_fail(e, "launching the TMA-staged payoff scan");
    return KPS_OK;
}

kps_status matvec(kps_game *g, int dir, const void *vin, void *vout, int32_t batch, kps_dtype dt,
                  void *stream_ptr) {
    if (!g) return fail(KPS_EINVAL, "game is NULL");
    if (batch < 0) return fail(KPS_EINVAL, "batch must be >= 0");
    if (dtype_size(dt) == 0) return fail(KPS_EINVAL, "unknown dtype");
    if (batch == 0) return KPS_OK;
    if (!vin || !vout) return fail(KPS_EINVAL, "vector pointer is NULL");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    kps_status st = upload(g, stream);
    if (st != KPS_OK) return st;
    const kps::HostGame &h = g->host;
    const int n_out = dir == 0 ? h.n[0] : h.n[1];
    const int n_in = dir == 0 ? h.n[1] : h.n[0];
    const size_t es = dtype_size(dt);
    const size_t in_bytes = (size_t)batch * n_in * h.hs * es;
    const size_t out_bytes = (size_t)batch * n_out * h.hs * es;
    const char *ci = static_cast<const char *>(vin), *co = static_cast<const char *>(vout);
    if (ci < co + out_bytes && co < ci + in_bytes) return fail(KPS_EINVAL, "input and output overlap");
    if ((long long)n_out * batch > 0x7fffffffLL * 32LL) return fail(KPS_ENOTSUP, "too many columns");

    kps::ScanParams p{};
    p.vin = vin;
    p.vout = vout;
    p.H = h.H;
    p.hs = h.hs;
    p.nc = h.ncards + 1;
    p.n_out = n_out;
    p.n_in = n_in;
    p.batch = batch;
    const bool f64 = dt == KPS_F64;
    const DeviceTables &t = g->dev;
    p.fcol = t.fcol[dir];
    p.scol = t.scol[dir];
    p.fcoef = f64 ? (const void *)t.fcoef_d[dir] : (const void *)t.fcoef_f[dir];
    p.scoef = f64 ? (const void *)t.scoef_d[dir] : (const void *)t.scoef_f[dir];
    p.hinfo = t.hinfo;
    const void *l1 = f64 ? (const void *)t.lam1_d : (const void *)t.lam1_f;
    const void *l2 = f64 ? (const void *)t.lam2_d : (const void *)t.lam2_f;
    p.lam_in = dir == 0 ? l2 : l1;
    p.lam_out = dir == 0 ? l1 : l2;
    const int storage = dt == KPS_F32 ? kps::kStoreF32 : dt == KPS_F64 ? kps::kStoreF64
                        : dt == KPS_BF16 ? kps::kStoreBF16 : kps::kStoreF16;
    if (storage == kps::kStoreF32) {
        bool taken = false;
        kps_status s2 = matvec_tma(g, dir, vin, vout, batch, stream, &taken);
        if (taken || s2 != KPS_OK) return s2;
    }
    if (h.max_tie <= kps::kTile) return matvec_fast(g, dir, p, storage, dt, stream);
    // general path: as many hand chunks (warps) as shared memory allows
    const int smem_max = kps::max_dyn_smem();
    bool pin = true;
    int nw = 0;
    for (int w = kps::kMaxWarps; w >= 1; --w)
        if (kps::scan_smem_bytes(storage, h.H, p.nc, w, true) <= (size_t)smem_max) { nw = w; break; }
    if (nw == 0) {
        if (storage != kps::kStoreF32 && storage != kps::kStoreF64)
            return fail(KPS_ENOTSUP, "hand count too large for half-precision storage");
        pin = false;
        for (int w = kps::kMaxWarps; w >= 1; --w)
            if (kps::scan_smem_bytes(storage, h.H, p.nc, w, false) <= (size_t)smem_max) { nw = w; break; }
        if (nw == 0) return fail(KPS_ENOTSUP, "card count too large for shared memory");
    }
    nw = std::min(nw, std::max(1, h.H));
    p.nw = nw;
    std::vector<int> cb = kps::chunk_bounds(h, nw);
    for (int i = 0; i <= nw; ++i) p.chunk[i] = cb[i];
    g->last_kernel[dir] = KPS_KERNEL_GENERAL;
    cudaError_t e = kps::launch_pair_scan(p, storage, h.k, pin, stream);
    if (e != cudaSuccess) return cuda_fail(e, "launching the payoff scan");
    return KPS_OK;
}

kps_status matvec_host(kps_game *g, int dir, const void *vin, void *vout, int32_t batch, kps_dtype dt,
                       void *stream_ptr) {
    if (!g) return fail(KPS_EINVAL, "game is NULL");
    if (batch < 0) return fail(KPS_EINVAL, "batch must be >= 0");
    if (dtype_size(dt) == 0) return fail(KPS_EINVAL, "unknown dtype");
    if (batch == 0) return KPS_OK;
    if (!vin || !vout) return fail(KPS_EINVAL, "vector pointer is NULL");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    const kps::HostGame &h = g->host;
    const int n_out = dir == 0 ? h.n[0] : h.n[1];
    const int n_in = dir == 0 ? h.n[1] : h.n[0];
    const size_t es = dtype_size(dt);
    const size_t in_bytes = (size_t)batch * n_in * h.hs * es;
    const size_t out_bytes = (size_t)batch * n_out * h.hs * es;
    cudaError_t e;
    if (g->stage_in_bytes < in_bytes) {
        if (g->stage_in) cudaFree(g->stage_in);
        g->stage_in = nullptr;
        g->stage_in_bytes = 0;
        e = cudaMalloc(&g->stage_in, in_bytes);
        if (e != cudaSuccess) return fail(KPS_ENOMEM, "staging buffer");
        g->stage_in_bytes = in_bytes;
    }
    if (g->stage_out_bytes < out_bytes) {
        if (g->stage_out) cudaFree(g->stage_out);
        g->stage_out = nullptr;
        g->stage_out_bytes = 0;
        e = cudaMalloc(&g->stage_out, out_bytes);
        if (e != cudaSuccess) return fail(KPS_ENOMEM, "staging buffer");
        g->stage_out_bytes = out_bytes;
    }
    // The batch goes in chunks of vectors: chunk c's copy in, product and
    // copy out run on three streams ordered by per-chunk events, so the two
    // copy directions and the products of neighbouring chunks overlap.  All
    // three streams start after the work already queued on `stream`.
    if (!g->host_streams) {
        for (auto &hs_ : g->hstream)
            if ((e = cudaStreamCreateWithFlags(&hs_, cudaStreamNonBlocking)) != cudaSuccess)
                return cuda_fail(e, "creating copy streams");
        if ((e = cudaEventCreateWithFlags(&g->hentry, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, "creating events");
        for (int c = 0; c < kps_game::kHostChunks; ++c)
            if ((e = cudaEventCreateWithFlags(&g->hin[c], cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&g->hdone[c], cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(e, "creating events");
        g->host_streams = true;
    }
    cudaStream_t s_in = g->hstream[0], s_mv = g->hstream[1], s_out = g->hstream[2];
    // on an error after work was queued, wait for it before returning: the
    // copies read and write the caller's host buffers
    auto drain = [&]() {
        for (cudaStream_t q : {s_in, s_mv, s_out}) cudaStreamSynchronize(q);
    };
    if ((e = cudaEventRecord(g->hentry, stream)) != cudaSuccess) return cuda_fail(e, "ordering the copies");
    for (cudaStream_t q : {s_in, s_mv, s_out})
        if ((e = cudaStreamWaitEvent(q, g->hentry, 0)) != cudaSuccess) {
            drain();
            return cuda_fail(e, "ordering the copies");
        }
    const int nch = std::min(kps_game::kHostChunks, (int)batch);
    const size_t vin_bytes = in_bytes / batch, vout_bytes = out_bytes / batch;
    for (int c = 0; c < nch; ++c) {
        const size_t b0 = (size_t)batch * c / nch, b1 = (size_t)batch * (c + 1) / nch;
        char *din = static_cast<char *>(g->stage_in) + b0 * vin_bytes;
        char *dout = static_cast<char *>(g->stage_out) + b0 * vout_bytes;
        e = cudaMemcpyAsync(din, static_cast<const char *>(vin) + b0 * vin_bytes, (b1 - b0) * vin_bytes,
                            cudaMemcpyHostToDevice, s_in);
        if (e == cudaSuccess) e = cudaEventRecord(g->hin[c], s_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s_mv, g->hin[c], 0);
        if (e != cudaSuccess) {
            drain();
            return cuda_fail(e, "copying input to the device");
        }
        kps_status st = matvec(g, dir, din, dout, (int32_t)(b1 - b0), dt, s_mv);
        if (st != KPS_OK) {
            drain();
            return st;
        }
        e = cudaEventRecord(g->hdone[c], s_mv);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out, g->hdone[c], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(static_cast<char *>(vout) + b0 * vout_bytes, dout, (b1 - b0) * vout_bytes,
                                cudaMemcpyDeviceToHost, s_out);
        if (e != cudaSuccess) {
            drain();
            return cuda_fail(e, "copying output to the host");
        }
    }
    for (cudaStream_t q : {s_in, s_mv, s_out})
        if ((e = cudaStreamSynchronize(q)) != cudaSuccess) {
            drain();
            return cuda_fail(e, "synchronising");
        }
    return KPS_OK;
}

}  // namespace kps_abi

extern "C" {

kps_status kps_sparsify(const kps_game_spec *spec, kps_game **out) {
    return create_game(spec, nullptr, out);
}

}  // extern "C"

namespace kps_abi {

kps_status create_game(const kps_game_spec *spec, const kps::BuildOptions *opt, kps_game **out) {
    if (!out) return fail(KPS_EINVAL, "out is NULL");
    *out = nullptr;
    kps_game *g = new (std::nothrow) kps_game();
    if (!g) return fail(KPS_ENOMEM, "host allocation");
    try {
        kps_status code = KPS_OK;
        std::string err = kps::build_game(spec, g->host, &code, opt);
        if (err.empty()) err = split_rows(g), code = err.empty() ? KPS_OK : KPS_ENOTSUP;
        if (!err.empty()) {
            delete g;
            return fail(code, err);
        }
    } catch (const std::bad_alloc &) {
        delete g;
        return fail(KPS_ENOMEM, "host allocation");
    } catch (...) {
        delete g;
        return fail(KPS_EINVAL, "unexpected failure while building the game");
    }
    *out = g;
    g_last_error.clear();
    return KPS_OK;
}

}  // namespace kps_abi

extern "C" {

kps_status kps_game_destroy(kps_game *g) {
    if (!g) return KPS_OK;
    if (g->dev.blob) cudaFree(g->dev.blob);
    if (g->stage_in) cudaFree(g->stage_in);
    if (g->stage_out) cudaFree(g->stage_out);
    if (g->host_streams) {
        for (cudaStream_t q : g->hstream)
            if (q) cudaStreamDestroy(q);
        if (g->hentry) cudaEventDestroy(g->hentry);
        for (int c = 0; c < kps_game::kHostChunks; ++c) {
            if (g->hin[c]) cudaEventDestroy(g->hin[c]);
            if (g->hdone[c]) cudaEventDestroy(g->hdone[c]);
        }
    }
    if (g->scratch) cudaFree(g->scratch);
    for (auto &kv : g->tiles) cudaFree(kv.second.dev);
    delete g;
    return KPS_OK;
}

kps_status kps_game_info(const kps_game *cg, kps_info *info) {
    if (!cg || !info) return fail(KPS_EINVAL, "NULL argument");
    kps_game *g = const_cast<kps_game *>(cg);
    try {
        kps::technique_b_counts(g->host);
    } catch (...) {
        return fail(KPS_ENOMEM, "counting Technique B sizes");
    }
    const kps::HostGame &h = g->host;
    std::memset(info, 0, sizeof(*info));
    info->H = h.H;
    info->hs = h.hs;
    info->n1 = h.n[0];
    info->n2 = h.n[1];
    info->T = h.T;
    info->T_fold = h.TF;
    info->T_showdown = h.TS;
    info->ncards = h.ncards;
    info->cards_per_hand = h.k;
    info->nodes1 = h.nodes[0];
    info->nodes2 = h.nodes[1];
    info->max_tie = h.max_tie;
    info->beta = h.beta;
    info->pot0 = h.pot0;
    info->nnz_A = h.counts[0];
    info->nnz_Ahat = h.counts[1];
    info->nnz_U = h.counts[2];
    info->nnz_M = h.counts[3];
    info->nnz_V = h.counts[4];
    info->pp_nnz_Ahat = h.counts[5];
    info->pp_nnz_U = h.counts[6];
    info->pp_nnz_M = h.counts[7];
    info->pp_nnz_V = h.counts[8];
    return KPS_OK;
}

kps_status kps_game_hands(const kps_game *g, int32_t *cards, int32_t *canon) {
    if (!g) return fail(KPS_EINVAL, "game is NULL");
    const kps::HostGame &h = g->host;
    for (int p = 0; p < h.H; ++p) {
        if (cards)
            for (int j = 0; j < h.k; ++j) cards[p * h.k + j] = h.slot_card[h.hand_slots[2 * p + j]];
        if (canon) canon[p] = h.canon[p];
    }
    return KPS_OK;
}

kps_status kps_game_sequences(const kps_game *g, int32_t player, int32_t *seq_node, int32_t *seq_parent,
                              int32_t *seq_action, double *seq_amount, int32_t *nodes_nact) {
    if (!g) return fail(KPS_EINVAL, "game is NULL");
    if (player != 0 && player != 1) return fail(KPS_EINVAL, "player must be 0 or 1");
    const kps::HostGame &h = g->host;
    const auto &sq = h.seqs[player];
    for (size_t s = 0; s < sq.size(); ++s) {
        if (seq_node) seq_node[s] = sq[s].node;
        if (seq_parent) seq_parent[s] = sq[s].parent;
        if (seq_action) seq_action[s] = sq[s].action;
        if (seq_amount) seq_amount[s] = sq[s].amount;
    }
    if (nodes_nact)
        for (size_t i = 0; i < h.nodes_nact[player].size(); ++i) nodes_nact[i] = h.nodes_nact[player][i];
    return KPS_OK;
}

kps_status kps_game_terminals(const kps_game *g, int32_t *s1, int32_t *s2, int32_t *kind, int32_t *folder,
                              double *c1, double *c2) {
    if (!g) return fail(KPS_EINVAL, "game is NULL");
    const auto &ts = g->host.terms;
    for (size_t t = 0; t < ts.size(); ++t) {
        if (s1) s1[t] = ts[t].s1;
        if (s2) s2[t] = ts[t].s2;
        if (kind) kind[t] = ts[t].kind;
        if (folder) folder[t] = ts[t].folder;
        if (c1) c1[t] = ts[t].c1;
        if (c2) c2[t] = ts[t].c2;
    }
    return KPS_OK;
}

kps_status kps_game_upload(kps_game *g, void *stream) {
    if (!g) return fail(KPS_EINVAL, "game is NULL");
    return upload(g, static_cast<cudaStream_t>(stream));
}

kps_status kps_game_kernel(const kps_game *g, int32_t dir, int32_t *kernel) {
    if (!g || !kernel) return fail(KPS_EINVAL, "NULL argument");
    if (dir != 0 && dir != 1) return fail(KPS_EINVAL, "dir must be 0 (A) or 1 (A^T)");
    *kernel = g->last_kernel[dir];
    return KPS_OK;
}

kps_status kps_matvec_A(kps_game *g, const void *y, void *out, int32_t batch, kps_dtype dt, void *stream) {
    return matvec(g, 0, y, out, batch, dt, stream);
}

kps_status kps_matvec_AT(kps_game *g, const void *x, void *out, int32_t batch, kps_dtype dt, void *stream) {
    return matvec(g, 1, x, out, batch, dt, stream);
}

kps_status kps_matvec_A_host(kps_game *g, const void *y, void *out, int32_t batch, kps_dtype dt,
                             void *stream) {
    return matvec_host(g, 0, y, out, batch, dt, stream);
}

kps_status kps_matvec_AT_host(kps_game *g, const void *x, void *out, int32_t batch, kps_dtype dt,
                              void *stream) {
    return matvec_host(g, 1, x, out, batch, dt, stream);
}

// A*y for BF16/FP16 storage whose FP32 partial results (and tile list) live
// in the library's statically reserved device array instead of memory
// obtained from cudaMalloc.  Same kernel and results as kps_matvec_A with the
// scalar-staging path; see include/kps.h for the contract.
kps_status kps_matvec_A_static_scratch(kps_game *g, const void *y, void *out, int32_t batch, kps_dtype dt,
                                       void *stream_ptr) {
    if (!g) return fail(KPS_EINVAL, "game is NULL");
    if (dt != KPS_BF16 && dt != KPS_F16) return fail(KPS_EINVAL, "dtype must be KPS_BF16 or KPS_F16");
    if (batch < 0) return fail(KPS_EINVAL, "batch must be >= 0");
    if (batch == 0) return KPS_OK;
    if (!y || !out) return fail(KPS_EINVAL, "vector pointer is NULL");
    if (!g->uploaded) return fail(KPS_EINVAL, "the game's tables are not on the device: call kps_game_upload first");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != g->device) return fail(KPS_EINVAL, "game tables live on another device");
    const kps::HostGame &h = g->host;
    const int n_out = h.n[0], n_in = h.n[1];
    const size_t floats = (size_t)batch * n_out * h.hs;
    if (floats > kps::kStaticScratchFloats)
        return fail(KPS_EINVAL, "batch * n1 * hs = " + std::to_string(floats) +
                                    " exceeds the static scratch of " + std::to_string(kps::kStaticScratchFloats) +
                                    " floats");
    const size_t in_bytes = (size_t)batch * n_in * h.hs * 2, out_bytes = floats * 2;
    const char *ci = static_cast<const char *>(y), *co = static_cast<const char *>(out);
    if (ci < co + out_bytes && co < ci + in_bytes) return fail(KPS_EINVAL, "input and output overlap");
    const int storage = dt == KPS_BF16 ? kps::kStoreBF16 : kps::kStoreF16;
    const int nc = h.ncards + 1;
    if (h.max_tie > kps::kTile) return fail(KPS_ENOTSUP, "tie groups longer than a tile");
    const int nw = fast_warps(storage, nc, h.H, false);
    if (kps::fast_smem_bytes(storage, nc, nw) > (size_t)kps::max_dyn_smem())
        return fail(KPS_ENOTSUP, "card count too large for shared memory");
    // the tile list kps_matvec_A's scalar-staging path uses for nw warps
    // (same chunk boundaries, hence the same summation order)
    std::vector<int> tchunk;
    bool spill = false;
    std::vector<std::pair<int, int>> tl = layout_tiles(h, nw, tchunk, &spill);
    if (tl.size() * sizeof(int2) > kps::kStaticTileBytes) return fail(KPS_ENOTSUP, "tile list too long");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    // the tile list is copied from a host vector that dies with this call,
    // so the call cannot be recorded into a graph
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(stream, &cap);
    if (e != cudaSuccess) return cuda_fail(e, "querying the stream's capture status");
    if (cap != cudaStreamCaptureStatusNone) return fail(KPS_EINVAL, "the stream is capturing a graph: this call cannot be captured");
    void *base = nullptr;
    e = kps::static_scratch_address(&base);
    if (e != cudaSuccess) return cuda_fail(e, "looking up the static scratch");
    std::vector<int2> tiles(tl.size());
    for (size_t i = 0; i < tl.size(); ++i) tiles[i] = make_int2(tl[i].first, tl[i].second);
    if (!tiles.empty()) {
        // pageable source: the copy is staged before this call returns
        e = cudaMemcpyAsync(base, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return cuda_fail(e, "copying the tile list");
    }
    const DeviceTables &t = g->dev;
    kps::FastParams p{};
    p.vin = y;
    p.vout = out;
    p.scratch = static_cast<unsigned char *>(base) + kps::kStaticTileBytes;
    p.H = h.H;
    p.hs = h.hs;
    p.nc = nc;
    p.n_out = n_out;
    p.n_in = n_in;
    p.batch = batch;
    p.fcol = t.fcol[0];
    p.scol = t.scol[0];
    p.fcoef = t.fcoef_f[0];
    p.scoef = t.scoef_f[0];
    p.hinfo = t.hinfo;
    p.lam_in = t.lam2_f;
    p.lam_out = t.lam1_f;
    p.tiles = static_cast<const int2 *>(base);
    p.nw = nw;
    for (int i = 0; i <= nw; ++i) p.tchunk[i] = tchunk[i];
    e = kps::launch_fast_scan(p, storage, h.k, stream);
    if (e != cudaSuccess) return cuda_fail(e, "launching the payoff scan");
    return KPS_OK;
}

const char *kps_last_error(void) { return g_last_error.c_str(); }

kps_status kps_device_status(void *stream) {
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "synchronising the stream");
    bool set = false, pset = false;
    e = kps::tma_take_error(&set);
    if (e == cudaSuccess) e = predict_take_error(&pset);
    if (e != cudaSuccess) return cuda_fail(e, "reading the device wait flags");
    if (set)
        return fail(KPS_ETIMEOUT, "a bounded wait of the TMA-staged kernel gave up: products since the last check "
                                  "are not valid");
    if (pset)
        return fail(KPS_ETIMEOUT, "a bounded wait of the warm-start predictor gave up: its predictions since the "
                                  "last check are not valid");
    return KPS_OK;
}

const char *kps_version(void) { return "kps 0.1.0 (sm_103a)"; }

}  // extern "C"
