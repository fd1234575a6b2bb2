// Batches of games in one persistent launch (C ABI in include/kps.h).
//
// A batch concatenates one player-1 and one player-2 vector per game: game
// g's vector of player p starts off[p][g] elements into the batch vector
// and has n_p(g) rows of hs(g) entries.  One launch of the multi-game kernel
// covers every (game, 32-column tile) of a direction; the CTAs are
// persistent and take tiles from an atomic ticket counter (or a static
// stride), so uneven hand counts and tree sizes share the machine without a
// launch per game.  The launch shape (warps per CTA, CTAs, schedule) comes
// from the batch's own autotuner (kps_batch_tune), which times every
// candidate with CUDA events on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "abi_internal.h"
#include "batch_internal.h"
#include "kernels.h"

using namespace kps_abi;

namespace kps_abi {

namespace {


int storage_of(kps_dtype dt) {
    return dt == KPS_F32 ? kps::kStoreF32 : dt == KPS_F64 ? kps::kStoreF64 : dt == KPS_BF16 ? kps::kStoreBF16
                                                                                             : kps::kStoreF16;
}

int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// Smallest warp count whose tile lists fit every game's chunks into the
// tensor-memory layout; 0 if none does.  Host only.
int tmem_min_warps(kps_batch *b) {
    for (int nw = 1; nw <= kps::kMaxWarps; ++nw) {
        bool ok = true;
        for (kps_game *g : b->games) {
            if (!kps_abi::tmem_split_fits(g->host, nw)) { ok = false; break; }
        }
        if (ok) return nw;
    }
    return 0;
}

}  // namespace

bool batch_staged_ready(kps_batch *b, cudaStream_t stream) {
    if (b->am_state != 0) return b->am_state == 1;
    b->am_state = -1;
    const int ng = (int)b->games.size();
    for (int dir = 0; dir < 2; ++dir) {
        std::vector<kps::AmGameDesc> d(ng);
        for (int i = 0; i < ng; ++i) {
            const kps_game *g = b->games[i];
            const kps::HostGame &h = g->host;
            kps::AmGameDesc &x = d[i];
            x.h = &h;
            x.lam_in = dir == 0 ? h.lam2.data() : h.lam1.data();
            x.lam_out = dir == 0 ? h.lam1.data() : h.lam2.data();
            x.n_out = dir == 0 ? h.n[0] : h.n[1];
            x.fcol = g->dev.fcol[dir];
            x.scol = g->dev.scol[dir];
            x.fcoef = g->dev.fcoef_f[dir];
            x.scoef = g->dev.scoef_f[dir];
            x.in_off = b->off[dir == 0 ? 1 : 0][i];
            x.out_off = b->off[dir == 0 ? 0 : 1][i];
        }
        std::string why;
        std::vector<char> taken;
        b->am[dir] = kps::am_create(d, 2 * sm_count(), stream, &taken, &why);
        bool ok = b->am[dir] != nullptr && kps::am_ctas_per_sm(b->am[dir]) >= 1;
        if (ok && dir == 1) ok = b->am_rest.size() == taken.size();
        for (int i = 0; ok && i < ng; ++i) {
            if (dir == 0) b->am_rest.push_back(taken[i] ? 0 : 1);
            else ok = b->am_rest[i] == (taken[i] ? 0 : 1);
        }
        if (!ok) {
            for (int k = 0; k < 2; ++k) {
                kps::am_destroy(b->am[k]);
                b->am[k] = nullptr;
            }
            b->am_rest.clear();
            return false;
        }
    }
    // the games left to the tensor-memory kernel, and its warp count for them
    b->am_nrest = 0;
    int lo = 0;
    bool fit4 = true;
    for (int i = 0; i < ng; ++i) {
        if (!b->am_rest[i]) continue;
        ++b->am_nrest;
        const kps::HostGame &h = b->games[i]->host;
        int w = 1;
        while (w <= kps::kMaxWarps && !kps_abi::tmem_split_fits(h, w)) ++w;
        lo = std::max(lo, w);
        fit4 = fit4 && kps_abi::tmem_split_fits(h, 4);
    }
    if (b->am_nrest > 0) {
        if (lo > kps::kMaxWarps || b->games[0]->host.ncards + 1 > 66) {
            for (int k = 0; k < 2; ++k) {
                kps::am_destroy(b->am[k]);
                b->am[k] = nullptr;
            }
            b->am_rest.clear();
            return false;
        }
        b->rest_nw = fit4 && lo <= 4 ? 4 : lo;
    }
    b->am_state = 1;
    return true;
}

namespace {

// Launch table of one (direction, FP64 or not, warp count) over every game,
// or over the games with only[i] != 0.
kps_status build_table(kps_batch *b, int dir, bool f64, int nw, const std::vector<char> *only, cudaStream_t stream,
                       BatchTable *tb_out) {
    const int ng = (int)b->games.size();
    std::vector<kps::FastParams> fp(ng);
    std::vector<long long> tstart(ng + 1, 0), in_off(ng), out_off(ng);
    std::vector<int> tgame;
    int nc = 0;
    bool any_spill = false;
    for (int i = 0; i < ng; ++i) {
        in_off[i] = b->off[dir == 0 ? 1 : 0][i];
        out_off[i] = b->off[dir == 0 ? 0 : 1][i];
        if (only && !(*only)[i]) {
            std::memset(&fp[i], 0, sizeof(fp[i]));
            tstart[i + 1] = tstart[i];
            continue;
        }
        kps_game *g = b->games[i];
        const kps::HostGame &h = g->host;
        const kps_game::Tiles *t = nullptr;
        kps_status st = tiles_for(g, nw, stream, &t);
        if (st != KPS_OK) return st;
        const DeviceTables &d = g->dev;
        kps::FastParams &p = fp[i];
        std::memset(&p, 0, sizeof(p));
        p.H = h.H;
        p.hs = h.hs;
        p.nc = h.ncards + 1;
        p.n_out = dir == 0 ? h.n[0] : h.n[1];
        p.n_in = dir == 0 ? h.n[1] : h.n[0];
        p.batch = 1;
        p.fcol = d.fcol[dir];
        p.scol = d.scol[dir];
        p.fcoef = f64 ? (const void *)d.fcoef_d[dir] : (const void *)d.fcoef_f[dir];
        p.scoef = f64 ? (const void *)d.scoef_d[dir] : (const void *)d.scoef_f[dir];
        p.hinfo = d.hinfo;
        const void *l1 = f64 ? (const void *)d.lam1_d : (const void *)d.lam1_f;
        const void *l2 = f64 ? (const void *)d.lam2_d : (const void *)d.lam2_f;
        p.lam_in = dir == 0 ? l2 : l1;
        p.lam_out = dir == 0 ? l1 : l2;
        p.tiles = t->dev;
        p.tie_work = t->tie_work;
        p.tie_trip = t->tie_trip;
        p.spill = t->spill ? 1 : 0;
        any_spill = any_spill || t->spill;
        p.nw = nw;
        for (int k = 0; k <= nw; ++k) p.tchunk[k] = t->tchunk[k];
        nc = std::max(nc, p.nc);
        const int nt = (p.n_out + 31) / 32;
        tstart[i + 1] = tstart[i] + nt;
        for (int k = 0; k < nt; ++k) tgame.push_back(i);
    }
    if (tstart[ng] > 0x7fffffffLL) return fail(KPS_ENOTSUP, "too many column tiles in one batch");
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t o_fp = 0, o_ts = al(o_fp + sizeof(kps::FastParams) * ng), o_tg = al(o_ts + 8 * (size_t)(ng + 1)),
                 o_in = al(o_tg + 4 * std::max<size_t>(1, tgame.size())), o_out = al(o_in + 8 * (size_t)ng),
                 total = al(o_out + 8 * (size_t)ng);
    std::vector<unsigned char> host(total, 0);
    std::memcpy(host.data() + o_fp, fp.data(), sizeof(kps::FastParams) * ng);
    std::memcpy(host.data() + o_ts, tstart.data(), 8 * (size_t)(ng + 1));
    if (!tgame.empty()) std::memcpy(host.data() + o_tg, tgame.data(), 4 * tgame.size());
    std::memcpy(host.data() + o_in, in_off.data(), 8 * (size_t)ng);
    std::memcpy(host.data() + o_out, out_off.data(), 8 * (size_t)ng);
    BatchTable tb;
    cudaError_t e = cudaMalloc(&tb.blob, total);
    if (e != cudaSuccess) return fail(KPS_ENOMEM, "batch launch table");
    e = cudaMemcpyAsync(tb.blob, host.data(), total, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        cudaFree(tb.blob);
        return cuda_fail(e, "uploading the batch launch table");
    }
    unsigned char *bl = static_cast<unsigned char *>(tb.blob);
    tb.m.games = reinterpret_cast<const kps::FastParams *>(bl + o_fp);
    tb.m.tile_start = reinterpret_cast<const long long *>(bl + o_ts);
    tb.m.tile_game = reinterpret_cast<const int *>(bl + o_tg);
    tb.m.in_off = reinterpret_cast<const long long *>(bl + o_in);
    tb.m.out_off = reinterpret_cast<const long long *>(bl + o_out);
    tb.m.ticket = b->ticket;
    tb.m.ngames = ng;
    tb.m.total_tiles = (int)tstart[ng];
    tb.m.nw = nw;
    tb.m.nc = nc;
    tb.m.spill = any_spill ? 1 : 0;
    tb.m.schedule = 0;
    *tb_out = tb;
    return KPS_OK;
}

}  // namespace

kps_status batch_table(kps_batch *b, int dir, bool f64, int nw, cudaStream_t stream, const BatchTable **out) {
    const auto key = std::make_tuple(dir, f64, nw);
    auto it = b->tables.find(key);
    if (it != b->tables.end()) {
        *out = &it->second;
        return KPS_OK;
    }
    BatchTable tb;
    kps_status st = build_table(b, dir, f64, nw, nullptr, stream, &tb);
    if (st != KPS_OK) return st;
    *out = &b->tables.emplace(key, tb).first->second;
    return KPS_OK;
}

kps_status batch_rest_table(kps_batch *b, int dir, cudaStream_t stream, const BatchTable **out) {
    auto it = b->rest_tables.find(dir);
    if (it != b->rest_tables.end()) {
        *out = &it->second;
        return KPS_OK;
    }
    BatchTable tb;
    kps_status st = build_table(b, dir, false, b->rest_nw, &b->am_rest, stream, &tb);
    if (st != KPS_OK) return st;
    *out = &b->rest_tables.emplace(dir, tb).first->second;
    return KPS_OK;
}

// The launch shape used for `dt` when the batch has not been tuned.
kps_status batch_default_shape(kps_batch *b, kps_dtype dt, cudaStream_t stream, BatchShape *out) {
    auto it = b->shape.find((int)dt);
    if (it != b->shape.end()) {
        *out = it->second;
        return KPS_OK;
    }
    BatchShape s;
    const int storage = storage_of(dt);
    int maxH = 0, maxnc = 0;
    for (kps_game *g : b->games) {
        maxH = std::max(maxH, g->host.H);
        maxnc = std::max(maxnc, g->host.ncards + 1);
    }
    if (dt == KPS_F64) {
        if (maxnc > 64) return fail(KPS_ENOTSUP, "card count too large for the FP64 batch kernel");
        s.nw = 8;
        while (s.nw > 1 && kps::vec_smem_bytes(storage, maxnc, s.nw) > (size_t)kps::max_dyn_smem()) --s.nw;
        s.nw = std::max(1, std::min(s.nw, (maxH + kps::kTile - 1) / kps::kTile));
        s.per_sm = std::max(1, kps::vec_multi_ctas_per_sm(storage, b->k, maxnc, s.nw));
    } else if (dt != KPS_F64 && batch_staged_ready(b, stream)) {
        s.kernel = KPS_BATCH_STAGED;
        s.nw = 4;
        s.per_sm = std::min(kps::am_ctas_per_sm(b->am[0]), kps::am_ctas_per_sm(b->am[1]));
    } else {
        if (maxnc > 66) return fail(KPS_ENOTSUP, "card count too large for the tensor-memory kernel");
        const int lo = tmem_min_warps(b);
        if (lo == 0) return fail(KPS_ENOTSUP, "hand chunk too long for tensor memory");
        s.nw = std::max(lo, std::min(kps::kMaxWarps, (maxH + kps::kTile - 1) / kps::kTile));
        // two CTAs of four warps per SM (their phases overlap) when every
        // game's four-way split fits
        if (s.nw > 4 && kps::tmem_multi_ctas_per_sm(storage, b->k, maxnc, 4) >= 2) {
            bool fit = true;
            for (kps_game *g : b->games) fit = fit && kps_abi::tmem_split_fits(g->host, 4);
            if (fit) s.nw = 4;
        }
        s.per_sm = std::max(1, kps::tmem_multi_ctas_per_sm(storage, b->k, maxnc, s.nw));
    }
    s.grid = sm_count() * s.per_sm;
    s.schedule = 0;
    b->shape[(int)dt] = s;
    *out = s;
    return KPS_OK;
}

kps_status batch_matvec(kps_batch *b, int dir, const void *vin, void *vout, kps_dtype dt, cudaStream_t stream) {
    if (!b) return fail(KPS_EINVAL, "batch is NULL");
    if (dtype_size(dt) == 0) return fail(KPS_EINVAL, "unknown dtype");
    if (!vin || !vout) return fail(KPS_EINVAL, "vector pointer is NULL");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != b->device) return fail(KPS_EINVAL, "batch tables live on another device");
    const size_t es = dtype_size(dt);
    const size_t in_bytes = (size_t)b->off[dir == 0 ? 1 : 0].back() * es;
    const size_t out_bytes = (size_t)b->off[dir == 0 ? 0 : 1].back() * es;
    const char *ci = static_cast<const char *>(vin), *co = static_cast<const char *>(vout);
    if (ci < co + out_bytes && co < ci + in_bytes) return fail(KPS_EINVAL, "input and output overlap");
    if (((reinterpret_cast<uintptr_t>(vin) | reinterpret_cast<uintptr_t>(vout)) & 15) != 0)
        return fail(KPS_EINVAL, "batch vectors must be 16-byte aligned");
    BatchShape s;
    kps_status st = batch_default_shape(b, dt, stream, &s);
    if (st != KPS_OK) return st;
    if (s.kernel == KPS_BATCH_STAGED) {
        cudaError_t e = cudaSuccess;
        if (s.schedule == 0) e = cudaMemsetAsync(b->ticket, 0, sizeof(int), stream);
        if (e != cudaSuccess) return cuda_fail(e, "clearing the work-item ticket");
        e = kps::launch_async_multi(b->am[dir], storage_of(dt), vin, vout, b->ticket, s.schedule, s.grid, stream);
        if (e != cudaSuccess) return cuda_fail(e, "launching the staged batched payoff scan");
        if (b->am_nrest > 0) {
            // the games the staged kernel leaves: tensor-memory kernel, static stride
            const BatchTable *t = nullptr;
            st = batch_rest_table(b, dir, stream, &t);
            if (st != KPS_OK) return st;
            kps::MultiParams m = t->m;
            m.vin = vin;
            m.vout = vout;
            m.schedule = 1;
            const int per = std::max(1, kps::tmem_multi_ctas_per_sm(storage_of(dt), b->k, m.nc, m.nw));
            const int grid = std::max(1, std::min(m.total_tiles, sm_count() * per));
            e = kps::launch_tmem_multi(m, storage_of(dt), b->k, grid, stream);
            if (e != cudaSuccess) return cuda_fail(e, "launching the batched payoff scan of the remaining games");
        }
        return KPS_OK;
    }
    const BatchTable *t = nullptr;
    st = batch_table(b, dir, dt == KPS_F64, s.nw, stream, &t);
    if (st != KPS_OK) return st;
    kps::MultiParams m = t->m;
    m.vin = vin;
    m.vout = vout;
    m.schedule = s.schedule;
    cudaError_t e = cudaSuccess;
    if (s.schedule == 0) e = cudaMemsetAsync(b->ticket, 0, sizeof(int), stream);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the tile ticket");
    const int storage = storage_of(dt);
    e = dt == KPS_F64 ? kps::launch_vec_multi(m, storage, b->k, s.grid, stream)
                      : kps::launch_tmem_multi(m, storage, b->k, s.grid, stream);
    if (e != cudaSuccess) return cuda_fail(e, "launching the batched payoff scan");
    return KPS_OK;
}

}  // namespace kps_abi

extern "C" {

kps_status kps_batch_create(kps_game *const *games, int32_t n, kps_batch **out) {
    if (!out) return fail(KPS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!games || n <= 0) return fail(KPS_EINVAL, "a batch needs at least one game");
    kps_batch *b = new (std::nothrow) kps_batch;
    if (!b) return fail(KPS_ENOMEM, "batch object");
    b->games.assign(games, games + n);
    b->k = games[0] ? games[0]->host.k : 0;
    for (int p = 0; p < 2; ++p) b->off[p].assign(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        kps_game *g = games[i];
        if (!g) { delete b; return fail(KPS_EINVAL, "game " + std::to_string(i) + " is NULL"); }
        if (g->host.k != b->k) { delete b; return fail(KPS_EINVAL, "games of a batch must share cards_per_hand"); }
        if (g->host.max_tie > kps::kTile) {
            delete b;
            return fail(KPS_ENOTSUP, "game " + std::to_string(i) + " has a tie group longer than 32 hands");
        }
        kps_status st = upload(g, nullptr);
        if (st != KPS_OK) { delete b; return st; }
        for (int p = 0; p < 2; ++p) b->off[p][i + 1] = b->off[p][i] + (long long)g->host.n[p] * g->host.hs;
    }
    cudaGetDevice(&b->device);
    cudaError_t e = cudaMalloc(&b->ticket, 256);
    if (e != cudaSuccess) { delete b; return fail(KPS_ENOMEM, "ticket counter"); }
    *out = b;
    return KPS_OK;
}

kps_status kps_batch_destroy(kps_batch *b) {
    if (!b) return KPS_OK;
    for (auto &kv : b->tables) cudaFree(kv.second.blob);
    for (auto &kv : b->rest_tables) cudaFree(kv.second.blob);
    for (int k = 0; k < 2; ++k) kps::am_destroy(b->am[k]);
    warm_free(b);
    if (b->ticket) cudaFree(b->ticket);
    delete b;
    return KPS_OK;
}

kps_status kps_batch_offsets(const kps_batch *b, int32_t player, int64_t *off) {
    if (!b || !off || player < 0 || player > 1) return fail(KPS_EINVAL, "bad argument");
    for (size_t i = 0; i < b->off[player].size(); ++i) off[i] = b->off[player][i];
    return KPS_OK;
}

kps_status kps_batch_matvec_A(kps_batch *b, const void *y, void *out, kps_dtype dt, void *stream) {
    return batch_matvec(b, 0, y, out, dt, static_cast<cudaStream_t>(stream));
}

kps_status kps_batch_matvec_AT(kps_batch *b, const void *x, void *out, kps_dtype dt, void *stream) {
    return batch_matvec(b, 1, x, out, dt, static_cast<cudaStream_t>(stream));
}

kps_status kps_batch_tune(kps_batch *b, kps_dtype dt, void *stream_ptr, kps_batch_shape *chosen) {
    if (!b) return fail(KPS_EINVAL, "batch is NULL");
    if (dtype_size(dt) == 0) return fail(KPS_EINVAL, "unknown dtype");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    BatchShape base;
    kps_status st = batch_default_shape(b, dt, stream, &base);
    if (st != KPS_OK) return st;
    const int storage = storage_of(dt);
    int maxnc = 0, maxH = 0;
    for (kps_game *g : b->games) {
        maxnc = std::max(maxnc, g->host.ncards + 1);
        maxH = std::max(maxH, g->host.H);
    }
    // candidates: every admissible warp count, both schedules, one or all
    // resident CTAs per SM
    int lo = 1;
    if (dt != KPS_F64) lo = tmem_min_warps(b);
    const int hi = std::min(kps::kMaxWarps, std::max(lo, (maxH + kps::kTile - 1) / kps::kTile));
    std::vector<BatchShape> cands;
    for (int nw = lo; nw <= hi; ++nw) {
        if (dt == KPS_F64 && kps::vec_smem_bytes(storage, maxnc, nw) > (size_t)kps::max_dyn_smem()) continue;
        const int per = dt == KPS_F64 ? kps::vec_multi_ctas_per_sm(storage, b->k, maxnc, nw)
                                      : kps::tmem_multi_ctas_per_sm(storage, b->k, maxnc, nw);
        if (per < 1) continue;
        for (int sched = 0; sched < 2; ++sched)
            for (int mul = 1; mul <= per; mul = mul == per ? per + 1 : per) {
                BatchShape s;
                s.nw = nw;
                s.per_sm = mul;
                s.grid = sm_count() * mul;
                s.schedule = sched;
                cands.push_back(s);
            }
    }
    if (dt != KPS_F64 && batch_staged_ready(b, stream)) {
        const int per = std::min(kps::am_ctas_per_sm(b->am[0]), kps::am_ctas_per_sm(b->am[1]));
        for (int sched = 0; sched < 2; ++sched)
            for (int mul = 1; mul <= per; ++mul) {
                BatchShape s;
                s.kernel = KPS_BATCH_STAGED;
                s.nw = 4;
                s.per_sm = mul;
                s.grid = sm_count() * mul;
                s.schedule = sched;
                cands.push_back(s);
            }
    }
    if (cands.empty()) return fail(KPS_ENOTSUP, "no launch shape fits this batch");
    const size_t es = dtype_size(dt);
    void *vin = nullptr, *vout = nullptr;
    const size_t nin = std::max(b->off[0].back(), b->off[1].back());
    cudaError_t e = cudaMalloc(&vin, nin * es);
    if (e == cudaSuccess) e = cudaMalloc(&vout, nin * es);
    if (e != cudaSuccess) {
        cudaFree(vin);
        return fail(KPS_ENOMEM, "tuning buffers");
    }
    cudaMemsetAsync(vin, 0, nin * es, stream);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // Warm the GPU up first (clocks rise over the first milliseconds of
    // work, which would penalise the candidates timed first), then time every
    // candidate in two passes and keep its faster one.
    b->shape[(int)dt] = base;
    for (int rep = 0; rep < 20; ++rep) {
        if (batch_matvec(b, 0, vin, vout, dt, stream) != KPS_OK || batch_matvec(b, 1, vin, vout, dt, stream) != KPS_OK)
            break;
    }
    cudaStreamSynchronize(stream);
    std::vector<float> cbest(cands.size(), -1.f);
    for (int pass = 0; pass < 2; ++pass)
        for (size_t ci = 0; ci < cands.size(); ++ci) {
            if (pass > 0 && cbest[ci] < 0.f) continue;       // failed in the first pass
            b->shape[(int)dt] = cands[ci];
            float tot = 0.f;
            bool ok = true;
            for (int rep = 0; rep < 4 && ok; ++rep) {
                cudaEventRecord(e0, stream);
                ok = batch_matvec(b, 0, vin, vout, dt, stream) == KPS_OK &&
                     batch_matvec(b, 1, vin, vout, dt, stream) == KPS_OK;
                cudaEventRecord(e1, stream);
                if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) tot += ms;   // the first run builds tables and warms up
            }
            if (!ok) {
                cbest[ci] = -1.f;
                continue;
            }
            if (cbest[ci] < 0.f || tot < cbest[ci]) cbest[ci] = tot;
        }
    float best = -1.f;
    BatchShape bs = base;
    for (size_t ci = 0; ci < cands.size(); ++ci) {
        if (cbest[ci] < 0.f) continue;
        if (best < 0.f || cbest[ci] < best) {
            best = cbest[ci];
            bs = cands[ci];
            bs.ms = cbest[ci] / 3.f;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(vin);
    cudaFree(vout);
    b->shape[(int)dt] = bs;
    e = cudaGetLastError();
    if (best < 0.f) return fail(KPS_ECUDA, "every candidate launch shape failed");
    if (chosen) {
        chosen->warps = bs.nw;
        chosen->grid = bs.grid;
        chosen->schedule = bs.schedule;
        chosen->kernel = bs.kernel;
        chosen->ms_per_pair = bs.ms;
    }
    return KPS_OK;
}

kps_status kps_batch_shape_get(kps_batch *b, kps_dtype dt, kps_batch_shape *shape) {
    if (!b || !shape) return fail(KPS_EINVAL, "bad argument");
    BatchShape s;
    kps_status st = batch_default_shape(b, dt, nullptr, &s);
    if (st != KPS_OK) return st;
    shape->warps = s.nw;
    shape->grid = s.grid;
    shape->schedule = s.schedule;
    shape->kernel = s.kernel;
    shape->ms_per_pair = s.ms;
    return KPS_OK;
}

kps_status kps_batch_shape_set(kps_batch *b, kps_dtype dt, const kps_batch_shape *shape) {
    if (!b || !shape) return fail(KPS_EINVAL, "bad argument");
    if (dtype_size(dt) == 0) return fail(KPS_EINVAL, "unknown dtype");
    BatchShape cur;
    kps_status st = batch_default_shape(b, dt, nullptr, &cur);
    if (st != KPS_OK) return st;
    if (shape->schedule != 0 && shape->schedule != 1) return fail(KPS_EINVAL, "schedule must be 0 or 1");
    if (shape->grid < 1) return fail(KPS_EINVAL, "grid must be >= 1");
    if (shape->kernel != KPS_BATCH_TMEM && shape->kernel != KPS_BATCH_STAGED)
        return fail(KPS_EINVAL, "kernel must be KPS_BATCH_TMEM or KPS_BATCH_STAGED");
    if (shape->kernel == KPS_BATCH_STAGED) {
        if (dt == KPS_F64) return fail(KPS_ENOTSUP, "the staged kernel takes FP32, BF16 or FP16 vectors");
        if (shape->warps != 4) return fail(KPS_ENOTSUP, "the staged kernel runs 4 warps per CTA");
        if (!batch_staged_ready(b, nullptr)) return fail(KPS_ENOTSUP, "a game of the batch does not fit the staged kernel");
        if (shape->grid > kps::am_grid_cap(b->am[0])) return fail(KPS_ENOTSUP, "the staged kernel runs at most 2 CTAs per SM");
        BatchShape s = cur;
        s.kernel = KPS_BATCH_STAGED;
        s.nw = 4;
        s.grid = shape->grid;
        s.schedule = shape->schedule;
        s.ms = 0.0;
        b->shape[(int)dt] = s;
        return KPS_OK;
    }
    const int nw = shape->warps;
    if (nw < 1 || nw > kps::kMaxWarps) return fail(KPS_EINVAL, "warps must be in 1..8");
    int maxnc = 0;
    for (kps_game *g : b->games) maxnc = std::max(maxnc, g->host.ncards + 1);
    if (dt == KPS_F64) {
        if (kps::vec_smem_bytes(storage_of(dt), maxnc, nw) > (size_t)kps::max_dyn_smem())
            return fail(KPS_ENOTSUP, "warp count needs too much shared memory");
    } else if (nw < tmem_min_warps(b)) {
        return fail(KPS_ENOTSUP, "warp count leaves a hand chunk too long for tensor memory");
    }
    // a shape the multi-game kernel cannot launch (shared memory, registers)
    const int per = dt == KPS_F64 ? kps::vec_multi_ctas_per_sm(storage_of(dt), b->k, maxnc, nw)
                                  : kps::tmem_multi_ctas_per_sm(storage_of(dt), b->k, maxnc, nw);
    if (per < 1) return fail(KPS_ENOTSUP, "warp count needs too much shared memory or too many registers");
    BatchShape s = cur;
    s.kernel = KPS_BATCH_TMEM;
    s.nw = nw;
    s.grid = shape->grid;
    s.schedule = shape->schedule;
    s.ms = 0.0;
    b->shape[(int)dt] = s;
    return KPS_OK;
}

kps_status kps_partition(const int64_t *weights, int32_t n, int32_t parts, int32_t *bounds) {
    if (!bounds || n < 0 || parts < 1 || (n > 0 && !weights)) return fail(KPS_EINVAL, "bad argument");
    long long total = 0;
    for (int i = 0; i < n; ++i) {
        if (weights[i] < 0) return fail(KPS_EINVAL, "negative weight");
        total += weights[i];
    }
    bounds[0] = 0;
    long long cum = 0;
    int i = 0;
    for (int k = 1; k < parts; ++k) {
        // cut where the prefix sum comes closest to k/parts of the total
        const double target = (double)total * k / parts;
        while (i < n && (double)(cum + weights[i]) <= target) cum += weights[i++];
        if (i < n && (double)(cum + weights[i]) - target < target - (double)cum) cum += weights[i++];
        bounds[k] = i;
    }
    bounds[parts] = n;
    return KPS_OK;
}

}  // extern "C"
