// Vectorised fast path of the Kronecker-form payoff products (sm_103a),
// FP32 and FP64 storage.
//
// Mathematics as in kernels.cu / kernels_fast.cu:
//   out / lambda_out = K_F(u - v) + 2 Lo(v) + TieC(v)
// (u, v: lambda-weighted fold and showdown inputs of an output column; K_F
// the card-removal fold operator; Lo the compatible strictly-weaker mass).
//
// What this version changes, all to cut instructions and latency per
// (hand, column):
//   * every global transfer is a coalesced 16-byte access: consecutive
//     lanes move consecutive 16-byte pieces of one column's row, by
//     cp.async into shared memory ([column][hand] tiles, pitch 36 floats /
//     34 doubles) or by vector stores out of shared memory;
//   * all arithmetic runs lane = column on those tiles (128-bit loads of 4
//     or 2 hands of the lane's own row, conflict free per quarter warp);
//   * tiles are double-buffered (the next tile is in flight while the
//     current one is scanned or finished);
//   * the scan is specialised by column kind: fold only (K_F alone: one
//     per-card total), showdown only (one per-card running sum, w = -v), or
//     both (float2 per card); hands of the staging window outside the tile
//     get weight 0 and a spare card slot, so the unrolled scan has no range
//     checks, and the next 4 (2) hands' records and inputs are loaded before
//     the current ones are stored;
//   * the per-card tables are [card][lane] (lane-private, conflict free).
// Tie groups are corrected inside tie-aligned tiles exactly as in
// kernels_fast.cu.  No atomics: results are bit-reproducible.
#include "kernels.h"

#include <cstdint>

namespace kps {
namespace {

constexpr int kZPitch = 65;      // [column][card] table pitch (>= cards + 1, odd)

enum Kind { kKindF = 1, kKindS = 2, kKindFS = 3 };

template <typename S> struct Cfg;
template <> struct Cfg<float> {
    static constexpr int V = 4;    // elements per 16-byte vector
    static constexpr int W = 9;    // vectors covering any 32-hand tile
    static constexpr int P = 36;   // pitch of a staged column
    using C2 = float2;
    using Vec = float4;
    __device__ static float get(const Vec &x, int k) { return k == 0 ? x.x : k == 1 ? x.y : k == 2 ? x.z : x.w; }
    __device__ static Vec make(const float *v) { return make_float4(v[0], v[1], v[2], v[3]); }
};
template <> struct Cfg<double> {
    static constexpr int V = 2;
    static constexpr int W = 17;
    static constexpr int P = 34;
    using C2 = double2;
    using Vec = double2;
    __device__ static double get(const Vec &x, int k) { return k == 0 ? x.x : x.y; }
    __device__ static Vec make(const double *v) { return make_double2(v[0], v[1]); }
};

struct Col {
    long long in_off;
    long long out_off;   // -1 = no column
    int foff, soff;      // -1 = no such terminal
};

__device__ __forceinline__ void cp16(void *smem, const void *gmem, int bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> __device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ constexpr int hw_pitch(int P) { return (P + 4 + 3) / 4 * 4; }

// Byte layout of one warp's shared memory.
struct WarpLayout {
    size_t r, stage, lam, hw, ptile, total;
};
__host__ __device__ inline WarpLayout warp_layout(int nc, size_t cs, int P) {
    WarpLayout L;
    size_t o = 0;
    L.r = o;     o = al16(o + (size_t)nc * 32 * 2 * cs);         // per-card state
    // [buf][term][col][P] in the scan; Z [nc][32] + [buf][col][P] afterwards
    const size_t st = 2 * 2 * 32 * (size_t)P * cs, fin = ((size_t)nc * 32 + 2 * 32 * (size_t)P) * cs;
    L.stage = o; o = al16(o + (st > fin ? st : fin));
    L.lam = o;   o = al16(o + 2 * (size_t)(P + 4) * cs);         // [buf][P+4]
    L.hw = o;    o = al16(o + 2 * (size_t)hw_pitch(P) * 4);      // [buf][hw_pitch] hand records
    L.ptile = o; o = al16(o + 32 * (size_t)P * cs);              // [col][P]
    L.total = o;
    return L;
}
__host__ __device__ inline size_t header_bytes(int nw, size_t cs) {
    return al16(32 * sizeof(Col) + 2 * 32 * cs + (size_t)nw * 3 * 32 * cs);
}

template <typename S, int K2, int KIND>
__device__ __forceinline__ void scan_body(const FastParams &p, unsigned char *smem, const Col *ci,
                                          const S *fco_s, const S *sco_s, S *sums, bool uni, int nvalid) {
    using C = S;
    using CF = Cfg<S>;
    using C2 = typename CF::C2;
    using Vec = typename CF::Vec;
    constexpr int V = CF::V, W = CF::W, P = CF::P, HP = hw_pitch(CF::P);
    constexpr bool HF = (KIND & kKindF) != 0, HS = (KIND & kKindS) != 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = p.nw, nc = p.nc;
    const int H = p.H, hs = p.hs;
    const size_t cs = sizeof(C);
    const WarpLayout WL = warp_layout(nc, cs, P);
    const size_t hdr = header_bytes(nw, cs);
    unsigned char *mine = smem + hdr + (size_t)warp * WL.total;
    C2 *R2 = reinterpret_cast<C2 *>(mine + WL.r) + lane;   // [card][32]: {v running, w total}
    C *R1 = reinterpret_cast<C *>(mine + WL.r) + lane;     // [card][32]: one kind
    C *stage = reinterpret_cast<C *>(mine + WL.stage);     // [buf][term][32][P]
    C *lamw = reinterpret_cast<C *>(mine + WL.lam);        // [buf][P + 4]
    uint32_t *hw = reinterpret_cast<uint32_t *>(mine + WL.hw);  // [buf][HP]
    C *ptile = reinterpret_cast<C *>(mine + WL.ptile);     // [32][P]
    const S *vin = static_cast<const S *>(p.vin);
    S *vout = static_cast<S *>(p.vout);
    C *scr = static_cast<C *>(p.scratch);
    const C *lam_in = static_cast<const C *>(p.lam_in);
    const C *lam_out = static_cast<const C *>(p.lam_out);
    const long long istride = (long long)p.n_in * hs, ostride = (long long)p.n_out * hs;
    const C fco = fco_s[lane], sco = sco_s[lane];
    const Col c0 = ci[0];
    // column jj's input rows and output row (coalesced transfers use any jj)
    auto col_in = [&](int jj, int term) -> const S * {
        if (uni) {
            const int o = term == 0 ? c0.foff : c0.soff;
            return (jj < nvalid && o >= 0) ? vin + c0.in_off + jj * istride + o : nullptr;
        }
        const Col cj = ci[jj];
        const int o = term == 0 ? cj.foff : cj.soff;
        return (cj.out_off >= 0 && o >= 0) ? vin + cj.in_off + o : nullptr;
    };
    auto col_out = [&](int jj) -> long long {
        if (uni) return jj < nvalid ? c0.out_off + jj * ostride : -1;
        return ci[jj].out_off;
    };
    // hands outside the current tile point at this card slot with weight 0
    const uint32_t kTrash = (uint32_t)(nc - 1) | ((uint32_t)(nc - 1) << 6);

    if (HF && HS) {
        for (int c = 0; c < nc; ++c) R2[c * 32] = C2{C(0), C(0)};
    } else {
        for (int c = 0; c < nc; ++c) R1[c * 32] = C(0);
    }

    // ---- phase 1: scan (lane = column)
    const int tb = p.tchunk[warp], te = p.tchunk[warp + 1];
    // 16-byte pieces of the window [wb, wb + nv V) of every column, coalesced:
    // lane l of step i moves piece (l + 32 i) % W of column (l + 32 i) / W.
    // Pieces past the tile end are zero-filled.
    auto stage_tile = [&](int t, int buf) {
        const int2 tl = p.tiles[t];
        const int wb = tl.x & ~(V - 1), end = tl.x + tl.y;
        const int nv = (end - wb + V - 1) / V;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const int idx = lane + 32 * i, jj = idx / W, v = idx - jj * W;
            if (v >= nv) continue;
            const int inside = min(V, end - (wb + v * V)) * (int)sizeof(C);
            if (HF) {
                const S *src = col_in(jj, 0);
                cp16(stage + ((size_t)(buf * 2 + 0) * 32 + jj) * P + v * V,
                     src ? (const void *)(src + wb + v * V) : (const void *)vin, src ? inside : 0);
            }
            if (HS) {
                const S *src = col_in(jj, 1);
                cp16(stage + ((size_t)(buf * 2 + 1) * 32 + jj) * P + v * V,
                     src ? (const void *)(src + wb + v * V) : (const void *)vin, src ? inside : 0);
            }
        }
        if (lane < nv) cp16(lamw + buf * (P + 4) + lane * V, lam_in + wb + lane * V, 16);
        const int hb = wb & ~3;
        const int nh = (wb + nv * V - hb + 3) / 4;
        if (lane < nh) cp16(hw + buf * HP + lane * 4, p.hinfo + hb + lane * 4, 16);
        cp_commit();
    };

    C Gv = C(0), Gw = C(0);
    if (tb < te) stage_tile(tb, 0);
    for (int t = tb; t < te; ++t) {
        const int buf = (t - tb) & 1;
        if (t + 1 < te) {
            stage_tile(t + 1, buf ^ 1);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncwarp();
        const int2 tl = p.tiles[t];
        const int t0 = tl.x, len = tl.y;
        const int wb = t0 & ~(V - 1), off = t0 - wb;
        const int nv = (off + len + V - 1) / V;
        C *lw = lamw + buf * (P + 4);
        uint32_t *hv = hw + buf * HP + (wb - (wb & ~3));
        for (int sl = lane; sl < nv * V; sl += 32) {
            if (sl < off || sl >= off + len) {
                lw[sl] = C(0);
                hv[sl] = kTrash;
            }
        }
        __syncwarp();
        const C *xf_s = stage + ((size_t)(buf * 2 + 0) * 32 + lane) * P;
        const C *xs_s = stage + ((size_t)(buf * 2 + 1) * 32 + lane) * P;
        C *prow = ptile + lane * P;
        uint32_t tie_any = 0;
        // loads of vector 0, then each step loads vector v+1 before storing v
        Vec xf4{}, xs4{};
        uint32_t h4[V];
        C l4[V];
        if (HF) xf4 = *reinterpret_cast<const Vec *>(xf_s);
        if (HS) xs4 = *reinterpret_cast<const Vec *>(xs_s);
#pragma unroll
        for (int k = 0; k < V; ++k) { h4[k] = hv[k]; l4[k] = lw[k]; }
#pragma unroll
        for (int v = 0; v < W; ++v) {
            if (v >= nv) break;
            Vec nf4{}, ns4{};
            uint32_t nh4[V];
            C nl4[V];
            if (v + 1 < W) {
                if (HF) nf4 = *reinterpret_cast<const Vec *>(xf_s + (v + 1) * V);
                if (HS) ns4 = *reinterpret_cast<const Vec *>(xs_s + (v + 1) * V);
#pragma unroll
                for (int k = 0; k < V; ++k) { nh4[k] = hv[(v + 1) * V + k]; nl4[k] = lw[(v + 1) * V + k]; }
            }
            C res[V];
#pragma unroll
            for (int k = 0; k < V; ++k) {
                const uint32_t h = h4[k];
                const C lam = l4[k];
                const int a = h & 63, b = (h >> 6) & 63;
                tie_any |= h;
                if (HF && HS) {
                    const C u = (fco * lam) * CF::get(xf4, k);
                    const C vv = (sco * lam) * CF::get(xs4, k);
                    const C w = u - vv;
                    const C2 ra = R2[a * 32];
                    const C2 rb = K2 == 2 ? R2[b * 32] : C2{C(0), C(0)};
                    res[k] = (K2 == 2 ? w : C(0)) + C(2) * (Gv - ra.x - rb.x);
                    R2[a * 32] = C2{ra.x + vv, ra.y + w};
                    if (K2 == 2) R2[b * 32] = C2{rb.x + vv, rb.y + w};
                    Gv += vv;
                    Gw += w;
                } else if (HS) {
                    const C vv = (sco * lam) * CF::get(xs4, k);
                    const C ra = R1[a * 32];
                    const C rb = K2 == 2 ? R1[b * 32] : C(0);
                    res[k] = (K2 == 2 ? -vv : C(0)) + C(2) * (Gv - ra - rb);
                    R1[a * 32] = ra + vv;
                    if (K2 == 2) R1[b * 32] = rb + vv;
                    Gv += vv;
                } else {
                    const C u = (fco * lam) * CF::get(xf4, k);
                    res[k] = K2 == 2 ? u : C(0);
                    const C ra = R1[a * 32];
                    const C rb = K2 == 2 ? R1[b * 32] : C(0);
                    R1[a * 32] = ra + u;
                    if (K2 == 2) R1[b * 32] = rb + u;
                    Gw += u;
                }
            }
            *reinterpret_cast<Vec *>(prow + v * V) = CF::make(res);
            xf4 = nf4;
            xs4 = ns4;
#pragma unroll
            for (int k = 0; k < V; ++k) { h4[k] = nh4[k]; l4[k] = nl4[k]; }
        }
        // tie groups of the tile: exact equal-strength term (see kernels_fast.cu)
        if (HS && (tie_any & (1u << 12))) {
            for (int i = 0; i < len; ++i) {
                const uint32_t hi = hv[off + i];
                if (!(hi & (1u << 13))) continue;
                const int g0 = i - (int)(hi >> 16);
                for (int q = g0; q <= i; ++q) {
                    const uint32_t hq = hv[off + q];
                    C corr = C(0);
                    for (int r = g0; r <= i; ++r) {
                        if (r == q) continue;
                        const uint32_t hr = hv[off + r];
                        const int qa = hq & 63, qb = (hq >> 6) & 63, ra = hr & 63, rb = (hr >> 6) & 63;
                        bool share = qa == ra;
                        if (K2 == 2) share = share || qa == rb || qb == ra || qb == rb;
                        if (share) continue;
                        const C vr = (sco * lw[off + r]) * xs_s[off + r];
                        corr += r > q ? vr : -vr;
                    }
                    prow[off + q] += corr;
                }
            }
        }
        __syncwarp();
        // partial results out, coalesced; tile edges element-wise
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const int idx = lane + 32 * i, jj = idx / W, v = idx - jj * W;
            if (v >= nv) continue;
            const long long o = col_out(jj);
            if (o < 0) continue;
            const Vec val = *reinterpret_cast<const Vec *>(ptile + jj * P + v * V);
            C *dst = scr + o + wb + v * V;
            if (v * V >= off && v * V + V <= off + len) {
                *reinterpret_cast<Vec *>(dst) = val;
            } else {
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    const int slot = v * V + k;
                    if (slot >= off && slot < off + len) dst[k] = CF::get(val, k);
                }
            }
        }
        __syncwarp();
    }
    sums[(warp * 3 + 0) * 32 + lane] = Gv;
    sums[(warp * 3 + 1) * 32 + lane] = Gw;
    __syncthreads();

    // ---- phase 2: Z_k[card][column] = Pw + 2 Xv_k, into warp k's stage area
    for (int c = warp; c < nc; c += nw) {
        C tot[kMaxWarps], run[kMaxWarps];
#pragma unroll
        for (int k = 0; k < kMaxWarps; ++k) {
            tot[k] = run[k] = C(0);
            if (k < nw) {
                const unsigned char *bk = smem + hdr + (size_t)k * WL.total + WL.r;
                if (HF && HS) {
                    const C2 r2 = reinterpret_cast<const C2 *>(bk)[c * 32 + lane];
                    tot[k] = r2.y;
                    run[k] = r2.x;
                } else if (HS) {
                    run[k] = reinterpret_cast<const C *>(bk)[c * 32 + lane];
                    tot[k] = -run[k];
                } else {
                    tot[k] = reinterpret_cast<const C *>(bk)[c * 32 + lane];
                }
            }
        }
        C pw = C(0);
#pragma unroll
        for (int k = 0; k < kMaxWarps; ++k) pw += tot[k];
        C xv = C(0);
#pragma unroll
        for (int k = 0; k < kMaxWarps; ++k) {
            if (k < nw) {
                C *Zk = reinterpret_cast<C *>(smem + hdr + (size_t)k * WL.total + WL.stage);
                Zk[c * 32 + lane] = pw + C(2) * xv;
                xv += run[k];
            }
        }
    }
    if (warp == 0) {
        C tw = C(0);
        for (int k = 0; k < nw; ++k)
            tw += HF ? sums[(k * 3 + 1) * 32 + lane] : -sums[(k * 3 + 0) * 32 + lane];
        C xg = C(0);
        for (int k = 0; k < nw; ++k) {
            sums[(k * 3 + 2) * 32 + lane] = tw + C(2) * xg;
            xg += sums[(k * 3 + 0) * 32 + lane];
        }
    }
    __syncthreads();

    // ---- phase 3: finish (lane = column): out = lambda_out (part + base - Z[a] - Z[b]).
    // Partial tiles come back by coalesced cp.async (double-buffered, after
    // the Z table in the stage area); results go out through ptile.
    const C *Z = reinterpret_cast<const C *>(mine + WL.stage) + lane;
    C *pbuf = reinterpret_cast<C *>(mine + WL.stage) + (size_t)nc * 32;   // [buf][32][P]
    const C base = sums[(warp * 3 + 2) * 32 + lane];
    auto load_partials = [&](int t, int buf) {
        const int2 tl = p.tiles[t];
        const int wb = tl.x & ~(V - 1), end = tl.x + tl.y;
        const int nv = (end - wb + V - 1) / V;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const int idx = lane + 32 * i, jj = idx / W, v = idx - jj * W;
            if (v >= nv) continue;
            const long long o = col_out(jj);
            // only the tile's own hands: the rest of the vector belongs to
            // neighbouring tiles that may not be written yet
            const int lo = max(0, tl.x - (wb + v * V)), hi = min(V, end - (wb + v * V));
            C *dst = pbuf + ((size_t)buf * 32 + jj) * P + v * V;
            if (o >= 0 && lo == 0 && hi == V) {
                cp16(dst, scr + o + wb + v * V, 16);
            } else {
#pragma unroll
                for (int k = 0; k < V; ++k) dst[k] = (o >= 0 && k >= lo && k < hi) ? scr[o + wb + v * V + k] : C(0);
            }
        }
        if (lane < nv) cp16(lamw + buf * (P + 4) + lane * V, lam_out + wb + lane * V, 16);
        const int hb = wb & ~3;
        const int nh = (wb + nv * V - hb + 3) / 4;
        if (lane < nh) cp16(hw + buf * HP + lane * 4, p.hinfo + hb + lane * 4, 16);
        cp_commit();
    };
    if (tb < te) load_partials(tb, 0);
    for (int t = tb; t < te; ++t) {
        const int buf = (t - tb) & 1;
        if (t + 1 < te) {
            load_partials(t + 1, buf ^ 1);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncwarp();
        const int2 tl = p.tiles[t];
        const int t0 = tl.x, len = tl.y;
        const int wb = t0 & ~(V - 1), off = t0 - wb;
        const int nv = (off + len + V - 1) / V;
        const C *lw = lamw + buf * (P + 4);
        const uint32_t *hv = hw + buf * HP + (wb - (wb & ~3));
        const C *prow_in = pbuf + ((size_t)buf * 32 + lane) * P;
        C *prow = ptile + lane * P;
#pragma unroll
        for (int v = 0; v < W; ++v) {
            if (v >= nv) break;
            const Vec x = *reinterpret_cast<const Vec *>(prow_in + v * V);
            C res[V];
#pragma unroll
            for (int k = 0; k < V; ++k) {
                const int slot = v * V + k;
                const uint32_t h = hv[slot];
                C val = CF::get(x, k) + base - Z[(h & 63) * 32];
                if (K2 == 2) val -= Z[((h >> 6) & 63) * 32];
                res[k] = lw[slot] * val;
            }
            *reinterpret_cast<Vec *>(prow + v * V) = CF::make(res);
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const int idx = lane + 32 * i, jj = idx / W, v = idx - jj * W;
            if (v >= nv) continue;
            const long long o = col_out(jj);
            if (o < 0) continue;
            const Vec val = *reinterpret_cast<const Vec *>(ptile + jj * P + v * V);
            S *dst = vout + o + wb + v * V;
            if (v * V >= off && v * V + V <= off + len) {
                *reinterpret_cast<Vec *>(dst) = val;
            } else {
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    const int slot = v * V + k;
                    if (slot >= off && slot < off + len) dst[k] = CF::get(val, k);
                }
            }
        }
        __syncwarp();
    }
    if (warp == nw - 1 && H + lane < hs) {
        for (int jj = 0; jj < 32; ++jj) {
            const long long o = col_out(jj);
            if (o >= 0) vout[o + H + lane] = S(0);
        }
    }
}

// One tile of 32 output columns (col = ctile * 32 + lane) of game p.
template <typename S, int K2>
__device__ __forceinline__ void vec_tile(const FastParams &p, long long ctile, unsigned char *smem_raw) {
    const int hs = p.hs;
    Col *ci = reinterpret_cast<Col *>(smem_raw);
    S *fco_s = reinterpret_cast<S *>(smem_raw + 32 * sizeof(Col));
    S *sco_s = fco_s + 32;
    S *sums = sco_s + 32;
    int kinds = 0;
    if (threadIdx.x < 32) {
        const long long col = ctile * 32 + threadIdx.x;
        Col c;
        S f = S(0), s = S(0);
        if (col < (long long)p.n_out * p.batch) {
            const int sg = (int)(col / p.batch), b = (int)(col % p.batch);
            const int fc = p.fcol[sg], sc = p.scol[sg];
            c.in_off = (long long)b * p.n_in * hs;
            c.out_off = ((long long)b * p.n_out + sg) * hs;
            c.foff = fc >= 0 ? fc * hs : -1;
            c.soff = sc >= 0 ? sc * hs : -1;
            if (fc >= 0) f = static_cast<const S *>(p.fcoef)[sg];
            if (sc >= 0) s = static_cast<const S *>(p.scoef)[sg];
        } else {
            c.in_off = 0;
            c.out_off = -1;
            c.foff = c.soff = -1;
        }
        ci[threadIdx.x] = c;
        fco_s[threadIdx.x] = f;
        sco_s[threadIdx.x] = s;
        kinds = (c.foff >= 0 ? 1 : 0) | (c.soff >= 0 ? 2 : 0);
    }
    const bool has_f = __syncthreads_or(kinds & 1) != 0;
    const bool has_s = __syncthreads_or(kinds & 2) != 0;
    const Col c0i = ci[0];
    int same = 1, valid = 0;
    if (threadIdx.x < 32) {
        const Col c = ci[threadIdx.x];
        if (c.out_off >= 0) {
            valid = 1;
            same = c.foff == c0i.foff && c.soff == c0i.soff &&
                   c.in_off == c0i.in_off + (long long)threadIdx.x * p.n_in * hs &&
                   c.out_off == c0i.out_off + (long long)threadIdx.x * p.n_out * hs;
        }
    }
    const bool uni = __syncthreads_and(same) != 0;
    const int nvalid = __syncthreads_count(valid);
    if (has_f && has_s) scan_body<S, K2, kKindFS>(p, smem_raw, ci, fco_s, sco_s, sums, uni, nvalid);
    else if (has_s) scan_body<S, K2, kKindS>(p, smem_raw, ci, fco_s, sco_s, sums, uni, nvalid);
    else scan_body<S, K2, kKindF>(p, smem_raw, ci, fco_s, sco_s, sums, uni, nvalid);
    __syncthreads();
}

template <typename S, int K2>
__global__ void __launch_bounds__(32 * kMaxWarps)
vec_scan_kernel(const FastParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    vec_tile<S, K2>(p, blockIdx.x, smem_raw);
}

// Persistent launch over the column tiles of several games.
template <typename S, int K2>
__global__ void __launch_bounds__(32 * kMaxWarps)
vec_multi_kernel(const MultiParams m) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ FastParams sp;
    __shared__ long long s_tile;
    __shared__ int s_game;
    int next = blockIdx.x;
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = m.schedule == 0 ? atomicAdd(m.ticket, 1) : next;
            next += gridDim.x;
            int g = -1;
            if (t < m.total_tiles) {
                g = m.tile_game[t];
                sp = m.games[g];
                sp.vin = static_cast<const S *>(m.vin) + m.in_off[g];
                sp.vout = static_cast<S *>(m.vout) + m.out_off[g];
                sp.scratch = sp.vout;   // partial results pass through the output rows
                s_tile = t - m.tile_start[g];
            }
            s_game = g;
        }
        __syncthreads();
        if (s_game < 0) break;
        vec_tile<S, K2>(sp, s_tile, smem_raw);
    }
}

template <typename S, int K2>
cudaError_t launch_t(const FastParams &p, size_t smem, cudaStream_t stream) {
    auto fn = vec_scan_kernel<S, K2>;
    {
        const cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void *>(fn), smem);
        if (e != cudaSuccess) return e;
    }
    const long long ncols = (long long)p.n_out * p.batch;
    const long long blocks = (ncols + 31) / 32;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    fn<<<(unsigned)blocks, 32 * p.nw, smem, stream>>>(p);
    return cudaGetLastError();
}

template <typename S, int K2>
cudaError_t launch_multi_t(const MultiParams &m, size_t smem, int grid, cudaStream_t stream) {
    auto fn = vec_multi_kernel<S, K2>;
    {
        const cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void *>(fn), smem);
        if (e != cudaSuccess) return e;
    }
    if (m.total_tiles <= 0) return cudaSuccess;
    fn<<<grid, 32 * m.nw, smem, stream>>>(m);
    return cudaGetLastError();
}

template <typename S, int K2>
int ctas_t(size_t smem, int nw) {
    auto fn = vec_multi_kernel<S, K2>;
    // raise the kernel's limit if needed (never lower it: another launch may need more)
    if (ensure_dyn_smem(reinterpret_cast<const void *>(fn), smem) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, 32 * nw, smem) != cudaSuccess) return 0;
    return n;
}

}  // namespace

size_t vec_smem_bytes(int storage, int nc, int nw) {
    const size_t cs = storage == kStoreF64 ? 8 : 4;
    const int P = storage == kStoreF64 ? Cfg<double>::P : Cfg<float>::P;
    return header_bytes(nw, cs) + (size_t)nw * warp_layout(nc, cs, P).total;
}

cudaError_t launch_vec_scan(const FastParams &p, int storage, int k, cudaStream_t stream) {
    if (p.nc > kZPitch - 1) return cudaErrorInvalidValue;
    const size_t smem = vec_smem_bytes(storage, p.nc, p.nw);
    switch (storage) {
        case kStoreF32: return k == 1 ? launch_t<float, 1>(p, smem, stream) : launch_t<float, 2>(p, smem, stream);
        case kStoreF64: return k == 1 ? launch_t<double, 1>(p, smem, stream) : launch_t<double, 2>(p, smem, stream);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_vec_multi(const MultiParams &m, int storage, int k, int grid, cudaStream_t stream) {
    if (m.nc > kZPitch - 1 || m.nw < 1 || m.nw > kMaxWarps || grid < 1) return cudaErrorInvalidValue;
    const size_t smem = vec_smem_bytes(storage, m.nc, m.nw);
    switch (storage) {
        case kStoreF32:
            return k == 1 ? launch_multi_t<float, 1>(m, smem, grid, stream) : launch_multi_t<float, 2>(m, smem, grid, stream);
        case kStoreF64:
            return k == 1 ? launch_multi_t<double, 1>(m, smem, grid, stream) : launch_multi_t<double, 2>(m, smem, grid, stream);
        default: return cudaErrorInvalidValue;
    }
}

int vec_multi_ctas_per_sm(int storage, int k, int nc, int nw) {
    const size_t smem = vec_smem_bytes(storage, nc, nw);
    switch (storage) {
        case kStoreF32: return k == 1 ? ctas_t<float, 1>(smem, nw) : ctas_t<float, 2>(smem, nw);
        case kStoreF64: return k == 1 ? ctas_t<double, 1>(smem, nw) : ctas_t<double, 2>(smem, nw);
        default: return 0;
    }
}

}  // namespace kps
