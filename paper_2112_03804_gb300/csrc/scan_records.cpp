// Host-side builder of the per-box hand records of the staged scan kernels
// (layout in scan_records.h).
#include "scan_records.h"

#include <algorithm>
#include <cstring>

namespace kps {

std::string build_scan_records(const HostGame &h, const double *lam_in, const double *lam_out, int max_extra,
                               ScanRecords *out) {
    ScanRecords &R = *out;
    if (h.k != 1 && h.k != 2) return "cards per hand";
    const int nc = h.ncards + 1;
    if (nc > 64) return "too many cards";
    const int H = h.H, hs = h.hs;
    const int nbox = (hs + kTmaBox - 1) / kTmaBox;
    // tie groups: at most 4 hands (partners within 3 positions)
    for (int i = 0; i < H; ++i)
        if (h.group_hi[i] - h.group_lo[i] > 3) return "tie group longer than 4 hands";
    // chunk boundaries at box boundaries that cut no tie group, as close to
    // an even split as possible
    auto clean = [&](int bx) { return bx <= 0 || bx >= nbox || 16 * bx >= H || h.group_lo[16 * bx] == 16 * bx; };
    R.bchunk[0] = 0;
    R.bchunk[kTmaWarps] = nbox;
    for (int k = 1; k < kTmaWarps; ++k) {
        const int ideal = (int)((long long)nbox * k / kTmaWarps);
        int best = -1;
        for (int d = 0; d <= 4 && best < 0; ++d) {
            for (int s : {ideal - d, ideal + d})
                if (best < 0 && s >= R.bchunk[k - 1] && s <= nbox && clean(s)) best = s;
        }
        if (best < 0) return "no chunk boundary free of tie groups";
        R.bchunk[k] = best;
    }
    int extra = 0;
    for (int k = 0; k < kTmaWarps; ++k) {
        const int n = R.bchunk[k + 1] - R.bchunk[k];
        if (n < 0) return "chunk order";
        extra = std::max(extra, n - 16);
    }
    if (extra > max_extra) return "chunk longer than tensor memory and its shared-memory overflow";
    R.H = H;
    R.hs = hs;
    R.nc = nc;
    R.k = h.k;
    R.nbox = nbox;
    R.extra = extra;
    // records: scan blocks, then finishing records
    const size_t scan_bytes = (size_t)nbox * kScanBlock, fin_bytes = (size_t)nbox * 8 * sizeof(TmaFinRec);
    R.bytes.assign(scan_bytes + fin_bytes, 0);
    auto card = [&](int hand, int j) { return h.hand_slots[2 * hand + j]; };
    auto off = [&](int hand, int j) -> uint32_t {
        // padding hands use the spare card row (their weights are zero)
        if (hand >= H || j >= h.k) return (uint32_t)h.ncards * 128u;
        return (uint32_t)card(hand, j) * 128u;
    };
    auto share = [&](int x, int y) {   // any card of hand y in hand x
        for (int j = 0; j < h.k; ++j)
            for (int l = 0; l < h.k; ++l)
                if (card(x, j) == card(y, l)) return true;
        return false;
    };
    for (int bx = 0; bx < nbox; ++bx) {
        unsigned char *blk = R.bytes.data() + (size_t)bx * kScanBlock;
        TmaFinRec *fin = reinterpret_cast<TmaFinRec *>(R.bytes.data() + scan_bytes) + 8 * bx;
        uint32_t tw[2] = {0u, 0u};
        for (int k = 0; k < 8; ++k) {
            const int i = 16 * bx + 2 * k;
            TmaScanRec r{};
            r.oa1 = off(i, 0);
            r.ob1 = off(i, 1);
            r.oa2 = off(i + 1, 0);
            r.ob2 = off(i + 1, 1);
            r.lin1 = i < H ? (float)lam_in[i] : 0.f;
            r.lin2 = i + 1 < H ? (float)lam_in[i + 1] : 0.f;
            if (i + 1 < H)
                for (int l = 0; l < h.k; ++l) {
                    if (card(i + 1, 0) == card(i, l)) r.ma = 1.f;
                    if (h.k == 2 && card(i + 1, 1) == card(i, l)) r.mb = 1.f;
                }
            std::memcpy(blk + 32 * k, &r, sizeof(r));
            TmaFinRec f{};
            f.oa1 = r.oa1;
            f.ob1 = r.ob1;
            f.oa2 = r.oa2;
            f.ob2 = r.ob2;
            f.lout1 = i < H ? (float)lam_out[i] : 0.f;
            f.lout2 = i + 1 < H ? (float)lam_out[i + 1] : 0.f;
            fin[k] = f;
            uint32_t bits = 0;
            for (int e = 0; e < 2; ++e) {
                const int hi = i + e;
                if (hi >= H) continue;
                for (int d = 1; d <= 3; ++d) {
                    const int q = hi - d;
                    if (q < h.group_lo[hi]) break;
                    if (share(hi, q)) continue;
                    bits |= 1u << (e ? 4 + d : 1 + d);
                }
            }
            tw[k / 4] |= bits << (8 * (k & 3));
        }
        std::memcpy(blk + 256, tw, sizeof(tw));
    }
    return "";
}

}  // namespace kps
