// Host-side grouping of the visiting order (see layout.h).
#include "layout.h"

#include <algorithm>
#include <atomic>
#include <thread>
#include <utility>

namespace s3 {

static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void seeded_order(uint64_t seed, int64_t n, std::vector<int64_t>& order) {
    std::vector<std::pair<uint64_t, int64_t>> kv((size_t)n);
    for (int64_t k = 0; k < n; ++k)
        kv[(size_t)k] = {mix64(seed + 0x9E3779B97F4A7C15ull * ((63ull << 40) + (uint64_t)k + 1)), k};
    std::sort(kv.begin(), kv.end());
    order.resize((size_t)n);
    for (int64_t k = 0; k < n; ++k) order[(size_t)k] = kv[(size_t)k].second;
}

namespace {

struct SegOut {
    std::vector<int32_t> row, start, cnt;
};

// worker: groups [g0, g1)
void sort_groups(const HostInput& in, HostGrouping& G, int64_t g0, int64_t g1,
                 std::vector<SegOut>& segs, std::vector<std::vector<int64_t>>& nseg_per_group,
                 std::vector<std::vector<int64_t>>& nlong_per_group,
                 std::vector<std::vector<int64_t>>& nhuge_per_group) {
    const int N = in.N, M = in.M, nF = N + M;
    std::vector<std::pair<int32_t, int32_t>> ev;
    SegOut tmp;
    for (int64_t g = g0; g < g1; ++g) {
        const int64_t t0 = G.t_off[(size_t)g], t1 = G.t_off[(size_t)g + 1];
        for (int F = 0; F < nF; ++F) {
            ev.clear();
            // local event ids: tensor entries first, then coupled matrices in order
            int32_t k = 0;
            std::vector<std::pair<int, int64_t>> ranges;  // (m or -1, base) per block
            if (F < N) {
                for (int64_t e = t0; e < t1; ++e) ev.push_back({G.tidx[F][(size_t)e], k++});
                for (int m = 0; m < M; ++m) {
                    if (in.cmode[m] != F) continue;
                    const int64_t c0 = G.c_off[m][(size_t)g], c1 = G.c_off[m][(size_t)g + 1];
                    for (int64_t e = c0; e < c1; ++e) ev.push_back({G.cr[m][(size_t)e], k++});
                }
            } else {
                const int m = F - N;
                const int64_t c0 = G.c_off[m][(size_t)g], c1 = G.c_off[m][(size_t)g + 1];
                for (int64_t e = c0; e < c1; ++e) ev.push_back({G.cc[m][(size_t)e], k++});
            }
            std::sort(ev.begin(), ev.end());
            // assign positions
            int32_t nseg = 0;
            const size_t nev = ev.size();
            for (size_t p = 0; p < nev;) {
                size_t q = p;
                while (q < nev && ev[q].first == ev[p].first) ++q;
                segs[(size_t)F].row.push_back(ev[p].first);
                segs[(size_t)F].start.push_back((int32_t)p);
                segs[(size_t)F].cnt.push_back((int32_t)(q - p));
                for (size_t r = p; r < q; ++r) {
                    const int32_t id = ev[r].second;
                    const int32_t pos = G.pos_kind == POS_SLOT ? (int32_t)r : nseg;
                    // map the local id back to its array
                    int32_t rem = id;
                    if (F < N) {
                        const int64_t nt = t1 - t0;
                        if (rem < nt) { G.tpos[F][(size_t)(t0 + rem)] = pos; continue; }
                        rem -= (int32_t)nt;
                        for (int m = 0; m < M; ++m) {
                            if (in.cmode[m] != F) continue;
                            const int64_t c0 = G.c_off[m][(size_t)g], c1 = G.c_off[m][(size_t)g + 1];
                            if (rem < c1 - c0) { G.cpos_u[m][(size_t)(c0 + rem)] = pos; break; }
                            rem -= (int32_t)(c1 - c0);
                        }
                    } else {
                        const int m = F - N;
                        G.cpos_v[m][(size_t)(G.c_off[m][(size_t)g] + rem)] = pos;
                    }
                }
                ++nseg;
                p = q;
            }
            nseg_per_group[(size_t)F][(size_t)(g - g0)] = nseg;
            // huge, then long segments to the front (slot positions do not depend on the
            // order of segments)
            int64_t nlong = 0, nhuge = 0;
            if (G.pos_kind == POS_SLOT && G.long_thr > 0) {
                SegOut& so = segs[(size_t)F];
                const size_t s0 = so.row.size() - (size_t)nseg;
                tmp.row.assign(so.row.begin() + (std::ptrdiff_t)s0, so.row.end());
                tmp.start.assign(so.start.begin() + (std::ptrdiff_t)s0, so.start.end());
                tmp.cnt.assign(so.cnt.begin() + (std::ptrdiff_t)s0, so.cnt.end());
                auto cls = [&](int32_t cnt) {
                    return (G.huge_thr > 0 && cnt > G.huge_thr) ? 2 : cnt > G.long_thr ? 1 : 0;
                };
                size_t w = s0;
                for (int want = 2; want >= 0; --want)
                    for (size_t i = 0; i < tmp.row.size(); ++i) {
                        const int k = cls(tmp.cnt[i]);
                        if (k != want) continue;
                        so.row[w] = tmp.row[i];
                        so.start[w] = tmp.start[i];
                        so.cnt[w] = tmp.cnt[i];
                        ++w;
                        nlong += k >= 1;
                        nhuge += k == 2;
                    }
            }
            nhuge_per_group[(size_t)F][(size_t)(g - g0)] = nhuge;
            nlong_per_group[(size_t)F][(size_t)(g - g0)] = nlong;
        }
    }
}

}  // namespace

std::string build_grouping(const HostInput& in, const int64_t* order, int64_t n_union, int rule,
                           int64_t size, int pos_kind, HostGrouping& G, int long_thr,
                           int huge_thr) {
    const int N = in.N, M = in.M, nF = N + M;
    G = HostGrouping();
    G.pos_kind = pos_kind;
    G.long_thr = long_thr;
    G.huge_thr = huge_thr;
    G.nF = nF;
    if (size <= 0) return "group size must be positive";
    // item -> (matrix, local index)
    int64_t cbase[9];
    cbase[0] = in.nnz;
    for (int m = 0; m < M; ++m) cbase[m + 1] = cbase[m] + in.ynnz[m];
    auto item_at = [&](int64_t p) { return order ? order[p] : p; };
    // group boundaries in order positions
    std::vector<int64_t> gpos{0};
    if (rule == RULE_UNION) {
        for (int64_t p = size; p < n_union; p += size) gpos.push_back(p);
    } else {
        int64_t nt = 0;
        for (int64_t p = 0; p < n_union; ++p) {
            if (item_at(p) < in.nnz) {
                if (nt == size) { gpos.push_back(p); nt = 0; }
                ++nt;
            }
        }
    }
    gpos.push_back(n_union);
    const int64_t ng = (int64_t)gpos.size() - 1;
    G.ngroups = ng;
    // counts per group
    G.t_off.assign((size_t)ng + 1, 0);
    for (int m = 0; m < M; ++m) G.c_off[m].assign((size_t)ng + 1, 0);
    for (int64_t g = 0; g < ng; ++g) {
        int64_t nt = 0, nc[8] = {};
        for (int64_t p = gpos[(size_t)g]; p < gpos[(size_t)g + 1]; ++p) {
            const int64_t it = item_at(p);
            if (it < in.nnz) ++nt;
            else
                for (int m = 0; m < M; ++m)
                    if (it < cbase[m + 1]) { ++nc[m]; break; }
        }
        G.t_off[(size_t)g + 1] = G.t_off[(size_t)g] + nt;
        G.max_t = std::max(G.max_t, nt);
        for (int m = 0; m < M; ++m) {
            G.c_off[m][(size_t)g + 1] = G.c_off[m][(size_t)g] + nc[m];
            G.max_c[m] = std::max(G.max_c[m], nc[m]);
        }
    }
    // fill the grouped arrays
    const int64_t nt_all = G.t_off[(size_t)ng];
    for (int n = 0; n < N; ++n) {
        G.tidx[n].resize((size_t)nt_all);
        G.tpos[n].resize((size_t)nt_all);
    }
    G.tval.resize((size_t)nt_all);
    G.t_src.resize((size_t)nt_all);
    for (int m = 0; m < M; ++m) {
        const size_t nc = (size_t)G.c_off[m][(size_t)ng];
        G.cr[m].resize(nc);
        G.cc[m].resize(nc);
        G.cval[m].resize(nc);
        G.cpos_u[m].resize(nc);
        G.cpos_v[m].resize(nc);
        G.c_src[m].resize(nc);
    }
    {
        int64_t tw = 0, cw[8] = {};
        for (int64_t p = 0; p < n_union; ++p) {
            const int64_t it = item_at(p);
            if (it < in.nnz) {
                for (int n = 0; n < N; ++n) G.tidx[n][(size_t)tw] = in.idx[n][it];
                G.tval[(size_t)tw] = in.val[it];
                G.t_src[(size_t)tw] = it;
                ++tw;
            } else {
                for (int m = 0; m < M; ++m) {
                    if (it >= cbase[m + 1]) continue;
                    const int64_t b = it - cbase[m];
                    const size_t w = (size_t)cw[m]++;
                    G.cr[m][w] = in.yr[m][b];
                    G.cc[m][w] = in.yc[m][b];
                    G.cval[m][w] = in.yv[m] ? in.yv[m][b] : 1.0f;
                    G.c_src[m][w] = b;
                    break;
                }
            }
        }
    }
    // sort every group's events into segments, in parallel over blocks of groups
    unsigned nthr = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    const int64_t nblk = std::min<int64_t>(ng, (int64_t)nthr * 8);
    std::vector<int64_t> bpos((size_t)nblk + 1);
    for (int64_t b = 0; b <= nblk; ++b) bpos[(size_t)b] = ng * b / nblk;
    std::vector<std::vector<SegOut>> segs((size_t)nblk, std::vector<SegOut>((size_t)nF));
    std::vector<std::vector<std::vector<int64_t>>> nsg((size_t)nblk), nlg((size_t)nblk), nhg((size_t)nblk);
    std::atomic<int64_t> next{0};
    auto worker = [&]() {
        for (;;) {
            const int64_t b = next.fetch_add(1);
            if (b >= nblk) break;
            nsg[(size_t)b].assign((size_t)nF, std::vector<int64_t>((size_t)(bpos[(size_t)b + 1] - bpos[(size_t)b])));
            nlg[(size_t)b] = nsg[(size_t)b];
            nhg[(size_t)b] = nsg[(size_t)b];
            sort_groups(in, G, bpos[(size_t)b], bpos[(size_t)b + 1], segs[(size_t)b], nsg[(size_t)b],
                        nlg[(size_t)b], nhg[(size_t)b]);
        }
    };
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nthr; ++t) th.emplace_back(worker);
    for (auto& t : th) t.join();
    // concatenate segments in group order
    for (int F = 0; F < nF; ++F) {
        G.seg_off[F].assign((size_t)ng + 1, 0);
        G.slot_off[F].assign((size_t)ng + 1, 0);
        G.seg_nlong[F].assign((size_t)ng, 0);
        G.seg_nhuge[F].assign((size_t)ng, 0);
        size_t total = 0;
        for (int64_t b = 0; b < nblk; ++b) total += segs[(size_t)b][(size_t)F].row.size();
        G.seg_row[F].reserve(total);
        G.seg_start[F].reserve(total);
        G.seg_cnt[F].reserve(total);
        for (int64_t b = 0; b < nblk; ++b) {
            SegOut& s = segs[(size_t)b][(size_t)F];
            G.seg_row[F].insert(G.seg_row[F].end(), s.row.begin(), s.row.end());
            G.seg_start[F].insert(G.seg_start[F].end(), s.start.begin(), s.start.end());
            G.seg_cnt[F].insert(G.seg_cnt[F].end(), s.cnt.begin(), s.cnt.end());
            for (int64_t g = bpos[(size_t)b]; g < bpos[(size_t)b + 1]; ++g) {
                const int64_t ns = nsg[(size_t)b][(size_t)F][(size_t)(g - bpos[(size_t)b])];
                G.seg_off[F][(size_t)g + 1] = G.seg_off[F][(size_t)g] + ns;
                G.seg_nlong[F][(size_t)g] = (int32_t)nlg[(size_t)b][(size_t)F][(size_t)(g - bpos[(size_t)b])];
                G.seg_nhuge[F][(size_t)g] = (int32_t)nhg[(size_t)b][(size_t)F][(size_t)(g - bpos[(size_t)b])];
                G.max_seg[F] = std::max(G.max_seg[F], ns);
            }
        }
        // events per group of this factor
        for (int64_t g = 0; g < ng; ++g) {
            int64_t ne = 0;
            if (F < N) {
                ne = G.t_off[(size_t)g + 1] - G.t_off[(size_t)g];
                for (int m = 0; m < M; ++m)
                    if (in.cmode[m] == F) ne += G.c_off[m][(size_t)g + 1] - G.c_off[m][(size_t)g];
            } else {
                const int m = F - N;
                ne = G.c_off[m][(size_t)g + 1] - G.c_off[m][(size_t)g];
            }
            G.slot_off[F][(size_t)g + 1] = G.slot_off[F][(size_t)g] + ne;
            G.max_ev[F] = std::max(G.max_ev[F], ne);
        }
    }
    return std::string();
}

}  // namespace s3
