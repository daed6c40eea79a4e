// Host-side layout builder: template sorting, CTA grouping and the
// bank-aware placement of filters into (round, lane, ring copy) cells.
#include "spiir_layout.h"

#include <algorithm>
#include <functional>
#include <numeric>
#include <queue>

namespace spiir {

namespace {

inline int mod32(int64_t v) { return (int)(((v % 32) + 32) % 32); }

// One (round, lane) cell of a template's warp.
struct Cell {
    int64_t filter = -1;
    int copy = 0;
    int delay = 0;
};

// Place the filters `fl` of one template into F rounds x 32 lanes.  Filter l
// read through ring copy c hits bank (c*CS - d_l) mod 32 at every sample (the
// ring length, history and block length are multiples of 32), and copy c is
// offset by c * (32/C) banks, so filter l can use any of the C banks of its
// class (-d_l) mod (32/C).  A round is conflict-free when its 32 lanes use 32
// different banks.  Each bank can therefore take F filters (one per round):
// the filters of a class are dealt round-robin over the class's C banks,
// filling rounds from 0 upwards.  Filters beyond a class's C*F capacity
// (unavoidable conflicts) are packed into the last rounds, so that as few
// rounds as possible pay a second shared-memory wavefront.  Empty cells
// become padding filters (a = b = 0) whose delay hits a bank unused in their
// round.  Returns the number of overflow filters; *wavefronts gets the summed
// worst-bank load over the rounds.
int place_template(const std::vector<int64_t> &fl, const int32_t *d, int F, int C, int CS,
                   std::vector<Cell> &cells, double *wavefronts)
{
    cells.assign((size_t)F * 32, Cell());
    const int width = 32 / C;                      // number of classes
    std::vector<std::vector<int64_t>> cls(width);
    for (int64_t l : fl) cls[mod32(-(int64_t)d[l]) % width].push_back(l);
    std::vector<int> load((size_t)F * 32, 0);      // filters per (round, bank)
    std::vector<char> lane_used((size_t)F * 32, 0);
    auto copy_for_bank = [&](int bank, int dl) {   // c with (c*CS - dl) mod 32 == bank
        for (int c = 0; c < C; ++c)
            if (mod32((int64_t)c * CS - dl) == bank) return c;
        return 0;
    };
    std::vector<int64_t> overflow;
    for (int r0 = 0; r0 < width; ++r0) {
        const std::vector<int64_t> &v = cls[r0];
        for (size_t i = 0; i < v.size(); ++i) {
            const int round = (int)(i / C);
            if (round >= F) {
                overflow.push_back(v[i]);
                continue;
            }
            const int dl = d[v[i]];
            const int bank = (r0 + (int)(i % C) * width) % 32;
            Cell &cell = cells[(size_t)round * 32 + bank];  // lane = bank
            cell.filter = v[i];
            cell.delay = dl;
            cell.copy = copy_for_bank(bank, dl);
            load[(size_t)round * 32 + bank] += 1;
            lane_used[(size_t)round * 32 + bank] = 1;
        }
    }
    // overflow: last rounds first, least-loaded bank of the filter's class
    for (int64_t l : overflow) {
        const int dl = d[l];
        int best_r = -1, best_bank = -1, best_cost = 1 << 30;
        for (int r = F - 1; r >= 0; --r) {
            int free_lanes = 0;
            int worst = 0;
            for (int i = 0; i < 32; ++i) {
                free_lanes += !lane_used[(size_t)r * 32 + i];
                worst = std::max(worst, load[(size_t)r * 32 + i]);
            }
            if (free_lanes == 0) continue;
            for (int c = 0; c < C; ++c) {
                const int bank = mod32((int64_t)c * CS - dl);
                const int after = load[(size_t)r * 32 + bank] + 1;
                const int cost = std::max(0, after - worst);  // added wavefronts
                if (cost < best_cost) {
                    best_cost = cost;
                    best_r = r;
                    best_bank = bank;
                }
            }
            if (best_cost == 0) break;
        }
        int lane = 0;
        while (lane_used[(size_t)best_r * 32 + lane]) ++lane;
        Cell &cell = cells[(size_t)best_r * 32 + lane];
        cell.filter = l;
        cell.delay = dl;
        cell.copy = copy_for_bank(best_bank, dl);
        load[(size_t)best_r * 32 + best_bank] += 1;
        lane_used[(size_t)best_r * 32 + lane] = 1;
    }
    // padding: every empty lane gets a bank nobody in its round uses
    for (int r = 0; r < F; ++r) {
        for (int lane = 0; lane < 32; ++lane) {
            if (lane_used[(size_t)r * 32 + lane]) continue;
            int bank = 0;
            while (bank < 32 && load[(size_t)r * 32 + bank] > 0) ++bank;
            if (bank == 32) bank = lane;
            load[(size_t)r * 32 + bank] += 1;
            lane_used[(size_t)r * 32 + lane] = 1;
            Cell &cell = cells[(size_t)r * 32 + lane];
            cell.filter = -1;
            cell.copy = 0;
            cell.delay = (32 - bank) % 32;  // (0 - delay) mod 32 == bank
        }
    }
    // wavefronts per round: largest number of distinct addresses in one bank
    double wf = 0.0;
    for (int r = 0; r < F; ++r) {
        int worst = 1;
        for (int bank = 0; bank < 32; ++bank) {
            std::vector<std::pair<int, int>> addr;
            for (int lane = 0; lane < 32; ++lane) {
                const Cell &c = cells[(size_t)r * 32 + lane];
                if (mod32((int64_t)c.copy * CS - c.delay) == bank)
                    addr.emplace_back(c.copy, c.delay);
            }
            std::sort(addr.begin(), addr.end());
            int distinct = (int)(std::unique(addr.begin(), addr.end()) - addr.begin());
            worst = std::max(worst, distinct);
        }
        wf += worst;
    }
    *wavefronts = wf;
    return (int)overflow.size();
}

// Half-warp mode: template A in lanes 0..15, template B in lanes 16..31 of
// F rounds.  Greedy: each filter takes the round with a free lane in its
// half where one of its C banks is unused by the whole warp round (most free
// lanes first); otherwise any free lane in its half (a conflict).  Empty
// cells become padding filters on unused banks.
void place_half(const std::vector<int64_t> &flA, const std::vector<int64_t> &flB,
                const int32_t *d, int F, int C, int CS, std::vector<Cell> &cells,
                double *wavefronts)
{
    cells.assign((size_t)F * 32, Cell());
    std::vector<uint32_t> used(F, 0u);
    std::vector<int> nfree(2 * F, 16);
    const std::vector<int64_t> *lists[2] = {&flA, &flB};
    for (int h = 0; h < 2; ++h) {
        for (int64_t l : *lists[h]) {
            const int dl = d[l];
            int br = -1, bc = -1;
            for (int r = 0; r < F; ++r) {
                if (nfree[2 * r + h] == 0) continue;
                if (br >= 0 && nfree[2 * r + h] <= nfree[2 * br + h]) continue;
                for (int c = 0; c < C; ++c)
                    if (!((used[r] >> mod32((int64_t)c * CS - dl)) & 1u)) {
                        br = r;
                        bc = c;
                        break;
                    }
            }
            if (br < 0) {
                for (int r = 0; r < F; ++r)
                    if (nfree[2 * r + h] > 0 && (br < 0 || nfree[2 * r + h] > nfree[2 * br + h]))
                        br = r;
                bc = 0;
            }
            const int lane = h * 16 + (16 - nfree[2 * br + h]);
            Cell &cell = cells[(size_t)br * 32 + lane];
            cell.filter = l;
            cell.copy = bc;
            cell.delay = dl;
            used[br] |= 1u << mod32((int64_t)bc * CS - dl);
            --nfree[2 * br + h];
        }
    }
    for (int r = 0; r < F; ++r)
        for (int h = 0; h < 2; ++h)
            for (int lane = h * 16 + (16 - nfree[2 * r + h]); lane < h * 16 + 16; ++lane) {
                int bank = 0;
                while (bank < 32 && ((used[r] >> bank) & 1u)) ++bank;
                if (bank == 32) bank = lane;
                used[r] |= 1u << (bank & 31);
                Cell &cell = cells[(size_t)r * 32 + lane];
                cell.filter = -1;
                cell.copy = 0;
                cell.delay = (32 - bank) % 32;
            }
    double wf = 0.0;
    for (int r = 0; r < F; ++r) {
        int worst = 1;
        for (int bank = 0; bank < 32; ++bank) {
            std::vector<std::pair<int, int>> addr;
            for (int lane = 0; lane < 32; ++lane) {
                const Cell &c = cells[(size_t)r * 32 + lane];
                if (mod32((int64_t)c.copy * CS - c.delay) == bank)
                    addr.emplace_back(c.copy, c.delay);
            }
            std::sort(addr.begin(), addr.end());
            worst = std::max(worst, (int)(std::unique(addr.begin(), addr.end()) - addr.begin()));
        }
        wf += worst;
    }
    *wavefronts = wf;
}

// First-fit packing of templates (F filters per lane, nw warps each, in
// the layout's sort order) into CTAs of W warps of one F: the F of every
// CTA in launch order.
std::vector<int> pack_groups(const std::vector<int> &F, const std::vector<int> &nw,
                             const std::vector<int64_t> &order, int W)
{
    std::vector<int> gF, used;
    std::vector<size_t> open;
    int curF = -1;
    for (int64_t t : order) {
        if (F[t] != curF) {
            open.clear();
            curF = F[t];
        }
        size_t gi = gF.size();
        for (size_t k = 0; k < open.size(); ++k)
            if (used[open[k]] + nw[t] <= W) {
                gi = open[k];
                break;
            }
        if (gi == gF.size()) {
            gF.push_back(F[t]);
            used.push_back(0);
            open.push_back(gi);
        }
        used[gi] += nw[t];
        if (used[gi] == W) open.erase(std::find(open.begin(), open.end(), gi));
    }
    return gF;
}

// Predicted length of one launch (filter-round-samples per lane) whose units
// -- every CTA group x every detector, largest F first -- are taken in order
// by `slots` resident CTAs, each unit going to the CTA that frees up first
// (longest-processing-time-first list scheduling).
double predict_launch(const std::vector<int> &gF, int D, int64_t slots)
{
    std::priority_queue<double, std::vector<double>, std::greater<double>> free_at;
    for (int64_t i = 0; i < slots; ++i) free_at.push(0.0);
    double end = 0.0;
    for (int f : gF)
        for (int d = 0; d < D; ++d) {
            const double t = free_at.top() + (double)f + kLaneOverhead;
            free_at.pop();
            free_at.push(t);
            end = std::max(end, t);
        }
    return end;
}

// Templates in launch order: filters per lane, then warps, then filter
// count, then largest delay, each descending (ties keep bank order).
std::vector<int64_t> sort_templates(const std::vector<int> &F, const std::vector<int> &nw,
                                    const std::vector<std::vector<int64_t>> &filters,
                                    const int32_t *d)
{
    std::vector<int32_t> dmax(F.size(), 0);
    for (size_t t = 0; t < F.size(); ++t)
        for (int64_t f : filters[t]) dmax[t] = std::max(dmax[t], d[f]);
    std::vector<int64_t> order(F.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
        if (F[x] != F[y]) return F[x] > F[y];
        if (nw[x] != nw[y]) return nw[x] > nw[y];
        if (filters[x].size() != filters[y].size()) return filters[x].size() > filters[y].size();
        return dmax[x] > dmax[y];
    });
    return order;
}

}  // namespace

bool build_layout(const std::vector<std::vector<int64_t>> &filters, int D, const float *a,
                  const float *b, const int32_t *d, const LayoutOptions &opt, Layout *out,
                  std::string *err)
{
    Layout L;
    L.T = (int64_t)filters.size();
    L.D = D;
    L.Tb = opt.Tb;
    if (L.T < 1 || D < 1) {
        *err = "layout: empty bank";
        return false;
    }
    if (L.Tb < 32 || L.Tb % 32 != 0 || L.Tb > 4096) {
        *err = "layout: block_len must be a multiple of 32 in [32, 4096]";
        return false;
    }
    L.C = opt.C == 0 ? 1 : opt.C;   // the default is settled below, once F is known
    if (L.C != 1 && L.C != 2 && L.C != 4) {
        *err = "layout: ring_copies must be 1, 2 or 4";
        return false;
    }
    L.Fcap = opt.Fcap == 0 ? kMaxF : opt.Fcap;
    if (L.Fcap < 1 || L.Fcap > kMaxF) {
        *err = "layout: max_filters_per_lane must be in [1, " + std::to_string(kMaxF) + "]";
        return false;
    }
    // lanes per template: half warps for small templates (more filters per lane)
    int64_t maxL = 0;
    for (int64_t t = 0; t < L.T; ++t) maxL = std::max<int64_t>(maxL, (int64_t)filters[t].size());
    // (only when the bank is large enough that halving the warp count still
    // leaves >= 16 warps per SM; small banks are latency-bound and need warps).
    // Templates of up to 3 rounds of 32 qualify: at 32 lanes they hold at
    // most 3 filters per lane, and 16 lanes halve the cross-lane sums per
    // filter (measured: 25-75 filters 13% faster at 16 lanes, 100-160
    // filters 4% slower)
    const bool small = (maxL + 31) / 32 <= 3 && (maxL + 15) / 16 <= L.Fcap;
    const bool many = (L.T * D + 1) / 2 >= 16 * (int64_t)opt.n_sm;
    L.G = opt.G != 0 ? opt.G : (small && many ? 16 : 32);
    if (L.G != 16 && L.G != 32) {
        *err = "layout: lanes per template must be 16 or 32";
        return false;
    }
    if (L.G == 16 && (maxL + 15) / 16 > L.Fcap) {
        *err = "layout: half-warp templates hold at most " + std::to_string(16 * L.Fcap) +
               " filters";
        return false;
    }
    // per template: rounds of G filters, warps w, filters per lane F
    int64_t maxd = 0, max_nw = 1, total_warps = 0;
    std::vector<int> F(L.T), nw(L.T);
    for (int64_t t = 0; t < L.T; ++t) {
        const int64_t n = (int64_t)filters[t].size();
        const int64_t rounds = std::max<int64_t>(1, (n + L.G - 1) / L.G);
        const int64_t w = (rounds + L.Fcap - 1) / L.Fcap;
        if (w > 8) {
            *err = "layout: template " + std::to_string(t) + " has " + std::to_string(n) +
                   " filters; with " + std::to_string(L.Fcap) + " filters per lane at most " +
                   std::to_string(32 * L.Fcap * 8) + " fit in a CTA";
            return false;
        }
        nw[t] = (int)w;
        max_nw = std::max<int64_t>(max_nw, w);
        total_warps += w;
        F[t] = (int)((rounds + w - 1) / w);
        for (int64_t l : filters[t]) maxd = std::max<int64_t>(maxd, d[l]);
        L.n_filters += n;
    }
    // warps per CTA: enough CTAs to cover the GPU twice over, at most 4 (more
    // warps per CTA wait longer at the per-block barrier)
    if (opt.W > 0) {
        L.W = opt.W;
    } else {
        const int64_t work = (L.G == 16 ? (total_warps + 1) / 2 : total_warps) * D;
        int w = max_nw > 4 ? 8 : 4;
        while (w > 1 && w / 2 >= max_nw && work / w < 2 * (int64_t)opt.n_sm) w /= 2;
        L.W = w;
    }
    if (L.W < 1 || L.W > 8) {
        *err = "layout: warps_per_cta must be in [1, 8]";
        return false;
    }
    if (max_nw > L.W) {
        *err = "layout: a template needs " + std::to_string(max_nw) + " warps at " +
               std::to_string(L.Fcap) + " filters per lane; warps_per_cta is " +
               std::to_string(L.W);
        return false;
    }
    // ring geometry
    L.H = (int)std::max<int64_t>(1, (maxd + L.Tb - 1) / L.Tb);
    L.S = L.H + 2;
    L.R = L.S * L.Tb;
    L.Dh = L.H * L.Tb;
    auto set_copies = [&L](int C) {
        L.C = C;
        const int skew = C == 1 ? 0 : 32 / C;   // bank offset between copies
        L.CS = L.R + L.Tb + skew;               // R + Tb is a multiple of 32
    };
    set_copies(L.C);
    // default copies: with at most 4 filters per lane the strain reads and
    // the cross-lane sums of a step are few enough that bank conflicts bound
    // the shared-memory pipe, and a second copy (the placement then spreads a
    // round over more banks) pays for its larger ring; full warps only
    // (measured on 2048-template bands: 2 filters per lane 64.8 -> 54.7 ms,
    // 4 per lane 24.9 -> 23.5 ms; 4 copies no faster than 2; half-warp
    // templates and banks of more filters per lane no faster with 2)
    if (opt.C == 0 && L.G == 32) {
        int maxF = 0;
        for (int64_t t = 0; t < L.T; ++t) maxF = std::max(maxF, F[t]);
        if (maxF <= 4) {
            set_copies(2);
            if (L.smem_bytes() > 227 * 1024) set_copies(1);
        }
    }
    if (L.smem_bytes() > 227 * 1024) {
        *err = "layout: strain ring and partial sums need " + std::to_string(L.smem_bytes()) +
               " bytes of shared memory (max delay " + std::to_string(maxd) +
               "); use fewer ring_copies, fewer warps per CTA or a shorter block_len";
        return false;
    }
    // tail split (full-warp templates): the smallest templates, by filter
    // rounds, get twice their warps (F halves), so the units that end the
    // launch are short.  Auto: the share of the bank's rounds, in steps of 1%
    // up to 20%, whose predicted launch (predict_launch on the resident CTAs
    // the kernel's registers and shared memory allow) is shortest.
    if (opt.tail >= 0 && L.G == 32) {
        const int regs = opt.regs > 0 ? opt.regs : 128;
        const int64_t by_regs = 65536 / ((int64_t)regs * 32 * L.W);
        const int64_t by_smem = (int64_t)(228 * 1024) / (L.smem_bytes() + 1024);
        const int64_t slots =
            std::max<int64_t>(1, std::min<int64_t>(std::min(by_regs, by_smem), 32)) * opt.n_sm;
        L.slots_model = slots;
        std::vector<int64_t> rounds_of(L.T);
        int64_t total_rounds = 0;
        for (int64_t t = 0; t < L.T; ++t) {
            rounds_of[t] = std::max<int64_t>(1, ((int64_t)filters[t].size() + 31) / 32);
            total_rounds += rounds_of[t];
        }
        // templates that can take twice their warps (each warp keeps >= 1
        // round), smallest first
        std::vector<int64_t> small;
        for (int64_t t = 0; t < L.T; ++t)
            if (2 * nw[t] <= L.W && rounds_of[t] >= 2 * nw[t]) small.push_back(t);
        std::stable_sort(small.begin(), small.end(), [&](int64_t x, int64_t y) {
            if (rounds_of[x] != rounds_of[y]) return rounds_of[x] < rounds_of[y];
            return filters[x].size() < filters[y].size();
        });
        const int64_t n_small = (int64_t)small.size();
        auto split_first = [&](int64_t k, std::vector<int> &F2, std::vector<int> &nw2) {
            F2 = F;
            nw2 = nw;
            for (int64_t i = 0; i < k; ++i) {
                const int64_t t = small[i];
                nw2[t] = 2 * nw[t];
                F2[t] = (int)((rounds_of[t] + nw2[t] - 1) / nw2[t]);
            }
        };
        std::vector<int64_t> cands;   // split counts to compare
        if (opt.tail > 0) {
            int64_t k = 0, acc = 0;
            while (k < n_small &&
                   1000 * (acc + rounds_of[small[k]]) <= (int64_t)opt.tail * total_rounds)
                acc += rounds_of[small[k++]];
            cands.push_back(k);
        } else {
            int64_t k = 0, acc = 0;
            for (int pct = 0; pct <= 20; ++pct) {
                while (k < n_small &&
                       100 * (acc + rounds_of[small[k]]) <= (int64_t)pct * total_rounds)
                    acc += rounds_of[small[k++]];
                if (cands.empty() || cands.back() != k) cands.push_back(k);
            }
        }
        int64_t best_k = 0;
        double best = 0.0;
        for (int64_t k : cands) {
            std::vector<int> F2, nw2;
            split_first(k, F2, nw2);
            const double len =
                predict_launch(pack_groups(F2, nw2, sort_templates(F2, nw2, filters, d), L.W), D,
                               slots);
            if (k == cands.front() || len < best) {
                best = len;
                best_k = k;
            }
        }
        if (best_k > 0) {
            std::vector<int> F2, nw2;
            split_first(best_k, F2, nw2);
            F.swap(F2);
            nw.swap(nw2);
        }
        L.tail_templates = best_k;
    }
    // sort templates: F descending, warps descending, filter count descending
    std::vector<int64_t> order = sort_templates(F, nw, filters, d);
    // first-fit packing of each template's warps into CTAs of the same F
    struct Group {
        int F;
        int used;
        std::vector<int64_t> tmpl;  // per warp
        std::vector<int> first;     // per warp: first warp of its template
        std::vector<int64_t> tmpl2; // per warp: the second template (half-warp mode)
    };
    std::vector<Group> groups;
    std::vector<size_t> open;       // groups of the current F with free warps
    int curF = -1;
    if (L.G == 16) {
        // two consecutive templates (sorted, so of similar F) per warp, W warps per CTA
        for (size_t i = 0; i < order.size(); i += 2) {
            const int64_t ta = order[i];
            const int64_t tb = i + 1 < order.size() ? order[i + 1] : -1;
            if (groups.empty() || groups.back().used == L.W) {
                groups.push_back(Group{F[ta], 0, std::vector<int64_t>(L.W, -1),
                                       std::vector<int>(L.W, -1),
                                       std::vector<int64_t>(L.W, -1)});
            }
            Group &grp = groups.back();
            grp.tmpl[grp.used] = ta;
            grp.tmpl2[grp.used] = tb;
            grp.first[grp.used] = grp.used;
            grp.used += 1;
        }
        order.clear();
    }
    for (int64_t t : order) {
        if (F[t] != curF) {
            open.clear();
            curF = F[t];
        }
        size_t gi = groups.size();
        for (size_t k = 0; k < open.size(); ++k)
            if (groups[open[k]].used + nw[t] <= L.W) {
                gi = open[k];
                break;
            }
        if (gi == groups.size()) {
            groups.push_back(Group{F[t], 0, std::vector<int64_t>(L.W, -1),
                                   std::vector<int>(L.W, -1), std::vector<int64_t>(L.W, -1)});
            open.push_back(gi);
        }
        Group &grp = groups[gi];
        for (int k = 0; k < nw[t]; ++k) {
            grp.tmpl[grp.used + k] = t;
            grp.first[grp.used + k] = grp.used;
        }
        grp.used += nw[t];
        if (grp.used == L.W) open.erase(std::find(open.begin(), open.end(), gi));
    }
    const int64_t G = (int64_t)groups.size();
    L.group_F.resize(G);
    L.group_pbase.resize(G);
    L.warp_info.assign((size_t)G * L.W * 4, 0);
    int64_t base = 0;
    for (int64_t g = 0; g < G; ++g) {
        L.group_F[g] = groups[g].F;
        L.group_pbase[g] = base;
        base += (int64_t)groups[g].F * L.W * 32;
        for (int w = 0; w < L.W; ++w) {
            const int64_t t = groups[g].tmpl[w];
            int32_t *wi = &L.warp_info[(g * L.W + w) * 4];
            wi[0] = (int32_t)t;
            wi[1] = t >= 0 ? groups[g].first[w] : w;
            wi[2] = t >= 0 ? nw[t] : 1;
            wi[3] = (int32_t)groups[g].tmpl2[w];
        }
    }
    L.n_slots = base;
    L.maxF = *std::max_element(L.group_F.begin(), L.group_F.end());
    L.params.assign((size_t)L.n_slots * 4, 0.f);
    L.ringoff.assign((size_t)L.n_slots * 2, 0);
    L.slot_filter.assign((size_t)L.n_slots, -1);
    L.slot_template.assign((size_t)L.n_slots, -1);
    double wf_total = 0.0;
    int64_t rounds_total = 0;
    std::vector<Cell> cells;
    static const std::vector<int64_t> none;
    for (int64_t g = 0; g < G; ++g) {
        const int Fg = L.group_F[g];
        for (int w = 0; w < L.W; ++w) {
            const int64_t t = groups[g].tmpl[w];
            if (t >= 0 && groups[g].first[w] != w) continue;  // placed with its first warp
            const int nwt = t >= 0 ? nw[t] : 1;
            const int rounds = Fg * nwt;   // the template's rounds over its warps
            const std::vector<int64_t> &fl = t >= 0 ? filters[t] : none;
            const int64_t t2 = groups[g].tmpl2[w];
            double wf = 0.0;
            if (L.G == 16)
                place_half(fl, t2 >= 0 ? filters[t2] : none, d, rounds, L.C, L.CS, cells, &wf);
            else
                place_template(fl, d, rounds, L.C, L.CS, cells, &wf);
            if (t >= 0) {
                wf_total += wf;
                rounds_total += rounds;
            }
            for (int r = 0; r < rounds; ++r) {
                const int ww = w + r / Fg, rl = r % Fg;  // warp and its local round
                for (int i = 0; i < 32; ++i) {
                    const Cell &c = cells[(size_t)r * 32 + i];
                    const int64_t s = L.slot(g, rl, ww, i);
                    float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
                    if (c.filter >= 0) {
                        ar = a[2 * c.filter];
                        ai = a[2 * c.filter + 1];
                        br = b[2 * c.filter];
                        bi = b[2 * c.filter + 1];
                    }
                    if (i & 1) {  // (im, re) order: pole conj(a), gain (Im b, Re b)
                        ai = -ai;
                        std::swap(br, bi);
                    }
                    L.params[4 * s + 0] = ar;
                    L.params[4 * s + 1] = ai;
                    L.params[4 * s + 2] = br;
                    L.params[4 * s + 3] = bi;
                    L.ringoff[2 * s + 0] = L.Dh - c.delay;  // window start at block 0
                    L.ringoff[2 * s + 1] = c.copy * L.CS;   // copy base word
                    L.slot_filter[s] = c.filter;
                    L.slot_template[s] = (L.G == 16 && i >= 16) ? t2 : t;
                }
            }
        }
    }
    L.conflict_ratio = rounds_total ? wf_total / (double)rounds_total : 1.0;
    // work units: groups in sorted (largest-first) order, detectors inner
    L.units.resize((size_t)G * D * 2);
    for (int64_t g = 0; g < G; ++g)
        for (int det = 0; det < D; ++det) {
            L.units[2 * (g * D + det)] = (int32_t)g;
            L.units[2 * (g * D + det) + 1] = det;
        }
    *out = std::move(L);
    return true;
}

}  // namespace spiir
