// Host-side layout of a SPIIR bank for the filter kernels.
//
// The paper's GPU design (section "GPU accelerated SPIIR method", subsection
// "Optimized GPU implementation of SPIIR") packs each template's parameter
// array "aligned and continuous" for coalesced loads, maps a template with
// more than 32 filters to more threads than a warp and a smaller one to a
// warp, and lets the filters of a template share the staged strain window.
// This layout keeps those ideas and re-plans them for sm_103a:
//  * a template of L filters is served by w warps of one CTA: lane i of each
//    warp holds the filters of "rounds" r = 0..F-1 (state in registers),
//    with F <= Fcap filters per lane, w = ceil(ceil(L/32) / Fcap) and
//    F = ceil(ceil(L/32) / w).  A small Fcap keeps registers per thread low
//    (more resident warps); the warps' partial sums meet in shared memory;
//  * templates are sorted by F and packed into CTAs of W warps (all warps of
//    a template in one CTA), so a CTA's warps do equal work and the CTAs run
//    largest-first;
//  * the strain window is one shared-memory ring per CTA; each filter reads
//    x[k - d_l] from it.  Lanes of one round read 32 different delays, so the
//    filters are placed in rounds (and in one of C bank-skewed copies of the
//    ring) such that the 32 reads of a round hit 32 different banks;
//  * odd lanes store their filter in the (im, re) order (pole conj(a),
//    gain (Im b, Re b)), which turns the first level of the cross-lane sum
//    into a plain exchange with no lane-dependent select.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace spiir {

constexpr int kMaxF = 10;   // largest filters-per-lane cap the plain kernel is built for
constexpr int kTS = 8;      // samples per register sub-block (cross-lane sum width)

struct LayoutOptions {
    int W = 0;          // warps per CTA; 0 = from the bank size
    int Fcap = 0;       // filters per lane cap (1..kMaxF); 0 = default (kMaxF)
    int G = 0;          // lanes per template: 32, or 16 (two templates per warp);
                        // 0 = 16 when every template fits 3 rounds of 32 (and 16 x
                        // Fcap) and the bank still fills >= 16 warps per SM at 16
    int Tb = 512;       // samples per staged strain block (multiple of 32)
    int C = 0;          // ring copies (1, 2, 4); 0 = default (1)
    int n_sm = 148;     // used to pick W when W == 0
    // tail split: the smallest templates run on twice their warps, so the
    // last units of a launch are short.  -1 = off, 0 = auto (the split with
    // the shortest predicted launch, see predict_launch), k > 0 = the
    // smallest templates holding k per mille of the bank's filter rounds
    int tail = -1;
    int regs = 0;       // registers per thread of the filter kernel (0: 128)
};

// Filter-round-samples of per-warp work that one step costs beyond its
// filters' recurrences (the lane's filter sum, the cross-lane
// transpose-reduce, the strain address updates), in units of one filter's
// recurrence: a unit of F filters per lane costs about F + this per sample.
constexpr double kLaneOverhead = 1.75;

// One bank (or one band of a multirate bank) as the kernels see it.
struct Layout {
    int64_t T = 0;          // templates
    int D = 1;              // detectors
    int W = 8, Tb = 256, C = 4;
    int H = 1;              // history blocks: Dh = H * Tb >= max delay
    int S = 3;              // ring slots (blocks) = H + 2
    int R = 0;              // ring length in samples = S * Tb
    int CS = 0;             // words between ring copies (>= R + Tb, bank-skewed)
    int Dh = 0;             // history samples kept = H * Tb
    int maxF = 1;           // largest F of any CTA (<= Fcap)
    int Fcap = 4;
    int G = 32;             // lanes per template (16: a warp serves two templates)
    int64_t n_slots = 0;    // filter slots including padding (per detector)
    int64_t n_filters = 0;  // real filters in this layout

    std::vector<int32_t> group_F;       // [G]
    std::vector<int64_t> group_pbase;   // [G] first slot of the group
    std::vector<int32_t> warp_info;     // [G * W][4] (template or -1, first warp of the
                                        //  template, its warp count, second template
                                        //  of a half-warp pair or -1)
    std::vector<float> params;          // [n_slots][4] kernel-form (ar, ai, br, bi)
    std::vector<int32_t> ringoff;       // [n_slots][2] (pos0, copy base word)
    std::vector<int64_t> slot_filter;   // [n_slots] bank filter index, -1 = padding
    std::vector<int64_t> slot_template; // [n_slots]
    std::vector<int32_t> units;         // [n_units][2] (group, detector)
    double conflict_ratio = 1.0;        // mean wavefronts per round of strain loads
    int64_t tail_templates = 0;         // templates the tail split gave twice their warps
    int64_t slots_model = 0;            // resident CTAs the split's launch model assumed

    int64_t n_groups() const { return (int64_t)group_F.size(); }
    int64_t n_units() const { return (int64_t)units.size() / 2; }
    // mbarriers, C ring copies, and two Tb-sample partial-sum buffers per
    // template slot (two per warp in half-warp mode)
    int smem_bytes() const { return 128 + C * CS * 4 + 2 * W * (32 / G) * Tb * 8; }
    // slot of (group g, round r, warp w, lane i)
    int64_t slot(int64_t g, int r, int w, int i) const {
        return group_pbase[g] + ((int64_t)r * W + w) * 32 + i;
    }
};

// filters[t] lists the bank filter indices of template t served by this
// layout; a, b are complex64 (re, im) arrays of the whole bank, d its delays.
bool build_layout(const std::vector<std::vector<int64_t>> &filters, int D,
                  const float *a, const float *b, const int32_t *d,
                  const LayoutOptions &opt, Layout *out, std::string *err);

}  // namespace spiir
