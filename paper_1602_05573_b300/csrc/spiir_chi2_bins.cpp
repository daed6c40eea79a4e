// Chi^2 bins of a SPIIR bank (spiir_chi2_split): host code, no device work.
//
// Allen's discriminator (the review's chi^2 section) cuts a template into p
// frequency bins that each carry an equal share of the template's power and
// compares the SNR each bin collects with that share.  A SPIIR template is
// already a sum over frequency -- one single-pole filter per stretch of the
// chirp, its frequency the pole's argument -- so a bin here is a contiguous
// run of a template's filters in order of arg(a_l), and a filter's power is
// the energy of its impulse response, sum_{k>=0} |b_l a_l^k|^2 =
// |b_l|^2 / (1 - |a_l|^2).  Filter l joins the bin holding the midpoint of
// its share of the template's cumulative energy.  Each bin then runs as a
// template of its own, so spiir_filter on the regrouped bank writes the bin
// series that spiir_chi2_peak reads.
#include "spiir.h"
#include "spiir_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <string>
#include <vector>

using spiir::detail::fail;
using spiir::detail::validate_bank;

extern "C" spiir_status spiir_chi2_split(const spiir_bank_desc *bank, int32_t n_bins,
                                         int64_t *group_off, int64_t *filter_of, float *a_out,
                                         float *b_out, int32_t *delay_out)
{
    spiir_status st = validate_bank(bank);
    if (st != SPIIR_OK) return st;
    if (bank->n_bands > 1)
        return fail(SPIIR_EUNSUPPORTED, "chi^2 bins of a multirate bank are not built");
    if (n_bins < 1 || n_bins > 64) return fail(SPIIR_EINVAL, "n_bins must be in [1, 64]");
    if (!group_off || !filter_of) return fail(SPIIR_EINVAL, "group_off and filter_of are required");
    const int64_t T = bank->n_templates;
    const int64_t *off = bank->filter_off;
    const float *a = bank->a_reim, *b = bank->b_reim;
    std::vector<int64_t> order;
    std::vector<double> angle, energy;
    std::vector<int32_t> bin;
    int64_t at = 0;                  // next position of the regrouped bank
    group_off[0] = 0;
    for (int64_t t = 0; t < T; ++t) {
        const int64_t l0 = off[t], n = off[t + 1] - off[t];
        order.resize((size_t)n);
        angle.resize((size_t)n);
        energy.resize((size_t)n);
        bin.assign((size_t)n, 0);
        for (int64_t i = 0; i < n; ++i) {
            const double ar = a[2 * (l0 + i)], ai = a[2 * (l0 + i) + 1];
            const double br = b[2 * (l0 + i)], bi = b[2 * (l0 + i) + 1];
            angle[(size_t)i] = std::atan2(ai, ar);
            energy[(size_t)i] = (br * br + bi * bi) / (1.0 - (ar * ar + ai * ai));
        }
        // frequency order (equal arguments keep bank order)
        std::iota(order.begin(), order.end(), (int64_t)0);
        std::stable_sort(order.begin(), order.end(),
                         [&](int64_t x, int64_t y) { return angle[(size_t)x] < angle[(size_t)y]; });
        double total = 0.0;
        for (int64_t i = 0; i < n; ++i) total += energy[(size_t)order[(size_t)i]];
        double cum = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            const double e = energy[(size_t)order[(size_t)i]];
            cum += e;
            const double mid = (cum - 0.5 * e) / total;
            // total > 0 unless every gain is zero; then everything is bin 0
            const int64_t k = total > 0.0 ? (int64_t)(mid * n_bins) : 0;
            bin[(size_t)i] = (int32_t)std::min<int64_t>(std::max<int64_t>(k, 0), n_bins - 1);
        }
        // bins of the template in turn, each in frequency order
        for (int32_t g = 0; g < n_bins; ++g) {
            for (int64_t i = 0; i < n; ++i) {
                if (bin[(size_t)i] != g) continue;
                const int64_t l = l0 + order[(size_t)i];
                filter_of[at] = l;
                if (a_out) {
                    a_out[2 * at] = a[2 * l];
                    a_out[2 * at + 1] = a[2 * l + 1];
                }
                if (b_out) {
                    b_out[2 * at] = b[2 * l];
                    b_out[2 * at + 1] = b[2 * l + 1];
                }
                if (delay_out) delay_out[at] = bank->delay[l];
                ++at;
            }
            group_off[t * n_bins + g + 1] = at;
        }
    }
    return SPIIR_OK;
}
