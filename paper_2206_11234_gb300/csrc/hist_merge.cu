// fpt_hist_merge: the weighted histograms of disjoint sets of runs (several
// GPUs, or several calls over split id ranges) combined into the histogram of
// their union, in binary64 on the host.
//
// Each bin of §2.1 Eq. (9) / §2.2 Eq. (16) is kept with max-shifted sums
// (fpt_bin): s1 = sum e^(x), s2 = sum e^(2x), l_k = sum x^k with
// x = ln w - max_lw.  Moving a part whose maximum is m_p to the common maximum
// M = max_p m_p shifts its x by d_p = m_p - M <= 0, so
//   s1 -> e^(d_p) s1,  s2 -> e^(2 d_p) s2,
//   l_k -> sum_i C(k, i) d_p^(k-i) l_i   (l_0 = count),
// and the merged bin is the sum over parts.  Parts whose bin is empty
// (max_lw = -inf) contribute nothing.
#include <cmath>

#include "abi_internal.h"
#include "fpt.h"

using namespace fpt;

extern "C" int fpt_hist_merge(const fpt_bin* parts, int32_t n_parts, int64_t n_bins,
                              const fpt_hist_counts* part_counts, fpt_bin* out, fpt_hist_counts* out_counts) {
    if (n_parts < 1 || n_bins < 0) return fail(FPT_EINVAL, "n_parts %d < 1 or n_bins < 0", n_parts);
    if (n_bins > 0 && (!parts || !out)) return fail(FPT_EINVAL, "bins pointer is NULL");
    if (out_counts && !part_counts) return fail(FPT_EINVAL, "out_counts needs part_counts");
    for (int64_t j = 0; j < n_bins; ++j) {
        double M = -INFINITY;
        for (int p = 0; p < n_parts; ++p) {
            const fpt_bin& b = parts[(int64_t)p * n_bins + j];
            if (std::isnan(b.max_lw)) return fail(FPT_EINVAL, "bin %lld of part %d has max_lw NaN", (long long)j, p);
            if (b.count < 0) return fail(FPT_EINVAL, "bin %lld of part %d has a negative count", (long long)j, p);
            if (b.max_lw > M) M = b.max_lw;
        }
        fpt_bin o{};
        o.max_lw = M;
        for (int p = 0; p < n_parts; ++p) {
            const fpt_bin& b = parts[(int64_t)p * n_bins + j];
            o.count += b.count;
            if (!(b.max_lw > -INFINITY)) continue;  // empty in this part
            const double d = b.max_lw - M;          // <= 0
            const double e = std::exp(d);
            o.s1 += e * b.s1;
            o.s2 += e * e * b.s2;
            const double L[5] = {(double)b.count, b.l1, b.l2, b.l3, b.l4};
            // sum over the part of (x + d)^k, expanded binomially
            const double d2 = d * d, d3 = d2 * d, d4 = d3 * d;
            o.l1 += L[1] + d * L[0];
            o.l2 += L[2] + 2.0 * d * L[1] + d2 * L[0];
            o.l3 += L[3] + 3.0 * d * L[2] + 3.0 * d2 * L[1] + d3 * L[0];
            o.l4 += L[4] + 4.0 * d * L[3] + 6.0 * d2 * L[2] + 4.0 * d3 * L[1] + d4 * L[0];
        }
        out[j] = o;
    }
    if (out_counts) {
        fpt_hist_counts c{};
        for (int p = 0; p < n_parts; ++p) {
            c.under += part_counts[p].under;
            c.over += part_counts[p].over;
            c.censored += part_counts[p].censored;
            c.total += part_counts[p].total;
        }
        *out_counts = c;
    }
    return FPT_OK;
}
