// Host-side plan arithmetic: pyramid level sizes, per-level feature quotas,
// bilinear source-coordinate tables and the exact fraction for Harris k.
// Compiled with -ffp-contract=off: every float64 step below is one IEEE
// operation, so the tables are identical on every host.
#include <math.h>
#include <stdint.h>

#include "of_plan.h"

namespace ofh {

// Level l has scale s_l = scale^l, a float64 running product starting at 1;
// w_l = floor(W / s_l + 0.5), h_l likewise (Sec. 1; Sec. 6.1 "decrease exponentially").
void level_sizes(int W, int H, int levels, float scale, int32_t* ws, int32_t* hs, double* ls) {
    double s = 1.0;
    for (int l = 0; l < levels; ++l) {
        ws[l] = (l == 0) ? W : (int32_t)floor((double)W / s + 0.5);
        hs[l] = (l == 0) ? H : (int32_t)floor((double)H / s + 0.5);
        if (ls) ls[l] = s;
        s = s * (double)scale;
    }
}

// Quota of level l for N features: proportional to level area, ratio
// f = 1/scale^2 per level: round(N (1-f)/(1-f^L) f^l), capped by what is left;
// the last level takes the remainder.
void level_quotas(int N, int L, float scale, int32_t* q) {
    const double sc = (double)scale;
    const double f = 1.0 / (sc * sc);
    double fpow = 1.0;
    for (int l = 0; l < L; ++l) fpow = fpow * f;
    const double share = (1.0 - f) / (1.0 - fpow);
    int left = N;
    double fl = 1.0;
    for (int l = 0; l < L; ++l) {
        int n;
        if (l + 1 == L) {
            n = left;
        } else {
            n = (int)floor((double)N * share * fl + 0.5);
            if (n > left) n = left;
        }
        q[l] = n;
        left -= n;
        fl = fl * f;
    }
}

// Source sample of each of n_dst destination pixels for a centre-aligned
// bilinear resize from n_src pixels: s = (d + 0.5) * (n_src / n_dst) - 0.5,
// clamped to [0, n_src - 1]; entry = (floor(s) << 12) | lrint(frac(s) * 2048).
void resize_table(int n_src, int n_dst, int32_t* tab) {
    const double ratio = (double)n_src / (double)n_dst;
    const double last = (double)(n_src - 1);
    for (int d = 0; d < n_dst; ++d) {
        double s = ((double)d + 0.5) * ratio - 0.5;
        s = s < 0.0 ? 0.0 : (s > last ? last : s);
        const double i0 = floor(s);
        const int32_t a = (int32_t)lrint((s - i0) * 2048.0);
        tab[d] = ((int32_t)i0 << 12) | a;
    }
}

// Harris k rounded to a multiple of 1e-6 and reduced to num/den.  The integer
// key den*det - num*trace^2 fits int64 for 7x7 windows when 0 <= k <= 0.25
// and den <= 3000; anything else is rejected.
bool k_fraction(float k, int64_t* num, int64_t* den) {
    const double kd = (double)k;
    if (!(kd >= 0.0 && kd <= 0.25)) return false;
    int64_t n = (int64_t)llrint(kd * 1000000.0), d = 1000000;
    int64_t a = n, b = d;
    while (b != 0) {
        const int64_t r = a % b;
        a = b;
        b = r;
    }
    if (a == 0) a = d;
    n /= a;
    d /= a;
    if (d > 3000) return false;
    *num = n;
    *den = d;
    return true;
}

float response_scale(int64_t den) {
    const double f = 1.0 / (4.0 * 7.0 * 255.0);
    return (float)((f * f * f * f) / (double)den);
}

}  // namespace ofh

extern "C" int of_plan_levels(int W, int H, int levels, float scale, int n_features, int32_t* ws,
                              int32_t* hs, int32_t* quota) {
    if (W <= 0 || H <= 0 || levels < 1 || levels > 64 || !(scale > 1.0f) || n_features < 0 ||
        !ws || !hs || !quota)
        return -1;
    ofh::level_sizes(W, H, levels, scale, ws, hs, nullptr);
    ofh::level_quotas(n_features, levels, scale, quota);
    return 0;
}
