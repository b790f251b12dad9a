// Host-side check of the compact float sin/cos of the float KPP flux
// (cgl::kpp_sincos) against float64 sin and cos: the maximum absolute error
// over a dense sweep of [-200, 200] and of the KPP range [pi/4, 3.5 pi], and
// the wide-argument fallback.  Prints one JSON line.
#include <cmath>
#include <cstdio>

#include "../../paper_2509_04673_gb300/csrc/common.cuh"

int main() {
    double worst = 0.0, worst_kpp = 0.0;
    long n = 0;
    for (long i = 0; i <= 4000000; ++i) {
        const float x = (float)(-200.0 + 400.0 * (double)i / 4000000.0);
        float s, c;
        cgl::kpp_sincos(x, s, c);
        const double es = std::fabs((double)s - std::sin((double)x)), ec = std::fabs((double)c - std::cos((double)x));
        const double e = es > ec ? es : ec;
        if (e > worst) worst = e;
        if (x >= 0.78f && x <= 11.0f && e > worst_kpp) worst_kpp = e;
        ++n;
    }
    double worst_wide = 0.0;
    for (int i = 0; i < 1000; ++i) {
        const float x = 4096.f + 37.3f * i;
        float s, c;
        cgl::kpp_sincos(x, s, c);
        const double e = std::fmax(std::fabs((double)s - std::sin((double)x)), std::fabs((double)c - std::cos((double)x)));
        if (e > worst_wide) worst_wide = e;
    }
    std::printf("{\"points\": %ld, \"max_abs_err\": %.3e, \"max_abs_err_kpp_range\": %.3e, \"max_abs_err_wide\": %.3e}\n",
                n, worst, worst_kpp, worst_wide);
    return 0;
}
