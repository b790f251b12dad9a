// Host-side check of the float32 certificate of the Appendix-A positivity
// factor (cgl::euler_alpha_is_one): whenever it returns true, the float64
// formula (cgl::euler_alpha<double>) on the corresponding float64 inputs must
// return exactly 1.  Inputs: admissible Euler states over many scales,
// random element contributions, and contributions rescaled onto the edge of
// each constraint (relative offsets down to 1e-12) so that near-ties occur.
// Prints one JSON line: {"trials", "certified", "wrong", "near", "near_certified"}.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>

#include "../../paper_2509_04673_gb300/csrc/common.cuh"

static uint64_t s_state = 0x2509046731ULL;
static uint64_t next_u64() {
    uint64_t z = (s_state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static double unif() { return (next_u64() >> 11) * 0x1p-53; }
static double logu(double lo, double hi) { return std::exp(std::log(lo) + (std::log(hi) - std::log(lo)) * unif()); }

int main(int argc, char** argv) {
    long trials = argc > 1 ? std::atol(argv[1]) : 1000000;
    const double eps = 1e-10;
    const float ome = (float)(1.0 - eps);
    long certified = 0, wrong = 0, near = 0, near_cert = 0;
    for (long t = 0; t < trials; ++t) {
        // admissible state with density and pressure over many decades
        double rho = logu(1e-8, 1e3), pr = rho * logu(1e-12, 1e4);
        double vx = (unif() - 0.5) * logu(1e-3, 1e2), vy = (unif() - 0.5) * logu(1e-3, 1e2);
        double ub[4] = {rho, rho * vx, rho * vy, pr / 0.4 + 0.5 * rho * (vx * vx + vy * vy)};
        double m = logu(1e-9, 1e-1);
        if (t % 3 == 1) m = (0.25 * 0.0625) * ((double)(float)logu(1.0, 50.0) * 16.0);  // facet form 0.25 h (s / h)
        double scale = m * logu(1e-4, 10.0);
        if (t % 5 == 2) scale = m * logu(1e-22, 1e-12);  // rounding noise of a quiescent state
        double f[4];
        for (int c = 0; c < 4; ++c) f[c] = (unif() - 0.5) * scale * (c == 3 ? ub[3] : (c == 0 ? rho : std::fabs(ub[c]) + rho));
        double fd[4];
        float ff[4], ubf[4];
        for (int c = 0; c < 4; ++c) ubf[c] = (float)ub[c];
        bool is_near = false;
        if (t % 2 == 1) {
            // move f onto a constraint boundary: scale by the exact factor, offset
            double a = cgl::euler_alpha<double>(ub, f, m, eps);
            if (a < 1.0 && a > 0.0) {
                double off = std::pow(10.0, -(double)(next_u64() % 13)) * ((next_u64() & 1) ? 1.0 : -1.0);
                if (next_u64() % 4 == 0) off = 0.0;
                for (int c = 0; c < 4; ++c) f[c] *= a * (1.0 + off);
                is_near = true;
            }
        }
        for (int c = 0; c < 4; ++c) {
            ff[c] = (float)f[c];
            fd[c] = (double)ff[c];
        }
        const bool cert = cgl::euler_alpha_is_one(ubf, ff, (float)m, ome);
        const double a64 = cgl::euler_alpha<double>(ub, fd, m, eps);
        if (cert) {
            ++certified;
            if (a64 != 1.0) {
                ++wrong;
                if (wrong < 5)
                    std::fprintf(stderr, "wrong: ub %.17g %.17g %.17g %.17g f %.9g %.9g %.9g %.9g m %.17g a %.17g\n",
                                 ub[0], ub[1], ub[2], ub[3], ff[0], ff[1], ff[2], ff[3], m, a64);
            }
        }
        if (is_near) {
            ++near;
            if (cert) ++near_cert;
        }
    }
    std::printf("{\"trials\": %ld, \"certified\": %ld, \"wrong\": %ld, \"near\": %ld, \"near_certified\": %ld}\n",
                trials, certified, wrong, near, near_cert);
    return wrong == 0 ? 0 : 1;
}
