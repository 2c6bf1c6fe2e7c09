// Twiddle-factor vectors of Section 4.2: Omega^i = [w_{n_i}^0, w_{n_i}^-1, ..., w_{n_i}^-(n_i-1)],
// w_n = exp(2 pi i / n).  Evaluated in FP64 and rounded once to FP32.
//
// The angle is reduced to an octant first, so cos/sin are only ever evaluated on [0, pi/4]
// and points a multiple of n/8 apart (n a power of two) come out with the exact symmetry of
// the unit circle: w^0 = 1, w^(n/4) = -i, w^(n/2) = -1 are exact; for every n, w^-j and
// w^-(n-j) are exact conjugates.  The library's twiddles are the only place cos/sin are called.
#include <cmath>
#include <cstdint>

#include "swdft_internal.h"

namespace swdft {

// (re, im) of exp(-2 pi i j / n), any n >= 1 (powers of two and of three are used).
static void omega_pow(int64_t n, int64_t j, double *re, double *im) {
    const double kQuarterPi = 0.78539816339744830961566084581988;
    j %= n;
    if (j < 0) j += n;
    // 8 j = oct * n + rem, 0 <= rem < n: angle = (oct + rem / n) * pi / 4
    const int64_t oct = (8 * j) / n;
    const int64_t rem = (8 * j) % n;
    const double th = kQuarterPi * (double)rem / (double)n;               // in [0, pi/4)
    const double thc = kQuarterPi * (double)(n - rem) / (double)n;        // pi/4 - th
    double c, s;  // cos and sin of the full angle 2 pi j / n
    switch (oct) {
        case 0: c = std::cos(th);   s = std::sin(th);   break;
        case 1: c = std::sin(thc);  s = std::cos(thc);  break;
        case 2: c = -std::sin(th);  s = std::cos(th);   break;
        case 3: c = -std::cos(thc); s = std::sin(thc);  break;
        case 4: c = -std::cos(th);  s = -std::sin(th);  break;
        case 5: c = -std::sin(thc); s = -std::cos(thc); break;
        case 6: c = std::sin(th);   s = -std::cos(th);  break;
        default: c = std::cos(thc); s = -std::sin(thc); break;
    }
    *re = c;
    *im = -s;
}

void make_omega(int n, float2 *out) {
    for (int j = 0; j < n; ++j) {
        double re, im;
        omega_pow(n, j, &re, &im);
        out[j] = make_float2((float)re, (float)im);
    }
}

}  // namespace swdft
