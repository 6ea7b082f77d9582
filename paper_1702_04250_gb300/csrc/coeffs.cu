// Host-side constants of the order-P charge assignment (Sec. 3.1: the
// stencil coefficients are a product of three 1-D polynomials of order S).
//
// The order-P assignment function is the centred cardinal B-spline
//   M_P(s) = 1/(P-1)! * sum_{j=0..P} (-1)^j C(P,j) (s + P/2 - j)_+^{P-1}.
// On each unit piece only a fixed set of the truncated powers is active, so
// the weight of stencil point k as a polynomial in delta = n - u is an exact
// rational with denominator 2^(P-1) (P-1)!.  We build its numerators in
// 64-bit integers and divide once, so every coefficient is correctly rounded.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "pppm_common.cuh"

namespace pppm {

namespace {

int64_t binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

__int128 ipow128(int64_t b, int e) {
    __int128 r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

}  // namespace

void stencil_polynomials(int P, double coef[MAXP][MAXP], double dcoef[MAXP][MAXP]) {
    for (int k = 0; k < MAXP; ++k)
        for (int l = 0; l < MAXP; ++l) coef[k][l] = dcoef[k][l] = 0.0;
    const int rlo = (P - 1) / 2;
    int64_t fact = 1;
    for (int i = 2; i <= P - 1; ++i) fact *= i;
    const double den = (double)((int64_t)1 << (P - 1)) * (double)fact;
    for (int k = 0; k < P; ++k) {
        // Work in half units: 2 * (s + P/2 - j) with s = k - rlo + delta.
        // The piece's midpoint delta_mid is 0 (odd P) or -1/2 (even P); a
        // truncated power is active on the whole piece iff it is positive at
        // the midpoint (it is never zero there).
        const int two_mid = 2 * (k - rlo) + ((P & 1) ? 0 : -1);
        int64_t num[MAXP] = {0};
        for (int j = 0; j <= P; ++j) {
            const int two_at_mid = two_mid + P - 2 * j;
            if (two_at_mid <= 0) continue;
            const int64_t two_a = 2 * (k - rlo) + P - 2 * j;  // 2 * (k - rlo + P/2 - j)
            const int64_t sgn = (j & 1) ? -1 : 1;
            // (a + delta)^(P-1) = sum_l C(P-1,l) a^(P-1-l) delta^l, a = two_a / 2;
            // scaled by 2^(P-1): sum_l C(P-1,l) two_a^(P-1-l) 2^l delta^l.
            for (int l = 0; l <= P - 1; ++l) {
                __int128 t = (__int128)sgn * binom(P, j) * binom(P - 1, l) *
                             ipow128(two_a, P - 1 - l) * ((int64_t)1 << l);
                num[l] += (int64_t)t;
            }
        }
        for (int l = 0; l < P; ++l) {
            coef[k][l] = (double)num[l] / den;
            if (l >= 1) dcoef[k][l - 1] = (double)(num[l] * l) / den;
        }
    }
}

double stencil_weight_max(int P, const double coef[MAXP][MAXP]) {
    // W_k on its piece: delta in [-1/2, 1/2] (odd P) or [-1, 0] (even P),
    // sampled on 4,096 steps (the maxima, at the piece's middle or ends, are
    // samples), with a 1e-4 relative margin
    const double lo = (P & 1) ? -0.5 : -1.0;
    double m = 0.0;
    for (int k = 0; k < P; ++k)
        for (int i = 0; i <= 4096; ++i) {
            const double d = lo + i / 4096.0;
            double w = coef[k][P - 1];
            for (int l = P - 2; l >= 0; --l) w = w * d + coef[k][l];
            m = std::max(m, std::fabs(w));
        }
    return m * (1.0 + 1e-4);
}

void spline2p_at_integers(int P, double out[MAXP + 1]) {
    // M_{2P}(g) = 1/(2P-1)! sum_j (-1)^j C(2P,j) (g + P - j)_+^(2P-1)
    const int Q = 2 * P;
    __int128 fact = 1;
    for (int i = 2; i <= Q - 1; ++i) fact *= i;
    for (int g = 0; g <= MAXP; ++g) {
        __int128 acc = 0;
        for (int j = 0; j <= Q; ++j) {
            const int64_t b = g + P - j;
            if (b <= 0) continue;
            __int128 t = ipow128(b, Q - 1) * binom(Q, j);
            acc += (j & 1) ? -t : t;
        }
        out[g] = (g <= P) ? (double)acc / (double)fact : 0.0;
    }
}

double grid_kappa(int m, int M) {
    const int mp = (2 * m < M) ? m : m - M;  // Nyquist (2m == M) -> -M/2
    return 2.0 * M_PI * (double)mp / (double)M;
}

static double u1(double kappa, int m, int P) {
    // sinc^P((kappa + 2 pi m)/2), using sin(kappa/2 + pi m) = (-1)^m sin(kappa/2)
    const double x = 0.5 * kappa + M_PI * (double)m;
    if (x == 0.0) return 1.0;
    const double s = ((m & 1) ? -1.0 : 1.0) * std::sin(0.5 * kappa) / x;
    double r = 1.0;
    for (int i = 0; i < P; ++i) r *= s;
    return r;
}

double alias_cross(double kappa, int n, int P, int mmax) {
    double acc = 0.0;
    for (int m = -mmax; m <= mmax; ++m) acc += u1(kappa, m, P) * u1(kappa, m - n, P);
    return acc;
}

}  // namespace pppm
