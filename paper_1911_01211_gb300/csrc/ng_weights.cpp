// Exact-rational generation of the integration weights (host side of libng).
//
// Reading of the Gregory weights: for n <= k the starting weights s_{n,j} = I_{0,n,j};
// for n > k the classical Gregory rule, i.e. the trapezoidal rule plus end corrections
// made of forward differences at the left end and backward differences at the right end up
// to order k, with the Gregory coefficients G_i defined by t/ln(1+t) = sum_i G_i t^i.
// This reproduces the paper's Table tab:gregory (the BDF construction in its prose does not).
#include "ng_weights.h"

#include <cstdlib>
#include <cstring>

namespace {

typedef __int128 i128;

i128 iabs(i128 x) { return x < 0 ? -x : x; }
i128 gcd128(i128 a, i128 b) {
    a = iabs(a);
    b = iabs(b);
    while (b) { i128 t = a % b; a = b; b = t; }
    return a;
}

struct Q {  // exact rational p/q, q > 0, reduced
    i128 p, q;
    Q(i128 a = 0, i128 b = 1) : p(a), q(b) { norm(); }
    void norm() {
        if (q < 0) { p = -p; q = -q; }
        i128 g = gcd128(p, q);
        if (g > 1) { p /= g; q /= g; }
        if (p == 0) q = 1;
    }
    double d() const { return (double)((long double)p / (long double)q); }
};
Q operator+(Q a, Q b) { return Q(a.p * b.q + b.p * a.q, a.q * b.q); }
Q operator-(Q a, Q b) { return Q(a.p * b.q - b.p * a.q, a.q * b.q); }
Q operator*(Q a, Q b) {
    i128 g1 = gcd128(a.p, b.q), g2 = gcd128(b.p, a.q);
    if (g1 == 0) g1 = 1;
    if (g2 == 0) g2 = 1;
    return Q((a.p / g1) * (b.p / g2), (a.q / g2) * (b.q / g1));
}
Q operator/(Q a, Q b) { return a * Q(b.q, b.p); }
Q qpow(i128 base, int e) {
    i128 r = 1;
    for (int i = 0; i < e; ++i) r *= base;
    return Q(r);
}
i128 binom(int n, int r) {
    i128 c = 1;
    for (int i = 1; i <= r; ++i) c = c * (n - r + i) / i;
    return c;
}
i128 fact(int n) {
    i128 f = 1;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

// P = M^{-1}, M_{ja} = j^a (j, a = 0..k), Gauss-Jordan over Q.
void vandermonde_inverse(int k, Q P[NG_KMAX + 1][NG_KMAX + 1]) {
    int n = k + 1;
    Q A[NG_KMAX + 1][2 * (NG_KMAX + 1)];
    for (int j = 0; j < n; ++j)
        for (int a = 0; a < 2 * n; ++a)
            A[j][a] = a < n ? qpow(j, a) : Q(a - n == j ? 1 : 0);
    for (int c = 0; c < n; ++c) {
        int piv = c;
        while (A[piv][c].p == 0) ++piv;
        if (piv != c)
            for (int a = 0; a < 2 * n; ++a) { Q t = A[c][a]; A[c][a] = A[piv][a]; A[piv][a] = t; }
        Q inv = Q(1) / A[c][c];
        for (int a = 0; a < 2 * n; ++a) A[c][a] = A[c][a] * inv;
        for (int r = 0; r < n; ++r) {
            if (r == c || A[r][c].p == 0) continue;
            Q f = A[r][c];
            for (int a = 0; a < 2 * n; ++a) A[r][a] = A[r][a] - f * A[c][a];
        }
    }
    for (int a = 0; a < n; ++a)
        for (int l = 0; l < n; ++l) P[a][l] = A[a][n + l];
}

}  // namespace

int ng_make_weights(int k, NgWeights *W) {
    if (k < 1 || k > NG_KMAX || !W) return 1;
    std::memset(W, 0, sizeof(*W));
    W->k = k;
    Q P[NG_KMAX + 1][NG_KMAX + 1];
    vandermonde_inverse(k, P);
    // D_{m,l} = sum_{a>=1} P_{a,l} a m^{a-1}
    Q D[NG_KMAX + 1][NG_KMAX + 1];
    for (int m = 0; m <= k; ++m)
        for (int l = 0; l <= k; ++l) {
            Q s(0);
            for (int a = 1; a <= k; ++a) s = s + P[a][l] * Q(a) * qpow(m, a - 1);
            D[m][l] = s;
            W->D[m][l] = s.d();
        }
    for (int j = 0; j <= k; ++j) W->a[j] = (Q(0) - D[0][j]).d();
    // I_{m,n,l} = sum_a P_{a,l} (n^{a+1} - m^{a+1})/(a+1)
    Q Iq[NG_KMAX + 1][NG_KMAX + 1][NG_KMAX + 1];
    for (int m = 0; m <= k; ++m)
        for (int n = 0; n <= k; ++n)
            for (int l = 0; l <= k; ++l) {
                Q s(0);
                for (int a = 0; a <= k; ++a) s = s + P[a][l] * (qpow(n, a + 1) - qpow(m, a + 1)) / Q(a + 1);
                Iq[m][n][l] = s;
                W->I[m][n][l] = s.d();
            }
    // Gregory coefficients G_0..G_{k+1}: reciprocal of the series ln(1+t)/t = sum (-1)^i t^i/(i+1)
    Q c[NG_KMAX + 3], G[NG_KMAX + 3];
    for (int i = 0; i <= k + 1; ++i) c[i] = Q(i % 2 ? -1 : 1, i + 1);
    G[0] = Q(1);
    for (int i = 1; i <= k + 1; ++i) {
        Q s(0);
        for (int j = 1; j <= i; ++j) s = s + c[j] * G[i - j];
        G[i] = Q(0) - s;
    }
    // rows n = 0..2k+1
    for (int n = 0; n <= 2 * k + 1; ++n) {
        Q w[2 * NG_KMAX + 2];
        if (n <= k) {
            for (int j = 0; j <= k; ++j) w[j] = Iq[0][n][j];
        } else {
            for (int j = 0; j <= n; ++j) w[j] = Q(1);
            for (int i = 1; i <= k + 1; ++i) {
                int p = i - 1;
                Q g = G[i].p < 0 ? Q(0) - G[i] : G[i];
                for (int q = 0; q <= p; ++q) {
                    // backward difference nabla^p y_n = sum_q (-1)^q C(p,q) y_{n-q}
                    w[n - q] = w[n - q] - g * Q(((q % 2) ? -1 : 1) * binom(p, q));
                    // (-1)^p forward difference Delta^p y_0 = (-1)^p sum_q (-1)^{p-q} C(p,q) y_q
                    w[q] = w[q] - g * Q((((p + (p - q)) % 2) ? -1 : 1) * binom(p, q));
                }
            }
        }
        int len = n <= k ? k + 1 : n + 1;
        for (int j = 0; j < len; ++j) W->greg[n][j] = w[j].d();
        if (n == 2 * k + 1)
            for (int j = 0; j <= k; ++j) W->omega[j] = w[j].d();
    }
    // R_{m;r,s} = sum_{a,b} P_{a,r} P_{b,s} m^{a+b+1} a! b!/(a+b+1)!
    for (int m = 0; m <= k; ++m)
        for (int r = 0; r <= k; ++r)
            for (int s = 0; s <= k; ++s) {
                Q acc(0);
                for (int a = 0; a <= k; ++a)
                    for (int b = 0; b <= k; ++b)
                        acc = acc + P[a][r] * P[b][s] * qpow(m, a + b + 1) * Q(fact(a) * fact(b), fact(a + b + 1));
                W->R[m][r][s] = acc.d();
            }
    // extrapolation: interpolant through y_{n-k..n} evaluated one step beyond
    for (int l = 0; l <= k; ++l) {
        Q s(0);
        for (int a = 0; a <= k; ++a) s = s + qpow(k + 1, a) * P[a][k - l];
        W->C[l] = s.d();
    }
    return 0;
}
