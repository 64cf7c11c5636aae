// Integration weights of the k-th order scheme, FP64 copies of exact rationals.
// Sec. "Basic integration and differentiation rules" of the NESSi paper:
//   P = M^-1 with M_ja = j^a (Eq. integrator_P), D (Eq. integrator_D), I (Eq. integrator_I),
//   BDF a_j = -D_{0,j} (Eq. integrator_bd), Gregory w_{n,j} (Eq. integrator_greg),
//   boundary convolution R_{m;r,s} (Eq. integrator_R), extrapolation C_l (Eq. polyextrap).
#pragma once

#define NG_KMAX 5

struct NgWeights {
    int k;
    double a[NG_KMAX + 1];                            // BDF a_0..a_k
    double D[NG_KMAX + 1][NG_KMAX + 1];               // D[m][l]
    double I[NG_KMAX + 1][NG_KMAX + 1][NG_KMAX + 1];  // I[m][n][l] = int_m^n of basis l
    double greg[2 * NG_KMAX + 2][2 * NG_KMAX + 2];    // w_{n,j} for n = 0..2k+1
    double omega[NG_KMAX + 1];                        // end weights for n >= 2k+1
    double R[NG_KMAX + 1][NG_KMAX + 1][NG_KMAX + 1];  // R[m][r][s], m = 0..k
    double C[NG_KMAX + 1];                            // y_{n+1} = sum_l C_l y_{n-l}
};

// Fill W for order k (1..NG_KMAX). Returns 0 on success.
int ng_make_weights(int k, NgWeights *W);
