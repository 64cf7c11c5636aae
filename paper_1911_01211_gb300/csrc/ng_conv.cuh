// Contour convolution C = A * f * B, one time slice at a time (Sec. "Numerical details:
// convolution integrals on C", Eqs. cm1, cm2, cr1, ctv1-ctv3, cles1-cles3; Sec.
// "Implementation: convolution", Table tab:convolution).
//
// A and B are hermitian pairs (X, Xcc) with Xcc = X^ddagger supplying the values outside the
// stored triangles (Eq. hermconjg); f is a single-time function (identity when absent).
// Slice n >= 0 of C: C^R(n, m) for m <= n, C^tv(n, m) for every tau_m, C^<(m, n) for
// m <= n; slice -1: C^M(tau_m).  For n <= k the start-up quadratures read slices 0..k of A
// and B.  One thread per (output element, orbital row a, column block, problem), problem index
// fastest; the thread accumulates its part of row a of the d x d result, streaming the factors'
// elements.
#pragma once

#include "ng_common.cuh"

// One factor of a product term: element e of a component array, read as stored or as its
// hermitian conjugate.
struct XRef {
    const cplx* p;
    int ldk;
    int64_t e;
    bool dag;
};

template <int D>
__device__ __forceinline__ cplx xat(const XRef& r, int x, int y, int kb) {
    const int64_t kk = r.ldk == 1 ? 0 : kb;
    if (!r.dag) return r.p[(r.e * (D * D) + x * D + y) * r.ldk + kk];
    return cconj(r.p[(r.e * (D * D) + y * D + x) * r.ldk + kk]);
}

__device__ __forceinline__ XRef xref(const Comp& c, int64_t e, bool dag) { return XRef{c.p, c.ldk, e, dag}; }

// X^R(n, j); for j > n the modified retarded continuation -[Xcc^R(j, n)]^dagger (Eq. Cretmod)
__device__ __forceinline__ XRef r_retx(const HermV& X, const HermV& Xcc, int n, int j, double& s) {
    if (j <= n) return xref(X.ret, tri(n) + j, false);
    s = -s;
    return xref(Xcc.ret, tri(j) + n, true);
}
// X^<(j, n); for j > n from the conjugate, -[Xcc^<(n, j)]^dagger (Eq. hermconjg_gtrless)
__device__ __forceinline__ XRef r_lesx(const HermV& X, const HermV& Xcc, int j, int n, double& s) {
    if (j <= n) return xref(X.les, tri(n) + j, false);
    s = -s;
    return xref(Xcc.les, tri(j) + n, true);
}
// X^A(j, n) = [Xcc^R(n, j)]^dagger; for j > n the continuation gives -X^R(j, n)
__device__ __forceinline__ XRef r_advx(const HermV& X, const HermV& Xcc, int j, int n, double& s) {
    if (j <= n) return xref(Xcc.ret, tri(n) + j, true);
    s = -s;
    return xref(X.ret, tri(j) + n, false);
}

// The single-time function: f_j (f_{-1} = f(0^-)), nullptr for the identity.
struct FRef {
    const cplx* p;
    int ldk;
};

// Columns of the result one thread accumulates: all of them up to d = 4, half a row for d = 8
// (keeps the row accumulators and the streamed factors within the register file).
template <int D>
struct ConvCols {
    static constexpr int W = D > 4 ? 4 : D;
};

// acc[b] += w * sum_c (X f_j)[a][c] Y[c][b0 + b], b = 0..W-1
template <int D>
__device__ __forceinline__ void conv_term(cplx (&acc)[ConvCols<D>::W], double w, const XRef& X, const FRef& f, int j,
                                          const XRef& Y, int a, int b0, int kb) {
    constexpr int NW = ConvCols<D>::W;
    cplx t[D];
    if (f.p == nullptr) {
#pragma unroll
        for (int c = 0; c < D; ++c) t[c] = xat<D>(X, a, c, kb);
    } else {
        const int64_t kk = f.ldk == 1 ? 0 : kb;
#pragma unroll
        for (int c = 0; c < D; ++c) t[c] = cz();
#pragma unroll(D > 2 ? 1 : D)
        for (int e = 0; e < D; ++e) {
            const cplx x = xat<D>(X, a, e, kb);
#pragma unroll
            for (int c = 0; c < D; ++c) t[c] = cfma(x, f.p[((int64_t)(j + 1) * (D * D) + e * D + c) * f.ldk + kk], t[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < D; ++c) {
        const cplx tc = cscal(w, t[c]);
#pragma unroll
        for (int b = 0; b < NW; ++b) acc[b] = cfma(tc, xat<D>(Y, c, b0 + b, kb), acc[b]);
    }
}

template <int NW>
__device__ __forceinline__ void row_zero(cplx (&r)[NW]) {
#pragma unroll
    for (int b = 0; b < NW; ++b) r[b] = cz();
}

// ---- Matsubara pieces (Eqs. cm1, cm2), without the factor h_tau ------------------------------
template <int D>
__device__ void conv_mat(const NgWeights& W, const Grid& g, const HermV& A, const FRef& f, const HermV& B, int m,
                         int a, int b0, int kb, cplx (&acc)[ConvCols<D>::W]) {
    const int k = W.k, T = g.ntau;
    const double xi = (double)g.sig;
    if (m <= k) {
        #pragma unroll 1
        for (int j = 0; j <= k; ++j)
            #pragma unroll 1
            for (int l = 0; l <= k; ++l)
                conv_term<D>(acc, W.R[m][j][l], xref(A.mat, j, false), f, -1, xref(B.mat, l, false), a, b0, kb);
    } else {
        #pragma unroll 1
        for (int l = 0; l <= m; ++l)
            conv_term<D>(acc, gw(W, m, l), xref(A.mat, m - l, false), f, -1, xref(B.mat, l, false), a, b0, kb);
    }
    if (m >= T - k) {
        #pragma unroll 1
        for (int j = 0; j <= k; ++j)
            #pragma unroll 1
            for (int l = 0; l <= k; ++l)
                conv_term<D>(acc, xi * W.R[T - m][j][l], xref(A.mat, T - j, false), f, -1, xref(B.mat, T - l, false),
                             a, b0, kb);
    } else {
        #pragma unroll 1
        for (int l = 0; l <= T - m; ++l)
            conv_term<D>(acc, xi * gw(W, T - m, l), xref(A.mat, T - l, false), f, -1, xref(B.mat, m + l, false), a, b0,
                         kb);
    }
}

// ---- retarded (Eq. cr1), without the factor h -------------------------------------------------
template <int D>
__device__ void conv_ret(const NgWeights& W, const HermV& A, const HermV& Acc, const FRef& f, const HermV& B,
                         const HermV& Bcc, int n, int m, int a, int b0, int kb, cplx (&acc)[ConvCols<D>::W]) {
    const int k = W.k;
    if (n > k && n - m > k) {
        #pragma unroll 1
        for (int j = m; j <= n; ++j)
            conv_term<D>(acc, gw(W, n - m, j - m), xref(A.ret, tri(n) + j, false), f, j, xref(B.ret, tri(j) + m, false),
                         a, b0, kb);
    } else if (n > k) {
        #pragma unroll 1
        for (int j = 0; j <= k; ++j) {
            double s = gw(W, n - m, j);
            XRef y = r_retx(B, Bcc, n - j, m, s);
            conv_term<D>(acc, s, xref(A.ret, tri(n) + n - j, false), f, n - j, y, a, b0, kb);
        }
    } else {
        #pragma unroll 1
        for (int j = 0; j <= k; ++j) {
            double s = W.I[m][n][j];
            XRef x = r_retx(A, Acc, n, j, s);
            XRef y = r_retx(B, Bcc, j, m, s);
            conv_term<D>(acc, s, x, f, j, y, a, b0, kb);
        }
    }
}

// ---- left-mixing (Eqs. ctv1, ctv2, ctv3): accR (factor h) and accM (factor h_tau) --------------
template <int D>
__device__ void conv_tv(const NgWeights& W, const Grid& g, const HermV& A, const HermV& Acc, const FRef& f,
                        const HermV& B, int n, int m, int a, int b0, int kb, cplx (&accR)[ConvCols<D>::W], cplx (&accM)[ConvCols<D>::W]) {
    const int k = W.k, T = g.ntau;
    const double xi = (double)g.sig;
    const int jmax = n > k ? n : k;
    #pragma unroll 1
    for (int j = 0; j <= jmax; ++j) {
        double s = gw(W, n, j);
        XRef x = r_retx(A, Acc, n, j, s);
        conv_term<D>(accR, s, x, f, j, xref(B.tv, (int64_t)j * (T + 1) + m, false), a, b0, kb);
    }
    const int64_t rowA = (int64_t)n * (T + 1);
    if (m <= k) {
        #pragma unroll 1
        for (int j = 0; j <= k; ++j)
            #pragma unroll 1
            for (int l = 0; l <= k; ++l)
                conv_term<D>(accM, xi * W.R[m][j][l], xref(A.tv, rowA + l, false), f, -1, xref(B.mat, T - j, false),
                             a, b0, kb);
    } else {
        #pragma unroll 1
        for (int l = 0; l <= m; ++l)
            conv_term<D>(accM, xi * gw(W, m, l), xref(A.tv, rowA + m - l, false), f, -1, xref(B.mat, T - l, false), a, b0,
                         kb);
    }
    if (m >= T - k) {
        #pragma unroll 1
        for (int j = 0; j <= k; ++j)
            #pragma unroll 1
            for (int l = 0; l <= k; ++l)
                conv_term<D>(accM, W.R[T - m][j][l], xref(A.tv, rowA + T - l, false), f, -1, xref(B.mat, j, false), a, b0,
                             kb);
    } else {
        #pragma unroll 1
        for (int l = 0; l <= T - m; ++l)
            conv_term<D>(accM, gw(W, T - m, l), xref(A.tv, rowA + m + l, false), f, -1, xref(B.mat, l, false), a, b0, kb);
    }
}

// ---- lesser C^<(t_m, t_n), m <= n (Eqs. cles1, cles2, cles3): accR (factor h) and acc3 -------
// (factor -i h_tau)
template <int D>
__device__ void conv_les(const NgWeights& W, const Grid& g, const HermV& A, const HermV& Acc, const FRef& f,
                         const HermV& B, const HermV& Bcc, int m, int n, int a, int b0, int kb, cplx (&accR)[ConvCols<D>::W],
                         cplx (&acc3)[ConvCols<D>::W]) {
    const int k = W.k, T = g.ntau;
    const double xi = (double)g.sig;
    // C^<_1 = int_0^{t_m} A^R(t_m, s) f(s) B^<(s, t_n)
    const int j1 = m > k ? m : k;
    #pragma unroll 1
    for (int j = 0; j <= j1; ++j) {
        double s = gw(W, m, j);
        XRef x = r_retx(A, Acc, m, j, s);
        XRef y = r_lesx(B, Bcc, j, n, s);
        conv_term<D>(accR, s, x, f, j, y, a, b0, kb);
    }
    // C^<_2 = int_0^{t_n} A^<(t_m, s) f(s) B^A(s, t_n)
    const int j2 = n > k ? n : k;
    #pragma unroll 1
    for (int j = 0; j <= j2; ++j) {
        double s = gw(W, n, j);
        XRef x = r_lesx(A, Acc, m, j, s);
        XRef y = r_advx(B, Bcc, j, n, s);
        conv_term<D>(accR, s, x, f, j, y, a, b0, kb);
    }
    // C^<_3 = -i int_0^beta A^tv(t_m, tau) f(0^-) B^vt(tau, t_n), B^vt(tau_j, t_n) =
    // -xi [Bcc^tv(t_n, beta - tau_j)]^dagger
    const int64_t rowA = (int64_t)m * (T + 1), rowB = (int64_t)n * (T + 1);
    #pragma unroll 1
    for (int j = 0; j <= T; ++j)
        conv_term<D>(acc3, -xi * gw(W, T, j), xref(A.tv, rowA + j, false), f, -1, xref(Bcc.tv, rowB + T - j, true), a, b0,
                     kb);
}

template <int D>
__device__ __forceinline__ void row_store(const Comp& c, int64_t e, int a, int b0, int kb,
                                          const cplx (&r)[ConvCols<D>::W], int* status) {
    const int64_t kk = c.ldk == 1 ? 0 : kb;
    bool ok = true;
#pragma unroll
    for (int b = 0; b < ConvCols<D>::W; ++b) {
        ok = ok && cfinite(r[b]);
        c.p[(e * (D * D) + a * D + b0 + b) * c.ldk + kk] = r[b];
    }
    if (!ok) atomicOr(status, NGF_NONFINITE);
}

// Slice n of C = A * f * B for nbe problems (nbe = C's ldk).  Items: (element, a, column block,
// problem), problem fastest; elements 0..n: C^R(n, m); n+1..n+T+1: C^tv(n, m); then C^<(m, n),
// m <= n.  For n = -1 the elements are C^M(tau_m), m = 0..T.
template <int D>
__global__ void __launch_bounds__(128) k_conv_slice(Grid g, int n, HermV C, HermV A, HermV Acc, FRef f, HermV B,
                                                    HermV Bcc, int nbe, int* status) {
    constexpr int NW = ConvCols<D>::W, NB = D / NW;
    const NgWeights& W = c_W[g.k - 1];
    const int T = g.ntau;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int cnt = n < 0 ? T + 1 : 2 * (n + 1) + T + 1;
    if (item >= (int64_t)cnt * D * NB * nbe) return;
    const int kb = (int)(item % nbe);
    int64_t r = item / nbe;
    const int b0 = (int)(r % NB) * NW;
    r /= NB;
    const int a = (int)(r % D);
    int el = (int)(r / D);
    cplx acc[NW], acc2[NW];
    row_zero<NW>(acc);
    row_zero<NW>(acc2);
    if (n < 0) {
        conv_mat<D>(W, g, A, f, B, el, a, b0, kb, acc);
#pragma unroll
        for (int b = 0; b < NW; ++b) acc[b] = cscal(g.htau, acc[b]);
        row_store<D>(C.mat, el, a, b0, kb, acc, status);
        return;
    }
    if (el <= n) {
        conv_ret<D>(W, A, Acc, f, B, Bcc, n, el, a, b0, kb, acc);
#pragma unroll
        for (int b = 0; b < NW; ++b) acc[b] = cscal(g.h, acc[b]);
        row_store<D>(C.ret, tri(n) + el, a, b0, kb, acc, status);
        return;
    }
    el -= n + 1;
    if (el <= T) {
        conv_tv<D>(W, g, A, Acc, f, B, n, el, a, b0, kb, acc, acc2);
#pragma unroll
        for (int b = 0; b < NW; ++b) acc[b] = cadd(cscal(g.h, acc[b]), cscal(g.htau, acc2[b]));
        row_store<D>(C.tv, (int64_t)n * (T + 1) + el, a, b0, kb, acc, status);
        return;
    }
    el -= T + 1;
    conv_les<D>(W, g, A, Acc, f, B, Bcc, el, n, a, b0, kb, acc, acc2);
    // h acc + (-i h_tau) acc2
#pragma unroll
    for (int b = 0; b < NW; ++b) acc[b] = cadd(cscal(g.h, acc[b]), cscal(g.htau, cmulmi(acc2[b])));
    row_store<D>(C.les, tri(n) + el, a, b0, kb, acc, status);
}
