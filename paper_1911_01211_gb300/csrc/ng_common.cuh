// Common device helpers of libng: complex arithmetic, small d x d matrices, the packed
// k-innermost layout of the contour store, and access to the integration weights.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ng_weights.h"

// integration weights for k = 1..NG_KMAX (index k-1), loaded once per device by ng_create
__constant__ NgWeights c_W[NG_KMAX];

typedef double2 cplx;

// ---------------------------------------------------------------------------------------
// complex scalar arithmetic (FP64)
// ---------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ cplx cz() { return make_double2(0.0, 0.0); }
__host__ __device__ __forceinline__ cplx cr(double x) { return make_double2(x, 0.0); }
__host__ __device__ __forceinline__ cplx cadd(cplx a, cplx b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ cplx csub(cplx a, cplx b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ cplx cneg(cplx a) { return make_double2(-a.x, -a.y); }
__host__ __device__ __forceinline__ cplx cconj(cplx a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ cplx cscal(double s, cplx a) { return make_double2(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ cplx cmuli(cplx a) { return make_double2(-a.y, a.x); }   // i a
__host__ __device__ __forceinline__ cplx cmulmi(cplx a) { return make_double2(a.y, -a.x); }  // -i a
__host__ __device__ __forceinline__ cplx cmul(cplx a, cplx b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// c + a b with four fused multiply-adds
__host__ __device__ __forceinline__ cplx cfma(cplx a, cplx b, cplx c) {
    c.x = fma(a.x, b.x, c.x);
    c.x = fma(-a.y, b.y, c.x);
    c.y = fma(a.x, b.y, c.y);
    c.y = fma(a.y, b.x, c.y);
    return c;
}
__host__ __device__ __forceinline__ double cabs2(cplx a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
    // Smith's algorithm (R. L. Smith, CACM 1962) for a / b
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, den = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / den, (a.y - a.x * r) / den);
    }
    double r = b.x / b.y, den = b.x * r + b.y;
    return make_double2((a.x * r + a.y) / den, (a.y * r - a.x) / den);
}
__host__ __device__ __forceinline__ bool cfinite(cplx a) { return isfinite(a.x) && isfinite(a.y); }

// ---------------------------------------------------------------------------------------
// d x d complex matrices in registers
// ---------------------------------------------------------------------------------------
template <int D>
struct Mat {
    cplx v[D][D];
};

template <int D>
__host__ __device__ __forceinline__ Mat<D> mzero() {
    Mat<D> r;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) r.v[a][b] = cz();
    return r;
}
template <int D>
__host__ __device__ __forceinline__ Mat<D> meye(cplx s) {
    Mat<D> r = mzero<D>();
#pragma unroll
    for (int a = 0; a < D; ++a) r.v[a][a] = s;
    return r;
}
template <int D>
__host__ __device__ __forceinline__ Mat<D> madd(const Mat<D>& x, const Mat<D>& y) {
    Mat<D> r;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) r.v[a][b] = cadd(x.v[a][b], y.v[a][b]);
    return r;
}
template <int D>
__host__ __device__ __forceinline__ Mat<D> msub(const Mat<D>& x, const Mat<D>& y) {
    Mat<D> r;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) r.v[a][b] = csub(x.v[a][b], y.v[a][b]);
    return r;
}
template <int D>
__host__ __device__ __forceinline__ Mat<D> mscal(double s, const Mat<D>& x) {
    Mat<D> r;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) r.v[a][b] = cscal(s, x.v[a][b]);
    return r;
}
template <int D>
__host__ __device__ __forceinline__ Mat<D> mcscal(cplx s, const Mat<D>& x) {
    Mat<D> r;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) r.v[a][b] = cmul(s, x.v[a][b]);
    return r;
}
template <int D>
__host__ __device__ __forceinline__ Mat<D> mmuli(const Mat<D>& x) {
    Mat<D> r;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) r.v[a][b] = cmuli(x.v[a][b]);
    return r;
}
template <int D>
__host__ __device__ __forceinline__ Mat<D> mdag(const Mat<D>& x) {
    Mat<D> r;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) r.v[a][b] = cconj(x.v[b][a]);
    return r;
}
template <int D>
__host__ __device__ __forceinline__ Mat<D> mmul(const Mat<D>& x, const Mat<D>& y) {
    Mat<D> r = mzero<D>();
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
            for (int b = 0; b < D; ++b) r.v[a][b] = cfma(x.v[a][c], y.v[c][b], r.v[a][b]);
    return r;
}
// acc += s * x * y  (s real)
template <int D>
__host__ __device__ __forceinline__ void mfma(Mat<D>& acc, const Mat<D>& x, const Mat<D>& y) {
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
            for (int b = 0; b < D; ++b) acc.v[a][b] = cfma(x.v[a][c], y.v[c][b], acc.v[a][b]);
}
template <int D>
__host__ __device__ __forceinline__ bool mfinite(const Mat<D>& x) {
    bool ok = true;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) ok = ok && cfinite(x.v[a][b]);
    return ok;
}
// inverse by Gauss-Jordan with partial pivoting; sets *sing if a pivot vanishes
template <int D>
__host__ __device__ __forceinline__ Mat<D> minv(const Mat<D>& x, int* sing) {
    if (D == 1) {
        Mat<D> r;
        if (cabs2(x.v[0][0]) == 0.0) *sing = 1;
        r.v[0][0] = cdiv(cr(1.0), x.v[0][0]);
        return r;
    }
    Mat<D> a = x, r = meye<D>(cr(1.0));
    for (int c = 0; c < D; ++c) {
        int p = c;
        double best = cabs2(a.v[c][c]);
        for (int i = c + 1; i < D; ++i)
            if (cabs2(a.v[i][c]) > best) { best = cabs2(a.v[i][c]); p = i; }
        if (best == 0.0) { *sing = 1; return r; }
        if (p != c)
            for (int j = 0; j < D; ++j) {
                cplx t = a.v[c][j]; a.v[c][j] = a.v[p][j]; a.v[p][j] = t;
                t = r.v[c][j]; r.v[c][j] = r.v[p][j]; r.v[p][j] = t;
            }
        cplx inv = cdiv(cr(1.0), a.v[c][c]);
        for (int j = 0; j < D; ++j) { a.v[c][j] = cmul(a.v[c][j], inv); r.v[c][j] = cmul(r.v[c][j], inv); }
        for (int i = 0; i < D; ++i) {
            if (i == c) continue;
            cplx f = a.v[i][c];
            for (int j = 0; j < D; ++j) {
                a.v[i][j] = csub(a.v[i][j], cmul(f, a.v[c][j]));
                r.v[i][j] = csub(r.v[i][j], cmul(f, r.v[c][j]));
            }
        }
    }
    return r;
}

// ---------------------------------------------------------------------------------------
// layout of the contour store (problem index innermost)
// ---------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ int64_t tri(int n) { return (int64_t)n * (n + 1) / 2; }

struct Grid {
    int nt, ntau, nf, nb, k, sig;
    double h, beta, mu, htau;
};

// A view of one herm component array: element e, orbital (a,b), problem kb.
struct Comp {
    cplx* p;
    int ldk;   // nb or 1
    int dd;    // nf*nf
    __host__ __device__ __forceinline__ int64_t idx(int64_t e, int a, int b, int kb, int nf) const {
        return (e * dd + a * nf + b) * ldk + (ldk == 1 ? 0 : kb);
    }
};

struct HermV {
    Comp mat, ret, les, tv;
};

struct FuncV {
    cplx* p;
    int ldk;
};

template <int D>
__device__ __forceinline__ Mat<D> ld(const Comp& c, int64_t e, int kb) {
    Mat<D> r;
    const int64_t kk = (c.ldk == 1 ? 0 : kb);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) r.v[a][b] = c.p[(e * (D * D) + a * D + b) * c.ldk + kk];
    return r;
}
template <int D>
__device__ __forceinline__ void st(const Comp& c, int64_t e, int kb, const Mat<D>& x) {
    const int64_t kk = (c.ldk == 1 ? 0 : kb);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) c.p[(e * (D * D) + a * D + b) * c.ldk + kk] = x.v[a][b];
}
template <int D>
__device__ __forceinline__ Mat<D> ldf(const FuncV& f, int n, int kb) {
    Mat<D> r;
    const int64_t kk = (f.ldk == 1 ? 0 : kb);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) r.v[a][b] = f.p[((int64_t)(n + 1) * (D * D) + a * D + b) * f.ldk + kk];
    return r;
}

// component accessors (Eq. hermconjg of the paper), all for hermitian-symmetric data
template <int D>
__device__ __forceinline__ Mat<D> gret(const HermV& X, int n, int j, int kb) {  // X^R(n,j), j <= n
    return ld<D>(X.ret, tri(n) + j, kb);
}
template <int D>
__device__ __forceinline__ Mat<D> gretx(const HermV& X, int n, int j, int kb) {  // continued to j > n
    if (j <= n) return ld<D>(X.ret, tri(n) + j, kb);
    return mscal<D>(-1.0, mdag<D>(ld<D>(X.ret, tri(j) + n, kb)));
}
template <int D>
__device__ __forceinline__ Mat<D> gles(const HermV& X, int j, int n, int kb) {  // X^<(j,n), any j,n
    if (j <= n) return ld<D>(X.les, tri(n) + j, kb);
    return mscal<D>(-1.0, mdag<D>(ld<D>(X.les, tri(j) + n, kb)));
}
template <int D>
__device__ __forceinline__ Mat<D> gtv(const HermV& X, const Grid& g, int n, int m, int kb) {
    return ld<D>(X.tv, (int64_t)n * (g.ntau + 1) + m, kb);
}
template <int D>
__device__ __forceinline__ Mat<D> gvt(const HermV& X, const Grid& g, int m, int n, int kb) {  // X^vt(tau_m, t_n)
    return mscal<D>(-(double)g.sig, mdag<D>(gtv<D>(X, g, n, g.ntau - m, kb)));
}
template <int D>
__device__ __forceinline__ Mat<D> gmat(const HermV& X, int m, int kb) {
    return ld<D>(X.mat, m, kb);
}

// ---------------------------------------------------------------------------------------
// Gregory weights w_{n,j} (Eq. integrator_greg): table rows for n <= 2k+1, end weights
// omega_j and interior ones beyond.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double gw(const NgWeights& W, int n, int j) {
    const int k = W.k;
    if (n <= 2 * k + 1) return W.greg[n][j];
    if (j <= k) return W.omega[j];
    if (j >= n - k) return W.omega[n - j];
    return 1.0;
}

// status word bits
#define NGF_NONFINITE 1
#define NGF_SINGULAR 2
