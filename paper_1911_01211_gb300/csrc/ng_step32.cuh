// FP32-compensated variant of the bulk time-step kernel (precision NG_F32C).
//
// The O(n) and O(ntau) history and source sums of the bulk items read FP32 copies of the
// committed slices (< n) of G and of slice n of Sigma, form every real product exactly as
// a sum of two FP32 numbers (TwoProd by fused multiply-add: p = a*b, e = fma(a, b, -p)) and
// accumulate with Kahan compensation, the product's low part folded into the compensation
// term.  The result of each sum is rounded once to FP64; the BDF terms, the per-step matrix
// M_n^-1 and the output stay FP64.  Same formulas and schedule as ng_step.cuh.
#pragma once

#include "ng_step.cuh"

typedef float2 cplx32;

struct Comp32 {
    cplx32* p;
    int ldk;
};
struct HermV32 {
    Comp32 mat, ret, les, tv;
};

// Kahan accumulator of a real sum of exact products: value = s - c
struct KSum {
    float s, c;
};
__device__ __forceinline__ void kadd(KSum& k, float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);  // a*b = p + e exactly
    const float y = p - k.c;
    const float t = k.s + y;
    k.c = ((t - k.s) - y) - e;
    k.s = t;
}

template <int D>
struct KMat {
    KSum re[D][D], im[D][D];
};
template <int D>
__device__ __forceinline__ KMat<D> kzero() {
    KMat<D> r;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) r.re[a][b] = KSum{0.f, 0.f}, r.im[a][b] = KSum{0.f, 0.f};
    return r;
}
template <int D>
struct M32 {
    cplx32 v[D][D];
};
// acc += x * y  (complex, compensated)
template <int D>
__device__ __forceinline__ void kfma(KMat<D>& acc, const M32<D>& x, const M32<D>& y) {
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
            for (int b = 0; b < D; ++b) {
                kadd(acc.re[a][b], x.v[a][c].x, y.v[c][b].x);
                kadd(acc.re[a][b], -x.v[a][c].y, y.v[c][b].y);
                kadd(acc.im[a][b], x.v[a][c].x, y.v[c][b].y);
                kadd(acc.im[a][b], x.v[a][c].y, y.v[c][b].x);
            }
}
// acc += x * y^dagger
template <int D>
__device__ __forceinline__ void kfma_db(KMat<D>& acc, const M32<D>& x, const M32<D>& y) {
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
            for (int b = 0; b < D; ++b) {
                // conj(y[b][c]) = (y.x, -y.y)
                kadd(acc.re[a][b], x.v[a][c].x, y.v[b][c].x);
                kadd(acc.re[a][b], x.v[a][c].y, y.v[b][c].y);
                kadd(acc.im[a][b], -x.v[a][c].x, y.v[b][c].y);
                kadd(acc.im[a][b], x.v[a][c].y, y.v[b][c].x);
            }
}
template <int D>
__device__ __forceinline__ Mat<D> kval(const KMat<D>& k) {
    Mat<D> r;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b)
            r.v[a][b] = make_double2((double)k.re[a][b].s - (double)k.re[a][b].c,
                                     (double)k.im[a][b].s - (double)k.im[a][b].c);
    return r;
}
template <int D>
__device__ __forceinline__ M32<D> ld32(const Comp32& c, int64_t e, int kb) {
    M32<D> r;
    const int64_t kk = (c.ldk == 1 ? 0 : kb);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) r.v[a][b] = c.p[(e * (D * D) + a * D + b) * c.ldk + kk];
    return r;
}
template <int D>
__device__ __forceinline__ M32<D> s32(float w, M32<D> x) {
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) x.v[a][b].x *= w, x.v[a][b].y *= w;
    return x;
}
template <int D>
__device__ __forceinline__ M32<D> ndag32(const M32<D>& x) {  // -x^dagger
    M32<D> r;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) r.v[a][b] = make_float2(-x.v[b][a].x, x.v[b][a].y);
    return r;
}

// -i (C^tv_2 + C^tv_3)[Sigma, 1, G^M](n, m) with FP32 inputs, compensated
template <int D>
__device__ Mat<D> q_tv32(const NgWeights& W, const Grid& g, const HermV32& G, const HermV32& S, int n, int m,
                         int kb) {
    const int k = W.k, T = g.ntau;
    const int64_t rowS = (int64_t)n * (T + 1);
    KMat<D> c2 = kzero<D>(), c3 = kzero<D>();
    if (m <= k) {
        for (int j = 0; j <= k; ++j) {
            M32<D> gm = ld32<D>(G.mat, T - j, kb);
            for (int l = 0; l <= k; ++l) kfma<D>(c2, s32<D>((float)W.R[m][j][l], ld32<D>(S.tv, rowS + l, kb)), gm);
        }
    } else {
        greg_for(W, m, m, [&](int l, double w) {
            kfma<D>(c2, s32<D>((float)w, ld32<D>(S.tv, rowS + m - l, kb)), ld32<D>(G.mat, T - l, kb));
        });
    }
    if (m >= T - k) {
        for (int j = 0; j <= k; ++j) {
            M32<D> gm = ld32<D>(G.mat, j, kb);
            for (int l = 0; l <= k; ++l)
                kfma<D>(c3, s32<D>((float)W.R[T - m][j][l], ld32<D>(S.tv, rowS + T - l, kb)), gm);
        }
    } else {
        greg_for(W, T - m, T - m, [&](int l, double w) {
            kfma<D>(c3, s32<D>((float)w, ld32<D>(S.tv, rowS + m + l, kb)), ld32<D>(G.mat, l, kb));
        });
    }
    Mat<D> v = madd<D>(mscal<D>((double)g.sig, kval<D>(c2)), kval<D>(c3));
    return mscal<D>(g.htau, mmuli<D>(mscal<D>(-1.0, v)));
}

template <int D>
__device__ __forceinline__ void ret_item32(const NgWeights& W, const Grid& g, const HermV& G, const HermV& S,
                                           const HermV32& G32, const HermV32& S32, const Mat<D>& Minv, int n,
                                           int m, int kb, int* status) {
    const int L = n - m;
    KMat<D> acc = kzero<D>();
    const int64_t rowS = tri(n);
    greg_for(W, L, L - 1, [&](int l, double w) {
        kfma<D>(acc, s32<D>((float)w, ld32<D>(S32.ret, rowS + m + l, kb)), ld32<D>(G32.ret, tri(m + l) + m, kb));
    });
    Mat<D> bdf = mzero<D>();
    for (int l = 1; l <= W.k; ++l) bdf = madd<D>(bdf, mscal<D>(W.a[l], gret<D>(G, n - l, m, kb)));
    Mat<D> rhs = msub<D>(mscal<D>(-1.0 / g.h, bdf), mscal<D>(g.h, mmuli<D>(kval<D>(acc))));
    Mat<D> y = mmul<D>(Minv, rhs);
    if (!mfinite<D>(y)) atomicOr(status, NGF_NONFINITE);
    st<D>(G.ret, tri(n) + m, kb, y);
}

template <int D>
__device__ __forceinline__ void tv_item32(const NgWeights& W, const Grid& g, const HermV& G, const HermV& S,
                                          const HermV32& G32, const HermV32& S32, const Mat<D>& Minv, int n,
                                          int m, int kb, const cplx* tvq, int* status) {
    KMat<D> acc = kzero<D>();
    const int64_t rowS = tri(n);
    const int T1 = g.ntau + 1;
    greg_for(W, n, n - 1, [&](int j, double w) {
        kfma<D>(acc, s32<D>((float)w, ld32<D>(S32.ret, rowS + j, kb)), ld32<D>(G32.tv, (int64_t)j * T1 + m, kb));
    });
    Mat<D> bdf = mzero<D>();
    for (int l = 1; l <= W.k; ++l) bdf = madd<D>(bdf, mscal<D>(W.a[l], gtv<D>(G, g, n - l, m, kb)));
    Mat<D> rhs = tvq ? q_tv_fft<D>(W, g, G, S, n, m, kb, tvq) : q_tv32<D>(W, g, G32, S32, n, m, kb);
    rhs = msub<D>(rhs, mscal<D>(1.0 / g.h, bdf));
    rhs = msub<D>(rhs, mscal<D>(g.h, mmuli<D>(kval<D>(acc))));
    Mat<D> y = mmul<D>(Minv, rhs);
    if (!mfinite<D>(y)) atomicOr(status, NGF_NONFINITE);
    st<D>(G.tv, (int64_t)n * T1 + m, kb, y);
}

template <int D>
__device__ __forceinline__ void les_item32(const NgWeights& W, const Grid& g, const HermV& G, const HermV& S,
                                           const HermV32& G32, const HermV32& S32, const Mat<D>& Minv, int n,
                                           int m, int kb, int* status) {
    const int k = W.k, T = g.ntau, T1 = g.ntau + 1;
    const int64_t colS = tri(n);
    KMat<D> c1 = kzero<D>();
    if (m <= k) {
        for (int j = 0; j <= k; ++j) {
            M32<D> gr = (j <= m) ? ld32<D>(G32.ret, tri(m) + j, kb) : ndag32<D>(ld32<D>(G32.ret, tri(j) + m, kb));
            kfma<D>(c1, s32<D>((float)W.greg[m][j], gr), ld32<D>(S32.les, colS + j, kb));
        }
    } else {
        const int64_t rowG = tri(m);
        greg_for(W, m, m, [&](int j, double w) {
            kfma<D>(c1, s32<D>((float)w, ld32<D>(G32.ret, rowG + j, kb)), ld32<D>(S32.les, colS + j, kb));
        });
    }
    KMat<D> c3 = kzero<D>();
    const int64_t rowGt = (int64_t)m * T1, rowSt = (int64_t)n * T1;
    greg_for(W, T, T, [&](int j, double w) {
        kfma_db<D>(c3, s32<D>((float)w, ld32<D>(G32.tv, rowGt + j, kb)), ld32<D>(S32.tv, rowSt + T - j, kb));
    });
    Mat<D> q = msub<D>(mscal<D>(g.h, mmuli<D>(kval<D>(c1))), mscal<D>((double)g.sig * g.htau, kval<D>(c3)));
    KMat<D> hist = kzero<D>();
    const int64_t rowS = tri(n), colM = tri(m);
    greg_for(W, n, n - 1, [&](int l, double w) {
        M32<D> gl = (l >= m) ? ld32<D>(G32.les, tri(l) + m, kb) : ndag32<D>(ld32<D>(G32.les, colM + l, kb));
        kfma_db<D>(hist, s32<D>((float)w, gl), ld32<D>(S32.ret, rowS + l, kb));
    });
    Mat<D> bdf = mzero<D>();
    for (int l = 1; l <= k; ++l) bdf = madd<D>(bdf, mscal<D>(W.a[l], ld<D>(G.les, tri(n - l) + m, kb)));
    Mat<D> rhs = msub<D>(q, mscal<D>(1.0 / g.h, bdf));
    rhs = madd<D>(rhs, mscal<D>(g.h, mmuli<D>(kval<D>(hist))));
    Mat<D> y = mmul<D>(rhs, mdag<D>(Minv));
    if (!mfinite<D>(y)) atomicOr(status, NGF_NONFINITE);
    st<D>(G.les, tri(n) + m, kb, y);
}

template <int D>
__global__ void __launch_bounds__(128) k_step_bulk32(Grid g, int n, HermV G, HermV S, HermV32 G32, HermV32 S32,
                                                     FuncV eps, const cplx* minv_ws, int nb_les, int nb_tv,
                                                     int nb_ret, const cplx* tvq, int* status) {
    const NgWeights& W = c_W[g.k - 1];
    int blk = blockIdx.x;
    int task;
    if (blk < nb_les) task = 0;
    else if ((blk -= nb_les) < nb_tv) task = 1;
    else { blk -= nb_tv; task = 2; }
    const int64_t item = (int64_t)blk * blockDim.x + threadIdx.x;
    const int kb = (int)(item % g.nb);
    const int64_t col = item / g.nb;
    int ncol;
    if (task == 0) ncol = n - W.k - 1;
    else if (task == 1) ncol = g.ntau + 1;
    else ncol = n - W.k;
    if (col >= ncol) return;
    const Mat<D> Minv = ld_minv<D>(minv_ws, kb);
    if (task == 0) les_item32<D>(W, g, G, S, G32, S32, Minv, n, (int)col + 1, kb, status);
    else if (task == 1) tv_item32<D>(W, g, G, S, G32, S32, Minv, n, (int)col, kb, tvq, status);
    else ret_item32<D>(W, g, G, S, G32, S32, Minv, n, (int)col, kb, status);
}

// FP32 copies of slices [n0, n1] of a contour function (mat when n0 = -1); one thread per
// (element, orbital pair, problem) over the slices' ret rows, les columns and tv rows.
__global__ void k_shadow(Grid g, int n0, int n1, HermV X, HermV32 Y, int ldk) {
    const int dd = g.nf * g.nf;
    const int T1 = g.ntau + 1;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // ret and les: elements tri(a)..tri(b+1)-1 for the slices a = max(n0,0)..n1; tv rows; mat
    const int a = n0 < 0 ? 0 : n0;
    const int64_t e_tri0 = tri(a), n_tri = tri(n1 + 1) - e_tri0;
    const int64_t n_tv = (int64_t)(n1 - a + 1) * T1;
    const int64_t n_mat = n0 < 0 ? T1 : 0;
    const int64_t per = (int64_t)dd * ldk;
    const int64_t tot = (2 * n_tri + n_tv + n_mat) * per;
    for (int64_t i = item; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t e = i / per, r = i % per;
        const cplx* src;
        cplx32* dst;
        int64_t off;
        if (e < n_tri) { off = (e_tri0 + e) * per + r; src = X.ret.p; dst = Y.ret.p; }
        else if ((e -= n_tri) < n_tri) { off = (e_tri0 + e) * per + r; src = X.les.p; dst = Y.les.p; }
        else if ((e -= n_tri) < n_tv) { off = ((int64_t)a * T1 + e) * per + r; src = X.tv.p; dst = Y.tv.p; }
        else { e -= n_tv; off = e * per + r; src = X.mat.p; dst = Y.mat.p; }
        const cplx v = src[off];
        dst[off] = make_float2((float)v.x, (float)v.y);
    }
}

// ----------------------------------------------------------------------------------------
// nf = 1 with two adjacent problems per thread: every history element of the pair is one
// 16-byte load (the FP32 copies keep the problem index innermost), and the two problems'
// compensated sums are independent chains, so each thread keeps twice the bytes and the
// arithmetic in flight.  Same formulas, order of terms and rounding as the one-problem items.
// Needs nb even (then every pair offset is 16-byte aligned).
// ----------------------------------------------------------------------------------------
struct P32 {
    float2 a, b;   // problems kb, kb+1
};
__device__ __forceinline__ P32 ldp(const Comp32& c, int64_t e, int kb) {
    if (c.ldk == 1) {
        const float2 v = c.p[e];
        return P32{v, v};
    }
    const float4 v = *reinterpret_cast<const float4*>(c.p + e * c.ldk + kb);
    return P32{make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ P32 pscal(float w, P32 x) {
    x.a.x *= w, x.a.y *= w, x.b.x *= w, x.b.y *= w;
    return x;
}
__device__ __forceinline__ P32 pndag(P32 x) {   // -conj, per problem
    x.a.x = -x.a.x, x.b.x = -x.b.x;
    return x;
}
struct KP {
    KSum re[2], im[2];
};
__device__ __forceinline__ KP kpzero() {
    KP r;
#pragma unroll
    for (int i = 0; i < 2; ++i) r.re[i] = KSum{0.f, 0.f}, r.im[i] = KSum{0.f, 0.f};
    return r;
}
__device__ __forceinline__ void kcadd(KSum& re, KSum& im, float2 x, float2 y) {   // += x y
    kadd(re, x.x, y.x);
    kadd(re, -x.y, y.y);
    kadd(im, x.x, y.y);
    kadd(im, x.y, y.x);
}
__device__ __forceinline__ void kcadd_db(KSum& re, KSum& im, float2 x, float2 y) {   // += x conj(y)
    kadd(re, x.x, y.x);
    kadd(re, x.y, y.y);
    kadd(im, -x.x, y.y);
    kadd(im, x.y, y.x);
}
__device__ __forceinline__ void kpfma(KP& k, const P32& x, const P32& y) {
    kcadd(k.re[0], k.im[0], x.a, y.a);
    kcadd(k.re[1], k.im[1], x.b, y.b);
}
__device__ __forceinline__ void kpfma_db(KP& k, const P32& x, const P32& y) {
    kcadd_db(k.re[0], k.im[0], x.a, y.a);
    kcadd_db(k.re[1], k.im[1], x.b, y.b);
}
__device__ __forceinline__ Mat<1> kpval(const KP& k, int i) {
    Mat<1> r;
    r.v[0][0] = make_double2((double)k.re[i].s - (double)k.re[i].c, (double)k.im[i].s - (double)k.im[i].c);
    return r;
}

// Tuning of the two-problems-per-thread kernel: blocks per SM it is compiled for, and how far
// the unit-weight middle of each Gregory sum is unrolled (more loads in flight per thread)
#ifndef NG_F32P_MINB
#define NG_F32P_MINB 8
#endif
#ifndef NG_F32P_UNROLL
#define NG_F32P_UNROLL 4
#endif

// greg_for with the unit-weight middle unrolled U times
template <int U, class F>
__device__ __forceinline__ void greg_for_u(const NgWeights& W, int L, int lmax, F&& f) {
    const int k = W.k;
    if (L <= 2 * k + 1) {
        for (int l = 0; l <= lmax; ++l) f(l, W.greg[L][l]);
        return;
    }
    const int e1 = min(k, lmax);
    for (int l = 0; l <= e1; ++l) f(l, W.omega[l]);
    const int e2 = min(L - k - 1, lmax);
#pragma unroll U
    for (int l = k + 1; l <= e2; ++l) f(l, 1.0);
    for (int l = L - k; l <= lmax; ++l) f(l, W.omega[L - l]);
}

__device__ __forceinline__ void ret_item32p(const NgWeights& W, const Grid& g, const HermV& G, const HermV32& G32,
                                            const HermV32& S32, const cplx* minv_ws, int n, int m, int kb,
                                            int* status) {
    const int L = n - m;
    KP acc = kpzero();
    const int64_t rowS = tri(n);
    greg_for_u<NG_F32P_UNROLL>(W, L, L - 1, [&](int l, double w) {
        kpfma(acc, pscal((float)w, ldp(S32.ret, rowS + m + l, kb)), ldp(G32.ret, tri(m + l) + m, kb));
    });
    for (int i = 0; i < 2; ++i) {
        Mat<1> bdf = mzero<1>();
        for (int l = 1; l <= W.k; ++l) bdf = madd<1>(bdf, mscal<1>(W.a[l], gret<1>(G, n - l, m, kb + i)));
        Mat<1> rhs = msub<1>(mscal<1>(-1.0 / g.h, bdf), mscal<1>(g.h, mmuli<1>(kpval(acc, i))));
        Mat<1> y = mmul<1>(ld_minv<1>(minv_ws, kb + i), rhs);
        if (!mfinite<1>(y)) atomicOr(status, NGF_NONFINITE);
        st<1>(G.ret, tri(n) + m, kb + i, y);
    }
}

__device__ __forceinline__ void tv_item32p(const NgWeights& W, const Grid& g, const HermV& G, const HermV& S,
                                           const HermV32& G32, const HermV32& S32, const cplx* minv_ws, int n, int m,
                                           int kb, const cplx* tvq, int* status) {
    KP acc = kpzero();
    const int64_t rowS = tri(n);
    const int T1 = g.ntau + 1;
    greg_for_u<NG_F32P_UNROLL>(W, n, n - 1, [&](int j, double w) {
        kpfma(acc, pscal((float)w, ldp(S32.ret, rowS + j, kb)), ldp(G32.tv, (int64_t)j * T1 + m, kb));
    });
    for (int i = 0; i < 2; ++i) {
        Mat<1> bdf = mzero<1>();
        for (int l = 1; l <= W.k; ++l) bdf = madd<1>(bdf, mscal<1>(W.a[l], gtv<1>(G, g, n - l, m, kb + i)));
        Mat<1> rhs = tvq ? q_tv_fft<1>(W, g, G, S, n, m, kb + i, tvq) : q_tv32<1>(W, g, G32, S32, n, m, kb + i);
        rhs = msub<1>(rhs, mscal<1>(1.0 / g.h, bdf));
        rhs = msub<1>(rhs, mscal<1>(g.h, mmuli<1>(kpval(acc, i))));
        Mat<1> y = mmul<1>(ld_minv<1>(minv_ws, kb + i), rhs);
        if (!mfinite<1>(y)) atomicOr(status, NGF_NONFINITE);
        st<1>(G.tv, (int64_t)n * T1 + m, kb + i, y);
    }
}

__device__ __forceinline__ void les_item32p(const NgWeights& W, const Grid& g, const HermV& G, const HermV32& G32,
                                            const HermV32& S32, const cplx* minv_ws, int n, int m, int kb,
                                            int* status) {
    const int k = W.k, T = g.ntau, T1 = g.ntau + 1;
    const int64_t colS = tri(n);
    KP c1 = kpzero();
    if (m <= k) {
        for (int j = 0; j <= k; ++j) {
            P32 gr = (j <= m) ? ldp(G32.ret, tri(m) + j, kb) : pndag(ldp(G32.ret, tri(j) + m, kb));
            kpfma(c1, pscal((float)W.greg[m][j], gr), ldp(S32.les, colS + j, kb));
        }
    } else {
        const int64_t rowG = tri(m);
        greg_for_u<NG_F32P_UNROLL>(W, m, m, [&](int j, double w) {
            kpfma(c1, pscal((float)w, ldp(G32.ret, rowG + j, kb)), ldp(S32.les, colS + j, kb));
        });
    }
    KP c3 = kpzero();
    const int64_t rowGt = (int64_t)m * T1, rowSt = (int64_t)n * T1;
    greg_for_u<NG_F32P_UNROLL>(W, T, T, [&](int j, double w) {
        kpfma_db(c3, pscal((float)w, ldp(G32.tv, rowGt + j, kb)), ldp(S32.tv, rowSt + T - j, kb));
    });
    KP hist = kpzero();
    const int64_t rowS = tri(n), colM = tri(m);
    greg_for_u<NG_F32P_UNROLL>(W, n, n - 1, [&](int l, double w) {
        P32 gl = (l >= m) ? ldp(G32.les, tri(l) + m, kb) : pndag(ldp(G32.les, colM + l, kb));
        kpfma_db(hist, pscal((float)w, gl), ldp(S32.ret, rowS + l, kb));
    });
    for (int i = 0; i < 2; ++i) {
        Mat<1> q = msub<1>(mscal<1>(g.h, mmuli<1>(kpval(c1, i))), mscal<1>((double)g.sig * g.htau, kpval(c3, i)));
        Mat<1> bdf = mzero<1>();
        for (int l = 1; l <= k; ++l) bdf = madd<1>(bdf, mscal<1>(W.a[l], ld<1>(G.les, tri(n - l) + m, kb + i)));
        Mat<1> rhs = msub<1>(q, mscal<1>(1.0 / g.h, bdf));
        rhs = madd<1>(rhs, mscal<1>(g.h, mmuli<1>(kpval(hist, i))));
        Mat<1> y = mmul<1>(rhs, mdag<1>(ld_minv<1>(minv_ws, kb + i)));
        if (!mfinite<1>(y)) atomicOr(status, NGF_NONFINITE);
        st<1>(G.les, tri(n) + m, kb + i, y);
    }
}

// nf = 1, nb even: items are (column, problem pair), pair index fastest
__global__ void __launch_bounds__(128, NG_F32P_MINB) k_step_bulk32p(Grid g, int n, HermV G, HermV S, HermV32 G32, HermV32 S32,
                                                      const cplx* minv_ws, int nb_les, int nb_tv, int nb_ret,
                                                      const cplx* tvq, int* status) {
    const NgWeights& W = c_W[g.k - 1];
    int blk = blockIdx.x;
    int task;
    if (blk < nb_les) task = 0;
    else if ((blk -= nb_les) < nb_tv) task = 1;
    else { blk -= nb_tv; task = 2; }
    const int np = g.nb >> 1;
    const int64_t item = (int64_t)blk * blockDim.x + threadIdx.x;
    const int kb = 2 * (int)(item % np);
    const int64_t col = item / np;
    int ncol;
    if (task == 0) ncol = n - W.k - 1;
    else if (task == 1) ncol = g.ntau + 1;
    else ncol = n - W.k;
    if (col >= ncol) return;
    if (task == 0) les_item32p(W, g, G, G32, S32, minv_ws, n, (int)col + 1, kb, status);
    else if (task == 1) tv_item32p(W, g, G, S, G32, S32, minv_ws, n, (int)col, kb, tvq, status);
    else ret_item32p(W, g, G, G32, S32, minv_ws, n, (int)col, kb, status);
}
