// Double-float variant of the bulk time-step kernel (precision NG_DF64).
//
// The O(n) and O(ntau) history and source sums read double-float copies of the committed
// slices (< n) of G and of slice n of Sigma: every real value x is stored as two FP32 numbers
// hi = fl32(x), lo = fl32(x - hi) (48 significand bits).  A product of two double-float
// numbers is formed as p = ah*bh with its error and the cross terms folded into
// e = fma(ah, bh, -p) + ah*bl + al*bh; sums use Knuth's TwoSum on the high parts and carry the
// low parts separately.  Quadrature weights enter as double-float numbers too.  The sum is
// rounded once to FP64; BDF terms, M_n^-1 and the output stay FP64.  Same formulas and
// schedule as ng_step.cuh.
#pragma once

#include "ng_step32.cuh"

struct Comp64x {
    float4* p;     // (re_hi, re_lo, im_hi, im_lo) per complex element
    int ldk;
};
struct HermVdf {
    Comp64x mat, ret, les, tv;
};

// double-float real accumulator: value = h + l
struct DSum {
    float h, l;
};
// s += (ah + al)(bh + bl), product error and cross terms folded into the low part
__device__ __forceinline__ void dfma_acc(DSum& s, float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    const float t = s.h + p;              // TwoSum(s.h, p)
    const float bp = t - s.h;
    const float err = (s.h - (t - bp)) + (p - bp);
    s.h = t;
    s.l += err + e;
}

// complex double-float value
struct CDF {
    float rh, rl, ih, il;
};
__device__ __forceinline__ CDF cdf_ld(const float4 v) { return CDF{v.x, v.y, v.z, v.w}; }
__device__ __forceinline__ CDF cdf_conj(CDF a) { return CDF{a.rh, a.rl, -a.ih, -a.il}; }
__device__ __forceinline__ CDF cdf_neg(CDF a) { return CDF{-a.rh, -a.rl, -a.ih, -a.il}; }
// scale by a real weight given as double: w = wh + wl, product (a w) kept as (p, e)
__device__ __forceinline__ void dfmul_real(float ah, float al, float wh, float wl, float& ph, float& pl) {
    ph = ah * wh;
    float e = fmaf(ah, wh, -ph);
    e = fmaf(ah, wl, e);
    pl = fmaf(al, wh, e);
}
__device__ __forceinline__ CDF cdf_scale(CDF a, double w) {
    const float wh = (float)w, wl = (float)(w - (double)wh);
    CDF r;
    dfmul_real(a.rh, a.rl, wh, wl, r.rh, r.rl);
    dfmul_real(a.ih, a.il, wh, wl, r.ih, r.il);
    return r;
}

template <int D>
struct DMat {
    DSum re[D][D], im[D][D];
};
template <int D>
struct MDF {
    CDF v[D][D];
};
template <int D>
__device__ __forceinline__ DMat<D> dzero() {
    DMat<D> r;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) r.re[a][b] = DSum{0.f, 0.f}, r.im[a][b] = DSum{0.f, 0.f};
    return r;
}
// acc += x y
template <int D>
__device__ __forceinline__ void dfma_m(DMat<D>& acc, const MDF<D>& x, const MDF<D>& y) {
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
            for (int b = 0; b < D; ++b) {
                const CDF& p = x.v[a][c];
                const CDF& q = y.v[c][b];
                dfma_acc(acc.re[a][b], p.rh, p.rl, q.rh, q.rl);
                dfma_acc(acc.re[a][b], -p.ih, -p.il, q.ih, q.il);
                dfma_acc(acc.im[a][b], p.rh, p.rl, q.ih, q.il);
                dfma_acc(acc.im[a][b], p.ih, p.il, q.rh, q.rl);
            }
}
// acc += x y^dagger
template <int D>
__device__ __forceinline__ void dfma_m_db(DMat<D>& acc, const MDF<D>& x, const MDF<D>& y) {
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
            for (int b = 0; b < D; ++b) {
                const CDF& p = x.v[a][c];
                const CDF q = cdf_conj(y.v[b][c]);
                dfma_acc(acc.re[a][b], p.rh, p.rl, q.rh, q.rl);
                dfma_acc(acc.re[a][b], -p.ih, -p.il, q.ih, q.il);
                dfma_acc(acc.im[a][b], p.rh, p.rl, q.ih, q.il);
                dfma_acc(acc.im[a][b], p.ih, p.il, q.rh, q.rl);
            }
}
template <int D>
__device__ __forceinline__ Mat<D> dval(const DMat<D>& k) {
    Mat<D> r;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b)
            r.v[a][b] = make_double2((double)k.re[a][b].h + (double)k.re[a][b].l,
                                     (double)k.im[a][b].h + (double)k.im[a][b].l);
    return r;
}
template <int D>
__device__ __forceinline__ MDF<D> lddf(const Comp64x& c, int64_t e, int kb) {
    MDF<D> r;
    const int64_t kk = (c.ldk == 1 ? 0 : kb);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) r.v[a][b] = cdf_ld(c.p[(e * (D * D) + a * D + b) * c.ldk + kk]);
    return r;
}
template <int D>
__device__ __forceinline__ MDF<D> sdf(double w, MDF<D> x) {
    if (w == 1.0) return x;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) x.v[a][b] = cdf_scale(x.v[a][b], w);
    return x;
}
template <int D>
__device__ __forceinline__ MDF<D> ndagdf(const MDF<D>& x) {  // -x^dagger
    MDF<D> r;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) r.v[a][b] = cdf_neg(cdf_conj(x.v[b][a]));
    return r;
}

template <int D>
__device__ Mat<D> q_tvdf(const NgWeights& W, const Grid& g, const HermVdf& G, const HermVdf& S, int n, int m, int kb) {
    const int k = W.k, T = g.ntau;
    const int64_t rowS = (int64_t)n * (T + 1);
    DMat<D> c2 = dzero<D>(), c3 = dzero<D>();
    if (m <= k) {
        for (int j = 0; j <= k; ++j) {
            MDF<D> gm = lddf<D>(G.mat, T - j, kb);
            for (int l = 0; l <= k; ++l) dfma_m<D>(c2, sdf<D>(W.R[m][j][l], lddf<D>(S.tv, rowS + l, kb)), gm);
        }
    } else {
        greg_for(W, m, m, [&](int l, double w) {
            dfma_m<D>(c2, sdf<D>(w, lddf<D>(S.tv, rowS + m - l, kb)), lddf<D>(G.mat, T - l, kb));
        });
    }
    if (m >= T - k) {
        for (int j = 0; j <= k; ++j) {
            MDF<D> gm = lddf<D>(G.mat, j, kb);
            for (int l = 0; l <= k; ++l) dfma_m<D>(c3, sdf<D>(W.R[T - m][j][l], lddf<D>(S.tv, rowS + T - l, kb)), gm);
        }
    } else {
        greg_for(W, T - m, T - m, [&](int l, double w) {
            dfma_m<D>(c3, sdf<D>(w, lddf<D>(S.tv, rowS + m + l, kb)), lddf<D>(G.mat, l, kb));
        });
    }
    Mat<D> v = madd<D>(mscal<D>((double)g.sig, dval<D>(c2)), dval<D>(c3));
    return mscal<D>(g.htau, mmuli<D>(mscal<D>(-1.0, v)));
}

template <int D>
__device__ __forceinline__ void ret_itemdf(const NgWeights& W, const Grid& g, const HermV& G, const HermVdf& Gd,
                                           const HermVdf& Sd, const Mat<D>& Minv, int n, int m, int kb, int* status) {
    const int L = n - m;
    DMat<D> acc = dzero<D>();
    const int64_t rowS = tri(n);
    greg_for(W, L, L - 1, [&](int l, double w) {
        dfma_m<D>(acc, sdf<D>(w, lddf<D>(Sd.ret, rowS + m + l, kb)), lddf<D>(Gd.ret, tri(m + l) + m, kb));
    });
    Mat<D> bdf = mzero<D>();
    for (int l = 1; l <= W.k; ++l) bdf = madd<D>(bdf, mscal<D>(W.a[l], gret<D>(G, n - l, m, kb)));
    Mat<D> rhs = msub<D>(mscal<D>(-1.0 / g.h, bdf), mscal<D>(g.h, mmuli<D>(dval<D>(acc))));
    Mat<D> y = mmul<D>(Minv, rhs);
    if (!mfinite<D>(y)) atomicOr(status, NGF_NONFINITE);
    st<D>(G.ret, tri(n) + m, kb, y);
}

template <int D>
__device__ __forceinline__ void tv_itemdf(const NgWeights& W, const Grid& g, const HermV& G, const HermV& S,
                                          const HermVdf& Gd, const HermVdf& Sd, const Mat<D>& Minv, int n, int m,
                                          int kb, const cplx* tvq, int* status) {
    DMat<D> acc = dzero<D>();
    const int64_t rowS = tri(n);
    const int T1 = g.ntau + 1;
    greg_for(W, n, n - 1, [&](int j, double w) {
        dfma_m<D>(acc, sdf<D>(w, lddf<D>(Sd.ret, rowS + j, kb)), lddf<D>(Gd.tv, (int64_t)j * T1 + m, kb));
    });
    Mat<D> bdf = mzero<D>();
    for (int l = 1; l <= W.k; ++l) bdf = madd<D>(bdf, mscal<D>(W.a[l], gtv<D>(G, g, n - l, m, kb)));
    Mat<D> rhs = tvq ? q_tv_fft<D>(W, g, G, S, n, m, kb, tvq) : q_tvdf<D>(W, g, Gd, Sd, n, m, kb);
    rhs = msub<D>(rhs, mscal<D>(1.0 / g.h, bdf));
    rhs = msub<D>(rhs, mscal<D>(g.h, mmuli<D>(dval<D>(acc))));
    Mat<D> y = mmul<D>(Minv, rhs);
    if (!mfinite<D>(y)) atomicOr(status, NGF_NONFINITE);
    st<D>(G.tv, (int64_t)n * T1 + m, kb, y);
}

template <int D>
__device__ __forceinline__ void les_itemdf(const NgWeights& W, const Grid& g, const HermV& G, const HermVdf& Gd,
                                           const HermVdf& Sd, const Mat<D>& Minv, int n, int m, int kb, int* status) {
    const int k = W.k, T = g.ntau, T1 = g.ntau + 1;
    const int64_t colS = tri(n);
    DMat<D> c1 = dzero<D>();
    if (m <= k) {
        for (int j = 0; j <= k; ++j) {
            MDF<D> gr = (j <= m) ? lddf<D>(Gd.ret, tri(m) + j, kb) : ndagdf<D>(lddf<D>(Gd.ret, tri(j) + m, kb));
            dfma_m<D>(c1, sdf<D>(W.greg[m][j], gr), lddf<D>(Sd.les, colS + j, kb));
        }
    } else {
        const int64_t rowG = tri(m);
        greg_for(W, m, m, [&](int j, double w) {
            dfma_m<D>(c1, sdf<D>(w, lddf<D>(Gd.ret, rowG + j, kb)), lddf<D>(Sd.les, colS + j, kb));
        });
    }
    DMat<D> c3 = dzero<D>();
    const int64_t rowGt = (int64_t)m * T1, rowSt = (int64_t)n * T1;
    greg_for(W, T, T, [&](int j, double w) {
        dfma_m_db<D>(c3, sdf<D>(w, lddf<D>(Gd.tv, rowGt + j, kb)), lddf<D>(Sd.tv, rowSt + T - j, kb));
    });
    Mat<D> q = msub<D>(mscal<D>(g.h, mmuli<D>(dval<D>(c1))), mscal<D>((double)g.sig * g.htau, dval<D>(c3)));
    DMat<D> hist = dzero<D>();
    const int64_t rowS = tri(n), colM = tri(m);
    greg_for(W, n, n - 1, [&](int l, double w) {
        MDF<D> gl = (l >= m) ? lddf<D>(Gd.les, tri(l) + m, kb) : ndagdf<D>(lddf<D>(Gd.les, colM + l, kb));
        dfma_m_db<D>(hist, sdf<D>(w, gl), lddf<D>(Sd.ret, rowS + l, kb));
    });
    Mat<D> bdf = mzero<D>();
    for (int l = 1; l <= k; ++l) bdf = madd<D>(bdf, mscal<D>(W.a[l], ld<D>(G.les, tri(n - l) + m, kb)));
    Mat<D> rhs = msub<D>(q, mscal<D>(1.0 / g.h, bdf));
    rhs = madd<D>(rhs, mscal<D>(g.h, mmuli<D>(dval<D>(hist))));
    Mat<D> y = mmul<D>(rhs, mdag<D>(Minv));
    if (!mfinite<D>(y)) atomicOr(status, NGF_NONFINITE);
    st<D>(G.les, tri(n) + m, kb, y);
}

template <int D>
__global__ void __launch_bounds__(128, D == 1 ? 6 : 1) k_step_bulkdf(Grid g, int n, HermV G, HermV S, HermVdf Gd, HermVdf Sd,
                                                     const cplx* minv_ws, int nb_les, int nb_tv, int nb_ret,
                                                     const cplx* tvq, int* status) {
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
    if (task == 0) les_itemdf<D>(W, g, G, Gd, Sd, Minv, n, (int)col + 1, kb, status);
    else if (task == 1) tv_itemdf<D>(W, g, G, S, Gd, Sd, Minv, n, (int)col, kb, tvq, status);
    else ret_itemdf<D>(W, g, G, Gd, Sd, Minv, n, (int)col, kb, status);
}

// double-float copies of slices [n0, n1] (mat when n0 = -1), layout as k_shadow
__global__ void k_shadow_df(Grid g, int n0, int n1, HermV X, HermVdf Y, int ldk) {
    const int dd = g.nf * g.nf;
    const int T1 = g.ntau + 1;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int a = n0 < 0 ? 0 : n0;
    const int64_t e_tri0 = tri(a), n_tri = tri(n1 + 1) - e_tri0;
    const int64_t n_tv = (int64_t)(n1 - a + 1) * T1;
    const int64_t n_mat = n0 < 0 ? T1 : 0;
    const int64_t per = (int64_t)dd * ldk;
    const int64_t tot = (2 * n_tri + n_tv + n_mat) * per;
    for (int64_t i = item; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t e = i / per, r = i % per;
        const cplx* src;
        float4* dst;
        int64_t off;
        if (e < n_tri) { off = (e_tri0 + e) * per + r; src = X.ret.p; dst = Y.ret.p; }
        else if ((e -= n_tri) < n_tri) { off = (e_tri0 + e) * per + r; src = X.les.p; dst = Y.les.p; }
        else if ((e -= n_tri) < n_tv) { off = ((int64_t)a * T1 + e) * per + r; src = X.tv.p; dst = Y.tv.p; }
        else { e -= n_tv; off = e * per + r; src = X.mat.p; dst = Y.mat.p; }
        const cplx v = src[off];
        const float rh = (float)v.x, ih = (float)v.y;
        dst[off] = make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
    }
}
