// Dyson equation in integral form, (1 + F) * G = Q (Sec. "vie2: Dyson equation in integral
// form", Sec. "Implementation: vie2"): start-up and time-step kernels for nf = 1, 2, 4.
//
// The Langreth rules give Volterra integral equations of the second kind (Eqs.
// vie2_langreth_r/_tv/_les) solved with the rules of Sec. "Volterra Integral equation of the
// second kind": start-up (Eq. MBCVSAMx01_start) and single steps (Eq. MBCVSAMx01_t, and
// Eq. MBCVSAMx01_cc)t for the conjugate form).  F need not be hermitian symmetric: its values
// outside the stored triangles come from Fcc = F^ddagger.  Q and G are hermitian.
//
// Time step n > k (conjugate (B) schedule of the lesser column):
//   retarded  G^R(n,n) = Q^R(n,n); every m < n a single explicit step: for n - m > k the
//             Gregory quadrature of Eq. cr1 over j = m..n, for n - m <= k the start-up
//             quadrature over the k+1 points n, .., n-k (earlier rows, continued past the
//             diagonal by -[G^R(m, n-j)]^dagger);
//   left-mixing one step per tau_m, kernel F^R, source Q^tv - (C^tv_2 + C^tv_3)[F, 1, G^M];
//   lesser    G^<(0,n) = -[G^tv(n,0)]^dagger (Eq. vie2_ini_les); for m = 1..n-1 the conjugate
//             step with kernel F^ddagger,A(l,n) = [F^R(n,l)]^dagger and source
//             Q^< - (C^<_1 + C^<_3)[G, 1, F^ddagger](m,n); finally m = n, whose history needs
//             G^<(n,l) = -[G^<(l,n)]^dagger of the column just computed.
#pragma once

#include "ng_step.cuh"
#include "ng_stepsplit.cuh"

// F~^R(n, l): stored for l <= n, continued by -[Fcc^R(l, n)]^dagger for l > n (Eq. Cretmod)
template <int D>
__device__ __forceinline__ Mat<D> v2_fretx(const HermV& F, const HermV& Fcc, int n, int l, int kb) {
    if (l <= n) return ld<D>(F.ret, tri(n) + l, kb);
    return mscal<D>(-1.0, mdag<D>(ld<D>(Fcc.ret, tri(l) + n, kb)));
}
// F^<(j, n) for any j, n: stored for j <= n, else -[Fcc^<(n, j)]^dagger
template <int D>
__device__ __forceinline__ Mat<D> v2_flesx(const HermV& F, const HermV& Fcc, int j, int n, int kb) {
    if (j <= n) return ld<D>(F.les, tri(n) + j, kb);
    return mscal<D>(-1.0, mdag<D>(ld<D>(Fcc.les, tri(j) + n, kb)));
}

// (C^tv_2 + C^tv_3)[F, 1, G^M](n, m): the Matsubara pieces of Eqs. ctv2, ctv3.  q_tv of the
// integro-differential step returns -i times this sum for a kernel in place of Sigma.
template <int D>
__device__ __forceinline__ Mat<D> v2_ctv23(const NgWeights& W, const Grid& g, const HermV& G, const HermV& F, int n,
                                           int m, int kb, const cplx* tvq) {
    // tvq: the unit-weight correlation of the FFT pre-pass (the quadrature's corrections added
    // here), else the direct sums
    return mmuli<D>(tvq ? q_tv_fft<D>(W, g, G, F, n, m, kb, tvq) : q_tv<D>(W, g, G, F, n, m, kb));
}

// (C^<_2 + C^<_3)[F, 1, G](m, n) (Eqs. cles2, cles3): h sum_j w_{n,j} F^<(m,j) G^A(j,n) with
// G^A(j,n) = [G~^R(n,j)]^dagger, plus i xi h_tau sum_j w_{T,j} F^tv(m,j) [G^tv(n, T-j)]^dagger
template <int D>
__device__ Mat<D> v2_cles23(const NgWeights& W, const Grid& g, const HermV& G, const HermV& F, const HermV& Fcc, int m,
                            int n, int kb) {
    const int k = W.k, T = g.ntau;
    Mat<D> c2 = mzero<D>(), c3 = mzero<D>();
    const int jmax = n > k ? n : k;
    for (int j = 0; j <= jmax; ++j)
        mfma_db<D>(c2, mscal<D>(gw(W, n, j), v2_flesx<D>(F, Fcc, m, j, kb)), gretx<D>(G, n, j, kb));
    greg_for(W, T, T, [&](int j, double w) {
        mfma_db<D>(c3, mscal<D>(w, gtv<D>(F, g, m, j, kb)), gtv<D>(G, g, n, T - j, kb));
    });
    return madd<D>(mscal<D>(g.h, c2), mcscal<D>(make_double2(0.0, (double)g.sig * g.htau), c3));
}

// M = 1 + c F, the matrix of a single step (c = h times the diagonal quadrature weight)
template <int D>
__device__ __forceinline__ Mat<D> v2_one_plus(double c, const Mat<D>& Fd) {
    Mat<D> M = mscal<D>(c, Fd);
#pragma unroll
    for (int a = 0; a < D; ++a) M.v[a][a].x += 1.0;
    return M;
}

// ---- time-step items ----------------------------------------------------------------------
// retarded G^R(n, m), m < n
template <int D>
__device__ __forceinline__ void v2_ret_item(const NgWeights& W, const Grid& g, const HermV& G, const HermV& F,
                                            const HermV& Q, int n, int m, int kb, int* status) {
    const int k = W.k, L = n - m;
    Mat<D> acc = mzero<D>();   // the known part of the quadrature
    double wd;                 // weight of the unknown term, j = n
    if (L > k) {
        greg_for(W, L, L - 1, [&](int l, double w) {
            mfma<D>(acc, mscal<D>(w, ld<D>(F.ret, tri(n) + m + l, kb)), gret<D>(G, m + l, m, kb));
        });
        wd = gw(W, L, L);
    } else {
        for (int j = 1; j <= k; ++j)
            mfma<D>(acc, mscal<D>(W.greg[L][j], ld<D>(F.ret, tri(n) + n - j, kb)), gretx<D>(G, n - j, m, kb));
        wd = W.greg[L][0];
    }
    int sing = 0;
    const Mat<D> Mi = minv<D>(v2_one_plus<D>(g.h * wd, ld<D>(F.ret, tri(n) + n, kb)), &sing);
    const Mat<D> y = mmul<D>(Mi, msub<D>(ld<D>(Q.ret, tri(n) + m, kb), mscal<D>(g.h, acc)));
    if (sing) atomicOr(status, NGF_SINGULAR);
    if (!mfinite<D>(y)) atomicOr(status, NGF_NONFINITE);
    st<D>(G.ret, tri(n) + m, kb, y);
}

// left-mixing G^tv(n, m)
template <int D>
__device__ __forceinline__ void v2_tv_item(const NgWeights& W, const Grid& g, const HermV& G, const HermV& F,
                                           const HermV& Q, int n, int m, int kb, const cplx* tvq, int* status) {
    Mat<D> acc = mzero<D>();
    greg_for(W, n, n - 1, [&](int j, double w) {
        mfma<D>(acc, mscal<D>(w, ld<D>(F.ret, tri(n) + j, kb)), gtv<D>(G, g, j, m, kb));
    });
    Mat<D> rhs = msub<D>(gtv<D>(Q, g, n, m, kb), v2_ctv23<D>(W, g, G, F, n, m, kb, tvq));
    rhs = msub<D>(rhs, mscal<D>(g.h, acc));
    int sing = 0;
    const Mat<D> y = mmul<D>(minv<D>(v2_one_plus<D>(g.h * gw(W, n, n), ld<D>(F.ret, tri(n) + n, kb)), &sing), rhs);
    if (sing) atomicOr(status, NGF_SINGULAR);
    if (!mfinite<D>(y)) atomicOr(status, NGF_NONFINITE);
    st<D>(G.tv, (int64_t)n * (g.ntau + 1) + m, kb, y);
}

// Partial sums of the conjugate lesser step's source and history for G^<(m, n), over the terms
// j0, j0 + js, ... of each sum (j0 = 0, js = 1: the whole sums):
//   c1   = sum_{j <= max(m,k)} w_{m,j} G~^R(m,j) Fcc^<(j,n)       (C^<_1[G,1,F^ddagger], no h)
//   c3   = sum_{j <= T} w_{T,j} G^tv(m,j) [F^tv(n, T-j)]^dagger   (C^<_3 = i xi h_tau c3)
//   hist = sum_{l < n} w_{n,l} G^<(m,l) [F^R(n,l)]^dagger
template <int D>
__device__ void v2_les_parts_strided(const NgWeights& W, const Grid& g, const HermV& G, const HermV& F,
                                     const HermV& Fcc, int n, int m, int kb, int j0, int js, Mat<D>& c1, Mat<D>& c3,
                                     Mat<D>& hist) {
    const int k = W.k, T = g.ntau;
    const int jm = m > k ? m : k;
    for (int j = j0; j <= jm; j += js)
        mfma<D>(c1, mscal<D>(gw(W, m, j), gretx<D>(G, m, j, kb)), ld<D>(Fcc.les, tri(n) + j, kb));
    for (int j = j0; j <= T; j += js)
        mfma_db<D>(c3, mscal<D>(gw(W, T, j), gtv<D>(G, g, m, j, kb)), gtv<D>(F, g, n, T - j, kb));
    for (int l = j0; l < n; l += js) {
        const Mat<D> gl = (l >= m) ? ld<D>(G.les, tri(l) + m, kb) : mscal<D>(-1.0, mdag<D>(ld<D>(G.les, tri(m) + l, kb)));
        mfma_db<D>(hist, mscal<D>(gw(W, n, l), gl), ld<D>(F.ret, tri(n) + l, kb));
    }
}

// The whole sums (one item per thread): the unit-weight middle of each Gregory quadrature runs
// without a weight multiply (greg_for), so the FP64 work per term is the complex product alone.
template <int D>
__device__ void v2_les_parts(const NgWeights& W, const Grid& g, const HermV& G, const HermV& F, const HermV& Fcc,
                             int n, int m, int kb, Mat<D>& c1, Mat<D>& c3, Mat<D>& hist) {
    const int k = W.k, T = g.ntau;
    if (m <= k) {
        for (int j = 0; j <= k; ++j)
            mfma<D>(c1, mscal<D>(W.greg[m][j], gretx<D>(G, m, j, kb)), ld<D>(Fcc.les, tri(n) + j, kb));
    } else {
        const int64_t rowG = tri(m), colF = tri(n);
        greg_for(W, m, m, [&](int j, double w) {
            mfma<D>(c1, mscal<D>(w, ld<D>(G.ret, rowG + j, kb)), ld<D>(Fcc.les, colF + j, kb));
        });
    }
    const int64_t rowGt = (int64_t)m * (T + 1), rowFt = (int64_t)n * (T + 1);
    greg_for(W, T, T, [&](int j, double w) {
        mfma_db<D>(c3, mscal<D>(w, ld<D>(G.tv, rowGt + j, kb)), ld<D>(F.tv, rowFt + T - j, kb));
    });
    const int64_t rowF = tri(n), colM = tri(m);
    greg_for(W, n, n - 1, [&](int l, double w) {
        const Mat<D> gl = (l >= m) ? ld<D>(G.les, tri(l) + m, kb) : mscal<D>(-1.0, mdag<D>(ld<D>(G.les, colM + l, kb)));
        mfma_db<D>(hist, mscal<D>(w, gl), ld<D>(F.ret, rowF + l, kb));
    });
}

// G^<(m,n) = [Q^<(m,n) - h c1 - i xi h_tau c3 - h hist] [1 + h w_{n,n} F^R(n,n)]^-dagger
template <int D>
__device__ __forceinline__ Mat<D> v2_les_solve(const NgWeights& W, const Grid& g, const HermV& F, const HermV& Q,
                                               int n, int m, int kb, const Mat<D>& c1, const Mat<D>& c3,
                                               const Mat<D>& hist, int* status) {
    Mat<D> rhs = msub<D>(ld<D>(Q.les, tri(n) + m, kb), mscal<D>(g.h, madd<D>(c1, hist)));
    rhs = msub<D>(rhs, mcscal<D>(make_double2(0.0, (double)g.sig * g.htau), c3));
    int sing = 0;
    const Mat<D> Mi = minv<D>(v2_one_plus<D>(g.h * gw(W, n, n), ld<D>(F.ret, tri(n) + n, kb)), &sing);
    if (sing) atomicOr(status, NGF_SINGULAR);
    return mmul<D>(rhs, mdag<D>(Mi));   // [M^dagger]^-1 = [M^-1]^dagger
}

// ---- the same items with one warp each (small batches): the lane partials of every sum are
// added by warp_rsum, which leaves element rs_elem(lane) of each sum on the lanes, and the item's
// closing solve runs one element per lane --------------------------------------------------------

// row i of [1 + c F^R(n,n)]^-1 on every lane of the warp (all lanes call it): by the adjugate for
// D <= 2; for D = 4 the warp solves M X = 1 in its scratch sh (2 D^2 + D values)
template <int D>
__device__ __forceinline__ void v2_inv_row(double c, const HermV& F, int n, int kb, int i, cplx (&row)[D], cplx* sh,
                                           int lane, int* status) {
    const int64_t e = tri(n) + n;
    auto mel = [&](int r, int q) {
        cplx x = cscal(c, elw(F.ret, e, r, q, D, kb));
        if (r == q) x.x += 1.0;
        return x;
    };
    if constexpr (D == 1) {
        const cplx m = mel(0, 0);
        if (cabs2(m) == 0.0 && lane == 0) atomicOr(status, NGF_SINGULAR);
        row[0] = cdiv(cr(1.0), m);
    } else if constexpr (D == 2) {
        const cplx p = mel(0, 0), q = mel(0, 1), r = mel(1, 0), t = mel(1, 1);
        const cplx det = csub(cmul(p, t), cmul(q, r));
        if (cabs2(det) == 0.0 && lane == 0) atomicOr(status, NGF_SINGULAR);
        const cplx idet = cdiv(cr(1.0), det);
        row[0] = cmul(i == 0 ? t : cneg(r), idet);
        row[1] = cmul(i == 0 ? cneg(q) : p, idet);
    } else {
        cplx* M = sh;
        cplx* X = sh + D * D;
        for (int x = lane; x < D * D; x += 32) {
            M[x] = mel(x / D, x % D);
            X[x] = cr(x / D == x % D ? 1.0 : 0.0);
        }
        __syncwarp();
        if (warp_dense_solve(M, D, X, D, sh + 2 * D * D, lane) && lane == 0) atomicOr(status, NGF_SINGULAR);
#pragma unroll
        for (int q = 0; q < D; ++q) row[q] = X[i * D + q];
        __syncwarp();
    }
}

template <int D>
__device__ __forceinline__ void v2_ret_item_w(const NgWeights& W, const Grid& g, const HermV& G, const HermV& F,
                                              const HermV& Q, int n, int m, int kb, int lane, cplx* sh, int* status) {
    const int k = W.k, L = n - m;
    Mat<D> acc = mzero<D>();
    double wd;
    if (L > k) {
        greg_for_lanes(W, L, L - 1, lane, [&](int l, double w) {
            mfma<D>(acc, mscal<D>(w, ld<D>(F.ret, tri(n) + m + l, kb)), gret<D>(G, m + l, m, kb));
        });
        wd = gw(W, L, L);
    } else {
        for (int j = 1 + lane; j <= k; j += 32)
            mfma<D>(acc, mscal<D>(W.greg[L][j], ld<D>(F.ret, tri(n) + n - j, kb)), gretx<D>(G, n - j, m, kb));
        wd = W.greg[L][0];
    }
    // y = [1 + h wd F^R(n,n)]^-1 (Q^R(n,m) - h acc), element (a, b) per lane
    const cplx ae = warp_rsum<D>(acc, lane);
    const int e = rs_elem<D>(lane), a = e / D, b = e % D;
    const cplx rhs = csub(elw(Q.ret, tri(n) + m, a, b, D, kb), cscal(g.h, ae));
    cplx mi[D];
    v2_inv_row<D>(g.h * wd, F, n, kb, a, mi, sh, lane, status);
    cplx y = cz();
#pragma unroll
    for (int c = 0; c < D; ++c) y = cfma(mi[c], rs_get<D>(rhs, c * D + b), y);
    if (rs_leader<D>(lane)) {
        if (!cfinite(y)) atomicOr(status, NGF_NONFINITE);
        G.ret.p[((tri(n) + m) * (D * D) + a * D + b) * G.ret.ldk + (G.ret.ldk == 1 ? 0 : kb)] = y;
    }
}

// the left-mixing item; its source (C^tv_2 + C^tv_3)[F, 1, G^M] = i q_tv with S := F is split over
// the lanes (no FFT pre-pass in this form)
template <int D>
__device__ __forceinline__ void v2_tv_item_w(const NgWeights& W, const Grid& g, const HermV& G, const HermV& F,
                                             const HermV& Q, int n, int m, int kb, int lane, cplx* sh, int* status) {
    Mat<D> acc = mzero<D>();
    greg_for_lanes(W, n, n - 1, lane, [&](int j, double w) {
        mfma<D>(acc, mscal<D>(w, ld<D>(F.ret, tri(n) + j, kb)), gtv<D>(G, g, j, m, kb));
    });
    // y = [1 + h w_{n,n} F^R(n,n)]^-1 (Q^tv(n,m) - i src - h acc), element (a, b) per lane
    const cplx ae = warp_rsum<D>(acc, lane);
    const cplx se = warp_rsum<D>(q_tv_part<D>(W, g, G, F, n, m, kb, lane), lane);
    const int e = rs_elem<D>(lane), a = e / D, b = e % D;
    cplx rhs = csub(elw(Q.tv, (int64_t)n * (g.ntau + 1) + m, a, b, D, kb), cmuli(se));
    rhs = csub(rhs, cscal(g.h, ae));
    cplx mi[D];
    v2_inv_row<D>(g.h * gw(W, n, n), F, n, kb, a, mi, sh, lane, status);
    cplx y = cz();
#pragma unroll
    for (int c = 0; c < D; ++c) y = cfma(mi[c], rs_get<D>(rhs, c * D + b), y);
    if (rs_leader<D>(lane)) {
        if (!cfinite(y)) atomicOr(status, NGF_NONFINITE);
        G.tv.p[(((int64_t)n * (g.ntau + 1) + m) * (D * D) + a * D + b) * G.tv.ldk + (G.tv.ldk == 1 ? 0 : kb)] = y;
    }
}

// the conjugate lesser item: y = [Q^<(m,n) - h (c1 + hist) - i xi h_tau c3] [1 + h w_{n,n} F^R(n,n)]^-dagger
template <int D>
__device__ __forceinline__ void v2_les_item_w(const NgWeights& W, const Grid& g, const HermV& G, const HermV& F,
                                              const HermV& Fcc, const HermV& Q, int n, int m, int kb, int lane,
                                              cplx* sh, int* status) {
    Mat<D> c1 = mzero<D>(), c3 = mzero<D>(), hist = mzero<D>();
    v2_les_parts_strided<D>(W, g, G, F, Fcc, n, m, kb, lane, 32, c1, c3, hist);
    const cplx c1e = warp_rsum<D>(c1, lane), c3e = warp_rsum<D>(c3, lane), he = warp_rsum<D>(hist, lane);
    const int e = rs_elem<D>(lane), a = e / D, b = e % D;
    cplx rhs = csub(elw(Q.les, tri(n) + m, a, b, D, kb), cscal(g.h, cadd(c1e, he)));
    rhs = csub(rhs, cmul(make_double2(0.0, (double)g.sig * g.htau), c3e));
    cplx mi[D];   // row b of M^-1: y_ab = sum_c rhs_ac conj(M^-1_bc)
    v2_inv_row<D>(g.h * gw(W, n, n), F, n, kb, b, mi, sh, lane, status);
    cplx y = cz();
#pragma unroll
    for (int c = 0; c < D; ++c) y = cfma(rs_get<D>(rhs, a * D + c), cconj(mi[c]), y);
    if (rs_leader<D>(lane)) {
        if (!cfinite(y)) atomicOr(status, NGF_NONFINITE);
        G.les.p[((tri(n) + m) * (D * D) + a * D + b) * G.les.ldk + (G.les.ldk == 1 ? 0 : kb)] = y;
    }
}

template <int D>
__global__ void __launch_bounds__(128, 1)
    k_v2_bulk_w(Grid g, int n, HermV G, HermV F, HermV Fcc, HermV Q, int64_t w_les, int64_t w_tv, int64_t w_ret,
                int* status) {
    const NgWeights& W = c_W[g.k - 1];
    __shared__ cplx sh[4][D <= 2 ? 1 : 2 * D * D + D];   // blockDim.x = 128: four warps
    int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    cplx* ws = sh[threadIdx.x >> 5];
    int task;
    if (item < w_les) task = 0;
    else if ((item -= w_les) < w_tv) task = 1;
    else if ((item -= w_tv) < w_ret) task = 2;
    else return;
    const int kb = (int)(item % g.nb), col = (int)(item / g.nb);
    if (task == 1) v2_tv_item_w<D>(W, g, G, F, Q, n, col, kb, lane, ws, status);
    else if (task == 2) v2_ret_item_w<D>(W, g, G, F, Q, n, col, kb, lane, ws, status);
    else v2_les_item_w<D>(W, g, G, F, Fcc, Q, n, col + 1, kb, lane, ws, status);
}

// Time step n: one launch over the retarded items (m = 0..n-1), the left-mixing items
// (m = 0..ntau) and the lesser items (m = 1..n-1); (column, problem) items, problem fastest.
template <int D>
__global__ void __launch_bounds__(128, D == 1 ? 6 : 1)
    k_v2_bulk(Grid g, int n, HermV G, HermV F, HermV Fcc, HermV Q, int nb_ret, int nb_tv, int nb_les, const cplx* tvq,
              int* status) {
    const NgWeights& W = c_W[g.k - 1];
    int blk = blockIdx.x, task;
    if (blk < nb_les) task = 0;
    else if ((blk -= nb_les) < nb_tv) task = 1;
    else { blk -= nb_tv; task = 2; }
    const int64_t item = (int64_t)blk * blockDim.x + threadIdx.x;
    const int kb = (int)(item % g.nb);
    const int64_t col = item / g.nb;
    const int ncol = task == 0 ? n - 1 : (task == 1 ? g.ntau + 1 : n);
    if (col >= ncol) return;
    if (task == 1) {
        v2_tv_item<D>(W, g, G, F, Q, n, (int)col, kb, tvq, status);
    } else if (task == 2) {
        v2_ret_item<D>(W, g, G, F, Q, n, (int)col, kb, status);
    } else {
        const int m = (int)col + 1;
        Mat<D> c1 = mzero<D>(), c3 = mzero<D>(), hist = mzero<D>();
        v2_les_parts<D>(W, g, G, F, Fcc, n, m, kb, c1, c3, hist);
        const Mat<D> y = v2_les_solve<D>(W, g, F, Q, n, m, kb, c1, c3, hist, status);
        if (!mfinite<D>(y)) atomicOr(status, NGF_NONFINITE);
        st<D>(G.les, tri(n) + m, kb, y);
    }
}

// After the bulk launch, one block per problem: G^R(n,n) = Q^R(n,n), G^<(0,n) from G^tv(n,0),
// then the conjugate step for m = n (its history reads the column just computed), its sums as
// block reductions in a fixed order.
template <int D>
__global__ void __launch_bounds__(NG_BND_THREADS) k_v2_diag(Grid g, int n, HermV G, HermV F, HermV Fcc, HermV Q,
                                                             int* status) {
    const NgWeights& W = c_W[g.k - 1];
    const int kb = blockIdx.x, t = threadIdx.x;
    __shared__ cplx red[NG_BND_THREADS * D * D];
    if (t == 0) {
        st<D>(G.ret, tri(n) + n, kb, ld<D>(Q.ret, tri(n) + n, kb));
        st<D>(G.les, tri(n) + 0, kb, mscal<D>(-1.0, mdag<D>(gtv<D>(G, g, n, 0, kb))));
    }
    __syncthreads();
    Mat<D> c1 = mzero<D>(), c3 = mzero<D>(), hist = mzero<D>();
    v2_les_parts_strided<D>(W, g, G, F, Fcc, n, n, kb, t, blockDim.x, c1, c3, hist);
    c1 = block_sum<D>(c1, red);
    c3 = block_sum<D>(c3, red);
    hist = block_sum<D>(hist, red);
    if (t == 0) {
        const Mat<D> y = v2_les_solve<D>(W, g, F, Q, n, n, kb, c1, c3, hist, status);
        if (!mfinite<D>(y)) atomicOr(status, NGF_NONFINITE);
        st<D>(G.les, tri(n) + n, kb, y);
    }
}

// ---- start-up, slices 0..k (Sec. "Implementation: vie2", Start) -------------------------------
// One thread per problem: the retarded column systems for m = 0..k,
//   sum_l M_{n,l} y_l = Q^R(n,m), M_{n,l} = delta_{nl} + h I_{m,n;l} F~^R(n,l), n = m+1..k,
// with y_l = -[G^R(m,l)]^dagger (l < m) and y_m = Q^R(m,m) known; then the VIE start-up matrix
// M_{n,l} = delta_{nl} + h s_{n,l} F~^R(n,l) (Eq. MBCVSAMx01_start) shared by the left-mixing and
// lesser start-up: the workspace receives inv(M[1..k][1..k]) (kD x kD) and the blocks M[n][0].
template <int D>
__global__ void k_v2_start_ret(Grid g, HermV G, HermV F, HermV Fcc, HermV Q, cplx* ws, int* status) {
    const NgWeights& W = c_W[g.k - 1];
    const int kb = blockIdx.x * blockDim.x + threadIdx.x;
    if (kb >= g.nb) return;
    const int k = W.k, N = k * D;
    cplx A[(NG_KMAX * D) * (NG_KMAX * D)];
    cplx B[(NG_KMAX * D) * (NG_KMAX * D)];
    for (int m = 0; m <= k; ++m) {
        Mat<D> y[NG_KMAX + 1];
        for (int l = 0; l < m; ++l) y[l] = mscal<D>(-1.0, mdag<D>(gret<D>(G, m, l, kb)));
        y[m] = ld<D>(Q.ret, tri(m) + m, kb);
        if (m < k) {
            const int nu = (k - m) * D;
            for (int n = m + 1; n <= k; ++n) {
                Mat<D> rhs = ld<D>(Q.ret, tri(n) + m, kb);
                for (int l = 0; l <= k; ++l) {
                    Mat<D> M = mscal<D>(g.h * W.I[m][n][l], v2_fretx<D>(F, Fcc, n, l, kb));
                    if (l == n)
                        for (int a = 0; a < D; ++a) M.v[a][a].x += 1.0;
                    if (l <= m) rhs = msub<D>(rhs, mmul<D>(M, y[l]));
                    else
                        for (int a = 0; a < D; ++a)
                            for (int b = 0; b < D; ++b) A[((n - m - 1) * D + a) * nu + (l - m - 1) * D + b] = M.v[a][b];
                }
                for (int a = 0; a < D; ++a)
                    for (int c = 0; c < D; ++c) B[((n - m - 1) * D + a) * D + c] = rhs.v[a][c];
            }
            if (dense_solve(A, nu, B, D)) atomicOr(status, NGF_SINGULAR);
            for (int n = m + 1; n <= k; ++n)
                for (int a = 0; a < D; ++a)
                    for (int c = 0; c < D; ++c) y[n].v[a][c] = B[((n - m - 1) * D + a) * D + c];
        }
        for (int n = m; n <= k; ++n) {
            if (!mfinite<D>(y[n])) atomicOr(status, NGF_NONFINITE);
            st<D>(G.ret, tri(n) + m, kb, y[n]);
        }
    }
    cplx* dst = ws + (int64_t)kb * (N * N + k * D * D);
    for (int n = 1; n <= k; ++n)
        for (int l = 0; l <= k; ++l) {
            Mat<D> M = mscal<D>(g.h * W.greg[n][l], v2_fretx<D>(F, Fcc, n, l, kb));
            if (l == n)
                for (int a = 0; a < D; ++a) M.v[a][a].x += 1.0;
            for (int a = 0; a < D; ++a)
                for (int b = 0; b < D; ++b) {
                    if (l == 0) dst[N * N + (n - 1) * D * D + a * D + b] = M.v[a][b];
                    else A[((n - 1) * D + a) * N + (l - 1) * D + b] = M.v[a][b];
                }
        }
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) B[i * N + j] = cr(i == j ? 1.0 : 0.0);
    if (dense_solve(A, N, B, N)) atomicOr(status, NGF_SINGULAR);
    for (int i = 0; i < N * N; ++i) dst[i] = B[i];
}

// y_n = sum_l inv(M)[n][l] (q_l - M[l][0] y_0), n = 1..k, from the workspace of k_v2_start_ret
template <int D>
__device__ void v2_start_apply(const cplx* ws, int k, const Mat<D>* q, const Mat<D>& y0, Mat<D>* y) {
    const int N = k * D;
    Mat<D> r[NG_KMAX];
    for (int l = 0; l < k; ++l) {
        Mat<D> M0;
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b) M0.v[a][b] = ws[N * N + l * D * D + a * D + b];
        r[l] = msub<D>(q[l], mmul<D>(M0, y0));
    }
    for (int n = 0; n < k; ++n) {
        Mat<D> acc = mzero<D>();
        for (int l = 0; l < k; ++l) {
            Mat<D> Mi;
            for (int a = 0; a < D; ++a)
                for (int b = 0; b < D; ++b) Mi.v[a][b] = ws[(n * D + a) * N + l * D + b];
            mfma<D>(acc, Mi, r[l]);
        }
        y[n] = acc;
    }
}

// left-mixing slices 1..k per (tau_m, problem): y_0 = i xi G^M(beta - tau_m) (Eq. vie2_ini_tv),
// sources Q^tv(n,m) - (C^tv_2 + C^tv_3)[F, 1, G^M](n,m)
template <int D>
__global__ void k_v2_start_tv(Grid g, HermV G, HermV F, HermV Q, const cplx* ws, int* status) {
    const NgWeights& W = c_W[g.k - 1];
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= (int64_t)(g.ntau + 1) * g.nb) return;
    const int kb = (int)(item % g.nb), m = (int)(item / g.nb);
    const int k = W.k, N = k * D;
    const Mat<D> y0 = mcscal<D>(make_double2(0.0, (double)g.sig), gmat<D>(G, g.ntau - m, kb));
    Mat<D> q[NG_KMAX], y[NG_KMAX];
    for (int n = 1; n <= k; ++n) q[n - 1] = msub<D>(gtv<D>(Q, g, n, m, kb), v2_ctv23<D>(W, g, G, F, n, m, kb, nullptr));
    v2_start_apply<D>(ws + (int64_t)kb * (N * N + k * D * D), k, q, y0, y);
    st<D>(G.tv, m, kb, y0);
    for (int n = 1; n <= k; ++n) {
        if (!mfinite<D>(y[n - 1])) atomicOr(status, NGF_NONFINITE);
        st<D>(G.tv, (int64_t)n * (g.ntau + 1) + m, kb, y[n - 1]);
    }
}

// lesser columns n = 0..k per (n, problem): y_0 = -[G^tv(n,0)]^dagger, sources
// Q^<(m,n) - (C^<_2 + C^<_3)[F, 1, G](m,n) for m = 1..k (Q^<(m,n) = -[Q^<(n,m)]^dagger for
// m > n); rows m <= n are stored
template <int D>
__global__ void k_v2_start_les(Grid g, HermV G, HermV F, HermV Fcc, HermV Q, const cplx* ws, int* status) {
    const NgWeights& W = c_W[g.k - 1];
    const int k = W.k, N = k * D;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= (int64_t)(k + 1) * g.nb) return;
    const int kb = (int)(item % g.nb), n = (int)(item / g.nb);
    const Mat<D> y0 = mscal<D>(-1.0, mdag<D>(gtv<D>(G, g, n, 0, kb)));
    Mat<D> q[NG_KMAX], y[NG_KMAX];
    for (int m = 1; m <= k; ++m) q[m - 1] = msub<D>(gles<D>(Q, m, n, kb), v2_cles23<D>(W, g, G, F, Fcc, m, n, kb));
    v2_start_apply<D>(ws + (int64_t)kb * (N * N + k * D * D), k, q, y0, y);
    st<D>(G.les, tri(n) + 0, kb, y0);
    for (int m = 1; m <= n; ++m) {
        if (!mfinite<D>(y[m - 1])) atomicOr(status, NGF_NONFINITE);
        st<D>(G.les, tri(n) + m, kb, y[m - 1]);
    }
}
