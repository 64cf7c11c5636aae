// Time-step bulk for small batches: one warp per (column, problem) item.
//
// The bulk items of a time step (Sec. "Time stepping": retarded (B) elements, the left-mixing
// row, lesser (B) elements) each carry O(n + ntau) history and source terms.  With one thread
// per item a batch of a few problems (a dimer, a real-space cluster) leaves almost every SM
// idle and each thread sums its terms serially.  Here the 32 lanes of a warp take the terms
// l = lane, lane + 32, ... of every sum of one item, with the item's Gregory weights; the lane
// partials are added by a fixed xor butterfly (every lane ends with the same, deterministic
// sum) and lane 0 finishes the item exactly as the one-thread kernel does: BDF terms, the
// left-mixing source (FFT correlation with its corrections, or the direct sums), the solve with
// M_n^-1 and the store.  The arithmetic is that of k_step_bulk up to the order of the additions.
#pragma once

#include "ng_step.cuh"

template <int D>
__device__ __forceinline__ Mat<D> warp_msum(Mat<D> x) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = 0; b < D; ++b) {
                x.v[a][b].x += __shfl_xor_sync(0xffffffffu, x.v[a][b].x, off);
                x.v[a][b].y += __shfl_xor_sync(0xffffffffu, x.v[a][b].y, off);
            }
    return x;
}

template <int D>
__device__ __forceinline__ void ret_item_w(const NgWeights& W, const Grid& g, const HermV& G, const HermV& S,
                                           const cplx* minv_ws, int n, int m, int kb, int lane, int* status) {
    const int L = n - m;  // > k
    Mat<D> acc = mzero<D>();
    for (int l = lane; l < L; l += 32)
        mfma<D>(acc, mscal<D>(gw(W, L, l), gret<D>(S, n, m + l, kb)), gret<D>(G, m + l, m, kb));
    acc = warp_msum<D>(acc);
    if (lane != 0) return;
    Mat<D> bdf = mzero<D>();
    for (int l = 1; l <= W.k; ++l) bdf = madd<D>(bdf, mscal<D>(W.a[l], gret<D>(G, n - l, m, kb)));
    Mat<D> rhs = msub<D>(mscal<D>(-1.0 / g.h, bdf), mscal<D>(g.h, mmuli<D>(acc)));
    Mat<D> y = mmul<D>(ld_minv<D>(minv_ws, kb), rhs);
    if (!mfinite<D>(y)) atomicOr(status, NGF_NONFINITE);
    st<D>(G.ret, tri(n) + m, kb, y);
}

template <int D>
__device__ __forceinline__ void tv_item_w(const NgWeights& W, const Grid& g, const HermV& G, const HermV& S,
                                          const cplx* minv_ws, int n, int m, int kb, const cplx* tvq, int lane,
                                          int* status) {
    Mat<D> acc = mzero<D>();
    for (int j = lane; j < n; j += 32)
        mfma<D>(acc, mscal<D>(gw(W, n, j), gret<D>(S, n, j, kb)), gtv<D>(G, g, j, m, kb));
    acc = warp_msum<D>(acc);
    if (lane != 0) return;
    Mat<D> bdf = mzero<D>();
    for (int l = 1; l <= W.k; ++l) bdf = madd<D>(bdf, mscal<D>(W.a[l], gtv<D>(G, g, n - l, m, kb)));
    Mat<D> rhs = tvq ? q_tv_fft<D>(W, g, G, S, n, m, kb, tvq) : q_tv<D>(W, g, G, S, n, m, kb);
    rhs = msub<D>(rhs, mscal<D>(1.0 / g.h, bdf));
    rhs = msub<D>(rhs, mscal<D>(g.h, mmuli<D>(acc)));
    Mat<D> y = mmul<D>(ld_minv<D>(minv_ws, kb), rhs);
    if (!mfinite<D>(y)) atomicOr(status, NGF_NONFINITE);
    st<D>(G.tv, (int64_t)n * (g.ntau + 1) + m, kb, y);
}

template <int D>
__device__ __forceinline__ void les_item_w(const NgWeights& W, const Grid& g, const HermV& G, const HermV& S,
                                           const cplx* minv_ws, int n, int m, int kb, int lane, int* status) {
    const int k = W.k, T = g.ntau;
    // C^<_1[G,1,Sigma](m,n) = int_0^{t_m} G^R(m,s) Sigma^<(s,n)
    Mat<D> c1 = mzero<D>();
    if (m <= k) {
        for (int j = lane; j <= k; j += 32)
            mfma<D>(c1, mscal<D>(W.greg[m][j], gretx<D>(G, m, j, kb)), ld<D>(S.les, tri(n) + j, kb));
    } else {
        for (int j = lane; j <= m; j += 32)
            mfma<D>(c1, mscal<D>(gw(W, m, j), gret<D>(G, m, j, kb)), ld<D>(S.les, tri(n) + j, kb));
    }
    // sum_j w_{T,j} G^tv(m,j) [Sigma^tv(n,T-j)]^dagger
    Mat<D> c3 = mzero<D>();
    for (int j = lane; j <= T; j += 32)
        mfma_db<D>(c3, mscal<D>(gw(W, T, j), gtv<D>(G, g, m, j, kb)), gtv<D>(S, g, n, T - j, kb));
    // history sum_{l<n} w_{n,l} G^<(m,l) [Sigma^R(n,l)]^dagger
    Mat<D> hist = mzero<D>();
    for (int l = lane; l < n; l += 32) {
        Mat<D> gl = (l >= m) ? ld<D>(G.les, tri(l) + m, kb) : mscal<D>(-1.0, mdag<D>(ld<D>(G.les, tri(m) + l, kb)));
        mfma_db<D>(hist, mscal<D>(gw(W, n, l), gl), gret<D>(S, n, l, kb));
    }
    c1 = warp_msum<D>(c1);
    c3 = warp_msum<D>(c3);
    hist = warp_msum<D>(hist);
    if (lane != 0) return;
    Mat<D> q = msub<D>(mscal<D>(g.h, mmuli<D>(c1)), mscal<D>((double)g.sig * g.htau, c3));
    Mat<D> bdf = mzero<D>();
    for (int l = 1; l <= k; ++l) bdf = madd<D>(bdf, mscal<D>(W.a[l], ld<D>(G.les, tri(n - l) + m, kb)));
    Mat<D> rhs = msub<D>(q, mscal<D>(1.0 / g.h, bdf));
    rhs = madd<D>(rhs, mscal<D>(g.h, mmuli<D>(hist)));
    Mat<D> y = mmul<D>(rhs, mdag<D>(ld_minv<D>(minv_ws, kb)));
    if (!mfinite<D>(y)) atomicOr(status, NGF_NONFINITE);
    st<D>(G.les, tri(n) + m, kb, y);
}

// One warp per item, items ordered as in k_step_bulk (lesser, left-mixing, retarded; problem
// fastest); w_les, w_tv, w_ret: the items of each task.
template <int D>
__global__ void __launch_bounds__(128, 1) k_step_bulk_w(Grid g, int n, HermV G, HermV S, const cplx* minv_ws,
                                                     int64_t w_les, int64_t w_tv, int64_t w_ret, const cplx* tvq,
                                                     int* status) {
    const NgWeights& W = c_W[g.k - 1];
    int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    int task;
    if (item < w_les) task = 0;
    else if ((item -= w_les) < w_tv) task = 1;
    else if ((item -= w_tv) < w_ret) task = 2;
    else return;
    const int kb = (int)(item % g.nb);
    const int col = (int)(item / g.nb);
    if (task == 0) les_item_w<D>(W, g, G, S, minv_ws, n, col + 1, kb, lane, status);
    else if (task == 1) tv_item_w<D>(W, g, G, S, minv_ws, n, col, kb, tvq, lane, status);
    else ret_item_w<D>(W, g, G, S, minv_ws, n, col, kb, lane, status);
}
