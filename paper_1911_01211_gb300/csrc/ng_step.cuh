// Time-step kernels of libng: slice n > k of G for a batch of problems (mixed schedule, and
// the serial one in k_step_serial).
//
// Sec. "Time stepping" of the NESSi paper:
//   retarded row   : (B) single VIDE steps for columns m <= n-k-1 (Eq. MBCVSAMx_t with
//                    y(t) = G^R(mh+t, mh), kernel i Sigma^R), (A) conjugate start-up for
//                    m = n-k..n (Eq. MBCVSAMx_cc_start along the row);
//   left-mixing row: one VIDE step per tau_m (Eq. dyson_langreth_tv), source
//                    -i (C^tv_2 + C^tv_3)[Sigma, 1, G^M] (Eqs. ctv2, ctv3);
//   lesser column  : (B) conjugate single steps for 1 <= m <= n-k-1 (Eq. MBCVSAMx_cc_t with
//                    y(t) = G^<(mh, t), kernel -i Sigma^A, source i (C^<_1 + C^<_3)[G,1,Sigma]),
//                    G^<(0,n) from Eq. dyson_ini_les, then serial VIDE steps (A) for
//                    m = n-k..n (source -i (C^<_2 + C^<_3)[Sigma,1,G]); the whole column by
//                    (A) when n <= 2k.
// All steps with implementation (B) and the left-mixing row share
//   M_n = a_0/h + i(eps_n - mu) + h w_{n,n} i Sigma^R(n,n).
#pragma once

#include "ng_common.cuh"


// calls f(l, w_{L,l}) for l = 0..lmax (lmax <= L), for a Gregory row L > k
template <class F>
__device__ __forceinline__ void greg_for(const NgWeights& W, int L, int lmax, F&& f) {
    const int k = W.k;
    if (L <= 2 * k + 1) {
        for (int l = 0; l <= lmax; ++l) f(l, W.greg[L][l]);
        return;
    }
    const int e1 = min(k, lmax);
    for (int l = 0; l <= e1; ++l) f(l, W.omega[l]);
    const int e2 = min(L - k - 1, lmax);
#pragma unroll 4
    for (int l = k + 1; l <= e2; ++l) f(l, 1.0);
    for (int l = L - k; l <= lmax; ++l) f(l, W.omega[L - l]);
}

// acc += x * y^dagger
template <int D>
__device__ __forceinline__ void mfma_db(Mat<D>& acc, const Mat<D>& x, const Mat<D>& y) {
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
            for (int b = 0; b < D; ++b) acc.v[a][b] = cfma(x.v[a][c], cconj(y.v[b][c]), acc.v[a][b]);
}

template <int D>
__device__ __forceinline__ Mat<D> step_matrix(const NgWeights& W, const Grid& g, const HermV& S,
                                              const FuncV& eps, int n, int kb) {
    Mat<D> e = ldf<D>(eps, n, kb);
    Mat<D> M = meye<D>(cr(W.a[0] / g.h));
#pragma unroll
    for (int a = 0; a < D; ++a) e.v[a][a].x -= g.mu;
    M = madd<D>(M, mmuli<D>(e));
    M = madd<D>(M, mscal<D>(g.h * gw(W, n, n), mmuli<D>(gret<D>(S, n, n, kb))));
    return M;
}

// -i (C^tv_2 + C^tv_3)[Sigma, 1, G^M](n, m)   (Eqs. ctv2, ctv3)
template <int D>
__device__ Mat<D> q_tv(const NgWeights& W, const Grid& g, const HermV& G, const HermV& S, int n, int m,
                       int kb) {
    const int k = W.k, T = g.ntau;
    const double xi = (double)g.sig;
    Mat<D> c2 = mzero<D>(), c3 = mzero<D>();
    if (m <= k) {
        for (int j = 0; j <= k; ++j) {
            Mat<D> gm = mscal<D>(xi, gmat<D>(G, T - j, kb));
            for (int l = 0; l <= k; ++l) {
                Mat<D> s = mscal<D>(W.R[m][j][l], gtv<D>(S, g, n, l, kb));
                mfma<D>(c2, s, gm);
            }
        }
    } else {
        greg_for(W, m, m, [&](int l, double w) {
            mfma<D>(c2, mscal<D>(w, gtv<D>(S, g, n, m - l, kb)), gmat<D>(G, T - l, kb));
        });
        c2 = mscal<D>(xi, c2);
    }
    if (m >= T - k) {
        for (int j = 0; j <= k; ++j) {
            Mat<D> gm = gmat<D>(G, j, kb);
            for (int l = 0; l <= k; ++l) {
                Mat<D> s = mscal<D>(W.R[T - m][j][l], gtv<D>(S, g, n, T - l, kb));
                mfma<D>(c3, s, gm);
            }
        }
    } else {
        greg_for(W, T - m, T - m, [&](int l, double w) {
            mfma<D>(c3, mscal<D>(w, gtv<D>(S, g, n, m + l, kb)), gmat<D>(G, l, kb));
        });
    }
    return mscal<D>(g.htau, mmuli<D>(mscal<D>(-1.0, madd<D>(c2, c3))));
}

// The same source from the unit-weight correlation F(m) of the FFT pre-pass (ng_tvfft.cu):
// q(m) = -i h_tau [F(m) + the difference between the quadrature of Eqs. ctv2, ctv3 and unit
// weights], i.e. (w - 1) terms at the Gregory ends of each piece (rows longer than 2k+1), every
// term of short rows, and the boundary (R) formulas minus their unit-weight sums for m <= k and
// m >= ntau - k.  Q: [m][a][b][kb] with ldk = nb.
template <int D>
__device__ Mat<D> q_tv_fft(const NgWeights& W, const Grid& g, const HermV& G, const HermV& S, int n, int m, int kb,
                           const cplx* Q) {
    const int k = W.k, T = g.ntau;
    const double xi = (double)g.sig;
    Mat<D> c2 = mzero<D>(), c3 = mzero<D>();   // corrections, C2 without its factor xi
    // C2: sum_l w_{m,l} S(m-l) G^M(T-l)
    auto t2 = [&](int l, double dw) { mfma<D>(c2, mscal<D>(dw, gtv<D>(S, g, n, m - l, kb)), gmat<D>(G, T - l, kb)); };
    if (m <= k) {
        for (int j = 0; j <= k; ++j) {
            Mat<D> gm = gmat<D>(G, T - j, kb);
            for (int l = 0; l <= k; ++l) mfma<D>(c2, mscal<D>(W.R[m][j][l], gtv<D>(S, g, n, l, kb)), gm);
        }
        for (int l = 0; l <= m; ++l) t2(l, -1.0);
    } else if (m <= 2 * k + 1) {
        for (int l = 0; l <= m; ++l) t2(l, W.greg[m][l] - 1.0);
    } else {
        for (int l = 0; l <= k; ++l) t2(l, W.omega[l] - 1.0);
        for (int l = m - k; l <= m; ++l) t2(l, W.omega[m - l] - 1.0);
    }
    // C3: sum_l w_{T-m,l} S(m+l) G^M(l)
    const int L3 = T - m;
    auto t3 = [&](int l, double dw) { mfma<D>(c3, mscal<D>(dw, gtv<D>(S, g, n, m + l, kb)), gmat<D>(G, l, kb)); };
    if (L3 <= k) {
        for (int j = 0; j <= k; ++j) {
            Mat<D> gm = gmat<D>(G, j, kb);
            for (int l = 0; l <= k; ++l) mfma<D>(c3, mscal<D>(W.R[L3][j][l], gtv<D>(S, g, n, T - l, kb)), gm);
        }
        for (int l = 0; l <= L3; ++l) t3(l, -1.0);
    } else if (L3 <= 2 * k + 1) {
        for (int l = 0; l <= L3; ++l) t3(l, W.greg[L3][l] - 1.0);
    } else {
        for (int l = 0; l <= k; ++l) t3(l, W.omega[l] - 1.0);
        for (int l = L3 - k; l <= L3; ++l) t3(l, W.omega[L3 - l] - 1.0);
    }
    Mat<D> F;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) F.v[a][b] = Q[((int64_t)m * (D * D) + a * D + b) * g.nb + kb];
    Mat<D> v = madd<D>(F, madd<D>(mscal<D>(xi, c2), c3));
    return mscal<D>(g.htau, mmuli<D>(mscal<D>(-1.0, v)));
}

// Partial sums of the (A)-source of the lesser column, -i (C^<_2 + C^<_3)[Sigma,1,G](m,n)
// (Eqs. cles2, cles3), over the terms j = j0, j0+js, ...  (j0 = 0, js = 1 for the full sum).
template <int D>
__device__ Mat<D> q_lesA_part(const NgWeights& W, const Grid& g, const HermV& G, const HermV& S, int m,
                              int n, int kb, int j0, int js) {
    const int k = W.k, T = g.ntau;
    Mat<D> c2 = mzero<D>(), c3 = mzero<D>();
    if (n <= k) {
        // s weights over j = 0..k with G~^A(j,n) = [G~^R(n,j)]^dagger
        for (int j = j0; j <= k; j += js)
            mfma_db<D>(c2, mscal<D>(W.greg[n][j], gles<D>(S, m, j, kb)), gretx<D>(G, n, j, kb));
    } else {
        for (int j = j0; j <= n; j += js)
            mfma_db<D>(c2, mscal<D>(gw(W, n, j), gles<D>(S, m, j, kb)), gret<D>(G, n, j, kb));
    }
    for (int j = j0; j <= T; j += js)   // Sigma^tv(m,j) G^vt(j,n), G^vt = -xi [G^tv(n, T-j)]^dag
        mfma_db<D>(c3, mscal<D>(gw(W, T, j), gtv<D>(S, g, m, j, kb)), gtv<D>(G, g, n, T - j, kb));
    // -i [h c2 - i htau (-xi) c3] = -i h c2 + xi htau c3
    return madd<D>(mscal<D>(g.h, mmuli<D>(mscal<D>(-1.0, c2))), mscal<D>((double)g.sig * g.htau, c3));
}

// ----------------------------------------------------------------------------------------
// bulk items
// ----------------------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void ret_item(const NgWeights& W, const Grid& g, const HermV& G, const HermV& S,
                                         const Mat<D>& Minv, int n, int m, int kb, int* status) {
    const int L = n - m;  // > k
    Mat<D> acc = mzero<D>();
    greg_for(W, L, L - 1, [&](int l, double w) {
        mfma<D>(acc, mscal<D>(w, gret<D>(S, n, m + l, kb)), gret<D>(G, m + l, m, kb));
    });
    Mat<D> bdf = mzero<D>();
    for (int l = 1; l <= W.k; ++l) bdf = madd<D>(bdf, mscal<D>(W.a[l], gret<D>(G, n - l, m, kb)));
    Mat<D> rhs = msub<D>(mscal<D>(-1.0 / g.h, bdf), mscal<D>(g.h, mmuli<D>(acc)));
    Mat<D> y = mmul<D>(Minv, rhs);
    if (!mfinite<D>(y)) atomicOr(status, NGF_NONFINITE);
    st<D>(G.ret, tri(n) + m, kb, y);
}

template <int D>
__device__ __forceinline__ void tv_item(const NgWeights& W, const Grid& g, const HermV& G, const HermV& S,
                                        const Mat<D>& Minv, int n, int m, int kb, const cplx* tvq, int* status) {
    Mat<D> acc = mzero<D>();
    greg_for(W, n, n - 1, [&](int j, double w) {
        mfma<D>(acc, mscal<D>(w, gret<D>(S, n, j, kb)), gtv<D>(G, g, j, m, kb));
    });
    Mat<D> bdf = mzero<D>();
    for (int l = 1; l <= W.k; ++l) bdf = madd<D>(bdf, mscal<D>(W.a[l], gtv<D>(G, g, n - l, m, kb)));
    Mat<D> rhs = tvq ? q_tv_fft<D>(W, g, G, S, n, m, kb, tvq) : q_tv<D>(W, g, G, S, n, m, kb);
    rhs = msub<D>(rhs, mscal<D>(1.0 / g.h, bdf));
    rhs = msub<D>(rhs, mscal<D>(g.h, mmuli<D>(acc)));
    Mat<D> y = mmul<D>(Minv, rhs);
    if (!mfinite<D>(y)) atomicOr(status, NGF_NONFINITE);
    st<D>(G.tv, (int64_t)n * (g.ntau + 1) + m, kb, y);
}

template <int D>
__device__ __forceinline__ void les_item(const NgWeights& W, const Grid& g, const HermV& G, const HermV& S,
                                         const Mat<D>& Minv, int n, int m, int kb, int* status) {
    const int k = W.k, T = g.ntau;
    // C^<_1[G,1,Sigma](m,n) = int_0^{t_m} G^R(m,s) Sigma^<(s,n)
    Mat<D> c1 = mzero<D>();
    if (m <= k) {
        for (int j = 0; j <= k; ++j)
            mfma<D>(c1, mscal<D>(W.greg[m][j], gretx<D>(G, m, j, kb)), ld<D>(S.les, tri(n) + j, kb));
    } else {
        greg_for(W, m, m, [&](int j, double w) {
            mfma<D>(c1, mscal<D>(w, gret<D>(G, m, j, kb)), ld<D>(S.les, tri(n) + j, kb));
        });
    }
    // sum_j w_{T,j} G^tv(m,j) [Sigma^tv(n,T-j)]^dagger ;  C^<_3 = -i htau (-xi) * that
    Mat<D> c3 = mzero<D>();
    greg_for(W, T, T, [&](int j, double w) {
        mfma_db<D>(c3, mscal<D>(w, gtv<D>(G, g, m, j, kb)), gtv<D>(S, g, n, T - j, kb));
    });
    // source q = i (C1 + C3) = i h c1 + i (-i htau)(-xi) c3 = i h c1 - xi htau c3
    Mat<D> q = msub<D>(mscal<D>(g.h, mmuli<D>(c1)), mscal<D>((double)g.sig * g.htau, c3));
    // history sum_{l<n} w_{n,l} G^<(m,l) [Sigma^R(n,l)]^dagger  (kernel -i Sigma^A(l,n))
    Mat<D> hist = mzero<D>();
    greg_for(W, n, n - 1, [&](int l, double w) {
        Mat<D> gl = (l >= m) ? ld<D>(G.les, tri(l) + m, kb)
                             : mscal<D>(-1.0, mdag<D>(ld<D>(G.les, tri(m) + l, kb)));
        mfma_db<D>(hist, mscal<D>(w, gl), gret<D>(S, n, l, kb));
    });
    Mat<D> bdf = mzero<D>();
    for (int l = 1; l <= k; ++l) bdf = madd<D>(bdf, mscal<D>(W.a[l], ld<D>(G.les, tri(n - l) + m, kb)));
    // rhs = q - bdf/h - h * (-i) hist
    Mat<D> rhs = msub<D>(q, mscal<D>(1.0 / g.h, bdf));
    rhs = madd<D>(rhs, mscal<D>(g.h, mmuli<D>(hist)));
    Mat<D> y = mmul<D>(rhs, mdag<D>(Minv));   // (M_n^dagger)^-1 = (M_n^-1)^dagger
    if (!mfinite<D>(y)) atomicOr(status, NGF_NONFINITE);
    st<D>(G.les, tri(n) + m, kb, y);
}

// One launch for the three independent bulk tasks of step n; blocks [0, nb_les) do the
// lesser (B) items, then the left-mixing row, then the retarded (B) items.  Items are
// (column, problem) pairs with the problem index fastest, so a warp reads contiguous
// problem vectors of each history element.
// M_n^-1 of every problem of the batch, once per step (one thread per problem); minv_ws
// holds D x D complex per problem
template <int D>
__global__ void k_minv_step(Grid g, int n, HermV S, FuncV eps, cplx* minv_ws, int* status) {
    const int kb = blockIdx.x * blockDim.x + threadIdx.x;
    if (kb >= g.nb) return;
    const NgWeights& W = c_W[g.k - 1];
    int sing = 0;
    Mat<D> Mi = minv<D>(step_matrix<D>(W, g, S, eps, n, kb), &sing);
    if (sing) atomicOr(status, NGF_SINGULAR);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) minv_ws[((int64_t)kb * D + a) * D + b] = Mi.v[a][b];
}
template <int D>
__device__ __forceinline__ Mat<D> ld_minv(const cplx* minv_ws, int kb) {
    Mat<D> r;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) r.v[a][b] = minv_ws[((int64_t)kb * D + a) * D + b];
    return r;
}

// tvq: the FFT pre-pass's correlation of the left-mixing source (nullptr: direct sums)
template <int D>
__global__ void __launch_bounds__(128, D == 1 ? 6 : 1) k_step_bulk(Grid g, int n, HermV G, HermV S, FuncV eps, const cplx* minv_ws,
                                                   int nb_les, int nb_tv, int nb_ret, const cplx* tvq, int* status) {
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
    if (task == 0) ncol = n - W.k - 1;      // m = 1..n-k-1
    else if (task == 1) ncol = g.ntau + 1;  // m = 0..ntau
    else ncol = n - W.k;                    // m = 0..n-k-1
    if (col >= ncol) return;
    const Mat<D> Minv = ld_minv<D>(minv_ws, kb);
    if (task == 0) les_item<D>(W, g, G, S, Minv, n, (int)col + 1, kb, status);
    else if (task == 1) tv_item<D>(W, g, G, S, Minv, n, (int)col, kb, tvq, status);
    else ret_item<D>(W, g, G, S, Minv, n, (int)col, kb, status);
}

// ----------------------------------------------------------------------------------------
// small dense solver (Gaussian elimination with partial pivoting), row-major A[N][N],
// right-hand sides B[N][nrhs]; one thread.
// ----------------------------------------------------------------------------------------
__device__ inline int dense_solve(cplx* A, int N, cplx* B, int nrhs) {
    for (int c = 0; c < N; ++c) {
        int p = c;
        double best = cabs2(A[c * N + c]);
        for (int r = c + 1; r < N; ++r)
            if (cabs2(A[r * N + c]) > best) { best = cabs2(A[r * N + c]); p = r; }
        if (best == 0.0) return 1;
        if (p != c) {
            for (int j = 0; j < N; ++j) { cplx t = A[c * N + j]; A[c * N + j] = A[p * N + j]; A[p * N + j] = t; }
            for (int j = 0; j < nrhs; ++j) { cplx t = B[c * nrhs + j]; B[c * nrhs + j] = B[p * nrhs + j]; B[p * nrhs + j] = t; }
        }
        cplx inv = cdiv(cr(1.0), A[c * N + c]);
        for (int r = c + 1; r < N; ++r) {
            cplx f = cmul(A[r * N + c], inv);
            if (f.x == 0.0 && f.y == 0.0) continue;
            for (int j = c; j < N; ++j) A[r * N + j] = csub(A[r * N + j], cmul(f, A[c * N + j]));
            for (int j = 0; j < nrhs; ++j) B[r * nrhs + j] = csub(B[r * nrhs + j], cmul(f, B[c * nrhs + j]));
        }
    }
    for (int c = N - 1; c >= 0; --c) {
        cplx inv = cdiv(cr(1.0), A[c * N + c]);
        for (int j = 0; j < nrhs; ++j) {
            cplx s = B[c * nrhs + j];
            for (int q = c + 1; q < N; ++q) s = csub(s, cmul(A[c * N + q], B[q * nrhs + j]));
            B[c * nrhs + j] = cmul(s, inv);
        }
    }
    return 0;
}

// The same elimination by the 32 lanes of one warp (every lane calls it; A, B and the scratch
// f[N] visible to the warp).  Per column the pivot is the first row of largest |A[r][c]|^2, as in
// dense_solve; the lanes swap the rows, form the factors of the rows below once and update the
// trailing elements, each element receiving the operations of dense_solve in the same order, so
// the reduced system is bitwise that of dense_solve.  The back substitution runs column by
// column (x_c = B[c] / A[c][c], then B[r] -= A[r][c] x_c for the rows r < c in parallel).
// Returns 1 on every lane when a pivot vanishes.  FP64 on this part is issued per warp
// instruction whatever the number of active lanes, so the lanes cost nothing over one thread.
__device__ inline int warp_dense_solve(cplx* A, int N, cplx* B, int nrhs, cplx* f, int lane) {
    const unsigned full = 0xffffffffu;
    for (int c = 0; c < N; ++c) {
        double best = -1.0;
        int p = N;
        for (int r = c + lane; r < N; r += 32) {
            const double v = cabs2(A[r * N + c]);
            if (v > best) { best = v; p = r; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double bo = __shfl_xor_sync(full, best, o);
            const int po = __shfl_xor_sync(full, p, o);
            if (bo > best || (bo == best && po < p)) { best = bo; p = po; }
        }
        if (best == 0.0) return 1;
        if (p >= N) p = c;   // no comparable entry (NaN column): keep the row, as dense_solve does
        if (p != c) {
            for (int j = lane; j < N; j += 32) {
                const cplx t = A[c * N + j]; A[c * N + j] = A[p * N + j]; A[p * N + j] = t;
            }
            for (int j = lane; j < nrhs; j += 32) {
                const cplx t = B[c * nrhs + j]; B[c * nrhs + j] = B[p * nrhs + j]; B[p * nrhs + j] = t;
            }
        }
        __syncwarp();
        const cplx inv = cdiv(cr(1.0), A[c * N + c]);
        for (int r = c + 1 + lane; r < N; r += 32) f[r] = cmul(A[r * N + c], inv);
        __syncwarp();
        const int wa = N - c, w = wa + nrhs, cnt = (N - c - 1) * w;
        for (int e = lane; e < cnt; e += 32) {
            const int r = c + 1 + e / w, j = e % w;
            const cplx fr = f[r];
            if (fr.x == 0.0 && fr.y == 0.0) continue;
            if (j < wa) A[r * N + c + j] = csub(A[r * N + c + j], cmul(fr, A[c * N + c + j]));
            else B[r * nrhs + j - wa] = csub(B[r * nrhs + j - wa], cmul(fr, B[c * nrhs + j - wa]));
        }
        __syncwarp();
    }
    for (int c = N - 1; c >= 0; --c) {
        const cplx inv = cdiv(cr(1.0), A[c * N + c]);
        for (int j = lane; j < nrhs; j += 32) B[c * nrhs + j] = cmul(B[c * nrhs + j], inv);
        __syncwarp();
        for (int e = lane; e < c * nrhs; e += 32) {
            const int r = e / nrhs, j = e % nrhs;
            B[r * nrhs + j] = csub(B[r * nrhs + j], cmul(A[r * N + c], B[c * nrhs + j]));
        }
        __syncwarp();
    }
    return 0;
}

// block-wide sum of a Mat<D> in a fixed order (deterministic); result valid in thread 0
template <int D>
__device__ Mat<D> block_sum(Mat<D> x, cplx* red /* blockDim.x * D*D */) {
    const int t = threadIdx.x;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) red[(a * D + b) * blockDim.x + t] = x.v[a][b];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (t < s)
#pragma unroll
            for (int e = 0; e < D * D; ++e)
                red[e * blockDim.x + t] = cadd(red[e * blockDim.x + t], red[e * blockDim.x + t + s]);
        __syncthreads();
    }
    Mat<D> r;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) r.v[a][b] = red[(a * D + b) * blockDim.x];
    __syncthreads();
    return r;
}

#define NG_BND_THREADS 128
#define NG_MAXQ (2 * NG_KMAX + 1)

// element (a, b) of block e of a component, problem kb
__device__ __forceinline__ cplx& cel(const Comp& c, int64_t e, int a, int b, int D, int kb) {
    return c.p[(e * (D * D) + a * D + b) * c.ldk + (c.ldk == 1 ? 0 : kb)];
}

// Conjugate VIDE start-up along row n (implementation (A), Eq. MBCVSAMx_cc_start): G^R(n, n) = -i
// and G^R(n, n-l), l = 1..k, by one (k nf)^2 solve.  One warp (all lanes call it): the lanes build
// the k (k+1) blocks of the system, then solve it together.  Ash, Bsh, f: the warp's scratch.
template <int D>
__device__ void ret_row_startup_w(const NgWeights& W, const Grid& g, int n, const HermV& G, const HermV& S,
                                  const FuncV& eps, int kb, cplx* Ash, cplx* Bsh, cplx* f, int lane, int* status) {
    const int k = W.k;
    // unknowns y_1..y_k (y_j = G^R(n, n-j)), y_0 = -i; sum_{l>=1} y_l Mh[l][j] = -y_0 Mh[0][j]
    // with Mh[l][j] = D_{j,l}/h + delta_{lj} i(eps_{n-j} - mu) + h s_{j,l} i Sigma~^R(n-l, n-j).
    // Transposed: sum_l Mh[l][j]^T y_l^T = -(y_0 Mh[0][j])^T.
    const int N = k * D;
    for (int p = lane; p < k * (k + 1); p += 32) {
        const int j = 1 + p / (k + 1), l = p % (k + 1);
        Mat<D> Mh = meye<D>(cr(W.D[j][l] / g.h));
        Mh = madd<D>(Mh, mscal<D>(g.h * W.greg[j][l], mmuli<D>(gretx<D>(S, n - l, n - j, kb))));
        if (l == j) {
            Mat<D> e = ldf<D>(eps, n - j, kb);
            for (int a = 0; a < D; ++a) e.v[a][a].x -= g.mu;
            Mh = madd<D>(Mh, mmuli<D>(e));
        }
        if (l == 0) {
            Mat<D> r = mmul<D>(meye<D>(make_double2(0.0, -1.0)), Mh);  // y_0 Mh[0][j]
            for (int a = 0; a < D; ++a)
                for (int c = 0; c < D; ++c) Bsh[((j - 1) * D + a) * D + c] = cneg(r.v[c][a]);
        } else {
            for (int a = 0; a < D; ++a)
                for (int b = 0; b < D; ++b) Ash[((j - 1) * D + a) * N + (l - 1) * D + b] = Mh.v[b][a];
        }
    }
    __syncwarp();
    const int bad = warp_dense_solve(Ash, N, Bsh, D, f, lane);
    if (lane == 0) {
        if (bad) atomicOr(status, NGF_SINGULAR);
        st<D>(G.ret, tri(n) + n, kb, meye<D>(make_double2(0.0, -1.0)));
    }
    for (int l = 1 + lane; l <= k; l += 32) {
        Mat<D> y;
        for (int a = 0; a < D; ++a)
            for (int c = 0; c < D; ++c) y.v[c][a] = Bsh[((l - 1) * D + a) * D + c];
        if (!mfinite<D>(y)) atomicOr(status, NGF_NONFINITE);
        st<D>(G.ret, tri(n) + n - l, kb, y);
    }
}

// VIDE start-up of column n for the rows m = 1..k (Eq. vdiff_start): sum_l M_{m,l} y_l =
// q_m - M_{m,0} y_0 with y_0 = G^<(0, n) and the sources q_m in qsrc[m-1].  One warp: the lanes
// build the blocks (m, l), then solve together.
template <int D>
__device__ void les_col_startup_w(const NgWeights& W, const Grid& g, int n, const HermV& G, const HermV& S,
                                  const FuncV& eps, int kb, const cplx (*qsrc)[D][D], cplx* Ash, cplx* Bsh, cplx* f,
                                  int lane, int* status) {
    const int k = W.k;
    const int N = k * D;
    for (int p = lane; p < k * (k + 1); p += 32) {
        const int m = 1 + p / (k + 1), l = p % (k + 1);
        Mat<D> M = meye<D>(cr(W.D[m][l] / g.h));
        M = madd<D>(M, mscal<D>(g.h * W.greg[m][l], mmuli<D>(gretx<D>(S, m, l, kb))));
        if (l == m) {
            Mat<D> e = ldf<D>(eps, m, kb);
            for (int a = 0; a < D; ++a) e.v[a][a].x -= g.mu;
            M = madd<D>(M, mmuli<D>(e));
        }
        if (l == 0) {
            Mat<D> rhs;
            for (int a = 0; a < D; ++a)
                for (int b = 0; b < D; ++b) rhs.v[a][b] = qsrc[m - 1][a][b];
            rhs = msub<D>(rhs, mmul<D>(M, ld<D>(G.les, tri(n) + 0, kb)));
            for (int a = 0; a < D; ++a)
                for (int c = 0; c < D; ++c) Bsh[((m - 1) * D + a) * D + c] = rhs.v[a][c];
        } else {
            for (int a = 0; a < D; ++a)
                for (int b = 0; b < D; ++b) Ash[((m - 1) * D + a) * N + (l - 1) * D + b] = M.v[a][b];
        }
    }
    __syncwarp();
    if (warp_dense_solve(Ash, N, Bsh, D, f, lane) && lane == 0) atomicOr(status, NGF_SINGULAR);
    for (int m = 1 + lane; m <= k; m += 32) {
        Mat<D> y;
        for (int a = 0; a < D; ++a)
            for (int c = 0; c < D; ++c) y.v[a][c] = Bsh[((m - 1) * D + a) * D + c];
        if (!mfinite<D>(y)) atomicOr(status, NGF_NONFINITE);
        st<D>(G.les, tri(n) + m, kb, y);
    }
    __syncwarp();
}

// scratch of les_steps_w: the weighted Sigma^R(m, l) of the chain's rows (at most k+1 rows of at
// most 2k terms) and the column values G^<(l, n) it reads (at most 2k+1)
#define NG_LS_ROWS (NG_KMAX + 1)
#define NG_LS_TERMS (2 * NG_KMAX)
#define NG_LS_COL (2 * NG_KMAX + 1)
template <int D>
__host__ __device__ constexpr int les_steps_scratch() { return (NG_LS_ROWS * NG_LS_TERMS + NG_LS_COL) * D * D; }

// Serial VIDE steps (Eq. MBCVSAMx_t) of column n in the first argument, rows m = mstep..n, with
// the sources qsrc[m - m0] and the partial histories hsrc[m - m0] over l < lfrom.  One warp: the
// inverse step matrices of all rows first, one lane per row (they do not depend on the column),
// and every value the chain reads from memory (w_{m,l} Sigma^R(m,l), the column below mstep) is
// staged in shared memory at once, so that the serial part waits on no global load; then per row,
// lane (grp, a, b) sums element (a, b) of the history and BDF terms l = grp, grp + 32/D^2, ...,
// the groups are added by a butterfly, and the lanes of group 0 store the elements of G^<(m, n).
// Mi: NG_MAXQ + 1 blocks; scr: les_steps_scratch<D>() values.
template <int D>
__device__ void les_steps_w(const NgWeights& W, const Grid& g, int n, const HermV& G, const HermV& S,
                            const FuncV& eps, int kb, const cplx (*qsrc)[D][D], const cplx (*hsrc)[D][D],
                            cplx (*Mi)[D][D], cplx* scr, int m0, int mstep, int lfrom, int lane, int* status) {
    static_assert(D * D <= 32, "one warp holds the elements of a block");
    const unsigned full = 0xffffffffu;
    constexpr int E = D * D, NGR = 32 / E;
    const int k = W.k;
    const int lo = min(lfrom, mstep - k);   // lowest column row the chain reads
    cplx* wS = scr;                                  // [row m - mstep][l - lfrom][E]
    cplx* col = scr + NG_LS_ROWS * NG_LS_TERMS * E;  // [l - lo][E]
    int sing = 0;
    for (int m = mstep + lane; m <= n; m += 32) {
        const Mat<D> mi = minv<D>(step_matrix<D>(W, g, S, eps, m, kb), &sing);
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b) Mi[m - m0][a][b] = mi.v[a][b];
    }
    if (__any_sync(full, sing) && lane == 0) atomicOr(status, NGF_SINGULAR);
    for (int i = lane; i < (n - mstep + 1) * NG_LS_TERMS * E; i += 32) {
        const int r = i / (NG_LS_TERMS * E), rem = i % (NG_LS_TERMS * E), l = lfrom + rem / E, e = rem % E;
        const int m = mstep + r;
        if (l < m) wS[i] = cscal(gw(W, m, l), cel(S.ret, tri(m) + l, e / D, e % D, D, kb));
    }
    for (int i = lane; i < (mstep - lo) * E; i += 32)
        col[i] = cel(G.les, tri(n) + lo + i / E, (i % E) / D, (i % E) % D, D, kb);
    __syncwarp();
    const int grp = lane / E, e = lane % E, a = e / D, b = e % D;
    const double hinv = 1.0 / g.h;
    for (int m = mstep; m <= n; ++m) {
        const int r = m - m0;
        const cplx* wrow = wS + (m - mstep) * NG_LS_TERMS * E;
        cplx hs = cr(0.0), bd = cr(0.0);
        for (int l = lfrom + grp; l < m; l += NGR) {
#pragma unroll
            for (int c = 0; c < D; ++c)
                hs = cfma(wrow[(l - lfrom) * E + a * D + c], col[(l - lo) * E + c * D + b], hs);
        }
        for (int l = 1 + grp; l <= k; l += NGR) {
            const cplx x = col[(m - l - lo) * E + e];
            bd = cadd(bd, make_double2(W.a[l] * x.x, W.a[l] * x.y));
        }
#pragma unroll
        for (int o = E; o < 32; o <<= 1) {
            hs.x += __shfl_xor_sync(full, hs.x, o);
            hs.y += __shfl_xor_sync(full, hs.y, o);
            bd.x += __shfl_xor_sync(full, bd.x, o);
            bd.y += __shfl_xor_sync(full, bd.y, o);
        }
        // acc = q - bdf / h - h i (h_partial + h_rows)
        const cplx h0 = cadd(hsrc[r][a][b], hs);
        cplx acc = csub(qsrc[r][a][b], make_double2(hinv * bd.x, hinv * bd.y));
        acc = csub(acc, make_double2(-g.h * h0.y, g.h * h0.x));
        cplx y = cr(0.0);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            cplx ac;
            ac.x = __shfl_sync(full, acc.x, c * D + b);
            ac.y = __shfl_sync(full, acc.y, c * D + b);
            y = cfma(Mi[r][a][c], ac, y);
        }
        if (grp == 0) {
            if (!isfinite(y.x) || !isfinite(y.y)) atomicOr(status, NGF_NONFINITE);
            cel(G.les, tri(n) + m, a, b, D, kb) = y;
            col[(m - lo) * E + e] = y;
        }
        __syncwarp();
    }
}

// Per-problem boundary of step n: retarded start-up (A) for m = n-k..n, then the lesser
// column's G^<(0,n) and serial (A) part.  One block per problem.
template <int D>
__global__ void __launch_bounds__(NG_BND_THREADS) k_step_boundary(Grid g, int n, HermV G, HermV S, FuncV eps,
                                                                  int* status) {
    const NgWeights& W = c_W[g.k - 1];
    const int k = W.k;
    const int kb = blockIdx.x;
    const int t = threadIdx.x;
    __shared__ cplx red[NG_BND_THREADS * D * D];
    __shared__ cplx qsrc[NG_MAXQ + 1][D][D];   // sources per boundary row
    __shared__ cplx hsrc[NG_MAXQ + 1][D][D];   // partial histories per boundary row
    __shared__ cplx Mi[NG_MAXQ + 1][D][D];     // inverse step matrices of the boundary rows
    __shared__ cplx Ash[(NG_KMAX * D) * (NG_KMAX * D)];
    __shared__ cplx Bsh[(NG_KMAX * D) * D];
    __shared__ cplx fsh[NG_KMAX * D];
    __shared__ cplx lsc[les_steps_scratch<D>()];

    // ---- retarded: conjugate start-up along row n (implementation (A)), warp 0 -------
    if (t < 32) {
        ret_row_startup_w<D>(W, g, n, G, S, eps, kb, Ash, Bsh, fsh, t, status);
        // G^<(0,n) = -[G^tv(n,0)]^dagger  (Eq. dyson_ini_les)
        if (t == 0) st<D>(G.les, tri(n) + 0, kb, mscal<D>(-1.0, mdag<D>(gtv<D>(G, g, n, 0, kb))));
    }
    __syncthreads();

    // ---- lesser: rows handled by (A) ------------------------------------------------
    const bool full = (n <= 2 * k);           // whole column by (A)
    const int m0 = full ? 1 : n - k;          // first (A) row
    const int nq = n - m0 + 1;                // number of (A) rows
    for (int r = 0; r < nq; ++r) {
        const int m = m0 + r;
        Mat<D> part = q_lesA_part<D>(W, g, G, S, m, n, kb, t, blockDim.x);
        Mat<D> q = block_sum<D>(part, red);
        // partial history over the rows below m0 (known values): sum_{l<m0} w_{m,l} Sigma^R(m,l) G^<(l,n)
        Mat<D> hp = mzero<D>();
        if (!full && m > k) {
            for (int l = t; l < m0; l += blockDim.x)
                mfma<D>(hp, mscal<D>(gw(W, m, l), gret<D>(S, m, l, kb)), ld<D>(G.les, tri(n) + l, kb));
        }
        Mat<D> hsum = block_sum<D>(hp, red);
        if (t == 0)
            for (int a = 0; a < D; ++a)
                for (int b = 0; b < D; ++b) { qsrc[r][a][b] = q.v[a][b]; hsrc[r][a][b] = hsum.v[a][b]; }
    }
    __syncthreads();
    if (t >= 32) return;
    int mstep = m0;
    if (full) {
        les_col_startup_w<D>(W, g, n, G, S, eps, kb, qsrc, Ash, Bsh, fsh, t, status);
        mstep = k + 1;
    }
    les_steps_w<D>(W, g, n, G, S, eps, kb, qsrc, hsrc, Mi, lsc, m0, mstep, full ? 0 : m0, t, status);
}

// Serial schedule of step n (the paper's dyson_timestep): the retarded row by the conjugate
// VIDE (A) along the whole row (start-up for l = 1..k, then single steps in l = n - m for
// l = k+1..n), and the lesser column by the VIDE (A) along the whole column (G^<(0, n) from
// Eq. dyson_ini_les, start-up for m = 1..k, then single steps m = k+1..n with the sources
// -i (C^<_2 + C^<_3)[Sigma, 1, G](m, n)).  The left-mixing row comes from the bulk launch
// before this one.  One block per problem; every step's sums are block reductions in a fixed
// order, the step itself runs on thread 0, the two start-up solves on warp 0.
template <int D>
__global__ void __launch_bounds__(NG_BND_THREADS) k_step_serial(Grid g, int n, HermV G, HermV S, FuncV eps,
                                                                int* status) {
    const NgWeights& W = c_W[g.k - 1];
    const int k = W.k;
    const int kb = blockIdx.x;
    const int t = threadIdx.x;
    __shared__ cplx red[NG_BND_THREADS * D * D];
    __shared__ cplx qsrc[NG_MAXQ + 1][D][D];
    __shared__ cplx Ash[(NG_KMAX * D) * (NG_KMAX * D)];
    __shared__ cplx Bsh[(NG_KMAX * D) * D];
    __shared__ cplx fsh[NG_KMAX * D];
    int sing = 0;

    // ---- retarded row: y_l = G^R(n, n-l), kernel i Sigma^R(n-l, n-j) ----------------------
    if (t < 32) ret_row_startup_w<D>(W, g, n, G, S, eps, kb, Ash, Bsh, fsh, t, status);
    __syncthreads();
    for (int j = k + 1; j <= n; ++j) {
        Mat<D> part = mzero<D>();
        for (int l = t; l < j; l += blockDim.x)
            mfma<D>(part, mscal<D>(gw(W, j, l), gret<D>(G, n, n - l, kb)), gret<D>(S, n - l, n - j, kb));
        Mat<D> hs = block_sum<D>(part, red);
        if (t == 0) {
            Mat<D> bdf = mzero<D>();
            for (int l = 1; l <= k; ++l) bdf = madd<D>(bdf, mscal<D>(W.a[l], gret<D>(G, n, n - j + l, kb)));
            Mat<D> rhs = msub<D>(mscal<D>(-1.0 / g.h, bdf), mscal<D>(g.h, mmuli<D>(hs)));
            Mat<D> e = ldf<D>(eps, n - j, kb);
            for (int a = 0; a < D; ++a) e.v[a][a].x -= g.mu;
            Mat<D> Mj = meye<D>(cr(W.a[0] / g.h));
            Mj = madd<D>(Mj, mmuli<D>(e));
            Mj = madd<D>(Mj, mscal<D>(g.h * gw(W, j, j), mmuli<D>(gret<D>(S, n - j, n - j, kb))));
            Mat<D> y = mmul<D>(rhs, minv<D>(Mj, &sing));
            if (!mfinite<D>(y)) atomicOr(status, NGF_NONFINITE);
            st<D>(G.ret, tri(n) + n - j, kb, y);
        }
        __syncthreads();
    }

    // ---- lesser column ------------------------------------------------------------------
    if (t == 0) st<D>(G.les, tri(n) + 0, kb, mscal<D>(-1.0, mdag<D>(gtv<D>(G, g, n, 0, kb))));
    for (int m = 1; m <= k; ++m) {
        Mat<D> q = block_sum<D>(q_lesA_part<D>(W, g, G, S, m, n, kb, t, blockDim.x), red);
        if (t == 0)
            for (int a = 0; a < D; ++a)
                for (int b = 0; b < D; ++b) qsrc[m - 1][a][b] = q.v[a][b];
    }
    __syncthreads();
    if (t < 32) les_col_startup_w<D>(W, g, n, G, S, eps, kb, qsrc, Ash, Bsh, fsh, t, status);
    __syncthreads();
    for (int m = k + 1; m <= n; ++m) {
        Mat<D> q = block_sum<D>(q_lesA_part<D>(W, g, G, S, m, n, kb, t, blockDim.x), red);
        Mat<D> hp = mzero<D>();
        for (int l = t; l < m; l += blockDim.x)
            mfma<D>(hp, mscal<D>(gw(W, m, l), gret<D>(S, m, l, kb)), ld<D>(G.les, tri(n) + l, kb));
        Mat<D> hsum = block_sum<D>(hp, red);
        if (t == 0) {
            Mat<D> bdf = mzero<D>();
            for (int l = 1; l <= k; ++l) bdf = madd<D>(bdf, mscal<D>(W.a[l], ld<D>(G.les, tri(n) + m - l, kb)));
            Mat<D> acc = msub<D>(q, mscal<D>(1.0 / g.h, bdf));
            acc = msub<D>(acc, mscal<D>(g.h, mmuli<D>(hsum)));
            Mat<D> y = mmul<D>(minv<D>(step_matrix<D>(W, g, S, eps, m, kb), &sing), acc);
            if (!mfinite<D>(y)) atomicOr(status, NGF_NONFINITE);
            st<D>(G.les, tri(n) + m, kb, y);
        }
        __syncthreads();
    }
    if (sing) atomicOr(status, NGF_SINGULAR);
}
