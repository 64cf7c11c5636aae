// Time step for small batches: one warp per (column, problem) bulk item, and the boundary of
// the step spread over blocks with its serial parts on one warp per problem.
//
// The bulk items of a time step (Sec. "Time stepping": retarded (B) elements, the left-mixing
// row, lesser (B) elements) each carry O(n + ntau) history and source terms.  With one thread
// per item a batch of a few problems (a dimer, a real-space cluster) leaves almost every SM
// idle and each thread sums its terms serially.  Here the 32 lanes of a warp take the terms of
// every sum of one item (the Gregory end terms one per lane, the unit-weight middle dealt out
// with no weight multiply; the left-mixing source by its direct quadrature), the lane partials
// are added by a fixed butterfly that leaves one element of the nf x nf result on each lane
// (warp_rsum), and the closing step (BDF terms, right-hand side, the product with M_n^-1, the
// store) runs one element per lane.  The arithmetic is that of k_step_bulk up to the order of
// the additions.
#pragma once

#include "ng_step.cuh"

// f(l, w_{L,l}) for this lane's share of the terms l = 0..lmax (L-1 <= lmax <= L) of a Gregory
// row L.  For rows L > 2k+1 the end terms (l <= k, L-k <= l <= lmax) take one lane each from
// lane 0 on (at most 2k+2 <= 32 of them for k <= 6), and the unit-weight middle is dealt out
// from the next lane on with w = 1.0, which the compiler folds (no weight multiply); every
// lane gets at most ceil((lmax+1)/32) terms, as with a plain stride over l.
template <class F>
__device__ __forceinline__ void greg_for_lanes(const NgWeights& W, int L, int lmax, int lane, F&& f) {
    const int k = W.k;
    if (L <= 2 * k + 1) {
        for (int l = lane; l <= lmax; l += 32) f(l, W.greg[L][l]);
        return;
    }
    const int ne = 2 * k + 2 - (L - lmax);  // end terms
    if (lane <= k) f(lane, W.omega[lane]);
    else if (lane < ne) f(L - 2 * k - 1 + lane, W.omega[2 * k + 1 - lane]);  // l = L-k .. lmax
    const int e2 = L - k - 1;
    for (int l = k + 1 + ((lane - ne) & 31); l <= e2; l += 32) f(l, 1.0);
}

// Lane sum scattered over the elements: lane l returns the sum over the 32 lanes of element
// rs_elem<D>(l) = l >> (5 - log2 D^2) of x.  The first log2 D^2 rounds halve what each lane
// carries (a lane keeps one half and adds its partner's copy of that half), the remaining rounds
// add the single value left: 2 (D^2 - 1) + 2 (5 - log2 D^2) FP64 additions per lane against
// 10 D^2 for a butterfly of every element, and the item's closing step then runs one element per
// lane.
template <int D>
struct RsLog { static constexpr int v = (D == 1) ? 0 : (D == 2) ? 2 : (D == 4) ? 4 : -1; };
template <int D>
__device__ __forceinline__ int rs_elem(int lane) { return lane >> (5 - RsLog<D>::v); }
template <int D>
__device__ __forceinline__ bool rs_leader(int lane) { return (lane & ((32 >> RsLog<D>::v) - 1)) == 0; }
template <int D>
__device__ __forceinline__ cplx rs_get(cplx x, int e) { return make_double2(
    __shfl_sync(0xffffffffu, x.x, e << (5 - RsLog<D>::v)), __shfl_sync(0xffffffffu, x.y, e << (5 - RsLog<D>::v))); }

template <int D>
__device__ __forceinline__ cplx warp_rsum(const Mat<D>& x, int lane) {
    constexpr int E = D * D, LG = RsLog<D>::v;
    static_assert(LG >= 0, "D = 1, 2 or 4");
    cplx v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = x.v[e / D][e % D];
#pragma unroll
    for (int r = 0; r < LG; ++r) {
        const int off = 16 >> r, h = E >> (r + 1);
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const cplx keep = up ? v[i + h] : v[i];
            const cplx give = up ? v[i] : v[i + h];
            v[i] = make_double2(keep.x + __shfl_xor_sync(0xffffffffu, give.x, off),
                                keep.y + __shfl_xor_sync(0xffffffffu, give.y, off));
        }
    }
#pragma unroll
    for (int off = 16 >> LG; off > 0; off >>= 1) {
        v[0].x += __shfl_xor_sync(0xffffffffu, v[0].x, off);
        v[0].y += __shfl_xor_sync(0xffffffffu, v[0].y, off);
    }
    return v[0];
}

// element (a, b) of a stored block
__device__ __forceinline__ cplx elw(const Comp& c, int64_t e, int a, int b, int D, int kb) {
    return c.p[(e * (D * D) + a * D + b) * c.ldk + (c.ldk == 1 ? 0 : kb)];
}

template <int D>
__device__ __forceinline__ void ret_item_w(const NgWeights& W, const Grid& g, const HermV& G, const HermV& S,
                                           const cplx* minv_ws, int n, int m, int kb, int lane, int* status) {
    const int L = n - m;  // > k
    Mat<D> acc = mzero<D>();
    greg_for_lanes(W, L, L - 1, lane, [&](int l, double w) {
        mfma<D>(acc, mscal<D>(w, gret<D>(S, n, m + l, kb)), gret<D>(G, m + l, m, kb));
    });
    // closing step, one element (a, b) per lane: rhs = -(1/h) bdf - h i acc, y = M_n^-1 rhs
    const cplx ae = warp_rsum<D>(acc, lane);
    const int e = rs_elem<D>(lane), a = e / D, b = e % D;
    cplx bdf = cz();
    for (int l = 1; l <= W.k; ++l) bdf = cadd(bdf, cscal(W.a[l], elw(G.ret, tri(n - l) + m, a, b, D, kb)));
    const cplx rhs = csub(cscal(-1.0 / g.h, bdf), cscal(g.h, cmuli(ae)));
    cplx y = cz();
#pragma unroll
    for (int c = 0; c < D; ++c) y = cfma(minv_ws[((int64_t)kb * D + a) * D + c], rs_get<D>(rhs, c * D + b), y);
    if (rs_leader<D>(lane)) {
        if (!cfinite(y)) atomicOr(status, NGF_NONFINITE);
        G.ret.p[((tri(n) + m) * (D * D) + a * D + b) * G.ret.ldk + (G.ret.ldk == 1 ? 0 : kb)] = y;
    }
}

// The left-mixing source -i (C^tv_2 + C^tv_3)[S, 1, G^M](n, tau_m) (Eqs. ctv2, ctv3) as q_tv
// computes it, over this lane's terms of its two Gregory sums and of the boundary (R) formulas
// of m <= k and m >= ntau - k ((k+1)^2 terms each).  The source is linear in the terms, so the
// lanes' parts add up to q_tv.
template <int D>
__device__ Mat<D> q_tv_part(const NgWeights& W, const Grid& g, const HermV& G, const HermV& S, int n, int m, int kb,
                            int lane) {
    const int l0 = lane;
    const int k = W.k, T = g.ntau;
    const double xi = (double)g.sig;
    Mat<D> c2 = mzero<D>(), c3 = mzero<D>();
    if (m <= k) {
        for (int p = l0; p < (k + 1) * (k + 1); p += 32) {
            const int j = p / (k + 1), l = p % (k + 1);
            mfma<D>(c2, mscal<D>(W.R[m][j][l], gtv<D>(S, g, n, l, kb)), mscal<D>(xi, gmat<D>(G, T - j, kb)));
        }
    } else {
        greg_for_lanes(W, m, m, lane, [&](int l, double w) {
            mfma<D>(c2, mscal<D>(w, gtv<D>(S, g, n, m - l, kb)), gmat<D>(G, T - l, kb));
        });
        c2 = mscal<D>(xi, c2);
    }
    if (m >= T - k) {
        for (int p = l0; p < (k + 1) * (k + 1); p += 32) {
            const int j = p / (k + 1), l = p % (k + 1);
            mfma<D>(c3, mscal<D>(W.R[T - m][j][l], gtv<D>(S, g, n, T - l, kb)), gmat<D>(G, j, kb));
        }
    } else {
        greg_for_lanes(W, T - m, T - m, lane, [&](int l, double w) {
            mfma<D>(c3, mscal<D>(w, gtv<D>(S, g, n, m + l, kb)), gmat<D>(G, l, kb));
        });
    }
    return mscal<D>(g.htau, mmuli<D>(mscal<D>(-1.0, madd<D>(c2, c3))));
}

// the left-mixing item: history and source sums over the lanes (no FFT pre-pass in this form)
template <int D>
__device__ __forceinline__ void tv_item_w(const NgWeights& W, const Grid& g, const HermV& G, const HermV& S,
                                          const cplx* minv_ws, int n, int m, int kb, int lane, int* status) {
    Mat<D> acc = mzero<D>();
    greg_for_lanes(W, n, n - 1, lane, [&](int j, double w) {
        mfma<D>(acc, mscal<D>(w, gret<D>(S, n, j, kb)), gtv<D>(G, g, j, m, kb));
    });
    // closing step, one element (a, b) per lane: rhs = src - bdf / h - h i acc, y = M_n^-1 rhs
    const cplx ae = warp_rsum<D>(acc, lane);
    const cplx se = warp_rsum<D>(q_tv_part<D>(W, g, G, S, n, m, kb, lane), lane);
    const int e = rs_elem<D>(lane), a = e / D, b = e % D;
    cplx bdf = cz();
    for (int l = 1; l <= W.k; ++l)
        bdf = cadd(bdf, cscal(W.a[l], elw(G.tv, (int64_t)(n - l) * (g.ntau + 1) + m, a, b, D, kb)));
    cplx rhs = csub(se, cscal(1.0 / g.h, bdf));
    rhs = csub(rhs, cscal(g.h, cmuli(ae)));
    cplx y = cz();
#pragma unroll
    for (int c = 0; c < D; ++c) y = cfma(minv_ws[((int64_t)kb * D + a) * D + c], rs_get<D>(rhs, c * D + b), y);
    if (rs_leader<D>(lane)) {
        if (!cfinite(y)) atomicOr(status, NGF_NONFINITE);
        G.tv.p[(((int64_t)n * (g.ntau + 1) + m) * (D * D) + a * D + b) * G.tv.ldk + (G.tv.ldk == 1 ? 0 : kb)] = y;
    }
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
        greg_for_lanes(W, m, m, lane, [&](int j, double w) {
            mfma<D>(c1, mscal<D>(w, gret<D>(G, m, j, kb)), ld<D>(S.les, tri(n) + j, kb));
        });
    }
    // sum_j w_{T,j} G^tv(m,j) [Sigma^tv(n,T-j)]^dagger
    Mat<D> c3 = mzero<D>();
    greg_for_lanes(W, T, T, lane, [&](int j, double w) {
        mfma_db<D>(c3, mscal<D>(w, gtv<D>(G, g, m, j, kb)), gtv<D>(S, g, n, T - j, kb));
    });
    // history sum_{l<n} w_{n,l} G^<(m,l) [Sigma^R(n,l)]^dagger
    Mat<D> hist = mzero<D>();
    greg_for_lanes(W, n, n - 1, lane, [&](int l, double w) {
        Mat<D> gl = (l >= m) ? ld<D>(G.les, tri(l) + m, kb) : mscal<D>(-1.0, mdag<D>(ld<D>(G.les, tri(m) + l, kb)));
        mfma_db<D>(hist, mscal<D>(w, gl), gret<D>(S, n, l, kb));
    });
    // closing step, one element (a, b) per lane: rhs = h i c1 - xi htau c3 - bdf / h + h i hist,
    // y = rhs [M_n^-1]^dagger
    const cplx c1e = warp_rsum<D>(c1, lane), c3e = warp_rsum<D>(c3, lane), he = warp_rsum<D>(hist, lane);
    const int e = rs_elem<D>(lane), a = e / D, b = e % D;
    const cplx q = csub(cscal(g.h, cmuli(c1e)), cscal((double)g.sig * g.htau, c3e));
    cplx bdf = cz();
    for (int l = 1; l <= k; ++l) bdf = cadd(bdf, cscal(W.a[l], elw(G.les, tri(n - l) + m, a, b, D, kb)));
    cplx rhs = csub(q, cscal(1.0 / g.h, bdf));
    rhs = cadd(rhs, cscal(g.h, cmuli(he)));
    cplx y = cz();
#pragma unroll
    for (int c = 0; c < D; ++c) y = cfma(rs_get<D>(rhs, a * D + c), cconj(minv_ws[((int64_t)kb * D + b) * D + c]), y);
    if (rs_leader<D>(lane)) {
        if (!cfinite(y)) atomicOr(status, NGF_NONFINITE);
        G.les.p[((tri(n) + m) * (D * D) + a * D + b) * G.les.ldk + (G.les.ldk == 1 ? 0 : kb)] = y;
    }
}

// ---- the boundary of a time step for small batches, in three launches -----------------------
// k_step_boundary runs one block per problem, so for a single problem its (A)-row sources, sums
// over n and ntau terms, run on one SM.  Here: (1) per problem, one warp, the retarded (A) row
// start-up (k_bnd_pre, or the leading warps of k_step_bulk_w); (2) the (A)-row sources and
// partial histories spread over blocks (row, problem, chunk), each block summing its chunk's
// terms (k_bnd_src); (3) per problem, one warp, G^<(0,n), the chunk partials added in chunk order
// and the (A) steps of the lesser column (k_bnd_fin), as in k_step_boundary.  G^<(0,n) =
// -[G^tv(n,0)]^dagger (Eq. dyson_ini_les) reads the left-mixing value of the bulk launch, so the
// start-up warps, which may run beside that launch, leave it to k_bnd_fin, and k_bnd_src forms
// its l = 0 term from G^tv(n,0) itself.

template <int D>
__device__ __forceinline__ Mat<D> les0_of_tv(const Grid& g, const HermV& G, int n, int kb) {
    return mscal<D>(-1.0, mdag<D>(gtv<D>(G, g, n, 0, kb)));
}

// the retarded start-up of problem kb by one warp; sh: the warp's scratch
template <int D>
__device__ __forceinline__ void bnd_pre_warp(const NgWeights& W, const Grid& g, int n, const HermV& G,
                                             const HermV& S, const FuncV& eps, int kb, cplx* sh, int lane,
                                             int* status) {
    constexpr int N = NG_KMAX * D;
    ret_row_startup_w<D>(W, g, n, G, S, eps, kb, sh, sh + N * N, sh + N * N + N * D, lane, status);
}
template <int D>
__host__ __device__ constexpr int bnd_pre_scratch() { return (NG_KMAX * D) * (NG_KMAX * D) + (NG_KMAX * D) * D + NG_KMAX * D; }

// one warp (block of 32) per problem
template <int D>
__global__ void __launch_bounds__(32) k_bnd_pre(Grid g, int n, HermV G, HermV S, FuncV eps, int* status) {
    __shared__ cplx sh[bnd_pre_scratch<D>()];
    bnd_pre_warp<D>(c_W[g.k - 1], g, n, G, S, eps, blockIdx.x, sh, threadIdx.x, status);
}

// One warp per item, items ordered as in k_step_bulk (lesser, left-mixing, retarded; problem
// fastest); w_les, w_tv, w_ret: the items of each task.  With w_pre = nb the first nb warps
// run the boundary's retarded start-up of problem kb = warp (bnd_pre_warp), which reads only
// Sigma and eps and writes G^R(n, n-k..n), which no bulk item reads, so that it overlaps the
// bulk instead of taking a launch of its own.
template <int D>
__global__ void __launch_bounds__(128, 1) k_step_bulk_w(Grid g, int n, HermV G, HermV S, FuncV eps,
                                                     const cplx* minv_ws, int64_t w_pre, int64_t w_les,
                                                     int64_t w_tv, int64_t w_ret, int* status) {
    const NgWeights& W = c_W[g.k - 1];
    int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (item < w_pre) {
        __shared__ cplx sh[4][bnd_pre_scratch<D>()];   // blockDim.x = 128: four warps
        bnd_pre_warp<D>(W, g, n, G, S, eps, (int)item, sh[threadIdx.x >> 5], lane, status);
        return;
    }
    item -= w_pre;
    int task;
    if (item < w_les) task = 0;
    else if ((item -= w_les) < w_tv) task = 1;
    else if ((item -= w_tv) < w_ret) task = 2;
    else return;
    const int kb = (int)(item % g.nb);
    const int col = (int)(item / g.nb);
    if (task == 0) les_item_w<D>(W, g, G, S, minv_ws, n, col + 1, kb, lane, status);
    else if (task == 1) tv_item_w<D>(W, g, G, S, minv_ws, n, col, kb, lane, status);
    else ret_item_w<D>(W, g, G, S, minv_ws, n, col, kb, lane, status);
}

// block (r, kb, c): row m = m0 + r, terms j = c B + t, c B + t + nchunk B, ...; partials at
// part[((r nb + kb) nchunk + c) 2 D^2 ...]: the source, then the partial history over l < m0
template <int D>
__global__ void __launch_bounds__(NG_BND_THREADS) k_bnd_src(Grid g, int n, HermV G, HermV S, int nchunk, cplx* part) {
    const NgWeights& W = c_W[g.k - 1];
    const int k = W.k;
    const bool full = (n <= 2 * k);
    const int m0 = full ? 1 : n - k;
    const int r = blockIdx.x, kb = blockIdx.y, c = blockIdx.z, t = threadIdx.x;
    const int m = m0 + r;
    __shared__ cplx red[NG_BND_THREADS * D * D];
    const int j0 = c * blockDim.x + t, js = nchunk * blockDim.x;
    const Mat<D> q = block_sum<D>(q_lesA_part<D>(W, g, G, S, m, n, kb, j0, js), red);
    Mat<D> hp = mzero<D>();
    if (!full && m > k)
        for (int l = j0; l < m0; l += js)
            mfma<D>(hp, mscal<D>(gw(W, m, l), gret<D>(S, m, l, kb)),
                    l == 0 ? les0_of_tv<D>(g, G, n, kb) : ld<D>(G.les, tri(n) + l, kb));
    const Mat<D> hsum = block_sum<D>(hp, red);
    if (t != 0) return;
    cplx* o = part + (((int64_t)r * g.nb + kb) * nchunk + c) * 2 * D * D;
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) {
            o[a * D + b] = q.v[a][b];
            o[D * D + a * D + b] = hsum.v[a][b];
        }
}

// one warp (block of 32) per problem
template <int D>
__global__ void __launch_bounds__(32) k_bnd_fin(Grid g, int n, HermV G, HermV S, FuncV eps, int nchunk,
                                                const cplx* part, int* status) {
    const int kb = blockIdx.x, lane = threadIdx.x;
    const NgWeights& W = c_W[g.k - 1];
    const int k = W.k;
    const bool full = (n <= 2 * k);
    const int m0 = full ? 1 : n - k;
    const int nq = n - m0 + 1;
    __shared__ cplx qsrc[NG_MAXQ + 1][D][D], hsrc[NG_MAXQ + 1][D][D], Mi[NG_MAXQ + 1][D][D];
    __shared__ cplx Ash[(NG_KMAX * D) * (NG_KMAX * D)], Bsh[(NG_KMAX * D) * D], fsh[NG_KMAX * D];
    __shared__ cplx lsc[les_steps_scratch<D>()];
    if (lane == 0) st<D>(G.les, tri(n) + 0, kb, les0_of_tv<D>(g, G, n, kb));
    // the chunk partials of each (row, element), added in chunk order (deterministic)
    for (int i = lane; i < nq * 2 * D * D; i += 32) {
        const int r = i / (2 * D * D), x = i % (2 * D * D);
        cplx v = cr(0.0);
        for (int c = 0; c < nchunk; ++c) v = cadd(v, part[(((int64_t)r * g.nb + kb) * nchunk + c) * 2 * D * D + x]);
        if (x < D * D) qsrc[r][x / D][x % D] = v;
        else hsrc[r][(x - D * D) / D][(x - D * D) % D] = v;
    }
    __syncwarp();
    int mstep = m0;
    if (full) {
        les_col_startup_w<D>(W, g, n, G, S, eps, kb, qsrc, Ash, Bsh, fsh, lane, status);
        mstep = k + 1;
    }
    les_steps_w<D>(W, g, n, G, S, eps, kb, qsrc, hsrc, Mi, lsc, m0, mstep, full ? 0 : m0, lane, status);
}
