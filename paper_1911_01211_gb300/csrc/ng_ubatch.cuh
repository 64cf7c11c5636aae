// Uneven batch (ng_batch_*): independent problems of different orbital dimension nf in
// {1, 2, 4, 8}, length nt and inverse temperature, each with its own fixed self-energy, stepped
// together.  One bulk launch per global time step covers the bulk items of every active
// problem; the orbital-element-wise formulation (one thread per (item, a, b)) keeps the
// register footprint independent of nf.  Same formulas and schedule as ng_step.cuh (paper
// Sec. "Time stepping", mixed schedule).
#pragma once

#include "ng_step.cuh"

#define NG_UMAXP 128    // problems per batch
#define NG_UMAXD 8

struct UProb {
    Grid g;          // g.nb = 1 (one problem), g.nf = D
    HermV G, S;      // ldk as stored; kb selects the problem inside interleaved storage
    FuncV eps;
    int kb;
    cplx* minv;      // D*D workspace: M_n^-1 of the current step
};

// per-step launch table: blocks [start[i], start[i+1]) belong to problem prob[i]; inside,
// the first nles[i] blocks are lesser items, then ntv[i] left-mixing, then retarded items
struct UTable {
    int np;
    int n;                      // global time step
    int start[NG_UMAXP + 1];
    int prob[NG_UMAXP];
    int nles[NG_UMAXP], ntv[NG_UMAXP];
    // partial sums of the (A) rows' sources and histories: src[((i * NG_MAXQ + r) * nchunk +
    // c) * 2 + {0: source, 1: history}][a * D + b], chunks of `chunk` summation indices
    cplx* src;
    int nchunk, chunk;
};
#define NG_USRC_THREADS 256

// element (a,b) of a stored d x d block
__device__ __forceinline__ cplx uel(const Comp& c, int64_t e, int D, int a, int b, int kb) {
    return c.p[(e * (D * D) + a * D + b) * c.ldk + (c.ldk == 1 ? 0 : kb)];
}
__device__ __forceinline__ void ust(const Comp& c, int64_t e, int D, int a, int b, int kb, cplx v) {
    c.p[(e * (D * D) + a * D + b) * c.ldk + (c.ldk == 1 ? 0 : kb)] = v;
}
__device__ __forceinline__ cplx ufunc(const FuncV& f, int n, int D, int a, int b, int kb) {
    return f.p[((int64_t)(n + 1) * (D * D) + a * D + b) * f.ldk + (f.ldk == 1 ? 0 : kb)];
}
// G^R(n,j) element with the modified retarded continuation for j > n
__device__ __forceinline__ cplx uretx(const HermV& X, int n, int j, int D, int a, int b, int kb) {
    if (j <= n) return uel(X.ret, tri(n) + j, D, a, b, kb);
    return cneg(cconj(uel(X.ret, tri(j) + n, D, b, a, kb)));
}
// G^<(j,n) element for any j, n
__device__ __forceinline__ cplx ules(const HermV& X, int j, int n, int D, int a, int b, int kb) {
    if (j <= n) return uel(X.les, tri(n) + j, D, a, b, kb);
    return cneg(cconj(uel(X.les, tri(j) + n, D, b, a, kb)));
}

// M_n^-1 of every active problem: one warp per problem builds M_n and solves M_n X = 1
__global__ void __launch_bounds__(32) k_uminv(const UProb* probs, UTable tab, int* status) {
    if (blockIdx.x >= tab.np) return;
    const UProb& P = probs[tab.prob[blockIdx.x]];
    const NgWeights& W = c_W[P.g.k - 1];
    const int D = P.g.nf, n = tab.n, kb = P.kb, lane = threadIdx.x;
    __shared__ cplx M[NG_UMAXD * NG_UMAXD], R[NG_UMAXD * NG_UMAXD], f[NG_UMAXD];
    for (int i = lane; i < D * D; i += 32) {
        const int a = i / D, b = i % D;
        cplx e = ufunc(P.eps, n, D, a, b, kb);
        if (a == b) e.x -= P.g.mu;
        cplx v = cmuli(e);
        v = cadd(v, cscal(P.g.h * gw(W, n, n), cmuli(uel(P.S.ret, tri(n) + n, D, a, b, kb))));
        if (a == b) v.x += W.a[0] / P.g.h;
        M[i] = v;
        R[i] = cr(a == b ? 1.0 : 0.0);
    }
    __syncwarp();
    if (warp_dense_solve(M, D, R, D, f, lane) && lane == 0) atomicOr(status, NGF_SINGULAR);
    for (int i = lane; i < D * D; i += 32) P.minv[i] = R[i];
}

// ---------------------------------------------------------------------------------------
// element-wise bulk items; each thread holds one complex accumulator per sum
// ---------------------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ cplx u_qtv(const NgWeights& W, const Grid& g, const HermV& G, const HermV& S, int n, int m,
                                      int a, int b, int kb) {
    const int k = W.k, T = g.ntau;
    const int64_t rowS = (int64_t)n * (T + 1);
    cplx c2 = cz(), c3 = cz();
    if (m <= k) {
        for (int j = 0; j <= k; ++j)
            for (int l = 0; l <= k; ++l) {
                const double r = W.R[m][j][l];
#pragma unroll
                for (int c = 0; c < D; ++c)
                    c2 = cfma(cscal(r, uel(S.tv, rowS + l, D, a, c, kb)), uel(G.mat, T - j, D, c, b, kb), c2);
            }
    } else {
        greg_for(W, m, m, [&](int l, double w) {
#pragma unroll
            for (int c = 0; c < D; ++c)
                c2 = cfma(cscal(w, uel(S.tv, rowS + m - l, D, a, c, kb)), uel(G.mat, T - l, D, c, b, kb), c2);
        });
    }
    if (m >= T - k) {
        for (int j = 0; j <= k; ++j)
            for (int l = 0; l <= k; ++l) {
                const double r = W.R[T - m][j][l];
#pragma unroll
                for (int c = 0; c < D; ++c)
                    c3 = cfma(cscal(r, uel(S.tv, rowS + T - l, D, a, c, kb)), uel(G.mat, j, D, c, b, kb), c3);
            }
    } else {
        greg_for(W, T - m, T - m, [&](int l, double w) {
#pragma unroll
            for (int c = 0; c < D; ++c)
                c3 = cfma(cscal(w, uel(S.tv, rowS + m + l, D, a, c, kb)), uel(G.mat, l, D, c, b, kb), c3);
        });
    }
    // -i htau (xi c2 + c3)
    return cscal(g.htau, cmulmi(cadd(cscal((double)g.sig, c2), c3)));
}

// rhs of one element (a, b) of a bulk item; task 0 les (m >= 1), 1 tv, 2 ret
template <int D>
__device__ cplx u_rhs(const NgWeights& W, const Grid& g, const HermV& G, const HermV& S, int n, int task, int m, int a,
                      int b, int kb) {
    const int k = W.k, T = g.ntau, T1 = g.ntau + 1;
    if (task == 2) {  // retarded (B): -bdf/h - h i sum_l w Sigma^R(n,m+l) G^R(m+l,m)
        const int L = n - m;
        cplx acc = cz();
        greg_for(W, L, L - 1, [&](int l, double w) {
#pragma unroll
            for (int c = 0; c < D; ++c)
                acc = cfma(cscal(w, uel(S.ret, tri(n) + m + l, D, a, c, kb)), uel(G.ret, tri(m + l) + m, D, c, b, kb), acc);
        });
        cplx bdf = cz();
        for (int l = 1; l <= k; ++l) bdf = cadd(bdf, cscal(W.a[l], uel(G.ret, tri(n - l) + m, D, a, b, kb)));
        return csub(cscal(-1.0 / g.h, bdf), cscal(g.h, cmuli(acc)));
    }
    if (task == 1) {  // left-mixing: q - bdf/h - h i sum_j w Sigma^R(n,j) G^tv(j,m)
        cplx acc = cz();
        greg_for(W, n, n - 1, [&](int j, double w) {
#pragma unroll
            for (int c = 0; c < D; ++c)
                acc = cfma(cscal(w, uel(S.ret, tri(n) + j, D, a, c, kb)), uel(G.tv, (int64_t)j * T1 + m, D, c, b, kb), acc);
        });
        cplx bdf = cz();
        for (int l = 1; l <= k; ++l) bdf = cadd(bdf, cscal(W.a[l], uel(G.tv, (int64_t)(n - l) * T1 + m, D, a, b, kb)));
        cplx r = u_qtv<D>(W, g, G, S, n, m, a, b, kb);
        r = csub(r, cscal(1.0 / g.h, bdf));
        return csub(r, cscal(g.h, cmuli(acc)));
    }
    // lesser (B): q - bdf/h + h i hist, q = i h C1 - xi htau C3
    cplx c1 = cz();
    if (m <= k) {
        for (int j = 0; j <= k; ++j)
#pragma unroll
            for (int c = 0; c < D; ++c)
                c1 = cfma(cscal(W.greg[m][j], uretx(G, m, j, D, a, c, kb)), uel(S.les, tri(n) + j, D, c, b, kb), c1);
    } else {
        greg_for(W, m, m, [&](int j, double w) {
#pragma unroll
            for (int c = 0; c < D; ++c)
                c1 = cfma(cscal(w, uel(G.ret, tri(m) + j, D, a, c, kb)), uel(S.les, tri(n) + j, D, c, b, kb), c1);
        });
    }
    cplx c3 = cz();   // sum_j w G^tv(m,j) [Sigma^tv(n,T-j)]^dagger
    greg_for(W, T, T, [&](int j, double w) {
#pragma unroll
        for (int c = 0; c < D; ++c)
            c3 = cfma(cscal(w, uel(G.tv, (int64_t)m * T1 + j, D, a, c, kb)),
                      cconj(uel(S.tv, (int64_t)n * T1 + T - j, D, b, c, kb)), c3);
    });
    cplx hist = cz();  // sum_l w G^<(m,l) [Sigma^R(n,l)]^dagger
    greg_for(W, n, n - 1, [&](int l, double w) {
#pragma unroll
        for (int c = 0; c < D; ++c) {
            cplx gl = (l >= m) ? uel(G.les, tri(l) + m, D, a, c, kb) : cneg(cconj(uel(G.les, tri(m) + l, D, c, a, kb)));
            hist = cfma(cscal(w, gl), cconj(uel(S.ret, tri(n) + l, D, b, c, kb)), hist);
        }
    });
    cplx bdf = cz();
    for (int l = 1; l <= k; ++l) bdf = cadd(bdf, cscal(W.a[l], uel(G.les, tri(n - l) + m, D, a, b, kb)));
    cplx q = csub(cscal(g.h, cmuli(c1)), cscal((double)g.sig * g.htau, c3));
    cplx r = csub(q, cscal(1.0 / g.h, bdf));
    return cadd(r, cscal(g.h, cmuli(hist)));
}

template <int D>
__device__ __forceinline__ void u_bulk_block(const UProb& P, int n, int lblk, int nles, int ntv, int* status) {
    const NgWeights& W = c_W[P.g.k - 1];
    constexpr int DD = D * D;
    const int ipb = blockDim.x / DD;  // items per block
    int task, base;
    if (lblk < nles) { task = 0; base = lblk; }
    else if (lblk < nles + ntv) { task = 1; base = lblk - nles; }
    else { task = 2; base = lblk - nles - ntv; }
    const int t = threadIdx.x;
    const int li = t / DD, ab = t % DD, a = ab / D, b = ab % D;
    const int col = base * ipb + li;
    const int k = W.k;
    int ncol, m;
    if (task == 0) { ncol = n - k - 1; m = col + 1; }
    else if (task == 1) { ncol = P.g.ntau + 1; m = col; }
    else { ncol = n - k; m = col; }
    const bool valid = (li < ipb) && (col < ncol);
    extern __shared__ cplx rhs[];   // blockDim.x entries
    cplx r = cz();
    if (valid) r = u_rhs<D>(W, P.g, P.G, P.S, n, task, m, a, b, P.kb);
    if (t < ipb * DD) rhs[t] = r;
    __syncthreads();
    if (!valid) return;
    const cplx* rr = rhs + li * DD;
    cplx y = cz();
    if (task == 0) {  // y = rhs (M_n^dagger)^-1 = rhs (M_n^-1)^dagger: y_ab = sum_c rhs_ac conj(Minv_bc)
#pragma unroll
        for (int c = 0; c < D; ++c) y = cfma(rr[a * D + c], cconj(P.minv[b * D + c]), y);
    } else {          // y = M_n^-1 rhs
#pragma unroll
        for (int c = 0; c < D; ++c) y = cfma(P.minv[a * D + c], rr[c * D + b], y);
    }
    if (!cfinite(y)) atomicOr(status, NGF_NONFINITE);
    const Comp& dst = task == 0 ? P.G.les : (task == 1 ? P.G.tv : P.G.ret);
    const int64_t e = task == 0 ? tri(n) + m : (task == 1 ? (int64_t)n * (P.g.ntau + 1) + m : tri(n) + m);
    ust(dst, e, D, a, b, P.kb, y);
}

__global__ void __launch_bounds__(256) k_ubulk(const UProb* probs, UTable tab, int* status) {
    // find the problem of this block (tables are short)
    int i = 0;
    while (i + 1 < tab.np && (int)blockIdx.x >= tab.start[i + 1]) ++i;
    const UProb& P = probs[tab.prob[i]];
    const int lblk = blockIdx.x - tab.start[i];
    switch (P.g.nf) {
        case 1: u_bulk_block<1>(P, tab.n, lblk, tab.nles[i], tab.ntv[i], status); break;
        case 2: u_bulk_block<2>(P, tab.n, lblk, tab.nles[i], tab.ntv[i], status); break;
        case 4: u_bulk_block<4>(P, tab.n, lblk, tab.nles[i], tab.ntv[i], status); break;
        default: u_bulk_block<8>(P, tab.n, lblk, tab.nles[i], tab.ntv[i], status); break;
    }
}

// ---------------------------------------------------------------------------------------
// boundary of step n for every active problem: one block per problem, runtime D <= 8
// ---------------------------------------------------------------------------------------
#define NG_UBND_THREADS 128
#define NG_UBND_SMEM                                                                                  \
    (sizeof(cplx) * ((NG_KMAX * NG_UMAXD) * (NG_KMAX * NG_UMAXD) + (NG_KMAX * NG_UMAXD) * NG_UMAXD + \
                     NG_UBND_THREADS + 2 * (2 * NG_KMAX + 1) * NG_UMAXD * NG_UMAXD))

// -i (C^<_2 + C^<_3)[Sigma,1,G](m,n) element (a,b), partial over the summation indices
// i = i0, i0+is, ... < i1 of the concatenated range: i <= jmax is the C^<_2 term j = i, the
// rest the C^<_3 term j = i - jmax - 1 (jmax = max(n, k))
__device__ cplx u_qlesA_range(const NgWeights& W, const Grid& g, const HermV& G, const HermV& S, int m, int n, int D,
                              int a, int b, int kb, int i0, int i1, int is) {
    const int k = W.k, T = g.ntau, T1 = g.ntau + 1;
    cplx c2 = cz(), c3 = cz();
    const int jmax = n <= k ? k : n;
    for (int i = i0; i < i1; i += is) {
        if (i <= jmax) {
            const int j = i;
            const double w = n <= k ? W.greg[n][j] : gw(W, n, j);
            for (int c = 0; c < D; ++c)   // Sigma^<(m,j) G^A(j,n), G^A(j,n)_cb = conj(G~^R(n,j)_bc)
                c2 = cfma(cscal(w, ules(S, m, j, D, a, c, kb)), cconj(uretx(G, n, j, D, b, c, kb)), c2);
        } else {
            const int j = i - jmax - 1;
            const double w = gw(W, T, j);
            for (int c = 0; c < D; ++c)   // Sigma^tv(m,j) [G^tv(n,T-j)]^dagger
                c3 = cfma(cscal(w, uel(S.tv, (int64_t)m * T1 + j, D, a, c, kb)),
                          cconj(uel(G.tv, (int64_t)n * T1 + T - j, D, b, c, kb)), c3);
        }
    }
    return cadd(cscal(g.h, cmulmi(c2)), cscal((double)g.sig * g.htau, c3));
}

// M_m = a_0/h + i(eps_m - mu) + h w_{m,m} i Sigma^R(m,m) into out[D*D]
__device__ void u_stepmat(const NgWeights& W, const UProb& P, int m, cplx* out) {
    const int D = P.g.nf;
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) {
            cplx e = ufunc(P.eps, m, D, a, b, P.kb);
            if (a == b) e.x -= P.g.mu;
            cplx v = cadd(cmuli(e), cscal(P.g.h * gw(W, m, m), cmuli(uel(P.S.ret, tri(m) + m, D, a, b, P.kb))));
            if (a == b) v.x += W.a[0] / P.g.h;
            out[a * D + b] = v;
        }
}

// The boundary of step n runs in three launches: k_uboundary_ret (retarded (A) start-up along
// row n and G^<(0,n), one block per problem), k_usrc (sources and partial histories of the
// lesser (A) rows, O((k+1)(n + ntau) nf^3) per problem, over many blocks), k_uboundary_les (the
// serial lesser (A) steps, one block per problem).  The dense solves run on one warp
// (warp_dense_solve) and the step matrices of the serial rows are inverted by the block's warps
// before the serial chain, whose steps are then element-parallel products: FP64 is issued per
// warp instruction on this part, so one thread doing them alone took as long as a whole warp.
__global__ void __launch_bounds__(NG_UBND_THREADS) k_uboundary_ret(const UProb* probs, UTable tab, int* status) {
    const UProb& P = probs[tab.prob[blockIdx.x]];
    const NgWeights& W = c_W[P.g.k - 1];
    const Grid& g = P.g;
    const int D = g.nf, DD = D * D, k = W.k, n = tab.n, kb = P.kb, t = threadIdx.x;
    // dynamic shared memory (NG_UBND_SMEM bytes): A[(kD)^2], B[kD x D], ...
    extern __shared__ unsigned char ub_smem[];
    cplx* A = reinterpret_cast<cplx*>(ub_smem);
    cplx* B = A + (NG_KMAX * NG_UMAXD) * (NG_KMAX * NG_UMAXD);
    const int N = k * D;
    // ---- retarded start-up along row n (conjugate VIDE, implementation (A)) ----------
    // transposed system: rows (j, a), columns (l, b): A = Mh[l][j]^T, B = -(y0 Mh[0][j])^T
    for (int q = t; q < k * (k + 1) * DD; q += blockDim.x) {
        const int j = 1 + q / ((k + 1) * DD), rem = q % ((k + 1) * DD), l = rem / DD, ab = rem % DD;
        const int a = ab / D, b = ab % D;
        // Mh[l][j]_{ba} = D_{j,l}/h delta_ba + delta_lj i(eps_{n-j} - mu)_ba + h s_{j,l} i Sigma~^R(n-l, n-j)_ba
        cplx v = cscal(g.h * W.greg[j][l], cmuli(uretx(P.S, n - l, n - j, D, b, a, kb)));
        if (a == b) v.x += W.D[j][l] / g.h;
        if (l == j) {
            cplx e = ufunc(P.eps, n - j, D, b, a, kb);
            if (a == b) e.x -= g.mu;
            v = cadd(v, cmuli(e));
        }
        if (l > 0) A[((j - 1) * D + a) * N + (l - 1) * D + b] = v;
    }
    // right-hand side from Mh[0][j]_{ca}
    for (int q = t; q < k * DD; q += blockDim.x) {
        const int j = 1 + q / DD, ab = q % DD, a = ab / D, c = ab % D;
        cplx v = cscal(g.h * W.greg[j][0], cmuli(uretx(P.S, n, n - j, D, c, a, kb)));
        if (a == c) v.x += W.D[j][0] / g.h;
        // -(y0 Mh[0][j])^T_{a c} = -(-i Mh[0][j]_{c a}) = i Mh[0][j]_{ca}
        B[((j - 1) * D + a) * D + c] = cmuli(v);
    }
    __syncthreads();
    if (t < 32 && warp_dense_solve(A, N, B, D, B + (NG_KMAX * NG_UMAXD) * NG_UMAXD, t) && t == 0)
        atomicOr(status, NGF_SINGULAR);
    __syncthreads();
    for (int q = t; q < (k + 1) * DD; q += blockDim.x) {
        const int l = q / DD, ab = q % DD, c = ab / D, a = ab % D;   // y_l[c][a] = B[((l-1)D + a)][c]
        cplx y = (l == 0) ? cr(0.0) : B[((l - 1) * D + a) * D + c];
        if (l == 0) y = (c == a) ? make_double2(0.0, -1.0) : cz();
        if (!cfinite(y)) atomicOr(status, NGF_NONFINITE);
        ust(P.G.ret, tri(n) + n - l, D, c, a, kb, y);
    }
    for (int q = t; q < DD; q += blockDim.x) {   // G^<(0,n) = -[G^tv(n,0)]^dagger
        const int a = q / D, b = q % D;
        ust(P.G.les, tri(n) + 0, D, a, b, kb, cneg(cconj(uel(P.G.tv, (int64_t)n * (g.ntau + 1), D, b, a, kb))));
    }
}

// Sources q_A(m,n) and partial histories sum_{l<m0} w_{m,l} Sigma^R(m,l) G^<(l,n) of the (A) rows
// of every active problem, spread over blocks (chunk, row, problem); within a block, groups of
// D^2 threads take the summation indices in turn and are combined in a fixed order.
__global__ void __launch_bounds__(NG_USRC_THREADS) k_usrc(const UProb* probs, UTable tab) {
    const int i = blockIdx.z, r = blockIdx.y, ch = blockIdx.x;
    const UProb& P = probs[tab.prob[i]];
    const NgWeights& W = c_W[P.g.k - 1];
    const Grid& g = P.g;
    const int D = g.nf, DD = D * D, k = W.k, n = tab.n, kb = P.kb, t = threadIdx.x;
    const bool full = (n <= 2 * k);
    const int m0 = full ? 1 : n - k;
    const int nq = n - m0 + 1;
    if (r >= nq) return;
    const int m = m0 + r;
    const int jmax = n <= k ? k : n;
    const int nsum = jmax + 1 + g.ntau + 1;
    const int i0 = ch * tab.chunk, i1 = min(nsum, i0 + tab.chunk);
    const int ngrp = NG_USRC_THREADS / DD, grp = t / DD, ab = t % DD, a = ab / D, b = ab % D;
    __shared__ cplx red[2][NG_USRC_THREADS];
    cplx qv = cz(), hv = cz();
    if (grp < ngrp && i0 < i1) {
        qv = u_qlesA_range(W, g, P.G, P.S, m, n, D, a, b, kb, i0 + grp, i1, ngrp);
        if (!full && m > k)
            for (int l = i0 + grp; l < min(i1, m0); l += ngrp)
                for (int c = 0; c < D; ++c)
                    hv = cfma(cscal(gw(W, m, l), uel(P.S.ret, tri(m) + l, D, a, c, kb)),
                              uel(P.G.les, tri(n) + l, D, c, b, kb), hv);
    }
    red[0][t] = qv;
    red[1][t] = hv;
    __syncthreads();
    if (t < DD) {
        cplx sq = cz(), sh = cz();
        for (int gi = 0; gi < ngrp; ++gi) {
            sq = cadd(sq, red[0][gi * DD + t]);
            sh = cadd(sh, red[1][gi * DD + t]);
        }
        cplx* dst = tab.src + ((int64_t)((i * NG_MAXQ + r) * tab.nchunk + ch) * 2) * (NG_UMAXD * NG_UMAXD);
        dst[t] = sq;
        dst[NG_UMAXD * NG_UMAXD + t] = sh;
    }
}

__global__ void __launch_bounds__(NG_UBND_THREADS) k_uboundary_les(const UProb* probs, UTable tab, int* status) {
    const UProb& P = probs[tab.prob[blockIdx.x]];
    const NgWeights& W = c_W[P.g.k - 1];
    const Grid& g = P.g;
    const int D = g.nf, DD = D * D, k = W.k, n = tab.n, kb = P.kb, t = threadIdx.x;
    // dynamic shared memory (NG_UBND_SMEM bytes): A[(kD)^2], B[kD x D], red[threads] (pivot
    // factors, then the step's right-hand side), qs/hs[(2k+1) x D^2] (sources and partial
    // histories of the (A) rows)
    extern __shared__ unsigned char ub_smem[];
    cplx* A = reinterpret_cast<cplx*>(ub_smem);
    cplx* B = A + (NG_KMAX * NG_UMAXD) * (NG_KMAX * NG_UMAXD);
    cplx* red = B + (NG_KMAX * NG_UMAXD) * NG_UMAXD;
    cplx(*qs)[NG_UMAXD * NG_UMAXD] = reinterpret_cast<cplx(*)[NG_UMAXD * NG_UMAXD]>(red + NG_UBND_THREADS);
    cplx(*hs)[NG_UMAXD * NG_UMAXD] = qs + (2 * NG_KMAX + 1);
    const int N = k * D;
    // ---- lesser column: rows by (A) ----------------------------------------------------
    const bool full = (n <= 2 * k);
    const int m0 = full ? 1 : n - k;
    const int nq = n - m0 + 1;
    // sources and partial histories: chunk partials of k_usrc summed in chunk order
    for (int q = t; q < nq * DD; q += blockDim.x) {
        const int r = q / DD, ab = q % DD;
        const cplx* src = tab.src + ((int64_t)(blockIdx.x * NG_MAXQ + r) * tab.nchunk * 2) * (NG_UMAXD * NG_UMAXD);
        cplx sq = cz(), sh = cz();
        for (int ch = 0; ch < tab.nchunk; ++ch) {
            sq = cadd(sq, src[(2 * ch) * (NG_UMAXD * NG_UMAXD) + ab]);
            sh = cadd(sh, src[(2 * ch + 1) * (NG_UMAXD * NG_UMAXD) + ab]);
        }
        qs[r][ab] = sq;
        hs[r][ab] = sh;
    }
    __syncthreads();
    int mstep = m0;
    if (full) {   // VIDE start-up for m = 1..k: the blocks (m, l) and right-hand sides, then one solve
        for (int q = t; q < k * k * DD; q += blockDim.x) {
            const int m = 1 + q / (k * DD), rem = q % (k * DD), l = 1 + rem / DD, ab = rem % DD;
            const int aa = ab / D, bb = ab % D;
            cplx v = cscal(g.h * W.greg[m][l], cmuli(uretx(P.S, m, l, D, aa, bb, kb)));
            if (aa == bb) v.x += W.D[m][l] / g.h;
            if (l == m) {
                cplx e = ufunc(P.eps, m, D, aa, bb, kb);
                if (aa == bb) e.x -= g.mu;
                v = cadd(v, cmuli(e));
            }
            A[((m - 1) * D + aa) * N + (l - 1) * D + bb] = v;
        }
        for (int q = t; q < k * DD; q += blockDim.x) {   // q_m - M[m][0] y0, element (aa, cc)
            const int m = 1 + q / DD, ab = q % DD, aa = ab / D, cc = ab % D;
            cplx acc = qs[m - 1][ab];
            for (int bb = 0; bb < D; ++bb) {
                cplx v = cscal(g.h * W.greg[m][0], cmuli(uretx(P.S, m, 0, D, aa, bb, kb)));
                if (aa == bb) v.x += W.D[m][0] / g.h;
                acc = csub(acc, cmul(v, uel(P.G.les, tri(n), D, bb, cc, kb)));
            }
            B[((m - 1) * D + aa) * D + cc] = acc;
        }
        __syncthreads();
        if (t < 32 && warp_dense_solve(A, N, B, D, red, t) && t == 0) atomicOr(status, NGF_SINGULAR);
        __syncthreads();
        for (int q = t; q < k * DD; q += blockDim.x) {
            const int m = 1 + q / DD, ab = q % DD, aa = ab / D, cc = ab % D;
            ust(P.G.les, tri(n) + m, D, aa, cc, kb, B[((m - 1) * D + aa) * D + cc]);
        }
        mstep = k + 1;
        __syncthreads();
    }
    // inverse step matrices of the rows m = mstep..n, one warp per row (A is free now):
    // Mi[r] at A + r D^2, the warps' scratch (M, X, pivot factors) after them
    cplx* Mi = A;
    const int warp = t >> 5, lane = t & 31, nwarp = blockDim.x >> 5;
    cplx* Mw = A + (2 * NG_KMAX + 1) * NG_UMAXD * NG_UMAXD + warp * (2 * NG_UMAXD * NG_UMAXD + NG_UMAXD);
    cplx* Xw = Mw + NG_UMAXD * NG_UMAXD;
    cplx* fw = Xw + NG_UMAXD * NG_UMAXD;
    for (int m = mstep + warp; m <= n; m += nwarp) {
        for (int i = lane; i < DD; i += 32) {
            const int aa = i / D, bb = i % D;
            cplx e = ufunc(P.eps, m, D, aa, bb, kb);
            if (aa == bb) e.x -= g.mu;
            cplx v = cadd(cmuli(e), cscal(g.h * gw(W, m, m), cmuli(uel(P.S.ret, tri(m) + m, D, aa, bb, kb))));
            if (aa == bb) v.x += W.a[0] / g.h;
            Mw[i] = v;
            Xw[i] = cr(aa == bb ? 1.0 : 0.0);
        }
        __syncwarp();
        if (warp_dense_solve(Mw, D, Xw, D, fw, lane) && lane == 0) atomicOr(status, NGF_SINGULAR);
        for (int i = lane; i < DD; i += 32) Mi[(m - m0) * DD + i] = Xw[i];
        __syncwarp();
    }
    __syncthreads();
    // serial VIDE steps: thread (grp, ab) sums element ab of the history and BDF terms
    // l = grp, grp + ngr, ...; the group partials (in B) are added in group order
    const int ngr = blockDim.x / DD, grp = t / DD, ab = t % DD, aa = ab / D, bb = ab % D;
    cplx* part = B;            // 2 ngr DD <= 2 blockDim.x values
    cplx* accv = red;          // DD values
    const int lfrom = full ? 0 : m0;
    for (int m = mstep; m <= n; ++m) {
        const int r = m - m0;
        if (grp < ngr) {
            cplx hsum = cz(), bdf = cz();
            for (int l = lfrom + grp; l < m; l += ngr) {
                const double w = gw(W, m, l);
                for (int cc = 0; cc < D; ++cc)
                    hsum = cfma(cscal(w, uel(P.S.ret, tri(m) + l, D, aa, cc, kb)), uel(P.G.les, tri(n) + l, D, cc, bb, kb), hsum);
            }
            for (int l = 1 + grp; l <= k; l += ngr) bdf = cadd(bdf, cscal(W.a[l], uel(P.G.les, tri(n) + m - l, D, aa, bb, kb)));
            part[grp * DD + ab] = hsum;
            part[(ngr + grp) * DD + ab] = bdf;
        }
        __syncthreads();
        if (t < DD) {
            cplx hsum = hs[r][t], bdf = cz();
            for (int q = 0; q < ngr; ++q) {
                hsum = cadd(hsum, part[q * DD + t]);
                bdf = cadd(bdf, part[(ngr + q) * DD + t]);
            }
            accv[t] = csub(csub(qs[r][t], cscal(1.0 / g.h, bdf)), cscal(g.h, cmuli(hsum)));
        }
        __syncthreads();
        if (t < DD) {
            cplx y = cz();
            for (int cc = 0; cc < D; ++cc) y = cfma(Mi[r * DD + aa * D + cc], accv[cc * D + bb], y);
            if (!cfinite(y)) atomicOr(status, NGF_NONFINITE);
            ust(P.G.les, tri(n) + m, D, aa, bb, kb, y);
        }
        __syncthreads();
    }
}
