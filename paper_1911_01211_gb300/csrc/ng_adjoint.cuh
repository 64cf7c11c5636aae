// Discrete adjoint (reverse mode) of the second-Born time stepping for one orbital (nf = 1).
//
// The forward algorithm is the executed one: predictor (polynomial extrapolation, Eq.
// polyextrap), then `corrector` passes of {k-reduction, Hartree mean field, second-Born
// slice (Eq. sigma_hubb_2b), Dyson time step} per step n > k (Sec. "Time stepping", mixed
// schedule), after the bootstrapped start slices 0..k (Sec. "Start").  Its adjoint runs the
// steps backwards; each Dyson step is linear in the history for a fixed self-energy, so its
// transpose scatters the cotangent of slice n into the history cotangents with the same
// Gregory/BDF weights and gathers the cotangent of the self-energy slice.
//
// Cotangent convention: for a complex quantity z and the real loss L, c(z) = dL/dRe z +
// i dL/dIm z.  Then y = a z gives c(z) += conj(a) c(y), y = conj(z) gives c(z) += conj(c(y)),
// and y = x z gives c(x) += conj(z) c(y), c(z) += conj(x) c(y).
//
// Storage (d = 1): per-k arrays have the problem index innermost (stride nb), shared ones
// (Sigma, G_loc) have ldk = 1.  A slice view holds the ret row n, the les column n and the tv
// row n of one time step.
#pragma once

#include "ng_step.cuh"
#include "ng_adjoint_types.h"

// ---- accessors -----------------------------------------------------------------------
__device__ __forceinline__ cplx adj_sigR(const AdjStep& a, int m, int l) {   // Sigma^R(m,l), l <= m <= n
    return m == a.n ? a.Sc.ret[l] : a.Sr[tri(m) + l];
}
__device__ __forceinline__ cplx adj_sigRx(const AdjStep& a, int p, int q) {  // Sigma~^R(p,q), continued
    if (q <= p) return adj_sigR(a, p, q);
    return cneg(cconj(adj_sigR(a, q, p)));
}
__device__ __forceinline__ cplx adj_sigL(const AdjStep& a, int m, int j) {   // Sigma^<(m,j), any m,j <= n
    if (m <= j) return j == a.n ? a.Sc.les[m] : a.Sl[tri(j) + m];
    return cneg(cconj(m == a.n ? a.Sc.les[j] : a.Sl[tri(m) + j]));
}
__device__ __forceinline__ cplx adj_sigT(const AdjStep& a, int m, int j) {   // Sigma^tv(m, tau_j)
    return m == a.n ? a.Sc.tv[j] : a.St[(int64_t)m * (a.g.ntau + 1) + j];
}
__device__ __forceinline__ cplx adj_mf(const AdjStep& a, int m, int kb) {
    return m == a.n ? a.mfc[kb] : a.mf[(int64_t)(m + 1) * a.g.nb + kb];
}
// *p += v (one writer per target: the callers map every contribution to its stored element)
__device__ __forceinline__ void cacc_to(cplx* p, cplx v) { *p = cadd(*p, v); }

// warp sum in a fixed butterfly order
__device__ __forceinline__ cplx warp_sum(cplx v) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}
// block sum (blockDim.x a multiple of 32, <= 1024), fixed order; valid in every thread
__device__ cplx block_csum(cplx v, cplx* sh /* >= 32 */) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    cplx r = cz();
    for (int w = 0; w < nw; ++w) r = cadd(r, sh[w]);
    __syncthreads();
    return r;
}

// ======================================================================================
// 1. lesser (A) rows m = n .. mstep in reverse, then the start-up block when n <= 2k.
//    One block per problem.  Forward: M_m G^<(m,n) = q_A(m) - (1/h) sum_l a_l G^<(m-l,n)
//    - h sum_{l<m} w_{m,l} i Sigma^R(m,l) G^<(l,n).
// ======================================================================================
__global__ void __launch_bounds__(128) k_adj_lesA(AdjStep a) {
    const NgWeights& W = c_W[a.g.k - 1];
    const int k = W.k, n = a.n, nb = a.g.nb, kb = blockIdx.x, t = threadIdx.x;
    const double h = a.g.h;
    __shared__ cplx sc;
    cplx* cwl = a.cw.les;
    const int mstep = a.full ? k + 1 : n - k;
    for (int m = n; m >= mstep; --m) {
        if (t == 0) {
            cplx e = adj_mf(a, m, kb);
            e.x -= a.g.mu;
            cplx M = cadd(cr(W.a[0] / h), cmuli(e));
            M = cadd(M, cscal(h * gw(W, m, m), cmuli(adj_sigR(a, m, m))));
            const cplx cacc = cmul(cconj(cdiv(cr(1.0), M)), cwl[(int64_t)m * nb + kb]);
            a.cA[(int64_t)(m - a.m0) * nb + kb] = cacc;
            // c(eps_m) += -i c(M_m),  c(M_m) = -conj(G^<(m,n)) cacc
            const cplx dm = cmuli(cmul(cconj(a.Gc.les[(int64_t)m * nb + kb]), cacc));
            if (m == n) a.cmfw[kb] = cadd(a.cmfw[kb], dm);
            else a.cmf[(int64_t)(m + 1) * nb + kb] = cadd(a.cmf[(int64_t)(m + 1) * nb + kb], dm);
            sc = cacc;
        }
        __syncthreads();
        const cplx cacc = sc;
        for (int l = t; l < m; l += blockDim.x) {
            // i h w_{m,l} conj(Sigma^R(m,l)) cacc, plus the BDF term
            cplx v = cmuli(cscal(h * gw(W, m, l), cmul(cconj(adj_sigR(a, m, l)), cacc)));
            if (l >= m - k) v = cadd(v, cscal(-W.a[m - l] / h, cacc));
            cwl[(int64_t)l * nb + kb] = cadd(cwl[(int64_t)l * nb + kb], v);
        }
        __syncthreads();
    }
    if (!a.full || t != 0) return;
    // start-up block m = 1..k (Eq. vdiff_start): sum_{l>=1} M_{m,l} y_l = q_m - M_{m,0} y_0,
    // M_{m,l} = D_{m,l}/h + h s_{m,l} i Sigma~^R(m,l) + delta_{ml} i(eps_m - mu)
    cplx AH[NG_KMAX * NG_KMAX], cb[NG_KMAX], M0[NG_KMAX + 1];
    for (int m = 1; m <= k; ++m) {
        cplx e = adj_mf(a, m, kb);
        e.x -= a.g.mu;
        for (int l = 0; l <= k; ++l) {
            cplx M = cadd(cr(W.D[m][l] / h), cscal(h * W.greg[m][l], cmuli(adj_sigRx(a, m, l))));
            if (l == m) M = cadd(M, cmuli(e));
            if (l == 0) M0[m] = M;
            else AH[(l - 1) * k + (m - 1)] = cconj(M);      // (A^H)[l][m] = conj(A[m][l])
        }
        cb[m - 1] = cwl[(int64_t)m * nb + kb];
    }
    dense_solve(AH, k, cb, 1);   // a singular system was flagged by the forward step
    cplx c0 = cz();
    for (int m = 1; m <= k; ++m) {
        a.cA[(int64_t)(m - a.m0) * nb + kb] = cb[m - 1];
        c0 = csub(c0, cmul(cconj(M0[m]), cb[m - 1]));
        const cplx dm = cmuli(cmul(cconj(a.Gc.les[(int64_t)m * nb + kb]), cb[m - 1]));
        a.cmf[(int64_t)(m + 1) * nb + kb] = cadd(a.cmf[(int64_t)(m + 1) * nb + kb], dm);
    }
    cwl[kb] = cadd(cwl[kb], c0);
}

// ======================================================================================
// 2. Per-problem parts of the (A) sources' transpose, q_A = -i h c2 + xi htau c3 with
//    c2 = sum_j w_{n,j} Sigma^<(m,j) conj(G^R(n,j)),  c3 = sum_j w_{T,j} Sigma^tv(m,j)
//    conj(G^tv(n,T-j)): cotangents of the current ret and tv rows; then G^<(0,n) =
//    -conj(G^tv(n,0)) (Eq. dyson_ini_les).  Thread per (j, problem).
// ======================================================================================
__global__ void k_adj_qA(AdjStep a) {
    const NgWeights& W = c_W[a.g.k - 1];
    const int n = a.n, nb = a.g.nb, T = a.g.ntau;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int kb = (int)(idx % nb), j = (int)(idx / nb);
    if (j > max(n, T)) return;
    const double h = a.g.h, ht = a.g.htau, xi = (double)a.g.sig;
    cplx accR = cz(), accT = cz();
    for (int r = 0; r < a.nq; ++r) {
        const int m = a.m0 + r;
        const cplx c = a.cA[(int64_t)r * nb + kb];
        if (j <= n) accR = cfma(cscal(gw(W, n, j), adj_sigL(a, m, j)), cconj(cmuli(cscal(h, c))), accR);
        if (j <= T) accT = cfma(cscal(gw(W, T, j), adj_sigT(a, m, j)), cconj(cscal(xi * ht, c)), accT);
    }
    if (j <= n) a.cw.ret[(int64_t)j * nb + kb] = cadd(a.cw.ret[(int64_t)j * nb + kb], accR);
    if (j <= T) {
        cplx* p = &a.cw.tv[(int64_t)(T - j) * nb + kb];
        *p = cadd(*p, accT);
        if (j == T) *p = csub(*p, cconj(a.cw.les[kb]));   // tv index 0
    }
}

// ======================================================================================
// 3. Shared cotangents of the (A) part, one warp per target, lanes over the problems:
//    group 0: Sigma^R(p,q), p in [m0,n], q <= p   (history term and M_m; start-up block)
//    group 1: Sigma^<(a,b), a in [m0,n], b in [a,n]
//    group 2: Sigma^<(a,b), a < m0, b in [m0,n]
//    group 3: Sigma^tv(m,j), m in [m0,n]
// ======================================================================================
__device__ __forceinline__ cplx* adj_tgt_ret(const AdjStep& a, int p, int q) {
    return p == a.n ? &a.cSw.ret[q] : &a.cSr[tri(p) + q];
}
__device__ __forceinline__ cplx* adj_tgt_les(const AdjStep& a, int x, int y) {   // Sigma^<(x,y), x <= y
    return y == a.n ? &a.cSw.les[x] : &a.cSl[tri(y) + x];
}
__device__ __forceinline__ cplx* adj_tgt_tv(const AdjStep& a, int m, int j) {
    return m == a.n ? &a.cSw.tv[j] : &a.cSt[(int64_t)m * (a.g.ntau + 1) + j];
}

__global__ void k_adj_sigA(AdjStep a, int width) {
    const NgWeights& W = c_W[a.g.k - 1];
    const int k = W.k, n = a.n, nb = a.g.nb, T = a.g.ntau;
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int grp = blockIdx.y;
    const int r = (int)(wid / width), q = (int)(wid % width);
    const double h = a.g.h, ht = a.g.htau, xi = (double)a.g.sig;
    if (grp == 0) {
        if (r >= a.nq) return;
        const int p = a.m0 + r;
        if (q > p) return;
        const bool sp = a.full && p <= k;                   // start-up row
        const double wd = sp ? W.greg[p][q] : gw(W, p, q);
        cplx s = cz(), s2 = cz();
        for (int kb = lane; kb < nb; kb += 32) {
            s = cfma(cconj(a.Gc.les[(int64_t)q * nb + kb]), a.cA[(int64_t)r * nb + kb], s);
            if (a.full && q >= 1 && q < p && p <= k)       // row q, continued index p > q
                s2 = cfma(cconj(a.Gc.les[(int64_t)p * nb + kb]), a.cA[(int64_t)(q - a.m0) * nb + kb], s2);
        }
        s = warp_sum(s);
        s2 = warp_sum(s2);
        if (lane == 0) {
            cplx v = cmuli(cscal(h * wd, s));
            if (a.full && q >= 1 && q < p && p <= k) v = csub(v, cconj(cmuli(cscal(h * W.greg[q][p], s2))));
            cacc_to(adj_tgt_ret(a, p, q), v);
        }
    } else if (grp == 1 || grp == 2) {
        int x, y;
        if (grp == 1) {
            if (r >= a.nq) return;
            x = a.m0 + r;
            y = q;
            if (y < x || y > n) return;
        } else {
            if (r >= a.nq || q >= a.m0) return;
            x = q;
            y = a.m0 + r;
        }
        // direct: row m = x, j = y (needs x in A rows); conjugate: row m = y, j = x < y
        const bool dir = (grp == 1);
        const bool cnj = (x < y);
        cplx s = cz(), s2 = cz();
        for (int kb = lane; kb < nb; kb += 32) {
            if (dir) s = cfma(a.Gc.ret[(int64_t)y * nb + kb], a.cA[(int64_t)(x - a.m0) * nb + kb], s);
            if (cnj) s2 = cfma(a.Gc.ret[(int64_t)x * nb + kb], a.cA[(int64_t)(y - a.m0) * nb + kb], s2);
        }
        s = warp_sum(s);
        s2 = warp_sum(s2);
        if (lane == 0) {
            cplx v = cz();
            if (dir) v = cmuli(cscal(h * gw(W, n, y), s));
            if (cnj) v = csub(v, cconj(cmuli(cscal(h * gw(W, n, x), s2))));
            cacc_to(adj_tgt_les(a, x, y), v);
        }
    } else {
        if (r >= a.nq || q > T) return;
        const int m = a.m0 + r;
        cplx s = cz();
        for (int kb = lane; kb < nb; kb += 32)
            s = cfma(a.Gc.tv[(int64_t)(T - q) * nb + kb], a.cA[(int64_t)r * nb + kb], s);
        s = warp_sum(s);
        if (lane == 0) cacc_to(adj_tgt_tv(a, m, q), cscal(gw(W, T, q) * xi * ht, s));
    }
}

// ======================================================================================
// 4. Per problem: cotangents of the (B) right-hand sides (ret columns, tv columns, lesser
//    rows), of M_n, and the retarded (A) block (Eq. MBCVSAMx_cc_start along row n).
// ======================================================================================
__global__ void __launch_bounds__(128) k_adj_bulk(AdjStep a) {
    const NgWeights& W = c_W[a.g.k - 1];
    const int k = W.k, n = a.n, nb = a.g.nb, T = a.g.ntau, kb = blockIdx.x, t = threadIdx.x;
    const double h = a.g.h;
    __shared__ cplx red[32];
    cplx e = a.mfc[kb];
    e.x -= a.g.mu;
    cplx M = cadd(cr(W.a[0] / h), cmuli(e));
    M = cadd(M, cscal(h * gw(W, n, n), cmuli(a.Sc.ret[n])));
    const cplx Minv = cdiv(cr(1.0), M);
    const cplx cMinvc = cconj(Minv);
    cplx cMi = cz();   // cotangent of M_n^-1
    for (int m = t; m <= n - k - 1; m += blockDim.x) {
        const cplx c = a.cw.ret[(int64_t)m * nb + kb];
        a.caccR[(int64_t)m * nb + kb] = cmul(cMinvc, c);
        cMi = cfma(cconj(cmul(a.Gc.ret[(int64_t)m * nb + kb], M)), c, cMi);    // conj(acc) c
    }
    for (int m = t; m <= T; m += blockDim.x) {
        const cplx c = a.cw.tv[(int64_t)m * nb + kb];
        a.caccT[(int64_t)m * nb + kb] = cmul(cMinvc, c);
        cMi = cfma(cconj(cmul(a.Gc.tv[(int64_t)m * nb + kb], M)), c, cMi);
    }
    if (!a.full)
        for (int m = 1 + t; m <= n - k - 1; m += blockDim.x) {
            const cplx c = a.cw.les[(int64_t)m * nb + kb];
            a.crhs[(int64_t)m * nb + kb] = cmul(Minv, c);
            // G^< = rhs conj(M^-1): c(M^-1) += rhs conj(c), rhs = G^< conj(M)
            cMi = cfma(cmul(a.Gc.les[(int64_t)m * nb + kb], cconj(M)), cconj(c), cMi);
        }
    cMi = block_csum(cMi, red);
    if (t != 0) return;
    const cplx cM = cneg(cmul(cconj(cmul(Minv, Minv)), cMi));
    a.cmfw[kb] = cadd(a.cmfw[kb], cmulmi(cM));
    a.cMn[kb] = cM;
    // retarded (A): y_l = G^R(n, n-l), y_0 = -i; sum_{l>=1} y_l Mh[l][j] = -y_0 Mh[0][j], j = 1..k,
    // Mh[l][j] = D_{j,l}/h + delta_{lj} i(eps_{n-j} - mu) + h s_{j,l} i Sigma~^R(n-l, n-j).
    // As A y = b with A[j][l] = Mh[l][j]:  c(b) = A^-H c(y), c(A) = -c(b) y^H.
    cplx AH[NG_KMAX * NG_KMAX], cb[NG_KMAX];
    for (int j = 1; j <= k; ++j)
        for (int l = 1; l <= k; ++l) {
            cplx Mh = cadd(cr(W.D[j][l] / h), cscal(h * W.greg[j][l], cmuli(adj_sigRx(a, n - l, n - j))));
            if (l == j) {
                cplx ej = adj_mf(a, n - j, kb);
                ej.x -= a.g.mu;
                Mh = cadd(Mh, cmuli(ej));
            }
            AH[(l - 1) * k + (j - 1)] = cconj(Mh);   // (A^H)[l][j] = conj(A[j][l]) = conj(Mh[l][j])
        }
    for (int l = 1; l <= k; ++l) cb[l - 1] = a.cw.ret[(int64_t)(n - l) * nb + kb];
    dense_solve(AH, k, cb, 1);
    const int K1 = k + 1;
    for (int j = 1; j <= k; ++j) {
        for (int l = 0; l <= k; ++l) {
            // c(Mh[l][j]): l >= 1: -c(b_j) conj(y_l); l = 0: b_j = i Mh[0][j] -> -i c(b_j)
            const cplx cMh = (l == 0) ? cmulmi(cb[j - 1])
                                      : cneg(cmul(cb[j - 1], cconj(a.Gc.ret[(int64_t)(n - l) * nb + kb])));
            // c(Sigma~^R(n-l, n-j)) += -i h s_{j,l} c(Mh)
            a.retA[(int64_t)(l * K1 + j) * nb + kb] = cmulmi(cscal(h * W.greg[j][l], cMh));
            if (l == j) {
                cplx* p = &a.cmf[(int64_t)(n - j + 1) * nb + kb];
                *p = cadd(*p, cmulmi(cMh));
            }
        }
    }
}

// ======================================================================================
// 5. History cotangents and the partial sums of the self-energy row / column cotangents.
// ======================================================================================
// The history kernels below run one block per history row (or column); each warp takes one
// index of the other time argument at a time and its lanes take the problems kb = lane,
// lane + 32, ..., so the weights and self-energy values of that index are warp-uniform and the
// per-problem arrays are read in contiguous 512-byte runs.

// tv history row j < n: tv step (all tau), BDF, and the C^<_3 source of the lesser (B) row j.
__global__ void __launch_bounds__(256) k_adj_tvrow(AdjStep a) {
    const NgWeights& W = c_W[a.g.k - 1];
    const int k = W.k, n = a.n, nb = a.g.nb, T = a.g.ntau, j = blockIdx.x;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int m0 = blockIdx.y * nw + wp, ms = nw * gridDim.y;   // this block's share of the row
    const double h = a.g.h, ht = a.g.htau, xi = (double)a.g.sig;
    __shared__ cplx red[32];
    const cplx coefA = cadd(cmuli(cscal(h * gw(W, n, j), cconj(a.Sc.ret[j]))),
                            cr(j >= n - k ? -W.a[n - j] / h : 0.0));
    const bool useB = !a.full && j >= 1 && j <= n - k - 1;
    const cplx* crj = a.crhs + (int64_t)j * nb;
    cplx acc = cz();
    for (int m = m0; m <= T; m += ms) {
        // w_{T,m} Sigma^tv(n, T-m) (-xi htau), multiplying crhs_j
        const cplx sB = useB ? cscal(-xi * ht * gw(W, T, m), a.Sc.tv[T - m]) : cz();
        const int64_t base = ((int64_t)j * (T + 1) + m) * nb;
        const cplx* cTm = a.caccT + (int64_t)m * nb;
#pragma unroll 4
        for (int kb = lane; kb < nb; kb += 32) {
            const cplx cT = cTm[kb];
            cplx v = cfma(coefA, cT, a.cGt[base + kb]);
            if (useB) v = cfma(sB, crj[kb], v);
            a.cGt[base + kb] = v;
            acc = cfma(cconj(a.Gt[base + kb]), cT, acc);
        }
    }
    acc = block_csum(acc, red);
    if (threadIdx.x == 0) a.part[(P_TVROW * NG_ADJ_SPLIT + blockIdx.y) * a.plen + j] = cmuli(cscal(h * gw(W, n, j), acc));
}

// tv column m: cotangent of Sigma^tv(n, T-m) from the C^<_3 sources of the lesser (B) rows
__global__ void __launch_bounds__(256) k_adj_tvcol(AdjStep a) {
    const NgWeights& W = c_W[a.g.k - 1];
    const int k = W.k, n = a.n, nb = a.g.nb, T = a.g.ntau, m = blockIdx.x;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int j0 = blockIdx.y * nw + wp, js = nw * gridDim.y;
    const double ht = a.g.htau, xi = (double)a.g.sig;
    __shared__ cplx red[32];
    cplx acc = cz();
    for (int j = 1 + j0; j <= n - k - 1; j += js) {
        const int64_t base = ((int64_t)j * (T + 1) + m) * nb;
        const cplx* crj = a.crhs + (int64_t)j * nb;
#pragma unroll 4
        for (int kb = lane; kb < nb; kb += 32) acc = cfma(a.Gt[base + kb], cconj(crj[kb]), acc);
    }
    acc = block_csum(acc, red);
    if (threadIdx.x == 0)
        a.part[(P_TVCOL * NG_ADJ_SPLIT + blockIdx.y) * a.plen + (T - m)] = cscal(-xi * ht * gw(W, T, m), acc);
}

// ret history row j < n: retarded (B) columns m <= n-k-1 (history term and BDF), and the
// C^<_1 source of the lesser (B) rows (row j itself, and rows m < j <= k through the
// modified retarded continuation).
__global__ void __launch_bounds__(256) k_adj_rrow(AdjStep a) {
    const NgWeights& W = c_W[a.g.k - 1];
    // rows in decreasing length (row j holds j + 1 entries): the longest are scheduled first
    const int k = W.k, n = a.n, nb = a.g.nb, j = gridDim.x - 1 - blockIdx.x;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int m0 = blockIdx.y * nw + wp, ms = nw * gridDim.y;
    const double h = a.g.h;
    __shared__ cplx red[32];
    const cplx sRc = cconj(a.Sc.ret[j]);
    const double bdf = (j >= n - k) ? -W.a[n - j] / h : 0.0;
    const bool rowB = !a.full && j >= 1 && j <= n - k - 1;
    const cplx* crj = a.crhs + (int64_t)j * nb;
    cplx acc = cz();
    for (int m = m0; m <= j; m += ms) {
        const int64_t base = (tri(j) + m) * nb;
        const bool colB = (m <= n - k - 1);
        const double w = colB ? gw(W, n - m, j - m) : 0.0;
        const cplx cR0 = cadd(cmuli(cscal(h * w, sRc)), cr(bdf));   // multiplies caccR_m
        // c1 of row j: w_{j,m} conj(Sigma^<(m,n)) (-i h) crhs_j
        const cplx c1 = rowB ? cmulmi(cscal(h * ((j > k) ? gw(W, j, m) : W.greg[j][m]), cconj(a.Sc.les[m]))) : cz();
        // row m < j <= k continued: -i h greg[m][j] Sigma^<(j,n) conj(crhs_m)
        const bool cont = !a.full && j <= k && m >= 1 && m < j && m <= n - k - 1;
        const cplx c2 = cont ? cmulmi(cscal(h * W.greg[m][j], a.Sc.les[j])) : cz();
        const cplx* cRm = a.caccR + (int64_t)m * nb;
        const cplx* crm = a.crhs + (int64_t)m * nb;
        cplx t = cz();   // sum over the problems of conj(G^R(j,m)) caccR_m, weighted once below
#pragma unroll 4
        for (int kb = lane; kb < nb; kb += 32) {
            cplx v = a.cGr[base + kb];
            if (colB) {
                const cplx cR = cRm[kb];
                v = cfma(cR0, cR, v);
                t = cfma(cconj(a.Gr[base + kb]), cR, t);
            }
            if (rowB) v = cfma(c1, crj[kb], v);
            if (cont) v = cfma(c2, cconj(crm[kb]), v);
            a.cGr[base + kb] = v;
        }
        acc = cadd(acc, cscal(w, t));
    }
    acc = block_csum(acc, red);
    if (threadIdx.x == 0) a.part[(P_RROW * NG_ADJ_SPLIT + blockIdx.y) * a.plen + j] = cmuli(cscal(h, acc));
}

// ret column b: cotangent of Sigma^<(b,n) from the C^<_1 sources of the lesser (B) rows
__global__ void __launch_bounds__(256) k_adj_rcol(AdjStep a) {
    const NgWeights& W = c_W[a.g.k - 1];
    const int k = W.k, n = a.n, nb = a.g.nb, b = blockIdx.x;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int a0 = blockIdx.y * nw + wp, as = nw * gridDim.y;
    const double h = a.g.h;
    __shared__ cplx red[32];
    cplx acc = cz();
    // rows ar >= max(1, b): R~(ar,b) = G^R(ar,b); rows 1 <= ar < b <= k: R~(ar,b) = -conj(G^R(b,ar))
    for (int ar = 1 + a0; ar <= n - k - 1; ar += as) {
        const bool dir = ar >= b;
        if (!dir && b > k) continue;
        const double w = (dir && ar > k) ? gw(W, ar, b) : W.greg[ar][b];
        const int64_t base = (dir ? tri(ar) + b : tri(b) + ar) * nb;
        const cplx* cra = a.crhs + (int64_t)ar * nb;
        // cc1 = -i h crhs:  dir: w conj(G^R(ar,b)) cc1;  continued: -w G^R(b,ar) cc1
        // (-i h applied once after the block sum, w once per row)
        cplx t = cz();
        if (dir) {
#pragma unroll 4
            for (int kb = lane; kb < nb; kb += 32) t = cfma(cconj(a.Gr[base + kb]), cra[kb], t);
        } else {
#pragma unroll 4
            for (int kb = lane; kb < nb; kb += 32) t = cfma(a.Gr[base + kb], cra[kb], t);
        }
        acc = cadd(acc, cscal(dir ? w : -w, t));
    }
    acc = block_csum(acc, red);
    if (threadIdx.x == 0) a.part[(P_RCOL * NG_ADJ_SPLIT + blockIdx.y) * a.plen + b] = cmulmi(cscal(h, acc));
}

// les history column b < n: history term and BDF of the lesser (B) rows; partial of
// Sigma^R(n,b) from rows m <= b
__global__ void __launch_bounds__(256) k_adj_lcol(AdjStep a) {
    const NgWeights& W = c_W[a.g.k - 1];
    // columns in decreasing length (column b holds b + 1 entries): the longest first
    const int k = W.k, n = a.n, nb = a.g.nb, b = gridDim.x - 1 - blockIdx.x;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int a0 = blockIdx.y * nw + wp, as = nw * gridDim.y;
    const double h = a.g.h;
    __shared__ cplx red[32];
    const double wb = gw(W, n, b);
    const double bdf = (b >= n - k) ? -W.a[n - b] / h : 0.0;
    const bool colB = b >= 1 && b <= n - k - 1;
    // -i h w_{n,b} Sigma^R(n,b) + bdf, multiplying crhs_ar
    const cplx c0 = cadd(cmulmi(cscal(h * wb, a.Sc.ret[b])), cr(bdf));
    const cplx* crb = a.crhs + (int64_t)b * nb;
    cplx acc = cz();
    for (int ar = a0; ar <= b; ar += as) {
        const int64_t base = (tri(b) + ar) * nb;
        const bool rowB = ar >= 1 && ar <= n - k - 1;
        const bool cnj = ar < b && colB;
        // row m = b, index l = ar < b:  -i h w_{n,ar} conj(Sigma^R(n,ar)) conj(crhs_b)
        const cplx c1 = cnj ? cmulmi(cscal(h * gw(W, n, ar), cconj(a.Sc.ret[ar]))) : cz();
        const cplx* cra = a.crhs + (int64_t)ar * nb;
#pragma unroll 4
        for (int kb = lane; kb < nb; kb += 32) {
            cplx v = a.cGl[base + kb];
            if (rowB) {
                const cplx cr_ = cra[kb];
                v = cfma(c0, cr_, v);
                acc = cfma(a.Gl[base + kb], cconj(cr_), acc);
            }
            if (cnj) v = cfma(c1, cconj(crb[kb]), v);
            a.cGl[base + kb] = v;
        }
    }
    acc = block_csum(acc, red);
    if (threadIdx.x == 0) a.part[(P_LCOL * NG_ADJ_SPLIT + blockIdx.y) * a.plen + b] = cmuli(cscal(h * wb, acc));
}

// les history row a: partial of Sigma^R(n,a) from the lesser (B) rows m > a
__global__ void __launch_bounds__(256) k_adj_lrow(AdjStep a) {
    const NgWeights& W = c_W[a.g.k - 1];
    const int k = W.k, n = a.n, nb = a.g.nb, ar = blockIdx.x;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int m0 = blockIdx.y * nw + wp, ms = nw * gridDim.y;
    const double h = a.g.h;
    __shared__ cplx red[32];
    cplx acc = cz();
    for (int m = max(ar + 1, 1) + m0; m <= n - k - 1; m += ms) {
        const int64_t base = (tri(m) + ar) * nb;
        const cplx* crm = a.crhs + (int64_t)m * nb;
        // G^<(m, a) = -conj(G^<(a, m))
#pragma unroll 4
        for (int kb = lane; kb < nb; kb += 32) acc = csub(acc, cconj(cmul(a.Gl[base + kb], crm[kb])));
    }
    acc = block_csum(acc, red);
    if (threadIdx.x == 0)
        a.part[(P_LROW * NG_ADJ_SPLIT + blockIdx.y) * a.plen + ar] = cmuli(cscal(h * gw(W, n, ar), acc));
}

// Matsubara source of the tv row, q = -i htau (C2 + C3) (Eqs. ctv2, ctv3): cotangent of
// Sigma^tv(n, tau_p), one block per p, sum over (m, problem).
__global__ void __launch_bounds__(256) k_adj_qtv(AdjStep a) {
    const NgWeights& W = c_W[a.g.k - 1];
    const int k = W.k, nb = a.g.nb, T = a.g.ntau, p = blockIdx.x;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int m0 = blockIdx.y * nw + wp, ms = nw * gridDim.y;
    const double ht = a.g.htau, xi = (double)a.g.sig;
    __shared__ cplx red[32];
    cplx acc = cz();
    for (int m = m0; m <= T; m += ms) {
        // C2 (with xi): m <= k: R[m][j][p] xi G^M(T-j), p <= k;  m > k: w_{m,m-p} xi G^M(T-m+p), p <= m
        // C3: m >= T-k: R[T-m][j][T-p] G^M(j), p >= T-k;  m < T-k: w_{T-m,p-m} G^M(p-m), p >= m
        const bool c2R = (m <= k) && (p <= k), c2G = (m > k) && (p <= m);
        const bool c3R = (m >= T - k) && (p >= T - k), c3G = (m < T - k) && (p >= m);
        if (!(c2R || c2G || c3R || c3G)) continue;
        const double w2 = c2G ? gw(W, m, m - p) * xi : 0.0, w3 = c3G ? gw(W, T - m, p - m) : 0.0;
        const cplx* cTm = a.caccT + (int64_t)m * nb;
        for (int kb = lane; kb < nb; kb += 32) {
            cplx w = cz();
            if (c2R)
                for (int j = 0; j <= k; ++j) w = cadd(w, cscal(W.R[m][j][p] * xi, cconj(a.Gm[(int64_t)(T - j) * nb + kb])));
            if (c2G) w = cadd(w, cscal(w2, cconj(a.Gm[(int64_t)(T - m + p) * nb + kb])));
            if (c3R)
                for (int j = 0; j <= k; ++j) w = cadd(w, cscal(W.R[T - m][j][T - p], cconj(a.Gm[(int64_t)j * nb + kb])));
            if (c3G) w = cadd(w, cscal(w3, cconj(a.Gm[(int64_t)(p - m) * nb + kb])));
            acc = cfma(w, cTm[kb], acc);
        }
    }
    acc = block_csum(acc, red);
    if (threadIdx.x == 0) a.part[(P_QTV * NG_ADJ_SPLIT + blockIdx.y) * a.plen + p] = cmuli(cscal(ht, acc));
}

// Current self-energy slice: add the partial sums, the M_n term and the retarded (A) block.
// Thread per target: ret slots 0..n, les slots 0..n, tv slots 0..T, then the (k+1)^2 entries
// of the retarded (A) block in history rows n-1..n-k.
__global__ void k_adj_cur(AdjStep a) {
    const NgWeights& W = c_W[a.g.k - 1];
    const int k = W.k, n = a.n, nb = a.g.nb, T = a.g.ntau, K1 = k + 1;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double h = a.g.h;
    // the NG_ADJ_SPLIT block partials of a history sum, added in split order
    auto part = [&](int which, int64_t idx) {
        cplx v = cz();
        for (int sp = 0; sp < NG_ADJ_SPLIT; ++sp) v = cadd(v, a.part[(which * NG_ADJ_SPLIT + sp) * a.plen + idx]);
        return v;
    };
    auto sumk = [&](int l, int j) {
        cplx s = cz();
        for (int kb = 0; kb < nb; ++kb) s = cadd(s, a.retA[(int64_t)(l * K1 + j) * nb + kb]);
        return s;
    };
    if (i <= n) {
        const int j = (int)i;
        cplx v = cz();
        if (j < n) {
            v = cadd(part(P_TVROW, j), part(P_RROW, j));
            if (!a.full) v = cadd(v, part(P_LCOL, j));
            if (!a.full && j <= n - k - 2) v = cadd(v, part(P_LROW, j));
            if (j >= n - k) v = cadd(v, sumk(0, n - j));   // retarded (A) block, row n
        } else {
            cplx s = cz();
            for (int kb = 0; kb < nb; ++kb) s = cadd(s, a.cMn[kb]);
            v = cmulmi(cscal(h * gw(W, n, n), s));
        }
        a.cSw.ret[j] = cadd(a.cSw.ret[j], v);
        return;
    }
    int64_t r = i - (n + 1);
    if (r <= n) {
        const int b = (int)r;
        if (!a.full && b <= n - k - 1) a.cSw.les[b] = cadd(a.cSw.les[b], part(P_RCOL, b));
        return;
    }
    r -= n + 1;
    if (r <= T) {
        const int p = (int)r;
        cplx v = part(P_QTV, p);
        if (!a.full) v = cadd(v, part(P_TVCOL, p));
        a.cSw.tv[p] = cadd(a.cSw.tv[p], v);
        return;
    }
    r -= T + 1;
    // retarded (A) block, history rows: target (n-x, n-y), 1 <= x <= y <= k
    if (r >= (int64_t)k * k) return;
    const int x = 1 + (int)(r / k), y = 1 + (int)(r % k);
    if (y < x) return;
    cplx v = sumk(x, y);                                   // l = x <= j = y
    if (y > x) v = csub(v, cconj(sumk(y, x)));             // l = y > j = x: continued
    cplx* p = &a.cSr[tri(n - x) + (n - y)];
    *p = cadd(*p, v);
}

// ======================================================================================
// 6. Second-Born slice (Eq. sigma_hubb_2b, d = 1) transposed at the G_loc slice of the
//    pass, and the Hartree term; thread per slice index.  Output: cotangent of G_loc slice.
//    Sigma^<(j,n) = u g<^2 g>,  Sigma^R(n,j) = u g>^2 g< + u conj(g<^2 g>),  g> = gR - conj(g<)
//    Sigma^tv(n,m) = -xi u' tv(m)^2 conj(tv(T-m))
// ======================================================================================
__global__ void k_adj_sigma2b(Grid g, int n, SliceV Lc /* ld 1 */, SliceV cS /* ld 1 */, const cplx* cmfw,
                              int ld_cmf, FuncV U, SliceV out /* ld 1 */) {
    const int T = g.ntau, nb = g.nb;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double xi = (double)g.sig;
    auto u = [&](int t) { return U.p[t + 1].x; };
    if (i <= n) {
        const int j = i;
        const double uu = u(n) * u(j);
        const cplx gl = Lc.les[j], gr = Lc.ret[j];
        const cplx gg = csub(gr, cconj(gl));
        const cplx cSL = cS.les[j], cSR = cS.ret[j];
        cplx cl = cmul(cconj(cscal(2.0 * uu, cmul(gl, gg))), cSL);
        cplx cg = cmul(cconj(cscal(uu, cmul(gl, gl))), cSL);
        cg = cfma(cconj(cscal(2.0 * uu, cmul(gg, gl))), cSR, cg);
        cl = cfma(cconj(cscal(uu, cmul(gg, gg))), cSR, cl);
        const cplx cP = cscal(uu, cconj(cSR));
        cl = cfma(cconj(cscal(2.0, cmul(gl, gg))), cP, cl);
        cg = cfma(cconj(cmul(gl, gl)), cP, cg);
        cl = csub(cl, cconj(cg));
        if (j == n) {   // Hartree: eps_mf(n) = eps0(n) + U_n (Im G_loc^<(n,n) - nbar)
            double s = 0.0;
            for (int kb = 0; kb < nb; ++kb) s += cmfw[(int64_t)kb * ld_cmf].x;
            cl = cadd(cl, cmuli(cr(u(n) * s)));
        }
        out.ret[j] = cg;
        out.les[j] = cl;
    }
    if (i <= T) {
        const int m = i;
        const double up = -xi * u(n) * u(-1);
        const cplx tvm = Lc.tv[m], tvr = Lc.tv[T - m];
        cplx c = cmul(cscal(2.0 * up, cmul(cconj(tvm), tvr)), cS.tv[m]);
        c = cfma(cscal(up, cmul(tvr, tvr)), cconj(cS.tv[T - m]), c);
        out.tv[m] = c;
    }
}

// eps0 cotangent of one step (real part of the eps_mf cotangent), thread per problem
__global__ void k_adj_ce0(int nb, const cplx* cmfw, int ld_cmf, double* ce0_row) {
    const int kb = blockIdx.x * blockDim.x + threadIdx.x;
    if (kb < nb) ce0_row[kb] += cmfw[(int64_t)kb * ld_cmf].x;
}

// per-problem slice cotangent = (shared slice cotangent)/nb, thread per (element, problem);
// also clears the shared cotangent of the next pass and the eps_mf cotangent
__global__ void k_adj_bcast(Grid g, int n, SliceV src, SliceV dst, SliceV sclear, cplx* cmfw) {
    const int nb = g.nb, T = g.ntau;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t len = 2 * (int64_t)(n + 1) + T + 1;
    if (i >= len * nb) return;
    const int kb = (int)(i % nb);
    const int e = (int)(i / nb);
    const double s = 1.0 / nb;
    if (e <= n) {
        dst.ret[(int64_t)e * nb + kb] = cscal(s, src.ret[e]);
        if (kb == 0) sclear.ret[e] = cz();
    } else if (e <= 2 * n + 1) {
        dst.les[(int64_t)(e - n - 1) * nb + kb] = cscal(s, src.les[e - n - 1]);
        if (kb == 0) sclear.les[e - n - 1] = cz();
    } else {
        const int m = e - 2 * (n + 1);
        dst.tv[(int64_t)m * nb + kb] = cscal(s, src.tv[m]);
        if (kb == 0) sclear.tv[m] = cz();
    }
    if (e == 0) cmfw[kb] = cz();
}

// copy a slice (ld = nb or 1) between two slice views; thread per (element, problem)
__global__ void k_slice_copy(int n, int T, int ld, SliceV src, SliceV dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t len = 2 * (int64_t)(n + 1) + T + 1;
    if (i >= len * ld) return;
    const int kb = (int)(i % ld);
    const int e = (int)(i / ld);
    if (e <= n) dst.ret[(int64_t)e * ld + kb] = src.ret[(int64_t)e * ld + kb];
    else if (e <= 2 * n + 1) dst.les[(int64_t)(e - n - 1) * ld + kb] = src.les[(int64_t)(e - n - 1) * ld + kb];
    else {
        const int m = e - 2 * (n + 1);
        dst.tv[(int64_t)m * ld + kb] = src.tv[(int64_t)m * ld + kb];
    }
}

// ======================================================================================
// 7. Predictor (Eq. polyextrap) transposed: slice n was extrapolated from slices n-1-l.
// ======================================================================================
// diagonals of ret and les and the tv rows: thread per (slice element, problem), loop over l
__global__ void k_adj_extrap_diag(Grid g, int n, SliceV cw, cplx* cGr, cplx* cGl, cplx* cGt) {
    const NgWeights& W = c_W[g.k - 1];
    const int k = W.k, nb = g.nb, T = g.ntau, Np = n - 1;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int nd = n - k;                  // ret diagonals jd = 0..n-k-1 (slice columns n-jd > k)
    const int nl = n - k;                  // les rows j = k+1..n
    const int64_t items = (int64_t)(nd + nl + T + 1) * nb;
    if (i >= items) return;
    const int kb = (int)(i % nb);
    int e = (int)(i / nb);
    if (e < nd) {
        const int jd = e;
        const cplx c = cw.ret[(int64_t)(n - jd) * nb + kb];
        for (int l = 0; l <= k; ++l) {
            const int r = Np - l;
            cplx* p = &cGr[(tri(r) + r - jd) * nb + kb];
            *p = cadd(*p, cscal(W.C[l], c));
        }
        return;
    }
    e -= nd;
    if (e < nl) {
        const int j = k + 1 + e, off = n - j;
        const cplx c = cw.les[(int64_t)j * nb + kb];
        for (int l = 0; l <= k; ++l) {
            const int col = Np - l;
            cplx* p = &cGl[(tri(col) + col - off) * nb + kb];
            *p = cadd(*p, cscal(W.C[l], c));
        }
        return;
    }
    e -= nl;
    const int m = e;
    const cplx c = cw.tv[(int64_t)m * nb + kb];
    for (int l = 0; l <= k; ++l) {
        cplx* p = &cGt[((int64_t)(Np - l) * (T + 1) + m) * nb + kb];
        *p = cadd(*p, cscal(W.C[l], c));
    }
}

// columns j <= k of ret and rows j <= k of les (with the hermitian continuation); thread per problem
__global__ void k_adj_extrap_cols(Grid g, int n, SliceV cw, cplx* cGr, cplx* cGl) {
    const NgWeights& W = c_W[g.k - 1];
    const int k = W.k, nb = g.nb, Np = n - 1;
    const int kb = blockIdx.x * blockDim.x + threadIdx.x;
    if (kb >= nb) return;
    for (int j = 0; j <= k; ++j) {
        const cplx cr_ = cw.ret[(int64_t)j * nb + kb], cl = cw.les[(int64_t)j * nb + kb];
        for (int l = 0; l <= k; ++l) {
            const int r = Np - l;
            const cplx vr = cscal(W.C[l], cr_), vl = cscal(W.C[l], cl);
            if (j <= r) {
                cGr[(tri(r) + j) * nb + kb] = cadd(cGr[(tri(r) + j) * nb + kb], vr);
                cGl[(tri(r) + j) * nb + kb] = cadd(cGl[(tri(r) + j) * nb + kb], vl);
            } else {
                cGr[(tri(j) + r) * nb + kb] = csub(cGr[(tri(j) + r) * nb + kb], cconj(vr));
                cGl[(tri(j) + r) * nb + kb] = csub(cGl[(tri(j) + r) * nb + kb], cconj(vl));
            }
        }
    }
}

// seed: c(G^<_k(n,n)) += seed[n][kb] for every n
__global__ void k_adj_seed(Grid g, const cplx* seed, cplx* cGl) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)(g.nt + 1) * g.nb) return;
    const int n = (int)(i / g.nb), kb = (int)(i % g.nb);
    cGl[(tri(n) + n) * g.nb + kb] = cadd(cGl[(tri(n) + n) * g.nb + kb], seed[i]);
}

// ======================================================================================
// 8. Start slices 0..k (Sec. "Start"): transpose of the start-up solves of one problem.
//    Compact slice layout of slices 0..k: ret (n,j) at tri(n)+j, les (j,n) at T3 + tri(n)+j,
//    tv (n,m) at 2 T3 + n (T+1) + m, T3 = tri(k+1); per-problem arrays have stride nb.
// ======================================================================================


__global__ void __launch_bounds__(NG_BOOT_THREADS) k_adj_start(AdjBoot b) {
    const NgWeights& W = c_W[b.g.k - 1];
    const int k = W.k, T = b.g.ntau, nb = b.g.nb, kb = blockIdx.x, t = threadIdx.x;
    const double h = b.g.h, ht = b.g.htau, xi = (double)b.g.sig;
    const int64_t T3 = tri(k + 1), E = boot_E(k, T);
    extern __shared__ cplx dsm[];
    cplx* c = dsm;                          // [E] local cotangent of the slices
    cplx* rt = c + E;                       // [k][T+1] tv right-hand-side cotangents
    __shared__ cplx red[32];
    __shared__ cplx M[NG_KMAX + 1][NG_KMAX + 1], cM[NG_KMAX + 1][NG_KMAX + 1];
    __shared__ cplx qsh[NG_KMAX + 1], crh[NG_KMAX + 1];
    auto GR = [&](int n, int j) { return b.Gr[(tri(n) + j) * nb + kb]; };
    auto GRx = [&](int n, int j) { return j <= n ? GR(n, j) : cneg(cconj(GR(j, n))); };
    auto GL = [&](int j, int n) { return b.Gl[(tri(n) + j) * nb + kb]; };
    auto GT = [&](int n, int m) { return b.Gt[((int64_t)n * (T + 1) + m) * nb + kb]; };
    auto GM = [&](int m) { return b.Gm[(int64_t)m * nb + kb]; };
    auto SR = [&](int n, int j) { return b.Sr[tri(n) + j]; };
    auto SRx = [&](int p, int q) { return q <= p ? SR(p, q) : cneg(cconj(SR(q, p))); };
    auto SL = [&](int m, int j) { return m <= j ? b.Sl[tri(j) + m] : cneg(cconj(b.Sl[tri(m) + j])); };
    auto ST = [&](int m, int j) { return b.St[(int64_t)m * (T + 1) + j]; };
    auto EPS = [&](int n) { cplx e = b.mf[(int64_t)(n + 1) * nb + kb]; e.x -= b.g.mu; return e; };
    auto cret = [&](int n, int j) -> cplx& { return c[tri(n) + j]; };
    auto cles = [&](int j, int n) -> cplx& { return c[T3 + tri(n) + j]; };
    auto ctv = [&](int n, int m) -> cplx& { return c[2 * T3 + (int64_t)n * (T + 1) + m]; };
    auto P = [&](int64_t e) -> cplx& { return b.Pk[e * nb + kb]; };
    auto Pret = [&](int p, int q, cplx v) {        // cotangent of Sigma~^R(p,q)
        if (q <= p) P(tri(p) + q) = cadd(P(tri(p) + q), v);
        else P(tri(q) + p) = csub(P(tri(q) + p), cconj(v));
    };
    auto Ples = [&](int m, int j, cplx v) {        // cotangent of Sigma^<(m,j)
        if (m <= j) P(T3 + tri(j) + m) = cadd(P(T3 + tri(j) + m), v);
        else P(T3 + tri(m) + j) = csub(P(T3 + tri(m) + j), cconj(v));
    };
    auto Ptv = [&](int m, int j) -> cplx& { return P(2 * T3 + (int64_t)m * (T + 1) + j); };
    auto cmf = [&](int n) -> cplx& { return b.cmfx[(int64_t)(n + 1) * nb + kb]; };

    for (int64_t e = t; e < E; e += blockDim.x) c[e] = b.mu[e * nb + kb];
    if (t == 0) {
        // shared start matrix M[n][l] = D_{n,l}/h + h s_{n,l} i Sigma~^R(n,l) + delta i(eps_n - mu)
        for (int n = 1; n <= k; ++n)
            for (int l = 0; l <= k; ++l) {
                cplx v = cadd(cr(W.D[n][l] / h), cscal(h * W.greg[n][l], cmuli(SRx(n, l))));
                if (l == n) v = cadd(v, cmuli(EPS(n)));
                M[n][l] = v;
                cM[n][l] = cz();
            }
    }
    __syncthreads();
    // ---- lesser columns n = k..0: y_0 = -conj(G^tv(n,0)), M[1:,1:] y = q_A - M[:,0] y_0 ----
    for (int n = k; n >= 0; --n) {
        // forward sources q_m = -i h c2 + xi htau c3, c2 = sum_{j<=k} s_{n,j} Sigma^<(m,j) conj(G~^R(n,j)),
        // c3 = sum_j w_{T,j} Sigma^tv(m,j) conj(G^tv(n,T-j))
        for (int m = 1; m <= k; ++m) {
            cplx p3 = cz();
            for (int j = t; j <= T; j += blockDim.x) p3 = cfma(cscal(gw(W, T, j), ST(m, j)), cconj(GT(n, T - j)), p3);
            p3 = block_csum(p3, red);
            if (t == 0) {
                cplx c2 = cz();
                for (int j = 0; j <= k; ++j) c2 = cfma(cscal(W.greg[n][j], SL(m, j)), cconj(GRx(n, j)), c2);
                qsh[m] = cadd(cmulmi(cscal(h, c2)), cscal(xi * ht, p3));
            }
        }
        __syncthreads();
        if (t == 0) {
            const cplx y0 = GL(0, n);
            cplx A[NG_KMAX * NG_KMAX], AH[NG_KMAX * NG_KMAX], sol[NG_KMAX], cs[NG_KMAX];
            for (int m = 1; m <= k; ++m) {
                sol[m - 1] = csub(qsh[m], cmul(M[m][0], y0));
                cs[m - 1] = (m <= n) ? cles(m, n) : cz();
                for (int l = 1; l <= k; ++l) {
                    A[(m - 1) * k + (l - 1)] = M[m][l];
                    AH[(l - 1) * k + (m - 1)] = cconj(M[m][l]);
                }
            }
            dense_solve(A, k, sol, 1);      // full forward solution (components m > n are not stored)
            dense_solve(AH, k, cs, 1);      // cotangent of the right-hand side
            cplx cy0 = cles(0, n);
            for (int m = 1; m <= k; ++m) {
                for (int l = 1; l <= k; ++l) cM[m][l] = csub(cM[m][l], cmul(cs[m - 1], cconj(sol[l - 1])));
                cM[m][0] = csub(cM[m][0], cmul(cconj(y0), cs[m - 1]));
                cy0 = csub(cy0, cmul(cconj(M[m][0]), cs[m - 1]));
                crh[m] = cs[m - 1];
            }
            ctv(n, 0) = csub(ctv(n, 0), cconj(cy0));
            // ret / les parts of the sources' transpose (j <= k)
            for (int m = 1; m <= k; ++m) {
                const cplx cc2 = cmuli(cscal(h, crh[m]));
                for (int j = 0; j <= k; ++j) {
                    Ples(m, j, cmul(cscal(W.greg[n][j], GRx(n, j)), cc2));
                    const cplx v = cmul(cscal(W.greg[n][j], SL(m, j)), cconj(cc2));
                    if (j <= n) cret(n, j) = cadd(cret(n, j), v);
                    else cret(j, n) = csub(cret(j, n), cconj(v));
                }
            }
        }
        __syncthreads();
        for (int j = t; j <= T; j += blockDim.x) {
            cplx acc = cz();
            for (int m = 1; m <= k; ++m) {
                const cplx cc3 = cscal(xi * ht, crh[m]);
                Ptv(m, j) = cfma(cscal(gw(W, T, j), GT(n, T - j)), cc3, Ptv(m, j));
                acc = cfma(cscal(gw(W, T, j), ST(m, j)), cconj(cc3), acc);
            }
            ctv(n, T - j) = cadd(ctv(n, T - j), acc);
        }
        __syncthreads();
    }
    // ---- left-mixing rows 1..k: M[1:,1:] y(m) = q_tv(m) - M[:,0] y_0(m), y_0 = i xi G^M(T-m) ----
    if (t == 0) {
        cplx AH[NG_KMAX * NG_KMAX];
        for (int r = 1; r <= k; ++r)
            for (int l = 1; l <= k; ++l) AH[(l - 1) * k + (r - 1)] = cconj(M[r][l]);
        for (int r = 0; r < k; ++r)
            for (int m = 0; m <= T; ++m) rt[(int64_t)r * (T + 1) + m] = ctv(r + 1, m);
        dense_solve(AH, k, rt, T + 1);
    }
    __syncthreads();
    for (int r = 1; r <= k; ++r)
        for (int l = 0; l <= k; ++l) {
            cplx p = cz();
            for (int m = t; m <= T; m += blockDim.x) {
                const cplx y = (l == 0) ? cmuli(cscal(xi, GM(T - m))) : GT(l, m);
                p = csub(p, cmul(cconj(y), rt[(int64_t)(r - 1) * (T + 1) + m]));
            }
            p = block_csum(p, red);
            if (t == 0) cM[r][l] = cadd(cM[r][l], p);
        }
    // Matsubara source q_tv = -i htau (C2 + C3) transposed, rows 1..k
    for (int64_t e = t; e < (int64_t)k * (T + 1); e += blockDim.x) {
        const int n = 1 + (int)(e / (T + 1)), p = (int)(e % (T + 1));
        const cplx* rr = rt + (int64_t)(n - 1) * (T + 1);
        cplx acc = cz();
        for (int m = 0; m <= T; ++m) {
            cplx w = cz();
            if (m <= k) {
                if (p <= k)
                    for (int j = 0; j <= k; ++j) w = cadd(w, cscal(W.R[m][j][p] * xi, cconj(GM(T - j))));
            } else if (p <= m) {
                w = cadd(w, cscal(gw(W, m, m - p) * xi, cconj(GM(T - m + p))));
            }
            if (m >= T - k) {
                if (p >= T - k)
                    for (int j = 0; j <= k; ++j) w = cadd(w, cscal(W.R[T - m][j][T - p], cconj(GM(j))));
            } else if (p >= m) {
                w = cadd(w, cscal(gw(W, T - m, p - m), cconj(GM(p - m))));
            }
            acc = cfma(w, cmuli(cscal(ht, rr[m])), acc);
        }
        Ptv(n, p) = cadd(Ptv(n, p), acc);
    }
    __syncthreads();
    if (t != 0) return;
    // start matrix cotangent -> Sigma~^R(n,l) and eps_n
    for (int n = 1; n <= k; ++n) {
        for (int l = 0; l <= k; ++l) Pret(n, l, cmulmi(cscal(h * W.greg[n][l], cM[n][l])));
        cmf(n) = cadd(cmf(n), cmulmi(cM[n][n]));
    }
    // ---- retarded columns m = k-1..0: Mf[n][l] y_l = 0 (n = m+1..k), y_m = -i,
    //      y_l = -conj(G^R(m,l)) for l < m; Mf = i D/h - h I_{m,n;l} Sigma~^R(n,l) - delta (eps_n - mu)
    for (int m = k - 1; m >= 0; --m) {
        const int N = k - m;
        cplx y[NG_KMAX + 1], Mf[NG_KMAX + 1][NG_KMAX + 1], AH[NG_KMAX * NG_KMAX], cb[NG_KMAX], cyl[NG_KMAX + 1];
        for (int l = 0; l < m; ++l) y[l] = cneg(cconj(GR(m, l)));
        y[m] = make_double2(0.0, -1.0);
        for (int l = m + 1; l <= k; ++l) y[l] = GR(l, m);
        for (int n = m + 1; n <= k; ++n)
            for (int l = 0; l <= k; ++l) {
                cplx v = csub(cmuli(cr(W.D[n][l] / h)), cscal(h * W.I[m][n][l], SRx(n, l)));
                if (l == n) v = csub(v, EPS(n));
                Mf[n][l] = v;
            }
        for (int n = m + 1; n <= k; ++n) {
            for (int l = m + 1; l <= k; ++l) AH[(l - m - 1) * N + (n - m - 1)] = cconj(Mf[n][l]);
            cb[n - m - 1] = cret(n, m);
        }
        dense_solve(AH, N, cb, 1);
        for (int l = 0; l <= k; ++l) cyl[l] = cz();
        for (int n = m + 1; n <= k; ++n) {
            const cplx crn = cb[n - m - 1];
            for (int l = 0; l <= k; ++l) {
                cplx cMf;
                if (l > m) cMf = cneg(cmul(crn, cconj(y[l])));
                else {
                    cMf = cneg(cmul(cconj(y[l]), crn));
                    cyl[l] = csub(cyl[l], cmul(cconj(Mf[n][l]), crn));
                }
                Pret(n, l, cscal(-h * W.I[m][n][l], cMf));
                if (l == n) cmf(n) = csub(cmf(n), cMf);
            }
        }
        for (int l = 0; l < m; ++l) cret(m, l) = csub(cret(m, l), cconj(cyl[l]));
    }
}

// shared Sigma cotangent of slices 0..k = sum over problems (fixed order); warp per entry
__global__ void k_adj_boot_reduce(int64_t E, int nb, const cplx* Pk, cplx* out) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= E) return;
    cplx s = cz();
    for (int kb = lane; kb < nb; kb += 32) s = cadd(s, Pk[w * nb + kb]);
    s = warp_sum(s);
    if (lane == 0) out[w] = s;
}

// mu_new = ctot + bcast(cL)/nb over slices 0..k; dist[0] += |mu_new - mu|, dist[1] += |mu_new|
__global__ void k_adj_boot_update(int64_t E, int nb, const cplx* ctot, const cplx* cL, cplx* mu, double* dist) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double d = 0.0, a = 0.0;
    if (i < E * nb) {
        const int64_t e = i / nb;
        const cplx v = cadd(ctot[i], cscal(1.0 / nb, cL[e]));
        d = fabs(v.x - mu[i].x) + fabs(v.y - mu[i].y);
        a = fabs(v.x) + fabs(v.y);
        mu[i] = v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        d += __shfl_xor_sync(0xffffffffu, d, o);
        a += __shfl_xor_sync(0xffffffffu, a, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (d != 0.0) atomicAdd(&dist[0], d);
        if (a != 0.0) atomicAdd(&dist[1], a);
    }
}

// gather the cotangent of slices 0..k of a herm (ld = nb or 1) into the compact layout
__global__ void k_boot_gather(Grid g, const cplx* r, const cplx* l, const cplx* tv, int ld, cplx* out) {
    const int k = g.k, T = g.ntau;
    const int64_t T3 = tri(k + 1), E = boot_E(k, T);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= E * ld) return;
    const int64_t e = i / ld;
    const int kb = (int)(i % ld);
    if (e < T3) out[i] = r[e * ld + kb];
    else if (e < 2 * T3) out[i] = l[(e - T3) * ld + kb];
    else out[i] = tv[(e - 2 * T3) * ld + kb];
}

// eps0 cotangent rows 0..k: ce0 += Re(cmf), thread per (row, problem)
__global__ void k_adj_ce0_rows(int rows, int nb, const cplx* cmf, double* ce0) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)rows * nb) return;
    ce0[nb + i] += cmf[nb + i].x;   // rows t = 0..rows-1 at index (t+1)
}
