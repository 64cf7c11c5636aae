// Setup kernels of libng: free Green's functions, the Matsubara solve and the start-up.
#pragma once

#include "ng_step.cuh"

// ----------------------------------------------------------------------------------------
// Hermitian eigen-decomposition of a small D x D matrix by cyclic Jacobi rotations
// (Jacobi 1846; complex form as in Golub & Van Loan, Sec. 8.5).  eps = R diag(e) R^dagger.
// ----------------------------------------------------------------------------------------
template <int D>
__device__ void herm_eig(Mat<D> A, double e[D], Mat<D>& R) {
    R = meye<D>(cr(1.0));
    for (int sweep = 0; sweep < 30; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < D; ++p)
            for (int q = p + 1; q < D; ++q) off += cabs2(A.v[p][q]);
        if (off < 1e-300) break;
        for (int p = 0; p < D; ++p)
            for (int q = p + 1; q < D; ++q) {
                double apq = sqrt(cabs2(A.v[p][q]));
                if (apq < 1e-300) continue;
                // phase so that the rotated element is real: A_pq = |A_pq| e^{i phi}
                cplx ph = make_double2(A.v[p][q].x / apq, A.v[p][q].y / apq);
                double app = A.v[p][p].x, aqq = A.v[q][q].x;
                double theta = 0.5 * atan2(2.0 * apq, aqq - app);
                double c = cos(theta), s = sin(theta);
                // unitary J acting on columns p, q: col_p' = c col_p - s conj(ph) col_q ... built as
                // J = [[c, s ph], [-s conj(ph), c]] in the (p, q) plane
                cplx jpp = cr(c), jpq = cscal(s, ph), jqp = cscal(-s, cconj(ph)), jqq = cr(c);
                // A <- J^dagger A J
                for (int r = 0; r < D; ++r) {  // A J (columns)
                    cplx arp = A.v[r][p], arq = A.v[r][q];
                    A.v[r][p] = cadd(cmul(arp, jpp), cmul(arq, jqp));
                    A.v[r][q] = cadd(cmul(arp, jpq), cmul(arq, jqq));
                    cplx rrp = R.v[r][p], rrq = R.v[r][q];
                    R.v[r][p] = cadd(cmul(rrp, jpp), cmul(rrq, jqp));
                    R.v[r][q] = cadd(cmul(rrp, jpq), cmul(rrq, jqq));
                }
                for (int r = 0; r < D; ++r) {  // J^dagger (rows)
                    cplx apr = A.v[p][r], aqr = A.v[q][r];
                    A.v[p][r] = cadd(cmul(cconj(jpp), apr), cmul(cconj(jqp), aqr));
                    A.v[q][r] = cadd(cmul(cconj(jpq), apr), cmul(cconj(jqq), aqr));
                }
            }
    }
    for (int a = 0; a < D; ++a) e[a] = A.v[a][a].x;
}

// (1 + xi f(e)) e^{-e tau} and f(e) e^{e tau} for fermions (xi = -1), overflow-safe
__device__ __forceinline__ void fermi_terms(double e, double beta, double tau, double* gm, double* gtv) {
    if (e >= 0.0) {
        double x = exp(-beta * e);
        *gm = exp(-e * tau) / (1.0 + x);
        *gtv = x / (1.0 + x) * exp(e * tau);
    } else {
        double x = exp(beta * e);
        *gm = exp(e * (beta - tau)) / (1.0 + x);
        *gtv = exp(e * tau) / (1.0 + x);
    }
}

// ----------------------------------------------------------------------------------------
// free Green's function of constant eps (Eq. G0_free), times `scale`; one thread per
// (element, problem).  eps_dev: [nb][D][D].
// ----------------------------------------------------------------------------------------
template <int D>
__global__ void k_free_gf(Grid g, HermV G, const cplx* eps_dev, double scale) {
    const int64_t nel_tri = tri(g.nt + 1);
    const int64_t nel_tv = (int64_t)(g.nt + 1) * (g.ntau + 1);
    const int64_t nel = (g.ntau + 1) + 2 * nel_tri + nel_tv;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= nel * g.nb) return;
    const int kb = (int)(item % g.nb);
    int64_t e = item / g.nb;
    Mat<D> E;
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) E.v[a][b] = eps_dev[(kb * D + a) * D + b];
    double ev[D];
    Mat<D> R;
    herm_eig<D>(E, ev, R);
    for (int a = 0; a < D; ++a) ev[a] -= g.mu;
    Mat<D> Rd = mdag<D>(R);
    auto sandwich = [&](const cplx* dg) {  // R diag(dg) R^dagger
        Mat<D> x;
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b) {
                cplx s = cz();
                for (int c = 0; c < D; ++c) s = cadd(s, cmul(cmul(R.v[a][c], dg[c]), Rd.v[c][b]));
                x.v[a][b] = s;
            }
        return x;
    };
    cplx dg[D];
    const double xi = (double)g.sig;
    if (e < g.ntau + 1) {  // mat: -R diag{(1 + xi f) e^{-e tau}} R^dagger
        const int m = (int)e;
        for (int c = 0; c < D; ++c) {
            double gm, gt;
            fermi_terms(ev[c], g.beta, m * g.htau, &gm, &gt);
            dg[c] = cr(-gm * scale);
        }
        st<D>(G.mat, m, kb, sandwich(dg));
        return;
    }
    e -= g.ntau + 1;
    if (e < 2 * nel_tri) {
        const bool isret = e < nel_tri;
        if (!isret) e -= nel_tri;
        // decode row n and column j of the packed triangle
        int n = (int)((sqrt(8.0 * (double)e + 1.0) - 1.0) * 0.5);
        while (tri(n + 1) <= e) ++n;
        while (tri(n) > e) --n;
        const int j = (int)(e - tri(n));
        const double dt = (n - j) * g.h;
        for (int c = 0; c < D; ++c) {
            double s, co;
            sincos(ev[c] * dt, &s, &co);
            if (isret) {
                dg[c] = cscal(scale, make_double2(-s, -co));    // -i e^{-i e dt}
            } else {
                double f = 0.5 * (1.0 - tanh(0.5 * g.beta * ev[c]));
                // G^<(j,n) = -xi i f e^{-i e (t_j - t_n)} = -xi i f e^{+i e dt}
                dg[c] = cscal(-xi * f * scale, make_double2(-s, co));
            }
        }
        st<D>(isret ? G.ret : G.les, e, kb, sandwich(dg));
        return;
    }
    e -= 2 * nel_tri;
    const int n = (int)(e / (g.ntau + 1)), m = (int)(e % (g.ntau + 1));
    for (int c = 0; c < D; ++c) {  // -i xi f e^{-i e t} e^{e tau}
        double gm, gt, s, co;
        fermi_terms(ev[c], g.beta, m * g.htau, &gm, &gt);
        sincos(ev[c] * n * g.h, &s, &co);
        cplx ph = make_double2(co, -s);
        dg[c] = cscal(xi * gt * scale, cmulmi(ph));  // -i xi f e^{e tau} e^{-i e t}
    }
    st<D>(G.tv, e, kb, sandwich(dg));
}

// ----------------------------------------------------------------------------------------
// Matsubara solve (Sec. "Matsubara"): g^M, K = [g * Sigma]^M, dense operator, LU.
// workspace layout per problem kb: gM[(T+1)][D][D], K[(T+1)][D][D], A[N][N+D] (augmented
// row-major, N = (T+1) D).
// ----------------------------------------------------------------------------------------
template <int D>
__global__ void k_mat_g(Grid g, FuncV eps, cplx* ws_g) {
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= (int64_t)(g.ntau + 1) * g.nb) return;
    const int kb = (int)(item % g.nb), m = (int)(item / g.nb);
    Mat<D> E = ldf<D>(eps, -1, kb);
    double ev[D];
    Mat<D> R;
    herm_eig<D>(E, ev, R);
    Mat<D> x;
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) {
            cplx s = cz();
            for (int c = 0; c < D; ++c) {
                double gm, gt;
                fermi_terms(ev[c] - g.mu, g.beta, m * g.htau, &gm, &gt);
                s = cadd(s, cscal(-gm, cmul(R.v[a][c], cconj(R.v[b][c]))));
            }
            x.v[a][b] = s;
        }
    cplx* dst = ws_g + ((int64_t)kb * (g.ntau + 1) + m) * D * D;
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) dst[a * D + b] = x.v[a][b];
}

// Matsubara convolution C^M_1[A,1,B](m) + C^M_2[A,1,B](m) (Eqs. cm1, cm2) with A taken from a
// per-problem workspace array and B from a herm component.
template <int D>
__device__ Mat<D> cmat_ws_comp(const NgWeights& W, const Grid& g, const cplx* Aws, const Comp& B, int m, int kb) {
    const int k = W.k, T = g.ntau;
    const double xi = (double)g.sig;
    auto A = [&](int i) {
        Mat<D> r;
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b) r.v[a][b] = Aws[i * D * D + a * D + b];
        return r;
    };
    Mat<D> c1 = mzero<D>(), c2 = mzero<D>();
    if (m <= k) {
        for (int j = 0; j <= k; ++j)
            for (int l = 0; l <= k; ++l) mfma<D>(c1, mscal<D>(W.R[m][j][l], A(j)), ld<D>(B, l, kb));
    } else {
        greg_for(W, m, m, [&](int l, double w) { mfma<D>(c1, mscal<D>(w, A(m - l)), ld<D>(B, l, kb)); });
    }
    if (m >= T - k) {
        for (int j = 0; j <= k; ++j)
            for (int l = 0; l <= k; ++l) mfma<D>(c2, mscal<D>(W.R[T - m][j][l], A(T - j)), ld<D>(B, T - l, kb));
    } else {
        greg_for(W, T - m, T - m, [&](int l, double w) { mfma<D>(c2, mscal<D>(w, A(T - l)), ld<D>(B, m + l, kb)); });
    }
    return mscal<D>(g.htau, madd<D>(c1, mscal<D>(xi, c2)));
}

template <int D>
__global__ void k_mat_K(Grid g, HermV S, const cplx* ws_g, cplx* ws_K) {
    const NgWeights& W = c_W[g.k - 1];
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= (int64_t)(g.ntau + 1) * g.nb) return;
    const int kb = (int)(item % g.nb), m = (int)(item / g.nb);
    Mat<D> K = cmat_ws_comp<D>(W, g, ws_g + (int64_t)kb * (g.ntau + 1) * D * D, S.mat, m, kb);
    cplx* dst = ws_K + ((int64_t)kb * (g.ntau + 1) + m) * D * D;
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) dst[a * D + b] = K.v[a][b];
}

// Augmented matrix [I - A | g] of the linear map X -> C^M_1[K,1,X] + C^M_2[K,1,X]; one
// thread per (problem, block row m, block column c).
template <int D>
__global__ void k_mat_assemble(Grid g, const cplx* ws_g, const cplx* ws_K, cplx* ws_A) {
    const NgWeights& W = c_W[g.k - 1];
    const int T = g.ntau, k = W.k;
    const int N = (T + 1) * D, ldA = N + D;
    const int64_t nblk = (int64_t)(T + 1) * (T + 2);
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= nblk * g.nb) return;
    const int kb = (int)(item / nblk);
    const int64_t r = item % nblk;
    const int m = (int)(r / (T + 2)), c = (int)(r % (T + 2));
    const cplx* K = ws_K + (int64_t)kb * (T + 1) * D * D;
    cplx* A = ws_A + (int64_t)kb * N * ldA;
    auto Kb = [&](int i) {
        Mat<D> x;
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b) x.v[a][b] = K[i * D * D + a * D + b];
        return x;
    };
    if (c == T + 1) {  // right-hand side g^M(tau_m)
        const cplx* gg = ws_g + ((int64_t)kb * (T + 1) + m) * D * D;
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b) A[(int64_t)(m * D + a) * ldA + N + b] = gg[a * D + b];
        return;
    }
    const double xi = (double)g.sig;
    Mat<D> blk = mzero<D>();
    if (m <= k) {
        if (c <= k)
            for (int j = 0; j <= k; ++j) blk = madd<D>(blk, mscal<D>(W.R[m][j][c], Kb(j)));
    } else if (c <= m) {
        blk = madd<D>(blk, mscal<D>(gw(W, m, c), Kb(m - c)));
    }
    if (m >= T - k) {
        if (c >= T - k)
            for (int j = 0; j <= k; ++j) blk = madd<D>(blk, mscal<D>(W.R[T - m][j][T - c] * xi, Kb(T - j)));
    } else if (c >= m) {
        blk = madd<D>(blk, mscal<D>(gw(W, T - m, c - m) * xi, Kb(T - (c - m))));
    }
    blk = mscal<D>(-g.htau, blk);
    if (c == m)
        for (int a = 0; a < D; ++a) blk.v[a][a].x += 1.0;
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) A[(int64_t)(m * D + a) * ldA + c * D + b] = blk.v[a][b];
}

// LU with partial pivoting of the augmented matrix [A | B] (N x (N + nrhs)) and back
// substitution; one block per problem; writes the solution into column block N..N+nrhs.
#define NG_LU_THREADS 512
__global__ void __launch_bounds__(NG_LU_THREADS) k_lu_solve(int N, int nrhs, cplx* ws_A, int* piv, int* status) {
    const int ld = N + nrhs;
    cplx* A = ws_A + (int64_t)blockIdx.x * N * ld;
    extern __shared__ unsigned char smem_raw[];
    cplx* prow = reinterpret_cast<cplx*>(smem_raw);                 // pivot row, ld entries
    cplx* mcol = prow + ld;                                          // multipliers, N entries
    double* rv = reinterpret_cast<double*>(mcol + N);                // reduction values
    int* ri = reinterpret_cast<int*>(rv + NG_LU_THREADS);            // reduction indices
    const int t = threadIdx.x, nt = blockDim.x;
    for (int c = 0; c < N; ++c) {
        // pivot search over rows c..N-1
        double best = -1.0;
        int bi = c;
        for (int r = c + t; r < N; r += nt) {
            double v = cabs2(A[(int64_t)r * ld + c]);
            if (v > best) { best = v; bi = r; }
        }
        rv[t] = best;
        ri[t] = bi;
        __syncthreads();
        for (int s = nt / 2; s > 0; s >>= 1) {
            if (t < s && (rv[t + s] > rv[t] || (rv[t + s] == rv[t] && ri[t + s] < ri[t]))) {
                rv[t] = rv[t + s];
                ri[t] = ri[t + s];
            }
            __syncthreads();
        }
        const int p = ri[0];
        if (rv[0] <= 0.0 && t == 0) atomicOr(status, NGF_SINGULAR);
        if (t == 0) piv[(int64_t)blockIdx.x * N + c] = p;   // row interchange of step c
        __syncthreads();
        // swap rows c and p, load the pivot row into shared memory
        for (int j = t; j < ld; j += nt) {
            cplx x = A[(int64_t)p * ld + j];
            if (p != c) {
                A[(int64_t)p * ld + j] = A[(int64_t)c * ld + j];
                A[(int64_t)c * ld + j] = x;
            }
            prow[j] = x;
        }
        __syncthreads();
        const cplx inv = cdiv(cr(1.0), prow[c]);
        for (int r = c + 1 + t; r < N; r += nt) {
            cplx f = cmul(A[(int64_t)r * ld + c], inv);
            mcol[r] = f;
            A[(int64_t)r * ld + c] = f;
        }
        __syncthreads();
        // trailing update of rows c+1.., columns c+1..ld-1: one warp per row, lanes over columns
        {
            const int warp = t >> 5, lane = t & 31, nw = nt >> 5;
            for (int r = c + 1 + warp; r < N; r += nw) {
                const cplx f = mcol[r];
                cplx* row = A + (int64_t)r * ld;
                for (int j = c + 1 + lane; j < ld; j += 32) row[j] = csub(row[j], cmul(f, prow[j]));
            }
        }
        __syncthreads();
    }
    // back substitution, column oriented: x_c = b_c / U_cc, then b_r -= U_rc x_c for r < c
    for (int c = N - 1; c >= 0; --c) {
        const cplx inv = cdiv(cr(1.0), A[(int64_t)c * ld + c]);
        if (t < nrhs) A[(int64_t)c * ld + N + t] = cmul(A[(int64_t)c * ld + N + t], inv);
        __syncthreads();
        for (int64_t q = t; q < (int64_t)c * nrhs; q += nt) {
            const int r = (int)(q / nrhs), j = (int)(q % nrhs);
            A[(int64_t)r * ld + N + j] = csub(A[(int64_t)r * ld + N + j], cmul(A[(int64_t)r * ld + c], A[(int64_t)c * ld + N + j]));
        }
        __syncthreads();
    }
}

// The same factorisation for a few problems, spread over the GPU (blockIdx.y or blockIdx.x =
// problem): per column c, the pivot search, row interchange and multipliers in one block per
// problem (k_lu_col), then the rank-1 update of the trailing rows and columns over many blocks
// (k_lu_rank1), then the back substitution (k_lu_backsub).  Every element receives the same
// operations in the same order as in k_lu_solve, so factors and solution agree bitwise.
__global__ void __launch_bounds__(NG_LU_THREADS) k_lu_col(int N, int nrhs, cplx* ws_A, int* piv, int c, int* status) {
    const int ld = N + nrhs;
    cplx* A = ws_A + (int64_t)blockIdx.x * N * ld;
    __shared__ double rv[NG_LU_THREADS];
    __shared__ int ri[NG_LU_THREADS];
    const int t = threadIdx.x, nt = blockDim.x;
    double best = -1.0;
    int bi = c;
    for (int r = c + t; r < N; r += nt) {
        double v = cabs2(A[(int64_t)r * ld + c]);
        if (v > best) { best = v; bi = r; }
    }
    rv[t] = best;
    ri[t] = bi;
    __syncthreads();
    for (int s = nt / 2; s > 0; s >>= 1) {
        if (t < s && (rv[t + s] > rv[t] || (rv[t + s] == rv[t] && ri[t + s] < ri[t]))) {
            rv[t] = rv[t + s];
            ri[t] = ri[t + s];
        }
        __syncthreads();
    }
    const int p = ri[0];
    if (rv[0] <= 0.0 && t == 0) atomicOr(status, NGF_SINGULAR);
    if (t == 0) piv[(int64_t)blockIdx.x * N + c] = p;
    if (p != c)
        for (int j = t; j < ld; j += nt) {
            const cplx x = A[(int64_t)p * ld + j];
            A[(int64_t)p * ld + j] = A[(int64_t)c * ld + j];
            A[(int64_t)c * ld + j] = x;
        }
    __syncthreads();
    const cplx inv = cdiv(cr(1.0), A[(int64_t)c * ld + c]);
    for (int r = c + 1 + t; r < N; r += nt) A[(int64_t)r * ld + c] = cmul(A[(int64_t)r * ld + c], inv);
}

__global__ void k_lu_rank1(int N, int nrhs, cplx* ws_A, int c) {
    const int ld = N + nrhs, w = ld - c - 1;
    cplx* A = ws_A + (int64_t)blockIdx.y * N * ld;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)(N - c - 1) * w) return;
    const int r = c + 1 + (int)(q / w), j = c + 1 + (int)(q % w);
    A[(int64_t)r * ld + j] = csub(A[(int64_t)r * ld + j], cmul(A[(int64_t)r * ld + c], A[(int64_t)c * ld + j]));
}

__global__ void __launch_bounds__(NG_LU_THREADS) k_lu_backsub(int N, int nrhs, cplx* ws_A) {
    const int ld = N + nrhs;
    cplx* A = ws_A + (int64_t)blockIdx.x * N * ld;
    const int t = threadIdx.x, nt = blockDim.x;
    for (int c = N - 1; c >= 0; --c) {
        const cplx inv = cdiv(cr(1.0), A[(int64_t)c * ld + c]);
        if (t < nrhs) A[(int64_t)c * ld + N + t] = cmul(A[(int64_t)c * ld + N + t], inv);
        __syncthreads();
        for (int64_t q = t; q < (int64_t)c * nrhs; q += nt) {
            const int r = (int)(q / nrhs), j = (int)(q % nrhs);
            A[(int64_t)r * ld + N + j] = csub(A[(int64_t)r * ld + N + j], cmul(A[(int64_t)r * ld + c], A[(int64_t)c * ld + N + j]));
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------------------
// Iterative refinement of the Matsubara solve with stored LU factors (from an earlier
// operator): residual r = g + [K * G]^M - G of the current operator (matrix-free, Eqs. cm1/cm2),
// x = (LU)^-1 r with the stored row interchanges, G += x.  The fixed point is the root of the
// current discretised equation; only the convergence path differs from a fresh LU.
// ----------------------------------------------------------------------------------------
template <int D>
__global__ void k_mat_resid(Grid g, const cplx* ws_g, const cplx* ws_K, HermV G, cplx* ws_r) {
    const NgWeights& W = c_W[g.k - 1];
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= (int64_t)(g.ntau + 1) * g.nb) return;
    const int kb = (int)(item % g.nb), m = (int)(item / g.nb);
    const int T1 = g.ntau + 1;
    Mat<D> kg = cmat_ws_comp<D>(W, g, ws_K + (int64_t)kb * T1 * D * D, G.mat, m, kb);
    const cplx* gg = ws_g + ((int64_t)kb * T1 + m) * D * D;
    Mat<D> Gm = gmat<D>(G, m, kb);
    cplx* r = ws_r + (int64_t)kb * T1 * D * D;   // row-major [(m a)][b] per problem
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) r[(m * D + a) * D + b] = csub(cadd(gg[a * D + b], kg.v[a][b]), Gm.v[a][b]);
}

// one block per problem: x = U^-1 L^-1 P r in place (r has nrhs columns), then G^M += x and
// *dsum += sum |x|
__global__ void __launch_bounds__(NG_LU_THREADS) k_lu_resolve(Grid g, int N, int nrhs, const cplx* ws_A, const int* piv,
                                                              cplx* ws_r, HermV G, double* dsum) {
    const int ld = N + nrhs;
    const cplx* A = ws_A + (int64_t)blockIdx.x * N * ld;
    const int* p = piv + (int64_t)blockIdx.x * N;
    cplx* r = ws_r + (int64_t)blockIdx.x * N * nrhs;
    const int t = threadIdx.x, nt = blockDim.x;
    if (t < nrhs)   // row interchanges in factorisation order
        for (int c = 0; c < N; ++c) {
            const int q = p[c];
            if (q != c) { cplx x = r[c * nrhs + t]; r[c * nrhs + t] = r[q * nrhs + t]; r[q * nrhs + t] = x; }
        }
    __syncthreads();
    for (int c = 0; c < N; ++c) {   // forward: unit lower triangle (multipliers below the diagonal)
        for (int64_t q = t; q < (int64_t)(N - c - 1) * nrhs; q += nt) {
            const int rr = c + 1 + (int)(q / nrhs), j = (int)(q % nrhs);
            r[rr * nrhs + j] = csub(r[rr * nrhs + j], cmul(A[(int64_t)rr * ld + c], r[c * nrhs + j]));
        }
        __syncthreads();
    }
    for (int c = N - 1; c >= 0; --c) {   // backward: upper triangle
        if (t < nrhs) r[c * nrhs + t] = cdiv(r[c * nrhs + t], A[(int64_t)c * ld + c]);
        __syncthreads();
        for (int64_t q = t; q < (int64_t)c * nrhs; q += nt) {
            const int rr = (int)(q / nrhs), j = (int)(q % nrhs);
            r[rr * nrhs + j] = csub(r[rr * nrhs + j], cmul(A[(int64_t)rr * ld + c], r[c * nrhs + j]));
        }
        __syncthreads();
    }
    // G^M += x: element (m, a, b) <-> r[(m nrhs + a) ... ] with N = (ntau+1) nrhs rows
    double s = 0.0;
    const int dd = nrhs * nrhs;
    for (int64_t q = t; q < (int64_t)N * nrhs; q += nt) {
        const int row = (int)(q / nrhs), b = (int)(q % nrhs);
        const int m = row / nrhs, a = row % nrhs;
        const int64_t off = ((int64_t)m * dd + a * nrhs + b) * G.mat.ldk + (G.mat.ldk == 1 ? 0 : blockIdx.x);
        const cplx x = r[q];
        G.mat.p[off] = cadd(G.mat.p[off], x);
        s += sqrt(cabs2(x));
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((t & 31) == 0 && s != 0.0) atomicAdd(dsum, s);
}

template <int D>
__global__ void k_mat_store(Grid g, const cplx* ws_A, HermV G, int* status) {
    const int T = g.ntau, N = (T + 1) * D, ld = N + D;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= (int64_t)(T + 1) * g.nb) return;
    const int kb = (int)(item % g.nb), m = (int)(item / g.nb);
    const cplx* A = ws_A + (int64_t)kb * N * ld;
    Mat<D> x;
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) x.v[a][b] = A[(int64_t)(m * D + a) * ld + N + b];
    if (!mfinite<D>(x)) atomicOr(status, NGF_NONFINITE);
    st<D>(G.mat, m, kb, x);
}

// ----------------------------------------------------------------------------------------
// start-up (Sec. "Start")
// ----------------------------------------------------------------------------------------
// Retarded columns m = 0..k (one thread per problem) and the common VIDE start-up matrix
// M_{n,l} = D_{n,l}/h + delta_{nl} i(eps_n - mu) + h s_{n,l} i Sigma~^R(n,l) (Eq. vdiff_start):
// the workspace receives inv(M[1..k][1..k]) (kD x kD) and the blocks M[n][0].
template <int D>
__global__ void k_start_ret(Grid g, HermV G, HermV S, FuncV eps, cplx* ws_st, int* status) {
    const NgWeights& W = c_W[g.k - 1];
    const int kb = blockIdx.x * blockDim.x + threadIdx.x;
    if (kb >= g.nb) return;
    const int k = W.k, N = k * D;
    cplx A[(NG_KMAX * D) * (NG_KMAX * D)];
    cplx B[(NG_KMAX * D) * (NG_KMAX * D)];
    const Mat<D> mi = meye<D>(make_double2(0.0, -1.0));
    for (int m = 0; m <= k; ++m) {
        Mat<D> y[NG_KMAX + 1];
        for (int l = 0; l < m; ++l) y[l] = mscal<D>(-1.0, mdag<D>(gret<D>(G, m, l, kb)));
        y[m] = mi;
        if (m < k) {
            const int nu = (k - m) * D;
            for (int n = m + 1; n <= k; ++n) {
                Mat<D> e = ldf<D>(eps, n, kb);
                for (int a = 0; a < D; ++a) e.v[a][a].x -= g.mu;
                Mat<D> rhs = mzero<D>();
                for (int l = 0; l <= k; ++l) {
                    // M_{n,l} = i D_{n,l}/h - delta_{nl}(eps_n - mu) - h I_{m,n;l} Sigma~^R(n,l)
                    Mat<D> M = meye<D>(make_double2(0.0, W.D[n][l] / g.h));
                    M = msub<D>(M, mscal<D>(g.h * W.I[m][n][l], gretx<D>(S, n, l, kb)));
                    if (l == n) M = msub<D>(M, e);
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
        for (int n = m; n <= k; ++n) st<D>(G.ret, tri(n) + m, kb, y[n]);
    }
    // VIDE start-up matrix: inverse of M[1..k][1..k] by solving with the identity
    for (int n = 1; n <= k; ++n) {
        Mat<D> e = ldf<D>(eps, n, kb);
        for (int a = 0; a < D; ++a) e.v[a][a].x -= g.mu;
        for (int l = 0; l <= k; ++l) {
            Mat<D> M = meye<D>(cr(W.D[n][l] / g.h));
            M = madd<D>(M, mscal<D>(g.h * W.greg[n][l], mmuli<D>(gretx<D>(S, n, l, kb))));
            if (l == n) M = madd<D>(M, mmuli<D>(e));
            cplx* dst0 = ws_st + (int64_t)kb * (N * N + k * D * D);
            if (l == 0) {
                for (int a = 0; a < D; ++a)
                    for (int b = 0; b < D; ++b) dst0[N * N + (n - 1) * D * D + a * D + b] = M.v[a][b];
            } else {
                for (int a = 0; a < D; ++a)
                    for (int b = 0; b < D; ++b) A[((n - 1) * D + a) * N + (l - 1) * D + b] = M.v[a][b];
            }
        }
    }
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) B[i * N + j] = cr(i == j ? 1.0 : 0.0);
    if (dense_solve(A, N, B, N)) atomicOr(status, NGF_SINGULAR);
    cplx* dst = ws_st + (int64_t)kb * (N * N + k * D * D);
    for (int i = 0; i < N * N; ++i) dst[i] = B[i];
}

// apply the start-up inverse: y_n (n=1..k) = sum_l Minv[n][l] (q_l - M[l][0] y0)
template <int D>
__device__ void start_apply(const cplx* st_ws, int k, const Mat<D>* q, const Mat<D>& y0, Mat<D>* y) {
    const int N = k * D;
    Mat<D> rhs[NG_KMAX];
    for (int l = 0; l < k; ++l) {
        Mat<D> M0;
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b) M0.v[a][b] = st_ws[N * N + l * D * D + a * D + b];
        rhs[l] = msub<D>(q[l], mmul<D>(M0, y0));
    }
    for (int n = 0; n < k; ++n) {
        Mat<D> acc = mzero<D>();
        for (int l = 0; l < k; ++l) {
            Mat<D> Mi;
            for (int a = 0; a < D; ++a)
                for (int b = 0; b < D; ++b) Mi.v[a][b] = st_ws[(n * D + a) * N + l * D + b];
            mfma<D>(acc, Mi, rhs[l]);
        }
        y[n] = acc;
    }
}

template <int D>
__global__ void k_start_tv(Grid g, HermV G, HermV S, const cplx* ws_st, int* status) {
    const NgWeights& W = c_W[g.k - 1];
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= (int64_t)(g.ntau + 1) * g.nb) return;
    const int kb = (int)(item % g.nb), m = (int)(item / g.nb);
    const int k = W.k, N = k * D;
    Mat<D> y0 = mcscal<D>(make_double2(0.0, (double)g.sig), gmat<D>(G, g.ntau - m, kb));  // i xi G^M(beta - tau_m)
    Mat<D> q[NG_KMAX], y[NG_KMAX];
    for (int n = 1; n <= k; ++n) q[n - 1] = q_tv<D>(W, g, G, S, n, m, kb);
    start_apply<D>(ws_st + (int64_t)kb * (N * N + k * D * D), k, q, y0, y);
    st<D>(G.tv, m, kb, y0);
    for (int n = 1; n <= k; ++n) {
        if (!mfinite<D>(y[n - 1])) atomicOr(status, NGF_NONFINITE);
        st<D>(G.tv, (int64_t)n * (g.ntau + 1) + m, kb, y[n - 1]);
    }
}

template <int D>
__global__ void k_start_les(Grid g, HermV G, HermV S, const cplx* ws_st, int* status) {
    const NgWeights& W = c_W[g.k - 1];
    const int k = W.k, N = k * D;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= (int64_t)(k + 1) * g.nb) return;
    const int kb = (int)(item % g.nb), n = (int)(item / g.nb);
    Mat<D> y0 = mscal<D>(-1.0, mdag<D>(gtv<D>(G, g, n, 0, kb)));
    Mat<D> q[NG_KMAX], y[NG_KMAX];
    for (int m = 1; m <= k; ++m) q[m - 1] = q_lesA_part<D>(W, g, G, S, m, n, kb, 0, 1);
    start_apply<D>(ws_st + (int64_t)kb * (N * N + k * D * D), k, q, y0, y);
    st<D>(G.les, tri(n) + 0, kb, y0);
    for (int m = 1; m <= n; ++m) {
        if (!mfinite<D>(y[m - 1])) atomicOr(status, NGF_NONFINITE);
        st<D>(G.les, tri(n) + m, kb, y[m - 1]);
    }
}
