// Observables of one time slice (ng_observables): particle number, kinetic energy, Hartree
// energy and the Galitskii-Migdal correlation energy, averaged over the batch.
//   rho_k(t)   = -i G_k^<(t,t)                                   (density matrix)
//   N          = (1/nb) sum_k Tr rho_k
//   E_kin      = (1/nb) sum_k Tr[rho_k eps0_k(t)]                  (k-space kinetic energy)
//   E_mf       = (1/nb) sum_k 1/2 Tr[rho_k (eps_mf_k(t) - eps0_k(t))]
//   E_corr     = (1/nb) sum_k 1/2 Im Tr[Sigma * G_k]^<(t,t)       (Eq. Total_ener, correlation part)
//   E_tot      = E_kin + E_mf + E_corr                            (Galitskii-Migdal total energy)
// [Sigma * G]^<(n,n) = C^<_1 + C^<_2 + C^<_3 [Sigma, 1, G](n,n) (Eqs. cles1-cles3).
#pragma once

#include "ng_step.cuh"

#define NG_OBS_THREADS 128
#define NG_NOBS 5

template <int D>
__global__ void __launch_bounds__(NG_OBS_THREADS) k_observables(Grid g, int n, HermV G, HermV S, FuncV eps0,
                                                                FuncV epsmf, double* ws) {
    const NgWeights& W = c_W[g.k - 1];
    const int k = W.k;
    const int kb = blockIdx.x, t = threadIdx.x;
    __shared__ cplx red[NG_OBS_THREADS * D * D];
    // C^<_1[Sigma,1,G](n,n) = h sum_j w_{n,j} Sigma~^R(n,j) G^<(j,n)
    Mat<D> c1 = mzero<D>();
    if (n <= k) {
        for (int j = t; j <= k; j += blockDim.x)
            mfma<D>(c1, mscal<D>(W.greg[n][j], gretx<D>(S, n, j, kb)), gles<D>(G, j, n, kb));
    } else {
        for (int j = t; j <= n; j += blockDim.x)
            mfma<D>(c1, mscal<D>(gw(W, n, j), gret<D>(S, n, j, kb)), ld<D>(G.les, tri(n) + j, kb));
    }
    Mat<D> s1 = block_sum<D>(c1, red);
    // -i (C^<_2 + C^<_3)[Sigma,1,G](n,n)
    Mat<D> q = block_sum<D>(q_lesA_part<D>(W, g, G, S, n, n, kb, t, blockDim.x), red);
    if (t != 0) return;
    Mat<D> C = madd<D>(mscal<D>(g.h, s1), mmuli<D>(q));  // C1 + (C2 + C3), with C2 + C3 = i q
    Mat<D> rho = mmul<D>(meye<D>(make_double2(0.0, -1.0)), ld<D>(G.les, tri(n) + n, kb));
    Mat<D> e0 = ldf<D>(eps0, n, kb), emf = ldf<D>(epsmf, n, kb);
    Mat<D> rk = mmul<D>(rho, e0), rm = mmul<D>(rho, msub<D>(emf, e0));
    double N = 0.0, ek = 0.0, em = 0.0, ec = 0.0;
    for (int a = 0; a < D; ++a) {
        N += rho.v[a][a].x;
        ek += rk.v[a][a].x;
        em += 0.5 * rm.v[a][a].x;
        ec += 0.5 * C.v[a][a].y;
    }
    double* o = ws + (size_t)kb * NG_NOBS;
    o[0] = N;
    o[1] = ek;
    o[2] = em;
    o[3] = ec;
    o[4] = ek + em + ec;
}

// batch average in a fixed order; one block
__global__ void k_observables_reduce(int nb, const double* ws, double* out) {
    __shared__ double red[NG_OBS_THREADS];
    for (int q = 0; q < NG_NOBS; ++q) {
        double s = 0.0;
        for (int kb = threadIdx.x; kb < nb; kb += blockDim.x) s += ws[(size_t)kb * NG_NOBS + q];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[q] = red[0] / nb;
        __syncthreads();
    }
}
