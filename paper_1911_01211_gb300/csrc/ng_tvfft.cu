// The Toeplitz part of the left-mixing Matsubara source of a time step by FFT.
//
// The source of the left-mixing row at step n is q(m) = -i (C^tv_2 + C^tv_3)[Sigma, 1, G^M](n, m)
// (Eqs. ctv2, ctv3).  With unit quadrature weights both pieces together are one correlation
//   F(m) = sum_{j=0..ntau} S(j) K(j - m),   S(j) = Sigma^tv(t_n, tau_j),
//   K(d) = xi G^M(tau_{ntau+d}) (d < 0),  K(0) = xi G^M(beta) + G^M(0),  K(d) = G^M(tau_d) (d > 0),
// which this kernel evaluates for all m at once as a cyclic convolution of length L >= 2 ntau + 1
// (a power of two): forward transforms of S and of the reversed K, their (matrix) product per
// frequency, one inverse transform.  The Gregory end weights and the boundary (R) formulas near
// m = 0 and m = ntau differ from unit weights in O(k) terms; the time-step kernels add those
// corrections per element (q_tv_fft in ng_step.cuh).
//
// One block per problem; the transforms are radix-2 in shared memory: decimation in frequency
// forward (natural order in, bit-reversed out), decimation in time inverse (bit-reversed in,
// natural out), so the spectra are multiplied in bit-reversed order without a permutation.
// Twiddles exp(-2 pi i p / L) come from a table built once per length.
#include "ng_tvfft.h"

namespace {

constexpr int kThreads = 256;

__global__ void k_twiddle(cplx* tw, int L) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= L / 2) return;
    double s, c;
    sincospi(-2.0 * (double)p / (double)L, &s, &c);
    tw[p] = make_double2(c, s);
}

// forward DIF: natural order in, bit-reversed out, kernel exp(-2 pi i jk / L)
__device__ void fft_forward(cplx* x, const cplx* __restrict__ tw, int L) {
    for (int span = L >> 1; span >= 1; span >>= 1) {
        const int str = (L >> 1) / span;
        for (int t = threadIdx.x; t < (L >> 1); t += blockDim.x) {
            const int pos = t & (span - 1), i = ((t - pos) << 1) + pos, j = i + span;
            const cplx a = x[i], b = x[j];
            x[i] = cadd(a, b);
            x[j] = cmul(csub(a, b), tw[pos * str]);
        }
        __syncthreads();
    }
}

// inverse DIT: bit-reversed order in, natural out, kernel exp(+2 pi i jk / L), unscaled
__device__ void fft_inverse(cplx* x, const cplx* __restrict__ tw, int L) {
    for (int span = 1; span < L; span <<= 1) {
        const int str = (L >> 1) / span;
        for (int t = threadIdx.x; t < (L >> 1); t += blockDim.x) {
            const int pos = t & (span - 1), i = ((t - pos) << 1) + pos, j = i + span;
            const cplx a = x[i], b = cmul(x[j], cconj(tw[pos * str]));
            x[i] = cadd(a, b);
            x[j] = csub(a, b);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ cplx el(const Comp& c, int64_t e, int ab, int kb) {
    return c.p[(e * c.dd + ab) * c.ldk + (c.ldk == 1 ? 0 : kb)];
}

// Q[(m nf^2 + a nf + b) nb + kb] = F_ab(m), m = 0..ntau, for problem kb = blockIdx.x
template <int D>
__global__ void __launch_bounds__(kThreads) k_tvsrc_fft(Grid g, int n, Comp Stv, Comp Gmat, const cplx* tw, int L,
                                                        cplx* Q) {
    extern __shared__ cplx sm[];
    constexpr int DD = D * D;
    cplx* FS = sm;            // [a c][L]: S_ac, then the product P_ab in place
    cplx* FK = sm + DD * L;   // [c b][L]: reversed K_cb
    const int kb = blockIdx.x, T = g.ntau;
    const double xi = (double)g.sig;
    const int64_t rowS = (int64_t)n * (T + 1);
    for (int e = 0; e < DD; ++e)
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
            FS[e * L + i] = i <= T ? el(Stv, rowS + i, e, kb) : cz();
            cplx v = cz();
            if (i == 0) v = cadd(cscal(xi, el(Gmat, T, e, kb)), el(Gmat, 0, e, kb));
            else if (i <= T) v = cscal(xi, el(Gmat, T - i, e, kb));          // K(-i)
            else if (i >= L - T) v = el(Gmat, L - i, e, kb);                 // K(L - i)
            FK[e * L + i] = v;
        }
    __syncthreads();
    for (int e = 0; e < DD; ++e) fft_forward(FS + e * L, tw, L);
    for (int e = 0; e < DD; ++e) fft_forward(FK + e * L, tw, L);
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        cplx s[D][D], k[D][D];
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = 0; b < D; ++b) s[a][b] = FS[(a * D + b) * L + i], k[a][b] = FK[(a * D + b) * L + i];
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = 0; b < D; ++b) {
                cplx p = cz();
#pragma unroll
                for (int c = 0; c < D; ++c) p = cfma(s[a][c], k[c][b], p);
                FS[(a * D + b) * L + i] = p;
            }
    }
    __syncthreads();
    for (int e = 0; e < DD; ++e) fft_inverse(FS + e * L, tw, L);
    const double inv = 1.0 / (double)L;
    for (int e = 0; e < DD; ++e)
        for (int m = threadIdx.x; m <= T; m += blockDim.x)
            Q[((int64_t)m * DD + e) * g.nb + kb] = cscal(inv, FS[e * L + m]);
}

}  // namespace

int tvfft_length(int ntau) {
    int L = 1;
    while (L < 2 * ntau + 1) L <<= 1;
    return L;
}

size_t tvfft_smem_bytes(int nf, int ntau) { return (size_t)2 * nf * nf * tvfft_length(ntau) * sizeof(cplx); }

bool tvfft_supported(int nf, int ntau) {
    return (nf == 1 || nf == 2) && tvfft_smem_bytes(nf, ntau) <= NG_TVFFT_MAX_SMEM;
}

cudaError_t tvfft_twiddles(cplx* tw, int L, cudaStream_t s) {
    k_twiddle<<<(L / 2 + 255) / 256, 256, 0, s>>>(tw, L);
    return cudaGetLastError();
}

cudaError_t tvfft_launch(const Grid& g, int n, const Comp& Stv, const Comp& Gmat, const cplx* tw, cplx* Q,
                         cudaStream_t s) {
    const int L = tvfft_length(g.ntau);
    const size_t smem = tvfft_smem_bytes(g.nf, g.ntau);
    cudaError_t e;
    if (g.nf == 1) {
        if ((e = cudaFuncSetAttribute(k_tvsrc_fft<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
            return e;
        k_tvsrc_fft<1><<<g.nb, kThreads, smem, s>>>(g, n, Stv, Gmat, tw, L, Q);
    } else {
        if ((e = cudaFuncSetAttribute(k_tvsrc_fft<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
            return e;
        k_tvsrc_fft<2><<<g.nb, kThreads, smem, s>>>(g, n, Stv, Gmat, tw, L, Q);
    }
    return cudaGetLastError();
}
