// Launch interface of the FFT evaluation of the left-mixing Matsubara source (ng_tvfft.cu).
#pragma once

#include "ng_common.cuh"

// shared memory a block may take for its transforms (the 227 KB per-block limit, with room)
#define NG_TVFFT_MAX_SMEM (200u * 1024u)

// transform length: the power of two >= 2 ntau + 1
int tvfft_length(int ntau);
size_t tvfft_smem_bytes(int nf, int ntau);
// nf = 1, 2 and transforms that fit the shared-memory budget
bool tvfft_supported(int nf, int ntau);
// tw[p] = exp(-2 pi i p / L), p = 0..L/2-1
cudaError_t tvfft_twiddles(cplx* tw, int L, cudaStream_t s);
// Q[(m nf^2 + a nf + b) nb + kb] = the unit-weight correlation F_ab(m) of step n, every problem
cudaError_t tvfft_launch(const Grid& g, int n, const Comp& Stv, const Comp& Gmat, const cplx* tw, cplx* Q,
                         cudaStream_t s);
