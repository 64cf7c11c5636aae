// Launch interface of the integral-form Dyson solver (ng_vie2.cu, a translation unit of its own
// with its own copy of the integration weights in constant memory).
#pragma once

#include "ng_common.cuh"

// integration weights of the vie2 kernels, k = 1..NG_KMAX, for the current device
cudaError_t vie2_load_weights(const NgWeights* all);
// start-up slices 0..k of G for nb problems (nf = 1, 2); ws: nb (k nf)^2 + nb k nf^2 complex
cudaError_t vie2_start_launch(const Grid& g, const HermV& G, const HermV& F, const HermV& Fcc, const HermV& Q,
                              cplx* ws, int* status, cudaStream_t s);
// time step n > k (conjugate schedule of the lesser column), nf = 1, 2; tvq: the FFT
// correlation of the left-mixing source of F and G^M at step n (the layout of tvfft_launch),
// or NULL for the direct sums; warp: one warp per item (small batches) instead of one thread,
// its source sums split over the lanes (tvq unused)
cudaError_t vie2_step_launch(const Grid& g, int n, const HermV& G, const HermV& F, const HermV& Fcc, const HermV& Q,
                             const cplx* tvq, bool warp, int* status, cudaStream_t s);
