// Launch interface of the contour convolution (ng_conv.cu, a translation unit of its own with
// its own copy of the integration weights in constant memory).
#pragma once

#include "ng_common.cuh"

// integration weights of the convolution kernels, k = 1..NG_KMAX, for the current device
cudaError_t conv_load_weights(const NgWeights* all);
// slice n (-1: Matsubara) of C = A * f * B for nbe problems; f.p == nullptr is the identity
cudaError_t conv_launch(const Grid& g, int n, const HermV& C, const HermV& A, const HermV& Acc, const FuncV& f,
                        const HermV& B, const HermV& Bcc, int nbe, int* status, cudaStream_t s);
