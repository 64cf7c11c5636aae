// Launch wrapper of the contour convolution kernel (ng_conv.cuh).
#include "ng_conv.cuh"
#include "ng_conv_launch.h"

cudaError_t conv_load_weights(const NgWeights* all) {
    return cudaMemcpyToSymbol(c_W, all, sizeof(NgWeights) * NG_KMAX);
}

cudaError_t conv_launch(const Grid& g, int n, const HermV& C, const HermV& A, const HermV& Acc, const FuncV& f,
                        const HermV& B, const HermV& Bcc, int nbe, int* status, cudaStream_t s) {
    const int cnt = n < 0 ? g.ntau + 1 : 2 * (n + 1) + g.ntau + 1;
    const int64_t items = (int64_t)cnt * g.nf * (g.nf > 4 ? 2 : 1) * nbe;
    const unsigned nblk = (unsigned)((items + 127) / 128);
    const FRef fr{f.p, f.ldk};
    switch (g.nf) {
        case 1: k_conv_slice<1><<<nblk, 128, 0, s>>>(g, n, C, A, Acc, fr, B, Bcc, nbe, status); break;
        case 2: k_conv_slice<2><<<nblk, 128, 0, s>>>(g, n, C, A, Acc, fr, B, Bcc, nbe, status); break;
        case 4: k_conv_slice<4><<<nblk, 128, 0, s>>>(g, n, C, A, Acc, fr, B, Bcc, nbe, status); break;
        default: k_conv_slice<8><<<nblk, 128, 0, s>>>(g, n, C, A, Acc, fr, B, Bcc, nbe, status); break;
    }
    return cudaGetLastError();
}
