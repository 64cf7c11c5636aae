// Launch wrappers of the integral-form Dyson solver (ng_vie2.cuh).
#include "ng_vie2.cuh"
#include "ng_vie2_launch.h"

namespace {
inline unsigned nblk(int64_t items, int threads) { return (unsigned)((items + threads - 1) / threads); }

template <int D>
cudaError_t start_d(const Grid& g, const HermV& G, const HermV& F, const HermV& Fcc, const HermV& Q, cplx* ws,
                    int* status, cudaStream_t s) {
    k_v2_start_ret<D><<<nblk(g.nb, 64), 64, 0, s>>>(g, G, F, Fcc, Q, ws, status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_v2_start_tv<D><<<nblk((int64_t)(g.ntau + 1) * g.nb, 128), 128, 0, s>>>(g, G, F, Q, ws, status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_v2_start_les<D><<<nblk((int64_t)(g.k + 1) * g.nb, 64), 64, 0, s>>>(g, G, F, Fcc, Q, ws, status);
    return cudaGetLastError();
}

template <int D>
cudaError_t step_d(const Grid& g, int n, const HermV& G, const HermV& F, const HermV& Fcc, const HermV& Q,
                   const cplx* tvq, bool warp, int* status, cudaStream_t s) {
    const int thr = 128;
    if (warp) {
        const int64_t w_les = (int64_t)g.nb * (n - 1), w_tv = (int64_t)g.nb * (g.ntau + 1), w_ret = (int64_t)g.nb * n;
        k_v2_bulk_w<D><<<nblk((w_les + w_tv + w_ret) * 32, thr), thr, 0, s>>>(g, n, G, F, Fcc, Q, w_les, w_tv, w_ret,
                                                                               status);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_v2_diag<D><<<g.nb, NG_BND_THREADS, 0, s>>>(g, n, G, F, Fcc, Q, status);
        return cudaGetLastError();
    }
    const int b_les = (int)nblk((int64_t)g.nb * (n - 1), thr), b_tv = (int)nblk((int64_t)g.nb * (g.ntau + 1), thr);
    const int b_ret = (int)nblk((int64_t)g.nb * n, thr);
    k_v2_bulk<D><<<b_les + b_tv + b_ret, thr, 0, s>>>(g, n, G, F, Fcc, Q, b_ret, b_tv, b_les, tvq, status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_v2_diag<D><<<g.nb, NG_BND_THREADS, 0, s>>>(g, n, G, F, Fcc, Q, status);
    return cudaGetLastError();
}
}  // namespace

cudaError_t vie2_load_weights(const NgWeights* all) {
    return cudaMemcpyToSymbol(c_W, all, sizeof(NgWeights) * NG_KMAX);
}

cudaError_t vie2_start_launch(const Grid& g, const HermV& G, const HermV& F, const HermV& Fcc, const HermV& Q,
                              cplx* ws, int* status, cudaStream_t s) {
    switch (g.nf) {
    case 1: return start_d<1>(g, G, F, Fcc, Q, ws, status, s);
    case 2: return start_d<2>(g, G, F, Fcc, Q, ws, status, s);
    case 4: return start_d<4>(g, G, F, Fcc, Q, ws, status, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t vie2_step_launch(const Grid& g, int n, const HermV& G, const HermV& F, const HermV& Fcc, const HermV& Q,
                             const cplx* tvq, bool warp, int* status, cudaStream_t s) {
    switch (g.nf) {
    case 1: return step_d<1>(g, n, G, F, Fcc, Q, tvq, warp, status, s);
    case 2: return step_d<2>(g, n, G, F, Fcc, Q, tvq, warp, status, s);
    case 4: return step_d<4>(g, n, G, F, Fcc, Q, tvq, warp, status, s);
    default: return cudaErrorInvalidValue;
    }
}
