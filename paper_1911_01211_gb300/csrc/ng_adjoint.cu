// Launch wrappers of the discrete adjoint kernels (ng_adjoint.cuh); a translation unit of its
// own, with its own copy of the integration weights in constant memory.
#include <algorithm>

#include "ng_adjoint.cuh"

namespace {
inline unsigned nblk(int64_t items, int threads) { return (unsigned)((items + threads - 1) / threads); }
}

cudaError_t adj_load_weights(const NgWeights* all) {
    return cudaMemcpyToSymbol(c_W, all, sizeof(NgWeights) * NG_KMAX);
}

cudaError_t adj_pass(const AdjStep& a, SliceV Glc, const cplx* U, SliceV cLoc, double* ce0_row, cudaStream_t s) {
    const int n = a.n, nb = a.g.nb, T = a.g.ntau, k = a.g.k;
    k_adj_lesA<<<nb, 128, 0, s>>>(a);
    k_adj_qA<<<nblk((int64_t)(std::max(n, T) + 1) * nb, 128), 128, 0, s>>>(a);
    const int width = std::max(n + 1, T + 1);
    k_adj_sigA<<<dim3(nblk((int64_t)a.nq * width * 32, 128), 4), 128, 0, s>>>(a, width);
    k_adj_bulk<<<nb, 128, 0, s>>>(a);
    const unsigned S = NG_ADJ_SPLIT;
    k_adj_tvrow<<<dim3(n, S), 256, 0, s>>>(a);
    k_adj_rrow<<<dim3(n, S), 256, 0, s>>>(a);
    if (!a.full) {
        k_adj_tvcol<<<dim3(T + 1, S), 256, 0, s>>>(a);
        k_adj_rcol<<<dim3(n - k, S), 256, 0, s>>>(a);
        k_adj_lcol<<<dim3(n, S), 256, 0, s>>>(a);
        if (n - k - 1 > 0) k_adj_lrow<<<dim3(n - k - 1, S), 256, 0, s>>>(a);
    }
    k_adj_qtv<<<dim3(T + 1, S), 256, 0, s>>>(a);
    k_adj_cur<<<nblk(2 * (int64_t)(n + 1) + T + 1 + (int64_t)k * k, 128), 128, 0, s>>>(a);
    k_adj_sigma2b<<<nblk(std::max(n, T) + 1, 128), 128, 0, s>>>(a.g, n, Glc, a.cSw, a.cmfw, 1, FuncV{(cplx*)U, 1},
                                                                cLoc);
    k_adj_ce0<<<nblk(nb, 128), 128, 0, s>>>(nb, a.cmfw, 1, ce0_row);
    k_adj_bcast<<<nblk((2 * (int64_t)(n + 1) + T + 1) * nb, 256), 256, 0, s>>>(a.g, n, cLoc, a.cw, a.cSw, a.cmfw);
    return cudaGetLastError();
}

cudaError_t adj_predictor(const Grid& g, int n, SliceV cw, cplx* cGr, cplx* cGl, cplx* cGt, cudaStream_t s) {
    k_adj_extrap_diag<<<nblk((int64_t)(2 * (n - g.k) + g.ntau + 1) * g.nb, 128), 128, 0, s>>>(g, n, cw, cGr, cGl, cGt);
    k_adj_extrap_cols<<<nblk(g.nb, 128), 128, 0, s>>>(g, n, cw, cGr, cGl);
    return cudaGetLastError();
}

cudaError_t adj_sigma2b(const Grid& g, int n, SliceV Lc, SliceV cS, const cplx* cmf_row, const cplx* U, SliceV out,
                        cudaStream_t s) {
    k_adj_sigma2b<<<nblk(std::max(n, g.ntau) + 1, 128), 128, 0, s>>>(g, n, Lc, cS, cmf_row, 1, FuncV{(cplx*)U, 1},
                                                                    out);
    return cudaGetLastError();
}

cudaError_t adj_slice_copy(int n, int ntau, int ld, SliceV src, SliceV dst, cudaStream_t s) {
    const int64_t items = (2 * (int64_t)(n + 1) + ntau + 1) * ld;
    k_slice_copy<<<nblk(items, 256), 256, 0, s>>>(n, ntau, ld, src, dst);
    return cudaGetLastError();
}

cudaError_t adj_seed(const Grid& g, const cplx* seed, cplx* cGl, cudaStream_t s) {
    k_adj_seed<<<nblk((int64_t)(g.nt + 1) * g.nb, 256), 256, 0, s>>>(g, seed, cGl);
    return cudaGetLastError();
}

cudaError_t adj_boot_gather(const Grid& g, const cplx* r, const cplx* l, const cplx* tv, int ld, cplx* out,
                            cudaStream_t s) {
    k_boot_gather<<<nblk(boot_E(g.k, g.ntau) * ld, 256), 256, 0, s>>>(g, r, l, tv, ld, out);
    return cudaGetLastError();
}

cudaError_t adj_boot_start(const AdjBoot& b, cudaStream_t s) {
    const size_t smem = sizeof(cplx) * (size_t)(boot_E(b.g.k, b.g.ntau) + (int64_t)b.g.k * (b.g.ntau + 1));
    cudaError_t e = cudaFuncSetAttribute(k_adj_start, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_adj_start<<<b.g.nb, NG_BOOT_THREADS, smem, s>>>(b);
    return cudaGetLastError();
}

cudaError_t adj_boot_reduce(int64_t E, int nb, const cplx* Pk, cplx* out, cudaStream_t s) {
    k_adj_boot_reduce<<<nblk(E * 32, 256), 256, 0, s>>>(E, nb, Pk, out);
    return cudaGetLastError();
}

cudaError_t adj_boot_update(int64_t E, int nb, const cplx* ctot, const cplx* cL, cplx* mu, double* dist,
                            cudaStream_t s) {
    k_adj_boot_update<<<nblk(E * nb, 256), 256, 0, s>>>(E, nb, ctot, cL, mu, dist);
    return cudaGetLastError();
}

cudaError_t adj_ce0_rows(int rows, int nb, const cplx* cmf, double* ce0, cudaStream_t s) {
    k_adj_ce0_rows<<<nblk((int64_t)rows * nb, 128), 128, 0, s>>>(rows, nb, cmf, ce0);
    return cudaGetLastError();
}
