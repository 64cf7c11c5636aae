// Types and launch wrappers of the discrete adjoint (ng_adjoint.cu), shared with the C ABI
// translation unit (ng_api.cu).
#pragma once

#include "ng_common.cuh"

struct SliceV {
    cplx* ret;   // element j (0..n) at ret[j * ld]
    cplx* les;   // element j (0..n) at les[j * ld]
    cplx* tv;    // element m (0..ntau) at tv[m * ld]
};

// Everything the kernels of one backward pass of step n read and write.
struct AdjStep {
    Grid g;
    int n, full, m0, nq;        // (A) rows of the lesser column: m0..n (nq rows); full: n <= 2k
    // final forward history (slices < n), per k (ldk = nb) and shared (ldk = 1)
    const cplx *Gr, *Gl, *Gt, *Gm;
    const cplx *Sr, *Sl, *St;
    const cplx* mf;             // eps_mf, val[(t+1) nb + kb]
    // values of slice n in this corrector pass
    SliceV Gc;                  // per k
    SliceV Sc;                  // shared
    const cplx* mfc;            // eps_mf(n) per k
    // cotangents: history (per k / shared), eps_mf (per k), and of slice n in this pass
    cplx *cGr, *cGl, *cGt;
    cplx *cSr, *cSl, *cSt;
    cplx* cmf;
    SliceV cw;                  // per k
    SliceV cSw;                 // shared
    cplx* cmfw;                 // [nb]
    // work vectors of this pass
    cplx* cA;                   // [NG_MAXQ][nb] cotangents of the (A) rows' right-hand sides
    cplx* caccR;                // [n+1][nb]   retarded (B) columns
    cplx* caccT;                // [ntau+1][nb] left-mixing columns
    cplx* crhs;                 // [n+1][nb]   lesser (B) rows
    cplx* cMn;                  // [nb]        cotangent of M_n
    cplx* retA;                 // [(k+1)^2][nb] cotangents of Sigma~^R(n-l, n-j) of the ret (A) block
    cplx* part;                 // [NG_ADJ_NPART][NG_ADJ_SPLIT][len] partial sums of shared cotangents
    int64_t plen;               // stride of part
};

#define NG_ADJ_NPART 8
// the history kernels split each row over NG_ADJ_SPLIT blocks (grid y); part holds one block
// sum per split, [NG_ADJ_NPART][NG_ADJ_SPLIT][plen]
#define NG_ADJ_SPLIT 4
enum { P_TVROW = 0, P_TVCOL, P_RROW, P_RCOL, P_LCOL, P_LROW, P_QTV };

struct AdjBoot {
    Grid g;
    const cplx *Gr, *Gl, *Gt, *Gm;   // final forward G (per k)
    const cplx *Sr, *Sl, *St;        // final Sigma (shared)
    const cplx* mf;                  // eps_mf (per k), val[(t+1) nb + kb]
    const cplx* mu;                  // [E][nb] cotangent of slices 0..k (input)
    cplx* Pk;                        // [E][nb] Sigma cotangent of slices 0..k (output, per k)
    cplx* cmfx;                      // [(k+2)][nb] eps_mf cotangent, row t+1 (output, added)
};
__host__ __device__ __forceinline__ int64_t boot_E(int k, int T) { return 2 * tri(k + 1) + (int64_t)(k + 1) * (T + 1); }

#define NG_BOOT_THREADS 128

// ---- launch wrappers (ng_adjoint.cu); each returns the launch status -------------------
// integration weights of the adjoint kernels, k = 1..NG_KMAX, for the current device
cudaError_t adj_load_weights(const NgWeights* all);
// one corrector pass of step n backwards: the Dyson step's transpose, then the second-Born
// slice and the Hartree term at the captured G_loc slice Glc, leaving the cotangent of the
// pass's input slice in a.cw (per problem) and adding Re c(eps_mf(n)) to ce0_row
cudaError_t adj_pass(const AdjStep& a, SliceV Glc, const cplx* U, SliceV cLoc, double* ce0_row, cudaStream_t s);
// predictor of step n transposed into the history cotangents
cudaError_t adj_predictor(const Grid& g, int n, SliceV cw, cplx* cGr, cplx* cGl, cplx* cGt, cudaStream_t s);
cudaError_t adj_sigma2b(const Grid& g, int n, SliceV Lc, SliceV cS, const cplx* cmf_row, const cplx* U, SliceV out,
                        cudaStream_t s);
cudaError_t adj_slice_copy(int n, int ntau, int ld, SliceV src, SliceV dst, cudaStream_t s);
cudaError_t adj_seed(const Grid& g, const cplx* seed, cplx* cGl, cudaStream_t s);
cudaError_t adj_boot_gather(const Grid& g, const cplx* r, const cplx* l, const cplx* tv, int ld, cplx* out,
                            cudaStream_t s);
cudaError_t adj_boot_start(const AdjBoot& b, cudaStream_t s);
cudaError_t adj_boot_reduce(int64_t E, int nb, const cplx* Pk, cplx* out, cudaStream_t s);
cudaError_t adj_boot_update(int64_t E, int nb, const cplx* ctot, const cplx* cL, cplx* mu, double* dist,
                            cudaStream_t s);
cudaError_t adj_ce0_rows(int rows, int nb, const cplx* cmf, double* ce0, cudaStream_t s);
