// C ABI of libng (include/ng.h): argument validation, workspaces and kernel launches.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/ng.h"
#include "ng_setup.cuh"
#include "ng_slice.cuh"
#include "ng_step32.cuh"
#include "ng_stepsplit.cuh"
#include "ng_obs.cuh"
#include "ng_ubatch.cuh"
#include "ng_stepdf.cuh"
#include "ng_conv_launch.h"
#include "ng_tvfft.h"
#include "ng_gw.cuh"
#include "ng_vie2_launch.h"
#include "ng_adjoint_types.h"
#include <cmath>

// double-float copy of one contour function (NG_DF64 time steps), as Shadow
struct ShadowDF {
    void* buf = nullptr;
    size_t bytes = 0;
    const void* key_ret = nullptr;
    int key_nt = -1, key_ntau = -1, key_nf = -1, key_ldk = -1;
    int upto = -2;
    HermVdf v;
};

// FP32 copy of one contour function (NG_F32C time steps): the buffer, the identity of the
// FP64 source it mirrors and the last slice converted (-2: nothing, -1: mat only).
struct Shadow {
    void* buf = nullptr;
    size_t bytes = 0;
    const void* key_ret = nullptr;
    int key_nt = -1, key_ntau = -1, key_nf = -1, key_ldk = -1;
    int upto = -2;
    HermV32 v;
};


struct ng_ctx {
    int k = 0;
    int device = 0;
    int sms = 1;                     // streaming multiprocessors of the device (grid sizing)
    NgWeights W;
    char err[512] = {0};
    int* d_status = nullptr;
    double* d_scalar = nullptr;      // one device double for distances
    cplx* d_eps = nullptr;           // scratch for host eps arrays
    size_t d_eps_bytes = 0;
    void* ws_mat = nullptr;          // Matsubara workspace
    size_t ws_mat_bytes = 0;
    void* ws_st = nullptr;           // start-up workspace
    size_t ws_st_bytes = 0;
    void* ws_prev = nullptr;         // previous iterate for the driver's convergence checks
    size_t ws_prev_bytes = 0;
    void* ws_gw = nullptr;           // GW driver: bosonic P, K, K^ddagger on the whole contour
    size_t ws_gw_bytes = 0;
    void* ws_bnd = nullptr;          // small-batch boundary: chunk partials of the (A)-row sums
    size_t ws_bnd_bytes = 0;
    void* ws_gwk = nullptr;          // k-space GW: compact real-space slice buffers
    size_t ws_gwk_bytes = 0;
    void* ws_gwmat = nullptr;        // GW driver: Matsubara workspace of the chi solve (ws_mat
    size_t ws_gwmat_bytes = 0;       // keeps the LU factors of G^M between iterations)
    // per-launch timing of the time-step kernels (ng_profile_enable / ng_profile_read)
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    double prof_flops = 0.0;
    std::vector<int> ev_kind;        // 0 bulk, 1 boundary, 2 FFT source pre-pass, 3 GW chain, per event pair
    Shadow shG, shS;                 // FP32 copies of G and Sigma for NG_F32C
    ShadowDF dfG, dfS;               // double-float copies of G and Sigma for NG_DF64
    void* ws_obs = nullptr;          // per-problem observables before the batch sum
    size_t ws_obs_bytes = 0;
    void* ws_minv = nullptr;         // M_n^-1 per problem of the current step
    size_t ws_minv_bytes = 0;
    void* ws_uni = nullptr;          // problem table of the element-wise step (nf = 4, 8)
    size_t ws_uni_bytes = 0;
    int uni_key_nb = -1;
    const void *uni_key_G = nullptr, *uni_key_S = nullptr, *uni_key_eps = nullptr;
    void* ws_usrc = nullptr;         // element-wise step: chunk partials of the (A) sources
    size_t ws_usrc_bytes = 0;
    void* ws_adj = nullptr;          // adjoint: iterate store, work vectors, start-slice buffers
    size_t ws_adj_bytes = 0;
    // the corrector iterates of every step held in ws_adj by ng_adjoint_forward, for
    // ng_adjoint_2b(segment = NG_ADJ_RECORDED); the shape they were recorded for
    bool adj_rec = false;
    int adj_rec_nt = 0, adj_rec_ntau = 0, adj_rec_nb = 0, adj_rec_corr = 0;
    const void* adj_rec_G = nullptr;
    // tuned bulk block sizes of earlier batches, by batch shape (problems per nf, largest
    // ntau, largest nt in steps of 256)
    std::vector<std::pair<std::vector<int>, int>> tune_cache;
    int tvsrc = NG_TVSRC_AUTO;       // evaluation of the left-mixing Matsubara source
    int bulk_split = NG_BULK_AUTO;   // one thread or one warp per bulk item (ng_set_bulk_split)
    void* ws_tvq = nullptr;          // FFT correlation of the source, [m][a][b][kb]
    size_t ws_tvq_bytes = 0;
    void* ws_tw = nullptr;           // twiddle table of length tw_L
    size_t ws_tw_bytes = 0;
    int tw_L = 0;
};

namespace {

bool g_weights_loaded[64] = {false};

// Integration weights of every order into constant memory of device `dev` (current): this
// file's c_W and the own copies of the adjoint, convolution and vie2 translation units,
// together, once per device.
ng_status load_weights_once(int dev) {
    if (dev < 0 || dev >= 64) return NG_EUNSUPPORTED;
    if (g_weights_loaded[dev]) return NG_OK;
    NgWeights all[NG_KMAX];
    for (int k = 1; k <= NG_KMAX; ++k) ng_make_weights(k, &all[k - 1]);
    if (cudaMemcpyToSymbol(c_W, all, sizeof(all)) != cudaSuccess || adj_load_weights(all) != cudaSuccess ||
        conv_load_weights(all) != cudaSuccess || vie2_load_weights(all) != cudaSuccess) {
        cudaGetLastError();
        return NG_ECUDA;
    }
    g_weights_loaded[dev] = true;
    return NG_OK;
}

ng_status fail(ng_ctx* c, ng_status s, const char* fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

#define CUDA_TRY(ctx, call)                                                                   \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(ctx, NG_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));       \
    } while (0)

ng_status check_launch(ng_ctx* c, const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, NG_ECUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
    return NG_OK;
}

ng_status ensure(ng_ctx* c, void** p, size_t* have, size_t need) {
    if (*have >= need) return NG_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *have = 0;
    if (cudaMalloc(p, need) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, NG_ENOMEM, "workspace allocation of %zu bytes failed", need);
    }
    *have = need;
    return NG_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// boson_ok: the call also takes bosonic functions (sig = +1; vie2 and convolution)
ng_status check_grid(ng_ctx* c, const ng_grid* g, Grid* out, bool boson_ok = false) {
    if (!c) return NG_EINVAL;
    if (!g) return fail(c, NG_EINVAL, "grid is NULL");
    if (g->korder != c->k) return fail(c, NG_EINVAL, "grid korder %d differs from the context order %d", g->korder, c->k);
    if (g->sig != -1 && !(boson_ok && g->sig == 1))
        return fail(c, NG_EINVAL, boson_ok ? "sig must be -1 (fermions) or +1 (bosons)" : "only fermions (sig = -1) are supported");
    if (g->nt < 2 * c->k + 2) return fail(c, NG_EINVAL, "nt = %d must be >= 2k+2 = %d", g->nt, 2 * c->k + 2);
    if (g->ntau < 2 * c->k + 2) return fail(c, NG_EINVAL, "ntau = %d must be >= 2k+2 = %d", g->ntau, 2 * c->k + 2);
    if (g->nbatch < 1) return fail(c, NG_EINVAL, "nbatch must be >= 1");
    if (!(g->h > 0.0) || !(g->beta > 0.0)) return fail(c, NG_EINVAL, "h and beta must be positive");
    if (g->nf < 1) return fail(c, NG_EINVAL, "nf must be >= 1");
    if (g->nf != 1 && g->nf != 2 && g->nf != 4 && g->nf != 8)
        return fail(c, NG_EUNSUPPORTED, "nf = %d: this build supports nf = 1, 2, 4, 8", g->nf);
    out->nt = g->nt;
    out->ntau = g->ntau;
    out->nf = g->nf;
    out->nb = g->nbatch;
    out->k = c->k;
    out->sig = g->sig;
    out->h = g->h;
    out->beta = g->beta;
    out->mu = g->mu;
    out->htau = g->beta / g->ntau;
    return NG_OK;
}

ng_status check_herm(ng_ctx* c, const Grid& g, const ng_herm& X, const char* name, bool need_rt, HermV* out,
                     int want_ldk /* 0: either */) {
    if (X.ldk != 1 && X.ldk != g.nb) return fail(c, NG_EINVAL, "%s.ldk = %d must be 1 or nbatch = %d", name, X.ldk, g.nb);
    if (want_ldk && X.ldk != want_ldk && !(g.nb == 1))
        return fail(c, NG_EINVAL, "%s.ldk = %d must be %d", name, X.ldk, want_ldk);
    if (!X.mat || !aligned16(X.mat)) return fail(c, NG_EINVAL, "%s.mat is NULL or not 16-byte aligned", name);
    if (need_rt) {
        if (!X.ret || !X.les || !X.tv || !aligned16(X.ret) || !aligned16(X.les) || !aligned16(X.tv))
            return fail(c, NG_EINVAL, "%s.ret/les/tv is NULL or not 16-byte aligned", name);
    }
    const int dd = g.nf * g.nf;
    out->mat = Comp{(cplx*)X.mat, X.ldk, dd};
    out->ret = Comp{(cplx*)X.ret, X.ldk, dd};
    out->les = Comp{(cplx*)X.les, X.ldk, dd};
    out->tv = Comp{(cplx*)X.tv, X.ldk, dd};
    return NG_OK;
}

ng_status check_func(ng_ctx* c, const Grid& g, const ng_func& f, const char* name, FuncV* out) {
    if (!f.val || !aligned16(f.val)) return fail(c, NG_EINVAL, "%s.val is NULL or not 16-byte aligned", name);
    if (f.ldk != 1 && f.ldk != g.nb) return fail(c, NG_EINVAL, "%s.ldk = %d must be 1 or nbatch", name, f.ldk);
    out->p = (cplx*)f.val;
    out->ldk = f.ldk;
    return NG_OK;
}

inline unsigned nblocks(int64_t items, int threads) { return (unsigned)((items + threads - 1) / threads); }

// event pair for one profiled launch; returns the index of the start event or -1
long prof_pair(ng_ctx* c, int kind) {
    if (!c->prof) return -1;
    while (c->ev_pool.size() < c->ev_used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return -1; }
        c->ev_pool.push_back(e);
    }
    long i = (long)c->ev_used;
    c->ev_used += 2;
    c->ev_kind.push_back(kind);
    return i;
}

// algorithmic complex block multiply-adds of one bulk launch at step n (history and source
// sums of the three bulk tasks; the BDF terms and the per-item matrix inverse are not counted).
// fft: the left-mixing source comes from the FFT pre-pass, the bulk items add only the
// quadrature corrections (q_tv_fft).
double bulk_cmacs(const Grid& g, int n, bool fft = false) {
    const int k = g.k, T = g.ntau;
    auto corr = [&](int L) {   // correction terms of one piece with row length L
        return L <= k ? (k + 1) * (k + 1) + L + 1 : (L <= 2 * k + 1 ? L + 1 : 2 * (k + 1));
    };
    double per_tv = 0.0;
    for (int m = 0; m <= T; ++m) {
        per_tv += n;                                              // history j = 0..n-1
        if (fft) {
            per_tv += corr(m) + corr(T - m);
            continue;
        }
        per_tv += (m <= k) ? (k + 1) * (k + 1) : (m + 1);         // C^tv_2
        per_tv += (m >= T - k) ? (k + 1) * (k + 1) : (T - m + 1); // C^tv_3
    }
    double per_ret = 0.0;
    for (int m = 0; m <= n - k - 1; ++m) per_ret += n - m;
    double per_les = 0.0;
    if (n >= 2 * k + 1)
        for (int m = 1; m <= n - k - 1; ++m) per_les += (m <= k ? k + 1 : m + 1) + (T + 1) + n;
    return (double)g.nb * (per_tv + per_ret + per_les);
}

// ---------------------------------------------------------------------------------------
// launch bodies templated on the orbital dimension
// ---------------------------------------------------------------------------------------
template <int D>
ng_status launch_minv(ng_ctx* c, const Grid& g, int n, const HermV& S, const FuncV& eps, cudaStream_t s) {
    ng_status st = ensure(c, &c->ws_minv, &c->ws_minv_bytes, sizeof(cplx) * D * D * (size_t)g.nb);
    if (st) return st;
    k_minv_step<D><<<nblocks(g.nb, 128), 128, 0, s>>>(g, n, S, eps, (cplx*)c->ws_minv, c->d_status);
    return check_launch(c, "k_minv_step");
}

// FFT pre-pass of the left-mixing source of step n (*tvq = nullptr when the direct sums are
// used: NG_TVSRC_DIRECT, or nf / ntau outside what the transforms support)
// prof: record the pre-pass as its own profile entry (not inside a GW evaluation, which is
// timed as a whole)
ng_status prep_tvfft(ng_ctx* c, const Grid& g, int n, const HermV& G, const HermV& S, cudaStream_t s,
                     const cplx** tvq, bool prof = true) {
    *tvq = nullptr;
    if (c->tvsrc == NG_TVSRC_DIRECT || !tvfft_supported(g.nf, g.ntau)) return NG_OK;
    ng_status st;
    const int L = tvfft_length(g.ntau);
    if (c->tw_L != L) {
        if ((st = ensure(c, &c->ws_tw, &c->ws_tw_bytes, sizeof(cplx) * (size_t)(L / 2)))) return st;
        if (tvfft_twiddles((cplx*)c->ws_tw, L, s) != cudaSuccess) return check_launch(c, "k_twiddle");
        c->tw_L = L;
    }
    const size_t need = sizeof(cplx) * (size_t)(g.ntau + 1) * g.nf * g.nf * g.nb;
    if ((st = ensure(c, &c->ws_tvq, &c->ws_tvq_bytes, need))) return st;
    long e = prof ? prof_pair(c, 2) : -1;
    if (e >= 0) cudaEventRecord(c->ev_pool[e], s);
    if (tvfft_launch(g, n, S.tv, G.mat, (const cplx*)c->ws_tw, (cplx*)c->ws_tvq, s) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, NG_ECUDA, "launch of k_tvsrc_fft failed");
    }
    if (e >= 0) cudaEventRecord(c->ev_pool[e + 1], s);
    *tvq = (const cplx*)c->ws_tvq;
    return NG_OK;
}

// the boundary of step n in three launches, its (A)-row sums over (row, problem, chunk) blocks;
// pre_done: the retarded start-up ran in the leading warps of the bulk launch
template <int D>
ng_status boundary_spread(ng_ctx* c, const Grid& g, int n, const HermV& G, const HermV& S, const FuncV& eps,
                          bool pre_done, cudaStream_t s) {
    ng_status st;
    const int k = g.k, nq = (n <= 2 * k) ? n : k + 1;
    const int64_t terms = std::max(n, g.ntau) + 1;
    const int64_t want = (4 * (int64_t)c->sms + (int64_t)nq * g.nb - 1) / ((int64_t)nq * g.nb);
    const int nchunk = (int)std::max<int64_t>(1, std::min<int64_t>({want, (terms + NG_BND_THREADS - 1) / NG_BND_THREADS, 64}));
    const size_t need = sizeof(cplx) * (size_t)nq * g.nb * nchunk * 2 * D * D;
    if ((st = ensure(c, &c->ws_bnd, &c->ws_bnd_bytes, need))) return st;
    if (!pre_done) {
        k_bnd_pre<D><<<g.nb, 32, 0, s>>>(g, n, G, S, eps, c->d_status);
        if ((st = check_launch(c, "k_bnd_pre"))) return st;
    }
    k_bnd_src<D><<<dim3(nq, g.nb, nchunk), NG_BND_THREADS, 0, s>>>(g, n, G, S, nchunk, (cplx*)c->ws_bnd);
    if ((st = check_launch(c, "k_bnd_src"))) return st;
    k_bnd_fin<D><<<g.nb, 32, 0, s>>>(g, n, G, S, eps, nchunk, (const cplx*)c->ws_bnd, c->d_status);
    return check_launch(c, "k_bnd_fin");
}

template <int D>
ng_status launch_timestep(ng_ctx* c, const Grid& g, int n, const HermV& G, const HermV& S, const FuncV& eps,
                          cudaStream_t s) {
    const int k = g.k, thr = 128;
    const int64_t it_les = (n >= 2 * k + 1) ? (int64_t)g.nb * (n - k - 1) : 0;
    const int64_t it_tv = (int64_t)g.nb * (g.ntau + 1);
    const int64_t it_ret = (int64_t)g.nb * (n - k);
    const int b_les = (int)nblocks(it_les, thr), b_tv = (int)nblocks(it_tv, thr), b_ret = (int)nblocks(it_ret, thr);
    // small batches: one warp per item when one thread per item would not give each SM a block;
    // the warp form splits the left-mixing source over its lanes instead of the FFT pre-pass
    const int64_t items = it_les + it_tv + it_ret;
    const bool warp = c->bulk_split == NG_BULK_WARP || (c->bulk_split == NG_BULK_AUTO && items < (int64_t)c->sms * thr);
    // small batches: the boundary's (A)-row sums spread over (row, problem, chunk) blocks, and
    // with the warp bulk its retarded start-up in the bulk launch's leading warps
    const int nq = (n <= 2 * k) ? n : k + 1;
    const bool spread = c->bulk_split == NG_BULK_WARP ||
                        (c->bulk_split == NG_BULK_AUTO && (int64_t)nq * g.nb < 2 * (int64_t)c->sms);
    const int64_t w_pre = (warp && spread) ? g.nb : 0;
    const cplx* tvq = nullptr;
    ng_status sm = warp ? NG_OK : prep_tvfft(c, g, n, G, S, s, &tvq);
    if (sm) return sm;
    long e0 = prof_pair(c, 0);
    if (e0 >= 0) cudaEventRecord(c->ev_pool[e0], s);
    if ((sm = launch_minv<D>(c, g, n, S, eps, s))) return sm;
    if (warp) {
        k_step_bulk_w<D><<<nblocks((w_pre + items) * 32, thr), thr, 0, s>>>(g, n, G, S, eps, (const cplx*)c->ws_minv,
                                                                           w_pre, it_les, it_tv, it_ret, c->d_status);
    } else {
        k_step_bulk<D><<<b_les + b_tv + b_ret, thr, 0, s>>>(g, n, G, S, eps, (const cplx*)c->ws_minv, b_les, b_tv,
                                                            b_ret, tvq, c->d_status);
    }
    ng_status st = check_launch(c, warp ? "k_step_bulk_w" : "k_step_bulk");
    if (st) return st;
    if (e0 >= 0) {
        cudaEventRecord(c->ev_pool[e0 + 1], s);
        c->prof_flops += 8.0 * D * D * D * bulk_cmacs(g, n, tvq != nullptr);
    }
    long e1 = prof_pair(c, 1);
    if (e1 >= 0) cudaEventRecord(c->ev_pool[e1], s);
    if (spread) {
        st = boundary_spread<D>(c, g, n, G, S, eps, w_pre > 0, s);
        if (e1 >= 0) cudaEventRecord(c->ev_pool[e1 + 1], s);
        return st;
    }
    k_step_boundary<D><<<g.nb, NG_BND_THREADS, 0, s>>>(g, n, G, S, eps, c->d_status);
    if (e1 >= 0) cudaEventRecord(c->ev_pool[e1 + 1], s);
    return check_launch(c, "k_step_boundary");
}

// Bring the FP32 copy of X up to date for a time step at n: slices <= n-1 once (they are
// final), slice n always when `current` (Sigma's slice n changes between corrector passes).
ng_status update_shadow(ng_ctx* c, Shadow& sh, const Grid& g, const HermV& X, int n, bool current, cudaStream_t s) {
    const int dd = g.nf * g.nf, ldk = X.ret.ldk, T1 = g.ntau + 1;
    if (sh.key_ret != X.ret.p || sh.key_nt != g.nt || sh.key_ntau != g.ntau || sh.key_nf != g.nf || sh.key_ldk != ldk) {
        const size_t el = (size_t)T1 + 2 * (size_t)tri(g.nt + 1) + (size_t)(g.nt + 1) * T1;
        ng_status st = ensure(c, &sh.buf, &sh.bytes, sizeof(cplx32) * el * dd * ldk);
        if (st) return st;
        cplx32* p = (cplx32*)sh.buf;
        sh.v.mat = Comp32{p, ldk};
        sh.v.ret = Comp32{p + (size_t)T1 * dd * ldk, ldk};
        sh.v.les = Comp32{sh.v.ret.p + (size_t)tri(g.nt + 1) * dd * ldk, ldk};
        sh.v.tv = Comp32{sh.v.les.p + (size_t)tri(g.nt + 1) * dd * ldk, ldk};
        sh.key_ret = X.ret.p;
        sh.key_nt = g.nt;
        sh.key_ntau = g.ntau;
        sh.key_nf = g.nf;
        sh.key_ldk = ldk;
        sh.upto = -2;
    }
    auto conv = [&](int n0, int n1) -> ng_status {
        if (n1 < n0 || n1 < -1) return NG_OK;
        const int a = n0 < 0 ? 0 : n0;
        const int64_t items = (2 * (tri(n1 + 1) - tri(a)) + (int64_t)(n1 - a + 1) * T1 + (n0 < 0 ? T1 : 0)) * dd * ldk;
        const unsigned blocks = (unsigned)std::min<int64_t>((items + 255) / 256, 152 * 16);
        k_shadow<<<blocks, 256, 0, s>>>(g, n0, n1, X, sh.v, ldk);
        return check_launch(c, "k_shadow");
    };
    ng_status st;
    if (sh.upto < n - 1) {
        if ((st = conv(sh.upto + 1, n - 1))) return st;
        sh.upto = n - 1;
    }
    if (current && (st = conv(n, n))) return st;
    return NG_OK;
}

ng_status update_shadow_df(ng_ctx* c, ShadowDF& sh, const Grid& g, const HermV& X, int n, bool current, cudaStream_t s) {
    const int dd = g.nf * g.nf, ldk = X.ret.ldk, T1 = g.ntau + 1;
    if (sh.key_ret != X.ret.p || sh.key_nt != g.nt || sh.key_ntau != g.ntau || sh.key_nf != g.nf || sh.key_ldk != ldk) {
        const size_t el = (size_t)T1 + 2 * (size_t)tri(g.nt + 1) + (size_t)(g.nt + 1) * T1;
        ng_status st = ensure(c, &sh.buf, &sh.bytes, sizeof(float4) * el * dd * ldk);
        if (st) return st;
        float4* p = (float4*)sh.buf;
        sh.v.mat = Comp64x{p, ldk};
        sh.v.ret = Comp64x{p + (size_t)T1 * dd * ldk, ldk};
        sh.v.les = Comp64x{sh.v.ret.p + (size_t)tri(g.nt + 1) * dd * ldk, ldk};
        sh.v.tv = Comp64x{sh.v.les.p + (size_t)tri(g.nt + 1) * dd * ldk, ldk};
        sh.key_ret = X.ret.p;
        sh.key_nt = g.nt;
        sh.key_ntau = g.ntau;
        sh.key_nf = g.nf;
        sh.key_ldk = ldk;
        sh.upto = -2;
    }
    auto conv = [&](int n0, int n1) -> ng_status {
        if (n1 < n0 || n1 < -1) return NG_OK;
        const int a = n0 < 0 ? 0 : n0;
        const int64_t items = (2 * (tri(n1 + 1) - tri(a)) + (int64_t)(n1 - a + 1) * T1 + (n0 < 0 ? T1 : 0)) * dd * ldk;
        const unsigned blocks = (unsigned)std::min<int64_t>((items + 255) / 256, 152 * 16);
        k_shadow_df<<<blocks, 256, 0, s>>>(g, n0, n1, X, sh.v, ldk);
        return check_launch(c, "k_shadow_df");
    };
    ng_status st;
    if (sh.upto < n - 1) {
        if ((st = conv(sh.upto + 1, n - 1))) return st;
        sh.upto = n - 1;
    }
    if (current && (st = conv(n, n))) return st;
    return NG_OK;
}

template <int D>
ng_status launch_timestepdf(ng_ctx* c, const Grid& g, int n, const HermV& G, const HermV& S, const FuncV& eps,
                            cudaStream_t s) {
    ng_status st;
    if ((st = update_shadow_df(c, c->dfG, g, G, n, false, s))) return st;
    if ((st = update_shadow_df(c, c->dfS, g, S, n, true, s))) return st;
    const int k = g.k, thr = 128;
    const int64_t it_les = (n >= 2 * k + 1) ? (int64_t)g.nb * (n - k - 1) : 0;
    const int64_t it_tv = (int64_t)g.nb * (g.ntau + 1);
    const int64_t it_ret = (int64_t)g.nb * (n - k);
    const int b_les = (int)nblocks(it_les, thr), b_tv = (int)nblocks(it_tv, thr), b_ret = (int)nblocks(it_ret, thr);
    if ((st = launch_minv<D>(c, g, n, S, eps, s))) return st;
    const cplx* tvq = nullptr;
    if ((st = prep_tvfft(c, g, n, G, S, s, &tvq))) return st;
    long e0 = prof_pair(c, 0);
    if (e0 >= 0) cudaEventRecord(c->ev_pool[e0], s);
    k_step_bulkdf<D><<<b_les + b_tv + b_ret, thr, 0, s>>>(g, n, G, S, c->dfG.v, c->dfS.v, (const cplx*)c->ws_minv,
                                                          b_les, b_tv, b_ret, tvq, c->d_status);
    if ((st = check_launch(c, "k_step_bulkdf"))) return st;
    if (e0 >= 0) {
        cudaEventRecord(c->ev_pool[e0 + 1], s);
        c->prof_flops += 8.0 * D * D * D * bulk_cmacs(g, n, tvq != nullptr);
    }
    long e1 = prof_pair(c, 1);
    if (e1 >= 0) cudaEventRecord(c->ev_pool[e1], s);
    k_step_boundary<D><<<g.nb, NG_BND_THREADS, 0, s>>>(g, n, G, S, eps, c->d_status);
    if (e1 >= 0) cudaEventRecord(c->ev_pool[e1 + 1], s);
    return check_launch(c, "k_step_boundary");
}

template <int D>
ng_status launch_timestep32(ng_ctx* c, const Grid& g, int n, const HermV& G, const HermV& S, const FuncV& eps,
                            cudaStream_t s) {
    ng_status st;
    if ((st = update_shadow(c, c->shG, g, G, n, false, s))) return st;
    if ((st = update_shadow(c, c->shS, g, S, n, true, s))) return st;
    const int k = g.k, thr = 128;
    const int64_t it_les = (n >= 2 * k + 1) ? (int64_t)g.nb * (n - k - 1) : 0;
    const int64_t it_tv = (int64_t)g.nb * (g.ntau + 1);
    const int64_t it_ret = (int64_t)g.nb * (n - k);
    const int b_les = (int)nblocks(it_les, thr), b_tv = (int)nblocks(it_tv, thr), b_ret = (int)nblocks(it_ret, thr);
    const cplx* tvq = nullptr;
    if ((st = prep_tvfft(c, g, n, G, S, s, &tvq))) return st;
    long e0 = prof_pair(c, 0);
    if (e0 >= 0) cudaEventRecord(c->ev_pool[e0], s);
    if ((st = launch_minv<D>(c, g, n, S, eps, s))) return st;
    if (D == 1 && g.nb % 2 == 0) {
        // two problems per thread (16-byte loads of the FP32 copies)
        const int np = g.nb / 2;
        const int p_les = it_les ? (int)nblocks((int64_t)np * (n - k - 1), thr) : 0;
        const int p_tv = (int)nblocks((int64_t)np * (g.ntau + 1), thr), p_ret = (int)nblocks((int64_t)np * (n - k), thr);
        k_step_bulk32p<<<p_les + p_tv + p_ret, thr, 0, s>>>(g, n, G, S, c->shG.v, c->shS.v, (const cplx*)c->ws_minv,
                                                            p_les, p_tv, p_ret, tvq, c->d_status);
    } else {
        k_step_bulk32<D><<<b_les + b_tv + b_ret, thr, 0, s>>>(g, n, G, S, c->shG.v, c->shS.v, eps,
                                                              (const cplx*)c->ws_minv, b_les, b_tv, b_ret, tvq,
                                                              c->d_status);
    }
    if ((st = check_launch(c, "k_step_bulk32"))) return st;
    if (e0 >= 0) {
        cudaEventRecord(c->ev_pool[e0 + 1], s);
        c->prof_flops += 8.0 * D * D * D * bulk_cmacs(g, n, tvq != nullptr);
    }
    long e1 = prof_pair(c, 1);
    if (e1 >= 0) cudaEventRecord(c->ev_pool[e1], s);
    k_step_boundary<D><<<g.nb, NG_BND_THREADS, 0, s>>>(g, n, G, S, eps, c->d_status);
    if (e1 >= 0) cudaEventRecord(c->ev_pool[e1 + 1], s);
    return check_launch(c, "k_step_boundary");
}

// Matsubara solve.  refine_steps = 0: exact solve by a fresh LU of the current operator (the
// factors and row interchanges are kept).  refine_steps > 0 (driver only, after a fresh LU of
// the same grid): iterative refinement of the current G^M against the current operator with
// the kept factors, at most refine_steps steps; *refined_ok reports convergence of the
// refinement (update sum below ref_tol); otherwise the caller falls back to a fresh LU.
// LU solve of nb augmented systems [A | B] (N x (N + nrhs)) in ws_A: one block per problem for
// batches that fill the SMs (or when several solves run concurrently on streams, spread =
// false), else column by column with the rank-1 updates over the whole GPU (the same factors
// bitwise)
ng_status lu_solve(ng_ctx* c, int N, int nrhs, int nb, cplx* ws_A, int* ws_piv, cudaStream_t s, bool spread = true) {
    ng_status st;
    if (!spread || 4 * (int64_t)nb >= c->sms) {
        const size_t smem = sizeof(cplx) * (size_t)(2 * N + nrhs) + NG_LU_THREADS * (sizeof(double) + sizeof(int));
        CUDA_TRY(c, cudaFuncSetAttribute(k_lu_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_lu_solve<<<nb, NG_LU_THREADS, smem, s>>>(N, nrhs, ws_A, ws_piv, c->d_status);
        return check_launch(c, "k_lu_solve");
    }
    for (int col = 0; col < N; ++col) {
        k_lu_col<<<nb, NG_LU_THREADS, 0, s>>>(N, nrhs, ws_A, ws_piv, col, c->d_status);
        const int64_t items = (int64_t)(N - col - 1) * (N + nrhs - col - 1);
        if (items > 0) k_lu_rank1<<<dim3(nblocks(items, 256), nb), 256, 0, s>>>(N, nrhs, ws_A, col);
        if (col % 256 == 0 && (st = check_launch(c, "k_lu_col/k_lu_rank1"))) return st;
    }
    k_lu_backsub<<<nb, NG_LU_THREADS, 0, s>>>(N, nrhs, ws_A);
    return check_launch(c, "k_lu_backsub");
}

template <int D>
ng_status launch_mat(ng_ctx* c, const Grid& g, const HermV& G, const HermV& S, const FuncV& eps, cudaStream_t s,
                     int refine_steps = 0, double ref_tol = 0.0, bool* refined_ok = nullptr, void* ws_ext = nullptr) {
    const int T = g.ntau, N = (T + 1) * D, ld = N + D;
    const size_t b_g = sizeof(cplx) * (size_t)g.nb * (T + 1) * D * D;
    const size_t b_A = sizeof(cplx) * (size_t)g.nb * N * ld;
    const size_t b_piv = sizeof(int) * (size_t)g.nb * N + 256;
    ng_status st = NG_OK;
    if (!ws_ext && (st = ensure(c, &c->ws_mat, &c->ws_mat_bytes, 3 * b_g + b_A + b_piv))) return st;
    cplx* ws_g = (cplx*)(ws_ext ? ws_ext : c->ws_mat);
    cplx* ws_K = ws_g + b_g / sizeof(cplx);
    cplx* ws_r = ws_K + b_g / sizeof(cplx);
    cplx* ws_A = ws_r + b_g / sizeof(cplx);
    int* ws_piv = (int*)(ws_A + b_A / sizeof(cplx));
    const int64_t items = (int64_t)(T + 1) * g.nb;
    k_mat_g<D><<<nblocks(items, 128), 128, 0, s>>>(g, eps, ws_g);
    if ((st = check_launch(c, "k_mat_g"))) return st;
    k_mat_K<D><<<nblocks(items, 128), 128, 0, s>>>(g, S, ws_g, ws_K);
    if ((st = check_launch(c, "k_mat_K"))) return st;
    if (refine_steps > 0) {
        *refined_ok = false;
        double prev = 1e300;
        for (int r = 0; r < refine_steps; ++r) {
            k_mat_resid<D><<<nblocks(items, 128), 128, 0, s>>>(g, ws_g, ws_K, G, ws_r);
            if ((st = check_launch(c, "k_mat_resid"))) return st;
            CUDA_TRY(c, cudaMemsetAsync(c->d_scalar, 0, sizeof(double), s));
            k_lu_resolve<<<g.nb, NG_LU_THREADS, 0, s>>>(g, N, D, ws_A, ws_piv, ws_r, G, c->d_scalar);
            if ((st = check_launch(c, "k_lu_resolve"))) return st;
            double dsum = 0.0;
            CUDA_TRY(c, cudaMemcpyAsync(&dsum, c->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, s));
            CUDA_TRY(c, cudaStreamSynchronize(s));
            if (!(dsum == dsum)) return NG_OK;               // non-finite: fall back
            if (dsum == 0.0 || dsum > 0.5 * prev) {           // at the round-off floor, or stalled
                *refined_ok = dsum < ref_tol;
                return NG_OK;
            }
            prev = dsum;
        }
        return NG_OK;
    }
    const int64_t ab = (int64_t)(T + 1) * (T + 2) * g.nb;
    k_mat_assemble<D><<<nblocks(ab, 256), 256, 0, s>>>(g, ws_g, ws_K, ws_A);
    if ((st = check_launch(c, "k_mat_assemble"))) return st;
    if ((st = lu_solve(c, N, D, g.nb, ws_A, ws_piv, s, ws_ext == nullptr))) return st;
    k_mat_store<D><<<nblocks(items, 128), 128, 0, s>>>(g, ws_A, G, c->d_status);
    return check_launch(c, "k_mat_store");
}

template <int D>
ng_status launch_start(ng_ctx* c, const Grid& g, const HermV& G, const HermV& S, const FuncV& eps, cudaStream_t s,
                       void* ws_ext = nullptr) {
    const int k = g.k, N = k * D;
    const size_t need = sizeof(cplx) * (size_t)g.nb * (N * N + k * D * D);
    ng_status st = NG_OK;
    if (!ws_ext && (st = ensure(c, &c->ws_st, &c->ws_st_bytes, need))) return st;
    cplx* ws = (cplx*)(ws_ext ? ws_ext : c->ws_st);
    k_start_ret<D><<<nblocks(g.nb, 64), 64, 0, s>>>(g, G, S, eps, ws, c->d_status);
    if ((st = check_launch(c, "k_start_ret"))) return st;
    k_start_tv<D><<<nblocks((int64_t)(g.ntau + 1) * g.nb, 128), 128, 0, s>>>(g, G, S, ws, c->d_status);
    if ((st = check_launch(c, "k_start_tv"))) return st;
    k_start_les<D><<<nblocks((int64_t)(k + 1) * g.nb, 64), 64, 0, s>>>(g, G, S, ws, c->d_status);
    return check_launch(c, "k_start_les");
}

// Matsubara slice of the integral form (Eq. vie2_langreth_m): the discretised equation
// G^M + [F * G]^M = Q^M is the linear system of the integro-differential Matsubara solve with
// K = -F^M and right-hand side Q^M, solved by the same dense LU per problem.
template <int D>
__global__ void k_v2_mat_fill(Grid g, HermV F, HermV Q, cplx* ws_g, cplx* ws_K) {
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= (int64_t)(g.ntau + 1) * g.nb) return;
    const int kb = (int)(item % g.nb), m = (int)(item / g.nb);
    const Mat<D> q = gmat<D>(Q, m, kb), f = gmat<D>(F, m, kb);
    const int64_t o = ((int64_t)kb * (g.ntau + 1) + m) * D * D;
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) {
            ws_g[o + a * D + b] = q.v[a][b];
            ws_K[o + a * D + b] = cneg(f.v[a][b]);
        }
}

// refine_steps > 0: refine the current G^M with the LU factors kept in *ws from the previous
// solve (the operator of a self-consistency loop changes little between iterations), as the
// Dyson Matsubara solve does; *refined_ok tells whether the residual reached ref_tol
template <int D>
ng_status launch_vie2_mat(ng_ctx* c, const Grid& g, const HermV& G, const HermV& F, const HermV& Q, cudaStream_t s,
                          void** ws, size_t* ws_bytes, int refine_steps = 0, double ref_tol = 0.0,
                          bool* refined_ok = nullptr) {
    const int T = g.ntau, N = (T + 1) * D, ld = N + D;
    const size_t b_g = sizeof(cplx) * (size_t)g.nb * (T + 1) * D * D;
    const size_t b_A = sizeof(cplx) * (size_t)g.nb * N * ld;
    const size_t b_piv = sizeof(int) * (size_t)g.nb * N + 256;
    ng_status st = NG_OK;
    if ((st = ensure(c, ws, ws_bytes, 3 * b_g + b_A + b_piv))) return st;
    cplx* ws_g = (cplx*)*ws;
    cplx* ws_K = ws_g + b_g / sizeof(cplx);
    cplx* ws_r = ws_K + b_g / sizeof(cplx);
    cplx* ws_A = ws_K + 2 * (b_g / sizeof(cplx));
    int* ws_piv = (int*)(ws_A + b_A / sizeof(cplx));
    const int64_t items = (int64_t)(T + 1) * g.nb;
    k_v2_mat_fill<D><<<nblocks(items, 128), 128, 0, s>>>(g, F, Q, ws_g, ws_K);
    if ((st = check_launch(c, "k_v2_mat_fill"))) return st;
    if (refine_steps > 0) {
        *refined_ok = false;
        double prev = 1e300;
        for (int r = 0; r < refine_steps; ++r) {
            k_mat_resid<D><<<nblocks(items, 128), 128, 0, s>>>(g, ws_g, ws_K, G, ws_r);
            if ((st = check_launch(c, "k_mat_resid"))) return st;
            CUDA_TRY(c, cudaMemsetAsync(c->d_scalar, 0, sizeof(double), s));
            k_lu_resolve<<<g.nb, NG_LU_THREADS, 0, s>>>(g, N, D, ws_A, ws_piv, ws_r, G, c->d_scalar);
            if ((st = check_launch(c, "k_lu_resolve"))) return st;
            double dsum = 0.0;
            CUDA_TRY(c, cudaMemcpyAsync(&dsum, c->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, s));
            CUDA_TRY(c, cudaStreamSynchronize(s));
            if (!(dsum == dsum)) return NG_OK;               // non-finite: a fresh solve follows
            if (dsum == 0.0 || dsum > 0.5 * prev) {           // at the round-off floor, or stalled
                *refined_ok = dsum < ref_tol;
                return NG_OK;
            }
            prev = dsum;
        }
        return NG_OK;
    }
    k_mat_assemble<D><<<nblocks((int64_t)(T + 1) * (T + 2) * g.nb, 256), 256, 0, s>>>(g, ws_g, ws_K, ws_A);
    if ((st = check_launch(c, "k_mat_assemble"))) return st;
    if ((st = lu_solve(c, N, D, g.nb, ws_A, ws_piv, s))) return st;
    k_mat_store<D><<<nblocks(items, 128), 128, 0, s>>>(g, ws_A, G, c->d_status);
    return check_launch(c, "k_mat_store");
}

// one warp per vie2 bulk item: forced, or for batches with fewer items than 128 per SM
bool vie2_warp(const ng_ctx* c, const Grid& g, int n) {
    const int64_t items = (int64_t)g.nb * ((n - 1) + (g.ntau + 1) + n);
    return c->bulk_split == NG_BULK_WARP || (c->bulk_split == NG_BULK_AUTO && items < (int64_t)c->sms * 128);
}

ng_status vie2_mat_d(ng_ctx* c, const Grid& g, const HermV& G, const HermV& F, const HermV& Q, cudaStream_t s,
                     void** ws, size_t* ws_bytes, int refine_steps = 0, double ref_tol = 0.0, bool* ok = nullptr) {
    switch (g.nf) {
    case 1: return launch_vie2_mat<1>(c, g, G, F, Q, s, ws, ws_bytes, refine_steps, ref_tol, ok);
    case 2: return launch_vie2_mat<2>(c, g, G, F, Q, s, ws, ws_bytes, refine_steps, ref_tol, ok);
    case 4: return launch_vie2_mat<4>(c, g, G, F, Q, s, ws, ws_bytes, refine_steps, ref_tol, ok);
    default: return fail(c, NG_EUNSUPPORTED, "the vie2 solver supports nf = 1, 2, 4");
    }
}

template <int D>
ng_status launch_free(ng_ctx* c, const Grid& g, const HermV& G, const cplx* eps_dev, double scale, cudaStream_t s) {
    const int64_t nel = (g.ntau + 1) + 2 * tri(g.nt + 1) + (int64_t)(g.nt + 1) * (g.ntau + 1);
    k_free_gf<D><<<nblocks(nel * g.nb, 128), 128, 0, s>>>(g, G, eps_dev, scale);
    return check_launch(c, "k_free_gf");
}

ng_status do_kreduce(ng_ctx* c, const Grid& g, int tstp, const HermV& L, const HermV& Gk, cudaStream_t s,
                     const double* wk = nullptr) {
    const int cnt = tstp < 0 ? g.ntau + 1 : 2 * (tstp + 1) + g.ntau + 1;
    const int64_t warps = (int64_t)cnt * g.nf * g.nf;
    k_kreduce<<<nblocks(warps * 32, 256), 256, 0, s>>>(g, tstp, L, Gk, wk);
    return check_launch(c, "k_kreduce");
}

// ---- k-point sharding over ranks -----------------------------------------------------------
// Rank r owns the whole blocks [floor(r B / P), floor((r+1) B / P)) of the B = ceil(nk / 32)
// blocks of NG_KBLK consecutive k indices.
void shard_map(int nk, int nranks, BlkMap* m) {
    const int64_t B = (nk + NG_KBLK - 1) / NG_KBLK;
    for (int r = 0; r <= nranks; ++r) m->first[r] = (int)(B * r / nranks);
}
int shard_maxb(const BlkMap& m, int nranks) {
    int mb = 0;
    for (int r = 0; r < nranks; ++r) mb = std::max(mb, m.first[r + 1] - m.first[r]);
    return mb;
}
size_t shard_send_bytes(const Grid& g, int maxb) {
    const size_t cnt_max = (size_t)2 * (g.nt + 1) + g.ntau + 1;
    return std::max<size_t>(sizeof(double), (size_t)maxb * cnt_max * g.nf * g.nf * sizeof(cplx));
}

// resolved shard of one rank for the driver
struct ShardRt {
    const ng_shard* sh;
    BlkMap map;
    int maxb;
    int kb0;  // global k index of local problem 0
};

ng_status check_shard(ng_ctx* c, const Grid& g, const ng_shard* sh, ShardRt* rt) {
    if (sh->nranks < 1 || sh->nranks > NG_MAXRANKS) return fail(c, NG_EINVAL, "nranks = %d must be in 1..%d", sh->nranks, NG_MAXRANKS);
    if (sh->rank < 0 || sh->rank >= sh->nranks) return fail(c, NG_EINVAL, "rank %d out of 0..%d", sh->rank, sh->nranks - 1);
    if ((sh->nk + NG_KBLK - 1) / NG_KBLK < sh->nranks)
        return fail(c, NG_EINVAL, "nk = %d gives fewer blocks of %d than ranks (%d)", sh->nk, NG_KBLK, sh->nranks);
    rt->sh = sh;
    shard_map(sh->nk, sh->nranks, &rt->map);
    rt->maxb = shard_maxb(rt->map, sh->nranks);
    rt->kb0 = rt->map.first[sh->rank] * NG_KBLK;
    const int count = std::min(sh->nk, rt->map.first[sh->rank + 1] * NG_KBLK) - rt->kb0;
    if (g.nb != count) return fail(c, NG_EINVAL, "grid.nbatch = %d, but rank %d owns %d k-points", g.nb, sh->rank, count);
    if (!sh->exchange) return fail(c, NG_EINVAL, "shard exchange callback is NULL");
    if (!sh->send || !sh->recv || !aligned16(sh->send) || !aligned16(sh->recv))
        return fail(c, NG_EINVAL, "shard send/recv buffers are NULL or not 16-byte aligned");
    if (sh->send_bytes < shard_send_bytes(g, rt->maxb))
        return fail(c, NG_EINVAL, "shard send_bytes %zu < %zu needed", sh->send_bytes, shard_send_bytes(g, rt->maxb));
    return NG_OK;
}

// Gloc slice tstp: on one GPU the single-kernel fixed-order reduction; over ranks, the block sums
// of the local k-points, the exchange of all ranks' block sums, and their sum in block order.
ng_status do_kreduce_rt(ng_ctx* c, const Grid& g, int tstp, const HermV& L, const HermV& Gk, cudaStream_t s,
                        const ShardRt* rt) {
    if (!rt) return do_kreduce(c, g, tstp, L, Gk, s);
    const ng_shard* sh = rt->sh;
    const int cnt = tstp < 0 ? g.ntau + 1 : 2 * (tstp + 1) + g.ntau + 1;
    const int dd = g.nf * g.nf;
    const int nbl = rt->map.first[sh->rank + 1] - rt->map.first[sh->rank];
    const int64_t warps = (int64_t)nbl * cnt * dd;
    k_kreduce_partial<<<nblocks(warps * 32, 256), 256, 0, s>>>(g, tstp, Gk, nullptr, rt->kb0, (cplx*)sh->send);
    ng_status st = check_launch(c, "k_kreduce_partial");
    if (st) return st;
    if (sh->exchange(sh->user, (size_t)rt->maxb * cnt * dd * sizeof(cplx)) != 0)
        return fail(c, NG_ECOMM, "the exchange of the k-block sums failed (slice %d)", tstp);
    k_kreduce_combine<<<nblocks((int64_t)cnt * dd, 128), 128, 0, s>>>(g, tstp, L, (const cplx*)sh->recv, sh->nk,
                                                                      sh->nranks, rt->maxb, rt->map, 0);
    return check_launch(c, "k_kreduce_combine");
}
ng_status do_sigma(ng_ctx* c, const Grid& g, int tstp, const HermV& S, const HermV& L, const FuncV& U, cudaStream_t s) {
    const int cnt = tstp < 0 ? g.ntau + 1 : 2 * (tstp + 1) + g.ntau + 1;
    k_sigma2b<<<nblocks((int64_t)cnt * g.nf * g.nf, 128), 128, 0, s>>>(g, tstp, S, L, U);
    return check_launch(c, "k_sigma2b");
}
// GW launches on slice tstp: local (L = 1, whole-contour views) or on the ring of L momenta
// (views of compact real-space slice buffers and the k-space stores)
inline SliceView whole(const HermV& h) { return SliceView{h, nullptr}; }
inline SliceView compact(cplx* buf) { return SliceView{HermV{}, buf}; }
ng_status do_gw_pol(ng_ctx* c, const Grid& g, int tstp, int L, const SliceView& P, const SliceView& K,
                    const SliceView& Kcc, const SliceView& G, const FuncV& U, cudaStream_t s) {
    const int cnt = tstp < 0 ? g.ntau + 1 : 2 * (tstp + 1) + g.ntau + 1;
    k_gw_pol<<<nblocks((int64_t)cnt * g.nf * g.nf * L, 128), 128, 0, s>>>(g, tstp, L, P, K, Kcc, G, U);
    return check_launch(c, "k_gw_pol");
}
ng_status do_gw_sigma(ng_ctx* c, const Grid& g, int tstp, int L, const SliceView& S, const SliceView& G,
                      const SliceView& X, const FuncV& U, cudaStream_t s) {
    const int cnt = tstp < 0 ? g.ntau + 1 : 2 * (tstp + 1) + g.ntau + 1;
    k_gw_sigma<<<nblocks((int64_t)cnt * g.nf * g.nf * L, 128), 128, 0, s>>>(g, tstp, L, S, G, X, U);
    return check_launch(c, "k_gw_sigma");
}
// lattice Fourier transform of every element of slice tstp along its L momenta / sites
ng_status do_kfft(ng_ctx* c, const Grid& g, int tstp, int L, const SliceView& in, const SliceView& out, int sign,
                  double scale, cudaStream_t s) {
    int log2L = -1;
    if ((L & (L - 1)) == 0) {
        log2L = 0;
        while ((1 << log2L) < L) ++log2L;
    }
    const int cnt = tstp < 0 ? g.ntau + 1 : 2 * (tstp + 1) + g.ntau + 1;
    const int64_t nvec = (int64_t)cnt * g.nf * g.nf;
    // vectors per block: up to 1024 values, but at least two blocks per SM when the slice allows
    const int64_t fill = std::max<int64_t>(1, nvec / (2 * (int64_t)c->sms));
    const int vpb = (int)std::max<int64_t>(1, std::min<int64_t>(std::max(1, 1024 / L), fill));
    const size_t smem = sizeof(cplx) * (size_t)(vpb + 1) * L;
    if (smem > 48 * 1024)
        CUDA_TRY(c, cudaFuncSetAttribute(k_kfft_slice, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int thr = std::min(256, std::max(64, vpb * L / 4 / 32 * 32));
    k_kfft_slice<<<(unsigned)((nvec + vpb - 1) / vpb), thr, smem, s>>>(g, tstp, L, log2L, vpb, in, out, sign, scale);
    return check_launch(c, "k_kfft_slice");
}
ng_status do_hartree(ng_ctx* c, const Grid& g, int tstp, const FuncV& mf, const FuncV& e0, const HermV& L, const FuncV& U,
                     double nbar, cudaStream_t s) {
    k_hartree<<<nblocks((int64_t)mf.ldk * g.nf * g.nf, 128), 128, 0, s>>>(g, tstp, mf, e0, L, U, nbar);
    return check_launch(c, "k_hartree");
}
// ---------------------------------------------------------------------------------------
// element-wise time step for nf = 4, 8 and for the uneven batch: one launch table per
// chunk of <= NG_UMAXP problems at the same global step n
// ---------------------------------------------------------------------------------------
struct UHost {
    int D, nt, ntau, k;
};
ng_status ustep(ng_ctx* c, const UProb* d_probs, const std::vector<UHost>& info, const std::vector<int>& active, int n,
                int threads, cudaStream_t s) {
    ng_status st;
    // the boundary kernels use more than the default 48 KB of dynamic shared memory (set on
    // every call: the attribute is per device, and ustep serves the batch and the nf = 4, 8 step)
    CUDA_TRY(c, cudaFuncSetAttribute(k_uboundary_ret, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NG_UBND_SMEM));
    CUDA_TRY(c, cudaFuncSetAttribute(k_uboundary_les, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NG_UBND_SMEM));
    for (size_t c0 = 0; c0 < active.size(); c0 += NG_UMAXP) {
        UTable tab;
        memset(&tab, 0, sizeof(tab));
        tab.n = n;
        int blk = 0;
        const size_t c1 = std::min(active.size(), c0 + (size_t)NG_UMAXP);
        for (size_t i = c0; i < c1; ++i) {
            const UHost& u = info[active[i]];
            const int ipb = threads / (u.D * u.D);
            const int j = (int)(i - c0);
            tab.prob[j] = active[i];
            tab.start[j] = blk;
            tab.nles[j] = (n >= 2 * u.k + 1) ? (n - u.k - 1 + ipb - 1) / ipb : 0;
            tab.ntv[j] = (u.ntau + 1 + ipb - 1) / ipb;
            const int nret = (n - u.k + ipb - 1) / ipb;
            blk += tab.nles[j] + tab.ntv[j] + nret;
        }
        tab.np = (int)(c1 - c0);
        tab.start[tab.np] = blk;
        // chunks of the (A) rows' source sums: max(n, k) + 1 + ntau + 1 summation indices
        int nsum = 0;
        for (size_t i = c0; i < c1; ++i) nsum = std::max(nsum, std::max(n, info[active[i]].k) + 2 + info[active[i]].ntau);
        tab.chunk = 128;
        tab.nchunk = (nsum + tab.chunk - 1) / tab.chunk;
        {   // capacity for twice the current need, so the buffer grows a logarithmic number of times
            const size_t per = sizeof(cplx) * (size_t)NG_MAXQ * 2 * NG_UMAXD * NG_UMAXD;
            const size_t need = per * (size_t)tab.np * tab.nchunk;
            if (need > c->ws_usrc_bytes && (st = ensure(c, &c->ws_usrc, &c->ws_usrc_bytes, 2 * need))) return st;
            tab.src = (cplx*)c->ws_usrc;
        }
        k_uminv<<<tab.np, 32, 0, s>>>(d_probs, tab, c->d_status);
        if ((st = check_launch(c, "k_uminv"))) return st;
        long e0 = prof_pair(c, 0);
        if (e0 >= 0) cudaEventRecord(c->ev_pool[e0], s);
        k_ubulk<<<blk, threads, sizeof(cplx) * threads, s>>>(d_probs, tab, c->d_status);
        if ((st = check_launch(c, "k_ubulk"))) return st;
        if (e0 >= 0) cudaEventRecord(c->ev_pool[e0 + 1], s);
        long e1 = prof_pair(c, 1);
        if (e1 >= 0) cudaEventRecord(c->ev_pool[e1], s);
        k_uboundary_ret<<<tab.np, NG_UBND_THREADS, NG_UBND_SMEM, s>>>(d_probs, tab, c->d_status);
        k_usrc<<<dim3(tab.nchunk, NG_MAXQ, tab.np), NG_USRC_THREADS, 0, s>>>(d_probs, tab);
        k_uboundary_les<<<tab.np, NG_UBND_THREADS, NG_UBND_SMEM, s>>>(d_probs, tab, c->d_status);
        if (e1 >= 0) cudaEventRecord(c->ev_pool[e1 + 1], s);
        if ((st = check_launch(c, "k_uboundary_ret/k_usrc/k_uboundary_les"))) return st;
        if (c->prof) {
            for (size_t i = c0; i < c1; ++i) {
                const UHost& u = info[active[i]];
                Grid gg;
                gg.k = u.k;
                gg.ntau = u.ntau;
                gg.nb = 1;
                c->prof_flops += 8.0 * u.D * u.D * u.D * bulk_cmacs(gg, n);
            }
        }
    }
    return NG_OK;
}

// uniform-batch time step with nf = 4, 8: every interleaved problem kb as one UProb
ng_status utimestep_uniform(ng_ctx* c, const Grid& g, int n, const HermV& G, const HermV& S, const FuncV& eps,
                            cudaStream_t s) {
    // the M_n^-1 blocks start on a 256-byte boundary after the table (sizeof(UProb) is a
    // multiple of 8 only, and the blocks are read as 16-byte complex numbers)
    const size_t off_minv = (sizeof(UProb) * (size_t)g.nb + 255) / 256 * 256;
    const size_t need = off_minv + sizeof(cplx) * 64 * (size_t)g.nb;
    ng_status st = ensure(c, &c->ws_uni, &c->ws_uni_bytes, need);
    if (st) return st;
    UProb* d_probs = (UProb*)c->ws_uni;
    cplx* d_minv = (cplx*)((char*)c->ws_uni + off_minv);
    if (c->uni_key_nb != g.nb || c->uni_key_G != G.ret.p || c->uni_key_S != S.ret.p || c->uni_key_eps != eps.p) {
        std::vector<UProb> h(g.nb);
        for (int kb = 0; kb < g.nb; ++kb) {
            h[kb].g = g;
            h[kb].g.nb = 1;
            h[kb].G = G;
            h[kb].S = S;
            h[kb].eps = eps;
            h[kb].kb = kb;
            h[kb].minv = d_minv + 64 * (size_t)kb;
        }
        CUDA_TRY(c, cudaMemcpyAsync(d_probs, h.data(), sizeof(UProb) * h.size(), cudaMemcpyHostToDevice, s));
        CUDA_TRY(c, cudaStreamSynchronize(s));
        c->uni_key_nb = g.nb;
        c->uni_key_G = G.ret.p;
        c->uni_key_S = S.ret.p;
        c->uni_key_eps = eps.p;
    }
    std::vector<UHost> info(g.nb, UHost{g.nf, g.nt, g.ntau, g.k});
    std::vector<int> active(g.nb);
    for (int kb = 0; kb < g.nb; ++kb) active[kb] = kb;
    return ustep(c, d_probs, info, active, n, 128, s);
}

// serial schedule: the left-mixing row by the bulk kernel (its other tasks empty), then the whole
// retarded row and lesser column by implementation (A), one block per problem
template <int D>
ng_status launch_timestep_serial(ng_ctx* c, const Grid& g, int n, const HermV& G, const HermV& S, const FuncV& eps,
                                 cudaStream_t s) {
    const int thr = 128;
    const int b_tv = (int)nblocks((int64_t)g.nb * (g.ntau + 1), thr);
    ng_status st = launch_minv<D>(c, g, n, S, eps, s);
    if (st) return st;
    const cplx* tvq = nullptr;
    if ((st = prep_tvfft(c, g, n, G, S, s, &tvq))) return st;
    k_step_bulk<D><<<b_tv, thr, 0, s>>>(g, n, G, S, eps, (const cplx*)c->ws_minv, 0, b_tv, 0, tvq, c->d_status);
    if ((st = check_launch(c, "k_step_bulk"))) return st;
    k_step_serial<D><<<g.nb, NG_BND_THREADS, 0, s>>>(g, n, G, S, eps, c->d_status);
    return check_launch(c, "k_step_serial");
}

ng_status do_timestep(ng_ctx* c, const Grid& g, int n, const HermV& G, const HermV& S, const FuncV& eps, cudaStream_t s,
                      int precision = NG_FP64) {
    if (g.nf > 2) {
        if (precision != NG_FP64) return fail(c, NG_EUNSUPPORTED, "NG_F32C and NG_DF64 need nf <= 2");
        // nf = 4, 8: the element-wise batch form (a warp holding 4 x 4 blocks per lane spills and
        // ran the 4-site chain's step at half this form's speed)
        return utimestep_uniform(c, g, n, G, S, eps, s);
    }
    if (precision == NG_DF64)
        return g.nf == 1 ? launch_timestepdf<1>(c, g, n, G, S, eps, s) : launch_timestepdf<2>(c, g, n, G, S, eps, s);
    if (precision == NG_F32C)
        return g.nf == 1 ? launch_timestep32<1>(c, g, n, G, S, eps, s) : launch_timestep32<2>(c, g, n, G, S, eps, s);
    return g.nf == 1 ? launch_timestep<1>(c, g, n, G, S, eps, s) : launch_timestep<2>(c, g, n, G, S, eps, s);
}
ng_status do_mat(ng_ctx* c, const Grid& g, const HermV& G, const HermV& S, const FuncV& eps, cudaStream_t s,
                 void* ws = nullptr) {
    switch (g.nf) {
        case 1: return launch_mat<1>(c, g, G, S, eps, s, 0, 0.0, nullptr, ws);
        case 2: return launch_mat<2>(c, g, G, S, eps, s, 0, 0.0, nullptr, ws);
        case 4: return launch_mat<4>(c, g, G, S, eps, s, 0, 0.0, nullptr, ws);
        default: return launch_mat<8>(c, g, G, S, eps, s, 0, 0.0, nullptr, ws);
    }
}
// workspace bytes of one Matsubara solve and of one start-up (nb problems of grid g)
size_t mat_ws_bytes(const Grid& g) {
    const size_t D = g.nf, T = g.ntau, N = (T + 1) * D, ld = N + D;
    return 3 * sizeof(cplx) * g.nb * (T + 1) * D * D + sizeof(cplx) * g.nb * N * ld + sizeof(int) * g.nb * N + 256;
}
size_t start_ws_bytes(const Grid& g) {
    const size_t D = g.nf, N = (size_t)g.k * D;
    return sizeof(cplx) * g.nb * (N * N + g.k * D * D);
}
ng_status do_mat_refine(ng_ctx* c, const Grid& g, const HermV& G, const HermV& S, const FuncV& eps, cudaStream_t s,
                        int steps, double tol, bool* ok) {
    switch (g.nf) {
        case 1: return launch_mat<1>(c, g, G, S, eps, s, steps, tol, ok);
        case 2: return launch_mat<2>(c, g, G, S, eps, s, steps, tol, ok);
        case 4: return launch_mat<4>(c, g, G, S, eps, s, steps, tol, ok);
        default: return launch_mat<8>(c, g, G, S, eps, s, steps, tol, ok);
    }
}
ng_status do_start(ng_ctx* c, const Grid& g, const HermV& G, const HermV& S, const FuncV& eps, cudaStream_t s,
                   void* ws = nullptr) {
    switch (g.nf) {
        case 1: return launch_start<1>(c, g, G, S, eps, s, ws);
        case 2: return launch_start<2>(c, g, G, S, eps, s, ws);
        case 4: return launch_start<4>(c, g, G, S, eps, s, ws);
        default: return launch_start<8>(c, g, G, S, eps, s, ws);
    }
}
ng_status do_extrap(ng_ctx* c, const Grid& g, int n, const HermV& G, cudaStream_t s) {
    const int64_t items = (int64_t)(2 * (n + 2) + g.ntau + 1) * g.nf * g.nf * G.ret.ldk;
    k_extrapolate<<<nblocks(items, 128), 128, 0, s>>>(g, n, G);
    return check_launch(c, "k_extrapolate");
}
ng_status do_distance(ng_ctx* c, const Grid& g, int tstp, const HermV& A, const HermV& B, double* out, cudaStream_t s) {
    k_distance<<<4 * 152, 256, 0, s>>>(g, tstp, A, B, out);
    return check_launch(c, "k_distance");
}

}  // namespace

// =========================================================================================
// C ABI
// =========================================================================================
extern "C" {

ng_status ng_create(int korder, int device, ng_ctx** out) {
    if (!out) return NG_EINVAL;
    *out = nullptr;
    if (korder < 1 || korder > NG_KMAX) return NG_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return NG_ECUDA; }
    ng_ctx* c = new ng_ctx();
    c->k = korder;
    c->device = device;
    ng_make_weights(korder, &c->W);
    if (ng_status ws = load_weights_once(device)) {
        delete c;
        return ws;
    }
    if (cudaMalloc(&c->d_status, sizeof(int)) != cudaSuccess || cudaMalloc(&c->d_scalar, sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return NG_ENOMEM;
    }
    cudaMemset(c->d_status, 0, sizeof(int));
    if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || c->sms < 1) {
        cudaGetLastError();
        c->sms = 1;
    }
    *out = c;
    return NG_OK;
}

void ng_destroy(ng_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    cudaFree(c->d_status);
    cudaFree(c->d_scalar);
    cudaFree(c->d_eps);
    cudaFree(c->ws_mat);
    cudaFree(c->ws_st);
    cudaFree(c->ws_prev);
    cudaFree(c->ws_gw);
    cudaFree(c->ws_gwmat);
    cudaFree(c->ws_gwk);
    cudaFree(c->ws_bnd);
    cudaFree(c->shG.buf);
    cudaFree(c->shS.buf);
    cudaFree(c->dfG.buf);
    cudaFree(c->dfS.buf);
    cudaFree(c->ws_obs);
    cudaFree(c->ws_uni);
    cudaFree(c->ws_minv);
    cudaFree(c->ws_adj);
    cudaFree(c->ws_usrc);
    cudaFree(c->ws_tvq);
    cudaFree(c->ws_tw);
    delete c;
}

const char* ng_last_error(const ng_ctx* c) { return c ? c->err : "NULL context"; }

ng_status ng_status_sync(ng_ctx* c, void* stream, int* flags) {
    if (!c) return NG_EINVAL;
    CUDA_TRY(c, cudaStreamSynchronize((cudaStream_t)stream));
    int f = 0;
    CUDA_TRY(c, cudaMemcpy(&f, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    CUDA_TRY(c, cudaMemset(c->d_status, 0, sizeof(int)));
    if (flags) *flags = f;
    if (f & NGF_NONFINITE) return fail(c, NG_ENONFINITE, "device reported non-finite values (flags %d)", f);
    if (f & NGF_SINGULAR) return fail(c, NG_ESINGULAR, "device reported a singular matrix (flags %d)", f);
    return NG_OK;
}

ng_status ng_set_bulk_split(ng_ctx* c, int mode) {
    if (!c) return NG_EINVAL;
    if (mode != NG_BULK_AUTO && mode != NG_BULK_THREAD && mode != NG_BULK_WARP)
        return fail(c, NG_EINVAL, "unknown bulk mode %d", mode);
    c->bulk_split = mode;
    return NG_OK;
}

ng_status ng_set_tv_source(ng_ctx* c, int mode) {
    if (!c) return NG_EINVAL;
    if (mode != NG_TVSRC_AUTO && mode != NG_TVSRC_DIRECT) return fail(c, NG_EINVAL, "unknown source mode %d", mode);
    c->tvsrc = mode;
    return NG_OK;
}

ng_status ng_profile_enable(ng_ctx* c, int enable) {
    if (!c) return NG_EINVAL;
    if (enable) {
        c->ev_used = 0;
        c->ev_kind.clear();
        c->prof_flops = 0.0;
    }
    c->prof = enable != 0;
    return NG_OK;
}

ng_status ng_profile_read(ng_ctx* c, double* out) {
    if (!c || !out) return NG_EINVAL;
    for (int i = 0; i < 9; ++i) out[i] = 0.0;
    if (c->ev_used) CUDA_TRY(c, cudaEventSynchronize(c->ev_pool[c->ev_used - 1]));
    static const int slot[4] = {0, 3, 5, 7};   // bulk, boundary, FFT source, GW chain
    for (size_t p = 0; p < c->ev_kind.size(); ++p) {
        float ms = 0.f;
        CUDA_TRY(c, cudaEventElapsedTime(&ms, c->ev_pool[2 * p], c->ev_pool[2 * p + 1]));
        const int kind = c->ev_kind[p];
        out[slot[kind]] += ms;
        out[slot[kind] + 1] += 1;
    }
    out[2] = c->prof_flops;
    return NG_OK;
}

ng_status ng_weights(const ng_ctx* c, double* out) {
    if (!c || !out) return NG_EINVAL;
    for (int i = 0; i < 18; ++i) out[i] = 0.0;
    for (int j = 0; j <= c->k; ++j) {
        out[j] = c->W.a[j];
        out[6 + j] = c->W.omega[j];
        out[12 + j] = c->W.C[j];
    }
    return NG_OK;
}

ng_status ng_green_from_H_const(ng_ctx* c, const ng_grid* grid, ng_herm G, const double* eps_host, double scale,
                                void* stream) {
    Grid g;
    HermV Gv;
    ng_status st;
    if ((st = check_grid(c, grid, &g))) return st;
    if ((st = check_herm(c, g, G, "G", true, &Gv, g.nb))) return st;
    if (!eps_host) return fail(c, NG_EINVAL, "eps_host is NULL");
    const size_t bytes = sizeof(cplx) * (size_t)g.nb * g.nf * g.nf;
    if ((st = ensure(c, (void**)&c->d_eps, &c->d_eps_bytes, bytes))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(c, cudaMemcpyAsync(c->d_eps, eps_host, bytes, cudaMemcpyHostToDevice, s));
    switch (g.nf) {
        case 1: return launch_free<1>(c, g, Gv, c->d_eps, scale, s);
        case 2: return launch_free<2>(c, g, Gv, c->d_eps, scale, s);
        case 4: return launch_free<4>(c, g, Gv, c->d_eps, scale, s);
        default: return launch_free<8>(c, g, Gv, c->d_eps, scale, s);
    }
}

ng_status ng_dyson_mat(ng_ctx* c, const ng_grid* grid, ng_herm G, ng_herm S, ng_func eps, void* stream) {
    Grid g;
    HermV Gv, Sv;
    FuncV ev;
    ng_status st;
    if ((st = check_grid(c, grid, &g))) return st;
    if ((st = check_herm(c, g, G, "G", false, &Gv, g.nb))) return st;
    if ((st = check_herm(c, g, S, "Sigma", false, &Sv, 0))) return st;
    if ((st = check_func(c, g, eps, "eps", &ev))) return st;
    return do_mat(c, g, Gv, Sv, ev, (cudaStream_t)stream);
}

ng_status ng_dyson_start(ng_ctx* c, const ng_grid* grid, ng_herm G, ng_herm S, ng_func eps, void* stream) {
    Grid g;
    HermV Gv, Sv;
    FuncV ev;
    ng_status st;
    if ((st = check_grid(c, grid, &g))) return st;
    if ((st = check_herm(c, g, G, "G", true, &Gv, g.nb))) return st;
    if ((st = check_herm(c, g, S, "Sigma", true, &Sv, 0))) return st;
    if ((st = check_func(c, g, eps, "eps", &ev))) return st;
    return do_start(c, g, Gv, Sv, ev, (cudaStream_t)stream);
}

ng_status ng_dyson_timestep(ng_ctx* c, const ng_grid* grid, int tstp, ng_herm G, ng_herm S, ng_func eps, int precision,
                            int schedule, void* stream) {
    Grid g;
    HermV Gv, Sv;
    FuncV ev;
    ng_status st;
    if ((st = check_grid(c, grid, &g))) return st;
    if (tstp <= g.k || tstp > g.nt) return fail(c, NG_EINVAL, "tstp = %d must be in k+1..nt = %d..%d", tstp, g.k + 1, g.nt);
    if (precision != NG_FP64 && precision != NG_F32C && precision != NG_DF64)
        return fail(c, NG_EINVAL, "unknown precision %d", precision);
    if ((st = check_herm(c, g, G, "G", true, &Gv, g.nb))) return st;
    if ((st = check_herm(c, g, S, "Sigma", true, &Sv, 0))) return st;
    if ((st = check_func(c, g, eps, "eps", &ev))) return st;
    if (schedule == NG_SERIAL) {
        if (precision != NG_FP64) return fail(c, NG_EUNSUPPORTED, "the serial schedule runs in NG_FP64 only");
        if (g.nf > 2) return fail(c, NG_EUNSUPPORTED, "the serial schedule supports nf <= 2");
        return g.nf == 1 ? launch_timestep_serial<1>(c, g, tstp, Gv, Sv, ev, (cudaStream_t)stream)
                         : launch_timestep_serial<2>(c, g, tstp, Gv, Sv, ev, (cudaStream_t)stream);
    }
    if (schedule != NG_MIXED) return fail(c, NG_EINVAL, "unknown schedule %d", schedule);
    return do_timestep(c, g, tstp, Gv, Sv, ev, (cudaStream_t)stream, precision);
}

// argument checks shared by the vie2 entry points
static ng_status vie2_args(ng_ctx* c, const ng_grid* grid, ng_herm G, ng_herm F, ng_herm Fcc, ng_herm Q, bool rt,
                           Grid* g, HermV* Gv, HermV* Fv, HermV* Fccv, HermV* Qv) {
    ng_status st;
    if ((st = check_grid(c, grid, g, true))) return st;
    if (g->nf > 4) return fail(c, NG_EUNSUPPORTED, "the vie2 solver supports nf = 1, 2, 4");
    if ((st = check_herm(c, *g, G, "G", rt, Gv, g->nb))) return st;
    if ((st = check_herm(c, *g, F, "F", rt, Fv, 0))) return st;
    if ((st = check_herm(c, *g, Fcc, "Fcc", rt, Fccv, 0))) return st;
    return check_herm(c, *g, Q, "Q", rt, Qv, 0);
}

ng_status ng_vie2_mat(ng_ctx* c, const ng_grid* grid, ng_herm G, ng_herm F, ng_herm Q, void* stream) {
    Grid g;
    HermV Gv, Fv, Fccv, Qv;
    ng_status st;
    if ((st = vie2_args(c, grid, G, F, F, Q, false, &g, &Gv, &Fv, &Fccv, &Qv))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    return vie2_mat_d(c, g, Gv, Fv, Qv, s, &c->ws_mat, &c->ws_mat_bytes);
}

ng_status ng_vie2_start(ng_ctx* c, const ng_grid* grid, ng_herm G, ng_herm F, ng_herm Fcc, ng_herm Q, void* stream) {
    Grid g;
    HermV Gv, Fv, Fccv, Qv;
    ng_status st;
    if ((st = vie2_args(c, grid, G, F, Fcc, Q, true, &g, &Gv, &Fv, &Fccv, &Qv))) return st;
    if ((st = ensure(c, &c->ws_st, &c->ws_st_bytes, start_ws_bytes(g)))) return st;
    if (vie2_start_launch(g, Gv, Fv, Fccv, Qv, (cplx*)c->ws_st, c->d_status, (cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, NG_ECUDA, "launch of the vie2 start-up kernels failed");
    }
    return NG_OK;
}

ng_status ng_vie2_timestep(ng_ctx* c, const ng_grid* grid, int tstp, ng_herm G, ng_herm F, ng_herm Fcc, ng_herm Q,
                           int schedule, void* stream) {
    Grid g;
    HermV Gv, Fv, Fccv, Qv;
    ng_status st;
    if ((st = vie2_args(c, grid, G, F, Fcc, Q, true, &g, &Gv, &Fv, &Fccv, &Qv))) return st;
    if (tstp <= g.k || tstp > g.nt) return fail(c, NG_EINVAL, "tstp = %d must be in k+1..nt = %d..%d", tstp, g.k + 1, g.nt);
    if (schedule == NG_SERIAL) return fail(c, NG_EUNSUPPORTED, "the vie2 time step runs the mixed schedule only");
    if (schedule != NG_MIXED) return fail(c, NG_EINVAL, "unknown schedule %d", schedule);
    const cplx* tvq = nullptr;
    const bool w = vie2_warp(c, g, tstp);
    if (!w && (st = prep_tvfft(c, g, tstp, Gv, Fv, (cudaStream_t)stream, &tvq))) return st;
    if (vie2_step_launch(g, tstp, Gv, Fv, Fccv, Qv, tvq, w, c->d_status, (cudaStream_t)stream) !=
        cudaSuccess) {
        cudaGetLastError();
        return fail(c, NG_ECUDA, "launch of the vie2 time-step kernels failed");
    }
    return NG_OK;
}

ng_status ng_convolution_timestep(ng_ctx* c, const ng_grid* grid, int tstp, ng_herm C, ng_herm A, ng_herm Acc,
                                  ng_func f, ng_herm B, ng_herm Bcc, void* stream) {
    Grid g;
    HermV Cv, Av, Accv, Bv, Bccv;
    ng_status st;
    if ((st = check_grid(c, grid, &g, true))) return st;
    if (tstp < -1 || tstp > g.nt) return fail(c, NG_EINVAL, "tstp = %d must be in -1..nt = %d", tstp, g.nt);
    const bool rt = tstp >= 0;
    if ((st = check_herm(c, g, C, "C", rt, &Cv, 0))) return st;
    if ((st = check_herm(c, g, A, "A", rt, &Av, 0))) return st;
    if ((st = check_herm(c, g, Acc, "Acc", rt, &Accv, 0))) return st;
    if ((st = check_herm(c, g, B, "B", rt, &Bv, 0))) return st;
    if ((st = check_herm(c, g, Bcc, "Bcc", rt, &Bccv, 0))) return st;
    FuncV fv{nullptr, 1};
    if (f.val && (st = check_func(c, g, f, "f", &fv))) return st;
    const int nbe = C.ldk;
    if (nbe == 1 && g.nb > 1 &&
        (A.ldk != 1 || Acc.ldk != 1 || B.ldk != 1 || Bcc.ldk != 1 || (f.val && f.ldk != 1)))
        return fail(c, NG_EINVAL, "C.ldk = 1 needs every input shared (ldk = 1)");
    if (conv_launch(g, tstp, Cv, Av, Accv, fv, Bv, Bccv, nbe, c->d_status, (cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, NG_ECUDA, "launch of k_conv_slice failed");
    }
    return NG_OK;
}

ng_status ng_observables(ng_ctx* c, const ng_grid* grid, int tstp, ng_herm G, ng_herm S, ng_func eps0, ng_func epsmf,
                         double* out_dev, void* stream) {
    Grid g;
    HermV Gv, Sv;
    FuncV e0, mf;
    ng_status st;
    if ((st = check_grid(c, grid, &g))) return st;
    if (tstp < 0 || tstp > g.nt) return fail(c, NG_EINVAL, "tstp = %d must be in 0..nt", tstp);
    if ((st = check_herm(c, g, G, "G", true, &Gv, g.nb))) return st;
    if ((st = check_herm(c, g, S, "Sigma", true, &Sv, 0))) return st;
    if ((st = check_func(c, g, eps0, "eps0", &e0))) return st;
    if ((st = check_func(c, g, epsmf, "eps_mf", &mf))) return st;
    if (!out_dev) return fail(c, NG_EINVAL, "out_dev is NULL");
    if ((st = ensure(c, &c->ws_obs, &c->ws_obs_bytes, sizeof(double) * NG_NOBS * (size_t)g.nb))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (g.nf > 2) return fail(c, NG_EUNSUPPORTED, "ng_observables supports nf <= 2");
    if (g.nf == 1) k_observables<1><<<g.nb, NG_OBS_THREADS, 0, s>>>(g, tstp, Gv, Sv, e0, mf, (double*)c->ws_obs);
    else k_observables<2><<<g.nb, NG_OBS_THREADS, 0, s>>>(g, tstp, Gv, Sv, e0, mf, (double*)c->ws_obs);
    if ((st = check_launch(c, "k_observables"))) return st;
    k_observables_reduce<<<1, NG_OBS_THREADS, 0, s>>>(g.nb, (const double*)c->ws_obs, out_dev);
    return check_launch(c, "k_observables_reduce");
}

ng_status ng_precision_reset(ng_ctx* c) {
    if (!c) return NG_EINVAL;
    c->shG.upto = -2;
    c->shG.key_ret = nullptr;
    c->shS.upto = -2;
    c->shS.key_ret = nullptr;
    c->dfG.upto = -2;
    c->dfG.key_ret = nullptr;
    c->dfS.upto = -2;
    c->dfS.key_ret = nullptr;
    return NG_OK;
}

ng_status ng_kreduce_timestep(ng_ctx* c, const ng_grid* grid, int tstp, ng_herm Gloc, ng_herm Gk, const double* wk,
                              void* stream) {
    Grid g;
    HermV L, K;
    ng_status st;
    if ((st = check_grid(c, grid, &g))) return st;
    if (tstp < -1 || tstp > g.nt) return fail(c, NG_EINVAL, "tstp = %d out of range", tstp);
    if (Gloc.ldk != 1) return fail(c, NG_EINVAL, "Gloc.ldk must be 1");
    if ((st = check_herm(c, g, Gloc, "Gloc", tstp >= 0, &L, 1))) return st;
    if ((st = check_herm(c, g, Gk, "Gk", tstp >= 0, &K, g.nb))) return st;
    if (wk && ((uintptr_t)wk & 7u)) return fail(c, NG_EINVAL, "wk is not 8-byte aligned");
    return do_kreduce(c, g, tstp, L, K, (cudaStream_t)stream, wk);
}

ng_status ng_shard_plan(int nk, int rank, int nranks, const ng_grid* grid, int* k_begin, int* k_count,
                        size_t* send_bytes) {
    if (nk < 1 || nranks < 1 || nranks > NG_MAXRANKS || rank < 0 || rank >= nranks) return NG_EINVAL;
    if ((nk + NG_KBLK - 1) / NG_KBLK < nranks) return NG_EINVAL;
    BlkMap m;
    shard_map(nk, nranks, &m);
    const int b = m.first[rank] * NG_KBLK, e = std::min(nk, m.first[rank + 1] * NG_KBLK);
    if (k_begin) *k_begin = b;
    if (k_count) *k_count = e - b;
    if (send_bytes) {
        if (!grid) return NG_EINVAL;
        Grid g{};
        g.nt = grid->nt;
        g.ntau = grid->ntau;
        g.nf = grid->nf;
        *send_bytes = shard_send_bytes(g, shard_maxb(m, nranks));
    }
    return NG_OK;
}

ng_status ng_kreduce_partial(ng_ctx* c, const ng_grid* grid, int tstp, void* partial, ng_herm Gk, const double* wk,
                             int k_begin, void* stream) {
    Grid g;
    HermV K;
    ng_status st;
    if ((st = check_grid(c, grid, &g))) return st;
    if (tstp < -1 || tstp > g.nt) return fail(c, NG_EINVAL, "tstp = %d out of range", tstp);
    if ((st = check_herm(c, g, Gk, "Gk", tstp >= 0, &K, g.nb))) return st;
    if (k_begin < 0 || k_begin % NG_KBLK) return fail(c, NG_EINVAL, "k_begin = %d must be a multiple of %d", k_begin, NG_KBLK);
    if (!partial || !aligned16(partial)) return fail(c, NG_EINVAL, "partial is NULL or not 16-byte aligned");
    if (wk && ((uintptr_t)wk & 7u)) return fail(c, NG_EINVAL, "wk is not 8-byte aligned");
    const int cnt = tstp < 0 ? g.ntau + 1 : 2 * (tstp + 1) + g.ntau + 1;
    const int64_t warps = (int64_t)((g.nb + NG_KBLK - 1) / NG_KBLK) * cnt * g.nf * g.nf;
    k_kreduce_partial<<<nblocks(warps * 32, 256), 256, 0, (cudaStream_t)stream>>>(g, tstp, K, wk, k_begin,
                                                                                  (cplx*)partial);
    return check_launch(c, "k_kreduce_partial");
}

ng_status ng_kreduce_combine(ng_ctx* c, const ng_grid* grid, int tstp, ng_herm Gloc, const void* gathered, int nk,
                             int nranks, int weighted, void* stream) {
    Grid g;
    HermV L;
    ng_status st;
    if ((st = check_grid(c, grid, &g))) return st;
    if (tstp < -1 || tstp > g.nt) return fail(c, NG_EINVAL, "tstp = %d out of range", tstp);
    if (Gloc.ldk != 1) return fail(c, NG_EINVAL, "Gloc.ldk must be 1");
    if ((st = check_herm(c, g, Gloc, "Gloc", tstp >= 0, &L, 0))) return st;
    if (nk < 1 || nranks < 1 || nranks > NG_MAXRANKS || (nk + NG_KBLK - 1) / NG_KBLK < nranks)
        return fail(c, NG_EINVAL, "nk = %d, nranks = %d invalid", nk, nranks);
    if (!gathered || !aligned16(gathered)) return fail(c, NG_EINVAL, "gathered is NULL or not 16-byte aligned");
    BlkMap m;
    shard_map(nk, nranks, &m);
    const int cnt = tstp < 0 ? g.ntau + 1 : 2 * (tstp + 1) + g.ntau + 1;
    k_kreduce_combine<<<nblocks((int64_t)cnt * g.nf * g.nf, 128), 128, 0, (cudaStream_t)stream>>>(
        g, tstp, L, (const cplx*)gathered, nk, nranks, shard_maxb(m, nranks), m, weighted ? 1 : 0);
    return check_launch(c, "k_kreduce_combine");
}

ng_status ng_sigma2b_timestep(ng_ctx* c, const ng_grid* grid, int tstp, ng_herm S, ng_herm Gloc, ng_func U, void* stream) {
    Grid g;
    HermV Sv, L;
    FuncV uv;
    ng_status st;
    if ((st = check_grid(c, grid, &g))) return st;
    if (tstp < -1 || tstp > g.nt) return fail(c, NG_EINVAL, "tstp = %d out of range", tstp);
    if (S.ldk != 1 || Gloc.ldk != 1) return fail(c, NG_EINVAL, "Sigma and Gloc must have ldk = 1");
    if ((st = check_herm(c, g, S, "Sigma", tstp >= 0, &Sv, 1))) return st;
    if ((st = check_herm(c, g, Gloc, "Gloc", tstp >= 0, &L, 1))) return st;
    if ((st = check_func(c, g, U, "U", &uv))) return st;
    if (U.ldk != 1) return fail(c, NG_EINVAL, "U.ldk must be 1");
    return do_sigma(c, g, tstp, Sv, L, uv, (cudaStream_t)stream);
}

ng_status ng_hartree_timestep(ng_ctx* c, const ng_grid* grid, int tstp, ng_func epsmf, ng_func eps0, ng_herm Gloc,
                              ng_func U, double nbar, void* stream) {
    Grid g;
    HermV L;
    FuncV mf, e0, uv;
    ng_status st;
    if ((st = check_grid(c, grid, &g))) return st;
    if (tstp < -1 || tstp > g.nt) return fail(c, NG_EINVAL, "tstp = %d out of range", tstp);
    if ((st = check_func(c, g, epsmf, "eps_mf", &mf))) return st;
    if ((st = check_func(c, g, eps0, "eps0", &e0))) return st;
    if ((st = check_func(c, g, U, "U", &uv))) return st;
    if ((st = check_herm(c, g, Gloc, "Gloc", tstp >= 0, &L, 1))) return st;
    return do_hartree(c, g, tstp, mf, e0, L, uv, nbar, (cudaStream_t)stream);
}

ng_status ng_extrapolate_timestep(ng_ctx* c, const ng_grid* grid, int tstp, ng_herm G, void* stream) {
    Grid g;
    HermV Gv;
    ng_status st;
    if ((st = check_grid(c, grid, &g))) return st;
    if (tstp < g.k || tstp + 1 > g.nt) return fail(c, NG_EINVAL, "tstp = %d must be in k..nt-1", tstp);
    if ((st = check_herm(c, g, G, "G", true, &Gv, 0))) return st;
    return do_extrap(c, g, tstp, Gv, (cudaStream_t)stream);
}

ng_status ng_distance_timestep(ng_ctx* c, const ng_grid* grid, int tstp, ng_herm A, ng_herm B, double* out_dev,
                               void* stream) {
    Grid g;
    HermV Av, Bv;
    ng_status st;
    if ((st = check_grid(c, grid, &g))) return st;
    if (tstp < -1 || tstp > g.nt) return fail(c, NG_EINVAL, "tstp = %d out of range", tstp);
    if (A.ldk != B.ldk) return fail(c, NG_EINVAL, "A and B must have the same ldk");
    if ((st = check_herm(c, g, A, "A", tstp >= 0, &Av, 0))) return st;
    if ((st = check_herm(c, g, B, "B", tstp >= 0, &Bv, 0))) return st;
    if (!out_dev) return fail(c, NG_EINVAL, "out_dev is NULL");
    return do_distance(c, g, tstp, Av, Bv, out_dev, (cudaStream_t)stream);
}

ng_status ng_solve_fixed(ng_ctx* c, const ng_grid* grid, ng_herm G, ng_herm S, ng_func eps, int n_to, void* stream) {
    Grid g;
    HermV Gv, Sv;
    FuncV ev;
    ng_status st;
    if ((st = check_grid(c, grid, &g))) return st;
    if (n_to < g.k || n_to > g.nt) return fail(c, NG_EINVAL, "n_to = %d must be in k..nt", n_to);
    if ((st = check_herm(c, g, G, "G", true, &Gv, g.nb))) return st;
    if ((st = check_herm(c, g, S, "Sigma", true, &Sv, 0))) return st;
    if ((st = check_func(c, g, eps, "eps", &ev))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = do_mat(c, g, Gv, Sv, ev, s))) return st;
    if ((st = do_start(c, g, Gv, Sv, ev, s))) return st;
    for (int n = g.k + 1; n <= n_to; ++n)
        if ((st = do_timestep(c, g, n, Gv, Sv, ev, s))) return st;
    return NG_OK;
}

// host buffers of ng_run_2b_host (all NULL otherwise)
struct HostIO {
    const cplx* eps0;   // [nt+2][nf][nf][nbatch]
    const cplx* U;      // [nt+2]
    cplx* gdiag;        // [nt+1][nf][nf]: Gloc^<(t_n, t_n)
};

// GW state of the driver: the bosonic grid (sig = +1, one problem), P, K, K^ddagger (context
// workspace) and chi (the caller's), all with ldk = 1
struct GwRt {
    Grid gb;
    HermV P, K, Kcc, X;
    int L = 1;                   // 1: GW of the local Gloc; nk: k-space GW on the ring of nk momenta
    cplx* slice_buf = nullptr;   // L > 1: compact real-space slices of G, P, K, K^ddagger, chi, Sigma
    int64_t slice_stride = 0;    // complex values per slice buffer
};

// the self-consistent driver, second-Born (gw = NULL) or GW; sh = NULL: all k-points on this
// GPU, else this rank's share; io = NULL: inputs and outputs stay on the device
static ng_status run_2b_impl(ng_ctx* c, const ng_grid* grid, ng_herm G, ng_herm Gloc, ng_herm S, ng_func eps0,
                             ng_func epsmf, ng_func U, const ng_run_params* p, const ng_shard* sh, const HostIO* io,
                             int* iters_out, void* stream, const GwRt* gw = nullptr) {
    Grid g;
    HermV Gv, Lv, Sv;
    FuncV e0, mf, uv;
    ng_status st;
    if ((st = check_grid(c, grid, &g))) return st;
    if (!p) return fail(c, NG_EINVAL, "params is NULL");
    if ((st = check_herm(c, g, G, "G", true, &Gv, g.nb))) return st;
    // Sigma: shared (ldk = 1), or one per k-point for the k-space GW
    const int s_ldk = (gw && gw->L > 1) ? g.nb : 1;
    if (Gloc.ldk != 1 || S.ldk != s_ldk) return fail(c, NG_EINVAL, "Gloc must have ldk = 1 and Sigma ldk = %d", s_ldk);
    if ((st = check_herm(c, g, Gloc, "Gloc", true, &Lv, 1))) return st;
    if ((st = check_herm(c, g, S, "Sigma", true, &Sv, s_ldk))) return st;
    if ((st = check_func(c, g, eps0, "eps0", &e0))) return st;
    if ((st = check_func(c, g, epsmf, "eps_mf", &mf))) return st;
    if ((st = check_func(c, g, U, "U", &uv))) return st;
    if (U.ldk != 1) return fail(c, NG_EINVAL, "U.ldk must be 1");
    if (epsmf.ldk != G.ldk) return fail(c, NG_EINVAL, "eps_mf.ldk must equal G.ldk");
    if (p->corrector < 1) return fail(c, NG_EINVAL, "corrector must be >= 1");
    if (p->precision != NG_FP64 && p->precision != NG_F32C && p->precision != NG_DF64)
        return fail(c, NG_EINVAL, "unknown precision %d", p->precision);
    if (p->n_to > g.nt || (p->n_to >= p->n_from && p->n_from <= g.k))
        return fail(c, NG_EINVAL, "stepping range %d..%d invalid (k = %d, nt = %d)", p->n_from, p->n_to, g.k, g.nt);
    ShardRt rt;
    const ShardRt* rtp = nullptr;
    if (sh) {
        if ((st = check_shard(c, g, sh, &rt))) return st;
        rtp = &rt;
    }
    // problems summed by the convergence distances (all ranks')
    const double nk_all = sh ? (double)sh->nk : (double)G.ldk;
    cudaStream_t s = (cudaStream_t)stream;
    // distance accumulated in c->d_scalar, summed over the ranks in rank order
    auto read_distance = [&](double* err) -> ng_status {
        if (!rtp) {
            CUDA_TRY(c, cudaMemcpyAsync(err, c->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, s));
            CUDA_TRY(c, cudaStreamSynchronize(s));
            return NG_OK;
        }
        double per[NG_MAXRANKS];
        CUDA_TRY(c, cudaMemcpyAsync(sh->send, c->d_scalar, sizeof(double), cudaMemcpyDeviceToDevice, s));
        if (sh->exchange(sh->user, sizeof(double)) != 0) return fail(c, NG_ECOMM, "the exchange of distances failed");
        CUDA_TRY(c, cudaMemcpyAsync(per, sh->recv, sizeof(double) * sh->nranks, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(c, cudaStreamSynchronize(s));
        *err = 0.0;
        for (int r = 0; r < sh->nranks; ++r) *err += per[r];
        return NG_OK;
    };
    const int k = g.k, dd = g.nf * g.nf, T = g.ntau;
    // Sigma slices from..to from Gloc: from = to = -1 the Matsubara slice, 0..k the start-up
    // slices, n > k one time step.  GW: P, K and K^ddagger on those slices, then the chi
    // equation (vie2 Matsubara, start-up or time step), then dW and Sigma.
    int gw_mats_calls = 0;   // Matsubara chi solves of this run (refinement after the first two)
    auto sigma_slices = [&](int from, int to) -> ng_status {
        ng_status r;
        if (!gw) {
            for (int n = from; n <= to; ++n)
                if ((r = do_sigma(c, g, n, Sv, Lv, uv, s))) return r;
            return NG_OK;
        }
        // one event pair around the whole GW evaluation (bubbles, transforms, chi solve)
        const long pe = prof_pair(c, 3);
        if (pe >= 0) CUDA_TRY(c, cudaEventRecord(c->ev_pool[pe], s));
        const int L = gw->L;
        // k-space: G(r) = (1/L) sum_k e^{ikr} G_k, the bubbles in real space (conjugation
        // r -> -r), X_k = sum_r e^{-ikr} X(r) back (Eqs. Pol, Sigmak)
        cplx* B = gw->slice_buf;
        const int64_t bs = gw->slice_stride;
        const SliceView vG = compact(B), vP = compact(B + bs), vK = compact(B + 2 * bs), vKcc = compact(B + 3 * bs),
                        vX = compact(B + 4 * bs), vS = compact(B + 5 * bs);
        for (int n = from; n <= to; ++n) {
            if (L == 1) {
                if ((r = do_gw_pol(c, g, n, 1, whole(gw->P), whole(gw->K), whole(gw->Kcc), whole(Lv), uv, s))) return r;
                continue;
            }
            if ((r = do_kfft(c, g, n, L, whole(Gv), vG, +1, 1.0 / L, s))) return r;
            if ((r = do_gw_pol(c, g, n, L, vP, vK, vKcc, vG, uv, s))) return r;
            if ((r = do_kfft(c, g, n, L, vP, whole(gw->P), -1, 1.0, s))) return r;
            if ((r = do_kfft(c, g, n, L, vK, whole(gw->K), -1, 1.0, s))) return r;
            if ((r = do_kfft(c, g, n, L, vKcc, whole(gw->Kcc), -1, 1.0, s))) return r;
        }
        cudaError_t e = cudaSuccess;
        if (from < 0) {
            // after two fresh solves, refine chi^M with the kept LU factors; refactor if that stalls
            bool refined = false;
            const double nel = (double)(T + 1) * dd * gw->gb.nb;
            if (gw_mats_calls >= 2 &&
                (r = vie2_mat_d(c, gw->gb, gw->X, gw->K, gw->P, s, &c->ws_gwmat, &c->ws_gwmat_bytes, 30, 1e-13 * nel,
                                &refined)))
                return r;
            if (!refined && (r = vie2_mat_d(c, gw->gb, gw->X, gw->K, gw->P, s, &c->ws_gwmat, &c->ws_gwmat_bytes)))
                return r;
            ++gw_mats_calls;
        } else if (from == 0) {
            e = vie2_start_launch(gw->gb, gw->X, gw->K, gw->Kcc, gw->P, (cplx*)c->ws_st, c->d_status, s);
        } else {
            for (int n = from; n <= to && e == cudaSuccess; ++n) {
                const cplx* tvq = nullptr;
                const bool w = vie2_warp(c, gw->gb, n);
                if (!w && (r = prep_tvfft(c, gw->gb, n, gw->X, gw->K, s, &tvq, false))) return r;
                e = vie2_step_launch(gw->gb, n, gw->X, gw->K, gw->Kcc, gw->P, tvq, w, c->d_status, s);
            }
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, NG_ECUDA, "launch of the chi solve failed: %s", cudaGetErrorString(e));
        }
        for (int n = from; n <= to; ++n) {
            if (L == 1) {
                if ((r = do_gw_sigma(c, g, n, 1, whole(Sv), whole(Lv), whole(gw->X), uv, s))) return r;
                continue;
            }
            if ((r = do_kfft(c, g, n, L, whole(Gv), vG, +1, 1.0 / L, s))) return r;
            if ((r = do_kfft(c, g, n, L, whole(gw->X), vX, +1, 1.0 / L, s))) return r;
            if ((r = do_gw_sigma(c, g, n, L, vS, vG, vX, uv, s))) return r;
            if ((r = do_kfft(c, g, n, L, vS, whole(Sv), -1, 1.0, s))) return r;
        }
        if (pe >= 0) CUDA_TRY(c, cudaEventRecord(c->ev_pool[pe + 1], s));
        return NG_OK;
    };
    // host I/O: eps0 slices (index n+1) and the whole U in, Gloc^<(t_n, t_n) out
    const size_t eps_slice = sizeof(cplx) * dd * (size_t)eps0.ldk;
    auto eps_in = [&](int from, int to) -> ng_status {   // slices from..to (index from+1..to+1)
        if (!io || to < from) return NG_OK;
        CUDA_TRY(c, cudaMemcpyAsync((char*)eps0.val + (size_t)(from + 1) * eps_slice,
                                    (const char*)io->eps0 + (size_t)(from + 1) * eps_slice,
                                    (size_t)(to - from + 1) * eps_slice, cudaMemcpyHostToDevice, s));
        return NG_OK;
    };
    auto gdiag_out = [&](int from, int to) -> ng_status {
        if (!io) return NG_OK;
        for (int n = from; n <= to; ++n)
            CUDA_TRY(c, cudaMemcpyAsync(io->gdiag + (size_t)n * dd, Lv.les.p + (size_t)(tri(n) + n) * dd,
                                        sizeof(cplx) * dd, cudaMemcpyDeviceToHost, s));
        return NG_OK;
    };
    if (io) CUDA_TRY(c, cudaMemcpyAsync(U.val, io->U, sizeof(cplx) * (size_t)(g.nt + 2), cudaMemcpyHostToDevice, s));
    int mats_it = 0, boot_it = 0;
    bool noconv = false;
    if (p->do_setup) {
        // previous-iterate buffer shaped like slices 0..k of G plus mat
        const size_t el_mat = (size_t)(T + 1), el_tri = (size_t)tri(k + 1), el_tv = (size_t)(k + 1) * (T + 1);
        const size_t per = sizeof(cplx) * dd * (size_t)G.ldk;
        if ((st = ensure(c, &c->ws_prev, &c->ws_prev_bytes, per * (el_mat + 2 * el_tri + el_tv)))) return st;
        cplx* pb = (cplx*)c->ws_prev;
        HermV Pv;
        Pv.mat = Comp{pb, G.ldk, dd};
        Pv.ret = Comp{pb + el_mat * dd * G.ldk, G.ldk, dd};
        Pv.les = Comp{Pv.ret.p + el_tri * dd * G.ldk, G.ldk, dd};
        // tv rows 0..k are contiguous in G.tv, so the previous copy keeps the same row stride
        Pv.tv = Comp{Pv.les.p + el_tri * dd * G.ldk, G.ldk, dd};
        const size_t fslice = sizeof(cplx) * dd * (size_t)epsmf.ldk;
        // ---- Matsubara loop ----
        if ((st = eps_in(-1, k))) return st;
        CUDA_TRY(c, cudaMemcpyAsync(epsmf.val, eps0.val, fslice, cudaMemcpyDeviceToDevice, s));
        CUDA_TRY(c, cudaMemsetAsync(S.mat, 0, sizeof(cplx) * dd * el_mat * (size_t)S.ldk, s));
        if ((st = do_mat(c, g, Gv, Sv, mf, s))) return st;
        double err = 0.0;
        // stopping floors: a summed distance cannot fall below round-off, about 1e-15 per element
        const double nel_mat = nk_all * el_mat * dd;
        const double mats_stop = std::max(p->mats_tol, 1e-15 * nel_mat);
        for (mats_it = 0; mats_it < p->mats_maxiter; ++mats_it) {
            if ((st = do_kreduce_rt(c, g, -1, Lv, Gv, s, rtp))) return st;
            if ((st = do_hartree(c, g, -1, mf, e0, Lv, uv, p->nbar, s))) return st;
            if ((st = sigma_slices(-1, -1))) return st;
            CUDA_TRY(c, cudaMemcpyAsync(Pv.mat.p, Gv.mat.p, per * el_mat, cudaMemcpyDeviceToDevice, s));
            // after two fresh solves the operator changes little between iterations: refine the
            // current iterate with the kept LU factors, refactor only if that stalls
            bool refined = false;
            if (mats_it >= 2 && (st = do_mat_refine(c, g, Gv, Sv, mf, s, 30, 1e-13 * nel_mat, &refined))) return st;
            if (!refined && (st = do_mat(c, g, Gv, Sv, mf, s))) return st;
            CUDA_TRY(c, cudaMemsetAsync(c->d_scalar, 0, sizeof(double), s));
            if ((st = do_distance(c, g, -1, Gv, Pv, c->d_scalar, s))) return st;
            if ((st = read_distance(&err))) return st;
            if (err < mats_stop) break;
        }
        if (mats_it == p->mats_maxiter) noconv = true;
        ++mats_it;
        if ((st = do_kreduce_rt(c, g, -1, Lv, Gv, s, rtp))) return st;
        if ((st = do_hartree(c, g, -1, mf, e0, Lv, uv, p->nbar, s))) return st;
        if ((st = sigma_slices(-1, -1))) return st;
        // ---- bootstrapping ----
        for (int n = 0; n <= k; ++n) {
            k_mf_init<<<nblocks((int64_t)dd * epsmf.ldk, 128), 128, 0, s>>>(g, n, mf, e0);
            if ((st = check_launch(c, "k_mf_init"))) return st;
        }
        if ((st = do_start(c, g, Gv, Sv, mf, s))) return st;
        for (boot_it = 0; boot_it < p->boot_maxiter; ++boot_it) {
            for (int n = 0; n <= k; ++n) {
                if ((st = do_kreduce_rt(c, g, n, Lv, Gv, s, rtp))) return st;
                if ((st = do_hartree(c, g, n, mf, e0, Lv, uv, p->nbar, s))) return st;
            }
            if ((st = sigma_slices(0, k))) return st;
            CUDA_TRY(c, cudaMemcpyAsync(Pv.ret.p, Gv.ret.p, per * el_tri, cudaMemcpyDeviceToDevice, s));
            CUDA_TRY(c, cudaMemcpyAsync(Pv.les.p, Gv.les.p, per * el_tri, cudaMemcpyDeviceToDevice, s));
            CUDA_TRY(c, cudaMemcpyAsync(Pv.tv.p, Gv.tv.p, per * el_tv, cudaMemcpyDeviceToDevice, s));
            if ((st = do_start(c, g, Gv, Sv, mf, s))) return st;
            CUDA_TRY(c, cudaMemsetAsync(c->d_scalar, 0, sizeof(double), s));
            for (int n = 0; n <= k; ++n)
                if ((st = do_distance(c, g, n, Gv, Pv, c->d_scalar, s))) return st;
            if ((st = read_distance(&err))) return st;
            if (err < std::max(p->boot_tol, 1e-15 * nk_all * dd * (2.0 * el_tri + el_tv)) && boot_it > 2) break;
        }
        if (boot_it == p->boot_maxiter) noconv = true;
        ++boot_it;
        if ((st = gdiag_out(0, k))) return st;
    }
    // ---- time stepping: predictor, then fixed corrector iterations ----
    for (int n = p->n_from; n <= p->n_to; ++n) {
        if ((st = eps_in(n, n))) return st;
        if ((st = do_extrap(c, g, n - 1, Gv, s))) return st;
        for (int it = 0; it < p->corrector; ++it) {
            if ((st = do_kreduce_rt(c, g, n, Lv, Gv, s, rtp))) return st;
            if ((st = do_hartree(c, g, n, mf, e0, Lv, uv, p->nbar, s))) return st;
            if ((st = sigma_slices(n, n))) return st;
            if ((st = do_timestep(c, g, n, Gv, Sv, mf, s, p->precision))) return st;
        }
        if ((st = gdiag_out(n, n))) return st;
    }
    if (iters_out) {
        iters_out[0] = mats_it;
        iters_out[1] = boot_it;
    }
    if (noconv) return fail(c, NG_ENOCONV, "setup loop reached its iteration limit (mats %d, boot %d)", mats_it, boot_it);
    return NG_OK;
}

ng_status ng_run_2b(ng_ctx* c, const ng_grid* grid, ng_herm G, ng_herm Gloc, ng_herm S, ng_func eps0, ng_func epsmf,
                    ng_func U, const ng_run_params* p, int* iters_out, void* stream) {
    return run_2b_impl(c, grid, G, Gloc, S, eps0, epsmf, U, p, nullptr, nullptr, iters_out, stream);
}

ng_status ng_run_2b_host(ng_ctx* c, const ng_grid* grid, ng_herm G, ng_herm Gloc, ng_herm S, ng_func eps0,
                         ng_func epsmf, ng_func U, const double* eps0_host, const double* U_host, double* gdiag_host,
                         const ng_run_params* p, const ng_shard* shard, int* iters_out, void* stream) {
    if (!c) return NG_EINVAL;
    if (!eps0_host || !U_host || !gdiag_host) return fail(c, NG_EINVAL, "a host buffer is NULL");
    if (eps0.ldk != (grid ? grid->nbatch : 0)) return fail(c, NG_EINVAL, "eps0.ldk must be nbatch");
    const HostIO io{(const cplx*)eps0_host, (const cplx*)U_host, (cplx*)gdiag_host};
    return run_2b_impl(c, grid, G, Gloc, S, eps0, epsmf, U, p, shard, &io, iters_out, stream);
}

ng_status ng_run_2b_sharded(ng_ctx* c, const ng_grid* grid, ng_herm G, ng_herm Gloc, ng_herm S, ng_func eps0,
                            ng_func epsmf, ng_func U, const ng_run_params* p, const ng_shard* shard, int* iters_out,
                            void* stream) {
    if (!c) return NG_EINVAL;
    if (!shard) return fail(c, NG_EINVAL, "shard is NULL");
    return run_2b_impl(c, grid, G, Gloc, S, eps0, epsmf, U, p, shard, nullptr, iters_out, stream);
}

// the six compact real-space slice buffers of the k-space chain (G, P, K, K^ddagger, chi, Sigma)
static ng_status gwk_slice_buffers(ng_ctx* c, const Grid& g, GwRt* gw) {
    const int L = g.nb, dd = g.nf * g.nf;
    const int64_t slice = (2 * (int64_t)(g.nt + 1) + g.ntau + 1) * dd * L;
    ng_status st;
    if ((st = ensure(c, &c->ws_gwk, &c->ws_gwk_bytes, sizeof(cplx) * 6 * (size_t)slice))) return st;
    gw->L = L;
    gw->slice_buf = (cplx*)c->ws_gwk;
    gw->slice_stride = slice;
    return NG_OK;
}

// GW state for ng_run_gw (kspace = false: one local problem) and ng_run_gw_kspace (the ring of
// nbatch momenta): bosonic grid, P, K, K^ddagger in the context, chi from the caller and, for
// the ring, the compact real-space slice buffers
static ng_status gw_prepare(ng_ctx* c, const Grid& g, ng_herm Chi, bool kspace, GwRt* gw) {
    ng_status st;
    if (g.nf > 4) return fail(c, NG_EUNSUPPORTED, "the GW driver supports nf = 1, 2, 4");
    if (kspace && g.nf != 1) return fail(c, NG_EUNSUPPORTED, "the k-space GW is one-band (nf = 1)");
    if (kspace && g.nb > 4096) return fail(c, NG_EUNSUPPORTED, "the k-space GW supports at most 4096 momenta");
    const int L = kspace ? g.nb : 1;
    if (Chi.ldk != L) return fail(c, NG_EINVAL, "Chi must have ldk = %d", L);
    gw->gb = g;
    gw->gb.sig = 1;
    gw->gb.nb = L;
    gw->L = L;
    if ((st = check_herm(c, gw->gb, Chi, "Chi", true, &gw->X, L))) return st;
    // P, K, K^ddagger: whole-contour bosonic functions in the packed layout, ldk = L
    const int dd = g.nf * g.nf;
    const int64_t n_mat = g.ntau + 1, n_tri = tri(g.nt + 1), n_tv = (int64_t)(g.nt + 1) * (g.ntau + 1);
    const int64_t per = (n_mat + 2 * n_tri + n_tv) * dd * L;
    if ((st = ensure(c, &c->ws_gw, &c->ws_gw_bytes, sizeof(cplx) * 3 * (size_t)per))) return st;
    auto view = [&](cplx* b) {
        HermV v;
        v.mat = Comp{b, L, dd};
        v.ret = Comp{b + n_mat * dd * L, L, dd};
        v.les = Comp{v.ret.p + n_tri * dd * L, L, dd};
        v.tv = Comp{v.les.p + n_tri * dd * L, L, dd};
        return v;
    };
    cplx* base = (cplx*)c->ws_gw;
    gw->P = view(base);
    gw->K = view(base + per);
    gw->Kcc = view(base + 2 * per);
    if (kspace && (st = gwk_slice_buffers(c, g, gw))) return st;
    return ensure(c, &c->ws_st, &c->ws_st_bytes, std::max(start_ws_bytes(g), start_ws_bytes(gw->gb)));
}

ng_status ng_run_gw(ng_ctx* c, const ng_grid* grid, ng_herm G, ng_herm Gloc, ng_herm S, ng_herm Chi, ng_func eps0,
                    ng_func epsmf, ng_func U, const ng_run_params* p, int* iters_out, void* stream) {
    Grid g;
    ng_status st;
    GwRt gw;
    if ((st = check_grid(c, grid, &g))) return st;
    if ((st = gw_prepare(c, g, Chi, false, &gw))) return st;
    return run_2b_impl(c, grid, G, Gloc, S, eps0, epsmf, U, p, nullptr, nullptr, iters_out, stream, &gw);
}

ng_status ng_run_gw_kspace(ng_ctx* c, const ng_grid* grid, ng_herm G, ng_herm Gloc, ng_herm Sigma, ng_herm Chi,
                           ng_func eps0, ng_func epsmf, ng_func U, const ng_run_params* p, int* iters_out,
                           void* stream) {
    Grid g;
    ng_status st;
    GwRt gw;
    if ((st = check_grid(c, grid, &g))) return st;
    if ((st = gw_prepare(c, g, Chi, true, &gw))) return st;
    if (p && p->precision != NG_FP64) return fail(c, NG_EUNSUPPORTED, "the k-space GW driver runs in NG_FP64");
    return run_2b_impl(c, grid, G, Gloc, Sigma, eps0, epsmf, U, p, nullptr, nullptr, iters_out, stream, &gw);
}

// one slice of the k-space chain (tests and callers composing their own loop)
static ng_status gwk_slice_args(ng_ctx* c, const ng_grid* grid, int tstp, ng_herm Gk, ng_func U, Grid* g, GwRt* gw,
                                HermV* Gv, FuncV* uv) {
    ng_status st;
    if ((st = check_grid(c, grid, g))) return st;
    if (tstp < -1 || tstp > g->nt) return fail(c, NG_EINVAL, "tstp = %d out of range", tstp);
    if (g->nf != 1) return fail(c, NG_EUNSUPPORTED, "the k-space GW is one-band (nf = 1)");
    if (g->nb > 4096) return fail(c, NG_EUNSUPPORTED, "the k-space GW supports at most 4096 momenta");
    gw->gb = *g;
    gw->gb.sig = 1;
    if ((st = gwk_slice_buffers(c, *g, gw))) return st;
    if ((st = check_herm(c, *g, Gk, "G", tstp >= 0, Gv, g->nb))) return st;
    if ((st = check_func(c, *g, U, "U", uv))) return st;
    if (U.ldk != 1) return fail(c, NG_EINVAL, "U.ldk must be 1");
    return NG_OK;
}

ng_status ng_gw_kspace_polarization_timestep(ng_ctx* c, const ng_grid* grid, int tstp, ng_herm P, ng_herm K,
                                             ng_herm Kcc, ng_herm Gk, ng_func U, void* stream) {
    Grid g;
    GwRt gw;
    HermV Gv, Pv, Kv, Kccv;
    FuncV uv;
    ng_status st;
    if ((st = gwk_slice_args(c, grid, tstp, Gk, U, &g, &gw, &Gv, &uv))) return st;
    if ((st = check_herm(c, gw.gb, P, "P", tstp >= 0, &Pv, g.nb))) return st;
    if ((st = check_herm(c, gw.gb, K, "K", tstp >= 0, &Kv, g.nb))) return st;
    if ((st = check_herm(c, gw.gb, Kcc, "Kcc", tstp >= 0, &Kccv, g.nb))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int L = g.nb;
    const int64_t bs = gw.slice_stride;
    cplx* B = gw.slice_buf;
    if ((st = do_kfft(c, g, tstp, L, whole(Gv), compact(B), +1, 1.0 / L, s))) return st;
    if ((st = do_gw_pol(c, g, tstp, L, compact(B + bs), compact(B + 2 * bs), compact(B + 3 * bs), compact(B), uv, s)))
        return st;
    if ((st = do_kfft(c, g, tstp, L, compact(B + bs), whole(Pv), -1, 1.0, s))) return st;
    if ((st = do_kfft(c, g, tstp, L, compact(B + 2 * bs), whole(Kv), -1, 1.0, s))) return st;
    return do_kfft(c, g, tstp, L, compact(B + 3 * bs), whole(Kccv), -1, 1.0, s);
}

ng_status ng_gw_kspace_sigma_timestep(ng_ctx* c, const ng_grid* grid, int tstp, ng_herm Sigma, ng_herm Gk,
                                      ng_herm Chi, ng_func U, void* stream) {
    Grid g;
    GwRt gw;
    HermV Gv, Sv;
    FuncV uv;
    ng_status st;
    HermV Xv;
    if ((st = gwk_slice_args(c, grid, tstp, Gk, U, &g, &gw, &Gv, &uv))) return st;
    if ((st = check_herm(c, g, Sigma, "Sigma", tstp >= 0, &Sv, g.nb))) return st;
    if ((st = check_herm(c, gw.gb, Chi, "Chi", tstp >= 0, &Xv, g.nb))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int L = g.nb;
    const int64_t bs = gw.slice_stride;
    cplx* B = gw.slice_buf;
    if ((st = do_kfft(c, g, tstp, L, whole(Gv), compact(B), +1, 1.0 / L, s))) return st;
    if ((st = do_kfft(c, g, tstp, L, whole(Xv), compact(B + 4 * bs), +1, 1.0 / L, s))) return st;
    if ((st = do_gw_sigma(c, g, tstp, L, compact(B + 5 * bs), compact(B), compact(B + 4 * bs), uv, s))) return st;
    return do_kfft(c, g, tstp, L, compact(B + 5 * bs), whole(Sv), -1, 1.0, s);
}

ng_status ng_gw_polarization_timestep(ng_ctx* c, const ng_grid* grid, int tstp, ng_herm P, ng_herm K, ng_herm Kcc,
                                      ng_herm Gloc, ng_func U, void* stream) {
    Grid g;
    HermV Pv, Kv, Kccv, L;
    FuncV uv;
    ng_status st;
    if ((st = check_grid(c, grid, &g))) return st;
    if (tstp < -1 || tstp > g.nt) return fail(c, NG_EINVAL, "tstp = %d out of range", tstp);
    if (P.ldk != 1 || K.ldk != 1 || Kcc.ldk != 1 || Gloc.ldk != 1)
        return fail(c, NG_EINVAL, "P, K, Kcc and Gloc must have ldk = 1");
    if ((st = check_herm(c, g, P, "P", tstp >= 0, &Pv, 1))) return st;
    if ((st = check_herm(c, g, K, "K", tstp >= 0, &Kv, 1))) return st;
    if ((st = check_herm(c, g, Kcc, "Kcc", tstp >= 0, &Kccv, 1))) return st;
    if ((st = check_herm(c, g, Gloc, "Gloc", tstp >= 0, &L, 1))) return st;
    if ((st = check_func(c, g, U, "U", &uv))) return st;
    if (U.ldk != 1) return fail(c, NG_EINVAL, "U.ldk must be 1");
    return do_gw_pol(c, g, tstp, 1, whole(Pv), whole(Kv), whole(Kccv), whole(L), uv, (cudaStream_t)stream);
}

ng_status ng_gw_sigma_timestep(ng_ctx* c, const ng_grid* grid, int tstp, ng_herm S, ng_herm Gloc, ng_herm Chi,
                               ng_func U, void* stream) {
    Grid g;
    HermV Sv, L, Xv;
    FuncV uv;
    ng_status st;
    if ((st = check_grid(c, grid, &g))) return st;
    if (tstp < -1 || tstp > g.nt) return fail(c, NG_EINVAL, "tstp = %d out of range", tstp);
    if (S.ldk != 1 || Gloc.ldk != 1 || Chi.ldk != 1) return fail(c, NG_EINVAL, "Sigma, Gloc and Chi must have ldk = 1");
    if ((st = check_herm(c, g, S, "Sigma", tstp >= 0, &Sv, 1))) return st;
    if ((st = check_herm(c, g, Gloc, "Gloc", tstp >= 0, &L, 1))) return st;
    if ((st = check_herm(c, g, Chi, "Chi", tstp >= 0, &Xv, 1))) return st;
    if ((st = check_func(c, g, U, "U", &uv))) return st;
    if (U.ldk != 1) return fail(c, NG_EINVAL, "U.ldk must be 1");
    return do_gw_sigma(c, g, tstp, 1, whole(Sv), whole(L), whole(Xv), uv, (cudaStream_t)stream);
}

}  // extern "C"

// =========================================================================================
// Allocation-free start-up (ng_dyson_start_noalloc): the start-up workspace is a file-scope
// static device array instead of context-owned memory; the kernels are those of
// ng_dyson_start.
// =========================================================================================
#define NG_NOALLOC_SCRATCH_BYTES (2u << 20)
#define NG_NOALLOC_STATUS_BYTES 256u
static __device__ __align__(256) unsigned char g_noalloc_scratch[NG_NOALLOC_SCRATCH_BYTES];

namespace {
// device address of g_noalloc_scratch per device, looked up once with that device current
void* g_noalloc_addr[64] = {nullptr};

template <int D>
ng_status noalloc_start(const Grid& g, const HermV& G, const HermV& S, const FuncV& eps, cplx* ws, int* status,
                        cudaStream_t s) {
    k_start_ret<D><<<nblocks(g.nb, 64), 64, 0, s>>>(g, G, S, eps, ws, status);
    if (cudaGetLastError() != cudaSuccess) return NG_ECUDA;
    k_start_tv<D><<<nblocks((int64_t)(g.ntau + 1) * g.nb, 128), 128, 0, s>>>(g, G, S, ws, status);
    if (cudaGetLastError() != cudaSuccess) return NG_ECUDA;
    k_start_les<D><<<nblocks((int64_t)(g.k + 1) * g.nb, 64), 64, 0, s>>>(g, G, S, ws, status);
    if (cudaGetLastError() != cudaSuccess) return NG_ECUDA;
    return NG_OK;
}
}  // namespace

extern "C" ng_status ng_dyson_start_noalloc(const ng_grid* grid, ng_herm G, ng_herm S, ng_func eps, void* stream) {
    // argument checks (no context, so status codes only)
    if (!grid) return NG_EINVAL;
    const ng_grid& q = *grid;
    if (q.korder < 1 || q.korder > NG_KMAX || q.sig != -1 || q.nbatch < 1 || !(q.h > 0.0) || !(q.beta > 0.0))
        return NG_EINVAL;
    if (q.nt < 2 * q.korder + 2 || q.ntau < 2 * q.korder + 2 || q.nf < 1) return NG_EINVAL;
    if (q.nf != 1 && q.nf != 2 && q.nf != 4 && q.nf != 8) return NG_EUNSUPPORTED;
    if (G.ldk != q.nbatch || (S.ldk != 1 && S.ldk != q.nbatch) || (eps.ldk != 1 && eps.ldk != q.nbatch))
        return NG_EINVAL;
    const void* ptrs[] = {G.mat, G.ret, G.les, G.tv, S.mat, S.ret, S.les, S.tv, eps.val};
    for (const void* p : ptrs)
        if (!p || !aligned16(p)) return NG_EINVAL;
    const size_t N = (size_t)q.korder * q.nf;
    const size_t need =
        NG_NOALLOC_STATUS_BYTES + sizeof(cplx) * (size_t)q.nbatch * (N * N + (size_t)q.korder * q.nf * q.nf);
    if (need > NG_NOALLOC_SCRATCH_BYTES) return NG_ESCRATCH;
    // one-time set-up per device, with that device current
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return NG_ECUDA; }
    if (dev < 0 || dev >= 64) return NG_EUNSUPPORTED;
    if (ng_status ws = load_weights_once(dev)) return ws;
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) { cudaGetLastError(); return NG_ECUDA; }
        g_noalloc_addr[dev] = p;
    }
    Grid g;
    g.nt = q.nt;
    g.ntau = q.ntau;
    g.nf = q.nf;
    g.nb = q.nbatch;
    g.k = q.korder;
    g.sig = q.sig;
    g.h = q.h;
    g.beta = q.beta;
    g.mu = q.mu;
    g.htau = q.beta / q.ntau;
    const int dd = q.nf * q.nf;
    HermV Gv{Comp{(cplx*)G.mat, G.ldk, dd}, Comp{(cplx*)G.ret, G.ldk, dd}, Comp{(cplx*)G.les, G.ldk, dd},
             Comp{(cplx*)G.tv, G.ldk, dd}};
    HermV Sv{Comp{(cplx*)S.mat, S.ldk, dd}, Comp{(cplx*)S.ret, S.ldk, dd}, Comp{(cplx*)S.les, S.ldk, dd},
             Comp{(cplx*)S.tv, S.ldk, dd}};
    FuncV ev{(cplx*)eps.val, eps.ldk};
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* base = (unsigned char*)g_noalloc_addr[dev];
    int* status = (int*)base;
    cplx* ws = (cplx*)(base + NG_NOALLOC_STATUS_BYTES);
    if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) { cudaGetLastError(); return NG_ECUDA; }
    switch (q.nf) {
        case 1: return noalloc_start<1>(g, Gv, Sv, ev, ws, status, s);
        case 2: return noalloc_start<2>(g, Gv, Sv, ev, ws, status, s);
        case 4: return noalloc_start<4>(g, Gv, Sv, ev, ws, status, s);
        default: return noalloc_start<8>(g, Gv, Sv, ev, ws, status, s);
    }
}

// =========================================================================================
// Uneven batch of independent problems (ng_batch_*) and the embedding sandwich
// =========================================================================================
struct ng_batch {
    int np = 0;
    int device = 0;
    std::vector<Grid> grids;
    std::vector<HermV> G, S;
    std::vector<FuncV> eps;
    std::vector<UHost> info;
    UProb* d_probs = nullptr;
    cplx* d_minv = nullptr;
    int threads = 0;      // block size of the bulk kernel chosen by the autotune (0: not tuned)
    double tune_ms[3] = {0, 0, 0};
    // concurrent per-problem setup: streams, join events and one workspace per stream
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    void* ws_setup = nullptr;
    size_t ws_setup_bytes = 0;
};
#define NG_SETUP_STREAMS 16

namespace {
__global__ void k_sandwich(Grid go, HermV O, Grid gi, HermV I, const cplx* V) {
    const int Do = go.nf, Di = gi.nf;
    const int64_t T1 = go.ntau + 1, ntri = tri(go.nt + 1), ntv = (int64_t)(go.nt + 1) * T1;
    const int64_t nel = T1 + 2 * ntri + ntv;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= nel * Do * Do) return;
    const int ab = (int)(item % (Do * Do));
    int64_t e = item / (Do * Do);
    const int a = ab / Do, b = ab % Do;
    const Comp* co;
    const Comp* ci;
    if (e < T1) { co = &O.mat; ci = &I.mat; }
    else if ((e -= T1) < ntri) { co = &O.ret; ci = &I.ret; }
    else if ((e -= ntri) < ntri) { co = &O.les; ci = &I.les; }
    else { e -= ntri; co = &O.tv; ci = &I.tv; }
    cplx s = cz();
    for (int c = 0; c < Di; ++c)
        for (int d = 0; d < Di; ++d)
            s = cfma(cmul(V[a * Di + c], ci->p[e * Di * Di + c * Di + d]), cconj(V[b * Di + d]), s);
    co->p[e * Do * Do + ab] = s;
}
}  // namespace

extern "C" {

ng_status ng_herm_sandwich(ng_ctx* c, const ng_grid* grid_out, ng_herm Out, const ng_grid* grid_in, ng_herm In,
                           const double* V_host, void* stream) {
    Grid go, gi;
    HermV Ov, Iv;
    ng_status st;
    if ((st = check_grid(c, grid_out, &go))) return st;
    if ((st = check_grid(c, grid_in, &gi))) return st;
    if (go.nb != 1 || gi.nb != 1) return fail(c, NG_EINVAL, "ng_herm_sandwich takes one problem (nbatch = 1)");
    if (go.nt != gi.nt || go.ntau != gi.ntau) return fail(c, NG_EINVAL, "grids differ in nt or ntau");
    if ((st = check_herm(c, go, Out, "Out", true, &Ov, 1))) return st;
    if ((st = check_herm(c, gi, In, "In", true, &Iv, 1))) return st;
    if (!V_host) return fail(c, NG_EINVAL, "V is NULL");
    const size_t bytes = sizeof(cplx) * go.nf * gi.nf;
    if ((st = ensure(c, (void**)&c->d_eps, &c->d_eps_bytes, bytes))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(c, cudaMemcpyAsync(c->d_eps, V_host, bytes, cudaMemcpyHostToDevice, s));
    const int64_t nel = (go.ntau + 1) + 2 * tri(go.nt + 1) + (int64_t)(go.nt + 1) * (go.ntau + 1);
    k_sandwich<<<nblocks(nel * go.nf * go.nf, 256), 256, 0, s>>>(go, Ov, gi, Iv, c->d_eps);
    return check_launch(c, "k_sandwich");
}

ng_status ng_batch_create(ng_ctx* c, int nprob, const ng_grid* grids, const ng_herm* G, const ng_herm* S,
                          const ng_func* eps, ng_batch** out) {
    if (!c || !out) return NG_EINVAL;
    *out = nullptr;
    if (nprob < 1 || !grids || !G || !S || !eps) return fail(c, NG_EINVAL, "empty or NULL problem arrays");
    ng_batch* b = new ng_batch();
    b->np = nprob;
    b->device = c->device;
    std::vector<UProb> h(nprob);
    for (int p = 0; p < nprob; ++p) {
        Grid g;
        HermV Gv, Sv;
        FuncV ev;
        ng_status st;
        if ((st = check_grid(c, &grids[p], &g)) || (g.nb != 1 && (st = fail(c, NG_EINVAL, "problem %d: nbatch must be 1", p))) ||
            (st = check_herm(c, g, G[p], "G", true, &Gv, 1)) || (st = check_herm(c, g, S[p], "Sigma", true, &Sv, 1)) ||
            (st = check_func(c, g, eps[p], "eps", &ev))) {
            delete b;
            return st;
        }
        b->grids.push_back(g);
        b->G.push_back(Gv);
        b->S.push_back(Sv);
        b->eps.push_back(ev);
        b->info.push_back(UHost{g.nf, g.nt, g.ntau, g.k});
        h[p].g = g;
        h[p].G = Gv;
        h[p].S = Sv;
        h[p].eps = ev;
        h[p].kb = 0;
    }
    if (cudaMalloc(&b->d_probs, sizeof(UProb) * nprob) != cudaSuccess ||
        cudaMalloc(&b->d_minv, sizeof(cplx) * 64 * nprob) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(b->d_probs);
        delete b;
        return fail(c, NG_ENOMEM, "batch tables");
    }
    for (int p = 0; p < nprob; ++p) h[p].minv = b->d_minv + 64 * (size_t)p;
    if (cudaMemcpy(b->d_probs, h.data(), sizeof(UProb) * nprob, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(b->d_probs);
        cudaFree(b->d_minv);
        delete b;
        return fail(c, NG_ECUDA, "upload of the batch table");
    }
    *out = b;
    return NG_OK;
}

void ng_batch_destroy(ng_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    cudaFree(b->d_probs);
    cudaFree(b->d_minv);
    cudaFree(b->ws_setup);
    for (cudaStream_t x : b->streams) cudaStreamDestroy(x);
    for (cudaEvent_t e : b->events) cudaEventDestroy(e);
    delete b;
}

ng_status ng_batch_setup(ng_ctx* c, ng_batch* b, void* stream) {
    if (!c || !b) return NG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    ng_status st;
    // The per-problem setups are independent and each Matsubara LU runs in one block, so they
    // run concurrently on up to NG_SETUP_STREAMS streams with a workspace each, the costliest
    // (nf^3 (ntau+1)^3) first, and are joined back into the caller's stream.
    const int ns = std::min(b->np, NG_SETUP_STREAMS);
    std::vector<int> order(b->np);
    for (int p = 0; p < b->np; ++p) order[p] = p;
    auto cost = [&](int p) {
        const double d = b->grids[p].nf, t = b->grids[p].ntau + 1;
        return d * d * d * t * t * t;
    };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost(x) > cost(y); });
    size_t wmat = 0, wst = 0;
    for (int p = 0; p < b->np; ++p) {
        wmat = std::max(wmat, (mat_ws_bytes(b->grids[p]) + 255) / 256 * 256);
        wst = std::max(wst, (start_ws_bytes(b->grids[p]) + 255) / 256 * 256);
    }
    if ((st = ensure(c, &b->ws_setup, &b->ws_setup_bytes, (size_t)ns * (wmat + wst)))) return st;
    for (int i = (int)b->streams.size(); i < ns; ++i) {
        cudaStream_t x;
        cudaEvent_t e;
        CUDA_TRY(c, cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
        CUDA_TRY(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        b->streams.push_back(x);
        b->events.push_back(e);
    }
    CUDA_TRY(c, cudaEventRecord(b->events[0], s));
    for (int i = 0; i < ns; ++i) CUDA_TRY(c, cudaStreamWaitEvent(b->streams[i], b->events[0], 0));
    for (int q = 0; q < b->np; ++q) {
        const int p = order[q], i = q % ns;
        char* ws = (char*)b->ws_setup + (size_t)i * (wmat + wst);
        if ((st = do_mat(c, b->grids[p], b->G[p], b->S[p], b->eps[p], b->streams[i], ws))) return st;
        if ((st = do_start(c, b->grids[p], b->G[p], b->S[p], b->eps[p], b->streams[i], ws + wmat))) return st;
    }
    for (int i = 0; i < ns; ++i) {
        CUDA_TRY(c, cudaEventRecord(b->events[i], b->streams[i]));
        CUDA_TRY(c, cudaStreamWaitEvent(s, b->events[i], 0));
    }
    return NG_OK;
}

ng_status ng_batch_step(ng_ctx* c, ng_batch* b, int n, int threads, void* stream) {
    if (!c || !b) return NG_EINVAL;
    if (threads == 0) threads = b->threads ? b->threads : 128;
    if (threads != 64 && threads != 128 && threads != 256) return fail(c, NG_EINVAL, "threads must be 64, 128 or 256");
    std::vector<int> active;
    for (int p = 0; p < b->np; ++p)
        if (n > b->info[p].k && n <= b->info[p].nt) active.push_back(p);
    if (active.empty()) return NG_OK;
    return ustep(c, b->d_probs, b->info, active, n, threads, (cudaStream_t)stream);
}

ng_status ng_batch_solve(ng_ctx* c, ng_batch* b, int* tuned_threads, void* stream) {
    if (!c || !b) return NG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    ng_status st;
    if ((st = ng_batch_setup(c, b, stream))) return st;
    int kmin = 1 << 30, ntmax = 0, ntmin = 1 << 30;
    for (const UHost& u : b->info) {
        kmin = std::min(kmin, u.k);
        ntmax = std::max(ntmax, u.nt);
        ntmin = std::min(ntmin, u.nt);
    }
    // autotune the bulk block size once per batch shape and context, on a representative step
    // (re-running a step is idempotent: slice n is recomputed from slices < n)
    std::vector<int> key(6, 0);
    for (const UHost& u : b->info) {
        key[u.D == 1 ? 0 : u.D == 2 ? 1 : u.D == 4 ? 2 : 3] += 1;
        key[4] = std::max(key[4], u.ntau);
        key[5] = std::max(key[5], (u.nt + 255) / 256);
    }
    if (b->threads == 0)
        for (const auto& e : c->tune_cache)
            if (e.first == key) b->threads = e.second;
    const bool tune = b->threads == 0;
    const int n_tune = std::max(2 * kmin + 2, ntmin / 2);
    for (int n = kmin + 1; n <= ntmax; ++n) {
        if (n == n_tune && b->threads == 0) {
            const int cand[3] = {64, 128, 256};
            cudaEvent_t e0, e1;
            CUDA_TRY(c, cudaEventCreate(&e0));
            CUDA_TRY(c, cudaEventCreate(&e1));
            float best = 1e30f;
            for (int i = 0; i < 3; ++i) {
                float t_best = 1e30f;
                for (int rep = 0; rep < 2; ++rep) {
                    CUDA_TRY(c, cudaEventRecord(e0, s));
                    if ((st = ng_batch_step(c, b, n, cand[i], stream))) return st;
                    CUDA_TRY(c, cudaEventRecord(e1, s));
                    CUDA_TRY(c, cudaEventSynchronize(e1));
                    float ms = 0.f;
                    CUDA_TRY(c, cudaEventElapsedTime(&ms, e0, e1));
                    t_best = std::min(t_best, ms);
                }
                b->tune_ms[i] = t_best;
                if (t_best < best) { best = t_best; b->threads = cand[i]; }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
        }
        if ((st = ng_batch_step(c, b, n, 0, stream))) return st;
    }
    if (tune && b->threads) c->tune_cache.push_back({key, b->threads});
    if (tuned_threads) *tuned_threads = b->threads;
    return NG_OK;
}

}  // extern "C"

// =========================================================================================
// Discrete adjoint of the second-Born time stepping (ng_adjoint_2b), nf = 1.
// The final forward history is kept in full (every slice depends on all earlier ones); the
// corrector iterates of slice n are recomputed from it segment by segment: the steps of a
// segment are re-run forward with their iterates captured, then walked backwards.
// =========================================================================================
namespace {

struct AdjLayout {
    int64_t L;           // longest slice: 2 (nt+1) + ntau + 1
    int64_t itstride;    // one captured pass: per-k slice, G_loc slice, Sigma slice, eps_mf(n)
    int seg, corr;
    cplx *store, *cw, *cSw, *cmfw, *cA, *caccR, *caccT, *crhs, *cMn, *retA, *part, *cLoc, *cmf;
    double* ce0;
    // start slices
    int64_t E;
    cplx *mu, *ctot, *ctot0, *Pk, *cSx, *cLb, *cmfx;
    double* dist;
};

size_t adj_layout(const Grid& g, int seg, int corr, AdjLayout* A, char* base) {
    const int64_t nb = g.nb, T = g.ntau, K1 = g.k + 1;
    A->L = 2 * (int64_t)(g.nt + 1) + T + 1;
    A->itstride = A->L * nb + 2 * A->L + nb;
    A->seg = seg;
    A->corr = corr;
    A->E = boot_E(g.k, g.ntau);
    size_t off = 0;
    auto take = [&](int64_t count) {   // count complex numbers, 256-byte aligned
        char* p = base ? base + off : nullptr;
        off += (((size_t)count * sizeof(cplx)) + 255) / 256 * 256;
        return (cplx*)p;
    };
    A->store = take((int64_t)seg * corr * A->itstride);
    A->cw = take(A->L * nb);
    A->cSw = take(A->L);
    A->cmfw = take(nb);
    A->cA = take((int64_t)NG_MAXQ * nb);
    A->caccR = take((int64_t)(g.nt + 1) * nb);
    A->caccT = take((T + 1) * nb);
    A->crhs = take((int64_t)(g.nt + 1) * nb);
    A->cMn = take(nb);
    A->retA = take(K1 * K1 * nb);
    A->part = take((int64_t)NG_ADJ_NPART * NG_ADJ_SPLIT * A->L);
    A->cLoc = take(A->L);
    A->cmf = take((int64_t)(g.nt + 2) * nb);
    A->ce0 = (double*)take(((int64_t)(g.nt + 2) * nb + 1) / 2);
    A->mu = take(A->E * nb);
    A->ctot = take(A->E * nb);
    A->ctot0 = take(A->E * nb);
    A->Pk = take(A->E * nb);
    A->cSx = take(A->E);
    A->cLb = take(A->E);
    A->cmfx = take((int64_t)(g.nt + 2) * nb);
    A->dist = (double*)take(1);
    return off;
}

// slice views: of a herm at step n (ld = nb or 1) ...
SliceV herm_slice(const HermV& X, int n, int ntau) {
    const int64_t ld = X.ret.ldk;
    return SliceV{X.ret.p + tri(n) * ld, X.les.p + tri(n) * ld, X.tv.p + (int64_t)n * (ntau + 1) * ld};
}
// ... of one captured pass in the iterate store
struct Captured {
    SliceV Gk, Gl, S;
    cplx* mf;
};
Captured captured(const AdjLayout& A, const Grid& g, int q, int it, int n) {
    cplx* b = A.store + ((int64_t)q * A.corr + it) * A.itstride;
    const int64_t nb = g.nb, n1 = n + 1;
    Captured c;
    c.Gk = SliceV{b, b + n1 * nb, b + 2 * n1 * nb};
    cplx* l = b + A.L * nb;
    c.Gl = SliceV{l, l + n1, l + 2 * n1};
    cplx* s = l + A.L;
    c.S = SliceV{s, s + n1, s + 2 * n1};
    c.mf = s + A.L;
    return c;
}
// ... of slice n of slices 0..k in the compact layout of ng_adjoint_types.h
SliceV boot_slice(cplx* base, int64_t ld, int k, int ntau, int n) {
    const int64_t T3 = tri(k + 1);
    return SliceV{base + tri(n) * ld, base + (T3 + tri(n)) * ld, base + (2 * T3 + (int64_t)n * (ntau + 1)) * ld};
}

#define ADJ_TRY(ctx, call, what)                                                               \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return fail(ctx, NG_ECUDA, "%s: %s", what, cudaGetErrorString(e_)); \
    } while (0)

// forward step n of the driver with the iterates of every corrector pass captured (FP64)
ng_status adj_forward_step(ng_ctx* c, const Grid& g, int n, int corr, const HermV& Gv, const HermV& Lv, const HermV& Sv,
                           const FuncV& mf, const FuncV& e0, const FuncV& uv, double nbar, const AdjLayout& A, int q,
                           cudaStream_t s) {
    ng_status st;
    if ((st = do_extrap(c, g, n - 1, Gv, s))) return st;
    for (int it = 0; it < corr; ++it) {
        const Captured cp = captured(A, g, q, it, n);
        if ((st = do_kreduce(c, g, n, Lv, Gv, s))) return st;
        ADJ_TRY(c, adj_slice_copy(n, g.ntau, 1, herm_slice(Lv, n, g.ntau), cp.Gl, s), "capture of G_loc");
        if ((st = do_hartree(c, g, n, mf, e0, Lv, uv, nbar, s))) return st;
        CUDA_TRY(c, cudaMemcpyAsync(cp.mf, mf.p + (int64_t)(n + 1) * g.nb, sizeof(cplx) * g.nb,
                                    cudaMemcpyDeviceToDevice, s));
        if ((st = do_sigma(c, g, n, Sv, Lv, uv, s))) return st;
        ADJ_TRY(c, adj_slice_copy(n, g.ntau, 1, herm_slice(Sv, n, g.ntau), cp.S, s), "capture of Sigma");
        if ((st = do_timestep(c, g, n, Gv, Sv, mf, s, NG_FP64))) return st;
        ADJ_TRY(c, adj_slice_copy(n, g.ntau, g.nb, herm_slice(Gv, n, g.ntau), cp.Gk, s), "capture of G");
    }
    return NG_OK;
}

// backward step n: the corrector passes in reverse, then the predictor
ng_status adj_backward_step(ng_ctx* c, const Grid& g, int n, const HermV& Gv, const HermV& Sv, const FuncV& mf,
                            const FuncV& uv, const HermV& cG, const HermV& cS, const AdjLayout& A, int q,
                            cudaStream_t s) {
    const int k = g.k, nb = g.nb, T = g.ntau;
    const SliceV cw{A.cw, A.cw + (int64_t)(n + 1) * nb, A.cw + 2 * (int64_t)(n + 1) * nb};
    const SliceV cSw{A.cSw, A.cSw + (n + 1), A.cSw + 2 * (n + 1)};
    const SliceV cLoc{A.cLoc, A.cLoc + (n + 1), A.cLoc + 2 * (n + 1)};
    // cotangents of the final slice n, of Sigma slice n and of eps_mf(n) start the last pass
    ADJ_TRY(c, adj_slice_copy(n, T, nb, herm_slice(cG, n, T), cw, s), "gather of c(G)");
    ADJ_TRY(c, adj_slice_copy(n, T, 1, herm_slice(cS, n, T), cSw, s), "gather of c(Sigma)");
    CUDA_TRY(c, cudaMemcpyAsync(A.cmfw, A.cmf + (int64_t)(n + 1) * nb, sizeof(cplx) * nb, cudaMemcpyDeviceToDevice, s));
    AdjStep a;
    a.g = g;
    a.n = n;
    a.full = (n <= 2 * k);
    a.m0 = a.full ? 1 : n - k;
    a.nq = n - a.m0 + 1;
    a.Gr = Gv.ret.p; a.Gl = Gv.les.p; a.Gt = Gv.tv.p; a.Gm = Gv.mat.p;
    a.Sr = Sv.ret.p; a.Sl = Sv.les.p; a.St = Sv.tv.p;
    a.mf = mf.p;
    a.cGr = cG.ret.p; a.cGl = cG.les.p; a.cGt = cG.tv.p;
    a.cSr = cS.ret.p; a.cSl = cS.les.p; a.cSt = cS.tv.p;
    a.cmf = A.cmf;
    a.cw = cw;
    a.cSw = cSw;
    a.cmfw = A.cmfw;
    a.cA = A.cA; a.caccR = A.caccR; a.caccT = A.caccT; a.crhs = A.crhs; a.cMn = A.cMn; a.retA = A.retA;
    a.part = A.part;
    a.plen = A.L;
    for (int it = A.corr - 1; it >= 0; --it) {
        const Captured cp = captured(A, g, q, it, n);
        a.Gc = cp.Gk;
        a.Sc = cp.S;
        a.mfc = cp.mf;
        ADJ_TRY(c, adj_pass(a, cp.Gl, uv.p, cLoc, A.ce0 + (int64_t)(n + 1) * nb, s), "adjoint corrector pass");
    }
    ADJ_TRY(c, adj_predictor(g, n, cw, cG.ret.p, cG.les.p, cG.tv.p, s), "adjoint predictor");
    return NG_OK;
}

// start slices 0..k: fixed point x = F(x, eps0) of the bootstrapping; implicit adjoint
// mu = c_tot + F_x^T mu by iteration, then d/deps0 = F_eps^T mu
ng_status adj_boot(ng_ctx* c, const Grid& g, const HermV& Gv, const HermV& Lv, const HermV& Sv, const FuncV& mf,
                   const FuncV& uv, const HermV& cG, const HermV& cS, const AdjLayout& A, double tol, int maxiter,
                   int* iters, cudaStream_t s) {
    const int k = g.k, nb = g.nb, T = g.ntau;
    const int64_t E = A.E;
    ng_status st;
    for (int n = 0; n <= k; ++n)   // G_loc slices 0..k of the final start slices
        if ((st = do_kreduce(c, g, n, Lv, Gv, s))) return st;
    // cotangent of the start slices: direct, plus through Sigma(0..k) and eps_mf(0..k)
    ADJ_TRY(c, adj_boot_gather(g, cG.ret.p, cG.les.p, cG.tv.p, nb, A.ctot0, s), "start-slice gather");
    auto through_sigma = [&](const cplx* cSig /* compact, ld 1 */, const cplx* cmfr, bool from_herm) -> ng_status {
        for (int n = 0; n <= k; ++n) {
            SliceV cs = from_herm ? herm_slice(cS, n, T) : boot_slice((cplx*)cSig, 1, k, T, n);
            ADJ_TRY(c, adj_sigma2b(g, n, herm_slice(Lv, n, T), cs, cmfr + (int64_t)(n + 1) * nb, uv.p,
                                   boot_slice(A.cLb, 1, k, T, n), s), "second-Born transpose (start slices)");
        }
        return NG_OK;
    };
    if ((st = through_sigma(nullptr, A.cmf, true))) return st;
    ADJ_TRY(c, adj_ce0_rows(k + 1, nb, A.cmf, A.ce0, s), "eps0 cotangent (start slices)");
    CUDA_TRY(c, cudaMemsetAsync(A.dist, 0, 2 * sizeof(double), s));
    ADJ_TRY(c, adj_boot_update(E, nb, A.ctot0, A.cLb, A.ctot, A.dist, s), "start-slice update");
    CUDA_TRY(c, cudaMemcpyAsync(A.mu, A.ctot, sizeof(cplx) * E * nb, cudaMemcpyDeviceToDevice, s));
    AdjBoot b;
    b.g = g;
    b.Gr = Gv.ret.p; b.Gl = Gv.les.p; b.Gt = Gv.tv.p; b.Gm = Gv.mat.p;
    b.Sr = Sv.ret.p; b.Sl = Sv.les.p; b.St = Sv.tv.p;
    b.mf = mf.p;
    b.mu = A.mu;
    b.Pk = A.Pk;
    b.cmfx = A.cmfx;
    auto start_vjp = [&]() -> ng_status {
        CUDA_TRY(c, cudaMemsetAsync(A.Pk, 0, sizeof(cplx) * E * nb, s));
        CUDA_TRY(c, cudaMemsetAsync(A.cmfx, 0, sizeof(cplx) * (size_t)(k + 2) * nb, s));
        ADJ_TRY(c, adj_boot_start(b, s), "start-up transpose");
        return NG_OK;
    };
    int it = 0;
    bool done = false;
    for (it = 1; it <= maxiter; ++it) {
        if ((st = start_vjp())) return st;
        ADJ_TRY(c, adj_boot_reduce(E, nb, A.Pk, A.cSx, s), "start-slice reduction");
        if ((st = through_sigma(A.cSx, A.cmfx, false))) return st;
        CUDA_TRY(c, cudaMemsetAsync(A.dist, 0, 2 * sizeof(double), s));
        ADJ_TRY(c, adj_boot_update(E, nb, A.ctot, A.cLb, A.mu, A.dist, s), "start-slice update");
        double d[2];
        CUDA_TRY(c, cudaMemcpyAsync(d, A.dist, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(c, cudaStreamSynchronize(s));
        if (!(d[0] == d[0]) || !(d[1] == d[1])) return fail(c, NG_ENONFINITE, "adjoint of the start slices is not finite");
        if (d[0] <= tol * d[1]) { done = true; break; }
    }
    // F_eps^T at the final mu
    if ((st = start_vjp())) return st;
    ADJ_TRY(c, adj_ce0_rows(k + 1, nb, A.cmfx, A.ce0, s), "eps0 cotangent (start slices)");
    if (iters) *iters = it;
    if (!done) return fail(c, NG_ENOCONV, "adjoint of the start slices did not converge in %d iterations", maxiter);
    return NG_OK;
}

}  // namespace

// the second-Born forward run with every corrector iterate kept for the adjoint: the setup of
// ng_run_2b, then each time step through the capturing forward step of the recomputation
extern "C" ng_status ng_adjoint_forward(ng_ctx* c, const ng_grid* grid, ng_herm G, ng_herm Gloc, ng_herm S,
                                        ng_func eps0, ng_func epsmf, ng_func U, const ng_run_params* p,
                                        int* iters_out, void* stream) {
    Grid g;
    HermV Gv, Lv, Sv;
    FuncV e0, mf, uv;
    ng_status st;
    if ((st = check_grid(c, grid, &g))) return st;
    if (g.nf != 1) return fail(c, NG_EUNSUPPORTED, "ng_adjoint_forward supports nf = 1 (nf = %d)", g.nf);
    if (!p) return fail(c, NG_EINVAL, "params is NULL");
    if (p->corrector < 1) return fail(c, NG_EINVAL, "corrector must be >= 1");
    if (G.ldk != g.nb) return fail(c, NG_EINVAL, "G must have ldk = nbatch");
    if ((st = check_herm(c, g, G, "G", true, &Gv, g.nb))) return st;
    if (Gloc.ldk != 1 || S.ldk != 1) return fail(c, NG_EINVAL, "Gloc and Sigma must have ldk = 1");
    if ((st = check_herm(c, g, Gloc, "Gloc", true, &Lv, 1))) return st;
    if ((st = check_herm(c, g, S, "Sigma", true, &Sv, 1))) return st;
    if ((st = check_func(c, g, eps0, "eps0", &e0))) return st;
    if ((st = check_func(c, g, epsmf, "eps_mf", &mf))) return st;
    if ((st = check_func(c, g, U, "U", &uv))) return st;
    if (U.ldk != 1 || epsmf.ldk != g.nb || eps0.ldk != g.nb)
        return fail(c, NG_EINVAL, "U.ldk must be 1 and eps0.ldk, eps_mf.ldk must be nbatch");
    c->adj_rec = false;
    const int k = g.k, nsteps = g.nt - k;
    AdjLayout A;
    const size_t need = adj_layout(g, nsteps, p->corrector, &A, nullptr);
    if ((st = ensure(c, &c->ws_adj, &c->ws_adj_bytes, need))) return st;
    adj_layout(g, nsteps, p->corrector, &A, (char*)c->ws_adj);
    ng_run_params q = *p;
    q.n_from = k + 1;
    q.n_to = k;            // setup only: Matsubara loop and bootstrapping
    q.do_setup = 1;
    q.precision = NG_FP64;
    if ((st = run_2b_impl(c, grid, G, Gloc, S, eps0, epsmf, U, &q, nullptr, nullptr, iters_out, stream))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    for (int n = k + 1; n <= g.nt; ++n)
        if ((st = adj_forward_step(c, g, n, p->corrector, Gv, Lv, Sv, mf, e0, uv, p->nbar, A, n - (k + 1), s)))
            return st;
    c->adj_rec = true;
    c->adj_rec_nt = g.nt;
    c->adj_rec_ntau = g.ntau;
    c->adj_rec_nb = g.nb;
    c->adj_rec_corr = p->corrector;
    c->adj_rec_G = G.ret;
    return NG_OK;
}

extern "C" ng_status ng_adjoint_2b(ng_ctx* c, const ng_grid* grid, ng_herm G, ng_herm Gloc, ng_herm S, ng_func eps0,
                                   ng_func epsmf, ng_func U, const ng_run_params* p, const void* seed, ng_herm cG,
                                   ng_herm cS, int segment, double* grad_eps0, int* info, void* stream) {
    Grid g;
    HermV Gv, Lv, Sv, cGv, cSv;
    FuncV e0, mf, uv;
    ng_status st;
    if ((st = check_grid(c, grid, &g))) return st;
    if (g.nf != 1) return fail(c, NG_EUNSUPPORTED, "ng_adjoint_2b supports nf = 1 (nf = %d)", g.nf);
    if (!p || !seed || !grad_eps0) return fail(c, NG_EINVAL, "params, seed and grad_eps0 must not be NULL");
    if (p->corrector < 1) return fail(c, NG_EINVAL, "corrector must be >= 1");
    if (G.ldk != g.nb || cG.ldk != g.nb) return fail(c, NG_EINVAL, "G and cG must have ldk = nbatch");
    if ((st = check_herm(c, g, G, "G", true, &Gv, g.nb))) return st;
    if ((st = check_herm(c, g, cG, "cG", true, &cGv, g.nb))) return st;
    if (Gloc.ldk != 1 || S.ldk != 1 || cS.ldk != 1) return fail(c, NG_EINVAL, "Gloc, Sigma and cS must have ldk = 1");
    if ((st = check_herm(c, g, Gloc, "Gloc", true, &Lv, 1))) return st;
    if ((st = check_herm(c, g, S, "Sigma", true, &Sv, 1))) return st;
    if ((st = check_herm(c, g, cS, "cS", true, &cSv, 1))) return st;
    if ((st = check_func(c, g, eps0, "eps0", &e0))) return st;
    if ((st = check_func(c, g, epsmf, "eps_mf", &mf))) return st;
    if ((st = check_func(c, g, U, "U", &uv))) return st;
    if (U.ldk != 1 || epsmf.ldk != g.nb || eps0.ldk != g.nb)
        return fail(c, NG_EINVAL, "U.ldk must be 1 and eps0.ldk, eps_mf.ldk must be nbatch");
    if (!aligned16(seed) || ((uintptr_t)grad_eps0 & 7u)) return fail(c, NG_EINVAL, "seed or grad_eps0 misaligned");
    cudaStream_t s = (cudaStream_t)stream;
    const int k = g.k, nb = g.nb, T = g.ntau, N = g.nt;
    const int nsteps = N - k;
    const bool recorded = segment == NG_ADJ_RECORDED;
    if (recorded && !(c->adj_rec && c->adj_rec_nt == N && c->adj_rec_ntau == T && c->adj_rec_nb == nb &&
                      c->adj_rec_corr == p->corrector && c->adj_rec_G == G.ret))
        return fail(c, NG_EINVAL, "segment = NG_ADJ_RECORDED needs a preceding ng_adjoint_forward of this G and shape");
    if (segment < 0 && !recorded) return fail(c, NG_EINVAL, "segment = %d invalid", segment);
    int seg = recorded ? nsteps : (segment > 0 ? segment : (int)std::ceil(std::sqrt((double)nsteps)));
    seg = std::max(1, std::min(seg, nsteps));
    if (!recorded) c->adj_rec = false;   // the recomputation reuses the store
    AdjLayout A;
    const size_t need = adj_layout(g, seg, p->corrector, &A, nullptr);
    if ((st = ensure(c, &c->ws_adj, &c->ws_adj_bytes, need))) return st;
    adj_layout(g, seg, p->corrector, &A, (char*)c->ws_adj);
    // cotangent stores start at zero, then the seed on the G^<(n,n) diagonal
    const size_t per = sizeof(cplx) * (size_t)nb;
    CUDA_TRY(c, cudaMemsetAsync(cG.ret, 0, per * tri(N + 1), s));
    CUDA_TRY(c, cudaMemsetAsync(cG.les, 0, per * tri(N + 1), s));
    CUDA_TRY(c, cudaMemsetAsync(cG.tv, 0, per * (size_t)(N + 1) * (T + 1), s));
    CUDA_TRY(c, cudaMemsetAsync(cS.ret, 0, sizeof(cplx) * tri(N + 1), s));
    CUDA_TRY(c, cudaMemsetAsync(cS.les, 0, sizeof(cplx) * tri(N + 1), s));
    CUDA_TRY(c, cudaMemsetAsync(cS.tv, 0, sizeof(cplx) * (size_t)(N + 1) * (T + 1), s));
    CUDA_TRY(c, cudaMemsetAsync(A.cmf, 0, per * (N + 2), s));
    CUDA_TRY(c, cudaMemsetAsync(A.ce0, 0, sizeof(double) * (size_t)(N + 2) * nb, s));
    ADJ_TRY(c, adj_seed(g, (const cplx*)seed, (cplx*)cG.les, s), "seed");
    // segments from the last: [s0, s1], recomputed forward with capture, then walked backwards
    int nseg = 0;
    for (int s1 = N; s1 > k; s1 -= seg, ++nseg) {
        const int s0 = std::max(k + 1, s1 - seg + 1);
        for (int n = s0; n <= s1 && !recorded; ++n)
            if ((st = adj_forward_step(c, g, n, p->corrector, Gv, Lv, Sv, mf, e0, uv, p->nbar, A, n - s0, s)))
                return st;
        for (int n = s1; n >= s0; --n)
            if ((st = adj_backward_step(c, g, n, Gv, Sv, mf, uv, cGv, cSv, A, n - s0, s))) return st;
    }
    int boot_it = 0;
    if ((st = adj_boot(c, g, Gv, Lv, Sv, mf, uv, cGv, cSv, A, p->boot_tol > 0 ? p->boot_tol : 1e-14,
                       p->boot_maxiter > 0 ? p->boot_maxiter : 200, &boot_it, s)))
        return st;
    CUDA_TRY(c, cudaMemcpyAsync(grad_eps0, A.ce0, sizeof(double) * (size_t)(N + 2) * nb, cudaMemcpyDeviceToDevice, s));
    if (info) {
        info[0] = boot_it;
        info[1] = nseg;
        info[2] = seg;
    }
    return NG_OK;
}
