// Slice kernels of libng: k-point reduction, second-Born self-energy, Hartree mean field,
// extrapolation (predictor) and the slice distance.
#pragma once

#include "ng_common.cuh"


// Elements of one time slice tstp >= 0: ret row (tstp+1), les column (tstp+1), tv row (ntau+1);
// tstp = -1: mat (ntau+1).  Maps a linear slice element index to (component, offset).
struct SliceEl {
    int comp;      // 0 mat, 1 ret, 2 les, 3 tv
    int64_t e;     // element index in that component
    int j;         // column / row / tau index within the slice
};
__device__ __forceinline__ int slice_count(const Grid& g, int tstp) {
    return tstp < 0 ? g.ntau + 1 : 2 * (tstp + 1) + g.ntau + 1;
}
__device__ __forceinline__ SliceEl slice_el(const Grid& g, int tstp, int i) {
    SliceEl s;
    if (tstp < 0) { s.comp = 0; s.e = i; s.j = i; return s; }
    if (i <= tstp) { s.comp = 1; s.e = tri(tstp) + i; s.j = i; return s; }
    i -= tstp + 1;
    if (i <= tstp) { s.comp = 2; s.e = tri(tstp) + i; s.j = i; return s; }
    i -= tstp + 1;
    s.comp = 3; s.e = (int64_t)tstp * (g.ntau + 1) + i; s.j = i;
    return s;
}
__device__ __forceinline__ const Comp& comp_of(const HermV& X, int c) {
    return c == 0 ? X.mat : (c == 1 ? X.ret : (c == 2 ? X.les : X.tv));
}

// ---------------------------------------------------------------------------------------
// k-point reduction Gloc = sum_kb w_kb Gk (w_kb = 1/nk without weights), in one fixed order
// that does not depend on how the k-points are split over ranks: the k axis is cut into
// blocks of NG_KBLK = 32 consecutive global k indices; a block's weighted values are added
// across a warp in a fixed butterfly order; the block sums are added in block order starting
// from zero; the 1/nk factor comes last.  A rank owning whole blocks produces the same block
// sums (k_kreduce_partial), and adding everybody's block sums in block order
// (k_kreduce_combine) gives bitwise the single-GPU result (k_kreduce).
// ---------------------------------------------------------------------------------------
#define NG_KBLK 32
#define NG_MAXRANKS 64

// first global block of every rank (first[nranks] = number of blocks), passed by value
struct BlkMap {
    int first[NG_MAXRANKS + 1];
};

// Block b of one slice element (kb = NG_KBLK b + lane global; local index kb - kb0 of the nbl
// local problems, value stride 1); every lane returns the same block sum (each butterfly stage
// adds a pair in both lanes, and floating-point addition commutes).
__device__ __forceinline__ cplx kblock_sum(const cplx* p, const double* wk, int b, int kb0, int nbl, int lane) {
    const int kl = b * NG_KBLK + lane - kb0;
    cplx v = cz();
    if (kl >= 0 && kl < nbl) {
        v = p[kl];
        if (wk) v = cscal(wk[kl], v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// Single GPU holding all nb problems: one warp per (slice element, a, b).
__global__ void k_kreduce(Grid g, int tstp, HermV Gloc, HermV Gk, const double* wk) {
    const int dd = g.nf * g.nf;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int cnt = slice_count(g, tstp);
    if (w >= (int64_t)cnt * dd) return;
    const int ab = (int)(w % dd), i = (int)(w / dd);
    const SliceEl s = slice_el(g, tstp, i);
    const Comp& src = comp_of(Gk, s.comp);
    const Comp& dst = comp_of(Gloc, s.comp);
    const cplx* p = src.p + (s.e * dd + ab) * (int64_t)src.ldk;
    const int nblk = (g.nb + NG_KBLK - 1) / NG_KBLK;
    cplx acc = cz();
    for (int b = 0; b < nblk; ++b) acc = cadd(acc, kblock_sum(p, wk, b, 0, g.nb, lane));
    if (lane == 0) dst.p[(s.e * dd + ab) * (int64_t)dst.ldk] = wk ? acc : cscal(1.0 / g.nb, acc);
}

// One rank's block sums: the local problems are global k indices kb0..kb0+nb-1 (kb0 a multiple
// of NG_KBLK); out[(bl * cnt + i) * dd + ab] for the local blocks bl = 0..nblk_local-1.
// One warp per (local block, slice element, a, b).
__global__ void k_kreduce_partial(Grid g, int tstp, HermV Gk, const double* wk, int kb0, cplx* out) {
    const int dd = g.nf * g.nf;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int cnt = slice_count(g, tstp);
    const int nblk = (g.nb + NG_KBLK - 1) / NG_KBLK;
    if (w >= (int64_t)nblk * cnt * dd) return;
    const int ab = (int)(w % dd);
    const int64_t r = w / dd;
    const int i = (int)(r % cnt), bl = (int)(r / cnt);
    const SliceEl s = slice_el(g, tstp, i);
    const Comp& src = comp_of(Gk, s.comp);
    const cplx* p = src.p + (s.e * dd + ab) * (int64_t)src.ldk;
    const cplx v = kblock_sum(p, wk, kb0 / NG_KBLK + bl, kb0, g.nb, lane);
    if (lane == 0) out[((int64_t)bl * cnt + i) * dd + ab] = v;
}

// Every rank's block sums gathered rank by rank, maxb block rows per rank (rows beyond a rank's
// own blocks unused); global block b of rank r sits in row r maxb + (b - first block of r).
// Adds them in global block order; one thread per (slice element, a, b).  nk: global problem
// count, map.first[r]: first global block of rank r (r = 0..nranks).
__global__ void k_kreduce_combine(Grid g, int tstp, HermV Gloc, const cplx* gathered, int nk, int nranks, int maxb,
                                  BlkMap map, int weighted) {
    const int dd = g.nf * g.nf;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int cnt = slice_count(g, tstp);
    if (item >= (int64_t)cnt * dd) return;
    const int ab = (int)(item % dd), i = (int)(item / dd);
    const SliceEl s = slice_el(g, tstp, i);
    const Comp& dst = comp_of(Gloc, s.comp);
    cplx acc = cz();
    for (int r = 0; r < nranks; ++r)
        for (int b = map.first[r]; b < map.first[r + 1]; ++b) {
            const int64_t row = (int64_t)r * maxb + (b - map.first[r]);
            acc = cadd(acc, gathered[(row * cnt + i) * dd + ab]);
        }
    dst.p[(s.e * dd + ab) * (int64_t)dst.ldk] = weighted ? acc : cscal(1.0 / nk, acc);
}

// Second-Born slice (Eq. sigma_hubb_2b), orbital-elementwise:
//   Sigma^<_ab(j,n)  = U_j U_n G^<_ab(j,n)^2 G^>_ba(n,j)
//   Sigma^R_ab(n,j)  = U_n U_j [G^>_ab(n,j)^2 G^<_ba(j,n) - G^<_ab(n,j)^2 G^>_ba(j,n)]
//   Sigma^tv_ab(n,m) = U_n U_{-1} G^tv_ab(n,m)^2 G^vt_ba(m,n)
//   Sigma^M_ab(tau)  = -U_{-1}^2 G^M_ab(tau)^2 G^M_ba(-tau)
// one thread per (slice element, a, b); G and Sigma have ldk = 1.
__global__ void k_sigma2b(Grid g, int tstp, HermV S, HermV G, FuncV U) {
    const int nf = g.nf, dd = nf * nf;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int cnt = slice_count(g, tstp);
    if (item >= (int64_t)cnt * dd) return;
    const int ab = (int)(item % dd), i = (int)(item / dd);
    const int a = ab / nf, b = ab % nf;
    const SliceEl s = slice_el(g, tstp, i);
    const double xi = (double)g.sig;
    auto u = [&](int n) { return U.p[n + 1].x; };
    auto ldG = [&](const Comp& c, int64_t e, int x, int y) { return c.p[e * dd + x * nf + y]; };
    auto sq = [](cplx z) { return cmul(z, z); };
    const int n = tstp;
    if (s.comp == 0) {
        const int m = s.j;
        cplx gab = ldG(G.mat, m, a, b);
        cplx gneg = cscal(xi, ldG(G.mat, g.ntau - m, b, a));  // G^M_ba(-tau) = xi G^M_ba(beta - tau)
        S.mat.p[(int64_t)m * dd + ab] = cscal(-u(-1) * u(-1), cmul(sq(gab), gneg));
        return;
    }
    if (s.comp == 1 || s.comp == 2) {
        const int j = s.j;
        // G^<_xy(j,n) stored; G^<_xy(n,j) = -conj(G^<_yx(j,n)); G^>(n,j) = G^R(n,j) + G^<(n,j);
        // G^>_xy(j,n) = -conj(G^>_yx(n,j))
        const int64_t eR = tri(n) + j, eL = tri(n) + j;
        auto lesjn = [&](int x, int y) { return ldG(G.les, eL, x, y); };
        auto lesnj = [&](int x, int y) { return cneg(cconj(ldG(G.les, eL, y, x))); };
        auto gtrnj = [&](int x, int y) { return cadd(ldG(G.ret, eR, x, y), lesnj(x, y)); };
        auto gtrjn = [&](int x, int y) { return cneg(cconj(gtrnj(y, x))); };
        const double uu = u(n) * u(j);
        if (s.comp == 1) {
            cplx sg = cmul(sq(gtrnj(a, b)), lesjn(b, a));
            cplx sl = cmul(sq(lesnj(a, b)), gtrjn(b, a));
            S.ret.p[eR * dd + ab] = cscal(uu, csub(sg, sl));
        } else {
            S.les.p[eL * dd + ab] = cscal(uu, cmul(sq(lesjn(a, b)), gtrnj(b, a)));
        }
        return;
    }
    const int m = s.j;
    cplx gtv = ldG(G.tv, (int64_t)n * (g.ntau + 1) + m, a, b);
    // G^vt_ba(tau_m, t_n) = -xi conj(G^tv_ab(t_n, beta - tau_m))
    cplx gvt = cscal(-xi, cconj(ldG(G.tv, (int64_t)n * (g.ntau + 1) + (g.ntau - m), a, b)));
    S.tv.p[s.e * dd + ab] = cscal(u(n) * u(-1), cmul(sq(gtv), gvt));
}

// eps_mf_kb(n) = eps0_kb(n) + U_n diag(Re rho_ii - nbar); one thread per (problem, a, b)
__global__ void k_hartree(Grid g, int tstp, FuncV epsmf, FuncV eps0, HermV G, FuncV U, double nbar) {
    const int nf = g.nf, dd = nf * nf;
    const int ldk = epsmf.ldk;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= (int64_t)ldk * dd) return;
    const int kb = (int)(item % ldk), ab = (int)(item / ldk);
    const int a = ab / nf, b = ab % nf;
    cplx v = eps0.p[((int64_t)(tstp + 1) * dd + ab) * eps0.ldk + (eps0.ldk == 1 ? 0 : kb)];
    if (a == b) {
        double rho;
        if (tstp < 0) rho = -G.mat.p[(int64_t)g.ntau * dd + a * nf + a].x;            // -G^M(beta^-)
        else rho = G.les.p[(tri(tstp) + tstp) * dd + a * nf + a].y;                   // Re(-i G^<)
        v.x += U.p[tstp + 1].x * (rho - nbar);
    }
    epsmf.p[((int64_t)(tstp + 1) * dd + ab) * ldk + kb] = v;
}

// Predictor (Eq. polyextrap): slice n+1 from slices n-k..n; one thread per
// (slice element of n+1, a, b, problem).
__global__ void k_extrapolate(Grid g, int n, HermV G) {
    const int nf = g.nf, dd = nf * nf, k = g.k;
    const double* Cw = c_W[k - 1].C;
    const int N1 = n + 1;
    const int cnt = 2 * (N1 + 1) + g.ntau + 1;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int ldk = G.ret.ldk;
    if (item >= (int64_t)cnt * dd * ldk) return;
    const int kb = (int)(item % ldk);
    const int64_t r = item / ldk;
    const int ab = (int)(r % dd);
    int i = (int)(r / dd);
    const int a = ab / nf, b = ab % nf;
    auto P = [&](const Comp& c, int64_t e, int x, int y) { return c.p[(e * dd + x * nf + y) * ldk + kb]; };
    cplx acc = cz();
    if (i <= N1) {  // ret row N1, column j = i
        const int j = i;
        if (j <= k) {   // column extrapolation of G~^R(t, j)
            for (int l = 0; l <= k; ++l) {
                const int t = n - l;
                cplx v = (j <= t) ? P(G.ret, tri(t) + j, a, b) : cneg(cconj(P(G.ret, tri(j) + t, b, a)));
                acc = cadd(acc, cscal(Cw[l], v));
            }
        } else {        // along the diagonal t - t' = N1 - j
            const int jd = N1 - j;
            for (int l = 0; l <= k; ++l) acc = cadd(acc, cscal(Cw[l], P(G.ret, tri(n - l) + n - l - jd, a, b)));
        }
        G.ret.p[((tri(N1) + j) * dd + ab) * ldk + kb] = acc;
        return;
    }
    i -= N1 + 1;
    if (i <= N1) {  // les column N1, row j = i
        const int j = i;
        if (j <= k) {   // row extrapolation of G^<(j, t), hermitian continuation for t < j
            for (int l = 0; l <= k; ++l) {
                const int t = n - l;
                cplx v = (j <= t) ? P(G.les, tri(t) + j, a, b) : cneg(cconj(P(G.les, tri(j) + t, b, a)));
                acc = cadd(acc, cscal(Cw[l], v));
            }
        } else {        // along the diagonal t' - t = N1 - j
            const int off = N1 - j;
            for (int l = 0; l <= k; ++l) acc = cadd(acc, cscal(Cw[l], P(G.les, tri(n - l) + n - l - off, a, b)));
        }
        G.les.p[((tri(N1) + j) * dd + ab) * ldk + kb] = acc;
        return;
    }
    i -= N1 + 1;
    for (int l = 0; l <= k; ++l)
        acc = cadd(acc, cscal(Cw[l], P(G.tv, (int64_t)(n - l) * (g.ntau + 1) + i, a, b)));
    G.tv.p[(((int64_t)N1 * (g.ntau + 1) + i) * dd + ab) * ldk + kb] = acc;
}

// out += sum |A - B| over slice tstp, all problems (Eq. distancenorm)
__global__ void k_distance(Grid g, int tstp, HermV A, HermV B, double* out) {
    const int dd = g.nf * g.nf;
    const int ldk = A.ret.ldk;
    const int cnt = slice_count(g, tstp);
    const int64_t tot = (int64_t)cnt * dd * ldk;
    double s = 0.0;
    for (int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; item < tot;
         item += (int64_t)gridDim.x * blockDim.x) {
        const int kb = (int)(item % ldk);
        const int64_t r = item / ldk;
        const int ab = (int)(r % dd), i = (int)(r / dd);
        const SliceEl e = slice_el(g, tstp, i);
        const int64_t off = (e.e * dd + ab) * ldk + kb;
        cplx x = csub(comp_of(A, e.comp).p[off], comp_of(B, e.comp).p[off]);
        s += sqrt(cabs2(x));
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(out, s);
}

// bootstrapping initial guess eps_mf(n) = eps_mf(-1) - eps0(-1) + eps0(n)
__global__ void k_mf_init(Grid g, int n, FuncV epsmf, FuncV eps0) {
    const int dd = g.nf * g.nf, ldk = epsmf.ldk;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= (int64_t)dd * ldk) return;
    const int kb = (int)(item % ldk), ab = (int)(item / ldk);
    const int k0 = eps0.ldk == 1 ? 0 : kb;
    cplx a = epsmf.p[(int64_t)(0 * dd + ab) * ldk + kb];
    cplx b = eps0.p[(int64_t)(0 * dd + ab) * eps0.ldk + k0];
    cplx c = eps0.p[(int64_t)((n + 1) * dd + ab) * eps0.ldk + k0];
    epsmf.p[(int64_t)((n + 1) * dd + ab) * ldk + kb] = cadd(csub(a, b), c);
}
