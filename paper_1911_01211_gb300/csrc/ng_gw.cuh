// GW self-energy chain on one time slice (Sec. "Self-energy approximation: GW", Eq. SigmaGW,
// Eq. dyson_chi), elementwise in the orbital indices; one thread per (slice element, a, b, r):
//   P_ab(t,t')   = -i G_ab(t,t') G_ba(t',t)  = -Bubble1[G, G]         (Eq. def_bubble1)
//   K = -P U(t'),  K^ddagger = -U(t) P       kernel of (1 + K) * chi = P
//   dW_ab(t,t')  = U(t) chi_ab(t,t') U(t')
//   Sigma_ab     = i G_ab(t,t') dW_ab(t,t')  = Bubble2[G, dW]          (Eq. def_bubble2)
// Keldysh components by the Langreth rules for products; the Matsubara components follow from
// C^M(tau) = -i C(-i tau, 0) (Eq. matsconv): Bubble1 C^M = -A^M(tau) B^M(-tau), Bubble2
// C^M = -A^M(tau) B^M(tau).  On the diagonal j = n the equal-time lesser value is used as
// stored (no conjugate continuation), so G^<(n,n) need not be exactly anti-hermitian.
//
// The last index r (0..L-1) is either absent (L = 1: a local function of the site/orbital
// indices) or the lattice vector of a translation-invariant function X(r) = X_{r_i - r_j} on a
// ring of L sites (k-space GW evaluated in real space, Eqs. Sigmak and Pol after the lattice
// Fourier transform).  Hermitian conjugation maps (a, b, r) to (b, a, -r mod L).
#pragma once

#include "ng_slice.cuh"

// Where the elements of slice tstp live: the whole-contour store (buf == nullptr; element
// indices of the packed layout, ldk = L) or a compact buffer holding that slice only,
// [i][a][b][r] with i the slice position of slice_el (mat: m; ret: j; les: n+1+j;
// tv: 2(n+1)+m).
struct SliceView {
    HermV h;
    cplx* buf;
    __device__ __forceinline__ int64_t pos_ret(const Grid& g, int n, int j) const {
        return buf ? (int64_t)j : tri(n) + j;
    }
    __device__ __forceinline__ int64_t pos_les(const Grid& g, int n, int j) const {
        return buf ? (int64_t)n + 1 + j : tri(n) + j;
    }
    __device__ __forceinline__ int64_t pos_tv(const Grid& g, int n, int m) const {
        return buf ? 2 * (int64_t)(n + 1) + m : (int64_t)n * (g.ntau + 1) + m;
    }
    __device__ __forceinline__ cplx* mat_p() const { return buf ? buf : h.mat.p; }
    __device__ __forceinline__ cplx* ret_p() const { return buf ? buf : h.ret.p; }
    __device__ __forceinline__ cplx* les_p() const { return buf ? buf : h.les.p; }
    __device__ __forceinline__ cplx* tv_p() const { return buf ? buf : h.tv.p; }
    // element (slice position i, orbital pair ab) of slice tstp: pointer to its L values
    __device__ __forceinline__ cplx* vec(const Grid& g, int tstp, int i, int ab, int L) const {
        const int dd = g.nf * g.nf;
        if (buf) return buf + ((int64_t)i * dd + ab) * L;
        const SliceEl s = slice_el(g, tstp, i);
        return comp_of(h, s.comp).p + (s.e * dd + ab) * L;
    }
};

// the index of (x, y, r) in an element's [a][b][r] block and of its conjugate partner
struct GwIdx {
    int nf, L;
    __device__ __forceinline__ int64_t own(int x, int y, int r) const { return ((int64_t)x * nf + y) * L + r; }
    __device__ __forceinline__ int64_t cnj(int x, int y, int r) const {
        return ((int64_t)y * nf + x) * L + (r == 0 ? 0 : L - r);
    }
};

// G^<, G^> at (n,j) and (j,n) of the element (x, y, r) for the slice element (n,j), j <= n
struct GwAcc {
    const cplx *R, *Lp;   // the element's [a][b][r] blocks of G^R(n,j) and G^<(j,n)
    GwIdx ix;
    bool diag;            // j == n
    __device__ __forceinline__ cplx les_jn(int x, int y, int r) const { return Lp[ix.own(x, y, r)]; }
    __device__ __forceinline__ cplx les_nj(int x, int y, int r) const {
        return diag ? Lp[ix.own(x, y, r)] : cneg(cconj(Lp[ix.cnj(x, y, r)]));
    }
    __device__ __forceinline__ cplx gtr_nj(int x, int y, int r) const { return cadd(R[ix.own(x, y, r)], les_nj(x, y, r)); }
    __device__ __forceinline__ cplx gtr_jn(int x, int y, int r) const {
        if (diag) return gtr_nj(x, y, r);
        // G^>(j,n) = -[G^>(n,j)]^dagger: the conjugate of the partner's G^>(n,j)
        const int rr = r == 0 ? 0 : ix.L - r;
        return cneg(cconj(gtr_nj(y, x, rr)));
    }
};

// P, K and K^ddagger on slice tstp (-1: Matsubara) from the fermionic G (g.sig); P and the
// kernels are bosonic.  L = 1 or the ring size.
__global__ void k_gw_pol(Grid g, int tstp, int L, SliceView P, SliceView K, SliceView Kcc, SliceView G, FuncV U) {
    const int nf = g.nf, dd = nf * nf;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int cnt = slice_count(g, tstp);
    if (item >= (int64_t)cnt * dd * L) return;
    const int r = (int)(item % L);
    const int ab = (int)((item / L) % dd), i = (int)(item / ((int64_t)L * dd));
    const int a = ab / nf, b = ab % nf;
    const SliceEl s = slice_el(g, tstp, i);
    const double xi = (double)g.sig;
    const GwIdx ix{nf, L};
    auto u = [&](int n) { return U.p[n + 1].x; };
    const int n = tstp;
    cplx p;          // P_ab(r) at this element
    double ul, ur;   // U(t) and U(t') of the element
    int64_t pos;     // slice element position in the views
    cplx *pP, *pK, *pKcc;
    if (s.comp == 0) {
        const int m = s.j;
        // P^M_ab(tau) = G^M_ab(tau) G^M_ba(-tau), G^M(-tau) = xi G^M(beta - tau)
        const cplx* gm = G.mat_p();
        p = cmul(gm[(int64_t)m * dd * L + ix.own(a, b, r)], cscal(xi, gm[(int64_t)(g.ntau - m) * dd * L + ix.cnj(a, b, r)]));
        ul = ur = u(-1);
        pos = m;
        pP = P.mat_p(), pK = K.mat_p(), pKcc = Kcc.mat_p();
    } else if (s.comp == 1 || s.comp == 2) {
        const int j = s.j;
        const GwAcc A{G.ret_p() + G.pos_ret(g, n, j) * dd * L, G.les_p() + G.pos_les(g, n, j) * dd * L, ix, j == n};
        const int rc = r == 0 ? 0 : L - r;
        if (s.comp == 1) {
            // C^R_ab(n,j) = C^>_ab(n,j) - C^<_ab(n,j) with
            // C^>_ab(n,j) = i G^>_ab(n,j) G^<_ba(j,n),  C^<_ab(n,j) = i G^<_ab(n,j) G^>_ba(j,n)
            const cplx c = cmuli(csub(cmul(A.gtr_nj(a, b, r), A.les_jn(b, a, rc)),
                                      cmul(A.les_nj(a, b, r), A.gtr_jn(b, a, rc))));
            p = cneg(c);
            ul = u(n);
            ur = u(j);
            pos = P.pos_ret(g, n, j);
            pP = P.ret_p(), pK = K.ret_p(), pKcc = Kcc.ret_p();
        } else {
            // C^<_ab(j,n) = i G^<_ab(j,n) G^>_ba(n,j)
            p = cneg(cmuli(cmul(A.les_jn(a, b, r), A.gtr_nj(b, a, rc))));
            ul = u(j);
            ur = u(n);
            pos = P.pos_les(g, n, j);
            pP = P.les_p(), pK = K.les_p(), pKcc = Kcc.les_p();
        }
    } else {
        const int m = s.j;
        const cplx* gt = G.tv_p();
        // C^tv_ab(n,m) = i G^tv_ab(n,m) G^vt_ba(m,n),  G^vt_ba(m,n) = -xi conj(G^tv_ab(n, ntau - m))
        const cplx gvt = cscal(-xi, cconj(gt[G.pos_tv(g, n, g.ntau - m) * dd * L + ix.own(a, b, r)]));
        p = cneg(cmuli(cmul(gt[G.pos_tv(g, n, m) * dd * L + ix.own(a, b, r)], gvt)));
        ul = u(n);
        ur = u(-1);
        pos = P.pos_tv(g, n, m);
        pP = P.tv_p(), pK = K.tv_p(), pKcc = Kcc.tv_p();
    }
    // P, K and K^ddagger share the view kind (all compact or all whole-contour)
    const int64_t o = pos * dd * L + ix.own(a, b, r);
    pP[o] = p;
    pK[o] = cneg(cscal(ur, p));
    pKcc[o] = cneg(cscal(ul, p));
}

// Sigma on slice tstp (-1: Matsubara) from the fermionic G and the bosonic chi:
// dW = U(t) chi U(t') formed on the fly, Sigma = Bubble2[G, dW] (same index r on both)
__global__ void k_gw_sigma(Grid g, int tstp, int L, SliceView S, SliceView G, SliceView X, FuncV U) {
    const int nf = g.nf, dd = nf * nf;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int cnt = slice_count(g, tstp);
    if (item >= (int64_t)cnt * dd * L) return;
    const int r = (int)(item % L);
    const int ab = (int)((item / L) % dd), i = (int)(item / ((int64_t)L * dd));
    const int a = ab / nf, b = ab % nf;
    const SliceEl s = slice_el(g, tstp, i);
    const GwIdx ix{nf, L};
    auto u = [&](int n) { return U.p[n + 1].x; };
    const int n = tstp;
    const int64_t io = ix.own(a, b, r);
    if (s.comp == 0) {
        const int64_t o = (int64_t)s.j * dd * L + io;
        const cplx w = cscal(u(-1), cscal(u(-1), X.mat_p()[o]));
        S.mat_p()[o] = cneg(cmul(G.mat_p()[o], w));   // -G^M(tau) dW^M(tau)
        return;
    }
    if (s.comp == 1 || s.comp == 2) {
        const int j = s.j;
        const GwAcc A{G.ret_p() + G.pos_ret(g, n, j) * dd * L, G.les_p() + G.pos_les(g, n, j) * dd * L, ix, j == n};
        const GwAcc C{X.ret_p() + X.pos_ret(g, n, j) * dd * L, X.les_p() + X.pos_les(g, n, j) * dd * L, ix, j == n};
        if (s.comp == 1) {
            // dW^R(n,j) = U_n chi^R U_j, dW^<(j,n) = U_j chi^< U_n, so dW^<(n,j) = U_n U_j chi^<(n,j)
            const cplx wr = cscal(u(j), cscal(u(n), C.R[io]));
            const cplx wl = C.diag ? cscal(u(n), cscal(u(j), C.Lp[io]))
                                   : cneg(cconj(cscal(u(n), cscal(u(j), C.Lp[ix.cnj(a, b, r)]))));
            const cplx wg = cadd(wr, wl);
            // Sigma^R(n,j) = i G^>(n,j) dW^>(n,j) - i G^<(n,j) dW^<(n,j)
            S.ret_p()[S.pos_ret(g, n, j) * dd * L + io] =
                csub(cmuli(cmul(A.gtr_nj(a, b, r), wg)), cmuli(cmul(A.les_nj(a, b, r), wl)));
        } else {
            const cplx wl = cscal(u(n), cscal(u(j), C.Lp[io]));
            S.les_p()[S.pos_les(g, n, j) * dd * L + io] = cmuli(cmul(A.les_jn(a, b, r), wl));   // i G^<(j,n) dW^<(j,n)
        }
        return;
    }
    const int m = s.j;
    const cplx w = cscal(u(-1), cscal(u(n), X.tv_p()[X.pos_tv(g, n, m) * dd * L + io]));
    S.tv_p()[S.pos_tv(g, n, m) * dd * L + io] = cmuli(cmul(G.tv_p()[G.pos_tv(g, n, m) * dd * L + io], w));   // i G^tv dW^tv
}

// Lattice Fourier transform along the innermost index of every element of slice tstp:
//   out(q) = scale * sum_p exp(sign * 2 pi i p q / L) in(p),  p, q = 0..L-1,
// radix-2 in shared memory for L a power of two (log2L >= 0), the direct sum otherwise
// (log2L = -1).  vpb vectors per block; dynamic shared memory holds the twiddle table
// tw[j] = exp(sign 2 pi i j / L), j < L (computed once per block: FP64 sin/cos is costly on this
// part, so no butterfly evaluates one), then the vpb * L values.  in and out are views of slice
// tstp (whole-contour store or compact buffer).
__global__ void k_kfft_slice(Grid g, int tstp, int L, int log2L, int vpb, SliceView in, SliceView out, int sign,
                             double scale) {
    extern __shared__ cplx sm_all[];
    cplx* tw = sm_all;
    cplx* sm = sm_all + L;
    const int dd = g.nf * g.nf;
    const int64_t nvec = (int64_t)slice_count(g, tstp) * dd;
    const int64_t v0 = (int64_t)blockIdx.x * vpb;
    for (int j = threadIdx.x; j < L; j += blockDim.x) {
        double sn, cs;
        sincospi((double)sign * 2.0 * (double)j / (double)L, &sn, &cs);
        tw[j] = make_double2(cs, sn);
    }
    // load (bit-reversed for the radix-2 path)
    for (int t = threadIdx.x; t < vpb * L; t += blockDim.x) {
        const int lv = t / L, p = t % L;
        const int64_t v = v0 + lv;
        if (v >= nvec) continue;
        const cplx x = in.vec(g, tstp, (int)(v / dd), (int)(v % dd), L)[p];
        const int dst = log2L > 0 ? (int)(__brev((unsigned)p) >> (32 - log2L)) : (log2L == 0 ? 0 : p);
        sm[lv * L + dst] = x;
    }
    __syncthreads();
    if (log2L >= 0) {
        for (int hs = 1, tstride = L / 2; hs < L; hs <<= 1, tstride >>= 1) {
            for (int t = threadIdx.x; t < vpb * (L / 2); t += blockDim.x) {
                const int lv = t / (L / 2), bt = t % (L / 2);
                const int j = bt % hs, blk = bt / hs;
                const int i0 = lv * L + blk * 2 * hs + j, i1 = i0 + hs;
                // exp(sign pi i j / hs) = tw[j L / (2 hs)]
                const cplx x0 = sm[i0], x1 = cmul(tw[j * tstride], sm[i1]);
                sm[i0] = cadd(x0, x1);
                sm[i1] = csub(x0, x1);
            }
            __syncthreads();
        }
        for (int t = threadIdx.x; t < vpb * L; t += blockDim.x) {
            const int lv = t / L, q = t % L;
            const int64_t v = v0 + lv;
            if (v >= nvec) continue;
            out.vec(g, tstp, (int)(v / dd), (int)(v % dd), L)[q] = cscal(scale, sm[t]);
        }
        return;
    }
    for (int t = threadIdx.x; t < vpb * L; t += blockDim.x) {
        const int lv = t / L, q = t % L;
        const int64_t v = v0 + lv;
        if (v >= nvec) continue;
        cplx acc = make_double2(0.0, 0.0);
        for (int p = 0; p < L; ++p) acc = cadd(acc, cmul(tw[(int)((int64_t)p * q % L)], sm[lv * L + p]));
        out.vec(g, tstp, (int)(v / dd), (int)(v % dd), L)[q] = cscal(scale, acc);
    }
}
