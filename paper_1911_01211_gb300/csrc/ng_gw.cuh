// GW self-energy chain on one time slice (Sec. "Self-energy approximation: GW", Eq. SigmaGW,
// Eq. dyson_chi), local and elementwise in the orbital indices; one thread per (slice element,
// a, b); every operand has ldk = 1.
//   P_ab(t,t')   = -i G_ab(t,t') G_ba(t',t)  = -Bubble1[G, G]         (Eq. def_bubble1)
//   K = -P U(t'),  K^ddagger = -U(t) P       kernel of (1 + K) * chi = P
//   dW_ab(t,t')  = U(t) chi_ab(t,t') U(t')
//   Sigma_ab     = i G_ab(t,t') dW_ab(t,t')  = Bubble2[G, dW]          (Eq. def_bubble2)
// Keldysh components by the Langreth rules for products; the Matsubara components follow from
// C^M(tau) = -i C(-i tau, 0) (Eq. matsconv): Bubble1 C^M = -A^M(tau) B^M(-tau), Bubble2
// C^M = -A^M(tau) B^M(tau).  On the diagonal j = n the equal-time lesser value is used as
// stored (no conjugate continuation), so G^<(n,n) need not be exactly anti-hermitian.
#pragma once

#include "ng_slice.cuh"

// G^<, G^> at (n,j) and (j,n) for the slice element (n,j), j <= n, from the stored triangles
struct GwAcc {
    const Comp *ret, *les;
    int64_t e;   // tri(n) + j: G^R(n,j) and G^<(j,n)
    int nf;
    bool diag;   // j == n
    __device__ __forceinline__ cplx r(int x, int y) const { return ret->p[e * nf * nf + x * nf + y]; }
    __device__ __forceinline__ cplx l(int x, int y) const { return les->p[e * nf * nf + x * nf + y]; }
    __device__ __forceinline__ cplx les_jn(int x, int y) const { return l(x, y); }
    __device__ __forceinline__ cplx les_nj(int x, int y) const { return diag ? l(x, y) : cneg(cconj(l(y, x))); }
    __device__ __forceinline__ cplx gtr_nj(int x, int y) const { return cadd(r(x, y), les_nj(x, y)); }
    __device__ __forceinline__ cplx gtr_jn(int x, int y) const { return diag ? gtr_nj(x, y) : cneg(cconj(gtr_nj(y, x))); }
};

// P, K and K^ddagger on slice tstp (-1: Matsubara) from the local fermionic G; g.sig is the
// statistics of G, P and the kernels are bosonic
__global__ void k_gw_pol(Grid g, int tstp, HermV P, HermV K, HermV Kcc, HermV G, FuncV U) {
    const int nf = g.nf, dd = nf * nf;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int cnt = slice_count(g, tstp);
    if (item >= (int64_t)cnt * dd) return;
    const int ab = (int)(item % dd), i = (int)(item / dd);
    const int a = ab / nf, b = ab % nf;
    const SliceEl s = slice_el(g, tstp, i);
    const double xi = (double)g.sig;
    auto u = [&](int n) { return U.p[n + 1].x; };
    const int n = tstp;
    cplx p;          // P_ab at this element
    double ul, ur;   // U(t) and U(t') of the element
    if (s.comp == 0) {
        const int m = s.j;
        // P^M_ab(tau) = G^M_ab(tau) G^M_ba(-tau), G^M(-tau) = xi G^M(beta - tau)
        p = cmul(G.mat.p[(int64_t)m * dd + ab], cscal(xi, G.mat.p[(int64_t)(g.ntau - m) * dd + b * nf + a]));
        ul = ur = u(-1);
    } else if (s.comp == 1 || s.comp == 2) {
        const int j = s.j;
        const GwAcc A{&G.ret, &G.les, s.e, nf, j == n};
        if (s.comp == 1) {
            // C^R_ab(n,j) = C^>_ab(n,j) - C^<_ab(n,j) with
            // C^>_ab(n,j) = i G^>_ab(n,j) G^<_ba(j,n),  C^<_ab(n,j) = i G^<_ab(n,j) G^>_ba(j,n)
            const cplx c = cmuli(csub(cmul(A.gtr_nj(a, b), A.les_jn(b, a)), cmul(A.les_nj(a, b), A.gtr_jn(b, a))));
            p = cneg(c);
            ul = u(n);
            ur = u(j);
        } else {
            // C^<_ab(j,n) = i G^<_ab(j,n) G^>_ba(n,j)
            p = cneg(cmuli(cmul(A.les_jn(a, b), A.gtr_nj(b, a))));
            ul = u(j);
            ur = u(n);
        }
    } else {
        const int m = s.j;
        const int64_t row = (int64_t)n * (g.ntau + 1);
        // C^tv_ab(n,m) = i G^tv_ab(n,m) G^vt_ba(m,n),  G^vt_ba(m,n) = -xi conj(G^tv_ab(n, ntau - m))
        const cplx gvt = cscal(-xi, cconj(G.tv.p[(row + g.ntau - m) * dd + ab]));
        p = cneg(cmuli(cmul(G.tv.p[(row + m) * dd + ab], gvt)));
        ul = u(n);
        ur = u(-1);
    }
    const int64_t o = s.e * dd + ab;
    comp_of(P, s.comp).p[o] = p;
    comp_of(K, s.comp).p[o] = cneg(cscal(ur, p));
    comp_of(Kcc, s.comp).p[o] = cneg(cscal(ul, p));
}

// Sigma on slice tstp (-1: Matsubara) from the local fermionic G and the bosonic chi:
// dW = U(t) chi U(t') formed on the fly, Sigma = Bubble2[G, dW]
__global__ void k_gw_sigma(Grid g, int tstp, HermV S, HermV G, HermV X, FuncV U) {
    const int nf = g.nf, dd = nf * nf;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int cnt = slice_count(g, tstp);
    if (item >= (int64_t)cnt * dd) return;
    const int ab = (int)(item % dd), i = (int)(item / dd);
    const int a = ab / nf, b = ab % nf;
    const SliceEl s = slice_el(g, tstp, i);
    auto u = [&](int n) { return U.p[n + 1].x; };
    const int n = tstp;
    const int64_t o = s.e * dd + ab;
    if (s.comp == 0) {
        const cplx w = cscal(u(-1), cscal(u(-1), X.mat.p[o]));
        S.mat.p[o] = cneg(cmul(G.mat.p[o], w));   // -G^M(tau) dW^M(tau)
        return;
    }
    if (s.comp == 1 || s.comp == 2) {
        const int j = s.j;
        const GwAcc A{&G.ret, &G.les, s.e, nf, j == n};
        const GwAcc C{&X.ret, &X.les, s.e, nf, j == n};
        if (s.comp == 1) {
            // dW^R(n,j) = U_n chi^R U_j, dW^<(j,n) = U_j chi^< U_n, so dW^<(n,j) = U_n U_j chi^<(n,j)
            const cplx wr = cscal(u(j), cscal(u(n), C.r(a, b)));
            const cplx wl = C.diag ? cscal(u(n), cscal(u(j), C.l(a, b))) : cneg(cconj(cscal(u(n), cscal(u(j), C.l(b, a)))));
            const cplx wg = cadd(wr, wl);
            // Sigma^R(n,j) = i G^>(n,j) dW^>(n,j) - i G^<(n,j) dW^<(n,j)
            S.ret.p[o] = csub(cmuli(cmul(A.gtr_nj(a, b), wg)), cmuli(cmul(A.les_nj(a, b), wl)));
        } else {
            const cplx wl = cscal(u(n), cscal(u(j), C.l(a, b)));
            S.les.p[o] = cmuli(cmul(A.les_jn(a, b), wl));   // i G^<(j,n) dW^<(j,n)
        }
        return;
    }
    const cplx w = cscal(u(-1), cscal(u(n), X.tv.p[o]));
    S.tv.p[o] = cmuli(cmul(G.tv.p[o], w));   // i G^tv(n,m) dW^tv(n,m)
}
