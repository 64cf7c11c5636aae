/*
 * ng.h -- C ABI of the GB300 contour Dyson time-stepper (libng.so).
 *
 * The library solves the Dyson equation in integro-differential form on the L-shaped
 * Kadanoff-Baym contour, i d/dt G - eps(t) G - Sigma * G = delta_C (paper Eq. dyson),
 * for a batch of problems (k-points or independent embedded clusters) with the k-th order
 * BDF/Gregory scheme of the paper (Sec. "Numerical details: Volterra integral equations",
 * Sec. "Implementation: dyson"), and evaluates the second-Born self-energy that couples
 * the batch through the local Green's function (Eq. sigma_hubb_2b).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - C linkage; every call returns ng_status and never throws, aborts or exits.
 *  - Statistics: grid.sig = -1 (fermions); the vie2 and convolution calls also take bosonic
 *    functions (grid.sig = +1, every operand of the call bosonic).  Orders korder = 1..5.
 *  - All contour data are caller-owned DEVICE buffers of complex128 stored as interleaved
 *    (re, im) double pairs.  The library never frees caller memory.
 *  - A contour function (struct ng_herm) holds the minimal component set of the paper's
 *    herm_matrix (Eq. storage_herm) for nbatch problems, problem index innermost:
 *        mat[m][a][b][kb]             m = 0..ntau                   C^M(m h_tau)
 *        ret[tri(n)+j][a][b][kb]      0 <= j <= n <= nt             C^R(n h, j h)
 *        les[tri(n)+j][a][b][kb]      0 <= j <= n <= nt             C^<(j h, n h)
 *        tv [n*(ntau+1)+m][a][b][kb]  n = 0..nt, m = 0..ntau         C^tv(n h, m h_tau)
 *    with tri(n) = n(n+1)/2, a, b = 0..nf-1 orbital indices and kb = 0..ldk-1.
 *    ldk is nbatch for per-problem data, or 1 for data shared by the whole batch
 *    (e.g. a local self-energy Sigma_loc).  Problem kb of a shared function is kb = 0.
 *  - A single-time contour function (struct ng_func) stores f_n, n = -1..nt,
 *    as val[n+1][a][b][kb] (f_{-1} = f(0^-), paper Sec. "Numerical representation").
 *  - The real-time grid is t_n = n h, the imaginary-time grid tau_m = m beta/ntau.
 *    The chemical potential mu enters as eps - mu.
 *  - stream is a cudaStream_t passed as void*; NULL is the legacy default stream.
 *    Every compute entry point is asynchronous and stream-ordered unless stated.
 *  - Argument errors are detected on the host before any launch and return NG_EINVAL
 *    (the text is available from ng_last_error).  Device-side conditions (non-finite
 *    values, a singular per-step matrix) set bits in a device status word that
 *    ng_status_sync reads back.
 *  - Preconditions follow the paper's Table tab:dyson: a call at time step tstp reads
 *    slices < tstp of G and slices <= tstp of Sigma and eps.
 *  - Thread safety: one context per host thread.  A context may be used with several
 *    streams, but calls that share its workspaces (ng_dyson_mat, ng_dyson_start,
 *    ng_distance_timestep, ng_dyson_timestep with nf = 4, 8 or a non-FP64 precision,
 *    ng_run_2b, ng_batch_*, ng_adjoint_2b) must not overlap on the device.
 */
#ifndef NG_H
#define NG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NG_OK = 0,
    NG_EINVAL = 1,        /* invalid argument (host-side check, nothing launched)        */
    NG_ENOMEM = 2,        /* workspace allocation failed                                 */
    NG_ECUDA = 3,         /* a CUDA runtime call failed                                  */
    NG_ENOCONV = 4,       /* a self-consistency loop hit its iteration limit             */
    NG_ETIMEOUT = 5,      /* reserved: a bounded device wait gave up                     */
    NG_ENONFINITE = 6,    /* a non-finite value was produced (device status word)        */
    NG_EUNSUPPORTED = 7,  /* valid but not implemented here (e.g. NG_F32C with nf > 2)    */
    NG_ESCRATCH = 8,      /* the problem needs more than the fixed static scratch of the  */
                          /* allocation-free entry point (nothing launched)              */
    NG_ECOMM = 9,         /* the caller's rank-exchange callback reported a failure       */
    NG_ESINGULAR = 10     /* a per-step or Matsubara matrix was singular (device status)  */
} ng_status;

/* device status word bits (ng_status_sync) */
#define NG_FLAG_NONFINITE 1
#define NG_FLAG_SINGULAR 2

typedef struct ng_ctx ng_ctx;

typedef struct {
    int nt;        /* number of real-time steps N_t (slices 0..nt)                       */
    int ntau;      /* number of imaginary-time intervals N_tau (points 0..ntau)            */
    int nf;        /* orbital dimension d: 1, 2, 4 or 8                                     */
    int nbatch;    /* number of problems stored innermost                                   */
    int korder;    /* solve order k, 1..5; requires nt >= 2k+2 and ntau >= 2k+2             */
    int sig;       /* -1: fermions (only value accepted)                                    */
    double h;      /* real-time step                                                        */
    double beta;   /* inverse temperature                                                   */
    double mu;     /* chemical potential                                                    */
} ng_grid;

typedef struct {
    void *mat, *ret, *les, *tv;  /* device pointers, complex128, layout above          */
    int ldk;                     /* nbatch (per problem) or 1 (shared by the batch)     */
} ng_herm;

typedef struct {
    void *val;                   /* device pointer, complex128 [nt+2][nf][nf][ldk]      */
    int ldk;                     /* nbatch or 1                                          */
} ng_func;

/* NG_FP64: every sum in FP64.  NG_F32C: the O(n) and O(ntau) history and source sums of the
 * time step read FP32 copies of the history and accumulate exact FP32 products with Kahan
 * compensation (rounded once to FP64); BDF terms, the per-step matrix inverses, the (A)
 * boundary steps, the start-up and the Matsubara solve stay FP64.  NG_DF64: the same sums in
 * double-float arithmetic (each value an FP32 pair, 48 significand bits; products with their
 * cross terms, TwoSum accumulation), FP64-class accuracy on the FP32 pipes. */
typedef enum { NG_FP64 = 0, NG_F32C = 1, NG_DF64 = 2 } ng_precision;

/* Evaluation of the left-mixing Matsubara source -i (C^tv_2 + C^tv_3)[Sigma, 1, G^M](n, tau_m) of
 * a time step (Eqs. ctv2, ctv3), set per context with ng_set_tv_source.  NG_TVSRC_DIRECT: the
 * quadrature sums as written, O(ntau^2) complex multiply-adds per problem and step.
 * NG_TVSRC_AUTO (default): the unit-weight part of both pieces is one correlation over tau,
 * evaluated for all tau_m by an FP64 FFT of length L (the power of two >= 2 ntau + 1; one
 * block per problem, transforms in shared memory), and the time-step kernels add the O(k)
 * Gregory end and boundary (R) corrections per element; used for nf = 1, 2 when the transforms
 * fit the shared memory (nf = 1: ntau <= 2047, nf = 2: ntau <= 511), the direct sums otherwise.
 * Both evaluate the same quadrature; they differ by rounding only. */
typedef enum { NG_TVSRC_AUTO = 0, NG_TVSRC_DIRECT = 1 } ng_tv_source;

/* Parallel decomposition of the FP64 time step (ng_set_bulk_split): NG_BULK_THREAD, one thread
 * per (column, problem) bulk item and one block per problem for the boundary; NG_BULK_WARP,
 * one warp per bulk item, its history and source sums (the left-mixing source by its direct
 * quadrature, no FFT pre-pass) split over the 32 lanes and added in a fixed butterfly order
 * that leaves one element of the nf x nf result per lane for the closing solve, the
 * boundary's (A)-row sums spread over (row, problem, chunk) blocks added in chunk order, and
 * the boundary's retarded start-up run by extra warps of the bulk launch (small batches: a
 * dimer, a real-space cluster); NG_BULK_AUTO (default), each warp/spread form when the batch
 * has fewer than 128 bulk items per SM, resp. fewer than 2 boundary rows per SM.  In every
 * mode the boundary's dense solves and serial steps run on one warp per problem.  The forms
 * differ by the order of additions only.  nf = 4, 8 always run the element-wise form. */
typedef enum { NG_BULK_AUTO = 0, NG_BULK_THREAD = 1, NG_BULK_WARP = 2 } ng_bulk_split;

/* Schedule of a time step (Sec. "Time stepping"): NG_MIXED is the paper's parallel variant
 * (implementation (B) for the bulk of the retarded row and lesser column, (A) near the
 * diagonal); NG_SERIAL is its serial variant, implementation (A) along the whole retarded row
 * (conjugate VIDE) and the whole lesser column.  The two agree to discretisation level. */
typedef enum { NG_MIXED = 0, NG_SERIAL = 1 } ng_schedule;

/* Parameters of the self-consistent second-Born driver (ng_run_2b). */
typedef struct {
    int corrector;       /* corrector iterations per time step (paper: CorrectorSteps)   */
    double mats_tol;     /* Matsubara loop stops when the G^M distance is below this     */
    int mats_maxiter;
    double boot_tol;     /* bootstrapping stops when the distance of slices 0..k is below */
    int boot_maxiter;    /* this and more than two iterations were made                   */
    double nbar;         /* Hartree reference filling (1/2 at half filling)               */
    int n_from;          /* first time step to propagate (k+1 for a full run)             */
    int n_to;            /* last time step to propagate (<= nt)                            */
    int do_setup;        /* 1: run the Matsubara loop and bootstrapping first              */
    int precision;       /* ng_precision of the time steps                                   */
} ng_run_params;

/* ---- context ------------------------------------------------------------------------ */

/* Create a context for solve order korder (1..5) on CUDA device `device`.  The context
 * owns the integration weights (exact rationals rounded to FP64: Sec. "Basic integration
 * and differentiation rules"), device workspaces and the device status word.
 * *out receives the context; NG_EINVAL for a bad order, NG_ECUDA if the device fails. */
ng_status ng_create(int korder, int device, ng_ctx **out);

/* Release a context and its workspaces (synchronises the device first). NULL is a no-op. */
void ng_destroy(ng_ctx *ctx);

/* Text of the last error recorded on ctx (static storage owned by ctx; never NULL). */
const char *ng_last_error(const ng_ctx *ctx);

/* Synchronise `stream`, read and clear the device status word (NG_FLAG_* bits) into
 * *device_flags.  Returns NG_ENONFINITE if NG_FLAG_NONFINITE was set, else NG_ESINGULAR if
 * NG_FLAG_SINGULAR was set (a pivot of a per-step, start-up or Matsubara solve was zero; the
 * affected values are not finite or not meaningful), NG_OK otherwise. */
ng_status ng_status_sync(ng_ctx *ctx, void *stream, int *device_flags);

/* Host copy of the FP64 integration weights for the context's order k, for inspection:
 * out[0..k] = BDF a_j (Eq. integrator_bd); out[6..6+k] = Gregory end weights omega_j
 * (Eq. integrator_greg); out[12..12+k] = extrapolation C_l (Eq. polyextrap).
 * `out` must hold 18 doubles. */
ng_status ng_weights(const ng_ctx *ctx, double *out);

/* ---- inputs ------------------------------------------------------------------------- */

/* Free Green's function of a constant hermitian Hamiltonian for every problem, all
 * components, times `scale` (Sec. "Implementation: Free Green's functions", Eq. G0_free,
 * exact for constant eps).  eps_host: host array [nbatch][nf][nf] complex128 (interleaved).
 * G must have ldk = nbatch.  Use scale = V^2 with nf = 1 for an embedding self-energy
 * Sigma = V^2 g0 (Sec. "Test of accuracy and scaling analysis"). */
ng_status ng_green_from_H_const(ng_ctx *ctx, const ng_grid *grid, ng_herm G,
                                const double *eps_host, double scale, void *stream);

/* ---- Dyson solver (Table tab:dyson) ------------------------------------------------- */

/* Matsubara slice T[G]_{-1} for every problem: the exact root of the k-th order
 * discretised integral equation G^M = g^M + [g^M * Sigma^M * G^M]^M
 * (Sec. "Matsubara", Eq. Gmat_dyson_integ, convolutions Eqs. cm1/cm2), found by a dense
 * LU solve per problem.  Reads Sigma.mat, eps at n = -1; writes G.mat.
 * Workspace: 16 (ntau+1)^2 nf^2 nbatch bytes, allocated on first use. */
ng_status ng_dyson_mat(ng_ctx *ctx, const ng_grid *grid, ng_herm G, ng_herm Sigma,
                       ng_func eps, void *stream);

/* Start-up slices T[G]_n, n = 0..k (Sec. "Start", Eq. vdiff_start): retarded column
 * systems, left-mixing and lesser VIDE start-up.  Reads G.mat and Sigma, eps on
 * slices -1..k; writes slices 0..k of G. */
ng_status ng_dyson_start(ng_ctx *ctx, const ng_grid *grid, ng_herm G, ng_herm Sigma,
                         ng_func eps, void *stream);

/* Time step tstp > k (Sec. "Time stepping"), the paper's parallel (mixed) schedule:
 * retarded row by single VIDE steps for columns m <= tstp-k-1 (implementation (B)) and the
 * conjugate start-up for m = tstp-k..tstp (implementation (A)); left-mixing row by one VIDE
 * step per tau_m; lesser column by conjugate single steps for 1 <= m <= tstp-k-1 (B) and
 * serial VIDE steps (A) for m >= tstp-k (the whole column by (A) when tstp <= 2k).
 * Reads slices < tstp of G, slices <= tstp of Sigma and eps; writes slice tstp of G.
 * precision: NG_FP64, NG_F32C or NG_DF64 (the last two for nf <= 2; NG_DF64 keeps 16-byte
 * double-float copies, otherwise as NG_F32C).  With NG_F32C the context keeps FP32 copies of G (ldk =
 * nbatch) and Sigma: slices < tstp are converted once when tstp first reaches them, Sigma's
 * slice tstp on every call.  Call ng_precision_reset after changing slices < tstp of G or
 * Sigma in place (the copies are also rebuilt when the buffers or the grid change).
 * Workspace: 8 bytes per complex element of G and Sigma.
 * schedule: NG_MIXED (above) or NG_SERIAL (the retarded row by the conjugate VIDE start-up and
 * steps along the whole row, the lesser column by the VIDE start-up and steps along the whole
 * column, each step's sums as block reductions, one block per problem; NG_FP64 and nf <= 2 only,
 * NG_EUNSUPPORTED otherwise). */
ng_status ng_dyson_timestep(ng_ctx *ctx, const ng_grid *grid, int tstp, ng_herm G,
                            ng_herm Sigma, ng_func eps, int precision, int schedule, void *stream);

/* Allocation-free start-up: the same computation as ng_dyson_start, for callers that must
 * not allocate device memory.  Examples: a host application whose caching allocator already
 * owns all free device memory (a cudaMalloc would fail, or fragment that pool); a latency-
 * critical loop that cannot afford cudaFree's implicit device synchronisation; a plug-in
 * whose host forbids libraries from managing device memory.  The paper has no counterpart to
 * this entry point.
 *  - No context is needed and none is created.  The start-up workspace (the inverted
 *    (k nf)^2 start-up matrix and k blocks of nf x nf per problem) lives in one file-scope
 *    static device array of NG_NOALLOC_SCRATCH_BYTES = 2 MiB, which every GPU that loads the
 *    library holds until the process exits; its first 256 bytes hold a status word.
 *  - Size limit: the call needs 256 + 16 nbatch ((k nf)^2 + k nf^2) bytes and returns
 *    NG_ESCRATCH, launching nothing, above 2 MiB (at k = 5: at most 4369 problems with nf = 1,
 *    1092 with nf = 2, 273 with nf = 4, 68 with nf = 8).  Other argument errors return
 *    NG_EINVAL / NG_EUNSUPPORTED.
 *  - It calls no cudaMalloc, cudaFree or allocating library routine.
 *  - The first call on a device does one-time set-up with that device current: it copies the
 *    integration weights to the constant memory of every part of the library (unless ng_create
 *    already did on that device), so contexts created later on that device need no copy of
 *    their own, and looks up the array's device address with cudaGetSymbolAddress.  Make that first call from
 *    one host thread, before any stream capture.
 *  - Every call uses the same array and leaves its contents there; the status word is cleared
 *    at the start of each call, and everything else is written before it is read.  Calls whose
 *    work overlaps on the GPU (different streams, or concurrent host threads) race on the
 *    array: serialise them.
 *  - Device-side flags (non-finite values, a singular start-up matrix) land in the array's
 *    status word and are not reported.
 * Arguments as for ng_dyson_start (G with ldk = nbatch; Sigma and eps with ldk = 1 or
 * nbatch); runs on the device that is current when it is called, stream-ordered on `stream`. */
ng_status ng_dyson_start_noalloc(const ng_grid *grid, ng_herm G, ng_herm Sigma, ng_func eps, void *stream);

/* Choose the decomposition of the FP64 time-step bulk (and of the vie2 time step) on ctx
 * (ng_bulk_split). */
ng_status ng_set_bulk_split(ng_ctx *ctx, int mode);

/* Choose the evaluation of the left-mixing source for later time steps on ctx (ng_tv_source). */
ng_status ng_set_tv_source(ng_ctx *ctx, int mode);

/* Forget the FP32 copies kept for NG_F32C time steps (they are rebuilt on the next call). */
ng_status ng_precision_reset(ng_ctx *ctx);

/* ---- Dyson equation in integral form (Table tab:vie2) --------------------------------- */

/* (1 + F) * G = Q (Sec. "vie2: Dyson equation in integral form", Eq. vie2), solved with the
 * k-th order rules of Sec. "Implementation: vie2" (Volterra integral equations of the second
 * kind, Eqs. MBCVSAMx01_start, MBCVSAMx01_t and the conjugate Eq. MBCVSAMx01_cc)t).  F is a
 * given kernel, Fcc = F^ddagger its hermitian partner (the values of F outside the stored
 * triangles; pass F itself when F is hermitian symmetric), Q a hermitian source; G is hermitian
 * when F * Q = Q * F^ddagger (Eq. ,masbX,.), e.g. F = -G0 * Sigma, Fcc = -Sigma * G0, Q = G0 for
 * the Dyson series.  G: ldk = nbatch; F, Fcc, Q: ldk 1 or nbatch.  nf = 1, 2, 4
 * (NG_EUNSUPPORTED otherwise; nf = 4 keeps its 4 x 4 blocks per thread and is meant for small
 * batches such as a real-space cluster).  grid.sig = +1 solves for bosonic functions (e.g. the susceptibility of Eq.
 * dyson_chi).  Preconditions follow Table tab:vie2. */

/* Matsubara slice: the k-th order discretised G^M + [F * G]^M = Q^M (Eqs. cm1, cm2), solved
 * exactly by a dense LU per problem.  Reads F.mat, Q.mat; writes G.mat.  Workspace as
 * ng_dyson_mat. */
ng_status ng_vie2_mat(ng_ctx *ctx, const ng_grid *grid, ng_herm G, ng_herm F, ng_herm Q, void *stream);

/* Start-up slices 0..k: retarded column systems, left-mixing and lesser VIE start-up (initial
 * values Eqs. vie2_ini_r/_tv/_les).  Reads G.mat and F, Fcc, Q on slices -1..k. */
ng_status ng_vie2_start(ng_ctx *ctx, const ng_grid *grid, ng_herm G, ng_herm F, ng_herm Fcc, ng_herm Q,
                        void *stream);

/* Time step tstp > k: G^R(n,n) = Q^R(n,n) and single steps for every retarded element m < n;
 * one step per tau_m of the left-mixing row (source Q^tv - (C^tv_2 + C^tv_3)[F, 1, G^M]); the
 * lesser column by the conjugate equation G * (1 + F^ddagger) = Q (implementation (B): kernel
 * [F^R(n,l)]^dagger, source Q^< - (C^<_1 + C^<_3)[G, 1, F^ddagger]) for m = 1..n-1, G^<(0,n)
 * from Eq. vie2_ini_les, then m = n.  Reads slices < tstp of G, slices <= tstp of F, Fcc, Q.
 * schedule: NG_MIXED only (NG_SERIAL returns NG_EUNSUPPORTED). */
ng_status ng_vie2_timestep(ng_ctx *ctx, const ng_grid *grid, int tstp, ng_herm G, ng_herm F, ng_herm Fcc,
                           ng_herm Q, int schedule, void *stream);

/* ---- convolution (Table tab:convolution) ---------------------------------------------- */

/* Time slice tstp of the contour convolution C = A * f * B (Sec. "Numerical details:
 * convolution integrals on C", Eqs. cm1, cm2, cr1, ctv1-ctv3, cles1-cles3; Sec. "Implementation:
 * convolution"), with the k-th order Gregory and boundary (R) quadratures of the context:
 *   tstp = -1: C^M(tau_m), m = 0..ntau;
 *   tstp >= 0: C^R(tstp, m) for m <= tstp, C^tv(tstp, m) for m = 0..ntau and C^<(m, tstp) for
 *              m <= tstp.
 * Acc and Bcc are the hermitian conjugates A^ddagger and B^ddagger, which supply the values
 * outside the stored triangles (Eq. hermconjg); pass A itself when A is hermitian symmetric.
 * f is a single-time function (f_{-1} enters the Matsubara and mixed pieces); f.val = NULL is
 * the identity.  Reads slices 0..max(tstp, k) of A, Acc, B, Bcc and f (the start-up quadrature
 * of tstp <= k uses slices up to k), writes slice tstp of C only.  C.ldk = nbatch (inputs with
 * ldk 1 or nbatch) or C.ldk = 1 with every input shared.  nf = 1, 2, 4, 8. */
ng_status ng_convolution_timestep(ng_ctx *ctx, const ng_grid *grid, int tstp, ng_herm C, ng_herm A, ng_herm Acc,
                                  ng_func f, ng_herm B, ng_herm Bcc, void *stream);

/* ---- slice operations ----------------------------------------------------------------- */

/* Local Green's function slice tstp (-1 = Matsubara): Gloc = sum_kb w_kb Gk_kb
 * (Sec. "GW for the translationally invariant Hubbard model", get_loc), w_kb = 1/nbatch when
 * wk is NULL, else wk = device array of nbatch doubles (k-point weights).  Deterministic, in a
 * fixed order that does not depend on a split of the k-points over ranks: the k axis is cut
 * into blocks of 32 consecutive indices, each block's weighted values are summed in a fixed
 * butterfly order, the block sums are added in block order, the 1/nbatch factor comes last.
 * Gloc must have ldk = 1, Gk ldk = nbatch. */
ng_status ng_kreduce_timestep(ng_ctx *ctx, const ng_grid *grid, int tstp, ng_herm Gloc,
                              ng_herm Gk, const double *wk, void *stream);

/* ---- k-point sharding over ranks (Sec. "MPI parallelization", Eq. dyson_kspace) --------
 * nk k-points are split over nranks ranks (one GPU each) in whole blocks of 32: with
 * B = ceil(nk / 32) blocks, rank r owns blocks [floor(r B / nranks), floor((r+1) B / nranks)),
 * i.e. the k indices k_begin .. k_begin + k_count - 1.  Each rank keeps the G_k of its own
 * k-points and a full copy of the shared Gloc and Sigma.  The only exchange is an allgather of
 * every rank's 32-block sums of the slice being reduced (at most 2 (nt+1) + ntau + 1 elements
 * of nf^2 complex values per block); adding them in block order on every rank gives bitwise the
 * single-GPU ng_kreduce_timestep result, so every rank computes the same Sigma. */

/* The share of rank `rank`: *k_begin, *k_count (may be NULL) and *send_bytes (may be NULL;
 * needs grid for nt, ntau, nf), the size of the per-rank exchange buffer.  Host only, no
 * device access.  NG_EINVAL if nranks exceeds 64 or the number of blocks. */
ng_status ng_shard_plan(int nk, int rank, int nranks, const ng_grid *grid, int *k_begin, int *k_count,
                        size_t *send_bytes);

/* Block sums of slice tstp over the local problems of Gk (ldk = nbatch = the local count), whose
 * global k indices start at k_begin (a multiple of 32): partial[(bl cnt + i) nf^2 + a nf + b]
 * (complex128) for the local blocks bl and the slice elements i in the order ret row, les column,
 * tv row (tstp >= 0; cnt = 2 (tstp+1) + ntau + 1) or mat (tstp = -1; cnt = ntau + 1).  wk: device
 * weights of the local problems, or NULL (the 1/nk factor is then applied by the combine). */
ng_status ng_kreduce_partial(ng_ctx *ctx, const ng_grid *grid, int tstp, void *partial, ng_herm Gk,
                             const double *wk, int k_begin, void *stream);

/* Gloc slice tstp from every rank's block sums: gathered is rank-major, each rank's chunk the
 * maxb-block send buffer of ng_kreduce_partial (maxb = the largest block count of a rank; rows
 * beyond a rank's own blocks are ignored).  weighted = 0 multiplies by 1/nk (no weights were
 * given to the partials), 1 takes the sum as it is.  Gloc: ldk = 1. */
ng_status ng_kreduce_combine(ng_ctx *ctx, const ng_grid *grid, int tstp, ng_herm Gloc, const void *gathered, int nk,
                             int nranks, int weighted, void *stream);

/* Rank-exchange description for ng_run_2b_sharded.  send and recv are caller-owned device
 * buffers of send_bytes (>= the ng_shard_plan value) and nranks * send_bytes.  exchange(user,
 * bytes) must allgather: after it returns, recv[r * bytes .. (r+1) * bytes) holds rank r's first
 * `bytes` of send for every r, ordered on the run's stream (an NCCL or torch.distributed
 * allgather issued on that stream does this); it returns 0 on success.  The driver calls it once
 * per k-reduction (the block sums) and once per convergence check of the setup loops (one
 * double, the rank's distance; the ranks' values are summed in rank order). */
typedef struct {
    int nk;                                       /* k-points over all ranks                */
    int rank, nranks;                             /* this rank, number of ranks (<= 64)      */
    void *send;                                   /* device, send_bytes                      */
    size_t send_bytes;
    void *recv;                                   /* device, nranks * send_bytes             */
    int (*exchange)(void *user, size_t bytes);    /* allgather of `bytes` per rank           */
    void *user;
} ng_shard;

/* Second-Born self-energy slice tstp (-1 = Matsubara) from a local G (Eq. sigma_hubb_2b):
 * Sigma_ab(t,t') = U(t)U(t') G_ab(t,t')^2 G_ba(t',t), components by the Langreth product
 * rules (Eqs. def_bubble1/2); Sigma^M(tau) = -U_{-1}^2 G^M(tau)^2 G^M(-tau).
 * U: scalar single-time function (nf = 1 layout, ldk = 1).  Sigma and G share ldk = 1. */
ng_status ng_sigma2b_timestep(ng_ctx *ctx, const ng_grid *grid, int tstp, ng_herm Sigma,
                              ng_herm Gloc, ng_func U, void *stream);

/* Hartree mean field (Sec. "Hubbard chain"): eps_mf_kb(n) = eps0_kb(n)
 * + U_n diag(Re rho_ii - nbar), rho = -i Gloc^<(n,n) (n >= 0) or -Gloc^M(beta^-) (n = -1).
 * eps_mf and eps0 have ldk = nbatch (or both 1); Gloc ldk = 1. */
ng_status ng_hartree_timestep(ng_ctx *ctx, const ng_grid *grid, int tstp, ng_func eps_mf,
                              ng_func eps0, ng_herm Gloc, ng_func U, double nbar,
                              void *stream);

/* Predictor: fill slice tstp+1 of G from slices tstp-k..tstp by polynomial extrapolation
 * (Appendix "Extrapolation of contour functions", Eq. polyextrap).  Requires tstp >= k. */
ng_status ng_extrapolate_timestep(ng_ctx *ctx, const ng_grid *grid, int tstp, ng_herm G,
                                  void *stream);

/* out_dev[0] += sum over problems of ||A - B||_tstp (Eq. distancenorm; tstp = -1:
 * Matsubara).  out_dev is a device double the caller zeroes; A and B have equal ldk. */
ng_status ng_distance_timestep(ng_ctx *ctx, const ng_grid *grid, int tstp, ng_herm A,
                               ng_herm B, double *out_dev, void *stream);

/* Observables of time slice tstp (0..nt), averaged over the batch (per spin):
 * out_dev[0] = N = Tr rho, rho(t) = -i G^<(t,t) (Sec. "Hubbard chain", density_matrix);
 * out_dev[1] = E_kin = Tr[rho eps0(t)] (k-space kinetic energy);
 * out_dev[2] = E_mf = 1/2 Tr[rho (eps_mf(t) - eps0(t))] (Hartree part);
 * out_dev[3] = E_corr = 1/2 Im Tr[Sigma * G]^<(t,t) from C^<_1 + C^<_2 + C^<_3 (Eqs. cles1-3);
 * out_dev[4] = E_kin + E_mf + E_corr, the Galitskii-Migdal total energy (Eq. Total_ener).
 * G: ldk = nbatch; Sigma: ldk 1 or nbatch; eps0, eps_mf: ldk nbatch (or 1).  out_dev is a
 * device array of 5 doubles.  Deterministic (fixed-order batch sum).  Workspace 40 nbatch bytes. */
ng_status ng_observables(ng_ctx *ctx, const ng_grid *grid, int tstp, ng_herm G, ng_herm Sigma, ng_func eps0,
                         ng_func eps_mf, double *out_dev, void *stream);

/* ---- uneven batch of independent problems ---------------------------------------------- */

/* Out(t,t') = V In(t,t') V^dagger for every component and element (one problem each,
 * nbatch = 1, ldk = 1): the embedding self-energy Sigma = V g_bath V^dagger of a cluster coupled
 * to a bath (Sec. "Test of accuracy and scaling analysis", downfolding).  V_host: host array
 * [nf_out][nf_in] complex128.  Grids must agree in nt and ntau. */
ng_status ng_herm_sandwich(ng_ctx *ctx, const ng_grid *grid_out, ng_herm Out, const ng_grid *grid_in, ng_herm In,
                           const double *V_host, void *stream);

/* A batch of nprob independent problems with their own grids (nf in {1, 2, 4, 8}, nt, ntau,
 * beta, h may all differ; korder equal to the context's; nbatch = 1 each) and fixed
 * self-energies.  G[p], Sigma[p] (ldk = 1) and eps[p] are caller-owned device buffers in the
 * layout of this header.  The batch owns a small device table (allocated here). */
typedef struct ng_batch ng_batch;
ng_status ng_batch_create(ng_ctx *ctx, int nprob, const ng_grid *grids, const ng_herm *G, const ng_herm *Sigma,
                          const ng_func *eps, ng_batch **out);
void ng_batch_destroy(ng_batch *batch);

/* Matsubara solve and start-up of every problem (as ng_dyson_mat, ng_dyson_start). */
ng_status ng_batch_setup(ng_ctx *ctx, ng_batch *batch, void *stream);

/* Global time step n for every problem with k < n <= nt_p: one launch computes M_n^-1 of all
 * active problems, one launch the bulk items of all of them (orbital-element-wise: one thread
 * per (item, a, b), mixed schedule of ng_dyson_timestep), one launch their boundaries.
 * threads: block size of the bulk launch, 64, 128 or 256 (0: the tuned or default value). */
ng_status ng_batch_step(ng_ctx *ctx, ng_batch *batch, int n, int threads, void *stream);

/* Setup, then every global time step until each problem reaches its nt.  The bulk block size
 * is tuned by timing each candidate on a re-run of one representative step (a step is
 * idempotent), once per batch shape and context: the context keeps the choice for batches with
 * the same number of problems of each nf, the same largest ntau and the same largest nt (in
 * steps of 256) and reuses it without timing.  *tuned_threads (may be NULL) receives it. */
ng_status ng_batch_solve(ng_ctx *ctx, ng_batch *batch, int *tuned_threads, void *stream);

/* ---- measurement ---------------------------------------------------------------------- */

/* Start (enable = 1, clearing any previous record) or stop (enable = 0) per-launch timing of
 * the time-step kernels of ng_dyson_timestep: CUDA events are recorded on the launching
 * stream around every launch of the merged bulk kernel, of the boundary kernel and of the FFT
 * pre-pass of the left-mixing source. */
ng_status ng_profile_enable(ng_ctx *ctx, int enable);

/* Read the record (synchronises on the last recorded event).  out[0] = total bulk-kernel
 * time in ms, out[1] = number of bulk launches, out[2] = algorithmic FP64 flops of those
 * launches (8 real flops per complex multiply-add of the history and source sums, nf^3
 * complex multiply-adds per d x d block product; with the FFT source, its quadrature
 * corrections in place of the O(ntau^2) sums), out[3] = total boundary-kernel time in ms,
 * out[4] = number of boundary launches, out[5] = total time of the FFT source pre-pass in ms,
 * out[6] = its launches, out[7] = total time of the GW self-energy evaluations of ng_run_gw /
 * ng_run_gw_kspace in ms (bubbles, lattice transforms and the chi solve), out[8] = their
 * number.  `out` must hold 9 doubles. */
ng_status ng_profile_read(ng_ctx *ctx, double *out);

/* FP64 throughput of the current device, for the roofline of the FP64 kernels: out[0] = the
 * sustained FP64 FMA-pipe rate (DFMA, 8 independent chains per thread, 8 blocks of 256 threads
 * per SM) and out[1] = the FP64 tensor rate (DMMA, mma.sync m8n8k4 f64, 4 independent
 * accumulators per warp), both in TFLOP/s (2 flop per multiply-add), out[2] = the SM count.
 * Synchronises `stream`; takes about a second (a warm-up, then the best of three timed launches
 * of each kernel).  `out` must hold 3 doubles. */
ng_status ng_fp64_probe(double *out, void *stream);

/* ---- driver --------------------------------------------------------------------------- */

/* Self-consistent second-Born run for a batch of problems coupled through
 * Gloc = (1/nbatch) sum_kb G_kb (Sec. "Hubbard chain" program structure):
 *  setup (if p->do_setup): Matsubara loop {Gloc, Hartree, Sigma^M, dyson_mat} to
 *  p->mats_tol; bootstrapping {Gloc, Hartree, Sigma on slices 0..k, dyson_start} to
 *  p->boot_tol with more than two iterations;
 *  stepping for n = p->n_from..p->n_to: extrapolate slice n, then p->corrector iterations of
 *  {Gloc(n), Hartree(n), Sigma(n), dyson_timestep(n)}.
 * G: ldk = nbatch; Gloc, Sigma: ldk = 1; eps0, eps_mf: ldk = nbatch; U: ldk = 1 scalar.
 * Host-synchronous in the setup loops (convergence checks), asynchronous in the stepping.
 * Returns NG_ENOCONV if a setup loop hit its iteration limit (results are still written).
 * iters_out (host, may be NULL) receives {Matsubara iterations, bootstrap iterations}. */
ng_status ng_run_2b(ng_ctx *ctx, const ng_grid *grid, ng_herm G, ng_herm Gloc, ng_herm Sigma,
                    ng_func eps0, ng_func eps_mf, ng_func U, const ng_run_params *p,
                    int *iters_out, void *stream);

/* ng_run_2b with its inputs and outputs in host memory, for callers that keep them there:
 * eps0_host (complex128, the layout of eps0: [nt+2][nf][nf][nbatch], index n+1 for t_n) is copied
 * into the device eps0 slice by slice as the run reaches it (slices -1..k with the setup, slice n
 * before step n), U_host (complex128 [nt+2]) into U once at the start, and after every step n
 * (and after the bootstrapping for n = 0..k) Gloc^<(t_n, t_n) as the last corrector pass reduced
 * it (before that pass's Dyson step) is copied to gdiag_host (complex128 [nt+1][nf][nf]; the
 * local density matrix is -i times it).  All copies are
 * stream-ordered cudaMemcpyAsync calls on `stream`; page-locked host buffers keep them
 * asynchronous (pageable ones make every copy wait).  The host buffers must stay valid until
 * the stream has passed the run.  shard: NULL for all k-points on this GPU, else this rank's
 * share as in ng_run_2b_sharded (eps0_host then holds the rank's own k-points).  Otherwise as
 * ng_run_2b; eps0.ldk must be nbatch. */
ng_status ng_run_2b_host(ng_ctx *ctx, const ng_grid *grid, ng_herm G, ng_herm Gloc, ng_herm Sigma, ng_func eps0,
                         ng_func eps_mf, ng_func U, const double *eps0_host, const double *U_host, double *gdiag_host,
                         const ng_run_params *p, const ng_shard *shard, int *iters_out, void *stream);

/* ng_run_2b for this rank's share of the k-points (see ng_shard): grid.nbatch, G, eps0 and
 * eps_mf hold the rank's own k-points (k_begin .. k_begin + k_count - 1 of ng_shard_plan); Gloc,
 * Sigma and U are full copies on every rank.  Every k-reduction goes through the exchange, so
 * Gloc, Sigma and the rank's G_k are bitwise those of a single-GPU ng_run_2b over all nk
 * k-points (up to the rounding of the convergence distances, which are summed per rank, so a
 * setup loop could stop one iteration apart when its distance lands within rounding of the
 * tolerance).  NG_ECOMM if the callback fails. */
ng_status ng_run_2b_sharded(ng_ctx *ctx, const ng_grid *grid, ng_herm G, ng_herm Gloc, ng_herm Sigma,
                            ng_func eps0, ng_func eps_mf, ng_func U, const ng_run_params *p, const ng_shard *shard,
                            int *iters_out, void *stream);

/* ---- GW self-energy (Sec. "Self-energy approximation: GW") ------------------------------ */

/* P, K and K^ddagger on slice tstp (-1 = Matsubara) from the local fermionic Gloc, elementwise
 * in the orbital indices: P_ab(t,t') = -i G_ab(t,t') G_ba(t',t) (minus the product of Eq.
 * def_bubble1), K = -P U(t'), K^ddagger = -U(t) P, the kernel pair of (1 + K) * chi = P
 * (Eq. dyson_chi with a local interaction U(t), real; U.val[n+1] holds U_n).  The Matsubara
 * component follows C^M(tau) = -i C(-i tau, 0) (Eq. matsconv): P^M_ab(tau) = G^M_ab(tau)
 * G^M_ba(-tau).  grid describes Gloc (sig = -1); P, K, Kcc are bosonic herms of the same shape;
 * all ldk = 1.  Reads slice tstp of Gloc (the whole Matsubara/left-mixing row), writes slice
 * tstp of P, K, Kcc. */
ng_status ng_gw_polarization_timestep(ng_ctx *ctx, const ng_grid *grid, int tstp, ng_herm P, ng_herm K,
                                      ng_herm Kcc, ng_herm Gloc, ng_func U, void *stream);

/* Sigma on slice tstp from Gloc and the susceptibility chi (Eq. SigmaGW):
 * dW_ab(t,t') = U(t) chi_ab(t,t') U(t'), Sigma_ab = i G_ab(t,t') dW_ab(t,t') (Eq. def_bubble2;
 * Matsubara Sigma^M = -G^M(tau) dW^M(tau)).  All ldk = 1. */
ng_status ng_gw_sigma_timestep(ng_ctx *ctx, const ng_grid *grid, int tstp, ng_herm Sigma, ng_herm Gloc,
                               ng_herm Chi, ng_func U, void *stream);

/* Self-consistent GW run: ng_run_2b with the GW self-energy of the local Gloc in place of the
 * second-Born one.  Each evaluation of Sigma forms P, K, K^ddagger on its slices, solves the
 * susceptibility equation (ng_vie2_mat in the Matsubara loop, ng_vie2_start for slices 0..k
 * in the bootstrapping, ng_vie2_timestep(n) in every corrector pass), then dW and Sigma.
 * Chi: caller-owned bosonic herm (ldk = 1, whole contour) receiving chi; P, K, K^ddagger are
 * kept in the context, so a run continued with do_setup = 0 must follow a GW run on the same
 * context and grid.  nf = 1, 2, 4.  Otherwise as ng_run_2b. */
ng_status ng_run_gw(ng_ctx *ctx, const ng_grid *grid, ng_herm G, ng_herm Gloc, ng_herm Sigma, ng_herm Chi,
                    ng_func eps0, ng_func eps_mf, ng_func U, const ng_run_params *p, int *iters_out, void *stream);

/* k-space GW of a translation-invariant one-band lattice (Sec. "GW for the translationally
 * invariant Hubbard model"): the nbatch problems are the momenta k_m = 2 pi m / nbatch of a ring
 * (m = 0..nbatch-1, the problem index), U(t) local:
 *     Pi_k(t,t')  = -(i/N_k) sum_q G_{k+q}(t,t') G_q(t',t)          (Eq. Pol)
 *     chi_k       = Pi_k + Pi_k * U * chi_k,  K_k = -Pi_k U(t'), K_k^ddagger = -U(t) Pi_k
 *     Sigma_k     = (i/N_k) sum_q G_{k-q}(t,t') U(t) chi_q(t,t') U(t')   (Eq. Sigmak)
 * The momentum sums are evaluated in real space: per slice element, G(r) = (1/N_k) sum_k
 * e^{ikr} G_k, the bubbles of r and -r, and X_k = sum_r e^{-ikr} X(r) back, by FP64 FFTs along
 * the k index (radix 2 for nbatch a power of two, the direct sum otherwise); the same sums as
 * the momentum convolutions up to rounding.  nf = 1, nbatch <= 4096.  G, Sigma, P, K, Kcc, Chi
 * have ldk = nbatch (P, K, Kcc, Chi bosonic). */
ng_status ng_gw_kspace_polarization_timestep(ng_ctx *ctx, const ng_grid *grid, int tstp, ng_herm P, ng_herm K,
                                             ng_herm Kcc, ng_herm Gk, ng_func U, void *stream);
ng_status ng_gw_kspace_sigma_timestep(ng_ctx *ctx, const ng_grid *grid, int tstp, ng_herm Sigma, ng_herm Gk,
                                      ng_herm Chi, ng_func U, void *stream);

/* Self-consistent k-space GW run: ng_run_gw with Sigma_k per momentum (Sigma.ldk = nbatch) in
 * the Dyson equation of each G_k, chi_k solved by the batched vie2 (Chi.ldk = nbatch); the
 * Hartree term from the local density as in ng_run_2b.  NG_FP64 only. */
ng_status ng_run_gw_kspace(ng_ctx *ctx, const ng_grid *grid, ng_herm G, ng_herm Gloc, ng_herm Sigma, ng_herm Chi,
                           ng_func eps0, ng_func eps_mf, ng_func U, const ng_run_params *p, int *iters_out,
                           void *stream);

/* Fixed-Sigma solve: dyson_mat, dyson_start, then dyson_timestep for n = k+1..n_to
 * (Sec. "Test of accuracy and scaling analysis", three-step procedure). */
ng_status ng_solve_fixed(ng_ctx *ctx, const ng_grid *grid, ng_herm G, ng_herm Sigma,
                         ng_func eps, int n_to, void *stream);

/* ---- adjoint -------------------------------------------------------------------------- */

/* Discrete adjoint (reverse mode) of ng_run_2b for nf = 1: the exact gradient of a real loss
 * L of the densities G_kb^<(t_n, t_n) with respect to the bare dispersion eps0_kb(t_n),
 * n = 0..nt, through the algorithm as executed in FP64 (predictor, p->corrector passes of
 * {Gloc, Hartree, second-Born, Dyson time step} per step, mixed schedule, and the
 * bootstrapped start slices 0..k, Sec. "Time stepping", "Start", "Hubbard chain").  The
 * paper has no adjoint; the method's own equations are transposed step by step.
 * Precondition: G, Gloc, Sigma, eps_mf hold the state that ng_run_2b (do_setup = 1,
 * stepping k+1..nt, FP64, the same p->corrector) left; eps0 and U are its inputs.
 * seed (device, [nt+1][nbatch] complex128): c_kb(n) = dL/dRe G^<_kb(n,n) + i dL/dIm G^<_kb(n,n).
 * cG (ldk = nbatch) and cS (ldk = 1): caller-owned herm buffers shaped like G and Sigma
 * (mat unused), overwritten with the cotangents of the final history.
 * The corrector iterates are recomputed from the kept history in segments of `segment` steps
 * (0: ceil(sqrt(nt - k))), each re-run forward with its iterates held in the context, then
 * walked backwards; segment = NG_ADJ_RECORDED uses the iterates that ng_adjoint_forward kept
 * for this G (no recomputation).  The start slices are a fixed point of the bootstrapping; their adjoint
 * is iterated to |change| <= p->boot_tol |mu| (default 1e-14), at most p->boot_maxiter times.
 * grad_eps0 (device, [nt+2][nbatch] double): dL/deps0_kb(t_n) at index n+1 (row 0 unused).
 * G, Sigma and eps_mf are rewritten with bitwise-equal values by the recomputation; Gloc is
 * rewritten too (its slices 0..k from the final start slices of G).
 * info (host, may be NULL) receives {start-slice iterations, segments, segment length}.
 * Errors: NG_EUNSUPPORTED for nf != 1; NG_EINVAL for bad layouts; NG_ENOCONV if the start-slice
 * adjoint did not converge; NG_ENOMEM if the context workspace cannot be allocated. */
#define NG_ADJ_RECORDED (-1)

/* ng_run_2b (do_setup = 1, stepping k+1..nt, FP64) that also keeps every corrector iterate of
 * every step (G_k, Gloc and Sigma slices, eps_mf) in the context for a following
 * ng_adjoint_2b(segment = NG_ADJ_RECORDED), which then needs no forward recomputation: it
 * trades (nt - k) p->corrector ((nbatch + 2)(2 nt + ntau + 3) + nbatch) complex values of device
 * memory for one forward run.  Same arguments, checks and results as ng_run_2b; nf = 1.  Any other
 * adjoint call on the context (segment >= 0) releases the record. */
ng_status ng_adjoint_forward(ng_ctx *ctx, const ng_grid *grid, ng_herm G, ng_herm Gloc, ng_herm Sigma,
                             ng_func eps0, ng_func eps_mf, ng_func U, const ng_run_params *p, int *iters_out,
                             void *stream);

ng_status ng_adjoint_2b(ng_ctx *ctx, const ng_grid *grid, ng_herm G, ng_herm Gloc, ng_herm Sigma,
                        ng_func eps0, ng_func eps_mf, ng_func U, const ng_run_params *p,
                        const void *seed, ng_herm cG, ng_herm cS, int segment, double *grad_eps0,
                        int *info, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* NG_H */
