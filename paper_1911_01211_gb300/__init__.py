"""GB300 contour Dyson time-stepper: thin Python binding of libng.so (C ABI in include/ng.h).

Every computation runs in the CUDA kernels of libng.so; this module only marshals
arguments.  PyTorch supplies device memory and streams.  Importing fails loudly when
the compiled library is missing: there is no CPU fallback.

Storage (see include/ng.h): a contour function for ``nbatch`` problems is four complex128
device tensors with the problem index innermost,
    mat [ntau+1,            nf, nf, ldk]
    ret [tri(nt+1),         nf, nf, ldk]   element (n, j), j <= n at tri(n) + j
    les [tri(nt+1),         nf, nf, ldk]   element (j, n), j <= n at tri(n) + j
    tv  [(nt+1)*(ntau+1),   nf, nf, ldk]   element (n, m) at n*(ntau+1) + m
and a single-time function is val [nt+2, nf, nf, ldk] with f_n at index n+1.
"""
import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libng.so")

(NG_OK, NG_EINVAL, NG_ENOMEM, NG_ECUDA, NG_ENOCONV, NG_ETIMEOUT, NG_ENONFINITE, NG_EUNSUPPORTED, NG_ESCRATCH,
 NG_ECOMM, NG_ESINGULAR) = range(11)
NG_FP64, NG_F32C, NG_DF64 = 0, 1, 2
NG_MIXED, NG_SERIAL = 0, 1
NG_TVSRC_AUTO, NG_TVSRC_DIRECT = 0, 1
NG_ADJ_RECORDED = -1
NG_BULK_AUTO, NG_BULK_THREAD, NG_BULK_WARP = 0, 1, 2
_STATUS_NAMES = ["NG_OK", "NG_EINVAL", "NG_ENOMEM", "NG_ECUDA", "NG_ENOCONV", "NG_ETIMEOUT",
                 "NG_ENONFINITE", "NG_EUNSUPPORTED", "NG_ESCRATCH", "NG_ECOMM", "NG_ESINGULAR"]


class NgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS_NAMES[status] if 0 <= status < len(_STATUS_NAMES) else status}: {msg}")
        self.status = status


class ng_grid(ctypes.Structure):
    _fields_ = [("nt", ctypes.c_int), ("ntau", ctypes.c_int), ("nf", ctypes.c_int), ("nbatch", ctypes.c_int),
                ("korder", ctypes.c_int), ("sig", ctypes.c_int), ("h", ctypes.c_double),
                ("beta", ctypes.c_double), ("mu", ctypes.c_double)]


class ng_herm(ctypes.Structure):
    _fields_ = [("mat", ctypes.c_void_p), ("ret", ctypes.c_void_p), ("les", ctypes.c_void_p),
                ("tv", ctypes.c_void_p), ("ldk", ctypes.c_int)]


class ng_func(ctypes.Structure):
    _fields_ = [("val", ctypes.c_void_p), ("ldk", ctypes.c_int)]


class ng_run_params(ctypes.Structure):
    _fields_ = [("corrector", ctypes.c_int), ("mats_tol", ctypes.c_double), ("mats_maxiter", ctypes.c_int),
                ("boot_tol", ctypes.c_double), ("boot_maxiter", ctypes.c_int), ("nbar", ctypes.c_double),
                ("n_from", ctypes.c_int), ("n_to", ctypes.c_int), ("do_setup", ctypes.c_int),
                ("precision", ctypes.c_int)]


EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t)


class ng_shard(ctypes.Structure):
    _fields_ = [("nk", ctypes.c_int), ("rank", ctypes.c_int), ("nranks", ctypes.c_int), ("send", ctypes.c_void_p),
                ("send_bytes", ctypes.c_size_t), ("recv", ctypes.c_void_p), ("exchange", EXCHANGE_FN),
                ("user", ctypes.c_void_p)]


# every symbol the header declares, with its ctypes signature
_P = ctypes.c_void_p
_G = ctypes.POINTER(ng_grid)
SIGNATURES = {
    "ng_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(_P)]),
    "ng_destroy": (None, [_P]),
    "ng_last_error": (ctypes.c_char_p, [_P]),
    "ng_status_sync": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int)]),
    "ng_weights": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "ng_green_from_H_const": (ctypes.c_int, [_P, _G, ng_herm, ctypes.POINTER(ctypes.c_double), ctypes.c_double, _P]),
    "ng_dyson_mat": (ctypes.c_int, [_P, _G, ng_herm, ng_herm, ng_func, _P]),
    "ng_dyson_start": (ctypes.c_int, [_P, _G, ng_herm, ng_herm, ng_func, _P]),
    "ng_dyson_timestep": (ctypes.c_int, [_P, _G, ctypes.c_int, ng_herm, ng_herm, ng_func, ctypes.c_int, ctypes.c_int,
                                         _P]),
    "ng_kreduce_timestep": (ctypes.c_int, [_P, _G, ctypes.c_int, ng_herm, ng_herm, _P, _P]),
    "ng_shard_plan": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _G, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_size_t)]),
    "ng_kreduce_partial": (ctypes.c_int, [_P, _G, ctypes.c_int, _P, ng_herm, _P, ctypes.c_int, _P]),
    "ng_kreduce_combine": (ctypes.c_int, [_P, _G, ctypes.c_int, ng_herm, _P, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, _P]),
    "ng_run_2b_host": (ctypes.c_int, [_P, _G, ng_herm, ng_herm, ng_herm, ng_func, ng_func, ng_func, _P, _P, _P,
                                      ctypes.POINTER(ng_run_params), ctypes.POINTER(ng_shard),
                                      ctypes.POINTER(ctypes.c_int), _P]),
    "ng_run_2b_sharded": (ctypes.c_int, [_P, _G, ng_herm, ng_herm, ng_herm, ng_func, ng_func, ng_func,
                                         ctypes.POINTER(ng_run_params), ctypes.POINTER(ng_shard),
                                         ctypes.POINTER(ctypes.c_int), _P]),
    "ng_sigma2b_timestep": (ctypes.c_int, [_P, _G, ctypes.c_int, ng_herm, ng_herm, ng_func, _P]),
    "ng_hartree_timestep": (ctypes.c_int, [_P, _G, ctypes.c_int, ng_func, ng_func, ng_herm, ng_func,
                                           ctypes.c_double, _P]),
    "ng_extrapolate_timestep": (ctypes.c_int, [_P, _G, ctypes.c_int, ng_herm, _P]),
    "ng_distance_timestep": (ctypes.c_int, [_P, _G, ctypes.c_int, ng_herm, ng_herm, _P, _P]),
    "ng_run_2b": (ctypes.c_int, [_P, _G, ng_herm, ng_herm, ng_herm, ng_func, ng_func, ng_func,
                                 ctypes.POINTER(ng_run_params), ctypes.POINTER(ctypes.c_int), _P]),
    "ng_run_gw": (ctypes.c_int, [_P, _G, ng_herm, ng_herm, ng_herm, ng_herm, ng_func, ng_func, ng_func,
                                 ctypes.POINTER(ng_run_params), ctypes.POINTER(ctypes.c_int), _P]),
    "ng_gw_polarization_timestep": (ctypes.c_int, [_P, _G, ctypes.c_int, ng_herm, ng_herm, ng_herm, ng_herm,
                                                   ng_func, _P]),
    "ng_gw_sigma_timestep": (ctypes.c_int, [_P, _G, ctypes.c_int, ng_herm, ng_herm, ng_herm, ng_func, _P]),
    "ng_run_gw_kspace": (ctypes.c_int, [_P, _G, ng_herm, ng_herm, ng_herm, ng_herm, ng_func, ng_func, ng_func,
                                        ctypes.POINTER(ng_run_params), ctypes.POINTER(ctypes.c_int), _P]),
    "ng_gw_kspace_polarization_timestep": (ctypes.c_int, [_P, _G, ctypes.c_int, ng_herm, ng_herm, ng_herm,
                                                          ng_herm, ng_func, _P]),
    "ng_gw_kspace_sigma_timestep": (ctypes.c_int, [_P, _G, ctypes.c_int, ng_herm, ng_herm, ng_herm, ng_func, _P]),
    "ng_solve_fixed": (ctypes.c_int, [_P, _G, ng_herm, ng_herm, ng_func, ctypes.c_int, _P]),
    "ng_precision_reset": (ctypes.c_int, [_P]),
    "ng_herm_sandwich": (ctypes.c_int, [_P, _G, ng_herm, _G, ng_herm, ctypes.POINTER(ctypes.c_double), _P]),
    "ng_batch_create": (ctypes.c_int, [_P, ctypes.c_int, _G, ctypes.POINTER(ng_herm), ctypes.POINTER(ng_herm),
                                       ctypes.POINTER(ng_func), ctypes.POINTER(_P)]),
    "ng_batch_destroy": (None, [_P]),
    "ng_batch_setup": (ctypes.c_int, [_P, _P, _P]),
    "ng_batch_step": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, _P]),
    "ng_batch_solve": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int), _P]),
    "ng_vie2_mat": (ctypes.c_int, [_P, _G, ng_herm, ng_herm, ng_herm, _P]),
    "ng_vie2_start": (ctypes.c_int, [_P, _G, ng_herm, ng_herm, ng_herm, ng_herm, _P]),
    "ng_vie2_timestep": (ctypes.c_int, [_P, _G, ctypes.c_int, ng_herm, ng_herm, ng_herm, ng_herm, ctypes.c_int, _P]),
    "ng_convolution_timestep": (ctypes.c_int, [_P, _G, ctypes.c_int, ng_herm, ng_herm, ng_herm, ng_func, ng_herm,
                                               ng_herm, _P]),
    "ng_observables": (ctypes.c_int, [_P, _G, ctypes.c_int, ng_herm, ng_herm, ng_func, ng_func, _P, _P]),
    "ng_dyson_start_noalloc": (ctypes.c_int, [_G, ng_herm, ng_herm, ng_func, _P]),
    "ng_set_bulk_split": (ctypes.c_int, [_P, ctypes.c_int]),
    "ng_set_tv_source": (ctypes.c_int, [_P, ctypes.c_int]),
    "ng_fp64_probe": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), _P]),
    "ng_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "ng_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "ng_adjoint_2b": (ctypes.c_int, [_P, _G, ng_herm, ng_herm, ng_herm, ng_func, ng_func, ng_func,
                                     ctypes.POINTER(ng_run_params), _P, ng_herm, ng_herm, ctypes.c_int, _P,
                                     ctypes.POINTER(ctypes.c_int), _P]),
    "ng_adjoint_forward": (ctypes.c_int, [_P, _G, ng_herm, ng_herm, ng_herm, ng_func, ng_func, ng_func,
                                          ctypes.POINTER(ng_run_params), ctypes.POINTER(ctypes.c_int), _P]),
}

_lib = None


def load_library(path=LIB_PATH):
    """Load libng.so and attach the signatures; raises if it is missing (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libng.so not found at {path}: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def tri(n):
    return n * (n + 1) // 2


@dataclass
class Grid:
    nt: int
    ntau: int
    nf: int
    nbatch: int
    korder: int
    h: float
    beta: float
    mu: float = 0.0
    sig: int = -1

    def c(self):
        return ng_grid(self.nt, self.ntau, self.nf, self.nbatch, self.korder, self.sig, self.h, self.beta, self.mu)


class Herm:
    """Device storage of a contour function for a batch (ldk = nbatch) or shared (ldk = 1)."""

    def __init__(self, grid, ldk=None, device="cuda", zero=True):
        g = grid
        self.grid = g
        self.ldk = g.nbatch if ldk is None else ldk
        d, L = g.nf, self.ldk
        alloc = torch.zeros if zero else torch.empty
        kw = dict(dtype=torch.complex128, device=device)
        self.mat = alloc((g.ntau + 1, d, d, L), **kw)
        self.ret = alloc((tri(g.nt + 1), d, d, L), **kw)
        self.les = alloc((tri(g.nt + 1), d, d, L), **kw)
        self.tv = alloc(((g.nt + 1) * (g.ntau + 1), d, d, L), **kw)

    def c(self):
        return ng_herm(self.mat.data_ptr(), self.ret.data_ptr(), self.les.data_ptr(), self.tv.data_ptr(), self.ldk)

    def tensors(self):
        return {"mat": self.mat, "ret": self.ret, "les": self.les, "tv": self.tv}


class Func:
    """Device storage of a single-time function f_n, n = -1..nt, index n+1.
    scalar=True gives the nf = 1, ldk = 1 layout of an interaction profile U_n."""

    def __init__(self, grid, ldk=None, device="cuda", values=None, scalar=False):
        g = grid
        nf = 1 if scalar else g.nf
        self.ldk = 1 if scalar else (g.nbatch if ldk is None else ldk)
        if values is not None:
            self.val = values.to(device=device, dtype=torch.complex128).contiguous()
            assert tuple(self.val.shape) == (g.nt + 2, nf, nf, self.ldk)
        else:
            self.val = torch.zeros((g.nt + 2, nf, nf, self.ldk), dtype=torch.complex128, device=device)

    def c(self):
        return ng_func(self.val.data_ptr(), self.ldk)


class Batch:
    """An uneven batch of independent problems (ng_batch_*): per-problem grids and buffers."""

    def __init__(self, ctx, grids, Gs, Ss, epss):
        self.ctx = ctx
        n = len(grids)
        self._keep = (grids, Gs, Ss, epss)
        self._g = (ng_grid * n)(*[g.c() for g in grids])
        self._G = (ng_herm * n)(*[x.c() for x in Gs])
        self._S = (ng_herm * n)(*[x.c() for x in Ss])
        self._e = (ng_func * n)(*[x.c() for x in epss])
        h = ctypes.c_void_p()
        ctx._chk(ctx.lib.ng_batch_create(ctx.h, n, self._g, self._G, self._S, self._e, ctypes.byref(h)))
        self.h = h

    def setup(self, stream=None):
        self.ctx._chk(self.ctx.lib.ng_batch_setup(self.ctx.h, self.h, _stream(stream)))

    def step(self, n, threads=0, stream=None):
        self.ctx._chk(self.ctx.lib.ng_batch_step(self.ctx.h, self.h, n, threads, _stream(stream)))

    def solve(self, stream=None):
        t = ctypes.c_int()
        self.ctx._chk(self.ctx.lib.ng_batch_solve(self.ctx.h, self.h, ctypes.byref(t), _stream(stream)))
        return t.value

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.ng_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dyson_start_noalloc(grid, G, S, eps, stream=None):
    """ng_dyson_start_noalloc: the start-up slices without any device allocation (no context;
    fixed 2 MiB static device scratch).  Returns the ng_status code (NG_ESCRATCH when the
    problem does not fit the static scratch)."""
    lib = load_library()
    return lib.ng_dyson_start_noalloc(ctypes.byref(grid.c()), G.c(), S.c(), eps.c(), _stream(stream))


def shard_plan(nk, rank, nranks, grid=None):
    """ng_shard_plan: (k_begin, k_count, send_bytes) of rank `rank` (send_bytes 0 without grid).
    Host only."""
    lib = load_library()
    b, c, nb = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
    st = lib.ng_shard_plan(nk, rank, nranks, ctypes.byref(grid.c()) if grid is not None else None, ctypes.byref(b),
                           ctypes.byref(c), ctypes.byref(nb) if grid is not None else None)
    if st != NG_OK:
        raise NgError(st, f"ng_shard_plan(nk={nk}, rank={rank}, nranks={nranks}) failed")
    return b.value, c.value, nb.value


def fp64_probe(stream=None):
    """ng_fp64_probe on the current device: {dfma_tflops, dmma_tflops, sms}."""
    lib = load_library()
    out = (ctypes.c_double * 3)()
    st = lib.ng_fp64_probe(out, _stream(stream))
    if st != NG_OK:
        raise NgError(st, "ng_fp64_probe failed")
    return {"dfma_tflops": out[0], "dmma_tflops": out[1], "sms": int(out[2])}


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """One libng context (integration weights of order k, workspaces, status word)."""

    def __init__(self, korder, device=0):
        self.lib = load_library()
        h = ctypes.c_void_p()
        st = self.lib.ng_create(korder, device, ctypes.byref(h))
        if st != NG_OK:
            raise NgError(st, "ng_create failed")
        self.h = h
        self.k = korder

    def close(self):
        if getattr(self, "h", None):
            self.lib.ng_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st):
        if st != NG_OK:
            raise NgError(st, self.lib.ng_last_error(self.h).decode())

    def weights(self):
        out = (ctypes.c_double * 18)()
        self._chk(self.lib.ng_weights(self.h, out))
        return list(out)

    def observables(self, grid, tstp, G, S, eps0, eps_mf, out, stream=None):
        """out: device float64 tensor of 5 -> [N, E_kin, E_mf, E_corr, E_tot] (batch averages)."""
        self._chk(self.lib.ng_observables(self.h, ctypes.byref(grid.c()), tstp, G.c(), S.c(), eps0.c(), eps_mf.c(),
                                          ctypes.c_void_p(out.data_ptr()), _stream(stream)))

    def herm_sandwich(self, grid_out, Out, grid_in, In, V, stream=None):
        import numpy as np
        v = np.ascontiguousarray(np.asarray(V, dtype=np.complex128).reshape(grid_out.nf, grid_in.nf))
        self._chk(self.lib.ng_herm_sandwich(self.h, ctypes.byref(grid_out.c()), Out.c(), ctypes.byref(grid_in.c()),
                                            In.c(), v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                            _stream(stream)))
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()

    def batch(self, grids, Gs, Ss, epss):
        return Batch(self, grids, Gs, Ss, epss)

    def precision_reset(self):
        self._chk(self.lib.ng_precision_reset(self.h))

    def profile_enable(self, on=True):
        self._chk(self.lib.ng_profile_enable(self.h, 1 if on else 0))

    def profile_read(self):
        """{bulk_ms, bulk_launches, bulk_flops, boundary_ms, boundary_launches, tvfft_ms, tvfft_launches,
        gw_ms, gw_evals}"""
        out = (ctypes.c_double * 9)()
        self._chk(self.lib.ng_profile_read(self.h, out))
        return dict(zip(("bulk_ms", "bulk_launches", "bulk_flops", "boundary_ms", "boundary_launches", "tvfft_ms",
                         "tvfft_launches", "gw_ms", "gw_evals"), list(out)))

    def set_bulk_split(self, mode):
        """NG_BULK_AUTO, NG_BULK_THREAD (one thread per bulk item) or NG_BULK_WARP (one warp)."""
        self._chk(self.lib.ng_set_bulk_split(self.h, mode))

    def set_tv_source(self, mode):
        """NG_TVSRC_AUTO (FFT where supported) or NG_TVSRC_DIRECT."""
        self._chk(self.lib.ng_set_tv_source(self.h, mode))

    def status_sync(self, stream=None):
        f = ctypes.c_int()
        st = self.lib.ng_status_sync(self.h, _stream(stream), ctypes.byref(f))
        return st, f.value

    # ---- entry points (same names as the C ABI, minus the ng_ prefix) ----------------
    def green_from_H_const(self, grid, G, eps, scale=1.0, stream=None):
        import numpy as np
        e = np.ascontiguousarray(np.asarray(eps, dtype=np.complex128).reshape(grid.nbatch, grid.nf, grid.nf))
        ptr = e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self._chk(self.lib.ng_green_from_H_const(self.h, ctypes.byref(grid.c()), G.c(), ptr, scale, _stream(stream)))
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()

    def dyson_mat(self, grid, G, S, eps, stream=None):
        self._chk(self.lib.ng_dyson_mat(self.h, ctypes.byref(grid.c()), G.c(), S.c(), eps.c(), _stream(stream)))

    def dyson_start(self, grid, G, S, eps, stream=None):
        self._chk(self.lib.ng_dyson_start(self.h, ctypes.byref(grid.c()), G.c(), S.c(), eps.c(), _stream(stream)))

    def dyson_timestep(self, grid, tstp, G, S, eps, precision=NG_FP64, schedule=NG_MIXED, stream=None):
        self._chk(self.lib.ng_dyson_timestep(self.h, ctypes.byref(grid.c()), tstp, G.c(), S.c(), eps.c(),
                                             precision, schedule, _stream(stream)))

    def vie2_mat(self, grid, G, F, Q, stream=None):
        self._chk(self.lib.ng_vie2_mat(self.h, ctypes.byref(grid.c()), G.c(), F.c(), Q.c(), _stream(stream)))

    def vie2_start(self, grid, G, F, Fcc, Q, stream=None):
        self._chk(self.lib.ng_vie2_start(self.h, ctypes.byref(grid.c()), G.c(), F.c(), Fcc.c(), Q.c(),
                                         _stream(stream)))

    def vie2_timestep(self, grid, tstp, G, F, Fcc, Q, schedule=NG_MIXED, stream=None):
        self._chk(self.lib.ng_vie2_timestep(self.h, ctypes.byref(grid.c()), tstp, G.c(), F.c(), Fcc.c(), Q.c(),
                                            schedule, _stream(stream)))

    def convolution_timestep(self, grid, tstp, C, A, Acc, f, B, Bcc, stream=None):
        """Slice tstp (-1: Matsubara) of C = A * f * B; f = None is the identity."""
        fc = f.c() if f is not None else ng_func(None, 1)
        self._chk(self.lib.ng_convolution_timestep(self.h, ctypes.byref(grid.c()), tstp, C.c(), A.c(), Acc.c(), fc,
                                                   B.c(), Bcc.c(), _stream(stream)))

    def kreduce_timestep(self, grid, tstp, Gloc, Gk, wk=None, stream=None):
        """wk: optional device float64 tensor of nbatch k-point weights (default 1/nbatch)."""
        w = ctypes.c_void_p(wk.data_ptr()) if wk is not None else None
        self._chk(self.lib.ng_kreduce_timestep(self.h, ctypes.byref(grid.c()), tstp, Gloc.c(), Gk.c(), w,
                                               _stream(stream)))

    def kreduce_partial(self, grid, tstp, partial, Gk, k_begin, wk=None, stream=None):
        w = ctypes.c_void_p(wk.data_ptr()) if wk is not None else None
        self._chk(self.lib.ng_kreduce_partial(self.h, ctypes.byref(grid.c()), tstp, ctypes.c_void_p(partial.data_ptr()),
                                              Gk.c(), w, k_begin, _stream(stream)))

    def kreduce_combine(self, grid, tstp, Gloc, gathered, nk, nranks, weighted=False, stream=None):
        self._chk(self.lib.ng_kreduce_combine(self.h, ctypes.byref(grid.c()), tstp, Gloc.c(),
                                              ctypes.c_void_p(gathered.data_ptr()), nk, nranks, 1 if weighted else 0,
                                              _stream(stream)))

    def sigma2b_timestep(self, grid, tstp, S, Gloc, U, stream=None):
        self._chk(self.lib.ng_sigma2b_timestep(self.h, ctypes.byref(grid.c()), tstp, S.c(), Gloc.c(), U.c(),
                                               _stream(stream)))

    def hartree_timestep(self, grid, tstp, eps_mf, eps0, Gloc, U, nbar, stream=None):
        self._chk(self.lib.ng_hartree_timestep(self.h, ctypes.byref(grid.c()), tstp, eps_mf.c(), eps0.c(), Gloc.c(),
                                               U.c(), nbar, _stream(stream)))

    def extrapolate_timestep(self, grid, tstp, G, stream=None):
        self._chk(self.lib.ng_extrapolate_timestep(self.h, ctypes.byref(grid.c()), tstp, G.c(), _stream(stream)))

    def distance_timestep(self, grid, tstp, A, B, out, stream=None):
        self._chk(self.lib.ng_distance_timestep(self.h, ctypes.byref(grid.c()), tstp, A.c(), B.c(),
                                                ctypes.c_void_p(out.data_ptr()), _stream(stream)))

    def solve_fixed(self, grid, G, S, eps, n_to=None, stream=None):
        n_to = grid.nt if n_to is None else n_to
        self._chk(self.lib.ng_solve_fixed(self.h, ctypes.byref(grid.c()), G.c(), S.c(), eps.c(), n_to, _stream(stream)))

    def run_2b(self, grid, G, Gloc, S, eps0, eps_mf, U, corrector=3, mats_tol=1e-12, mats_maxiter=200,
               boot_tol=1e-12, boot_maxiter=200, nbar=0.5, n_from=None, n_to=None, do_setup=True,
               stream=None, allow_noconv=False, precision=NG_FP64):
        p = ng_run_params(corrector, mats_tol, mats_maxiter, boot_tol, boot_maxiter, nbar,
                          grid.korder + 1 if n_from is None else n_from,
                          grid.nt if n_to is None else n_to, 1 if do_setup else 0, precision)
        iters = (ctypes.c_int * 2)()
        st = self.lib.ng_run_2b(self.h, ctypes.byref(grid.c()), G.c(), Gloc.c(), S.c(), eps0.c(), eps_mf.c(), U.c(),
                                ctypes.byref(p), iters, _stream(stream))
        if not (allow_noconv and st == NG_ENOCONV):
            self._chk(st)
        return list(iters)

    def run_gw(self, grid, G, Gloc, S, Chi, eps0, eps_mf, U, corrector=3, mats_tol=1e-12, mats_maxiter=200,
               boot_tol=1e-12, boot_maxiter=200, nbar=0.5, n_from=None, n_to=None, do_setup=True,
               stream=None, allow_noconv=False, precision=NG_FP64):
        """ng_run_gw: Chi is a bosonic Herm (ldk = 1) on the grid of G receiving chi."""
        p = ng_run_params(corrector, mats_tol, mats_maxiter, boot_tol, boot_maxiter, nbar,
                          grid.korder + 1 if n_from is None else n_from,
                          grid.nt if n_to is None else n_to, 1 if do_setup else 0, precision)
        iters = (ctypes.c_int * 2)()
        st = self.lib.ng_run_gw(self.h, ctypes.byref(grid.c()), G.c(), Gloc.c(), S.c(), Chi.c(), eps0.c(),
                                eps_mf.c(), U.c(), ctypes.byref(p), iters, _stream(stream))
        if not (allow_noconv and st == NG_ENOCONV):
            self._chk(st)
        return list(iters)

    def run_gw_kspace(self, grid, G, Gloc, S, Chi, eps0, eps_mf, U, corrector=3, mats_tol=1e-12, mats_maxiter=200,
                      boot_tol=1e-12, boot_maxiter=200, nbar=0.5, n_from=None, n_to=None, do_setup=True,
                      stream=None, allow_noconv=False):
        """ng_run_gw_kspace: S and Chi have ldk = nbatch (momenta k_m = 2 pi m / nbatch)."""
        p = ng_run_params(corrector, mats_tol, mats_maxiter, boot_tol, boot_maxiter, nbar,
                          grid.korder + 1 if n_from is None else n_from,
                          grid.nt if n_to is None else n_to, 1 if do_setup else 0, NG_FP64)
        iters = (ctypes.c_int * 2)()
        st = self.lib.ng_run_gw_kspace(self.h, ctypes.byref(grid.c()), G.c(), Gloc.c(), S.c(), Chi.c(), eps0.c(),
                                       eps_mf.c(), U.c(), ctypes.byref(p), iters, _stream(stream))
        if not (allow_noconv and st == NG_ENOCONV):
            self._chk(st)
        return list(iters)

    def gw_kspace_polarization_timestep(self, grid, tstp, P, K, Kcc, Gk, U, stream=None):
        self._chk(self.lib.ng_gw_kspace_polarization_timestep(self.h, ctypes.byref(grid.c()), tstp, P.c(), K.c(),
                                                              Kcc.c(), Gk.c(), U.c(), _stream(stream)))

    def gw_kspace_sigma_timestep(self, grid, tstp, S, Gk, Chi, U, stream=None):
        self._chk(self.lib.ng_gw_kspace_sigma_timestep(self.h, ctypes.byref(grid.c()), tstp, S.c(), Gk.c(), Chi.c(),
                                                       U.c(), _stream(stream)))

    def gw_polarization_timestep(self, grid, tstp, P, K, Kcc, Gloc, U, stream=None):
        self._chk(self.lib.ng_gw_polarization_timestep(self.h, ctypes.byref(grid.c()), tstp, P.c(), K.c(), Kcc.c(),
                                                       Gloc.c(), U.c(), _stream(stream)))

    def gw_sigma_timestep(self, grid, tstp, S, Gloc, Chi, U, stream=None):
        self._chk(self.lib.ng_gw_sigma_timestep(self.h, ctypes.byref(grid.c()), tstp, S.c(), Gloc.c(), Chi.c(),
                                                U.c(), _stream(stream)))

    def run_2b_host(self, grid, G, Gloc, S, eps0, eps_mf, U, eps0_host, U_host, gdiag_host, corrector=3,
                    mats_tol=1e-12, mats_maxiter=200, boot_tol=1e-12, boot_maxiter=200, nbar=0.5, n_from=None,
                    n_to=None, do_setup=True, stream=None, allow_noconv=False, precision=NG_FP64, exchange=None):
        """ng_run_2b_host: eps0_host [nt+2, nf, nf, nbatch] and U_host [nt+2] complex128 CPU tensors
        (pinned for asynchronous copies), gdiag_host [nt+1, nf, nf] complex128 CPU tensor
        receiving Gloc^<(t_n, t_n).  exchange: this rank's shard.DistExchange (None: one GPU)."""
        for t in (eps0_host, U_host, gdiag_host):
            assert t.device.type == "cpu" and t.dtype == torch.complex128 and t.is_contiguous()
        p = ng_run_params(corrector, mats_tol, mats_maxiter, boot_tol, boot_maxiter, nbar,
                          grid.korder + 1 if n_from is None else n_from,
                          grid.nt if n_to is None else n_to, 1 if do_setup else 0, precision)
        iters = (ctypes.c_int * 2)()
        st = self.lib.ng_run_2b_host(self.h, ctypes.byref(grid.c()), G.c(), Gloc.c(), S.c(), eps0.c(), eps_mf.c(),
                                     U.c(), ctypes.c_void_p(eps0_host.data_ptr()), ctypes.c_void_p(U_host.data_ptr()),
                                     ctypes.c_void_p(gdiag_host.data_ptr()), ctypes.byref(p),
                                     ctypes.byref(exchange.c()) if exchange is not None else None, iters,
                                     _stream(stream))
        if exchange is not None and exchange.error is not None:
            raise exchange.error
        if not (allow_noconv and st == NG_ENOCONV):
            self._chk(st)
        return list(iters)

    def run_2b_sharded(self, grid, G, Gloc, S, eps0, eps_mf, U, exchange, corrector=3, mats_tol=1e-12,
                       mats_maxiter=200, boot_tol=1e-12, boot_maxiter=200, nbar=0.5, n_from=None, n_to=None,
                       do_setup=True, stream=None, allow_noconv=False, precision=NG_FP64):
        """ng_run_2b_sharded: grid, G, eps0, eps_mf hold this rank's k-points; `exchange` supplies
        nk, rank, nranks, the send/recv device tensors and the allgather callback (see shard.py)."""
        p = ng_run_params(corrector, mats_tol, mats_maxiter, boot_tol, boot_maxiter, nbar,
                          grid.korder + 1 if n_from is None else n_from,
                          grid.nt if n_to is None else n_to, 1 if do_setup else 0, precision)
        sh = exchange.c()
        iters = (ctypes.c_int * 2)()
        st = self.lib.ng_run_2b_sharded(self.h, ctypes.byref(grid.c()), G.c(), Gloc.c(), S.c(), eps0.c(), eps_mf.c(),
                                        U.c(), ctypes.byref(p), ctypes.byref(sh), iters, _stream(stream))
        if exchange.error is not None:
            raise exchange.error
        if not (allow_noconv and st == NG_ENOCONV):
            self._chk(st)
        return list(iters)

    def adjoint_forward(self, grid, G, Gloc, S, eps0, eps_mf, U, corrector=3, mats_tol=1e-14, mats_maxiter=200,
                        boot_tol=1e-14, boot_maxiter=200, nbar=0.5, stream=None):
        """ng_adjoint_forward: ng_run_2b keeping every corrector iterate for
        adjoint_2b(segment=NG_ADJ_RECORDED)."""
        p = ng_run_params(corrector, mats_tol, mats_maxiter, boot_tol, boot_maxiter, nbar, grid.korder + 1, grid.nt,
                          1, NG_FP64)
        iters = (ctypes.c_int * 2)()
        self._chk(self.lib.ng_adjoint_forward(self.h, ctypes.byref(grid.c()), G.c(), Gloc.c(), S.c(), eps0.c(),
                                              eps_mf.c(), U.c(), ctypes.byref(p), iters, _stream(stream)))
        return list(iters)

    def adjoint_2b(self, grid, G, Gloc, S, eps0, eps_mf, U, seed, cG, cS, grad_eps0, corrector=3, nbar=0.5,
                   boot_tol=1e-14, boot_maxiter=200, segment=0, stream=None):
        """ng_adjoint_2b: seed = device complex128 [nt+1, nbatch] cotangent of G^<_kb(n,n);
        grad_eps0 = device float64 [nt+2, nbatch] (index n+1).  Returns
        [start-slice iterations, segments, segment length]."""
        p = ng_run_params(corrector, 0.0, 0, boot_tol, boot_maxiter, nbar, grid.korder + 1, grid.nt, 0, NG_FP64)
        info = (ctypes.c_int * 3)()
        self._chk(self.lib.ng_adjoint_2b(self.h, ctypes.byref(grid.c()), G.c(), Gloc.c(), S.c(), eps0.c(),
                                         eps_mf.c(), U.c(), ctypes.byref(p), ctypes.c_void_p(seed.data_ptr()),
                                         cG.c(), cS.c(), segment, ctypes.c_void_p(grad_eps0.data_ptr()), info,
                                         _stream(stream)))
        return list(info)
