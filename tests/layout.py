"""Copies between the device store (packed, problem index innermost) and the oracle's
full-storage containers; test helpers only (layout marshalling, no method arithmetic)."""
import numpy as np
import torch

from oracle.contour import Func as OFunc
from oracle.contour import Herm as OHerm


def tri(n):
    return n * (n + 1) // 2


def herm_to_oracle(H, g, kb):
    """Device Herm -> oracle Herm of problem kb (kb = 0 for shared data)."""
    N, T, d = g.nt, g.ntau, g.nf
    o = OHerm(N, T, d)
    mat = H.mat[..., kb].cpu().numpy()
    ret = H.ret[..., kb].cpu().numpy()
    les = H.les[..., kb].cpu().numpy()
    tv = H.tv[..., kb].cpu().numpy()
    o.mat[...] = mat
    for n in range(N + 1):
        o.ret[n, :n + 1] = ret[tri(n):tri(n) + n + 1]
        o.les[:n + 1, n] = les[tri(n):tri(n) + n + 1]
    o.tv[...] = tv.reshape(N + 1, T + 1, d, d)
    return o


def oracle_to_herm(objs, H, g, nmax=None):
    """List of oracle Herm (one per problem, or one for shared) -> device Herm slices -1..nmax."""
    N, T, d = g.nt, g.ntau, g.nf
    nmax = N if nmax is None else nmax
    L = H.ldk
    mat = np.zeros((T + 1, d, d, L), complex)
    ret = np.zeros((tri(N + 1), d, d, L), complex)
    les = np.zeros((tri(N + 1), d, d, L), complex)
    tv = np.zeros(((N + 1) * (T + 1), d, d, L), complex)
    for kb, o in enumerate(objs):
        mat[..., kb] = o.mat
        for n in range(nmax + 1):
            ret[tri(n):tri(n) + n + 1, ..., kb] = o.ret[n, :n + 1]
            les[tri(n):tri(n) + n + 1, ..., kb] = o.les[:n + 1, n]
            tv[n * (T + 1):(n + 1) * (T + 1), ..., kb] = o.tv[n]
    for name, arr in (("mat", mat), ("ret", ret), ("les", les), ("tv", tv)):
        getattr(H, name).copy_(torch.from_numpy(arr))


def funcs_to_device(ofuncs, F):
    """List of oracle Func (per problem) -> device Func values."""
    arr = np.stack([f.val for f in ofuncs], axis=-1)
    F.val.copy_(torch.from_numpy(np.ascontiguousarray(arr)))


def device_to_funcs(F, g):
    arr = F.val.cpu().numpy()
    out = []
    for kb in range(arr.shape[-1]):
        f = OFunc(g.nt, g.nf)
        f.val[...] = arr[..., kb]
        out.append(f)
    return out
