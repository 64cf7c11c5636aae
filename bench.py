#!/usr/bin/env python
"""Benchmark of the GB300 contour Dyson time-stepper.

Workload (default): the chain_kspace model -- 1D Hubbard chain in momentum space, nk = 512
k-points, eps_k(t) = -2 cos(k - A(t)) with a Peierls pulse, local second-Born self-energy
(U = 2) from the k-summed G_loc; beta = 10, ntau = 800, nt = 2000, h = 0.01, order k = 5,
3 corrector iterations per time step, FP64 complex arithmetic.

Metric: k-point timesteps per second.  A "step" is one time step n of the whole hot path
for all k-points: predictor (extrapolation of slice n), then 3 corrector passes of
{k-reduction of slice n, Hartree mean field, second-Born slice, Dyson time step}.
The Matsubara loop, the bootstrapping and the steps before the timed window run untimed;
the timed window is the LAST K steps of the nt = 2000 propagation (default: every step after
the W warm-up steps), so a short window measures the most expensive steps.

Lines printed: one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on the
host cores for the same metric (a bounded sample of k-point steps of the same workload).
Other workloads: --workload uneven (64 independent clusters, the batch path; --compare-plain
adds the same problems solved one after another), --workload adjoint (gradient of the final
kinetic energy on the 16 x 16 square lattice, with finite-difference checks), --workload dimer
(the Hubbard dimer quench and its energy drift) and --workload gw (the k-space GW chain,
nk = 128, nt = 2500).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# FP64 (DFMA, non-tensor) peak of one GB300 from its unit counts: SMs (152, read from the
# device) x 2 DFMA per clock per SM x 2 flop, times the SM clock (1.2586 TFLOP/s at the
# 2070 MHz maximum, the nominal 1.25 TFLOP/s).  The clock is the median sampled during the timed
# region.
GB300_SMS = 152
FP64_FLOP_PER_CLK_PER_SM = 4
SM_MAX_MHZ = 2070.0


def fp64_peak_tflops(sm_mhz, sms=GB300_SMS):
    return sms * FP64_FLOP_PER_CLK_PER_SM * (sm_mhz or SM_MAX_MHZ) * 1e6 / 1e12


def max_over_ranks(x, device="cuda"):
    """Largest value of x over the ranks of the default process group (x itself when there is
    none or it has one rank): the slowest rank's time sets the whole job's rate."""
    import torch
    import torch.distributed as td
    if not (td.is_available() and td.is_initialized()) or td.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0, help="timed time steps (0: all after warm-up)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    # development overrides (a run with any of these is not the headline workload)
    ap.add_argument("--nk", type=int, default=512)
    ap.add_argument("--nt", type=int, default=2000)
    ap.add_argument("--ntau", type=int, default=800)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the oracle's time step n = nt on four k-points (headline-size parity)")
    ap.add_argument("--workload", choices=["chain", "uneven", "adjoint", "dimer", "gw"], default="chain",
                    help="chain: the headline chain_kspace run; uneven: the 64-cluster uneven batch; "
                         "adjoint: gradient of E_kin(t_N) on the 16x16 square lattice; dimer: the Hubbard "
                         "dimer quench at nt = 1000 and its energy drift; gw: the k-space GW chain "
                         "(nk = 128, nt = 2500)")
    ap.add_argument("--gw-nk", type=int, default=128, help="gw: momenta (development override)")
    ap.add_argument("--gw-nt", type=int, default=2500, help="gw: nt (development override)")
    ap.add_argument("--fd-slices", type=int, default=20, help="adjoint: time slices checked by central differences")
    ap.add_argument("--fd-deltas", default="1e-4,1e-5,1e-6",
                    help="adjoint: central-difference steps (comma separated); the fourth-order stencil is added")
    ap.add_argument("--adj-nt", type=int, default=1000, help="adjoint: nt (development override)")
    ap.add_argument("--nprob", type=int, default=64, help="problems of the uneven batch")
    ap.add_argument("--max-nf", type=int, default=8,
                    help="uneven: keep only the problems with nf <= this (4: a subset where no problem dominates "
                         "the cost)")
    ap.add_argument("--compare-plain", action="store_true",
                    help="uneven: also solve the same problems one after another with the plain path")
    ap.add_argument("--precision", choices=["f64", "both"], default="both",
                    help="f64: the FP64 headline only; both: also re-propagate with the FP32-compensated "
                         "(f32c) and double-float (df64) modes and report them beside the headline")
    return ap.parse_args()


def workload(a):
    from paper_1911_01211_gb300 import workloads as wl
    return wl.chain_kspace(nk=a.nk, nt=a.nt, ntau=a.ntau)


def config_of(w, K, W, world=1):
    return {
        "workload": f"chain_kspace nk={w.nbatch} nt={w.nt} ntau={w.ntau} h={w.h} beta={w.beta} U={w.U[1]:g} "
                    f"k={w.korder} corrector={w.corrector} (1D Hubbard chain, local second-Born, Peierls pulse)",
        "global_batch": w.nbatch, "nt": w.nt, "ntau": w.ntau, "nf": w.nf,
        "timed_steps": f"last {K} of {w.nt - w.korder} time steps (n = {w.nt - K + 1}..{w.nt}), {W} warm-up",
        "l2": "inputs larger than L2 (per-k history of tens of GB re-read every step)",
        "parallelism": ("single GPU, all k-points in one batch" if world == 1 else
                        f"{world} GPUs, k-points sharded in whole 32-blocks, one allgather of the block sums "
                        f"per k-reduction"),
    }


# ------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ------------------------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------------------------------
# the oracle's k-point time step, used by the cpu_baseline and the reference arm
# ------------------------------------------------------------------------------------------
_ORACLE = {}


def _oracle_init(nt, ntau, korder, seed):
    """Worker set-up: a seeded synthetic history of the workload's shape (values do not
    change the oracle's operation count)."""
    import numpy as np
    from oracle.contour import Func, Herm
    from oracle.weights import Weights
    rng = np.random.default_rng(seed)
    G, S = Herm(nt, ntau, 1), Herm(nt, ntau, 1)
    for X, sc in ((G, 0.3), (S, 0.05)):
        for c in ("mat", "ret", "les", "tv"):
            a = getattr(X, c)
            a[...] = sc * (rng.standard_normal(a.shape) + 1j * rng.standard_normal(a.shape))
    eps = Func(nt, 1)
    eps.val[:] = -2.0 * np.cos(0.3)
    _ORACLE.update(G=G, S=S, eps=eps, W=Weights(korder))


def _oracle_kstep(args):
    """One k-point time step of the oracle at step n: `corrector` solves of slice n."""
    n, beta, h, corrector = args
    from oracle import dyson
    o = _ORACLE
    t = time.perf_counter()
    for _ in range(corrector):
        dyson.dyson_timestep(n, o["G"], o["S"], o["eps"], 0.0, beta, h, o["W"])
    return time.perf_counter() - t


def oracle_rate(w, ns, workers):
    """Aggregate k-point steps/s of `workers` oracle processes (spawn) over the steps ns:
    workers x jobs / summed per-job compute time (history synthesis excluded)."""
    import multiprocessing as mp
    nmax = max(ns)
    jobs = [(n, w.beta, w.h, w.corrector) for n in ns]
    ctx = mp.get_context("spawn")
    t = time.perf_counter()
    with ctx.Pool(workers, initializer=_oracle_init, initargs=(nmax, w.ntau, w.korder, 7)) as pool:
        times = pool.map(_oracle_kstep, jobs, chunksize=1)
    wall = time.perf_counter() - t
    return workers * len(jobs) / sum(times), wall, sum(times)


def cpu_baseline(w, ns_window):
    """Bounded sample (~10-30 s of CPU work): k-point steps at the window's mean-cost step."""
    import numpy as np
    T = w.ntau
    cost = lambda n: 2 * n * n + 2 * n * T + T * T
    mean_cost = float(np.mean([cost(n) for n in ns_window]))
    n_ref = min(ns_window, key=lambda n: abs(cost(n) - mean_cost))
    workers = max(1, min(16, os.cpu_count() or 1))
    rate, wall, cpu = oracle_rate(w, [n_ref] * (3 * workers), workers)
    return {"value": rate, "unit": "k-point timesteps/s", "cores": workers, "kind": "oracle",
            "sample": f"{3 * workers} k-point time steps of the workload at n={n_ref} (the step whose cost equals "
                      f"the timed window's mean), {w.corrector} corrector solves each, seeded synthetic history, "
                      f"{workers} oracle processes; {cpu:.1f} s of CPU, wall {wall:.1f} s"}


# ------------------------------------------------------------------------------------------
def run_reference(a):
    w = workload(a)
    K = a.steps if a.steps > 0 else w.nt - w.korder - a.warmup
    W = a.warmup
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    ns = list(range(w.nt - K + 1, w.nt + 1))
    ns_warm = list(range(w.nt - K - W + 1, w.nt - K + 1))
    workers = max(1, min(16, os.cpu_count() or 1))
    if ns_warm:
        oracle_rate(w, ns_warm, workers)
    rate, wall, cpu = oracle_rate(w, ns, workers)
    line = {"metric": "k-point timesteps/s", "value": rate, "unit": "k-point timesteps/s", "impl": "reference",
            "n_gpus": a.gpus, "steps": K, "warmup": W, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_of(w, K, W),
            "cpu_baseline": {"value": rate, "unit": "k-point timesteps/s", "cores": workers, "kind": "oracle",
                             "sample": f"one k-point time step per bench step for each of the timed steps "
                                       f"n={ns[0]}..{ns[-1]} (3 corrector solves, synthetic history), "
                                       f"{workers} processes"},
            "e2e": {"value": rate, "unit": "k-point timesteps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "ms_per_step": 1000.0 * wall / len(ns)}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# headline-size parity: the oracle's own time step from the GPU's history
# ------------------------------------------------------------------------------------------
def _oracle_step_check(args):
    """Worker: the oracle's Dyson time step n of one k-point from the GPU's history (slices < n
    of G_k), its self-energy (slices <= n of Sigma) and eps_mf(n) of its last corrector pass;
    returns max |gpu - oracle| / max |oracle| per component of slice n."""
    import numpy as np
    from oracle import dyson
    from oracle.contour import Func, Herm
    from oracle.weights import Weights
    n, nt, ntau, beta, h, korder, Gp, Sp, eps, gpu_slice = args
    d = Gp["mat"].shape[-1]

    def herm(packed, upto):
        X = Herm(n, ntau, d)
        X.mat[...] = packed["mat"]
        for m in range(upto + 1):
            X.ret[m, :m + 1] = packed["ret"][m * (m + 1) // 2:m * (m + 1) // 2 + m + 1]
            X.les[:m + 1, m] = packed["les"][m * (m + 1) // 2:m * (m + 1) // 2 + m + 1]
            X.tv[m] = packed["tv"][m * (ntau + 1):(m + 1) * (ntau + 1)]
        return X
    G, S = herm(Gp, n - 1), herm(Sp, n)
    e = Func(n, d)
    e.val[...] = eps[:n + 2]
    dyson.dyson_timestep(n, G, S, e, 0.0, beta, h, Weights(korder))
    ref = {"ret": G.ret[n, :n + 1], "les": G.les[:n + 1, n], "tv": G.tv[n]}
    return {c: float(np.abs(gpu_slice[c] - ref[c]).max() / np.abs(ref[c]).max()) for c in ref}


def oracle_check_args(ng, g, n, G, S, mf, kbs):
    """Per k-point inputs of _oracle_step_check (host copies of the device history)."""
    T = g.ntau
    cut = {"mat": slice(0, T + 1), "ret": slice(0, ng.tri(n + 1)), "les": slice(0, ng.tri(n + 1)),
           "tv": slice(0, (n + 1) * (T + 1))}
    Sp = {c: getattr(S, c)[cut[c], ..., 0].cpu().numpy() for c in cut}
    out = []
    for kb in kbs:
        Gp = {c: getattr(G, c)[cut[c], ..., kb].cpu().numpy() for c in cut}
        gs = {"ret": Gp["ret"][ng.tri(n):ng.tri(n) + n + 1].copy(), "les": Gp["les"][ng.tri(n):ng.tri(n) + n + 1].copy(),
              "tv": Gp["tv"][n * (T + 1):(n + 1) * (T + 1)].copy()}
        eps = mf.val[..., kb].cpu().numpy()
        out.append((n, g.nt, T, g.beta, g.h, g.korder, Gp, Sp, eps, gs))
    return out


def fp64_probe_summary(ng):
    try:
        return ng.fp64_probe()
    except Exception as e:      # noqa: BLE001 - the probe is supporting evidence only
        return {"error": str(e)}


def run_ours(a):
    import multiprocessing as mp

    import numpy as np
    import torch
    import paper_1911_01211_gb300 as ng

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = world > 1
    # oracle workers for the headline-size parity check: spawned before the first GPU call
    pool = None
    if rank == 0 and not a.no_oracle_check:
        pool = mp.get_context("spawn").Pool(min(4, os.cpu_count() or 1))
    if dist:
        import torch.distributed as td
        td.init_process_group("nccl")
    torch.cuda.set_device(local)
    w = workload(a)
    k = w.korder
    W = a.warmup
    K = a.steps if a.steps > 0 else w.nt - k - W
    if K + W > w.nt - k:
        raise SystemExit(f"steps + warmup must be <= {w.nt - k}")
    n_first_timed = w.nt - K + 1
    nk = w.nbatch
    g_all = ng.Grid(nt=w.nt, ntau=w.ntau, nf=w.nf, nbatch=nk, korder=k, h=w.h, beta=w.beta, mu=w.mu)
    # this rank's k-points: whole blocks of 32 (all of them on one GPU)
    kb0, nkl, _ = ng.shard_plan(nk, rank, world, g_all)
    g = ng.Grid(nt=w.nt, ntau=w.ntau, nf=w.nf, nbatch=nkl, korder=k, h=w.h, beta=w.beta, mu=w.mu)
    exchange = None
    if dist:
        from paper_1911_01211_gb300.shard import DistExchange
        exchange = DistExchange(nk, g, f"cuda:{local}")
    ctx = ng.Context(k, local)
    probe = fp64_probe_summary(ng)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    G = ng.Herm(g, zero=False)
    L, S = ng.Herm(g, ldk=1), ng.Herm(g, ldk=1)
    e0, mf = ng.Func(g), ng.Func(g)
    U = ng.Func(g, scalar=True)
    # inputs and outputs in pinned host memory; the library copies eps_k(t_n) in and
    # Gloc^<(t_n, t_n) out step by step (ng_run_2b_host)
    eps_host = torch.from_numpy(np.ascontiguousarray(w.eps0[..., kb0:kb0 + nkl])).pin_memory()
    U_host = torch.from_numpy(w.U.astype(np.complex128)).pin_memory()
    gd_host = torch.zeros((w.nt + 1, w.nf, w.nf), dtype=torch.complex128).pin_memory()
    stream = torch.cuda.current_stream()
    h2d_bytes = eps_host[0].numel() * 16
    d2h_bytes = w.nf * w.nf * 16

    def barrier():
        torch.cuda.synchronize()
        if dist:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def run(n_from, n_to, setup, precision):
        return ctx.run_2b_host(g, G, L, S, e0, mf, U, eps_host, U_host, gd_host, corrector=w.corrector,
                               n_from=n_from, n_to=n_to, do_setup=setup, precision=precision, exchange=exchange)

    def propagate(precision, setup):
        """Steps k+1..nt (after the setup when `setup`); the last K are timed (CUDA events on the
        launching stream and the host clock, synchronised on both sides)."""
        barrier()
        t0 = time.perf_counter()
        run(k + 1, n_first_timed - 1, setup, precision)
        barrier()
        clocks = ClockSampler(local)
        clocks.start()
        ctx.profile_enable(True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tw0 = time.perf_counter()
        ev0.record(stream)
        run(n_first_timed, w.nt, False, precision)
        ev1.record(stream)
        barrier()
        t1 = time.perf_counter()
        ctx.profile_enable(False)
        clk = clocks.stop()
        return {"ms": ev0.elapsed_time(ev1), "prof": ctx.profile_read(), "clk": clk, "job_s": t1 - t0,
                "window_s": t1 - tw0}

    check_kbs = sorted(set(np.random.default_rng(191101211).choice(nkl, size=min(4, nkl), replace=False).tolist()))
    pending = {}

    def submit_check(name):
        if pool is not None:
            args = oracle_check_args(ng, g, w.nt, G, S, mf, check_kbs)
            pending[name] = pool.map_async(_oracle_step_check, args, chunksize=1)

    r = propagate(ng.NG_FP64, True)
    st, flags = ctx.status_sync()
    submit_check("f64")
    ms = max_over_ranks(r["ms"])
    value = nk * K / (ms / 1e3)
    e2e_value = nk * (w.nt - k) / max_over_ranks(r["job_s"])
    e2e_window = nk * K / max_over_ranks(r["window_s"])
    prof, clk = r["prof"], r["clk"]
    # per step: extrapolation, then per corrector pass k-reduce (or partial + combine), Hartree,
    # 2B, M_n^-1 (+ bulk, boundary)
    launches = int(prof["bulk_launches"] + prof["boundary_launches"] + prof["tvfft_launches"]) + \
        K * (1 + 3 * (4 + (1 if dist else 0)))
    achieved = prof["bulk_flops"] / (prof["bulk_ms"] / 1e3) / 1e12
    peak = fp64_peak_tflops(clk.get("sm_mhz"), sms)
    bulk_launches = max(1, prof["bulk_launches"])
    cmac_per_launch = prof["bulk_flops"] / 8.0 / w.nf ** 3 / bulk_launches
    traffic, traffic_note = None, None
    try:
        import hashlib
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tr = json.load(f)
        src = open(os.path.join(ROOT, "paper_1911_01211_gb300", "csrc", "ng_step.cuh"), "rb").read()
        if tr.get("ng_step_sha1") == hashlib.sha1(src).hexdigest():
            traffic = tr["captured"]["dram_bytes_per_cmac"] * cmac_per_launch
            traffic_note = (f"{tr['captured']['dram_bytes_per_cmac']:.2f} DRAM bytes per complex multiply-add "
                            f"(ncu capture: {tr['captured']['launch']}) x {cmac_per_launch:.4g} multiply-adds per "
                            f"launch of this window")
        else:
            traffic_note = "null: the time-step kernels changed since the ncu capture"
    except (OSError, ValueError, KeyError):
        traffic_note = "null: no ncu capture recorded"
    gd = gd_host.numpy().copy()
    # properties that hold at any size: particle number conserved for all t; Galitskii-Migdal
    # total energy conserved once the pulse has decayed (t >= 10: A(t) < 1e-5)
    obs = torch.zeros(5, dtype=torch.float64, device="cuda")
    n_after = [n for n in range(k + 1, w.nt + 1) if n * w.h >= 10.0]
    sample_n = sorted(set([k + 1] + list(range(k + 1, w.nt + 1, max(1, (w.nt - k) // 20))) + [w.nt]))
    vals = {}
    properties = None
    if not dist:
        for n in sorted(set(sample_n + n_after[:: max(1, len(n_after) // 20)] + ([n_after[-1]] if n_after else []))):
            ctx.observables(g, n, G, S, e0, mf, obs)
            vals[n] = obs.cpu().numpy().copy()
        Ns = np.array([v[0] for v in vals.values()])
        Eafter = np.array([vals[n][4] for n in vals if n * w.h >= 10.0])
        properties = {"N_drift_all_t": float(np.ptp(Ns)), "N_mean": float(Ns.mean()),
                      "E_tot_drift_after_pulse": float(np.ptp(Eafter)) if len(Eafter) else None,
                      "E_tot_at_end": float(vals[w.nt][4]), "E_kin_at_end": float(vals[w.nt][1]),
                      "E_corr_at_end": float(vals[w.nt][3]), "samples": len(vals)}
    modes = {}
    if a.precision == "both":
        # FP32-compensated and double-float time steps, each re-propagated from the same setup
        # (slices 0..k are not touched by the stepping) over the same timed window; error
        # against the FP64 run on the final slice n = nt (all local k-points, ret row / les
        # column / tv row) and on Gloc^<(t, t) for every t.
        nt = w.nt
        sl = lambda: {"ret": G.ret[ng.tri(nt):ng.tri(nt) + nt + 1], "les": G.les[ng.tri(nt):ng.tri(nt) + nt + 1],
                      "tv": G.tv[nt * (w.ntau + 1):(nt + 1) * (w.ntau + 1)]}
        ref = {c: x.clone() for c, x in sl().items()}
        bytes_per_elem = {"f32c": 8, "df64": 16}
        k32 = "k_step_bulk32p (two k-points per thread)" if w.nbatch % 2 == 0 else "k_step_bulk32<1>"
        for name, prec, kern in (("f32c", ng.NG_F32C, k32), ("df64", ng.NG_DF64, "k_step_bulkdf<1>")):
            rm = propagate(prec, False)
            stm, flagsm = ctx.status_sync()
            submit_check(name)
            err = {c: float((x - ref[c]).abs().max() / ref[c].abs().max()) for c, x in sl().items()}
            err["gloc_diag_abs"] = float(np.abs(gd_host.numpy()[k + 1:] - gd[k + 1:]).max())
            msm, profm = max_over_ranks(rm["ms"]), rm["prof"]
            vm = nk * K / (msm / 1e3)
            cmacs = profm["bulk_flops"] / (8.0 * w.nf ** 3)
            modes[name] = {
                "value": vm, "unit": "k-point timesteps/s", "ms_per_step": msm / K, "dtype": name,
                "speedup_vs_f64": vm / value, "max_rel_err_vs_f64_final_slice": err,
                "e2e_window": {"value": nk * K / max_over_ranks(rm["window_s"]), "unit": "k-point timesteps/s"},
                "bulk_kernel": {"kernel": kern,
                                "algorithmic_fp64_equiv_tflops": profm["bulk_flops"] / (profm["bulk_ms"] / 1e3) / 1e12,
                                "history_gbs": cmacs * bytes_per_elem[name] / (profm["bulk_ms"] / 1e3) / 1e9,
                                "hbm_frac_of_measured": None,
                                "avg_launch_ms": profm["bulk_ms"] / max(1, profm["bulk_launches"]),
                                "share_of_timed": profm["bulk_ms"] / rm["ms"]},
                "clocks": rm["clk"], "device_status": {"status": stm, "flags": flagsm}}
            hbm = measured_hbm_gbs()
            if hbm:
                modes[name]["bulk_kernel"]["hbm_frac_of_measured"] = modes[name]["bulk_kernel"]["history_gbs"] / hbm
    if rank != 0:
        if dist:
            torch.distributed.destroy_process_group()
        return
    oracle_err = None
    if pending:
        oracle_err = {"step": w.nt, "k_points": [kb0 + kb for kb in check_kbs],
                      "what": "the oracle's Dyson time step n = nt of each listed k-point from the GPU's own history, "
                              "self-energy and eps_mf of its last corrector pass, against the GPU's slice n; "
                              "max |gpu - oracle| / max |oracle| per component, worst k-point"}
        for name, res in pending.items():
            per = res.get(timeout=1800)
            oracle_err[name] = {c: max(p[c] for p in per) for c in ("ret", "les", "tv")}
        pool.close()
    line = {
        "metric": "k-point timesteps/s", "value": value, "unit": "k-point timesteps/s",
        "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": ms / K, "higher_is_better": True,
        "scaling": "strong" if dist else "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(w, K, W, world),
        "max_rel_err_vs_oracle": oracle_err,
        "e2e": {"value": e2e_value, "unit": "k-point timesteps/s", "h2d_bytes_per_step": h2d_bytes,
                "d2h_bytes_per_step": d2h_bytes,
                "scope": "whole job through ng_run_2b_host (the C-ABI driver with host buffers): setup (Matsubara "
                         "loop, bootstrapping) and every time step; each step copies eps_k(t_n) from pinned host "
                         "memory to the device and Gloc^<(t_n, t_n) back",
                "window": {"value": e2e_window, "unit": "k-point timesteps/s",
                           "scope": "the timed window's steps only, same call, host clock"}},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic, "traffic_note": traffic_note,
                     "kernel": "k_step_bulk<1>",
                     "peak_source": f"FP64 DFMA from unit counts: {sms} SMs (device property) x "
                                    f"{FP64_FLOP_PER_CLK_PER_SM} flop/clk x median SM clock {clk.get('sm_mhz')} MHz; "
                                    f"measured by ng_fp64_probe in this run: {probe}",
                     "avg_launch_ms": prof["bulk_ms"] / bulk_launches,
                     "share_of_timed": prof["bulk_ms"] / r["ms"],
                     "tv_source_fft_share_of_timed": prof["tvfft_ms"] / r["ms"],
                     "boundary_share_of_timed": prof["boundary_ms"] / r["ms"]},
        "gpu_launches": launches, "clocks": clk,
        "device_status": {"status": st, "flags": flags},
        "observables": {"N_loc_first_timed": float(np.real(-1j * gd[n_first_timed, 0, 0])),
                        "N_loc_last": float(np.real(-1j * gd[-1, 0, 0]))},
        "properties": properties,
    }
    line.update(modes)
    if world == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, list(range(n_first_timed, w.nt + 1)))
    print(json.dumps(line), flush=True)
    if dist:
        torch.distributed.destroy_process_group()


def measured_hbm_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return None


def run_dimer(a):
    """The Hubbard dimer of the paper's quench example at its stated size (nf = 2, J = 1,
    U: 1 -> 2 at t = 0, beta = 20, ntau = 400, nt = 1000, h = 0.02, k = 5, 3 corrector passes):
    the whole self-consistent second-Born run (Matsubara loop, bootstrapping, every time step)
    timed with CUDA events, the particle number and the Galitskii-Migdal total energy for
    t >= 0 (conserved by the second-Born dynamics after the quench), the same at h / 2
    (nt = 2000, same t_max) to show the drift falling with the step, and the oracle's time
    step n = nt from the GPU's history."""
    import multiprocessing as mp

    import numpy as np
    import torch
    import paper_1911_01211_gb300 as ng
    from paper_1911_01211_gb300 import workloads as wl
    pool = mp.get_context("spawn").Pool(1) if not a.no_oracle_check else None
    out = {}
    for label, nt, h in (("h", 1000, 0.02), ("h/2", 2000, 0.01)):
        w = wl.hubbard_dimer(nt=nt, h=h)
        g = ng.Grid(nt=w.nt, ntau=w.ntau, nf=2, nbatch=1, korder=w.korder, h=w.h, beta=w.beta)
        ctx = ng.Context(w.korder)
        G = ng.Herm(g)
        L, S = ng.Herm(g, ldk=1), ng.Herm(g, ldk=1)
        e0 = ng.Func(g, values=torch.from_numpy(w.eps0))
        mf = ng.Func(g)
        U = ng.Func(g, scalar=True)
        U.val[:, 0, 0, 0] = torch.from_numpy(w.U.astype(complex))
        torch.cuda.synchronize()
        clocks = ClockSampler(0)
        clocks.start()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        its = ctx.run_2b(g, G, L, S, e0, mf, U, corrector=w.corrector, mats_tol=1e-14, boot_tol=1e-14)
        ev1.record()
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = ev0.elapsed_time(ev1)
        st = ctx.status_sync()
        obs = torch.zeros(5, dtype=torch.float64, device="cuda")
        E, N = [], []
        for n in range(0, w.nt + 1, max(1, w.nt // 200)):
            ctx.observables(g, n, G, S, e0, mf, obs)
            v = obs.cpu().numpy()
            N.append(v[0])
            E.append(v[4])
        E, N = np.array(E), np.array(N)
        res = {"nt": nt, "h": h, "time_s": ms / 1e3, "timesteps_per_s": (w.nt - w.korder) / (ms / 1e3),
               "setup_iterations": its, "E_tot_drift_t_ge_0": float(np.ptp(E)), "E_tot_t0": float(E[0]),
               "N_drift": float(np.ptp(N)), "N_mean": float(N.mean()), "clocks": clk,
               "device_status": {"status": st[0], "flags": st[1]}}
        if pool is not None and label == "h":
            args = oracle_check_args(ng, g, w.nt, G, S, mf, [0])
            res["max_rel_err_vs_oracle_step_nt"] = pool.map(_oracle_step_check, args)[0]
        if label == "h":
            # the same run again on a fresh context, split into setup (Matsubara loop,
            # bootstrapping) and time steps, the steps with the library's per-launch profile
            # record (CUDA events on its stream): bulk launch, boundary, flops of the bulk
            ctx2 = ng.Context(w.korder)
            G2, L2, S2, mf2 = ng.Herm(g), ng.Herm(g, ldk=1), ng.Herm(g, ldk=1), ng.Func(g)
            kw = dict(corrector=w.corrector, mats_tol=1e-14, boot_tol=1e-14)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx2.run_2b(g, G2, L2, S2, e0, mf2, U, n_to=w.korder, **kw)
            torch.cuda.synchronize()
            t_setup = time.perf_counter() - t0
            ctx2.profile_enable(True)
            e2a, e2b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e2a.record()
            ctx2.run_2b(g, G2, L2, S2, e0, mf2, U, n_from=w.korder + 1, do_setup=False, **kw)
            e2b.record()
            torch.cuda.synchronize()
            prof = ctx2.profile_read()
            ctx2.profile_enable(False)
            ms2 = e2a.elapsed_time(e2b)
            peak = fp64_peak_tflops(clk.get("sm_mhz") or 2070.0)
            bulk_tf = prof["bulk_flops"] / (prof["bulk_ms"] * 1e-3) / 1e12 if prof["bulk_ms"] > 0 else None
            res["split"] = {"setup_s": t_setup, "steps_ms_per_step": ms2 / (w.nt - w.korder),
                            "bulk_share_of_steps": prof["bulk_ms"] / ms2,
                            "boundary_share_of_steps": prof["boundary_ms"] / ms2, "profile": prof}
            res["roofline"] = {"bound": "alu", "achieved": bulk_tf, "peak": peak, "unit": "TFLOP/s",
                               "frac": bulk_tf / peak if bulk_tf else None, "traffic": None,
                               "kernel": "k_step_bulk_w<2>"}
            ctx2.close()
            del G2, L2, S2
        out[label] = res
        ctx.close()
        del G, L, S
        torch.cuda.empty_cache()
    if pool is not None:
        pool.close()
    r = out["h"]
    line = {"metric": "timesteps/s (Hubbard dimer, second-Born quench)", "value": r["timesteps_per_s"],
            "unit": "timesteps/s", "n_gpus": 1, "steps": 1000 - 5, "warmup": 0, "ms_per_step": 1e3 * r["time_s"] / 995,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "hubbard_dimer nf=2 J=1 U 1->2 at t=0 beta=20 ntau=400 nt=1000 h=0.02 k=5 "
                                   "corrector=3 (whole run: Matsubara loop, bootstrapping, time steps)"},
            "roofline": out["h"].get("roofline"),
            "runs": out,
            "drift_ratio_h_over_h2": out["h"]["E_tot_drift_t_ge_0"] / max(out["h/2"]["E_tot_drift_t_ge_0"], 1e-300)}
    print(json.dumps(line), flush=True)


def run_gw(a):
    """k-space GW of the 1D Hubbard chain (the paper's GW example: nk = 128 momenta, U = 2,
    nt = 2500; here ntau = 400, beta = 10, h = 0.02, k = 5, 3 corrector passes, the Peierls pulse
    of chain_kspace): ng_run_gw_kspace with Sigma_k from the momentum sums (lattice FFTs), chi_k by
    the batched bosonic vie2.  Setup and W warm-up steps are a first call; the timed window is the
    remaining steps, CUDA events around one call, with the Dyson bulk kernel and the whole GW
    evaluation timed per launch by the library's profile record."""
    import numpy as np
    import torch
    import paper_1911_01211_gb300 as ng
    from paper_1911_01211_gb300 import workloads as wl
    w = wl.chain_kspace(nk=a.gw_nk, nt=a.gw_nt, ntau=400, beta=10.0, h=0.02, U=2.0)
    g = ng.Grid(nt=w.nt, ntau=w.ntau, nf=1, nbatch=w.nbatch, korder=w.korder, h=w.h, beta=w.beta)
    ctx = ng.Context(w.korder)
    G, S, X = ng.Herm(g), ng.Herm(g), ng.Herm(g)
    L = ng.Herm(g, ldk=1)
    e0 = ng.Func(g, values=torch.from_numpy(w.eps0))
    mf = ng.Func(g)
    U = ng.Func(g, scalar=True)
    U.val[:, 0, 0, 0] = torch.from_numpy(w.U.astype(complex))
    W = max(3, a.warmup)
    n_w = w.korder + W
    t0 = time.perf_counter()
    its = ctx.run_gw_kspace(g, G, L, S, X, e0, mf, U, corrector=w.corrector, n_to=n_w)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    n_to = w.nt if a.steps <= 0 else min(w.nt, n_w + a.steps)
    K = n_to - n_w
    clocks = ClockSampler(0)
    clocks.start()
    ctx.profile_enable(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    ctx.run_gw_kspace(g, G, L, S, X, e0, mf, U, corrector=w.corrector, n_from=n_w + 1, n_to=n_to, do_setup=False)
    ev1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    ms = ev0.elapsed_time(ev1)
    st = ctx.status_sync()
    obs = torch.zeros(5, dtype=torch.float64, device="cuda")
    E, N = [], []
    for n in range(0, n_to + 1, max(1, n_to // 100)):
        ctx.observables(g, n, G, S, e0, mf, obs)
        v = obs.cpu().numpy()
        N.append(v[0])
        E.append(v[4])
    peak = fp64_peak_tflops(clk.get("sm_mhz") or 2070.0)
    bulk_tf = prof["bulk_flops"] / (prof["bulk_ms"] * 1e-3) / 1e12 if prof["bulk_ms"] > 0 else None
    line = {"metric": "k-point timesteps/s (k-space GW chain)", "value": w.nbatch * K / (ms / 1e3),
            "unit": "k-point timesteps/s", "n_gpus": 1, "steps": K, "warmup": W, "ms_per_step": ms / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"chain_kspace GW nk={w.nbatch} nt={w.nt} ntau={w.ntau} h={w.h} beta={w.beta} "
                                   f"U=2 k={w.korder} corrector={w.corrector} (k-space GW, Eqs. Sigmak/Pol, Peierls "
                                   f"pulse)", "timed": f"steps {n_w + 1}..{n_to} (setup and {W} warm-up steps untimed)"},
            "roofline": {"bound": "alu", "achieved": bulk_tf, "peak": peak, "unit": "TFLOP/s",
                         "frac": bulk_tf / peak if bulk_tf else None, "traffic": None, "kernel": "k_step_bulk<1>",
                         "share_of_timed": prof["bulk_ms"] / ms},
            "gw_chain_share_of_timed": prof["gw_ms"] / ms, "gw_chain_ms_per_eval": prof["gw_ms"] / max(prof["gw_evals"], 1),
            "setup": {"s": t_setup, "iterations": its},
            "E_tot_drift_after_pulse": float(np.ptp(E[len(E) // 2:])), "N_drift": float(np.ptp(N)),
            "clocks": clk, "device_status": {"status": st[0], "flags": st[1]}}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_uneven(a):
    """Uneven batch of independent embedded clusters (nf in {1,2,4,8}, nt in [500,3000],
    ntau = 300, beta in [5,30], h = 0.02, 4-site baths): the whole batch solve (Matsubara and
    start-up of every problem, bulk block-size tuning, all global time steps) is timed; the
    unit is problem timesteps (sum over problems of nt - k)."""
    import numpy as np
    import torch
    import paper_1911_01211_gb300 as ng
    from paper_1911_01211_gb300 import workloads as wl
    probs = [p for p in wl.uneven_clusters(nprob=a.nprob) if p["nf"] <= a.max_nf]
    ctx = ng.Context(5)
    grids, Gs, Ss, es = [], [], [], []
    for p in probs:
        g = ng.Grid(nt=p["nt"], ntau=p["ntau"], nf=p["nf"], nbatch=1, korder=5, h=p["h"], beta=p["beta"])
        gb = ng.Grid(nt=p["nt"], ntau=p["ntau"], nf=4, nbatch=1, korder=5, h=p["h"], beta=p["beta"])
        bath = ng.Herm(gb)
        ctx.green_from_H_const(gb, bath, p["hb"][None])
        S = ng.Herm(g)
        ctx.herm_sandwich(g, S, gb, bath, p["V"])
        del bath
        e = ng.Func(g)
        e.val[:] = torch.from_numpy(np.asarray(p["hs"], complex))[None, :, :, None]
        grids.append(g), Gs.append(ng.Herm(g)), Ss.append(S), es.append(e)
    torch.cuda.synchronize()
    batch = ctx.batch(grids, Gs, Ss, es)
    clocks = ClockSampler(0)
    clocks.start()
    ctx.profile_enable(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    threads = batch.solve()
    ev1.record()
    torch.cuda.synchronize()
    ctx.profile_enable(False)
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    prof = ctx.profile_read()
    st, flags = ctx.status_sync()
    units = sum(p["nt"] - 5 for p in probs)
    achieved = prof["bulk_flops"] / (prof["bulk_ms"] / 1e3) / 1e12
    peak = fp64_peak_tflops(clk.get("sm_mhz"))
    line = {"metric": "problem timesteps/s (uneven batch)", "value": units / (ms / 1e3), "unit": "problem timesteps/s",
            "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"uneven_clusters nprob={a.nprob} seed=191101211 nf in (1,2,4,8) nt in [500,3000] "
                                   f"ntau=300 h=0.02 beta in [5,30] 4-site bath V~N(0,0.3^2), fixed Sigma"
                                   + (f"; the {len(probs)} problems with nf <= {a.max_nf}" if a.max_nf < 8 else ""),
                       "nf_counts": {str(d): sum(1 for p in probs if p["nf"] == d) for d in (1, 2, 4, 8)},
                       "timed": "whole batch solve: setup of every problem, block-size tuning, all global steps"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "k_ubulk",
                         "share_of_timed": prof["bulk_ms"] / ms},
            "tuned_threads": threads, "clocks": clk, "device_status": {"status": st, "flags": flags}}
    if a.compare_plain:
        # the plain GPU form on the same problems: one problem after another through
        # ng_solve_fixed (Matsubara, start-up, every time step of that problem alone)
        for G in Gs:
            for x in G.tensors().values():
                x.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for g, G, S, e in zip(grids, Gs, Ss, es):
            ctx.solve_fixed(g, G, S, e)
        e1.record()
        torch.cuda.synchronize()
        ms_plain = e0.elapsed_time(e1)
        line["plain_form"] = {"value": units / (ms_plain / 1e3), "unit": "problem timesteps/s", "ms": ms_plain,
                              "what": "same problems solved one after another with ng_solve_fixed",
                              "batch_speedup": ms_plain / ms}
    print(json.dumps(line), flush=True)
    batch.close()


def run_adjoint(a):
    """Gradient dE_kin(t_N)/dA(t_n), n = 1..N, on the square_kspace model (16 x 16 k-points,
    nt = 1000, ntau = 400, h = 0.02, beta = 10, U = 1.5, 3 corrector passes, Peierls pulse
    A0 = 0.5, omega = 2, t0 = 5, sigma = 1.5): FP64 forward (Matsubara loop, bootstrapping, all
    time steps) and the discrete adjoint, each timed with CUDA events; the gradient is checked
    against central finite differences of the GPU forward at several steps (default 1e-4, 1e-5,
    1e-6) and against the fourth-order stencil (delta = 1e-3) on seeded slices."""
    import numpy as np
    import torch
    import paper_1911_01211_gb300 as ng
    from paper_1911_01211_gb300 import workloads as wl
    from paper_1911_01211_gb300.adjoint import densities
    L, nt, ntau, beta, h, U = 16, a.adj_nt, 400, 10.0, 0.02, 1.5
    g = ng.Grid(nt=nt, ntau=ntau, nf=1, nbatch=L * L, korder=5, h=h, beta=beta)
    ctx = ng.Context(5)
    kx, ky = np.meshgrid(2 * np.pi * np.arange(L) / L, 2 * np.pi * np.arange(L) / L, indexing="ij")
    kx = torch.as_tensor(kx.ravel(), device="cuda")
    ky = torch.as_tensor(ky.ravel(), device="cuda")
    t = np.concatenate([[0.0], h * np.arange(nt + 1)])
    A0 = wl.pulse_A(t)
    A0[0] = 0.0
    Ut = torch.full((nt + 2,), U, dtype=torch.float64, device="cuda")

    def loss(A, segment=0):
        e0 = -2.0 * torch.cos(kx[None, :] - A[:, None]) - 2.0 * torch.cos(ky[None, :])
        rho = densities(e0, ctx, g, Ut, segment=segment)
        return (rho[nt].real * e0[nt + 1]).mean()

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    At = torch.tensor(A0, dtype=torch.float64, device="cuda", requires_grad=True)
    loss(At)            # warm-up (context workspaces, library load)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    ev[0].record()
    Lv = loss(At)
    ev[1].record()
    Lv.backward()
    ev[2].record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_fwd, t_bwd = ev[0].elapsed_time(ev[1]) / 1e3, ev[1].elapsed_time(ev[2]) / 1e3
    grad = At.grad.cpu().numpy()
    # the same gradient with every corrector iterate kept by the forward (no recomputation)
    Ar = torch.tensor(A0, dtype=torch.float64, device="cuda", requires_grad=True)
    torch.cuda.synchronize()
    ev[0].record()
    Lr = loss(Ar, segment=ng.NG_ADJ_RECORDED)
    ev[1].record()
    Lr.backward()
    ev[2].record()
    torch.cuda.synchronize()
    t_fwd_rec, t_bwd_rec = ev[0].elapsed_time(ev[1]) / 1e3, ev[1].elapsed_time(ev[2]) / 1e3
    grad_rec = Ar.grad.cpu().numpy()
    recorded = {"forward_s": t_fwd_rec, "backward_s": t_bwd_rec, "backward_over_forward": t_bwd_rec / t_fwd_rec,
                "max_abs_diff_vs_checkpointed": float(np.abs(grad_rec - grad).max()),
                "iterate_store_gb": 16e-9 * (nt - 5) * 3 * ((L * L + 2) * (2 * nt + ntau + 3) + L * L),
                "what": "ng_adjoint_forward keeps every corrector iterate; ng_adjoint_2b(segment=NG_ADJ_RECORDED) "
                        "walks back without recomputing the forward"}
    del Lr, Ar
    rng = np.random.default_rng(191101211)
    idx = sorted(rng.choice(np.arange(2, nt + 2), a.fd_slices, replace=False).tolist()) if a.fd_slices > 0 else []
    # Finite differences of the GPU forward.  A(t_n) (index i = n + 1) enters the run from step
    # n on, so a perturbed forward restarts there (ng_run_2b from n_from = n without the setup,
    # keeping the unperturbed slices < n); runs go from the latest restart to the earliest, so
    # every run finds unperturbed slices below its restart.  Slices n <= k need the full run.
    Gf = ng.Herm(g)
    Lf, Sf = ng.Herm(g, ldk=1), ng.Herm(g, ldk=1)
    e0f, mff = ng.Func(g), ng.Func(g)
    Uf = ng.Func(g, scalar=True)
    Uf.val[:, 0, 0, 0] = U
    diag = ng.tri(nt) + nt

    def set_eps(A):
        At_ = torch.as_tensor(A, device="cuda")
        e0f.val[:, 0, 0, :] = (-2.0 * torch.cos(kx[None, :] - At_[:, None]) - 2.0 * torch.cos(ky[None, :])).to(
            torch.complex128)

    def ekin_final():
        rho = -1j * Gf.les[diag, 0, 0, :]
        return float((rho.real * e0f.val[nt + 1, 0, 0, :].real).mean().item())

    def forward(A, n_from):
        set_eps(A)
        if n_from > 5:
            ctx.run_2b(g, Gf, Lf, Sf, e0f, mff, Uf, corrector=3, n_from=n_from, do_setup=False)
        else:
            ctx.run_2b(g, Gf, Lf, Sf, e0f, mff, Uf, corrector=3, mats_tol=1e-14, boot_tol=1e-14)
        return ekin_final()

    deltas = [float(x) for x in a.fd_deltas.split(",")] if a.fd_deltas else [1e-6]
    stencils = [(f"central_{d:g}", d, ((1.0, 1.0), (-1.0, -1.0)), 2 * d) for d in deltas]
    stencils.append(("fourth_order_0.001", 1e-3, ((2.0, -1.0), (1.0, 8.0), (-1.0, -8.0), (-2.0, 1.0)), 12e-3))
    jobs = []
    for i in idx:
        for name, d, taps, den in stencils:
            for sgn, coef in taps:
                jobs.append((i - 1, i, name, sgn * d, coef, den))
    jobs.sort(key=lambda j: -max(j[0], 0))
    forward(A0, 0)                      # unperturbed base state
    acc = {}
    t_fd = time.perf_counter()
    with torch.no_grad():
        for n_from, i, name, dA, coef, den in jobs:
            A = A0.copy()
            A[i] += dA
            v = forward(A, n_from)
            acc[(name, i)] = acc.get((name, i), 0.0) + coef * v / den
    t_fd = time.perf_counter() - t_fd
    fd_report = {}
    gi = grad[idx] if idx else np.zeros(0)
    for name, d, _, _ in stencils if idx else []:
        fd = np.array([acc[(name, i)] for i in idx])
        per = [float(abs(x - y) / max(abs(y), 1e-300)) for x, y in zip(gi, fd)]
        fd_report[name] = {"delta": d, "max_rel_err_normwise": float(np.abs(gi - fd).max() / np.abs(fd).max()),
                           "max_rel_err_per_slice": max(per), "median_rel_err_per_slice": float(np.median(per))}
    units = L * L * (nt - 5)
    line = {"metric": "adjoint gradient k-point timesteps/s", "value": units / t_bwd,
            "unit": "k-point timesteps/s (backward sweep)", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": 1e3 * t_bwd / (nt - 5), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"square_kspace 16x16 nt={nt} ntau={ntau} h={h} beta={beta} U={U} k=5 corrector=3, "
                                   "loss E_kin(t_N), parameters A(t_1..t_N)",
                       "segment_steps": int(np.ceil(np.sqrt(nt - 5)))},
            "forward_s": t_fwd, "backward_s": t_bwd, "backward_over_forward": t_bwd / t_fwd,
            "recorded_iterates": recorded,
            "loss": Lv.item(),
            "fd_check": {"slices": [int(i) - 1 for i in idx],
                         "how": "central differences of the GPU forward at each delta and the fourth-order stencil "
                                "(delta = 1e-3), perturbed forwards restarted at the perturbed slice",
                         "stencils": fd_report, "seconds": t_fd},
            "grad_norm_inf": float(np.abs(grad).max()), "clocks": clk,
            "device_status": dict(zip(("status", "flags"), ctx.status_sync()))}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "uneven":
        run_uneven(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    elif args.workload == "dimer":
        run_dimer(args)
    elif args.workload == "gw":
        run_gw(args)
    else:
        run_ours(args)
