#!/usr/bin/env python
"""Benchmark of the variational HCI hot path on GB300.

One step = one pass of the whole path on one active space:
  rotate the integrals by U = exp(kappa)          (a0)
  heat-bath lists, selection loop with Davidson    (a1-a6, hci_solve)
  1- and 2-RDM                                    (a7)
  dE/dkappa through the rotation adjoint           (a8)
on the synthetic (44e,44o) density-fitted Hamiltonian at eps1 = 1e-4.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# The batched solve runs one stream per in-flight instance (16 at the
# autotuned setting); with the default 8 hardware work queues pairs of
# streams share one and their kernels wait on each other.  Read when the
# process creates its CUDA context, so it is set before torch touches CUDA.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import numpy as np  # noqa: E402

import hci_inputs as hi  # noqa: E402

METRIC = "(44e,44o) HCI solve+2-RDM seconds"

WORKLOADS = {
    "df44": {"make": hi.df_44o, "eps1": 1e-4,
             "desc": "synthetic DF (44e,44o), naux=176, w_P=exp(-P/40), 0.3 Ha gap, eps1=1e-4"},
    "pentacene22": {"make": hi.ppp_pentacene, "eps1": 5e-5,
                    "desc": "PPP pentacene-shaped lattice (22e,22o), Hueckel MOs, eps1=5e-5"},
    "pentacene22_e4": {"make": hi.ppp_pentacene, "eps1": 1e-4,
                       "desc": "PPP pentacene-shaped lattice (22e,22o), Hueckel MOs, eps1=1e-4 (profiling size)"},
    "df12": {"make": hi.df_12o, "eps1": 1e-3, "desc": "synthetic DF (12e,12o), naux=48, eps1=1e-3"},
    "polyene8": {"make": lambda: hi.ppp_polyene(8), "eps1": 1e-4, "desc": "PPP 8-site polyene (8e,8o)"},
}

# Work structure of one solve of each workload (selection source passes,
# sigma row passes, sigma connection passes), as counted by the library's
# own counters (hci_stats) in a bench run on GB300 at DAV_TOL; the reference
# arm, which runs no GPU code, scales its sampled per-row and per-source
# oracle costs by these.  The GPU arm's cpu_baseline uses the counters of its
# own run instead, and each JSON line records the counts it used.
WORK_PROFILE = {
    "df44": {"select_sources": 18311266, "sigma_rows": 256134997, "sigma_nnz": 488299005664},
}

DAV_TOL = 1e-10     # Davidson residual ||Hc - Ec||_2 at every selection (the parity tests' value)
PT2_EPS2 = 1e-5      # eps2 of the perturbative correction (the paper's HCISCF value)
PT2_SS_EPS2 = 1e-6   # semistochastic correction: tighter eps2, sampled on top of E2^D(PT2_EPS2)
PT2_SS_DRAWS = 1000
PT2_SS_SAMPLES = 10
DAV_MAXIT = 400


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="df44", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="budget of one CPU sample")
    ap.add_argument("--sigma-reps", type=int, default=20)
    ap.add_argument("--rotation-reps", type=int, default=20, help="launches of the quarter transform timed alone")
    ap.add_argument("--fwd-bwd-reps", type=int, default=5)
    ap.add_argument("--pt2-reps", type=int, default=2)
    ap.add_argument("--direct-reps", type=int, default=2)
    ap.add_argument("--batch", type=int, default=1, help="also time the 64-instance batched solve")
    ap.add_argument("--sigma-mode", default="auto", choices=["auto", "stored", "half", "direct"],
                    help="connection-graph form of the timed step and the sigma section (hci_set_sigma_mode)")
    ap.add_argument("--large", type=int, default=1,
                    help="also time one solve + RDMs of the ~1e7-determinant (44e,44o) space")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# DRAM traffic of one sigma launch per (connection, row), from the ncu
# capture of k_sigma1 on the pentacene (22e,22o) space (profiles/);
# traffic grows in proportion to the connections, so it is scaled to the
# launch.  None while the kernel differs from the captured one.
SIGMA_TRAFFIC_PER_CONN = 12.40


def traffic_per_launch(nnz, nV):
    if SIGMA_TRAFFIC_PER_CONN is None:
        return None
    return int(SIGMA_TRAFFIC_PER_CONN * (nnz + nV))


def max_over_ranks(value, world, device=None):
    """Largest value over the ranks of the default process group."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_seconds(ms_per_step_max, world):
    """Replicas: every rank solves one instance per step, so the whole job
    completes `world` solves per (max-over-ranks) step time."""
    return ms_per_step_max / 1e3 / world


def fp64_peak_tflops(dev):
    """FP64 rate of the part: SMs x 2 DFMA per clock x 2 flop at the maximum
    SM clock (152 x 2 x 2 x 2.07 GHz = 1.26 TFLOP/s on GB300, consistent
    with the nominal 1.25 TFLOP/s; the sigma kernel's ncu capture shows one
    FP64 warp instruction per 16 cycles per SM at full pipe utilisation).
    The SM count is the device's, the clock the measured maximum."""
    import torch

    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = 2070.0
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            mhz = float(json.load(fh).get("sm_max_mhz", mhz))
    return nsm * 2 * 2 * mhz * 1e6 / 1e12, f"derived FP64 ({nsm} SM x 2 DFMA/clk x {mhz / 1e3:.2f} GHz)"


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def gpu_arm(args):
    import torch
    import torch.distributed as dist

    import paper_1708_07544_gb300 as pkg
    from paper_1708_07544_gb300 import _abi

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    wl = WORKLOADS[args.workload]
    inst = wl["make"]()
    eps1 = wl["eps1"]
    n = inst.norb
    kap = hi.random_kappa(n, seed=1709, sigma=0.01)
    h_d = torch.tensor(inst.h, device=dev)
    eri_d = torch.tensor(inst.eri, device=dev)
    k_d = torch.tensor(kap, device=dev)
    cap = 1 << 22
    sigma_mode = {"auto": _abi.SIGMA_AUTO, "stored": _abi.SIGMA_STORED, "half": _abi.SIGMA_HALF,
                  "direct": _abi.SIGMA_DIRECT}[args.sigma_mode]

    def step(h_in, eri_in, k_in, record=None):
        U, h2, e2 = _abi.hci_rotate(k_in, h_in, eri_in)
        s = pkg.HCISolver(n, inst.nalpha, inst.nbeta, h2, e2, inst.e_core)
        try:
            s.set_sigma_mode(sigma_mode)
            s.profile(True)
            keys, c, E, it = _abi.hci_solve(s.ctx, eps1, 30, DAV_TOL, DAV_MAXIT, cap, device=dev)
            r1, r2 = s.rdm12(keys, c)
            dh, de, dk = _abi.hci_rotate_backward(k_in, h_in, eri_in, r1, r2, want_dh=False, want_deri=False)
            if record is not None:
                record["timers"] = s.timers()
                record["stats"] = s.stats()
                record["nV"] = int(keys.shape[0])
                record["E"] = E
                record["iters"] = it
                record["keys"] = keys
                record["c"] = c
                record["rdm"] = (r1, r2)
        finally:
            s.close()
        return E, r1, r2, dk

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up
    for w in range(max(args.warmup, 0)):
        step(h_d, eri_d, k_d)
    # timed region: device-resident inputs
    clocks = Clocks(local)
    barrier()
    clocks.start()
    l0 = _abi.hci_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.nvtx.range_push("timed_steps")
    ev0.record()
    recs = []
    rec = {}
    for _ in range(args.steps):
        rec = {}
        step(h_d, eri_d, k_d, rec)
        recs.append({k: rec[k] for k in ("timers", "stats", "nV", "E", "iters")})
    ev1.record()
    torch.cuda.nvtx.range_pop()
    barrier()
    launches = _abi.hci_launch_count() - l0
    clk = clocks.stop()
    ms_step = max_over_ranks(ev0.elapsed_time(ev1), world, dev) / args.steps

    # end-to-end through the public API with host buffers (H2D of the
    # integrals and kappa, D2H of E, rdm1, rdm2 and dE/dkappa every step)
    h_host = torch.tensor(inst.h).pin_memory()
    eri_host = torch.tensor(inst.eri).pin_memory()
    k_host = torch.tensor(kap).pin_memory()
    r1_host = torch.empty((n, n), dtype=torch.float64).pin_memory()
    r2_host = torch.empty((n,) * 4, dtype=torch.float64).pin_memory()
    dk_host = torch.empty((n, n), dtype=torch.float64).pin_memory()
    h_e = torch.empty_like(h_d)
    eri_e = torch.empty_like(eri_d)
    k_e = torch.empty_like(k_d)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        h_e.copy_(h_host, non_blocking=True)
        eri_e.copy_(eri_host, non_blocking=True)
        k_e.copy_(k_host, non_blocking=True)
        E, r1, r2, dk = step(h_e, eri_e, k_e)
        r1_host.copy_(r1, non_blocking=True)
        r2_host.copy_(r2, non_blocking=True)
        dk_host.copy_(dk, non_blocking=True)
    e1.record()
    barrier()
    e2e_step = max_over_ranks(e0.elapsed_time(e1), world, dev) / args.steps
    h2d = (n * n + n ** 4 + n * n) * 8
    d2h = (n * n + n ** 4 + n * n) * 8 + 8

    # sigma roofline on the converged space: the sigma kernel alone
    last = rec
    U, h2, e2 = _abi.hci_rotate(k_d, h_d, eri_d)
    s = pkg.HCISolver(n, inst.nalpha, inst.nbeta, h2, e2, inst.e_core)
    s.set_sigma_mode(sigma_mode)
    keys, c = last["keys"], last["c"]
    s.sigma(keys, c)                 # builds the graph
    s.timers()
    s.profile(True)
    sig = torch.empty_like(c)
    cc = c.clone()
    torch.cuda.nvtx.range_push("sigma_reps")
    for _ in range(args.sigma_reps):
        sig = s.sigma(keys, cc)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    tm = s.timers()
    st = s.stats()
    # second-order Epstein-Nesbet correction on the converged space at the
    # paper's HCISCF setting eps2 = 1e-5 Ha (host clock around the
    # synchronising call)
    pt2 = {}
    if args.pt2_reps > 0:
        ts = []
        torch.cuda.nvtx.range_push("pt2")
        for _ in range(args.pt2_reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2v, n_ext = s.pt2(keys, c, PT2_EPS2, last["E"])
            ts.append(time.perf_counter() - t0)
        torch.cuda.nvtx.range_pop()
        # the same with the correction's density matrices (Gamma^dd, Gamma^dc)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.pt2(keys, c, PT2_EPS2, last["E"], rdms=True)
        t_rdm = time.perf_counter() - t0
        # the relaxed density of E_var + E2 (z-vector solve included)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.relaxed_rdm12(keys, c, last["E"], PT2_EPS2, zv_tol=1e-9, zv_maxit=500)
        t_rel = time.perf_counter() - t0
        # semistochastic E2 at a tighter eps2 (Eq. semistoc): E2^D at the
        # paper's eps2 plus the sampled difference down to PT2_SS_EPS2
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("pt2_ss")
        t0 = time.perf_counter()
        ss = s.pt2_semistochastic(keys, c, last["E"], PT2_SS_EPS2, PT2_EPS2, PT2_SS_DRAWS, PT2_SS_SAMPLES, seed=1708)
        t_ss = time.perf_counter() - t0
        torch.cuda.nvtx.range_pop()
        pt2 = {"eps2": PT2_EPS2, "E2": e2v, "E_var_plus_E2": last["E"] + e2v, "targets": n_ext,
               "seconds": round(statistics.median(ts), 4), "seconds_with_rdms": round(t_rdm, 4),
               "relaxed_rdm_seconds": round(t_rel, 4), "reps": args.pt2_reps,
               "semistochastic": {"eps2": PT2_SS_EPS2, "eps2_det": PT2_EPS2, "n_draws": PT2_SS_DRAWS,
                                  "n_samples": PT2_SS_SAMPLES, "E2": ss["estimate"], "error": ss["error"],
                                  "E2_det": ss["e2_det"], "seconds": round(t_ss, 4)}}
    s.close()
    # the same H c with the connections searched and evaluated again in every
    # product (no stored graph; the form for spaces whose connections exceed
    # device memory): its first call builds the search structures
    direct = {}
    if args.direct_reps > 0:
        sd = pkg.HCISolver(n, inst.nalpha, inst.nbeta, h2, e2, inst.e_core)
        sd.set_sigma_mode(_abi.SIGMA_DIRECT)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sd_sig = sd.sigma(keys, c)
        torch.cuda.synchronize()
        t_first = time.perf_counter() - t0
        td = []
        for _ in range(args.direct_reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sd_sig = sd.sigma(keys, c)
            torch.cuda.synchronize()
            td.append(time.perf_counter() - t0)
        dev_max = float((sd_sig - sig).abs().max().item())
        st_d = sd.stats()
        sd.close()
        direct = {"sigma_ms": round(1e3 * statistics.median(td), 3), "first_call_ms": round(1e3 * t_first, 3),
                  "connections": st_d["graph_nnz"], "max_abs_diff_vs_stored": dev_max, "reps": args.direct_reps}
    sig_ms = tm["sigma"][0] / max(tm["sigma"][1], 1)
    nnz = st["graph_nnz"]
    nV = int(keys.shape[0])
    half = bool(st["graph_half"])
    # algorithmic bytes of one product: 12 per stored entry (both
    # orientations: one per connection; one orientation: one per pair) and
    # 40 per row (row pointer, row start, diagonal, c_i, sigma_i)
    sig_bytes = 12 * (nnz // 2 if half else nnz) + 40 * nV + 8
    sig_kernel = "k_sigma1_half (one orientation, FP64 atomic scatter)" if half else "k_sigma1 (pooled-CSR FP64 H c)"
    sig_flops = 2 * (nnz + nV)
    peak, peak_kind = measured_peaks()
    fp64_tf, fp64_kind = fp64_peak_tflops(dev)
    achieved = sig_bytes / (sig_ms * 1e-3) / 1e9
    achieved_tf = sig_flops / (sig_ms * 1e-3) / 1e12

    # forward vs forward + backward through the autograd Function (the
    # backward recomputes c by Davidson on the saved space, then the RDMs and
    # the rotation adjoint)
    fb = {}
    if args.fwd_bwd_reps > 0:
        t_f, t_fb = [], []
        for _ in range(args.fwd_bwd_reps):
            kk = k_d.clone().requires_grad_(True)
            e0f = torch.cuda.Event(enable_timing=True)
            e1f = torch.cuda.Event(enable_timing=True)
            e2f = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0f.record()
            E = pkg.HCIEnergy.apply(h_d, eri_d, kk, inst.nalpha, inst.nbeta, inst.e_core, eps1, 30, DAV_TOL)
            e1f.record()
            E.backward()
            e2f.record()
            torch.cuda.synchronize()
            t_f.append(e0f.elapsed_time(e1f))
            t_fb.append(e0f.elapsed_time(e2f))
        fwd = statistics.median(t_f) / 1e3
        fwdbwd = statistics.median(t_fb) / 1e3
        fb = {"fwd_s": round(fwd, 4), "fwd_bwd_s": round(fwdbwd, 4), "ratio": round(fwdbwd / fwd, 4),
              "reps": args.fwd_bwd_reps}

    phases = {}
    for r in recs:
        for k, (ms, cnt) in r["timers"].items():
            a = phases.setdefault(k, [0.0, 0.0])
            a[0] += ms / len(recs)
            a[1] += cnt / len(recs)
    work = recs[-1]["stats"]

    # batching: 64 uneven DF active spaces (norb 10-24) solved concurrently,
    # stream count picked by the autotuner, against one-at-a-time solves
    batch = {}
    if args.batch:
        from paper_1708_07544_gb300 import tune

        binst = hi.df_batch(64)
        lst = [(i.norb, i.nalpha, i.nbeta, torch.tensor(i.h, device=dev), torch.tensor(i.eri, device=dev),
                i.e_core) for i in binst]
        best, tuned = tune.tune_nstreams(lst, 1e-4, want_rdm=True)
        reps = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            en, nv, _, _ = _abi.hci_solve_batch(lst, 1e-4, dav_tol=DAV_TOL, nstreams=best, want_rdm=True)
            torch.cuda.synchronize()
            reps.append(time.perf_counter() - t0)
        seq = tuned.get(1)
        batch = {"instances": len(lst), "total_dets": int(nv.sum()), "max_dets": int(nv.max()),
                 "nstreams": best, "batched_s": round(statistics.median(reps), 4),
                 "sequential_s": round(seq, 4) if seq else None,
                 "speedup": round(seq / statistics.median(reps), 3) if seq else None,
                 "tuning_s": {str(k): round(v, 4) for k, v in tuned.items()},
                 "includes": "solve + 1/2-RDM per instance"}

    # the ~1e7-determinant (44e,44o) space (Fe(P)-sized, Sec. V.C): one
    # solve + RDMs through the same public API, the graph form chosen by
    # HCI_SIGMA_AUTO (both orientations, one orientation, or direct, as
    # device memory allows)
    large = {}
    if args.large:
        linst = hi.df_44o_large()
        lh = torch.tensor(linst.h, device=dev)
        leri = torch.tensor(linst.eri, device=dev)
        _, lh2, le2 = _abi.hci_rotate(k_d, lh, leri)
        sl = pkg.HCISolver(n, linst.nalpha, linst.nbeta, lh2, le2, linst.e_core)
        try:
            sl.profile(True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lk, lc, lE, lit = _abi.hci_solve(sl.ctx, eps1, 30, DAV_TOL, DAV_MAXIT, 1 << 25, device=dev)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            sl.rdm12(lk, lc)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            ltm = sl.timers()
            lst = sl.stats()
            lsig = []
            for _ in range(2):
                torch.cuda.synchronize()
                a0 = time.perf_counter()
                sl.sigma(lk, lc)
                torch.cuda.synchronize()
                lsig.append(time.perf_counter() - a0)
            lnV = int(lk.shape[0])
            form = "direct" if lst["sigma_direct"] else ("one orientation" if lst["graph_half"] else "both orientations")
            lnnz = lst["graph_nnz"]
            large = {"workload": f"synthetic DF (44e,44o), factor scale {hi.DF44_LARGE_SCALE_FACTOR} x sqrt(0.5/sum w_P^2), eps1=1e-4",
                     "nV": lnV, "E": lE, "selections": lit, "solve_s": round(t1 - t0, 3), "rdm_s": round(t2 - t1, 3),
                     "graph_form": form, "graph_nnz": lnnz, "sigma_calls": lst["sigma_calls"],
                     "sigma_ms": round(1e3 * min(lsig), 2),
                     "hc_connections_per_s": (lnnz + lnV) / min(lsig),
                     "stored_bytes": 6 * lnnz if lst["graph_half"] else None,
                     "phases_ms": {k: round(v[0], 1) for k, v in ltm.items() if v[1]}}
        finally:
            sl.close()

    # the rotation's quarter transform alone (Sec. III.A), on the tensor
    # cores: per-launch time over buffers rotated through more than L2, the
    # FP64-equivalent rate 2 n^5 / t, the bf16 tensor work of the digit
    # products against the measured bf16 peak, and its HBM bytes
    rotation = {}
    if args.rotation_reps > 0:
        rotation = rotation_section(args, n, h_d, eri_d, k_d, dev)

    out = None
    if rank == 0:
        value = aggregate_seconds(ms_step, world)
        out = {
            "metric": METRIC,
            "value": round(value, 6),
            "unit": "s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(ms_step, 3),
            "higher_is_better": False,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {wl['desc']}", "norb": n, "nelec": inst.nelec,
                       "nV": recs[-1]["nV"], "graph_nnz": nnz, "selections": recs[-1]["iters"],
                       "E": recs[-1]["E"], "davidson_tol": DAV_TOL,
                       "l2": "inputs larger than L2 (connection graph %.1f GB)" % (sig_bytes / 1e9),
                       "parallelism": f"replicas x{world}"},
            "hc_connections_per_s": (nnz + nV) / (sig_ms * 1e-3),
            "phases_ms": {k: round(v[0], 3) for k, v in phases.items()},
            "phase_counts": {k: v[1] for k, v in phases.items()},
            "work": work,
            "roofline": {"kernel": sig_kernel, "bound": "alu", "achieved": round(achieved_tf, 4),
                         "peak": round(fp64_tf, 4), "unit": "TFLOP/s", "frac": round(achieved_tf / fp64_tf, 4),
                         "traffic": None if half else traffic_per_launch(nnz, nV), "peak_kind": fp64_kind,
                         "flops_per_launch": sig_flops, "launch_ms": round(sig_ms, 4)},
            "roofline_hbm": {"kernel": sig_kernel.split()[0], "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                             "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                             "bytes_per_launch": sig_bytes},
            "fwd_bwd": fb,
            "pt2": pt2,
            "sigma_direct": direct,
            "batch": batch,
            "large": large,
            "rotation": rotation,
            "e2e": {"value": round(aggregate_seconds(e2e_step, world), 6), "unit": "s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "clocks": clk,
        }
    if world > 1:
        dist.barrier()
    return out, last, inst


def qtrans_mma_flops(n):
    """bf16 tensor work of one quarter transform as the kernel issues it:
    per tile of 128 rows, every pair (s, t) of the seven digits of each
    operand with s + t <= 9 (34 pairs), one M=128 x N=np x K=np product each
    (np = n rounded up to 16)."""
    npad = -(-n // 16) * 16
    pairs = sum(min(L - 1, 7) - max(1, L - 7) + 1 for L in range(2, 10))
    tiles = -(-n ** 3 // 128)
    return tiles * pairs * 2 * 128 * npad * npad


def rotation_section(args, n, h_d, eri_d, k_d, dev):
    import torch

    from paper_1708_07544_gb300 import _abi

    U, _, _ = _abi.hci_rotate(k_d, h_d, eri_d)
    n4 = n ** 4
    # enough distinct input/output pairs that each launch misses L2
    nbuf = max(2, int(math.ceil(3 * 129e6 / (16 * n4))) + 1)
    ins = [eri_d.clone() for _ in range(nbuf)]
    outs = [torch.empty_like(eri_d) for _ in range(nbuf)]
    st = torch.cuda.current_stream()
    for i in range(3):
        _abi.hci_qtrans(ins[i % nbuf], U, outs[i % nbuf], check=False, stream=st)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("qtrans_reps")
    e0.record(st)
    for i in range(args.rotation_reps):
        _abi.hci_qtrans(ins[i % nbuf], U, outs[i % nbuf], check=False, stream=st)
    e1.record(st)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    _abi.hci_qtrans(ins[0], U, outs[0], check=True, stream=st)
    t = e0.elapsed_time(e1) / args.rotation_reps * 1e-3
    # whole rotation and its backward (host clock around the synchronising calls)
    r1 = torch.eye(n, dtype=torch.float64, device=dev)
    r2 = torch.zeros((n,) * 4, dtype=torch.float64, device=dev)
    tr, tb = [], []
    for _ in range(5):
        torch.cuda.synchronize()
        a = time.perf_counter()
        _abi.hci_rotate(k_d, h_d, eri_d)
        b = time.perf_counter()
        _abi.hci_rotate_backward(k_d, h_d, eri_d, r1, r2, want_dh=False, want_deri=False)
        tr.append(b - a)
        tb.append(time.perf_counter() - b)
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    pk = {}
    if os.path.exists(path):
        with open(path) as fh:
            pk = json.load(fh)
    bf16 = float(pk.get("bf16_tflops", 1900.0))
    hbm = float(pk.get("hbm_gbs", 6800.0))
    mma = qtrans_mma_flops(n)
    byt = 2 * n4 * 8
    del ins, outs
    return {"kernel": "k_qtrans_tc (digit products on tcgen05 bf16, FP32 in tensor memory, rounded to FP64)",
            "norb": n, "launch_ms": round(t * 1e3, 4), "reps": args.rotation_reps, "buffers": nbuf,
            "fp64_equiv_tflops": round(2 * n ** 5 / t / 1e12, 3),
            "tensor": {"achieved": round(mma / t / 1e12, 1), "peak": bf16, "unit": "TFLOP/s",
                       "frac": round(mma / t / 1e12 / bf16, 4), "flops_per_launch": mma,
                       "peak_kind": "measured" if pk else "fallback"},
            "hbm": {"achieved": round(byt / t / 1e9, 1), "peak": hbm, "unit": "GB/s",
                    "frac": round(byt / t / 1e9 / hbm, 4), "bytes_per_launch": byt},
            "rotate_ms": round(1e3 * min(tr), 3), "rotate_backward_ms": round(1e3 * min(tb), 3)}


# ----------------------------------------------------------------------------
# CPU oracle (cpu_baseline leg and reference arm)
# ----------------------------------------------------------------------------
def oracle_sample(inst, eps1, keys_np, c_np, budget_s, work):
    """Time the CPU oracle on sampled rows and sources of a space and scale to
    one solve with the given work counters."""
    import oracle

    rng = np.random.default_rng(7)
    nV = len(keys_np)
    P = oracle.Problem.of(inst)
    threads = oracle.num_threads()
    # sigma rows
    rows = np.sort(rng.choice(nV, size=min(nV, 64), replace=False))
    t0 = time.perf_counter()
    oracle.sigma_rows(P, keys_np, c_np, rows)
    t_rows = time.perf_counter() - t0
    k = len(rows)
    while t_rows < budget_s * 0.4 and k < nV:
        more = np.sort(rng.choice(nV, size=min(nV, 2 * k), replace=False))
        t0 = time.perf_counter()
        oracle.sigma_rows(P, keys_np, c_np, more)
        t_rows = time.perf_counter() - t0
        k = len(more)
        if t_rows > budget_s * 0.4:
            break
    per_row = t_rows / k
    # selection sources (the largest |c| first: those do the most work)
    order = np.argsort(-np.abs(c_np))
    ns = 16
    t0 = time.perf_counter()
    oracle.select(P, keys_np, c_np, eps1, sources=order[:ns])
    t_src = time.perf_counter() - t0
    while t_src < budget_s * 0.3 and ns < nV:
        ns = min(nV, ns * 2)
        t0 = time.perf_counter()
        oracle.select(P, keys_np, c_np, eps1, sources=order[:ns])
        t_src = time.perf_counter() - t0
    per_src = t_src / ns
    est = per_row * work["sigma_rows"] + per_src * work["select_sources"]
    return est, threads, f"{k} sigma rows and {ns} selection sources (largest |c|) of the sampled space, " \
                         f"scaled by the solve's row passes ({work['sigma_rows']}) and source passes " \
                         f"({work['select_sources']})"


def reference_arm(args):
    """The CPU oracle on a bounded sample of the same workload (host cores).

    The sample space is the oracle's own first selection from the aufbau
    determinant (exact and cheap); the oracle's cost per sigma row and per
    selection source does not depend on the coefficients, so the sampled
    per-unit times are scaled by the solve's row and source passes."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    import oracle

    wl = WORKLOADS[args.workload]
    prof = WORK_PROFILE.get(args.workload)
    if prof is None:
        return {"impl": "reference", "unavailable": f"no work profile recorded for workload {args.workload}"}
    inst = wl["make"]()
    eps1 = wl["eps1"]
    P = oracle.Problem.of(inst)
    k0 = oracle.aufbau(inst.nalpha, inst.nbeta)
    new, _, _ = oracle.select(P, k0, [1.0], eps1)
    keys, c = oracle.merge(k0, [1.0], new)
    c = np.full(len(keys), 1e-3)
    c[np.flatnonzero((keys[:, 0] == k0[0, 0]) & (keys[:, 1] == k0[0, 1]))] = 1.0
    budget = args.cpu_seconds
    vals = []
    desc = ""
    threads = oracle.num_threads()
    for _ in range(args.warmup + args.steps):
        est, threads, desc = oracle_sample(inst, eps1, keys, c, budget, prof)
        vals.append(est)
    vals = vals[args.warmup:]
    value = statistics.median(vals)
    desc = "first selection space from the aufbau determinant (%d dets); " % len(keys) + desc
    return {"metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False, "impl": "reference",
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {wl['desc']}"},
            "cpu_baseline": {"value": value, "unit": "s", "cores": threads, "kind": "oracle", "sample": desc,
                             "work_counts": prof},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    if args.impl == "reference":
        out = reference_arm(args)
        if out is not None:
            print(json.dumps(out))
        return
    out, last, inst = gpu_arm(args)
    if out is None:
        return
    if not args.no_cpu_baseline and int(os.environ.get("WORLD_SIZE", "1")) == 1:
        keys_np = last["keys"].cpu().numpy().view(np.uint64).reshape(-1, 2)
        c_np = last["c"].cpu().numpy()
        est, threads, desc = oracle_sample(inst, WORKLOADS[args.workload]["eps1"], keys_np, c_np,
                                           args.cpu_seconds, out["work"])
        out["cpu_baseline"] = {"value": est, "unit": "s", "cores": threads, "kind": "oracle", "sample": desc,
                               "work_counts": {k: out["work"][k] for k in ("select_sources", "sigma_rows",
                                                                           "sigma_nnz")}}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
