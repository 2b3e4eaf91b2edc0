#!/usr/bin/env python
"""Throughput of composed implicit propagation (trapezoidal rule / implicit
midpoint, GMRES implicit solves, Suzuki / triple-jump composition) on the
synthetic NaI-like two-surface workload, one persistent launch per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step propagates every wavepacket of the batch by one composed time step.
value = propagated wavepacket-steps per second over all ranks (device timed,
inputs resident in HBM); e2e = the same through the C-ABI with the states
copied from pinned host memory and read back every step.  The reference arm
times the dense CPU oracle on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Hψ grid-point-applications/s and propagated steps/s at error 1e-10; % HBM peak"

FS = 41.341373335182
# Operating point: NaI-like model on the paper's grid, implicit midpoint
# composed by Suzuki's fractal to order 8 with dt = t_f / 1024 (t_f = 10500
# a.u.), implicit steps solved to tol 1e-15: the convergence sweeps
# (--sweep) put the error ||psi_dt(t_f) - psi_dt/2(t_f)|| of this point at
# the 1e-10 level; looser solves add an accumulated error of the same size.
WORKLOAD = dict(name="nai_like_n2048_s2_midpoint_suzuki8_dt10.25au", N=2048, S=2, method=1, order=8, scheme=1,
                dt_fs=10500.0 / 1024 / FS, tol=1e-15, restart=30)


def _flops_per_launch(stats, N, S, reorth=True, mixed=False):
    """Algorithmic FP64 flops of the stats' work (complex FFT = 5 n log2 n):
    H psi: 4 S FFTs of length N plus (4 S^2 + 10 S) N pointwise; Arnoldi:
    16 S N per basis vector and Gram-Schmidt pass, 6 S N per iteration for the
    norm and scaling; solution update 8 S N per basis vector.  In the mixed
    form the Krylov work is complex64 and only the FP64 H psi (residuals,
    right-hand sides) and the refinement update (8 S N) count."""
    hpsi = 4 * S * 5 * N * math.log2(N) + (4 * S * S + 10 * S) * N
    ortho = (2 if reorth else 1) * 16 * S * N
    tot = 0.0
    for s in stats:
        if mixed:
            tot += s["n_hpsi"] * hpsi + s["n_outer"] * 8 * S * N
        else:
            tot += s["n_hpsi"] * hpsi + s["n_ortho"] * ortho + s["n_krylov"] * 6 * S * N + s["n_update"] * 8 * S * N
    return tot


def _bytes_per_launch(stats, N, S):
    """Algorithmic DRAM bytes if every vector pass went to HBM: H psi reads psi
    and the fields and writes the result (16 S N + 8 N (S + S(S-1)/2) + 16 S N);
    each Arnoldi basis vector touched is read twice per pass (dot, update)."""
    hpsi = 16 * S * N * 2 + 8 * N * (S + S * (S - 1) // 2)
    tot = 0.0
    for s in stats:
        tot += s["n_hpsi"] * hpsi + s["n_ortho"] * 2 * 2 * 16 * S * N + s["n_update"] * 16 * S * N
    return tot


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def fp64_peak_tflops(sm_mhz=None):
    """FP64 FMA peak: 152 SMs x 2 DFMA/clock (4 flops) x SM clock.  The rate
    of 2 DFMA per SM per clock is measured on the GB300 itself by the
    library's probe (qg_probe_fp64), reported beside every roofline."""
    mhz = sm_mhz or 2070.0
    return 152 * 4 * mhz * 1e6 / 1e12


# DRAM traffic of one propagate_kernel launch of the default workload comes
# from the kept ncu record (profiles/propagate_kernel_nai_n2048_traffic.json),
# which names the hash of the kernel's sources it was captured with; when the
# sources have changed since, the bench reports no traffic.
TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "propagate_kernel_nai_n2048_traffic.json")
KERNEL_SOURCES = ["qg_propagate.cu", "qg_dom1d.cuh", "qg_solver.cuh", "qg_device.cuh", "qg_internal.h"]


def kernel_sources_sha16():
    """Hash of the one-CTA propagator's sources."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1902_04661_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def _traffic(args, B, tuning=None):
    default = (args.precision == "fp64" and args.solver == "lanczos" and _guess(args) == 0 and B == 152
               and getattr(args, "workload", "nai") == "nai")
    if not default or not os.path.exists(TRAFFIC_RECORD):
        return None
    rec = json.load(open(TRAFFIC_RECORD))
    if rec.get("sources_sha16") != kernel_sources_sha16():
        return None
    if tuning is not None and rec.get("surfaces_per_fft") not in (None, tuning.get("surfaces_per_fft")):
        return None
    return rec.get("dram_bytes_per_launch")


def _guess(args):
    """Start of each implicit solve: 0 = explicit Euler (Sec. II B, the
    default), 1 = zero."""
    g = getattr(args, "guess", None) or "euler"
    return 1 if g == "zero" else 0


def _guess_name(args):
    return "zero" if _guess(args) else "euler"


def shard_seeds(rank, per_rank):
    """Seeds of the wavepackets rank `rank` propagates (weak scaling: every
    rank owns per_rank independent wavepackets; no data is exchanged)."""
    return [rank * per_rank + i for i in range(per_rank)]


def max_over_ranks(value, device=None):
    """Largest value over all ranks (the job time is the slowest rank's);
    the single collective of a multi-GPU run, on timing only."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _setup_batch(qg, wl, B, rank, stream, precision=0):
    N = WORKLOAD["N"]
    grid = qg.Grid([N], [wl.NAI_QMIN], [wl.NAI_QMAX])
    q = grid.points()
    W, dW = wl.nai_like_diabatic(q)
    model = qg.Model(grid, 2, [wl.NAI_REDUCED_MASS], W=W, dW=dW)
    states = []
    for seed in shard_seeds(rank, B):
        st = qg.State(model, precision=precision, stream=stream)
        q0, p0, s0 = wl.initial_gaussian_params(seed)
        st.set_gaussian(1, [q0], [p0], [s0])
        states.append(st)
    return grid, model, states


def run_ours(args):
    import torch
    import torch.distributed as dist
    import __graft_entry__
    import workloads as wl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    __graft_entry__.build()
    import paper_1902_04661_gb300 as qg

    sms = torch.cuda.get_device_properties(local).multi_processor_count
    B = args.batch or sms
    stream = torch.cuda.current_stream()
    prec = qg.QG_C64_MIXED if args.precision == "mixed" else qg.QG_C128
    grid, model, states = _setup_batch(qg, wl, B, rank, stream.cuda_stream, prec)
    batch = qg.Batch(states)
    opts = qg.default_solver_opts(tol=WORKLOAD["tol"], restart=WORKLOAD["restart"], max_iters=600, guess=_guess(args),
                                  solver=qg.QG_SOLVER_LANCZOS if args.solver == "lanczos" else qg.QG_SOLVER_GMRES)
    dt = WORKLOAD["dt_fs"] * FS
    m, o, sc = WORKLOAD["method"], WORKLOAD["order"], WORKLOAD["scheme"]
    N, S = WORKLOAD["N"], WORKLOAD["S"]
    tuning = batch.autotune(m, o, sc, dt, 1, opts) if not args.no_autotune else None
    for _ in range(args.warmup):
        batch.run(m, o, sc, dt, 1, opts)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    stats_all = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev[0].record(stream)
        for k in range(args.steps):
            stt, st = batch.run(m, o, sc, dt, 1, opts)
            ev[k + 1].record(stream)
            stats_all.append(st)
        torch.cuda.synchronize()
    launch_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    t_ms = sum(launch_ms)
    if world > 1:
        t_ms = max_over_ranks(t_ms, "cuda")
        dist.barrier()
    psi_after = states[0].get() if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None
    flat = [s for st in stats_all for s in st]
    n_hpsi = sum(s["n_hpsi"] for s in flat)
    n_sub = sum(s["n_substeps"] for s in flat)
    steps_done = B * args.steps
    value = steps_done * world / (t_ms / 1e3)
    hpsi_rate = n_hpsi * N * world / (t_ms / 1e3)
    flops = _flops_per_launch(flat, N, S, mixed=(args.precision == "mixed")) / args.steps
    abytes = _bytes_per_launch(flat, N, S) / args.steps
    avg_launch_s = (t_ms / args.steps) / 1e3
    clocks = clk.summary()
    peak = fp64_peak_tflops()
    achieved = flops / avg_launch_s / 1e12
    probe = qg.probe_fp64()

    # end to end through the C-ABI: pinned host -> device, step, device -> host
    len_state = S * N
    host_in = [torch.empty(len_state, dtype=torch.complex128, pin_memory=True) for _ in range(B)]
    host_out = [torch.empty(len_state, dtype=torch.complex128, pin_memory=True) for _ in range(B)]
    for i, st in enumerate(states):
        st.get(host_in[i].numpy().reshape(st.shape))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e_steps = max(1, min(args.steps, 3))
    e0.record(stream)
    for _ in range(e_steps):
        for i, st in enumerate(states):
            st.set(host_in[i].numpy().reshape(st.shape))
        batch.run(m, o, sc, dt, 1, opts)
        for i, st in enumerate(states):
            st.get(host_out[i].numpy().reshape(st.shape))
    e1.record(stream)
    torch.cuda.synchronize()
    e_ms = e0.elapsed_time(e1)
    if world > 1:
        e_ms = max_over_ranks(e_ms, "cuda")
    e2e = B * e_steps * world / (e_ms / 1e3)

    if rank == 0:
        mp = _peaks()
        line = {
            "metric": METRIC, "value": value, "unit": "wavepacket-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == qg.QG_C128 else "c64 inner / f64 residual",
            "data": "synthetic (seeded NaI-like model and Gaussians)",
            "config": {"workload": WORKLOAD["name"], "N": N, "S": S, "wavepackets_per_gpu": B,
                       "method": "implicit midpoint" if m == 1 else "trapezoidal",
                       "order": o, "scheme": "suzuki" if sc == 1 else "triple_jump",
                       "dt_fs": WORKLOAD["dt_fs"], "solver_tol": WORKLOAD["tol"], "restart": WORKLOAD["restart"],
                       "precision": args.precision, "solver": args.solver, "guess": _guess_name(args),
                       "l2": "working set %.0f MB > L2 (129 MB): no flush needed" %
                             (B * (WORKLOAD["restart"] + 6) * len_state * 16 / 1e6)},
            "hpsi_grid_point_applications_per_s": hpsi_rate,
            "substeps_per_s": n_sub * world / (t_ms / 1e3),
            "krylov_iters_per_substep": sum(s["n_krylov"] for s in flat) / max(1, n_sub),
            "fp64_hpsi_per_substep": n_hpsi / max(1, n_sub),
            "c64_hpsi_per_substep": sum(s["n_hpsi32"] for s in flat) / max(1, n_sub),
            "hbm_frac_if_streamed": abytes / avg_launch_s / 1e9 / mp.get("hbm_gbs", 6695.2),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": _traffic(args, B, tuning),
                         "kernel": "qg::propagate_kernel",
                         "peak_source": "FP64 FMA peak 152 SMs x 2 DFMA/clk (4 flop) x 2070 MHz",
                         "probe": dict(probe, how="qg_probe_fp64: register FMA / add chains, 8 CTAs per SM, "
                                                   "SM clock from clock64 against the global timer")},
            "gpu_launches": args.steps,
            "autotune": tuning,
            "clocks": clocks,
            "e2e": {"value": e2e, "unit": "wavepacket-steps/s", "h2d_bytes_per_step": B * len_state * 16,
                    "d2h_bytes_per_step": B * len_state * 16},
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(budget_s=args.cpu_seconds)
            line["cpu_same_algorithm"] = cpu_same_algorithm(budget_s=args.cpu_seconds)
            ksteps = args.warmup + args.steps
            line["error_vs_exact"] = error_vs_exact(wl, psi_after, shard_seeds(rank, B)[0], ksteps, dt)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


_CPU = {}


def cpu_baseline(budget_s=15.0):
    """The dense CPU oracle on a bounded sample of the workload: one wavepacket,
    composed steps until budget_s of stepping has elapsed.  The one-time dense
    H build and LU factorisations are timed separately and excluded."""
    import workloads as wl
    from oracle import fields, grid as ogrid, hamiltonian as ham, initial, propagate as prop, composition as comp

    N = WORKLOAD["N"]
    order = WORKLOAD["order"]
    dt = WORKLOAD["dt_fs"] * FS
    if not _CPU:
        t0 = time.perf_counter()
        q, dq = ogrid.points(wl.NAI_QMIN, wl.NAI_QMAX, N)
        W, dW = wl.nai_like_diabatic(q)
        V, F = fields.two_state(W, dW)
        H = ham.dense_h([wl.NAI_QMIN], [wl.NAI_QMAX], [N], [wl.NAI_REDUCED_MASS], V, F)
        q0, p0, s0 = wl.initial_gaussian_params(0)
        _CPU["psi"] = initial.state_on_surface(2, 1, initial.gaussian([q], [q0], [p0], [s0]))
        st = prop.DenseStepper(H)
        for f in sorted(set(comp.schedule(order, WORKLOAD["scheme"]))):
            st.impl(_CPU["psi"], f * dt / 2)            # factor every distinct implicit step once
        _CPU["st"] = st
        _CPU["setup"] = time.perf_counter() - t0
    st, psi, setup = _CPU["st"], _CPU["psi"], _CPU["setup"]
    t1 = time.perf_counter()
    n = 0
    while True:
        psi = st.composed(psi, dt, WORKLOAD["method"], order, WORKLOAD["scheme"])
        n += 1
        if time.perf_counter() - t1 >= budget_s:
            break
    el = time.perf_counter() - t1
    _CPU["psi"] = psi
    threads = _blas_threads()
    return {"value": n / el, "unit": "wavepacket-steps/s", "cores": threads, "kind": "oracle",
            "sample": "1 wavepacket, %d composed steps of the workload (N=%d, order %d); one-time dense H + LU "
                      "set-up %.1f s excluded" % (n, N, order, setup)}


_ORA = {}


def _oracle_nai(N):
    """The oracle's dense H of the NaI-like model on N points (cached)."""
    if N not in _ORA:
        import workloads as wl
        from oracle import fields, grid as ogrid, hamiltonian as ham
        q, dq = ogrid.points(wl.NAI_QMIN, wl.NAI_QMAX, N)
        W, dW = wl.nai_like_diabatic(q)
        V, F = fields.two_state(W, dW)
        H = ham.dense_h([wl.NAI_QMIN], [wl.NAI_QMAX], [N], [wl.NAI_REDUCED_MASS], V, F)
        _ORA[N] = dict(q=q, dq=dq, V=V, F=F, H=H)
    return _ORA[N]


def _exact_evolution(N):
    from oracle import propagate as prop
    o = _oracle_nai(N)
    if "ev" not in o:
        o["ev"] = prop.ExactEvolution(o["H"])
    return o["ev"]


def _psi0_oracle(N, seed):
    import workloads as wl
    from oracle import initial
    o = _oracle_nai(N)
    q0, p0, s0 = wl.initial_gaussian_params(seed)
    return initial.state_on_surface(2, 1, initial.gaussian([o["q"]], [q0], [p0], [s0]))


def error_vs_exact(wl, psi_gpu, seed, ksteps, dt):
    """L2 error of one propagated packet against the exact evolution
    e^{-iHt} psi0 of the same discrete H (the oracle's eigen-decomposition),
    after the bench's ksteps composed steps; the linear extrapolation to
    t_f = 10500 a.u. is an estimate (the per-step error of a unitary method
    adds up roughly linearly)."""
    N = WORKLOAD["N"]
    t0 = time.perf_counter()
    ex = _exact_evolution(N)(_psi0_oracle(N, seed), ksteps * dt)
    err = float(np.linalg.norm(psi_gpu - ex) * np.sqrt(_oracle_nai(N)["dq"]))
    nf = 10500.0 / dt
    return {"value": err, "t_au": ksteps * dt, "composed_steps": ksteps,
            "estimate_at_tf": err * nf / ksteps, "reference": "oracle eigen-decomposition of the dense H",
            "host_s": time.perf_counter() - t0}


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_same_algorithm(budget_s=10.0):
    """The same algorithm in plain C on all host cores (oracle/cpu_baseline:
    radix-2 FFT, Lanczos, carried H psi, OpenMP over packets), on a sample of
    the workload: one packet per core, composed steps until budget_s."""
    from oracle import cpu_baseline as cb
    import workloads as wl
    N = WORKLOAD["N"]
    o = _oracle_nai(N)
    npk = os.cpu_count() or 1
    psi = np.stack([_psi0_oracle(N, s) for s in range(npk)])
    dt = WORKLOAD["dt_fs"] * FS
    t1 = time.perf_counter()
    n = 0
    info = None
    while True:
        info = cb.propagate(psi, wl.NAI_QMIN, wl.NAI_QMAX, wl.NAI_REDUCED_MASS, o["V"], o["F"][0], WORKLOAD["order"],
                            dt, 1, tol=WORKLOAD["tol"])
        n += 1
        if time.perf_counter() - t1 >= budget_s:
            break
    el = time.perf_counter() - t1
    return {"value": npk * n / el, "unit": "wavepacket-steps/s", "cores": info["threads"], "nproc": os.cpu_count(),
            "cpu": _cpu_model(), "kind": "same algorithm in C, FP64 (FFT + Lanczos, OpenMP over packets)",
            "status": info["status"],
            "sample": "%d packets (one per core) x %d composed steps of the workload" % (npk, n)}


def _blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count() or 1


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    vals = []
    cb = None
    for _ in range(args.warmup):
        cpu_baseline(budget_s=1.0)
    for _ in range(args.steps):
        cb = cpu_baseline(budget_s=args.cpu_seconds / max(1, args.steps))
        vals.append(cb["value"])
    v = float(np.mean(vals))
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "wavepacket-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded NaI-like)",
            "config": {"workload": WORKLOAD["name"], "N": WORKLOAD["N"], "S": WORKLOAD["S"],
                       "wavepackets_per_gpu": 1, "order": WORKLOAD["order"], "dt_fs": WORKLOAD["dt_fs"]},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "wavepacket-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


BATCHED = dict(name="avoided_crossing_x4096_midpoint_suzuki4", models=4096, seed0=1000, method=1, order=4,
               scheme=1, dt_fs=0.1, tol=1e-12, restart=30)


def run_batched(args):
    """Batched workload: independent seeded avoided-crossing models (S = 2-3,
    N = 256..8192 log-uniform), all propagated by one persistent launch per
    composed step, replayed from a CUDA graph.  Also times the per-instance
    path (one launch per model) on a sample of the same models."""
    import torch
    import __graft_entry__
    import workloads as wl

    torch.cuda.set_device(0)
    __graft_entry__.build()
    import paper_1902_04661_gb300 as qg

    nmod = args.models or BATCHED["models"]
    prec = qg.QG_C64_MIXED if args.precision == "mixed" else qg.QG_C128
    stream = torch.cuda.current_stream()
    keep, states, sizes = [], [], []
    for i in range(nmod):
        m = wl.avoided_crossing_model(BATCHED["seed0"] + i)
        g = qg.Grid([m["N"]], [m["qmin"]], [m["qmax"]])
        lm = qg.Model(g, m["S"], [m["mass"]], W=m["W"], dW=m["dW"])
        st = qg.State(lm, precision=prec, stream=stream.cuda_stream)
        st.set_gaussian(m["surface"], [m["q0"]], [m["p0"]], [m["sigma0"]])
        keep += [g, lm]
        states.append(st)
        sizes.append((m["N"], m["S"]))
    batch = qg.Batch(states)
    opts = qg.default_solver_opts(tol=BATCHED["tol"], restart=BATCHED["restart"], guess=_guess(args))
    dt = BATCHED["dt_fs"] * FS
    m_, o_, s_ = BATCHED["method"], BATCHED["order"], BATCHED["scheme"]
    tuning = batch.autotune(m_, o_, s_, dt, 1, opts)
    batch.capture(m_, o_, s_, dt, 1, opts)
    bstream = torch.cuda.ExternalStream(batch.stream)
    for _ in range(args.warmup):
        batch.replay()
    batch.stats()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    stats_all = []
    with ClockSampler(0) as clk:
        ev[0].record(bstream)
        for k in range(args.steps):
            batch.replay()
            ev[k + 1].record(bstream)
        torch.cuda.synchronize()
        stt, st_ = batch.stats()
    t_ms = ev[0].elapsed_time(ev[args.steps])
    # every replay ran the same step; the statistics of the last one stand for each
    hpsi_pts = sum(s["n_hpsi"] * n * S for s, (n, S) in zip(st_, sizes))
    value = nmod * args.steps / (t_ms / 1e3)
    # per-instance path filling the GPU: one qg_propagate launch per model
    # (one CTA each), issued from 128 host threads on 128 streams so that
    # up to 128 launches run at once
    import concurrent.futures as cf
    nthreads = 128
    streams = [torch.cuda.Stream() for _ in range(nthreads)]
    for i, st in enumerate(states):
        st.set_stream(streams[i % nthreads])
    ns = nmod if args.per_instance_sample <= 0 else min(nmod, args.per_instance_sample)

    def lane(t):
        for st in states[t:ns:nthreads]:
            st.propagate(m_, o_, s_, dt, 1, opts)

    torch.cuda.synchronize()
    w0 = time.perf_counter()
    with cf.ThreadPoolExecutor(nthreads) as ex:
        list(ex.map(lane, range(nthreads)))
    torch.cuda.synchronize()
    per_ms = (time.perf_counter() - w0) * 1e3
    per_value = ns / (per_ms / 1e3)
    line = {"metric": METRIC, "value": value, "unit": "wavepacket-steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == qg.QG_C128 else "c64 inner / f64 residual",
            "data": "synthetic (seeded avoided-crossing models)",
            "config": {"workload": BATCHED["name"], "models": nmod, "S": "2-3", "N": "256-8192 log-uniform",
                       "method": "implicit midpoint", "order": o_, "scheme": "suzuki", "dt_fs": BATCHED["dt_fs"],
                       "solver_tol": BATCHED["tol"], "precision": args.precision,
                       "launch": "one persistent launch per step, CUDA graph replay"},
            "hpsi_grid_point_applications_per_s": hpsi_pts * args.steps / (t_ms / 1e3),
            "per_instance_path": {"value": per_value, "unit": "wavepacket-steps/s", "sample_models": ns,
                                  "launch": "one launch per model from 128 host threads on 128 streams "
                                            "(wall clock)",
                                  "speedup_of_batched": value / per_value},
            "gpu_launches": args.steps, "clocks": clk.summary(), "autotune": tuning,
            "statuses_ok": sum(1 for x in stt if x == 0)}
    print(json.dumps(line), flush=True)


SWEEP_JOBS = {
    # (scheme, order): step counts n (dt = t_f / n) to run; each error uses n and 2n
    (1, 2): [1024, 2048, 4096, 8192, 16384, 32768],
    (0, 4): [512, 1024, 2048, 4096, 8192],
    (1, 4): [256, 512, 1024, 2048, 4096],
    (0, 6): [256, 512, 1024, 2048],
    (1, 6): [128, 256, 512, 1024],
    (0, 8): [128, 256],
    (1, 8): [64, 128, 256],
}


def run_2d(args):
    """2-D two-surface model, 256 x 256 grid, Suzuki order 6, one instance over
    the whole GPU (cooperative launch): complex64-inner / FP64-refined form
    timed against the plain FP64 path on the same steps, with the difference
    between the two results."""
    import torch
    import __graft_entry__
    import workloads as wl

    torch.cuda.set_device(0)
    __graft_entry__.build()
    import paper_1902_04661_gb300 as qg

    p = wl.MODEL2D_PARAMS
    ns = (256, 256)
    q1 = p["qmin"][0] + (p["qmax"][0] - p["qmin"][0]) / ns[0] * np.arange(ns[0])
    q2 = p["qmin"][1] + (p["qmax"][1] - p["qmin"][1]) / ns[1] * np.arange(ns[1])
    W, dW = wl.model2d_diabatic(q1, q2, p)
    g = qg.Grid(list(ns), list(p["qmin"]), list(p["qmax"]))
    m = qg.Model(g, 2, list(p["mass"]), W=W, dW=dW)
    q0, p0, s0 = wl.model2d_initial()
    dt = 0.1 * FS
    tol = args.tol2d
    opts = qg.default_solver_opts(tol=tol, guess=_guess(args),
                                  solver=qg.QG_SOLVER_LANCZOS if args.solver == "lanczos" else qg.QG_SOLVER_GMRES)
    res = {}
    # reference for the error of both arms: the same steps in FP64 with the
    # solver at tol 1e-15 (untimed)
    ref = qg.State(m)
    ref.set_gaussian(1, q0, p0, s0)
    ref.propagate(1, 6, 1, dt, args.steps,
                  qg.default_solver_opts(tol=1e-15, max_iters=600, solver=qg.QG_SOLVER_LANCZOS, guess=_guess(args)))
    psi_ref = ref.get()
    for name, prec in (("mixed", qg.QG_C64_MIXED), ("fp64", qg.QG_C128)):
        st = qg.State(m, precision=prec)
        st.set_gaussian(1, q0, p0, s0)
        for _ in range(args.warmup):
            st.propagate(1, 6, 1, dt, 1, opts)
        tune = st.autotune(1, 6, 1, dt, 1, opts) if not args.no_autotune else None
        st.set_gaussian(1, q0, p0, s0)
        e_start = st.energy()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        s_ = st.propagate(1, 6, 1, dt, args.steps, opts)
        e1.record()
        torch.cuda.synchronize()
        res[name] = dict(ms=e0.elapsed_time(e1), stats=s_, psi=st.get(), norm=st.norm(), tune=tune,
                         energy_drift=abs(st.energy() - e_start) / max(1e-300, abs(e_start)))
    dv = np.prod([(p["qmax"][d] - p["qmin"][d]) / ns[d] for d in range(2)])
    err = float(np.linalg.norm(res["mixed"]["psi"] - res["fp64"]["psi"]) * np.sqrt(dv))
    err_ref = {k: float(np.linalg.norm(res[k]["psi"] - psi_ref) * np.sqrt(dv)) for k in ("mixed", "fp64")}
    t_m, t_f = res["mixed"]["ms"], res["fp64"]["ms"]
    line = {"metric": METRIC, "value": args.steps / (t_m / 1e3), "unit": "wavepacket-steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_m / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "c64 inner / f64 residual",
            "data": "synthetic (2-D two-state model)",
            "config": {"workload": "model2d_256x256_midpoint_suzuki6", "grid": list(ns), "S": 2, "order": 6,
                       "dt_fs": 0.1, "solver_tol": tol, "solver": args.solver, "guess": _guess_name(args),
                       "launch": "one cooperative launch over all SMs"},
            "fp64_path": {"value": args.steps / (t_f / 1e3), "ms_per_step": t_f / args.steps,
                          "fp64_hpsi": res["fp64"]["stats"]["n_hpsi"]},
            "speedup_mixed_over_fp64": t_f / t_m,
            "mixed_vs_fp64_l2": err, "norm_drift": abs(res["mixed"]["norm"] - 1.0),
            "drift": {k: {"norm": abs(res[k]["norm"] - 1.0), "energy_rel": res[k]["energy_drift"]}
                      for k in ("mixed", "fp64")},
            # L2 error of each arm against FP64 at solver tol 1e-15, same steps
            "error_vs_tight_fp64": err_ref,
            "mixed_hpsi": {"fp64": res["mixed"]["stats"]["n_hpsi"], "c64": res["mixed"]["stats"]["n_hpsi32"]},
            "hpsi_grid_point_applications_per_s":
                (res["mixed"]["stats"]["n_hpsi"] + res["mixed"]["stats"]["n_hpsi32"]) * ns[0] * ns[1] / (t_m / 1e3),
            # one-step trial times (ms) at the automatic cooperative width, 1/2 and 1/4 of it
            "launch_width_trials_ms": {k: res[k]["tune"] for k in ("mixed", "fp64")}}
    print(json.dumps(line), flush=True)


def run_adjoint(args):
    """Gradients of the final excited-state population of seeded NaI-like
    models (8 diabatic parameters perturbed by up to 5 %) by the adjoint form:
    one batched checkpointed forward launch and one batched adjoint launch."""
    import torch
    import __graft_entry__
    import workloads as wl

    torch.cuda.set_device(0)
    __graft_entry__.build()
    import paper_1902_04661_gb300 as qg
    from paper_1902_04661_gb300 import autograd as qad

    nm = args.models or 256
    N = WORKLOAD["N"]
    g = qg.Grid([N], [wl.NAI_QMIN], [wl.NAI_QMAX])
    q = g.points()
    base = wl.nai_like_params()
    keys = ["E_ion", "A_ion", "rho_ion", "B_cov", "rho_cov", "A_c", "beta_c", "q_c"]
    Vs, Fs = [], []
    for i in range(nm):
        rng = np.random.default_rng(5000 + i)
        par = dict(base)
        for k in keys:
            par[k] = base[k] * (1 + 0.05 * rng.uniform(-1, 1))
        W, dW = wl.nai_like_diabatic(q, par)
        V, F = qg.Model(g, 2, [wl.NAI_REDUCED_MASS], W=W, dW=dW).fields()
        Vs.append(V)
        Fs.append(F[0])
    V = torch.tensor(np.stack(Vs), device="cuda", requires_grad=True)
    F = torch.tensor(np.stack(Fs), device="cuda", requires_grad=True)
    st = qg.State(qg.Model(g, 2, [wl.NAI_REDUCED_MASS], V=Vs[0], F=Fs[0][None]))
    st.set_gaussian(1, [wl.NAI_Q0], [0.0], [wl.NAI_SIGMA0])
    psi0 = torch.tensor(np.stack([st.get()] * nm), device="cuda", requires_grad=True)
    dt, nsteps = 0.5 * FS, args.steps
    opts = qg.default_solver_opts(tol=1e-12, guess=_guess(args),
                                  solver=qg.QG_SOLVER_LANCZOS if args.solver == "lanczos" else qg.QG_SOLVER_GMRES)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e2 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    out = qad.propagate_batch(V, F, psi0, g, wl.NAI_REDUCED_MASS, 1, 4, 1, dt, nsteps, 8, opts)
    e1.record()
    L = (g.dq[0] * (out[:, 1].abs() ** 2)).sum()
    L.backward()
    e2.record()
    torch.cuda.synchronize()
    tf, tb = qad.last_stats["forward_ms"], qad.last_stats["adjoint_ms"]

    def agg(key):
        st = qad.last_stats[key]
        sub = sum(x["n_substeps"] for x in st)
        return {"substeps": sub, "hpsi_per_substep": sum(x["n_hpsi"] for x in st) / max(1, sub),
                "krylov_per_substep": sum(x["n_krylov"] for x in st) / max(1, sub),
                "restarts": sum(x["n_restart"] for x in st)}
    line = {"metric": METRIC, "value": nm * nsteps / ((tf + tb) / 1e3), "unit": "wavepacket-steps/s (forward+adjoint)",
            "n_gpus": 1, "steps": nsteps, "warmup": 0, "ms_per_step": (tf + tb) / nsteps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (perturbed NaI-like models)",
            "config": {"workload": "nai_like_adjoint_x%d_n2048_suzuki4" % nm, "models": nm, "N": N, "order": 4,
                       "dt_fs": 0.5, "checkpoint_every": 8},
            "forward_ms": tf, "adjoint_ms": tb, "adjoint_over_forward": tb / tf,
            "forward_stats": agg("forward"), "adjoint_stats": agg("adjoint"),
            "wall_ms_incl_setup": e0.elapsed_time(e2),
            "grad_norms": {"V": float(V.grad.norm()), "F": float(F.grad.norm()), "psi0": float(psi0.grad.norm())}}
    # the gradient along one seeded direction against a central difference of
    # two more forward propagations (outside the timed launches)
    gen = torch.Generator().manual_seed(77)

    def direction(x):
        r = torch.randn(x.shape, generator=gen, dtype=torch.float64)
        if x.is_complex():
            r = torch.complex(r, torch.randn(x.shape, generator=gen, dtype=torch.float64))
        return (r * float(x.detach().abs().mean())).to(x.device)

    dV, dF, dP = direction(V), direction(F), direction(psi0)

    def loss_at(s):
        with torch.no_grad():
            o = qad.propagate_batch(V.detach() + s * dV, F.detach() + s * dF, psi0.detach() + s * dP, g,
                                    wl.NAI_REDUCED_MASS, 1, 4, 1, dt, nsteps, 8, opts)
            return float((g.dq[0] * (o[:, 1].abs() ** 2)).sum())

    h = 1e-5
    fd = (loss_at(h) - loss_at(-h)) / (2 * h)
    ad = float((V.grad * dV).sum() + (F.grad * dF).sum() + (psi0.grad.conj() * dP).real.sum())
    line["gradient_check"] = {"adjoint_directional": ad, "central_difference": fd,
                              "rel_diff": abs(ad - fd) / max(abs(fd), 1e-300), "h": h,
                              "direction": "seeded normal in V, F and psi0, scaled by each input's mean magnitude"}
    print(json.dumps(line), flush=True)


# the cheapest point of the coarse sweep, refined: Suzuki order 8 around
# dt = t_f / 1024
SWEEP_VERIFY = {(1, 8): [768, 1024, 1536, 2048]}
# one propagation at the operating point, compared offline with the
# n = 2048 run of the verify set
SWEEP_POINT = {(1, 8): [1024]}


def run_sweep(args):
    """Convergence error ||psi_dt(t_f) - psi_dt/2(t_f)|| (Sec. III, Fig. 3) of the
    NaI-like workload for every (scheme, order, dt = t_f / n) in SWEEP_JOBS,
    each propagation one CTA on its own stream, all concurrent.  Prints one
    JSON line per finished propagation (wall time, H psi count) as it
    completes, then one line per (scheme, order, dt) with the error."""
    import concurrent.futures as cf
    import torch
    import __graft_entry__
    import workloads as wl

    torch.cuda.set_device(0)
    __graft_entry__.build()
    import paper_1902_04661_gb300 as qg

    N = WORKLOAD["N"]
    tf = args.tf
    grid = qg.Grid([N], [wl.NAI_QMIN], [wl.NAI_QMAX])
    W, dW = wl.nai_like_diabatic(grid.points())
    model = qg.Model(grid, 2, [wl.NAI_REDUCED_MASS], W=W, dW=dW)
    prec = qg.QG_C64_MIXED if args.precision == "mixed" else qg.QG_C128
    table = {"verify": SWEEP_VERIFY, "coarse": SWEEP_JOBS, "point": SWEEP_POINT}[args.sweep_set]
    jobs = [(sc, o, n) for (sc, o), ns in table.items() for n in ns]
    jobs.sort(key=lambda j: -j[2] * (3 if j[0] == 0 else 5) ** (j[1] // 2 - 1))
    opts = qg.default_solver_opts(tol=args.sweep_tol, max_iters=600, guess=_guess(args),
                                  solver=qg.QG_SOLVER_LANCZOS if args.solver == "lanczos" else qg.QG_SOLVER_GMRES)
    outdir = args.sweep_dir
    if outdir:
        os.makedirs(outdir, exist_ok=True)

    def one(job):
        scheme, order, n = job
        stream = torch.cuda.Stream()
        st = qg.State(model, precision=prec, stream=stream)
        st.set_gaussian(1, [wl.NAI_Q0], [wl.NAI_P0], [wl.NAI_SIGMA0])
        t0 = time.perf_counter()
        stats = st.propagate(WORKLOAD["method"], order, scheme, tf / n, n, opts, allow_fail=True)
        el = time.perf_counter() - t0
        psi = st.get()
        row = {"scheme": "suzuki" if scheme == 1 else "triple_jump", "order": order, "nsteps": n, "dt_au": tf / n,
               "dt_fs": tf / n / FS, "status": stats["status"], "wall_s": el, "hpsi": stats["n_hpsi"],
               "substeps": stats["n_substeps"], "krylov_per_substep": stats["n_krylov"] / max(1, stats["n_substeps"])}
        print(json.dumps(row), flush=True)
        if outdir:
            np.save(os.path.join(outdir, "psi_%d_%d_%d.npy" % job), psi)
        return job, psi, row

    with cf.ThreadPoolExecutor(len(jobs)) as ex:
        res = list(ex.map(one, jobs))
    byk = {j: (psi, row) for j, psi, row in res}
    dq = grid.dq[0]
    best = None
    for (scheme, order, n), (psi, row) in sorted(byk.items()):
        nxt = byk.get((scheme, order, 2 * n))
        if nxt is None or row["status"] != 0 or nxt[1]["status"] != 0:
            continue
        err = float(np.linalg.norm(psi - nxt[0]) * np.sqrt(dq))
        row = dict(row, error=err)
        print(json.dumps({"error_row": row}), flush=True)
        if err <= 1e-10 and (best is None or row["wall_s"] < best["wall_s"]):
            best = row
    print(json.dumps({"sweep_best_at_1e-10": best, "t_f": tf, "tol": args.sweep_tol,
                      "precision": args.precision}), flush=True)


def _single_cases(args):
    ns = args.single_steps
    return [
        dict(name="nai_like_n1024_trapezoidal_dt0.1fs_200steps", N=1024, method=0, order=2, scheme=1, dt=0.1 * FS,
             nsteps=200, tol=1e-12, note="the n1024 trapezoidal configuration, whole run"),
        dict(name="nai_like_n2048_midpoint_suzuki8_dt10.25au_one_packet", N=2048, method=1, order=8, scheme=1,
             dt=10500.0 / 1024, nsteps=ns, tol=1e-15, note="the error-1e-10 point, %d of 1024 steps to t_f" % ns),
        dict(name="nai_like_n4096_midpoint_suzuki8_dt10.25au_one_packet", N=4096, method=1, order=8, scheme=1,
             dt=10500.0 / 1024, nsteps=ns, tol=1e-15, note="the same point on 4096 points, %d steps" % ns),
    ]


def run_single(args):
    """One wavepacket at a time (latency): the one-CTA form against the
    shared-memory cluster form at its smallest cluster size and twice it.
    Prints one JSON line per case with the time per elementary step, the
    FP64 rate against the peak of the SMs the form occupies, and the
    time to t_f = 10500 a.u. where the case is the error-1e-10 point."""
    import torch
    import __graft_entry__
    import workloads as wl

    torch.cuda.set_device(0)
    __graft_entry__.build()
    import paper_1902_04661_gb300 as qg

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for case in _single_cases(args):
        N = case["N"]
        grid = qg.Grid([N], [wl.NAI_QMIN], [wl.NAI_QMAX])
        W, dW = wl.nai_like_diabatic(grid.points())
        model = qg.Model(grid, 2, [wl.NAI_REDUCED_MASS], W=W, dW=dW)
        q0, p0, s0 = wl.initial_gaussian_params(0)
        opts = qg.default_solver_opts(tol=case["tol"], restart=30, max_iters=600, solver=qg.QG_SOLVER_LANCZOS)
        g0 = qg.cluster_size(N, 2)
        forms = {}
        for G in (0, g0, 2 * g0 if 0 < g0 < 16 else 0):
            if G == 0 and 0 in forms:
                continue
            st = qg.State(model)
            if G:
                st.set_cluster(G)
            st.set_gaussian(1, [q0], [p0], [s0])
            st.propagate(case["method"], case["order"], case["scheme"], case["dt"], 1, opts)   # warm-up
            st.set_gaussian(1, [q0], [p0], [s0])
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            stats = st.propagate(case["method"], case["order"], case["scheme"], case["dt"], case["nsteps"], opts)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            flops = _flops_per_launch([stats], N, 2)
            used = max(1, G)
            peak = fp64_peak_tflops() * used / sms
            forms["cluster%d" % G if G else "one_cta"] = {
                "ms": ms, "us_per_substep": 1e3 * ms / max(1, stats["n_substeps"]),
                "ms_per_composed_step": ms / case["nsteps"], "sms": used,
                "fp64_tflops": flops / (ms * 1e-3) / 1e12, "frac_of_used_sms_peak": flops / (ms * 1e-3) / 1e12 / peak,
                "hpsi_per_substep": stats["n_hpsi"] / max(1, stats["n_substeps"]), "status": stats["status"]}
        best = min(forms.values(), key=lambda f: f["ms"])
        line = {"metric": "time per elementary step of one wavepacket (latency)", "value": best["us_per_substep"],
                "unit": "us/substep", "n_gpus": 1, "steps": case["nsteps"], "warmup": 1,
                "ms_per_step": best["ms_per_composed_step"], "higher_is_better": False, "scaling": "none",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded NaI-like model and Gaussian)",
                "config": {"workload": case["name"], "N": N, "S": 2, "note": case["note"], "solver_tol": case["tol"]},
                "forms": forms}
        if case["nsteps"] != 200:
            line["time_to_tf_s_estimate"] = best["ms_per_composed_step"] * 1024 / 1e3
        print(json.dumps(line), flush=True)


CONFIG2 = {
    # (scheme, order): step counts n over t_f (dt = t_f / n)
    (1, 8): [512, 768, 1024, 1536],
    (2, 8): [1024, 1536, 2048, 3072, 4096],
    (2, 6): [2048, 4096, 8192],
    (1, 6): [2048, 4096],
}


def run_config2(args):
    """Wavefunction error against the exact evolution (Sec. III, Fig. 5): the
    NaI-like packet propagated to t_f = 10500 a.u. for each scheme, order and
    dt, one packet per job (shared-memory cluster form), all jobs concurrent on
    their own streams; error = ||psi_dt(t_f) - e^{-iHt_f} psi0|| with the
    oracle's eigen-decomposition of the same dense H.  Prints one line per job
    and, per grid, the cheapest job at error <= 1e-10."""
    import concurrent.futures as cf
    import torch
    import __graft_entry__
    import workloads as wl

    torch.cuda.set_device(0)
    __graft_entry__.build()
    import paper_1902_04661_gb300 as qg

    tf = args.tf
    for N in [int(x) for x in args.config2_n.split(",")]:
        t0 = time.perf_counter()
        ex = _exact_evolution(N)(_psi0_oracle(N, None), tf)
        ref_s = time.perf_counter() - t0
        dq = _oracle_nai(N)["dq"]
        grid = qg.Grid([N], [wl.NAI_QMIN], [wl.NAI_QMAX])
        W, dW = wl.nai_like_diabatic(grid.points())
        model = qg.Model(grid, 2, [wl.NAI_REDUCED_MASS], W=W, dW=dW)
        G = qg.cluster_size(N, 2)
        opts = qg.default_solver_opts(tol=args.sweep_tol, restart=30, max_iters=600, solver=qg.QG_SOLVER_LANCZOS)
        jobs = [(sc, o, n) for (sc, o), ns in CONFIG2.items() for n in ns]

        def one(job):
            scheme, order, n = job
            stream = torch.cuda.Stream()
            st = qg.State(model, stream=stream)
            st.set_cluster(G)
            st.set_gaussian(1, [wl.NAI_Q0], [wl.NAI_P0], [wl.NAI_SIGMA0])
            t1 = time.perf_counter()
            stats = st.propagate(WORKLOAD["method"], order, scheme, tf / n, n, opts, allow_fail=True)
            el = time.perf_counter() - t1
            err = float(np.linalg.norm(st.get() - ex) * np.sqrt(dq))
            row = {"N": N, "scheme": {0: "triple_jump", 1: "suzuki", 2: "optimal"}[scheme], "order": order,
                   "nsteps": n, "dt_au": tf / n, "status": stats["status"], "error_vs_exact": err,
                   "wall_s": el, "hpsi": stats["n_hpsi"], "substeps": stats["n_substeps"], "cluster": G}
            print(json.dumps(row), flush=True)
            return row

        with cf.ThreadPoolExecutor(len(jobs)) as exe:
            rows = list(exe.map(one, jobs))
        ok = [r for r in rows if r["status"] == 0 and r["error_vs_exact"] <= 1e-10]
        best = min(ok, key=lambda r: r["hpsi"]) if ok else None
        print(json.dumps({"config2_best_at_1e-10": best, "N": N, "t_f": tf, "tol": args.sweep_tol,
                          "reference": "oracle eigen-decomposition, %.1f s on the host" % ref_s}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=0, help="wavepackets per GPU (default: one per SM)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--guess", default=None, choices=["euler", "zero"],
                    help="start of each implicit solve: explicit Euler (Sec. II B; default) or zero")
    ap.add_argument("--sweep", action="store_true", help="convergence-error sweep that fixes the operating point")
    ap.add_argument("--solver", default="lanczos", choices=["gmres", "lanczos"],
                    help="Krylov method of the implicit steps (same minimal-residual iterates)")
    ap.add_argument("--workload", default="nai", choices=["nai", "batched", "2d", "adjoint", "single", "config2"])
    ap.add_argument("--single-steps", type=int, default=16, help="composed steps of the one-packet cases")
    ap.add_argument("--config2-n", default="2048,4096", help="grid sizes of the config2 error sweep")
    ap.add_argument("--models", type=int, default=0)
    ap.add_argument("--tol2d", type=float, default=1e-12, help="solver tolerance of the 2-D workload")
    ap.add_argument("--per-instance-sample", type=int, default=0, help="models timed one launch each (0: all)")
    ap.add_argument("--tf", type=float, default=10500.0)
    ap.add_argument("--sweep-tol", type=float, default=1e-15)
    ap.add_argument("--sweep-dir", default="")
    ap.add_argument("--sweep-set", default="verify", choices=["verify", "coarse", "point"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="fp64: every Krylov iteration in FP64; mixed: complex64 inner solves, FP64 refinement")
    args = ap.parse_args()
    if args.sweep:
        run_sweep(args)
    elif args.workload == "batched" and args.impl == "ours":
        run_batched(args)
    elif args.workload == "2d" and args.impl == "ours":
        run_2d(args)
    elif args.workload == "adjoint" and args.impl == "ours":
        run_adjoint(args)
    elif args.workload == "single" and args.impl == "ours":
        run_single(args)
    elif args.workload == "config2" and args.impl == "ours":
        run_config2(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
