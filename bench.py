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

# Operating point: NaI-like model on the paper's grid, implicit midpoint
# composed by Suzuki's fractal.  (order, dt) is the cheapest measured point
# whose convergence error ||psi_dt(t_f) - psi_dt/2(t_f)|| at t_f = 10500 a.u.
# is below 1e-10 (operating point).
WORKLOAD = dict(name="nai_like_n2048_s2_midpoint_suzuki", N=2048, S=2, method=1, order=6, scheme=1,
                dt_fs=0.5, tol=1e-12, restart=30)
FS = 41.341373335182


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
    of 2 DFMA per SM per clock was measured on GB300 with an FMA-chain probe
    (1.20 TFLOP/s at 2002 MHz)."""
    mhz = sm_mhz or 2070.0
    return 152 * 4 * mhz * 1e6 / 1e12


def _setup_batch(qg, wl, B, rank, stream, precision=0):
    N = WORKLOAD["N"]
    grid = qg.Grid([N], [wl.NAI_QMIN], [wl.NAI_QMAX])
    q = grid.points()
    W, dW = wl.nai_like_diabatic(q)
    model = qg.Model(grid, 2, [wl.NAI_REDUCED_MASS], W=W, dW=dW)
    states = []
    for i in range(B):
        st = qg.State(model, precision=precision, stream=stream)
        q0, p0, s0 = wl.initial_gaussian_params(rank * B + i)
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
    opts = qg.default_solver_opts(tol=WORKLOAD["tol"], restart=WORKLOAD["restart"])
    dt = WORKLOAD["dt_fs"] * FS
    m, o, sc = WORKLOAD["method"], WORKLOAD["order"], WORKLOAD["scheme"]
    N, S = WORKLOAD["N"], WORKLOAD["S"]
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
        tt = torch.tensor([t_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_ms = float(tt.item())
        dist.barrier()
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
        tt = torch.tensor([e_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e_ms = float(tt.item())
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
                       "dt_fs": WORKLOAD["dt_fs"], "gmres_tol": WORKLOAD["tol"], "restart": WORKLOAD["restart"],
                       "precision": args.precision,
                       "l2": "working set %.0f MB > L2 (129 MB): no flush needed" %
                             (B * (WORKLOAD["restart"] + 6) * len_state * 16 / 1e6)},
            "hpsi_grid_point_applications_per_s": hpsi_rate,
            "substeps_per_s": n_sub * world / (t_ms / 1e3),
            "krylov_iters_per_substep": sum(s["n_krylov"] for s in flat) / max(1, n_sub),
            "fp64_hpsi_per_substep": n_hpsi / max(1, n_sub),
            "c64_hpsi_per_substep": sum(s["n_hpsi32"] for s in flat) / max(1, n_sub),
            "hbm_frac_if_streamed": abytes / avg_launch_s / 1e9 / mp.get("hbm_gbs", 6695.2),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "qg::propagate_kernel",
                         "peak_source": "FP64 FMA peak 152 SMs x 4 flop/clk x 2070 MHz (measured 2 DFMA/SM/clk)"},
            "gpu_launches": args.steps,
            "clocks": clocks,
            "e2e": {"value": e2e, "unit": "wavepacket-steps/s", "h2d_bytes_per_step": B * len_state * 16,
                    "d2h_bytes_per_step": B * len_state * 16},
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(budget_s=args.cpu_seconds)
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=0, help="wavepackets per GPU (default: one per SM)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="fp64: every Krylov iteration in FP64; mixed: complex64 inner solves, FP64 refinement")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
