"""torch.autograd.Function wrappers of the propagation and its adjoint.

forward: the library propagates psi0 through nsteps composed steps, storing
psi every `every` steps (QG_RUN_CHECKPOINT).  backward: the library's adjoint
run (QG_RUN_ADJOINT) walks back from psi(t_f), re-propagating psi with the
exactly time-reversible integrator (reset to the checkpoints), propagating the
adjoint with U^dagger = U(-dt) and accumulating dL/dV and dL/dF per grid point.
Both run entirely in libqgeom; this module only allocates the torch tensors
and passes their device pointers.  Gradients follow torch's complex
convention dL = Re(sum conj(g) dpsi).
"""
import ctypes

import torch

from . import _binding as B

# statistics of the most recent batched forward and adjoint launches:
# {"forward": [per-instance stats], "forward_ms": launch time, "adjoint": [...], "adjoint_ms": ...}
last_stats = {}


def _timed_batch_run(batch, run, method, order, scheme, dt, nsteps, opts, n):
    stt, sts = (ctypes.c_int32 * n)(), (B.StepStats * n)()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.ExternalStream(B.lib().qg_batch_stream(batch.handle))
    e0.record(stream)
    r = B.lib().qg_batch_run_ex(batch.handle, run, method, order, scheme, float(dt), int(nsteps), ctypes.byref(opts),
                                stt, sts)
    e1.record(stream)
    B._check(r, "qg_batch_run_ex")
    e1.synchronize()
    return [x.as_dict() for x in sts], e0.elapsed_time(e1)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class _Run:
    """One model/state pair with its adjoint buffers."""

    def __init__(self, grid, V, F, psi0, mass, nsteps, every, precision=B.QG_C128):
        S, N = psi0.shape
        self.model = B.Model(grid, S, [mass], V=V.detach().contiguous(), F=F.detach().reshape(1, -1, N).contiguous())
        self.state = B.State(self.model, precision=precision, stream=torch.cuda.current_stream())
        self.state.set(psi0.detach().contiguous())
        self.nck = (nsteps - 1) // every + 1 if nsteps > 0 else 1
        dev = psi0.device
        self.ckpt = torch.empty((self.nck, S, N), dtype=torch.complex128, device=dev)
        self.grad = torch.zeros((S, N), dtype=torch.complex128, device=dev)
        self.gV = torch.zeros((S, N), dtype=torch.float64, device=dev)
        self.gF = torch.zeros((S * (S - 1) // 2, N), dtype=torch.float64, device=dev)
        B._check(B.lib().qg_state_set_adjoint(self.state.handle, _ptr(self.ckpt), self.nck, every, _ptr(self.grad),
                                              _ptr(self.gV), _ptr(self.gF)), "qg_state_set_adjoint")


def _run_ex(state, run, method, order, scheme, dt, nsteps, opts):
    st = B.StepStats()
    r = B.lib().qg_propagate_ex(state.handle, run, method, order, scheme, float(dt), int(nsteps), ctypes.byref(opts),
                                ctypes.byref(st))
    B._check(r, "qg_propagate_ex")
    return st.as_dict()


class Propagate(torch.autograd.Function):
    """psi(t_f) = U(dt)^nsteps psi0 for the adiabatic model (V, F) on `grid`.

    Inputs: V (S, N) float64, F (S(S-1)/2, N) float64, psi0 (S, N) complex128,
    all CUDA tensors; grid: a Grid; mass; method, order, scheme, dt, nsteps;
    every: composed steps between checkpoints; opts: SolverOpts or None.
    Returns psi(t_f) (S, N) complex128; backward gives dL/dV, dL/dF, dL/dpsi0."""

    @staticmethod
    def forward(ctx, V, F, psi0, grid, mass, method, order, scheme, dt, nsteps, every=8, opts=None):
        opts = opts if opts is not None else B.default_solver_opts()
        run = _Run(grid, V, F, psi0, mass, nsteps, every)
        stats = _run_ex(run.state, B.QG_RUN_CHECKPOINT, method, order, scheme, dt, nsteps, opts)
        out = torch.empty_like(psi0)
        run.state.get(out)
        ctx.run = run
        ctx.args = (method, order, scheme, dt, nsteps, opts)
        ctx.forward_stats = stats
        return out

    @staticmethod
    def backward(ctx, g_out):
        run = ctx.run
        method, order, scheme, dt, nsteps, opts = ctx.args
        run.grad.copy_(g_out.contiguous())
        run.gV.zero_()
        run.gF.zero_()
        _run_ex(run.state, B.QG_RUN_ADJOINT, method, order, scheme, dt, nsteps, opts)
        return run.gV.clone(), run.gF.clone(), run.grad.clone(), None, None, None, None, None, None, None, None, None


class PropagateBatch(torch.autograd.Function):
    """Batched Propagate: V (B, S, N), F (B, S(S-1)/2, N), psi0 (B, S, N) on
    one grid shape, all instances in one persistent launch for the forward and
    one for the adjoint."""

    @staticmethod
    def forward(ctx, V, F, psi0, grid, mass, method, order, scheme, dt, nsteps, every=8, opts=None):
        opts = opts if opts is not None else B.default_solver_opts()
        runs = [_Run(grid, V[b], F[b], psi0[b], mass, nsteps, every) for b in range(psi0.shape[0])]
        batch = B.Batch([r.state for r in runs])
        stats, ms = _timed_batch_run(batch, B.QG_RUN_CHECKPOINT, method, order, scheme, dt, nsteps, opts, len(runs))
        last_stats.clear()
        last_stats.update(forward=stats, forward_ms=ms)
        out = torch.empty_like(psi0)
        for b, run in enumerate(runs):
            run.state.get(out[b])
        ctx.runs, ctx.batch = runs, batch
        ctx.args = (method, order, scheme, dt, nsteps, opts)
        return out

    @staticmethod
    def backward(ctx, g_out):
        method, order, scheme, dt, nsteps, opts = ctx.args
        for b, run in enumerate(ctx.runs):
            run.grad.copy_(g_out[b].contiguous())
            run.gV.zero_()
            run.gF.zero_()
        torch.cuda.synchronize()
        stats, ms = _timed_batch_run(ctx.batch, B.QG_RUN_ADJOINT, method, order, scheme, dt, nsteps, opts,
                                     len(ctx.runs))
        last_stats.update(adjoint=stats, adjoint_ms=ms)
        gV = torch.stack([r_.gV for r_ in ctx.runs])
        gF = torch.stack([r_.gF for r_ in ctx.runs])
        gpsi = torch.stack([r_.grad for r_ in ctx.runs])
        return gV, gF, gpsi, None, None, None, None, None, None, None, None, None


def propagate(V, F, psi0, grid, mass, method, order, scheme, dt, nsteps, every=8, opts=None):
    """Differentiable propagation (see Propagate)."""
    return Propagate.apply(V, F, psi0, grid, mass, method, order, scheme, dt, nsteps, every, opts)


def propagate_batch(V, F, psi0, grid, mass, method, order, scheme, dt, nsteps, every=8, opts=None):
    """Differentiable batched propagation (see PropagateBatch)."""
    return PropagateBatch.apply(V, F, psi0, grid, mass, method, order, scheme, dt, nsteps, every, opts)
