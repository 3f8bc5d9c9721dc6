"""Thin Python binding of the C ABI in ``include/abp.h`` (argument marshalling only).

Every computation runs in ``libabp.so`` (sm_103a CUDA).  PyTorch is used for device
memory and streams only.  There is no fallback: if the library is missing or cannot be
loaded, every entry point raises.

The functions keep the ABI's names (``abp_create``, ``abp_set_params``, ``abp_integrate``,
``abp_reduce``, ``abp_backward`` ...); :class:`Ensemble` wraps them for the common
"set parameters, integrate, reduce" flow and :class:`MeanVelocity` exposes the adjoint
as a ``torch.autograd.Function``.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
# ABP_LIB selects another build of the library (the checked build, for instance)
LIB_PATH = os.environ.get("ABP_LIB") or os.path.join(_HERE, "_build", "libabp.so")

ABP_OK, ABP_EINVAL, ABP_ENOMEM, ABP_ECUDA, ABP_ETIMEOUT, ABP_ESTATE = range(6)
_STATUS = {0: "ABP_OK", 1: "ABP_EINVAL", 2: "ABP_ENOMEM", 3: "ABP_ECUDA", 4: "ABP_ETIMEOUT", 5: "ABP_ESTATE"}
GRAD_PARAMS = ("D", "q", "c", "d", "gamma0", "asym")
MOMENT_NAMES = ("mean_v", "se_v", "msd", "d_eff", "sum_vbar", "sum_vbar2", "sum_dx", "sum_dx2")


class AbpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_STATUS.get(status, str(status)), msg))
        self.status = status


class abp_params(C.Structure):
    _fields_ = [(n, C.c_double) for n in W.PARAM_NAMES]


class abp_config(C.Structure):
    _fields_ = [
        ("seed", C.c_uint64),
        ("dt", C.c_double),
        ("v0_mode", C.c_int32),
        ("state_fp64", C.c_int32),
        ("hist_x_bins", C.c_int32),
        ("hist_v_bins", C.c_int32),
        ("v_lo", C.c_double),
        ("v_hi", C.c_double),
        ("snapshot_every", C.c_int64),
        ("checkpoint_every", C.c_int64),
        ("particles_per_thread", C.c_int32),
        ("schedule", C.c_int32),
        ("steps_per_launch", C.c_int64),
        ("traj_base", C.c_uint64),
        ("scheme", C.c_int32),
        ("noise", C.c_int32),
    ]


_lock = threading.Lock()
_lib = None
_VP = C.c_void_p


def lib():
    """Load libabp.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libabp.so not found at %s: build it with "
                               "`python -m paper_1104_2499_gb300.build` (needs nvcc)" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        st = C.c_int
        L.abp_create.argtypes = [C.POINTER(_VP), C.POINTER(abp_config), _VP]
        L.abp_create.restype = st
        L.abp_set_params.argtypes = [_VP, C.c_int32, C.POINTER(abp_params), C.POINTER(C.c_int64),
                                     C.POINTER(C.c_int64)]
        L.abp_set_params.restype = st
        L.abp_reset.argtypes = [_VP, C.c_uint64]
        L.abp_reset.restype = st
        L.abp_kernel_launches.argtypes = [_VP, C.POINTER(C.c_int64)]
        L.abp_kernel_launches.restype = st
        L.abp_set_wait_limit.argtypes = [_VP, C.c_int64]
        L.abp_set_wait_limit.restype = st
        L.abp_test_hold_tile.argtypes = [_VP, C.c_int32]
        L.abp_test_hold_tile.restype = st
        L.abp_tuning.argtypes = [_VP, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                                 C.POINTER(C.c_int32)]
        L.abp_tuning.restype = st
        L.abp_tiles.argtypes = [_VP, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.abp_tuning_report.argtypes = [_VP, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]
        L.abp_tuning_report.restype = st
        P64, P32 = C.POINTER(C.c_int64), C.POINTER(C.c_int32)
        L.abp_plan.argtypes = [C.c_int32, P64, P64, C.c_int32, C.c_int32, C.c_int32, C.c_int32, P32, P32, P32,
                               P64, P32, P32, C.c_int32]
        L.abp_plan.restype = st
        L.abp_plan_efficiency.argtypes = [C.c_int32, P64, P64, C.c_int32, C.c_int32, C.c_int32, C.c_int64,
                                          C.c_int64, C.POINTER(C.c_double)]
        L.abp_plan_efficiency.restype = st
        L.abp_xorshift.argtypes = [C.c_uint64, C.c_uint64, C.c_int64, _VP, _VP]
        L.abp_xorshift.restype = st
        L.abp_live.argtypes = [_VP, _VP, _VP, _VP]
        L.abp_live.restype = st
        L.abp_live_ready.argtypes = [_VP, C.POINTER(C.c_int64)]
        L.abp_live_ready.restype = st
        L.abp_tiles.restype = st
        L.abp_integrate.argtypes = [_VP, C.c_int64]
        L.abp_integrate.restype = st
        L.abp_progress.argtypes = [_VP, C.POINTER(C.c_int64)]
        L.abp_progress.restype = st
        L.abp_num_snapshots.argtypes = [_VP, C.POINTER(C.c_int64)]
        L.abp_num_snapshots.restype = st
        L.abp_reduce.argtypes = [_VP, _VP, _VP, _VP]
        L.abp_reduce.restype = st
        L.abp_get_state.argtypes = [_VP, _VP, _VP, _VP, _VP, _VP]
        L.abp_get_state.restype = st
        L.abp_save.argtypes = [_VP, _VP, C.POINTER(C.c_size_t)]
        L.abp_save.restype = st
        L.abp_load.argtypes = [_VP, _VP, C.c_size_t]
        L.abp_load.restype = st
        L.abp_backward.argtypes = [_VP, _VP, _VP]
        L.abp_backward.restype = st
        L.abp_backward_windowed.argtypes = [_VP, _VP, _VP, C.c_int64]
        L.abp_backward_windowed.restype = st
        L.abp_backward_traj.argtypes = [_VP, _VP]
        L.abp_backward_traj.restype = st
        L.abp_synchronize.argtypes = [_VP]
        L.abp_synchronize.restype = st
        L.abp_destroy.argtypes = [_VP]
        L.abp_destroy.restype = None
        L.abp_last_error.argtypes = [_VP]
        L.abp_last_error.restype = C.c_char_p
        L.abp_philox.argtypes = [C.c_uint64, _VP, _VP, C.c_int64, _VP, _VP]
        L.abp_philox.restype = st
        L.abp_normals.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, C.c_int64, _VP, _VP]
        L.abp_normals.restype = st
        L.abp_version.argtypes = []
        L.abp_version.restype = C.c_char_p
        L.abp_combine_moments.argtypes = [C.c_int32, _VP, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.c_double, _VP]
        L.abp_combine_moments.restype = st
        L.abp_run_set_noalloc.argtypes = [C.POINTER(abp_params), C.POINTER(abp_config), C.c_int64, C.c_int64, _VP,
                                          _VP, _VP, _VP, C.c_char_p, C.c_size_t]
        L.abp_run_set_noalloc.restype = st
        _lib = L
        return L


def _check(status: int, ctx=None, what: str = ""):
    if status != ABP_OK:
        msg = lib().abp_last_error(ctx).decode() if ctx else what
        raise AbpError(status, msg or what)


def _ptr(x):
    """Raw address of a torch tensor / numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return x.data_ptr()


def _stream_ptr(stream):
    if stream is None:
        return None
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


# ----------------------------------------------------------------------- ABI names

def abp_create(cfg: abp_config, stream=None):
    h = _VP()
    _check(lib().abp_create(C.byref(h), C.byref(cfg), _stream_ptr(stream)), what="abp_create rejected the configuration")
    return h


def abp_set_params(ctx, sets, n_traj, n_steps):
    """sets: a sequence of parameter dicts, or a host float64 array [n_sets, 9] in
    workloads.PARAM_NAMES order (the abp_params layout, passed without a copy)."""
    if isinstance(sets, np.ndarray):
        P = np.ascontiguousarray(sets, dtype=np.float64)
        if P.ndim != 2 or P.shape[1] != len(W.PARAM_NAMES):
            raise ValueError("parameter array must be [n_sets, %d] float64" % len(W.PARAM_NAMES))
    else:
        P = np.array([[s[k] for k in W.PARAM_NAMES] for s in sets], dtype=np.float64).reshape(-1, len(W.PARAM_NAMES))
    n = P.shape[0]
    M = np.ascontiguousarray(n_traj, dtype=np.int64)
    N = np.ascontiguousarray(n_steps, dtype=np.int64)
    if M.shape != (n,) or N.shape != (n,):
        raise ValueError("n_traj and n_steps need one entry per parameter set")
    if n == 0:  # the library reads nothing then; pass valid one-element buffers
        P, M, N = np.zeros((1, len(W.PARAM_NAMES))), np.zeros(1, np.int64), np.zeros(1, np.int64)
    _check(lib().abp_set_params(ctx, n, P.ctypes.data_as(C.POINTER(abp_params)), M.ctypes.data_as(C.POINTER(C.c_int64)),
                                N.ctypes.data_as(C.POINTER(C.c_int64))), ctx)


def abp_reset(ctx, seed: int):
    _check(lib().abp_reset(ctx, int(seed)), ctx)


def abp_kernel_launches(ctx) -> int:
    out = C.c_int64()
    _check(lib().abp_kernel_launches(ctx, C.byref(out)), ctx)
    return int(out.value)


def abp_set_wait_limit(ctx, wait_limit_ns: int):
    _check(lib().abp_set_wait_limit(ctx, int(wait_limit_ns)), ctx)


def abp_test_hold_tile(ctx, tile: int):
    _check(lib().abp_test_hold_tile(ctx, int(tile)), ctx)


def abp_tuning(ctx):
    sc, p, s, b = C.c_int32(), C.c_int32(), C.c_int64(), C.c_int32()
    _check(lib().abp_tuning(ctx, C.byref(sc), C.byref(p), C.byref(s), C.byref(b)), ctx)
    return {"schedule": sc.value, "particles_per_thread": p.value, "steps_per_item": s.value, "blocks": b.value}


def abp_tuning_report(ctx) -> dict:
    """The autotuner's record for the current batch (candidates, probe times, choice)."""
    import json

    n = C.c_size_t()
    _check(lib().abp_tuning_report(ctx, None, 0, C.byref(n)), ctx)
    buf = C.create_string_buffer(n.value)
    _check(lib().abp_tuning_report(ctx, buf, n.value, None), ctx)
    return json.loads(buf.value.decode() or "{}")


def abp_tiles(ctx):
    t, p, n = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib().abp_tiles(ctx, C.byref(t), C.byref(p), C.byref(n)), ctx)
    return {"tiles": t.value, "packed": p.value, "narrow": n.value}


def abp_plan(n_traj, n_steps, schedule: int, particles_per_thread: int, checkpoints: bool = False,
             sm_count: int = 152) -> dict:
    """The tiling abp_set_params makes for this batch (host only, no GPU needed)."""
    n = len(n_traj)
    M = (C.c_int64 * max(n, 1))(*[int(v) for v in n_traj])
    N = (C.c_int64 * max(n, 1))(*[int(v) for v in n_steps])
    nt, npk, nar = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib().abp_plan(n, M, N, schedule, particles_per_thread, 1 if checkpoints else 0, sm_count, C.byref(nt),
                          C.byref(npk), C.byref(nar), None, None, None, 0), what="abp_plan")
    k = nt.value
    first, count, sset = (C.c_int64 * max(k, 1))(), (C.c_int32 * max(k, 1))(), (C.c_int32 * max(k, 1))()
    _check(lib().abp_plan(n, M, N, schedule, particles_per_thread, 1 if checkpoints else 0, sm_count, None, None,
                          None, first, count, sset, k), what="abp_plan")
    return {"tiles": k, "packed": npk.value, "narrow": nar.value, "tile_first": list(first[:k]),
            "tile_count": list(count[:k]), "tile_set": list(sset[:k])}


def abp_plan_efficiency(n_traj, n_steps, schedule: int, particles_per_thread: int, units: int,
                        checkpoints: bool = False, steps_per_launch: int = 0) -> float:
    """Busy fraction of `units` parallel units (the autotuner passes the SM count) for this batch."""
    n = len(n_traj)
    M = (C.c_int64 * max(n, 1))(*[int(v) for v in n_traj])
    N = (C.c_int64 * max(n, 1))(*[int(v) for v in n_steps])
    e = C.c_double()
    _check(lib().abp_plan_efficiency(n, M, N, schedule, particles_per_thread, 1 if checkpoints else 0,
                                     steps_per_launch, units, C.byref(e)), what="abp_plan_efficiency")
    return e.value


def abp_xorshift(seed: int, traj: int, out, stream=None):
    """The first out.numel() words of trajectory traj's xorshift stream (device int32 tensor)."""
    _check(lib().abp_xorshift(seed, traj, out.numel(), _ptr(out), _stream_ptr(stream)), what="abp_xorshift")


def abp_live(ctx, moments=None, hist_x=None, hist_v=None):
    """Stream every snapshot (moments [n_snap, n_sets, 8] float64, histograms int32) into
    page-locked host tensors while the integration runs; all None switches it off."""
    _check(lib().abp_live(ctx, _ptr(moments), _ptr(hist_x), _ptr(hist_v)), ctx)


def abp_live_ready(ctx) -> int:
    n = C.c_int64()
    _check(lib().abp_live_ready(ctx, C.byref(n)), ctx)
    return n.value


def abp_integrate(ctx, max_steps: int = -1):
    _check(lib().abp_integrate(ctx, int(max_steps)), ctx)


def abp_progress(ctx, n_sets: int):
    out = (C.c_int64 * max(n_sets, 1))()
    _check(lib().abp_progress(ctx, out), ctx)
    return [int(out[i]) for i in range(n_sets)]


def abp_num_snapshots(ctx) -> int:
    out = C.c_int64()
    _check(lib().abp_num_snapshots(ctx, C.byref(out)), ctx)
    return int(out.value)


def abp_reduce(ctx, moments=None, hist_x=None, hist_v=None):
    _check(lib().abp_reduce(ctx, _ptr(moments), _ptr(hist_x), _ptr(hist_v)), ctx)


def abp_get_state(ctx, x=None, x0=None, v=None, e=None, vbar=None):
    _check(lib().abp_get_state(ctx, _ptr(x), _ptr(x0), _ptr(v), _ptr(e), _ptr(vbar)), ctx)


def abp_save(ctx, buf=None):
    """Image of the context's batch.  buf: None (a new numpy uint8 host array is returned)
    or a contiguous host/device tensor or array large enough."""
    n = C.c_size_t(0)
    _check(lib().abp_save(ctx, None, C.byref(n)), ctx)
    if buf is None:
        buf = np.empty(n.value, dtype=np.uint8)
    have = C.c_size_t(buf.nbytes if isinstance(buf, np.ndarray) else buf.numel() * buf.element_size())
    _check(lib().abp_save(ctx, _ptr(buf), C.byref(have)), ctx)
    return buf


def abp_load(ctx, buf):
    nbytes = buf.nbytes if isinstance(buf, np.ndarray) else buf.numel() * buf.element_size()
    _check(lib().abp_load(ctx, _ptr(buf), nbytes), ctx)


def abp_backward(ctx, dJ_dmean_v=None, grad=None, window: int = 0):
    if window:
        _check(lib().abp_backward_windowed(ctx, _ptr(dJ_dmean_v), _ptr(grad), int(window)), ctx)
    else:
        _check(lib().abp_backward(ctx, _ptr(dJ_dmean_v), _ptr(grad)), ctx)


def abp_backward_traj(ctx, dvbar):
    """Per-trajectory derivatives [total_traj, 6] of the last backward call into dvbar."""
    _check(lib().abp_backward_traj(ctx, _ptr(dvbar)), ctx)


def abp_synchronize(ctx):
    _check(lib().abp_synchronize(ctx), ctx)


def abp_destroy(ctx):
    if ctx:
        lib().abp_destroy(ctx)


def abp_philox(seed: int, traj, m, out, stream=None):
    """traj, m: uint64 device tensors (int64 dtype reinterpreted); out: int32 device tensor [n, 4]."""
    n = traj.numel()
    _check(lib().abp_philox(seed, _ptr(traj), _ptr(m), n, _ptr(out), _stream_ptr(stream)),
           what="abp_philox rejected its arguments")


def abp_normals(seed: int, traj: int, n0: int, out, stream=None):
    _check(lib().abp_normals(seed, traj, n0, out.numel(), _ptr(out), _stream_ptr(stream)),
           what="abp_normals rejected its arguments")


def abp_version() -> str:
    return lib().abp_version().decode()


def abp_combine_moments(moments, n_traj, n_steps, dt: float, stream=None):
    """In place: columns 0..3 of ``moments`` [n_sets, 8] (float64, host array / tensor or device
    tensor) from the combined per-set sums in its columns 4..7, for n_traj[s] trajectories in all
    after n_steps[s] steps.  Host memory is processed at once, device memory on ``stream``."""
    shape = tuple(moments.shape)
    dtype_ok = (moments.dtype == np.float64) if isinstance(moments, np.ndarray) else (str(moments.dtype) == "torch.float64")
    if len(shape) != 2 or shape[1] != 8 or not dtype_ok:
        raise ValueError("moments must be a float64 array of shape [n_sets, 8], got %s %s" % (moments.dtype, shape))
    n = shape[0]
    if len(n_traj) != n or len(n_steps) != n:
        raise ValueError("n_traj and n_steps need one value per set")
    M = (C.c_int64 * max(n, 1))(*[int(v) for v in n_traj])
    N = (C.c_int64 * max(n, 1))(*[int(v) for v in n_steps])
    _check(lib().abp_combine_moments(n, _ptr(moments), M, N, float(dt), _stream_ptr(stream)),
           what="abp_combine_moments rejected its arguments")


# ----------------------------------------------------------------------- convenience

def make_config(w: "W.Workload", *, state_fp64: bool = False, particles_per_thread: int = 0,
                steps_per_launch: int = 0, traj_base: int = 0, schedule: int = 0,
                scheme: int | None = None, noise: int | None = None) -> abp_config:
    c = abp_config()
    c.seed = int(w.seed)
    c.dt = float(w.dt)
    c.v0_mode = int(w.v0_mode)
    c.state_fp64 = 1 if state_fp64 else 0
    c.hist_x_bins = int(w.hist_x_bins)
    c.hist_v_bins = int(w.hist_v_bins)
    c.v_lo = float(w.v_lo)
    c.v_hi = float(w.v_hi)
    c.snapshot_every = int(w.snapshot_every)
    c.checkpoint_every = int(w.checkpoint_every)
    c.particles_per_thread = int(particles_per_thread)
    c.schedule = int(schedule)
    c.steps_per_launch = int(steps_per_launch)
    c.traj_base = int(traj_base)
    c.scheme = int(w.scheme if scheme is None else scheme)
    c.noise = int(w.noise if noise is None else noise)
    return c


class Ensemble:
    """One context bound to a workload: ``run()`` integrates it and ``results()`` reduces it.

    Outputs are torch tensors on the context's device unless ``host=True``.
    """

    def __init__(self, w: "W.Workload", *, stream=None, state_fp64=False, particles_per_thread=0,
                 steps_per_launch=0, traj_base=0, schedule=0, scheme=None, device=None):
        import torch

        self.torch = torch
        self.w = w
        self.device = torch.device(device or "cuda")
        self.stream = stream
        with torch.cuda.device(self.device):
            self.ctx = abp_create(make_config(w, state_fp64=state_fp64, particles_per_thread=particles_per_thread,
                                              steps_per_launch=steps_per_launch, traj_base=traj_base,
                                              schedule=schedule, scheme=scheme), stream)
        self._params_set = False

    def close(self):
        if getattr(self, "ctx", None):
            abp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_params(self):
        abp_set_params(self.ctx, self.w.sets, self.w.n_traj, self.w.n_steps)
        self._params_set = True

    def reset(self, seed: int | None = None):
        abp_reset(self.ctx, self.w.seed if seed is None else seed)

    def launches(self) -> int:
        return abp_kernel_launches(self.ctx)

    def tuning(self) -> dict:
        return abp_tuning(self.ctx)

    def tiles(self) -> dict:
        return abp_tiles(self.ctx)

    def tuning_report(self) -> dict:
        return abp_tuning_report(self.ctx)

    def integrate(self, max_steps: int = -1):
        abp_integrate(self.ctx, max_steps)

    def run(self):
        self.set_params()
        self.integrate(-1)

    def n_snapshots(self) -> int:
        return abp_num_snapshots(self.ctx)

    def results(self, host: bool = False) -> dict:
        torch = self.torch
        dev = "cpu" if host else self.device
        kw = dict(device=dev)
        if host:
            kw["pin_memory"] = True
        S = self.w.n_sets
        mom = torch.empty((S, 8), dtype=torch.float64, **kw)
        ns = self.n_snapshots()
        hx = torch.empty((ns, S, self.w.hist_x_bins), dtype=torch.int32, **kw) if self.w.hist_x_bins and ns else None
        hv = (torch.empty((ns, S, self.w.hist_v_bins + 2), dtype=torch.int32, **kw)
              if self.w.hist_v_bins and ns else None)
        abp_reduce(self.ctx, mom, hx, hv)
        out = {"moments": mom}
        if hx is not None:
            out["hist_x"] = hx
        if hv is not None:
            out["hist_v"] = hv
        return out

    def state(self, host: bool = False) -> dict:
        torch = self.torch
        T = self.w.total_traj
        dev = "cpu" if host else self.device
        out = {k: torch.empty(T, dtype=torch.float64, device=dev) for k in ("x", "x0", "v", "e", "vbar")}
        abp_get_state(self.ctx, out["x"], out["x0"], out["v"], out["e"], out["vbar"])
        return out

    def backward(self, dJ=None, host: bool = False, window: int = 0):
        torch = self.torch
        dev = "cpu" if host else self.device
        g = torch.empty((self.w.n_sets, 6), dtype=torch.float64, device=dev)
        abp_backward(self.ctx, dJ, g, window)
        return g

    def traj_grad(self, host: bool = False):
        """d vbar_i / d theta for every trajectory, [total_traj, 6], from the last backward()."""
        torch = self.torch
        out = torch.empty((self.w.total_traj, 6), dtype=torch.float64, device="cpu" if host else self.device)
        abp_backward_traj(self.ctx, out)
        return out

    def synchronize(self):
        abp_synchronize(self.ctx)


class MeanVelocity:
    """``torch.autograd.Function`` over the ensemble: ``theta`` [n_sets, 6] holds
    (D, q, c, d, gamma0, asym) of every set (the other parameters come from the workload);
    the forward integrates the batch and returns the mean velocity of every set, the
    backward is the pathwise adjoint (noise held fixed) of ``abp_backward``.

    Usage: ``mean_v = MeanVelocity.apply(theta, workload)``.
    """

    _fn = None

    @classmethod
    def apply(cls, theta, w, **kw):
        if cls._fn is None:
            import torch

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, th, wl, opts):
                    sets = []
                    th_h = th.detach().double().cpu().numpy()
                    for i, base in enumerate(wl.sets):
                        s = dict(base)
                        for j, name in enumerate(GRAD_PARAMS):
                            s[name] = float(th_h[i, j])
                        sets.append(s)
                    import dataclasses

                    w2 = dataclasses.replace(wl, sets=sets, checkpoint_every=wl.checkpoint_every or 1000)
                    ens = Ensemble(w2, **opts)
                    ens.run()
                    mom = ens.results()["moments"]
                    ctx.ens = ens
                    return mom[:, 0].to(th.device, dtype=th.dtype)

                @staticmethod
                def backward(ctx, g):
                    ens = ctx.ens
                    w = g.detach().double().contiguous().to(ens.device)
                    grad = ens.backward(w)
                    ens.close()
                    return grad.to(g.device, dtype=g.dtype), None, None

            cls._fn = _F
        return cls._fn.apply(theta, w, kw)


def noalloc_snapshots(cfg: abp_config, n_steps: int) -> int:
    """Snapshot rows the allocation-free entry point writes for one set of n_steps steps."""
    if cfg.hist_x_bins <= 0 and cfg.hist_v_bins <= 0:
        return 0
    return int(n_steps) // int(cfg.snapshot_every) if cfg.snapshot_every > 0 else 1


def abp_run_set_noalloc(params: dict, cfg: abp_config, n_traj: int, n_steps: int, moments, hist_x=None, hist_v=None,
                        stream=None):
    """One parameter set integrated and reduced by the allocation-free entry point; the
    outputs are caller-owned tensors on the current CUDA device (moments >= 8 float64,
    histograms of a 4-byte integer type and at least n_snap x bins elements).  The C side
    cannot see the extent of these buffers, so they are checked here before the call."""
    import torch

    n_snap = noalloc_snapshots(cfg, n_steps)
    if moments is None or moments.dtype != torch.float64 or moments.numel() < 8:
        raise ValueError("moments must be a float64 tensor of at least 8 elements")
    need = (("hist_x", hist_x, cfg.hist_x_bins), ("hist_v", hist_v, cfg.hist_v_bins + 2 if cfg.hist_v_bins else 0))
    for name, t, bins in need:
        if bins <= 0:
            continue
        if t is None or t.dtype not in (torch.int32, getattr(torch, "uint32", torch.int32)):
            raise ValueError("%s must be an int32 tensor when its bins are > 0" % name)
        if t.numel() < n_snap * bins:
            raise ValueError("%s holds %d elements, %d snapshots x %d bins needed" % (name, t.numel(), n_snap, bins))
    dev = torch.cuda.current_device() if torch.cuda.is_available() else None
    for name, t in (("moments", moments), ("hist_x", hist_x), ("hist_v", hist_v)):
        if t is not None and (t.device.type != "cuda" or t.device.index != dev):
            raise ValueError("%s must be on the current CUDA device (cuda:%s), not %s" % (name, dev, t.device))
    p = abp_params()
    for k in W.PARAM_NAMES:
        setattr(p, k, float(params[k]))
    err = C.create_string_buffer(512)
    st = lib().abp_run_set_noalloc(C.byref(p), C.byref(cfg), int(n_traj), int(n_steps), _ptr(moments),
                                   _ptr(hist_x), _ptr(hist_v), _stream_ptr(stream), err, 512)
    if st != ABP_OK:
        raise AbpError(st, err.value.decode())
