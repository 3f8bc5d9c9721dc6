"""Python access to the FP64 CPU oracle (``abp_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Imported by the tests, by the smoke check and by the
benchmark's CPU-baseline / reference leg; the library path never imports it.
It shares no code with the CUDA path.

``build()`` compiles ``abp_oracle.c`` with the host C compiler into
``oracle/_build/libabp_oracle.so``; ``lib()`` loads it (building on first use).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "abp_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libabp_oracle.so")
_lock = threading.Lock()
_lib = None

# Order of the tangent directions returned by the gradient.
GRAD_PARAMS = ("D", "q", "c", "d", "gamma0", "asym")


class Params(C.Structure):
    """Model parameters of one set, Sec. 2: Eqs. (ereservoir), (velocity), (pot)."""

    _fields_ = [(n, C.c_double) for n in ("q", "c", "d", "gamma0", "F0", "D", "h", "L", "asym")]


class RunArgs(C.Structure):
    _fields_ = [
        ("p", Params),
        ("seed", C.c_uint64),
        ("dt", C.c_double),
        ("traj_base", C.c_int64),
        ("n_traj", C.c_int64),
        ("n_steps", C.c_int64),
        ("snapshot_every", C.c_int64),
        ("v0_mode", C.c_int32),
        ("n_threads", C.c_int32),
        ("hist_x_bins", C.c_int32),
        ("hist_v_bins", C.c_int32),
        ("v_lo", C.c_double),
        ("v_hi", C.c_double),
        ("want_grad", C.c_int32),
        ("scheme", C.c_int32),
        ("noise", C.c_int32),
        ("reserved", C.c_int32),
        ("grad_window", C.c_int64),
    ]


_PD = C.POINTER(C.c_double)
_PU64 = C.POINTER(C.c_uint64)


class RunOut(C.Structure):
    _fields_ = [
        ("x0", _PD), ("x", _PD), ("v", _PD), ("e", _PD), ("vbar", _PD), ("dvbar", _PD),
        ("hist_x", _PU64), ("hist_v", _PU64),
        ("sums", C.c_double * 4), ("grad", C.c_double * 6),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, FP64, no FMA contraction so both hosts agree)."""
    with _lock:
        if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
            return _SO
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _SO + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-D_GNU_SOURCE", _SRC, "-o", tmp, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
        return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
        L.or_noise_words.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, C.POINTER(C.c_uint32)]
        L.or_box_muller.argtypes = [C.c_uint32, C.c_uint32, _PD]
        L.or_normal.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
        L.or_normal.restype = C.c_double
        L.or_potential.argtypes = [C.POINTER(Params), C.c_double]
        L.or_potential.restype = C.c_double
        L.or_potential_dx.argtypes = [C.POINTER(Params), C.c_double]
        L.or_potential_dx.restype = C.c_double
        L.or_em_step.argtypes = [C.POINTER(Params), C.c_double, C.c_double, _PD]
        L.or_heun_step.argtypes = [C.POINTER(Params), C.c_double, C.c_double, _PD, _PD]
        L.or_xorshift128_step.argtypes = [C.POINTER(C.c_uint32)]
        L.or_xorshift128_step.restype = C.c_uint32
        L.or_xorshift_seed.argtypes = [C.c_uint64, C.c_uint64, C.POINTER(C.c_uint32)]
        L.or_xorshift_normal.argtypes = [C.POINTER(C.c_uint32)]
        L.or_xorshift_normal.restype = C.c_double
        L.or_initial_state.argtypes = [C.POINTER(Params), C.c_uint64, C.c_int32, C.c_uint64, _PD]
        L.or_n_snapshots.argtypes = [C.c_int64, C.c_int64]
        L.or_n_snapshots.restype = C.c_int64
        L.or_run_set.argtypes = [C.POINTER(RunArgs), C.POINTER(RunOut)]
        L.or_run_set.restype = C.c_int
        _lib = L
    return _lib


def make_params(**kw) -> Params:
    p = Params()
    for name, _ in Params._fields_:
        setattr(p, name, float(kw[name]))
    return p


# ---------------------------------------------------------------- primitives

def philox(ctr, key):
    """Philox4x32-10 of one (counter[4], key[2]) block."""
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return tuple(int(v) for v in o)


def noise_words(seed: int, traj: int, m: int):
    o = (C.c_uint32 * 4)()
    lib().or_noise_words(seed, traj, m, o)
    return tuple(int(v) for v in o)


def box_muller(wa: int, wb: int):
    z = (C.c_double * 2)()
    lib().or_box_muller(wa, wb, z)
    return z[0], z[1]


def normal(seed: int, traj: int, n: int) -> float:
    return lib().or_normal(seed, traj, n)


def potential(params: dict, x: float) -> float:
    return lib().or_potential(C.byref(make_params(**params)), x)


def potential_dx(params: dict, x: float) -> float:
    return lib().or_potential_dx(C.byref(make_params(**params)), x)


def em_step(params: dict, dt: float, z: float, state):
    s = (C.c_double * 3)(*state)
    lib().or_em_step(C.byref(make_params(**params)), dt, z, s)
    return s[0], s[1], s[2]


def heun_step(params: dict, dt: float, z: float, state):
    """One stochastic Heun step; returns the new (x, v, e) and the predictor's velocity."""
    s = (C.c_double * 3)(*state)
    vp = C.c_double()
    lib().or_heun_step(C.byref(make_params(**params)), dt, z, s, C.byref(vp))
    return (s[0], s[1], s[2]), vp.value


def xorshift_step(state):
    """One xorshift call: returns (output word, new state)."""
    s = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in state])
    out = lib().or_xorshift128_step(s)
    return int(out), tuple(int(v) for v in s)


def xorshift_seed(seed: int, traj: int):
    s = (C.c_uint32 * 4)()
    lib().or_xorshift_seed(seed, traj, s)
    return tuple(int(v) for v in s)


def xorshift_words(seed: int, traj: int, count: int):
    """The first `count` words of trajectory traj's xorshift stream."""
    s = (C.c_uint32 * 4)(*xorshift_seed(seed, traj))
    return [int(lib().or_xorshift128_step(s)) for _ in range(count)]


def initial_state(params: dict, seed: int, v0_mode: int, traj: int):
    s = (C.c_double * 3)()
    lib().or_initial_state(C.byref(make_params(**params)), seed, v0_mode, traj, s)
    return s[0], s[1], s[2]


def n_snapshots(n_steps: int, snapshot_every: int) -> int:
    return int(lib().or_n_snapshots(n_steps, snapshot_every))


# ---------------------------------------------------------------- ensemble run

def run_set(params: dict, *, seed: int, dt: float, n_traj: int, n_steps: int, traj_base: int = 0,
            v0_mode: int = 0, snapshot_every: int = 0, hist_x_bins: int = 0, hist_v_bins: int = 0,
            v_lo: float = -5.0, v_hi: float = 5.0, want_states: bool = False, want_grad: bool = False,
            want_traj_grad: bool = False, n_threads: int | None = None, scheme: int = 0, noise: int = 0,
            grad_window: int = 0) -> dict:
    """Integrate one parameter set's ensemble in FP64 and reduce it.

    ``scheme`` 0 is the paper's explicit Euler-Maruyama step, 1 the stochastic Heun
    predictor-corrector on the same noise (no gradient for it).  ``noise`` 0 is the
    counter-based Philox stream, 1 Marsaglia's xorshift per trajectory (two words and one
    Box-Muller cosine per step; no gradient for it).  ``grad_window`` W > 0 restarts the
    tangents at steps W, 2W, ...: the windowed gradient (each window's contribution to the
    time average differentiated with the window's initial state held fixed).

    Returns a dict with ``sums`` = (sum vbar, sum vbar^2, sum dx, sum dx^2), the derived
    ``mean_v``, ``se_v``, ``msd``, ``d_eff``, per-trajectory ``vbar`` and (optionally) the
    final states, the histograms ``hist_x`` [n_snap, bins] and ``hist_v`` [n_snap, bins+2]
    and the tangent-linear gradient ``grad`` of mean(vbar) w.r.t. GRAD_PARAMS.
    """
    L = lib()
    a = RunArgs()
    a.p = make_params(**params)
    a.seed, a.dt, a.traj_base, a.n_traj, a.n_steps = seed, dt, traj_base, n_traj, n_steps
    a.snapshot_every, a.v0_mode = snapshot_every, v0_mode
    a.n_threads = n_threads if n_threads else (os.cpu_count() or 1)
    a.hist_x_bins, a.hist_v_bins, a.v_lo, a.v_hi = hist_x_bins, hist_v_bins, v_lo, v_hi
    a.want_grad = 1 if (want_grad or want_traj_grad) else 0
    a.scheme = int(scheme)
    a.noise = int(noise)
    a.grad_window = int(grad_window)
    o = RunOut()
    out: dict = {}
    keep = []

    def buf(name, shape, dtype, field):
        arr = np.zeros(shape, dtype=dtype)
        keep.append(arr)
        setattr(o, field, arr.ctypes.data_as(_PU64 if dtype == np.uint64 else _PD))
        out[name] = arr

    buf("vbar", (n_traj,), np.float64, "vbar")
    if want_states:
        for f in ("x0", "x", "v", "e"):
            buf(f, (n_traj,), np.float64, f)
    if want_traj_grad:
        buf("dvbar", (n_traj, 6), np.float64, "dvbar")
    n_snap = n_snapshots(n_steps, snapshot_every)
    if hist_x_bins > 0:
        buf("hist_x", (n_snap, hist_x_bins), np.uint64, "hist_x")
    if hist_v_bins > 0:
        buf("hist_v", (n_snap, hist_v_bins + 2), np.uint64, "hist_v")
    rc = L.or_run_set(C.byref(a), C.byref(o))
    if rc != 0:
        raise ValueError("oracle run_set failed with code %d" % rc)
    sums = np.array(o.sums[:], dtype=np.float64)
    out["sums"] = sums
    out.update(derived_moments(sums, n_traj, n_steps, dt))
    if a.want_grad:
        out["grad"] = np.array(o.grad[:], dtype=np.float64)
    return out


def derived_moments(sums, n_traj: int, n_steps: int, dt: float) -> dict:
    """Ensemble mean of the time-averaged velocity, its standard error, the mean squared
    displacement and D_eff = Var(dx) / (2 T) from the four per-set sums."""
    M = float(n_traj)
    if M == 0:
        return dict(mean_v=0.0, se_v=0.0, msd=0.0, d_eff=0.0)
    mean_v = sums[0] / M
    var_v = (sums[1] - M * mean_v * mean_v) / (M - 1) if M > 1 else 0.0
    se_v = float(np.sqrt(max(var_v, 0.0) / M))
    msd = sums[3] / M
    mdx = sums[2] / M
    T = n_steps * dt
    d_eff = (msd - mdx * mdx) / (2.0 * T) if T > 0 else 0.0
    return dict(mean_v=float(mean_v), se_v=se_v, msd=float(msd), d_eff=float(d_eff))
