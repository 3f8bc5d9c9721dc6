"""Pins of the FP64 oracle against facts fixed outside it (no GPU needed).

Each test checks the oracle against something other than itself: an independent
Philox implementation (ATen's host engine), closed forms of limits of the model of
Sec. 2, exact fixed points of the Euler-Maruyama map, equilibrium statistical
mechanics (Boltzmann / Maxwell densities) and the reflection symmetry of the model.
The choices are such that a dropped term, a wrong sign, a wrong factor (e.g. sqrt(D)
instead of sqrt(2D)) or a wrong index (x updated with v_{n+1}) fails at least one.
"""
import math
import os
import subprocess

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
BASE = dict(q=1.0, c=0.1, d=1.0, gamma0=1.0, F0=0.0, D=0.1, h=1.0, L=1.0, asym=0.25)


def P(**kw):
    p = dict(BASE)
    p.update(kw)
    return p


# --------------------------------------------------------------------------- Philox

@pytest.fixture(scope="module")
def aten_kat(tmp_path_factory):
    """Compile the ATen-engine known-answer helper (host C++, header-only engine)."""
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("ATen Philox header not present")
    exe = str(tmp_path_factory.mktemp("kat") / "aten_philox_kat")
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", inc, os.path.join(HERE, "helpers", "aten_philox_kat.cpp"),
                    "-o", exe], check=True)

    def run(triples):
        txt = "\n".join("%d %d %d" % t for t in triples) + "\n"
        out = subprocess.run([exe], input=txt, capture_output=True, text=True, check=True).stdout
        return [tuple(int(v) for v in line.split()) for line in out.strip().splitlines()]

    return run


def test_philox_matches_aten_engine(aten_kat):
    rng = np.random.default_rng(12345)
    triples = [(0, 0, 0), (0, 0, 1), (1, 0, 0), (0, 1, 0), (2**64 - 1, 2**64 - 1, 2**64 - 1),
               (3, 5, 2**63), (4, 2**32 + 7, 2**32 - 1), (0xDEADBEEFCAFEF00D, 123456789, 987654321)]
    for _ in range(300):
        triples.append((int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2)),
                        int(rng.integers(0, 2**40)), int(rng.integers(0, 2**36))))
    ref = aten_kat(triples)
    got = [O.noise_words(*t) for t in triples]
    assert got == ref


def test_philox_rounds_and_key_schedule_matter(aten_kat):
    # Distinct keys, counters and subsequences give distinct words (catches a dropped
    # key or counter word in the round function).
    a = O.noise_words(7, 11, 13)
    for alt in [(8, 11, 13), (7, 12, 13), (7, 11, 14), (7 + 2**32, 11, 13), (7, 11 + 2**32, 13),
                (7, 11, 13 + 2**32)]:
        assert O.noise_words(*alt) != a
        assert aten_kat([alt])[0] == O.noise_words(*alt)


# --------------------------------------------------------------------------- Box-Muller

def _normals(seed, traj, n0, count):
    import ctypes as C
    L = O.lib()
    L.or_normals.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, C.c_int64, C.POINTER(C.c_double)]
    out = np.zeros(count)
    L.or_normals(seed, traj, n0, count, out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def test_box_muller_branches_and_mapping():
    # u2 = 0 -> (r, 0); u2 = 1/2 -> (-r, 0); u2 = 1/4 -> (0, r): the cosine branch feeds
    # the even step, the sine branch the odd step, and u2 keeps the top 23 bits.
    r_half = math.sqrt(-2.0 * math.log(0.5 + 2.0**-33))  # u1 for w_a = 2^31
    z = O.box_muller(2**31, 0)
    assert z[0] == pytest.approx(r_half, rel=1e-15) and z[1] == 0.0
    z = O.box_muller(2**31, 2**31)
    assert z[0] == pytest.approx(-r_half, rel=1e-15) and abs(z[1]) < 1e-15
    z = O.box_muller(2**31, 2**30)
    assert abs(z[0]) < 1e-15 and z[1] == pytest.approx(r_half, rel=1e-15)
    # the low 9 bits of w_b do not enter u2
    assert O.box_muller(2**31, 2**30 + 511) == O.box_muller(2**31, 2**30)
    # u1 is never 0 or 1: both extreme words give finite r
    assert math.isfinite(O.box_muller(0, 0)[0]) and O.box_muller(0, 0)[0] > 6.6
    assert 0.0 < O.box_muller(2**32 - 1, 0)[0] < 1e-4
    # step n uses word pair (n mod 4) // 2 of counter n >> 2
    w = O.noise_words(9, 3, 5)
    assert O.normal(9, 3, 20) == O.box_muller(w[0], w[1])[0]
    assert O.normal(9, 3, 21) == O.box_muller(w[0], w[1])[1]
    assert O.normal(9, 3, 22) == O.box_muller(w[2], w[3])[0]
    assert O.normal(9, 3, 23) == O.box_muller(w[2], w[3])[1]


def test_box_muller_is_standard_normal():
    z = np.concatenate([_normals(0, t, 0, 250_000) for t in range(8)])  # 2e6 draws
    n = z.size
    assert abs(z.mean()) < 4.0 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 4.0 * math.sqrt(2.0 / n)
    assert abs(stats.kurtosis(z, fisher=False) - 3.0) < 4.0 * math.sqrt(24.0 / n)
    assert abs(stats.skew(z)) < 4.0 * math.sqrt(6.0 / n)
    # chi^2 against N(0,1) on 64 equiprobable bins
    edges = stats.norm.ppf(np.linspace(0, 1, 65))
    counts, _ = np.histogram(z, bins=edges)
    p = stats.chisquare(counts).pvalue
    assert p > 1e-3
    # consecutive steps are uncorrelated (pairs share r)
    assert abs(np.corrcoef(z[:-1], z[1:])[0, 1]) < 4.0 / math.sqrt(n)


# --------------------------------------------------------------------------- potential

def _golden_extrema():
    vals = {}
    with open(os.path.join(HERE, "golden", "eq_pot_extrema.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    return vals


def test_potential_extrema_closed_form():
    g = _golden_extrema()
    p = P(h=1.0, L=1.0, asym=g["const_asym"])
    xs = np.linspace(-0.5, 0.5, 200_001)
    U = np.array([O.potential(p, x) for x in xs])
    i = int(np.argmin(U))
    assert xs[i] == pytest.approx(g["x_min"], abs=2e-5)
    assert U[i] == pytest.approx(g["U_min"], abs=2e-7)
    xs2 = np.linspace(0.5, 0.75, 100_001)
    U2 = np.array([O.potential(p, x) for x in xs2])
    j = int(np.argmax(U2))
    assert xs2[j] == pytest.approx(g["x_max"], abs=2e-5)
    assert U2[j] == pytest.approx(g["U_max"], abs=2e-7)
    # barrier normalised to h by the 0.499 / 0.453 pair
    assert U2[j] - U[i] == pytest.approx(2 * g["const_amplitude"] * g["S"], abs=1e-6)


def test_potential_derivative_scaling_and_period():
    for p in [P(), P(asym=0.0), P(asym=0.5, h=2.5), P(L=2.0), P(L=0.5, h=0.3, asym=0.1)]:
        L = p["L"]
        for x in np.linspace(-1.3 * L, 2.1 * L, 37):
            hstep = 1e-5 * L
            fd = (O.potential(p, x + hstep) - O.potential(p, x - hstep)) / (2 * hstep)
            assert O.potential_dx(p, x) == pytest.approx(fd, rel=1e-7, abs=1e-8 * p["h"] / L)
            assert O.potential(p, x + L) == pytest.approx(O.potential(p, x), abs=1e-12)
        # zero mean force over one period
        xs = np.linspace(0, L, 4096, endpoint=False)
        assert abs(np.mean([O.potential_dx(p, x) for x in xs])) < 1e-12
    # period L stretches x: U_L(L x) = U_1(x), h scales U linearly
    for x in np.linspace(0, 1, 11):
        assert O.potential(P(L=3.0), 3.0 * x) == pytest.approx(O.potential(P(L=1.0), x), abs=1e-12)
        assert O.potential(P(h=2.0), x) == pytest.approx(2.0 * O.potential(P(h=1.0), x), abs=1e-12)


def test_potential_asymmetry():
    # a = 1/4: minimum at 0, maximum at ~0.62 -> asymmetric ratchet; a = 0: maximum half a period away
    xs = np.linspace(0, 1, 20_000, endpoint=False)
    U = np.array([O.potential(P(asym=0.0), x) for x in xs])
    gap = (xs[np.argmax(U)] - xs[np.argmin(U)]) % 1.0
    assert gap == pytest.approx(0.5, abs=1e-3)
    U = np.array([O.potential(P(asym=0.25), x) for x in xs])
    gap = (xs[np.argmax(U)] - xs[np.argmin(U)]) % 1.0
    assert 0.55 < gap < 0.7


# --------------------------------------------------------------------------- deterministic limits

def test_depot_relaxation_exact():
    # d = 0, D = 0, h = 0, F0 = 0, v0 = 0: e_n = q/c + (e_0 - q/c)(1 - c dt)^n exactly
    p = P(d=0.0, D=0.0, h=0.0, q=0.7, c=0.3)
    dt, N = 1e-3, 4000
    r = O.run_set(p, seed=5, dt=dt, n_traj=3, n_steps=N, want_states=True)
    e_exact = p["q"] / p["c"] * (1.0 - (1.0 - p["c"] * dt) ** N)
    np.testing.assert_allclose(r["e"], e_exact, rtol=1e-12)
    np.testing.assert_allclose(r["v"], 0.0, atol=0)
    np.testing.assert_allclose(r["x"], r["x0"], atol=0)


def test_depot_fixed_point_frozen_velocity():
    # with the velocity pinned by the force balance the depot sits at e0 = q/(c + d v^2):
    # a state (x, v, q/(c + d v^2)) keeps e exactly when the step is taken
    for v in (0.0, 0.3, -1.2):
        p = P()
        e0 = p["q"] / (p["c"] + p["d"] * v * v)
        _, _, e1 = O.em_step(p, 1e-3, 0.0, (0.2, v, e0))
        assert e1 == pytest.approx(e0, rel=1e-14)


def test_active_motion_fixed_point():
    # D = 0, h = 0, F0 = 0, q d / c > gamma0: v -> +-sqrt(q/gamma0 - c/d), e -> gamma0/d,
    # an exact fixed point of the map and the attractor from v = 0.3, e = 0
    p = P(D=0.0, h=0.0, q=1.3, c=0.2, d=0.8, gamma0=0.9)
    v_star = math.sqrt(p["q"] / p["gamma0"] - p["c"] / p["d"])
    e_star = p["gamma0"] / p["d"]
    x1, v1, e1 = O.em_step(p, 1e-3, 0.7, (0.4, -v_star, e_star))
    assert v1 == pytest.approx(-v_star, rel=1e-14) and e1 == pytest.approx(e_star, rel=1e-14)
    assert x1 == pytest.approx(0.4 - v_star * 1e-3, rel=1e-14)
    s = (0.0, 0.3, 0.0)
    for _ in range(30_000):
        s = O.em_step(p, 5e-3, 0.0, s)
    assert s[1] == pytest.approx(v_star, rel=1e-6) and s[2] == pytest.approx(e_star, rel=1e-6)


def test_constant_force_passive_exact():
    # d = 0, h = 0, D = 0: v_n = (F0/gamma0)(1 - (1 - gamma0 dt)^n);
    # x_N - x_0 = dt sum_{n<N} v_n  (position uses the velocity of step n)
    p = P(d=0.0, h=0.0, D=0.0, F0=0.5, gamma0=2.0)
    dt, N = 1e-3, 3000
    r = O.run_set(p, seed=6, dt=dt, n_traj=2, n_steps=N, want_states=True)
    rho = 1.0 - p["gamma0"] * dt
    vinf = p["F0"] / p["gamma0"]
    np.testing.assert_allclose(r["v"], vinf * (1 - rho**N), rtol=1e-12)
    dx = dt * vinf * (N - (1 - rho**N) / (1 - rho))
    np.testing.assert_allclose(r["x"] - r["x0"], dx, rtol=1e-10)
    np.testing.assert_allclose(r["vbar"], dx / (N * dt), rtol=1e-10)


def test_em_identity_time_average_equals_displacement():
    # sum_{n<N} v_n dt = x_N - x_0 holds path by path for the scheme
    r = O.run_set(P(D=0.3), seed=7, dt=1e-3, n_traj=64, n_steps=2000, v0_mode=1, want_states=True)
    np.testing.assert_allclose(r["vbar"] * 2000 * 1e-3, r["x"] - r["x0"], rtol=1e-9, atol=1e-12)


# --------------------------------------------------------------------------- stochastic limits

def test_free_passive_ou_variance_and_msd():
    # d = 0, h = 0, F0 = 0: Ornstein-Uhlenbeck velocity.  For the EM map, with v0 = 0,
    #   Var v_N = 2 D dt (1 - rho^{2N}) / (1 - rho^2),      rho = 1 - gamma0 dt
    #   Var(x_N - x_0) = dt^2 2 D dt sum_{k<N} ((1 - rho^{N-1-k}) / (1 - rho))^2
    # -> stationary <v^2> = D / (gamma0 (1 - gamma0 dt / 2)); MSD slope 2 D / gamma0^2.
    p = P(d=0.0, h=0.0, F0=0.0, D=0.3, gamma0=2.0)
    dt, N, M = 1e-2, 1500, 20_000
    r = O.run_set(p, seed=8, dt=dt, n_traj=M, n_steps=N, want_states=True)
    rho = 1 - p["gamma0"] * dt
    s2 = 2 * p["D"] * dt
    var_v = s2 * (1 - rho ** (2 * N)) / (1 - rho**2)
    v2 = np.mean(r["v"] ** 2)
    assert abs(v2 - var_v) < 4 * var_v * math.sqrt(2.0 / M)
    k = np.arange(N)
    var_dx = dt * dt * s2 * np.sum(((1 - rho ** (N - 1 - k)) / (1 - rho)) ** 2)
    msd = np.mean((r["x"] - r["x0"]) ** 2)
    assert abs(msd - var_dx) < 4 * var_dx * math.sqrt(2.0 / M)
    # long-time diffusion: D_eff -> D / gamma0^2 (Einstein), to O(1/(gamma0 T))
    assert r["d_eff"] == pytest.approx(p["D"] / p["gamma0"] ** 2, rel=0.08)
    # the moments the oracle derives from its four ensemble sums, against the same closed
    # form: E[dx] = 0, so msd -> Var(dx); vbar = dx / (N dt), so the standard error of the
    # mean velocity is sqrt(Var(dx) / M) / (N dt).  The sample variance of M Gaussian values
    # has relative spread sqrt(2 / (M - 1)), its square root half of that.
    T = N * dt
    assert abs(r["msd"] - var_dx) < 4 * var_dx * math.sqrt(2.0 / M)
    se_exact = math.sqrt(var_dx / M) / T
    assert abs(r["se_v"] - se_exact) < 4 * se_exact * math.sqrt(0.5 / (M - 1))
    assert abs(r["mean_v"]) < 4 * se_exact
    assert r["d_eff"] == pytest.approx((r["msd"] - (r["sums"][2] / M) ** 2) / (2 * T), rel=1e-12)


def test_standard_error_of_a_two_point_ensemble():
    # brute force on the smallest ensemble with a standard error: two trajectories whose
    # time averages are a and b have mean (a + b) / 2 and standard error |a - b| / 2
    # (sample variance (a - b)^2 / 2 over M = 2), whatever the dynamics
    r = O.run_set(P(D=0.4), seed=15, dt=1e-3, n_traj=2, n_steps=300, want_states=True)
    a, b = r["vbar"]
    assert r["mean_v"] == pytest.approx((a + b) / 2, rel=1e-12)
    assert r["se_v"] == pytest.approx(abs(a - b) / 2, rel=1e-12)
    dx = r["x"] - r["x0"]
    assert r["msd"] == pytest.approx((dx[0] ** 2 + dx[1] ** 2) / 2, rel=1e-12)
    assert r["d_eff"] == pytest.approx(((dx[0] - dx[1]) / 2) ** 2 / (2 * 300 * 1e-3), rel=1e-9)
    # one trajectory has no standard error, an empty ensemble no moments
    r1 = O.run_set(P(D=0.4), seed=15, dt=1e-3, n_traj=1, n_steps=300)
    assert r1["se_v"] == 0.0 and r1["mean_v"] == pytest.approx(a, rel=1e-12)


def test_initial_conditions():
    p = P(D=0.37, L=2.0)
    x0 = np.empty(20_000)
    v0 = np.empty(20_000)
    for t in range(x0.size):
        x0[t], v0[t], e0 = O.initial_state(p, 11, 1, t)
        assert e0 == 0.0
    assert x0.min() >= 0.0 and x0.max() < p["L"]
    k = x0 / p["L"] * 2**24
    assert np.all(k == np.floor(k))  # 24-bit uniform grid
    assert stats.kstest(x0 / p["L"], "uniform").pvalue > 1e-3
    assert stats.kstest(v0 / math.sqrt(p["D"]), "norm").pvalue > 1e-3
    assert O.initial_state(p, 11, 0, 5)[1] == 0.0
    # the initial draw does not reuse the counters of the steps
    w_init = O.noise_words(11, 5, 2**63)
    assert all(O.noise_words(11, 5, m) != w_init for m in range(64))


def test_passive_particle_reaches_boltzmann_and_maxwell():
    # d = 0, F0 = 0: stationary density of x mod L is exp(-U(x) gamma0 / D) and v ~ N(0, D/gamma0)
    p = P(d=0.0, F0=0.0, D=0.5, gamma0=1.0)
    dt, N, M, B = 2e-3, 10_000, 4_000, 20
    r = O.run_set(p, seed=9, dt=dt, n_traj=M, n_steps=N, hist_x_bins=B, hist_v_bins=B, v_lo=-3.0, v_hi=3.0)
    kT = p["D"] / p["gamma0"]
    fine = np.linspace(0, 1, B * 200, endpoint=False) + 0.5 / (B * 200)
    w = np.exp(-np.array([O.potential(p, x) for x in fine]) / kT)
    expect = w.reshape(B, 200).sum(1)
    expect = expect / expect.sum() * M
    hx = r["hist_x"][0].astype(float)
    assert hx.sum() == M
    assert stats.chisquare(hx, expect).pvalue > 1e-3
    hv = r["hist_v"][0].astype(float)
    edges = np.linspace(-3, 3, B + 1)
    cdf = stats.norm.cdf(edges, scale=math.sqrt(kT))
    ev = np.diff(cdf) * M
    tails = np.array([cdf[0] * M, (1 - cdf[-1]) * M])
    obs = np.concatenate([hv[:B], [hv[B] + hv[B + 1]]])
    exp = np.concatenate([ev, [tails.sum()]])
    assert stats.chisquare(obs, exp * obs.sum() / exp.sum()).pvalue > 1e-3


def test_symmetric_potential_has_no_current():
    # a = 0, F0 = 0: the model is invariant under reflection about a potential extremum,
    # so the mean velocity vanishes; with a = 1/4 the current is allowed to be non-zero.
    p = P(asym=0.0, D=0.1)
    r = O.run_set(p, seed=10, dt=2e-3, n_traj=3000, n_steps=10_000)
    assert abs(r["mean_v"]) < 3.5 * r["se_v"]


# --------------------------------------------------------------------------- gradient

def test_tangent_linear_matches_central_differences():
    # central differences of mean(vbar) with common random numbers (same seed), FP64
    base = P(D=0.08)
    kw = dict(seed=12, dt=1e-3, n_traj=16, n_steps=800, v0_mode=1)
    g = O.run_set(base, want_grad=True, **kw)["grad"]
    for j, name in enumerate(O.GRAD_PARAMS):
        h = 1e-4 * abs(base[name])
        up = O.run_set(dict(base, **{name: base[name] + h}), **kw)["mean_v"]
        dn = O.run_set(dict(base, **{name: base[name] - h}), **kw)["mean_v"]
        fd = (up - dn) / (2 * h)
        assert g[j] == pytest.approx(fd, rel=2e-5, abs=1e-9), name


def test_tangent_in_D_is_undefined_at_zero_noise():
    # sigma = sqrt(2 D dt) has no derivative at D = 0: the D-component is NaN there (for any
    # run of two or more steps, or a random initial velocity); the other five components
    # are those of the deterministic model, checked against central differences
    base = P(D=0.0, F0=0.1)
    for v0_mode, n_steps in ((0, 400), (1, 400), (1, 1)):
        kw = dict(seed=14, dt=1e-3, n_traj=8, n_steps=n_steps, v0_mode=v0_mode)
        g = O.run_set(base, want_grad=True, **kw)["grad"]
        assert math.isnan(g[0]), (v0_mode, n_steps)
        for j, name in enumerate(O.GRAD_PARAMS[1:], start=1):
            h = 1e-4 * abs(base[name])
            up = O.run_set(dict(base, **{name: base[name] + h}), **kw)["mean_v"]
            dn = O.run_set(dict(base, **{name: base[name] - h}), **kw)["mean_v"]
            assert g[j] == pytest.approx((up - dn) / (2 * h), rel=2e-5, abs=1e-9), (v0_mode, name)
    # no step taken: the time average is defined as 0, and so is every derivative
    assert np.all(O.run_set(base, want_grad=True, seed=14, dt=1e-3, n_traj=4, n_steps=0)["grad"] == 0.0)


# --------------------------------------------------------------------------- bookkeeping

def test_snapshots_histograms_and_threads():
    p = P(D=0.2)
    kw = dict(seed=13, dt=1e-3, n_traj=257, n_steps=1000, snapshot_every=300, hist_x_bins=32,
              hist_v_bins=16, v_lo=-1.0, v_hi=1.0)
    a = O.run_set(p, n_threads=1, **kw)
    b = O.run_set(p, n_threads=7, **kw)
    assert a["hist_x"].shape == (3, 32) and a["hist_v"].shape == (3, 18)
    assert np.all(a["hist_x"].sum(1) == 257) and np.all(a["hist_v"].sum(1) == 257)
    for k in ("hist_x", "hist_v", "vbar"):
        np.testing.assert_array_equal(a[k], b[k])
    np.testing.assert_array_equal(a["sums"], b["sums"])
    # the last snapshot of a run of N = 900 steps is the final-state histogram of that run
    c = O.run_set(p, n_threads=3, **dict(kw, n_steps=900, snapshot_every=0))
    np.testing.assert_array_equal(c["hist_x"][0], a["hist_x"][2])


def test_edge_cases():
    p = P()
    r = O.run_set(p, seed=1, dt=1e-3, n_traj=0, n_steps=100, hist_x_bins=8)
    assert r["sums"].tolist() == [0, 0, 0, 0] and r["hist_x"].sum() == 0
    r = O.run_set(p, seed=1, dt=1e-3, n_traj=5, n_steps=0, hist_x_bins=8, want_states=True)
    assert r["hist_x"].sum() == 5 and np.all(r["vbar"] == 0) and np.all(r["x"] == r["x0"])
    with pytest.raises(ValueError):
        O.run_set(p, seed=1, dt=-1e-3, n_traj=5, n_steps=10)


# --------------------------------------------------------------------------- windowed gradient

def _gamma_tangent_closed_form(F0, g, dt, N, W):
    # D = 0, d = 0, h = 0, v0 = 0: v_i = vinf (1 - rho^i), rho = 1 - g dt, and the tangent along
    # gamma0 obeys t_{i+1} = rho t_i - dt v_i from t = 0 at each window start s:
    #   t_{s+j} = -dt vinf [ (1 - rho^j) / (1 - rho) - j rho^(s+j-1) ]
    rho, vinf = 1 - g * dt, F0 / g
    n = np.arange(N)
    s = (n // W) * W if W > 0 else np.zeros_like(n)
    j = n - s
    t = -dt * vinf * ((1 - rho**j) / (1 - rho) - j * rho ** np.maximum(s + j - 1, 0))
    t[j == 0] = 0.0
    return t.mean()


@pytest.mark.parametrize("W", [0, 1, 37, 500, 5000])
def test_windowed_tangent_closed_form(W):
    p = P(d=0.0, h=0.0, D=0.0, F0=0.4, gamma0=1.5)
    dt, N = 1e-2, 1200
    r = O.run_set(p, seed=2, dt=dt, n_traj=3, n_steps=N, want_grad=True, grad_window=W)
    expect = _gamma_tangent_closed_form(p["F0"], p["gamma0"], dt, N, W if W < N else 0)
    gi = O.GRAD_PARAMS.index("gamma0")
    assert r["grad"][gi] == pytest.approx(expect, rel=1e-10)


def test_windowed_gradient_limits():
    p = P(D=0.2)
    kw = dict(seed=4, dt=1e-3, n_traj=16, n_steps=700, v0_mode=1, want_grad=True)
    full = O.run_set(p, **kw)["grad"]
    np.testing.assert_array_equal(O.run_set(p, grad_window=700, **kw)["grad"], full)
    np.testing.assert_array_equal(O.run_set(p, grad_window=10_000, **kw)["grad"], full)
    # one-step windows: only the initial velocity's dependence on D survives, in step 0
    r = O.run_set(p, grad_window=1, **kw)
    assert np.all(r["grad"][1:] == 0.0)
    v0 = np.array([O.initial_state(p, 4, 1, t)[1] for t in range(16)])
    assert r["grad"][0] == pytest.approx(v0.mean() / (2 * p["D"]) / 700, rel=1e-12)
