"""Pins of the oracle's stochastic Heun step (the higher-order variant of the step of
Fig. 1) against facts fixed outside it: closed forms of the Heun map in the linear
limits of the model of Sec. 2, its fixed points, the single entry of the noise
increment, and its second-order convergence on the deterministic model.

A corrector that averages the wrong stages, a noise increment counted twice or
averaged, a position advanced with v_n instead of (v_n + v~)/2, or a predictor
without the noise each fails at least one of these.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O

BASE = dict(q=1.0, c=0.1, d=1.0, gamma0=1.0, F0=0.0, D=0.1, h=1.0, L=1.0, asym=0.25)


def P(**kw):
    p = dict(BASE)
    p.update(kw)
    return p


def test_heun_depot_relaxation_exact():
    # d = 0, D = 0, h = 0, F0 = 0, v0 = 0: e' = e + dt/2 [(q - c e) + (q - c e~)] with
    # e~ = e + dt (q - c e), so e_n - q/c = (e_0 - q/c) rho^n, rho = 1 - c dt + (c dt)^2 / 2
    p = P(d=0.0, D=0.0, h=0.0, q=0.7, c=0.3)
    dt, N = 2e-2, 3000
    r = O.run_set(p, seed=5, dt=dt, n_traj=3, n_steps=N, want_states=True, scheme=1)
    rho = 1.0 - p["c"] * dt + 0.5 * (p["c"] * dt) ** 2
    np.testing.assert_allclose(r["e"], p["q"] / p["c"] * (1.0 - rho**N), rtol=1e-12)
    np.testing.assert_allclose(r["v"], 0.0, atol=0)
    np.testing.assert_allclose(r["x"], r["x0"], atol=0)


def test_heun_constant_force_passive_exact():
    # d = 0, h = 0, D = 0: v' = a v + F0 dt (1 - g dt / 2), a = 1 - g dt + (g dt)^2 / 2, so
    # v_n = (F0/g)(1 - a^n); x advances by dt (v (1 - g dt / 2) + F0 dt / 2)
    p = P(d=0.0, h=0.0, D=0.0, F0=0.5, gamma0=2.0)
    dt, N = 1e-2, 700
    g = p["gamma0"]
    r = O.run_set(p, seed=6, dt=dt, n_traj=2, n_steps=N, want_states=True, scheme=1)
    a = 1.0 - g * dt + 0.5 * (g * dt) ** 2
    vinf = p["F0"] / g
    np.testing.assert_allclose(r["v"], vinf * (1 - a**N), rtol=1e-12)
    sum_v = vinf * (N - (1 - a**N) / (1 - a))
    dx = dt * ((1 - 0.5 * g * dt) * sum_v + N * p["F0"] * dt / 2)
    np.testing.assert_allclose(r["x"] - r["x0"], dx, rtol=1e-10)
    np.testing.assert_allclose(r["vbar"], dx / (N * dt), rtol=1e-10)


def test_heun_noise_enters_once():
    # no drift at all (d = 0, h = 0, F0 = 0, gamma0 = 0, q = c = 0): both stages see the
    # same increment w_n = sqrt(2 D dt) z_n, which the corrector adds once:
    #   v_N = v_0 + sum w_n,   x_N - x_0 = dt sum_n (v_n + w_n / 2)
    p = P(d=0.0, h=0.0, F0=0.0, gamma0=0.0, q=0.0, c=0.0, D=0.4)
    dt, N, seed = 1e-2, 257, 11
    r = O.run_set(p, seed=seed, dt=dt, n_traj=3, n_steps=N, v0_mode=1, want_states=True, scheme=1)
    for t in range(3):
        w = np.array([math.sqrt(2 * p["D"] * dt) * O.normal(seed, t, n) for n in range(N)])
        _, v0, _ = O.initial_state(p, seed, 1, t)
        v = v0 + np.concatenate([[0.0], np.cumsum(w)])
        assert r["v"][t] == pytest.approx(v[-1], rel=1e-12, abs=1e-13)
        assert r["x"][t] - r["x0"][t] == pytest.approx(dt * np.sum(v[:-1] + w / 2), rel=1e-10, abs=1e-13)


def test_heun_ou_variance():
    # d = 0, h = 0, F0 = 0: v' = a v + b z with a = 1 - g dt + (g dt)^2/2,
    # b = sqrt(2 D dt)(1 - g dt / 2); from v0 = 0, Var v_N = b^2 (1 - a^{2N}) / (1 - a^2),
    # whose stationary value is D/g (1 + O((g dt)^2)) -- Euler-Maruyama's is off at O(g dt)
    p = P(d=0.0, h=0.0, F0=0.0, D=0.3, gamma0=2.0)
    dt, N, M = 5e-2, 400, 20_000
    g = p["gamma0"]
    r = O.run_set(p, seed=8, dt=dt, n_traj=M, n_steps=N, want_states=True, scheme=1)
    a = 1 - g * dt + 0.5 * (g * dt) ** 2
    b2 = 2 * p["D"] * dt * (1 - 0.5 * g * dt) ** 2
    var_v = b2 * (1 - a ** (2 * N)) / (1 - a**2)
    v2 = np.mean(r["v"] ** 2)
    assert abs(v2 - var_v) < 4 * var_v * math.sqrt(2.0 / M)
    # the closed form itself: within (g dt)^2 of D/g, while EM's D/(g (1 - g dt/2)) is not
    assert abs(var_v / (p["D"] / g) - 1) < (g * dt) ** 2
    assert abs(1 / (1 - g * dt / 2) - 1) > 5 * (g * dt) ** 2


def test_heun_active_motion_fixed_point():
    # D = 0, h = 0, F0 = 0: the active fixed point v* = sqrt(q/g - c/d), e* = g/d has zero
    # drift, so predictor and corrector both return it; x advances by v* dt
    p = P(D=0.0, h=0.0, q=1.3, c=0.2, d=0.8, gamma0=0.9)
    v_star = math.sqrt(p["q"] / p["gamma0"] - p["c"] / p["d"])
    e_star = p["gamma0"] / p["d"]
    (x1, v1, e1), vp = O.heun_step(p, 1e-2, 0.0, (0.4, v_star, e_star))
    assert v1 == pytest.approx(v_star, rel=1e-14) and e1 == pytest.approx(e_star, rel=1e-14)
    assert vp == pytest.approx(v_star, rel=1e-14)
    assert x1 == pytest.approx(0.4 + v_star * 1e-2, rel=1e-14)


def _integrate(step, p, dt, T, s0):
    s = s0
    for _ in range(int(round(T / dt))):
        s = step(p, dt, s)
    return np.array(s)


def test_heun_is_second_order_on_the_deterministic_model():
    # D = 0, the full model (ratchet force, depot, external force): global error at t = 1
    # against a fine Heun run shrinks 4x per halving of dt (EM: 2x)
    p = P(D=0.0, F0=0.2, asym=0.3)
    s0, T = (0.13, 0.4, 0.2), 1.0
    heun = lambda p, dt, s: O.heun_step(p, dt, 0.0, s)[0]
    em = lambda p, dt, s: O.em_step(p, dt, 0.0, s)
    ref = _integrate(heun, p, 6.25e-5, T, s0)
    err_h = [np.abs(_integrate(heun, p, dt, T, s0) - ref).max() for dt in (0.01, 0.005, 0.0025)]
    err_e = [np.abs(_integrate(em, p, dt, T, s0) - ref).max() for dt in (0.01, 0.005, 0.0025)]
    for a, b in zip(err_h, err_h[1:]):
        assert 3.6 < a / b < 4.4, err_h
    for a, b in zip(err_e, err_e[1:]):
        assert 1.5 < a / b < 2.5, err_e


def test_heun_time_average_is_displacement():
    # the time average of the scheme's velocity (v_n + v~_n)/2 equals (x_N - x_0)/(N dt)
    r = O.run_set(P(D=0.3), seed=7, dt=1e-2, n_traj=64, n_steps=500, v0_mode=1, want_states=True, scheme=1)
    np.testing.assert_allclose(r["vbar"] * 500 * 1e-2, r["x"] - r["x0"], rtol=1e-9, atol=1e-12)


def test_heun_rejects_gradient_and_unknown_scheme():
    with pytest.raises(ValueError):
        O.run_set(P(), seed=1, dt=1e-3, n_traj=2, n_steps=10, want_grad=True, scheme=1)
    with pytest.raises(ValueError):
        O.run_set(P(), seed=1, dt=1e-3, n_traj=2, n_steps=10, scheme=2)
