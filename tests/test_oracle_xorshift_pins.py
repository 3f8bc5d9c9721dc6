"""Pins of the oracle's xorshift noise option (Marsaglia's generator of Fig. 1) against facts
fixed outside it.

The generator is a linear map T of the 128-bit state over GF(2).  The published shift triple
(11, 8, 19) makes T's order exactly 2^128 - 1 (the full period of the 2003 paper); a wrong
shift, direction or word order almost surely breaks that, and a wrong output word or
non-linear step breaks the linearity checks.  The seeding must equal the Philox block of the
documented counter, and the normals drawn from the stream (two words, Box-Muller cosine)
must be standard normal, also through the model's free velocity.
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O

# 2^128 - 1 = (2^64 - 1)(2^64 + 1), with 2^64 + 1 = 274177 * 67280421310721
FACTORS_2_128_M1 = (3, 5, 17, 257, 641, 65537, 6700417, 274177, 67280421310721)


def state_bits(s):
    return np.array([(int(s[i // 32]) >> (i % 32)) & 1 for i in range(128)], dtype=np.float64)


def bits_state(b):
    out = [0, 0, 0, 0]
    for i in range(128):
        if int(b[i]) & 1:
            out[i // 32] |= 1 << (i % 32)
    return tuple(out)


def transition_matrix():
    cols = []
    for i in range(128):
        e = [0, 0, 0, 0]
        e[i // 32] = 1 << (i % 32)
        _, s = O.xorshift_step(e)
        cols.append(state_bits(s))
    return np.stack(cols, axis=1)


def mat_mul(a, b):
    return np.mod(a @ b, 2.0)


def mat_pow(a, e):
    r = np.eye(a.shape[0])
    base = a.copy()
    while e:
        if e & 1:
            r = mat_mul(r, base)
        base = mat_mul(base, base)
        e >>= 1
    return r


def test_xorshift_is_linear_shift_register():
    rng = np.random.default_rng(1)
    for _ in range(50):
        a = tuple(int(v) for v in rng.integers(0, 2**32, 4, dtype=np.uint64))
        b = tuple(int(v) for v in rng.integers(0, 2**32, 4, dtype=np.uint64))
        oa, sa = O.xorshift_step(a)
        ob, sb = O.xorshift_step(b)
        oab, sab = O.xorshift_step(tuple(x ^ y for x, y in zip(a, b)))
        assert sab == tuple(x ^ y for x, y in zip(sa, sb))
        assert oa == sa[3] and oab == oa ^ ob
        assert sa[:3] == a[1:]  # the words move down by one; only w is new


def test_xorshift_has_full_period():
    T = transition_matrix()
    n = 2**128 - 1
    I = np.eye(128)
    assert np.array_equal(mat_pow(T, n), I)
    for p in FACTORS_2_128_M1:
        assert not np.array_equal(mat_pow(T, n // p), I), p
    # the matrix reproduces the step on a random state
    s = (123456789, 362436069, 521288629, 88675123)
    _, s1 = O.xorshift_step(s)
    assert bits_state(mat_mul(T, state_bits(s))) == s1


def test_xorshift_seeding_from_philox():
    for seed, t in [(0, 0), (7, 12345), (2**40 + 3, 2**33 + 9)]:
        assert O.xorshift_seed(seed, t) == O.noise_words(seed, t, 2**63 + 1)
        words = O.xorshift_words(seed, t, 3)
        s = O.xorshift_seed(seed, t)
        for w in words:
            out, s = O.xorshift_step(s)
            assert out == w


def test_xorshift_normals_are_standard_normal():
    p = dict(q=1.0, c=0.0, d=0.0, gamma0=0.0, F0=0.0, D=0.5, h=0.0, L=1.0, asym=0.0)
    # with no drift v_N - v_0 = sqrt(2 D dt) sum of N normals: moments of the normals from v
    dt, N, M = 1.0, 1, 200_000
    r = O.run_set(p, seed=5, dt=dt, n_traj=M, n_steps=N, v0_mode=0, want_states=True, noise=1)
    z = r["v"] / math.sqrt(2 * p["D"] * dt)
    assert abs(z.mean()) < 4 / math.sqrt(M)
    assert abs(z.var() - 1) < 4 * math.sqrt(2 / M)
    assert abs(stats.kurtosis(z)) < 4 * math.sqrt(24 / M)
    edges = np.linspace(-4, 4, 41)
    counts, _ = np.histogram(z, bins=edges)
    expected = M * np.diff(stats.norm.cdf(edges))
    keep = expected > 5
    chi2 = np.sum((counts[keep] - expected[keep]) ** 2 / expected[keep])
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-3


def test_xorshift_free_velocity_variance_and_same_initial_condition():
    # d = 0, h = 0, F0 = 0: the EM closed form of Var v_N holds for any standard normal noise
    p = dict(q=1.0, c=0.1, d=0.0, gamma0=2.0, F0=0.0, D=0.3, h=0.0, L=1.0, asym=0.25)
    dt, N, M = 1e-2, 1500, 20_000
    r = O.run_set(p, seed=8, dt=dt, n_traj=M, n_steps=N, want_states=True, noise=1)
    rho = 1 - p["gamma0"] * dt
    var_v = 2 * p["D"] * dt * (1 - rho ** (2 * N)) / (1 - rho**2)
    assert abs(np.mean(r["v"] ** 2) - var_v) < 4 * var_v * math.sqrt(2.0 / M)
    rp = O.run_set(p, seed=8, dt=dt, n_traj=64, n_steps=10, want_states=True, noise=0)
    np.testing.assert_array_equal(rp["x0"], r["x0"][:64])
    assert not np.array_equal(rp["v"], r["v"][:64])
    with pytest.raises(ValueError):
        O.run_set(p, seed=8, dt=dt, n_traj=2, n_steps=10, want_grad=True, noise=1)


def test_xorshift_step_uses_two_words_and_the_cosine_branch():
    # no drift: v_N = v_0 + sqrt(2 D dt) sum_n z_n exactly, with z_n the Box-Muller cosine of
    # words 2n and 2n+1 of the trajectory's stream (read here from the generator itself)
    p = dict(q=1.0, c=0.0, d=0.0, gamma0=0.0, F0=0.0, D=0.5, h=0.0, L=1.0, asym=0.0)
    dt, N, seed = 0.01, 5, 13
    r = O.run_set(p, seed=seed, dt=dt, n_traj=4, n_steps=N, v0_mode=0, want_states=True, noise=1)
    for t in range(4):
        w = O.xorshift_words(seed, t, 2 * N)
        z = [O.box_muller(w[2 * n], w[2 * n + 1])[0] for n in range(N)]
        assert r["v"][t] == pytest.approx(math.sqrt(2 * p["D"] * dt) * sum(z), rel=1e-12)
