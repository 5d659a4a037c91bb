"""Pins of the learned-ladder oracle (features, MLP gradients, Adam, BF16
rounding, the log-binning judge) against closed forms, symmetries, finite
differences and an independent BF16 conversion."""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import learned as OL

FRUSTRATION_FEATURES = [0] + list(range(6, 34)) + list(range(36, 64))


def _random_J(L, seed):
    rng = np.random.default_rng(seed)
    return (1 - 2 * rng.integers(0, 2, size=(2, L, L))).astype(np.int8)


def test_features_of_the_ferromagnet():
    L = 8
    f = OL.features(np.ones((2, L, L), dtype=np.int8))
    want = np.zeros(64)
    want[5] = 1      # every site has bond sum +4
    want[6] = 1      # no frustrated plaquette around any site
    want[11] = 1     # every 2x2 block has none
    want[36] = want[42] = 1  # every row / column in the lowest bin
    assert np.array_equal(f, want.astype(np.float32))


def test_one_negative_bond_frustrates_its_two_plaquettes():
    L = 6
    J = np.ones((2, L, L), dtype=np.int8)
    J[0, 2, 3] = -1  # bond (3,2)-(4,2): plaquettes (3,1) and (3,2)
    F = OL.frustration(J)
    assert F.sum() == 2 and F[1, 3] == 1 and F[2, 3] == 1
    f = OL.features(J)
    assert f[0] == np.float32(2 / 36)
    assert f[56 + 0] == np.float32(1 / 36)  # the pair at offset (0, 1)
    assert f[34] == np.float32(1 / 36) and f[35] == 0


@pytest.mark.parametrize("L", [4, 8, 12])
def test_frustration_features_are_gauge_invariant(L):
    """Flipping the four bonds of any set of sites (S_x -> -S_x) leaves every
    plaquette product, hence every frustration feature, unchanged."""
    J = _random_J(L, L)
    rng = np.random.default_rng(99)
    G = J.copy()
    for y, x in zip(rng.integers(0, L, 10), rng.integers(0, L, 10)):
        G[0, y, x] *= -1
        G[0, y, (x - 1) % L] *= -1
        G[1, y, x] *= -1
        G[1, (y - 1) % L, x] *= -1
    fa, fb = OL.features(J), OL.features(G)
    assert np.array_equal(fa[FRUSTRATION_FEATURES], fb[FRUSTRATION_FEATURES])
    assert not np.array_equal(fa, fb)  # the bond-sign features do see the gauge


def test_translation_leaves_the_unaligned_features_unchanged():
    L = 8
    J = _random_J(L, 5)
    S = np.roll(np.roll(J, 3, axis=2), 1, axis=1)  # odd shift: block alignment changes too
    fa, fb = OL.features(J), OL.features(S)
    keep = [i for i in range(64) if not (11 <= i <= 31)]
    assert np.allclose(fa[keep], fb[keep], rtol=0, atol=1e-7)


def test_frustrated_fraction_of_random_couplings_is_one_half():
    fs = [OL.features(_random_J(16, s))[0] for s in range(40)]
    assert abs(np.mean(fs) - 0.5) < 4 * 0.5 / math.sqrt(40 * 256)


def test_mlp_gradient_matches_finite_differences():
    theta = OL.init_params(3).astype(np.float64)
    rng = np.random.default_rng(4)
    X = rng.uniform(0, 1, size=(7, 64))
    T = np.zeros((7, 33))
    T[:, :32] = rng.dirichlet(np.ones(32), size=7)
    T[:, 32] = rng.uniform(0.4, 0.9, size=7)
    _, g = OL.loss_and_grad(theta, X, T)
    idx = rng.choice(OL.N_PARAMS, size=60, replace=False)
    for i in idx:
        h = 1e-6
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (OL.loss_and_grad(tp, X, T)[0] - OL.loss_and_grad(tm, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_loss_at_zero_output_is_log32_plus_budget_square():
    theta = np.zeros(OL.N_PARAMS)
    T = np.zeros((3, 33))
    T[:, :32] = 1 / 32
    T[:, 32] = 0.5
    loss, _ = OL.loss_and_grad(theta, np.ones((3, 64)), T)
    assert abs(loss - (math.log(32) + 0.25)) < 1e-12


def test_first_adam_step_is_lr_times_sign():
    g = np.array([3.0, -1e-3, 0.5])
    th, m, v = OL.adam(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, lr=0.01)
    assert np.allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    a = np.concatenate([rng.normal(scale=10 ** rng.uniform(-5, 5), size=2000).astype(np.float32),
                        np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -0.0, 65504.0], dtype=np.float32)])
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(OL.to_bf16(a), ref)


def test_judge_on_a_geometric_drift():
    """Bin means E_m = -1 - 0.5 * 2^-m at every k with replica standard error
    0.01 (and a flat q^2): the first bin m with 0.5 (2^-(m-2) - 2^-m) <=
    2 sqrt(2) * 0.01 passes (two combined standard errors)."""
    nb, R, K = 12, 4, 2
    P = R * (R - 1) // 2
    E = np.zeros((nb, 1, R, K))
    q = np.full((nb, 1, K, P), 0.3)
    spread = 0.01 * math.sqrt(R - 1)  # so that the standard error over replicas is 0.01
    dev = np.array([-1, 1, -1, 1]) * spread
    for m in range(nb):
        E[m, 0, :, :] = (-1 - 0.5 * 2.0 ** -m) + dev[:, None]
    want = next(m for m in range(2, nb) if 0.5 * (2.0 ** -(m - 2) - 2.0 ** -m) <= 2 * math.sqrt(2) * 0.01)
    assert OL.judge(E, q)[0] == want


def test_judge_jackknife_error_of_q2_over_replicas():
    """q^2 of pair (a, b) = u_a + u_b: leaving replica r out, the pair mean
    moves by a known amount; the jackknife error of the mean over pairs is
    then sqrt((R-1)/R sum_r (J_r - mean J)^2) with J_r the mean over pairs
    without r.  A drift of the q^2 mean by exactly 2.001 of those combined
    errors fails, 1.999 passes."""
    R, K = 4, 1
    u = np.array([0.0, 0.01, 0.03, 0.02])
    pairs = [(a, b) for a in range(R) for b in range(a + 1, R)]
    base = np.array([u[a] + u[b] for a, b in pairs])
    Jr = np.array([np.mean([base[i] for i, (a, b) in enumerate(pairs) if r not in (a, b)]) for r in range(R)])
    se = math.sqrt((R - 1) / R * ((Jr - Jr.mean()) ** 2).sum())
    for factor, want in ((1.999, 2), (2.001, 3)):
        step = factor * math.sqrt(2) * se
        nb = 4
        E = np.zeros((nb, 1, R, K)) + np.array([-1, 1, -1, 1])[None, None, :, None] * 1e-3
        q = np.zeros((nb, 1, K, len(pairs)))
        q[0, 0, 0] = base
        q[1, 0, 0] = base + step        # bins 1, 2, 3 agree; bin 0 is one step below
        q[2, 0, 0] = base + step
        q[3, 0, 0] = base + step
        assert OL.judge(E, q)[0] == want, factor


def test_judge_never_passes_a_steady_trend():
    nb, R, K = 10, 4, 1
    P = R * (R - 1) // 2
    E = np.zeros((nb, 1, R, K))
    for m in range(nb):
        E[m] = -m + np.array([-1, 1, -1, 1])[:, None] * 0.01
    q = np.full((nb, 1, K, P), 0.2) + np.linspace(-1e-3, 1e-3, P)
    assert OL.judge(E, q)[0] == -1
