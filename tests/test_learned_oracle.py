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


# ---------------------------------------------------------------------------
# the element-wise rounding bounds, pinned against an independent
# single-precision implementation (numpy float32: BLAS summation order, not
# the library's), which must fall inside them
# ---------------------------------------------------------------------------
def _f32_forward(theta, X, bf16=False):
    W1, b1, W2, b2, W3, b3 = [p.astype(np.float32) for p in OL.unpack(theta)]
    if bf16:
        W1, b1, W2, b2, W3, b3 = [OL.to_bf16(p).astype(np.float32) for p in (W1, b1, W2, b2, W3, b3)]
    r = (lambda a: OL.to_bf16(a).astype(np.float32)) if bf16 else (lambda a: a)
    h = r(np.asarray(X, dtype=np.float32))
    z1 = h @ W1.T + b1
    h1 = r(np.maximum(z1, 0))
    z2 = h1 @ W2.T + b2
    h2 = r(np.maximum(z2, 0))
    return (h2 @ W3.T + b3).astype(np.float64), (z1, h1, z2, h2)


def _f32_loss_and_grad(theta, X, T):
    W1, b1, W2, b2, W3, b3 = [p.astype(np.float32) for p in OL.unpack(theta)]
    X = np.asarray(X, dtype=np.float32)
    T = np.asarray(T, dtype=np.float32)
    B = np.float32(T.shape[0])
    y, (z1, h1, z2, h2) = _f32_forward(theta, X)
    y = y.astype(np.float32)
    a = y[:, :32] - y[:, :32].max(axis=1, keepdims=True)
    logp = a - np.log(np.exp(a).sum(axis=1, keepdims=True))
    r = y[:, 32] - T[:, 32]
    loss = ((-(T[:, :32] * logp).sum(axis=1) + r * r).sum() / B)
    dy = np.zeros_like(y)
    dy[:, :32] = (np.exp(logp) * T[:, :32].sum(axis=1, keepdims=True) - T[:, :32]) / B
    dy[:, 32] = 2 * r / B
    dz2 = (dy @ W3) * (z2 > 0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    g = OL.pack([dz1.T @ X, dz1.sum(0), dz2.T @ h1, dz2.sum(0), dy.T @ h2, dy.sum(0)])
    return float(loss), g


def _mlp_case(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, size=(n, 64)).astype(np.float32)
    T = np.zeros((n, 33), dtype=np.float32)
    T[:, :32] = rng.dirichlet(np.ones(32), size=n)
    T[:, 32] = rng.uniform(0.4, 0.9, size=n)
    return OL.init_params(seed).astype(np.float64), X, T


@pytest.mark.parametrize("n,seed", [(1, 1), (37, 2), (256, 3)])
def test_fp32_gradient_and_forward_fall_inside_the_rounding_bounds(n, seed):
    theta, X, T = _mlp_case(n, seed)
    lref, gref = OL.loss_and_grad(theta, X, T)
    lb, gb = OL.grad_error_bound(theta, X, T)
    l32, g32 = _f32_loss_and_grad(theta, X, T)
    assert abs(l32 - lref) <= lb
    assert np.all(np.abs(g32 - gref) <= gb)
    y, ey, _ = OL.fp32_forward_bound(theta, X)
    y32, _ = _f32_forward(theta, X)
    assert np.all(np.abs(y32 - y) <= ey)
    # not vacuous: the largest elements are pinned to within their own size
    # (worst-case bounds loosen with cancellation in long batch sums, so the
    # fraction is larger for B = 256)
    top = np.argsort(-np.abs(gref))[:100]
    assert np.max(gb[top] / np.abs(gref[top])) < 1.0  # sign and magnitude pinned


def test_gradient_bound_catches_a_wrong_element():
    theta, X, T = _mlp_case(37, 4)
    lref, gref = OL.loss_and_grad(theta, X, T)
    _, gb = OL.grad_error_bound(theta, X, T)
    k = int(np.argmax(np.abs(gref)))
    bad = gref.copy()
    bad[k] *= 1.05  # one element off by 5 %: outside its bound
    assert not np.all(np.abs(bad - gref) <= gb)
    bad = gref.copy()
    bad[-1] = -bad[-1]  # a sign error in one bias gradient
    assert not np.all(np.abs(bad - gref) <= gb)


@pytest.mark.parametrize("seed", [5, 6])
def test_bf16_inference_falls_inside_its_interval(seed):
    theta, X, _ = _mlp_case(200, seed)
    lo, hi = OL.forward_bf16_interval(theta, X)
    y64 = OL.forward_bf16(theta, X)
    y32, _ = _f32_forward(theta, X, bf16=True)
    assert np.all((y64 >= lo) & (y64 <= hi))
    assert np.all((y32 >= lo) & (y32 <= hi))
    # one BF16 step (2^-8 relative) of the output scale bounds the width
    assert np.median(hi - lo) < 2.0 ** -8 * np.abs(y64).max()


def test_fp32_adam_falls_inside_its_bound():
    theta, X, T = _mlp_case(64, 7)
    th32 = theta.astype(np.float32)
    m32 = np.zeros_like(th32)
    v32 = np.zeros_like(th32)
    m = v = em = ev = np.zeros_like(theta)
    lr = 1e-3
    for t in range(1, 4):
        _, g = OL.loss_and_grad(th32.astype(np.float64), X, T)
        g32 = g.astype(np.float32)
        th1, m, v, em, ev, eth = OL.adam_step_bound(th32.astype(np.float64), m, v, em, ev, g32.astype(np.float64), t,
                                                    lr)
        b1, b2 = np.float32(0.9), np.float32(0.999)
        m32 = b1 * m32 + np.float32(0.1) * g32
        v32 = b2 * v32 + np.float32(0.001) * g32 * g32
        c1, c2 = np.float32(1 - 0.9 ** t), np.float32(1 - 0.999 ** t)
        th32 = th32 - np.float32(lr) * (m32 / c1) / (np.sqrt(v32 / c2) + np.float32(1e-8))
        assert np.all(np.abs(th32.astype(np.float64) - th1) <= eth), t
