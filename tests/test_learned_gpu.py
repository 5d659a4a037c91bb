"""Learned-ladder kernels through the C ABI against the oracle: coupling
features bit for bit, per-pair overlap sums bit for bit, the judge (identical
decisions), and the MLP element by element within rounding bounds derived
from the arithmetic (oracle/learned.py): the FP32 loss and gradient within
the first-order forward error bounds of FP32 dot products and their
propagation, each Adam step within the bound of its FP32 operations (given the
same gradient), FP32 inference within its forward bound, and BF16 inference
inside the interval of every value the BF16 roundings can give."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import learned as OL
from paper_2310_07486_gb300 import qsg as Q

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, size=(n, 64)).astype(np.float32)
    T = np.zeros((n, 33), dtype=np.float32)
    T[:, :32] = rng.dirichlet(np.ones(32), size=n)
    T[:, 32] = rng.uniform(0.4, 0.9, size=n)
    return X, T


@pytest.mark.parametrize("L,ns", [(4, 70), (6, 64), (8, 130), (12, 5), (24, 64), (2, 3)])
def test_features_match_oracle(L, ns):
    shape = Q.Shape(L, 8, ns, 1, 1)
    ctx = Q.Context([shape])
    ctx.qsg_init_samples(17 + L, [np.array([0.3])])
    F = ctx.qsg_sample_features()
    orc = oracle.OracleGroup(L, 8, ns, 1, 1)
    orc.init(17 + L, np.array([0.3]))
    J = orc.couplings()  # the same couplings, drawn from the same seed
    for b in range(ns):
        assert np.array_equal(F[b], OL.features(J[b])), b


def test_pair_overlap_sums_match_oracle():
    shape = Q.Shape(6, 16, 70, 4, 2, Q.HEATBATH, Q.PBC)
    ctx = Q.Context([shape])
    ctx.qsg_init_samples(5, [np.array([0.3, 0.4])])
    orc = oracle.OracleGroup(6, 16, 70, 4, 2, algo="heatbath")
    orc.init(5, np.array([0.3, 0.4]))
    for _ in range(3):
        ctx.qsg_sweep(2)
        orc.sweep(2)
        ctx.qsg_measure_correlators()
        orc.measure()
    pp = ctx.qsg_read_pair_overlaps()
    assert np.array_equal(pp, orc.read_pair_overlaps())
    assert np.array_equal(pp.sum(axis=2), ctx.qsg_read_onetime()["raw"][:, :, 0])


@pytest.mark.parametrize("batch", [1, 16, 37, 256])
def test_mlp_loss_and_gradient_match_oracle(batch):
    X, T = _data(300, batch)
    theta = OL.init_params(11)
    m = Q.MLP(300, 256)
    m.set_params(theta)
    m.set_data(X, T)
    idx = np.random.default_rng(batch).choice(300, size=batch, replace=False).astype(np.int32)
    loss, g = m.grad(idx)
    th = theta.astype(np.float64)
    lref, gref = OL.loss_and_grad(th, X[idx], T[idx])
    lb, gb = OL.grad_error_bound(th, X[idx], T[idx])
    assert abs(loss - lref) <= lb
    bad = np.abs(g.astype(np.float64) - gref) > gb
    assert not bad.any(), (int(bad.sum()), np.flatnonzero(bad)[:10])


def test_mlp_adam_steps_match_oracle():
    X, T = _data(128, 3)
    theta = OL.init_params(5)
    m = Q.MLP(128, 64)
    m.set_params(theta)
    m.set_data(X, T)
    rng = np.random.default_rng(9)
    idx = np.stack([rng.choice(128, size=64, replace=False) for _ in range(3)]).astype(np.int32)
    # each step: the library's gradient at its own parameters (training is
    # deterministic, so the step below uses this very gradient), then one Adam
    # step; the oracle applies Adam in FP64 to the same parameters and gradient
    # and bounds the FP32 step's rounding, with the moments' errors carried on
    mo = vo = em = ev = np.zeros(OL.N_PARAMS)
    for t in range(1, 4):
        th = m.get_params().astype(np.float64)
        loss, g = m.grad(idx[t - 1])
        lref, gref = OL.loss_and_grad(th, X[idx[t - 1]], T[idx[t - 1]])
        lb, gb = OL.grad_error_bound(th, X[idx[t - 1]], T[idx[t - 1]])
        assert np.all(np.abs(g.astype(np.float64) - gref) <= gb)
        losses = m.train(idx[t - 1:t], lr=1e-3)
        assert abs(losses[0] - lref) <= lb
        want, mo, vo, em, ev, eth = OL.adam_step_bound(th, mo, vo, em, ev, g.astype(np.float64), t, 1e-3)
        got = m.get_params().astype(np.float64)
        bad = np.abs(got - want) > eth
        assert not bad.any(), (t, int(bad.sum()))


def test_mlp_training_reduces_the_loss():
    X, T = _data(512, 4)
    m = Q.MLP(512, 128)
    m.set_params(OL.init_params(6))
    m.set_data(X, T)
    rng = np.random.default_rng(1)
    idx = np.stack([rng.permutation(512)[:128] for _ in range(300)]).astype(np.int32)
    losses = m.train(idx, lr=3e-3)
    assert losses[-20:].mean() < 0.9 * losses[:20].mean()


@pytest.mark.parametrize("bf16", [False, True])
def test_mlp_inference_matches_oracle(bf16):
    X, _ = _data(200, 8)
    theta = OL.init_params(12)
    m = Q.MLP(200, 16)
    m.set_params(theta)
    Y = m.predict(X, bf16=bf16).astype(np.float64)
    th = theta.astype(np.float64)
    if bf16:
        lo, hi = OL.forward_bf16_interval(th, X)
        assert np.all((Y >= lo) & (Y <= hi))
    else:
        ref, e, _ = OL.fp32_forward_bound(th, X)
        assert np.all(np.abs(Y - ref) <= e)


def test_judge_matches_oracle():
    rng = np.random.default_rng(3)
    nb, ns, R, K, P = 10, 40, 4, 3, 6  # P = R (R - 1) / 2
    drift = (2.0 ** -np.arange(nb))[:, None, None, None] * rng.uniform(0, 0.2, size=(1, ns, 1, K))
    E = -1 - drift + rng.normal(scale=0.01, size=(nb, ns, R, K))
    q = 0.3 + drift[:, :, 0, :][..., None] + rng.normal(scale=0.01, size=(nb, ns, K, P))
    got = Q.qsg_judge(E, q)
    want = OL.judge(E, q)
    assert np.array_equal(got, want)
    assert (got >= 0).sum() > 5 and (got < 0).sum() + (got > 2).sum() > 5
