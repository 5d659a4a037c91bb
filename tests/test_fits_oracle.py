"""Pins of the fit oracle (Methods, "Fitting process and Euclidean correlation
length estimation") against values fixed outside it: exact model data, the
transfer-matrix gaps of Eq. (Trotter-transfer-matrix), and the statistics of
fits to data with known Gaussian noise."""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import fits
from tests import exact


def _two_replicas(mean, sigma):
    """Two replicas whose mean is `mean` and whose standard error is `sigma`."""
    return np.stack([mean + sigma, mean - sigma])


def test_tau_tilde_is_tau_at_short_lags_and_lt_over_pi_at_the_middle():
    Lt = 256
    tt = fits.tau_tilde(Lt)
    tau = np.arange(Lt // 2 + 1)
    assert tt[0] == 0.0 and abs(tt[-1] - Lt / math.pi) < 1e-12
    # sin x >= x - x^3/6: tau - tilde tau <= pi^2 tau^3 / (6 L_tau^2)
    assert np.all(tau - tt >= -1e-12)
    assert np.all(tau - tt <= math.pi ** 2 * tau ** 3 / (6 * Lt ** 2) + 1e-12)
    assert np.all(np.diff(tt) > 0)


def test_replica_error_is_the_standard_error_of_the_mean():
    rng = np.random.default_rng(1)
    reps = rng.normal(size=(6, 50))
    m, se = fits.replica_stats(reps)
    assert np.allclose(m, reps.mean(0))
    assert np.allclose(se, reps.std(0, ddof=1) / math.sqrt(6))


@pytest.mark.parametrize("zeta", [1.0, -1.0])
def test_c_fit_recovers_exact_model_parameters(zeta):
    Lt, B, eta = 64, 0.7, 3.3
    tau = np.arange(Lt // 2 + 1)
    C = B * (np.exp(-tau / eta) + zeta * np.exp(-(Lt - tau) / eta))
    s = np.full_like(C, 1e-4)
    s[0] = 0.0
    r = fits.fit_C(*fits.replica_stats(_two_replicas(C, s)), Lt, zeta)
    # window: the first lag where C <= 3.5 sigma
    assert 1 < r["tau_w"] < Lt // 2
    assert r["tau_w"] == int(np.argmax((C <= 3.5e-4) & (tau >= 1)))
    assert r["ok"] and r["tau_min"] == max(1, r["tau_w"] // 10)
    assert abs(r["eta"] - eta) < 1e-8 and abs(r["B"] - B) < 1e-8


def test_c_never_below_window_is_not_estimated():
    Lt = 32
    tau = np.arange(Lt // 2 + 1)
    C = 0.5 * (np.exp(-tau / 200.0) + np.exp(-(Lt - tau) / 200.0))
    s = np.full_like(C, 1e-3)
    r = fits.fit_C(C, s, Lt, 1.0)
    assert not r["ok"] and r["tau_w"] == Lt // 2


def test_q2_fit_recovers_two_exponentials_and_plateau():
    Lt = 128
    tau = np.arange(Lt // 2 + 1).astype(float)
    Q = 0.3 + 0.4 * np.exp(-tau / 2.0) + 0.3 * np.exp(-tau / 0.7)
    s = np.full_like(Q, 1e-6)
    s[0] = 0.0
    r = fits.fit_Q2(*fits.replica_stats(_two_replicas(Q, s)), Lt)
    assert r["plateau_ok"] and abs(r["Q_pl"] - 0.3) < 1e-8
    assert r["ok"] and r["n_exp"] == 2
    assert abs(r["eta_e"] - 2.0) < 1e-4 and abs(r["eta_2"] - 0.7) < 1e-4


def test_q2_fit_frees_the_plateau_when_the_constant_fit_fails():
    """A plateau region that still decays: chi2/dof of the constant is large,
    the window becomes L_tau/2 and Q_pl is fitted with the exponentials."""
    Lt = 64
    tau = np.arange(Lt // 2 + 1).astype(float)
    Q = 0.2 + 0.5 * np.exp(-tau / 12.0)
    s = np.full_like(Q, 1e-6)
    s[0] = 0.0
    r = fits.fit_Q2(*fits.replica_stats(_two_replicas(Q, s)), Lt)
    assert not r["plateau_ok"] and r["tau_w"] == Lt // 2
    assert r["ok"] and abs(r["Q_pl"] - 0.2) < 1e-6 and abs(r["eta_e"] - 12.0) < 1e-4


def test_fits_of_exact_transfer_matrix_correlators_give_the_two_gaps():
    """C decays with the odd gap and Q2 - plateau with the even gap: eta =
    1 / ln(lambda_0 / lambda_odd), eta_e = 1 / ln(lambda_0 / lambda_even) of the
    2x2 transfer matrix, Eq. (Trotter-transfer-matrix) and Fig. (spectrum)."""
    r = np.random.default_rng(21)
    J = (1 - 2 * r.integers(0, 2, size=(2, 2, 2))).astype(np.int8)
    k, Lt = 0.4, 128
    T, _ = exact.transfer_matrix(J, 2, k)
    w, V = np.linalg.eigh(T)
    o = np.argsort(w)[::-1]
    w, V = w[o], V[:, o]
    dim = 16
    P = np.zeros((dim, dim))
    P[np.arange(dim), (dim - 1) ^ np.arange(dim)] = 1.0
    par = [float(V[:, i] @ P @ V[:, i]) for i in range(dim)]
    eta_odd = 1 / math.log(w[0] / w[next(i for i in range(1, dim) if par[i] < 0)])
    eta_even = 1 / math.log(w[0] / w[next(i for i in range(1, dim) if par[i] > 0)])
    C, Q, _ = exact.transfer_correlators(J, 2, Lt, k)
    sc = np.maximum(1e-6 * np.abs(C), 1e-9)
    sq = np.maximum(1e-6 * np.abs(Q - Q[-1]), 1e-9)
    sc[0] = sq[0] = 0.0
    res = fits.fit_sample(_two_replicas(C, sc), _two_replicas(Q, sq), Lt)
    assert res["C"]["ok"] and abs(res["C"]["eta"] / eta_odd - 1) < 1e-3
    assert res["Q2"]["ok"] and abs(res["Q2"]["eta_e"] / eta_even - 1) < 1e-3


def test_c_fit_under_known_noise_is_centred_and_its_errors_match_the_spread():
    """Gaussian noise of known sigma on the model: over independent draws the
    median eta is the true one and the quoted errors match the observed
    spread (within a factor that allows for the noise-dependent window)."""
    Lt, B, eta, sig = 64, 0.8, 4.0, 2e-3
    tau = np.arange(Lt // 2 + 1)
    C = B * (np.exp(-tau / eta) + np.exp(-(Lt - tau) / eta))
    rng = np.random.default_rng(7)
    etas, errs = [], []
    for _ in range(300):
        Cn = C + rng.normal(scale=sig, size=C.shape)
        Cn[0] = 1.0
        s = np.full_like(C, sig)
        s[0] = 0.0
        r = fits.fit_C(Cn, s, Lt, 1.0)
        if r["ok"]:
            etas.append(r["eta"])
            errs.append(r["eta_err"])
    etas, errs = np.array(etas), np.array(errs)
    assert len(etas) > 230
    assert abs(np.median(etas) / eta - 1) < 0.02
    spread = 1.4826 * np.median(np.abs(etas - np.median(etas)))  # robust standard deviation
    ratio = spread / np.median(errs)
    assert 0.7 < ratio < 2.5, ratio
