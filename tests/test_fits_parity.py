"""The library's correlation-length fits (qsg_fit_correlators, host FP64)
against the fit oracle on seeded synthetic replica correlators: identical
windows, lags and model choices, fitted values to 1e-6 relative (the same
Levenberg-Marquardt iteration written twice, stopping at the same minimum),
parameter errors to 1e-4.  Where a Q2 fit is ill-conditioned (a parameter not
determined to a quarter of its size) its end point is not unique and the two
sides may accept different tau_min; there the library's result is checked
for validity instead (its chi2/dof below the threshold, a decay length in
(0, L_tau])."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import fits as ofits
from paper_2310_07486_gb300 import qsg as Q

pytestmark = pytest.mark.gpu  # calls into the compiled library

RTOL = 1e-6
# Parameter errors come from (J^T W J)^-1; for two-exponential fits its
# condition number reaches 1e10 and more, so the two sides' different
# summation orders (1e-16 relative in J^T W J) show up at up to ~1e-5 there.
RTOL_ERR = 1e-4
INT_FIELDS = ("C_ok", "C_tau_w", "C_tau_min", "Q_ok", "Q_tau_w", "Q_tau_min", "Q_n_exp", "plateau_ok")


def _synthetic(rng, R, n, Ltau, zeta):
    """Per-replica correlators of n series.  As in Monte Carlo data, the
    replica fluctuations are correlated along tau: every replica has its own
    amplitudes and decay lengths (a few per cent off the series' values), plus
    a small white noise.  C: one decaying pair; Q2: plateau + two exponentials."""
    nl = Ltau // 2 + 1
    tau = np.arange(nl, dtype=float)
    C = np.zeros((R, n, nl))
    Q2 = np.zeros((R, n, nl))
    for i in range(n):
        eta, B = rng.uniform(1.0, Ltau / 6), rng.uniform(0.3, 0.9)
        qpl, b1 = rng.uniform(0.05, 0.6), rng.uniform(0.1, 0.4)
        e1 = rng.uniform(0.8, Ltau / 10)
        e2 = e1 * rng.uniform(0.2, 0.5)
        spread = 10 ** rng.uniform(-2.5, -1.5)
        white = 10 ** rng.uniform(-6, -4)
        for r in range(R):
            d = 1 + spread * rng.normal(size=6)
            C[r, i] = B * d[0] * (np.exp(-tau / (eta * d[1])) + zeta * np.exp(-(Ltau - tau) / (eta * d[1])))
            Q2[r, i] = (qpl * d[2] + b1 * d[3] * np.exp(-tau / (e1 * d[4]))
                        + (1 - qpl - b1) * np.exp(-tau / (e2 * d[5])))
            C[r, i] += rng.normal(scale=white, size=nl)
            Q2[r, i] += rng.normal(scale=white, size=nl)
        C[:, i, 0] = 1.0
        Q2[:, i, 0] = 1.0
    return C, Q2


def _ill_conditioned(lib_res, q):
    """A Q2 fit whose parameters are not determined to better than a quarter of
    their size (a five-parameter fit on a few lags, a free plateau): its end
    point is not unique, so rounding differences between platforms may move
    the first accepted tau_min."""
    rel = []
    for v, e in ((q["Q_pl"], q["Q_pl_err"]), (q["eta_e"], q["eta_e_err"]),
                 (lib_res["Q_pl"], lib_res["Q_pl_err"]), (lib_res["eta_e"], lib_res["eta_e_err"])):
        if np.isfinite(v) and np.isfinite(e) and v != 0:
            rel.append(abs(e / v))
    return bool(rel) and max(rel) > 0.25


def _compare(lib_res, orc_res, Ltau=None):
    c, q = orc_res["C"], orc_res["Q2"]
    want = dict(C_ok=int(c["ok"]), C_tau_w=c["tau_w"], C_tau_min=c["tau_min"], Q_ok=int(q["ok"]),
                Q_tau_w=q["tau_w"], Q_tau_min=q["tau_min"], Q_n_exp=q["n_exp"], plateau_ok=int(q["plateau_ok"]))
    q_unique = True
    if (lib_res["Q_tau_min"], lib_res["Q_n_exp"], lib_res["Q_ok"]) != (q["tau_min"], q["n_exp"], int(q["ok"])) \
            and _ill_conditioned(lib_res, q):
        # several outcomes are correct: the library's must be a valid one
        q_unique = False
        if lib_res["Q_ok"]:
            assert lib_res["Q_chi2dof"] < 0.5 and 1 <= lib_res["Q_tau_min"] <= lib_res["Q_tau_w"]
            assert 0 < lib_res["eta_e"] and (Ltau is None or lib_res["eta_e"] <= Ltau)
    for f in INT_FIELDS:
        if not q_unique and f in ("Q_ok", "Q_tau_min", "Q_n_exp"):
            continue
        assert lib_res[f] == want[f], (f, lib_res[f], want[f])
    pairs = [("plateau_chi2dof", q["plateau_chi2dof"])]
    if q["plateau_ok"] or q_unique:
        pairs += [("Q_pl", q["Q_pl"]), ("Q_pl_err", q["Q_pl_err"])]
    if c["ok"]:
        pairs += [("eta", c["eta"]), ("eta_err", c["eta_err"]), ("C_amp", c["B"]), ("C_chi2dof", c["chi2dof"])]
    if q["ok"] and q_unique:
        pairs += [("eta_e", q["eta_e"]), ("eta_e_err", q["eta_e_err"]), ("Q_chi2dof", q["chi2dof"])]
        if q["n_exp"] == 2:
            pairs += [("eta_2", q["eta_2"])]
    for f, v in pairs:
        tol = RTOL_ERR if f.endswith("_err") else RTOL
        assert abs(lib_res[f] - v) <= tol * max(abs(v), 1e-300), (f, lib_res[f], v)
    return q_unique


@pytest.mark.parametrize("R,n,Ltau,boundary", [(2, 12, 64, Q.PBC), (4, 16, 128, Q.PBC), (6, 10, 32, Q.APBC),
                                               (3, 8, 256, Q.APBC)])
def test_library_fits_match_oracle(R, n, Ltau, boundary):
    rng = np.random.default_rng(1000 * R + Ltau)
    zeta = -1.0 if boundary == Q.APBC else 1.0
    C, Q2 = _synthetic(rng, R, n, Ltau, zeta)
    lib = Q.qsg_fit_correlators(C, Q2, Ltau, boundary)
    n_ok = n_unique = 0
    for i in range(n):
        orc = ofits.fit_sample(C[:, i], Q2[:, i], Ltau, boundary)
        n_unique += _compare(lib[i], orc, Ltau)
        n_ok += lib[i]["C_ok"] + lib[i]["Q_ok"]
    assert n_ok >= n  # the cases exercise accepted fits, not only rejections
    assert n_unique >= n - 2


def test_tau_tilde_matches_oracle():
    for Lt in (4, 32, 2048):
        assert np.allclose(Q.qsg_tau_tilde(Lt), ofits.tau_tilde(Lt), rtol=1e-15, atol=1e-13)


def test_fit_rejects_bad_arguments():
    C = np.zeros((1, 1, 17))
    with pytest.raises(Q.QSGError):
        Q.qsg_fit_correlators(C, C, 32)  # one replica: no error bars


def test_fits_of_gpu_correlators_match_oracle():
    """End to end: correlators of a short GPU run, fitted by the library and
    by the oracle, series by series."""
    pytest.importorskip("torch")
    shape = Q.Shape(6, 32, 64, 4, 2, Q.HEATBATH, Q.PBC)
    ctx = Q.Context([shape])
    ctx.qsg_init_samples(77, [np.array([0.3, 0.45])])
    ctx.qsg_sweep(50)
    for _ in range(60):
        ctx.qsg_sweep(2)
        ctx.qsg_tempering_swap()
        ctx.qsg_measure_correlators()
    res = ctx.qsg_read_correlators()
    nl = shape.n_lag
    C = res["C"].reshape(shape.n_replicas, -1, nl)
    Q2 = res["Q2"].reshape(shape.n_replicas, -1, nl)
    lib = Q.qsg_fit_correlators(C, Q2, shape.Ltau, shape.boundary)
    assert len(lib) == shape.n_samples * shape.n_k
    n_unique = 0
    for i in range(len(lib)):
        n_unique += _compare(lib[i], ofits.fit_sample(C[:, i], Q2[:, i], shape.Ltau, shape.boundary), shape.Ltau)
    assert sum(r["Q_ok"] for r in lib) > 0
    assert n_unique >= 0.8 * len(lib)
