"""Oracle of the per-sample correlation-length fits (Methods, "Fitting process
and Euclidean correlation length estimation") and of the tau-tilde variable
of Sect. "On the magnetic susceptibilities".

TEST INFRASTRUCTURE ONLY: loaded by the tests and nothing else.  It shares no
code with the library's fits (csrc/fits.cpp).

The paper does not name its minimiser; what it defines is the minimum of
chi2 over the model's parameters.  This oracle reaches it with scipy's
trust-region-reflective least squares (scipy.optimize.least_squares,
method "trf"), with every decay length bounded to (0, 10 L_tau] and
tolerances of 1e-15: a different algorithm from the library's, so that the
two agree on the minimum and not on an iteration path.  One-exponential fits
have a single minimum in that box; two-exponential fits can have several, and
there the two sides may end at different ones.

Steps, in the paper's order, for one sample at one k given the correlators of
its R replicas at lags 0 .. L_tau/2:
  1. mean over replicas and its standard error sigma (the replica spread);
  2. plateau: a constant fitted to Q2 on [L_tau/4, L_tau/2] (weights
     1/sigma^2); "acceptable" iff chi2/dof <= PLATEAU_CHI2;
  3. windows: tau_w,f = the first lag tau >= 1 with f(tau) <= 3.5 sigma_f(tau)
     for f = C and f = Q2 - Q_pl; when the plateau fit is not acceptable,
     tau_w,Q2 = L_tau/2 and Q_pl becomes a fit parameter; when C never drops
     to 3.5 sigma the sample's eta exceeds L_tau and is not estimated;
  4. fits with the diagonal covariance: C = B [e^{-tau/eta} + z e^{-(L_tau - tau)/eta}]
     (z = +1 PBC, -1 APBC) on [tau_min, tau_w,C], tau_min starting at
     tau_w,C / 10 and growing until chi2/dof < 1; Q2 = Q_pl + sum_i B_i e^{-tau/eta_i}
     with one and with two terms on [tau_min, tau_w,Q2], tau_min from 1 until
     chi2/dof < 0.5; the one of the two with the smaller chi2/dof is kept and
     eta_e is its largest eta.
Lags with sigma = 0 (tau = 0, where C = Q2 = 1 exactly) carry no weight and
are left out of every fit.  A decay length beyond L_tau cannot be estimated
(the paper says so of samples whose window reaches L_tau/2): the minimiser
keeps every decay length in (0, 10 L_tau], and a fit that ends above L_tau
marks its correlator (or its one- or two-term model) as not estimated.
"""
from __future__ import annotations

import math

import numpy as np

PLATEAU_CHI2 = 2.0
WINDOW_SIGMAS = 3.5
C_CHI2 = 1.0
Q_CHI2 = 0.5


def tau_tilde(Ltau):
    """tilde tau = (L_tau / pi) sin(pi tau / L_tau), tau = 0 .. L_tau/2."""
    tau = np.arange(Ltau // 2 + 1)
    return Ltau / math.pi * np.sin(math.pi * tau / Ltau)


def replica_stats(reps):
    """Mean over replicas (axis 0) and the standard error of that mean."""
    reps = np.asarray(reps, dtype=np.float64)
    R = reps.shape[0]
    m = reps.mean(axis=0)
    se = np.sqrt(((reps - m) ** 2).sum(axis=0) / (R * (R - 1)))
    return m, se


def plateau_fit(Q, s, Ltau):
    lo, hi = -(-Ltau // 4), Ltau // 2
    idx = np.arange(lo, hi + 1)
    idx = idx[s[idx] > 0]
    w = 1.0 / s[idx] ** 2
    qpl = float((w * Q[idx]).sum() / w.sum())
    err = float(1.0 / math.sqrt(w.sum()))
    dof = len(idx) - 1
    chi2 = float((w * (Q[idx] - qpl) ** 2).sum())
    return qpl, err, (chi2 / dof if dof > 0 else 0.0)


def window(f, s, Ltau):
    """First lag tau >= 1 with f(tau) <= 3.5 sigma(tau); None if there is none."""
    for t in range(1, Ltau // 2 + 1):
        if f[t] <= WINDOW_SIGMAS * s[t]:
            return t
    return None


def _loglin_guess(tau, y):
    """Amplitude and decay length from a straight line through log y (points
    with y > 0); used to start the minimiser."""
    ok = y > 0
    if ok.sum() >= 2:
        slope, icpt = np.polyfit(tau[ok], np.log(y[ok]), 1)
        if slope < 0:
            return math.exp(icpt), -1.0 / slope
    return (float(y[ok][0]) if ok.any() else 1.0), max(1.0, (tau[-1] - tau[0]) / 2)


def _lsq(model, jac, p0, tau, y, s, eta_index, Ltau):
    """Minimum of sum ((model - y) / s)^2 with the decay lengths p[eta_index]
    in (0, 10 L_tau]; parameter errors from (J^T W J)^-1 at the minimum."""
    from scipy.optimize import least_squares

    def res(p):
        return (model(p, tau) - y) / s

    def jres(p):
        return jac(p, tau) / s[:, None]

    lo = np.full(len(p0), -np.inf)
    hi = np.full(len(p0), np.inf)
    lo[eta_index] = 1e-12
    hi[eta_index] = 10.0 * Ltau
    x0 = np.clip(np.asarray(p0, dtype=np.float64), lo + 1e-12, hi)
    r = least_squares(res, x0, jac=jres, method="trf", bounds=(lo, hi), xtol=1e-15, ftol=1e-15, gtol=1e-15,
                      max_nfev=20000)
    p = r.x
    chi2 = float((res(p) ** 2).sum())
    Jw = jres(p)
    try:
        err = np.sqrt(np.abs(np.diag(np.linalg.inv(Jw.T @ Jw))))
    except np.linalg.LinAlgError:
        err = np.full(len(p), np.nan)
    return p, err, chi2


def fit_C_at(C, s, Ltau, zeta, tmin, tw):
    """The C fit on [tmin, tw]: (chi2, dof, params (B, eta), errors), or None
    when fewer than three lags carry weight."""
    def model(p, t):
        B, eta = p
        return B * (np.exp(-t / eta) + zeta * np.exp(-(Ltau - t) / eta))

    def jac(p, t):
        B, eta = p
        e1, e2 = np.exp(-t / eta), np.exp(-(Ltau - t) / eta)
        return np.stack([e1 + zeta * e2, B * (e1 * t + zeta * e2 * (Ltau - t)) / eta ** 2], axis=1)

    tau = np.arange(tmin, tw + 1)
    tau = tau[s[tau] > 0]
    dof = len(tau) - 2
    if dof < 1:
        return None
    B0, eta0 = _loglin_guess(tau.astype(float), C[tau])
    p, err, chi2 = _lsq(model, jac, np.array([B0, min(eta0, 10.0 * Ltau)]), tau.astype(float), C[tau], s[tau],
                        [1], Ltau)
    return chi2, dof, p, err


def fit_C(C, s, Ltau, zeta):
    """Decay length eta of the odd correlator; dict with the window and fit."""
    tw = window(C, s, Ltau)
    out = dict(tau_w=tw if tw is not None else Ltau // 2, ok=False, eta=np.nan, eta_err=np.nan, B=np.nan,
               chi2dof=np.nan, tau_min=0)
    if tw is None:
        return out  # eta > L_tau: not estimated
    tmin = max(1, tw // 10)
    while True:
        r = fit_C_at(C, s, Ltau, zeta, tmin, tw)
        if r is None:
            return out
        chi2, dof, p, err = r
        if chi2 / dof < C_CHI2:
            if p[1] > Ltau:
                return out  # eta beyond L_tau: not estimated
            out.update(ok=True, eta=float(p[1]), eta_err=float(err[1]), B=float(p[0]), chi2dof=chi2 / dof,
                       tau_min=int(tmin))
            return out
        tmin += 1


def fit_Q_at(Q, s, Ltau, tmin, tw, nexp, qpl, free_pl):
    """Q2 = Q_pl + sum of nexp exponentials on [tmin, tw] (Q_pl a parameter
    when free_pl): (chi2, dof, params, errors), or None without a degree of
    freedom.  Parameters: [Q_pl,] B_1, eta_1[, B_2, eta_2]."""
    def split(p):
        if free_pl:
            return p[0], p[1:]
        return qpl, p

    def model(p, t):
        c, q = split(p)
        return c + sum(q[2 * i] * np.exp(-t / q[2 * i + 1]) for i in range(nexp))

    def jac(p, t):
        c, q = split(p)
        cols = [np.ones_like(t)] if free_pl else []
        for i in range(nexp):
            e = np.exp(-t / q[2 * i + 1])
            cols += [e, q[2 * i] * e * t / q[2 * i + 1] ** 2]
        return np.stack(cols, axis=1)

    npar = 2 * nexp + (1 if free_pl else 0)
    tau = np.arange(tmin, tw + 1)
    tau = tau[s[tau] > 0]
    dof = len(tau) - npar
    if dof < 1:
        return None
    t = tau.astype(float)
    base = qpl if not free_pl else float(Q[tau[-1]])
    B0, eta0 = _loglin_guess(t, Q[tau] - base)
    q0 = [B0, eta0] if nexp == 1 else [0.5 * B0, 2.0 * eta0, 0.5 * B0, 0.5 * eta0]
    p0 = np.array(([base] if free_pl else []) + q0)
    off = 1 if free_pl else 0
    p0[off + 1::2] = np.minimum(p0[off + 1::2], 10.0 * Ltau)
    p, err, chi2 = _lsq(model, jac, p0, t, Q[tau], s[tau], list(range(off + 1, len(p0), 2)), Ltau)
    return chi2, dof, p, err


def _fit_Q_terms(Q, s, tw, nexp, qpl, free_pl, Ltau):
    """tau_min from 1 up until chi2/dof < 0.5; returns (chi2/dof, params,
    errors, tau_min) or None."""
    off = 1 if free_pl else 0
    for tmin in range(1, tw + 1):
        r = fit_Q_at(Q, s, Ltau, tmin, tw, nexp, qpl, free_pl)
        if r is None:
            return None
        chi2, dof, p, err = r
        if chi2 / dof < Q_CHI2:
            if np.any(p[off + 1::2] > Ltau):
                return None  # a decay length beyond L_tau: this model is not estimated
            return chi2 / dof, p, err, int(tmin)
    return None


def fit_Q2(Q, s, Ltau):
    qpl, qerr, pchi = plateau_fit(Q, s, Ltau)
    pl_ok = pchi <= PLATEAU_CHI2
    if pl_ok:
        tw = window(Q - qpl, s, Ltau)
        tw = tw if tw is not None else Ltau // 2
    else:
        tw = Ltau // 2
    out = dict(plateau_ok=pl_ok, Q_pl=qpl, Q_pl_err=qerr, plateau_chi2dof=pchi, tau_w=tw, ok=False, n_exp=0,
               eta_e=np.nan, eta_e_err=np.nan, eta_2=np.nan, chi2dof=np.nan, tau_min=0)
    best = None
    for nexp in (1, 2):
        r = _fit_Q_terms(Q, s, tw, nexp, qpl, free_pl=not pl_ok, Ltau=Ltau)
        if r is not None and (best is None or r[0] < best[1][0]):
            best = (nexp, r)
    if best is None:
        return out
    nexp, (cd, p, err, tmin) = best
    off = 0 if pl_ok else 1
    etas = p[off + 1::2]
    eerr = err[off + 1::2]
    i = int(np.argmax(etas))
    out.update(ok=True, n_exp=nexp, eta_e=float(etas[i]), eta_e_err=float(eerr[i]),
               eta_2=float(etas[1 - i]) if nexp == 2 else np.nan, chi2dof=float(cd), tau_min=tmin)
    if not pl_ok:
        out["Q_pl"], out["Q_pl_err"] = float(p[0]), float(err[0])
    return out


def fit_sample(C_reps, Q_reps, Ltau, boundary=0):
    """Both fits of one sample from its per-replica C and Q2 (lags 0..L_tau/2)."""
    C, sc = replica_stats(C_reps)
    Q, sq = replica_stats(Q_reps)
    zeta = -1.0 if boundary == 1 else 1.0
    return dict(C=fit_C(C, sc, Ltau, zeta), Q2=fit_Q2(Q, sq, Ltau))
