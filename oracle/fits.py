"""Oracle of the per-sample correlation-length fits (Methods, "Fitting process
and Euclidean correlation length estimation") and of the tau-tilde variable
of Sect. "On the magnetic susceptibilities".

TEST INFRASTRUCTURE ONLY: loaded by the tests and nothing else.  It shares no
code with the library's fits (csrc/fits.cpp).

The paper does not name its minimiser.  Both sides read it as Marquardt's
damped Gauss-Newton (Levenberg-Marquardt): damping lambda = 1e-3 to start,
the normal matrix's diagonal scaled by (1 + lambda), lambda x10 after a
rejected step (chi2 not lower, or a decay length not positive), /10 after an
accepted one (not below 1e-15); stop when an accepted step is below 1e-14 of
every parameter, when chi2 falls by less than 1e-15 of itself, after 2000
iterations or when lambda exceeds 1e30.  Following the same iteration from
the same start, two-exponential fits reach the same one of their several
minima on both sides.

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


def _lsq(model, jac, p0, tau, y, s, valid):
    """Levenberg-Marquardt minimisation of sum ((model - y) / s)^2."""
    w = 1.0 / s ** 2

    def chi2_of(p):
        return float((w * (model(p, tau) - y) ** 2).sum())

    def normal(p):
        J = jac(p, tau)
        r = model(p, tau) - y
        return (J * w[:, None]).T @ J, (J * w[:, None]).T @ r

    p = np.array(p0, dtype=np.float64)
    chi2 = chi2_of(p)
    lam = 1e-3
    A, g = normal(p)
    it = 0
    while it < 2000 and lam < 1e30:
        it += 1
        diag = np.where(np.diag(A) > 0, np.diag(A), 1.0)
        M = A + lam * np.diag(diag)
        try:
            step = np.linalg.solve(M, -g)
        except np.linalg.LinAlgError:
            lam *= 10.0
            continue
        trial = p + step
        c2 = chi2_of(trial) if valid(trial) else math.inf
        if not c2 < chi2:
            lam *= 10.0
            continue
        small = bool(np.all(np.abs(step) <= 1e-14 * (np.abs(p) + 1e-14)))
        flat = chi2 - c2 <= 1e-15 * chi2
        p, chi2 = trial, c2
        lam = max(lam * 0.1, 1e-15)
        A, g = normal(p)
        if small or flat:
            break
    try:
        err = np.sqrt(np.abs(np.diag(np.linalg.inv(A))))
    except np.linalg.LinAlgError:
        err = np.full(len(p), np.nan)
    return p, err, chi2


def fit_C(C, s, Ltau, zeta):
    """Decay length eta of the odd correlator; dict with the window and fit."""
    tw = window(C, s, Ltau)
    out = dict(tau_w=tw if tw is not None else Ltau // 2, ok=False, eta=np.nan, eta_err=np.nan, B=np.nan,
               chi2dof=np.nan, tau_min=0)
    if tw is None:
        return out  # eta > L_tau: not estimated

    def model(p, t):
        B, eta = p
        return B * (np.exp(-t / eta) + zeta * np.exp(-(Ltau - t) / eta))

    def jac(p, t):
        B, eta = p
        e1, e2 = np.exp(-t / eta), np.exp(-(Ltau - t) / eta)
        return np.stack([e1 + zeta * e2, B * (e1 * t + zeta * e2 * (Ltau - t)) / eta ** 2], axis=1)

    tmin = max(1, tw // 10)
    while True:
        tau = np.arange(tmin, tw + 1)
        tau = tau[s[tau] > 0]
        dof = len(tau) - 2
        if dof < 1:
            return out
        B0, eta0 = _loglin_guess(tau.astype(float), C[tau])
        p, err, chi2 = _lsq(model, jac, np.array([B0, min(eta0, 10.0 * Ltau)]), tau.astype(float), C[tau], s[tau],
                            lambda q: 0 < q[1] <= 10.0 * Ltau)
        if chi2 / dof < C_CHI2:
            if p[1] > Ltau:
                return out  # eta beyond L_tau: not estimated
            out.update(ok=True, eta=float(p[1]), eta_err=float(err[1]), B=float(p[0]), chi2dof=chi2 / dof,
                       tau_min=int(tmin))
            return out
        tmin += 1


def _fit_Q_terms(Q, s, lo_max, tw, nexp, qpl, free_pl, Ltau):
    """Q2 = Q_pl + sum of nexp exponentials, tau_min from 1 up until
    chi2/dof < 0.5; returns (chi2/dof, params, errors, tau_min) or None."""
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
    for tmin in range(1, lo_max + 1):
        tau = np.arange(tmin, tw + 1)
        tau = tau[s[tau] > 0]
        dof = len(tau) - npar
        if dof < 1:
            return None
        t = tau.astype(float)
        base = qpl if not free_pl else float(Q[tau[-1]])
        B0, eta0 = _loglin_guess(t, Q[tau] - base)
        if nexp == 1:
            q0 = [B0, eta0]
        else:
            q0 = [0.5 * B0, 2.0 * eta0, 0.5 * B0, 0.5 * eta0]
        p0 = np.array(([base] if free_pl else []) + q0)
        off = 1 if free_pl else 0
        p0[off + 1::2] = np.minimum(p0[off + 1::2], 10.0 * Ltau)
        p, err, chi2 = _lsq(model, jac, p0, t, Q[tau], s[tau],
                            lambda q: bool(np.all((q[off + 1::2] > 0) & (q[off + 1::2] <= 10.0 * Ltau))))
        etas = p[off + 1::2]
        if chi2 / dof < Q_CHI2:
            if np.any(etas > Ltau):
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
        r = _fit_Q_terms(Q, s, tw, tw, nexp, qpl, free_pl=not pl_ok, Ltau=Ltau)
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
