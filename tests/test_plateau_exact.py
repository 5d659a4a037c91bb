"""The Q2 plateau for both boundaries against the paper's Eq. (plateau-2).

With parity a symmetry of the transfer matrix, the ground states of its even
and odd sectors, |0e> and |0o> (top eigenvalues lambda_e > lambda_o), govern
the plateau of an even operator once L_tau is long compared with every other
correlation length, but not necessarily with eta = 1 / log(lambda_e /
lambda_o): with eps = (lambda_o / lambda_e)^L_tau and zeta = +1 (PBC) or -1
(APBC, the parity operator closing the trace),

    Q2(tau >> eta_e, eta_o) = Q2_e + (Q2_o - Q2_e) zeta eps / (1 + zeta eps),

Q2_e, Q2_o the averages over site pairs (x, y) of <0e|s_x s_y|0e>^2 and
<0o|s_x s_y|0o>^2 (Methods, "The limit of zero temperature").  The test takes
the exact correlators of Eq. (C_A_transfer) from ``exact.transfer_correlators``
(the construction the oracle is pinned to for both boundaries) at tau = L_tau
/ 2 and compares them with the formula evaluated from the two sector ground
states, for 2 x 2 samples at k where eps is neither 0 nor 1.  A boundary
term with the wrong sign, or a missing parity operator, moves the APBC value
by about 2 eps |Q2_o - Q2_e|, which the test requires to exceed its
tolerance twentyfold.
"""
from __future__ import annotations

import numpy as np
import pytest

import exact


def _sector_ground_states(T):
    dim = T.shape[0]
    P = np.zeros((dim, dim))
    P[np.arange(dim), (dim - 1) ^ np.arange(dim)] = 1.0  # flips every spin
    out = {}
    for name, sign in (("e", 1.0), ("o", -1.0)):
        proj = 0.5 * (np.eye(dim) + sign * P)
        w, V = np.linalg.eigh(proj @ T @ proj)
        out[name] = (w[-1], V[:, -1])
    return out


@pytest.mark.parametrize("seed,k", [(5, 1.3), (11, 1.0)])
def test_q2_plateau_follows_the_parity_formula(seed, k):
    rng = np.random.default_rng(seed)
    L, Ltau = 2, 256
    J = (1 - 2 * rng.integers(0, 2, size=(2, L, L))).astype(np.int8)
    T, sl = exact.transfer_matrix(J, L, k)
    gs = _sector_ground_states(T)
    (lam_e, ve), (lam_o, vo) = gs["e"], gs["o"]
    assert lam_e > lam_o > 0
    eps = (lam_o / lam_e) ** Ltau
    assert 0.01 < eps < 0.5
    S = sl.astype(np.float64)
    n = L * L
    # <0|s_x s_y|0> for every pair (diagonal operators in the sigma^z basis)
    Ae = np.einsum("a,ax,ay->xy", ve * ve, S, S)
    Ao = np.einsum("a,ax,ay->xy", vo * vo, S, S)
    q2e, q2o = np.mean(Ae ** 2), np.mean(Ao ** 2)
    tol = 1e-7

    def plateau(zeta):
        return q2e + (q2o - q2e) * zeta * eps / (1.0 + zeta * eps)

    for boundary, zeta in (("pbc", 1.0), ("apbc", -1.0)):
        _, Q, _ = exact.transfer_correlators(J, L, Ltau, k, boundary)
        assert abs(Q[Ltau // 2] - plateau(zeta)) < tol, (boundary, Q[Ltau // 2], plateau(zeta))
        # the other boundary's formula is far off: the test resolves zeta
        assert abs(Q[Ltau // 2] - plateau(-zeta)) > 20 * tol
    # the two boundaries bracket the zero-temperature value Q2_e
    _, Qp, _ = exact.transfer_correlators(J, L, Ltau, k, "pbc")
    _, Qa, _ = exact.transfer_correlators(J, L, Ltau, k, "apbc")
    lo, hi = sorted((Qp[Ltau // 2], Qa[Ltau // 2]))
    assert lo <= q2e <= hi
