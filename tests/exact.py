"""Exact results for tiny lattices, used to pin the oracle.

Everything here is computed from the paper's definitions by routes that do not
go through the oracle's Monte Carlo code:

* ``enumerate_states`` sums the classical weight exp(-k E(S)) of
  Eq. (Trotter-action) over all 2^(L^2 L_tau) configurations (brute force).
* ``transfer_matrix`` builds the Trotter-Suzuki transfer matrix of
  Eq. (Trotter-transfer-matrix), T = exp(-k H0/2) exp(-k H1) exp(-k H0/2),
  from the quantum Hamiltonian of Eq. (H-def) with Gamma = -ln(tanh k)/(2k);
  correlators then follow from Eq. (C_A_transfer) by matrix powers.
* ``hamiltonian`` is H of Eq. (H-def) itself, for exact diagonalisation.

Couplings use the layout J[2][L][L]: J[0][y][x] couples (x,y)-(x+1,y),
J[1][y][x] couples (x,y)-(x,y+1) (periodic).
"""
from __future__ import annotations

import numpy as np


def gamma_of_k(k):
    """Transverse field of Eq. (Trotter-action): Gamma = -ln(tanh k) / (2k)."""
    return -np.log(np.tanh(k)) / (2.0 * k)


def bonds(L):
    """List of (site_a, site_b, direction, y, x) for the 2 L^2 space bonds."""
    out = []
    for y in range(L):
        for x in range(L):
            a = y * L + x
            out.append((a, y * L + (x + 1) % L, 0, y, x))
            out.append((a, ((y + 1) % L) * L + x, 1, y, x))
    return out


def slice_states(L):
    """All 2^(L^2) spin slices as an int8 array [n_states][L^2] (bit=1 -> -1)."""
    n = L * L
    idx = np.arange(2 ** n, dtype=np.int64)[:, None]
    bits = (idx >> np.arange(n)[None, :]) & 1
    return (1 - 2 * bits).astype(np.int8)


def space_energy(states, J, L):
    """-(sum over space bonds J S S) of each slice (the H0 eigenvalue)."""
    e = np.zeros(states.shape[0], dtype=np.float64)
    for a, b, d, y, x in bonds(L):
        e -= J[d, y, x] * states[:, a].astype(np.float64) * states[:, b]
    return e


def enumerate_states(J, L, Ltau, k, boundary="pbc"):
    """Brute-force Boltzmann average over all classical configurations.

    Returns dict with Z (unnormalised, exp(-k E) summed), mean action <E>,
    C[lag], Q2[lag] for lag = 0 .. Ltau/2 following Eq. (def-C-Q2-tau) with the
    estimator normalisation 1/(L_tau L^D) and 1/(L_tau L^2D).
    """
    n = L * L * Ltau
    assert n <= 20
    sl = slice_states(L)
    ns = sl.shape[0]
    # configuration = tuple of slice indices; enumerate via mixed radix
    idx = np.arange(ns ** Ltau, dtype=np.int64)
    slices = [(idx // ns ** t) % ns for t in range(Ltau)]
    esp = space_energy(sl, J, L)
    E = np.zeros(idx.shape[0])
    for t in range(Ltau):
        E += esp[slices[t]]
        s1 = sl[slices[t]].astype(np.float64)
        s2 = sl[slices[(t + 1) % Ltau]].astype(np.float64)
        sign = -1.0 if (boundary == "apbc" and t == Ltau - 1) else 1.0
        E -= sign * (s1 * s2).sum(axis=1)
    w = np.exp(-k * (E - E.min()))
    Z = w.sum()
    p = w / Z
    nl = Ltau // 2 + 1
    C = np.zeros(nl)
    Q = np.zeros(nl)
    L2 = L * L
    for lag in range(nl):
        csum = np.zeros(idx.shape[0])
        qsum = np.zeros(idx.shape[0])
        for t1 in range(Ltau):
            t2 = t1 + lag
            sgn = 1.0
            if t2 >= Ltau:
                t2 -= Ltau
                if boundary == "apbc":
                    sgn = -1.0
            cc = (sl[slices[t1]].astype(np.float64) * sl[slices[t2]]).sum(axis=1)
            csum += sgn * cc
            qsum += cc * cc
        C[lag] = (p * csum).sum() / (Ltau * L2)
        Q[lag] = (p * qsum).sum() / (Ltau * L2 * L2)
    # M_xy = <S_x S_y> at equal time (averaged over the L_tau slices), Eq. (def-M)
    M = np.zeros((L2, L2))
    for t in range(Ltau):
        s = sl[slices[t]].astype(np.float64)
        M += np.einsum("n,nx,ny->xy", p, s, s)
    M /= Ltau
    # four-point function at equal time, sum_{xyzu} <S_x S_y S_z S_u>^2 (Eq. (Binder))
    M4 = np.zeros((L2,) * 4)
    for t in range(Ltau):
        s = sl[slices[t]].astype(np.float64)
        M4 += np.einsum("n,nx,ny,nz,nu->xyzu", p, s, s, s, s)
    M4 /= Ltau
    # momentum-space traces with p = (2 pi / L, 0) and (0, 2 pi / L), Eq. (def-M)
    xs = np.arange(L2) % L
    ys = np.arange(L2) // L
    trMhatM, trMhatM2 = [], []
    for coord in (xs, ys):
        ph = np.exp(2j * np.pi * coord / L)
        Mhat = M * ph[:, None] * np.conj(ph)[None, :]
        trMhatM.append(np.trace(Mhat @ M).real)
        trMhatM2.append(np.trace(Mhat @ M @ M).real)
    return dict(Z_scaled=Z, Emin=E.min(), E=(p * E).sum(), E2=(p * E * E).sum(), C=C, Q2=Q,
                logZ=np.log(Z) - k * E.min(), trM2=(M * M).sum() / (L2 * L2), M=M,
                chi2=np.trace(M @ M) / L2, chi3=np.trace(M @ M @ M) / L2,
                F2=np.mean(trMhatM) / L2, F3=np.mean(trMhatM2) / L2, q4=(M4 * M4).sum() / L2 ** 4)


def transfer_matrix(J, L, k):
    """T = exp(-k H0/2) exp(-k H1) exp(-k H0/2) in the sigma^z basis, H1 = -Gamma sum sigma^x."""
    sl = slice_states(L)
    h0 = space_energy(sl, J, L)
    g = gamma_of_k(k)
    n = L * L
    # exp(k Gamma sigma^x) on one site = [[cosh, sinh],[sinh, cosh]]; tensor product
    c, s = np.cosh(k * g), np.sinh(k * g)
    # element <a| prod_x exp(kG sx) |b> = cosh^(n - d) sinh^d with d = Hamming distance
    ia = np.arange(2 ** n)
    ham = np.zeros((2 ** n, 2 ** n), dtype=np.int64)
    x = ia[:, None] ^ ia[None, :]
    for bit in range(n):
        ham += (x >> bit) & 1
    M1 = c ** (n - ham) * s ** ham
    d = np.exp(-0.5 * k * h0)
    return d[:, None] * M1 * d[None, :], sl


def per_site_norm(k):
    """A^2 = sinh(2 k Gamma)/2: the per-site factor between T and the classical weight."""
    return 0.5 * np.sinh(2.0 * k * gamma_of_k(k))


def transfer_correlators(J, L, Ltau, k, boundary="pbc"):
    """C(lag), Q2(lag) from Eq. (C_A_transfer); APBC inserts the parity operator P."""
    T, sl = transfer_matrix(J, L, k)
    w, V = np.linalg.eigh(T)
    w = w / w.max()
    n = L * L
    dim = 2 ** n
    P = np.zeros((dim, dim))
    P[np.arange(dim), (dim - 1) ^ np.arange(dim)] = 1.0  # flips every spin
    def Tpow(m):
        return (V * w ** m) @ V.T
    TL = Tpow(Ltau)
    Pend = P if boundary == "apbc" else np.eye(dim)
    Z = np.trace(TL @ Pend)
    nl = Ltau // 2 + 1
    C = np.zeros(nl)
    Q = np.zeros(nl)
    S = sl.astype(np.float64)
    for lag in range(nl):
        A = Tpow(lag)
        B = Tpow(Ltau - lag) @ Pend
        # sum_x Tr(sz_x T^lag sz_x T^(Lt-lag) P): diagonal operators
        # Tr(D1 A D2 B) = sum_ab D1[a] A[a,b] D2[b] B[b,a]
        AB = A * B.T
        for xsite in range(n):
            C[lag] += S[:, xsite] @ AB @ S[:, xsite]
        # sum_xy (s_x s_y)(s'_x s'_y) = (sum_x s_x s'_x)^2
        G = S @ S.T
        Q[lag] = np.sum(AB * G * G)
    return C / (Z * n), Q / (Z * n * n), Z


def hamiltonian(J, L, gamma):
    """Dense H of Eq. (H-def): -sum_bonds J sz sz - Gamma sum_x sx (dimension 2^(L^2))."""
    sl = slice_states(L)
    n = L * L
    dim = 2 ** n
    H = np.diag(space_energy(sl, J, L)).astype(np.float64)
    ia = np.arange(dim)
    for bit in range(n):
        H[ia, ia ^ (1 << bit)] -= gamma
    return H


def one_sweep_markov_matrix(J, L, Ltau, k, algo="metropolis"):
    """Exact one-sweep transition matrix of the quantised checkerboard chain.

    Uses the acceptance probabilities T/2^32 of the 32-bit integer thresholds,
    computed here from the paper's Boltzmann factors (not from the oracle).
    Colour 0 sites update simultaneously (they do not interact), then colour 1.
    """
    n = L * L * Ltau
    assert n <= 10
    dim = 2 ** n
    states = ((np.arange(dim)[:, None] >> np.arange(n)[None, :]) & 1)
    spins = 1 - 2 * states

    def nb(xs, ys, ts):
        return (ts % Ltau) * L * L + (ys % L) * L + (xs % L)

    def prob_flip_or_up(spin_row, site):
        t, rem = divmod(site, L * L)
        y, x = divmod(rem, L)
        h = (J[0, y, x] * spin_row[nb(x + 1, y, t)] + J[0, y, (x - 1) % L] * spin_row[nb(x - 1, y, t)]
             + J[1, y, x] * spin_row[nb(x, y + 1, t)] + J[1, (y - 1) % L, x] * spin_row[nb(x, y - 1, t)]
             + spin_row[nb(x, y, t + 1)] + spin_row[nb(x, y, t - 1)])
        if algo == "metropolis":
            Sh = spin_row[site] * h
            if Sh <= 0:
                return 1.0
            return np.floor(np.exp(-2.0 * k * Sh) * 2.0 ** 32) / 2.0 ** 32
        p = 1.0 / (1.0 + np.exp(-2.0 * k * h))
        return min(np.floor(p * 2.0 ** 32), 2.0 ** 32 - 1) / 2.0 ** 32

    def half(colour):
        M = np.zeros((dim, dim))
        sites = [i for i in range(n) if ((i % L) + (i // L) % L + i // (L * L)) % 2 == colour]
        for a in range(dim):
            row = spins[a]
            probs = []
            for sidx in sites:
                p = prob_flip_or_up(row, sidx)
                probs.append(p)
            # enumerate outcomes of the independent site updates
            for m in range(2 ** len(sites)):
                new = row.copy()
                pr = 1.0
                for q, sidx in enumerate(sites):
                    bit = (m >> q) & 1
                    if algo == "metropolis":
                        if bit:
                            new[sidx] = -row[sidx]
                            pr *= probs[q]
                        else:
                            pr *= 1.0 - probs[q]
                    else:
                        new[sidx] = 1 if bit else -1
                        pr *= probs[q] if bit else 1.0 - probs[q]
                if pr == 0.0:
                    continue
                b = int(((1 - new) // 2) @ (1 << np.arange(n)))
                M[a, b] += pr
        return M

    return half(0) @ half(1), spins


def classical_action(spins, J, L, Ltau, boundary="pbc"):
    """E(S) of Eq. (Trotter-action) for spins [..., Ltau, L, L]."""
    S = spins.astype(np.int64)
    E = -(J[0][None] * S * np.roll(S, -1, axis=-1)).sum(axis=(-1, -2, -3))
    E = E - (J[1][None] * S * np.roll(S, -1, axis=-2)).sum(axis=(-1, -2, -3))
    sign = np.ones(Ltau, dtype=np.int64)
    if boundary == "apbc":
        sign[-1] = -1
    E = E - (sign[:, None, None] * S * np.roll(S, -1, axis=-3)).sum(axis=(-1, -2, -3))
    return E
