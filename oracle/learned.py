"""Oracle of the learned-ladder part: per-sample coupling features, the MLP
(64 -> 128 -> 128 -> 33, ReLU) with its loss and gradients in FP64, its BF16
inference, Adam, and the log-binning thermalisation judge.

TEST INFRASTRUCTURE ONLY: loaded by the tests and nothing else; it shares no
code with the library's kernels (csrc/k_features.cu, csrc/k_mlp.cu,
csrc/judge.cpp).  The paper has no learned component; the definitions below
are this project's, stated once here and in the library's header.

Couplings J[2][L][L] (+-1): J[0][y][x] couples (x,y)-(x+1,y), J[1][y][x]
couples (x,y)-(x,y+1), periodic.  The plaquette at (x,y) has corners (x,y),
(x+1,y), (x,y+1), (x+1,y+1); it is frustrated when the product of its four
bonds J[0][y][x] J[1][y][x+1] J[0][y+1][x] J[1][y][x] is -1.

Features (64, each a count divided by its number of cases, computed in FP64
and rounded once to FP32):
   0      fraction of frustrated plaquettes
   1-5    sites by the sum of their four bonds: -4, -2, 0, 2, 4
   6-10   sites by the number of frustrated plaquettes among the four touching them: 0..4
   11-15  2x2 blocks of plaquettes (corners at even x, y) by frustrated count: 0..4
   16-31  frustrated fraction in each cell of a 4x4 coarse grid
          (cell (floor(4x/L), floor(4y/L)), index 16 + 4 cy + cx; empty cells 0)
   32, 33 frustrated pairs at diagonal offsets (+1,+1) and (+1,-1), per plaquette
   34, 35 fraction of negative x bonds, of negative y bonds
   36-41  plaquette rows by frustrated fraction, 6 bins [i/6, (i+1)/6) (last closed)
   42-47  plaquette columns likewise
   48-55  frustrated pairs at offset (d, 0), d = 1..8 (mod L), per plaquette
   56-63  frustrated pairs at offset (0, d), d = 1..8
"""
from __future__ import annotations

import math

import numpy as np

N_FEAT, N_H, N_OUT = 64, 128, 33
# parameter vector: W1 [128][64], b1 [128], W2 [128][128], b2 [128], W3 [33][128], b3 [33]
SHAPES = [(N_H, N_FEAT), (N_H,), (N_H, N_H), (N_H,), (N_OUT, N_H), (N_OUT,)]
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES)


# --------------------------------------------------------------------------
# features
# --------------------------------------------------------------------------
def frustration(J):
    L = J.shape[-1]
    F = np.zeros((L, L), dtype=np.int64)
    for y in range(L):
        for x in range(L):
            p = int(J[0, y, x]) * int(J[1, y, (x + 1) % L]) * int(J[0, (y + 1) % L, x]) * int(J[1, y, x])
            F[y, x] = 1 if p < 0 else 0
    return F


def features(J):
    """The 64 features of one sample's couplings J[2][L][L]."""
    J = np.asarray(J, dtype=np.int64)
    L = J.shape[-1]
    F = frustration(J)
    n = L * L
    f = np.zeros(N_FEAT, dtype=np.float64)
    f[0] = F.sum() / n
    for y in range(L):
        for x in range(L):
            s = J[0, y, x] + J[0, y, (x - 1) % L] + J[1, y, x] + J[1, (y - 1) % L, x]
            f[1 + (s + 4) // 2] += 1
            c = F[y, x] + F[y, (x - 1) % L] + F[(y - 1) % L, x] + F[(y - 1) % L, (x - 1) % L]
            f[6 + c] += 1
    f[1:11] /= n
    nb = 0
    for y in range(0, L - 1, 2):
        for x in range(0, L - 1, 2):
            f[11 + F[y, x] + F[y, x + 1] + F[y + 1, x] + F[y + 1, x + 1]] += 1
            nb += 1
    if nb:
        f[11:16] /= nb
    cnt = np.zeros(16)
    tot = np.zeros(16)
    for y in range(L):
        for x in range(L):
            c = (4 * y // L) * 4 + (4 * x // L)
            cnt[c] += F[y, x]
            tot[c] += 1
    f[16:32] = np.where(tot > 0, cnt / np.maximum(tot, 1), 0.0)
    d1 = d2 = 0
    for y in range(L):
        for x in range(L):
            d1 += F[y, x] * F[(y + 1) % L, (x + 1) % L]
            d2 += F[y, x] * F[(y - 1) % L, (x + 1) % L]
    f[32], f[33] = d1 / n, d2 / n
    f[34] = (J[0] < 0).sum() / n
    f[35] = (J[1] < 0).sum() / n
    for y in range(L):
        f[36 + min(int(6 * F[y, :].sum() // L), 5)] += 1
    for x in range(L):
        f[42 + min(int(6 * F[:, x].sum() // L), 5)] += 1
    f[36:48] /= L
    for d in range(1, 9):
        f[47 + d] = sum(F[y, x] * F[y, (x + d) % L] for y in range(L) for x in range(L)) / n
        f[55 + d] = sum(F[y, x] * F[(y + d) % L, x] for y in range(L) for x in range(L)) / n
    return f.astype(np.float32)


# --------------------------------------------------------------------------
# MLP in FP64
# --------------------------------------------------------------------------
def unpack(theta):
    out, o = [], 0
    for s in SHAPES:
        k = int(np.prod(s))
        out.append(np.asarray(theta[o:o + k], dtype=np.float64).reshape(s))
        o += k
    return out


def pack(parts):
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def init_params(seed):
    """He-uniform weights, zero biases (seeded host draw, an input of both sides)."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in SHAPES:
        if len(s) == 2:
            lim = math.sqrt(6.0 / s[1])
            parts.append(rng.uniform(-lim, lim, size=s))
        else:
            parts.append(np.zeros(s))
    return pack(parts).astype(np.float32)


def forward(theta, X):
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0)
    y = h2 @ W3.T + b3
    return y, (X, z1, h1, z2, h2)


def loss_and_grad(theta, X, T):
    """Mean over the batch of: cross-entropy between softmax(y[0:32]) and the
    target fractions T[0:32], plus (y[32] - T[32])^2.  Returns (loss, grad)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    T = np.asarray(T, dtype=np.float64)
    B = T.shape[0]
    y, (X, z1, h1, z2, h2) = forward(theta, X)
    a = y[:, :32]
    a = a - a.max(axis=1, keepdims=True)
    lse = np.log(np.exp(a).sum(axis=1, keepdims=True))
    logp = a - lse
    ce = -(T[:, :32] * logp).sum(axis=1)
    r = y[:, 32] - T[:, 32]
    loss = float((ce + r * r).mean())
    dy = np.zeros_like(y)
    p = np.exp(logp)
    dy[:, :32] = (p * T[:, :32].sum(axis=1, keepdims=True) - T[:, :32]) / B
    dy[:, 32] = 2 * r / B
    gW3 = dy.T @ h2
    gb3 = dy.sum(0)
    dh2 = dy @ W3
    dz2 = dh2 * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (z1 > 0)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(0)
    return loss, pack([gW1, gb1, gW2, gb2, gW3, gb3])


def adam(theta, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) at step number t >= 1, in FP64."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def to_bf16(a):
    """Round FP32 values to bfloat16 (nearest, ties to even), returned as FP64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(theta, X):
    """Inference with BF16 weights, inputs and hidden activations, exact
    products and sums (FP64 here), outputs not rounded."""
    W1, b1, W2, b2, W3, b3 = [to_bf16(p) for p in unpack(theta)]
    h = to_bf16(X)
    h = to_bf16(np.maximum(h @ W1.T + b1, 0))
    h = to_bf16(np.maximum(h @ W2.T + b2, 0))
    return h @ W3.T + b3


def ladder_from_output(y, k_min, k_max):
    """k_j = k_min + (k_max - k_min) sum_{i<=j} softmax(y[0:32])_i; budget 2^(16 y[32])."""
    a = np.asarray(y[:32], dtype=np.float64)
    p = np.exp(a - a.max())
    p /= p.sum()
    return k_min + (k_max - k_min) * np.cumsum(p), 2.0 ** (16.0 * float(y[32]))


# --------------------------------------------------------------------------
# log-binning judge
# --------------------------------------------------------------------------
def judge(E_bins, q_bins, n_last=3, n_sigma=2.0):
    """First bin at which a sample counts as thermalised, or -1.

    E_bins [n_bins][n_samples][R][K]: per replica, the mean energy per site over
    the tempering steps of bin m (sweeps in [2^m, 2^(m+1))).
    q_bins [n_bins][n_samples][K][n_pairs]: per replica pair (pairs in the order
    (0,1), (0,2), ..., (R-2,R-1)), the mean q^2 of the measurements of bin m.
    Each replica's (pair's) bin means are averaged over the K ladder points.
    Energy: mean over replicas, standard error from the replica spread.  q^2:
    mean over pairs, standard error by the jackknife over replicas (leaving
    out replica r drops the pairs that contain it), since pairs that share a
    replica are not independent.  Bin m passes when each of the bins
    m-1 .. m-n_last+1 agrees with it within n_sigma combined standard errors
    (n_sigma sqrt(se_m^2 + se_i^2)) for both observables."""
    E_bins = np.asarray(E_bins, dtype=np.float64)
    q_bins = np.asarray(q_bins, dtype=np.float64)
    nb, ns, R = E_bins.shape[0], E_bins.shape[1], E_bins.shape[2]
    pairs = [(a, b) for a in range(R) for b in range(a + 1, R)]
    out = np.full(ns, -1, dtype=np.int64)

    e = E_bins.mean(axis=3)                       # [nb][ns][R]
    Em = e.mean(axis=2)
    Es = np.sqrt(((e - Em[..., None]) ** 2).sum(axis=2) / (R * (R - 1)))
    q = q_bins.mean(axis=2)                       # [nb][ns][pairs]
    qm = q.mean(axis=2)
    jk = np.stack([q[:, :, [i for i, (a, b) in enumerate(pairs) if r not in (a, b)]].mean(axis=2)
                   for r in range(R)], axis=2)    # [nb][ns][R] leave-one-replica-out means
    jm = jk.mean(axis=2)
    qs = np.sqrt((R - 1) / R * ((jk - jm[..., None]) ** 2).sum(axis=2))
    for b in range(ns):
        for m in range(n_last - 1, nb):
            ok = True
            for i in range(1, n_last):
                for mean, se in ((Em, Es), (qm, qs)):
                    if abs(mean[m, b] - mean[m - i, b]) > n_sigma * math.sqrt(se[m, b] ** 2 + se[m - i, b] ** 2):
                        ok = False
            if ok:
                out[b] = m
                break
    return out


# --------------------------------------------------------------------------
# element-wise error bounds of the FP32 / BF16 arithmetic, for comparing a
# single-precision implementation with the FP64 definitions above
#
# Standard forward error analysis (Higham, "Accuracy and Stability of
# Numerical Algorithms", 2nd ed., Sect. 3.1): an n-term sum or dot product
# evaluated in any order with fused multiply-adds in a format of unit roundoff
# u satisfies |fl(s) - s| <= gamma_n * sum |terms|, gamma_n = n u / (1 - n u).
# Errors of the inputs add through the Lipschitz constant of each step
# (|W| for a matrix product, 1 for ReLU, p for exp).  A ReLU mask is
# ambiguous where |z| does not exceed the bound on z's error: there the
# single-precision result may take either branch, and the bound allows both.
# The bounds are first order; they are doubled to cover the neglected
# second-order terms and the roundings of single operations not itemised
# (the max of the softmax, the constant 1/B, each final store).
# --------------------------------------------------------------------------
U32 = 2.0 ** -24  # unit roundoff of IEEE binary32


def gamma(n, u=U32):
    return n * u / (1.0 - n * u)


def prop(E, A):
    """Error that input errors E (rows: samples) carry through a product with
    A = |weights|: at most E @ A."""
    return E @ A


def _tiles(B, tile=16):
    """Terms of a batch sum computed as per-tile sums of <= `tile` samples,
    then the tile sums in order: at most tile + number of tiles roundings."""
    return min(B, tile) + (B + tile - 1) // tile


def fp32_forward_bound(theta, X):
    """(y, e_y, and per-layer (z, e_z)) for the FP32 forward pass: e bounds
    |y_fp32 - y| element-wise."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    e1 = gamma(W1.shape[1] + 1) * (np.abs(X) @ np.abs(W1).T + np.abs(b1))
    h1 = np.maximum(z1, 0)
    z2 = h1 @ W2.T + b2
    e2 = gamma(W2.shape[1] + 1) * (h1 @ np.abs(W2).T + np.abs(b2)) + prop(e1, np.abs(W2).T)
    h2 = np.maximum(z2, 0)
    y = h2 @ W3.T + b3
    ey = gamma(W3.shape[1] + 1) * (h2 @ np.abs(W3).T + np.abs(b3)) + prop(e2, np.abs(W3).T)
    return y, 2.0 * ey, (z1, 2.0 * e1, z2, 2.0 * e2)


def grad_error_bound(theta, X, T, tile=16):
    """Element-wise bounds on |loss_fp32 - loss| and |g_fp32 - g| for the FP32
    loss and backpropagation of `loss_and_grad` over one batch (per-tile sums
    of <= 16 samples, then the tiles in order).  Returns (loss_bound, g_bound)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    B = T.shape[0]
    nb = _tiles(B, tile)
    y, ey, (z1, e1, z2, e2) = fp32_forward_bound(theta, X)
    h1, h2 = np.maximum(z1, 0), np.maximum(z2, 0)
    # softmax, loss and dL/dy
    a = y[:, :32]
    mx = a.max(axis=1, keepdims=True)
    lse = np.log(np.exp(a - mx).sum(axis=1, keepdims=True))
    logp = a - mx - lse
    p = np.exp(logp)
    t = T[:, :32]
    tsum = t.sum(axis=1, keepdims=True)
    emax = ey[:, :32].max(axis=1, keepdims=True)
    # logp: y, the max and the log-sum (each shifted by <= emax, the sum of 32
    # exponentials of <= 2 ulp each), two subtractions
    e_lse = 2.0 * emax + gamma(34) + 2.0 * U32 * np.abs(lse)
    e_logp = ey[:, :32] + emax + e_lse + 2.0 * U32 * (np.abs(a - mx) + np.abs(lse))
    e_p = p * (e_logp + 3.0 * U32)
    e_tsum = gamma(32) * tsum
    dy = np.zeros_like(y)
    e_dy = np.zeros_like(y)
    dy[:, :32] = (p * tsum - t) / B
    e_dy[:, :32] = (e_p * tsum + p * e_tsum + 3.0 * U32 * (p * tsum + t)) / B + U32 * np.abs(dy[:, :32])
    r = y[:, 32] - T[:, 32]
    dy[:, 32] = 2 * r / B
    e_dy[:, 32] = 2.0 * (ey[:, 32] + U32 * np.abs(r)) / B + 2.0 * U32 * np.abs(dy[:, 32])
    M_dy = np.abs(dy) + e_dy
    # loss = sum over tiles of (sum over the tile of ce + r^2) / B
    ce = -(t * logp).sum(axis=1)
    e_ce = (t * e_logp).sum(axis=1) + gamma(33) * (t * np.abs(logp)).sum(axis=1)
    e_r = ey[:, 32] + U32 * np.abs(r)
    per = (e_ce + 2.0 * np.abs(r) * e_r + 2.0 * U32 * r * r) / B
    loss_bound = per.sum() + gamma(nb + 1) * (np.abs(ce) + r * r).sum() / B

    def outer(d, e_d, h, e_h):
        # sum over the batch of d (x) h: rounding, then the inputs' errors
        Md = np.abs(d) + e_d
        return gamma(nb) * Md.T @ (np.abs(h) + e_h) + e_d.T @ np.abs(h) + np.abs(d).T @ e_h

    def colsum(d, e_d):
        return gamma(nb) * (np.abs(d) + e_d).sum(0) + e_d.sum(0)

    def relu_back(dh, e_dh, z, e_z):
        ambiguous = np.abs(z) <= e_z
        dz = dh * (z > 0)
        e_dz = np.where(ambiguous, np.abs(dh) + e_dh, np.where(z > 0, e_dh, 0.0))
        return dz, e_dz

    gW3 = outer(dy, e_dy, h2, e2)
    gb3 = colsum(dy, e_dy)
    dh2 = dy @ W3
    e_dh2 = gamma(33) * M_dy @ np.abs(W3) + prop(e_dy, np.abs(W3))
    dz2, e_dz2 = relu_back(dh2, e_dh2, z2, e2)
    gW2 = outer(dz2, e_dz2, h1, e1)
    gb2 = colsum(dz2, e_dz2)
    dh1 = dz2 @ W2
    e_dh1 = gamma(W2.shape[0]) * (np.abs(dz2) + e_dz2) @ np.abs(W2) + prop(e_dz2, np.abs(W2))
    dz1, e_dz1 = relu_back(dh1, e_dh1, z1, e1)
    gW1 = outer(dz1, e_dz1, X, np.zeros_like(X))
    gb1 = colsum(dz1, e_dz1)
    return 2.0 * float(loss_bound), 2.0 * pack([gW1, gb1, gW2, gb2, gW3, gb3])


def adam_step_bound(theta, m, v, e_m, e_v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in FP64 from the FP32 state (theta, m, v, the same
    gradient g) with element-wise bounds: returns (theta', m', v', e_m', e_v',
    e_theta) where e_m, e_v bound the single-precision moments' accumulated
    errors and e_theta bounds |theta'_fp32 - theta'| (given equal theta and g).
    Each FP32 operation rounds once (<= u relative); the factor 1 - b^t and
    the learning rate are rounded to FP32 once each."""
    g = np.asarray(g, dtype=np.float64)
    m1 = b1 * m + (1 - b1) * g
    v1 = b2 * v + (1 - b2) * g * g
    e_m1 = b1 * e_m + 3.0 * U32 * (b1 * np.abs(m) + (1 - b1) * np.abs(g))
    e_v1 = b2 * e_v + 4.0 * U32 * (b2 * v + (1 - b2) * g * g)
    c1, c2 = 1 - b1 ** t, 1 - b2 ** t
    mh, vh = m1 / c1, v1 / c2
    den = np.sqrt(vh) + eps
    step = lr * mh / den
    # relative errors: the quotient m^ (moment and factor), the square root of
    # v^ (half of v^'s relative error), the sum with eps, the final quotient
    # and product, the learning rate
    e_mh = e_m1 / c1 + 2.0 * U32 * np.abs(mh)
    rel_den = (0.5 * (e_v1 / np.maximum(v1, 1e-300) + 2.0 * U32) * np.sqrt(vh) + U32 * den) / den
    e_step = lr * e_mh / den + np.abs(step) * (rel_den + 4.0 * U32)
    theta1 = theta - step
    e_theta = e_step + U32 * np.abs(theta1)
    return theta1, m1, v1, e_m1, e_v1, 2.0 * e_theta


def _bf16_interval(lo, hi):
    """Every bfloat16 value that rounding (to nearest even) of an FP32 value in
    [lo, hi] can give, as an interval; the endpoints are first widened by one
    FP32 ulp for their own conversion to FP32."""
    lo = lo - np.abs(lo) * 2.0 ** -23
    hi = hi + np.abs(hi) * 2.0 ** -23
    return to_bf16(lo), to_bf16(hi)


def forward_bf16_interval(theta, X):
    """Interval [lo, hi] holding every output the BF16 inference can give:
    BF16 weights, inputs and hidden activations (round to nearest even), FP32
    accumulation with fused multiply-adds (products of two BF16 values are
    exact in FP32; each sum errs by <= gamma_n sum |terms|), outputs in FP32.
    An activation whose FP32 value may fall on either side of a BF16 rounding
    boundary takes both neighbours, and the spread is carried forward."""
    W1, b1, W2, b2, W3, b3 = [to_bf16(p) for p in unpack(theta)]
    h = to_bf16(X)
    lo = hi = h
    for W, b, last in ((W1, b1, False), (W2, b2, False), (W3, b3, True)):
        mid, rad = (lo + hi) / 2, (hi - lo) / 2
        c = mid @ W.T + b
        mag = np.maximum(np.abs(lo), np.abs(hi)) @ np.abs(W).T + np.abs(b)
        r = prop(rad, np.abs(W).T) + 2.0 * gamma(W.shape[1] + 1) * mag
        zlo, zhi = c - r, c + r
        if last:
            return zlo - 2.0 * U32 * np.abs(zlo), zhi + 2.0 * U32 * np.abs(zhi)
        lo, hi = _bf16_interval(np.maximum(zlo, 0), np.maximum(zhi, 0))
