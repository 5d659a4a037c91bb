"""How much the one-uniform-per-site-word reading correlates the samples of a
word (the oracle's chain, which the GPU reproduces bit for bit).

The 64 disorder samples of a multispin word share one 32-bit uniform per site
and sweep; samples of different words do not.  Each sample's chain is exact in
law, but their Monte Carlo noise is correlated: measured here as the
equal-time correlation of per-sample energy fluctuations, for pairs in the
same word and pairs in different words, and as the variance of the word-sum
of the fluctuations against the sum of their variances (1 for independent
samples).  The couplings of all samples are drawn the same way, so the two
kinds of pairs differ only in the shared uniforms.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle


def _energy_series(algo, k, T, L=4, Lt=8, seed=3):
    orc = oracle.OracleGroup(L, Lt, 128, 1, 1, algo=algo)
    orc.init(seed, np.array([k]))
    orc.sweep(300)
    E = np.empty((T, 128))
    for t in range(T):
        orc.sweep(1)
        E[t] = orc.energies()[:, 0, 0]
    return E - E.mean(axis=0)


@pytest.mark.parametrize("algo", ["heatbath", "metropolis"])
def test_samples_of_a_word_share_noise_and_words_do_not(algo):
    d = _energy_series(algo, 0.29, 3000)
    C = np.corrcoef(d.T)
    iu = np.triu_indices(64, 1)
    same = np.concatenate([C[:64, :64][iu], C[64:, 64:][iu]]).mean()
    cross = C[:64, 64:].mean()
    ratio = np.mean([d[:, w * 64:(w + 1) * 64].sum(axis=1).var() / d[:, w * 64:(w + 1) * 64].var(axis=0).sum()
                     for w in (0, 1)])
    # different words: independent noise (the mean over 4096 pairs of ~3000
    # correlated sweeps scatters by about 0.01)
    assert abs(cross) < 0.03, cross
    # one word: correlated noise -- at L = 4, L_tau = 8, k = 0.29 the measured
    # values are rho = 0.14 (heat bath) and 0.26 (Metropolis), a word-sum
    # variance of 10 and 17 times the independent value
    assert 0.05 < same < 0.5, same
    assert 1 + 63 * same == pytest.approx(ratio, rel=0.25)
