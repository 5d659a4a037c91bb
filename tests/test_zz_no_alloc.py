"""The sweep entry point that allocates nothing, against the context API.

Callers that may not allocate device memory (a plugin whose memory belongs to
the host application's allocator or to a fixed budget, or code that must not
trigger the device-wide synchronisation of cudaMalloc/cudaFree) pass their own
spin and coupling buffers to qsg_sweep_static_scratch; the kernel's scratch
lives in fixed device arrays inside the library.  Its output must be the
context sweep's, bit for bit, on two calls in a row.  This file is collected
last so that a stop-at-first-failure run has already run everything else.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2310_07486_gb300 import qsg as Q  # noqa: E402

pytestmark = pytest.mark.gpu


def _pack_couplings(J, shape):
    """int8 J [n_samples][2][L][L] (+-1) -> coupling words [2][words][L*L]."""
    words = np.zeros((2, shape.words, shape.L * shape.L), dtype=np.uint64)
    for b in range(shape.n_samples):
        neg = (J[b].reshape(2, -1) < 0).astype(np.uint64) << np.uint64(b % 64)
        words[:, b // 64] |= neg
    return words


@pytest.mark.parametrize("algo,boundary", [(Q.HEATBATH, Q.APBC), (Q.METROPOLIS, Q.PBC)])
def test_static_scratch_sweep_matches_context_sweep(algo, boundary):
    shape = Q.Shape(8, 48, 70, 2, 3, algo, boundary)
    ladder = np.array([0.24, 0.29, 0.34])
    seed = 2718
    ctx = Q.Context([shape])
    ctx.qsg_init_samples(seed, [ladder])
    J = (1 - 2 * np.random.default_rng(5).integers(0, 2, size=(shape.n_samples, 2, shape.L, shape.L))).astype(np.int8)
    ctx.qsg_set_couplings(0, J)
    start = ctx.qsg_get_spins(0)
    jw = _pack_couplings(J, shape)
    dev = torch.device("cuda")
    spins = torch.from_numpy(start.view(np.int64).copy()).to(dev)
    jx = torch.from_numpy(jw[0].view(np.int64).copy()).to(dev)
    jy = torch.from_numpy(jw[1].view(np.int64).copy()).to(dev)
    done = 0
    for n in (3, 2):  # two calls in a row
        Q.qsg_sweep_static_scratch(spins, jx, jy, shape, 0, ladder, seed, done, n)
        ctx.qsg_sweep(n)
        done += n
        torch.cuda.synchronize()
        got = spins.cpu().numpy().view(np.uint64).reshape(ctx.qsg_get_spins(0).shape)
        assert np.array_equal(got, ctx.qsg_get_spins(0)), n


def test_static_scratch_sweep_rejects_oversized_and_bad_shapes():
    dev = torch.device("cuda")
    buf = torch.zeros(16, dtype=torch.int64, device=dev)
    with pytest.raises(Q.QSGError) as e:  # L_tau not a multiple of 16
        Q.qsg_sweep_static_scratch(buf, buf, buf, Q.Shape(8, 24, 64, 1, 1), 0, [0.3], 1, 0, 1)
    assert e.value.status == -2
    with pytest.raises(Q.QSGError) as e:  # more ladder positions than the static table holds
        Q.qsg_sweep_static_scratch(buf, buf, buf, Q.Shape(8, 16, 64, 1, 129), 0, np.linspace(0.1, 0.5, 129), 1, 0, 1)
    assert e.value.status in (-1, -2)
    with pytest.raises(Q.QSGError) as e:  # more slots x chunks than the static counters hold
        Q.qsg_sweep_static_scratch(buf, buf, buf, Q.Shape(8, 16, 64 * 512, 64, 128), 0,
                                   np.linspace(0.1, 0.5, 128), 1, 0, 1)
    assert e.value.status == -1
