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


# L_tau = 48 runs each slot as one chunk; L_tau = 256 with 12 slots runs 8
# chunks of 32 planes per slot, so the boundary counters of several chunks,
# their indexing and the wrap from the last chunk to the first are exercised.
@pytest.mark.parametrize("algo,boundary,Ltau", [(Q.HEATBATH, Q.APBC, 48), (Q.METROPOLIS, Q.PBC, 48),
                                                (Q.HEATBATH, Q.PBC, 256), (Q.METROPOLIS, Q.APBC, 256)])
def test_static_scratch_sweep_matches_context_sweep(algo, boundary, Ltau):
    shape = Q.Shape(8, Ltau, 70, 2, 3, algo, boundary)
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


def test_static_scratch_wrapper_rejects_buffers_that_do_not_fit_the_shape():
    # the wrapper raises before the C entry point is called, so nothing is launched
    dev = torch.device("cuda")
    shape = Q.Shape(8, 16, 64, 1, 1)
    spins = torch.zeros(shape.slots * 16 * 64, dtype=torch.int64, device=dev)
    J = torch.zeros(64, dtype=torch.int64, device=dev)
    small = torch.zeros(16, dtype=torch.int64, device=dev)
    for args in ((small, J, J), (spins, small, J), (spins, J, small), (spins.int(), J, J), (spins.cpu(), J, J)):
        with pytest.raises(Q.QSGError) as e:
            Q.qsg_sweep_static_scratch(*args, shape, 0, [0.3], 1, 0, 1)
        assert e.value.status == -1
    with pytest.raises(Q.QSGError) as e:  # ladder length differs from n_k
        Q.qsg_sweep_static_scratch(spins, J, J, shape, 0, [0.3, 0.4], 1, 0, 1)
    assert e.value.status == -1
