"""Bounded device waits give up with a status instead of hanging.

The tensor-core correlator kernel hands stages between its warp roles through
mbarrier waits, each limited to a number of polls.  With the limit set to zero
every wait gives up at once: no MMA is issued, every role runs out its loops,
the tensor memory is freed and the kernel returns normally; the context's
device flag makes qsg_read_correlators report QSG_ERR_TIMEOUT.  Nothing waits
on anything that cannot arrive, and no fault is raised.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2310_07486_gb300 import qsg as Q  # noqa: E402

pytestmark = pytest.mark.gpu


def _run(shape, lad, seed, wait_limit=None):
    ctx = Q.Context([shape])
    ctx.qsg_init_samples(seed, [lad])
    ctx.qsg_set_option(Q.OPT_CORR_KERNEL, Q.CORR_TENSOR)
    if wait_limit is not None:
        ctx.qsg_set_option(Q.OPT_WAIT_LIMIT, wait_limit)
    ctx.qsg_sweep(2)
    ctx.qsg_measure_correlators()
    return ctx


def test_wait_that_gives_up_reports_timeout_and_the_next_context_works():
    shape = Q.Shape(8, 256, 64, 2, 1, Q.HEATBATH, Q.PBC)
    lad = np.array([0.3])
    ctx = _run(shape, lad, 7, wait_limit=0)
    with pytest.raises(Q.QSGError) as e:
        ctx.qsg_read_correlators()
    assert e.value.status == -4
    # the flag stays set for that context
    with pytest.raises(Q.QSGError) as e:
        ctx.qsg_read_correlators()
    assert e.value.status == -4
    # the device and a fresh context are unaffected
    ctx.qsg_sweep(1)
    torch.cuda.synchronize()
    good = _run(shape, lad, 7)
    orc = oracle.OracleGroup(shape.L, shape.Ltau, shape.n_samples, shape.n_replicas, shape.n_k,
                             algo=shape.algo, boundary=shape.boundary)
    orc.init(7, lad)
    orc.sweep(2)
    orc.measure()
    got, ref = good.qsg_read_correlators(raw=True), orc.read()
    for key in ("C_raw", "Q2_raw", "q2_raw"):
        assert np.array_equal(got[key], ref[key]), key


def test_wait_limit_is_validated():
    shape = Q.Shape(8, 16, 64, 1, 1)
    ctx = Q.Context([shape])
    for bad in (-1, 1 << 31):
        with pytest.raises(Q.QSGError):
            ctx.qsg_set_option(Q.OPT_WAIT_LIMIT, bad)
    ctx.qsg_set_option(Q.OPT_WAIT_LIMIT, 1 << 22)


def test_asynchronous_read_reports_the_flag_when_waited_for():
    """qsg_read_correlators_async queues its copies without checking the
    device flag; qsg_wait_correlators reports it once the copies are done,
    and a context whose waits never gave up reports nothing."""
    shape = Q.Shape(8, 256, 64, 2, 1, Q.HEATBATH, Q.PBC)
    lad = np.array([0.3])
    copy_stream = torch.cuda.Stream()
    bad = _run(shape, lad, 7, wait_limit=0)
    bad.qsg_read_correlators_async(bad.correlator_buffers(pinned=True), copy_stream)
    with pytest.raises(Q.QSGError) as e:
        bad.qsg_wait_correlators()
    assert e.value.status == -4
    good = _run(shape, lad, 7)
    out = good.correlator_buffers(pinned=True)
    good.qsg_read_correlators_async(out, copy_stream)
    good.qsg_wait_correlators()
    ref = good.qsg_read_correlators()
    for key in ("C", "Q2", "q2"):
        assert np.array_equal(out[key], ref[key]), key
