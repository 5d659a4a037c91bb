"""Launch-option autotuner: candidate generation on the host, and on the GPU
that a tuned context samples exactly the bits of an untuned one."""
from __future__ import annotations

import json

import numpy as np
import pytest

from paper_2310_07486_gb300 import qsg as Q
from paper_2310_07486_gb300 import tuner


def test_candidate_chunks_divide_every_ltau():
    shapes = [Q.Shape(8, 96, 64, 1, 2), Q.Shape(12, 64, 64, 1, 2)]
    assert tuner.candidate_chunks(shapes) == [0, 16, 32]
    assert tuner.candidate_chunks([Q.Shape(24, 2048, 64, 1, 1)]) == [0, 16, 32, 64, 128, 256, 512]
    assert tuner.candidate_chunks([Q.Shape(8, 24, 64, 1, 1)]) == [0]


def test_candidates_cover_persistent_and_graph_only_where_they_apply():
    one = list(tuner.candidates([Q.Shape(8, 32, 64, 1, 1)], sweeps_per_call=1))
    assert {c["persistent"] for c in one} == {1} and {c["graph"] for c in one} == {0}
    two = list(tuner.candidates([Q.Shape(8, 32, 64, 1, 1), Q.Shape(6, 32, 64, 1, 1)], sweeps_per_call=30))
    assert {c["persistent"] for c in two} == {1, 2, 3} and {c["graph"] for c in two} == {0, 30}
    assert len(two) == len({json.dumps(c, sort_keys=True) for c in two})


def test_units_per_block_stage_only_where_the_generic_kernel_runs():
    compiled = [Q.Shape(24, 2048, 64, 1, 1), Q.Shape(20, 1024, 64, 1, 1), Q.Shape(16, 512, 64, 1, 1),
                Q.Shape(12, 256, 64, 1, 1), Q.Shape(8, 128, 64, 1, 1)]
    assert not tuner.uses_generic_kernel(compiled, variant=0)
    assert tuner.uses_generic_kernel([Q.Shape(24, 2048, 64, 1, 1), Q.Shape(10, 512, 64, 1, 1)], variant=0)
    assert tuner.uses_generic_kernel([Q.Shape(24, 2048, 64, 1, 1)], variant=2)
    first = list(tuner.candidates([Q.Shape(8, 32, 64, 1, 1)], sweeps_per_call=4))
    assert {c["upb"] for c in first} == {0}  # the first stage keeps the automatic grouping
    assert tuner.UPB == [1, 2, 4, 8, 16] and tuner.DEFAULTS["upb"] == 0


def test_candidates_restricted_to_a_space():
    shapes = [Q.Shape(8, 128, 64, 1, 1), Q.Shape(24, 2048, 64, 1, 1)]
    space = {"graph": [30], "chunk": [0, 64, 128, 999], "variant": [0, 3]}
    got = list(tuner.candidates(shapes, sweeps_per_call=30, space=space))
    assert {c["chunk"] for c in got} == {0, 64, 128}  # 999 is not a valid chunk
    assert {c["variant"] for c in got} == {0, 3} and {c["graph"] for c in got} == {30}
    assert {c["persistent"] for c in got} == {1, 2, 3}
    assert len(got) == 3 * 2 * 3


@pytest.mark.gpu
def test_tuned_context_samples_the_same_bits(tmp_path):
    torch = pytest.importorskip("torch")
    shapes = [Q.Shape(8, 32, 70, 2, 3, Q.HEATBATH, Q.PBC), Q.Shape(12, 64, 5, 1, 2, Q.HEATBATH, Q.APBC)]
    lads = [np.array([0.2, 0.3, 0.4]), np.array([0.25, 0.33])]
    cache = str(tmp_path / "tuning.json")

    def run(tune):
        ctx = Q.Context(shapes)
        ctx.qsg_init_samples(31, lads)
        ctx.qsg_sweep(2)
        info = tuner.tune(ctx, sweeps_per_call=4, reps=1, cache_path=cache) if tune else None
        for _ in range(3):
            ctx.qsg_sweep(4)
            ctx.qsg_tempering_swap()
        torch.cuda.synchronize()
        return [ctx.qsg_get_spins(g) for g in range(len(shapes))], ctx.qsg_get_counters(), info

    plain, c_plain, _ = run(False)
    tuned, c_tuned, info = run(True)
    assert not info["cached"] and info["table"]
    assert c_plain == c_tuned
    for a, b in zip(plain, tuned):
        assert np.array_equal(a, b)
    again, _, info2 = run(True)
    assert info2["cached"] and info2["options"] == info["options"]
    for a, b in zip(plain, again):
        assert np.array_equal(a, b)
