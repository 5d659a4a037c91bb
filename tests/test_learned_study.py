"""What the trained predictor gains: the whole learned-ladder study on the
GPU (plain runs for labels, training with the library's kernels, then plain
against learned ladders on fresh samples, judged by qsg_judge).  Everything
is seeded and the sampler and training are deterministic, so the outcome is
reproducible."""
from __future__ import annotations

import json
import os

import pytest

pytestmark = pytest.mark.gpu


def test_learned_ladder_study_gains_over_the_uniform_ladder(tmp_path):
    pytest.importorskip("torch")
    from paper_2310_07486_gb300 import ladder, workloads
    out = ladder.study_main(workloads.ladder_study(), log=lambda *a: None)
    (tmp_path / "ladder_study.json").write_text(json.dumps(out))
    print(json.dumps(out))
    assert out["train_loss_first_last"][1] < out["train_loss_first_last"][0]
    assert out["plain"]["passed"] > 0.5 and out["learned"]["passed"] >= out["plain"]["passed"] - 0.02
    # fewer GPU-seconds per sample to pass the judge than the uniform ladder
    assert out["gain"] > 1.0, out
