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
    st = workloads.ladder_study()
    out = ladder.study_main(st, seeds=[st.seeds[0]], log=lambda *a: None)
    (tmp_path / "ladder_study.json").write_text(json.dumps(out))
    print(json.dumps({k: v for k, v in out.items() if k != "per_seed"}))
    one = out["per_seed"][0]
    assert one["train_loss_first_last"][1] < one["train_loss_first_last"][0]
    # more samples reach the judge's criterion within the cap with the learned ladders
    assert out["learned_passed"] > out["plain_passed"]
    # fewer GPU-seconds per thermalised sample: the lower end of the paired
    # bootstrap interval (resampled evaluation samples) is above 1
    assert out["gain_interval95"][0] > 1.0, out
    # the size input carries the budget's growth with the lattice size
    by_size = out["budget_by_training_size"]
    pred = [b["pred_mean_log2_budget"] for b in by_size]
    assert pred == sorted(pred)
