"""Batching form: many uneven systems in one plan (one device run, one captured graph),
with the sweep size and evaluation grid chosen by the autotuner; results equal the
oracle's for every system."""

import numpy as np
import pytest

from paper_1802_00330_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00330_gb300 import _binding, build
    build.build()
    _binding.load()
    return _binding


def test_autotuned_batch_matches_oracle(B, orc):
    systems = synth.config_batched(count=48, seed=555, n_range=(2, 7))
    tuned = B.autotune(systems, trial_boxes=20_000)
    assert tuned["wave_children"] in (1 << 20, 1 << 22, 1 << 24) and tuned["eval_blocks"] > 0
    plan = B.Plan(systems, wave_children=tuned["wave_children"], eval_blocks=tuned["eval_blocks"])
    try:
        plan.run()
        for k, s in enumerate(systems):
            g = plan.result(k)
            o = orc.solve(s)
            assert g["status"] == o["status"]
            assert np.array_equal(g["lo"], o["lo"]) and np.array_equal(g["hi"], o["hi"])
            assert g["stats"]["boxes"] == o["stats"]["boxes"]
    finally:
        plan.close()


def test_batch_results_independent_of_schedule(B):
    systems = synth.config_batched(count=16, seed=77, n_range=(3, 6))
    outs = []
    for w, eb in ((1 << 16, 152), (1 << 22, 2432)):
        plan = B.Plan(systems, wave_children=w, eval_blocks=eb)
        plan.run()
        outs.append([plan.result(k) for k in range(len(systems))])
        plan.close()
    for a, b in zip(*outs):
        assert np.array_equal(a["lo"], b["lo"]) and np.array_equal(a["hi"], b["hi"])
