"""Batching form: many uneven systems in one plan (one device run, one captured graph),
with the sweep size and evaluation grid chosen by the autotuner; results equal the
oracle's for every system.

The oracle takes about 1.5 s per 100k boxes, so the batch is the systems of a seeded
draw that the oracle itself finishes within 100k boxes (n = 2..5, from a few dozen to
about 90k boxes each); the selection uses the oracle alone.
"""

import numpy as np
import pytest

from paper_1802_00330_gb300 import synth

pytestmark = pytest.mark.gpu

ORACLE_BOX_BUDGET = 100_000


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00330_gb300 import _binding, build
    build.build()
    _binding.load()
    return _binding


@pytest.fixture(scope="module")
def small_batch(orc):
    """(systems, oracle results) for the draw's systems the oracle finishes."""
    systems, results = [], []
    for s in synth.config_batched(count=64, seed=555, n_range=(2, 5)):
        o = orc.solve(s, max_boxes=ORACLE_BOX_BUDGET)
        if o["status"] == 0:
            systems.append(s)
            results.append(o)
    assert len(systems) >= 40 and len({s.n_vars for s in systems}) >= 4
    return systems, results


def test_autotuned_batch_matches_oracle(B, small_batch):
    systems, expected = small_batch
    tuned = B.autotune(systems, trial_boxes=20_000)
    assert tuned["wave_children"] in (1 << 20, 1 << 22, 1 << 24) and tuned["eval_blocks"] > 0
    plan = B.Plan(systems, wave_children=tuned["wave_children"], eval_blocks=tuned["eval_blocks"])
    try:
        plan.run()
        for k, o in enumerate(expected):
            g = plan.result(k)
            assert g["status"] == o["status"], k
            assert np.array_equal(g["lo"], o["lo"]) and np.array_equal(g["hi"], o["hi"]), k
            assert np.array_equal(g["flags"], o["flags"]), k
            assert g["stats"]["boxes"] == o["stats"]["boxes"], k
    finally:
        plan.close()


def test_batch_results_independent_of_schedule(B, small_batch):
    systems = small_batch[0][:16]
    outs = []
    for w, eb in ((1 << 16, 152), (1 << 22, 2432)):
        plan = B.Plan(systems, wave_children=w, eval_blocks=eb)
        try:
            plan.run()
            outs.append([plan.result(k) for k in range(len(systems))])
        finally:
            plan.close()
    for a, b in zip(*outs):
        assert a["status"] == b["status"] and a["stats"]["boxes"] == b["stats"]["boxes"]
        assert np.array_equal(a["lo"], b["lo"]) and np.array_equal(a["hi"], b["hi"])
