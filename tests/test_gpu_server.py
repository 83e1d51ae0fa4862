"""Serving form: continuous batching over one shared device queue.

Each result must be the same alone (ivs_solve) and in the mix (served while other
systems of different sizes share the same sweeps), bit for bit; requests submitted
while others are running are admitted and finish.
"""

import time

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


def wait_all(sv, tickets, budget_s=180.0):
    """Results of all tickets, or a failure once the overall budget is spent."""
    deadline = time.time() + budget_s
    out = []
    for t in tickets:
        left = deadline - time.time()
        assert left > 0, "server did not finish in time: " + str(sv.stats())
        r = sv.wait(t, timeout_s=left)
        assert r is not None, "server did not finish in time: " + str(sv.stats())
        out.append(r)
    return out


def same(a, b):
    return (a["status"] == b["status"] and np.array_equal(a["lo"], b["lo"]) and np.array_equal(a["hi"], b["hi"])
            and np.array_equal(a["flags"], b["flags"]) and a["stats"]["boxes"] == b["stats"]["boxes"])


def mix_systems():
    small = synth.config_batched(count=40, seed=31337, n_range=(2, 6))
    return small


@pytest.mark.parametrize("schedule", [0, 1])
def test_alone_equals_in_the_mix(B, schedule):
    """Both schedules (least attained service first; rotating equal shares) leave every
    result as it is alone."""
    systems = mix_systems()
    targets = [0, 7, 19, 33]
    alone = {i: B.solve(systems[i]) for i in targets}
    sv = B.Server(workspace_bytes=1 << 30, max_slots=64, wave_children=1 << 20, max_vars=8, schedule=schedule)
    try:
        tickets = [sv.submit(s) for s in systems]
        results = wait_all(sv, tickets)
        for i in targets:
            assert same(results[i], alone[i]), i
        for i in (3, 11, 25):
            assert same(results[i], B.solve(systems[i])), i
        st = sv.stats()
        assert st["last_error"] == "", st["last_error"]
        assert st["admitted"] == len(systems) and st["completed"] == len(systems)
    finally:
        sv.close()


def test_requests_join_while_others_run(B):
    systems = mix_systems()
    big = synth.config_n6()
    sv = B.Server(workspace_bytes=1 << 30, max_slots=16, wave_children=1 << 20, sweeps_per_step=1, max_vars=8)
    try:
        t_big = sv.submit(big)
        time.sleep(0.002)
        later = [sv.submit(s) for s in systems[:10]]
        res_later = wait_all(sv, later)
        res_big = wait_all(sv, [t_big])[0]
        assert same(res_big, B.solve(big))
        for s, r in zip(systems[:10], res_later):
            assert same(r, B.solve(s))
        # the per-request clocks are filled
        assert res_big["stats"]["solve_ms"] > 0
    finally:
        sv.close()


def test_poll_and_unknown_ticket(B):
    sv = B.Server(workspace_bytes=1 << 28, max_slots=4, wave_children=1 << 18, max_vars=4)
    try:
        t = sv.submit(synth.config_n2())
        r = None
        deadline = time.time() + 60
        while r is None and time.time() < deadline:
            r = sv.poll(t)
            time.sleep(0.001)
        assert r is not None and r["status"] == 0 and len(r["lo"]) == 2
        with pytest.raises(B.IvsError):
            sv.poll(t)          # already handed out
    finally:
        sv.close()


def test_many_slots_and_a_large_admission_burst(B):
    """More than 128 slots and hundreds of requests admitted in few steps: every
    result equals the single-system solve."""
    systems = synth.config_batched(count=300, seed=4242, n_range=(2, 3))
    sv = B.Server(workspace_bytes=1 << 30, max_slots=512, wave_children=1 << 18, max_vars=3)
    try:
        tickets = [sv.submit(s) for s in systems]
        results = wait_all(sv, tickets)
        st = sv.stats()
        assert st["last_error"] == "", st["last_error"]
        assert st["admitted"] == len(systems)
        for i in range(0, len(systems), 37):
            assert same(results[i], B.solve(systems[i])), i
        assert all(r["status"] == 0 for r in results)
    finally:
        sv.close()


def test_time_budget_frees_the_queue(B):
    """A request that runs out of its time budget completes with IVS_ERR_TIMEOUT soon
    after the budget, its queue entries are purged, and the requests sharing the queue
    with it still finish with exact results."""
    hard = synth.config_n10()
    small = synth.config_batched(count=12, seed=99, n_range=(2, 4))
    sv = B.Server(workspace_bytes=1 << 31, max_slots=32, wave_children=1 << 20, max_vars=10)
    try:
        t0 = time.time()
        th = sv.submit(hard, time_budget_s=0.3)
        ts = [sv.submit(s) for s in small]
        r_hard = wait_all(sv, [th], budget_s=60.0)[0]
        assert r_hard["status"] == 4                       # IVS_ERR_TIMEOUT
        assert time.time() - t0 < 10.0
        res = wait_all(sv, ts)
        for s, r in zip(small, res):
            assert same(r, B.solve(s))
        st = sv.stats()
        assert st["last_error"] == "" and st["in_flight"] == 0
        # the server keeps working after the purge
        again = wait_all(sv, [sv.submit(small[0])])[0]
        assert same(again, res[0])
    finally:
        sv.close()


@pytest.mark.parametrize("schedule", [0, 1])
def test_each_request_gets_its_share(B, schedule):
    """Every request in flight has its own queue region and a share of each sweep (the
    least served first, or equal shares): small requests interleaved with hard ones in
    one burst finish promptly and exactly while the hard ones run until their time
    budget."""
    hard = [synth.config_n10()] * 3
    small = synth.config_batched(count=12, seed=1212, n_range=(2, 4))
    sv = B.Server(workspace_bytes=1 << 31, max_slots=32, wave_children=1 << 20, max_vars=10, schedule=schedule)
    try:
        tickets, kinds = [], []
        for k, s in enumerate(small):
            if k % 4 == 0 and k // 4 < len(hard):
                tickets.append(sv.submit(hard[k // 4], time_budget_s=6.0))
                kinds.append("hard")
            tickets.append(sv.submit(s))
            kinds.append(k)
        t0 = time.time()
        done_small = {}
        for t, kind in zip(tickets, kinds):
            if kind == "hard":
                continue
            r = wait_all(sv, [t], budget_s=60.0)[0]
            done_small[kind] = (time.time() - t0, r)
        # all small requests finish well before the hard ones' budget runs out
        assert max(v[0] for v in done_small.values()) < 3.0, [round(v[0], 2) for v in done_small.values()]
        for k, (_, r) in done_small.items():
            assert same(r, B.solve(small[k])), k
        for t, kind in zip(tickets, kinds):
            if kind == "hard":
                assert wait_all(sv, [t], budget_s=60.0)[0]["status"] == 4
        assert sv.stats()["last_error"] == ""
    finally:
        sv.close()


def test_plans_on_another_thread_while_serving(B):
    """A server's captured sweep graph keeps working while other host threads build and run
    plans of other shapes (the kernels' shared-memory limits are raised once, never
    lowered)."""
    small = synth.config_batched(count=6, seed=6060, n_range=(2, 4))
    sv = B.Server(workspace_bytes=1 << 30, max_slots=64, wave_children=1 << 20, max_vars=10)
    try:
        th = sv.submit(synth.config_n10(), time_budget_s=2.0)
        for s in small:                      # plans on this thread meanwhile
            assert B.solve(s)["status"] == 0
        assert B.solve(synth.config_n6())["status"] == 0
        later = [sv.submit(s) for s in small]
        res = wait_all(sv, later)
        for s, r in zip(small, res):
            assert same(r, B.solve(s))
        assert wait_all(sv, [th])[0]["status"] == 4
        assert sv.stats()["last_error"] == ""
    finally:
        sv.close()


def test_served_options_per_request(B, orc):
    """Requests carry their own options: Krawczyk contraction, centred form, several
    sweeps per visit, mixed in one server with plain requests; each result equals the
    oracle's for its options, bit for bit."""
    systems = synth.config_batched(count=12, seed=4711, n_range=(2, 5))
    kinds = [dict(), dict(krawczyk=True), dict(centred_form=True), dict(krawczyk=True, hs_iters=3)]
    sv = B.Server(workspace_bytes=1 << 28, max_slots=16, wave_children=1 << 18, max_vars=8)
    try:
        tickets = [sv.submit(s, tol=1e-4, **kinds[i % 4]) for i, s in enumerate(systems)]
        results = wait_all(sv, tickets)
    finally:
        sv.close()
    for i, (s, r) in enumerate(zip(systems, results)):
        k = kinds[i % 4]
        o = orc.solve(s, tol=1e-4, krawczyk=k.get("krawczyk", False), centred=k.get("centred_form", False),
                      hs_iters=k.get("hs_iters", 1))
        assert same(r, o), i
