"""Solve service (labs_serve_*): continuous batching.  Requests submitted
while others run are admitted as slots free up, and every result equals
the run of the same instance alone (labs_mts_launch) and the oracle's,
whatever the mix, the quantum size or the memory budget.  Failure paths
(cancel, full queue, unknown ticket, quantum timeout) are driven from the
host; no GPU fault is involved."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def labs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2504_00987_gb300 as labs

    return labs


def wait_all(srv, tickets, timeout=180.0):
    out = {}
    deadline = time.time() + timeout
    while len(out) < len(tickets):
        assert time.time() < deadline, f"{len(tickets) - len(out)} requests still pending"
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = r
        time.sleep(0.001)
    return [out[t] for t in tickets]


def random_requests(labs, count, seed, max_n=160, max_k=100, steps=(500, 20_000)):
    rng = np.random.default_rng(seed)
    Ns = rng.integers(32, max_n + 1, count)
    Ks = rng.integers(10, max_k + 1, count)
    Ss = rng.integers(steps[0], steps[1], count)
    return [labs.make_instance(int(N), int(K), seed=seed, instance=i, max_steps=int(S))
            for i, (N, K, S) in enumerate(zip(Ns, Ks, Ss))]


def alone(labs, r):
    P = labs.make_params(r.N, r.K, max_steps=r.max_steps, target_E=r.target_E,
                         max_generations=r.max_generations)
    return labs.decode_results(labs.mts_launch(P, r.seed, r.instance, 1), r.N, r.instance)[0]


def same(a, b):
    return (a["E"], a["seq"], a["steps"], a["generations"], a["status"]) == \
        (b["E"], b["seq"], b["steps"], b["generations"], b["status"])


def test_mix_equals_alone_and_oracle(labs, orc):
    reqs = random_requests(labs, 150, seed=21)
    with labs.Server(max_slots=64, max_N=160, max_K=100, quantum_steps=300) as srv:
        tickets = []
        for i, r in enumerate(reqs):
            tickets.append(srv.submit(r))
            if i % 10 == 9:
                time.sleep(0.003)  # later requests arrive while earlier quanta run
        res = wait_all(srv, tickets)
        st = srv.stats()
    assert st["completed"] == 150 and st["quanta"] > 1 and st["failed"] == 0
    for r, g in zip(reqs, res):
        assert same(g, alone(labs, r))
        assert g["seconds"] > 0
    for r, g in list(zip(reqs, res))[::15]:
        o, _, _ = orc.mts_run(orc.make_params(r.N, r.K, max_steps=r.max_steps), r.seed, r.instance)
        assert g["E"] == o["E"] and g["seq"] == [int(x) for x in o["seq"]] and g["steps"] == o["steps"]


def test_quantum_size_and_budget_do_not_change_results(labs):
    reqs = random_requests(labs, 40, seed=4, steps=(100, 6000))
    outs = []
    for q, budget in ((1, 0), (100_000, 0), (997, 40_000)):
        with labs.Server(max_slots=16, max_N=160, max_K=100, quantum_steps=q,
                         hbm_budget_bytes=budget) as srv:
            outs.append(wait_all(srv, [srv.submit(r) for r in reqs]))
    for a, b, c in zip(*outs):
        assert same(a, b) and same(a, c)


def test_time_budget_quanta_do_not_change_results(labs):
    """Quanta ended by a device-time budget (slots of every N suspend at the
    first generation boundary past it) give the results of step quanta."""
    reqs = random_requests(labs, 40, seed=33, steps=(1000, 30_000))
    outs = []
    for kw in (dict(quantum_steps=500), dict(quantum_steps=1 << 40, quantum_us=300),
               dict(quantum_steps=1 << 40, quantum_us=3000)):
        with labs.Server(max_slots=12, max_N=160, max_K=100, **kw) as srv:
            outs.append(wait_all(srv, [srv.submit(r) for r in reqs]))
            st = srv.stats()
        assert st["completed"] == 40 and st["failed"] == 0
    for a, b, c in zip(*outs):
        assert same(a, b) and same(a, c)


def test_target_requests_stop_on_target(labs):
    reqs = [labs.make_instance(40, 50, seed=3, instance=i, target_E=140, max_steps=2_000_000)
            for i in range(12)]
    with labs.Server(max_slots=8, max_N=64, max_K=64, quantum_steps=500) as srv:
        res = wait_all(srv, [srv.submit(r) for r in reqs])
    for r, g in zip(reqs, res):
        assert g["status"] == labs.RUN_REACHED and g["E"] <= 140
        assert same(g, alone(labs, r))


def test_cancel_busy_and_unknown(labs):
    from paper_2504_00987_gb300 import _native as nat

    long_req = [labs.make_instance(160, 100, seed=1, instance=i, max_steps=3_000_000) for i in range(3)]
    with labs.Server(max_slots=1, max_N=160, max_K=100, quantum_steps=200, queue_capacity=2) as srv:
        t0 = srv.submit(long_req[0])
        time.sleep(0.05)  # t0 is admitted into the only slot
        t1 = srv.submit(long_req[1])
        t2 = srv.submit(long_req[2])
        with pytest.raises(labs.LabsError) as ei:
            srv.submit(long_req[0])
        assert ei.value.code == nat.LABS_EBUSY
        srv.cancel(t1)  # pending
        srv.cancel(t0)  # running: leaves at the next quantum boundary
        srv.cancel(t2)
        for t in (t0, t1, t2):
            deadline = time.time() + 30
            while True:
                try:
                    srv.poll(t)
                except labs.LabsError as e:
                    assert e.code == nat.LABS_ECANCELED
                    break
                assert time.time() < deadline
                time.sleep(0.002)
        with pytest.raises(labs.LabsError) as ei:
            srv.poll(12345)
        assert ei.value.code == nat.LABS_ENOTFOUND
        with pytest.raises(labs.LabsError) as ei:
            srv.submit(labs.make_instance(200, 10, max_steps=10))  # beyond max_N
        assert ei.value.code == nat.LABS_EINVAL
        assert srv.stats()["canceled"] == 3


def test_quantum_timeout_fails_the_server_cleanly(labs):
    """A quantum that outlives quantum_timeout_ms stops the server with
    LABS_ETIMEOUT on the host; the launch itself is bounded and finishes,
    and destroy waits for it."""
    from paper_2504_00987_gb300 import _native as nat

    srv = labs.Server(max_slots=4, max_N=160, max_K=100, quantum_steps=1_000_000, quantum_timeout_ms=1)
    t = srv.submit(labs.make_instance(160, 100, seed=2, max_steps=400_000))
    deadline = time.time() + 60
    while True:
        try:
            srv.poll(t)
        except labs.LabsError as e:
            assert e.code == nat.LABS_ETIMEOUT
            break
        assert time.time() < deadline
        time.sleep(0.005)
    assert srv.stats()["failed"] == nat.LABS_ETIMEOUT
    with pytest.raises(labs.LabsError):
        srv.submit(labs.make_instance(40, 10, max_steps=10))
    srv.close()
    # the device is still usable afterwards
    P = labs.make_params(40, 10, max_steps=100)
    assert labs.mts_run(P, 0, 0, 2)[0]["steps"] == 100


def test_admission_waits_for_arena_memory(labs):
    """A request waits for arena memory, not for a slot: the arena holds one
    N = 64, K = 100 population (K (nw + 1) 4 = 1,200 bytes, nw = 2) and there
    are 8 slots, so the three requests run one after another; each result is
    its run alone."""
    reqs = [labs.make_instance(64, 100, seed=9, instance=i, max_steps=3000) for i in range(3)]
    with labs.Server(max_slots=8, max_N=64, max_K=100, quantum_steps=200, hbm_budget_bytes=1216) as srv:
        res = wait_all(srv, [srv.submit(r) for r in reqs])
        st = srv.stats()
    assert st["completed"] == 3 and st["failed"] == 0
    assert st["deferred_hbm"] >= 1 and st["deferred_slots"] == 0 and st["deferred_smem"] == 0
    assert st["arena_bytes"] == 1216 and st["arena_used_bytes"] == 0
    for r, g in zip(reqs, res):
        assert same(g, alone(labs, r))


def test_arena_smaller_than_one_request_is_refused(labs):
    with pytest.raises(labs.LabsError):
        labs.Server(max_slots=8, max_N=64, max_K=100, hbm_budget_bytes=1000)


def test_admission_waits_for_shared_memory(labs):
    """With populations of up to K = 1024, the 256-bit class's quantum kernel
    keeps few warps resident per SM; requests beyond one resident wave wait in
    the queue (held by shared memory, not by slots or arena) and all finish
    with their results alone.  A 64-bit request shares the wave by fraction."""
    reqs = [labs.make_instance(256, 2, seed=5, instance=i, max_steps=3000) for i in range(1500)]
    reqs.append(labs.make_instance(64, 50, seed=5, instance=9999, max_steps=5000))
    with labs.Server(max_slots=4096, max_N=256, max_K=1024, quantum_steps=500) as srv:
        res = wait_all(srv, [srv.submit(r) for r in reqs], timeout=300.0)
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["deferred_smem"] >= 1 and st["deferred_slots"] == 0 and st["deferred_hbm"] == 0
    for r, g in list(zip(reqs, res))[::97] + [(reqs[-1], res[-1])]:
        assert same(g, alone(labs, r))


def test_warp_pairs_do_not_change_results(labs, orc):
    """Quanta that run requests on two warps (warps_per_request = 2, taken
    whenever the active requests fit one resident wave that way) give the
    results of one warp per request, of the run alone and of the oracle --
    with device-time quanta, so the pair's shared suspension decision is
    exercised too."""
    reqs = random_requests(labs, 60, seed=45, max_n=256, steps=(500, 12_000))
    outs, stats = [], []
    for wpr, kw in ((1, dict(quantum_steps=700)), (2, dict(quantum_steps=700)),
                    (2, dict(quantum_steps=1 << 40, quantum_us=400))):
        with labs.Server(max_slots=24, max_N=256, max_K=100, warps_per_request=wpr, **kw) as srv:
            outs.append(wait_all(srv, [srv.submit(r) for r in reqs]))
            stats.append(srv.stats())
    assert stats[0]["pair_quanta"] == 0 and stats[1]["pair_quanta"] > 0 and stats[2]["pair_quanta"] > 0
    for st in stats:
        assert st["completed"] == 60 and st["failed"] == 0
    for a, b, c in zip(*outs):
        assert same(a, b) and same(a, c) and a["status"] == labs.RUN_BUDGET
    for r, g in list(zip(reqs, outs[1]))[::12]:
        assert same(g, alone(labs, r))
        o, _, _ = orc.mts_run(orc.make_params(r.N, r.K, max_steps=r.max_steps), r.seed, r.instance)
        assert g["E"] == o["E"] and g["seq"] == [int(x) for x in o["seq"]]
