"""Batched uneven instances in one persistent launch (labs_batch_*): every
instance equals the oracle's run of that instance, whatever the mapping,
queue order or relaunch."""
import os
from concurrent.futures import ThreadPoolExecutor

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


def to_instances(labs, wl_list):
    return [labs.make_instance(x.N, x.K, seed=x.seed, instance=x.instance, max_steps=x.max_steps,
                               target_E=x.target_E) for x in wl_list]


def oracle_results(orc, wl_list):
    def one(x):
        P = orc.make_params(x.N, x.K, max_steps=x.max_steps, target_E=x.target_E)
        return orc.mts_run(P, x.seed, x.instance)[0]

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        return list(ex.map(one, wl_list))


def assert_same(gpu, ora):
    assert gpu["E"] == ora["E"]
    assert gpu["seq"] == [int(v) for v in ora["seq"]]
    assert gpu["steps"] == ora["steps"] and gpu["generations"] == ora["generations"]
    assert gpu["status"] == ora["status"]


def test_uneven_512_equals_oracle(labs, orc):
    """512 instances, N ~ U{40..127}, K ~ U{50..200}, budget 10 N^2 steps, one
    autotuned persistent launch: every instance equals the oracle."""
    from paper_2504_00987_gb300 import workloads

    wl_list = workloads.uneven_batch(512, seed=7, steps_per_n2=10)
    inst = to_instances(labs, wl_list)
    with labs.Batch(inst) as b:
        b.launch()
        got = b.results()
        mapping = b.mapping
    assert mapping["warps_per_block"] in (1, 2, 4, 8) and mapping["blocks_per_sm"] >= 1
    assert mapping["warps_per_seq"] in (1, 2)
    ora = oracle_results(orc, wl_list)
    for g, o, x in zip(got, ora, wl_list):
        assert g["N"] == x.N and g["instance"] == x.instance
        assert_same(g, o)
        assert g["steps"] == x.max_steps
    # the same 512 on two warps per replica (whichever mapping the tuner chose)
    other = 2 if mapping["warps_per_seq"] == 1 else 1
    got2 = labs.mts_batch_run(inst, mapping={"warps_per_block": 4, "blocks_per_sm": 2, "order": 0,
                                             "warps_per_seq": other})
    for g, o in zip(got2, ora):
        assert_same(g, o)


def test_mapping_and_order_do_not_change_results(labs):
    from paper_2504_00987_gb300 import workloads

    wl_list = workloads.uneven_batch(96, seed=3, steps_per_n2=2)
    inst = to_instances(labs, wl_list)
    ref = labs.mts_batch_run(inst, mapping={"warps_per_block": 4, "blocks_per_sm": 1, "order": 0})
    for m in ({"warps_per_block": 1, "blocks_per_sm": 1, "order": 1},
              {"warps_per_block": 8, "blocks_per_sm": 2, "order": 0},
              {"warps_per_block": 2, "blocks_per_sm": 4, "order": 1},
              {"warps_per_block": 2, "blocks_per_sm": 1, "order": 0, "warps_per_seq": 2},
              {"warps_per_block": 4, "blocks_per_sm": 3, "order": 1, "warps_per_seq": 2},
              {"warps_per_block": 8, "blocks_per_sm": 1, "order": 0, "warps_per_seq": 2}):
        got = labs.mts_batch_run(inst, mapping=m)
        for a, b in zip(ref, got):
            assert a["E"] == b["E"] and a["seq"] == b["seq"] and a["steps"] == b["steps"]
            assert a["status"] == b["status"] == labs.RUN_BUDGET


def test_relaunch_and_single_instance_equivalence(labs):
    """A graph relaunch recomputes the same results; a batch instance equals
    the same instance run alone through labs_mts_launch."""
    inst = [labs.make_instance(N, K, seed=11, instance=i, max_steps=5000)
            for i, (N, K) in enumerate([(40, 50), (64, 100), (65, 70), (127, 200), (100, 33)])]
    with labs.Batch(inst, mapping={"warps_per_block": 4, "blocks_per_sm": 1, "order": 0}) as b:
        b.launch()
        first = b.results()
        b.launch()
        second = b.results()
    assert first == second
    for i, x in enumerate(inst):
        P = labs.make_params(x.N, x.K, max_steps=5000)
        alone = labs.decode_results(labs.mts_launch(P, 11, i, 1), x.N, i)[0]
        assert alone["E"] == first[i]["E"] and alone["seq"] == first[i]["seq"]


@pytest.mark.parametrize("wps", [1, 2])
def test_mixed_widths_up_to_256(labs, orc, wps):
    wl = []
    from paper_2504_00987_gb300.workloads import Instance

    for i, (N, K) in enumerate([(3, 2), (64, 10), (65, 10), (128, 8), (129, 6), (192, 5), (193, 4), (256, 3)]):
        wl.append(Instance(N, K, 5, 100 + i, 600))
    got = labs.mts_batch_run(to_instances(labs, wl), mapping={"warps_per_block": 2, "blocks_per_sm": 1,
                                                              "order": 0, "warps_per_seq": wps})
    for g, o in zip(got, oracle_results(orc, wl)):
        assert_same(g, o)


def test_two_warps_per_replica_with_targets_variants_and_ties(labs, orc):
    """Two warps per replica on the decisions that cross the pair: targets
    (the replica stops mid-run), s_1 = +1 (bit 0 never moves, in the lower
    half), replace-worst, small N where ties for the minimum are frequent,
    and every word count."""
    from paper_2504_00987_gb300.workloads import Instance

    wl = [Instance(N, K, 8, i, 3000, target_E=t) for i, (N, K, t) in
          enumerate([(5, 3, -1), (9, 4, -1), (13, 10, 14), (40, 20, 108), (70, 12, -1), (100, 30, -1),
                     (150, 8, -1), (200, 5, -1), (256, 4, -1)])]
    inst = to_instances(labs, wl)
    m2 = {"warps_per_block": 4, "blocks_per_sm": 1, "order": 0, "warps_per_seq": 2}
    for g, o in zip(labs.mts_batch_run(inst, mapping=m2), oracle_results(orc, wl)):
        assert_same(g, o)
    for variant, policy in ((2, 0), (1, 1), (3, 1)):
        inst = [labs.make_instance(x.N, x.K, seed=8, instance=x.instance, max_steps=3000, variant=variant,
                                   replace_policy=policy) for x in wl]
        got = labs.mts_batch_run(inst, mapping=m2)
        for g, x in zip(got, wl):
            o, _, _ = orc.mts_run(orc.make_params(x.N, x.K, max_steps=3000, variant=variant,
                                                  replace_policy=policy), 8, x.instance)
            assert_same(g, o)


def test_mapping_errors(labs):
    inst = [labs.make_instance(40, 10, max_steps=100)]
    for bad in ({"warps_per_block": 1, "blocks_per_sm": 1, "warps_per_seq": 2},
                {"warps_per_block": 4, "blocks_per_sm": 1, "warps_per_seq": 3}):
        with pytest.raises(labs.LabsError):
            labs.mts_batch_run(inst, mapping=bad)


def test_batch_with_targets_and_generation_budgets(labs, orc):
    from paper_2504_00987_gb300.workloads import Instance

    wl = [Instance(30, 20, 2, i, 4000, target_E=90 - i) for i in range(8)]
    got = labs.mts_batch_run(to_instances(labs, wl))
    for g, o in zip(got, oracle_results(orc, wl)):
        assert_same(g, o)
    inst = [labs.make_instance(50, 16, seed=1, instance=i, max_generations=7) for i in range(4)]
    got = labs.mts_batch_run(inst)
    for i, g in enumerate(got):
        o, _, _ = orc.mts_run(orc.make_params(50, 16, max_generations=7), 1, i)
        assert_same(g, o)


def test_batch_errors(labs):
    bad = [labs.make_instance(64, 100, max_steps=100), labs.make_instance(64, 100)]  # second unbounded
    with pytest.raises(labs.LabsError) as ei:
        labs.mts_batch_run(bad)
    assert "instance 1" in str(ei.value)
    assert labs.mts_batch_run([]) == []
