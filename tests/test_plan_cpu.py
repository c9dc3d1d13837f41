"""The launch planner on the host (no GPU): pm_plan_for_device on host-only
sets, for a GB300-shaped device (152 SMs, 227 KB of dynamic shared memory
per block, 228 KB per SM) and a small one. Checks the budgets every plan
must keep and the choices the planner documents: the whole table in shared
memory where it fits, late terminal ids when the whole id structure does
not fit beside it at 20 or more warps, pinned parameters obeyed, PFAC at 24
warps, at most 16 warps where the 768-thread kernels do not apply."""
import numpy as np
import pytest

from paper_1407_2889_gb300 import pmscan as pm, synth

GB300 = (152, 232448, 233472)
SMALL = (16, 49152, 102400)


@pytest.fixture(scope="module")
def est_text():
    return synth.est_text(4 << 20, 1)


def _plan(P, device, algo="ac", **params):
    make = pm.PatternSet.pfac if algo == "pfac" else pm.PatternSet.ac
    s = make(P, dict(params, host_only=1))
    try:
        return s.plan_for(*device)
    finally:
        s.close()


def _within_budget(plan, device):
    _, optin, per_sm = device
    for key in ("smem_bytes", "smem_bytes_list"):
        assert 0 < plan[key] <= optin - 1024, (key, plan)
    if plan["placement"] == pm.PM_PLACE_SMEM:
        assert (plan["smem_bytes"] + 1024) * plan["ctas_per_sm"] <= per_sm, plan


@pytest.mark.parametrize("d,m", [(1000, 8), (8000, 8), (20000, 8), (1000, 16), (1000, 32), (8000, 16)])
@pytest.mark.parametrize("device", [GB300, SMALL])
def test_every_plan_keeps_its_budgets(est_text, d, m, device):
    _, P = synth.est_case(d, m, text=est_text)
    for params in ({}, {"warps_per_cta": 16}, {"warps_per_cta": 8}, {"ids_place": 1, "counters": 1},
                   {"ids_place": 3}, {"counters": 2}, {"placement": pm.PM_PLACE_HYBRID}):
        try:
            plan = _plan(P, device, **params)
        except pm.PmError as e:
            # a 48 KB device cannot hold 16 warps' text buffers and pools (a
            # hybrid plan keeps 16 unless pinned): no plan, said so
            assert device == SMALL and e.code == pm.PM_ETOOBIG, (params, e)
            continue
        _within_budget(plan, device)
        assert 1 <= plan["warps"] <= 24 and 1 <= plan["warps_list"] <= 24, plan
        if params.get("warps_per_cta"):
            assert plan["warps"] == plan["warps_list"] == min(params["warps_per_cta"], 24)


def test_headline_set_takes_late_ids_at_24_warps(est_text):
    """d=8000, m=8: the whole id structure and 32-bit counters fit beside
    the table only up to 17 warps, so the first pass takes late ids; its
    list mode runs 24 warps with the whole table in shared memory."""
    _, P = synth.est_case(8000, 8, text=est_text)
    plan = _plan(P, GB300)
    assert plan["placement"] == pm.PM_PLACE_SMEM
    assert plan["ids_place"] == 3 and plan["warps_list"] == 24
    assert plan["warps"] >= 20 and plan["counters"] in (1, 2)
    # pinned parameters are obeyed: everything in shared memory at the most
    # warps that fit (the plan the first pass turns down)
    pinned = _plan(P, GB300, ids_place=1, counters=1)
    assert (pinned["ids_place"], pinned["counters"]) == (1, 1)
    assert 16 <= pinned["warps"] == pinned["warps_list"] < 20
    sixteen = _plan(P, GB300, warps_per_cta=16)
    assert sixteen["ids_place"] == 1 and sixteen["warps"] == 16


def test_small_set_keeps_everything_in_shared_memory(est_text):
    _, P = synth.est_case(1000, 8, text=est_text)
    plan = _plan(P, GB300)
    assert plan["placement"] == pm.PM_PLACE_SMEM
    assert (plan["ids_place"], plan["counters"]) == (1, 1)
    assert plan["warps"] == plan["warps_list"] == 24


def test_large_tables_go_hybrid_and_a_small_device_too(est_text):
    _, P = synth.est_case(8000, 16, text=est_text)
    plan = _plan(P, GB300)
    assert plan["placement"] == pm.PM_PLACE_HYBRID and plan["warps"] == 16
    assert 0 < plan["smem_rows"]
    # an 89 KB table on a 48 KB device: a table prefix at pinned warps (a
    # hybrid plan keeps 16 warps unless pinned, and 16 warps' buffers alone
    # exceed 48 KB, which the planner reports)
    _, P = synth.est_case(8000, 8, text=est_text)
    with pytest.raises(pm.PmError) as e:
        _plan(P, SMALL)
    assert e.value.code == pm.PM_ETOOBIG
    small = _plan(P, SMALL, warps_per_cta=4)
    assert small["placement"] == pm.PM_PLACE_HYBRID and small["warps"] == 4
    _within_budget(small, SMALL)
    full = _plan(P, GB300)
    assert 0 < small["smem_rows"] < full["smem_rows"]
    glob = _plan(P, GB300, placement=pm.PM_PLACE_GLOBAL)
    assert glob["placement"] == pm.PM_PLACE_GLOBAL and glob["smem_rows"] == 0


def test_pfac_runs_24_warps(est_text):
    _, P = synth.est_case(8000, 8, text=est_text)
    plan = _plan(P, GB300, algo="pfac")
    assert plan["warps"] == plan["warps_list"] == 24
    assert plan["ids_place"] != 3  # late ids are not offered to PFAC sets


def test_wide_kernels_only_where_they_apply(est_text):
    """More than 16 warps only for ACGT-like tables at one CTA per SM."""
    rng = np.random.default_rng(7)
    P = rng.integers(ord("a"), ord("z") + 1, size=(500, 8), dtype=np.uint8)
    plan = _plan(P, GB300)
    assert plan["warps"] <= 16 and plan["warps_list"] <= 16
    assert _plan(P, GB300, warps_per_cta=24)["warps"] == 16
    _, P = synth.est_case(1000, 8, text=est_text)
    two = _plan(P, GB300, ctas_per_sm=2)
    assert two["ctas_per_sm"] == 2 and two["warps"] <= 16


def test_bad_arguments():
    P = np.frombuffer(b"ACGTACGT", np.uint8).reshape(1, 8)
    s = pm.PatternSet.ac(P, {"host_only": 1})
    for dev in ((0, 232448, 233472), (152, 0, 233472), (152, 232448, -1)):
        with pytest.raises(pm.PmError) as e:
            s.plan_for(*dev)
        assert e.value.code == pm.PM_EINVAL
    s.close()
    w = pm.PatternSet.wm(P, 2, {"host_only": 1})
    with pytest.raises(pm.PmError) as e:
        w.plan_for(*GB300)
    assert e.value.code == pm.PM_EINVAL
    w.close()
