"""Route tuning at plan creation (opts.autotune, enufft_get_tuning): the tuned plan reports a threshold
taken from the measured ladder and a fused-kernel grid, gives the oracle's coefficients and EMS
selection on whichever route each cell took, and a second plan with the same cache file reads the
record instead of measuring.  For n_f = 256 plans the tuner picks the tile side of the sorted
spreading, and every side gives the oracle's result."""
import json

import numpy as np
import pytest

import oracle
import synth
from oracle import EMSParams as OEMS

pytestmark = pytest.mark.gpu

enufft = pytest.importorskip("paper_2606_21278_b300")


def test_autotuned_plan_matches_oracle_and_caches(tmp_path):
    cache = str(tmp_path / "tune.json")
    wl = synth.make("tri81920_p64_mixed", seed=4, n_cells=48, q_scale=0.4)   # cells from 200 to ~20000 samples
    g = wl.to("cuda")
    plan = enufft.Plan.for_workload(g, autotune=True, tune_cache=cache)
    info = plan.info()
    t = plan.tuning()
    assert info["autotuned"] == 1 and not t["from_cache"]
    assert t["ladder"] == [128, 256, 512, 1024, 2048]          # the sizes not above the cap of 3000
    assert all(v > 0 for v in t["ns_fused"] + t["ns_tc"])
    assert info["tc_max_points"] == t["tc_max_points"] and t["tc_max_points"] in [0] + t["ladder"]
    expect_tc = int((wl.counts() <= t["tc_max_points"]).sum()) if t["tc_max_points"] else 0
    assert info["cells_tensor"] == expect_tc and info["cells_fused"] == wl.n_cells - expect_tc
    assert info["fused_blocks_per_sm"] == t["fused_blocks_per_sm"] in (1, 2)
    c, ks, sel, _ = plan.type1_ems(g.x, g.y, g.h, g.w)
    plan.sync_status()
    cn = c.cpu().numpy()
    ref = oracle.type1(wl)
    err = np.linalg.norm((cn - ref).reshape(wl.n_cells, -1), axis=1) / np.linalg.norm(ref.reshape(wl.n_cells, -1), axis=1)
    assert err.max() <= 1e-5, err
    oks, osel, _, _ = oracle.ems(cn, OEMS(), energy_fp32=True)
    assert np.array_equal(ks.cpu().numpy(), oks) and np.array_equal(sel.cpu().numpy(), osel)
    plan2 = enufft.Plan.for_workload(g, autotune=True, tune_cache=cache)
    t2 = plan2.tuning()
    assert t2["from_cache"] and t2["tc_max_points"] == t["tc_max_points"] and t2["ladder"] == t["ladder"]
    assert plan2.info()["cells_tensor"] == info["cells_tensor"]


def test_autotune_without_tensor_core_cap_tunes_the_grid_only():
    wl = synth.make("tri20480_p64", seed=5, n_cells=64, q_scale=0.3).to("cuda")
    plan = enufft.Plan.for_workload(wl, autotune=True)
    t = plan.tuning()
    assert t["ladder"] == [] and t["tc_max_points"] == 0 and plan.info()["cells_tensor"] == 0
    assert plan.info()["fused_blocks_per_sm"] == t["fused_blocks_per_sm"]


def _large_workload():
    # n_f = 256 cells (P = 128) of about 1,200 to 20,000 samples: several sort blocks per cell
    return synth.make("mixed2560_p128", seed=6, n_cells=6, q_scale=0.012)


def test_large_route_tile_tuning_and_every_tile_side_matches_oracle(tmp_path):
    cache = str(tmp_path / "tune.json")
    wl = _large_workload()
    g = wl.to("cuda")
    plan = enufft.Plan.for_workload(g, autotune=True, tune_cache=cache)
    info, t = plan.info(), plan.tuning()
    assert info["cells_large"] == wl.n_cells and info["autotuned"] == 1 and not t["from_cache"]
    assert t["ladder"] == [16, 32, 64] and all(v > 0 for v in t["ns_fused"])
    assert t["large_tile"] == t["ladder"][int(np.argmin(t["ns_fused"]))] == info["large_tile"]
    ref = oracle.type1(wl)
    (key,) = json.load(open(cache)).keys()
    for side in (16, 32, 64):   # each side through the cache record
        d = json.load(open(cache))
        d[key]["large_tile"] = side
        json.dump(d, open(cache, "w"))
        p2 = enufft.Plan.for_workload(g, autotune=True, tune_cache=cache)
        assert p2.tuning()["from_cache"] and p2.info()["large_tile"] == side
        c, ks, sel, _ = p2.type1_ems(g.x, g.y, g.h, g.w)
        p2.sync_status()
        cn = c.cpu().numpy()
        err = np.linalg.norm((cn - ref).reshape(wl.n_cells, -1), axis=1) / np.linalg.norm(ref.reshape(wl.n_cells, -1), axis=1)
        assert err.max() <= 1e-5, (side, err)
        oks, osel, _, _ = oracle.ems(cn, OEMS(), energy_fp32=True)
        assert np.array_equal(ks.cpu().numpy(), oks) and np.array_equal(sel.cpu().numpy(), osel)


def test_large_route_default_tile_without_tuning():
    g = _large_workload().to("cuda")
    plan = enufft.Plan.for_workload(g)
    assert plan.info()["large_tile"] == 32 and plan.info()["autotuned"] == 0
