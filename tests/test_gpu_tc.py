"""GPU parity of the tensor-core direct-sum route (small cells, split binary16 MMAs) against the FP64 oracle.

Coefficients within relative l2 1e-5 per cell; EMS indices bit-exact against the oracle's ranking of the
same binary32 spectra; routing by sample count as the plan reports it.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import EMSParams as OEMS

pytestmark = pytest.mark.gpu

enufft = pytest.importorskip("paper_2606_21278_b300")


def _rel_l2(a, b):
    a = np.asarray(a).reshape(len(a), -1)
    b = np.asarray(b).reshape(len(b), -1)
    den = np.linalg.norm(b, axis=1)
    den[den == 0] = 1.0
    return np.linalg.norm(a - b, axis=1) / den


def _with_counts(wl, new_counts):
    """Keep the first new_counts[j] samples of every cell j (0 empties a cell)."""
    off = wl.offsets
    keep = torch.zeros(wl.n_points, dtype=torch.bool)
    for j, n in enumerate(new_counts):
        keep[int(off[j]):int(off[j]) + n] = True
    cnt = torch.tensor(new_counts, dtype=torch.int64)
    return synth.Workload(**{**wl.__dict__, "x": wl.x[keep], "y": wl.y[keep], "h": wl.h[keep], "w": wl.w[keep],
                             "offsets": torch.cat([torch.zeros(1, dtype=torch.int64), torch.cumsum(cnt, 0)])})


def _run(wl, **kw):
    g = wl.to("cuda")
    plan = enufft.Plan.for_workload(g, **kw)
    c, ks, sel, ret = plan.type1_ems(g.x, g.y, g.h, g.w)
    plan.sync_status()
    return plan, c.cpu().numpy(), ks.cpu().numpy(), sel.cpu().numpy()


def test_routing_splits_cells_and_both_routes_match_oracle():
    """tri81920 workload (threshold 3000 samples): cells at or below it take the tensor-core sum, the
    rest the fused spread/FFT kernel; every cell matches the oracle and EMS indices are exact."""
    wl = synth.make("tri81920_p64_mixed", seed=5, n_cells=20, q_scale=0.5)
    cnt = wl.counts()
    n_small = int((cnt <= wl.tc_max_points).sum())
    assert 0 < n_small < wl.n_cells
    plan, c, ks, sel = _run(wl)
    info = plan.info()
    assert info["cells_tensor"] == n_small and info["cells_fused"] == wl.n_cells - n_small
    assert info["kernels_per_type1_ems"] == 3
    err = _rel_l2(c, oracle.type1(wl))
    assert err.max() <= 1e-5, err
    oks, osel, _, _ = oracle.ems(c, OEMS(), energy_fp32=True)
    assert np.array_equal(ks, oks) and np.array_equal(sel, osel)


@pytest.mark.parametrize("modes", [64, 48, 32])
def test_all_cells_on_tensor_cores(modes):
    """Every cell routed to the tensor cores (threshold above every count), P = 64 and the padded
    feature slots of P = 48 and 32; ragged chunks, an empty cell and a one-sample cell."""
    wl = synth.make("tri20480_p64", seed=9, n_cells=7, q_scale=0.25)
    wl.modes = modes
    cnt = wl.counts().tolist()
    cnt[1] = 0
    cnt[2] = 1
    cnt[3] = 33      # one full chunk of 32 and one sample
    wl = _with_counts(wl, cnt)
    plan, c, ks, sel = _run(wl, tc_max_points=1 << 30)
    assert plan.info()["cells_tensor"] == wl.n_cells and plan.info()["cells_fused"] == 0
    assert np.abs(c[1]).max() == 0
    err = _rel_l2(c, oracle.type1(wl))
    assert err.max() <= 1e-5, err
    oks, osel, _, _ = oracle.ems(c, OEMS(), energy_fp32=True)
    assert np.array_equal(ks, oks) and np.array_equal(sel, osel)


@pytest.mark.parametrize("mask", [1, 2])
def test_tensor_core_route_masks(mask):
    wl = synth.make("hex4096_p48", seed=4, n_cells=5, q_scale=0.3)
    wl.mask = mask
    _, c, _, _ = _run(wl, tc_max_points=1 << 30)
    err = _rel_l2(c, oracle.type1(wl))
    assert err.max() <= 1e-5, err


def test_tensor_core_route_large_counts_and_weight_range():
    """Cells of 10,000+ samples (hundreds of chunks) and weights spanning 6 decades: the per-cell scale
    keeps the binary16 operands in range."""
    wl = synth.make("tri20480_p64", seed=12, n_cells=3, q_scale=3.0)
    gen = torch.Generator().manual_seed(1)
    wl.w = wl.w * torch.exp(torch.empty(wl.n_points).uniform_(-7.0, 7.0, generator=gen)).to(wl.w.dtype)
    _, c, _, _ = _run(wl, tc_max_points=1 << 30)
    err = _rel_l2(c, oracle.type1(wl))
    assert err.max() <= 1e-5, err


def test_tensor_core_route_nonfinite_sample_reported():
    wl = synth.make("tri20480_p64", seed=5, n_cells=3, q_scale=0.1)
    bad = int(wl.offsets[1]) + 3
    g = wl.to("cuda")
    g.y[bad] = float("inf")
    plan = enufft.Plan.for_workload(g, tc_max_points=1 << 30)
    c = plan.type1(g.x, g.y, g.h, g.w)
    with pytest.raises(enufft.EnufftError, match="non-finite"):
        plan.sync_status()
    keep = torch.ones(wl.n_points, dtype=torch.bool)
    keep[bad] = False
    wl2 = synth.Workload(**{**wl.__dict__, "x": wl.x[keep], "y": wl.y[keep], "h": wl.h[keep], "w": wl.w[keep],
                            "offsets": wl.offsets - (torch.arange(4) > 1).long()})
    assert _rel_l2(c.cpu().numpy(), oracle.type1(wl2)).max() <= 1e-5


def test_tensor_core_route_adjoint_covers_every_cell():
    """The adjoint runs for all cells of a plan with routed cells (gradient vs oracle)."""
    wl = synth.make("tri81920_p64_mixed", seed=6, n_cells=6, q_scale=0.4)
    g = wl.to("cuda")
    plan = enufft.Plan.for_workload(g)
    assert plan.info()["cells_tensor"] > 0
    rng = np.random.default_rng(0)
    G = rng.standard_normal((wl.n_cells, wl.modes, wl.modes)) + 1j * rng.standard_normal((wl.n_cells, wl.modes, wl.modes))
    gh, gw = plan.type1_backward(torch.tensor(G, dtype=plan.complex_dtype, device="cuda"), g.x, g.y, g.h, g.w)
    oh, ow = oracle.type1_backward(wl, G)
    for got, ref in ((gh, oh), (gw, ow)):
        got = got.cpu().double().numpy()
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


def test_tensor_core_route_rejected_where_not_built():
    wl = synth.make("tri1_q2000_p32_fp64", seed=0)
    g = wl.to("cuda")
    with pytest.raises(enufft.EnufftError, match="tensor-core"):
        enufft.Plan.for_workload(g, tc_max_points=100)


def test_bounded_wait_timeout_is_reported_and_the_context_stays_usable():
    """A wait that nothing completes gives up after its poll limit, latches the timeout bit, and the
    next sync reports ENUFFT_ERR_TIMEOUT; the plan then runs normally."""
    wl = synth.make("tri81920_p64_mixed", seed=2, n_cells=6, q_scale=0.4)
    g = wl.to("cuda")
    plan = enufft.Plan.for_workload(g)
    plan.selftest_wait_timeout(64)
    with pytest.raises(enufft.EnufftError, match="status 4.*bounded wait expired"):
        plan.sync_status()
    plan.sync_status()   # cleared once reported
    c = plan.type1(g.x, g.y, g.h, g.w)
    plan.sync_status()
    assert _rel_l2(c.cpu().numpy(), oracle.type1(wl)).max() <= 1e-5
