"""The benchmarked step (type-1 + EMS) captured in a CUDA graph and replayed: the calls issue only
stream-ordered work (no host synchronisation), so a replay reproduces the eager result exactly --
through a caller-owned torch graph and through the plan's own graph (enufft_type1_ems_graph)."""
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

enufft = pytest.importorskip("paper_2606_21278_b300")


@pytest.mark.parametrize("name,n,qs", [("tri81920_p64_mixed", 40, 0.5), ("mixed2560_p128", 6, 0.01)])
def test_type1_ems_graph_replay_matches_eager(name, n, qs):
    wl = synth.make(name, seed=8, n_cells=n, q_scale=qs).to("cuda")
    plan = enufft.Plan.for_workload(wl)
    info = plan.info()
    prm = enufft.EMSParams()
    ref = plan.type1_ems(wl.x, wl.y, wl.h, wl.w, prm)
    torch.cuda.synchronize()
    plan.sync_status()
    coeffs = plan.new_coeffs()
    out = (torch.empty_like(ref[1]), torch.empty_like(ref[2]), torch.empty_like(ref[3]))
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):   # warm-up on a side stream before capture
        plan.type1_ems(wl.x, wl.y, wl.h, wl.w, prm, coeffs=coeffs, out=out)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        plan.type1_ems(wl.x, wl.y, wl.h, wl.w, prm, coeffs=coeffs, out=out)
    for t in (coeffs,) + out:
        t.zero_()
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    plan.sync_status()
    # every route is bit-reproducible: integer spreading sums, fixed-order reductions elsewhere
    assert torch.equal(coeffs, ref[0])
    assert torch.equal(out[0], ref[1]) and torch.equal(out[1], ref[2]) and torch.equal(out[2], ref[3])


@pytest.mark.parametrize("name,n,qs", [("tri81920_p64_mixed", 40, 0.5), ("mixed2560_p128", 4, 0.01)])
def test_plan_owned_graph(name, n, qs):
    """The plan's graph replays the eager result, follows new buffer contents, and is captured again
    when an output buffer or an EMS parameter changes."""
    wl = synth.make(name, seed=9, n_cells=n, q_scale=qs).to("cuda")
    plan = enufft.Plan.for_workload(wl)
    prm = enufft.EMSParams()
    ref = plan.type1_ems(wl.x, wl.y, wl.h, wl.w, prm)
    coeffs = plan.new_coeffs()
    out = (torch.empty_like(ref[1]), torch.empty_like(ref[2]), torch.empty_like(ref[3]))
    for _ in range(3):
        plan.type1_ems_graph(wl.x, wl.y, wl.h, wl.w, coeffs, out, prm)
    torch.cuda.synchronize()
    plan.sync_status()
    assert torch.equal(coeffs, ref[0]) and torch.equal(out[0], ref[1]) and torch.equal(out[1], ref[2])
    assert torch.equal(out[2], ref[3])
    # new contents of the captured input buffer: the replay reads them
    h2 = wl.h * 0.5 + 3.0
    ref2 = plan.type1_ems(wl.x, wl.y, h2, wl.w, prm)
    wl.h.copy_(h2)
    plan.type1_ems_graph(wl.x, wl.y, wl.h, wl.w, coeffs, out, prm)
    torch.cuda.synchronize()
    assert torch.equal(coeffs, ref2[0]) and torch.equal(out[0], ref2[1]) and torch.equal(out[2], ref2[3])
    # other output buffers and another K_max: captured again
    prm3 = enufft.EMSParams(k_max=6)
    ref3 = plan.type1_ems(wl.x, wl.y, wl.h, wl.w, prm3)
    coeffs3 = plan.new_coeffs()
    out3 = (torch.empty_like(ref3[1]), torch.empty_like(ref3[2]), torch.empty_like(ref3[3]))
    plan.type1_ems_graph(wl.x, wl.y, wl.h, wl.w, coeffs3, out3, prm3)
    torch.cuda.synchronize()
    plan.sync_status()
    assert torch.equal(coeffs3, ref3[0]) and torch.equal(out3[1], ref3[2]) and torch.equal(out3[2], ref3[3])
