"""GPU parity of the Voronoi quadrature weights (enufft_voronoi_weights) against the oracle.  The
nearest-sample decisions are integers taken from binary32 arithmetic on both sides in the same
operation order, so the counts agree exactly; the weights then agree to the last bit (up to one unit
of binary32 rounding through |D|)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

enufft = pytest.importorskip("paper_2606_21278_b300")


def _close(got, ref):
    rel = np.abs(got.astype(np.float64) - ref.astype(np.float64)) / np.maximum(np.abs(ref.astype(np.float64)), 1e-30)
    return rel.max() <= 1.2e-7   # one binary32 rounding; a count off by one moves a weight by >= 1/n_q


@pytest.mark.parametrize("name,n,qs,mask,ng", [("tri20480_p64", 6, 0.1, 0, 64), ("hex4096_p48", 4, 0.1, 0, 48),
                                               ("tri20480_p64", 3, 0.1, 1, 40), ("hex4096_p48", 3, 0.1, 2, 64),
                                               ("tri20480_p64", 2, 0.6, 0, 96),
                                               ("tri20480_p64", 2, 7.0, 0, 32)])   # > 16384 windowed samples
def test_voronoi_weights_match_oracle(name, n, qs, mask, ng):
    wl = synth.make(name, seed=12, n_cells=n, q_scale=qs)
    wl.mask = mask
    g = wl.to("cuda")
    plan = enufft.Plan.for_workload(g)
    w = plan.voronoi_weights(g.x, g.y, ng)
    plan.sync_status()
    ow, cnt = oracle.voronoi_weights(wl, ng)
    assert _close(w.cpu().numpy(), ow)
    off = wl.offsets.numpy()
    for j in range(n):
        area = oracle.frame(int(wl.nverts[j]), wl.verts[j], wl.eta, wl.mask)["area"]
        assert abs(w[off[j]:off[j + 1]].double().sum().item() - area) < 1e-5 * area


def test_voronoi_weights_feed_the_transform():
    """Clustered samples (Sec. A's case for Voronoi weights): the transform with the GPU weights equals the
    oracle's with the oracle's weights; a non-finite sample is reported and gets no weight."""
    wl = synth.make("hex4096_p48", seed=13, n_cells=4, q_scale=0.3)
    bad = int(wl.offsets[2]) + 1
    wl.x[bad] = float("nan")
    g = wl.to("cuda")
    plan = enufft.Plan.for_workload(g)
    w = plan.voronoi_weights(g.x, g.y, 64)
    with pytest.raises(enufft.EnufftError, match="non-finite"):
        plan.sync_status()
    assert w[bad].item() == 0.0
    ow, _ = oracle.voronoi_weights(wl, 64)
    assert _close(w.cpu().numpy(), ow)
    keep = torch.ones(wl.n_points, dtype=torch.bool)
    keep[bad] = False
    wl2 = synth.Workload(**{**wl.__dict__, "x": wl.x[keep], "y": wl.y[keep], "h": wl.h[keep],
                            "w": torch.tensor(ow)[keep], "offsets": wl.offsets - (torch.arange(5) > 2).long()})
    g2 = wl2.to("cuda")
    plan2 = enufft.Plan.for_workload(g2)
    c = plan2.type1(g2.x, g2.y, g2.h, w.cuda()[keep.cuda()].contiguous())
    plan2.sync_status()
    ref = oracle.type1(wl2)
    cn = c.cpu().numpy()
    err = np.linalg.norm((cn - ref).reshape(4, -1), axis=1) / np.linalg.norm(ref.reshape(4, -1), axis=1)
    assert err.max() <= 1e-5, err
