"""GPU parity of the Voronoi quadrature weights (enufft_voronoi_weights) against the oracle.  The
oracle takes each nearest-sample decision (App. A, Eq. nn_assignment) with binary64 distances; the
kernel takes it in binary32 where the gap to the second-nearest sample exceeds a certified rounding
bound and in binary64 otherwise, so the counts agree exactly; the weights then agree to the last bit
(up to one unit of binary32 rounding through |D|)."""
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


def _square(xs, ys, half=0.5):
    """One square cell [-half, half]^2 (window = the square) with the given binary32 samples."""
    wl = synth.regular_grid_square_cell(1, lambda a, b: torch.zeros_like(a), half=half, dtype=torch.float32)
    n = len(xs)
    return synth.Workload(**{**wl.__dict__, "x": torch.tensor(xs, dtype=torch.float32),
                             "y": torch.tensor(ys, dtype=torch.float32), "h": torch.ones(n, dtype=torch.float32),
                             "w": torch.ones(n, dtype=torch.float32), "offsets": torch.tensor([0, n], dtype=torch.int64),
                             "precision": "mixed", "width": 7, "tol": 0.0})


@pytest.mark.parametrize("extra", [0, 17000])   # bucketed search; brute force (> 16384 windowed samples)
def test_voronoi_binary32_ties_are_decided_in_binary64(extra):
    """On a raster column whose abscissa X is not a binary32 number, two samples symmetric about
    binary32(X) tie in binary32 but not in binary64: the sample on X's side must own the column (the
    first sample, on the other side, would win a binary32 tie).  With `extra` duplicate samples in the
    far corner the cell takes the brute-force search."""
    Ng, D = 10, 2.0 ** -7
    fr = oracle.frame(4, _square([0.0], [0.0]).verts[0], 1.0, 1)
    x0, y0, step = fr["cx"] - fr["H"], fr["cy"] - fr["H"], fr["L"] / Ng
    a = next(a for a in range(Ng) if float(np.float32(x0 + step * (a + 0.5))) != x0 + step * (a + 0.5))
    X = x0 + step * (a + 0.5)
    Xf = float(np.float32(X))
    near, far = (Xf + D, Xf - D) if X > Xf else (Xf - D, Xf + D)
    Yf = float(np.float32(y0 + step * 3.5))
    xs, ys = [far, near] + [0.49] * extra, [Yf, Yf] + [-0.49] * extra
    wl = _square(xs, ys)
    g = wl.to("cuda")
    plan = enufft.Plan.for_workload(g)
    w = plan.voronoi_weights(g.x, g.y, Ng).cpu().numpy()
    plan.sync_status()
    ow, cnt = oracle.voronoi_weights(wl, Ng)
    assert _close(w, ow)
    assert cnt[1] >= Ng   # the near sample owns column a (and every column on its side)
