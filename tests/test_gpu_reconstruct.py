"""GPU parity of the Sec. 3.2 diagnostics (enufft_reconstruct) against the oracle: the truncated series
h_rec over the EMS selection at the samples, the relative reconstructed RMSE and the Parseval variances,
on deplaned elevations (Eq. alps_deplaning).  Both sides take the same coefficients and selection (the
GPU's), so the comparison isolates the reconstruction."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

enufft = pytest.importorskip("paper_2606_21278_b300")


def _deplaned(wl):
    """h'_q = h_q - sum_q w_q h_q / sum_q w_q per cell (the weights sum to |D| for these workloads)."""
    cnt = wl.counts()
    cell = torch.repeat_interleave(torch.arange(wl.n_cells), cnt)
    hw = torch.zeros(wl.n_cells, dtype=torch.float64).index_add_(0, cell, (wl.h * wl.w).double())
    ws = torch.zeros(wl.n_cells, dtype=torch.float64).index_add_(0, cell, wl.w.double())
    hbar = (hw / ws.clamp(min=1e-300))[cell]
    return synth.Workload(**{**wl.__dict__, "h": (wl.h.double() - hbar).to(wl.h.dtype)})


CASES = [
    ("tri20480_p64", dict(n_cells=10, q_scale=0.3), {}, 1e-5),
    ("hex4096_p48", dict(n_cells=6, q_scale=0.2), {}, 1e-5),
    ("tri81920_p64_mixed", dict(n_cells=8, q_scale=0.4), {}, 1e-5),     # coefficients partly from the tensor cores
    ("tri1_q2000_p32_fp64", {}, {}, 1e-9),
]


@pytest.mark.parametrize("name,mk,kw,tol", CASES)
def test_reconstruction_matches_oracle(name, mk, kw, tol):
    wl = _deplaned(synth.make(name, seed=4, **mk))
    g = wl.to("cuda")
    plan = enufft.Plan.for_workload(g, **kw)
    c, ks, sel, _ = plan.type1_ems(g.x, g.y, g.h, g.w)
    hrec, st = plan.reconstruct(c, ks, sel, g.x, g.y, g.h, g.w)
    plan.sync_status()
    cn = c.cpu().numpy()
    mask = oracle.selection_mask(ks.cpu().numpy(), sel.cpu().numpy(), wl.modes)
    ohrec, ost = oracle.reconstruct(wl, cn, mask)
    hg = hrec.cpu().double().numpy()
    off = wl.offsets.numpy()
    for j in range(wl.n_cells):
        a, b = off[j], off[j + 1]
        ref = np.linalg.norm(ohrec[a:b])
        if ref > 0:
            assert np.linalg.norm(hg[a:b] - ohrec[a:b]) <= tol * ref, j
        else:
            assert np.all(hg[a:b] == 0)
    sg = st.cpu().numpy()
    assert np.allclose(sg[:, 0], ost[:, 0], rtol=10 * tol, atol=0), (sg[:, 0], ost[:, 0])
    assert np.allclose(sg[:, 1], ost[:, 1], rtol=tol, atol=0)
    assert np.allclose(sg[:, 2:], ost[:, 2:], rtol=1e-12, atol=0)
    assert np.all(sg[:, 2] <= sg[:, 3] * (1 + 1e-12))


def test_reconstruction_edge_cases():
    """A cell with no selected pair reconstructs zero (eps_rel = 1); an empty cell gives zeros."""
    wl = _deplaned(synth.make("tri20480_p64", seed=5, n_cells=3, q_scale=0.1))
    cnt = wl.counts().tolist()
    keep = torch.ones(wl.n_points, dtype=torch.bool)
    keep[int(wl.offsets[2]):int(wl.offsets[3])] = False   # cell 2 empty
    cnt[2] = 0
    wl = synth.Workload(**{**wl.__dict__, "x": wl.x[keep], "y": wl.y[keep], "h": wl.h[keep], "w": wl.w[keep],
                           "offsets": torch.cat([torch.zeros(1, dtype=torch.int64), torch.cumsum(torch.tensor(cnt), 0)])})
    g = wl.to("cuda")
    plan = enufft.Plan.for_workload(g)
    c, ks, sel, _ = plan.type1_ems(g.x, g.y, g.h, g.w)
    ks0 = ks.clone()
    ks0[0] = 0
    hrec, st = plan.reconstruct(c, ks0, sel, g.x, g.y, g.h, g.w)
    plan.sync_status()
    a, b = int(wl.offsets[0]), int(wl.offsets[1])
    assert torch.all(hrec[a:b] == 0) and abs(st[0, 0].item() - 1.0) < 1e-6 and st[0, 2].item() == 0
    assert st[2].abs().sum().item() == 0 or st[2, 0].item() == 0
