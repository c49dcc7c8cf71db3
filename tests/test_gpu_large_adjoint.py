"""The adjoint (type-2) and the reconstruction of the n_f = 256 route (P = 128, w = 6) against the
oracle: G -> dL/dh, dL/dw on small cells, on sampled samples of a cell split into several work items
(more than 2^18 samples), the EMS-retained-power gradient through autograd, and the Sec. 3.2
diagnostics."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import EMSParams as OEMS

pytestmark = pytest.mark.gpu

enufft = pytest.importorskip("paper_2606_21278_b300")


def _rand_g(n, P, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, P, P)) + 1j * rng.standard_normal((n, P, P))


def test_large_adjoint_matches_oracle():
    wl = synth.make("mixed2560_p128", seed=5, n_cells=4, q_scale=0.01)
    g = wl.to("cuda")
    plan = enufft.Plan.for_workload(g)
    assert plan.info()["cells_large"] == 4
    G = _rand_g(wl.n_cells, wl.modes, 1)
    gh, gw = plan.type1_backward(torch.tensor(G, dtype=torch.complex64, device="cuda"), g.x, g.y, g.h, g.w)
    plan.sync_status()
    oh, ow = oracle.type1_backward(wl, G)
    for a, b in ((gh, oh), (gw, ow)):
        a = a.cpu().double().numpy()
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)


def test_large_adjoint_of_a_split_cell_on_sampled_samples():
    """A cell of 347,664 samples (two work items of the interpolation) and one of 161,319: the
    adjoint at 4,000 sampled samples of each (v_q depends on the sample alone), against the oracle
    evaluated on those samples."""
    wl = synth.make("mixed2560_p128", seed=1, n_cells=2, q_scale=1.0)
    assert int(wl.counts().max()) > 1 << 18
    g = wl.to("cuda")
    plan = enufft.Plan.for_workload(g)
    G = _rand_g(wl.n_cells, wl.modes, 2)
    gh, gw = plan.type1_backward(torch.tensor(G, dtype=torch.complex64, device="cuda"), g.x, g.y, g.h, g.w)
    plan.sync_status()
    gh, gw = gh.cpu().double().numpy(), gw.cpu().double().numpy()
    rng = np.random.default_rng(3)
    off = wl.offsets.tolist()
    idx = np.sort(np.concatenate([rng.choice(np.arange(off[j], off[j + 1]), 4000, replace=False) for j in range(2)]))
    cnt = [int(((idx >= off[j]) & (idx < off[j + 1])).sum()) for j in range(2)]
    it = torch.tensor(idx)
    sub = synth.Workload(**{**wl.__dict__, "x": wl.x[it], "y": wl.y[it], "h": wl.h[it], "w": wl.w[it],
                            "offsets": torch.tensor([0, cnt[0], cnt[0] + cnt[1]], dtype=torch.int64)})
    oh, ow = oracle.type1_backward(sub, G)
    assert np.linalg.norm(gh[idx] - oh) <= 1e-5 * np.linalg.norm(oh)
    assert np.linalg.norm(gw[idx] - ow) <= 1e-5 * np.linalg.norm(ow)


def test_large_gradient_autograd_matches_oracle():
    wl = synth.make("mixed2560_p128", seed=7, n_cells=3, q_scale=0.01)
    g = wl.to("cuda")
    plan = enufft.Plan.for_workload(g)
    h = g.h.clone().requires_grad_(True)
    w = g.w.clone().requires_grad_(True)
    power, coeffs, ks, sel = enufft.EMSRetainedPower.apply(h, w, plan, g.x, g.y)
    power.sum().backward()
    plan.sync_status()
    ref = oracle.type1(wl)
    G = oracle.ems_grad_coeffs(ref, ks.cpu().numpy(), sel.cpu().numpy(), np.ones(wl.n_cells), 12)
    oh, ow = oracle.type1_backward(wl, G)
    assert np.linalg.norm(h.grad.cpu().double().numpy() - oh) <= 1e-4 * np.linalg.norm(oh)
    assert np.linalg.norm(w.grad.cpu().double().numpy() - ow) <= 1e-4 * np.linalg.norm(ow)


def test_large_reconstruction_matches_oracle():
    wl = synth.make("mixed2560_p128", seed=8, n_cells=4, q_scale=0.01)
    g = wl.to("cuda")
    plan = enufft.Plan.for_workload(g)
    c, ks, sel, _ = plan.type1_ems(g.x, g.y, g.h, g.w)
    hrec, st = plan.reconstruct(c, ks, sel, g.x, g.y, g.h, g.w)
    plan.sync_status()
    cn = c.cpu().numpy()
    mask = oracle.selection_mask(ks.cpu().numpy(), sel.cpu().numpy(), wl.modes)
    ohrec, ost = oracle.reconstruct(wl, cn, mask)
    hg = hrec.cpu().double().numpy()
    assert np.linalg.norm(hg - ohrec) <= 1e-5 * np.linalg.norm(ohrec)
    sg = st.cpu().numpy()
    assert np.allclose(sg[:, 0], ost[:, 0], rtol=1e-4, atol=0)
    assert np.allclose(sg[:, 1], ost[:, 1], rtol=1e-5, atol=0)
    assert np.allclose(sg[:, 2:], ost[:, 2:], rtol=1e-12, atol=0)
