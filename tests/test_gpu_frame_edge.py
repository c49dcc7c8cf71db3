"""GPU parity of the edge-aligned local frame (App. A, Eq. rotation_matrix) against the FP64 oracle.

Every route (fused, tensor core, n_f = 256, plain binary32, adjoint, reconstruction) reads the local
coordinates written by the per-call pre-pass; the tolerances are the default frame's: coefficient
relative l2 per cell <= 1e-5 for binary32/mixed plans and <= 1e-9 for binary64 plans, EMS indices
bit-exact on the same binary32 spectra, window decisions those of the binary64 definition.
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


def _edge(wl):
    wl.frame = 1
    return wl


def _type1_ems(wl, **kw):
    g = wl.to("cuda")
    plan = enufft.Plan.for_workload(g, **kw)
    c, ks, sel, _ = plan.type1_ems(g.x, g.y, g.h, g.w)
    plan.sync_status()
    return plan, c.cpu().numpy(), ks.cpu().numpy(), sel.cpu().numpy()


@pytest.mark.parametrize("name,n,qs,mask", [
    ("tri20480_p64", 16, 0.3, 0),
    ("tri20480_p64", 6, 0.2, 1),
    ("tri20480_p64", 6, 0.2, 2),
    ("hex4096_p48", 6, 0.2, 0),
])
def test_edge_frame_fused_mixed_matches_oracle(name, n, qs, mask):
    wl = _edge(synth.make(name, seed=11, n_cells=n, q_scale=qs))
    wl.mask = mask
    plan, c, ks, sel = _type1_ems(wl)
    info = plan.info()
    assert info["frame"] == 1 and info["kernels_per_type1_ems"] == 3   # local coordinates, transform, EMS finish
    assert _rel_l2(c, oracle.type1(wl)).max() <= 1e-5
    oks, osel, _, _ = oracle.ems(c, OEMS(), energy_fp32=True)
    assert np.array_equal(ks, oks) and np.array_equal(sel, osel)


def test_edge_frame_changes_the_spectrum():
    """The two frames give different spectra for rotated cells (the option is not a no-op)."""
    wl = synth.make("tri20480_p64", seed=11, n_cells=4, q_scale=0.2)
    _, c0, _, _ = _type1_ems(wl)
    _, c1, _, _ = _type1_ems(_edge(wl))
    assert _rel_l2(c1, c0).min() > 1e-2


def test_edge_frame_fp64_single_triangle_matches_oracle():
    wl = _edge(synth.make("tri1_q2000_p32_fp64", seed=0))
    _, c, _, _ = _type1_ems(wl)
    err = _rel_l2(c, oracle.type1(wl))
    assert err.max() <= 1e-9, err


def test_edge_frame_tensor_core_route_matches_oracle():
    wl = _edge(synth.make("tri81920_p64_mixed", seed=5, n_cells=12, q_scale=0.5))
    plan, c, ks, sel = _type1_ems(wl)
    assert plan.info()["cells_tensor"] > 0
    assert _rel_l2(c, oracle.type1(wl)).max() <= 1e-5
    oks, osel, _, _ = oracle.ems(c, OEMS(), energy_fp32=True)
    assert np.array_equal(ks, oks) and np.array_equal(sel, osel)


def test_edge_frame_large_grid_route_matches_oracle():
    wl = _edge(synth.make("mixed2560_p128", seed=2, n_cells=4, q_scale=0.01))
    plan, c, _, _ = _type1_ems(wl)
    assert plan.info()["cells_large"] == wl.n_cells
    assert _rel_l2(c, oracle.type1(wl)).max() <= 1e-5


def test_edge_frame_plain_fp32_path_matches_oracle():
    wl = _edge(synth.make("tri20480_p64", seed=3, n_cells=5, q_scale=0.3))
    plan, c, _, _ = _type1_ems(wl, precision="fp32")
    assert plan.info()["cells_plain"] == wl.n_cells
    assert _rel_l2(c, oracle.type1(wl)).max() <= 1e-5


def test_edge_frame_boundary_samples_follow_the_binary64_decision():
    """Binary32 samples on (and within rounding of) the cell edges, with eta = 1 so that the rotated
    square B also clips the cell: every sample is kept or dropped as the binary64 definition decides
    in the edge frame (a single flip would move a coefficient by about 1/Q)."""
    wl = _edge(synth.make("tri20480_p64", seed=4, n_cells=3, q_scale=0.1, dtype=torch.float64))
    wl.eta = 1.0
    rng = np.random.default_rng(0)
    for j in range(wl.n_cells):
        V = wl.verts[j, :3].numpy()
        a, b = int(wl.offsets[j]), int(wl.offsets[j + 1])
        n = min(300, b - a)
        t = rng.random(n)
        e = rng.integers(0, 3, n)
        pts = V[e] + t[:, None] * (V[(e + 1) % 3] - V[e]) + rng.standard_normal((n, 2)) * 1e-7
        wl.x[a:a + n] = torch.tensor(pts[:, 0])
        wl.y[a:a + n] = torch.tensor(pts[:, 1])
    wl32 = synth.Workload(**{**wl.__dict__, "x": wl.x.float(), "y": wl.y.float(), "h": wl.h.float(),
                             "w": wl.w.float()})
    _, c, _, _ = _type1_ems(wl32)
    err = _rel_l2(c, oracle.type1(wl32))
    assert err.max() <= 1e-5, err


@pytest.mark.parametrize("prec,tol", [("mixed", 1e-5), ("fp64", 1e-9)])
def test_edge_frame_adjoint_matches_oracle(prec, tol):
    if prec == "fp64":
        wl = _edge(synth.make("tri1_q2000_p32_fp64", seed=1))
    else:
        wl = _edge(synth.make("hex4096_p48", seed=6, n_cells=6, q_scale=0.2))
    g = wl.to("cuda")
    plan = enufft.Plan.for_workload(g)
    P = wl.modes
    rng = np.random.default_rng(2)
    G = rng.standard_normal((wl.n_cells, P, P)) + 1j * rng.standard_normal((wl.n_cells, P, P))
    gh, gw = plan.type1_backward(torch.tensor(G, dtype=plan.complex_dtype, device="cuda"), g.x, g.y, g.h, g.w)
    oh, ow = oracle.type1_backward(wl, G)
    for a, b in ((gh, oh), (gw, ow)):
        a = a.cpu().double().numpy()
        assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b)


def test_edge_frame_reconstruction_matches_oracle():
    wl = _edge(synth.make("tri20480_p64", seed=4, n_cells=8, q_scale=0.3))
    g = wl.to("cuda")
    plan = enufft.Plan.for_workload(g)
    c, ks, sel, _ = plan.type1_ems(g.x, g.y, g.h, g.w)
    hrec, st = plan.reconstruct(c, ks, sel, g.x, g.y, g.h, g.w)
    plan.sync_status()
    mask = oracle.selection_mask(ks.cpu().numpy(), sel.cpu().numpy(), wl.modes)
    ohrec, ost = oracle.reconstruct(wl, c.cpu().numpy(), mask)
    hg = hrec.cpu().double().numpy()
    assert np.linalg.norm(hg - ohrec) <= 1e-5 * np.linalg.norm(ohrec)
    assert np.allclose(st.cpu().numpy()[:, 2:], ost[:, 2:], rtol=1e-12, atol=0)


def test_edge_frame_voronoi_weights_not_built():
    wl = _edge(synth.make("tri20480_p64", seed=1, n_cells=2, q_scale=0.05))
    g = wl.to("cuda")
    plan = enufft.Plan.for_workload(g)
    with pytest.raises(enufft.EnufftError, match="edge-frame"):
        plan.voronoi_weights(g.x, g.y, 32)
