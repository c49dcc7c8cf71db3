"""Full-size workloads in the benchmark's launch configuration, checked against the binary64 oracle on
sampled cells:
  * the 81,920-triangle mixed batch (cells of at most 3,000 samples on the tensor cores, the rest on
    the fused spread/FFT kernel), replayed from a CUDA graph as the benchmark times it;
  * the 2,560-cell n_f = 256 batch on all 128 x 128 modes, the oracle's sum for a large cell taken as
    the sum over parts of its samples (Eq. discrete_quadrature is linear in the samples);
  * the 4,096-hexagon differentiation batch: the hand-written backward against binary64 central
    differences of the EMS-retained power on 64 sampled cells.
Tolerances: coefficient rel-l2 per cell <= 1e-5, EMS mode sets through oracle.mode_set_gate, gradient
rel-err <= 1e-4."""
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


def _graph_type1_ems(plan, wl, prm):
    co = plan.new_coeffs()
    out = plan._ems_out(prm)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        plan.type1_ems(wl.x, wl.y, wl.h, wl.w, prm, coeffs=co, out=out)
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.type1_ems(wl.x, wl.y, wl.h, wl.w, prm, coeffs=co, out=out)
    for t in (co,) + out:
        t.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    plan.sync_status()
    return co, out


def test_full_size_mixed_batch_tri81920_both_routes():
    """81,920 triangles (5.6e8 samples), graph-replayed: the 16 largest cells, the tensor-core cells
    closest below the 3,000-sample threshold and the smallest ones, and a seeded random set."""
    wl = synth.make("tri81920_p64_mixed", seed=0, device="cuda")
    plan = enufft.Plan.for_workload(wl)
    info = plan.info()
    assert info["cells_tensor"] > 5000 and info["cells_fused"] > 70000
    prm = enufft.EMSParams()
    c, (ks, sel, ret) = _graph_type1_ems(plan, wl, prm)
    cnt = wl.counts().cpu()
    order = torch.argsort(cnt, descending=True).tolist()
    tc = [j for j in order if cnt[j] <= wl.tc_max_points]
    rng = np.random.default_rng(5)
    cells = sorted(set(order[:16] + tc[:12] + tc[-4:] + rng.choice(wl.n_cells, 32, replace=False).tolist()))
    assert sum(1 for j in cells if cnt[j] <= wl.tc_max_points) >= 16
    sub = wl.cell_slice(cells).to("cpu")
    got = c[cells].cpu().numpy()
    gks, gsel = ks[cells].cpu().numpy(), sel[cells].cpu().numpy()
    del wl, plan, c
    ref = oracle.type1(sub)
    err = _rel_l2(got, ref)
    assert err.max() <= 1e-5, sorted(zip(err.tolist(), cells))[-4:]
    gate = oracle.mode_set_gate(got, gks, gsel, ref, OEMS())
    assert gate["all_near_ties"], gate["mismatches"]
    oks, osel, _, _ = oracle.ems(got, OEMS(), energy_fp32=True)   # EMS logic bit-exact in the kernel's precision
    assert np.array_equal(gks, oks) and np.array_equal(gsel, osel)


def _oracle_in_parts(sub, part):
    """oracle.type1 of every cell of `sub`, each cell's samples cut into parts of at most `part`
    samples evaluated as cells of their own (same polygon, frame and |D|) and summed."""
    off = sub.offsets.tolist()
    pieces, owner = [], []
    for j in range(sub.n_cells):
        for a in range(off[j], max(off[j + 1], off[j] + 1), part):
            pieces.append((j, a, min(off[j + 1], a + part)))
    idx_cells = torch.tensor([p[0] for p in pieces])
    cnt = torch.tensor([p[2] - p[1] for p in pieces])
    new_off = torch.cat([torch.zeros(1, dtype=torch.int64), torch.cumsum(cnt, 0)])
    idx = torch.cat([torch.arange(p[1], p[2]) for p in pieces])
    parts = synth.Workload(**{**sub.__dict__, "n_cells": len(pieces), "nverts": sub.nverts[idx_cells],
                              "verts": sub.verts[idx_cells], "offsets": new_off, "x": sub.x[idx], "y": sub.y[idx],
                              "h": sub.h[idx], "w": sub.w[idx]})
    r = oracle.type1(parts)
    out = np.zeros((sub.n_cells,) + r.shape[1:], dtype=r.dtype)
    for k, (j, _, _) in enumerate(pieces):
        out[j] += r[k]
    return out


def test_full_size_n_f256_all_modes():
    """The 2,560-cell n_f = 256 workload (1.06e9 samples, P = 128, w = 6): the largest cell (about 2e6
    samples, spread in several parts), the two smallest and a random one, on all 128 x 128 modes --
    the outer modes carry the largest deconvolution factors 1/Phi."""
    wl = synth.make("mixed2560_p128", seed=0, device="cuda")
    plan = enufft.Plan.for_workload(wl)
    c = plan.type1(wl.x, wl.y, wl.h, wl.w)
    plan.sync_status()
    cnt = wl.counts().cpu()
    order = torch.argsort(cnt, descending=True).tolist()
    rng = np.random.default_rng(2)
    cells = sorted(set(order[:1] + order[-2:] + rng.choice(wl.n_cells, 1).tolist()))
    sub = wl.cell_slice(cells).to("cpu")
    got = c[cells].cpu().numpy()
    del wl, plan, c
    ref = _oracle_in_parts(sub, 125_000)
    err = _rel_l2(got, ref)
    assert err.max() <= 1e-5, err
    # the outer ring of modes (|m| or |n| >= 48) on its own
    P = 128
    mm = np.abs(np.arange(P) - P // 2)
    ring = (mm[None, :] >= 48) | (mm[:, None] >= 48)
    e_out = np.linalg.norm((got - ref)[:, ring], axis=1) / np.linalg.norm(ref[:, ring], axis=1)
    assert e_out.max() <= 1e-4, e_out


def test_fd_gradient_hex4096_on_64_cells():
    """Differentiation batch (4,096 hexagons, P = 48): dL/dh and dL/dw of L = sum of EMS-retained power
    from the full-batch backward, against binary64 central differences of the oracle's loss with the
    selection held fixed (step 1e-6 relative to the perturbed value) for two samples of each of 64
    seeded cells."""
    wl = synth.make("hex4096_p48", seed=0, device="cuda")
    plan = enufft.Plan.for_workload(wl)
    h = wl.h.clone().requires_grad_(True)
    w = wl.w.clone().requires_grad_(True)
    power, _, ks, sel = enufft.EMSRetainedPower.apply(h, w, plan, wl.x, wl.y)
    power.sum().backward()
    plan.sync_status()
    gh, gw = h.grad.cpu().double().numpy(), w.grad.cpu().double().numpy()
    rng = np.random.default_rng(9)
    cells = sorted(rng.choice(wl.n_cells, 64, replace=False).tolist())
    sub = wl.cell_slice(cells).to("cpu")
    off = wl.offsets.cpu().numpy()
    soff = sub.offsets.numpy()
    ksn, seln = ks[cells].cpu().numpy(), sel[cells].cpu().numpy()
    del wl, plan
    x64, y64, h64, w64 = (t.double() for t in (sub.x, sub.y, sub.h, sub.w))
    # every perturbed copy of a cell is a cell of one batched oracle call
    copies, meta = [], []
    for k, j in enumerate(cells):
        a, b = int(soff[k]), int(soff[k + 1])
        for q in rng.choice(b - a, 2, replace=False).tolist():
            for which in ("h", "w"):
                base = (h64 if which == "h" else w64)[a + q].item()
                step = 1e-6 * max(abs(base), 1.0) if which == "h" else 1e-6 * abs(base)
                for sgn in (1.0, -1.0):
                    hh, ww = h64[a:b].clone(), w64[a:b].clone()
                    (hh if which == "h" else ww)[q] += sgn * step
                    copies.append((k, hh, ww))
                meta.append((k, which, int(off[j]) + q, step))
    n = len(copies)
    cnts = torch.tensor([int(soff[k + 1] - soff[k]) for k, _, _ in copies])
    batch = synth.Workload(**{**sub.__dict__, "n_cells": n, "nverts": sub.nverts[[k for k, _, _ in copies]],
                              "verts": sub.verts[[k for k, _, _ in copies]],
                              "offsets": torch.cat([torch.zeros(1, dtype=torch.int64), torch.cumsum(cnts, 0)]),
                              "x": torch.cat([x64[int(soff[k]):int(soff[k + 1])] for k, _, _ in copies]),
                              "y": torch.cat([y64[int(soff[k]):int(soff[k + 1])] for k, _, _ in copies]),
                              "h": torch.cat([hh for _, hh, _ in copies]), "w": torch.cat([ww for _, _, ww in copies])})
    ref = oracle.type1(batch)
    kk = [k for k, _, _ in copies]
    L = oracle.selected_power(ref, ksn[kk], seln[kk], 12)
    gmax = max(np.abs(gh).max(), 1e-30), max(np.abs(gw).max(), 1e-30)
    bad = []
    for i, (k, which, q, step) in enumerate(meta):
        fd = (L[2 * i] - L[2 * i + 1]) / (2 * step)
        g = (gh if which == "h" else gw)[q]
        scale = max(abs(fd), 1e-2 * (gmax[0] if which == "h" else gmax[1]))
        if abs(fd - g) > 1e-4 * scale:
            bad.append((cells[k], which, q, fd, g))
    assert not bad, bad[:5]
