"""FP64 CPU oracle for the ENUFFT type-1 transform, EMS and gradient (test infrastructure).

Only the tests, ``__graft_entry__.smoke()``, the CPU-baseline leg of ``bench.py`` and its untimed
parity check use this package; the CUDA library never imports, links or calls it, and it shares no
code with the library.  The arithmetic lives in ``enufft_oracle.c`` (plain C, FP64, direct sums, one function
per passage of the paper); this module compiles it with gcc and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "enufft_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, OpenMP, no FP contraction so binary32 steps round as written)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i64, i32, vp = ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        _lib.oracle_frame.argtypes = [i32, vp, d, i32, i32, vp]
        _lib.oracle_window.argtypes = [i32, vp, d, i32, i32, i64, vp, vp, vp]
        _lib.oracle_type1_batch.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, i32, d, i32, i32, vp, i32]
        _lib.oracle_type1_backward_batch.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, i32, d, i32, i32, vp,
                                                     vp, vp, i32]
        _lib.oracle_ems_batch.argtypes = [i64, i32, vp, vp, i32, i32, i32, d, d, d, d, d, i32, i32, i32, d,
                                          vp, vp, vp, vp, i32]
        _lib.oracle_ems_energies.argtypes = [i32, vp, i32, i32, d, d, d, d, d, i32, d, vp, vp, vp, vp]
        _lib.oracle_ems_grad_coeffs.argtypes = [i64, i32, vp, vp, i32, i32, vp, vp, vp, vp]
        _lib.oracle_voronoi_weights_f32.argtypes = [i64, vp, vp, vp, vp, vp, d, i32, i32, vp, vp, i32]
        _lib.oracle_reconstruct_batch.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, i32, d, i32, i32, vp, vp,
                                                  vp, vp, i32]
        for f in ("oracle_frame", "oracle_window", "oracle_type1_batch", "oracle_type1_backward_batch",
                  "oracle_ems_batch", "oracle_ems_energies", "oracle_ems_grad_coeffs",
                  "oracle_threads_used", "oracle_reconstruct_batch", "oracle_voronoi_weights_f32"):
            getattr(_lib, f).restype = ctypes.c_int
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype=np.float64)


def _arr(a, dt) -> np.ndarray:
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype=dt)


@dataclass
class EMSParams:
    """Sec. 2.2 parameters; defaults are the values of the paper's EMS illustration."""
    k_min: int = 1
    k_max: int = 12
    alpha_min: float = 0.0
    alpha_max: float = 0.7
    delta: float = 0.02
    w1: float = 0.5
    w2: float = 0.5
    sum_all: int = 0      # 0 HEAD reading (sums over J_max = min(J*, K_max)), 1 ALL reading (J*)
    include_dc: int = 0
    sens_eps: float = 2e-5   # relative energy error for the alpha_C sensitivity (twice the 1e-5
                             # coefficient gate: an energy is a sum of squared moduli)


def frame(nverts: int, verts, eta: float = 1.5, mask: int = 0, frame: int = 0) -> dict:
    """App. A frame of one cell (frame 0 centroid-aligned, 1 edge-aligned): centroid, H, L, |D|, the
    rotation (cos t, sin t) and the vertices in the local frame u = R (x - x-bar)."""
    out = np.zeros(19)
    v = _f64(verts).reshape(-1)
    assert lib().oracle_frame(int(nverts), _p(v), float(eta), int(mask), int(frame), _p(out)) == 0
    n = int(nverts)
    return dict(cx=out[0], cy=out[1], H=out[2], L=out[3], area=out[4], cos=out[5], sin=out[6],
                ux=out[7:7 + n].copy(), uy=out[13:13 + n].copy())


def window(nverts: int, verts, x, y, eta: float = 1.5, mask: int = 0, frame: int = 0) -> np.ndarray:
    v = _f64(verts).reshape(-1)
    x, y = _f64(x), _f64(y)
    win = np.zeros(len(x), dtype=np.int32)
    assert lib().oracle_window(int(nverts), _p(v), float(eta), int(mask), int(frame), len(x), _p(x), _p(y),
                               _p(win)) == 0
    return win


def _cells(wl):
    off = _arr(wl.offsets, np.int64)
    nv = _arr(wl.nverts, np.int32)
    vv = _f64(wl.verts).reshape(len(nv), 12)
    return off, nv, vv


def type1(wl, nthreads: int = 0, P: int | None = None) -> np.ndarray:
    """Coefficients [n_cells, P, P] complex128, index [cell, n + P/2, m + P/2] (App. B sum)."""
    P = P or wl.modes
    off, nv, vv = _cells(wl)
    x, y, h, w = (_f64(a) for a in (wl.x, wl.y, wl.h, wl.w))
    out = np.zeros((len(nv), P, P, 2))
    r = lib().oracle_type1_batch(len(nv), _p(off), _p(nv), _p(vv), _p(x), _p(y), _p(h), _p(w), int(P),
                                 float(wl.eta), int(wl.mask), int(wl.frame), _p(out), int(nthreads))
    assert r == 0, "oracle_type1_batch failed"
    return out[..., 0] + 1j * out[..., 1]


def threads_used() -> int:
    return lib().oracle_threads_used()


def type1_backward(wl, G: np.ndarray, nthreads: int = 0):
    """(dL/dh, dL/dw) for G = dL/dRe(coeffs) + i dL/dIm(coeffs), shape [n_cells, P, P]."""
    P = wl.modes
    off, nv, vv = _cells(wl)
    x, y, h, w = (_f64(a) for a in (wl.x, wl.y, wl.h, wl.w))
    g = np.ascontiguousarray(np.stack([G.real, G.imag], -1), dtype=np.float64)
    gh = np.zeros(len(x)); gw = np.zeros(len(x))
    r = lib().oracle_type1_backward_batch(len(nv), _p(off), _p(nv), _p(vv), _p(x), _p(y), _p(h), _p(w),
                                          int(P), float(wl.eta), int(wl.mask), int(wl.frame), _p(g), _p(gh),
                                          _p(gw),
                                          int(nthreads))
    assert r == 0
    return gh, gw


def voronoi_weights(wl, Ng: int = 64, nthreads: int = 0):
    """App. A Voronoi weights by raster sampling for binary32 samples: (w[n_points] float32,
    counts[n_points] int32, -1 for samples outside their window); see oracle_voronoi_weights_f32.
    Centroid-aligned frame only."""
    assert int(wl.frame) == 0, "Voronoi weights: centroid-aligned frame only"
    off, nv, vv = _cells(wl)
    x = np.ascontiguousarray(np.asarray(wl.x.cpu() if hasattr(wl.x, "cpu") else wl.x, dtype=np.float32))
    y = np.ascontiguousarray(np.asarray(wl.y.cpu() if hasattr(wl.y, "cpu") else wl.y, dtype=np.float32))
    w = np.zeros(len(x), dtype=np.float32)
    cnt = np.zeros(len(x), dtype=np.int32)
    r = lib().oracle_voronoi_weights_f32(len(nv), _p(off), _p(nv), _p(vv), _p(x), _p(y), float(wl.eta),
                                         int(wl.mask), int(Ng), _p(w), _p(cnt), int(nthreads))
    assert r == 0, "oracle_voronoi_weights_f32 failed"
    return w, cnt


def selection_mask(kstar, sel, P: int) -> np.ndarray:
    """Mode mask [n_cells, P, P] of the selected pairs: for k < K*, pair index p = (n + P/2) P + (m + P/2)
    marks (m, n) and its partner (-m, -n) (Sec. 2.2 selects mode pairs)."""
    kstar = np.asarray(kstar)
    sel = np.asarray(sel)
    mask = np.zeros((len(kstar), P, P), dtype=np.uint8)
    for j in range(len(kstar)):
        for k in range(int(kstar[j])):
            p = int(sel[j, k])
            n, m = p // P - P // 2, p % P - P // 2
            mask[j, n + P // 2, m + P // 2] = 1
            mask[j, -n + P // 2, -m + P // 2] = 1
    return mask


def reconstruct(wl, coeffs: np.ndarray, mask: np.ndarray, nthreads: int = 0):
    """Sec. 3.2 diagnostics for coefficients [n_cells, P, P] and a mode mask [n_cells, P, P]:
    (hrec[n_points], stats[n_cells, 4] = eps_rel, sigma2_phys, sigma2_spec over the mask,
    sigma2_spec over the box), see oracle_reconstruct_batch."""
    P = wl.modes
    off, nv, vv = _cells(wl)
    x, y, h, w = (_f64(a) for a in (wl.x, wl.y, wl.h, wl.w))
    c = np.ascontiguousarray(np.stack([np.asarray(coeffs).real, np.asarray(coeffs).imag], -1), dtype=np.float64)
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    hrec = np.zeros(len(x))
    stats = np.zeros((len(nv), 4))
    r = lib().oracle_reconstruct_batch(len(nv), _p(off), _p(nv), _p(vv), _p(x), _p(y), _p(h), _p(w), int(P),
                                       float(wl.eta), int(wl.mask), int(wl.frame), _p(c), _p(m), _p(hrec),
                                       _p(stats),
                                       int(nthreads))
    assert r == 0, "oracle_reconstruct_batch failed"
    return hrec, stats


def ems(coeffs: np.ndarray, params: EMSParams = EMSParams(), mode_weights=None, energy_fp32: bool = False,
        nthreads: int = 0):
    """EMS per spectrum.  Returns (kstar[n], sel[n, K_max] pair indices (-1 padded),
    retained_power[n], diag[n, 12]).  diag columns: N_eff, S_delta, C, alpha_C, total energy,
    theta(K*), margin_rank, margin_theta, J*, pairs with positive energy, gap at the K_max boundary,
    alpha_C sensitivity to a relative energy error params.sens_eps (NaN where undefined)."""
    coeffs = np.asarray(coeffs)
    n, P, _ = coeffs.shape
    c = np.ascontiguousarray(np.stack([coeffs.real, coeffs.imag], -1), dtype=np.float64)
    W = None
    per_cell = 0
    if mode_weights is not None:
        W = _f64(mode_weights)
        per_cell = int(W.ndim == 3)
    ks = np.zeros(n, dtype=np.int32)
    sel = np.zeros((n, params.k_max), dtype=np.int32)
    ret = np.zeros(n)
    diag = np.zeros((n, 12))
    r = lib().oracle_ems_batch(n, P, _p(c), _p(W) if W is not None else None, per_cell, params.k_min,
                               params.k_max, params.alpha_min, params.alpha_max, params.delta, params.w1,
                               params.w2, params.sum_all, params.include_dc, int(energy_fp32),
                               params.sens_eps, _p(ks), _p(sel), _p(ret), _p(diag), int(nthreads))
    assert r == 0
    return ks, sel, ret, diag


def pair_energies(coeffs: np.ndarray) -> dict:
    """Sec. 2.2 pair energies E_p = |h_p|^2 + |h_-p|^2 of one P x P spectrum (binary64, no weights) over
    the symmetric box |m|, |n| <= P/2 - 1 without DC, keyed by the pair index p = (n + P/2) P + (m + P/2)
    of the half-plane member (n > 0, or n = 0 and m > 0)."""
    c = np.asarray(coeffs, dtype=np.complex128)
    P = c.shape[-1]
    half = P // 2
    out = {}
    for n in range(0, half):
        for m in range(-(half - 1), half):
            if n == 0 and m <= 0:
                continue
            out[(n + half) * P + (m + half)] = abs(c[n + half, m + half]) ** 2 + abs(c[-n + half, -m + half]) ** 2
    return out


def mode_set_gate(got_coeffs, got_kstar, got_sel, ref_coeffs, params: EMSParams = EMSParams(), factor: float = 3.0):
    """End-to-end EMS mode-set check of a mixed-precision spectrum against the binary64 one.

    The selection of the binary64 oracle (ems on ref_coeffs) is compared with (got_kstar, got_sel)
    cell by cell.  For a cell that differs, eta is the measured relative error of the pair energies
    that decide the selection (the K_max + 1 largest oracle energies and both selections); the
    mismatch is a near-tie only when a decision of the oracle is closer than `factor` * eta: a
    relative gap between consecutive energies of the K_max + 1 largest (the order of the selection,
    K* and the K_max boundary), the threshold margin of theta(K*), or an alpha_C that moves by at least
    that margin when the energies carry a relative error `factor` * eta.  Returns a dict with
    the number of cells, the mismatching cells with their margins, eta and verdict, and whether every
    mismatch is a near-tie."""
    got_coeffs = np.asarray(got_coeffs)
    ref_coeffs = np.asarray(ref_coeffs)
    got_kstar = np.asarray(got_kstar)
    got_sel = np.asarray(got_sel)
    oks, osel, _, _ = ems(ref_coeffs, params)
    bad = np.nonzero((got_kstar != oks) | (got_sel != osel).any(1))[0]
    out = []
    for j in bad.tolist():
        Eo = pair_energies(ref_coeffs[j])
        Eg = pair_energies(got_coeffs[j])
        keys = sorted(Eo, key=lambda p: (-Eo[p], p))[: params.k_max + 1]
        keys += [int(p) for p in osel[j][: oks[j]]] + [int(p) for p in got_sel[j][: got_kstar[j]]]
        eta = max(abs(Eg[p] - Eo[p]) / Eo[p] for p in keys if p in Eo and Eo[p] > 0)
        prm = EMSParams(**{**params.__dict__, "sens_eps": factor * eta})
        _, _, _, d = ems(ref_coeffs[j:j + 1], prm)
        m_rank, m_theta, gap_kmax, sens = d[0, 6], d[0, 7], d[0, 10], d[0, 11]
        top = sorted(Eo.values(), reverse=True)[: params.k_max + 1]
        # smallest relative gap between consecutive energies of the head (the order of sel, K* and
        # the K_max boundary all hang on these comparisons)
        gap_order = min([(top[i] - top[i + 1]) / top[i] for i in range(len(top) - 1) if top[i] > 0] or [np.inf])
        gaps = [abs(v) for v in (gap_order, m_theta) if np.isfinite(v)]
        near = (min(gaps) if gaps else np.inf) <= factor * eta or (np.isfinite(sens) and sens >= abs(m_theta))
        out.append(dict(cell=int(j), kstar_gpu=int(got_kstar[j]), kstar_oracle=int(oks[j]), margin_rank=float(m_rank),
                        margin_theta=float(m_theta), gap_kmax=float(gap_kmax), gap_order=float(gap_order),
                        alpha_sensitivity=float(sens), energy_err=float(eta), near_tie=bool(near)))
    return dict(cells=int(len(oks)), mismatches=out, all_near_ties=all(m["near_tie"] for m in out))


def ems_energies(E, params: EMSParams = EMSParams()):
    """EMS on an explicit energy list.  Returns (K*, selected positions, retained, diag[12]) with the
    diag columns of ``ems``."""
    E = _f64(E)
    ks = np.zeros(1, dtype=np.int32)
    sel = np.zeros(params.k_max, dtype=np.int32)
    ret = np.zeros(1)
    diag = np.zeros(12)
    r = lib().oracle_ems_energies(len(E), _p(E), params.k_min, params.k_max, params.alpha_min,
                                  params.alpha_max, params.delta, params.w1, params.w2, params.sum_all,
                                  params.sens_eps, _p(ks), _p(sel), _p(ret), _p(diag))
    assert r == 0
    return int(ks[0]), sel[: int(ks[0])].copy(), float(ret[0]), diag


def ems_grad_coeffs(coeffs, kstar, sel, grad_power, k_max: int, mode_weights=None) -> np.ndarray:
    """G = grad_power_j * d(retained power_j)/d(coeffs) with the selection held fixed."""
    coeffs = np.asarray(coeffs)
    n, P, _ = coeffs.shape
    c = np.ascontiguousarray(np.stack([coeffs.real, coeffs.imag], -1), dtype=np.float64)
    W = _f64(mode_weights) if mode_weights is not None else None
    per_cell = int(W is not None and W.ndim == 3)
    G = np.zeros((n, P, P, 2))
    ks = _arr(kstar, np.int32); sl = _arr(sel, np.int32); gp = _f64(grad_power)
    lib().oracle_ems_grad_coeffs(n, P, _p(c), _p(W) if W is not None else None, per_cell, int(k_max),
                                 _p(ks), _p(sl), _p(gp), _p(G))
    return G[..., 0] + 1j * G[..., 1]


def selected_power(coeffs, kstar, sel, k_max: int, mode_weights=None) -> np.ndarray:
    """P_j = sum over the selected pairs of W_p (|h_p|^2 + |h_-p|^2) (DC pair counted once)."""
    coeffs = np.asarray(coeffs)
    n, P, _ = coeffs.shape
    half = P // 2
    out = np.zeros(n)
    for j in range(n):
        for k in range(int(kstar[j])):
            p = int(sel[j][k])
            m, nn = p % P - half, p // P - half
            wt = 1.0 if mode_weights is None else float(np.asarray(mode_weights).reshape(-1, P, P)[
                j if np.asarray(mode_weights).ndim == 3 else 0][nn + half, m + half])
            e = abs(coeffs[j, nn + half, m + half]) ** 2
            if (m, nn) != (0, 0):
                e += abs(coeffs[j, -nn + half, -m + half]) ** 2
            out[j] += wt * e
    return out
