"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Every check here compares the oracle with something other than itself: numpy's FFT, closed-form
Fourier transforms, the Monte Carlo statistics of App. C, the Gibbs step of App. C.3, the EMS
limits of App. D, hand derivations of the EMS families of Sec. 2.2, or finite differences of the
oracle's own forward sum (for the gradient).
"""
import math

import numpy as np
import pytest
import scipy.special
import torch

import oracle
import synth
from oracle import EMSParams


def _idx(P, m, n):
    return n + P // 2, m + P // 2


# ----------------------------------------------------------------------------------------------
# type-1 quadrature (App. B, Eq. discrete_quadrature; Sec. 2.1.1 regular-grid special case)
# ----------------------------------------------------------------------------------------------

@pytest.mark.parametrize("N,P", [(16, 16), (16, 8), (12, 12)])
def test_regular_grid_is_the_2d_dft(N, P):
    """On an equidistant grid the quadrature reduces to the 2-D DFT (Sec. 2.1.1): compare with numpy.fft."""
    rng = np.random.default_rng(N * 100 + P)
    vals = torch.tensor(rng.standard_normal(N * N))
    wl = synth.regular_grid_square_cell(N, lambda xp, yp: vals, half=0.6, center=(0.3, -0.2), modes=P)
    c = oracle.type1(wl)[0]
    F = np.fft.fft2(vals.numpy().reshape(N, N)) / (N * N)     # F[kn, km], rows = y
    for n in range(-P // 2, P // 2):
        for m in range(-P // 2, P // 2):
            assert abs(c[_idx(P, m, n)] - F[n % N, m % N]) < 1e-13


def test_regular_grid_parseval():
    """DFT Parseval: sum over all N x N modes of |h_mn|^2 equals (1/Q) sum h^2."""
    N = 16
    rng = np.random.default_rng(5)
    vals = torch.tensor(rng.standard_normal(N * N))
    wl = synth.regular_grid_square_cell(N, lambda xp, yp: vals, modes=N)
    c = oracle.type1(wl)[0]
    assert abs((np.abs(c) ** 2).sum() - (vals.numpy() ** 2).mean()) < 1e-13


def test_regular_grid_plane_wave_is_one_mode_pair():
    """A single cosine with integer wavenumbers gives exactly A/2 e^{+-i phi} at +-(m, n), 0 elsewhere
    (discrete orthogonality, App. C.2)."""
    N, P, A, phi, ms, ns = 16, 8, 1000.0, 0.7, 3, -2
    L = 1.5
    f = lambda xp, yp: A * torch.cos(2 * math.pi * (ms * xp + ns * yp) / L + phi)
    wl = synth.regular_grid_square_cell(N, f, half=L / 2, modes=P)
    c = oracle.type1(wl)[0]
    expect = np.zeros((P, P), complex)
    expect[_idx(P, ms, ns)] = A / 2 * np.exp(1j * phi)
    expect[_idx(P, -ms, -ns)] = A / 2 * np.exp(-1j * phi)
    assert np.abs(c - expect).max() < 1e-10 * A


def test_monte_carlo_error_statistics():
    """App. C.1/C.2: with Q uniform random samples of a plane wave, h_mn = A/2 e^{i phi} + eps with
    E[eps] = 0 and E|eps|^2 = A^2/(4Q); an off-peak mode has E|h|^2 = 2 A^2/(4Q)."""
    Q, A, m, n, phi, P, seeds = 400, 2.0, 2, 1, 0.3, 8, 300
    g = torch.Generator().manual_seed(11)
    eps, leak = [], []
    for s in range(seeds):
        wl = synth.plane_wave_cell(Q, A, m, n, phi, g, modes=P)
        c = oracle.type1(wl)[0]
        eps.append(c[_idx(P, m, n)] - A / 2 * np.exp(1j * phi))
        leak.append(c[_idx(P, -1, 3)])
    eps, leak = np.array(eps), np.array(leak)
    sig2 = A * A / (4 * Q)
    assert abs(eps.mean()) < 4 * math.sqrt(sig2 / seeds)
    assert abs(np.mean(np.abs(eps) ** 2) / sig2 - 1) < 0.2
    assert abs(np.mean(np.abs(leak) ** 2) / (2 * sig2) - 1) < 0.2


def test_gibbs_step_coefficients():
    """App. C.3, Eq. gibbs_coefficients: a step of height dh on x' in (0, L/2) has h_0 = dh/2 and
    h_m = dh [1 - (-1)^m] / (2 pi i m); dense midpoint sampling reaches it to O((m/N)^2)."""
    N, dh, P = 4096, 3.0, 16
    f = lambda xp, yp: torch.where(xp < 0.75, torch.tensor(dh, dtype=torch.float64), torch.tensor(0.0, dtype=torch.float64))
    wl = synth.regular_grid_square_cell(N, f, half=0.75, modes=P, offset=0.5, ny=4)
    c = oracle.type1(wl)[0]
    assert abs(c[_idx(P, 0, 0)] - dh / 2) < 1e-12
    for m in range(-P // 2 + 1, P // 2):
        if m == 0:
            continue
        exact = dh * (1 - (-1) ** m) / (2j * math.pi * m)
        assert abs(c[_idx(P, m, 0)] - exact) < 1e-4 * dh, m
        for n in (1, -3):
            assert abs(c[_idx(P, m, n)]) < 1e-12
    # the sign of the exponent and the x' = u + H origin are both fixed by m = 1: -i dh / pi
    assert abs(c[_idx(P, 1, 0)] - (-1j * dh / math.pi)) < 1e-4


def _triangle_ft(k, V):
    """Closed form of int_T exp(-i k.x) dA over a triangle (simplex exponential integral)."""
    area = 0.5 * abs((V[1, 0] - V[0, 0]) * (V[2, 1] - V[0, 1]) - (V[1, 1] - V[0, 1]) * (V[2, 0] - V[0, 0]))
    s = -1j * np.asarray(k)
    tot = 0
    for j in range(3):
        den = 1
        for l in range(3):
            if l != j:
                den = den * (s @ (V[j] - V[l]))
        tot = tot + np.exp(s @ V[j]) / den
    return 2 * area * tot


def test_triangle_mask_indicator_transform():
    """Cell mask (App. A): unit terrain sampled densely over B, cell mask, pixel weights: h_mn tends to
    (1/|T|) int_T e^{-i k.x'} dA (closed form), and h_00 to 1; also |D| = |T| when B contains T."""
    V = np.array([[-0.41, -0.33], [0.52, -0.18], [0.07, 0.49]])
    V = V - V.mean(0)
    N, P = 1536, 8
    H = 0.75 * (np.ptp(V, axis=0).max())
    L = 2 * H
    r = (np.arange(N) + 0.5) * L / N - H
    X, Y = np.meshgrid(r, r)
    verts = torch.zeros(1, 6, 2, dtype=torch.float64)
    verts[0, :3] = torch.tensor(V)
    wl = synth.Workload(name="tri_indicator", n_cells=1, nverts=torch.tensor([3], dtype=torch.int32),
                        verts=verts, offsets=torch.tensor([0, N * N]), x=torch.tensor(X.ravel()),
                        y=torch.tensor(Y.ravel()), h=torch.ones(N * N, dtype=torch.float64),
                        w=torch.full((N * N,), (L / N) ** 2, dtype=torch.float64), modes=P, eta=1.5,
                        mask=0, precision="fp64")
    fr = oracle.frame(3, verts[0], 1.5, 0)
    e1, e2 = V[1] - V[0], V[2] - V[0]
    area = 0.5 * abs(e1[0] * e2[1] - e1[1] * e2[0])
    assert abs(fr["area"] - area) < 1e-14 and abs(fr["H"] - H) < 1e-15
    c = oracle.type1(wl)[0]
    for n in range(-P // 2 + 1, P // 2):
        for m in range(-P // 2 + 1, P // 2):
            k = 2 * math.pi * np.array([m, n]) / L
            exact = 1.0 if (m, n) == (0, 0) else np.exp(-1j * k @ np.array([H, H])) * _triangle_ft(k, V) / area
            assert abs(c[_idx(P, m, n)] - exact) < 4e-3, (m, n)


def test_circle_mask_is_the_airy_transform():
    """Circle mask (App. A): the disk of radius H inside B transforms to e^{-i k.(H,H)} 2 J1(|k|H)/(|k|H)."""
    N, P, H = 1024, 8, 0.5
    r = (np.arange(N) + 0.5) * (2 * H) / N - H
    X, Y = np.meshgrid(r, r)
    verts = torch.zeros(1, 6, 2, dtype=torch.float64)
    verts[0, :4] = torch.tensor([[-H, -H], [H, -H], [H, H], [-H, H]])
    wl = synth.Workload(name="disk", n_cells=1, nverts=torch.tensor([4], dtype=torch.int32), verts=verts,
                        offsets=torch.tensor([0, N * N]), x=torch.tensor(X.ravel()), y=torch.tensor(Y.ravel()),
                        h=torch.ones(N * N, dtype=torch.float64),
                        w=torch.full((N * N,), (2 * H / N) ** 2, dtype=torch.float64), modes=P, eta=1.0,
                        mask=2, precision="fp64")
    assert abs(oracle.frame(4, verts[0], 1.0, 2)["area"] - math.pi * H * H) < 1e-15
    c = oracle.type1(wl)[0]
    for n in range(-P // 2, P // 2):
        for m in range(-P // 2, P // 2):
            k = math.pi * np.array([m, n]) / H
            kk = np.linalg.norm(k) * H
            airy = 1.0 if kk == 0 else 2 * scipy.special.j1(kk) / kk
            exact = np.exp(-1j * (k[0] + k[1]) * H) * airy
            assert abs(c[_idx(P, m, n)] - exact) < 3e-3, (m, n)


def test_constant_terrain_gives_cell_area_dc():
    """Constant terrain with weights summing to |D| gives h_00 = the constant (Eq. discrete_quadrature,
    Eq. uniform_weights); checked on triangles and hexagons of the synthetic workloads."""
    for name in ("tri20480_p64", "hex4096_p48"):
        wl = synth.make(name, seed=3, n_cells=6, q_scale=0.05, dtype=torch.float64)
        wl.h = torch.full_like(wl.h, 137.5)
        c = oracle.type1(wl, P=8)
        assert np.abs(c[:, 4, 4] - 137.5).max() < 1e-10


def test_hermitian_symmetry():
    """Realness h_{-m,-n} = conj(h_{m,n}) (Eq. series) for real terrain."""
    wl = synth.make("tri20480_p64", seed=1, n_cells=3, q_scale=0.1)
    P = 16
    c = oracle.type1(wl, P=P)
    for j in range(3):
        for n in range(-P // 2 + 1, P // 2):
            for m in range(-P // 2 + 1, P // 2):
                assert abs(c[j][_idx(P, -m, -n)] - np.conj(c[j][_idx(P, m, n)])) <= 1e-12 * np.abs(c[j]).max()


def test_window_clips_and_closed_edges():
    """App. A with eta = 1: the equilateral triangle's apex sticks out of B, so |D| = |B n T| (closed form);
    samples outside the cell get window 0, samples on an edge or vertex count (closed mask)."""
    s3 = math.sqrt(3)
    V = np.array([[-0.5, -s3 / 6], [0.5, -s3 / 6], [0.0, s3 / 3]])
    fr = oracle.frame(3, V, 1.0, 0)
    assert abs(fr["H"] - 0.5) < 1e-15
    apex = s3 / 3 - 0.5                     # height of the part above y = H
    cut = (s3 / 4) * (apex / (s3 / 2)) ** 2  # similar triangle
    assert abs(fr["area"] - (s3 / 4 - cut)) < 1e-14
    xs = np.array([0.0, 0.0, 0.5, -0.5, 0.25, 0.0, 0.6, 0.0])
    ys = np.array([0.0, 0.55, -s3 / 6, -s3 / 6, -s3 / 6, -0.3, 0.0, 0.5])
    win = oracle.window(3, V, xs, ys, eta=1.0, mask=0)
    # centre in; apex region above H out; base vertices in (closed); base edge in; below base out;
    # right of the cell out; exactly at y = H on the axis in
    assert win.tolist() == [1, 0, 1, 1, 1, 0, 0, 1]


def test_single_sample_scales_with_weight_over_area():
    """Linearity of the sum in w_q h_q / |D|: doubling one sample's weight adds exactly its term."""
    wl = synth.make("tri20480_p64", seed=2, n_cells=1, q_scale=0.01, dtype=torch.float64)
    c0 = oracle.type1(wl, P=8)
    wl2 = synth.Workload(**{**wl.__dict__, "w": wl.w.clone()})
    wl2.w[0] *= 2
    c1 = oracle.type1(wl2, P=8)
    one = synth.Workload(**{**wl.__dict__, "offsets": torch.tensor([0, 1]), "x": wl.x[:1], "y": wl.y[:1],
                            "h": wl.h[:1], "w": wl.w[:1]})
    ct = oracle.type1(one, P=8)
    assert np.abs(c1 - c0 - ct).max() < 1e-12 * np.abs(c0).max()


# ----------------------------------------------------------------------------------------------
# EMS (Sec. 2.2 and App. D)
# ----------------------------------------------------------------------------------------------

def _families(J=20):
    j = np.arange(1, J + 1)
    return {
        "uniform": np.full(J, 0.5),
        "exponential": np.exp(1.0 - j),
        "peak": np.where(j == 1, 1.0, 0.05),
        "step": np.where(j <= 5, 0.7, 0.35),
        "geometric": 0.9 * 0.85 ** (j - 1),
        "cosine": 0.9 * np.cos(np.pi * (j - 1) / (2 * J)),
    }


# K* derived by hand from Eqs. n_eff, s_delta, c_score, alpha_c, f_cum, k_elastic for the spectra of
# the EMS illustration (J* = 20, K_min 1, K_max 12, alpha 0..0.7, delta 0.02, w1 = w2 = 0.5):
#   uniform   HEAD: N_eff=12, S=1, C=1, alpha=.7, theta(K)=K/12  -> 9;  ALL: theta=K/20 -> 14 -> cap 12
#   exponential: G=e, S~0, N_eff~(1+r)/(1-r)=2.16 (r=1/e), alpha~.063 <= theta(1)=.63 -> 1 (both)
#   peak      HEAD: N_eff=1.55^2/1.0275, S=10/11, alpha=.386 <= theta(1)=1/1.55 -> 1; ALL likewise -> 1
#   step      HEAD: N_eff=5.95^2/3.3075=10.7, S=10/11, alpha=.630; theta(5)=.588, theta(6)=.647 -> 6
#             ALL:  N_eff=17.9->12, alpha=.668; theta(11)=5.6/8.75=.64, theta(12)=.68 -> 12
#   geometric HEAD: N_eff=9.26, S=1.5e-4, alpha=.270; theta(1)=.175, theta(2)=.324 -> 2
#             ALL:  N_eff=11.41, alpha=.333; theta(2)=.289, theta(3)=.402 -> 3
#   cosine    HEAD 5, ALL 7 (flat head: S and N_eff both large, theta grows almost linearly)
FAMILY_KSTAR = {"uniform": (9, 12), "exponential": (1, 1), "peak": (1, 1), "step": (6, 12),
                "geometric": (2, 3), "cosine": (5, 7)}


@pytest.mark.parametrize("fam", list(FAMILY_KSTAR))
def test_ems_families(fam):
    E = _families()[fam]
    for sum_all in (0, 1):
        k, sel, ret, diag = oracle.ems_energies(E, EMSParams(sum_all=sum_all))
        assert k == FAMILY_KSTAR[fam][sum_all], (fam, sum_all, k, diag)
        assert sel.tolist() == list(range(k))          # the top-K* positions, already descending
        assert abs(ret - E[:k].sum()) < 1e-14


def test_ems_uniform_head_closed_forms():
    k, _, _, d = oracle.ems_energies(np.full(20, 0.5), EMSParams())
    assert abs(d[0] - 12) < 1e-12 and abs(d[1] - 1) < 1e-15 and abs(d[2] - 1) < 1e-12 and abs(d[3] - 0.7) < 1e-12


def test_ems_sdelta_flat_tail_limit():
    """App. D.1: E = (1, eps, ..., eps), J* = K_max: S_delta -> (K_max-2)/(K_max-1), N_eff -> 1, K* = 1."""
    K, eps = 12, 1e-6
    E = np.array([1.0] + [eps] * (K - 1))
    k, _, _, d = oracle.ems_energies(E, EMSParams(k_max=K))
    assert abs(d[1] - (K - 2) / (K - 1)) < 1e-15
    assert abs(d[0] - (1 + (K - 1) * eps) ** 2 / (1 + (K - 1) * eps ** 2)) < 1e-12
    assert k == 1


def test_ems_neff_moment_degeneracy():
    """App. D.2: a geometric spectrum and the step spectrum with the same (M1, M2) (b, c from
    Eqs. dformula, bcformula) share N_eff; S_delta is exp(-(1/rho-1)/delta) versus
    (K_max - 2 + exp(-(b/c-1)/delta)) / (K_max - 1)."""
    K, rho, p, delta = 12, 0.8, 3, 0.02
    EA = rho ** np.arange(K)
    M1, M2 = EA.sum(), (EA ** 2).sum()
    r = K - p
    d = math.sqrt((K * M2 - M1 ** 2) / (p * r))
    b, c = M1 / K + r / K * d, M1 / K - p / K * d
    EB = np.array([b] * p + [c] * r)
    _, _, _, dA = oracle.ems_energies(EA, EMSParams(k_max=K, delta=delta))
    _, _, _, dB = oracle.ems_energies(EB, EMSParams(k_max=K, delta=delta))
    assert abs(dA[0] - dB[0]) < 1e-12 * dA[0]
    assert abs(dA[0] - M1 ** 2 / M2) < 1e-12 * dA[0]
    assert abs(dA[1] - math.exp(-(1 / rho - 1) / delta)) < 1e-15
    assert abs(dB[1] - (K - 2 + math.exp(-(b / c - 1) / delta)) / (K - 1)) < 1e-14


def test_ems_degenerate_cases():
    z, _, ret, _ = oracle.ems_energies(np.zeros(10), EMSParams())
    assert z == 0 and ret == 0.0                                  # no power: nothing selected
    k, sel, _, _ = oracle.ems_energies(np.array([0.0, 2.0, 0.0]), EMSParams(k_min=3, k_max=3))
    assert k == 1 and sel.tolist() == [1]                          # never select zero-energy pairs
    k, sel, _, _ = oracle.ems_energies(np.array([1.0, 3.0, 3.0, 1.0]), EMSParams(k_min=3, k_max=4))
    assert sel.tolist() == [1, 2, 0]                               # ties: lower index first
    k, _, _, d = oracle.ems_energies(np.array([5.0]), EMSParams())
    assert k == 1 and d[1] == 0.0                                  # J_max < 2: S_delta = 0


def test_ems_margins_closed_forms():
    """Per-cell margins of the selection (near-tie diagnostics), on spectra worked by hand.

    E = (4, 3, 2, 1), K_max = 4, HEAD sums: total 10, N_eff = 100/30, S_delta = (e^(-50/3) + e^(-25) +
    e^(-50)) / 3 ~ 1.9e-8, C = 0.5 (10/3)/4 + 0.5 S_delta, alpha_C = 0.7 C = 0.291667 (+1.3e-8);
    theta(1) = 0.4 >= alpha_C, so K* = 1: margin_theta = min(0.4 - alpha_C, alpha_C - 0) = 0.108333,
    margin_rank = (4 - 3)/4; no gap at K_max (J* = K_max).  With K_max = 3 and K_min = 3 the
    budget clamps K* to 3: margin_rank = (2 - 1)/2 and the K_max gap is (2 - 1)/2."""
    k, _, _, d = oracle.ems_energies(np.array([1.0, 4.0, 2.0, 3.0]), EMSParams(k_max=4))
    assert k == 1
    assert abs(d[3] - 0.7 * 0.5 * (10 / 3) / 4) < 1e-7
    assert abs(d[6] - 0.25) < 1e-15
    assert abs(d[7] - (0.4 - 0.7 * 0.5 * (10 / 3) / 4)) < 1e-7
    assert math.isnan(d[10])
    k, _, _, d = oracle.ems_energies(np.array([4.0, 3.0, 2.0, 1.0]), EMSParams(k_min=3, k_max=3))
    assert k == 3 and abs(d[6] - 0.5) < 1e-15 and abs(d[10] - 0.5) < 1e-15


def test_ems_alpha_sensitivity_two_pairs():
    """Two equal pairs (J* = K_max = 2): N_eff = 2, S_delta = 1, C = 1, alpha_C = 0.7.  A relative
    error eps on alternate energies gives (1 + eps, 1 - eps): N_eff = 2 / (1 + eps^2) and
    S_delta = exp(-(2 eps / (1 - eps)) / delta), so alpha_C moves by
    0.7 - 0.7 (0.5 / (1 + eps^2) + 0.5 exp(-2 eps / ((1 - eps) delta))).  A common factor on every
    energy changes nothing, and eps = 0 gives 0."""
    for eps in (1e-3, 2e-5):
        prm = EMSParams(k_max=2, sens_eps=eps)
        _, _, _, d = oracle.ems_energies(np.array([1.0, 1.0]), prm)
        want = 0.7 - 0.7 * (0.5 / (1 + eps * eps) + 0.5 * math.exp(-2 * eps / ((1 - eps) * 0.02)))
        assert abs(d[3] - 0.7) < 1e-15 and abs(d[11] - want) < 1e-12, (eps, d[11], want)
        _, _, _, d2 = oracle.ems_energies(np.array([3.5, 3.5]), prm)
        assert abs(d2[11] - d[11]) < 1e-14
    _, _, _, d = oracle.ems_energies(np.array([1.0, 1.0]), EMSParams(k_max=2, sens_eps=0.0))
    assert d[11] == 0.0


def test_ems_on_spectrum_pairs_and_indices():
    """A spectrum with two plane waves: the selected pairs are those two, encoded by the half-plane
    member (n > 0, or n = 0 and m > 0), p = (n + P/2) P + (m + P/2); DC is excluded."""
    P = 8
    c = np.zeros((1, P, P), complex)
    c[0][_idx(P, 0, 0)] = 100.0                          # DC (excluded by default)
    for (m, n, a) in [(2, -1, 3.0), (1, 0, 2.0)]:
        c[0][_idx(P, m, n)] = a
        c[0][_idx(P, -m, -n)] = a
    ks, sel, ret, diag = oracle.ems(c, EMSParams(k_min=2))
    pidx = lambda m, n: (n + P // 2) * P + (m + P // 2)
    assert ks[0] == 2 and sel[0, :2].tolist() == [pidx(-2, 1), pidx(1, 0)]
    assert abs(ret[0] - 2 * 9.0 - 2 * 4.0) < 1e-12
    assert diag[0, 8] == ((P - 1) ** 2 - 1) // 2          # J* pairs in the symmetric box


# ----------------------------------------------------------------------------------------------
# gradient of the EMS-retained power (adjoint of the quadrature)
# ----------------------------------------------------------------------------------------------

def test_adjoint_identity():
    """Re <G, T1 h> = <dL/dh, h> for the linear loss L = Re sum conj(G) h_mn (T2 is the adjoint of T1)."""
    wl = synth.make("hex4096_p48", seed=4, n_cells=2, q_scale=0.03, dtype=torch.float64)
    P = 8
    wl = synth.Workload(**{**wl.__dict__, "modes": P})
    rng = np.random.default_rng(0)
    G = rng.standard_normal((2, P, P)) + 1j * rng.standard_normal((2, P, P))
    c = oracle.type1(wl)
    gh, gw = oracle.type1_backward(wl, G)
    lhs = np.real(np.sum(np.conj(G) * c))
    assert abs(lhs - gh @ wl.h.numpy()) < 1e-11 * abs(lhs)
    assert abs(lhs - gw @ wl.w.numpy()) < 1e-11 * abs(lhs)


def test_gradient_matches_finite_differences():
    """With the selected set fixed, the retained power is an exact quadratic in h and in w, so central
    differences reproduce the analytic gradient up to rounding (FD step 1e-6 relative to the sample)."""
    wl = synth.make("hex4096_p48", seed=5, n_cells=2, q_scale=0.03, dtype=torch.float64)
    P = 8
    wl = synth.Workload(**{**wl.__dict__, "modes": P})
    prm = EMSParams(k_max=6)
    c = oracle.type1(wl)
    ks, sel, ret, _ = oracle.ems(c, prm)
    gp = np.array([1.0, 0.5])
    G = oracle.ems_grad_coeffs(c, ks, sel, gp, prm.k_max)
    gh, gw = oracle.type1_backward(wl, G)

    def loss(h, w):
        wl2 = synth.Workload(**{**wl.__dict__, "h": h, "w": w})
        return float(gp @ oracle.selected_power(oracle.type1(wl2), ks, sel, prm.k_max))

    rng = np.random.default_rng(1)
    for q in rng.choice(wl.n_points, 6, replace=False):
        for which, grad in (("h", gh), ("w", gw)):
            h, w = wl.h.clone(), wl.w.clone()
            arr = h if which == "h" else w
            step = 1e-6 * max(abs(float(arr[q])), 1.0)
            arr[q] += step
            lp = loss(h, w)
            arr[q] -= 2 * step
            lm = loss(h, w)
            fd = (lp - lm) / (2 * step)
            assert abs(fd - grad[q]) <= 1e-4 * max(abs(grad[q]), 1e-3 * np.abs(grad).max()), (which, q)


def _golden(name):
    import os
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_gibbs_overshoot_matches_printed_constant():
    """App. C.3, Eq. gibbs_overshoot: rebuild S_{2N+1}(x_N) from the oracle's coefficients of a step and
    compare the overshoot with the printed 0.08949 dh (finite N and quadrature add < 2e-3)."""
    Nt, dh, L = 24, 2.0, 1.5
    P = 4 * Nt + 8
    f = lambda xp, yp: torch.where(xp < L / 2, torch.tensor(dh, dtype=torch.float64),
                                   torch.tensor(0.0, dtype=torch.float64))
    wl = synth.regular_grid_square_cell(8192, f, half=L / 2, modes=P, offset=0.5, ny=1)
    c = oracle.type1(wl)[0][P // 2, :]            # n = 0 row, m = -P/2 .. P/2-1
    xN = L / (4 * (Nt + 1))
    S = 0.0
    for m in range(-(2 * Nt + 1), 2 * Nt + 2):
        S += (c[m + P // 2] * np.exp(2j * math.pi * m * xN / L)).real
    assert abs((S - dh) / dh - _golden("gibbs_overshoot.txt")["overshoot_over_dh"]) < 2e-3


# ----------------------------------------------------------------------------------------------
# reconstruction diagnostics (Sec. 3.2: Eqs. tri_series, alps_relative_rmse, spectral_variance)
# ----------------------------------------------------------------------------------------------

def test_reconstruction_with_every_mode_is_the_inverse_dft():
    """On an equidistant grid the truncated series over the full N x N box is the inverse DFT: h_rec = h
    at every sample (eps_rel = 0), and Parseval holds exactly: sigma2_phys = sigma2_spec(box) + |h_00|^2."""
    N = 16
    rng = np.random.default_rng(21)
    vals = torch.tensor(rng.standard_normal(N * N) * 300.0 + 40.0)
    wl = synth.regular_grid_square_cell(N, lambda xp, yp: vals, half=0.6, center=(0.3, -0.2), modes=N)
    c = oracle.type1(wl)
    mask = np.ones((1, N, N), dtype=np.uint8)
    hrec, st = oracle.reconstruct(wl, c, mask)
    assert np.abs(hrec - vals.numpy()).max() < 1e-10 * np.abs(vals.numpy()).max()
    assert st[0, 0] < 1e-12
    dc = abs(c[0, N // 2, N // 2]) ** 2
    assert abs(st[0, 1] - (st[0, 3] + dc)) < 1e-12 * st[0, 1]
    assert st[0, 2] == st[0, 3]


def test_reconstruction_of_a_plane_wave_from_its_pair():
    """A cosine with integer wavenumbers is one mode pair; the series over that pair reproduces it at the
    samples (eps_rel = 0) and both variances equal A^2 / 2."""
    N, P, A, phi, ms, ns = 16, 8, 700.0, 0.4, 2, 3
    L = 1.5
    f = lambda xp, yp: A * torch.cos(2 * math.pi * (ms * xp + ns * yp) / L + phi)
    wl = synth.regular_grid_square_cell(N, f, half=L / 2, modes=P)
    c = oracle.type1(wl)
    kstar = np.array([1])
    sel = np.array([[(ns + P // 2) * P + (ms + P // 2)] + [-1] * 11])
    mask = oracle.selection_mask(kstar, sel, P)
    assert mask.sum() == 2 and mask[0, _idx(P, -ms, -ns)[0], _idx(P, -ms, -ns)[1]] == 1
    hrec, st = oracle.reconstruct(wl, c, mask)
    assert np.abs(hrec - wl.h.numpy()).max() < 1e-9 * A
    assert st[0, 0] < 1e-11
    assert abs(st[0, 1] - A * A / 2) < 1e-9 * A * A and abs(st[0, 2] - A * A / 2) < 1e-9 * A * A


def test_reconstruction_from_no_modes():
    """An empty mode set reconstructs zero: eps_rel = 1 and no spectral variance in the set."""
    wl = synth.make("tri20480_p64", seed=3, n_cells=2, q_scale=0.05)
    c = oracle.type1(wl)
    hrec, st = oracle.reconstruct(wl, c, np.zeros((2, 64, 64), dtype=np.uint8))
    assert np.all(hrec == 0) and np.allclose(st[:, 0], 1.0) and np.all(st[:, 2] == 0)
    assert np.all(st[:, 3] > 0) and np.all(st[:, 1] > 0)


def _setpair(c, m, n, amp):
    P = c.shape[-1]
    half = P // 2
    c[0, n + half, m + half] = amp
    c[0, -n + half, -m + half] = np.conj(amp)


def test_mode_set_gate_separates_near_ties_from_errors():
    """The end-to-end EMS mode-set gate: an identical spectrum passes with no mismatch; a selection that
    differs from the oracle's while every energy agrees exactly is an error, not a near-tie; two head
    energies 1e-9 apart, swapped by a 1e-8 relative change of one of them, are a near-tie whose measured
    energy error is about 2e-8."""
    rng = np.random.default_rng(4)
    P = 16
    c = 0.01 * (rng.standard_normal((1, P, P)) + 1j * rng.standard_normal((1, P, P)))
    pos = [(m, n) for n in range(1, 5) for m in range(-3, 4)][:14]
    for k, (m, n) in enumerate(pos):                  # a flat head: K* = 6 of 14 strong pairs
        _setpair(c, m, n, 10.0 * (1 - 0.01 * k))
    ks, sel, _, _ = oracle.ems(c)
    assert ks[0] >= 3
    g = oracle.mode_set_gate(c, ks, sel, c)
    assert g["mismatches"] == [] and g["all_near_ties"]
    sel2 = sel.copy()
    sel2[0, 0] = (P // 2 + 6) * P + (P // 2 - 5)      # a background pair, far below the head
    g = oracle.mode_set_gate(c, ks, sel2, c)
    assert len(g["mismatches"]) == 1 and not g["all_near_ties"]
    c3 = c.copy()
    _setpair(c3, *pos[2], 10.0 * 0.99 * (1 - 1e-9))   # nearly ties with the second pair
    c4 = c3.copy()
    _setpair(c4, *pos[2], 10.0 * 0.99 * (1 - 1e-9) * (1 + 1e-8))
    ks4, sel4, _, _ = oracle.ems(c4)
    g = oracle.mode_set_gate(c4, ks4, sel4, c3)
    assert len(g["mismatches"]) == 1 and g["all_near_ties"]
    assert 1e-8 < g["mismatches"][0]["energy_err"] < 3e-8


# ----------------------------------------------------------------------------------------------
# Voronoi quadrature weights by raster sampling (App. A, Eqs. raster_grid .. voronoi_weights)
# ----------------------------------------------------------------------------------------------

def _square_cell(xs, ys, half=0.5):
    """One square cell [-half, half]^2 (window = the square) with the given binary32 samples."""
    n = len(xs)
    wl = synth.regular_grid_square_cell(1, lambda a, b: torch.zeros_like(a), half=half, dtype=torch.float32)
    return synth.Workload(**{**wl.__dict__, "x": torch.tensor(xs, dtype=torch.float32),
                             "y": torch.tensor(ys, dtype=torch.float32), "h": torch.zeros(n, dtype=torch.float32),
                             "w": torch.zeros(n, dtype=torch.float32),
                             "offsets": torch.tensor([0, n], dtype=torch.int64)})


def test_voronoi_weights_of_a_lattice_are_equal():
    """Samples at the midpoints of an n x n lattice with Ng = 2n raster points per side: every sample is
    nearest to exactly its own 2 x 2 block of raster points, so every weight is |D| / n^2."""
    n = 12
    wl = synth.regular_grid_square_cell(n, lambda a, b: torch.zeros_like(a), half=0.6, offset=0.5, dtype=torch.float32)
    w, cnt = oracle.voronoi_weights(wl, Ng=2 * n)
    assert np.all(cnt == 4)
    assert np.allclose(w, (1.2 ** 2) / n ** 2, rtol=1e-6, atol=0)


def test_voronoi_weights_split_at_the_bisector():
    """Two samples mirrored about x = 0 in the unit square: the bisector splits the raster evenly."""
    w, cnt = oracle.voronoi_weights(_square_cell([-0.2, 0.2], [0.1, 0.1]), Ng=32)
    assert cnt.tolist() == [512, 512] and np.allclose(w, [0.5, 0.5], rtol=1e-7)


def test_voronoi_duplicate_sample_takes_the_floor():
    """A coincident second sample loses every tie (lowest index wins), gets the floor 1/2 and the weights
    still partition the area (Eq. area_partition)."""
    w, cnt = oracle.voronoi_weights(_square_cell([-0.1, -0.1, 0.3], [0.2, 0.2, -0.25]), Ng=40)
    assert cnt[1] == 0 and cnt[0] > 0 and cnt[2] > 0 and cnt[0] + cnt[2] == 40 * 40
    s = cnt[0] + cnt[2] + 0.5
    assert abs(w[1] - 0.5 / s) < 1e-7 and abs(w.sum() - 1.0) < 1e-6


def _f32_column_case(Ng=10, D=2.0 ** -7):
    """Raster column a of the unit square whose binary64 abscissa X is not a binary32 number, and two
    binary32 samples at binary32(X) -/+ D on one raster row: the far one (the side of binary32(X) away
    from X) first, so that it wins every tie of a decision taken in binary32."""
    base = _square_cell([0.0], [0.0])
    fr = oracle.frame(4, base.verts[0], base.eta, base.mask)
    x0, y0, step = fr["cx"] - fr["H"], fr["cy"] - fr["H"], fr["L"] / Ng
    a = next(a for a in range(Ng) if float(np.float32(x0 + step * (a + 0.5))) != x0 + step * (a + 0.5))
    X = x0 + step * (a + 0.5)
    Xf = float(np.float32(X))
    near, far = (Xf + D, Xf - D) if X > Xf else (Xf - D, Xf + D)
    Yf = float(np.float32(y0 + step * 3.5))
    assert float(np.float32(near)) == near and float(np.float32(far)) == far
    return [far, near], [Yf, Yf], (x0, y0, step), a


def test_voronoi_nearest_sample_is_decided_exactly():
    """Eq. nn_assignment assigns each raster point to its nearest sample, an exact decision.  On the
    column whose abscissa X binary32 cannot represent, two samples symmetric about binary32(X) are at
    equal binary32 distances, while in exact arithmetic the sample on X's side is nearer for every
    point of the column.  The counts must be those of exact rational arithmetic (ties to the lower
    index), which differ from a decision taken in binary32."""
    from fractions import Fraction as Fr
    Ng = 10
    xs, ys, (x0, y0, step), a = _f32_column_case(Ng)
    _, cnt = oracle.voronoi_weights(_square_cell(xs, ys), Ng=Ng)
    exact, f32 = [0, 0], [0, 0]
    for b in range(Ng):
        Y = y0 + step * (b + 0.5)
        for a2 in range(Ng):
            X = x0 + step * (a2 + 0.5)
            d = [(Fr(X) - Fr(xs[i])) ** 2 + (Fr(Y) - Fr(ys[i])) ** 2 for i in range(2)]
            exact[0 if d[0] <= d[1] else 1] += 1
            Xf, Yf = np.float32(X), np.float32(Y)
            e = [(Xf - np.float32(xs[i])) * (Xf - np.float32(xs[i])) + (Yf - np.float32(ys[i])) * (Yf - np.float32(ys[i]))
                 for i in range(2)]
            f32[0 if e[0] <= e[1] else 1] += 1
    assert exact != f32                       # the case separates the two precisions
    assert cnt.tolist() == exact
    assert exact[1] == Ng * (Ng - a - 1) + Ng or exact[1] == Ng * (a + 1)   # the near sample owns column a


def test_voronoi_weights_partition_the_window():
    """Triangles: the weights of the windowed samples sum to |D|, every windowed sample has a positive
    weight, and samples outside the window get none."""
    wl = synth.make("tri20480_p64", seed=8, n_cells=3, q_scale=0.05)
    wl.x[int(wl.offsets[1]) + 2] += 50.0           # one sample far outside its window
    w, cnt = oracle.voronoi_weights(wl, Ng=48)
    for j in range(3):
        a, b = int(wl.offsets[j]), int(wl.offsets[j + 1])
        area = oracle.frame(int(wl.nverts[j]), wl.verts[j], wl.eta, wl.mask)["area"]
        assert abs(w[a:b].sum() - area) < 1e-5 * area
        inside = cnt[a:b] >= 0
        assert np.all(w[a:b][inside] > 0) and np.all(w[a:b][~inside] == 0)
    assert cnt[int(wl.offsets[1]) + 2] == -1


# ---------------------------------------------------------------------------------------------
# edge-aligned frame (App. A, Eq. rotation_matrix)
# ---------------------------------------------------------------------------------------------

def _one_cell(V, n=400, seed=0, frame=1, mask=0, P=16):
    """One triangle V (3 x 2) with n uniform samples inside and a smooth field on them."""
    rng = np.random.default_rng(seed)
    r1, r2 = rng.random(n), rng.random(n)
    flip = r1 + r2 > 1
    r1[flip], r2[flip] = 1 - r1[flip], 1 - r2[flip]
    P0, P1, P2 = (np.asarray(v, float) for v in V)
    pts = P0 + r1[:, None] * (P1 - P0) + r2[:, None] * (P2 - P0)
    h = np.cos(3 * pts[:, 0] + 1) + 0.5 * np.sin(2 * pts[:, 1] - 0.3) + 0.2
    verts = torch.zeros(1, 6, 2, dtype=torch.float64)
    verts[0, :3] = torch.tensor(np.asarray(V, float))
    e1, e2 = P1 - P0, P2 - P0
    area = 0.5 * abs(e1[0] * e2[1] - e1[1] * e2[0])
    return synth.Workload(name="one_cell", n_cells=1, nverts=torch.tensor([3], dtype=torch.int32), verts=verts,
                          offsets=torch.tensor([0, n]), x=torch.tensor(pts[:, 0]), y=torch.tensor(pts[:, 1]),
                          h=torch.tensor(h), w=torch.full((n,), area / n, dtype=torch.float64), modes=P, eta=1.5,
                          mask=mask, precision="fp64", frame=frame)


def test_edge_frame_right_triangle_by_hand():
    """Legs 4 (x) and 3 (y): the hypotenuse e2 = (-4, 3) is the longest edge, so cos t = -0.8,
    sin t = 0.6; in the edge frame that edge is (5, 0), the extents are 5 (along it) and the height
    12/5, hence H = eta/2 * 5, against eta/2 * 4 in the centroid frame; |D| is the triangle's area 6
    (eta = 1.5 contains it) or L^2 for the square mask."""
    V = np.array([[0.0, 0.0], [4.0, 0.0], [0.0, 3.0], [0, 0], [0, 0], [0, 0]])
    fe = oracle.frame(3, V, 1.5, 0, frame=1)
    fc = oracle.frame(3, V, 1.5, 0, frame=0)
    assert abs(fe["cos"] + 0.8) < 1e-15 and abs(fe["sin"] - 0.6) < 1e-15
    assert abs(fe["ux"][2] - fe["ux"][1] - 5.0) < 1e-14 and abs(fe["uy"][2] - fe["uy"][1]) < 1e-14
    assert abs(np.ptp(fe["uy"]) - 2.4) < 1e-14
    assert abs(fe["H"] - 0.75 * 5.0) < 1e-14 and abs(fc["H"] - 0.75 * 4.0) < 1e-14
    assert abs(fe["area"] - 6.0) < 1e-13
    assert abs(oracle.frame(3, V, 1.5, 1, frame=1)["area"] - (1.5 * 5.0) ** 2) < 1e-12


def test_edge_frame_is_the_identity_when_the_longest_edge_points_along_x():
    """Longest edge v1 -> v2 = (2, 0): R = I, so both frames give the same spectrum bit for bit."""
    V = [[0.0, 0.0], [2.0, 0.0], [0.5, 1.0]]
    c1 = oracle.type1(_one_cell(V, frame=1))
    c0 = oracle.type1(_one_cell(V, frame=0))
    assert np.array_equal(c1, c0)


def test_edge_frame_half_turn_conjugates_the_spectrum():
    """Longest edge v1 -> v2 = (-2, 0): R = -I, u -> -u and x' = -u + H, so for real h
    h_mn(edge) = sum c e^{+i k.u} e^{-i k.H} = conj(h_mn(centroid)) e^{-2i(k_m + k_n) H}, and
    (k_m + k_n) H = pi (m + n) makes the last factor 1: the edge-frame spectrum is the conjugate."""
    V = [[2.0, 0.0], [0.0, 0.0], [0.5, 1.0]]
    c1 = oracle.type1(_one_cell(V, frame=1))
    c0 = oracle.type1(_one_cell(V, frame=0))
    assert np.abs(c1 - np.conj(c0)).max() <= 1e-12 * np.abs(c0).max()


@pytest.mark.parametrize("mask", [0, 1, 2])
def test_edge_frame_is_attached_to_the_cell(mask):
    """Rotating and translating the whole cell (vertices and samples) leaves the edge-frame spectrum
    unchanged, for every mask, while the centroid-frame spectrum changes (a transposed or sign-flipped
    R would turn the frame by twice the rotation and fail)."""
    V = np.array([[0.1, -0.2], [1.3, 0.4], [0.2, 1.1]])
    wl = _one_cell(V, mask=mask, seed=3)
    a = 0.7
    Rm = np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])
    shift = np.array([3.0, -2.0])
    V2 = V @ Rm.T + shift
    wl2 = _one_cell(V2, mask=mask, seed=3)
    pts = np.stack([wl.x.numpy(), wl.y.numpy()], 1) @ Rm.T + shift
    wl2.x, wl2.y = torch.tensor(pts[:, 0]), torch.tensor(pts[:, 1])
    wl2.h = wl.h.clone()
    c, c2 = oracle.type1(wl), oracle.type1(wl2)
    assert np.abs(c - c2).max() <= 1e-10 * np.abs(c).max()
    wl.frame = wl2.frame = 0
    d, d2 = oracle.type1(wl), oracle.type1(wl2)
    assert np.abs(d - d2).max() > 1e-3 * np.abs(d).max()
