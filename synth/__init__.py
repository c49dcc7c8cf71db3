"""Seeded synthetic workloads for the batched per-cell ENUFFT type-1 transform and EMS.

This module only *draws inputs*: convex cell polygons in local tangent-plane
coordinates, scattered DEM-like samples inside each cell, a power-law terrain
evaluated at those samples, and quadrature weights.  It holds none of the
transform or mode-selection arithmetic; the CPU oracle and the CUDA library both
consume what it returns, and neither is imported here.

Workload recipes (shapes follow the five benchmark configurations of the
method's hot path; structure follows the paper's terrain description: power-law
spectra with ridges, Sec. 1 and App. F):

* cells: faces of a subdivided icosahedron, each projected gnomonically onto its
  own centroid tangent plane and rescaled to unit mean edge length (equal nominal
  area), randomly rotated; or regular hexagons of side 1, randomly rotated;
* samples: 80 % on a jittered lattice folded onto the triangle by the reflection
  map, 20 % uniform (triangles); 70 % uniform + 30 % clustered along three ridge
  lines (hexagons);
* elevation: 200 random-phase plane waves with amplitude 500 m (|k|/2pi)^-1.5,
  |k| log-uniform in [2pi, 40pi], plus one Gaussian ridge of height 1000 m and
  width 0.05 through the centroid;
* weights: uniform w_q = |cell| / Q (App. B, uniform weights), or positive
  jittered weights renormalised to the cell area for the gradient workload.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

__all__ = ["Workload", "CONFIGS", "make", "plane_wave_cell", "regular_grid_square_cell", "MONO_AXES", "mono_sweep"]


@dataclass
class Workload:
    name: str
    n_cells: int
    nverts: torch.Tensor      # int32 [n_cells]        3 or 6
    verts: torch.Tensor       # float64 [n_cells, 6, 2] (unused rows zero), CCW
    offsets: torch.Tensor     # int64 [n_cells + 1]     CSR offsets of each cell's samples
    x: torch.Tensor           # [N] local tangent-plane x (float32 or float64)
    y: torch.Tensor           # [N]
    h: torch.Tensor           # [N] elevation (m)
    w: torch.Tensor           # [N] quadrature weight (area units)
    modes: int                # P: retained modes per dimension, m,n in [-P/2, P/2)
    sigma: float = 2.0        # oversampling factor
    width: int = 7            # spreading kernel width (grid points)
    tol: float = 1e-6
    precision: str = "fp32"   # fp32 | mixed | fp64
    eta: float = 1.5          # window expansion factor
    mask: int = 0             # 0 cell, 1 square, 2 circle
    tc_max_points: int = 0    # cells with Q <= this go to the tensor-core direct path (0 = off)
    frame: int = 0            # 0 centroid-aligned, 1 edge-aligned local frame (App. A)
    meta: dict = field(default_factory=dict)

    @property
    def n_points(self) -> int:
        return int(self.offsets[-1])

    def counts(self) -> torch.Tensor:
        return self.offsets[1:] - self.offsets[:-1]

    def to(self, device) -> "Workload":
        kw = dict(self.__dict__)
        for k in ("nverts", "verts", "offsets", "x", "y", "h", "w"):
            kw[k] = kw[k].to(device)
        return Workload(**kw)

    def truncated(self, max_q: int) -> "Workload":
        """The first min(Q, max_q) samples of every cell (a workload of bounded cell size)."""
        cnt = self.counts()
        keep_cnt = torch.clamp(cnt, max=max_q)
        pos = torch.arange(self.n_points, device=self.offsets.device)
        cell = torch.repeat_interleave(torch.arange(self.n_cells, device=cnt.device), cnt)
        keep = (pos - self.offsets[cell]) < keep_cnt[cell]
        new_off = torch.zeros(self.n_cells + 1, dtype=torch.int64, device=cnt.device)
        new_off[1:] = torch.cumsum(keep_cnt, 0)
        kw = dict(self.__dict__)
        kw.update(offsets=new_off, x=self.x[keep], y=self.y[keep], h=self.h[keep], w=self.w[keep])
        return Workload(**kw)

    def cell_slice(self, cells) -> "Workload":
        """Sub-workload holding only the listed cells (in the given order)."""
        cells = torch.as_tensor(cells, dtype=torch.int64, device=self.offsets.device)
        lo, hi = self.offsets[cells], self.offsets[cells + 1]
        cnt = hi - lo
        new_off = torch.zeros(len(cells) + 1, dtype=torch.int64, device=cnt.device)
        new_off[1:] = torch.cumsum(cnt, 0)
        total = int(new_off[-1])
        # sample j of the slice: its cell's first source sample + its rank inside the cell
        idx = (torch.repeat_interleave(lo - new_off[:-1], cnt, output_size=total)
               + torch.arange(total, dtype=torch.int64, device=cnt.device))
        kw = dict(self.__dict__)
        kw.update(n_cells=len(cells), nverts=self.nverts[cells], verts=self.verts[cells],
                  offsets=new_off, x=self.x[idx], y=self.y[idx], h=self.h[idx], w=self.w[idx])
        return Workload(**kw)


# --------------------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------------------

def _icosahedron(level: int) -> torch.Tensor:
    """Faces [20*4**level, 3, 3] of a subdivided icosahedron on the unit sphere (CCW seen from outside)."""
    p = (1.0 + 5 ** 0.5) / 2
    v = torch.tensor([[-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
                      [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
                      [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1]], dtype=torch.float64)
    v = v / v.norm(dim=1, keepdim=True)
    f = torch.tensor([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                      [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                      [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                      [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]])
    faces = v[f]  # [20,3,3]
    for _ in range(level):
        a, b, c = faces[:, 0], faces[:, 1], faces[:, 2]
        ab = a + b; ab = ab / ab.norm(dim=1, keepdim=True)
        bc = b + c; bc = bc / bc.norm(dim=1, keepdim=True)
        ca = c + a; ca = ca / ca.norm(dim=1, keepdim=True)
        faces = torch.cat([torch.stack([a, ab, ca], 1), torch.stack([ab, b, bc], 1),
                           torch.stack([ca, bc, c], 1), torch.stack([ab, bc, ca], 1)], 0)
    return faces


def _project_faces(faces: torch.Tensor, gen: torch.Generator) -> torch.Tensor:
    """Gnomonic projection of each face onto its centroid tangent plane, unit mean edge, random rotation."""
    c = faces.sum(1)
    c = c / c.norm(dim=1, keepdim=True)
    ref = torch.where(c[:, 2:3].abs() < 0.9, torch.tensor([[0.0, 0.0, 1.0]], dtype=torch.float64),
                      torch.tensor([[1.0, 0.0, 0.0]], dtype=torch.float64))
    e1 = torch.cross(ref.expand_as(c), c, dim=1); e1 = e1 / e1.norm(dim=1, keepdim=True)
    e2 = torch.cross(c, e1, dim=1)
    pr = faces / (faces * c[:, None, :]).sum(-1, keepdim=True) - c[:, None, :]
    xy = torch.stack([(pr * e1[:, None, :]).sum(-1), (pr * e2[:, None, :]).sum(-1)], -1)  # [F,3,2]
    edges = (xy.roll(-1, 1) - xy).norm(dim=-1).mean(1)
    xy = xy / edges[:, None, None]
    th = torch.rand(len(xy), generator=gen, dtype=torch.float64) * 2 * math.pi
    rot = torch.stack([torch.stack([th.cos(), -th.sin()], -1), torch.stack([th.sin(), th.cos()], -1)], -2)
    xy = torch.einsum("fij,fvj->fvi", rot, xy)
    # enforce counter-clockwise order
    cr = ((xy[:, 1, 0] - xy[:, 0, 0]) * (xy[:, 2, 1] - xy[:, 0, 1])
          - (xy[:, 1, 1] - xy[:, 0, 1]) * (xy[:, 2, 0] - xy[:, 0, 0]))
    flip = cr < 0
    xy[flip] = xy[flip].flip(1)
    return xy


def _hexagons(n: int, gen: torch.Generator, side: float = 1.0) -> torch.Tensor:
    th = torch.rand(n, generator=gen, dtype=torch.float64) * (math.pi / 3)
    ang = th[:, None] + torch.arange(6, dtype=torch.float64)[None, :] * (math.pi / 3)
    return torch.stack([side * ang.cos(), side * ang.sin()], -1)  # [n,6,2] CCW


def _tri_area(t: torch.Tensor) -> torch.Tensor:
    a, b, c = t[:, 0], t[:, 1], t[:, 2]
    return 0.5 * ((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])).abs()


# --------------------------------------------------------------------------------------
# sampling
# --------------------------------------------------------------------------------------

def _fold_to_triangle(r1, r2, a, b, c):
    """Reflection map of the unit square onto triangle abc (uniform density preserved)."""
    fold = (r1 + r2) > 1
    r1 = torch.where(fold, 1 - r1, r1)
    r2 = torch.where(fold, 1 - r2, r2)
    return a + r1[:, None] * (b - a) + r2[:, None] * (c - a)


def _segment_ids(counts: torch.Tensor) -> torch.Tensor:
    return torch.repeat_interleave(torch.arange(len(counts), device=counts.device), counts)


def _triangle_samples(tri: torch.Tensor, q: torch.Tensor, gen: torch.Generator, jitter_frac=0.8):
    """80 % jittered lattice + 20 % uniform samples in each triangle; returns points [sum q, 2]."""
    dev = tri.device
    n_j = torch.round(jitter_frac * q.double()).long()
    G = torch.ceil(torch.sqrt(n_j.double())).long().clamp(min=1)
    slots = G * G
    seg = _segment_ids(slots)
    start = torch.zeros_like(slots); start[1:] = torch.cumsum(slots, 0)[:-1]
    keys = seg.double() + torch.rand(len(seg), generator=gen, dtype=torch.float64, device=dev)
    order = torch.argsort(keys)                       # random order of lattice slots inside each cell
    slot_of_sorted = order - start[seg]               # lattice slot id at each sorted position
    rank = torch.arange(len(seg), device=dev) - start[seg]
    keep = rank < n_j[seg]
    cell_j = seg[keep]
    l = slot_of_sorted[keep]
    Gj = G[cell_j]
    u1 = (l % Gj).double() + torch.rand(len(l), generator=gen, dtype=torch.float64, device=dev)
    u2 = (l // Gj).double() + torch.rand(len(l), generator=gen, dtype=torch.float64, device=dev)
    pj = _fold_to_triangle(u1 / Gj, u2 / Gj, tri[cell_j, 0], tri[cell_j, 1], tri[cell_j, 2])
    n_u = q - n_j
    cell_u = _segment_ids(n_u)
    r = torch.rand(len(cell_u), 2, generator=gen, dtype=torch.float64, device=dev)
    pu = _fold_to_triangle(r[:, 0], r[:, 1], tri[cell_u, 0], tri[cell_u, 1], tri[cell_u, 2])
    cell = torch.cat([cell_j, cell_u])
    pts = torch.cat([pj, pu])
    o = torch.argsort(cell, stable=True)
    return pts[o]


def _hexagon_samples(hexv: torch.Tensor, q: torch.Tensor, gen: torch.Generator, clustered=0.3,
                     line_sd=0.02):
    dev = hexv.device
    n_c = torch.round(clustered * q.double()).long()
    n_u = q - n_c
    # uniform: a fan triangle (center, v_k, v_k+1) chosen uniformly, then the reflection map
    cu = _segment_ids(n_u)
    k = torch.randint(0, 6, (len(cu),), generator=gen, device=dev)
    ctr = hexv.mean(1)
    a = ctr[cu]
    b = hexv[cu, k]
    c = hexv[cu, (k + 1) % 6]
    r = torch.rand(len(cu), 2, generator=gen, dtype=torch.float64, device=dev)
    pu = _fold_to_triangle(r[:, 0], r[:, 1], a, b, c)
    # clustered: three random lines through the centroid, gaussian perpendicular offset, rejection
    cc = _segment_ids(n_c)
    line_ang = torch.rand(len(hexv), 3, generator=gen, dtype=torch.float64, device=dev) * math.pi
    side = (hexv[:, 1] - hexv[:, 0]).norm(dim=-1)
    apothem = side * math.sqrt(3) / 2
    hex_rot = torch.atan2(hexv[:, 0, 1] - ctr[:, 1], hexv[:, 0, 0] - ctr[:, 0])
    pc = torch.empty(len(cc), 2, dtype=torch.float64, device=dev)
    todo = torch.arange(len(cc), device=dev)
    while len(todo):
        cj = cc[todo]
        li = torch.randint(0, 3, (len(todo),), generator=gen, device=dev)
        ang = line_ang[cj, li]
        t = (torch.rand(len(todo), generator=gen, dtype=torch.float64, device=dev) * 2 - 1) * side[cj]
        o = torch.randn(len(todo), generator=gen, dtype=torch.float64, device=dev) * line_sd
        px = ctr[cj, 0] + t * ang.cos() - o * ang.sin()
        py = ctr[cj, 1] + t * ang.sin() + o * ang.cos()
        # inside test of a regular hexagon: |projection on the 3 apothem directions| <= apothem
        inside = torch.ones(len(todo), dtype=torch.bool, device=dev)
        for e in range(3):
            na = hex_rot[cj] + math.pi / 6 + e * math.pi / 3
            d = (px - ctr[cj, 0]) * na.cos() + (py - ctr[cj, 1]) * na.sin()
            inside &= d.abs() < apothem[cj] * (1 - 1e-9)
        pc[todo[inside]] = torch.stack([px[inside], py[inside]], -1)
        todo = todo[~inside]
    cell = torch.cat([cu, cc])
    pts = torch.cat([pu, pc])
    # interleave uniform and clustered samples randomly inside each cell
    keys = cell.double() + torch.rand(len(cell), generator=gen, dtype=torch.float64, device=dev)
    o = torch.argsort(keys)
    return pts[o]


# --------------------------------------------------------------------------------------
# terrain
# --------------------------------------------------------------------------------------

def _terrain(pts: torch.Tensor, cell: torch.Tensor, ctr: torch.Tensor, gen: torch.Generator,
             n_waves=200, dtype=torch.float64, chunk=1 << 20):
    """Power-law plane-wave sum plus one Gaussian ridge per cell, evaluated at the samples."""
    dev = pts.device
    n = len(ctr)
    kmag = 2 * math.pi * torch.exp(torch.rand(n, n_waves, generator=gen, dtype=torch.float64, device=dev)
                                   * math.log(20.0))
    kdir = torch.rand(n, n_waves, generator=gen, dtype=torch.float64, device=dev) * 2 * math.pi
    phase = torch.rand(n, n_waves, generator=gen, dtype=torch.float64, device=dev) * 2 * math.pi
    amp = 500.0 * (kmag / (2 * math.pi)) ** -1.5
    ridge = torch.rand(n, generator=gen, dtype=torch.float64, device=dev) * math.pi
    kx = (kmag * kdir.cos()).to(dtype)
    ky = (kmag * kdir.sin()).to(dtype)
    amp = amp.to(dtype)
    phase = phase.to(dtype)
    nx, ny = (-ridge.sin()).to(dtype), ridge.cos().to(dtype)
    out = torch.empty(len(pts), dtype=dtype, device=dev)
    for s in range(0, len(pts), chunk):
        e = min(len(pts), s + chunk)
        c = cell[s:e]
        px = pts[s:e, 0].to(dtype)[:, None]
        py = pts[s:e, 1].to(dtype)[:, None]
        arg = kx[c] * px + ky[c] * py + phase[c]
        hv = (amp[c] * torch.cos(arg)).sum(1)
        d = (px[:, 0] - ctr[c, 0].to(dtype)) * nx[c] + (py[:, 0] - ctr[c, 1].to(dtype)) * ny[c]
        hv = hv + 1000.0 * torch.exp(-d * d / (2 * 0.05 ** 2))
        out[s:e] = hv
    return out


# --------------------------------------------------------------------------------------
# configurations
# --------------------------------------------------------------------------------------

CONFIGS = {
    # one equilateral triangle, FP64 throughout, 32x32 modes, tol 1e-10
    "tri1_q2000_p32_fp64": dict(kind="single", n_cells=1, q=("fixed", 2000), modes=32, sigma=2.0,
                                width=8, tol=1e-10, precision="fp64"),
    # 20,480 icosahedral triangles, lognormal counts (median 4000, 500..20000), 64x64 modes
    "tri20480_p64": dict(kind="ico", level=5, q=("lognormal", 4000, 0.55, 500, 20000), modes=64,
                         sigma=2.0, width=7, tol=1e-6, precision="mixed"),
    # 81,920 icosahedral triangles, lognormal counts (median 6000, max 50000), 64x64 modes,
    # cells with <= 3000 samples routed to the tensor-core direct NUDFT
    "tri81920_p64_mixed": dict(kind="ico", level=6, q=("lognormal", 6000, 0.5, 500, 50000), modes=64,
                               sigma=2.0, width=7, tol=1e-6, precision="mixed", tc_max_points=3000),
    # 4,096 regular hexagons, 2k..8k samples (30 % clustered on ridge lines), 48x48 modes, gradients
    "hex4096_p48": dict(kind="hex", n_cells=4096, q=("uniform", 2000, 8000), modes=48, sigma=2.0,
                        width=7, tol=1e-6, precision="mixed", weights="jitter"),
    # 2,560 mixed triangles/hexagons, 100k..2M samples (heavy-tailed lognormal), 128x128 modes
    "mixed2560_p128": dict(kind="mixed", n_tri=1280, n_hex=1280, q=("lognormal", 3.0e5, 0.8, 1.0e5, 2.0e6),
                           modes=128, sigma=2.0, width=6, tol=1e-5, precision="mixed"),
}


def _counts(spec, n, gen, dev, q_scale):
    kind = spec[0]
    if kind == "fixed":
        q = torch.full((n,), spec[1], dtype=torch.float64, device=dev)
    elif kind == "lognormal":
        _, med, sd, lo, hi = spec
        z = torch.randn(n, generator=gen, dtype=torch.float64, device=dev)
        q = torch.exp(math.log(med) + sd * z).clamp(lo, hi)
    elif kind == "uniform":
        _, lo, hi = spec
        q = torch.randint(lo, hi + 1, (n,), generator=gen, device=dev).double()
    else:
        raise ValueError(kind)
    return torch.round(q * q_scale).long().clamp(min=1)


def make(name: str, seed: int = 0, device="cpu", n_cells: int | None = None, q_scale: float = 1.0,
         dtype: torch.dtype | None = None) -> Workload:
    """Draw workload `name` with a given seed on `device`.

    n_cells limits the batch to a seeded subset of cells; q_scale scales every cell's sample
    count (both exist so that the same recipe also yields oracle-sized cases).
    """
    spec = CONFIGS[name]
    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(1000 * (list(CONFIGS).index(name) + 1) + seed)
    # geometry is drawn on the CPU in float64 (cheap), samples on `device`
    cgen = torch.Generator()
    cgen.manual_seed(7919 * (list(CONFIGS).index(name) + 1) + seed)
    kind = spec["kind"]
    if kind == "single":
        tri = torch.tensor([[[0.0, 0.0], [1.0, 0.0], [0.5, math.sqrt(3) / 2]]], dtype=torch.float64)
        tri = tri - tri.mean(1, keepdim=True)
        polys = [("tri", tri)]
    elif kind == "ico":
        faces = _project_faces(_icosahedron(spec["level"]), cgen)
        if n_cells is not None and n_cells < len(faces):
            faces = faces[torch.randperm(len(faces), generator=cgen)[:n_cells]]
        polys = [("tri", faces)]
    elif kind == "hex":
        polys = [("hex", _hexagons(n_cells or spec["n_cells"], cgen))]
    elif kind == "mixed":
        nt, nh = spec["n_tri"], spec["n_hex"]
        if n_cells is not None:
            nt = (n_cells + 1) // 2
            nh = n_cells - nt
        faces = _project_faces(_icosahedron(5), cgen)
        faces = faces[torch.randperm(len(faces), generator=cgen)[:nt]]
        polys = [("tri", faces), ("hex", _hexagons(nh, cgen))]
    else:
        raise ValueError(kind)

    nverts, verts, pts_all, cells_all, areas, counts = [], [], [], [], [], []
    base = 0
    for pk, pv in polys:
        n = len(pv)
        if n == 0:
            continue
        q = _counts(spec["q"], n, gen, dev, q_scale)
        pvd = pv.to(dev)
        if pk == "tri":
            pts = _triangle_samples(pvd, q, gen)
            area = _tri_area(pvd)
            vv = torch.zeros(n, 6, 2, dtype=torch.float64, device=dev); vv[:, :3] = pvd
            nv = torch.full((n,), 3, dtype=torch.int32, device=dev)
        else:
            pts = _hexagon_samples(pvd, q, gen)
            side = (pvd[:, 1] - pvd[:, 0]).norm(dim=-1)
            area = 1.5 * math.sqrt(3) * side * side
            vv = pvd.clone()
            nv = torch.full((n,), 6, dtype=torch.int32, device=dev)
        nverts.append(nv); verts.append(vv); pts_all.append(pts); areas.append(area); counts.append(q)
        cells_all.append(_segment_ids(q) + base)
        base += n
    nverts = torch.cat(nverts); verts = torch.cat(verts); pts = torch.cat(pts_all)
    cell = torch.cat(cells_all); area = torch.cat(areas); q = torch.cat(counts)
    offsets = torch.zeros(len(q) + 1, dtype=torch.int64, device=dev)
    offsets[1:] = torch.cumsum(q, 0)

    prec = spec["precision"]
    if dtype is None:
        dtype = torch.float64 if prec == "fp64" else torch.float32
    ctr = verts.sum(1) / nverts[:, None].double()
    h = _terrain(pts, cell, ctr, gen, dtype=torch.float64 if dtype == torch.float64 else torch.float32)
    w = (area / q.double())[cell]
    if spec.get("weights") == "jitter":
        jw = 1.0 + 0.5 * (torch.rand(len(w), generator=gen, dtype=torch.float64, device=dev) * 2 - 1)
        tot = torch.zeros(len(q), dtype=torch.float64, device=dev).index_add_(0, cell, jw)
        w = jw * (area / tot)[cell]
    return Workload(name=name, n_cells=len(q), nverts=nverts, verts=verts, offsets=offsets,
                    x=pts[:, 0].to(dtype).contiguous(), y=pts[:, 1].to(dtype).contiguous(),
                    h=h.to(dtype).contiguous(), w=w.to(dtype).contiguous(),
                    modes=spec["modes"], sigma=spec["sigma"], width=spec["width"], tol=spec["tol"],
                    precision=prec, tc_max_points=spec.get("tc_max_points", 0),
                    meta=dict(seed=seed, q_scale=q_scale))


# --------------------------------------------------------------------------------------
# analytic test cases (closed-form answers are known for these)
# --------------------------------------------------------------------------------------

def regular_grid_square_cell(n: int, field, half: float = 0.75, center=(0.0, 0.0), modes: int = 8,
                             dtype=torch.float64, offset: float = 0.0, ny: int | None = None) -> Workload:
    """One square cell [-half, half]^2 + center sampled on an equispaced n x ny grid at
    x' = (r + offset) L / n (offset 0: starts at the lower-left corner; 0.5: cell midpoints), with
    uniform weights L^2 / (n ny); `field(xp, yp)` gives h as a function of the square-domain
    coordinates x' = x - center + half."""
    L = 2 * half
    ny = ny or n
    rx = torch.arange(n, dtype=torch.float64)
    ry = torch.arange(ny, dtype=torch.float64)
    xp = ((rx + offset) * L / n)[None, :].expand(ny, n).reshape(-1)
    yp = ((ry + offset) * L / ny)[:, None].expand(ny, n).reshape(-1)
    h = field(xp, yp)
    verts = torch.zeros(1, 6, 2, dtype=torch.float64)
    sq = torch.tensor([[-half, -half], [half, -half], [half, half], [-half, half]], dtype=torch.float64)
    verts[0, :4] = sq + torch.tensor(center, dtype=torch.float64)
    # a square is described with 4 vertices; the eta that makes the window equal the square is 1
    return Workload(name="regular_grid", n_cells=1, nverts=torch.tensor([4], dtype=torch.int32),
                    verts=verts, offsets=torch.tensor([0, n * ny], dtype=torch.int64),
                    x=(xp - half + center[0]).to(dtype), y=(yp - half + center[1]).to(dtype),
                    h=h.to(dtype), w=torch.full((n * ny,), L * L / (n * ny), dtype=dtype),
                    modes=modes, eta=1.0, mask=1, precision="fp64", width=12, tol=1e-12)


def plane_wave_cell(q: int, amp: float, m: int, n: int, phase: float, gen: torch.Generator,
                    half: float = 0.75, modes: int = 8, dtype=torch.float64) -> Workload:
    """One square cell with q uniform random samples of h = amp cos(k_m x' + k_n y' + phase)."""
    L = 2 * half
    xp = torch.rand(q, generator=gen, dtype=torch.float64) * L
    yp = torch.rand(q, generator=gen, dtype=torch.float64) * L
    h = amp * torch.cos(2 * math.pi * (m * xp + n * yp) / L + phase)
    verts = torch.zeros(1, 6, 2, dtype=torch.float64)
    verts[0, :4] = torch.tensor([[-half, -half], [half, -half], [half, half], [-half, half]],
                                dtype=torch.float64)
    return Workload(name="plane_wave", n_cells=1, nverts=torch.tensor([4], dtype=torch.int32),
                    verts=verts, offsets=torch.tensor([0, q], dtype=torch.int64),
                    x=(xp - half).to(dtype), y=(yp - half).to(dtype), h=h.to(dtype),
                    w=torch.full((q,), L * L / q, dtype=dtype), modes=modes, eta=1.0, mask=1,
                    precision="fp64", width=12, tol=1e-12)


# --------------------------------------------------------------------------------------
# monochromatic sweep (Sec. 3.1, Table mono_sweep_config)
# --------------------------------------------------------------------------------------

MONO_AXES = dict(dy=(-0.211, -0.077, 0.0), theta=(0.0, 60.0, 120.0, 180.0, 240.0, 300.0), u=(0.0, 0.5, 1.0),
                 r_exp=(1.0, 1.5, 2.0), Q=(500, 1000, 2000), sigma=(1.25, 1.5, 2.0), k_max=(4, 6, 8, 10))


def mono_sweep(r_exp: float, seed: int = 0, amplitude: float = 1000.0, modes: int = 16) -> tuple[Workload, dict]:
    """One cell per (dy, theta, u, Q) of the monochromatic sweep at expansion ratio r_exp.

    A cell is a triangle of base 1 and height (1 + u)/2 * sqrt(3)/2 (u = 1 equilateral), rotated by
    theta about its centroid (the origin of its coordinates).  Its window is the square of side
    L = 2H, H = (r_exp/2) * max extent; the sample domain D is that square moved by dy * L
    vertically (the triangle sits dy * L above the domain's centre), with Q samples uniform on D.
    D is split into four regions -- the triangle and the three sectors cut by the rays from the
    centroid through the vertices -- each carrying one monochromatic elevation
    A cos(2 pi (m x' + n y') / L + phi) with x' = x + H, y' = y + H, integer (m, n) drawn per region
    (the triangle's mode different from its neighbours' and their negatives) and a random phase.
    Weights are uniform, |D| / Q.  Returns the workload (cell mask, eta = r_exp) and per-cell
    metadata: dy, theta, u, Q and the triangle's mode (m_T, n_T)."""
    gen = torch.Generator()
    gen.manual_seed(424242 + int(1000 * r_exp) + seed)
    verts, xs, ys, hs, ws, counts = [], [], [], [], [], []
    meta = {k: [] for k in ("dy", "theta", "u", "Q", "m", "n")}
    for dy in MONO_AXES["dy"]:
        for th in MONO_AXES["theta"]:
            for u in MONO_AXES["u"]:
                for Q in MONO_AXES["Q"]:
                    hgt = 0.5 * (1.0 + u) * math.sqrt(3.0) / 2.0
                    tri = torch.tensor([[-0.5, -hgt / 3], [0.5, -hgt / 3], [0.0, 2 * hgt / 3]], dtype=torch.float64)
                    a = math.radians(th)
                    rot = torch.tensor([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]], dtype=torch.float64)
                    tri = tri @ rot.T
                    ext = max(float(tri[:, 0].max() - tri[:, 0].min()), float(tri[:, 1].max() - tri[:, 1].min()))
                    H = 0.5 * r_exp * ext
                    L = 2 * H
                    pts = (torch.rand(Q, 2, generator=gen, dtype=torch.float64) - 0.5) * L
                    pts[:, 1] -= dy * L
                    # regions: 0 the triangle, 1..3 the sectors between consecutive vertex rays
                    inside = torch.ones(Q, dtype=torch.bool)
                    for i in range(3):
                        p0, p1 = tri[i], tri[(i + 1) % 3]
                        cr = (p1[0] - p0[0]) * (pts[:, 1] - p0[1]) - (p1[1] - p0[1]) * (pts[:, 0] - p0[0])
                        inside &= cr >= 0
                    va = torch.atan2(tri[:, 1], tri[:, 0])
                    order = torch.argsort(va)
                    pa = torch.atan2(pts[:, 1], pts[:, 0])
                    sector = torch.zeros(Q, dtype=torch.long)
                    for k in range(3):
                        lo, hi = va[order[k]], va[order[(k + 1) % 3]]
                        sel = ((pa >= lo) & (pa < hi)) if k < 2 else ((pa >= lo) | (pa < hi))
                        sector[sel] = k + 1
                    region = torch.where(inside, torch.zeros_like(sector), sector)
                    # one mode per region; the triangle's differs from the others and their negatives
                    mt = int(torch.randint(1, 5, (1,), generator=gen))
                    nt = int(torch.randint(-4, 5, (1,), generator=gen))
                    mods = [(mt, nt)]
                    while len(mods) < 4:
                        mm = int(torch.randint(-4, 5, (1,), generator=gen))
                        nn = int(torch.randint(-4, 5, (1,), generator=gen))
                        if (mm, nn) not in ((0, 0), (mt, nt), (-mt, -nt)):
                            mods.append((mm, nn))
                    phase = torch.rand(4, generator=gen, dtype=torch.float64) * 2 * math.pi
                    km = torch.tensor([mm for mm, _ in mods], dtype=torch.float64)[region]
                    kn = torch.tensor([nn for _, nn in mods], dtype=torch.float64)[region]
                    xp, yp = pts[:, 0] + H, pts[:, 1] + H
                    h = amplitude * torch.cos(2 * math.pi * (km * xp + kn * yp) / L + phase[region])
                    vv = torch.zeros(6, 2, dtype=torch.float64)
                    vv[:3] = tri
                    verts.append(vv)
                    xs.append(pts[:, 0]); ys.append(pts[:, 1]); hs.append(h)
                    ws.append(torch.full((Q,), L * L / Q, dtype=torch.float64))
                    counts.append(Q)
                    for k, v in (("dy", dy), ("theta", th), ("u", u), ("Q", Q), ("m", mt), ("n", nt)):
                        meta[k].append(v)
    n = len(counts)
    off = torch.zeros(n + 1, dtype=torch.int64)
    off[1:] = torch.cumsum(torch.tensor(counts), 0)
    wl = Workload(name=f"mono_rexp{r_exp}", n_cells=n, nverts=torch.full((n,), 3, dtype=torch.int32),
                  verts=torch.stack(verts), offsets=off, x=torch.cat(xs).float(), y=torch.cat(ys).float(),
                  h=torch.cat(hs).float(), w=torch.cat(ws).float(), modes=modes, sigma=2.0, width=7, tol=1e-6,
                  precision="mixed", eta=r_exp, mask=0)
    return wl, {k: np.asarray(v) for k, v in meta.items()}
