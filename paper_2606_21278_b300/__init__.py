"""Python binding of the B300 ENUFFT library (libenufft.so, C ABI in include/enufft.h).

Argument marshalling only: tensors are passed to the C ABI by device pointer on the caller's
current CUDA stream, and every step of the transform, the mode selection and the adjoint runs in
the library's kernels.  There is no fallback: if the compiled library is missing, or no CUDA
device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

__all__ = ["Plan", "EMSParams", "EMSRetainedPower", "load_library", "LIB_PATH", "EnufftError", "tune_cache_lookup",
           "tune_cache_store", "probe_peaks"]

LIB_PATH = os.environ.get("ENUFFT_LIB", os.path.join(os.path.dirname(os.path.abspath(__file__)), "libenufft.so"))
_lib = None

_PREC = {"fp64": 0, "fp32": 1, "mixed": 2}
_KERNEL = {"es": 0, "kb": 1}
_FRAME = {"centroid": 0, "edge": 1}
_MASK = {"cell": 0, "square": 1, "circle": 2}


class EnufftError(RuntimeError):
    pass


class _Opts(ctypes.Structure):
    _fields_ = [("modes", ctypes.c_int), ("oversamp", ctypes.c_double), ("kernel_width", ctypes.c_int),
                ("tol", ctypes.c_double), ("prec", ctypes.c_int), ("mask", ctypes.c_int),
                ("eta", ctypes.c_double), ("tc_max_points", ctypes.c_int), ("kernel", ctypes.c_int),
                ("frame", ctypes.c_int), ("autotune", ctypes.c_int), ("tune_cache", ctypes.c_char_p),
                ("deterministic", ctypes.c_int)]


class _Ems(ctypes.Structure):
    _fields_ = [("k_min", ctypes.c_int), ("k_max", ctypes.c_int), ("alpha_min", ctypes.c_double),
                ("alpha_max", ctypes.c_double), ("delta", ctypes.c_double), ("w1", ctypes.c_double),
                ("w2", ctypes.c_double), ("sum_over", ctypes.c_int), ("include_dc", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("modes", ctypes.c_int), ("fine_grid", ctypes.c_int), ("kernel_width", ctypes.c_int),
                ("beta", ctypes.c_double), ("oversamp_effective", ctypes.c_double),
                ("n_cells", ctypes.c_int64), ("n_points", ctypes.c_int64), ("cells_fused", ctypes.c_int64),
                ("cells_tensor", ctypes.c_int64), ("cells_large", ctypes.c_int64), ("precision", ctypes.c_int),
                ("cells_plain", ctypes.c_int64), ("kernels_per_type1_ems", ctypes.c_int64),
                ("kernel", ctypes.c_int), ("frame", ctypes.c_int), ("tc_max_points", ctypes.c_int),
                ("autotuned", ctypes.c_int), ("fused_blocks_per_sm", ctypes.c_int), ("large_tile", ctypes.c_int)]


class _Tuning(ctypes.Structure):
    _fields_ = [("tc_max_points", ctypes.c_int), ("fused_blocks_per_sm", ctypes.c_int), ("n_ladder", ctypes.c_int),
                ("ladder", ctypes.c_int * 8), ("ns_fused", ctypes.c_double * 8), ("ns_tc", ctypes.c_double * 8),
                ("from_cache", ctypes.c_int), ("large_tile", ctypes.c_int)]


def _tuning_dict(t: _Tuning) -> dict:
    n = t.n_ladder
    return {"tc_max_points": t.tc_max_points, "fused_blocks_per_sm": t.fused_blocks_per_sm,
            "ladder": list(t.ladder[:n]), "ns_fused": list(t.ns_fused[:n]), "ns_tc": list(t.ns_tc[:n]),
            "from_cache": bool(t.from_cache), "large_tile": t.large_tile}


def load_library(path: str = LIB_PATH):
    """Load libenufft.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise EnufftError(f"{path} not found: build it with `python -m paper_2606_21278_b300.build`")
    lib = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    P = ctypes.POINTER
    lib.enufft_default_opts.argtypes = [P(_Opts)]
    lib.enufft_default_opts.restype = None
    lib.enufft_default_ems.argtypes = [P(_Ems)]
    lib.enufft_default_ems.restype = None
    lib.enufft_plan_create.argtypes = [P(vp), P(_Opts), i64, vp, vp, vp, vp]
    lib.enufft_plan_destroy.argtypes = [vp]
    lib.enufft_type1.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.enufft_ems.argtypes = [vp, vp, vp, i32, P(_Ems), vp, vp, vp]
    lib.enufft_type1_ems.argtypes = [vp, vp, vp, vp, vp, vp, vp, i32, P(_Ems), vp, vp, vp]
    lib.enufft_type1_ems_graph.argtypes = [vp, vp, vp, vp, vp, vp, vp, i32, P(_Ems), vp, vp, vp]
    lib.enufft_ems_backward.argtypes = [vp, vp, vp, i32, P(_Ems), vp, vp, vp, vp]
    lib.enufft_type1_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    lib.enufft_sync_status.argtypes = [vp]
    lib.enufft_plan_sync_status.argtypes = [vp]
    lib.enufft_set_stream.argtypes = [vp, vp]
    lib.enufft_last_error.argtypes = [vp]
    lib.enufft_last_error.restype = ctypes.c_char_p
    lib.enufft_get_plan_info.argtypes = [vp, P(_Info)]
    lib.enufft_selftest_wait_timeout.argtypes = [vp, ctypes.c_uint]
    lib.enufft_reconstruct.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp, vp, vp, vp]
    lib.enufft_voronoi_weights.argtypes = [vp, vp, vp, i32, vp]
    lib.enufft_get_tuning.argtypes = [vp, P(_Tuning)]
    lib.enufft_tune_cache_lookup.argtypes = [ctypes.c_char_p, ctypes.c_char_p, P(_Tuning)]
    lib.enufft_tune_cache_store.argtypes = [ctypes.c_char_p, ctypes.c_char_p, P(_Tuning)]
    for f in ("enufft_plan_create", "enufft_plan_destroy", "enufft_type1", "enufft_ems", "enufft_type1_ems",
              "enufft_type1_ems_graph", "enufft_ems_backward", "enufft_type1_backward", "enufft_sync_status",
              "enufft_plan_sync_status", "enufft_set_stream",
              "enufft_get_plan_info", "enufft_selftest_wait_timeout", "enufft_reconstruct",
              "enufft_voronoi_weights", "enufft_get_tuning", "enufft_tune_cache_lookup", "enufft_tune_cache_store"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


@dataclass
class EMSParams:
    """Sec. 2.2 parameters (defaults: the paper's EMS illustration)."""
    k_min: int = 1
    k_max: int = 12
    alpha_min: float = 0.0
    alpha_max: float = 0.7
    delta: float = 0.02
    w1: float = 0.5
    w2: float = 0.5
    sum_over: int = 0
    include_dc: int = 0

    def c(self) -> _Ems:
        return _Ems(self.k_min, self.k_max, self.alpha_min, self.alpha_max, self.delta, self.w1, self.w2,
                    self.sum_over, self.include_dc)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Plan:
    """A plan over a fixed set of cells and CSR sample offsets (see enufft_plan_create)."""

    def __init__(self, offsets: torch.Tensor, nverts: torch.Tensor, verts: torch.Tensor, modes: int = 64,
                 oversamp: float = 2.0, kernel_width: int = 7, tol: float = 0.0, precision: str = "mixed",
                 mask: str | int = "cell", eta: float = 1.5, tc_max_points: int = 0, kernel: str = "es",
                 frame: str | int = "centroid", autotune: bool = False, tune_cache: str | None = None,
                 deterministic: bool = True):
        self._lib = load_library()
        if not torch.cuda.is_available():
            raise EnufftError("no CUDA device")
        dev = torch.device("cuda", torch.cuda.current_device())
        self.offsets = offsets.to(dev, torch.int64).contiguous()
        self.nverts = nverts.to(dev, torch.int32).contiguous()
        self.verts = verts.to(dev, torch.float64).reshape(-1, 6, 2).contiguous()
        self.n_cells = len(self.nverts)
        self.modes = modes
        self.precision = precision
        self.real_dtype = torch.float64 if precision == "fp64" else torch.float32
        self.complex_dtype = torch.complex128 if precision == "fp64" else torch.complex64
        if kernel not in _KERNEL:
            raise EnufftError(f"kernel must be one of {sorted(_KERNEL)}")
        if isinstance(frame, str) and frame not in _FRAME:
            raise EnufftError(f"frame must be one of {sorted(_FRAME)}")
        o = _Opts(modes, oversamp, kernel_width, tol, _PREC[precision],
                  _MASK[mask] if isinstance(mask, str) else int(mask), eta, tc_max_points, _KERNEL[kernel],
                  _FRAME[frame] if isinstance(frame, str) else int(frame), int(bool(autotune)),
                  tune_cache.encode() if tune_cache else None, int(bool(deterministic)))
        h = ctypes.c_void_p()
        st = self._lib.enufft_plan_create(ctypes.byref(h), ctypes.byref(o), self.n_cells, _ptr(self.offsets),
                                          _ptr(self.nverts), _ptr(self.verts), _stream())
        if st != 0:
            raise EnufftError(f"enufft_plan_create: status {st}: {self._lib.enufft_last_error(None).decode()}")
        self._h = h
        self.n_points = int(self.offsets[-1]) if self.n_cells else 0

    @classmethod
    def for_workload(cls, wl, **kw) -> "Plan":
        args = dict(modes=wl.modes, oversamp=wl.sigma, kernel_width=wl.width, tol=wl.tol,
                    precision="fp64" if wl.precision == "fp64" else "mixed", mask=wl.mask, eta=wl.eta,
                    tc_max_points=wl.tc_max_points, frame=int(getattr(wl, "frame", 0)))
        args.update(kw)
        return cls(wl.offsets, wl.nverts, wl.verts, **args)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.enufft_plan_destroy(h)
            self._h = None

    def _check(self, st, what):
        if st != 0:
            raise EnufftError(f"{what}: status {st}: {self._lib.enufft_last_error(self._h).decode()}")

    def _bind(self):
        self._check(self._lib.enufft_set_stream(self._h, _stream()), "set_stream")

    def _samples(self, *ts):
        out = []
        for t in ts:
            if t.dtype != self.real_dtype or not t.is_cuda or not t.is_contiguous() or t.numel() != self.n_points:
                raise EnufftError(f"sample arrays must be contiguous CUDA {self.real_dtype} of length {self.n_points}")
            out.append(t)
        return out

    def info(self) -> dict:
        i = _Info()
        self._check(self._lib.enufft_get_plan_info(self._h, ctypes.byref(i)), "get_plan_info")
        return {f: getattr(i, f) for f, _ in _Info._fields_}

    def tuning(self) -> dict:
        """The plan's route tuning record (see enufft_get_tuning); raises if the plan was not tuned."""
        t = _Tuning()
        self._check(self._lib.enufft_get_tuning(self._h, ctypes.byref(t)), "get_tuning")
        return _tuning_dict(t)

    def voronoi_weights(self, x, y, ng: int = 64) -> torch.Tensor:
        """Voronoi quadrature weights by raster sampling (see enufft_voronoi_weights)."""
        x, y = self._samples(x, y)
        w = torch.empty_like(x)
        self._bind()
        self._check(self._lib.enufft_voronoi_weights(self._h, _ptr(x), _ptr(y), int(ng), _ptr(w)), "voronoi_weights")
        return w

    def reconstruct(self, coeffs, kstar, sel, x, y, h, w, want_hrec: bool = True):
        """Sec. 3.2 diagnostics (see enufft_reconstruct): (h_rec at the samples or None,
        stats[n_cells, 4] float64 = eps_rel, sigma2_phys, sigma2_spec over the selection, over the box)."""
        x, y, h, w = self._samples(x, y, h, w)
        hrec = torch.empty_like(h) if want_hrec else None
        stats = torch.empty(self.n_cells, 4, dtype=torch.float64, device=h.device)
        ks = kstar.to(torch.int32).contiguous()
        sl = sel.to(torch.int32).contiguous()
        self._bind()
        self._check(self._lib.enufft_reconstruct(self._h, _ptr(coeffs.contiguous()), _ptr(ks), _ptr(sl), sl.shape[1],
                                                 _ptr(x), _ptr(y), _ptr(h), _ptr(w), _ptr(hrec), _ptr(stats)),
                    "reconstruct")
        return hrec, stats

    def selftest_wait_timeout(self, polls: int = 64):
        """Latch a bounded-wait timeout on the device (see enufft_selftest_wait_timeout)."""
        self._bind()
        self._check(self._lib.enufft_selftest_wait_timeout(self._h, polls), "selftest_wait_timeout")

    def sync_status(self):
        self._check(self._lib.enufft_sync_status(self._h), "sync_status")

    def new_coeffs(self) -> torch.Tensor:
        return torch.empty(self.n_cells, self.modes, self.modes, dtype=self.complex_dtype, device=self.offsets.device)

    def type1(self, x, y, h, w, coeffs: torch.Tensor | None = None) -> torch.Tensor:
        x, y, h, w = self._samples(x, y, h, w)
        coeffs = self.new_coeffs() if coeffs is None else coeffs
        self._bind()
        self._check(self._lib.enufft_type1(self._h, _ptr(x), _ptr(y), _ptr(h), _ptr(w), _ptr(coeffs)), "type1")
        return coeffs

    def new_ems_out(self, params: EMSParams = EMSParams()):
        """Preallocated EMS outputs (kstar, sel, retained) for `type1_ems(out=...)` and
        `type1_ems_graph`."""
        return self._ems_out(params)

    def _ems_out(self, params: EMSParams):
        dev = self.offsets.device
        return (torch.empty(self.n_cells, dtype=torch.int32, device=dev),
                torch.empty(self.n_cells, params.k_max, dtype=torch.int32, device=dev),
                torch.empty(self.n_cells, dtype=torch.float64, device=dev))

    @staticmethod
    def _weights(mode_weights):
        if mode_weights is None:
            return None, 0
        mw = mode_weights.to(torch.float64).contiguous()
        return mw, int(mw.dim() == 3)

    def ems(self, coeffs, params: EMSParams = EMSParams(), mode_weights=None):
        ks, sel, ret = self._ems_out(params)
        mw, per = self._weights(mode_weights)
        pc = params.c()
        self._bind()
        self._check(self._lib.enufft_ems(self._h, _ptr(coeffs), _ptr(mw), per, ctypes.byref(pc), _ptr(ks),
                                         _ptr(sel), _ptr(ret)), "ems")
        return ks, sel, ret

    def type1_ems(self, x, y, h, w, params: EMSParams = EMSParams(), mode_weights=None, coeffs=None, out=None):
        """Coefficients and EMS in one call; `coeffs` and `out` = (kstar, sel, retained) may be
        preallocated (e.g. for capture in a CUDA graph)."""
        x, y, h, w = self._samples(x, y, h, w)
        coeffs = self.new_coeffs() if coeffs is None else coeffs
        ks, sel, ret = self._ems_out(params) if out is None else out
        mw, per = self._weights(mode_weights)
        pc = params.c()
        self._bind()
        self._check(self._lib.enufft_type1_ems(self._h, _ptr(x), _ptr(y), _ptr(h), _ptr(w), _ptr(coeffs), _ptr(mw),
                                               per, ctypes.byref(pc), _ptr(ks), _ptr(sel), _ptr(ret)), "type1_ems")
        return coeffs, ks, sel, ret

    def type1_ems_graph(self, x, y, h, w, coeffs, out, params: EMSParams = EMSParams(), mode_weights=None):
        """type1_ems through the plan's own CUDA graph (enufft_type1_ems_graph): captured on the first
        call and again whenever a buffer or parameter changes, replayed otherwise.  `coeffs` and
        `out` = (kstar, sel, retained) must stay allocated while the graph may replay."""
        x, y, h, w = self._samples(x, y, h, w)
        ks, sel, ret = out
        mw, per = self._weights(mode_weights)
        self._graph_keep = (x, y, h, w, coeffs, ks, sel, ret, mw)   # buffers the graph reads or writes
        pc = params.c()
        self._bind()
        self._check(self._lib.enufft_type1_ems_graph(self._h, _ptr(x), _ptr(y), _ptr(h), _ptr(w), _ptr(coeffs),
                                                     _ptr(mw), per, ctypes.byref(pc), _ptr(ks), _ptr(sel),
                                                     _ptr(ret)), "type1_ems_graph")
        return coeffs, ks, sel, ret

    def ems_backward(self, coeffs, kstar, sel, grad_power, params: EMSParams = EMSParams(), mode_weights=None):
        g = torch.empty_like(coeffs)
        mw, per = self._weights(mode_weights)
        pc = params.c()
        gp = grad_power.to(torch.float64).contiguous()
        self._bind()
        self._check(self._lib.enufft_ems_backward(self._h, _ptr(coeffs), _ptr(mw), per, ctypes.byref(pc), _ptr(kstar),
                                                  _ptr(sel), _ptr(gp), _ptr(g)), "ems_backward")
        return g

    def type1_backward(self, grad_coeffs, x, y, h, w, need_h: bool = True, need_w: bool = True):
        x, y, h, w = self._samples(x, y, h, w)
        gh = torch.empty_like(h) if need_h else None
        gw = torch.empty_like(w) if need_w else None
        g = grad_coeffs.to(self.complex_dtype).contiguous()
        self._bind()
        self._check(self._lib.enufft_type1_backward(self._h, _ptr(g), _ptr(x), _ptr(y), _ptr(h), _ptr(w), _ptr(gh),
                                                    _ptr(gw)), "type1_backward")
        return gh, gw


class EMSRetainedPower(torch.autograd.Function):
    """Per-cell EMS-retained launch power  P_j = sum_{p in S_j} W_p (|h_p|^2 + |h_-p|^2)  as a function
    of the sample elevations h and weights w (Sec. 2.2 on the spectra of App. B), with a hand-written
    backward: the selection S_j is held fixed, dP/dh and dP/dw come from enufft_ems_backward and the
    type-2 adjoint enufft_type1_backward.  Returns (power[n_cells] float64, coeffs, kstar, sel)."""

    @staticmethod
    def forward(ctx, h, w, plan: Plan, x, y, params: EMSParams = EMSParams(), mode_weights=None):
        coeffs, ks, sel, ret = plan.type1_ems(x, y, h.detach(), w.detach(), params, mode_weights)
        ctx.plan, ctx.params, ctx.mw = plan, params, mode_weights
        ctx.save_for_backward(h, w, x, y, coeffs, ks, sel)
        ctx.mark_non_differentiable(coeffs, ks, sel)
        return ret, coeffs, ks, sel

    @staticmethod
    def backward(ctx, grad_power, _gc, _gk, _gs):
        h, w, x, y, coeffs, ks, sel = ctx.saved_tensors
        plan = ctx.plan
        g = plan.ems_backward(coeffs, ks, sel, grad_power, ctx.params, ctx.mw)
        gh, gw = plan.type1_backward(g, x, y, h.detach(), w.detach(), ctx.needs_input_grad[0], ctx.needs_input_grad[1])
        return gh, gw, None, None, None, None, None


class _Peaks(ctypes.Structure):
    _fields_ = [("fp32_tflops", ctypes.c_double), ("f16_tflops", ctypes.c_double),
                ("smem_red_u32_gops", ctypes.c_double), ("smem_red_u32_random_gops", ctypes.c_double),
                ("smem_red_f32_gops", ctypes.c_double), ("num_sms", ctypes.c_int)]


def probe_peaks() -> dict:
    """Compute peaks of the current GPU (see enufft_probe_peaks), on the current stream."""
    lib = load_library()
    lib.enufft_probe_peaks.argtypes = [ctypes.POINTER(_Peaks), ctypes.c_void_p]
    lib.enufft_probe_peaks.restype = ctypes.c_int
    p = _Peaks()
    st = lib.enufft_probe_peaks(ctypes.byref(p), _stream())
    if st != 0:
        raise EnufftError(f"probe_peaks: status {st}: {lib.enufft_last_error(None).decode()}")
    return {f: getattr(p, f) for f, _ in _Peaks._fields_}


def tune_cache_lookup(path: str, key: str) -> dict | None:
    """The record of `key` in a tuning cache file, or None (see enufft_tune_cache_lookup)."""
    lib = load_library()
    t = _Tuning()
    if lib.enufft_tune_cache_lookup(path.encode(), key.encode(), ctypes.byref(t)) != 0:
        return None
    return _tuning_dict(t)


def tune_cache_store(path: str, key: str, rec: dict) -> None:
    """Store a tuning record under `key` (see enufft_tune_cache_store)."""
    lib = load_library()
    t = _Tuning()
    t.tc_max_points = int(rec["tc_max_points"])
    t.fused_blocks_per_sm = int(rec["fused_blocks_per_sm"])
    t.large_tile = int(rec.get("large_tile", 0))
    n = len(rec.get("ladder", []))
    t.n_ladder = n
    for i in range(n):
        t.ladder[i] = int(rec["ladder"][i])
        t.ns_fused[i] = float(rec["ns_fused"][i])
        t.ns_tc[i] = float(rec["ns_tc"][i])
    if lib.enufft_tune_cache_store(path.encode(), key.encode(), ctypes.byref(t)) != 0:
        raise EnufftError(f"tune_cache_store: {lib.enufft_last_error(None).decode()}")
