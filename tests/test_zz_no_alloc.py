"""The allocation-free EMS entry point (enufft_ems_noalloc) against the planned enufft_ems.

enufft_ems_noalloc exists for callers that cannot allocate device memory when they need the mode
selection (a cudaMalloc there would synchronise the device, or another allocator owns the memory);
its scratch is a fixed static device array shared by all calls.  This file runs last so that a
failure here cannot hide the result of any other test; it also passes on its own.
"""
import ctypes

import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

enufft = pytest.importorskip("paper_2606_21278_b300")


def _lib():
    lib = enufft.load_library()
    vp = ctypes.c_void_p
    lib.enufft_ems_noalloc.argtypes = [ctypes.c_int, ctypes.c_int64, vp, vp, ctypes.c_int,
                                       ctypes.POINTER(enufft._Ems), vp, vp, vp, vp]
    lib.enufft_ems_noalloc.restype = ctypes.c_int
    return lib


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def test_ems_noalloc_matches_planned_ems_on_two_calls():
    lib = _lib()
    wl = synth.make("tri20480_p64", seed=21, n_cells=96, q_scale=0.2)
    g = wl.to("cuda")
    plan = enufft.Plan.for_workload(g)
    coeffs = plan.type1(g.x, g.y, g.h, g.w)
    W = torch.rand(wl.n_cells, 64, 64, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for prm, mw in ((enufft.EMSParams(), None), (enufft.EMSParams(k_min=3, k_max=64, sum_over=1), None),
                    (enufft.EMSParams(include_dc=1, k_max=20), W)):
        ks_ref, sel_ref, ret_ref = plan.ems(coeffs, prm, mode_weights=mw)
        for _ in range(2):   # the shared scratch keeps the previous call's contents
            ks = torch.full_like(ks_ref, -7)
            sel = torch.full_like(sel_ref, -7)
            ret = torch.full_like(ret_ref, float("nan"))
            pc = prm.c()
            st = lib.enufft_ems_noalloc(64, wl.n_cells, _p(coeffs), _p(mw), int(mw is not None), ctypes.byref(pc),
                                        _p(ks), _p(sel), _p(ret), stream)
            assert st == 0, lib.enufft_last_error(None).decode()
            torch.cuda.synchronize()
            assert torch.equal(ks, ks_ref) and torch.equal(sel, sel_ref) and torch.equal(ret, ret_ref)


def test_ems_noalloc_rejects_batches_beyond_its_scratch():
    lib = _lib()
    pc = enufft.EMSParams().c()
    dummy = torch.zeros(1, device="cuda")
    st = lib.enufft_ems_noalloc(64, 2049, _p(dummy), None, 0, ctypes.byref(pc), _p(dummy), _p(dummy), _p(dummy), None)
    assert st == 1
    assert "2048" in lib.enufft_last_error(None).decode()
