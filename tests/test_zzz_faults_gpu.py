"""Fault paths of the C ABI on a set-up context (two-level slab, FP64), none
of which launches a kernel on invalid memory: arguments rejected on the host
(NULL, non-positive tolerance, zero iterations, calls before prd_setup), a
start vector holding NaN (the solve stops with PRD_E_NAN), and an iteration
cap below what the tolerance needs (PRD_E_NOCONV, with the iterate kept)."""
import ctypes

import numpy as np
import pytest

from paper_2505_20968_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E_ARG, E_STATE, E_NOCONV, E_NAN = -1, -2, -5, -7


def _case():
    return inputs.twolevel_slab(n_z=6, n_x=9, n_mu_half=1, n_chi=4, eps=1e-2)


def test_host_argument_and_state_checks():
    from paper_2505_20968_gb300.binding import PRD, lib
    L = lib()
    Q = PRD(_case(), precision="fp64", device=0, setup=False)
    x = torch.zeros(64, dtype=torch.float64, device="cuda")
    y = torch.zeros(64, dtype=torch.float64, device="cuda")
    px, py = ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr())
    assert L.prd_apply_operator(Q.h, px, py) == E_STATE          # before prd_setup
    Q.close()
    P = PRD(_case(), precision="fp64", device=0)
    a, b = P.empty(), P.empty()
    pa, pb = ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr())
    assert L.prd_apply_operator(P.h, None, pb) == E_ARG
    assert L.prd_apply_operator(P.h, pa, pa) == E_ARG              # aliased
    it, res = ctypes.c_int(), ctypes.c_double()
    assert L.prd_solve(P.h, 0.0, 10, 10, None, pb, ctypes.byref(it), ctypes.byref(res), None) == E_ARG
    assert L.prd_solve(P.h, 1e-8, 0, 10, None, pb, ctypes.byref(it), ctypes.byref(res), None) == E_ARG
    assert L.prd_last_error(P.h)                                   # a reason is given
    P.close()


def test_nan_start_vector_stops_the_solve():
    from paper_2505_20968_gb300.binding import PRD
    P = PRD(_case(), precision="fp64", device=0)
    x0 = torch.full(P.shape, float("nan"), dtype=P.dtype, device=P.device)
    _, info = P.solve(tol=1e-10, max_iter=50, restart=20, x0=x0, check=False)
    assert info["rc"] == E_NAN, info
    x, info = P.solve(tol=1e-10, max_iter=200, restart=40)       # the context is still usable
    assert info["rc"] == 0 and bool(torch.isfinite(x).all())
    P.close()


def test_iteration_cap_reports_no_convergence():
    from paper_2505_20968_gb300.binding import PRD
    P = PRD(_case(), precision="fp64", device=0)
    x, info = P.solve(tol=1e-14, max_iter=1, restart=10, check=False)
    assert info["rc"] == E_NOCONV and info["iters"] == 1, info
    assert bool(torch.isfinite(x).all()) and float(x.abs().max()) > 0   # the iterate is kept
    assert info["true_rel_res"] > 1e-14
    P.close()
