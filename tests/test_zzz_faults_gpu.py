"""Fault paths of the C ABI on a set-up context (two-level slab, FP64, and a
reduced H I case in FP32), none of which launches a kernel on invalid memory:
arguments rejected on the host (NULL, non-positive tolerance, zero
iterations, calls before prd_setup), a start vector holding NaN (the solve
stops with PRD_E_NAN), an iteration cap below what the tolerance needs
(PRD_E_NOCONV, with the iterate kept), an Arnoldi breakdown on an injected
zero operator (PRD_E_BREAKDOWN), and the bounded waits of the tensor-core
contraction running out (PRD_E_TIMEOUT from prd_device_status; the waits are
given a few polls, every thread block drains what it issued, and the context
applies correctly afterwards)."""
import ctypes

import numpy as np
import pytest

from paper_2505_20968_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E_ARG, E_STATE, E_NOCONV, E_BREAKDOWN, E_NAN, E_TIMEOUT = -1, -2, -5, -6, -7, -8
OPT_WAIT_POLLS, OPT_TEST_ZERO_OPERATOR = 3, 4


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


def test_breakdown_on_injected_zero_operator():
    """With the operator replaced by the zero map, the first Arnoldi vector
    is annihilated (h_10 = 0): GMRES stops at the breakdown with the residual
    still ||b||, returns PRD_E_BREAKDOWN and keeps a finite iterate; with the
    operator restored the same context solves."""
    from paper_2505_20968_gb300.binding import PRD, lib
    P = PRD(_case(), precision="fp64", device=0)
    assert lib().prd_set_option(P.h, OPT_TEST_ZERO_OPERATOR, 1) == 0
    x, info = P.solve(tol=1e-10, max_iter=50, restart=20, check=False)
    assert info["rc"] == E_BREAKDOWN, info
    assert info["true_rel_res"] > 0.5 and bool(torch.isfinite(x).all())
    assert lib().prd_set_option(P.h, OPT_TEST_ZERO_OPERATOR, 0) == 0
    x, info = P.solve(tol=1e-10, max_iter=200, restart=40)
    assert info["rc"] == 0 and info["true_rel_res"] < 1e-10
    P.close()


def test_contraction_wait_expiry_reports_timeout():
    """The tensor-core contraction with its pipeline waits limited to 4 polls:
    the first waits run out before the first bulk copies land, so thread
    blocks stop, drain the copies and products they issued (those waits keep
    the default limit) and record the failure: prd_device_status returns
    PRD_E_TIMEOUT.  With the default limit restored the same context gives
    the emissivity of a fresh apply again (to FP32 summation order)."""
    from paper_2505_20968_gb300.binding import PRD, lib
    cfg = inputs.hi_lya(n_z=4, n_core=13, n_wing=8, n_mu_half=2, n_chi=4, seed=31)
    P = PRD(cfg, device=0)
    x = torch.from_numpy(inputs.seeded_vector(P.shape, 3, 0.1, 1.0)).to(P.device, P.dtype)
    ref = P.apply_sigma(x).clone()
    P.device_status()
    assert lib().prd_set_option(P.h, OPT_WAIT_POLLS, 4) == 0
    P.apply_sigma(x)
    assert lib().prd_device_status(P.h) == E_TIMEOUT
    assert lib().prd_device_status(P.h) == 0                      # reported once
    assert lib().prd_set_option(P.h, OPT_WAIT_POLLS, 0) == 0
    out = P.apply_sigma(x)
    P.device_status()
    assert torch.max(torch.abs(out - ref)).item() <= 1e-6 * torch.max(torch.abs(ref)).item()
    P.close()
