"""prd_apply_sigma_noalloc: the Sigma apply for callers that cannot allocate
device memory at call time (another framework owns the allocator, or
allocation is forbidden after initialisation).  It keeps its intermediates in
the library's static device array instead of the context's workspace, so its
result must equal prd_apply_sigma's, call after call.

This file is collected last on purpose: a failure here leaves every other test
already run.  It passes alone in a fresh process and after the other tests."""
import ctypes

import numpy as np
import pytest

from paper_2505_20968_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["fp64_twolevel", "fp32_hi"])
def test_noalloc_sigma_matches_sigma_on_two_calls(case):
    from paper_2505_20968_gb300.binding import PRD, lib
    if case == "fp64_twolevel":
        cfg, tol = inputs.twolevel_slab(n_z=8, n_x=11, n_mu_half=2, n_chi=4, eps=1e-2), 1e-12
    else:
        cfg, tol = inputs.hi_lya(n_z=10, n_core=13, n_wing=8, n_mu_half=2, n_chi=4, seed=31), 1e-6
    P = PRD(cfg, device=0)
    L = lib()
    for seed in (3, 4):
        x = inputs.seeded_vector(P.shape, seed, 0.1, 1.0)
        x[..., 1:] *= 0.05
        xt = torch.from_numpy(x).to(device=P.device, dtype=P.dtype)
        ref = torch.empty_like(xt)
        out = torch.full_like(xt, float("nan"))
        P._stream()
        assert L.prd_apply_sigma(P.h, ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(ref.data_ptr())) == 0
        rc = L.prd_apply_sigma_noalloc(P.h, ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(out.data_ptr()))
        assert rc == 0, L.prd_last_error(P.h)
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.max(np.abs(a - b)) <= tol * np.max(np.abs(b))
    P.close()
