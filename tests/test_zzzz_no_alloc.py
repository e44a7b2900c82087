"""prd_apply_sigma_noalloc: the Sigma apply for callers that cannot allocate
device memory at call time (another framework owns the allocator, or
allocation is forbidden after initialisation).  It keeps its intermediates in
the library's static device array instead of the context's workspace, so its
result must equal prd_apply_sigma's, call after call, and it must not call the
context's allocator nor change the device's free memory.

The file name sorts after every other test file, so pytest collects it last:
a failure here leaves every other test already run.  It passes alone in a
fresh process and after the other tests."""
import ctypes

import numpy as np
import pytest

from paper_2505_20968_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["fp64_twolevel", "fp32_hi"])
def test_noalloc_sigma_matches_sigma_on_two_calls(case):
    """Same result as prd_apply_sigma on two calls in a row, with no call of
    the context's allocator (a counting allocator routes every library
    allocation through PyTorch) and unchanged free device memory around the
    second call (the first may load the library's device code).  The bound
    is the FP64 / FP32 rounding of the emissivity, since the two paths add
    their contributions in a different order (the tensor-core epilogue
    accumulates with atomics): 1e-12 / 1e-6 of its maximum."""
    from paper_2505_20968_gb300.binding import PRD, lib
    if case == "fp64_twolevel":
        cfg, tol = inputs.twolevel_slab(n_z=8, n_x=11, n_mu_half=2, n_chi=4, eps=1e-2), 1e-12
    else:
        cfg, tol = inputs.hi_lya(n_z=10, n_core=13, n_wing=8, n_mu_half=2, n_chi=4, seed=31), 1e-6
    P = PRD(cfg, device=0, allocator="torch")
    assert P.alloc_stats["n_alloc"] > 0          # the workspace came through the counting allocator
    L = lib()
    for call, seed in enumerate((3, 4)):
        x = inputs.seeded_vector(P.shape, seed, 0.1, 1.0)
        x[..., 1:] *= 0.05
        xt = torch.from_numpy(x).to(device=P.device, dtype=P.dtype)
        ref = torch.empty_like(xt)
        out = torch.full_like(xt, float("nan"))
        P._stream()
        assert L.prd_apply_sigma(P.h, ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(ref.data_ptr())) == 0
        torch.cuda.synchronize()
        n_alloc, n_free = P.alloc_stats["n_alloc"], P.alloc_stats["n_free"]
        free0 = torch.cuda.mem_get_info(P.device)[0]
        rc = L.prd_apply_sigma_noalloc(P.h, ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(out.data_ptr()))
        assert rc == 0, L.prd_last_error(P.h)
        torch.cuda.synchronize()
        assert L.prd_device_status(P.h) == 0
        assert (P.alloc_stats["n_alloc"], P.alloc_stats["n_free"]) == (n_alloc, n_free)
        if call == 1:
            assert torch.cuda.mem_get_info(P.device)[0] == free0
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.max(np.abs(a - b)) <= tol * np.max(np.abs(b))
    P.close()
