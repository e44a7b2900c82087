"""Thin Python binding of libprd.so (include/prd.h): argument marshalling only,
plus a torch.autograd.Function that routes gradients with respect to the
magnetic field through prd_grad_B (solve_with_field).

PyTorch provides device memory and the current CUDA stream; every step of the
operator runs in the library's CUDA kernels.  There is no CPU fallback: if the
shared library is missing or cannot be loaded this module raises.
"""
import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libprd.so")

PRD_OK = 0
ERRORS = {-1: "PRD_E_ARG", -2: "PRD_E_STATE", -3: "PRD_E_CUDA", -4: "PRD_E_NOMEM", -5: "PRD_E_NOCONV",
          -6: "PRD_E_BREAKDOWN", -7: "PRD_E_NAN", -8: "PRD_E_TIMEOUT"}
PRD_FP64, PRD_FP32, PRD_FP32_BF16X3, PRD_FP32_BF16X2 = 0, 1, 2, 3
# prd_set_option ids and values (include/prd.h)
PRD_OPT_TENSOR_CORES, PRD_OPT_PRECOND_SWEEPS, PRD_OPT_WAIT_POLLS, PRD_OPT_TEST_ZERO_OPERATOR = 1, 2, 3, 4
PRD_OPT_REFINE_FLOOR, PRD_OPT_FORMAL_SOLVER, PRD_OPT_CONTRACTION, PRD_OPT_TILE_STAGES = 5, 6, 7, 8
PRD_OPT_GRAPH, PRD_OPT_STAGED_SWEEP, PRD_OPT_GRAD_FULL_SETUP = 9, 10, 11
PRD_CONTRACTION_TF32X3, PRD_CONTRACTION_BF16X3 = 0, 1
PRD_DELO_LINEAR, PRD_DELOPAR = 0, 1


class PrdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class _Atom(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("twoS", ctypes.c_int), ("E_u_cm", ctypes.c_double * 2),
                ("mass_amu", ctypes.c_double), ("g_s", ctypes.c_double), ("nu0_hz", ctypes.c_double)]


_lib = None
EXPORTS = ["prd_create", "prd_destroy", "prd_last_error", "prd_set_stream", "prd_set_atom",
           "prd_set_atmosphere", "prd_set_quadrature", "prd_setup", "prd_sizes", "prd_directions",
           "prd_workspace_bytes", "prd_rhs", "prd_apply_sigma", "prd_apply_lambda", "prd_apply_operator",
           "prd_apply_preconditioner", "prd_set_precond_sweeps", "prd_solve", "prd_emergent_stokes",
           "prd_set_profiling", "prd_stage_times", "prd_apply_sigma_noalloc", "prd_set_option",
           "prd_device_status", "prd_contraction_work",
           "prd_apply_operator_T", "prd_solve_adjoint", "prd_solve_batch",
           "prd_grad_B", "prd_set_allocator", "prd_narrowband", "prd_set_continuum", "prd_graph_launches"]


def lib():
    """Load libprd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} not found: run __graft_entry__.build() first")
        L = ctypes.CDLL(LIB_PATH)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        DP = ctypes.POINTER(ctypes.c_double)
        L.prd_create.argtypes = [ctypes.POINTER(P), I, I]
        L.prd_destroy.argtypes = [P]
        L.prd_last_error.argtypes = [P]
        L.prd_last_error.restype = ctypes.c_char_p
        L.prd_set_stream.argtypes = [P, P]
        L.prd_set_allocator.argtypes = [P, _ALLOC_FN, _FREE_FN, P]
        L.prd_set_atom.argtypes = [P, ctypes.POINTER(_Atom)]
        L.prd_set_atmosphere.argtypes = [P, I] + [DP] * 12
        L.prd_set_quadrature.argtypes = [P, I, DP, I, I, I, I, I]
        L.prd_set_continuum.argtypes = [P, DP, DP, DP]
        L.prd_setup.argtypes = [P]
        L.prd_sizes.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I),
                                ctypes.POINTER(I), ctypes.POINTER(ctypes.c_int64)]
        L.prd_directions.argtypes = [P, DP, DP, DP]
        L.prd_workspace_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
        L.prd_contraction_work.argtypes = [P, DP, DP]
        L.prd_apply_operator_T.argtypes = [P, P, P]
        L.prd_grad_B.argtypes = [P, P, P, DP]
        L.prd_solve_batch.argtypes = [ctypes.POINTER(P), I, D, I, I, ctypes.POINTER(P), ctypes.POINTER(I), DP,
                                      ctypes.POINTER(I)]
        L.prd_solve_adjoint.argtypes = [P, P, D, I, I, P, ctypes.POINTER(I), DP, DP]
        for f in ("prd_rhs",):
            getattr(L, f).argtypes = [P, P]
        for f in ("prd_apply_sigma", "prd_apply_lambda", "prd_apply_operator", "prd_apply_preconditioner",
                  "prd_apply_sigma_noalloc"):
            getattr(L, f).argtypes = [P, P, P]
        L.prd_set_precond_sweeps.argtypes = [P, I]
        L.prd_solve.argtypes = [P, D, I, I, P, P, ctypes.POINTER(I), DP, DP]
        L.prd_emergent_stokes.argtypes = [P, P, I, DP, DP, P]
        L.prd_narrowband.argtypes = [P, P, I, DP, DP, D, D, D, DP]
        L.prd_set_profiling.argtypes = [P, I]
        L.prd_set_option.argtypes = [P, I, I]
        L.prd_device_status.argtypes = [P]
        L.prd_graph_launches.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
        L.prd_stage_times.argtypes = [P, DP, ctypes.POINTER(ctypes.c_int64), I]
        _lib = L
    return _lib


def _dp(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


def _torch_allocator(device, stats):
    """prd_set_allocator callbacks backed by PyTorch's caching allocator;
    stats counts the calls, the bytes handed out and the pointers still live."""
    def alloc(nbytes, user, stream):
        stats["n_alloc"] += 1
        try:
            p = torch.cuda.caching_allocator_alloc(int(nbytes), device=device, stream=int(stream or 0))
        except Exception:   # out of memory: the library reports PRD_E_NOMEM
            return None
        stats["bytes"] += int(nbytes)
        stats["live"][p] = int(nbytes)
        return p

    def free(ptr, user):
        stats["n_free"] += 1
        stats["live"].pop(int(ptr), None)
        torch.cuda.caching_allocator_delete(int(ptr))
    return _ALLOC_FN(alloc), _FREE_FN(free)


class PRD:
    """One library context: a configured problem resident on one GPU.

    allocator="torch" routes the library's device memory through PyTorch's
    caching allocator (prd_set_allocator) instead of cudaMalloc."""

    def __init__(self, cfg, precision=None, device=0, mode=None, setup=True, allocator=None):
        L = lib()
        prec = cfg.get("precision", "fp32") if precision is None else precision
        self.prec = PRD_FP64 if prec in ("fp64", PRD_FP64) else PRD_FP32
        create = {"fp32_bf16x3": PRD_FP32_BF16X3, "fp32_bf16x2": PRD_FP32_BF16X2}.get(prec, self.prec)
        self.dtype = torch.float64 if self.prec == PRD_FP64 else torch.float32
        self.device = torch.device("cuda", device)
        h = ctypes.c_void_p()
        self._check(L.prd_create(ctypes.byref(h), device, create), None)
        self.h = h
        atom = cfg["atom"]
        A = _Atom(atom["kind"], atom["twoS"], (ctypes.c_double * 2)(*atom["E_u_cm"]), atom["mass_amu"],
                  atom.get("g_s", 2.0), atom.get("nu0_hz", 0.0))
        self._check(L.prd_set_atom(self.h, ctypes.byref(A)))
        atm = cfg["atm"]
        keep = [_dp(atm[k]) for k in ("z_km", "T_K", "xi_kms", "a", "eps", "r_el", "k_line", "W_T", "B_G",
                                      "thetaB", "chiB", "v_kms")]
        self._check(L.prd_set_atmosphere(self.h, len(atm["z_km"]), *[p for _, p in keep]))
        q = cfg["quad"]
        g, gp = _dp(q["grid"])
        self._check(L.prd_set_quadrature(self.h, len(g), gp, q["grid_kind"], q["n_mu_half"], q["n_chi"],
                                         q.get("mu_rule", 0), q.get("mode", 0) if mode is None else mode))
        if "sigma_c" in atm:
            cont = [_dp(atm[k]) for k in ("kappa_c", "sigma_c", "eps_c_th")]
            self._check(L.prd_set_continuum(self.h, *[p for _, p in cont]))
        self._alloc = None
        self.alloc_stats = {"bytes": 0, "live": {}, "n_alloc": 0, "n_free": 0}
        if allocator == "torch":
            self._alloc = _torch_allocator(device, self.alloc_stats)   # kept alive as long as the ctx
            self._stream()
            self._check(L.prd_set_allocator(self.h, self._alloc[0], self._alloc[1], None))
        elif allocator is not None:
            raise ValueError("allocator must be None or 'torch'")
        if setup:
            self.setup()

    def _check(self, rc, h=0):
        if rc != PRD_OK:
            msg = lib().prd_last_error(self.h if h == 0 else h)
            raise PrdError(rc, msg.decode() if msg else "")

    def setup(self):
        self._check(lib().prd_setup(self.h))
        nz, nO, nN, nT = (ctypes.c_int() for _ in range(4))
        n = ctypes.c_int64()
        self._check(lib().prd_sizes(self.h, ctypes.byref(nz), ctypes.byref(nO), ctypes.byref(nN),
                                    ctypes.byref(nT), ctypes.byref(n)))
        self.nz, self.nO, self.nN, self.n_theta, self.n = nz.value, nO.value, nN.value, nT.value, n.value
        self.shape = (self.nz, self.nO, self.nN, 4)
        mu, chi, w = (np.zeros(self.nO) for _ in range(3))
        self._check(lib().prd_directions(self.h, mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         chi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        self.mu, self.chi, self.w = mu, chi, w

    def apply_operator_T(self, x, out=None):
        """y = (Id - Lambda Sigma)^T x (FP64 arithmetic)."""
        self._stream()
        out = self.empty() if out is None else out
        self._check(lib().prd_apply_operator_T(self.h, self._vec(x), self._vec(out)))
        return out

    def solve_adjoint(self, g, tol=1e-8, max_iter=400, restart=60, out=None, check=True):
        """lam with (Id - Lambda Sigma)^T lam = g."""
        self._stream()
        out = self.empty() if out is None else out
        it = ctypes.c_int()
        res = ctypes.c_double()
        hist = np.zeros(max_iter + 2)
        rc = lib().prd_solve_adjoint(self.h, self._vec(g), tol, max_iter, restart, self._vec(out), ctypes.byref(it),
                                     ctypes.byref(res), hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        if check:
            self._check(rc)
        return out, dict(iters=it.value, true_rel_res=res.value, rc=rc)

    def grad_B(self, x, dJdI):
        """dJ/d(B, theta_B, chi_B) per height, shape (nz, 3), by the adjoint method."""
        self._stream()
        g = np.zeros((self.nz, 3))
        self._check(lib().prd_grad_B(self.h, self._vec(x), self._vec(dJdI),
                                     g.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return g

    def contraction_work(self):
        """(flops, bytes) of one R_II contraction (roofline accounting)."""
        f, b = ctypes.c_double(), ctypes.c_double()
        self._check(lib().prd_contraction_work(self.h, ctypes.byref(f), ctypes.byref(b)))
        return f.value, b.value

    def workspace_bytes(self):
        b = ctypes.c_int64()
        self._check(lib().prd_workspace_bytes(self.h, ctypes.byref(b)))
        return b.value

    def _stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        self._check(lib().prd_set_stream(self.h, ctypes.c_void_p(s)))

    def empty(self):
        return torch.empty(self.shape, dtype=self.dtype, device=self.device)

    def _vec(self, x):
        assert x.is_cuda and x.dtype == self.dtype and x.is_contiguous() and tuple(x.shape) == self.shape
        return ctypes.c_void_p(x.data_ptr())

    def rhs(self, out=None):
        self._stream()
        out = self.empty() if out is None else out
        self._check(lib().prd_rhs(self.h, self._vec(out)))
        return out

    def apply_sigma(self, x, out=None):
        self._stream()
        out = self.empty() if out is None else out
        self._check(lib().prd_apply_sigma(self.h, self._vec(x), self._vec(out)))
        return out

    def apply_sigma_noalloc(self, x, out):
        """Sigma x with the library's static scratch (allocates nothing; out must be given)."""
        self._stream()
        self._check(lib().prd_apply_sigma_noalloc(self.h, self._vec(x), self._vec(out)))
        return out

    def apply_lambda(self, eps, out=None):
        self._stream()
        out = self.empty() if out is None else out
        self._check(lib().prd_apply_lambda(self.h, self._vec(eps), self._vec(out)))
        return out

    def apply_operator(self, x, out=None):
        self._stream()
        out = self.empty() if out is None else out
        self._check(lib().prd_apply_operator(self.h, self._vec(x), self._vec(out)))
        return out

    def apply_preconditioner(self, y, out=None):
        self._stream()
        out = self.empty() if out is None else out
        self._check(lib().prd_apply_preconditioner(self.h, self._vec(y), self._vec(out)))
        return out

    def set_tensor_cores(self, on=True):
        self._check(lib().prd_set_option(self.h, PRD_OPT_TENSOR_CORES, 1 if on else 0))

    def set_tile_stages(self, n):
        """Depth of the contraction's tile ring (0: the deepest that fits)."""
        self._check(lib().prd_set_option(self.h, PRD_OPT_TILE_STAGES, int(n)))

    def set_contraction(self, kind):
        """Split products of the tensor-core contraction: "tf32x3" or "bf16x3"."""
        self._check(lib().prd_set_option(self.h, PRD_OPT_CONTRACTION,
                                         {"tf32x3": PRD_CONTRACTION_TF32X3, "bf16x3": PRD_CONTRACTION_BF16X3}[kind]))

    def device_status(self):
        self._check(lib().prd_device_status(self.h))

    def set_graph(self, on):
        """Run each GMRES iteration as one CUDA-graph launch (default) or not."""
        self._check(lib().prd_set_option(self.h, PRD_OPT_GRAPH, 1 if on else 0))

    def graph_launches(self):
        """CUDA-graph launches of the GMRES step made by this context so far."""
        n = ctypes.c_int64()
        self._check(lib().prd_graph_launches(self.h, ctypes.byref(n)))
        return n.value

    def set_precond_sweeps(self, m):
        self._check(lib().prd_set_precond_sweeps(self.h, m))

    def solve(self, tol=1e-6, max_iter=200, restart=30, x0=None, out=None, history=False, check=True):
        self._stream()
        out = self.empty() if out is None else out
        it = ctypes.c_int()
        res = ctypes.c_double()
        hist = np.zeros(max_iter + 2)
        rc = lib().prd_solve(self.h, tol, max_iter, restart, None if x0 is None else self._vec(x0),
                             self._vec(out), ctypes.byref(it), ctypes.byref(res),
                             hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        if check:
            self._check(rc)
        info = dict(iters=it.value, true_rel_res=res.value, rc=rc, history=hist[:max(it.value, 1)])
        return out, info

    def emergent_stokes(self, x, mu, chi, out=None):
        self._stream()
        mu, mup = _dp(mu)
        chi, chip = _dp(chi)
        out = torch.empty((len(mu), self.nN, 4), dtype=self.dtype, device=self.device) if out is None else out
        self._check(lib().prd_emergent_stokes(self.h, self._vec(x), len(mu), mup, chip, ctypes.c_void_p(out.data_ptr())))
        return out

    def narrowband(self, x, mu, chi, lambda0, fwhm, half_width):
        """Gaussian-weighted wavelength integrals of the emergent Stokes
        vectors along lines of sight (mu, chi): array [nlos][4] (Sect. 6.5)."""
        self._stream()
        mu, mup = _dp(mu)
        chi, chip = _dp(chi)
        out = np.zeros((len(mu), 4))
        self._check(lib().prd_narrowband(self.h, self._vec(x), len(mu), mup, chip, lambda0, fwhm, half_width,
                                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    STAGES = ("S1_interp_in", "S5_R3", "S3_R2_contraction", "S6_interp_back", "S7_delo")

    def set_profiling(self, on=True):
        self._check(lib().prd_set_profiling(self.h, 1 if on else 0))

    def stage_times(self):
        ms = np.zeros(8)
        cnt = np.zeros(8, dtype=np.int64)
        self._check(lib().prd_stage_times(self.h, ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), 8))
        return {k: (ms[i], int(cnt[i])) for i, k in enumerate(self.STAGES)}

    def close(self):
        if getattr(self, "h", None):
            lib().prd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batch(problems, tol=1e-6, max_iter=200, restart=30, check=True):
    """Solve independent problems (PRD instances, ragged sizes allowed) with one
    prd_solve_batch call: each instance on its own CUDA stream and host thread.
    Returns the solutions and a list of per-instance info dicts."""
    n = len(problems)
    streams = [torch.cuda.Stream(device=P.device) for P in problems]
    outs = []
    for P, s in zip(problems, streams):
        lib().prd_set_stream(P.h, ctypes.c_void_p(s.cuda_stream))
        with torch.cuda.stream(s):
            outs.append(P.empty())
    for s in streams:
        s.synchronize()
    hs = (ctypes.c_void_p * n)(*[P.h for P in problems])
    xs = (ctypes.c_void_p * n)(*[ctypes.c_void_p(o.data_ptr()) for o in outs])
    it = (ctypes.c_int * n)()
    res = (ctypes.c_double * n)()
    rcs = (ctypes.c_int * n)()
    rc = lib().prd_solve_batch(hs, n, tol, max_iter, restart, xs, it, res, rcs)
    infos = [dict(iters=it[i], true_rel_res=res[i], rc=rcs[i]) for i in range(n)]
    if check and rc != 0:
        bad = [i for i in range(n) if rcs[i] != 0]
        problems[bad[0]]._check(rcs[bad[0]])
    return outs, infos



class _FieldSolve(torch.autograd.Function):
    """The solution I(p) of A(p) I = b(p) as a function of the magnetic field
    p = (B [G], theta_B, chi_B [rad]) of every height, shape (nz, 3).  Forward
    sets the problem up with that field and solves it (prd_solve); backward is
    the adjoint method of prd_grad_B: one solve A^T lam = dJ/dI, then
    dJ/dp = lam^T (db/dp - (dA/dp) I)."""

    @staticmethod
    def forward(ctx, field, cfg, make, solve_kw):
        f = field.detach().to("cpu", torch.float64).numpy()
        atm = dict(cfg["atm"], B_G=f[:, 0].copy(), thetaB=f[:, 1].copy(), chiB=f[:, 2].copy())
        P = make(dict(cfg, atm=atm))
        x, _ = P.solve(**solve_kw)
        ctx.P = P
        ctx.field_like = (field.dtype, field.device)
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        g = ctx.P.grad_B(x, gx.to(x.dtype).contiguous())
        ctx.P.close()
        dtype, device = ctx.field_like
        return torch.as_tensor(g, dtype=dtype, device=device), None, None, None


def solve_with_field(cfg, field, precision="fp64", device=0, tol=1e-12, max_iter=600, restart=80, make=None):
    """Solve the problem `cfg` with its magnetic field replaced by `field`
    ((nz, 3): B, theta_B, chi_B per height) and return the Stokes field
    I[z][Omega][nu][4] as a differentiable function of `field`: the gradient of
    any scalar built from I reaches `field` through one adjoint solve.  `make`
    builds the solver object from a problem dict (default: PRD)."""
    if make is None:
        def make(c):
            return PRD(c, precision=precision, device=device)
    return _FieldSolve.apply(field, cfg, make, dict(tol=tol, max_iter=max_iter, restart=restart))
