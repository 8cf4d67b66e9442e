"""BDDC-preconditioned CG on one GB300 (sm_103a): Python binding of libbddc.

Every step of the preconditioner and of PCG runs in the library's CUDA
kernels; this module only marshals arguments (PyTorch tensors for device
memory and the current CUDA stream, NumPy arrays for host inputs). Method:
Goebel, Cojean, Anzt, "BDDC preconditioning on GPUs for Cardiac
Simulations", arXiv 2410.14786, Sec. 2.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _lib
from ._lib import (CORNERS, EDGES, FACES, PREC_BF16, PREC_FP32, PREC_FP64, PREC_TF32,  # noqa: F401
                   BDDCError)

PRECISIONS = {"fp64": PREC_FP64, "fp32": PREC_FP32, "bf16": PREC_BF16, "tf32": PREC_TF32}
TENSOR_CORES = {"auto": _lib.TC_AUTO, True: _lib.TC_ON, False: _lib.TC_OFF}
COARSE = {"auto": _lib.COARSE_AUTO, "dense": _lib.COARSE_DENSE, "sparse": _lib.COARSE_SPARSE, "cg": _lib.COARSE_CG}
LOCAL = {"dense": _lib.LOCAL_DENSE, "sparse": _lib.LOCAL_SPARSE}


@dataclass
class SolveResult:
    iters: np.ndarray
    relres: np.ndarray
    status: int


def _stream_ptr(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dev_ptr(t, nrhs_expected=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError("expected a CUDA float64 tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous (node-major, right-hand side fastest)")
    return C.c_void_p(t.data_ptr())


class BDDC:
    """A BDDC preconditioner for one decomposed Q1 diffusion problem.

    Parameters mirror `bddc_problem_t` / `bddc_options_t`: dim, ne,
    elem_sigma [ne^dim] float64 > 0, elem_subdomain [ne^dim] int32,
    n_sub; precision in {"fp64", "fp32", "bf16"}; constraints bitmask of
    CORNERS | EDGES | FACES (0 = all); nrhs_max; host threads for setup;
    coarse in {"auto", "dense", "sparse"} (exact float64 coarse solve either way);
    graph=False launches each PCG iteration directly (for profilers);
    phi_fp64=True keeps the coarse basis Phi_i in float64 in the fp32, bf16
    and tf32 forms (by default it is float32 there, float64 in the fp64 form);
    tensor_cores in {"auto", True, False}: where the local operators of the
    bf16 / tf32 forms run (auto: tf32 always, bf16 from nrhs_max 8 on);
    autotune=True times the launch-parameter candidates on this handle's
    operators for nrhs_max columns and keeps the fastest (`autotune()`);
    tune_cache=path keeps those results in a JSON file keyed by the problem's
    shape, partition and form, so a later handle for the same problem reuses
    them without measuring again; coarse_blocks: blocks of the one-column
    sparse coarse solve (0 = one per SM); full_operators=True stores the
    symmetric local operators in full where they would otherwise be stored
    as lower triangles (fp32 / bf16 on the CUDA cores with nrhs_max = 1);
    history: PCG iterations whose scalars (||r_k||, alpha_k, beta_k) the
    handle keeps for `pcg_history()` (0 = none); coarse="cg" solves the
    coarse system inexactly by plain CG (the paper's choice) to
    coarse_cg_rtol (0: 1e-10) within coarse_cg_maxit iterations (0: 2000);
    local_solver="sparse" factorises every A_II (sparse Cholesky in nested-
    dissection order, float64) and runs the interior solves as its sweeps
    instead of forming A_II^-1 (subdomains of 10^4 dofs and more), with
    dense fronts of up to local_leaf dofs (0: 32).
    """

    def __init__(self, dim, ne, elem_sigma, elem_subdomain, n_sub, precision="fp64",
                 constraints=0, nrhs_max=1, n_threads=0, device=None, coarse="auto", graph=True,
                 phi_fp64=False, tensor_cores="auto", autotune=False, tune_cache=None, coarse_blocks=0,
                 full_operators=False, history=0, coarse_cg_rtol=0.0, coarse_cg_maxit=0,
                 local_solver="dense", local_leaf=0):
        import torch
        self._L = _lib.lib()
        self.handle = C.c_void_p()
        sig = np.ascontiguousarray(elem_sigma, dtype=np.float64)
        part = np.ascontiguousarray(elem_subdomain, dtype=np.int32)
        if device is None:
            device = torch.cuda.current_device() if torch.cuda.is_available() else 0
        prob = _lib.Problem(int(dim), int(ne), sig.ctypes.data_as(C.POINTER(C.c_double)),
                            part.ctypes.data_as(C.POINTER(C.c_int32)), int(n_sub))
        opts = _lib.Options(PRECISIONS[precision] if isinstance(precision, str) else int(precision),
                            int(constraints), int(nrhs_max), int(n_threads), int(device),
                            COARSE[coarse] if isinstance(coarse, str) else int(coarse), 0 if graph else 1,
                            1 if phi_fp64 else 0, TENSOR_CORES[tensor_cores], int(coarse_blocks),
                            1 if full_operators else 0, int(history), int(coarse_cg_maxit),
                            float(coarse_cg_rtol),
                            LOCAL[local_solver] if isinstance(local_solver, str) else int(local_solver),
                            int(local_leaf))
        _lib.check(self._L.bddc_setup(C.byref(prob), C.byref(opts), C.byref(self.handle)))
        self.dim, self.ne, self.nrhs_max = int(dim), int(ne), int(nrhs_max)
        self.n_nodes = (self.ne + 1) ** self.dim
        self.precision = precision
        self.history = int(history)
        self.tuned_from_cache = False
        if tune_cache is not None or autotune:
            self._tune(part, tune_cache, autotune)

    # -- launch-parameter tuning --------------------------------------------
    def get_tuning(self) -> dict:
        t = _lib.Tuning()
        _lib.check(self._L.bddc_get_tuning(self.handle, C.byref(t)))
        return {n: getattr(t, n) for n, _ in _lib.Tuning._fields_}

    def set_tuning(self, tuning: dict):
        t = _lib.Tuning(**{k: int(v) for k, v in tuning.items()})
        _lib.check(self._L.bddc_set_tuning(self.handle, C.byref(t)))

    def autotune(self, nrhs=None, stream=None) -> dict:
        """Measure the launch-parameter candidates for blocks of nrhs columns
        (default nrhs_max) on this handle and apply the fastest."""
        t = _lib.Tuning()
        _lib.check(self._L.bddc_autotune(self.handle, int(nrhs or self.nrhs_max), C.byref(t),
                                         _stream_ptr(stream)))
        return {n: getattr(t, n) for n, _ in _lib.Tuning._fields_}

    def _tune(self, part, cache, run):
        import hashlib
        import json
        import os
        key = "|".join([f"dim{self.dim}", f"ne{self.ne}", f"nrhs{self.nrhs_max}", f"prec{self.precision}",
                        f"tc{self.info()['tensor_cores']}", f"sym{self.info()['symmetric_operators']}",
                        f"local{self.info()['local_solver']}",
                        hashlib.sha1(np.ascontiguousarray(part, dtype=np.int32).tobytes()).hexdigest()[:16]])
        table = {}
        if cache is not None and os.path.exists(cache):
            with open(cache) as fh:
                table = json.load(fh)
        if key in table:
            self.set_tuning(table[key])
            self.tuned_from_cache = True
            return
        if not run and cache is None:
            return
        table[key] = self.autotune()
        if cache is not None:
            tmp = f"{cache}.{os.getpid()}.tmp"
            with open(tmp, "w") as fh:
                json.dump(table, fh, indent=1, sort_keys=True)
            os.replace(tmp, cache)

    @classmethod
    def from_problem(cls, p, **kw):
        return cls(p.dim, p.ne, p.elem_sigma, p.elem_subdomain, p.n_sub, **kw)

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            self._L.bddc_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        inf = _lib.Info()
        _lib.check(self._L.bddc_query(self.handle, C.byref(inf)))
        return {n: getattr(inf, n) for n, _ in _lib.Info._fields_}

    def _nrhs(self, t):
        return 1 if t.dim() == 1 else int(t.shape[1])

    def empty(self, nrhs=1):
        import torch
        shape = (self.n_nodes,) if nrhs == 1 else (self.n_nodes, nrhs)
        return torch.empty(shape, dtype=torch.float64, device="cuda")

    def apply(self, r, out=None, stream=None):
        """z = M^-1 r (device tensors [n_nodes] or [n_nodes, nrhs])."""
        z = out if out is not None else self.empty(self._nrhs(r))
        _lib.check(self._L.bddc_apply(self.handle, _dev_ptr(r), _dev_ptr(z), self._nrhs(r), _stream_ptr(stream)))
        return z

    def matvec(self, x, out=None, stream=None):
        y = out if out is not None else self.empty(self._nrhs(x))
        _lib.check(self._L.bddc_matvec(self.handle, _dev_ptr(x), _dev_ptr(y), self._nrhs(x), _stream_ptr(stream)))
        return y

    def rhs(self, f, out=None, stream=None):
        b = out if out is not None else self.empty(self._nrhs(f))
        _lib.check(self._L.bddc_rhs(self.handle, _dev_ptr(f), _dev_ptr(b), self._nrhs(f), _stream_ptr(stream)))
        return b

    def elem_grad(self, u, lam, out=None, stream=None):
        """g[e] = -sum_k lam_k,e^T K_ref u_k,e: the element term of an adjoint
        gradient dJ/dsigma (u, lam device tensors [n_nodes] or [n_nodes, nrhs])."""
        import torch
        n_el = self.ne ** self.dim
        g = out if out is not None else torch.empty(n_el, dtype=torch.float64, device=u.device)
        if u.shape != lam.shape:
            raise ValueError("u and lam must have the same shape")
        _lib.check(self._L.bddc_elem_grad(self.handle, _dev_ptr(u), _dev_ptr(lam), _dev_ptr(g), self._nrhs(u),
                                          _stream_ptr(stream)))
        return g

    def coarse_vectors(self, nrhs=1, stream=None):
        import torch
        n_c = self.info()["n_c"]
        rc = torch.zeros((n_c, nrhs), dtype=torch.float64, device="cuda")
        uc = torch.zeros_like(rc)
        _lib.check(self._L.bddc_coarse_vectors(self.handle, _dev_ptr(rc), _dev_ptr(uc), nrhs, _stream_ptr(stream)))
        return rc, uc

    def pcg_solve(self, b, x=None, rtol=1e-8, maxit=1000, stream=None, allow_breakdown=False) -> tuple:
        """Solve A x = b; returns (x, SolveResult). Device tensors. With
        allow_breakdown=True a PCG breakdown in some column (status
        ERR_BREAKDOWN) returns the per-column results instead of raising."""
        nrhs = self._nrhs(b)
        x = x if x is not None else self.empty(nrhs)
        iters = (C.c_int32 * nrhs)()
        rel = (C.c_double * nrhs)()
        st = self._L.bddc_pcg_solve(self.handle, _dev_ptr(b), _dev_ptr(x), nrhs, float(rtol), int(maxit),
                                    iters, rel, _stream_ptr(stream))
        _lib.check(st, allow=(_lib.OK, _lib.NOT_CONVERGED) + ((_lib.ERR_BREAKDOWN,) if allow_breakdown else ()))
        return x, SolveResult(np.array(iters[:]), np.array(rel[:]), st)

    def pcg_solve_host(self, b: np.ndarray, rtol=1e-8, maxit=1000, out: np.ndarray | None = None, stream=None):
        """Same with host (NumPy, ideally pinned) buffers; copies inside the call."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        nrhs = 1 if b.ndim == 1 else b.shape[1]
        x = out if out is not None else np.empty_like(b)
        iters = (C.c_int32 * nrhs)()
        rel = (C.c_double * nrhs)()
        st = self._L.bddc_pcg_solve_host(self.handle, C.c_void_p(b.ctypes.data), C.c_void_p(x.ctypes.data), nrhs,
                                         float(rtol), int(maxit), iters, rel, _stream_ptr(stream))
        _lib.check(st, allow=(_lib.OK, _lib.NOT_CONVERGED))
        return x, SolveResult(np.array(iters[:]), np.array(rel[:]), st)

    def pcg_history(self, nrhs=1, n_iter=None) -> dict:
        """Per-iteration scalars of the most recent PCG solve: arrays of shape
        (n_iter + 1, nrhs) named rnorm (||r_k||), alpha (alpha_k) and beta (the
        beta computed after iteration k + 1); NaN where not recorded."""
        n_iter = self.history if n_iter is None else int(n_iter)
        out = {k: np.empty((n_iter + 1) * nrhs) for k in ("rnorm", "alpha", "beta")}
        ptr = {k: v.ctypes.data_as(C.POINTER(C.c_double)) for k, v in out.items()}
        _lib.check(self._L.bddc_pcg_history(self.handle, int(nrhs), n_iter, ptr["rnorm"], ptr["alpha"],
                                            ptr["beta"]))
        return {k: v.reshape(n_iter + 1, nrhs) for k, v in out.items()}

    def test_coarse_stall(self, enable: bool, limit_cycles: int = 2_000_000):
        """Test hook: make every grid barrier of the sparse coarse solve wait
        for an arrival that never comes (bounded by limit_cycles), or restore it."""
        _lib.check(self._L.bddc_test_coarse_stall(self.handle, 1 if enable else 0, int(limit_cycles)))

    def clear_device_error(self):
        _lib.check(self._L.bddc_clear_device_error(self.handle))

    def profile_apply(self, r, reps=5, stream=None):
        z = self.empty(self._nrhs(r))
        out = (C.c_double * 9)()
        _lib.check(self._L.bddc_profile_apply(self.handle, _dev_ptr(r), _dev_ptr(z), self._nrhs(r), int(reps), out,
                                              _stream_ptr(stream)))
        names = ["restrict", "interior_op", "iface_rhs", "interface_op", "coarse_residual", "coarse_solve",
                 "prolong", "interior_rhs", "interior_op_final"]
        return dict(zip(names, out[:]))
