"""Host-side checks of libbddc that need no GPU: exported symbols, argument
validation, and the float64 setup (globs, Phi_i, A_ci, A_c) against the
oracle's explicit saddle-point construction (Sec. 2, Eq. saddlepoint)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import synth
from oracle import CORNER, EDGE, FACE, Oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2410_14786_gb300 import _lib, build
    build.build()
    return _lib.lib()


def _declared_functions():
    txt = open(os.path.join(ROOT, "include", "bddc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bddc_[a-z_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(L):
    from paper_2410_14786_gb300 import _lib
    names = _declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n
    assert sorted(_lib.EXPORTED) == names


def test_no_unresolved_library_symbols(L):
    """Every function of the library's own namespace that one translation
    unit calls is defined in another (a shared library links with unresolved
    symbols and would fail only when loaded)."""
    import shutil
    import subprocess
    from paper_2410_14786_gb300 import _lib
    if not shutil.which("nm"):
        pytest.skip("nm not available")
    out = subprocess.run(["nm", "-D", "--undefined-only", _lib.LIB_PATH], capture_output=True,
                         text=True).stdout
    ours = [ln for ln in out.splitlines() if "_ZN4bddc" in ln or " bddc_" in ln]
    assert ours == [], ours


def _structs(p, precision=0, constraints=0, nrhs_max=1, local_solver=0, local_leaf=0):
    from paper_2410_14786_gb300 import _lib
    sig = np.ascontiguousarray(p.elem_sigma, dtype=np.float64)
    part = np.ascontiguousarray(p.elem_subdomain, dtype=np.int32)
    prob = _lib.Problem(p.dim, p.ne, sig.ctypes.data_as(C.POINTER(C.c_double)),
                        part.ctypes.data_as(C.POINTER(C.c_int32)), p.n_sub)
    opts = _lib.Options(precision, constraints, nrhs_max, 4, 0, 0, 0)
    opts.local_solver = local_solver
    opts.local_leaf = local_leaf
    return prob, opts, (sig, part)


def _inspect(L, p, constraints=0, local_solver=0, local_leaf=0):
    from paper_2410_14786_gb300 import _lib
    prob, opts, keep = _structs(p, constraints=constraints, local_solver=local_solver, local_leaf=local_leaf)
    info = _lib.Info()
    rc = L.bddc_setup_inspect(C.byref(prob), C.byref(opts), 1, C.byref(info), None, 0)
    assert rc == 0, L.bddc_last_error()
    n = info.n_c
    Ac = np.zeros(max(1, n * n))
    rc = L.bddc_setup_inspect(C.byref(prob), C.byref(opts), 1, C.byref(info),
                              Ac.ctypes.data_as(C.POINTER(C.c_double)), Ac.size)
    assert rc == 0, L.bddc_last_error()
    return info, Ac[:n * n].reshape(n, n)


CASES = [
    ("2d_cfg1", lambda: synth.config(1), CORNER | EDGE),
    ("2d_lognormal_3x3", lambda: synth.make_problem(2, 24, 3, "lognormal", k=11), 0),
    ("3d_lognormal_3cubed", lambda: synth.make_problem(3, 12, 3, "lognormal", k=12), 0),
    ("3d_corners_only", lambda: synth.make_problem(3, 8, 2, "lognormal", k=13), CORNER),
    ("3d_voronoi", lambda: _small_voronoi(), 0),
]


def _small_voronoi():
    sub, n, cell = synth.voronoi_partition(10, 6, 77)
    s = synth.layer_sigma(10, cell)
    f = synth.uniform(78, 11 ** 3).reshape(-1, 1)
    return synth.Problem(3, 10, s, sub, n, f, "voronoi_10_6")


@pytest.mark.parametrize("local", ["dense", "sparse", "sparse_leaf2"])
@pytest.mark.parametrize("name,make,mask", CASES, ids=[c[0] for c in CASES])
def test_coarse_matrix_matches_oracle(L, name, make, mask, local):
    """A_c = sum R_ci^T Phi_i^T A_i Phi_i R_ci (Sec. 2, Eq. coarsegrid) from
    the library's host setup against the oracle's, with the dense local
    solver and with the sparse one (Schur complement from the partial
    factorisation; leaf 2: deep dissection trees even on these small
    subdomains)."""
    p = make()
    info, Ac = _inspect(L, p, mask, local_solver=0 if local == "dense" else 1,
                        local_leaf=2 if local == "sparse_leaf2" else 0)
    o = Oracle(p.dim, p.ne, p.elem_sigma, p.elem_subdomain, p.n_sub,
               constraints=mask or (CORNER | EDGE | FACE))
    assert info.n_c == o.n_c
    kinds = [g.kind for g in o.globs]
    assert (info.n_corners, info.n_edges, info.n_faces) == (kinds.count(CORNER), kinds.count(EDGE),
                                                            kinds.count(FACE))
    assert info.n_free == o.n_free
    assert info.n_interior == int(np.sum(o.kappa == 1))
    Ao = o.Ac.toarray()
    assert np.abs(Ac - Ao).max() <= 1e-10 * np.abs(Ao).max()


def test_structured_sizes_config2_shape(L):
    # 96^3 grid with 12^3 subdomains: the glob counts of the size table
    p = synth.make_problem(3, 96, 12, "one")
    from paper_2410_14786_gb300 import _lib
    prob, opts, keep = _structs(p)
    info = _lib.Info()
    rc = L.bddc_setup_inspect(C.byref(prob), C.byref(opts), 0, C.byref(info), None, 0)
    assert rc == 0
    assert (info.n_corners, info.n_edges, info.n_faces, info.n_c) == (1331, 4356, 4752, 10439)
    assert info.n_free == 857375 and info.max_ni == 729
    assert info.sum_ni == 1191016 and info.sum_nI2 == 1728 * 343 ** 2


def _rc(L, p, **kw):
    prob, opts, keep = _structs(p, **kw)
    from paper_2410_14786_gb300 import _lib
    info = _lib.Info()
    return L.bddc_setup_inspect(C.byref(prob), C.byref(opts), 1, C.byref(info), None, 0), info


def test_invalid_arguments(L):
    base = synth.make_problem(2, 8, 2, "one")
    bad = synth.make_problem(2, 8, 2, "one")
    bad.elem_sigma = bad.elem_sigma.copy()
    bad.elem_sigma[3] = -1.0
    assert _rc(L, bad)[0] == -1
    bad.elem_sigma[3] = np.nan
    assert _rc(L, bad)[0] == -1
    bad = synth.make_problem(2, 8, 2, "one")
    bad.elem_subdomain = bad.elem_subdomain.copy()
    bad.elem_subdomain[0] = 99
    assert _rc(L, bad)[0] == -1
    assert b"out of range" in L.bddc_last_error()
    # an id range with an empty subdomain
    bad = synth.make_problem(2, 8, 2, "one")
    bad.n_sub = 5
    assert _rc(L, bad)[0] == -1
    assert _rc(L, base, precision=7)[0] == -1
    assert _rc(L, base, nrhs_max=65)[0] == -1
    assert _rc(L, base, constraints=8)[0] == -1
    assert b"constraint" in L.bddc_last_error()


def test_floating_subdomain_without_constraints_is_singular(L):
    # 2D, faces only: no constraints at all; the centre subdomain of 3x3 floats
    p = synth.make_problem(2, 12, 3, "one")
    rc, _ = _rc(L, p, constraints=FACE)
    assert rc == -4
    assert b"subdomain 4" in L.bddc_last_error()


def test_setup_without_device_fails_cleanly(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    from paper_2410_14786_gb300 import _lib
    p = synth.make_problem(2, 8, 2, "one")
    prob, opts, keep = _structs(p)
    h = C.c_void_p()
    rc = L.bddc_setup(C.byref(prob), C.byref(opts), C.byref(h))
    assert rc == -7 and not h.value


@pytest.mark.parametrize("precision,phi_fp64,expect", [(0, 0, 0), (1, 0, 1), (2, 0, 1), (2, 1, 0), (1, 1, 0)])
def test_phi_precision_follows_the_form(L, precision, phi_fp64, expect):
    """Phi_i is float64 in the FP64 form and float32 in the FP32 / BF16 forms
    unless phi_fp64 asks for float64 (the coarse solve is float64 in all)."""
    from paper_2410_14786_gb300 import _lib
    prob, opts, keep = _structs(synth.config(1), precision=precision)
    opts.phi_fp64 = phi_fp64
    info = _lib.Info()
    rc = L.bddc_setup_inspect(C.byref(prob), C.byref(opts), 0, C.byref(info), None, 0)
    assert rc == 0, L.bddc_last_error()
    assert info.precision == precision
    assert info.phi_precision == expect


@pytest.mark.parametrize("precision,tc,nrhs_max,expect,runs_as", [
    (2, 0, 1, 0, 2), (2, 0, 4, 0, 2), (2, 0, 8, 1, 2), (2, 1, 1, 1, 2), (2, 2, 64, 0, 2), (3, 0, 1, 0, 1),
    (3, 0, 7, 0, 1), (3, 0, 8, 1, 3), (3, 1, 1, 1, 3), (3, 1, 8, 1, 3), (1, 0, 64, 0, 1)])
def test_tensor_core_selection(L, precision, tc, nrhs_max, expect, runs_as):
    """BF16 and TF32 run on the tensor cores from 8 right-hand sides or when
    asked; below 8 a TF32 request under AUTO runs the FP32 form on the CUDA
    cores (the reported precision says so); FP32 / FP64 on CUDA cores."""
    from paper_2410_14786_gb300 import _lib
    prob, opts, keep = _structs(synth.config(1), precision=precision, nrhs_max=nrhs_max)
    opts.tensor_cores = tc
    info = _lib.Info()
    rc = L.bddc_setup_inspect(C.byref(prob), C.byref(opts), 0, C.byref(info), None, 0)
    assert rc == 0, L.bddc_last_error()
    assert info.tensor_cores == expect
    assert info.precision == runs_as


@pytest.mark.parametrize("precision,tc", [(3, 2), (0, 1), (1, 1), (2, 3), (4, 0)])
def test_tensor_core_option_rejects_invalid(L, precision, tc):
    from paper_2410_14786_gb300 import _lib
    prob, opts, keep = _structs(synth.config(1), precision=precision)
    opts.tensor_cores = tc
    info = _lib.Info()
    rc = L.bddc_setup_inspect(C.byref(prob), C.byref(opts), 0, C.byref(info), None, 0)
    assert rc == _lib.ERR_INVALID_ARG


def test_coarse_blocks_and_full_operators_options_validated(L):
    from paper_2410_14786_gb300 import _lib
    prob, opts, keep = _structs(synth.config(1))
    info = _lib.Info()
    opts.coarse_blocks = -1
    assert L.bddc_setup_inspect(C.byref(prob), C.byref(opts), 0, C.byref(info), None, 0) == _lib.ERR_INVALID_ARG
    opts.coarse_blocks = 4
    assert L.bddc_setup_inspect(C.byref(prob), C.byref(opts), 0, C.byref(info), None, 0) == 0
    opts.full_operators = 2
    assert L.bddc_setup_inspect(C.byref(prob), C.byref(opts), 0, C.byref(info), None, 0) == _lib.ERR_INVALID_ARG
    opts.full_operators = 1
    assert L.bddc_setup_inspect(C.byref(prob), C.byref(opts), 0, C.byref(info), None, 0) == 0


def test_local_solver_options_validated(L):
    from paper_2410_14786_gb300 import _lib
    prob, opts, keep = _structs(synth.config(1))
    info = _lib.Info()
    for ls, leaf, ok in ((2, 0, False), (-1, 0, False), (1, -1, False), (1, 4097, False), (1, 4096, True),
                         (1, 1, True), (0, 0, True)):
        opts.local_solver, opts.local_leaf = ls, leaf
        rc = L.bddc_setup_inspect(C.byref(prob), C.byref(opts), 1, C.byref(info), None, 0)
        assert rc == (0 if ok else _lib.ERR_INVALID_ARG), (ls, leaf, rc)


def test_struct_mirrors_match_the_header():
    """The ctypes mirrors of bddc_options_t, bddc_info_t and bddc_tuning_t
    list the header's fields in order."""
    import re
    from paper_2410_14786_gb300 import _lib
    hdr = open(os.path.join(ROOT, "include", "bddc.h")).read()
    for cname, pyname in (("bddc_options_t", "Options"), ("bddc_info_t", "Info"), ("bddc_tuning_t", "Tuning")):
        body = re.search(r"typedef struct \{((?:(?!typedef).)*?)\}\s*" + cname + ";", hdr, re.S).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        fields = [n.strip() for decl in re.findall(r"\b(?:int32_t|uint32_t|int64_t|double)\s+([\w\s,]+?);", body)
                  for n in decl.split(",")]
        assert fields == [n for n, _ in getattr(_lib, pyname)._fields_], cname
