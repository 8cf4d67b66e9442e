"""The sparse local solver (BDDC_LOCAL_SPARSE; the paper's local solves by a
sparse direct factorisation, Sec. 3 implementation paragraph): every A_II
factorised by nested dissection of its elements, the interior solves of
Eqs. compzi and inner run as the forward and backward sweeps of all
subdomains' factors at once, and the interface Schur complement comes from
the same factorisation. GPU results against the oracle of Sec. 2 (which
solves with A_II by a dense Cholesky factorisation and takes K from the full
saddle-point system), element by element, on subdomains with large
interiors (2D squares of 32^2 and 48^2 elements, 3D cubes, uneven Voronoi
cells with one cell that has no interior), one and several right-hand sides,
every precision form, and PCG iterates."""
import numpy as np
import pytest

import synth
from oracle import CORNER, EDGE, FACE, Oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _voronoi_large():
    sub, n, cell = synth.voronoi_partition(24, 6, 96)
    sigma = synth.layer_sigma(24, cell)
    f = synth.uniform(97, 25 ** 3 * 2).reshape(-1, 2)
    return synth.Problem(3, 24, sigma, sub, n, f, "voronoi_24_6")


CASES = {
    # name: (problem, constraint mask, float64 bound)
    "2d_96_2x2": (lambda: synth.make_problem(2, 96, 2, "lognormal", k=71), CORNER | EDGE, 1e-11),
    "2d_96_3x3": (lambda: synth.make_problem(2, 96, 3, "lognormal", k=72), CORNER | EDGE, 1e-11),
    "3d_24_3cubed": (lambda: synth.make_problem(3, 24, 3, "lognormal", k=73), 0, 1e-11),
    # cond(A_c) 253 and up to 1357 interface rows: the bound of the large-cell
    # parity cases (n_G,max cond(A_c) eps = 7.6e-11)
    "3d_voronoi_large_cells": (_voronoi_large, 0, 1e-10),
}
_CACHE = {}


def _case(name):
    if name not in _CACHE:
        from paper_2410_14786_gb300 import build
        build.build()
        make, mask, tol = CASES[name]
        p = make()
        o = Oracle(p.dim, p.ne, p.elem_sigma, p.elem_subdomain, p.n_sub, constraints=mask or (CORNER | EDGE | FACE))
        _CACHE[name] = (p, mask, tol, o)
    return _CACHE[name]


def _bddc(p, mask, **kw):
    from paper_2410_14786_gb300 import BDDC
    kw.setdefault("local_solver", "sparse")
    return BDDC.from_problem(p, constraints=mask, **kw)


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _cols(A, k):
    return np.ascontiguousarray(A[:, 0] if k == 1 else A[:, :k])


def _rel(a, b):
    assert a.shape == b.shape, (a.shape, b.shape)
    return float(np.abs(a - b).max() / np.abs(b).max())


def _residuals(o, nrhs, seed):
    R = synth.uniform(seed, o.n_nodes * nrhs).reshape(-1, nrhs)
    R[o.dir] = 0
    return R


@pytest.mark.parametrize("nrhs", [1, 8])
@pytest.mark.parametrize("name", list(CASES))
def test_sparse_local_apply_fp64_matches_the_oracle(name, nrhs):
    p, mask, tol, o = _case(name)
    R = _residuals(o, nrhs, 81)
    Z = o.apply_nodes(R)
    g = _bddc(p, mask, precision="fp64", nrhs_max=nrhs)
    info = g.info()
    assert info["local_solver"] == 1 and info["interior_levels"] >= 2 and info["interior_factor_entries"] > 0
    z = g.apply(_cuda(_cols(R, nrhs))).cpu().numpy()
    assert _rel(z, _cols(Z, nrhs)) < tol
    g.close()


def test_sparse_local_one_column_on_a_multi_column_handle_and_64_columns():
    """nrhs_max = 64 builds the node matrices for several columns as well:
    a one-column call still takes the gather form, 64 columns the
    row-blocked sweeps; both match the oracle."""
    p, mask, tol, o = _case("2d_96_3x3")
    R = _residuals(o, 64, 82)
    Z = o.apply_nodes(R)
    g = _bddc(p, mask, precision="fp64", nrhs_max=64)
    assert _rel(g.apply(_cuda(R[:, 0])).cpu().numpy(), Z[:, 0]) < tol
    for k in (3, 64):
        assert _rel(g.apply(_cuda(R[:, :k])).cpu().numpy(), Z[:, :k]) < tol
    g.close()


@pytest.mark.parametrize("leaf", [1, 8, 512])
def test_leaf_sizes_give_the_same_preconditioner(leaf):
    """Leaf 1 (dissection down to single dofs), 8, and 512 (one dense front
    per 3D cube): the same M^-1 r to float64 rounding."""
    p, mask, tol, o = _case("3d_24_3cubed")
    R = _residuals(o, 1, 83)
    Z = o.apply_nodes(R)
    g = _bddc(p, mask, precision="fp64", local_leaf=leaf)
    assert _rel(g.apply(_cuda(R[:, 0])).cpu().numpy(), Z[:, 0]) < tol
    g.close()


@pytest.mark.parametrize("name", ["2d_96_2x2", "3d_voronoi_large_cells"])
def test_every_split_height_gives_the_same_preconditioner(name):
    """The one-column interior sweeps split at every height (gather form
    below, block form from it on: all gather, all block, and each mix) give
    M^-1 r to the float64 bound; the autotuner's choice is one of them."""
    p, mask, tol, o = _case(name)
    R = _residuals(o, 1, 86)
    Z = o.apply_nodes(R)[:, 0]
    g = _bddc(p, mask, precision="fp64")
    L = g.info()["interior_levels"]
    r = _cuda(R[:, 0])
    for k in range(L + 1):
        t = g.get_tuning()
        t["interior_block_height"] = k
        g.set_tuning(t)
        assert g.get_tuning()["interior_block_height"] == k
        assert _rel(g.apply(r).cpu().numpy(), Z) < tol, k
    t = g.autotune(1)
    assert 0 <= t["interior_block_height"] <= L
    assert _rel(g.apply(r).cpu().numpy(), Z) < tol
    g.close()


def test_sparse_and_dense_local_solvers_agree():
    p, mask, tol, o = _case("3d_voronoi_large_cells")
    R = _residuals(o, 8, 84)
    gs = _bddc(p, mask, precision="fp64", nrhs_max=8)
    gd = _bddc(p, mask, precision="fp64", nrhs_max=8, local_solver="dense")
    X = _cuda(R)
    assert _rel(gs.apply(X).cpu().numpy(), gd.apply(X).cpu().numpy()) < 1e-11
    ig, idn = gs.info(), gd.info()
    # the factor's sweeps read far fewer bytes than the dense inverses
    assert ig["interior_op_bytes"] < idn["interior_op_bytes"]
    gs.close()
    gd.close()


# Low-precision forms: K_GG in the form's precision, the interior sweeps in
# float64; bounds of the dense forms (operator rounding u: fp32 6.0e-8,
# bf16 3.9e-3, plus float32 accumulation).
@pytest.mark.parametrize("prec,nrhs,tc,bound", [("fp32", 1, "auto", 5e-6), ("bf16", 1, "auto", 1e-2),
                                                ("bf16", 8, True, 1e-2), ("tf32", 8, "auto", 2e-3)])
def test_sparse_local_low_precision_forms(prec, nrhs, tc, bound):
    p, mask, tol, o = _case("2d_96_3x3")
    R = _residuals(o, nrhs, 85)
    Z = o.apply_nodes(R)
    g = _bddc(p, mask, precision=prec, nrhs_max=nrhs, tensor_cores=tc)
    z = g.apply(_cuda(_cols(R, nrhs))).cpu().numpy()
    assert _rel(z, _cols(Z, nrhs)) < bound
    g.close()


@pytest.mark.parametrize("name", ["2d_96_2x2", "3d_voronoi_large_cells"])
def test_sparse_local_pcg_fp64_iterates(name):
    """The same iterations, solution, residual norms, alphas and betas as the
    oracle's PCG (to the bounds of the dense form's iterate tests)."""
    p, mask, tol, o = _case(name)
    b = o.rhs(p.f[:, 0])
    xo, h = o.pcg(b, 1e-8)
    g = _bddc(p, mask, precision="fp64", history=300)
    x, res = g.pcg_solve(_cuda(b), rtol=1e-8, maxit=300)
    it = h[0]["iters"]
    assert res.status == 0 and int(res.iters[0]) == it
    assert _rel(x.cpu().numpy(), xo) < 1e-10
    hg = g.pcg_history()
    rn = np.asarray(h[0]["rnorm"])
    assert np.all(np.abs(hg["rnorm"][:it + 1, 0] - rn) <= 1e-12 * rn[0])
    al = np.asarray(h[0]["alpha"])
    assert np.all(np.abs(hg["alpha"][:it, 0] - al) <= 1e-10 * np.abs(al))
    be = np.asarray(h[0]["beta"])
    assert np.all(np.abs(hg["beta"][:it - 1, 0] - be) <= 1e-10 * np.abs(be))
    g.close()


def test_sparse_local_mixed_pcg_and_graph_replay():
    """Flexible PCG with bf16 K_GG reaches a true residual below 1.5e-8 and
    the oracle's solution; graph replay and direct launches give bitwise the
    same solution."""
    p, mask, tol, o = _case("2d_96_3x3")
    b = o.rhs(p.f[:, 0])
    xo, _ = o.pcg(b, 1e-12)
    xs = []
    for graph in (True, False):
        g = _bddc(p, mask, precision="bf16", graph=graph)
        x, res = g.pcg_solve(_cuda(b), rtol=1e-8, maxit=300)
        assert res.status == 0
        x = x.cpu().numpy()
        tr = np.linalg.norm(o.to_free(b) - o.A @ o.to_free(x)) / np.linalg.norm(o.to_free(b))
        assert tr < 1.5e-8
        assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-6
        xs.append(x)
        g.close()
    assert np.array_equal(xs[0], xs[1])


def test_static_scratch_refuses_the_sparse_local_solver():
    import ctypes as C
    from paper_2410_14786_gb300 import _lib
    p, mask, tol, o = _case("2d_96_2x2")
    g = _bddc(p, mask)
    r = torch.zeros(o.n_nodes, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    st = int(torch.cuda.current_stream().cuda_stream)
    assert _lib.lib().bddc_apply_static_scratch(g.handle, C.c_void_p(r.data_ptr()), C.c_void_p(z.data_ptr()), 1,
                                                st) == _lib.ERR_INVALID_ARG
    g.close()
