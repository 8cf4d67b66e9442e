"""The inexact coarse solve by plain CG (BDDC_COARSE_CG; the paper's choice,
Sec. 3: the coarse system of Eq. coarsegrid solved with plain CG) against
the oracle's CG on the same coarse residual, and BDDC-PCG with it against
the oracle's solution."""
import numpy as np
import pytest

import synth
from oracle import CORNER, EDGE, FACE, Oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _small_voronoi():
    sub, n, cell = synth.voronoi_partition(12, 8, 91)
    s = synth.layer_sigma(12, cell)
    f = synth.uniform(92, 13 ** 3 * 2).reshape(-1, 2)
    return synth.Problem(3, 12, s, sub, n, f, "voronoi_12_8")


CASES = {
    "cfg1_2d": (lambda: synth.config(1), CORNER | EDGE),
    "3d_24_3cubed": (lambda: synth.make_problem(3, 24, 3, "lognormal", k=21), 0),
    "3d_voronoi": (_small_voronoi, 0),
}
_CACHE = {}


def _case(name):
    if name not in _CACHE:
        from paper_2410_14786_gb300 import build
        build.build()
        make, mask = CASES[name]
        p = make()
        _CACHE[name] = (p, mask, Oracle(p.dim, p.ne, p.elem_sigma, p.elem_subdomain, p.n_sub,
                                        constraints=mask or (CORNER | EDGE | FACE)))
    return _CACHE[name]


def _bddc(p, mask, **kw):
    from paper_2410_14786_gb300 import BDDC
    return BDDC.from_problem(p, constraints=mask, coarse="cg", **kw)


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("name", list(CASES))
def test_coarse_cg_matches_the_oracle_cg(name):
    """Same coarse residual, same CG from 0, same stop test: the iteration
    counts agree (to one, the stop test sees float64 sums in another order),
    the result satisfies the stop test with the oracle's A_c, and it matches
    the oracle's CG iterate to 1e-8 (cond(A_c) <= 253 times the rounding of
    up to a few hundred float64 steps)."""
    p, mask, o = _case(name)
    rtol = 1e-10
    g = _bddc(p, mask, coarse_cg_rtol=rtol)
    assert g.info()["coarse_levels"] == 0
    r = synth.uniform(45, o.n_nodes)
    r[o.dir] = 0
    g.apply(_cuda(r))
    rc, uc = g.coarse_vectors()
    rc, uc = rc.cpu().numpy()[:, 0], uc.cpu().numpy()[:, 0]
    parts = o.apply_parts(o.to_free(r))
    assert _rel(rc, parts["rc"]) < 1e-12
    u_o, it_o, _ = o.coarse_solve_cg(rc, rtol)
    it_g = g.info()["coarse_cg_iters"]
    assert abs(it_g - it_o) <= 1, (it_g, it_o)
    assert np.linalg.norm(rc - o.Ac @ uc) <= 2 * rtol * np.linalg.norm(rc)
    assert _rel(uc, u_o) < 1e-8
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
@pytest.mark.parametrize("name", list(CASES))
def test_pcg_with_coarse_cg_reaches_the_oracle_solution(name, prec):
    """Flexible BDDC-PCG with the coarse CG (default tolerance 1e-10):
    fp64 takes the oracle's iteration count with the exact coarse solve (to
    one) and reaches its solution to 1e-9; bf16 reaches a true residual below
    1.5e-8 and the solution to 1e-6."""
    p, mask, o = _case(name)
    b = o.rhs(p.f[:, 0])
    x_ref, h = o.pcg(b, 1e-8)
    g = _bddc(p, mask, precision=prec)
    x, res = g.pcg_solve(_cuda(b), rtol=1e-8, maxit=300)
    assert res.status == 0
    x = x.cpu().numpy()
    if prec == "fp64":
        assert abs(int(res.iters[0]) - h[0]["iters"]) <= 1
        assert _rel(x, x_ref) < 1e-9
    else:
        tr = np.linalg.norm(o.to_free(b) - o.A @ o.to_free(x)) / np.linalg.norm(o.to_free(b))
        assert tr < 1.5e-8
        assert _rel(x, x_ref) < 1e-6
    g.close()


def test_loose_coarse_tolerance_multi_rhs_and_iteration_limit():
    """A loose inner tolerance (1e-4) changes the preconditioner from apply
    to apply; flexible PCG still converges every column (a zero column takes
    no iteration) to the solution; the oracle's PCG with the same inexact
    coarse solve takes the same iterations (to two). The iteration limit is
    honoured."""
    p, mask, o = _case("3d_24_3cubed")
    nrhs = 4
    f = synth.uniform(46, o.n_nodes * nrhs).reshape(-1, nrhs)
    b = o.rhs(f)
    b[:, 2] = 0.0
    g = _bddc(p, mask, nrhs_max=nrhs, coarse_cg_rtol=1e-4)
    X, res = g.pcg_solve(_cuda(b), rtol=1e-8, maxit=300)
    assert res.status == 0 and int(res.iters[2]) == 0
    X = X.cpu().numpy()
    assert np.all(X[:, 2] == 0)
    try:
        o.set_coarse_cg(1e-4)
        xo, ho = o.pcg(b[:, [0, 3]], 1e-8, flexible=True)
    finally:
        o.set_coarse_cg(None)
    for j, c in enumerate((0, 3)):
        assert abs(int(res.iters[c]) - ho[j]["iters"]) <= 2
        assert np.linalg.norm(X[:, c] - xo[:, j]) / np.linalg.norm(xo[:, j]) < 1e-6
    g3 = _bddc(p, mask, coarse_cg_maxit=3)
    g3.apply(_cuda(b[:, 0]))
    assert g3.info()["coarse_cg_iters"] == 3
    g.close()
    g3.close()


def test_coarse_cg_graph_and_direct_bitwise_and_timeout():
    """Graph replay and direct launches give bitwise the same iterates (fixed
    reduction order); the kernel's bounded grid barrier returns a timeout
    status through the stall hook, and the handle recovers."""
    from paper_2410_14786_gb300 import BDDC, BDDCError, _lib
    p, mask, o = _case("3d_voronoi")
    b = _cuda(o.rhs(p.f[:, 0]))
    xs = []
    for graph in (True, False):
        g = BDDC.from_problem(p, constraints=mask, coarse="cg", graph=graph)
        x, res = g.pcg_solve(b, rtol=1e-8)
        xs.append((x.cpu().numpy(), int(res.iters[0])))
        if graph:
            g.test_coarse_stall(True, limit_cycles=2_000_000)
            with pytest.raises(BDDCError) as ei:
                g.pcg_solve(b, rtol=1e-8)
            assert ei.value.code == _lib.ERR_TIMEOUT
            g.test_coarse_stall(False)
            g.clear_device_error()
            x2, r2 = g.pcg_solve(b, rtol=1e-8)
            assert r2.status == 0 and np.array_equal(x2.cpu().numpy(), xs[0][0])
        g.close()
    assert xs[0][1] == xs[1][1] and np.array_equal(xs[0][0], xs[1][0])


def test_static_scratch_refuses_the_coarse_cg_mode():
    import ctypes as C
    from paper_2410_14786_gb300 import _lib
    p, mask, o = _case("cfg1_2d")
    g = _bddc(p, mask)
    r = torch.zeros(o.n_nodes, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    st = int(torch.cuda.current_stream().cuda_stream)
    rc = _lib.lib().bddc_apply_static_scratch(g.handle, C.c_void_p(r.data_ptr()), C.c_void_p(z.data_ptr()), 1, st)
    assert rc == _lib.ERR_INVALID_ARG
    g.close()
