"""GPU: the tensor-core path (tcgen05) for the local and interior operators.

The BF16 operator values are the same on the tensor cores and on the CUDA
cores (both round the float64 operators to bfloat16 once), so the two paths
must agree far below the form's own error: they differ only in the operand
(split into bfloat16 hi + lo, about 2^-17 relative, against float32) and in
the float32 accumulation order. Against the oracle each form keeps the bound
derived from its unit roundoff (BF16 2^-8, TF32 2^-10)."""
import numpy as np
import pytest

import synth
from oracle import CORNER, EDGE, FACE, Oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2410_14786_gb300 import build
    build.build()


def _small_voronoi():
    sub, n, cell = synth.voronoi_partition(12, 8, 91)
    s = synth.layer_sigma(12, cell)
    f = synth.uniform(92, 13 ** 3 * 2).reshape(-1, 2)
    return synth.Problem(3, 12, s, sub, n, f, "voronoi_12_8")


CASES = {
    # 8^3-element cubes: interior 343, interface up to 386 dofs (3 and 4 row tiles)
    "3d_24_3cubed": lambda: synth.make_problem(3, 24, 3, "lognormal", k=21),
    # uneven cells
    "3d_voronoi": _small_voronoi,
    # 2D: small operators (one partial row tile, narrow column chunks)
    "cfg1_2d": lambda: synth.config(1),
}
_CACHE = {}


def _case(name):
    if name not in _CACHE:
        p = CASES[name]()
        mask = (CORNER | EDGE) if p.dim == 2 else 0
        o = Oracle(p.dim, p.ne, p.elem_sigma, p.elem_subdomain, p.n_sub, constraints=mask or (CORNER | EDGE | FACE))
        _CACHE[name] = (p, mask, o)
    return _CACHE[name]


def _bddc(p, mask, **kw):
    from paper_2410_14786_gb300 import BDDC
    return BDDC.from_problem(p, constraints=mask, **kw)


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _colrel(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    return max(float(np.linalg.norm(a[:, k] - b[:, k]) / max(np.linalg.norm(b[:, k]), 1e-300))
               for k in range(b.shape[1]))


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("nrhs", [1, 5, 16, 40, 64])
def test_tc_bf16_matches_cuda_core_bf16(name, nrhs):
    p, mask, o = _case(name)
    tc = _bddc(p, mask, precision="bf16", nrhs_max=64, tensor_cores=True)
    cc = _bddc(p, mask, precision="bf16", nrhs_max=64, tensor_cores=False)
    assert tc.info()["tensor_cores"] == 1 and cc.info()["tensor_cores"] == 0
    r = synth.uniform(300 + nrhs, o.n_nodes * nrhs).reshape(o.n_nodes, nrhs)
    r[o.dir] = 0
    rt = _cuda(r if nrhs > 1 else r[:, 0])
    z_tc = tc.apply(rt).cpu().numpy().reshape(o.n_nodes, nrhs)
    z_cc = cc.apply(rt).cpu().numpy().reshape(o.n_nodes, nrhs)
    assert np.all(np.isfinite(z_tc))
    assert _colrel(z_tc, z_cc) < 2e-4
    assert np.all(z_tc[o.dir] == 0)
    if nrhs <= 5:
        want = o.apply_nodes(r if nrhs > 1 else r[:, 0]).reshape(o.n_nodes, nrhs)
        assert _colrel(z_tc, want) < 3e-2


@pytest.mark.parametrize("name", list(CASES))
def test_tc_tf32_apply_error_bound(name):
    # operators read as TF32 (u = 2^-10 or 2^-11), operand split hi + lo in
    # float32 (about 2^-21), float32 accumulation over n <= 729 terms
    p, mask, o = _case(name)
    g = _bddc(p, mask, precision="tf32", nrhs_max=4, tensor_cores=True)
    assert g.info()["tensor_cores"] == 1
    r = synth.uniform(41, o.n_nodes * 3).reshape(o.n_nodes, 3)
    r[o.dir] = 0
    z = g.apply(_cuda(r)).cpu().numpy()
    want = o.apply_nodes(r)
    assert _colrel(z, want) < 1e-2
    g32 = _bddc(p, mask, precision="fp32", nrhs_max=4)
    z32 = g32.apply(_cuda(r)).cpu().numpy()
    # TF32 sits between FP32 and BF16
    assert _colrel(z, want) > _colrel(z32, want)


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_tc_flexible_pcg_reaches_fp64_accuracy(prec):
    p, mask, o = _case("3d_24_3cubed")
    b = o.rhs(p.f[:, 0])
    x_star, _ = o.pcg(b, 1e-12)
    g64 = _bddc(p, mask)
    x64, r64 = g64.pcg_solve(_cuda(b), rtol=1e-8)
    g = _bddc(p, mask, precision=prec, tensor_cores=True)
    x, res = g.pcg_solve(_cuda(b), rtol=1e-8, maxit=500)
    assert res.status == 0
    bt = torch.from_numpy(b).cuda()
    true_res = (bt - g64.matvec(_cuda(x.cpu().numpy()))).norm() / bt.norm()
    assert float(true_res) < 1.5e-8
    e64 = np.linalg.norm(x64.cpu().numpy() - x_star) / np.linalg.norm(x_star)
    e = np.linalg.norm(x.cpu().numpy() - x_star) / np.linalg.norm(x_star)
    assert e < 10 * max(e64, 1e-12)
    assert int(res.iters[0]) <= 2 * int(r64.iters[0]) + 2


def test_tc_pcg_many_rhs():
    # 24 right-hand sides (N = 32) on uneven cells: every column converges, and
    # a column solved alone takes the same number of iterations (+-1)
    p, mask, o = _case("3d_voronoi")
    nrhs = 24
    g = _bddc(p, mask, precision="bf16", nrhs_max=nrhs)
    assert g.info()["tensor_cores"] == 1
    f = synth.uniform(42, o.n_nodes * nrhs).reshape(-1, nrhs)
    B = _cuda(o.rhs(f))
    X, res = g.pcg_solve(B, rtol=1e-8)
    assert res.status == 0
    x7, r7 = g.pcg_solve(B[:, 7].contiguous(), rtol=1e-8)
    assert abs(int(res.iters[7]) - int(r7.iters[0])) <= 1
    xs = o.pcg(o.rhs(f[:, [7]]), 1e-10)[0][:, 0]
    assert np.linalg.norm(X[:, 7].cpu().numpy() - xs) / np.linalg.norm(xs) < 1e-6


@pytest.mark.parametrize("nrhs_max", [1, 4])
def test_tf32_auto_below_eight_rhs_runs_the_fp32_form(nrhs_max):
    """AUTO keeps TF32 off the tensor cores below 8 right-hand sides: the
    handle stores and applies float32 operators on the CUDA cores, exactly
    what the FP32 form does (bitwise the same apply and solve)."""
    p, mask, o = _case("3d_24_3cubed")
    gt = _bddc(p, mask, precision="tf32", nrhs_max=nrhs_max)
    gf = _bddc(p, mask, precision="fp32", nrhs_max=nrhs_max)
    it, jf = gt.info(), gf.info()
    assert it["tensor_cores"] == 0 and it["precision"] == 1
    assert it["symmetric_operators"] == jf["symmetric_operators"]
    r = synth.uniform(44, o.n_nodes * nrhs_max).reshape(o.n_nodes, nrhs_max)
    r[o.dir] = 0
    R = _cuda(r if nrhs_max > 1 else r[:, 0])
    assert torch.equal(gt.apply(R), gf.apply(R))
    b = _cuda(o.rhs(p.f[:, 0]))
    xt, rt = gt.pcg_solve(b, rtol=1e-8)
    xf, rf = gf.pcg_solve(b, rtol=1e-8)
    assert rt.status == 0 and list(rt.iters) == list(rf.iters) and torch.equal(xt, xf)
