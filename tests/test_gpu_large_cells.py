"""GPU parity at the operator sizes of the 128^3 Voronoi workload (cells of
64 to 4862 dofs), on a small mesh the oracle finishes in seconds: 24^3
elements split by 6 Voronoi seeds into 7 cells of 8 to 4626 dofs (interior
operators A_II^-1 of up to 3580 rows, interface operators K_GG of up to 1357
rows, one cell of 8 dofs with no interior). This reaches the code paths of
that workload: tensor-core GEMM units of several 128-row tiles and operators
of more than 1024 rows (several units per operator), and the CUDA-core
streamed GEMV on rows of about 3600 entries. Comparisons are element-wise
(largest entry difference over the largest entry), against the oracle of
Sec. 2 (arXiv 2410.14786)."""
import numpy as np
import pytest

import synth
from oracle import Oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NRHS = 64


@pytest.fixture(scope="module")
def case():
    from paper_2410_14786_gb300 import build
    build.build()
    sub, n, cell = synth.voronoi_partition(24, 6, 96)
    sigma = synth.layer_sigma(24, cell)
    f = synth.uniform(97, 25 ** 3 * NRHS).reshape(-1, NRHS)
    p = synth.Problem(3, 24, sigma, sub, n, f, "voronoi_24_6")
    o = Oracle(p.dim, p.ne, p.elem_sigma, p.elem_subdomain, p.n_sub)
    R = synth.uniform(98, o.n_nodes * NRHS).reshape(-1, NRHS)
    R[o.dir] = 0
    Z = o.apply_nodes(R)
    return p, o, R, Z


def _cols(A, k):
    """The first k columns: a vector for k = 1 (as the binding returns)."""
    return np.ascontiguousarray(A[:, 0] if k == 1 else A[:, :k])


def _rel(a, b):
    assert a.shape == b.shape, (a.shape, b.shape)
    return float(np.abs(a - b).max() / np.abs(b).max())


def _fp64_tol(o):
    """Float64 parity bound for this case: the coarse residual sums up to
    n_G,max terms (rounding n_G,max eps relative) and the coarse solve
    amplifies that by cond(A_c) (253 here, against 42 for the cubes of 8^3
    elements whose cases use 1e-11): n_G,max cond(A_c) eps = 7.6e-11."""
    ng = max(len(r) - len(i) for r, i in zip(o.R, o.interior))
    return ng * np.linalg.cond(o.Ac.toarray()) * np.finfo(np.float64).eps


def _bddc(p, **kw):
    from paper_2410_14786_gb300 import BDDC
    return BDDC.from_problem(p, **kw)


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_the_case_reaches_the_large_operator_sizes(case):
    p, o, R, Z = case
    ni = [len(r) for r in o.R]
    nI = [len(i) for i in o.interior]
    assert max(ni) > 4500 and max(nI) > 3500 and min(nI) == 0
    assert max(a - b for a, b in zip(ni, nI)) > 1024    # K_GG: more than 8 tensor-core tiles
    g = _bddc(p, nrhs_max=1)
    assert g.info()["max_ni"] == max(ni)
    g.close()


@pytest.mark.parametrize("nrhs", [1, 8])
def test_large_cells_fp64(case, nrhs):
    p, o, R, Z = case
    tol = _fp64_tol(o)
    assert tol < 1e-10
    g = _bddc(p, precision="fp64", nrhs_max=nrhs)
    z = g.apply(_cuda(_cols(R, nrhs))).cpu().numpy()
    assert _rel(z, _cols(Z, nrhs)) < tol
    rc, uc = g.coarse_vectors(nrhs)
    parts = o.apply_parts(o.to_free(R[:, 0]))
    assert _rel(rc.cpu().numpy()[:, 0], parts["rc"]) < 1e-12
    assert _rel(uc.cpu().numpy()[:, 0], parts["uc"]) < tol
    g.close()


# The low-precision bounds, on the largest entry error over the largest
# entry: operator entries rounded to the format's unit roundoff u (fp32
# 6.0e-8, tf32 4.9e-4, bf16 3.9e-3) plus float32 accumulation over up to
# 3580 terms (sqrt(3580) u = 3.6e-6 for fp32). Bounds: fp32 5e-6, tf32 2e-3
# (4 u), bf16 1e-2 (2.6 u); measured on GB300: 5.3e-7, 5.8e-4, 2.3e-3.
@pytest.mark.parametrize("nrhs", [1, 8, NRHS])
def test_large_cells_fp32_cuda_cores(case, nrhs):
    p, o, R, Z = case
    g = _bddc(p, precision="fp32", nrhs_max=nrhs)
    assert g.info()["tensor_cores"] == 0
    z = g.apply(_cuda(_cols(R, nrhs))).cpu().numpy()
    assert _rel(z, _cols(Z, nrhs)) < 5e-6
    g.close()


@pytest.mark.parametrize("nrhs", [1, 8])
def test_large_cells_bf16_cuda_cores(case, nrhs):
    p, o, R, Z = case
    g = _bddc(p, precision="bf16", nrhs_max=nrhs, tensor_cores=False)
    z = g.apply(_cuda(_cols(R, nrhs))).cpu().numpy()
    assert _rel(z, _cols(Z, nrhs)) < 1e-2
    g.close()


@pytest.mark.parametrize("nrhs", [8, 40, NRHS])
def test_large_cells_bf16_tensor_cores_match_cuda_cores(case, nrhs):
    """The same BF16 operator values on both engines: the tensor-core GEMM
    (units of several 128-row tiles, operators split over several units)
    matches the CUDA-core GEMV entry by entry to the operand split's rounding
    (about 2^-17) and float32 summation order."""
    p, o, R, Z = case
    gt = _bddc(p, precision="bf16", nrhs_max=nrhs, tensor_cores=True)
    gc = _bddc(p, precision="bf16", nrhs_max=nrhs, tensor_cores=False)
    assert gt.info()["tensor_cores"] == 1
    X = _cuda(R[:, :nrhs])
    zt, zc = gt.apply(X).cpu().numpy(), gc.apply(X).cpu().numpy()
    assert _rel(zt, zc) < 2e-4
    assert _rel(zt, Z[:, :nrhs]) < 1e-2
    gt.close()
    gc.close()


@pytest.mark.parametrize("nrhs", [8, NRHS])
def test_large_cells_tf32_tensor_cores(case, nrhs):
    p, o, R, Z = case
    g = _bddc(p, precision="tf32", nrhs_max=nrhs)
    assert g.info()["tensor_cores"] == 1
    z = g.apply(_cuda(R[:, :nrhs])).cpu().numpy()
    assert _rel(z, Z[:, :nrhs]) < 2e-3
    g.close()


def test_large_cells_pcg_fp64_iterates(case):
    """PCG on the large cells: the same iterations, solution and per-iteration
    residual norms, alphas and betas as the oracle's."""
    p, o, R, Z = case
    b = o.rhs(p.f[:, 0])
    xo, h = o.pcg(b, 1e-8)
    g = _bddc(p, precision="fp64", history=300)
    x, res = g.pcg_solve(_cuda(b), rtol=1e-8, maxit=300)
    assert res.status == 0 and int(res.iters[0]) == h[0]["iters"]
    assert _rel(x.cpu().numpy(), xo) < 1e-10
    hg = g.pcg_history()
    it = h[0]["iters"]
    # ||r_k|| to 1e-12 ||r_0|| (the recursively updated residual carries
    # absolute rounding of order eps ||r_0||), alpha_k and beta_k to 1e-10
    rn = np.asarray(h[0]["rnorm"])
    assert np.all(np.abs(hg["rnorm"][:it + 1, 0] - rn) <= 1e-12 * rn[0])
    al = np.asarray(h[0]["alpha"])
    assert np.all(np.abs(hg["alpha"][:it, 0] - al) <= 1e-10 * np.abs(al))
    be = np.asarray(h[0]["beta"])
    assert np.all(np.abs(hg["beta"][:it - 1, 0] - be) <= 1e-10 * np.abs(be))
    g.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_large_cells_flexible_pcg_many_rhs(case, prec):
    """64 right-hand sides through the mixed forms (tensor cores for bf16):
    every column reaches a true residual below 1.5e-8 and the oracle's
    solution to the solver tolerance."""
    p, o, R, Z = case
    cols = [0, 17, NRHS - 1]
    b = o.rhs(p.f)
    g = _bddc(p, precision=prec, nrhs_max=NRHS)
    g64 = _bddc(p, precision="fp64", nrhs_max=NRHS)
    B = _cuda(b)
    X, res = g.pcg_solve(B, rtol=1e-8, maxit=300)
    assert res.status == 0
    tr = (B - g64.matvec(X)).norm(dim=0) / B.norm(dim=0)
    assert float(tr.max()) < 1.5e-8
    xo, _ = o.pcg(b[:, cols], 1e-12)
    Xc = X[:, cols].cpu().numpy()
    assert np.linalg.norm(Xc - xo) / np.linalg.norm(xo) < 1e-6
    g.close()
    g64.close()
