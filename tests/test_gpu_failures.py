"""Failure detection on the GPU without a GPU fault: a non-finite right-hand
side injected on the host must end PCG with BDDC_ERR_BREAKDOWN, and a
bounded device wait that runs out (a grid barrier of the coarse solve told
to wait for one arrival more than its grid makes, with a limit of about a
millisecond) must come back as BDDC_ERR_TIMEOUT. In both cases the handle
and the CUDA context stay usable: the next clean solve matches the oracle."""
import numpy as np
import pytest

import synth
from oracle import Oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def case():
    from paper_2410_14786_gb300 import build
    build.build()
    p = synth.make_problem(3, 16, 2, "lognormal", k=71)
    o = Oracle(p.dim, p.ne, p.elem_sigma, p.elem_subdomain, p.n_sub)
    b = o.rhs(p.f[:, 0])
    x_ref, h = o.pcg(b, 1e-8)
    return p, o, b, x_ref, h[0]["iters"]


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
@pytest.mark.parametrize("graph", [True, False])
def test_nan_right_hand_side_is_a_breakdown(case, prec, graph):
    from paper_2410_14786_gb300 import BDDC, _lib
    p, o, b, x_ref, iters = case
    g = BDDC.from_problem(p, precision=prec, graph=graph, nrhs_max=2)
    bad = b.copy()
    bad[o.n_nodes // 2 + 3] = np.nan
    B = torch.from_numpy(np.stack([b, bad], axis=1)).cuda()
    _, res = g.pcg_solve(B, rtol=1e-8, maxit=200, allow_breakdown=True)
    assert res.status == _lib.ERR_BREAKDOWN
    assert int(res.iters[1]) == 0
    assert int(res.iters[0]) >= iters - 1       # the clean column still converged
    # the next clean solve on the same handle succeeds
    x, res = g.pcg_solve(torch.from_numpy(b).cuda(), rtol=1e-8, maxit=200)
    assert res.status == _lib.OK
    assert _rel(x.cpu().numpy(), x_ref) < (1e-10 if prec == "fp64" else 1e-6)
    assert g.info()["device_error"] == 0
    g.close()


@pytest.mark.parametrize("graph", [True, False])
def test_coarse_barrier_wait_runs_out(case, graph):
    """The coarse solve's grid barrier waits, bounded, for an arrival that
    never comes: the apply records BDDC_ERR_TIMEOUT, PCG stops with it, and
    after the flag is cleared the handle solves normally."""
    from paper_2410_14786_gb300 import BDDC, BDDCError, _lib
    p, o, b, x_ref, iters = case
    g = BDDC.from_problem(p, coarse="sparse", graph=graph)
    bt = torch.from_numpy(b).cuda()
    x, res = g.pcg_solve(bt, rtol=1e-8)
    assert res.status == _lib.OK
    g.test_coarse_stall(True, limit_cycles=2_000_000)      # about 1 ms at 2 GHz
    g.apply(bt)
    torch.cuda.synchronize()
    assert g.info()["device_error"] == _lib.ERR_TIMEOUT
    with pytest.raises(BDDCError) as ei:
        g.pcg_solve(bt, rtol=1e-8)
    assert ei.value.code == _lib.ERR_TIMEOUT
    # the flag stays set until cleared, even with the normal barrier back
    g.test_coarse_stall(False)
    with pytest.raises(BDDCError):
        g.pcg_solve(bt, rtol=1e-8)
    g.clear_device_error()
    assert g.info()["device_error"] == 0
    x, res = g.pcg_solve(bt, rtol=1e-8)
    assert res.status == _lib.OK and int(res.iters[0]) == iters
    assert _rel(x.cpu().numpy(), x_ref) < 1e-10
    # a second handle on the same context was never affected
    g2 = BDDC.from_problem(p, coarse="sparse")
    x2, r2 = g2.pcg_solve(bt, rtol=1e-8)
    assert r2.status == _lib.OK and torch.equal(x2, x)
    g.close()
    g2.close()


def test_coarse_stall_needs_the_sparse_coarse_solve(case):
    from paper_2410_14786_gb300 import BDDC, BDDCError
    p = case[0]
    g = BDDC.from_problem(p, coarse="dense")
    with pytest.raises(BDDCError):
        g.test_coarse_stall(True, 1000)
    g.close()
