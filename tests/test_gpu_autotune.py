"""GPU: the launch-parameter autotuner and the tuning cache. The candidates
differ only in scheduling: with one right-hand side the apply is bitwise
unchanged; with several, only the order of the coarse sums may change."""
import json

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2410_14786_gb300 import build
    build.build()


def _p():
    return synth.make_problem(3, 24, 3, "lognormal", k=21)


def _r(n, nrhs, seed):
    r = synth.uniform(seed, n * nrhs).reshape(n, nrhs)
    return torch.from_numpy(r if nrhs > 1 else r[:, 0].copy()).cuda()


def test_autotune_one_rhs_is_bitwise_neutral():
    from paper_2410_14786_gb300 import BDDC
    p = _p()
    g = BDDC.from_problem(p, precision="bf16")
    r = _r(g.n_nodes, 1, 101)
    z0 = g.apply(r).clone()
    t = g.autotune()
    # one right-hand side in bf16: the symmetric GEMV, tuned over (stages, stage size)
    assert g.info()["symmetric_operators"] == 1
    assert t["gemv_stage_kb_interior"] in (10, 12, 16, 20, 24)
    assert t["gemv_stage_kb_interface"] in (10, 12, 16, 20, 24)
    assert t["sym_stages_interior"] in (3, 4) and t["sym_stages_interface"] in (3, 4)
    assert t["gemv_rows_interior"] in (64, 128, 256) and t["gemv_rows_interface"] in (64, 128, 256)
    assert g.get_tuning() == t
    z1 = g.apply(r)
    assert torch.equal(z0, z1)


def test_autotune_several_rhs():
    from paper_2410_14786_gb300 import BDDC
    p = _p()
    g = BDDC.from_problem(p, precision="fp32", nrhs_max=8, tensor_cores="auto")
    r = _r(g.n_nodes, 8, 102)
    z0 = g.apply(r).clone()
    t = g.autotune(8)
    assert 2 <= t["coarse_rowblock_min_nrhs"] <= 65
    z1 = g.apply(r)
    assert float((z1 - z0).norm() / z0.norm()) < 1e-12
    # a solve after the change re-captures its iteration graph
    b = g.rhs(_r(g.n_nodes, 8, 103))
    x, res = g.pcg_solve(b, rtol=1e-8)
    assert res.status == 0


def test_set_tuning_rejects_out_of_range():
    from paper_2410_14786_gb300 import BDDC, BDDCError
    g = BDDC.from_problem(_p())
    before = g.get_tuning()
    for bad in ({"gemv_stage_kb_interior": 0}, {"gemv_stage_kb_interface": 65}, {"coarse_rowblock_min_nrhs": 1},
                {"gemv_rows_interior": 100}, {"coarse_overlap": 2}, {"sym_stages_interior": 5},
                {"sym_stages_interface": 2}):
        t = dict(before)
        t.update(bad)
        with pytest.raises(BDDCError):
            g.set_tuning(t)
    assert g.get_tuning() == before


def test_tune_cache_roundtrip(tmp_path):
    from paper_2410_14786_gb300 import BDDC
    p = _p()
    path = str(tmp_path / "tune.json")
    g1 = BDDC.from_problem(p, precision="bf16", tune_cache=path)
    assert not g1.tuned_from_cache
    table = json.load(open(path))
    assert len(table) == 1
    g2 = BDDC.from_problem(p, precision="bf16", tune_cache=path)
    assert g2.tuned_from_cache
    assert g2.get_tuning() == g1.get_tuning() == list(table.values())[0]
    # another form is another key
    g3 = BDDC.from_problem(p, precision="fp32", tune_cache=path)
    assert not g3.tuned_from_cache
    assert len(json.load(open(path))) == 2


@pytest.mark.parametrize("prec,nrhs", [("bf16", 1), ("fp64", 1), ("bf16", 8)])
def test_coarse_overlap_is_bitwise_neutral(prec, nrhs):
    """The interface operator on a second stream, concurrent with the coarse
    residual and solve, computes exactly what the one-stream apply does, in
    direct launches and inside the captured solve graph."""
    from paper_2410_14786_gb300 import BDDC
    p = _p()
    g = BDDC.from_problem(p, precision=prec, nrhs_max=nrhs)
    r = _r(g.n_nodes, nrhs, 104)
    t = g.get_tuning()
    z0 = g.apply(r).clone()
    b = g.rhs(_r(g.n_nodes, nrhs, 105))
    x0, r0 = g.pcg_solve(b, rtol=1e-8)
    t1 = dict(t)
    t1["coarse_overlap"] = 1
    g.set_tuning(t1)
    assert g.get_tuning()["coarse_overlap"] == 1
    z1 = g.apply(r)
    assert torch.equal(z0, z1)
    x1, r1 = g.pcg_solve(b, rtol=1e-8)
    assert list(r0.iters) == list(r1.iters)
    assert torch.equal(x0, x1)
