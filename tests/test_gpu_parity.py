"""GPU parity: libbddc (through its C ABI) against the CPU oracle on the same
seeded inputs (arXiv 2410.14786, Sec. 2). FP64 to 1e-11 relative per apply
and 1e-10 per PCG solution; low-precision forms within bounds derived from
their unit roundoff."""
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


def _oracle(p, mask=0):
    return Oracle(p.dim, p.ne, p.elem_sigma, p.elem_subdomain, p.n_sub,
                  constraints=mask or (CORNER | EDGE | FACE))


def _bddc(p, precision="fp64", mask=0, nrhs_max=1, coarse="auto", phi_fp64=False, coarse_blocks=0,
          full_operators=False, history=0, graph=True):
    from paper_2410_14786_gb300 import BDDC
    return BDDC.from_problem(p, precision=precision, constraints=mask, nrhs_max=nrhs_max, coarse=coarse,
                             phi_fp64=phi_fp64, coarse_blocks=coarse_blocks, full_operators=full_operators,
                             history=history, graph=graph)


def _assert_history_matches(hg, ho, col, tol=1e-10, tol_r=1e-12):
    """Per-iteration PCG scalars of one column against the oracle's: alpha_k
    for k < iters and the beta after iteration k + 1 for k < iters - 1, each
    to `tol` relative; ||r_k|| for k = 0 .. iters to tol_r ||r_0||; NaN
    beyond. The residual is updated recursively (r_k+1 = r_k - alpha_k A p_k),
    so both sides carry absolute rounding of order eps ||r_0|| in it: by
    iteration k its norm has fallen to about 1e-8 ||r_0|| and agrees only to
    about 1e-8 of itself, but to 1e-15 ||r_0|| (measured on GB300; alpha and
    beta agree to 7e-12 relative at every k)."""
    it = ho["iters"]
    rn = hg["rnorm"][:, col]
    al = hg["alpha"][:, col]
    be = hg["beta"][:, col]
    want_rn = np.asarray(ho["rnorm"])
    assert np.all(np.abs(rn[:it + 1] - want_rn) <= tol_r * want_rn[0]), (rn[:it + 1], want_rn)
    assert np.all(np.isnan(rn[it + 1:]))
    if it:
        want_al = np.asarray(ho["alpha"])
        assert np.all(np.abs(al[:it] - want_al) <= tol * np.abs(want_al)), (al[:it], want_al)
    assert np.all(np.isnan(al[it:]))
    if it > 1:
        want_be = np.asarray(ho["beta"])
        assert want_be.size == it - 1
        assert np.all(np.abs(be[:it - 1] - want_be) <= tol * np.abs(want_be)), (be[:it - 1], want_be)
    assert np.all(np.isnan(be[max(it - 1, 0):]))


def _small_voronoi():
    sub, n, cell = synth.voronoi_partition(12, 8, 91)
    s = synth.layer_sigma(12, cell)
    f = synth.uniform(92, 13 ** 3 * 2).reshape(-1, 2)
    return synth.Problem(3, 12, s, sub, n, f, "voronoi_12_8")


CASES = {
    "cfg1_2d": (lambda: synth.config(1), CORNER | EDGE),
    "3d_24_3cubed": (lambda: synth.make_problem(3, 24, 3, "lognormal", k=21), 0),
    "3d_voronoi": (_small_voronoi, 0),
    "3d_corners_only": (lambda: synth.make_problem(3, 16, 2, "lognormal", k=22), CORNER),
    "2d_single_sub": (lambda: synth.make_problem(2, 20, 1, "lognormal", k=23), 0),
}
_CACHE = {}


def _case(name):
    if name not in _CACHE:
        make, mask = CASES[name]
        p = make()
        _CACHE[name] = (p, mask, _oracle(p, mask))
    return _CACHE[name]


def _rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("name", list(CASES))
def test_matvec_and_rhs(name):
    p, mask, o = _case(name)
    g = _bddc(p, mask=mask, nrhs_max=3)
    x = synth.uniform(31, o.n_nodes * 3).reshape(-1, 3)
    y = g.matvec(_cuda(x)).cpu().numpy()
    want = np.stack([o.matvec_nodes(np.where(o.dir, 0, x[:, k])) for k in range(3)], axis=1)
    assert _rel(y, want) < 1e-13
    f = synth.uniform(32, o.n_nodes * 3).reshape(-1, 3)
    b = g.rhs(_cuda(f)).cpu().numpy()
    assert _rel(b, o.rhs(f)) < 1e-13


@pytest.mark.parametrize("name", list(CASES))
def test_apply_fp64(name):
    p, mask, o = _case(name)
    g = _bddc(p, mask=mask)
    r = synth.uniform(33, o.n_nodes)
    r[o.dir] = 0
    z = g.apply(_cuda(r)).cpu().numpy()
    parts = o.apply_parts(o.to_free(r))
    assert _rel(z, o.to_nodes(parts["z"])) < 1e-11
    assert np.all(z[o.dir] == 0)
    if o.n_c:
        rc, uc = g.coarse_vectors()
        assert _rel(rc.cpu().numpy()[:, 0], parts["rc"]) < 1e-11
        assert _rel(uc.cpu().numpy()[:, 0], parts["uc"]) < 1e-11


@pytest.mark.parametrize("name", ["cfg1_2d", "3d_24_3cubed", "3d_voronoi", "3d_corners_only"])
def test_apply_sparse_coarse(name):
    """The supernodal (nested-dissection) coarse factorisation gives the same
    exact coarse solve as the dense inverse."""
    p, mask, o = _case(name)
    g = _bddc(p, mask=mask, nrhs_max=3, coarse="sparse")
    assert g.info()["coarse_levels"] >= 1
    r = synth.uniform(37, o.n_nodes * 3).reshape(-1, 3)
    r[o.dir] = 0
    z = g.apply(_cuda(r)).cpu().numpy()
    assert _rel(z, o.apply_nodes(r)) < 1e-11
    rc, uc = g.coarse_vectors(3)
    want = np.stack([o.apply_parts(o.to_free(r[:, k]))["uc"] for k in range(3)], axis=1)
    assert _rel(uc.cpu().numpy(), want) < 1e-11


def _coarse_level_launches(g, on):
    t = g.get_tuning()
    t["coarse_level_launches"] = 1 if on else 0
    g.set_tuning(t)


@pytest.mark.parametrize("level", [False, True])
@pytest.mark.parametrize("name,blocks", [("cfg1_2d", 0), ("3d_24_3cubed", 0), ("3d_voronoi", 0),
                                         ("3d_corners_only", 0), ("3d_voronoi", 1)])
def test_one_column_sparse_coarse(name, blocks, level):
    """One right-hand side: the sweeps of the sparse coarse solve in their
    gather form (one dot product per output value; one cooperative launch
    with warps assigned on the host, or one launch per level with groups of
    lanes sized to the rows) give the oracle's exact u_c."""
    p, mask, o = _case(name)
    g = _bddc(p, mask=mask, coarse="sparse", coarse_blocks=blocks)
    _coarse_level_launches(g, level)
    r = synth.uniform(38, o.n_nodes)
    r[o.dir] = 0
    z = g.apply(_cuda(r)).cpu().numpy()
    parts = o.apply_parts(o.to_free(r))
    assert _rel(z, o.to_nodes(parts["z"])) < 1e-11
    rc, uc = g.coarse_vectors()
    assert _rel(rc.cpu().numpy()[:, 0], parts["rc"]) < 1e-11
    assert _rel(uc.cpu().numpy()[:, 0], parts["uc"]) < 1e-11


@pytest.mark.parametrize("blocks", [0, 1, 3])
def test_one_column_sparse_coarse_many_levels(blocks):
    """48^3 elements in 8^3 cubes: 2863 coarse dofs, 4 levels. With one or
    three blocks every warp walks more than 32 units of a level. The one-column
    sweeps against the dense inverse (pinned to the oracle above) and against
    the multi-column sweeps; the PCG iteration count is unchanged."""
    p = synth.make_problem(3, 48, 8, "lognormal", k=24)
    gs = _bddc(p, coarse="sparse", coarse_blocks=blocks)
    assert gs.info()["coarse_levels"] >= 3
    _coarse_level_launches(gs, blocks == 3)   # the per-level launches once
    gd = _bddc(p, coarse="dense")
    gm = _bddc(p, coarse="sparse", nrhs_max=2)
    n = (p.ne + 1) ** 3
    r = torch.from_numpy(synth.uniform(39, n * 2).reshape(n, 2)).cuda()
    zs, zd = gs.apply(r[:, 0].contiguous()), gd.apply(r[:, 0].contiguous())
    _, uc_s = gs.coarse_vectors()
    _, uc_d = gd.coarse_vectors()
    zm = gm.apply(r)
    _, uc_m = gm.coarse_vectors(2)
    assert float((uc_s[:, 0] - uc_d[:, 0]).abs().max() / uc_d.abs().max()) < 1e-11
    assert float((uc_s[:, 0] - uc_m[:, 0]).abs().max() / uc_d.abs().max()) < 1e-11
    assert float((zs - zd).abs().max() / zd.abs().max()) < 1e-11
    assert float((zs - zm[:, 0]).abs().max() / zd.abs().max()) < 1e-11
    b = gs.rhs(torch.from_numpy(p.f[:, 0].copy()).cuda())
    xs, rs = gs.pcg_solve(b, rtol=1e-8)
    xd, rd = gd.pcg_solve(b, rtol=1e-8)
    assert rs.status == 0 and int(rs.iters[0]) == int(rd.iters[0])
    assert float((xs - xd).norm() / xd.norm()) < 1e-9
    for g in (gs, gd, gm):
        g.close()


@pytest.mark.parametrize("name", ["3d_voronoi", "3d_corners_only", "cfg1_2d"])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_symmetric_operator_storage(name, prec):
    """At one right-hand side the fp32 and bf16 forms store A_II^-1 and K_GG
    as lower triangles (diagonal halved) and apply y = L' x + L'^T x: the
    apply matches full storage to the accumulation's rounding, and PCG
    reaches the oracle's solution. Uneven subdomains (Voronoi), 343- and
    386-row operators (8^3-element cubes) and 2D."""
    p, mask, o = _case(name)
    gs = _bddc(p, precision=prec, mask=mask)
    gf = _bddc(p, precision=prec, mask=mask, full_operators=True)
    assert gs.info()["symmetric_operators"] == 1 and gf.info()["symmetric_operators"] == 0
    assert gs.info()["interior_op_bytes"] < 0.7 * gf.info()["interior_op_bytes"]
    r = synth.uniform(43, o.n_nodes)
    r[o.dir] = 0
    zs, zf = gs.apply(_cuda(r)).cpu().numpy(), gf.apply(_cuda(r)).cpu().numpy()
    # same stored values (bf16 / fp32 roundings of the same entries), float32
    # sums in another order
    assert _rel(zs, zf) < (3e-5 if prec == "bf16" else 3e-6)
    assert np.all(zs[o.dir] == 0)
    b = o.rhs(p.f[:, 0])
    xo, _ = o.pcg(b, 1e-8)
    x, res = gs.pcg_solve(_cuda(b), rtol=1e-8)
    assert res.status == 0 and _rel(x.cpu().numpy(), xo) < 1e-6
    gs.close()
    gf.close()


def test_pcg_sparse_coarse_matches_oracle():
    p, mask, o = _case("3d_voronoi")
    g = _bddc(p, mask=mask, coarse="sparse")
    b = o.rhs(p.f[:, 0])
    xo, h = o.pcg(b, 1e-8)
    x, res = g.pcg_solve(_cuda(b), rtol=1e-8)
    assert int(res.iters[0]) == h[0]["iters"]
    assert _rel(x.cpu().numpy(), xo) < 1e-10


def test_apply_ignores_dirichlet_input_and_multi_rhs():
    p, mask, o = _case("3d_24_3cubed")
    g = _bddc(p, mask=mask, nrhs_max=5)
    r = synth.uniform(34, o.n_nodes * 5).reshape(-1, 5)   # nonzero Dirichlet entries
    z = g.apply(_cuda(r)).cpu().numpy()
    want = o.apply_nodes(np.where(o.dir[:, None], 0, r))
    assert _rel(z, want) < 1e-11
    z1 = g.apply(_cuda(np.ascontiguousarray(r[:, 2]))).cpu().numpy()
    assert _rel(z1, want[:, 2]) < 1e-11


@pytest.mark.parametrize("graph", [True, False])
@pytest.mark.parametrize("name", ["cfg1_2d", "3d_24_3cubed", "3d_voronoi", "3d_corners_only"])
def test_pcg_fp64_matches_oracle(name, graph):
    """The FP64 PCG iterates match the oracle's: the same iteration count, the
    solution to 1e-10, and at every iteration k the residual norm ||r_k||,
    alpha_k and beta_k to 1e-10 relative (whole-solve graph and direct
    launches)."""
    p, mask, o = _case(name)
    g = _bddc(p, mask=mask, history=200, graph=graph)
    b = o.rhs(p.f[:, 0])
    xo, h = o.pcg(b, 1e-8)
    x, res = g.pcg_solve(_cuda(b), rtol=1e-8, maxit=500)
    x = x.cpu().numpy()
    assert res.status == 0
    assert int(res.iters[0]) == h[0]["iters"]
    assert _rel(x, xo) < 1e-10
    assert abs(res.relres[0] - h[0]["rnorm"][-1] / np.linalg.norm(o.to_free(b))) < 1e-10
    _assert_history_matches(g.pcg_history(), h[0], 0)
    g.close()


def test_pcg_multi_rhs_and_zero_column():
    """Independent columns (one of them zero): per-column iteration counts,
    solutions and per-iteration histories match the oracle's."""
    p, mask, o = _case("cfg1_2d")
    g = _bddc(p, mask=mask, nrhs_max=3, history=100)
    f = synth.uniform(35, o.n_nodes * 3).reshape(-1, 3)
    b = o.rhs(f)
    b[:, 1] = 0.0
    xo, h = o.pcg(b, 1e-8)
    x, res = g.pcg_solve(_cuda(b), rtol=1e-8)
    x = x.cpu().numpy()
    assert list(res.iters) == [hh["iters"] for hh in h]
    assert np.all(x[:, 1] == 0)
    assert _rel(x, xo) < 1e-10
    hg = g.pcg_history(nrhs=3)
    for k in (0, 2):
        _assert_history_matches(hg, h[k], k)
    assert hg["rnorm"][0, 1] == 0.0 and np.all(np.isnan(hg["rnorm"][1:, 1]))


@pytest.mark.parametrize("name,nrhs", [("3d_24_3cubed", 8), ("3d_voronoi", 64), ("cfg1_2d", 16)])
def test_apply_many_rhs_matches_single_columns(name, nrhs):
    """Blocks of 8..64 right-hand sides: every column equals the apply of that
    column alone, and the oracle (columns in blocks wider than the lanes per
    operator row included)."""
    p, mask, o = _case(name)
    g = _bddc(p, mask=mask, nrhs_max=nrhs)
    R = synth.uniform(38, o.n_nodes * nrhs).reshape(-1, nrhs)
    R[o.dir] = 0
    Z = g.apply(_cuda(R)).cpu().numpy()
    for k in (0, nrhs // 2, nrhs - 1):
        zk = g.apply(_cuda(np.ascontiguousarray(R[:, k]))).cpu().numpy()
        assert _rel(Z[:, k], zk) < 1e-13
    cols = [0, 5, nrhs - 1]
    want = o.apply_nodes(R[:, cols])
    assert _rel(Z[:, cols], want) < 1e-11


def test_pcg_many_rhs_converges_like_single():
    p, mask, o = _case("3d_voronoi")
    nrhs = 8
    g = _bddc(p, mask=mask, nrhs_max=nrhs, precision="bf16")
    f = synth.uniform(39, o.n_nodes * nrhs).reshape(-1, nrhs)
    B = _cuda(o.rhs(f))
    X, res = g.pcg_solve(B, rtol=1e-8)
    assert res.status == 0
    x3, r3 = g.pcg_solve(B[:, 3].contiguous(), rtol=1e-8)
    assert abs(int(res.iters[3]) - int(r3.iters[0])) <= 1
    xs = o.pcg(o.rhs(f[:, [3]]), 1e-10)[0][:, 0]
    assert np.linalg.norm(X[:, 3].cpu().numpy() - xs) / np.linalg.norm(xs) < 1e-6


def test_graph_and_direct_launches_are_bitwise_identical():
    """The captured-graph iteration and directly launched kernels compute the
    same thing, and reductions have a fixed order: solutions agree bit for bit,
    run after run."""
    p, mask, o = _case("3d_24_3cubed")
    b = _cuda(o.rhs(p.f[:, 0]))
    from paper_2410_14786_gb300 import BDDC
    xs = []
    for graph in (True, True, False):
        g = BDDC.from_problem(p, precision="bf16", constraints=mask, graph=graph)
        x, res = g.pcg_solve(b, rtol=1e-8)
        xs.append((x.cpu().numpy(), int(res.iters[0])))
        g.close()
    assert xs[0][1] == xs[1][1] == xs[2][1]
    assert np.array_equal(xs[0][0], xs[1][0]) and np.array_equal(xs[0][0], xs[2][0])


def test_pcg_host_buffers():
    p, mask, o = _case("3d_24_3cubed")
    g = _bddc(p, mask=mask)
    b = o.rhs(p.f[:, 0])
    xo, h = o.pcg(b, 1e-8)
    x, res = g.pcg_solve_host(b, rtol=1e-8)
    assert int(res.iters[0]) == h[0]["iters"]
    assert _rel(x, xo) < 1e-10


def test_single_subdomain_converges_in_one_iteration():
    p, mask, o = _case("2d_single_sub")
    g = _bddc(p, mask=mask)
    b = o.rhs(p.f[:, 0])
    x, res = g.pcg_solve(_cuda(b), rtol=1e-8)
    assert int(res.iters[0]) <= 1


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-5), ("bf16", 3e-2)])
def test_apply_low_precision_error_bound(prec, tol):
    # operators rounded to the format's unit roundoff u (fp32 6e-8, bf16 4e-3),
    # operand rounded as well, float32 accumulation over n <= 729 terms
    p, mask, o = _case("3d_24_3cubed")
    g = _bddc(p, precision=prec, mask=mask)
    r = synth.uniform(36, o.n_nodes)
    r[o.dir] = 0
    z = g.apply(_cuda(r)).cpu().numpy()
    want = o.apply_nodes(r)
    err = np.linalg.norm(z - want) / np.linalg.norm(want)
    assert err < tol


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-5), ("bf16", 3e-2)])
def test_phi_precision_option(prec, tol):
    # Phi_i is float32 by default in the low-precision forms; kept in float64
    # the apply obeys the same bound, and the two differ by float32 rounding of
    # the coarse component (operand and products rounded to 6e-8, float32
    # accumulation over n_G <= 386 terms), far below the form's own error
    p, mask, o = _case("3d_24_3cubed")
    r = synth.uniform(37, o.n_nodes)
    r[o.dir] = 0
    want = o.apply_nodes(r)
    g32 = _bddc(p, precision=prec, mask=mask)
    g64 = _bddc(p, precision=prec, mask=mask, phi_fp64=True)
    assert g32.info()["phi_precision"] == 1 and g64.info()["phi_precision"] == 0
    z32 = g32.apply(_cuda(r)).cpu().numpy()
    z64 = g64.apply(_cuda(r)).cpu().numpy()
    assert np.linalg.norm(z64 - want) / np.linalg.norm(want) < tol
    assert np.linalg.norm(z32 - z64) / np.linalg.norm(z64) < 1e-5


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_flexible_pcg_reaches_fp64_accuracy(prec):
    p, mask, o = _case("3d_24_3cubed")
    b = o.rhs(p.f[:, 0])
    x_star, _ = o.pcg(b, 1e-12)
    g64 = _bddc(p, mask=mask)
    x64, r64 = g64.pcg_solve(_cuda(b), rtol=1e-8)
    g = _bddc(p, precision=prec, mask=mask)
    x, res = g.pcg_solve(_cuda(b), rtol=1e-8, maxit=500)
    assert res.status == 0
    xt = _cuda(x.cpu().numpy())
    true_res = (torch.from_numpy(b).cuda() - g64.matvec(xt)).norm() / torch.from_numpy(b).cuda().norm()
    assert float(true_res) < 1.5e-8
    e64 = np.linalg.norm(x64.cpu().numpy() - x_star) / np.linalg.norm(x_star)
    e = np.linalg.norm(x.cpu().numpy() - x_star) / np.linalg.norm(x_star)
    assert e < 10 * max(e64, 1e-12)
    assert int(res.iters[0]) <= 2 * int(r64.iters[0]) + 2


def test_full_size_config2_properties():
    """96^3 elements, 12^3 subdomains (the benchmark workload): properties that
    hold at any size, since the oracle cannot run this size inside a test."""
    from oracle import dirichlet_mask
    p = synth.config(2)
    g = _bddc(p)
    inf = g.info()
    assert inf["n_c"] == 10439 and inf["n_free"] == 857375
    n1 = p.ne + 1
    idx = np.arange(g.n_nodes)
    coords = np.stack([idx % n1, (idx // n1) % n1, idx // (n1 * n1)])
    dmask = dirichlet_mask(3, p.ne)
    iface = (np.any(coords % 8 == 0, axis=0)) & ~dmask      # box subdomains of 8^3
    gen = torch.Generator(device="cuda").manual_seed(5)

    def rand_iface():
        v = torch.rand(g.n_nodes, dtype=torch.float64, device="cuda", generator=gen) - 0.5
        v[torch.from_numpy(~iface).cuda()] = 0
        return v

    # on residuals with zero interior part M^-1 is symmetric positive definite
    u, v = rand_iface(), rand_iface()
    Mu, Mv = g.apply(u), g.apply(v)
    assert abs(float(u @ Mv - v @ Mu)) < 1e-10 * float(u.norm() * Mv.norm())
    assert float(u @ Mu) > 0 and float(v @ Mv) > 0
    # PCG reaches rtol with a true residual below the tolerance
    f = torch.from_numpy(p.f[:, 0].copy()).cuda()
    b = g.rhs(f)
    x, res = g.pcg_solve(b, rtol=1e-8, maxit=300)
    assert res.status == 0 and 5 <= int(res.iters[0]) <= 80
    tr = (b - g.matvec(x)).norm() / b.norm()
    assert float(tr) < 1.5e-8
    # the sparse coarse factorisation agrees with the dense inverse at this size
    gs = _bddc(p, coarse="sparse")
    assert gs.info()["coarse_levels"] > 3
    r = rand_iface()
    z_d = g.apply(r)
    _, uc_d = g.coarse_vectors()
    z_s = gs.apply(r)
    _, uc_s = gs.coarse_vectors()
    assert float((uc_s - uc_d).abs().max() / uc_d.abs().max()) < 1e-11
    assert float((z_s - z_d).abs().max() / z_d.abs().max()) < 1e-11
    _coarse_level_launches(gs, True)
    z_l = gs.apply(r)
    _, uc_l = gs.coarse_vectors()
    assert float((uc_l - uc_d).abs().max() / uc_d.abs().max()) < 1e-11
    assert float((z_l - z_d).abs().max() / z_d.abs().max()) < 1e-11
    gs.close()
    # the mixed forms reach the same solution to the solver tolerance
    for prec in ("fp32", "bf16"):
        gm = _bddc(p, precision=prec)
        xm, rm = gm.pcg_solve(b, rtol=1e-8, maxit=300)
        assert rm.status == 0
        assert float((xm - x).norm() / x.norm()) < 1e-6
        gm.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_whole_solve_graph(prec):
    """The whole solve runs as one CUDA graph (a conditional WHILE node over
    the iteration, its condition set on the device) and gives the same
    iterates as launching every kernel directly."""
    p, mask, o = _case("3d_24_3cubed")
    b = _cuda(o.rhs(p.f[:, 0]))
    from paper_2410_14786_gb300 import BDDC
    gg = BDDC.from_problem(p, precision=prec, constraints=mask)
    gd = BDDC.from_problem(p, precision=prec, constraints=mask, graph=False)
    xg, rg = gg.pcg_solve(b, rtol=1e-8)
    assert gg.info()["solve_graph"] == 1
    xd, rd = gd.pcg_solve(b, rtol=1e-8)
    assert list(rg.iters) == list(rd.iters)
    assert torch.equal(xg, xd)
    # maxit is honoured inside the graph, and a second solve replays it
    x3, r3 = gg.pcg_solve(b, rtol=1e-8, maxit=3)
    assert int(r3.iters[0]) == 3 and r3.status == 1
    x4, r4 = gg.pcg_solve(b, rtol=1e-8)
    assert torch.equal(x4, xg)


def test_history_graph_equals_direct_and_mixed_form():
    """The flexible (BF16) PCG records its history too: the graph replay and
    direct launches give bitwise equal scalars, ||r_k|| decreases to below
    rtol ||b||, and a history shorter than the solve keeps its first entries."""
    p, mask, o = _case("3d_24_3cubed")
    b = _cuda(o.rhs(p.f[:, 0]))
    hs = []
    for graph in (True, False):
        g = _bddc(p, precision="bf16", mask=mask, history=64, graph=graph)
        x, res = g.pcg_solve(b, rtol=1e-8)
        hs.append((g.pcg_history(), int(res.iters[0])))
        g.close()
    (h1, it1), (h2, it2) = hs
    assert it1 == it2
    for key in ("rnorm", "alpha", "beta"):
        assert np.array_equal(h1[key], h2[key], equal_nan=True)
    rn = h1["rnorm"][:it1 + 1, 0]
    assert rn[-1] <= 1e-8 * float(b.norm()) < rn[-2]
    g = _bddc(p, mask=mask, history=4)
    g.pcg_solve(b, rtol=1e-8)
    short = g.pcg_history()
    gl = _bddc(p, mask=mask, history=64)
    gl.pcg_solve(b, rtol=1e-8)
    long = gl.pcg_history()
    assert np.array_equal(short["rnorm"], long["rnorm"][:5])
    from paper_2410_14786_gb300 import BDDCError
    with pytest.raises(BDDCError):
        g.pcg_history(n_iter=5)
