"""Pins for the CPU oracle: closed forms, exact special cases, brute force and
invariants, each independent of the oracle's own code path (arXiv
2410.14786, Sec. 2 unless stated)."""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import synth
from oracle import ALL_GLOBS, CORNER, EDGE, FACE, Oracle, q1_element_matrices

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _oracle(p, **kw):
    return Oracle(p.dim, p.ne, p.elem_sigma, p.elem_subdomain, p.n_sub, **kw)


def _read_gold(name):
    rows = []
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.fixture(scope="module")
def cfg1():
    p = synth.config(1)
    return p, _oracle(p, constraints=CORNER | EDGE)


@pytest.fixture(scope="module")
def small3d():
    p = synth.make_problem(3, 12, 3, "lognormal", k=7)
    return p, _oracle(p)


# ---------------------------------------------------------------- inputs
def test_splitmix64_published_vectors():
    for seed, *vals in _read_gold("splitmix64.txt"):
        got = synth.splitmix64(int(seed), 3)
        assert [int(v) for v in got] == [int(v) for v in vals]


def test_uniform_and_normal_moments():
    u = synth.uniform(5, 200000)
    assert -1 <= u.min() and u.max() < 1 and abs(u.mean()) < 0.01
    z = synth.normal(6, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01


# ---------------------------------------------------------------- P1 element matrices
def test_q1_2d_closed_form():
    gold = {r[0]: r for r in _read_gold("q1_closed_forms.txt")}
    st = np.array([float(v) for v in gold["stiff2d"][1:17]]).reshape(4, 4) / 6.0
    for h in (1.0, 0.25, 1 / 64):
        K, M = q1_element_matrices(2, h)
        assert np.allclose(K, st, atol=1e-14)
        ms = np.array([float(v) for v in gold["mass2d"][1:17]]).reshape(4, 4) * h * h / 36
        assert np.allclose(M, ms, atol=1e-16)


def test_q1_3d_stencil_and_mass():
    h = 0.25
    K, M = q1_element_matrices(3, h)
    assert np.allclose(K.sum(axis=1), 0, atol=1e-15)
    ham = np.array([[bin(a ^ b).count("1") for b in range(8)] for a in range(8)])
    assert np.allclose(M, h ** 3 / 216 * 2.0 ** (3 - ham), atol=1e-17)
    # assembled stencil at an interior node of a 4^3 grid (unit sigma)
    p = synth.make_problem(3, 4, 1, "one")
    o = _oracle(p)
    n1 = 5
    c = 2 + n1 * (2 + n1 * 2)
    row = o.A.getrow(o.node2free[c]).toarray().ravel()
    hh = 1 / 4
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                nb = o.node2free[c + dx + n1 * (dy + n1 * dz)]
                k = abs(dx) + abs(dy) + abs(dz)
                want = {0: 8 * hh / 3, 1: 0.0, 2: -hh / 6, 3: -hh / 12}[k]
                assert row[nb] == pytest.approx(want, abs=1e-15)


def test_rhs_is_integral_of_interpolant():
    # sum_j (M f)_j over all nodes = integral of f_h; f = 1 gives the volume 1
    p = synth.make_problem(3, 6, 2, "one")
    o = _oracle(p)
    ones = np.ones(o.n_nodes)
    assert (o.M_full @ ones).sum() == pytest.approx(1.0, rel=1e-14)
    # f = x: integral over the unit cube is 1/2
    n1 = p.ne + 1
    x = (np.arange(o.n_nodes) % n1) / p.ne
    assert (o.M_full @ x).sum() == pytest.approx(0.5, rel=1e-14)
    b = o.rhs(ones)
    assert np.all(b[o.dir] == 0)


# ---------------------------------------------------------------- P2 subassembly
def test_subassembly_equals_global(small3d):
    p, o = small3d
    S = np.zeros((o.n_free, o.n_free))
    for i in range(o.n_sub):
        S[np.ix_(o.R[i], o.R[i])] += o.Ai[i]
    A = o.A.toarray()
    assert np.abs(S - A).max() <= 1e-14 * np.abs(A).max()


# ---------------------------------------------------------------- P3 weights
def test_weights_partition_of_unity(small3d):
    p, o = small3d
    acc = np.zeros(o.n_free)
    for i in range(o.n_sub):
        acc[o.R[i]] += o.W[i]
    assert np.allclose(acc, 1.0, atol=1e-15)


def test_weights_2d_paper_example(cfg1):
    p, o = cfg1
    w = 1.0 / o.kappa
    for kind, val, count in _read_gold("weights_2d.txt"):
        assert int(np.sum(np.isclose(w, float(val)))) == int(count), kind


def test_glob_counts_structured():
    # 2D 4x4: 9 corners + 24 edges; 3D 3^3: 8 corners + 36 edges + 54 faces
    p = synth.config(1)
    o = _oracle(p, constraints=ALL_GLOBS)
    kinds = [g.kind for g in o.globs]
    assert kinds.count(CORNER) == 9 and kinds.count(EDGE) == 24 and o.n_c == 33
    p = synth.make_problem(3, 12, 3, "one")
    o = _oracle(p)
    kinds = [g.kind for g in o.globs]
    assert (kinds.count(CORNER), kinds.count(EDGE), kinds.count(FACE)) == (8, 36, 54)
    assert {g.nodes.size for g in o.globs if g.kind == FACE} == {9}
    assert {g.nodes.size for g in o.globs if g.kind == EDGE} == {3}


# ---------------------------------------------------------------- P4 Phi, A_c
def test_phi_constraints_and_energy(small3d):
    p, o = small3d
    rng = np.random.default_rng(0)
    for i in range(o.n_sub):
        C, Phi, A = o.Ci[i], o.Phi[i], o.Ai[i]
        assert np.abs(C @ Phi - np.eye(C.shape[0])).max() < 1e-12
        # A_ci = Phi^T A Phi equals -Lambda_i (from the first block row)
        assert np.abs(o.Aci[i] + o.Lam[i]).max() < 1e-11 * max(1, np.abs(o.Aci[i]).max())
        # energy minimality among all Psi with C Psi = I
        N = sla.null_space(C)
        Psi = Phi + N @ rng.standard_normal((N.shape[1], Phi.shape[1])) * 1e-2
        assert np.trace(Psi.T @ A @ Psi) > np.trace(Phi.T @ A @ Phi)
    Ac = o.Ac.toarray()
    assert np.abs(Ac - Ac.T).max() < 1e-12 * np.abs(Ac).max()
    assert np.linalg.eigvalsh(Ac).min() > 0


# ---------------------------------------------------------------- P5 local solve
def test_local_solve_kkt(small3d):
    p, o = small3d
    rng = np.random.default_rng(1)
    for i in range(o.n_sub):
        y = rng.standard_normal(o.R[i].size)
        z, lam = o.local_solve(i, y)
        assert np.abs(o.Ci[i] @ z).max() < 1e-12 * np.abs(z).max()
        res = o.Ai[i] @ z + o.Ci[i].T @ lam - y
        assert np.abs(res).max() < 1e-11 * np.abs(y).max()


# ---------------------------------------------------------------- P6, P7 exact cases
def test_single_subdomain_is_exact():
    p = synth.make_problem(3, 6, 1, "lognormal", k=3)
    o = _oracle(p)
    assert o.n_c == 0
    r = np.random.default_rng(2).standard_normal(o.n_free)
    z = o.apply(r)
    xs = spla.spsolve(o.A.tocsc(), r)
    assert np.abs(z - xs).max() < 1e-12 * np.abs(xs).max()
    b = o.rhs(p.f[:, 0])
    _, h = o.pcg(b, 1e-8)
    assert h[0]["iters"] <= 1


@pytest.mark.parametrize("dim,ne,nsub", [(2, 12, 3), (3, 6, 2)])
def test_all_primal_is_exact(dim, ne, nsub):
    p = synth.make_problem(dim, ne, nsub, "lognormal", k=4)
    o = _oracle(p, all_primal=True)
    r = np.random.default_rng(3).standard_normal(o.n_free)
    z = o.apply(r)
    xs = spla.spsolve(o.A.tocsc(), r)
    assert np.abs(z - xs).max() < 1e-11 * np.abs(xs).max()


# ---------------------------------------------------------------- P8 explicit M
def _explicit(o):
    n = o.n_free
    Mp = np.zeros((n, n))
    B = np.zeros((n, n))
    PI = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1
        parts = o.apply_parts(e)
        Mp[:, j] = parts["z"]
        B[:, j] = parts["v1"] + parts["v2"]
        PI[:, j] = o.interior_correction(e)
    return Mp, B, PI


@pytest.mark.parametrize("dim,ne,nsub", [(2, 8, 2), (3, 4, 2)])
def test_explicit_preconditioner(dim, ne, nsub):
    p = synth.make_problem(dim, ne, nsub, "lognormal", k=5)
    o = _oracle(p)
    A = o.A.toarray()
    Mp, B, PI = _explicit(o)
    I = np.eye(o.n_free)
    Msym = PI + (I - PI @ A) @ B @ (I - A @ PI)
    assert np.abs(Msym - Msym.T).max() < 1e-12 * np.abs(Msym).max()
    # On residuals with zero interior part the paper's M^-1 equals Msym
    gam = np.flatnonzero(o.kappa >= 2)
    assert np.abs(Mp[:, gam] - Msym[:, gam]).max() < 1e-12 * np.abs(Msym).max()
    # BDDC lower bound: eigenvalues of Msym A are >= 1 (Mandel-Dohrmann 2003)
    ev = np.sort(np.linalg.eigvals(Msym @ A).real)
    assert ev[0] > 1 - 1e-10
    assert ev[-1] < 20


@pytest.mark.parametrize("dim,ne,nsub", [(2, 12, 3), (3, 6, 2), (3, 9, 3)])
def test_coarse_plus_local_is_constrained_minimiser(dim, ne, nsub):
    """v1 + v2 = sum_i R_i^T W_i w_i where (w_i, u_c) minimise
    sum_i (1/2 w_i^T A_i w_i - (W_i R_i r)^T w_i) subject to C_i w_i = R_ci u_c.
    The constrained problem is solved here as one dense KKT system, without
    Phi_i, A_c or the local solves (the BDDC definition of Dohrmann 2003)."""
    p = synth.make_problem(dim, ne, nsub, "lognormal", k=9)
    o = _oracle(p)
    r = np.random.default_rng(7).standard_normal(o.n_free)
    ns = [R.size for R in o.R]
    ms = [Rc.size for Rc in o.Rc]
    off_w = np.concatenate([[0], np.cumsum(ns)])
    off_m = off_w[-1] + np.concatenate([[0], np.cumsum(ms)])
    off_c = off_m[-1]
    N = off_c + o.n_c
    K = np.zeros((N, N))
    f = np.zeros(N)
    for i in range(o.n_sub):
        w = slice(off_w[i], off_w[i + 1])
        m = slice(off_m[i], off_m[i + 1])
        K[w, w] = o.Ai[i]
        K[w, m] = o.Ci[i].T
        K[m, w] = o.Ci[i]
        for row, g in enumerate(o.Rc[i]):
            K[off_m[i] + row, off_c + g] = -1.0
            K[off_c + g, off_m[i] + row] = -1.0
        f[w] = o.W[i] * r[o.R[i]]
    sol = np.linalg.solve(K, f)
    v = np.zeros(o.n_free)
    for i in range(o.n_sub):
        v[o.R[i]] += o.W[i] * sol[off_w[i]:off_w[i + 1]]
    parts = o.apply_parts(r)
    assert np.abs(parts["v1"] + parts["v2"] - v).max() < 1e-11 * np.abs(v).max()
    assert np.abs(parts["uc"] - sol[off_c:]).max() < 1e-11 * np.abs(sol[off_c:]).max()


# ---------------------------------------------------------------- P9, P10 invariance
def test_constraint_scaling_invariance(small3d):
    p, o = small3d
    rng = np.random.default_rng(4)
    scale = dict(enumerate(rng.uniform(0.2, 5.0, size=o.n_c)))
    o2 = _oracle(p, constraint_scale=lambda g: scale[g])
    r = rng.standard_normal(o.n_free)
    z1, z2 = o.apply(r), o2.apply(r)
    assert np.abs(z1 - z2).max() < 1e-12 * np.abs(z1).max()


def test_subdomain_renumbering_invariance(small3d):
    p, o = small3d
    perm = np.random.default_rng(5).permutation(p.n_sub)
    o2 = _oracle(synth.Problem(p.dim, p.ne, p.elem_sigma, perm[p.elem_subdomain].astype(np.int32),
                               p.n_sub, p.f))
    r = np.random.default_rng(6).standard_normal(o.n_free)
    z1, z2 = o.apply(r), o2.apply(r)
    assert np.abs(z1 - z2).max() < 1e-12 * np.abs(z1).max()


# ---------------------------------------------------------------- P11-P13 PCG
def test_pcg_start_has_zero_interior_residual(small3d):
    p, o = small3d
    b = o.to_free(o.rhs(p.f[:, 0]))
    x0 = o.interior_correction(b)
    r0 = b - o.A @ x0
    interior = np.flatnonzero(o.kappa == 1)
    assert np.abs(r0[interior]).max() < 1e-14 * np.abs(b).max()


def test_pcg_matches_direct_solve(small3d):
    p, o = small3d
    b = o.rhs(p.f[:, 0])
    x, h = o.pcg(b, 1e-10)
    assert h[0]["converged"]
    xs = spla.spsolve(o.A.tocsc(), o.to_free(b))
    assert np.linalg.norm(o.to_free(x) - xs) / np.linalg.norm(xs) < 1e-8
    true_res = np.linalg.norm(o.to_free(b) - o.A @ o.to_free(x)) / np.linalg.norm(o.to_free(b))
    assert true_res < 1.5e-10


def test_flexible_equals_standard_in_fp64(cfg1):
    p, o = cfg1
    b = o.rhs(p.f[:, 0])
    x1, h1 = o.pcg(b, 1e-8)
    x2, h2 = o.pcg(b, 1e-8, flexible=True)
    assert h1[0]["iters"] == h2[0]["iters"]
    assert np.allclose(h1[0]["alpha"], h2[0]["alpha"], rtol=1e-6)
    assert np.abs(x1 - x2).max() < 1e-8 * np.abs(x1).max()


def test_bddc_iterations_bounded_as_subdomains_grow():
    # fixed H/h = 8, 2x2 -> 4x4 -> 8x8 subdomains (the weak-scaling claim, Sec. 3)
    it_bddc, it_cg = [], []
    for nsub in (2, 4, 8):
        p = synth.make_problem(2, 8 * nsub, nsub, "one", k=8)
        o = _oracle(p, constraints=CORNER | EDGE)
        b = o.rhs(p.f[:, 0])
        _, h = o.pcg(b, 1e-8)
        _, hc = o.pcg(b, 1e-8, precond=False)
        it_bddc.append(h[0]["iters"])
        it_cg.append(hc[0]["iters"])
    assert max(it_bddc) <= 12 and it_bddc[-1] - it_bddc[0] <= 3
    assert it_cg[-1] > 4 * it_bddc[-1] and it_cg[-1] > it_cg[0]


def test_zero_rhs_column():
    p = synth.make_problem(2, 8, 2, "one")
    o = _oracle(p)
    b = np.zeros((o.n_nodes, 2))
    b[:, 1] = o.rhs(p.f[:, 0])
    x, h = o.pcg(b, 1e-8)
    assert h[0]["iters"] == 0 and np.all(x[:, 0] == 0)
    assert h[1]["converged"]


# ---------------------------------------------- inexact coarse solve (Sec. 3)
# The paper solves the coarse system of Eq. coarsegrid with plain CG. Pins of
# the oracle's CG: properties the method has whatever the matrix.
def _energy(A, e):
    return float(np.sqrt(e @ (A @ e)))


def test_coarse_cg_energy_error_decreases_and_residuals_are_true(small3d):
    p, o = small3d
    rc = o.coarse_residual(o.to_free(o.rhs(p.f[:, 0])))
    u_star = o.Ac_lu.solve(rc)
    errs = []
    for k in range(0, 25):
        u, it, norms = o.coarse_solve_cg(rc, 0.0, maxit=k)
        assert it == k
        errs.append(_energy(o.Ac, u - u_star))
        # the recursively updated residual norm is the true one
        assert abs(norms[-1] - np.linalg.norm(rc - o.Ac @ u)) <= 1e-10 * np.linalg.norm(rc)
    # CG minimises the A-norm error over the Krylov space: strictly decreasing
    assert all(b < a for a, b in zip(errs, errs[1:]))


def test_coarse_cg_finite_termination_and_stop_test(cfg1):
    p, o = cfg1
    assert o.n_c == 33
    rc = o.coarse_residual(o.to_free(o.rhs(p.f[:, 0])))
    u_star = o.Ac_lu.solve(rc)
    u, it, norms = o.coarse_solve_cg(rc, 1e-13)
    # exact in at most n_c steps in exact arithmetic; a few more in float64
    assert it <= o.n_c + 5
    assert np.linalg.norm(u - u_star) <= 1e-10 * np.linalg.norm(u_star)
    assert norms[-1] <= 1e-13 * norms[0] < norms[-2]
    u0, it0, _ = o.coarse_solve_cg(np.zeros_like(rc), 1e-8)
    assert it0 == 0 and not u0.any()


def test_pcg_with_inexact_coarse_solve(small3d):
    p, o = small3d
    b = o.rhs(p.f[:, 0])
    x_ref, h_ref = o.pcg(b, 1e-8)
    try:
        o.set_coarse_cg(1e-13)      # tight: the same preconditioner up to rounding
        x1, h1 = o.pcg(b, 1e-8, flexible=True)
        o.set_coarse_cg(1e-4)       # loose: the flexible iteration still converges
        x2, h2 = o.pcg(b, 1e-8, flexible=True)
    finally:
        o.set_coarse_cg(None)
    assert h1[0]["iters"] == h_ref[0]["iters"]
    assert np.abs(x1 - x_ref).max() < 1e-9 * np.abs(x_ref).max()
    assert h2[0]["converged"] and h2[0]["iters"] <= h_ref[0]["iters"] + 5
    xs = spla.spsolve(o.A.tocsc(), o.to_free(b))
    assert np.linalg.norm(o.to_free(x2) - xs) / np.linalg.norm(xs) < 1e-6
