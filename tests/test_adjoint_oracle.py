"""Pins of the adjoint-gradient oracle (CPU).

J(sigma) = 1/2 ||u(sigma) - u_obs||^2 with A(sigma) u = b. Pinned by
(a) central finite differences of J (step 1e-6, direct solves) on seeded
elements, (b) the homogeneity identity: A is linear in sigma, so
u(c sigma) = u / c and d/dc J(c sigma) at c = 1 gives
sum_e sigma_e dJ/dsigma_e = -(u - u_obs)^T u, a closed form independent of
the element formula, (c) J = 0 and g = 0 when u_obs = u, (d) the element
term on a single element against the assembled matrix."""
import numpy as np
import pytest

import synth
from oracle import adjoint_oracle as ad
from oracle import dirichlet_mask


def _problem(dim, ne, k):
    p = synth.make_problem(dim, ne, 2, "lognormal", nrhs=1, k=k)
    sigma = p.elem_sigma
    n_nodes = (ne + 1) ** dim
    # load b = M f from the same seeded f as the workloads
    from oracle.bddc_oracle import element_nodes, q1_element_matrices
    _, Mref = q1_element_matrices(dim, 1.0 / ne)
    en = element_nodes(dim, ne)
    b = np.zeros(n_nodes)
    np.add.at(b, en, (p.f[en, 0] @ Mref.T))
    b[dirichlet_mask(dim, ne)] = 0.0
    # observations: the solution at sigma * exp(0.1 N(0,1)) (own seed)
    pert = sigma * np.exp(0.1 * synth.normal(3000 + k, sigma.size))
    u_obs = ad.solve(dim, ne, pert, b)
    return sigma, b, u_obs


@pytest.mark.parametrize("dim,ne", [(2, 8), (3, 6)])
def test_gradient_matches_central_differences(dim, ne):
    sigma, b, u_obs = _problem(dim, ne, 31 + dim)
    J, g, u, lam = ad.gradient(dim, ne, sigma, b, u_obs)
    assert J > 0
    picks = [int(v % np.uint64(sigma.size)) for v in synth.splitmix64(5000 + dim, 8)]
    step = 1e-6
    for e in picks:
        sp_, sm_ = sigma.copy(), sigma.copy()
        sp_[e] += step
        sm_[e] -= step
        fd = (ad.objective(dim, ne, sp_, b, u_obs) - ad.objective(dim, ne, sm_, b, u_obs)) / (2 * step)
        assert abs(fd - g[e]) <= 1e-5 * abs(g[e]) + 1e-9 * np.abs(g).max(), (e, fd, g[e])


@pytest.mark.parametrize("dim,ne", [(2, 10), (3, 6)])
def test_homogeneity_identity(dim, ne):
    sigma, b, u_obs = _problem(dim, ne, 41 + dim)
    J, g, u, lam = ad.gradient(dim, ne, sigma, b, u_obs)
    free = ~dirichlet_mask(dim, ne)
    lhs = float(sigma @ g)
    rhs = -float((u - u_obs)[free] @ u[free])
    assert abs(lhs - rhs) <= 1e-11 * abs(rhs)


def test_zero_misfit_gives_zero_gradient():
    sigma, b, _ = _problem(3, 6, 51)
    u = ad.solve(3, 6, sigma, b)
    J, g, _, lam = ad.gradient(3, 6, sigma, b, u)
    assert J == 0.0
    assert np.abs(g).max() == 0.0


def test_element_term_is_the_assembled_bilinear_form():
    # with one right-hand side, sum_e g_e sigma_e' for sigma' = indicator of
    # element e0 equals -lambda^T A(indicator) u, A assembled independently
    dim, ne = 3, 4
    rng_u = synth.uniform(61, (ne + 1) ** dim)
    rng_l = synth.uniform(62, (ne + 1) ** dim)
    d = dirichlet_mask(dim, ne)
    rng_u[d] = 0
    rng_l[d] = 0
    g = ad.element_gradient(dim, ne, rng_u, rng_l)
    for e0 in (0, 13, ne ** dim - 1):
        ind = np.zeros(ne ** dim)
        ind[e0] = 1.0
        A, free, _, _ = ad.stiffness(dim, ne, ind)
        want = -float(rng_l[free] @ (A @ rng_u[free]))
        assert abs(g[e0] - want) <= 1e-13 * max(1.0, abs(want))


def test_several_columns_sum():
    sigma, b, u_obs = _problem(2, 8, 71)
    B = np.stack([b, 0.5 * b], axis=1)
    Uo = np.stack([u_obs, 0.3 * u_obs], axis=1)
    J2, g2, _, _ = ad.gradient(2, 8, sigma, B, Uo)
    Ja, ga, _, _ = ad.gradient(2, 8, sigma, b, u_obs)
    Jb, gb, _, _ = ad.gradient(2, 8, sigma, 0.5 * b, 0.3 * u_obs)
    assert abs(J2 - (Ja + Jb)) <= 1e-12 * J2
    assert np.abs(g2 - (ga + gb)).max() <= 1e-12 * np.abs(g2).max()
