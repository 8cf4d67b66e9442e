"""GPU: the adjoint gradient dJ/dsigma through the C ABI and torch.autograd,
against the adjoint oracle (direct solves, itself pinned by central
differences). J(sigma) = 1/2 ||u(sigma) - u_obs||^2."""
import numpy as np
import pytest

import synth
from oracle import adjoint_oracle as ad
from oracle import dirichlet_mask
from oracle.bddc_oracle import element_nodes, q1_element_matrices

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2410_14786_gb300 import build
    build.build()


def _load(p):
    dim, ne = p.dim, p.ne
    _, Mref = q1_element_matrices(dim, 1.0 / ne)
    en = element_nodes(dim, ne)
    B = np.zeros((((ne + 1) ** dim), p.f.shape[1]))
    for k in range(p.f.shape[1]):
        np.add.at(B[:, k], en, p.f[en, k] @ Mref.T)
    B[dirichlet_mask(dim, ne)] = 0.0
    return B


def _setup(dim, ne, nsub, k, nrhs=1):
    p = synth.make_problem(dim, ne, nsub, "lognormal", nrhs=nrhs, k=k)
    B = _load(p)
    pert = p.elem_sigma * np.exp(0.1 * synth.normal(3000 + k, p.elem_sigma.size))
    Uobs = ad.solve(dim, ne, pert, B)
    return p, B, Uobs


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("dim,ne,nrhs", [(2, 12, 1), (3, 8, 1), (3, 8, 3)])
def test_elem_grad_kernel_matches_oracle(dim, ne, nrhs):
    from paper_2410_14786_gb300 import BDDC
    p = synth.make_problem(dim, ne, 2, "lognormal", nrhs=1, k=81)
    g = BDDC.from_problem(p, nrhs_max=nrhs)
    n = (ne + 1) ** dim
    U = synth.uniform(82, n * nrhs).reshape(n, nrhs)
    L = synth.uniform(83, n * nrhs).reshape(n, nrhs)
    want = ad.element_gradient(dim, ne, np.where(dirichlet_mask(dim, ne)[:, None], 0.0, U),
                               np.where(dirichlet_mask(dim, ne)[:, None], 0.0, L))
    # Dirichlet entries are treated as 0 whatever they hold
    got = g.elem_grad(_cuda(U if nrhs > 1 else U[:, 0]), _cuda(L if nrhs > 1 else L[:, 0])).cpu().numpy()
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("dim,ne,nsub,prec", [(2, 24, 3, "fp64"), (3, 12, 3, "fp64"), (3, 12, 3, "bf16")])
def test_autograd_gradient_matches_oracle(dim, ne, nsub, prec):
    from paper_2410_14786_gb300 import adjoint
    p, B, Uobs = _setup(dim, ne, nsub, 91 + dim)
    b, u_obs = B[:, 0], Uobs[:, 0]
    J_o, g_o, u_o, lam_o = ad.gradient(dim, ne, p.elem_sigma, b, u_obs)
    sigma = torch.tensor(p.elem_sigma, dtype=torch.float64, requires_grad=True)
    free = torch.from_numpy(~dirichlet_mask(dim, ne)).cuda()
    u = adjoint.solve(sigma, _cuda(b), dim, ne, p.elem_subdomain, p.n_sub, rtol=1e-12, precision=prec)
    J = 0.5 * ((u - _cuda(u_obs))[free] ** 2).sum()
    J.backward()
    # PCG to rtol 1e-12 in both the forward and the adjoint solve
    assert abs(float(J.detach()) - J_o) <= 1e-9 * J_o
    gs = sigma.grad.numpy()
    assert np.linalg.norm(gs - g_o) <= 1e-8 * np.linalg.norm(g_o)
    # homogeneity: sum_e sigma_e dJ/dsigma_e = -(u - u_obs)^T u
    un = u.detach().cpu().numpy()
    fr = ~dirichlet_mask(dim, ne)
    rhs = -float((un - u_obs)[fr] @ un[fr])
    assert abs(float(p.elem_sigma @ gs) - rhs) <= 1e-8 * abs(rhs)


def test_autograd_several_columns_and_b_gradient():
    from paper_2410_14786_gb300 import adjoint
    dim, ne = 3, 12
    p, B, Uobs = _setup(dim, ne, 3, 97, nrhs=3)
    J_o, g_o, _, lam_o = ad.gradient(dim, ne, p.elem_sigma, B, Uobs)
    sigma = torch.tensor(p.elem_sigma, dtype=torch.float64, requires_grad=True)
    b = _cuda(B).requires_grad_(True)
    free = torch.from_numpy(~dirichlet_mask(dim, ne)).cuda()
    u = adjoint.solve(sigma, b, dim, ne, p.elem_subdomain, p.n_sub, rtol=1e-12)
    J = 0.5 * ((u - _cuda(Uobs))[free] ** 2).sum()
    J.backward()
    assert np.linalg.norm(sigma.grad.numpy() - g_o) <= 1e-8 * np.linalg.norm(g_o)
    # dJ/db = lambda
    assert np.abs(b.grad.cpu().numpy() - lam_o).max() <= 1e-8 * np.abs(lam_o).max()
