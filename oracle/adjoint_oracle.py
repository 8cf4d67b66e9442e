"""CPU oracle for the adjoint gradient of a BDDC-solved diffusion problem.

TEST INFRASTRUCTURE ONLY: imported by the tests (and the smoke check); the
product path never calls it and shares no code with it.

Objective (read from the workload statement; the paper itself has no
gradient): J(sigma) = 1/2 sum_k ||u_k(sigma) - u_obs,k||_2^2 over the free
nodal values, where A(sigma) u_k = b_k, A(sigma) = sum_e sigma_e R_e^T K_ref
R_e is the Q1 stiffness matrix with homogeneous Dirichlet nodes eliminated,
and b does not depend on sigma.

Gradient by the adjoint method: because A is symmetric,
    lambda_k = A^-1 (u_k - u_obs,k),
    dJ/dsigma_e = - sum_k lambda_k,e^T K_ref u_k,e,
with u_k,e, lambda_k,e the 2^dim nodal values of element e (zero on
Dirichlet nodes). Every linear solve here is a sparse direct solve (SciPy
SuperLU), so the oracle's only error is rounding.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .bddc_oracle import dirichlet_mask, element_nodes, q1_element_matrices


def stiffness(dim: int, ne: int, sigma: np.ndarray):
    """(A on the free nodes as CSR, free-node indices, element nodes, K_ref)."""
    h = 1.0 / ne
    K, _ = q1_element_matrices(dim, h)
    en = element_nodes(dim, ne)
    nloc = en.shape[1]
    rows = np.repeat(en, nloc, axis=1).reshape(-1)
    cols = np.tile(en, (1, nloc)).reshape(-1)
    vals = (np.asarray(sigma, dtype=np.float64)[:, None] * K.reshape(1, -1)).reshape(-1)
    n = (ne + 1) ** dim
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    free = np.flatnonzero(~dirichlet_mask(dim, ne))
    return A[free][:, free].tocsc(), free, en, K


def solve(dim: int, ne: int, sigma: np.ndarray, b_nodes: np.ndarray) -> np.ndarray:
    """u = A(sigma)^-1 b on the free nodes, returned at all nodes (0 on Dirichlet)."""
    A, free, _, _ = stiffness(dim, ne, sigma)
    b = np.asarray(b_nodes, dtype=np.float64)
    two = b.ndim == 2
    B = b if two else b[:, None]
    U = np.zeros_like(B)
    U[free] = spla.splu(A).solve(np.ascontiguousarray(B[free]))
    return U if two else U[:, 0]


def objective(dim, ne, sigma, b_nodes, u_obs) -> float:
    """J(sigma) = 1/2 ||u(sigma) - u_obs||^2 over the free nodes (summed over columns)."""
    u = solve(dim, ne, sigma, b_nodes)
    d = (u - u_obs)[~dirichlet_mask(dim, ne)]
    return 0.5 * float(np.sum(d * d))


def element_gradient(dim: int, ne: int, u_nodes: np.ndarray, lam_nodes: np.ndarray) -> np.ndarray:
    """g_e = - sum_k lambda_k,e^T K_ref u_k,e for every element (the dA/dsigma_e term)."""
    K = q1_element_matrices(dim, 1.0 / ne)[0]
    en = element_nodes(dim, ne)
    U = u_nodes if u_nodes.ndim == 2 else u_nodes[:, None]
    L = lam_nodes if lam_nodes.ndim == 2 else lam_nodes[:, None]
    g = np.zeros(en.shape[0])
    for k in range(U.shape[1]):
        ue = U[en, k]                 # [n_elems, 2^dim]
        le = L[en, k]
        g -= np.einsum("ea,ab,eb->e", le, K, ue)
    return g


def gradient(dim, ne, sigma, b_nodes, u_obs):
    """(J, dJ/dsigma, u, lambda) by one forward and one adjoint direct solve."""
    A, free, _, _ = stiffness(dim, ne, sigma)
    lu = spla.splu(A)
    b = np.asarray(b_nodes, dtype=np.float64)
    two = b.ndim == 2
    B = b if two else b[:, None]
    Uo = u_obs if two else u_obs[:, None]
    U = np.zeros_like(B)
    U[free] = lu.solve(np.ascontiguousarray(B[free]))
    R = np.zeros_like(B)
    R[free] = (U - Uo)[free]
    Lam = np.zeros_like(B)
    Lam[free] = lu.solve(np.ascontiguousarray(R[free]))    # A symmetric: A^T = A
    J = 0.5 * float(np.sum(R * R))
    g = element_gradient(dim, ne, U, Lam)
    if not two:
        U, Lam = U[:, 0], Lam[:, 0]
    return J, g, U, Lam
