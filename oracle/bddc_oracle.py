"""CPU oracle for BDDC-preconditioned CG (Goebel, Cojean, Anzt: "BDDC
preconditioning on GPUs for Cardiac Simulations", arXiv 2410.14786, Sec. 2).

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU
baseline leg of the benchmark may import this module. The product path (the
CUDA library and its Python binding) never calls it and shares no code with
it.

Plain, slow and literal, in float64:
  * Q1 element matrices by 2-point Gauss quadrature; global A by sparse
    assembly over all elements; b = M f with the consistent Q1 mass matrix.
  * Subassembly A = sum_i R_i^T A_i R_i with local Neumann matrices A_i
    (Sec. 2, first paragraph).
  * Constraints C_i: point values on corners, averages over edges and faces;
    weights W_i = diag(1/kappa) (Sec. 2, second paragraph).
  * Phi_i, Lambda_i from the saddle-point system (Eq. saddlepoint) solved as
    a whole with an LU factorisation of the full KKT matrix; A_ci =
    Phi_i^T A_i Phi_i; A_c = sum_i R_ci^T A_ci R_ci.
  * M^-1 r = v1 + v2 + v3 (Sec. 2): coarse residual r_c, coarse correction
    v1 (Eq. coarsegrid), local saddle-point solves for z_i (Eq. compzi),
    local correction v2 (Eq. localsubdomain), r1 = r - A (v1 + v2) with the
    global A, interior correction v3 (Eq. inner).
  * PCG from the static-condensation start x0 = P_I b, standard or flexible.
  * Optionally the coarse system solved inexactly by plain CG (Sec. 3).

Readings where the paper is silent (each is listed with its reason in the
design notes): Dirichlet nodes are eliminated; b = M f; globs are classes of
interface nodes with the same set of subdomains, split into mesh-connected
components (one node = corner, else edge / face average with weight 1/|G|);
stop when ||r_k||_2 <= rtol ||b||_2 per right-hand side.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

CORNER, EDGE, FACE = 1, 2, 4
ALL_GLOBS = CORNER | EDGE | FACE


# ---------------------------------------------------------------------------
# Q1 finite elements
# ---------------------------------------------------------------------------

def q1_element_matrices(dim: int, h: float):
    """Stiffness and mass matrix of one Q1 element [0,h]^dim, unit sigma.

    Local node a sits at the corner with coordinate bit d = (a >> d) & 1.
    Both integrals use the tensor 2-point Gauss rule, which is exact for the
    Q1 integrands.
    """
    g = 1.0 / math.sqrt(3.0)
    pts = [(1.0 - g) / 2.0, (1.0 + g) / 2.0]
    nloc = 2 ** dim
    K = np.zeros((nloc, nloc))
    M = np.zeros((nloc, nloc))

    def phi(bit, x):
        return x if bit else 1.0 - x

    def dphi(bit):
        return 1.0 if bit else -1.0

    for q in range(2 ** dim):
        xi = [pts[(q >> d) & 1] for d in range(dim)]
        w = 0.5 ** dim                              # reference weights
        vals = np.empty(nloc)
        grads = np.empty((nloc, dim))
        for a in range(nloc):
            bits = [(a >> d) & 1 for d in range(dim)]
            vals[a] = np.prod([phi(bits[d], xi[d]) for d in range(dim)])
            for d in range(dim):
                grads[a, d] = dphi(bits[d]) * np.prod(
                    [phi(bits[e], xi[e]) for e in range(dim) if e != d])
        jac = h ** dim
        K += w * (grads @ grads.T) / (h * h) * jac
        M += w * np.outer(vals, vals) * jac
    return K, M


def element_nodes(dim: int, ne: int) -> np.ndarray:
    """[n_elems, 2^dim] global node ids of every element, local order a."""
    n1 = ne + 1
    e = np.arange(ne ** dim)
    ex = e % ne
    ey = (e // ne) % ne
    ez = e // (ne * ne) if dim == 3 else np.zeros_like(e)
    out = np.empty((e.size, 2 ** dim), dtype=np.int64)
    for a in range(2 ** dim):
        bx, by, bz = a & 1, (a >> 1) & 1, (a >> 2) & 1
        out[:, a] = (ex + bx) + n1 * ((ey + by) + n1 * (ez + bz))
    return out


def dirichlet_mask(dim: int, ne: int) -> np.ndarray:
    n1 = ne + 1
    idx = np.arange(n1 ** dim)
    coords = [idx % n1, (idx // n1) % n1]
    if dim == 3:
        coords.append(idx // (n1 * n1))
    m = np.zeros(idx.size, dtype=bool)
    for c in coords:
        m |= (c == 0) | (c == ne)
    return m


# ---------------------------------------------------------------------------
# The decomposed problem
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Glob:
    nodes: np.ndarray          # free-node indices (free numbering), sorted
    subs: tuple                # subdomains sharing it
    kind: int                  # CORNER, EDGE or FACE


class Oracle:
    """Setup of the BDDC preconditioner for one problem (all in float64).

    Parameters
    ----------
    dim, ne, elem_sigma, elem_subdomain, n_sub : the problem (see `synth`).
    constraints : bitmask of CORNER | EDGE | FACE globs that become primal.
    all_primal : every interface node is its own corner constraint (the
        special case in which BDDC is exact).
    constraint_scale : optional callable(glob_id) -> float that multiplies
        the constraint row of that glob (used to check that M^-1 does not
        depend on the scaling of C_i).
    """

    def __init__(self, dim, ne, elem_sigma, elem_subdomain, n_sub,
                 constraints=ALL_GLOBS, all_primal=False, constraint_scale=None):
        self.dim, self.ne = dim, ne
        self.h = 1.0 / ne
        self.sigma = np.asarray(elem_sigma, dtype=np.float64)
        self.part = np.asarray(elem_subdomain, dtype=np.int64)
        self.n_sub = int(n_sub)
        self.n_nodes = (ne + 1) ** dim
        self.Kref, self.Mref = q1_element_matrices(dim, self.h)
        self.enodes = element_nodes(dim, ne)
        self.dir = dirichlet_mask(dim, ne)
        self.free = np.flatnonzero(~self.dir)               # free -> node
        self.node2free = -np.ones(self.n_nodes, dtype=np.int64)
        self.node2free[self.free] = np.arange(self.free.size)
        self.n_free = self.free.size
        self._assemble_global()
        self._subdomains()
        self._globs(constraints, all_primal)
        self._local_setup(constraint_scale)
        self._coarse_setup()

    # -- global operators --------------------------------------------------
    def _assemble_global(self):
        nloc = self.enodes.shape[1]
        rows = np.repeat(self.enodes, nloc, axis=1).reshape(-1)
        cols = np.tile(self.enodes, (1, nloc)).reshape(-1)
        kv = (self.sigma[:, None] * self.Kref.reshape(1, -1)).reshape(-1)
        mv = np.broadcast_to(self.Mref.reshape(1, -1), (self.enodes.shape[0], nloc * nloc)).reshape(-1)
        n = self.n_nodes
        A_full = sp.csr_matrix((kv, (rows, cols)), shape=(n, n))
        self.M_full = sp.csr_matrix((mv, (rows, cols)), shape=(n, n))
        self.A = A_full[self.free][:, self.free].tocsr()      # free x free

    def rhs(self, f_nodal: np.ndarray) -> np.ndarray:
        """b = (M f)[free], returned as an n_nodes vector (0 on Dirichlet)."""
        f = np.asarray(f_nodal, dtype=np.float64)
        out = np.zeros_like(f)
        out[self.free] = (self.M_full @ f)[self.free]
        return out

    def matvec_nodes(self, x_nodes: np.ndarray) -> np.ndarray:
        out = np.zeros_like(x_nodes)
        out[self.free] = self.A @ x_nodes[self.free]
        return out

    # -- subdomains, multiplicity, interior / interface --------------------
    def _subdomains(self):
        ne_tot = self.enodes.shape[0]
        nloc = self.enodes.shape[1]
        inc = sp.csr_matrix(
            (np.ones(ne_tot * nloc, dtype=np.int64),
             (np.repeat(self.part, nloc), self.enodes.reshape(-1))),
            shape=(self.n_sub, self.n_nodes))
        inc.sum_duplicates()
        inc = inc[:, self.free].tocsr()                     # sub x free
        inc.data[:] = 1
        self.kappa = np.asarray(inc.sum(axis=0)).reshape(-1).astype(np.int64)
        self.R = [np.sort(inc.indices[inc.indptr[i]:inc.indptr[i + 1]])
                  for i in range(self.n_sub)]                # free indices
        self.W = [1.0 / self.kappa[Ri] for Ri in self.R]
        self.interior = [np.flatnonzero(self.kappa[Ri] == 1) for Ri in self.R]   # local
        self.inc_T = inc.T.tocsr()                           # free x sub
        # element lists per subdomain
        order = np.argsort(self.part, kind="stable")
        bounds = np.searchsorted(self.part[order], np.arange(self.n_sub + 1))
        self.elems = [order[bounds[i]:bounds[i + 1]] for i in range(self.n_sub)]

    def _globs(self, mask, all_primal):
        iface = np.flatnonzero(self.kappa >= 2)
        sets = {}
        set_id = -np.ones(self.n_free, dtype=np.int64)
        for j in iface:
            s = tuple(self.inc_T.indices[self.inc_T.indptr[j]:self.inc_T.indptr[j + 1]].tolist())
            set_id[j] = sets.setdefault(s, len(sets))
        set_list = [None] * len(sets)
        for s, k in sets.items():
            set_list[k] = s
        if all_primal:
            comp = np.arange(self.n_free)
            n_comp = self.n_free
        else:
            # mesh edges between interface nodes with the same sharing set
            n1 = self.ne + 1
            strides = [1, n1] + ([n1 * n1] if self.dim == 3 else [])
            node = self.free
            coords = [node % n1, (node // n1) % n1] + ([node // (n1 * n1)] if self.dim == 3 else [])
            ra, rb = [], []
            for d, st in enumerate(strides):
                ok = coords[d] < self.ne
                a = np.flatnonzero(ok)
                nb = self.node2free[node[a] + st]
                good = nb >= 0
                a, nb = a[good], nb[good]
                same = (set_id[a] >= 0) & (set_id[a] == set_id[nb])
                ra.append(a[same])
                rb.append(nb[same])
            ra = np.concatenate(ra)
            rb = np.concatenate(rb)
            g = sp.coo_matrix((np.ones(ra.size), (ra, rb)), shape=(self.n_free, self.n_free))
            n_comp, comp = sp.csgraph.connected_components(g, directed=False)
        globs = {}
        for j in iface:
            globs.setdefault(comp[j], []).append(j)
        out = []
        for nodes in globs.values():
            nodes = np.array(sorted(nodes), dtype=np.int64)
            subs = set_list[set_id[nodes[0]]]
            if nodes.size == 1:
                kind = CORNER
            elif self.dim == 3 and len(subs) == 2:
                kind = FACE
            else:
                kind = EDGE
            if all_primal or (kind & mask):
                out.append(Glob(nodes, subs, kind))
        out.sort(key=lambda G: int(G.nodes[0]))
        self.globs = out
        self.n_c = len(out)
        self.Rc = [[] for _ in range(self.n_sub)]
        for gid, G in enumerate(out):
            for s in G.subs:
                self.Rc[s].append(gid)
        self.Rc = [np.array(r, dtype=np.int64) for r in self.Rc]

    # -- local Neumann matrices, constraints, Phi_i, A_ci -----------------
    def local_matrix(self, i: int) -> np.ndarray:
        """Dense A_i: subdomain i's elements only, free local dofs only."""
        Ri = self.R[i]
        loc = -np.ones(self.n_free, dtype=np.int64)
        loc[Ri] = np.arange(Ri.size)
        E = self.elems[i]
        nloc = self.enodes.shape[1]
        fl = self.node2free[self.enodes[E]]                  # [n_e, nloc]
        li = np.where(fl >= 0, loc[np.maximum(fl, 0)], -1)
        rows = np.repeat(li, nloc, axis=1).reshape(-1)       # entry (a, b) -> row a
        cols = np.tile(li, (1, nloc)).reshape(-1)            #               col b
        vals = (self.sigma[E][:, None] * self.Kref.reshape(1, -1)).reshape(-1)
        keep = (rows >= 0) & (cols >= 0)
        n = Ri.size
        Ai = np.bincount(rows[keep] * n + cols[keep], weights=vals[keep],
                         minlength=n * n).reshape(n, n)
        return Ai

    def constraint_matrix(self, i: int, scale=None) -> np.ndarray:
        Ri = self.R[i]
        loc = -np.ones(self.n_free, dtype=np.int64)
        loc[Ri] = np.arange(Ri.size)
        C = np.zeros((self.Rc[i].size, Ri.size))
        for row, gid in enumerate(self.Rc[i]):
            G = self.globs[gid]
            s = 1.0 if scale is None else scale(int(gid))
            if G.kind == CORNER:
                C[row, loc[G.nodes[0]]] = s
            else:
                C[row, loc[G.nodes]] = s / G.nodes.size
        return C

    def _local_setup(self, scale):
        self.Ai, self.Ci, self.kkt, self.Phi, self.Lam, self.Aci, self.AII = [], [], [], [], [], [], []
        for i in range(self.n_sub):
            Ai = self.local_matrix(i)
            Ci = self.constraint_matrix(i, scale)
            ni, nc = Ai.shape[0], Ci.shape[0]
            K = np.zeros((ni + nc, ni + nc))
            K[:ni, :ni] = Ai
            K[:ni, ni:] = Ci.T
            K[ni:, :ni] = Ci
            lu = sla.lu_factor(K) if ni + nc > 0 else None
            # Eq. saddlepoint: [A_i C_i^T; C_i 0][Phi_i; Lambda_i] = [0; I]
            rhs = np.zeros((ni + nc, nc))
            rhs[ni:, :] = np.eye(nc)
            sol = sla.lu_solve(lu, rhs) if nc > 0 else np.zeros((ni + nc, 0))
            Phi, Lam = sol[:ni], sol[ni:]
            self.Ai.append(Ai)
            self.Ci.append(Ci)
            self.kkt.append(lu)
            self.Phi.append(Phi)
            self.Lam.append(Lam)
            self.Aci.append(Phi.T @ Ai @ Phi)
            I = self.interior[i]
            self.AII.append(sla.cho_factor(Ai[np.ix_(I, I)]) if I.size else None)

    def _coarse_setup(self):
        rows, cols, vals = [], [], []
        for i in range(self.n_sub):
            Rc = self.Rc[i]
            rows.append(np.repeat(Rc, Rc.size))
            cols.append(np.tile(Rc, Rc.size))
            vals.append(self.Aci[i].reshape(-1))
        if self.n_c:
            self.Ac = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                    shape=(self.n_c, self.n_c))
            self.Ac_lu = spla.splu(self.Ac)
        else:
            self.Ac = sp.csc_matrix((0, 0))
            self.Ac_lu = None

    # -- the preconditioner (free-dof vectors) ----------------------------
    def coarse_residual(self, r: np.ndarray) -> np.ndarray:
        """r_c = sum_i R_ci^T Phi_i^T W_i R_i r."""
        rc = np.zeros(self.n_c)
        for i in range(self.n_sub):
            rc[self.Rc[i]] += self.Phi[i].T @ (self.W[i] * r[self.R[i]])
        return rc

    def coarse_solve(self, rc: np.ndarray) -> np.ndarray:
        """u_c = A_c^-1 r_c: a sparse direct solve, or, after set_coarse_cg,
        the inexact solve by plain CG."""
        cg = getattr(self, "coarse_cg", None)
        if cg is not None and self.n_c:
            return self.coarse_solve_cg(rc, *cg)[0]
        return self.Ac_lu.solve(rc) if self.n_c else rc.copy()

    def set_coarse_cg(self, rtol, maxit=10000):
        """Solve the coarse system of Eq. coarsegrid inexactly by plain CG
        (Sec. 3, implementation paragraph: the coarse system is solved with a
        plain CG solver) to ||r_k|| <= rtol ||r_c||; None restores the direct
        solve."""
        self.coarse_cg = None if rtol is None else (float(rtol), int(maxit))

    def coarse_solve_cg(self, rc: np.ndarray, rtol: float, maxit: int = 10000):
        """Plain (unpreconditioned) conjugate gradients on A_c u = r_c from
        u_0 = 0: alpha_k = rho_k / p_k^T A_c p_k, u += alpha p, r -= alpha A_c p,
        beta_k = rho_k+1 / rho_k, p = r + beta p, with rho = r^T r; stops
        before an iteration when ||r_k||_2 <= rtol ||r_c||_2 (or after maxit).
        Returns u, the iteration count and the residual norms ||r_k||."""
        A = self.Ac
        u = np.zeros_like(rc)
        r = np.array(rc, dtype=np.float64)
        p = r.copy()
        rho = float(r @ r)
        tol = rtol * math.sqrt(rho)
        norms = [math.sqrt(rho)]
        it = 0
        while it < maxit and math.sqrt(rho) > tol:
            q = A @ p
            alpha = rho / float(p @ q)
            u = u + alpha * p
            r = r - alpha * q
            rho_new = float(r @ r)
            p = r + (rho_new / rho) * p
            rho = rho_new
            it += 1
            norms.append(math.sqrt(rho))
        return u, it, norms

    def local_solve(self, i: int, yi: np.ndarray):
        """Eq. compzi: [A_i C_i^T; C_i 0][z_i; lambda_i] = [y_i; 0]."""
        ni = yi.size
        rhs = np.concatenate([yi, np.zeros(self.Rc[i].size)])
        sol = sla.lu_solve(self.kkt[i], rhs) if rhs.size else rhs
        return sol[:ni], sol[ni:]

    def interior_correction(self, r1: np.ndarray) -> np.ndarray:
        """Eq. inner: sum_i R_i^T R_Ii^T (R_Ii A_i R_Ii^T)^-1 R_Ii R_i r1."""
        v3 = np.zeros(self.n_free)
        for i in range(self.n_sub):
            I = self.interior[i]
            if I.size:
                gi = self.R[i][I]
                v3[gi] += sla.cho_solve(self.AII[i], r1[gi])
        return v3

    def apply_parts(self, r: np.ndarray) -> dict:
        """All pieces of M^-1 r for one free-dof vector r (Sec. 2)."""
        rc = self.coarse_residual(r)
        uc = self.coarse_solve(rc)
        v1 = np.zeros(self.n_free)
        v2 = np.zeros(self.n_free)
        for i in range(self.n_sub):
            Ri, Wi = self.R[i], self.W[i]
            v1[Ri] += Wi * (self.Phi[i] @ uc[self.Rc[i]])          # Eq. coarsegrid
            zi, _ = self.local_solve(i, Wi * r[Ri])                  # Eq. compzi
            v2[Ri] += Wi * zi                                        # Eq. localsubdomain
        r1 = r - self.A @ (v1 + v2)
        v3 = self.interior_correction(r1)                            # Eq. inner
        return dict(rc=rc, uc=uc, v1=v1, v2=v2, r1=r1, v3=v3, z=v1 + v2 + v3)

    def apply(self, r: np.ndarray) -> np.ndarray:
        return self.apply_parts(r)["z"]

    # -- n_nodes-vector wrappers ------------------------------------------
    def to_free(self, x_nodes):
        return np.asarray(x_nodes, dtype=np.float64)[self.free]

    def to_nodes(self, x_free):
        out = np.zeros((self.n_nodes,) + np.shape(x_free)[1:])
        out[self.free] = x_free
        return out

    def apply_nodes(self, r_nodes: np.ndarray) -> np.ndarray:
        """M^-1 r on [n_nodes] or [n_nodes, nrhs] vectors (Dirichlet -> 0)."""
        r_nodes = np.asarray(r_nodes, dtype=np.float64)
        if r_nodes.ndim == 1:
            return self.to_nodes(self.apply(self.to_free(r_nodes)))
        cols = [self.apply(self.to_free(r_nodes[:, k])) for k in range(r_nodes.shape[1])]
        return self.to_nodes(np.stack(cols, axis=1))

    # -- PCG ----------------------------------------------------------------
    def pcg(self, b_nodes, rtol=1e-8, maxit=500, flexible=False, precond=True):
        """PCG per column from x0 = P_I b (the interior correction of b).

        Standard PCG: beta = (r_k+1, z_k+1) / (r_k, z_k). Flexible PCG:
        beta = (r_k+1, z_k+1 - z_k) / (r_k, z_k). Stops when ||r||_2 <=
        rtol ||b||_2 on the updated residual. Returns x (n_nodes[, nrhs])
        and a list of per-column histories with alpha, beta, rnorm.
        """
        b_nodes = np.asarray(b_nodes, dtype=np.float64)
        single = b_nodes.ndim == 1
        B = b_nodes[:, None] if single else b_nodes
        X = np.zeros_like(B)
        hist = []
        for k in range(B.shape[1]):
            x, h = self._pcg1(self.to_free(B[:, k]), rtol, maxit, flexible, precond)
            X[:, k] = self.to_nodes(x)
            hist.append(h)
        return (X[:, 0] if single else X), hist

    def _pcg1(self, b, rtol, maxit, flexible, precond):
        M = self.apply if precond else (lambda v: v.copy())
        bnorm = float(np.linalg.norm(b))
        x = self.interior_correction(b) if precond else np.zeros_like(b)
        r = b - self.A @ x
        h = dict(alpha=[], beta=[], rnorm=[float(np.linalg.norm(r))], x0=x.copy(),
                 iters=0, converged=False)
        if h["rnorm"][0] <= rtol * bnorm:
            h["converged"] = True
            return x, h
        z = M(r)
        rho = float(r @ z)
        p = z.copy()
        for it in range(1, maxit + 1):
            q = self.A @ p
            alpha = rho / float(p @ q)
            x = x + alpha * p
            r = r - alpha * q
            rn = float(np.linalg.norm(r))
            h["alpha"].append(alpha)
            h["rnorm"].append(rn)
            h["iters"] = it
            if rn <= rtol * bnorm:
                h["converged"] = True
                break
            z_new = M(r)
            rho_new = float(r @ z_new)
            beta = (float(r @ (z_new - z)) if flexible else rho_new) / rho
            h["beta"].append(beta)
            p = z_new + beta * p
            z, rho = z_new, rho_new
        return x, h
