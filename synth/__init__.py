"""Seeded synthetic inputs for the BDDC diffusion problems.

This module only draws random numbers and lays out the structured Q1 grid
and the element-to-subdomain map. It holds none of the preconditioner's
arithmetic (no element matrices, no assembly, no solves), so that the CPU
oracle and the CUDA library can both be fed from it without sharing any of
the method.

Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used in counter mode: draw k
of stream `seed` is mix(seed + (k + 1) * golden_gamma). Doubles take the top
53 bits; normals come from the Box-Muller transform, one normal per pair of
uniforms.

Grid conventions (shared by every consumer):
  * dim in {2, 3}; ne elements per direction on the unit square / cube;
    h = 1 / ne.
  * node (ix, iy[, iz]) has id ix + (ne+1) * (iy + (ne+1) * iz).
  * element (ex, ey[, ez]) has id ex + ne * (ey + ne * ez).
  * homogeneous Dirichlet conditions on the whole outer boundary.
"""
from __future__ import annotations

import dataclasses

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Return draws offset .. offset+n-1 of the SplitMix64 stream `seed`."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each draw."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform(seed: int, n: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, n)


def normal(seed: int, n: int) -> np.ndarray:
    """N(0, 1) by Box-Muller on the pairs (u[2k], u[2k+1])."""
    u = uniform01(seed, 2 * n)
    u1 = 1.0 - u[0::2]           # in (0, 1]: log is finite
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


@dataclasses.dataclass
class Problem:
    """A structured Q1 diffusion problem and its element partition."""

    dim: int
    ne: int
    elem_sigma: np.ndarray        # [n_elems] float64 > 0
    elem_subdomain: np.ndarray    # [n_elems] int32 in [0, n_sub)
    n_sub: int
    f: np.ndarray                 # [n_nodes, nrhs] float64 nodal load values
    name: str = ""

    @property
    def n_nodes(self) -> int:
        return (self.ne + 1) ** self.dim

    @property
    def n_elems(self) -> int:
        return self.ne ** self.dim

    @property
    def nrhs(self) -> int:
        return self.f.shape[1]


def box_partition(dim: int, ne: int, nsub_per_dir: int) -> np.ndarray:
    """Element -> subdomain id for an nsub^dim grid of equal boxes."""
    assert ne % nsub_per_dir == 0
    H = ne // nsub_per_dir
    idx = np.arange(ne) // H
    if dim == 2:
        sx, sy = np.meshgrid(idx, idx, indexing="xy")
        part = sx + nsub_per_dir * sy
    else:
        sz, sy, sx = np.meshgrid(idx, idx, idx, indexing="ij")
        part = sx + nsub_per_dir * (sy + nsub_per_dir * sz)
    return part.reshape(-1).astype(np.int32)


def _face_pairs(dim: int, ne: int):
    """(a, b) element pairs sharing a face, one array pair per axis."""
    e = np.arange(ne ** dim).reshape((ne,) * dim)   # axis order (z,) y, x
    out = []
    for ax in range(dim):
        sl_a = [slice(None)] * dim
        sl_b = [slice(None)] * dim
        sl_a[ax] = slice(0, ne - 1)
        sl_b[ax] = slice(1, ne)
        out.append((e[tuple(sl_a)].reshape(-1), e[tuple(sl_b)].reshape(-1)))
    return out


def voronoi_partition(ne: int, n_seeds: int, seed: int):
    """Cell-like partition of a 3D grid: nearest seed by element centroid.

    Seeds are uniform in [0,1]^3. Ties go to the lowest seed index. Empty
    cells are dropped and cells that are not face-connected are split into
    their connected components, each one a subdomain. Returns
    (elem_subdomain, n_sub, elem_cell) where elem_cell is the raw Voronoi
    cell (before the component split).
    """
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    from scipy.spatial import cKDTree

    u = uniform01(seed, 3 * n_seeds).reshape(n_seeds, 3)
    c = (np.arange(ne) + 0.5) / ne
    cz, cy, cx = np.meshgrid(c, c, c, indexing="ij")
    cent = np.stack([cx.reshape(-1), cy.reshape(-1), cz.reshape(-1)], axis=1)
    tree = cKDTree(u)
    _, cell = tree.query(cent, k=1)
    cell = cell.astype(np.int64)
    rows, cols = [], []
    for a, b in _face_pairs(3, ne):
        same = cell[a] == cell[b]
        rows.append(a[same])
        cols.append(b[same])
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    n = ne ** 3
    g = coo_matrix((np.ones(rows.size, dtype=np.int8), (rows, cols)), shape=(n, n))
    n_comp, comp = connected_components(g, directed=False)
    # number components in order of first element appearance (deterministic)
    _, first = np.unique(comp, return_index=True)
    order = np.argsort(first)
    relabel = np.empty(n_comp, dtype=np.int64)
    relabel[order] = np.arange(n_comp)
    sub = relabel[comp].astype(np.int32)
    return sub, int(n_comp), cell


def layer_sigma(ne: int, cell: np.ndarray, inside: float = 1.0, layer: float = 0.1) -> np.ndarray:
    """sigma = `layer` on elements with a face-neighbour in another cell."""
    sigma = np.full(ne ** 3, inside)
    for a, b in _face_pairs(3, ne):
        diff = cell[a] != cell[b]
        sigma[a[diff]] = layer
        sigma[b[diff]] = layer
    return sigma


# Seed streams: sigma = 1000+k, f = 2000+k, sigma perturbation = 3000+k,
# Voronoi seeds = 4000+k, finite-difference element pick = 5000+k.

def make_problem(dim: int, ne: int, nsub: int, sigma: str = "one", nrhs: int = 1,
                 k: int = 0, name: str = "") -> Problem:
    """Structured box partition; sigma 'one' or 'lognormal' (exp(N(0,1)))."""
    n_el = ne ** dim
    if sigma == "one":
        s = np.ones(n_el)
    elif sigma == "lognormal":
        s = np.exp(normal(1000 + k, n_el))
    else:
        raise ValueError(sigma)
    part = box_partition(dim, ne, nsub)
    n_nodes = (ne + 1) ** dim
    f = uniform(2000 + k, n_nodes * nrhs).reshape(n_nodes, nrhs)
    return Problem(dim, ne, s, part, nsub ** dim, f, name or f"{dim}d_{ne}_{nsub}")


def config(k: int, nrhs: int | None = None) -> Problem:
    """The five workload shapes, numbered 1..5.

    1: 2D Laplace, 64^2 elements, 4x4 subdomains, sigma = 1, 1 RHS.
    2: 3D, 96^3 elements, 12^3 subdomains of 8^3, sigma = exp(N(0,1)), 1 RHS.
    3: 3D, 128^3 elements, ~2000 Voronoi cells, sigma 1.0 / 0.1 layers, 64 RHS.
    4: adjoint-gradient workload on config 2's grid (forward problem only here).
    5: 3D, 192^3 elements, 24^3 subdomains, sigma = exp(N(0,1)), 8 RHS.
    """
    if k == 1:
        return make_problem(2, 64, 4, "one", nrhs or 1, k=1, name="cfg1_2d_64_4x4")
    if k == 2:
        return make_problem(3, 96, 12, "lognormal", nrhs or 1, k=2, name="cfg2_3d_96_12cubed")
    if k == 4:
        return make_problem(3, 96, 12, "lognormal", nrhs or 1, k=2, name="cfg4_3d_96_12cubed")
    if k == 5:
        return make_problem(3, 192, 24, "lognormal", nrhs or 8, k=5, name="cfg5_3d_192_24cubed")
    if k == 3:
        ne = 128
        sub, n_sub, cell = voronoi_partition(ne, 2000, 4003)
        s = layer_sigma(ne, cell)
        n_nodes = (ne + 1) ** 3
        r = nrhs or 64
        f = uniform(2003, n_nodes * r).reshape(n_nodes, r)
        return Problem(3, ne, s, sub, n_sub, f, "cfg3_3d_128_voronoi2000")
    raise ValueError(k)
