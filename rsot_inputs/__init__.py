"""Seeded synthetic inputs for the semi-discrete entropic OT dual (RSOT).

This module builds the *inputs* of the dual evaluation and nothing else: a
structured simplex mesh of the unit square / unit cube, a quadrature rule on
it, a Gaussian-mixture source density interpolated in P1 and turned into
quadrature masses m_q = w_q * rho_h(x_q) (Sec. 3.1-3.2, Remark 3.1), and
target points y_j with weights nu_j (Sec. 2).  It holds none of the method's
arithmetic (no log-sum-exp, no softmax, no gradient, no truncation), so both
the CPU oracle and the CUDA path consume it.

All randomness uses numpy's PCG64 generator with an explicit seed, which gives
the same numbers on x86_64 and aarch64.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

__all__ = [
    "Problem", "unit_square_tri_mesh", "unit_cube_tet_mesh", "interval_mesh",
    "tri_rule_deg2", "tet_rule_deg2", "gauss_legendre_interval",
    "quadrature", "Mixture", "random_mixture", "mixture_density",
    "sample_mixture", "source_measure", "make_problem",
    "small_2d", "cube_3d", "batch_problem", "warmstart_problem",
    "mixture_from_params16", "uniform_targets", "random_nu",
]


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------

def interval_mesh(n: int):
    """[0,1] split into n equal segments: (vertices (n+1,1), cells (n,2))."""
    v = np.linspace(0.0, 1.0, n + 1).reshape(-1, 1)
    c = np.stack([np.arange(n), np.arange(1, n + 1)], axis=1)
    return v, c


def unit_square_tri_mesh(n: int):
    """Unit square, n x n squares, each cut along its (0,0)-(1,1) diagonal.

    Returns vertices (V,2) float64 and triangles (2 n^2, 3) int64.
    """
    g = np.linspace(0.0, 1.0, n + 1)
    X, Y = np.meshgrid(g, g, indexing="ij")
    verts = np.stack([X.ravel(), Y.ravel()], axis=1)

    def vid(i, j):
        return i * (n + 1) + j

    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    i = i.ravel()
    j = j.ravel()
    v00, v10, v01, v11 = vid(i, j), vid(i + 1, j), vid(i, j + 1), vid(i + 1, j + 1)
    t1 = np.stack([v00, v10, v11], axis=1)
    t2 = np.stack([v00, v11, v01], axis=1)
    cells = np.empty((2 * n * n, 3), dtype=np.int64)
    cells[0::2] = t1
    cells[1::2] = t2
    return verts, cells


def unit_cube_tet_mesh(n: int):
    """Unit cube, n^3 hexes, each split into the 6 Kuhn (Freudenthal)
    tetrahedra that share the hex's main diagonal (0,0,0)-(1,1,1).

    Returns vertices (V,3) float64 and tetrahedra (6 n^3, 4) int64.
    """
    g = np.linspace(0.0, 1.0, n + 1)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    verts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    m = n + 1

    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    base = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
    unit = np.eye(3, dtype=np.int64)
    tets = []
    for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        p0 = base
        p1 = p0 + unit[perm[0]]
        p2 = p1 + unit[perm[1]]
        p3 = p2 + unit[perm[2]]
        ids = [p[:, 0] * m * m + p[:, 1] * m + p[:, 2] for p in (p0, p1, p2, p3)]
        tets.append(np.stack(ids, axis=1))
    cells = np.stack(tets, axis=1).reshape(-1, 4)
    return verts, cells


# --------------------------------------------------------------------------
# quadrature rules (reference simplex, barycentric coordinates, weights
# summing to 1 so that a rule's weights scale by the cell measure)
# --------------------------------------------------------------------------

def tri_rule_deg2():
    """3-point triangle rule exact for polynomials of degree <= 2:
    barycentric (2/3, 1/6, 1/6) and its permutations, equal weights."""
    a, b = 2.0 / 3.0, 1.0 / 6.0
    bary = np.array([[a, b, b], [b, a, b], [b, b, a]])
    return bary, np.full(3, 1.0 / 3.0)


def tet_rule_deg2():
    """4-point tetrahedron rule exact for polynomials of degree <= 2:
    barycentric (a, b, b, b) and permutations with a = (5 + 3 sqrt5)/20,
    b = (5 - sqrt5)/20, equal weights."""
    s5 = math.sqrt(5.0)
    a, b = (5.0 + 3.0 * s5) / 20.0, (5.0 - s5) / 20.0
    bary = np.full((4, 4), b)
    np.fill_diagonal(bary, a)
    return bary, np.full(4, 0.25)


def gauss_legendre_interval(npts: int):
    """Gauss-Legendre rule on a segment, as barycentric pairs + weights."""
    t, w = np.polynomial.legendre.leggauss(npts)
    s = 0.5 * (t + 1.0)
    return np.stack([1.0 - s, s], axis=1), 0.5 * w


def _cell_measure(verts, cells):
    d = verts.shape[1]
    P = verts[cells]                      # (C, d+1, d)
    E = P[:, 1:, :] - P[:, :1, :]         # (C, d, d)
    det = np.linalg.det(E) if d > 1 else E[:, 0, 0]
    return np.abs(det) / math.factorial(d)


def quadrature(verts, cells, rule):
    """Quadrature points x_q, weights w_q (cell measure x rule weight), and the
    per-point (cell id, barycentric coords) used for P1 interpolation."""
    bary, rw = rule
    vol = _cell_measure(verts, cells)                     # (C,)
    P = verts[cells]                                      # (C, d+1, d)
    x = np.einsum("qa,cad->cqd", bary, P).reshape(-1, verts.shape[1])
    w = (vol[:, None] * rw[None, :]).reshape(-1)
    cell_id = np.repeat(np.arange(cells.shape[0]), bary.shape[0])
    lam = np.tile(bary, (cells.shape[0], 1))
    return x, w, cell_id, lam


# --------------------------------------------------------------------------
# densities and target samplers
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Mixture:
    means: np.ndarray      # (K, d)
    sigmas: np.ndarray     # (K,)
    weights: np.ndarray    # (K,) summing to 1


def random_mixture(d: int, k: int, seed: int, sigma=(0.1, 0.2), mean=(0.15, 0.85)) -> Mixture:
    """Equal-weight isotropic Gaussian mixture with seeded means and widths."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(mean[0], mean[1], size=(k, d))
    sig = rng.uniform(sigma[0], sigma[1], size=k)
    return Mixture(means, sig, np.full(k, 1.0 / k))


def mixture_from_params16(theta: np.ndarray) -> Mixture:
    """A 2-D 4-component mixture from a 16-vector
    (mu_x, mu_y, log sigma, weight logit) per component."""
    th = np.asarray(theta, dtype=np.float64).reshape(4, 4)
    w = np.exp(th[:, 3] - th[:, 3].max())
    return Mixture(th[:, :2].copy(), np.exp(th[:, 2]), w / w.sum())


def mixture_density(mix: Mixture, pts: np.ndarray) -> np.ndarray:
    d = pts.shape[1]
    out = np.zeros(pts.shape[0])
    for mu, s, w in zip(mix.means, mix.sigmas, mix.weights):
        r2 = np.sum((pts - mu) ** 2, axis=1)
        out += w * np.exp(-0.5 * r2 / s ** 2) / ((2.0 * math.pi) ** (d / 2) * s ** d)
    return out


def sample_mixture(mix: Mixture, n: int, seed: int) -> np.ndarray:
    """n points of the mixture restricted to [0,1]^d (rejection sampling)."""
    rng = np.random.default_rng(seed)
    d = mix.means.shape[1]
    out = np.empty((0, d))
    while out.shape[0] < n:
        m = 2 * (n - out.shape[0]) + 16
        comp = rng.choice(len(mix.weights), size=m, p=mix.weights)
        pts = mix.means[comp] + mix.sigmas[comp, None] * rng.standard_normal((m, d))
        ok = np.all((pts >= 0.0) & (pts <= 1.0), axis=1)
        out = np.concatenate([out, pts[ok]], axis=0)
    return np.ascontiguousarray(out[:n])


def uniform_targets(n: int, d: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=(n, d))


def random_nu(n: int, seed: Optional[int], lo=0.5, hi=1.5) -> np.ndarray:
    """nu_j proportional to U(lo, hi), normalised; seed None gives 1/n."""
    if seed is None:
        return np.full(n, 1.0 / n)
    v = np.random.default_rng(seed).uniform(lo, hi, size=n)
    return v / v.sum()


def source_measure(verts, cells, rule, density_at_vertices: np.ndarray, normalize=True):
    """Discrete source measure sum_q m_q delta_{x_q} with m_q = w_q rho_h(x_q),
    rho_h the P1 nodal interpolant of the density (Sec. 3.1-3.2)."""
    x, w, cid, lam = quadrature(verts, cells, rule)
    rho_h = np.einsum("qa,qa->q", lam, density_at_vertices[cells[cid]])
    m = w * rho_h
    if normalize:
        m = m / m.sum()
    return np.ascontiguousarray(x), np.ascontiguousarray(m)


# --------------------------------------------------------------------------
# problems
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Problem:
    x: np.ndarray       # (nq, d) quadrature points, float64, C-contiguous
    mass: np.ndarray    # (nq,) m_q, sums to 1
    y: np.ndarray       # (n, d) targets
    nu: np.ndarray      # (n,) target weights, sum to 1
    eps: float
    name: str = ""

    @property
    def d(self):
        return self.x.shape[1]

    @property
    def nq(self):
        return self.x.shape[0]

    @property
    def n(self):
        return self.y.shape[0]


def make_problem(d, mesh_n, n_targets, eps, src_seed, src_k, tgt_seed,
                 tgt_k=None, nu_seed=None, name="") -> Problem:
    """Mesh + degree-2 rule + mixture density -> (x_q, m_q); targets uniform
    (tgt_k None) or drawn from a tgt_k-component mixture; nu uniform or random."""
    if d == 2:
        verts, cells = unit_square_tri_mesh(mesh_n)
        rule = tri_rule_deg2()
    elif d == 3:
        verts, cells = unit_cube_tet_mesh(mesh_n)
        rule = tet_rule_deg2()
    else:
        raise ValueError("d must be 2 or 3")
    mix = random_mixture(d, src_k, src_seed)
    x, m = source_measure(verts, cells, rule, mixture_density(mix, verts))
    if tgt_k is None:
        y = uniform_targets(n_targets, d, tgt_seed)
    else:
        y = sample_mixture(random_mixture(d, tgt_k, tgt_seed), n_targets, tgt_seed + 7919)
    nu = random_nu(n_targets, nu_seed)
    return Problem(x, m, np.ascontiguousarray(y), nu, float(eps), name)


def small_2d() -> Problem:
    """Unit square, 64x64x2 P1 triangles, 3-point rule (24,576 points),
    3-component mixture (seed 1); 512 uniform targets (seed 2); nu = 1/512;
    eps = 1e-2."""
    return make_problem(2, 64, 512, 1e-2, src_seed=1, src_k=3, tgt_seed=2,
                        name="square-24576x512")


def cube_3d(mesh_n: int = 32, n_targets: int = 65536, eps: float = 1e-3) -> Problem:
    """Unit cube, mesh_n^3 hexes x 6 tets x 4 points (786,432 points at 32),
    5-component mixture (seed 3); targets from a 4-component mixture (seed 4);
    nu ~ U(0.5,1.5) normalised (seed 5)."""
    return make_problem(3, mesh_n, n_targets, eps, src_seed=3, src_k=5, tgt_seed=4,
                        tgt_k=4, nu_seed=5,
                        name=f"cube-{6 * 4 * mesh_n ** 3}x{n_targets}")


def batch_problem(seed: int) -> Problem:
    """One problem of the uneven batch: d alternates 2/3 with the seed; the
    point count ~ log-uniform[20k, 500k] realised through the mesh size; the
    target count ~ log-uniform[1k, 32k]; eps ~ log-uniform[1e-3, 1e-1]; the
    density is a mixture drawn from a seeded 16-parameter vector."""
    rng = np.random.default_rng(seed)
    d = 2 if seed % 2 == 0 else 3
    nq_goal = math.exp(rng.uniform(math.log(2e4), math.log(5e5)))
    n = int(round(math.exp(rng.uniform(math.log(1e3), math.log(3.2e4)))))
    eps = math.exp(rng.uniform(math.log(1e-3), math.log(1e-1)))
    if d == 2:
        mesh_n = max(2, int(round(math.sqrt(nq_goal / 6.0))))
        verts, cells = unit_square_tri_mesh(mesh_n)
        rule = tri_rule_deg2()
    else:
        mesh_n = max(2, int(round((nq_goal / 24.0) ** (1.0 / 3.0))))
        verts, cells = unit_cube_tet_mesh(mesh_n)
        rule = tet_rule_deg2()
    theta = params16(rng)
    mix = mixture_from_params16(theta)
    if d == 3:
        mix = Mixture(np.concatenate([mix.means, rng.uniform(0.15, 0.85, (4, 1))], axis=1),
                      mix.sigmas, mix.weights)
    x, m = source_measure(verts, cells, rule, mixture_density(mix, verts))
    y = uniform_targets(n, d, seed + 100000)
    return Problem(x, m, y, random_nu(n, None), float(eps), name=f"batch-{seed}")


def params16(rng) -> np.ndarray:
    """Seeded 16-vector: 4 x (mu_x, mu_y, log sigma, weight logit)."""
    th = np.empty((4, 4))
    th[:, 0:2] = rng.uniform(0.15, 0.85, size=(4, 2))
    th[:, 2] = np.log(rng.uniform(0.1, 0.2, size=4))
    th[:, 3] = rng.normal(0.0, 0.5, size=4)
    return th.reshape(16)


_MESH_CACHE = {}


def _square_quadrature(mesh_n):
    """(vertices, cells, x_q, w_q, cell ids, barycentric) of the square mesh, cached."""
    if mesh_n not in _MESH_CACHE:
        verts, cells = unit_square_tri_mesh(mesh_n)
        _MESH_CACHE[mesh_n] = (verts, cells) + quadrature(verts, cells, tri_rule_deg2())
    return _MESH_CACHE[mesh_n]


def warmstart_problem(seed: int, mesh_n: int = 64, n_targets: int = 4096, eps: float = 5e-3):
    """d = 2, 4,096 uniform targets, eps = 5e-3, density from a seeded
    16-parameter vector.  Returns (problem, theta16)."""
    rng = np.random.default_rng(seed)
    theta = params16(rng)
    verts, cells, xq, wq, cid, lam = _square_quadrature(mesh_n)
    rho_v = mixture_density(mixture_from_params16(theta), verts)
    m = wq * np.einsum("qa,qa->q", lam, rho_v[cells[cid]])
    x, m = xq, m / m.sum()
    y = uniform_targets(n_targets, 2, seed + 100000)
    return Problem(x, m, y, random_nu(n_targets, None), float(eps), f"warm-{seed}"), theta
