"""Seeded synthetic inputs shaped like the paper's test meshes.

This module only *draws inputs*: structured-then-jittered simplex meshes, nodal
alpha, element beta, right-hand sides and warm-start perturbations.  It holds
none of the pressure operator's arithmetic, so both the FP64 CPU oracle and the
CUDA path can be fed from it without sharing any of the method.

Mesh families (Section 3.1: a primal mesh of triangles or tetrahedra with the
P1 unknowns on its vertices):
  * 2D: the unit square with n x n cells, each cut into the triangles
    (v00, v10, v11) and (v00, v11, v01).  n = 64 gives 8,192 triangles and
    4,225 vertices, the size of mesh M3 of the Taylor-Green study (Section 5.1,
    Table TGV_mesh).
  * 3D: the unit cube with n^3 hexahedra, each cut into the 6 Kuhn tetrahedra
    (one per permutation of the axes), all stored with positive orientation.

Interior vertices are moved by an independent U(-j h, j h) per coordinate;
boundary vertices stay put so the faces stay planar and x = 0 is exact.

Random draws for a case happen in a fixed order from numpy's PCG64
``default_rng(seed)``: jitter, alpha modes, beta, inclusion, right-hand side,
warm-start perturbation.  A node/element shuffle (to present the mesh with an
arbitrary numbering) uses a separate generator so that it never changes the
other draws.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Case", "square_mesh", "kuhn_cube_mesh", "jitter_nodes", "alpha_c1",
    "alpha_fourier", "make_c1", "make_c2", "make_c3", "make_batch_case",
    "make_served_case", "served_step_drift", "grid_n_for_nodes", "shuffle_case",
    "case_by_name",
]


@dataclass
class Case:
    """One pressure system: mesh, coefficients, right-hand side, first guess.

    coords  [N, d] float64, conn [E, d+1] int32 (0-based), dirichlet [N] uint8
    (1 = the pressure correction is fixed to 0 there), alpha [N] float64 nodal
    (the 1/(gamma-1) mass coefficient of the weak problem, Section 3.4),
    beta [E] float64 per element (the enthalpy H, Section 3.3), dt2 = dt^2,
    b [N] float64 nodal load vector (0 on Dirichlet nodes), x0 [N] first guess.
    """
    name: str
    dim: int
    coords: np.ndarray
    conn: np.ndarray
    dirichlet: np.ndarray
    alpha: np.ndarray
    beta: np.ndarray
    dt2: float
    b: np.ndarray
    x0: np.ndarray
    n: int = 0
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_elems(self) -> int:
        return int(self.conn.shape[0])

    @property
    def n_free(self) -> int:
        return int(self.n_nodes - int(self.dirichlet.sum()))


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------

def square_mesh(n: int):
    """Unit square, n x n cells, two triangles per cell; node id = i + (n+1) j."""
    m = n + 1
    j, i = np.indices((m, m))
    coords = np.stack([i.ravel(), j.ravel()], axis=1).astype(np.float64) / n
    ci, cj = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    v00 = (ci + m * cj).ravel().astype(np.int64)
    v10, v01 = v00 + 1, v00 + m
    v11 = v01 + 1
    t1 = np.stack([v00, v10, v11], axis=1)
    t2 = np.stack([v00, v11, v01], axis=1)
    conn = np.stack([t1, t2], axis=1).reshape(-1, 3).astype(np.int32)
    return coords, conn


_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def _kuhn_templates():
    """Vertex offsets (as unit-cube corners) of the 6 Kuhn tetrahedra, each
    ordered so that its Jacobian determinant is positive."""
    e = np.eye(3, dtype=np.int64)
    temps = []
    for s in _PERMS:
        v = [np.zeros(3, np.int64), e[s[0]], e[s[0]] + e[s[1]], np.ones(3, np.int64)]
        jac = np.stack([v[1] - v[0], v[2] - v[0], v[3] - v[0]], axis=1)
        if np.linalg.det(jac.astype(np.float64)) < 0:
            v[2], v[3] = v[3], v[2]
        temps.append(v)
    return temps


def kuhn_cube_mesh(n: int):
    """Unit cube, n^3 hexahedra, 6 Kuhn tetrahedra per hexahedron;
    node id = i + (n+1) (j + (n+1) k)."""
    m = n + 1
    k, j, i = np.indices((m, m, m))
    coords = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64) / n
    ck, cj, ci = np.indices((n, n, n))
    base = (ci + m * (cj + m * ck)).ravel().astype(np.int64)
    stride = np.array([1, m, m * m], dtype=np.int64)
    conn = np.empty((base.size, 6, 4), dtype=np.int32)
    for t, verts in enumerate(_kuhn_templates()):
        for a, off in enumerate(verts):
            conn[:, t, a] = base + int(off @ stride)
    return coords, conn.reshape(-1, 4)


def jitter_nodes(coords: np.ndarray, n: int, frac: float, rng) -> np.ndarray:
    """Move every strictly interior node by U(-frac h, frac h) per coordinate."""
    h = 1.0 / n
    d = rng.uniform(-frac * h, frac * h, size=coords.shape)
    eps = 0.25 * h
    interior = np.all((coords > eps) & (coords < 1.0 - eps), axis=1)
    out = coords.copy()
    out[interior] += d[interior]
    return out


def grid_n_for_nodes(target: float, dim: int) -> int:
    """Cells per side n >= 1 whose (n+1)^dim node count is nearest to target."""
    base = max(1, int(math.floor(target ** (1.0 / dim))) - 1)
    best = None
    for n in range(max(1, base - 1), base + 3):
        err = abs((n + 1) ** dim - target)
        if best is None or err < best[0]:
            best = (err, n)
    return best[1]


# --------------------------------------------------------------------------
# coefficients
# --------------------------------------------------------------------------

def alpha_c1(coords: np.ndarray) -> np.ndarray:
    """alpha = 1 + 0.5 sin(2 pi x) cos(2 pi y) [cos(2 pi z) in 3D]."""
    x = coords[:, 0]
    y = coords[:, 1]
    a = np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    if coords.shape[1] == 3:
        a = a * np.cos(2 * np.pi * coords[:, 2])
    return 1.0 + 0.5 * a


def alpha_fourier(coords: np.ndarray, rng, n_modes: int = 8) -> np.ndarray:
    """alpha = 2^s in [0.5, 2], s = sum_m a_m cos(2 pi k_m.x + phi_m) / sum|a_m|,
    k_m integer vectors in [-4, 4]^d without 0, a_m ~ U(-1,1), phi_m ~ U(0, 2 pi)."""
    d = coords.shape[1]
    k = rng.integers(-4, 5, size=(n_modes, d))
    for m in range(n_modes):
        while not k[m].any():
            k[m] = rng.integers(-4, 5, size=d)
    a = rng.uniform(-1.0, 1.0, size=n_modes)
    phi = rng.uniform(0.0, 2 * np.pi, size=n_modes)
    s = np.zeros(coords.shape[0])
    for m in range(n_modes):
        s += a[m] * np.cos(2 * np.pi * (coords @ k[m].astype(np.float64)) + phi[m])
    s /= np.abs(a).sum()
    return np.power(2.0, s)


def _centroids(coords: np.ndarray, conn: np.ndarray, block: int = 1 << 20) -> np.ndarray:
    out = np.empty((conn.shape[0], coords.shape[1]))
    for s in range(0, conn.shape[0], block):
        out[s:s + block] = coords[conn[s:s + block]].mean(axis=1)
    return out


def _dirichlet_x0(coords: np.ndarray) -> np.ndarray:
    return (coords[:, 0] == 0.0).astype(np.uint8)


def _rhs(rng, dirichlet: np.ndarray) -> np.ndarray:
    b = rng.standard_normal(dirichlet.size)
    b[dirichlet.astype(bool)] = 0.0
    return b


# --------------------------------------------------------------------------
# the five workload recipes
# --------------------------------------------------------------------------

def make_c1(n: int = 64, seed: int = 0) -> Case:
    """2D square n x n, jitter 0.2h, alpha = C1 form, beta ~ LN(0, 0.5),
    dt^2 = 1e-3, Dirichlet on x = 0, b ~ N(0,1), x0 = 0."""
    rng = np.random.default_rng(seed)
    coords, conn = square_mesh(n)
    coords = jitter_nodes(coords, n, 0.2, rng)
    alpha = alpha_c1(coords)
    beta = np.exp(0.5 * rng.standard_normal(conn.shape[0]))
    dirichlet = _dirichlet_x0(coords)
    b = _rhs(rng, dirichlet)
    return Case("c1_2d_%d" % n, 2, coords, conn, dirichlet, alpha, beta, 1e-3, b,
                np.zeros(coords.shape[0]), n=n, seed=seed)


def make_c2(n: int = 64, seed: int = 0) -> Case:
    """3D Kuhn cube n^3, jitter 0.15h, alpha Fourier in [0.5, 2],
    beta ~ LN(0, 0.5), dt^2 = 1e-2, Dirichlet x = 0, b ~ N(0,1), x0 = 0."""
    rng = np.random.default_rng(seed)
    coords, conn = kuhn_cube_mesh(n)
    coords = jitter_nodes(coords, n, 0.15, rng)
    alpha = alpha_fourier(coords, rng)
    beta = np.exp(0.5 * rng.standard_normal(conn.shape[0]))
    dirichlet = _dirichlet_x0(coords)
    b = _rhs(rng, dirichlet)
    return Case("c2_3d_%d" % n, 3, coords, conn, dirichlet, alpha, beta, 1e-2, b,
                np.zeros(coords.shape[0]), n=n, seed=seed)


def make_c3(n: int = 160, seed: int = 0) -> Case:
    """Stiff low-Mach 3D case: Kuhn cube n^3, jitter 0.15h, alpha Fourier x 1e-4,
    beta ~ LN(0, 1) with a x100 spherical inclusion (centre U(0.25,0.75)^3,
    radius U(0.15,0.25), element centroid inside), dt^2 = 1e-2, Dirichlet x = 0.

    The exact solution xstar ~ N(0,1) on free nodes is drawn in the RHS slot;
    b is left empty (callers form b = A xstar with whatever operator they
    test), and ``extra['warm_xi']`` holds the N(0,1) warm-start perturbation so
    that x0 = xstar (1 + 0.01 xi)."""
    rng = np.random.default_rng(seed)
    coords, conn = kuhn_cube_mesh(n)
    coords = jitter_nodes(coords, n, 0.15, rng)
    alpha = 1e-4 * alpha_fourier(coords, rng)
    beta = np.exp(1.0 * rng.standard_normal(conn.shape[0]))
    centre = rng.uniform(0.25, 0.75, size=3)
    radius = rng.uniform(0.15, 0.25)
    cen = _centroids(coords, conn)
    inside = np.sum((cen - centre) ** 2, axis=1) < radius * radius
    beta[inside] *= 100.0
    dirichlet = _dirichlet_x0(coords)
    xstar = _rhs(rng, dirichlet)
    warm_xi = rng.standard_normal(coords.shape[0])
    x0 = xstar * (1.0 + 0.01 * warm_xi)
    return Case("c3_3d_%d" % n, 3, coords, conn, dirichlet, alpha, beta, 1e-2,
                np.zeros(coords.shape[0]), x0, n=n, seed=seed,
                extra={"xstar": xstar, "warm_xi": warm_xi,
                       "inclusion": (centre, radius, int(inside.sum()))})


def make_batch_case(i: int, lo: float = 2e3, hi: float = 2e5) -> Case:
    """Mesh i of the 256-mesh batch: seed i, 2D if i is even else 3D, node count
    exp(U(ln lo, ln hi)) rounded to the nearest (n+1)^d grid; alpha in the C1
    form, beta ~ LN(0, 0.5), dt^2 = 1e-3, Dirichlet x = 0, b ~ N(0,1)."""
    rng = np.random.default_rng(i)
    dim = 2 if i % 2 == 0 else 3
    target = math.exp(rng.uniform(math.log(lo), math.log(hi)))
    n = grid_n_for_nodes(target, dim)
    if dim == 2:
        coords, conn = square_mesh(n)
        coords = jitter_nodes(coords, n, 0.2, rng)
    else:
        coords, conn = kuhn_cube_mesh(n)
        coords = jitter_nodes(coords, n, 0.15, rng)
    alpha = alpha_c1(coords)
    beta = np.exp(0.5 * rng.standard_normal(conn.shape[0]))
    dirichlet = _dirichlet_x0(coords)
    b = _rhs(rng, dirichlet)
    return Case("batch_%03d_%dd_%d" % (i, dim, n), dim, coords, conn, dirichlet, alpha,
                beta, 1e-3, b, np.zeros(coords.shape[0]), n=n, seed=i)


def make_served_case(c: int, lo: float = 5e3, hi: float = 2e6,
                     median: float = 1e5, sigma_ln: float = 1.2) -> Case:
    """Case c of the served stream: seed 1000 + c, 3D Kuhn cube whose node count
    is lognormal (median 1e5, sigma_ln 1.2) clipped to [lo, hi]; alpha Fourier,
    beta ~ LN(0, 0.5), dt^2 = 1e-2, Dirichlet x = 0, b ~ N(0,1), x0 = 0.
    ``extra['rng']`` continues the case's stream for the per-step drift."""
    rng = np.random.default_rng(1000 + c)
    target = float(np.clip(math.exp(math.log(median) + sigma_ln * rng.standard_normal()), lo, hi))
    n = grid_n_for_nodes(target, 3)
    coords, conn = kuhn_cube_mesh(n)
    coords = jitter_nodes(coords, n, 0.15, rng)
    alpha = alpha_fourier(coords, rng)
    beta = np.exp(0.5 * rng.standard_normal(conn.shape[0]))
    dirichlet = _dirichlet_x0(coords)
    b = _rhs(rng, dirichlet)
    return Case("served_%02d_3d_%d" % (c, n), 3, coords, conn, dirichlet, alpha, beta, 1e-2,
                b, np.zeros(coords.shape[0]), n=n, seed=1000 + c, extra={"rng": rng})


def served_step_drift(case: Case, beta: np.ndarray, b: np.ndarray):
    """One time step of drift: beta <- beta exp(0.01 xi_e), b <- b + 0.01 xi
    (0 kept on Dirichlet nodes).  Returns new (beta, b)."""
    rng = case.extra["rng"]
    beta = beta * np.exp(0.01 * rng.standard_normal(beta.size))
    b = b + 0.01 * rng.standard_normal(b.size)
    b[case.dirichlet.astype(bool)] = 0.0
    return beta, b


def shuffle_case(case: Case, seed: int = 12345) -> Case:
    """Same system under a random node numbering and element order (and a
    random vertex rotation inside each element that keeps its orientation
    sign irrelevant to the operator)."""
    rng = np.random.default_rng(seed)
    N, E = case.n_nodes, case.n_elems
    p = rng.permutation(N)            # new id of old node i is p[i]
    inv = np.empty_like(p)
    inv[p] = np.arange(N)
    q = rng.permutation(E)
    conn = p[case.conn[q]].astype(np.int32)
    c = Case(case.name + "_shuf", case.dim, case.coords[inv], conn, case.dirichlet[inv],
             case.alpha[inv], case.beta[q], case.dt2, case.b[inv], case.x0[inv],
             n=case.n, seed=case.seed, extra=dict(case.extra))
    c.extra["node_new_of_old"] = p
    c.extra["elem_old_of_new"] = q
    return c


def case_by_name(name: str, n: int | None = None) -> Case:
    if name == "c1":
        return make_c1(64 if n is None else n)
    if name == "c2":
        return make_c2(64 if n is None else n)
    if name == "c3":
        return make_c3(160 if n is None else n)
    raise ValueError(name)


def make_projection_case(dim: int = 3, n: int = 64, seed: int = 0, gamma: float = 1.4) -> Case:
    """One time step's projection stage on a jittered unit square / Kuhn cube
    (Dirichlet x = 0): ideal gas, alpha = 1/(gamma - 1) at every node, and
    seeded smooth primal-element fields in ``extra``:
      rho  [E]     1 + 0.2 s1(centroid) with s a unit-amplitude product of sines,
      wu   [E, d]  a divergence-free vortex (Taylor-Green-like) of amplitude 1
                   plus 5 % N(0,1) noise,
      pn   [N]     1 + 0.05 s2(node) + 0.01 N(0,1),
      we   [E]     mean(pn)/(gamma - 1) + |wu|^2/(2 rho) + 0.01 N(0,1),
      gamma, dt    dt = 0.5 h / max |wu| (a flow-speed CFL, Section 3).
    beta is a placeholder (the step sets it to the enthalpy); dt2 = dt^2."""
    rng = np.random.default_rng(7000 + seed)
    if dim == 2:
        coords, conn = square_mesh(n)
        coords = jitter_nodes(coords, n, 0.2, rng)
    else:
        coords, conn = kuhn_cube_mesh(n)
        coords = jitter_nodes(coords, n, 0.15, rng)
    N, E = coords.shape[0], conn.shape[0]
    cen = coords[conn].mean(axis=1)
    two_pi = 2.0 * np.pi
    ph = rng.uniform(0.0, two_pi, size=(2, dim))
    s1 = np.prod(np.sin(two_pi * cen + ph[0]), axis=1)
    rho = 1.0 + 0.2 * s1
    wu = np.zeros((E, dim))
    x, y = cen[:, 0], cen[:, 1]
    if dim == 2:
        wu[:, 0] = np.sin(np.pi * x) * np.cos(np.pi * y)
        wu[:, 1] = -np.cos(np.pi * x) * np.sin(np.pi * y)
    else:
        z = cen[:, 2]
        wu[:, 0] = np.sin(np.pi * x) * np.cos(np.pi * y) * np.cos(np.pi * z)
        wu[:, 1] = -np.cos(np.pi * x) * np.sin(np.pi * y) * np.cos(np.pi * z)
    wu += 0.05 * rng.standard_normal((E, dim))
    s2 = np.prod(np.cos(two_pi * coords + ph[1]), axis=1)
    pn = 1.0 + 0.05 * s2 + 0.01 * rng.standard_normal(N)
    rhok = 0.5 * (wu * wu).sum(axis=1) / rho
    we = pn[conn].mean(axis=1) / (gamma - 1.0) + rhok + 0.01 * rng.standard_normal(E)
    dt = 0.5 / n / float(np.abs(wu).max())
    dirichlet = _dirichlet_x0(coords)
    alpha = np.full(N, 1.0 / (gamma - 1.0))
    return Case("projection_%dd_%d" % (dim, n), dim, coords, conn, dirichlet, alpha, np.ones(E), dt * dt,
                np.zeros(N), np.zeros(N), n=n, seed=seed,
                extra={"rho": rho, "wu": wu, "we": we, "pn": pn, "gamma": gamma, "dt": dt})


def make_eos_case(dim: int = 3, n: int = 64, seed: int = 0, eos_a: float = 2.5, eos_b: float = 0.5) -> Case:
    """The projection-stage fields of make_projection_case for a gas whose
    internal energy density is rho e = eos_a P + eos_b P^2 / rho (a thermally
    perfect gas with c_v linear in the temperature; eos_b = 0 is the ideal
    gas of make_projection_case with eos_a = 1/(gamma - 1)):
      we [E]  eos_a Pbar + eos_b Pbar^2 / rho + |wu|^2 / (2 rho) + 0.01 N(0,1),
    Pbar the vertex mean of pn; ``extra`` gains eos_a and eos_b, and alpha is
    eos_a at every node (a placeholder: the Newton iteration sets it)."""
    case = make_projection_case(dim, n, seed=seed, gamma=1.0 + 1.0 / eos_a)
    e = case.extra
    rng = np.random.default_rng(9100 + seed)
    pbar = e["pn"][case.conn].mean(axis=1)
    rhok = 0.5 * (e["wu"] * e["wu"]).sum(axis=1) / e["rho"]
    we = eos_a * pbar + eos_b * pbar * pbar / e["rho"] + rhok + 0.01 * rng.standard_normal(case.n_elems)
    extra = dict(e, we=we, eos_a=float(eos_a), eos_b=float(eos_b))
    return Case("eos_%dd_%d" % (dim, n), dim, case.coords, case.conn, case.dirichlet,
                np.full(case.n_nodes, float(eos_a)), case.beta, case.dt2, case.b, case.x0, n=n, seed=seed,
                extra=extra)


def periodic_master(coords: np.ndarray, axes) -> np.ndarray:
    """master[i] for a unit square / cube periodic along `axes`: a node with
    coordinate 1 on a periodic axis is merged into the node at 0 there (all
    periodic axes folded at once); every other node is its own master.
    Boundary nodes are never jittered, so matching nodes have equal folded
    coordinates."""
    folded = coords.copy()
    for a in axes:
        folded[folded[:, a] == 1.0, a] = 0.0
    index = {tuple(x): i for i, x in enumerate(coords)}
    return np.array([index[tuple(x)] for x in folded], dtype=np.int32)


def make_periodic_case(dim: int = 3, n: int = 16, seed: int = 0) -> Case:
    """The C1 (2D) or C2 (3D) set-up made periodic in y (and z): Dirichlet on
    x = 0, Neumann on x = 1, vertices on y = 1 (z = 1) merged into their
    images on y = 0 (z = 0) (Section 3.6: periodic boundaries by vertex
    merging).  alpha is sampled at each node's master, so it is periodic;
    b ~ N(0,1) per node (slaves included: their loads add onto the merged
    unknown).  ``extra['master']`` holds the merge map."""
    rng = np.random.default_rng(9000 + seed)
    if dim == 2:
        coords, conn = square_mesh(n)
        coords = jitter_nodes(coords, n, 0.2, rng)
        axes = (1,)
    else:
        coords, conn = kuhn_cube_mesh(n)
        coords = jitter_nodes(coords, n, 0.15, rng)
        axes = (1, 2)
    master = periodic_master(coords, axes)
    alpha = alpha_fourier(coords, rng)[master]
    beta = np.exp(0.5 * rng.standard_normal(conn.shape[0]))
    dirichlet = _dirichlet_x0(coords)
    b = _rhs(rng, dirichlet)
    return Case("periodic_%dd_%d" % (dim, n), dim, coords, conn, dirichlet, alpha, beta,
                1e-2 if dim == 3 else 1e-3, b, np.zeros(coords.shape[0]), n=n, seed=seed,
                extra={"master": master})
