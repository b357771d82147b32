"""Seeded synthetic inputs for the V-ASMG-PCG solve path.

This module only builds *inputs*: vertex coordinates, P1 simplices, per-element
Lame parameters, Dirichlet degrees of freedom and a constant body force.  It
holds none of the solver's arithmetic (no assembly, no tree, no transfer
weights) and imports nothing else from this package, so the CPU oracle and the
CUDA library can both be fed from it without sharing method code.

Problem statement (Sec. 2, eq. (prob) and the weak form): isotropic linear
elasticity, -div sigma(u) = f with sigma = 2 mu eps + lambda tr(eps) I and the
Lame constants mu = E/(2(1+nu)), lambda = E nu/((1+nu)(1-2nu)).  The paper's own
meshes are not available; the workloads here are synthetic stand-ins with the
same kind of structure (unstructured P1 triangles / tetrahedra, 7 vertex blocks
per row in 2D and about 15 in 3D, matching the nnz/row of the paper's Sec. 5
tables).

Randomness is a counter-based splitmix64 stream (Steele, Lea and Flood, 2014;
the public-domain reference constants by S. Vigna), so the same seed yields the
same mesh on any machine and numpy version.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """splitmix64 output function applied to a uint64 counter array."""
    with np.errstate(over="ignore"):
        z = counter.astype(np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class Stream:
    """Counter-based splitmix64 stream: draw k returns splitmix64(seed*2^32 + k)."""

    def __init__(self, seed: int):
        self.base = np.uint64((int(seed) & 0xFFFFFFFF) << 32)
        self.pos = 0

    def u64(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            c = self.base + np.arange(self.pos, self.pos + n, dtype=np.uint64)
        self.pos += n
        return splitmix64(c)

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        """Uniform doubles in [lo, hi) from the top 53 bits."""
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def bernoulli(self, n: int) -> np.ndarray:
        return (self.u64(n) >> np.uint64(63)).astype(bool)


def lame(E, nu):
    """Lame constants from Young's modulus and Poisson's ratio (Sec. 2)."""
    E = np.asarray(E, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return lam, mu


def _signed_measure(coords: np.ndarray, elems: np.ndarray) -> np.ndarray:
    """Signed d!*volume of each simplex (input validation only)."""
    x0 = coords[elems[:, 0]]
    J = np.stack([coords[elems[:, k]] - x0 for k in range(1, elems.shape[1])], axis=-1)
    return np.linalg.det(J)


def square_mesh(n: int, jitter: float = 0.2, seed: int = 1, graded_ratio: float | None = None):
    """n x n vertex grid on the unit square, interior vertices jittered by
    U(-jitter*h, jitter*h) per axis, each quad split along a random diagonal.

    Returns (coords[N,2] float64, elems[2(n-1)^2, 3] int32), vertex id = j*n + i.
    """
    if n < 2:
        raise ValueError("n >= 2")
    for attempt in range(8):
        rs = Stream(seed + attempt)
        t = _axis(n, graded_ratio)
        h = 1.0 / (n - 1)
        X, Y = np.meshgrid(t, t, indexing="xy")
        coords = np.stack([X.ravel(), Y.ravel()], axis=1).copy()
        if jitter > 0 and n > 2:
            interior = np.zeros((n, n), dtype=bool)
            interior[1:-1, 1:-1] = True
            idx = np.nonzero(interior.ravel())[0]
            coords[idx] += rs.uniform(2 * idx.size, -jitter * h, jitter * h).reshape(-1, 2)
        i, j = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="xy")
        v00 = (j * n + i).ravel()
        v10 = v00 + 1
        v01 = v00 + n
        v11 = v01 + 1
        diag = rs.bernoulli(v00.size)
        # diagonal v00-v11 or v10-v01; both splits counter-clockwise
        t1 = np.where(diag[:, None], np.stack([v00, v10, v11], 1), np.stack([v00, v10, v01], 1))
        t2 = np.where(diag[:, None], np.stack([v00, v11, v01], 1), np.stack([v10, v11, v01], 1))
        elems = np.empty((2 * v00.size, 3), dtype=np.int32)
        elems[0::2] = t1
        elems[1::2] = t2
        if np.all(_signed_measure(coords, elems) > 0):
            return coords, elems
    raise RuntimeError("could not draw a valid mesh")


def _axis(n: int, graded_ratio: float | None) -> np.ndarray:
    if graded_ratio is None or graded_ratio == 1.0:
        return np.linspace(0.0, 1.0, n)
    # spacing grows geometrically: last spacing / first spacing = graded_ratio
    r = graded_ratio ** (1.0 / (n - 2))
    i = np.arange(n, dtype=np.float64)
    t = (r ** i - 1.0) / (r ** (n - 1) - 1.0)
    t[-1] = 1.0
    return t


# Kuhn (Freudenthal) split of the unit hex into 6 tetrahedra sharing the main
# diagonal (0,0,0)-(1,1,1): one per permutation of the axes.
_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def cube_mesh(n: int, jitter: float = 0.15, seed: int = 3, graded_ratio: float | None = None):
    """n^3 vertex grid on the unit cube, interior vertices jittered, each hex
    split into 6 Kuhn tetrahedra (conforming).  Vertex id = (k*n + j)*n + i."""
    if n < 2:
        raise ValueError("n >= 2")
    for attempt in range(8):
        rs = Stream(seed + attempt)
        t = _axis(n, graded_ratio)
        h = 1.0 / (n - 1)
        Z, Y, X = np.meshgrid(t, t, t, indexing="ij")
        coords = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).copy()
        if jitter > 0 and n > 2:
            interior = np.zeros((n, n, n), dtype=bool)
            interior[1:-1, 1:-1, 1:-1] = True
            idx = np.nonzero(interior.ravel())[0]
            coords[idx] += rs.uniform(3 * idx.size, -jitter * h, jitter * h).reshape(-1, 3)
        k, j, i = np.meshgrid(np.arange(n - 1), np.arange(n - 1), np.arange(n - 1), indexing="ij")
        base = ((k * n + j) * n + i).ravel()
        step = np.array([1, n, n * n], dtype=np.int64)
        tets = []
        for p in _PERMS:
            a = base
            b = a + step[p[0]]
            c = b + step[p[1]]
            d = c + step[p[2]]
            # even permutations are positively oriented, odd ones swap two vertices
            parity = sum(1 for x in range(3) for y in range(x + 1, 3) if p[x] > p[y]) % 2
            tets.append(np.stack([a, b, c, d] if parity == 0 else [a, c, b, d], 1))
        elems = np.stack(tets, 1).reshape(-1, 4).astype(np.int32)
        if np.all(_signed_measure(coords, elems) > 0):
            return coords, elems
    raise RuntimeError("could not draw a valid mesh")


def clamped_face_dofs(coords: np.ndarray) -> np.ndarray:
    """All components of every vertex on the x = 0 edge/face (int64 dof ids,
    dof = vertex*dim + component)."""
    dim = coords.shape[1]
    v = np.nonzero(coords[:, 0] == 0.0)[0].astype(np.int64)
    return (v[:, None] * dim + np.arange(dim, dtype=np.int64)[None, :]).ravel()


def element_centroids(coords, elems):
    return coords[elems].mean(axis=1)


# Workloads.  Sizes follow the configurations the solver is benchmarked on.
WORKLOADS = {
    # 2D plane strain, unit square, 64x64 jittered grid, E=1, nu=0.3, f=(0,-1)
    "square64": dict(dim=2, n=64, jitter=0.2, seed=1, E=1.0, nu=0.3, checker=False, graded=None),
    # 2D plane strain, 1024x1024, E in {1,100} on an 8x8 checkerboard, nu=0.3
    "square1024_checker": dict(dim=2, n=1024, jitter=0.2, seed=2, E=1.0, nu=0.3, checker=True, graded=None),
    # 3D, unit cube 64^3, jitter 0.15h, Kuhn tets, E=1, nu=0.3, f=(0,0,-1)
    "cube64": dict(dim=3, n=64, jitter=0.15, seed=3, E=1.0, nu=0.3, checker=False, graded=None),
    # 3D graded 128^3 (spacing ratio 16 toward the origin), no jitter, nu=0.45
    "cube128_graded": dict(dim=3, n=128, jitter=0.0, seed=4, E=1.0, nu=0.45, checker=False, graded=16.0),
}


def make_problem(name: str | None = None, *, dim=2, n=16, jitter=0.2, seed=1, E=1.0, nu=0.3,
                 checker=False, graded=None):
    """Build one synthetic problem as a dict of numpy arrays.

    Keys: dim, coords, elems, lam, mu (per element), dirichlet_dofs,
    dirichlet_values (None = homogeneous), body_force (length dim).
    """
    if name is not None:
        cfg = dict(WORKLOADS[name])
        dim, n, jitter, seed = cfg["dim"], cfg["n"], cfg["jitter"], cfg["seed"]
        E, nu, checker, graded = cfg["E"], cfg["nu"], cfg["checker"], cfg["graded"]
    if dim == 2:
        coords, elems = square_mesh(n, jitter, seed, graded)
    else:
        coords, elems = cube_mesh(n, jitter, seed, graded)
    ne = elems.shape[0]
    if checker:
        c = element_centroids(coords, elems)
        cell = np.floor(8.0 * c[:, 0]).astype(np.int64) + np.floor(8.0 * c[:, 1]).astype(np.int64)
        Ev = np.where(cell % 2 == 0, 1.0, 100.0)
    else:
        Ev = np.full(ne, float(E))
    lam, mu = lame(Ev, np.full(ne, float(nu)))
    f = np.zeros(dim)
    f[-1] = -1.0
    return dict(dim=dim, coords=np.ascontiguousarray(coords), elems=np.ascontiguousarray(elems),
                lam=np.ascontiguousarray(lam), mu=np.ascontiguousarray(mu),
                dirichlet_dofs=clamped_face_dofs(coords), dirichlet_values=None, body_force=f)


def random_problem(seed: int, dim: int | None = None, n_range=(3, 12)):
    """Small random problem for property tests: random size, material and jitter."""
    rs = Stream(1000 + seed)
    u = rs.uniform(6)
    if dim is None:
        dim = 2 if u[0] < 0.5 else 3
    n = int(n_range[0] + (n_range[1] - n_range[0] + 1) * u[1])
    if dim == 3:
        n = max(3, min(n, 9))
    E = 1.0 + 99.0 * u[2]
    nu = 0.2 + 0.25 * u[3]
    jit = (0.2 if dim == 2 else 0.15) * u[4]
    return make_problem(None, dim=dim, n=n, jitter=jit, seed=seed, E=E, nu=nu)


# ---------------------------------------------------------------- the paper's 2D examples (Sec. 5)
#
# Mapped structured P1 meshes of the four 2D geometries of Sec. 5 (Examples
# 4.1-4.4), with their boundary conditions.  The paper's own unstructured meshes
# are not available, so the vertex counts follow its tables instead.  Line
# forces are given to the solver as a load vector of nodal forces: a uniform
# traction q on a boundary edge of length l puts q l / 2 on each of its ends.

PAPER_EXAMPLES = {
    # name: (paper example, vertices in the paper's table, V-ASMG iterations in the paper's table)
    "hole_round": ("4.1 round-hole plate", 99054, 9),
    "ring": ("4.2 quarter ring", 150129, 11),
    "hole_square": ("4.3 square-hole plate", 200185, 10),
    "dam": ("4.4 thin-walled water retaining structure", 249278, 12),
}


def _grid_triangles(P: np.ndarray):
    """Vertices P[a, b] (a-major) of a mapped grid; each cell split in two
    triangles along alternating diagonals, all counter-clockwise."""
    n1, n2 = P.shape[:2]
    coords = np.ascontiguousarray(P.reshape(-1, 2))
    a, b = np.meshgrid(np.arange(n1 - 1), np.arange(n2 - 1), indexing="ij")
    v00 = (a * n2 + b).ravel()
    v01 = v00 + 1
    v10 = v00 + n2
    v11 = v10 + 1
    alt = ((a + b) % 2 == 0).ravel()
    t1 = np.where(alt[:, None], np.stack([v00, v10, v11], 1), np.stack([v00, v10, v01], 1))
    t2 = np.where(alt[:, None], np.stack([v00, v11, v01], 1), np.stack([v10, v11, v01], 1))
    elems = np.empty((2 * v00.size, 3), dtype=np.int32)
    elems[0::2] = t1
    elems[1::2] = t2
    neg = _signed_measure(coords, elems) < 0
    elems[neg] = elems[neg][:, [0, 2, 1]]
    if not np.all(_signed_measure(coords, elems) > 0):
        raise RuntimeError("degenerate mapped mesh")
    return coords, elems


def _edge_load(coords: np.ndarray, chain: np.ndarray, q) -> np.ndarray:
    """Nodal forces of a uniform traction q along the boundary polyline
    through the vertices `chain` (in order)."""
    F = np.zeros(coords.shape[0] * 2)
    x = coords[chain]
    seg = np.linalg.norm(x[1:] - x[:-1], axis=1)
    for c in range(2):
        np.add.at(F, chain[:-1] * 2 + c, 0.5 * q[c] * seg)
        np.add.at(F, chain[1:] * 2 + c, 0.5 * q[c] * seg)
    return F


def _graded(n: int, ratio: float) -> np.ndarray:
    """n points on [0, 1], spacing growing geometrically by `ratio` overall."""
    if ratio == 1.0:
        return np.linspace(0.0, 1.0, n)
    g = ratio ** (1.0 / (n - 2))
    t = (g ** np.arange(n) - 1.0) / (g ** (n - 1) - 1.0)
    t[-1] = 1.0
    return t


def paper_example(name: str, scale: float = 1.0) -> dict:
    """One of the paper's 2D examples (E = 2.1e5, nu = 0.3) with about
    `scale` times the paper's vertex count.  Returns the problem dict of
    make_problem with the load vector in key "F" (body_force is zero)."""
    E, nu = 2.1e5, 0.3
    nvert = max(200, int(PAPER_EXAMPLES[name][1] * scale))
    if name in ("hole_round", "hole_square"):
        # O-grid of the top-right quarter of the 10 x 10 plate around the hole
        nt = int(np.sqrt(nvert)) | 1          # odd: the corner (10, 10) is a grid line
        nr = max(3, nvert // nt)
        th = np.linspace(0.0, np.pi / 2, nt)
        rho = _graded(nr, 10.0)
        c, s = np.cos(th), np.sin(th)
        c[-1], s[0] = 0.0, 0.0
        lower = th <= np.pi / 4
        half = nt // 2
        outer = np.where(lower[:, None], np.stack([np.full(nt, 10.0), 10.0 * np.tan(th)], 1),
                         np.stack([10.0 * c / np.where(s > 0, s, 1.0), np.full(nt, 10.0)], 1))
        outer[half] = (10.0, 10.0)
        outer[-1] = (0.0, 10.0)
        outer[0] = (10.0, 0.0)
        if name == "hole_round":
            inner = np.stack([c, s], 1)
        else:
            inner = np.where(lower[:, None], np.stack([np.ones(nt), np.tan(th)], 1),
                             np.stack([c / np.where(s > 0, s, 1.0), np.ones(nt)], 1))
            inner[half] = (1.0, 1.0)
            inner[-1] = (0.0, 1.0)
            inner[0] = (1.0, 0.0)
        P = inner[:, None, :] + rho[None, :, None] * (outer - inner)[:, None, :]
        coords, elems = _grid_triangles(P)
        vid = np.arange(nt * nr).reshape(nt, nr)
        left = vid[-1, :]              # x = 0: u1 = 0
        bottom = vid[0, :]             # y = 0: u2 = 0
        dd = np.concatenate([left * 2, bottom * 2 + 1]).astype(np.int64)
        F = _edge_load(coords, vid[: half + 1, -1], (10.0, 0.0))   # x = 10: q1 = 10
        lam_c, mu_c = lame(E, nu)
    elif name == "ring":
        # quarter ring 1 <= r <= 10, left boundary clamped, bottom loaded
        nt = int(np.sqrt(nvert))
        nr = max(3, nvert // nt)
        th = np.linspace(0.0, np.pi / 2, nt)
        r = 10.0 ** np.linspace(0.0, 1.0, nr)
        c, s = np.cos(th), np.sin(th)
        c[-1], s[0] = 0.0, 0.0
        P = np.stack([c[:, None] * r[None, :], s[:, None] * r[None, :]], -1)
        coords, elems = _grid_triangles(P)
        vid = np.arange(nt * nr).reshape(nt, nr)
        left = vid[-1, :]              # x = 0: u1 = u2 = 0
        dd = np.concatenate([left * 2, left * 2 + 1]).astype(np.int64)
        F = _edge_load(coords, vid[0, :], (0.0, -10.0))            # y = 0: q2 = -10
        lam_c, mu_c = lame(E, nu)
    elif name == "dam":
        # trapezoid: height 20, bottom width 10, top width 3, left side vertical
        ny = int(np.sqrt(2 * nvert))
        nx = max(3, nvert // ny)
        y = np.linspace(0.0, 20.0, ny)
        t = np.linspace(0.0, 1.0, nx)
        xr = 10.0 - 7.0 * y / 20.0
        P = np.stack([t[None, :] * xr[:, None], np.broadcast_to(y[:, None], (ny, nx))], -1)
        coords, elems = _grid_triangles(P)
        vid = np.arange(ny * nx).reshape(ny, nx)
        bottom = vid[0, :]             # y = 0: u1 = u2 = 0
        dd = np.concatenate([bottom * 2, bottom * 2 + 1]).astype(np.int64)
        F = _edge_load(coords, vid[:, 0], (10.0, 0.0))             # x = 0: q1 = 10
        lam3, mu_c = lame(E, nu)
        lam_c = 2.0 * lam3 * mu_c / (lam3 + 2.0 * mu_c)           # plane stress
    else:
        raise KeyError(name)
    ne = elems.shape[0]
    F[dd] = 0.0
    return dict(dim=2, coords=coords, elems=elems, lam=np.full(ne, float(lam_c)), mu=np.full(ne, float(mu_c)),
                dirichlet_dofs=np.unique(dd), dirichlet_values=None, body_force=np.zeros(2), F=F)
