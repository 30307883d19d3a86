"""Seeded synthetic inputs: domains (simplicial meshes) and site sets.

This module holds no Voronoi arithmetic. It only draws random numbers and
builds meshes, and it is the one module that both the CUDA path (through the
tests and the bench) and the CPU oracle are fed from.

Every generator is deterministic for a given seed (numpy PCG64). Coordinates
of the FP32 workloads are rounded to float32 here, so that the GPU path and
the oracle read the same values (the oracle widens them exactly to float64).

Workloads (the paper's datasets are not available; these stand in for them,
with the shapes the paper's experiments use, Sec. 6):
  * ``square``   unit square as 2 triangles, 1,000 uniform sites (2D, FP64)
  * ``cube``     unit cube split into 6 tetrahedra, 100,000 uniform sites
  * ``shell``    tetrahedralised spherical shell (radii 0.5 / 1.0, 172,032
                 tets), 1,000,000 sites: 16-component Gaussian mixture
                 (sigma 0.02) plus 10% uniform background
  * ``torus``    torus surface (R=1, r=0.3, 500,000 triangles), 200,000 sites
                 sampled by area and jittered off the surface
  * ``cube2m``   unit cube (6 tets), 2,000,000 uniform sites
  * ``box``, ``box5m``  the unit cube as one box: 100,000 / 5,000,000 uniform
                 sites (white noise)
  * ``grid5m``   the unit cube as one box: 171^3 perturbed lattice centres
  * ``blue5m``   box5m's sites marked for 100 Lloyd iterations of the library
                 (blue noise by centroidal Voronoi relaxation, the paper's recipe)
  * ``blue100k`` the unit cube as one box: 100,000 Poisson-disk (blue noise)
                 sites drawn here, on the CPU
"""
from __future__ import annotations

import itertools

import numpy as np

SEED_BASE = 0xB3000000

MODE_2D = 2        # sites in the plane z=0, triangles in z=0
MODE_SURFACE = 3   # sites in R^3, triangle mesh in R^3 (restricted VD)
MODE_3D = 4        # sites in R^3, tetrahedral mesh (clipped VD)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------
# domains
# --------------------------------------------------------------------------
def square_2tri(lo: float = 0.0, hi: float = 1.0):
    """Unit square split on the (lo,lo)-(hi,hi) diagonal into two triangles."""
    verts = np.array([[lo, lo, 0.0], [hi, lo, 0.0], [hi, hi, 0.0], [lo, hi, 0.0]])
    tris = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    return verts, tris


def square_grid_tris(N: int, lo: float = 0.0, hi: float = 1.0, ticks=None):
    """Square [lo,hi]^2 as an N x N grid of quads, each split on its diagonal.

    ``ticks`` (length N+1) overrides the grid-line positions."""
    g = np.linspace(lo, hi, N + 1) if ticks is None else np.asarray(ticks, dtype=np.float64)
    X, Y = np.meshgrid(g, g, indexing="ij")
    verts = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    idx = lambda i, j: i * (N + 1) + j  # noqa: E731
    tris = []
    for i in range(N):
        for j in range(N):
            a, b, c, d = idx(i, j), idx(i + 1, j), idx(i + 1, j + 1), idx(i, j + 1)
            tris.append([a, b, c])
            tris.append([a, c, d])
    return verts, np.array(tris, dtype=np.int32)


_KUHN_PATHS = list(itertools.permutations(range(3)))


def _kuhn_cube(corner_index):
    """6 tets of one cube as lists of 4 lattice offsets (Kuhn / Freudenthal split).

    Tet for permutation s: 0 -> e_s0 -> e_s0+e_s1 -> (1,1,1); every cube of a
    lattice uses the same 6 paths, so the split is conforming across cubes.
    """
    out = []
    for s in _KUHN_PATHS:
        p = [0, 0, 0]
        tet = [tuple(p)]
        for ax in s:
            p[ax] += 1
            tet.append(tuple(p))
        out.append(tet)
    return out


def kuhn_lattice_tets(N: int, keep=None, lo: float = 0.0, hi: float = 1.0, ticks=None):
    """Lattice of N^3 cubes on [lo,hi]^3, each split into 6 tets.

    ``keep(ix, iy, iz)`` selects cubes (by lower-corner index); vertices that no
    kept cube uses are dropped.  ``ticks`` (length N+1) overrides the lattice
    plane positions.  Tets are oriented to positive volume.
    """
    tk = np.linspace(lo, hi, N + 1) if ticks is None else np.asarray(ticks, dtype=np.float64)
    vid = {}
    verts = []
    tets = []
    for ix in range(N):
        for iy in range(N):
            for iz in range(N):
                if keep is not None and not keep(ix, iy, iz):
                    continue
                for tet in _kuhn_cube(None):
                    ids = []
                    for (dx, dy, dz) in tet:
                        key = (ix + dx, iy + dy, iz + dz)
                        if key not in vid:
                            vid[key] = len(verts)
                            verts.append([tk[key[0]], tk[key[1]], tk[key[2]]])
                        ids.append(vid[key])
                    tets.append(ids)
    verts = np.array(verts, dtype=np.float64)
    tets = np.array(tets, dtype=np.int32)
    return verts, _orient_tets(verts, tets)


def _tet_volumes(verts, tets):
    a = verts[tets[:, 0]]
    e1 = verts[tets[:, 1]] - a
    e2 = verts[tets[:, 2]] - a
    e3 = verts[tets[:, 3]] - a
    return np.einsum("ij,ij->i", e1, np.cross(e2, e3)) / 6.0


def _orient_tets(verts, tets):
    vol = _tet_volumes(verts, tets)
    tets = tets.copy()
    neg = vol < 0
    tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()
    return tets


def cube_6tet():
    """Unit cube as the 6 Kuhn tetrahedra around the (0,0,0)-(1,1,1) diagonal."""
    return kuhn_lattice_tets(1)


def shell_domain(ncube: int = 32, seed: int = SEED_BASE + 3, jitter: float = 0.05):
    """Tetrahedralised spherical shell, radii 0.5 and 1.0.

    A lattice of ``ncube``^3 cubes on [-1,1]^3 keeps the cubes lying in the
    L-infinity shell 0.5 <= |x|_inf <= 1 (28,672 cubes for ncube=32), splits each
    into 6 Kuhn tets (172,032 tets), maps every vertex x -> x |x|_inf / |x|_2
    (the L-inf shell onto the Euclidean shell) and jitters the interior
    vertices by U[-jitter*h, jitter*h] per coordinate (h = 2/ncube).  Vertices
    are rounded to float32.  The tets keep the orientation of the unjittered
    mesh (a proper tetrahedralisation of the region), and a vertex whose jitter
    would invert one of its tets stays unjittered: re-orienting an inverted tet
    would fold it over its neighbours, so that tets overlap.
    """
    h = 2.0 / ncube
    lo_in = int(round(0.5 / h))  # number of cubes from -1 to -0.5

    def keep(ix, iy, iz):
        # cube [x0, x0+h] lies outside the open cube (-0.5, 0.5)^3
        for i in (ix, iy, iz):
            if i < ncube // 2 - lo_in or i >= ncube // 2 + lo_in:
                return True
        return False

    verts, tets = kuhn_lattice_tets(ncube, keep, -1.0, 1.0)
    linf = np.abs(verts).max(axis=1)
    l2 = np.linalg.norm(verts, axis=1)
    verts = verts * (linf / l2)[:, None]
    interior = (np.abs(linf - 0.5) > 1e-12) & (np.abs(linf - 1.0) > 1e-12)
    tets = _orient_tets(verts, tets)
    rng = _rng(seed)
    jit = rng.uniform(-jitter * h, jitter * h, size=verts.shape) * interior[:, None]
    for _ in range(64):
        vj = (verts + jit).astype(np.float32).astype(np.float64)
        bad = _tet_volumes(vj, tets) <= 0
        if not bad.any():
            break
        jit[np.unique(tets[bad])] = 0.0
    vol = _tet_volumes(vj, tets)
    assert (vol > 0).all(), "shell tet with non-positive volume"
    return vj, tets


def torus_domain(nu: int = 1000, nv: int = 250, R: float = 1.0, r: float = 0.3,
                 seed: int = SEED_BASE + 4, jitter: float = 1e-3):
    """Torus surface mesh: (u,v) grid nu x nv, 2 triangles per quad.

    Every vertex coordinate is jittered by U[-jitter*L, jitter*L], L the mean
    edge length; coordinates are rounded to float32.
    """
    u = 2 * np.pi * np.arange(nu) / nu
    v = 2 * np.pi * np.arange(nv) / nv
    U, V = np.meshgrid(u, v, indexing="ij")
    X = (R + r * np.cos(V)) * np.cos(U)
    Y = (R + r * np.cos(V)) * np.sin(U)
    Z = r * np.sin(V)
    verts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    I, J = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    a = (I * nv + J).ravel()
    b = (((I + 1) % nu) * nv + J).ravel()
    c = (((I + 1) % nu) * nv + (J + 1) % nv).ravel()
    d = (I * nv + (J + 1) % nv).ravel()
    tris = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)]).astype(np.int32)
    e = np.concatenate([np.linalg.norm(verts[tris[:, k]] - verts[tris[:, (k + 1) % 3]], axis=1)
                        for k in range(3)])
    L = float(e.mean())
    rng = _rng(seed)
    verts = verts + rng.uniform(-jitter * L, jitter * L, size=verts.shape)
    verts = verts.astype(np.float32).astype(np.float64)
    return verts, tris


# --------------------------------------------------------------------------
# sites
# --------------------------------------------------------------------------
def _dedupe(pts, regen):
    while True:
        _, first = np.unique(pts, axis=0, return_index=True)
        if len(first) == len(pts):
            return pts
        dup = np.setdiff1d(np.arange(len(pts)), first)
        pts[dup] = regen(len(dup))


def uniform_sites(n: int, dim: int, seed: int, lo: float = 0.0, hi: float = 1.0,
                  f32: bool = True):
    """n i.i.d. uniform sites in [lo,hi]^dim (returned as n x 3, z=0 in 2D)."""
    rng = _rng(seed)

    def gen(k):
        p = np.zeros((k, 3))
        p[:, :dim] = rng.uniform(lo, hi, size=(k, dim))
        return p.astype(np.float32).astype(np.float64) if f32 else p

    return _dedupe(gen(n), gen)


def perturbed_grid_sites(k: int, seed: int, amp: float = 0.1):
    """Centres of a k^3 lattice in the unit cube moved by U[-amp h, amp h] per
    coordinate (h = 1/k), rounded to float32."""
    rng = _rng(seed)
    h = 1.0 / k
    g = (np.stack(np.meshgrid(np.arange(k), np.arange(k), np.arange(k), indexing="ij"), -1).reshape(-1, 3) + 0.5) * h
    g = g + rng.uniform(-amp * h, amp * h, size=g.shape)
    return g.astype(np.float32).astype(np.float64)


def poisson_disk_sites(n: int, seed: int, rounds: int = 6):
    """Blue noise in the unit cube: dart throwing with a minimum distance r between
    sites (Poisson-disk sampling), then n of the accepted sites kept at random.

    Cells of edge r / sqrt(3) hold at most one site.  Cells are visited in 27
    phases (cell index mod 3 per axis); within a phase no two cells are closer
    than 2 r / sqrt(3) > r, so each empty cell draws one candidate and keeps it
    if no site within r of it exists (cells within two of its own).  r is set
    from the density such samples reach (about 0.65 / r^3 sites per unit
    volume) so that the accepted sites exceed n.  Rounded to float32.
    """
    rng = _rng(seed)
    r = (0.60 / n) ** (1.0 / 3.0)
    G = int(np.ceil(np.sqrt(3.0) / r))
    h = 1.0 / G
    cell = -np.ones((G + 4,) * 3, dtype=np.int64)   # padded by 2: site index per cell
    pts = np.zeros((0, 3))
    grid = np.stack(np.meshgrid(np.arange(G), np.arange(G), np.arange(G), indexing="ij"), -1).reshape(-1, 3)
    phases = [grid[np.all(grid % 3 == np.array(ph), axis=1)] for ph in itertools.product(range(3), repeat=3)]
    offs = np.array([o for o in itertools.product(range(-2, 3), repeat=3) if o != (0, 0, 0)])
    r2 = r * r
    for _ in range(rounds):
        for cells in phases:
            cells = cells[cell[cells[:, 0] + 2, cells[:, 1] + 2, cells[:, 2] + 2] < 0]
            if len(cells) == 0:
                continue
            cand = (cells + rng.uniform(0, 1, size=cells.shape)) * h
            ok = np.ones(len(cells), dtype=bool)
            for o in offs:
                nb = cell[cells[:, 0] + 2 + o[0], cells[:, 1] + 2 + o[1], cells[:, 2] + 2 + o[2]]
                has = nb >= 0
                if not has.any():
                    continue
                d = pts[nb[has]] - cand[has]
                bad = np.einsum("ij,ij->i", d, d) < r2
                ok[np.nonzero(has)[0][bad]] = False
            keep = np.nonzero(ok)[0]
            cell[cells[keep, 0] + 2, cells[keep, 1] + 2, cells[keep, 2] + 2] = len(pts) + np.arange(len(keep))
            pts = np.concatenate([pts, cand[keep]])
    if len(pts) < n:
        raise ValueError(f"Poisson-disk sampling kept {len(pts)} < {n} sites")
    pts = pts[np.sort(rng.choice(len(pts), n, replace=False))]
    out = np.clip(pts, 0.0, 1.0).astype(np.float32).astype(np.float64)
    return _dedupe(out, lambda k: rng.uniform(0, 1, size=(k, 3)).astype(np.float32).astype(np.float64))


def lattice_sites(N: int, dim: int, lo: float = 0.0, hi: float = 1.0):
    """Sites at the centres of an N^dim lattice of boxes: lo + (k+1/2) h."""
    h = (hi - lo) / N
    g = lo + (np.arange(N) + 0.5) * h
    if dim == 2:
        X, Y = np.meshgrid(g, g, indexing="ij")
        return np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


SHELL_R_MIN, SHELL_R_MAX = 0.5, 0.99


def _in_shell(p):
    r = np.linalg.norm(p, axis=1)
    return (r >= SHELL_R_MIN) & (r <= SHELL_R_MAX)


def _uniform_in_shell(rng, k):
    out = np.empty((0, 3))
    while len(out) < k:
        p = rng.uniform(-1, 1, size=(2 * k + 64, 3))
        out = np.concatenate([out, p[_in_shell(p)]])
    return out[:k]


def shell_sites(n: int = 1_000_000, seed: int = SEED_BASE + 3, ncomp: int = 16,
                sigma: float = 0.02, background: float = 0.1):
    """Gaussian-mixture sites in the shell plus a uniform background.

    ``ncomp`` equal-weight isotropic Gaussians (std ``sigma``) with centres
    uniform in the shell; samples outside 0.5 <= |x| <= 0.99 are redrawn (that
    region lies inside the tetrahedralised shell: its boundary faces are flat
    chords of the two spheres).  A fraction ``background`` of the sites is
    uniform in the same region.  Float32 coordinates.
    """
    rng = _rng(seed)
    nbg = int(round(n * background))
    ncl = n - nbg
    centres = _uniform_in_shell(rng, ncomp)
    comp = np.arange(ncl) % ncomp
    pts = centres[comp] + sigma * rng.standard_normal((ncl, 3))
    bad = ~_in_shell(pts)
    while bad.any():
        pts[bad] = centres[comp[bad]] + sigma * rng.standard_normal((int(bad.sum()), 3))
        bad = ~_in_shell(pts)
    pts = np.concatenate([pts, _uniform_in_shell(rng, nbg)])
    pts = pts.astype(np.float32).astype(np.float64)
    return _dedupe(pts, lambda k: _uniform_in_shell(rng, k).astype(np.float32).astype(np.float64))


def surface_sites(n: int, verts, tris, seed: int, offset: float = 1e-4):
    """n sites on a triangle mesh: triangle chosen by area, uniform barycentric,
    then moved along the unit normal by U[-offset, offset].  Float32."""
    rng = _rng(seed)
    a, b, c = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    nrm = np.cross(b - a, c - a)
    area = 0.5 * np.linalg.norm(nrm, axis=1)
    unit = nrm / (2 * area)[:, None]
    cdf = np.cumsum(area)
    cdf /= cdf[-1]

    def gen(k):
        t = np.minimum(np.searchsorted(cdf, rng.uniform(0, 1, size=k)), len(cdf) - 1)
        r1 = np.sqrt(rng.uniform(0, 1, size=k))
        r2 = rng.uniform(0, 1, size=k)
        p = (1 - r1)[:, None] * a[t] + (r1 * (1 - r2))[:, None] * b[t] + (r1 * r2)[:, None] * c[t]
        p = p + rng.uniform(-offset, offset, size=k)[:, None] * unit[t]
        return p.astype(np.float32).astype(np.float64)

    return _dedupe(gen(n), gen)


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------
def workload(name: str, n: int | None = None, seed: int | None = None):
    """Return dict(mode, sites (n,3) f64, verts (nv,3) f64, simp (m,k) i32, f64, name).

    ``f64`` tells whether the path runs in float64 (the 2D square workload) or
    float32 (all others).  ``n`` and ``seed`` override the defaults so that the
    same recipe serves small parity cases.
    """
    if name == "square":
        verts, simp = square_2tri()
        n = 1000 if n is None else n
        seed = SEED_BASE + 1 if seed is None else seed
        sites = uniform_sites(n, 2, seed, f32=False)
        return dict(name=name, mode=MODE_2D, sites=sites, verts=verts, simp=simp, f64=True)
    if name in ("cube", "cube2m", "cube1m"):
        verts, simp = cube_6tet()
        n = {"cube": 100_000, "cube1m": 1_000_000, "cube2m": 2_000_000}[name] if n is None else n
        seed = (SEED_BASE + {"cube": 2, "cube1m": 6, "cube2m": 5}[name]) if seed is None else seed
        sites = uniform_sites(n, 3, seed)
        return dict(name=name, mode=MODE_3D, sites=sites, verts=verts, simp=simp, f64=False)
    if name in ("box", "box5m"):
        # the unit cube as one convex domain (the box form); the same cube as 6
        # tetrahedra is what the oracle clips
        verts, simp = cube_6tet()
        n = {"box": 100_000, "box5m": 5_000_000}[name] if n is None else n
        seed = (SEED_BASE + {"box": 2, "box5m": 7}[name]) if seed is None else seed
        sites = uniform_sites(n, 3, seed)
        return dict(name=name, mode=MODE_3D, sites=sites, verts=verts, simp=simp, f64=False,
                    box=((0.0, 0.0, 0.0), (1.0, 1.0, 1.0)))
    if name == "blue5m":
        # blue noise as the paper makes it (Sec. 6: sites relaxed by centroidal
        # Voronoi tessellation): the 5M white-noise box sites, to be relaxed by
        # `lloyd` graph-captured Lloyd iterations of the library before timing
        w = workload("box5m", n, seed)
        return dict(w, name=name, lloyd=100)
    if name == "blue100k":
        # blue noise drawn on the CPU (Poisson-disk dart throwing, no Voronoi
        # arithmetic), for checks against the oracle
        verts, simp = cube_6tet()
        n = 100_000 if n is None else n
        seed = SEED_BASE + 9 if seed is None else seed
        return dict(name=name, mode=MODE_3D, sites=poisson_disk_sites(n, seed), verts=verts, simp=simp, f64=False,
                    box=((0.0, 0.0, 0.0), (1.0, 1.0, 1.0)))
    if name == "grid5m":
        # perturbed grid: the centres of a 171^3 lattice (5,000,211 sites) moved by
        # U[-0.1 h, 0.1 h] per coordinate, in the unit cube as one convex domain
        verts, simp = cube_6tet()
        k = 171 if n is None else max(2, int(round(n ** (1.0 / 3.0))))
        seed = SEED_BASE + 8 if seed is None else seed
        sites = perturbed_grid_sites(k, seed)
        return dict(name=name, mode=MODE_3D, sites=sites, verts=verts, simp=simp, f64=False,
                    box=((0.0, 0.0, 0.0), (1.0, 1.0, 1.0)))
    if name == "shell":
        verts, simp = shell_domain()
        n = 1_000_000 if n is None else n
        seed = SEED_BASE + 3 if seed is None else seed
        sites = shell_sites(n, seed)
        return dict(name=name, mode=MODE_3D, sites=sites, verts=verts, simp=simp, f64=False)
    if name == "torus":
        verts, simp = torus_domain()
        n = 200_000 if n is None else n
        seed = SEED_BASE + 4 if seed is None else seed
        sites = surface_sites(n, verts, simp, seed)
        return dict(name=name, mode=MODE_SURFACE, sites=sites, verts=verts, simp=simp, f64=False)
    raise ValueError(f"unknown workload {name!r}")


def domain_measure(mode: int, verts, simp) -> float:
    """Total area (2D, surface) or volume (3D) of the mesh, in float64."""
    if mode == MODE_3D:
        return float(np.abs(_tet_volumes(verts, simp)).sum())
    a, b, c = verts[simp[:, 0]], verts[simp[:, 1]], verts[simp[:, 2]]
    return float(0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1).sum())


def simplex_measures(mode: int, verts, simp):
    if mode == MODE_3D:
        return np.abs(_tet_volumes(verts, simp))
    a, b, c = verts[simp[:, 0]], verts[simp[:, 1]], verts[simp[:, 2]]
    return 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)


def small_torus(nu: int = 40, nv: int = 12, seed: int = SEED_BASE + 40):
    return torus_domain(nu, nv, seed=seed)


def small_shell(ncube: int = 8, seed: int = SEED_BASE + 30):
    return shell_domain(ncube, seed)

