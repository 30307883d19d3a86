"""Exact rational computation of one 3D piece P_{a,i} = T_a ∩ ⋂_j H_ij (test helper).

Every input coordinate is a float (float32 values, held exactly as Fractions),
so each tetrahedron face and each bisector has an exact rational plane, and the
piece's corners follow exactly by Cramer's rule over all triples of planes.
The piece has positive volume iff its corners span 3D, and a plane bounds a
face of positive area iff the corners on it span 2D (Sec. 2.2: pieces and faces
count only with positive measure).  Brute force: C(m, 3) triples for m planes,
for small m only.  No code is shared with the oracle or with the CUDA path.
"""
from fractions import Fraction as F
from itertools import combinations

import numpy as np


def _det3(a, b, c):
    return (a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0])
            + a[2] * (b[0] * c[1] - b[1] * c[0]))


def _rank(points):
    """affine rank of a list of exact points (0..3)"""
    if not points:
        return -1
    p0 = points[0]
    rows = [[q[k] - p0[k] for k in range(3)] for q in points[1:]]
    rank, m = 0, [r[:] for r in rows]
    for col in range(3):
        piv = next((r for r in range(rank, len(m)) if m[r][col] != 0), None)
        if piv is None:
            continue
        m[rank], m[piv] = m[piv], m[rank]
        for r in range(len(m)):
            if r != rank and m[r][col] != 0:
                f = m[r][col] / m[rank][col]
                m[r] = [m[r][k] - f * m[rank][k] for k in range(3)]
        rank += 1
    return rank


def piece(tet_verts, vi, others):
    """tet_verts: 4x3 floats; vi: the site; others: (site id, coords) of the
    candidate sites.  Returns (positive volume, set of ids whose bisector bounds
    a face of positive area, number of tet faces of positive area, largest
    corner distance from vi -- a site farther than twice it cannot cut)."""
    tv = [tuple(F(float(x)) for x in v) for v in tet_verts]
    fi = tuple(F(float(x)) for x in vi)
    planes = []  # (n, c, source): n.x <= c ; source -1-f tet face f, else the site id
    for f in range(4):
        o = [tv[k] for k in range(4) if k != f]
        u = [o[1][k] - o[0][k] for k in range(3)]
        v = [o[2][k] - o[0][k] for k in range(3)]
        n = [u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]]
        c = sum(n[k] * o[0][k] for k in range(3))
        if sum(n[k] * tv[f][k] for k in range(3)) > c:  # the opposite vertex inside
            n, c = [-x for x in n], -c
        planes.append((n, c, -1 - f))
    for j, vj in others:
        fj = tuple(F(float(x)) for x in vj)
        n = [fj[k] - fi[k] for k in range(3)]
        c = (sum(x * x for x in fj) - sum(x * x for x in fi)) / 2
        planes.append((n, c, int(j)))
    corners = set()
    for x, y, z in combinations(range(len(planes)), 3):
        A = [planes[x][0], planes[y][0], planes[z][0]]
        D = _det3(*A)
        if D == 0:
            continue
        b = [planes[x][1], planes[y][1], planes[z][1]]
        q = []
        for k in range(3):
            M = [list(r) for r in A]
            for r in range(3):
                M[r][k] = b[r]
            q.append(_det3(*M) / D)
        if all(sum(p[0][k] * q[k] for k in range(3)) <= p[1] for p in planes):
            corners.add(tuple(q))
    corners = list(corners)
    positive = _rank(corners) == 3
    faces, tet_faces = set(), 0
    if positive:
        for n, c, src in planes:
            on = [q for q in corners if sum(n[k] * q[k] for k in range(3)) == c]
            if _rank(on) == 2:
                if src >= 0:
                    faces.add(src)
                else:
                    tet_faces += 1
    reach = max((float(sum((q[k] - fi[k]) ** 2 for k in range(3))) ** 0.5 for q in corners), default=0.0)
    return positive, faces, tet_faces, reach


def candidates(sites, i, k):
    """the k nearest sites of site i (by float64 distance), as (id, coords), and
    the distance of the nearest site left out"""
    d = np.linalg.norm(sites - sites[i], axis=1)
    d[i] = np.inf
    order = np.argsort(d, kind="stable")
    nb = order[:k]
    return [(int(j), sites[j]) for j in nb], float(d[order[k]]) if k < len(order) - 1 else np.inf


def polygon_piece(tri_verts, vi, others):
    """2D analogue: triangle T (3x2 floats) clipped by the bisectors of vi with
    the candidate sites, exactly.  Returns (positive area, set of ids whose
    bisector bounds an edge of positive length, number of triangle edges of
    positive length)."""
    tv = [tuple(F(float(x)) for x in v[:2]) for v in tri_verts]
    fi = tuple(F(float(x)) for x in vi[:2])
    lines = []  # (n, c, source): n.x <= c
    for f in range(3):
        a, b = [tv[k] for k in range(3) if k != f]
        n = [b[1] - a[1], a[0] - b[0]]
        c = n[0] * a[0] + n[1] * a[1]
        if n[0] * tv[f][0] + n[1] * tv[f][1] > c:
            n, c = [-n[0], -n[1]], -c
        lines.append((n, c, -1 - f))
    for j, vj in others:
        fj = tuple(F(float(x)) for x in vj[:2])
        n = [fj[0] - fi[0], fj[1] - fi[1]]
        c = (fj[0] ** 2 + fj[1] ** 2 - fi[0] ** 2 - fi[1] ** 2) / 2
        lines.append((n, c, int(j)))
    return _polygon(lines)


def surface_piece(tri_verts, vi, others):
    """Surface: triangle T in 3D (3x3 floats) clipped by the 3D bisectors of vi,
    exactly, in the triangle's own coordinates p = A + s (B - A) + t (C - A)
    (an affine map: positive length and area are kept).  Same returns as
    polygon_piece."""
    A, Bv, Cv = [tuple(F(float(x)) for x in v) for v in tri_verts]
    e1 = [Bv[k] - A[k] for k in range(3)]
    e2 = [Cv[k] - A[k] for k in range(3)]
    fi = tuple(F(float(x)) for x in vi)
    # triangle edges opposite vertex 0, 1, 2: s + t <= 1, s >= 0 (-s <= 0), t >= 0
    lines = [([F(1), F(1)], F(1), -1), ([F(-1), F(0)], F(0), -2), ([F(0), F(-1)], F(0), -3)]
    for j, vj in others:
        fj = tuple(F(float(x)) for x in vj)
        n = [fj[k] - fi[k] for k in range(3)]
        c = (sum(x * x for x in fj) - sum(x * x for x in fi)) / 2
        ns = sum(n[k] * e1[k] for k in range(3))
        nt = sum(n[k] * e2[k] for k in range(3))
        lines.append(([ns, nt], c - sum(n[k] * A[k] for k in range(3)), int(j)))
    return _polygon(lines)


def _polygon(lines):
    corners = set()
    for x, y in combinations(range(len(lines)), 2):
        (n0, c0, _), (n1, c1, _) = lines[x], lines[y]
        D = n0[0] * n1[1] - n0[1] * n1[0]
        if D == 0:
            continue
        q = ((c0 * n1[1] - c1 * n0[1]) / D, (n0[0] * c1 - n1[0] * c0) / D)
        if all(n[0] * q[0] + n[1] * q[1] <= c for n, c, _ in lines):
            corners.add(q)
    corners = list(corners)

    def rank2(pts):
        if not pts:
            return -1
        p0 = pts[0]
        vecs = [(p[0] - p0[0], p[1] - p0[1]) for p in pts[1:]]
        if all(v == (0, 0) for v in vecs):
            return 0
        v0 = next(v for v in vecs if v != (0, 0))
        return 2 if any(v0[0] * v[1] - v0[1] * v[0] != 0 for v in vecs) else 1

    positive = rank2(corners) == 2
    edges, tri_edges = set(), 0
    if positive:
        for n, c, src in lines:
            on = [q for q in corners if n[0] * q[0] + n[1] * q[1] == c]
            if rank2(on) == 1:
                if src >= 0:
                    edges.add(src)
                else:
                    tri_edges += 1
    return positive, edges, tri_edges
