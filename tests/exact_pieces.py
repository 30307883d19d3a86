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
