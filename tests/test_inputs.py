"""The seeded tetrahedral domains are proper tetrahedralisations.

The clipped diagram of Eq. 1 is a partition of the region only when the
tetrahedra do not overlap; the split of Alg. 5 computes a cell inside the region
as one piece, which equals the sum of its per-tetrahedron pieces only then.  With
every tetrahedron positively oriented, the sum of their volumes equals the
volume the boundary faces enclose (divergence theorem) exactly when no region
is covered twice."""
import numpy as np
import pytest

from paper_2509_07175_b300 import inputs as I


def _enclosed(verts, tets):
    faces = {}
    for a, t in enumerate(tets):
        for f in range(4):
            faces.setdefault(tuple(sorted(int(x) for k, x in enumerate(t) if k != f)), []).append((a, f))
    vol = 0.0
    for lst in faces.values():
        if len(lst) != 1:
            continue
        a, f = lst[0]
        t = tets[a]
        P = verts[[int(x) for k, x in enumerate(t) if k != f]]
        n = np.cross(P[1] - P[0], P[2] - P[0])
        if np.dot(n, verts[int(t[f])] - P[0]) > 0:
            n = -n  # outward
        vol += np.dot(n, P[0]) / 6.0
    return vol


@pytest.mark.parametrize("name", ["shell8", "shell16", "lattice3", "cube6"])
def test_tet_domains_do_not_overlap(name):
    if name.startswith("shell"):
        v, t = I.small_shell(int(name[5:]))
    elif name == "lattice3":
        v, t = I.kuhn_lattice_tets(3)
    else:
        v, t = I.cube_6tet()
    vol = I._tet_volumes(v, t)
    assert (vol > 0).all()
    assert abs(vol.sum() - _enclosed(v, t)) <= 1e-12 * vol.sum()


def test_shell_workload_domain_does_not_overlap():
    v, t = I.shell_domain()
    vol = I._tet_volumes(v, t)
    assert len(t) == 172032 and (vol > 0).all()
    assert abs(vol.sum() - _enclosed(v, t)) <= 1e-12 * vol.sum()
    # most interior vertices keep their jitter
    v0, _ = I.shell_domain(jitter=0.0)
    assert np.any(v != v0, axis=1).mean() > 0.6


def test_fold_detector_sees_an_inverted_tet():
    # the check above is not vacuous: re-orienting an inverted tet (what the
    # generator must not do) makes the volumes exceed the enclosed volume
    v, t = I.kuhn_lattice_tets(2)
    v = v.copy()
    k = np.argmin(np.linalg.norm(v - 0.5, axis=1))  # the centre vertex
    v[k] += 0.6                                       # pushed out through the boundary
    t2 = I._orient_tets(v, t)
    vol = I._tet_volumes(v, t2)
    assert vol.sum() - _enclosed(v, t2) > 1e-3
