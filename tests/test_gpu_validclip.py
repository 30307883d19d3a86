"""Valid clippings (Sec. 3.3): with the search starting inside the cell's own
simplex, every clip leaves a bisector face of positive measure on the final
piece, so the clips equal the bisector faces.  Alg. 3 searches on the virtual
edge v_i -> p (Sec. 4.1); where v_i lies outside the simplex the exit point of
Omega_i may lie outside it too, and such clips are counted apart
(VD_STAT_EXCESS_CLIPS).  A clip by a corner's certified witness after an FP32
search failed (VD_STAT_FALLBACK) may also leave no face."""
import numpy as np
import pytest

from paper_2509_07175_b300 import binding as B
from paper_2509_07175_b300 import inputs as I

pytestmark = pytest.mark.gpu


def _faces_from_pieces(p):
    m = p["measure"].double().cpu().numpy()
    off = p["flag_off"].cpu().numpy()
    fl = p["flags"].cpu().numpy()
    return int(sum((fl[off[q]:off[q + 1]] >= 0).sum() for q in np.nonzero(m > 0)[0]))


@pytest.mark.parametrize("learned", [0, 1])
def test_box_form_every_clip_contributes(gpu, learned):
    """Box form (Sec. 4.2): every site lies in the box, so every clip found by the
    search contributes; the bisector faces are the neighbour entries."""
    w = I.workload("box", n=20000)
    d = B.diagram_from_workload(w, options=dict(stats=1, learned=learned, topk=16))
    r = d.compute()
    s = r["stats"]
    assert s["clips"] == s["bisector_faces"] + s["excess_clips"]
    assert s["excess_clips"] <= s["fallback"], s
    assert s["bisector_faces"] == int(r["nbr_off"][-1].item())
    d.close()


@pytest.mark.parametrize("name,n", [("cube", 20000), ("square", 1000)])
def test_per_simplex_excess_is_counted(gpu, name, n):
    """Per-simplex pieces: the bisector faces counted by the kernel equal the
    positive flags of the exported pieces, and every clip is either one of them or
    an excess clip."""
    w = I.workload(name, n=n)
    d = B.diagram_from_workload(w, options=dict(stats=1))
    r = d.compute()
    s = r["stats"]
    assert s["clips"] == s["bisector_faces"] + s["excess_clips"]
    assert s["bisector_faces"] == _faces_from_pieces(d.pieces())
    print(f"{name}: clips {s['clips']} bisector faces {s['bisector_faces']} excess {s['excess_clips']} "
          f"fallback {s['fallback']}")
    d.close()


def test_split_whole_cells(gpu):
    """The split (Alg. 5): whole cells start from the mesh box around their site,
    so their clips contribute; only the boundary sites' per-tetrahedron pieces can
    add excess clips."""
    w = I.workload("cube", n=20000)
    d = B.diagram_from_workload(w, options=dict(stats=1, split=1, learned=1))
    r = d.compute()
    s = r["stats"]
    assert s["whole_cells"] > 0
    assert s["clips"] == s["bisector_faces"] + s["excess_clips"]
    assert s["bisector_faces"] == _faces_from_pieces(d.pieces())
    d.close()
