"""Asynchronous compute with a lazily read status, capture of that compute into a
caller's CUDA graph, and the network's state saved to and loaded from a file."""
import os

import numpy as np
import pytest
import torch

from paper_2509_07175_b300 import binding as B
from paper_2509_07175_b300 import inputs as I

pytestmark = pytest.mark.gpu

KEYS = ("measure", "centroid", "nbr_off", "nbr_idx")


def _case(n=3000, seed=I.SEED_BASE + 0x310):
    v, s = I.kuhn_lattice_tets(3)
    return dict(name="async", mode=B.MODE_3D, sites=I.uniform_sites(n, 3, seed), verts=v, simp=s, f64=False)


@pytest.mark.parametrize("opts", [dict(), dict(learned=1, topk=16), dict(learned=1, split=1)])
def test_async_equals_compute(gpu, opts):
    """vd_compute_async + vd_get_status + vd_get_result give the bytes of vd_compute."""
    w = _case()
    d = B.diagram_from_workload(w, options=opts)
    ref = d.compute()
    d.compute_async()
    assert d.status() == 0
    got = d.get_result()
    for k in KEYS:
        assert torch.equal(ref[k], got[k]), k
    d.close()


def test_async_refuses_untuned_mapping(gpu):
    """mapping = 0 needs the autotuner, which synchronises: the async call refuses
    until a choice is cached, then runs."""
    w = _case()
    d = B.diagram_from_workload(w, options=dict(mapping=0))
    with pytest.raises(B.VDError) as e:
        d.compute_async()
    assert e.value.code == -8
    d.autotune()
    d.compute_async()
    assert d.status() == 0
    d.close()


def test_async_reports_device_error_lazily(gpu):
    """A device-side error of an enqueued compute surfaces in vd_get_status."""
    w = _case()
    d = B.diagram_from_workload(w, options=dict(max_clips=1, mapping=1))
    d.compute_async()
    assert d.status() == -5
    d.close()


def test_async_compute_in_cuda_graph(gpu):
    """The caller captures vd_compute_async into its own CUDA graph on the
    diagram's stream and replays it; each replay's result equals vd_compute's."""
    w = _case()
    s = torch.cuda.Stream()
    sites = torch.tensor(w["sites"], dtype=torch.float32, device="cuda")
    v = torch.tensor(w["verts"], dtype=torch.float32, device="cuda")
    t = torch.tensor(w["simp"], dtype=torch.int32, device="cuda")
    d = B.Diagram(sites, v, t, options=dict(learned=1, topk=16), stream=s)
    with torch.cuda.stream(s):
        ref = d.compute()
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        d.compute_async()
    for _ in range(2):
        with torch.cuda.stream(s):
            g.replay()
        assert d.status() == 0
        got = d.get_result()
        for k in KEYS:
            assert torch.equal(ref[k], got[k]), k
    d.close()


def _trained(d, steps_seed=3):
    d.compute()
    x, y = d.mlp_features()
    d.mlp_init(steps_seed)
    d.mlp_train(x, y, batch=512, epochs=2, lr=1e-3, seed=steps_seed)
    return x, y


def test_model_file_round_trip(gpu, tmp_path):
    """vd_model_save then vd_model_load on another context restores parameters,
    Adam moments and step bit for bit: equal logits, equal learned ranking, and
    training resumes identically."""
    w = _case()
    d1 = B.diagram_from_workload(w)
    x, y = _trained(d1)
    path = str(tmp_path / "net.vdm")
    d1.model_save(path)
    d2 = B.diagram_from_workload(w)
    d2.model_load(path)
    s1, s2 = d1.mlp_get_state(), d2.mlp_get_state()
    for k in ("params", "adam_m", "adam_v"):
        assert torch.equal(s1[k], s2[k]), k
    assert s1["step"] == s2["step"] > 0
    assert torch.equal(d1.mlp_forward(x), d2.mlp_forward(x))
    for d in (d1, d2):
        d.set_options(learned=1, proposal=B.PROPOSAL_MLP, topk=16)
    r1, r2 = d1.compute(), d2.compute()
    assert torch.equal(d1.candidate_masks(), d2.candidate_masks())
    for k in KEYS:
        assert torch.equal(r1[k], r2[k]), k
    # resumed training: one more epoch on each continues from the same step; the
    # weights agree up to the order of the FP32 atomic gradient sums (see vd.h)
    l1 = d1.mlp_train(x, y, batch=512, epochs=1, lr=1e-3, seed=9)
    l2 = d2.mlp_train(x, y, batch=512, epochs=1, lr=1e-3, seed=9)
    t1, t2 = d1.mlp_get_state(), d2.mlp_get_state()
    assert t1["step"] == t2["step"] == s1["step"] + (len(y) + 511) // 512
    assert np.allclose(l1, l2, rtol=1e-5)
    assert torch.allclose(t1["params"], t2["params"], rtol=1e-4, atol=1e-6)
    d1.close()
    d2.close()


def test_model_file_rejects_bad_files(gpu, tmp_path):
    """Missing, truncated, foreign or corrupted files give VD_ERR_IO and leave the
    network as it was."""
    w = _case(n=800)
    d = B.diagram_from_workload(w)
    _trained(d)
    good = str(tmp_path / "good.vdm")
    d.model_save(good)
    before = d.mlp_get_state()
    raw = open(good, "rb").read()
    cases = {"missing": None, "truncated": raw[:-9], "foreign": b"NOTAMODEL" + raw[9:],
             "flipped": raw[:100] + bytes([raw[100] ^ 1]) + raw[101:], "trailing": raw + b"x"}
    for name, data in cases.items():
        p = str(tmp_path / f"{name}.vdm")
        if data is not None:
            open(p, "wb").write(data)
        with pytest.raises(B.VDError) as e:
            d.model_load(p)
        assert e.value.code == -10, name
        after = d.mlp_get_state()
        for k in ("params", "adam_m", "adam_v"):
            assert torch.equal(before[k], after[k]), (name, k)
    assert os.path.getsize(good) == 8 + 16 + 3 * 4 * B.MLP_NPARAM + 8
    d.close()
