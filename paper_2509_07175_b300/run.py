"""Compute the diagram of one seeded workload and print its timings and counters.

    python -m paper_2509_07175_b300.run --workload shell --form learned --repeat 3

--form plain      the paper's search alone (Sec. 3.2 / 5.1)
--form learned    the learned form, ranking by distance or by the network
                  (--proposal mlp trains it first on labels from plain computes
                  of seeded 100k-site cube instances, --train-epochs epochs)
--mapping 0|1|2   clip kernel: autotuned, warp per pair, thread per pair
--split           3D: interior sites' cells computed whole after the boundary
                  pass (Alg. 5); the others per tetrahedron

One JSON line per compute: phase times (CUDA events), clip-kernel mapping and
the work counters.  Every compute runs the whole path through the C ABI.
"""
from __future__ import annotations

import argparse
import json

from . import binding as B
from . import inputs as I


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--workload", default="cube",
                    choices=["square", "cube", "cube1m", "cube2m", "shell", "torus", "box", "box5m", "grid5m"])
    ap.add_argument("--n", type=int, default=None, help="sites (default: the workload's own)")
    ap.add_argument("--form", default="learned", choices=["plain", "learned"])
    ap.add_argument("--proposal", default="distance", choices=["distance", "mlp"])
    ap.add_argument("--topk", type=int, default=24)
    ap.add_argument("--mapping", type=int, default=1, choices=[0, 1, 2])
    ap.add_argument("--chunk", type=int, default=1)
    ap.add_argument("--train-epochs", type=int, default=None)
    ap.add_argument("--split", action="store_true")
    ap.add_argument("--repeat", type=int, default=1)
    args = ap.parse_args(argv)

    w = I.workload(args.workload, args.n)
    d = B.diagram_from_workload(w)
    prop = B.PROPOSAL_DISTANCE
    if args.form == "learned" and args.proposal == "mlp":
        from . import learned as L
        x, y = L.training_set()
        kw = {} if args.train_epochs is None else {"epochs": args.train_epochs}
        tr = L.train(x, y, **kw)
        L.load_state(d, tr["state"])
        prop = B.PROPOSAL_MLP
        print(json.dumps({"training": {"rows": tr["rows"], "epochs": tr["epochs"], "train_s": tr["train_s"],
                                       "loss": tr["epoch_loss"][-1]}}), flush=True)
    d.set_options(learned=int(args.form == "learned"), topk=args.topk, proposal=prop, mapping=args.mapping,
                  chunk=args.chunk, stats=1, timing=1, split=int(args.split))
    for k in range(args.repeat):
        r = d.compute()
        s = r["stats"]
        print(json.dumps({"workload": args.workload, "n": len(w["sites"]), "form": args.form,
                          "proposal": args.proposal if args.form == "learned" else None, "step": k,
                          "status": r["status"], "phase_ms": r["phase_ms"],
                          "mapping": s["mapping"], "chunk": s["chunk"],
                          "stats": {key: s[key] for key in ("pairs", "nonempty", "nn_queries", "corner_tests",
                                                            "clips", "search_steps", "sites_scanned",
                                                            "learned_hits", "list_tests", "fp64", "uncertain",
                                                            "whole_cells", "boundary_sites")}}),
              flush=True)
    d.close()


if __name__ == "__main__":
    main()
