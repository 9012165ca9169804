"""Write tests/golden/nnz.json: exact (ray, voxel) nonzero counts of the projector per
multigrid level of each workload, counted by the FP64 oracle (calls only oracle/).

    python tests/golden/make_nnz.py

The counts are the algorithmic work units of the projector and of its adjoint (one
intersection length per nonzero); the benchmark divides them by kernel times.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402


def main():
    out = {}
    for name in ("small", "medium", "large", "large30", "large20"):
        cfg = synth.CONFIGS[name]
        g = synth.geometry_for(cfg)
        per_level = []
        for level in range(cfg["levels"]):
            lg = oracle.level_geom(g, level)
            per_level.append(dict(level=level, nnz=oracle.count_nnz(lg),
                                  vol=[lg["nx"], lg["ny"], lg["nz"]],
                                  det=[len(lg["angles"]), lg["nv"], lg["nu"]]))
        out[name] = per_level
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "nnz.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
