"""Writes the stored expected values under tests/golden/ from the FP64
oracle alone (oracle/fastalign_ref.py); no value here comes from the CUDA
path.  The paper prints no worked example, so these fixtures are oracle
regression values on a hand-written instance, not values from the paper.

  python tests/golden/make_golden.py        # rewrites tiny_pair.txt

Instance (stated in full below): G1 is a 7-node graph, a 4-cycle 0-1-2-3
with a chord 0-2, a tail 3-4-5 and a pendant 6 on node 1; G2 is G1
relabelled by PERM with the chord 0-2 replaced by the edge 4-6 (in G1's
labels); 3-dim attributes X1 by hand and X2 = X1 relabelled plus a fixed
perturbation; two anchors.  Outputs (Algorithm 1 with the oracle's
default parameters): C_node after propagation (Algorithm 1, Phase 1), log S after
one outer iteration of 30 Sinkhorn iterations and after three (Eq. 3-4),
and the top-1 column of every row of the final plan.
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import fastalign_ref as R  # noqa: E402

N = 7
EDGES1 = np.array([[0, 1], [1, 2], [2, 3], [3, 0], [0, 2], [3, 4], [4, 5], [1, 6]])
PERM = np.array([3, 0, 6, 2, 5, 1, 4])          # node i of G1 is node PERM[i] of G2
EDGES2_G1_LABELS = np.array([[0, 1], [1, 2], [2, 3], [3, 0], [4, 6], [3, 4], [4, 5], [1, 6]])
X1 = np.array([[0.9, -0.2, 0.4], [-0.5, 0.8, 0.1], [0.3, 0.3, -0.9], [-0.7, -0.6, 0.2],
               [0.1, 0.9, 0.6], [0.8, 0.1, -0.3], [-0.2, -0.8, -0.5]])
DX = np.array([[0.05, -0.02, 0.01], [-0.03, 0.04, 0.0], [0.02, 0.0, -0.04], [0.0, 0.03, 0.02],
               [-0.04, 0.01, 0.03], [0.01, -0.05, 0.0], [0.03, 0.02, -0.01]])
ANCHORS_G1 = np.array([0, 4])
N_SINK = 30


def instance():
    edges2 = PERM[EDGES2_G1_LABELS]
    X2 = np.empty_like(X1)
    X2[PERM] = X1 + DX
    anchors = np.stack([ANCHORS_G1, PERM[ANCHORS_G1]], axis=1)
    return EDGES1, edges2, X1, X2, anchors


def compute() -> dict:
    e1, e2, x1, x2, anchors = instance()
    p = R.Params()
    ph = R.phase1(N, N, e1, e2, x1, x2, anchors, p)
    one = R.fastalign(N, N, e1, e2, x1, x2, anchors, p, 1, N_SINK, ph=ph)
    three = R.fastalign(N, N, e1, e2, x1, x2, anchors, p, 3, N_SINK, ph=ph)
    top1 = R.topk(np.exp(three["logS"]), 1)[:, 0]
    return {"C_node": ph.C_node, "logS_1": one["logS"], "logS_3": three["logS"],
            "top1": top1.astype(np.int64)}


def render(vals: dict) -> str:
    out = ["# Oracle regression fixture (not a value from the paper, which prints no",
           "# worked example): written by tests/golden/make_golden.py from",
           "# oracle/fastalign_ref.py, Algorithm 1 with the default parameters,",
           f"# Eq. 3 with {N_SINK} iterations per outer iteration, Eq. 4 for the plan.",
           "# Instance: see make_golden.py.  One block per quantity: a header line",
           "# '@ name rows cols', then the rows."]
    for name in ("C_node", "logS_1", "logS_3", "top1"):
        a = np.atleast_2d(vals[name])
        if name == "top1":
            a = a.reshape(1, -1)
        out.append(f"@ {name} {a.shape[0]} {a.shape[1]}")
        for row in a:
            out.append(" ".join(str(int(x)) if name == "top1" else f"{x:.17g}" for x in row))
    return "\n".join(out) + "\n"


def parse(text: str) -> dict:
    vals, name, rows = {}, None, []
    for line in text.splitlines():
        if not line or line.startswith("#"):
            continue
        if line.startswith("@"):
            if name:
                vals[name] = np.array(rows)
            _, name, _, _ = line.split()
            rows = []
        else:
            rows.append([float(x) for x in line.split()])
    vals[name] = np.array(rows)
    vals["top1"] = vals["top1"].reshape(-1).astype(np.int64)
    return vals


if __name__ == "__main__":
    with open(os.path.join(HERE, "tiny_pair.txt"), "w") as f:
        f.write(render(compute()))
