"""Train the learned Sinkhorn warm start on the method's own solves and
compare it with the cold start on a larger pair.

  python -m paper_2607_11952_gb300.train_warmstart [--pairs 67 --large-pairs 12
        --outer 30 --epochs 20 --eval-n 20000 --out paper_2607_11952_gb300/gnn_weights.json]

Training pairs: Chung-Lu, n ~ U[2000, 5000], exponent ~ U[2.1, 2.8], edge
noise ~ U[5%, 20%], 64-dim attributes (seed 7), and larger pairs with
n ~ U[10000, 30000] and 64- or 128-dim attributes (seed 8); one sample per
outer iteration (pairs x outer solves, 2010 + 360 by default, spanning all
30 outer iterations of the workloads).  Evaluation: a 20000-node pair with
64-dim attributes; at every outer iteration the same Gibbs kernel is solved
to the marginal tolerance three times (cold start, previous-correction warm
start, learned warm start) and the iterations and times are reported.
"""
from __future__ import annotations

import argparse
import json
import time

import torch

from . import api, gnn, synth


def evaluate(g: synth.GraphPair, model: gnn.WarmStartModel, outer: int = 6,
             tol: float = 1e-4, check_every: int = 5, dtype: str = "bf16",
             max_sweeps: int = 20000):
    G1, G2 = api.Graph(g.n1, g.edges1), api.Graph(g.n2, g.edges2)
    al = api.Aligner(G1, G2, api.Params(dtype=dtype))
    al.node_cost(g.X1, g.X2, g.anchors)
    al.plan_init()
    ws = gnn.WarmStarter(al, "learned", model)
    K0, u0, v0 = torch.empty_like(al.K), torch.empty_like(al.log_u), torch.empty_like(al.log_v)
    warm_p = torch.empty_like(al.log_v)
    rows = []
    from . import _lib as L
    for t in range(outer):
        al.align_iter()
        K0.copy_(al.K)
        u0.copy_(al.log_u)
        v0.copy_(al.log_v)
        warm_l = ws.before_solve()                    # learned warm vector
        L.fa_vec_axpby(al.n2, 1.0, ws.log_v1, 1.0, ws.corr, warm_p)
        res = {}
        for mode, warm in (("cold", None), ("prev", warm_p), ("learned", warm_l)):
            al.K.copy_(K0)
            al.log_u.copy_(u0)
            al.log_v.copy_(v0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fell_back = False
            try:
                it, err, st = al.sinkhorn(max_sweeps, tol, check_every, warm)
            except L.FastAlignError as e:        # cold-start fallback
                if e.status != L.FA_ERR_NUMERIC:
                    raise
                al.log_v.copy_(v0)
                it, err, st = al.sinkhorn(max_sweeps, tol, check_every, None)
                fell_back = True
            torch.cuda.synchronize()
            res[mode] = {"iters": int(it), "ms": (time.perf_counter() - t0) * 1e3,
                         "err": float(err), "status": int(st), "fallback": fell_back}
        ws.after_solve()          # the trajectory continues from the learned solve
        rows.append(res)
    hits = al.hits_mrr(g.test_pairs)
    al.close()
    return rows, hits


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=67)
    ap.add_argument("--outer", type=int, default=30)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--large-pairs", type=int, default=12)
    ap.add_argument("--large-seed", type=int, default=8)
    ap.add_argument("--eval-n", type=int, default=20000)
    ap.add_argument("--eval-outer", type=int, default=30)
    ap.add_argument("--out", default=gnn.WEIGHTS_PATH)
    ap.add_argument("--report", default=None)
    ap.add_argument("--eval-only", action="store_true",
                    help="evaluate the weights in --out without training")
    args = ap.parse_args(argv)

    def log(s):
        print(s, flush=True)

    t0 = t1 = t2 = time.time()
    samples, hist = [], []
    if args.eval_only:
        model = gnn.WarmStartModel.load(args.out)
    else:
        samples = gnn.generate_solves(args.pairs, args.outer, seed=args.seed, log=log)
        if args.large_pairs > 0:
            samples += gnn.generate_solves(args.large_pairs, args.outer, seed=args.large_seed,
                                           log=log, pair_fn=gnn.large_training_pair)
        t1 = time.time()
        log(f"{len(samples)} solves generated in {t1 - t0:.1f} s")
        model, hist = gnn.train(samples, epochs=args.epochs, lr=args.lr, seed=args.seed, log=log)
        t2 = time.time()
        log(f"trained in {t2 - t1:.1f} s")
        model.save(args.out, meta={"pairs": args.pairs, "large_pairs": args.large_pairs,
                                   "large_seed": args.large_seed, "outer": args.outer,
                                   "epochs": args.epochs, "lr": args.lr, "seed": args.seed,
                                   "loss": hist})
    g = synth.config_pair("cl20k", n=args.eval_n)
    rows, hits = evaluate(g, model, outer=args.eval_outer)
    tot = {m: {"iters": sum(r[m]["iters"] for r in rows), "ms": sum(r[m]["ms"] for r in rows)}
           for m in ("cold", "prev", "learned")}
    for t, r in enumerate(rows):
        log(f"outer {t}: " + ", ".join(f"{m} {r[m]['iters']} it {r[m]['ms']:.1f} ms"
                                       for m in ("cold", "prev", "learned")))
    log(f"total: {json.dumps(tot)}  hits {hits}")
    if args.report:
        json.dump({"train_loss": hist, "eval": rows, "total": tot, "hits": hits,
                   "n_samples": len(samples), "gen_s": t1 - t0, "train_s": t2 - t1},
                  open(args.report, "w"), indent=1)


if __name__ == "__main__":
    main()
