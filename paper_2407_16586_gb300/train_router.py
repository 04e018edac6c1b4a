"""Train the block router on seeded 30-80-atom clusters and write its weights.

  python -m paper_2407_16586_gb300.train_router [--clusters 200] [--stride 40]
         [--out paper_2407_16586_gb300/data/router.bin]

Every cluster comes from synth.router_cluster(i) (seed 20240716 + i); every
stride-th screened quartet tile of each is evaluated in fp64 and fp32
(tg_tile_samples), the MLP is trained on the GPU (tg_router_train) and the
margin / eps_rel calibration is taken on 20 % held-out tiles; the margin is
then lowered on a budget set (--budget-clusters clusters and --budget-chains
chains) while the measured error of the whole mixed route stays within a
fifth of mixed_tol (router.calibrate_budget).  --recalibrate FILE keeps FILE's network and
redoes only that last step."""
import argparse
import json
import os
import time

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--clusters", type=int, default=200)
    ap.add_argument("--first", type=int, default=0)
    ap.add_argument("--stride", type=int, default=40)
    ap.add_argument("--cap", type=int, default=20000)
    ap.add_argument("--epochs", type=int, default=600)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "router.bin"))
    ap.add_argument("--budget-clusters", type=int, default=2)
    ap.add_argument("--budget-natom", type=int, default=24)
    ap.add_argument("--budget-chains", type=int, default=2, help="20-atom chains added to the budget set")
    ap.add_argument("--budget-first", type=int, default=100000, help="first cluster index of the budget set")
    ap.add_argument("--recalibrate", default=None, help="router file whose network is kept")
    ap.add_argument("--budget-c4-nranks", type=int, default=200,
                    help="add pair-key shard 0 of this many of the 300-atom cluster to the budget set (0: none)")
    ap.add_argument("--safety", type=float, default=2.0)
    args = ap.parse_args()
    from paper_2407_16586_gb300 import build
    build.build()
    import paper_2407_16586_gb300 as tg
    from paper_2407_16586_gb300 import router, synth
    t0 = time.time()
    # budget set: compact clusters and chains (seeds unrelated to the workloads)
    budget_set = [synth.router_cluster(i, natom=args.budget_natom)
                  for i in range(args.budget_first, args.budget_first + args.budget_clusters)]
    budget_set += [synth.molecule(args.budget_first + i, 8, 12) for i in range(args.budget_chains)]
    shards = [None] * len(budget_set)
    if args.budget_c4_nranks > 0:
        budget_set.append(synth.config(3))
        shards.append((0, args.budget_c4_nranks))
    budget_desc = ("router_cluster(%d..%d, natom=%d) + molecule(%d..%d, 8, 12)%s; safety %g" % (
        args.budget_first, args.budget_first + args.budget_clusters - 1, args.budget_natom, args.budget_first,
        args.budget_first + args.budget_chains - 1,
        " + c4 pair-key shard 0/%d" % args.budget_c4_nranks if args.budget_c4_nranks > 0 else "", args.safety))
    if args.recalibrate:
        r = tg.Router(path=args.recalibrate)
        info = dict(recalibrated_from=os.path.basename(args.recalibrate), budget_set=budget_desc)
        info["budget_log"] = router.calibrate_budget(r, budget_set, safety=args.safety, shards=shards)
        info["margin"] = float(r.get()[3][0])
        r.save(args.out)
        with open(args.out + ".json", "w") as f:
            json.dump(info, f, indent=1)
        print(json.dumps(info))
        return
    Xs, ys, es = [], [], []
    for i in range(args.first, args.first + args.clusters):
        s = synth.router_cluster(i)
        X, y, e = router.collect([s], stride=args.stride, cap=args.cap)
        Xs.append(X)
        ys.append(y)
        es.append(e)
    X, y, e = np.concatenate(Xs), np.concatenate(ys), np.concatenate(es)
    t1 = time.time()
    r, info = router.fit(X, y, e, epochs=args.epochs)
    info["budget_set"] = budget_desc
    info["budget_log"] = router.calibrate_budget(r, budget_set, safety=args.safety, shards=shards)
    info["margin"] = float(r.get()[3][0])
    r.save(args.out)
    info.update(clusters=args.clusters, stride=args.stride, tiles=int(len(y)), sample_s=t1 - t0,
                train_s=time.time() - t1)
    with open(args.out + ".json", "w") as f:
        json.dump(info, f, indent=1)
    print(json.dumps(info))


if __name__ == "__main__":
    main()
