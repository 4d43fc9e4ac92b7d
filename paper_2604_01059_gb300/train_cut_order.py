"""Train the cut-order network and write its weights next to this file.

    python -m paper_2604_01059_gb300.train_cut_order [--dataset PATH] [--epochs N] ...

Training data: marginal diagrams of seeded random Clifford+T circuits with 20
to 80 T/T_DAG gates, each labelled with the exact stabilizer-term counts the
compiler measures when a candidate spider is cut first (written by
``tsim_cut_dataset``; the file is reused when it exists).  Training runs the
library's CUDA kernels (BF16 weights, FP32 accumulation, Adam).  Output:
``cut_order.f32`` (the parameter vector, little-endian float32, in the layout
``tsim_cut_num_params`` documents) and ``cut_order.json`` (how it was made).
``--evaluate PATH`` reports the ranking quality of the weights on a held-out
dataset; ``--policy N`` compares, on N held-out graphs drawn like the
training ones (data seed + 1), the term counts of the compiler's LEARNED
policy with the weights against the heuristic order that judges it, a
random first cut and the best first cut.
"""
import argparse
import json
import os
import time

import numpy as np

from . import (read_cut_dataset, tsim_cut_dataset, tsim_cut_init_params, tsim_cut_loss_grad, tsim_cut_num_params,
               tsim_cut_train)

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "cut_order.f32")


def load_weights(path=WEIGHTS):
    """The trained parameter vector (float32), or None when absent."""
    if not os.path.exists(path):
        return None
    p = np.fromfile(path, dtype="<f4")
    if p.size != tsim_cut_num_params():
        raise ValueError(f"{path}: {p.size} parameters, the library expects {tsim_cut_num_params()}")
    return p


def evaluate(params, dataset_path):
    """Ranking quality on a dataset: per graph with two or more labelled
    spiders, the term count (log2) of the spider the network ranks first
    against the mean over the labelled spiders (a random first cut) and the
    best one; scores come from the library's CUDA forward pass."""
    from . import tsim_cut_forward
    x, rp, col, y, go = read_cut_dataset(dataset_path)
    s = tsim_cut_forward(params, x, rp, col)
    top, rnd, best, hits, n = [], [], [], 0, 0
    for g in range(len(go) - 1):
        idx = np.arange(go[g], go[g + 1])
        lab = idx[~np.isnan(y[idx])]
        if len(lab) < 2:
            continue
        n += 1
        pick = lab[np.argmin(s[lab])]
        top.append(float(y[pick]))
        rnd.append(float(np.mean(y[lab])))
        best.append(float(np.min(y[lab])))
        hits += int(y[pick] == np.min(y[lab]))
    top, rnd, best = np.array(top), np.array(rnd), np.array(best)
    return {"graphs": n, "top_ranked_log2_terms": float(top.mean()), "random_log2_terms": float(rnd.mean()),
            "best_log2_terms": float(best.mean()), "top_is_best": hits / max(n, 1),
            "terms_ratio_random_over_top": float(np.mean(2.0 ** (rnd - top))),
            "terms_ratio_top_over_best": float(np.mean(2.0 ** (top - best)))}


def policy_report(params, n_graphs, seed, t_min, t_max, budget):
    """LEARNED against the heuristic on held-out graphs (tsim_cut_evaluate)."""
    from . import tsim_cut_evaluate, tsim_cut_model_set
    tsim_cut_model_set(params)
    try:
        r = tsim_cut_evaluate(seed, n_graphs, t_min, t_max, budget)
    finally:
        tsim_cut_model_set(None)
    heur, learned, rnd, best = (np.log2(np.maximum(r[:, k], 1.0)) for k in (1, 2, 3, 4))
    return {"graphs": int(n_graphs), "seed": int(seed), "budget": int(budget),
            "mean_log2_terms": {"heuristic": float(heur.mean()), "learned": float(learned.mean()),
                                "random_first_cut": float(rnd.mean()), "best_first_cut": float(best.mean())},
            "total_terms": {"heuristic": float(r[:, 1].sum()), "learned": float(r[:, 2].sum()),
                            "best_first_cut": float(r[:, 4].sum())},
            "learned_fewer": int((r[:, 2] < r[:, 1]).sum()), "learned_equal": int((r[:, 2] == r[:, 1]).sum()),
            "learned_more": int((r[:, 2] > r[:, 1]).sum()),
            "best_first_cut_fewer_than_heuristic": int((r[:, 4] < r[:, 1]).sum())}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--dataset", default=None, help="dataset file (generated when missing)")
    ap.add_argument("--graphs", type=int, default=2000)
    ap.add_argument("--t-min", type=int, default=20)
    ap.add_argument("--t-max", type=int, default=80)
    ap.add_argument("--budget", type=int, default=1024, help="term budget of one label")
    ap.add_argument("--candidates", type=int, default=8, help="labelled spiders per graph")
    ap.add_argument("--data-seed", type=int, default=0)
    ap.add_argument("--epochs", type=int, default=150)
    ap.add_argument("--batch", type=int, default=32, help="graphs per minibatch")
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--evaluate", default=None, help="held-out dataset: report the ranking quality of --out")
    ap.add_argument("--policy", type=int, default=0, help="held-out graphs for the LEARNED-vs-heuristic report")
    a = ap.parse_args(argv)
    if a.evaluate or a.policy:
        rep = {}
        if a.evaluate:
            rep["ranking"] = evaluate(load_weights(a.out), a.evaluate)
        if a.policy:
            rep["policy"] = policy_report(load_weights(a.out), a.policy, a.data_seed + 1, a.t_min, a.t_max,
                                          a.budget)
        print(json.dumps(rep))
        return
    ds = a.dataset or os.path.join(os.path.dirname(os.path.abspath(a.out)), "cut_order_dataset.bin")
    t0 = time.time()
    reused = os.path.exists(ds)
    if not reused:
        tsim_cut_dataset(a.data_seed, a.graphs, a.t_min, a.t_max, a.budget, a.candidates, ds)
    t_data = None if reused else round(time.time() - t0, 1)
    x, rp, col, y, go = read_cut_dataset(ds)
    lab = ~np.isnan(y)
    p0 = tsim_cut_init_params(a.seed)
    L0, _ = tsim_cut_loss_grad(p0, x, rp, col, y, go)
    t1 = time.time()
    p, hist = tsim_cut_train(ds, p0, epochs=a.epochs, batch_graphs=a.batch, lr=a.lr, seed=a.seed)
    t_train = time.time() - t1
    L1, _ = tsim_cut_loss_grad(p, x, rp, col, y, go)
    p.astype("<f4").tofile(a.out)
    rec = {
        "dataset": {"graphs": int(len(go) - 1), "nodes": int(len(rp) - 1), "labelled": int(lab.sum()),
                    "t_min": a.t_min, "t_max": a.t_max, "budget": a.budget, "candidates": a.candidates,
                    "seed": a.data_seed, "seconds": t_data, "reused_file": reused},
        "training": {"epochs": a.epochs, "batch_graphs": a.batch, "lr": a.lr, "seed": a.seed,
                     "seconds": round(t_train, 2), "loss_init": L0, "loss_final": L1,
                     "loss_per_epoch": [round(float(v), 5) for v in hist]},
    }
    with open(os.path.splitext(a.out)[0] + ".json", "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps({k: v for k, v in rec["training"].items() if k != "loss_per_epoch"}))


if __name__ == "__main__":
    main()
