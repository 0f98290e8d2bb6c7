"""Run one kernel case a few times, for profilers (ncu) and quick timing.

    python profile_case.py <case> [--reps R]

Cases (synthetic inputs from `synth`):
  forward-xgb        qts_shap_values on the 1,000-tree depth-8 ensemble, M = 10,000
  adjoint-xgb        qts_shap_backward on the same
  interactions-500   qts_shap_interactions on the 500-tree depth-6 ensemble, F = 30, M = 2,000
  fused-xgb          qts_batched_fwd_bwd with the depth-8 ensemble as a single request
  fused-deep         qts_batched_fwd_bwd, one request shaped like the heaviest member of the
                     64-ensemble batch (depth 14, F = 57), 60 trees, M = 4,096
  adjoint-deep       qts_shap_backward on the same
  interactions3-500  qts_shap_interactions3 (third order) on the 500-tree depth-6 ensemble
  forward-adultlike  qts_shap_values on a Table-1-shaped stand-in for the paper's Adult-large
                     model (1,000 trees, depth 16, F = 14, ~610 leaves per tree), 1,000 rows
  forward-deep20     qts_shap_values on 200 unbalanced trees of depth <= 20 over F = 24
                     (repeated features merged), M = 5,000
  orders-covtypelike qts_shap_interactions_order on 800 trees of depth 16 over F = 54 (a
                     CovType-large-shaped stand-in): orders 2-6 for 1 row, 2-4 for 64
  alg1-xgb, alg1-deep20, alg1-adultlike
                     qts_shap_values_alg1 (depth-first form) on the same inputs as
                     forward-xgb, forward-deep20 and forward-adultlike
  batch64            qts_batched_fwd_bwd on the benchmark's 64-ensemble batch (one
                     graph launch per call; the bench's default parameters)
Prints the median CUDA-event time per call and the algorithmic FP32-pipe
operation rate (4 ops per sample x element x node forward, 11 adjoint/fused;
4 per sample x edge x node for the depth-first form).
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    import torch

    import synth
    import paper_2605_04497_gb300 as qts

    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["forward-xgb", "adjoint-xgb", "interactions-500", "fused-xgb",
                                     "fused-deep", "adjoint-deep", "interactions3-500",
                                     "forward-adultlike", "forward-deep20", "alg1-xgb", "alg1-deep20",
                                     "alg1-adultlike", "orders-covtypelike", "batch64"])
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    if args.case == "orders-covtypelike":
        return orders_case(args.reps)
    if args.case == "batch64":
        return batch64_case(args.reps)
    if args.case.endswith("-deep"):
        seed = synth.SEED_BASE + 4
        trees, depth, feats, samples = synth.batch_draw(seed, 64)
        e = int(np.argmax(trees * samples * 2.0 ** np.minimum(depth, 14)))
        es = seed * 1000 + e
        F = int(feats[e])
        ens = synth.grow(es, 60, int(depth[e]), F, int(min(100000, 20 * 2 ** int(depth[e]))), 0.1, min_rows=5)
        w = synth.Workload("deep", ens, synth.normal(es, synth.STREAM_X, (4096, F)),
                           synth.normal(es, synth.STREAM_GRAD, (4096, F + 1)))
    elif args.case in ("forward-adultlike", "alg1-adultlike"):
        seed = synth.SEED_BASE + 100
        ens = synth.grow(seed, 1000, 16, 14, 1850, 0.1, min_rows=5)
        w = synth.Workload("adultlike", ens, synth.normal(seed, synth.STREAM_X, (1000, 14)),
                           synth.normal(seed, synth.STREAM_GRAD, (1000, 15)))
    elif args.case in ("forward-deep20", "alg1-deep20"):
        w = synth.workload("deep-depth20", with_grad=True)
    else:
        w = synth.workload("pairs-depth6" if args.case.startswith("interactions") else "xgb-depth8",
                           with_grad=True)
    E = qts.Ensemble.from_arrays(w.ens)
    info = E.info()
    X = torch.from_numpy(w.X).cuda()
    G = torch.from_numpy(w.grad_phi).cuda()
    phi = torch.empty((w.M, w.F + 1), dtype=torch.float64, device="cuda")
    dl = torch.empty(E.n_nodes, dtype=torch.float64, device="cuda")
    dz = torch.empty(E.n_nodes, dtype=torch.float64, device="cuda")
    reqs = qts.make_requests([dict(ens=E, X=X, grad_phi=G, phi=phi, d_leaf=dl, d_z=dz)])
    fn, ops = {
        "forward-xgb": (lambda: qts.shap_values(E, X, 8, out=phi), 4),
        "adjoint-xgb": (lambda: qts.shap_backward(E, X, G, 8), 11),
        "interactions-500": (lambda: qts.shap_interactions(E, X, 8), 0),
        "fused-xgb": (lambda: qts.batched_fwd_bwd(reqs, 8), 11),
        "fused-deep": (lambda: qts.batched_fwd_bwd(reqs, 8), 11),
        "adjoint-deep": (lambda: qts.shap_backward(E, X, G, 8), 11),
        "interactions3-500": (lambda: qts.shap_interactions3(E, X, 8), 0),
        "forward-adultlike": (lambda: qts.shap_values(E, X, 8, out=phi), 4),
        "forward-deep20": (lambda: qts.shap_values(E, X, 8, out=phi), 4),
        "alg1-xgb": (lambda: qts.shap_values_alg1(E, X, 8, out=phi), -4),
        "alg1-deep20": (lambda: qts.shap_values_alg1(E, X, 8, out=phi), -4),
        "alg1-adultlike": (lambda: qts.shap_values_alg1(E, X, 8, out=phi), -4),
    }[args.case]
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(args.reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    E.sync_status()
    ms = float(np.median(ts))
    # path form: ops per (sample, merged element, node); depth-first form
    # (negative): ops per (sample, edge, node), edges = nodes - trees
    units = info["sum_unique"] if ops >= 0 else (E.n_nodes - w.ens.n_trees)
    work = abs(ops) * 8 * units * w.M
    print(f"{args.case}: paths {info['n_paths']}, buckets {info['buckets']}")
    print(f"{args.case}: {ms:.3f} ms/call, {w.M * w.ens.n_trees / ms * 1e3:.3e} sample*trees/s"
          + (f", {work / ms / 1e9:.2f} Tops/s algorithmic" if ops else ""))
    E.close()


def batch64_case(reps):
    """The 64-ensemble batch: one batched call to warm up, then `reps` calls."""
    import torch

    import synth
    import paper_2605_04497_gb300 as qts

    works = synth.batch_config()
    ens = [qts.Ensemble.from_arrays(w.ens) for w in works]
    items = [dict(ens=e, X=torch.from_numpy(w.X).cuda(), grad_phi=torch.from_numpy(w.grad_phi).cuda(),
                  phi=torch.empty((w.M, w.F + 1), dtype=torch.float64, device="cuda"),
                  d_leaf=torch.empty(e.n_nodes, dtype=torch.float64, device="cuda"),
                  d_z=torch.empty(e.n_nodes, dtype=torch.float64, device="cuda")) for e, w in zip(ens, works)]
    reqs = qts.make_requests(items)
    qts.batched_fwd_bwd(reqs)
    torch.cuda.synchronize()
    for _ in range(reps):
        qts.batched_fwd_bwd(reqs)
        torch.cuda.synchronize()
        print(f"batch64: persistent kernels {qts.batched_last_kernel_ms():.1f} ms, "
              f"{qts.batched_kernel_count()} launches per call")
    for e in ens:
        e.sync_status()
        e.close()


def orders_case(reps):
    """Interactions of orders 2-6 on a stand-in for the paper's CovType-large
    model (Table 1: depth 16, F = 54, up to 14 unique features per path), with
    800 trees instead of 8,000, for one explained row (as in Table 4; orders
    2-6) and for 64 rows (orders 2-4)."""
    import math

    import torch

    import synth
    import paper_2605_04497_gb300 as qts

    seed = synth.SEED_BASE + 101
    ens = synth.grow(seed, 800, 16, 54, 20000, 0.1, min_rows=5)
    E = qts.Ensemble.from_arrays(ens)
    info = E.info()
    print(f"orders-covtypelike: {ens.n_trees} trees, paths {info['n_paths']}, max unique {info['max_unique']}")
    X = torch.from_numpy(synth.normal(seed, synth.STREAM_X, (64, 54))).cuda()
    for rows, orders in ((1, range(2, 7)), (64, range(2, 5))):
        for order in orders:
            fn = lambda: qts.shap_interactions_order(E, X[:rows], order)
            fn()
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                fn()
                b.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            E.sync_status()
            print(f"orders-covtypelike: rows {rows}, order {order}: {float(np.median(ts)):.3f} ms/call, "
                  f"{math.comb(54, order)} subsets per row")
    E.close()


if __name__ == "__main__":
    main()
