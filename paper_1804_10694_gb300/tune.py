"""Tile-choice tuning pipeline: autotune a training set of shapes, train the
MLP cost model on the GPU from those timings, and measure on held-out shapes
how far the model's pick (and the built-in heuristic's pick) is from the
exhaustive autotuner's best -- the regret -- and how much tuning time the
model saves.  The paper tunes tile sizes by search (Section VI-A); this is
that search, its learned replacement and the comparison between them.

    python -m paper_1804_10694_gb300.tune --out-dir DIR [--train 700]
        [--heldout 100] [--reps 5] [--epochs 6000] [--mode bf16x3[,bf16x6,...]]
        [--reuse-timings DIR2]

Writes DIR/timings_train.csv, DIR/timings_heldout.csv, DIR/costmodel.txt and
DIR/regret.json.  Several modes (comma-separated) train one model on all of
their timings (the mode is one of its features); regret is reported per
mode.  With --reuse-timings the timing rows of DIR2 are copied and only the
modes missing from them are measured.
"""
from __future__ import annotations

import argparse
import csv
import json
import os
import sys
import time

import numpy as np

import paper_1804_10694_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CONV_SHAPES = ((50176, 64, 576), (12544, 128, 1152), (3136, 256, 2304))


def read_table(path, mode=None):
    """{(M, N, K): {config_id: median ms}} of one mode (all rows if None)."""
    table = {}
    want = None if mode is None else pkg.MODES[mode]
    with open(path) as f:
        for r in csv.DictReader(f):
            if want is not None and int(r["mode"]) != want:
                continue
            key = (int(r["M"]), int(r["N"]), int(r["K"]))
            table.setdefault(key, {})[int(r["config_id"])] = float(r["median_ms"])
    return table


def modes_in(path):
    if not os.path.exists(path):
        return set()
    with open(path) as f:
        return {int(r["mode"]) for r in csv.DictReader(f)}


def effective_key(mode, cid, M, N, K):
    c = pkg.config_get(mode, cid)
    chunk = 32 if mode == "tf32x3" else 64
    chunks = max(1, -(-K // chunk))
    sk = max(1, min(c["split_k"], chunks))
    per = -(-chunks // sk)
    sk = -(-chunks // per)
    tiles_m = -(-M // (128 * c["cluster"]))   # a CTA pair's tile is 256 rows
    return (c["block_n"], sk, min(c["kb"], per), max(1, min(c["group_m"], tiles_m)), c["fused"],
            c["cluster"])


def timed_choice(times, mode, cid, shape):
    """Measured time of configuration cid on the shape: the tuner timed one
    representative of each distinct effective configuration."""
    if cid in times:
        return times[cid]
    want = effective_key(mode, cid, *shape)
    for other, t in times.items():
        if effective_key(mode, other, *shape) == want:
            return t
    raise KeyError((shape, cid))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out-dir", required=True)
    ap.add_argument("--mode", default="bf16x3",
                    help="tensor-core mode(s), comma-separated: bf16x3, tf32x3, bf16x6")
    ap.add_argument("--train", type=int, default=700)
    ap.add_argument("--heldout", type=int, default=100)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--epochs", type=int, default=6000)
    ap.add_argument("--seed", type=int, default=2024)
    ap.add_argument("--reuse-timings", default=None,
                    help="directory with timings_train.csv and timings_heldout.csv to reuse")
    args = ap.parse_args(argv)
    modes = [m.strip() for m in args.mode.split(",") if m.strip()]
    for m in modes:
        if m not in ("bf16x3", "tf32x3", "bf16x6"):
            ap.error(f"unknown mode {m}")

    import workloads as W
    os.makedirs(args.out_dir, exist_ok=True)
    tpath = os.path.join(args.out_dir, "timings_train.csv")
    hpath = os.path.join(args.out_dir, "timings_heldout.csv")
    mpath = os.path.join(args.out_dir, "costmodel.txt")
    for p in (tpath, hpath):
        if os.path.exists(p):
            os.remove(p)
    train = W.training_shapes(args.train, seed=args.seed)
    held = list(CONV_SHAPES) + W.training_shapes(args.heldout, seed=args.seed + 1)

    t_train, per_shape_s = {}, {}
    if args.reuse_timings:
        import shutil
        shutil.copyfile(os.path.join(args.reuse_timings, "timings_train.csv"), tpath)
        shutil.copyfile(os.path.join(args.reuse_timings, "timings_heldout.csv"), hpath)
    have = modes_in(tpath) & modes_in(hpath)
    for mode in modes:
        if pkg.MODES[mode] in have:
            continue
        t0 = time.time()
        pkg.autotune(train, mode=mode, reps=args.reps, out_path=tpath)
        t_train[mode] = time.time() - t0
        per_shape_s[mode] = []
        for s in held:
            t1 = time.time()
            pkg.autotune([s], mode=mode, reps=args.reps, out_path=hpath)
            per_shape_s[mode].append(time.time() - t1)
    t2 = time.time()
    loss = pkg.costmodel_train(tpath, epochs=args.epochs, seed=args.seed, out_model=mpath)
    t_fit = time.time() - t2

    with open(tpath) as f:
        n_train_rows = sum(1 for _ in csv.DictReader(f))
    report = {
        "modes": modes,
        "training_shapes": len(train),
        "training_timings": n_train_rows,
        "heldout_shapes": len(held),
        "epochs": args.epochs,
        "final_train_mse_normalised": loss,
        "autotune_train_seconds": t_train,
        "fit_seconds": t_fit,
        "per_mode": {},
    }
    for mode in modes:
        table = read_table(hpath, mode)
        rows = []
        pred_s = []
        for s in held:
            times = table[tuple(s)]
            best = min(times.values())
            t3 = time.time()
            cid_model, pred_ms = pkg.costmodel_predict(*s, mode)
            pred_s.append(time.time() - t3)
            cid_default = pkg.config_default(mode, *s)
            rows.append({
                "shape": list(s),
                "best_ms": best,
                "model_ms": timed_choice(times, mode, cid_model, s),
                "model_pred_ms": pred_ms,
                "default_ms": timed_choice(times, mode, cid_default, s),
                "model_config": pkg.config_get(mode, cid_model),
                "default_config": pkg.config_get(mode, cid_default),
            })
        for r in rows:
            r["model_regret"] = r["model_ms"] / r["best_ms"] - 1.0
            r["default_regret"] = r["default_ms"] / r["best_ms"] - 1.0
        mr = np.array([r["model_regret"] for r in rows])
        dr = np.array([r["default_regret"] for r in rows])
        ps = per_shape_s.get(mode)
        report["per_mode"][mode] = {
            "exhaustive_seconds_per_heldout_shape_mean": float(np.mean(ps)) if ps else None,
            "model_predict_seconds_mean": float(np.mean(pred_s)),
            "model_regret_mean": float(mr.mean()),
            "model_regret_median": float(np.median(mr)),
            "model_regret_max": float(mr.max()),
            "default_regret_mean": float(dr.mean()),
            "default_regret_median": float(np.median(dr)),
            "default_regret_max": float(dr.max()),
            "conv_shapes": [r for r in rows if tuple(r["shape"]) in CONV_SHAPES],
            "per_shape": rows,
        }
    with open(os.path.join(args.out_dir, "regret.json"), "w") as f:
        json.dump(report, f, indent=1)
    print(json.dumps({k: (v if k != "per_mode" else
                          {m: {a: b for a, b in pm.items() if a not in ("per_shape", "conv_shapes")}
                           for m, pm in v.items()})
                      for k, v in report.items()}, indent=1))


if __name__ == "__main__":
    main()
