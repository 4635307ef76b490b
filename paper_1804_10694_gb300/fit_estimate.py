"""Fit the constants of the built-in tile-choice estimate (default_config in
csrc/runtime.cpp) to exhaustive autotuner timings.

    python -m paper_1804_10694_gb300.fit_estimate TRAIN.csv [MORE.csv ...]
        [--heldout HELD.csv] [--samples 8000] [--seed 3]

The estimate of a packed candidate (128 x 64 or 128 x 128 tiles on one SM,
256 x 256 on a CTA pair; 1-8 splits) is

    waves x (a0 + per x chunk[tile] x (six if BF16x6) + epi[tile])
        + [splits > 1] (fix0 + fix1 x M N splits / 1e6),

waves = ceil(tiles x splits / slots), per = k-chunks a split.  The search
draws `--samples` constant sets from a grid, keeps the one with the lowest
sum over the timed modes of the mean regret over their shapes (regret = time of the
pick / time of the fastest timed configuration - 1, the pick mapped onto the
timed representative of its effective configuration as the autotuner times
each distinct one once), then refines it one constant at a time.  Prints the
constants (to be copied into runtime.cpp) and the regret on the training and
held-out timings.
"""
from __future__ import annotations

import argparse
import csv
import itertools
import json
import random
from collections import defaultdict

SPLITS = (1, 2, 3, 4, 6, 8)
KEYS = ("chunk128", "chunk_pair", "epi64", "epi128", "epi_pair", "a0", "fix0", "fix1", "six")


def chunks_of(K, mode):
    return max(1, -(-K // (64 if mode in (2, 4) else 32)))


def effective(c, M, N, K, mode):
    bn, sk, kb, g, fused, cl = c
    chunks = chunks_of(K, mode)
    sk = max(1, min(sk, chunks))
    per = -(-chunks // sk)
    sk = -(-chunks // per)
    return (bn, sk, min(kb, per), max(1, min(g, -(-M // (128 * cl)))), fused, cl)


def load(paths):
    table = defaultdict(dict)
    for path in paths:
        with open(path) as f:
            for r in csv.DictReader(f):
                M, N, K, mode = int(r["M"]), int(r["N"]), int(r["K"]), int(r["mode"])
                c = tuple(int(r[k]) for k in ("block_n", "split_k", "kb", "group_m", "fused", "cluster"))
                table[(M, N, K, mode)][effective(c, M, N, K, mode)] = float(r["median_ms"])
    return table


def pick(M, N, K, mode, k, sms=152):
    """The estimate's configuration (block_n, split_k, kb, group_m, fused, cluster)."""
    chunks = chunks_of(K, mode)
    six = mode == 4
    best, out = None, None
    for bn, cl, tc, te in ((64, 1, 1.0, k["epi64"]), (128, 1, k["chunk128"], k["epi128"]),
                           (256, 2, k["chunk_pair"], k["epi_pair"])):
        tiles = -(-M // (128 * cl)) * -(-N // bn)
        slots = sms // cl
        for sk in SPLITS:
            if sk > 1 and sk > chunks:
                break
            per = -(-chunks // sk)
            eff = -(-chunks // per)
            est = -(-(tiles * eff) // slots) * (k["a0"] + per * tc * (k["six"] if six else 1.0) + te)
            if eff > 1:
                est += k["fix0"] + k["fix1"] * M * N * eff * 1e-6
            if best is None or est < best:
                best, out = est, (bn, sk, 8 if (six and cl == 2) else 4, 16, 0, cl)
    return out


def regret(table, k, mode):
    rs = []
    for (M, N, K, m), times in table.items():
        if m != mode:
            continue
        e = effective(pick(M, N, K, m, k), M, N, K, m)
        if e in times:
            rs.append(times[e] / min(times.values()) - 1.0)
    return sum(rs) / len(rs) if rs else float("nan"), len(rs)


def fit(table, samples=8000, seed=3):
    grid = dict(chunk128=[1.3, 1.5, 1.7, 1.9], chunk_pair=[2.0, 2.5, 3.0, 3.5], epi64=[1, 2, 3, 4, 6],
                epi128=[2, 4, 6, 8, 12], epi_pair=[8, 16, 24, 32, 48], a0=[2, 4, 8, 12, 16],
                fix0=[0, 2, 4, 8], fix1=[0, 0.1, 0.25, 0.5, 1], six=[1.5, 2.0])
    combos = list(itertools.product(*(grid[k] for k in KEYS)))
    random.Random(seed).shuffle(combos)

    modes = sorted({key[3] for key in table})

    def score(k):
        return sum(regret(table, k, m)[0] for m in modes)

    best_k, best_s = None, None
    for vals in combos[:samples]:
        k = dict(zip(KEYS, vals))
        s = score(k)
        if best_s is None or s < best_s:
            best_k, best_s = k, s
    improved = True
    while improved:
        improved = False
        for name in KEYS:
            for m in (0.8, 0.9, 1.1, 1.25):
                k = dict(best_k)
                k[name] = round(best_k[name] * m, 4) if best_k[name] else (0.25 if m > 1 else 0.0)
                s = score(k)
                if s < best_s - 1e-5:
                    best_k, best_s, improved = k, s, True
    return best_k


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("timings", nargs="+", help="autotuner CSV files to fit on")
    ap.add_argument("--heldout", default=None)
    ap.add_argument("--samples", type=int, default=8000)
    ap.add_argument("--seed", type=int, default=3)
    args = ap.parse_args(argv)
    table = load(args.timings)
    k = fit(table, args.samples, args.seed)
    print(json.dumps(k))
    for mode, name in ((2, "bf16x3"), (3, "tf32x3"), (4, "bf16x6")):
        if not any(key[3] == mode for key in table):
            continue
        line = f"{name}: train regret {regret(table, k, mode)[0]:.4f}"
        if args.heldout:
            line += f", held-out {regret(load([args.heldout]), k, mode)[0]:.4f}"
        print(line)


if __name__ == "__main__":
    main()
