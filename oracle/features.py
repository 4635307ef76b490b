"""Oracle restatement of the cost model's input features -- test
infrastructure only.

The cost model replaces the paper's tile-size search (Section VI-A) with a
prediction from features of the shape and the candidate configuration.  Each
feature is written here from its definition, in float64:

  log2 M, log2 N, log2 K
  tile width / 128
  log2 split-K   (effective: at most one split per k-chunk, no empty split)
  fold length / 8 (effective: at most the k-chunks of one split)
  log2 raster group (effective: at most the number of row tiles)
  log2 output tiles
  log2(1 + waves), waves = tiles * splits / processors
  fill of the last wave (1 when the last wave is full)
  padded-work fraction = (tile-rounded M*N*K) / (M*N*K) - 1
  log2 arithmetic intensity, 2MNK / (4 (MK + KN + 2 MN))
  log2 k-chunks per split
  1 for the tf32 mode, else 0
  1 when A is split inside the gemm kernel, else 0
  1 for the six-product bf16 mode, else 0
  1 when a tile runs on a pair of SMs, else 0

A k-chunk is 128 bytes of one row: 64 bf16 or 32 tf32 elements.  An output
tile is 128 rows high on one SM, 256 on a pair of SMs (cluster 2); the
processors that run units at the same time are the SMs, or the pairs.
"""
from __future__ import annotations

import math


def effective(block_n: int, split_k: int, kb: int, group_m: int, M: int, N: int, K: int,
              tf32: bool, cluster: int = 1):
    chunk = 32 if tf32 else 64
    chunks = max(1, -(-K // chunk))
    sk = max(1, min(split_k, chunks))
    per = -(-chunks // sk)
    sk = -(-chunks // per)
    tile_h = 128 * cluster
    tiles_m = -(-M // tile_h)
    tiles = tiles_m * -(-N // block_n)
    return {"bn": block_n, "split_k": sk, "per": per, "kb": min(kb, per),
            "group_m": max(1, min(group_m, tiles_m)), "tiles": tiles, "chunks": chunks,
            "chunk": chunk, "cluster": cluster, "tile_h": tile_h}


def features(M: int, N: int, K: int, cfg: dict, tf32: bool, sms: int, x6: bool = False) -> list[float]:
    cluster = cfg.get("cluster", 1)
    e = effective(cfg["block_n"], cfg["split_k"], cfg["kb"], cfg["group_m"], M, N, K, tf32, cluster)
    procs = sms // cluster
    units = e["tiles"] * e["split_k"]
    waves = units / procs
    rem = units - math.floor(waves) * procs
    fill = 1.0 if rem == 0 else rem / procs
    tiles_m = -(-M // e["tile_h"])
    tiles_n = -(-N // e["bn"])
    padded = (tiles_m * e["tile_h"]) * (tiles_n * e["bn"]) * (e["chunks"] * e["chunk"]) / (M * N * K) - 1
    ai = 2.0 * M * N * K / (4.0 * (M * K + K * N + 2.0 * M * N))
    return [math.log2(M), math.log2(N), math.log2(K), e["bn"] / 128.0, math.log2(e["split_k"]),
            e["kb"] / 8.0, math.log2(e["group_m"]), math.log2(e["tiles"]), math.log2(1 + waves),
            fill, padded, math.log2(ai), math.log2(e["per"]), 1.0 if tf32 else 0.0,
            1.0 if cfg.get("fused", 0) else 0.0, 1.0 if x6 else 0.0, 1.0 if cluster == 2 else 0.0]
