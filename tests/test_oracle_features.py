"""Pins of the oracle's cost-model features (oracle/features.py) against values
worked out by hand from each feature's definition -- independent of both the
oracle's code and the library's.

The cost model stands in for the paper's search over tile sizes (Section
VI-A): for a shape (M, N, K) and a candidate configuration it describes the
work the kernel will do -- output tiles of 128 x BN, k-chunks of 128 bytes
(64 bf16 or 32 tf32 elements), the split of the k-chunks over split-K
partitions, waves of units over the SMs.  Every expected value below is a
literal, with the arithmetic that gives it written out in the comment, so
that a wrong chunk width, an off-by-one in the wave count or in the fill of
the last wave, a missing clamp of the fold length or of the raster group, or
split-K not re-derived after rounding changes at least one of them."""
import math

import pytest

from oracle import features as F

NAMES = ["log2M", "log2N", "log2K", "bn/128", "log2sk", "kb/8", "log2group", "log2tiles",
         "log2(1+waves)", "fill", "padded", "log2ai", "log2per", "tf32", "fused", "x6", "pair"]


def cfg(bn, sk, kb, g, fused=0, cluster=1):
    return {"block_n": bn, "split_k": sk, "kb": kb, "group_m": g, "fused": fused, "cluster": cluster}


CASES = [
    # 8192^3, BN 128, no split, fold 4, group 16, bf16, 152 SMs.
    #   k-chunks: 8192 / 64 = 128, one split of 128 (per = 128, log2 = 7)
    #   tiles: (8192/128) x (8192/128) = 64 x 64 = 4096 (log2 = 12)
    #   waves: 4096 / 152 = 26.947..; log2(1 + 26.947..) = 4.8046405
    #   last wave: 4096 - 26*152 = 144 units, fill 144/152 = 0.9473684
    #   padding: none (every size a multiple of its tile)
    #   intensity: 2 n^3 / (4 (n^2 + n^2 + 2 n^2)) = n / 8 = 1024, log2 = 10
    #   group: min(16, 64) = 16 (log2 = 4); fold: min(4, 128) = 4, /8 = 0.5
    ((8192, 8192, 8192), cfg(128, 1, 4, 16), False, 152, False,
     [13, 13, 13, 1.0, 0, 0.5, 4, 12, 4.804640537, 0.947368421, 0, 10, 7, 0, 0, 0, 0]),
    # 1060^3 (the paper's sgemm size), BN 64, bf16, 152 SMs.
    #   k-chunks: ceil(1060/64) = 17 (16 x 64 = 1024 < 1060), per = 17, log2 = 4.0874628
    #   tiles: ceil(1060/128) = 9 rows x ceil(1060/64) = 17 columns = 153, log2 = 7.2573878
    #   waves: 153/152, log2(1 + 153/152) = 1.0047379; last wave 1 unit: fill 1/152 = 0.0065789
    #   padding: (9*128)(17*64)(17*64) / 1060^3 - 1 = 1152*1088*1088/1191016000 - 1 = 0.1449662
    #   intensity: 1060/8 = 132.5, log2 = 7.0498485; group: min(16, 9) = 9, log2 = 3.1699250
    ((1060, 1060, 1060), cfg(64, 1, 4, 16), False, 152, False,
     [10.04984855, 10.04984855, 10.04984855, 0.5, 0, 0.5, 3.169925001, 7.257387843,
      1.004737919, 0.006578947, 0.144966220, 7.049848549, 4.087462841, 0, 0, 0, 0]),
    # tf32, 256 x 256 x 96, BN 128, split 8 requested, fold 8, group 1.
    #   k-chunks of 32 tf32 elements: 96/32 = 3 (bf16 would be 2 chunks of 64,
    #   padding K to 128); split: min(8, 3) = 3, per = 1, split = ceil(3/1) = 3,
    #   log2 3 = 1.5849625; fold: min(8, per = 1) = 1, /8 = 0.125
    #   tiles: 2 x 2 = 4 (log2 2); units 4 x 3 = 12: waves 12/152, log2(1 + 12/152) = 0.1096245,
    #   fill 12/152 = 0.0789474; padding: 3 x 32 = 96 = K, none
    #   intensity: 2*256*256*96 / (4 (256*96 + 96*256 + 2*256*256)) = 17.4545, log2 = 4.1255309
    ((256, 256, 96), cfg(128, 8, 8, 1), True, 152, False,
     [8, 8, 6.584962501, 1.0, 1.584962501, 0.125, 0, 2, 0.109624491, 0.078947368, 0,
      4.125530882, 0, 1, 0, 0, 0]),
    # split-K re-derived after rounding: 512 x 512 x 640 bf16, split 6 requested, fold 8, group 16.
    #   k-chunks: 640/64 = 10; per = ceil(10/6) = 2; split = ceil(10/2) = 5 (not 6), log2 5 = 2.3219281
    #   fold: min(8, 2) = 2, /8 = 0.25; group: min(16, 4) = 4, log2 = 2
    #   tiles: 4 x 4 = 16 (log2 4); units 16 x 5 = 80: log2(1 + 80/152) = 0.6100535, fill 80/152
    #   intensity: 2*512*512*640 / (4 (2*512*640 + 2*512*512)) = 71.111, log2 = 6.1520031
    #   fused configuration: feature 1
    ((512, 512, 640), cfg(128, 6, 8, 16, fused=1), False, 152, False,
     [9, 9, 9.321928095, 1.0, 2.321928095, 0.25, 2, 4, 0.610053482, 0.526315789, 0,
      6.152003093, 1, 0, 1, 0, 0]),
    # a last wave that is exactly full: 2432 x 1024 x 512 bf16, BN 128 on 152 SMs.
    #   tiles: (2432/128 = 19) x (1024/128 = 8) = 152 = one full wave: log2(1 + 1) = 1, fill 1
    #   k-chunks 512/64 = 8, per 8 (log2 3); group min(16, 19) = 16
    #   intensity: 2*2432*1024*512 / (4 (2432*512 + 512*1024 + 2*2432*1024)), log2 = 6.5614270
    #   six-product mode: feature 1
    ((2432, 1024, 512), cfg(128, 1, 4, 16), False, 152, True,
     [11.24792751, 10, 9, 1.0, 0, 0.5, 4, 7.247927513, 1, 1.0, 0, 6.561426986, 3, 0, 0, 1, 0]),
    # the same shape on 148 SMs: 152 units = one wave and 4 units, fill 4/148 = 0.0270270,
    #   log2(1 + 152/148) = 1.0193653
    ((2432, 1024, 512), cfg(128, 1, 4, 16), False, 148, False,
     [11.24792751, 10, 9, 1.0, 0, 0.5, 4, 7.247927513, 1.019365325, 0.027027027, 0,
      6.561426986, 3, 0, 0, 0, 0]),
    # a CTA pair (cluster 2) runs 256 x BN tiles, one unit per pair of SMs:
    # 8192^3 at BN 256 on 152 SMs = 76 pairs.
    #   tiles: (8192/256) x (8192/256) = 32 x 32 = 1024 (log2 10); bn/128 = 2
    #   waves: 1024 / 76 = 13.47..; log2(1 + 13.47..) = 3.8553603
    #   last wave: 1024 - 13*76 = 36 units, fill 36/76 = 0.4736842
    #   group min(16, 32) = 16; k-chunks 128 (log2 7); no padding; intensity 1024 (log2 10)
    ((8192, 8192, 8192), cfg(256, 1, 4, 16, cluster=2), False, 152, False,
     [13, 13, 13, 2.0, 0, 0.5, 4, 10, 3.855360295, 0.473684211, 0, 10, 7, 0, 0, 0, 1]),
    # 1060^3 on pairs at BN 128: row tiles of 256: ceil(1060/256) = 5 (4 x 256 = 1024 < 1060),
    #   column tiles ceil(1060/128) = 9: 45 tiles (log2 5.4918531) on 76 pairs:
    #   log2(1 + 45/76) = 0.6709357, fill 45/76 = 0.5921053
    #   padding: (5*256)(9*128)(17*64) / 1060^3 - 1 = 1280*1152*1088/1191016000 - 1 = 0.3470191
    #   group: min(16, 5) = 5 (log2 2.3219281); k-chunks 17 (log2 4.0874628)
    ((1060, 1060, 1060), cfg(128, 1, 4, 16, cluster=2), False, 152, False,
     [10.04984855, 10.04984855, 10.04984855, 1.0, 0, 0.5, 2.321928095, 5.491853096,
      0.670935724, 0.592105263, 0.347019083, 7.049848549, 4.087462841, 0, 0, 0, 1]),
]


@pytest.mark.parametrize("shape,c,tf32,sms,x6,want", CASES)
def test_features_match_hand_derived_values(shape, c, tf32, sms, x6, want):
    M, N, K = shape
    got = F.features(M, N, K, c, tf32, sms, x6=x6)
    assert len(got) == len(want) == 17
    for name, g, w in zip(NAMES, got, want):
        assert math.isclose(g, w, rel_tol=1e-8, abs_tol=1e-8), (name, g, w)


def test_effective_configuration_by_hand():
    # split 6 over 10 chunks: 2 chunks a split, 5 splits; fold clamped to 2
    e = F.effective(128, 6, 8, 16, 512, 512, 640, tf32=False)
    assert (e["split_k"], e["per"], e["kb"], e["group_m"], e["tiles"], e["chunks"]) == (5, 2, 2, 4, 16, 10)
    # split 4 over 10 chunks: 3 chunks a split, still 4 splits (3 + 3 + 3 + 1)
    e = F.effective(128, 4, 4, 1, 512, 512, 640, tf32=False)
    assert (e["split_k"], e["per"]) == (4, 3)
    # more splits than chunks: one chunk each
    e = F.effective(64, 8, 4, 16, 100, 100, 100, tf32=True)   # ceil(100/32) = 4 chunks
    assert (e["split_k"], e["per"], e["kb"], e["chunks"], e["chunk"]) == (4, 1, 1, 4, 32)
    assert e["tiles"] == 1 * 2 and e["group_m"] == 1             # 100 rows: 1 row tile; 100/64: 2
    # K = 0 still counts one (empty) chunk, so the model never takes log2 0
    e = F.effective(128, 1, 4, 16, 128, 128, 0, tf32=False)
    assert (e["chunks"], e["split_k"], e["per"]) == (1, 1, 1)
