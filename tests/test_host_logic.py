"""CPU checks of host-side logic: cost-model features against the oracle's
restatement, model/table file parsing and error handling, grouped-plan
argument validation (no device is touched)."""
import ctypes
import os

import numpy as np
import pytest

import paper_1804_10694_gb300 as pkg
from oracle import features as ofeat
import workloads as W


F = 17   # cost-model features (the oracle's restatement lists them)

SHAPES = [(8192, 8192, 8192), (1060, 1060, 1060), (50176, 64, 576), (12544, 128, 1152),
          (3136, 256, 2304), (33, 17, 5), (1, 1, 1), (129, 4099, 63), (300, 70, 20000)]


@pytest.mark.parametrize("mode,tf32", [("bf16x3", False), ("tf32x3", True), ("bf16x6", False)])
def test_features_match_oracle_restatement(mode, tf32):
    n = pkg.config_count(mode)
    assert pkg.costmodel_feature_count() == F
    for (M, N, K) in SHAPES:
        for cid in range(0, n, 5):
            cfg = pkg.config_get(mode, cid)
            for sms in (152, 148):
                got = pkg.costmodel_features(M, N, K, mode, cid, sms)
                ref = np.array(ofeat.features(M, N, K, cfg, tf32, sms, x6=(mode == "bf16x6")))
                assert np.allclose(got, ref, rtol=1e-5, atol=1e-5), (M, N, K, cfg, got, ref)


def test_features_reject_bad_arguments():
    lib = pkg.load()
    out = np.zeros(F, np.float32)
    assert lib.gemm_costmodel_features(0, 4, 4, 2, 0, 152, out.ctypes.data) == 1
    assert lib.gemm_costmodel_features(4, 4, 4, 1, 0, 152, out.ctypes.data) == 1   # SIMT
    assert lib.gemm_costmodel_features(4, 4, 4, 2, 10 ** 6, 152, out.ctypes.data) == 1


def test_costmodel_load_rejects_missing_and_corrupt_files(tmp_path):
    lib = pkg.load()
    assert lib.gemm_costmodel_load(str(tmp_path / "missing.txt").encode()) == 7
    bad = tmp_path / "bad.txt"
    bad.write_text("gb300-gemm-costmodel 1\nfeatures %d hidden 64 params 5\n" % F)
    assert lib.gemm_costmodel_load(str(bad).encode()) == 7
    assert b"malformed" in lib.gemm_last_error()
    bad.write_text("not a model\n")
    assert lib.gemm_costmodel_load(str(bad).encode()) == 7
    # truncated theta
    P = 64 * F + 64 + 64 * 64 + 64 + 64 + 1
    txt = ("gb300-gemm-costmodel 1\nfeatures %d hidden 64 params %d\nmean %s\nstd %s\n"
           "target 0 1\ntheta %s\n" % (F, P, " ".join(["0"] * F), " ".join(["1"] * F),
                                       " ".join(["0.5"] * (P - 3))))
    bad.write_text(txt)
    assert lib.gemm_costmodel_load(str(bad).encode()) == 7


def test_costmodel_load_accepts_well_formed_file(tmp_path):
    P = 64 * F + 64 + 64 * 64 + 64 + 64 + 1
    good = tmp_path / "good.txt"
    good.write_text("gb300-gemm-costmodel 1\nfeatures %d hidden 64 params %d\nmean %s\nstd %s\n"
                    "target -1.5 2\ntheta %s\n" % (F, P, " ".join(["0"] * F), " ".join(["1"] * F),
                                                   " ".join(["0.01"] * P)))
    assert pkg.load().gemm_costmodel_load(str(good).encode()) == 0


def test_autotune_table_file_parsing(tmp_path):
    lib = pkg.load()
    assert lib.gemm_autotune_load(str(tmp_path / "none.csv").encode()) == 7
    f = tmp_path / "t.csv"
    f.write_text("M,N,K,lda,ldb,ldc,mode,config_id,median_ms,block_n,split_k,kb,group_m,fused\n"
                 "777,555,333,333,555,555,2,3,0.5,128,1,2,1,0\n"
                 "777,555,333,333,555,555,2,7,0.25,128,2,2,1,0\n"
                 "777,555,333,333,555,555,2,99999,0.01,0,0,0,0,0\ngarbage line\n")
    assert lib.gemm_autotune_load(str(f).encode()) == 0
    assert pkg.autotune_best(777, 555, 333, "bf16x3") == (7, 0.25)
    with pytest.raises(pkg.GemmError):
        pkg.autotune_best(777, 555, 334, "bf16x3")
    # rows of the earlier format (no leading dimensions) are tight shapes
    g = tmp_path / "old.csv"
    g.write_text("M,N,K,mode,config_id,median_ms,block_n,split_k,kb,group_m\n"
                 "901,503,207,2,11,0.75,128,1,2,1,0\n")
    assert lib.gemm_autotune_load(str(g).encode()) == 0
    assert pkg.autotune_best(901, 503, 207, "bf16x3", lda=207, ldb=503, ldc=503) == (11, 0.75)


def test_table_selection_keys_on_leading_dimensions(tmp_path):
    """A shape is (M, N, K, lda, ldb, ldc): the tuned table holds a tight
    shape and the same sizes with ldc = N + 3 apart, and GEMM_SELECT_TABLE
    picks each one's own best configuration (no device needed)."""
    M, N, K = 1200, 650, 900
    f = tmp_path / "lds.csv"
    f.write_text("M,N,K,lda,ldb,ldc,mode,config_id,median_ms,block_n,split_k,kb,group_m,fused\n"
                 f"{M},{N},{K},{K},{N},{N},2,5,0.40,128,1,2,1,0\n"
                 f"{M},{N},{K},{K},{N},{N},2,9,0.30,128,2,2,1,0\n"
                 f"{M},{N},{K},{K},{N},{N + 3},2,9,0.50,128,2,2,1,0\n"
                 f"{M},{N},{K},{K},{N},{N + 3},2,41,0.45,64,1,2,1,0\n")
    pkg.autotune_load(str(f))
    assert pkg.autotune_best(M, N, K, "bf16x3") == (9, pytest.approx(0.30))
    assert pkg.autotune_best(M, N, K, "bf16x3", ldc=N + 3) == (41, pytest.approx(0.45))
    assert pkg.select_config(M, N, K, "bf16x3", "table") == 9
    assert pkg.select_config(M, N, K, "bf16x3", "table", ldc=N + 3) == 41
    # an untuned leading dimension falls back to the heuristic
    assert pkg.select_config(M, N, K, "bf16x3", "table", lda=K + 1) == \
        pkg.select_config(M, N, K, "bf16x3", "default")
    assert pkg.select_config(M, N, K, "simt", "table") == -1
    with pytest.raises(pkg.GemmError):
        pkg.select_config(M, N, K, "bf16x3", "table", ldc=N - 1)


def test_autotune_rejects_bad_shapes_before_running():
    lib = pkg.load()
    bad = (ctypes.c_int64 * 6)(64, 64, 64, 63, 64, 64)      # lda < K
    assert lib.gemm_autotune(bad, 1, 2, 3, None) == 1
    assert b"shape 0" in lib.gemm_last_error()


def test_grouped_plan_argument_validation():
    lib = pkg.load()
    h = ctypes.c_void_p()
    a = (ctypes.c_int64 * 2)(4, 4)
    neg = (ctypes.c_int64 * 2)(4, -1)
    small_ld = (ctypes.c_int64 * 2)(4, 3)
    assert lib.gemm_grouped_plan_create(2, neg, a, a, a, a, a, 2, 0, ctypes.byref(h)) == 1
    assert lib.gemm_grouped_plan_create(2, a, a, a, small_ld, a, a, 2, 0, ctypes.byref(h)) == 1
    assert b"problem 1" in lib.gemm_last_error()
    assert lib.gemm_grouped_plan_create(-1, a, a, a, a, a, a, 2, 0, ctypes.byref(h)) == 1
    assert lib.gemm_grouped_plan_create(2, None, a, a, a, a, a, 2, 0, ctypes.byref(h)) == 1
    assert lib.gemm_grouped_plan_create_config(2, a, a, a, a, a, a, 2, 96, 4, ctypes.byref(h)) == 1
    assert lib.gemm_grouped_plan_create_config(2, a, a, a, a, a, a, 2, 128, 9, ctypes.byref(h)) == 1
    assert lib.gemm_grouped_execute(None, None, None, None, None, None, None) == 1


def test_grouped_workload_shapes():
    shapes = W.grouped_shapes()
    assert len(shapes) == 512
    arr = np.array(shapes)
    assert arr.min() >= 32 and arr.max() <= 1024
    # log-uniform: the median of each dimension is near sqrt(32 * 1024) = 181
    assert 120 < np.median(arr[:, 0]) < 260
    flops = sum(2.0 * m * n * k for m, n, k in shapes)
    assert 5e9 < flops < 6e10


def test_training_shapes_bounded():
    shapes = W.training_shapes(200, seed=7)
    assert len(shapes) == 200
    for m, n, k in shapes:
        assert m * n * k <= 2 ** 37
        assert min(m, n, k) >= 1


def test_costmodel_ensemble_file_format(tmp_path):
    """Version 2 files hold `members` networks (one theta line each); a
    missing member or a bad member count is rejected."""
    P = 64 * F + 64 + 64 * 64 + 64 + 64 + 1
    head = ("gb300-gemm-costmodel 2\nfeatures %d hidden 64 params %d members %%d\nmean %s\nstd %s\n"
            "target -1.5 2\n" % (F, P, " ".join(["0"] * F), " ".join(["1"] * F)))
    theta = "theta %s\n" % " ".join(["0.01"] * P)
    lib = pkg.load()
    f = tmp_path / "m.txt"
    f.write_text(head % 3 + theta * 3)
    assert lib.gemm_costmodel_load(str(f).encode()) == 0
    f.write_text(head % 3 + theta * 2)
    assert lib.gemm_costmodel_load(str(f).encode()) == 7
    f.write_text(head % 0 + theta)
    assert lib.gemm_costmodel_load(str(f).encode()) == 7


def _estimate_pick(M, N, K, mode, sms=152):
    """The built-in tile choice, restated from its definition: for each
    packed candidate (128 x 64 or 128 x 128 tiles on one SM, 256 x 256 on a
    CTA pair) and split count, waves x (prologue + k-chunks a split x chunk
    cost + epilogue) plus, when K is split, the fix-up's cost; the first
    minimum in the order 64, 128, pair and 1, 2, 3, 4, 6, 8 splits."""
    chunk_elems = 32 if mode == "tf32x3" else 64
    chunks = max(1, -(-K // chunk_elems))
    six = mode == "bf16x6"
    best, pick = None, None
    for bn, cl, tc, te in ((64, 1, 1.0, 3.3), (128, 1, 1.5, 7.2), (256, 2, 2.0, 28.8)):
        tiles = -(-M // (128 * cl)) * -(-N // bn)
        slots = sms // cl
        for sk in (1, 2, 3, 4, 6, 8):
            if sk > 1 and sk > chunks:
                break
            per = -(-chunks // sk)
            eff = -(-chunks // per)
            waves = -(-(tiles * eff) // slots)
            est = waves * (3.6 + per * tc * (1.6 if six else 1.0) + te)
            if eff > 1:
                est += 4.0 + 0.99 * M * N * eff * 1e-6
            if best is None or est < best:
                best, pick = est, (bn, sk, 8 if (six and cl == 2) else 4, 16, cl)
    return pick


def test_default_tile_choice_is_its_estimate():
    """The default configuration of a shape is the candidate with the
    smallest estimated time (the restatement above) for every mode, over
    squares, the convolution-as-gemm shapes and random shapes; and a few
    anchors: the paper's 1060^3 runs unsplit 128 x 128 tiles, one 128-row
    tile (128^3) the narrower 128 x 64 tile, 8192^3 the CTA pair, and an
    N <= 64 problem 64-wide tiles."""
    rng = np.random.default_rng(5)
    shapes = [(n, n, n) for n in (128, 256, 512, 768, 1024, 1060, 2048, 4099, 8192)]
    shapes += [(50176, 64, 576), (12544, 128, 1152), (3136, 256, 2304), (1, 1, 1), (7, 3000, 5)]
    shapes += [tuple(int(x) for x in 2 ** rng.uniform(4, 14, 3)) for _ in range(300)]
    for mode in ("bf16x3", "tf32x3", "bf16x6"):
        for M, N, K in shapes:
            c = pkg.config_get(mode, pkg.config_default(mode, M, N, K))
            got = (c["block_n"], c["split_k"], c["kb"], c["group_m"], c["cluster"])
            assert c["fused"] == 0
            assert got == _estimate_pick(M, N, K, mode), (mode, M, N, K)

    def pick(n, mode="bf16x3"):
        c = pkg.config_get(mode, pkg.config_default(mode, n, n, n))
        return c["block_n"], c["split_k"], c["cluster"]
    assert pick(1060) == (128, 1, 1)
    assert pick(128)[0] == 64 and pick(128)[2] == 1
    assert pick(8192) == (256, 1, 2)
    c = pkg.config_get("bf16x3", pkg.config_default("bf16x3", 50176, 64, 576))
    assert c["block_n"] == 64 and c["cluster"] == 1

