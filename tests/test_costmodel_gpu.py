"""The learned part on the GPU: the MLP's forward/backward kernels against the
FP64 oracle's gradient, the Adam kernel against the oracle's update, the
autotuner's table and selection policy, and what a trained model gains over
the built-in heuristic on shapes it was not trained on (regret against the
exhaustive autotune, the paper's method of picking tiles, Section VI-A)."""
import csv

import numpy as np
import pytest
import torch

import oracle
import paper_1804_10694_gb300 as pkg
import workloads as W
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

F = 17   # the library's feature count (checked in the host-logic tests)
H = 64


def _theta(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(omlp.param_count(F, H)) * scale).astype(np.float32)


@pytest.mark.parametrize("n", [1, 37, 1000, 4099])
def test_mlp_gradient_matches_fp64_oracle(n):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, F)).astype(np.float32)
    t = rng.standard_normal(n).astype(np.float32)
    theta = _theta(n)
    loss, grad = pkg.mlp_loss_grad(theta, X, t)
    ref_loss, ref_grad = omlp.backward(theta.astype(np.float64), X.astype(np.float64),
                                       t.astype(np.float64), H)
    assert abs(loss - ref_loss) <= 1e-4 * max(ref_loss, 1e-6)
    err = np.linalg.norm(grad - ref_grad) / np.linalg.norm(ref_grad)
    assert err <= 1e-5, err
    scale = np.abs(ref_grad).max()
    assert np.all(np.abs(grad - ref_grad) <= 1e-4 * np.maximum(np.abs(ref_grad), 1e-2 * scale))


def test_adam_kernel_matches_oracle_over_steps():
    rng = np.random.default_rng(3)
    P = omlp.param_count(F, H)
    theta = rng.standard_normal(P).astype(np.float32)
    m = np.zeros(P, np.float32)
    v = np.zeros(P, np.float32)
    th_ref, m_ref, v_ref = theta.astype(np.float64), np.zeros(P), np.zeros(P)
    # the kernel receives FP32 hyperparameters: 1 - float32(0.999) differs from
    # 0.001 by 1.3e-5 relative, so the oracle gets the same FP32 values, widened
    lr, b1, b2, eps = (float(np.float32(x)) for x in (1e-2, 0.9, 0.999, 1e-8))
    for step in range(1, 6):
        g = rng.standard_normal(P).astype(np.float32)
        theta, m, v = pkg.mlp_adam_step(theta, g, m, v, step, lr=lr, beta1=b1, beta2=b2, eps=eps)
        th_ref, m_ref, v_ref = omlp.adam_step(th_ref, g.astype(np.float64), m_ref, v_ref, step, lr,
                                              b1, b2, eps)
        assert np.allclose(theta, th_ref, rtol=1e-5, atol=1e-6)
        assert np.allclose(m, m_ref, rtol=1e-5, atol=1e-7)
        assert np.allclose(v, v_ref, rtol=1e-5, atol=1e-9)


def _read_rows(path):
    with open(path) as f:
        return [r for r in csv.DictReader(f)]


def test_autotune_table_and_table_selection(tmp_path):
    """Shapes carry leading dimensions: the tight 640 x 384 x 1000 and the same
    sizes with ldc = N + 3 (staged stores of C) are tuned and looked up
    apart."""
    path = str(tmp_path / "timings.csv")
    shapes = [(640, 384, 1000, 1000, 384, 384), (640, 384, 1000, 1000, 384, 387),
              (96, 2000, 300, 300, 2000, 2000), (3000, 64, 5000, 5001, 64, 64)]
    pkg.autotune(shapes, mode="bf16x3", reps=3, out_path=path)
    rows = _read_rows(path)
    for sh in shapes:
        mine = [r for r in rows
                if tuple(int(r[k]) for k in ("M", "N", "K", "lda", "ldb", "ldc")) == sh]
        assert len(mine) >= 2
        ids = {int(r["config_id"]) for r in mine}
        assert len(ids) == len(mine)          # every distinct configuration timed once
        best = min(mine, key=lambda r: float(r["median_ms"]))
        M, N, K, lda, ldb, ldc = sh
        cid, ms = pkg.autotune_best(M, N, K, "bf16x3", lda=lda, ldb=ldb, ldc=ldc)
        assert cid == int(best["config_id"])
        assert pkg.select_config(M, N, K, "bf16x3", "table", lda=lda, ldb=ldb, ldc=ldc) == cid
        plan = pkg.Plan(M, N, K, lda, ldb, ldc, mode="bf16x3", select="table")
        assert plan.info()["config_id"] == cid
        plan.destroy()


def _regret(table, shape, cid):
    times = table[shape]
    return times[cid] / min(times.values()) - 1.0


def test_trained_model_beats_the_untrained_heuristic(tmp_path):
    """Train on the autotuner's timings of 240 shapes, then compare, on 40
    held-out shapes timed exhaustively, the mean regret of the model's pick
    with that of the built-in heuristic's pick (the fitted estimate of each
    candidate's time): the model must be better."""
    train = W.training_shapes(240, seed=11, hi=8192, max_mnk_log2=33.0)
    held = W.training_shapes(40, seed=12, hi=8192, max_mnk_log2=33.0)
    tpath, hpath = str(tmp_path / "train.csv"), str(tmp_path / "held.csv")
    pkg.autotune(train, mode="bf16x3", reps=3, out_path=tpath)
    pkg.autotune(held, mode="bf16x3", reps=3, out_path=hpath)
    loss = pkg.costmodel_train(tpath, epochs=3000, seed=1, out_model=str(tmp_path / "m.txt"))
    assert np.isfinite(loss) and loss < 0.5            # normalised MSE
    table = {}
    for r in _read_rows(hpath):   # tight shapes: keyed by the sizes
        table.setdefault((int(r["M"]), int(r["N"]), int(r["K"])), {})[int(r["config_id"])] = float(r["median_ms"])
    model_regret, default_regret = [], []
    for s in held:
        cid, _ = pkg.costmodel_predict(*s, "bf16x3")
        model_regret.append(_regret(table, tuple(s), cid))
        default_regret.append(_regret(table, tuple(s), _canonical(table[tuple(s)], s)))
    m, d = float(np.mean(model_regret)), float(np.mean(default_regret))
    print(f"held-out mean regret: model {m:.3f}, heuristic {d:.3f}")
    assert m < d, (m, d)
    # the loaded model drives GEMM_SELECT_MODEL
    pkg.costmodel_load(str(tmp_path / "m.txt"))
    plan = pkg.Plan(*held[0], mode="bf16x3", select="model")
    assert plan.info()["config_id"] == pkg.costmodel_predict(*held[0], "bf16x3")[0]
    plan.destroy()


def _canonical(times, shape):
    """The heuristic's configuration, mapped onto the timed representative of
    its effective configuration (the tuner times each distinct one once)."""
    M, N, K = shape
    d = pkg.config_default("bf16x3", M, N, K)
    if d in times:
        return d
    from oracle import features as ofeat
    dc = pkg.config_get("bf16x3", d)
    want = ofeat.effective(**{k: dc[k] for k in ("block_n", "split_k", "kb", "group_m", "cluster")},
                           M=M, N=N, K=K, tf32=False)
    for cid in times:
        c = pkg.config_get("bf16x3", cid)
        e = ofeat.effective(c["block_n"], c["split_k"], c["kb"], c["group_m"], M, N, K, False, c["cluster"])
        if all(e[k] == want[k] for k in ("bn", "split_k", "kb", "group_m", "cluster")) and not c["fused"]:
            return cid
    raise AssertionError("heuristic configuration was not timed")
