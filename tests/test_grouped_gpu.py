"""Grouped gemm on the GPU: every problem of one persistent launch against the
FP64 oracle (relative Frobenius error <= 1e-5 per problem, bit-exact on
integer inputs), bit-identical to running each problem alone with the same
tile configuration, graph replay identical to eager execution, and the
per-problem pointer table refreshed when the caller's pointers change."""
import numpy as np
import pytest
import torch

import oracle
import paper_1804_10694_gb300 as pkg
import workloads as W
from gpu_helpers import TOL

pytestmark = pytest.mark.gpu


def _problems(shapes, seed, gen=W.uniform, pad=0):
    probs = []
    for i, (M, N, K) in enumerate(shapes):
        A = gen(M, K, seed + 3 * i, ld=K + pad) if M and K else np.zeros((max(M, 1), K + pad + 1), np.float32)
        B = gen(K, N, seed + 3 * i + 1, ld=N + pad) if K and N else np.zeros((max(K, 1), N + pad + 1), np.float32)
        C = gen(M, N, seed + 3 * i + 2, ld=N + pad) if M and N else np.zeros((max(M, 1), N + pad + 1), np.float32)
        probs.append((A, B, C))
    return probs


def _run(plan, probs, alphas, betas, graph=True):
    dA = [torch.from_numpy(A).cuda() for A, _, _ in probs]
    dB = [torch.from_numpy(B).cuda() for _, B, _ in probs]
    dC = [torch.from_numpy(C).cuda() for _, _, C in probs]
    plan.execute(dA, dB, dC, alphas, betas, graph=graph)
    torch.cuda.synchronize()
    return [c.cpu().numpy() for c in dC]


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3", "bf16x6", "simt"])
def test_grouped_small_uneven_against_oracle(mode):
    shapes = [(300, 200, 100), (1, 1, 1), (129, 65, 1000), (64, 64, 64), (0, 5, 5), (7, 300, 0),
              (513, 33, 257), (31, 129, 77), (250, 1024, 40), (5, 0, 9)]
    probs = _problems(shapes, 100, pad=3)
    alphas = [1.0, 1.5, -2.0, 1.0, 1.0, 0.5, 1.0, 0.0, 1.0, 1.0]
    betas = [1.0, 0.5, 0.0, -1.0, 1.0, 2.0, 1.0, 0.75, 0.0, 1.0]
    lds = [(K + 3, N + 3, N + 3) for (M, N, K) in shapes]
    plan = pkg.GroupedPlan(shapes, lds=lds, mode=mode)
    outs = _run(plan, probs, alphas, betas)
    for (M, N, K), (A, B, C), out, a, b in zip(shapes, probs, outs, alphas, betas):
        if M == 0 or N == 0:
            assert np.array_equal(out, C)
            continue
        ref = oracle.gemm_f64(M, N, K, a, A, B, b, C)
        assert oracle.rel_frob(out, ref) <= TOL, (M, N, K)
        assert np.array_equal(out[:, N:].view(np.uint32), C[:, N:].view(np.uint32))   # padding
    plan.destroy()


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3", "bf16x6"])
def test_grouped_integer_inputs_bit_exact(mode):
    shapes = W.grouped_shapes(24, seed=77, lo=16, hi=700)
    probs = _problems(shapes, 300, gen=W.integers)
    alphas, betas = [1.5] * len(shapes), [0.5] * len(shapes)
    plan = pkg.GroupedPlan(shapes, mode=mode)
    outs = _run(plan, probs, alphas, betas)
    for (M, N, K), (A, B, C), out in zip(shapes, probs, outs):
        ref = oracle.gemm_f64(M, N, K, 1.5, A, B, 0.5, C).astype(np.float32)
        assert np.array_equal(out, ref)


@pytest.mark.parametrize("block_n,kb", [(128, 4), (64, 2), (128, 8)])
def test_grouped_equals_single_problem_plans(block_n, kb):
    """Same tile width, fold length and no split-K: every output element is
    computed by the same sequence of operations, so results are identical."""
    shapes = W.grouped_shapes(16, seed=5, lo=32, hi=600)
    probs = _problems(shapes, 500)
    alphas, betas = [1.5] * len(shapes), [0.5] * len(shapes)
    plan = pkg.GroupedPlan(shapes, mode="bf16x3", block_n=block_n, kb=kb)
    outs = _run(plan, probs, alphas, betas)
    ncfg = pkg.config_count("bf16x3")
    cid = next(i for i in range(ncfg) if pkg.config_get("bf16x3", i) ==
               {"block_n": block_n, "stages": 4 if block_n == 64 else 3, "split_k": 1, "kb": kb,
                "group_m": 16, "fused": 0, "cluster": 1})
    for (M, N, K), (A, B, C), out in zip(shapes, probs, outs):
        dA, dB, dC = (torch.from_numpy(x).cuda() for x in (A, B, C))
        single = pkg.Plan(M, N, K, mode="bf16x3", config_id=cid)
        single.execute(dA, dB, dC, 1.5, 0.5)
        torch.cuda.synchronize()
        assert np.array_equal(dC.cpu().numpy(), out), (M, N, K)
        single.destroy()


def test_graph_replay_equals_eager_and_tracks_pointer_changes():
    shapes = W.grouped_shapes(32, seed=9, lo=32, hi=512)
    probs = _problems(shapes, 700)
    alphas, betas = [1.0] * 32, [1.0] * 32
    plan = pkg.GroupedPlan(shapes, mode="bf16x3")
    eager = _run(plan, probs, alphas, betas, graph=False)
    graph1 = _run(plan, probs, alphas, betas, graph=True)     # captures
    graph2 = _run(plan, probs, alphas, betas, graph=True)     # replays, new buffers
    for e, g1, g2 in zip(eager, graph1, graph2):
        assert np.array_equal(e, g1) and np.array_equal(e, g2)
    # new scalars and new output buffers on a replay
    alphas2 = [0.5 * (i % 3 + 1) for i in range(32)]
    betas2 = [0.0 if i % 2 else 1.0 for i in range(32)]
    graph3 = _run(plan, probs, alphas2, betas2, graph=True)
    for (M, N, K), (A, B, C), out, a, b in zip(shapes, probs, graph3, alphas2, betas2):
        ref = oracle.gemm_f64(M, N, K, a, A, B, b, C)
        assert oracle.rel_frob(out, ref) <= TOL
    plan.destroy()


def test_grouped_512_problem_workload():
    """The grouped workload: 512 problems, M, N, K log-uniform in [32, 1024]
    (seed 4000), uniform[-1, 1] entries, alpha = beta = 1, one persistent
    launch replayed from a CUDA graph; error reported per problem."""
    shapes = W.grouped_shapes()
    sa, _, _ = W.seeds(W.CONFIG_GROUPED)
    probs = _problems(shapes, sa)
    plan = pkg.GroupedPlan(shapes, mode="bf16x3")
    outs = _run(plan, probs, [1.0] * 512, [1.0] * 512)
    worst = 0.0
    for (M, N, K), (A, B, C), out in zip(shapes, probs, outs):
        ref = oracle.gemm_f64(M, N, K, 1.0, A, B, 1.0, C)
        worst = max(worst, oracle.rel_frob(out, ref))
    assert worst <= TOL
    plan.destroy()


def test_grouped_exhaustive_selection_runs_and_is_correct():
    shapes = W.grouped_shapes(40, seed=21, lo=32, hi=400)
    probs = _problems(shapes, 900)
    plan = pkg.GroupedPlan(shapes, mode="bf16x3", select="exhaustive")
    info = plan.info()
    assert info["block_n"] in (64, 128) and 1 <= info["kb"] <= 8
    outs = _run(plan, probs, [1.0] * 40, [1.0] * 40)
    for (M, N, K), (A, B, C), out in zip(shapes, probs, outs):
        ref = oracle.gemm_f64(M, N, K, 1.0, A, B, 1.0, C)
        assert oracle.rel_frob(out, ref) <= TOL
    plan.destroy()


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3", "bf16x6"])
@pytest.mark.parametrize("graph", [True, False])
def test_grouped_plan_state_is_clean_between_executions(mode, graph):
    """The block maxima, pack counters and unit counter of a grouped plan are
    cleared by the last CTA of each execution's gemm launch: one plan run on
    problems whose blocks need scaling (2^70 and 2^-90), then ordinary ones,
    then the scaled ones again gives, each time, the bits of a fresh plan."""
    shapes = [(300, 200, 100), (129, 65, 1000), (513, 33, 257), (64, 300, 64)]
    base = _problems(shapes, 500)
    scaled = [(W.scaled(A, 70), W.scaled(B, -90), C) for A, B, C in base]
    alphas, betas = [1.5] * len(shapes), [0.5] * len(shapes)
    fresh = []
    for probs in (scaled, base):
        p = pkg.GroupedPlan(shapes, mode=mode)
        fresh.append(_run(p, probs, alphas, betas, graph=graph))
        p.destroy()
    plan = pkg.GroupedPlan(shapes, mode=mode)
    for i in (0, 1, 0, 1):
        outs = _run(plan, (scaled, base)[i], alphas, betas, graph=graph)
        for o, f in zip(outs, fresh[i]):
            assert np.array_equal(o, f), i
    plan.destroy()
    pkg.device_error()
