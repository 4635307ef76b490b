"""GPU parity of every gemm mode against the FP64 CPU oracle, through the C ABI.

Bar: relative Frobenius error <= 1e-5 on every result; bit-exact results on
integer-valued inputs (products and sums exact in FP32); identical results
across tile configurations on integer inputs (a schedule must not change the
answer, Tiramisu Section III); full and partial tiles alike (Section V-B)."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_1804_10694_gb300 as pkg
import workloads as W
from gpu_helpers import MODES, TOL, check_padding_untouched, dev, run_gemm, square_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _device():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    pkg.load()
    yield
    pkg.device_error()


# ------------------------------------------------------------ small parity
@pytest.mark.parametrize("mode", MODES)
def test_config0_512_cubed(mode):
    sa, sb, sc = W.seeds(W.CONFIG_SMALL)
    n = 512
    A, B, C0 = W.uniform(n, n, sa), W.uniform(n, n, sb), W.uniform(n, n, sc)
    ref = oracle.gemm_f64(n, n, n, 1.5, A, B, 0.5, C0)
    got = run_gemm(mode, n, n, n, 1.5, A, B, 0.5, C0)
    assert oracle.rel_frob(got, ref) <= TOL


RAGGED = [(300, 260, 333, 0), (129, 257, 1060, 1), (1060, 1060, 1060, 0), (1, 1, 1, 0),
          (5, 3, 7, 3), (128, 128, 64, 0), (17, 300, 5, 1), (260, 65, 97, 3), (2, 500, 1, 0),
          (777, 64, 129, 0), (64, 777, 4099, 1)]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("M,N,K,pad", RAGGED)
@pytest.mark.parametrize("alpha,beta", W.ALPHA_BETA)
def test_ragged_shapes(mode, M, N, K, pad, alpha, beta):
    A = W.uniform(M, K, 11, ld=K + pad)
    B = W.uniform(K, N, 12, ld=N + pad)
    C0 = W.uniform(M, N, 13, ld=N + pad)
    ref = oracle.gemm_f64(M, N, K, alpha, A, B, beta, C0)
    got = run_gemm(mode, M, N, K, alpha, A, B, beta, C0)
    assert oracle.rel_frob(got, ref) <= TOL, (M, N, K)
    check_padding_untouched(C0, got, N)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("alpha,beta", W.ALPHA_BETA)
def test_integer_inputs_bit_exact(mode, alpha, beta):
    M, N, K = 700, 650, 1100
    A, B, C0 = W.integers(M, K, 1), W.integers(K, N, 2), W.integers(M, N, 3)
    ref = oracle.gemm_f64(M, N, K, alpha, A, B, beta, C0)
    got = run_gemm(mode, M, N, K, alpha, A, B, beta, C0)
    assert np.array_equal(got, ref.astype(np.float32))


@pytest.mark.parametrize("mode", MODES)
def test_brute_force_tiny_shapes(mode):
    shapes = [(m, n, k) for m in range(1, 10) for n in range(1, 10) for k in range(1, 10)][::11]
    shapes += [(13, 17, 31), (33, 13, 17), (127, 129, 31), (129, 127, 33), (31, 255, 257)]
    for i, (M, N, K) in enumerate(shapes):
        pad = (0, 1, 3)[i % 3]
        A = W.uniform(M, K, 500 + i, ld=K + pad)
        B = W.uniform(K, N, 600 + i, ld=N + pad)
        C0 = W.uniform(M, N, 700 + i, ld=N + pad)
        ref = oracle.gemm_f64(M, N, K, 1.5, A, B, -0.75, C0)
        got = run_gemm(mode, M, N, K, 1.5, A, B, -0.75, C0)
        assert oracle.rel_frob(got, ref) <= TOL, (M, N, K)
        check_padding_untouched(C0, got, N)


@pytest.mark.parametrize("mode", MODES)
def test_blas_special_cases(mode):
    M, N, K = 70, 50, 40
    A, B, C0 = W.uniform(M, K, 1), W.uniform(K, N, 2), W.uniform(M, N, 3)
    # K == 0 -> C = beta*C
    got = run_gemm(mode, M, N, 0, 1.0, A, B, 0.5, C0)
    assert np.array_equal(got, (C0 * np.float32(0.5)))
    # alpha == 0: A and B are not read (NaN there must not propagate)
    Anan = np.full_like(A, np.nan)
    got = run_gemm(mode, M, N, K, 0.0, Anan, B, 2.0, C0)
    assert np.array_equal(got, C0 * np.float32(2.0))
    # beta == 0: old C is not read
    Cnan = np.full_like(C0, np.nan)
    got = run_gemm(mode, M, N, K, 1.0, A, B, 0.0, Cnan)
    ref = oracle.gemm_f64(M, N, K, 1.0, A, B, 0.0, None)
    assert np.isfinite(got).all() and oracle.rel_frob(got, ref) <= TOL
    # NaN in A propagates to its row only
    Ap = A.copy()
    Ap[3, 7] = np.nan
    got = run_gemm(mode, M, N, K, 1.0, Ap, B, 0.0, C0)
    assert np.isnan(got[3]).all()
    assert np.isfinite(np.delete(got, 3, axis=0)).all()


# ------------------------------------------------------------- split/pack
@pytest.mark.parametrize("mode,prec", [("bf16x3", "bf16"), ("tf32x3", "tf32")])
@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("gen", ["uniform", "wide", "tiny"])
def test_split_pack_bit_exact(mode, prec, transpose, gen):
    from oracle import split
    rows, cols = (300, 77) if not transpose else (77, 300)
    if gen == "uniform":
        X = W.uniform(rows, cols, 5, ld=cols + 3)
    elif gen == "wide":
        X = W.wide_range(rows, cols, 6, ld=cols + 3, lo=-40, hi=40)
    else:
        X = W.scaled(W.uniform(rows, cols, 7), -120)
        X = W._with_ld(X, cols + 3, np.nan)
    planes, amax = pkg.split_pack(dev(X)[:, :cols], mode=mode, transpose=transpose)
    torch.cuda.synchronize()
    P = planes.float().cpu().numpy()
    logical = X[:, :cols]
    src = logical.T.copy() if transpose else logical
    prow, K = src.shape
    hi, lo, exps = split.split_rows(src, prow, K, prec)
    got_exps = [split.block_exponent(np.array([v], np.int32).view(np.float32)[0])
                for v in amax.cpu().numpy()]
    assert list(exps) == got_exps
    assert np.array_equal(P[0, :, :K].view(np.uint32), hi.view(np.uint32))
    assert np.array_equal(P[1, :, :K].view(np.uint32), lo.view(np.uint32))
    assert not P[:, :, K:].any()          # pitch padding is zero


# --------------------------------------------------- schedule invariance
@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3"])
def test_every_configuration(mode):
    M, N, K = 520, 390, 700
    A, B, C0 = W.uniform(M, K, 31), W.uniform(K, N, 32), W.uniform(M, N, 33)
    Ai, Bi, Ci = W.integers(M, K, 34), W.integers(K, N, 35), W.integers(M, N, 36)
    ref = oracle.gemm_f64(M, N, K, 1.5, A, B, 0.5, C0)
    refi = oracle.gemm_f64(M, N, K, 1.5, Ai, Bi, 0.5, Ci).astype(np.float32)
    for cid in range(pkg.config_count(mode)):
        got = run_gemm(mode, M, N, K, 1.5, A, B, 0.5, C0, config_id=cid)
        assert oracle.rel_frob(got, ref) <= TOL, pkg.config_get(mode, cid)
        goti = run_gemm(mode, M, N, K, 1.5, Ai, Bi, 0.5, Ci, config_id=cid)
        assert np.array_equal(goti, refi), pkg.config_get(mode, cid)


# ------------------------------------------------------ full-size configs
# Every full-size result is compared with the oracle over the whole M x N
# matrix (every 128-row tile, every column tile): one FP64 product per input
# set (about 15 s at 8192^3 on 16 host cores), then the definition's last
# step per (alpha, beta) pair.
@pytest.mark.parametrize("n", W.SQUARE_SWEEP)
def test_square_sweep(n):
    """Square sweep at full size, every mode, both (alpha, beta) pairs."""
    A, B, C0 = square_inputs(n, W.CONFIG_SWEEP)
    P = oracle.product_f64(n, n, n, A, B)
    for alpha, beta in W.ALPHA_BETA:
        ref = oracle.axpby_f64(alpha, P, beta, C0)
        for mode in MODES:
            got = run_gemm(mode, n, n, n, alpha, A, B, beta, C0)
            err = oracle.rel_frob(got, ref)
            assert err <= TOL, (mode, n, alpha, beta, err)


def test_wide_range_8192():
    """Entries sign * 2^u, u ~ U[-10, 10]: every mode, both (alpha, beta)
    pairs, the whole matrix."""
    n = 8192
    A, B, C0 = square_inputs(n, W.CONFIG_WIDE, "wide")
    P = oracle.product_f64(n, n, n, A, B)
    for alpha, beta in W.ALPHA_BETA:
        ref = oracle.axpby_f64(alpha, P, beta, C0)
        for mode in MODES:
            got = run_gemm(mode, n, n, n, alpha, A, B, beta, C0)
            err = oracle.rel_frob(got, ref)
            assert err <= TOL, (mode, alpha, beta, err)


def test_integer_8192_bit_exact():
    """Integers in [-8, 8]: every partial sum is exact in FP32, so every mode
    must give the oracle's value element by element, both (alpha, beta)
    pairs."""
    n = 8192
    A, B, C0 = square_inputs(n, W.CONFIG_WIDE, "int")
    P = oracle.product_f64(n, n, n, A, B)
    for alpha, beta in W.ALPHA_BETA:
        ref = oracle.axpby_f64(alpha, P, beta, C0).astype(np.float32)
        for mode in MODES:
            got = run_gemm(mode, n, n, n, alpha, A, B, beta, C0)
            bad = np.count_nonzero(got != ref)
            assert bad == 0, (mode, alpha, beta, bad)


@pytest.mark.parametrize("M,N,K", W.CONV_SHAPES)
def test_conv_shapes(M, N, K):
    sa, sb, _ = W.seeds(W.CONFIG_CONV)
    A, B = W.uniform(M, K, sa), W.uniform(K, N, sb)
    C0 = np.zeros((M, N), np.float32)
    ref = oracle.gemm_f64(M, N, K, 1.0, A, B, 0.0, None)
    for mode in MODES:
        got = run_gemm(mode, M, N, K, 1.0, A, B, 0.0, C0)
        assert oracle.rel_frob(got, ref) <= TOL, mode


# ------------------------------------------------------ block scaling
@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3"])
def test_scaling_keeps_tiny_and_huge_operands(mode):
    M, N, K = 300, 200, 500
    base_a, base_b = W.uniform(M, K, 41), W.uniform(K, N, 42)
    # tiny: products near 2^-120 (low parts far below the normal range unscaled)
    A, B = W.scaled(base_a, -100), W.scaled(base_b, -20)
    ref = oracle.gemm_f64(M, N, K, 1.0, A, B, 0.0, None)
    got = run_gemm(mode, M, N, K, 1.0, A, B, 0.0, np.zeros((M, N), np.float32))
    assert oracle.rel_frob(got, ref) <= TOL
    # huge: A*B overflows FP32 but alpha*A*B does not
    A, B = W.scaled(base_a, 64), W.scaled(base_b, 64)
    alpha = math.ldexp(1.0, -20)
    ref = oracle.gemm_f64(M, N, K, alpha, A, B, 0.0, None)
    got = run_gemm(mode, M, N, K, alpha, A, B, 0.0, np.zeros((M, N), np.float32))
    assert np.isfinite(got).all()
    assert oracle.rel_frob(got, ref) <= TOL


# ------------------------------------------------------- API surfaces
def test_host_buffer_entry_point():
    M, N, K = 333, 222, 444
    A, B, C0 = W.uniform(M, K, 51), W.uniform(K, N, 52), W.uniform(M, N, 53)
    ref = oracle.gemm_f64(M, N, K, 1.5, A, B, 0.5, C0)
    for mode in MODES:
        C = C0.copy()
        pkg.gemm_host(A, B, C, 1.5, 0.5, mode=mode)
        assert oracle.rel_frob(C, ref) <= TOL, mode


def test_plan_replays_in_cuda_graph():
    M, N, K = 640, 384, 1024
    A, B, C0 = W.uniform(M, K, 61), W.uniform(K, N, 62), W.uniform(M, N, 63)
    dA, dB = dev(A), dev(B)
    dC_eager, dC_graph = dev(C0), dev(C0)
    plan = pkg.Plan(M, N, K, mode="bf16x3")
    plan.execute(dA, dB, dC_eager, 1.5, 0.5)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        plan.execute(dA, dB, dC_graph, 1.0, 0.0, stream=s)     # warm-up outside capture
        torch.cuda.synchronize()
        dC_graph.copy_(dev(C0))
        with torch.cuda.graph(g, stream=s):
            plan.execute(dA, dB, dC_graph, 1.5, 0.5, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(dC_graph, dC_eager)
    plan.destroy()


def test_plan_cache_under_stream_capture():
    """A cached plan found during a capture is captured and replays
    correctly; a shape with no cached plan is refused during the capture
    (creating one would allocate) without breaking the capture."""
    M, N, K = 96, 80, 72
    A, B, C0 = W.uniform(M, K, 91), W.uniform(K, N, 92), W.uniform(M, N, 93)
    dA, dB, dC = dev(A), dev(B), dev(C0)
    dA2, dB2, dC2 = dev(W.uniform(M + 1, K, 94)), dev(W.uniform(K, N, 95)), dev(W.uniform(M + 1, N, 96))
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        pkg.gemm(dA, dB, dC, 1.0, 0.0, mode="bf16x3", stream=s)      # cached outside the capture
        torch.cuda.synchronize()
        dC.copy_(dev(C0))
        with torch.cuda.graph(g, stream=s):
            pkg.gemm(dA, dB, dC, 1.5, 0.5, mode="bf16x3", stream=s)
            with pytest.raises(pkg.GemmError) as exc:
                pkg.gemm(dA2, dB2, dC2, 1.0, 0.0, mode="bf16x3", stream=s)
            assert exc.value.status == 1 and "captured" in str(exc.value)
    g.replay()
    torch.cuda.synchronize()
    assert oracle.rel_frob(dC.cpu().numpy(), oracle.gemm_f64(M, N, K, 1.5, A, B, 0.5, C0)) <= TOL


def test_torch_tensor_api_and_views():
    M, N, K = 200, 150, 300
    A = torch.from_numpy(W.uniform(M, K + 5, 71)).cuda()[:, :K]   # ld = K + 5
    B = torch.from_numpy(W.uniform(K, N, 72)).cuda()
    C = torch.zeros(M, N, device="cuda")
    pkg.gemm(A, B, C, mode="bf16x3")
    ref = oracle.gemm_f64(M, N, K, 1.0, A.cpu().numpy(), B.cpu().numpy(), 0.0, None)
    assert oracle.rel_frob(C.cpu().numpy(), ref) <= TOL
    with pytest.raises(ValueError):
        pkg.gemm(A.t(), B, C)


def test_device_error_word_clear():
    pkg.device_error()


def test_bounded_wait_reports_timeout_and_context_survives():
    """Failure detection without a fault: a wait on a barrier nothing arrives
    on must give up after its limit and report GEMM_ERR_TIMEOUT; the device
    then still runs gemms."""
    lib = pkg.load()
    assert lib.gemm_selftest_wait_timeout() == 6
    pkg.device_error()            # cleared
    M = N = K = 256
    A, B = W.uniform(M, K, 1), W.uniform(K, N, 2)
    got = run_gemm("bf16x3", M, N, K, 1.0, A, B, 0.0, np.zeros((M, N), np.float32))
    assert oracle.rel_frob(got, oracle.gemm_f64(M, N, K, 1.0, A, B, 0.0, None)) <= TOL


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3", "bf16x6"])
@pytest.mark.parametrize("alpha,beta", W.ALPHA_BETA)
def test_host_buffer_pipelined_panels(mode, alpha, beta):
    """Host-buffer calls large enough for the row-panel pipeline (B packed
    once, panels of A and C streamed in and out while others compute)."""
    M, N, K = 1000, 300, 700
    A, B, C0 = W.uniform(M, K, 81, ld=K + 5), W.uniform(K, N, 82, ld=N + 3), W.uniform(M, N, 83, ld=N + 1)
    ref = oracle.gemm_f64(M, N, K, alpha, A, B, beta, C0)
    lib = pkg.load()

    def pinned(x):                # the pipeline runs only on page-locked buffers
        t = torch.empty(x.shape, dtype=torch.float32, pin_memory=True)
        t.numpy()[...] = x
        return t

    for make in (pinned, lambda x: torch.from_numpy(x.copy())):   # pinned, then pageable
        hA, hB, hC = make(A), make(B), make(C0)
        st = lib.gemm_f32_host(M, N, K, alpha, hA.data_ptr(), A.shape[1], hB.data_ptr(), B.shape[1],
                               beta, hC.data_ptr(), C0.shape[1], pkg.MODES[mode], None)
        assert st == 0, lib.gemm_last_error()
        C = hC.numpy()
        assert oracle.rel_frob(C, ref) <= TOL
        check_padding_untouched(C0, C, N)
    # integer inputs stay bit-exact through the pipeline
    Ai, Bi, Ci = W.integers(M, K, 84), W.integers(K, N, 85), W.integers(M, N, 86)
    hA, hB, hC = pinned(Ai), pinned(Bi), pinned(Ci)
    st = lib.gemm_f32_host(M, N, K, alpha, hA.data_ptr(), K, hB.data_ptr(), N, beta, hC.data_ptr(), N,
                           pkg.MODES[mode], None)
    assert st == 0, lib.gemm_last_error()
    assert np.array_equal(hC.numpy(), oracle.gemm_f64(M, N, K, alpha, Ai, Bi, beta, Ci).astype(np.float32))


# ------------------------------------------------------- extreme shapes
@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3", "bf16x6", "simt"])
def test_tall_skinny_many_row_tiles(mode):
    """M of 2^21 + 37 rows (16385 row tiles, a ragged last one), N and K
    just past a tile edge: the whole result against the oracle."""
    M, N, K = (1 << 21) + 37, 65, 129
    A, B, C0 = W.uniform(M, K, 301), W.uniform(K, N, 302), W.uniform(M, N, 303)
    got = run_gemm(mode, M, N, K, 1.5, A, B, 0.5, C0)
    ref = oracle.gemm_f64(M, N, K, 1.5, A, B, 0.5, C0)
    assert oracle.rel_frob(got, ref) <= TOL


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3", "bf16x6"])
def test_long_k(mode):
    """K = 2^17 + 5: 2049 k-chunks of bf16 (4097 of tf32), folded from TMEM
    every few chunks; a ragged last chunk."""
    M, N, K = 130, 131, (1 << 17) + 5
    A, B, C0 = W.uniform(M, K, 304), W.uniform(K, N, 305), W.uniform(M, N, 306)
    ref = oracle.gemm_f64(M, N, K, 1.0, A, B, -1.0, C0)
    got = run_gemm(mode, M, N, K, 1.0, A, B, -1.0, C0)
    assert oracle.rel_frob(got, ref) <= TOL


# ------------------------------------------------------------ concurrency
def test_concurrent_host_threads_and_streams():
    """Four host threads call the library at once (the calls release the
    GIL), each on its own stream with its own shapes and modes, through the
    cached-plan entry point and the host-buffer entry point: every result
    matches the oracle (plan cache and per-thread buffers are thread-safe),
    while a fifth thread pushes plans out of the cache."""
    import threading
    jobs = [("bf16x3", 300, 260, 333), ("tf32x3", 129, 257, 1060), ("bf16x6", 520, 390, 700),
            ("simt", 257, 129, 65)]
    errors, results = [], {}

    def work(t, mode, M, N, K):
        try:
            stream = torch.cuda.Stream()
            A, B, C0 = W.uniform(M, K, 400 + t), W.uniform(K, N, 410 + t), W.uniform(M, N, 420 + t)
            ref = oracle.gemm_f64(M, N, K, 1.5, A, B, 0.5, C0)
            for rep in range(3):
                with torch.cuda.stream(stream):
                    dA, dB, dC = dev(A), dev(B), dev(C0)
                    pkg.gemm(dA, dB, dC, 1.5, 0.5, mode=mode, stream=stream)
                stream.synchronize()
                results[(t, rep, "dev")] = oracle.rel_frob(dC.cpu().numpy(), ref)
                hC = C0.copy()
                pkg.gemm_host(torch.from_numpy(A), torch.from_numpy(B), torch.from_numpy(hC), 1.5, 0.5,
                              mode=mode)
                results[(t, rep, "host")] = oracle.rel_frob(hC, ref)
        except Exception as e:   # surfaced below
            errors.append((t, repr(e)))

    def churn():
        # 24 distinct shapes through the 16-plan cache: evictions while the
        # other threads hold their plans
        try:
            for i in range(24):
                M, N, K = 64 + 8 * i, 72, 40 + 4 * i
                A, B = W.uniform(M, K, 500 + i), W.uniform(K, N, 530 + i)
                dC = torch.zeros(M, N, device="cuda")
                pkg.gemm(dev(A), dev(B), dC, 1.0, 0.0, mode="bf16x3")
                torch.cuda.synchronize()
                results[("churn", i)] = oracle.rel_frob(dC.cpu().numpy(),
                                                        oracle.gemm_f64(M, N, K, 1.0, A, B, 0.0, None))
        except Exception as e:
            errors.append(("churn", repr(e)))

    threads = [threading.Thread(target=work, args=(t, *job)) for t, job in enumerate(jobs)]
    threads.append(threading.Thread(target=churn))
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    assert len(results) == 4 * 3 * 2 + 24
    assert all(err <= TOL for err in results.values()), results


# ------------------------------------------- per-execution state of plans
def _cfg_ids(mode):
    """One configuration of each kind: packed single CTA, split-K, fused-split,
    CTA pair (those the mode has)."""
    want = [dict(block_n=128, split_k=1, fused=0, cluster=1), dict(block_n=64, split_k=3, fused=0, cluster=1),
            dict(block_n=128, split_k=1, fused=1, cluster=1), dict(block_n=256, split_k=1, fused=0, cluster=2)]
    out = []
    for w in want:
        for cid in range(pkg.config_count(mode)):
            c = pkg.config_get(mode, cid)
            if all(c[k] == v for k, v in w.items()):
                out.append(cid)
                break
    return out


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3", "bf16x6"])
def test_plan_state_is_clean_between_executions(mode):
    """The block maxima and counters of a plan are cleared by the last CTA of
    each execution's gemm launch (no memset before an execution): one plan
    run on operands whose blocks need scaling (2^70 and 2^-90), then on
    ordinary ones, then on the scaled ones again gives, each time, the bits
    of a fresh plan on the same operands, for every kind of configuration."""
    M, N, K = 600, 300, 700
    base_a, base_b, C0 = W.uniform(M, K, 91), W.uniform(K, N, 92), W.uniform(M, N, 93)
    inputs = [(W.scaled(base_a, 70), W.scaled(base_b, -90)), (base_a, base_b)]
    for cid in _cfg_ids(mode):
        fresh = [run_gemm(mode, M, N, K, 1.5, a, b, 0.5, C0, config_id=cid) for a, b in inputs]
        plan = pkg.Plan(M, N, K, mode=mode, config_id=cid)
        dC = dev(C0)
        for i in (0, 1, 0, 1):
            a, b = inputs[i]
            dC.copy_(dev(C0))
            plan.execute(dev(a), dev(b), dC, 1.5, 0.5)
            torch.cuda.synchronize()
            assert np.array_equal(dC.cpu().numpy(), fresh[i]), (cid, i)
        plan.destroy()
    pkg.device_error()


# ---------------------------------------------------------- split-K sums
def _config(mode, **want):
    for cid in range(pkg.config_count(mode)):
        c = pkg.config_get(mode, cid)
        if all(c[k] == v for k, v in want.items()):
            return cid
    raise AssertionError(f"no configuration {want}")


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3", "bf16x6"])
@pytest.mark.parametrize("block_n,split_k,cluster", [(64, 3, 1), (128, 2, 1), (128, 4, 1), (256, 2, 2)])
def test_split_k_is_the_ordered_sum_of_its_splits(mode, block_n, split_k, cluster):
    """Split K: each split writes alpha times its share of the product (its
    k-chunks) as a partial sum, and the fix-up adds the partials in
    increasing split index, then beta * C.  The result must be, bit for bit,
    that FP32 sum of the shares -- each share computed by an unsplit plan of
    the same tile width on the split's range of K -- plus beta * C (beta =
    0.5: beta * C is exact, so a fused or a separate multiply-add give the
    same bits), and the same bits on each of ten executions.  Ragged M, N
    and K (partial tiles, a partial last chunk); operands in the unscaled
    range, so that every share has the same block exponents."""
    M, N, K = 333, 290, 1000
    alpha, beta = 1.25, 0.5
    A, B, C0 = W.uniform(M, K, 61), W.uniform(K, N, 62), W.uniform(M, N, 63)
    cid = _config(mode, block_n=block_n, split_k=split_k, kb=4, group_m=16, fused=0, cluster=cluster)
    one = _config(mode, block_n=block_n, split_k=1, kb=4, group_m=16, fused=0, cluster=cluster)
    dA, dB = dev(A), dev(B)
    plan = pkg.Plan(M, N, K, mode=mode, config_id=cid)
    results = []
    for _ in range(10):
        dC = dev(C0)
        plan.execute(dA, dB, dC, alpha, beta)
        torch.cuda.synchronize()
        results.append(dC.cpu().numpy())
    plan.destroy()
    for r in results[1:]:
        assert np.array_equal(r.view(np.uint32), results[0].view(np.uint32))
    # the splits' k ranges: whole chunks, ceil(chunks / split_k) a split
    bk = 32 if mode == "tf32x3" else 64
    chunks = -(-K // bk)
    per = -(-chunks // split_k)
    assert -(-chunks // per) == split_k
    total = np.zeros((M, N), np.float32)
    for s in range(split_k):
        k0, k1 = s * per * bk, min(K, (s + 1) * per * bk)
        sub = pkg.Plan(M, N, k1 - k0, K, N, N, mode=mode, config_id=one)
        dS = torch.zeros((M, N), dtype=torch.float32, device="cuda")
        sub.execute_ptrs(alpha, dA.data_ptr() + 4 * k0, dB.data_ptr() + 4 * k0 * N, 0.0, dS.data_ptr())
        torch.cuda.synchronize()
        sub.destroy()
        share = dS.cpu().numpy()
        total = share if s == 0 else (total + share).astype(np.float32)
    want = (total + (np.float32(beta) * C0).astype(np.float32)).astype(np.float32)
    assert np.array_equal(results[0].view(np.uint32), want.view(np.uint32))
    assert oracle.rel_frob(results[0], oracle.gemm_f64(M, N, K, alpha, A, B, beta, C0)) <= TOL
    pkg.device_error()


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3", "bf16x6"])
@pytest.mark.parametrize("M,N,K", [(100, 100, 300), (130, 120, 200), (300, 129, 257), (257, 385, 64)])
def test_pair_tiles_past_the_matrix(mode, M, N, K):
    """CTA-pair tiles are 256 rows high and 128 or 256 columns wide: in the
    last pair tile, the second CTA's half of the rows (or of the columns)
    can lie wholly past M (or N).  Its loads only zero-fill, and the TMA
    producer must not wait for a packed block there (there is none): every
    pair configuration gives the oracle's result, with no timeout recorded."""
    A, B, C0 = W.uniform(M, K, 71), W.uniform(K, N, 72), W.uniform(M, N, 73)
    ref = oracle.gemm_f64(M, N, K, 1.5, A, B, 0.5, C0)
    for bn in (128, 256):
        for sk in (1, 2):
            cid = _config(mode, block_n=bn, split_k=sk, kb=4, group_m=16, fused=0, cluster=2)
            got = run_gemm(mode, M, N, K, 1.5, A, B, 0.5, C0, config_id=cid)
            pkg.device_error()
            assert oracle.rel_frob(got, ref) <= TOL, (bn, sk)
