"""Pins for the FP64 gemm oracle (C = alpha*A*B + beta*C, Tiramisu paper
Section I) against facts that do not come from the oracle itself: closed forms,
exact rational arithmetic, integer arithmetic and numpy's float64 matmul."""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rel_err_exact(out, exact):
    num = sum(float((Fraction(out[i, j]) - exact[i][j]) ** 2)
              for i in range(out.shape[0]) for j in range(out.shape[1]))
    den = sum(float(exact[i][j] ** 2) for i in range(out.shape[0]) for j in range(out.shape[1]))
    return (num / den) ** 0.5 if den else num ** 0.5


def test_identity_gives_b_bit_exact():
    M = K = 37
    N = 23
    A = np.eye(M, K, dtype=np.float32)
    B = W.uniform(K, N, 11)
    out = oracle.gemm_f64(M, N, K, 1.0, A, B, 0.0, None)
    assert np.array_equal(out.astype(np.float32), B)


def test_permutation_permutes_rows_bit_exact():
    M = K = 29
    N = 17
    perm = np.random.default_rng(5).permutation(M)
    A = np.zeros((M, K), np.float32)
    A[np.arange(M), perm] = 1.0
    B = W.uniform(K, N, 12)
    out = oracle.gemm_f64(M, N, K, 1.0, A, B, 0.0, None)
    assert np.array_equal(out.astype(np.float32), B[perm])


def test_rank_one_closed_form():
    # A[i][k] = u_i, B[k][j] = v_j  =>  C = alpha*K*u_i*v_j + beta*C0 (exact for integers)
    M, N, K = 19, 13, 41
    u = np.arange(-9, -9 + M, dtype=np.float32)
    v = np.arange(3, 3 + N, dtype=np.float32) * -1
    A = np.repeat(u[:, None], K, axis=1).astype(np.float32)
    B = np.repeat(v[None, :], K, axis=0).astype(np.float32)
    C0 = W.integers(M, N, 7)
    alpha, beta = 1.5, 0.5
    out = oracle.gemm_f64(M, N, K, alpha, A, B, beta, C0)
    expect = alpha * K * np.outer(u.astype(np.float64), v.astype(np.float64)) + beta * C0
    assert np.array_equal(out, expect)
    # not symmetric in (i, j): a transposed operand would fail
    assert not np.array_equal(out[:N, :N], out[:N, :N].T)


def test_integer_inputs_exact_against_integer_matmul():
    M, N, K = 67, 45, 300
    A = W.integers(M, K, 1)
    B = W.integers(K, N, 2)
    C0 = W.integers(M, N, 3)
    exact = (A.astype(np.int64) @ B.astype(np.int64)) * 3 + C0.astype(np.int64)  # alpha=1.5,beta=.5 doubled
    out = oracle.gemm_f64(M, N, K, 1.5, A, B, 0.5, C0)
    assert np.array_equal(out * 2, exact.astype(np.float64))


@pytest.mark.parametrize("M,N,K", [(127, 129, 255), (257, 31, 33), (64, 64, 1060)])
def test_matches_numpy_float64(M, N, K):
    A = W.uniform(M, K, 21)
    B = W.uniform(K, N, 22)
    C0 = W.uniform(M, N, 23)
    out = oracle.gemm_f64(M, N, K, 1.5, A, B, 0.5, C0)
    ref = 1.5 * (A.astype(np.float64) @ B.astype(np.float64)) + 0.5 * C0.astype(np.float64)
    err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    assert err <= 1e-13


def test_brute_force_tiny_shapes_exact_rational():
    """Every M, N, K in 1..9 (ld offsets cycling through 0, 1, 3) against exact
    rational arithmetic, and primes 13, 17, 31, 33."""
    offs = itertools.cycle((0, 1, 3))
    shapes = [(m, n, k) for m in range(1, 10) for n in range(1, 10) for k in range(1, 10)]
    shapes = shapes[::7] + [(13, 17, 31), (33, 13, 17), (17, 33, 13)]
    for idx, (M, N, K) in enumerate(shapes):
        o = next(offs)
        A = W.uniform(M, K, 100 + idx, ld=K + o)
        B = W.uniform(K, N, 200 + idx, ld=N + o)
        C0 = W.uniform(M, N, 300 + idx, ld=N + o)
        out = oracle.gemm_f64(M, N, K, 1.5, A, B, -0.75, C0)
        exact = oracle.gemm_exact(M, N, K, 1.5, A, B, -0.75, C0)
        assert _rel_err_exact(out, exact) <= 1e-15, (M, N, K)


def test_blas_special_cases():
    M, N, K = 9, 7, 5
    A = W.uniform(M, K, 1)
    B = W.uniform(K, N, 2)
    C0 = W.uniform(M, N, 3)
    # beta == 0: C0 is not read (NaN must not propagate)
    Cnan = np.full((M, N), np.nan, np.float32)
    out = oracle.gemm_f64(M, N, K, 1.0, A, B, 0.0, Cnan)
    assert np.isfinite(out).all()
    # alpha == 0: A and B are not read
    Anan = np.full((M, K), np.nan, np.float32)
    out = oracle.gemm_f64(M, N, K, 0.0, Anan, B, 0.5, C0)
    assert np.array_equal(out, 0.5 * C0.astype(np.float64))
    # K == 0: C = beta*C0
    out = oracle.gemm_f64(M, N, 0, 1.0, np.zeros((M, 1), np.float32),
                          np.zeros((1, N), np.float32), 2.0, C0)
    assert np.array_equal(out, 2.0 * C0.astype(np.float64))
    # M == 0 / N == 0: empty
    assert oracle.gemm_f64(0, N, K, 1.0, A, B, 0.0, None).shape == (0, N)
    assert oracle.gemm_f64(M, 0, K, 1.0, A, B, 0.0, None).shape == (M, 0)


def test_padding_is_not_read():
    # storage arrays wider than the logical matrix carry NaN in the padding
    M, N, K = 11, 6, 9
    A = W.uniform(M, K, 1, ld=K + 3)
    B = W.uniform(K, N, 2, ld=N + 5)
    C0 = W.uniform(M, N, 3, ld=N + 1)
    out = oracle.gemm_f64(M, N, K, 1.0, A, B, 1.0, C0)
    assert np.isfinite(out).all()
    ref = A[:, :K].astype(np.float64) @ B[:, :N].astype(np.float64) + C0[:, :N]
    assert np.allclose(out, ref, rtol=1e-14, atol=0)


def test_sampled_rows_equal_full_rows():
    M, N, K = 70, 33, 50
    A = W.uniform(M, K, 1)
    B = W.uniform(K, N, 2)
    C0 = W.uniform(M, N, 3)
    full = oracle.gemm_f64(M, N, K, 1.5, A, B, 0.5, C0)
    rows = [0, 5, 69, 31]
    part = oracle.gemm_f64_rows(rows, N, K, 1.5, A, B, 0.5, C0)
    assert np.array_equal(part, full[rows])


@pytest.mark.parametrize("alpha,beta", [(1.5, 0.5), (1.0, 0.0), (0.0, 2.0), (-0.75, -1.25), (0.0, 0.0)])
def test_product_then_epilogue_equals_one_step_definition(alpha, beta):
    """Two steps (the double sums once, then alpha * P + beta * C0) give the
    one-step result bit for bit, for any (alpha, beta), with padded leading
    dimensions; beta == 0 reads no C (NaN there stays out)."""
    M, N, K = 67, 45, 93
    A = W.uniform(M, K, 21, ld=K + 3)
    B = W.uniform(K, N, 22, ld=N + 1)
    C0 = W.uniform(M, N, 23, ld=N + 2)
    P = oracle.product_f64(M, N, K, A, B)
    one = oracle.gemm_f64(M, N, K, alpha, A, B, beta, C0)
    two = oracle.axpby_f64(alpha, P, beta, C0 if beta != 0 else np.full_like(C0, np.nan))
    assert np.array_equal(one.view(np.uint64), two.view(np.uint64))
    # and P is the plain sum: numpy's float64 matmul of the widened inputs
    ref = A[:, :K].astype(np.float64) @ B[:, :N].astype(np.float64)
    assert np.allclose(P, ref, rtol=1e-13, atol=1e-13)


def test_rel_frob_metric():
    ref = np.array([[3.0, 4.0]])
    got = np.array([[3.0, 4.0 + 5e-3]], np.float32)
    assert abs(oracle.rel_frob(got, ref) - float(np.float32(4.0 + 5e-3) - 4.0) / 5.0) < 1e-12
    zero = np.zeros((2, 2))
    assert oracle.rel_frob(np.zeros((2, 2), np.float32), zero) == 0.0
    assert oracle.rel_frob(np.ones((2, 2), np.float32), zero) == 2.0


def test_golden_worked_example():
    """Hand-checkable 2x3 * 3x2 example stored as text (exact rationals)."""
    path = os.path.join(GOLDEN, "gemm_2x3x2.txt")
    vals = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, rest = line.split("=", 1)
            vals[key.strip()] = rest.strip()
    A = np.array([[float(x) for x in r.split()] for r in vals["A"].split(";")], np.float32)
    B = np.array([[float(x) for x in r.split()] for r in vals["B"].split(";")], np.float32)
    C0 = np.array([[float(x) for x in r.split()] for r in vals["C0"].split(";")], np.float32)
    alpha, beta = float(vals["alpha"]), float(vals["beta"])
    expect = np.array([[float(Fraction(x)) for x in r.split()] for r in vals["C"].split(";")])
    out = oracle.gemm_f64(2, 2, 3, alpha, A, B, beta, C0)
    assert np.array_equal(out, expect)


# ------------------------------------------- FP32 evaluation of the definition
def _gamma(n: int) -> float:
    u = 2.0 ** -24
    return n * u / (1.0 - n * u)


@pytest.mark.parametrize("gen", ["uniform", "wide"])
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (1.5, -0.75), (-2.0, 1.0)])
def test_f32_seq_within_recursive_summation_bound(gen, alpha, beta):
    """Every element obeys the classical bound of recursive summation with
    rounded products, |fl(s) - s| <= gamma_(K+2) (|alpha| sum|a||b| + |beta c|)."""
    M, N, K = 37, 29, 301
    f = W.uniform if gen == "uniform" else (lambda r, c, s: W.wide_range(r, c, s, lo=-20, hi=20))
    A, B, C0 = f(M, K, 31), f(K, N, 32), f(M, N, 33)
    got = oracle.gemm_f32_seq(M, N, K, alpha, A, B, beta, C0).astype(np.float64)
    ref = oracle.gemm_f64(M, N, K, alpha, A, B, beta, C0)
    mag = abs(alpha) * (np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64)))
    if beta != 0.0:
        mag += abs(beta) * np.abs(C0.astype(np.float64))
    assert (np.abs(got - ref) <= _gamma(K + 2) * mag).all()


def test_f32_seq_rounds_every_step_in_single_precision():
    """Not a double computation rounded once: most results differ from the
    correctly rounded FP64 value, and the error is of the order u sqrt(K)."""
    M, N, K = 40, 40, 2000
    A, B = W.uniform(M, K, 41), W.uniform(K, N, 42)
    got = oracle.gemm_f32_seq(M, N, K, 1.0, A, B, 0.0, None)
    ref = oracle.gemm_f64(M, N, K, 1.0, A, B, 0.0, None)
    assert np.mean(got != ref.astype(np.float32)) > 0.5
    err = oracle.rel_frob(got, ref)
    assert 2.0 ** -24 < err < 2.0 ** -24 * 8 * np.sqrt(K)


def test_f32_seq_sums_in_increasing_k():
    """2^24 + 1 rounds back to 2^24 (ties to even) before -2^24 cancels it, so
    the increasing-k sum of [2^24, 1, -2^24] is 0 where the exact value is 1;
    in the other order the sum would be exact."""
    A = np.array([[2.0 ** 24, 1.0, -(2.0 ** 24)]], np.float32)
    B = np.ones((3, 1), np.float32)
    assert oracle.gemm_f32_seq(1, 1, 3, 1.0, A, B, 0.0, None)[0, 0] == 0.0
    assert oracle.gemm_f32_seq(1, 1, 3, 1.0, A[:, ::-1].copy(), B, 0.0, None)[0, 0] == 1.0
    assert oracle.gemm_f64(1, 1, 3, 1.0, A, B, 0.0, None)[0, 0] == 1.0


def test_f32_seq_exact_on_integers_and_blas_cases():
    M, N, K = 30, 20, 50
    A, B, C0 = W.integers(M, K, 1), W.integers(K, N, 2), W.integers(M, N, 3)
    got = oracle.gemm_f32_seq(M, N, K, 2.0, A, B, -1.0, C0)
    assert np.array_equal(got, oracle.gemm_f64(M, N, K, 2.0, A, B, -1.0, C0).astype(np.float32))
    Cnan = np.full((M, N), np.nan, np.float32)
    assert np.isfinite(oracle.gemm_f32_seq(M, N, K, 1.0, A, B, 0.0, Cnan)).all()
    Anan = np.full((M, K), np.nan, np.float32)
    assert np.array_equal(oracle.gemm_f32_seq(M, N, K, 0.0, Anan, B, 0.5, C0), C0 * np.float32(0.5))
