"""CPU oracle for C = alpha*A*B + beta*C and for the pieces of the split-precision
method and the cost model (FP64 unless the method fixes another precision).

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline / reference leg.  The library never imports it and
it never imports the library; the two share no code.  Inputs come from
``workloads`` (number generation only).

Modules:
  gemm   -- FP64 gemm (C shared object, OpenMP), sampled rows, error metric,
            exact rational gemm for tiny shapes.
  split  -- the operand split (power-of-two block scaling, round-to-nearest-even
            to bf16 / tf32, hi/lo planes).
  mlp    -- the cost model's MLP: forward, MSE loss, analytic backward, Adam.
  conv   -- direct 3x3 convolution (stride 1, zero padding 1), FP64 and exact.
"""
from .gemm import (build, gemm_f64, gemm_f64_rows, gemm_f32_seq, rel_frob, gemm_exact,  # noqa: F401
                   library_path, num_threads, set_num_threads, product_f64, axpby_f64)
