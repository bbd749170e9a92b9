"""Plain CPU FP64 oracle for norm-pruned block SpAMM (arXiv 2103.13042).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link this package: only the test suite, the smoke check and the CPU-baseline
leg of the benchmark use it.  It shares no code with the CUDA library; the only
module both sides use is ``synth`` (seeded input draws, no method arithmetic).

Modules
-------
spamm      block Frobenius norms (Eq. 2), recursive quadtree SpAMM (Algorithm 1),
           the flat leaf-level skip rule (Section 3.1), dense reference, errors
           (Eq. 5) and the skipped-product bounds.
precision  reduced-precision emulation: power-of-two block scaling, RNE rounding
           to BF16 / FP16 / TF32, hi+lo splits, dominant-triple flags and the
           a-priori error bound of each precision mode.
tau        valid ratio and its tau search (Section 3.5.2), the log-histogram of
           block-norm products, tau bisection on the achieved error.
mlp        the 65-64-64-1 GELU network for learned tau: forward, analytic
           backward, pinball loss, Adam, all in FP64 numpy.
general    the general statement of Section 2, C = alpha*A*B + beta*C on
           rectangular operands, and chained products for matrix powers.

Every function is pinned by ``tests/test_oracle_*.py`` against values the
paper prints (Table 1), closed forms, brute force on tiny inputs, invariants
and independent library routines.
"""
