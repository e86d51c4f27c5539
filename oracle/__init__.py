"""FP64 CPU oracle for the block-randomized stochastic TR step (TEST INFRASTRUCTURE).

This package is test infrastructure only.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  The CUDA library never calls it, and it
shares no code, table or helper with the CUDA path: both sides implement the
same published definitions independently (the Philox4x32-10 counter-based
generator of Salmon et al., SC'11, and the paper's equations), and only the
seeded input generators in ``paper_2303_16492_gb300.synth`` feed both.

Modules
-------
philox  Philox4x32-10 and the integer index draws (uniform and integer-CDF).
tr      TR model definitions of Sec. 2 (element formula, unfoldings, subchain
        product / tensor, slices-Hadamard product, per-mode identity).
brsgd   One TR-BRSGD / TR-ScaledBRSGD step (Algorithm 3 with Algorithm 2),
        the four sampling distributions (Sec. 3.2), the AdaGrad rule
        (Remark after Algorithm 3), the damped preconditioner (Remark in
        Sec. 3.3), RSE (Sec. 4), the full loss/gradient (Eq. gradient) and the
        full-batch baselines used as pins.

Everything is plain numpy in float64; matrix products, Cholesky, SVD and
least squares are the library primitives used as single steps.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
(brute force, closed forms, finite differences, Monte Carlo, known-answer
vectors); none is "parity unpinned".
"""
