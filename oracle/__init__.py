"""FP64 CPU oracle for the butterfly-interaction bootstrap particle filter.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
leg of ``bench.py`` may use it.  It shares no code, header, table or constant
generator with the CUDA path under ``paper_1812_01502_gb300/``; the two meet
only in the seeded inputs of the ``synthetic`` module.

Contents (each function cites the passage of Heine, Whiteley & Cemgil,
"Parallelising particle filters with butterfly interactions", arXiv
1812.01502, that it follows):

* ``philox``      Philox4x32-7 counter-based generator (Salmon et al., SC'11)
                  and Box-Muller normals; the counter layout of the filter.
* ``butterfly``   the mixed-radix butterfly matrices A_s of Section 1.2 and
                  Lemmas 1-3, as dense matrices for small N, and the group
                  numbering of digit stages and digit sets.
* ``resample``    the integer multinomial draw shared as a *specification*
                  with the CUDA path (Algorithm 2 / Algorithm 3 line "xi ~").
* ``bpf``         the particle filter: Algorithm 1 with one stage of
                  Algorithm 3 per time step (digit k = n mod m), with all
                  stages per step (``step_all_stages``), with the paper's own
                  stage matrices (``step_digit_sets``, eq. (A matrices)), with
                  fully adapted stage skipping (``step_adaptive``, Section 1.2)
                  and as AIRPF / AIRPF2 (``step_islands``, Algorithms 4-7).
* ``kalman``      the Kalman filter (exact reference for linear-Gaussian
                  models, Section 6.1).
* ``gridfilter``  a point-mass grid filter (near-exact reference for the
                  1-D stochastic-volatility model).

Parity status (what each function is pinned to) is recorded in
``tests/test_oracle_*.py``.  Philox's bit pattern is *parity unpinned*
against published known-answer vectors (none are available offline); it is
pinned only by statistical and structural properties.
"""
