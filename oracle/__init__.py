"""CPU oracle for the memoized multi-amplitude contraction and linear XEB.

TEST INFRASTRUCTURE ONLY.  Nothing in the library (``paper_2108_05665_gb300``)
imports, links or executes anything here; only the tests, the smoke check and
the CPU-baseline leg of the benchmark do.  The oracle shares no code with the
CUDA path: the only common module is the seeded input generator
(``paper_2108_05665_gb300.inputs``), which holds none of the method's
arithmetic.

Parts (each module cites the passage it follows):

* ``statevec``  FP64 state-vector simulator (plain definition of <x|C|0^n>),
  in C with OpenMP, n <= 30.
* ``brute``     full 2^n x 2^n unitary from per-gate operators, n <= 6.
* ``network``   the circuit's tensor network (fused gates), the worked
  example network of App. B, and leaf projections.
* ``contract``  naive FP64 pairwise contractor with its own min-size greedy
  order (no memoization).
* ``memo``      the memoization semantics: per-node key tables by plain
  sort/dedup, Alg. 1/2 with a dictionary cache, Alg. 3/4 (eval_all / eval'),
  and the cost counters of App. C.
* ``xeb``       linear XEB, Eq. (1).

Every function is pinned in ``tests/test_oracle_*.py`` against something other
than itself (brute force, closed forms, invariants, the paper's worked
example, statistics).
"""
