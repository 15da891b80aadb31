"""CPU oracle for single-source SimRank (arXiv 2304.04015).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, link or
run this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it.  It shares no code, header, table or
constant generator with the CUDA library; both take their inputs from
``srk_inputs`` alone.

Contents (each function cites the passage of the paper it restates):

* ``params``  -- the sample-count table of Algorithm 1 (truncation length,
  per-length walk counts N_l) and Algorithm 2 / Lemma 7 (z, |Z_l|, rounding
  weights), computed in FP64.
* ``exact``   -- exact SimRank by the Jeh-Widom fixed point of Eq. 1, the
  first-meeting decomposition behind Lemma 2, and from it the exact
  expectation of the estimator.
* ``sampler`` -- the Monte Carlo method itself, step by step (walk
  generation, shuffling/pairing, meeting detection, weighted counting),
  written in plain C with a Philox4x32-10 generator restated from its
  published definition (Salmon et al., SC'11).
* ``alg2``    -- a literal restatement of Algorithm 2 (tuples, lexicographic
  sort, labels, PREDECESSOR, deduplicated walk-meet messages) for tiny graphs.
* ``linear``  -- the truncated linearised single-source form of Appendix A
  (s = sum_t c^t (P^T)^t D P^t e_s, D = (1-c)I) in FP64, its reverse-mode
  gradient w.r.t. edge weights (torch CPU autograd) and finite differences.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
against closed forms, invariants, brute force or published test vectors; no
function is "parity unpinned".
"""
from . import params, exact  # noqa: F401

__all__ = ["params", "exact"]
