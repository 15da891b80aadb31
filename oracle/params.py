"""Sample-count table of the method, in FP64 (oracle; test infrastructure only).

Restates, in the paper's notation:

* Algorithm 1, truncation length ``l = log_{1/sqrt(c)} n`` (read as the integer
  L = floor(ln n / ln(1/sqrt c)), because the loop "for i = 0 to l" runs over
  integers; Appendix B.5 scales it by p >= 1).
* Algorithm 1 / Algorithm 2, ``z = ln(2n) / (2 (eps - 3/n)^2)`` (natural log:
  only then does 2 e^{-2 z lambda^2} = 1/n hold, Appendix B.4); Appendix B.5
  generalises it to z = ln(2 n^q) / (2 (eps - 3/n^p)^2).
* Algorithm 2 line 2 / Lemma 7: |Z_l| = z sqrt(c)^l (1 - sqrt(c)),
  |Z^_l| = N_l = ceil(|Z_l|), and the rounding weight a(l) = |Z_l| / |Z^_l|.
* The pair weight of Lemma 7, a(l1) a(l2) / z, quantised to an integer number of
  2^-32 units: wq(l1, l2) = round_half_even(a(l1) * a(l2) * 2^32).

Length-0 walks are included (Algorithm 1 runs i from 0), so N_tot counts them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

TWO32 = 4294967296.0


@dataclass
class Table:
    n: int
    c: float
    eps: float
    z: float
    L: int
    N: List[int]          # N_l, l = 0..L
    P: List[int]          # stratum prefix, P[0] = 0, P[l+1] = P[l] + N[l]
    a: List[float]        # rounding weight a(l) = Z_l / N_l
    Z: List[float] = field(default_factory=list)  # expected counts |Z_l|

    @property
    def N_tot(self) -> int:
        return self.P[-1]

    def stratum(self, r: int) -> int:
        """Length l of walk r in stratum order: P[l] <= r < P[l+1]."""
        lo, hi = 0, self.L
        while lo < hi:
            mid = (lo + hi + 1) // 2
            if self.P[mid] <= r:
                lo = mid
            else:
                hi = mid - 1
        return lo

    def wq(self, l1: int, l2: int) -> int:
        """Quantised pair weight (Lemma 7) in units of 2^-32."""
        return int(round(self.a[l1] * self.a[l2] * TWO32))


def sample_table(n: int, c: float, eps: float, *, p: float = 1.0,
                 q: float = 1.0, z_override: Optional[float] = None,
                 L_override: Optional[int] = None, warmup_rule: bool = False) -> Table:
    """Build the per-length walk counts for a query on a graph of n nodes.

    Follows Algorithm 1 lines 3-5, Algorithm 2 line 2 and Appendix B.5.
    ``z_override`` / ``L_override`` replace the paper's formulas for z and the
    truncation length (used by the small configuration that fixes both).
    When z is overridden, eps is not used.  ``warmup_rule`` takes the sample
    size and truncation of the warm-up algorithm of Section 3 instead:
    z = ln(2 n^2) / (2 eps^2) and L = floor(3 log_{1/sqrt c}(n / eps)).
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    if not (0.0 < c < 1.0):
        raise ValueError("c must lie in (0, 1)")
    if p < 1.0 or q < 1.0:
        raise ValueError("p and q must be >= 1")
    rc = math.sqrt(c)
    if z_override is not None and z_override > 0:
        z = float(z_override)
    elif warmup_rule:
        if not (0.0 < eps < 1.0):
            raise ValueError("eps must lie in (0, 1)")
        z = math.log(2.0 * n * n) / (2.0 * eps * eps)
    else:
        thr = 3.0 / math.pow(n, p)
        if not (thr < eps < 1.0):
            raise ValueError("eps must satisfy 3/n^p < eps < 1")
        lam = eps - thr
        z = math.log(2.0 * math.pow(n, q)) / (2.0 * lam * lam)
    if L_override is not None and L_override >= 0:
        L = int(L_override)
    elif warmup_rule:
        if not (0.0 < eps < 1.0):
            raise ValueError("eps must lie in (0, 1)")
        L = int(math.floor(3.0 * math.log(float(n) / eps) / (-math.log(rc))))
    else:
        L = int(math.floor(p * math.log(float(n)) / (-math.log(rc))))
    N, P, a, Z = [], [0], [], []
    for l in range(L + 1):
        Zl = z * (math.pow(rc, l) * (1.0 - rc))
        Nl = int(math.ceil(Zl))
        Z.append(Zl)
        N.append(Nl)
        a.append(Zl / Nl)
        P.append(P[-1] + Nl)
    return Table(n=n, c=c, eps=eps, z=z, L=L, N=N, P=P, a=a, Z=Z)
