"""Exact SimRank and the exact expectation of the estimator (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``jeh_widom``: Eq. 1 iterated to its fixed point.  With T the row-stochastic
  in-neighbour matrix, T[u, u'] = 1/|I(u)| for u' in I(u) (a zero row when I(u)
  is empty), Eq. 1 reads S = c T S T^T off the diagonal and S(u, u) = 1.  Dense
  n x n, so only for n up to a few thousand.
* ``first_meeting``: F_k(a, b), the probability that two independent walks
  which move to a uniform in-neighbour at every step (the walks of Lemma 2
  without their stopping coin) first occupy the same node at step k >= 1.
  F_0 = I, F_k = offdiag(T F'_{k-1} T^T), F'_0 = I, F'_k = F_k.
  Lemma 2 then gives s(a, b) = sum_k c^k F_k(a, b): both sqrt(c)-walks survive
  k steps with probability c^k.
* ``estimator_expectation``: E[s~(s, u)] of the method with length strata,
  truncation at L, uniform pairing and the rounding weights of Lemma 7:
  pair j has length l2 = stratum(j) and its source walk is uniform over the
  N_tot source walks, so
  E[s~] = 1/(z N_tot) sum_{l1, l2} N_l1 N_l2 w(l1, l2) G(min(l1, l2)),
  with G(k) = sum_{i<=k} F_i(s, u) and w the pair weight (exact or quantised).
  With exact weights this is (z / N_tot) sum_k F_k (sqrt(c)^k - sqrt(c)^{L+1})^2.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .params import Table, TWO32


def transition(row_ptr: np.ndarray, col: np.ndarray, n: int) -> sp.csr_matrix:
    """Row-stochastic in-neighbour matrix T of Eq. 1 (zero rows for I(u) empty)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    deg = np.diff(row_ptr)
    rows = np.repeat(np.arange(n), deg)
    vals = np.repeat(np.where(deg > 0, 1.0 / np.maximum(deg, 1), 0.0), deg)
    return sp.csr_matrix((vals, (rows, np.asarray(col, dtype=np.int64))),
                         shape=(n, n))


def jeh_widom(row_ptr, col, n: int, c: float, tol: float = 1e-12,
              max_iter: int = 10000):
    """All-pairs SimRank by the fixed point of Eq. 1, FP64, dense.

    Iterates S_{k+1} = c T S_k T^T with the diagonal reset to 1, starting from
    S_0 = I.  The map is a contraction with factor c in the max norm, so
    stopping once max|S_{k+1} - S_k| <= tol (1 - c) / c leaves an error <= tol.
    Returns (S, iterations).
    """
    T = transition(row_ptr, col, n)
    S = np.eye(n)
    stop = tol * (1.0 - c) / c
    for it in range(1, max_iter + 1):
        TS = T @ S                       # (T S)
        S_new = c * (T @ TS.T).T         # c T S T^T
        np.fill_diagonal(S_new, 1.0)
        delta = np.max(np.abs(S_new - S))
        S = S_new
        if delta <= stop:
            return S, it
    raise RuntimeError("Jeh-Widom iteration did not converge")


def first_meeting(row_ptr, col, n: int, K: int, rows=None):
    """F_k for k = 1..K (see module doc).

    Returns an array of shape (K+1, len(rows), n) holding F_k(a, b) for a in
    ``rows`` (all nodes when None) and every b; entry k = 0 is the identity
    restricted to those rows.  The recursion runs on full n x n matrices, so
    n must stay small (a few thousand).
    """
    T = transition(row_ptr, col, n)
    rows = np.arange(n) if rows is None else np.asarray(rows)
    out = np.zeros((K + 1, rows.size, n))
    F = np.eye(n)
    out[0] = F[rows]
    for k in range(1, K + 1):
        TF = T @ F
        F = (T @ TF.T).T                 # T F' T^T
        np.fill_diagonal(F, 0.0)         # first meeting at step 0 excluded
        out[k] = F[rows]
    return out


def simrank_from_first_meeting(F: np.ndarray, c: float, diag_rows=None):
    """s = sum_{k>=1} c^k F_k (Lemma 2); 1 on the diagonal of ``diag_rows``."""
    K = F.shape[0] - 1
    w = c ** np.arange(K + 1)
    w[0] = 0.0
    S = np.tensordot(w, F, axes=1)
    if diag_rows is not None:
        for i, r in enumerate(diag_rows):
            S[i, r] = 1.0
    return S


def estimator_expectation(F_row: np.ndarray, tab: Table,
                          quantised: bool = True) -> np.ndarray:
    """E[s~(s, u)] for all u from F_k(s, u), k = 0..>=L (see module doc).

    ``F_row`` has shape (>=L+1, n).  With ``quantised`` the pair weight is the
    2^-32-quantised a(l1) a(l2) the sampler adds; otherwise the exact product.
    """
    L = tab.L
    F = F_row[:L + 1].copy()
    F[0] = 0.0                                     # step 0 never counts
    G = np.cumsum(F, axis=0)                       # G[k] = sum_{1<=i<=k} F_i
    acc = np.zeros(F_row.shape[1])
    for l1 in range(L + 1):
        for l2 in range(L + 1):
            if quantised:
                w = tab.wq(l1, l2) / TWO32
            else:
                w = tab.a[l1] * tab.a[l2]
            acc += tab.N[l1] * tab.N[l2] * w * G[min(l1, l2)]
    return acc / (tab.z * tab.N_tot)


def estimator_expectation_closed(F_row: np.ndarray, tab: Table) -> np.ndarray:
    """Closed form of the unquantised expectation (see module doc)."""
    rc = np.sqrt(tab.c)
    L = tab.L
    k = np.arange(1, L + 1)
    coef = (rc ** k - rc ** (L + 1)) ** 2
    return tab.z / tab.N_tot * np.tensordot(coef, F_row[1:L + 1], axes=1)
