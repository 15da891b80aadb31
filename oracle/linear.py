"""FP64 oracle of the truncated linearised single-source SimRank (test only).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The linearised form of SimRank (Appendix A, Eq. for S = c P^T S P + D and its
truncation to K terms in the discussion of DISK) gives, for one source s,

    s_vec = sum_{t=0}^{L} c^t (P^T)^t D P^t e_s,

with P the column-normalised in-neighbour matrix of the edge-weighted graph:
P[u, a] = w(u -> a) / sum_{u' in I(a)} w(u' -> a) for u in I(a), and
D = (1 - c) I (a simplification the paper does not make: it estimates D).
Edge weights are indexed like the CSR ``col`` array (entry e of I(a)).

* ``forward``: the sum, evaluated term by term with scipy sparse products.
* ``forward_dense``: the same sum with dense matrix powers (tiny graphs only).
* ``grad``: d(g . s_vec)/dw by reverse-mode automatic differentiation of the
  definition written with plain torch CPU ops in FP64.
* ``finite_difference``: central differences of ``forward`` in FP64.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def column_normalised(row_ptr, col, w, n):
    """P as a scipy CSR matrix (n x n), P[u, a] = w_e / W_a."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    deg = np.diff(row_ptr)
    a_of_e = np.repeat(np.arange(n), deg)
    w = np.asarray(w, dtype=np.float64)
    Wa = np.bincount(a_of_e, weights=w, minlength=n)
    vals = w / Wa[a_of_e] if w.size else w
    return sp.csr_matrix((vals, (np.asarray(col, dtype=np.int64), a_of_e)), shape=(n, n))


def forward(row_ptr, col, w, n, s, c, L):
    """s_vec = sum_t c^t (P^T)^t D P^t e_s, D = (1 - c) I, in FP64."""
    P = column_normalised(row_ptr, col, w, n)
    PT = P.T.tocsr()
    y = np.zeros(n)
    y[s] = 1.0
    out = np.zeros(n)
    for t in range(L + 1):
        v = (1.0 - c) * y          # D P^t e_s
        for _ in range(t):
            v = PT @ v             # (P^T)^t
        out += c ** t * v
        y = P @ y                  # P^{t+1} e_s
    return out


def forward_horner(row_ptr, col, w, n, s, c, L, P=None):
    """The same sum nested as h_L = D y_L, h_t = D y_t + c P^T h_{t+1}, s_vec =
    h_0 with y_t = P^t e_s: 2L sparse products instead of O(L^2).  Used for
    finite differences; pinned equal to ``forward``."""
    if P is None:
        P = column_normalised(row_ptr, col, w, n)
    PT = P.T.tocsr()
    ys = [np.zeros(n)]
    ys[0][s] = 1.0
    for _ in range(L):
        ys.append(P @ ys[-1])
    h = (1.0 - c) * ys[L]
    for t in range(L - 1, -1, -1):
        h = (1.0 - c) * ys[t] + c * (PT @ h)
    return h


def _fd_one(args):
    row_ptr, col, w, n, s, c, L, g, e, rel_step = args
    h = rel_step * w[e]
    wp = w.copy()
    wp[e] += h
    wm = w.copy()
    wm[e] -= h
    return (g @ forward_horner(row_ptr, col, wp, n, s, c, L) -
            g @ forward_horner(row_ptr, col, wm, n, s, c, L)) / (2.0 * h)


def finite_difference_pool(row_ptr, col, w, n, s, c, L, g, edges, rel_step=1e-4,
                           processes=None):
    """``finite_difference`` with the Horner forward, spread over a process
    pool started with the spawn method."""
    import multiprocessing as mp
    w = np.asarray(w, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    args = [(row_ptr, col, w, n, s, c, L, g, int(e), rel_step) for e in edges]
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes=processes) as pool:
        return np.array(pool.map(_fd_one, args, chunksize=max(1, len(args) // 64)))


def forward_dense(row_ptr, col, w, n, s, c, L):
    """The same sum with dense matrix powers (tiny graphs)."""
    P = column_normalised(row_ptr, col, w, n).toarray()
    e = np.zeros(n)
    e[s] = 1.0
    out = np.zeros(n)
    for t in range(L + 1):
        Pt = np.linalg.matrix_power(P, t)
        out += c ** t * (Pt.T @ ((1.0 - c) * (Pt @ e)))
    return out


def grad(row_ptr, col, w, n, s, c, L, g):
    """d(g . s_vec) / dw by reverse-mode autodiff (torch CPU, FP64)."""
    import torch
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    deg = np.diff(row_ptr)
    a_idx = torch.from_numpy(np.repeat(np.arange(n), deg))
    u_idx = torch.from_numpy(np.asarray(col, dtype=np.int64))
    wt = torch.tensor(np.asarray(w, dtype=np.float64), requires_grad=True)
    Wa = torch.zeros(n, dtype=torch.float64).index_add(0, a_idx, wt)
    Pe = wt / Wa[a_idx]

    def P_apply(v):   # (P v)[u] = sum_{e: u_e = u} P_e v[a_e]
        return torch.zeros(n, dtype=torch.float64).index_add(0, u_idx, Pe * v[a_idx])

    def PT_apply(v):  # (P^T v)[a] = sum_{e in I(a)} P_e v[u_e]
        return torch.zeros(n, dtype=torch.float64).index_add(0, a_idx, Pe * v[u_idx])

    y = torch.zeros(n, dtype=torch.float64)
    y[s] = 1.0
    out = torch.zeros(n, dtype=torch.float64)
    for t in range(L + 1):
        v = (1.0 - c) * y
        for _ in range(t):
            v = PT_apply(v)
        out = out + c ** t * v
        y = P_apply(y)
    loss = (torch.from_numpy(np.asarray(g, dtype=np.float64)) * out).sum()
    loss.backward()
    return wt.grad.numpy().copy(), out.detach().numpy()


def finite_difference(row_ptr, col, w, n, s, c, L, g, edges, rel_step=1e-4):
    """Central differences of g . s_vec w.r.t. the listed edge weights."""
    w = np.asarray(w, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    out = np.empty(len(edges))
    for k, e in enumerate(edges):
        h = rel_step * w[e]
        wp = w.copy()
        wp[e] += h
        wm = w.copy()
        wm[e] -= h
        out[k] = (g @ forward(row_ptr, col, wp, n, s, c, L) -
                  g @ forward(row_ptr, col, wm, n, s, c, L)) / (2.0 * h)
    return out
