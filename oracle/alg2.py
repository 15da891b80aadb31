"""Algorithm 2 of the paper, literally, for tiny graphs (oracle; test only).

Follows Sections 4.2 and 5.3-5.5 and Algorithm 2 in their order:

1. Decompose every walk into tuples (j, i, v_i, t, v_0), one per visited node
   after the start (Section 5.3): j is the walk's label after shuffling, i the
   step, v_i the node at step i, t the walk's length and v_0 its start node.
   Walks come from every node; the source's walks carry the labels of the
   shuffle (source walk sigma[j] gets label j), the other nodes' walks keep
   their stratum-order index as label.
2. Sort all tuples lexicographically (Section 5.4, Alg. 2 line 1), with the
   source's tuple placed first among tuples that share (j, i, v_i).
3. Label tuples of the source 1 and all others 0 (Alg. 2 lines 3-7).
4. PREDECESSOR: link each label-0 tuple to the closest label-1 tuple before it
   (Alg. 2 line 10); if the two share the walk label and the visited node
   (and, by the sort, the step) the walks meet (Lemma 3).
5. Send one walk-meet message (j, s, l1, u, l2) per meeting and keep one copy
   per (j, u) (Section 5.5), adding the quantised Lemma 7 weight per message.

The walks themselves come from the C oracle (``sampler.walks``), the shuffle
from ``sampler.fisher_yates``.  Returns per-node meet counts and weight sums,
which must equal the direct step-by-step comparison of ``sampler.run``.
"""
from __future__ import annotations

import numpy as np

from . import sampler
from .params import sample_table


def tuples_of_walk(j: int, walk_nodes, length: int, v0: int):
    """Decomposition of one walk {v0, v1, ..., v_t} into its tuples."""
    return [(j, i, int(v), length, v0) for i, v in enumerate(walk_nodes, 1)]


def run(row_ptr, col, n: int, s: int, c: float, eps: float, seed: int, *,
        z_override=None, L_override=None, literal_shuffle=False, shared_walks=False):
    """``literal_shuffle``: every target's walk r carries the label j with
    pi_u(j) = r (the keyed per-target permutation), as the paper shuffles
    every node's walks.  ``shared_walks``: the other nodes' walks are drawn
    with the shared key (the same walks for every source)."""
    tab = sample_table(n, c, eps, z_override=z_override, L_override=L_override)
    L, N_tot = tab.L, tab.N_tot
    lengths = np.array([tab.stratum(r) for r in range(N_tot)], dtype=np.int64)
    sigma = sampler.fisher_yates(s, seed, N_tot)
    inv = np.empty(N_tot, dtype=np.int64)
    inv[sigma] = np.arange(N_tot)          # source walk sigma[j] -> label j

    J, I, V, T, V0 = [], [], [], [], []
    for v0 in range(n):
        key = sampler.SHARED_KEY if shared_walks and v0 != s else s
        pos, eff = sampler.walks(row_ptr, col, v0, key, seed, tab)
        inv_u = None
        if literal_shuffle and v0 != s:
            inv_u = np.empty(N_tot, dtype=np.int64)
            for j in range(N_tot):
                inv_u[sampler.feistel(v0, s, seed, N_tot, j)] = j
        for r in range(N_tot):
            e = int(eff[r])
            if e == 0:
                continue
            if v0 == s:
                label = int(inv[r])
            else:
                label = int(inv_u[r]) if inv_u is not None else r
            J.append(np.full(e, label))
            I.append(np.arange(1, e + 1))
            V.append(pos[r, :e].astype(np.int64))
            T.append(np.full(e, lengths[r]))
            V0.append(np.full(e, v0))
    if not J:
        return np.zeros(n, np.uint32), np.zeros(n, np.uint64)
    J, I, V = np.concatenate(J), np.concatenate(I), np.concatenate(V)
    T, V0 = np.concatenate(T), np.concatenate(V0)

    lab = (V0 == s).astype(np.int64)       # label 1 for the source's tuples
    # lexicographic order on (j, i, v_i, source-first, t, v_0)
    order = np.lexsort((V0, T, 1 - lab, V, I, J))
    J, I, V, T, V0, lab = J[order], I[order], V[order], T[order], V0[order], lab[order]

    # PREDECESSOR: index of the closest label-1 tuple at or before each position
    idx = np.where(lab == 1, np.arange(J.size), -1)
    pred = np.maximum.accumulate(idx)
    zero = (lab == 0) & (pred >= 0)
    p = pred[zero]
    meet = (J[zero] == J[p]) & (V[zero] == V[p]) & (I[zero] == I[p])
    msg_j = J[zero][meet]
    msg_u = V0[zero][meet]
    msg_l1 = T[p][meet]
    msg_l2 = T[zero][meet]
    # one message per (j, u): a pair meeting at several steps counts once
    key = msg_j * n + msg_u
    _, first = np.unique(key, return_index=True)
    count = np.bincount(msg_u[first], minlength=n).astype(np.uint32)
    wsum = np.zeros(n, dtype=np.uint64)
    for k in first:
        wsum[msg_u[k]] += np.uint64(tab.wq(int(msg_l1[k]), int(msg_l2[k])))
    return count, wsum
