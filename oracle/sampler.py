"""ctypes front end of the C oracle sampler (test infrastructure only).

``build()`` compiles ``sampler.c`` with the host C compiler into
``oracle/libsrk_oracle.so`` (git-ignored).  ``run`` performs steps a1-a5 of the
method for one query: the sample-count table comes from ``oracle.params``,
steps a2-a4 from the C code, and the score of step a5 is
s~(s, u) = W_u 2^-32 / z (Algorithm 2, line 10), with s~(s, s) = 1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

from .params import Table, sample_table

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sampler.c")
_LIB = os.path.join(_HERE, "libsrk_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or \
            os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off",
               "-fPIC", "-shared", "-o", tmp, _SRC]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        i32p, u32p, u64p = P(ctypes.c_int32), P(ctypes.c_uint32), P(ctypes.c_uint64)
        L.srko_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.srko_philox4x32_10.restype = None
        L.srko_index.argtypes = [ctypes.c_uint64, ctypes.c_uint32]
        L.srko_index.restype = ctypes.c_uint32
        L.srko_philox2x32_10.argtypes = [u32p, ctypes.c_uint32, u32p]
        L.srko_philox2x32_10.restype = None
        L.srko_walk_key.argtypes = [ctypes.c_uint64, ctypes.c_uint32]
        L.srko_walk_key.restype = ctypes.c_uint32
        L.srko_bounded.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64]
        L.srko_bounded.restype = ctypes.c_uint32
        L.srko_step_index.argtypes = [ctypes.c_uint32, ctypes.c_int, ctypes.c_uint32,
                                      ctypes.c_uint32, ctypes.c_uint32]
        L.srko_step_index.restype = ctypes.c_uint32
        L.srko_walk.argtypes = [i32p, i32p, ctypes.c_int32, ctypes.c_int32,
                                ctypes.c_int32, ctypes.c_uint64, ctypes.c_int, i32p]
        L.srko_walk.restype = ctypes.c_int
        L.srko_walks.argtypes = [i32p, i32p, ctypes.c_int32, ctypes.c_int32,
                                 ctypes.c_uint64, ctypes.c_int, i32p, i32p, i32p]
        L.srko_walks.restype = None
        L.srko_fisher_yates.argtypes = [ctypes.c_int32, ctypes.c_uint64,
                                        ctypes.c_int32, i32p]
        L.srko_fisher_yates.restype = None
        L.srko_sampler.argtypes = [i32p, i32p, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_uint64, ctypes.c_int, i32p, u64p,
                                   i32p, ctypes.c_int64, u32p, u64p, u64p, u64p,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.srko_sampler.restype = ctypes.c_int
        L.srko_feistel.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                   ctypes.c_int32, ctypes.c_int32]
        L.srko_feistel.restype = ctypes.c_int32
        _lib = L
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().srko_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                             _ptr(out, ctypes.c_uint32))
    return [int(x) for x in out]


def philox2x32_10(ctr, key: int):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    out = np.zeros(2, dtype=np.uint32)
    lib().srko_philox2x32_10(_ptr(c, ctypes.c_uint32), ctypes.c_uint32(key),
                             _ptr(out, ctypes.c_uint32))
    return [int(x) for x in out]


def index(r: int, d: int) -> int:
    return int(lib().srko_index(ctypes.c_uint64(r), ctypes.c_uint32(d)))


def walk_key(seed: int, q: int) -> int:
    """kappa(seed, q), the Philox2x32-10 key of the walks of key word q."""
    return int(lib().srko_walk_key(ctypes.c_uint64(seed), ctypes.c_uint32(q & 0xFFFFFFFF)))


def bounded(w: int, d: int, r: int) -> int:
    """Lemire's bounded draw below d from the word w (r when w is rejected)."""
    return int(lib().srko_bounded(ctypes.c_uint32(w), ctypes.c_uint32(d), ctypes.c_uint64(r)))


def step_index(key: int, i: int, r: int, v: int, d: int) -> int:
    return int(lib().srko_step_index(ctypes.c_uint32(key), i, ctypes.c_uint32(r),
                                     ctypes.c_uint32(v), ctypes.c_uint32(d)))


# Key word of the shared target walks in place of the source.
SHARED_KEY = -2


def walk(row_ptr, col, v: int, r: int, s: int, seed: int, length: int):
    pos = np.full(max(length, 1), -1, dtype=np.int32)
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    eff = lib().srko_walk(_ptr(rp, ctypes.c_int32), _ptr(cl, ctypes.c_int32),
                          v, r, s, ctypes.c_uint64(seed), length,
                          _ptr(pos, ctypes.c_int32))
    return pos[:eff].copy()


def walks(row_ptr, col, v: int, s: int, seed: int, tab: Table):
    """All N_tot walks of node v (stratum order), as (pos[N_tot, L], eff)."""
    stride = max(tab.L, 1)
    pos = np.empty((tab.N_tot, stride), dtype=np.int32)
    eff = np.empty(tab.N_tot, dtype=np.int32)
    P = np.asarray(tab.P, dtype=np.int32)
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    lib().srko_walks(_ptr(rp, ctypes.c_int32), _ptr(cl, ctypes.c_int32), v, s,
                     ctypes.c_uint64(seed), tab.L, _ptr(P, ctypes.c_int32),
                     _ptr(pos, ctypes.c_int32), _ptr(eff, ctypes.c_int32))
    return pos, eff


def feistel(u: int, s: int, seed: int, N: int, j: int) -> int:
    """pi_u(j) of the literal target shuffle."""
    return int(lib().srko_feistel(u, s, ctypes.c_uint64(seed), N, j))


def fisher_yates(s: int, seed: int, N_tot: int) -> np.ndarray:
    sigma = np.empty(N_tot, dtype=np.int32)
    lib().srko_fisher_yates(s, ctypes.c_uint64(seed), N_tot,
                            _ptr(sigma, ctypes.c_int32))
    return sigma


def weight_table(tab: Table) -> np.ndarray:
    """(L+1) x (L+1) quantised pair weights wq(l1, l2) (Lemma 7)."""
    L = tab.L
    w = np.empty((L + 1, L + 1), dtype=np.uint64)
    for l1 in range(L + 1):
        for l2 in range(L + 1):
            w[l1, l2] = tab.wq(l1, l2)
    return w


@dataclass
class Result:
    table: Table
    targets: np.ndarray
    count: np.ndarray        # uint32 meet counts
    wsum: np.ndarray         # uint64 weight sums, 2^-32 units
    steps: np.ndarray        # uint64 target-walk steps per target
    source_steps: int
    scores: np.ndarray       # FP64 s~(s, u)


def run(row_ptr, col, n: int, s: int, c: float, eps: float, seed: int, *,
        targets=None, z_override=None, L_override=None, p: float = 1.0,
        q: float = 1.0, warmup_rule: bool = False, literal_shuffle: bool = False,
        shared_walks: bool = False, threads: int = 0) -> Result:
    """One single-source query, steps a1-a5, for ``targets`` (all nodes if None).
    ``literal_shuffle``: also shuffle every target's walks (by pi_u).
    ``shared_walks``: target walks keyed by (node, replica) alone, the same for
    every source (``SHARED_KEY``)."""
    tab = sample_table(n, c, eps, p=p, q=q, z_override=z_override,
                       L_override=L_override, warmup_rule=warmup_rule)
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    if targets is None:
        targets = np.arange(n, dtype=np.int32)
    targets = np.ascontiguousarray(targets, dtype=np.int32)
    k = targets.size
    count = np.zeros(k, dtype=np.uint32)
    wsum = np.zeros(k, dtype=np.uint64)
    steps = np.zeros(k, dtype=np.uint64)
    src_steps = np.zeros(1, dtype=np.uint64)
    P = np.asarray(tab.P, dtype=np.int32)
    wq = weight_table(tab)
    rc = lib().srko_sampler(_ptr(rp, ctypes.c_int32), _ptr(cl, ctypes.c_int32),
                            n, s, ctypes.c_uint64(seed), tab.L,
                            _ptr(P, ctypes.c_int32), _ptr(wq, ctypes.c_uint64),
                            _ptr(targets, ctypes.c_int32), k,
                            _ptr(count, ctypes.c_uint32),
                            _ptr(wsum, ctypes.c_uint64),
                            _ptr(steps, ctypes.c_uint64),
                            _ptr(src_steps, ctypes.c_uint64), threads,
                            1 if literal_shuffle else 0, 1 if shared_walks else 0)
    if rc != 0:
        raise MemoryError("oracle sampler ran out of memory")
    # a5: s~(s, u) = W_u 2^-32 / z; s~(s, s) = 1
    scores = wsum.astype(np.float64) * (1.0 / 4294967296.0) / tab.z
    scores[targets == s] = 1.0
    return Result(tab, targets, count, wsum, steps, int(src_steps[0]), scores)
