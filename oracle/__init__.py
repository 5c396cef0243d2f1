"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg of
``bench.py`` may import this package.  The product path (``paper_2307_07611_gb300``)
never does, and this package imports nothing from it.

Two layers:

* ``oracle.c`` (compiled here with gcc): the column recurrence of CRIT (Section 4.2),
  Crout LU in SKUL's row order (Section 5.1), A^-1 = U^-1 L^-1, Algorithms SKUL and SQR
  as printed (Section 5.1) and the adjoint dT = -P(X^T G X^T).  Plain loops in binary64, no fast-math, no FMA contraction.
* NumPy pieces (matrix products as a library primitive): BRSI with gamma blocks
  (Section 5.2, the steps of BRSI(gamma): A_{l+1} = I + M_l^-1 N_l, A = M_0 ... L,
  Step 1's column permutation P_0), and columns of A^-1 by a library solve.
* Pure-Python pieces for tiny sizes: the Hopscotch series H(a, b) (Definition 3.1,
  Example "H(1,5)"), the combinatorial entry formula of the main Theorem of Section 3
  (Eq. "TMatrixInversecombinatorixFormula") and an instrumented CRIT* that counts its
  multiplications and additions (Algorithm CRIT*, Eqs. "phimult"/"phiaddsub").

Parity of the FP32 and mixed-precision GPU outputs against this oracle is a tolerance,
not bit-exactness, except on the integer families of Corollary "integer closure".
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_SO)
        i64, i32, dp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        lib.oracle_tri_inv.argtypes = [i32, i32, i64, dp, i64, dp, i64, i32]
        lib.oracle_tri_inv.restype = i64
        lib.oracle_tri_inv_cols.argtypes = [i32, i32, i64, dp, i64, i64, dp, dp, i32]
        lib.oracle_tri_inv_cols.restype = i64
        lib.oracle_view_create.argtypes = [i32, i32, i64, dp, i64]
        lib.oracle_view_create.restype = ctypes.c_void_p
        lib.oracle_view_free.argtypes = [ctypes.c_void_p]
        lib.oracle_view_free.restype = None
        lib.oracle_view_cols.argtypes = [i64, ctypes.c_void_p, i64, dp, dp, i32]
        lib.oracle_view_cols.restype = i64
        lib.oracle_crout.argtypes = [i64, dp, i64, dp, dp, i32]
        lib.oracle_crout.restype = i64
        lib.oracle_gen_inv.argtypes = [i64, dp, i64, dp, i64, i32]
        lib.oracle_gen_inv.restype = i64
        lib.oracle_skul.argtypes = [i64, dp, i64, dp, dp, dp, dp]
        lib.oracle_skul.restype = i64
        lib.oracle_sqr.argtypes = [i64, dp, i64, dp, dp, dp]
        lib.oracle_sqr.restype = i64
        lib.oracle_tri_grad.argtypes = [i32, i32, i64, dp, i64, dp, i64, dp, i64, i32]
        lib.oracle_tri_grad.restype = None
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = i32
        _lib = lib
        return lib


def max_threads() -> int:
    return int(_load().oracle_max_threads())


class SingularError(ValueError):
    def __init__(self, index: int):
        super().__init__(f"zero or non-finite pivot at index {index}")
        self.index = int(index)


def _f64_colmajor(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _check(bad: int):
    if bad == -2:
        raise MemoryError("oracle allocation failed")
    if bad >= 0:
        raise SingularError(bad)


def tri_inv(t, lower: bool = True, unit: bool = False, threads: int = 0) -> np.ndarray:
    """T^-1 in FP64 by the column recurrence.  ``t`` is a logical n x n matrix; only its
    ``lower``/upper triangle (and the diagonal unless ``unit``) is read.  Returns the full
    n x n inverse with zeros in the other triangle."""
    tc = _f64_colmajor(t)
    n = tc.shape[0]
    x = np.zeros((n, n), dtype=np.float64, order="F")
    if n == 0:
        return x
    bad = _load().oracle_tri_inv(0 if lower else 1, 1 if unit else 0, n, tc.ctypes.data, n,
                                 x.ctypes.data, n, threads)
    _check(bad)
    return np.ascontiguousarray(x)


def tri_inv_cols(t, cols, lower: bool = True, unit: bool = False, threads: int = 0) -> np.ndarray:
    """Columns ``cols`` of (lower view of T)^-1 as an n x len(cols) array.  For an upper
    T these are the rows ``cols`` of T^-1 (transposed into columns)."""
    tc = _f64_colmajor(t)
    n = tc.shape[0]
    c = np.ascontiguousarray(np.asarray(cols, dtype=np.int64))
    out = np.zeros((n, len(c)), dtype=np.float64, order="F")
    if n == 0 or len(c) == 0:
        return out
    bad = _load().oracle_tri_inv_cols(0 if lower else 1, 1 if unit else 0, n, tc.ctypes.data, n,
                                      len(c), c.ctypes.data, out.ctypes.data, threads)
    _check(bad)
    return out


class LowerView:
    """The oracle's row-major lower view of a triangular T, built once; ``cols`` then runs
    the column recurrence of ``tri_inv_cols`` for any set of columns without rebuilding it
    (the same arithmetic; only the preparation is shared between requests)."""

    def __init__(self, t, lower: bool = True, unit: bool = False):
        tc = _f64_colmajor(t)
        self.n = tc.shape[0]
        self._lib = _load()
        self._r = self._lib.oracle_view_create(0 if lower else 1, 1 if unit else 0, self.n, tc.ctypes.data,
                                               self.n) if self.n else None
        if self.n and not self._r:
            raise MemoryError("oracle allocation failed")

    def cols(self, cols, threads: int = 0) -> np.ndarray:
        c = np.ascontiguousarray(np.asarray(cols, dtype=np.int64))
        out = np.zeros((self.n, len(c)), dtype=np.float64, order="F")
        if self.n == 0 or len(c) == 0:
            return out
        _check(self._lib.oracle_view_cols(self.n, self._r, len(c), c.ctypes.data, out.ctypes.data, threads))
        return out

    def __del__(self):
        if getattr(self, "_r", None):
            self._lib.oracle_view_free(self._r)
            self._r = None


def inverse_columns(a, cols) -> np.ndarray:
    """Columns ``cols`` of A^-1 in FP64, straight from the definition: column j is the
    solution x of A x = e_j.  The solve is LAPACK's (numpy.linalg.solve: LU with partial
    pivoting, a library primitive), which costs one O(n^3) factorisation for all
    requested columns; it serves sizes where ``gen_inv`` (plain loops) would take far too
    long, and is pinned against ``gen_inv`` and the residual ``A x = e_j``."""
    a64 = np.asarray(a, dtype=np.float64)
    n = a64.shape[0]
    c = np.asarray(cols, dtype=np.int64)
    e = np.zeros((n, len(c)), dtype=np.float64)
    e[c, np.arange(len(c))] = 1.0
    return np.linalg.solve(a64, e)


def crout(a, threads: int = 0):
    """Crout LU in SKUL's order: returns (L, U) with L lower (non-unit), U unit upper."""
    ac = _f64_colmajor(a)
    n = ac.shape[0]
    lo = np.zeros((n, n), order="F")
    up = np.zeros((n, n), order="F")
    if n:
        _check(_load().oracle_crout(n, ac.ctypes.data, n, lo.ctypes.data, up.ctypes.data, threads))
    return np.ascontiguousarray(lo), np.ascontiguousarray(up)


def skul(a):
    """Algorithm SKUL (Section 5.1): returns (L, U, S, K) with A = L U (L lower, U unit
    upper), S = U^-1, K = L^-1, so A^-1 = S K.  Sequential, FP64."""
    ac = _f64_colmajor(a)
    n = ac.shape[0]
    outs = [np.zeros((n, n), order="F") for _ in range(4)]
    if n:
        _check(_load().oracle_skul(n, ac.ctypes.data, n, *[o.ctypes.data for o in outs]))
    return tuple(np.ascontiguousarray(o) for o in outs)


def sqr(a):
    """Algorithm SQR (Section 5.1): returns (Q, R, S) with A = Q R by modified
    Gram-Schmidt and S = R^-1, so A^-1 = S Q^T.  Sequential, FP64."""
    ac = _f64_colmajor(a)
    n = ac.shape[0]
    outs = [np.zeros((n, n), order="F") for _ in range(3)]
    if n:
        _check(_load().oracle_sqr(n, ac.ctypes.data, n, *[o.ctypes.data for o in outs]))
    return tuple(np.ascontiguousarray(o) for o in outs)


def gen_inv(a, threads: int = 0) -> np.ndarray:
    """A^-1 = U^-1 L^-1 from unpivoted Crout LU, all in FP64."""
    ac = _f64_colmajor(a)
    n = ac.shape[0]
    x = np.zeros((n, n), order="F")
    if n:
        _check(_load().oracle_gen_inv(n, ac.ctypes.data, n, x.ctypes.data, n, threads))
    return np.ascontiguousarray(x)


# --- BRSI with gamma blocks (Section 5.2, "Steps of BRSI(gamma)") ----------------------

def brsi_bounds(n: int, gamma: int):
    """Block boundaries of the gamma-block split: blocks of q = ceil(n / gamma) rows, the
    last one ragged; empty blocks are dropped (so n < gamma gives n blocks of one)."""
    q = -(-n // gamma) if n else 1
    b = sorted(set(min(i * q, n) for i in range(gamma + 1)))
    return b


def _block_upper_inverse(m, b, gamma, leaf):
    """Inverse of the block upper triangular M (diagonal blocks full) by block back
    substitution: X_ii = M_ii^-1 (by BRSI itself, the double recursion of Step 4), then
    for j > i, X_ij = -X_ii sum_{k=i+1}^{j} M_ik X_kj."""
    nb = len(b) - 1
    x = np.zeros_like(m)
    for i in range(nb):
        s = slice(b[i], b[i + 1])
        x[s, s] = _brsi_core(m[s, s], gamma, leaf)
    for j in range(nb):
        sj = slice(b[j], b[j + 1])
        for i in range(j - 1, -1, -1):
            si = slice(b[i], b[i + 1])
            acc = np.zeros((b[i + 1] - b[i], b[j + 1] - b[j]))
            for k in range(i + 1, j + 1):
                sk = slice(b[k], b[k + 1])
                acc += m[si, sk] @ x[sk, sj]
            x[si, sj] = -(x[si, si] @ acc)
    return x


def _block_lower_inverse(l_, b, gamma, leaf):
    """Inverse of the block lower triangular L (diagonal blocks full) by block forward
    substitution: X_ii = L_ii^-1, then for i > j, X_ij = -X_ii sum_{k=j}^{i-1} L_ik X_kj."""
    nb = len(b) - 1
    x = np.zeros_like(l_)
    for i in range(nb):
        s = slice(b[i], b[i + 1])
        x[s, s] = _brsi_core(l_[s, s], gamma, leaf)
    for j in range(nb):
        sj = slice(b[j], b[j + 1])
        for i in range(j + 1, nb):
            si = slice(b[i], b[i + 1])
            acc = np.zeros((b[i + 1] - b[i], b[j + 1] - b[j]))
            for k in range(j, i):
                sk = slice(b[k], b[k + 1])
                acc += l_[si, sk] @ x[sk, sj]
            x[si, sj] = -(x[si, si] @ acc)
    return x


def brsi_factors(a, gamma: int, leaf: int = 8):
    """The factors of Steps 2-5 of BRSI(gamma) (Section 5.2) for A (no permutation):
    returns (b, [M_0, ..., M_{nb-2}], [M_0^-1, ...], L) with A = M_0 M_1 ... M_{nb-2} L.

    For l = 0 .. nb - 2 (nb blocks of the split, boundaries b):
        A_l = M_l + N_l   (M_l: the block upper part of A_l, diagonal blocks included;
                           N_l: its strictly block lower part)
        A_{l+1} = I + M_l^-1 N_l
    N_l has a zero last block column, and so on: A_{l+1} has l + 1 trailing block columns
    that are identity columns above and on the diagonal, and M_{l+1} is the identity
    there.  After the loop L = A_{nb-1} is block lower triangular (one full diagonal
    block, the others the identity).  Diagonal blocks of the M_l are inverted by BRSI
    itself (the double recursion of Step 4)."""
    n = a.shape[0]
    b = brsi_bounds(n, gamma)
    nb = len(b) - 1
    al = np.array(a, dtype=np.float64, copy=True)
    ms, minvs = [], []
    for _ in range(nb - 1):
        m = np.zeros((n, n))
        for i in range(nb):
            for j in range(i, nb):
                m[b[i]:b[i + 1], b[j]:b[j + 1]] = al[b[i]:b[i + 1], b[j]:b[j + 1]]
        nmat = al - m
        minv = _block_upper_inverse(m, b, gamma, leaf)
        al = np.eye(n) + minv @ nmat
        ms.append(m)
        minvs.append(minv)
    return b, ms, minvs, al


def _brsi_core(a, gamma, leaf):
    """A^-1 = L^-1 M_{nb-2}^-1 ... M_0^-1 from brsi_factors.  Blocks of at most `leaf`
    rows are inverted directly by the Crout route of gen_inv (Section 5.1)."""
    n = a.shape[0]
    if n <= leaf:
        return gen_inv(a)
    b, _, minvs, l_ = brsi_factors(a, gamma, leaf)
    y = np.eye(n)
    for minv in minvs:
        y = minv @ y
    return _block_lower_inverse(l_, b, gamma, leaf) @ y


def brsi(a, gamma: int, perm=None, leaf: int = 8) -> np.ndarray:
    """A^-1 by BRSI(gamma) (Section 5.2) in FP64.  perm: the column permutation P_0 of
    Step 1 (A_0 = A P_0, column j of A_0 is column perm[j] of A; None = identity); the
    later permutations P_l are the identity.  Then A^-1 = P_0 (A P_0)^-1: row perm[j] of
    A^-1 is row j of (A P_0)^-1.  The block products are matrix products (a library
    primitive); nothing else is blocked or reordered beyond the paper's steps."""
    a = np.asarray(a, dtype=np.float64)
    n = a.shape[0]
    p = np.arange(n) if perm is None else np.asarray(perm, dtype=np.int64)
    x = _brsi_core(a[:, p], int(gamma), int(leaf))
    out = np.empty_like(x)
    out[p, :] = x
    return out


def tri_grad(x, g, lower: bool = True, unit: bool = False, threads: int = 0) -> np.ndarray:
    """dT = -P(X^T G X^T) for X = T^-1; P keeps the free entries of T."""
    xc = _f64_colmajor(x)
    gc = _f64_colmajor(g)
    n = xc.shape[0]
    d = np.zeros((n, n), order="F")
    if n:
        _load().oracle_tri_grad(0 if lower else 1, 1 if unit else 0, n, xc.ctypes.data, n,
                                gc.ctypes.data, n, d.ctypes.data, n, threads)
    return np.ascontiguousarray(d)


# ----------------------------------------------------------------------------------
# Section 3: the combinatorial formula, for tiny n (pure Python loops).
# ----------------------------------------------------------------------------------

def hopscotch(a: int, b: int):
    """The Hopscotch series H(a, b) of Definition 3.1 as a list of tuples.

    Reading of the (garbled) definition: every increasing sequence that starts at a,
    ends at b and keeps any subset of the integers strictly between them, so there are
    2^(b-a-1) sequences for a < b, and H(a, a) is empty.  Sequences are listed by the
    number of removed interior integers, then lexicographically by the removed set,
    which reproduces the order of Example "H(1,5)".
    """
    if b <= a:
        return []
    interior = list(range(a + 1, b))
    out = []
    for r in range(len(interior) + 1):
        for removed in itertools.combinations(interior, r):
            rs = set(removed)
            out.append(tuple([a] + [v for v in interior if v not in rs] + [b]))
    return out


def combinatorial_unit_upper(t) -> np.ndarray:
    """S = T^-1 for a UNIT UPPER T (paper's Eq. "defT") by the main Theorem of Section 3:
    S_ij = sum over sequences in H(i, j) of (-1)^(len-1) * prod of T over consecutive
    index pairs; S_ii = 1; 0 below the diagonal.  Indices are 1-based in the paper and
    0-based here.  Exponential cost: only for n <= 10."""
    t = np.asarray(t, dtype=np.float64)
    n = t.shape[0]
    s = np.zeros((n, n))
    for i in range(n):
        s[i, i] = 1.0
        for j in range(i + 1, n):
            total = 0.0
            for seq in hopscotch(i, j):
                prod = 1.0
                for p, q in zip(seq[:-1], seq[1:]):
                    prod *= t[p, q]
                total += (-1.0) ** (len(seq) - 1) * prod
            s[i, j] = total
    return s


def combinatorial_tri_inv(t, lower: bool = True) -> np.ndarray:
    """Brute-force T^-1 for a general non-singular triangular T (n <= 10).

    Uses the decomposition R = D T* of Section 4 (D the diagonal of R, T* unit upper):
    T*_ij = R_ij / R_ii, so R^-1 = T*^-1 D^-1, i.e. (R^-1)_ij = S*_ij / R_jj with S* from
    the combinatorial formula.  A lower T is handled through its transpose (Section 2).
    """
    r = np.asarray(t, dtype=np.float64)
    if lower:
        r = r.T
    n = r.shape[0]
    d = np.diag(r).copy()
    tstar = np.triu(r) / d[:, None]
    sstar = combinatorial_unit_upper(tstar)
    inv = sstar / d[None, :]
    return inv.T.copy() if lower else inv


def crit_star(t):
    """Algorithm CRIT* (Section 4.2) on a UNIT UPPER matrix, instrumented.

    Row by row: S_ii = 1 and, for j > i, S_ij = -S_{i,i:j-1} . T_{i:j-1,j}.  Reading A2
    of the printed loop start (j = i+2): the entry S_{i,i+1} = -T_{i,i+1} is set too.
    Counting follows Eqs. "phimult"/"phiaddsub": the leading term S_ii * T_ij = T_ij is
    a copy, so S_ij for j >= i+2 costs (j-i-1) multiplications (p = i+1..j-1) and
    (j-i-2) additions among those products; the final combination with T_ij and the
    sign are not counted.  Returns (S, multiplications, additions).
    """
    t = np.asarray(t, dtype=np.float64)
    n = t.shape[0]
    s = np.eye(n)
    mults = adds = 0
    for i in range(n):
        for j in range(i + 1, n):
            acc = None
            for p in range(i + 1, j):
                prod = s[i, p] * t[p, j]
                mults += 1
                if acc is None:
                    acc = prod
                else:
                    acc = acc + prod
                    adds += 1
            s[i, j] = -(t[i, j] + (0.0 if acc is None else acc))
    return s, mults, adds
