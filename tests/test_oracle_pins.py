"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test ties the oracle to something other than itself: values printed in the paper
(tests/golden/), the combinatorial formula by brute force, closed forms of integer
families, LAPACK through SciPy, algebraic invariants and the operation counts of
Section 4.2.  A plausible slip in the oracle (a dropped term, a wrong sign or index, a
transposed operand, the wrong triangle) fails at least one of them.
"""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_2307_07611_gb300 import inputs
from tests._golden import load, matrices


# --- Section 3: Hopscotch series and the combinatorial theorem ----------------------

def test_hopscotch_example_h15_order_and_lengths():
    rows = load("hopscotch_H_1_5.txt")["H_1_5"]
    printed = []
    for r in rows:
        seq, ln = r.split("|")
        printed.append((tuple(int(v) for v in seq.split()), int(ln)))
    got = oracle.hopscotch(1, 5)
    assert [s for s, _ in printed] == got
    assert [ln for _, ln in printed] == [len(s) for s in got]


def test_hopscotch_translation_example():
    blocks = load("hopscotch_translation.txt")
    h14 = [tuple(int(v) for v in r.split()) for r in blocks["H_1_4"]]
    h58 = [tuple(int(v) for v in r.split()) for r in blocks["H_5_8"]]
    assert set(oracle.hopscotch(1, 4)) == set(h14)
    assert set(oracle.hopscotch(5, 8)) == set(h58)
    assert [tuple(v + 4 for v in s) for s in oracle.hopscotch(1, 4)] == oracle.hopscotch(5, 8)


@pytest.mark.parametrize("a,b", [(1, 2), (1, 3), (2, 9), (3, 11), (1, 12)])
def test_hopscotch_count_proposition(a, b):
    seqs = oracle.hopscotch(a, b)
    assert len(seqs) == 2 ** (b - a - 1)          # Proposition "corrTranlation"
    assert len(set(seqs)) == len(seqs)
    for s in seqs:
        assert s[0] == a and s[-1] == b and list(s) == sorted(set(s))
    assert oracle.hopscotch(a, a) == []


def test_theorem_worked_example_exact():
    g = matrices("theorem_example_4x4.txt")
    t, tinv = g["T"], g["Tinv"]
    assert np.array_equal(oracle.combinatorial_unit_upper(t), tinv)
    assert np.array_equal(oracle.tri_inv(t, lower=False, unit=True), tinv)
    assert np.array_equal(oracle.tri_inv(t, lower=False, unit=False), tinv)
    # lower orientation by transposition (Section 2)
    assert np.array_equal(oracle.tri_inv(t.T, lower=True, unit=True), tinv.T)
    s, _, _ = oracle.crit_star(t)
    assert np.array_equal(s, tinv)


def test_theorem_n3_closed_form():
    # S_13 = -T_13 + T_12 T_23 (proof of the main Theorem, n = 3)
    t = np.array([[1.0, 0.3, -0.7], [0, 1, 1.9], [0, 0, 1]])
    s = oracle.tri_inv(t, lower=False, unit=True)
    assert s[0, 2] == pytest.approx(-t[0, 2] + t[0, 1] * t[1, 2], abs=1e-15)
    assert s[0, 1] == -t[0, 1] and s[1, 2] == -t[1, 2]


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("lower", [True, False])
def test_oracle_matches_combinatorial_bruteforce(n, lower):
    for seed in range(3):
        t = inputs.tri_lower(n, seed=seed, law="uniform")
        if not lower:
            t = t.T.copy()
        brute = oracle.combinatorial_tri_inv(t, lower=lower)
        x = oracle.tri_inv(t, lower=lower)
        scale = max(1.0, np.abs(brute).max())
        assert np.abs(x - brute).max() <= 1e-14 * scale * n


def test_oracle_unit_flag_ignores_stored_diagonal():
    t = inputs.tri_lower(7, seed=4)
    t_unit = t.copy()
    np.fill_diagonal(t_unit, 1.0)
    garbage = t.copy()
    np.fill_diagonal(garbage, np.nan)
    want = oracle.combinatorial_tri_inv(t_unit, lower=True)
    got = oracle.tri_inv(garbage, lower=True, unit=True)
    assert np.abs(got - want).max() < 1e-14


def test_oracle_reads_only_its_triangle():
    t = inputs.tri_lower(40, seed=2)
    p = inputs.poison_upper(t)
    assert np.array_equal(oracle.tri_inv(p, lower=True), oracle.tri_inv(t, lower=True))
    pu = inputs.poison_upper(t).T.copy()
    assert np.array_equal(oracle.tri_inv(pu, lower=False), oracle.tri_inv(t.T, lower=False))


# --- Corollary "integer closure": exact integer families -----------------------------

@pytest.mark.parametrize("n", [1, 2, 17, 130])
def test_all_ones_unit_lower_closed_form(n):
    x = oracle.tri_inv(inputs.ones_unit_lower(n), lower=True, unit=True)
    want = np.eye(n) - np.eye(n, k=-1)
    assert np.array_equal(x, want)


@pytest.mark.parametrize("vals", [(-1.0, 1.0), (-2.0, -1.0, 1.0, 2.0)])
def test_bidiagonal_closed_form(vals):
    n = 60 if len(vals) == 2 else 20
    t, b = inputs.bidiagonal_unit_lower(n, seed=5, values=vals)
    x = oracle.tri_inv(t, lower=True, unit=True)
    want = np.zeros((n, n))
    for j in range(n):
        for i in range(j, n):
            want[i, j] = (-1.0) ** (i - j) * np.prod(b[j:i])
    assert np.array_equal(x, want)


@pytest.mark.parametrize("n,half", [(64, 16), (200, 64), (257, 128)])
def test_level_nilpotent_closed_form(n, half):
    t, nmat = inputs.level_nilpotent_unit_lower(n, half, seed=3)
    assert not np.any(nmat @ nmat)
    x = oracle.tri_inv(t, lower=True, unit=True)
    assert np.array_equal(x, np.eye(n) - nmat)


def test_integer_product_family_exact():
    n = 96
    t1, n1 = inputs.level_nilpotent_unit_lower(n, 16, seed=1, lo=-1, hi=1)
    t2, n2 = inputs.level_nilpotent_unit_lower(n, 32, seed=2, lo=-1, hi=1)
    t = t1 @ t2
    want = (np.eye(n) - n2) @ (np.eye(n) - n1)
    x = oracle.tri_inv(t, lower=True, unit=True)
    assert np.array_equal(x, want)
    assert np.array_equal(x, np.round(x))


# --- invariants and an independent library routine -----------------------------------

def normwise_residual(t, x):
    n = t.shape[0]
    r = t @ x - np.eye(n)
    return np.linalg.norm(r) / (np.linalg.norm(t) * np.linalg.norm(x))


@pytest.mark.parametrize("lower", [True, False])
def test_invariants_config_law_n512(lower):
    t = inputs.tri_lower(512, seed=0, law="uniform")
    if not lower:
        t = t.T.copy()
    x = oracle.tri_inv(t, lower=lower)
    assert normwise_residual(t, x) <= 1e-13
    other = np.triu(x, 1) if lower else np.tril(x, -1)
    assert not np.any(other)
    assert np.array_equal(np.diag(x), 1.0 / np.diag(t))


def test_block_identity():
    n, h = 300, 128
    t = inputs.tri_lower(n, seed=1, law="normal")
    x = oracle.tri_inv(t)
    xa = oracle.tri_inv(t[:h, :h])
    xc = oracle.tri_inv(t[h:, h:])
    assert np.abs(x[:h, :h] - xa).max() < 1e-14
    assert np.abs(x[h:, h:] - xc).max() < 1e-14
    x21 = -xc @ t[h:, :h] @ xa
    assert np.abs(x[h:, :h] - x21).max() < 1e-13 * max(1, np.abs(x21).max())


@pytest.mark.parametrize("n", [33, 257])
@pytest.mark.parametrize("lower", [True, False])
@pytest.mark.parametrize("unit", [False, True])
def test_matches_lapack_trtrs(n, lower, unit):
    t = inputs.tri_lower(n, seed=n, law="normal")
    if not lower:
        t = t.T.copy()
    want = sla.solve_triangular(t, np.eye(n), lower=lower, unit_diagonal=unit)
    got = oracle.tri_inv(t, lower=lower, unit=unit)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


def test_selected_columns_equal_full():
    n = 150
    t = inputs.tri_lower(n, seed=9, law="normal")
    cols = [0, 1, 77, 148, 149]
    full = oracle.tri_inv(t)
    assert np.array_equal(oracle.tri_inv_cols(t, cols), full[:, cols])
    fullu = oracle.tri_inv(t.T, lower=False)
    assert np.array_equal(oracle.tri_inv_cols(t.T, cols, lower=False), fullu[cols, :].T)


def test_singular_pivot_reported():
    t = inputs.tri_lower(20, seed=1)
    t[7, 7] = 0.0
    t[12, 12] = np.inf
    with pytest.raises(oracle.SingularError) as e:
        oracle.tri_inv(t)
    assert e.value.index == 7
    x = oracle.tri_inv(t, unit=True)  # diagonal not read
    assert np.isfinite(x).all()


# --- Section 4.2: CRIT* operation counts ---------------------------------------------

@pytest.mark.parametrize("n", list(range(2, 26)))
def test_crit_star_counts_match_paper(n):
    t = np.triu(np.random.default_rng(n).uniform(-1, 1, (n, n)), 1) + np.eye(n)
    s, mults, adds = oracle.crit_star(t)
    assert mults == n * (n - 1) * (n - 2) // 6            # Eq. "phimult"
    assert adds == (n - 1) * (n - 2) * (n - 3) // 6       # Eq. "phiaddsub"
    # I_T^CRIT(m) = m(m+1)/2 + phi_x + phi_pm = (m^3 - 3m^2 + 8m - 3)/3
    assert 3 * (n * (n + 1) // 2 + mults + adds) == n ** 3 - 3 * n ** 2 + 8 * n - 3
    assert np.abs(s - oracle.tri_inv(t, lower=False, unit=True)).max() < 1e-12


@pytest.mark.parametrize("n", [3, 6, 11])
def test_bordered_block_inverse(n):
    # Section 3, proof of the main Theorem: [R v; 0 1]^-1 = [S -S v; 0 1] with S = R^-1
    g = np.random.default_rng(20 + n)
    r = np.triu(g.uniform(-1, 1, (n, n)), 1) + np.eye(n)
    v = g.uniform(-1, 1, n)
    big = np.zeros((n + 1, n + 1))
    big[:n, :n] = r
    big[:n, n] = v
    big[n, n] = 1.0
    s = oracle.tri_inv(r, lower=False, unit=True)
    x = oracle.tri_inv(big, lower=False, unit=True)
    assert np.allclose(x[:n, :n], s, rtol=0, atol=1e-13)
    assert np.allclose(x[:n, n], -s @ v, rtol=0, atol=1e-13)
    assert x[n, n] == 1.0 and not np.any(x[n, :n])


@pytest.mark.parametrize("m", range(2, 12))
def test_combrit_star_total_count_closed_form(m):
    # Section 4.1: sum_{j=2}^{m} (m - j + 1)(j + 2) 2^(j-3) = m/2 (2^m - 2), in exact integers
    # (times 2 to clear the 2^-1 of j = 2)
    lhs2 = sum((m - j + 1) * (j + 2) * 2 ** (j - 2) for j in range(2, m + 1))
    assert lhs2 == m * (2 ** m - 2)


def test_crit_total_flops_small_values():
    f = lambda m: (m ** 3 - 3 * m ** 2 + 8 * m - 3) // 3
    assert f(3) == 7 and f(4) == 15


# --- Section 5 / 6.1: Crout (SKUL) factors and the general inverse ------------------

def test_skul_printed_factors():
    g = matrices("skul_sqr_5x5.txt")
    lo, up = oracle.crout(g["A"])
    assert np.abs(lo - g["L"]).max() < 1.5e-4
    assert np.abs(up - g["U"]).max() < 1.5e-4
    assert np.abs(oracle.tri_inv(up, lower=False, unit=True) - g["S"]).max() < 1.5e-4
    assert np.abs(oracle.tri_inv(lo, lower=True) - g["K"]).max() < 1.5e-4
    # A^-1 = S K
    assert np.abs(oracle.gen_inv(g["A"]) - g["S"] @ g["K"]).max() < 2e-4


def test_sqr_printed_r_inverse():
    g = matrices("skul_sqr_5x5.txt")
    assert np.abs(oracle.tri_inv(g["R"], lower=False) - g["S_R"]).max() < 1.5e-4


def test_skul_algorithm_printed_example():
    # Algorithm SKUL run as printed reproduces the four factors of the example (Section 6.1)
    g = matrices("skul_sqr_5x5.txt")
    lo, up, s, k = oracle.skul(g["A"])
    for name, got in (("L", lo), ("U", up), ("S", s), ("K", k)):
        assert np.abs(got - g[name]).max() < 1.5e-4, name


def test_sqr_algorithm_printed_example():
    # Algorithm SQR reproduces the printed Q, R and S = R^-1 (Section 6.1); the printed A
    # carries 4 decimals, so R (entries up to 4.8) agrees to about 1.5e-4.
    g = matrices("skul_sqr_5x5.txt")
    q, r, s = oracle.sqr(g["A"])
    assert np.abs(q - g["Q"]).max() < 1.5e-4
    assert np.abs(r - g["R"]).max() < 2e-4
    assert np.abs(s - g["S_R"]).max() < 1.5e-4


@pytest.mark.parametrize("n", [1, 2, 9, 70])
def test_skul_factors_invariants(n):
    a = inputs.general(n, seed=40 + n, dtype=np.float64)
    lo, up, s, k = oracle.skul(a)
    assert np.abs(lo @ up - a).max() < 1e-13 * max(1.0, np.abs(a).max())
    assert not np.any(np.triu(lo, 1)) and not np.any(np.tril(up, -1))
    assert not np.any(np.tril(s, -1)) and not np.any(np.triu(k, 1))
    assert np.array_equal(np.diag(up), np.ones(n)) and np.array_equal(np.diag(s), np.ones(n))
    eye = np.eye(n)
    # S = U^-1 and K = L^-1 against LAPACK's triangular solves
    assert np.abs(s - sla.solve_triangular(up, eye, lower=False, unit_diagonal=True)).max() < 1e-13
    want_k = sla.solve_triangular(lo, eye, lower=True)
    assert np.abs(k - want_k).max() <= 1e-13 * np.abs(want_k).max()
    want = np.linalg.inv(a)
    assert np.abs(s @ k - want).max() <= 1e-12 * np.abs(want).max()


def test_skul_singular_pivot():
    # the leading 2 x 2 block is singular: L_11 = 4 - 2 * 2 = 0 exactly, so SKUL stops at
    # row 1 (the algorithm's "stop" on a zero pivot)
    a = np.array([[1.0, 2.0, 3.0], [2.0, 4.0, 7.0], [1.0, 1.0, 1.0]])
    with pytest.raises(oracle.SingularError) as e:
        oracle.skul(a)
    assert e.value.index == 1
    with pytest.raises(oracle.SingularError) as e:
        oracle.skul(np.zeros((3, 3)))
    assert e.value.index == 0


@pytest.mark.parametrize("n", [1, 3, 16, 64])
def test_sqr_factors_invariants(n):
    a = inputs.general(n, seed=80 + n, dtype=np.float64)
    q, r, s = oracle.sqr(a)
    eye = np.eye(n)
    assert np.abs(q @ r - a).max() < 1e-13 * max(1.0, np.abs(a).max())
    assert np.abs(q.T @ q - eye).max() < 1e-12
    assert not np.any(np.tril(r, -1)) and np.all(np.diag(r) > 0)
    # the QR with a positive diagonal is unique: LAPACK's Householder QR, signs fixed
    qh, rh = np.linalg.qr(a)
    sg = np.sign(np.diag(rh))
    assert np.abs(q - qh * sg).max() < 1e-11
    assert np.abs(r - sg[:, None] * rh).max() < 1e-11 * np.abs(rh).max()
    assert np.abs(s - sla.solve_triangular(r, eye, lower=False)).max() < 1e-12 * np.abs(s).max()
    want = np.linalg.inv(a)
    assert np.abs(s @ q.T - want).max() <= 1e-11 * np.abs(want).max()


def test_sqr_rank_deficient_column():
    a = np.random.default_rng(5).standard_normal((4, 4))
    a[:, 2] = 2.0 * a[:, 0] - a[:, 1]    # column 2 in the span of columns 0 and 1
    with pytest.raises(oracle.SingularError):
        oracle.sqr(np.zeros((3, 3)))
    q, r, s = None, None, None
    try:
        q, r, s = oracle.sqr(a)
    except oracle.SingularError as e:
        assert e.index == 2
    else:                                 # rounding may leave a tiny nonzero R_22
        assert abs(r[2, 2]) < 1e-12 * np.abs(r).max()


@pytest.mark.parametrize("n", [1, 7, 120])
def test_gen_inv_matches_lapack(n):
    a = inputs.general(n, seed=n, dtype=np.float64)
    lo, up = oracle.crout(a)
    assert np.abs(lo @ up - a).max() < 1e-13
    assert not np.any(np.triu(lo, 1)) and not np.any(np.tril(up, -1))
    assert np.array_equal(np.diag(up), np.ones(n))
    x = oracle.gen_inv(a)
    want = np.linalg.inv(a)
    assert np.abs(x - want).max() <= 1e-12 * np.abs(want).max()


def test_gen_inv_singular_leading_block():
    a = inputs.general(6, seed=1, dtype=np.float64)
    a[0, 0] = 0.0
    with pytest.raises(oracle.SingularError) as e:
        oracle.gen_inv(a)
    assert e.value.index == 0


# --- adjoint: dT = -P(X^T G X^T) ------------------------------------------------------

def _loss(t, w, lower, unit):
    x = sla.solve_triangular(t, np.eye(t.shape[0]), lower=lower, unit_diagonal=unit)
    return float(np.sum(w * x))


@pytest.mark.parametrize("lower,unit,n", [(True, False, 32), (False, False, 16), (True, True, 16)])
def test_tri_grad_central_differences(lower, unit, n):
    t = inputs.tri_lower(n, seed=11, law="uniform")
    if not lower:
        t = t.T.copy()
    w = np.random.default_rng(12).standard_normal((n, n))
    x = sla.solve_triangular(t, np.eye(n), lower=lower, unit_diagonal=unit)
    got = oracle.tri_grad(x, w, lower=lower, unit=unit)
    fd = np.zeros((n, n))
    for i, j in itertools.product(range(n), range(n)):
        free = (i >= j) if lower else (i <= j)
        if unit and i == j:
            free = False
        if not free:
            continue
        h = 1e-6 * max(1.0, abs(t[i, j]))
        tp, tm = t.copy(), t.copy()
        tp[i, j] += h
        tm[i, j] -= h
        fd[i, j] = (_loss(tp, w, lower, unit) - _loss(tm, w, lower, unit)) / (2 * h)
    assert np.linalg.norm(got - fd) <= 1e-7 * np.linalg.norm(fd)
    outside = np.triu(got, 1) if lower else np.tril(got, -1)
    assert not np.any(outside)


def test_tri_grad_ignores_other_triangle_of_g():
    n = 24
    t = inputs.tri_lower(n, seed=2)
    x = oracle.tri_inv(t)
    g = np.random.default_rng(3).standard_normal((n, n))
    g2 = g.copy()
    g2[np.triu_indices(n, 1)] = 1e3
    assert np.abs(oracle.tri_grad(x, g) - oracle.tri_grad(x, g2)).max() < 1e-9


def test_prepared_view_gives_the_same_columns():
    """oracle.LowerView only shares the preparation of the lower view between requests:
    its columns are bit-identical to tri_inv_cols (lower, upper and unit views)."""
    t = inputs.tri_lower(97, seed=3, law="normal")
    cols = [0, 1, 40, 96]
    for lower, unit in ((True, False), (False, False), (True, True)):
        m = t if lower else t.T.copy()
        a = oracle.LowerView(m, lower=lower, unit=unit).cols(cols)
        b = oracle.tri_inv_cols(m, cols, lower=lower, unit=unit)
        assert np.array_equal(a, b)


def test_inverse_columns_match_gen_inv_and_solve_the_system():
    """oracle.inverse_columns (A x = e_j by a library solve) agrees with the pinned
    oracle.gen_inv (Crout, U^-1 L^-1, Section 5.1) and solves A x = e_j to FP64 rounding."""
    n = 300
    a = inputs.general(n, seed=9, dtype=np.float64)
    cols = [0, 7, 150, 299]
    x = oracle.inverse_columns(a, cols)
    full = oracle.gen_inv(a)
    assert np.abs(x - full[:, cols]).max() <= 1e-12 * np.abs(full).max()
    e = np.zeros((n, len(cols)))
    e[cols, range(len(cols))] = 1.0
    assert np.abs(a @ x - e).max() <= 1e-13



# --- Section 5.2: BRSI with gamma blocks ----------------------------------------------

def _gamma2_closed_form(a, m1):
    """The last block formula of Section 5.2 for gamma = 2 (Schur complement form):
    A^-1 = [Z, -Z A12 A22^-1; -A22^-1 A21 Z, A22^-1 A21 Z A12 A22^-1 + A22^-1] with
    Z = (A11 - A12 A22^-1 A21)^-1, computed with LAPACK inverses."""
    a11, a12, a21, a22 = a[:m1, :m1], a[:m1, m1:], a[m1:, :m1], a[m1:, m1:]
    i22 = np.linalg.inv(a22)
    z = np.linalg.inv(a11 - a12 @ i22 @ a21)
    return np.block([[z, -z @ a12 @ i22], [-i22 @ a21 @ z, i22 @ a21 @ z @ a12 @ i22 + i22]])


@pytest.mark.parametrize("n", [6, 40, 129])
def test_brsi_gamma2_matches_the_printed_block_formula(n):
    a = inputs.general(n, seed=n, dtype=np.float64)
    m1 = oracle.brsi_bounds(n, 2)[1]
    want = _gamma2_closed_form(a, m1)
    assert np.abs(oracle.brsi(a, 2, leaf=4) - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("n,gamma", [(7, 3), (50, 3), (64, 4), (97, 5), (200, 8), (16, 16)])
def test_brsi_equals_the_inverse(n, gamma):
    a = inputs.general(n, seed=n + gamma, dtype=np.float64)
    x = oracle.brsi(a, gamma, leaf=4)
    want = np.linalg.inv(a)
    assert np.abs(x - want).max() <= 1e-12 * np.abs(want).max()
    assert np.abs(a @ x - np.eye(n)).max() <= 1e-12


@pytest.mark.parametrize("gamma", [2, 3, 4])
def test_brsi_factorisation_structure(gamma):
    """A = M_0 M_1 ... M_{nb-2} L (Section 5.2, "A P = U_0 U_1 ... L"): every M_l block
    upper triangular with identity blocks where the earlier steps made the columns
    canonical, L block lower triangular with identity diagonal blocks after the first."""
    n = 45
    a = inputs.general(n, seed=3, dtype=np.float64)
    b, ms, minvs, l_ = oracle.brsi_factors(a, gamma, leaf=4)
    nb = len(b) - 1
    prod = np.eye(n)
    for m in ms:
        prod = prod @ m
    assert np.abs(prod @ l_ - a).max() <= 1e-12
    for li, (m, mi) in enumerate(zip(ms, minvs)):
        assert np.abs(m @ mi - np.eye(n)).max() <= 1e-12
        for i in range(nb):
            for j in range(nb):
                blk = m[b[i]:b[i + 1], b[j]:b[j + 1]]
                if j < i:
                    assert not blk.any()                          # block upper
                if j >= nb - li and i == j:
                    assert np.array_equal(blk, np.eye(blk.shape[0]))   # canonical columns
    for i in range(nb):
        for j in range(nb):
            blk = l_[b[i]:b[i + 1], b[j]:b[j + 1]]
            if j > i:
                assert not blk.any()                              # block lower
            if i == j and i > 0:
                assert np.array_equal(blk, np.eye(blk.shape[0]))


def test_brsi_paper_example_and_permutation():
    """The 5x5 example of Section 6.1 (printed inverse factors S K), for gamma = 2..5; and
    Step 1's column permutation P_0: a matrix whose diagonal blocks are singular is
    inverted once P_0 swaps its block columns, and A^-1 = P_0 (A P_0)^-1."""
    g = matrices("skul_sqr_5x5.txt")
    for gamma in (2, 3, 4, 5):
        assert np.abs(oracle.brsi(g["A"], gamma, leaf=1) - g["S"] @ g["K"]).max() < 2e-4
    n = 40
    rng = np.random.default_rng(5)
    a = np.zeros((n, n))
    a[:20, 20:] = np.eye(20) * 2.0 + rng.standard_normal((20, 20)) / np.sqrt(n)
    a[20:, :20] = np.eye(20) * 2.0 + rng.standard_normal((20, 20)) / np.sqrt(n)
    perm = np.r_[np.arange(20, 40), np.arange(0, 20)]
    x = oracle.brsi(a, 2, perm=perm, leaf=4)
    assert np.abs(x - np.linalg.inv(a)).max() <= 1e-12 * np.abs(x).max()
    with pytest.raises(oracle.SingularError):
        oracle.brsi(a, 2, leaf=4)                                 # A_11 = 0 without P_0
