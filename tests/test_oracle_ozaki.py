"""Pins for the Ozaki-product oracle (Sec. "Ozaki Scheme").

Every check here compares the oracle with something other than itself: the
paper's printed counts, exact rational arithmetic, Python exact-integer
products, the exact product of integer matrices, or the correctly rounded exact
product. The planted-mistake tests show that a plausible slip in the oracle
(a dropped level, a transposed operand, a wrong digit sign) fails these pins.
"""

import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import ozaki as oz


def _rng(seed):
    return np.random.default_rng(seed)


def _mixed_matrix(m, k, seed):
    """Entries of both signs spanning many binades, plus a zero row and exact zeros."""
    rng = _rng(seed)
    A = rng.standard_normal((m, k)) * np.exp2(rng.integers(-30, 10, size=(m, k)))
    A[1, :] = 0.0
    A[2, 3] = 0.0
    A[3, :] *= 2.0 ** -400
    return A


# ----------------------------------------------------------------- paper's counts

def test_paper_product_counts(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "paper_counts.json")))
    for row in g["products_per_split_count"]:
        assert oz.product_count(row["splits"]) == row["products"], row["where"]
    for row in g["symmetric_square_products"]:
        assert oz.symmetric_square_product_count(row["splits"]) == row["products"], row["where"]
    be = g["break_even"]
    assert be["calls"] * oz.product_count(be["splits_low"]) == be["products_low"]
    assert be["calls"] * oz.product_count(be["splits_high"]) == be["products_high"]


def test_memory_factor_two_s():
    """S digit planes per operand, each the size of the operand: 2S for A and B."""
    A = _rng(0).standard_normal((6, 5))
    B = _rng(1).standard_normal((5, 4))
    for s in (1, 3, 6):
        _, DA, _ = oz.split_rows(A, s, 7)
        _, DBt, _ = oz.split_cols(B, s, 7)
        assert DA.size + DBt.size == s * (A.size + B.size)


def test_kept_pairs_are_the_levels():
    for s in range(1, 10):
        pairs = oz.kept_pairs(s)
        assert all(i + j <= s + 1 for i, j in pairs)
        assert len(set(pairs)) == len(pairs)
        assert sorted({i + j for i, j in pairs}) == list(range(2, s + 2))


# ----------------------------------------------------------------- split

def _check_split(split_rows, A, s, beta):
    e, D, res = split_rows(A, s, beta)
    m, k = A.shape
    for r in range(m):
        rowmax = max(abs(Fraction(float(v))) for v in A[r])
        if rowmax == 0:
            assert e[r] == 0
        else:
            assert rowmax < Fraction(2) ** int(e[r]) <= 2 * rowmax
        for c in range(k):
            x = Fraction(float(A[r, c])) / Fraction(2) ** int(e[r])
            # digits are the beta-bit expansion of |x| carrying the sign of x
            sign = -1 if x < 0 else 1
            ax = abs(x)
            prev = 0
            for i in range(1, s + 1):
                whole = int(ax * 2 ** (beta * i))  # floor of a nonnegative rational
                digit = whole - prev * 2 ** beta
                prev = whole
                assert D[i - 1, r, c] == sign * digit
                assert abs(D[i - 1, r, c]) <= 2 ** beta - 1
            # exact reconstruction with the residual
            recon = sum(Fraction(int(D[i, r, c])) / Fraction(2) ** (beta * (i + 1)) for i in range(s))
            recon += Fraction(float(res[r, c])) / Fraction(2) ** (beta * s)
            assert recon * Fraction(2) ** int(e[r]) == Fraction(float(A[r, c]))
            assert abs(res[r, c]) < 1.0


@pytest.mark.parametrize("beta", [7, 8])
@pytest.mark.parametrize("s", [1, 3, 7])
def test_split_matches_exact_expansion(beta, s):
    A = _mixed_matrix(5, 9, seed=11 + s + beta)
    _check_split(oz.split_rows, A, s, beta)


def test_split_cols_is_split_of_transpose():
    B = _mixed_matrix(7, 6, seed=3)
    f, DBt, _ = oz.split_cols(B, 4, 7)
    e, DT, _ = oz.split_rows(B.T.copy(), 4, 7)
    assert np.array_equal(f, e) and np.array_equal(DBt, DT)


def test_split_rejects_nonfinite():
    A = np.ones((3, 3))
    A[1, 1] = np.nan
    with pytest.raises(ValueError):
        oz.split_rows(A, 3, 7)


# ----------------------------------------------------------------- level sums

def _brute_levels(DA, DBt):
    s, m, k = DA.shape
    n = DBt.shape[1]
    out = {}
    for L in range(2, s + 2):
        S = [[0] * n for _ in range(m)]
        for i in range(1, s + 1):
            j = L - i
            if not (1 <= j <= s):
                continue
            for r in range(m):
                for c in range(n):
                    S[r][c] += sum(int(DA[i - 1, r, t]) * int(DBt[j - 1, c, t]) for t in range(k))
        out[L] = S
    return out


def _check_levels(level_sums, A, B, s, beta):
    _, DA, _ = oz.split_rows(A, s, beta)
    _, DBt, _ = oz.split_cols(B, s, beta)
    got = level_sums(DA, DBt, beta)
    want = _brute_levels(DA, DBt)
    assert sorted(got) == sorted(want)
    for L in want:
        assert np.array_equal(got[L], np.array(want[L], dtype=np.int64)), L


@pytest.mark.parametrize("s,beta", [(3, 7), (5, 8), (6, 7)])
def test_level_sums_equal_exact_integer_products(s, beta):
    A = _mixed_matrix(5, 7, seed=21)
    B = _mixed_matrix(7, 4, seed=22)
    _check_levels(oz.level_sums, A, B, s, beta)


# ----------------------------------------------------------------- full product

def _exact_product(A, B):
    m, k = A.shape
    n = B.shape[1]
    return [[sum(Fraction(float(A[r, t])) * Fraction(float(B[t, c])) for t in range(k)) for c in range(n)]
            for r in range(m)]


def _check_bound(gemm, A, B, s, beta):
    C, parts = gemm(A, B, s, beta, return_parts=True)
    exact = _exact_product(A, B)
    bound = oz.truncation_bound(parts["e"], parts["f"], A.shape[1], s, beta)
    for r in range(A.shape[0]):
        for c in range(B.shape[1]):
            err = abs(Fraction(float(C[r, c])) - exact[r][c])
            assert err <= Fraction(float(bound[r, c])), (r, c, float(err), bound[r, c])


@pytest.mark.parametrize("s,beta", [(2, 7), (4, 7), (3, 8), (6, 7)])
def test_error_within_truncation_bound(s, beta):
    A = _mixed_matrix(6, 8, seed=31)
    B = _mixed_matrix(8, 5, seed=32)
    _check_bound(oz.ozaki_gemm, A, B, s, beta)


def test_integer_matrices_are_exact():
    """Entries that are integers below 2^beta need one slice: the product is exact."""
    rng = _rng(5)
    A = rng.integers(-127, 128, size=(9, 11)).astype(np.float64)
    B = rng.integers(-127, 128, size=(11, 6)).astype(np.float64)
    A[:, 0] = 127.0
    B[0, :] = -100.0
    want = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    for s in (1, 2, 5):
        assert np.array_equal(oz.ozaki_gemm(A, B, s, 7), want)


def test_full_coverage_is_correctly_rounded():
    """With beta*s >= 70 on nonnegative inputs (the random [0, 1] matrices of
    Fig. 3), the result is within 2 ulp of the correctly rounded exact product."""
    rng = _rng(6)
    A = rng.random((6, 10))
    B = rng.random((10, 5))
    C = oz.ozaki_gemm(A, B, 10, 7)
    exact = _exact_product(A, B)
    for r in range(6):
        for c in range(5):
            ref = float(exact[r][c])
            assert abs(C[r, c] - ref) <= 2 * np.spacing(ref), (r, c)


def test_error_falls_with_splits():
    """Fig. 3: the error of the product of random [0, 1] matrices falls with the
    number of splits until it reaches the FP64 floor."""
    rng = _rng(7)
    A = rng.random((40, 64))
    B = rng.random((64, 30))
    ref = np.array(_exact_product_float(A, B))
    errs = [np.linalg.norm(oz.ozaki_gemm(A, B, s, 7) - ref) for s in range(1, 10)]
    for a, b in zip(errs, errs[1:]):
        assert b <= a or b < 1e-12
    assert errs[0] > 1e-3 and errs[-1] < 1e-12


def _exact_product_float(A, B):
    return [[float(v) for v in row] for row in _exact_product(A, B)]


def _exact_level_value(S, s, beta, r, c):
    return sum(Fraction(int(S[L][r, c]), 2 ** (beta * L)) for L in range(2, s + 2))


@pytest.mark.parametrize("s", [1, 3, 4, 5, 7, 8])
def test_recombination_is_correctly_rounded_up_to_two_groups(s):
    """With at most two exactly combined groups of levels (s <= 8, beta = 7)
    the float64 result is the correctly rounded exact sum of the level sums."""
    beta = 7
    rng = np.random.default_rng(40 + s)
    S = {L: rng.integers(-(2 ** 30), 2 ** 30, size=(6, 5), dtype=np.int64) for L in range(2, s + 2)}
    C = oz.recombine(S, np.zeros(6, dtype=np.int64), np.zeros(5, dtype=np.int64), s, beta)
    for r in range(6):
        for c in range(5):
            assert C[r, c] == float(_exact_level_value(S, s, beta, r, c))


def test_recombination_three_groups_smallest_first():
    """s = 10 gives three groups (levels 11..8, 7..4, 3..2), added smallest
    first. The largest group is (2^37 - 1) 2^-21 with ulp 2^-37; the other two
    are worth 0.375 and 0.25 of that ulp. Added first, they sum exactly to 0.625
    ulp and round the result up by one ulp; added last, each would be rounded
    away."""
    s, beta = 10, 7
    S = {L: np.zeros((1, 1), dtype=np.int64) for L in range(2, s + 2)}
    S[2][0, 0] = 2 ** 30 - 1
    S[3][0, 0] = 127           # group (3, 2): T = 2^37 - 1, value T 2^-21
    S[7][0, 0] = 3 * 2 ** 9    # group (7..4): value 3 2^-40 = 0.375 ulp
    S[8][0, 0] = 2 ** 17       # group (11..8): T = 2^38, value 2^-39 = 0.25 ulp
    C = oz.recombine(S, np.array([0]), np.array([0]), s, beta)
    g3 = (2 ** 37 - 1) * 2.0 ** -21
    assert C[0, 0] == g3 + 2.0 ** -37
    assert (g3 + 3 * 2.0 ** -40) + 2.0 ** -39 == g3  # the other order would lose both


# ----------------------------------------------------------------- planted mistakes

def test_planted_dropped_level_fails_the_bound():
    def gemm_drop_level(A, B, s, beta, return_parts=False):
        C, parts = oz.ozaki_gemm(A, B, s, beta, return_parts=True)
        S = dict(parts["S"])
        S[s + 1] = np.zeros_like(S[s + 1])
        S[2] = S[2] * 0  # a dropped leading level
        C = oz.recombine(S, parts["e"], parts["f"], s, beta)
        return (C, parts) if return_parts else C

    A = _mixed_matrix(6, 8, seed=41)
    B = _mixed_matrix(8, 5, seed=42)
    with pytest.raises(AssertionError):
        _check_bound(gemm_drop_level, A, B, 4, 7)


def test_planted_transposed_operand_fails_brute_force():
    def levels_transposed(DA, DBt, beta):
        s = DA.shape[0]
        out = {}
        for L in range(2, s + 2):
            acc = np.zeros((DA.shape[1], DBt.shape[1]))
            for i in range(1, L):
                j = L - i
                if i <= s and j <= s:
                    acc = acc + DA[i - 1].astype(np.float64) @ DBt[j - 1].astype(np.float64)  # missing .T
            out[L] = acc.astype(np.int64)
        return out

    A = _mixed_matrix(5, 5, seed=51)
    B = _mixed_matrix(5, 5, seed=52)
    with pytest.raises(AssertionError):
        _check_levels(levels_transposed, A, B, 3, 7)


def test_planted_wrong_digit_sign_fails_reconstruction():
    def split_abs(A, s, beta):
        e, D, res = oz.split_rows(A, s, beta)
        return e, np.abs(D), res

    A = _mixed_matrix(4, 6, seed=61)
    with pytest.raises(AssertionError):
        _check_split(split_abs, A, 3, 7)


# ----------------------------------------------------------------- nearest digits (E4M3 mode)

def _e4m3_values():
    """Every finite value of the FP8 format E4M3 (sign, 4 exponent bits with
    bias 7, 3 fraction bits; exponent field 0 is subnormal; S.1111.111 is NaN)."""
    vals = set()
    for code in range(256):
        sign = -1 if code & 0x80 else 1
        ex = (code >> 3) & 0xF
        fr = code & 0x7
        if ex == 0xF and fr == 0x7:
            continue
        v = Fraction(fr, 8) * Fraction(2) ** -6 if ex == 0 else (1 + Fraction(fr, 8)) * Fraction(2) ** (ex - 7)
        vals.add(sign * v)
    return vals


def test_nearest_digits_are_exact_in_e4m3():
    """Sec. "Ozaki Scheme": slices must multiply without error on the hardware;
    every nearest digit of beta = 5 (|d| <= 16) is an E4M3 value, 17 is not."""
    vals = _e4m3_values()
    assert oz.max_digit(oz.BETA["e4m3"], oz.ROUNDING["e4m3"]) == 16
    assert all(Fraction(d) in vals for d in range(-16, 17))
    assert Fraction(17) not in vals


def _tie_matrix():
    """Rows whose scaled entries hit the digit rule's edges: ties (y = k + 1/2
    of both signs, even and odd k) and a first digit of 16. Row max 1.96875:
    e = 2, x = a / 4, y = 32 x = 8 a."""
    A = np.array([
        [1.96875, 0.4375, -0.4375, 0.3125, -0.3125, 0.0625, 2.0 ** -40],
        [1.5, -1.96875 + 2.0 ** -30, 0.1875, -0.1875, 1.0 / 3.0, -2.0 / 7.0, 0.0],
    ])
    return A


def _check_nearest_split(split_rows, A, s, beta):
    e, D, res = split_rows(A, s, beta, "nearest")
    m, k = A.shape
    half = Fraction(1, 2)
    for r in range(m):
        rowmax = max(abs(Fraction(float(v))) for v in A[r])
        if rowmax == 0:
            assert e[r] == 0
        else:
            assert 2 * rowmax < Fraction(2) ** int(e[r]) <= 4 * rowmax
        for c in range(k):
            x = Fraction(float(A[r, c])) / Fraction(2) ** int(e[r])
            assert -half < x < half
            for i in range(s):
                y = x * 2 ** beta
                d = int(D[i, r, c])
                # d = floor(y + 1/2) is the one integer with y - d in [-1/2, 1/2)
                assert -half <= y - d < half, (r, c, i, y, d)
                assert abs(d) <= 2 ** (beta - 1)
                x = y - d
            assert Fraction(float(res[r, c])) == x
            recon = sum(Fraction(int(D[i, r, c])) / Fraction(2) ** (beta * (i + 1)) for i in range(s))
            recon += x / Fraction(2) ** (beta * s)
            assert recon * Fraction(2) ** int(e[r]) == Fraction(float(A[r, c]))


@pytest.mark.parametrize("s", [1, 3, 7, 12])
def test_nearest_split_matches_digit_rule(s):
    _check_nearest_split(oz.split_rows, _mixed_matrix(5, 9, seed=70 + s), s, 5)
    _check_nearest_split(oz.split_rows, _tie_matrix(), s, 5)


def test_nearest_tie_and_edge_digits():
    """The tie matrix's first digits, worked by hand: y = 8 a."""
    e, D, _ = oz.split_rows(_tie_matrix(), 2, 5, "nearest")
    assert list(e) == [2, 2]
    # 1.96875 -> y = 15.75 -> 16; +-0.4375 -> y = +-3.5 -> 4 and -3 (ties upward);
    # +-0.3125 -> y = +-2.5 -> 3 and -2; 0.0625 -> 0.5 -> 1; 2^-40 -> 0
    assert list(D[0, 0]) == [16, 4, -3, 3, -2, 1, 0]
    # second digits: 15.75 - 16 = -1/4 -> -8; 3.5 - 4 = -1/2 -> -16; -3.5 + 3 = -1/2 -> -16
    assert list(D[1, 0, :3]) == [-8, -16, -16]


@pytest.mark.parametrize("s", [2, 5, 7])
def test_nearest_level_sums_equal_exact_integer_products(s):
    A = _mixed_matrix(5, 7, seed=81)
    B = _mixed_matrix(7, 4, seed=82)
    _, DA, _ = oz.split_rows(A, s, 5, "nearest")
    _, DBt, _ = oz.split_cols(B, s, 5, "nearest")
    got = oz.level_sums(DA, DBt, 5, "nearest")
    want = _brute_levels(DA, DBt)
    for L in want:
        assert np.array_equal(got[L], np.array(want[L], dtype=np.int64)), L


@pytest.mark.parametrize("s", [2, 4, 7, 9])
def test_nearest_error_within_bound(s):
    A = _mixed_matrix(6, 8, seed=91)
    B = _mixed_matrix(8, 5, seed=92)
    C, parts = oz.ozaki_gemm(A, B, s, 5, return_parts=True, rounding="nearest")
    exact = _exact_product(A, B)
    bound = oz.truncation_bound(parts["e"], parts["f"], A.shape[1], s, 5, rounding="nearest")
    for r in range(A.shape[0]):
        for c in range(B.shape[1]):
            assert abs(Fraction(float(C[r, c])) - exact[r][c]) <= Fraction(float(bound[r, c])), (r, c)


def test_nearest_small_integers_need_one_slice():
    """Integer entries in [-15, 15] with a row (column) maximum of at least 8:
    e = 5, so y = a is its own single digit and the one-slice product is exact."""
    rng = _rng(95)
    A = rng.integers(-15, 16, size=(7, 9)).astype(np.float64)
    B = rng.integers(-15, 16, size=(9, 6)).astype(np.float64)
    A[:, 0] = -9.0
    B[0, :] = 12.0
    want = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    for s in (1, 3):
        assert np.array_equal(oz.ozaki_gemm(A, B, s, 5, rounding="nearest"), want)


def test_nearest_full_coverage_is_correctly_rounded():
    """beta s = 60 on nonnegative inputs: within 2 ulp of the correctly rounded product."""
    rng = _rng(96)
    A = rng.random((6, 10))
    B = rng.random((10, 5))
    C = oz.ozaki_gemm(A, B, 12, 5, rounding="nearest")
    exact = _exact_product(A, B)
    for r in range(6):
        for c in range(5):
            ref = float(exact[r][c])
            assert abs(C[r, c] - ref) <= 2 * np.spacing(ref), (r, c)


def test_nearest_matches_truncated_accuracy_per_bit():
    """Seven nearest digits of 5 bits (34 bits below the row maximum) and five
    truncated digits of 7 bits (35 bits) give errors of the same order."""
    rng = _rng(97)
    A = rng.standard_normal((24, 96))
    B = rng.standard_normal((96, 20))
    ref = np.array(_exact_product_float(A, B))
    e_near = np.abs(oz.ozaki_gemm(A, B, 7, 5, rounding="nearest") - ref).max()
    e_trunc = np.abs(oz.ozaki_gemm(A, B, 5, 7) - ref).max()
    assert 0.1 < e_near / e_trunc < 10.0


def test_planted_half_even_rounding_fails_the_digit_rule():
    def split_half_even(A, s, beta, rounding):
        e = oz.row_exponents(A, "nearest")
        x = np.ldexp(np.asarray(A, dtype=np.float64), -e[:, None])
        D = np.zeros((s,) + A.shape, dtype=np.int64)
        for i in range(s):
            y = x * 2.0 ** beta
            d = np.round(y)  # ties to even
            x = y - d
            D[i] = d.astype(np.int64)
        return e, D, x

    with pytest.raises(AssertionError):
        _check_nearest_split(split_half_even, _tie_matrix(), 2, 5)


def test_planted_truncated_digits_fail_the_nearest_rule():
    def split_trunc_digits(A, s, beta, rounding):
        e = oz.row_exponents(A, "nearest")
        x = np.ldexp(np.asarray(A, dtype=np.float64), -e[:, None])
        D = np.zeros((s,) + A.shape, dtype=np.int64)
        for i in range(s):
            y = x * 2.0 ** beta
            d = np.trunc(y)
            x = y - d
            D[i] = d.astype(np.int64)
        return e, D, x

    with pytest.raises(AssertionError):
        _check_nearest_split(split_trunc_digits, _mixed_matrix(4, 6, seed=98), 3, 5)


# ----------------------------------------------------------------- nearest 8-bit digits (BF16 mode)

def _bf16_integer_values():
    """Integers a bfloat16 holds exactly (8 significant bits) up to 300 in magnitude."""
    vals = set()
    for v in range(0, 301):
        b = bin(v)[2:].rstrip("0") if v else "0"
        if len(b) <= 8:
            vals.update({v, -v})
    return vals


def test_nearest_8bit_digits_are_exact_in_bf16_and_products_fit_2_14():
    vals = _bf16_integer_values()
    assert oz.max_digit(oz.BETA["bf16"], oz.ROUNDING["bf16"]) == 128
    assert all(d in vals for d in range(-128, 129))
    assert 128 * 128 == 2 ** 14 and 1024 * 2 ** 14 == 2 ** 24  # an fp32 chunk of 1024 stays exact


@pytest.mark.parametrize("s", [1, 4, 9])
def test_nearest_8bit_split_matches_digit_rule(s):
    _check_nearest_split(oz.split_rows, _mixed_matrix(5, 9, seed=170 + s), s, 8)
    _check_nearest_split(oz.split_rows, _tie_matrix(), s, 8)


@pytest.mark.parametrize("s", [2, 5, 6])
def test_nearest_8bit_error_within_bound_and_levels_exact(s):
    A = _mixed_matrix(6, 8, seed=191)
    B = _mixed_matrix(8, 5, seed=192)
    C, parts = oz.ozaki_gemm(A, B, s, 8, return_parts=True, rounding="nearest")
    want = _brute_levels(parts["DA"], parts["DBt"])
    for L in want:
        assert np.array_equal(parts["S"][L], np.array(want[L], dtype=np.int64)), L
    exact = _exact_product(A, B)
    bound = oz.truncation_bound(parts["e"], parts["f"], A.shape[1], s, 8, rounding="nearest")
    for r in range(A.shape[0]):
        for c in range(B.shape[1]):
            assert abs(Fraction(float(C[r, c])) - exact[r][c]) <= Fraction(float(bound[r, c])), (r, c)


@pytest.mark.parametrize("s", [1, 3, 4, 6])
def test_recombination_8bit_groups_of_three_correctly_rounded(s):
    """Groups of three levels for beta = 8: level sums up to 2^30 weighted by 1,
    2^8, 2^16 stay exact, and with at most two groups (s <= 6) the float64
    result is the correctly rounded exact sum."""
    beta = 8
    assert all(len(g) <= 3 for g in oz.level_groups(s, beta))
    assert len(oz.level_groups(s, beta)) <= 2
    rng = np.random.default_rng(300 + s)
    S = {L: rng.integers(-(2 ** 30), 2 ** 30, size=(6, 5), dtype=np.int64) for L in range(2, s + 2)}
    C = oz.recombine(S, np.zeros(6, dtype=np.int64), np.zeros(5, dtype=np.int64), s, beta)
    for r in range(6):
        for c in range(5):
            assert C[r, c] == float(_exact_level_value(S, s, beta, r, c))


# ----------------------------------------------------------------- exact equivariances

@pytest.mark.parametrize("beta,rounding", [(7, "trunc"), (8, "nearest"), (5, "nearest")])
def test_power_of_two_scaling_is_exact(beta, rounding):
    """Scaling A by 2^k scales every row exponent by k and leaves the digits
    unchanged, so C scales by exactly 2^k (a wrong exponent offset breaks this)."""
    A = _mixed_matrix(6, 9, seed=401)
    B = _mixed_matrix(9, 5, seed=402)
    C = oz.ozaki_gemm(A, B, 4, beta, rounding=rounding)
    for k in (-37, 1, 12):
        Ck = oz.ozaki_gemm(np.ldexp(A, k), B, 4, beta, rounding=rounding)
        assert np.array_equal(Ck, np.ldexp(C, k)), k
        Cb = oz.ozaki_gemm(A, np.ldexp(B, k), 4, beta, rounding=rounding)
        assert np.array_equal(Cb, np.ldexp(C, k)), k


@pytest.mark.parametrize("beta,rounding", [(7, "trunc"), (8, "nearest"), (5, "nearest")])
def test_row_and_column_permutations_commute_exactly(beta, rounding):
    """Row scaling and digits depend on each row alone (columns of B alone), so
    permuting rows of A or columns of B permutes C bit for bit."""
    rng = _rng(403)
    A = _mixed_matrix(7, 8, seed=404)
    B = _mixed_matrix(8, 6, seed=405)
    C = oz.ozaki_gemm(A, B, 5, beta, rounding=rounding)
    pr, pc = rng.permutation(7), rng.permutation(6)
    assert np.array_equal(oz.ozaki_gemm(A[pr], B, 5, beta, rounding=rounding), C[pr])
    assert np.array_equal(oz.ozaki_gemm(A, B[:, pc], 5, beta, rounding=rounding), C[:, pc])


@pytest.mark.parametrize("beta,rounding", [(7, "trunc"), (8, "nearest"), (5, "nearest")])
def test_square_of_a_symmetric_matrix_is_exactly_symmetric(beta, rounding):
    """For symmetric P the column split of P is its row split, the level sums of
    P P are exactly symmetric integers and so is the recombined product (the
    GPU therefore computes only the upper triangle of P^2 and mirrors it)."""
    rng = _rng(406)
    X = rng.standard_normal((12, 12)) * np.exp2(rng.integers(-8, 4, size=(12, 12)))
    P = 0.5 * (X + X.T)
    C, parts = oz.ozaki_gemm(P, P, 6, beta, return_parts=True, rounding=rounding)
    assert np.array_equal(parts["e"], parts["f"])
    for L, S in parts["S"].items():
        assert np.array_equal(S, S.T), L
    assert np.array_equal(C, C.T)
