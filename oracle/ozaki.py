"""Ozaki error-free splitting product, float64 CPU oracle (Sec. "Ozaki Scheme").

TEST INFRASTRUCTURE ONLY (see the package header).

What the paper states (Sec. "Ozaki Scheme" and the caption of Fig. 2): each
operand is scaled to keep its exponent range (row-wise for A, column-wise for
B), split into S slice matrices of the input's size that multiply without
rounding error, the slice products A_i B_j with i + j <= S + 1 are formed, and
the products are summed in the original (FP64) precision. S splits cost 2S
times the memory and S(S+1)/2 products.

The paper does not print the split formula (it points to the improved
extraction of Minamihata et al.). The reading implemented here, used by the GPU
path as well:

* scaling: e_r = ilogb(max_j |A_rj|) + 1 for a nonzero row (0 for a zero row),
  so every scaled entry x = A_rj 2^-e_r lies in (-1, 1). B is scaled per column
  the same way (f_c), i.e. B^T is scaled per row.
* digits: for i = 1..S, y = x 2^beta, d_i = trunc(y), x = y - d_i. Every step is
  exact in FP64 and |d_i| <= 2^beta - 1. beta = 7 gives digits in int8 range
  (the INT8 mode). There is no remainder slice: the truncation of the last digit is the error
  that the diagonal i + j = S + 1 carries.
* nearest digits (the E4M3 and BF16 modes): the extraction of the original Ozaki scheme
  rounds to nearest instead of truncating. Here the row exponent is one larger
  (e_r = ilogb(max_j |A_rj|) + 2, so x lies in (-1/2, 1/2)) and
  d_i = floor(y + 1/2) (ties upward), x = y - d_i in [-1/2, 1/2). With
  beta = 5 every digit lies in [-16, 16]: integers of at most four
  significant bits, exact in the FP8 format E4M3 (4-bit exponent, 3-bit
  fraction). With beta = 8 every digit lies in [-128, 128], exact in bfloat16
  (8 significant bits), and a product of two is at most 2^14, as for 7-bit
  truncated digits. Each slice carries one bit more than a truncated digit of
  the same range would.
* level sums: S_L = sum over i + j = L of D_i^A (D_j^B)^T, exact integers,
  for L = 2 .. S + 1 (these are exactly the kept pairs).
* recombination: C = 2^(e_r + f_c) * (S_{S+1} 2^-beta(S+1) + ... + S_2 2^-2beta)
  in FP64. Up to four consecutive levels (beta <= 7; three for beta = 8) are
  first combined exactly as one integer whose value is an exact float64; these
  group values are added in FP64 from the smallest group to the largest,
  rounding at each addition. For S <= 8 (S <= 6 for beta = 8) there are at
  most two groups, so C is the correctly rounded value of the exact sum of the
  kept pairs.

Parity: pinned. The tests check digit reconstruction with exact rationals,
the digit rule (truncation, or the nearest-digit remainder interval) on exact
rationals, level sums against Python exact-integer products, the truncation
bound against the exact rational product, agreement with the correctly rounded
product when beta*S covers FP64, and the paper's printed product counts.
"""

from __future__ import annotations

import numpy as np

# digit width per precision mode (bits of magnitude per slice) and digit rule
BETA = {"int8": 7, "bf16": 8, "e4m3": 5}
ROUNDING = {"int8": "trunc", "bf16": "nearest", "e4m3": "nearest"}


def max_digit(beta: int, rounding: str = "trunc") -> int:
    """Largest |d_i|: 2^beta - 1 for truncated digits, 2^(beta-1) for nearest ones."""
    if rounding == "trunc":
        return 2 ** beta - 1
    if rounding == "nearest":
        return 2 ** (beta - 1)
    raise ValueError("rounding must be 'trunc' or 'nearest'")


def kept_pairs(s: int):
    """Slice pairs (i, j), 1-based, with i + j <= s + 1 (Sec. "Ozaki Scheme")."""
    if s < 1:
        raise ValueError("need at least one slice")
    return [(i, j) for i in range(1, s + 1) for j in range(1, s + 1) if i + j <= s + 1]


def product_count(s: int) -> int:
    """Number of slice products; the paper states S(S+1)/2."""
    return len(kept_pairs(s))


def symmetric_square_product_count(s: int) -> int:
    """Products for a symmetric square A*A with the transpose trick (Sec. "Comparison
    with the Markidis Method").

    Reading: the error-free terms (i + j <= s) need one product per unordered
    pair because A_j A_i = (A_i A_j)^T, while the s terms on the diagonal
    i + j = s + 1 that carry the truncation error are all formed. This gives the
    paper's 8 (four splits) and 11 (five splits).
    """
    exact_unordered = len([(i, j) for (i, j) in kept_pairs(s) if i <= j and i + j <= s])
    diagonal = len([(i, j) for (i, j) in kept_pairs(s) if i + j == s + 1])
    return exact_unordered + diagonal


def row_exponents(A: np.ndarray, rounding: str = "trunc") -> np.ndarray:
    """e_r with max_j |A_rj| < 2^e_r <= 2 max_j |A_rj| (truncated digits) or
    2 max_j |A_rj| < 2^e_r <= 4 max_j |A_rj| (nearest digits); 0 for an
    all-zero row."""
    A = np.asarray(A, dtype=np.float64)
    if not np.all(np.isfinite(A)):
        raise ValueError("non-finite input")
    max_digit(1, rounding)  # validates the rule
    m = np.max(np.abs(A), axis=1) if A.shape[1] > 0 else np.zeros(A.shape[0])
    _, e = np.frexp(m)  # m = f 2^e with 1/2 <= f < 1
    e = e.astype(np.int64) + (1 if rounding == "nearest" else 0)
    e[m == 0] = 0
    return e


def split_rows(A: np.ndarray, s: int, beta: int, rounding: str = "trunc"):
    """Row-scaled digit planes of A.

    Returns (e, D, residual): e[r] the row exponents, D an (s, m, k) int64 array
    of digits, residual the (m, k) float64 remainder after s digits (in (-1, 1)
    for truncated digits, in [-1/2, 1/2) for nearest ones), so that
    A = 2^e (sum_i D_i 2^-beta i + residual 2^-beta s) exactly.
    """
    A = np.asarray(A, dtype=np.float64)
    e = row_exponents(A, rounding)
    x = np.ldexp(A, -e[:, None])
    D = np.zeros((s,) + A.shape, dtype=np.int64)
    radix = 2.0 ** beta
    for i in range(s):
        y = x * radix
        if rounding == "trunc":
            d = np.trunc(y)
        else:
            # floor(y + 1/2) without rounding y + 1/2: the fractional part
            # y - floor(y) is exact
            f = np.floor(y)
            d = f + (y - f >= 0.5)
        x = y - d
        D[i] = d.astype(np.int64)
    return e, D, x


def split_cols(B: np.ndarray, s: int, beta: int, rounding: str = "trunc"):
    """Column-scaled digit planes of B, stored as the row split of B^T."""
    return split_rows(np.asarray(B, dtype=np.float64).T, s, beta, rounding)


def level_sums(DA: np.ndarray, DBt: np.ndarray, beta: int, rounding: str = "trunc"):
    """Exact level sums S_L = sum_{i+j=L} D_i^A (D_j^B)^T for L = 2 .. s+1.

    DA is (s, m, k), DBt is (s, n, k) (digits of B^T). The products are taken
    with float64 matrix multiplication on integer-valued operands; every partial
    sum is an integer of magnitude at most (L-1) k dmax^2 < 2^53 (asserted;
    dmax = max_digit(beta, rounding)), so each is exact whatever order the
    library adds in.
    """
    s, m, k = DA.shape
    n = DBt.shape[1]
    bound = s * max(k, 1) * max_digit(beta, rounding) ** 2
    if bound >= 2 ** 53:
        raise ValueError("level sums could exceed 2^53; not exact in float64")
    out = {}
    for L in range(2, s + 2):
        acc = np.zeros((m, n), dtype=np.float64)
        for i in range(1, L):
            j = L - i
            if i > s or j > s:
                continue
            acc = acc + DA[i - 1].astype(np.float64) @ DBt[j - 1].astype(np.float64).T
        out[L] = acc.astype(np.int64)
    return out


def level_groups(s: int, beta: int):
    """Consecutive levels combined exactly before any rounding: groups of up to
    four for beta <= 7 (four level sums below 2^31 weighted by 1, 2^beta,
    2^2beta, 2^3beta stay below 2^53), of up to three for beta = 8 (weights 1,
    2^8, 2^16). Groups start from the smallest level L = s + 1; each is listed
    largest L first."""
    size = 4 if beta <= 7 else 3
    levels = list(range(s + 1, 1, -1))
    return [levels[i:i + size] for i in range(0, len(levels), size)]


def recombine(S: dict, e_row: np.ndarray, f_col: np.ndarray, s: int, beta: int) -> np.ndarray:
    """FP64 sum of the levels, then the power-of-two unscaling.

    Each group of levels (see level_groups) is first combined exactly as the
    integer T = sum_L S_L 2^(beta (L_a - L)), L_a the group's largest L, so that
    its value T 2^(-beta L_a) is an exact float64; the groups are then added in
    float64 from the smallest to the largest, rounding at each addition. With at
    most two groups (s <= 8 for beta <= 7, s <= 6 for beta = 8) the result is
    the correctly rounded value of the exact sum.
    """
    m = e_row.shape[0]
    n = f_col.shape[0]
    C = np.zeros((m, n), dtype=np.float64)
    for group in level_groups(s, beta):
        L_a = group[0]
        T = np.zeros((m, n), dtype=np.int64)
        for L in group:
            T = T + (S[L].astype(np.int64) << (beta * (L_a - L)))
        if np.max(np.abs(T), initial=0) >= 2 ** 53:
            raise ValueError("group sum not exact in float64")
        C = C + T.astype(np.float64) * (2.0 ** (-beta * L_a))
    return np.ldexp(C, e_row[:, None] + f_col[None, :])


def ozaki_gemm(A: np.ndarray, B: np.ndarray, s: int, beta: int = 7, return_parts: bool = False,
               rounding: str = "trunc"):
    """C ~= A B through the Ozaki scheme with s slices of beta bits."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    if A.ndim != 2 or B.ndim != 2 or A.shape[1] != B.shape[0]:
        raise ValueError("shape mismatch")
    e, DA, _ = split_rows(A, s, beta, rounding)
    f, DBt, _ = split_cols(B, s, beta, rounding)
    S = level_sums(DA, DBt, beta, rounding)
    C = recombine(S, e, f, s, beta)
    if return_parts:
        return C, dict(e=e, f=f, DA=DA, DBt=DBt, S=S)
    return C


def truncation_bound(e_row: np.ndarray, f_col: np.ndarray, k: int, s: int, beta: int,
                     rounding: str = "trunc") -> np.ndarray:
    """Elementwise bound on |C - A B| for the scheme above.

    Per scaled product the dropped pairs (i + j >= s + 2) and the residuals
    contribute less than (s + 2) 2^-beta s for truncated digits. For nearest
    digits the tail of a scaled entry after t digits is at most 2^(-beta t - 1)
    and |d_i| 2^(-beta i) <= 2^(-beta (i - 1) - 1), so the s products of a kept
    digit with the other operand's tail and the residual of A times |b| < 1/2
    give at most (s + 1) 2^(-beta s - 2). The FP64 recombination adds at most s
    roundings of a sum below k in magnitude. All scale by k and 2^(e_r+f_c).
    """
    scale = np.ldexp(np.ones((e_row.shape[0], f_col.shape[0])), e_row[:, None] + f_col[None, :])
    if rounding == "trunc":
        per = (s + 2) * 2.0 ** (-beta * s) + s * 2.0 ** (-53)
    else:
        per = (s + 1) * 2.0 ** (-beta * s - 2) + s * 2.0 ** (-53)
    return scale * max(k, 1) * per
