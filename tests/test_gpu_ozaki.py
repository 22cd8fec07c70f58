"""GPU vs oracle: the Ozaki split, the integer level sums and the product.

Bit-exact comparisons: the exponents and digit planes, the int32 level sums,
and the float64 product (the recombination order is fixed, so the float64
result is reproducible bit for bit). Sizes span several 128 x 128 tiles with
ragged tails; the full-size case checks sampled outputs of an 8192^3 product
one by one against the oracle.
"""

import numpy as np
import pytest
import torch

from oracle import ozaki as oz

pytestmark = pytest.mark.gpu

EXECUTORS = ["imma", "tc"]


def _mixed(m, k, seed, zero_row=True):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, k)) * np.exp2(rng.integers(-20, 6, size=(m, k)))
    if zero_row and m > 3:
        A[3, :] = 0.0
    if m > 5:
        A[5, :] *= 2.0 ** -300
    A[0, 0] = 0.0
    return A


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("executor", EXECUTORS)
@pytest.mark.parametrize("m,k,s", [(200, 300, 7), (129, 64, 3), (1, 5, 1), (257, 1000, 10)])
def test_split_bit_exact(dmp, executor, m, k, s):
    A = _mixed(m, k, seed=m + k)
    e, D, _ = oz.split_rows(A, s, 7)
    ge, gd = dmp.ozaki_split(_dev(A), "int8", s, executor)
    assert np.array_equal(ge.cpu().numpy(), e.astype(np.int32))
    got = gd.float().cpu().numpy().astype(np.int64) if gd.dtype == torch.bfloat16 else gd.cpu().numpy().astype(np.int64)
    assert np.array_equal(got, D)


@pytest.mark.parametrize("executor", EXECUTORS)
@pytest.mark.parametrize("m,n,k,s", [(300, 200, 257, 7), (128, 128, 64, 1), (130, 260, 129, 4), (40, 7, 3, 9)])
def test_level_sums_bit_exact(dmp, executor, m, n, k, s):
    A = _mixed(m, k, seed=1)
    B = _mixed(k, n, seed=2)
    _, parts = oz.ozaki_gemm(A, B, s, 7, return_parts=True)
    S = dmp.ozaki_level_sums(_dev(A), _dev(B), "int8", s, executor).cpu().numpy()
    for L in range(2, s + 2):
        assert np.array_equal(S[L - 2].astype(np.int64), parts["S"][L]), L


@pytest.mark.parametrize("executor", EXECUTORS)
@pytest.mark.parametrize("m,n,k,s", [(300, 200, 257, 7), (256, 256, 256, 3), (33, 500, 77, 10), (1, 1, 1, 2),
                                     (520, 700, 2100, 7)])
def test_ozaki_gemm_bit_exact(dmp, executor, m, n, k, s):
    A = _mixed(m, k, seed=3)
    B = _mixed(k, n, seed=4)
    want = oz.ozaki_gemm(A, B, s, 7)
    got = dmp.ozaki_gemm(_dev(A), _dev(B), "int8", s, executor).cpu().numpy()
    assert np.array_equal(got.view(np.int64), want.view(np.int64))


def test_ozaki_gemm_nonfinite_rows_and_columns(dmp):
    A = _mixed(150, 90, seed=5)
    B = _mixed(90, 140, seed=6)
    A[7, 3] = np.nan
    B[11, 20] = np.inf
    got = dmp.ozaki_gemm(_dev(A), _dev(B), "int8", 5, "imma").cpu().numpy()
    assert np.all(np.isnan(got[7, :])) and np.all(np.isnan(got[:, 20]))
    A2, B2 = A.copy(), B.copy()
    A2[7, :] = 0.0
    B2[:, 20] = 0.0
    want = oz.ozaki_gemm(A2, B2, 5, 7)
    mask = np.ones_like(got, dtype=bool)
    mask[7, :] = False
    mask[:, 20] = False
    assert np.array_equal(got[mask], want[mask])


def test_fp64_gemm_matches_float64(dmp):
    rng = np.random.default_rng(7)
    A = rng.standard_normal((301, 199))
    B = rng.standard_normal((199, 250))
    got = dmp.ozaki_gemm(_dev(A), _dev(B), "fp64").cpu().numpy()
    want = A @ B
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want)) * 10


@pytest.mark.parametrize("executor", EXECUTORS)
def test_full_size_sampled_outputs(dmp, executor):
    """8192^3 at s = 7, the size of the purification benchmark: 48 sampled
    outputs, each recomputed by the oracle from its own row and column."""
    n, s = 8192, 7
    rng = np.random.default_rng(8)
    A = rng.standard_normal((n, n)) * 0.01
    B = rng.standard_normal((n, n)) * 0.01
    C = dmp.ozaki_gemm(_dev(A), _dev(B), "int8", s, executor)
    rows = rng.integers(0, n, size=48)
    cols = rng.integers(0, n, size=48)
    rows[:2] = [0, n - 1]
    cols[:2] = [n - 1, 0]
    Cs = C[torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()].cpu().numpy()
    for t, (r, c) in enumerate(zip(rows, cols)):
        want = oz.ozaki_gemm(A[r:r + 1, :], B[:, c:c + 1], s, 7)[0, 0]
        assert Cs[t] == want, (r, c)


@pytest.mark.parametrize("executor", EXECUTORS)
def test_extreme_digits_stay_exact(dmp, executor):
    """Entries 1 - 2^-49 give seven digits of 127 each: every fp32 chunk sum of
    the tensor-core executor sits at its bound 1024 * 127^2 (just under 2^24),
    with both signs, so any loss in the accumulator shows up as a wrong bit."""
    n, k, s = 256, 2048, 7
    v = 1.0 - 2.0 ** -49
    rng = np.random.default_rng(12)
    A = np.full((n, k), v)
    B = np.full((k, n), v)
    A[n // 2:, :] *= -1.0
    B[:, ::3] *= -1.0
    A[7, :] = rng.choice([-v, v], size=k)
    _, parts = oz.ozaki_gemm(A, B, s, 7, return_parts=True)
    assert np.all(np.abs(parts["DA"]) == 127)
    S = dmp.ozaki_level_sums(_dev(A), _dev(B), "int8", s, executor).cpu().numpy()
    for L in range(2, s + 2):
        assert np.array_equal(S[L - 2].astype(np.int64), parts["S"][L]), L
    want = oz.ozaki_gemm(A, B, s, 7)
    got = dmp.ozaki_gemm(_dev(A), _dev(B), "int8", s, executor).cpu().numpy()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("pairing", [1, 0])
@pytest.mark.parametrize("m,n,k,s", [(300, 260, 520, 6), (128, 128, 4096, 5), (64, 500, 77, 9)])
def test_bf16_mode_bit_exact(dmp, pairing, m, n, k, s):
    """Nearest beta = 8 digits (|d| <= 128) on the tensor-core executor: 1024-wide
    K chunks and groups of three levels, on CTA pairs and on single CTAs."""
    A = _mixed(m, k, seed=21)
    B = _mixed(k, n, seed=22)
    want = oz.ozaki_gemm(A, B, s, 8, rounding="nearest")
    prev = dmp.set_tc_pairing(pairing)
    try:
        got = dmp.ozaki_gemm(_dev(A), _dev(B), "bf16", s, "tc").cpu().numpy()
    finally:
        dmp.set_tc_pairing(prev)
    assert np.array_equal(got.view(np.int64), want.view(np.int64))
    e, D, _ = oz.split_rows(A, s, 8, "nearest")
    ge, gd = dmp.ozaki_split(_dev(A), "bf16", s, "tc")
    assert np.array_equal(ge.cpu().numpy(), e.astype(np.int32))
    assert np.array_equal(gd.float().cpu().numpy().astype(np.int64), D)


def test_bf16_mode_chunk_bound(dmp):
    """Entries 0.4990234375 give a first digit of 128 (y = 127.75) and a second
    of -64: every 1024-long fp32 chunk of the level-2 product sums 1024 * 2^14
    = 2^24, the exactness bound, with both signs across the columns."""
    n, k, s = 256, 8192, 4
    v = 127.75 / 256.0
    A = np.full((n, k), v)
    B = np.full((k, n), v)
    B[:, 1::2] *= -1.0
    A[3, ::5] *= -1.0
    _, parts = oz.ozaki_gemm(A, B, s, 8, return_parts=True, rounding="nearest")
    assert np.all(np.abs(parts["DA"][0]) == 128)
    S = dmp.ozaki_level_sums(_dev(A), _dev(B), "bf16", s, "tc").cpu().numpy()
    for L in range(2, s + 2):
        assert np.array_equal(S[L - 2].astype(np.int64), parts["S"][L]), L
    want = oz.ozaki_gemm(A, B, s, 8, rounding="nearest")
    got = dmp.ozaki_gemm(_dev(A), _dev(B), "bf16", s, "tc").cpu().numpy()
    assert np.array_equal(got, want)


def test_invalid_arguments(dmp):
    A = _dev(np.ones((4, 4)))
    with pytest.raises(dmp.DmpError):
        dmp.ozaki_gemm(A, A, "int8", 11, "imma")  # s beyond 10 for beta 7
    with pytest.raises(dmp.DmpError):
        dmp.ozaki_gemm(A, A, "bf16", 3, "imma")  # the BF16 mode runs on the tensor-core executor only
