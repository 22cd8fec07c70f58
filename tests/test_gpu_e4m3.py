"""GPU vs oracle: the E4M3 mode (nearest 5-bit digits on kind::f8f6f4).

Bit-exact comparisons of the row exponents and digit planes (decoded from
their E4M3 bytes by the format's definition), the int32 level sums and the
float64 product, on the paired and the single-CTA kernel; long K that spans
several fp32 chunks; sampled outputs of the full 8192^3 product; purification
and the refinement step against the oracle run in the same mode.
"""

from functools import partial

import numpy as np
import pytest
import torch

from oracle import ozaki as oz
from oracle import purify as pu
from synth import make_hamiltonian

pytestmark = pytest.mark.gpu

BETA = 5


def _e4m3_table():
    """Value of every E4M3 byte: sign bit 7, exponent bits 3..6 (bias 7), fraction bits 0..2."""
    t = np.full(256, np.nan)
    for code in range(256):
        ex, fr = (code >> 3) & 0xF, code & 0x7
        if ex == 0xF and fr == 0x7:
            continue
        v = fr / 8.0 * 2.0 ** -6 if ex == 0 else (1.0 + fr / 8.0) * 2.0 ** (ex - 7)
        t[code] = -v if code & 0x80 else v
    return t


E4M3 = _e4m3_table()


def _mixed(m, k, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, k)) * np.exp2(rng.integers(-20, 6, size=(m, k)))
    if m > 3:
        A[3, :] = 0.0
    if m > 5:
        A[5, :] *= 2.0 ** -300
    A[0, 0] = 0.0
    if m > 8 and k > 6:
        # the digit rule's edges: ties of both signs and a first digit of 16
        A[8, :6] = np.array([1.96875, 0.4375, -0.4375, 0.3125, -0.3125, 0.0625]) * 2.0 ** 7
        A[8, 6:] = np.clip(A[8, 6:], -2.0 ** 7, 2.0 ** 7)
    return A


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _decode(planes):
    vals = E4M3[planes.cpu().numpy()]
    assert not np.any(np.isnan(vals))
    assert np.array_equal(vals, np.round(vals))
    return vals.astype(np.int64)


@pytest.mark.parametrize("m,k,s", [(200, 300, 7), (129, 64, 3), (1, 5, 1), (257, 1000, 12), (300, 777, 9)])
def test_split_bit_exact(dmp, m, k, s):
    A = _mixed(m, k, seed=m + k)
    e, D, _ = oz.split_rows(A, s, BETA, "nearest")
    ge, gd = dmp.ozaki_split(_dev(A), "e4m3", s, "tc")
    assert gd.dtype == torch.uint8
    assert np.array_equal(ge.cpu().numpy(), e.astype(np.int32))
    assert np.array_equal(_decode(gd), D)


@pytest.mark.parametrize("pairing", [1, 0])
@pytest.mark.parametrize("m,n,k,s", [(300, 200, 257, 7), (128, 128, 64, 1), (520, 260, 777, 4), (40, 7, 3, 12)])
def test_level_sums_bit_exact(dmp, pairing, m, n, k, s):
    A = _mixed(m, k, seed=1)
    B = _mixed(k, n, seed=2)
    _, parts = oz.ozaki_gemm(A, B, s, BETA, return_parts=True, rounding="nearest")
    prev = dmp.set_tc_pairing(pairing)
    try:
        S = dmp.ozaki_level_sums(_dev(A), _dev(B), "e4m3", s, "tc").cpu().numpy()
    finally:
        dmp.set_tc_pairing(prev)
    for L in range(2, s + 2):
        assert np.array_equal(S[L - 2].astype(np.int64), parts["S"][L]), L


@pytest.mark.parametrize("pairing", [1, 0])
@pytest.mark.parametrize("m,n,k,s", [(300, 200, 257, 7), (256, 256, 256, 2), (33, 500, 77, 9), (1, 1, 1, 3),
                                     (520, 700, 2100, 7), (64, 64, 300, 12)])
def test_product_bit_exact(dmp, pairing, m, n, k, s):
    A = _mixed(m, k, seed=3)
    B = _mixed(k, n, seed=4)
    want = oz.ozaki_gemm(A, B, s, BETA, rounding="nearest")
    prev = dmp.set_tc_pairing(pairing)
    try:
        got = dmp.ozaki_gemm(_dev(A), _dev(B), "e4m3", s, "tc").cpu().numpy()
    finally:
        dmp.set_tc_pairing(prev)
    assert np.array_equal(got, want)


def test_long_k_spans_chunks_exactly(dmp):
    """K = 16384 at s = 7: the seven-pair level spans 7 x 16384 digits, two fp32
    chunks of up to 65536; rows of 1.96875 2^j put 16 in every first digit, so
    the level-2 chunk sums reach 16384 * 256 = 2^22 with both signs."""
    n, k, s = 256, 16384, 7
    rng = np.random.default_rng(21)
    A = rng.standard_normal((n, k))
    B = rng.standard_normal((k, n))
    A[:8, :] = 1.96875
    A[4:8, ::2] *= -1.0
    B[:, :8] = 1.96875
    _, parts = oz.ozaki_gemm(A, B, s, BETA, return_parts=True, rounding="nearest")
    assert np.all(np.abs(parts["DA"][0, :8]) == 16)
    S = dmp.ozaki_level_sums(_dev(A), _dev(B), "e4m3", s, "tc").cpu().numpy()
    for L in range(2, s + 2):
        assert np.array_equal(S[L - 2].astype(np.int64), parts["S"][L]), L
    got = dmp.ozaki_gemm(_dev(A), _dev(B), "e4m3", s, "tc").cpu().numpy()
    assert np.array_equal(got, oz.recombine(parts["S"], parts["e"], parts["f"], s, BETA))


def test_full_size_sampled_outputs(dmp):
    """8192^3 at s = 7 (the benchmark's size): 48 sampled outputs, each
    recomputed by the oracle from its own row and column."""
    n, s = 8192, 7
    rng = np.random.default_rng(9)
    A = rng.standard_normal((n, n)) * 0.01
    B = rng.standard_normal((n, n)) * 0.01
    C = dmp.ozaki_gemm(_dev(A), _dev(B), "e4m3", s, "tc")
    rows = rng.integers(0, n, size=48)
    cols = rng.integers(0, n, size=48)
    rows[:2] = [0, n - 1]
    cols[:2] = [n - 1, 0]
    Cs = C[torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()].cpu().numpy()
    for t, (r, c) in enumerate(zip(rows, cols)):
        want = oz.ozaki_gemm(A[r:r + 1, :], B[:, c:c + 1], s, BETA, rounding="nearest")[0, 0]
        assert Cs[t] == want, (r, c)


def _projector(h):
    V = h.Q[:, : h.n_occ]
    return V @ V.T


@pytest.mark.parametrize("n,n_occ,s", [(300, 75, 9), (600, 150, 10), (200, 13, 12)])
def test_purify_matches_oracle(dmp, n, n_occ, s):
    h = make_hamiltonian(n, n_occ, seed=n + s)
    ref = pu.purify(h.H, n_occ, tol=1e-10, product=partial(oz.ozaki_gemm, s=s, beta=BETA, rounding="nearest"))
    P, info = dmp.purify(_dev(h.H), n_occ, mode="e4m3", slices=s, executor="tc", tol=1e-10)
    P = P.cpu().numpy()
    assert info["status"] in (dmp.OK, dmp.C_OUT_OF_RANGE, dmp.STALLED)
    assert abs(info["iters"] - ref["iters"]) <= 1
    assert np.max(np.abs(P - ref["P"])) <= 1e-8
    assert np.max(np.abs(P - _projector(h))) <= 1e-8
    assert np.array_equal(P, P.T)


def test_refinement_matches_oracle(dmp):
    """s = 7 loop (34 bits) plus one McWeeny step with 11-slice products (54 bits)."""
    h = make_hamiltonian(384, 96, seed=23)
    low = partial(oz.ozaki_gemm, s=7, beta=BETA, rounding="nearest")
    ref = pu.purify(h.H, 96, tol=1e-10, product=low,
                    refine_product=partial(oz.ozaki_gemm, s=11, beta=BETA, rounding="nearest"))
    P, info = dmp.purify(_dev(h.H), 96, mode="e4m3", slices=7, executor="tc", tol=1e-10, refine=11)
    P = P.cpu().numpy()
    assert info["refined"] == 1
    assert abs(info["iters"] - ref["iters"]) <= 1
    # both loops stop at the 34-bit products' noise floor, 2e-8 from the
    # projector; the GPU's P lies as close to it as the oracle's
    P_star = _projector(h)
    assert np.max(np.abs(P - P_star)) <= 2.0 * np.max(np.abs(ref["P"] - P_star))
    assert np.max(np.abs(P - ref["P"])) <= 1e-7
    assert abs(info["energy_unrefined"] - ref["energy_unrefined"]) <= 1e-8 * abs(ref["energy"])
    E_star = float(np.sum(h.e[:96]))
    # the refinement fixes the energy (1e-14 in the oracle), not P (2e-8 from the projector)
    assert abs(info["energy"] - E_star) <= 1e-11 * abs(E_star)


def test_rejected_combinations(dmp):
    A = _dev(np.eye(8))
    with pytest.raises(RuntimeError):
        dmp.ozaki_gemm(A, A, "e4m3", 13, "tc")  # s beyond 12 (60 bits)
    with pytest.raises(RuntimeError):
        dmp.ozaki_gemm(A, A, "e4m3", 5, "imma")  # E4M3 digits run on the tensor-core executor only
    with pytest.raises(RuntimeError):
        dmp.purify(A, 2, mode="e4m3", slices=5, executor="imma")


def test_nonfinite_rows_and_columns(dmp):
    """A NaN in a row of A or an Inf in a column of B gives that row or column
    of NaN; every other output is the oracle's product of the finite parts."""
    A = _mixed(150, 90, seed=5)
    B = _mixed(90, 300, seed=6)
    A[7, 3] = np.nan
    B[11, 20] = np.inf
    got = dmp.ozaki_gemm(_dev(A), _dev(B), "e4m3", 7, "tc").cpu().numpy()
    assert np.all(np.isnan(got[7, :])) and np.all(np.isnan(got[:, 20]))
    A2, B2 = A.copy(), B.copy()
    A2[7, :] = 0.0
    B2[:, 20] = 0.0
    want = oz.ozaki_gemm(A2, B2, 7, BETA, rounding="nearest")
    mask = np.ones_like(got, dtype=bool)
    mask[7, :] = False
    mask[:, 20] = False
    assert np.array_equal(got[mask], want[mask])


def test_purify_ragged_size_and_nonfinite_input(dmp):
    """n = 333 (padded to 512 rows and K): same iterations and P as the oracle;
    a NaN in H is refused."""
    h = make_hamiltonian(333, 80, seed=41)
    ref = pu.purify(h.H, 80, tol=1e-10, product=partial(oz.ozaki_gemm, s=10, beta=BETA, rounding="nearest"))
    P, info = dmp.purify(_dev(h.H), 80, mode="e4m3", slices=10, tol=1e-10)
    assert abs(info["iters"] - ref["iters"]) <= 1
    assert np.max(np.abs(P.cpu().numpy() - ref["P"])) <= 1e-8
    H = h.H.copy()
    H[5, 9] = np.nan
    with pytest.raises(dmp.DmpError) as e:
        dmp.purify(_dev(H), 80, mode="e4m3", slices=7)
    assert e.value.code == dmp.ERR_NONFINITE
