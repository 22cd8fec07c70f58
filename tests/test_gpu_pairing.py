"""The tcgen05 executor on CTA pairs (2-SM MMA, 256 x 256 tiles) against the
same executor on single CTAs (128 x 256 tiles) and the oracle.

Both compute the same exact integer level sums and recombine them in the same
order, so products, level sums and whole purifications agree bit for bit.
Shapes have ragged row, column and K tails and odd numbers of 256-row pairs.
"""

import numpy as np
import pytest
import torch

from oracle import ozaki as oz
from synth import make_hamiltonian

pytestmark = pytest.mark.gpu


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _both(dmp, fn):
    prev = dmp.set_tc_pairing(True)
    try:
        a = fn()
        dmp.set_tc_pairing(False)
        b = fn()
    finally:
        dmp.set_tc_pairing(prev)
    return a, b


@pytest.mark.parametrize("m,n,k,s", [(300, 520, 700, 6), (513, 256, 1100, 7), (1, 1, 1, 2), (768, 130, 64, 10)])
def test_gemm_pair_equals_single_and_oracle(dmp, m, n, k, s):
    rng = np.random.default_rng(m * 7 + n)
    A = rng.standard_normal((m, k)) * np.exp2(rng.integers(-12, 4, size=(m, k)))
    B = rng.standard_normal((k, n))
    Ad, Bd = _dev(A), _dev(B)
    C1, C2 = _both(dmp, lambda: dmp.ozaki_gemm(Ad, Bd, "int8", s, "tc").cpu().numpy())
    assert np.array_equal(C1.view(np.int64), C2.view(np.int64))
    assert np.array_equal(C1, oz.ozaki_gemm(A, B, s, 7))


def test_level_sums_pair_equals_single(dmp):
    rng = np.random.default_rng(77)
    A = rng.standard_normal((600, 333))
    B = rng.standard_normal((333, 290))
    Ad, Bd = _dev(A), _dev(B)
    S1, S2 = _both(dmp, lambda: dmp.ozaki_level_sums(Ad, Bd, "int8", 5, "tc").cpu().numpy())
    assert np.array_equal(S1, S2)
    want = oz.ozaki_gemm(A, B, 5, 7, return_parts=True)[1]["S"]
    for L in range(2, 7):
        assert np.array_equal(S1[L - 2].astype(np.int64), want[L])


@pytest.mark.parametrize("n,n_occ", [(700, 170), (1024, 256)])
def test_purification_pair_equals_single(dmp, n, n_occ):
    h = make_hamiltonian(n, n_occ, occ=(-2.0, -0.2), virt=(0.2, 2.0), seed=n)
    Hd = _dev(h.H)
    (P1, i1), (P2, i2) = _both(dmp, lambda: tuple(
        (lambda P, info: (P.cpu().numpy(), info))(*dmp.purify(Hd, n_occ, mode="int8", slices=6, executor="tc"))))
    assert i1["iters"] == i2["iters"] and i1["status"] == i2["status"]
    assert np.array_equal(P1, P2)
