"""Split launches of the tcgen05 product kernel (dmp_set_tc_split_tiles): when
a product's output tiles fill at most half a wave of CTAs (CTA pairs), every
tile is cut into units of one exact fp32 chunk and the units are shared out
over all CTAs, whose partial level sums are added at L2. Integer sums do not
depend on the split, so every result must be bit-for-bit that of whole tiles:
purifications (INT8 with one and two level groups, E4M3, BF16 with two and
three groups -- the latter runs whole tiles), on CTA pairs and single CTAs, at
sizes that split (n <= about 2000) and sizes that do not, the non-symmetric
products of the adjoint, and the expansion.
"""

import numpy as np
import pytest
import torch

from synth import make_hamiltonian, symmetric_gaussian

pytestmark = pytest.mark.gpu


def _both(dmp, fn):
    prev = dmp.set_tc_split_tiles(True)
    try:
        a = fn()
        dmp.set_tc_split_tiles(False)
        b = fn()
    finally:
        dmp.set_tc_split_tiles(prev)
    return a, b


@pytest.mark.parametrize("pairing", [True, False])
@pytest.mark.parametrize("n,mode,s,refine", [(300, "int8", 5, 8), (1000, "int8", 7, 0), (2500, "int8", 5, 0),
                                              (4200, "int8", 5, 8), (1000, "e4m3", 7, 0), (1000, "bf16", 5, 0),
                                              (1000, "bf16", 7, 0)])
def test_purification_is_bit_identical_with_and_without_the_split(dmp, pairing, n, mode, s, refine):
    h = make_hamiltonian(n, n // 4, seed=n + s)
    Hd = torch.from_numpy(h.H).cuda()
    prev = dmp.set_tc_pairing(pairing)
    try:
        (P1, i1), (P2, i2) = _both(dmp, lambda: dmp.purify(Hd, n // 4, mode=mode, slices=s, executor="tc",
                                                           refine=refine))
    finally:
        dmp.set_tc_pairing(prev)
    assert i1["status"] >= 0 and i1["iters"] == i2["iters"]
    assert torch.equal(P1, P2)
    assert i1["energy"] == i2["energy"]


def test_adjoint_products_are_bit_identical(dmp):
    n, n_occ = 700, 175
    h = make_hamiltonian(n, n_occ, occ=(-2.0, -0.1), virt=(0.1, 2.0), seed=61)
    W = torch.from_numpy(symmetric_gaussian(n, seed=62)).cuda()

    def grad():
        Hd = torch.from_numpy(h.H).cuda().requires_grad_(True)
        P = dmp.purify_autograd(Hd, n_occ, mode="int8", slices=6, executor="tc", checkpoint_every=4)
        (P * W).sum().backward()
        return Hd.grad.clone()

    g1, g2 = _both(dmp, grad)
    assert torch.equal(g1, g2)


def test_expansion_is_bit_identical(dmp):
    h = make_hamiltonian(900, 300, occ=(-2.0, 0.0), virt=(0.0, 2.0), seed=63)
    Hd = torch.from_numpy(h.H).cuda()
    (P1, i1), (P2, i2) = _both(dmp, lambda: dmp.foe(Hd, 0.1, 40, n_occ=300, bounds=(-2.0, 2.0), mode="int8",
                                                    slices=6, scheme="ps"))
    assert torch.equal(P1, P2) and i1["mu"] == i2["mu"]
