"""GPU properties that hold at any size, for every slice mode: power-of-two
scaling and permutation equivariance of the product (bit for bit), run-to-run
determinism of the purification, and sampled outputs of the full 8192^3 BF16
product against the oracle."""

import numpy as np
import pytest
import torch

from oracle import ozaki as oz
from synth import make_hamiltonian

pytestmark = pytest.mark.gpu

MODES = [("int8", 6, 7, "trunc"), ("bf16", 5, 8, "nearest"), ("e4m3", 8, 5, "nearest")]


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _mixed(m, k, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((m, k)) * np.exp2(rng.integers(-12, 4, size=(m, k)))


@pytest.mark.parametrize("mode,s,beta,rounding", MODES)
def test_power_of_two_scaling_and_permutations(dmp, mode, s, beta, rounding):
    A = _mixed(300, 520, seed=11)
    B = _mixed(520, 270, seed=12)
    C = dmp.ozaki_gemm(_dev(A), _dev(B), mode, s, "tc").cpu().numpy()
    C8 = dmp.ozaki_gemm(_dev(np.ldexp(A, 9)), _dev(B), mode, s, "tc").cpu().numpy()
    assert np.array_equal(C8, np.ldexp(C, 9))
    rng = np.random.default_rng(13)
    pr, pc = rng.permutation(300), rng.permutation(270)
    Cp = dmp.ozaki_gemm(_dev(A[pr]), _dev(B[:, pc]), mode, s, "tc").cpu().numpy()
    assert np.array_equal(Cp, C[pr][:, pc])


@pytest.mark.parametrize("mode,s,beta,rounding", MODES)
def test_purification_is_deterministic(dmp, mode, s, beta, rounding):
    h = make_hamiltonian(520, 130, seed=14)
    H = _dev(h.H)
    P1, i1 = dmp.purify(H, 130, mode=mode, slices=s + 2, executor="tc")
    P2, i2 = dmp.purify(H, 130, mode=mode, slices=s + 2, executor="tc")
    assert torch.equal(P1, P2) and i1 == i2


def test_bf16_full_size_sampled_outputs(dmp):
    """8192^3 at s = 5 on CTA pairs (the benchmark's size): 48 sampled outputs,
    each recomputed by the oracle from its own row and column."""
    n, s = 8192, 5
    rng = np.random.default_rng(15)
    A = rng.standard_normal((n, n)) * 0.01
    B = rng.standard_normal((n, n)) * 0.01
    C = dmp.ozaki_gemm(_dev(A), _dev(B), "bf16", s, "tc")
    rows = rng.integers(0, n, size=48)
    cols = rng.integers(0, n, size=48)
    rows[:2] = [0, n - 1]
    cols[:2] = [n - 1, 0]
    Cs = C[torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()].cpu().numpy()
    for t, (r, c) in enumerate(zip(rows, cols)):
        want = oz.ozaki_gemm(A[r:r + 1, :], B[:, c:c + 1], s, 8, rounding="nearest")[0, 0]
        assert Cs[t] == want, (r, c)
