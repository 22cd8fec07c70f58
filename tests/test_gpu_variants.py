"""SP2 and TRS4 purification on the GPU (opts.method) against the oracle's
variants (oracle/variants.py): FP64 mode to 1e-10, Ozaki-INT8 at s >= 7 to
1e-8, both executors, with the refinement step, and the rejected uses."""

from functools import partial

import numpy as np
import pytest
import torch

from oracle import ozaki as oz
from oracle import variants as va
from synth import config_hamiltonian, make_hamiltonian

pytestmark = pytest.mark.gpu

METHODS = ["trs4", "sp2"]


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _projector(h):
    V = h.Q[:, : h.n_occ]
    return V @ V.T


@pytest.mark.parametrize("method", METHODS)
def test_fp64_variants_match_oracle(dmp, method):
    h = config_hamiltonian(0)
    ref = va.purify(h.H, h.n_occ, method=method, tol=1e-10)
    P, info = dmp.purify(_dev(h.H), h.n_occ, mode="fp64", tol=1e-10, method=method)
    P = P.cpu().numpy()
    assert info["status"] == dmp.OK and abs(info["iters"] - ref["iters"]) <= 1
    assert np.max(np.abs(P - ref["P"])) <= 1e-10
    assert np.max(np.abs(P - _projector(h))) <= 1e-10
    assert np.array_equal(P, P.T)


@pytest.mark.parametrize("executor", ["tc", "imma"])
@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("n,n_occ,s", [(300, 75, 7), (520, 130, 8)])
def test_ozaki_variants_match_oracle(dmp, executor, method, n, n_occ, s):
    h = make_hamiltonian(n, n_occ, seed=n + s + 7)
    ref = va.purify(h.H, n_occ, method=method, tol=1e-10, product=partial(oz.ozaki_gemm, s=s, beta=7))
    P, info = dmp.purify(_dev(h.H), n_occ, mode="int8", slices=s, executor=executor, tol=1e-10, method=method)
    P = P.cpu().numpy()
    assert info["status"] in (dmp.OK, dmp.C_OUT_OF_RANGE)
    assert np.max(np.abs(P - ref["P"])) <= 1e-8
    # distance to the exact projector and energy error: those the method itself
    # reaches with these products (the oracle's), up to a factor 2
    proj = _projector(h)
    assert np.max(np.abs(P - proj)) <= max(1e-8, 2.0 * np.max(np.abs(ref["P"] - proj)))
    E_star = float(np.sum(h.e[:n_occ]))
    assert abs(info["energy"] - E_star) <= max(1e-8 * abs(E_star), 2.0 * abs(ref["energy"] - E_star))
    assert np.array_equal(P, P.T)


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("mode,s,beta", [("bf16", 6, 8), ("e4m3", 9, 5)])
def test_nearest_digit_modes_match_oracle(dmp, method, mode, s, beta):
    """SP2 and TRS4 with the nearest-digit modes (BF16: 8-bit digits in
    bfloat16; E4M3: 5-bit digits in FP8) against the oracle run in the same mode."""
    n, n_occ = 300, 75
    h = make_hamiltonian(n, n_occ, seed=n + s + 17)
    prod = partial(oz.ozaki_gemm, s=s, beta=beta, rounding="nearest")
    ref = va.purify(h.H, n_occ, method=method, tol=1e-10, product=prod)
    P, info = dmp.purify(_dev(h.H), n_occ, mode=mode, slices=s, executor="tc", tol=1e-10, method=method)
    P = P.cpu().numpy()
    assert info["status"] in (dmp.OK, dmp.C_OUT_OF_RANGE)
    assert np.max(np.abs(P - ref["P"])) <= 1e-8
    proj = _projector(h)
    assert np.max(np.abs(P - proj)) <= max(1e-8, 2.0 * np.max(np.abs(ref["P"] - proj)))
    assert np.array_equal(P, P.T)


@pytest.mark.parametrize("method", METHODS)
def test_variants_with_refinement_reach_the_energy_target(dmp, method):
    """n = 2048, the benchmark's spectrum: s = 5 loop plus the refinement step."""
    n, n_occ = 2048, 512
    h = make_hamiltonian(n, n_occ, occ=(-1.5, -0.01), virt=(0.01, 1.5), seed=94)
    E_star = float(np.sum(np.sort(h.e)[:n_occ]))
    _, info = dmp.purify(_dev(h.H), n_occ, mode="int8", slices=5, executor="tc", method=method, refine=8)
    assert info["refined"] == 1
    assert abs(info["energy"] - E_star) / abs(E_star) < 1e-8


def test_variant_rejections(dmp):
    h = make_hamiltonian(128, 32, seed=96)
    Hd = _dev(h.H)
    opts = dmp.make_opts("int8", 6, "tc", method="trs4")
    tape = dmp.workspace(dmp.tape_bytes(128, opts))
    with pytest.raises(dmp.DmpError) as e:
        dmp.purify(Hd, 32, mode="int8", slices=6, executor="tc", method="trs4", tape=tape)
    assert e.value.code == dmp.ERR_UNSUPPORTED
    bad = dmp.make_opts("int8", 6, "tc")
    bad.method = 3
    with pytest.raises(dmp.DmpError) as e:
        dmp.purify_workspace_bytes(128, bad)
    assert e.value.code == dmp.ERR_INVALID_ARG
