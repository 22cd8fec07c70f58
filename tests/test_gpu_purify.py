"""GPU vs oracle: canonical purification through dm_purify.

FP64 mode agrees with the FP64 oracle to 1e-10 max-abs; Ozaki INT8 with s >= 7
agrees with the oracle run in the same mode to 1e-8 max-abs (and with the exact
projector). Edge cases: the smallest n, ragged n, invalid arguments, NaN input,
a degenerate H, the iteration cap. The full-size case (n = 8192) checks the
properties that hold at any size: energy against the exact spectrum, trace,
idempotency.
"""

from functools import partial

import numpy as np
import pytest
import torch

from oracle import ozaki as oz
from oracle import purify as pu
from synth import config_hamiltonian, make_hamiltonian

pytestmark = pytest.mark.gpu


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _projector(h):
    V = h.Q[:, : h.n_occ]
    return V @ V.T


def test_config0_fp64_matches_oracle(dmp):
    h = config_hamiltonian(0)
    ref = pu.purify(h.H, h.n_occ, tol=1e-10)
    P, info = dmp.purify(_dev(h.H), h.n_occ, mode="fp64", tol=1e-10)
    P = P.cpu().numpy()
    assert info["status"] == dmp.OK
    assert abs(info["iters"] - ref["iters"]) <= 1
    assert np.max(np.abs(P - ref["P"])) <= 1e-10
    assert np.max(np.abs(P - _projector(h))) <= 1e-10
    assert abs(info["energy"] - ref["energy"]) <= 1e-10 * abs(ref["energy"])
    assert np.array_equal(P, P.T)


@pytest.mark.parametrize("executor", ["imma", "tc"])
@pytest.mark.parametrize("n,n_occ,s", [(300, 75, 7), (300, 75, 8), (200, 13, 9), (600, 150, 7)])
def test_ozaki_int8_matches_oracle(dmp, executor, n, n_occ, s):
    h = make_hamiltonian(n, n_occ, seed=n + s)
    ref = pu.purify(h.H, n_occ, tol=1e-10, product=partial(oz.ozaki_gemm, s=s, beta=7))
    P, info = dmp.purify(_dev(h.H), n_occ, mode="int8", slices=s, executor=executor, tol=1e-10)
    P = P.cpu().numpy()
    assert info["status"] in (dmp.OK, dmp.C_OUT_OF_RANGE, dmp.STALLED)
    assert np.max(np.abs(P - ref["P"])) <= 1e-8
    assert np.max(np.abs(P - _projector(h))) <= 1e-8
    E_star = float(np.sum(h.e[:n_occ]))
    assert abs(info["energy"] - E_star) <= 1e-8 * abs(E_star)
    assert np.array_equal(P, P.T)


def test_bf16_mode_matches_oracle(dmp):
    h = make_hamiltonian(300, 75, seed=17)
    ref = pu.purify(h.H, 75, tol=1e-10, product=partial(oz.ozaki_gemm, s=6, beta=8, rounding="nearest"))
    P, info = dmp.purify(_dev(h.H), 75, mode="bf16", slices=6, executor="tc", tol=1e-10)
    P = P.cpu().numpy()
    assert np.max(np.abs(P - ref["P"])) <= 1e-8
    assert np.max(np.abs(P - _projector(h))) <= 1e-8


@pytest.mark.parametrize("executor", ["imma", "tc"])
def test_ozaki_error_falls_with_slices(dmp, executor):
    h = make_hamiltonian(384, 96, seed=11)
    P_star = _projector(h)
    errs = []
    for s in (3, 5, 7, 9):
        P, _ = dmp.purify(_dev(h.H), 96, mode="int8", slices=s, executor=executor, tol=1e-10)
        errs.append(np.max(np.abs(P.cpu().numpy() - P_star)))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs


def test_smallest_and_ragged_sizes(dmp):
    for n, n_occ in [(2, 1), (3, 1), (129, 40), (255, 64)]:
        h = make_hamiltonian(n, n_occ, seed=n)
        for mode in ("fp64", "int8"):
            P, info = dmp.purify(_dev(h.H), n_occ, mode=mode, slices=9, tol=1e-10)
            assert info["status"] in (dmp.OK, dmp.C_OUT_OF_RANGE), (n, mode, info)
            assert np.max(np.abs(P.cpu().numpy() - _projector(h))) <= 1e-8, (n, mode)


def test_leading_dimension(dmp):
    h = make_hamiltonian(150, 30, seed=3)
    Hpad = np.zeros((150, 160))
    Hpad[:, :150] = h.H
    Hd = _dev(Hpad)[:, :150]
    Pd = torch.zeros((150, 170), dtype=torch.float64, device="cuda")[:, :150]
    P, info = dmp.purify(Hd, 30, mode="int8", slices=8, P=Pd)
    assert np.max(np.abs(P.cpu().numpy() - _projector(h))) <= 1e-8


def test_errors_and_statuses(dmp):
    h = make_hamiltonian(64, 16, seed=4)
    with pytest.raises(dmp.DmpError) as e:
        dmp.purify(_dev(h.H), 0)
    assert e.value.code == dmp.ERR_INVALID_ARG
    with pytest.raises(dmp.DmpError):
        dmp.purify(_dev(h.H), 64)
    H = h.H.copy()
    H[3, 9] = np.nan
    with pytest.raises(dmp.DmpError) as e:
        dmp.purify(_dev(H), 16)
    assert e.value.code == dmp.ERR_NONFINITE
    with pytest.raises(dmp.DmpError) as e:
        dmp.purify(_dev(2.0 * np.eye(16)), 4)
    assert e.value.code == dmp.ERR_INVALID_ARG
    P, info = dmp.purify(_dev(h.H), 16, mode="fp64", max_iter=1)
    assert info["status"] == dmp.NOT_CONVERGED and info["iters"] == 1
    ref = pu.purify(h.H, 16, max_iter=1)
    assert np.max(np.abs(P.cpu().numpy() - ref["P"])) <= 1e-12


def test_deterministic_and_executors_agree(dmp):
    """The two executors produce the same level sums, so the whole purification
    is bit-identical between them (and between runs)."""
    h = make_hamiltonian(260, 65, seed=5)
    P1, i1 = dmp.purify(_dev(h.H), 65, mode="int8", slices=7, executor="tc")
    P2, i2 = dmp.purify(_dev(h.H), 65, mode="int8", slices=7, executor="tc")
    P3, i3 = dmp.purify(_dev(h.H), 65, mode="int8", slices=7, executor="imma")
    assert torch.equal(P1, P2) and i1 == i2
    assert torch.equal(P1, P3) and i1["iters"] == i3["iters"]


def test_full_size_config2_int8(dmp):
    """n = 8192, n_occ = 2048, gap 0.02: the benchmark workload at s = 7."""
    h = config_hamiltonian(2, device="cuda")
    P, info = dmp.purify(h.H, h.n_occ, mode="int8", slices=7, executor="tc", tol=1e-10)
    E_star = float(np.sum(h.e[: h.n_occ]))
    assert info["status"] in (dmp.OK, dmp.C_OUT_OF_RANGE, dmp.STALLED), info
    assert abs(info["energy"] - E_star) <= 1e-8 * abs(E_star), info
    assert abs(info["trace"] - h.n_occ) <= 1e-8 * h.n
    assert torch.equal(P, P.T)
