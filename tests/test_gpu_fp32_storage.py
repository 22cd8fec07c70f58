"""GPU vs oracle: FP32 storage of the iterates (DMP_FLAG_FP32_STORAGE,
Sec. "Mixed Precision Purification").

Every matrix the GPU loop keeps is an FP32 value (checked bit for bit on the
returned P); P agrees with the oracle run under the same storage rule to the
FP32 resolution both reach; the energy stays far closer to the exact one. The
flag is refused where it is not offered (tape, backward, batched).
"""

from functools import partial

import numpy as np
import pytest
import torch

from oracle import ozaki as oz
from oracle import purify as pu
from oracle import variants as va
from synth import make_hamiltonian

pytestmark = pytest.mark.gpu


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _projector(h):
    V = h.Q[:, : h.n_occ]
    return V @ V.T


def _fp32_valued(M):
    return np.array_equal(M, M.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("mode,s", [("fp64", 0), ("int8", 7), ("e4m3", 9)])
def test_canonical_matches_oracle(dmp, mode, s):
    n, n_occ = 300, 75
    h = make_hamiltonian(n, n_occ, seed=31)
    if mode == "fp64":
        product = pu.fp64_product
    else:
        beta, rounding = (7, "trunc") if mode == "int8" else (5, "nearest")
        product = partial(oz.ozaki_gemm, s=s, beta=beta, rounding=rounding)
    ref = pu.purify(h.H, n_occ, tol=1e-10, product=product, store=pu.fp32_store)
    P, info = dmp.purify(_dev(h.H), n_occ, mode=mode, slices=s or 7, executor="auto", tol=1e-10,
                         fp32_storage=True)
    P = P.cpu().numpy()
    assert _fp32_valued(P)
    assert info["status"] in (dmp.OK, dmp.C_OUT_OF_RANGE, dmp.STALLED)
    P_star = _projector(h)
    # both loops end at the FP32 storage floor (about 5e-7 from the projector)
    assert np.max(np.abs(P - P_star)) <= 2.0 * np.max(np.abs(ref["P"] - P_star)) + 1e-7
    assert np.max(np.abs(P - ref["P"])) <= 2e-6
    E_star = float(np.sum(h.e[:n_occ]))
    assert abs(info["energy"] - E_star) <= 2e-8 * abs(E_star)
    assert np.array_equal(P, P.T)


def test_refinement_after_fp32_storage_is_unrounded(dmp):
    """The refinement step writes its result in full precision: P leaves the
    FP32 grid and the energy error drops further."""
    h = make_hamiltonian(256, 64, seed=32)
    _, plain = dmp.purify(_dev(h.H), 64, mode="int8", slices=7, fp32_storage=True)
    P, info = dmp.purify(_dev(h.H), 64, mode="int8", slices=7, fp32_storage=True, refine=9)
    assert info["refined"] == 1 and not _fp32_valued(P.cpu().numpy())
    E_star = float(np.sum(h.e[:64]))
    assert abs(info["energy"] - E_star) < abs(plain["energy"] - E_star)


@pytest.mark.parametrize("method", ["trs4", "sp2"])
def test_variants_keep_fp32_values(dmp, method):
    h = make_hamiltonian(256, 64, seed=33)
    ref = va.purify(h.H, 64, method=method, tol=1e-10, product=partial(oz.ozaki_gemm, s=7, beta=7),
                    store=pu.fp32_store)
    P, info = dmp.purify(_dev(h.H), 64, mode="int8", slices=7, method=method, fp32_storage=True)
    P = P.cpu().numpy()
    assert _fp32_valued(P)
    P_star = _projector(h)
    assert np.max(np.abs(P - P_star)) <= 2.0 * np.max(np.abs(ref["P"] - P_star)) + 1e-7


def test_refused_where_not_offered(dmp):
    h = make_hamiltonian(64, 16, seed=34)
    H = _dev(h.H)
    opts = dmp.make_opts("int8", 7, "tc", fp32_storage=True)
    tape = torch.empty(dmp.tape_bytes(64, opts), dtype=torch.uint8, device="cuda")
    with pytest.raises(RuntimeError):
        dmp.purify(H, 16, mode="int8", slices=7, tape=tape, fp32_storage=True)
