"""GPU vs oracle: the late-slice schedule of dm_purify (opts late_slices,
late_idem): the same passes switch to fewer slices as in the oracle, P and the
refined energy agree with the oracle's, and the energy keeps most of the
accuracy of the full slice count while a large share of the passes run with
fewer slices. Rejected where not offered (tape, SP2 / TRS4, batched)."""

from functools import partial

import numpy as np
import pytest
import torch

from oracle import ozaki as oz
from oracle import purify as pu
from synth import make_hamiltonian

pytestmark = pytest.mark.gpu


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("mode,s,late,refine", [("int8", 5, 4, 8), ("int8", 7, 5, 0), ("e4m3", 8, 6, 11)])
def test_matches_oracle(dmp, mode, s, late, refine):
    n, n_occ = 300, 75
    h = make_hamiltonian(n, n_occ, occ=(-1.5, -0.01), virt=(0.01, 1.5), seed=61)
    beta, rounding = (7, "trunc") if mode == "int8" else (5, "nearest")

    def prod(k):
        return partial(oz.ozaki_gemm, s=k, beta=beta, rounding=rounding)

    rp = prod(refine) if refine else None
    ref = pu.purify(h.H, n_occ, tol=1e-10, product=prod(s), late_product=prod(late), late_idem=1.0,
                    refine_product=rp)
    ref_lo = pu.purify(h.H, n_occ, tol=1e-10, product=prod(late), refine_product=rp)
    P, info = dmp.purify(_dev(h.H), n_occ, mode=mode, slices=s, executor="tc", tol=1e-10, refine=refine,
                         late_slices=late, late_idem=1.0)
    P = P.cpu().numpy()
    assert ref["late_iters"] > 0
    # the switch (the first iterate within 1 of idempotency) is the oracle's; the
    # stop at the late slices' noise floor may come a few passes apart
    assert abs((info["iters"] - info["late_iters"]) - (ref["iters"] - ref["late_iters"])) <= 1
    assert abs(info["iters"] - ref["iters"]) <= 4
    # both runs end at the late slices' noise floor, where the pass they stop at
    # differs with rounding: P and the energy are at least as accurate as the
    # oracle's run with the late slice count throughout
    V = h.Q[:, :n_occ]
    P_star = V @ V.T
    assert np.max(np.abs(P - P_star)) <= 2.0 * np.max(np.abs(ref_lo["P"] - P_star))
    E_star = float(np.sum(h.e[:n_occ]))
    assert abs(info["energy"] - E_star) <= 2.0 * abs(ref_lo["energy"] - E_star) + 1e-13 * abs(E_star)


def test_keeps_the_refined_energy_at_the_benchmark_spectrum(dmp):
    """n = 2048 with the benchmark's spectrum: five slices switching to four
    once the iterate is within 0.5 of idempotency, plus the refinement step,
    stay well more accurate than four slices throughout."""
    n, n_occ = 2048, 512
    h = make_hamiltonian(n, n_occ, occ=(-1.5, -0.01), virt=(0.01, 1.5), seed=62)
    H = _dev(h.H)
    E_star = float(np.sum(h.e[:n_occ]))
    _, low = dmp.purify(H, n_occ, mode="int8", slices=4, refine=8)
    _, sch = dmp.purify(H, n_occ, mode="int8", slices=5, refine=8, late_slices=4, late_idem=0.5)
    assert sch["late_iters"] > 0.1 * sch["iters"]
    assert abs(sch["energy"] - E_star) < 0.2 * abs(low["energy"] - E_star)


def test_rejected_where_not_offered(dmp):
    h = make_hamiltonian(64, 16, seed=63)
    H = _dev(h.H)
    with pytest.raises(dmp.DmpError):
        dmp.purify(H, 16, mode="int8", slices=5, method="trs4", late_slices=4, late_idem=1.0)
    with pytest.raises(dmp.DmpError):
        dmp.purify(H, 16, mode="int8", slices=5, late_slices=11, late_idem=1.0)  # beyond 10 slices
    opts = dmp.make_opts("int8", 5, "tc", late_slices=4, late_idem=1.0)
    tape = torch.empty(dmp.tape_bytes(64, opts), dtype=torch.uint8, device="cuda")
    with pytest.raises(dmp.DmpError):
        dmp.purify(H, 16, mode="int8", slices=5, tape=tape, late_slices=4, late_idem=1.0)
