"""The bounded device waits of the tcgen05 product kernel, made to run out.

dmp_test_stall_next_product withholds the first operand stage of every CTA of
the next product launch and bounds its waits by a short limit: the MMA
issuer's wait on that stage's barrier expires, the kernel raises the call's
error flag, drains the copies it did issue, frees its tensor memory and
returns. The call must report DMP_ERR_TIMEOUT within about the limit (not the
normal 5 s), and the next call on the same stream must again be bit-exact
against the oracle -- for the single-CTA and the paired kernel, the INT8 and
E4M3 digits, a whole purification and the finite-temperature expansion (whose
later products must stop). No memory is touched by the injected condition and
nothing faults: the failure is a barrier that never completes.
"""

import time
from functools import partial

import numpy as np
import pytest
import torch

from oracle import ozaki as oz
from oracle import purify as pu
from synth import make_hamiltonian

pytestmark = pytest.mark.gpu

LIMIT_US = 2000  # 2 ms


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _expect_timeout(dmp, fn):
    t0 = time.perf_counter()
    with pytest.raises(dmp.DmpError) as ei:
        fn()
    torch.cuda.synchronize()
    assert ei.value.code == dmp.ERR_TIMEOUT
    return time.perf_counter() - t0


@pytest.mark.parametrize("pairing", [False, True])
@pytest.mark.parametrize("mode,beta,rounding", [("int8", 7, "trunc"), ("e4m3", 5, "nearest")])
def test_product_wait_runs_out_then_recovers(dmp, pairing, mode, beta, rounding):
    rng = np.random.default_rng(41)
    m, n, k, s = 512, 384, 640, 5
    A = rng.standard_normal((m, k))
    B = rng.standard_normal((k, n))
    Ad, Bd = _dev(A), _dev(B)
    want = oz.ozaki_gemm(A, B, s, beta, rounding=rounding)
    prev = dmp.set_tc_pairing(pairing)
    try:
        dmp.test_stall_next_product(LIMIT_US)
        dt = _expect_timeout(dmp, lambda: dmp.ozaki_gemm(Ad, Bd, mode, s, "tc"))
        assert dt < 1.0, f"the abort took {dt:.3f} s: the short limit was not applied"
        # one-shot: the next call on the same stream is normal and exact
        got = dmp.ozaki_gemm(Ad, Bd, mode, s, "tc").cpu().numpy()
        assert np.array_equal(got, want)
    finally:
        dmp.set_tc_pairing(prev)


def test_purification_reports_the_timeout_then_recovers(dmp):
    h = make_hamiltonian(320, 80, seed=43)
    Hd = _dev(h.H)
    dmp.test_stall_next_product(LIMIT_US)
    _expect_timeout(dmp, lambda: dmp.purify(Hd, 80, mode="int8", slices=7, executor="tc"))
    ref = pu.purify(h.H, 80, tol=1e-10, product=partial(oz.ozaki_gemm, s=7, beta=7))
    P, info = dmp.purify(Hd, 80, mode="int8", slices=7, executor="tc")
    assert info["status"] >= 0
    assert np.max(np.abs(P.cpu().numpy() - ref["P"])) <= 1e-8


def test_expansion_stops_after_a_stalled_product(dmp):
    h = make_hamiltonian(256, 80, occ=(-2.0, 0.0), virt=(0.0, 2.0), seed=44)
    Hd = _dev(h.H)
    kw = dict(mu=0.0, bounds=(-2.0, 2.0), mode="int8", slices=6, scheme="recurrence")
    before = dmp.launch_count()
    _, info = dmp.foe(Hd, 0.1, 60, **kw)
    normal = dmp.launch_count() - before
    assert info["products"] == 58
    before = dmp.launch_count()
    dmp.test_stall_next_product(LIMIT_US)
    _expect_timeout(dmp, lambda: dmp.foe(Hd, 0.1, 60, **kw))
    stalled = dmp.launch_count() - before
    # the host stops enqueueing at its next check of the flag (every 8 products)
    assert stalled < normal // 3, (stalled, normal)
    P, info = dmp.foe(Hd, 0.1, 60, **kw)
    assert info["status"] == dmp.OK and bool(torch.isfinite(P).all())


def test_hook_rejects_a_negative_limit_and_cancels(dmp):
    with pytest.raises(dmp.DmpError):
        dmp.test_stall_next_product(-1)
    dmp.test_stall_next_product(LIMIT_US)
    dmp.test_stall_next_product(0)  # cancelled: the next product runs normally
    rng = np.random.default_rng(45)
    A = rng.standard_normal((200, 200))
    got = dmp.ozaki_gemm(_dev(A), _dev(A), "int8", 6, "tc").cpu().numpy()
    assert np.array_equal(got, oz.ozaki_gemm(A, A, 6, 7))
