"""Batched purification (dm_purify_batched): many Hamiltonians of different
sizes in one graph launch, each checked against the single-matrix call, the
oracle and the exact projector."""

from functools import partial

import numpy as np
import pytest
import torch

from oracle import ozaki as oz
from oracle import purify as pu
from synth import batch_sizes, make_hamiltonian

pytestmark = pytest.mark.gpu


def _proj(h):
    V = h.Q[:, : h.n_occ]
    return V @ V.T


@pytest.mark.parametrize("mode,s", [("int8", 7), ("bf16", 6), ("e4m3", 10)])
def test_small_mixed_batch_matches_single_and_oracle(dmp, mode, s):
    sizes = [(128, 32), (160, 40), (256, 64), (300, 75), (448, 112), (520, 130)]
    hs = [make_hamiltonian(n, o, seed=700 + n) for n, o in sizes]
    Hs = [torch.from_numpy(h.H).cuda() for h in hs]
    Ps, infos, rc = dmp.purify_batched(Hs, [o for _, o in sizes], mode=mode, slices=s)
    assert rc in (dmp.OK, dmp.C_OUT_OF_RANGE, dmp.STALLED)
    for h, H, P, info in zip(hs, Hs, Ps, infos):
        Pn = P.cpu().numpy()
        P1, i1 = dmp.purify(H, h.n_occ, mode=mode, slices=s, executor="tc")
        assert np.max(np.abs(Pn - P1.cpu().numpy())) <= 1e-10, h.n
        assert abs(info["iters"] - i1["iters"]) <= 1
        assert np.max(np.abs(Pn - _proj(h))) <= 1e-8
        assert np.array_equal(Pn, Pn.T)
    # one of them against the oracle run in the same mode
    h = hs[3]
    beta, rounding = {"int8": (7, "trunc"), "bf16": (8, "nearest"), "e4m3": (5, "nearest")}[mode]
    ref = pu.purify(h.H, h.n_occ, tol=1e-10, product=partial(oz.ozaki_gemm, s=s, beta=beta, rounding=rounding))
    assert np.max(np.abs(Ps[3].cpu().numpy() - ref["P"])) <= 1e-8


def test_batch_of_64_autotuned(dmp):
    """The 64-matrix workload: n = 32 U{4..48}, n_occ = n/4, spectrum as in the
    n = 256 case (gap 0.2); s and the tile width chosen by the autotuner."""
    sizes = batch_sizes()
    hs = [make_hamiltonian(n, o, occ=(-2.0, -0.1), virt=(0.1, 2.0), seed=sd) for n, o, sd in sizes]
    Hs = [torch.from_numpy(h.H).cuda() for h in hs]
    Ps, infos, rc = dmp.purify_batched(Hs, [o for _, o, _ in sizes], mode="int8", slices=0)
    assert rc >= 0
    s = infos[0]["slices_used"]
    assert 4 <= s <= 10
    for h, P, info in zip(hs, Ps, infos):
        E = float(np.sum(h.e[: h.n_occ]))
        assert abs(info["energy"] - E) <= 1e-7 * abs(E), (h.n, info)
        assert abs(info["trace"] - h.n_occ) <= 1e-7 * h.n
    # a second call reuses the tuned choice and the cached graph
    Ps2, infos2, _ = dmp.purify_batched(Hs, [o for _, o, _ in sizes], mode="int8", slices=0)
    assert all(torch.equal(a, b) for a, b in zip(Ps, Ps2))


def test_batch_member_errors_are_reported(dmp):
    h1 = make_hamiltonian(200, 50, seed=1)
    h2 = make_hamiltonian(150, 30, seed=2)
    H2 = h2.H.copy()
    H2[4, 7] = np.nan
    Hs = [torch.from_numpy(h1.H).cuda(), torch.from_numpy(H2).cuda()]
    Ps, infos, rc = dmp.purify_batched(Hs, [50, 30], mode="int8", slices=7, raise_on_error=False)
    assert rc == dmp.ERR_NONFINITE
    assert infos[1]["status"] == dmp.ERR_NONFINITE
    assert infos[0]["status"] in (dmp.OK, dmp.C_OUT_OF_RANGE, dmp.STALLED)
    assert np.max(np.abs(Ps[0].cpu().numpy() - _proj(h1))) <= 1e-8


@pytest.mark.parametrize("mode,s,max_iter", [("int8", 7, 100), ("e4m3", 10, 100), ("int8", 6, 3)])
def test_stream_launches_match_the_graph(dmp, mode, s, max_iter):
    """DMP_FLAG_BATCHED_STREAM runs the same kernels as plain launches with a
    host check every two iterations: bit-identical P and the same reports, also
    when the iteration cap (odd here) stops the loop; and the per-phase
    profiler sees the launches."""
    sizes = [(128, 32), (224, 56), (300, 75), (512, 128)]
    hs = [make_hamiltonian(n, o, seed=900 + n) for n, o in sizes]
    Hs = [torch.from_numpy(h.H).cuda() for h in hs]
    occ = [o for _, o in sizes]
    Pg, ig, rg = dmp.purify_batched(Hs, occ, mode=mode, slices=s, max_iter=max_iter, raise_on_error=False)
    dmp.profile_enable(True)
    dmp.profile_reset()
    try:
        Ps, is_, rs = dmp.purify_batched(Hs, occ, mode=mode, slices=s, max_iter=max_iter, raise_on_error=False,
                                         stream_launches=True)
        torch.cuda.synchronize()
        prof = {k: dmp.profile_read(k) for k in (0, 1, 2)}
    finally:
        dmp.profile_enable(False)
    assert rs == rg
    assert all(torch.equal(a, b) for a, b in zip(Pg, Ps))
    for a, b in zip(ig, is_):
        assert a["iters"] == b["iters"] and a["status"] == b["status"] and a["energy"] == b["energy"]
    iters = max(i["iters"] for i in is_)
    assert iters <= max_iter
    # two products, two splits and one measure per iteration, in bodies of two
    # iterations, at least as many as the longest member ran
    products, splits, measures = prof[0][1], prof[1][1], prof[2][1]
    assert products == splits == 2 * measures and measures % 2 == 0 and measures >= iters
    assert all(prof[k][0] > 0 for k in prof)


@pytest.mark.parametrize("mode,tiles", [("int8", (128, 256, 512)), ("e4m3", (256, 512))])
def test_forced_tile_shapes_give_the_tuned_result(dmp, mode, tiles):
    """dmp_set_batched_tile: every tile shape gives bit-for-bit the autotuned
    call's P (the level sums are exact whatever the tiling); a shape the mode
    cannot use is refused, and 0 hands the choice back to the tuner."""
    sizes = [(160, 40), (256, 64), (416, 104)]
    hs = [make_hamiltonian(n, o, seed=950 + n) for n, o in sizes]
    Hs = [torch.from_numpy(h.H).cuda() for h in hs]
    occ = [o for _, o in sizes]
    s = 7 if mode == "int8" else 10
    want, _, _ = dmp.purify_batched(Hs, occ, mode=mode, slices=s)
    try:
        for t in tiles:
            dmp.set_batched_tile(t)
            got, _, _ = dmp.purify_batched(Hs, occ, mode=mode, slices=s)
            assert all(torch.equal(a, b) for a, b in zip(want, got)), t
        if mode == "e4m3":
            dmp.set_batched_tile(128)
            _, _, rc = dmp.purify_batched(Hs, occ, mode=mode, slices=s, raise_on_error=False)
            assert rc == dmp.ERR_UNSUPPORTED
    finally:
        assert dmp.set_batched_tile(0) in tiles + (128,)
    assert dmp.lib().dmp_set_batched_tile(384) == dmp.ERR_INVALID_ARG


@pytest.mark.parametrize("mode,s,r", [("int8", 5, 8), ("e4m3", 7, 10), ("bf16", 5, 7)])
def test_batched_refinement_matches_single_and_oracle(dmp, mode, s, r):
    """opts.refine_slices in the batched call: every member gets dm_purify's
    refinement step (one McWeeny step with r-slice products after the loop), so
    it matches its own refined dm_purify call; one member against the oracle's
    refinement in the same digit rule."""
    sizes = [(128, 32), (200, 50), (320, 80), (448, 112)]
    hs = [make_hamiltonian(n, o, seed=970 + n) for n, o in sizes]
    Hs = [torch.from_numpy(h.H).cuda() for h in hs]
    Ps, infos, rc = dmp.purify_batched(Hs, [o for _, o in sizes], mode=mode, slices=s, refine=r)
    assert rc in (dmp.OK, dmp.C_OUT_OF_RANGE, dmp.STALLED)
    beta = {"int8": 7, "bf16": 8, "e4m3": 5}[mode]
    # the batched and single loops sum their traces in different orders, and at
    # these small slice counts a last-bit difference of an iterate moves
    # truncated digits: agreement to a few dozen units of the slices' resolution
    tol = 50.0 * 2.0 ** (-beta * s)
    for h, H, P, info in zip(hs, Hs, Ps, infos):
        assert info["refined"] == 1
        assert info["band_energy"] == 2.0 * info["energy"]
        P1, i1 = dmp.purify(H, h.n_occ, mode=mode, slices=s, executor="tc", refine=r)
        Pn = P.cpu().numpy()
        assert np.max(np.abs(Pn - P1.cpu().numpy())) <= tol, h.n
        assert abs(info["energy"] - i1["energy"]) <= tol * abs(i1["energy"]), h.n
        assert np.array_equal(Pn, Pn.T)
        # the refinement beats the loop's own energy error
        E = float(np.sum(h.e[: h.n_occ]))
        assert abs(info["energy"] - E) <= abs(info["energy_unrefined"] - E) + 1e-14 * abs(E)
    h = hs[2]
    beta, rounding = {"int8": (7, "trunc"), "bf16": (8, "nearest"), "e4m3": (5, "nearest")}[mode]
    ref = pu.purify(h.H, h.n_occ, tol=1e-10, product=partial(oz.ozaki_gemm, s=s, beta=beta, rounding=rounding),
                    refine_product=partial(oz.ozaki_gemm, s=r, beta=beta, rounding=rounding))
    assert np.max(np.abs(Ps[2].cpu().numpy() - ref["P"])) <= 1e-8
    assert abs(infos[2]["energy"] - ref["energy"]) <= 1e-10 * abs(ref["energy"])


def test_batched_refinement_with_tuned_slices_on_the_64_workload(dmp):
    """The 64-matrix workload with the refinement step and the slice count left
    to the tuner (which then compares refined energies): every member within
    1e-8 of its exact band energy."""
    sizes = batch_sizes()
    hs = [make_hamiltonian(n, o, occ=(-2.0, -0.1), virt=(0.1, 2.0), seed=sd) for n, o, sd in sizes]
    Hs = [torch.from_numpy(h.H).cuda() for h in hs]
    Ps, infos, rc = dmp.purify_batched(Hs, [o for _, o, _ in sizes], mode="int8", slices=0, refine=8)
    assert rc >= 0
    assert 4 <= infos[0]["slices_used"] <= 10
    for h, info in zip(hs, infos):
        E = float(np.sum(h.e[: h.n_occ]))
        assert info["refined"] == 1
        assert abs(info["energy"] - E) <= 1e-8 * abs(E), (h.n, info)
