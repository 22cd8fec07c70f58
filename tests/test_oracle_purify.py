"""Pins for the purification oracle.

Checks against closed forms and mathematical properties: the spectral projector
of H = Q diag(e) Q^T, a dense eigensolver, a hand-worked n = 3 case, McWeeny's
printed step (Sec. "Density Matrix Purification"), trace conservation of the
canonical update, Gershgorin's theorem, and the stopping rules.
"""

import json
import os
from fractions import Fraction
from functools import partial

import numpy as np
import pytest

from oracle import ozaki as oz
from oracle import purify as pu
from oracle import variants as va
from synth import config_hamiltonian, make_hamiltonian


def _projector(Q, n_occ):
    V = Q[:, :n_occ]
    return V @ V.T


def _random_spd_spectrum_matrix(n, vals, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (Q * vals) @ Q.T


@pytest.fixture(scope="module")
def c0():
    h = config_hamiltonian(0)
    return h, pu.purify(h.H, h.n_occ, tol=1e-10)


def test_config0_closed_form(c0):
    h, r = c0
    P_star = _projector(h.Q, h.n_occ)
    assert r["status"] == pu.CONVERGED
    assert np.max(np.abs(r["P"] - P_star)) <= 1e-10
    assert abs(np.trace(r["P"]) - h.n_occ) <= 1e-10 * h.n
    assert r["idem"] < 1e-10
    E_star = float(np.sum(h.e[: h.n_occ]))
    assert abs(r["energy"] - E_star) <= 1e-12 * abs(E_star)
    assert all(0.0 <= c <= 1.0 for c in r["c_history"])


def test_trace_conserved_along_iterations(c0):
    h, r = c0
    assert max(abs(t - h.n_occ) for t in r["trace_history"]) <= 1e-11 * h.n


def test_energy_non_increasing(c0):
    _, r = c0
    b = r["band_history"]
    assert all(b[i + 1] <= b[i] + 1e-12 * abs(b[i]) for i in range(len(b) - 1))


def test_tiny_against_eigensolver():
    rng = np.random.default_rng(8)
    for n, n_occ in [(5, 2), (16, 5), (48, 20)]:
        G = rng.standard_normal((n, n))
        H = 0.5 * (G + G.T)
        w, V = np.linalg.eigh(H)
        if w[n_occ] - w[n_occ - 1] < 0.05:
            continue
        r = pu.purify(H, n_occ, tol=1e-12)
        assert r["status"] == pu.CONVERGED
        assert np.max(np.abs(r["P"] - V[:, :n_occ] @ V[:, :n_occ].T)) < 1e-10


def test_hand_worked_n3(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "pm_n3_hand.json")))
    H = np.diag(g["H_diag"])
    P0, info = pu.initial_guess(H, g["n_occ"])
    assert info["lam"] == pytest.approx(g["lambda"], rel=1e-15)
    assert info["mu"] == pytest.approx(g["mu"], rel=1e-15)
    assert np.allclose(np.diag(P0), g["P0_diag"], rtol=0, atol=1e-15)
    t1, t2, t3 = np.trace(P0), np.trace(P0 @ P0), np.trace(P0 @ P0 @ P0)
    c = pu.pm_coefficient(t1, t2, t3)
    assert c == pytest.approx(g["c0"], abs=1e-14)
    P1 = pu.pm_update(P0, P0 @ P0, P0 @ P0 @ P0, c)
    assert np.allclose(np.diag(P1), g["P1_diag"], rtol=0, atol=1e-14)


@pytest.mark.parametrize("branch", ["low", "high"])
def test_update_conserves_trace(branch):
    """tr(P') = tr(P) for any spectrum in (0, 1): the defining property of the
    canonical coefficient. A dropped term in c or in a branch breaks it."""
    rng = np.random.default_rng(9 if branch == "low" else 10)
    n = 30
    for _ in range(20):
        if branch == "low":
            vals = rng.uniform(0.05, 0.45, size=n)  # mostly below 1/2: c < 1/2
        else:
            vals = rng.uniform(0.55, 0.95, size=n)  # mostly above 1/2: c > 1/2
        P = _random_spd_spectrum_matrix(n, vals, rng.integers(1 << 30))
        X2, X3 = P @ P, P @ P @ P
        c = pu.pm_coefficient(np.trace(P), np.trace(X2), np.trace(X3))
        assert (c < 0.5) == (branch == "low")
        P1 = pu.pm_update(P, X2, X3, c)
        assert abs(np.trace(P1) - np.trace(P)) < 1e-12 * n
        # the update maps [0, 1] into [0, 1] with fixed points 0 and 1
        w = np.linalg.eigvalsh(0.5 * (P1 + P1.T))
        assert w.min() > -1e-12 and w.max() < 1 + 1e-12


def test_c_half_is_mcweeny():
    """With c = 1/2 both branches equal McWeeny's printed step 3P^2 - 2P^3."""
    rng = np.random.default_rng(11)
    x = rng.uniform(0.05, 0.45, size=10)
    vals = np.concatenate([x, 1.0 - x])  # symmetric about 1/2 -> c = 1/2 exactly
    P = _random_spd_spectrum_matrix(20, vals, 12)
    X2, X3 = P @ P, P @ P @ P
    c = pu.pm_coefficient(np.trace(P), np.trace(X2), np.trace(X3))
    assert c == pytest.approx(0.5, abs=1e-12)
    mcweeny = 3 * X2 - 2 * X3
    for cc in (0.5, np.nextafter(0.5, 0)):
        assert np.allclose(pu.pm_update(P, X2, X3, cc), mcweeny, atol=1e-12)


def test_gershgorin_encloses_spectrum_and_p0_in_unit_interval():
    for seed in range(4):
        h = make_hamiltonian(64, 16, seed=100 + seed)
        h_min, h_max, _, _ = pu.gershgorin(h.H)
        w = np.linalg.eigvalsh(h.H)
        assert h_min <= w.min() and w.max() <= h_max
        P0, _ = pu.initial_guess(h.H, 16)
        w0 = np.linalg.eigvalsh(P0)
        assert w0.min() >= -1e-14 and w0.max() <= 1 + 1e-14
        assert abs(np.trace(P0) - 16) < 1e-12


def test_diagonal_hamiltonian_gives_occupation_diagonal():
    e = np.array([0.3, -1.0, 0.7, -0.2, 1.5, -0.6])
    r = pu.purify(np.diag(e), 3, tol=1e-12)
    occ = np.argsort(e)[:3]
    want = np.zeros(6)
    want[occ] = 1.0
    assert np.allclose(r["P"], np.diag(want), atol=1e-12)


def test_stopping_rules_and_errors():
    h = make_hamiltonian(32, 8, seed=5)
    r = pu.purify(h.H, 8, max_iter=1)
    assert r["status"] == pu.NOT_CONVERGED and r["iters"] == 1
    r = pu.purify(h.H, 8, tol=0.0, max_iter=100)  # tol 0 can never be met
    assert r["status"] in (pu.C_OUT_OF_RANGE, pu.STALLED, pu.NOT_CONVERGED)
    assert np.max(np.abs(r["P"] - _projector(h.Q, 8))) < 1e-10
    for bad in (0, 32, -1):
        with pytest.raises(ValueError):
            pu.purify(h.H, bad)
    H = h.H.copy()
    H[2, 3] = np.nan
    with pytest.raises(ValueError):
        pu.purify(H, 8)
    with pytest.raises(ValueError):
        pu.purify(2.0 * np.eye(8), 3)


def test_energy_tolerance_rule():
    h = make_hamiltonian(64, 16, seed=6)
    r = pu.purify(h.H, 16, tol=0.0, energy_tol=1e-8)
    assert r["status"] == pu.CONVERGED
    assert abs(r["band_history"][-1] - r["band_history"][-2]) < 1e-8


def test_ozaki_mode_converges_towards_projector():
    """An Ozaki-mode run reaches the projector to within an error that falls
    with the slice count (the behaviour Fig. 6 reports)."""
    h = make_hamiltonian(96, 24, seed=7)
    P_star = _projector(h.Q, 24)
    errs = []
    for s in (3, 5, 7):
        r = pu.purify(h.H, 24, tol=1e-10, product=partial(oz.ozaki_gemm, s=s, beta=7))
        errs.append(np.max(np.abs(r["P"] - P_star)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-9


def test_nearest_digit_mode_converges_towards_projector():
    """The same with nearest 5-bit digits (the E4M3 mode): the error falls with
    the slice count, and 7 such slices land near 5 truncated 7-bit ones."""
    h = make_hamiltonian(96, 24, seed=7)
    P_star = _projector(h.Q, 24)
    errs = []
    for s in (4, 7, 10):
        r = pu.purify(h.H, 24, tol=1e-10, product=partial(oz.ozaki_gemm, s=s, beta=5, rounding="nearest"))
        errs.append(np.max(np.abs(r["P"] - P_star)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-9
    r5 = pu.purify(h.H, 24, tol=1e-10, product=partial(oz.ozaki_gemm, s=5, beta=7))
    ratio = errs[1] / np.max(np.abs(r5["P"] - P_star))
    assert 0.05 < ratio < 20.0


def test_error_metrics_paper_conventions():
    h = make_hamiltonian(40, 10, seed=8)
    P = _projector(h.Q, 10)
    m = pu.error_metrics(P, h.H, P_ref=P, E_ref=float(np.sum(h.e[:10])))
    assert m["rmsd"] == 0.0 and m["max_abs"] == 0.0
    assert m["band_energy"] == pytest.approx(2 * np.sum(h.e[:10]), rel=1e-12)
    assert m["commutator"] < 1e-12 and m["rel_energy"] < 1e-13


def test_spectral_loop_matches_matrix_loop():
    """The eigenvalue form of the loop reproduces the matrix loop: same
    iteration count, same coefficients, final eigenvalues equal to those of
    the final P (checked against a dense eigensolver)."""
    h = make_hamiltonian(80, 20, seed=21)
    r = pu.purify(h.H, 20, tol=1e-10)
    x0 = pu.initial_eigenvalues(h.H, 20, h.e)
    sp = pu.spectral_purify(x0, h.e, tol=1e-10)
    assert sp["iters"] == r["iters"] and sp["status"] == r["status"]
    # c is a ratio of traces that both vanish at convergence: compare the
    # well-conditioned early steps tightly, the last ones loosely
    assert np.allclose(sp["c_history"][:-5], r["c_history"][:-5], rtol=0, atol=1e-10)
    assert np.allclose(sp["c_history"], r["c_history"], rtol=0, atol=1e-4)
    w = np.sort(np.linalg.eigvalsh(0.5 * (r["P"] + r["P"].T)))
    assert np.allclose(np.sort(sp["x"]), w, atol=1e-10)
    P0, _ = pu.initial_guess(h.H, 20)
    assert np.allclose(np.sort(np.linalg.eigvalsh(P0)), np.sort(x0), atol=1e-13)


# ---- refinement: one McWeeny step after the loop (Sec. "Precision Requirements Sweep")

def test_mcweeny_step_matches_printed_polynomial_exactly_on_diagonals():
    """P = diag(l): P' = diag(3 l^2 - 2 l^3) of the printed equation, checked
    against exact rationals (the FP64 products of diagonal matrices are exact,
    so only the last multiply-adds round)."""
    rng = np.random.default_rng(3)
    lam = np.concatenate([rng.uniform(-0.2, 1.2, 40), [0.0, 1.0, 0.5, -1e-9, 1.0 + 1e-9]])
    got = pu.mcweeny_step(np.diag(lam))
    assert np.count_nonzero(got - np.diag(np.diag(got))) == 0
    for x, g in zip(lam, np.diag(got)):
        q = Fraction(float(x))
        exact = 3 * q * q - 2 * q * q * q
        assert abs(Fraction(float(g)) - exact) <= Fraction(1, 2 ** 50) * max(1, abs(exact))


def test_mcweeny_step_maps_eigenvalues_of_a_rotated_matrix():
    rng = np.random.default_rng(4)
    n = 60
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = rng.uniform(-0.1, 1.1, n)
    P = (Q * lam) @ Q.T
    P = 0.5 * (P + P.T)
    got = np.linalg.eigvalsh(pu.mcweeny_step(P))
    want = np.sort(3 * lam ** 2 - 2 * lam ** 3)
    assert np.max(np.abs(got - want)) < 1e-13


def test_refinement_squares_the_distance_to_a_projector():
    """Eigenvalues 0 + d and 1 - d move to 3 d^2 - 2 d^3 and 1 - (3 d^2 - 2 d^3):
    the idempotency error goes from O(d) to O(d^2)."""
    rng = np.random.default_rng(5)
    n, n_occ = 80, 20
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    d = rng.uniform(1e-5, 1e-4, n)
    lam = np.where(np.arange(n) < n_occ, 1.0 - d, d)
    P = (Q * lam) @ Q.T
    P = 0.5 * (P + P.T)
    R = pu.mcweeny_step(P)
    lam_r = np.where(np.arange(n) < n_occ, 1.0 - (3 * d ** 2 - 2 * d ** 3), 3 * d ** 2 - 2 * d ** 3)
    idem_r = np.sqrt(np.sum((lam_r ** 2 - lam_r) ** 2))
    assert abs(np.linalg.norm(R @ R - R) - idem_r) <= 1e-3 * idem_r + 1e-13
    assert np.linalg.norm(R @ R - R) < 1e-3 * np.linalg.norm(P @ P - P)


def test_refinement_fixes_the_energy_of_a_low_slice_purification():
    """The paper's observation: one full-precision McWeeny step after a
    low-precision purification cuts the energy error by orders of magnitude.
    Here Ozaki-INT8 products with s = 4, refined with FP64 and with s = 9
    Ozaki products (FP64 level)."""
    h = make_hamiltonian(128, 32, occ=(-1.5, -0.01), virt=(0.01, 1.5), seed=61)
    E_star = float(np.sum(np.sort(h.e)[:32]))
    low = partial(oz.ozaki_gemm, s=4, beta=7)
    r64 = pu.purify(h.H, 32, tol=1e-10, product=low, refine_product=pu.fp64_product)
    r9 = pu.purify(h.H, 32, tol=1e-10, product=low, refine_product=partial(oz.ozaki_gemm, s=9, beta=7))
    before = abs(r64["energy_unrefined"] - E_star) / abs(E_star)
    after = abs(r64["energy"] - E_star) / abs(E_star)
    assert r64["refined"] and after < 1e-2 * before and after < 1e-9
    assert np.max(np.abs(r9["P"] - r64["P"])) < 1e-13
    assert r64["iters"] == r9["iters"] and r64["band_energy"] == 2.0 * r64["energy"]


# ----------------------------------------------------------------- FP32 storage (Sec. "Mixed Precision Purification")

def _is_fp32_valued(M):
    return np.array_equal(M, M.astype(np.float32).astype(np.float64))


def test_fp32_storage_keeps_float32_values_and_reaches_the_projector():
    """Every stored matrix is an FP32 value; the result still approaches the
    exact projector to FP32 resolution, and the band energy (second order in
    the error of P) far closer: the paper's finding that FP32 storage with
    FP64 accumulation is adequate."""
    h = make_hamiltonian(96, 24, seed=7)
    P_star = _projector(h.Q, 24)
    E_star = float(np.sum(h.e[:24]))
    r = pu.purify(h.H, 24, tol=1e-10, store=pu.fp32_store, record=True)
    assert all(_is_fp32_valued(P) for P in r["iterates"])
    assert all(_is_fp32_valued(X2) for X2 in r["squares"])
    err = np.max(np.abs(r["P"] - P_star))
    assert 1e-9 < err < 2e-6  # FP32 resolution: well above FP64's, well below single digits
    assert abs(r["energy"] - E_star) <= 2e-8 * abs(E_star)
    ref = pu.purify(h.H, 24, tol=1e-10)
    assert np.max(np.abs(ref["P"] - P_star)) < 1e-12  # the same loop with FP64 storage


def test_fp32_storage_with_ozaki_products():
    h = make_hamiltonian(96, 24, seed=9)
    P_star = _projector(h.Q, 24)
    r = pu.purify(h.H, 24, tol=1e-10, product=partial(oz.ozaki_gemm, s=7, beta=7), store=pu.fp32_store,
                  record=True)
    assert all(_is_fp32_valued(P) for P in r["iterates"])
    assert np.max(np.abs(r["P"] - P_star)) < 2e-6


def test_fp32_storage_in_trs4_and_sp2():
    h = make_hamiltonian(96, 24, seed=10)
    P_star = _projector(h.Q, 24)
    for method in ("trs4", "sp2"):
        r = va.purify(h.H, 24, method=method, tol=1e-10, store=pu.fp32_store, record=True)
        assert all(_is_fp32_valued(X) for X in r["iterates"]), method
        assert np.max(np.abs(r["P"] - P_star)) < 2e-6, method


def test_planted_store_of_the_initial_guess_only_fails():
    """A storage rule applied to P_0 alone leaves the later iterates off the FP32 grid."""
    h = make_hamiltonian(64, 16, seed=11)
    calls = {"n": 0}

    def first_only(M):
        calls["n"] += 1
        return pu.fp32_store(M) if calls["n"] == 1 else M

    r = pu.purify(h.H, 16, tol=1e-10, store=first_only, record=True)
    assert _is_fp32_valued(r["iterates"][0])
    assert not all(_is_fp32_valued(P) for P in r["iterates"])


# ----------------------------------------------------------------- late-slice schedule

def test_late_schedule_with_the_same_product_changes_nothing():
    h = make_hamiltonian(96, 24, seed=12)
    prod = partial(oz.ozaki_gemm, s=6, beta=7)
    ref = pu.purify(h.H, 24, tol=1e-10, product=prod)
    same = pu.purify(h.H, 24, tol=1e-10, product=prod, late_product=prod, late_idem=10.0)
    off = pu.purify(h.H, 24, tol=1e-10, product=prod, late_product=partial(oz.ozaki_gemm, s=3, beta=7), late_idem=0.0)
    for r in (same, off):
        assert np.array_equal(r["P"], ref["P"]) and r["iters"] == ref["iters"]
        assert r["idem_history"] == ref["idem_history"]
    assert same["late_iters"] > 0 and off["late_iters"] == 0


def test_late_schedule_switches_after_the_first_iterate_below_the_threshold():
    """The passes after the first update whose iterate had ||P^2 - P||_F below
    the threshold use the late product, and only those."""
    h = make_hamiltonian(128, 32, seed=13)
    seen = []

    def tag(s):
        def prod(A, B):
            seen.append(s)
            return oz.ozaki_gemm(A, B, s, 7)
        return prod

    tau = 1.0
    r = pu.purify(h.H, 32, tol=1e-10, product=tag(6), late_product=tag(4), late_idem=tau)
    idem = r["idem_history"]
    k_star = next(k for k, v in enumerate(idem) if v < tau)
    # pass k forms P^2 and P^3 (the last pass stops after P^2, or after P^3
    # when c leaves [0, 1]): late from pass k_star + 1 on
    last = 2 if r["status"] == pu.C_OUT_OF_RANGE else 1
    passes = []
    for k in range(r["iters"] + 1):
        passes += [k] * (2 if k < r["iters"] else last)
    assert [s for s in seen] == [4 if k > k_star else 6 for k in passes]
    assert r["late_iters"] == r["iters"] - k_star


def test_late_slices_keep_most_of_the_refined_energy():
    """With the refinement step, loop products of four slices once the iterate
    is within 1 of idempotency cost little energy accuracy: the error stays far
    below that of four slices throughout (the subspace is fixed early, while
    the gap between occupied and virtual eigenvalues is small)."""
    h = make_hamiltonian(256, 64, occ=(-1.5, -0.01), virt=(0.01, 1.5), seed=77)
    E = float(np.sum(h.e[:64]))
    s5, s4 = partial(oz.ozaki_gemm, s=5, beta=7), partial(oz.ozaki_gemm, s=4, beta=7)
    r8 = partial(oz.ozaki_gemm, s=8, beta=7)
    low = pu.purify(h.H, 64, tol=1e-10, product=s4, refine_product=r8)
    sched = pu.purify(h.H, 64, tol=1e-10, product=s5, late_product=s4, late_idem=1.0, refine_product=r8)
    assert sched["late_iters"] > 0.25 * sched["iters"]
    assert abs(sched["energy"] - E) < 0.1 * abs(low["energy"] - E)
