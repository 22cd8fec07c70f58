"""Oracle pins for SP2 and TRS4 purification (oracle/variants.py): the
closed-form projector, the eigenvalue form of both loops, the TRS4 polynomial
identity and trace reset, fixed points, and Ozaki-mode convergence."""

from functools import partial

import numpy as np
import pytest

from oracle import ozaki as oz
from oracle import purify as pu
from oracle import variants as va
from synth import config_hamiltonian, make_hamiltonian

METHODS = [va.SP2, va.TRS4]


def _projector(h):
    V = h.Q[:, : h.n_occ]
    return V @ V.T


@pytest.mark.parametrize("method", METHODS)
def test_config0_projector(method):
    h = config_hamiltonian(0)
    r = va.purify(h.H, h.n_occ, method=method, tol=1e-10)
    assert r["status"] == pu.CONVERGED
    assert np.max(np.abs(r["P"] - _projector(h))) < 1e-10
    assert abs(np.trace(r["P"]) - h.n_occ) < 1e-9
    E_star = float(np.sum(h.e[: h.n_occ]))
    assert abs(r["energy"] - E_star) < 1e-10 * abs(E_star)


@pytest.mark.parametrize("method", METHODS)
def test_matrix_loop_matches_eigenvalue_loop(method):
    """Every iterate is a polynomial in X_0 = (h_max I - H)/(h_max - h_min): the
    eigenvalue loop on x_0 = (h_max - e)/(h_max - h_min) takes the same steps."""
    h = make_hamiltonian(96, 30, occ=(-2.0, -0.3), virt=(0.3, 2.0), seed=71)
    r = va.purify(h.H, 30, method=method, tol=1e-10)
    x0 = (r["init"]["h_max"] - h.e) / (r["init"]["h_max"] - r["init"]["h_min"])
    s = va.spectral_purify(x0, 30, method=method, tol=1e-10)
    # the last step may cross tol one iteration apart (rounding of the two forms)
    assert s["status"] == r["status"] and abs(s["iters"] - r["iters"]) <= 1
    m = min(len(s["steps"]), len(r["steps"]))
    if method == va.SP2:
        assert s["steps"][:m] == r["steps"][:m]
    else:
        # gamma = (n_occ - tr F)/tr G loses its digits once tr G ~ idem^2 is tiny
        early = [k for k, v in enumerate(s["idem_history"][:m]) if v > 1e-3]
        assert np.allclose(np.array(s["steps"])[early], np.array(r["steps"])[early], rtol=1e-8, atol=1e-10)
    got = np.sort(np.linalg.eigvalsh(r["P"]))
    assert np.max(np.abs(got - np.sort(s["x"]))) < 1e-9


def test_trs4_polynomial_identity_and_trace_reset():
    rng = np.random.default_rng(72)
    n, n_occ = 50, 17
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([rng.uniform(0.7, 1.0, n_occ), rng.uniform(0.0, 0.3, n - n_occ)])
    X = (Q * lam) @ Q.T
    X = 0.5 * (X + X.T)
    X2 = X @ X
    X3, X4 = X2 @ X, X2 @ X2
    for gamma in (0.0, 1.3, 3.0, 6.0):
        F_plus = 4 * X3 - 3 * X4 + gamma * (X2 - 2 * X3 + X4)
        assert np.max(np.abs(X2 @ va.trs4_z(X, X2, gamma) - F_plus)) < 1e-12
    gamma = va.trs4_gamma(float(np.sum(X * X2)), float(np.sum(X2 * X2)), float(np.linalg.norm(X2 - X)), n_occ)
    assert 0.0 <= gamma <= 6.0
    Xn = X2 @ va.trs4_z(X, X2, gamma)
    assert abs(np.trace(Xn) - n_occ) < 1e-10 * n_occ
    # tr G = tr X^2 (I - X)^2 = ||X^2 - X||_F^2 for symmetric X
    G = X2 @ (np.eye(n) - X) @ (np.eye(n) - X)
    assert abs(np.trace(G) - np.linalg.norm(X2 - X) ** 2) < 1e-12


def test_fixed_points_of_both_maps():
    for x in (0.0, 1.0):
        assert x * x == x and 2 * x - x * x == x
        for gamma in (0.0, 2.5, 6.0):
            assert x * x * (gamma + (4 - 2 * gamma) * x + (gamma - 3) * x * x) == x


def test_sp2_step_choice_by_hand():
    # tr X = 5, tr X^2 = 3, n_occ = 4: squaring gives trace 3 (off by 1), 2X - X^2 gives 7 (off by 3)
    assert va.sp2_square(5.0, 3.0, 4)
    # tr X = 3, tr X^2 = 2.5, n_occ = 4: squaring 2.5 (off 1.5), 2X - X^2 3.5 (off 0.5)
    assert not va.sp2_square(3.0, 2.5, 4)


@pytest.mark.parametrize("method", METHODS)
def test_ozaki_products_reach_the_projector(method):
    h = make_hamiltonian(160, 40, occ=(-2.0, -0.25), virt=(0.25, 2.0), seed=73)
    r = va.purify(h.H, 40, method=method, tol=1e-10, product=partial(oz.ozaki_gemm, s=7, beta=7))
    assert r["status"] in (pu.CONVERGED, pu.C_OUT_OF_RANGE)
    assert np.max(np.abs(r["P"] - _projector(h))) < 1e-8


@pytest.mark.parametrize("method", METHODS)
def test_variants_agree_with_canonical_purification(method):
    h = make_hamiltonian(120, 33, occ=(-1.5, -0.1), virt=(0.1, 1.5), seed=74)
    a = va.purify(h.H, 33, method=method, tol=1e-10)
    b = pu.purify(h.H, 33, tol=1e-10)
    assert np.max(np.abs(a["P"] - b["P"])) < 1e-9
