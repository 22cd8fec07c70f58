"""Pins for the reverse-mode oracle.

Each piece is compared with central finite differences of the forward map it
differentiates (one canonical step with its coefficient recomputed, the initial
guess with its Gershgorin bounds, and the whole purification), and the full
gradient is compared with the closed-form derivative of the spectral projector
(Daleckii-Krein divided differences), which the converged purification must
reproduce.
"""

import numpy as np
import pytest

from oracle import adjoint as ad
from oracle import purify as pu
from synth import make_hamiltonian, symmetric_gaussian


def _step_map(P):
    X2 = P @ P
    X3 = X2 @ P
    c = pu.pm_coefficient(np.trace(P), np.trace(X2), np.trace(X3))
    return pu.pm_update(P, X2, X3, c), c


def _random_density(n, lo, hi, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (Q * rng.uniform(lo, hi, size=n)) @ Q.T


@pytest.mark.parametrize("lo,hi", [(0.05, 0.45), (0.55, 0.95)])
def test_step_adjoint_matches_fd(lo, hi):
    """General (unsymmetric) perturbations of P, coefficient recomputed: checks
    every product-rule term and the dc/dP term on both branches."""
    n = 9
    P = _random_density(n, lo, hi, seed=int(lo * 100))
    rng = np.random.default_rng(3)
    G = rng.standard_normal((n, n))
    _, c = _step_map(P)
    grad = ad.step_adjoint(P, c, G)
    h = 1e-6
    for (i, j) in [(0, 0), (1, 4), (4, 1), (8, 3), (5, 5)]:
        E = np.zeros((n, n))
        E[i, j] = h
        fp, cp = _step_map(P + E)
        fm, cm = _step_map(P - E)
        assert (cp >= 0.5) == (c >= 0.5) == (cm >= 0.5)
        fd = (np.sum(G * fp) - np.sum(G * fm)) / (2 * h)
        assert fd == pytest.approx(grad[i, j], rel=1e-6, abs=1e-8)


def test_step_adjoint_without_c_term_fails_fd():
    """Planted mistake: freezing c (dropping dc/dP) disagrees with FD."""
    n = 9
    P = _random_density(n, 0.05, 0.45, seed=21)
    G = np.random.default_rng(4).standard_normal((n, n))
    _, c = _step_map(P)
    alpha, b2, b3, _ = pu.pm_weights(c)
    frozen = alpha * G + b2 * (G @ P.T + P.T @ G) + b3 * (G @ (P @ P).T + P.T @ G @ P.T + (P @ P).T @ G)
    h = 1e-6
    E = np.zeros((n, n))
    E[2, 2] = h
    fd = (np.sum(G * _step_map(P + E)[0]) - np.sum(G * _step_map(P - E)[0])) / (2 * h)
    assert abs(fd - frozen[2, 2]) > 1e-4 * max(1.0, abs(fd))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_initial_guess_adjoint_matches_fd(seed):
    """<G0, P0(H)> is piecewise linear in H: FD with unsymmetric perturbations
    must reproduce the direct, mu, lambda and Gershgorin-row terms."""
    h = make_hamiltonian(12, 4, seed=40 + seed)
    H = h.H
    G0 = np.random.default_rng(seed).standard_normal((12, 12))
    _, info = pu.initial_guess(H, 4)
    grad = ad.initial_guess_adjoint(H, 4, info, G0)
    a, b = info["row_max"], info["row_min"]
    step = 1e-7
    for (i, j) in [(0, 0), (3, 7), (a, a), (a, (a + 1) % 12), (b, (b + 5) % 12), (b, b)]:
        E = np.zeros((12, 12))
        E[i, j] = step
        fp = np.sum(G0 * pu.initial_guess(H + E, 4)[0])
        fm = np.sum(G0 * pu.initial_guess(H - E, 4)[0])
        assert (fp - fm) / (2 * step) == pytest.approx(grad[i, j], rel=1e-6, abs=1e-9)


def _loss(H, n_occ, W, tol=1e-13):
    r = pu.purify(H, n_occ, tol=tol, max_iter=200)
    return float(np.sum(r["P"] * W))


def _daleckii_krein(Q, e, n_occ, W):
    """dL/dH for L = tr(P W), P the projector onto the n_occ lowest eigenvectors."""
    occ = np.zeros(len(e), dtype=bool)
    occ[np.argsort(e)[:n_occ]] = True
    diff = e[:, None] - e[None, :]
    mixed = occ[:, None] != occ[None, :]
    Gam = np.zeros_like(diff)
    Gam[mixed] = (occ[:, None].astype(float) - occ[None, :].astype(float))[mixed] / diff[mixed]
    return Q @ (Gam * (Q.T @ W @ Q)) @ Q.T


@pytest.fixture(scope="module")
def small_case():
    h = make_hamiltonian(40, 10, occ=(-2.0, -0.25), virt=(0.25, 2.0), seed=77)
    W = symmetric_gaussian(40, seed=78)
    L, G, fwd = ad.grad_trace_loss(h.H, 10, W, tol=1e-12)
    return h, W, L, G, fwd


def test_full_gradient_matches_fd(small_case):
    h, W, _, G, _ = small_case
    rng = np.random.default_rng(79)
    step = 1e-6
    idx = [(int(i), int(j)) for i, j in rng.integers(0, 40, size=(10, 2))] + [(3, 3)]
    for (i, j) in idx:
        E = np.zeros((40, 40))
        E[i, j] += step
        E[j, i] += step if i != j else 0.0
        fd = (_loss(h.H + E, 10, W) - _loss(h.H - E, 10, W)) / (2 * step)
        an = G[i, j] + G[j, i] if i != j else G[i, i]
        assert fd == pytest.approx(an, rel=1e-6, abs=1e-7), (i, j)


def test_full_gradient_matches_projector_derivative(small_case):
    h, W, _, G, _ = small_case
    dk = _daleckii_krein(h.Q, h.e, 10, W)
    Gs = 0.5 * (G + G.T)
    assert np.max(np.abs(Gs - dk)) <= 1e-8 * np.max(np.abs(dk))


def test_bounds_stop_gradient_agrees_at_convergence(small_case):
    h, W, _, G, fwd = small_case
    G2 = ad.purify_backward(h.H, 10, fwd, W.T, bounds_grad=False)
    assert np.max(np.abs(G - G2)) <= 1e-8 * np.max(np.abs(G))
