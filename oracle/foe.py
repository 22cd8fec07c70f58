"""Fermi-operator expansion at finite electronic temperature, float64 CPU oracle.

TEST INFRASTRUCTURE ONLY (see the package header).

What the paper states (Sec. "Introduction"): purification applies to
insulators only; finite-temperature methods whose bottleneck is again matrix
multiplication cover metallic systems, and the Fermi Operator Expansion of
Goedecker and Teter (Phys. Rev. B 51, 9455, the paper's citation) is its
representative one, with experiments in its Supplementary Information (not
available here). The Ozaki products therefore apply unchanged.

Reading implemented here (the GPU path implements the same reading):

* the density matrix at electronic temperature kT and chemical potential mu is
  P = f(H) with the Fermi-Dirac occupation f(e) = 1 / (1 + exp((e - mu) / kT)),
  occupations in [0, 1] (the paper's K = 2P);
* H is mapped into [-1, 1] by an enclosure [h_min, h_max] of its spectrum:
  a = (h_max + h_min) / 2, b = (h_max - h_min) / 2 (b = 1 when the enclosure is
  a point, H a multiple of the identity), H_s = (H - a I) / b. The enclosure is
  the caller's when given, else the Gershgorin bounds (which for a dense H can
  be many times wider than the spectrum, and the number of terms needed grows
  with b / kT);
* g(x) = f(a + b x) is replaced by its Chebyshev series truncated after M
  terms. The coefficients come from Gauss-Chebyshev quadrature on N = 2M nodes,
  theta_j = pi (j + 1/2) / N, x_j = cos(theta_j):
  c_k = (2 / N) sum_j g(x_j) cos(k theta_j), k = 0 .. M-1;
* P = (c_0 / 2) I + sum_{k=1}^{M-1} c_k T_k(H_s), with the three-term
  recurrence T_0 = I, T_1 = H_s, T_{k+1} = 2 H_s T_k - T_{k-1}: M - 2 matrix
  products H_s T_k, each one an Ozaki product in the Ozaki modes;
* canonical use (a target n_occ instead of mu): mu solves
  sum_k c_k(mu) tr T_k(H_s) = n_occ, the expansion's own trace, found by 100
  bisection halvings of [h_min - 40 kT, h_max + 40 kT] (the trace is below
  n_occ at the lower end and above it at the upper end). The traces come from
  a first pass of the recurrence, P from a second one with the coefficients of
  that mu.

No damping kernel is applied to the coefficients (the cited expansion has none).

Symmetric products: `symmetric_output` forms a product's upper triangle and
mirrors it (the products H_s T_k are symmetric in exact arithmetic).

Parity: pinned. The tests check the coefficients of polynomials (exact
Chebyshev coefficients), the truncated series against the Fermi function on a
grid, the matrix recurrence against a dense eigensolver with the same
polynomial (numpy's Chebyshev evaluation on the eigenvalues) and with the
Fermi function itself, the closed form for a multiple of the identity, the
particle-hole identity P(2 mu I - H) = I - P(H), permutation equivariance,
tr(P) = n_occ in canonical use, and the approach to the zero-temperature
projector as kT falls.
"""

from __future__ import annotations

import numpy as np

from .purify import fp64_product, gershgorin

MU_BRACKET_KT = 40.0  # the bisection bracket reaches this many kT past the spectral enclosure
MU_HALVINGS = 100


def fermi(e, mu: float, kT: float):
    """Fermi-Dirac occupation 1 / (1 + exp((e - mu)/kT)), evaluated without overflow."""
    z = (np.asarray(e, dtype=np.float64) - mu) / kT
    out = np.empty_like(z)
    pos = z > 0
    ez = np.exp(-z[pos])
    out[pos] = ez / (1.0 + ez)
    out[~pos] = 1.0 / (1.0 + np.exp(z[~pos]))
    return out


def nodes(M: int):
    """Gauss-Chebyshev angles theta_j = pi (j + 1/2) / N and points x_j = cos(theta_j), N = 2M."""
    N = 2 * M
    theta = np.pi * (np.arange(N) + 0.5) / N
    return theta, np.cos(theta)


def chebyshev_coefficients(g, M: int) -> np.ndarray:
    """c_k = (2/N) sum_j g(x_j) cos(k theta_j), k = 0 .. M-1, on N = 2M nodes."""
    if M < 2:
        raise ValueError("need at least two terms")
    theta, x = nodes(M)
    gx = np.asarray(g(x), dtype=np.float64)
    N = 2 * M
    return np.array([2.0 / N * np.sum(gx * np.cos(k * theta)) for k in range(M)])


def scaling(H, bounds=None):
    """(a, b, h_min, h_max): the centre and half-width of the spectral enclosure
    (the given bounds, else the Gershgorin bounds of H); b = 1 if it is a point."""
    if bounds is None:
        h_min, h_max, _, _ = gershgorin(H)
    else:
        h_min, h_max = float(bounds[0]), float(bounds[1])
    a = 0.5 * (h_max + h_min)
    b = 0.5 * (h_max - h_min)
    if not b > 0.0:
        b = 1.0
    return a, b, h_min, h_max


def symmetric_output(product):
    """The product with symmetric output: the upper triangle of A B, mirrored.

    H_s T_k is symmetric in exact arithmetic (T_k is a polynomial in H_s); a
    computed product is not quite. Keeping the upper triangle and mirroring it
    keeps every T_k, and P, exactly symmetric. This is the reading the GPU path
    takes for its symmetric products, so parity tests run the recurrence with
    it; the default recurrence forms the products as written.
    """

    def sym(A, B):
        C = product(A, B)
        return np.triu(C) + np.triu(C, 1).T

    return sym


def recurrence(Hs, M: int, product=None, coeffs=None):
    """Run T_0 = I, T_1 = H_s, T_{k+1} = 2 H_s T_k - T_{k-1} up to T_{M-1}.

    Returns (traces, P, n_products): traces[k] = tr T_k, and, when coeffs are
    given, P = (c_0/2) I + sum_{k>=1} c_k T_k (else None).
    """
    product = product or fp64_product
    n = Hs.shape[0]
    I = np.eye(n)
    T_prev, T_cur = I, Hs.copy()
    traces = [float(n), float(np.trace(Hs))]
    P = None
    if coeffs is not None:
        P = 0.5 * coeffs[0] * I + coeffs[1] * Hs
    products = 0
    for k in range(1, M - 1):
        Y = product(Hs, T_cur)
        products += 1
        T_next = 2.0 * Y - T_prev
        traces.append(float(np.trace(T_next)))
        if P is not None:
            P = P + coeffs[k + 1] * T_next
        T_prev, T_cur = T_cur, T_next
    return np.array(traces), P, products


def expansion_trace(traces, a: float, b: float, mu: float, kT: float, M: int) -> float:
    """sum_k c_k(mu) tr T_k, the trace of the expansion at chemical potential mu."""
    c = chebyshev_coefficients(lambda x: fermi(a + b * x, mu, kT), M)
    return 0.5 * c[0] * traces[0] + float(np.dot(c[1:], traces[1:]))


def solve_mu(traces, a: float, b: float, h_min: float, h_max: float, kT: float, M: int, n_occ: float) -> float:
    """mu with expansion_trace(mu) = n_occ, by bisection of the bracket stated in the header."""
    lo = h_min - MU_BRACKET_KT * kT
    hi = h_max + MU_BRACKET_KT * kT
    for _ in range(MU_HALVINGS):
        mid = 0.5 * (lo + hi)
        if expansion_trace(traces, a, b, mid, kT, M) < n_occ:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def foe(H, kT: float, n_terms: int, mu: float | None = None, n_occ: int | None = None, product=None,
        bounds=None):
    """Chebyshev Fermi-operator expansion of H.

    Exactly one of mu (grand-canonical) and n_occ (canonical: mu from the
    expansion's trace) is given. Returns P and a dict with mu, a, b, the
    Gershgorin bounds, the coefficients, the traces of T_k (canonical use), the
    number of matrix products, tr(P) and the energy tr(P H). `bounds` =
    (h_min, h_max) is a spectral enclosure to scale H by instead of the
    Gershgorin bounds.
    """
    H = np.asarray(H, dtype=np.float64)
    if (mu is None) == (n_occ is None):
        raise ValueError("give exactly one of mu and n_occ")
    if not kT > 0.0:
        raise ValueError("kT must be positive")
    M = int(n_terms)
    if M < 2:
        raise ValueError("need at least two terms")
    a, b, h_min, h_max = scaling(H, bounds)
    n = H.shape[0]
    Hs = (H - a * np.eye(n)) / b
    products = 0
    traces = None
    if n_occ is not None:
        traces, _, used = recurrence(Hs, M, product)
        products += used
        mu = solve_mu(traces, a, b, h_min, h_max, kT, M, float(n_occ))
    coeffs = chebyshev_coefficients(lambda x: fermi(a + b * x, mu, kT), M)
    _, P, used = recurrence(Hs, M, product, coeffs)
    products += used
    info = dict(mu=float(mu), a=a, b=b, h_min=h_min, h_max=h_max, coeffs=coeffs, traces=traces,
                products=products, trace=float(np.trace(P)), energy=float(np.sum(P * H)))
    return P, info


def exact_fermi_matrix(H, mu: float, kT: float):
    """Q f(Lambda) Q^T from a dense eigensolver (the definition of P = f(H))."""
    w, Q = np.linalg.eigh(np.asarray(H, dtype=np.float64))
    return (Q * fermi(w, mu, kT)) @ Q.T
