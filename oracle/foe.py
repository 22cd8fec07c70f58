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

Second scheme, `scheme="ps"`: the same truncated series evaluated with about
2 sqrt(M) products instead of M - 2, after Liang, Saravanan, Shao, Baer, Bell
and Head-Gordon (J. Chem. Phys. 119, 4117 (2003), "Improved Fermi operator
expansion methods"), a Paterson-Stockmeyer evaluation in the Chebyshev basis.
With q = ceil(sqrt(M)) and y = T_q(H_s):
* baby steps T_0 .. T_q by the recurrence (q - 1 products, all kept);
* T_{qm + j} = 2 T_m(y) T_j - T_{qm - j} (the product rule
  2 T_a T_b = T_{a+b} + T_{|a-b|} and T_{qm} = T_m(T_q)) rewrites the series
  as sum_{m<r} T_m(y) B_m with B_m = sum_{j<q} w_{m,j} T_j, r = ceil(M/q): the
  blocks are folded from the top, each term c_{qm+j} (m >= 1, j >= 1) giving
  2 c to w_{m,j} and -c to the coefficient of T_{qm-j} one block lower;
* Clenshaw's recurrence in y, b_m = B_m + 2 y b_{m+1} - b_{m+2},
  P = B_0 + y b_1 - b_2 (r - 1 products);
* canonical use: the traces come from the giant steps T_{qm} = T_m(y)
  (r - 2 more products) and tr T_{qm+j} = 2 <T_{qm}, T_j>_F - tr T_{qm-j}
  (T's symmetric, so tr(AB) is the Frobenius product).
In exact arithmetic both schemes give the same P.

Symmetric products: `symmetric_output` forms a product's upper triangle and
mirrors it (the products H_s T_k are symmetric in exact arithmetic).

Parity: pinned. The tests check the coefficients of polynomials (exact
Chebyshev coefficients) and of the Fermi function (the exact Chebyshev
integrals, by mpmath at 30 digits), the truncated series against the Fermi
function on a grid, the closed-form Fermi matrix of a 2 x 2 H, the matrix
recurrence against a dense eigensolver with the same polynomial (numpy's
Chebyshev evaluation on the eigenvalues) and with the Fermi function itself,
the closed form for a multiple of the identity, the particle-hole identity P(2
mu I - H) = I - P(H), permutation equivariance, tr(P) = n_occ in canonical
use, and the approach to the zero-temperature projector as kT falls. For the
Paterson-Stockmeyer scheme: the folded weights reproduce the series on scalars
(numpy's Chebyshev evaluation, every block layout), P agrees with the
recurrence and the eigensolver to rounding, the traces of the giant steps
equal the recurrence's, and the product counts.
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


def ps_blocks(M: int):
    """(q, r): the baby-step count q = ceil(sqrt(M)) and the block count r = ceil(M / q)."""
    q = 1
    while q * q < M:
        q += 1
    return q, -(-M // q)


def ps_fold(coeffs, q: int):
    """The weights w[m][j] of B_m = sum_{j<q} w[m][j] T_j with P = sum_m T_m(y) B_m.

    a_k starts as the series coefficient of T_k (c_0 / 2 for k = 0). Blocks are
    folded from the top: T_{qm} = T_m(y) T_0, and for j >= 1
    T_{qm+j} = 2 T_m(y) T_j - T_{qm-j}, so a_{qm+j} adds 2 a_{qm+j} to w[m][j]
    and -a_{qm+j} to a_{qm-j}, a term of block m - 1 (not yet folded).
    """
    M = len(coeffs)
    r = -(-M // q)
    a = np.zeros(r * q)
    a[:M] = coeffs
    a[0] = 0.5 * coeffs[0]
    w = np.zeros((r, q))
    for m in range(r - 1, 0, -1):
        w[m, 0] = a[q * m]
        for j in range(1, q):
            d = a[q * m + j]
            w[m, j] = 2.0 * d
            a[q * m - j] -= d
    w[0, :] = a[:q]
    return w


def _combine(wrow, T):
    acc = np.zeros_like(T[0])
    for j, wj in enumerate(wrow):
        acc = acc + wj * T[j]
    return acc


def ps_baby_steps(Hs, q: int, product):
    """T_0 .. T_q by the recurrence: q - 1 products."""
    T = [np.eye(Hs.shape[0]), Hs.copy()]
    for j in range(1, q):
        T.append(2.0 * product(Hs, T[j]) - T[j - 1])
    return T


def ps_traces(T, q: int, M: int, product):
    """tr T_k, k < M, from the baby steps and the giant steps T_{qm} = T_m(y):
    tr T_{qm+j} = 2 <T_{qm}, T_j>_F - tr T_{qm-j}. Returns (traces, products)."""
    traces = np.zeros(M)
    for k in range(min(q, M)):
        traces[k] = np.trace(T[k])
    y = T[q]
    G_prev, G = T[0], y
    products = 0
    m = 1
    while q * m < M:
        if m >= 2:
            G_next = 2.0 * product(y, G) - G_prev
            products += 1
            G_prev, G = G, G_next
        traces[q * m] = np.trace(G)
        for j in range(1, q):
            if q * m + j < M:
                traces[q * m + j] = 2.0 * float(np.sum(G * T[j])) - traces[q * m - j]
        m += 1
    return traces, products


def ps_evaluate(T, w, product):
    """Clenshaw in y = T_q: b_m = B_m + 2 y b_{m+1} - b_{m+2}, P = B_0 + y b_1 - b_2.
    Returns (P, products)."""
    r = w.shape[0]
    q = w.shape[1]
    if r == 1:
        return _combine(w[0], T), 0
    y = T[q]
    products = 0
    b1 = _combine(w[r - 1], T)
    b2 = np.zeros_like(b1)
    for m in range(r - 2, 0, -1):
        Y = product(y, b1)
        products += 1
        bm = (_combine(w[m], T) + 2.0 * Y) - b2
        b2, b1 = b1, bm
    Y = product(y, b1)
    products += 1
    return (_combine(w[0], T) + Y) - b2, products


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
        bounds=None, scheme: str = "recurrence"):
    """Chebyshev Fermi-operator expansion of H.

    Exactly one of mu (grand-canonical) and n_occ (canonical: mu from the
    expansion's trace) is given. Returns P and a dict with mu, a, b, the
    Gershgorin bounds, the coefficients, the traces of T_k (canonical use), the
    number of matrix products, tr(P) and the energy tr(P H). `bounds` =
    (h_min, h_max) is a spectral enclosure to scale H by instead of the
    Gershgorin bounds. `scheme` is "recurrence" (M - 2 products per pass) or
    "ps" (the Paterson-Stockmeyer evaluation of the header).
    """
    H = np.asarray(H, dtype=np.float64)
    if scheme not in ("recurrence", "ps"):
        raise ValueError("scheme must be 'recurrence' or 'ps'")
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
    if scheme == "ps":
        prod = product or fp64_product
        q, r = ps_blocks(M)
        T = ps_baby_steps(Hs, q if r > 1 else q - 1, prod)
        products += len(T) - 2
        if n_occ is not None:
            traces, used = ps_traces(T, q, M, prod)
            products += used
            mu = solve_mu(traces, a, b, h_min, h_max, kT, M, float(n_occ))
        coeffs = chebyshev_coefficients(lambda x: fermi(a + b * x, mu, kT), M)
        P, used = ps_evaluate(T, ps_fold(coeffs, q), prod)
        products += used
        info = dict(mu=float(mu), a=a, b=b, h_min=h_min, h_max=h_max, coeffs=coeffs, traces=traces,
                    products=products, trace=float(np.trace(P)), energy=float(np.sum(P * H)), q=q, r=r)
        return P, info
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
