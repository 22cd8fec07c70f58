"""Oracle pins for the Chebyshev Fermi-operator expansion (oracle/foe.py).

Pinned against what the mathematics fixes: the Chebyshev coefficients of
polynomials, the Fermi function itself, a dense eigensolver applying the same
polynomial (numpy's Chebyshev evaluation) or the exact Fermi function to the
eigenvalues, the closed form for a multiple of the identity, the particle-hole
identity, permutation equivariance, the trace in canonical use and the
zero-temperature projector."""

from functools import partial

import numpy as np
import pytest
from numpy.polynomial import chebyshev as cheb

from oracle import foe as fo
from oracle import ozaki as oz
from synth import make_hamiltonian

BOUNDS = (-2.0, 2.0)  # every synthetic spectrum below lies in [-2, 2]


def _metallic(n=96, seed=5):
    """A gapless spectrum: the metallic case finite-temperature methods are for."""
    return make_hamiltonian(n, n // 3, occ=(-2.0, 0.0), virt=(0.0, 2.0), seed=seed)


def _series(c):
    """numpy's Chebyshev-series convention: the constant term is c_0 / 2 here."""
    cc = np.array(c, dtype=np.float64)
    cc[0] *= 0.5
    return cc


def _eigen_polynomial(H, info):
    """Q p(Lambda) Q^T with p the truncated series, from a dense eigensolver."""
    w, Q = np.linalg.eigh(H)
    x = (w - info["a"]) / info["b"]
    return (Q * cheb.chebval(x, _series(info["coeffs"]))) @ Q.T


def test_coefficients_of_polynomials():
    """Quadrature on 2M nodes is exact for polynomials of degree < 2M."""
    c = fo.chebyshev_coefficients(lambda x: 4 * x**3 - 3 * x, 6)  # T_3
    assert np.max(np.abs(c - [0, 0, 0, 1, 0, 0])) < 1e-14
    c = fo.chebyshev_coefficients(lambda x: x**2, 5)  # (T_0 + T_2) / 2
    assert np.max(np.abs(c - [1.0, 0, 0.5, 0, 0])) < 1e-14
    c = fo.chebyshev_coefficients(lambda x: np.ones_like(x), 3)
    assert np.max(np.abs(c - [2.0, 0, 0])) < 1e-14


def test_coefficients_match_the_chebyshev_integrals():
    """The quadrature coefficients equal the exact Chebyshev coefficients
    c_k = (2/pi) int_0^pi g(cos t) cos(k t) dt, integrated by mpmath at 30
    digits, to rounding: on 2M nodes the aliasing error is of the size of the
    coefficients beyond 3M, far below 1e-15 here."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    a, b, mu, kT, M = 0.1, 1.3, 0.2, 0.13, 40

    def integrand(k):
        return lambda t: mp.cos(k * t) / (1 + mp.exp((a + b * mp.cos(t) - mu) / kT))

    exact = np.array([float(2 / mp.pi * mp.quad(integrand(k), [0, mp.pi / 2, mp.pi])) for k in range(M)])
    c = fo.chebyshev_coefficients(lambda x: fo.fermi(a + b * x, mu, kT), M)
    assert np.max(np.abs(c - exact)) < 1e-14
    assert abs(c[-1]) > 1e-7  # the last coefficients still matter: the comparison is not vacuous


def test_fermi_function():
    e = np.array([-1e4, -1.0, 0.0, 0.25, 1.0, 1e4])
    f = fo.fermi(e, 0.25, 0.5)
    assert f[0] == 1.0 and f[-1] == 0.0  # no overflow at either end
    assert f[3] == 0.5
    assert abs(f[1] - 1 / (1 + np.exp(-2.5))) < 1e-16
    assert abs(f[4] - 1 / (1 + np.exp(1.5))) < 1e-16
    # f(mu + t) + f(mu - t) = 1
    t = np.linspace(-3, 3, 61)
    assert np.max(np.abs(fo.fermi(0.25 + t, 0.25, 0.5) + fo.fermi(0.25 - t, 0.25, 0.5) - 1)) < 1e-15


def test_series_converges_to_fermi():
    """Truncated series against the Fermi function on a grid: the error falls
    geometrically with M (the function is analytic in a strip of half-width
    pi kT / b around [-1, 1])."""
    x = np.linspace(-1, 1, 2001)
    errs = []
    for M in (32, 64, 128, 256):
        c = fo.chebyshev_coefficients(lambda t: fo.fermi(t, 0.1, 0.05), M)
        errs.append(np.max(np.abs(cheb.chebval(x, _series(c)) - fo.fermi(x, 0.1, 0.05))))
    assert all(b < a / 10 for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-12


def test_recurrence_matches_eigensolver_polynomial():
    """The matrix recurrence is the series applied to H_s: it matches the same
    polynomial applied to the eigenvalues by a dense eigensolver."""
    h = _metallic()
    P, info = fo.foe(h.H, 0.1, 60, mu=0.0)  # Gershgorin bounds
    assert np.max(np.abs(P - _eigen_polynomial(h.H, info))) < 1e-13
    P, info = fo.foe(h.H, 0.1, 120, mu=0.3, bounds=BOUNDS)
    assert np.max(np.abs(P - _eigen_polynomial(h.H, info))) < 1e-13
    assert info["products"] == 118


def test_matches_exact_fermi_matrix():
    """With enough terms P = f(H) to the series' own error on the spectrum."""
    h = _metallic()
    P, info = fo.foe(h.H, 0.1, 160, mu=0.2, bounds=BOUNDS)
    w = np.linalg.eigvalsh(h.H)
    scal = np.max(np.abs(cheb.chebval((w - info["a"]) / info["b"], _series(info["coeffs"])) - fo.fermi(w, 0.2, 0.1)))
    assert scal < 1e-10
    assert np.max(np.abs(P - fo.exact_fermi_matrix(h.H, 0.2, 0.1))) < 1e-10


def test_planted_recurrence_errors_fail_the_pin():
    """A wrong sign in the recurrence, or c_0 not halved, fails the eigensolver pin."""
    h = _metallic()
    P, info = fo.foe(h.H, 0.1, 60, mu=0.0, bounds=BOUNDS)
    ref = _eigen_polynomial(h.H, info)
    Hs = (h.H - info["a"] * np.eye(h.n)) / info["b"]
    c = info["coeffs"]
    T_prev, T_cur = np.eye(h.n), Hs.copy()
    bad = 0.5 * c[0] * np.eye(h.n) + c[1] * Hs
    for k in range(1, 59):
        T_next = 2.0 * Hs @ T_cur + T_prev  # planted: + instead of -
        bad = bad + c[k + 1] * T_next
        T_prev, T_cur = T_cur, T_next
    assert np.max(np.abs(bad - ref)) > 1e-3
    assert np.max(np.abs((P + 0.5 * c[0] * np.eye(h.n)) - ref)) > 1e-3  # c_0 counted in full
    assert np.max(np.abs(P - ref)) < 1e-13


def test_multiple_of_identity():
    """H = h I: the enclosure is a point, H_s = 0, and P = p(0) I with p the
    series of f(h + x), which is f(h) to the series' error."""
    n, hval, mu, kT = 16, 0.3, 0.1, 0.2
    H = hval * np.eye(n)
    P, info = fo.foe(H, kT, 60, mu=mu)
    assert info["b"] == 1.0 and info["a"] == hval
    p0 = cheb.chebval(0.0, _series(info["coeffs"]))
    assert np.max(np.abs(P - p0 * np.eye(n))) < 1e-15
    assert abs(p0 - fo.fermi(np.array([hval]), mu, kT)[0]) < 1e-12


def test_two_by_two_closed_form():
    """H = [[d, t], [t, d]] has eigenvalues d +- t on (1, +-1)/sqrt(2), so
    f(H) = (f(d+t) + f(d-t))/2 I + (f(d+t) - f(d-t))/2 [[0, 1], [1, 0]];
    at mu = d this is I/2 - tanh(t / 2kT)/2 [[0, 1], [1, 0]]."""
    d, t, kT = 0.3, 0.7, 0.15
    H = np.array([[d, t], [t, d]])
    X = np.array([[0.0, 1.0], [1.0, 0.0]])
    for mu in (d, -0.2, 1.1):
        fp, fm = fo.fermi(np.array([d + t, d - t]), mu, kT)
        closed = 0.5 * (fp + fm) * np.eye(2) + 0.5 * (fp - fm) * X
        for scheme in ("recurrence", "ps"):
            P, _ = fo.foe(H, kT, 120, mu=mu, scheme=scheme)  # Gershgorin bounds: exactly d -+ t
            assert np.max(np.abs(P - closed)) < 1e-12, (mu, scheme)
    P, _ = fo.foe(H, kT, 120, mu=d)
    assert np.max(np.abs(P - (0.5 * np.eye(2) - 0.5 * np.tanh(t / (2 * kT)) * X))) < 1e-12


def test_particle_hole_identity():
    """f(2 mu - e) = 1 - f(e): P(2 mu I - H) = I - P(H), with the Gershgorin
    enclosure mirrored as well."""
    h = _metallic(seed=6)
    mu = 0.05
    P1, _ = fo.foe(h.H, 0.1, 80, mu=mu)
    P2, _ = fo.foe(2 * mu * np.eye(h.n) - h.H, 0.1, 80, mu=mu)
    assert np.max(np.abs(P2 - (np.eye(h.n) - P1))) < 1e-12


def test_permutation_equivariance():
    h = _metallic(seed=7)
    perm = np.random.default_rng(3).permutation(h.n)
    P, _ = fo.foe(h.H, 0.1, 80, mu=-0.1)
    Pp, _ = fo.foe(h.H[np.ix_(perm, perm)], 0.1, 80, mu=-0.1)
    assert np.max(np.abs(Pp - P[np.ix_(perm, perm)])) < 1e-12


def test_canonical_trace_and_mu():
    """With n_occ given, mu makes tr(P) = n_occ; for a gapped spectrum at low
    temperature it lies inside the gap."""
    h = make_hamiltonian(96, 30, occ=(-2.0, -0.3), virt=(0.3, 2.0), seed=71)
    P, info = fo.foe(h.H, 0.05, 200, n_occ=30, bounds=BOUNDS)
    assert abs(np.trace(P) - 30) < 1e-9
    assert abs(info["trace"] - 30) < 1e-9
    assert -0.3 < info["mu"] < 0.3
    assert info["products"] == 2 * 198
    # the expansion's trace at mu is the trace the first pass predicted
    assert abs(fo.expansion_trace(info["traces"], info["a"], info["b"], info["mu"], 0.05, 200) - 30) < 1e-9


def test_zero_temperature_limit():
    """As kT falls (with enough terms) P approaches the projector onto the
    n_occ lowest eigenvectors."""
    h = make_hamiltonian(96, 30, occ=(-2.0, -0.3), virt=(0.3, 2.0), seed=71)
    V = h.Q[:, :30]
    proj = V @ V.T
    errs = []
    for kT, M in ((0.1, 200), (0.05, 300), (0.025, 600)):
        P, _ = fo.foe(h.H, kT, M, n_occ=30, bounds=BOUNDS)
        errs.append(np.max(np.abs(P - proj)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-4


@pytest.mark.parametrize("mode", ["int8", "bf16", "e4m3"])
def test_ozaki_products_converge_to_fp64(mode):
    """The recurrence with Ozaki products approaches the FP64 one as the slice
    count grows."""
    h = _metallic(n=64, seed=8)
    beta, rounding = oz.BETA[mode], oz.ROUNDING[mode]
    ref, _ = fo.foe(h.H, 0.1, 60, mu=0.0, bounds=BOUNDS)
    errs = []
    for s in (3, 5, 7):
        prod = partial(oz.ozaki_gemm, s=s, beta=beta, rounding=rounding)
        P, _ = fo.foe(h.H, 0.1, 60, mu=0.0, bounds=BOUNDS, product=prod)
        errs.append(np.max(np.abs(P - ref)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-8


def test_symmetric_output_product():
    """The mirrored product keeps the upper triangle of A B exactly, and the
    recurrence built on it returns an exactly symmetric P that differs from the
    plain one at the Ozaki error level only."""
    rng = np.random.default_rng(4)
    A, B = rng.standard_normal((40, 40)), rng.standard_normal((40, 40))
    C = fo.symmetric_output(fo.fp64_product)(A, B)
    iu = np.triu_indices(40)
    assert np.array_equal(C[iu], (A @ B)[iu]) and np.array_equal(C, C.T)
    h = _metallic(n=64, seed=9)
    prod = partial(oz.ozaki_gemm, s=5, beta=7)
    ref64, _ = fo.foe(h.H, 0.1, 60, mu=0.0, bounds=BOUNDS)
    P, _ = fo.foe(h.H, 0.1, 60, mu=0.0, bounds=BOUNDS, product=prod)
    Ps, _ = fo.foe(h.H, 0.1, 60, mu=0.0, bounds=BOUNDS, product=fo.symmetric_output(prod))
    assert np.array_equal(Ps, Ps.T)
    d = np.max(np.abs(P - ref64))
    assert 0 < d < 1e-8
    assert np.max(np.abs(Ps - ref64)) < 4 * d


def test_ps_fold_reproduces_the_series_on_scalars():
    """sum_m T_m(T_q(x)) B_m(x) with the folded weights equals the series
    sum_k c_k' T_k(x) (numpy's Chebyshev evaluation) for every block layout."""
    x = np.linspace(-1, 1, 501)
    rng = np.random.default_rng(11)
    for M in (2, 3, 7, 16, 17, 50, 199):
        c = rng.standard_normal(M)
        q, r = fo.ps_blocks(M)
        assert q * q >= M > (q - 1) * (q - 1) and (r - 1) * q < M <= r * q
        w = fo.ps_fold(c, q)
        y = cheb.chebval(x, np.eye(q + 1)[q])  # T_q(x)
        Tj = np.array([cheb.chebval(x, np.eye(q)[j]) for j in range(q)])
        val = sum(cheb.chebval(y, np.eye(r)[m]) * (w[m] @ Tj) for m in range(r))
        assert np.max(np.abs(val - cheb.chebval(x, _series(c)))) < 1e-12 * np.sum(np.abs(c))
    # planted: the fold without the -c carried into block m - 1 misses the series
    M, c = 50, rng.standard_normal(50)
    q, r = fo.ps_blocks(M)
    a = np.concatenate([[0.5 * c[0]], c[1:], np.zeros(r * q - M)])
    w_bad = np.array([[a[q * m] if j == 0 or m == 0 else 2.0 * a[q * m + j] for j in range(q)] for m in range(r)])
    w_bad[0] = a[:q]
    y = cheb.chebval(x, np.eye(q + 1)[q])
    Tj = np.array([cheb.chebval(x, np.eye(q)[j]) for j in range(q)])
    bad = sum(cheb.chebval(y, np.eye(r)[m]) * (w_bad[m] @ Tj) for m in range(r))
    assert np.max(np.abs(bad - cheb.chebval(x, _series(c)))) > 1e-3


@pytest.mark.parametrize("M", [2, 3, 5, 17, 60, 200])
def test_ps_matches_the_recurrence(M):
    """Both schemes evaluate the same truncated series: in FP64 they agree to
    rounding, the scheme uses (q - 1) + (r - 1) products (q - 2 for r = 1),
    and it matches the eigensolver polynomial."""
    h = _metallic()
    P, info = fo.foe(h.H, 0.1, M, mu=0.05, bounds=BOUNDS)
    Pp, ip = fo.foe(h.H, 0.1, M, mu=0.05, bounds=BOUNDS, scheme="ps")
    assert np.max(np.abs(Pp - P)) < 1e-14
    q, r = fo.ps_blocks(M)
    assert ip["products"] == ((q - 1) + (r - 1) if r > 1 else q - 2)
    assert np.max(np.abs(Pp - _eigen_polynomial(h.H, ip))) < 1e-13


def test_ps_canonical():
    """Traces from the giant steps and Frobenius products equal the
    recurrence's traces, so mu and P agree as well; 2 (q - 1) + 2 r - 3 products."""
    h = make_hamiltonian(96, 30, occ=(-2.0, -0.3), virt=(0.3, 2.0), seed=71)
    P, info = fo.foe(h.H, 0.05, 200, n_occ=30, bounds=BOUNDS)
    Pp, ip = fo.foe(h.H, 0.05, 200, n_occ=30, bounds=BOUNDS, scheme="ps")
    assert np.max(np.abs(ip["traces"] - info["traces"])) < 1e-12
    assert abs(ip["mu"] - info["mu"]) < 1e-12
    assert np.max(np.abs(Pp - P)) < 1e-13 and abs(np.trace(Pp) - 30) < 1e-9
    q, r = fo.ps_blocks(200)
    assert ip["products"] == (q - 1) + (r - 2) + (r - 1) == 39


@pytest.mark.parametrize("mode", ["int8", "e4m3"])
def test_ps_with_ozaki_products(mode):
    """With Ozaki products the scheme's error stays at the recurrence's level."""
    h = _metallic(n=64, seed=8)
    beta, rounding = oz.BETA[mode], oz.ROUNDING[mode]
    ref, _ = fo.foe(h.H, 0.1, 120, mu=0.0, bounds=BOUNDS)
    for s in (5, 7):
        prod = fo.symmetric_output(partial(oz.ozaki_gemm, s=s, beta=beta, rounding=rounding))
        P, _ = fo.foe(h.H, 0.1, 120, mu=0.0, bounds=BOUNDS, product=prod)
        Pp, _ = fo.foe(h.H, 0.1, 120, mu=0.0, bounds=BOUNDS, product=prod, scheme="ps")
        assert np.max(np.abs(Pp - ref)) <= 3 * np.max(np.abs(P - ref)) + 1e-14


def test_argument_errors():
    H = np.eye(4)
    with pytest.raises(ValueError):
        fo.foe(H, 0.1, 10)
    with pytest.raises(ValueError):
        fo.foe(H, 0.1, 10, mu=0.0, n_occ=2)
    with pytest.raises(ValueError):
        fo.foe(H, 0.0, 10, mu=0.0)
    with pytest.raises(ValueError):
        fo.foe(H, 0.1, 1, mu=0.0)
    with pytest.raises(ValueError):
        fo.foe(H, 0.1, 10, mu=0.0, scheme="horner")
