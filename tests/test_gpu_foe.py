"""Chebyshev Fermi-operator expansion on the GPU (dm_foe) against the oracle
(oracle/foe.py).

The GPU forms each product's upper triangle and mirrors it; the oracle run with
`symmetric_output` products takes the same reading. Every recurrence term T_k
is then the same on both sides (the Ozaki products are bit-exact, and
2 Y - T_{k-1} rounds once on both), and P differs only through the rounding of
the coefficients (cosine and exponential evaluations, about 1e-13 summed over
k <= 200) and of the accumulation: 1e-12 is the bound. FP64 products differ in
summation order as well (1e-12 on these sizes). Also: canonical use (mu from
n_occ), the Gershgorin enclosure, the degenerate H = h I, the particle-hole
identity, non-finite input, and sampled rows at n = 8192 against the exact
f(H) from the known eigenpairs."""

from functools import partial

import numpy as np
import pytest
import torch

from oracle import foe as fo
from oracle import ozaki as oz
from synth import config_hamiltonian, make_hamiltonian

pytestmark = pytest.mark.gpu

BOUNDS = (-2.0, 2.0)


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _metallic(n, seed):
    return make_hamiltonian(n, n // 3, occ=(-2.0, 0.0), virt=(0.0, 2.0), seed=seed)


def _series_values(e, rinfo):
    """p(x_i) on the scaled eigenvalues, p the oracle's truncated series."""
    c = np.array(rinfo["coeffs"], dtype=np.float64)
    c[0] *= 0.5
    return np.polynomial.chebyshev.chebval((np.asarray(e) - rinfo["a"]) / rinfo["b"], c)


def _oz(mode, s, sym=True):
    prod = partial(oz.ozaki_gemm, s=s, beta=oz.BETA[mode], rounding=oz.ROUNDING[mode])
    return fo.symmetric_output(prod) if sym else prod


@pytest.mark.parametrize("n", [256, 333])
def test_fp64_matches_oracle(dmp, n):
    h = _metallic(n, seed=n)
    ref, rinfo = fo.foe(h.H, 0.1, 80, mu=0.1, bounds=BOUNDS)
    P, info = dmp.foe(_dev(h.H), 0.1, 80, mu=0.1, bounds=BOUNDS, mode="fp64")
    P = P.cpu().numpy()
    assert info["status"] == dmp.OK and info["products"] == 78 and info["n_terms"] == 80
    assert np.max(np.abs(P - ref)) <= 1e-12
    assert np.array_equal(P, P.T)
    assert info["mu"] == 0.1 and (info["e_min"], info["e_max"]) == BOUNDS
    assert abs(info["trace"] - rinfo["trace"]) <= 1e-10
    assert abs(info["energy"] - rinfo["energy"]) <= 1e-10
    assert abs(info["tail"] - (abs(rinfo["coeffs"][-2]) + abs(rinfo["coeffs"][-1]))) <= 1e-14
    # and f(H) itself, to the series' error on the spectrum: P - f(H) =
    # Q (p - f)(Lambda) Q^T, so no entry exceeds max_i |p(x_i) - f(e_i)|
    series = np.max(np.abs(_series_values(h.e, rinfo) - fo.fermi(h.e, 0.1, 0.1)))
    assert np.max(np.abs(P - fo.exact_fermi_matrix(h.H, 0.1, 0.1))) <= series + 1e-12


@pytest.mark.parametrize("mode,s", [("int8", 5), ("int8", 7), ("bf16", 5), ("e4m3", 8)])
@pytest.mark.parametrize("n", [256, 333])
def test_ozaki_modes_match_oracle(dmp, mode, s, n):
    h = _metallic(n, seed=n + s)
    ref, rinfo = fo.foe(h.H, 0.1, 80, mu=0.0, bounds=BOUNDS, product=_oz(mode, s))
    P, info = dmp.foe(_dev(h.H), 0.1, 80, mu=0.0, bounds=BOUNDS, mode=mode, slices=s)
    P = P.cpu().numpy()
    assert info["status"] == dmp.OK and info["slices_used"] == s
    assert np.max(np.abs(P - ref)) <= 1e-12
    assert np.array_equal(P, P.T)
    assert abs(info["energy"] - rinfo["energy"]) <= 1e-10
    # the Ozaki error itself: the distance from the FP64 expansion is the oracle's
    ref64, _ = fo.foe(h.H, 0.1, 80, mu=0.0, bounds=BOUNDS)
    assert np.max(np.abs(P - ref64)) <= np.max(np.abs(ref - ref64)) + 1e-12


@pytest.mark.parametrize("mode,s", [("fp64", 0), ("int8", 7)])
def test_canonical_mu_from_n_occ(dmp, mode, s):
    h = make_hamiltonian(300, 75, occ=(-2.0, -0.3), virt=(0.3, 2.0), seed=301)
    prod = None if mode == "fp64" else _oz(mode, s)
    ref, rinfo = fo.foe(h.H, 0.05, 200, n_occ=75, bounds=BOUNDS, product=prod)
    P, info = dmp.foe(_dev(h.H), 0.05, 200, n_occ=75, bounds=BOUNDS, mode=mode, slices=max(s, 1))
    P = P.cpu().numpy()
    assert info["status"] == dmp.OK and info["products"] == 2 * 198
    assert abs(info["trace"] - 75) <= 1e-8
    assert abs(info["mu"] - rinfo["mu"]) <= 1e-9
    assert -0.3 < info["mu"] < 0.3
    assert np.max(np.abs(P - ref)) <= 1e-11


def test_gershgorin_enclosure(dmp):
    """Without a given enclosure both sides scale by their Gershgorin bounds,
    which may differ in the last bits (other summation orders): the terms then
    agree to the Ozaki error of s = 7, not bit for bit."""
    h = _metallic(200, seed=9)
    ref, rinfo = fo.foe(h.H, 0.2, 120, mu=-0.2, product=_oz("int8", 7))
    P, info = dmp.foe(_dev(h.H), 0.2, 120, mu=-0.2, mode="int8", slices=7)
    assert abs(info["e_min"] - rinfo["h_min"]) <= 1e-12 and abs(info["e_max"] - rinfo["h_max"]) <= 1e-12
    assert np.max(np.abs(P.cpu().numpy() - ref)) <= 1e-9


@pytest.mark.parametrize("mode", ["fp64", "int8"])
def test_multiple_of_identity(dmp, mode):
    """H = h I: the enclosure is a point (b = 1), H_s = 0, P = p(0) I."""
    H = 0.3 * np.eye(64)
    ref, _ = fo.foe(H, 0.2, 60, mu=0.1)
    P, info = dmp.foe(_dev(H), 0.2, 60, mu=0.1, mode=mode, slices=5)
    P = P.cpu().numpy()
    assert info["status"] == dmp.OK and info["e_min"] == info["e_max"] == 0.3
    assert np.max(np.abs(P - ref)) <= 1e-13
    assert abs(P[0, 0] - fo.fermi(np.array([0.3]), 0.1, 0.2)[0]) <= 1e-10


def test_particle_hole_identity(dmp):
    """f(2 mu - e) = 1 - f(e): the GPU expansion of 2 mu I - H is I - P(H)."""
    h = _metallic(256, seed=12)
    mu = 0.05
    P1, _ = dmp.foe(_dev(h.H), 0.1, 100, mu=mu, mode="fp64")
    P2, _ = dmp.foe(_dev(2 * mu * np.eye(256) - h.H), 0.1, 100, mu=mu, mode="fp64")
    assert np.max(np.abs(P2.cpu().numpy() - (np.eye(256) - P1.cpu().numpy()))) <= 1e-11


def test_errors(dmp):
    h = _metallic(128, seed=13)
    H = h.H.copy()
    H[3, 90] = np.nan
    with pytest.raises(dmp.DmpError) as e:
        dmp.foe(_dev(H), 0.1, 40, mu=0.0, mode="int8", slices=5)
    assert e.value.code == dmp.ERR_NONFINITE
    with pytest.raises(dmp.DmpError) as e:
        dmp.foe(_dev(h.H), -0.1, 40, mu=0.0)
    assert e.value.code == dmp.ERR_INVALID_ARG
    with pytest.raises(dmp.DmpError) as e:
        dmp.foe(_dev(h.H), 0.1, 40, n_occ=128)  # n_occ must be below n
    assert e.value.code == dmp.ERR_INVALID_ARG
    # two terms: no product at all, P = c_0/2 I + c_1 H_s
    P, info = dmp.foe(_dev(h.H), 0.1, 2, mu=0.0, bounds=BOUNDS, mode="int8", slices=5)
    ref, _ = fo.foe(h.H, 0.1, 2, mu=0.0, bounds=BOUNDS)
    assert info["products"] == 0 and np.max(np.abs(P.cpu().numpy() - ref)) <= 1e-14


def test_full_size_sampled_rows(dmp):
    """n = 8192 (the purification benchmark's Hamiltonian, spectrum in
    [-1.5, 1.5]) with the benchmark's expansion: sampled rows of P against the
    exact f(H) = Q f(Lambda) Q^T from the known eigenpairs, the trace against
    sum_i f(e_i), and exact symmetry."""
    h = config_hamiltonian(2, device="cuda")
    kT, M, mu = 0.05, 200, 0.0
    P, info = dmp.foe(h.H, kT, M, mu=mu, bounds=(-1.5, 1.5), mode="int8", slices=6)
    assert info["status"] == dmp.OK
    fe = torch.from_numpy(fo.fermi(h.e, mu, kT)).cuda()
    rows = torch.from_numpy(np.random.default_rng(5).choice(h.n, 64, replace=False)).cuda()
    exact = (h.Q[rows] * fe[None, :]) @ h.Q.T
    err = float((P[rows] - exact).abs().max())
    # the series error on this spectrum is about 3e-11 and the oracle's Ozaki
    # error of the same expansion (s = 6) 2e-11 at n = 1024; with the error
    # growing at most in proportion to n, 1e-7 leaves a wide margin
    assert err <= 1e-7, err
    # the trace adds n such errors at most
    assert abs(info["trace"] - float(fe.sum())) <= 1e-5
    assert bool((P[rows][:, rows] == P[rows][:, rows].T).all())


# ---- the Paterson-Stockmeyer scheme (scheme="ps")
# Baby and giant steps carry no coefficients, so they are the same on both
# sides as in the recurrence. The Clenshaw terms B_m are combinations whose
# weights and roundings differ in the last bit, and a product of such a term
# can then truncate one digit differently. With one-ulp noise on every weight
# and element, the oracle moved by at most 1.3 % of its own Ozaki error on
# these cases; the bound below is a quarter of that error (plus 1e-12).


def _ps_tol(ref, ref64):
    return 1e-12 + 0.25 * float(np.max(np.abs(ref - ref64)))


@pytest.mark.parametrize("mode,s", [("int8", 5), ("int8", 7), ("bf16", 5), ("e4m3", 8)])
@pytest.mark.parametrize("n", [256, 333])
def test_ps_modes_match_oracle(dmp, mode, s, n):
    h = _metallic(n, seed=n + s)
    ref64, _ = fo.foe(h.H, 0.1, 80, mu=0.0, bounds=BOUNDS)
    ref, rinfo = fo.foe(h.H, 0.1, 80, mu=0.0, bounds=BOUNDS, product=_oz(mode, s), scheme="ps")
    P, info = dmp.foe(_dev(h.H), 0.1, 80, mu=0.0, bounds=BOUNDS, mode=mode, slices=s, scheme="ps")
    P = P.cpu().numpy()
    assert info["status"] == dmp.OK and info["products"] == rinfo["products"] == 8 + 8
    assert np.max(np.abs(P - ref)) <= _ps_tol(ref, ref64)
    assert np.array_equal(P, P.T)


@pytest.mark.parametrize("M", [2, 3, 5, 17, 80])
def test_ps_fp64_matches_oracle_and_recurrence(dmp, M):
    h = _metallic(333, seed=M)
    ref, rinfo = fo.foe(h.H, 0.1, M, mu=0.1, bounds=BOUNDS, scheme="ps")
    P, info = dmp.foe(_dev(h.H), 0.1, M, mu=0.1, bounds=BOUNDS, mode="fp64", scheme="ps")
    Pr, _ = dmp.foe(_dev(h.H), 0.1, M, mu=0.1, bounds=BOUNDS, mode="fp64")
    P, Pr = P.cpu().numpy(), Pr.cpu().numpy()
    assert info["products"] == rinfo["products"]
    assert np.max(np.abs(P - ref)) <= 1e-12
    assert np.max(np.abs(P - Pr)) <= 1e-12
    assert np.array_equal(P, P.T)


@pytest.mark.parametrize("mode,s", [("fp64", 0), ("int8", 7), ("int8", 5)])
def test_ps_canonical(dmp, mode, s):
    """mu from the traces of the giant steps: 39 products at M = 200 against
    the recurrence's 396."""
    h = make_hamiltonian(300, 75, occ=(-2.0, -0.3), virt=(0.3, 2.0), seed=301)
    prod = None if mode == "fp64" else _oz(mode, s)
    ref, rinfo = fo.foe(h.H, 0.05, 200, n_occ=75, bounds=BOUNDS, product=prod, scheme="ps")
    ref64, _ = fo.foe(h.H, 0.05, 200, n_occ=75, bounds=BOUNDS, scheme="ps")
    P, info = dmp.foe(_dev(h.H), 0.05, 200, n_occ=75, bounds=BOUNDS, mode=mode, slices=max(s, 1), scheme="ps")
    P = P.cpu().numpy()
    assert info["status"] == dmp.OK and info["products"] == rinfo["products"] == 39
    # P comes from the Clenshaw sum, the trace mu was solved on from the giant
    # steps: the two agree to the products' error (about 1e-9 at s = 5)
    assert abs(info["trace"] - 75) <= 1e-7
    assert abs(info["mu"] - rinfo["mu"]) <= 1e-9
    assert np.max(np.abs(P - ref)) <= 1e-11 + 0.25 * float(np.max(np.abs(ref - ref64)))


def test_ps_multiple_of_identity(dmp):
    """P = p(0) I. The two sides' coefficients differ by about 3e-14 summed
    over k (cosine and exponential roundings); the folding moves each into up
    to r = 8 block weights, so p(0) may differ by some 1e-13 (1.0e-13 seen)."""
    H = 0.3 * np.eye(64)
    ref, _ = fo.foe(H, 0.2, 60, mu=0.1, scheme="ps")
    P, info = dmp.foe(_dev(H), 0.2, 60, mu=0.1, mode="int8", slices=5, scheme="ps")
    assert info["status"] == dmp.OK
    assert np.max(np.abs(P.cpu().numpy() - ref)) <= 1e-12


def test_ps_full_size_sampled_rows(dmp):
    """The benchmark's expansion (n = 8192, kT = 0.05, M = 200, mu from n_occ,
    Ozaki-INT8 s = 6) by the Paterson-Stockmeyer scheme: sampled rows against
    the exact f(H) at the returned mu, the trace against n_occ, 39 products."""
    h = config_hamiltonian(2, device="cuda")
    kT, M = 0.05, 200
    P, info = dmp.foe(h.H, kT, M, n_occ=h.n_occ, bounds=(-1.5, 1.5), mode="int8", slices=6, scheme="ps")
    assert info["status"] == dmp.OK and info["products"] == 39
    fe = torch.from_numpy(fo.fermi(h.e, info["mu"], kT)).cuda()
    rows = torch.from_numpy(np.random.default_rng(6).choice(h.n, 64, replace=False)).cuda()
    exact = (h.Q[rows] * fe[None, :]) @ h.Q.T
    err = float((P[rows] - exact).abs().max())
    assert err <= 1e-7, err
    assert abs(info["trace"] - h.n_occ) <= 1e-6
    assert abs(info["trace"] - float(fe.sum())) <= 1e-5
