"""GPU reverse mode (dm_purify_backward, PurifyFunction) against the oracle's
gradient, central finite differences of the GPU forward, and the closed-form
derivative of the spectral projector (Daleckii-Krein).

dLdH from the library is the gradient for symmetric H (the symmetric part of
the general-matrix gradient the oracle returns).
"""

from functools import partial

import numpy as np
import pytest
import torch

from oracle import adjoint as ad
from oracle import ozaki as oz
from synth import config_hamiltonian, make_hamiltonian, symmetric_gaussian

pytestmark = pytest.mark.gpu


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _dk(Q, e, n_occ, W):
    occ = np.zeros(len(e), dtype=bool)
    occ[np.argsort(e)[:n_occ]] = True
    diff = e[:, None] - e[None, :]
    mixed = occ[:, None] != occ[None, :]
    Gam = np.zeros_like(diff)
    Gam[mixed] = (occ[:, None].astype(float) - occ[None, :].astype(float))[mixed] / diff[mixed]
    return Q @ (Gam * (Q.T @ W @ Q)) @ Q.T


def _gpu_grad(dmp, H, n_occ, W, **kw):
    Hd = _dev(H).requires_grad_(True)
    P = dmp.purify_autograd(Hd, n_occ, **kw)
    L = (P * _dev(W)).sum()
    L.backward()
    return float(L.item()), Hd.grad.cpu().numpy()


@pytest.mark.parametrize("mode,s", [("fp64", 0), ("int8", 7), ("e4m3", 10)])
def test_matches_oracle_gradient(dmp, mode, s):
    h = make_hamiltonian(160, 40, occ=(-2.0, -0.25), virt=(0.25, 2.0), seed=51)
    W = symmetric_gaussian(160, seed=52)
    if mode == "fp64":
        prod = None
    elif mode == "int8":
        prod = partial(oz.ozaki_gemm, s=s, beta=7)
    else:
        prod = partial(oz.ozaki_gemm, s=s, beta=5, rounding="nearest")
    _, G_or, _ = ad.grad_trace_loss(h.H, 40, W, tol=1e-10, product=prod)
    G_or = 0.5 * (G_or + G_or.T)
    _, G = _gpu_grad(dmp, h.H, 40, W, mode=mode, slices=s or 7, executor="tc", tol=1e-10, checkpoint_every=4)
    scale = np.max(np.abs(G_or))
    assert np.max(np.abs(G - G_or)) <= 1e-7 * scale
    assert np.array_equal(G, G.T)
    dk = _dk(h.Q, h.e, 40, W)
    assert np.max(np.abs(G - dk)) <= 1e-6 * np.max(np.abs(dk))


def test_checkpoint_spacing_does_not_change_the_gradient(dmp):
    """Recomputed iterates are bit-identical to the forward's, so the gradient
    does not depend on how often the tape keeps a checkpoint."""
    h = make_hamiltonian(130, 30, occ=(-2.0, -0.25), virt=(0.25, 2.0), seed=53)
    W = symmetric_gaussian(130, seed=54)
    grads = [_gpu_grad(dmp, h.H, 30, W, mode="int8", slices=7, executor="tc", checkpoint_every=k)[1]
             for k in (1, 3, 8)]
    assert np.array_equal(grads[0], grads[1]) and np.array_equal(grads[0], grads[2])


def test_bounds_constant_agrees_at_convergence(dmp):
    h = make_hamiltonian(96, 24, occ=(-2.0, -0.25), virt=(0.25, 2.0), seed=55)
    W = symmetric_gaussian(96, seed=56)
    _, G1 = _gpu_grad(dmp, h.H, 24, W, mode="fp64")
    _, G2 = _gpu_grad(dmp, h.H, 24, W, mode="fp64", bounds_constant=True)
    assert np.max(np.abs(G1 - G2)) <= 1e-8 * np.max(np.abs(G1))


@pytest.mark.parametrize("mode", ["fp64", "int8"])
def test_config4_against_fd_and_oracle(dmp, mode):
    """n = 1024, n_occ = 256, gap 0.1, L = tr(P W), checkpoints every 8 steps:
    the gradient matches the closed form, the FP64 oracle gradient, and central
    differences (step 1e-6, FP64 forward) on 32 seeded entries: to 1e-6 of the
    gradient's scale (max |dL/dH|) on every entry, and to 1e-6 of the entry
    itself on the entries with |dL/dH_ij| >= 0.25."""
    h = config_hamiltonian(4)
    W = symmetric_gaussian(1024, seed=1004 + 7)
    n, n_occ = 1024, 256
    _, G = _gpu_grad(dmp, h.H, n_occ, W, mode=mode, slices=7, executor="tc", checkpoint_every=8)
    scale = np.max(np.abs(G))
    dk = _dk(h.Q, h.e, n_occ, W)
    assert np.max(np.abs(G - dk)) <= 1e-6 * np.max(np.abs(dk))
    if mode == "fp64":
        _, G_or, _ = ad.grad_trace_loss(h.H, n_occ, W, tol=1e-10)  # FP64 oracle
        G_or = 0.5 * (G_or + G_or.T)
        assert np.max(np.abs(G - G_or)) <= 1e-7 * np.max(np.abs(G_or))
    Hd = _dev(h.H)
    Wd = _dev(W)
    ws = dmp.workspace(dmp.purify_workspace_bytes(n, dmp.make_opts("fp64")))

    def loss(Hp):
        P, _ = dmp.purify(Hp, n_occ, mode="fp64", ws=ws)
        return float((P * Wd).sum().item())

    rng = np.random.default_rng(1004)
    idx = rng.integers(0, n, size=(32, 2))
    idx[0] = (5, 5)
    step = 1e-6
    errs = []
    for i, j in idx:
        E = torch.zeros_like(Hd)
        E[i, j] += step
        if i != j:
            E[j, i] += step
        fd = (loss(Hd + E) - loss(Hd - E)) / (2 * step)
        an = 2 * G[i, j] if i != j else G[i, i]
        errs.append(abs(fd - an))
    # the difference quotient carries the FP64 forward's rounding noise
    # (about 1e-13 in L) divided by 2e-6, hence the scale-relative measure
    assert max(errs) <= 1e-6 * scale, (max(errs), scale)
    # per entry: where |dL/dH| is large enough that this noise (at most a few
    # 1e-7 absolute) is below 1e-6 of the entry, the entry itself matches to 1e-6
    # relative (|G| >= 0.25 here, about an eighth of max |G| and half the sampled entries)
    rel = [(e / abs(a), abs(a)) for e, a in zip(errs, [2 * G[i, j] if i != j else G[i, i] for i, j in idx])]
    big = [r for r, a in rel if a >= 0.25]
    assert len(big) >= 8, rel
    assert max(big) <= 1e-6, sorted(rel, reverse=True)[:5]


def test_int8_forward_gradient_matches_the_oracle_at_mid_size(dmp):
    """The config-4 spectrum (gap 0.1) at n = 384: the gradient of an
    Ozaki-INT8 forward (s = 7) against the oracle's reverse sweep through the
    same Ozaki products, and against the closed form."""
    n, n_occ = 384, 96
    h = make_hamiltonian(n, n_occ, occ=(-2.0, -0.05), virt=(0.05, 2.0), seed=57)
    W = symmetric_gaussian(n, seed=58)
    _, G_or, _ = ad.grad_trace_loss(h.H, n_occ, W, tol=1e-10, product=partial(oz.ozaki_gemm, s=7, beta=7))
    G_or = 0.5 * (G_or + G_or.T)
    _, G = _gpu_grad(dmp, h.H, n_occ, W, mode="int8", slices=7, executor="tc", tol=1e-10, checkpoint_every=8)
    scale = np.max(np.abs(G_or))
    assert np.max(np.abs(G - G_or)) <= 1e-7 * scale
    dk = _dk(h.Q, h.e, n_occ, W)
    assert np.max(np.abs(G - dk)) <= 1e-6 * np.max(np.abs(dk))
