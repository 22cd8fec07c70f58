"""Synthetic orthogonal Hamiltonians with an exactly known spectrum.

The paper's Hamiltonians (BigDFT, PySCF and NTChem runs on molecules and
clusters, Sec. "Implementation Details" and "Numerical Experiments") are not
available, so every workload here is synthetic: H = Q diag(e) Q^T with Q a
Haar-random orthogonal matrix (QR of a seeded N(0,1) matrix, column signs fixed
by sign(diag R)) and e drawn uniformly from an occupied and a virtual interval
separated by a gap. The occupied eigenvalues come first, so the exact density
matrix is the projector onto the first n_occ columns of Q.

Nothing here computes a purification step, a split or a product of the method;
this module only draws and assembles inputs.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Workload table. Seeds are 1000 + index; spectra are given as
# (occupied interval, virtual interval).
CONFIGS = {
    0: dict(n=256, n_occ=64, occ=(-2.0, -0.1), virt=(0.1, 2.0), seed=1000, decay=None),
    1: dict(n=2048, n_occ=512, occ=(-2.0, -0.025), virt=(0.025, 2.0), seed=1001, decay=64.0),
    2: dict(n=8192, n_occ=2048, occ=(-1.5, -0.01), virt=(0.01, 1.5), seed=1002, decay=None),
    # config 3 is a batch: see batch_sizes(); each member uses the config-0 spectrum.
    3: dict(batch=64, n_lo=128, n_hi=1536, step=32, occ=(-2.0, -0.1), virt=(0.1, 2.0), seed=1003),
    4: dict(n=1024, n_occ=256, occ=(-2.0, -0.05), virt=(0.05, 2.0), seed=1004, decay=None),
}


@dataclass
class Hamiltonian:
    """A test Hamiltonian and the eigenpairs it was assembled from."""

    H: object  # np.ndarray (host) or torch.Tensor (device), float64, n x n
    e: np.ndarray  # eigenvalues, occupied block first (host, float64)
    Q: object  # eigenvectors as columns, same container type as H
    n_occ: int
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.e.shape[0])


def spectrum(n: int, n_occ: int, occ, virt, rng: np.random.Generator) -> np.ndarray:
    """n_occ values uniform in `occ`, then n - n_occ values uniform in `virt`."""
    lo_o, hi_o = occ
    lo_v, hi_v = virt
    e_occ = rng.uniform(lo_o, hi_o, size=n_occ)
    e_vir = rng.uniform(lo_v, hi_v, size=n - n_occ)
    return np.concatenate([e_occ, e_vir]).astype(np.float64)


def random_orthogonal(n: int, rng: np.random.Generator, device=None):
    """Haar-random orthogonal matrix from QR of a seeded N(0,1) matrix.

    The Gaussian is always drawn on the host with `rng`, so the draw is the same
    everywhere; with `device` set the QR runs through torch on that device (used
    for n in the thousands, where a host QR takes minutes).
    """
    G = rng.standard_normal((n, n))
    if device is None:
        Q, R = np.linalg.qr(G)
        sgn = np.sign(np.diag(R))
        sgn[sgn == 0] = 1.0
        return Q * sgn[None, :]
    import torch

    Gt = torch.from_numpy(G).to(device=device, dtype=torch.float64)
    Q, R = torch.linalg.qr(Gt)
    sgn = torch.sign(torch.diagonal(R))
    sgn[sgn == 0] = 1.0
    return Q * sgn[None, :]


def _assemble(Q, e):
    """H = Q diag(e) Q^T, symmetrised as (H + H^T)/2."""
    if isinstance(Q, np.ndarray):
        H = (Q * e[None, :]) @ Q.T
        return 0.5 * (H + H.T)
    import torch

    et = torch.from_numpy(e).to(device=Q.device, dtype=Q.dtype)
    H = (Q * et[None, :]) @ Q.T
    return 0.5 * (H + H.T)


def make_hamiltonian(n: int, n_occ: int, occ=(-2.0, -0.1), virt=(0.1, 2.0), seed: int = 0,
                     decay: float | None = None, device=None) -> Hamiltonian:
    """Seeded H = Q diag(e) Q^T with a gapped spectrum.

    With `decay` set, the LCAO-like variant is built: H0 = Q diag(e) Q^T is
    damped elementwise by exp(-|i-j|/decay), symmetrised, and re-orthogonalised
    by taking the eigenvectors V of the damped matrix and setting
    H = V diag(sort(e)) V^T, which keeps the drawn spectrum exactly while giving
    H the decaying structure of a localised basis.
    """
    rng = np.random.default_rng(seed)
    e = spectrum(n, n_occ, occ, virt, rng)
    Q = random_orthogonal(n, rng, device=device)
    meta = dict(n=n, n_occ=n_occ, occ=tuple(occ), virt=tuple(virt), seed=seed, decay=decay)
    if decay is None:
        return Hamiltonian(_assemble(Q, e), e, Q, n_occ, meta)
    H0 = _assemble(Q, e)
    idx = np.arange(n)
    D = np.exp(-np.abs(idx[:, None] - idx[None, :]) / float(decay))
    if isinstance(H0, np.ndarray):
        H1 = H0 * D
        H1 = 0.5 * (H1 + H1.T)
        _, V = np.linalg.eigh(H1)
    else:
        import torch

        Dt = torch.from_numpy(D).to(device=H0.device, dtype=H0.dtype)
        H1 = H0 * Dt
        H1 = 0.5 * (H1 + H1.T)
        _, V = torch.linalg.eigh(H1)
    e_sorted = np.sort(e)
    return Hamiltonian(_assemble(V, e_sorted), e_sorted, V, n_occ, meta)


def config_hamiltonian(index: int, device=None) -> Hamiltonian:
    """The single-matrix workload of table entry `index` (0, 1, 2 or 4)."""
    c = CONFIGS[index]
    if "batch" in c:
        raise ValueError("config 3 is a batch; use batch_sizes() and make_hamiltonian()")
    return make_hamiltonian(c["n"], c["n_occ"], c["occ"], c["virt"], c["seed"], c["decay"], device=device)


def batch_sizes(batch: int | None = None, seed: int | None = None, lo: int | None = None,
                hi: int | None = None, step: int | None = None):
    """Seeded matrix sizes for the batched workload: n = step * U{lo/step .. hi/step}.

    Returns a list of (n, n_occ = n/4, member seed).
    """
    c = CONFIGS[3]
    batch = c["batch"] if batch is None else batch
    seed = c["seed"] if seed is None else seed
    lo = c["n_lo"] if lo is None else lo
    hi = c["n_hi"] if hi is None else hi
    step = c["step"] if step is None else step
    rng = np.random.default_rng(seed)
    mult = rng.integers(lo // step, hi // step + 1, size=batch)
    out = []
    for b, m in enumerate(mult):
        n = int(m) * step
        out.append((n, n // 4, seed * 1000 + b))
    return out


def symmetric_gaussian(n: int, seed: int) -> np.ndarray:
    """W = (G + G^T)/2 with G seeded N(0,1): the weight of the loss tr(P W)."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n))
    return 0.5 * (G + G.T)
