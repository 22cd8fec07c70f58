"""Canonical density-matrix purification, float64 CPU oracle.

TEST INFRASTRUCTURE ONLY (see the package header).

Problem statement (Sec. "Density Matrix Purification"): for an orthogonalised
Hamiltonian H (n x n, symmetric) and n_occ occupied orbitals, find the density
matrix P, the projector onto the n_occ lowest eigenvectors of H; K = 2P is the
spin-restricted density matrix. Purification builds P from matrix products
only: McWeeny's recurrence P_{k+1} = 3 P_k^2 - 2 P_k^3 is the one the paper
prints, and the canonical method of Palser and Manolopoulos (the paper's
reference for purification) is the one implemented here. Its formulas are not
printed in the paper; they are taken from the cited method:

  initial guess   mu = tr(H)/n,
                  lambda = min(n_occ/(h_max - mu), (n - n_occ)/(mu - h_min)),
                  P_0 = (lambda/n)(mu I - H) + (n_occ/n) I,
                  with [h_min, h_max] the Gershgorin bounds of H;
  coefficient     c = tr(P^2 - P^3) / tr(P - P^2);
  update          c >= 1/2:  P' = ((1 + c) P^2 - P^3) / c
                  c <  1/2:  P' = ((1 - 2c) P + (1 + c) P^2 - P^3) / (1 - c).

With c = 1/2 both branches equal McWeeny's step. The update keeps tr(P)
fixed, so tr(P_k) = n_occ throughout.

Stopping rules (readings; the paper runs TRS4 with an energy-change test, Sec.
"Implementation Details"):
  1. ||P_k^2 - P_k||_F < tol                          -> CONVERGED, return P_k
  2. band energy rose on each of the last two steps by
     less than 1e-2 in absolute value (the paper's halt rule)  -> STALLED
  3. optional: |change of band energy| < energy_tol     -> CONVERGED
     (the paper's own criterion; off unless energy_tol > 0)
  4. k == max_iter (the paper stops at iteration 100)  -> NOT_CONVERGED
  5. tr(P - P^2) <= 0 or c outside [0, 1]: the trace
     difference has sunk into rounding noise          -> C_OUT_OF_RANGE
The rules are tested in this order on each iterate, before the update.

Refinement (Sec. "Precision Requirements Sweep"): after the loop has
stopped, one McWeeny step P' = 3 P^2 - 2 P^3 taken in full precision (the
paper's mixed-precision recommendation when the energy matters). Reading: the
step's two products use the `refine_product` passed in (FP64, or an Ozaki
product with enough slices to reach FP64 accuracy); the returned P, energy and
band energy are those of P', and the unrefined values are kept. The step is
the update above with c = 1/2, but is written here as printed.

Late-slice schedule (an option; Sec. "Precision Requirements Sweep" weighs
adjusting the precision across iterations): the subspace an iterate spans is
disturbed by a product error in proportion to the error over the gap between
its occupied and virtual eigenvalues, a gap that doubles about every three
iterations of the loop, while the refinement step repairs the eigenvalues.
Reading: once an iterate's ||P^2 - P||_F is below a threshold, all later
passes use a second product (fewer slices); the switch is taken after the
update, so it applies from the next pass on, and it is never undone.

FP32 storage (Sec. "Mixed Precision Purification"): the paper finds that the
matrices of purification may be stored in FP32 as long as they are multiplied
with FP64 accumulation, and tests it by rounding every matrix that enters a
product to FP32. Reading: `store` rounds every matrix the loop keeps between
products (P_0, each P^2, each updated P) to the nearest float32; P^3 is used at
once and the refined P is left as computed.

Energies: tr(P H) is reported as `energy`; the paper's band energy
Tr(H K) = 2 tr(P H) is reported as `band_energy` (Sec. "Error Evaluation
Criteria"), as are the RMSD of P and the commutator norm ||H K - K H||_F.

Parity: pinned. The tests check the closed-form projector of H = Q diag(e) Q^T,
tr(P) = n_occ, idempotency, c in [0, 1], trace conservation of every update on
arbitrary spectra, energy monotonicity, the c = 1/2 reduction to McWeeny's
printed step, the Gershgorin enclosure of the spectrum, and agreement with a
dense eigensolver on tiny inputs; with FP32 storage, that every stored matrix
is a float32 value and the projector and energy are reached to FP32
resolution. The exact iteration counts of the Ozaki modes are measured outputs
and are not pinned.
"""

from __future__ import annotations

import numpy as np

CONVERGED, NOT_CONVERGED, STALLED, C_OUT_OF_RANGE = 0, 1, 2, 3
STATUS_NAMES = {CONVERGED: "CONVERGED", NOT_CONVERGED: "NOT_CONVERGED", STALLED: "STALLED",
                C_OUT_OF_RANGE: "C_OUT_OF_RANGE"}

STALL_ABS = 1e-2  # halt threshold on the band energy change (Sec. "Implementation Details")


def fp64_product(A, B):
    return np.asarray(A, dtype=np.float64) @ np.asarray(B, dtype=np.float64)


def gershgorin(H: np.ndarray):
    """Gershgorin enclosure of the spectrum of H.

    Returns (h_min, h_max, row_of_min, row_of_max); the rows are the first
    indices attaining the extremes.
    """
    H = np.asarray(H, dtype=np.float64)
    off = np.abs(H)
    np.fill_diagonal(off, 0.0)
    radius = off.sum(axis=1)
    d = np.diag(H)
    lo = d - radius
    hi = d + radius
    b = int(np.argmin(lo))
    a = int(np.argmax(hi))
    return float(lo[b]), float(hi[a]), b, a


def initial_guess(H: np.ndarray, n_occ: int):
    """P_0 of canonical purification and the scalars it was built from."""
    H = np.asarray(H, dtype=np.float64)
    n = H.shape[0]
    if H.ndim != 2 or H.shape[1] != n:
        raise ValueError("H must be square")
    if not (0 < n_occ < n):
        raise ValueError("need 0 < n_occ < n")
    if not np.all(np.isfinite(H)):
        raise ValueError("non-finite H")
    h_min, h_max, row_min, row_max = gershgorin(H)
    mu = float(np.trace(H)) / n
    if not (h_max > mu and mu > h_min):
        raise ValueError("degenerate spectrum bounds (H is a multiple of the identity)")
    lam1 = n_occ / (h_max - mu)
    lam2 = (n - n_occ) / (mu - h_min)
    branch = 1 if lam1 <= lam2 else 2
    lam = lam1 if branch == 1 else lam2
    P0 = (lam / n) * (mu * np.eye(n) - H) + (n_occ / n) * np.eye(n)
    info = dict(h_min=h_min, h_max=h_max, row_min=row_min, row_max=row_max, mu=mu,
                lam=lam, lam_branch=branch)
    return P0, info


def pm_coefficient(t1: float, t2: float, t3: float) -> float:
    """c = tr(P^2 - P^3) / tr(P - P^2) from t1 = tr P, t2 = tr P^2, t3 = tr P^3."""
    return (t2 - t3) / (t1 - t2)


def pm_weights(c: float):
    """(alpha, b2, b3) with P' = alpha P + b2 P^2 + b3 P^3, and the branch (1: c >= 1/2)."""
    if c >= 0.5:
        return 0.0, (1.0 + c) / c, -1.0 / c, 1
    return (1.0 - 2.0 * c) / (1.0 - c), (1.0 + c) / (1.0 - c), -1.0 / (1.0 - c), 2


def pm_update(P, X2, X3, c):
    """One canonical purification step given P^2, P^3 and c."""
    alpha, b2, b3, _ = pm_weights(c)
    return alpha * P + b2 * X2 + b3 * X3


def fp32_store(M):
    """A matrix as FP32 storage holds it (Sec. "Mixed Precision Purification":
    matrices kept in FP32, products formed with FP64 accumulation): every
    element rounded to the nearest float32 (ties to even), returned as float64."""
    return np.asarray(M, dtype=np.float64).astype(np.float32).astype(np.float64)


def mcweeny_step(P, product=None):
    """One McWeeny step P' = 3 P^2 - 2 P^3 (the equation printed in Sec.
    "Precision Requirements Sweep"), with P^2 = P P and P^3 = P P^2 formed by
    `product` (FP64 by default)."""
    product = fp64_product if product is None else product
    X2 = product(P, P)
    X3 = product(P, X2)
    return 3.0 * X2 - 2.0 * X3


def purify(H, n_occ: int, tol: float = 1e-10, max_iter: int = 100, product=None,
           energy_tol: float = 0.0, record: bool = False, refine_product=None, store=None,
           late_product=None, late_idem: float = 0.0):
    """Canonical purification of H with the stopping rules of the module header.

    `product(A, B)` forms every matrix product (FP64 by default; pass a partial
    of `oracle.ozaki.ozaki_gemm` for an Ozaki mode). Returns a dict with P,
    status, iters (number of updates applied), energy = tr(PH), band_energy,
    idem = ||P^2 - P||_F, trace, the per-iteration histories, the initial-guess
    scalars and, with record=True, every iterate P_0 .. P_iters.

    With `refine_product` set, the stopped iterate gets one McWeeny step whose
    products use it (the refinement of the module header); P, energy and
    band_energy then describe the refined matrix, energy_unrefined the one
    before, and idem stays that of the unrefined iterate.

    `store(M)` is applied to every matrix the loop keeps between products: the
    initial guess, each P^2 and each updated P (fp32_store for FP32 storage;
    X3 is used at once and the refined P is left as computed). With
    record=True the P^2 of every pass are returned as well ("squares").

    With `late_product` set, once an iterate's idempotency ||P^2 - P||_F has
    fallen below `late_idem`, every later pass forms its products with
    `late_product` instead (the late-slice schedule of the module header);
    `late_iters` counts the passes (P^2 products) that did.
    """
    product = fp64_product if product is None else product
    store = (lambda M: M) if store is None else store
    H = np.asarray(H, dtype=np.float64)
    P, init = initial_guess(H, n_occ)
    P = store(P)
    squares = [] if record else None
    late = False
    late_iters = 0
    band = []
    idems = []
    traces = []
    cs = []
    branches = []
    iterates = [P.copy()] if record else None
    status = NOT_CONVERGED
    k = 0
    while True:
        prod_k = late_product if late else product
        late_iters += 1 if late else 0
        X2 = store(prod_k(P, P))
        if record:
            squares.append(X2.copy())
        t1 = float(np.trace(P))
        t2 = float(np.trace(X2))
        idem = float(np.linalg.norm(X2 - P))
        e_band = 2.0 * float(np.sum(P * H))
        band.append(e_band)
        idems.append(idem)
        traces.append(t1)
        if idem < tol:
            status = CONVERGED
            break
        if k >= 2 and band[-1] > band[-2] > band[-3] and abs(band[-1] - band[-2]) < STALL_ABS \
                and abs(band[-2] - band[-3]) < STALL_ABS:
            status = STALLED
            break
        if energy_tol > 0 and k >= 1 and abs(band[-1] - band[-2]) < energy_tol:
            status = CONVERGED
            break
        if k >= max_iter:
            status = NOT_CONVERGED
            break
        X3 = prod_k(P, X2)
        t3 = float(np.trace(X3))
        if not (t1 - t2 > 0):
            status = C_OUT_OF_RANGE
            break
        c = pm_coefficient(t1, t2, t3)
        if not (0.0 <= c <= 1.0):
            status = C_OUT_OF_RANGE
            break
        alpha, b2, b3, br = pm_weights(c)
        P = store(alpha * P + b2 * X2 + b3 * X3)
        cs.append(c)
        branches.append(br)
        if late_product is not None and idem < late_idem:
            late = True
        if record:
            iterates.append(P.copy())
        k += 1
    energy_unrefined = 0.5 * band[-1]
    energy = energy_unrefined
    if refine_product is not None:
        P = mcweeny_step(P, refine_product)
        energy = float(np.sum(P * H))
    out = dict(P=P, status=status, status_name=STATUS_NAMES[status], iters=k,
               energy=energy, band_energy=2.0 * energy, energy_unrefined=energy_unrefined,
               refined=refine_product is not None, idem=idems[-1], trace=traces[-1],
               band_history=band, idem_history=idems, trace_history=traces, c_history=cs,
               branch_history=branches, init=init, late_iters=late_iters)
    if record:
        out["iterates"] = iterates
        out["squares"] = squares
    return out


def spectral_purify(x0, e, tol: float = 1e-10, max_iter: int = 100, energy_tol: float = 0.0):
    """The purification loop of `purify` acting on eigenvalues.

    When H = V diag(e) V^T, P_0 = V diag(x0) V^T with x0 = (lambda/n)(mu - e)
    + n_occ/n, and every iterate is a polynomial in P_0, so all iterates share
    V and each step maps the eigenvalues alone: tr(P^k) = sum x^k,
    ||P^2 - P||_F = ||x^2 - x||_2 and tr(P H) = sum x e. This runs the same
    stopping rules in O(n) per step (exact arithmetic; rounding differs from
    the matrix loop). Returns iters, status, the final x and the histories.
    """
    x = np.asarray(x0, dtype=np.float64).copy()
    e = np.asarray(e, dtype=np.float64)
    band, cs = [], []
    status = NOT_CONVERGED
    k = 0
    while True:
        x2 = x * x
        t1, t2 = float(np.sum(x)), float(np.sum(x2))
        idem = float(np.linalg.norm(x2 - x))
        band.append(2.0 * float(np.sum(x * e)))
        if idem < tol:
            status = CONVERGED
            break
        if k >= 2 and band[-1] > band[-2] > band[-3] and abs(band[-1] - band[-2]) < STALL_ABS \
                and abs(band[-2] - band[-3]) < STALL_ABS:
            status = STALLED
            break
        if energy_tol > 0 and k >= 1 and abs(band[-1] - band[-2]) < energy_tol:
            status = CONVERGED
            break
        if k >= max_iter:
            break
        x3 = x2 * x
        t3 = float(np.sum(x3))
        if not (t1 - t2 > 0):
            status = C_OUT_OF_RANGE
            break
        c = pm_coefficient(t1, t2, t3)
        if not (0.0 <= c <= 1.0):
            status = C_OUT_OF_RANGE
            break
        alpha, b2, b3, _ = pm_weights(c)
        x = alpha * x + b2 * x2 + b3 * x3
        cs.append(c)
        k += 1
    return dict(x=x, iters=k, status=status, band_history=band, c_history=cs)


def initial_eigenvalues(H, n_occ: int, e):
    """Eigenvalues of P_0 for H with eigenvalues e (same order as e)."""
    n = np.asarray(H).shape[0]
    h_min, h_max, _, _ = gershgorin(H)
    mu = float(np.trace(H)) / n
    lam = min(n_occ / (h_max - mu), (n - n_occ) / (mu - h_min))
    return (lam / n) * (mu - np.asarray(e, dtype=np.float64)) + n_occ / n


def error_metrics(P, H, P_ref=None, E_ref=None):
    """Error measures of Sec. "Error Evaluation Criteria", with K = 2P.

    rmsd = ||K - K_ref||_F / n, max_abs = max |P - P_ref|, commutator =
    ||H K - K H||_F, band_energy = Tr(H K), rel_energy = |E - E_ref| / |E_ref|
    with E = tr(P H), idempotency = ||P^2 - P||_F.
    """
    P = np.asarray(P, dtype=np.float64)
    H = np.asarray(H, dtype=np.float64)
    n = P.shape[0]
    K = 2.0 * P
    out = dict(band_energy=float(np.sum(H * K)), energy=float(np.sum(H * P)),
               commutator=float(np.linalg.norm(H @ K - K @ H)),
               idempotency=float(np.linalg.norm(P @ P - P)), trace=float(np.trace(P)))
    if P_ref is not None:
        P_ref = np.asarray(P_ref, dtype=np.float64)
        out["rmsd"] = float(np.linalg.norm(K - 2.0 * P_ref)) / n
        out["max_abs"] = float(np.max(np.abs(P - P_ref)))
    if E_ref is not None:
        out["rel_energy"] = abs(out["energy"] - E_ref) / abs(E_ref)
    return out
