"""SP2 and TRS4 purification, float64 CPU oracle.

TEST INFRASTRUCTURE ONLY (see the package header).

The paper runs TRS4 (trace-resetting fourth-order purification) through NTPoly
(Sec. "Implementation Details"); SP2 is the second-order recursion of the same
family. Neither is printed in the paper; the steps are those of the cited
methods (Niklasson, 2002), written here in their notation with X the iterate:

  initial guess  X_0 = (h_max I - H) / (h_max - h_min), with [h_min, h_max]
                 the Gershgorin bounds of H, so the occupied (lowest)
                 eigenvalues of H map nearest 1;
  SP2 step       X' = X^2 or X' = 2X - X^2, whichever brings the trace closer
                 to n_occ (|tr X^2 - n_occ| <= |2 tr X - tr X^2 - n_occ|:
                 square), one product per step;
  TRS4 step      F = X^2 (4X - 3X^2), G = X^2 (I - X)^2,
                 gamma = (n_occ - tr F) / tr G;
                 gamma > 6: X' = 2X - X^2;  gamma < 0: X' = X^2;
                 else X' = F + gamma G, so tr X' = n_occ (the trace reset).

Readings where the methods leave a choice:
  * traces: tr X^3 = <X, X^2>_F and tr X^4 = ||X^2||_F^2 (X symmetric), so a
    TRS4 step needs the products X^2 and X^2 Z with
    Z = gamma I + (4 - 2 gamma) X + (gamma - 3) X^2 (F + gamma G = X^2 Z);
    and tr G = tr (X - X^2)^2 = ||X^2 - X||_F^2, taken from the idempotency
    (the trace form t2 - 2 t3 + t4 cancels to rounding noise near a projector);
  * stopping, tested in this order on each iterate X_k:
      1. ||X_k^2 - X_k||_F < tol                        -> CONVERGED
      2. k >= 2, the value two steps earlier is below 1
         (the iterate is near a projector, where exact
         steps only lower it) and ||X_k^2 - X_k||_F is
         not below it: the product's rounding floor     -> C_OUT_OF_RANGE
      3. k == max_iter                                  -> NOT_CONVERGED
    The returned X is X_k. (No energy rule: neither recursion is variational.)

Parity: pinned. The tests check the closed-form projector of H = Q diag(e) Q^T,
tr X = n_occ, idempotency, agreement of the matrix loops with their eigenvalue
forms (every iterate is a polynomial in X_0), the TRS4 polynomial identity and
trace reset, and the fixed points 0 and 1 of both maps.
"""

from __future__ import annotations

import numpy as np

from .purify import C_OUT_OF_RANGE, CONVERGED, NOT_CONVERGED, STATUS_NAMES, fp64_product, gershgorin

SP2, TRS4 = "sp2", "trs4"


def initial_guess(H: np.ndarray):
    """X_0 = (h_max I - H) / (h_max - h_min) and the bounds."""
    H = np.asarray(H, dtype=np.float64)
    n = H.shape[0]
    if H.ndim != 2 or H.shape[1] != n:
        raise ValueError("H must be square")
    if not np.all(np.isfinite(H)):
        raise ValueError("non-finite H")
    h_min, h_max, row_min, row_max = gershgorin(H)
    if not h_max > h_min:
        raise ValueError("H is a multiple of the identity")
    X0 = (h_max * np.eye(n) - H) / (h_max - h_min)
    return X0, dict(h_min=h_min, h_max=h_max, row_min=row_min, row_max=row_max)


def sp2_square(t1: float, t2: float, n_occ: int) -> bool:
    """True if the SP2 step squares (X' = X^2), else X' = 2X - X^2."""
    return abs(t2 - n_occ) <= abs(2.0 * t1 - t2 - n_occ)


def trs4_gamma(t3: float, t4: float, idem: float, n_occ: int) -> float:
    """gamma = (n_occ - tr F) / tr G from tr X^3, tr X^4 and ||X^2 - X||_F."""
    trF = 4.0 * t3 - 3.0 * t4
    return (n_occ - trF) / (idem * idem)


def trs4_z(X, X2, gamma: float):
    """Z with F + gamma G = X^2 Z."""
    n = X.shape[0]
    return gamma * np.eye(n) + (4.0 - 2.0 * gamma) * X + (gamma - 3.0) * X2


def purify(H, n_occ: int, method: str = TRS4, tol: float = 1e-10, max_iter: int = 100, product=None,
           record: bool = False, store=None):
    """SP2 or TRS4 purification of H with the stopping rules of the module
    header; `product(A, B)` forms every matrix product (FP64 by default);
    `store(M)` is applied to every matrix kept between products (X_0, each X^2,
    each updated X and the TRS4 factor Z; purify.fp32_store for FP32 storage).
    Returns P (= the stopped iterate), status, iters (updates applied), energy
    = tr(P H), band_energy, idem, trace, the histories (idempotency, trace,
    steps: 'sq' / 'up' for SP2 steps, gamma for TRS4 steps) and, with
    record=True, every iterate."""
    if method not in (SP2, TRS4):
        raise ValueError("method must be 'sp2' or 'trs4'")
    product = fp64_product if product is None else product
    store = (lambda M: M) if store is None else store
    H = np.asarray(H, dtype=np.float64)
    n = H.shape[0]
    if not (0 < n_occ < n):
        raise ValueError("need 0 < n_occ < n")
    X, init = initial_guess(H)
    X = store(X)
    idems, traces, steps = [], [], []
    iterates = [X.copy()] if record else None
    status = NOT_CONVERGED
    k = 0
    while True:
        X2 = store(product(X, X))
        t1 = float(np.trace(X))
        t2 = float(np.trace(X2))
        idem = float(np.linalg.norm(X2 - X))
        idems.append(idem)
        traces.append(t1)
        if idem < tol:
            status = CONVERGED
            break
        if k >= 2 and idems[-3] < 1.0 and idem >= idems[-3]:
            status = C_OUT_OF_RANGE
            break
        if k >= max_iter:
            status = NOT_CONVERGED
            break
        if method == SP2:
            if sp2_square(t1, t2, n_occ):
                X = X2
                steps.append("sq")
            else:
                X = store(2.0 * X - X2)
                steps.append("up")
        else:
            t3 = float(np.sum(X * X2))
            t4 = float(np.sum(X2 * X2))
            gamma = trs4_gamma(t3, t4, idem, n_occ)
            if gamma > 6.0:
                X = store(2.0 * X - X2)
            elif gamma < 0.0:
                X = X2
            else:
                X = store(product(X2, store(trs4_z(X, X2, gamma))))
            steps.append(gamma)
        if record:
            iterates.append(X.copy())
        k += 1
    energy = float(np.sum(X * H))
    out = dict(P=X, status=status, status_name=STATUS_NAMES[status], iters=k, energy=energy,
               band_energy=2.0 * energy, idem=idems[-1], trace=traces[-1], idem_history=idems,
               trace_history=traces, steps=steps, init=init)
    if record:
        out["iterates"] = iterates
    return out


def spectral_purify(x0, n_occ: int, method: str = TRS4, tol: float = 1e-10, max_iter: int = 100):
    """The loop of `purify` acting on the eigenvalues x of X (every iterate is a
    polynomial in X_0, so tr X^k = sum x^k and ||X^2 - X||_F = ||x^2 - x||_2).
    Same decisions and stopping rules in O(n) per step."""
    x = np.asarray(x0, dtype=np.float64).copy()
    idems, steps = [], []
    status = NOT_CONVERGED
    k = 0
    while True:
        x2 = x * x
        t1, t2 = float(np.sum(x)), float(np.sum(x2))
        idem = float(np.linalg.norm(x2 - x))
        idems.append(idem)
        if idem < tol:
            status = CONVERGED
            break
        if k >= 2 and idems[-3] < 1.0 and idem >= idems[-3]:
            status = C_OUT_OF_RANGE
            break
        if k >= max_iter:
            break
        if method == SP2:
            sq = sp2_square(t1, t2, n_occ)
            x = x2 if sq else 2.0 * x - x2
            steps.append("sq" if sq else "up")
        else:
            gamma = trs4_gamma(float(np.sum(x * x2)), float(np.sum(x2 * x2)), idem, n_occ)
            if gamma > 6.0:
                x = 2.0 * x - x2
            elif gamma < 0.0:
                x = x2
            else:
                x = x2 * (gamma + (4.0 - 2.0 * gamma) * x + (gamma - 3.0) * x2)
            steps.append(gamma)
        k += 1
    return dict(x=x, status=status, iters=k, idem_history=idems, steps=steps)
