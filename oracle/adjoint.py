"""Reverse mode through canonical purification, float64 CPU oracle.

TEST INFRASTRUCTURE ONLY (see the package header).

The forward map H -> P is the composition of the initial guess and the
purification updates of `oracle.purify` (canonical purification, cited by the
paper in Sec. "Introduction"; the paper's Supplementary II on gradients is not
part of this method). The reverse sweep below differentiates exactly the steps
the forward executed, with the iteration count and the branch of each step
frozen, and keeps the dependence of each coefficient c_k on P_k.

Step k, with X2 = P^2, X3 = P^3, t_n = tr(P^2 - P^3), t_d = tr(P - P^2),
c = t_n / t_d and P' = alpha(c) P + b2(c) X2 + b3(c) X3. For G = dL/dP' the
matrix gradient with respect to P is

  alpha G + b2 (G P^T + P^T G) + b3 (G X2^T + P^T G P^T + X2^T G)
    + <G, alpha' P + b2' X2 + b3' X3> * [(2 P^T - 3 X2^T) t_d - t_n (I - 2 P^T)] / t_d^2,

with alpha', b2', b3' the derivatives of the branch weights with respect to c.

Initial guess: P_0 = (lambda/n)(mu I - H) + (n_occ/n) I gives the direct term
-(lambda/n) G_0, the mu = tr(H)/n term (lambda/n) tr(G_0) I / n, and the lambda
term <G_0, mu I - H>/n chained through the active branch of the min, into mu
and into the Gershgorin extreme row (H_aa + sum_j |H_aj|, a subgradient with
sign(H_aj) off the diagonal). `bounds_grad=False` treats h_min and h_max as
constants instead.

The gradient returned is the gradient with respect to H as a general matrix;
a symmetric perturbation H + h (E_ij + E_ji) changes L by h (G_ij + G_ji).

Parity: pinned. The tests compare with central finite differences of the FP64
forward and with the closed-form gradient of the spectral projector
(Daleckii-Krein divided differences), which the converged purification must
reproduce.
"""

from __future__ import annotations

import numpy as np

from .purify import fp64_product, pm_weights, purify


def pm_weight_derivatives(c: float):
    """(alpha', b2', b3') = d(alpha, b2, b3)/dc on the branch that c selects."""
    if c >= 0.5:
        return 0.0, -1.0 / c ** 2, 1.0 / c ** 2
    d = (1.0 - c) ** 2
    return -1.0 / d, 2.0 / d, -1.0 / d


def step_adjoint(P, c, G, product=fp64_product):
    """dL/dP_k from G = dL/dP_{k+1} for the step taken with coefficient c."""
    n = P.shape[0]
    I = np.eye(n)
    X2 = product(P, P)
    X3 = product(P, X2)
    t1 = float(np.trace(P))
    t2 = float(np.trace(X2))
    t3 = float(np.trace(X3))
    t_n = t2 - t3
    t_d = t1 - t2
    alpha, b2, b3, _ = pm_weights(c)
    da, db2, db3 = pm_weight_derivatives(c)
    Pt = P.T
    X2t = X2.T
    grad = alpha * G
    grad = grad + b2 * (product(G, Pt) + product(Pt, G))
    grad = grad + b3 * (product(G, X2t) + product(product(Pt, G), Pt) + product(X2t, G))
    dL_dc = float(np.sum(G * (da * P + db2 * X2 + db3 * X3)))
    dc_dP = ((2.0 * Pt - 3.0 * X2t) * t_d - t_n * (I - 2.0 * Pt)) / (t_d ** 2)
    return grad + dL_dc * dc_dP


def initial_guess_adjoint(H, n_occ, init, G0, bounds_grad=True):
    """dL/dH from G0 = dL/dP_0 through the initial guess."""
    H = np.asarray(H, dtype=np.float64)
    n = H.shape[0]
    lam, mu = init["lam"], init["mu"]
    h_min, h_max = init["h_min"], init["h_max"]
    dH = -(lam / n) * G0
    dL_dlam = float(np.sum(G0 * (mu * np.eye(n) - H))) / n
    dL_dmu = (lam / n) * float(np.trace(G0))
    dL_dhmax = 0.0
    dL_dhmin = 0.0
    if init["lam_branch"] == 1:
        den = (h_max - mu) ** 2
        dL_dmu += dL_dlam * n_occ / den
        dL_dhmax = -dL_dlam * n_occ / den
    else:
        den = (mu - h_min) ** 2
        dL_dmu += -dL_dlam * (n - n_occ) / den
        dL_dhmin = dL_dlam * (n - n_occ) / den
    dH = dH + (dL_dmu / n) * np.eye(n)
    if bounds_grad:
        a = init["row_max"]
        row = np.sign(H[a]) * dL_dhmax
        row[a] = dL_dhmax
        dH[a] += row
        b = init["row_min"]
        row = -np.sign(H[b]) * dL_dhmin
        row[b] = dL_dhmin
        dH[b] += row
    return dH


def purify_backward(H, n_occ, fwd, G_final, product=fp64_product, bounds_grad=True):
    """dL/dH for L depending on the returned P through G_final = dL/dP.

    `fwd` is the result of `oracle.purify.purify(..., record=True)`; every
    iterate is kept, so nothing is recomputed from checkpoints here.
    """
    G = np.asarray(G_final, dtype=np.float64)
    iters = fwd["iterates"]
    cs = fwd["c_history"]
    for k in range(fwd["iters"] - 1, -1, -1):
        G = step_adjoint(iters[k], cs[k], G, product=product)
    return initial_guess_adjoint(H, n_occ, fwd["init"], G, bounds_grad=bounds_grad)


def grad_trace_loss(H, n_occ, W, tol=1e-10, max_iter=100, product=None, bounds_grad=True):
    """(L, dL/dH) for L = tr(P W), with the forward run by the oracle."""
    fwd = purify(H, n_occ, tol=tol, max_iter=max_iter, product=product, record=True)
    W = np.asarray(W, dtype=np.float64)
    L = float(np.sum(fwd["P"] * W.T))
    prod = fp64_product if product is None else product
    G = purify_backward(H, n_occ, fwd, W.T, product=prod, bounds_grad=bounds_grad)
    return L, G, fwd
