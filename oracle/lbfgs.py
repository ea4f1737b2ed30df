"""Projected L-BFGS with backtracking (oracle, FP64).

Follows Sec. 3: x_{k+1} = P(x_k - alpha_k H_k g_k) (Eq. BFGS_iterations) with
the inverse-Hessian approximation built from the last l pairs, applied with
the two-loop recursion (Algorithm 1), the box projection P (Eq.
bound_constraints) and a backtracking line search on alpha.

Readings where the paper is silent or garbled:

* Algorithm 1 is the textbook two-loop recursion (Nocedal & Wright, which the
  paper cites): the first loop uses the current vector (printed as q) and the
  pair's gradient difference phi_j (printed as phi_i); the second loop ADDS
  varkappa_j (lambda_j - beta) (printed with a minus), which is the sign for
  which the result equals H_k of the paper's product formula for H_k.
* H_k^0 = (varkappa^T phi / phi^T phi) I from the newest pair; with no pair
  yet, H^0 = alpha0 / ||g||_inf (a first step of alpha0 in the scaled units).
* Variables are block-scaled, z_b = x_b / sigma_b, before the recursion.
* Components of the direction that point out of the box at a variable that is
  already on a bound are set to zero; if the result is not a descent
  direction, the memory is dropped and d = -H^0 g is used.
* Backtracking: alpha = 1, halved up to ``max_halvings`` times until the
  Armijo condition J(x(alpha)) <= J(x) + c1 g^T (x(alpha) - x) holds with
  x(alpha) = P(x + alpha d).  On failure the memory is dropped and steepest
  descent is tried once; if that fails too, the loop stops.
* A pair is kept only if s^T y > 1e-10 ||s|| ||y||.
* Stop after ``max_iter`` iterations or when (J_prev - J)/J_prev < rtol.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def two_loop(g, pairs, h0):
    """Algorithm 1: returns H g for the pairs [(s_j, y_j)] (oldest first)."""
    q = np.array(g, dtype=np.float64, copy=True)
    lam = []
    for s, y in reversed(pairs):
        rho = 1.0 / float(np.dot(y, s))
        l_ = rho * float(np.dot(s, q))
        q -= l_ * y
        lam.append(l_)
    lam.reverse()
    psi = h0 * q
    for (s, y), l_ in zip(pairs, lam):
        rho = 1.0 / float(np.dot(y, s))
        beta = rho * float(np.dot(y, psi))
        psi += s * (l_ - beta)
    return psi


def hessian_product_form(pairs, h0, n):
    """H_k from the paper's product formula (dense, for small n): V^T...H0...V + sum rho s s^T."""
    Hm = h0 * np.eye(n)
    for s, y in pairs:  # oldest first: H <- V^T H V + rho s s^T
        rho = 1.0 / float(np.dot(y, s))
        V = np.eye(n) - rho * np.outer(y, s)
        Hm = V.T @ Hm @ V + rho * np.outer(s, s)
    return Hm


def project(z, lo, hi):
    """Eq. (bound_constraints): clamp to [lo, hi] componentwise."""
    return np.minimum(np.maximum(z, lo), hi)


@dataclass
class LbfgsResult:
    x: np.ndarray
    J: float
    history: list = field(default_factory=list)   # dicts per iteration
    stopped: str = ""


def projected_lbfgs(fun, fun_grad, x0, lower, upper, scale, mem=20, max_iter=20,
                    alpha0=0.1, c1=1e-4, max_halvings=20, rtol=1e-4, callback=None):
    """Minimise fun over the box [lower, upper] (all arrays of x's shape, flat).

    ``fun(x) -> J`` and ``fun_grad(x) -> (J, g)`` work in the original
    variables; ``scale`` holds sigma_b per component.
    """
    scale = np.asarray(scale, dtype=np.float64)
    lo = np.asarray(lower, dtype=np.float64) / scale
    hi = np.asarray(upper, dtype=np.float64) / scale
    z = project(np.asarray(x0, dtype=np.float64) / scale, lo, hi)
    J, g = fun_grad(z * scale)
    g = g * scale
    pairs = []
    h0_last = None
    hist = []
    stopped = "max_iter"

    def steepest(gv):
        gi = np.max(np.abs(gv))
        return -(alpha0 / gi) * gv if gi > 0 else np.zeros_like(gv)

    def clip_dir(d):
        d = d.copy()
        d[(z <= lo) & (d < 0)] = 0.0
        d[(z >= hi) & (d > 0)] = 0.0
        return d

    for it in range(max_iter):
        if pairs:
            d = -two_loop(g, pairs[-mem:] if mem > 0 else [], h0_last)
        elif h0_last is not None:
            d = -h0_last * g
        else:
            d = steepest(g)
        d = clip_dir(d)
        if float(np.dot(g, d)) >= 0.0:
            pairs.clear()
            d = clip_dir(steepest(g))
        accepted = False
        tried_reset = False
        trials = 0
        while True:
            alpha = 1.0
            for _ in range(max_halvings + 1):
                zt = project(z + alpha * d, lo, hi)
                Jt = fun(zt * scale)
                trials += 1
                if Jt <= J + c1 * float(np.dot(g, zt - z)):
                    accepted = True
                    break
                alpha *= 0.5
            if accepted or tried_reset:
                break
            tried_reset = True
            pairs.clear()
            h0_last = None
            d = clip_dir(steepest(g))
        if not accepted:
            stopped = "line_search"
            hist.append(dict(it=it, J=J, gnorm=float(np.linalg.norm(g)), alpha=0.0, trials=trials))
            break
        Jn, gn = fun_grad(zt * scale)
        gn = gn * scale
        s = zt - z
        yv = gn - g
        sy = float(np.dot(s, yv))
        if sy > 1e-10 * np.linalg.norm(s) * np.linalg.norm(yv):
            pairs.append((s, yv))
            if mem > 0 and len(pairs) > mem:
                pairs.pop(0)
            if mem == 0:
                pairs.clear()
            h0_last = sy / float(np.dot(yv, yv))
        hist.append(dict(it=it, J=J, gnorm=float(np.linalg.norm(g)), alpha=alpha, trials=trials, J_new=Jn))
        if callback is not None:
            callback(it, zt * scale, Jn)
        rel = (J - Jn) / J if J > 0 else 0.0
        z, J, g = zt, Jn, gn
        if rel < rtol:
            stopped = "rtol"
            break
    return LbfgsResult(x=z * scale, J=J, history=hist, stopped=stopped)
