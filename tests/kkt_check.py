"""Checks of a returned QP solution against definitions that the paper states
directly (no solver arithmetic): the optimality conditions of §2
(Eqs. prim_feas, dual_feas, compl_slack), the benchmark acceptance test of §8
and the infeasibility certificates of §2.1."""
import numpy as np


def full_P(qp):
    return qp.P_full() if hasattr(qp, "P_full") else qp.P


def acceptance(qp, x, y, eps_abs, eps_rel):
    """§8 acceptance test: ‖(Ax−u)₊ + (Ax−l)₋‖∞ ≤ ε_prim and
    ‖Px + q + Aᵀy‖∞ ≤ ε_dual with the tolerances of §3.4."""
    P = full_P(qp)
    Ax = qp.A @ x
    Px = P @ x
    Aty = qp.A.T @ y
    viol = np.maximum(Ax - qp.u, 0.0) + np.minimum(Ax - qp.l, 0.0)
    prim = np.max(np.abs(viol)) if qp.m else 0.0
    dual = np.max(np.abs(Px + qp.q + Aty))
    z = np.clip(Ax, qp.l, qp.u)
    eps_p = eps_abs + eps_rel * max(np.max(np.abs(Ax), initial=0.0), np.max(np.abs(z), initial=0.0))
    eps_d = eps_abs + eps_rel * max(np.max(np.abs(Px)), np.max(np.abs(Aty), initial=0.0),
                                    np.max(np.abs(qp.q)))
    return prim, dual, eps_p, eps_d


U32 = 2.0 ** -24  # unit roundoff of IEEE single precision (round to nearest)


def fp32_data_allowance(qp, x, y):
    """How far the residuals of (x, y) can move when every entry of P and A
    is rounded to FP32: each entry then carries a relative error of at most
    2⁻²⁴, whatever diagonal scaling precedes the rounding, so the primal
    residual moves by at most u·‖|A||x|‖∞ and the dual one by at most
    u·‖|P||x| + |Aᵀ||y|‖∞.  A solver that keeps its matrices in FP32
    certifies its tolerances on the rounded problem; on the problem as given
    its residuals may exceed them by these amounts and no more."""
    P = abs(full_P(qp))
    A = abs(qp.A)
    ax, ay = np.abs(x), np.abs(y)
    ap = U32 * np.max(A @ ax, initial=0.0) if qp.m else 0.0
    ad = U32 * np.max(P @ ax + A.T @ ay)
    return float(ap), float(ad)


def objective(qp, x):
    P = full_P(qp)
    return 0.5 * x @ (P @ x) + qp.q @ x


def primal_cert_ok(qp, y, eps=1e-3):
    """Eq. (prim-infeas-linear): Aᵀy = 0 (relative to ‖y‖∞) and
    uᵀy₊ + lᵀy₋ < 0, with y paired only with finite bounds."""
    ny = np.max(np.abs(y))
    if ny == 0:
        return False
    yp, ym = np.maximum(y, 0.0), np.minimum(y, 0.0)
    if np.any((yp > 0) & ~np.isfinite(qp.u)) or np.any((ym < 0) & ~np.isfinite(qp.l)):
        return False
    s = float(np.sum(qp.u[yp > 0] * yp[yp > 0]) + np.sum(qp.l[ym < 0] * ym[ym < 0]))
    return np.max(np.abs(qp.A.T @ y)) <= eps * ny and s < 0


def dual_cert_ok(qp, x, eps=1e-3):
    """Eq. (dual-infeas-linear): Px = 0, qᵀx < 0, and (Ax)_i = 0 / ≥ 0 / ≤ 0
    by bound type, all relative to ‖x‖∞."""
    nx = np.max(np.abs(x))
    if nx == 0:
        return False
    P = full_P(qp)
    if np.max(np.abs(P @ x)) > eps * nx or not (qp.q @ x < 0):
        return False
    Ax = qp.A @ x
    lf, uf = np.isfinite(qp.l), np.isfinite(qp.u)
    ok = np.where(lf & uf, np.abs(Ax) <= eps * nx, True)
    ok &= np.where(~uf & lf, Ax >= -eps * nx, True)
    ok &= np.where(~lf & uf, Ax <= eps * nx, True)
    return bool(np.all(ok))


def objective_interval(qp, x, z, y, x_star, y_star):
    """Bounds on f(x) − f* for a point with z ∈ C and y ∈ N_C(z) (true of
    every ADMM iterate, §3.3), from convexity of f and the normal-cone
    inequalities, with (x*, y*) an optimal primal-dual pair:
        −‖y*‖₁‖r_p‖∞ ≤ f(x) − f* ≤ ‖r_d‖∞‖x − x*‖₁ + ‖y‖₁‖r_p‖∞,
    r_p = Ax − z, r_d = Px + q + Aᵀy (Eqs. res_prim, res_dual)."""
    P = full_P(qp)
    rp = np.max(np.abs(qp.A @ x - z), initial=0.0)
    rd = np.max(np.abs(P @ x + qp.q + qp.A.T @ y))
    lo = -np.sum(np.abs(y_star)) * rp
    hi = rd * np.sum(np.abs(x - x_star)) + np.sum(np.abs(y)) * rp
    return lo, hi
