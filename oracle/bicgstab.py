"""O3: BiCGStab, the paper's "bi-stabilized conjugate gradient" inverter (oracle; test
infrastructure).

The paper names the algorithm (abstract; Sec. 2.3, QOPQDP's general-purpose inverter) but does not
print it. This follows van der Vorst, SIAM J. Sci. Stat. Comput. 13 (1992) 631, in its order:
  r_0 = b - A x_0, rhat = r_0, rho_0 = alpha = omega_0 = 1, v_0 = p_0 = 0; for i = 1, 2, ...:
  rho_i = <rhat, r_{i-1}>, beta = (rho_i / rho_{i-1}) (alpha / omega_{i-1}),
  p_i = r_{i-1} + beta (p_{i-1} - omega_{i-1} v_{i-1}), v_i = A p_i, alpha = rho_i / <rhat, v_i>,
  s = r_{i-1} - alpha v_i, t = A s, omega_i = <t, s> / <t, t>, x_i = x_{i-1} + alpha p_i + omega_i s,
  r_i = s - omega_i t.
<a, b> = sum conj(a) b. Stopping: |r_i| / |b| < tol on the iterated residual, then the true
residual b - A x is recomputed; if it is not below tol the method restarts from it (at most
`max_restarts` times). A breakdown (|rho_i| or |<rhat, v>| below 1e-30 |rhat| |.|, or omega = 0)
also restarts from the true residual.
"""
import numpy as np


def _dot(a, b):
    return np.vdot(a.reshape(-1), b.reshape(-1))


def _norm(a):
    return float(np.sqrt(_dot(a, a).real))


def solve(apply, b, x0=None, tol=1e-10, maxiter=10000, max_restarts=5, breakdown=1e-30):
    """Solve A x = b. Returns (x, info) with info = dict(converged, iters, restarts,
    true_relres, iter_relres)."""
    bnorm = _norm(b)
    info = dict(converged=False, iters=0, restarts=0, true_relres=0.0, iter_relres=0.0)
    if bnorm == 0.0:
        return np.zeros_like(b), dict(info, converged=True)
    x = np.zeros_like(b) if x0 is None else x0.astype(np.complex128).copy()
    r = b - apply(x) if x0 is not None and np.any(x0) else b.copy()
    iters = 0
    while True:
        rhat = r.copy()
        rho_prev, alpha, omega = 1.0 + 0j, 1.0 + 0j, 1.0 + 0j
        v = np.zeros_like(b)
        p = np.zeros_like(b)
        rel = _norm(r) / bnorm
        broke = False
        while rel >= tol and iters < maxiter:
            rho = _dot(rhat, r)
            if abs(rho) < breakdown * _norm(rhat) * _norm(r):
                broke = True
                break
            beta = (rho / rho_prev) * (alpha / omega)
            p = r + beta * (p - omega * v)
            v = apply(p)
            rv = _dot(rhat, v)
            if abs(rv) < breakdown * _norm(rhat) * _norm(v):
                broke = True
                break
            alpha = rho / rv
            s = r - alpha * v
            t = apply(s)
            tt = _dot(t, t).real
            if tt == 0.0:
                x = x + alpha * p
                r = s
                iters += 1
                rel = _norm(r) / bnorm
                break
            omega = _dot(t, s) / tt
            x = x + alpha * p + omega * s
            r = s - omega * t
            iters += 1
            rho_prev = rho
            rel = _norm(r) / bnorm
            if omega == 0:
                broke = True
                break
        info["iter_relres"] = rel
        r = b - apply(x)
        true_rel = _norm(r) / bnorm
        info.update(iters=iters, true_relres=true_rel)
        if true_rel < tol:
            info["converged"] = True
            return x, info
        if iters >= maxiter or info["restarts"] >= max_restarts:
            return x, info
        info["restarts"] += 1
        del broke
