"""Oracle fit driver -- TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

A quasi-Newton minimiser fed by exact oracle gradients.  Sec. 4 uses AD
gradients inside ROOT's fitter and notes that the minimiser still takes its
second derivatives numerically, i.e. it is driven by the gradient alone; the
gradient-only analogue used here is BFGS with a backtracking Armijo line
search.  The steps, in order, for one iteration:

  1. direction d = -H g (H = inverse-Hessian approximation); if g.d >= 0
     the approximation is reset to its initial diagonal and d recomputed;
  2. trial points theta + alpha d, alpha = 1 first; a trial is accepted when
     F(trial) <= F + c1 alpha g.d (c1 = 1e-4); otherwise alpha is replaced by
     the minimiser of the quadratic through F, g.d and F(trial), clamped to
     [0.1 alpha, 0.5 alpha]; a non-finite F(trial) gives 0.1 alpha; at most
     `max_trials` trials;
  3. s = step, y = change of gradient; if s.y > 1e-12 |s| |y| the BFGS update
     H <- (I - r s y^T) H (I - r y s^T) + r s s^T, r = 1/(s.y);
  4. convergence when EDM = g.H.g / 2 < tol * max(1, |F|).
The initial H is diag(1 / GN_k) with GN_k the Gauss-Newton diagonal of the
objective (GN_k <= 0 gives 1).

`lm_fit` is the second-order alternative: the minimiser handed the
Gauss-Newton matrix GN = sum_i h_i J_i J_i^T (the second derivatives Sec. 4
leaves to finite differences, here from the same adjoints) and damped as in
Levenberg-Marquardt (Levenberg 1944, Marquardt 1963).  One evaluation:

  1. at the trial point, F, g and GN; the trial is accepted when F(trial) < F
     (then lambda /= 10, at least 1e-12), otherwise lambda *= 10 and the fit
     fails once lambda > 1e16;
  2. after an acceptance, EDM = g^T GN^-1 g / 2 with the undamped matrix;
     converged when EDM < tol * max(1, |F|);
  3. the next trial is theta + delta, (GN + lambda diag(GN)) delta = -g
     (diagonal entries <= 0 count as 1); where the damped matrix is not
     positive definite, delta_k = -g_k / ((1 + lambda) diag_k).
The start evaluates theta0 with lambda = 1e-3 and checks EDM before the
first step.
"""
import numpy as np

RUNNING, CONVERGED, MAX_ITER, LINESEARCH_FAILED = 0, 1, 2, 3


def bfgs_fit(fg, gn, theta0, max_iter=50, tol=1e-9, max_trials=20, c1=1e-4):
    """Minimise F with value+gradient callback fg(theta)->(F, g) and Gauss-Newton
    diagonal callback gn(theta)->GN.  Returns dict(theta, F, g, iters, evals, status, edm, H)."""
    theta = np.array(theta0, dtype=np.float64)
    F, g = fg(theta)
    evals = 1
    d0 = gn(theta)
    Hdiag = np.where(d0 > 0, 1.0 / np.where(d0 > 0, d0, 1.0), 1.0)
    H = np.diag(Hdiag)
    status = RUNNING
    it = 0
    edm = 0.5 * g @ H @ g
    if edm < tol * max(1.0, abs(F)):
        status = CONVERGED
    while status == RUNNING and it < max_iter:
        d = -H @ g
        gd = g @ d
        if not gd < 0:
            H = np.diag(Hdiag)
            d = -H @ g
            gd = g @ d
        alpha = 1.0
        accepted = False
        for _ in range(max_trials):
            tt = theta + alpha * d
            Ft, gt = fg(tt)
            evals += 1
            if np.isfinite(Ft) and Ft <= F + c1 * alpha * gd:
                accepted = True
                break
            if np.isfinite(Ft):
                denom = 2.0 * (Ft - F - gd * alpha)
                a_new = -gd * alpha * alpha / denom if denom > 0 else 0.5 * alpha
                alpha = min(max(a_new, 0.1 * alpha), 0.5 * alpha)
            else:
                alpha = 0.1 * alpha
        if not accepted:
            status = LINESEARCH_FAILED
            break
        s = tt - theta
        y = gt - g
        sy = s @ y
        if sy > 1e-12 * np.linalg.norm(s) * np.linalg.norm(y):
            r = 1.0 / sy
            I = np.eye(len(theta))
            H = (I - r * np.outer(s, y)) @ H @ (I - r * np.outer(y, s)) + r * np.outer(s, s)
        theta, F, g = tt, Ft, gt
        it += 1
        edm = 0.5 * g @ H @ g
        if edm < tol * max(1.0, abs(F)):
            status = CONVERGED
    if status == RUNNING:
        status = MAX_ITER
    return dict(theta=theta, F=F, g=g, iters=it, evals=evals, status=status, edm=edm, H=H)


def _chol_solve(M, b):
    """Solution of M x = b by Cholesky, or None where M is not positive definite."""
    try:
        L = np.linalg.cholesky(M)
    except np.linalg.LinAlgError:
        return None
    return np.linalg.solve(L.T, np.linalg.solve(L, b))


def _edm(g, G):
    z = _chol_solve(G, g)
    if z is None:
        dg = np.diag(G)
        z = g / np.where(dg > 0, dg, 1.0)
    return 0.5 * g @ z


def lm_fit(fgh, theta0, max_evals=60, tol=1e-9, lam0=1e-3):
    """Minimise F with callback fgh(theta) -> (F, g, GN).  Returns
    dict(theta, F, g, iters, evals, status, edm, lam)."""
    theta = np.array(theta0, dtype=np.float64)
    F, g, G = fgh(theta)
    evals, it, lam = 1, 0, lam0
    status = RUNNING if np.isfinite(F) else 4
    edm = 0.0
    if status == RUNNING:
        edm = _edm(g, G)
        if edm < tol * max(1.0, abs(F)):
            status = CONVERGED
    while status == RUNNING and evals < max_evals:
        dg = np.diag(G)
        dpos = np.where(dg > 0, dg, 1.0)
        delta = _chol_solve(G + lam * np.diag(dpos), -g)
        if delta is None:
            delta = -g / ((1.0 + lam) * dpos)
        tt = theta + delta
        Ft, gt, Gt = fgh(tt)
        evals += 1
        if np.isfinite(Ft) and Ft < F:
            theta, F, g, G = tt, Ft, gt, Gt
            it += 1
            lam = max(lam * 0.1, 1e-12)
            edm = _edm(g, G)
            if edm < tol * max(1.0, abs(F)):
                status = CONVERGED
        else:
            lam *= 10.0
            if lam > 1e16:
                status = LINESEARCH_FAILED
    return dict(theta=theta, F=F, g=g, iters=it, evals=evals, status=status, edm=edm, lam=lam)
