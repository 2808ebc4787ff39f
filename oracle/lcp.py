"""Exact solution of the contact problem of one Newton step (Eq. 12-13, 22-23).

With the prescribed DOFs eliminated and K symmetric positive definite, the QP of Eq. 23
  min 1/2 dx^T K dx + g^T dx   s.t.  A dx <= b
has the unique minimiser dx = -K^{-1} (g + A^T y), where y >= 0 solves the LCP
  w = W y + q >= 0,  y >= 0,  y^T w = 0,   W = A K^{-1} A^T,  q = b + A K^{-1} g
(w is the slack b - A dx of Eq. 8; y the contact forces of Eq. 11).  W is symmetric
positive definite when the rows of A are independent (one contact per node), so the LCP
has exactly one solution.  Two exact finite methods are given: Murty's least-index
principal pivoting (finite for P-matrices in exact arithmetic) and, for small m, enumeration of all
2^m complementary sets; the solver uses the QP form (non-negative least squares), which stays
robust when W is ill-conditioned.
"""
import itertools

import numpy as np
import scipy.linalg as sla
from scipy.optimize import nnls


def qp_nnls(W, q):
    """The LCP solution as the minimiser of the convex QP 1/2 y^T W y + q^T y over y >= 0 (its KKT
    conditions are the LCP): with W = L L^T, min |L^T y + L^-1 q|^2 subject to y >= 0, solved by
    the Lawson-Hanson non-negative least squares routine of scipy.  Returns (y, w, iterations)."""
    m = len(q)
    if m == 0:
        return np.zeros(0), np.zeros(0), 0
    L = sla.cholesky(W, lower=True)
    b = -sla.solve_triangular(L, q, lower=True)
    y, _ = nnls(L.T, b, maxiter=50 * m + 100)
    w = W @ y + q
    return y, w, 0


def _solve_set(W, q, P):
    y = np.zeros(len(q))
    if P.any():
        y[P] = np.linalg.solve(W[np.ix_(P, P)], -q[P])
    return y


def murty(W, q, tol=0.0, max_pivots=100000):
    """Least-index principal pivoting (K. G. Murty, 1974).  Start from y = 0; while some
    complementary variable is negative (y_i < -tol for i in P, w_i < -tol for i not in P),
    move the lowest such index across.  Returns (y, w, pivots)."""
    m = len(q)
    P = np.zeros(m, dtype=bool)
    for it in range(max_pivots + 1):
        y = _solve_set(W, q, P)
        w = W @ y + q
        w[P] = 0.0
        bad = np.where((P & (y < -tol)) | (~P & (w < -tol)))[0]
        if len(bad) == 0:
            return y, w, it
        i = bad[0]
        P[i] = not P[i]
    raise RuntimeError("LCP pivoting did not terminate")


def enumerate_lcp(W, q, tol=1e-12):
    """All complementary sets P; returns every (y, w) that satisfies the LCP (for m <= 12)."""
    m = len(q)
    sols = []
    scale = max(1.0, np.abs(q).max()) if m else 1.0
    for bits in itertools.product([False, True], repeat=m):
        P = np.array(bits, dtype=bool)
        try:
            y = _solve_set(W, q, P)
        except np.linalg.LinAlgError:
            continue
        w = W @ y + q
        w[P] = 0.0
        if (y >= -tol * scale).all() and (w >= -tol * scale).all():
            sols.append((y, w))
    return sols


def admm(W, q, rho=None, sigma=1.0e-6, alpha=1.6, eps_abs=0.0, eps_rel=1.0e-3, max_iter=4000, check_every=10):
    """OSQP's ADMM (Stellato et al., "OSQP: an operator splitting solver for quadratic programs",
    2020, the solver the paper uses for Eq. 23) on the contact-space form of the QP,
        min 1/2 y^T W y + q^T y   s.t.  0 <= y,
    i.e. OSQP's problem with P = W, constraint matrix I, l = 0, u = +inf.  One iteration with the
    step sizes sigma, rho and the relaxation alpha:
        (W + (sigma + rho) I) yt = sigma y - q + rho z - lam      (the matrix is factored once)
        y <- alpha yt + (1 - alpha) y
        zh = alpha yt + (1 - alpha) z
        z <- max(zh + lam / rho, 0),   lam <- lam + rho (zh - z)
    stopped when the primal residual |y - z|_inf and the dual residual |W y + q + lam|_inf are
    below eps_abs + eps_rel times the scale of their terms.  rho defaults to 0.1 max(diag W).
    Returns (y, z, lam, iterations)."""
    m = len(q)
    if m == 0:
        return np.zeros(0), np.zeros(0), np.zeros(0), 0
    W = np.asarray(W, float)
    q = np.asarray(q, float)
    if rho is None:
        rho = 0.1 * float(np.max(np.diag(W)))
    c = sla.cho_factor(W + (sigma + rho) * np.eye(m))
    y = np.zeros(m)
    z = np.zeros(m)
    lam = np.zeros(m)
    it = 0
    while it < max_iter:
        it += 1
        yt = sla.cho_solve(c, sigma * y - q + rho * z - lam)
        y = alpha * yt + (1.0 - alpha) * y
        zh = alpha * yt + (1.0 - alpha) * z
        z = np.maximum(zh + lam / rho, 0.0)
        lam = lam + rho * (zh - z)
        if it % check_every == 0:
            Wy = W @ y
            r_prim = np.abs(y - z).max()
            r_dual = np.abs(Wy + q + lam).max()
            if (r_prim <= eps_abs + eps_rel * max(np.abs(y).max(), np.abs(z).max()) and
                    r_dual <= eps_abs + eps_rel * max(np.abs(Wy).max(), np.abs(lam).max(), np.abs(q).max())):
                break
    return y, z, lam, it


def admm_polish(W, q, **admm_args):
    """The paper's solve of Eq. 23 (OSQP) carried to the exact solution: ADMM gives the guess of
    the rows whose bound y >= 0 is not binding (z_i > -lam_i: the projection did not clip), the
    equality-constrained problem on them, W_FF y_F = -q_F with y = 0 elsewhere, is solved exactly
    ("polish"), and the result is accepted when it satisfies the LCP (y_F > 0, w = W y + q >= 0 on
    the other rows, to a relative tolerance of 1e-12); otherwise the exact active-set solution of
    qp_nnls is returned.  Returns (y, w, admm_iterations, polished)."""
    m = len(q)
    if m == 0:
        return np.zeros(0), np.zeros(0), 0, True
    y, z, lam, it = admm(W, q, **admm_args)
    F = z > -lam
    yp = _solve_set(W, q, F)
    w = W @ yp + q
    scale_y = max(np.abs(yp).max(), 1e-300)
    scale_w = max(np.abs(q).max(), 1e-300)
    if (yp[F] > 0.0).all() and (w[~F] >= -1e-12 * scale_w).all() and (np.abs(yp[~F]) <= 1e-12 * scale_y).all():
        return yp, w, it, True
    ye, we, _ = qp_nnls(W, q)
    return ye, we, it, False


def primal_admm(solve_M, K_mul, g, A, b, rho, sigma=1.0e-6, alpha=1.6, eps_rel=1.0e-3, max_iter=4000,
                check_every=10, refactor=None):
    """OSQP's ADMM (Stellato et al. 2020) on the primal QP of Eq. 23,
        min 1/2 dx^T K dx + g^T dx   s.t.  A dx <= b,
    i.e. OSQP's problem with P = K, l = -inf, u = b.  solve_M applies (K + sigma I + rho A^T A)^-1
    (factored once by the caller), K_mul applies K.  One iteration:
        xt = (K + sigma I + rho A^T A)^-1 (sigma x - g + A^T (rho z - lam)),  zt = A xt
        x <- alpha xt + (1 - alpha) x,  zh = alpha zt + (1 - alpha) z
        z <- min(zh + lam / rho, b),    lam <- lam + rho (zh - z)
    stopped when |A x - z| <= eps_rel max(|A x|, |z|) and |K x + g + A^T lam| <= eps_rel max(|K x|,
    |A^T lam|, |g|) (infinity norms, tested every check_every iterations).  With refactor (rho ->
    a new solve_M), rho adapts as in OSQP (the same paper, Sec. 5.2): at each test, with the two
    residuals relative to their scales, rho_new = rho sqrt(primal / dual), taken (and the matrix
    refactored) when it differs from rho by more than a factor 5.  Returns (x, z, lam, iters)."""
    n, m = len(g), len(b)
    x = np.zeros(n)
    z = np.zeros(m)
    lam = np.zeros(m)
    it = 0
    while it < max_iter:
        it += 1
        xt = solve_M(sigma * x - g + A.T @ (rho * z - lam))
        zt = A @ xt
        x = alpha * xt + (1.0 - alpha) * x
        zh = alpha * zt + (1.0 - alpha) * z
        z = np.minimum(zh + lam / rho, b)
        lam = lam + rho * (zh - z)
        if it % check_every == 0:
            Ax, Kx, Atl = A @ x, K_mul(x), A.T @ lam
            rp, sp = np.abs(Ax - z).max(), max(np.abs(Ax).max(), np.abs(z).max())
            rd, sd = np.abs(Kx + g + Atl).max(), max(np.abs(Kx).max(), np.abs(Atl).max(), np.abs(g).max())
            if rp <= eps_rel * sp and rd <= eps_rel * sd:
                break
            if refactor is not None and rp > 0.0 and rd > 0.0 and sp > 0.0 and sd > 0.0:
                rho_new = rho * np.sqrt((rp / sp) / (rd / sd))
                if rho_new > 5.0 * rho or rho_new < rho / 5.0:
                    rho = rho_new
                    solve_M = refactor(rho)
    return x, z, lam, it


def primal_admm_polish(solve_M, K_mul, g, A, b, rho, W, q, **kw):
    """The primal ADMM's guess of the active rows (lam > 0: the upper bound z <= b binds), polished
    exactly: the multipliers of those rows from the contact-space equations W_AA y_A = -q_A
    (W = A K^-1 A^T, q = b + A K^-1 g, as the caller forms them) and y = 0 elsewhere, accepted when
    y_A > 0 and every other row keeps A dx <= b (relative 1e-12); otherwise the exact contact-space
    solution (qp_nnls).  Returns (y, admm_iterations, polished); dx = -K^-1 (g + A^T y)."""
    x, z, lam, it = primal_admm(solve_M, K_mul, g, A, b, rho, **kw)
    act = lam > 0.0
    y = _solve_set(W, q, act)
    w = W @ y + q
    sw = max(np.abs(q).max(), 1e-300)
    if (y[act] > 0.0).all() and (w[~act] >= -1e-12 * sw).all():
        return y, it, True
    y, _, _ = qp_nnls(W, q)
    return y, it, False
