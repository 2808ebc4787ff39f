"""Quasi-static Newton solve with contacts (Sec. II-III of the paper), plain FP64.

One call of ``Model.solve`` is one quasi-static step at a given cable tension and insertion:

  * prescribed nodes (Eq. 14-15): the robot is fed through a clamp at the lumen entrance.
    At insertion delta every node with arc length s_i <= L - delta (count from
    k = floor((L - delta) M / L + 1e-6)) sits on the entrance axis,
    x_i = e + (s_i - L + delta) d with the rest triad E0; the remaining nodes are free.
    Their DOFs are eliminated, which replaces y_fn; the reaction is F(x) at node k.
  * cable load (Eq. 16-18): cable j at angle phi_j on radius r_c pulls the tip towards the
    base, F_j = (-tau_j, 0, 0) and d_j = r_c (0, cos phi_j, sin phi_j) in the tip frame; the
    tip receives T_M F_j and T_M (d_j x F_j), evaluated at the current iterate (follower load).
  * Newton step (Eq. 20-23): K(x) and F(x) at the current iterate, contact set and A_c, b_c
    at the current iterate (Eq. 8-10), QP of Eq. 23 solved exactly through its LCP, whose
    matrix W = A K^-1 A^T carries the compliance 1e-12 max(diag W) on its diagonal (rows of
    one node are dependent where four or more wall faces meet).
  * step limiter (Eq. 25-27): alpha = min(1, rho / max_i |du_i|) scales the whole step and
    the multipliers; translations add, rotations update as T <- exp([alpha dtheta]x) T.  The
    bound rho starts at beta0.  A step that points against the previous one
    (sum_i du_i . du_i^prev < 0) is an overshoot: rho drops to half of the smaller of rho and
    that step (so the step is at most halved, and a repeating cycle shrinks geometrically);
    otherwise rho grows by 1.5 back towards beta0.  (A fixed beta0 lets a node on a faceted wall
    overshoot the crease between two facets forever, and the material tangent overshoots the
    twist of a long bent span by ~2x.)  The material tangent also converges only linearly (a slow
    bending or twist mode of a long compressed span shrinks by ~0.3-0.96 per iteration), so in the
    first ACCEL_ITERS iterations of a solve, while the active contact rows stay the same and the
    step is not clipped, the
    iteration x <- x (+) dx(x) is accelerated by Anderson's method of depth ACCEL_DEPTH (Walker & Ni
    2011, "Anderson acceleration for fixed-point iterations"): with f_j the unscaled step of
    iterate j and d_j the increment applied there, gamma minimises |W (f_k - sum_j gamma_j
    (f_{k-j} - f_{k-j-1}))| (W weighs rotations by r_o), and the increment is
    f_k - sum_j gamma_j (d_{k-j-1} + f_{k-j} - f_{k-j-1}); it is taken only when its largest nodal
    translation, bounded by max|f_k| + sum_j |gamma_j| (max|d_{k-j}| + max|f_{k-j+1} - f_{k-j}|), stays
    within beta0 and sum |gamma_j| <= ACCEL_GAMMA_MAX; a reversal right after an accelerated
    step does not shrink rho (extrapolation overshoots by design).  Later iterations (a solve that
    has not converged by then) use the 1-D secant over-relaxation instead: after a full step, an
    unclipped step with the same contact rows, pointing the same way (cosine >= 0.99) and shrinking
    by lam in [0.5, 0.98], is extended to alpha = min(1 / (1 - lam), 8, rho / max|du|).
  * convergence: unscaled step max_i max(|du_i|, r_o |dtheta_i|) <= tol and the same contact
    set as the previous iteration.
  * warm start (follow the path): with a resident state at insertion delta_old, material
    point s takes the old position of material point s + (delta - delta_old) (linear in x,
    geodesic in T between nodes; straight along the tip axis beyond the old tip).
"""
import math
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla

from . import beam, contact, lcp, segment
from .rotation import expm, logm, to_quat

CONTACT_COMPLIANCE = 1e-12
ACCEL_DEPTH = 3            # Anderson acceleration: previous iterates used
ACCEL_GAMMA_MAX = 10.0     # largest sum |gamma_j| of an accepted accelerated step
ACCEL_ITERS = 100          # iterations of a solve that may take accelerated steps (then the secant rule)

OK, E_INVALID_ARG, E_NOMEM, E_CUDA, E_NOT_CONVERGED, E_CONTACT_CAPACITY, E_NOT_SPD, E_TIMEOUT, E_PENETRATION = range(9)


@dataclass
class Options:
    # The C ABI's contact_tol (the relative sign tolerance of its active-set LCP) has no counterpart
    # here: the oracle's LCP solvers take their own tolerances (lcp.py).
    activation_gap: float = 1.0e-3
    step_limit: float = 5.0e-4
    newton_tol: float = 1.0e-11
    max_newton_iters: int = 200
    max_contact_iters: int = 4000
    max_contacts: int = 256
    tangent_mode: int = 0          # 0: material tangent K_M; 1: symmetric part of K_T (K_M if not PD)
    contact_model: str = "node"    # "node": rows at the nodes (xi = 0); "segment": Eq. 3-7 at any xi
    qp_solver: str = "contact"     # "contact": exact contact-space LCP; "primal_admm": OSQP's ADMM on Eq. 23, polished
    accel_depth: int = ACCEL_DEPTH  # Anderson acceleration of the Newton iteration (0: off)


@dataclass
class Result:
    status: int
    node_pos: np.ndarray
    node_quat: np.ndarray
    contacts: list
    newton_iters: int
    contact_iters: int
    residual: float
    base_reaction: np.ndarray


def entrance_frame(lumen):
    d = np.asarray(lumen.entrance_dir, float)
    d = d / np.linalg.norm(d)
    up = np.asarray(lumen.entrance_up, float)
    up = up - np.dot(up, d) * d
    up = up / np.linalg.norm(up)
    return np.column_stack([d, up, np.cross(d, up)])


def n_prescribed_last(L, M, delta):
    """Index k of the last prescribed node."""
    return int(math.floor((L - delta) * M / L + 1e-6))


def cable_load(T_tip, tensions, robot):
    """Eq. 16-18: tip force and moment in global coordinates."""
    F = np.zeros(3)
    Mo = np.zeros(3)
    for tau, phi in zip(tensions, robot.cable_angles):
        d_j = robot.cable_radius * np.array([0.0, math.cos(phi), math.sin(phi)])
        F_j = np.array([-tau, 0.0, 0.0])
        F += T_tip @ F_j
        Mo += T_tip @ np.cross(d_j, F_j)
    return F, Mo


def _band_mul(ab, v):
    """K v for K in symmetric upper banded form ab (ab[u + i - j, j] = K[i, j], i <= j)."""
    u = ab.shape[0] - 1
    n = len(v)
    out = ab[u] * v
    for d in range(1, u + 1):
        out[:n - d] += ab[u - d, d:] * v[d:]      # K[i, i + d] v[i + d]
        out[d:] += ab[u - d, d:] * v[:n - d]      # K[i + d, i] v[i]
    return out


class Model:
    def __init__(self, robot, lumen, options=None):
        self.robot = robot
        self.lumen = lumen
        self.opt = options or Options()
        self.secs = beam.element_sections(robot)
        self.M = robot.n_elements
        self.L = robot.length
        self.l0 = self.L / self.M
        self.E0 = entrance_frame(lumen)
        self.e = np.asarray(lumen.entrance_point, float)
        self.V = np.asarray(lumen.vertices, float)
        self.T = np.asarray(lumen.triangles, np.int64).reshape(-1, 3)
        self.state = None          # (x, R, delta)
        self.trace = None          # list -> per-iteration (alpha, umax, step, residual, m)

    # ---- configuration helpers -------------------------------------------------------
    def straight(self, delta):
        N = self.M + 1
        x = np.array([self.e + (i * self.l0 - self.L + delta) * self.E0[:, 0] for i in range(N)])
        R = np.array([self.E0.copy() for _ in range(N)])
        return x, R

    def follow_path(self, x_old, R_old, delta_old, delta):
        dd = delta - delta_old
        N = self.M + 1
        x = np.zeros((N, 3))
        R = np.zeros((N, 3, 3))
        for i in range(N):
            s = i * self.l0 + dd
            if s >= self.L:
                x[i] = x_old[self.M] + (s - self.L) * R_old[self.M][:, 0]
                R[i] = R_old[self.M]
            elif s <= 0.0:
                x[i] = x_old[0] + s * R_old[0][:, 0]
                R[i] = R_old[0]
            else:
                j = min(int(math.floor(s / self.l0)), self.M - 1)
                f = (s - j * self.l0) / self.l0
                x[i] = (1.0 - f) * x_old[j] + f * x_old[j + 1]
                R[i] = R_old[j] @ expm(f * logm(R_old[j].T @ R_old[j + 1]))
        return x, R

    def clamp(self, x, R, delta, k):
        for i in range(k + 1):
            x[i] = self.e + (i * self.l0 - self.L + delta) * self.E0[:, 0]
            R[i] = self.E0
        return x, R

    # ---- assembly ----------------------------------------------------------------------
    def assemble(self, x, R, k, mode):
        """Internal force F (6N) and the banded upper form of K on the free DOFs."""
        M = self.M
        nf = M - k
        F = np.zeros(6 * (M + 1))
        u = 11
        ab = np.zeros((u + 1, 6 * nf))
        for e in range(k, M):
            Fe = beam.internal_force(x[e], R[e], x[e + 1], R[e + 1], self.secs[e])
            F[6 * e:6 * e + 12] += Fe
            if mode == 0:
                Ke = beam.material_tangent(x[e], R[e], x[e + 1], R[e + 1], self.secs[e])
            else:
                Kt = beam.consistent_tangent(x[e], R[e], x[e + 1], R[e + 1], self.secs[e])
                Ke = 0.5 * (Kt + Kt.T)
            base = 6 * (e - (k + 1))          # free dof index of element dof 0
            for i in range(12):
                gi = base + i
                if gi < 0:
                    continue
                for j in range(i, 12):
                    gj = base + j
                    ab[u + gi - gj, gj] += Ke[i, j]
        return F, ab

    # ---- one solve ---------------------------------------------------------------------
    def solve(self, tensions=None, delta=0.0, warm=None, tip_load=None):
        """``tip_load`` = (f, m, follower) replaces the cable load (test hook)."""
        opt = self.opt
        M, L = self.M, self.L
        if not (0.0 <= delta <= L):
            raise ValueError("insertion outside [0, L]")
        k = n_prescribed_last(L, M, delta)
        if warm is not None:
            x, R = warm[0].copy(), warm[1].copy()
        elif self.state is not None:
            x, R = self.follow_path(*self.state, delta)
        else:
            x, R = self.straight(delta)
        x, R = self.clamp(x, R, delta, k)
        nf = M - k
        free = list(range(k + 1, M + 1))
        r_o = self.robot.outer_radius
        contacts = []
        y = np.zeros(0)
        prev_key = None
        it = 0
        piv_total = 0
        residual = 0.0
        rho = opt.step_limit           # step bound of the limiter (shrinks when consecutive steps reverse)
        du_prev = None
        hist_f, hist_d, hist_m = [], [], []   # previous iterates: unscaled steps, applied increments and
                                              # a bound on each increment's largest nodal translation
        accel_prev = False
        act_key_prev = None
        nrm2_prev = 0.0
        alpha_prev = 0.0
        status = E_NOT_CONVERGED
        base_reaction = np.zeros(6)
        if nf == 0:
            status = OK
        while nf > 0 and it < opt.max_newton_iters:
            it += 1
            F, ab = self.assemble(x, R, k, opt.tangent_mode)
            # external cable (or test) load at the tip node, Eq. 16-18
            Fa = np.zeros(6 * (M + 1))
            if tip_load is None:
                f, mo = cable_load(R[M], tensions, self.robot)
            else:
                f, mo, follower = tip_load
                f, mo = (R[M] @ np.asarray(f), R[M] @ np.asarray(mo)) if follower else (np.asarray(f), np.asarray(mo))
            Fa[6 * M:6 * M + 3] = f
            Fa[6 * M + 3:6 * M + 6] = mo
            g = (F - Fa)[6 * (k + 1):]
            try:
                c = sla.cholesky_banded(ab, lower=False)
            except np.linalg.LinAlgError:
                if opt.tangent_mode == 0:
                    status = E_NOT_SPD
                    break
                _, ab = self.assemble(x, R, k, 0)
                c = sla.cholesky_banded(ab, lower=False)
            solve = lambda rhs: sla.cho_solve_banded((c, False), rhs)
            if not len(self.T):
                contacts = []
            elif opt.contact_model == "segment":
                contacts = segment.detect_elements(x, k, self.V, self.T, r_o, opt.activation_gap)
            else:
                contacts = contact.detect(x, free, self.V, self.T, r_o, opt.activation_gap)
            m = len(contacts)
            if m > opt.max_contacts:
                status = E_CONTACT_CAPACITY
                break
            dxf = -solve(g)
            if m:
                A = np.zeros((m, 6 * nf))
                b = np.zeros(m)
                for i, rec in enumerate(contacts):
                    if "elem" in rec:
                        # segment row (Eq. 3, 9): n^T du(xi), du(xi) = R_r N(xi) [R_r^T du_a; R_r^T du_b]
                        e = rec["elem"]
                        _, Rr = beam.corotated_frame(x[e], R[e], x[e + 1], R[e + 1])
                        row = rec["normal"] @ segment.row_weights(Rr, rec["s"] * self.l0, self.l0)
                        for j, node in enumerate((e, e + 1)):
                            if node > k:
                                col = 6 * (node - (k + 1))
                                A[i, col:col + 3] = row[3 * j:3 * j + 3]
                    else:
                        col = 6 * (rec["node"] - (k + 1))
                        A[i, col:col + 3] = rec["normal"]
                    b[i] = rec["gap"]
                X = solve(A.T)
                W = A @ X
                # rows of one node can be linearly dependent (four or more wall faces meeting at a
                # mesh vertex), which leaves W singular; a contact compliance eps = 1e-12 max W_ii
                # makes the LCP uniquely solvable (interpenetration at most eps * y)
                W = W + CONTACT_COMPLIANCE * np.max(np.diag(W)) * np.eye(m)
                q = b - A @ dxf
                if opt.qp_solver == "primal_admm":
                    # OSQP on the primal QP: K + sigma I + rho A^T A keeps K's band (a row touches
                    # the translations of one node, or of the two nodes of an element)
                    u = ab.shape[0] - 1
                    rho_admm = 0.1 * float(np.max(ab[u]))

                    def factor(rho_):
                        mb = ab.copy()
                        mb[u] += 1.0e-6
                        for i in range(m):
                            nz = np.nonzero(A[i])[0]
                            for p_ in nz:
                                for q_ in nz:
                                    if p_ <= q_:
                                        mb[u + p_ - q_, q_] += rho_ * A[i, p_] * A[i, q_]
                        cm = sla.cholesky_banded(mb, lower=False)
                        return lambda r_: sla.cho_solve_banded((cm, False), r_)
                    y, piv, _ = lcp.primal_admm_polish(
                        factor(rho_admm), lambda v: _band_mul(ab, v), g, A, b, rho_admm, W, q, refactor=factor)
                else:
                    y, w, piv = lcp.qp_nnls(W, q)
                piv_total += piv
                dx = dxf - X @ y
                r = g + A.T @ y
            else:
                y = np.zeros(0)
                dx = dxf
                r = g
            residual = float(np.abs(r).max())
            base_reaction = F[6 * k:6 * k + 6].copy()
            du = dx.reshape(nf, 6)[:, :3]
            dth = dx.reshape(nf, 6)[:, 3:]
            umax = float(np.sqrt((du * du).sum(axis=1)).max())
            step = float(max(umax, r_o * np.sqrt((dth * dth).sum(axis=1)).max()))
            key = tuple((rec["node"] if "node" in rec else -1 - rec["elem"], rec["tri"]) for rec in contacts)
            act_key = tuple(key[i] for i in range(m) if y[i] > 0.0) if m else ()
            dot = float(np.sum(du * du_prev)) if du_prev is not None else 0.0
            # a step against the previous one is an overshoot, unless the previous one was extrapolated
            reverse = du_prev is not None and dot < 0.0 and not accel_prev
            if du_prev is not None:
                if reverse:
                    rho = max(0.5 * min(rho, umax), opt.step_limit * 2.0 ** -40)
                else:
                    rho = min(1.5 * rho, opt.step_limit)
            alpha = 1.0 if umax <= rho else rho / umax
            inc = alpha * dx
            # Anderson acceleration while the active rows and the full step persist
            anderson = opt.accel_depth > 0 and it <= ACCEL_ITERS
            steady = anderson and du_prev is not None and alpha == 1.0 and act_key == act_key_prev
            # after that (or without acceleration) the secant over-relaxation of a slow monotone mode
            nrm2 = float(np.sum(du * du))
            if (not anderson and du_prev is not None and not reverse and alpha_prev == 1.0 and alpha == 1.0
                    and key == prev_key and nrm2_prev > 0.0 and nrm2 > 0.0):
                lam = math.sqrt(nrm2 / nrm2_prev)
                cosang = dot / math.sqrt(nrm2 * nrm2_prev)
                if cosang >= 0.99 and 0.5 <= lam <= 0.98:
                    alpha = min(1.0 / (1.0 - lam), 8.0, rho / umax)
                    inc = alpha * dx
            accel = False
            bound = alpha * umax
            if steady and hist_f:
                wgt = np.tile(np.array([1.0, 1.0, 1.0, r_o, r_o, r_o]), nf)
                F = np.array(hist_f + [dx])
                dF = np.diff(F, axis=0).T                      # columns f_{i+1} - f_i, oldest first
                dD = np.array(hist_d).T                        # matching increments d_i
                Wd = dF * wgt[:, None]
                G = Wd.T @ Wd
                if np.max(np.diag(G)) > 0.0:
                    G = G + 1e-10 * np.max(np.diag(G)) * np.eye(len(G))
                    gam = np.linalg.solve(G, Wd.T @ (dx * wgt))
                    if np.all(np.isfinite(gam)) and np.sum(np.abs(gam)) <= ACCEL_GAMMA_MAX:
                        # bound on the largest nodal translation of the accelerated increment
                        cu = dF.T.reshape(len(gam), nf, 6)[:, :, :3]
                        cmax = np.sqrt((cu * cu).sum(axis=2)).max(axis=1)
                        bnd = umax + float(np.sum(np.abs(gam) * (np.array(hist_m) + cmax)))
                        if bnd <= opt.step_limit:
                            inc, accel, bound = dx - (dD + dF) @ gam, True, bnd
            if not steady:
                hist_f, hist_d, hist_m = [], [], []
            hist_f.append(dx.copy())
            hist_d.append(inc.copy())
            hist_m.append(bound)
            if len(hist_f) > opt.accel_depth:
                hist_f.pop(0)
                hist_d.pop(0)
                hist_m.pop(0)
            du_prev = du.copy()
            accel_prev = accel
            act_key_prev = act_key
            nrm2_prev = nrm2
            alpha_prev = alpha
            incr = inc.reshape(nf, 6)
            for j, i in enumerate(free):
                x[i] = x[i] + incr[j, :3]
                R[i] = expm(incr[j, 3:]) @ R[i]
            # Eq. 27 scales the multipliers of a limited step by alpha; the reported forces are the
            # multipliers of the last (converged, sub-tolerance) step, i.e. the equilibrium forces
            if self.trace is not None:
                self.trace.append((alpha, umax, step, residual, m))
            if getattr(self, "trace_detail", None) is not None:
                jmax = int(np.argmax(np.sqrt((du * du).sum(axis=1))))
                act = [(rec["node"], rec["tri"], round(float(yy), 4)) for rec, yy in zip(contacts, y) if yy > 0]
                self.trace_detail.append((free[jmax], du[jmax].copy(), act))
            if step <= opt.newton_tol and key == prev_key:
                status = OK
                break
            prev_key = key
        self.state = (x.copy(), R.copy(), delta)
        for i, rec in enumerate(contacts):
            rec["force"] = float(y[i]) if i < len(y) else 0.0
        quat = np.array([to_quat(Ri) for Ri in R])
        return Result(status, x, quat, contacts, it, piv_total, residual, base_reaction)
