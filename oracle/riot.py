"""FP64 reference of the RIOT inner loop and its incremental 4D-Var setting.

Test infrastructure: a plain, slow, dense restatement of the method that the
GPU library is checked against.  Citations are to the paper's sections,
equations and algorithms (Bousserez, Guerrette & Henze, arXiv:1906.01413).

Notation (Section 2.1 and Algorithm 3):
  x        model initial state (the control of Lorenz-96 4D-Var)
  L        prior square root, B = L L^T (Eq. 3), dx = L dv
  d        innovation d = H(x) - y           (Algorithm 3 sign; Eq. 3 uses y - H(x))
  A        prior-preconditioned Hessian A = L^T H^T R^-1 H L (Eq. 4)
  b        b = L^T H^T R^-1 d; the increment acts on g = b + v (Algorithm 3)
  Omega    Gaussian sketch, Y = A Omega, Q = orth(Y), K Q^T Omega = Q^T Y,
           K = Z Lambda Z^T, U = Q Z                           (Algorithm 3)
  LRA/LRU  increment and covariance forms of Eqs. 8-10, chosen by the
           smallest retained eigenvalue (Algorithm 3: lambda_m > 1 -> LRA)

Readings where the paper is ambiguous (each is also listed in the design notes):
  * Eqs. 8/9 print L^T(...)L; with B = L L^T the posterior covariance is
    L(...)L^T, which is what is computed here.
  * The LRA/LRU switch follows Algorithm 3 (strict lambda_m > 1), not the
    ">= 1" of Eq. 11; lambda are eigenvalues of A (not I + A).
  * K solves K (Q^T W) = Q^T Y by an LU solve with pivoting and is then
    symmetrised, K <- (K + K^T)/2.  With power iterations, W is the last
    block fed to the Hessian (Halko et al. subspace iteration, Section 2.2
    mentions randomized power iteration as a remedy for flat spectra).
  * Eigenpairs are sorted by decreasing eigenvalue (Eq. 8 "decreasing
    eigenvalue order"), and each eigenvector's sign is fixed so that its
    largest-magnitude component is positive.
  * Spectral preconditioning (Algorithm 3, precond): v stays the control of
    x = x_b + L v; loop k solves for w with v = v_{k-1} + P_k w, so its gradient
    is P_k^T (b + v_{k-1}) and v += P_k dw.  Factors are built from the pairs
    with positive eigenvalue (the solve for K can return values below -1).
  * Algorithm 2 (VarBL): the final increment acts on the unperturbed gradient
    g = b + v; L_R = diag(sigma_o).
  * Algorithm 4 (RIOT-PSAS): d = y - H(x) (the dual's own sign), the state is
    x_k = x_b + B H^T dw (the listing's x_{k-1} + B H^T dw counts x_{k-1} - x_b
    twice from the second cycle on).
"""
from dataclasses import dataclass

import numpy as np

from . import l96


@dataclass
class L96Problem:
    """One Lorenz-96 assimilation window (Section 3.1)."""
    n: int
    T: int
    dt: float
    F: float
    obs_step: np.ndarray     # (p,) int, step of each observation, 0..T
    obs_idx: np.ndarray      # (p,) int, observed variable
    y: np.ndarray            # (p,) observed values
    sigma_o: np.ndarray      # (p,) observation error standard deviations
    L: np.ndarray            # (n, n) prior square root
    x_b: np.ndarray          # (n,) background

    @property
    def p(self):
        return self.obs_idx.size

    @property
    def rinv(self):
        return 1.0 / (self.sigma_o * self.sigma_o)


# --- model pieces ---------------------------------------------------------------

def trajectory(prob, x):
    """Integrate and store the trajectory H(x) (Algorithm 3, outer loop)."""
    return l96.nl(x, prob.T, prob.dt, prob.F)


def observe(prob, states):
    """Observation operator: state (T+1, n) -> values at (obs_step, obs_idx)."""
    return states[prob.obs_step, prob.obs_idx]


def innovation(prob, traj):
    """d = H(x) - y (Algorithm 3)."""
    return observe(prob, traj) - prob.y


def obs_forcing(prob, r):
    """Dense adjoint forcing: scatter r (p,) into a (T+1, n) array (H^T r)."""
    f = np.zeros((prob.T + 1, prob.n))
    np.add.at(f, (prob.obs_step, prob.obs_idx), r)
    return f


def cost(prob, traj, v):
    """Non-quadratic cost (Eq. 2) in control space:
    J = 1/2 ||R^-1/2 (H(x) - y)||^2 + 1/2 ||v||^2, with x - x_b = L v."""
    d = innovation(prob, traj)
    return 0.5 * float(np.sum(d * d * prob.rinv)) + 0.5 * float(np.dot(v, v))


def gradient_b(prob, traj, d):
    """b = L^T H^T R^-1 d: one adjoint integration (Algorithm 3)."""
    lam0 = l96.ad(traj, obs_forcing(prob, d * prob.rinv), prob.dt, prob.F)
    return prob.L.T @ lam0


def hvp(prob, traj, W):
    """A W for the columns of W (n, m): A w = L^T sum_t M_{0->t}^T H_t^T R^-1 H_t M_{0->t} L w
    (Eq. 4, Algorithm 3: one TL forward and one AD backward integration per column)."""
    W = np.atleast_2d(np.asarray(W, dtype=np.float64).T).T
    out = np.empty_like(W)
    for j in range(W.shape[1]):
        dx0 = prob.L @ W[:, j]
        dxs = l96.tl(traj, dx0, prob.dt, prob.F)
        r = observe(prob, dxs) * prob.rinv
        lam0 = l96.ad(traj, obs_forcing(prob, r), prob.dt, prob.F)
        out[:, j] = prob.L.T @ lam0
    return out


def dense_hessian(prob, traj):
    """A as a dense matrix, by applying it to the identity (tiny n only)."""
    return hvp(prob, traj, np.eye(prob.n))


def tl_matrix(prob, traj):
    """G = d(observations)/d(v): the (p, n) Jacobian H M L (tiny n only)."""
    G = np.empty((prob.p, prob.n))
    for j in range(prob.n):
        dxs = l96.tl(traj, prob.L[:, j], prob.dt, prob.F)
        G[:, j] = observe(prob, dxs)
    return G


# --- inner-loop solvers ------------------------------------------------------------

def cg_solve(apply, rhs, tol=1e-13, maxiter=None):
    """Conjugate gradients for an SPD operator (textbook, Hestenes-Stiefel)."""
    x = np.zeros_like(rhs)
    r = rhs.copy()
    p = r.copy()
    rr = float(r @ r)
    r0 = np.sqrt(rr)
    maxiter = maxiter or 10 * rhs.size
    for _ in range(maxiter):
        if np.sqrt(rr) <= tol * r0 or r0 == 0.0:
            break
        Ap = apply(p)
        alpha = rr / float(p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x


def converged_increment(prob, traj, g, tol=1e-13):
    """The exact inner-loop minimiser dv* = -(I + A)^-1 g by CG (Eq. 3 with
    Algorithm 3's g = b + v)."""
    return -cg_solve(lambda p: p + hvp(prob, traj, p[:, None])[:, 0], g, tol=tol)


def varcg(prob, traj, g, m):
    """Algorithm 1 (VarCG in Lanczos form) with full re-orthogonalisation.
    Readings of its typos: beta_0 = ||r_0||, and the three-term recurrence
    subtracts beta_{i-1} q_{i-1}.  Returns (dv, theta, U)."""
    n = g.size
    Qs = []
    alphas, betas = [], []
    r = g.copy()
    beta = np.linalg.norm(r)
    q_prev = np.zeros(n)
    beta_prev = 0.0
    for i in range(m):
        if beta == 0.0:
            break
        q = r / beta
        Qs.append(q)
        w = hvp(prob, traj, q[:, None])[:, 0]
        alpha = float(q @ w)
        r = w - alpha * q - beta_prev * q_prev
        Qm = np.array(Qs).T
        r -= Qm @ (Qm.T @ r)
        r -= Qm @ (Qm.T @ r)
        alphas.append(alpha)
        beta_prev, q_prev = beta, q
        beta = np.linalg.norm(r)
        betas.append(beta)
    mm = len(alphas)
    Tm = np.diag(alphas) + np.diag(betas[:mm - 1], 1) + np.diag(betas[:mm - 1], -1)
    theta, Z = np.linalg.eigh(Tm)
    U = np.array(Qs).T @ Z
    c = U.T @ g
    dv = -U @ (c / (1.0 + theta))
    return dv, theta, U


def gradient_samples(prob, x, v, eps_obs, eps_b):
    """Starting block of Algorithm 2 (VarBL): for sample j, the gradient at the perturbed state
    x + L eps_b_j with perturbed observations,
        b_j = L^T H_j^T R^-1 d_j + v + eps_b_j,   d_j = H(x + L eps_b_j) - y + L_R eps_obs_j,
    H_j^T the adjoint at x + L eps_b_j and L_R = diag(sigma_o) (R = L_R L_R^T).
    eps_obs: (p, l), eps_b: (n, l); the listing sets eps_b_1 = 0, which is the caller's choice."""
    eps_obs = np.asarray(eps_obs, dtype=np.float64)
    eps_b = np.asarray(eps_b, dtype=np.float64)
    l = eps_b.shape[1]
    B = np.empty((prob.n, l))
    for j in range(l):
        traj = trajectory(prob, x + prob.L @ eps_b[:, j])
        d = observe(prob, traj) - prob.y + prob.sigma_o * eps_obs[:, j]
        B[:, j] = gradient_b(prob, traj, d) + v + eps_b[:, j]
    return B


def varbl(prob, traj, B0, m, g, apply=None):
    """Algorithm 2 (VarBL): block Lanczos on A from the orthonormalised gradient samples B0
    (n, l), m block steps.  Step i: Y_i = A Q_i, M_i = Q_i^T Y_i; unless i = m, the residual
    r = Y_i - Q_i M_i - Q_{i-1} W_{i-1}^T is factored r = Q_{i+1} W_i (QR) and Q_{i+1} is
    re-orthonormalised against Q_1 .. Q_i (twice, as the listing asks; the second QR's factor
    is carried into W_i so that r = Q_{i+1} W_i still holds).  T (ml x ml) has M_i on
    the diagonal and W_i / W_i^T below / above it; T = Z Lambda Z^T, U = Q Z and
    dv = -U diag(1 / (1 + lambda)) U^T g.
    Reading: the listing's final b is the gradient of the unperturbed problem, g = b + v at
    x_{k-1} (the samples only span the Krylov space).  The recurrence stops early when a
    residual block loses rank (|diag W_i| below 1e-12 of the largest |M| seen): the Krylov
    space is then invariant.  Returns (dv, lam descending, U, T, Q)."""
    apply = apply or (lambda W: hvp(prob, traj, W))
    B0 = np.asarray(B0, dtype=np.float64)
    l = B0.shape[1]
    Qs = [orthonormal_basis(B0)]
    Ms, Ws = [], []
    scale = 0.0
    for i in range(m):
        Qi = Qs[-1]
        Yi = apply(Qi)
        Mi = Qi.T @ Yi
        Ms.append(Mi)
        scale = max(scale, float(np.abs(Mi).max()))
        if i == m - 1:
            break
        r = Yi - Qi @ Mi
        if i > 0:
            r = r - Qs[-2] @ Ws[-1].T
        Qn, Wi = np.linalg.qr(r, mode="reduced")
        if np.abs(np.diag(Wi)).min() <= 1e-12 * scale:
            break
        Qprev = np.hstack(Qs)
        for _ in range(2):
            Qn = Qn - Qprev @ (Qprev.T @ Qn)
        Qn, R2 = np.linalg.qr(Qn, mode="reduced")     # r = Q_{i+1} (R2 W_i) after the re-orthonormalisation
        Ws.append(R2 @ Wi)
        Qs.append(Qn)
    nb = len(Ms)
    T = np.zeros((nb * l, nb * l))
    for i in range(nb):
        T[i * l:(i + 1) * l, i * l:(i + 1) * l] = Ms[i]
        if i + 1 < nb:
            T[(i + 1) * l:(i + 2) * l, i * l:(i + 1) * l] = Ws[i]
            T[i * l:(i + 1) * l, (i + 1) * l:(i + 2) * l] = Ws[i].T
    T = 0.5 * (T + T.T)
    lam, Z = np.linalg.eigh(T)
    order = np.argsort(-lam, kind="stable")
    lam, Z = lam[order], Z[:, order]
    Q = np.hstack(Qs[:nb])
    U = Q @ Z
    dv = -U @ ((U.T @ g) / (1.0 + lam))
    return dv, lam, U, T, Q


def orthonormal_basis(Y):
    """Q of a Householder QR of Y (LAPACK geqrf/orgqr via numpy)."""
    Q, _ = np.linalg.qr(Y, mode="reduced")
    return Q


def fix_signs(U):
    """Make the largest-magnitude entry of each column positive."""
    idx = np.argmax(np.abs(U), axis=0)
    s = np.sign(U[idx, np.arange(U.shape[1])])
    s[s == 0] = 1.0
    return U * s


def rsvd(prob, traj, Omega, q=0, exact_rr=False, apply=None):
    """Randomized eigendecomposition of A (Algorithm 3, inner loop).

    Omega: (n, m) sketch.  Y = A Omega; q rounds of subspace iteration
    (Q = orth(Y); Y = A Q); Q = orth(Y); K solves K (Q^T W) = Q^T Y with W
    the last block applied, symmetrised (or K = Q^T A Q when exact_rr);
    K = Z Lambda Z^T; U = Q Z.  Returns (lam descending, U (n, m), info)."""
    apply = apply or (lambda W: hvp(prob, traj, W))
    W = np.asarray(Omega, dtype=np.float64)
    Y = apply(W)
    for _ in range(q):
        W = orthonormal_basis(Y)
        Y = apply(W)
    Q = orthonormal_basis(Y)
    if exact_rr:
        K = Q.T @ apply(Q)
    else:
        Mq = Q.T @ W
        Nq = Q.T @ Y
        K = np.linalg.solve(Mq.T, Nq.T).T
    K = 0.5 * (K + K.T)
    lam, Z = np.linalg.eigh(K)
    order = np.argsort(-lam, kind="stable")
    lam, Z = lam[order], Z[:, order]
    U = fix_signs(Q @ Z)
    return lam, U, {"Q": Q, "K": K, "Y": Y, "W": W}


def increment(lam, U, g):
    """Adaptive increment of Algorithm 3 (Eqs. 8-11):
    lambda_m > 1: dv = -U diag(1/(1+lambda)) U^T g              (LRA, mode 0)
    otherwise:    dv = -(g - U diag(lambda/(1+lambda)) U^T g)   (LRU, mode 1)."""
    c = U.T @ g
    if lam[-1] > 1.0:
        return -(U @ (c / (1.0 + lam))), 0
    return -(g - U @ (c * lam / (1.0 + lam))), 1


def analysis_cov_lowrank(L, lam, U):
    """Low-rank posterior covariance (Eqs. 8/9 with B = L L^T):
    LRU: P_a = B - (L U) diag(lambda/(1+lambda)) (L U)^T
    LRA: P_a = (L U) diag(1/(1+lambda)) (L U)^T.
    Returns (LU, coefficients, mode) with the same mode rule as the increment."""
    LU = L @ U
    if lam[-1] > 1.0:
        return LU, 1.0 / (1.0 + lam), 0
    return LU, lam / (1.0 + lam), 1


def analysis_cov_dense(L, lam, U):
    LU, coef, mode = analysis_cov_lowrank(L, lam, U)
    low = (LU * coef) @ LU.T
    if mode == 0:
        return low
    return L @ L.T - low


def dofs(lam):
    """Degrees of freedom for signal, sum lambda/(1+lambda) (Section 3.2)."""
    lam = np.asarray(lam)
    return float(np.sum(lam / (1.0 + lam)))


# --- outer loop ---------------------------------------------------------------------

def outer_step(prob, x, v, Omega, q=0, exact_rr=False):
    """One cycle of Algorithm 3 (precond = rotation = false).
    Returns a dict with J (at x), g, lam, U, dv, mode, and the updated x, v."""
    traj = trajectory(prob, x)
    d = innovation(prob, traj)
    J = cost(prob, traj, v)
    b = gradient_b(prob, traj, d)
    g = b + v
    lam, U, info = rsvd(prob, traj, Omega, q=q, exact_rr=exact_rr)
    dv, mode = increment(lam, U, g)
    return {"traj": traj, "J": J, "b": b, "g": g, "lam": lam, "U": U, "dv": dv, "mode": mode,
            "x_next": x + prob.L @ dv, "v_next": v + dv, "info": info}


# --- spectral preconditioner and rotation (Section 2.2 "Preconditioning", Eq. 7, Algorithm 3) ---

class SpectralPreconditioner:
    """P_k = P'_0 P'_1 ... P'_{k-1} of Algorithm 3 with P'_0 = I and, for each finished outer
    loop j, P'_j = I + V_j (Lt_j^{-1/2} - I) V_j^T (the spectral form of Eq. 7, with the
    eigenvalues of I + A as Algorithm 3 writes them, not of A as Eq. 7 does), where V_j
    (orthonormal columns) and Lt_j = Lambda_j + I are the Ritz vectors and the eigenvalues of
    I + A_j estimated in loop j.  Since V_j^T V_j = I, P'_j^{-1} = I + V_j (Lt_j^{1/2} - I) V_j^T.

    Reading (the listing mixes variables here): the control v of x = x_b + L v stays in the
    unpreconditioned variable, so loop k solves for w with v = v_{k-1} + P_k w; its gradient is
    P_k^T (b + v_{k-1}), its Hessian I + A_k with A_k = P_k^T P_k - I + P_k^T A P_k, and the
    updates are v += P_k dw, x += L P_k dw.  At k = 1 (P_1 = I) this is the listing exactly.

    Rotation: U_k is an orthonormal basis of [P_1 V_1, ..., P_{k-1} V_{k-1}] (taken here from an
    SVD, which Algorithm 3 names) and each sketch column becomes P_k^{-1} (I - U_k U_k^T) omega."""

    def __init__(self, n):
        self.n = n
        self.V = []      # V_j, (n, m_j)
        self.lt = []     # Lt_j = lambda_j + 1, (m_j,)
        self.rot = []    # P_j V_j, the resolved directions in the control variable

    @property
    def count(self):
        return len(self.V)

    @staticmethod
    def _cols(X):
        X = np.array(X, dtype=np.float64, copy=True)
        return X[:, None] if X.ndim == 1 else X

    def _factor(self, X, j, power):
        V, lt = self.V[j], self.lt[j]
        return X + V @ ((lt ** power - 1.0)[:, None] * (V.T @ X))

    def apply(self, X):
        """P_k X = P'_0 (P'_1 (... (P'_{k-1} X)))."""
        X = self._cols(X)
        for j in reversed(range(self.count)):
            X = self._factor(X, j, -0.5)
        return X

    def apply_t(self, X):
        """P_k^T X = P'_{k-1} (... (P'_0 X)) (each P'_j is symmetric)."""
        X = self._cols(X)
        for j in range(self.count):
            X = self._factor(X, j, -0.5)
        return X

    def apply_inv(self, X):
        """P_k^{-1} X = P'_{k-1}^{-1} (... (P'_0^{-1} X))."""
        X = self._cols(X)
        for j in range(self.count):
            X = self._factor(X, j, 0.5)
        return X

    def push(self, lam, V):
        """Append P'_k from outer loop k's eigenpairs (lam of A_k, V orthonormal): the next
        loop runs with P_{k+1} = P_k P'_k.  P_k V is recorded for the rotation first."""
        lam = np.asarray(lam, dtype=np.float64)
        if np.any(lam + 1.0 <= 0.0):
            raise ValueError("eigenvalues of I + A_k must be positive")
        V = np.asarray(V, dtype=np.float64)
        self.rot.append(self.apply(V))
        self.V.append(V.copy())
        self.lt.append(lam + 1.0)

    def rotation_basis(self):
        """U_k: orthonormal basis of the span of [P_1 V_1, ..., P_{k-1} V_{k-1}]."""
        if not self.rot:
            return np.zeros((self.n, 0))
        X = np.hstack(self.rot)
        U, s, _ = np.linalg.svd(X, full_matrices=False)
        return U[:, s > s[0] * X.shape[1] * np.finfo(float).eps]

    def rotate(self, Omega):
        """Sketch columns restricted to the complement of the resolved directions and mapped
        to the preconditioned variable: P_k^{-1} (I - U_k U_k^T) Omega."""
        Ur = self.rotation_basis()
        Om = np.asarray(Omega, dtype=np.float64)
        return self.apply_inv(Om - Ur @ (Ur.T @ Om))

    def hessian(self, apply_a):
        """W -> A_k W = P_k^T P_k W - W + P_k^T A (P_k W) (Algorithm 3), apply_a: W -> A W."""
        def op(W):
            PW = self.apply(W)
            return self.apply_t(PW) - W + self.apply_t(apply_a(PW))
        return op


def outer_step_precond(prob, x, v, Omega, pc, q=0, exact_rr=False, rotation=False):
    """One cycle of Algorithm 3 with precond = true (rotation as given), with P_k held by pc
    (the caller pushes this loop's eigenpairs afterwards, which forms P'_k for the next loop).
    Returns the entries of outer_step plus dw (the increment of the preconditioned variable)."""
    traj = trajectory(prob, x)
    d = innovation(prob, traj)
    J = cost(prob, traj, v)
    b = gradient_b(prob, traj, d)
    g = pc.apply_t(b + v)[:, 0]
    Om = pc.rotate(Omega) if (rotation and pc.count) else np.asarray(Omega, dtype=np.float64)
    op = pc.hessian(lambda W: hvp(prob, traj, W))
    lam, U, info = rsvd(prob, traj, Om, q=q, exact_rr=exact_rr, apply=op)
    dw, mode = increment(lam, U, g)
    dv = pc.apply(dw)[:, 0]
    info["Omega"] = Om
    return {"traj": traj, "J": J, "b": b, "g": g, "lam": lam, "U": U, "dw": dw, "dv": dv, "mode": mode,
            "x_next": x + prob.L @ dv, "v_next": v + dv, "info": info}


# --- RIOT-PSAS: the observation-space dual (Appendix, Algorithm 4) --------------------------

def dual_hvp(prob, traj, W):
    """A_dual W = L_{R^-1} H B H^T L_{R^-1}^T W for the columns of W (p, m) (Algorithm 4), with
    R = diag(sigma_o^2) so L_{R^-1} = diag(1 / sigma_o), and B = L L^T: per column one adjoint
    integration from the observation-space forcing, L L^T, one tangent-linear integration."""
    W = np.atleast_2d(np.asarray(W, dtype=np.float64).T).T
    s = 1.0 / prob.sigma_o
    out = np.empty_like(W)
    for j in range(W.shape[1]):
        lam0 = l96.ad(traj, obs_forcing(prob, s * W[:, j]), prob.dt, prob.F)
        z = prob.L @ (prob.L.T @ lam0)
        out[:, j] = s * observe(prob, l96.tl(traj, z, prob.dt, prob.F))
    return out


def psas_weights(lam, U, sigma_o, d, bprime):
    """Adaptive observation-space weights of Algorithm 4 with S = L_{R^-1} = diag(1 / sigma_o):
        lambda_m > 1: dw = S U diag(1/(1+lambda)) U^T S (d - b')              (LRA, mode 0)
        otherwise:    dw = S (I - U diag(lambda/(1+lambda)) U^T) S (d - b')   (LRU, mode 1)."""
    s = 1.0 / sigma_o
    r = s * (d - bprime)
    c = U.T @ r
    if lam[-1] > 1.0:
        return s * (U @ (c / (1.0 + lam))), 0
    return s * (r - U @ (c * lam / (1.0 + lam))), 1


def psas_outer_step(prob, x, Omega, q=0, exact_rr=False):
    """One cycle of Algorithm 4 (RIOT-PSAS).  d = y - H(x_{k-1}) (the dual's sign),
    b' = H_{k-1}(x_b - x_{k-1}) (tangent linear), the randomized eigendecomposition of A_dual
    (p x p) on the sketch Omega (p, m) exactly as in Algorithm 3 (K Q^T Omega = Q^T Y, or
    K = Q^T A Q), and the adaptive weights of psas_weights.
    Reading: the state is x_k = x_b + B H^T dw.  Linearised about x_{k-1}, the minimiser of the
    cost is x_b + B H^T (H B H^T + R)^-1 (d - b'); the listing's x_{k-1} + B H^T dw adds
    x_{k-1} - x_b twice from the second loop on (both agree at k = 1, where x_0 = x_b).
    Returns a dict with J (at x), d, bprime, lam, U, dw, mode, x_next."""
    traj = trajectory(prob, x)
    d = prob.y - observe(prob, traj)
    J = 0.5 * float(np.sum(d * d * prob.rinv))
    vb = np.linalg.solve(prob.L, x - prob.x_b)
    J += 0.5 * float(vb @ vb)
    bprime = observe(prob, l96.tl(traj, prob.x_b - x, prob.dt, prob.F))
    lam, U, info = rsvd(prob, traj, Omega, q=q, exact_rr=exact_rr, apply=lambda W: dual_hvp(prob, traj, W))
    dw, mode = psas_weights(lam, U, prob.sigma_o, d, bprime)
    lam0 = l96.ad(traj, obs_forcing(prob, dw), prob.dt, prob.F)
    x_next = prob.x_b + prob.L @ (prob.L.T @ lam0)
    return {"traj": traj, "J": J, "d": d, "bprime": bprime, "lam": lam, "U": U, "dw": dw, "mode": mode,
            "x_next": x_next, "info": info}


def quadratic_cost(prob, traj, d, v, dv):
    """Inner-loop quadratic cost J~(dv) = 1/2||R^-1/2(d + H M L dv)||^2 + 1/2||v + dv||^2
    (Eq. 3 with Algorithm 3's sign of d and accumulated control v)."""
    dxs = l96.tl(traj, prob.L @ dv, prob.dt, prob.F)
    r = d + observe(prob, dxs)
    return 0.5 * float(np.sum(r * r * prob.rinv)) + 0.5 * float(np.dot(v + dv, v + dv))
