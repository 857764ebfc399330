"""FP64 CPU oracle for coupled nonnegative CP decomposition by alternating
proximal gradient (CoNCPD-APG) and its low-rank-approximation variant
(lraCoNCPD-APG), arXiv 2302.05119.

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain reference that the
CUDA path is checked against.  Only the test-suite, the smoke check and the
CPU-baseline leg of the benchmark may import it; the library never does.

Everything here is written from the paper's definitions in float64 with
numpy: tensors are numpy arrays of shape (I_1, ..., I_N); factor matrices are
(I_n, R) arrays; a "block" is one of the K (the paper's S) coupled tensors.
Library primitives (matmul, eigvalsh, Cholesky) serve as single steps; there
is no blocking, fusion or reordering beyond what the paper states.

Notation (paper Table I): mode-n unfolding X_(n) follows Kolda's convention
(the remaining indices ordered with the lowest mode varying fastest);
U^{(.)odot} = U^(N) (.) ... (.) U^(1) is the Khatri-Rao product in that order,
and U^{odot_-n} omits mode n.

Readings of points where the paper is silent or garbled (each also listed in
the design notes):
  R1  momentum: hat w_{k-1} = (t_{k-1} - 1) / t_k with t_0 = 1 (Appendix A,
      Eq. eqextrawu), so the first iteration extrapolates with weight 0.
  R2  first iteration: U_{k-2} := U_{k-1} and the ratio L_{k-2}/L_{k-1} := 1.
  R3  the shared part U_C^(n) is extrapolated once, with weight
      w_C = min(hat w, delta_w sqrt(sum_k L_prev / sum_k L)).
  R4  the step for U_C^(n) is 1 / sum_k L_u^(n,k) (Eq. solUnC).
  R5  L is the exact largest eigenvalue of the PSD matrix H; L == 0 means
      the corresponding update is skipped (U left unchanged).
  R6  modes are updated in order (Gauss-Seidel); within one mode every block
      sees the state before that mode's update (Jacobi across blocks).
  R7  re-update (Algorithm 1, safeguard): when F(k) >= F(k-1) the whole sweep
      is redone from the iteration's start with every extrapolation weight 0;
      t is not reset; F is recomputed; there is no second check.
  R8  a tie |F(k) - F(k-1)| <= 1e-13 F(k-1) counts as "not increased".
  R9  no column normalisation anywhere.
  R10 the core tensor D^(s) is optional (use_core); without it lambda == 1.
  R11 any LRA rank R_tilde is allowed (Eq. eqlrau holds for any R_tilde).
  R12 the step-2 (LRA) objective, safeguard and stopping test use the
      approximation X_tilde = [[U_tilde]] (Eq. cosfunclra); the reported
      global Fit uses the original tensors.
  R13 ALS for the LRA solves U_tilde^(n) = M V^{-1} by Cholesky; a matrix V
      that is not positive definite is an error (no silent regularisation).
"""

import math

import numpy as np
import scipy.linalg

TIE_TOL = 1e-13


# ---------------------------------------------------------------- Table I ---

def unfold(X, n):
    """Mode-n matricization X_(n) (Table I, Kolda ordering).

    Element (i_1, ..., i_N) lands at row i_n, column
    sum_{k != n} i_k * prod_{m < k, m != n} I_m.
    """
    X = np.asarray(X)
    return np.reshape(np.moveaxis(X, n, 0), (X.shape[n], -1), order="F")


def fold(Xn, n, shape):
    """Inverse of :func:`unfold`."""
    shape = tuple(shape)
    rest = tuple(s for m, s in enumerate(shape) if m != n)
    T = np.reshape(Xn, (shape[n],) + rest, order="F")
    return np.moveaxis(T, 0, n)


def khatri_rao(mats):
    """Column-wise Kronecker product A (.) B (.) ... (Table I).

    The row index of A (.) B is i_A * I_B + i_B (the last factor varies
    fastest), so khatri_rao([U^(N), ..., U^(1)]) matches :func:`unfold`.
    """
    mats = [np.asarray(M, dtype=np.float64) for M in mats]
    R = mats[0].shape[1]
    out = mats[0]
    for M in mats[1:]:
        assert M.shape[1] == R
        out = np.einsum("ir,jr->ijr", out, M).reshape(-1, R)
    return out


def kr_all(U):
    """U^{(.)odot} = U^(N) (.) ... (.) U^(1) (Table I)."""
    return khatri_rao(list(reversed(U)))


def kr_except(U, n):
    """U^{odot_-n}: the Khatri-Rao product of all factors but mode n, in the
    order U^(N) (.) ... (.) U^(n+1) (.) U^(n-1) (.) ... (.) U^(1) (Table I)."""
    return khatri_rao([U[m] for m in reversed(range(len(U))) if m != n])


def gram(U):
    """U^T U (Table II, operation 1)."""
    U = np.asarray(U, dtype=np.float64)
    return U.T @ U


def hadamard(mats):
    """Element-wise product of a list of equal-shape matrices (Table I)."""
    out = np.array(mats[0], dtype=np.float64, copy=True)
    for M in mats[1:]:
        out = out * M
    return out


def hadamard_except(grams, n):
    """(U^T U)^{circledast_-n}: Hadamard product of all Grams but mode n
    (Table I; Table II operation 4)."""
    return hadamard([G for m, G in enumerate(grams) if m != n])


# ------------------------------------------------ model and objective ----

def mttkrp(X, U, n):
    """X_(n) U^{odot_-n} (Eq. solapgU; Table II operations 6 and 7).

    Written as the explicit unfolding times the explicit Khatri-Rao matrix,
    exactly as the paper states the product.
    """
    return unfold(X, n) @ kr_except(U, n)


def kruskal(lam, U):
    """[[D; U^(1), ..., U^(N)]] with D super-diagonal holding lam
    (Eq. tensormodel).  Built as the mode-1 unfolding U^(1) D (U^{odot_-1})^T
    and folded back."""
    U = [np.asarray(A, dtype=np.float64) for A in U]
    shape = tuple(A.shape[0] for A in U)
    lam = np.asarray(lam, dtype=np.float64)
    X1 = (U[0] * lam[None, :]) @ kr_except(U, 0).T
    return fold(X1, 0, shape)


def objective(Xs, Us, lams):
    """F = 1/2 sum_k ||X^(k) - [[D^(k); U^(.,k)]]||_F^2 (Eq. costfunc),
    by explicit reconstruction."""
    F = 0.0
    for X, U, lam in zip(Xs, Us, lams):
        E = np.asarray(X, dtype=np.float64) - kruskal(lam, U)
        F += 0.5 * float(np.sum(E * E))
    return F


def block_relerrs(Xs, Us, lams):
    """||X^(k) - X_hat^(k)||_F / ||X^(k)||_F per block (termination criteria,
    Section III-C)."""
    out = []
    for X, U, lam in zip(Xs, Us, lams):
        X = np.asarray(X, dtype=np.float64)
        out.append(float(np.linalg.norm(X - kruskal(lam, U)) / np.linalg.norm(X)))
    return out


def relerr(Xs, Us, lams):
    """RelErr = (1/S) sum_s ||M^(s) - M_hat^(s)||_F / ||M^(s)||_F (Section
    III-C, termination criteria)."""
    return float(np.mean(block_relerrs(Xs, Us, lams)))


def fit(Xs, Us, lams):
    """Fit = (1/S) sum_s [1 - ||M - M_hat||_F / ||M||_F] (Section IV,
    experiment settings)."""
    return 1.0 - relerr(Xs, Us, lams)


def core_term(X, U):
    """(U^{(.)odot})^T vec(X) (Eq. solapgG; Table II operations 2 and 3),
    with vec() in the same column-major order as the unfolding."""
    vecX = np.reshape(np.asarray(X, dtype=np.float64), (-1,), order="F")
    return kr_all(U).T @ vecX


def spectral_norm(H):
    """||H||_2 of a symmetric positive semi-definite matrix = its largest
    eigenvalue (Eqs. eqLipsLd and eqLipsLu)."""
    H = np.asarray(H, dtype=np.float64)
    if H.size == 0:
        return 0.0
    return float(max(np.linalg.eigvalsh(0.5 * (H + H.T))[-1], 0.0))


# ------------------------------------------------------- APG parameters ----

def t_next(t):
    """t_k = (1 + sqrt(1 + 4 t_{k-1}^2)) / 2 (Appendix A, parameter
    settings)."""
    return 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))


def extrapolation_weight(w_hat, L_prev, L_cur, delta_w):
    """w = min(hat w, delta_w sqrt(L_{k-2} / L_{k-1})) (Eqs. eqextrawd,
    eqextrawu).  L_prev None (first iteration) reads as ratio 1 (R2)."""
    if L_cur <= 0.0:
        return 0.0
    ratio = 1.0 if L_prev is None else L_prev / L_cur
    return min(w_hat, delta_w * math.sqrt(ratio))


def project(A, nonneg):
    """P(.) of Section II-B: max(0, .) for a nonnegative mode, identity
    otherwise."""
    return np.maximum(A, 0.0) if nonneg else A


# ----------------------------------------------------------- the solver ----

class Problem:
    """K coupled N-th order tensors with ranks R_k and coupling counts L_n
    (Eq. tensormodel).  ``mttkrp_fn(k, U, n)`` returns X^(k)_(n) U^{odot_-n};
    ``core_fn(k, U)`` returns (U^{(.)odot})^T vec(X^(k)); ``objective_fn`` and
    ``relerr_fn`` evaluate Eq. costfunc / RelErr on the current factors.  The
    plain method reads the tensors; the LRA method replaces these four by the
    collapsed forms of Eqs. eqlrag and eqlrau on X_tilde = [[U_tilde]]."""

    def __init__(self, Xs, R, L, nonneg=None):
        self.Xs = [np.asarray(X, dtype=np.float64) for X in Xs]
        self.K = len(self.Xs)
        self.N = self.Xs[0].ndim
        self.R = [int(r) for r in (R if np.ndim(R) else [R] * self.K)]
        self.L = [int(x) for x in L]
        self.nonneg = [True] * self.N if nonneg is None else [bool(b) for b in nonneg]
        assert len(self.L) == self.N and len(self.R) == self.K
        for n in range(self.N):
            assert 0 <= self.L[n] <= min(self.R), "L_n must be <= min_k R_k"
            if self.L[n] > 0:
                assert len({X.shape[n] for X in self.Xs}) == 1, "coupled mode sizes differ"

    def mttkrp_fn(self, k, U, n):
        return mttkrp(self.Xs[k], U, n)

    def core_fn(self, k, U):
        return core_term(self.Xs[k], U)

    def objective_fn(self, Us, lams):
        return objective(self.Xs, Us, lams)

    def relerr_fn(self, Us, lams):
        return relerr(self.Xs, Us, lams)


class LRAProblem(Problem):
    """Step 2 of lraCoNCPD-APG (Algorithm 2): the tensors are replaced by
    their low-rank approximations X_tilde^(k) = [[U_tilde^(.,k)]]."""

    def __init__(self, Uts, R, L, nonneg=None):
        self.Uts = [[np.asarray(A, dtype=np.float64) for A in Ut] for Ut in Uts]
        Xts = [kruskal(np.ones(Ut[0].shape[1]), Ut) for Ut in self.Uts]
        super().__init__(Xts, R, L, nonneg)

    def mttkrp_fn(self, k, U, n):
        return collapsed_mttkrp(self.Uts[k], U, n)

    def core_fn(self, k, U):
        return collapsed_core_term(self.Uts[k], U)


def collapsed_mttkrp(Ut, U, n):
    """M_(n) U^{odot_-n} = U_tilde^(n) (U_tilde^T U)^{circledast_-n}
    (Eq. eqlrau; Table II operations 9 and 10)."""
    C = [np.asarray(Ut[m], dtype=np.float64).T @ np.asarray(U[m], dtype=np.float64)
         for m in range(len(U))]
    return np.asarray(Ut[n], dtype=np.float64) @ hadamard_except(C, n)


def collapsed_core_term(Ut, U):
    """(U^{(.)odot})^T vec(M) = (U^T U_tilde)^{circledast} ddiag(I)
    (Eq. eqlrag; Table II operation 8)."""
    C = [np.asarray(U[m], dtype=np.float64).T @ np.asarray(Ut[m], dtype=np.float64)
         for m in range(len(U))]
    return hadamard(C) @ np.ones(C[0].shape[1])


class State:
    """Current and previous iterates of every factor and core."""

    def __init__(self, U1, U2, lam1, lam2):
        self.U1, self.U2, self.lam1, self.lam2 = U1, U2, lam1, lam2

    def copy(self):
        return State([[A.copy() for A in U] for U in self.U1],
                     [[A.copy() for A in U] for U in self.U2],
                     [l.copy() for l in self.lam1], [l.copy() for l in self.lam2])


def sweep(prob, st, w_hat, Lprev, use_core, delta_w):
    """One pass of Algorithm 1's inner loops: the cores D^(1..S), then
    U^(1,1..S), ..., U^(N,1..S), each by one proximal-gradient step from an
    extrapolated point.  Returns the new state and the Lipschitz constants
    used (they become L_{k-2} of the next iteration)."""
    st = st.copy()
    K, N = prob.K, prob.N
    Lnew = {}

    if use_core:
        for k in range(K):
            U = st.U1[k]
            Hd = hadamard([gram(A) for A in U])                      # Eq. solapgG
            Ld = spectral_norm(Hd)                                   # Eq. eqLipsLd
            Lnew[("d", k)] = Ld
            if Ld <= 0.0:
                continue
            w = extrapolation_weight(w_hat, Lprev.get(("d", k)), Ld, delta_w)   # Eq. eqextrawd
            lam_hat = st.lam1[k] + w * (st.lam1[k] - st.lam2[k])     # Eq. eqextraPG
            g = Hd @ lam_hat - prob.core_fn(k, U)                    # Eq. solapgG
            st.lam2[k] = st.lam1[k]
            st.lam1[k] = np.maximum(0.0, lam_hat - g / Ld)           # Eq. solD

    for n in range(N):
        Ln = prob.L[n]
        H, M, Lu, w = [], [], [], []
        for k in range(K):
            U, lam = st.U1[k], st.lam1[k]
            D = np.diag(lam)
            Hk = D @ hadamard_except([gram(A) for A in U], n) @ D    # Eq. solapgU, first term
            Mk = prob.mttkrp_fn(k, U, n) @ D                          # Eq. solapgU, second term
            Lk = spectral_norm(Hk)                                   # Eq. eqLipsLu
            H.append(Hk)
            M.append(Mk)
            Lu.append(Lk)
            Lnew[("u", n, k)] = Lk
            w.append(extrapolation_weight(w_hat, Lprev.get(("u", n, k)), Lk, delta_w))

        U1n = [st.U1[k][n] for k in range(K)]
        U2n = [st.U2[k][n] for k in range(K)]
        Uhat = [U1n[k] + w[k] * (U1n[k] - U2n[k]) for k in range(K)]   # Eq. eqextraPU
        LC = float(sum(Lu))
        Lnew[("c", n)] = LC
        if Ln > 0:
            wC = extrapolation_weight(w_hat, Lprev.get(("c", n)), LC, delta_w)   # reading R3
            UC1, UC2 = U1n[0][:, :Ln], U2n[0][:, :Ln]
            UhatC = UC1 + wC * (UC1 - UC2)
            for k in range(K):
                Uhat[k][:, :Ln] = UhatC
        Ghat = [Uhat[k] @ H[k] - M[k] for k in range(K)]              # Eq. solapgU

        new = [U1n[k].copy() for k in range(K)]
        for k in range(K):
            if Lu[k] > 0.0:                                          # Eq. solUnsI / solUns
                new[k][:, Ln:] = project(Uhat[k][:, Ln:] - Ghat[k][:, Ln:] / Lu[k], prob.nonneg[n])
        if Ln > 0 and LC > 0.0:                                      # Eq. solUnC
            GC = sum(Ghat[k][:, :Ln] for k in range(K))
            newC = project(UhatC - GC / LC, prob.nonneg[n])
            for k in range(K):
                new[k][:, :Ln] = newC
        for k in range(K):
            st.U2[k][n] = U1n[k]
            st.U1[k][n] = new[k]
    return st, Lnew


def couple_initial(prob, U0):
    """Copy each block's initial factors, taking the shared first L_n columns
    from block 0 (Eq. tensormodel: U_C^(n,1) = ... = U_C^(n,S))."""
    U = [[np.array(A, dtype=np.float64, copy=True) for A in Uk] for Uk in U0]
    for n in range(prob.N):
        Ln = prob.L[n]
        if Ln > 0:
            for k in range(1, prob.K):
                U[k][n][:, :Ln] = U[0][n][:, :Ln]
    return U


def apg(prob, U0, lam0=None, use_core=False, max_it=1000, eps=1e-8,
        delta_w=0.9999, reupdate=True, callback=None):
    """CoNCPD-APG (Algorithm 1) on ``prob``; with an :class:`LRAProblem` it is
    step 2 of lraCoNCPD-APG (Algorithm 2).

    Returns a dict with the final factors U[k][n], cores lam[k], the
    iteration count, the re-update flags per iteration and the F / RelErr
    history.  ``callback(it, state, info)`` sees every accepted iterate.
    """
    K = prob.K
    U = couple_initial(prob, U0)
    if lam0 is None or not use_core:
        lam = [np.ones(prob.R[k]) for k in range(K)]
    else:
        lam = [np.array(l, dtype=np.float64, copy=True) for l in lam0]
    st = State(U, [[A.copy() for A in Uk] for Uk in U], lam, [l.copy() for l in lam])
    F_prev = prob.objective_fn(st.U1, st.lam1)
    rel_prev = prob.relerr_fn(st.U1, st.lam1)
    hist = {"F": [F_prev], "relerr": [rel_prev], "redo": []}
    t = 1.0
    Lprev = {}
    it = 0
    for it in range(1, max_it + 1):
        t_new = t_next(t)
        w_hat = (t - 1.0) / t_new                                     # reading R1
        cand, Lc = sweep(prob, st, w_hat, Lprev, use_core, delta_w)
        F = prob.objective_fn(cand.U1, cand.lam1)
        redo = bool(reupdate and (F - F_prev) > TIE_TOL * abs(F_prev))   # Algorithm 1 safeguard, R8
        if redo:
            cand, Lc = sweep(prob, st, 0.0, Lprev, use_core, delta_w)    # reading R7
            F = prob.objective_fn(cand.U1, cand.lam1)
        st, Lprev = cand, Lc
        rel = prob.relerr_fn(st.U1, st.lam1)
        hist["F"].append(F)
        hist["relerr"].append(rel)
        hist["redo"].append(redo)
        if callback is not None:
            callback(it, st, {"F": F, "relerr": rel, "redo": redo, "w_hat": w_hat})
        t, F_prev = t_new, F
        if abs(rel - rel_prev) < eps:                                 # termination criteria
            break
        rel_prev = rel
    return {"U": st.U1, "lam": st.lam1, "iters": it, "hist": hist, "state": st}


# ------------------------------------------------------ LRA step (i) -------

def als_cpd(X, Ut0, max_it=200, eps=1e-4):
    """Unconstrained rank-R_tilde CPD of one tensor by alternating least
    squares (Section III-B step (i); ALS as named in Section IV settings).

    Each sweep solves U_tilde^(n) = X_(n) U_tilde^{odot_-n} V^{-1} with
    V = (U_tilde^T U_tilde)^{circledast_-n}, modes in order; it stops when
    the relative error changes by less than eps (Section III-C).
    Returns (factors, sweeps, relerr history).
    """
    X = np.asarray(X, dtype=np.float64)
    Ut = [np.array(A, dtype=np.float64, copy=True) for A in Ut0]
    N = X.ndim
    nX = float(np.linalg.norm(X))
    ones = np.ones(Ut[0].shape[1])
    rel_prev = float(np.linalg.norm(X - kruskal(ones, Ut)) / nX)
    hist = [rel_prev]
    s = 0
    for s in range(1, max_it + 1):
        for n in range(N):
            V = hadamard_except([gram(A) for A in Ut], n)
            M = mttkrp(X, Ut, n)
            try:
                c = scipy.linalg.cho_factor(V, lower=True)
            except np.linalg.LinAlgError as e:
                raise np.linalg.LinAlgError(f"ALS normal matrix not positive definite (mode {n})") from e
            Ut[n] = scipy.linalg.cho_solve(c, M.T).T
        rel = float(np.linalg.norm(X - kruskal(ones, Ut)) / nX)
        hist.append(rel)
        if abs(rel - rel_prev) < eps:
            break
        rel_prev = rel
    return Ut, s, hist


def lra_apg(Xs, Ut0s, R, L, U0, nonneg=None, lam0=None, use_core=False,
            lra_max_it=200, lra_eps=1e-4, max_it=1000, eps=1e-8, delta_w=0.9999,
            reupdate=True, callback=None):
    """lraCoNCPD-APG (Algorithm 2): (i) ALS low-rank approximation of each
    tensor in turn, (ii) CoNCPD-APG on the approximations with the collapsed
    products of Eqs. eqlrag and eqlrau.  The returned ``global_fit`` is
    measured against the original tensors."""
    Uts, sweeps = [], []
    for X, Ut0 in zip(Xs, Ut0s):
        Ut, s, _ = als_cpd(X, Ut0, lra_max_it, lra_eps)
        Uts.append(Ut)
        sweeps.append(s)
    prob = LRAProblem(Uts, R, L, nonneg)
    res = apg(prob, U0, lam0, use_core, max_it, eps, delta_w, reupdate, callback)
    res["Ut"] = Uts
    res["als_sweeps"] = sweeps
    res["global_fit"] = fit(Xs, res["U"], res["lam"])
    return res


# ------------------------------------------------------------- metrics ------

def performance_index(U_est, U_true):
    """PI of Section IV (experiment settings): G = U_est^+ U_true, then the
    row- and column-normalised sums of |g_ij| / max_k |g_ik| minus one per row
    or column, divided by 2R(R-1).  0 for a scaled permutation.  (The printed
    formula's garbled summation index is read as the standard form.)"""
    G = np.abs(np.linalg.pinv(np.asarray(U_est, dtype=np.float64)) @ np.asarray(U_true, dtype=np.float64))
    R = G.shape[0]
    if R < 2:
        return 0.0
    rows = np.sum(G / np.max(G, axis=1, keepdims=True), axis=1) - 1.0
    cols = np.sum(G / np.max(G, axis=0, keepdims=True), axis=0) - 1.0
    return float((np.sum(rows) + np.sum(cols)) / (2.0 * R * (R - 1)))


def gradient(prob, U, lam, k, n):
    """Block-partial gradient of Eq. costfunc with respect to U^(n,k) at U
    (no extrapolation): U D (U^T U)^{circledast_-n} D - X_(n) U^{odot_-n} D
    (Eq. solbpgU in Appendix A)."""
    D = np.diag(lam[k])
    H = D @ hadamard_except([gram(A) for A in U[k]], n) @ D
    return U[k][n] @ H - prob.mttkrp_fn(k, U[k], n) @ D
