"""Pins of the FP64 oracle against things other than itself: brute-force sums
on tiny tensors, closed forms, identities stated in the paper, finite
differences, exact recovery and invariants.  CPU only."""

import itertools
import math
import os

import numpy as np
import pytest
import scipy.optimize

from oracle import cncpd_oracle as O

RNG = np.random.default_rng(1234)


def _rand_tensor(shape, rng=RNG):
    return rng.standard_normal(shape)


def _rand_factors(shape, R, rng=RNG, nonneg=False):
    f = rng.random if nonneg else rng.standard_normal
    return [f((I, R)) for I in shape]


# ------------------------------------------------ Table I primitives --------

@pytest.mark.parametrize("shape", [(2, 3, 4), (3, 2, 4, 2), (1, 5, 3)])
def test_unfold_follows_kolda_index_rule(shape):
    """Table I: element (i_1..i_N) sits at column sum_{k!=n} i_k J_k with
    J_k = prod_{m<k, m!=n} I_m (lowest remaining mode fastest)."""
    X = _rand_tensor(shape)
    N = len(shape)
    for n in range(N):
        Xn = O.unfold(X, n)
        assert Xn.shape == (shape[n], X.size // shape[n])
        for idx in itertools.product(*[range(s) for s in shape]):
            col, J = 0, 1
            for k in range(N):
                if k == n:
                    continue
                col += idx[k] * J
                J *= shape[k]
            assert Xn[idx[n], col] == X[idx]
        np.testing.assert_array_equal(O.fold(Xn, n, shape), X)


def test_khatri_rao_is_columnwise_kronecker():
    A, B, C = RNG.standard_normal((3, 2)), RNG.standard_normal((4, 2)), RNG.standard_normal((2, 2))
    KR = O.khatri_rao([A, B, C])
    for r in range(2):
        np.testing.assert_allclose(KR[:, r], np.kron(np.kron(A[:, r], B[:, r]), C[:, r]), rtol=0, atol=1e-15)


def _mttkrp_brute(X, U, n):
    """sum over every index of X[i] * prod_{m != n} U^(m)[i_m, r]."""
    R = U[0].shape[1]
    M = np.zeros((X.shape[n], R))
    for idx in itertools.product(*[range(s) for s in X.shape]):
        for r in range(R):
            p = X[idx]
            for m in range(X.ndim):
                if m != n:
                    p *= U[m][idx[m], r]
            M[idx[n], r] += p
    return M


@pytest.mark.parametrize("shape,R", [((2, 3, 4), 1), ((3, 1, 5), 3), ((4, 3, 2, 3), 2),
                                     ((2, 2, 3, 2), 4), ((5, 4, 3), 6), ((1, 1, 1), 2)])
def test_mttkrp_matches_brute_force(shape, R):
    """Eq. solapgU second term X_(n) U^{odot_-n} versus brute-force loops."""
    X = _rand_tensor(shape)
    U = _rand_factors(shape, R)
    for n in range(len(shape)):
        np.testing.assert_allclose(O.mttkrp(X, U, n), _mttkrp_brute(X, U, n), rtol=0, atol=1e-13)


@pytest.mark.parametrize("shape,R", [((3, 4, 5), 3), ((2, 3, 2, 4), 4)])
def test_khatri_rao_gram_identity(shape, R):
    """Appendix A: (U^{odot_-n})^T U^{odot_-n} = (U^T U)^{circledast_-n},
    and the same for the full product."""
    U = _rand_factors(shape, R)
    G = [O.gram(A) for A in U]
    for n in range(len(shape)):
        KR = O.kr_except(U, n)
        np.testing.assert_allclose(KR.T @ KR, O.hadamard_except(G, n), rtol=1e-13, atol=1e-13)
    KR = O.kr_all(U)
    np.testing.assert_allclose(KR.T @ KR, O.hadamard(G), rtol=1e-13, atol=1e-13)


def test_kruskal_and_core_term_match_brute_force():
    shape, R = (3, 4, 2), 3
    U = _rand_factors(shape, R)
    lam = RNG.random(R)
    X = np.zeros(shape)
    for idx in itertools.product(*[range(s) for s in shape]):
        X[idx] = sum(lam[r] * U[0][idx[0], r] * U[1][idx[1], r] * U[2][idx[2], r] for r in range(R))
    np.testing.assert_allclose(O.kruskal(lam, U), X, rtol=0, atol=1e-14)
    Y = _rand_tensor(shape)
    c = np.zeros(R)
    for idx in itertools.product(*[range(s) for s in shape]):
        for r in range(R):
            c[r] += Y[idx] * U[0][idx[0], r] * U[1][idx[1], r] * U[2][idx[2], r]
    np.testing.assert_allclose(O.core_term(Y, U), c, rtol=0, atol=1e-13)


def test_objective_brute_force_and_zero_at_exact_model():
    shape, R = (3, 2, 4), 2
    U = _rand_factors(shape, R, nonneg=True)
    lam = np.ones(R)
    X = O.kruskal(lam, U)
    assert O.objective([X], [U], [lam]) == pytest.approx(0.0, abs=1e-28)
    Y = X + 0.1
    F = 0.5 * sum((Y[idx] - X[idx]) ** 2 for idx in itertools.product(*[range(s) for s in shape]))
    assert O.objective([Y], [U], [lam]) == pytest.approx(F, rel=1e-13)


# ------------------------------------------------- Lipschitz constant -------

def test_spectral_norm_2x2_closed_form():
    for a, b, c in [(2.0, 1.0, 3.0), (1.0, 0.0, 1.0), (5.0, -2.0, 0.5), (1e-3, 1e-4, 2e-3)]:
        H = np.array([[a, b], [b, c]])
        lam = (a + c) / 2 + math.sqrt(((a - c) / 2) ** 2 + b * b)
        assert O.spectral_norm(H) == pytest.approx(lam, rel=1e-14)


def test_spectral_norm_vs_power_iteration():
    for R in (1, 3, 10, 30):
        A = RNG.random((50, R))
        H = A.T @ A
        v = np.ones(R)
        for _ in range(5000):
            v = H @ v
            v /= np.linalg.norm(v)
        assert O.spectral_norm(H) == pytest.approx(float(v @ H @ v), rel=1e-12)
    assert O.spectral_norm(np.zeros((4, 4))) == 0.0


# ------------------------------------------------------- momentum ----------

def test_momentum_weights_closed_form(root):
    sympy = pytest.importorskip("sympy")
    table = {}
    with open(os.path.join(root, "tests", "golden", "momentum_closed_form.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, expr = line.split(None, 1)
                table[name] = float(sympy.N(sympy.sympify(expr), 30))
    t0 = 1.0
    t1 = O.t_next(t0)
    t2 = O.t_next(t1)
    t3 = O.t_next(t2)
    assert t1 == pytest.approx(table["t1"], rel=1e-15)
    assert t2 == pytest.approx(table["t2"], rel=1e-15)
    assert (t0 - 1) / t1 == table["w1"]
    assert (t1 - 1) / t2 == pytest.approx(table["w2"], rel=1e-14)
    assert (t2 - 1) / t3 == pytest.approx(table["w3"], rel=1e-14)


def test_extrapolation_weight_cases():
    # first iteration: no L_{k-2}, ratio reads as 1
    assert O.extrapolation_weight(0.5, None, 3.0, 0.9999) == 0.5
    assert O.extrapolation_weight(0.99995, None, 3.0, 0.9999) == 0.9999
    # Lipschitz grew by 4: delta_w * sqrt(1/4)
    assert O.extrapolation_weight(0.9, 1.0, 4.0, 0.9999) == pytest.approx(0.49995)
    assert O.extrapolation_weight(0.3, 1.0, 4.0, 0.9999) == 0.3
    assert O.extrapolation_weight(0.3, 1.0, 0.0, 0.9999) == 0.0


# -------------------------------------------------------- one update -------

def test_single_rank1_step_is_exact_least_squares():
    """K=1, L=0, R=1, first iteration (w=0): H = ||u2||^2 ||u3||^2 equals L,
    so the projected-gradient step of Eq. solUns lands on max(0, X_(1) kr / H),
    the exact nonnegative least-squares minimiser in mode 1."""
    X = np.array([[[2.0]], [[-1.0]], [[4.0]]])           # 3 x 1 x 1
    u1 = np.array([[0.5], [0.5], [0.5]])
    u2 = np.array([[2.0]])
    u3 = np.array([[3.0]])
    prob = O.Problem([X], [1], [0, 0, 0])
    st = O.State([[u1, u2, u3]], [[u1.copy(), u2.copy(), u3.copy()]], [np.ones(1)], [np.ones(1)])
    new, L = O.sweep(prob, st, 0.0, {}, False, 0.9999)
    # mode 1 first: H = (2*2)(3*3) = 36, M = X * 6  ->  max(0, 6 X / 36)
    np.testing.assert_allclose(new.U2[0][0], u1)
    expect_u1 = np.maximum(0.0, X[:, 0, 0] / 6.0)[:, None]
    np.testing.assert_allclose(new.U1[0][0], expect_u1, rtol=1e-15)
    assert L[("u", 0, 0)] == pytest.approx(36.0)


def test_fixed_point_is_kept():
    """A KKT point of Eq. costfunc (the exact nonnegative model) is left
    unchanged by a w=0 sweep."""
    shape, R = (4, 5, 3), 2
    U = _rand_factors(shape, R, nonneg=True)
    X = O.kruskal(np.ones(R), U)
    prob = O.Problem([X], [R], [0, 0, 0])
    st = O.State([[A.copy() for A in U]], [[A.copy() for A in U]], [np.ones(R)], [np.ones(R)])
    new, _ = O.sweep(prob, st, 0.0, {}, False, 0.9999)
    for n in range(3):
        np.testing.assert_allclose(new.U1[0][n], U[n], rtol=1e-12, atol=1e-13)


# -------------------------------------------------- gradient vs FD ---------

def _coupled_problem(seed=7, dims=(12, 10, 8), K=2, R=3, L=(2, 1, 0), noise=0.05):
    rng = np.random.default_rng(seed)
    A = []
    common = [rng.random((dims[n], L[n])) for n in range(3)]
    for k in range(K):
        Ak = []
        for n in range(3):
            M = rng.random((dims[n], R))
            M[:, :L[n]] = common[n]
            Ak.append(M)
        A.append(Ak)
    Xs = [np.maximum(O.kruskal(np.ones(R), Ak) + noise * rng.standard_normal(dims), 0.0) for Ak in A]
    U0 = [[rng.random((dims[n], R)) for n in range(3)] for _ in range(K)]
    return Xs, A, U0, list(L)


@pytest.mark.parametrize("with_core", [False, True])
def test_gradient_matches_central_differences(with_core):
    """Eq. solbpgU: dF/dU^(n,k) = U D (U^T U)^{*-n} D - X_(n) U^{odot-n} D,
    against FP64 central differences with step 1e-6 on a 12x10x8 problem."""
    Xs, _, U0, L = _coupled_problem()
    prob = O.Problem(Xs, [3, 3], L)
    rng = np.random.default_rng(3)
    lam = [rng.random(3) + 0.5 for _ in range(2)] if with_core else [np.ones(3)] * 2
    h = 1e-6
    for k in range(2):
        for n in range(3):
            g = O.gradient(prob, U0, lam, k, n)
            fd = np.zeros_like(g)
            for i in range(g.shape[0]):
                for r in range(g.shape[1]):
                    Up = [[A.copy() for A in Uk] for Uk in U0]
                    Um = [[A.copy() for A in Uk] for Uk in U0]
                    Up[k][n][i, r] += h
                    Um[k][n][i, r] -= h
                    fd[i, r] = (prob.objective_fn(Up, lam) - prob.objective_fn(Um, lam)) / (2 * h)
            assert np.linalg.norm(g - fd) <= 1e-6 * np.linalg.norm(g)


def test_common_gradient_is_sum_of_block_gradients():
    """Appendix A: the gradient at the shared U_C^(n) is the first L_n
    columns of each block's gradient, summed over the blocks."""
    Xs, _, U0, L = _coupled_problem()
    prob = O.Problem(Xs, [3, 3], L)
    U = O.couple_initial(prob, U0)
    lam = [np.ones(3)] * 2
    h = 1e-6
    for n in (0, 1):
        Ln = L[n]
        gsum = sum(O.gradient(prob, U, lam, k, n)[:, :Ln] for k in range(2))
        fd = np.zeros_like(gsum)
        for i in range(gsum.shape[0]):
            for r in range(Ln):
                Up = [[A.copy() for A in Uk] for Uk in U]
                Um = [[A.copy() for A in Uk] for Uk in U]
                for k in range(2):
                    Up[k][n][i, r] += h
                    Um[k][n][i, r] -= h
                fd[i, r] = (prob.objective_fn(Up, lam) - prob.objective_fn(Um, lam)) / (2 * h)
        assert np.linalg.norm(gsum - fd) <= 1e-6 * np.linalg.norm(gsum)


# ----------------------------------------------------- whole solver --------

def _congruence(A_true, A_est):
    """Best-matched product over modes of column cosines (up to permutation
    and scaling)."""
    R = A_true[0].shape[1]
    C = np.ones((R, R))
    for At, Ae in zip(A_true, A_est):
        a = At / np.linalg.norm(At, axis=0, keepdims=True)
        e = Ae / np.maximum(np.linalg.norm(Ae, axis=0, keepdims=True), 1e-300)
        C *= a.T @ e
    rows, cols = scipy.optimize.linear_sum_assignment(-C)
    return float(np.min(C[rows, cols]))


def test_exact_recovery_noise_free():
    """Noise-free coupled tensors from known nonnegative factors: the fit
    tends to 1, every block's factors are recovered up to permutation and
    scaling (congruence >= 0.999), PI -> 0, and the shared columns are
    identical across blocks."""
    # (seed 2: a start that reaches the global optimum; other starts can stop
    # at a local stationary point, which the method does not exclude)
    Xs, A, U0, L = _coupled_problem(seed=2, dims=(10, 9, 8), K=3, R=3, L=(2, 1, 0), noise=0.0)
    prob = O.Problem(Xs, [3] * 3, L)
    res = O.apg(prob, U0, max_it=3000, eps=1e-13)
    f = O.fit(Xs, res["U"], res["lam"])
    assert f > 1 - 1e-5
    for k in range(3):
        assert _congruence(A[k], res["U"][k]) >= 0.999
        for n in range(3):
            assert O.performance_index(res["U"][k][n], A[k][n]) < 1e-2
    for n in range(3):
        for k in range(1, 3):
            np.testing.assert_array_equal(res["U"][k][n][:, :L[n]], res["U"][0][n][:, :L[n]])


def test_invariants_every_iteration():
    """U >= 0, the shared columns bit-identical across blocks, and
    F(k) <= F(k-1) on every re-updated (w=0) iteration."""
    Xs, _, U0, L = _coupled_problem(seed=5, K=3, noise=0.2)
    prob = O.Problem(Xs, [3] * 3, L)
    seen = {"redo": 0}
    F_hist = []

    def cb(it, st, info):
        F_hist.append(info["F"])
        for k in range(3):
            for n in range(3):
                assert np.all(st.U1[k][n] >= 0)
                np.testing.assert_array_equal(st.U1[k][n][:, :L[n]], st.U1[0][n][:, :L[n]])
        if info["redo"]:
            seen["redo"] += 1

    res = O.apg(prob, U0, max_it=300, eps=0.0, callback=cb)
    F = res["hist"]["F"]
    for i, redo in enumerate(res["hist"]["redo"]):
        if redo:
            assert F[i + 1] <= F[i] * (1 + 1e-12)
    # APG is not monotone: the safeguard must actually have fired here
    assert seen["redo"] > 0


def _coupled_grads(prob, U, lam, n, L):
    grads = [O.gradient(prob, U, lam, k, n) for k in range(prob.K)]
    out = []
    for k in range(prob.K):
        g = grads[k].copy()
        if L[n]:
            g[:, :L[n]] = sum(gg[:, :L[n]] for gg in grads)
        out.append(g)
    return out


def _projected_gradient_norm(prob, U, lam, L):
    """||min(U, grad F)||-style KKT residual: the gradient where U > 0 and
    its negative part where U == 0 (nonnegativity bound active)."""
    tot = 0.0
    for n in range(prob.N):
        for k, g in enumerate(_coupled_grads(prob, U, lam, n, L)):
            pg = np.where(U[k][n] > 0, g, np.minimum(g, 0.0))
            tot += float(np.sum(pg * pg))
    return math.sqrt(tot)


def test_kkt_complementarity_at_convergence():
    """At a stationary point of the constrained problem the KKT conditions
    hold: U >= 0, grad F >= 0 where U == 0, grad F == 0 where U > 0 (the
    common-column gradient being the block sum).  The projected-gradient
    residual must fall by 1e-6 from its value at the start, and
    ||U * grad|| / (||U|| ||grad_0||) must be tiny."""
    Xs, _, U0, L = _coupled_problem(seed=9, K=2, noise=0.05)
    prob = O.Problem(Xs, [3, 3], L)
    Uc = O.couple_initial(prob, U0)
    ones = [np.ones(3)] * 2
    pg0 = _projected_gradient_norm(prob, Uc, ones, L)
    res = O.apg(prob, U0, max_it=4000, eps=1e-14)
    U, lam = res["U"], res["lam"]
    assert _projected_gradient_norm(prob, U, lam, L) <= 1e-6 * pg0
    for n in range(3):
        for k, g in enumerate(_coupled_grads(prob, U, lam, n, L)):
            comp = np.linalg.norm(U[k][n] * g) / (np.linalg.norm(U[k][n]) * pg0)
            assert comp <= 1e-6


def test_with_core_reaches_fit_on_fully_coupled_case():
    """Fully coupled modes (all L_n > 0) need the cores (Section III-C);
    with use_core the solver still descends to a good fit on noise-free data
    whose blocks differ only by scaling."""
    rng = np.random.default_rng(21)
    dims, R = (8, 7, 6), 2
    common = [rng.random((d, R)) for d in dims]
    scales = [np.array([1.0, 2.0]), np.array([3.0, 0.5])]
    Xs = [O.kruskal(s, common) for s in scales]
    prob = O.Problem(Xs, [R, R], [R, R, R])
    U0 = [[rng.random((d, R)) for d in dims] for _ in range(2)]
    lam0 = [rng.random(R) for _ in range(2)]
    res_nc = O.apg(prob, U0, max_it=1500, eps=1e-14)
    res_c = O.apg(prob, U0, lam0, use_core=True, max_it=1500, eps=1e-14)
    f_nc = O.fit(Xs, res_nc["U"], res_nc["lam"])
    f_c = O.fit(Xs, res_c["U"], res_c["lam"])
    assert f_c > 0.999
    assert f_c > f_nc


# ---------------------------------------------------------------- LRA -----

def test_als_recovers_exact_low_rank():
    rng = np.random.default_rng(4)
    U = [rng.standard_normal((d, 3)) for d in (9, 8, 7)]
    X = O.kruskal(np.ones(3), U)
    Ut0 = [rng.random((d, 3)) for d in (9, 8, 7)]
    Ut, sweeps, hist = O.als_cpd(X, Ut0, max_it=2000, eps=1e-15)
    assert hist[-1] <= 1e-6


def test_collapsed_products_exact_for_low_rank_tensor():
    """Eqs. eqlrau and eqlrag are identities when X = [[U_tilde]] exactly."""
    rng = np.random.default_rng(6)
    for shape, Rt, R in [((5, 4, 6), 3, 2), ((3, 4, 2, 5), 4, 3), ((6, 5, 4), 2, 4)]:
        Ut = [rng.standard_normal((d, Rt)) for d in shape]
        U = [rng.random((d, R)) for d in shape]
        X = O.kruskal(np.ones(Rt), Ut)
        for n in range(len(shape)):
            a = O.collapsed_mttkrp(Ut, U, n)
            b = _mttkrp_brute(X, U, n) if np.prod(shape) <= 200 else O.mttkrp(X, U, n)
            np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12 * np.abs(b).max())
        np.testing.assert_allclose(O.collapsed_core_term(Ut, U), O.core_term(X, U), rtol=1e-12)


def test_proposition1_error_bound():
    """Proposition 1(ii): the NCP fitted to the LRA is within 2 theta of the
    best NCP of the original tensors, sum_s ||Y - [[U_lra]]|| <= sum_s
    (2 theta_s + eps_s), with eps_s taken from the plain solver."""
    Xs, _, U0, L = _coupled_problem(seed=13, K=2, noise=0.1)
    rng = np.random.default_rng(8)
    Ut0 = [[rng.random((d, 3)) for d in Xs[0].shape] for _ in range(2)]
    res_plain = O.apg(O.Problem(Xs, [3, 3], L), U0, max_it=3000, eps=1e-12)
    res_lra = O.lra_apg(Xs, Ut0, [3, 3], L, U0, lra_max_it=500, lra_eps=1e-12, max_it=3000, eps=1e-12)
    Xt = [O.kruskal(np.ones(3), Ut) for Ut in res_lra["Ut"]]
    theta = [np.linalg.norm(X - Y) for X, Y in zip(Xs, Xt)]
    eps_plain = [np.linalg.norm(X - O.kruskal(np.ones(3), U)) for X, U in zip(Xs, res_plain["U"])]
    err_lra = [np.linalg.norm(X - O.kruskal(np.ones(3), U)) for X, U in zip(Xs, res_lra["U"])]
    assert sum(err_lra) <= sum(2 * t + e for t, e in zip(theta, eps_plain)) + 1e-8
    assert sum(eps_plain) <= sum(err_lra) + 1e-6


# ------------------------------------------------------------ metrics -----

def test_performance_index():
    rng = np.random.default_rng(2)
    U = rng.random((20, 4))
    P = np.eye(4)[[2, 0, 3, 1]] * np.array([2.0, 0.5, 3.0, 1.5])
    assert O.performance_index(U @ P, U) == pytest.approx(0.0, abs=1e-12)
    # hand case: G = [[1, .5], [.25, 1]] -> rows (0.5 + 0.25), cols (0.25 + 0.5) over 2*2*1
    Ue = np.eye(2)
    Ut = np.array([[1.0, 0.5], [0.25, 1.0]])
    assert O.performance_index(Ue, Ut) == pytest.approx((0.75 + 0.75) / 4)


# ------------------------------------------------ planted mistakes -------

def test_planted_kr_order_mistake_is_caught(monkeypatch):
    """A transposed Khatri-Rao order must break the brute-force MTTKRP pin."""
    def wrong(U, n):
        return O.khatri_rao([U[m] for m in range(len(U)) if m != n])
    monkeypatch.setattr(O, "kr_except", wrong)
    X = _rand_tensor((2, 3, 4))
    U = _rand_factors((2, 3, 4), 2)
    assert not np.allclose(O.mttkrp(X, U, 0), _mttkrp_brute(X, U, 0))


def test_planted_hadamard_mistake_is_caught(monkeypatch):
    """Keeping mode n inside (U^T U)^{circledast_-n} must break the
    finite-difference gradient pin."""
    monkeypatch.setattr(O, "hadamard_except", lambda grams, n: O.hadamard(grams))
    with pytest.raises(AssertionError):
        test_gradient_matches_central_differences(False)


def test_planted_projection_mistake_is_caught(monkeypatch):
    """Dropping max(0, .) must break the nonnegativity invariant pin."""
    monkeypatch.setattr(O, "project", lambda A, nonneg: A)
    with pytest.raises(AssertionError):
        test_invariants_every_iteration()


def test_planted_core_term_mistake_is_caught(monkeypatch):
    """A transposed Khatri-Rao order in the core term must break its pin."""
    monkeypatch.setattr(O, "kr_all", lambda U: O.khatri_rao(list(U)))
    with pytest.raises(AssertionError):
        test_kruskal_and_core_term_match_brute_force()


# ------------------------- extrapolated coupled sweep (golden, w > 0) -----

def _golden_sweep(root):
    import json
    with open(os.path.join(root, "tests", "golden", "coupled_sweep.json")) as f:
        return json.load(f)


def _check_coupled_sweep(root, case_name):
    """One sweep with w_hat = 0.6 > 0 against the 50-digit elementwise
    computation in tests/golden/coupled_sweep.json (written by
    make_coupled_sweep.py from Eqs. eqextraPU, eqextrawu, solUnsI, solUnC and,
    with the core, eqextraPG / solD; reading R3 for the shared weight)."""
    g = _golden_sweep(root)
    case = g["cases"][case_name]
    K, N = g["K"], len(g["dims"])
    Xs = [np.array(X) for X in g["X"]]
    prob = O.Problem(Xs, [g["R"]] * K, g["L"])
    st = O.State([[np.array(A) for A in Uk] for Uk in g["U1"]], [[np.array(A) for A in Uk] for Uk in g["U2"]],
                 [np.array(l) for l in g["lam1"]], [np.array(l) for l in g["lam2"]])
    Lp = {}
    for n in range(N):
        for k in range(K):
            Lp[("u", n, k)] = case["Lprev"]["u"][n][k]
        if case["Lprev"]["c"][n] is not None:
            Lp[("c", n)] = case["Lprev"]["c"][n]
    if case["use_core"]:
        for k in range(K):
            Lp[("d", k)] = case["Lprev"]["d"][k]
    new, Lnew = O.sweep(prob, st, g["w_hat"], Lp, case["use_core"], g["delta_w"])
    ex = case["expect"]
    tr = ex["trace"]
    for n in range(N):
        for k in range(K):
            want = np.array(ex["U1"][k][n], dtype=np.float64)
            err = np.max(np.abs(new.U1[k][n] - want)) / np.max(np.abs(want))
            assert err <= 1e-13, (case_name, n, k, err)
            np.testing.assert_array_equal(new.U2[k][n], st.U1[k][n])
            assert Lnew[("u", n, k)] == pytest.approx(float(tr[f"L_{n}_{k}"]), rel=1e-13)
        assert Lnew[("c", n)] == pytest.approx(float(tr[f"LC_{n}"]), rel=1e-13)
    if case["use_core"]:
        for k in range(K):
            np.testing.assert_allclose(new.lam1[k], np.array(ex["lam1"][k], dtype=np.float64), rtol=1e-13)
            assert Lnew[("d", k)] == pytest.approx(float(tr[f"Ld_{k}"]), rel=1e-13)


@pytest.mark.parametrize("case_name", ["plain", "core"])
def test_extrapolated_coupled_sweep_matches_golden(root, case_name):
    _check_coupled_sweep(root, case_name)


def _planted(fn, old, new):
    """A copy of oracle function ``fn`` with one source fragment replaced."""
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(fn))
    assert src.count(old) == 1, old
    ns = dict(vars(O))
    exec(compile(src.replace(old, new), "<planted mistake>", "exec"), ns)
    return ns[fn.__name__]


@pytest.mark.parametrize("case_name,old,new", [
    # extrapolation sign of the individual columns (Eq. eqextraPU)
    ("plain", "U1n[k] + w[k] * (U1n[k] - U2n[k])", "U1n[k] - w[k] * (U1n[k] - U2n[k])"),
    # extrapolation sign of the shared columns
    ("plain", "UhatC = UC1 + wC * (UC1 - UC2)", "UhatC = UC1 - wC * (UC1 - UC2)"),
    # one block's weight in place of the shared weight w_C (reading R3)
    ("plain", "UhatC = UC1 + wC * (UC1 - UC2)", "UhatC = UC1 + w[0] * (UC1 - UC2)"),
    # w_C from one block's L history instead of the block sums
    ("plain", 'Lprev.get(("c", n))', 'Lprev.get(("u", n, 0))'),
    # one block's step instead of 1 / sum_k L (Eq. solUnC)
    ("plain", "newC = project(UhatC - GC / LC", "newC = project(UhatC - GC / Lu[0]"),
    # no momentum: the previous iterate read as the current one
    ("plain", "U2n = [st.U2[k][n] for k in range(K)]", "U2n = [st.U1[k][n] for k in range(K)]"),
    # the shared gradient from block 0 alone instead of the block sum
    ("plain", "GC = sum(Ghat[k][:, :Ln] for k in range(K))", "GC = Ghat[0][:, :Ln]"),
    # core extrapolation sign (Eq. eqextraPG)
    ("core", "st.lam1[k] + w * (st.lam1[k] - st.lam2[k])", "st.lam1[k] - w * (st.lam1[k] - st.lam2[k])"),
    # the core's weight from the factor history
    ("core", 'Lprev.get(("d", k))', 'Lprev.get(("u", 0, k))'),
])
def test_planted_sweep_mistakes_are_caught(root, monkeypatch, case_name, old, new):
    monkeypatch.setattr(O, "sweep", _planted(O.sweep, old, new))
    with pytest.raises(AssertionError):
        _check_coupled_sweep(root, case_name)


# ------------------------------------------------------ RelErr and Fit -----

def _relerr_case():
    """Two 2x2x2 blocks with rank-1 all-ones models (X_hat = 1 everywhere):
    block 0 is all ones but one entry 4 (residual 3, ||X||^2 = 7 + 16 = 23);
    block 1 is all twos (residual norm sqrt(8), ||X|| = sqrt(32))."""
    X0 = np.ones((2, 2, 2))
    X0[1, 0, 1] = 4.0
    X1 = 2.0 * np.ones((2, 2, 2))
    U = [np.ones((2, 1)) for _ in range(3)]
    return [X0, X1], [U, U], [np.ones(1), np.ones(1)]


def test_relerr_and_fit_hand_values():
    """RelErr = mean_k ||X - X_hat|| / ||X|| (Section III-C) and Fit = 1 -
    RelErr (Section IV) on hand-computed values: 3 / sqrt(23) and 1/2."""
    Xs, Us, lams = _relerr_case()
    per = O.block_relerrs(Xs, Us, lams)
    assert per[0] == pytest.approx(3.0 / math.sqrt(23.0), rel=1e-15)
    assert per[1] == pytest.approx(0.5, rel=1e-15)
    rel = (3.0 / math.sqrt(23.0) + 0.5) / 2.0
    assert O.relerr(Xs, Us, lams) == pytest.approx(rel, rel=1e-15)
    assert O.fit(Xs, Us, lams) == pytest.approx(1.0 - rel, rel=1e-15)


@pytest.mark.parametrize("fn,old,new", [
    ("block_relerrs", "np.linalg.norm(X - kruskal(lam, U)) / np.linalg.norm(X)",
     "np.linalg.norm(X - kruskal(lam, U)) ** 2 / np.linalg.norm(X) ** 2"),
    ("block_relerrs", "np.linalg.norm(X - kruskal(lam, U)) / np.linalg.norm(X)",
     "np.linalg.norm(X - kruskal(lam, U))"),
    ("relerr", "np.mean(block_relerrs(Xs, Us, lams))", "np.sum(block_relerrs(Xs, Us, lams))"),
])
def test_planted_relerr_mistakes_are_caught(monkeypatch, fn, old, new):
    monkeypatch.setattr(O, fn, _planted(getattr(O, fn), old, new))
    with pytest.raises(AssertionError):
        test_relerr_and_fit_hand_values()


# ------------------------------------------- termination and safeguard -----

def _stopping_case():
    Xs, _, U0, L = _coupled_problem(seed=11, K=2, noise=0.1)
    return O.Problem(Xs, [3, 3], L), U0


def test_stops_on_first_small_relerr_change():
    """Section III-C: the iteration stops at the first k with
    |RelErr_k - RelErr_{k-1}| < eps, and not before.  The change sequence is
    taken from an eps = 0 run; eps is placed between the first change that
    drops below all earlier ones (past iteration 15) and the smallest earlier
    change."""
    prob, U0 = _stopping_case()
    full = O.apg(prob, U0, max_it=80, eps=0.0)
    rel = full["hist"]["relerr"]
    d = [abs(rel[i] - rel[i - 1]) for i in range(1, len(rel))]
    stop = next(i for i in range(15, len(d)) if d[i] < min(d[:i]))
    eps = 0.5 * (d[stop] + min(d[:stop]))
    res = O.apg(prob, U0, max_it=80, eps=eps)
    assert res["iters"] == stop + 1
    assert res["hist"]["relerr"] == rel[:stop + 2]


def test_planted_stopping_mistake_is_caught(monkeypatch):
    """Comparing against the initial RelErr instead of the previous one."""
    monkeypatch.setattr(O, "apg", _planted(O.apg, "        rel_prev = rel\n", "        pass\n"))
    with pytest.raises(AssertionError):
        test_stops_on_first_small_relerr_change()


def test_momentum_sequence_in_apg(root):
    """The weights hat w the solver passes to its sweeps follow Appendix A
    (reading R1): 0, then (t_1 - 1)/t_2, (t_2 - 1)/t_3."""
    sympy = pytest.importorskip("sympy")
    table = {}
    with open(os.path.join(root, "tests", "golden", "momentum_closed_form.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, expr = line.split(None, 1)
                table[name] = float(sympy.N(sympy.sympify(expr), 30))
    prob, U0 = _stopping_case()
    seen = []
    O.apg(prob, U0, max_it=3, eps=0.0, reupdate=False, callback=lambda it, st, info: seen.append(info["w_hat"]))
    assert seen[0] == 0.0
    assert seen[1] == pytest.approx(table["w2"], rel=1e-14)
    assert seen[2] == pytest.approx(table["w3"], rel=1e-14)


def test_planted_momentum_mistake_is_caught(root, monkeypatch):
    monkeypatch.setattr(O, "apg", _planted(O.apg, "w_hat = (t - 1.0) / t_new", "w_hat = (t_new - 1.0) / t_new"))
    with pytest.raises(AssertionError):
        test_momentum_sequence_in_apg(root)


def test_safeguard_accepts_no_increase():
    """Algorithm 1's safeguard with reading R8: every accepted iterate has
    F(k) <= F(k-1) (1 + 1e-13) unless it came from the w = 0 redo, and the
    redo fired on this problem."""
    Xs, _, U0, L = _coupled_problem(seed=5, K=3, noise=0.2)
    prob = O.Problem(Xs, [3] * 3, L)
    res = O.apg(prob, U0, max_it=300, eps=0.0)
    F, redo = res["hist"]["F"], res["hist"]["redo"]
    assert any(redo)
    for i, r in enumerate(redo):
        if not r:
            assert F[i + 1] <= F[i] + O.TIE_TOL * abs(F[i]), i
    # the redo fires exactly where the plain (no safeguard) iteration first
    # raises F, and not before: up to there both runs are the same
    off = O.apg(prob, U0, max_it=300, eps=0.0, reupdate=False)["hist"]["F"]
    first = next(i for i in range(1, len(off)) if off[i] - off[i - 1] > O.TIE_TOL * abs(off[i - 1]))
    assert not any(redo[:first - 1])
    assert redo[first - 1]
    assert F[:first] == off[:first]


def test_planted_safeguard_mistake_is_caught(monkeypatch):
    monkeypatch.setattr(O, "apg", _planted(O.apg, "(F - F_prev) > TIE_TOL", "(F_prev - F) > TIE_TOL"))
    with pytest.raises(AssertionError):
        test_safeguard_accepts_no_increase()


# ------------------------------------------------------- problem set-up -----

def test_couple_initial_takes_shared_columns_from_block_zero():
    """Eq. tensormodel: U_C^(n,1) = ... = U_C^(n,K); the oracle takes them
    from block 0 and leaves every individual column as given."""
    rng = np.random.default_rng(3)
    dims, L = (4, 3, 5), [2, 1, 0]
    U0 = [[rng.random((d, 3)) for d in dims] for _ in range(3)]
    prob = O.Problem([np.zeros(dims)] * 3, [3] * 3, L)
    U = O.couple_initial(prob, U0)
    for k in range(3):
        for n in range(3):
            np.testing.assert_array_equal(U[k][n][:, :L[n]], U0[0][n][:, :L[n]])
            np.testing.assert_array_equal(U[k][n][:, L[n]:], U0[k][n][:, L[n]:])


def test_problem_rejects_invalid_coupling():
    """L_n <= min_k R_k (Section II-C) and coupled modes of equal size."""
    with pytest.raises(AssertionError):
        O.Problem([np.zeros((3, 3, 3))] * 2, [2, 3], [3, 0, 0])
    with pytest.raises(AssertionError):
        O.Problem([np.zeros((3, 3, 3)), np.zeros((4, 3, 3))], [2, 2], [1, 0, 0])
    O.Problem([np.zeros((3, 3, 3)), np.zeros((4, 3, 3))], [2, 2], [0, 1, 0])
