"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs.  Tolerances: FP64 path 1e-9 relative Frobenius on factors; FP32
path 1e-5 (first iterations) as stated for the method's FP32 form; the
final fit within 1e-4."""

import numpy as np
import pytest

from oracle import cncpd_oracle as O
from tests.gpu_common import coupled_inputs, need_gpu, rel_fro, run_oracle_steps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _P():
    import paper_2302_05119_gb300 as P
    return P


# ------------------------------------------------------------- MTTKRP ----

@pytest.mark.parametrize("dt", [np.float64, np.float32])
@pytest.mark.parametrize("dims,R", [
    ([(7, 13, 37), (7, 13, 37)], 3),
    ([(33, 65, 40)], 12),
    ([(5, 9, 11), (6, 9, 3)], 7),
    ([(1, 1, 1)], 1),
    ([(64, 33, 129)], 20),
    ([(3, 4, 5, 6), (2, 4, 7, 3)], 5),
    ([(9, 7, 5, 4, 3)], 4),
    ([(40, 40, 40)], 33),
    # one case in every rank bucket of the compiled kernels
    ([(12, 10, 9)], 10),
    ([(10, 11, 12)], 16),
    ([(9, 8, 10)], 24),
    ([(8, 9, 10)], 32),
    ([(7, 6, 9)], 48),
    ([(6, 7, 8)], 64),
])
def test_mttkrp_matches_oracle(dims, R, dt):
    rng = np.random.default_rng(len(dims) * 100 + R)
    Xs = [rng.random(d).astype(dt) for d in dims]
    N = len(dims[0])
    U = [[rng.random((I, R)).astype(dt) for I in d] for d in dims]
    m = _P().CoupledNCP(Xs, R, [0] * N)
    m.set_factors(U)
    tol = 1e-12 if dt == np.float64 else 2e-6
    for k in range(len(dims)):
        for n in range(N):
            got = m.mttkrp(k, n)
            want = O.mttkrp(Xs[k].astype(np.float64), [A.astype(np.float64) for A in U[k]], n)
            assert rel_fro(got, want) <= tol, (k, n)
    m.close()


def _to_bf16(a):
    """Round FP32 values to the nearest BF16 (ties to even), returned as FP32."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("dims,R", [
    ([(70, 37, 150), (9, 64, 130)], 10),
    ([(33, 41, 200)], 20),
    ([(5, 6, 7, 8)], 12),
    ([(20, 30, 40)], 33),
])
@pytest.mark.parametrize("tensor_cores", [True, False])
def test_mttkrp_bf16_storage_exact_inputs(dims, R, tensor_cores):
    """BF16 storage of a tensor whose values are already BF16 numbers is
    lossless, so the MTTKRP (FP32 accumulation) must match the FP64 oracle on
    the same values to FP32 accumulation accuracy; shapes span several tiles
    with ragged tails.  Third-order cases with R <= 32 run on the tcgen05
    passes when tensor_cores is set (the factors enter as three BF16 parts)."""
    rng = np.random.default_rng(R * 7 + len(dims))
    Xs = [_to_bf16(rng.random(d).astype(np.float32)) for d in dims]
    N = len(dims[0])
    U = [[rng.random((I, R)).astype(np.float32) for I in d] for d in dims]
    m = _P().CoupledNCP(Xs, R, [0] * N, storage="bf16", tensor_cores=tensor_cores)
    m.set_factors(U)
    for k in range(len(dims)):
        for n in range(N):
            got = m.mttkrp(k, n)
            want = O.mttkrp(Xs[k].astype(np.float64), [A.astype(np.float64) for A in U[k]], n)
            assert rel_fro(got, want) <= 2e-6, (k, n)
    m.close()


@pytest.mark.parametrize("R", [12, 20])
def test_mttkrp_bf16_tensor_cores_many_units(R):
    """The tcgen05 passes with many work units per CTA (hundreds of 256-row
    tiles, i0 slabs split across CTAs, ragged K and column tails) against the
    FP64 oracle on BF16-exact values."""
    rng = np.random.default_rng(40 + R)
    dims = [(300, 260, 200), (280, 260, 136)]
    Xs = [_to_bf16(rng.random(d).astype(np.float32)) for d in dims]
    U = [[rng.random((I, R)).astype(np.float32) for I in d] for d in dims]
    m = _P().CoupledNCP(Xs, R, [0, 0, 0], storage="bf16", tensor_cores=True)
    m.set_factors(U)
    for k in range(len(dims)):
        for n in range(3):
            got = m.mttkrp(k, n)
            want = O.mttkrp(Xs[k].astype(np.float64), [A.astype(np.float64) for A in U[k]], n)
            assert rel_fro(got, want) <= 2e-6, (k, n)
    m.close()


# --------------------------------------------------------- Lipschitz -----

@pytest.mark.parametrize("R", [1, 2, 5, 10, 20, 33, 64])
def test_lipschitz_matches_eigvalsh(R):
    """||H||_2 (Eqs. eqLipsLd / eqLipsLu) to 1e-12 relative when the two
    largest eigenvalues are separated; when they agree to within a relative
    gap below FP32 resolution, the error is bounded by that gap."""
    P = _P()
    rng = np.random.default_rng(R)
    A = rng.random((3 * R + 2, R))
    H = A.T @ A
    assert P.lipschitz(H) == pytest.approx(O.spectral_norm(H), rel=1e-12)
    Q, _ = np.linalg.qr(rng.standard_normal((R, R)))
    ev = np.linspace(0.1, 1.0, R)
    H1 = (Q * ev) @ Q.T
    assert P.lipschitz(H1) == pytest.approx(O.spectral_norm(H1), rel=1e-12)
    if R > 1:
        gap = 1e-9
        ev[-2] = 1.0 - gap
        H2 = (Q * ev) @ Q.T
        lm = P.lipschitz(H2)
        assert lm <= O.spectral_norm(H2) * (1 + 1e-12)
        assert lm >= O.spectral_norm(H2) * (1 - gap)
    assert P.lipschitz(np.zeros((R, R))) == 0.0


# ---------------------------------------------------- iteration parity ---

def _gpu_steps(Xs, R, L, U0, iters, dt, storage=None, nonneg=None, use_core=False, lam0=None, use_graph=True):
    P = _P()
    m = P.CoupledNCP([X.astype(dt) for X in Xs], R, L, nonneg=nonneg, storage=storage,
                     use_core=use_core, use_graph=use_graph)
    m.set_factors(U0)
    if lam0 is not None:
        m.set_cores(lam0)
    snaps, redo = [], []
    for _ in range(iters):
        s = m.step(1)
        redo.append(s["reupdates"] > 0)
        snaps.append((m.factors(), [m.core(k) for k in range(len(Xs))], s))
    return m, snaps, redo


@pytest.mark.parametrize("dt,tol", [(np.float64, 1e-9), (np.float32, 1e-5)])
@pytest.mark.parametrize("use_graph", [True, False])
def test_first_iterations_match_oracle_small_40cube(dt, tol, use_graph):
    """K=3 blocks of 40^3, R=5, L=[2,0,0] (the small simulation workload):
    factors after each of the first 10 iterations and the re-update
    decisions match the oracle."""
    import synth
    w = synth.workload("small_40cube")
    Xs, _ = synth.make_tensors(w)
    Xs = [X.astype(dt) for X in Xs]
    U0 = synth.init_factors(w.dims, w.R, w.seed)
    snaps_o, res_o = run_oracle_steps([X.astype(np.float64) for X in Xs], [w.R] * w.K, w.L, U0, 10)
    m, snaps_g, redo_g = _gpu_steps(Xs, w.R, w.L, U0, 10, dt, use_graph=use_graph)
    assert redo_g == res_o["hist"]["redo"]
    for it in range(10):
        Ug = snaps_g[it][0]
        Uo = snaps_o[it][0]
        for k in range(w.K):
            for n in range(w.N):
                assert rel_fro(Ug[k][n], Uo[k][n]) <= tol, (it, k, n)
        assert snaps_g[it][2]["F"] == pytest.approx(res_o["hist"]["F"][it + 1], rel=max(tol, 1e-12) * 10)
    m.close()


def test_fit_after_200_iterations_small_40cube_fp32():
    """Final fit of the FP32 path within 1e-4 of the FP64 oracle's."""
    import synth
    w = synth.workload("small_40cube")
    Xs, _ = synth.make_tensors(w)
    X32 = [X.astype(np.float32) for X in Xs]
    U0 = synth.init_factors(w.dims, w.R, w.seed)
    res_o = O.apg(O.Problem([X.astype(np.float64) for X in X32], [w.R] * w.K, w.L), U0, max_it=200, eps=0.0)
    fit_o = O.fit([X.astype(np.float64) for X in X32], res_o["U"], res_o["lam"])
    m = _P().CoupledNCP(X32, w.R, w.L)
    m.set_factors(U0)
    s = m.step(200)
    assert s["iters"] == 200
    assert abs(s["fit"] - fit_o) <= 1e-4
    assert abs(m.global_fit() - fit_o) <= 1e-4
    m.close()


def test_common_columns_bit_identical_and_nonnegative():
    Xs, _, U0 = coupled_inputs([(12, 10, 9)] * 4, 4, [2, 3, 1], seed=3)
    m = _P().CoupledNCP([X.astype(np.float32) for X in Xs], 4, [2, 3, 1])
    m.set_factors(U0)
    for _ in range(5):
        m.step(3)
        U = m.factors(np.float32)
        for n, Ln in enumerate([2, 3, 1]):
            for k in range(1, 4):
                assert np.array_equal(U[k][n][:, :Ln], U[0][n][:, :Ln])
            for k in range(4):
                assert np.all(U[k][n] >= 0)
    m.close()


@pytest.mark.parametrize("dt,tol", [(np.float64, 1e-9), (np.float32, 1e-5)])
def test_uneven_fourth_order_blocks(dt, tol):
    """Fourth-order blocks of different sizes in the uncoupled modes (the
    EEG-shaped batching case), L = [2, 2, 0, 0]."""
    dims = [(6, 5, 7, 4), (6, 5, 3, 9), (6, 5, 10, 2)]
    Xs, _, U0 = coupled_inputs(dims, 3, [2, 2, 0, 0], seed=4, dist="gamma")
    Xs = [X.astype(dt) for X in Xs]
    snaps_o, res_o = run_oracle_steps([X.astype(np.float64) for X in Xs], [3] * 3, [2, 2, 0, 0], U0, 8)
    m, snaps_g, redo_g = _gpu_steps(Xs, 3, [2, 2, 0, 0], U0, 8, dt)
    assert redo_g == res_o["hist"]["redo"]
    for it in range(8):
        for k in range(3):
            for n in range(4):
                assert rel_fro(snaps_g[it][0][k][n], snaps_o[it][0][k][n]) <= tol, (it, k, n)
    m.close()


@pytest.mark.parametrize("dt,tol", [(np.float64, 1e-9), (np.float32, 1e-5)])
def test_core_tensors_fully_coupled(dt, tol):
    """use_core on a fully coupled case (all L_n > 0, Section III-C)."""
    dims = [(9, 8, 7)] * 2
    Xs, _, U0 = coupled_inputs(dims, 3, [3, 3, 3], seed=5)
    rng = np.random.default_rng(9)
    lam0 = [rng.random(3) for _ in range(2)]
    Xs = [X.astype(dt) for X in Xs]
    snaps_o, res_o = run_oracle_steps([X.astype(np.float64) for X in Xs], [3, 3], [3, 3, 3], U0, 8,
                                      use_core=True, lam0=lam0)
    m, snaps_g, redo_g = _gpu_steps(Xs, 3, [3, 3, 3], U0, 8, dt, use_core=True, lam0=lam0)
    assert redo_g == res_o["hist"]["redo"]
    for it in range(8):
        for k in range(2):
            assert rel_fro(snaps_g[it][1][k], snaps_o[it][1][k]) <= tol
            for n in range(3):
                assert rel_fro(snaps_g[it][0][k][n], snaps_o[it][0][k][n]) <= tol, (it, k, n)
    m.close()


def test_nonneg_flag_off_in_one_mode():
    dims = [(10, 9, 8)] * 2
    Xs, _, U0 = coupled_inputs(dims, 3, [1, 0, 0], seed=6)
    nonneg = [True, False, True]
    snaps_o, res_o = run_oracle_steps(Xs, [3, 3], [1, 0, 0], U0, 6, nonneg=nonneg)
    m, snaps_g, redo_g = _gpu_steps(Xs, 3, [1, 0, 0], U0, 6, np.float64, nonneg=nonneg)
    for it in range(6):
        for k in range(2):
            for n in range(3):
                assert rel_fro(snaps_g[it][0][k][n], snaps_o[it][0][k][n]) <= 1e-9
    m.close()


def test_gradient_matches_oracle():
    dims = [(12, 10, 8)] * 2
    Xs, _, U0 = coupled_inputs(dims, 3, [2, 1, 0], seed=7)
    m = _P().CoupledNCP(Xs, 3, [2, 1, 0])
    m.set_factors(U0)
    F, gU, gC = m.objective_grad()
    prob = O.Problem(Xs, [3, 3], [2, 1, 0])
    Uc = O.couple_initial(prob, U0)
    lam = [np.ones(3)] * 2
    assert F == pytest.approx(prob.objective_fn(Uc, lam), rel=1e-10)
    for k in range(2):
        for n in range(3):
            assert rel_fro(gU[k][n], O.gradient(prob, Uc, lam, k, n)) <= 1e-10
    for n, Ln in enumerate([2, 1, 0]):
        if Ln:
            want = sum(O.gradient(prob, Uc, lam, k, n)[:, :Ln] for k in range(2))
            assert rel_fro(gC[n], want) <= 1e-10
    m.close()


def test_autograd_loss_matches_oracle_gradient():
    """CoupledCPLoss: F and torch.autograd gradients equal the oracle's
    objective and gradient; the shared columns' gradient (the sum over
    blocks) lands on block 0's copy."""
    torch = pytest.importorskip("torch")
    dims = [(12, 10, 8)] * 2
    L = [2, 1, 0]
    Xs, _, U0 = coupled_inputs(dims, 3, L, seed=9)
    P = _P()
    m = P.CoupledNCP(Xs, 3, L)
    fac = [torch.tensor(U0[k][n], dtype=torch.float64, requires_grad=True) for k in range(2) for n in range(3)]
    F = P.CoupledCPLoss.apply(m, *fac)
    grads = torch.autograd.grad(F, fac)
    prob = O.Problem(Xs, [3, 3], L)
    Uc = O.couple_initial(prob, U0)
    lam = [np.ones(3)] * 2
    assert float(F.detach()) == pytest.approx(prob.objective_fn(Uc, lam), rel=1e-10)
    for k in range(2):
        for n in range(3):
            want = O.gradient(prob, Uc, lam, k, n).copy()
            if L[n]:
                want[:, :L[n]] = sum(O.gradient(prob, Uc, lam, kk, n)[:, :L[n]] for kk in range(2)) if k == 0 else 0.0
            assert rel_fro(grads[k * 3 + n].numpy(), want) <= 1e-10
    m.close()


def test_checkpoint_resume_is_bitwise():
    dims = [(14, 11, 9)] * 3
    Xs, _, U0 = coupled_inputs(dims, 4, [2, 0, 0], seed=8)
    X32 = [X.astype(np.float32) for X in Xs]
    P = _P()
    a = P.CoupledNCP(X32, 4, [2, 0, 0])
    a.set_factors(U0)
    a.step(20)
    Ua = a.factors(np.float32)
    b = P.CoupledNCP(X32, 4, [2, 0, 0])
    b.set_factors(U0)
    b.step(10)
    blob = b.save_state()
    c = P.CoupledNCP(X32, 4, [2, 0, 0])
    c.load_state(blob)
    c.step(10)
    Uc = c.factors(np.float32)
    for k in range(3):
        for n in range(3):
            assert np.array_equal(Ua[k][n], Uc[k][n])
    for m in (a, b, c):
        m.close()


def test_host_and_device_inputs_agree():
    torch = pytest.importorskip("torch")
    dims = [(16, 12, 20)] * 2
    Xs, _, U0 = coupled_inputs(dims, 4, [2, 0, 0], seed=10)
    P = _P()
    a = P.CoupledNCP([X.astype(np.float32) for X in Xs], 4, [2, 0, 0])
    b = P.CoupledNCP([torch.from_numpy(X.astype(np.float32)).cuda() for X in Xs], 4, [2, 0, 0])
    a.set_factors(U0)
    b.set_factors([[torch.from_numpy(A).cuda() for A in Uk] for Uk in U0])
    a.step(5)
    b.step(5)
    for k in range(2):
        for n in range(3):
            assert np.array_equal(a.factor(k, n, np.float32), b.factor(k, n, np.float32))
    out = torch.empty((16, 4), dtype=torch.float32, device="cuda")
    b.factor(0, 0, out=out)
    assert np.array_equal(out.cpu().numpy(), a.factor(0, 0, np.float32))
    a.close()
    b.close()


# ------------------------------------------------------------------ LRA ---

@pytest.mark.parametrize("dt,tol,Rt,storage", [(np.float64, 1e-9, 4, None), (np.float64, 1e-9, 3, None),
                                               (np.float32, 1e-5, 3, None), (np.float32, 1e-5, 3, "bf16")])
def test_lra_path_matches_oracle(dt, tol, Rt, storage):
    """lraCoNCPD-APG: ALS low-rank approximation of each block, then the
    collapsed APG iterations, against the oracle's Algorithm 2, at the
    method's tolerances (FP64 1e-9, FP32 1e-5 relative Frobenius): the ALS
    factors and every APG factor over 10 iterations.  FP32 runs at R~ = R,
    the paper's setting, on data of rank R with 20 dB noise; FP64 also at
    R~ above the data's rank."""
    dims = [(14, 12, 10)] * 3
    Xs, _, U0 = coupled_inputs(dims, 3, [2, 0, 0], seed=12)
    Xs = [X.astype(dt) for X in Xs]
    if storage == "bf16":  # values already BF16 numbers: the stored tensor is exact
        Xs = [_to_bf16(X) for X in Xs]
    X64 = [X.astype(np.float64) for X in Xs]
    rng = np.random.default_rng(13)
    Ut0 = [[rng.random((d, Rt)) for d in dims[0]] for _ in range(3)]
    Uts, sweeps = [], []
    for X, Ut in zip(X64, Ut0):
        u, s, _ = O.als_cpd(X, Ut, 200, 1e-4)
        Uts.append(u)
        sweeps.append(s)
    prob = O.LRAProblem(Uts, [3] * 3, [2, 0, 0])
    snaps = []
    res = O.apg(prob, U0, max_it=10, eps=0.0,
                callback=lambda it, st, info: snaps.append([[A.copy() for A in Uk] for Uk in st.U1]))
    P = _P()
    m = P.CoupledNCP(Xs, 3, [2, 0, 0], storage=storage)
    m.set_factors(U0)
    st = m.lra(Rt, Ut0)
    assert st["lra_sweeps"] == max(sweeps)
    worst_u = worst_x = worst = 0.0
    for k in range(3):
        for n in range(3):
            worst_u = max(worst_u, rel_fro(m.lra_factor(k, n), Uts[k][n]))
            assert rel_fro(m.lra_factor(k, n), Uts[k][n]) <= tol
        worst_x = max(worst_x, rel_fro(O.kruskal(np.ones(Rt), [m.lra_factor(k, n) for n in range(3)]),
                                       O.kruskal(np.ones(Rt), Uts[k])))
    for it in range(10):
        s = m.step(1)
        assert (s["reupdates"] > 0) == res["hist"]["redo"][it]
        for k in range(3):
            for n in range(3):
                worst = max(worst, rel_fro(m.factor(k, n), snaps[it][k][n]))
                assert rel_fro(m.factor(k, n), snaps[it][k][n]) <= tol, (it, k, n)
    print(f"LRA noisy ({np.dtype(dt).name}, R~={Rt}, {storage}): sweeps {max(sweeps)}, U~ {worst_u:.3e}, "
          f"[[U~]] {worst_x:.3e}, APG factors {worst:.3e}")
    gfit = O.fit(X64, res["U"], res["lam"])
    assert abs(m.global_fit() - gfit) <= 1e-4
    m.close()


# --------------------------------------------------------- BF16 storage ---

@pytest.mark.parametrize("storage,tol", [("bf16", 3e-3), ("bf16x2", 3e-4)])
def test_bf16_storage_error_vs_fp64_oracle(storage, tol):
    """X streamed in BF16 (or hi+lo BF16 pairs) with FP32 accumulation:
    factors after 10 iterations within the stated error of the FP64 oracle
    run on the unquantised data."""
    dims = [(48, 40, 36)] * 2
    Xs, _, U0 = coupled_inputs(dims, 5, [2, 0, 0], seed=14)
    snaps_o, res_o = run_oracle_steps(Xs, [5, 5], [2, 0, 0], U0, 10)
    m, snaps_g, redo_g = _gpu_steps(Xs, 5, [2, 0, 0], U0, 10, np.float32, storage=storage)
    for it in range(10):
        for k in range(2):
            for n in range(3):
                assert rel_fro(snaps_g[it][0][k][n], snaps_o[it][0][k][n]) <= tol, (it, k, n)
    m.close()


@pytest.mark.parametrize("tdt", ["float64", "float32"])
def test_autograd_loss_on_cuda_tensors(tdt):
    """CoupledCPLoss with CUDA factors: the gradients come back as CUDA
    tensors written by the library (no host round trip of the factors) and
    match the oracle's gradient (Eq. solbpgU; App. A for the shared
    columns)."""
    torch = pytest.importorskip("torch")
    dt = getattr(torch, tdt)
    dims = [(12, 10, 8)] * 2
    L = [2, 1, 0]
    Xs, _, U0 = coupled_inputs(dims, 3, L, seed=19)
    P = _P()
    m = P.CoupledNCP([X.astype(np.float32 if tdt == "float32" else np.float64) for X in Xs], 3, L)
    fac = [torch.tensor(U0[k][n], dtype=dt, device="cuda", requires_grad=True) for k in range(2) for n in range(3)]
    F = P.CoupledCPLoss.apply(m, *fac)
    grads = torch.autograd.grad(F, fac)
    assert F.is_cuda and all(g.is_cuda and g.dtype == dt for g in grads)
    X64 = [X.astype(np.float32).astype(np.float64) if tdt == "float32" else X for X in Xs]
    Ucast = [[np.asarray(A, dtype=np.float32 if tdt == "float32" else np.float64).astype(np.float64) for A in Uk]
             for Uk in U0]
    prob = O.Problem(X64, [3, 3], L)
    Uc = O.couple_initial(prob, Ucast)
    lam = [np.ones(3)] * 2
    tol = 1e-10 if tdt == "float64" else 2e-5
    assert float(F.detach()) == pytest.approx(prob.objective_fn(Uc, lam), rel=tol)
    for k in range(2):
        for n in range(3):
            want = O.gradient(prob, Uc, lam, k, n).copy()
            if L[n]:
                want[:, :L[n]] = sum(O.gradient(prob, Uc, lam, kk, n)[:, :L[n]] for kk in range(2)) if k == 0 else 0.0
            assert rel_fro(grads[k * 3 + n].cpu().numpy(), want) <= tol, (k, n)
    m.close()


def test_loss_evaluation_leaves_the_solver_state_alone():
    """Evaluating the loss and its gradient at other factors in the middle of
    a fit does not change the iterates that follow (the APG extrapolation
    and its history are kept)."""
    torch = pytest.importorskip("torch")
    dims = [(16, 12, 10)] * 3
    Xs, _, U0 = coupled_inputs(dims, 4, [2, 0, 0], seed=20)
    X32 = [X.astype(np.float32) for X in Xs]
    P = _P()
    a = P.CoupledNCP(X32, 4, [2, 0, 0])
    a.set_factors(U0)
    a.step(6)
    rng = np.random.default_rng(3)
    other = [torch.tensor(rng.random((d, 4)), dtype=torch.float32, device="cuda", requires_grad=True)
             for _ in range(3) for d in dims[0]]
    F = P.CoupledCPLoss.apply(a, *other)
    torch.autograd.grad(F, other)
    a.step(6)
    b = P.CoupledNCP(X32, 4, [2, 0, 0])
    b.set_factors(U0)
    b.step(12)
    for k in range(3):
        for n in range(3):
            assert np.array_equal(a.factor(k, n, np.float32), b.factor(k, n, np.float32)), (k, n)
    a.close()
    b.close()


def test_load_state_on_the_same_handle():
    """Save, step, load the saved state back into the same handle, step
    again: the iterate equals the one the first step produced."""
    dims = [(14, 11, 9)] * 2
    Xs, _, U0 = coupled_inputs(dims, 4, [2, 0, 0], seed=25)
    m = _P().CoupledNCP([X.astype(np.float32) for X in Xs], 4, [2, 0, 0])
    m.set_factors(U0)
    m.step(5)
    blob = m.save_state()
    m.step(1)
    U6 = m.factors(np.float32)
    m.load_state(blob)
    m.step(1)
    for k in range(2):
        for n in range(3):
            assert np.array_equal(m.factor(k, n, np.float32), U6[k][n])
    m.close()


def _bf16x2_exact(a, rng):
    """Values x = hi + lo with hi a BF16 number and lo a BF16 number below a
    quarter of hi's last place, so the hi + lo storage split reproduces x
    exactly (and the lo plane is not zero)."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    hi = _to_bf16(a)
    lo = _to_bf16(0.25 * (a - hi))
    return (hi + lo).astype(np.float32)


@pytest.mark.parametrize("dims,R", [
    ([(70, 37, 150), (9, 64, 130)], 10),
    ([(33, 41, 200)], 20),
    ([(300, 260, 136)], 12),
    ([(5, 6, 7, 8)], 12),
])
@pytest.mark.parametrize("tensor_cores", [True, False])
def test_mttkrp_bf16x2_storage_exact_inputs(dims, R, tensor_cores):
    """BF16 hi + lo storage of values whose split is exact: the MTTKRP (both
    planes, FP32 accumulation; on the tcgen05 passes for third-order tensors
    with R <= 32, the lo plane's K chunks after the hi plane's) matches the
    FP64 oracle to FP32 accumulation accuracy."""
    rng = np.random.default_rng(R * 11 + len(dims))
    Xs = [_bf16x2_exact(rng.random(d), rng) for d in dims]
    assert any(np.any(X != _to_bf16(X)) for X in Xs)  # the lo plane carries something
    N = len(dims[0])
    U = [[rng.random((I, R)).astype(np.float32) for I in d] for d in dims]
    m = _P().CoupledNCP(Xs, R, [0] * N, storage="bf16x2", tensor_cores=tensor_cores)
    m.set_factors(U)
    for k in range(len(dims)):
        for n in range(N):
            got = m.mttkrp(k, n)
            want = O.mttkrp(Xs[k].astype(np.float64), [A.astype(np.float64) for A in U[k]], n)
            assert rel_fro(got, want) <= 2e-6, (k, n)
    m.close()
