"""Write tests/golden/coupled_sweep.json: one full extrapolated sweep of
CoNCPD-APG over two coupled third-order blocks, computed elementwise in
50-digit arithmetic (mpmath) straight from the paper's equations.

This generator does not import the oracle: every quantity is written out as
the scalar sums of the equations it comes from, so that the oracle's matrix
form can be checked against it.

  Gram and Hadamard (Eq. solapgU, first term):
      H^(n,k)[a, b] = lam_a lam_b prod_{m != n} sum_i U^(m,k)[i, a] U^(m,k)[i, b]
  MTTKRP (Eq. solapgU, second term):
      M^(n,k)[i, r] = lam_r sum over the other indices of
                      X^(k)[i_1, i_2, i_3] prod_{m != n} U^(m,k)[i_m, r]
  Lipschitz constant (Eq. eqLipsLu): the largest eigenvalue of the 2 x 2
      symmetric H, (a + c)/2 + sqrt(((a - c)/2)^2 + b^2)
  Weights (Eq. eqextrawu; shared part: one weight from the block sums of L):
      w = min(w_hat, delta_w sqrt(L_prev / L))
  Extrapolation (Eq. eqextraPU):  U_hat = U_1 + w (U_1 - U_2)
  Gradient at U_hat:  G_hat = U_hat H - M
  Individual columns (Eq. solUnsI):  max(0, U_hat - G_hat / L^(n,k))
  Shared columns (Eq. solUnC):  max(0, U_hat_C - sum_k G_hat_C^(k) / sum_k L^(n,k))
  Core (Eqs. eqLipsLd, eqextraPG, solapgG, solD), before the factors:
      H_d[a, b] = prod_m sum_i U^(m,k)[i, a] U^(m,k)[i, b]
      g = H_d lam_hat - t,  t_r = sum X[i_1, i_2, i_3] prod_m U^(m,k)[i_m, r]
      lam = max(0, lam_hat - g / L_d)

Modes are updated in order and every block of a mode sees the factors as
they were before that mode's update (the Gauss-Seidel / Jacobi reading).

    python tests/golden/make_coupled_sweep.py
"""

import itertools
import json
import os

import mpmath as mp
import numpy as np

mp.mp.dps = 50
HERE = os.path.dirname(os.path.abspath(__file__))

DIMS = (3, 4, 5)
K, R, N = 2, 2, 3
L = [1, 0, 0]
DELTA_W = mp.mpf("0.9999")
W_HAT = mp.mpf("0.6")


def draw(rng, shape, lo, hi, digits=3):
    """Inputs rounded to a few decimals, so the fixture stores them exactly."""
    return np.round(rng.uniform(lo, hi, size=shape), digits)


def mat(a):
    return [[mp.mpf(float(v)) for v in row] for row in np.atleast_2d(a)]


def lmax2(H):
    a, b, c = H[0][0], H[0][1], H[1][1]
    return (a + c) / 2 + mp.sqrt(((a - c) / 2) ** 2 + b * b)


def weight(w_hat, L_prev, L_cur):
    if L_cur <= 0:
        return mp.mpf(0)
    return min(w_hat, DELTA_W * mp.sqrt(L_prev / L_cur))


def gram_entry(U, a, b):
    return mp.fsum(U[i][a] * U[i][b] for i in range(len(U)))


def sweep(X, U1, U2, lam1, lam2, Lprev, use_core):
    U1 = [[[row[:] for row in U1[k][n]] for n in range(N)] for k in range(K)]
    U2 = [[[row[:] for row in U2[k][n]] for n in range(N)] for k in range(K)]
    lam1 = [l[:] for l in lam1]
    lam2 = [l[:] for l in lam2]
    trace = {}
    if use_core:
        for k in range(K):
            Hd = [[mp.fprod(gram_entry(U1[k][m], a, b) for m in range(N)) for b in range(R)] for a in range(R)]
            Ld = lmax2(Hd)
            w = weight(W_HAT, Lprev["d"][k], Ld)
            lam_hat = [lam1[k][r] + w * (lam1[k][r] - lam2[k][r]) for r in range(R)]
            t = [mp.fsum(X[k][i][j][l] * U1[k][0][i][r] * U1[k][1][j][r] * U1[k][2][l][r]
                         for i, j, l in itertools.product(*[range(d) for d in DIMS])) for r in range(R)]
            g = [mp.fsum(Hd[r][s] * lam_hat[s] for s in range(R)) - t[r] for r in range(R)]
            lam2[k] = lam1[k]
            lam1[k] = [max(mp.mpf(0), lam_hat[r] - g[r] / Ld) for r in range(R)]
            trace[f"Ld_{k}"] = Ld
            trace[f"wd_{k}"] = w
    for n in range(N):
        H, M, Lu, w = [], [], [], []
        for k in range(K):
            lam = lam1[k]
            Hk = [[lam[a] * lam[b] * mp.fprod(gram_entry(U1[k][m], a, b) for m in range(N) if m != n)
                   for b in range(R)] for a in range(R)]
            Mk = [[mp.mpf(0)] * R for _ in range(DIMS[n])]
            for idx in itertools.product(*[range(d) for d in DIMS]):
                x = X[k][idx[0]][idx[1]][idx[2]]
                for r in range(R):
                    p = x * lam[r]
                    for m in range(N):
                        if m != n:
                            p *= U1[k][m][idx[m]][r]
                    Mk[idx[n]][r] += p
            Lk = lmax2(Hk)
            H.append(Hk)
            M.append(Mk)
            Lu.append(Lk)
            w.append(weight(W_HAT, Lprev["u"][n][k], Lk))
        LC = mp.fsum(Lu)
        Ln = L[n]
        I = DIMS[n]
        Uhat = [[[U1[k][n][i][r] + w[k] * (U1[k][n][i][r] - U2[k][n][i][r]) for r in range(R)] for i in range(I)]
                for k in range(K)]
        wC = None
        if Ln > 0:
            wC = weight(W_HAT, Lprev["c"][n], LC)
            for i in range(I):
                for r in range(Ln):
                    shared = U1[0][n][i][r] + wC * (U1[0][n][i][r] - U2[0][n][i][r])
                    for k in range(K):
                        Uhat[k][i][r] = shared
        Ghat = [[[mp.fsum(Uhat[k][i][s] * H[k][s][r] for s in range(R)) - M[k][i][r] for r in range(R)]
                 for i in range(I)] for k in range(K)]
        new = [[[max(mp.mpf(0), Uhat[k][i][r] - Ghat[k][i][r] / Lu[k]) for r in range(R)] for i in range(I)]
               for k in range(K)]
        if Ln > 0:
            for i in range(I):
                for r in range(Ln):
                    v = max(mp.mpf(0), Uhat[0][i][r] - mp.fsum(Ghat[k][i][r] for k in range(K)) / LC)
                    for k in range(K):
                        new[k][i][r] = v
        for k in range(K):
            U2[k][n] = U1[k][n]
            U1[k][n] = new[k]
            trace[f"L_{n}_{k}"] = Lu[k]
            trace[f"w_{n}_{k}"] = w[k]
            trace[f"Uhat_{n}_{k}"] = Uhat[k]
        trace[f"LC_{n}"] = LC
        if wC is not None:
            trace[f"wC_{n}"] = wC
    return U1, U2, lam1, lam2, trace


def s(v):
    if isinstance(v, list):
        return [s(x) for x in v]
    return mp.nstr(v, 30)


def main():
    rng = np.random.default_rng(20230210)
    X = [draw(rng, DIMS, 0.0, 2.0) for _ in range(K)]
    U1 = [[draw(rng, (d, R), 0.05, 1.0) for d in DIMS] for _ in range(K)]
    U2 = [[draw(rng, (d, R), 0.05, 1.5) for d in DIMS] for _ in range(K)]
    for n in range(N):  # the shared columns start equal across blocks
        for k in range(1, K):
            U1[k][n][:, :L[n]] = U1[0][n][:, :L[n]]
            U2[k][n][:, :L[n]] = U2[0][n][:, :L[n]]
    lam1 = [draw(rng, (R,), 0.5, 1.5) for _ in range(K)]
    lam2 = [draw(rng, (R,), 0.5, 1.5) for _ in range(K)]
    # L of the previous iteration, chosen so that the weights take both
    # branches of the min: some stay at w_hat, the shared one and some
    # individual ones are set by the ratio of Lipschitz constants
    Lprev = {"u": [[0.9, 0.3], [0.25, 2.0], [0.2, 0.1]], "c": [0.2, None, None], "d": [3.0, 0.2]}

    # the binary doubles the fixture stores, converted exactly
    Xm = [[[[mp.mpf(float(v)) for v in row] for row in plane] for plane in Xk] for Xk in X]
    U1m = [[mat(A) for A in Uk] for Uk in U1]
    U2m = [[mat(A) for A in Uk] for Uk in U2]
    lam1m = [[mp.mpf(float(v)) for v in l] for l in lam1]
    lam2m = [[mp.mpf(float(v)) for v in l] for l in lam2]
    cases = {}
    for use_core in (False, True):
        # the previous L must be comparable with this state's: scale them by
        # the constants of this sweep's inputs so the ratios are near 1
        Lp = {"u": [[mp.mpf(x) for x in row] for row in Lprev["u"]],
              "c": [None if x is None else mp.mpf(x) for x in Lprev["c"]],
              "d": [mp.mpf(x) for x in Lprev["d"]]}
        _, _, _, _, tr0 = sweep(Xm, U1m, U2m, lam1m, lam2m,
                                {"u": [[mp.mpf(1)] * K] * N, "c": [mp.mpf(1)] * N, "d": [mp.mpf(1)] * K},
                                use_core)
        # first pass gives the scale of every L at its update; use the chosen
        # factors times those (the ratio is then the chosen factor inverted)
        for n in range(N):
            for k in range(K):
                Lp["u"][n][k] = Lp["u"][n][k] * tr0[f"L_{n}_{k}"]
            if Lp["c"][n] is not None:
                Lp["c"][n] = Lp["c"][n] * tr0[f"LC_{n}"]
        if use_core:
            for k in range(K):
                Lp["d"][k] = Lp["d"][k] * tr0[f"Ld_{k}"]
        # stored as doubles; the sweep below uses exactly those doubles
        Lp = {"u": [[mp.mpf(float(x)) for x in row] for row in Lp["u"]],
              "c": [None if x is None else mp.mpf(float(x)) for x in Lp["c"]],
              "d": [mp.mpf(float(x)) for x in Lp["d"]]}
        U1n, U2n, l1n, l2n, tr = sweep(Xm, U1m, U2m, lam1m, lam2m, Lp, use_core)
        # the case must exercise what it is meant to pin
        ws = [tr[f"w_{n}_{k}"] for n in range(N) for k in range(K)]
        assert any(w == W_HAT for w in ws) and any(w < W_HAT for w in ws)
        assert tr["wC_0"] < W_HAT and all(tr["wC_0"] != tr[f"w_0_{k}"] for k in range(K))
        clipped = sum(1 for k in range(K) for n in range(N) for row in U1n[k][n] for v in row if v == 0)
        assert clipped > 0
        cases["core" if use_core else "plain"] = {
            "use_core": use_core,
            "Lprev": {"u": [[float(x) for x in row] for row in Lp["u"]],
                      "c": [None if x is None else float(x) for x in Lp["c"]],
                      "d": [float(x) for x in Lp["d"]] if use_core else None},
            "expect": {"U1": [[s(A) for A in Uk] for Uk in U1n], "lam1": s(l1n),
                       "trace": {key: s(v) for key, v in tr.items()}},
            "clipped_entries": clipped,
        }
    out = {
        "about": "one extrapolated CoNCPD-APG sweep, K=2 blocks of 3x4x5, R=2, L=[1,0,0], w_hat=0.6, "
                 "delta_w=0.9999; computed elementwise in 50-digit arithmetic by make_coupled_sweep.py "
                 "from Eqs. solapgU, eqLipsLu, eqextrawu, eqextraPU, solUnsI, solUnC (and eqLipsLd, "
                 "eqextraPG, solapgG, solD for the core case)",
        "dims": list(DIMS), "K": K, "R": R, "L": L, "w_hat": 0.6, "delta_w": 0.9999,
        "X": [Xk.tolist() for Xk in X],
        "U1": [[A.tolist() for A in Uk] for Uk in U1], "U2": [[A.tolist() for A in Uk] for Uk in U2],
        "lam1": [l.tolist() for l in lam1], "lam2": [l.tolist() for l in lam2],
        "cases": cases,
    }
    with open(os.path.join(HERE, "coupled_sweep.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
