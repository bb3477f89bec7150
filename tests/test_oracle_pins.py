"""Pins of the CPU oracle to facts outside itself (no GPU).

Each test checks the oracle against something the paper or the mathematics fixes: the
hs45 solution printed in Sec. 4.2, closed-form minimisers, brute force on tiny
problems, library factorizations and roots, finite differences and autograd of the
branch objective, complex power flow, and KKT conditions of the ADMM closed forms.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2106_14995_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ core operations

def test_chol_matches_numpy():
    rng = np.random.default_rng(0)
    for m in (1, 2, 5, 17, 32):
        G = rng.standard_normal((m, m))
        A = G @ G.T + m * np.eye(m)
        L = oracle.chol(A)
        np.testing.assert_allclose(L, np.linalg.cholesky(A), rtol=1e-12, atol=1e-12)


def test_chol_rejects_indefinite():
    A = np.diag([1.0, -1.0, 2.0])
    assert oracle.chol(A) is None


def test_chol_shifted_factor_and_mirror():
    rng = np.random.default_rng(1)
    for m in (3, 8, 20):
        G = rng.standard_normal((m, m))
        U, _ = np.linalg.qr(G)
        ev = rng.uniform(0.5, 2.0, m)
        ev[0] = -1.0  # indefinite by construction
        A = (U * ev) @ U.T
        A = 0.5 * (A + A.T)
        L, alpha = oracle.chol_shifted(A)
        assert L is not None and alpha > 0
        Lo = np.tril(L)
        np.testing.assert_allclose(Lo @ Lo.T, A + alpha * np.eye(m), rtol=1e-10, atol=1e-10)
        # L^T mirrored into the strict upper triangle (Sec. 4.4)
        np.testing.assert_array_equal(np.triu(L, 1), np.triu(Lo.T, 1))
        # positive definite input: no shift
        Apd = G @ G.T + np.eye(m)
        L2, a2 = oracle.chol_shifted(Apd)
        assert a2 == 0.0
        np.testing.assert_allclose(np.tril(L2), np.linalg.cholesky(Apd), rtol=1e-12, atol=1e-12)


def test_chol_shift_sequence_first_success():
    # the shift is the first of alpha0 = beta - min A_ii, then max(2 alpha, beta) ...
    # that makes A + alpha I positive definite; check minimality within the sequence
    A = np.array([[1.0, 2.0], [2.0, 1.0]])  # eigenvalues -1, 3
    L, alpha = oracle.chol_shifted(A, shift_frac=1e-3)
    beta = 1e-3 * 1.0
    seq = [0.0]  # min diag > 0 -> alpha0 = 0
    while len(seq) < 40:
        seq.append(max(2 * seq[-1], beta))
    ok = [a for a in seq if np.all(np.linalg.eigvalsh(A + a * np.eye(2)) > 0)]
    assert alpha == ok[0]


def test_trqsol_is_positive_root():
    rng = np.random.default_rng(2)
    for _ in range(50):
        n = rng.integers(1, 10)
        x = rng.standard_normal(n) * 0.1
        p = rng.standard_normal(n)
        delta = np.linalg.norm(x) + rng.uniform(0.1, 2.0)
        sig = oracle.trqsol(x, p, delta)
        roots = np.roots([p @ p, 2 * x @ p, x @ x - delta * delta])
        pos = max(r.real for r in roots)
        assert sig >= 0
        assert abs(sig - pos) <= 1e-12 * max(1.0, abs(pos))
        assert abs(np.linalg.norm(x + sig * p) - delta) <= 1e-12 * delta


def test_pgnorm_definition_cases():
    l = np.array([0.0, 0.0, 0.0, 0.0, -1.0])
    u = np.array([1.0, 1.0, 1.0, 1.0, -1.0])
    x = np.array([0.0, 0.0, 1.0, 0.5, -1.0])
    g = np.array([2.0, -3.0, -4.0, 0.7, 9.0])
    # at lower with g > 0 -> 0; at lower with g < 0 -> |g|; at upper with g < 0 -> 0;
    # interior -> |g|; fixed variable (l = u) -> 0
    assert oracle.pgnorm(x, g, l, u) == 3.0
    g2 = np.array([2.0, 0.0, -4.0, -0.7, -9.0])
    assert oracle.pgnorm(x, g2, l, u) == 0.7


def test_breakpt_cases():
    x = np.array([0.0, 0.5, 1.0, 0.2])
    l = np.zeros(4)
    u = np.ones(4)
    w = np.array([1.0, -0.25, 1.0, 0.0])
    nb, bmin, bmax = oracle.breakpt(x, w, l, u)
    # var0: (1-0)/1 = 1; var1: (0-0.5)/-0.25 = 2; var2 at u moving up: blocked; var3: w=0
    assert nb == 2 and bmin == 1.0 and bmax == 2.0


def test_steihaug_one_iteration_on_pd():
    # Sec. 4.3: with the complete factor of a positive definite A, Ahat = I and CG
    # finishes in one iteration; the step is the Newton step -A^-1 r when inside.
    rng = np.random.default_rng(3)
    m = 12
    G = rng.standard_normal((m, m))
    A = G @ G.T + np.eye(m)
    L, alpha = oracle.chol_shifted(A)
    assert alpha == 0.0
    r = rng.standard_normal(m)
    bhat = np.linalg.solve(np.tril(L), r)
    newton = -np.linalg.solve(A, r)
    for norm in (0, 1):
        w, info, it = oracle.steihaug(A, L, bhat, delta=1e6, norm=norm)
        assert it == 1 and info in (0, 1)
        np.testing.assert_allclose(w, newton, rtol=1e-9, atol=1e-12)
    # boundary, as Algorithm 1 prints it (norm 0): the CG iterate s = L^T w is bounded,
    # ||s||^2 = w'(L L^T)w = w'Aw = delta^2; the step is the Newton direction cut there
    delta = 0.3 * np.sqrt(newton @ A @ newton)
    w2, info2, _, tl = oracle.steihaug(A, L, bhat, delta=delta, norm=0, with_len=True)
    assert info2 == 2
    assert abs(np.sqrt(w2 @ A @ w2) - delta) < 1e-12 * delta
    assert abs(tl - delta) < 1e-12 * delta
    np.testing.assert_allclose(w2 / np.linalg.norm(w2), newton / np.linalg.norm(newton),
                               rtol=1e-9, atol=1e-12)
    # a radius between the two lengths of the Newton step, ||w||_2 < delta < ||L^T w||
    # (A's eigenvalues are >= 1, so ||L^T w|| >= ||w||): inside for one norm, outside
    # for the other
    wl, sl = np.linalg.norm(newton), np.sqrt(newton @ A @ newton)
    assert wl < 0.9 * sl
    delta = np.sqrt(wl * sl)
    w4, info4, _ = oracle.steihaug(A, L, bhat, delta=delta, norm=0)
    assert info4 == 2 and abs(np.sqrt(w4 @ A @ w4) - delta) < 1e-12 * delta
    w5, info5, _ = oracle.steihaug(A, L, bhat, delta=delta, norm=1)
    assert info5 in (0, 1)
    np.testing.assert_allclose(w5, newton, rtol=1e-9, atol=1e-12)
    # the other reading (norm 1): the step itself is bounded, ||w||_2 = delta
    delta = 0.3 * np.linalg.norm(newton)
    w3, info3, _, tl = oracle.steihaug(A, L, bhat, delta=delta, norm=1, with_len=True)
    assert info3 == 2
    assert abs(np.linalg.norm(w3) - delta) < 1e-12 * delta
    assert abs(tl - delta) < 1e-12 * delta
    np.testing.assert_allclose(w3 / np.linalg.norm(w3), newton / np.linalg.norm(newton),
                               rtol=1e-9, atol=1e-12)


def test_steihaug_preconditioned_norm_with_a_shift():
    # an indefinite A factored with a shift: the bound of Algorithm 1 is ||L^T w||_2 with
    # L L^T = A + alpha I, i.e. w'(A + alpha I)w = delta^2 at the boundary, not w'Aw
    rng = np.random.default_rng(11)
    m = 6
    Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
    A = Q @ np.diag([5.0, 3.0, 2.0, 1.0, 0.5, -0.2]) @ Q.T
    L, alpha = oracle.chol_shifted(A)
    assert alpha > 0.0
    M = A + alpha * np.eye(m)
    np.testing.assert_allclose(np.tril(L) @ np.tril(L).T, M, rtol=1e-12, atol=1e-12)
    r = rng.standard_normal(m)
    bhat = np.linalg.solve(np.tril(L), r)
    for delta in (0.05, 0.3, 2.0):
        w, info, it, tl = oracle.steihaug(A, L, bhat, delta=delta, norm=0, with_len=True)
        assert np.sqrt(w @ M @ w) <= delta * (1 + 1e-12)
        assert abs(tl - np.sqrt(w @ M @ w)) < 1e-12 * max(1.0, tl)
        if info in (2, 3):
            assert abs(np.sqrt(w @ M @ w) - delta) < 1e-11 * delta
        # a descent step of the model r'w + 1/2 w'Aw
        assert r @ w + 0.5 * w @ A @ w < 0.0


def test_steihaug_negative_curvature_goes_to_boundary():
    A = np.diag([2.0, -1.0])
    L = np.diag([1.0, 1.0])  # identity preconditioner
    L_full = L.copy()
    bhat = np.array([0.0, 1.0])  # gradient only along the negative-curvature direction
    w, info, _ = oracle.steihaug(A, L_full, bhat, delta=0.5)
    assert info == 3
    np.testing.assert_allclose(w, [0.0, -0.5], atol=1e-15)


# ------------------------------------------------------------------------- objectives

def test_dense_eval_closed_form():
    rng = np.random.default_rng(4)
    n = 7
    rec, _, _, _ = synth.dense_records(rng, 1, n)
    Q = rec[0, :n * n].reshape(n, n)
    c = rec[0, n * n:n * n + n]
    d = rec[0, n * n + n:]
    x = rng.standard_normal(n)
    f, g, H = oracle.eval_obj(oracle.OBJ_DENSE, rec[0], x)
    assert abs(f - (0.5 * x @ Q @ x + c @ x + d @ x ** 4)) < 1e-12 * max(1, abs(f))
    np.testing.assert_allclose(g, Q @ x + c + 4 * d * x ** 3, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(H, Q + np.diag(12 * d * x ** 2), rtol=1e-12, atol=1e-12)


def _branch_points(rng, k):
    out = []
    for _ in range(k):
        out.append(np.array([rng.uniform(0.9, 1.1), rng.uniform(0.9, 1.1),
                             rng.uniform(-1, 1), rng.uniform(-1, 1)]))
    return out


def test_branch_gradient_hessian_finite_differences():
    d = synth.branch_batch(16, seed_index=5)
    rng = np.random.default_rng(5)
    for p in range(16):
        rec = d["params"][p].copy()
        if p % 2:
            rec[32] = 0.01  # force the line-limit term active
        for x in _branch_points(rng, 3):
            f, g, H = oracle.eval_obj(oracle.OBJ_BRANCH, rec, x)
            h = 1e-6
            gfd = np.zeros(4)
            Hfd = np.zeros((4, 4))
            for i in range(4):
                e = np.zeros(4)
                e[i] = h
                fp, gp, _ = oracle.eval_obj(oracle.OBJ_BRANCH, rec, x + e)
                fm, gm, _ = oracle.eval_obj(oracle.OBJ_BRANCH, rec, x - e)
                gfd[i] = (fp - fm) / (2 * h)
                Hfd[:, i] = (gp - gm) / (2 * h)
            scale = max(1.0, np.abs(g).max())
            assert np.abs(g - gfd).max() < 1e-6 * scale
            hs = max(1.0, np.abs(H).max())
            assert np.abs(H - Hfd).max() < 1e-6 * hs
            np.testing.assert_allclose(H, H.T, rtol=0, atol=1e-9 * hs)


def test_branch_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    d = synth.branch_batch(8, seed_index=6)
    rng = np.random.default_rng(6)

    def f_torch(rec, x):
        cf, lam, tg, rh = rec[0:8], rec[8:16], rec[16:24], rec[24:32]
        vi, vj, ti, tj = x[0], x[1], x[2], x[3]
        wi, wj = vi * vi, vj * vj
        wR = vi * vj * torch.cos(ti - tj)
        wI = vi * vj * torch.sin(ti - tj)
        # eqs. pij-qji written out independently of the oracle's coefficient table
        pij = cf[0] * wi - cf[2] * wR + cf[3] * wI
        qij = cf[1] * wi - cf[3] * wR - cf[2] * wI
        pji = cf[4] * wj - cf[6] * wR - cf[7] * wI
        qji = cf[5] * wj - cf[7] * wR + cf[6] * wI
        F = torch.stack([pij, qij, pji, qji, wi, wj, ti, tj])
        r = F - tg
        val = (lam * r + 0.5 * rh * r * r).sum()
        for a, b in ((pij, qij), (pji, qji)):
            m = a * a + b * b - rec[32]
            val = val + 0.5 * rec[33] * torch.clamp(m, min=0.0) ** 2
        return val

    for p in range(8):
        rec = d["params"][p].copy()
        if p % 2:
            rec[32] = 0.02
        rt = torch.tensor(rec, dtype=torch.float64)
        for x in _branch_points(rng, 3):
            xt = torch.tensor(x, dtype=torch.float64, requires_grad=True)
            ft = f_torch(rt, xt)
            gt, = torch.autograd.grad(ft, xt, create_graph=True)
            Ht = torch.stack([torch.autograd.grad(gt[i], xt, retain_graph=True)[0]
                              for i in range(4)])
            f, g, H = oracle.eval_obj(oracle.OBJ_BRANCH, rec, x)
            assert abs(f - ft.item()) <= 1e-10 * max(1, abs(f))
            np.testing.assert_allclose(g, gt.detach().numpy(), rtol=1e-10, atol=1e-9)
            np.testing.assert_allclose(H, Ht.detach().numpy(), rtol=1e-10, atol=1e-8)


def test_branch_flows_match_complex_power():
    """p_ij + j q_ij = V_i conj(I_ij) for the pi-model with series y and charging bc."""
    rng = np.random.default_rng(7)
    r, x, bc, _ = synth.random_lines(rng, 20)
    coef = synth.line_coefficients(r, x, bc)
    for k in range(20):
        rec = np.zeros(36)
        rec[0:8] = coef[k]
        rec[24:32] = 1.0  # unit penalties, zero multipliers and targets:
        # f = 1/2 sum F_k^2 ; recover the flows through f at a point and its gradient
        vi, vj = rng.uniform(0.9, 1.1, 2)
        ti, tj = rng.uniform(-0.5, 0.5, 2)
        Vi = vi * np.exp(1j * ti)
        Vj = vj * np.exp(1j * tj)
        y = 1.0 / (r[k] + 1j * x[k])
        Iij = y * (Vi - Vj) + 1j * bc[k] / 2 * Vi
        Iji = y * (Vj - Vi) + 1j * bc[k] / 2 * Vj
        Sij = Vi * np.conj(Iij)
        Sji = Vj * np.conj(Iji)
        want = np.array([Sij.real, Sij.imag, Sji.real, Sji.imag])
        # f = 1/2 (sum flows^2 + vi^4 + vj^4 + ti^2 + tj^2); subtract the voltage terms
        f, _, _ = oracle.eval_obj(oracle.OBJ_BRANCH, rec, np.array([vi, vj, ti, tj]))
        rest = 0.5 * (vi ** 4 + vj ** 4 + ti ** 2 + tj ** 2)
        assert abs((f - rest) - 0.5 * (want ** 2).sum()) < 1e-12
        # and flow by flow: a unit multiplier on one pair returns that flow
        for a in range(4):
            rec2 = np.zeros(36)
            rec2[0:8] = coef[k]
            rec2[8 + a] = 1.0
            f2, _, _ = oracle.eval_obj(oracle.OBJ_BRANCH, rec2, np.array([vi, vj, ti, tj]))
            assert abs(f2 - want[a]) < 1e-12


# ---------------------------------------------------------------------------- TRON

def _solve(kind, rec, l, u, x0, **over):
    return oracle.tron_solve(kind, rec, l, u, x0, 1.0, oracle.default_opts(**over))


def test_hs45_printed_solution():
    """Sec. 4.2 footnote: the solution of f = 120 - prod x_i, x_i <= i is x*_i = i."""
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "hs45.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 7
    for row in rows:
        n = int(row[0])
        fstar = float(row[1])
        xstar = np.array([float(v) for v in row[2:]])
        d = synth.hs45_batch(1, n)
        r = oracle.tron_solve(oracle.OBJ_HS45, None, d["l"][0], d["u"][0], d["x0"][0], 1.0)
        assert r["status"] == oracle.CONVERGED
        np.testing.assert_allclose(r["x"], xstar, rtol=0, atol=1e-9)
        assert abs(r["f"] - fstar) <= 1e-9 * max(1, abs(fstar))
        assert fstar == 120 - math.factorial(n)


def test_separable_quadratic_closed_form():
    rng = np.random.default_rng(8)
    for n in (1, 3, 8, 32):
        for _ in range(5):
            rec, l, u, x0 = synth.dense_records(rng, 1, n, quartic=0.0, diag_only=True)
            q = np.diag(rec[0, :n * n].reshape(n, n))
            c = rec[0, n * n:n * n + n]
            want = np.clip(-c / q, l[0], u[0])
            r = _solve(oracle.OBJ_DENSE, rec[0], l[0], u[0], x0[0])
            assert r["status"] == oracle.CONVERGED and r["pg"] <= 1e-6
            np.testing.assert_allclose(r["x"], want, rtol=0, atol=1e-6)
            fwant = 0.5 * (q * want * want).sum() + c @ want
            assert abs(r["f"] - fwant) <= 1e-8 * max(1.0, abs(fwant))


def _bisect(fun, a, b, it=200):
    fa = fun(a)
    for _ in range(it):
        m = 0.5 * (a + b)
        fm = fun(m)
        if (fm > 0) == (fa > 0):
            a, fa = m, fm
        else:
            b = m
    return 0.5 * (a + b)


def test_separable_quartic_closed_form():
    rng = np.random.default_rng(9)
    for n in (2, 5, 16):
        rec, l, u, x0 = synth.dense_records(rng, 1, n, quartic=0.1, diag_only=True)
        q = np.diag(rec[0, :n * n].reshape(n, n))
        c = rec[0, n * n:n * n + n]
        want = np.zeros(n)
        for i in range(n):
            # unique real root of q x + c + 0.4 x^3 (strictly increasing), then clip
            root = _bisect(lambda t: q[i] * t + c[i] + 0.4 * t ** 3, -100.0, 100.0)
            want[i] = min(max(root, l[0, i]), u[0, i])
        r = _solve(oracle.OBJ_DENSE, rec[0], l[0], u[0], x0[0])
        assert r["status"] == oracle.CONVERGED
        np.testing.assert_allclose(r["x"], want, rtol=0, atol=1e-6)


def test_dense_convex_vs_lbfgsb():
    scipy_opt = pytest.importorskip("scipy.optimize")
    d = synth.dense_batch(12, 32, seed_index=1)
    for p in range(12):
        rec = d["params"][p]
        n = 32
        Q = rec[:n * n].reshape(n, n)
        c = rec[n * n:n * n + n]
        dd = rec[n * n + n:]

        def fg(x):
            return (0.5 * x @ Q @ x + c @ x + dd @ x ** 4, Q @ x + c + 4 * dd * x ** 3)

        res = scipy_opt.minimize(fg, d["x0"][p], jac=True, method="L-BFGS-B",
                                 bounds=list(zip(d["l"][p], d["u"][p])),
                                 options=dict(gtol=1e-12, ftol=1e-15, maxiter=10000))
        r = _solve(oracle.OBJ_DENSE, rec, d["l"][p], d["u"][p], d["x0"][p])
        assert r["status"] == oracle.CONVERGED
        np.testing.assert_allclose(r["x"], res.x, rtol=0, atol=1e-6)
        assert abs(r["f"] - res.fun) <= 1e-8 * max(1.0, abs(res.fun))


def test_two_variable_bruteforce_grid():
    """Nonconvex 2-variable problems: the oracle's answer is a local minimiser on the
    box (no lower value in a grid neighbourhood) and the global one when the grid's
    best point lies in its basin (checked from that start)."""
    rng = np.random.default_rng(10)
    ng = 2001
    for trial in range(6):
        A = rng.standard_normal((2, 2))
        Q = 0.5 * (A + A.T) * 4.0  # indefinite in general
        c = rng.normal(0, 2, 2)
        dq = np.array([0.3, 0.3])
        rec = np.concatenate([Q.ravel(), c, dq])
        l = np.array([-2.0, -1.5])
        u = np.array([1.5, 2.0])
        X, Y = np.meshgrid(np.linspace(l[0], u[0], ng), np.linspace(l[1], u[1], ng),
                           indexing="ij")
        F = (0.5 * (Q[0, 0] * X * X + 2 * Q[0, 1] * X * Y + Q[1, 1] * Y * Y) + c[0] * X
             + c[1] * Y + dq[0] * X ** 4 + dq[1] * Y ** 4)
        i, j = np.unravel_index(np.argmin(F), F.shape)
        xg = np.array([X[i, j], Y[i, j]])
        r = _solve(oracle.OBJ_DENSE, rec, l, u, xg)
        assert r["status"] == oracle.CONVERGED
        h = (u - l) / (ng - 1)
        assert np.all(np.abs(r["x"] - xg) <= 1.01 * h)
        assert r["f"] <= F[i, j] + 1e-12
        # from the centre: a KKT point that no grid point near it improves on
        r2 = _solve(oracle.OBJ_DENSE, rec, l, u, np.zeros(2))
        assert r2["status"] == oracle.CONVERGED
        ii = int(round((r2["x"][0] - l[0]) / h[0]))
        jj = int(round((r2["x"][1] - l[1]) / h[1]))
        win = F[max(ii - 5, 0):ii + 6, max(jj - 5, 0):jj + 6]
        assert r2["f"] <= win.min() + 1e-9


def test_kkt_on_dense_workload_sample():
    d = synth.dense_batch(64, 32, seed_index=1)
    r = oracle.tron_batch(oracle.OBJ_DENSE, d["params"], d["l"], d["u"], d["x0"],
                          d["delta0"])
    assert np.all(r["status"] == oracle.CONVERGED)
    n = 32
    for p in range(64):
        rec = d["params"][p]
        Q = rec[:n * n].reshape(n, n)
        x = r["x"][p]
        g = Q @ x + rec[n * n:n * n + n] + 4 * rec[n * n + n:] * x ** 3
        pg = g.copy()
        pg[(x <= d["l"][p]) & (g > 0)] = 0
        pg[(x >= d["u"][p]) & (g < 0)] = 0
        assert np.abs(pg).max() <= 1e-6
        assert np.all(x >= d["l"][p]) and np.all(x <= d["u"][p])


def test_branch_workload_kkt():
    d = synth.branch_batch(256, seed_index=0)
    r = oracle.tron_batch(oracle.OBJ_BRANCH, d["params"], d["l"], d["u"], d["x0"],
                          d["delta0"])
    assert np.all(r["status"] == oracle.CONVERGED)
    for p in range(0, 256, 7):
        x = r["x"][p]
        # gradient by central differences, independent of the oracle's derivative code
        g = np.zeros(4)
        for i in range(4):
            e = np.zeros(4)
            e[i] = 1e-7
            fp, _, _ = oracle.eval_obj(oracle.OBJ_BRANCH, d["params"][p], x + e)
            fm, _, _ = oracle.eval_obj(oracle.OBJ_BRANCH, d["params"][p], x - e)
            g[i] = (fp - fm) / 2e-7
        pg = g.copy()
        pg[(x <= d["l"][p]) & (g > 0)] = 0
        pg[(x >= d["u"][p]) & (g < 0)] = 0
        # central differences with h = 1e-7 are accurate to about 1e-6 relative to |g|
        assert np.abs(pg).max() <= 1e-6 + 1e-6 * max(1.0, np.abs(g).max())


def test_status_codes_for_bad_input():
    n = 3
    rec, l, u, x0 = synth.dense_records(np.random.default_rng(11), 1, n)
    lb = l[0].copy()
    lb[1] = u[0][1] + 1.0
    r = _solve(oracle.OBJ_DENSE, rec[0], lb, u[0], x0[0])
    assert r["status"] == oracle.BAD_BOUNDS and r["iters"] == 0
    rec2 = rec[0].copy()
    rec2[n * n] = np.nan
    r = _solve(oracle.OBJ_DENSE, rec2, l[0], u[0], x0[0])
    assert r["status"] == oracle.NONFINITE
    r = _solve(oracle.OBJ_DENSE, rec[0], l[0], u[0], x0[0], max_outer=1, gtol=1e-300)
    assert r["status"] == oracle.MAX_ITER and r["iters"] == 1


def test_branch_entries_that_enter_f_only_past_the_line_limit():
    # reading R19: an infinite or NaN line limit leaves the penalty off (m > 0 is false),
    # so the solve is the one with a huge finite limit, bit for bit; an infinite line
    # weight does not matter while no line is over; an infinite target makes f infinite
    d = synth.branch_batch(6, seed_index=85)
    base = d["params"].copy()
    base[:, 32] = 1e300
    ref = oracle.tron_batch(d["kind"], base, d["l"], d["u"], d["x0"], d["delta0"])
    assert np.all(ref["status"] == oracle.CONVERGED)
    for smax2 in (np.inf, np.nan):
        p = base.copy()
        p[:, 32] = smax2
        r = oracle.tron_batch(d["kind"], p, d["l"], d["u"], d["x0"], d["delta0"])
        np.testing.assert_array_equal(r["status"], ref["status"])
        np.testing.assert_array_equal(r["x"], ref["x"])
    p = base.copy()
    p[:, 33] = np.inf
    r = oracle.tron_batch(d["kind"], p, d["l"], d["u"], d["x0"], d["delta0"])
    np.testing.assert_array_equal(r["x"], ref["x"])
    p = base.copy()
    p[0, 20] = np.inf
    r = oracle.tron_batch(d["kind"], p, d["l"], d["u"], d["x0"], d["delta0"])
    assert r["status"][0] == oracle.NONFINITE


def test_newton_step_solves_an_interior_quadratic_in_one_iteration():
    """Strictly convex quadratic with its minimiser inside the box and a large radius:
    the Cauchy point, the complete factorization (Sec. 4.3: one PCG iteration) and the
    back transform give the exact Newton step, so one outer iteration converges."""
    rng = np.random.default_rng(12)
    for n in (3, 8, 20):
        G = rng.standard_normal((n, n))
        Q = G @ G.T + n * np.eye(n)
        xs = rng.uniform(-0.5, 0.5, n)
        c = -Q @ xs
        rec = np.concatenate([Q.ravel(), c, np.zeros(n)])
        r = oracle.tron_solve(oracle.OBJ_DENSE, rec, -np.ones(n) * 10, np.ones(n) * 10,
                              np.zeros(n), 1e3)
        assert r["status"] == oracle.CONVERGED
        assert r["iters"] == 1, r["iters"]
        np.testing.assert_allclose(r["x"], xs, rtol=0, atol=1e-9)
        assert r["counters"]["cg_iters"] == 1


def test_converged_start_takes_no_iteration():
    n = 4
    Q = np.eye(n)
    rec = np.concatenate([Q.ravel(), np.zeros(n), np.zeros(n)])
    r = _solve(oracle.OBJ_DENSE, rec, -np.ones(n), np.ones(n), np.zeros(n))
    assert r["status"] == oracle.CONVERGED and r["iters"] == 0


# ---------------------------------------------------------------------------- ADMM

def _small_net(nbus=12, seed=3):
    return synth.network(nbus, nchord=max(1, nbus // 4), ngen=max(1, nbus // 3),
                         rng=np.random.default_rng(seed))


def test_admm_generator_update_is_scalar_qp_minimiser():
    net = _small_net()
    A = oracle.Admm(net)
    A.run(3)
    pre = {k: v.copy() for k, v in A.arrays.items()}
    A.run(1)
    rho = 400.0
    for g in range(len(net["gen_bus"])):
        pt, qt = pre["gen_tilde"][g]
        lp, lq = pre["gen_lam"][g]
        c2, c1 = net["gen_c2"][g], net["gen_c1"][g]
        # brute force on a fine grid of the box, then compare
        pg = np.linspace(net["gen_pmin"][g], net["gen_pmax"][g], 200001)
        fp = c2 * pg * pg + c1 * pg + lp * (pg - pt) + 0.5 * rho * (pg - pt) ** 2
        qg = np.linspace(net["gen_qmin"][g], net["gen_qmax"][g], 200001)
        fq = lq * (qg - qt) + 0.5 * rho * (qg - qt) ** 2
        hp = pg[1] - pg[0]
        hq = qg[1] - qg[0]
        assert abs(A.arrays["gen_pq"][g, 0] - pg[np.argmin(fp)]) <= hp
        assert abs(A.arrays["gen_pq"][g, 1] - qg[np.argmin(fq)]) <= hq


def _ends(net):
    nb = net["nbus"]
    ends = [[] for _ in range(nb)]
    for k, (i, j) in enumerate(zip(net["br_from"], net["br_to"])):
        ends[i].append((k, 0))
        ends[j].append((k, 1))
    gens = [[] for _ in range(nb)]
    for g, b in enumerate(net["gen_bus"]):
        gens[b].append(g)
    return ends, gens


def test_admm_bus_update_kkt_and_multipliers():
    net = _small_net(15, seed=4)
    A = oracle.Admm(net)
    A.run(2)
    pre = {k: v.copy() for k, v in A.arrays.items()}
    hp, hd = A.run(1)
    st = A.arrays
    rho = 400.0
    ends, gens = _ends(net)
    for b in range(net["nbus"]):
        # balance: sum_g pt_g - sum_e pt_e = p_d (no shunts)
        sp = sum(st["gen_tilde"][g, 0] for g in gens[b]) - sum(
            st["br_tilde"][k, 2 * s] for k, s in ends[b])
        sq = sum(st["gen_tilde"][g, 1] for g in gens[b]) - sum(
            st["br_tilde"][k, 2 * s + 1] for k, s in ends[b])
        assert abs(sp - net["bus_pd"][b]) < 1e-12 * max(1, abs(sp))
        assert abs(sq - net["bus_qd"][b]) < 1e-12 * max(1, abs(sq))
        # stationarity: rho (xt - a) equal to -mu on generator copies and +mu on flows
        mus = []
        for g in gens[b]:
            a = st["gen_pq"][g, 0] + pre["gen_lam"][g, 0] / rho
            mus.append(-rho * (st["gen_tilde"][g, 0] - a))
        for k, s in ends[b]:
            a = st["br_val"][k, 2 * s] + pre["br_lam"][k, 2 * s] / rho
            mus.append(rho * (st["br_tilde"][k, 2 * s] - a))
        assert max(mus) - min(mus) < 1e-9 * max(1, max(abs(m) for m in mus))
        # voltage / angle copies: the mean of x + lambda/rho over incident ends
        if ends[b]:
            aw = np.mean([st["br_val"][k, 4 + s] + pre["br_lam"][k, 4 + s] / rho
                          for k, s in ends[b]])
            at = np.mean([st["br_val"][k, 6 + s] + pre["br_lam"][k, 6 + s] / rho
                          for k, s in ends[b]])
            assert abs(st["bus_w"][b] - aw) < 1e-12
            assert abs(st["bus_th"][b] - at) < 1e-12
    # multiplier update and residuals recomputed from the state
    xs, xt, xp = [], [], []
    for g in range(len(net["gen_bus"])):
        for a in range(2):
            xs.append(st["gen_pq"][g, a])
            xt.append(st["gen_tilde"][g, a])
            xp.append(pre["gen_tilde"][g, a])
            np.testing.assert_allclose(
                st["gen_lam"][g, a],
                pre["gen_lam"][g, a] + rho * (st["gen_pq"][g, a] - st["gen_tilde"][g, a]),
                rtol=1e-12, atol=1e-9)
    for k, (i, j) in enumerate(zip(net["br_from"], net["br_to"])):
        tild = [st["br_tilde"][k, 0], st["br_tilde"][k, 1], st["br_tilde"][k, 2],
                st["br_tilde"][k, 3], st["bus_w"][i], st["bus_w"][j], st["bus_th"][i],
                st["bus_th"][j]]
        prev = [pre["br_tilde"][k, 0], pre["br_tilde"][k, 1], pre["br_tilde"][k, 2],
                pre["br_tilde"][k, 3], pre["bus_w"][i], pre["bus_w"][j], pre["bus_th"][i],
                pre["bus_th"][j]]
        for a in range(8):
            xs.append(st["br_val"][k, a])
            xt.append(tild[a])
            xp.append(prev[a])
            np.testing.assert_allclose(
                st["br_lam"][k, a], pre["br_lam"][k, a] + rho * (st["br_val"][k, a] - tild[a]),
                rtol=1e-12, atol=1e-9)
    xs, xt, xp = map(np.asarray, (xs, xt, xp))
    assert abs(hp[0] - np.linalg.norm(xs - xt)) <= 1e-12 * max(1, hp[0])
    assert abs(hd[0] - rho * np.linalg.norm(xt - xp)) <= 1e-12 * max(1, hd[0])


def test_admm_branch_values_are_tron_solutions():
    net = _small_net(10, seed=5)
    A = oracle.Admm(net)
    A.run(2)
    recs = [A.branch_record(k) for k in range(len(net["br_from"]))]
    x_before = A.arrays["br_x"].copy()
    d_before = A.arrays["br_delta"].copy()
    # re-solve the records the next iteration will see, independently, and compare
    A.run(1)
    for k, rec in enumerate(recs[:5]):
        r = oracle.tron_solve(oracle.OBJ_BRANCH, rec, [0.9, 0.9, -2 * np.pi, -2 * np.pi],
                              [1.1, 1.1, 2 * np.pi, 2 * np.pi], x_before[k], d_before[k])
        np.testing.assert_array_equal(r["x"], A.arrays["br_x"][k])


def test_admm_residuals_decay_on_convex_case():
    """Zero line charging, lightly loaded, small network: the residuals fall by orders
    of magnitude over the iterations."""
    net = _small_net(6, seed=6)
    hp, hd = oracle.Admm(net).run(300)
    assert hp[-1] < 1e-2 * hp[:5].max()
    assert hd[-1] < 1e-2 * hd[:5].max()
    assert np.all(np.isfinite(hp)) and np.all(np.isfinite(hd))


def test_admm_two_bus_by_hand():
    """Radial 2-bus case: after the bus update the flows balance the loads exactly:
    bus 0 holds the generator, bus 1 only a load, so pt_ji = -p_d1 and qt_ji = -q_d1."""
    net = synth.network(2, nchord=0, ngen=1, rng=np.random.default_rng(7))
    net["gen_bus"] = np.array([0], dtype=np.int32)
    net["br_from"] = np.array([0], dtype=np.int32)
    net["br_to"] = np.array([1], dtype=np.int32)
    A = oracle.Admm(net)
    A.run(5)
    st = A.arrays
    assert abs(st["br_tilde"][0, 2] + net["bus_pd"][1]) < 1e-12
    assert abs(st["br_tilde"][0, 3] + net["bus_qd"][1]) < 1e-12
    assert abs(st["gen_tilde"][0, 0] - st["br_tilde"][0, 0] - net["bus_pd"][0]) < 1e-12


# ------------------------------------------------ multi-period generator and ADMM

def _genramp_points(rng, rec, T, k):
    """points away from the ramp kinks (| |p_t - p_{t-1}| - R | > 1e-3)"""
    out = []
    R = rec[4]
    while len(out) < k:
        x = rng.uniform(0.0, 1.2, T)
        d = np.abs(np.diff(x))
        if np.all(np.abs(d - R) > 1e-3) and np.any(d > R):
            out.append(x)
    return out


def test_genramp_gradient_hessian_finite_differences():
    d = synth.genramp_batch(8, 7, seed_index=30)
    rng = np.random.default_rng(30)
    for p in range(8):
        rec = d["params"][p]
        for x in _genramp_points(rng, rec, 7, 3):
            f, g, H = oracle.eval_obj(oracle.OBJ_GENRAMP, rec, x)
            h = 1e-6
            gfd = np.zeros(7)
            Hfd = np.zeros((7, 7))
            for i in range(7):
                e = np.zeros(7)
                e[i] = h
                fp, gp, _ = oracle.eval_obj(oracle.OBJ_GENRAMP, rec, x + e)
                fm, gm, _ = oracle.eval_obj(oracle.OBJ_GENRAMP, rec, x - e)
                gfd[i] = (fp - fm) / (2 * h)
                Hfd[:, i] = (gp - gm) / (2 * h)
            scale = max(1.0, np.abs(g).max())
            assert np.abs(g - gfd).max() < 1e-6 * scale
            hs = max(1.0, np.abs(H).max())
            assert np.abs(H - Hfd).max() < 1e-5 * hs
            # tridiagonal
            assert np.all(np.triu(H, 2) == 0.0) and np.all(np.tril(H, -2) == 0.0)


def test_genramp_without_binding_ramps_is_the_per_period_closed_form():
    # R beyond any possible step: the periods separate and each is the box-clipped
    # minimiser of c2 p^2 + c1 p + lambda (p - t) + rho/2 (p - t)^2
    d = synth.genramp_batch(20, 12, seed_index=31)
    for p in range(20):
        rec = d["params"][p].copy()
        rec[4] = 1e6
        c2, c1, rho = rec[0], rec[1], rec[2]
        lam, tgt = rec[8:20], rec[20:32]
        closed = np.clip((rho * tgt - lam - c1) / (2 * c2 + rho), d["l"][p], d["u"][p])
        r = _solve(oracle.OBJ_GENRAMP, rec, d["l"][p], d["u"][p], d["x0"][p])
        assert r["status"] == oracle.CONVERGED
        np.testing.assert_allclose(r["x"], closed, rtol=0, atol=1e-9)


def test_genramp_binding_ramps_vs_lbfgsb():
    scipy_opt = pytest.importorskip("scipy.optimize")
    T = 9
    d = synth.genramp_batch(16, T, seed_index=32)
    for p in range(16):
        rec = d["params"][p]
        c2, c1, rho, rr, R = rec[:5]
        lam, tgt = rec[8:8 + T], rec[8 + T:]

        def fg(x):
            r = x - tgt
            f = np.sum(c2 * x * x + c1 * x + lam * r + 0.5 * rho * r * r)
            g = 2 * c2 * x + c1 + lam + rho * r
            dd = np.diff(x)
            e = np.maximum(np.abs(dd) - R, 0.0)
            f += 0.5 * rr * np.sum(e * e)
            w = rr * e * np.sign(dd)
            g[1:] += w
            g[:-1] -= w
            return f, g

        res = scipy_opt.minimize(fg, d["x0"][p], jac=True, method="L-BFGS-B",
                                 bounds=list(zip(d["l"][p], d["u"][p])),
                                 options=dict(gtol=1e-13, ftol=1e-16, maxiter=20000))
        r = _solve(oracle.OBJ_GENRAMP, rec, d["l"][p], d["u"][p], d["x0"][p])
        assert r["status"] == oracle.CONVERGED
        np.testing.assert_allclose(r["x"], res.x, rtol=0, atol=1e-6)
        assert abs(r["f"] - res.fun) <= 1e-8 * max(1.0, abs(res.fun))


def test_multiperiod_admm_without_binding_ramps_equals_single_period_runs():
    net = _small_net(30, seed=33)
    scale = [0.85, 1.0, 1.15]
    mp = oracle.MultiPeriodAdmm(net, scale, ramp=1e6)
    hp, hd = mp.run(12)
    pr2 = np.zeros(12)
    du2 = np.zeros(12)
    for t, s in enumerate(scale):
        nt = dict(net, bus_pd=net["bus_pd"] * s, bus_qd=net["bus_qd"] * s)
        a = oracle.Admm(nt)
        p1, d1 = a.run(12)
        pr2 += p1 ** 2
        du2 += d1 ** 2
        for k in ("gen_pq", "gen_lam", "bus_w", "bus_th", "br_x", "br_lam"):
            np.testing.assert_allclose(mp.state(t)[k], a.arrays[k], rtol=1e-9, atol=1e-9,
                                       err_msg=k)
    np.testing.assert_allclose(hp, np.sqrt(pr2), rtol=1e-9)
    np.testing.assert_allclose(hd, np.sqrt(du2), rtol=1e-9)


def test_multiperiod_admm_generator_step_satisfies_chain_kkt():
    # after an iteration, the chain problem built from the state before it is solved:
    # the projected gradient of its objective at the new p is below gtol
    net = _small_net(30, seed=34)
    mp = oracle.MultiPeriodAdmm(net, synth.load_profile(6), ramp=0.01, rho_ramp=1e4)
    mp.run(3)
    recs = [mp.genramp_record(g) for g in range(len(net["gen_bus"]))]
    p_before = np.array([mp.state(t)["gen_pq"][:, 0] for t in range(6)]).T.copy()
    mp.run(1)
    p_after = np.array([mp.state(t)["gen_pq"][:, 0] for t in range(6)]).T
    assert np.abs(p_after - p_before).max() > 0
    for g, rec in enumerate(recs):
        f, gr, _ = oracle.eval_obj(oracle.OBJ_GENRAMP, rec, p_after[g])
        lo = np.full(6, net["gen_pmin"][g])
        hi = np.full(6, net["gen_pmax"][g])
        assert oracle.pgnorm(p_after[g], gr, lo, hi) <= 1e-6


# ------------------------------------------- step rules, one iteration computed by hand
# Readings R2 (Cauchy search), R5 (PCG norm), R7 (radius update) and the projected
# search of Algorithm 1, each pinned by a case small enough to follow on paper: a dense
# problem f = 1/2 x'Qx + c'x + sum d x^4 stopped after max_outer iterations, with the
# returned x, radius, status and trial counters compared with the values derived in the
# comments.  mu0 = 0.01, interpolation x0.1, extrapolation x10, eta = (1e-4, .25, .75),
# sigma1 = 0.25, sigma3 = 4, projected-search factor 0.5.

def _dense1(Q, c, d, x0, delta, max_outer=1, l=-10.0, u=10.0, **opt):
    Q = np.atleast_2d(np.asarray(Q, dtype=float))
    n = Q.shape[0]
    rec = np.concatenate([Q.ravel(), np.asarray(c, float).ravel(), np.asarray(d, float).ravel()])
    return oracle.tron_solve(oracle.OBJ_DENSE, rec, np.broadcast_to(l, (n,)),
                             np.broadcast_to(u, (n,)), x0, delta,
                             opts=oracle.default_opts(max_outer=max_outer, **opt))


def test_cauchy_interpolation_preconditioned_boundary_and_expansion():
    # f = 5 x^2 - x, x0 = 0, delta = 0.015: g = -1, H = 10.
    # Cauchy: alpha = 1 (s = 1: q = -1 + 5 > 0.01 g's) and alpha = 0.1 (||s|| = 0.1 >
    # delta) fail, alpha = 0.01 holds (s = 0.01, q = -0.0095): three trials, x_c = 0.01.
    # Subspace: r = g + H s = -0.9, L = sqrt(10); the CG iterate s_hat = -bhat has
    # ||s_hat|| = 0.9/sqrt(10) > delta, so CG stops on the boundary ||s_hat|| = delta and
    # w = L^-T s_hat = 0.015/sqrt(10); the full step passes the projected search.
    # The model is exact (rho = 1 > eta2) and the subspace step reached its bound
    # (beta ||s_hat|| = delta), so delta = 4 * 0.015.
    r = _dense1([10.0], [-1.0], [0.0], [0.0], 0.015)
    assert r["status"] == oracle.MAX_ITER and r["iters"] == 1
    assert r["counters"]["cauchy_trials"] == 3 and r["counters"]["proj_trials"] == 1
    assert abs(r["x"][0] - (0.01 + 0.015 / math.sqrt(10.0))) < 1e-15
    assert r["delta"] == 0.06
    # the other norm reading bounds w itself: w = 0.015, x = 0.025; the radius update
    # then measures ||x+ - x|| = 0.025 >= 0.99 delta and expands as well
    r = _dense1([10.0], [-1.0], [0.0], [0.0], 0.015, tr_norm=1)
    assert abs(r["x"][0] - 0.025) < 1e-15 and r["delta"] == 0.06


def test_cauchy_alpha_persists_between_iterations():
    # the case above for two iterations: x1 = 0.01 + 0.015/sqrt(10), g1 = 10 x1 - 1,
    # delta = 0.06.  The second search starts from the stored alpha = 0.01: it holds
    # (s = 0.01 |g1| = 0.0085, within delta), the extrapolated 0.1 does not (||s|| =
    # 0.085 > 0.06): two trials (restarting at 1 would take three).  x_c = x1 - 0.01 g1,
    # r = 0.9 g1, CG stops on the boundary again: w = 0.06/sqrt(10), delta = 0.24.
    r = _dense1([10.0], [-1.0], [0.0], [0.0], 0.015, max_outer=2)
    x1 = 0.01 + 0.015 / math.sqrt(10.0)
    g1 = 10.0 * x1 - 1.0
    assert r["status"] == oracle.MAX_ITER and r["iters"] == 2
    assert r["counters"]["cauchy_trials"] == 3 + 2
    assert abs(r["x"][0] - (x1 - 0.01 * g1 + 0.06 / math.sqrt(10.0))) < 1e-14
    assert abs(r["delta"] - 0.24) < 1e-15


def test_cauchy_extrapolation_stops_at_the_largest_breakpoint():
    # f = 0.0005 x^2 - x on [-10, 10], x0 = 0, delta = 100: alpha = 1 holds (q = -0.9995),
    # the only breakpoint along -g is 10, alpha = 10 holds (s = 10, q = -9.95) and the
    # search stops there (alpha is no longer below the breakpoint): two trials.  x_c = 10
    # is on the bound, the free set is empty, the step is accepted (rho = 1) but is far
    # inside the radius (10 < 0.99 * 100): delta stays 100.  At x = 10 the gradient
    # -0.99 pushes against the bound: converged after one iteration.
    r = _dense1([0.001], [-1.0], [0.0], [0.0], 100.0)
    assert r["status"] == oracle.CONVERGED and r["iters"] == 1
    assert r["counters"]["cauchy_trials"] == 2 and r["counters"]["proj_trials"] == 0
    assert r["x"][0] == 10.0 and r["delta"] == 100.0


def test_radius_shrinks_to_a_quarter_of_the_shorter_of_step_and_radius():
    # f = 1/2 x^2 - x + x^4, x0 = 0, delta = 2: the model 1/2 s^2 - s is minimised by
    # the Cauchy point alpha = 1 (x_c = 1, alpha = 10 exceeds the radius), the subspace
    # step is zero (r = 0).  f(1) = 0.5 > f(0) = 0: rho ~ -1, the step is rejected and
    # delta = 0.25 * min(||s|| = 1, 2) = 0.25.
    r = _dense1([1.0], [-1.0], [1.0], [0.0], 2.0)
    assert r["status"] == oracle.MAX_ITER and r["iters"] == 1
    assert r["x"][0] == 0.0 and r["delta"] == 0.25
    assert r["counters"]["cauchy_trials"] == 2


# f = 1/2 x^2 - x + d x^4, x0 = 0: the step is s = 1 (Cauchy point alpha = 1, the
# model's minimiser), pred = 0.5, ared = 0.5 - d, rho = 1 - 2d (> eta0: accepted)
RADIUS_CASES = [
    (0.25, 1.0, 1.0, 1.0),      # rho = 0.5: accepted, radius kept
    (0.05, 1.0, 1.0, 4.0),      # rho = 0.9 > eta2 and ||s|| = delta: expanded x4
    (0.05, 1.005, 1.0, 4.02),   # ||s|| = 1 >= 0.99 * 1.005: expanded
    (0.05, 1.02, 1.0, 1.02),    # ||s|| = 1 < 0.99 * 1.02: kept
    (0.40, 1.0, 1.0, 0.25),     # rho = 0.2 < eta1: accepted, and shrunk to 0.25 * 1
]


def _radius_case(d, delta0, x1, delta1):
    r = _dense1([1.0], [-1.0], [d], [0.0], delta0)
    assert r["iters"] == 1 and r["x"][0] == x1
    assert abs(r["delta"] - delta1) < 1e-15


@pytest.mark.parametrize("d,delta0,x1,delta1", RADIUS_CASES)
def test_radius_update_by_ratio_and_step_length(d, delta0, x1, delta1):
    _radius_case(d, delta0, x1, delta1)


def radius_update_all_cases():
    for case in RADIUS_CASES:
        _radius_case(*case)


def test_projected_search_halves_the_step_until_the_model_decreases():
    # Q = [[1, .8], [.8, 1]], c = (-1, 1), box [-10, 2] x [-10, 10], x0 = 0, delta = 100.
    # Cauchy: alpha = 1 holds (s = (1, -1), q = -2 + 0.2); alpha = 10 (s = (2, -10),
    # q = -12 + 36) fails: x_c = (1, -1), model gradient r = c + Q s = (-0.8, 0.8).
    # Newton step w = -Q^-1 r = (4, -4) (||s_hat||^2 = r'Q^-1 r = 6.4, inside).
    # beta = 1: P[x_c + w] = (2, -5), d = (1, -4): r'd = -4, d'Qd = 10.6, the model change
    # -4 + 5.3 > 0.01 r'd -- fails.  beta = 1/2: P[x_c + w/2] = (2, -3), d = (1, -2):
    # r'd = -2.4, d'Qd = 1.8, -2.4 + 0.9 <= -0.024 -- holds.  x1 = (2, -3) (variable 1 now
    # active, which ends the pass), accepted (quadratic: rho = 1), delta kept (the
    # step's pieces are ||s_c|| = sqrt 2 and ||s_hat|| / 2, far inside 100).
    r = _dense1([[1.0, 0.8], [0.8, 1.0]], [-1.0, 1.0], [0.0, 0.0], [0.0, 0.0], 100.0,
                l=np.array([-10.0, -10.0]), u=np.array([2.0, 10.0]))
    assert r["status"] == oracle.MAX_ITER and r["iters"] == 1
    assert r["counters"]["cauchy_trials"] == 2 and r["counters"]["proj_trials"] == 2
    np.testing.assert_allclose(r["x"], [2.0, -3.0], rtol=0, atol=1e-14)
    assert r["delta"] == 100.0


def test_guard_scale_is_the_magnitude_of_the_terms_of_f():
    # R6: the ratio's rounding guard is 1e-13 max(1, S), S the sum of the magnitudes of
    # the terms f is assembled from, not |f|.  Dense: x = 10, Q = 20, c = -99.9 gives
    # f = 1000 - 999 = 1 with S = 1000 + 999 = 1999.
    rec = np.array([20.0, -99.9, 0.0])
    f, _, _ = oracle.eval_obj(oracle.OBJ_DENSE, rec, np.array([10.0]))
    assert abs(f - 1.0) < 1e-12
    assert abs(oracle.fscale(oracle.OBJ_DENSE, rec, np.array([10.0])) - 1999.0) < 1e-9
    # quartic term: d x^4 with d = -2 at x = 10 counts |d| x^4 = 2e4
    rec = np.array([20.0, -99.9, -2.0])
    assert abs(oracle.fscale(oracle.OBJ_DENSE, rec, np.array([10.0])) - 21999.0) < 1e-8
    # branch at v = (1, 1), theta = (0, 0): w_i = w_j = wR = 1, wI = 0.  Only the pair
    # p_ij carries a multiplier (200) and a penalty (400): p_ij = gc_ij - g_ij = 20 - 20
    # = 0 is its target, so f = 0; each flow term counts (|lambda| + rho |p - t|) times
    # the magnitudes of its terms, |gc_ij w_i| + |g_ij wR| + |b_ij wI| = 40: S = 8000.
    rec = np.zeros(36)
    rec[0], rec[2], rec[3] = 20.0, 20.0, 5.0
    rec[8], rec[24] = 200.0, 400.0
    rec[32], rec[33] = 100.0, 400.0  # line limit 10: inactive
    x = np.array([1.0, 1.0, 0.0, 0.0])
    f, _, _ = oracle.eval_obj(oracle.OBJ_BRANCH, rec, x)
    assert f == 0.0
    assert abs(oracle.fscale(oracle.OBJ_BRANCH, rec, x) - 8000.0) < 1e-9


def test_branch_solves_at_an_admm_state_all_converge():
    # branch subproblems as the ADMM poses them after 20 iterations on a 200-bus network:
    # f ~ 1..100 is a difference of terms ~ 1e3 (multipliers ~ 1e2 times flows with
    # coefficients ~ 20).  TRON reaches a KKT point on every one; a guard scaled by |f|
    # instead of S lets rounding noise of f decide the ratio and collapses the radius on
    # some of them (TR_TOO_SMALL).
    net = synth.network(200, 60, 60, rng=np.random.default_rng(7))
    a = oracle.Admm(net)
    a.run(20, nthreads=4)
    nl = len(net["br_from"])
    recs = np.array([a.branch_record(k) for k in range(nl)])
    lo = np.tile([0.9, 0.9, -2 * np.pi, -2 * np.pi], (nl, 1))
    hi = np.tile([1.1, 1.1, 2 * np.pi, 2 * np.pi], (nl, 1))
    r = oracle.tron_batch(oracle.OBJ_BRANCH, recs, lo, hi, a.arrays["br_x"], np.ones(nl),
                          nthreads=4)
    assert np.all(r["status"] == oracle.CONVERGED), np.bincount(r["status"])
    assert np.all(r["pg"] <= 1e-6)


def test_admm_phases_on_masks_reproduce_the_iteration():
    # the phase entry points (components on a mask; buses on a mask, each with the
    # multipliers of the pairs it holds) performed over all components -- the buses in
    # two disjoint masks -- give the undivided iteration's iterates bit for bit, and its
    # residuals up to the order of the sums
    net = synth.network(150, 40, 50, rng=np.random.default_rng(17))
    nl, ng, nb = len(net["br_from"]), len(net["gen_bus"]), net["nbus"]
    ref = oracle.Admm(net)
    hp, hd = ref.run(25)
    ph = oracle.Admm(net)
    half = np.arange(nb) % 2 == 0
    for it in range(25):
        ph.phase_components(np.ones(ng), np.ones(nl))
        p1, d1 = ph.phase_buses(half)
        p2, d2 = ph.phase_buses(~half)
        assert abs(math.sqrt(p1 + p2) - hp[it]) <= 1e-12 * hp[it]
        assert abs(400.0 * math.sqrt(d1 + d2) - hd[it]) <= 1e-12 * hd[it]
    for k in ref.arrays:
        np.testing.assert_array_equal(ph.arrays[k], ref.arrays[k], err_msg=k)


def test_cauchy_test_in_the_hessian_norm_option():
    # options cauchy_norm = 1: the Cauchy trial's trust-region test uses
    # ||s||_H = (s'Hs)^(1/2).  f = 5 x^2 - x, x0 = 0, delta = 0.015 (H = 10):
    # alpha = 1, 0.1, 0.01 give ||s||_H = sqrt(10) |s| = 3.16, 0.316, 0.0316 > delta;
    # alpha = 0.001 gives 0.00316: four trials, x_c = 0.001.  PCG: r = -1 + 10 x_c = -0.99,
    # the CG iterate's Newton length 0.99/sqrt(10) > delta, so w = delta/sqrt(10) on the
    # boundary; x1 = 0.001 + 0.015/sqrt(10), rho = 1 and the step reached the boundary in
    # the PCG's norm: delta = 0.06
    r = _dense1([10.0], [-1.0], [0.0], [0.0], 0.015, cauchy_norm=1)
    assert r["status"] == oracle.MAX_ITER and r["iters"] == 1
    assert r["counters"]["cauchy_trials"] == 4
    assert abs(r["x"][0] - (0.001 + 0.015 / math.sqrt(10.0))) < 1e-15
    assert r["delta"] == 0.06
    # where s'Hs <= 0 (negative curvature along -g) the test falls back to ||s||_2:
    # f = -0.02 x^2 - x on [-100, 100] from 0, delta = 25: alpha = 1 and 10 hold
    # (||s||_2 = 1, 10), alpha = 100 does not (100 > 25): x_c = 10 after three trials,
    # exactly as with cauchy_norm = 0.  The subspace step follows the negative curvature
    # to the PCG's boundary (length 25 = delta in its norm) and the projected search to
    # the bound x = 100; the step reached the radius, rho = 1: delta = 4 * 25.  (A test on
    # |s'Hs|^(1/2) = 0.2 |s| would accept alpha = 100, leave no free variable and keep
    # delta = 25.)
    kw = dict(l=-100.0, u=100.0)
    a = _dense1([-0.04], [-1.0], [0.0], [0.0], 25.0, cauchy_norm=1, **kw)
    b = _dense1([-0.04], [-1.0], [0.0], [0.0], 25.0, cauchy_norm=0, **kw)
    assert a["counters"]["cauchy_trials"] == b["counters"]["cauchy_trials"] == 3
    assert a["counters"]["subspace_passes"] == b["counters"]["subspace_passes"] == 1
    np.testing.assert_array_equal(a["x"], b["x"])
    assert a["delta"] == b["delta"] == 100.0
