"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed
forms, brute force with scalar ``math`` loops, textbook CG properties,
invariants of the Woodbury identity, Monte-Carlo convergence of the random
Fourier features, and finite differences.
"""
import math

import numpy as np
import pytest

import krr_synth as ks
from oracle import krr_oracle as O


def _rng(seed=0):
    return np.random.Generator(np.random.PCG64(seed))


# ------------------------------------------------------------ kernel ------

def test_kernel_bruteforce_tiny():
    """Gaussian kernel (Section 5 definition) against scalar loops."""
    rng = _rng(1)
    Xa = rng.standard_normal((5, 3))
    Xb = rng.standard_normal((4, 3))
    sigma = 0.7
    K = O.gaussian_kernel(Xa, Xb, sigma)
    for i in range(5):
        for j in range(4):
            d2 = sum((Xa[i, t] - Xb[j, t]) ** 2 for t in range(3))
            assert K[i, j] == pytest.approx(math.exp(-d2 / (2 * sigma * sigma)), rel=1e-13, abs=0)


def test_kernel_closed_forms():
    """exp(-||x-z||^2/2sigma^2) at distances where the value is known in closed form."""
    s = 1.3
    assert O.gaussian_kernel(np.zeros((1, 1)), np.array([[s]]), s)[0, 0] == pytest.approx(math.exp(-0.5))
    assert O.gaussian_kernel(np.zeros((1, 2)), np.ones((1, 2)), 1.0)[0, 0] == pytest.approx(math.exp(-1.0))
    x = np.array([[0.25, -1.0, 3.0]])
    assert O.gaussian_kernel(x, x, 0.1)[0, 0] == 1.0
    # shift invariance
    rng = _rng(2)
    A, B = rng.standard_normal((3, 4)), rng.standard_normal((2, 4))
    sh = rng.standard_normal(4) * 10
    np.testing.assert_allclose(O.gaussian_kernel(A + sh, B + sh, 2.0), O.gaussian_kernel(A, B, 2.0),
                               rtol=1e-12)


def test_kernel_symmetric_psd_unit_diag():
    rng = _rng(3)
    X = rng.standard_normal((60, 5))
    lam = 1e-3
    K = O.gaussian_kernel(X, X, 1.5)
    assert np.array_equal(K, K.T)
    assert np.all(np.diag(K) == 1.0)
    ev = np.linalg.eigvalsh(K)
    assert ev[0] >= -1e-12
    evA = np.linalg.eigvalsh(O.kernel_matrix_system(X, 1.5, lam))
    # trace(K) = n and K is PSD, so eig(A) lies in [lam, n + lam]
    assert evA[0] >= lam * (1 - 1e-9) and evA[-1] <= 60 + lam


def test_blocked_matvec_matches_direct():
    rng = _rng(4)
    Xa, Xb = rng.standard_normal((70, 6)) * 3, rng.standard_normal((90, 6)) * 3
    V = rng.standard_normal((90, 3))
    ref = O.gaussian_kernel(Xa, Xb, 2.5) @ V
    got = O.kernel_matvec_blocked(Xa, Xb, V, 2.5, block=16)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-13)


# ------------------------------------------------------- direct solve -----

def test_direct_solve_n1_closed_form():
    """n=1: K = [1], so c = y / (1 + lambda) (Eq. (1))."""
    for lam in (1e-3, 0.5, 7.0):
        c = O.direct_solve(np.array([[0.3, -2.0]]), np.array([[2.5]]), 0.9, lam)
        assert c[0, 0] == pytest.approx(2.5 / (1 + lam), rel=1e-15)


def test_direct_solve_n2_closed_form():
    """n=2: explicit inverse of [[1+l, k], [k, 1+l]]."""
    x = np.array([[0.0], [1.2]])
    sigma, lam = 0.8, 0.05
    k = math.exp(-1.44 / (2 * 0.64))
    y = np.array([[1.0], [-3.0]])
    det = (1 + lam) ** 2 - k * k
    c0 = ((1 + lam) * 1.0 - k * (-3.0)) / det
    c1 = (-k * 1.0 + (1 + lam) * (-3.0)) / det
    c = O.direct_solve(x, y, sigma, lam)
    assert c[0, 0] == pytest.approx(c0, rel=1e-14)
    assert c[1, 0] == pytest.approx(c1, rel=1e-14)


def test_direct_solve_residual_and_lu_crosscheck():
    P = ks.make_config(1, n=200)
    C = O.direct_solve(P.X, P.Y, P.sigma, P.lam)
    assert O.true_rel_residual(P.X, P.Y, C, P.sigma, P.lam)[0] <= 1e-13
    A = O.kernel_matrix_system(P.X.astype(np.float64), P.sigma, P.lam)
    np.testing.assert_allclose(C, np.linalg.solve(A, P.Y), rtol=1e-9, atol=1e-12)


# -------------------------------------------------- random features -------

def test_rff_bruteforce_tiny():
    rng = _rng(5)
    X = rng.standard_normal((4, 3))
    W = rng.standard_normal((3, 5))
    b = rng.uniform(0, 2 * math.pi, 5)
    Z = O.rff_features(X, W, b)
    for i in range(4):
        for j in range(5):
            arg = sum(X[i, t] * W[t, j] for t in range(3)) + b[j]
            assert Z[i, j] == pytest.approx(math.sqrt(2 / 5) * math.cos(arg), rel=1e-13, abs=1e-15)


def test_rff_monte_carlo_converges_to_kernel():
    """Section 2.2: E[phi(x).phi(z)] = k(x,z); the error falls like s^-1/2.

    A wrong scale (s^-1/2 without the factor 2) or a wrong frequency variance
    leaves a bias that makes the fitted slope flat instead of -1/2.
    """
    rng = _rng(6)
    n, d, sigma = 40, 3, 1.1
    X = rng.standard_normal((n, d))
    K = O.gaussian_kernel(X, X, sigma)
    svals = [64, 256, 1024, 4096, 16384]
    errs = []
    for s in svals:
        e = []
        for seed in range(8):
            W, b = ks.rff_draw(100 + seed, d, s, sigma)
            Z = O.rff_features(X, W, b)
            e.append(np.linalg.norm(Z @ Z.T - K) / np.linalg.norm(K))
        errs.append(np.mean(e))
    slope = np.polyfit(np.log(svals), np.log(errs), 1)[0]
    assert -0.6 <= slope <= -0.4, (slope, errs)
    W, b = ks.rff_draw(7, d, 16384, sigma)
    Z = O.rff_features(X, W, b)
    assert np.mean(np.sum(Z * Z, axis=1)) == pytest.approx(1.0, abs=0.03)


# ------------------------------------------------------- Woodbury ---------

def _small_precond(n=120, s=30, lam_p=1e-2, seed=8):
    P = ks.make_config(1, n=n, s=s)
    Z = O.rff_features(P.X, P.W, P.b)
    return P, Z, O.precond_setup(Z, lam_p)


def test_woodbury_inverts_preconditioner():
    """M^-1 (Z Z^T + lambda_p I) v = v (Section 3.1 Woodbury identity)."""
    P, Z, pre = _small_precond()
    rng = _rng(9)
    V = rng.standard_normal((Z.shape[0], 3))
    M = Z @ Z.T + pre["lam_p"] * np.eye(Z.shape[0])
    np.testing.assert_allclose(O.precond_apply(pre, M @ V), V, rtol=1e-9, atol=1e-9)


def test_woodbury_factor_invariants():
    """U^T U = Z G^-1 Z^T, L L^T = G with L lower, and ||U||_2 < 1."""
    P, Z, pre = _small_precond()
    L, U, G = pre["L"], pre["U"], pre["G"]
    assert np.allclose(np.triu(L, 1), 0.0)
    np.testing.assert_allclose(L @ L.T, G, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(U.T @ U, Z @ np.linalg.solve(G, Z.T), rtol=1e-8, atol=1e-10)
    assert np.linalg.norm(U, 2) < 1.0
    np.testing.assert_allclose(G, Z.T @ Z + pre["lam_p"] * np.eye(Z.shape[1]), rtol=1e-14)


# ------------------------------------------------------------ PCG ---------

def test_pcg_matches_direct_solve():
    P = ks.make_config(1, n=300, s=60)
    out = O.krr_pcg_solve(P.X, P.Y, P.sigma, P.lam, P.W, P.b, tol=1e-10)
    assert out["status"] == "converged"
    C = O.direct_solve(P.X, P.Y, P.sigma, P.lam)
    kappa = np.linalg.cond(O.kernel_matrix_system(P.X.astype(np.float64), P.sigma, P.lam))
    err = np.linalg.norm(out["x"] - C) / np.linalg.norm(C)
    assert err <= kappa * 1e-10
    assert O.true_rel_residual(P.X, P.Y, out["x"], P.sigma, P.lam)[0] <= 1e-10


def test_pcg_anorm_error_monotone():
    """CG minimises the A-norm error over growing Krylov spaces, so it never increases."""
    P = ks.make_config(1, n=150, s=20)
    X = P.X.astype(np.float64)
    A = O.kernel_matrix_system(X, P.sigma, P.lam)
    cstar = np.linalg.solve(A, P.Y)
    Z = O.rff_features(P.X, P.W, P.b)
    pre = O.precond_setup(Z, P.lam)
    errs = []

    def mv(V):
        return A @ V

    for m in range(1, 30):
        out = O.pcg(mv, lambda R: O.precond_apply(pre, R), P.Y, tol=0.0, max_iter=m)
        e = out["x"] - cstar
        errs.append(float(np.sqrt(np.sum(e * (A @ e)))))
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-9) for i in range(len(errs) - 1)), errs


def test_pcg_exact_preconditioner_one_iteration():
    """With Z Z^T = K exactly (Z = Cholesky factor of K) and lambda_p = lambda, M = A: one step."""
    rng = _rng(10)
    X = rng.standard_normal((40, 3))
    sigma, lam = 1.0, 1e-2
    K = O.gaussian_kernel(X, X, sigma)
    Zc = np.linalg.cholesky(K + 1e-13 * np.eye(40))
    pre = O.precond_setup(Zc, lam)
    A = K + lam * np.eye(40)
    y = rng.standard_normal((40, 1))
    out = O.pcg(lambda V: A @ V, lambda R: O.precond_apply(pre, R), y, tol=1e-9)
    assert out["iters"][0] == 1


def test_plain_cg_finite_termination():
    """M = I reduces PCG to CG, which terminates within about n steps."""
    rng = _rng(11)
    X = rng.standard_normal((25, 2))
    out = O.krr_pcg_solve(X, rng.standard_normal((25, 1)), 1.0, 0.1, None, None,
                          precond=False, tol=1e-12)
    assert out["status"] == "converged" and out["iters"][0] <= 25 + 5


def test_multi_rhs_columns_independent():
    """Section 5: each right-hand side must converge; columns share only M."""
    P = ks.make_config(1, n=120, s=30)
    rng = _rng(12)
    Y = np.concatenate([P.Y, rng.standard_normal((120, 2))], axis=1)
    both = O.krr_pcg_solve(P.X, Y, P.sigma, P.lam, P.W, P.b, tol=1e-9)
    for j in range(3):
        one = O.krr_pcg_solve(P.X, Y[:, j:j + 1], P.sigma, P.lam, P.W, P.b, tol=1e-9)
        # same recurrence per column; only BLAS rounding of the block product differs
        np.testing.assert_allclose(both["x"][:, j], one["x"][:, 0], rtol=1e-6, atol=1e-9)
        assert abs(int(both["iters"][j]) - int(one["iters"][0])) <= 1


def test_lanczos_kappa_recovers_spectrum():
    diag = np.linspace(1.0, 100.0, 60)
    y = np.ones((60, 1))
    out = O.pcg(lambda V: diag[:, None] * V, lambda R: R.copy(), y, tol=1e-14, max_iter=60)
    assert O.lanczos_kappa(out["alphas"][0], out["betas"][0]) == pytest.approx(100.0, rel=1e-3)


# ------------------------------------------------------ predict / grad ----

def test_predict_at_training_points():
    """f(x_i) = (K c)_i = y_i - lambda c_i by Eq. (1)."""
    P = ks.make_config(1, n=150)
    C = O.direct_solve(P.X, P.Y, P.sigma, P.lam)
    F = O.predict(P.X, P.X, C, P.sigma)
    np.testing.assert_allclose(F, P.Y - P.lam * C, rtol=1e-9, atol=1e-10)


def test_rfm_push_through_identity():
    """The random-features fit seen at the training points is kernel ridge
    regression with the approximate kernel Z Z^T: Z (Z^T Z + lam I)^-1 Z^T y =
    (Z Z^T)(Z Z^T + lam I)^-1 y.  The right side is an n x n solve, a different
    route from the oracle's s x s Cholesky."""
    P = ks.make_config(1, n=300, s=40)
    Z = O.rff_features(P.X, P.W, P.b)
    w = O.rfm_fit(P.X, P.W, P.b, 0.05, P.Y)
    Kt = Z @ Z.T
    c = np.linalg.solve(Kt + 0.05 * np.eye(300), P.Y)
    np.testing.assert_allclose(O.rfm_predict(P.X, P.W, P.b, w), Kt @ c, rtol=1e-9, atol=1e-10)
    # and the normal equations' residual is orthogonal to the features
    r = P.Y - Z @ w
    np.testing.assert_allclose(Z.T @ r, 0.05 * w, rtol=1e-8, atol=1e-10)


def test_rfm_converges_to_kernel_ridge_regression():
    """With s growing, Z Z^T -> K (Section 2.2), so the random-features predictor
    approaches the exact kernel ridge regression predictor of Eq. (1)."""
    P = ks.make_config(1, n=200)
    rng = _rng(5)
    C = O.direct_solve(P.X, P.Y, P.sigma, 0.1)
    f_exact = O.predict(P.X, P.X[:50], C, P.sigma)
    errs = []
    for s in (32, 256, 2048):
        W = rng.standard_normal((P.X.shape[1], s)) / P.sigma
        b = rng.uniform(0.0, 2.0 * math.pi, s)
        w = O.rfm_fit(P.X, W, b, 0.1, P.Y)
        errs.append(np.linalg.norm(O.rfm_predict(P.X[:50], W, b, w) - f_exact)
                    / np.linalg.norm(f_exact))
    assert errs[2] < errs[1] < errs[0] and errs[2] < 0.1, errs


def test_poly_kernel_bruteforce():
    """(gamma x.z + c)^q against scalar loops."""
    rng = _rng(21)
    X = rng.standard_normal((5, 3))
    Kp = O.poly_kernel(X, X[:4], 0.7, 1.3, 3)
    for i in range(5):
        for j in range(4):
            dot = sum(X[i, t] * X[j, t] for t in range(3))
            assert math.isclose(Kp[i, j], (0.7 * dot + 1.3) ** 3, rel_tol=1e-13, abs_tol=1e-13)


def test_countsketch_is_a_sparse_matrix_product():
    """CountSketch equals the s x d matrix with column j = g(j) e_{h(j)} (Section 2.2)."""
    h, g = ks.tensorsketch_draw(3, 7, 1, 5)
    X = _rng(22).standard_normal((4, 7))
    Cm = np.zeros((5, 7))
    for j in range(7):
        Cm[h[0, j], j] = g[0, j]
    np.testing.assert_allclose(O.countsketch(X, h[0], g[0], 5), X @ Cm.T, rtol=0, atol=1e-14)


def test_tensorsketch_explicit_matrix_tiny():
    """phi(x) = S v_q(x~) with S and v_q built as explicit arrays from the definition."""
    import itertools
    q, d, s, gam, c = 2, 3, 5, 0.5, 2.0
    h, g = ks.tensorsketch_draw(4, d + 1, q, s)
    X = _rng(23).standard_normal((3, d))
    Xa = np.hstack([math.sqrt(gam) * X, np.full((3, 1), math.sqrt(c))])
    cols = list(itertools.product(range(d + 1), repeat=q))
    S = np.zeros((s, len(cols)))
    V = np.zeros((3, len(cols)))
    for m, ii in enumerate(cols):
        S[sum(int(h[t, ii[t]]) for t in range(q)) % s, m] += np.prod([g[t, ii[t]] for t in range(q)])
        V[:, m] = np.prod([Xa[:, ii[t]] for t in range(q)], axis=0)
    np.testing.assert_allclose(O.tensorsketch_features(X, h, g, s, gam, c), V @ S.T,
                               rtol=1e-12, atol=1e-12)


def test_tensorsketch_equals_convolved_countsketches():
    """Pagh's identity: the TensorSketch is the circular convolution of the q
    CountSketches, computed here through the FFT (a different route)."""
    q, d, s, gam, c = 3, 6, 32, 0.8, 0.5
    h, g = ks.tensorsketch_draw(5, d + 1, q, s)
    X = _rng(24).standard_normal((4, d))
    Xa = np.hstack([math.sqrt(gam) * X, np.full((4, 1), math.sqrt(c))])
    prod = np.ones((4, s), dtype=complex)
    for t in range(q):
        prod *= np.fft.fft(O.countsketch(Xa, h[t], g[t], s), axis=1)
    ref = np.real(np.fft.ifft(prod, axis=1))
    np.testing.assert_allclose(O.tensorsketch_features(X, h, g, s, gam, c), ref,
                               rtol=1e-10, atol=1e-10)


def test_tensorsketch_inner_products_are_unbiased():
    """E phi(x).phi(z) = (gamma x.z + c)^q over the hash draws (Section 2.2)."""
    q, d, s, gam, c = 2, 4, 16, 0.5, 1.0
    rng = _rng(25)
    x, z = rng.standard_normal((2, d))
    exact = (gam * x @ z + c) ** q
    vals = []
    for seed in range(3000):
        h, g = ks.tensorsketch_draw(10_000 + seed, d + 1, q, s)
        F = O.tensorsketch_features(np.vstack([x, z]), h, g, s, gam, c)
        vals.append(F[0] @ F[1])
    vals = np.asarray(vals)
    assert abs(vals.mean() - exact) <= 5.0 * vals.std() / math.sqrt(len(vals)), \
        (vals.mean(), exact)


def test_poly_pcg_matches_direct_solve():
    """Algorithm 1 with the polynomial kernel and the TensorSketch preconditioner
    reaches the direct solve of (K + lambda I) c = y."""
    rng = _rng(26)
    X = rng.standard_normal((150, 4)) / 2.0
    Y = np.sin(X.sum(axis=1, keepdims=True))
    h, g = ks.tensorsketch_draw(6, 5, 2, 64)
    r = O.krr_poly_pcg_solve(X, Y, 0.5, 1.0, 2, 1e-2, h, g, 64, tol=1e-11, max_iter=500)
    A = O.poly_kernel(X, X, 0.5, 1.0, 2) + 1e-2 * np.eye(150)
    Cd = np.linalg.solve(A, Y)
    np.testing.assert_allclose(r["x"], Cd, rtol=1e-7, atol=1e-9)


def test_kernel_dlogsigma_central_differences():
    """D o K against Richardson-extrapolated central differences of K in log sigma."""
    rng = np.random.default_rng(31)
    Xa = rng.standard_normal((9, 5))
    Xb = rng.standard_normal((7, 5))
    sig = 1.7
    G = O.kernel_dlogsigma(Xa, Xb, sig)
    fd = []
    for h in (1e-3, 5e-4):
        fd.append((O.gaussian_kernel(Xa, Xb, sig * math.exp(h))
                   - O.gaussian_kernel(Xa, Xb, sig * math.exp(-h))) / (2 * h))
    rich = (4 * fd[1] - fd[0]) / 3
    np.testing.assert_allclose(G, rich, rtol=1e-7, atol=1e-12)
    # zero on the diagonal of a square set and never negative
    Gs = O.kernel_dlogsigma(Xa, Xa, sig)
    assert np.all(np.diag(Gs) == 0.0) and np.all(Gs >= 0.0)
    # maximum of r^2/s^2 exp(-r^2/(2 s^2)) over r is 2/e, at r^2 = 2 s^2
    x = np.array([[0.0], [math.sqrt(2.0) * sig]])
    assert O.kernel_dlogsigma(x, x, sig)[0, 1] == pytest.approx(2.0 / math.e, rel=1e-14)


@pytest.mark.parametrize("which", ["dlogsigma", "dloglambda"])
def test_hypergrad_central_differences(which):
    P = ks.make_config(5, n=80, m=30, s=16)
    sig, lam = P.sigma, P.lam
    g = O.hypergrad(P.X, P.Y, P.Xte, P.Yte, sig, lam)[which]

    def loss(ls, ll):
        return O.heldout_loss(P.X, P.Y, P.Xte, P.Yte, math.exp(ls), math.exp(ll))

    ls, ll = math.log(sig), math.log(lam)
    fd = []
    for h in (1e-3, 5e-4):
        if which == "dlogsigma":
            fd.append((loss(ls + h, ll) - loss(ls - h, ll)) / (2 * h))
        else:
            fd.append((loss(ls, ll + h) - loss(ls, ll - h)) / (2 * h))
    rich = (4 * fd[1] - fd[0]) / 3
    assert g == pytest.approx(rich, rel=1e-7, abs=1e-12)


# ------------------------------------------------------------ golden -------

def _golden_path(name):
    import os
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)


def test_golden_closed_forms():
    """Closed forms stored in tests/golden/closed_forms.txt (Eq. (1), Section 5 kernel)."""
    rows = [ln.split() for ln in open(_golden_path("closed_forms.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for case, sig, lam, x, z, y, exp in rows:
        sig, lam, exp = float(sig), float(lam), float(exp)
        xa = np.array([[float(v) for v in x.split(",")]])
        if case.startswith("kernel"):
            za = np.array([[float(v) for v in z.split(",")]])
            assert O.gaussian_kernel(xa, za, sig)[0, 0] == pytest.approx(exp, rel=1e-15)
        else:
            c = O.direct_solve(xa, np.array([[float(y)]]), sig, lam)
            assert c[0, 0] == pytest.approx(exp, rel=1e-15)


def test_golden_six_point_problem_frozen():
    """The oracle still reproduces the six-point fixture written by tests/golden/make_golden.py."""
    import json
    g = json.load(open(_golden_path("six_point_problem.json")))
    X, y = np.array(g["X"]), np.array(g["y"])
    W, b = np.array(g["W"]), np.array(g["b"])
    sig, lam = g["sigma"], g["lambda"]
    np.testing.assert_allclose(O.gaussian_kernel(X, X, sig), g["K"], rtol=1e-14)
    np.testing.assert_allclose(O.direct_solve(X, y, sig, lam), g["c_direct"], rtol=1e-12)
    np.testing.assert_allclose(O.rff_features(X, W, b), g["Z"], rtol=1e-13, atol=1e-15)
    pre = O.precond_setup(O.rff_features(X, W, b), lam)
    np.testing.assert_allclose(pre["U"], g["U"], rtol=1e-10, atol=1e-13)
    # the fixture's PCG and direct solutions agree (s=3 < n=6, tol 1e-12)
    np.testing.assert_allclose(g["c_pcg"], g["c_direct"], rtol=1e-9, atol=1e-10)


# ------------------------------------------- multiple-level sketching ---

@pytest.mark.parametrize("m", [1, 2, 4, 8, 32, 64])
def test_walsh_hadamard_is_sylvesters_matrix(m):
    """H_m from the recursion equals scipy's Sylvester Hadamard matrix and
    H H^T = m I."""
    import scipy.linalg as sla
    H = O.walsh_hadamard(m)
    assert np.array_equal(H, sla.hadamard(m))
    np.testing.assert_array_equal(H @ H.T, m * np.eye(m))


def test_walsh_hadamard_rejects_non_powers_of_two():
    with pytest.raises(ValueError):
        O.walsh_hadamard(12)


def test_srht_without_subsampling_is_orthogonal():
    """With every row kept (s2 = m), S2 = m^-1/2 H D is orthogonal, so
    Z2 Z2^T = Z1 Z1^T exactly (up to rounding)."""
    rng = np.random.default_rng(0)
    Z1 = rng.standard_normal((20, 13))
    signs, rows = ks.srht_draw(1, 16, 16)
    Z2 = O.srht_apply(Z1, signs, rows)
    np.testing.assert_allclose(Z2 @ Z2.T, Z1 @ Z1.T, rtol=1e-12, atol=1e-12)


def test_srht_of_a_unit_vector():
    """Closed form: for z1 = e_j, (S2 z1)_k = signs_j H[rows_k, j] / sqrt(s2); for
    j = 0 (a column of ones in H) every entry is signs_0 / sqrt(s2)."""
    signs, rows = ks.srht_draw(2, 32, 8)
    Z1 = np.zeros((2, 32))
    Z1[0, 0] = 1.0
    Z1[1, 5] = 1.0
    Z2 = O.srht_apply(Z1, signs, rows)
    np.testing.assert_allclose(Z2[0], signs[0] / math.sqrt(8) * np.ones(8), rtol=1e-15)
    bits = np.array([bin(int(r) & 5).count("1") for r in rows])
    np.testing.assert_allclose(Z2[1], signs[5] * (-1.0) ** bits / math.sqrt(8), rtol=1e-15)


def test_srht_is_unbiased():
    """E S2^T S2 = I (signs and sampled rows random): the mean of Z2 Z2^T over
    draws approaches Z1 Z1^T with error ~ draws^-1/2."""
    rng = np.random.default_rng(3)
    Z1 = rng.standard_normal((6, 50))
    G1 = Z1 @ Z1.T
    errs = []
    for draws in (50, 800):
        acc = np.zeros_like(G1)
        for t in range(draws):
            signs, rows = ks.srht_draw(1000 + t, 64, 16)
            Z2 = O.srht_apply(Z1, signs, rows)
            acc += Z2 @ Z2.T
        errs.append(np.linalg.norm(acc / draws - G1) / np.linalg.norm(G1))
    assert errs[1] < 0.5 * errs[0] and errs[1] < 0.05, errs


def test_gaussian_projection_is_unbiased_and_exact_for_scaled_identity():
    rng = np.random.default_rng(4)
    Z2 = rng.standard_normal((5, 12))
    # S3 = sqrt(s3) I gives Z3 = Z2
    np.testing.assert_allclose(O.gaussian_projection(Z2, math.sqrt(12) * np.eye(12)), Z2,
                               rtol=1e-14)
    acc = np.zeros((5, 5))
    draws = 400
    for t in range(draws):
        Z3 = O.gaussian_projection(Z2, ks.gaussian_draw(50 + t, 8, 12))
        acc += Z3 @ Z3.T
    G2 = Z2 @ Z2.T
    assert np.linalg.norm(acc / draws - G2) / np.linalg.norm(G2) < 0.06


def test_multilevel_pcg_matches_direct_solve():
    """Algorithm 2 (RFF -> SRHT -> Gaussian projection -> Woodbury PCG) reaches the
    direct solution of Eq. (1)."""
    P = ks.make_config(1, n=400, s=128)
    signs, rows = ks.srht_draw(7, 128, 64)
    G = ks.gaussian_draw(8, 48, 64)
    out = O.krr_multilevel_pcg_solve(P.X, P.Y, P.sigma, P.lam, P.W, P.b, signs, rows, G,
                                     tol=1e-10, max_iter=2000)
    assert out["status"] == "converged"
    c = O.direct_solve(P.X, P.Y, P.sigma, P.lam)
    kappa = np.linalg.cond(O.kernel_matrix_system(P.X, P.sigma, P.lam))
    assert np.linalg.norm(out["x"] - c) <= kappa * 1e-10 * np.linalg.norm(c)


# ---------------------------------------------- adaptive sketch size ---

def test_eig_projector_properties():
    rng = np.random.default_rng(5)
    Z = rng.standard_normal((30, 8)) * np.linspace(0.01, 3.0, 8)
    M = Z @ Z.T
    ev = np.linalg.eigvalsh(M)
    thresh = 0.5
    P = O.eig_projector(Z, thresh)
    np.testing.assert_allclose(P @ P, P, atol=1e-12)
    np.testing.assert_allclose(P, P.T, atol=1e-14)
    np.testing.assert_allclose(P @ M, M @ P, atol=1e-10)
    assert round(np.trace(P)) == int(np.sum(ev > thresh))
    assert np.allclose(O.eig_projector(Z, 1e9), 0.0)
    Pr = O.eig_projector(Z, -1.0)   # the whole range of Z
    np.testing.assert_allclose(Pr @ Z, Z, atol=1e-10)


def test_condition1_power_iteration_converges_to_the_norm():
    P = ks.make_config(1, n=200, s=16)
    K = O.gaussian_kernel(P.X, P.X, P.sigma)
    Z = O.rff_features(P.X, P.W, P.b)
    Pp = O.eig_projector(Z, 0.05 * P.lam)
    exact = O.condition1_norm(K, Pp)
    x0 = np.random.default_rng(9).standard_normal(200)
    est = O.condition1_power(lambda v: K @ v, Pp, x0, 300)
    assert est == pytest.approx(exact, rel=1e-6)
    # with P = I the condition holds trivially (zero)
    assert O.condition1_norm(K, np.eye(200)) == pytest.approx(0.0, abs=1e-12)


def test_adaptive_sketch_size_doubles_until_condition1_holds():
    P = ks.make_config(1, n=300)
    W, b = ks.rff_draw(77, P.d, 2048, P.sigma)
    x0 = np.random.default_rng(1).standard_normal(300)
    lam = 1e-1
    out = O.adaptive_sketch_size(P.X, P.sigma, lam, W, b, 16, x0, iters=60)
    ss = [s for s, _ in out["history"]]
    assert ss[0] == 16 and all(b2 == 2 * a for a, b2 in zip(ss, ss[1:]))
    assert out["passed"] and out["estimate"] <= 0.1 * lam
    # every rejected s failed the test
    assert all(est > 0.1 * lam for _, est in out["history"][:-1])
    # capped at the columns available
    capped = O.adaptive_sketch_size(P.X, P.sigma, 1e-9, W[:, :64], b[:64], 16, x0, iters=20)
    assert capped["s"] == 64 and not capped["passed"]
