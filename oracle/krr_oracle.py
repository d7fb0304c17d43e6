"""FP64 CPU oracle for RFF-preconditioned kernel ridge regression.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The product path (the
CUDA library and its Python binding) never imports it and shares no code with
it: the two meet only through the seeded inputs from ``krr_synth``.

Everything here is plain, slow and written to be checked against the paper
by eye (Avron, Clarkson, Woodruff, "Faster Kernel Ridge Regression Using
Sketching and Preconditioning"):

* ``gaussian_kernel``         -- K_ij = exp(-||x_i - x_j||^2 / (2 sigma^2)),
                                 Section 5 (kernel definition), squared
                                 distances summed from coordinate differences.
* ``direct_solve``            -- (K + lambda I) c = y, Eq. (1), by Cholesky.
* ``rff_features``            -- random Fourier features, Section 2.2, with the
                                 sqrt(2/s) scale (reading: the printed s^-1/2
                                 misses the factor 2 of E[cos cos] = k / 2).
* ``precond_setup/apply``     -- the set-up of Algorithm 1 and the Woodbury form of
                                 Section 3.1: L L^T = Z^T Z + lambda_p I,
                                 U = L^-1 Z^T, M^-1 v = (v - U^T U v)/lambda_p.
* ``pcg``                     -- PCG from x0 = 0 (Algorithm 1; the
                                 Hestenes-Stiefel recurrences), stopping on the
                                 true relative residual (Section 5).
* ``krr_pcg_solve``           -- Algorithm 1 end to end.
* ``predict``                 -- f(x) = sum_i c_i k(x_i, x), Section 1.
* ``rfm_fit/rfm_predict``     -- the random-features method: ridge regression on
                                 the features of Section 2.2,
                                 w = (Z^T Z + lambda I)^-1 Z^T y by Cholesky of
                                 the s x s Gram matrix, f(x) = phi(x)^T w.
* ``poly_kernel``             -- k(x, z) = (gamma x^T z + c)^q, the second
                                 kernel of the experiments (Section 6).
* ``countsketch``             -- z_i = sum over j with h(j) = i of g(j) x_j
                                 (Section 2.2).
* ``tensorsketch_features``   -- phi(x) = S v_q(x) for the degree-q TensorSketch
                                 of Section 2.2, by enumerating the d^q monomials
                                 (readings: the composite hash is taken mod s,
                                 printed "mod m", and the t-th sign factor reads
                                 i_t, printed i_1 in the second factor); the
                                 offset c enters as an extra coordinate sqrt(c)
                                 and gamma as a factor sqrt(gamma) on x, so that
                                 E phi(x)^T phi(z) = (gamma x^T z + c)^q.
* ``krr_poly_pcg_solve``      -- Algorithm 1 for the polynomial kernel with the
                                 TensorSketch preconditioner.
* ``walsh_hadamard``, ``srht_apply``, ``gaussian_projection``,
  ``multilevel_features``, ``krr_multilevel_pcg_solve``
                              -- Algorithm 2 (Section 4): the SRHT
                                 s2^-1/2 P H D of the features, then a dense
                                 Gaussian projection (reading: the algorithm
                                 omits the Cholesky step and writes Z for Z3).
* ``eig_projector``, ``condition1_norm``, ``condition1_power``,
  ``adaptive_sketch_size``
                              -- Section 5 / Theorem 4: the projection P, the
                                 first condition ||(I-P)K(I-P)|| <= 0.1 lambda
                                 by power iteration, and doubling s.
* ``kernel_dlogsigma``        -- D o K, the derivative of K in log sigma.
* ``hypergrad``               -- gradient of a held-out MSE with respect to
                                 log sigma and log lambda (not in the paper;
                                 derived by implicit differentiation of Eq. (1)).

``kernel_matvec_blocked`` evaluates K v for n too large to hold K: it forms
row blocks of K with the exact identity ||x-z||^2 = ||x||^2 + ||z||^2 - 2 x.z
in FP64 (a library matmul as one step), which differs from the direct sum by
FP64 rounding only (pinned in the tests to 1e-12 relative).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

__all__ = [
    "sqdist_direct", "gaussian_kernel", "kernel_matrix_system", "direct_solve",
    "rff_features", "gram", "precond_setup", "precond_apply", "pcg",
    "krr_pcg_solve", "predict", "kernel_matvec_blocked", "true_rel_residual",
    "lanczos_kappa", "hypergrad", "heldout_loss", "rfm_fit", "rfm_predict",
    "poly_kernel", "countsketch", "tensorsketch_features", "krr_poly_pcg_solve",
]


# ---------------------------------------------------------------- kernel ---

def sqdist_direct(Xa: np.ndarray, Xb: np.ndarray, block: int = 256) -> np.ndarray:
    """Squared distances ||a_i - b_j||^2 summed from coordinate differences.

    Blocked over rows of ``Xa`` only to bound memory; each entry is the plain
    sum over coordinates of (a_it - b_jt)^2 in FP64.
    """
    Xa = np.asarray(Xa, np.float64)
    Xb = np.asarray(Xb, np.float64)
    out = np.empty((Xa.shape[0], Xb.shape[0]))
    for i0 in range(0, Xa.shape[0], block):
        diff = Xa[i0:i0 + block, None, :] - Xb[None, :, :]
        out[i0:i0 + block] = np.einsum("ijt,ijt->ij", diff, diff)
    return out


def gaussian_kernel(Xa: np.ndarray, Xb: np.ndarray, sigma: float) -> np.ndarray:
    """K_ij = exp(-||a_i - b_j||^2 / (2 sigma^2)) (the paper's Gaussian kernel, Section 5)."""
    return np.exp(-sqdist_direct(Xa, Xb) / (2.0 * sigma * sigma))


def kernel_dlogsigma(Xa: np.ndarray, Xb: np.ndarray, sigma: float) -> np.ndarray:
    """d K / d log(sigma) for the Gaussian kernel of Section 5 (not in the paper).

    With D_ij = ||a_i - b_j||^2 / sigma^2 the kernel is exp(-D/2) and
    d D / d log(sigma) = -2 D, so the derivative is D o K.
    """
    D = sqdist_direct(Xa, Xb) / (sigma * sigma)
    return D * np.exp(-0.5 * D)


def kernel_matrix_system(X: np.ndarray, sigma: float, lam: float) -> np.ndarray:
    """A = K + lambda I_n, the matrix of Eq. (1)."""
    A = gaussian_kernel(X, X, sigma)
    A[np.diag_indices_from(A)] += lam
    return A


def direct_solve(X: np.ndarray, Y: np.ndarray, sigma: float, lam: float) -> np.ndarray:
    """Solve (K + lambda I) C = Y (Eq. (1)) by FP64 Cholesky and two triangular solves."""
    A = kernel_matrix_system(X, sigma, lam)
    L = np.linalg.cholesky(A)
    Y = np.asarray(Y, np.float64).reshape(A.shape[0], -1)
    T = sla.solve_triangular(L, Y, lower=True)
    return sla.solve_triangular(L.T, T, lower=False)


def kernel_matvec_blocked(Xa: np.ndarray, Xb: np.ndarray, V: np.ndarray, sigma: float,
                          block: int = 1024) -> np.ndarray:
    """K(Xa, Xb) @ V in FP64 without storing K (row blocks of K, one at a time).

    Squared distances use ||a||^2 + ||b||^2 - 2 a.b in FP64, clamped at 0.
    """
    Xa = np.asarray(Xa, np.float64)
    Xb = np.asarray(Xb, np.float64)
    V = np.asarray(V, np.float64).reshape(Xb.shape[0], -1)
    na = np.einsum("ij,ij->i", Xa, Xa)
    nb = np.einsum("ij,ij->i", Xb, Xb)
    out = np.empty((Xa.shape[0], V.shape[1]))
    g = -1.0 / (2.0 * sigma * sigma)
    for i0 in range(0, Xa.shape[0], block):
        D = na[i0:i0 + block, None] + nb[None, :] - 2.0 * (Xa[i0:i0 + block] @ Xb.T)
        np.maximum(D, 0.0, out=D)
        np.multiply(D, g, out=D)
        np.exp(D, out=D)
        out[i0:i0 + block] = D @ V
    return out


def true_rel_residual(X: np.ndarray, Y: np.ndarray, C: np.ndarray, sigma: float,
                      lam: float, explicit_max: int = 8192) -> np.ndarray:
    """Per-column ||y - (K + lambda I) c|| / ||y|| in FP64 (the stopping quantity of Section 5)."""
    Y = np.asarray(Y, np.float64).reshape(X.shape[0], -1)
    C = np.asarray(C, np.float64).reshape(X.shape[0], -1)
    if X.shape[0] <= explicit_max:
        KC = gaussian_kernel(X, X, sigma) @ C
    else:
        KC = kernel_matvec_blocked(X, X, C, sigma)
    R = Y - KC - lam * C
    return np.linalg.norm(R, axis=0) / np.linalg.norm(Y, axis=0)


# ------------------------------------------------- random Fourier features ---

def rff_features(X: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Z_ij = sqrt(2/s) cos(sum_t X_it W_tj + b_j) (Section 2.2; sqrt(2/s) scale, see module doc)."""
    X = np.asarray(X, np.float64)
    W = np.asarray(W, np.float64)
    b = np.asarray(b, np.float64)
    s = W.shape[1]
    return math.sqrt(2.0 / s) * np.cos(X @ W + b[None, :])


# ------------------------------------------------------ preconditioner ----

def gram(Z: np.ndarray, lam_p: float) -> np.ndarray:
    """G = Z^T Z + lambda_p I_s (the Gram step of Algorithm 1)."""
    Z = np.asarray(Z, np.float64)
    G = Z.T @ Z
    G[np.diag_indices_from(G)] += lam_p
    return G


def precond_setup(Z: np.ndarray, lam_p: float) -> dict:
    """Cholesky L L^T = G and U = L^-1 Z^T (Section 3.1; the set-up of Algorithm 1).

    Reading: the printed text pairs L L^T with U = L^-T Z^T and the algorithm
    pairs L^T L with L^T U = Z^T; both give U^T U = Z G^-1 Z^T only as
    L L^T with U = L^-1 Z^T, which is the form used here.
    """
    G = gram(Z, lam_p)
    L = np.linalg.cholesky(G)
    U = sla.solve_triangular(L, np.asarray(Z, np.float64).T, lower=True)
    return {"G": G, "L": L, "U": U, "lam_p": float(lam_p)}


def precond_apply(P: dict, R: np.ndarray) -> np.ndarray:
    """M^-1 R = lambda_p^-1 (R - U^T (U R)) (Algorithm 1, Section 3.1 Woodbury form)."""
    U = P["U"]
    R = np.asarray(R, np.float64)
    return (R - U.T @ (U @ R)) / P["lam_p"]


# ------------------------------------------------------------------- PCG ---

def pcg(matvec, apply_minv, Y: np.ndarray, tol: float, max_iter: int = 1000,
        true_residual=None, x0: np.ndarray | None = None) -> dict:
    """Preconditioned conjugate gradients on each column of Y, from x0 = 0.

    Per column j (Hestenes-Stiefel recurrences):
        r = y - A x, z = M^-1 r, p = z
        repeat: q = A p, alpha = r.z / p.q, x += alpha p, r -= alpha q,
                stop when ||y - A x|| <= tol ||y|| (the true residual is
                evaluated whenever the recursive one passes the test),
                z' = M^-1 r, beta = r'.z' / r.z, p = z' + beta p.
    Columns are independent; a converged column is frozen.  ``matvec`` and
    ``apply_minv`` act on n x k blocks.  Returns the iterate, per-column
    iteration counts, the alpha/beta sequences and residual histories.
    """
    Y = np.asarray(Y, np.float64)
    n, k = Y.shape
    X = np.zeros((n, k)) if x0 is None else np.array(x0, np.float64).reshape(n, k)
    R = Y - matvec(X) if x0 is not None else Y.copy()
    ynorm = np.linalg.norm(Y, axis=0)
    Z = apply_minv(R)
    Pd = Z.copy()
    rz = np.einsum("ij,ij->j", R, Z)
    active = np.ones(k, bool)
    iters = np.zeros(k, int)
    alphas = [[] for _ in range(k)]
    betas = [[] for _ in range(k)]
    hist = [[float(np.linalg.norm(R[:, j]) / ynorm[j])] for j in range(k)]
    status = "maxiter"
    for it in range(max_iter):
        if not active.any():
            status = "converged"
            break
        Q = matvec(Pd)
        pq = np.einsum("ij,ij->j", Pd, Q)
        for j in np.nonzero(active)[0]:
            a = rz[j] / pq[j]
            alphas[j].append(a)
            X[:, j] += a * Pd[:, j]
            R[:, j] -= a * Q[:, j]
            iters[j] += 1
            rel = float(np.linalg.norm(R[:, j]) / ynorm[j])
            hist[j].append(rel)
            if rel <= tol:
                tr = (true_residual(X[:, j:j + 1], j) if true_residual is not None else rel)
                if tr <= tol:
                    active[j] = False
        if not active.any():
            status = "converged"
            break
        Znew = apply_minv(R)
        rz_new = np.einsum("ij,ij->j", R, Znew)
        for j in np.nonzero(active)[0]:
            bt = rz_new[j] / rz[j]
            betas[j].append(bt)
            Pd[:, j] = Znew[:, j] + bt * Pd[:, j]
            rz[j] = rz_new[j]
    else:
        status = "converged" if not active.any() else "maxiter"
    return {"x": X, "iters": iters, "alphas": alphas, "betas": betas,
            "hist": hist, "status": status}


def lanczos_kappa(alphas, betas) -> float:
    """Condition-number estimate of M^-1 A from the CG coefficients.

    The Lanczos tridiagonal has diagonal 1/a_0, 1/a_k + b_{k-1}/a_{k-1} and
    off-diagonal sqrt(b_{k-1})/a_{k-1}; its extreme eigenvalues estimate those
    of the preconditioned operator.
    """
    m = len(alphas)
    if m == 0:
        return 1.0
    T = np.zeros((m, m))
    for i in range(m):
        T[i, i] = 1.0 / alphas[i] + (betas[i - 1] / alphas[i - 1] if i > 0 else 0.0)
        if i + 1 < m and i < len(betas):
            T[i, i + 1] = T[i + 1, i] = math.sqrt(max(betas[i], 0.0)) / alphas[i]
    ev = np.linalg.eigvalsh(T)
    return float(ev[-1] / ev[0])


def krr_pcg_solve(X, Y, sigma: float, lam: float, W, b, lam_p: float | None = None,
                  tol: float = 1e-6, max_iter: int = 1000, precond: bool = True,
                  explicit_max: int = 8192) -> dict:
    """Algorithm 1: RFF features, Woodbury preconditioner, PCG on (K + lambda I) c = y.

    K is formed explicitly (as Algorithm 1 does) for n <= ``explicit_max``;
    above that its row blocks are recomputed at every product.
    ``precond=False`` runs plain CG (M = I), the comparator of Table 4.
    """
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64).reshape(X.shape[0], -1)
    lam_p = lam if lam_p is None else lam_p
    n = X.shape[0]
    if n <= explicit_max:
        A = kernel_matrix_system(X, sigma, lam)

        def matvec(V):
            return A @ V
    else:
        def matvec(V):
            return kernel_matvec_blocked(X, X, V, sigma) + lam * V
    if precond:
        Z = rff_features(X, W, b)
        P = precond_setup(Z, lam_p)

        def apply_minv(R):
            return precond_apply(P, R)
    else:
        P = None

        def apply_minv(R):
            return R.copy()

    ynorm = np.linalg.norm(Y, axis=0)

    def true_res(xcol, j):
        return float(np.linalg.norm(Y[:, j] - matvec(xcol)[:, 0]) / ynorm[j])

    out = pcg(matvec, apply_minv, Y, tol, max_iter, true_residual=true_res)
    out["precond"] = P
    return out


# --------------------------------------------------------------- predict ---

def predict(Xtr, Xte, C, sigma: float) -> np.ndarray:
    """f(x) = sum_i c_i k(x_i, x) at each held-out point (Section 1)."""
    return gaussian_kernel(Xte, Xtr, sigma) @ np.asarray(C, np.float64).reshape(len(Xtr), -1)


# ------------------------------------------------- random-features method ---

def rfm_fit(X, W, b, lam: float, Y) -> np.ndarray:
    """w = (Z^T Z + lambda I_s)^-1 Z^T Y with Z = rff_features(X, W, b) (Section 2.2's
    features as the model: ridge regression in feature space), by Cholesky of G."""
    Z = rff_features(X, W, b)
    G = gram(Z, lam)
    L = np.linalg.cholesky(G)
    rhs = Z.T @ np.asarray(Y, np.float64).reshape(Z.shape[0], -1)
    u = sla.solve_triangular(L, rhs, lower=True)
    return sla.solve_triangular(L.T, u, lower=False)


def rfm_predict(Xte, W, b, w) -> np.ndarray:
    """f(x) = phi(x)^T w with phi the random Fourier features of Section 2.2."""
    return rff_features(Xte, W, b) @ np.asarray(w, np.float64)


# ------------------------------------ polynomial kernel and TensorSketch ---

def poly_kernel(Xa, Xb, gamma: float, c: float, q: int) -> np.ndarray:
    """K_ij = (gamma a_i^T b_j + c)^q (the polynomial kernel of Section 6)."""
    G = np.asarray(Xa, np.float64) @ np.asarray(Xb, np.float64).T
    return (gamma * G + c) ** q


def countsketch(X, h, g, s: int) -> np.ndarray:
    """CountSketch of each row of X (Section 2.2): z_i = sum_{j: h(j) = i} g(j) x_j."""
    X = np.asarray(X, np.float64).reshape(-1, len(h))
    Z = np.zeros((X.shape[0], s))
    for j in range(len(h)):
        Z[:, int(h[j])] += float(g[j]) * X[:, j]
    return Z


def _augment(X, gamma: float, c: float) -> np.ndarray:
    """[sqrt(gamma) x, sqrt(c)]: its degree-q monomial products give (gamma x^T z + c)^q."""
    X = np.asarray(X, np.float64)
    return np.hstack([math.sqrt(gamma) * X, np.full((X.shape[0], 1), math.sqrt(c))])


def tensorsketch_features(X, h, g, s: int, gamma: float = 1.0, c: float = 0.0) -> np.ndarray:
    """phi(x) = S v_q(x~) with x~ = [sqrt(gamma) x, sqrt(c)] (Section 2.2).

    h, g: q x d~ hash and sign tables (d~ = d + 1 when c > 0, else d).  Column
    (i_1..i_q) of S is G e_H with H = (h_1(i_1) + ... + h_q(i_q)) mod s and
    G = g_1(i_1) ... g_q(i_q); v_q(x) lists the products x_{i_1} ... x_{i_q}.
    The d~^q monomials are enumerated one multi-index at a time.
    """
    Xa = _augment(X, gamma, c) if c > 0.0 else math.sqrt(gamma) * np.asarray(X, np.float64)
    h = np.asarray(h)
    g = np.asarray(g)
    q, dd = h.shape
    if Xa.shape[1] != dd:
        raise ValueError("hash tables must cover every (augmented) coordinate")
    Z = np.zeros((Xa.shape[0], s))
    idx = [0] * q
    for _ in range(dd ** q):
        H = sum(int(h[t, idx[t]]) for t in range(q)) % s
        G = 1.0
        mono = np.ones(Xa.shape[0])
        for t in range(q):
            G *= float(g[t, idx[t]])
            mono = mono * Xa[:, idx[t]]
        Z[:, H] += G * mono
        # next multi-index (i_1 fastest)
        t = 0
        while t < q:
            idx[t] += 1
            if idx[t] < dd:
                break
            idx[t] = 0
            t += 1
    return Z


def krr_poly_pcg_solve(X, Y, gamma: float, c: float, q: int, lam: float, h, g, s: int,
                       lam_p: float | None = None, tol: float = 1e-8,
                       max_iter: int = 1000) -> dict:
    """Algorithm 1 for the polynomial kernel: the TensorSketch features build the
    preconditioner Z Z^T + lambda_p I (Woodbury form), PCG runs on K + lambda I."""
    X = np.asarray(X, np.float64)
    Z = tensorsketch_features(X, h, g, s, gamma, c)
    P = precond_setup(Z, lam if lam_p is None else lam_p)
    A = poly_kernel(X, X, gamma, c, q)
    A[np.diag_indices_from(A)] += lam
    return pcg(lambda V: A @ V, lambda R: precond_apply(P, R), Y, tol, max_iter)


# ---------------------------------------- multiple-level sketching ---

def walsh_hadamard(m: int) -> np.ndarray:
    """H_m of Section 4 from its recursive definition: H_2 = [[1, 1], [1, -1]],
    H_m = [[H_{m/2}, H_{m/2}], [H_{m/2}, -H_{m/2}]] (m a power of 2)."""
    if m < 1 or m & (m - 1):
        raise ValueError("m must be a power of 2")
    H = np.ones((1, 1))
    while H.shape[0] < m:
        H = np.block([[H, H], [H, -H]])
    return H


def srht_apply(Z1, signs, rows) -> np.ndarray:
    """Z2 = Z1 S2^T for the SRHT S2 = s2^-1/2 P H D of Section 4 (its definition):
    D = diag(signs) (m random signs), H = H_m, P keeps rows `rows` of H D.  The
    s1 columns of Z1 are padded with zeros to m = len(signs)."""
    Z1 = np.asarray(Z1, np.float64)
    m, s2 = len(signs), len(rows)
    if Z1.shape[1] > m:
        raise ValueError("m must be at least the number of columns of Z1")
    Zp = np.zeros((Z1.shape[0], m))
    Zp[:, :Z1.shape[1]] = Z1
    D = np.asarray(signs, np.float64)
    H = walsh_hadamard(m)
    S2 = H[np.asarray(rows), :] * D[None, :] / math.sqrt(s2)
    return Zp @ S2.T


def gaussian_projection(Z2, G) -> np.ndarray:
    """Z3 = s3^-1/2 Z2 S3^T with S3 = G, an s3 x s2 matrix of independent
    standard normal entries (Algorithm 2)."""
    G = np.asarray(G, np.float64)
    return np.asarray(Z2, np.float64) @ G.T / math.sqrt(G.shape[0])


def multilevel_features(Z1, signs, rows, G) -> np.ndarray:
    """Z3 of Algorithm 2: the SRHT of the first-level features, then the dense
    Gaussian projection."""
    return gaussian_projection(srht_apply(Z1, signs, rows), G)


def krr_multilevel_pcg_solve(X, Y, sigma: float, lam: float, W, b, signs, rows, G,
                             lam_p: float | None = None, tol: float = 1e-6,
                             max_iter: int = 1000) -> dict:
    """Algorithm 2 for the Gaussian kernel: random Fourier features Z1 (s1 of
    them), Z2 = Z1 S2^T (SRHT), Z3 = s3^-1/2 Z2 S3^T, then PCG on K + lambda I
    with the preconditioner Z3 Z3^T + lambda_p I in the Woodbury form."""
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64).reshape(X.shape[0], -1)
    Z3 = multilevel_features(rff_features(X, W, b), signs, rows, G)
    P = precond_setup(Z3, lam if lam_p is None else lam_p)
    A = kernel_matrix_system(X, sigma, lam)
    out = pcg(lambda V: A @ V, lambda R: precond_apply(P, R), Y, tol, max_iter)
    out["precond"] = P
    return out


# ---------------------------------------------- adaptive sketch size ---

def eig_projector(Z, thresh: float) -> np.ndarray:
    """P of Theorem 4: the orthogonal projection on the eigenvectors of Z Z^T
    whose eigenvalues exceed `thresh` (from the SVD Z = U S V^T: the columns of U
    with s_k^2 > thresh)."""
    U, sv, _ = np.linalg.svd(np.asarray(Z, np.float64), full_matrices=False)
    Uk = U[:, sv * sv > thresh]
    return Uk @ Uk.T


def condition1_norm(K, P) -> float:
    """||(I - P) K (I - P)||_2 of Theorem 4's first condition, exactly (dense)."""
    n = K.shape[0]
    R = np.eye(n) - P
    return float(np.max(np.abs(np.linalg.eigvalsh(R @ K @ R))))


def condition1_power(matvec, P, x0, iters: int) -> float:
    """Power iteration for ||(I - P) K (I - P)||_2 (Theorem 4: "testing condition 1
    can be accomplished using simple power-iteration"), from the start vector
    x0; `matvec` applies K.  Returns the last Rayleigh quotient."""
    x = np.asarray(x0, np.float64).reshape(-1)
    x = x / np.linalg.norm(x)
    est = 0.0
    for _ in range(iters):
        y = x - P @ x
        w = matvec(y)
        w = w - P @ w
        est = float(x @ w)
        nw = np.linalg.norm(w)
        if nw == 0.0:
            return 0.0
        x = w / nw
    return est


def adaptive_sketch_size(X, sigma: float, lam: float, W, b, s0: int, x0,
                         iters: int = 30) -> dict:
    """Section 5's adaptive choice of s with Theorem 4's first condition: from
    s = s0, form the random Fourier features of the first s columns of (W, b),
    test ||(I - P) K (I - P)|| <= 0.1 lambda (P: eigenvalues of Z Z^T above
    0.05 lambda) by power iteration from x0, and double s until the test passes
    or s reaches the number of columns of W (the second condition's test is
    left out, as in the paper)."""
    X = np.asarray(X, np.float64)
    s_max = np.asarray(W).shape[1]
    K = gaussian_kernel(X, X, sigma)
    s = s0
    history = []
    while True:
        Z = rff_features(X, np.asarray(W)[:, :s], np.asarray(b)[:s])
        P = eig_projector(Z, 0.05 * lam)
        est = condition1_power(lambda v: K @ v, P, x0, iters)
        history.append((s, est))
        if est <= 0.1 * lam or s >= s_max:
            return {"s": s, "Z": Z, "estimate": est, "history": history,
                    "passed": est <= 0.1 * lam}
        s = min(2 * s, s_max)


# ------------------------------------------------------------- gradient ---

def heldout_loss(X, Y, Xte, Yte, sigma: float, lam: float) -> float:
    """L = (1/m) ||K(Xte, X) c - yte||^2 with c from the direct solve of Eq. (1)."""
    C = direct_solve(X, Y, sigma, lam)
    F = predict(X, Xte, C, sigma)
    Yte = np.asarray(Yte, np.float64).reshape(F.shape)
    return float(np.sum((F - Yte) ** 2) / F.shape[0])


def hypergrad(X, Y, Xte, Yte, sigma: float, lam: float) -> dict:
    """Analytic dL/dlog(sigma) and dL/dlog(lambda) of ``heldout_loss``.

    With A = K + lambda I, c = A^-1 y, f = Kte c, g_f = (2/m)(f - yte),
    w = A^-1 Kte^T g_f and D_ij = ||x_i - x_j||^2 / sigma^2 (so that
    dK/dlog sigma = D o K):
        dL/dlog lambda = -lambda w.c
        dL/dlog sigma  = g_f.((Dte o Kte) c) - w.((D o K) c)
    """
    X = np.asarray(X, np.float64)
    Xte = np.asarray(Xte, np.float64)
    Y = np.asarray(Y, np.float64).reshape(X.shape[0], -1)
    Yte = np.asarray(Yte, np.float64).reshape(Xte.shape[0], -1)
    m = Xte.shape[0]
    Dtr = sqdist_direct(X, X) / (sigma * sigma)
    Dte = sqdist_direct(Xte, X) / (sigma * sigma)
    K = np.exp(-0.5 * Dtr)
    Kte = np.exp(-0.5 * Dte)
    A = K + lam * np.eye(X.shape[0])
    L = np.linalg.cholesky(A)

    def solve(B):
        return sla.solve_triangular(L.T, sla.solve_triangular(L, B, lower=True), lower=False)

    C = solve(Y)
    F = Kte @ C
    gF = (2.0 / m) * (F - Yte)
    Wd = solve(Kte.T @ gF)
    dlam = -lam * float(np.sum(Wd * C))
    dsig = float(np.sum(gF * ((Dte * Kte) @ C)) - np.sum(Wd * ((Dtr * K) @ C)))
    return {"dlogsigma": dsig, "dloglambda": dlam, "loss": float(np.sum((F - Yte) ** 2) / m),
            "c": C, "w": Wd}
