"""Write the small fixtures under tests/golden/ from the FP64 oracle only.

Run from the repository root:  python tests/golden/make_golden.py
The fixture freezes oracle outputs for a six-point problem so a later change
to the oracle's arithmetic shows up as a diff; its inputs are written out in
full so the file stands alone.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from oracle import krr_oracle as O  # noqa: E402


def main():
    X = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0], [0.5, -0.5], [-1.0, 0.25]])
    y = np.array([[1.0], [-1.0], [0.5], [2.0], [0.0], [-0.75]])
    W = np.array([[0.5, -1.25, 2.0], [1.5, 0.75, -0.5]])
    b = np.array([0.25, 3.0, 5.5])
    sigma, lam = 0.75, 0.1
    K = O.gaussian_kernel(X, X, sigma)
    C = O.direct_solve(X, y, sigma, lam)
    Z = O.rff_features(X, W, b)
    pre = O.precond_setup(Z, lam)
    pcg = O.krr_pcg_solve(X, y, sigma, lam, W, b, tol=1e-12)
    out = {
        "cite": "Eq. (1) system, Section 5 Gaussian kernel, Section 2.2 random Fourier "
                "features (sqrt(2/s) scale), Algorithm 1 / Section 3.1 Woodbury factors",
        "X": X.tolist(), "y": y.tolist(), "W": W.tolist(), "b": b.tolist(),
        "sigma": sigma, "lambda": lam,
        "K": K.tolist(), "c_direct": C.tolist(), "Z": Z.tolist(),
        "L": pre["L"].tolist(), "U": pre["U"].tolist(),
        "c_pcg": pcg["x"].tolist(), "pcg_iters": int(pcg["iters"][0]),
        "predict_at": [[0.25, 0.25], [2.0, -1.0]],
        "predict": O.predict(X, np.array([[0.25, 0.25], [2.0, -1.0]]), C, sigma).tolist(),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "six_point_problem.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
