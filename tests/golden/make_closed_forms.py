"""Write closed_forms.json: textbook singular values used to pin the oracle.

1D Dirichlet Laplacian tridiag(-1, 2, -1) of order n:
    lambda_j = 4 sin^2(j pi / (2 (n + 1))),  j = 1..n   (SPD: sigma = lambda)
2D 5-point Dirichlet Laplacian on an N x N grid:
    lambda_jk = 4 [sin^2(j pi / (2(N+1))) + sin^2(k pi / (2(N+1)))]
2x2 matrix [[a, b], [c, d]]: sigma^2 are the roots of
    s^2 - (a^2 + b^2 + c^2 + d^2) s + (ad - bc)^2 = 0.
Uses only the standard library (no oracle, no CUDA code).
"""
import json
import math
from pathlib import Path


def lap1d(n):
    h = math.pi / (2 * (n + 1))
    lam = [4 * math.sin(j * h) ** 2 for j in range(1, n + 1)]
    return {"n": n, "sigma_max": max(lam), "sigma_min": min(lam), "kappa": 1 / math.tan(h) ** 2}


def lap2d(N):
    h = math.pi / (2 * (N + 1))
    lam = [4 * (math.sin(j * h) ** 2 + math.sin(k * h) ** 2)
           for j in range(1, N + 1) for k in range(1, N + 1)]
    return {"N": N, "sigma_max": max(lam), "sigma_min": min(lam), "kappa": 1 / math.tan(h) ** 2}


def two_by_two(a, b, c, d):
    T = a * a + b * b + c * c + d * d
    D = (a * d - b * c) ** 2
    r = math.sqrt(T * T - 4 * D)
    smax2 = (T + r) / 2
    smin2 = D / smax2  # product of the roots, avoids cancellation
    return {"M": [[a, b], [c, d]], "sigma_max": math.sqrt(smax2), "sigma_min": math.sqrt(smin2)}


def main():
    out = {
        "lap1d": [lap1d(n) for n in (8, 10)],
        "lap2d": [lap2d(N) for N in (3, 4, 5)],
        "two_by_two": [two_by_two(3.0, 1.0, -2.0, 0.5), two_by_two(1.0, 2.0, 3.0, 4.0)],
    }
    Path(__file__).with_name("closed_forms.json").write_text(json.dumps(out, indent=1) + "\n")


if __name__ == "__main__":
    main()
