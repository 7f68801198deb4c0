"""Writes the closed-form fixtures in this folder with exact symbolic arithmetic
(sympy), independent of both the oracle and the CUDA path.

laplacian_n8_eigs.txt: eigenvalues 2 - 2 cos(k pi / 9), k = 1..8, of the 8 x 8
1D Laplacian tridiag(-1, 2, -1), to 25 significant digits.
"""
from pathlib import Path

import sympy as sp

HERE = Path(__file__).resolve().parent


def main():
    n = 8
    vals = [sp.N(2 - 2 * sp.cos(k * sp.pi / (n + 1)), 25) for k in range(1, n + 1)]
    (HERE / "laplacian_n8_eigs.txt").write_text(
        "# 1D Laplacian n=8: lambda_k = 2 - 2 cos(k pi/9), exact to 25 digits (sympy)\n"
        + "\n".join(str(v) for v in vals) + "\n")


if __name__ == "__main__":
    main()
