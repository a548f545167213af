"""Writes exp2_poly.cuh: minimax polynomials for 2^f on [-1/2, 1/2], the
kernel of the FMA-pipe exp2 used beside the MUFU ex2 in the forward kernels.

Method: the Remez exchange algorithm for the best approximation in the
relative sense, max |p(f) / 2^f - 1| over [-1/2, 1/2] (Remez 1934; see e.g.
Muller, "Elementary Functions", ch. 3).  Starting from Chebyshev nodes, each
step solves the linear system p(x_i) - 2^x_i = (-1)^i E 2^x_i on deg + 2
reference points and moves the points to the extrema of the new error curve,
until the error equioscillates.  The coefficients are then rounded to FP32
(the precision the kernels evaluate them in) and the error of the rounded
polynomial is measured again on a fine grid.

Run from anywhere:  python paper_2412_20884_gb300/csrc/gen_exp2_poly.py
"""
from __future__ import annotations

import os

import numpy as np

DEGREES = (3, 5)
LO, HI = -0.5, 0.5


def remez(deg: int, iters: int = 40):
    n = deg + 2
    x = 0.5 * (LO + HI) + 0.5 * (HI - LO) * np.cos(np.pi * np.arange(n)[::-1] / (n - 1))
    grid = np.linspace(LO, HI, 200001)
    coef = None
    for _ in range(iters):
        A = np.zeros((n, n))
        for i in range(n):
            A[i, :deg + 1] = x[i] ** np.arange(deg + 1)
            A[i, deg + 1] = (-1) ** i * np.exp2(x[i])
        sol = np.linalg.solve(A, np.exp2(x))
        coef = sol[:deg + 1]
        err = np.polynomial.polynomial.polyval(grid, coef) / np.exp2(grid) - 1.0
        # one extremum of |err| between consecutive sign changes
        segs = np.split(np.arange(grid.size), np.where(np.diff(np.sign(err)) != 0)[0] + 1)
        ext = np.array([s[np.argmax(np.abs(err[s]))] for s in segs])
        if ext.size != n:
            break
        x_new = grid[ext]
        if np.max(np.abs(x_new - x)) < 1e-12:
            x = x_new
            break
        x = x_new
    return coef


def rounded_error(coef32: np.ndarray) -> float:
    grid = np.linspace(LO, HI, 400001)
    p = np.polynomial.polynomial.polyval(grid, coef32.astype(np.float64))
    return float(np.max(np.abs(p / np.exp2(grid) - 1.0)))


def main() -> None:
    lines = [
        "// Generated by gen_exp2_poly.py: minimax (relative error) polynomials",
        "// for 2^f on [-1/2, 1/2], coefficients rounded to FP32, in Horner form.",
        "#pragma once",
        "",
        "#include <cuda_runtime.h>",
        "",
        "namespace kmv {",
    ]
    for deg in DEGREES:
        c32 = remez(deg).astype(np.float32)
        err = rounded_error(c32)
        # Horner form with the literal coefficients, highest degree innermost
        expr = f"{float(c32[deg])!r}f"
        for k in range(deg - 1, -1, -1):
            expr = f"fmaf({expr}, f, {float(c32[k])!r}f)"
        lines.append(f"// degree {deg}: max relative error {err:.3e} (FP64 evaluation of the FP32 coefficients)")
        lines.append(f"__host__ __device__ __forceinline__ float exp2_poly{deg}(float f) {{ return {expr}; }}")
        lines.append(f"constexpr double kExp2Poly{deg}Err = {err:.6e};")
    lines.append("}  // namespace kmv")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "exp2_poly.cuh")
    with open(out, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
