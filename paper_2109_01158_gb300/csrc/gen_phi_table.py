#!/usr/bin/env python
"""Writes phi_table_f64.h: the breakpoint table of phi(x) = x - log(1 + x) used by the FP64
element kernels.

Breakpoints c_j = (j - J0) / 1024, j = 0 .. N - 1, cover x in [-306/1024, 306/1024].  For each
breakpoint, with F_j = 1 + c_j (exact dyadic rationals):
  A_j = c_j - ln(F_j)  (= phi(c_j))  as a pair of doubles hi + lo,
  B_j = c_j / F_j      (= 1 - 1/F_j) rounded to double,
  R_j = 1 / F_j                       rounded to double.
The values are computed with Python's decimal module at 60 significant digits (its ln is
correctly rounded at that precision) and each double is the correctly rounded conversion.
Run from this directory: python gen_phi_table.py > phi_table_f64.h
"""
from decimal import Decimal, getcontext

getcontext().prec = 60

SCALE = 1024
J0 = 306
N = 613


def split(d: Decimal):
    hi = float(d)
    lo = float(d - Decimal(hi))
    return hi, lo


def main():
    rows = []
    for j in range(N):
        c = Decimal(j - J0) / SCALE
        F = 1 + c
        A = c - F.ln()
        hi, lo = split(A)
        B = float(c / F)
        R = float(1 / F)
        rows.append((hi, lo, B, R))
    out = ["// Generated by gen_phi_table.py: breakpoints of phi(x) = x - log(1 + x).",
           "// Row j: {A_hi, A_lo, B, R} at c_j = (j - FE_PHI_J0) / FE_PHI_SCALE with F_j = 1 + c_j:",
           "// A = c_j - ln(F_j) (hi + lo), B = c_j / F_j, R = 1 / F_j.",
           "#pragma once",
           f"#define FE_PHI_SCALE {SCALE}",
           f"#define FE_PHI_J0 {J0}",
           f"#define FE_PHI_N {N}",
           "#define FE_PHI_TABLE_ROWS \\"]
    for k, (hi, lo, B, R) in enumerate(rows):
        sep = "," if k + 1 < N else ""
        out.append(f"  {{{hi.hex()}, {lo.hex()}, {B.hex()}, {R.hex()}}}{sep} \\")
    out.append("")
    print("\n".join(out))


if __name__ == "__main__":
    main()
