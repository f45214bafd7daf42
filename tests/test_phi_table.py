"""The FP64 kernels' phi(x) = x - log(1 + x) and 1/(1 + x) for |x| < 306/1024 come from a
breakpoint table (csrc/phi_table_f64.h) and short series.  The table rows are checked against
60-digit decimal values, and the kernels' arithmetic is replayed on the CPU with every
operation rounded once, as on the GPU (a fused multiply-add rounds the exact a*b + c).  The
replay is compared with exact or 60-digit references: phi within 6 and 1/(1 + x) within 3
units of 2^-53 relative."""
import os
import random
import re
from decimal import Decimal, getcontext
from fractions import Fraction as Fr

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2109_01158_gb300", "csrc",
                   "phi_table_f64.h")


def _table():
    txt = open(HDR).read()
    scale = int(re.search(r"FE_PHI_SCALE (\d+)", txt).group(1))
    j0 = int(re.search(r"FE_PHI_J0 (\d+)", txt).group(1))
    n = int(re.search(r"FE_PHI_N (\d+)", txt).group(1))
    rows = re.findall(r"\{([^}]*)\}", txt.split("FE_PHI_TABLE_ROWS")[1])
    tab = [[float.fromhex(x.strip()) for x in r.split(",")] for r in rows]
    assert len(tab) == n
    return scale, j0, tab


def _fma(a, b, c):
    return float(Fr(a) * Fr(b) + Fr(c))


def _mul(a, b):
    return float(Fr(a) * Fr(b))


def _add(a, b):
    return float(Fr(a) + Fr(b))


def _kernel_phi_rcp(x, scale, j0, tab):
    """phi_arg / phi_from / rcp_from of the FP64 kernels, one rounding per operation."""
    shift = 1.5 * 2.0 ** 52
    t = _fma(x, float(scale), shift)
    k = int(t - shift)
    a_hi, a_lo, b, rj = tab[k + j0]
    f = _fma(t - shift, -1.0 / scale, x)
    assert Fr(f) == Fr(x) - Fr(k, scale)          # x - c_j is exact
    r = _mul(f, rj)
    s = _add(1.0, -r)
    for _ in range(4):
        s = _fma(-r, s, 1.0)
    p = 1.0 / 6.0
    for c in (-1.0 / 5.0, 1.0 / 4.0, -1.0 / 3.0, 1.0 / 2.0):
        p = _fma(p, r, c)
    psi = _mul(_mul(r, r), p)
    return _add(a_hi, _add(a_lo, _fma(f, b, psi))), _mul(rj, s)


def _phi_exact(x):
    if abs(x) < 1e-6:
        X = Fr(x)
        return sum(((-1) ** k) * X ** k / k for k in range(2, 9))
    getcontext().prec = 60
    d = Decimal(x)
    return Fr(d - (1 + d).ln())


def test_table_rows_are_the_correctly_rounded_values():
    scale, j0, tab = _table()
    getcontext().prec = 60
    for j in list(range(0, len(tab), 37)) + [j0, len(tab) - 1]:
        c = Decimal(j - j0) / scale
        F = 1 + c
        A = c - F.ln()
        a_hi, a_lo, b, r = tab[j]
        assert a_hi == float(A) and a_lo == float(A - Decimal(a_hi))
        assert b == float(c / F) and r == float(1 / F)


def test_kernel_phi_and_reciprocal_accuracy():
    scale, j0, tab = _table()
    lim = 306 / 1024
    rnd = random.Random(7)
    xs = [rnd.uniform(-lim, lim) for _ in range(1200)] + [rnd.uniform(-2e-3, 2e-3) for _ in range(400)]
    xs += [k / scale + d for k in range(-306, 307, 17) for d in (0.4995 / scale, -0.4995 / scale, 1e-9)
           if abs(k / scale + d) < lim]
    xs += [1e-8, -1e-8, 0.2988, -0.2988]
    worst_phi = worst_rcp = 0.0
    for x in xs:
        phi, rcp = _kernel_phi_rcp(x, scale, j0, tab)
        ref = _phi_exact(x)
        worst_phi = max(worst_phi, float(abs(Fr(phi) - ref) / abs(ref)) / 2.0 ** -53)
        rr = 1 / (1 + Fr(x))
        worst_rcp = max(worst_rcp, float(abs(Fr(rcp) - rr) / rr) / 2.0 ** -53)
    assert worst_phi <= 6.0, worst_phi
    assert worst_rcp <= 3.0, worst_rcp
