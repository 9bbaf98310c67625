"""Pins of the oracle against values the paper prints (fixtures under
tests/golden/, each citing its table or appendix)."""

import ast
import math
import operator
from fractions import Fraction
from pathlib import Path

import numpy as np

from oracle import schemes as S

GOLDEN = Path(__file__).parent / "golden"


def _rows(name):
    return [ln.split() for ln in (GOLDEN / name).read_text().splitlines() if ln.strip() and not ln.startswith("#")]


_OPS = {ast.Add: operator.add, ast.Sub: operator.sub, ast.Mult: operator.mul, ast.Div: operator.truediv}


def _value(expr):
    # +, -, *, /, sqrt(), parentheses and integer literals only
    def ev(n):
        if isinstance(n, ast.Expression):
            return ev(n.body)
        if isinstance(n, ast.Constant) and isinstance(n.value, int):
            return float(n.value)
        if isinstance(n, ast.BinOp) and type(n.op) in _OPS:
            return _OPS[type(n.op)](ev(n.left), ev(n.right))
        if isinstance(n, ast.UnaryOp) and isinstance(n.op, ast.USub):
            return -ev(n.operand)
        if isinstance(n, ast.Call) and isinstance(n.func, ast.Name) and n.func.id == "sqrt" and len(n.args) == 1:
            return math.sqrt(ev(n.args[0]))
        raise ValueError(f"unsupported expression {expr!r}")
    return ev(ast.parse(expr, mode="eval"))


def test_gauss_legendre_table():
    # Table tab:GaussLeg: the oracle's rules equal the printed closed forms, and
    # the printed closed forms equal numpy's Gauss-Legendre rule mapped to [0, 1]
    rows = _rows("gauss_legendre.txt")
    for M in range(1, 5):
        xs = [_value(r[2]) for r in rows if int(r[0]) == M]
        ws = [_value(r[3]) for r in rows if int(r[0]) == M]
        x, w = S.gauss_legendre(M)
        assert np.allclose(x, xs, atol=1e-15, rtol=0) and np.allclose(w, ws, atol=1e-15, rtol=0)
        t, v = np.polynomial.legendre.leggauss(M)
        assert np.allclose((t + 1) / 2, xs, atol=1e-14) and np.allclose(v / 2, ws, atol=1e-14)


def test_cf65_f21_printed_digits():
    # Appendix C: f21 of CF6:5 with f11 = 4/25 to the 9 printed digits, and the
    # printed quintic has exactly one real root there
    f11, digits, coeffs = _rows("cf65_f21.txt")
    f = S.full_table(S.SCHEMES["CF6:5"])
    assert f[0, 0] == float(Fraction(f11[0]))
    assert abs(f[1, 0] - float(digits[0])) < 5e-10
    roots = np.roots([float(c) for c in coeffs][::-1])
    real = roots[np.abs(roots.imag) < 1e-9].real
    assert len(real) == 1 and abs(real[0] - float(digits[0])) < 5e-10
