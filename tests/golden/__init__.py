"""Hand-derived worked examples (JSON) and their loader.

Every expected value in these files is a closed form derived by hand from the
paper's definitions, written as an arithmetic expression (numbers, + - * /,
parentheses and sqrt); nothing here is produced by either implementation.
"""
import ast
import json
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))


def load(name):
    with open(os.path.join(_HERE, name)) as f:
        return json.load(f)


def value(expr):
    """Evaluates an expression of numbers, + - * /, parentheses and sqrt."""

    def ev(node):
        if isinstance(node, ast.Expression):
            return ev(node.body)
        if isinstance(node, ast.Constant) and isinstance(node.value, (int, float)):
            return float(node.value)
        if isinstance(node, ast.UnaryOp) and isinstance(node.op, ast.USub):
            return -ev(node.operand)
        if isinstance(node, ast.BinOp):
            a, b = ev(node.left), ev(node.right)
            ops = {ast.Add: lambda: a + b, ast.Sub: lambda: a - b, ast.Mult: lambda: a * b,
                   ast.Div: lambda: a / b}
            if type(node.op) in ops:
                return ops[type(node.op)]()
        if (isinstance(node, ast.Call) and isinstance(node.func, ast.Name)
                and node.func.id == "sqrt" and len(node.args) == 1 and not node.keywords):
            return math.sqrt(ev(node.args[0]))
        raise ValueError(f"unsupported expression: {expr!r}")

    return ev(ast.parse(str(expr), mode="eval"))


def _bound(v, inf):
    return np.array([inf if e is None else e for e in v], dtype=np.float64)


def lp_data(case):
    """The case's LP as an lpgen.LPData (CSR from the dense A; null bounds = infinite)."""
    from paper_2105_12715_gb300 import lpgen

    m, n = len(case["b"]), len(case["c"])
    A = np.array(case["A"], dtype=np.float64).reshape(m, n)
    rows, cols = np.nonzero(A)
    row_ptr = np.zeros(m + 1, dtype=np.int32)
    np.cumsum(np.bincount(rows, minlength=m), out=row_ptr[1:])
    return lpgen.LPData(m, n, row_ptr, cols.astype(np.int32), A[rows, cols],
                        np.array(case["c"], dtype=np.float64),
                        np.array(case["b"], dtype=np.float64),
                        _bound(case["lb"], -np.inf), _bound(case["ub"], np.inf),
                        np.array(case["row_type"], dtype=np.int8))
