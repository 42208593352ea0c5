"""The oracle's LGL basis against the closed forms in tests/golden/ (nodes,
weights and derivative matrices of low degree, Sec. 2.2)."""
import os

import numpy as np
import pytest

from oracle import oracle as O

sympy = pytest.importorskip("sympy")
HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rows(name):
    out = []
    for line in open(os.path.join(HERE, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append(line.split())
    return out


def val(expr):
    return float(sympy.sympify(expr).evalf(30))


def test_lgl_nodes_and_weights_closed_forms():
    table = {}
    for N, i, x, w in rows("lgl_closed_forms.txt"):
        table.setdefault(int(N), []).append((int(i), val(x), val(w)))
    assert sorted(table) == [1, 2, 3, 4, 5]
    for N, entries in table.items():
        xi, w, _, _, _ = O.basis(N)
        assert len(entries) == N + 1
        for i, x, wt in entries:
            assert abs(xi[i] - x) < 2e-16 * 4, (N, i)
            assert abs(w[i] - wt) < 2e-16 * 8, (N, i)


def test_derivative_matrix_closed_forms():
    for r in rows("dmat_closed_forms.txt"):
        N, i = int(r[0]), int(r[1])
        _, _, D, _, _ = O.basis(N)
        ref = np.array([val(e) for e in r[2:]])
        assert np.max(np.abs(D[i] - ref)) < 1e-15, (N, i)
