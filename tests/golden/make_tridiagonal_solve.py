"""Writes tridiagonal_solve.json: solve(A, b) for a 16 x 16 tridiagonal A
with small-integer entries, zeros at every fifth diagonal position (so
elimination must exchange rows), and b = A x for an integer x.  The expected
solution is x itself, exact by construction; b is computed here with
integer arithmetic (Sec. III (10): solve(A, b) with A tridiagonal)."""
import json
import os

n = 16
x = [((7 * i) % 11) - 5 for i in range(n)]
A = [[0] * n for _ in range(n)]
for i in range(n):
    A[i][i] = 0 if i % 5 == 0 else (i % 4) + 2
    if i + 1 < n:
        A[i + 1][i] = (i % 3) + 1          # subdiagonal
        A[i][i + 1] = -((i % 2) + 1)       # superdiagonal
b = [[sum(A[i][j] * x[j] for j in range(n))] for i in range(n)]
fx = {
    "cite": "Sec. III, expression (10): solve(A, b) with A tridiagonal; the band solver must "
            "exchange rows where the diagonal is zero",
    "how": "x chosen (integers), b = A x in integer arithmetic, expected = x exactly",
    "inputs": {"A": A, "b": b},
    "nodes": [{"op": "input", "slot": 0, "rows": n, "cols": n},
              {"op": "input", "slot": 1, "rows": n, "cols": 1},
              {"op": "solve", "a": 0, "b": 1}],
    "slots": ["A", "b"], "outputs": [2],
    "expected": [[[v] for v in x]], "tol": 1e-13,
}
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "tridiagonal_solve.json"), "w") as f:
    json.dump(fx, f)
