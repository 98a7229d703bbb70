"""Pins of the oracle's lattice tables against what the paper fixes.

The paper does not print the weights.  It states the constraints they obey:
normalisation (sum of weights = 1) and second moment = c_s^2 = 1/3 (the
constraints stated after Eq. (2)), isotropy of the lattice tensors up to 8th
order for the 24-speed lattice (paragraph after Fig. 4), and, through the
effective couplings after Eq. (5), a ratio 12/7 between the fourth moments of
the p and w weight systems.  Here the p weights are solved for exactly from
those constraints (rational arithmetic) and compared with the oracle's table.
"""
from fractions import Fraction as Fr

import numpy as np

SHELLS = {1: [(1, 0), (0, 1), (-1, 0), (0, -1)],
          2: [(1, 1), (-1, 1), (-1, -1), (1, -1)],
          4: [(2, 0), (0, 2), (-2, 0), (0, -2)],
          5: [(2, 1), (1, 2), (-1, 2), (-2, 1), (-2, -1), (-1, -2), (1, -2), (2, -1)],
          8: [(2, 2), (-2, 2), (-2, -2), (2, -2)]}


def shell_moment(shell, a, b):
    return sum(Fr(cx) ** a * Fr(cy) ** b for cx, cy in SHELLS[shell])


def solve(A, rhs):
    """Exact Gauss-Jordan elimination over the rationals."""
    n = len(A)
    M = [list(map(Fr, row)) + [Fr(r)] for row, r in zip(A, rhs)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        M[c] = [v / M[c][c] for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                M[r] = [a - M[r][c] * b for a, b in zip(M[r], M[c])]
    return [M[r][n] for r in range(n)]


def exact_p():
    """Shell weights p(|c|^2) for |c|^2 in (1, 2, 4, 5, 8)."""
    sh = [1, 2, 4, 5, 8]
    rows, rhs = [], []
    # second moment per Cartesian component = c_s^2
    rows.append([shell_moment(s, 2, 0) for s in sh]); rhs.append(Fr(1, 3))
    # 4th order isotropy: <x^4> = 3 <x^2 y^2>
    rows.append([shell_moment(s, 4, 0) - 3 * shell_moment(s, 2, 2) for s in sh]); rhs.append(0)
    # 6th order isotropy: <x^6> = 5 <x^4 y^2>
    rows.append([shell_moment(s, 6, 0) - 5 * shell_moment(s, 4, 2) for s in sh]); rhs.append(0)
    # 8th order isotropy: <x^8> : <x^6 y^2> : <x^4 y^4> = 105 : 15 : 9
    rows.append([9 * shell_moment(s, 8, 0) - 105 * shell_moment(s, 4, 4) for s in sh]); rhs.append(0)
    rows.append([9 * shell_moment(s, 6, 2) - 15 * shell_moment(s, 4, 4) for s in sh]); rhs.append(0)
    return dict(zip(sh, solve(rows, rhs)))


def test_multirange_weights_solve_matches_oracle(O):
    p_exact = exact_p()
    assert p_exact == {1: Fr(4, 63), 2: Fr(4, 135), 4: Fr(1, 180), 5: Fr(2, 945), 8: Fr(1, 15120)}
    cx, cy = O.velocities()
    w, p = O.weights()
    for i in range(1, 25):
        c2 = int(cx[i] ** 2 + cy[i] ** 2)
        assert p[i] == float(p_exact[c2]), (i, c2)
    # rest weight closes the normalisation sum p = 1
    p0 = 1 - sum(len(SHELLS[s]) * p_exact[s] for s in SHELLS)
    assert abs(p[0] - float(p0)) < 4e-16  # a 24-term float sum
    assert p0 == Fr(247, 420)


def test_velocity_sets(O):
    cx, cy = O.velocities()
    vecs = list(zip(cx.tolist(), cy.tolist()))
    assert vecs[0] == (0, 0)
    belt1 = set(vecs[1:9])
    belt2 = set(vecs[9:25])
    assert belt1 == set(SHELLS[1]) | set(SHELLS[2])            # b1 = 8
    assert belt2 == set(SHELLS[4]) | set(SHELLS[5]) | set(SHELLS[8])  # b2 = 16
    assert len(set(vecs)) == 25
    for i in range(9):
        j = O.opposite(i)
        assert (cx[j], cy[j]) == (-cx[i], -cy[i])


def test_d2q9_weights(O):
    cx, cy = O.velocities()
    w, _ = O.weights()
    W = [Fr(4, 9)] + [Fr(1, 9)] * 4 + [Fr(1, 36)] * 4
    assert [float(v) for v in W] == w.tolist()
    c = list(zip(cx[:9], cy[:9]))
    assert sum(W) == 1
    assert sum(wi * x * x for wi, (x, y) in zip(W, c)) == Fr(1, 3)
    assert sum(wi * x * y for wi, (x, y) in zip(W, c)) == 0
    assert sum(wi * x ** 4 for wi, (x, y) in zip(W, c)) == 3 * sum(
        wi * x * x * y * y for wi, (x, y) in zip(W, c))


def test_isotropy_and_twelve_sevenths(O):
    """All odd moments vanish, even moments are isotropic to 8th order, and
    sum p c_x^4 / sum w c_x^4 = 12/7 (effective couplings after Eq. (5))."""
    cx, cy = O.velocities()
    w, p = O.weights()
    pe = exact_p()
    P = [(Fr(int(x)), Fr(int(y)), pe[int(x * x + y * y)]) for x, y in zip(cx[1:], cy[1:])]
    W = [(Fr(int(x)), Fr(int(y)), Fr(1, 9) if x * x + y * y == 1 else Fr(1, 36))
         for x, y in zip(cx[1:9], cy[1:9])]

    def mom(S, a, b):
        return sum(k * x ** a * y ** b for x, y, k in S)

    for a in range(0, 9):
        for b in range(0, 9 - a):
            if (a + b) % 2 == 1 or a % 2 == 1 or b % 2 == 1:
                assert mom(P, a, b) == 0
    assert mom(P, 2, 0) == mom(P, 0, 2) == Fr(1, 3)
    assert mom(P, 4, 0) == 3 * mom(P, 2, 2)
    assert mom(P, 6, 0) == 5 * mom(P, 4, 2) == 5 * mom(P, 2, 4)
    assert 9 * mom(P, 8, 0) == 105 * mom(P, 4, 4)
    assert 9 * mom(P, 6, 2) == 15 * mom(P, 4, 4)
    assert mom(P, 4, 0) / mom(W, 4, 0) == Fr(12, 7)
    # fourth-order lattice constants of the Taylor expansion of Eq. (2)
    assert mom(W, 2, 2) == Fr(1, 9) and mom(P, 2, 2) == Fr(4, 21)
    # the floats in the oracle are the correctly rounded rationals
    assert np.allclose(p[1:], [float(k) for _, _, k in P], rtol=0, atol=0)
