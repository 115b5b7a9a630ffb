"""The integer facts the FP64 kernels rely on (CPU; no GPU needed).

The FP64 stage kernel forms chi's stencil sums, and the FP64 prolongation each
interpolation line, exactly in 64-bit integers.  That is exact only because the
coefficients involved are integers and the sums stay inside the bounds the kernels' shifts
were chosen for:

* the 4th-order second difference (-1, 16, -30, 16, -1) and the Kreiss-Oliger sixth
  difference (1, -6, 15, -20, 15, -6, 1) summed over three axes give integer weights whose
  absolute sums are 192 at most (Sec. 4 wave equation, R3);
* 46080 = 2^6 x 720 times every weight of the degree-6 Lagrange interpolation from 7 nodes
  to the 13 half-node positions (Sec. 3.3, Fig. unzip) is an integer, with absolute sums at
  most 196,470 per position and 332,640 over a mirrored pair's combined sum and difference
  weights; with inputs below 2^62 split into 31-bit halves those keep every accumulator
  below 2^49.4, and the kernel's final shift by 18 keeps results below 2^63.

The weights are derived here as exact rationals from the interpolation's definition and
compared with the oracle's floating-point table."""
from fractions import Fraction
from math import comb, log2

import numpy as np

D = 46080


def lagrange_half_node_weights():
    """W[r][j] = l_j(r / 2), the Lagrange basis on nodes 0..6 at half-node position r"""
    W = []
    for r in range(13):
        x = Fraction(r, 2)
        row = []
        for j in range(7):
            w = Fraction(1)
            for m in range(7):
                if m != j:
                    w *= (x - m) / (j - m)
            row.append(w)
        W.append(row)
    return W


def test_stencil_weight_sums():
    lap = [-90] + [16] * 6 + [-1] * 6  # centre, distance 1 (6), distance 2 (6): 12 h^2 Laplacian
    ko = [-60] + [15] * 6 + [-6] * 6 + [1] * 6  # the three axes' sixth differences summed
    assert sum(abs(c) for c in lap) == 192 and sum(abs(c) for c in ko) == 192
    # 192 x 2^53 < 2^61: the exact sums of 53-bit grid values fit in 64 bits
    assert 192 * 2 ** 53 < 2 ** 61


def test_interpolation_weights_are_integers_over_46080():
    W = lagrange_half_node_weights()
    for r in range(13):
        c = [w * D for w in W[r]]
        assert all(v.denominator == 1 for v in c), r
        if r % 2 == 0:  # nodes: copies
            assert c == [D if j == r // 2 else 0 for j in range(7)]
        else:  # the closed form C(6, j) (-1)^(6 - j) prod_{m != j} (r - 2m)
            for j in range(7):
                p = 1
                for m in range(7):
                    if m != j:
                        p *= r - 2 * m
                assert c[j] == comb(6, j) * (-1) ** (6 - j) * p
        # mirror symmetry the pair form uses: W[12 - r][j] = W[r][6 - j]
        assert all(W[12 - r][j] == W[r][6 - j] for j in range(7))


def test_interpolation_bounds_behind_the_shifts():
    W = lagrange_half_node_weights()
    worst_sum, worst_pair = 0, 0
    for k in (1, 3, 5):
        c = [int(w * D) for w in W[k]]
        worst_sum = max(worst_sum, sum(abs(v) for v in c))
        ec = [c[j] + c[6 - j] for j in range(3)] + [2 * c[3]]
        oc = [c[j] - c[6 - j] for j in range(3)]
        worst_pair = max(worst_pair, sum(map(abs, ec)) + sum(map(abs, oc)))
        assert max(map(abs, ec + oc)) < 2 ** 31  # 32-bit weights for mad.wide
    assert worst_sum == 196470 and log2(worst_sum) < 17.6
    assert worst_pair == 332640
    # halves of inputs below 2^62 are below 2^31: accumulators below 2^49.4 ...
    acc = worst_pair * 2 ** 31
    assert log2(acc) < 49.4
    # ... and the final shift by 18 (high half shifted left by 31 - 18 = 13) stays below 2^63
    assert acc * 2 ** 13 < 2 ** 63


def test_oracle_table_matches_the_exact_weights():
    """the oracle's FP64 table rounds the exact rationals (so 46080 W rounds to the integer)"""
    import oracle as O
    Wf = O.interp_weights()
    W = lagrange_half_node_weights()
    for r in range(13):
        for j in range(7):
            assert abs(Wf[r, j] - float(W[r][j])) <= 2 ** -52 * max(1.0, abs(float(W[r][j])))
            assert round(D * Wf[r, j]) == D * W[r][j]
            assert abs(D * Wf[r, j] - round(D * Wf[r, j])) < 1e-9
    assert np.isfinite(Wf).all()
