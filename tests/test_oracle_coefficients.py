"""Pins of the oracle's composition/splitting coefficients against what the
paper prints (Table II, the fourth-order coefficients of Sec. II E) and
against textbook identities (order conditions, sums, symmetry)."""
import os
from decimal import Decimal

import pytest

from oracle import coefficients as C

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2.txt")


def _table2():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        sch, o, before, after, na, nb = line.split()
        rows.append((sch, int(o), int(before), int(after), int(na), int(nb)))
    return rows


@pytest.mark.parametrize("row", _table2(), ids=lambda r: f"{r[0]}{r[1]}")
def test_table2_counts(row):
    sch, order, before, after, na, nb = row
    sp = C.Splitting(order, {"elementary": C.TRIPLE_JUMP, "triple_jump": C.TRIPLE_JUMP, "suzuki": C.SUZUKI,
                             "optimal": C.OPTIMAL}[sch])
    assert sp.n_actions_before == before
    assert sp.n_actions_after == after
    assert len(sp.a_unq_dec) == na
    assert len(sp.b_unq_dec) == nb
    # footnotes of Table II: N_A = 2 N_B before, N_A = N_B + 1 after the merge
    assert len(sp.a_full) == 2 * sum(1 for b in sp.b_full if b != 0)
    assert len(sp.a) == len(sp.b) + 1


def test_fourth_order_triple_jump_printed_coefficients():
    """Eq. (triple_jump_fourth_order_so): N = 6, a_1 = a_2 = 1/(2(2-2^{1/3})),
    a_3 = -2^{1/3}/(2(2-2^{1/3})), b_1 = 1/(2-2^{1/3}), b_3 = -2^{1/3}/(2-2^{1/3}),
    b_2 = b_6 = 0, the rest by symmetry."""
    r = 2.0 ** (1.0 / 3.0)
    a = [1 / (2 * (2 - r)), 1 / (2 * (2 - r)), -r / (2 * (2 - r))]
    b = [1 / (2 - r), 0.0, -r / (2 - r)]
    a = a + a[::-1]                       # a_{N-j+1} = a_j
    b = b + [b[1], b[0], 0.0]             # b_{N-j} = b_j, b_6 = 0
    sp = C.Splitting(4, C.TRIPLE_JUMP, pruned=False)
    assert len(sp.a) == 6
    for x, y in zip(sp.a, a):
        assert x == pytest.approx(y, rel=1e-14, abs=1e-15)
    for x, y in zip(sp.b, b):
        assert x == pytest.approx(y, rel=1e-14, abs=1e-15)


def test_fourth_order_suzuki_printed_coefficients():
    """Eq. (suzukis_fractals_fourth_order_so): N = 10, a_1..a_4 =
    1/(2(4-4^{1/3})), a_5 = -4^{1/3}/(2(4-4^{1/3})), b_1 = b_3 = 1/(4-4^{1/3}),
    b_2 = b_4 = b_10 = 0, b_5 = -4^{1/3}/(4-4^{1/3})."""
    r = 4.0 ** (1.0 / 3.0)
    y = 1 / (4 - r)
    a = [y / 2] * 4 + [-r * y / 2]
    a = a + a[::-1]
    b = [y, 0.0, y, 0.0, -r * y]
    b = b + [b[3], b[2], b[1], b[0], 0.0]
    sp = C.Splitting(4, C.SUZUKI, pruned=False)
    assert len(sp.a) == 10
    for x, yv in zip(sp.a, a):
        assert x == pytest.approx(yv, rel=1e-14, abs=1e-15)
    for x, yv in zip(sp.b, b):
        assert x == pytest.approx(yv, rel=1e-14, abs=1e-15)


@pytest.mark.parametrize("scheme", [C.TRIPLE_JUMP, C.SUZUKI])
@pytest.mark.parametrize("p", [2, 4, 6, 8])
def test_order_conditions(scheme, p):
    """A symmetric composition raises the order from p to p+2 when
    sum gamma = 1 and sum gamma^{p+1} = 0 (textbook condition)."""
    g = C.gamma_triple_jump(p) if scheme == C.TRIPLE_JUMP else C.gamma_suzuki(p)
    assert abs(sum(g) - 1) < Decimal("1e-50")
    assert abs(sum(x ** (p + 1) for x in g)) < Decimal("1e-50")
    assert g == g[::-1]


@pytest.mark.parametrize("scheme", [C.TRIPLE_JUMP, C.SUZUKI])
@pytest.mark.parametrize("order", [2, 4, 6, 8, 10])
@pytest.mark.parametrize("pruned", [False, True])
def test_sums_and_symmetry(scheme, order, pruned):
    sp = C.Splitting(order, scheme, pruned)
    assert abs(sum(sp.a_dec) - 1) < Decimal("1e-50")
    assert abs(sum(sp.b_dec) - 1) < Decimal("1e-50")
    a, b = sp.a_dec, sp.b_dec
    if pruned:
        # pruned sequences are palindromes: a~ (N_B+1 entries) and b~ (N_B)
        assert all(abs(a[j] - a[-1 - j]) < Decimal("1e-50") for j in range(len(a)))
        assert all(abs(b[j] - b[-1 - j]) < Decimal("1e-50") for j in range(len(b)))
        assert all(x != 0 for x in b)
    else:
        N = len(a)
        # Eq. (symmetric_splitting_coefficients), 1-based: a_{N-j+1} = a_j, b_{N-j} = b_j
        assert all(abs(a[j] - a[N - 1 - j]) < Decimal("1e-50") for j in range(N))
        assert all(abs(b[j] - b[N - 2 - j]) < Decimal("1e-50") for j in range(N - 1))
        assert b[N - 1] == 0


@pytest.mark.parametrize("scheme", [C.TRIPLE_JUMP, C.SUZUKI])
@pytest.mark.parametrize("order", [4, 6, 8, 10])
def test_index_arrays_reproduce_sequence(scheme, order):
    sp = C.Splitting(order, scheme)
    for j, v in enumerate(sp.a_dec):
        assert abs(sp.a_unq_dec[sp.Ia[j]] - v) <= Decimal("1e-12") * abs(v)
    for j, v in enumerate(sp.b_dec):
        assert abs(sp.b_unq_dec[sp.Ib[j]] - v) <= Decimal("1e-12") * abs(v)
    # the unique values are genuinely distinct
    u = sorted(float(x) for x in sp.a_unq_dec)
    assert all(u[i + 1] - u[i] > 1e-6 for i in range(len(u) - 1))


def test_composition_length_and_bad_input():
    assert len(C.composition(10, C.TRIPLE_JUMP)) == 81
    assert len(C.composition(10, C.SUZUKI)) == 625
    with pytest.raises(ValueError):
        C.composition(3, C.SUZUKI)
    with pytest.raises(ValueError):
        C.composition(4, "optimal")


@pytest.mark.parametrize("order,scheme", [(4, C.TRIPLE_JUMP), (6, C.SUZUKI), (8, C.TRIPLE_JUMP)])
def test_explicit_gammas_reproduce_the_recursive_schemes(order, scheme):
    """Splitting from explicit elementary-step coefficients (any symmetric
    composition) equals the recursive construction when given its gammas
    (rounded to double: the values agree to 1e-15)."""
    ref = C.Splitting(order, scheme)
    sp = C.Splitting(order, scheme, gammas=[float(g) for g in C.composition(order, scheme)])
    assert len(sp.a) == len(ref.a) and len(sp.b) == len(ref.b)
    assert max(abs(x - y) for x, y in zip(sp.a + sp.b, ref.a + ref.b)) < 1e-14
    assert sp.Ia == ref.Ia and sp.Ib == ref.Ib


@pytest.mark.parametrize("order", [6, 8])
def test_optimal_compositions_order_conditions(order):
    """Consistency and the power-sum conditions sum gamma^k = 0 for odd
    k = 3..order-1 that every symmetric composition of a symmetric
    second-order method of this order must meet (the other order conditions
    are checked by the measured convergence order in the propagation tests);
    symmetric and of the stage counts of Table II (9 and 17)."""
    g = C.composition(order, C.OPTIMAL)
    assert len(g) == {6: 9, 8: 17}[order]
    assert all(g[k] == g[-1 - k] for k in range(len(g)))
    assert abs(sum(g) - 1) < Decimal("1e-19")
    for k in range(3, order, 2):
        assert abs(sum(x ** k for x in g)) < Decimal("1e-18"), k
    # the next power sum is not zero: the order is not higher by accident
    assert abs(sum(x ** (order + 1) for x in g)) > Decimal("1e-4")
