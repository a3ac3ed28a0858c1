"""Composition and splitting coefficients (oracle).

Follows Sec. II D (symmetric composition of a symmetric method, triple jump
M = 3 and Suzuki's fractal M = 5), Sec. II E (splitting coefficients of a
composed second-order split-operator method, Eqs. (second_order_so),
(triple_jump_fourth_order_so), (suzukis_fractals_fourth_order_so) and the
symmetry relation (symmetric_splitting_coefficients)) and Sec. II F (pruning,
Eq. (merging_splitting_coeff_b_zero), and unique coefficients with index arrays,
Eq. (range_index_unq), Table II).

All arithmetic is carried in ``decimal`` with 60 significant digits and
rounded to float64 only when a value leaves this module.

Readings where the paper is silent:

* the composition exponent for going from order p to order p + 2 is 1/(p+1)
  (the paper prints only p = 2: exponent 1/3 in Eqs. for the fourth-order
  methods); Table II's counts and the order conditions pin it;
* the outer (new) composition is applied to the whole inner sequence, i.e. the
  elementary-step coefficients of order p+2 are gamma_m * c_i with m the outer
  index and i the inner one, in time order;
* a trailing b_N = 0 is dropped after pruning (footnote of Table II:
  N_A = N_B + 1 after the merge);
* "repeated" coefficients are those equal to within a relative 1e-12; the
  values are far apart otherwise.
"""
from __future__ import annotations

from decimal import Decimal, getcontext

getcontext().prec = 60

TRIPLE_JUMP = "triple_jump"
SUZUKI = "suzuki"
OPTIMAL = "optimal"

# The "optimal" compositions of Sec. II D (Table II's last rows) are not
# recursive: their coefficients come from a numerical optimisation in the
# literature the paper cites (Kahan and Li, Math. Comp. 66, 1089 (1997)):
# 9 stages for order 6 and 17 for order 8, symmetric.  Only the first half and
# the middle coefficient are listed (gamma_1 .. gamma_{(M+1)/2}), to 20
# significant digits.  They satisfy the consistency and power-sum order
# conditions to that precision, and the propagation tests measure their
# convergence order.
OPTIMAL_HALF = {
    6: ("0.39216144400731413928", "0.33259913678935943860", "-0.70624617255763935981",
        "0.082213596293550800230", "0.79854399093482996340"),
    8: ("0.13020248308889008088", "0.56116298177510838456", "-0.38947496264484728641",
        "0.15884190655515560090", "-0.39590389413323757734", "0.18453964097831570709",
        "0.25837438768632204729", "0.29501172360931029887", "-0.60550853383003451170"),
}


def gamma_triple_jump(p: int):
    """Triple-jump coefficients lifting a symmetric order-p method to p+2
    (Sec. II D, M = 3): gamma_1 = gamma_3 = x, gamma_2 = 1 - 2x with
    x = 1/(2 - 2^(1/(p+1))).  1 - 2x equals -2^(1/(p+1)) x."""
    r = Decimal(2) ** (Decimal(1) / Decimal(p + 1))
    x = Decimal(1) / (Decimal(2) - r)
    return [x, Decimal(1) - 2 * x, x]


def gamma_suzuki(p: int):
    """Suzuki-fractal coefficients lifting order p to p+2 (Sec. II D, M = 5):
    gamma_{1,2,4,5} = y, gamma_3 = 1 - 4y with y = 1/(4 - 4^(1/(p+1)))."""
    r = Decimal(4) ** (Decimal(1) / Decimal(p + 1))
    y = Decimal(1) / (Decimal(4) - r)
    return [y, y, Decimal(1) - 4 * y, y, y]


def composition(order: int, scheme: str):
    """Elementary-step coefficients gamma (time order) of the recursive
    composition of a second-order method up to ``order`` (Sec. II D):
    U_{p+2}(dt) = U_p(gamma_M dt) ... U_p(gamma_1 dt); for the OPTIMAL scheme
    the tabulated non-recursive coefficients above."""
    if order < 2 or order % 2:
        raise ValueError("order must be even and >= 2")
    if scheme == OPTIMAL:
        if order not in OPTIMAL_HALF:
            raise ValueError("the optimal compositions are available for orders 6 and 8")
        half = [Decimal(x) for x in OPTIMAL_HALF[order]]
        return half[:-1] + [half[-1]] + half[:-1][::-1]
    if scheme not in (TRIPLE_JUMP, SUZUKI):
        raise ValueError(f"unknown scheme {scheme!r}")
    seq = [Decimal(1)]
    p = 2
    while p < order:
        outer = gamma_triple_jump(p) if scheme == TRIPLE_JUMP else gamma_suzuki(p)
        seq = [g * c for g in outer for c in seq]
        p += 2
    return seq


def expand(gammas):
    """Splitting coefficients of the composed second-order method (Sec. II E):
    each elementary step gamma contributes a = (gamma/2, gamma/2) and
    b = (gamma, 0), Eq. (second_order_so) scaled by gamma (Fig. 1 caption)."""
    a, b = [], []
    for g in gammas:
        a += [g / 2, g / 2]
        b += [g, Decimal(0)]
    return a, b


def prune(a, b):
    """Remove zero b_j and merge the neighbouring a's (Sec. II F, Eq.
    (merging_splitting_coeff_b_zero)); a final b_N = 0 is dropped, leaving
    N_A = N_B + 1 (footnote of Table II)."""
    N = len(a)
    at, bt = [], []
    pending = Decimal(0)
    have = False
    for j in range(N):
        pending = a[j] if not have else pending + a[j]
        have = True
        if b[j] != 0:
            at.append(pending)
            bt.append(b[j])
            have = False
    if have:
        at.append(pending)
    return at, bt


def unique_index(values, rel_tol=Decimal("1e-12")):
    """Unique coefficient values and the index array I (0-based here; the
    paper's Eq. (range_index_unq) counts from 1).  Following Sec. II F, only
    the first half of the symmetric sequence is searched and the second half
    is mirrored."""
    n = len(values)
    half = (n + 1) // 2
    uniq, idx = [], [None] * n
    for j in range(half):
        v = values[j]
        for u, w in enumerate(uniq):
            if abs(v - w) <= rel_tol * max(abs(v), abs(w)):
                idx[j] = u
                break
        else:
            uniq.append(v)
            idx[j] = len(uniq) - 1
    for j in range(half, n):
        idx[j] = idx[n - 1 - j]
    return uniq, idx


class Splitting:
    """Pruned splitting coefficients of one scheme/order, with unique-value
    tables; float64 views are exposed for the propagation."""

    def __init__(self, order: int, scheme: str = TRIPLE_JUMP, pruned: bool = True, gammas=None):
        """With `gammas` (elementary-step coefficients of any symmetric
        composition, time order) they replace the recursive TJ / Suzuki ones
        and `order`, `scheme` are only labels."""
        self.order, self.scheme, self.pruned = order, scheme, pruned
        self.gamma = composition(order, scheme) if gammas is None else [Decimal(float(g)) for g in gammas]
        self.a_full, self.b_full = expand(self.gamma)
        if pruned:
            self.a_dec, self.b_dec = prune(self.a_full, self.b_full)
        else:
            self.a_dec, self.b_dec = list(self.a_full), list(self.b_full)
        self.a = [float(x) for x in self.a_dec]
        self.b = [float(x) for x in self.b_dec]
        self.a_unq_dec, self.Ia = unique_index(self.a_dec)
        self.b_unq_dec, self.Ib = unique_index(self.b_dec)

    @property
    def n_actions_before(self):
        """N_A + N_B before the merge, zero-time kinetic actions not counted
        (Table II, third column)."""
        return len(self.a_full) + sum(1 for x in self.b_full if x != 0)

    @property
    def n_actions_after(self):
        """N_A + N_B after the merge (Table II, fourth column)."""
        a, b = prune(self.a_full, self.b_full)
        return len(a) + len(b)

    @property
    def n_substeps(self):
        """Kinetic actions per time step."""
        return sum(1 for x in self.b if x != 0)


def first_order():
    """First-order VT/TV coefficients a_1 = b_1 = 1 (Sec. II E)."""
    return [1.0], [1.0]
