"""Closed-form and combinatorial candidate counts used to pin the oracle.

TEST INFRASTRUCTURE ONLY (imported by ``tests/`` and the golden-value script).

Two independent references for how many slots and how many unit-valid
candidates each rung has, computed without generating any expression:

* ``closed_form_sizes`` -- no pruning at all.  With m = |new_{r-1}| and
  o = |Phi_{r-2}|, rung r has U*m unary slots and S*(m(m-1)/2 + m*o) binary
  slots (every unordered pair with at least one operand from the newest rung,
  once per binary slot).  This is the counting statement of the iterative
  generation in "Software Description".
* ``unit_class_counts`` -- pruning by dimensional consistency only
  ("Physics-Informed Constraints").  Features are grouped by their exact unit
  vector (``fractions.Fraction`` exponents); equal-unit pairs are counted per
  class, so no pair is ever visited.
"""
from __future__ import annotations

from collections import Counter
from fractions import Fraction

UNARY = range(0, 6)
BINARY = range(6, 12)
SQUARE, CUBE, INV, SQRT, EXP, LOG, ADD, SUB, MUL, DIV, RDIV, ABSDIFF = range(12)


def closed_form_sizes(n0: int, n_unary: int, n_binary: int, max_rung: int):
    """|Phi_r| for r = 0..max_rung with every slot valid."""
    sizes = [n0]
    o, m = 0, n0
    for _ in range(max_rung):
        new = n_unary * m + n_binary * (m * (m - 1) // 2 + m * o)
        sizes.append(sizes[-1] + new)
        o, m = o + m, new
    return sizes


def rung_slot_counts(n0: int, n_unary: int, n_binary: int, max_rung: int):
    """Slots of each rung r = 1..max_rung when nothing is pruned."""
    s = closed_form_sizes(n0, n_unary, n_binary, max_rung)
    return [s[r] - s[r - 1] for r in range(1, max_rung + 1)]


def _unary_unit(op, u, explog_dimensionless):
    if op == SQUARE:
        return tuple(2 * x for x in u)
    if op == CUBE:
        return tuple(3 * x for x in u)
    if op == INV:
        return tuple(-x for x in u)
    if op == SQRT:
        return tuple(x / 2 for x in u)
    if op in (EXP, LOG):
        if explog_dimensionless and any(x != 0 for x in u):
            return None
        return tuple(Fraction(0) for _ in u)
    raise ValueError(op)


def _binary_unit(op, ua, ub, check_addsub):
    if op in (ADD, SUB, ABSDIFF):
        if check_addsub and ua != ub:
            return None
        return ua
    if op == MUL:
        return tuple(x + y for x, y in zip(ua, ub))
    if op == DIV:
        return tuple(x - y for x, y in zip(ua, ub))
    if op == RDIV:
        return tuple(y - x for x, y in zip(ua, ub))
    raise ValueError(op)


def unit_class_counts(primary_units, ops, max_rung, unit_check_addsub=True, explog_dimensionless=True):
    """Per rung r = 1..max_rung: (slots, unit-valid count), pruning by units only.

    Features are handled as classes (exact unit vector -> multiplicity), so
    pairs are counted from class sizes and never visited one by one.  The two
    division slots must be enabled together (or not at all): then every pair
    yields both u_a - u_b and u_b - u_a whichever operand has the higher id.
    """
    unary = [o for o in ops if o in UNARY]
    binary = [o for o in ops if o in BINARY]
    if (DIV in binary) != (RDIV in binary):
        raise ValueError("a/b and b/a must be enabled together for class counting")
    if not unit_check_addsub and max_rung > 1:
        raise ValueError("unchecked + - |a-b| keep the higher id's unit: not a class property")
    old = Counter()  # Phi_{r-2}
    new = Counter(tuple(Fraction(int(x)) for x in u) for u in primary_units)
    out = []
    for r in range(1, max_rung + 1):
        m = sum(new.values())
        o = sum(old.values())
        slots = len(unary) * m + len(binary) * (m * (m - 1) // 2 + m * o)
        # unordered class pairs with their number of feature pairs
        pairs = Counter()
        nk = sorted(new)
        for x, ui in enumerate(nk):
            pairs[(ui, ui)] += new[ui] * (new[ui] - 1) // 2
            for uj in nk[x + 1:]:
                pairs[(ui, uj)] += new[ui] * new[uj]
            for uj, cj in old.items():
                pairs[(ui, uj)] += new[ui] * cj
        nxt = Counter()
        for u, c in new.items():
            for op in unary:
                w = _unary_unit(op, u, explog_dimensionless)
                if w is not None:
                    nxt[w] += c
        for (ui, uj), npairs in pairs.items():
            if npairs == 0:
                continue
            for op in binary:
                if op == RDIV:
                    continue  # counted with DIV below
                if op == DIV:
                    nxt[tuple(x - y for x, y in zip(ui, uj))] += npairs
                    nxt[tuple(y - x for x, y in zip(ui, uj))] += npairs
                    continue
                w = _binary_unit(op, ui, uj, unit_check_addsub)
                if w is not None:
                    nxt[w] += npairs
        out.append((slots, sum(nxt.values())))
        old = old + new
        new = nxt
    return out
