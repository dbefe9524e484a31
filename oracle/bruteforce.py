"""Brute-force enumeration of a tiny feature space, in pure Python.

TEST INFRASTRUCTURE ONLY.  It pins the oracle's flat-index decoding, ordering
and unit rules: expressions are built as explicit trees, rung by rung, with
exact ``fractions.Fraction`` unit exponents, and printed in the same canonical
form as the oracle's expression strings.  Nothing here does index arithmetic:
the position of an expression in the returned list is its global id.

Only unit pruning and the user rules on variable combinations and functional
forms are modelled, so inputs must be chosen such that no domain, magnitude or
realised test can fail (positive data, a huge magnitude limit, degeneracy test
off).  The rules are checked on the whole tree of each expression (the list of
its leaves and, per operator node, the leaves below it), not incrementally.
Follows the iterative generation of "Software Description", the
dimensional-consistency rule of "Physics-Informed Constraints" and the user
rules of "Design Philosophy and Constraints".
"""
from __future__ import annotations

from fractions import Fraction

SQUARE, CUBE, INV, SQRT, EXP, LOG, ADD, SUB, MUL, DIV, RDIV, ABSDIFF = range(12)
_UNARY_FMT = {SQUARE: "sq({})", CUBE: "cb({})", INV: "inv({})", SQRT: "sqrt({})", EXP: "exp({})", LOG: "log({})"}


class Expr:
    """An expression tree: ``kids`` are the operand trees (empty for a
    primary, whose index is ``leaf``)."""
    __slots__ = ("text", "unit", "rung", "op", "kids", "leaf")

    def __init__(self, text, unit, rung, op=None, kids=(), leaf=None):
        self.text, self.unit, self.rung = text, unit, rung
        self.op, self.kids, self.leaf = op, tuple(kids), leaf

    def leaves(self):
        """Primary indices of the leaves, with multiplicity."""
        if not self.kids:
            return [self.leaf]
        return [p for k in self.kids for p in k.leaves()]

    def nodes(self):
        """Every operator node of the tree."""
        if not self.kids:
            return []
        return [self] + [n for k in self.kids for n in k.nodes()]


def breaks_rules(e, pair_deny, op_deny):
    """Whole-tree check of the user rules.  pair_deny: set of frozensets
    {p, q} (a one-element set {p}: p may occur at most once); op_deny: dict
    op -> set of primaries that may not occur below that op."""
    lv = e.leaves()
    for p in set(lv):
        if frozenset((p,)) in pair_deny and lv.count(p) >= 2:
            return True
        for q in set(lv):
            if p != q and frozenset((p, q)) in pair_deny:
                return True
    for n in e.nodes():
        if set(n.leaves()) & set(op_deny.get(n.op, ())):
            return True
    return False


def _unary(op, e, explog_dimensionless):
    u = e.unit
    if op == SQUARE:
        w = tuple(2 * x for x in u)
    elif op == CUBE:
        w = tuple(3 * x for x in u)
    elif op == INV:
        w = tuple(-x for x in u)
    elif op == SQRT:
        w = tuple(x / 2 for x in u)
    else:
        if explog_dimensionless and any(x != 0 for x in u):
            return None
        w = tuple(Fraction(0) for _ in u)
    return Expr(_UNARY_FMT[op].format(e.text), w, e.rung + 1, op, (e,))


def _binary(op, a, b, check_addsub, rung):
    A, B = a.text, b.text
    if op in (ADD, SUB, ABSDIFF):
        if check_addsub and a.unit != b.unit:
            return None
        w = a.unit
        text = {ADD: f"({A}+{B})", SUB: f"({A}-{B})", ABSDIFF: f"|{A}-{B}|"}[op]
    elif op == MUL:
        w, text = tuple(x + y for x, y in zip(a.unit, b.unit)), f"({A}*{B})"
    elif op == DIV:
        w, text = tuple(x - y for x, y in zip(a.unit, b.unit)), f"({A}/{B})"
    else:
        w, text = tuple(y - x for x, y in zip(a.unit, b.unit)), f"({B}/{A})"
    return Expr(text, w, rung, op, (a, b))


RULE = "rule"


def enumerate_bruteforce(primary_units, ops, max_rung, unit_check_addsub=True, explog_dimensionless=True,
                         pair_deny=None, op_deny=None):
    """Returns (stored, last): ``stored`` lists the expressions of rungs
    < max_rung in id order; ``last`` lists one entry per rung-max_rung slot in
    flat order, the Expr, None when the slot is unit-invalid, or ``RULE`` when
    it is unit-valid but breaks a user rule."""
    unary = sorted(o for o in ops if o <= LOG)
    binary = sorted(o for o in ops if o >= ADD)
    pair_deny = pair_deny or set()
    op_deny = op_deny or {}

    def assessed(e):
        if e is not None and breaks_rules(e, pair_deny, op_deny):
            return RULE
        return e

    stored = [Expr(f"x{p}", tuple(Fraction(int(x)) for x in u), 0, leaf=p) for p, u in enumerate(primary_units)]
    begin = 0  # first id of the newest rung
    for r in range(1, max_rung + 1):
        newest = stored[begin:]
        slots = []
        for f in newest:
            for op in unary:
                slots.append(assessed(_unary(op, f, explog_dimensionless)))
        for i_rel, a in enumerate(newest):
            i = begin + i_rel
            for j in range(i):
                for op in binary:
                    slots.append(assessed(_binary(op, a, stored[j], unit_check_addsub, r)))
        if r == max_rung:
            return stored, slots
        begin = len(stored)
        stored = stored + [e for e in slots if isinstance(e, Expr)]
    raise AssertionError("unreachable")
