"""Least Herbrand models of Datalog programs over binary predicates, by symbolic evaluation.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.  It knows nothing of matrices: facts are
pairs of constant indices and clauses are applied as relational joins, which is the T_P operator
of Sec. 2 (the immediate consequences of a set of facts).

  parse(text)                  clauses of a program written as
                                   r2(X,Z) :- r1(X,Y), r2(Y,Z).
                               (variables start with an upper-case letter; every predicate is
                               binary; "not p(X,Y)" negates an atom; a clause without a body is not
                               allowed: base facts come in as relations)
  least_model(clauses, edb)    the least model by semi-naive evaluation per stratum: predicates
                               are ordered so that a negated atom's predicate is complete before
                               it is read (stratified negation), and inside a stratum a round
                               only joins clauses that have a body atom whose relation grew in
                               the previous round, against that atom's new facts
  naive_model(clauses, edb)    the same by naive iteration of T_P (every clause against every
                               fact, until nothing changes); small inputs only
Relations are Python sets of (i, j) pairs over constants 0 .. n-1.
"""
from __future__ import annotations

import re
from dataclasses import dataclass

_ATOM = re.compile(r"\s*(not\s+)?([a-z_][A-Za-z0-9_]*)\s*\(\s*([A-Za-z_][A-Za-z0-9_]*)\s*,\s*([A-Za-z_][A-Za-z0-9_]*)\s*\)\s*")


@dataclass(frozen=True)
class Atom:
    pred: str
    a: str
    b: str
    neg: bool = False


@dataclass(frozen=True)
class Clause:
    head: Atom
    body: tuple


def parse(text: str) -> list:
    clauses = []
    for raw in text.replace("\n", " ").split("."):
        if not raw.strip():
            continue
        if ":-" not in raw:
            raise ValueError(f"a clause needs a body: {raw.strip()}")
        head_s, body_s = raw.split(":-", 1)
        m = _ATOM.fullmatch(head_s)
        if not m or m.group(1):
            raise ValueError(f"bad head: {head_s.strip()}")
        head = Atom(m.group(2), m.group(3), m.group(4))
        body = []
        for part in re.split(r",(?![^()]*\))", body_s):
            m = _ATOM.fullmatch(part)
            if not m:
                raise ValueError(f"bad body atom: {part.strip()}")
            body.append(Atom(m.group(2), m.group(3), m.group(4), bool(m.group(1))))
        clauses.append(Clause(head, tuple(body)))
    return clauses


def _is_var(t: str) -> bool:
    return t[0].isupper() or t[0] == "_"


def _index(rel):
    by_first, by_second = {}, {}
    for (i, j) in rel:
        by_first.setdefault(i, []).append(j)
        by_second.setdefault(j, []).append(i)
    return by_first, by_second


def _solutions(body, rels, n, pinned=None):
    """All variable bindings satisfying the body; `pinned` = (index, relation) replaces the
    relation of one positive body atom (semi-naive: a delta)."""
    binds = [dict()]
    # the pinned atom first (it is the smallest), then the other positive atoms, negated last
    # (their variables are bound by then)
    order = sorted(range(len(body)), key=lambda k: (body[k].neg, pinned is None or pinned[0] != k))
    for k in order:
        at = body[k]
        rel = pinned[1] if pinned is not None and pinned[0] == k else rels.get(at.pred, set())
        first, second = _index(rel) if not at.neg else (None, None)
        out = []
        for bd in binds:
            x, y = bd.get(at.a), bd.get(at.b)
            if at.neg:
                if x is None or y is None:
                    raise ValueError(f"unsafe negated atom {at}")
                if (x, y) not in rel:
                    out.append(bd)
                continue
            if x is not None:
                cands = [(x, j) for j in first.get(x, ())]
            elif y is not None:
                cands = [(i, y) for i in second.get(y, ())]
            else:
                cands = rel
            for (i, j) in cands:
                if (y is not None and j != y) or (at.a == at.b and i != j):
                    continue
                nb = dict(bd)
                nb[at.a] = i
                nb[at.b] = j
                out.append(nb)
        binds = out
    return binds


def _head_facts(clause, binds):
    return {(bd[clause.head.a], bd[clause.head.b]) for bd in binds}


def strata(clauses, edb_preds):
    """Predicates in evaluation order: a list of sets (each set a stratum)."""
    idb = {c.head.pred for c in clauses}
    deps = {p: set() for p in idb}  # p -> (q, negated)
    for c in clauses:
        for at in c.body:
            if at.pred in idb:
                deps[c.head.pred].add((at.pred, at.neg))
    # stratum numbers by relaxation: s(p) >= s(q) (positive), > s(q) (negated)
    level = {p: 0 for p in idb}
    for _ in range(len(idb) + 1):
        changed = False
        for p in idb:
            for q, neg in deps[p]:
                need = level[q] + (1 if neg else 0)
                if level[p] < need:
                    level[p] = need
                    changed = True
        if not changed:
            break
    else:
        raise ValueError("negation through recursion: the program is not stratified")
    out = {}
    for p, lv in level.items():
        out.setdefault(lv, set()).add(p)
    return [out[k] for k in sorted(out)]


def least_model(clauses, edb: dict, n: int) -> dict:
    rels = {p: set(r) for p, r in edb.items()}
    for stratum in strata(clauses, set(edb)):
        cls = [c for c in clauses if c.head.pred in stratum]
        for p in stratum:
            rels.setdefault(p, set())
        # first round: every clause on the full relations
        delta = {p: set() for p in stratum}
        for c in cls:
            for f in _head_facts(c, _solutions(c.body, rels, n)):
                if f not in rels[c.head.pred]:
                    delta[c.head.pred].add(f)
        for p in stratum:
            rels[p] |= delta[p]
        while any(delta.values()):
            new = {p: set() for p in stratum}
            for c in cls:
                for k, at in enumerate(c.body):
                    if at.neg or at.pred not in stratum or not delta[at.pred]:
                        continue
                    for f in _head_facts(c, _solutions(c.body, rels, n, (k, delta[at.pred]))):
                        if f not in rels[c.head.pred]:
                            new[c.head.pred].add(f)
            for p in stratum:
                rels[p] |= new[p]
            delta = new
    return {p: rels[p] for p in {c.head.pred for c in clauses}}


def naive_model(clauses, edb: dict, n: int) -> dict:
    rels = {p: set(r) for p, r in edb.items()}
    for stratum in strata(clauses, set(edb)):
        cls = [c for c in clauses if c.head.pred in stratum]
        for p in stratum:
            rels.setdefault(p, set())
        while True:
            nxt = {p: set(rels[p]) for p in stratum}
            for c in cls:
                nxt[c.head.pred] |= _head_facts(c, _solutions(c.body, rels, n))
            if all(nxt[p] == rels[p] for p in stratum):
                break
            rels.update(nxt)
    return {p: rels[p] for p in {c.head.pred for c in clauses}}


def to_pairs(m) -> set:
    """Pairs (i, j) of a dense 0/1 matrix."""
    import numpy as np
    return set(map(tuple, np.argwhere(np.asarray(m) != 0).tolist()))


def to_matrix(pairs, n: int):
    import numpy as np
    m = np.zeros((n, n), dtype=np.uint8)
    for i, j in pairs:
        m[i, j] = 1
    return m
