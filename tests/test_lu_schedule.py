"""The mixed path's factorisation schedule, as a model checked on the CPU.

csrc/dl_mixed.cu factors A = L U in steps of 128-row blocks: within units of G = 2 or 4 steps the
updates are left-looking (before step j's pivot, block row and column j receive the updates of
the steps since the unit's start, or of the whole previous unit when j starts one), and each
unit's last step issues one bulk update of the rows and columns from the second block after it.
Six streams carry it: the chain P (the diagonal block's update, diag, L21), Rs (the rest of the
row and column update), Q (the row-panel transposes T), U (bulk updates), V (the inverse's
groups), ordered by events.

This file restates that schedule in Python, block by block, in the order the host issues it, and
checks two properties the GPU parity tests can only observe indirectly:
  * coverage: every trailing block (i, c) with i, c > k receives step k's update exactly once,
    and nothing else does (the block elimination of Prop. 1's LU);
  * ordering: every two launches that touch a common block, one of them writing it, are ordered
    by stream order and event waits the way the sequential algorithm orders them.
A model cannot follow later edits of the C++ by itself; it pins the schedule's design."""
import pytest

K_SOLVE_GROUP = 8  # blocks per group of the inverse W (kSolveGroup)


def shape(nb, G, grouped_req):
    grouped = max(0, min(grouped_req, nb - 6)) // G * G
    unit_of = lambda k: k // G if k < grouped else grouped // G + (k - grouped)
    pos_of = lambda k: k % G if k < grouped else 0
    size_of = lambda k: G if k < grouped else 1
    start_of = lambda k: k - pos_of(k)
    return unit_of, pos_of, size_of, start_of


def cells(rows, cols):
    return {(r, c) for r in rows for c in cols}


def tcells(par, pos, rows):
    return {("T", par, pos, r) for r in rows}


def coverage(nb, G, grouped_req):
    """Count, per (step k, block i, block c), the updates the schedule applies."""
    unit_of, pos_of, size_of, start_of = shape(nb, G, grouped_req)
    cnt = {}

    def add(steps, rows, cols):
        for k in steps:
            for r in rows:
                for c in cols:
                    cnt[(k, r, c)] = cnt.get((k, r, c), 0) + 1

    for j in range(1, nb):
        q, k0 = pos_of(j), start_of(j)
        s = k0 if q >= 1 else start_of(j - 1)
        add(range(s, j), [j], [j])                       # the diagonal block (on the chain)
        add(range(s, j), range(j + 1, nb), [j])          # column j below it
        add(range(s, j), [j], range(j + 1, nb))          # row j right of it
    for k in range(nb):
        if pos_of(k) == size_of(k) - 1 and nb - k - 2 > 0:  # the unit's bulk update
            add(range(start_of(k), k + 1), range(k + 2, nb), range(k + 2, nb))
    return cnt


def schedule(nb, G, grouped_req, drop=None):
    """The launches (name, reads, writes) and their happens-before ancestors, issued as the host
    issues them.  `drop` names one wait to leave out (to check that the check can fail)."""
    unit_of, pos_of, size_of, start_of = shape(nb, G, grouped_req)
    has_bulk = [pos_of(j) == size_of(j) - 1 and nb - j - 2 > 0 for j in range(nb)]
    ops, deps, pos, pend, events = [], [], {}, {}, {}

    def launch(name, stream, reads, writes):
        i = len(ops)
        ops.append((name, set(reads) | set(writes), set(writes)))
        d = set(pend.pop(stream, set()))
        if stream in pos:
            d.add(pos[stream])
        deps.append(d)
        pos[stream] = i

    def record(ev, stream):
        events[ev] = ({pos[stream]} if stream in pos else set()) | pend.get(stream, set())

    def wait(stream, ev, tag=None):
        if tag is not None and tag == drop:
            return
        pend.setdefault(stream, set()).update(events.get(ev, set()))

    bulks = []
    for j in range(nb):
        rem = nb - j - 1
        if j > 0:
            wait("P", "evQ")
            jp = j - 1
            if has_bulk[jp]:
                par = unit_of(jp) & 1
                for b in bulks:
                    if b[1] == par:
                        wait("P", "evB%d" % par)
                record("evT%d" % par, "P")
                wait("U", "evT%d" % par)
                k0, rows = start_of(jp), range(jp + 2, nb)
                reads = cells(rows, range(k0, jp + 1)).union(
                    *[tcells(par, p, rows) for p in range(jp - k0 + 1)])
                launch("bulk%d" % jp, "U", reads, cells(rows, rows))
                record("evB%d" % par, "U")
                bulks.append((jp, par))
            while bulks and bulks[0][0] + 2 <= j:
                wait("P", "evB%d" % bulks[0][1], tag="bulk")
                bulks.pop(0)
            record("evL", "P")
            q, k0 = pos_of(j), start_of(j)
            s = k0 if q >= 1 else start_of(j - 1)
            par = unit_of(s) & 1
            Ts = lambda rows: set().union(*[tcells(par, p, rows) for p in range(j - s)])
            launch("udiag%d" % j, "P", cells([j], range(s, j)) | Ts([j]), {(j, j)})
            if rem > 0:
                wait("Rs", "evL", tag="rest")
                rows = range(j + 1, nb)
                launch("urest%d" % j, "Rs", cells(range(j, nb), range(s, j)) | Ts(range(j, nb)),
                       cells(rows, [j]) | cells([j], rows))
                record("evR", "Rs")
        launch("diag%d" % j, "P", {(j, j)}, {("S", j)})
        if rem <= 0:
            break
        if j > 0:
            wait("P", "evR", tag="l21")
        rows = range(j + 1, nb)
        launch("l21_%d" % j, "P", {("S", j)}, cells(rows, [j]))
        if (j + 1) % K_SOLVE_GROUP == 0:
            g = (j + 1) // K_SOLVE_GROUP - 1
            record("gev%d" % g, "P")
            wait("V", "gev%d" % g)
            gs, ge = g * K_SOLVE_GROUP, min(nb, (g + 1) * K_SOLVE_GROUP)
            reads = cells(range(gs, nb), range(gs, ge)) | cells(range(gs, ge), range(gs, nb)) | {
                ("S", k) for k in range(gs, ge)}
            launch("inverse%d" % g, "V", reads, {("W", g)})
        if j > 0:
            wait("Q", "evR", tag="transpose")
        launch("T%d" % j, "Q", cells([j], range(j + 1, nb)), tcells(unit_of(j) & 1, pos_of(j), range(j + 1, nb)))
        record("evQ", "Q")
    return ops, deps


def unordered_conflicts(ops, deps):
    anc = []
    for d in deps:
        a = set(d)
        for x in d:
            a |= anc[x]
        anc.append(a)
    bad = []
    for b in range(len(ops)):
        for a in range(b):
            _, ta, wa = ops[a]
            _, tb, wb = ops[b]
            if (wa & tb or wb & ta) and a not in anc[b]:
                bad.append((ops[a][0], ops[b][0]))
    return bad


SHAPES = [(nb, G, grouped) for nb in (1, 2, 3, 5, 7, 9, 12, 17, 20) for G in (2, 4) for grouped in (0, 8, 64)]


@pytest.mark.parametrize("nb,G,grouped", SHAPES)
def test_every_step_updates_every_trailing_block_once(nb, G, grouped):
    cnt = coverage(nb, G, grouped)
    for k in range(nb):
        for i in range(nb):
            for c in range(nb):
                assert cnt.get((k, i, c), 0) == (1 if i > k and c > k else 0), (k, i, c)


@pytest.mark.parametrize("nb,G,grouped", SHAPES)
def test_conflicting_launches_are_ordered(nb, G, grouped):
    ops, deps = schedule(nb, G, grouped)
    assert unordered_conflicts(ops, deps) == []


@pytest.mark.parametrize("drop", ["bulk", "rest", "l21", "transpose"])
def test_a_missing_wait_is_caught(drop):
    ops, deps = schedule(17, 4, 64, drop=drop)
    assert unordered_conflicts(ops, deps)
