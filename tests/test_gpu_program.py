"""The program front-end (dl_program_*, the class C_lin of Sec. 5) on the GPU against the symbolic
oracle (oracle/program.py, semi-naive T_P per stratum) and the C oracle.

Every model must equal the oracle's bit for bit.  The cases cover each route a layer can take
(non-recursive, tail recursive left and right, mutually recursive by the stacked closure, the
transposed class, the same-generation form, the series of Lemma 3), stratified negation in chain
bodies (Sec. 8), seeded random C_lin programs, the errors of the checks, and sizes up to 2048."""
import re

import numpy as np
import pytest

import oracle
from oracle import program as pg
from oracle import transposed as tr
from paper_1608_00139_gb300 import dl, inputs

pytestmark = pytest.mark.gpu


def unpack(bits, n):
    return np.unpackbits(np.asarray(bits).view(np.uint8), axis=1, bitorder="little")[:, :n]


def run(ctx, text, rels):
    """Models of every defined predicate from the library, with the program (for its plan)."""
    prog = ctx.program(text)
    for k, v in rels.items():
        if k in prog.base:  # a random program need not read every relation
            prog.set(k, v)
    prog.run()
    n = next(iter(rels.values())).shape[0]
    return {p: unpack(prog.get(p), n) for p in prog.defined}, prog


def expected(text, rels):
    n = next(iter(rels.values())).shape[0]
    text = re.sub(r"%[^\n]*", "", text)  # the oracle's parser takes no comments
    m = pg.least_model(pg.parse(text), {k: pg.to_pairs(v) for k, v in rels.items()}, n)
    return {p: pg.to_matrix(r, n) for p, r in m.items()}


def check(ctx, text, rels, route=None):
    got, prog = run(ctx, text, rels)
    want = expected(text, rels)
    assert set(got) == set(want)
    for p in want:
        assert np.array_equal(got[p], want[p]), (p, text)
    if route is not None:
        assert any(route in ln for ln in prog.plan), prog.plan
    return prog


def er(n, p, seed):
    return inputs.er_digraph(n, p, seed)


TC = "r2(X,Z) :- r1(X,Z).  r2(X,Z) :- r1(X,Y), r2(Y,Z)."
TC_RIGHT = "r(X,Z) :- e(X,Z).  r(X,Z) :- r(X,Y), e(Y,Z)."
SG = "sg(X,Y) :- b(X,Y).  sg(X,Y) :- p(X,Z), sg(Z,W), p(Y,W)."
TRANS = "r2(X,Z) :- r1(X,Z).  r2(X,Z) :- r1(X,Y), r2(Z,Y)."
EVEN_ODD = """
    ev(X,Y) :- e(X,Z), e(Z,Y).   ev(X,Y) :- e(X,Z), od(Z,Y).
    od(X,Y) :- e(X,Y).           od(X,Y) :- e(X,Z), ev(Z,Y).
"""


@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 257])
def test_closure_program_against_the_c_oracle(ctx, n):
    e = er(n, min(0.5, 2.0 / max(n, 1)), 300 + n)
    got, prog = run(ctx, TC, {"r1": e})
    assert np.array_equal(got["r2"], unpack(oracle.tc_model(e), n))
    assert any("tail recursive (Sec. 6.1)" in ln for ln in prog.plan)


def test_right_recursive_closure(ctx):
    e = er(200, 0.01, 11)
    got, prog = run(ctx, TC_RIGHT, {"e": e})
    assert np.array_equal(got["r"], unpack(oracle.tc_model(e), 200))
    assert any("on the transposes" in ln for ln in prog.plan)


def test_same_generation_program_against_the_c_oracle(ctx):
    n = 300
    p = inputs.forest_dag(n, 5)
    b = np.eye(n, dtype=np.uint8)
    got, prog = run(ctx, SG, {"p": p, "b": b})
    assert np.array_equal(got["sg"], unpack(oracle.sg_model(p, None), n))
    assert any("same-generation form" in ln for ln in prog.plan)


@pytest.mark.parametrize("n,p,seed", [(40, 0.05, 1), (129, 0.02, 2), (300, 0.005, 3)])
def test_transposed_program(ctx, n, p, seed):
    r1 = er(n, p, seed)
    got, prog = run(ctx, TRANS, {"r1": r1})
    assert np.array_equal(got["r2"], tr.trans_model(r1))
    assert any("transposed class" in ln for ln in prog.plan)


def test_transposed_on_the_right(ctx):
    text = "r(X,Z) :- a(X,Z).  r(X,Z) :- r(Y,X), c(Y,Z)."
    rels = {"a": er(60, 0.03, 4), "c": er(60, 0.04, 5)}
    check(ctx, text, rels, "transposed class")


def test_mutual_recursion_by_the_stacked_closure(ctx):
    rels = {"e": er(50, 0.04, 6)}
    check(ctx, EVEN_ODD, rels, "stacked system")
    # the hand-derived chain 0 -> 1 -> 2 -> 3
    e = np.zeros((4, 4), np.uint8)
    e[[0, 1, 2], [1, 2, 3]] = 1
    got, _ = run(ctx, EVEN_ODD, {"e": e})
    assert pg.to_pairs(got["od"]) == {(0, 1), (1, 2), (2, 3), (0, 3)}
    assert pg.to_pairs(got["ev"]) == {(0, 2), (1, 3)}


def test_two_sided_not_same_generation_takes_the_series(ctx):
    text = "s(X,Y) :- b(X,Y).  s(X,Y) :- p(X,Z), s(Z,W), q(W,Y)."
    rels = {"b": er(70, 0.02, 7), "p": er(70, 0.03, 8), "q": er(70, 0.03, 9)}
    check(ctx, text, rels, "series of Lemma 3")


def test_mutually_recursive_two_sided_layer(ctx):
    text = """
        s(X,Y) :- b(X,Y).      s(X,Y) :- p(X,Z), t(Z,W), p(Y,W).
        t(X,Y) :- s(X,Z), q(Z,Y).
    """
    rels = {"b": er(48, 0.03, 10), "p": er(48, 0.04, 11), "q": er(48, 0.05, 12)}
    check(ctx, text, rels, "series of Lemma 3")


def test_negation_in_chains(ctx):
    # negated base and lower-layer atoms as interior links of chain bodies (1 - R, Sec. 8); every
    # negated atom's variables are bound by its neighbours, so the rules are safe
    text = """
        r(X,Y) :- e(X,Y).   r(X,Y) :- e(X,Z), r(Z,Y).
        nr(X,Y) :- e(X,Z), not r(Z,W), e(W,Y).
        k(X,Y) :- nr(X,Z), not f(Z,W), e(Y,W).
        k(X,Y) :- e(X,Z), k(Z,Y).
    """
    rels = {"e": er(40, 0.05, 13), "f": er(40, 0.3, 14)}
    prog = check(ctx, text, rels)
    order = [set(l) for l in prog.layers]
    assert order.index({"r"}) < order.index({"nr"}) < order.index({"k"})


def test_negation_over_the_domain(ctx):
    # a negated atom that ends a chain reads 1 - R over all n x n pairs (the closed forms)
    n = 70
    e, f = er(n, 0.05, 21), er(n, 0.4, 22)
    got, _ = run(ctx, "m(X,Y) :- not f(X,Y).  q(X,Y) :- e(X,Z), not f(Z,Y).", {"e": e, "f": f})
    assert np.array_equal(got["m"], 1 - f)
    want = (e.astype(np.int64) @ (1 - f).astype(np.int64) > 0).astype(np.uint8)
    assert np.array_equal(got["q"], want)


def test_multi_layer_program(ctx):
    text = """
        % reachability, then pairs reaching a common node, then their closure
        reach(X,Y) :- e(X,Y).      reach(X,Y) :- e(X,Z), reach(Z,Y).
        meet(X,Y) :- reach(X,Z), reach(Y,Z).
        link(X,Y) :- meet(X,Y).    link(X,Y) :- meet(X,Z), link(Z,Y).
        cs(X,Y) :- reach(X,Y).     cs(X,Y) :- f(X,Z), cs(Z,W), f(Y,W).
    """
    rels = {"e": er(90, 0.015, 15), "f": er(90, 0.02, 16)}
    prog = check(ctx, text, rels)
    assert len(prog.layers) == 4
    assert prog.base == ["e", "f"] and prog.defined == ["cs", "link", "meet", "reach"]


def random_clin_program(rng, npred=4, nedb=2):
    """A random C_lin program: predicates p0.. grouped into SCC candidates in order; a body is a
    chain X0 - X1 - ... - Xk of EDB atoms, atoms of lower groups and at most one atom of its own
    group, each in either argument order; negation on EDB and lower-group atoms."""
    idb = [f"p{i}" for i in range(npred)]
    edb = [f"e{i}" for i in range(nedb)]
    cuts = sorted(rng.choice(np.arange(1, npred), size=int(rng.integers(0, npred)), replace=False).tolist())
    groups, start = [], 0
    for c in cuts + [npred]:
        groups.append(idb[start:c])
        start = c
    lines = []
    for gi, grp in enumerate(groups):
        lower = [p for g in groups[:gi] for p in g]
        for h in grp:
            for ci in range(int(rng.integers(1, 4))):
                k = int(rng.integers(1, 5))
                own = int(rng.integers(0, k)) if (ci > 0 and rng.random() < 0.8) else -1
                atoms = []
                for t in range(k):
                    neg = False
                    if t == own:
                        pred = str(rng.choice(grp))
                    else:
                        pred = str(rng.choice(edb + lower))
                        # safe negation: an interior link whose neighbours are positive
                        neg = 0 < t < k - 1 and t + 1 != own and t - 1 != own and not atoms[-1].startswith("not") \
                            and rng.random() < 0.4
                    a, b = f"X{t}", f"X{t + 1}"
                    if rng.random() < 0.3:
                        a, b = b, a
                    atoms.append(("not " if neg else "") + f"{pred}({a},{b})")
                head = f"{h}(X0,X{k})" if rng.random() < 0.8 else f"{h}(X{k},X0)"
                lines.append(f"{head} :- {', '.join(atoms)}.")
    return "\n".join(lines), edb


def test_random_clin_programs(ctx):
    rng = np.random.default_rng(17)
    routes = set()
    for trial in range(25):
        text, edb = random_clin_program(rng)
        n = int(rng.integers(3, 40))
        rels = {e: (rng.random((n, n)) < rng.uniform(0.02, 0.15)).astype(np.uint8) for e in edb}
        prog = check(ctx, text, rels)
        for ln in prog.plan:
            routes.add(ln.split("} ", 1)[1].split(" (")[0].split(":")[0])
    # the seeded programs reach the non-recursive, tail recursive and series routes at least
    assert {"non-recursive", "tail recursive", "the series of Lemma 3"} <= routes, routes


@pytest.mark.parametrize("text,needle", [
    ("p(X,Y) :- e(X,Y), f(X,Y).", "branches"),
    ("p(X,Y) :- e(X,Z).", "does not end"),
    ("p(X,X) :- e(X,Y).", "repeats a variable"),
    ("p(X,Y) :- e(X,Y).  p(X,Y) :- p(X,Z), p(Z,Y).", "not linear"),
    ("p(X,Y) :- e(X,Y).  p(X,Y) :- e(X,Z), not p(Z,Y).", "not stratified"),
    ("p(X,Y) :- e(X,a).", "constants"),
    ("p(X,Y,Z) :- e(X,Y).", "binary"),
    ("p(X,Y) :- e(X,Y)", "'.'"),
    ("", "no clauses"),
])
def test_rejected_programs(ctx, text, needle):
    with pytest.raises(dl.DLError) as err:
        ctx.program(text)
    assert err.value.status == dl.DL_EINVAL
    assert needle in err.value.message, err.value.message


def test_run_errors(ctx):
    prog = ctx.program(TC)
    with pytest.raises(dl.DLError):
        prog.run()  # r1 unset
    with pytest.raises(dl.DLError):
        prog.set("r2", np.zeros((4, 4), np.uint8))  # not a base relation
    bad = np.zeros((8, 8), np.uint8)
    bad[2, 3] = 7
    prog.set("r1", bad)
    with pytest.raises(dl.DLError) as err:
        prog.run()
    assert err.value.status == dl.DL_EINVAL
    with pytest.raises(dl.DLError):
        prog.get("r2")  # no successful run yet
    two = ctx.program("p(X,Y) :- e(X,Z), f(Z,Y).")
    two.set("e", np.zeros((5, 5), np.uint8))
    with pytest.raises(dl.DLError):
        two.set("f", np.zeros((6, 6), np.uint8))  # n differs


def test_empty_relations(ctx):
    prog = ctx.program(TC)
    prog.set("r1", np.zeros((0, 0), np.uint8))
    prog.run()
    assert prog.get("r2").shape == (0, 0)


def test_device_inputs_and_outputs(ctx):
    torch = pytest.importorskip("torch")
    n = 500
    e = er(n, 0.004, 18)
    prog = ctx.program(TC_RIGHT)
    prog.set("e", torch.from_numpy(e).cuda())
    prog.run()
    bits = prog.get("r", device=True)
    assert bits.is_cuda
    assert np.array_equal(unpack(bits.cpu().numpy(), n), unpack(oracle.tc_model(e), n))


def test_n2048_layered_program(ctx):
    """Closure, a join of two closures, and same generation over it, at N = 2048."""
    n = 2048
    e = er(n, 1.0 / n, 19)
    p = inputs.forest_dag(n, 20)
    text = """
        r(X,Y) :- e(X,Y).   r(X,Y) :- e(X,Z), r(Z,Y).
        sg(X,Y) :- r(X,Y).  sg(X,Y) :- p(X,Z), sg(Z,W), p(Y,W).
    """
    got, prog = run(ctx, text, {"e": e, "p": p})
    r = unpack(oracle.tc_model(e), n)
    assert np.array_equal(got["r"], r)
    assert np.array_equal(got["sg"], unpack(oracle.sg_model(p, r), n))


def test_context_closed_before_its_programs():
    """Closing a context closes its live programs first (a program's destruction uses its
    context), so the programs' later close or collection does not touch a freed context."""
    e = inputs.er_digraph(300, 0.01, 11)
    c = dl.Context(0)
    progs = [c.program("r(X,Y) :- e(X,Y).  r(X,Y) :- e(X,Z), r(Z,Y).") for _ in range(3)]
    progs[0].set("e", e)
    progs[0].run()
    assert np.array_equal(progs[0].get("r"), oracle.tc_model(e))
    progs[2].close()
    c.close()
    assert all(p._h is None for p in progs)
    for p in progs:
        p.close()  # no-op now
    del progs
