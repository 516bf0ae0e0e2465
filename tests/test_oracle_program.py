"""Pins of the symbolic program oracle (oracle/program.py): semi-naive evaluation of Datalog
programs over binary predicates, the T_P fixpoint of Sec. 2.

It must agree with the C oracle on the closure program (Sec. 3) and the same-generation program
(Sec. 7.2), with the transposed-class oracle on prog:2 (Sec. 6.2), with naive iteration of T_P on
random programs (mutual recursion, transposed and two-sided atoms, stratified negation), and with
hand-derived cases."""
import numpy as np
import pytest

import oracle
from oracle import program as pg
from oracle import transposed as tr
from paper_1608_00139_gb300 import inputs


def unpack(bits, n):
    return np.unpackbits(bits.view(np.uint8), axis=1, bitorder="little")[:, :n]


TC = "r2(X,Z) :- r1(X,Z).  r2(X,Z) :- r1(X,Y), r2(Y,Z)."
SG = "sg(X,Y) :- b(X,Y).  sg(X,Y) :- p(X,Z), sg(Z,W), p(Y,W)."
TRANS = "r2(X,Z) :- r1(X,Z).  r2(X,Z) :- r1(X,Y), r2(Z,Y)."


@pytest.mark.parametrize("n,p,seed", [(20, 0.1, 1), (50, 0.04, 2), (80, 0.02, 3)])
def test_closure_program_matches_the_c_oracle(n, p, seed):
    e = inputs.er_digraph(n, p, seed)
    got = pg.least_model(pg.parse(TC), {"r1": pg.to_pairs(e)}, n)["r2"]
    assert pg.to_matrix(got, n).tolist() == unpack(oracle.tc_model(e), n).tolist()


@pytest.mark.parametrize("n,seed", [(30, 1), (60, 2)])
def test_same_generation_program_matches_the_c_oracle(n, seed):
    p = inputs.forest_dag(n, seed)
    rng = np.random.default_rng(seed)
    b = (rng.random((n, n)) < 0.03).astype(np.uint8)
    got = pg.least_model(pg.parse(SG), {"p": pg.to_pairs(p), "b": pg.to_pairs(b)}, n)["sg"]
    assert pg.to_matrix(got, n).tolist() == unpack(oracle.sg_model(p, b), n).tolist()


@pytest.mark.parametrize("n,p,seed", [(25, 0.08, 4), (60, 0.03, 5)])
def test_transposed_program_matches_the_transposed_oracle(n, p, seed):
    r1 = inputs.er_digraph(n, p, seed)
    got = pg.least_model(pg.parse(TRANS), {"r1": pg.to_pairs(r1)}, n)["r2"]
    assert np.array_equal(pg.to_matrix(got, n), tr.trans_model(r1))


def test_hand_derived_negation_and_mutual_recursion():
    # even/odd path lengths by mutual recursion, then pairs at an even but no odd distance
    prog = pg.parse("""
        ev(X,Y) :- e(X,Z), e(Z,Y).   ev(X,Y) :- e(X,Z), od(Z,Y).
        od(X,Y) :- e(X,Y).           od(X,Y) :- e(X,Z), ev(Z,Y).
        only(X,Y) :- ev(X,Y), not od(X,Y).
    """)
    # chain 0 -> 1 -> 2 -> 3
    edb = {"e": {(0, 1), (1, 2), (2, 3)}}
    m = pg.least_model(prog, edb, 4)
    assert m["od"] == {(0, 1), (1, 2), (2, 3), (0, 3)}
    assert m["ev"] == {(0, 2), (1, 3)}
    assert m["only"] == {(0, 2), (1, 3)}
    # with the edge 3 -> 0 the cycle has length 4: every pair is at an even or odd distance
    edb = {"e": {(0, 1), (1, 2), (2, 3), (3, 0)}}
    m = pg.least_model(prog, edb, 4)
    assert m["only"] == {(i, j) for i in range(4) for j in range(4) if (j - i) % 2 == 0}


def test_negation_through_recursion_is_rejected():
    with pytest.raises(ValueError):
        pg.strata(pg.parse("p(X,Y) :- e(X,Y), not p(Y,X)."), {"e"})


def random_program(rng, npred=3, nedb=2):
    """A random program: heads among p0..; bodies of one to three atoms chaining X0 .. Xk, each
    atom forward or reversed, over EDB e0.. and IDB predicates; negation only on EDB atoms."""
    idb = [f"p{i}" for i in range(npred)]
    edb = [f"e{i}" for i in range(nedb)]
    lines = []
    for h in idb:
        for _ in range(int(rng.integers(1, 4))):
            k = int(rng.integers(1, 4))
            atoms = []
            for t in range(k):
                pred = rng.choice(idb + edb) if t > 0 or rng.random() < 0.5 else rng.choice(edb)
                a, b = f"X{t}", f"X{t + 1}"
                if rng.random() < 0.3:
                    a, b = b, a
                atoms.append(f"{pred}({a},{b})")
            if rng.random() < 0.2:
                atoms.append(f"not {rng.choice(edb)}(X0,X{k})")
            head = f"{h}(X0,X{k})" if rng.random() < 0.7 else f"{h}(X{k},X0)"
            lines.append(f"{head} :- {', '.join(atoms)}.")
    return " ".join(lines), edb


def test_random_programs_agree_with_naive_iteration():
    rng = np.random.default_rng(7)
    for _ in range(60):
        text, edb = random_program(rng)
        n = int(rng.integers(2, 9))
        facts = {e: {(int(i), int(j)) for i in range(n) for j in range(n) if rng.random() < 0.25} for e in edb}
        cl = pg.parse(text)
        assert pg.least_model(cl, facts, n) == pg.naive_model(cl, facts, n), text
