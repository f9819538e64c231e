"""Pins for the two options of the oracle's SSO run: the interval order Eq.
2.1 prints (keep, pBest, gBest, fresh with Cw <= Cp <= Cg) and the
asynchronous flow of Alg. 1 (particle by particle, gBest replaced as soon as a
particle beats it, "<" for both replacements).

Special cases that reduce to closed forms, per-variable branch checks against
the separately pinned Philox rho words and fresh values, binomial branch
frequencies, invariants of Alg. 1, and the special case where the two flows
must agree (no gBest branch: the particles are independent)."""
import numpy as np
import pytest

import oracle
import workload


def _p(fn="sphere", N=16, D=6, lattice="f64", seed=1, sid=0, **kw):
    return workload.problem(fn, N, D, seed=seed, lattice=lattice, stream=sid, **kw)


# ---- interval order ------------------------------------------------------------------
def test_paper_order_all_keep():
    """Cw = 1 in the printed order: the first interval covers every draw, so
    every particle keeps its initial position for ever."""
    p = _p(Cg=1.0, Cp=1.0, Cw=1.0, order="paper")
    r0, r = oracle.run_problem(p, 0), oracle.run_problem(p, 7)
    assert np.array_equal(r["X"], r0["X"]) and np.array_equal(r["P"], r0["P"])
    assert np.all(r["log_acc"][1:] == 16)          # f(x) = f(pBest): "<=" accepts
    assert r["branch"][2] == 16 * 6 * 7


def test_paper_order_all_gbest():
    """Cw = Cp = 0, Cg = 1: every draw lands in the third interval, gBest."""
    p = _p(Cg=1.0, Cp=0.0, Cw=0.0, order="paper")
    r0, r1 = oracle.run_problem(p, 0), oracle.run_problem(p, 1)
    G0 = r0["P"][r0["log_b"][0]]
    assert np.array_equal(r1["X"], np.tile(G0, (16, 1)))
    assert r1["branch"][0] == 16 * 6


def test_paper_order_all_pbest():
    """Cw = 0, Cp = 1: every draw lands in the second interval, pBest."""
    p = _p(Cg=1.0, Cp=1.0, Cw=0.0, order="paper")
    r0, r = oracle.run_problem(p, 0), oracle.run_problem(p, 5)
    assert np.array_equal(r["X"], r0["X"])
    assert r["branch"][1] == 16 * 6 * 5


@pytest.mark.parametrize("lattice", ["f64", "f32"])
def test_paper_order_per_variable(lattice):
    """Generation g of the printed order, variable by variable: r < T(Cw) keeps
    x, r < T(Cp) takes pBest, r < T(Cg) takes gBest, else the fresh value --
    each read from generation g-1 (the synchronous flow)."""
    N, D, g = 12, 9, 4
    Cw, Cp, Cg = 0.3, 0.6, 0.8
    p = _p(N=N, D=D, lattice=lattice, Cg=Cg, Cp=Cp, Cw=Cw, order="paper")
    prev, cur = oracle.run_problem(p, g - 1), oracle.run_problem(p, g)
    T1, T2, T3 = (int(round(c * 2**32)) for c in (Cw, Cp, Cg))
    seen = set()
    for i in range(N):
        for j in range(D):
            r = oracle.rho(1, 0, g, i, j)
            if r < T1:
                want, br = prev["X"][i, j], "keep"
            elif r < T2:
                want, br = prev["P"][i, j], "pbest"
            elif r < T3:
                want, br = prev["G"][j], "gbest"
            else:
                want, br = oracle.fresh(lattice, 1, 0, oracle.TAG_FRESH, g, i, j, p["lb"], p["ub"]), "fresh"
            assert cur["X"][i, j] == want, (i, j, br)
            seen.add(br)
    assert seen == {"keep", "pbest", "gbest", "fresh"}


def test_paper_order_branch_frequencies():
    """Empirical branch frequencies within 5 sigma of the printed interval
    widths: keep Cw, pBest Cp - Cw, gBest Cg - Cp, fresh 1 - Cg."""
    Cw, Cp, Cg = 0.3, 0.6, 0.8
    p = _p(N=64, D=40, Cg=Cg, Cp=Cp, Cw=Cw, order="paper")
    r = oracle.run_problem(p, 30)
    n = r["branch"].sum()
    want = np.array([Cg - Cp, Cp - Cw, Cw, 1 - Cg])      # gBest, pBest, keep, fresh
    assert np.all(np.abs(r["branch"] / n - want) <= 5 * np.sqrt(want * (1 - want) / n))


def test_order_thresholds_validated():
    p = _p(Cg=0.4, Cp=0.7, Cw=0.9, order="paper")      # needs Cw <= Cp <= Cg
    with pytest.raises(ValueError):
        oracle.run_problem(p, 1)


# ---- asynchronous flow (Alg. 1) ------------------------------------------------------------
@pytest.mark.parametrize("fn", ["sphere", "rastrigin", "rosenbrock", "ackley"])
def test_async_without_gbest_branch_equals_sync(fn):
    """Cg = 0: no particle reads gBest, so the particles are independent and the
    asynchronous flow moves exactly as the synchronous one (positions, pBests,
    pBest fitness and the gBest value; only the tie rule "<" vs "<=" differs,
    which leaves P unchanged when it fires on an identical row)."""
    p = _p(fn, N=20, D=7, Cg=0.0, Cp=0.6, Cw=0.9)
    a = oracle.run_problem(p, 25, flow="async")
    s = oracle.run_problem(p, 25, flow="sync")
    assert np.array_equal(a["X"], s["X"]) and np.array_equal(a["P"], s["P"])
    assert np.array_equal(a["pF"], s["pF"]) and np.array_equal(a["log_v"], s["log_v"])


@pytest.mark.parametrize("order", ["gpx", "paper"])
def test_async_invariants(order):
    """Alg. 1: the gBest value never increases and after every generation it is
    the minimum pBest value, the gBest row is that particle's pBest row, and
    every pBest value is the fitness of its row."""
    kw = dict(Cg=0.4, Cp=0.7, Cw=0.9) if order == "gpx" else dict(Cg=0.8, Cp=0.6, Cw=0.3)
    p = _p("rastrigin", N=30, D=8, order=order, **kw)
    prev = None
    for t in (0, 1, 2, 5, 9):
        r = oracle.run_problem(p, t, flow="async")
        assert np.all(np.diff(r["log_v"]) <= 0)
        assert r["log_v"][t] == r["pF"].min()
        b = r["log_b"][t]
        assert r["pF"][b] == r["log_v"][t]
        assert np.array_equal(r["G"], r["P"][b])
        f = np.array([oracle.fitness("rastrigin", x, p["o"]) for x in r["P"]])
        assert np.array_equal(r["pF"], f)
        if prev is not None:
            assert np.all(r["pF"] <= prev["pF"])
        prev = r


def test_async_sees_gbest_of_same_generation():
    """The defining difference from Alg. 2: some particle of a generation reads
    a gBest row that an earlier particle of the same generation produced, so
    the flows part ways (with Cg > 0) after the first improving generation."""
    p = _p("sphere", N=40, D=10, Cg=0.4, Cp=0.7, Cw=0.9)
    a = oracle.run_problem(p, 6, flow="async")
    s = oracle.run_problem(p, 6, flow="sync")
    assert not np.array_equal(a["X"], s["X"])
    # generation 1 up to the first particle that improves gBest is identical
    a1 = oracle.run_problem(p, 1, flow="async")
    s1 = oracle.run_problem(p, 1, flow="sync")
    s0 = oracle.run_problem(p, 0, flow="sync")
    f1 = np.array([oracle.fitness("sphere", x, p["o"]) for x in s1["X"]])
    k = int(np.argmax(f1 < s0["log_v"][0])) if np.any(f1 < s0["log_v"][0]) else 40
    assert np.array_equal(a1["X"][:k + 1], s1["X"][:k + 1])


def test_async_sequential_consistency_check():
    """A plain restatement of Alg. 1 on the oracle's own primitives (rho words,
    fresh values, fitness) reproduces the compiled oracle's generation 2 from
    its generation 1 -- a consistency check of the loop structure."""
    N, D, g = 14, 5, 2
    Cg, Cp, Cw = 0.4, 0.7, 0.9
    p = _p("rastrigin", N=N, D=D, Cg=Cg, Cp=Cp, Cw=Cw)
    r1 = oracle.run_problem(p, g - 1, flow="async")
    r2 = oracle.run_problem(p, g, flow="async")
    X, P, pF, G = r1["X"].copy(), r1["P"].copy(), r1["pF"].copy(), r1["G"].copy()
    gF = r1["log_v"][g - 1]
    T = [int(round(c * 2**32)) for c in (Cg, Cp, Cw)]
    for i in range(N):
        for j in range(D):
            r = oracle.rho(1, 0, g, i, j)
            if r < T[0]:
                X[i, j] = G[j]
            elif r < T[1]:
                X[i, j] = P[i, j]
            elif r >= T[2]:
                X[i, j] = oracle.fresh("f64", 1, 0, oracle.TAG_FRESH, g, i, j, p["lb"], p["ub"])
        f = oracle.fitness("rastrigin", X[i], p["o"])
        if f < pF[i]:
            P[i], pF[i] = X[i], f
            if f < gF:
                G, gF = X[i].copy(), f
    assert np.array_equal(X, r2["X"]) and np.array_equal(P, r2["P"]) and np.array_equal(G, r2["G"])
