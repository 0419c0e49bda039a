"""Pins of the oracle's paper mode: the GS-LEX smoother of Sec. 2.4 (mode=1)
and the reading of the extra sweeps as one block after a whole smoothing
phase (extra_once=1).

The paper measured its printed factors with GS-LEX (lexicographic
Gauss-Seidel over Omega_h u Gamma_h, the ghost rows relaxed in place with the
step of Eqs. (dir2d)/(neu2d)), so the tables are checked here in that mode:
  * Table rhoC (Sec. 3.3.1): W-cycle, lambda = 5, delta = 3h, nu = 2 and 3;
  * Table badrho (Sec. 3.2): without extra sweeps TGCS and W stay near 0.6
    while the V-cycle degrades as h shrinks;
  * what makes the sweep lexicographic: after one sweep a perturbation has
    moved only forward in node order (nothing before it changes, except the
    few rows that read it) and has reached nodes far ahead of it;
  * the ghost rows take part in the main sweep and in the band sweeps;
  * the discrete solution is a fixed point of every relaxation.
The extra_once reading coincides with the default when nu = 1 and relaxes
less than it otherwise, so its factor lies between the two.
"""
import json
import os

import numpy as np
import pytest

from helpers import direct_solve, oracle_for, problem_rhs, rho_homogeneous
from paper_1111_0983_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")
PAPER = dict(rhs=False, junction_sweeps=0, mode=1)


def _table(key):
    with open(os.path.join(GOLD, "paper_rho.json")) as fh:
        return json.load(fh)[key]


# ------------------------------------------------------------ paper tables
def test_gslex_table_rhoC_W_cycle_nu3():
    """Table rhoC (right): circle, W-cycle, lambda = 5, nu1 + nu2 = 3, N_c = 8,
    GS-LEX.  The printed factors scatter by about 0.03 from one N to the next;
    each must lie within 0.07 and their mean deviation within 0.04."""
    gold = _table("rhoC_W_lambda5_nu3_Nc8")
    P = inputs.circle_paper()
    dev = []
    for N, rho_p in zip(gold["N"][:4], gold["rho"][:4]):
        rho = rho_homogeneous(oracle_for(P, N + 1, 9, gamma=2, nu1=2, nu2=1, **PAPER))
        dev.append(abs(rho - rho_p))
        assert dev[-1] < 0.07, (N, rho, rho_p)
    assert np.mean(dev) < 0.04, dev


def test_gslex_table_rhoC_W_cycle_nu2():
    """Table rhoC (left): same, nu1 = nu2 = 1."""
    gold = _table("rhoC_W_lambda5_nu2_Nc8")
    P = inputs.circle_paper()
    for N, rho_p in zip(gold["N"][:4], gold["rho"][:4]):
        rho = rho_homogeneous(oracle_for(P, N + 1, 9, gamma=2, nu1=1, nu2=1, **PAPER))
        assert abs(rho - rho_p) < 0.08, (N, rho, rho_p)


def test_gslex_table_badrho():
    """Table badrho (right): no extra sweeps, nu1 = 2, nu2 = 1.  TGCS and the
    W-cycle stay near the printed 0.58-0.61; the V-cycle degrades as h
    shrinks (printed 0.72, 0.73, 0.83) and ends well above the W-cycle; the
    extra sweeps (lambda = 5) restore the factor (Sec. 3.2)."""
    gold = _table("badrho_nu21_no_extra")
    P = inputs.circle_paper()
    v = {}
    for N, tg_p, w_p in zip(gold["N"], gold["TGCS"], gold["W"]):
        w = rho_homogeneous(oracle_for(P, N + 1, 9, lam=0, gamma=2, nu1=2, nu2=1, **PAPER))
        v[N] = rho_homogeneous(oracle_for(P, N + 1, 9, lam=0, gamma=1, nu1=2, nu2=1, **PAPER))
        assert abs(w - w_p) < 0.08, (N, w, w_p)
        if N <= 128:
            tg = rho_homogeneous(oracle_for(P, N + 1, N // 2 + 1, lam=0, nu1=2, nu2=1, **PAPER))
            assert abs(tg - tg_p) < 0.08, (N, tg, tg_p)
            good = rho_homogeneous(oracle_for(P, N + 1, 9, lam=5, gamma=2, nu1=2, nu2=1, **PAPER))
            assert good < 0.25 * w, (N, good, w)
    assert v[256] > v[128] > v[64] - 0.05, v
    assert v[256] > 0.8, v


# -------------------------------------------------- what GS-LEX is made of
def _direct(P, n, nc, **kw):
    O = oracle_for(P, n, nc, **kw)
    f, g = problem_rhs(O, P, n)
    O.set_rhs(f, g)
    return O, f, g, direct_solve(O, f, g)


@pytest.mark.parametrize("mode", [0, 1])
def test_discrete_solution_is_a_fixed_point_of_each_relaxation(mode):
    """Every relaxation (base sweep, lambda band sweeps) leaves the discrete
    solution unchanged: each interior row is solved for its own node and each
    ghost moves by c (g - L_G u) = 0 there."""
    P = inputs.flower()
    O, f, g, ud = _direct(P, 65, 17, junction_sweeps=0, mode=mode)
    u1 = O.relax(ud, f, g, 0, with_extra=True)
    T = O.types(0) > 0
    assert np.abs(u1 - ud)[T].max() < 1e-11 * np.abs(ud)[T].max()


def test_gslex_moves_a_perturbation_forward_in_node_order():
    """One GS-LEX sweep (no extra sweeps) of the discrete solution with and
    without a perturbation at one inside node p: nodes that come before p and
    whose rows do not read p get bitwise the same values, and the change reaches nodes many rows
    ahead of p (a red-black sweep moves it by two nodes at most)."""
    P = inputs.disk()
    n = 65
    O, f, g, ud = _direct(P, n, 17, lam=0, junction_sweeps=0, mode=1)
    T = O.types(0)
    p = (n // 2) * n + n // 2 - 8          # an inside node left of the centre
    assert T.ravel()[p] == 1
    u0 = ud.copy()
    u0.ravel()[p] += 1.0
    d = np.abs(O.relax(u0, f, g, 0, with_extra=False) - O.relax(ud, f, g, 0, with_extra=False)).ravel()
    reach = 2 * n + 2                       # farthest read of any row (ghost stencils)
    assert d[: p - reach].max() == 0.0
    assert d[p + 6 * n] > 1e-9              # six x-rows ahead
    # the same perturbation under red-black + Jacobi ghosts stays local
    O0 = oracle_for(P, n, 17, lam=0, junction_sweeps=0, mode=0)
    O0.set_rhs(f, g)
    d0 = np.abs(O0.relax(u0, f, g, 0, with_extra=False) - O0.relax(ud, f, g, 0, with_extra=False)).ravel()
    assert d0[p + 6 * n] == 0.0


def test_gslex_relaxes_the_ghost_rows():
    """A perturbation at a ghost shrinks in one GS-LEX sweep (its row is
    relaxed in the main sweep), and shrinks further when the lambda band
    sweeps follow (their sweeps take the ghosts too)."""
    P = inputs.disk()
    n = 65
    O, f, g, ud = _direct(P, n, 17, lam=5, junction_sweeps=0, mode=1)
    G = O.ghosts(0)
    q = int(np.argmax(G["case"] == 0))      # a ghost with a full quadratic stencil
    node = int(G["node"][q])
    u0 = ud.copy()
    u0.ravel()[node] += 1.0
    e_base = abs(O.relax(u0, f, g, 0, with_extra=False).ravel()[node] - ud.ravel()[node])
    e_extra = abs(O.relax(u0, f, g, 0, with_extra=True).ravel()[node] - ud.ravel()[node])
    assert e_base < 0.95
    assert e_extra < 0.5 * e_base, (e_base, e_extra)


# ------------------------------------------------------------- extra_once
def test_extra_once_equals_default_for_single_sweeps():
    """With nu1 = nu2 = 1 a smoothing phase is one relaxation, so the two
    readings of "after a single relaxation" (Sec. 3.2) give the same cycle."""
    P = inputs.circle_paper()
    a = oracle_for(P, 65, 9, nu1=1, nu2=1, junction_sweeps=0, mode=1, extra_once=0).solve(rtol=1e-12, max_cycles=8)[1]
    b = oracle_for(P, 65, 9, nu1=1, nu2=1, junction_sweeps=0, mode=1, extra_once=1).solve(rtol=1e-12, max_cycles=8)[1]
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("mode", [0, 1])
def test_extra_once_relaxes_between_none_and_every_sweep(mode):
    """nu1 = 2: lambda sweeps after the whole phase help (far below lambda =
    0) but less than after every relaxation; the solution is unchanged."""
    P = inputs.circle_paper()
    kw = dict(rhs=False, nu1=2, nu2=1, gamma=2, junction_sweeps=0, mode=mode)
    none = rho_homogeneous(oracle_for(P, 65, 9, lam=0, **kw))
    once = rho_homogeneous(oracle_for(P, 65, 9, lam=5, extra_once=1, **kw))
    each = rho_homogeneous(oracle_for(P, 65, 9, lam=5, extra_once=0, **kw))
    assert once < 0.5 * none and each < once, (none, once, each)
    F = inputs.flower()
    O, f, g, ud = _direct(F, 65, 17, junction_sweeps=0, mode=mode, extra_once=1)
    u, _, ok = O.solve(rtol=1e-13, max_cycles=100)
    T = O.types(0) > 0
    assert ok and np.abs(u - ud)[T].max() < 1e-11 * np.abs(ud)[T].max()
