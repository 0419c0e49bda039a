"""Shared test helpers: oracle set-up for a problem, direct sparse solves."""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl

import oracle
from paper_1111_0983_gb300 import inputs


def oracle_for(P: inputs.Problem, n: int, n_coarse: int | None = None, rhs=True, **kw):
    """Oracle hierarchy for problem P on n^d nodes with the boundary types set
    on every level from the problem's split and (optionally) f, g on level 0."""
    phi = P.phi_grid(n)
    O = oracle.Oracle(phi, n_coarse or P.n_coarse, **kw)
    for l in range(O.nlev):
        G = O.ghosts(l)
        O.set_bc(l, P.bc_types(G["B"]))
    if rhs:
        G = O.ghosts(0)
        types = P.bc_types(G["B"])
        O.set_rhs(P.f_grid(n), P.g_values(G["B"], G["nu"], types))
    return O


def rhs_vector(O, f, g, l=0):
    rows, cols, vals, uon = O.assemble(l)
    N = int(uon.max()) + 1
    T = O.types(l)
    b = np.zeros(N)
    b[uon[T == 1]] = f[T == 1]
    b[uon.ravel()[O.ghosts(l)["node"]]] = g
    return b


def direct_solve(O, f, g, l=0):
    """Direct sparse LU (scipy SuperLU) of the assembled level-l system; the
    result is scattered to the grid (0 off Omega_h u Gamma_h)."""
    rows, cols, vals, uon = O.assemble(l)
    N = int(uon.max()) + 1
    A = sp.csc_matrix((vals, (rows, cols)), shape=(N, N))
    b = rhs_vector(O, f, g, l)
    x = spl.spsolve(A, b)
    u = np.zeros(uon.shape)
    m = uon >= 0
    u[m] = x[uon[m]]
    return u


def problem_rhs(O, P, n):
    G = O.ghosts(0)
    types = P.bc_types(G["B"])
    return P.f_grid(n), P.g_values(G["B"], G["nu"], types)


def level_rhs(O, P, l):
    """f and g of problem P sampled on level l of a hierarchy (the level's
    nodes and its ghosts' boundary points)."""
    n = O.level_n(l)
    G = O.ghosts(l)
    return P.f_grid(n), P.g_values(G["B"], G["nu"], P.bc_types(G["B"]))


def set_level_rhs(O, P):
    """f and g on every level of an oracle hierarchy (for full multigrid)."""
    for l in range(O.nlev):
        O.set_rhs_level(l, *level_rhs(O, P, l))


def rel_maxdiff(a, b, mask):
    return np.abs(a - b)[mask].max() / max(np.abs(b)[mask].max(), 1e-300)


def rho_homogeneous(O, cycles=30, seed=1):
    """Convergence factor by the paper's recipe (Sec. 3): homogeneous problem,
    seeded nonzero guess, stop when |rho_m - rho_{m-1}| / rho_m < 1e-3."""
    shape = O.shape(0)
    O.set_rhs(np.zeros(shape), np.zeros(O.num_ghosts(0)))
    u0 = inputs.homogeneous_guess(shape, seed)
    _, norms, _ = O.solve(u0, rtol=1e-300, max_cycles=cycles)
    r = norms[1:] / norms[:-1]
    for m in range(1, len(r)):
        if abs(r[m] - r[m - 1]) / r[m] < 1e-3:
            return float(r[m])
    return float(r[-1])
