"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand) fails one of them:
  * brute force: multigrid converges to the direct sparse solution of the
    assembled system (checks the cycle's transfer operators and smoother);
  * polynomial exactness of every equation row (quadratic for the full
    3^d stencils, linear for the reduced ones), in 2D and 3D, Dirichlet and
    Neumann: pins interior stencil, closest point B, stencil orientation,
    Lagrange weights and the discrete normal;
  * a whole-system quadratic patch test (discrete solution == exact u);
  * second-order convergence to manufactured solutions (Sec. 2.3 accuracy);
  * h-independent V-cycle factor on Dirichlet domains (the central claim);
  * the paper's printed convergence factors (Tables rhoC, badrho);
  * invariants of restriction (printed stencils, partition of unity),
    extension (constants, fields constant along normals), interpolation
    (linear exactness), mirror symmetry and the CFL bounds of Sec. 2.3.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1111_0983_gb300 import inputs
from helpers import direct_solve, oracle_for, problem_rhs, rel_maxdiff, rho_homogeneous, set_level_rhs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as fh:
        return json.load(fh)


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("P,n,nc", [(inputs.disk(), 33, 9), (inputs.flower(), 65, 17),
                                    (inputs.star(4), 65, 33), (inputs.torus(), 17, 9)])
def test_multigrid_matches_direct_solve(P, n, nc):
    O = oracle_for(P, n, nc)
    f, g = problem_rhs(O, P, n)
    ud = direct_solve(O, f, g)
    u, norms, ok = O.solve(rtol=1e-13, max_cycles=200)
    assert ok
    T = O.types(0)
    assert rel_maxdiff(u, ud, T > 0) < 1e-11


# ------------------------------------------------------ polynomial exactness
def _row_residuals(O, P, n, l=0):
    """Residual of the exact u in every equation row of level l."""
    G = O.ghosts(l)
    types = P.bc_types(G["B"])
    O.set_bc(l, types)
    f = P.f_grid(n)
    g = P.g_values(G["B"], G["nu"], types)
    if l == 0:
        O.set_rhs(f, g)
    r, _ = O.defect(P.u_grid(n), l)
    return r, G


@pytest.mark.parametrize("dim,n,neumann", [(2, 33, "none"), (2, 33, "all"), (2, 65, "half"),
                                           (3, 17, "none"), (3, 17, "all"), (3, 33, "half")])
def test_quadratic_rows_exact(dim, n, neumann):
    P = inputs.quadratic_patch(dim, neumann=neumann)
    O = oracle.Oracle(P.phi_grid(n), 9)
    r, G = _row_residuals(O, P, n)
    T = O.types(0)
    scale = np.abs(P.u_grid(n)).max()
    assert np.abs(r[T == 1]).max() < 1e-9 * scale * (n * n)        # 5/7-point Laplacian
    quad = G["case"] == oracle.ST_QUAD
    assert quad.sum() > 0.8 * len(quad)
    rg = r.ravel()[G["node"]]
    assert np.abs(rg[quad]).max() < 1e-11 * scale * n


@pytest.mark.parametrize("P,n", [(inputs.star(4), 33), (inputs.star(27), 33), (inputs.star(21), 33),
                                 (inputs.quadratic_patch(3), 17)])
def test_linear_rows_exact_all_stencils(P, n):
    rng = np.random.default_rng(3)
    c = rng.uniform(-1, 1, size=P.dim + 1)
    lin = inputs.quadratic_patch(P.dim, coef=np.concatenate([c, np.zeros(P.dim * (P.dim + 1) // 2)]))
    lin.phi = P.phi
    lin.is_neumann = lambda B: B[:, 0] > 0.05
    O = oracle.Oracle(lin.phi_grid(n), 17)
    r, G = _row_residuals(O, lin, n)
    cases = np.bincount(G["case"], minlength=4)
    assert cases[1:].sum() > 0          # reduced stencils present
    T = O.types(0)
    assert np.abs(r[T == 1]).max() < 1e-11 * n * n
    # every ghost row is exact for linear u, except the two-point axis
    # stencil with Dirichlet data: it interpolates at the projection of B on
    # its axis line (first order, the "less accurate" stencil of Remark 3)
    types = lin.bc_types(G["B"])
    exact = ~((G["case"] == oracle.ST_AXIS) & (types == 0))
    rg = r.ravel()[G["node"]]
    assert np.abs(rg[exact]).max() < 1e-11 * n * n
    assert (~exact).sum() <= 0.05 * len(exact)


def test_ghost_weight_identities():
    """Dirichlet weights interpolate constants (sum 1); Neumann weights
    differentiate constants (sum 0) and give nu . grad for linear fields."""
    P = inputs.star(4)
    n = 65
    O = oracle.Oracle(P.phi_grid(n), 17)
    G = O.ghosts(0)
    h = 2.0 / (n - 1)
    X = inputs.coords(2, n)
    for q in range(len(G["node"])):
        k = G["nk"][q]
        st = G["stn"][q, :k]
        assert abs(G["wD"][q, :k].sum() - 1.0) < 1e-13
        assert abs(G["wN"][q, :k].sum()) < 1e-10 / h
        for a in range(2):
            if G["case"][q] == oracle.ST_AXIS and G["s"][q, a] == 0:
                continue        # the two-point stencil sees only its own axis
            xa = X[a].ravel()[st]
            assert abs(G["wD"][q, :k] @ xa - G["B"][q, a]) < 1e-13
            assert abs(G["wN"][q, :k] @ xa - G["nu"][q, a]) < 1e-10
        assert abs(np.linalg.norm(G["nu"][q]) - 1) < 1e-14


def test_closest_point_lies_on_sdf_boundary():
    """For a signed distance function, B = G - phi grad phi/|grad phi|^2 lies on
    the circle up to the O(h^2) central-difference error (Eq. clpt)."""
    P = inputs.circle_paper()
    for n in (65, 129):
        O = oracle.Oracle(P.phi_grid(n), 9)
        B = O.ghosts(0)["B"]
        c = (math.sqrt(2) / 20, math.sqrt(3) / 30)
        d = np.hypot(B[:, 0] - c[0], B[:, 1] - c[1]) - 0.563
        h = 2.0 / (n - 1)
        assert np.abs(d).max() < 0.5 * h * h


# --------------------------------------------------------- whole-system patch
@pytest.mark.parametrize("neumann", ["none", "half"])
def test_quadratic_patch_solution_exact(neumann):
    P = inputs.quadratic_patch(2, neumann=neumann)
    n = 65
    O = oracle_for(P, n, 9)
    assert np.all(O.ghosts(0)["case"] == oracle.ST_QUAD)
    f, g = problem_rhs(O, P, n)
    u = direct_solve(O, f, g)
    T = O.types(0)
    assert np.abs(u - P.u_grid(n))[T > 0].max() < 1e-10


# ------------------------------------------------------------- second order
@pytest.mark.parametrize("P,ns", [(inputs.flower(), (257, 513, 1025)), (inputs.disk(), (65, 129, 257)),
                                  (inputs.torus(), (65, 129))])
def test_second_order_convergence(P, ns):
    errs = []
    for n in ns:
        O = oracle_for(P, n, 17 if P.dim == 3 else P.n_coarse)
        f, g = problem_rhs(O, P, n)
        u = direct_solve(O, f, g) if P.dim == 2 else O.solve(rtol=1e-10, max_cycles=40)[0]
        T = O.types(0)
        errs.append(np.abs(u - P.u_grid(n))[T == 1].max())
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert min(ratios) > 3.0, (errs, ratios)


# ----------------------------------------------------- convergence factors
def test_vcycle_rho_h_independent_dirichlet():
    """Sec. 3 central claim on a Dirichlet domain: V(2,1) factor bounded as h -> 0."""
    P = inputs.flower()
    P.is_neumann = lambda B: np.zeros(B.shape[0], bool)
    rhos = [rho_homogeneous(oracle_for(P, n, 33, rhs=False)) for n in (129, 257, 513)]
    assert max(rhos) < 0.12, rhos
    assert rhos[-1] <= 1.1 * rhos[0] + 0.01, rhos


def test_paper_table_rhoC_W_cycle_nu3():
    """Circle, W-cycle, lambda = 5, nu = 3, Nc = 8 (Table rhoC, right)."""
    gold = _gold("paper_rho.json")["rhoC_W_lambda5_nu3_Nc8"]
    P = inputs.circle_paper()
    for N, rho_p in zip(gold["N"][:4], gold["rho"][:4]):
        rho = rho_homogeneous(oracle_for(P, N + 1, 9, rhs=False, gamma=2, nu1=2, nu2=1, junction_sweeps=0))
        assert abs(rho - rho_p) < 0.045, (N, rho, rho_p)


def test_paper_table_rhoC_W_cycle_nu2():
    """Circle, W-cycle, lambda = 5, nu = 2 (Table rhoC, left): same size as printed."""
    gold = _gold("paper_rho.json")["rhoC_W_lambda5_nu2_Nc8"]
    P = inputs.circle_paper()
    for N, rho_p in zip(gold["N"][:4], gold["rho"][:4]):
        rho = rho_homogeneous(oracle_for(P, N + 1, 9, rhs=False, gamma=2, nu1=1, nu2=1, junction_sweeps=0))
        assert abs(rho - rho_p) < 0.08, (N, rho, rho_p)


def test_paper_table_badrho_degradation():
    """Without extra sweeps the factor is far from LFA (Table badrho); the
    extra sweeps (lambda = 5) restore it (Sec. 3.2)."""
    gold = _gold("paper_rho.json")["badrho_nu21_no_extra"]
    P = inputs.circle_paper()
    for N, tg_p, w_p in zip(gold["N"][:2], gold["TGCS"][:2], gold["W"][:2]):
        paper = dict(rhs=False, nu1=2, nu2=1, junction_sweeps=0)
        tg = rho_homogeneous(oracle_for(P, N + 1, N // 2 + 1, lam=0, **paper))
        w = rho_homogeneous(oracle_for(P, N + 1, 9, lam=0, gamma=2, **paper))
        assert abs(tg - tg_p) < 0.08 and abs(w - w_p) < 0.08, (N, tg, w)
        good = rho_homogeneous(oracle_for(P, N + 1, 9, lam=5, gamma=2, **paper))
        assert good < 0.25 * tg


def test_junction_relaxation_restores_mixed_bc_vcycle():
    """Where Dirichlet and Neumann ghosts meet, the V-cycle of the paper's
    smoother degrades with h (and diverges on star 0); the junction relaxation
    keeps the factor bounded."""
    P = inputs.star(0)
    assert rho_homogeneous(oracle_for(P, 257, 65, rhs=False, junction_sweeps=0)) > 1.0
    assert rho_homogeneous(oracle_for(P, 257, 65, rhs=False)) < 0.15
    F = inputs.flower()
    plain = [rho_homogeneous(oracle_for(F, n, 33, rhs=False, junction_sweeps=0)) for n in (257, 513)]
    fixed = [rho_homogeneous(oracle_for(F, n, 33, rhs=False)) for n in (257, 513)]
    assert plain[1] > 0.5 and fixed[1] < 0.2 and fixed[0] < 0.15, (plain, fixed)


def test_junction_solve_is_exact_on_its_set():
    """The exact junction solve leaves a zero defect on every equation it
    solves (with all other values held fixed); its set holds each junction
    ghost and, for each ghost in it, the ghost's whole stencil."""
    F = inputs.flower()
    n = 129
    O = oracle_for(F, n, 33)
    rng = np.random.default_rng(3)
    u = rng.standard_normal(O.shape(0))
    G = O.ghosts(0)
    f = F.f_grid(n)
    g = F.g_values(G["B"], G["nu"], F.bc_types(G["B"]))
    O.set_rhs(f, g)
    r_before = np.abs(O.defect(u, 0)[0]).max()
    u1 = O.relax(u, f, g, 0)
    r = np.abs(O.defect(u1, 0)[0]).ravel()
    S = O.junction_solve_set(0).ravel().astype(bool)
    assert S.sum() > 100
    assert r[S].max() < 1e-9 * r_before
    assert r[~S].max() > 1e-3 * r_before          # elsewhere only relaxed
    T = O.types(0).ravel() & 3
    assert np.all(T[S] > 0)                      # unknowns only
    bc = F.bc_types(G["B"])
    pos = {int(x): q for q, x in enumerate(G["node"])}
    for q, node in enumerate(G["node"]):
        if S[node]:
            assert all(S[int(m)] for m in G["stn"][q][:G["nk"][q]]), q
    Z = O.junction_zone(0).ravel().astype(bool)
    nl = O.level_n(0)
    for q, node in enumerate(G["node"]):
        i, j = divmod(int(node), nl)
        nb = [pos.get((i + a) * nl + j + b) for a in (-1, 0, 1) for b in (-1, 0, 1)]
        if any(k is not None and bc[k] != bc[q] for k in nb):
            assert Z[node]


def test_junction_solve_stable_where_sweeps_grow():
    """Next to a Dirichlet ghost whose own weight in its condition is almost
    zero (star 167 at 1025^2: 0.004), mu_J = 40 sweeps of the 12h zone grow
    a local mode, while the exact zone solve (the 2D default) converges."""
    P = inputs.star(167)
    n = P.meta["n"]
    assert n == 1025
    _, norms, ok = oracle_for(P, n, 33, junction_sweeps=40, junction_solve=0,
                              junction_radius=12.0).solve(rtol=1e-10, max_cycles=8)
    assert norms[-1] > 1e3 * norms[0]
    _, norms, ok = oracle_for(P, n, 33).solve(rtol=1e-10, max_cycles=30)
    assert ok and len(norms) - 1 <= 20


# -------------------------------------------------------------- restriction
def test_restriction_printed_stencils():
    """Sec. 2.5: the partial transfer over Omega_h of an axis-aligned square
    gives full weighting inside, the 3x2 stencil (Fstencil23) on an edge and
    the 2x2 stencil (Fstencil22) at a corner."""
    gold = _gold("restriction_stencils.json")
    n = 33
    h = 2.0 / (n - 1)
    X = inputs.coords(2, n)
    # interior nodes: |x|, |y| <= 0.5; coarse nodes at x = 0.5 have their +x fine
    # neighbour outside
    phi = np.maximum(np.abs(X[0]), np.abs(X[1])) - (0.5 + 0.5 * h)
    O = oracle.Oracle(phi, 17)
    nc = 17
    hc = 2 * h
    J = lambda x: int(round((x + 1) / hc))
    cases = {"full_3x3": (J(0.0), J(0.0)),
             "rect_3x2_x_in_-1_0": (J(0.5), J(0.0)),     # x in {-1,0}, y in {-1,1}
             "rect_2x2": (J(0.5), J(-0.5))}             # x in {-1,0}, y in {0,1}
    for key, (jx, jy) in cases.items():
        wt = O.restrict_weights(0, np.ravel_multi_index((jx, jy), (nc, nc)), 1)
        want = np.array(gold[key]["w16"], float) / 16.0
        # printed stencils: rows = y offset, columns = x offset; ours [x][y]
        assert wt is not None and np.allclose(wt.T, want), (key, wt.T * 16)


def test_restriction_partition_of_unity():
    P = inputs.star(4)
    n = 65
    O = oracle_for(P, n, 17, rhs=False)
    Tc = O.types(1)
    cnt = 0
    for X in np.flatnonzero(Tc.ravel() > 0):
        wt = O.restrict_weights(0, X, 1 if Tc.ravel()[X] == 1 else 0)
        assert wt is not None and abs(wt.sum() - 1) < 1e-14
        cnt += 1
    assert cnt > 100
    # a constant defect restricts to the same constant everywhere
    r = np.full(O.shape(0), 2.5)
    fc, gc = O.restrict(r)
    assert np.allclose(fc[Tc == 1], 2.5) and np.allclose(gc, 2.5)


# ---------------------------------------------------------------- extension
def test_extension_constants_and_normal_invariance():
    P = inputs.disk()
    n = 129
    O = oracle_for(P, n, 17, rhs=False)
    E = O.extension(0)
    assert len(E["node"]) > 0
    r = np.zeros(O.shape(0))
    T = O.types(0)
    r[T == 2] = 1.75
    re = O.extend(r)
    assert np.allclose(re.ravel()[E["node"]], 1.75, rtol=0, atol=1e-14)
    # a field constant along the normals of the (SDF) disk is kept to O(h)
    X = inputs.coords(2, n)
    ang = np.arctan2(X[1] - 0.01, X[0] - 0.02)
    field = np.cos(3 * ang)
    r = np.where(T == 2, field, 0.0)
    re = O.extend(r)
    h = 2.0 / (n - 1)
    err = np.abs(re.ravel()[E["node"]] - field.ravel()[E["node"]]).max()
    assert err < 12 * h, err


def test_extension_is_upwind_ordered():
    O = oracle_for(inputs.flower(), 129, 33, rhs=False)
    E = O.extension(0)
    phi = inputs.flower().phi_grid(129).ravel()
    pos = {int(v): i for i, v in enumerate(E["node"])}
    for i, P in enumerate(E["node"]):
        for s in E["src"][i, :E["nsrc"][i]]:
            assert phi[s] < phi[P]
            if int(s) in pos:
                assert pos[int(s)] < i


# --------------------------------------------------------------- prolongation
def test_prolongation_linear_exact_where_parents_exist():
    P = inputs.flower()
    n = 129
    O = oracle_for(P, n, 33, rhs=False)
    Xc = inputs.coords(2, 65)
    e = 0.3 + 1.7 * Xc[0] - 0.9 * Xc[1]
    Tc = O.types(1)
    ec = np.where(Tc > 0, e, 0.0)
    out = O.prolong(ec)
    X = inputs.coords(2, n)
    want = 0.3 + 1.7 * X[0] - 0.9 * X[1]
    T = O.types(0)
    # fine nodes whose coarse parents all lie in Omega_2h u Gamma_2h
    ok = np.zeros(T.shape, bool)
    for i, j in zip(*np.nonzero(T > 0)):
        par = [(a, b) for a in {i // 2, (i + 1) // 2} for b in {j // 2, (j + 1) // 2}]
        ok[i, j] = all(Tc[a, b] > 0 for a, b in par)
    assert ok.sum() > 0.9 * (T > 0).sum()
    assert np.abs(out - want)[ok].max() < 1e-13
    # a constant is reproduced at every unknown (renormalised weights)
    out = O.prolong(np.where(Tc > 0, 4.0, 0.0))
    assert np.allclose(out[T > 0], 4.0)


# ------------------------------------------------------ symmetry and CFL
def test_mirror_symmetry_sgn_zero_rule():
    """A domain and data symmetric under y -> -y give a symmetric solution to
    rounding; ghosts on y = 0 exercise the sgn(0) reading."""
    P = inputs.Problem("mirror", 2,
                       phi=lambda x, y: np.sqrt((x - 0.031) ** 2 + y * y) - 0.57,
                       u=lambda x, y: np.cos(2 * x) * np.cosh(y),
                       grad_u=lambda x, y: [-2 * np.sin(2 * x) * np.cosh(y), np.cos(2 * x) * np.sinh(y)],
                       f=lambda x, y: 3 * np.cos(2 * x) * np.cosh(y),
                       is_neumann=lambda B: B[:, 0] > 0.1)
    n = 129
    O = oracle_for(P, n, 17)
    G = O.ghosts(0)
    assert (G["s"] == 0).any()
    T = O.types(0)
    assert np.array_equal(T, T[:, ::-1])
    f, g = problem_rhs(O, P, n)
    ud = direct_solve(O, f, g)
    # an asymmetric discretisation would show at the O(h^2) ~ 1e-4 level; the
    # sparse LU's rounding stays near cond * eps
    assert np.abs(ud - ud[:, ::-1])[T > 0].max() < 1e-9 * np.abs(ud).max()
    # red-black + Jacobi ghost sweeps commute with the mirror (n - 1 even)
    u, norms, ok = O.solve(rtol=1e-10, max_cycles=100)
    assert ok
    assert np.abs(u - u[:, ::-1])[T > 0].max() < 1e-9 * np.abs(u).max()


@pytest.mark.parametrize("P,n", [(inputs.flower(), 257), (inputs.star(4), 129), (inputs.torus(), 33)])
def test_cfl_bounds(P, n):
    """Sec. 2.3: mu_D dt = 0.9 and mu_N dt = 0.9 * 2h / (3 sqrt d) keep every
    ghost's self coefficient times its step in (0, 0.9]."""
    O = oracle_for(P, n, 17, rhs=False)
    G = O.ghosts(0)
    h = 2.0 / (n - 1)
    types = P.bc_types(G["B"])
    cN = 0.9 * 2 * h / (3 * math.sqrt(P.dim))
    for q in range(len(G["node"])):
        k = G["nk"][q]
        self_k = np.flatnonzero(G["stn"][q, :k] == G["node"][q])
        assert len(self_k) == 1
        wself = (G["wN"] if types[q] else G["wD"])[q, self_k[0]]
        c = cN if types[q] else 0.9
        assert 0 < c * wself <= 0.9 + 1e-12, (q, c * wself)


def test_geometry_errors_reported():
    n = 33
    X = inputs.coords(2, n)
    with pytest.raises(oracle.OracleError):
        oracle.Oracle(np.hypot(X[0], X[1]) - 0.99, 9)       # touches the box edge
    with pytest.raises(oracle.OracleError):
        oracle.Oracle(np.zeros((n, n)) - 1.0, 9)            # everything inside


# ------------------------------------------------------------ full multigrid
def test_fmg_single_level_is_direct_solve():
    """With one level, full multigrid is the coarsest solve: the direct
    solution of the assembled system."""
    P = inputs.disk()
    O = oracle_for(P, 17, 17)
    assert O.nlev == 1
    set_level_rhs(O, P)
    f, g = problem_rhs(O, P, 17)
    u = O.fmg(1)
    ud = direct_solve(O, f, g)
    assert rel_maxdiff(u, ud, O.types(0) > 0) < 1e-12


def test_fmg_many_cycles_reach_the_discrete_solution():
    """Enough cycles per level make every level's result its discrete
    solution, so the fine result is the direct solve's."""
    P = inputs.flower()
    O = oracle_for(P, 129, 33)
    set_level_rhs(O, P)
    f, g = problem_rhs(O, P, 129)
    u = O.fmg(20)
    assert rel_maxdiff(u, direct_solve(O, f, g), O.types(0) > 0) < 1e-9


def test_fmg_error_falls_with_cycles():
    """The error against the exact solution falls as cycles are added, towards
    the discretisation error; on the torus (boundary smooth on the coarsest
    grid) one cycle a level already reaches it, the property that defines
    full multigrid.  (Near a 2D boundary the method's interpolation is first
    order for a full solution, so one cycle a level does not reach it there.)"""
    P = inputs.flower()
    errs = []
    for nu in (1, 2, 3, 6):
        O = oracle_for(P, 257, 33)
        set_level_rhs(O, P)
        m = O.types(0) == 1
        errs.append(np.abs(O.fmg(nu) - P.u_grid(257))[m].max())
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    O = oracle_for(P, 257, 33)
    uc = O.solve(np.zeros(O.shape(0)), rtol=1e-12, max_cycles=100)[0]
    assert errs[-1] <= 1.1 * np.abs(uc - P.u_grid(257))[O.types(0) == 1].max()
    T = inputs.torus()
    O = oracle_for(T, 65, 17)
    set_level_rhs(O, T)
    m = O.types(0) == 1
    e1 = np.abs(O.fmg(1) - T.u_grid(65))[m].max()
    O = oracle_for(T, 65, 17)
    uc = O.solve(np.zeros(O.shape(0)), rtol=1e-12, max_cycles=100)[0]
    assert e1 <= 1.05 * np.abs(uc - T.u_grid(65))[m].max()


# ------------------------------------------------------- reinitialisation
@pytest.mark.parametrize("dim,n", [(2, 129), (3, 33)])
def test_reinit_distance_function(dim, n):
    """Reinitialisation (Eq. sdf) keeps an exact signed distance function and
    turns a level set with the same zero set but another profile into it,
    within a fraction of h in the band |phi| <= 3h where the ghost geometry
    reads it; no node changes sign (the zero set stays put); the error halves
    with h (the scheme is first order)."""
    errs = []
    tol = 0.3 if dim == 2 else 0.4   # the first-order constant grows with the dimension
    for m in (n, 2 * n - 1):
        h = 2.0 / (m - 1)
        X = inputs.coords(dim, m)
        c = (math.sqrt(2) / 20, math.sqrt(3) / 30, 0.01)[:dim]
        r = np.sqrt(sum((X[a] - c[a]) ** 2 for a in range(dim)))
        R = 0.563
        sdf = r - R
        band = np.abs(sdf) <= 3 * h
        p = oracle.reinit(sdf, 20)
        assert np.abs(p - sdf)[band].max() <= tol * h
        q = oracle.reinit(3.0 * (r ** 2 - R ** 2), 20)
        err = np.abs(q - sdf)[band].max()
        assert err <= tol * h, (m, err / h)
        assert np.array_equal(np.sign(q)[sdf != 0], np.sign(sdf)[sdf != 0])
        errs.append(err)
    assert errs[0] / errs[1] > 1.7, errs


# ------------------------------------------------ Kaczmarz comparison (Sec. 3.3)
def _kaczmarz_oracle(P, n, nc, lam=5, **kw):
    return oracle_for(P, n, nc, smoother=1, lam=lam, junction_solve=0, junction_sweeps=0, **kw)


def test_kaczmarz_step_moves_along_its_row_and_satisfies_it():
    """Sec. 3.3, Kaczmarz iteration: a step on row j changes u only on the row's
    support, by a multiple of the row (inside node: 2d t at the node, -t at
    each neighbour; ghost: t w_k at its stencil nodes), and leaves that row's
    equation satisfied."""
    P, n = inputs.disk(), 33
    O = _kaczmarz_oracle(P, n, 9)
    f, g = problem_rhs(O, P, n)
    T = O.types(0)
    band = O.band(0)
    rng = np.random.default_rng(7)
    u0 = np.where(T > 0, rng.standard_normal(T.shape), 0.0)
    r0, _ = O.defect(u0)
    # an inside node of the band
    i = int(np.flatnonzero(((T == 1) & (band > 0)).ravel())[17])
    u1 = O.kaczmarz_row(i, u0, f, g).ravel()
    d = u1 - u0.ravel()
    nb = [i + 1, i - 1, i + n, i - n]
    assert set(np.flatnonzero(d)) <= set([i] + nb)
    t = -d[nb[0]]
    assert t != 0.0 and np.allclose(d[nb], -t, rtol=1e-12, atol=0) and d[i] == pytest.approx(4 * t, rel=1e-12)
    r1, _ = O.defect(u1.reshape(T.shape))
    assert abs(r1.ravel()[i]) <= 1e-12 * abs(r0.ravel()[i])
    # a ghost
    G = O.ghosts(0)
    q = 5
    u2 = O.kaczmarz_row(int(G["node"][q]), u0, f, g).ravel()
    d = u2 - u0.ravel()
    types = P.bc_types(G["B"])
    w = (G["wN"] if types[q] else G["wD"])[q, : G["nk"][q]]
    stn = G["stn"][q, : G["nk"][q]]
    assert set(np.flatnonzero(d)) <= set(stn.tolist())
    m = w != 0
    ratio = d[stn[m]] / w[m]
    assert np.allclose(ratio, ratio[0], rtol=1e-10, atol=0) and ratio[0] != 0.0
    r2, _ = O.defect(u2.reshape(T.shape))
    assert abs(r2.ravel()[G["node"][q]]) <= 1e-12 * abs(r0.ravel()[G["node"][q]])


@pytest.mark.parametrize("P,n,nc", [(inputs.disk(), 33, 9), (inputs.flower(), 65, 17)])
def test_kaczmarz_relaxation_fixes_the_discrete_solution(P, n, nc):
    """The exact discrete solution (a direct sparse solve) is a fixed point of
    the Kaczmarz comparison relaxation: every row it steps on is satisfied."""
    O = _kaczmarz_oracle(P, n, nc)
    f, g = problem_rhs(O, P, n)
    us = direct_solve(O, f, g)
    u1 = O.relax(us, f, g, 0, True)
    assert np.max(np.abs(u1 - us)) <= 1e-11 * np.max(np.abs(us))


def test_kaczmarz_comparison_falls_slower_than_the_paper_relaxation():
    """Sec. 3.3 (Fig. convFactLambda): the V-cycle factor with the Kaczmarz
    comparison falls with lambda but more slowly than with the paper's
    relaxation; at lambda = 5 the cycle converges."""
    P, n, nc = inputs.disk(), 65, 17
    rho = {}
    for sm in (0, 1):
        for lam in (3, 5):
            O = oracle_for(P, n, nc, smoother=sm, lam=lam, junction_solve=0, junction_sweeps=0)
            _, norms, _ = O.solve(rtol=1e-10, max_cycles=100)
            k = len(norms) - 1
            rho[sm, lam] = (norms[-1] / norms[0]) ** (1.0 / k)
    assert rho[1, 5] < rho[1, 3] < 1.0
    assert rho[0, 3] < rho[1, 3] and rho[0, 5] < rho[1, 5]


# ---------------------------------------------------------------- threads
@pytest.mark.parametrize("P,n,nc", [(inputs.flower(), 129, 33), (inputs.torus(), 33, 17)])
def test_thread_count_does_not_change_results(P, n, nc):
    """The oracle's OpenMP loops are order-independent: a solve with one
    thread and with several gives bitwise the same iterates and norms."""
    out = []
    for k in (1, 4):
        oracle.set_threads(k)
        u, norms, ok = oracle_for(P, n, nc).solve(rtol=1e-12, max_cycles=12)
        out.append((u, norms))
    oracle.set_threads(1)
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
