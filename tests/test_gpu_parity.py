"""GPU parity: the CUDA library against the FP64 oracle, element by element.

Every step of the cycle (defect, relaxation with the extra sweeps, defect
extension, composite restriction, interpolation) is compared on the same
seeded inputs, then whole solves: the converged solution must match the
oracle's converged discrete solution within 1e-10 relative max-norm over
Omega_h u Gamma_h, and the per-cycle convergence factors are compared.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1111_0983_gb300 import inputs  # noqa: E402
from helpers import level_rhs, oracle_for, problem_rhs, rel_maxdiff, set_level_rhs  # noqa: E402

PARITY = 1e-10


def _gcmg():
    from paper_1111_0983_gb300 import gcmg
    return gcmg


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    return t.detach().cpu().numpy()


def solver_for(P, n, nc, **kw):
    S = _gcmg().Solver(P.phi_grid(n), nc, **kw)
    for l in range(S.nlev):
        S.set_bc_types(l, P.bc_types(S.ghosts(l)["B"]))
    return S


def set_problem_rhs(S, P, n):
    G = S.ghosts(0)
    types = P.bc_types(G["B"])
    f = P.f_grid(n)
    g = P.g_values(G["B"], G["nu"], types)
    S.set_rhs(dev(f), dev(g))
    return f, g


CASES = [(inputs.disk(), 65, 17), (inputs.flower(), 257, 33), (inputs.star(27), 257, 33),
         (inputs.star(0), 257, 65), (inputs.torus(), 33, 17)]


# ----------------------------------------------------------------- records
@pytest.mark.parametrize("P,n,nc", CASES)
def test_ghost_records_match_oracle(P, n, nc):
    S = solver_for(P, n, nc)
    O = oracle_for(P, n, nc, rhs=False)
    assert S.nlev == O.nlev
    for l in range(S.nlev):
        assert np.array_equal(S.node_types(l) & 3, O.types(l))
        assert np.array_equal((S.node_types(l) & 4) > 0, O.band(l) > 0)
        Gs, Go = S.ghosts(l), O.ghosts(l)
        assert np.array_equal(Gs["node"], Go["node"])
        assert np.array_equal(Gs["case"], Go["case"])
        assert np.abs(Gs["B"] - Go["B"]).max(initial=0) < 1e-13
        assert np.abs(Gs["nu"] - Go["nu"]).max(initial=0) < 1e-12
        Es = S.ghost_equations(l)
        assert np.array_equal(Es["stn"], Go["stn"])
        h = 2.0 / (S.level_n(l) - 1)
        assert np.abs(Es["wD"] - Go["wD"]).max(initial=0) < 1e-12
        assert np.abs(Es["wN"] - Go["wN"]).max(initial=0) * h < 1e-12
        assert S.num_unknowns(l) == int((O.types(l) > 0).sum())
        assert np.array_equal(S.junction_zone(l), O.junction_zone(l))
        assert np.array_equal(S.junction_solve_set(l), O.junction_solve_set(l))


# -------------------------------------------------------------- each step
def zone_condition(O, l):
    """2-norm condition number of the equations the exact junction solve of
    level l solves (1 when there are none)."""
    Z = O.junction_solve_set(l).ravel().astype(bool)
    if not Z.any():
        return 1.0
    rows, cols, vals, uon = O.assemble(l)
    uon = uon.ravel()
    keep = np.zeros(uon.max() + 1, bool)
    keep[uon[Z]] = True
    m = np.full(uon.max() + 1, -1)
    m[uon[Z]] = np.arange(Z.sum())
    sel = keep[rows] & keep[cols]
    A = np.zeros((Z.sum(), Z.sum()))
    np.add.at(A, (m[rows[sel]], m[cols[sel]]), vals[sel])
    return float(np.linalg.cond(A))


@pytest.mark.parametrize("P,n,nc", CASES)
def test_cycle_steps_match_oracle(P, n, nc):
    S = solver_for(P, n, nc)
    O = oracle_for(P, n, nc, rhs=False)
    S0 = O0 = None
    if P.dim == 2:   # the same steps without the junction solve
        S0 = solver_for(P, n, nc, junction_solve=0, junction_sweeps=0)
        O0 = oracle_for(P, n, nc, rhs=False, junction_solve=0, junction_sweeps=0)
    rng = np.random.default_rng(11)
    for l in range(S.nlev - 1):
        shape, cshape = S.shape(l), S.shape(l + 1)
        T = O.types(l)
        unk = T > 0
        u = np.where(unk, rng.uniform(-1, 1, shape), 0.0)
        f = np.where(T == 1, rng.uniform(-1, 1, shape), 0.0)
        g = rng.uniform(-1, 1, O.num_ghosts(l))
        # defect
        r_d = torch.zeros(shape, dtype=torch.float64, device="cuda")
        nrm = S.defect(l, dev(u), dev(f), dev(g), r_d)
        if l == 0:
            O.set_rhs(f, g)
            r_o, nrm_o = O.defect(u, 0)
            assert rel_maxdiff(host(r_d), r_o, unk) < 1e-13
            assert abs(nrm - nrm_o) <= 1e-13 * nrm_o
        # relaxation with the extra sweeps and the junction solve: the GPU
        # applies the explicit inverse of each zone system, the oracle an LU
        # solve, so they agree to a few kappa(A_ZZ) eps; the rest of the
        # relaxation is checked at 1e-13 with the junction solve off
        u_d = dev(u)
        S.relax(l, u_d, dev(f), dev(g), True)
        u_o = O.relax(u, f, g, l, True)
        assert rel_maxdiff(host(u_d), u_o, unk) < max(1e-13, 8 * zone_condition(O, l) * 2.2e-16)
        if l == 0 and S0 is not None:
            u_d = dev(u)
            S0.relax(l, u_d, dev(f), dev(g), True)
            assert rel_maxdiff(host(u_d), O0.relax(u, f, g, l, True), unk) < 1e-13
        # extension of a defect-like field (values on unknowns)
        r = np.where(unk, rng.uniform(-1, 1, shape), 0.0)
        r_d = dev(r)
        S.extend(l, r_d)
        r_o = O.extend(r, l)
        E = O.extension(l)
        if len(E["node"]):
            assert np.abs(host(r_d).ravel()[E["node"]] - r_o.ravel()[E["node"]]).max() < 1e-14
        # composite restriction of the extended field
        fc_d = torch.zeros(cshape, dtype=torch.float64, device="cuda")
        gc_d = torch.zeros(max(S.num_ghosts(l + 1), 1), dtype=torch.float64, device="cuda")
        S.restrict(l, dev(r_o), fc_d, gc_d)
        fc_o, gc_o = O.restrict(r_o, l)
        Tc = O.types(l + 1)
        assert np.abs(host(fc_d) - fc_o)[Tc == 1].max(initial=0) < 1e-14
        assert np.abs(host(gc_d)[: len(gc_o)] - gc_o).max(initial=0) < 1e-14
        # interpolation
        ec = np.where(Tc > 0, rng.uniform(-1, 1, cshape), 0.0)
        out_d = torch.zeros(shape, dtype=torch.float64, device="cuda")
        S.prolong(l, dev(ec), out_d)
        assert np.abs(host(out_d) - O.prolong(ec, l)).max() < 1e-14


# --------------------------------------------------------------- solves
def oracle_solution(P, n, nc, **kw):
    O = oracle_for(P, n, nc, **kw)
    u, norms, ok = O.solve(rtol=1e-13, max_cycles=60)
    return O, u, norms


@pytest.mark.parametrize("P,n,nc,kw", [(inputs.disk(), 65, 17, {}),
                                       (inputs.flower(), 257, 33, {}),
                                       (inputs.flower(), 257, 33, {"gamma": 2}),
                                       (inputs.flower(), 257, 33, {"junction_sweeps": 0, "junction_solve": 0}),
                                       (inputs.flower(), 257, 33, {"junction_sweeps": 40, "junction_solve": 0}),
                                       (inputs.star(167), 1025, 33, {"rtol": 4e-11}),
                                       (inputs.star(0), 257, 65, {}),
                                       (inputs.star(2), 257, 33, {}),
                                       (inputs.torus(), 33, 17, {"junction_radius": 3.0}),
                                       (inputs.torus(), 65, 17, {})])
def test_solve_matches_oracle(P, n, nc, kw):
    # rtol 1e-11 except at 1025^2, where the FP64 defect of any FP64 vector is
    # about 2.6e-11 of ||(f, g)|| (rounding of u times 8 / h^2)
    kw = dict(kw)
    rtol = kw.pop("rtol", 1e-11)
    S = solver_for(P, n, nc, rtol=rtol, max_cycles=200, **kw)
    set_problem_rhs(S, P, n)
    u = torch.zeros(S.shape(0), dtype=torch.float64, device="cuda")
    st = S.solve(u)
    O, u_o, norms = oracle_solution(P, n, nc, **kw)
    T = O.types(0)
    assert st["converged"], st["rel"]
    assert rel_maxdiff(host(u), u_o, T > 0) < PARITY
    assert np.all(host(u)[T == 0] == 0)
    # per-cycle convergence factors beside the oracle's (same algorithm)
    k = min(6, st["cycles"], len(norms) - 1)
    rel_o = norms[: k + 1] / norms[0]
    # rounding differs by summation order: about 1e-13 of ||r0|| per cycle
    assert np.allclose(st["rel"][1: k + 1], rel_o[1: k + 1], rtol=1e-6, atol=1e-11), (st["rel"][: k + 1], rel_o)


@pytest.mark.parametrize("P,n,nc", [(inputs.flower(), 257, 33), (inputs.torus(), 65, 17),
                                    (inputs.disk(), 65, 17)])
def test_mixed_precision_refinement_matches_oracle(P, n, nc):
    S = solver_for(P, n, nc, rtol=1e-11, max_cycles=200, precision=1)
    set_problem_rhs(S, P, n)
    u = torch.zeros(S.shape(0), dtype=torch.float64, device="cuda")
    st = S.solve(u)
    assert st["converged"], st["rel"]
    O, u_o, _ = oracle_solution(P, n, nc)
    T = O.types(0)
    assert rel_maxdiff(host(u), u_o, T > 0) < PARITY
    # residual measured by the oracle (FP64) on the GPU's solution
    f, g = problem_rhs(O, P, n)
    O.set_rhs(f, g)
    _, rn = O.defect(host(u))
    assert rn <= 2e-11 * st["r0_norm"]


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_solve_start(precision):
    """A graph solve computes ||(f, g)|| and the first defect on the device and
    opens its loop there: r0, rel[0], the cycles and the solution equal those of
    the launch-by-launch loop (kernel timing on); a start that already meets the
    tolerance runs no cycle and leaves u as it was; a zero right-hand side
    returns at once with u = 0."""
    P, n, nc = inputs.flower(), 129, 33
    S = solver_for(P, n, nc, precision=precision, rtol=1e-10, max_cycles=100)
    f, g = set_problem_rhs(S, P, n)
    u = torch.zeros(S.shape(0), dtype=torch.float64, device="cuda")
    st = S.solve(u)
    S.set_kernel_timing(S.KERNEL_SMOOTH)
    u2 = torch.zeros_like(u)
    st2 = S.solve(u2)
    S.set_kernel_timing(-1)
    assert st["converged"] and st2["converged"]
    assert st["r0_norm"] == st2["r0_norm"] > 0 and st["rel"][0] == st2["rel"][0] == 1.0
    assert st["cycles"] == st2["cycles"] > 0
    assert np.array_equal(host(u), host(u2))
    u3 = u.clone()
    st3 = S.solve(u3)
    assert st3["converged"] and st3["cycles"] == 0 and st3["rel"][0] <= 1e-10
    assert torch.equal(u3, u)
    S.set_rhs(dev(np.zeros_like(f)), dev(np.zeros_like(g)))
    u4 = torch.zeros_like(u)
    st4 = S.solve(u4)
    assert st4["converged"] and st4["cycles"] == 0 and st4["r0_norm"] == 0.0
    assert not torch.any(u4)


@pytest.mark.parametrize("precision", [0, 1])
def test_max_cycles_split_solve(precision):
    """gcmg_set_max_cycles changes the limit of a captured graph solve: one
    cycle, then a solve from its result, gives the cycles and the solution of
    one uninterrupted solve (a solve's state between cycles is u alone)."""
    P, n, nc = inputs.flower(), 129, 33
    S = solver_for(P, n, nc, precision=precision, rtol=1e-10, max_cycles=100)
    set_problem_rhs(S, P, n)
    u = torch.zeros(S.shape(0), dtype=torch.float64, device="cuda")
    st = S.solve(u)
    S.set_max_cycles(1)
    u1 = torch.zeros_like(u)
    st1 = S.solve(u1)
    assert st1["cycles"] == 1 and not st1["converged"] and st1["rel"][1] == st["rel"][1]
    S.set_max_cycles(100)
    st2 = S.solve(u1)
    assert st2["converged"] and st1["cycles"] + st2["cycles"] == st["cycles"]
    assert rel_maxdiff(host(u1), host(u), np.ones(u.shape, bool)) < 1e-14
    with pytest.raises(_gcmg().GcmgError):
        S.set_max_cycles(0)


def test_solve_host_equals_device():
    P, n, nc = inputs.flower(), 257, 33
    S = solver_for(P, n, nc)
    f, g = set_problem_rhs(S, P, n)
    u = torch.zeros(S.shape(0), dtype=torch.float64, device="cuda")
    st = S.solve(u)
    uh, sth = S.solve_host(f, g)
    assert np.array_equal(uh, host(u))
    assert sth["cycles"] == st["cycles"]


@pytest.mark.parametrize("P,n,nc", [(inputs.flower(), 257, 33), (inputs.torus(), 65, 17)])
@pytest.mark.parametrize("pinned", [True, False])
def test_solve_host_uses_f_on_the_inside_nodes_only(P, n, nc, pinned):
    """gcmg_solve_host with f NaN off Omega_h and stale device values from an
    earlier right-hand side: page-locked f is read by the device at the
    inside nodes only and page-locked u stored by the device, other host
    memory is copied whole; either way the solution is bitwise the device
    solve's."""
    S = solver_for(P, n, nc)
    f, g = set_problem_rhs(S, P, n)
    u = torch.zeros(S.shape(0), dtype=torch.float64, device="cuda")
    st = S.solve(u)
    T = S.node_types(0) & 3
    f_nan = np.where(T == 1, f, np.nan)
    S.set_rhs(dev(np.full_like(f, 7.0)), dev(g))
    if pinned:
        fh = torch.from_numpy(f_nan).pin_memory().numpy()
        gh = torch.from_numpy(np.ascontiguousarray(g)).pin_memory().numpy()
        uh = torch.empty(S.shape(0), dtype=torch.float64).pin_memory().numpy()
    else:
        fh, gh, uh = f_nan, np.ascontiguousarray(g), np.empty(S.shape(0))
    out, sth = S.solve_host(fh, gh, uh)
    assert sth["converged"] and sth["cycles"] == st["cycles"]
    assert np.array_equal(out, host(u))


def test_boundary_block_timing():
    """Timing the boundary blocks (every level) leaves the result bit for bit
    unchanged, times every launch of every relaxation, and reports bytes."""
    P, n, nc = inputs.flower(), 257, 33
    S = solver_for(P, n, nc, precision=1)
    set_problem_rhs(S, P, n)
    u = torch.zeros(S.shape(0), dtype=torch.float64, device="cuda")
    st = S.solve(u)
    ut = torch.zeros_like(u)
    S.set_kernel_timing(S.KERNEL_BOUNDARY)
    stt = S.solve(ut)
    launches, ms, nbytes = S.kernel_timing_ex()
    S.set_kernel_timing(-1)
    assert stt["cycles"] == st["cycles"]
    assert torch.equal(u, ut)
    per_cycle = 3 * (S.nlev - 1)     # nu1 + nu2 relaxations on every level above the coarsest
    assert launches == st["cycles"] * per_cycle
    assert ms > 0 and nbytes > 0
    # every launch reads and writes at least each band node of its level (FP32)
    band = [int(((S.node_types(l) & 4) > 0).sum()) for l in range(S.nlev - 1)]
    assert nbytes >= st["cycles"] * 3 * sum(2 * 4 * b for b in band)


@pytest.mark.parametrize("P,n,nc,nu", [(inputs.disk(), 129, 17, 2), (inputs.flower(), 257, 33, 2),
                                       (inputs.star(3), 257, 33, 1), (inputs.torus(), 65, 17, 1)])
def test_fmg_matches_oracle(P, n, nc, nu):
    """Full multigrid (plain FP64): the fine result equals the oracle's element
    by element (same steps, summation order and the junction solve's explicit
    inverse against LU aside)."""
    S = solver_for(P, n, nc, precision=0)
    set_problem_rhs(S, P, n)
    O = oracle_for(P, n, nc)
    for l in range(1, S.nlev):
        f, g = level_rhs(O, P, l)
        S.set_rhs_level(l, dev(f), dev(g))
    u = torch.zeros(S.shape(0), dtype=torch.float64, device="cuda")
    S.fmg(nu, u)
    set_level_rhs(O, P)
    uo = O.fmg(nu)
    assert rel_maxdiff(host(u), uo, O.types(0) > 0) < 1e-9


def test_fmg_needs_plain_fp64():
    gcmg = _gcmg()
    P, n = inputs.disk(), 65
    S = solver_for(P, n, 17, precision=1)
    set_problem_rhs(S, P, n)
    u = torch.zeros(S.shape(0), dtype=torch.float64, device="cuda")
    with pytest.raises(gcmg.GcmgError) as e:
        S.fmg(1, u)
    assert e.value.status == gcmg.GCMG_E_STATE


def _ellipse_phi(dim, n):
    """The paper's rotated ellipse (Sec. 3.3, not a distance function); in 3D an
    ellipsoid with the same profile."""
    X = inputs.coords(dim, n)
    c, s = math.cos(math.pi / 6), math.sin(math.pi / 6)
    xr, yr = c * X[0] - s * X[1], s * X[0] + c * X[1]
    phi = (xr - math.sqrt(2) / 20) ** 2 / 0.563 ** 2 + (yr - math.sqrt(3) / 30) ** 2 / 0.263 ** 2 - 1
    if dim == 3:
        phi = phi + X[2] ** 2 / 0.4 ** 2
    return np.ascontiguousarray(phi)


@pytest.mark.parametrize("dim,n,steps", [(2, 129, 20), (2, 65, 7), (2, 65, 0), (3, 33, 12)])
def test_reinit_matches_oracle(dim, n, steps):
    gcmg = _gcmg()
    phi0 = _ellipse_phi(dim, n)
    out = host(gcmg.reinit(dev(phi0), steps))
    ref = oracle.reinit(phi0, steps)
    assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.array_equal(np.sign(out), np.sign(phi0))


def test_reinit_arguments():
    gcmg = _gcmg()
    lib = gcmg.lib()
    phi = dev(_ellipse_phi(2, 33))
    assert lib.gcmg_reinit(4, 33, gcmg._ptr(phi), 3, gcmg._ptr(torch.empty_like(phi)), None) == gcmg.GCMG_E_ARG
    assert lib.gcmg_reinit(2, 33, gcmg._ptr(phi), 3, gcmg._ptr(phi), None) == gcmg.GCMG_E_ARG


def test_reinitialised_ellipse_solve_matches_oracle():
    """End to end: the ellipse level set reinitialised on the GPU, the
    hierarchy built on it, solved to 1e-10, equals the oracle's solution on
    its own reinitialisation of the same level set."""
    gcmg = _gcmg()
    n, nc = 257, 33
    phi0 = _ellipse_phi(2, n)
    phi = host(gcmg.reinit(dev(phi0), 20))
    P = inputs.circle_paper()   # its u, f and its D/N split (Neumann where B_x > 0)
    S = gcmg.Solver(phi, nc, rtol=1e-11, max_cycles=200)
    O = oracle.Oracle(oracle.reinit(phi0, 20), nc)
    for l in range(S.nlev):
        S.set_bc_types(l, P.bc_types(S.ghosts(l)["B"]))
        O.set_bc(l, P.bc_types(O.ghosts(l)["B"]))
    for T in (S, O):
        G = T.ghosts(0)
        f, g = P.f_grid(n), P.g_values(G["B"], G["nu"], P.bc_types(G["B"]))
        if T is S:
            T.set_rhs(dev(f), dev(g))
        else:
            T.set_rhs(f, g)
    u = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    st = S.solve(u)
    assert st["converged"]
    uo = O.solve(np.zeros((n, n)), rtol=1e-12, max_cycles=200)[0]
    assert np.array_equal(S.node_types(0) & 3, O.types(0))
    assert rel_maxdiff(host(u), uo, O.types(0) > 0) < PARITY


def test_errors_are_reported():
    gcmg = _gcmg()
    X = inputs.coords(2, 65)
    with pytest.raises(gcmg.GcmgError) as e:
        gcmg.Solver(np.hypot(X[0], X[1]) - 0.995, 17)
    assert e.value.status == gcmg.GCMG_E_GEOM
    with pytest.raises(gcmg.GcmgError) as e:
        gcmg.Solver(np.hypot(X[0], X[1]) - 0.5, 13)      # 64 is not 12 * 2^k
    assert e.value.status == gcmg.GCMG_E_ARG
    S = gcmg.Solver(np.hypot(X[0], X[1]) - 0.5, 17)
    u = torch.zeros((65, 65), dtype=torch.float64, device="cuda")
    with pytest.raises(gcmg.GcmgError) as e:
        S.solve(u)                                        # no right-hand side yet
    assert e.value.status == gcmg.GCMG_E_STATE


def test_nan_rhs_reports_noconv():
    P, n, nc = inputs.disk(), 65, 17
    S = solver_for(P, n, nc, max_cycles=5)
    f = P.f_grid(n)
    f[32, 32] = np.nan
    G = S.ghosts(0)
    S.set_rhs(dev(f), dev(P.g_values(G["B"], G["nu"], P.bc_types(G["B"]))))
    u = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    st = S.solve(u)
    assert not st["converged"]


@pytest.mark.parametrize("P,n,nc", [(inputs.flower(), 1025, 33), (inputs.star(27), 257, 33),
                                    (inputs.disk(), 65, 17)])
def test_fused_coarse_cycle_equals_per_level_launches(P, n, nc):
    """The coarse end of the FP32 V-cycle in one cluster launch runs the same
    steps in the same order as one launch per step: the same solution bit for
    bit and the same residual history."""
    sols, hists = [], []
    for fused in (0, 257):
        S = solver_for(P, n, nc, rtol=1e-10, max_cycles=100, precision=1, fused_coarse_n=fused)
        set_problem_rhs(S, P, n)
        u = torch.zeros(S.shape(0), dtype=torch.float64, device="cuda")
        st = S.solve(u)
        assert st["converged"]
        sols.append(host(u))
        hists.append(st["rel"])
        S.close()
    assert np.array_equal(sols[0], sols[1])
    assert np.array_equal(hists[0], hists[1])


# ------------------------------------------------ Kaczmarz comparison (Sec. 3.3)
KACZ = dict(smoother=1, junction_solve=0, junction_sweeps=0)


def test_kaczmarz_relaxation_matches_oracle():
    """The Kaczmarz comparison smoother (Sec. 3.3), plain FP64: one relaxation
    (Gauss-Seidel over the inside nodes, then lambda Kaczmarz sweeps over the
    ghosts and the band's inside nodes, colour by colour) on every level equals
    the oracle's element by element."""
    P, n, nc = inputs.disk(), 65, 17
    S = solver_for(P, n, nc, **KACZ)
    O = oracle_for(P, n, nc, rhs=False, **KACZ)
    rng = np.random.default_rng(5)
    for l in range(S.nlev - 1):
        shape = S.shape(l)
        T = O.types(l)
        unk = T > 0
        u = np.where(unk, rng.uniform(-1, 1, shape), 0.0)
        f = np.where(T == 1, rng.uniform(-1, 1, shape), 0.0)
        g = rng.uniform(-1, 1, O.num_ghosts(l))
        u_d = dev(u)
        S.relax(l, u_d, dev(f), dev(g), True)
        assert rel_maxdiff(host(u_d), O.relax(u, f, g, l, True), unk) < 1e-12, l


def test_kaczmarz_solve_matches_oracle():
    """V-cycles with the Kaczmarz comparison smoother: the converged solution
    matches the oracle's within 1e-10 and the per-cycle factors match; the
    factor is reported beside the paper relaxation's (it falls more slowly
    with lambda, Sec. 3.3)."""
    import time
    P, n, nc = inputs.disk(), 65, 17
    S = solver_for(P, n, nc, rtol=1e-11, max_cycles=200, **KACZ)
    set_problem_rhs(S, P, n)
    u = torch.zeros(S.shape(0), dtype=torch.float64, device="cuda")
    st = S.solve(u)
    O, u_o, norms = oracle_solution(P, n, nc, **KACZ)
    T = O.types(0)
    assert st["converged"], st["rel"]
    assert rel_maxdiff(host(u), u_o, T > 0) < PARITY
    k = min(6, st["cycles"], len(norms) - 1)
    rel_o = norms[: k + 1] / norms[0]
    assert np.allclose(st["rel"][1: k + 1], rel_o[1: k + 1], rtol=1e-6, atol=1e-11)
    for sm, kw in (("kaczmarz", KACZ), ("paper", dict(junction_solve=0, junction_sweeps=0))):
        for lam in (3, 5):
            S2 = solver_for(P, n, nc, rtol=1e-10, max_cycles=200, lam=lam, **kw)
            set_problem_rhs(S2, P, n)
            u2 = torch.zeros_like(u)
            S2.solve(u2)
            u2.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s2 = S2.solve(u2)
            ms = (time.perf_counter() - t0) * 1e3
            rho = s2["rel"][-1] ** (1.0 / s2["cycles"])
            print(f"disk 65^2 FP64 {sm} lambda={lam}: cycles {s2['cycles']} rho {rho:.3f} {ms:.2f} ms")


def test_kaczmarz_needs_plain_fp64_2d():
    gcmg = _gcmg()
    for P, n, nc, kw in ((inputs.disk(), 65, 17, dict(smoother=1)),
                         (inputs.disk(), 65, 17, dict(KACZ, precision=1)),
                         (inputs.torus(), 33, 17, dict(KACZ))):
        with pytest.raises(gcmg.GcmgError) as e:
            solver_for(P, n, nc, **kw)
        assert e.value.status == gcmg.GCMG_E_ARG
