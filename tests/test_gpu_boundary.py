"""GPU tests of the boundary calls that follow the paper's problem statement
(Sec. 2.1, Eq. mainpr; Sec. 2.3): the Dirichlet/Neumann mask, a grid with its
own spacing and origin, the residual of a given u, and the stop on a diverging
cycle."""
import numpy as np
import pytest

import oracle
from helpers import oracle_for, problem_rhs
from paper_1111_0983_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _gcmg():
    from paper_1111_0983_gb300 import gcmg
    return gcmg


def _nearest_mask_types(S, l, mask, h0, origin):
    """Host reading of the mask rule: the fine node nearest B, ties to G."""
    G = S.ghosts(l)
    n0 = mask.shape[0]
    nl = S.level_n(l)
    step = (n0 - 1) // (nl - 1)
    idx = np.zeros(len(G["node"]), np.int64)
    for a in range(S.dim):
        x = (G["B"][:, a] - origin[a]) / h0
        fl = np.floor(x)
        fr = x - fl
        g = (np.unravel_index(G["node"], (nl,) * S.dim)[a] * step).astype(float)
        j = fl + (fr > 0.5)
        j = np.where(fr == 0.5, np.where(g > x, fl + 1, fl), j)
        idx = idx * n0 + np.clip(j, 0, n0 - 1).astype(np.int64)
    return (mask.ravel()[idx] != 0).astype(np.uint8)


@pytest.mark.parametrize("P,n,nc", [(inputs.flower(), 257, 33), (inputs.torus(), 65, 17)])
def test_mask_gives_the_types_of_the_nearest_node_and_the_same_solve(P, n, nc):
    gcmg = _gcmg()
    X = inputs.coords(P.dim, n)
    pts = np.stack([x.ravel() for x in X], axis=1)
    mask = P.is_neumann(pts).reshape((n,) * P.dim).astype(np.uint8)
    A = gcmg.Solver(P.phi_grid(n), nc)
    A.set_bc_types_from_mask(torch.from_numpy(mask).cuda())
    B = gcmg.Solver(P.phi_grid(n), nc)
    h0 = 2.0 / (n - 1)
    differ = 0
    for l in range(A.nlev):
        want = _nearest_mask_types(A, l, mask, h0, [-1.0] * P.dim)
        np.testing.assert_array_equal(A.bc_types(l), want)
        B.set_bc_types(l, want)
        differ += int((want != P.bc_types(A.ghosts(l)["B"])).sum())
    # the analytic split and the nearest-node mask disagree only next to the split
    assert differ <= 0.02 * sum(A.num_ghosts(l) for l in range(A.nlev))
    G = A.ghosts(0)
    g = P.g_values(G["B"], G["nu"], A.bc_types(0))
    f = torch.from_numpy(P.f_grid(n)).cuda()
    g = torch.from_numpy(g).cuda()
    ua = torch.zeros((n,) * P.dim, dtype=torch.float64, device="cuda")
    ub = torch.zeros_like(ua)
    A.set_rhs(f, g)
    B.set_rhs(f, g)
    sa, sb = A.solve(ua), B.solve(ub)
    assert sa["converged"] and sb["converged"]
    assert torch.equal(ua, ub)


def test_grid_spacing_and_origin_scale_the_problem():
    """x' = 3x + 0.5 maps the flower problem on [-1,1]^2 to a grid of spacing
    3h and origin -2.5: with phi' = 3 phi, f' = f / 9, g_D' = g_D and
    g_N' = g_N / 3 the discrete system is the same (Eqs. discr, clpt, dir2d,
    neu2d are invariant under the scaling), so the solutions agree to
    rounding; B' = 3 B + 0.5."""
    gcmg = _gcmg()
    P, n, nc = inputs.flower(), 257, 33
    h = 2.0 / (n - 1)
    A = gcmg.Solver(P.phi_grid(n), nc, rtol=1e-11)
    S = gcmg.Solver(3.0 * P.phi_grid(n), nc, grid=(3.0 * h, (-2.5, -2.5)), rtol=1e-11)
    for l in range(A.nlev):
        Ba, Bs = A.ghosts(l)["B"], S.ghosts(l)["B"]
        np.testing.assert_allclose(Bs, 3.0 * Ba + 0.5, rtol=0, atol=1e-12)
        t = P.bc_types(Ba)
        A.set_bc_types(l, t)
        S.set_bc_types(l, t)
    G = A.ghosts(0)
    t = P.bc_types(G["B"])
    g = P.g_values(G["B"], G["nu"], t)
    gs = np.where(t == 1, g / 3.0, g)
    A.set_rhs(torch.from_numpy(P.f_grid(n)).cuda(), torch.from_numpy(g).cuda())
    S.set_rhs(torch.from_numpy(P.f_grid(n) / 9.0).cuda(), torch.from_numpy(gs).cuda())
    ua = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    us = torch.zeros_like(ua)
    assert A.solve(ua)["converged"] and S.solve(us)["converged"]
    T = torch.from_numpy(A.node_types(0) & 3 > 0).cuda()
    rel = float((ua - us).abs()[T].max() / ua.abs()[T].max())
    assert rel < 1e-10, rel


@pytest.mark.parametrize("precision", [0, 1])
def test_residual_of_a_solution_and_of_zero(precision):
    gcmg = _gcmg()
    P, n, nc = inputs.flower(), 257, 33
    S = gcmg.Solver(P.phi_grid(n), nc, precision=precision, rtol=1e-10)
    for l in range(S.nlev):
        S.set_bc_types(l, P.bc_types(S.ghosts(l)["B"]))
    G = S.ghosts(0)
    f = torch.from_numpy(P.f_grid(n)).cuda()
    g = torch.from_numpy(P.g_values(G["B"], G["nu"], P.bc_types(G["B"]))).cuda()
    S.set_rhs(f, g)
    u = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    r = torch.empty_like(u)
    assert S.residual(u, r) == pytest.approx(1.0, rel=0, abs=0)   # r0 = (f, g)
    st = S.solve(u)
    assert st["converged"]
    rel = S.residual(u, r)
    assert rel == pytest.approx(st["rel_residual"], rel=1e-12)
    # the same defect as the single-step call on the caller's f and g
    r2 = torch.empty_like(u)
    S.defect(0, u, f, g, r2)
    assert torch.equal(r, r2)
    # and the oracle's defect of the same u (its own discretisation)
    O = oracle_for(P, n, nc)
    ro, nrm = O.defect(u.cpu().numpy(), 0)
    ff, gg = problem_rhs(O, P, n)
    T = O.types(0) > 0
    r0 = max(np.abs(ff[O.types(0) == 1]).max(), np.abs(gg).max())
    assert abs(nrm / r0 - rel) < 5e-12   # summation order: ~1e-13 of ||(f, g)|| per row


@pytest.mark.parametrize("plain", [False, True])
def test_diverging_cycle_stops_with_noconv(plain):
    """Star 0 at 257^2 without the junction relaxation: the paper's V-cycle
    diverges there (the oracle's factor exceeds 1).  The solve stops once the
    defect has grown in 3 consecutive cycles, long before max_cycles, and
    reports GCMG_E_NOCONV with diverged set."""
    gcmg = _gcmg()
    P, n, nc = inputs.star(0), 257, 65
    S = gcmg.Solver(P.phi_grid(n), nc, precision=0, junction_solve=0, junction_sweeps=0, max_cycles=200)
    for l in range(S.nlev):
        S.set_bc_types(l, P.bc_types(S.ghosts(l)["B"]))
    G = S.ghosts(0)
    S.set_rhs(torch.from_numpy(P.f_grid(n)).cuda(),
              torch.from_numpy(P.g_values(G["B"], G["nu"], P.bc_types(G["B"]))).cuda())
    if plain:
        S.set_kernel_timing(S.KERNEL_SMOOTH)   # the host-driven loop
    u = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    st = S.solve(u)
    assert not st["converged"] and st["diverged"], st
    m = st["cycles"]
    assert 3 <= m < 200
    rel = st["rel"]
    assert np.all(rel[m - 2:m + 1] > rel[m - 3:m])
    # with the check off the same solve runs on to max_cycles
    S2 = gcmg.Solver(P.phi_grid(n), nc, precision=0, junction_solve=0, junction_sweeps=0, max_cycles=m + 5,
                     diverge_cycles=0)
    for l in range(S2.nlev):
        S2.set_bc_types(l, P.bc_types(S2.ghosts(l)["B"]))
    S2.set_rhs(torch.from_numpy(P.f_grid(n)).cuda(),
               torch.from_numpy(P.g_values(G["B"], G["nu"], P.bc_types(G["B"]))).cuda())
    u.zero_()
    st2 = S2.solve(u)
    assert st2["cycles"] == m + 5 and not st2["diverged"]
