"""The 3D boundary relaxation as one launch (the ghost sweep, the lambda band
sweeps of Sec. 3.2 and the junction sweeps, with grid-wide barriers between
the phases) against the same phases launched one by one, and its bounded
barrier waits: made to run out from the host, the solve reports
GCMG_E_TIMEOUT and the context stays usable."""
import numpy as np
import pytest

from paper_1111_0983_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _solver(precision, n=65, **kw):
    from paper_1111_0983_gb300 import gcmg
    P = inputs.torus()
    S = gcmg.Solver(P.phi_grid(n), 17, precision=precision, rtol=1e-11, max_cycles=100, **kw)
    for l in range(S.nlev):
        S.set_bc_types(l, P.bc_types(S.ghosts(l)["B"]))
    G = S.ghosts(0)
    g = P.g_values(G["B"], G["nu"], P.bc_types(G["B"]))
    S.set_rhs(torch.from_numpy(P.f_grid(n)).cuda(), torch.from_numpy(g).cuda())
    return S


@pytest.mark.parametrize("precision,n", [(0, 65), (1, 65), (1, 129)])
def test_one_launch_equals_one_launch_per_phase(precision, n):
    """Same arithmetic in the same order: bitwise equal solutions and
    per-cycle residuals whether the boundary phases run as one launch each
    (the default), as thread-block clusters or as one grid with software
    barriers, with and without junction sweeps on global lists."""
    S = _solver(precision, n)
    runs = []
    for mode in (0, 1, 2):
        S.set_boundary3d(mode)
        u = torch.zeros((n,) * 3, dtype=torch.float64, device="cuda")
        runs.append((u, S.solve(u)))
    for u, st in runs:
        assert st["converged"]
        assert torch.equal(u, runs[0][0])
        np.testing.assert_array_equal(st["rel"], runs[0][1]["rel"])
    # the single relaxation of the step API takes the same paths
    S.set_boundary3d(1)
    P = inputs.torus()
    rng = np.random.default_rng(5)
    T = torch.from_numpy(S.node_types(0) & 3 > 0).cuda()
    u = torch.from_numpy(rng.standard_normal((n,) * 3)).cuda() * T
    f = torch.from_numpy(P.f_grid(n)).cuda()
    G = S.ghosts(0)
    g = torch.from_numpy(P.g_values(G["B"], G["nu"], P.bc_types(G["B"]))).cuda()
    a = u.clone()
    S.relax(0, a, f, g)
    S.set_boundary3d(0)
    b = u.clone()
    S.relax(0, b, f, g)
    assert torch.equal(a, b)
    S.set_boundary3d(2)
    c = u.clone()
    S.relax(0, c, f, g)
    assert torch.equal(a, c)


def test_barrier_wait_runs_out_and_context_stays_usable():
    from paper_1111_0983_gb300 import gcmg
    S = _solver(1)
    u = torch.zeros((65,) * 3, dtype=torch.float64, device="cuda")
    S.debug_barrier(enable=True, phantom_blocks=1, spin_limit=2000)
    with pytest.raises(gcmg.GcmgError) as e:
        S.solve(u)
    assert e.value.status == gcmg.GCMG_E_TIMEOUT
    S.debug_barrier(enable=True)
    u.zero_()
    st = S.solve(u)
    assert st["converged"]
    S2 = _solver(1)                  # default: one launch a phase
    u2 = torch.zeros_like(u)
    S2.solve(u2)
    assert torch.equal(u, u2)


@pytest.mark.parametrize("precision,n", [(0, 65), (1, 129), (1, 257)])
def test_sweep_kernels_agree_bitwise(precision, n):
    """The 3D interior sweeps -- the two one-colour launches over row
    segments (the default), the fused sweep over row spans (FP32), the planes
    in registers and the planes staged in shared memory -- compute the same
    sums in the same order: bitwise equal solves, also with the row-span items
    rebuilt for every lane width and for short items."""
    S = _solver(precision, n)
    if precision == 1:
        items, cols = S.span3d_info(0)
        assert items > 0 and 2 <= cols <= 5
    u1 = torch.zeros((n,) * 3, dtype=torch.float64, device="cuda")
    st1 = S.solve(u1)
    assert st1["converged"]
    variants = [("sweep", 1), ("sweep", 0), ("sweep", 2)]
    if precision == 1:
        variants += [("span", (2, 7)), ("span", (3, 32)), ("span", (5, 1)), ("span", (0, 0))]
    for kind, arg in variants:
        if kind == "sweep":
            S.set_sweep3d(arg)
        else:
            S.set_sweep3d(2)
            S.set_span3d(*arg)
            if arg[0]:
                assert S.span3d_info(0)[1] == arg[0]
        u2 = torch.zeros_like(u1)
        st2 = S.solve(u2)
        assert st2["converged"], (kind, arg)
        assert torch.equal(u1, u2), (kind, arg)
        np.testing.assert_array_equal(st1["rel"], st2["rel"])


@pytest.mark.parametrize("precision,n", [(1, 257)])
def test_junction_blocks_equal_global_junction_sweeps(precision, n):
    """The junction zone relaxed in overlapping shared-memory blocks (each
    updating the zone within 4 mu nodes of its block, writing back its own
    nodes) gives bitwise the solve of the global junction sweeps (FP32
    cycles: the blocks of the finest level fit in shared memory)."""
    S = _solver(precision, n)
    S.set_junction_blocks(True)
    modes = [S.junction_mode(l) for l in range(S.nlev)]
    assert 2 in modes, modes
    u1 = torch.zeros((n,) * 3, dtype=torch.float64, device="cuda")
    st1 = S.solve(u1)
    S.set_junction_blocks(False)
    assert 2 not in [S.junction_mode(l) for l in range(S.nlev)]
    u2 = torch.zeros_like(u1)
    st2 = S.solve(u2)
    assert st1["converged"] and st2["converged"]
    assert torch.equal(u1, u2)
    np.testing.assert_array_equal(st1["rel"], st2["rel"])
