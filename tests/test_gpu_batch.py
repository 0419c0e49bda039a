"""Batched solves: many star domains of uneven sizes in one graph launch.

Each domain's converged solution must equal the single-domain solver's and
the FP64 oracle's converged discrete solution within 1e-10 relative max-norm;
every strip height of the fused sweep gives the same result; the autotuner picks
one of them.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1111_0983_gb300 import inputs  # noqa: E402
from helpers import oracle_for, rel_maxdiff  # noqa: E402

PARITY = 1e-10


def make_batch(ids, sizes, nc=33, **kw):
    from paper_1111_0983_gb300 import gcmg
    probs = [inputs.star(i) for i in ids]
    B = gcmg.Batch([P.phi_grid(n) for P, n in zip(probs, sizes)], nc, rtol=1e-11, max_cycles=100, **kw)
    rhs = []
    for S, P, n in zip(B.domains, probs, sizes):
        for l in range(S.nlev):
            S.set_bc_types(l, P.bc_types(S.ghosts(l)["B"]))
        G = S.ghosts(0)
        f = P.f_grid(n)
        g = P.g_values(G["B"], G["nu"], P.bc_types(G["B"]))
        S.set_rhs(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda())
        rhs.append((f, g))
    return B, probs, rhs


def test_batch_matches_single_domain_and_oracle():
    from paper_1111_0983_gb300 import gcmg
    ids, sizes = [0, 1, 2, 3, 5, 8], [129, 257, 129, 257, 129, 257]
    B, probs, rhs = make_batch(ids, sizes)
    stats, steps = B.solve()
    assert all(s["converged"] for s in stats), [s["rel_residual"] for s in stats]
    for k, (P, n) in enumerate(zip(probs, sizes)):
        u = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        B.solution(k, u)
        ub = u.cpu().numpy()
        S = gcmg.Solver(P.phi_grid(n), 33, precision=1, rtol=1e-11, max_cycles=100)
        for l in range(S.nlev):
            S.set_bc_types(l, P.bc_types(S.ghosts(l)["B"]))
        f, g = rhs[k]
        S.set_rhs(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda())
        us = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        st = S.solve(us)
        assert st["converged"]
        T = (S.node_types(0) & 3) > 0
        assert rel_maxdiff(ub, us.cpu().numpy(), T) < PARITY, k
        if k < 2:
            O = oracle_for(P, n, 33)
            uo, _, _ = O.solve(rtol=1e-13, max_cycles=60)
            assert rel_maxdiff(ub, uo, T) < PARITY, k
        S.close()
    B.close()


def test_batch_strip_heights_agree_and_autotune():
    ids, sizes = [4, 6, 9], [257, 129, 257]
    B, probs, _ = make_batch(ids, sizes)
    sols = []
    for v in range(3):
        B.set_tiles(v)
        stats, steps = B.solve()
        assert all(s["converged"] for s in stats)
        sols.append([])
        for k, n in enumerate(sizes):
            u = torch.zeros((n, n), dtype=torch.float64, device="cuda")
            B.solution(k, u)
            sols[-1].append(u.cpu().numpy())
    for v in (1, 2):
        for a, b in zip(sols[0], sols[v]):
            assert np.array_equal(a, b)
    best, ms = B.autotune()
    assert best in (0, 1, 2) and all(t > 0 for t in ms)
    stats, _ = B.solve()
    assert all(s["converged"] for s in stats)
    B.close()


def test_batch_plain_launches_equal_graph():
    """The plain-launch form of a batched solve (for profilers) runs the same
    kernels: the same steps and bit-identical solutions."""
    ids, sizes = [4, 9], [257, 129]
    B, probs, _ = make_batch(ids, sizes)
    out = []
    for graph in (True, False):
        B.set_graph(graph)
        stats, steps = B.solve()
        assert all(s["converged"] for s in stats)
        sols = []
        for k, n in enumerate(sizes):
            u = torch.zeros((n, n), dtype=torch.float64, device="cuda")
            B.solution(k, u)
            sols.append(u.cpu().numpy())
        out.append((steps, sols))
    assert out[0][0] == out[1][0]
    for a, b in zip(out[0][1], out[1][1]):
        assert np.array_equal(a, b)
    B.close()


def test_batch_w_cycle_matches_single_domain_and_oracle():
    """W-cycles (gamma = 2) in a batch of domains with the same number of
    levels: the solution of each domain equals a single domain's W-cycle solve
    and the oracle's, with about as many steps; domains with different numbers
    of levels are refused."""
    from paper_1111_0983_gb300 import gcmg
    with pytest.raises(gcmg.GcmgError) as e:
        make_batch([0, 1], [129, 257], gamma=2)
    assert e.value.status == gcmg.GCMG_E_ARG
    ids, sizes = [1, 3, 8], [257, 257, 257]
    B, probs, rhs = make_batch(ids, sizes, gamma=2)
    stats, steps = B.solve()
    assert all(s["converged"] for s in stats), [s["rel_residual"] for s in stats]
    for k, (P, n) in enumerate(zip(probs, sizes)):
        u = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        B.solution(k, u)
        ub = u.cpu().numpy()
        S = gcmg.Solver(P.phi_grid(n), 33, precision=1, gamma=2, rtol=1e-11, max_cycles=100)
        for l in range(S.nlev):
            S.set_bc_types(l, P.bc_types(S.ghosts(l)["B"]))
        f, g = rhs[k]
        S.set_rhs(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda())
        us = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        st = S.solve(us)
        assert st["converged"] and abs(st["cycles"] - stats[k]["cycles"]) <= 1
        T = (S.node_types(0) & 3) > 0
        assert rel_maxdiff(ub, us.cpu().numpy(), T) < PARITY, k
        if k == 0:
            O = oracle_for(P, n, 33, gamma=2)
            uo, _, _ = O.solve(rtol=1e-13, max_cycles=60)
            assert rel_maxdiff(ub, uo, T) < PARITY
        S.close()
    B.close()
