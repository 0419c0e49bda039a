"""gcmg_defect_noalloc, the allocation-free defect entry point.

It serves callers that cannot allocate device memory themselves (their device
memory belongs to another allocator, or they run in a loop that must not
synchronise the device through cudaMalloc / cudaFree): its only scratch is a
fixed array inside the library.  This test checks, through the C ABI, that two
calls in a row give the same defect and norm as gcmg_defect, the entry point
that works on a context.  The test's own buffers come from torch; the entry
point under test allocates nothing.  This file is named so that pytest
collects it after every other test file.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1111_0983_gb300 import inputs  # noqa: E402

TOL = 1e-13


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _ptr(t):
    return C.c_void_p(t.data_ptr())


@pytest.mark.parametrize("P,n,nc", [(inputs.flower(), 257, 33), (inputs.torus(), 33, 17)])
def test_noalloc_defect_matches_context_defect(P, n, nc):
    from paper_1111_0983_gb300 import gcmg
    L = gcmg.lib()
    S = gcmg.Solver(P.phi_grid(n), nc)
    for l in range(S.nlev):
        S.set_bc_types(l, P.bc_types(S.ghosts(l)["B"]))
    G = S.ghosts(0)
    bc = P.bc_types(G["B"])
    E = S.ghost_equations(0)
    w = np.where(bc[:, None] == 1, E["wN"], E["wD"])
    types = _dev(S.node_types(0))
    gnode = _dev(G["node"].astype(np.int32))
    stn = _dev(E["stn"].astype(np.int32))
    wd = _dev(w)
    ng = len(G["node"])
    h = 2.0 / (n - 1)
    rng = np.random.default_rng(5)
    T = S.node_types(0) & 3
    for call in range(2):
        u = np.where(T > 0, rng.uniform(-1, 1, T.shape), 0.0)
        f = np.where(T == 1, rng.uniform(-3, 3, T.shape), 0.0)
        g = rng.uniform(-1, 1, ng)
        ud, fd, gd = _dev(u), _dev(f), _dev(g)
        r_ref = torch.zeros(T.shape, dtype=torch.float64, device="cuda")
        norm_ref = S.defect(0, ud, fd, gd, r_ref)
        r_na = torch.full(T.shape, float("nan"), dtype=torch.float64, device="cuda")
        norm = C.c_double(-1.0)
        st = L.gcmg_defect_noalloc(P.dim, n, h, _ptr(types), _ptr(ud), _ptr(fd), ng, _ptr(gnode), _ptr(stn),
                                   _ptr(wd), _ptr(gd), _ptr(r_na), C.byref(norm), None)
        torch.cuda.synchronize()
        assert st == gcmg.GCMG_OK, (call, st)
        ra, rb = r_na.cpu().numpy(), r_ref.cpu().numpy()
        assert np.abs(ra - rb).max() <= TOL * np.abs(rb).max(), call
        assert abs(norm.value - norm_ref) <= TOL * norm_ref, (call, norm.value, norm_ref)
    S.close()


def test_noalloc_rejects_problems_beyond_its_capacity():
    from paper_1111_0983_gb300 import gcmg
    L = gcmg.lib()
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = _ptr(dummy)
    # 8193^2 = 67,125,249 grid nodes exceed the 67,108,864 items the scratch covers
    st = L.gcmg_defect_noalloc(2, 8193, 2.0 / 8192, p, p, p, 0, None, None, None, None, p, None, None)
    assert st == gcmg.GCMG_E_SIZE
    st = L.gcmg_defect_noalloc(4, 65, 2.0 / 64, p, p, p, 0, None, None, None, None, p, None, None)
    assert st == gcmg.GCMG_E_ARG
