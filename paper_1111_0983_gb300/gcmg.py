"""ctypes binding of libgcmg.so (include/gcmg.h).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  Device buffers are torch CUDA tensors (float64, contiguous);
PyTorch only provides device memory and streams.  Loading fails loudly when
the compiled library is missing -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgcmg.so")

GCMG_OK, GCMG_E_ARG, GCMG_E_CUDA, GCMG_E_OOM, GCMG_E_GEOM, GCMG_E_NOCONV, GCMG_E_STATE, GCMG_E_SIZE, GCMG_E_TIMEOUT = range(9)
STATUS_NAMES = {0: "OK", 1: "E_ARG", 2: "E_CUDA", 3: "E_OOM", 4: "E_GEOM", 5: "E_NOCONV", 6: "E_STATE",
                7: "E_SIZE", 8: "E_TIMEOUT"}
KMAX = 27


class Params(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int), ("n_coarse", C.c_int), ("nu1", C.c_int), ("nu2", C.c_int),
                ("lam", C.c_int), ("gamma", C.c_int), ("delta_over_h", C.c_double), ("c_dirichlet", C.c_double),
                ("c_neumann_factor", C.c_double), ("precision", C.c_int), ("max_cycles", C.c_int),
                ("rtol", C.c_double), ("junction_sweeps", C.c_int), ("junction_radius", C.c_double),
                ("junction_solve", C.c_int), ("fused_coarse_n", C.c_int), ("smoother", C.c_int),
                ("h", C.c_double), ("origin", C.c_double * 3), ("diverge_cycles", C.c_int)]


class Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int64 * 3), ("h", C.c_double), ("origin", C.c_double * 3)]


class Stats(C.Structure):
    _fields_ = [("cycles", C.c_int), ("converged", C.c_int), ("rel_residual", C.c_double),
                ("r0_norm", C.c_double), ("rel", C.c_double * 257), ("diverged", C.c_int)]

    def to_dict(self):
        m = self.cycles
        return dict(cycles=m, converged=bool(self.converged), rel_residual=self.rel_residual,
                    r0_norm=self.r0_norm, rel=np.array(self.rel[: min(m, 256) + 1]),
                    diverged=bool(self.diverged))


class GcmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"gcmg {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1111_0983_gb300.build`")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, dbl, st = C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_int
        sig = {
            "gcmg_default_params": (st, [C.POINTER(Params), i32, i32, i32]),
            "gcmg_create": (st, [C.POINTER(Params), vp, vp, C.POINTER(vp)]),
            "gcmg_create_grid": (st, [C.POINTER(Grid), vp, C.POINTER(Params), vp, C.POINTER(vp)]),
            "gcmg_set_bc_types_from_mask": (st, [vp, vp]),
            "gcmg_bc_types": (st, [vp, i32, vp]),
            "gcmg_debug_barrier": (st, [vp, i32, i32, C.c_uint]),
            "gcmg_set_sweep3d": (st, [vp, i32]),
            "gcmg_set_span3d": (st, [vp, i32, i32]),
            "gcmg_set_junction_blocks": (st, [vp, i32]),
            "gcmg_junction_mode": (i32, [vp, i32]),
            "gcmg_set_split2d": (st, [vp, i32]),
            "gcmg_set_max_cycles": (st, [vp, i32]),
            "gcmg_span3d_info": (st, [vp, i32, C.POINTER(i32), C.POINTER(i32)]),
            "gcmg_set_boundary3d": (st, [vp, i32]),
            "gcmg_residual": (st, [vp, vp, vp, C.POINTER(dbl)]),
            "gcmg_destroy": (None, [vp]),
            "gcmg_last_error": (C.c_char_p, [vp]),
            "gcmg_num_levels": (i32, [vp]),
            "gcmg_level_n": (i32, [vp, i32]),
            "gcmg_num_ghosts": (st, [vp, i32, C.POINTER(i64)]),
            "gcmg_num_unknowns": (st, [vp, i32, C.POINTER(i64)]),
            "gcmg_ghost_geometry": (st, [vp, i32, vp, vp, vp, vp]),
            "gcmg_ghost_equations": (st, [vp, i32, vp, vp, vp]),
            "gcmg_node_types": (st, [vp, i32, vp]),
            "gcmg_set_bc_types": (st, [vp, i32, vp]),
            "gcmg_set_rhs": (st, [vp, vp, vp]),
            "gcmg_solve": (st, [vp, vp, C.POINTER(Stats)]),
            "gcmg_solve_host": (st, [vp, vp, vp, vp, C.POINTER(Stats)]),
            "gcmg_defect": (st, [vp, i32, vp, vp, vp, vp, C.POINTER(dbl)]),
            "gcmg_relax": (st, [vp, i32, vp, vp, vp, i32]),
            "gcmg_extend": (st, [vp, i32, vp]),
            "gcmg_restrict": (st, [vp, i32, vp, vp, vp]),
            "gcmg_prolong": (st, [vp, i32, vp, vp]),
            "gcmg_set_kernel_timing": (st, [vp, i32]),
            "gcmg_kernel_timing": (st, [vp, C.POINTER(i64), C.POINTER(dbl)]),
            "gcmg_kernel_timing_ex": (st, [vp, C.POINTER(i64), C.POINTER(dbl), C.POINTER(dbl)]),
            "gcmg_set_rhs_level": (st, [vp, i32, vp, vp]),
            "gcmg_fmg": (st, [vp, i32, vp]),
            "gcmg_reinit": (st, [i32, i32, vp, i32, vp, vp]),
            "gcmg_launch_counter": (i64, []),
            "gcmg_junction_zone": (st, [vp, i32, vp]),
            "gcmg_junction_solve_set": (st, [vp, i32, vp]),
            "gcmg_defect_noalloc": (st, [i32, i32, dbl, vp, vp, vp, i64, vp, vp, vp, vp, vp, C.POINTER(dbl), vp]),
            "gcmg_batch_create": (st, [i32, C.POINTER(Params), C.POINTER(vp), vp, C.POINTER(vp)]),
            "gcmg_batch_destroy": (None, [vp]),
            "gcmg_batch_last_error": (C.c_char_p, [vp]),
            "gcmg_batch_size": (i32, [vp]),
            "gcmg_batch_domain": (vp, [vp, i32]),
            "gcmg_batch_solve": (st, [vp, C.POINTER(Stats), C.POINTER(i32)]),
            "gcmg_batch_get_solution": (st, [vp, i32, vp]),
            "gcmg_batch_set_tiles": (st, [vp, i32]),
            "gcmg_batch_set_graph": (st, [vp, i32]),
            "gcmg_batch_autotune": (st, [vp, C.POINTER(i32), C.POINTER(dbl)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def default_params(dim, n, n_coarse, **kw):
    p = Params()
    lib().gcmg_default_params(C.byref(p), dim, n, n_coarse)
    for k, v in kw.items():
        setattr(p, "lam" if k == "lam" or k == "lambda_" else k, v)
    return p


def _ptr(t):
    """Device (torch) or host (numpy) buffer -> void*."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags.c_contiguous
        return C.c_void_p(t.ctypes.data)
    assert t.is_contiguous()
    return C.c_void_p(t.data_ptr())


class Solver:
    """One multigrid hierarchy (a gcmg context) on the current CUDA device."""

    @classmethod
    def _borrow(cls, handle, dim, n, params):
        """Wraps a context owned by someone else (a batch domain)."""
        self = cls.__new__(cls)
        self._h = C.c_void_p(handle)
        self.dim, self.n, self.params, self.stream = dim, n, params, None
        self.nlev = lib().gcmg_num_levels(self._h)
        self._borrowed = True
        return self

    def __init__(self, phi, n_coarse, stream=None, grid=None, **params):
        """grid: optional (h, origin) of the nodes (default: the box [-1,1]^d)."""
        import torch
        phi_t = phi if isinstance(phi, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(phi))
        phi_t = phi_t.to(device="cuda", dtype=torch.float64).contiguous()
        self.dim = phi_t.dim()
        self.n = phi_t.shape[0]
        self.params = default_params(self.dim, self.n, n_coarse, **params)
        self.stream = stream
        h = C.c_void_p()
        sp = C.c_void_p(stream.cuda_stream) if stream else None
        if grid is None:
            s = lib().gcmg_create(C.byref(self.params), _ptr(phi_t), sp, C.byref(h))
        else:
            g = Grid()
            g.dim = self.dim
            for a in range(3):
                g.n[a] = self.n if a < self.dim else 1
                g.origin[a] = grid[1][a] if a < self.dim else -1.0
            g.h = grid[0]
            s = lib().gcmg_create_grid(C.byref(g), _ptr(phi_t), C.byref(self.params), sp, C.byref(h))
        self._h = h
        if s != GCMG_OK:
            msg = lib().gcmg_last_error(h).decode() if h.value else ""
            if h.value:
                lib().gcmg_destroy(h)
            self._h = None
            raise GcmgError(s, msg)
        self.nlev = lib().gcmg_num_levels(self._h)

    def close(self):
        if getattr(self, "_h", None) and not getattr(self, "_borrowed", False):
            lib().gcmg_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, s):
        if s != GCMG_OK:
            raise GcmgError(s, lib().gcmg_last_error(self._h).decode())

    # ---- geometry
    def level_n(self, l):
        return lib().gcmg_level_n(self._h, l)

    def shape(self, l):
        return (self.level_n(l),) * self.dim

    def num_ghosts(self, l):
        v = C.c_int64()
        self._check(lib().gcmg_num_ghosts(self._h, l, C.byref(v)))
        return v.value

    def num_unknowns(self, l=0):
        v = C.c_int64()
        self._check(lib().gcmg_num_unknowns(self._h, l, C.byref(v)))
        return v.value

    def ghosts(self, l):
        ng, d = self.num_ghosts(l), self.dim
        out = dict(node=np.empty(ng, np.int64), B=np.empty((ng, d)), nu=np.empty((ng, d)),
                   case=np.empty(ng, np.uint8))
        self._check(lib().gcmg_ghost_geometry(self._h, l, *[_ptr(out[k]) for k in ("node", "B", "nu", "case")]))
        return out

    def ghost_equations(self, l):
        ng = self.num_ghosts(l)
        out = dict(stn=np.empty((ng, KMAX), np.int64), wD=np.empty((ng, KMAX)), wN=np.empty((ng, KMAX)))
        self._check(lib().gcmg_ghost_equations(self._h, l, *[_ptr(out[k]) for k in ("stn", "wD", "wN")]))
        return out

    def junction_zone(self, l):
        out = np.empty(self.shape(l), np.uint8)
        self._check(lib().gcmg_junction_zone(self._h, l, _ptr(out)))
        return out

    def junction_solve_set(self, l):
        out = np.empty(self.shape(l), np.uint8)
        self._check(lib().gcmg_junction_solve_set(self._h, l, _ptr(out)))
        return out

    def node_types(self, l):
        out = np.empty(self.shape(l), np.uint8)
        self._check(lib().gcmg_node_types(self._h, l, _ptr(out)))
        return out

    # ---- data
    def set_bc_types(self, l, types):
        t = np.ascontiguousarray(types, dtype=np.uint8)
        assert t.shape == (self.num_ghosts(l),)
        self._check(lib().gcmg_set_bc_types(self._h, l, _ptr(t)))

    def debug_barrier(self, enable=True, phantom_blocks=0, spin_limit=1 << 22):
        """3D boundary relaxation: one launch with barriers (enable) or one
        launch per phase; phantom_blocks > 0 makes its barrier waits run out."""
        self._check(lib().gcmg_debug_barrier(self._h, int(bool(enable)), int(phantom_blocks), int(spin_limit)))

    def set_boundary3d(self, mode):
        """3D boundary relaxation: 0 a launch a phase (default), 1 clusters on
        small levels, 2 one grid with software barriers."""
        self._check(lib().gcmg_set_boundary3d(self._h, int(mode)))

    def set_sweep3d(self, variant):
        """3D interior sweep kernel: 0 shared-memory planes, 1 register planes,
        2 row spans (default)."""
        self._check(lib().gcmg_set_sweep3d(self._h, int(variant)))

    def set_span3d(self, columns=0, planes=0):
        """Rebuild the row-span sweep's items: columns a lane (2..5, 0 auto),
        planes an item (1..32, 0 = 32)."""
        self._check(lib().gcmg_set_span3d(self._h, int(columns), int(planes)))

    def set_junction_blocks(self, enable=True):
        """3D junction zone in overlapping shared-memory blocks (default) or
        as whole components."""
        self._check(lib().gcmg_set_junction_blocks(self._h, int(bool(enable))))

    def set_max_cycles(self, k):
        """Cycle limit of the next solves (1..256), without a new solve graph."""
        self._check(lib().gcmg_set_max_cycles(self._h, int(k)))

    def set_split2d(self, min_strips):
        """2D FP32 levels with at least min_strips strips relax as two launches
        side by side (0: always one merged launch)."""
        self._check(lib().gcmg_set_split2d(self._h, int(min_strips)))

    def junction_mode(self, l):
        """Level l's junction sweeps: 0 global lists, 1 whole components in
        shared memory, 2 blocks in shared memory."""
        return int(lib().gcmg_junction_mode(self._h, int(l)))

    def span3d_info(self, l):
        """(items, columns) of the row-span sweep on level l."""
        it, co = C.c_int(0), C.c_int(0)
        self._check(lib().gcmg_span3d_info(self._h, int(l), C.byref(it), C.byref(co)))
        return it.value, co.value

    def bc_types(self, l):
        out = np.empty(self.num_ghosts(l), np.uint8)
        self._check(lib().gcmg_bc_types(self._h, l, _ptr(out)))
        return out

    def set_bc_types_from_mask(self, mask):
        """Boundary types of every level from a Dirichlet(0)/Neumann(1) mask on
        the fine grid (device uint8 tensor, n^d)."""
        assert mask.dtype.itemsize == 1 and mask.is_cuda and mask.numel() == self.n ** self.dim
        self._check(lib().gcmg_set_bc_types_from_mask(self._h, _ptr(mask.contiguous())))

    def set_rhs(self, f, g):
        self._check(lib().gcmg_set_rhs(self._h, _ptr(f), _ptr(g)))

    def residual(self, u, r):
        """FP64 defect of u (device tensor) into r; returns ||r|| / ||(f, g)||."""
        rel = C.c_double()
        self._check(lib().gcmg_residual(self._h, _ptr(u), _ptr(r), C.byref(rel)))
        return rel.value

    def set_rhs_level(self, l, f, g):
        """f and g of level l (device tensors), for fmg (plain FP64 solvers)."""
        self._check(lib().gcmg_set_rhs_level(self._h, int(l), _ptr(f), _ptr(g)))

    def fmg(self, nu, u):
        """Full multigrid with nu cycles a level into the device tensor u."""
        self._check(lib().gcmg_fmg(self._h, int(nu), _ptr(u)))

    def solve(self, u):
        st = Stats()
        s = lib().gcmg_solve(self._h, _ptr(u), C.byref(st))
        if s not in (GCMG_OK, GCMG_E_NOCONV):
            self._check(s)
        return st.to_dict()

    def solve_host(self, f, g, u_out=None):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        u = np.empty(self.shape(0)) if u_out is None else u_out
        st = Stats()
        s = lib().gcmg_solve_host(self._h, _ptr(f), _ptr(g), _ptr(u), C.byref(st))
        if s not in (GCMG_OK, GCMG_E_NOCONV):
            self._check(s)
        return u, st.to_dict()

    # ---- single steps (FP64, caller buffers of the level's size)
    def defect(self, l, u, f, g, r):
        nrm = C.c_double()
        self._check(lib().gcmg_defect(self._h, l, _ptr(u), _ptr(f), _ptr(g), _ptr(r), C.byref(nrm)))
        return nrm.value

    def relax(self, l, u, f, g, with_extra=True):
        self._check(lib().gcmg_relax(self._h, l, _ptr(u), _ptr(f), _ptr(g), int(with_extra)))

    def extend(self, l, r):
        self._check(lib().gcmg_extend(self._h, l, _ptr(r)))

    def restrict(self, l, r, fc, gc):
        self._check(lib().gcmg_restrict(self._h, l, _ptr(r), _ptr(fc), _ptr(gc)))

    def prolong(self, l, ec, out):
        self._check(lib().gcmg_prolong(self._h, l, _ptr(ec), _ptr(out)))

    # ---- measurement
    KERNEL_SMOOTH, KERNEL_DEFECT, KERNEL_PROLONG, KERNEL_RESTRICT, KERNEL_BOUNDARY = 0, 1, 2, 3, 4

    def set_kernel_timing(self, kind):
        self._check(lib().gcmg_set_kernel_timing(self._h, int(kind)))

    def kernel_timing(self):
        n, ms = C.c_int64(), C.c_double()
        self._check(lib().gcmg_kernel_timing(self._h, C.byref(n), C.byref(ms)))
        return n.value, ms.value

    def kernel_timing_ex(self):
        """(launches, total ms, algorithmic bytes) of the timed launches."""
        n, ms, b = C.c_int64(), C.c_double(), C.c_double()
        self._check(lib().gcmg_kernel_timing_ex(self._h, C.byref(n), C.byref(ms), C.byref(b)))
        return n.value, ms.value, b.value


def launch_counter():
    return lib().gcmg_launch_counter()


def reinit(phi0, steps, stream=None):
    """Level set phi0 (device tensor, n^dim doubles) after `steps` steps of the
    reinitialisation equation (gcmg_reinit); returns a new device tensor."""
    import torch
    phi0 = phi0.contiguous()
    out = torch.empty_like(phi0)
    s = lib().gcmg_reinit(phi0.dim(), phi0.shape[0], _ptr(phi0), int(steps), _ptr(out),
                          C.c_void_p(stream.cuda_stream) if stream else None)
    if s != GCMG_OK:
        raise GcmgError(s, "gcmg_reinit failed")
    return out


class Batch:
    """Many 2D domains solved together (gcmg_batch): one launch per cycle step
    over all domains, one graph launch per solve."""

    def __init__(self, phis, n_coarse, stream=None, **params):
        import torch
        self.count = len(phis)
        ts = [torch.from_numpy(np.ascontiguousarray(p)).to("cuda", torch.float64) for p in phis]
        ncs = n_coarse if isinstance(n_coarse, (list, tuple)) else [n_coarse] * self.count
        P = (Params * self.count)()
        for i, t in enumerate(ts):
            P[i] = default_params(2, t.shape[0], ncs[i], precision=1, **params)
        ptrs = (C.c_void_p * self.count)(*[t.data_ptr() for t in ts])
        h = C.c_void_p()
        s = lib().gcmg_batch_create(self.count, P, ptrs, C.c_void_p(stream.cuda_stream) if stream else None,
                                    C.byref(h))
        self._h = h
        if s != GCMG_OK:
            msg = lib().gcmg_batch_last_error(h).decode() if h.value else ""
            if h.value:
                lib().gcmg_batch_destroy(h)
            self._h = None
            raise GcmgError(s, msg)
        self.domains = [Solver._borrow(lib().gcmg_batch_domain(self._h, i), 2, ts[i].shape[0], P[i])
                        for i in range(self.count)]

    def close(self):
        if getattr(self, "_h", None):
            lib().gcmg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, s):
        if s != GCMG_OK:
            raise GcmgError(s, lib().gcmg_batch_last_error(self._h).decode())

    def solve(self):
        st = (Stats * self.count)()
        steps = C.c_int()
        s = lib().gcmg_batch_solve(self._h, st, C.byref(steps))
        if s not in (GCMG_OK, GCMG_E_NOCONV):
            self._check(s)
        return [x.to_dict() for x in st], steps.value

    def solution(self, i, out):
        self._check(lib().gcmg_batch_get_solution(self._h, i, _ptr(out)))

    def set_tiles(self, variant):
        self._check(lib().gcmg_batch_set_tiles(self._h, int(variant)))

    def set_graph(self, on):
        """False: solves as plain launches (same results; for profilers)."""
        self._check(lib().gcmg_batch_set_graph(self._h, int(bool(on))))

    def autotune(self):
        best = C.c_int()
        ms = (C.c_double * 3)()
        self._check(lib().gcmg_batch_autotune(self._h, C.byref(best), ms))
        return best.value, list(ms)

