"""FP64 CPU oracle of the ghost-cell multigrid (Coco & Russo, arXiv 1111.0983).

TEST INFRASTRUCTURE ONLY: the correctness reference for the CUDA library.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does.

The C source ``gcmg_oracle.c`` holds the arithmetic; this module compiles it
with gcc (``build()``) and wraps it with ctypes.  Arrays are numpy, C order,
axis 0 (x) slowest; node j of an n-point axis sits at -1 + j h, h = 2/(n-1).
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gcmg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_gcmg.so")
MAXK = 27

T_EXT, T_INT, T_GHOST = 0, 1, 2
ST_QUAD, ST_LIN, ST_CORNER, ST_AXIS = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle shared library next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        _compile(_SRC, tmp)
        os.replace(tmp, _LIB)
    return _LIB


def _compile(src, out):
    """gcc with OpenMP where it is available (the loops it splits are
    order-independent: results do not depend on the thread count)."""
    base = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", "-o", out, src, "-lm"]
    try:
        subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
    except (subprocess.CalledProcessError, OSError):
        subprocess.check_call(base)


class Params(C.Structure):
    _fields_ = [("nu1", C.c_int), ("nu2", C.c_int), ("lam", C.c_int), ("gamma", C.c_int),
                ("mode", C.c_int), ("extra_once", C.c_int), ("delta_over_h", C.c_double),
                ("c_dirichlet", C.c_double), ("c_neumann_factor", C.c_double), ("junction_sweeps", C.c_int), ("junction_radius", C.c_double),
                ("junction_solve", C.c_int), ("smoother", C.c_int)]


_lib = None


def _load(path):
    """Loads a compiled oracle library and declares its functions."""
    if True:
        L = C.CDLL(path)
        vp, i64, dbl = C.c_void_p, C.c_int64, C.c_double
        L.orc_create.restype = vp
        L.orc_create.argtypes = [C.c_int, C.c_int, C.c_int, vp, C.POINTER(Params)]
        for name, res in [("orc_status", C.c_int), ("orc_num_levels", C.c_int), ("orc_error", C.c_char_p),
                          ("orc_num_coarse_unknowns", i64)]:
            getattr(L, name).restype = res
            getattr(L, name).argtypes = [vp]
        for name, res in [("orc_level_n", C.c_int), ("orc_level_h", dbl), ("orc_num_ghosts", i64),
                          ("orc_num_ext", i64)]:
            getattr(L, name).restype = res
            getattr(L, name).argtypes = [vp, C.c_int]
        L.orc_destroy.argtypes = [vp]
        L.orc_set_bc.argtypes = [vp, C.c_int, vp]
        L.orc_set_rhs.argtypes = [vp, vp, vp]
        L.orc_set_rhs_level.argtypes = [vp, C.c_int, vp, vp]
        L.orc_reinit.argtypes = [C.c_int, C.c_int, vp, C.c_int, vp]
        L.orc_fmg.argtypes = [vp, C.c_int, vp]
        L.orc_get_types.argtypes = [vp, C.c_int, vp]
        L.orc_get_band.argtypes = [vp, C.c_int, vp]
        L.orc_get_jzone.argtypes = [vp, C.c_int, vp]
        L.orc_get_jsolve.argtypes = [vp, C.c_int, vp]
        L.orc_get_ghosts.argtypes = [vp, C.c_int] + [vp] * 10
        L.orc_get_ext.argtypes = [vp, C.c_int, vp, vp, vp, vp]
        L.orc_defect.restype = dbl
        L.orc_defect.argtypes = [vp, C.c_int, vp, vp]
        L.orc_extend.argtypes = [vp, C.c_int, vp]
        L.orc_restrict.argtypes = [vp, C.c_int, vp, vp, vp]
        L.orc_restrict_weights.restype = C.c_int
        L.orc_restrict_weights.argtypes = [vp, C.c_int, i64, C.c_int, vp]
        L.orc_prolong.argtypes = [vp, C.c_int, vp, vp]
        L.orc_relax.argtypes = [vp, C.c_int, vp, vp, vp, C.c_int]
        L.orc_kaczmarz_row.argtypes = [vp, C.c_int, C.c_int64, vp, vp, vp]
        L.orc_assemble.restype = i64
        L.orc_assemble.argtypes = [vp, C.c_int, vp, vp, vp, vp]
        L.orc_set_threads.restype = C.c_int
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_solve.restype = C.c_int
        L.orc_solve.argtypes = [vp, vp, dbl, C.c_int, vp, C.POINTER(C.c_int)]
    return L


def lib():
    """The oracle library in use (compiled on first use)."""
    global _lib
    if _lib is None:
        _lib = _load(build())
    return _lib


def build_variant(source: str, out_dir: str) -> str:
    """Compiles a modified copy of the oracle source (the planted-slip tests
    plant one mistake in it) into out_dir; returns the library path."""
    src = os.path.join(out_dir, "gcmg_oracle_variant.c")
    out = os.path.join(out_dir, "liboracle_variant.so")
    with open(src, "w") as fh:
        fh.write(source)
    _compile(src, out)
    return out


@contextlib.contextmanager
def variant(path: str):
    """Within the block, new Oracle objects use the library at `path`."""
    global _lib
    saved = lib()
    _lib = _load(path)
    try:
        yield _lib
    finally:
        _lib = saved


def set_threads(k: int) -> int:
    """Threads of the oracle's parallel loops (1: serial); returns the count
    in effect (1 when the library was built without OpenMP)."""
    return lib().orc_set_threads(int(k))


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class OracleError(RuntimeError):
    pass


def reinit(phi0, steps):
    """Level set phi0 (n^dim nodes of [-1,1]^dim) after `steps` steps of the
    reinitialisation equation phi_t = sgn(phi0)(1 - |grad phi|) (Sec. 2.1)."""
    phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
    out = np.empty_like(phi0)
    lib().orc_reinit(phi0.ndim, phi0.shape[0], _p(phi0), int(steps), _p(out))
    return out


class Oracle:
    """One multigrid hierarchy built from a fine level set ``phi`` (shape n^dim)."""

    def __init__(self, phi, n_coarse, nu1=2, nu2=1, lam=5, gamma=1, mode=0, extra_once=0,
                 delta_over_h=3.0, c_dirichlet=0.9, c_neumann_factor=0.9, junction_sweeps=None, junction_radius=None,
                 junction_solve=None, smoother=0):
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        self.dim = phi.ndim
        # junction relaxation defaults: 2D an exact solve of the zone within
        # 20h; 3D (the zone is a tube around junction curves) 10 sweeps
        # within 2h.  junction_sweeps=0 alone turns it off.
        if junction_solve is None:
            junction_solve = 1 if (self.dim == 2 and junction_sweeps is None) else 0
        if junction_sweeps is None:
            junction_sweeps = 0 if self.dim == 2 else 10
        if junction_radius is None:
            junction_radius = 20.0 if self.dim == 2 else 2.0
        self.n = phi.shape[0]
        assert all(s == self.n for s in phi.shape)
        self.params = Params(nu1, nu2, lam, gamma, mode, extra_once, delta_over_h, c_dirichlet,
                             c_neumann_factor, junction_sweeps, junction_radius, junction_solve, smoother)
        L = self._L = lib()   # kept: a variant build may be swapped in later
        self._h = L.orc_create(self.dim, self.n, n_coarse, _p(phi), C.byref(self.params))
        if not self._h:
            raise MemoryError("oracle allocation failed")
        st = L.orc_status(self._h)
        if st != 0:
            msg = L.orc_error(self._h).decode()
            L.orc_destroy(self._h)
            self._h = None
            raise OracleError(f"oracle status {st}: {msg}")
        self.nlev = L.orc_num_levels(self._h)

    def __del__(self):
        if getattr(self, "_h", None):
            self._L.orc_destroy(self._h)
            self._h = None

    # ---- geometry
    def level_n(self, l):
        return self._L.orc_level_n(self._h, l)

    def level_h(self, l):
        return self._L.orc_level_h(self._h, l)

    def shape(self, l):
        return (self.level_n(l),) * self.dim

    def num_ghosts(self, l):
        return self._L.orc_num_ghosts(self._h, l)

    def types(self, l):
        out = np.empty(self.shape(l), np.uint8)
        self._L.orc_get_types(self._h, l, _p(out))
        return out

    def band(self, l):
        out = np.empty(self.shape(l), np.uint8)
        self._L.orc_get_band(self._h, l, _p(out))
        return out

    def junction_zone(self, l):
        out = np.empty(self.shape(l), np.uint8)
        self._L.orc_get_jzone(self._h, l, _p(out))
        return out

    def junction_solve_set(self, l):
        """Mask of the unknowns whose equations the exact junction solve solves."""
        out = np.empty(self.shape(l), np.uint8)
        self._L.orc_get_jsolve(self._h, l, _p(out))
        return out

    def ghosts(self, l):
        ng, d = self.num_ghosts(l), self.dim
        rec = dict(node=np.empty(ng, np.int64), B=np.empty((ng, d)), nu=np.empty((ng, d)),
                   t=np.empty((ng, d)), s=np.empty((ng, d), np.int8), case=np.empty(ng, np.uint8),
                   nk=np.empty(ng, np.int32), stn=np.empty((ng, MAXK), np.int64),
                   wD=np.empty((ng, MAXK)), wN=np.empty((ng, MAXK)))
        self._L.orc_get_ghosts(self._h, l, *[_p(rec[k]) for k in
                                           ("node", "B", "nu", "t", "s", "case", "nk", "stn", "wD", "wN")])
        return rec

    def extension(self, l):
        ne = self._L.orc_num_ext(self._h, l)
        out = dict(node=np.empty(ne, np.int64), nsrc=np.empty(ne, np.int32),
                   src=np.empty((ne, 6), np.int64), w=np.empty((ne, 6)))
        if ne:
            self._L.orc_get_ext(self._h, l, _p(out["node"]), _p(out["nsrc"]), _p(out["src"]), _p(out["w"]))
        return out

    def coarse_unknowns(self):
        return self._L.orc_num_coarse_unknowns(self._h)

    # ---- data
    def set_bc(self, l, bc):
        bc = np.ascontiguousarray(bc, dtype=np.uint8)
        assert bc.shape == (self.num_ghosts(l),)
        self._L.orc_set_bc(self._h, l, _p(bc))
        st = self._L.orc_status(self._h)
        if st != 0:
            raise OracleError(f"oracle status {st}: {self._L.orc_error(self._h).decode()}")

    def set_rhs(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        assert f.shape == self.shape(0) and g.shape == (self.num_ghosts(0),)
        self._L.orc_set_rhs(self._h, _p(f), _p(g))

    def set_rhs_level(self, l, f, g):
        """f and g of level l (the problem's data sampled there), for fmg."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        assert f.shape == self.shape(l) and g.shape == (self.num_ghosts(l),)
        self._L.orc_set_rhs_level(self._h, l, _p(f), _p(g))

    def fmg(self, nu=1):
        """Full multigrid: exact coarsest solve, then per finer level the
        interpolated coarser solution improved by nu cycles.  Needs every
        level's f and g (set_rhs_level; level 0 may come from set_rhs)."""
        u = np.zeros(self.shape(0))
        self._L.orc_fmg(self._h, int(nu), _p(u))
        return u

    # ---- operators
    def defect(self, u, l=0):
        u = np.ascontiguousarray(u, dtype=np.float64)
        r = np.empty_like(u)
        nrm = self._L.orc_defect(self._h, l, _p(u), _p(r))
        return r, nrm

    def extend(self, r, l=0):
        r = np.array(r, dtype=np.float64, order="C", copy=True)
        self._L.orc_extend(self._h, l, _p(r))
        return r

    def restrict(self, r, l=0):
        r = np.ascontiguousarray(r, dtype=np.float64)
        fc = np.zeros(self.shape(l + 1))
        gc = np.zeros(max(self.num_ghosts(l + 1), 1))
        self._L.orc_restrict(self._h, l, _p(r), _p(fc), _p(gc))
        return fc, gc[: self.num_ghosts(l + 1)]

    def restrict_weights(self, l, X, interior_set):
        wt = np.zeros(3 ** self.dim)
        ok = self._L.orc_restrict_weights(self._h, l, int(X), int(interior_set), _p(wt))
        return (wt.reshape((3,) * self.dim) if ok else None)

    def prolong(self, e_coarse, l=0):
        e = np.ascontiguousarray(e_coarse, dtype=np.float64)
        out = np.empty(self.shape(l))
        self._L.orc_prolong(self._h, l, _p(e), _p(out))
        return out

    def kaczmarz_row(self, i, u, f, g, l=0):
        """One Kaczmarz step (Sec. 3.3 comparison) on the row of node i of level
        l: an inside node of the band or a ghost."""
        u = np.array(u, dtype=np.float64, order="C", copy=True)
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        self._L.orc_kaczmarz_row(self._h, l, C.c_int64(int(i)), _p(u), _p(f), _p(g))
        return u

    def relax(self, u, f, g, l=0, with_extra=True):
        u = np.array(u, dtype=np.float64, order="C", copy=True)
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        self._L.orc_relax(self._h, l, _p(u), _p(f), _p(g), int(with_extra))
        return u

    def assemble(self, l=0):
        """COO triplets of the level-l system over unknowns in increasing node order,
        and the node -> unknown map (-1 off Omega_h u Gamma_h)."""
        L = self._L
        nnz = L.orc_assemble(self._h, l, None, None, None, None)
        rows = np.empty(nnz, np.int64)
        cols = np.empty(nnz, np.int64)
        vals = np.empty(nnz)
        uon = np.empty(self.shape(l), np.int64)
        L.orc_assemble(self._h, l, _p(rows), _p(cols), _p(vals), _p(uon))
        return rows, cols, vals, uon

    def solve(self, u0=None, rtol=1e-10, max_cycles=100):
        """Cycles from u0 (zeros by default) until ||r||inf <= rtol ||r0||inf.
        Returns (u, norms, converged)."""
        u = np.zeros(self.shape(0)) if u0 is None else np.array(u0, dtype=np.float64, order="C", copy=True)
        norms = np.zeros(max_cycles + 1)
        st = C.c_int(0)
        m = self._L.orc_solve(self._h, _p(u), rtol, max_cycles, _p(norms), C.byref(st))
        return u, norms[: m + 1], st.value == 0
