"""Seeded synthetic problems for the ghost-cell multigrid (numpy only).

This module is shared by the tests, the benchmark and the CPU oracle's
callers.  It holds problem DATA only -- level sets, exact solutions, the
Dirichlet/Neumann split of the boundary and the boundary values evaluated at
the projection points that the solver reports -- and none of the solver's
arithmetic.  It imports nothing else from this package.

Grid convention: n nodes per axis on [-1, 1], node j at -1 + j h with
h = 2/(n-1); arrays are C ordered with axis 0 (x) slowest (``indexing='ij'``).

Workloads (shapes of the paper's tests, Sec. 3, plus the library's own
configurations):
  * ``disk``   : phi = |x - (0.02, 0.01)| - 0.7, u = e^x sin y (f = 0), all Dirichlet.
  * ``flower`` : phi = r - 0.5 - 0.15 sin(5 theta), u = cos(3x) e^y, f = 8 cos(3x) e^y;
                 Dirichlet where B_y > 0, Neumann elsewhere.
  * ``torus``  : phi = sqrt((sqrt(x^2+y^2) - 0.5)^2 + z^2) - 0.25,
                 u = sin x cos y e^z, f = u; Neumann where B_z < 0, Dirichlet elsewhere.
  * ``star``   : phi = r - R0 (1 + a sin(k theta + p)) with seeded R0, a, k, p and a
                 seeded split line through the origin (Dirichlet on the side
                 B . (cos al, sin al) > 0); u as for the flower.
  * ``circle`` : the paper's circle (centre (sqrt2/20, sqrt3/30), radius 0.563)
                 with its split Gamma_D = {x <= 0}, Gamma_N = {x > 0} (Sec. 3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """One output of Steele, Lea & Flood's SplitMix64 for state x (published constants)."""
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


class SplitMix:
    """Counter-based stream: value k of stream s is splitmix64(s + k * golden)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo=0.0, hi=1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi]."""
        return lo + self.next_u64() % (hi - lo + 1)


def coords(dim: int, n: int):
    # exact node coordinates -1 + j h (linspace may differ in the last bit)
    h = 2.0 / (n - 1)
    x = -1.0 + np.arange(n) * h
    return np.meshgrid(*([x] * dim), indexing="ij")


@dataclass
class Problem:
    """A boundary-value problem -Lap u = f in {phi < 0} with a D/N split."""
    name: str
    dim: int
    phi: Callable           # phi(*X) on arrays
    u: Callable             # exact solution (None for data-only problems)
    grad_u: Callable        # returns list of d arrays
    f: Callable             # f = -Lap u
    is_neumann: Callable    # boolean per boundary point B (array (m, d)) -> array (m,)
    n_coarse: int = 33
    meta: dict = field(default_factory=dict)

    def phi_grid(self, n):
        return np.ascontiguousarray(self.phi(*coords(self.dim, n)), dtype=np.float64)

    def f_grid(self, n):
        return np.ascontiguousarray(self.f(*coords(self.dim, n)), dtype=np.float64)

    def u_grid(self, n):
        return np.ascontiguousarray(self.u(*coords(self.dim, n)), dtype=np.float64)

    def bc_types(self, B):
        """0 = Dirichlet, 1 = Neumann for boundary points B (m, d)."""
        B = np.asarray(B, dtype=np.float64).reshape(-1, self.dim)
        return np.ascontiguousarray(self.is_neumann(B).astype(np.uint8))

    def g_values(self, B, nu, types):
        """Boundary data per ghost: u(B) (Dirichlet) or grad u(B) . nu (Neumann),
        with nu the discrete normal the solver reports for that ghost."""
        B = np.asarray(B, dtype=np.float64).reshape(-1, self.dim)
        nu = np.asarray(nu, dtype=np.float64).reshape(-1, self.dim)
        cols = [B[:, a] for a in range(self.dim)]
        gd = self.u(*cols)
        gu = self.grad_u(*cols)
        gn = sum(gu[a] * nu[:, a] for a in range(self.dim))
        return np.ascontiguousarray(np.where(np.asarray(types) == 0, gd, gn), dtype=np.float64)


def disk() -> Problem:
    cx, cy, r = 0.02, 0.01, 0.7
    return Problem(
        "disk", 2,
        phi=lambda x, y: np.sqrt((x - cx) ** 2 + (y - cy) ** 2) - r,
        u=lambda x, y: np.exp(x) * np.sin(y),
        grad_u=lambda x, y: [np.exp(x) * np.sin(y), np.exp(x) * np.cos(y)],
        f=lambda x, y: np.zeros_like(x),
        is_neumann=lambda B: np.zeros(B.shape[0], bool),
        n_coarse=17)


def _flower_u():
    u = lambda x, y: np.cos(3 * x) * np.exp(y)
    gu = lambda x, y: [-3 * np.sin(3 * x) * np.exp(y), np.cos(3 * x) * np.exp(y)]
    f = lambda x, y: 8.0 * np.cos(3 * x) * np.exp(y)
    return u, gu, f


def flower(amp: float = 0.15) -> Problem:
    u, gu, f = _flower_u()
    return Problem(
        "flower", 2,
        phi=lambda x, y: np.sqrt(x * x + y * y) - 0.5 - amp * np.sin(5 * np.arctan2(y, x)),
        u=u, grad_u=gu, f=f,
        is_neumann=lambda B: ~(B[:, 1] > 0),
        n_coarse=33)


def torus() -> Problem:
    R, rr = 0.5, 0.25
    return Problem(
        "torus", 3,
        phi=lambda x, y, z: np.sqrt((np.sqrt(x * x + y * y) - R) ** 2 + z * z) - rr,
        u=lambda x, y, z: np.sin(x) * np.cos(y) * np.exp(z),
        grad_u=lambda x, y, z: [np.cos(x) * np.cos(y) * np.exp(z), -np.sin(x) * np.sin(y) * np.exp(z),
                                np.sin(x) * np.cos(y) * np.exp(z)],
        f=lambda x, y, z: np.sin(x) * np.cos(y) * np.exp(z),
        is_neumann=lambda B: B[:, 2] < 0,
        n_coarse=17)


def circle_paper(radius: float = 0.563) -> Problem:
    cx, cy = math.sqrt(2) / 20, math.sqrt(3) / 30
    u, gu, f = _flower_u()
    return Problem(
        "circle", 2,
        phi=lambda x, y: np.sqrt((x - cx) ** 2 + (y - cy) ** 2) - radius,
        u=u, grad_u=gu, f=f,
        is_neumann=lambda B: B[:, 0] > 0,
        n_coarse=9)


def star_min_concave_radius(R0: float, a: float, k: int) -> float:
    """Smallest radius of curvature on the concave parts of the boundary
    r(theta) = R0 (1 + a sin(k theta + p)) (inf if it is convex); the
    curvature depends on k theta + p only, sampled finely over one period."""
    ph = np.linspace(0.0, 2 * math.pi, 8192, endpoint=False)
    r = R0 * (1 + a * np.sin(ph))
    r1 = R0 * a * k * np.cos(ph)
    r2 = -R0 * a * k * k * np.sin(ph)
    kap = (r * r + 2 * r1 * r1 - r * r2) / (r * r + r1 * r1) ** 1.5
    return float(1.0 / -kap.min()) if kap.min() < 0 else math.inf


STAR_MIN_RADIUS = 0.02


def star_params(i: int, base: int = 1111 << 20):
    """Seeded star i: R0 ~ U[0.4,0.7], a ~ U[0,0.3], k ~ U{3..8}, p ~ U[0,2pi),
    split angle al ~ U[0,2pi), n ~ U{129,257,513,1025}.  A draw whose concave
    radius of curvature falls below STAR_MIN_RADIUS (about 1.3 h of the 129^2
    grid, 0.3 h of the 65^2 one) is rejected and drawn again from the same
    stream: the coarse levels of the hierarchy must resolve the boundary."""
    rng = SplitMix(splitmix64(base + i))
    while True:
        R0 = rng.uniform(0.4, 0.7)
        a = rng.uniform(0.0, 0.3)
        k = rng.randint(3, 8)
        p = rng.uniform(0.0, 2 * math.pi)
        al = rng.uniform(0.0, 2 * math.pi)
        n = (129, 257, 513, 1025)[rng.randint(0, 3)]
        if star_min_concave_radius(R0, a, k) >= STAR_MIN_RADIUS:
            return dict(R0=R0, a=a, k=k, p=p, al=al, n=n)


def star(i: int = 0, base: int = 1111 << 20, params: dict | None = None) -> Problem:
    sp = params or star_params(i, base)
    R0, a, k, p, al = sp["R0"], sp["a"], sp["k"], sp["p"], sp["al"]
    u, gu, f = _flower_u()
    ca, sa = math.cos(al), math.sin(al)
    return Problem(
        f"star{i}", 2,
        phi=lambda x, y: np.sqrt(x * x + y * y) - R0 * (1 + a * np.sin(k * np.arctan2(y, x) + p)),
        u=u, grad_u=gu, f=f,
        is_neumann=lambda B: ~(B[:, 0] * ca + B[:, 1] * sa > 0),
        n_coarse=33, meta=sp)


def quadratic_patch(dim: int, coef=None, domain: str = "disk", neumann: str = "none") -> Problem:
    """u = a quadratic polynomial, f = -Lap u (constant).  The discrete solution
    equals u wherever every ghost uses a full quadratic stencil."""
    rng = np.random.default_rng(7)
    if coef is None:
        coef = rng.uniform(-1, 1, size=(1 + dim + dim * (dim + 1) // 2))
    c0 = coef[0]
    lin = coef[1:1 + dim]
    quad = coef[1 + dim:]
    pairs = [(a, b) for a in range(dim) for b in range(a, dim)]

    def u(*X):
        v = c0 + sum(lin[a] * X[a] for a in range(dim))
        for q, (a, b) in zip(quad, pairs):
            v = v + q * X[a] * X[b]
        return v

    def grad_u(*X):
        g = [lin[a] + 0 * X[0] for a in range(dim)]
        for q, (a, b) in zip(quad, pairs):
            if a == b:
                g[a] = g[a] + 2 * q * X[a]
            else:
                g[a] = g[a] + q * X[b]
                g[b] = g[b] + q * X[a]
        return g

    lap = sum(2 * q for q, (a, b) in zip(quad, pairs) if a == b)
    if domain == "disk":
        if dim == 2:
            phi = lambda x, y: np.sqrt((x - 0.03) ** 2 + (y + 0.02) ** 2) - 0.61
        else:
            phi = lambda x, y, z: np.sqrt((x - 0.03) ** 2 + (y + 0.02) ** 2 + (z - 0.01) ** 2) - 0.61
    elif domain == "torus":
        phi = torus().phi
    else:
        raise ValueError(domain)
    if neumann == "none":
        isn = lambda B: np.zeros(B.shape[0], bool)
    elif neumann == "all":
        isn = lambda B: np.ones(B.shape[0], bool)
    else:  # half
        isn = lambda B: B[:, 0] > 0
    return Problem(f"quad{dim}", dim, phi=phi, u=u, grad_u=grad_u,
                   f=lambda *X: -lap + 0 * X[0], is_neumann=isn, n_coarse=9)


def homogeneous_guess(shape, seed: int = 1):
    """Seeded uniform[-1,1] initial guess for convergence-factor runs (Sec. 3)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=shape)


def gaussian_rhs(i: int, n: int, R0: float, base: int = 0):
    """f = sum_{m=1..M} A_m exp(-|x - c_m|^2 / (2 s_m^2)), M ~ U{1..4},
    A ~ U[-10, 10], c uniform in the disk of radius R0, s ~ U[0.05, 0.25]."""
    rng = SplitMix(splitmix64(base + 7919 * i + 13))
    x, y = coords(2, n)
    f = np.zeros_like(x)
    M = rng.randint(1, 4)
    for _ in range(M):
        A = rng.uniform(-10, 10)
        rad = R0 * math.sqrt(rng.uniform())
        th = rng.uniform(0, 2 * math.pi)
        cx, cy = rad * math.cos(th), rad * math.sin(th)
        s = rng.uniform(0.05, 0.25)
        f += A * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * s * s))
    return f


CONFIGS = {
    "disk65": (disk, 65),
    "flower1025": (flower, 1025),
    "flower4097": (flower, 4097),
    "torus257": (torus, 257),
    "torus513": (torus, 513),
}
