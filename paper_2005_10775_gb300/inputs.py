"""Seeded synthetic inputs: triangle meshes, N-gon offsets and workload presets.

This module is the one piece shared by the CUDA path and the FP64 oracle.  It
holds none of the method's arithmetic (no geometry predicates, no quadrature,
no assembly): it only produces the inputs both sides consume.

Meshes follow the paper's setting (Sec. 3.1 and Sec. 8): Omega = (0,1)^2 with
an interaction layer Omega_I around it, covered by a uniform split-square grid
(grid (a) of Sec. 8, nested refinement), optionally with seeded vertex jitter.

Readings of details the paper leaves open:
  * every square cell is split by its lower-left -> upper-right diagonal and
    both triangles are counter-clockwise;
  * jitter moves each coordinate by U[-j h, j h] (numpy PCG64, given seed);
    vertices on the outer boundary and on grid lines that coincide with the
    boundary of Omega move only along that line, and corners stay fixed;
  * node j belongs to Omega iff it lies strictly inside (0,1)^2 by at least
    1e-12 h; nodes on the boundary of Omega belong to Omega_I (Sec. 3.1);
  * an element is labelled Omega iff its barycentre lies in (0,1)^2.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Mesh:
    vx: np.ndarray            # float64 [J]
    vy: np.ndarray            # float64 [J]
    tri: np.ndarray           # int32 [K, 3], counter-clockwise, 0-based
    node_in_omega: np.ndarray  # uint8 [J]: 1 = open Omega, 0 = Omega_I (incl. boundary)
    elem_in_omega: np.ndarray  # uint8 [K]: barycentre label (used for the load vector)
    h: float                  # grid cell size
    lo: float
    hi: float
    n: int

    @property
    def nv(self) -> int:
        return int(self.vx.shape[0])

    @property
    def nt(self) -> int:
        return int(self.tri.shape[0])


def split_square_mesh(lo: float, hi: float, n: int, jitter: float = 0.0,
                      seed: int | None = None, omega=(0.0, 1.0),
                      warp_y_square: bool = False) -> Mesh:
    """Uniform n x n split-square grid over (lo, hi)^2.

    jitter: amplitude as a fraction of h (0.2 -> U[-0.2h, 0.2h]).
    warp_y_square: apply (x1, x2) -> (x1, x2^2) to the grid rows inside 0 < x2 < 1
    (grid (b) of Sec. 8, Fig. 12b).
    """
    h = (hi - lo) / n
    ii, jj = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="xy")
    ii = ii.ravel()
    jj = jj.ravel()
    x = lo + ii * h
    y = lo + jj * h
    tol = 1e-9 * h
    o0, o1 = omega
    on_x_line = (np.abs(x - o0) < tol) | (np.abs(x - o1) < tol)   # vertical boundary lines of Omega
    on_y_line = (np.abs(y - o0) < tol) | (np.abs(y - o1) < tol)
    # only the parts of those lines that bound Omega
    on_x_bdry = on_x_line & (y > o0 - tol) & (y < o1 + tol)
    on_y_bdry = on_y_line & (x > o0 - tol) & (x < o1 + tol)
    x = np.where(np.abs(x - o0) < tol, o0, np.where(np.abs(x - o1) < tol, o1, x))
    y = np.where(np.abs(y - o0) < tol, o0, np.where(np.abs(y - o1) < tol, o1, y))
    if jitter > 0.0:
        rng = np.random.Generator(np.random.PCG64(seed))
        dx = rng.uniform(-jitter * h, jitter * h, size=x.shape)
        dy = rng.uniform(-jitter * h, jitter * h, size=y.shape)
        fix_x = (ii == 0) | (ii == n) | on_x_bdry
        fix_y = (jj == 0) | (jj == n) | on_y_bdry
        x = np.where(fix_x, x, x + dx)
        y = np.where(fix_y, y, y + dy)
    if warp_y_square:
        # grid (b) of Sec. 8: x2 -> x2^2 on every grid row strictly between the lines x2 = 0 and
        # x2 = 1 (the layer columns too, so the grid stays a tensor product; the printed h_min and
        # h_max of Table 4(b) are those of this grid)
        rows = (y > o0 + tol) & (y < o1 - tol)
        y = np.where(rows, y * y, y)
    vid = lambda i, j: j * (n + 1) + i  # noqa: E731
    ci, cj = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    ci = ci.ravel()
    cj = cj.ravel()
    v00 = vid(ci, cj)
    v10 = vid(ci + 1, cj)
    v11 = vid(ci + 1, cj + 1)
    v01 = vid(ci, cj + 1)
    t1 = np.stack([v00, v10, v11], axis=1)
    t2 = np.stack([v00, v11, v01], axis=1)
    tri = np.empty((2 * n * n, 3), dtype=np.int32)
    tri[0::2] = t1
    tri[1::2] = t2
    eps = 1e-12 * h
    node_in = ((x > o0 + eps) & (x < o1 - eps) & (y > o0 + eps) & (y < o1 - eps)).astype(np.uint8)
    bx = x[tri].mean(axis=1)
    by = y[tri].mean(axis=1)
    elem_in = ((bx > o0) & (bx < o1) & (by > o0) & (by < o1)).astype(np.uint8)
    return Mesh(vx=np.ascontiguousarray(x, dtype=np.float64),
                vy=np.ascontiguousarray(y, dtype=np.float64),
                tri=np.ascontiguousarray(tri), node_in_omega=node_in,
                elem_in_omega=elem_in, h=h, lo=lo, hi=hi, n=n)


def ngon_offsets(n: int, delta: float) -> np.ndarray:
    """Vertices of the regular inscribed N-gon relative to its centre:
    delta * (cos 2 pi k / N, sin 2 pi k / N), k = 0..N-1 (Sec. 9, regular
    inscribed polygon).  Shape [N, 2], float64, counter-clockwise."""
    k = np.arange(n, dtype=np.float64)
    ang = 2.0 * math.pi * k / n
    return np.ascontiguousarray(np.stack([delta * np.cos(ang), delta * np.sin(ang)], axis=1))


# ---------------------------------------------------------------------------
# Workload presets (ball, rules, kernel and mesh of each benchmark workload).
# Ball / rule / kernel / precision names are plain strings; each side maps them
# to its own enums.
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Problem:
    name: str
    mesh: Mesh
    delta: float
    kernel: str          # "const" | "inv_dist"
    kernel_c: float
    ball: str            # "barycenter" | "nocaps" | "approxcaps" | "exactcaps" | "ngon" | "overlap"
    outer: str           # "gauss3" | "gauss4" | "paper7" | "dunavant7" | "dunavant16" | "switch47"
    inner: str
    ngon_n: int = 0
    cap_m: int = 2
    ngon_off: np.ndarray | None = None

    def with_(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def const_kernel_c(delta: float) -> float:
    # psi = 4 / (pi delta^4)  (Sec. 8): makes L u = Laplacian u for cubics
    return 4.0 / (math.pi * delta ** 4)


def inv_dist_kernel_c(delta: float) -> float:
    # psi = 3 / (pi delta^3) / |x - y|: integral of |z| over B_delta is 2 pi delta^3 / 3
    return 3.0 / (math.pi * delta ** 3)


def problem(name: str) -> Problem:
    """Named workloads.  Sizes follow the benchmark configurations:

    barycenter_32   : (-0.1,1.1)^2, 32x32 structured, delta 0.1, barycenter ball,
                      7-point (degree-5) outer and inner rules, constant kernel.
    ngon32_96       : (-0.1,1.1)^2, 96x96 jittered +-0.2h (seed 1077502), delta 0.1,
                      regular 32-gon, 16-point outer, 7-point inner, constant kernel.
    singular_128    : (-0.05,1.05)^2, 128x128 jittered (seed 1077503), delta 0.05,
                      32-gon, psi = 3/(pi delta^3)/|x-y|, 16-point outer, 7-point inner.
    solve_220       : (-0.05,1.05)^2, 220x220 jittered (seed 1077505), delta 0.05, 32-gon,
                      16-point outer, 7-point inner (assembly followed by the CG solve).
    Small variants (suffix _small) keep the structure at sizes the oracle finishes in
    seconds.
    """
    d = 0.1
    if name == "barycenter_32":
        m = split_square_mesh(-0.1, 1.1, 32)
        return Problem(name, m, d, "const", const_kernel_c(d), "barycenter", "dunavant7", "dunavant7")
    if name == "barycenter_small":
        m = split_square_mesh(-0.1, 1.1, 12)
        return Problem(name, m, d, "const", const_kernel_c(d), "barycenter", "dunavant7", "dunavant7")
    if name in ("ngon32_96", "ngon32_small", "ngon32_mid"):
        n = {"ngon32_96": 96, "ngon32_small": 24, "ngon32_mid": 48}[name]
        m = split_square_mesh(-0.1, 1.1, n, jitter=0.2, seed=1077502)
        return Problem(name, m, d, "const", const_kernel_c(d), "ngon", "dunavant16", "dunavant7",
                       ngon_n=32, ngon_off=ngon_offsets(32, d))
    if name in ("singular_128", "singular_small"):
        dd, lo, hi, n = 0.05, -0.05, 1.05, 128
        if name == "singular_small":
            dd, lo, hi, n = 0.2, -0.2, 1.2, 16
        m = split_square_mesh(lo, hi, n, jitter=0.2, seed=1077503)
        return Problem(name, m, dd, "inv_dist", inv_dist_kernel_c(dd), "ngon", "dunavant16", "dunavant7",
                       ngon_n=32, ngon_off=ngon_offsets(32, dd))
    if name in ("solve_220",):
        dd = 0.05
        m = split_square_mesh(-0.05, 1.05, 220, jitter=0.2, seed=1077505)
        return Problem(name, m, dd, "const", const_kernel_c(dd), "ngon", "dunavant16", "dunavant7",
                       ngon_n=32, ngon_off=ngon_offsets(32, dd))
    raise KeyError(name)


BATCH_DELTAS = (0.05, 0.075, 0.1, 0.15, 0.2)


def batch_cells(delta: float, kmin: int = 2000, kmax: int = 40000, mmin: int = 3, mmax: int = 9):
    """Cells per side n of the meshes over (-delta, 1 + delta)^2 with delta / h = m an
    integer in [mmin, mmax] and K = 2 n^2 in [kmin, kmax]: n = m (1 + 2 delta) / delta."""
    out = []
    for m in range(mmin, mmax + 1):
        x = m * (1.0 + 2.0 * delta) / delta
        n = int(round(x))
        if abs(x - n) < 1e-9 and kmin <= 2 * n * n <= kmax:
            out.append(n)
    return out


def batch_problems(count: int = 64, seed: int = 1077600, kmin: int = 2000, kmax: int = 40000,
                   mmax: int = 9) -> list[Problem]:
    """The batched workload: `count` independent assemblies of uneven size and delta.

    Problem i: delta = BATCH_DELTAS[i % 5]; a mesh over (-delta, 1 + delta)^2 whose cells
    per side make delta / h an integer and K in [kmin, kmax] (drawn with a seeded PCG64
    among the admissible sizes); structured if i is even, else jittered +-0.2 h with seed
    seed + i; the paper's nocaps ball if i % 4 < 2, else approxcaps with one arc point per
    cap (m = 2); 7-point rules (degree 5) outer and inner; constant kernel 4 / (pi delta^4).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        d = BATCH_DELTAS[i % len(BATCH_DELTAS)]
        opts = batch_cells(d, kmin, kmax, 3, mmax)
        n = int(opts[int(rng.integers(len(opts)))])
        jit = 0.0 if i % 2 == 0 else 0.2
        m = split_square_mesh(-d, 1.0 + d, n, jitter=jit, seed=seed + i if jit else None)
        ball = "nocaps" if i % 4 < 2 else "approxcaps"
        out.append(Problem(f"batch{i}", m, d, "const", const_kernel_c(d), ball, "dunavant7", "dunavant7",
                           cap_m=2))
    return out


def paper_grid(h: float, warped: bool = False) -> Mesh:
    """Uniform grid (a) of Sec. 8 / Table 1: (-0.1, 1.1)^2 with cell size h (delta = 0.1); with
    warped=True the nonuniform grid (b) of Table 4, x2 -> x2^2 on the rows inside (0, 1)."""
    n = int(round(1.2 / h))
    return split_square_mesh(-0.1, 1.1, n, warp_y_square=warped)


def manufactured_u(x, y):
    """u = x1^2 x2 + x2^2 (Sec. 8)."""
    return x * x * y + y * y


def manufactured_f(x, y):
    """f = -Laplacian u = -2 (x2 + 1) (Sec. 8)."""
    return -2.0 * (y + 1.0)
