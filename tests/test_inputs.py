"""The seeded synthetic workloads (CPU only): sizes, domains, horizons, kernels and balls of the
named problems and of the 64-problem batch as stated for the benchmark configurations, valid
meshes (counter-clockwise, non-degenerate, conforming split squares), the jitter bound, and
repeatability from the seed."""
import math

import numpy as np
import pytest

from paper_2005_10775_gb300 import inputs as I


def _signed_areas(m):
    V = np.stack([m.vx[m.tri], m.vy[m.tri]], axis=-1)   # [K, 3, 2]
    e1, e2 = V[:, 1] - V[:, 0], V[:, 2] - V[:, 0]
    return 0.5 * (e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])


def _check_mesh(m, lo, hi, n, jitter):
    h = (hi - lo) / n
    assert m.n == n and m.h == pytest.approx(h)
    assert m.nt == 2 * n * n and m.nv == (n + 1) ** 2
    assert m.tri.dtype == np.int32 and m.tri.min() == 0 and m.tri.max() == m.nv - 1
    A = _signed_areas(m)
    assert A.min() > 0.0                                   # counter-clockwise, non-degenerate
    assert A.sum() == pytest.approx((hi - lo) ** 2, rel=1e-12)   # the triangles tile the square
    assert m.vx.min() == pytest.approx(lo) and m.vx.max() == pytest.approx(hi)
    assert m.vy.min() == pytest.approx(lo) and m.vy.max() == pytest.approx(hi)
    ii, jj = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="xy")
    dx = np.abs(m.vx - (lo + ii.ravel() * h))
    dy = np.abs(m.vy - (lo + jj.ravel() * h))
    assert max(dx.max(), dy.max()) <= jitter * h + 1e-12   # (grid lines snapped to 0 and 1 move by an ulp)
    if jitter > 0:
        assert max(dx.max(), dy.max()) > 0.5 * jitter * h


@pytest.mark.parametrize("name,lo,hi,n,delta,ball,kernel,outer,inner,jitter", [
    ("barycenter_32", -0.1, 1.1, 32, 0.1, "barycenter", "const", "dunavant7", "dunavant7", 0.0),
    ("ngon32_96", -0.1, 1.1, 96, 0.1, "ngon", "const", "dunavant16", "dunavant7", 0.2),
    ("singular_128", -0.05, 1.05, 128, 0.05, "ngon", "inv_dist", "dunavant16", "dunavant7", 0.2),
    ("solve_220", -0.05, 1.05, 220, 0.05, "ngon", "const", "dunavant16", "dunavant7", 0.2),
])
def test_named_workloads(name, lo, hi, n, delta, ball, kernel, outer, inner, jitter):
    p = I.problem(name)
    _check_mesh(p.mesh, lo, hi, n, jitter)
    assert (p.delta, p.ball, p.kernel, p.outer, p.inner) == (delta, ball, kernel, outer, inner)
    if kernel == "const":
        assert p.kernel_c == pytest.approx(4 / (math.pi * delta ** 4))
    else:
        assert p.kernel_c == pytest.approx(3 / (math.pi * delta ** 3))
    if ball == "ngon":
        assert p.ngon_n == 32 and p.ngon_off.shape == (32, 2)
        r = np.hypot(p.ngon_off[:, 0], p.ngon_off[:, 1])
        np.testing.assert_allclose(r, delta, rtol=1e-15)   # vertices on the circle of radius delta
    # the horizon exceeds every triangle's diameter (the method's standing assumption)
    V = np.stack([p.mesh.vx[p.mesh.tri], p.mesh.vy[p.mesh.tri]], axis=-1)
    diam = max(np.hypot(*(V[:, i] - V[:, k]).T).max() for i, k in ((0, 1), (1, 2), (0, 2)))
    assert delta > diam


def test_omega_labels():
    # nodes strictly inside (0, 1)^2 belong to Omega, the rest (boundary included) to Omega_I;
    # an element belongs to Omega when its barycentre does
    m = I.problem("solve_220").mesh
    inside = (m.vx > 0) & (m.vx < 1) & (m.vy > 0) & (m.vy < 1)
    np.testing.assert_array_equal(m.node_in_omega.astype(bool), inside)
    assert int(m.node_in_omega.sum()) == 39601            # the 199 x 199 interior nodes
    bx, by = m.vx[m.tri].mean(axis=1), m.vy[m.tri].mean(axis=1)
    np.testing.assert_array_equal(m.elem_in_omega.astype(bool), (bx > 0) & (bx < 1) & (by > 0) & (by < 1))


def test_seeded_meshes_repeat():
    a, b = I.problem("ngon32_small").mesh, I.problem("ngon32_small").mesh
    np.testing.assert_array_equal(a.vx, b.vx)
    np.testing.assert_array_equal(a.vy, b.vy)
    c = I.split_square_mesh(-0.1, 1.1, 24, jitter=0.2, seed=1)
    assert not np.array_equal(a.vx, c.vx)


def test_batch_workload():
    P = I.batch_problems()
    assert len(P) == 64
    Ks = [p.mesh.nt for p in P]
    assert min(Ks) == 2450 and max(Ks) == 38088 and sum(Ks) == 731278
    for i, p in enumerate(P):
        d = I.BATCH_DELTAS[i % 5]
        assert p.delta == d and p.kernel == "const" and p.cap_m == 2
        assert p.ball == ("nocaps" if i % 4 < 2 else "approxcaps")
        assert (p.outer, p.inner) == ("dunavant7", "dunavant7")
        n = p.mesh.n
        _check_mesh(p.mesh, -d, 1 + d, n, 0.0 if i % 2 == 0 else 0.2)
        assert d / p.mesh.h == pytest.approx(round(d / p.mesh.h))   # delta / h an integer
        assert 2000 <= p.mesh.nt <= 40000
    assert [p.mesh.nt for p in I.batch_problems()] == Ks    # seeded


def test_paper_grids():
    # grid (a) of Sec. 8 and its warped variant (b): x2 -> x2^2 on the rows inside (0, 1)
    a, b = I.paper_grid(0.05), I.paper_grid(0.05, warped=True)
    _check_mesh(a, -0.1, 1.1, 24, 0.0)
    assert _signed_areas(b).min() > 0
    inside = (a.vy > 1e-12) & (a.vy < 1 - 1e-12)
    np.testing.assert_allclose(b.vy[inside], a.vy[inside] ** 2, rtol=0, atol=1e-15)
    np.testing.assert_array_equal(b.vy[~inside], a.vy[~inside])
    np.testing.assert_array_equal(b.vx, a.vx)
