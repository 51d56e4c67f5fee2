"""The pins catch plausible mistakes (CPU only).  Each case compiles a copy of the oracle with
one mistake planted in its source (a dropped term, a wrong sign, a wrong index, a transposed
operand) and checks that the matrix-level pins fail on it: symmetry and zero row sums of D, the
closed form of a ball that covers the mesh, and the quadratic manufactured solution on the
N-gon.  The unmodified source passes the same checks."""
import math
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_2005_10775_gb300 import inputs as I

MUTANTS = [
    ("dropped M_bb block", "hm_add(&maps[tid], (int64_t)bi * m->nv + bk, Mbb[i][k]);", "(void)0;"),
    ("wrong sign of the transposed M_ab block", "(int64_t)bk * m->nv + ai, -Mab[i][k]",
     "(int64_t)bk * m->nv + ai, +Mab[i][k]"),
    ("transposed M_ab operand", "(int64_t)ai * m->nv + bk, -Mab[i][k]", "(int64_t)ai * m->nv + bk, -Mab[k][i]"),
    ("wrong index in the inner phi_b phi_b sum", "I->S2[i][k] += omega * phi[i] * phi[k];",
     "I->S2[i][k] += omega * phi[i] * phi[i];"),
    ("wrong index in the outer phi_a phi_a product", "Maa[i][k] += W * I.s0 * L[i] * L[k];",
     "Maa[i][k] += W * I.s0 * L[i] * L[i];"),
    ("dropped barycentric term", "phi[0] = 1.0 - l1 - l2;", "phi[0] = 1.0 - l1;"),
    ("outer weight without |T_a|", "double W = L[3] * area_a;", "double W = L[3];"),
]


def _compile(tmp_path, name, src):
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"lib{name}.so"
    c.write_text(src)
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
                           "-o", str(so), str(c), "-lm"])
    return O.load(str(so))


def _failures():
    """The matrix-level pins that fail for the oracle currently loaded."""
    failed = []
    # symmetry and zero row sums of D (full Omega u Omega_I matrix), N-gon, jittered mesh
    m = I.split_square_mesh(-0.3, 1.3, 8, jitter=0.2, seed=5)
    d = 0.45
    cfg = dict(delta=d, ball="ngon", ngon_off=I.ngon_offsets(32, d), outer="dunavant7", inner="dunavant7",
               kernel_c=I.const_kernel_c(d))
    D = O.to_csr(O.assemble(m, cfg)).toarray()
    scale = np.abs(D).max()
    if not (np.abs(D - D.T).max() <= 1e-12 * scale and np.abs(D.sum(axis=1)).max() <= 1e-12 * scale):
        failed.append("structure")
    # a ball covering the mesh: D = c (2 |Omega| M - 2 m m^T)
    mc = I.split_square_mesh(0.0, 1.0, 3, jitter=0.2, seed=9, omega=(-1, 2))
    c = 0.37
    Dc = O.to_csr(O.assemble(mc, dict(delta=20.0, ball="nocaps", outer="dunavant7", inner="dunavant7",
                                      kernel_c=c))).toarray()
    M = np.zeros((mc.nv, mc.nv))
    mm = np.zeros(mc.nv)
    tot = 0.0
    for t in mc.tri:
        V = np.stack([mc.vx[t], mc.vy[t]], axis=1)
        A = 0.5 * abs((V[1, 0] - V[0, 0]) * (V[2, 1] - V[0, 1]) - (V[2, 0] - V[0, 0]) * (V[1, 1] - V[0, 1]))
        tot += A
        M[np.ix_(t, t)] += A * (np.ones((3, 3)) + np.eye(3)) / 12
        mm[t] += A / 3
    ref = c * (2 * tot * M - 2 * np.outer(mm, mm))
    if not np.abs(Dc - ref).max() <= 1e-12 * np.abs(ref).max():
        failed.append("covering ball")
    # u = |x|^2 on the 32-gon: (D U)_j = -(2N / 3 pi) sin(2 pi / N) (2 + cos(2 pi / N)) int phi_j
    d, N, n = 0.1, 32, 24
    mq = I.split_square_mesh(-d, 1 + d, n)
    Dq = O.to_csr(O.assemble(mq, dict(delta=d, ball="ngon", ngon_off=I.ngon_offsets(N, d), outer="dunavant7",
                                      inner="dunavant7", kernel_c=I.const_kernel_c(d))))
    mass = np.zeros(mq.nv)
    for t in mq.tri:
        V = np.stack([mq.vx[t], mq.vy[t]], axis=1)
        mass[t] += 0.5 * abs((V[1, 0] - V[0, 0]) * (V[2, 1] - V[0, 1]) - (V[2, 0] - V[0, 0]) * (V[1, 1] - V[0, 1])) / 3
    h = 1.2 / n
    far = (mq.vx > 2 * d + h) & (mq.vx < 1 - d - h) & (mq.vy > 2 * d + h) & (mq.vy < 1 - d - h)
    want = -(2 * N / (3 * math.pi)) * math.sin(2 * math.pi / N) * (2 + math.cos(2 * math.pi / N))
    got = (Dq @ (mq.vx ** 2 + mq.vy ** 2))[far] / mass[far]
    if not np.abs(got - want).max() <= 1e-10:
        failed.append("quadratic")
    return failed


@pytest.fixture(scope="module")
def source():
    with open(O.SRC) as f:
        return f.read()


def test_unmodified_oracle_passes(tmp_path, monkeypatch, source):
    monkeypatch.setattr(O, "_LIB", _compile(tmp_path, "clean", source))
    assert _failures() == []


@pytest.mark.parametrize("what,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, monkeypatch, source, what, old, new):
    assert source.count(old) >= 1, f"{what}: the line to mutate is not in the oracle"
    monkeypatch.setattr(O, "_LIB", _compile(tmp_path, "mutant", source.replace(old, new)))
    assert _failures() != [], f"no pin caught: {what}"


# --------------------------------------------------------------------------
# geometry mistakes against the region pins
# --------------------------------------------------------------------------

REGION_MUTANTS = [
    ("wrong N-gon clip intersection parameter", "double t = ds / (ds - de);", "double t = de / (ds - de);"),
    ("wrong circle-edge root", "    double l2 = (-bh + s) / a;\n", "    double l2 = (-bh + s) / (2.0 * a);\n"),
    ("cap area halved", "*area = delta * delta * two_th_minus_sin / (printed ? 4.0 : 2.0);",
     "*area = delta * delta * two_th_minus_sin / (printed ? 4.0 : 4.0);"),
    ("arc point off the circle", "double s = delta / sqrt(ux * ux + uy * uy);",
     "double s = 0.5 * delta / sqrt(ux * ux + uy * uy);"),
    ("entry and exit roots swapped", "lam[0] = l1; is_entry[0] = 1;", "lam[0] = l1; is_entry[0] = 0;"),
    ("cap centroid off", "4.0 * delta * st * st * st / (3.0 * two_th_minus_sin)",
     "2.0 * delta * st * st * st / (3.0 * two_th_minus_sin)"),
    ("overlap test without its edge-crossing branch",
     "if ((l1 >= 0.0 && l1 <= 1.0) || (l2 >= 0.0 && l2 <= 1.0)) return 1;", "(void)l1; (void)l2;"),
    ("overlap test without its enclosing branch", "int in = 1;", "int in = 0;"),
    ("overlap test with a strict vertex test", "for (int i = 0; i < 3; i++) if (in_ball(V[i], x, d2)) return 1;",
     "for (int i = 0; i < 3; i++) if (in_ball(V[i], x, 0.25 * d2)) return 1;"),
]


def _region_failures():
    """The region-level pins (tests/test_oracle_pins.py) that fail for the oracle loaded."""
    import test_oracle_pins as P
    checks = [P.test_nocaps_exactcaps_quarter_disc, P.test_approxcaps_quarter_disc,
              P.test_ngon_clip_matches_independent_intersection, P.test_support_nesting,
              P.test_one_edge_cut_twice, P.test_tangent_edge_gives_zero_cap,
              lambda: P.test_ngon_area_and_moments(0.2), lambda: P.test_exactcaps_and_approxcaps_area(0.2),
              lambda: P.test_ball_covering_mesh_closed_form("exactcaps", "dunavant7", "dunavant7"),
              P.test_overlap_ball_is_the_distance_test]
    failed = []
    for k, f in enumerate(checks):
        try:
            f()
        except AssertionError:
            failed.append(k)
    return failed


def test_unmodified_oracle_passes_the_region_pins(tmp_path, monkeypatch, source):
    monkeypatch.setattr(O, "_LIB", _compile(tmp_path, "clean", source))
    assert _region_failures() == []


@pytest.mark.parametrize("what,old,new", REGION_MUTANTS, ids=[m[0] for m in REGION_MUTANTS])
def test_planted_geometry_mistake_is_caught(tmp_path, monkeypatch, source, what, old, new):
    assert source.count(old) >= 1, f"{what}: the line to mutate is not in the oracle"
    monkeypatch.setattr(O, "_LIB", _compile(tmp_path, "mutant", source.replace(old, new)))
    assert _region_failures() != [], f"no pin caught: {what}"


# --------------------------------------------------------------------------
# near-singular rule mistakes against the singular-kernel pins
# --------------------------------------------------------------------------

NEAR_MUTANTS = [
    ("wrong side of the edge's foot", "double sigma = (fx * ey - fy * ex) > 0.0 ? 1.0 : -1.0;",
     "double sigma = (fx * ey - fy * ex) > 0.0 ? -1.0 : 1.0;"),
    ("one right triangle of each edge dropped", "        near_right_triangle(cfg, Vb, x, F, ex, ey, d, tA, -sigma, I);\n",
     "        (void)0;\n"),
    ("sinh substitution without its Jacobian d", "add_point(I, Vb, y, sign * sg * d * ws * wu * cfg->kernel_c);",
     "add_point(I, Vb, y, sign * sg * ws * wu * cfg->kernel_c);"),
    ("Duffy point not scaled in x", "y.x = x.x + sv * wx;", "y.x = x.x + wx;"),
]


def _near_failures():
    import test_oracle_pins as P
    failed = []
    for k, f in enumerate([P.test_singular_kernel_ngon_closed_forms, P.test_quadratic_manufactured_solution]):
        try:
            f()
        except AssertionError:
            failed.append(k)
    return failed


def test_unmodified_oracle_passes_the_singular_pins(tmp_path, monkeypatch, source):
    monkeypatch.setattr(O, "_LIB", _compile(tmp_path, "clean", source))
    assert _near_failures() == []


@pytest.mark.parametrize("what,old,new", NEAR_MUTANTS, ids=[m[0] for m in NEAR_MUTANTS])
def test_planted_near_rule_mistake_is_caught(tmp_path, monkeypatch, source, what, old, new):
    assert source.count(old) >= 1, f"{what}: the line to mutate is not in the oracle"
    monkeypatch.setattr(O, "_LIB", _compile(tmp_path, "mutant", source.replace(old, new)))
    assert _near_failures() != [], f"no pin caught: {what}"


# --------------------------------------------------------------------------
# the outer-support (barycenter ball, Sec. 6.2) composite against its pins
# --------------------------------------------------------------------------

SUPPORT_MUTANTS = [
    ("support M_bb dropped", "                                Mbb[i][k2] += W * I.S2[i][k2];\n", "(void)0;\n"),
    ("support outer weight without the subtriangle area", "const double W = L[3] * area;",
     "const double W = L[3];"),
    ("support outer point from two vertices", "x.x = L[0] * S0.x + L[1] * S1.x + L[2] * S2p.x;",
     "x.x = L[0] * S0.x + L[1] * S1.x + L[2] * S1.x;"),
]


def _support_failures():
    import test_oracle_pins as P
    failed = []
    checks = [lambda: P.test_outer_support_matrix_structure("bary_nocaps"),
              lambda: P.test_shifted_ball_equals_barycenter_outer_support("nocaps")]
    for k, f in enumerate(checks):
        try:
            f()
        except AssertionError:
            failed.append(k)
    return failed


def test_unmodified_oracle_passes_the_support_pins(tmp_path, monkeypatch, source):
    monkeypatch.setattr(O, "_LIB", _compile(tmp_path, "clean", source))
    assert _support_failures() == []


@pytest.mark.parametrize("what,old,new", SUPPORT_MUTANTS, ids=[m[0] for m in SUPPORT_MUTANTS])
def test_planted_support_mistake_is_caught(tmp_path, monkeypatch, source, what, old, new):
    assert source.count(old) == 1, f"{what}: the line to mutate is not in the oracle once"
    monkeypatch.setattr(O, "_LIB", _compile(tmp_path, "mutant", source.replace(old, new)))
    assert _support_failures() != [], f"no pin caught: {what}"
