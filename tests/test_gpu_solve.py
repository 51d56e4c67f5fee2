"""Right-hand side and solve on the GPU (through the C ABI) against the oracle's
numpy/scipy steps: A = D[Omega, Omega], B = D[Omega, Omega_I], F = G - B g,
matrix-vector products and the mixed-precision CG solve."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2005_10775_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nl():
    from paper_2005_10775_gb300 import nlfem
    return nlfem


@pytest.fixture(scope="module")
def ctx(nl):
    c = nl.nl_create(0)
    yield c
    nl.nl_destroy(c)


@pytest.fixture(scope="module")
def system(nl, ctx):
    d = 0.1
    m = I.split_square_mesh(-0.1, 1.1, 36, jitter=0.2, seed=1077505)
    p = I.Problem("solve", m, d, "const", I.const_kernel_c(d), "ngon", "dunavant7", "dunavant7", ngon_n=32,
                  ngon_off=I.ngon_offsets(32, d))
    keep = nl._Keep()
    mesh = nl.make_mesh(m, keep)
    cfg = nl.config_of(p, keep, prec="fp64")
    D = nl.nl_assemble(ctx, mesh, cfg)
    A, B = nl.nl_extract(ctx, D, mesh)
    out = O.assemble(m, dict(delta=d, ball="ngon", outer="dunavant7", inner="dunavant7",
                             kernel_c=p.kernel_c, ngon_off=p.ngon_off))
    yield dict(m=m, mesh=mesh, keep=keep, D=D, A=A, B=B, Do=O.to_csr(out))
    for x in (D, A, B):
        nl.nl_csr_free(ctx, x)


def test_extract(nl, ctx, system):
    m = system["m"]
    om = m.node_in_omega.astype(bool)
    Ao = system["Do"][om][:, om].tocsr()
    Bo = system["Do"][om][:, ~om].tocsr()
    Ag = nl.to_scipy(ctx, system["A"])
    Bg = nl.to_scipy(ctx, system["B"], ncols=int((~om).sum()))
    for G, R in ((Ag, Ao), (Bg, Bo)):
        R.sort_indices()
        np.testing.assert_array_equal(G.indptr, R.indptr)
        np.testing.assert_array_equal(G.indices, R.indices)
        assert np.abs(G.data - R.data).max() <= 1e-12 * np.abs(system["Do"].data).max()


def test_rhs(nl, ctx, system):
    m = system["m"]
    u = I.manufactured_u(m.vx, m.vy)
    f = I.manufactured_f(m.vx, m.vy)
    F = nl.nl_rhs(ctx, system["B"], system["mesh"], f, u)
    Fo = O.rhs(system["Do"], m, f, u)
    np.testing.assert_allclose(F, Fo, rtol=0, atol=1e-12 * np.abs(Fo).max())


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32c", 2e-6)])
def test_matvec(nl, ctx, system, prec, tol):
    m = system["m"]
    om = m.node_in_omega.astype(bool)
    Ao = system["Do"][om][:, om]
    x = np.random.default_rng(3).standard_normal(Ao.shape[0])
    y = nl.nl_matvec(ctx, system["A"], x, prec=prec)
    ref = Ao @ x
    assert np.abs(y - ref).max() <= tol * np.abs(Ao).sum(axis=1).max() * np.abs(x).max()


def test_cg_solve_matches_direct(nl, ctx, system):
    m = system["m"]
    u = I.manufactured_u(m.vx, m.vy)
    f = I.manufactured_f(m.vx, m.vy)
    om = m.node_in_omega.astype(bool)
    F = nl.nl_rhs(ctx, system["B"], system["mesh"], f, u)
    x = np.zeros(F.shape[0])
    it, rel = nl.nl_cg(ctx, system["A"], F, x, rtol=1e-10, max_it=5000)
    assert rel <= 1e-10 and it > 0
    Uo = O.solve(system["Do"], m, f, u)[om]
    assert np.abs(x - Uo).max() <= 1e-8 * np.abs(Uo).max()
    # the discrete solution approximates u = x1^2 x2 + x2^2 (Sec. 8)
    assert np.abs(x - u[om]).max() < 5e-2


def test_cg_reports_nonconvergence(nl, ctx, system):
    F = np.ones(system["A"].n)
    x = np.zeros_like(F)
    with pytest.raises(nl.NlError) as e:
        nl.nl_cg(ctx, system["A"], F, x, rtol=1e-14, max_it=3)
    assert e.value.status == nl.NL_ENOCONV


def test_cg_unreachable_tolerance_is_not_success(nl, ctx, system):
    # rtol below the FP64 residual floor with iterations to spare: the refinement passes run
    # out before ||b - Ax|| <= rtol ||b||, which is a failure, not a converged solve
    F = np.ones(system["A"].n)
    x = np.zeros_like(F)
    with pytest.raises(nl.NlError) as e:
        nl.nl_cg(ctx, system["A"], F, x, rtol=1e-18, max_it=200000)
    assert e.value.status == nl.NL_ENOCONV
    assert np.isfinite(x).all()


def test_cg_rejects_nan_right_hand_side(nl, ctx, system):
    F = np.ones(system["A"].n)
    F[F.shape[0] // 2] = np.nan
    x = np.zeros_like(F)
    with pytest.raises(nl.NlError) as e:
        nl.nl_cg(ctx, system["A"], F, x, rtol=1e-10, max_it=5000)
    assert e.value.status == nl.NL_EINVAL


def test_cg_reports_breakdown_on_indefinite_matrix(nl, ctx, system):
    # -A is negative definite: the first direction has p.Ap < 0, a breakdown (not convergence)
    torch = pytest.importorskip("torch")
    import ctypes
    A = system["A"]
    keep = []
    val = torch.empty(A.nnz, dtype=torch.float64, device="cuda")
    rp = torch.empty(A.n + 1, dtype=torch.int64, device="cuda")
    col = torch.empty(A.nnz, dtype=torch.int32, device="cuda")
    Ah = nl.to_scipy(ctx, A)
    val.copy_(torch.tensor(-Ah.data))
    rp.copy_(torch.tensor(Ah.indptr.astype(np.int64)))
    col.copy_(torch.tensor(Ah.indices.astype(np.int32)))
    keep += [val, rp, col]
    neg = nl.nl_csr(n=A.n, nnz=A.nnz, row_ptr=ctypes.c_void_p(rp.data_ptr()), col_idx=ctypes.c_void_p(col.data_ptr()),
                    val=ctypes.c_void_p(val.data_ptr()))
    F = np.ones(A.n)
    x = np.zeros_like(F)
    try:
        with pytest.raises(nl.NlError) as e:
            nl.nl_cg(ctx, neg, F, x, rtol=1e-10, max_it=5000)
        assert e.value.status == nl.NL_ENOCONV
        assert "breakdown" in str(e.value)
    finally:
        # release the FP32 copy of the values the call made; the arrays themselves are torch's
        neg.row_ptr = neg.col_idx = neg.val = None
        nl.nl_csr_free(ctx, neg)


def _golden(name):
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    rows = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            rows[(f[0], float(f[1]))] = float(f[2])
    return rows


def gpu_l2_error(nl, ctx, m, ball, outer, inner, prec="fp32c", **over):
    """The whole pipeline on the GPU (assembly, extraction, right-hand side, CG to 1e-10) for the
    manufactured solution u = x1^2 x2 + x2^2 of Sec. 8; the L2(Omega) error of u_h."""
    d = 0.1
    p = I.Problem("paper", m, d, "const", I.const_kernel_c(d), ball, outer, inner)
    keep = nl._Keep()
    mesh = nl.make_mesh(m, keep)
    D = nl.nl_assemble(ctx, mesh, nl.config_of(p, keep, prec=prec, **over))
    A, B = nl.nl_extract(ctx, D, mesh)
    try:
        u = I.manufactured_u(m.vx, m.vy)
        F = nl.nl_rhs(ctx, B, mesh, I.manufactured_f(m.vx, m.vy), u)
        x = np.zeros(A.n)
        nl.nl_cg(ctx, A, F, x, rtol=1e-10, max_it=20000)
    finally:
        for z in (D, A, B):
            nl.nl_csr_free(ctx, z)
    U = u.copy()
    U[m.node_in_omega.astype(bool)] = x
    return O.l2_error_omega(m, U, I.manufactured_u)


# Table 1 (Sec. 8) end to end on the GPU with the paper's rule protocol (outer gauss4 / paper7 by
# the switch, inner gauss3, caps one centroid point with the printed weight), against the printed
# L2 errors (tests/golden/paper_table1.txt) within 15 %, from h = delta = 0.1 (diameters above
# delta) to the finest grid h = 0.00625 (K = 73728).  Not listed: the barycenter column (not
# reproduced, a documented reading) and nocaps at h = 0.1 (checked against the oracle below).
TABLE1_GPU = ([("exactcaps", h) for h in (0.1, 0.05, 0.025, 0.0125)] +
              [("approxcaps", h) for h in (0.1, 0.05, 0.025, 0.0125, 0.00625)] +
              [("nocaps", h) for h in (0.05, 0.025, 0.0125, 0.00625)] +
              [("overlap", h) for h in (0.1, 0.05, 0.025, 0.0125)])


@pytest.mark.parametrize("ball,h", TABLE1_GPU)
def test_paper_table1_end_to_end_on_gpu(nl, ctx, ball, h):
    over = {"cap_printed": 1} if ball == "exactcaps" else {}
    err = gpu_l2_error(nl, ctx, I.paper_grid(h), ball, "switch47", "gauss3", **over)
    assert err == pytest.approx(_golden("paper_table1.txt")[(ball, h)], rel=0.15)


def test_paper_table1_nocaps_coarsest_grid_matches_oracle(nl, ctx):
    # nocaps at h = delta = 0.1: the oracle's L2 error is 0.66 x the printed one (a documented
    # reading); the GPU pipeline reproduces the oracle's value
    m = I.paper_grid(0.1)
    err = gpu_l2_error(nl, ctx, m, "nocaps", "switch47", "gauss3", prec="fp64")
    d = 0.1
    cfg = dict(delta=d, ball="nocaps", outer="switch47", inner="gauss3", kernel_c=I.const_kernel_c(d))
    ref = O.l2_error_omega(m, O.solve(O.to_csr(O.assemble(m, cfg)), m, I.manufactured_f(m.vx, m.vy),
                                      I.manufactured_u(m.vx, m.vy)), I.manufactured_u)
    assert err == pytest.approx(ref, rel=1e-6)


@pytest.mark.parametrize("ball", ["bary_nocaps", "bary_approxcaps"])
def test_paper_table4b_nonuniform_grid_on_gpu(nl, ctx, ball):
    # grid (b) of Sec. 8 (x2 -> x2^2 inside (0, 1); h_max 0.2147, 0.1096, 0.0553 against delta = 0.1),
    # barycenter ball with the outer integral over its support, gauss4 outer / gauss3 inner (Table 4(b)):
    # the GPU pipeline gives the oracle's L2 errors at every grid, and their second-order rate
    errs = []
    d = 0.1
    for h in (0.1, 0.05, 0.025):
        m = I.paper_grid(h, warped=True)
        err = gpu_l2_error(nl, ctx, m, ball, "gauss4", "gauss3", prec="fp64")
        cfg = dict(delta=d, ball=ball, outer="gauss4", inner="gauss3", kernel_c=I.const_kernel_c(d))
        ref = O.l2_error_omega(m, O.solve(O.to_csr(O.assemble(m, cfg)), m, I.manufactured_f(m.vx, m.vy),
                                          I.manufactured_u(m.vx, m.vy)), I.manufactured_u)
        assert err == pytest.approx(ref, rel=1e-6), h
        errs.append(err)
    assert 1.6 < np.log2(errs[1] / errs[2]) < 2.4
    printed = _golden("paper_table4b.txt")
    assert 0.3 < errs[2] / printed[(ball, 0.025)] < 3.0


def test_paper_table2_shifted_nocaps_on_gpu(nl, ctx):
    # Table 2, column (6): shifted-centre ball with nocaps, 4-point outer and 3-point inner rules,
    # assembled, extracted and solved on the GPU (h = 0.05, printed L2 error 6.89e-3)
    d, h = 0.1, 0.05
    m = I.paper_grid(h)
    p = I.Problem("paper", m, d, "const", I.const_kernel_c(d), "nocaps", "gauss4", "gauss3")
    keep = nl._Keep()
    mesh = nl.make_mesh(m, keep)
    D = nl.nl_assemble(ctx, mesh, nl.config_of(p, keep, prec="fp32c", shifted=1))
    A, B = nl.nl_extract(ctx, D, mesh)
    try:
        u = I.manufactured_u(m.vx, m.vy)
        F = nl.nl_rhs(ctx, B, mesh, I.manufactured_f(m.vx, m.vy), u)
        x = np.zeros(A.n)
        nl.nl_cg(ctx, A, F, x, rtol=1e-10, max_it=20000)
    finally:
        for z in (D, A, B):
            nl.nl_csr_free(ctx, z)
    U = u.copy()
    U[m.node_in_omega.astype(bool)] = x
    assert O.l2_error_omega(m, U, I.manufactured_u) == pytest.approx(6.89e-3, rel=0.15)


@pytest.mark.parametrize("ball,ref", [("bary_nocaps", 7.47e-3), ("bary_approxcaps", 9.68e-3)])
def test_paper_table3_on_gpu(nl, ctx, ball, ref):
    # Table 3, columns (7) and (8): barycenter ball with the outer integral over its support,
    # 4-point outer (on T_a or each support subtriangle) and 3-point inner rules, h = 0.05
    d, h = 0.1, 0.05
    m = I.paper_grid(h)
    p = I.Problem("paper", m, d, "const", I.const_kernel_c(d), ball, "gauss4", "gauss3", cap_m=2)
    keep = nl._Keep()
    mesh = nl.make_mesh(m, keep)
    D = nl.nl_assemble(ctx, mesh, nl.config_of(p, keep, prec="fp32c"))
    A, B = nl.nl_extract(ctx, D, mesh)
    try:
        u = I.manufactured_u(m.vx, m.vy)
        F = nl.nl_rhs(ctx, B, mesh, I.manufactured_f(m.vx, m.vy), u)
        x = np.zeros(A.n)
        nl.nl_cg(ctx, A, F, x, rtol=1e-10, max_it=20000)
    finally:
        for z in (D, A, B):
            nl.nl_csr_free(ctx, z)
    U = u.copy()
    U[m.node_in_omega.astype(bool)] = x
    assert O.l2_error_omega(m, U, I.manufactured_u) == pytest.approx(ref, rel=0.05)

