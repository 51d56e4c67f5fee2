"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bar (the FP64 bar is the FP64 path's rounding; the FP32 bar is the FP32
unit round-off times the quadrature's term count, with margin):
  * CSR pattern (row pointers, column indices) and the interaction set
    (per-outer-triangle count, qp-pair count and record hash) are bit-exact;
  * values: |D_gpu - D_oracle| <= 1e-12 max|D| for the FP64 path and
    <= 1e-6 max|D| for the FP32-compensated path.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2005_10775_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32c": 1e-6}


@pytest.fixture(scope="module")
def nl():
    from paper_2005_10775_gb300 import nlfem
    return nlfem


@pytest.fixture(scope="module")
def ctx(nl):
    c = nl.nl_create(0)
    yield c
    nl.nl_destroy(c)


def oracle_cfg(p, **over):
    kw = dict(delta=p.delta, ball=p.ball, outer=p.outer, inner=p.inner, kernel=p.kernel, kernel_c=p.kernel_c,
              ngon_off=p.ngon_off, cap_m=p.cap_m)
    kw.update(over)
    return kw


def gpu_assemble(nl, ctx, p, prec, **over):
    keep = nl._Keep()
    mesh = nl.make_mesh(p.mesh, keep)
    cfg = nl.config_of(p, keep, prec=prec, **over)
    m = nl.nl_assemble(ctx, mesh, cfg)
    try:
        D = nl.to_scipy(ctx, m)
        stats = (m.n_pairs, m.n_qp_pairs, m.n_inter)
    finally:
        nl.nl_csr_free(ctx, m)
    return D, stats


def gpu_interactions(nl, ctx, p, **over):
    keep = nl._Keep()
    mesh = nl.make_mesh(p.mesh, keep)
    cfg = nl.config_of(p, keep, **over)
    return nl.nl_interactions(ctx, mesh, cfg)


def compare(Dg, Do, prec):
    Do = Do.tocsr()
    Do.sort_indices()
    np.testing.assert_array_equal(Dg.indptr, Do.indptr)
    np.testing.assert_array_equal(Dg.indices, Do.indices)
    scale = np.abs(Do.data).max()
    err = np.abs(Dg.data - Do.data).max() / scale
    assert err <= TOL[prec], err
    return err


def small_problem(ball, n=24, jitter=0.2, kernel="const", **kw):
    d = 0.1
    m = I.split_square_mesh(-0.1, 1.1, n, jitter=jitter, seed=1077502)
    c = I.const_kernel_c(d) if kernel == "const" else I.inv_dist_kernel_c(d)
    p = I.Problem(f"{ball}_{n}", m, d, kernel, c, ball, "dunavant7", "dunavant7")
    if ball == "ngon":
        p = p.with_(ngon_n=32, ngon_off=I.ngon_offsets(32, d))
    return p.with_(**kw) if kw else p


CASES = [
    ("barycenter", {}), ("nocaps", {}), ("approxcaps", {}), ("approxcaps", {"cap_m": 4}),
    ("exactcaps", {}), ("ngon", {}), ("overlap", {}),
    ("bary_nocaps", {}), ("bary_approxcaps", {}),
]


@pytest.mark.parametrize("ball,kw", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_parity_small(nl, ctx, ball, kw, prec):
    p = small_problem(ball, **kw)
    out = O.assemble(p.mesh, oracle_cfg(p), want_hash=True)
    Dg, stats = gpu_assemble(nl, ctx, p, prec)
    compare(Dg, O.to_csr(out), prec)
    assert stats == (out["n_pairs"], out["n_qp_pairs"], out["n_inter"])
    # the interaction records of the same precision's path (FP32 paths certify their regions)
    h, c, q = gpu_interactions(nl, ctx, p, prec=prec)
    np.testing.assert_array_equal(c, out["count_a"])
    np.testing.assert_array_equal(q, out["qp_a"])
    np.testing.assert_array_equal(h, out["hash_a"])


def test_parity_barycenter_32_full_size(nl, ctx):
    # barycenter ball, 32x32 structured grid (2048 triangles), 7-point rules, FP64
    p = I.problem("barycenter_32")
    out = O.assemble(p.mesh, oracle_cfg(p), want_hash=True)
    Dg, stats = gpu_assemble(nl, ctx, p, "fp64")
    compare(Dg, O.to_csr(out), "fp64")
    assert stats == (out["n_pairs"], out["n_qp_pairs"], out["n_inter"])
    h, c, q = gpu_interactions(nl, ctx, p)
    np.testing.assert_array_equal(h, out["hash_a"])


@pytest.mark.parametrize("ball", ["ngon", "approxcaps", "nocaps", "barycenter"])
@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_parity_inv_dist_kernel(nl, ctx, ball, prec):
    # psi = c/|x-y|: far pairs, pairs in the near field of the outer point and cut pairs all
    # evaluate the points of the oracle's rule (same counts and hashes)
    p = small_problem(ball, n=24, kernel="inv_dist")
    out = O.assemble(p.mesh, oracle_cfg(p, duffy_n=4), want_hash=True)
    Dg, stats = gpu_assemble(nl, ctx, p, prec, duffy_n=4)
    compare(Dg, O.to_csr(out), prec)
    assert stats == (out["n_pairs"], out["n_qp_pairs"], out["n_inter"])
    h, c, q = gpu_interactions(nl, ctx, p, prec=prec, duffy_n=4)
    np.testing.assert_array_equal(q, out["qp_a"])
    np.testing.assert_array_equal(h, out["hash_a"])


@pytest.mark.parametrize("ball,kernel", [("ngon", "const"), ("ngon", "inv_dist"), ("nocaps", "inv_dist"),
                                         ("exactcaps", "const")])
def test_fp64_items_queued_or_inline(nl, ctx, monkeypatch, ball, kernel):
    # FP32 path: the items whose region the FP64 geometry builds are queued for the deferred
    # kernel.  Without a queue (capacity 0: all inline in the boundary kernel) or with a
    # queue of one item (the rest inline), the records are the same and the values stay
    # within the FP32 bound.
    p = small_problem(ball, n=24, kernel=kernel)
    over = dict(duffy_n=4) if kernel == "inv_dist" else {}
    out = O.assemble(p.mesh, oracle_cfg(p, **over), want_hash=True)
    counts = {}
    for cap in (None, "0", "1"):
        if cap is None:
            monkeypatch.delenv("NL_DEFER_CAP", raising=False)
        else:
            monkeypatch.setenv("NL_DEFER_CAP", cap)
        h, c, q = gpu_interactions(nl, ctx, p, prec="fp32c", **over)
        counts[cap] = nl.nl_last_fp64_items(ctx)
        np.testing.assert_array_equal(c, out["count_a"])
        np.testing.assert_array_equal(q, out["qp_a"])
        np.testing.assert_array_equal(h, out["hash_a"])
        Dg, stats = gpu_assemble(nl, ctx, p, "fp32c", **over)
        compare(Dg, O.to_csr(out), "fp32c")
        assert stats == (out["n_pairs"], out["n_qp_pairs"], out["n_inter"])
        assert nl.nl_last_fp64_items(ctx) == counts[cap]
    assert counts[None] == counts["0"] == counts["1"]
    if kernel == "inv_dist":
        assert counts[None] > 0


@pytest.mark.parametrize("cap_printed", [0, 1])
def test_exactcaps_fp32_region_certified(nl, ctx, cap_printed):
    # exactcaps on the FP32 path: the certified FP32 walk builds the nocaps polygon and the caps
    # (one centroid point each, with the true or the printed area), so only a few items are left
    # to the FP64 geometry; the records are the oracle's and the values within the FP32 bound
    p = small_problem("exactcaps", n=24)
    out = O.assemble(p.mesh, oracle_cfg(p, cap_printed=cap_printed), want_hash=True)
    h, c, q = gpu_interactions(nl, ctx, p, prec="fp32c", cap_printed=cap_printed)
    np.testing.assert_array_equal(c, out["count_a"])
    np.testing.assert_array_equal(q, out["qp_a"])
    np.testing.assert_array_equal(h, out["hash_a"])
    assert nl.nl_last_fp64_items(ctx) < 0.01 * out["n_inter"]
    Dg, stats = gpu_assemble(nl, ctx, p, "fp32c", cap_printed=cap_printed)
    compare(Dg, O.to_csr(out), "fp32c")
    assert stats == (out["n_pairs"], out["n_qp_pairs"], out["n_inter"])


@pytest.mark.parametrize("ball", ["ngon", "nocaps"])
def test_near_field_items_queued_or_inline(nl, ctx, monkeypatch, ball):
    # FP32 singular kernel: the near-field whole items go to k_near through a queue.  Without the
    # queue (capacity 0: the boundary kernel integrates them in its own drain) or with a queue of
    # one item (the rest integrated by their owner lanes), the records and the values are the
    # oracle's, as with the default queue.
    p = small_problem(ball, n=24, kernel="inv_dist")
    out = O.assemble(p.mesh, oracle_cfg(p, duffy_n=4), want_hash=True)
    for cap in (None, "0", "1"):
        if cap is None:
            monkeypatch.delenv("NL_NEAR_CAP", raising=False)
        else:
            monkeypatch.setenv("NL_NEAR_CAP", cap)
        h, c, q = gpu_interactions(nl, ctx, p, prec="fp32c", duffy_n=4)
        np.testing.assert_array_equal(c, out["count_a"])
        np.testing.assert_array_equal(q, out["qp_a"])
        np.testing.assert_array_equal(h, out["hash_a"])
        Dg, stats = gpu_assemble(nl, ctx, p, "fp32c", duffy_n=4)
        compare(Dg, O.to_csr(out), "fp32c")
        assert stats == (out["n_pairs"], out["n_qp_pairs"], out["n_inter"])


def test_fp64_items_zero_on_fp64_path(nl, ctx):
    p = small_problem("ngon", n=24, kernel="inv_dist")
    gpu_interactions(nl, ctx, p, prec="fp64", duffy_n=4)
    assert nl.nl_last_fp64_items(ctx) == 0


@pytest.mark.parametrize("ball", ["nocaps", "approxcaps", "exactcaps"])
@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_parity_paper_protocol(nl, ctx, ball, prec):
    # rule switch of Sec. 8: 4-point rule for near pairs, 7-point vertex rule otherwise; 3-point inner
    d = 0.1
    m = I.paper_grid(0.05)
    p = I.Problem("paper", m, d, "const", I.const_kernel_c(d), ball, "switch47", "gauss3")
    out = O.assemble(m, oracle_cfg(p, cap_printed=1), want_hash=True)
    Dg, stats = gpu_assemble(nl, ctx, p, prec, cap_printed=1)
    compare(Dg, O.to_csr(out), prec)
    h, c, q = gpu_interactions(nl, ctx, p, prec=prec, cap_printed=1)
    np.testing.assert_array_equal(h, out["hash_a"])


@pytest.mark.parametrize("ball", ["nocaps", "approxcaps", "ngon"])
@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_parity_shifted_ball(nl, ctx, ball, prec):
    # shifted-centre ball (Sec. 4.3): the region of every outer point of T_a is built around bary_a
    p = small_problem(ball, outer="gauss4", inner="gauss3")
    out = O.assemble(p.mesh, oracle_cfg(p, shifted=1), want_hash=True)
    Dg, stats = gpu_assemble(nl, ctx, p, prec, shifted=1)
    compare(Dg, O.to_csr(out), prec)
    assert stats == (out["n_pairs"], out["n_qp_pairs"], out["n_inter"])
    h, c, q = gpu_interactions(nl, ctx, p, prec=prec, shifted=1)
    np.testing.assert_array_equal(q, out["qp_a"])
    np.testing.assert_array_equal(h, out["hash_a"])


def test_shifted_ball_needs_constant_kernel(nl, ctx):
    p = small_problem("nocaps", n=24, kernel="inv_dist")
    keep = nl._Keep()
    mesh = nl.make_mesh(p.mesh, keep)
    with pytest.raises(nl.NlError) as e:
        nl.nl_assemble(ctx, mesh, nl.config_of(p, keep, shifted=1))
    assert e.value.status == nl.NL_EUNSUPPORTED


def test_ragged_and_tiny(nl, ctx):
    # 7x7 cells -> 98 triangles (not a multiple of the warps per block), and a single triangle
    p = small_problem("ngon", n=7).with_(delta=0.4, ngon_off=I.ngon_offsets(32, 0.4))
    out = O.assemble(p.mesh, oracle_cfg(p))
    Dg, _ = gpu_assemble(nl, ctx, p, "fp64")
    compare(Dg, O.to_csr(out), "fp64")
    one = I.Mesh(vx=np.array([0.0, 1.0, 0.0]), vy=np.array([0.0, 0.0, 1.0]), tri=np.array([[0, 1, 2]], np.int32),
                 node_in_omega=np.zeros(3, np.uint8), elem_in_omega=np.zeros(1, np.uint8), h=1.0, lo=0, hi=1, n=1)
    q = p.with_(mesh=one, delta=2.0, ball="nocaps", ngon_off=None, ngon_n=0)
    out = O.assemble(one, oracle_cfg(q))
    Dg, _ = gpu_assemble(nl, ctx, q, "fp64")
    compare(Dg, O.to_csr(out), "fp64")


def refined_patch_mesh(n=48, frac=0.25, width=0.05):
    """Split-square grid over (-0.1, 1.1)^2 whose first frac*n grid lines in each direction are
    packed into [-0.1, -0.1 + width]: a refined corner patch, so that the matrix rows of its nodes
    are far longer than the mean candidate list of the mesh."""
    m = I.split_square_mesh(-0.1, 1.1, n)
    k = int(round(frac * n))
    lines = np.concatenate([-0.1 + width * np.arange(k) / k,
                            -0.1 + width + (1.2 - width) * np.arange(n - k + 1) / (n - k)])
    vx = lines[np.rint((m.vx + 0.1) / m.h).astype(int)]
    vy = lines[np.rint((m.vy + 0.1) / m.h).astype(int)]
    node_in = ((vx > 0) & (vx < 1) & (vy > 0) & (vy < 1)).astype(np.uint8)
    bx, by = vx[m.tri].mean(axis=1), vy[m.tri].mean(axis=1)
    elem_in = ((bx > 0) & (bx < 1) & (by > 0) & (by < 1)).astype(np.uint8)
    return I.Mesh(vx=np.ascontiguousarray(vx), vy=np.ascontiguousarray(vy), tri=m.tri, node_in_omega=node_in,
                  elem_in_omega=elem_in, h=m.h, lo=m.lo, hi=m.hi, n=n)


@pytest.mark.parametrize("bits", [None, "6", "7"])
def test_pattern_long_rows(nl, ctx, monkeypatch, bits):
    """The symbolic phase counts each row in a hash set of the smallest power of two >= twice the
    mean candidate list (at least 64) slots and keeps the rows of fewer than half its slots
    sorted for the column write; longer rows are built again, and rows that fill the set are
    counted again in a full one.  A refined corner patch gives rows of half the set and more,
    and a small first set (NL_ROW_SET_BITS) sends most rows through the second count: the
    pattern and the values match the oracle either way."""
    m = refined_patch_mesh()
    d = 0.1
    p = I.Problem("patch_48", m, d, "const", I.const_kernel_c(d), "nocaps", "dunavant7", "dunavant7")
    if bits is None:
        monkeypatch.delenv("NL_ROW_SET_BITS", raising=False)
    else:
        monkeypatch.setenv("NL_ROW_SET_BITS", bits)
    out = O.assemble(m, oracle_cfg(p))
    Dg, stats = gpu_assemble(nl, ctx, p, "fp64")
    compare(Dg, O.to_csr(out), "fp64")
    assert stats == (out["n_pairs"], out["n_qp_pairs"], out["n_inter"])
    # the mesh does what it is for: rows of half the first set and more (the candidate test
    # |bary_a - bary_b| <= delta + r_a + r_b, here in FP64; 2 E / K is far from a power of two)
    xy = np.stack([m.vx[m.tri], m.vy[m.tri]], -1)
    b = xy.mean(axis=1)
    r = np.sqrt(((xy - b[:, None]) ** 2).sum(-1)).max(axis=1)
    dist = np.sqrt(((b[:, None] - b[None]) ** 2).sum(-1))
    n_cand = int((dist <= d + r[:, None] + r[None]).sum())
    h0 = 64
    while h0 < 2 * n_cand // m.nt:
        h0 *= 2
    rows = np.diff(Dg.indptr)
    assert (rows >= h0 // 2).sum() > 20
    if bits is not None:
        assert (rows > (1 << int(bits))).sum() > m.nv // 4


def test_device_pointer_inputs(nl, ctx):
    torch = pytest.importorskip("torch")
    p = small_problem("approxcaps", n=24)
    keep = nl._Keep()
    m = p.mesh
    dev = type("M", (), dict(vx=torch.tensor(m.vx, device="cuda"), vy=torch.tensor(m.vy, device="cuda"),
                             tri=torch.tensor(m.tri, device="cuda")))
    mesh = nl.make_mesh(dev, keep)
    cfg = nl.config_of(p, keep, prec="fp64")
    out = nl.nl_assemble(ctx, mesh, cfg)
    try:
        Dg = nl.to_scipy(ctx, out)
    finally:
        nl.nl_csr_free(ctx, out)
    compare(Dg, O.to_csr(O.assemble(m, oracle_cfg(p))), "fp64")


# Two runs of one assembly.  FP64 path: only the order of FP64 atomic additions differs (M_aa,
# M_bb, the scatter into D), about 1e-16 relative.  FP32 path: the boundary kernel adds the
# blocks of the items into each pair's shared column in fixed point (integer sums: the same for
# any order of the lanes), and the FP64-decided items are queued per warp in (pair, outer point)
# order and added onto each pair in that order, so only the FP64 atomic order is left.  The
# singular kernel's near-field items are summed by k_near in FP32 in a grouping that follows
# their place in the queue (which the warps fill in any order): a pair block may change by a few
# units in its last place (2^-24 of the block, a block about 1/400 of a diagonal entry),
# measured up to 3e-8 of max|D|, tested at 1e-7.
REPEAT_TOL = {"fp64": 1e-14, "fp32c": 1e-13, "fp32c_near": 1e-7}


def repeat_tol(prec, kernel):
    return REPEAT_TOL["fp32c_near" if (prec, kernel) == ("fp32c", "inv_dist") else prec]


@pytest.mark.parametrize("ball,kernel,prec", [("ngon", "const", "fp32c"), ("exactcaps", "const", "fp32c"),
                                              ("ngon", "inv_dist", "fp32c"), ("ngon", "const", "fp64"),
                                              ("nocaps", "inv_dist", "fp64")])
def test_numeric_reassembly_is_repeatable(nl, ctx, monkeypatch, ball, kernel, prec):
    # re-assembly of the values on the same pattern, then a second full assembly
    monkeypatch.setenv("NL_DEFER_CAP", "1000000")   # every FP64-decided item queued (none inline)
    p = small_problem(ball, n=24, kernel=kernel)
    over = dict(duffy_n=4) if kernel == "inv_dist" else {}
    keep = nl._Keep()
    mesh = nl.make_mesh(p.mesh, keep)
    cfg = nl.config_of(p, keep, prec=prec, **over)
    m = nl.nl_assemble(ctx, mesh, cfg)
    try:
        D1 = nl.to_scipy(ctx, m)
        if prec == "fp32c" and kernel == "inv_dist":
            assert nl.nl_last_fp64_items(ctx) > 0   # the deferred queue is exercised
        nl.nl_assemble_numeric(ctx, m)
        D2 = nl.to_scipy(ctx, m)
    finally:
        nl.nl_csr_free(ctx, m)
    m = nl.nl_assemble(ctx, mesh, cfg)
    try:
        D3 = nl.to_scipy(ctx, m)
    finally:
        nl.nl_csr_free(ctx, m)
    np.testing.assert_array_equal(D1.indices, D2.indices)
    np.testing.assert_array_equal(D1.indices, D3.indices)
    scale = np.abs(D1.data).max()
    assert np.abs(D1.data - D2.data).max() <= repeat_tol(prec, kernel) * scale
    assert np.abs(D1.data - D3.data).max() <= repeat_tol(prec, kernel) * scale


@pytest.mark.parametrize("kernel", ["const", "inv_dist"])
def test_full_queue_reruns_repeatably(nl, ctx, monkeypatch, kernel):
    # queues that start with room for 64 items: the first numeric run leaves the excess to the
    # boundary kernel's lanes and nl_assemble runs it again with queues that hold them all; two
    # assemblies agree to the FP64 atomic order (and to the oracle)
    monkeypatch.delenv("NL_DEFER_CAP", raising=False)
    monkeypatch.delenv("NL_NEAR_CAP", raising=False)
    monkeypatch.setenv("NL_DEFER_CAP_INIT", "64")
    monkeypatch.setenv("NL_NEAR_CAP_INIT", "64")
    p = small_problem("ngon", n=24, kernel=kernel)
    over = dict(duffy_n=4) if kernel == "inv_dist" else {}
    keep = nl._Keep()
    mesh = nl.make_mesh(p.mesh, keep)
    cfg = nl.config_of(p, keep, prec="fp32c", **over)
    vals = []
    for _ in range(2):
        m = nl.nl_assemble(ctx, mesh, cfg)
        try:
            vals.append(nl.to_scipy(ctx, m))
            assert nl.nl_last_fp64_items(ctx) > 64
        finally:
            nl.nl_csr_free(ctx, m)
    np.testing.assert_array_equal(vals[0].indices, vals[1].indices)
    assert np.abs(vals[0].data - vals[1].data).max() <= repeat_tol("fp32c", kernel) * np.abs(vals[0].data).max()
    compare(vals[0], O.to_csr(O.assemble(p.mesh, oracle_cfg(p, **over))), "fp32c")


def test_numeric_reassembly_in_a_graph(nl):
    """nl_assemble_numeric captured in a CUDA graph on the context's stream (the interior
    kernel's second stream joins the capture through events): after the values are wiped, a
    replay computes them again."""
    torch = pytest.importorskip("torch")
    import ctypes
    try:
        rt = ctypes.CDLL("libcudart.so.13")   # the runtime the library is linked against
    except OSError:
        rt = ctypes.CDLL("/usr/local/cuda/lib64/libcudart.so.13")
    p = small_problem("ngon", n=24)
    s = torch.cuda.Stream()
    c = nl.nl_create(0, s.cuda_stream)
    try:
        keep = nl._Keep()
        m = nl.nl_assemble(c, nl.make_mesh(p.mesh, keep), nl.config_of(p, keep, prec="fp32c"))
        try:
            D0 = nl.to_scipy(c, m)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                nl.nl_assemble_numeric(c, m)
            assert rt.cudaMemset(ctypes.c_void_p(m.val), 0, ctypes.c_size_t(8 * m.nnz)) == 0
            assert rt.cudaDeviceSynchronize() == 0
            assert np.abs(nl.to_scipy(c, m).data).max() == 0.0
            g.replay()
            torch.cuda.synchronize()
            D1 = nl.to_scipy(c, m)
        finally:
            nl.nl_csr_free(c, m)
    finally:
        nl.nl_destroy(c)
    np.testing.assert_array_equal(D1.indptr, D0.indptr)
    np.testing.assert_array_equal(D1.indices, D0.indices)
    assert np.abs(D1.data - D0.data).max() <= REPEAT_TOL["fp32c"] * np.abs(D0.data).max()


@pytest.mark.parametrize("ball", ["nocaps", "approxcaps", "exactcaps", "ngon", "overlap", "bary_nocaps"])
@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_parity_delta_below_triangle_diameter(nl, ctx, ball, prec):
    # delta = 0.045 on a jittered grid with h = 0.05 (diameters up to about 0.09): an edge can be
    # cut twice with no vertex inside, three arcs per triangle, regions of up to six walk points
    p = small_problem(ball, n=24)
    d = 0.045
    p = p.with_(delta=d, kernel_c=I.const_kernel_c(d))
    if ball == "ngon":
        p = p.with_(ngon_off=I.ngon_offsets(32, d))
    out = O.assemble(p.mesh, oracle_cfg(p), want_hash=True)
    assert O.hmax(p.mesh) > d
    Dg, stats = gpu_assemble(nl, ctx, p, prec)
    compare(Dg, O.to_csr(out), prec)
    assert stats == (out["n_pairs"], out["n_qp_pairs"], out["n_inter"])
    h, c, q = gpu_interactions(nl, ctx, p, prec=prec)
    np.testing.assert_array_equal(c, out["count_a"])
    np.testing.assert_array_equal(h, out["hash_a"])


def test_errors(nl, ctx):
    p = small_problem("nocaps", n=24)
    # clockwise triangle
    bad = I.Mesh(vx=p.mesh.vx, vy=p.mesh.vy, tri=p.mesh.tri[:, ::-1].copy(), node_in_omega=p.mesh.node_in_omega,
                 elem_in_omega=p.mesh.elem_in_omega, h=p.mesh.h, lo=0, hi=1, n=24)
    with pytest.raises(nl.NlError) as e:
        gpu_assemble(nl, ctx, p.with_(mesh=bad), "fp64")
    assert e.value.status == nl.NL_EGEOM
    # bad enum
    keep = nl._Keep()
    cfg = nl.config_of(p, keep)
    cfg.ball = 42
    with pytest.raises(nl.NlError) as e:
        nl.nl_assemble(ctx, nl.make_mesh(p.mesh, keep), cfg)
    assert e.value.status == nl.NL_EINVAL


_FULL = {}


def oracle_full(name, **over):
    """The oracle's whole matrix and every outer triangle's records for a named workload (all
    K x K element pairs on every host core: about 25 s for ngon32_96 and a minute for
    singular_128 on a 16-core host), computed once per test session."""
    key = (name, tuple(sorted(over.items())))
    if key not in _FULL:
        p = I.problem(name)
        out = O.assemble(p.mesh, oracle_cfg(p, **over), want_hash=True, nthreads=os.cpu_count() or 1)
        Do = O.to_csr(out)
        Do.sort_indices()
        _FULL[key] = (p, out, Do)
    return _FULL[key]


def compare_full(nl, ctx, name, prec, **over):
    """Every output of the workload at full size, in the launch configuration bench.py times:
    every row pointer and column index, every outer triangle's interaction count, qp-pair
    count and record hash, and the totals exactly; every value within the bar of the
    precision, relative to the oracle's max|D|."""
    p, out, Do = oracle_full(name, **over)
    keep = nl._Keep()
    mesh = nl.make_mesh(p.mesh, keep)
    cfg = nl.config_of(p, keep, prec=prec, **over)
    h, c, q = nl.nl_interactions(ctx, mesh, cfg)
    np.testing.assert_array_equal(c, out["count_a"])
    np.testing.assert_array_equal(q, out["qp_a"])
    np.testing.assert_array_equal(h, out["hash_a"])
    m = nl.nl_assemble(ctx, mesh, cfg)
    try:
        Dg = nl.to_scipy(ctx, m)
        stats = (m.n_pairs, m.n_qp_pairs, m.n_inter)
    finally:
        nl.nl_csr_free(ctx, m)
    assert stats == (out["n_pairs"], out["n_qp_pairs"], out["n_inter"])
    return compare(Dg, Do, prec)


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_parity_bench_workload_full_size(nl, ctx, prec):
    # the benchmark workload itself (32-gon, 96x96 jittered, K = 18432, 16-point outer rule):
    # the whole matrix (2.75 M entries) and all 18432 outer triangles' records
    compare_full(nl, ctx, "ngon32_96", prec)


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_parity_singular_workload_full_size(nl, ctx, prec):
    # integrable singular kernel 3/(pi delta^3)/|x-y|, delta 0.05, 128x128 jittered (K = 32768):
    # the near-singular rule runs on every pair near the outer point; the whole matrix and all records
    compare_full(nl, ctx, "singular_128", prec, duffy_n=4)


def test_parity_solve_workload_full_size_sampled(nl, ctx):
    # the assembly of the solve workload (32-gon, delta 0.05, 220x220 jittered, K = 96800,
    # delta/h = 10), FP32-compensated as the bench times it; sampled outputs from the oracle
    p = I.problem("solve_220")
    K, J = p.mesh.nt, p.mesh.nv
    keep = nl._Keep()
    mesh = nl.make_mesh(p.mesh, keep)
    cfg = nl.config_of(p, keep, prec="fp32c")
    h, c, q = nl.nl_interactions(ctx, mesh, cfg)
    rng = np.random.default_rng(23)
    a_list = np.unique(np.concatenate([rng.choice(K, 30, replace=False), [0, K - 1, K // 2 + 221]]))
    out = O.assemble(p.mesh, oracle_cfg(p), a_list=a_list.astype(np.int32), want_hash=True)
    np.testing.assert_array_equal(h[a_list], out["hash_a"][a_list])
    np.testing.assert_array_equal(c[a_list], out["count_a"][a_list])
    np.testing.assert_array_equal(q[a_list], out["qp_a"][a_list])
    m = nl.nl_assemble(ctx, mesh, cfg)
    try:
        Dg = nl.to_scipy(ctx, m)
    finally:
        nl.nl_csr_free(ctx, m)
    # 64 rows spread over the mesh (interior, layer and corner nodes) plus three fixed ones; the
    # bar is relative to the oracle's largest entry in those rows
    rows = np.unique(np.concatenate([rng.choice(J, 61, replace=False), [J // 2 + 3, 221 * 7 + 5, J - 2]]))
    mask = np.zeros(J, np.uint8)
    mask[rows] = 1
    Dr = O.to_csr(O.assemble(p.mesh, oracle_cfg(p), row_mask=mask, nthreads=os.cpu_count() or 1))
    Dr.sort_indices()
    scale = max(np.abs(Dr[r].data).max() for r in rows)
    for r in rows:
        g_row, o_row = Dg[r], Dr[r]
        np.testing.assert_array_equal(g_row.indices, o_row.indices)
        assert np.abs(g_row.data - o_row.data).max() <= TOL["fp32c"] * scale
