"""Batched assembly on the GPU (nl_batch_*, through the C ABI): every problem of a
batch of uneven size, delta, ball, precision and kernel equals the oracle's matrix
(pattern bit-exact, values within the precision's bound) and the matrix nl_assemble
makes of it; the captured re-assembly graph reproduces the values; the autotuner's
schedule is cached per batch shape; a bad problem fails the whole batch cleanly."""
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


def mixed_batch():
    """Six small problems that exercise four numeric groups (fp32c/fp64 x const/inv_dist),
    two scatter groups and four ball modes, with meshes of different sizes and deltas."""
    out = []
    specs = [  # (delta, cells, jitter, ball, kernel, prec)
        (0.1, 24, 0.2, "nocaps", "const", "fp32c"),
        (0.15, 18, 0.0, "approxcaps", "const", "fp32c"),
        (0.2, 16, 0.2, "ngon", "const", "fp64"),
        (0.1, 26, 0.2, "barycenter", "const", "fp32c"),
        (0.2, 17, 0.2, "ngon", "inv_dist", "fp32c"),
        (0.15, 20, 0.2, "nocaps", "inv_dist", "fp64"),
        (0.2, 15, 0.2, "bary_approxcaps", "const", "fp32c"),
    ]
    for i, (d, n, jit, ball, kernel, prec) in enumerate(specs):
        m = I.split_square_mesh(-d, 1 + d, n, jitter=jit, seed=1077700 + i if jit else None)
        c = I.const_kernel_c(d) if kernel == "const" else I.inv_dist_kernel_c(d)
        p = I.Problem(f"mixed{i}", m, d, kernel, c, ball, "dunavant7", "dunavant7", cap_m=2)
        if ball == "ngon":
            p = p.with_(ngon_n=32, ngon_off=I.ngon_offsets(32, d))
        out.append((p, prec))
    return out


def oracle_cfg(p):
    return dict(delta=p.delta, ball=p.ball, outer=p.outer, inner=p.inner, kernel=p.kernel,
                kernel_c=p.kernel_c, ngon_off=p.ngon_off, cap_m=p.cap_m, duffy_n=4)


def compare(Dg, Do, tol):
    Do = Do.tocsr()
    Do.sort_indices()
    np.testing.assert_array_equal(Dg.indptr, Do.indptr)
    np.testing.assert_array_equal(Dg.indices, Do.indices)
    scale = np.abs(Do.data).max()
    assert np.abs(Dg.data - Do.data).max() <= tol * scale


@pytest.fixture(scope="module")
def mixed(nl, ctx):
    probs = mixed_batch()
    keep = nl._Keep()
    meshes = [nl.make_mesh(p.mesh, keep) for p, _ in probs]
    cfgs = [nl.config_of(p, keep, prec=prec, duffy_n=4) for p, prec in probs]
    h, outs = nl.nl_batch_create(ctx, meshes, cfgs)
    yield dict(probs=probs, keep=keep, meshes=meshes, cfgs=cfgs, h=h, outs=outs)
    nl.nl_batch_destroy(ctx, h)
    for o in outs:
        nl.nl_csr_free(ctx, o)


def test_batch_matches_oracle(nl, ctx, mixed):
    for (p, prec), out in zip(mixed["probs"], mixed["outs"]):
        ref = O.assemble(p.mesh, oracle_cfg(p))
        compare(nl.to_scipy(ctx, out), O.to_csr(ref), TOL[prec])
        assert (out.n_pairs, out.n_qp_pairs, out.n_inter) == (ref["n_pairs"], ref["n_qp_pairs"], ref["n_inter"])


def test_batch_matches_single_assembly(nl, ctx, mixed):
    for (p, prec), mesh, cfg, out in zip(mixed["probs"], mixed["meshes"], mixed["cfgs"], mixed["outs"]):
        single = nl.nl_assemble(ctx, mesh, cfg)
        try:
            S = nl.to_scipy(ctx, single)
            st = (single.n_pairs, single.n_qp_pairs, single.n_inter)
        finally:
            nl.nl_csr_free(ctx, single)
        B = nl.to_scipy(ctx, out)
        # the same interaction set and pattern, bit for bit (FP64 geometry is exactly rounded)
        assert (out.n_pairs, out.n_qp_pairs, out.n_inter) == st
        np.testing.assert_array_equal(B.indptr, S.indptr)
        np.testing.assert_array_equal(B.indices, S.indices)
        # values: the quadrature is the same code in another kernel, where the compiler may
        # fuse multiply-adds differently, and the FP64 scatter adds in another order
        assert np.abs(B.data - S.data).max() <= TOL[prec] * np.abs(S.data).max()


def test_batch_graph_replay_reproduces_values(nl, ctx, mixed):
    before = [nl.to_scipy(ctx, o).data.copy() for o in mixed["outs"]]
    n0 = nl.nl_launch_count(ctx)
    for _ in range(2):
        nl.nl_batch_run(ctx, mixed["h"])
    assert nl.nl_launch_count(ctx) > n0
    # FP64 values agree up to the order of the FP64 scatter's atomic adds; FP32 pair blocks
    # also take the FP64-decided items' blocks by FP32 atomic adds, in any order
    for b, o, (_, prec) in zip(before, mixed["outs"], mixed["probs"]):
        after = nl.to_scipy(ctx, o).data
        tol = 1e-14 if prec == "fp64" else 1e-6
        assert np.abs(after - b).max() <= tol * np.abs(b).max()


def test_batch_schedule_info_and_cache(nl, ctx, mixed):
    info = nl.nl_batch_get_info(mixed["h"])
    assert info["source"] in ("tuned", "cached")
    assert info["launches"] == 9 and info["blocks"] > 0
    assert info["chunk"] in (1, 2, 4, 8) and info["order"] in (0, 1)
    assert info["mode"] in (0, 1) and (info["mode"] == 0 or info["streams"] in (4, 8))
    assert info["n_tried"] in (0, 7)
    # the same batch shape again: the schedule comes from the context's cache
    h2, outs2 = nl.nl_batch_create(ctx, mixed["meshes"], mixed["cfgs"])
    try:
        info2 = nl.nl_batch_get_info(h2)
        assert info2["source"] == "cached"
        assert (info2["chunk"], info2["order"], info2["mode"], info2["streams"]) == \
            (info["chunk"], info["order"], info["mode"], info["streams"])
    finally:
        nl.nl_batch_destroy(ctx, h2)
        for o in outs2:
            nl.nl_csr_free(ctx, o)
    h3, outs3 = nl.nl_batch_create(ctx, mixed["meshes"][:2], mixed["cfgs"][:2], flags=nl.NL_BATCH_NO_TUNE)
    try:
        info3 = nl.nl_batch_get_info(h3)
        assert info3["source"] == "default" and info3["chunk"] == 1 and info3["order"] == 0
    finally:
        nl.nl_batch_destroy(ctx, h3)
        for o in outs3:
            nl.nl_csr_free(ctx, o)


def test_batch_rejects_a_bad_problem(nl, ctx):
    keep = nl._Keep()
    good = I.split_square_mesh(-0.1, 1.1, 24, jitter=0.2, seed=3)
    # the same mesh with its triangles clockwise
    bad = I.Mesh(vx=good.vx, vy=good.vy, tri=good.tri[:, ::-1].copy(), node_in_omega=good.node_in_omega,
                 elem_in_omega=good.elem_in_omega, h=good.h, lo=good.lo, hi=good.hi, n=good.n)
    p = I.Problem("g", good, 0.1, "const", I.const_kernel_c(0.1), "nocaps", "dunavant7", "dunavant7")
    meshes = [nl.make_mesh(good, keep), nl.make_mesh(bad, keep)]
    cfgs = [nl.config_of(p, keep, prec="fp32c"), nl.config_of(p, keep, prec="fp32c")]
    with pytest.raises(nl.NlError) as e:
        nl.nl_batch_create(ctx, meshes, cfgs)
    assert e.value.status == nl.NL_EGEOM
    assert "problem 1" in str(e.value)
    # the context stays usable
    out = nl.nl_assemble(ctx, meshes[0], cfgs[0])
    nl.nl_csr_free(ctx, out)


def test_batch_workload_sampled_against_oracle(nl, ctx):
    # the 64-problem batched workload (K from 2450 to 38088, delta 0.05 .. 0.2, nocaps and
    # approxcaps): full batch on the GPU, rows of a few problems from the oracle
    probs = I.batch_problems()
    keep = nl._Keep()
    meshes = [nl.make_mesh(p.mesh, keep) for p in probs]
    cfgs = [nl.config_of(p, keep, prec="fp32c") for p in probs]
    h, outs = nl.nl_batch_create(ctx, meshes, cfgs)
    try:
        rng = np.random.default_rng(11)
        for i in (0, 3, 6, 63):
            p = probs[i]
            G = nl.to_scipy(ctx, outs[i])
            J = p.mesh.nv
            rows = rng.choice(J, 2, replace=False)
            mask = np.zeros(J, np.uint8)
            mask[rows] = 1
            R = O.to_csr(O.assemble(p.mesh, oracle_cfg(p), row_mask=mask))
            scale = np.abs(G.diagonal()).max()
            for r in rows:
                g_row, o_row = G[r], R[r]
                o_row.sort_indices()
                np.testing.assert_array_equal(g_row.indices, o_row.indices)
                assert np.abs(g_row.data - o_row.data).max() <= TOL["fp32c"] * scale
    finally:
        nl.nl_batch_destroy(ctx, h)
        for o in outs:
            nl.nl_csr_free(ctx, o)


@pytest.mark.parametrize("flags", ["per_problem", "no_tune"])
def test_batch_each_schedule_family(nl, ctx, mixed, flags):
    # both schedule families, forced: persistent launches over all problems (NL_BATCH_NO_TUNE)
    # and each problem's own kernels over the side streams (NL_BATCH_PER_PROBLEM): the same
    # values as the tuned batch, and a graph replay (numeric phase and scatter) that repeats them
    f = nl.NL_BATCH_PER_PROBLEM if flags == "per_problem" else nl.NL_BATCH_NO_TUNE
    h, outs = nl.nl_batch_create(ctx, mixed["meshes"], mixed["cfgs"], flags=f)
    try:
        info = nl.nl_batch_get_info(h)
        assert info["mode"] == (1 if flags == "per_problem" else 0) and info["source"] == "default"
        ref = [nl.to_scipy(ctx, o) for o in mixed["outs"]]
        got = [nl.to_scipy(ctx, o) for o in outs]
        nl.nl_batch_run(ctx, h)
        again = [nl.to_scipy(ctx, o) for o in outs]
        for r, g, a, (_, prec) in zip(ref, got, again, mixed["probs"]):
            np.testing.assert_array_equal(g.indptr, r.indptr)
            np.testing.assert_array_equal(g.indices, r.indices)
            scale = np.abs(r.data).max()
            assert np.abs(g.data - r.data).max() <= TOL[prec] * scale
            assert np.abs(a.data - g.data).max() <= (1e-14 if prec == "fp64" else 1e-6) * scale
    finally:
        nl.nl_batch_destroy(ctx, h)
        for o in outs:
            nl.nl_csr_free(ctx, o)



def test_assemble_batch_pipelined_matches_single_assembly(nl, ctx, mixed):
    # nl_assemble_batch: each problem's nl_assemble steps, pipelined over the side streams;
    # the same interaction set and pattern as nl_assemble, values to the FP64 atomic order
    outs = nl.nl_assemble_batch(ctx, mixed["meshes"], mixed["cfgs"])
    try:
        for (p, prec), mesh, cfg, out in zip(mixed["probs"], mixed["meshes"], mixed["cfgs"], outs):
            single = nl.nl_assemble(ctx, mesh, cfg)
            try:
                S = nl.to_scipy(ctx, single)
                st = (single.n_pairs, single.n_qp_pairs, single.n_inter)
            finally:
                nl.nl_csr_free(ctx, single)
            B = nl.to_scipy(ctx, out)
            assert (out.n_pairs, out.n_qp_pairs, out.n_inter) == st
            np.testing.assert_array_equal(B.indptr, S.indptr)
            np.testing.assert_array_equal(B.indices, S.indices)
            tol = 1e-13 if (prec == "fp64" or p.kernel == "const") else 1e-6
            assert np.abs(B.data - S.data).max() <= tol * np.abs(S.data).max()
        ref = O.assemble(mixed["probs"][0][0].mesh, oracle_cfg(mixed["probs"][0][0]))
        compare(nl.to_scipy(ctx, outs[0]), O.to_csr(ref), TOL[mixed["probs"][0][1]])
    finally:
        for o in outs:
            nl.nl_csr_free(ctx, o)


def test_assemble_batch_pipelined_rejects_a_bad_problem(nl, ctx):
    keep = nl._Keep()
    good = I.split_square_mesh(-0.1, 1.1, 24, jitter=0.2, seed=3)
    bad = I.Mesh(vx=good.vx, vy=good.vy, tri=good.tri[:, ::-1].copy(), node_in_omega=good.node_in_omega,
                 elem_in_omega=good.elem_in_omega, h=good.h, lo=good.lo, hi=good.hi, n=good.n)
    p = I.Problem("g", good, 0.1, "const", I.const_kernel_c(0.1), "nocaps", "dunavant7", "dunavant7")
    meshes = [nl.make_mesh(good, keep), nl.make_mesh(bad, keep), nl.make_mesh(good, keep)]
    cfgs = [nl.config_of(p, keep, prec="fp32c") for _ in range(3)]
    with pytest.raises(nl.NlError) as e:
        nl.nl_assemble_batch(ctx, meshes, cfgs)
    assert e.value.status == nl.NL_EGEOM
    assert "problem 1" in str(e.value)
    out = nl.nl_assemble(ctx, meshes[0], cfgs[0])   # the context stays usable
    nl.nl_csr_free(ctx, out)
