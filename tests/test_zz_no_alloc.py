"""nl_cg_noalloc: the CG solve for callers that cannot allocate device memory (a
framework whose caching allocator owns all device memory, or a loop that cannot
take an allocation's synchronisation).  Its work vectors live in one fixed device
array inside the library; it must give the same solution as nl_cg, call after
call, and refuse systems larger than that array.

Kept in a file of its own, collected last, and self-contained: it passes alone in
a fresh process and after the other tests.
"""
import numpy as np
import pytest

from paper_2005_10775_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    from paper_2005_10775_gb300 import nlfem as nl
    ctx = nl.nl_create(0)
    d = 0.1
    m = I.split_square_mesh(-0.1, 1.1, 36, jitter=0.2, seed=1077505)
    p = I.Problem("noalloc", m, d, "const", I.const_kernel_c(d), "ngon", "dunavant7", "dunavant7", ngon_n=32,
                  ngon_off=I.ngon_offsets(32, d))
    keep = nl._Keep()
    mesh = nl.make_mesh(m, keep)
    D = nl.nl_assemble(ctx, mesh, nl.config_of(p, keep, prec="fp64"))
    A, B = nl.nl_extract(ctx, D, mesh)
    F = nl.nl_rhs(ctx, B, mesh, I.manufactured_f(m.vx, m.vy), I.manufactured_u(m.vx, m.vy))
    yield dict(nl=nl, torch=torch, ctx=ctx, A=A, F=F)
    for x in (D, A, B):
        nl.nl_csr_free(ctx, x)
    nl.nl_destroy(ctx)


def test_noalloc_cg_matches_cg_twice(setup):
    nl, torch, ctx, A, F = setup["nl"], setup["torch"], setup["ctx"], setup["A"], setup["F"]
    x_ref = np.zeros_like(F)
    it_ref, rel_ref = nl.nl_cg(ctx, A, F, x_ref, rtol=1e-10, max_it=5000)
    assert rel_ref <= 1e-10
    b = torch.tensor(F, device="cuda")
    for _ in range(2):   # two calls in a row share (and must reset) the scratch array
        x = torch.zeros_like(b)
        it, rel = nl.nl_cg_noalloc(ctx, A, b, x, rtol=1e-10, max_it=5000)
        torch.cuda.synchronize()
        xs = x.cpu().numpy()
        assert rel <= 1e-10 and it > 0
        assert np.abs(xs - x_ref).max() <= 1e-8 * np.abs(x_ref).max()


def test_noalloc_rejects_oversized_and_host_inputs(setup):
    nl, torch, ctx, A, F = setup["nl"], setup["torch"], setup["ctx"], setup["A"], setup["F"]
    big = nl.nl_csr(n=(1 << 18) + 1, nnz=A.nnz, row_ptr=A.row_ptr, col_idx=A.col_idx, val=A.val)
    b = torch.zeros((1 << 18) + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(nl.NlError) as e:
        nl.nl_cg_noalloc(ctx, big, b, b.clone())
    assert e.value.status == nl.NL_EUNSUPPORTED
    with pytest.raises(nl.NlError) as e:
        nl.nl_cg_noalloc(ctx, A, F, np.zeros_like(F))    # host arrays
    assert e.value.status == nl.NL_EINVAL


def test_noalloc_reports_failures_like_cg(setup):
    # the same failure reports as nl_cg: an rtol below the FP64 residual floor is not reached
    # (NL_ENOCONV once the refinement passes run out) and a NaN in b is rejected (NL_EINVAL);
    # a good solve right after each shows that the shared array was left usable
    nl, torch, ctx, A, F = setup["nl"], setup["torch"], setup["ctx"], setup["A"], setup["F"]
    b = torch.tensor(F, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(nl.NlError) as e:
        nl.nl_cg_noalloc(ctx, A, b, x, rtol=1e-18, max_it=200000)
    assert e.value.status == nl.NL_ENOCONV
    bn = b.clone()
    bn[bn.numel() // 2] = float("nan")
    with pytest.raises(nl.NlError) as e:
        nl.nl_cg_noalloc(ctx, A, bn, torch.zeros_like(b), rtol=1e-10, max_it=5000)
    assert e.value.status == nl.NL_EINVAL
    x = torch.zeros_like(b)
    it, rel = nl.nl_cg_noalloc(ctx, A, b, x, rtol=1e-10, max_it=5000)
    assert rel <= 1e-10 and it > 0

