// numeric_f64.cu -- instantiation of the pair geometry + quadrature kernels with double quadrature.
#include "numeric.cuh"

namespace {

template <int BALL, bool INV>
nl_status launch_boundary_k(nl_ctx *ctx, const nlq::NumArgs &A, unsigned grid, unsigned threads)
{
    const size_t smem = sizeof(nlq::BoundaryShared<double>) * nlq::kWarpsPerBlock;
    NL_CK(cudaFuncSetAttribute(nlq::k_boundary<BALL, double, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem));
    nlq::k_boundary<BALL, double, INV><<<grid, threads, smem, ctx->stream>>>(A); ++ctx->launches;
    NL_CK(cudaGetLastError());
    return NL_OK;
}

template <int BALL>
nl_status launch_boundary(nl_ctx *ctx, const nlq::NumArgs &A, unsigned grid, unsigned threads)
{
    if (A.kernel == NL_KERNEL_INV_DIST) return launch_boundary_k<BALL, true>(ctx, A, grid, threads);
    return launch_boundary_k<BALL, false>(ctx, A, grid, threads);
}

nl_status launch_ball(nl_ctx *ctx, const nlq::NumArgs &A, int ball, unsigned grid, unsigned threads)
{
    switch (ball) {
    case NL_BALL_BARYCENTER: return launch_boundary<NL_BALL_BARYCENTER>(ctx, A, grid, threads);
    case NL_BALL_NOCAPS: return launch_boundary<NL_BALL_NOCAPS>(ctx, A, grid, threads);
    case NL_BALL_APPROXCAPS: return launch_boundary<NL_BALL_APPROXCAPS>(ctx, A, grid, threads);
    case NL_BALL_EXACTCAPS: return launch_boundary<NL_BALL_EXACTCAPS>(ctx, A, grid, threads);
    case NL_BALL_NGON: return launch_boundary<NL_BALL_NGON>(ctx, A, grid, threads);
    case NL_BALL_OVERLAP: return launch_boundary<NL_BALL_OVERLAP>(ctx, A, grid, threads);
    case NL_BALL_BARY_NOCAPS: return launch_boundary_k<NL_BALL_BARY_NOCAPS, false>(ctx, A, grid, threads);
    case NL_BALL_BARY_APPROXCAPS: return launch_boundary_k<NL_BALL_BARY_APPROXCAPS, false>(ctx, A, grid, threads);
    default: return nl_fail(ctx, NL_EINVAL, "unknown ball mode");
    }
}

}  // namespace

nl_status nl_launch_numeric_f64(nl_ctx *ctx, const nlq::NumArgs &A, int ball, bool one_stream)
{
    const unsigned grid = (unsigned)((A.K + nlq::kWarpsPerBlock - 1) / nlq::kWarpsPerBlock);
    const unsigned threads = nlq::kWarpsPerBlock * 32;
    nl_status s = one_stream ? nl_numeric_zero(ctx, A) : nl_numeric_fork(ctx, A);
    if (s != NL_OK) return s;
    // the boundary kernel first, so that its blocks are dispatched before the interior kernel's
    s = launch_ball(ctx, A, ball, grid, threads);
    return one_stream ? nl_numeric_interior_same<double>(ctx, A, grid, threads, s)
                      : nl_numeric_interior_join<double>(ctx, A, grid, threads, s);
}
