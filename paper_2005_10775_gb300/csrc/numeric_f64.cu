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
    return NL_OK;
}

template <int BALL>
nl_status launch_boundary(nl_ctx *ctx, const nlq::NumArgs &A, unsigned grid, unsigned threads)
{
    if (A.kernel == NL_KERNEL_INV_DIST) return launch_boundary_k<BALL, true>(ctx, A, grid, threads);
    return launch_boundary_k<BALL, false>(ctx, A, grid, threads);
}

}  // namespace

nl_status nl_launch_numeric_f64(nl_ctx *ctx, const nlq::NumArgs &A, int ball)
{
    const unsigned grid = (unsigned)((A.K + nlq::kWarpsPerBlock - 1) / nlq::kWarpsPerBlock);
    const unsigned threads = nlq::kWarpsPerBlock * 32;
    nlq::k_interior<double><<<grid, threads, 0, ctx->stream>>>(A); ++ctx->launches;
    NL_CK(cudaGetLastError());
    nl_status s;
    switch (ball) {
    case NL_BALL_BARYCENTER: s = launch_boundary<NL_BALL_BARYCENTER>(ctx, A, grid, threads); break;
    case NL_BALL_NOCAPS: s = launch_boundary<NL_BALL_NOCAPS>(ctx, A, grid, threads); break;
    case NL_BALL_APPROXCAPS: s = launch_boundary<NL_BALL_APPROXCAPS>(ctx, A, grid, threads); break;
    case NL_BALL_EXACTCAPS: s = launch_boundary<NL_BALL_EXACTCAPS>(ctx, A, grid, threads); break;
    case NL_BALL_NGON: s = launch_boundary<NL_BALL_NGON>(ctx, A, grid, threads); break;
    case NL_BALL_OVERLAP: s = launch_boundary<NL_BALL_OVERLAP>(ctx, A, grid, threads); break;
    case NL_BALL_BARY_NOCAPS: s = launch_boundary_k<NL_BALL_BARY_NOCAPS, false>(ctx, A, grid, threads); break;
    case NL_BALL_BARY_APPROXCAPS: s = launch_boundary_k<NL_BALL_BARY_APPROXCAPS, false>(ctx, A, grid, threads); break;
    default: return nl_fail(ctx, NL_EINVAL, "unknown ball mode");
    }
    if (s != NL_OK) return s;
    NL_CK(cudaGetLastError());
    return NL_OK;
}
