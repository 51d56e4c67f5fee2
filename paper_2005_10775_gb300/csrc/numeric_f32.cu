// numeric_f32.cu -- instantiation of the pair geometry + quadrature kernel with float quadrature.
#include "numeric.cuh"

nl_status nl_launch_numeric_f32(nl_ctx *ctx, const nlq::NumArgs &A, int ball)
{
    const unsigned grid = (unsigned)((A.K + nlq::kWarpsPerBlock - 1) / nlq::kWarpsPerBlock);
    const unsigned threads = nlq::kWarpsPerBlock * 32;
    switch (ball) {
    case NL_BALL_BARYCENTER: nlq::k_numeric<NL_BALL_BARYCENTER, float><<<grid, threads, 0, ctx->stream>>>(A); ++ctx->launches; break;
    case NL_BALL_NOCAPS: nlq::k_numeric<NL_BALL_NOCAPS, float><<<grid, threads, 0, ctx->stream>>>(A); ++ctx->launches; break;
    case NL_BALL_APPROXCAPS: nlq::k_numeric<NL_BALL_APPROXCAPS, float><<<grid, threads, 0, ctx->stream>>>(A); ++ctx->launches; break;
    case NL_BALL_EXACTCAPS: nlq::k_numeric<NL_BALL_EXACTCAPS, float><<<grid, threads, 0, ctx->stream>>>(A); ++ctx->launches; break;
    case NL_BALL_NGON: nlq::k_numeric<NL_BALL_NGON, float><<<grid, threads, 0, ctx->stream>>>(A); ++ctx->launches; break;
    case NL_BALL_OVERLAP: nlq::k_numeric<NL_BALL_OVERLAP, float><<<grid, threads, 0, ctx->stream>>>(A); ++ctx->launches; break;
    default: return nl_fail(ctx, NL_EINVAL, "unknown ball mode");
    }
    NL_CK(cudaGetLastError());
    return NL_OK;
}
