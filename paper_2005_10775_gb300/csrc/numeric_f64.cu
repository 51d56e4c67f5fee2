// numeric_f64.cu -- instantiation of the pair geometry + quadrature kernel with double quadrature.
#include "numeric.cuh"

nl_status nl_launch_numeric_f64(nl_ctx *ctx, const nlq::NumArgs &A, int ball)
{
    const unsigned grid = (unsigned)((A.K + nlq::kWarpsPerBlock - 1) / nlq::kWarpsPerBlock);
    const unsigned threads = nlq::kWarpsPerBlock * 32;
    switch (ball) {
    case NL_BALL_BARYCENTER: nlq::k_numeric<NL_BALL_BARYCENTER, double><<<grid, threads, 0, ctx->stream>>>(A); ++ctx->launches; break;
    case NL_BALL_NOCAPS: nlq::k_numeric<NL_BALL_NOCAPS, double><<<grid, threads, 0, ctx->stream>>>(A); ++ctx->launches; break;
    case NL_BALL_APPROXCAPS: nlq::k_numeric<NL_BALL_APPROXCAPS, double><<<grid, threads, 0, ctx->stream>>>(A); ++ctx->launches; break;
    case NL_BALL_EXACTCAPS: nlq::k_numeric<NL_BALL_EXACTCAPS, double><<<grid, threads, 0, ctx->stream>>>(A); ++ctx->launches; break;
    case NL_BALL_NGON: nlq::k_numeric<NL_BALL_NGON, double><<<grid, threads, 0, ctx->stream>>>(A); ++ctx->launches; break;
    case NL_BALL_OVERLAP: nlq::k_numeric<NL_BALL_OVERLAP, double><<<grid, threads, 0, ctx->stream>>>(A); ++ctx->launches; break;
    default: return nl_fail(ctx, NL_EINVAL, "unknown ball mode");
    }
    NL_CK(cudaGetLastError());
    return NL_OK;
}
