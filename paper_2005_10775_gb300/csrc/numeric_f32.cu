// numeric_f32.cu -- the pair geometry + quadrature kernels with float quadrature: the assembly's
// instantiation (no record hashes) and the entry that picks it or the statistics one
// (numeric_f32_stats.cu).
#include "numeric_launch_f32.cuh"

nl_status nl_launch_numeric_f32_stats(nl_ctx *ctx, const nlq::NumArgs &A, int ball, bool one_stream);

nl_status nl_deferred_blocks(nl_ctx *ctx, int *blocks)
{
    int nsm = 0;
    NL_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    *blocks = 2 * (nsm > 0 ? nsm : 1);
    return NL_OK;
}

nl_status nl_launch_numeric_f32(nl_ctx *ctx, const nlq::NumArgs &A, int ball, bool one_stream)
{
    if (A.stats) return nl_launch_numeric_f32_stats(ctx, A, ball, one_stream);
    return nlf32::launch_numeric_f32_sts<0>(ctx, A, ball, one_stream);
}
