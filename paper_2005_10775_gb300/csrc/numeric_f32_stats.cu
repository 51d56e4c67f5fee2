// numeric_f32_stats.cu -- the pair geometry + quadrature kernels with float quadrature that also
// accumulate the interaction records' hashes (nl_interactions).
#include "numeric_launch_f32.cuh"

nl_status nl_launch_numeric_f32_stats(nl_ctx *ctx, const nlq::NumArgs &A, int ball, bool one_stream)
{
    return nlf32::launch_numeric_f32_sts<1>(ctx, A, ball, one_stream);
}
