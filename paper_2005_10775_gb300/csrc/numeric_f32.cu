// numeric_f32.cu -- instantiation of the pair geometry + quadrature kernels with float quadrature.
#include "numeric.cuh"

namespace {

// stage 0: the boundary kernel (and its queue counter reset); stage 1: the deferred items
template <int BALL, bool INV>
nl_status launch_boundary_k(nl_ctx *ctx, const nlq::NumArgs &A, unsigned grid, unsigned threads, int stage)
{
    // the outer-support balls integrate their candidates without the item queue
    constexpr bool kQueue = BALL != NL_BALL_BARY_NOCAPS && BALL != NL_BALL_BARY_APPROXCAPS;
    const bool defer = kQueue && A.defer;
    if (stage == 0) {
        if (defer) NL_CK(cudaMemsetAsync(A.defer_n, 0, sizeof(int), ctx->stream));
        if (A.nearq) NL_CK(cudaMemsetAsync(A.near_n, 0, sizeof(int), ctx->stream));
        const size_t smem = sizeof(nlq::BoundaryShared<float>) * nlq::kWarpsPerBlock;
        // the singular kernel with its near-field queue: a kernel without the near rule's code
        constexpr bool kNQ = INV && kQueue;
        if (kNQ && A.nearq) {
            NL_CK(cudaFuncSetAttribute(nlq::k_boundary<BALL, float, INV, kNQ>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            nlq::k_boundary<BALL, float, INV, kNQ><<<grid, threads, smem, ctx->stream>>>(A); ++ctx->launches;
        } else {
            NL_CK(cudaFuncSetAttribute(nlq::k_boundary<BALL, float, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
            nlq::k_boundary<BALL, float, INV><<<grid, threads, smem, ctx->stream>>>(A); ++ctx->launches;
        }
        NL_CK(cudaGetLastError());
        return NL_OK;
    }
    if constexpr (kQueue && INV) {
        if (A.nearq) {   // the near-field whole items the boundary kernel queued
            // one resident wave: every warp strides over the queue, so a second wave of blocks
            // would only idle while the first finishes
            int nsm = 0, per_sm = 0;
            NL_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
            NL_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, nlq::k_near<BALL>, threads, 0));
            const int blocks = (nsm > 0 ? nsm : 1) * (per_sm > 0 ? per_sm : 1);
            nlq::k_near<BALL><<<blocks, threads, 0, ctx->stream>>>(A); ++ctx->launches;
            NL_CK(cudaGetLastError());
        }
    }
    if constexpr (kQueue) {
        if (defer) {
            int blocks = 0;
            nl_status s = nl_deferred_blocks(ctx, &blocks);
            if (s != NL_OK) return s;
            nlq::k_deferred<BALL><<<blocks, threads, 0, ctx->stream>>>(A); ++ctx->launches;
            nlq::k_defer_merge<float><<<blocks, 256, 0, ctx->stream>>>(A); ++ctx->launches;
            NL_CK(cudaGetLastError());
        }
    }
    return NL_OK;
}

template <int BALL>
nl_status launch_boundary(nl_ctx *ctx, const nlq::NumArgs &A, unsigned grid, unsigned threads, int stage)
{
    if (A.kernel == NL_KERNEL_INV_DIST) return launch_boundary_k<BALL, true>(ctx, A, grid, threads, stage);
    return launch_boundary_k<BALL, false>(ctx, A, grid, threads, stage);
}

nl_status launch_ball(nl_ctx *ctx, const nlq::NumArgs &A, int ball, unsigned grid, unsigned threads, int stage)
{
    switch (ball) {
    case NL_BALL_BARYCENTER: return launch_boundary<NL_BALL_BARYCENTER>(ctx, A, grid, threads, stage);
    case NL_BALL_NOCAPS: return launch_boundary<NL_BALL_NOCAPS>(ctx, A, grid, threads, stage);
    case NL_BALL_APPROXCAPS: return launch_boundary<NL_BALL_APPROXCAPS>(ctx, A, grid, threads, stage);
    case NL_BALL_EXACTCAPS: return launch_boundary<NL_BALL_EXACTCAPS>(ctx, A, grid, threads, stage);
    case NL_BALL_NGON: return launch_boundary<NL_BALL_NGON>(ctx, A, grid, threads, stage);
    case NL_BALL_OVERLAP: return launch_boundary<NL_BALL_OVERLAP>(ctx, A, grid, threads, stage);
    case NL_BALL_BARY_NOCAPS: return launch_boundary_k<NL_BALL_BARY_NOCAPS, false>(ctx, A, grid, threads, stage);
    case NL_BALL_BARY_APPROXCAPS:
        return launch_boundary_k<NL_BALL_BARY_APPROXCAPS, false>(ctx, A, grid, threads, stage);
    default: return nl_fail(ctx, NL_EINVAL, "unknown ball mode");
    }
}

}  // namespace

nl_status nl_deferred_blocks(nl_ctx *ctx, int *blocks)
{
    int nsm = 0;
    NL_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    *blocks = 2 * (nsm > 0 ? nsm : 1);
    return NL_OK;
}

nl_status nl_launch_numeric_f32(nl_ctx *ctx, const nlq::NumArgs &A, int ball, bool one_stream)
{
    const unsigned grid = (unsigned)((A.K + nlq::kWarpsPerBlock - 1) / nlq::kWarpsPerBlock);
    const unsigned threads = nlq::kWarpsPerBlock * 32;
    nl_status s = one_stream ? nl_numeric_zero(ctx, A) : nl_numeric_fork(ctx, A);
    if (s != NL_OK) return s;
    // the boundary kernel first, so that its blocks are dispatched before the interior kernel's
    s = launch_ball(ctx, A, ball, grid, threads, 0);
    s = one_stream ? nl_numeric_interior_same<float>(ctx, A, grid, threads, s)
                   : nl_numeric_interior_join<float>(ctx, A, grid, threads, s);
    if (s != NL_OK) return s;
    return launch_ball(ctx, A, ball, grid, threads, 1);
}
