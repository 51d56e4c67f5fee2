// numeric_launch_f32.cuh -- the launches of the pair geometry + quadrature kernels with float
// quadrature, templated on the statistics switch STS (0: the assembly's kernels, without the
// record hashes; 1: nl_interactions' kernels, with them).  Included by numeric_f32.cu (STS = 0)
// and numeric_f32_stats.cu (STS = 1), so that the two sets of kernels compile side by side.
#pragma once

#include "numeric.cuh"

namespace nlf32 {


// stage 0: the boundary kernel (and its queue counter reset); stage 1: the deferred items
template <int BALL, bool INV, int STS>
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
            NL_CK(cudaFuncSetAttribute(nlq::k_boundary<BALL, float, INV, kNQ, STS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            nlq::k_boundary<BALL, float, INV, kNQ, STS><<<grid, threads, smem, ctx->stream>>>(A); ++ctx->launches;
        } else {
            NL_CK(cudaFuncSetAttribute(nlq::k_boundary<BALL, float, INV, false, STS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
            nlq::k_boundary<BALL, float, INV, false, STS><<<grid, threads, smem, ctx->stream>>>(A); ++ctx->launches;
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

template <int BALL, int STS>
nl_status launch_boundary(nl_ctx *ctx, const nlq::NumArgs &A, unsigned grid, unsigned threads, int stage)
{
    if (A.kernel == NL_KERNEL_INV_DIST) return launch_boundary_k<BALL, true, STS>(ctx, A, grid, threads, stage);
    return launch_boundary_k<BALL, false, STS>(ctx, A, grid, threads, stage);
}

template <int STS>
nl_status launch_ball(nl_ctx *ctx, const nlq::NumArgs &A, int ball, unsigned grid, unsigned threads, int stage)
{
    switch (ball) {
    case NL_BALL_BARYCENTER: return launch_boundary<NL_BALL_BARYCENTER, STS>(ctx, A, grid, threads, stage);
    case NL_BALL_NOCAPS: return launch_boundary<NL_BALL_NOCAPS, STS>(ctx, A, grid, threads, stage);
    case NL_BALL_APPROXCAPS: return launch_boundary<NL_BALL_APPROXCAPS, STS>(ctx, A, grid, threads, stage);
    case NL_BALL_EXACTCAPS: return launch_boundary<NL_BALL_EXACTCAPS, STS>(ctx, A, grid, threads, stage);
    case NL_BALL_NGON: return launch_boundary<NL_BALL_NGON, STS>(ctx, A, grid, threads, stage);
    case NL_BALL_OVERLAP: return launch_boundary<NL_BALL_OVERLAP, STS>(ctx, A, grid, threads, stage);
    case NL_BALL_BARY_NOCAPS: return launch_boundary_k<NL_BALL_BARY_NOCAPS, false, STS>(ctx, A, grid, threads, stage);
    case NL_BALL_BARY_APPROXCAPS:
        return launch_boundary_k<NL_BALL_BARY_APPROXCAPS, false, STS>(ctx, A, grid, threads, stage);
    default: return nl_fail(ctx, NL_EINVAL, "unknown ball mode");
    }
}


template <int STS>
nl_status launch_numeric_f32_sts(nl_ctx *ctx, const nlq::NumArgs &A, int ball, bool one_stream)
{
    const unsigned grid = (unsigned)((A.K + nlq::kWarpsPerBlock - 1) / nlq::kWarpsPerBlock);
    const unsigned threads = nlq::kWarpsPerBlock * 32;
    nl_status s = one_stream ? nl_numeric_zero(ctx, A) : nl_numeric_fork(ctx, A);
    if (s != NL_OK) return s;
    // the boundary kernel first, so that its blocks are dispatched before the interior kernel's
    s = launch_ball<STS>(ctx, A, ball, grid, threads, 0);
    s = one_stream ? nl_numeric_interior_same<float, STS>(ctx, A, grid, threads, s)
                   : nl_numeric_interior_join<float, STS>(ctx, A, grid, threads, s);
    if (s != NL_OK) return s;
    return launch_ball<STS>(ctx, A, ball, grid, threads, 1);
}

}  // namespace nlf32
