// numeric_batch_f32.cu -- instantiation of the persistent batched numeric kernels with float
// quadrature: one interior launch for every problem of a batch with this value type, one
// boundary launch per ball mode x kernel type present.
#include "numeric.cuh"

namespace {

constexpr size_t kBoundarySmem = sizeof(nlq::BoundaryShared<float>) * nlq::kWarpsPerBlock;

template <int BALL, bool INV>
nl_status boundary(nl_ctx *ctx, const nlq::NumArgs *dA, const nlq::BatchItem *items, int n_items, int *counter,
                   int blocks, bool set_attr, int *per_sm)
{
    if (per_sm) {
        NL_CK(cudaFuncSetAttribute(nlq::k_boundary_batch<BALL, float, INV>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBoundarySmem));
        NL_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, nlq::k_boundary_batch<BALL, float, INV>,
                                                            nlq::kWarpsPerBlock * 32, kBoundarySmem));
        return NL_OK;
    }
    if (set_attr)
        NL_CK(cudaFuncSetAttribute(nlq::k_boundary_batch<BALL, float, INV>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBoundarySmem));
    nlq::k_boundary_batch<BALL, float, INV><<<blocks, nlq::kWarpsPerBlock * 32, kBoundarySmem, ctx->stream>>>(
        dA, items, n_items, counter);
    ++ctx->launches;
    NL_CK(cudaGetLastError());
    return NL_OK;
}

template <bool INV>
nl_status boundary_ball(nl_ctx *ctx, int ball, const nlq::NumArgs *dA, const nlq::BatchItem *items, int n_items,
                        int *counter, int blocks, bool set_attr, int *per_sm)
{
    switch (ball) {
    case NL_BALL_BARYCENTER:
        return boundary<NL_BALL_BARYCENTER, INV>(ctx, dA, items, n_items, counter, blocks, set_attr, per_sm);
    case NL_BALL_NOCAPS: return boundary<NL_BALL_NOCAPS, INV>(ctx, dA, items, n_items, counter, blocks, set_attr, per_sm);
    case NL_BALL_APPROXCAPS:
        return boundary<NL_BALL_APPROXCAPS, INV>(ctx, dA, items, n_items, counter, blocks, set_attr, per_sm);
    case NL_BALL_EXACTCAPS:
        return boundary<NL_BALL_EXACTCAPS, INV>(ctx, dA, items, n_items, counter, blocks, set_attr, per_sm);
    case NL_BALL_NGON: return boundary<NL_BALL_NGON, INV>(ctx, dA, items, n_items, counter, blocks, set_attr, per_sm);
    case NL_BALL_OVERLAP:
        return boundary<NL_BALL_OVERLAP, INV>(ctx, dA, items, n_items, counter, blocks, set_attr, per_sm);
    case NL_BALL_BARY_NOCAPS:
        return boundary<NL_BALL_BARY_NOCAPS, false>(ctx, dA, items, n_items, counter, blocks, set_attr, per_sm);
    case NL_BALL_BARY_APPROXCAPS:
        return boundary<NL_BALL_BARY_APPROXCAPS, false>(ctx, dA, items, n_items, counter, blocks, set_attr, per_sm);
    default: return nl_fail(ctx, NL_EINVAL, "unknown ball mode");
    }
}

}  // namespace

nl_status nl_launch_interior_batch_f32(nl_ctx *ctx, const nlq::NumArgs *dA, const nlq::BatchItem *items,
                                       int n_items, int *counter, int blocks)
{
    nlq::k_interior_batch<float><<<blocks, nlq::kWarpsPerBlock * 32, 0, ctx->stream>>>(dA, items, n_items, counter);
    ++ctx->launches;
    NL_CK(cudaGetLastError());
    return NL_OK;
}

nl_status nl_launch_boundary_batch_f32(nl_ctx *ctx, int ball, bool inv, const nlq::NumArgs *dA,
                                       const nlq::BatchItem *items, int n_items, int *counter, int blocks,
                                       bool set_attr)
{
    return inv ? boundary_ball<true>(ctx, ball, dA, items, n_items, counter, blocks, set_attr, nullptr)
               : boundary_ball<false>(ctx, ball, dA, items, n_items, counter, blocks, set_attr, nullptr);
}

nl_status nl_launch_deferred_batch_f32(nl_ctx *ctx, int ball, const nlq::NumArgs *dA, const nlq::DeferItem *items,
                                       const int *count, int cap)
{
    int blocks = 0;
    nl_status s = nl_deferred_blocks(ctx, &blocks);
    if (s != NL_OK) return s;
    const unsigned threads = nlq::kWarpsPerBlock * 32;
    switch (ball) {
    case NL_BALL_BARYCENTER:
        nlq::k_deferred_batch<NL_BALL_BARYCENTER><<<blocks, threads, 0, ctx->stream>>>(dA, items, count, cap); break;
    case NL_BALL_NOCAPS:
        nlq::k_deferred_batch<NL_BALL_NOCAPS><<<blocks, threads, 0, ctx->stream>>>(dA, items, count, cap); break;
    case NL_BALL_APPROXCAPS:
        nlq::k_deferred_batch<NL_BALL_APPROXCAPS><<<blocks, threads, 0, ctx->stream>>>(dA, items, count, cap); break;
    case NL_BALL_EXACTCAPS:
        nlq::k_deferred_batch<NL_BALL_EXACTCAPS><<<blocks, threads, 0, ctx->stream>>>(dA, items, count, cap); break;
    case NL_BALL_NGON:
        nlq::k_deferred_batch<NL_BALL_NGON><<<blocks, threads, 0, ctx->stream>>>(dA, items, count, cap); break;
    case NL_BALL_OVERLAP:
        nlq::k_deferred_batch<NL_BALL_OVERLAP><<<blocks, threads, 0, ctx->stream>>>(dA, items, count, cap); break;
    default: return nl_fail(ctx, NL_EINVAL, "no deferred items for this ball mode");
    }
    ++ctx->launches;
    nlq::k_defer_merge_batch<float><<<blocks, 256, 0, ctx->stream>>>(dA, items, count, cap); ++ctx->launches;
    NL_CK(cudaGetLastError());
    return NL_OK;
}

nl_status nl_batch_occupancy_f32(nl_ctx *ctx, int ball, bool inv, int *per_sm)
{
    if (ball < 0) {
        NL_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, nlq::k_interior_batch<float>,
                                                            nlq::kWarpsPerBlock * 32, 0));
        return NL_OK;
    }
    return inv ? boundary_ball<true>(ctx, ball, nullptr, nullptr, 0, nullptr, 0, false, per_sm)
               : boundary_ball<false>(ctx, ball, nullptr, nullptr, 0, nullptr, 0, false, per_sm);
}
