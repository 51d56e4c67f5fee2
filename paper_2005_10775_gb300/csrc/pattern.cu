// pattern.cu -- CSR sparsity pattern of D and the numeric scatter (Sec. 7.2).
//
// Pattern: D[j, j'] is stored iff some element pair (T_a, T_b) with a non-empty
// region for at least one outer point has j, j' in nodes(T_a) u nodes(T_b)
// (the nonlocal fill of Sec. 7.2, "reduced sparsity"; sparsification by the
// finite horizon).  The pattern is symmetric: the pair flag is symmetrised and
// row j collects nodes(T_c) for every T containing j and every candidate T_c of
// T whose pair interacts in either direction (every triangle interacts with itself).
//
// Numeric scatter: D = W + W^T with the one-sided accumulator W receiving, per
// interacting pair, -M_ab at (a_i, b_k) and the upper triangle of M_bb (diagonal
// halved), and per outer triangle the upper triangle of M_aa (diagonal halved).
// That is 9 + 6 FP64 atomics per pair instead of 27, and the transposed blocks
// come from the final W + W^T pass through the transposed-slot map.
#include <cuda_runtime.h>

#include "internal.cuh"

namespace {

__device__ __forceinline__ int64_t find_slot(const int64_t *row_ptr, const int32_t *col, int r, int c)
{
    int64_t lo = row_ptr[r], hi = row_ptr[r + 1] - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) >> 1;
        int v = col[mid];
        if (v == c) return mid;
        if (v < c) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

__device__ __forceinline__ int64_t find_in(const int32_t *idx, int64_t lo, int64_t hi, int v)
{
    hi -= 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) >> 1;
        int x = idx[mid];
        if (x == v) return mid;
        if (x < v) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

// symmetric flag: pair (a, b) or (b, a) interacts; warp per a.  Each candidate list
// holds two sorted segments (interior, boundary) split at split[b].
__global__ void k_symflag(int K, const int64_t *ptr, const int64_t *split, const int32_t *idx, const uint8_t *flag,
                          uint8_t *sym)
{
    int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (a >= K) return;
    for (int64_t e = ptr[a] + lane; e < ptr[a + 1]; e += 32) {
        int b = idx[e];
        uint8_t f = flag[e];
        if (!f) {
            int64_t m = find_in(idx, ptr[b], split[b], a);
            if (m < 0) m = find_in(idx, split[b], ptr[b + 1], a);
            if (m >= 0) f = flag[m];
        }
        sym[e] = f;
    }
}

__global__ void k_node_count(int K, const int32_t *tri, int64_t *cnt)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= K) return;
    for (int i = 0; i < 3; i++) atomicAdd((unsigned long long *)&cnt[tri[3 * t + i]], 1ull);
}

__global__ void k_node_fill(int K, const int32_t *tri, const int64_t *start, int64_t *cursor, int32_t *ntri)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= K) return;
    for (int i = 0; i < 3; i++) {
        int v = tri[3 * t + i];
        int64_t pos = start[v] + (int64_t)atomicAdd((unsigned long long *)&cursor[v], 1ull);
        ntri[pos] = t;
    }
}

constexpr int kRowThreads = 256;
constexpr int kListCap = NL_HASH_CAP / 2;

// block per row: hash set of the row's columns in shared memory.
// pass 0: count; pass 1: write sorted columns at row_ptr[j].
__global__ void __launch_bounds__(kRowThreads) k_rows(int J, const int64_t *nt_ptr, const int32_t *ntri,
                                                      const int32_t *tri, const int64_t *ptr, const int32_t *idx,
                                                      const uint8_t *sym, int64_t *cnt, const int64_t *row_ptr,
                                                      int32_t *col, int *overflow, int pass)
{
    extern __shared__ int32_t sm[];
    int32_t *tab = sm;                    // [NL_HASH_CAP]
    int32_t *lst = sm + NL_HASH_CAP;      // [kListCap]
    __shared__ int s_n, s_ovf;
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < NL_HASH_CAP; i += blockDim.x) tab[i] = -1;
    if (threadIdx.x == 0) { s_n = 0; s_ovf = 0; }
    __syncthreads();
    for (int64_t q = nt_ptr[j]; q < nt_ptr[j + 1]; q++) {
        const int T = ntri[q];
        for (int64_t e = ptr[T] + threadIdx.x; e < ptr[T + 1]; e += blockDim.x) {
            if (!sym[e]) continue;
            const int c = idx[e];
            for (int i = 0; i < 3; i++) {
                const int v = tri[3 * c + i];
                unsigned h = ((unsigned)v * 2654435761u) & (NL_HASH_CAP - 1);
                for (int probe = 0; probe < NL_HASH_CAP; probe++) {
                    int old = atomicCAS(&tab[h], -1, v);
                    if (old == -1) {
                        if (atomicAdd(&s_n, 1) >= kListCap - 1) s_ovf = 1;
                        break;
                    }
                    if (old == v) break;
                    h = (h + 1) & (NL_HASH_CAP - 1);
                }
            }
        }
    }
    __syncthreads();
    if (s_ovf) {
        if (threadIdx.x == 0) atomicAdd(overflow, 1);
        return;
    }
    const int n = s_n;
    if (pass == 0) {
        if (threadIdx.x == 0) cnt[j] = n;
        return;
    }
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < NL_HASH_CAP; i += blockDim.x)
        if (tab[i] >= 0) lst[atomicAdd(&s_n, 1)] = tab[i];
    int p = 1;
    while (p < n) p <<= 1;
    for (int i = n + threadIdx.x; i < p; i += blockDim.x) lst[i] = 0x7fffffff;
    __syncthreads();
    for (int k = 2; k <= p; k <<= 1)
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int i = threadIdx.x; i < p; i += blockDim.x) {
                int l = i ^ jj;
                if (l > i) {
                    bool up = (i & k) == 0;
                    int u = lst[i], v = lst[l];
                    if ((u > v) == up) { lst[i] = v; lst[l] = u; }
                }
            }
            __syncthreads();
        }
    const int64_t o = row_ptr[j];
    for (int i = threadIdx.x; i < n; i += blockDim.x) col[o + i] = lst[i];
}

// slots of the six upper local pairs (00, 11, 22, 01, 02, 12) of each triangle
__global__ void k_local_slots(int K, const int32_t *tri, const int64_t *row_ptr, const int32_t *col, int64_t *lslot)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= K) return;
    const int pi[6] = {0, 1, 2, 0, 0, 1}, pk[6] = {0, 1, 2, 1, 2, 2};
    for (int p = 0; p < 6; p++) {
        int u = tri[3 * t + pi[p]], v = tri[3 * t + pk[p]];
        int r = min(u, v), c = max(u, v);
        lslot[(int64_t)p * K + t] = find_slot(row_ptr, col, r, c);
    }
}

// transposed slot map; warp per row
__global__ void k_tslot(int J, const int64_t *row_ptr, const int32_t *col, int64_t *tslot)
{
    int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (j >= J) return;
    for (int64_t s = row_ptr[j] + lane; s < row_ptr[j + 1]; s += 32) tslot[s] = find_slot(row_ptr, col, col[s], j);
}

// One-sided numeric scatter, warp per outer triangle.  The -M_ab contributions of all
// of T_a's pairs land in the three rows of T_a's nodes: the warp accumulates them in
// shared memory (columns of those rows staged there, `cap` per row) and adds each row
// entry to W once, instead of one FP64 atomic per pair and entry.  The upper M_bb of
// every pair and T_a's own M_aa go straight to W through the local slot map.
template <typename T>
__global__ void k_scatter(int K, int64_t E, const int32_t *tri, const int64_t *ptr, const int32_t *idx,
                          const uint8_t *flag, const T *blk, const double *maa, const int64_t *lslot,
                          const int64_t *row_ptr, const int32_t *col, double *W, int *err, int cap)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int a = blockIdx.x * (blockDim.x >> 5) + wib;
    int32_t *scol = (int32_t *)(smem_raw + (size_t)wib * 3 * cap * (sizeof(int32_t) + sizeof(T)));
    T *sacc = (T *)(scol + 3 * cap);
    if (a >= K) return;
    const int ar[3] = {tri[3 * a], tri[3 * a + 1], tri[3 * a + 2]};
    int64_t r0[3];
    int len[3];
    bool cached[3];
    for (int i = 0; i < 3; i++) {
        r0[i] = row_ptr[ar[i]];
        len[i] = (int)(row_ptr[ar[i] + 1] - r0[i]);
        cached[i] = len[i] <= cap;
        if (cached[i])
            for (int k = lane; k < len[i]; k += 32) {
                scol[i * cap + k] = col[r0[i] + k];
                sacc[i * cap + k] = (T)0;
            }
    }
    __syncwarp();
    for (int64_t e = ptr[a] + lane; e < ptr[a + 1]; e += 32) {
        if (!flag[e]) continue;
        const int b = idx[e];
        const int bn[3] = {tri[3 * b], tri[3 * b + 1], tri[3 * b + 2]};
        for (int i = 0; i < 3; i++)
            for (int k = 0; k < 3; k++) {
                const T v = blk[(int64_t)(3 * i + k) * E + e];
                if (cached[i]) {
                    int lo = 0, hi = len[i] - 1, pos = -1;
                    while (lo <= hi) {
                        const int mid = (lo + hi) >> 1;
                        const int c = scol[i * cap + mid];
                        if (c == bn[k]) { pos = mid; break; }
                        if (c < bn[k]) lo = mid + 1; else hi = mid - 1;
                    }
                    if (pos >= 0) atomicAdd(&sacc[i * cap + pos], -v); else atomicOr(err, 2);
                } else {
                    const int64_t sl = find_slot(row_ptr, col, ar[i], bn[k]);
                    if (sl >= 0) atomicAdd(&W[sl], -(double)v); else atomicOr(err, 2);
                }
            }
        for (int p = 0; p < 6; p++) {
            double v = (double)blk[(int64_t)(9 + p) * E + e];
            if (p < 3) v *= 0.5;
            const int64_t sl = lslot[(int64_t)p * K + b];
            if (sl >= 0) atomicAdd(&W[sl], v); else atomicOr(err, 2);
        }
    }
    __syncwarp();
    for (int i = 0; i < 3; i++)
        if (cached[i])
            for (int k = lane; k < len[i]; k += 32) {
                const T v = sacc[i * cap + k];
                if (v != (T)0) atomicAdd(&W[r0[i] + k], (double)v);
            }
    if (lane == 0)
        for (int p = 0; p < 6; p++) {
            double v = maa[(int64_t)p * K + a];
            if (p < 3) v *= 0.5;
            const int64_t sl = lslot[(int64_t)p * K + a];
            if (sl >= 0) atomicAdd(&W[sl], v); else atomicOr(err, 2);
        }
}

__global__ void k_symmetrize(int64_t nnz, const double *W, const int64_t *tslot, double *val, int *err)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nnz) return;
    int64_t t = tslot[s];
    if (t >= 0) val[s] = W[s] + W[t];
    else atomicOr(err, 4);
}

__global__ void k_row_max(int J, const int64_t *rcnt, unsigned long long *out)
{
    unsigned long long m = 0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < J; j += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)rcnt[j]);
    for (int off = 16; off; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(&out[3], m);
}

__global__ void k_sum_stats(int K, int64_t E, const uint8_t *flag, const int64_t *qp, const int64_t *cnt,
                            unsigned long long *out)
{
    unsigned long long p = 0, q = 0, c = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x)
        p += flag[e];
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < K; a += (int64_t)gridDim.x * blockDim.x) {
        q += qp[a];
        c += cnt[a];
    }
    for (int off = 16; off; off >>= 1) {
        p += __shfl_xor_sync(0xffffffffu, p, off);
        q += __shfl_xor_sync(0xffffffffu, q, off);
        c += __shfl_xor_sync(0xffffffffu, c, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], p);
        atomicAdd(&out[1], q);
        atomicAdd(&out[2], c);
    }
}

}  // namespace

nl_status nl_build_pattern(nl_ctx *ctx, nl_plan *P, nl_csr *out)
{
    const int K = P->K, J = P->J;
    nl_status s;
    uint8_t *sym = nullptr;
    int64_t *ncnt = nullptr, *nptr = nullptr, *ncur = nullptr, *rcnt = nullptr;
    int32_t *ntri = nullptr;
    int *ovf = nullptr;
    unsigned long long *st = nullptr;
    NL_CK(cudaMallocAsync((void **)&sym, P->E ? P->E : 1, ctx->stream));
    NL_CK(cudaMallocAsync((void **)&ncnt, sizeof(int64_t) * (J + 1), ctx->stream));
    NL_CK(cudaMallocAsync((void **)&nptr, sizeof(int64_t) * (J + 1), ctx->stream));
    NL_CK(cudaMallocAsync((void **)&ncur, sizeof(int64_t) * (J + 1), ctx->stream));
    NL_CK(cudaMallocAsync((void **)&rcnt, sizeof(int64_t) * (J + 1), ctx->stream));
    NL_CK(cudaMallocAsync((void **)&ntri, sizeof(int32_t) * 3 * (size_t)K, ctx->stream));
    NL_CK(cudaMallocAsync((void **)&ovf, sizeof(int), ctx->stream));
    NL_CK(cudaMallocAsync((void **)&st, sizeof(unsigned long long) * 4, ctx->stream));
    NL_CK(cudaMemsetAsync(ncnt, 0, sizeof(int64_t) * (J + 1), ctx->stream));
    NL_CK(cudaMemsetAsync(ncur, 0, sizeof(int64_t) * (J + 1), ctx->stream));
    NL_CK(cudaMemsetAsync(ovf, 0, sizeof(int), ctx->stream));
    NL_CK(cudaMemsetAsync(st, 0, sizeof(unsigned long long) * 4, ctx->stream));
    const unsigned wgrid = (unsigned)(((int64_t)K * 32 + 255) / 256);
    k_symflag<<<wgrid, 256, 0, ctx->stream>>>(K, P->nbr_ptr, P->nbr_split, P->nbr_idx, P->flag, sym); ++ctx->launches;
    k_node_count<<<(K + 255) / 256, 256, 0, ctx->stream>>>(K, P->tri, ncnt); ++ctx->launches;
    NL_CK(cudaGetLastError());
    if ((s = nl_scan_i64(ctx, ncnt, nptr, J)) != NL_OK) return s;
    k_node_fill<<<(K + 255) / 256, 256, 0, ctx->stream>>>(K, P->tri, nptr, ncur, ntri); ++ctx->launches;
    const size_t smem = sizeof(int32_t) * (NL_HASH_CAP + kListCap);
    NL_CK(cudaFuncSetAttribute(k_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_rows<<<J, kRowThreads, smem, ctx->stream>>>(J, nptr, ntri, P->tri, P->nbr_ptr, P->nbr_idx, sym, rcnt,
                                                   nullptr, nullptr, ovf, 0); ++ctx->launches;
    NL_CK(cudaGetLastError());
    if ((s = nl_alloc(ctx, &out->row_ptr, (size_t)J + 1)) != NL_OK) return s;
    if ((s = nl_scan_i64(ctx, rcnt, out->row_ptr, J)) != NL_OK) return s;
    k_sum_stats<<<256, 256, 0, ctx->stream>>>(K, P->E, P->flag, P->qp_a, P->cnt_a, st); ++ctx->launches;
    k_row_max<<<64, 256, 0, ctx->stream>>>(J, rcnt, st); ++ctx->launches;
    NL_CK(cudaGetLastError());
    int64_t nnz = 0;
    int hovf = 0, herr = 0;
    unsigned long long hst[4];
    NL_CK(cudaMemcpyAsync(&herr, P->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    NL_CK(cudaMemcpyAsync(&nnz, out->row_ptr + J, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    NL_CK(cudaMemcpyAsync(&hovf, ovf, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    NL_CK(cudaMemcpyAsync(hst, st, sizeof hst, cudaMemcpyDeviceToHost, ctx->stream));
    NL_CK(cudaStreamSynchronize(ctx->stream));
    if (hovf) return nl_fail(ctx, NL_EUNSUPPORTED, "a matrix row has more than 4095 columns");
    if (herr) return nl_fail(ctx, NL_EUNSUPPORTED, "a region exceeded the vertex buffer (error word " +
                                                     std::to_string(herr) + ")");
    out->n = J;
    out->nnz = nnz;
    out->n_pairs = (int64_t)hst[0];
    out->n_qp_pairs = (int64_t)hst[1];
    out->n_inter = (int64_t)hst[2];
    P->max_row = (int64_t)hst[3];
    if ((s = nl_alloc(ctx, &out->col_idx, (size_t)nnz)) != NL_OK) return s;
    if ((s = nl_alloc(ctx, &out->val, (size_t)nnz)) != NL_OK) return s;
    k_rows<<<J, kRowThreads, smem, ctx->stream>>>(J, nptr, ntri, P->tri, P->nbr_ptr, P->nbr_idx, sym, nullptr,
                                                   out->row_ptr, out->col_idx, ovf, 1); ++ctx->launches;
    NL_CK(cudaGetLastError());
    if ((s = nl_alloc(ctx, &P->lslot, 6 * (size_t)K)) != NL_OK) return s;
    if ((s = nl_alloc(ctx, &P->tslot, (size_t)nnz)) != NL_OK) return s;
    if ((s = nl_alloc(ctx, &P->W, (size_t)nnz)) != NL_OK) return s;
    k_local_slots<<<(K + 255) / 256, 256, 0, ctx->stream>>>(K, P->tri, out->row_ptr, out->col_idx, P->lslot); ++ctx->launches;
    k_tslot<<<(unsigned)(((int64_t)J * 32 + 255) / 256), 256, 0, ctx->stream>>>(J, out->row_ptr, out->col_idx,
                                                                              P->tslot); ++ctx->launches;
    NL_CK(cudaGetLastError());
    NL_CK(cudaFreeAsync(sym, ctx->stream));
    NL_CK(cudaFreeAsync(ncnt, ctx->stream));
    NL_CK(cudaFreeAsync(nptr, ctx->stream));
    NL_CK(cudaFreeAsync(ncur, ctx->stream));
    NL_CK(cudaFreeAsync(rcnt, ctx->stream));
    NL_CK(cudaFreeAsync(ntri, ctx->stream));
    NL_CK(cudaFreeAsync(ovf, ctx->stream));
    NL_CK(cudaFreeAsync(st, ctx->stream));
    return NL_OK;
}

template <typename T>
static nl_status launch_scatter(nl_ctx *ctx, nl_plan *P, nl_csr *out)
{
    const int K = P->K;
    int cap = (int)(((P->max_row > 0 ? P->max_row : 1) + 3) & ~3LL);   // multiple of 4: keeps the T array aligned
    int warps = 4;
    while (warps > 1 && (size_t)warps * 3 * cap * (sizeof(int32_t) + sizeof(T)) > 96 * 1024) warps >>= 1;
    size_t smem = (size_t)warps * 3 * cap * (sizeof(int32_t) + sizeof(T));
    if (smem > 96 * 1024) {   // very long rows: stage none, search in global memory
        cap = 0;
        smem = 0;
    }
    NL_CK(cudaFuncSetAttribute(k_scatter<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(96 * 1024)));
    const unsigned grid = (unsigned)((K + warps - 1) / warps);
    k_scatter<T><<<grid, 32 * warps, smem, ctx->stream>>>(K, P->E, P->tri, P->nbr_ptr, P->nbr_idx, P->flag,
                                                           (const T *)P->blk, P->maa, P->lslot, out->row_ptr,
                                                           out->col_idx, P->W, P->err, cap); ++ctx->launches;
    NL_CK(cudaGetLastError());
    return NL_OK;
}

nl_status nl_run_scatter(nl_ctx *ctx, nl_plan *P, nl_csr *out)
{
    NL_CK(cudaMemsetAsync(P->W, 0, sizeof(double) * (size_t)out->nnz, ctx->stream));
    nl_status s = P->cfg.prec == NL_PREC_FP64 ? launch_scatter<double>(ctx, P, out) : launch_scatter<float>(ctx, P, out);
    if (s != NL_OK) return s;
    if (out->nnz > 0) {
        k_symmetrize<<<(unsigned)((out->nnz + 255) / 256), 256, 0, ctx->stream>>>(out->nnz, P->W, P->tslot,
                                                                                 out->val, P->err); ++ctx->launches;
    }
    NL_CK(cudaGetLastError());
    return NL_OK;
}
