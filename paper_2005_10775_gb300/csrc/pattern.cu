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

#include <new>

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
    __syncthreads();   // every thread has read the column count before the counter is reused
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
__device__ __forceinline__ void scatter_outer(int K, int J, int64_t E, const int32_t *tri, const int64_t *ptr,
                                              const int32_t *idx, const uint8_t *flag, const T *blk,
                                              const double *maa, const int64_t *lslot, const int64_t *row_ptr,
                                              const int32_t *col, double *W, int *err, int cap, int a, int lane,
                                              int32_t *scol, T *sacc)
{
    const int ar[3] = {tri[3 * a], tri[3 * a + 1], tri[3 * a + 2]};
#ifdef NL_CHECKS
    // debug build: indices checked, a bad one recorded (bit 64) and its access skipped
    const int64_t nnz_chk = row_ptr[J];
    for (int i = 0; i < 3; i++)
        if (ar[i] < 0 || ar[i] >= J) {
            atomicOr(err, 64);
            return;
        }
    if (ptr[a] < 0 || ptr[a + 1] > E || ptr[a] > ptr[a + 1]) {
        atomicOr(err, 64);
        return;
    }
#endif
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
#ifdef NL_CHECKS
        if (b < 0 || b >= K) {
            atomicOr(err, 64);
            continue;
        }
#endif
        const int bn[3] = {tri[3 * b], tri[3 * b + 1], tri[3 * b + 2]};
#ifdef NL_CHECKS
        if (bn[0] < 0 || bn[0] >= J || bn[1] < 0 || bn[1] >= J || bn[2] < 0 || bn[2] >= J) {
            atomicOr(err, 64);
            continue;
        }
#endif
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
#ifdef NL_CHECKS
                    if (sl >= nnz_chk) {
                        atomicOr(err, 64);
                        continue;
                    }
#endif
                    if (sl >= 0) atomicAdd(&W[sl], -(double)v); else atomicOr(err, 2);
                }
            }
        for (int p = 0; p < 6; p++) {
            double v = (double)blk[(int64_t)(9 + p) * E + e];
            if (p < 3) v *= 0.5;
            const int64_t sl = lslot[(int64_t)p * K + b];
#ifdef NL_CHECKS
            if (sl >= nnz_chk) {
                atomicOr(err, 64);
                continue;
            }
#endif
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

template <typename T>
__global__ void k_scatter(int K, int J, int64_t E, const int32_t *tri, const int64_t *ptr, const int32_t *idx,
                          const uint8_t *flag, const T *blk, const double *maa, const int64_t *lslot,
                          const int64_t *row_ptr, const int32_t *col, double *W, int *err, int cap)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int a = blockIdx.x * (blockDim.x >> 5) + wib;
    int32_t *scol = (int32_t *)(smem_raw + (size_t)wib * 3 * cap * (sizeof(int32_t) + sizeof(T)));
    T *sacc = (T *)(scol + 3 * cap);
    if (a >= K) return;
    scatter_outer<T>(K, J, E, tri, ptr, idx, flag, blk, maa, lslot, row_ptr, col, W, err, cap, a, lane, scol, sacc);
}

// ---- batched scatter: every problem of a batch in one launch per value type ----
// off: prefix sums over the problems (of K for the scatter, of nnz for the others);
// the problem of global index g is the last p with off[p] <= g.
__device__ __forceinline__ int batch_problem(const int64_t *off, int n, int64_t g)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename T>
__global__ void k_scatter_batch(const ScatterArgs *__restrict__ S, const int64_t *__restrict__ koff, int n, int cap)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (g >= koff[n]) return;
    int32_t *scol = (int32_t *)(smem_raw + (size_t)wib * 3 * cap * (sizeof(int32_t) + sizeof(T)));
    T *sacc = (T *)(scol + 3 * cap);
    const int p = batch_problem(koff, n, g);
    const ScatterArgs &A = S[p];
    scatter_outer<T>(A.K, A.J, A.E, A.tri, A.ptr, A.idx, A.flag, (const T *)A.blk, A.maa, A.lslot, A.row_ptr, A.col,
                     A.W, A.err, cap, (int)(g - koff[p]), lane, scol, sacc);
}

__global__ void k_zero_batch(const ScatterArgs *__restrict__ S, const int64_t *__restrict__ zoff, int n)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= zoff[n]) return;
    const int p = batch_problem(zoff, n, g);
    S[p].W[g - zoff[p]] = 0.0;
}

__global__ void k_symmetrize_batch(const ScatterArgs *__restrict__ S, const int64_t *__restrict__ zoff, int n)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= zoff[n]) return;
    const int p = batch_problem(zoff, n, g);
    const ScatterArgs &A = S[p];
    const int64_t sl = g - zoff[p], t = A.tslot[sl];
#ifdef NL_CHECKS
    if (t >= zoff[p + 1] - zoff[p]) {
        atomicOr(A.err, 64);
        return;
    }
#endif
    if (t >= 0) A.val[sl] = A.W[sl] + A.W[t];
    else atomicOr(A.err, 4);
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

struct nl_pat {
    uint8_t *sym = nullptr;
    int64_t *ncnt = nullptr, *nptr = nullptr, *ncur = nullptr, *rcnt = nullptr;
    int32_t *ntri = nullptr;
    int *ovf = nullptr;
    unsigned long long *st = nullptr;
};

nl_pat *nl_pat_new() { return new (std::nothrow) nl_pat(); }

namespace {
template <class T>
void free_async(T *&p, cudaStream_t s)
{
    if (p) cudaFreeAsync((void *)p, s);
    p = nullptr;
}
}  // namespace

void nl_pat_delete(nl_pat *T, cudaStream_t s)
{
    if (!T) return;
    free_async(T->sym, s); free_async(T->ncnt, s); free_async(T->nptr, s); free_async(T->ncur, s);
    free_async(T->rcnt, s); free_async(T->ntri, s); free_async(T->ovf, s); free_async(T->st, s);
    delete T;
}

nl_status nl_pattern_a(nl_ctx *ctx, nl_plan *P, nl_csr *out, nl_pat *T, nl_host_slot *h)
{
    const int K = P->K, J = P->J;
    cudaStream_t st = ctx->stream;
    nl_status s;
    NL_CK(cudaMallocAsync((void **)&T->sym, P->E ? P->E : 1, st));
    NL_CK(cudaMallocAsync((void **)&T->ncnt, sizeof(int64_t) * (J + 1), st));
    NL_CK(cudaMallocAsync((void **)&T->nptr, sizeof(int64_t) * (J + 1), st));
    NL_CK(cudaMallocAsync((void **)&T->ncur, sizeof(int64_t) * (J + 1), st));
    NL_CK(cudaMallocAsync((void **)&T->rcnt, sizeof(int64_t) * (J + 1), st));
    NL_CK(cudaMallocAsync((void **)&T->ntri, sizeof(int32_t) * 3 * (size_t)K, st));
    NL_CK(cudaMallocAsync((void **)&T->ovf, sizeof(int), st));
    NL_CK(cudaMallocAsync((void **)&T->st, sizeof(unsigned long long) * 4, st));
    NL_CK(cudaMemsetAsync(T->ncnt, 0, sizeof(int64_t) * (J + 1), st));
    NL_CK(cudaMemsetAsync(T->ncur, 0, sizeof(int64_t) * (J + 1), st));
    NL_CK(cudaMemsetAsync(T->ovf, 0, sizeof(int), st));
    NL_CK(cudaMemsetAsync(T->st, 0, sizeof(unsigned long long) * 4, st));
    const unsigned wgrid = (unsigned)(((int64_t)K * 32 + 255) / 256);
    k_symflag<<<wgrid, 256, 0, st>>>(K, P->nbr_ptr, P->nbr_split, P->nbr_idx, P->flag, T->sym); ++ctx->launches;
    k_node_count<<<(K + 255) / 256, 256, 0, st>>>(K, P->tri, T->ncnt); ++ctx->launches;
    NL_CK(cudaGetLastError());
    if ((s = nl_scan_i64(ctx, T->ncnt, T->nptr, J)) != NL_OK) return s;
    k_node_fill<<<(K + 255) / 256, 256, 0, st>>>(K, P->tri, T->nptr, T->ncur, T->ntri); ++ctx->launches;
    const size_t smem = sizeof(int32_t) * (NL_HASH_CAP + kListCap);
    NL_CK(cudaFuncSetAttribute(k_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_rows<<<J, kRowThreads, smem, st>>>(J, T->nptr, T->ntri, P->tri, P->nbr_ptr, P->nbr_idx, T->sym, T->rcnt,
                                         nullptr, nullptr, T->ovf, 0); ++ctx->launches;
    NL_CK(cudaGetLastError());
    if ((s = nl_alloc(ctx, &out->row_ptr, (size_t)J + 1)) != NL_OK) return s;
    if ((s = nl_scan_i64(ctx, T->rcnt, out->row_ptr, J)) != NL_OK) return s;
    k_sum_stats<<<256, 256, 0, st>>>(K, P->E, P->flag, P->qp_a, P->cnt_a, T->st); ++ctx->launches;
    k_row_max<<<64, 256, 0, st>>>(J, T->rcnt, T->st); ++ctx->launches;
    NL_CK(cudaGetLastError());
    NL_CK(cudaMemcpyAsync(&h->err, P->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    NL_CK(cudaMemcpyAsync(&h->nnz, out->row_ptr + J, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    NL_CK(cudaMemcpyAsync(&h->row_ovf, T->ovf, sizeof(int), cudaMemcpyDeviceToHost, st));
    NL_CK(cudaMemcpyAsync(h->pat, T->st, sizeof h->pat, cudaMemcpyDeviceToHost, st));
    return NL_OK;
}

nl_status nl_pattern_b(nl_ctx *ctx, nl_plan *P, nl_csr *out, nl_pat *T, const nl_host_slot *h)
{
    const int K = P->K, J = P->J;
    cudaStream_t st = ctx->stream;
    nl_status s;
    if (h->row_ovf) return nl_fail(ctx, NL_EUNSUPPORTED, "a matrix row has more than 4095 columns");
    if (h->err) return nl_fail(ctx, NL_EUNSUPPORTED, "a region exceeded the vertex buffer (error word " +
                                                       std::to_string(h->err) + ")");
    const int64_t nnz = h->nnz;
    out->n = J;
    out->nnz = nnz;
    out->n_pairs = (int64_t)h->pat[0];
    out->n_qp_pairs = (int64_t)h->pat[1];
    out->n_inter = (int64_t)h->pat[2];
    P->max_row = (int64_t)h->pat[3];
    if ((s = nl_alloc(ctx, &out->col_idx, (size_t)nnz)) != NL_OK) return s;
    if ((s = nl_alloc(ctx, &out->val, (size_t)nnz)) != NL_OK) return s;
    const size_t smem = sizeof(int32_t) * (NL_HASH_CAP + kListCap);
    k_rows<<<J, kRowThreads, smem, st>>>(J, T->nptr, T->ntri, P->tri, P->nbr_ptr, P->nbr_idx, T->sym, nullptr,
                                         out->row_ptr, out->col_idx, T->ovf, 1); ++ctx->launches;
    NL_CK(cudaGetLastError());
    if ((s = nl_alloc(ctx, &P->lslot, 6 * (size_t)K)) != NL_OK) return s;
    if ((s = nl_alloc(ctx, &P->tslot, (size_t)nnz)) != NL_OK) return s;
    if ((s = nl_alloc(ctx, &P->W, (size_t)nnz)) != NL_OK) return s;
    k_local_slots<<<(K + 255) / 256, 256, 0, st>>>(K, P->tri, out->row_ptr, out->col_idx, P->lslot); ++ctx->launches;
    k_tslot<<<(unsigned)(((int64_t)J * 32 + 255) / 256), 256, 0, st>>>(J, out->row_ptr, out->col_idx, P->tslot);
    ++ctx->launches;
    NL_CK(cudaGetLastError());
    return NL_OK;
}

nl_status nl_build_pattern(nl_ctx *ctx, nl_plan *P, nl_csr *out)
{
    nl_host_slot *h = nullptr;
    nl_status s = nl_host_slots(ctx, 1, &h);
    if (s != NL_OK) return s;
    nl_pat *T = nl_pat_new();
    if (!T) return nl_fail(ctx, NL_ENOMEM, "host allocation failed");
    if ((s = nl_pattern_a(ctx, P, out, T, h)) == NL_OK) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        s = e == cudaSuccess ? nl_pattern_b(ctx, P, out, T, h) : nl_cuda_fail(ctx, e, "cudaStreamSynchronize");
    }
    nl_pat_delete(T, ctx->stream);
    return s;
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
    k_scatter<T><<<grid, 32 * warps, smem, ctx->stream>>>(K, P->J, P->E, P->tri, P->nbr_ptr, P->nbr_idx, P->flag,
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

// ---- batched scatter launches ----
nl_status nl_launch_zero_batch(nl_ctx *ctx, const ScatterArgs *dS, const int64_t *dzoff, int n, int64_t total)
{
    if (total <= 0) return NL_OK;
    k_zero_batch<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(dS, dzoff, n); ++ctx->launches;
    NL_CK(cudaGetLastError());
    return NL_OK;
}

nl_status nl_launch_symmetrize_batch(nl_ctx *ctx, const ScatterArgs *dS, const int64_t *dzoff, int n,
                                     int64_t total)
{
    if (total <= 0) return NL_OK;
    k_symmetrize_batch<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(dS, dzoff, n); ++ctx->launches;
    NL_CK(cudaGetLastError());
    return NL_OK;
}

template <typename T>
static nl_status launch_scatter_batch(nl_ctx *ctx, const ScatterArgs *dS, const int64_t *dkoff, int n,
                                      int64_t totalK, int64_t max_row, bool set_attr)
{
    if (totalK <= 0) return NL_OK;
    int cap = (int)(((max_row > 0 ? max_row : 1) + 3) & ~3LL);
    int warps = 4;
    while (warps > 1 && (size_t)warps * 3 * cap * (sizeof(int32_t) + sizeof(T)) > 96 * 1024) warps >>= 1;
    size_t smem = (size_t)warps * 3 * cap * (sizeof(int32_t) + sizeof(T));
    if (smem > 96 * 1024) {
        cap = 0;
        smem = 0;
    }
    if (set_attr)
        NL_CK(cudaFuncSetAttribute(k_scatter_batch<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(96 * 1024)));
    const unsigned grid = (unsigned)((totalK + warps - 1) / warps);
    k_scatter_batch<T><<<grid, 32 * warps, smem, ctx->stream>>>(dS, dkoff, n, cap); ++ctx->launches;
    NL_CK(cudaGetLastError());
    return NL_OK;
}

nl_status nl_launch_scatter_batch(nl_ctx *ctx, bool f64, const ScatterArgs *dS, const int64_t *dkoff, int n,
                                  int64_t totalK, int64_t max_row, bool set_attr)
{
    return f64 ? launch_scatter_batch<double>(ctx, dS, dkoff, n, totalK, max_row, set_attr)
               : launch_scatter_batch<float>(ctx, dS, dkoff, n, totalK, max_row, set_attr);
}
