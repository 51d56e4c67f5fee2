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
// interacting pair, -M_ab at (a_i, b_k), and per triangle the upper triangles of M_aa
// and of the summed M_bb of its pairs (diagonals halved).  The transposed blocks come
// from the final W + W^T pass through the transposed-slot map.
#include <cuda_runtime.h>

#include <stdlib.h>

#include <new>
#include <type_traits>

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

constexpr int kSymWarps = 8;

// sym[e] for a pair (a, b) that does not interact in direction a: the flag of (b, a), found
// in T_b's list (two sorted segments, interior then boundary, split at split[b]; a triangle
// appears once).  A pair that fails in one direction lies near the edge of the horizon, so
// T_a is looked up in the boundary segment first.
__device__ __forceinline__ void sym_lookup(const int64_t *ptr, const int64_t *split, const int32_t *idx,
                                           const uint8_t *flag, uint8_t *sym, int a, int64_t e, int b)
{
    int64_t m = find_in(idx, split[b], ptr[b + 1], a);
    if (m < 0) m = find_in(idx, ptr[b], split[b], a);
    sym[e] = m >= 0 ? flag[m] : (uint8_t)0;
}

// symmetric flag: pair (a, b) or (b, a) interacts; warp per a.  The lanes whose pair does not
// interact in direction a queue it in shared memory, and the warp runs the lookups 32 at a
// time, so a round of the list never waits on one lane's binary searches.
__global__ void __launch_bounds__(kSymWarps * 32) k_symflag(int K, const int64_t *ptr, const int64_t *split,
                                                             const int32_t *idx, const uint8_t *flag, uint8_t *sym)
{
    __shared__ int32_t qoff[kSymWarps][64], qb[kSymWarps][64];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int a = blockIdx.x * kSymWarps + w;
    if (a >= K) return;   // the whole warp: no block barrier follows
    const int64_t e0 = ptr[a], e1 = ptr[a + 1];
    int nq = 0;   // queued lookups, < 32 between rounds
    for (int64_t eb = e0; eb < e1; eb += 32) {
        const int64_t e = eb + lane;
        const bool in = e < e1;
        const int b = in ? idx[e] : 0;
        const uint8_t f = in ? flag[e] : (uint8_t)1;
        const bool need = in && !f;
        if (in && f) sym[e] = f;
        const unsigned m = __ballot_sync(0xffffffffu, need);
        if (need) {
            const int p = nq + __popc(m & ((1u << lane) - 1u));
            qoff[w][p] = (int32_t)(e - e0);
            qb[w][p] = b;
        }
        nq += __popc(m);
        __syncwarp();
        if (nq >= 32) {
            sym_lookup(ptr, split, idx, flag, sym, a, e0 + qoff[w][lane], qb[w][lane]);
            const int rest = nq - 32;
            int o2 = 0, b2 = 0;
            if (lane < rest) {
                o2 = qoff[w][32 + lane];
                b2 = qb[w][32 + lane];
            }
            __syncwarp();
            if (lane < rest) {
                qoff[w][lane] = o2;
                qb[w][lane] = b2;
            }
            nq = rest;
            __syncwarp();
        }
    }
    if (lane < nq) sym_lookup(ptr, split, idx, flag, sym, a, e0 + qoff[w][lane], qb[w][lane]);
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

// FP32 scatter: exponent of a bound on what node j's column of a row of T_a receives per unit
// of sum_q |W_q| (that is, per |T_a| sum_q |w_q|).  Each triangle T_b at j adds at most
// s0max(T_b), a bound on int_{S cap T_b} gamma(x, y) dy over all points x and sets S: kc |T_b|
// for a constant kernel, c 2 sqrt(pi |T_b|) for c / |x - y| (1/r integrated over the disc of
// area |T_b| centred at x, the largest such integral), each with the per-point margin of the
// numeric phase (1.25, 2.5 for the singular quadrature).  The bound taken, (triangles at j) x
// max s0max, is order-free and so the same in every run.  fxe (zeroed) receives 128 + the
// largest floor(log2) of it in FP32 over the nodes (an integer maximum: the same in every run).
__global__ void k_node_exp(int J, const int64_t *nptr, const int32_t *ntri, const double *area, int inv, double c,
                           int *fxe)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= J) return;
    double m = 0.0;
    for (int64_t s = nptr[j]; s < nptr[j + 1]; s++) {
        const double A = area[ntri[s]];
        m = fmax(m, inv ? 2.5 * c * 2.0 * sqrt(3.14159265358979323846 * A) : 1.25 * c * A);
    }
    const double nb = (double)(nptr[j + 1] - nptr[j]) * m;
    int e = nb < 1e38 ? ((__float_as_int((float)nb) >> 23) & 255) - 127 : 126;
    e = e < -126 ? -126 : (e > 126 ? 126 : e);
    atomicMax(fxe, e + 128);
}

constexpr int kRowThreads = 256;
constexpr int kListCap = NL_HASH_CAP / 2;   // longest row (columns) the pattern accepts, plus one
constexpr int kRowWaveBlocks = 152 * 8;   // one wave of k_rows blocks on 152 SMs (the rebuild pass)

// insert c into the shared hash set tab (mask + 1 slots): 1 new, 0 present, -1 set full
__device__ __forceinline__ int set_insert(int32_t *tab, unsigned mask, int c)
{
    unsigned h = ((unsigned)c * 2654435761u) & mask;
    for (unsigned t = 0; t <= mask; t++) {
        const int old = atomicCAS(&tab[h], -1, c);
        if (old == -1) return 1;
        if (old == c) return 0;
        h = (h + 1) & mask;
    }
    return -1;
}

// Block scratch of set_sorted (shared memory)
struct SortScratch {
    int n, lo, hi;
    int wsum[kRowThreads / 32 + 1];
};

// The n columns held in the hash set tab (H slots, -1 empty) in ascending order at out[0, n),
// with lst (2^lbits ints of shared memory) as scratch.  The columns of a row are the nodes near
// node j, so they usually span few indices: one bit per column in a bitmap over [min, max]
// (lst as 2^lbits words), written in order through prefix counts over the words.  A wider span
// takes a bitonic sort of the compacted columns (2^lbits >= n slots).  Every thread of the
// block calls it.
__device__ __forceinline__ void set_sorted(const int32_t *tab, int H, int32_t *lst, int lbits, int n, SortScratch &sc,
                                           int32_t *out)
{
    const int lane = threadIdx.x & 31;
    __syncthreads();   // every thread has read the column count before the scratch is reused
    if (threadIdx.x == 0) {
        sc.n = 0;
        sc.lo = 0x7fffffff;
        sc.hi = -1;
    }
    __syncthreads();
    int lo = 0x7fffffff, hi = -1;
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        const int v = tab[i];
        if (v >= 0) {
            lo = min(lo, v);
            hi = max(hi, v);
        }
    }
    for (int off = 16; off; off >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, off));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, off));
    }
    if (lane == 0) {
        atomicMin(&sc.lo, lo);
        atomicMax(&sc.hi, hi);
    }
    __syncthreads();
    lo = sc.lo;
    const int64_t span = n > 0 ? (int64_t)sc.hi - lo + 1 : 0;
    if (span <= ((int64_t)32 << lbits)) {
        uint32_t *bm = reinterpret_cast<uint32_t *>(lst);
        const int nw = (int)((span + 31) >> 5);
        for (int w = threadIdx.x; w < nw; w += blockDim.x) bm[w] = 0u;
        __syncthreads();
        for (int i = threadIdx.x; i < H; i += blockDim.x) {
            const int v = tab[i];
            if (v >= 0) atomicOr(&bm[(v - lo) >> 5], 1u << ((v - lo) & 31));
        }
        __syncthreads();
        // each thread owns a run of consecutive words
        const int per = (nw + kRowThreads - 1) / kRowThreads;
        const int w0 = min(nw, (int)threadIdx.x * per), w1 = min(nw, w0 + per);
        int c = 0;
        for (int w = w0; w < w1; w++) c += __popc(bm[w]);
        int total = 0;
        int p = nl_block_scan<kRowThreads>(c, sc.wsum, &total);
        for (int w = w0; w < w1; w++)
            for (uint32_t m = bm[w]; m; m &= m - 1) out[p++] = lo + (w << 5) + __ffs(m) - 1;
        return;
    }
    for (int i0 = 0; i0 < H; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        const int val = i < H ? tab[i] : -1;
        const unsigned bal = __ballot_sync(0xffffffffu, val >= 0);
        int base = 0;
        if (lane == 0 && bal) base = atomicAdd(&sc.n, __popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (val >= 0) lst[base + __popc(bal & ((1u << lane) - 1u))] = val;
    }
    int p = 1;
    while (p < n) p <<= 1;
    for (int i = n + threadIdx.x; i < p; i += blockDim.x) lst[i] = 0x7fffffff;
    __syncthreads();
    for (int k = 2; k <= p; k <<= 1)
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int i = threadIdx.x; i < p; i += blockDim.x) {
                const int l = i ^ jj;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const int u = lst[i], w = lst[l];
                    if ((u > w) == up) {
                        lst[i] = w;
                        lst[l] = u;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = lst[i];
}

// Block per row j: the distinct nodes of the interacting candidates of the triangles around
// node j, in a shared hash set of 2^hbits slots.  Rows come from `list` (its length at *nlist,
// grid-stride) or are the block indices.  Each thread issues the loads of four candidates
// before inserting their nodes.
//   pass 0 counts.  A row whose set fills up is appended to ovf_list for a second count with
//   a larger set (without ovf_list it counts as an overflow).  With buf, a row of fewer than
//   2^lbits columns also leaves them sorted in its buffer row buf[j << lbits] (bflag[j] = 1),
//   and every other row is appended to rlist for pass 1.
//   pass 1 writes the sorted columns at row_ptr[j] (lst: 2^lbits slots).
__global__ void __launch_bounds__(kRowThreads) k_rows(int J, const int64_t *nt_ptr, const int32_t *ntri,
                                                      const int32_t *tri, const int64_t *ptr, const int32_t *idx,
                                                      const uint8_t *sym, int hbits, int lbits, const int *list,
                                                      const int *nlist, int64_t *cnt, const int64_t *row_ptr,
                                                      int32_t *col, int *ovf_list, int *ovf_n, int *overflow,
                                                      int32_t *buf, uint8_t *bflag, int *rlist, int *rn, int pass)
{
    extern __shared__ int32_t sm[];
    const int H = 1 << hbits;
    const unsigned mask = (unsigned)H - 1u;
    int32_t *tab = sm;        // [H]
    int32_t *lst = sm + H;    // [2^lbits] (pass 1, and pass 0 with buf)
    __shared__ int s_n, s_ovf;
    __shared__ SortScratch sc;
    const int nrows = list ? *nlist : J;
    const int lane = threadIdx.x & 31;
    for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
        const int j = list ? list[r] : r;
        for (int i = threadIdx.x; i < H; i += blockDim.x) tab[i] = -1;
        if (threadIdx.x == 0) {
            s_n = 0;
            s_ovf = 0;
        }
        __syncthreads();
        int mine = 0;
        bool full = false;
        for (int64_t q = nt_ptr[j]; q < nt_ptr[j + 1]; q++) {
            const int T = ntri[q];
            const int64_t e1 = ptr[T + 1];
            for (int64_t eb = ptr[T] + threadIdx.x; eb < e1; eb += 4 * (int64_t)blockDim.x) {
                int c[4];
                bool ok[4];
                for (int u = 0; u < 4; u++) {
                    const int64_t e = eb + (int64_t)u * blockDim.x;
                    ok[u] = e < e1;
                    c[u] = ok[u] ? idx[e] : 0;
                    ok[u] = ok[u] && sym[e];
                }
                int v[4][3];
                for (int u = 0; u < 4; u++)
                    for (int i = 0; i < 3; i++) v[u][i] = ok[u] ? tri[3 * c[u] + i] : -1;
                for (int u = 0; u < 4; u++)
                    if (ok[u])
                        for (int i = 0; i < 3; i++) {
                            const int st = set_insert(tab, mask, v[u][i]);
                            mine += st > 0;
                            full = full || st < 0;
                        }
            }
        }
        // block totals: one shared atomic per warp
        for (int off = 16; off; off >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, off);
        const bool wfull = __any_sync(0xffffffffu, full);
        if (lane == 0) {
            atomicAdd(&s_n, mine);
            if (wfull) s_ovf = 1;
        }
        __syncthreads();
        const int n = s_n;
        const bool ovf = s_ovf != 0 || n >= kListCap;
        const bool keep = pass == 0 && buf && !ovf && n < (1 << lbits);
        if (ovf) {
            if (threadIdx.x == 0) {
                if (ovf_list) ovf_list[atomicAdd(ovf_n, 1)] = j;
                else atomicAdd(overflow, 1);
            }
        } else if (pass == 0) {
            if (threadIdx.x == 0) cnt[j] = n;
            if (keep) set_sorted(tab, H, lst, lbits, n, sc, buf + ((int64_t)j << lbits));
        } else {
            set_sorted(tab, H, lst, lbits, n, sc, col + row_ptr[j]);
        }
        if (pass == 0 && buf && threadIdx.x == 0) {
            bflag[j] = keep ? 1 : 0;
            if (!keep) rlist[atomicAdd(rn, 1)] = j;
        }
        __syncthreads();   // the set and the counters are reused by the next row
    }
}

// the columns of the rows pass 0 kept sorted in their buffer rows; warp per row
__global__ void k_row_copy(int J, const uint8_t *bflag, const int32_t *buf, int lbits, const int64_t *row_ptr,
                           int32_t *col)
{
    const int j = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (j >= J || !bflag[j]) return;
    const int64_t o = row_ptr[j], n = row_ptr[j + 1] - o;
    const int32_t *src = buf + ((int64_t)j << lbits);
    for (int64_t i = lane; i < n; i += 32) col[o + i] = src[i];
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
// shared memory (`cap` entries per row) and adds each row entry to W once, instead of
// one FP64 atomic per pair and entry.  The columns of the three rows are indexed by a
// shared hash table (key: column node; value: the column's position in each of the
// three rows, 10 bits each), so each node of T_b costs one lookup for all three rows.
// The upper M_bb of every pair was summed per triangle b by the numeric kernels (mbb, FP64
// atomics); k_local_blocks adds M_aa + M_bb of every triangle through the local slot map.
constexpr unsigned kPosAbsent = 1023u;   // 10-bit position field: column not in that row
constexpr int kMaxCachedRow = 1022;

__device__ __forceinline__ unsigned col_hash(int c, int hbits)
{
    return ((unsigned)c * 2654435761u) >> (32 - hbits);
}

// insert column c (or find it): its slot, or -1 when the table is full
__device__ __forceinline__ int hash_insert(int32_t *key, int H, int hbits, int c)
{
    unsigned h = col_hash(c, hbits);
    for (int t = 0; t < H; t++) {
        const int old = atomicCAS(&key[h], -1, c);
        if (old == -1 || old == c) return (int)h;
        h = (h + 1) & (unsigned)(H - 1);
    }
    return -1;
}

__device__ __forceinline__ int hash_find(const int32_t *key, int H, int hbits, int c)
{
    unsigned h = col_hash(c, hbits);
    for (int t = 0; t < H; t++) {
        const int k = key[h];
        if (k == c) return (int)h;
        if (k == -1) return -1;
        h = (h + 1) & (unsigned)(H - 1);
    }
    return -1;
}

// FP32 blocks: the shared row sums are 32-bit fixed point on a power-of-two grid from their
// bound (fx_row_shift), added with native integer atomics, so they do not depend on the order
// of the adds; a sum beyond its bound sets error bit 256.  FP64 blocks: FP64 shared sums.
// 2^s as an FP32 number (s in [-126, 126]: a normal power of two, built from its bits)
__device__ __forceinline__ float pow2f(int s) { return __int_as_float((s + 127) << 23); }

// floor(log2 x) of a positive normal FP32 number, from its exponent field, clamped to [-126, 126]
__device__ __forceinline__ int exp2_floor(float x)
{
    const int e = ((__float_as_int(x) >> 23) & 255) - 127;
    return e < -126 ? -126 : (e > 126 ? 126 : e);
}

// Fixed-point shift of the rows of T_a: the sum a column of node j receives is below
// 2^(ea + 1) 2^(ej + 1) (ea: exponent of |T_a| sum_q |w_q|, ej the largest node exponent of
// k_node_exp), so every sum scaled by 2^s stays below 2^30.
__device__ __forceinline__ int fx_row_shift(int ea, int ej)
{
    const int s = 28 - ea - ej;
    return s < -126 ? -126 : (s > 126 ? 126 : s);
}

// One pair (a, b) of the scatter: flag f, its M_ab block v, added to the three rows of T_a's
// nodes (shared sums, fixed point for FP32 blocks, when cached; else FP64 atomics on W).
template <typename T, typename Acc>
__device__ __forceinline__ void scatter_pair(uint8_t f, int b, const T *v, int K, int J, const int32_t *tri,
                                             const int64_t *row_ptr, const int32_t *col, double *W, int *err,
                                             bool cached, int H, int hbits, const int *ar, const int *len, int cap,
                                             float sc, Acc *sacc, const int32_t *skey, const uint32_t *spk)
{
    if (!f) return;
#ifdef NL_CHECKS
    const int64_t nnz_chk = row_ptr[J];
    if (b < 0 || b >= K) {
        atomicOr(err, 64);
        return;
    }
#endif
    const int bn[3] = {tri[3 * b], tri[3 * b + 1], tri[3 * b + 2]};
#ifdef NL_CHECKS
    if (bn[0] < 0 || bn[0] >= J || bn[1] < 0 || bn[1] >= J || bn[2] < 0 || bn[2] >= J) {
        atomicOr(err, 64);
        return;
    }
#endif
    for (int k = 0; k < 3; k++) {
        if (cached) {
            const int sl = hash_find(skey, H, hbits, bn[k]);
            const unsigned pk = sl >= 0 ? spk[sl] : 0xffffffffu;
            for (int i = 0; i < 3; i++) {
                const unsigned pos = (pk >> (10 * i)) & kPosAbsent;
                if (pos < (unsigned)len[i]) {
                    if constexpr (sizeof(T) == sizeof(float))
                        atomicAdd(&sacc[i * cap + pos], -__float2int_rn(v[3 * i + k] * sc));
                    else
                        atomicAdd(&sacc[i * cap + pos], -v[3 * i + k]);
                } else {
                    atomicOr(err, 2);
                }
            }
        } else {
            for (int i = 0; i < 3; i++) {
                const int64_t sl = find_slot(row_ptr, col, ar[i], bn[k]);
#ifdef NL_CHECKS
                if (sl >= nnz_chk) {
                    atomicOr(err, 64);
                    continue;
                }
#endif
                if (sl >= 0) atomicAdd(&W[sl], -(double)v[3 * i + k]); else atomicOr(err, 2);
            }
        }
    }
}

template <typename T>
__device__ __forceinline__ void scatter_outer(int K, int J, int64_t E, const int32_t *tri, const int64_t *ptr,
                                              const int32_t *idx, const uint8_t *flag, const T *blk,
                                              const int64_t *row_ptr, const int32_t *col, double *W, int *err,
                                              int cap, int hbits, int a, int lane, T *sacc_t, int32_t *skey,
                                              uint32_t *spk, const double *area, const int *fxe, float ws)
{
    constexpr bool kFx = sizeof(T) == sizeof(float);
    using Acc = typename std::conditional<kFx, int, T>::type;
    Acc *sacc = reinterpret_cast<Acc *>(sacc_t);
    const int ar[3] = {tri[3 * a], tri[3 * a + 1], tri[3 * a + 2]};
#ifdef NL_CHECKS
    // debug build: indices checked, a bad one recorded (bit 64) and its access skipped
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
    const int H = 1 << hbits;
    int64_t r0[3];
    int len[3];
    for (int i = 0; i < 3; i++) {
        r0[i] = row_ptr[ar[i]];
        len[i] = (int)(row_ptr[ar[i] + 1] - r0[i]);
    }
    bool cached = cap > 0 && len[0] <= cap && len[1] <= cap && len[2] <= cap;
    int shift = 0;   // FP32 blocks: fixed-point shift of the shared row sums
    if (cached) {
        for (int k = lane; k < H; k += 32) {
            skey[k] = -1;
            spk[k] = 0xffffffffu;
        }
        for (int k = lane; k < 3 * cap; k += 32) sacc[k] = (Acc)0;
        __syncwarp();
        bool full = false;
        for (int i = 0; i < 3; i++)
            for (int k = lane; k < len[i]; k += 32) {
                const int sl = hash_insert(skey, H, hbits, col[r0[i] + k]);
                if (sl < 0) {
                    full = true;
                    continue;
                }
                atomicAnd(&spk[sl], ~((kPosAbsent ^ (unsigned)k) << (10 * i)));
            }
        cached = !__any_sync(0xffffffffu, full);   // a full table: this triangle searches in global memory
        if constexpr (kFx) shift = fx_row_shift(exp2_floor((float)(area[a] * (double)ws)), *fxe - 128);
        __syncwarp();
    }
    const float sc = pow2f(shift);
    // the next pair's loads are issued before this pair's lookups and adds: the DRAM latency
    // of one iteration overlaps the shared-memory work of the previous one
    const int64_t e_end = ptr[a + 1];
    int64_t e = ptr[a] + lane;
    uint8_t f = 0;
    int b = 0;
    T v[9];
    if (e < e_end) {
        f = flag[e];
        b = idx[e];
        for (int p = 0; p < 9; p++) v[p] = blk[(int64_t)p * E + e];
    }
    for (; e < e_end; e += 32) {
        const int64_t en = e + 32;
        uint8_t fn = 0;
        int bnx = 0;
        T vn[9];
        if (en < e_end) {
            fn = flag[en];
            bnx = idx[en];
            for (int p = 0; p < 9; p++) vn[p] = blk[(int64_t)p * E + en];
        } else {
            for (int p = 0; p < 9; p++) vn[p] = (T)0;
        }
        scatter_pair<T, Acc>(f, b, v, K, J, tri, row_ptr, col, W, err, cached, H, hbits, ar, len, cap, sc, sacc,
                             skey, spk);
        f = fn;
        b = bnx;
        for (int p = 0; p < 9; p++) v[p] = vn[p];
    }
    __syncwarp();
    if (cached) {
        const double inv = (double)pow2f(-shift);
        for (int i = 0; i < 3; i++)
            for (int k = lane; k < len[i]; k += 32) {
                const Acc x = sacc[i * cap + k];
                if (x == (Acc)0) continue;
                if constexpr (kFx) {
                    if (x > (1 << 30) || x < -(1 << 30)) atomicOr(err, 256);
                    atomicAdd(&W[r0[i] + k], (double)x * inv);
                } else {
                    atomicAdd(&W[r0[i] + k], (double)x);
                }
            }
    }
}

// M_aa + M_bb of every triangle into W through its local slots (diagonal halved: D = W + W^T),
// leaving mbb zeroed (the numeric phase also zeroes it before it sums)
__device__ __forceinline__ void local_block(int K, int t, const double *maa, double *mbb, const int64_t *lslot,
                                            double *W, int *err)
{
    for (int p = 0; p < 6; p++) {
        double v = maa[(int64_t)p * K + t] + mbb[(int64_t)p * K + t];
        mbb[(int64_t)p * K + t] = 0.0;
        if (p < 3) v *= 0.5;
        const int64_t sl = lslot[(int64_t)p * K + t];
        if (sl >= 0) atomicAdd(&W[sl], v); else atomicOr(err, 2);
    }
}

__global__ void k_local_blocks(int K, const double *maa, double *mbb, const int64_t *lslot, double *W, int *err)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < K) local_block(K, t, maa, mbb, lslot, W, err);
}

// shared memory of one warp of the scatter: row accumulators [3][cap] (T), hash keys and
// packed positions [H] (cap a multiple of 4 keeps the int arrays aligned after a float array)
template <typename T>
__host__ __device__ constexpr size_t scatter_warp_bytes(int cap, int hbits)
{
    return cap > 0 ? 3 * (size_t)cap * sizeof(T) + ((size_t)8 << hbits) : 0;
}

template <typename T>
__device__ __forceinline__ void scatter_warp_smem(unsigned char *raw, int wib, int cap, int hbits, T *&sacc,
                                                  int32_t *&skey, uint32_t *&spk)
{
    unsigned char *base = raw + (size_t)wib * scatter_warp_bytes<T>(cap, hbits);
    sacc = (T *)base;
    skey = (int32_t *)(base + 3 * (size_t)cap * sizeof(T));
    spk = (uint32_t *)(skey + (1 << hbits));
}

template <typename T>
__global__ void k_scatter(int K, int J, int64_t E, const int32_t *tri, const int64_t *ptr, const int32_t *idx,
                          const uint8_t *flag, const T *blk, const int64_t *row_ptr, const int32_t *col,
                          double *W, int *err, int cap, int hbits, const double *area, const int *fxe,
                          float ws)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int a = blockIdx.x * (blockDim.x >> 5) + wib;
    T *sacc;
    int32_t *skey;
    uint32_t *spk;
    scatter_warp_smem<T>(smem_raw, wib, cap, hbits, sacc, skey, spk);
    if (a >= K) return;
    scatter_outer<T>(K, J, E, tri, ptr, idx, flag, blk, row_ptr, col, W, err, cap, hbits, a, lane, sacc, skey,
                     spk, area, fxe, ws);
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
__global__ void k_scatter_batch(const ScatterArgs *__restrict__ S, const int64_t *__restrict__ koff, int n, int cap,
                                int hbits)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (g >= koff[n]) return;
    T *sacc;
    int32_t *skey;
    uint32_t *spk;
    scatter_warp_smem<T>(smem_raw, wib, cap, hbits, sacc, skey, spk);
    const int p = batch_problem(koff, n, g);
    const ScatterArgs &A = S[p];
    scatter_outer<T>(A.K, A.J, A.E, A.tri, A.ptr, A.idx, A.flag, (const T *)A.blk, A.row_ptr, A.col, A.W,
                     A.err, cap, hbits, (int)(g - koff[p]), lane, sacc, skey, spk, A.area, A.fxe, A.ws);
}

// M_aa + M_bb of every triangle of every problem (koff: prefix sums of K)
__global__ void k_local_blocks_batch(const ScatterArgs *__restrict__ S, const int64_t *__restrict__ koff, int n)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= koff[n]) return;
    const int p = batch_problem(koff, n, g);
    const ScatterArgs &A = S[p];
    local_block(A.K, (int)(g - koff[p]), A.maa, A.mbb, A.lslot, A.W, A.err);
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
    // the flags are bytes of 0 or 1: 16 at a time from the first 16-byte boundary, summed by bit
    // counts; the bytes before it and after the last full 16 one at a time
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
    const int64_t head = min(E, (int64_t)((16u - ((uintptr_t)flag & 15u)) & 15u));
    const int64_t n16 = (E - head) >> 4;
    const uint4 *f16 = reinterpret_cast<const uint4 *>(flag + head);
    for (int64_t v = tid; v < n16; v += nth) {
        const uint4 w = f16[v];
        p += __popc(w.x) + __popc(w.y) + __popc(w.z) + __popc(w.w);
    }
    if (tid < head) p += flag[tid];
    for (int64_t e = head + (n16 << 4) + tid; e < E; e += nth) p += flag[e];
    for (int64_t a = tid; a < K; a += nth) {
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
    int *olist = nullptr, *on = nullptr;   // rows whose first count filled its hash set
    int32_t *buf = nullptr;                // rows sorted by the first count: J rows of 2^lbits
    uint8_t *bflag = nullptr;              // row j is in buf
    int *rlist = nullptr, *rn = nullptr;   // the other rows, rebuilt by the column write
    int lbits = 0;
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
    free_async(T->olist, s); free_async(T->on, s);
    free_async(T->buf, s); free_async(T->bflag, s); free_async(T->rlist, s); free_async(T->rn, s);
    delete T;
}

// log2 of the smallest power of two >= n, within [64, NL_HASH_CAP]
static int row_set_bits(int64_t n)
{
    int b = 6;
    while ((int64_t(1) << b) < n && (1 << b) < NL_HASH_CAP) b++;
    return b;
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
    NL_CK(cudaMallocAsync((void **)&T->olist, sizeof(int) * (J + 1), st));
    NL_CK(cudaMallocAsync((void **)&T->on, sizeof(int), st));
    NL_CK(cudaMemsetAsync(T->on, 0, sizeof(int), st));
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
    if (P->cfg.prec != NL_PREC_FP64 && J > 0) {
        nl_free(P->fxe, st);
        if ((s = nl_alloc(ctx, &P->fxe, 1)) != NL_OK) return s;
        NL_CK(cudaMemsetAsync(P->fxe, 0, sizeof(int), st));
        k_node_exp<<<(J + 255) / 256, 256, 0, st>>>(J, T->nptr, T->ntri, P->area,
                                                    P->cfg.kernel == NL_KERNEL_INV_DIST ? 1 : 0,
                                                    fabs(P->cfg.kernel_c), P->fxe); ++ctx->launches;
    }
    NL_CK(cudaFuncSetAttribute(k_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(sizeof(int32_t) * (NL_HASH_CAP + kListCap))));
    // first count with a set of about 3x the expected row (0.6 x the candidates per triangle);
    // rows that fill it are counted again with the full set.  The first count also leaves every
    // row of fewer than half its set's slots sorted in a buffer row of that size, so that the
    // column write copies those rows instead of building their sets again.
    int hb0 = row_set_bits(P->K > 0 ? 2 * P->E / P->K : 1);
    // NL_ROW_SET_BITS in the environment (6..13) sets the first count's set size instead: a
    // small set sends rows through the second count and the rebuild; the pattern is the same
    if (const char *v = getenv("NL_ROW_SET_BITS")) {
        const int b = atoi(v);
        if (b >= 6 && (1 << b) <= NL_HASH_CAP) hb0 = b;
    }
    const int lb0 = hb0 - 1;
    T->lbits = lb0;
    NL_CK(cudaMallocAsync((void **)&T->buf, sizeof(int32_t) * ((size_t)J << lb0), st));
    NL_CK(cudaMallocAsync((void **)&T->bflag, (size_t)J + 1, st));
    NL_CK(cudaMallocAsync((void **)&T->rlist, sizeof(int) * (J + 1), st));
    NL_CK(cudaMallocAsync((void **)&T->rn, sizeof(int), st));
    NL_CK(cudaMemsetAsync(T->rn, 0, sizeof(int), st));
    k_rows<<<J, kRowThreads, sizeof(int32_t) * ((1u << hb0) + (1u << lb0)), st>>>(
        J, T->nptr, T->ntri, P->tri, P->nbr_ptr, P->nbr_idx, T->sym, hb0, lb0, nullptr, nullptr, T->rcnt, nullptr,
        nullptr, T->olist, T->on, T->ovf, T->buf, T->bflag, T->rlist, T->rn, 0); ++ctx->launches;
    NL_CK(cudaGetLastError());
    const int hbf = row_set_bits(NL_HASH_CAP);
    k_rows<<<256, kRowThreads, sizeof(int32_t) << hbf, st>>>(J, T->nptr, T->ntri, P->tri, P->nbr_ptr, P->nbr_idx,
                                                            T->sym, hbf, 0, T->olist, T->on, T->rcnt, nullptr,
                                                            nullptr, nullptr, nullptr, T->ovf, nullptr, nullptr,
                                                            nullptr, nullptr, 0); ++ctx->launches;
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
    if (h->err & 256) return nl_fail(ctx, NL_EUNSUPPORTED, "a fixed-point sum left its range (error word " +
                                                          std::to_string(h->err) + ")");
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
    // the rows the first count kept sorted are copied; the others (usually none) are built again,
    // and every row has at most max_row columns: a set of 2 max_row slots never fills
    k_row_copy<<<(unsigned)(((int64_t)J * 32 + 255) / 256), 256, 0, st>>>(J, T->bflag, T->buf, T->lbits,
                                                                         out->row_ptr, out->col_idx);
    ++ctx->launches;
    const int hb1 = row_set_bits(2 * P->max_row), lb1 = row_set_bits(P->max_row);
    const size_t smem1 = sizeof(int32_t) * (((size_t)1 << hb1) + ((size_t)1 << lb1));
    const unsigned g1 = J < kRowWaveBlocks ? (unsigned)J : (unsigned)kRowWaveBlocks;
    k_rows<<<g1, kRowThreads, smem1, st>>>(J, T->nptr, T->ntri, P->tri, P->nbr_ptr, P->nbr_idx,
                                                            T->sym, hb1, lb1, T->rlist, T->rn, nullptr, out->row_ptr,
                                                            out->col_idx, nullptr, nullptr, T->ovf, nullptr, nullptr,
                                                            nullptr, nullptr, 1); ++ctx->launches;
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

// Shared-memory plan of the scatter for rows of at most max_row columns: cap per row (a
// multiple of 4), a hash table of 2^hbits >= 1.25 cap slots (the three rows of a triangle's
// nodes share most columns: their union is about 1.15 rows, a load near 0.9 at worst; a
// triangle whose union does not fit searches in global memory), and the warps per block
// that fit 96 KB; cap = 0 (every triangle searches in global memory) when one warp does not
// fit or the rows are too long for the 10-bit positions.
template <typename T>
static void scatter_plan(int64_t max_row, int *cap, int *hbits, int *warps, size_t *smem)
{
    int c = (int)(((max_row > 0 ? max_row : 1) + 3) & ~3LL);
    int hb = 6;
    while ((4 << hb) < 5 * c) hb++;
    int w = 4;
    while (w > 1 && w * scatter_warp_bytes<T>(c, hb) > 96 * 1024) w >>= 1;
    if (max_row > kMaxCachedRow || w * scatter_warp_bytes<T>(c, hb) > 96 * 1024) {
        c = 0;
        hb = 6;
    }
    *cap = c;
    *hbits = hb;
    *warps = w;
    *smem = (size_t)w * scatter_warp_bytes<T>(c, hb);
}

template <typename T>
static nl_status launch_scatter(nl_ctx *ctx, nl_plan *P, nl_csr *out)
{
    const int K = P->K;
    int cap, hbits, warps;
    size_t smem;
    scatter_plan<T>(P->max_row, &cap, &hbits, &warps, &smem);
    NL_CK(cudaFuncSetAttribute(k_scatter<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(96 * 1024)));
    const unsigned grid = (unsigned)((K + warps - 1) / warps);
    k_scatter<T><<<grid, 32 * warps, smem, ctx->stream>>>(K, P->J, P->E, P->tri, P->nbr_ptr, P->nbr_idx, P->flag,
                                                           (const T *)P->blk, out->row_ptr, out->col_idx,
                                                           P->W, P->err, cap, hbits, P->area, P->fxe,
                                                           nl_outer_abs_weight(P)); ++ctx->launches;
    NL_CK(cudaGetLastError());
    k_local_blocks<<<(K + 255) / 256, 256, 0, ctx->stream>>>(K, P->maa, P->mbb, P->lslot, P->W, P->err);
    ++ctx->launches;
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
    int cap, hbits, warps;
    size_t smem;
    scatter_plan<T>(max_row, &cap, &hbits, &warps, &smem);
    if (set_attr)
        NL_CK(cudaFuncSetAttribute(k_scatter_batch<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(96 * 1024)));
    const unsigned grid = (unsigned)((totalK + warps - 1) / warps);
    k_scatter_batch<T><<<grid, 32 * warps, smem, ctx->stream>>>(dS, dkoff, n, cap, hbits); ++ctx->launches;
    NL_CK(cudaGetLastError());
    k_local_blocks_batch<<<(unsigned)((totalK + 255) / 256), 256, 0, ctx->stream>>>(dS, dkoff, n);
    ++ctx->launches;
    NL_CK(cudaGetLastError());
    return NL_OK;
}

nl_status nl_launch_scatter_batch(nl_ctx *ctx, bool f64, const ScatterArgs *dS, const int64_t *dkoff, int n,
                                  int64_t totalK, int64_t max_row, bool set_attr)
{
    return f64 ? launch_scatter_batch<double>(ctx, dS, dkoff, n, totalK, max_row, set_attr)
               : launch_scatter_batch<float>(ctx, dS, dkoff, n, totalK, max_row, set_attr);
}
