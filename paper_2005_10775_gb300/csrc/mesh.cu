// mesh.cu -- preprocessing of the mesh and cell-list neighbour search.
//
// Per triangle (Sec. 7.1 task 1): vertex coordinates gathered into SoA arrays,
// barycentre ((v0 + v1) + v2) / 3 in round-to-nearest FP64 (the same expression
// the geometry tests use), radius r_k = max |v_i - bary_k|, area, and the longest
// edge (h_max, used by the outer-rule switch of Sec. 8).
//
// Candidate pairs (Sec. 7.1 task 2): T_b is a candidate of T_a iff
// |bary_a - bary_b| <= delta + r_a + r_b (inflated by 1e-9 relative).  This is
// a superset of every pair whose region can be non-empty: a point x of T_a and
// a point y of T_b with |x - y| <= delta lie within r_a and r_b of the
// barycentres.  (The paper's radius delta + h_max is not sufficient for every
// triangle shape; the two-radius bound is.)  Candidates are found with a uniform
// cell list over the barycentres: deterministic buckets (sorted by triangle
// index) and per-triangle candidate lists sorted by triangle index.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <new>

#include "internal.cuh"

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanBlock = kScanThreads * kScanItems;

__global__ void k_scan_block(const int64_t *in, int64_t *out, int64_t *bsum, int64_t n)
{
    __shared__ int64_t wsum[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t tot = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + i;
        v[i] = idx < n ? in[idx] : 0;
        tot += v[i];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = tot;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < (kScanThreads / 32) ? wsum[lane] : 0;
        int64_t s = w;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, s, off);
            if (lane >= off) s += y;
        }
        if (lane < (kScanThreads / 32)) wsum[lane] = s - w;
        if (lane == (kScanThreads / 32) - 1) bsum[blockIdx.x] = s;
    }
    __syncthreads();
    int64_t run = wsum[warp] + (x - tot);
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + i;
        if (idx < n) out[idx] = run;
        run += v[i];
    }
}

__global__ void k_scan_add(int64_t *out, const int64_t *boff, int64_t n)
{
    int64_t idx = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    int64_t add = boff[blockIdx.x];
    for (int i = 0; i < kScanItems; i++, idx += kScanThreads)
        if (idx < n) out[idx] += add;
}

__global__ void k_copy1(int64_t *dst, const int64_t *src) { *dst = *src; }

// ---------------------------------------------------------------------------
// preprocessing
// ---------------------------------------------------------------------------
__global__ void k_prepare(int K, int J, const int32_t *__restrict__ tri, const double *__restrict__ vx,
                          const double *__restrict__ vy, double *tx, double *ty, double *bx, double *by,
                          double *rad, double *area, double *diam, float4 *cf, double kc, float *akc, int *bad)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= K) return;
    int i0 = tri[3 * t], i1 = tri[3 * t + 1], i2 = tri[3 * t + 2];
    if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= J || i1 >= J || i2 >= J) {
        atomicAdd(bad, 1);
        return;
    }
    double x0 = vx[i0], y0 = vy[i0], x1 = vx[i1], y1 = vy[i1], x2 = vx[i2], y2 = vy[i2];
    tx[t] = x0; tx[K + t] = x1; tx[2 * K + t] = x2;
    ty[t] = y0; ty[K + t] = y1; ty[2 * K + t] = y2;
    // barycentre ((v0 + v1) + v2) / 3, round-to-nearest, no contraction
    double cx = __ddiv_rn(__dadd_rn(__dadd_rn(x0, x1), x2), 3.0);
    double cy = __ddiv_rn(__dadd_rn(__dadd_rn(y0, y1), y2), 3.0);
    bx[t] = cx;
    by[t] = cy;
    double r = 0.0;
    const double xs[3] = {x0, x1, x2}, ys[3] = {y0, y1, y2};
    double dmax = 0.0;
    for (int i = 0; i < 3; i++) {
        double dx = xs[i] - cx, dy = ys[i] - cy;
        r = fmax(r, sqrt(dx * dx + dy * dy));
        // longest edge: sqrt(dx*dx + dy*dy) with dx = q - p, exactly rounded
        double ex = __dsub_rn(xs[(i + 1) % 3], xs[i]), ey = __dsub_rn(ys[(i + 1) % 3], ys[i]);
        dmax = fmax(dmax, __dsqrt_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey))));
    }
    rad[t] = r;
    diam[t] = dmax;
    cf[t] = make_float4((float)cx, (float)cy, (float)r, 0.f);   // FP32 copy for the candidate filters
    double cr = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0);
    area[t] = 0.5 * fabs(cr);
    akc[t] = (float)(0.5 * fabs(cr) * kc);
    if (!(cr > 0.0)) atomicAdd(bad, 1);
}

// Every FP64 coordinate v as an FP32 pair hi = fl32(v), lo = fl32(v - hi) (v - hi is exact in
// FP64), so that FP32 differences of nearby points keep their FP64 accuracy: rows 0-2 / 3-5 hold
// hi / lo of the vertices' x, rows 6-8 / 9-11 of their y, rows 12-15 bary x hi, lo, y hi, lo.
__global__ void k_hilo(int K, const double *tx, const double *ty, const double *bx, const double *by, float *hl)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= K) return;
    auto put = [&](int row, double v) {
        const float h = (float)v;
        hl[(int64_t)row * K + t] = h;
        hl[(int64_t)(row + 3) * K + t] = (float)(v - (double)h);
    };
    for (int i = 0; i < 3; i++) {
        put(i, tx[(int64_t)i * K + t]);
        put(6 + i, ty[(int64_t)i * K + t]);
    }
    const double b[2] = {bx[t], by[t]};
    for (int i = 0; i < 2; i++) {
        const float h = (float)b[i];
        hl[(int64_t)(12 + 2 * i) * K + t] = h;
        hl[(int64_t)(13 + 2 * i) * K + t] = (float)(b[i] - (double)h);
    }
}

struct MeshStats {
    double xmin, xmax, ymin, ymax, rmax, hmax;
};

// Order-preserving map of a double to an unsigned key (so that integer atomics take minima
// and maxima) and its inverse.
enum { kStatXmin, kStatYmin, kStatXmax, kStatYmax, kStatRmax, kStatHmax, kStats };
__device__ __forceinline__ unsigned long long stat_key(double d)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    return (u >> 63) ? ~u : (u | (1ull << 63));
}
inline double stat_value(unsigned long long k)
{
    const unsigned long long u = (k >> 63) ? (k & ~(1ull << 63)) : ~k;
    double d;
    memcpy(&d, &u, sizeof d);
    return d;
}

// bounding box of the barycenters, largest barycenter radius and largest diameter; block sums
// in shared memory, one atomic per block and statistic (keys preset: minima ~0, maxima 0)
__global__ void k_mesh_stats(int K, const double *bx, const double *by, const double *rad, const double *diam,
                             unsigned long long *key)
{
    __shared__ double s[kStats][32];
    double v[kStats] = {INFINITY, INFINITY, -INFINITY, -INFINITY, 0.0, 0.0};
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < K; t += gridDim.x * blockDim.x) {
        const double x = bx[t], y = by[t];
        v[kStatXmin] = fmin(v[kStatXmin], x); v[kStatXmax] = fmax(v[kStatXmax], x);
        v[kStatYmin] = fmin(v[kStatYmin], y); v[kStatYmax] = fmax(v[kStatYmax], y);
        v[kStatRmax] = fmax(v[kStatRmax], rad[t]); v[kStatHmax] = fmax(v[kStatHmax], diam[t]);
    }
    for (int off = 16; off; off >>= 1)
        for (int i = 0; i < kStats; i++) {
            const double o = __shfl_xor_sync(0xffffffffu, v[i], off);
            v[i] = i < kStatXmax ? fmin(v[i], o) : fmax(v[i], o);
        }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
        for (int i = 0; i < kStats; i++) s[i][w] = v[i];
    __syncthreads();
    if (threadIdx.x < kStats) {
        const int i = threadIdx.x;
        double r = s[i][0];
        for (int k = 1; k < nw; k++) r = i < kStatXmax ? fmin(r, s[i][k]) : fmax(r, s[i][k]);
        if (i < kStatXmax) atomicMin(&key[i], stat_key(r));
        else atomicMax(&key[i], stat_key(r));
    }
}

// ---------------------------------------------------------------------------
// cell list
// ---------------------------------------------------------------------------
struct Grid {
    double x0, y0, cs;
    int nx, ny, m;  // m: cells searched in each direction
};

__device__ __forceinline__ int cell_of(const Grid &g, double x, double y, int *cx, int *cy)
{
    int ix = (int)floor((x - g.x0) / g.cs), iy = (int)floor((y - g.y0) / g.cs);
    ix = min(max(ix, 0), g.nx - 1);
    iy = min(max(iy, 0), g.ny - 1);
    *cx = ix; *cy = iy;
    return iy * g.nx + ix;
}

__global__ void k_cell_count(int K, Grid g, const double *bx, const double *by, int32_t *cell, int64_t *cnt)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= K) return;
    int cx, cy;
    int c = cell_of(g, bx[t], by[t], &cx, &cy);
    cell[t] = c;
    atomicAdd((unsigned long long *)&cnt[c], 1ull);
}

__global__ void k_cell_fill(int K, const int32_t *cell, const int64_t *start, int64_t *cursor, int32_t *bucket)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= K) return;
    int c = cell[t];
    int64_t pos = start[c] + (int64_t)atomicAdd((unsigned long long *)&cursor[c], 1ull);
    bucket[pos] = t;
}

// sort each bucket by triangle index (rank by counting; buckets are small)
__global__ void k_cell_sort(const int64_t *start, int32_t *bucket, int *overflow)
{
    extern __shared__ int32_t sb[];
    int c = blockIdx.x;
    int64_t s = start[c], n = start[c + 1] - s;
    if (n > NL_MAXCAND) {
        if (threadIdx.x == 0) atomicAdd(overflow, 1);
        return;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) sb[i] = bucket[s + i];
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int v = sb[i], rank = 0;
        for (int k = 0; k < n; k++) rank += sb[k] < v;
        bucket[s + rank] = v;
    }
}

// candidate search, warp per outer triangle; pass 0 counts, pass 1 writes.  The test is
// evaluated in FP32 on a radius inflated by 1e-5 (relative), far above the FP32 rounding of
// the coordinates: a superset of the exact condition, symmetric in (a, b).
__global__ void k_candidates(int K, Grid g, float delta, const float4 *__restrict__ cf,
                             const int64_t *__restrict__ start, const int32_t *__restrict__ bucket,
                             int64_t *cnt, const int64_t *ptr, int32_t *idx, int pass)
{
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= K) return;
    int a = warp;
    const float4 ca = cf[a];
    const float ax = ca.x, ay = ca.y, ra = ca.z;
    int cx, cy;
    cell_of(g, ax, ay, &cx, &cy);
    int64_t n = 0;
    int64_t out = pass ? ptr[a] : 0;
    const int y0 = max(cy - g.m, 0), y1 = min(cy + g.m, g.ny - 1);
    const int x0 = max(cx - g.m, 0), x1 = min(cx + g.m, g.nx - 1);
    // the cells x0..x1 of one row are contiguous in the bucket array: one range per row
    for (int yy = y0; yy <= y1; yy++) {
        const int64_t s = start[yy * g.nx + x0], e = start[yy * g.nx + x1 + 1];
        for (int64_t base = s; base < e; base += 32) {
            const int64_t k = base + lane;
            bool hit = false;
            int b = -1;
            if (k < e) {
                b = bucket[k];
                const float4 cb = cf[b];
                const float ddx = cb.x - ax, ddy = cb.y - ay;
                const float R = (delta + (ra + cb.z)) * (1.0f + 1e-5f);   // symmetric in (a, b)
                hit = ddx * ddx + ddy * ddy <= R * R;
            }
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (pass && hit) idx[out + n + __popc(m & ((1u << lane) - 1u))] = b;
            n += __popc(m);
        }
    }
    if (!pass && lane == 0) cnt[a] = n;
}

// Sort each candidate list by triangle index, interior candidates first.  A candidate is
// interior when every point of T_b lies, with margin, inside the kept region of every outer
// point of T_a (whole for every q):
//   mode 0: |bary_a - bary_b| + r_a + r_b <= lim   (lim = r_in - 2 tau: disc or polygon inradius)
//   mode 1: |bary_a - bary_b| + r_a <= lim         (barycenter ball, lim = delta - 2 tau)
//   mode 2: no interior fast path
//   mode 3: mode 0 and |bary_a - bary_b| - r_a - 3 r_b > far_margin (singular kernel: no near field)
// split[a] = index of the first boundary candidate.  Candidate indices of a mesh numbered
// with any locality span far fewer than kSortBits values: the list is then sorted by setting
// one bit per candidate in an interior and a boundary bitmap and writing the set bits in
// order (prefix counts over the words); a wider span takes a bitonic sort.
constexpr int kSortThreads = 256;
constexpr int kSortWords = 2048;   // 65536 bits per bitmap

__device__ __forceinline__ bool interior_cand(const float4 &ca, const float4 &cb, int mode, float lim,
                                              float far_margin)
{
    if (mode == 2) return false;
    // FP32 with lim already reduced by 1e-5 delta (far above the FP32 rounding): conservative
    const float dx = cb.x - ca.x, dy = cb.y - ca.y;
    const float D = sqrtf(dx * dx + dy * dy);
    bool in = (mode == 1 ? D + ca.z : D + ca.z + cb.z) <= lim;
    // singular kernel: also far from the near field for every outer point
    // (distance >= D - r_a - r_b >= 2 r_b >= diameter of T_b)
    if (mode == 3) in = in && (D - ca.z - 3.0f * cb.z > far_margin);
    return in;
}

__global__ void __launch_bounds__(kSortThreads) k_sort_lists(const int64_t *ptr, int32_t *idx, int64_t *split,
                                                             const float4 *cf, int mode, float lim, float far_margin,
                                                             int *overflow)
{
    __shared__ int32_t s[NL_MAXCAND];
    __shared__ uint32_t bm[2][kSortWords];
    __shared__ int wsum[kSortThreads / 32 + 1];
    __shared__ int s_lo, s_hi, s_int;
    const int a = blockIdx.x;
    const int64_t b0 = ptr[a];
    const int n = (int)(ptr[a + 1] - b0);
    if (n > NL_MAXCAND) {
        if (threadIdx.x == 0) atomicAdd(overflow, 1);
        return;
    }
    if (threadIdx.x == 0) {
        s_lo = 0x7fffffff;
        s_hi = -1;
        s_int = 0;
    }
    const float4 ca = cf[a];
    __syncthreads();
    // classify: interior candidates carry bit 30 clear, boundary ones set
    int lo = 0x7fffffff, hi = -1, my_int = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int b = idx[b0 + i];
        const bool in = interior_cand(ca, cf[b], mode, lim, far_margin);
        my_int += in;
        s[i] = in ? b : (b | 0x40000000);
        lo = min(lo, b);
        hi = max(hi, b);
    }
    for (int off = 16; off; off >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, off));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, off));
        my_int += __shfl_xor_sync(0xffffffffu, my_int, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&s_lo, lo);
        atomicMax(&s_hi, hi);
        atomicAdd(&s_int, my_int);
    }
    __syncthreads();
    lo = s_lo;
    const int span = n > 0 ? s_hi - lo + 1 : 0;
    if (span <= kSortWords * 32) {
        const int nw = (span + 31) >> 5;
        for (int w = threadIdx.x; w < nw; w += blockDim.x) bm[0][w] = bm[1][w] = 0u;
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int key = s[i], o = (key & 0x3fffffff) - lo;
            atomicOr(&bm[key >> 30][o >> 5], 1u << (o & 31));
        }
        __syncthreads();
        // each thread owns a run of consecutive words of both bitmaps
        const int per = (nw + kSortThreads - 1) / kSortThreads;
        const int w0 = min(nw, (int)threadIdx.x * per), w1 = min(nw, w0 + per);
        int c0 = 0, c1 = 0;
        for (int w = w0; w < w1; w++) {
            c0 += __popc(bm[0][w]);
            c1 += __popc(bm[1][w]);
        }
        int t0 = 0, t1 = 0;
        int p0 = nl_block_scan<kSortThreads>(c0, wsum, &t0);
        int p1 = nl_block_scan<kSortThreads>(c1, wsum, &t1) + t0;
        for (int w = w0; w < w1; w++) {
            for (uint32_t m = bm[0][w]; m; m &= m - 1) idx[b0 + p0++] = lo + (w << 5) + __ffs(m) - 1;
            for (uint32_t m = bm[1][w]; m; m &= m - 1) idx[b0 + p1++] = lo + (w << 5) + __ffs(m) - 1;
        }
    } else {
        int p = 1;
        while (p < n) p <<= 1;
        for (int i = n + threadIdx.x; i < p; i += blockDim.x) s[i] = 0x7fffffff;
        __syncthreads();
        for (int k = 2; k <= p; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < p; i += blockDim.x) {
                    const int l = i ^ j;
                    if (l > i) {
                        const bool up = (i & k) == 0;
                        const int u = s[i], v = s[l];
                        if ((u > v) == up) {
                            s[i] = v;
                            s[l] = u;
                        }
                    }
                }
                __syncthreads();
            }
        for (int i = threadIdx.x; i < n; i += blockDim.x) idx[b0 + i] = s[i] & 0x3fffffff;
    }
    if (threadIdx.x == 0) split[a] = b0 + s_int;
}

}  // namespace

nl_status nl_scan_i64(nl_ctx *ctx, const int64_t *in, int64_t *out, int64_t n)
{
    if (n <= 0) {
        NL_CK(cudaMemsetAsync(out, 0, sizeof(int64_t), ctx->stream));
        return NL_OK;
    }
    int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    int64_t *bsum = nullptr;
    NL_CK(cudaMallocAsync((void **)&bsum, sizeof(int64_t) * (nb + 1), ctx->stream));
    k_scan_block<<<(unsigned)nb, kScanThreads, 0, ctx->stream>>>(in, out, bsum, n); ++ctx->launches;
    NL_CK(cudaGetLastError());
    if (nb == 1) {
        k_copy1<<<1, 1, 0, ctx->stream>>>(out + n, bsum); ++ctx->launches;
    } else {
        nl_status s = nl_scan_i64(ctx, bsum, bsum, nb);
        if (s != NL_OK) return s;
        k_scan_add<<<(unsigned)nb, kScanThreads, 0, ctx->stream>>>(out, bsum, n); ++ctx->launches;
        k_copy1<<<1, 1, 0, ctx->stream>>>(out + n, bsum + nb); ++ctx->launches;
    }
    NL_CK(cudaGetLastError());
    NL_CK(cudaFreeAsync(bsum, ctx->stream));
    return NL_OK;
}

double nl_polygon_inradius(const double *o, int N)
{
    // distance from the centre to the nearest edge line of the ccw polygon o_0 .. o_{N-1}
    double rin = INFINITY;
    for (int k = 0; k < N; k++) {
        const int k1 = (k + 1) % N;
        const double ex = o[2 * k1] - o[2 * k], ey = o[2 * k1 + 1] - o[2 * k + 1];
        const double el = sqrt(ex * ex + ey * ey);
        const double dk = (o[2 * k] * o[2 * k1 + 1] - o[2 * k + 1] * o[2 * k1]) / (el > 0.0 ? el : 1.0);
        rin = fmin(rin, dk);
    }
    return rin;
}

struct nl_prep {
    void *dvx = nullptr, *dvy = nullptr, *dtri = nullptr;
    bool own_vx = false, own_vy = false, own_tri = false;
    double *diam = nullptr;
    int *bad = nullptr;
    unsigned long long *st = nullptr;   // k_mesh_stats keys
    float4 *cf = nullptr;
    Grid g{};
    int ncell = 0;
    int32_t *cell = nullptr, *bucket = nullptr;
    int64_t *ccnt = nullptr, *cstart = nullptr, *cursor = nullptr, *cnt = nullptr;
    int *ovf = nullptr;
};

nl_prep *nl_prep_new() { return new (std::nothrow) nl_prep(); }

namespace {
template <class T>
void free_async(T *&p, cudaStream_t s)
{
    if (p) cudaFreeAsync((void *)p, s);
    p = nullptr;
}

void prep_release(nl_prep *T, cudaStream_t s)
{
    void *vx = T->own_vx ? T->dvx : nullptr, *vy = T->own_vy ? T->dvy : nullptr;
    void *tr = T->own_tri ? T->dtri : nullptr;
    free_async(vx, s); free_async(vy, s); free_async(tr, s);
    T->dvx = T->dvy = T->dtri = nullptr;
    T->own_vx = T->own_vy = T->own_tri = false;
    free_async(T->diam, s); free_async(T->bad, s); free_async(T->st, s); free_async(T->cf, s);
    free_async(T->cell, s); free_async(T->bucket, s); free_async(T->ccnt, s); free_async(T->cstart, s);
    free_async(T->cursor, s); free_async(T->cnt, s); free_async(T->ovf, s);
}
}  // namespace

void nl_prep_delete(nl_prep *T, cudaStream_t s)
{
    if (!T) return;
    prep_release(T, s);
    delete T;
}

nl_status nl_prepare_a(nl_ctx *ctx, const nl_mesh *mesh, const nl_config *cfg, nl_plan *P, nl_prep *T,
                       nl_host_slot *h)
{
    const int K = mesh->nt, J = mesh->nv;
    P->stream = ctx->stream;
    P->K = K;
    P->J = J;
    P->cfg = *cfg;
    P->d2 = cfg->delta * cfg->delta;
    nl_status s;
    if ((s = nl_stage(ctx, mesh->vx, sizeof(double) * J, &T->dvx, &T->own_vx)) != NL_OK) return s;
    if ((s = nl_stage(ctx, mesh->vy, sizeof(double) * J, &T->dvy, &T->own_vy)) != NL_OK) return s;
    if ((s = nl_stage(ctx, mesh->tri, sizeof(int32_t) * 3 * K, &T->dtri, &T->own_tri)) != NL_OK) return s;
    if ((s = nl_alloc(ctx, &P->tri, 3 * (size_t)K)) != NL_OK) return s;
    NL_CK(cudaMemcpyAsync(P->tri, T->dtri, sizeof(int32_t) * 3 * K, cudaMemcpyDeviceToDevice, ctx->stream));
    if ((s = nl_alloc(ctx, &P->tx, 3 * (size_t)K)) != NL_OK) return s;
    if ((s = nl_alloc(ctx, &P->ty, 3 * (size_t)K)) != NL_OK) return s;
    if ((s = nl_alloc(ctx, &P->bx, K)) != NL_OK) return s;
    if ((s = nl_alloc(ctx, &P->by, K)) != NL_OK) return s;
    if ((s = nl_alloc(ctx, &P->rad, K)) != NL_OK) return s;
    if ((s = nl_alloc(ctx, &P->area, K)) != NL_OK) return s;
    if ((s = nl_alloc(ctx, &P->akc, K)) != NL_OK) return s;
    if ((s = nl_alloc(ctx, &P->hl, 16 * (size_t)K)) != NL_OK) return s;
    if (cfg->ball == NL_BALL_NGON) {
        const size_t nb = sizeof(double) * 2 * cfg->ngon_n;
        P->ngon_host.resize(2 * (size_t)cfg->ngon_n);
        if ((s = nl_alloc(ctx, &P->ngon, 2 * (size_t)cfg->ngon_n)) != NL_OK) return s;
        if (nl_is_device_ptr(cfg->ngon_offsets)) {
            NL_CK(cudaMemcpyAsync(P->ngon, cfg->ngon_offsets, nb, cudaMemcpyDeviceToDevice, ctx->stream));
            NL_CK(cudaMemcpyAsync(P->ngon_host.data(), cfg->ngon_offsets, nb, cudaMemcpyDeviceToHost, ctx->stream));
            NL_CK(cudaStreamSynchronize(ctx->stream));
        } else {
            memcpy(P->ngon_host.data(), cfg->ngon_offsets, nb);
            NL_CK(cudaMemcpyAsync(P->ngon, P->ngon_host.data(), nb, cudaMemcpyHostToDevice, ctx->stream));
        }
        P->rin = nl_polygon_inradius(P->ngon_host.data(), cfg->ngon_n);
    }
    NL_CK(cudaMallocAsync((void **)&T->diam, sizeof(double) * K, ctx->stream));
    NL_CK(cudaMallocAsync((void **)&T->bad, sizeof(int), ctx->stream));
    NL_CK(cudaMallocAsync((void **)&T->st, sizeof(unsigned long long) * kStats, ctx->stream));
    NL_CK(cudaMemsetAsync(T->st, 0xff, sizeof(unsigned long long) * kStatXmax, ctx->stream));
    NL_CK(cudaMemsetAsync(T->st + kStatXmax, 0, sizeof(unsigned long long) * (kStats - kStatXmax), ctx->stream));
    NL_CK(cudaMemsetAsync(T->bad, 0, sizeof(int), ctx->stream));
    NL_CK(cudaMallocAsync((void **)&T->cf, sizeof(float4) * K, ctx->stream));
    k_prepare<<<(K + 255) / 256, 256, 0, ctx->stream>>>(K, J, (const int32_t *)T->dtri, (const double *)T->dvx,
                                                        (const double *)T->dvy, P->tx, P->ty, P->bx, P->by,
                                                        P->rad, P->area, T->diam, T->cf, cfg->kernel_c, P->akc,
                                                        T->bad); ++ctx->launches;
    k_hilo<<<(K + 255) / 256, 256, 0, ctx->stream>>>(K, P->tx, P->ty, P->bx, P->by, P->hl); ++ctx->launches;
    NL_CK(cudaGetLastError());
    {
        const int nb = (K + 255) / 256;
        k_mesh_stats<<<nb < 608 ? nb : 608, 256, 0, ctx->stream>>>(K, P->bx, P->by, P->rad, T->diam, T->st);
        ++ctx->launches;
    }
    NL_CK(cudaGetLastError());
    static_assert(sizeof(unsigned long long) * kStats == sizeof(h->mesh), "mesh statistics slot");
    NL_CK(cudaMemcpyAsync(h->mesh, T->st, sizeof h->mesh, cudaMemcpyDeviceToHost, ctx->stream));
    NL_CK(cudaMemcpyAsync(&h->bad, T->bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    return NL_OK;
}

nl_status nl_prepare_b(nl_ctx *ctx, nl_plan *P, nl_prep *T, nl_host_slot *h)
{
    const int K = P->K;
    const nl_config *cfg = &P->cfg;
    cudaStream_t st = ctx->stream;
    // the staged inputs and the statistics buffers are no longer needed
    {
        void *vx = T->own_vx ? T->dvx : nullptr, *vy = T->own_vy ? T->dvy : nullptr;
        void *tr = T->own_tri ? T->dtri : nullptr;
        free_async(vx, st); free_async(vy, st); free_async(tr, st);
        T->dvx = T->dvy = T->dtri = nullptr;
        T->own_vx = T->own_vy = T->own_tri = false;
        free_async(T->diam, st); free_async(T->bad, st); free_async(T->st, st);
    }
    MeshStats hst;
    hst.xmin = stat_value(h->mesh[kStatXmin]);
    hst.xmax = stat_value(h->mesh[kStatXmax]);
    hst.ymin = stat_value(h->mesh[kStatYmin]);
    hst.ymax = stat_value(h->mesh[kStatYmax]);
    hst.rmax = stat_value(h->mesh[kStatRmax]);
    hst.hmax = stat_value(h->mesh[kStatHmax]);
    if (h->bad)
        return nl_fail(ctx, NL_EGEOM, std::to_string(h->bad) +
                                          " triangles are degenerate, clockwise or index a missing vertex");
    P->hmax = hst.hmax;
    P->rmax = hst.rmax;
    // grid for the candidate search
    double R = (cfg->delta + 2.0 * hst.rmax) * (1.0 + 2e-5);
    double Lx = hst.xmax - hst.xmin, Ly = hst.ymax - hst.ymin, L = fmax(fmax(Lx, Ly), 1e-300);
    double cs = fmin(R, L / sqrt(fmax(K / 32.0, 1.0)));
    Grid &g = T->g;
    g.cs = cs;
    g.m = (int)ceil(R / cs);
    g.x0 = hst.xmin;
    g.y0 = hst.ymin;
    g.nx = (int)floor(Lx / cs) + 1;
    g.ny = (int)floor(Ly / cs) + 1;
    const int ncell = g.nx * g.ny;
    T->ncell = ncell;
    NL_CK(cudaMallocAsync((void **)&T->cell, sizeof(int32_t) * K, st));
    NL_CK(cudaMallocAsync((void **)&T->bucket, sizeof(int32_t) * K, st));
    NL_CK(cudaMallocAsync((void **)&T->ccnt, sizeof(int64_t) * (ncell + 1), st));
    NL_CK(cudaMallocAsync((void **)&T->cstart, sizeof(int64_t) * (ncell + 1), st));
    NL_CK(cudaMallocAsync((void **)&T->cursor, sizeof(int64_t) * (ncell + 1), st));
    NL_CK(cudaMallocAsync((void **)&T->ovf, sizeof(int), st));
    NL_CK(cudaMemsetAsync(T->ccnt, 0, sizeof(int64_t) * (ncell + 1), st));
    NL_CK(cudaMemsetAsync(T->cursor, 0, sizeof(int64_t) * (ncell + 1), st));
    NL_CK(cudaMemsetAsync(T->ovf, 0, sizeof(int), st));
    k_cell_count<<<(K + 255) / 256, 256, 0, st>>>(K, g, P->bx, P->by, T->cell, T->ccnt); ++ctx->launches;
    NL_CK(cudaGetLastError());
    nl_status s;
    if ((s = nl_scan_i64(ctx, T->ccnt, T->cstart, ncell)) != NL_OK) return s;
    k_cell_fill<<<(K + 255) / 256, 256, 0, st>>>(K, T->cell, T->cstart, T->cursor, T->bucket); ++ctx->launches;
    NL_CK(cudaGetLastError());
    k_cell_sort<<<ncell, 256, sizeof(int32_t) * NL_MAXCAND, st>>>(T->cstart, T->bucket, T->ovf); ++ctx->launches;
    NL_CK(cudaGetLastError());
    // candidate counts and their prefix sum
    if ((s = nl_alloc(ctx, &P->nbr_ptr, (size_t)K + 1)) != NL_OK) return s;
    NL_CK(cudaMallocAsync((void **)&T->cnt, sizeof(int64_t) * K, st));
    const unsigned wblocks = (unsigned)(((int64_t)K * 32 + 255) / 256);
    k_candidates<<<wblocks, 256, 0, st>>>(K, g, (float)cfg->delta, T->cf, T->cstart, T->bucket, T->cnt, nullptr,
                                          nullptr, 0); ++ctx->launches;
    NL_CK(cudaGetLastError());
    if ((s = nl_scan_i64(ctx, T->cnt, P->nbr_ptr, K)) != NL_OK) return s;
    NL_CK(cudaMemcpyAsync(&h->E, P->nbr_ptr + K, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    NL_CK(cudaMemcpyAsync(&h->ovf, T->ovf, sizeof(int), cudaMemcpyDeviceToHost, st));
    return NL_OK;
}

nl_status nl_prepare_c(nl_ctx *ctx, nl_plan *P, nl_prep *T, nl_host_slot *h)
{
    const int K = P->K;
    const nl_config *cfg = &P->cfg;
    cudaStream_t st = ctx->stream;
    if (h->ovf) return nl_fail(ctx, NL_EUNSUPPORTED, "cell-list bucket exceeds the shared-memory sort limit");
    const int64_t E = h->E;
    P->E = E;
    nl_status s;
    if ((s = nl_alloc(ctx, &P->nbr_idx, (size_t)E)) != NL_OK) return s;
    const unsigned wblocks = (unsigned)(((int64_t)K * 32 + 255) / 256);
    k_candidates<<<wblocks, 256, 0, st>>>(K, T->g, (float)cfg->delta, T->cf, T->cstart, T->bucket, nullptr,
                                          P->nbr_ptr, P->nbr_idx, 1); ++ctx->launches;
    NL_CK(cudaGetLastError());
    // interior fast path: the region is whole for every outer point (certified with margin tau)
    {
        const double tau = 1e-5 * cfg->delta;
        int mode = 0;
        double lim = cfg->delta - 2.0 * tau;
        if (cfg->ball == NL_BALL_BARYCENTER || cfg->ball == NL_BALL_BARY_NOCAPS ||
            cfg->ball == NL_BALL_BARY_APPROXCAPS)
            mode = 1;   // whole T_b (and whole support T_a) iff |bary_a - bary_b| + r_a <= delta
        else if (cfg->ball == NL_BALL_NGON) lim = P->rin - 2.0 * tau;
        if (cfg->kernel == NL_KERNEL_INV_DIST) mode = cfg->ball == NL_BALL_BARYCENTER ? 2 : 3;
        if ((s = nl_alloc(ctx, &P->nbr_split, (size_t)K)) != NL_OK) return s;
        k_sort_lists<<<K, kSortThreads, 0, st>>>(P->nbr_ptr, P->nbr_idx, P->nbr_split, T->cf, mode, (float)lim,
                                        (float)(2.0 * tau), T->ovf); ++ctx->launches;
    }
    NL_CK(cudaGetLastError());
    NL_CK(cudaMemcpyAsync(&h->ovf, T->ovf, sizeof(int), cudaMemcpyDeviceToHost, st));
    prep_release(T, st);
    return NL_OK;
}

nl_status nl_prepare_check(nl_ctx *ctx, const nl_host_slot *h)
{
    if (h->ovf) return nl_fail(ctx, NL_EUNSUPPORTED, "a triangle has more than 4096 candidate neighbours");
    return NL_OK;
}

nl_status nl_prepare_mesh(nl_ctx *ctx, const nl_mesh *mesh, const nl_config *cfg, nl_plan *P)
{
    nl_host_slot *h = nullptr;
    nl_status s = nl_host_slots(ctx, 1, &h);
    if (s != NL_OK) return s;
    nl_prep *T = nl_prep_new();
    if (!T) return nl_fail(ctx, NL_ENOMEM, "host allocation failed");
    if ((s = nl_prepare_a(ctx, mesh, cfg, P, T, h)) == NL_OK) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) s = nl_cuda_fail(ctx, e, "cudaStreamSynchronize");
    }
    if (s == NL_OK && (s = nl_prepare_b(ctx, P, T, h)) == NL_OK) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) s = nl_cuda_fail(ctx, e, "cudaStreamSynchronize");
    }
    if (s == NL_OK && (s = nl_prepare_c(ctx, P, T, h)) == NL_OK) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) s = nl_cuda_fail(ctx, e, "cudaStreamSynchronize");
    }
    if (s == NL_OK) s = nl_prepare_check(ctx, h);
    nl_prep_delete(T, ctx->stream);
    return s;
}
