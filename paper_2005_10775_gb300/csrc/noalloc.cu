// noalloc.cu -- nl_cg_noalloc: the conjugate-gradient solve of nl_cg without any
// device allocation.
//
// Some callers cannot call cudaMalloc: a framework that has handed all device
// memory to its own caching allocator or a pre-reserved arena and forbids
// allocations outside it, or a latency-critical loop that cannot afford the
// implicit synchronisation and the failure modes of an allocation on every call.
// For them this entry point keeps its work vectors in one file-scope device array
// of fixed size (kScratchBytes below, about 6 MB), which every GPU that loads the
// library holds until the process exits.  The caller passes the matrix, the
// right-hand side and the solution vector in device memory.
//
// Set-up: the first call on a device looks up the array's device address with
// cudaGetSymbolAddress (that device current) and caches it; make that first call
// before any stream capture.  Every call shares the one array and leaves its
// contents behind: everything that must start at zero is cleared by the call's own
// kernels.  Calls whose work overlaps on the GPU (two streams, two host threads)
// race on the array and must be serialised by the caller.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "internal.cuh"

namespace {

constexpr int64_t kMaxN = int64_t(1) << 18;   // largest system this entry point accepts
constexpr size_t kScratchBytes = size_t(kMaxN) * sizeof(double)       // r
                               + 4 * size_t(kMaxN) * sizeof(float)     // z, p, q, d
                               + 256;                                   // scalars

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct NaScal {
    double rho, pq, zz, rr, bb;
    int brk;   // breakdown: p.Ap not positive (or not a number) while the residual is not yet zero
};

// below rho = 1e-20 the inner iteration has converged (the host stops it); above it a
// direction with p.Ap <= 0 or a non-finite p.Ap ends the solve
constexpr double kBreakdownRho = 1e-20;

struct NaView {
    double *r;
    float *z, *p, *q, *d;
    NaScal *sc;
};

NaView carve(void *base)
{
    unsigned char *b = (unsigned char *)base;
    NaView v;
    v.r = (double *)b;
    b += size_t(kMaxN) * sizeof(double);
    v.z = (float *)b;
    b += size_t(kMaxN) * sizeof(float);
    v.p = (float *)b;
    b += size_t(kMaxN) * sizeof(float);
    v.q = (float *)b;
    b += size_t(kMaxN) * sizeof(float);
    v.d = (float *)b;
    b += size_t(kMaxN) * sizeof(float);
    v.sc = (NaScal *)b;
    return v;
}

std::mutex g_mu;
constexpr int kMaxDevices = 64;
void *g_addr[kMaxDevices] = {};

// the array's device address on ctx's device, looked up once per device
nl_status scratch_address(nl_ctx *ctx, void **out)
{
    if (ctx->device < 0 || ctx->device >= kMaxDevices) return nl_fail(ctx, NL_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[ctx->device]) {
        NL_CK(cudaSetDevice(ctx->device));
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return nl_fail(ctx, NL_ECUDA, std::string("cudaGetSymbolAddress of the no-allocation scratch: ") +
                                              cudaGetErrorString(e));
        }
        g_addr[ctx->device] = p;
    }
    *out = g_addr[ctx->device];
    return NL_OK;
}

__global__ void k_na_clear(NaScal *sc)
{
    sc->rho = 0.0;
    sc->pq = 0.0;
    sc->zz = 0.0;
    sc->rr = 0.0;
    sc->bb = 0.0;
    sc->brk = 0;
}

// sum of v over the block's warps (lane 0 of each warp holds its warp's v), added to *dst by
// one atomic per block (an atomic per row on one address would serialise the launch)
__device__ __forceinline__ void na_block_add(double v, double *dst)
{
    __shared__ double part[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) part[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += part[i];
        atomicAdd(dst, t);
    }
    __syncthreads();
}

// r = b - A x in FP64, with ||r||^2 and ||b||^2; warp per row
__global__ void k_na_residual(int n, const int64_t *rp, const int32_t *col, const double *val, const double *x,
                              const double *b, double *r, NaScal *sc)
{
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    double rr = 0.0, bb = 0.0;
    if (row < n) {
        double s = 0.0;
        for (int64_t k = rp[row] + lane; k < rp[row + 1]; k += 32) s += val[k] * x[col[k]];
        for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        const double v = b[row] - s;
        if (lane == 0) r[row] = v;
        rr = v * v;
        bb = b[row] * b[row];
    }
    na_block_add(rr, &sc->rr);
    na_block_add(bb, &sc->bb);
}

__global__ void k_na_init(int n, const double *r, double inv_norm, float *z, float *p, float *d, NaScal *sc)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        float v = (float)(r[i] * inv_norm);
        z[i] = v;
        p[i] = v;
        d[i] = 0.0f;
    }
    if (i == 0) {
        sc->rho = 1.0;
        sc->pq = 0.0;
        sc->zz = 0.0;
        sc->brk = 0;
    }
}

// q = A p with the values rounded to FP32 as they are read, and p.q
__global__ void k_na_spmv(int n, const int64_t *rp, const int32_t *col, const double *val, const float *p, float *q,
                          NaScal *sc)
{
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    double pq = 0.0;
    if (r < n) {
        float s = 0.0f;
        for (int64_t k = rp[r] + lane; k < rp[r + 1]; k += 32) s += (float)val[k] * p[col[k]];
        for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) q[r] = s;
        pq = (double)s * (double)p[r];
    }
    na_block_add(pq, &sc->pq);
}

__global__ void k_na_update(int n, const float *p, const float *q, float *d, float *z, NaScal *sc)
{
    __shared__ double part[8];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double pq = sc->pq;
    float alpha = (pq > 0.0) ? (float)(sc->rho / pq) : 0.0f;
    if (i == 0 && sc->rho > kBreakdownRho && !(pq > 0.0)) sc->brk = 1;
    double zz = 0.0;
    if (i < n) {
        d[i] += alpha * p[i];
        float zn = z[i] - alpha * q[i];
        z[i] = zn;
        zz = (double)zn * zn;
    }
    for (int off = 16; off; off >>= 1) zz += __shfl_xor_sync(0xffffffffu, zz, off);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = zz;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += part[w];
        atomicAdd(&sc->zz, t);
    }
}

__global__ void k_na_dir(int n, const float *z, float *p, const NaScal *sc)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float beta = sc->rho != 0.0 ? (float)(sc->zz / sc->rho) : 0.0f;
    if (i < n) p[i] = z[i] + beta * p[i];
}

__global__ void k_na_shift(NaScal *sc)
{
    sc->rho = sc->zz;
    sc->pq = 0.0;
    sc->zz = 0.0;
}

__global__ void k_na_axpy(int n, double s, const float *d, double *x)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += s * (double)d[i];
}

}  // namespace

extern "C" nl_status nl_cg_noalloc(nl_ctx *ctx, const nl_csr *A, const double *b, double *x, double rtol,
                                   int32_t max_it, int32_t *iters, double *relres)
{
    if (!ctx) return NL_EINVAL;
    if (iters) *iters = 0;
    if (relres) *relres = INFINITY;
    if (!A || !b || !x) return nl_fail(ctx, NL_EINVAL, "null argument");
    if (!(rtol > 0.0) || max_it < 1) return nl_fail(ctx, NL_EINVAL, "need rtol > 0 and max_it >= 1");
    if (A->n < 0 || (int64_t)A->n > kMaxN)
        return nl_fail(ctx, NL_EUNSUPPORTED, "nl_cg_noalloc accepts at most " + std::to_string(kMaxN) +
                                                 " unknowns (got " + std::to_string(A->n) + "); use nl_cg");
    const int n = A->n;
    auto on_dev = [&](const void *p) { return nl_ptr_kind(p, ctx->device) == NL_PTR_DEVICE; };
    if (n > 0 && (!on_dev(b) || !on_dev(x) || !on_dev(A->row_ptr) ||
                  (A->nnz > 0 && (!on_dev(A->col_idx) || !on_dev(A->val)))))
        return nl_fail(ctx, NL_EINVAL, "nl_cg_noalloc needs device pointers on the context's device for the "
                                       "matrix, b and x");
    void *base = nullptr;
    nl_status s = scratch_address(ctx, &base);
    if (s != NL_OK) return s;
    NL_CK(cudaSetDevice(ctx->device));
    NaView v = carve(base);
    const unsigned rows = (unsigned)(((int64_t)n * 32 + 255) / 256), eg = (unsigned)((n + 255) / 256);
    const int kCheck = 8;
    const double kInnerTol = 1e-5;
    const int kPasses = 64;   // FP64 refinement passes
    int total = 0;
    double rel = INFINITY;
    bool conv = false, stop = false;
    nl_status out = NL_OK;
    for (int outer = 0; outer < kPasses && !stop; outer++) {
        k_na_clear<<<1, 1, 0, ctx->stream>>>(v.sc); ++ctx->launches;
        if (n > 0) {
            k_na_residual<<<rows, 256, 0, ctx->stream>>>(n, A->row_ptr, A->col_idx, A->val, x, b, v.r, v.sc);
            ++ctx->launches;
        }
        NaScal h;
        NL_CK(cudaMemcpyAsync(&h, v.sc, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
        NL_CK(cudaStreamSynchronize(ctx->stream));
        double rn = sqrt(h.rr), bn = sqrt(h.bb);
        rel = bn > 0.0 ? rn / bn : rn;
        if (!isfinite(rel)) {
            out = nl_fail(ctx, NL_EINVAL, "non-finite residual: A, b or the initial x holds a NaN or an Inf");
            break;
        }
        if (rel <= rtol || rn == 0.0) {
            conv = true;
            break;
        }
        if (total >= max_it) {
            out = nl_fail(ctx, NL_ENOCONV, "CG did not reach the tolerance within max_it iterations");
            break;
        }
        k_na_init<<<eg, 256, 0, ctx->stream>>>(n, v.r, 1.0 / rn, v.z, v.p, v.d, v.sc); ++ctx->launches;
        while (total < max_it) {
            const int chunk = (max_it - total) < kCheck ? (max_it - total) : kCheck;
            for (int c = 0; c < chunk; c++) {
                k_na_spmv<<<rows, 256, 0, ctx->stream>>>(n, A->row_ptr, A->col_idx, A->val, v.p, v.q, v.sc);
                k_na_update<<<eg, 256, 0, ctx->stream>>>(n, v.p, v.q, v.d, v.z, v.sc);
                k_na_dir<<<eg, 256, 0, ctx->stream>>>(n, v.z, v.p, v.sc);
                k_na_shift<<<1, 1, 0, ctx->stream>>>(v.sc);
                ctx->launches += 4;
            }
            NL_CK(cudaGetLastError());
            total += chunk;
            NaScal hs;
            NL_CK(cudaMemcpyAsync(&hs, v.sc, sizeof hs, cudaMemcpyDeviceToHost, ctx->stream));
            NL_CK(cudaStreamSynchronize(ctx->stream));
            if (hs.brk || !isfinite(hs.rho)) {   // breakdown: the correction d is not usable
                out = nl_fail(ctx, NL_ENOCONV, "CG breakdown: a search direction with p.Ap <= 0 or not a number "
                                               "(A not symmetric positive definite, or non-finite values)");
                stop = true;
                break;
            }
            if (!(sqrt(hs.rho) > kInnerTol)) break;   // inner tolerance reached
        }
        if (stop) break;
        k_na_axpy<<<eg, 256, 0, ctx->stream>>>(n, rn, v.d, x); ++ctx->launches;
        NL_CK(cudaGetLastError());
    }
    if (out == NL_OK && !conv)
        out = nl_fail(ctx, NL_ENOCONV, "CG did not reach the tolerance within " + std::to_string(kPasses) +
                                           " FP64 refinement passes (is rtol above the FP64 residual floor?)");
    NL_CK(cudaStreamSynchronize(ctx->stream));
    if (iters) *iters = total;
    if (relres) *relres = rel;
    return out;
}
