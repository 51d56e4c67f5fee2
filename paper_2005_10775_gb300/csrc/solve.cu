// solve.cu -- from D to the linear system and its solution.
//
//   A = D[Omega, Omega], B = D[Omega, Omega_I]        (Eq. (weakja); rules A-C of Sec. 7.2)
//   F = G - B g,  G_j = int_Omega f phi_j             (Eq. (lfunc3) with u = g on Omega_I, Eq. (appr))
//   A U = F by conjugate gradients (A is symmetric positive definite, Sec. 2; the paper
//   names no solver): FP32 inner iterations (FP32 values, FP32 vectors) inside an FP64
//   residual-refinement loop r = b - A x in FP64 until ||r|| <= rtol ||b||.
// The matrix-vector products are HBM-bound: one warp per row, values and column
// indices streamed once per product.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <new>

#include "internal.cuh"

namespace {

__global__ void k_labels(int J, const uint8_t *lab, int64_t *inO, int64_t *inI)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < J) {
        inO[j] = lab[j] != 0;
        inI[j] = lab[j] == 0;
    }
}

__global__ void k_inverse(int J, const uint8_t *lab, const int64_t *ro, const int64_t *ri, int32_t *omap, int32_t *imap)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= J) return;
    if (lab[j]) omap[ro[j]] = j; else imap[ri[j]] = j;
}

// pass 0: per Omega row, count entries of A (Omega columns) and B (Omega_I columns);
// pass 1: write them renumbered, keeping the column order
__global__ void k_split(int J, const int64_t *rp, const int32_t *col, const double *val, const uint8_t *lab,
                        const int64_t *ro, const int64_t *ri, int64_t *cA, int64_t *cB, const int64_t *rpA,
                        int32_t *colA, double *valA, const int64_t *rpB, int32_t *colB, double *valB, int pass)
{
    int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (j >= J || !lab[j]) return;
    const int64_t r = ro[j];
    int64_t na = 0, nb = 0;
    const int64_t oA = pass ? rpA[r] : 0, oB = pass ? rpB[r] : 0;
    for (int64_t base = rp[j]; base < rp[j + 1]; base += 32) {
        int64_t s = base + lane;
        bool valid = s < rp[j + 1];
        int c = valid ? col[s] : 0;
        bool inO = valid && lab[c];
        bool inI = valid && !lab[c];
        unsigned mO = __ballot_sync(0xffffffffu, inO), mI = __ballot_sync(0xffffffffu, inI);
        unsigned below = (1u << lane) - 1u;
        if (pass) {
            if (inO) {
                int64_t p = oA + na + __popc(mO & below);
                colA[p] = (int32_t)ro[c];
                valA[p] = val[s];
            }
            if (inI) {
                int64_t p = oB + nb + __popc(mI & below);
                colB[p] = (int32_t)ri[c];
                valB[p] = val[s];
            }
        }
        na += __popc(mO);
        nb += __popc(mI);
    }
    if (!pass && lane == 0) {
        cA[r] = na;
        cB[r] = nb;
    }
}

// G_j += |T|/12 (2 f_j + f_k + f_l) over elements of Omega (P1 mass matrix times nodal f)
__global__ void k_load(int K, const int32_t *tri, const double *vx, const double *vy, const uint8_t *elem,
                       const double *f, double *G)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= K || !elem[t]) return;
    int i0 = tri[3 * t], i1 = tri[3 * t + 1], i2 = tri[3 * t + 2];
    double ar = 0.5 * fabs((vx[i1] - vx[i0]) * (vy[i2] - vy[i0]) - (vx[i2] - vx[i0]) * (vy[i1] - vy[i0]));
    double f0 = f[i0], f1 = f[i1], f2 = f[i2];
    atomicAdd(&G[i0], ar * (2.0 * f0 + f1 + f2) / 12.0);
    atomicAdd(&G[i1], ar * (f0 + 2.0 * f1 + f2) / 12.0);
    atomicAdd(&G[i2], ar * (f0 + f1 + 2.0 * f2) / 12.0);
}

__global__ void k_gather(int n, const int32_t *map, const double *src, double *dst)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[map[i]];
}

// F[r] = G[omap[r]] - (B gI)[r]; warp per row
__global__ void k_rhs(int n, const int64_t *rp, const int32_t *col, const double *val, const double *gI,
                      const int32_t *omap, const double *G, double *F)
{
    int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (r >= n) return;
    double s = 0.0;
    for (int64_t k = rp[r] + lane; k < rp[r + 1]; k += 32) s += val[k] * gI[col[k]];
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) F[r] = G[omap[r]] - s;
}

__global__ void k_to_f32(int64_t n, const double *a, float *b)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

// this lane's part of row [b, e) of A times x: lane l takes entries l, l + 32, ... (each load
// instruction of the warp reads 32 consecutive entries, and the gathers of x touch the few
// cache lines of 32 consecutive columns), four entries a lane in flight before their gathers
template <typename TV, typename TX>
__device__ __forceinline__ TV row_dot(const TV *__restrict__ val, const int32_t *__restrict__ col,
                                      const TX *__restrict__ x, int64_t b, int64_t e, int lane)
{
    TV s = 0;
    for (int64_t k0 = b + lane; k0 < e; k0 += 128) {
        TV v[4];
        int c[4];
        for (int u = 0; u < 4; u++) {
            const int64_t k = k0 + 32 * u;
            v[u] = k < e ? val[k] : (TV)0;
            c[u] = k < e ? col[k] : -1;
        }
        for (int u = 0; u < 4; u++)
            if (c[u] >= 0) s += v[u] * (TV)x[c[u]];
    }
    return s;
}

// y = A x, warp per row (TV: value type, TX: vector type, accumulation in TV)
template <typename TV, typename TX, typename TY>
__global__ void k_spmv(int n, const int64_t *rp, const int32_t *__restrict__ col, const TV *__restrict__ val,
                       const TX *__restrict__ x, TY *y)
{
    int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (r >= n) return;
    TV s = row_dot<TV, TX>(val, col, x, rp[r], rp[r + 1], lane);
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) y[r] = (TY)s;
}

// r = b - A x (FP64) and ||r||^2, ||b||^2 accumulated into acc[0], acc[1]
// sum of v over the block's warps (lane 0 of each warp holds its warp's v), added to *dst by
// one atomic per block: one address taking an atomic per row would serialise the launch
__device__ __forceinline__ void block_atomic_add(double v, double *dst)
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

__global__ void k_residual(int n, const int64_t *rp, const int32_t *__restrict__ col, const double *__restrict__ val,
                           const double *__restrict__ x, const double *b, double *r, double *acc)
{
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    double rr = 0.0, bb = 0.0;
    if (row < n) {
        double s = row_dot<double, double>(val, col, x, rp[row], rp[row + 1], lane);
        for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        const double v = b[row] - s;
        if (lane == 0) r[row] = v;
        rr = v * v;
        bb = b[row] * b[row];
    }
    block_atomic_add(rr, &acc[0]);
    block_atomic_add(bb, &acc[1]);
}

// inner FP32 conjugate gradients on A d = z0 (z0 = r / ||r||)
struct CgScal {
    double rho, pq, zz;
    int brk;   // breakdown: p.Ap not positive (or not a number) while the residual is not yet zero
};

// a direction with p.Ap <= 0 (A not positive definite along p) or a non-finite p.Ap ends the
// solve; below rho = 1e-20 (the inner residual 1e-10 of its start) the iteration has converged
// and the host stops it
constexpr double kBreakdownRho = 1e-20;

__global__ void k_cg_init(int n, const double *r, double inv_norm, float *z, float *p, float *d, CgScal *sc)
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

// q = A p and p.q
__global__ void k_cg_spmv(int n, const int64_t *rp, const int32_t *__restrict__ col, const float *__restrict__ val,
                          const float *__restrict__ p, float *q, CgScal *sc)
{
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    double pq = 0.0;
    if (r < n) {
        float s = row_dot<float, float>(val, col, p, rp[r], rp[r + 1], lane);
        for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) q[r] = s;
        pq = (double)s * (double)p[r];
    }
    block_atomic_add(pq, &sc->pq);
}

__global__ void k_cg_update(int n, const float *p, const float *q, float *d, float *z, CgScal *sc)
{
    __shared__ double part[8];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double pq = sc->pq;
    const bool brk = sc->rho > kBreakdownRho && !(pq > 0.0);
    float alpha = (pq > 0.0) ? (float)(sc->rho / pq) : 0.0f;
    if (i == 0 && brk) sc->brk = 1;
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

__global__ void k_cg_dir(int n, const float *z, float *p, const CgScal *sc)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float beta = sc->rho != 0.0 ? (float)(sc->zz / sc->rho) : 0.0f;
    if (i < n) p[i] = z[i] + beta * p[i];
}

__global__ void k_cg_shift(CgScal *sc)
{
    sc->rho = sc->zz;
    sc->pq = 0.0;
    sc->zz = 0.0;
}

__global__ void k_axpy_f32(int n, double s, const float *d, double *x)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += s * (double)d[i];
}

nl_plan *plan_of(nl_csr *m)
{
    if (!m->priv) m->priv = new (std::nothrow) nl_plan();
    return (nl_plan *)m->priv;
}

nl_status ensure_f32(nl_ctx *ctx, nl_csr *A)
{
    nl_plan *P = plan_of(A);
    if (!P) return nl_fail(ctx, NL_ENOMEM, "host allocation failed");
    if (P->val32) return NL_OK;
    nl_status s = nl_alloc(ctx, &P->val32, (size_t)A->nnz);
    if (s != NL_OK) return s;
    if (A->nnz) {
        k_to_f32<<<(unsigned)((A->nnz + 255) / 256), 256, 0, ctx->stream>>>(A->nnz, A->val, P->val32); ++ctx->launches;
    }
    NL_CK(cudaGetLastError());
    return NL_OK;
}

unsigned wgrid(int64_t rows) { return (unsigned)((rows * 32 + 255) / 256); }

// A CUDA graph of a fixed sequence of kernel launches on one stream, captured once and replayed
// (released with its holder).  A capture the runtime refuses (the stream already capturing, a
// launch error) leaves `failed` set and the caller launches the kernels itself.
struct ChunkGraph {
    cudaGraphExec_t exec = nullptr;
    bool failed = false;
    template <class Launches>
    void capture(cudaStream_t st, Launches launches)
    {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            failed = true;
            return;
        }
        launches();
        const cudaError_t e = cudaStreamEndCapture(st, &g);
        if (e == cudaSuccess && g && cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) exec = nullptr;
        if (g) cudaGraphDestroy(g);
        if (!exec) {
            cudaGetLastError();
            failed = true;
        }
    }
    ~ChunkGraph()
    {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

nl_status extract_body(nl_ctx *ctx, const nl_csr *D, const nl_mesh *mesh, nl_csr *A, nl_csr *B)
{
    nl_temps tmp(ctx->stream);
    const int J = D->n;
    nl_status s;
    void *lab = nullptr;
    bool own = false;
    if ((s = nl_stage(ctx, mesh->node_in_omega, (size_t)J, &lab, &own)) != NL_OK) return s;
    if (own) tmp.adopt(lab);
    int64_t *inO, *inI, *ro, *ri, *cA, *cB;
    if ((s = tmp.get(ctx, &inO, (size_t)J + 1)) != NL_OK) return s;
    if ((s = tmp.get(ctx, &inI, (size_t)J + 1)) != NL_OK) return s;
    if ((s = tmp.get(ctx, &ro, (size_t)J + 1)) != NL_OK) return s;
    if ((s = tmp.get(ctx, &ri, (size_t)J + 1)) != NL_OK) return s;
    k_labels<<<(J + 255) / 256, 256, 0, ctx->stream>>>(J, (const uint8_t *)lab, inO, inI); ++ctx->launches;
    if ((s = nl_scan_i64(ctx, inO, ro, J)) != NL_OK) return s;
    if ((s = nl_scan_i64(ctx, inI, ri, J)) != NL_OK) return s;
    int64_t nO = 0, nI = 0;
    NL_CK(cudaMemcpyAsync(&nO, ro + J, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    NL_CK(cudaMemcpyAsync(&nI, ri + J, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    NL_CK(cudaStreamSynchronize(ctx->stream));
    if ((s = tmp.get(ctx, &cA, (size_t)nO + 1)) != NL_OK) return s;
    if ((s = tmp.get(ctx, &cB, (size_t)nO + 1)) != NL_OK) return s;
    k_split<<<wgrid(J), 256, 0, ctx->stream>>>(J, D->row_ptr, D->col_idx, D->val, (const uint8_t *)lab, ro, ri, cA,
                                               cB, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0); ++ctx->launches;
    NL_CK(cudaGetLastError());
    if ((s = nl_alloc(ctx, &A->row_ptr, (size_t)nO + 1)) != NL_OK) return s;
    if ((s = nl_alloc(ctx, &B->row_ptr, (size_t)nO + 1)) != NL_OK) return s;
    if ((s = nl_scan_i64(ctx, cA, A->row_ptr, nO)) != NL_OK) return s;
    if ((s = nl_scan_i64(ctx, cB, B->row_ptr, nO)) != NL_OK) return s;
    int64_t nzA = 0, nzB = 0;
    NL_CK(cudaMemcpyAsync(&nzA, A->row_ptr + nO, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    NL_CK(cudaMemcpyAsync(&nzB, B->row_ptr + nO, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    NL_CK(cudaStreamSynchronize(ctx->stream));
    A->n = B->n = (int32_t)nO;
    A->nnz = nzA;
    B->nnz = nzB;
    if ((s = nl_alloc(ctx, &A->col_idx, (size_t)nzA)) != NL_OK) return s;
    if ((s = nl_alloc(ctx, &A->val, (size_t)nzA)) != NL_OK) return s;
    if ((s = nl_alloc(ctx, &B->col_idx, (size_t)nzB)) != NL_OK) return s;
    if ((s = nl_alloc(ctx, &B->val, (size_t)nzB)) != NL_OK) return s;
    k_split<<<wgrid(J), 256, 0, ctx->stream>>>(J, D->row_ptr, D->col_idx, D->val, (const uint8_t *)lab, ro, ri,
                                               nullptr, nullptr, A->row_ptr, A->col_idx, A->val, B->row_ptr,
                                               B->col_idx, B->val, 1); ++ctx->launches;
    NL_CK(cudaGetLastError());
    nl_plan *PB = plan_of(B);
    if (!PB) return nl_fail(ctx, NL_ENOMEM, "host allocation failed");
    PB->ncols = (int32_t)nI;
    NL_CK(cudaStreamSynchronize(ctx->stream));
    return NL_OK;
}

}  // namespace

extern "C" {

nl_status nl_extract(nl_ctx *ctx, const nl_csr *D, const nl_mesh *mesh, nl_csr *A, nl_csr *B)
{
    if (!ctx) return NL_EINVAL;
    if (!D || !mesh || !A || !B || !mesh->node_in_omega) return nl_fail(ctx, NL_EINVAL, "null argument");
    if (mesh->nv != D->n) return nl_fail(ctx, NL_EINVAL, "mesh and matrix sizes differ");
    memset(A, 0, sizeof *A);
    memset(B, 0, sizeof *B);
    const nl_status s = extract_body(ctx, D, mesh, A, B);
    if (s != NL_OK) {   // no partial results
        nl_csr_free(ctx, A);
        nl_csr_free(ctx, B);
    }
    return s;
}


nl_status nl_rhs(nl_ctx *ctx, const nl_csr *B, const nl_mesh *mesh, const double *f_nodal, const double *g_nodal,
                 double *F)
{
    if (!ctx) return NL_EINVAL;
    if (!B || !mesh || !f_nodal || !g_nodal || !F || !mesh->node_in_omega || !mesh->elem_in_omega)
        return nl_fail(ctx, NL_EINVAL, "null argument (nl_rhs needs both node and element labels)");
    const int J = mesh->nv, K = mesh->nt;
    nl_status s;
    nl_temps tmp(ctx->stream);   // released on every return path
    void *lab, *elem, *vx, *vy, *tri, *f, *g;
    bool o1, o2, o3, o4, o5, o6, o7;
    if ((s = nl_stage(ctx, mesh->node_in_omega, (size_t)J, &lab, &o1)) != NL_OK) return s;
    if ((s = nl_stage(ctx, mesh->elem_in_omega, (size_t)K, &elem, &o2)) != NL_OK) return s;
    if ((s = nl_stage(ctx, mesh->vx, sizeof(double) * J, &vx, &o3)) != NL_OK) return s;
    if ((s = nl_stage(ctx, mesh->vy, sizeof(double) * J, &vy, &o4)) != NL_OK) return s;
    if ((s = nl_stage(ctx, mesh->tri, sizeof(int32_t) * 3 * K, &tri, &o5)) != NL_OK) return s;
    if ((s = nl_stage(ctx, f_nodal, sizeof(double) * J, &f, &o6)) != NL_OK) return s;
    if ((s = nl_stage(ctx, g_nodal, sizeof(double) * J, &g, &o7)) != NL_OK) return s;
    {
        void *st[] = {lab, elem, vx, vy, tri, f, g};
        bool own[] = {o1, o2, o3, o4, o5, o6, o7};
        for (int i = 0; i < 7; i++)
            if (own[i]) tmp.adopt(st[i]);
    }
    int64_t *inO, *inI, *ro, *ri;
    int32_t *omap, *imap;
    double *G, *gI, *Fd;
    if ((s = tmp.get(ctx, &inO, (size_t)J + 1)) != NL_OK) return s;
    if ((s = tmp.get(ctx, &inI, (size_t)J + 1)) != NL_OK) return s;
    if ((s = tmp.get(ctx, &ro, (size_t)J + 1)) != NL_OK) return s;
    if ((s = tmp.get(ctx, &ri, (size_t)J + 1)) != NL_OK) return s;
    if ((s = tmp.get(ctx, &omap, (size_t)J + 1)) != NL_OK) return s;
    if ((s = tmp.get(ctx, &imap, (size_t)J + 1)) != NL_OK) return s;
    if ((s = tmp.get(ctx, &G, (size_t)J)) != NL_OK) return s;
    if ((s = tmp.get(ctx, &gI, (size_t)J + 1)) != NL_OK) return s;
    NL_CK(cudaMemsetAsync(G, 0, sizeof(double) * J, ctx->stream));
    k_labels<<<(J + 255) / 256, 256, 0, ctx->stream>>>(J, (const uint8_t *)lab, inO, inI); ++ctx->launches;
    if ((s = nl_scan_i64(ctx, inO, ro, J)) != NL_OK) return s;
    if ((s = nl_scan_i64(ctx, inI, ri, J)) != NL_OK) return s;
    k_inverse<<<(J + 255) / 256, 256, 0, ctx->stream>>>(J, (const uint8_t *)lab, ro, ri, omap, imap); ++ctx->launches;
    k_load<<<(K + 255) / 256, 256, 0, ctx->stream>>>(K, (const int32_t *)tri, (const double *)vx, (const double *)vy,
                                                     (const uint8_t *)elem, (const double *)f, G); ++ctx->launches;
    int64_t nO = 0, nI = 0;
    NL_CK(cudaMemcpyAsync(&nO, ro + J, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    NL_CK(cudaMemcpyAsync(&nI, ri + J, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    NL_CK(cudaStreamSynchronize(ctx->stream));
    if (nO != B->n) return nl_fail(ctx, NL_EINVAL, "B does not match the mesh labels");
    k_gather<<<(unsigned)((nI + 255) / 256 + 1), 256, 0, ctx->stream>>>((int)nI, imap, (const double *)g, gI); ++ctx->launches;
    const int fk = nl_ptr_kind(F, ctx->device);
    if (fk == NL_PTR_OTHER) return nl_fail(ctx, NL_EINVAL, "F lives on another device than the context's");
    const bool dev_out = fk == NL_PTR_DEVICE;
    if (dev_out) Fd = F;
    else if ((s = tmp.get(ctx, &Fd, (size_t)nO + 1)) != NL_OK) return s;
    k_rhs<<<wgrid(nO), 256, 0, ctx->stream>>>((int)nO, B->row_ptr, B->col_idx, B->val, gI, omap, G, Fd); ++ctx->launches;
    NL_CK(cudaGetLastError());
    if (!dev_out) NL_CK(cudaMemcpyAsync(F, Fd, sizeof(double) * nO, cudaMemcpyDeviceToHost, ctx->stream));
    NL_CK(cudaStreamSynchronize(ctx->stream));
    return NL_OK;
}

nl_status nl_matvec(nl_ctx *ctx, const nl_csr *Ac, const double *x, double *y, int32_t prec)
{
    if (!ctx) return NL_EINVAL;
    if (!Ac || !x || !y) return nl_fail(ctx, NL_EINVAL, "null argument");
    nl_csr *A = const_cast<nl_csr *>(Ac);
    const int n = A->n;
    int ncols = n;
    if (A->priv && ((nl_plan *)A->priv)->ncols) ncols = ((nl_plan *)A->priv)->ncols;
    nl_status s;
    nl_temps tmp(ctx->stream);   // host operands only: none with device x and y (stream-ordered call)
    void *xd;
    bool ox;
    if ((s = nl_stage(ctx, x, sizeof(double) * ncols, &xd, &ox)) != NL_OK) return s;
    if (ox) tmp.adopt(xd);
    const int yk = nl_ptr_kind(y, ctx->device);
    if (yk == NL_PTR_OTHER) return nl_fail(ctx, NL_EINVAL, "y lives on another device than the context's");
    const bool dev_out = yk == NL_PTR_DEVICE;
    double *yd = y;
    if (!dev_out && (s = tmp.get(ctx, &yd, (size_t)n + 1)) != NL_OK) return s;
    if (prec == NL_PREC_FP64) {
        k_spmv<double, double, double><<<wgrid(n), 256, 0, ctx->stream>>>(n, A->row_ptr, A->col_idx, A->val,
                                                                           (const double *)xd, yd);
        ++ctx->launches;
    } else {
        if ((s = ensure_f32(ctx, A)) != NL_OK) return s;
        nl_plan *P = (nl_plan *)A->priv;
        // x rounded to FP32 once (the products use FP32 operands either way): no FP64
        // conversion per stored entry
        if (!P->x32 && (s = nl_alloc(ctx, &P->x32, (size_t)ncols)) != NL_OK) return s;
        if (ncols > 0) {
            k_to_f32<<<(unsigned)((ncols + 255) / 256), 256, 0, ctx->stream>>>(ncols, (const double *)xd, P->x32);
            ++ctx->launches;
        }
        k_spmv<float, float, double><<<wgrid(n), 256, 0, ctx->stream>>>(n, A->row_ptr, A->col_idx, P->val32,
                                                                         P->x32, yd);
        ++ctx->launches;
    }
    NL_CK(cudaGetLastError());
    if (!dev_out) NL_CK(cudaMemcpyAsync(y, yd, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    // host buffers: the copies must be complete when the call returns; device buffers: stream-ordered
    if (!dev_out || ox) NL_CK(cudaStreamSynchronize(ctx->stream));
    return NL_OK;
}

nl_status nl_cg(nl_ctx *ctx, const nl_csr *Ac, const double *b, double *x, double rtol, int32_t max_it,
                int32_t *iters, double *relres)
{
    if (!ctx) return NL_EINVAL;
    if (iters) *iters = 0;
    if (relres) *relres = INFINITY;
    if (!Ac || !b || !x) return nl_fail(ctx, NL_EINVAL, "null argument");
    if (!(rtol > 0.0) || max_it < 1) return nl_fail(ctx, NL_EINVAL, "need rtol > 0 and max_it >= 1");
    nl_csr *A = const_cast<nl_csr *>(Ac);
    const int n = A->n;
    nl_status s;
    // every temporary below is released on every return path (stream-ordered)
    nl_temps tmp(ctx->stream);
    if ((s = ensure_f32(ctx, A)) != NL_OK) return s;
    const float *v32 = ((nl_plan *)A->priv)->val32;
    void *bd;
    bool ob;
    if ((s = nl_stage(ctx, b, sizeof(double) * n, &bd, &ob)) != NL_OK) return s;
    if (ob) tmp.adopt(bd);
    const int xk = nl_ptr_kind(x, ctx->device);
    if (xk == NL_PTR_OTHER) return nl_fail(ctx, NL_EINVAL, "x lives on another device than the context's");
    const bool dev_x = xk == NL_PTR_DEVICE;
    double *xd = x;
    if (!dev_x) {
        if ((s = tmp.get(ctx, &xd, (size_t)n + 1)) != NL_OK) return s;
        NL_CK(cudaMemcpyAsync(xd, x, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
    }
    double *r, *acc;
    float *z, *p, *q, *d;
    CgScal *sc;
    if ((s = tmp.get(ctx, &r, (size_t)n + 1)) != NL_OK || (s = tmp.get(ctx, &acc, 2)) != NL_OK ||
        (s = tmp.get(ctx, &z, (size_t)n + 1)) != NL_OK || (s = tmp.get(ctx, &p, (size_t)n + 1)) != NL_OK ||
        (s = tmp.get(ctx, &q, (size_t)n + 1)) != NL_OK || (s = tmp.get(ctx, &d, (size_t)n + 1)) != NL_OK ||
        (s = tmp.get(ctx, &sc, 1)) != NL_OK)
        return s;
    const unsigned eg = (unsigned)((n + 255) / 256);
    int total = 0;
    double rel = INFINITY;
    bool conv = false, stop = false;
    nl_status out = NL_OK;
    const int kCheck = 8;          // inner iterations between host convergence checks
    const double kInnerTol = 1e-5; // inner relative reduction per refinement step
    const int kPasses = 64;        // FP64 refinement passes
    ChunkGraph graph;              // the captured inner chunk (released with the call)
    for (int outer = 0; outer < kPasses && !stop; outer++) {
        NL_CK(cudaMemsetAsync(acc, 0, sizeof(double) * 2, ctx->stream));
        k_residual<<<wgrid(n), 256, 0, ctx->stream>>>(n, A->row_ptr, A->col_idx, A->val, xd, (const double *)bd, r,
                                                      acc); ++ctx->launches;
        double h[2];
        NL_CK(cudaMemcpyAsync(h, acc, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
        NL_CK(cudaStreamSynchronize(ctx->stream));
        double rn = sqrt(h[0]), bn = sqrt(h[1]);
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
        k_cg_init<<<eg, 256, 0, ctx->stream>>>(n, r, 1.0 / rn, z, p, d, sc); ++ctx->launches;
        while (total < max_it) {
            const int chunk = (max_it - total) < kCheck ? (max_it - total) : kCheck;
            auto iterate = [&](int count) {
                for (int c = 0; c < count; c++) {
                    k_cg_spmv<<<wgrid(n), 256, 0, ctx->stream>>>(n, A->row_ptr, A->col_idx, v32, p, q, sc);
                    k_cg_update<<<eg, 256, 0, ctx->stream>>>(n, p, q, d, z, sc);
                    k_cg_dir<<<eg, 256, 0, ctx->stream>>>(n, z, p, sc);
                    k_cg_shift<<<1, 1, 0, ctx->stream>>>(sc);
                }
                ctx->launches += 4 * count;
            };
            // a full chunk is one launch of a graph of its 4 x kCheck kernels (captured at the first
            // full chunk of the call: its buffers are the call's own), which removes most of the
            // launch gaps between these short kernels; a capture that fails falls back to launches
            if (chunk == kCheck && !graph.exec && !graph.failed) {
                const int64_t l0 = ctx->launches;   // captured, not launched
                graph.capture(ctx->stream, [&] { iterate(kCheck); });
                ctx->launches = l0;
            }
            if (chunk == kCheck && graph.exec) {
                NL_CK(cudaGraphLaunch(graph.exec, ctx->stream));
                ctx->launches += 4 * kCheck;
            } else {
                iterate(chunk);
            }
            NL_CK(cudaGetLastError());
            total += chunk;
            CgScal hs;
            NL_CK(cudaMemcpyAsync(&hs, sc, sizeof hs, cudaMemcpyDeviceToHost, ctx->stream));
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
        k_axpy_f32<<<eg, 256, 0, ctx->stream>>>(n, rn, d, xd); ++ctx->launches;
        NL_CK(cudaGetLastError());
    }
    if (out == NL_OK && !conv)
        out = nl_fail(ctx, NL_ENOCONV, "CG did not reach the tolerance within " + std::to_string(kPasses) +
                                           " FP64 refinement passes (is rtol above the FP64 residual floor?)");
    if (!dev_x) NL_CK(cudaMemcpyAsync(x, xd, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    NL_CK(cudaStreamSynchronize(ctx->stream));
    if (iters) *iters = total;
    if (relres) *relres = rel;
    return out;
}

}  // extern "C"
