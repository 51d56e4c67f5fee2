// internal.cuh -- state and helpers shared by the libnlfem translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "nlfem.h"

#define NL_MAXV 68          // region polygon vertices: 3 + ngon_n (<= 64), or 6 + 3 (cap_m - 1) (<= 51)
#define NL_MAXQ 16          // outer / inner rule points
#define NL_MAXCAND 4096     // candidate neighbours per triangle (sorted in shared memory)
#define NL_HASH_CAP 8192    // per-row column hash set (shared memory) in the symbolic phase

struct nl_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    double last_ms[4] = {0, 0, 0, 0};
    int64_t launches = 0;         // kernels this context has launched (nl_launch_count)
};

// Device-resident state of one assembled problem (held by nl_csr.priv).
struct nl_plan {
    int K = 0, J = 0;
    nl_config cfg{};
    double d2 = 0.0, hmax = 0.0, rmax = 0.0, rin = 0.0;
    // mesh (device)
    int32_t *tri = nullptr;       // [3K]
    double *tx = nullptr, *ty = nullptr;   // [3][K] vertex coordinates per triangle
    double *bx = nullptr, *by = nullptr, *rad = nullptr, *area = nullptr;  // [K]
    double *ngon = nullptr;       // [2 ngon_n]
    std::vector<double> ngon_host; // host copy of the polygon offsets
    // candidates
    int64_t E = 0;
    int64_t *nbr_ptr = nullptr;   // [K+1]
    int32_t *nbr_idx = nullptr;   // [E], per triangle: interior candidates, then boundary ones, each sorted
    int64_t *nbr_split = nullptr; // [K] first boundary candidate of each triangle
    // numeric phase outputs
    uint8_t *flag = nullptr;      // [E] directed: some outer point of a sees a non-empty region in b
    void *blk = nullptr;          // [15][E] pair blocks (float or double)
    double *maa = nullptr;        // [6][K] outer-triangle self block
    int64_t *qp_a = nullptr, *cnt_a = nullptr;   // [K]
    uint64_t *hash_a = nullptr;   // [K]
    // pattern
    int64_t *lslot = nullptr;     // [6][K] slots of the upper local pairs of each triangle
    int64_t *tslot = nullptr;     // [nnz] slot of the transposed entry
    double *W = nullptr;          // [nnz] one-sided accumulation, D = W + W^T
    int64_t max_row = 0;          // longest row of the pattern
    // extracted sub-matrix state (nl_extract)
    float *val32 = nullptr;       // FP32 copy of the values (nl_matvec / nl_cg), lazily built
    int32_t ncols = 0;            // column count of a rectangular result (nl_extract's B)
    int *err = nullptr;           // device error word of the numeric phase and the scatter
    int64_t blk_elems() const { return 15 * E; }
};

// ---- error helpers ----
nl_status nl_fail(nl_ctx *ctx, nl_status s, const std::string &msg);
nl_status nl_cuda_fail(nl_ctx *ctx, cudaError_t e, const char *what);

#define NL_CK(call)                                                       \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return nl_cuda_fail(ctx, e_, #call);       \
    } while (0)

// Device allocation that reports failures as NL_ENOMEM.
template <class T>
inline nl_status nl_alloc(nl_ctx *ctx, T **p, size_t n)
{
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return nl_fail(ctx, NL_ENOMEM, "cudaMalloc of " + std::to_string(n * sizeof(T)) + " bytes failed");
    }
    return NL_OK;
}

template <class T>
inline void nl_free(T *&p)
{
    if (p) cudaFree((void *)p);
    p = nullptr;
}

// ---- device-wide exclusive scan of int64 counts (mesh.cu) ----
// out[i] = sum_{k<i} in[i]; out[n] = total.  in and out may alias.
nl_status nl_scan_i64(nl_ctx *ctx, const int64_t *in, int64_t *out, int64_t n);

// ---- phases ----
nl_status nl_prepare_mesh(nl_ctx *ctx, const nl_mesh *mesh, const nl_config *cfg, nl_plan *P);
nl_status nl_build_candidates(nl_ctx *ctx, nl_plan *P);
nl_status nl_run_numeric(nl_ctx *ctx, nl_plan *P, bool with_hash);
nl_status nl_build_pattern(nl_ctx *ctx, nl_plan *P, nl_csr *out);
nl_status nl_run_scatter(nl_ctx *ctx, nl_plan *P, nl_csr *out);
void nl_plan_free(nl_plan *P);
double nl_polygon_inradius(const double *offsets, int n);

// host pointer / device pointer staging
bool nl_is_device_ptr(const void *p);
nl_status nl_stage(nl_ctx *ctx, const void *src, size_t bytes, void **dev, bool *owned);
