// internal.cuh -- state and helpers shared by the libnlfem translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <stdlib.h>
#include <string>
#include <vector>

#include "nlfem.h"

#define NL_MAXV 68          // region polygon vertices: 3 + ngon_n (<= 64), or 6 + 3 (cap_m - 1) (<= 51)
#define NL_MAXQ 16          // outer / inner rule points
#define NL_MAXCAND 4096     // candidate neighbours per triangle (sorted in shared memory)
#define NL_HASH_CAP 8192    // per-row column hash set (shared memory) in the symbolic phase

// exclusive prefix sum of v over a block of NT threads (a multiple of 32, at most 1024);
// *total = the sum.  wsum: NT / 32 + 1 ints of shared memory.  Every thread of the block calls it.
template <int NT>
__device__ __forceinline__ int nl_block_scan(int v, int *wsum, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int w = lane < NT / 32 ? wsum[lane] : 0;
        int t = w;
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, off);
            if (lane >= off) t += y;
        }
        if (lane < NT / 32) wsum[lane] = t - w;
        if (lane == NT / 32 - 1) wsum[NT / 32] = t;
    }
    __syncthreads();
    const int r = wsum[warp] + x - v;
    *total = wsum[NT / 32];
    __syncthreads();
    return r;
}

// Small results of the device phases that the host needs (sizes, statistics, error
// words).  The phases copy them, stream-ordered, into pinned slots owned by the
// context; the host reads a slot only after synchronising the stream, so a batch of
// problems needs one synchronisation per phase instead of one per problem.
struct nl_host_slot {
    unsigned long long mesh[6];   // order-preserving keys: xmin, ymin, xmax, ymax, r_max, h_max
    int64_t E;                    // candidate pairs
    int64_t nnz;                  // pattern entries
    unsigned long long pat[4];    // pairs, qp-pairs, interactions, longest row
    int bad;                      // degenerate / clockwise / out-of-range triangles
    int ovf;                      // cell-list or candidate-list overflow
    int row_ovf;                  // pattern row overflow
    int err;                      // numeric-phase error word
    int deferred;                 // FP32 path: items the FP64 geometry decided
    int near;                     // FP32 path, singular kernel: near-field items queued for k_near
};

struct nl_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    double last_ms[4] = {0, 0, 0, 0};
    int64_t launches = 0;         // kernels this context has launched (nl_launch_count)
    nl_host_slot *slots = nullptr;  // pinned
    int nslots = 0;
    struct nl_tune_cache *tune = nullptr;   // batch schedules picked by the autotuner (batch.cu)
    int64_t last_fp64_items = 0;  // nl_last_fp64_items
    // side streams of a batch's preparation and symbolic stages (created on first use) and
    // their ordering events: [k] for side stream k, [kSideStreams] for the fork
    static constexpr int kSideStreams = 8;
    cudaStream_t side[kSideStreams] = {};
    cudaEvent_t side_ev[kSideStreams + 1] = {};
};

// the context's side streams and their events (created on first use)
nl_status nl_side_streams(nl_ctx *ctx);

// pinned host slots for n problems (grown on demand; invalidates earlier slot pointers)
nl_status nl_host_slots(nl_ctx *ctx, int n, nl_host_slot **out);

// Device-resident state of one assembled problem (held by nl_csr.priv).
struct nl_plan {
    cudaStream_t stream = nullptr;   // stream the buffers were allocated on (freed stream-ordered)
    int K = 0, J = 0;
    nl_config cfg{};
    double d2 = 0.0, hmax = 0.0, rmax = 0.0, rin = 0.0;
    // mesh (device)
    int32_t *tri = nullptr;       // [3K]
    double *tx = nullptr, *ty = nullptr;   // [3][K] vertex coordinates per triangle
    double *bx = nullptr, *by = nullptr, *rad = nullptr, *area = nullptr;  // [K]
    float *akc = nullptr;         // [K] |T| times the kernel constant, rounded to FP32
    float *hl = nullptr;          // [16][K] vertex coordinates and barycentre as FP32 hi + lo pairs
    double *ngon = nullptr;       // [2 ngon_n]
    std::vector<double> ngon_host; // host copy of the polygon offsets
    // candidates
    int64_t E = 0;
    int64_t *nbr_ptr = nullptr;   // [K+1]
    int32_t *nbr_idx = nullptr;   // [E], per triangle: interior candidates, then boundary ones, each sorted
    int64_t *nbr_split = nullptr; // [K] first boundary candidate of each triangle
    // numeric phase outputs
    uint8_t *flag = nullptr;      // [E] directed: some outer point of a sees a non-empty region in b
    void *blk = nullptr;          // [9][E] pair blocks M_ab (float or double)
    double *maa = nullptr;        // [6][K] outer-triangle self block
    int64_t *qp_a = nullptr, *cnt_a = nullptr;   // [K]
    uint64_t *hash_a = nullptr;   // [K]
    // pattern
    int64_t *lslot = nullptr;     // [6][K] slots of the upper local pairs of each triangle
    double *mbb = nullptr;        // [6][K] per-triangle sum of the pairs' upper M_bb (numeric phase; zeroed by it)
    int64_t *tslot = nullptr;     // [nnz] slot of the transposed entry
    double *W = nullptr;          // [nnz] one-sided accumulation, D = W + W^T
    int64_t max_row = 0;          // longest row of the pattern
    int *fxe = nullptr;           // FP32 plans: 128 + e with every scatter column bound per unit of
                                  // |T_a| sum_q |w_q| below 2^(e+1) (k_node_exp)
    // extracted sub-matrix state (nl_extract)
    float *val32 = nullptr;       // FP32 copy of the values (nl_matvec / nl_cg), lazily built
    float *x32 = nullptr;         // [ncols] nl_matvec's x rounded to FP32
    int32_t ncols = 0;            // column count of a rectangular result (nl_extract's B)
    int *err = nullptr;           // device error word of the numeric phase and the scatter
    // FP32 path: queue of the items the FP64 geometry decides (nlq::DeferItem), allocated at
    // the first numeric run, and its fill count
    void *defer = nullptr;
    int *defer_n = nullptr;
    int defer_cap = 0;
    int defer_min = 0;            // capacity the next allocation takes at least (a run overflowed)
    // FP32 path of the singular kernel: queue of the near-field whole items (nlq::DeferItem)
    // that k_near integrates, and its fill count
    void *nearq = nullptr;
    int *near_n = nullptr;
    int near_cap = 0;
    int near_min = 0;             // capacity the next allocation takes at least (a run overflowed)
    void *otab = nullptr;         // [K][outer points] nlq::OuterPt staged by the boundary kernel for k_near
};

// capacity of the near-field queue of the singular kernel's FP32 path for E candidate pairs:
// about 27 near-field triangles per outer point on the benchmark meshes, 16 outer points, some
// 330 candidates per triangle (1.3 E items); a full queue sends the excess to the boundary
// kernel's own lanes.  NL_NEAR_CAP in the environment sets it (0: no queue, all inline).
// is the capacity of the near-field queue set by NL_NEAR_CAP (fixed, for tests)?
inline bool nl_near_cap_fixed()
{
    const char *v = getenv("NL_NEAR_CAP");
    return v && *v;
}

inline int nl_near_cap(int64_t E)
{
    const char *v = getenv("NL_NEAR_CAP");
    if (v && *v) {
        const long long c = strtoll(v, nullptr, 10);
        return c < 0 ? 0 : (int)(c > (1ll << 30) ? (1ll << 30) : c);
    }
    // NL_NEAR_CAP_INIT: the first capacity only (a full queue still grows, for tests)
    const char *w = getenv("NL_NEAR_CAP_INIT");
    if (w && *w) {
        const long long c = strtoll(w, nullptr, 10);
        return c < 1 ? 1 : (int)(c > (1ll << 30) ? (1ll << 30) : c);
    }
    int64_t c = 2 * E;
    if (c < 4096) c = 4096;
    if (c > (int64_t(1) << 30)) c = int64_t(1) << 30;
    return (int)c;
}

// ---- error helpers ----
nl_status nl_fail(nl_ctx *ctx, nl_status s, const std::string &msg);
nl_status nl_cuda_fail(nl_ctx *ctx, cudaError_t e, const char *what);

#define NL_CK(call)                                                       \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return nl_cuda_fail(ctx, e_, #call);       \
    } while (0)

// capacity of a deferred-item queue for E candidate pairs: the FP64 items are a small
// fraction of the exact items on jittered meshes (about 0.1 %), but rules with outer points on
// the triangles' vertices and edges (the paper's 7-point rule) put x_q on vertices of its
// neighbours, whose orientations FP32 cannot certify (1.35 M items for E = 10 M on the
// uniform Table 1 grid h = 0.0125); a full queue sends the excess back to the boundary
// kernel's own lanes (and nl_assemble to a second numeric run with a larger queue)
// is the capacity of the deferred-item queue set by NL_DEFER_CAP (fixed, for tests)?
inline bool nl_defer_cap_fixed()
{
    const char *v = getenv("NL_DEFER_CAP");
    return v && *v;
}

inline int nl_defer_cap(int64_t E)
{
    // NL_DEFER_CAP in the environment sets the capacity (0: no queue, every such item inline)
    const char *v = getenv("NL_DEFER_CAP");
    if (v && *v) {
        const long long c = strtoll(v, nullptr, 10);
        return c < 0 ? 0 : (int)(c > (1ll << 24) ? (1ll << 24) : c);
    }
    // NL_DEFER_CAP_INIT: the first capacity only (a full queue still grows, for tests)
    const char *w = getenv("NL_DEFER_CAP_INIT");
    if (w && *w) {
        const long long c = strtoll(w, nullptr, 10);
        return c < 1 ? 1 : (int)(c > (1ll << 24) ? (1ll << 24) : c);
    }
    int64_t c = E / 4;
    if (c < 4096) c = 4096;
    if (c > (int64_t(1) << 24)) c = int64_t(1) << 24;
    return (int)c;
}

// Device allocation from the device's stream-ordered pool, on the context's stream
// (no device synchronisation); failures are reported as NL_ENOMEM.
template <class T>
inline nl_status nl_alloc(nl_ctx *ctx, T **p, size_t n)
{
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMallocAsync((void **)p, n * sizeof(T), ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return nl_fail(ctx, NL_ENOMEM, "device allocation of " + std::to_string(n * sizeof(T)) + " bytes failed");
    }
    return NL_OK;
}

// stream-ordered release of an nl_alloc buffer
template <class T>
inline void nl_free(T *&p, cudaStream_t s)
{
    if (p) cudaFreeAsync((void *)p, s);
    p = nullptr;
}

// ---- device-wide exclusive scan of int64 counts (mesh.cu) ----
// out[i] = sum_{k<i} in[i]; out[n] = total.  in and out may alias.
nl_status nl_scan_i64(nl_ctx *ctx, const int64_t *in, int64_t *out, int64_t n);

// argument checks of one problem (api.cu)
nl_status nl_validate(nl_ctx *ctx, const nl_mesh *m, const nl_config *c);

// ---- phases ----
// The preparation and the symbolic phase are split into stages that only enqueue
// work on ctx->stream and stream-ordered copies into a host slot; the caller
// synchronises the stream between two stages (once for a whole batch).
struct nl_prep;   // temporaries between the preparation stages (mesh.cu)
nl_prep *nl_prep_new();
void nl_prep_delete(nl_prep *T, cudaStream_t s);
// A: inputs, per-triangle data, mesh statistics -> slot
nl_status nl_prepare_a(nl_ctx *ctx, const nl_mesh *mesh, const nl_config *cfg, nl_plan *P, nl_prep *T,
                       nl_host_slot *h);
// B (slot A read): validation, cell list, candidate counts -> slot
nl_status nl_prepare_b(nl_ctx *ctx, nl_plan *P, nl_prep *T, nl_host_slot *h);
// C (slot B read): candidate lists, interior/boundary split; overflow -> slot (checked by nl_prepare_check)
nl_status nl_prepare_c(nl_ctx *ctx, nl_plan *P, nl_prep *T, nl_host_slot *h);
nl_status nl_prepare_check(nl_ctx *ctx, const nl_host_slot *h);
// all stages with a synchronisation between them
nl_status nl_prepare_mesh(nl_ctx *ctx, const nl_mesh *mesh, const nl_config *cfg, nl_plan *P);

struct nl_pat;    // temporaries between the symbolic stages (pattern.cu)
nl_pat *nl_pat_new();
void nl_pat_delete(nl_pat *T, cudaStream_t s);
// A (after the numeric phase): symmetric flags, row counts, row pointers; nnz and statistics -> slot
nl_status nl_pattern_a(nl_ctx *ctx, nl_plan *P, nl_csr *out, nl_pat *T, nl_host_slot *h);
// B (slot A read): column indices, slot maps, value buffers
nl_status nl_pattern_b(nl_ctx *ctx, nl_plan *P, nl_csr *out, nl_pat *T, const nl_host_slot *h);

nl_status nl_alloc_numeric(nl_ctx *ctx, nl_plan *P);
// numeric phase of one assembled problem with every kernel on ctx->stream (api.cu): the first
// call allocates the problem's FP64-item and near-field queues
nl_status nl_run_numeric_one_stream(nl_ctx *ctx, nl_plan *P);
nl_status nl_run_scatter(nl_ctx *ctx, nl_plan *P, nl_csr *out);
// sum_q |w_q| of the outer rule (the larger of the switching rule's two; api.cu): the FP32
// scatter's bound on a row sum per unit of |T_a|
float nl_outer_abs_weight(const nl_plan *P);
// the steps of nl_assemble after the preparation's stage B (api.cu): C = stage C, numeric phase,
// symbolic stage A (slot: queue counts, pattern size); D (slot C read) = checks, a second numeric
// run if a queue overflowed, symbolic stage B, scatter.  Events (may be null) mark the phases.
nl_status nl_assemble_step_c(nl_ctx *ctx, nl_plan *P, nl_prep *T, nl_pat *Q, nl_host_slot *h, nl_csr *out,
                             bool one_stream, cudaEvent_t ev_num, cudaEvent_t ev_sym);
nl_status nl_assemble_step_d(nl_ctx *ctx, nl_plan *P, nl_pat *Q, const nl_host_slot *h, nl_csr *out,
                             bool one_stream, cudaEvent_t ev_sct);

// ---- batched scatter (pattern.cu): the scatter of every problem of a batch ----
struct ScatterArgs {   // one problem
    int K, J;
    int64_t E;
    const int32_t *tri;
    const int64_t *ptr;
    const int32_t *idx;
    const uint8_t *flag;
    const void *blk;
    const double *maa;
    double *mbb;
    const int64_t *lslot, *row_ptr;
    const int32_t *col;
    double *W;
    const int64_t *tslot;
    double *val;
    int *err;
    const double *area;   // [K] |T_a| (the FP32 scatter's fixed-point grids)
    const int *fxe;       // nl_plan::fxe
    float ws;             // nl_outer_abs_weight
};
// W = 0 over all problems (zoff: prefix sums of nnz, device, n + 1 entries; total = zoff[n])
nl_status nl_launch_zero_batch(nl_ctx *ctx, const ScatterArgs *dS, const int64_t *dzoff, int n, int64_t total);
// scatter of the problems in dS (all of one value type; koff: prefix sums of K; max_row: longest row)
nl_status nl_launch_scatter_batch(nl_ctx *ctx, bool f64, const ScatterArgs *dS, const int64_t *dkoff, int n,
                                  int64_t totalK, int64_t max_row, bool set_attr);
// val = W + W^T over all problems
nl_status nl_launch_symmetrize_batch(nl_ctx *ctx, const ScatterArgs *dS, const int64_t *dzoff, int n,
                                     int64_t total);
// the autotuner's cache of batch schedules (batch.cu)
void nl_tune_cache_free(struct nl_tune_cache *c);
void nl_plan_free(nl_plan *P, cudaStream_t s);   // stream-ordered release of the plan's buffers
double nl_polygon_inradius(const double *offsets, int n);

// host pointer / device pointer staging
bool nl_is_device_ptr(const void *p);
// where p lives, seen from the context's device: host memory, device memory the context's
// kernels may read (its own device's, or managed), or another device's memory (rejected:
// the kernels would dereference it as a peer pointer)
enum { NL_PTR_HOST = 0, NL_PTR_DEVICE = 1, NL_PTR_OTHER = 2 };
int nl_ptr_kind(const void *p, int device);
// device view of a host-or-device input; *owned: the call staged a copy it must free.
// NL_EINVAL for memory of another device.
nl_status nl_stage(nl_ctx *ctx, const void *src, size_t bytes, void **dev, bool *owned);

// Stream-ordered temporaries of one call: every buffer taken with get() (or handed over with
// adopt()) is released with cudaFreeAsync on the context's stream when the holder goes out of
// scope, so that no return path, early error returns included, leaks one.
struct nl_temps {
    cudaStream_t s;
    std::vector<void *> p;
    explicit nl_temps(cudaStream_t st) : s(st) {}
    nl_temps(const nl_temps &) = delete;
    nl_temps &operator=(const nl_temps &) = delete;
    ~nl_temps()
    {
        for (void *q : p)
            if (q) cudaFreeAsync(q, s);
    }
    template <class T>
    nl_status get(nl_ctx *ctx, T **out, size_t n)
    {
        nl_status st = nl_alloc(ctx, out, n);
        if (st == NL_OK) p.push_back((void *)*out);
        return st;
    }
    void adopt(void *q)
    {
        if (q) p.push_back(q);
    }
};
