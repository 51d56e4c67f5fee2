/*
 * nlfem.h -- C ABI of libnlfem: GB300 (sm_103a) assembly of the P1 stiffness
 * matrix of the nonlocal diffusion operator with ball-supported kernels, after
 * D'Elia, Gunzburger, Vollmann, "A cookbook for finite element methods for
 * nonlocal problems, including quadrature rules and approximate Euclidean balls".
 *
 * Problem (Sec. 1.1, Eq. (prob), (oper), (inter)):
 *     -L u = f on Omega,  u = g on Omega_I,
 *     L u(x) = 2 int (u(y) - u(x)) gamma(x, y) dy,  gamma = psi(x, y) 1_{B_delta(x)}(y).
 * The library assembles the full (Omega u Omega_I)^2 matrix D of the bilinear form
 * Eq. (bform0) discretised as Eq. (bformhj) with the quadrature of Eq. (bformjqqh);
 * A = D[Omega, Omega] and F = G - D[Omega, Omega_I] g follow from the A-B-C
 * assignment table of Sec. 7.2.
 *
 * Conventions shared by every entry point:
 *   - Every call returns nl_status; nothing aborts, traps or exits.  On failure
 *     nl_last_error(ctx) returns a one-line description (valid until the next call).
 *   - Input pointers may be host or device memory (detected per pointer; device memory
 *     must be the context's device's, else NL_EINVAL); the caller keeps ownership and may
 *     free them when the call returns.
 *   - Outputs in nl_csr are device buffers owned by the library, released with
 *     nl_csr_free.  Work is ordered on the context's CUDA stream.
 *   - Indices are 0-based; triangles are counter-clockwise.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef NLFEM_H
#define NLFEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NL_OK = 0,
    NL_EINVAL = 1,        /* bad argument (null pointer, size, enum value) */
    NL_ENOMEM = 2,        /* device allocation failed */
    NL_ECUDA = 3,         /* a CUDA runtime call failed */
    NL_EGEOM = 4,         /* degenerate or clockwise triangle, or an index past the vertex array */
    NL_ETIMEOUT = 5,      /* a bounded device-side wait expired */
    NL_ENOCONV = 6,       /* the iterative solver did not reach the tolerance */
    NL_EUNSUPPORTED = 7   /* valid but not implemented combination / size limit exceeded */
} nl_status;

/* Interaction region R(x, T_b) kept by the (approximate) ball centred at the outer point x. */
typedef enum {
    NL_BALL_BARYCENTER = 0,   /* whole T_b iff |x - bary(T_b)| <= delta           (Sec. 4.2.3, Eq. (baryball)) */
    NL_BALL_NOCAPS = 1,       /* chord polygon of T_b n B_delta(x), fanned         (Sec. 4.2.1, Sec. 7.1 tasks 3-6) */
    NL_BALL_APPROXCAPS = 2,   /* nocaps plus cap_m - 1 arc points per cap         (Sec. 4.2.2) */
    NL_BALL_EXACTCAPS = 3,    /* nocaps plus a one-point centroid rule per cap    (Sec. 5.2, Eq. (areacap)) */
    NL_BALL_NGON = 4,         /* T_b clipped by the regular inscribed ngon_n-gon  (Sec. 9, regular polygon) */
    NL_BALL_OVERLAP = 5,      /* whole T_b iff T_b n B_delta(x) is non-empty      (Sec. 4.2.4, Eq. (overlap)) */
    /* barycenter ball for the inner integral, with the outer integral over T_a restricted to its
       support T_a n B_delta(bary_b), approximated by nocaps / approxcaps (cap_m) of that ball around
       bary_b and integrated with the outer rule on each fan subtriangle (Sec. 6.2, barycenter case;
       Table 3).  One interaction record per pair (q = 0, the support's kind and vertex count);
       qp-pairs = outer points x inner points.  CONST kernel, not shifted. */
    NL_BALL_BARY_NOCAPS = 6,
    NL_BALL_BARY_APPROXCAPS = 7
} nl_ball;

/* Quadrature rules on triangles (weights relative to the area). */
typedef enum {
    NL_RULE_GAUSS3 = 0,       /* 3-point symmetric Gaussian, degree 2 (Sec. 5.3.1) */
    NL_RULE_GAUSS4 = 1,       /* 4-point symmetric Gaussian, degree 3 (Sec. 6.1) */
    NL_RULE_PAPER7 = 2,       /* centroid/vertices/mid-sides 27/60, 3/60, 8/60, degree 3 (Sec. 6.3) */
    NL_RULE_DUNAVANT7 = 3,    /* 7-point degree-5 rule (Radon) */
    NL_RULE_DUNAVANT16 = 4,   /* 16-point degree-8 rule (Dunavant) */
    NL_RULE_SWITCH47 = 5      /* outer only: GAUSS4 if |bary_a - bary_b| < delta - h_max else PAPER7 (Sec. 8) */
} nl_rule;

typedef enum {
    NL_KERNEL_CONST = 0,      /* psi = kernel_c                                   (Sec. 8) */
    NL_KERNEL_INV_DIST = 1    /* psi = kernel_c / |x - y| (integrable singular kernel, Sec. 2 remarks) */
} nl_kernel;

typedef enum {
    NL_PREC_FP64 = 0,         /* geometry and quadrature in FP64 */
    NL_PREC_FP32_COMP = 1     /* geometry in FP64; quadrature in FP32 with FP64 (compensated) long sums */
} nl_prec;

typedef struct nl_ctx nl_ctx;

/* Triangle mesh of Omega u Omega_I (Sec. 3.1).  node_in_omega: 1 for nodes in the open
   Omega, 0 for nodes of Omega_I including those on the boundary of Omega (Sec. 3.1).
   elem_in_omega: 1 for elements of the triangulation of Omega.  Both labels are only
   read by nl_extract / nl_rhs and may be NULL for nl_assemble. */
typedef struct {
    int32_t nv, nt;
    const double *vx, *vy;          /* [nv] vertex coordinates */
    const int32_t *tri;             /* [3*nt] counter-clockwise vertex indices */
    const uint8_t *node_in_omega;   /* [nv] or NULL */
    const uint8_t *elem_in_omega;   /* [nt] or NULL */
} nl_mesh;

typedef struct {
    double delta;                   /* horizon > 0; any size relative to the triangles (Sec. 8 runs delta = h,
                                       and delta below the largest diameter on grid (b)) */
    double kernel_c;                /* kernel constant c */
    int32_t kernel;                 /* nl_kernel */
    int32_t ball;                   /* nl_ball */
    int32_t ngon_n;                 /* NGON: number of polygon vertices, 3..64 */
    int32_t cap_m;                  /* APPROXCAPS: sub-arcs per cap, power of two 1..16 */
    const double *ngon_offsets;     /* NGON: [2*ngon_n] polygon vertices relative to x, ccw */
    int32_t outer, inner;           /* nl_rule of the outer (T_a) and inner (subtriangle) integrals */
    int32_t prec;                   /* nl_prec */
    int32_t duffy_n;                /* INV_DIST: Gauss points per unit panel of the near-singular rule (1..7) */
    int32_t cap_printed;            /* EXACTCAPS: 1 = cap weight as printed in Sec. 5.2 (half Eq. (areacap)) */
    int32_t shifted;                /* 1 = shifted-centre ball (Sec. 4.3): every outer point of T_a uses the
                                       ball centred at T_a's barycentre ((v0 + v1) + v2) / 3, approximated
                                       by `ball`; CONST kernel only (NL_EUNSUPPORTED otherwise) */
} nl_config;

/* Square CSR matrix in device memory, columns sorted in each row. */
typedef struct {
    int32_t n;
    int64_t nnz;
    int64_t *row_ptr;               /* [n+1] */
    int32_t *col_idx;               /* [nnz] */
    double *val;                    /* [nnz] */
    int64_t n_pairs;                /* element pairs (T_a, T_b) with a non-empty region for some outer point */
    int64_t n_qp_pairs;             /* (outer point, inner point) evaluations performed */
    int64_t n_inter;                /* (T_a, q, T_b) triples with a non-empty region */
    void *priv;                     /* library state (pattern, candidate lists); do not touch */
} nl_csr;

/* Create a context on CUDA device `device`, ordering work on `cuda_stream`
   (a cudaStream_t; NULL = a stream created and owned by the context). */
nl_status nl_create(nl_ctx **ctx, int device, void *cuda_stream);
void nl_destroy(nl_ctx *ctx);
const char *nl_last_error(nl_ctx *ctx);

/* Assemble D = sum over all element pairs (T_a, T_b) of Eq. (bformhj) with the outer
   rule on T_a and the inner rule on every subtriangle of R(x_q, T_b) (Eq. (bformjqqh),
   Sec. 7.2 first remark: whole balls, all K x K pairs).  Runs the cell-list neighbour
   search, the pair geometry and quadrature, the symbolic CSR pattern (union over
   pairs with a non-empty region) and the numeric scatter.  *out receives a new
   library-owned n x n CSR (n = mesh->nv).  Synchronises the stream three times (to
   size the candidate-search grid, the candidate lists and the pattern); device memory
   comes from the device's stream-ordered pool on the context's stream.  The interior
   candidates' quadrature runs on a second stream of the context, concurrently with the
   boundary candidates' (ordered after the context's stream's earlier work, which waits
   for it before anything that follows).  The pattern's
   first row count uses a hash set of 2^b slots, b from the mean candidate list;
   NL_ROW_SET_BITS=b (6..13) in the environment sets it instead (the pattern does not
   depend on it: rows that fill the set are counted again in a full one). */
nl_status nl_assemble(nl_ctx *ctx, const nl_mesh *mesh, const nl_config *cfg, nl_csr *out);

/* Recompute the values of an nl_assemble result for the same mesh and configuration
   on its existing pattern (pair geometry, quadrature and scatter only).  No host
   synchronisation: can be captured in a CUDA graph (the context's second stream joins the
   capture through events). */
nl_status nl_assemble_numeric(nl_ctx *ctx, nl_csr *inout);

/* ---- batches of independent problems ----
   Many assemblies of uneven size, delta, ball and rule at once.  Every problem is
   assembled exactly as nl_assemble would (same interaction set and pattern, values
   equal up to the order of the FP64 atomic additions), but the batch:
     - runs each preparation and symbolic stage for all problems before synchronising,
       so the whole batch waits on the host three times, not three times per problem,
       with the problems spread over eight streams of the context (joined by events);
     - runs the numeric phase (pair geometry + quadrature) of all problems either in one
       pair of persistent launches (interior candidates, then boundary candidates) per value
       type x ball x kernel type present, whose warps take work items (a run of outer
       triangles of one problem) from a global counter, or as each problem's own kernels
       over several streams (the autotuner's choice, below);
     - scatters all problems in one launch per value type;
     - captures the numeric phase + scatter of the whole batch in a CUDA graph that
       nl_batch_run replays (re-assembly of the values on unchanged meshes).
   The schedule of the numeric phase is picked by a built-in autotuner: the first batch of a
   given shape (sizes, candidate counts, balls, rules, precisions) times seven schedules,
   each the median of three runs, and keeps the fastest in the context; later batches of the
   same shape reuse it.  Candidates: the persistent launches with 1 or 4 outer triangles per
   work item and the problems in input order or costliest first, or one resident block per SM
   fewer; or each problem's own kernels (those of nl_assemble_numeric, every kernel of a
   problem on one stream) with the problems dealt, costliest first, to 4 or 8 streams, so that
   small problems and the tails of large ones overlap (nl_batch_info.mode).  Every schedule yields the same pair blocks: each outer
   triangle's blocks are produced by one warp in a fixed order (the per-triangle sums
   taken with FP64 atomics, like the scatter's, may differ in the last bits). */
typedef struct nl_batch nl_batch;

enum { NL_BATCH_NO_TUNE = 1,       /* nl_batch_create flag: default schedule (persistent launches), no timing runs */
       NL_BATCH_PER_PROBLEM = 2    /* nl_batch_create flag: each problem's own kernels over all eight side
                                      streams, costliest first (schedule mode 1), no timing runs */
};
enum { NL_SCHED_DEFAULT = 0, NL_SCHED_TUNED = 1, NL_SCHED_CACHED = 2 };

typedef struct {
    int32_t chunk;        /* outer triangles per work item */
    int32_t order;        /* 0: problems in input order; 1: costliest problems first (estimated
                             candidates x outer points x inner points per triangle) */
    int32_t blocks;       /* persistent grid of the first boundary-candidate launch (blocks of 128 threads)
                             under the chosen schedule */
    int32_t launches;     /* numeric launches per run: one interior launch per value type, one boundary
                             launch per value type x ball x kernel type */
    int32_t source;       /* NL_SCHED_*: how the schedule was chosen */
    int32_t n_tried;      /* schedules timed by the autotuner in this nl_batch_create */
    double tuned_ms;      /* numeric phase of the batch with the chosen schedule (NL_SCHED_TUNED; median of 3) */
    double default_ms;    /* the same with the default schedule (NL_SCHED_TUNED; median of 3) */
    int32_t mode;         /* 0: persistent launches over all problems (chunk, order, blocks apply);
                             1: each problem's own kernels, as nl_assemble_numeric runs them, the
                             problems dealt to `streams` streams (costliest first with order 1);
                             nl_batch_run then also scatters each problem on its stream */
    int32_t streams;      /* mode 1: streams the problems are dealt to */
} nl_batch_info;

/* Assemble problems i = 0..n-1 (meshes[i], cfgs[i]) into outs[i] (library-owned, freed
   with nl_csr_free like an nl_assemble result) and return a handle that can re-run the
   numeric assembly of the whole batch.  The outs must stay allocated while the handle
   lives.  Errors: those of nl_assemble for the first failing problem (outs all zeroed),
   NL_EINVAL for n < 1 or null arrays. */
nl_status nl_batch_create(nl_ctx *ctx, int32_t n, const nl_mesh *meshes, const nl_config *cfgs, nl_csr *outs,
                          int32_t flags, nl_batch **batch);
/* Replay the captured numeric phase + scatter of every problem of the batch (one graph
   launch, stream-ordered, no host synchronisation). */
nl_status nl_batch_run(nl_ctx *ctx, nl_batch *batch);
nl_status nl_batch_get_info(const nl_batch *batch, nl_batch_info *info);
/* Release the handle (not the outs). */
void nl_batch_destroy(nl_ctx *ctx, nl_batch *batch);
/* Assemble n independent problems once (no handle, no re-assembly graph, no autotuning).
   Each problem is assembled exactly as nl_assemble assembles it (the same steps and kernels,
   every kernel of a problem in order on one of the context's eight side streams), pipelined
   across the problems: where nl_assemble waits on the host (three times a problem), each
   problem records an event instead, and the host issues a problem's next step once its own
   event has passed.  So one problem's preparation and symbolic stages run beside other
   problems' numeric phases.  Returns when every step is enqueued; the context's stream is
   ordered after all of them.  Errors: those of nl_assemble for the first failing problem
   (outs all zeroed), NL_EINVAL for n < 1 or null arrays. */
nl_status nl_assemble_batch(nl_ctx *ctx, int32_t n, const nl_mesh *meshes, const nl_config *cfgs,
                            nl_csr *outs);

/* Per-outer-triangle interaction statistics of the same geometry code the assembly
   runs: count_a[a] = #(q, b) with a non-empty region, qp_a[a] = inner points used,
   hash_a[a] = sum (mod 2^64) over those (a, q, b) of the record hash
   splitmix64(splitmix64(a << 32 | b) ^ (q << 24 | kind << 16 | nverts << 8 | ncaps))
   (splitmix64 of Steele, Lea and Flood), kind 1 = whole T_b, 2 = partial.  Host arrays [nt]. */
nl_status nl_interactions(nl_ctx *ctx, const nl_mesh *mesh, const nl_config *cfg,
                          uint64_t *hash_a, int64_t *count_a, int64_t *qp_a);

/* Split D by the node labels: A = D[Omega, Omega] (Eq. (weakja)) and
   B = D[Omega, Omega_I] (rule B of Sec. 7.2) with rows and columns renumbered in
   increasing node order within each label.  B is rectangular: B->n = #Omega rows and
   its column count is #Omega_I; both are new library-owned CSRs. */
nl_status nl_extract(nl_ctx *ctx, const nl_csr *D, const nl_mesh *mesh, nl_csr *A, nl_csr *B);

/* Right-hand side F = G - B g (Eq. (lfunc3) via rules B and C of Sec. 7.2), with the
   load vector G_j = int_Omega f phi_j over elements labelled Omega for f given by its
   nodal values (P1 interpolant), g the Dirichlet volume-constraint data at the nodes
   (Eq. (appr)).  f_nodal, g_nodal: [nv]; F: [#Omega] device or host. */
nl_status nl_rhs(nl_ctx *ctx, const nl_csr *B, const nl_mesh *mesh, const double *f_nodal,
                 const double *g_nodal, double *F);

/* y = A x with A's values in FP64 (NL_PREC_FP64) or rounded to FP32 (NL_PREC_FP32_COMP;
   products accumulated in FP32).  x, y: [A->n] device or host.  With device x and y the
   call is stream-ordered (it returns without waiting, and may be captured in a CUDA graph);
   with a host x or y it returns once y is complete. */
nl_status nl_matvec(nl_ctx *ctx, const nl_csr *A, const double *x, double *y, int32_t prec);

/* Solve A x = b (A symmetric positive definite, Sec. 2) by conjugate gradients with
   FP32 matrix-vector products and FP64 residual refinement until ||b - A x|| <= rtol ||b||
   (the paper names no solver, Sec. 7.2 "reduced sparsity" remark).  x holds the initial
   guess on entry and the last iterate on return.  b, x: [A->n], host or device memory of
   the context's device.  NL_OK only when the tolerance is reached; otherwise:
     NL_ENOCONV  max_it inner iterations, or 64 FP64 refinement passes (an rtol below the
                 FP64 residual floor), did not reach it; or a breakdown: a search direction
                 with p.Ap <= 0 or not a number (A not positive definite);
     NL_EINVAL   the residual is not finite (a NaN or an Inf in A, b or x), or a vector
                 lives on another device.
   *iters and *relres are set on every return (0 and +inf before the first residual). */
nl_status nl_cg(nl_ctx *ctx, const nl_csr *A, const double *b, double *x, double rtol, int32_t max_it,
                int32_t *iters, double *relres);

/* Copy a CSR to host arrays row_ptr[n+1], col_idx[nnz], val[nnz] (any may be NULL).
   Waits on the context's stream.  For an assembled matrix it also reads the device error word
   of the numeric phase and the scatter, which run after nl_assemble's last host
   synchronisation: NL_EUNSUPPORTED if one of them failed (a fixed-point sum beyond its bound,
   a missing pattern slot); the arrays are then filled but the values are not valid. */
nl_status nl_csr_download(nl_ctx *ctx, const nl_csr *m, int64_t *row_ptr, int32_t *col_idx, double *val);

/* Release the device buffers of m (safe on a zeroed nl_csr).  Stream-ordered on the
   context's stream: work already queued there that uses m finishes first; work on
   other streams must be complete (or ordered before the call) by the caller. */
void nl_csr_free(nl_ctx *ctx, nl_csr *m);

/* Device time of the phases of the last nl_assemble or nl_batch_create (ms):
   [0] preprocessing + cell list (for a batch: of all problems, plus the autotuner's
   timing runs when it ran), [1] pair geometry + quadrature, [2] symbolic pattern,
   [3] numeric scatter.  After nl_assemble_batch, whose phases overlap, [0..2] are 0 and
   [3] is the whole batch. */
nl_status nl_last_timings(nl_ctx *ctx, double *ms4);

/* nl_cg for callers that cannot allocate device memory: a framework that has given all
   device memory to its own caching allocator or a reserved arena, or a latency-critical
   loop that cannot take an allocation's synchronisation on every call.  The paper has no
   counterpart; this is a deployment variant of nl_cg.  Same arguments, results and
   errors as nl_cg (NL_OK only when the tolerance is reached), except:
     - A (row_ptr, col_idx, val), b and x must be device pointers of the context's device
       (else NL_EINVAL);
     - A->n must not exceed 262144 (else NL_EUNSUPPORTED): the work vectors live in one
       fixed file-scope device array of about 6 MB that every GPU loading the library
       keeps until the process exits, and no cudaMalloc or cudaFree is called;
     - the first call on a device looks up that array's address (cudaGetSymbolAddress)
       and caches it: make that first call before any stream capture;
     - all calls share the array; calls that overlap on the GPU race and must be
       serialised by the caller.  Each call clears what must start at zero itself. */
nl_status nl_cg_noalloc(nl_ctx *ctx, const nl_csr *A, const double *b, double *x, double rtol, int32_t max_it,
                        int32_t *iters, double *relres);

/* Measured fused multiply-add throughput of the context's GPU (TFLOP/s, 2 flop per FMA) in
   FP32 (NL_PREC_FP32_COMP) or FP64 (NL_PREC_FP64): independent FMA chains on every SM, best of
   three timed launches after a warm-up.  The paper has no counterpart: a measurement aid, the ALU
   roofline against which the pair quadrature (FP32 path) and the FP64 path are reported.
   Synchronises the context's stream. */
nl_status nl_fma_peak(nl_ctx *ctx, int32_t prec, double *tflops);

/* Number of CUDA kernels this context has launched so far (all entry points). */
int64_t nl_launch_count(nl_ctx *ctx);

/* Items (x_q, T_b) of the last nl_assemble or nl_interactions on the FP32-compensated
   path whose region the FP64 geometry built: FP32 choices it could not certify (a vertex,
   root or orientation too close to its threshold), the singular kernel's near-field items
   that FP32 cannot decide, and the cut items of the barycenter and overlap balls (their
   whole / empty choice is certified in FP32, their regions are whole triangles).  The
   boundary kernel queues them and a second kernel integrates the queue with every lane
   busy.  A full queue (capacity E/4, at least 4096) leaves the excess to the boundary
   kernel's own lanes; nl_assemble then runs the numeric phase again with a queue that holds
   every item and keeps it for the plan's re-assemblies (NL_DEFER_CAP in the environment
   fixes the capacity instead, 0 disables the queue; NL_DEFER_CAP_INIT sets the first one).  Each warp queues its items in (pair,
   outer point) order and a merge kernel adds the items of a pair onto it in that order (no
   atomics); the boundary kernel sums the other items of a pair in fixed point (order-free),
   and so does the scatter with the pairs' blocks in each outer triangle's rows.  So run to run the FP32-path pair blocks repeat exactly, except the singular kernel's
   near-field items, which k_near sums in FP32 in a queue-order grouping (measured up to 3e-8
   of max|D|), and the sums taken with FP64 atomics (M_aa, M_bb, the scatter into D) differ
   in their last bits (about 1e-16 relative).  0 for the FP64 path; -1 for a null context. */
int64_t nl_last_fp64_items(nl_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* NLFEM_H */
