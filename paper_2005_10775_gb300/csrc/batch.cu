// batch.cu -- many independent assemblies at once (nl_batch_*).
//
// Each problem is the assembly of Sec. 7 (Eq. (bformhj) with the quadrature of
// Eq. (bformjqqh)) exactly as nl_assemble performs it; what the batch changes is
// how the work reaches the GPU:
//   * preparation and symbolic stages run for every problem before the host waits,
//     so a batch synchronises three times in all, with the problems spread over the
//     context's eight side streams (problem i on stream i mod 8, joined by events);
//   * the numeric phase of every problem runs in a few persistent launches: the
//     interior candidates of all problems of a value type (nlq::k_interior_batch), then
//     the boundary candidates of all problems of a ball mode x kernel type
//     (nlq::k_boundary_batch); warps take work items (a run of `chunk` outer triangles
//     of one problem) from the launch's global counter;
//   * the scatter of every problem runs in one launch per value type;
//   * numeric phase + scatter are captured once in a CUDA graph (nl_batch_run).
// The autotuner times the numeric launches under eight schedules (item size, item order,
// resident blocks per SM), the median of three runs each, on the batch itself and keeps the
// fastest per batch shape in the context.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "internal.cuh"
#include "numeric.cuh"

namespace {

// zero the per-triangle M_bb sums of every problem of one argument array (block per problem)
__global__ void k_zero_mbb_batch(const nlq::NumArgs *__restrict__ As)
{
    const nlq::NumArgs &A = As[blockIdx.x];
    const int64_t n = 6 * (int64_t)A.K;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) A.mbb[i] = 0.0;
}

struct Sched {
    int mode = 0;    // 0: persistent launches over all problems; 1: each problem's own kernels, the
                     // problems spread over `streams` of the context's side streams
    int chunk = 1;   // mode 0: outer triangles per work item
    int order = 0;   // problems in input order (0) or costliest first (1)
    int fewer = 0;   // mode 0: resident blocks per SM below the occupancy limit, every persistent launch
    int streams = 0; // mode 1: side streams
};

// Host arrays that feed a cudaMemcpyAsync stay alive until the stream has passed the
// copy: on a coherent CPU-GPU system the copy engine may read pageable memory when the
// copy runs, not when it is issued.
struct PrecGroup {                 // the kernel arguments of the problems of one value type
    bool f64 = false;
    std::vector<int> probs;
    std::vector<nlq::NumArgs> host;
    nlq::NumArgs *dA = nullptr;    // [probs.size()]
};

struct Launch {                    // one persistent numeric launch
    int prec = 0;                  // index into nl_batch::pgroups
    int ball = -1;                 // -1: interior candidates; else the boundary candidates of this ball
    bool inv = false;
    std::vector<int> probs;        // problems (batch indices)
    std::vector<nlq::BatchItem> host_items;
    nlq::BatchItem *items = nullptr;
    int n_items = 0, cap_items = 0;
    int blocks = 0;
    int per_sm = 1;                    // resident blocks per SM at the occupancy limit
    nlq::DeferItem *defer = nullptr;   // float boundary launches: queue of the FP64-decided items
    int defer_cap = 0;
};

// does a boundary launch of this value type and ball queue items for the deferred kernel?
bool uses_queue(bool f64, int ball)
{
    return !f64 && ball >= 0 && ball != NL_BALL_BARY_NOCAPS && ball != NL_BALL_BARY_APPROXCAPS;
}

struct ScatterGroup {              // one scatter launch: problems of one value type
    bool f64 = false;
    std::vector<int> probs;
    std::vector<ScatterArgs> host_S;
    std::vector<int64_t> host_koff;
    ScatterArgs *dS = nullptr;
    int64_t *dkoff = nullptr;
    int64_t totalK = 0, max_row = 0;
};

}  // namespace

struct nl_tune_cache {
    std::vector<std::pair<uint64_t, Sched>> entries;
};

void nl_tune_cache_free(nl_tune_cache *c) { delete c; }

struct nl_batch {
    int n = 0;
    std::vector<nl_plan *> P;      // owned by the outs (nl_csr.priv)
    std::vector<nl_csr *> out;
    std::vector<PrecGroup> pgroups;
    std::vector<Launch> launches;
    int *counters = nullptr;       // two per launch: work items taken, deferred items queued
    std::vector<ScatterGroup> sgroups;
    std::vector<ScatterArgs> host_S_all;
    std::vector<int64_t> host_zoff;
    ScatterArgs *dS_all = nullptr; // every problem, for the W reset and the symmetrisation
    int64_t *dzoff = nullptr;
    int64_t total_nnz = 0;
    Sched sched;
    nl_batch_info info{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t graph_kernels = 0;     // kernels one replay launches
    cudaEvent_t tev[2] = {nullptr, nullptr};   // the autotuner's timing events
};

namespace {

template <class T>
void free_async(T *&p, cudaStream_t s)
{
    if (p) cudaFreeAsync((void *)p, s);
    p = nullptr;
}

void release(nl_batch *b, cudaStream_t s)
{
    for (cudaEvent_t &e : b->tev)
        if (e) {
            cudaEventDestroy(e);
            e = nullptr;
        }
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    for (PrecGroup &g : b->pgroups) free_async(g.dA, s);
    for (Launch &l : b->launches) {
        free_async(l.items, s);
        free_async(l.defer, s);
    }
    free_async(b->counters, s);
    for (ScatterGroup &g : b->sgroups) {
        free_async(g.dS, s);
        free_async(g.dkoff, s);
    }
    free_async(b->dS_all, s);
    free_async(b->dzoff, s);
}

// FNV-1a over the values that decide the numeric work of the batch
uint64_t batch_signature(const nl_batch *b)
{
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) {
        for (int i = 0; i < 8; i++) {
            h ^= (v >> (8 * i)) & 0xff;
            h *= 1099511628211ull;
        }
    };
    mix((uint64_t)b->n);
    for (const nl_plan *P : b->P) {
        const nl_config &c = P->cfg;
        mix((uint64_t)P->K);
        mix((uint64_t)P->E);
        mix((uint64_t)c.ball | ((uint64_t)c.prec << 8) | ((uint64_t)c.kernel << 16) | ((uint64_t)c.outer << 24) |
            ((uint64_t)c.inner << 32) | ((uint64_t)c.ngon_n << 40) | ((uint64_t)c.cap_m << 48));
    }
    return h;
}

int rule_points(int id)
{
    switch (id) {
    case NL_RULE_GAUSS3: return 3;
    case NL_RULE_GAUSS4: return 4;
    case NL_RULE_PAPER7: return 7;
    case NL_RULE_DUNAVANT7: return 7;
    case NL_RULE_DUNAVANT16: return 16;
    case NL_RULE_SWITCH47: return 7;
    default: return 7;
    }
}

// estimated numeric work per outer triangle of problem P (for the costliest-first order)
double triangle_cost(const nl_plan *P)
{
    const double cand = P->K > 0 ? (double)P->E / (double)P->K : 0.0;
    return cand * rule_points(P->cfg.outer) * rule_points(P->cfg.inner);
}

// persistent grid of every launch under schedule sc (SM count nsm)
void apply_grid(nl_batch *b, const Sched &sc, int nsm)
{
    for (Launch &l : b->launches) l.blocks = std::max(1, l.per_sm - sc.fewer) * nsm;
}

nl_status build_items(nl_ctx *ctx, nl_batch *b, const Sched &sc)
{
    // the previous item lists may still be in flight to the device
    for (const Launch &l : b->launches)
        if (!l.host_items.empty()) {
            NL_CK(cudaStreamSynchronize(ctx->stream));
            break;
        }
    for (Launch &l : b->launches) {
        const std::vector<int> &local_of = b->pgroups[l.prec].probs;
        std::vector<int> order = l.probs;
        if (sc.order == 1)
            std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
                return triangle_cost(b->P[x]) > triangle_cost(b->P[y]);
            });
        std::vector<nlq::BatchItem> &items = l.host_items;
        items.clear();
        for (int p : order) {
            // index of problem p within its value type's argument array
            const int local = (int)(std::find(local_of.begin(), local_of.end(), p) - local_of.begin());
            const int K = b->P[p]->K;
            for (int a0 = 0; a0 < K; a0 += sc.chunk) items.push_back({local, a0, std::min(K, a0 + sc.chunk)});
        }
        if ((int)items.size() > l.cap_items) {
            free_async(l.items, ctx->stream);
            nl_status s = nl_alloc(ctx, &l.items, items.size());
            if (s != NL_OK) return s;
            l.cap_items = (int)items.size();
        }
        l.n_items = (int)items.size();
        if (l.n_items)
            NL_CK(cudaMemcpyAsync(l.items, items.data(), sizeof(nlq::BatchItem) * items.size(),
                                  cudaMemcpyHostToDevice, ctx->stream));
    }
    return NL_OK;
}

// problems in the order of schedule sc
std::vector<int> problem_order(const nl_batch *b, const Sched &sc)
{
    std::vector<int> order(b->n);
    for (int i = 0; i < b->n; i++) order[i] = i;
    if (sc.order == 1)
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            return triangle_cost(b->P[x]) > triangle_cost(b->P[y]);
        });
    return order;
}

// Schedule mode 1: each problem's numeric phase as nl_assemble_numeric runs it (its kernels on
// one stream), the problems dealt round-robin to `streams` side streams that start after the
// context's stream's earlier work and that the context's stream waits for, so that small
// problems and the tails of large ones overlap.
nl_status launch_numeric_streams(nl_ctx *ctx, nl_batch *b, const Sched &sc, bool scatter)
{
    nl_status s = nl_side_streams(ctx);
    if (s != NL_OK) return s;
    const int ns = std::max(1, std::min(sc.streams, (int)nl_ctx::kSideStreams));
    cudaStream_t st = ctx->stream;
    NL_CK(cudaEventRecord(ctx->side_ev[nl_ctx::kSideStreams], st));
    for (int k = 0; k < ns; k++) NL_CK(cudaStreamWaitEvent(ctx->side[k], ctx->side_ev[nl_ctx::kSideStreams], 0));
    const std::vector<int> order = problem_order(b, sc);
    for (int j = 0; j < b->n && s == NL_OK; j++) {
        ctx->stream = ctx->side[j % ns];
        s = nl_run_numeric_one_stream(ctx, b->P[order[j]]);
        // the re-assembly: each problem's scatter right after its numeric phase, on its stream
        if (s == NL_OK && scatter) s = nl_run_scatter(ctx, b->P[order[j]], b->out[order[j]]);
    }
    ctx->stream = st;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < ns; k++) {
        cudaError_t e1 = cudaEventRecord(ctx->side_ev[k], ctx->side[k]);
        if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(st, ctx->side_ev[k], 0);
        if (e1 != cudaSuccess) {
            cudaStreamSynchronize(ctx->side[k]);
            if (e == cudaSuccess) e = e1;
        }
    }
    if (s == NL_OK && e != cudaSuccess) return nl_cuda_fail(ctx, e, "joining the side streams");
    return s;
}

nl_status launch_numeric(nl_ctx *ctx, nl_batch *b, bool set_attr)
{
    if (b->sched.mode == 1) return launch_numeric_streams(ctx, b, b->sched, false);
    const size_t nl = b->launches.size();
    NL_CK(cudaMemsetAsync(b->counters, 0, sizeof(int) * 2 * nl, ctx->stream));
    // the per-triangle M_bb sums start at zero in every numeric run (the autotuner's too)
    for (const PrecGroup &g : b->pgroups) {
        k_zero_mbb_batch<<<(unsigned)g.probs.size(), 256, 0, ctx->stream>>>(g.dA); ++ctx->launches;
        NL_CK(cudaGetLastError());
    }
    for (size_t k = 0; k < nl; k++) {
        const Launch &l = b->launches[k];
        if (!l.n_items) continue;
        const PrecGroup &g = b->pgroups[l.prec];
        int *c = b->counters + k;
        nl_status s;
        if (l.ball < 0)
            s = g.f64 ? nl_launch_interior_batch_f64(ctx, g.dA, l.items, l.n_items, c, l.blocks)
                      : nl_launch_interior_batch_f32(ctx, g.dA, l.items, l.n_items, c, l.blocks);
        else
            s = g.f64 ? nl_launch_boundary_batch_f64(ctx, l.ball, l.inv, g.dA, l.items, l.n_items, c, l.blocks,
                                                     set_attr)
                      : nl_launch_boundary_batch_f32(ctx, l.ball, l.inv, g.dA, l.items, l.n_items, c, l.blocks,
                                                     set_attr);
        if (s == NL_OK && l.defer)
            s = nl_launch_deferred_batch_f32(ctx, l.ball, g.dA, l.defer, b->counters + nl + k, l.defer_cap);
        if (s != NL_OK) return s;
    }
    return NL_OK;
}

nl_status launch_scatter(nl_ctx *ctx, nl_batch *b, bool set_attr)
{
    nl_status s = nl_launch_zero_batch(ctx, b->dS_all, b->dzoff, b->n, b->total_nnz);
    if (s != NL_OK) return s;
    for (ScatterGroup &g : b->sgroups)
        if ((s = nl_launch_scatter_batch(ctx, g.f64, g.dS, g.dkoff, (int)g.probs.size(), g.totalK, g.max_row,
                                         set_attr)) != NL_OK)
            return s;
    return nl_launch_symmetrize_batch(ctx, b->dS_all, b->dzoff, b->n, b->total_nnz);
}

// device time of the numeric phase of the batch under schedule sc: the median of `reps` runs
nl_status time_numeric(nl_ctx *ctx, nl_batch *b, const Sched &sc, int nsm, int reps, double *ms)
{
    nl_status s = build_items(ctx, b, sc);
    if (s != NL_OK) return s;
    apply_grid(b, sc, nsm);
    b->sched = sc;
    if (!b->tev[0]) NL_CK(cudaEventCreate(&b->tev[0]));
    if (!b->tev[1]) NL_CK(cudaEventCreate(&b->tev[1]));
    std::vector<double> t;
    for (int r = 0; r < reps; r++) {
        NL_CK(cudaEventRecord(b->tev[0], ctx->stream));
        if ((s = launch_numeric(ctx, b, false)) != NL_OK) return s;
        NL_CK(cudaEventRecord(b->tev[1], ctx->stream));
        NL_CK(cudaEventSynchronize(b->tev[1]));
        float f = 0.0f;
        NL_CK(cudaEventElapsedTime(&f, b->tev[0], b->tev[1]));
        t.push_back(f);
    }
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return NL_OK;
}

nl_status pick_schedule(nl_ctx *ctx, nl_batch *b, int flags, int nsm)
{
    const uint64_t sig = batch_signature(b);
    Sched def;   // one outer triangle per item, input order
    b->info.source = NL_SCHED_DEFAULT;
    b->sched = def;
    if (flags & NL_BATCH_PER_PROBLEM) {   // each problem's own kernels, costliest first, all side streams
        b->sched.mode = 1;
        b->sched.order = 1;
        b->sched.streams = nl_ctx::kSideStreams;
        return NL_OK;
    }
    if (flags & NL_BATCH_NO_TUNE) return NL_OK;
    if (!ctx->tune) ctx->tune = new (std::nothrow) nl_tune_cache();
    if (!ctx->tune) return nl_fail(ctx, NL_ENOMEM, "host allocation failed");
    for (const auto &e : ctx->tune->entries)
        if (e.first == sig) {
            b->sched = e.second;
            b->info.source = NL_SCHED_CACHED;
            return NL_OK;
        }
    // warm-up (instruction cache, L2, clocks), then every candidate: the median of three runs.
    // Candidates: outer triangles per item (1, 4), problem order (input, costliest first) and
    // resident blocks per SM (the occupancy limit, one fewer: fewer blocks leave each one more
    // of the SM's L1 and issue slots, more blocks hide more latency)
    double ms = 0.0;
    nl_status s = time_numeric(ctx, b, def, nsm, 1, &ms);
    if (s != NL_OK) return s;
    std::vector<Sched> cands;
    for (int order = 0; order < 2; order++)
        for (int c : {1, 4}) {
            Sched sc;
            sc.chunk = c;
            sc.order = order;
            cands.push_back(sc);
        }
    {
        Sched sc;   // one resident block per SM fewer
        sc.order = 1;
        sc.fewer = 1;
        cands.push_back(sc);
    }
    for (int ns : {4, 8}) {   // each problem's own kernels over ns streams, costliest first
        Sched sc;
        sc.mode = 1;
        sc.order = 1;
        sc.streams = ns;
        cands.push_back(sc);
    }
    double best = INFINITY;
    Sched bs = def;
    int tried = 0;
    for (const Sched &sc : cands) {
        if ((s = time_numeric(ctx, b, sc, nsm, 3, &ms)) != NL_OK) return s;
        tried++;
        if (sc.mode == def.mode && sc.chunk == def.chunk && sc.order == def.order && sc.fewer == def.fewer)
            b->info.default_ms = ms;
        if (ms < best) {
            best = ms;
            bs = sc;
        }
    }
    b->sched = bs;
    b->info.source = NL_SCHED_TUNED;
    b->info.n_tried = tried;
    b->info.tuned_ms = best;
    ctx->tune->entries.push_back({sig, bs});
    return NL_OK;
}

nl_status sync(nl_ctx *ctx)
{
    NL_CK(cudaStreamSynchronize(ctx->stream));
    return NL_OK;
}

// One stage of the preparation or symbolic phase for problems 0..n-1: stage(i) runs with
// ctx->stream set to side stream i mod kSideStreams, so that the small kernels of different
// problems overlap.  The side streams start after the work already on the context's stream,
// and that stream waits for all of them before anything that follows (also after a failure,
// so that no buffer it frees is still in use).  A problem keeps its side stream in every
// stage, so its buffers stay stream-ordered between stages as well.
template <class Stage>
nl_status fan_out(nl_ctx *ctx, int n, int *fail_at, Stage stage)
{
    nl_status s = nl_side_streams(ctx);
    if (s != NL_OK) return s;
    cudaStream_t st = ctx->stream;
    const int ns = nl_ctx::kSideStreams;
    NL_CK(cudaEventRecord(ctx->side_ev[ns], st));
    for (int k = 0; k < ns; k++) NL_CK(cudaStreamWaitEvent(ctx->side[k], ctx->side_ev[ns], 0));
    for (int i = 0; i < n && s == NL_OK; i++) {
        ctx->stream = ctx->side[i % ns];
        s = stage(i);
        if (s != NL_OK) *fail_at = i;
    }
    ctx->stream = st;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < ns; k++) {
        cudaError_t e1 = cudaEventRecord(ctx->side_ev[k], ctx->side[k]);
        if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(st, ctx->side_ev[k], 0);
        if (e1 != cudaSuccess) {
            cudaStreamSynchronize(ctx->side[k]);   // no ordering event: wait on the host instead
            if (e == cudaSuccess) e = e1;
        }
    }
    if (s == NL_OK && e != cudaSuccess) return nl_cuda_fail(ctx, e, "joining the side streams");
    return s;
}

// NL_SYNC_CHECK=1 in the environment: synchronise and check after every phase of
// nl_batch_create, so that a device error is reported with the phase that raised it
bool sync_check_enabled()
{
    static const bool on = [] {
        const char *v = getenv("NL_SYNC_CHECK");
        return v && v[0] && v[0] != '0';
    }();
    return on;
}

nl_status phase_check(nl_ctx *ctx, nl_batch *b, const char *phase)
{
    if (!sync_check_enabled()) return NL_OK;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return nl_fail(ctx, NL_ECUDA, std::string(phase) + ": " + cudaGetErrorString(e));
    for (size_t i = 0; i < b->P.size(); i++) {
        int herr = 0;
        if (b->P[i]->err) {
            e = cudaMemcpy(&herr, b->P[i]->err, sizeof(int), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return nl_fail(ctx, NL_ECUDA, std::string(phase) + ": " + cudaGetErrorString(e));
        }
        if (herr)
            return nl_fail(ctx, NL_EUNSUPPORTED, std::string(phase) + ": problem " + std::to_string(i) +
                                                     " error word " + std::to_string(herr));
    }
    return NL_OK;
}

// nl_assemble_batch: each problem's assembly exactly as nl_assemble performs it (the same steps,
// every kernel of a problem in order on one of the context's side streams), pipelined across
// the problems.  The problems are dealt to the streams costliest first, each to the stream with
// the least cost so far (cost K^2 delta^2: candidate pairs on a mesh of the unit square's scale),
// and issued in that order.  nl_assemble waits on the host three times (the
// candidate-search grid, the candidate count, the pattern size); here each problem records an
// event after each of those steps, and the host polls the events and issues a problem's next
// step as soon as its own values have arrived.  So one problem's preparation and symbolic
// stages (small, latency-bound kernels) run beside other problems' numeric phases instead of
// the whole batch waiting at each synchronisation.  No autotuning and no re-assembly graph
// (nl_batch_create builds those).
nl_status assemble_pipelined(nl_ctx *ctx, int n, const nl_mesh *meshes, const nl_config *cfgs, nl_csr *outs)
{
    nl_status s = nl_side_streams(ctx);
    if (s != NL_OK) return s;
    cudaStream_t st = ctx->stream;
    const int ns = nl_ctx::kSideStreams;
    std::vector<nl_prep *> T(n, nullptr);
    std::vector<nl_pat *> Q(n, nullptr);
    std::vector<cudaEvent_t> ev(n, nullptr);
    std::vector<int> step(n, 0), sidx(n, 0), order(n);
    {
        std::vector<double> cost(n), load(ns, 0.0);
        for (int i = 0; i < n; i++) {
            order[i] = i;
            const double K = (double)meshes[i].nt, d = cfgs[i].delta;
            cost[i] = K * K * d * d;
        }
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
        for (int i : order) {
            const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            sidx[i] = k;
            load[k] += cost[i];
        }
    }
    nl_host_slot *h = nullptr;
    int fail_at = -1;
    bool forked = false;
    auto finish = [&](nl_status code) {
        ctx->stream = st;
        if (forked)   // the context's stream continues after every side stream
            for (int k = 0; k < ns; k++) {
                cudaError_t e = cudaEventRecord(ctx->side_ev[k], ctx->side[k]);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->side_ev[k], 0);
                if (e != cudaSuccess) cudaStreamSynchronize(ctx->side[k]);
            }
        if (code != NL_OK) cudaStreamSynchronize(st);
        for (int i = 0; i < n; i++) {
            nl_prep_delete(T[i], st);
            nl_pat_delete(Q[i], st);
            if (ev[i]) cudaEventDestroy(ev[i]);
            if (code != NL_OK) {
                nl_csr_free(ctx, &outs[i]);
            } else if (outs[i].priv) {
                ((nl_plan *)outs[i].priv)->stream = st;   // the plans' buffers are freed on the context's stream
            }
        }
        if (code != NL_OK && fail_at >= 0) ctx->err = "problem " + std::to_string(fail_at) + ": " + ctx->err;
        return code;
    };
    if ((s = nl_host_slots(ctx, n, &h)) != NL_OK) return finish(s);
    for (int i = 0; i < n; i++) {
        nl_plan *P = new (std::nothrow) nl_plan();
        T[i] = nl_prep_new();
        Q[i] = nl_pat_new();
        if (!P || !T[i] || !Q[i]) {
            delete P;
            return finish(nl_fail(ctx, NL_ENOMEM, "host allocation failed"));
        }
        outs[i].priv = P;
        if (cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess) {
            ev[i] = nullptr;
            return finish(nl_fail(ctx, NL_ECUDA, "cudaEventCreate"));
        }
    }
    // the phases overlap: nl_last_timings reports the whole batch as its last phase
    for (int k = 0; k < 4; k++)
        if (cudaEventRecord(ctx->ev[k], st) != cudaSuccess) return finish(nl_fail(ctx, NL_ECUDA, "cudaEventRecord"));
    if (cudaEventRecord(ctx->side_ev[ns], st) != cudaSuccess) return finish(nl_fail(ctx, NL_ECUDA, "cudaEventRecord"));
    for (int k = 0; k < ns; k++)
        if (cudaStreamWaitEvent(ctx->side[k], ctx->side_ev[ns], 0) != cudaSuccess)
            return finish(nl_fail(ctx, NL_ECUDA, "cudaStreamWaitEvent"));
    forked = true;
    // step k of problem i (k = 0 .. 3); the steps before 3 end with an event
    auto issue = [&](int i) -> nl_status {
        ctx->stream = ctx->side[sidx[i]];
        nl_plan *P = (nl_plan *)outs[i].priv;
        nl_status r = NL_OK;
        switch (step[i]) {
        case 0: r = nl_prepare_a(ctx, &meshes[i], &cfgs[i], P, T[i], &h[i]); break;
        case 1: r = nl_prepare_b(ctx, P, T[i], &h[i]); break;
        case 2: r = nl_assemble_step_c(ctx, P, T[i], Q[i], &h[i], &outs[i], true, nullptr, nullptr); break;
        default:
            r = nl_assemble_step_d(ctx, P, Q[i], &h[i], &outs[i], true, nullptr);
            if (r == NL_OK) {
                nl_prep_delete(T[i], ctx->stream);
                nl_pat_delete(Q[i], ctx->stream);
                T[i] = nullptr;
                Q[i] = nullptr;
            }
        }
        if (r == NL_OK && step[i] < 3 && cudaEventRecord(ev[i], ctx->stream) != cudaSuccess)
            r = nl_fail(ctx, NL_ECUDA, "cudaEventRecord");
        ctx->stream = st;
        step[i]++;
        return r;
    };
    for (int i : order)
        if ((s = issue(i)) != NL_OK) {
            fail_at = i;
            return finish(s);
        }
    int64_t fp64_items = 0;
    for (;;) {
        int open = 0;
        bool moved = false;
        for (int i : order) {
            if (step[i] > 3) continue;
            open++;
            const cudaError_t q = cudaEventQuery(ev[i]);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                fail_at = i;
                return finish(nl_cuda_fail(ctx, q, "a batch problem's stream"));
            }
            if (step[i] == 3) fp64_items += h[i].deferred;
            if ((s = issue(i)) != NL_OK) {
                fail_at = i;
                return finish(s);
            }
            moved = true;
        }
        if (!open) break;
        if (!moved) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    s = finish(NL_OK);
    if (cudaEventRecord(ctx->ev[4], st) != cudaSuccess) return nl_fail(ctx, NL_ECUDA, "cudaEventRecord");
    ctx->last_fp64_items = fp64_items;
    return s;
}

}  // namespace

extern "C" {

nl_status nl_batch_create(nl_ctx *ctx, int32_t n, const nl_mesh *meshes, const nl_config *cfgs, nl_csr *outs,
                          int32_t flags, nl_batch **batch)
{
    if (!ctx) return NL_EINVAL;
    if (!batch) return nl_fail(ctx, NL_EINVAL, "null batch handle");
    *batch = nullptr;
    if (n < 1 || !meshes || !cfgs || !outs) return nl_fail(ctx, NL_EINVAL, "need n >= 1 and non-null arrays");
    nl_status s;
    for (int i = 0; i < n; i++) {
        if ((s = nl_validate(ctx, &meshes[i], &cfgs[i])) != NL_OK) {
            ctx->err = "problem " + std::to_string(i) + ": " + ctx->err;
            return s;
        }
    }
    NL_CK(cudaSetDevice(ctx->device));
    for (int i = 0; i < n; i++) memset(&outs[i], 0, sizeof outs[i]);
    nl_batch *b = new (std::nothrow) nl_batch();
    if (!b) return nl_fail(ctx, NL_ENOMEM, "host allocation failed");
    b->n = n;
    std::vector<nl_prep *> T(n, nullptr);
    std::vector<nl_pat *> Q(n, nullptr);
    nl_host_slot *h = nullptr;
    int fail_at = -1;
    cudaStream_t st = ctx->stream;
    auto fail = [&](nl_status code) {
        cudaStreamSynchronize(st);
        for (int i = 0; i < n; i++) {
            nl_prep_delete(T[i], st);
            nl_pat_delete(Q[i], st);
            nl_csr_free(ctx, &outs[i]);
        }
        release(b, st);
        delete b;
        if (fail_at >= 0) ctx->err = "problem " + std::to_string(fail_at) + ": " + ctx->err;
        return code;
    };
    if ((s = nl_host_slots(ctx, n, &h)) != NL_OK) return fail(s);
    for (int i = 0; i < n; i++) {
        nl_plan *P = new (std::nothrow) nl_plan();
        T[i] = nl_prep_new();
        Q[i] = nl_pat_new();
        if (!P || !T[i] || !Q[i]) {
            delete P;
            return fail(nl_fail(ctx, NL_ENOMEM, "host allocation failed"));
        }
        outs[i].priv = P;
        b->P.push_back(P);
        b->out.push_back(&outs[i]);
    }
    if (cudaEventRecord(ctx->ev[0], st) != cudaSuccess) return fail(nl_fail(ctx, NL_ECUDA, "cudaEventRecord"));
    // ---- preparation, all problems per stage, spread over the side streams ----
    if ((s = fan_out(ctx, n, &fail_at, [&](int i) {
             return nl_prepare_a(ctx, &meshes[i], &cfgs[i], b->P[i], T[i], &h[i]);
         })) != NL_OK)
        return fail(s);
    for (int i = 0; i < n; i++) b->P[i]->stream = st;   // the plans' buffers are freed on the context's stream
    if ((s = sync(ctx)) != NL_OK) return fail(s);
    if ((s = fan_out(ctx, n, &fail_at, [&](int i) { return nl_prepare_b(ctx, b->P[i], T[i], &h[i]); })) != NL_OK)
        return fail(s);
    if ((s = sync(ctx)) != NL_OK) return fail(s);
    if ((s = fan_out(ctx, n, &fail_at, [&](int i) {
             nl_status r = nl_prepare_c(ctx, b->P[i], T[i], &h[i]);
             return r == NL_OK ? nl_alloc_numeric(ctx, b->P[i]) : r;
         })) != NL_OK)
        return fail(s);
    // ---- numeric launches: interior per value type, boundary per value type x ball x kernel ----
    for (int f = 0; f < 2; f++) {
        PrecGroup g;
        g.f64 = f == 1;
        for (int i = 0; i < n; i++)
            if ((b->P[i]->cfg.prec == NL_PREC_FP64) == g.f64) g.probs.push_back(i);
        if (g.probs.empty()) continue;
        b->pgroups.push_back(g);
        const int pg = (int)b->pgroups.size() - 1;
        Launch li;
        li.prec = pg;
        li.probs = g.probs;
        b->launches.push_back(li);
        for (int i : g.probs) {
            const int ball = b->P[i]->cfg.ball;
            const bool inv = b->P[i]->cfg.kernel == NL_KERNEL_INV_DIST;
            Launch *l = nullptr;
            for (Launch &x : b->launches)
                if (x.prec == pg && x.ball == ball && x.inv == inv) l = &x;
            if (!l) {
                Launch lb;
                lb.prec = pg;
                lb.ball = ball;
                lb.inv = inv;
                b->launches.push_back(lb);
                l = &b->launches.back();
            }
            l->probs.push_back(i);
        }
    }
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess)
        return fail(nl_fail(ctx, NL_ECUDA, "cudaDeviceGetAttribute"));
    const size_t nlaunch = b->launches.size();
    if ((s = nl_alloc(ctx, &b->counters, 2 * nlaunch)) != NL_OK) return fail(s);
    // one deferred-item queue per float boundary launch, sized by its problems' candidate pairs
    for (Launch &l : b->launches) {
        if (!uses_queue(b->pgroups[l.prec].f64, l.ball)) continue;
        int64_t E = 0;
        for (int i : l.probs) E += b->P[i]->E;
        l.defer_cap = nl_defer_cap(E);
        if ((s = nl_alloc(ctx, &l.defer, nlq::defer_alloc_items(l.defer_cap))) != NL_OK) return fail(s);
    }
    for (int pg = 0; pg < (int)b->pgroups.size(); pg++) {
        PrecGroup &g = b->pgroups[pg];
        std::vector<nlq::NumArgs> &args = g.host;
        args.resize(g.probs.size());
        for (size_t k = 0; k < g.probs.size(); k++) {
            if ((s = nl_fill_args(ctx, b->P[g.probs[k]], args[k], false)) != NL_OK) return fail(s);
            for (size_t j = 0; j < nlaunch; j++) {
                const Launch &l = b->launches[j];
                if (l.prec != pg || !l.defer ||
                    std::find(l.probs.begin(), l.probs.end(), g.probs[k]) == l.probs.end())
                    continue;
                args[k].defer = l.defer;
                args[k].dval = nlq::defer_values(l.defer, l.defer_cap);
                args[k].defer_n = b->counters + nlaunch + j;
                args[k].defer_cap = l.defer_cap;
                args[k].prob = (int)k;
            }
        }
        if ((s = nl_alloc(ctx, &g.dA, args.size())) != NL_OK) return fail(s);
        if (cudaMemcpyAsync(g.dA, args.data(), sizeof(nlq::NumArgs) * args.size(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
            return fail(nl_fail(ctx, NL_ECUDA, "upload of the kernel arguments"));
    }
    for (Launch &l : b->launches) {
        int per_sm = 0;
        s = b->pgroups[l.prec].f64 ? nl_batch_occupancy_f64(ctx, l.ball, l.inv, &per_sm)
                                   : nl_batch_occupancy_f32(ctx, l.ball, l.inv, &per_sm);
        if (s != NL_OK) return fail(s);
        l.per_sm = std::max(1, per_sm);
        l.blocks = l.per_sm * nsm;
    }
    b->info.launches = (int)b->launches.size();
    if ((s = pick_schedule(ctx, b, flags, nsm)) != NL_OK) return fail(s);
    b->info.chunk = b->sched.chunk;
    b->info.order = b->sched.order;
    b->info.mode = b->sched.mode;
    b->info.streams = b->sched.streams;
    if ((s = build_items(ctx, b, b->sched)) != NL_OK) return fail(s);
    apply_grid(b, b->sched, nsm);
    for (const Launch &l : b->launches)
        if (l.ball >= 0) {
            b->info.blocks = l.blocks;
            break;
        }
    if (cudaEventRecord(ctx->ev[1], st) != cudaSuccess) return fail(nl_fail(ctx, NL_ECUDA, "cudaEventRecord"));
    if ((s = launch_numeric(ctx, b, true)) != NL_OK || (s = phase_check(ctx, b, "numeric")) != NL_OK) return fail(s);
    if (cudaEventRecord(ctx->ev[2], st) != cudaSuccess) return fail(nl_fail(ctx, NL_ECUDA, "cudaEventRecord"));
    // ---- symbolic phase, all problems per stage, spread over the side streams ----
    if ((s = fan_out(ctx, n, &fail_at, [&](int i) { return nl_pattern_a(ctx, b->P[i], &outs[i], Q[i], &h[i]); })) !=
        NL_OK)
        return fail(s);
    if ((s = sync(ctx)) != NL_OK) return fail(s);
    if ((s = fan_out(ctx, n, &fail_at, [&](int i) {
             nl_status r = nl_prepare_check(ctx, &h[i]);
             return r == NL_OK ? nl_pattern_b(ctx, b->P[i], &outs[i], Q[i], &h[i]) : r;
         })) != NL_OK)
        return fail(s);
    if ((s = phase_check(ctx, b, "symbolic")) != NL_OK) return fail(s);
    if (cudaEventRecord(ctx->ev[3], st) != cudaSuccess) return fail(nl_fail(ctx, NL_ECUDA, "cudaEventRecord"));
    // ---- scatter arguments ----
    {
        std::vector<ScatterArgs> &all = b->host_S_all;
        std::vector<int64_t> &zoff = b->host_zoff;
        all.assign(n, ScatterArgs{});
        zoff.assign(n + 1, 0);
        for (int i = 0; i < n; i++) {
            const nl_plan *P = b->P[i];
            ScatterArgs &a = all[i];
            a.K = P->K;
            a.J = P->J;
            a.E = P->E;
            a.tri = P->tri;
            a.ptr = P->nbr_ptr;
            a.idx = P->nbr_idx;
            a.flag = P->flag;
            a.blk = P->blk;
            a.maa = P->maa;
            a.mbb = P->mbb;
            a.lslot = P->lslot;
            a.row_ptr = outs[i].row_ptr;
            a.col = outs[i].col_idx;
            a.W = P->W;
            a.tslot = P->tslot;
            a.val = outs[i].val;
            a.err = P->err;
            a.area = P->area;
            a.fxe = P->fxe;
            a.ws = nl_outer_abs_weight(P);
            zoff[i + 1] = zoff[i] + outs[i].nnz;
        }
        b->total_nnz = zoff[n];
        if ((s = nl_alloc(ctx, &b->dS_all, (size_t)n)) != NL_OK || (s = nl_alloc(ctx, &b->dzoff, (size_t)n + 1)) != NL_OK)
            return fail(s);
        if (cudaMemcpyAsync(b->dS_all, all.data(), sizeof(ScatterArgs) * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(b->dzoff, zoff.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st) !=
                cudaSuccess)
            return fail(nl_fail(ctx, NL_ECUDA, "upload of the scatter arguments"));
        b->sgroups.reserve(2);
        for (int f = 0; f < 2; f++) {
            b->sgroups.emplace_back();
            ScatterGroup &g = b->sgroups.back();
            g.f64 = f == 1;
            std::vector<ScatterArgs> &sa = g.host_S;
            std::vector<int64_t> &koff = g.host_koff;
            koff.assign(1, 0);
            for (int i = 0; i < n; i++)
                if ((b->P[i]->cfg.prec == NL_PREC_FP64) == g.f64) {
                    g.probs.push_back(i);
                    sa.push_back(all[i]);
                    koff.push_back(koff.back() + b->P[i]->K);
                    g.max_row = std::max(g.max_row, b->P[i]->max_row);
                }
            if (g.probs.empty()) {
                b->sgroups.pop_back();
                continue;
            }
            g.totalK = koff.back();
            if ((s = nl_alloc(ctx, &g.dS, sa.size())) != NL_OK || (s = nl_alloc(ctx, &g.dkoff, koff.size())) != NL_OK)
                return fail(s);
            if (cudaMemcpyAsync(g.dS, sa.data(), sizeof(ScatterArgs) * sa.size(), cudaMemcpyHostToDevice, st) !=
                    cudaSuccess ||
                cudaMemcpyAsync(g.dkoff, koff.data(), sizeof(int64_t) * koff.size(), cudaMemcpyHostToDevice, st) !=
                    cudaSuccess)
                return fail(nl_fail(ctx, NL_ECUDA, "upload of the scatter arguments"));
        }
    }
    if ((s = phase_check(ctx, b, "scatter arguments")) != NL_OK) return fail(s);
    if ((s = launch_scatter(ctx, b, true)) != NL_OK || (s = phase_check(ctx, b, "scatter")) != NL_OK) return fail(s);
    if (cudaEventRecord(ctx->ev[4], st) != cudaSuccess) return fail(nl_fail(ctx, NL_ECUDA, "cudaEventRecord"));
    // ---- the re-assembly graph: numeric phase + scatter of every problem ----
    {
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return fail(nl_cuda_fail(ctx, e, "cudaStreamBeginCapture"));
        const int64_t l0 = ctx->launches;
        nl_status s1, s2;
        if (b->sched.mode == 1) {   // each problem's numeric phase and scatter on its stream
            s1 = launch_numeric_streams(ctx, b, b->sched, true);
            s2 = s1;
        } else {
            s1 = launch_numeric(ctx, b, false);
            s2 = s1 == NL_OK ? launch_scatter(ctx, b, false) : s1;
        }
        // captured, not launched: nl_batch_run counts them per replay
        b->graph_kernels = ctx->launches - l0;
        ctx->launches = l0;
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(st, &g);
        if (s2 != NL_OK) {
            if (g) cudaGraphDestroy(g);
            return fail(s2);
        }
        if (e != cudaSuccess) return fail(nl_cuda_fail(ctx, e, "cudaStreamEndCapture"));
        b->graph = g;
        e = cudaGraphInstantiate(&b->exec, g, 0);
        if (e != cudaSuccess) return fail(nl_cuda_fail(ctx, e, "cudaGraphInstantiate"));
    }
    for (int i = 0; i < n; i++) {
        nl_prep_delete(T[i], st);
        nl_pat_delete(Q[i], st);
    }
    T.assign(n, nullptr);
    Q.assign(n, nullptr);
    if ((s = phase_check(ctx, b, "release of the temporaries")) != NL_OK) return fail(s);
    *batch = b;
    return NL_OK;
}

nl_status nl_batch_run(nl_ctx *ctx, nl_batch *b)
{
    if (!ctx) return NL_EINVAL;
    if (!b || !b->exec) return nl_fail(ctx, NL_EINVAL, "not an nl_batch_create handle");
    NL_CK(cudaGraphLaunch(b->exec, ctx->stream));
    ctx->launches += b->graph_kernels;
    return NL_OK;
}

nl_status nl_batch_get_info(const nl_batch *b, nl_batch_info *info)
{
    if (!b || !info) return NL_EINVAL;
    *info = b->info;
    return NL_OK;
}

void nl_batch_destroy(nl_ctx *ctx, nl_batch *b)
{
    if (!b) return;
    cudaStream_t st = ctx ? ctx->stream : nullptr;
    if (st) cudaStreamSynchronize(st);
    release(b, st);
    delete b;
}

nl_status nl_assemble_batch(nl_ctx *ctx, int32_t n, const nl_mesh *meshes, const nl_config *cfgs, nl_csr *outs)
{
    if (!ctx) return NL_EINVAL;
    if (n < 1 || !meshes || !cfgs || !outs) return nl_fail(ctx, NL_EINVAL, "need n >= 1 and non-null arrays");
    nl_status s;
    for (int i = 0; i < n; i++) {
        if ((s = nl_validate(ctx, &meshes[i], &cfgs[i])) != NL_OK) {
            ctx->err = "problem " + std::to_string(i) + ": " + ctx->err;
            return s;
        }
    }
    NL_CK(cudaSetDevice(ctx->device));
    for (int i = 0; i < n; i++) memset(&outs[i], 0, sizeof outs[i]);
    return assemble_pipelined(ctx, n, meshes, cfgs, outs);
}

}  // extern "C"
