// api.cu -- C ABI entry points of libnlfem (declared in include/nlfem.h).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <new>
#include <string>

#include "numeric.cuh"


// ---------------------------------------------------------------------------
// errors and staging
// ---------------------------------------------------------------------------
nl_status nl_fail(nl_ctx *ctx, nl_status s, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return s;
}

nl_status nl_cuda_fail(nl_ctx *ctx, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return nl_fail(ctx, e == cudaErrorMemoryAllocation ? NL_ENOMEM : NL_ECUDA, m);
}

bool nl_is_device_ptr(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int nl_ptr_kind(const void *p, int device)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return NL_PTR_HOST;
    }
    if (at.type == cudaMemoryTypeManaged) return NL_PTR_DEVICE;
    if (at.type == cudaMemoryTypeDevice) return at.device == device ? NL_PTR_DEVICE : NL_PTR_OTHER;
    return NL_PTR_HOST;
}

// device view of a host-or-device input; *owned says whether the caller must free it
nl_status nl_stage(nl_ctx *ctx, const void *src, size_t bytes, void **dev, bool *owned)
{
    *owned = false;
    const int kind = nl_ptr_kind(src, ctx->device);
    if (kind == NL_PTR_OTHER) return nl_fail(ctx, NL_EINVAL, "an input lives on another device than the context's");
    if (kind == NL_PTR_DEVICE) {
        *dev = const_cast<void *>(src);
        return NL_OK;
    }
    NL_CK(cudaMallocAsync(dev, bytes ? bytes : 1, ctx->stream));
    NL_CK(cudaMemcpyAsync(*dev, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
    *owned = true;
    return NL_OK;
}

// ---------------------------------------------------------------------------
// quadrature tables (the kernel side's own construction of the published rules)
// ---------------------------------------------------------------------------
namespace {

struct TabBuilder {
    nlq::RuleTab *t;
    void pt(double l0, double l1, double l2, double w)
    {
        t->l[t->n][0] = l0;
        t->l[t->n][1] = l1;
        t->l[t->n][2] = l2;
        t->w[t->n] = w;
        t->n++;
    }
    void s3(double w) { pt(1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0, w); }
    void s21(double a, double w)
    {
        const double c = 1.0 - 2.0 * a;
        pt(a, a, c, w); pt(a, c, a, w); pt(c, a, a, w);
    }
    void s111(double a, double b, double w)
    {
        const double c = 1.0 - a - b;
        pt(a, b, c, w); pt(a, c, b, w); pt(b, a, c, w);
        pt(b, c, a, w); pt(c, a, b, w); pt(c, b, a, w);
    }
};

bool fill_rule(int id, nlq::RuleTab *t)
{
    TabBuilder B{t};
    switch (id) {
    case NL_RULE_GAUSS3:   // symmetric 3-point Gaussian rule, degree 2
        B.s21(1.0 / 6.0, 1.0 / 3.0);
        return true;
    case NL_RULE_GAUSS4:   // symmetric 4-point Gaussian rule, degree 3
        B.s3(-27.0 / 48.0);
        B.s21(0.2, 25.0 / 48.0);
        return true;
    case NL_RULE_PAPER7:   // centroid 27/60, vertices 3/60, mid-sides 8/60 (Sec. 6.3)
        B.s3(27.0 / 60.0);
        B.pt(1.0, 0.0, 0.0, 3.0 / 60.0);
        B.pt(0.0, 1.0, 0.0, 3.0 / 60.0);
        B.pt(0.0, 0.0, 1.0, 3.0 / 60.0);
        B.pt(0.5, 0.5, 0.0, 8.0 / 60.0);
        B.pt(0.0, 0.5, 0.5, 8.0 / 60.0);
        B.pt(0.5, 0.0, 0.5, 8.0 / 60.0);
        return true;
    case NL_RULE_DUNAVANT7: {   // Radon's 7-point degree-5 rule
        const double r = sqrt(15.0);
        B.s3(9.0 / 40.0);
        B.s21((6.0 - r) / 21.0, (155.0 - r) / 1200.0);
        B.s21((6.0 + r) / 21.0, (155.0 + r) / 1200.0);
        return true;
    }
    case NL_RULE_DUNAVANT16:   // Dunavant's 16-point degree-8 rule
        B.s3(0.1443156076777871682510911);
        B.s21(0.4592925882927231560288155, 0.0950916342672846247938961);
        B.s21(0.1705693077517602066222935, 0.1032173705347182502817916);
        B.s21(0.05054722831703097545842355, 0.03245849762319808031092593);
        B.s111(0.008394777409957605337213835, 0.2631128296346381134217858, 0.02723031417443499426484469);
        return true;
    default:
        return false;
    }
}

// Gauss-Legendre nodes and weights on [0, 1] (Newton on the Legendre recurrence)
void gauss_legendre01(int n, double *x, double *w)
{
    for (int i = 0; i < n; i++) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 60; it++) {
            double p = 1.0, pm = 0.0;
            for (int k = 1; k <= n; k++) {
                double pk = ((2.0 * k - 1.0) * z * p - (k - 1.0) * pm) / k;
                pm = p;
                p = pk;
            }
            dp = n * (z * p - pm) / (z * z - 1.0);
            double step = p / dp;
            z -= step;
            if (fabs(step) < 1e-17) break;
        }
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
}

}  // namespace

nl_status nl_validate(nl_ctx *ctx, const nl_mesh *m, const nl_config *c)
{
    if (!ctx) return NL_EINVAL;
    if (!m || !c) return nl_fail(ctx, NL_EINVAL, "null mesh or config");
    if (m->nv <= 0 || m->nt <= 0 || !m->vx || !m->vy || !m->tri)
        return nl_fail(ctx, NL_EINVAL, "mesh needs nv > 0, nt > 0 and vx, vy, tri");
    if (!(c->delta > 0.0) || !isfinite(c->delta)) return nl_fail(ctx, NL_EINVAL, "delta must be positive");
    if (c->ball < NL_BALL_BARYCENTER || c->ball > NL_BALL_BARY_APPROXCAPS) return nl_fail(ctx, NL_EINVAL, "bad ball");
    if (c->kernel != NL_KERNEL_CONST && c->kernel != NL_KERNEL_INV_DIST) return nl_fail(ctx, NL_EINVAL, "bad kernel");
    if (c->prec != NL_PREC_FP64 && c->prec != NL_PREC_FP32_COMP) return nl_fail(ctx, NL_EINVAL, "bad precision");
    if (c->inner < NL_RULE_GAUSS3 || c->inner > NL_RULE_DUNAVANT16) return nl_fail(ctx, NL_EINVAL, "bad inner rule");
    if (c->outer < NL_RULE_GAUSS3 || c->outer > NL_RULE_SWITCH47) return nl_fail(ctx, NL_EINVAL, "bad outer rule");
    if (c->ball == NL_BALL_NGON && (c->ngon_n < 3 || c->ngon_n > 64 || !c->ngon_offsets))
        return nl_fail(ctx, NL_EINVAL, "ngon needs 3 <= ngon_n <= 64 and ngon_offsets");
    if ((c->ball == NL_BALL_APPROXCAPS || c->ball == NL_BALL_BARY_APPROXCAPS) &&
        (c->cap_m < 1 || c->cap_m > 16 || (c->cap_m & (c->cap_m - 1)) != 0))
        return nl_fail(ctx, NL_EINVAL, "cap_m must be a power of two in 1..16");
    if (c->kernel == NL_KERNEL_INV_DIST && (c->duffy_n < 1 || c->duffy_n > 7))
        return nl_fail(ctx, NL_EINVAL, "duffy_n must be in 1..7");
    if (c->shifted != 0 && c->shifted != 1) return nl_fail(ctx, NL_EINVAL, "shifted must be 0 or 1");
    if (c->shifted && c->kernel != NL_KERNEL_CONST)
        return nl_fail(ctx, NL_EUNSUPPORTED, "the shifted-centre ball is defined for the constant kernel");
    if ((c->ball == NL_BALL_BARY_NOCAPS || c->ball == NL_BALL_BARY_APPROXCAPS) &&
        (c->kernel != NL_KERNEL_CONST || c->shifted))
        return nl_fail(ctx, NL_EUNSUPPORTED, "the outer-support barycenter balls take the constant kernel, unshifted");
    return NL_OK;
}

// Bound on the sum over all T_b of s0(x, T_b) = int_{region(x) cap T_b} gamma(x, y) dy at any
// outer point x: every region of x lies in B(x, delta + h_max) (the shifted, barycenter and
// overlap balls included), so the sum is at most kc pi (delta + h_max)^2 for a constant kernel
// and c 2 pi (delta + h_max) for c / |x - y| (the integral of 1/r over the disc); here with a
// margin of 1.25 (twice that for the singular kernel's quadrature).
static double s0_sum_bound(const nl_config &c, double hmax)
{
    const double r = c.delta + hmax, pi = 3.14159265358979323846;
    return c.kernel == NL_KERNEL_INV_DIST ? 2.5 * fabs(c.kernel_c) * 2.0 * pi * r
                                          : 1.25 * fabs(c.kernel_c) * pi * r * r;
}

static double abs_weight_sum(int rule)
{
    nlq::RuleTab t;
    memset(&t, 0, sizeof t);
    if (!fill_rule(rule, &t)) return 0.0;   // unreachable: the rule was checked when the plan was made
    double ws = 0.0;
    for (int q = 0; q < t.n; q++) ws += fabs(t.w[q]);
    return ws;
}

float nl_outer_abs_weight(const nl_plan *P)
{
    // the switching rule integrates each pair with one of its two rules
    if (P->cfg.outer == NL_RULE_SWITCH47)
        return (float)fmax(abs_weight_sum(NL_RULE_GAUSS4), abs_weight_sum(NL_RULE_PAPER7));
    return (float)abs_weight_sum(P->cfg.outer);
}

nl_status nl_fill_args(nl_ctx *ctx, const nl_plan *P, nlq::NumArgs &A, bool stats)
{
    memset(&A, 0, sizeof A);
    const nl_config &c = P->cfg;
    A.K = P->K;
    A.E = P->E;
    A.tx = P->tx;
    A.ty = P->ty;
    A.bx = P->bx;
    A.by = P->by;
    A.area = P->area;
    A.akc = P->akc;
    A.hl = P->hl;
    A.nbr_ptr = P->nbr_ptr;
    A.nbr_split = P->nbr_split;
    A.nbr_idx = P->nbr_idx;
    if (c.outer == NL_RULE_SWITCH47) {
        fill_rule(NL_RULE_GAUSS4, &A.outer);
        A.outer.nsplit = A.outer.n;
        fill_rule(NL_RULE_PAPER7, &A.outer);
        A.switch47 = 1;
        double thr = c.delta - P->hmax;
        A.thr2 = thr > 0.0 ? thr * thr : -1.0;
    } else {
        if (!fill_rule(c.outer, &A.outer)) return nl_fail(ctx, NL_EINVAL, "bad outer rule");
        A.outer.nsplit = A.outer.n;
    }
    if (!fill_rule(c.inner, &A.inner)) return nl_fail(ctx, NL_EINVAL, "bad inner rule");
    if (A.outer.n > NL_MAXQ || A.inner.n > NL_MAXQ)
        return nl_fail(ctx, NL_EUNSUPPORTED, "rules of more than NL_MAXQ points");   // the kernels' stage sizes
    A.inner.nsplit = A.inner.n;
    A.duffy_n = c.kernel == NL_KERNEL_INV_DIST ? c.duffy_n : 1;
    gauss_legendre01(A.duffy_n, A.gl_x, A.gl_w);
    gauss_legendre01(2, A.gl2_x, A.gl2_w);
    for (int j = 0; j < 8; j++) {
        A.glf_x[j] = j < A.duffy_n ? (float)A.gl_x[j] : 0.f;
        A.glf_w[j] = j < A.duffy_n ? (float)A.gl_w[j] : 0.f;
        A.glf_sh[j] = j < A.duffy_n ? (float)sinh(A.gl_x[j]) : 0.f;
        A.glf_ch[j] = j < A.duffy_n ? (float)cosh(A.gl_x[j]) : 1.f;
    }
    A.sh1f = (float)sinh(1.0);
    A.ch1f = (float)cosh(1.0);
    for (int j = 0; j < 2; j++) {
        A.gl2f_x[j] = (float)A.gl2_x[j];
        A.gl2f_w[j] = (float)A.gl2_w[j];
    }
    A.kernel = c.kernel;
    A.ball = c.ball;
    A.shifted = c.shifted ? 1 : 0;
    A.outer_support = (c.ball == NL_BALL_BARY_NOCAPS || c.ball == NL_BALL_BARY_APPROXCAPS) ? 1 : 0;
    A.kc = c.kernel_c;
    A.kcf = (float)c.kernel_c;
    {
        // grid of the boundary kernel's fixed-point sums of s0 per outer point: the bound,
        // rounded up to a power of two 2^e, maps to 2^30
        const double bound = s0_sum_bound(c, P->hmax);
        int e = 0;
        frexp(bound > 1e-30 ? bound : 1e-30, &e);   // bound < 2^e
        A.s0q_grid = (float)ldexp(1.0, 30 - e);
    }
    A.geo.delta = c.delta;
    A.geo.deltaf = (float)c.delta;
    A.geo.d2 = P->d2;
    A.geo.ngon = P->ngon;
    A.geo.ngon_n = c.ball == NL_BALL_NGON ? c.ngon_n : 0;
    int level = 0;
    while ((1 << level) < (c.cap_m > 0 ? c.cap_m : 1)) level++;
    A.geo.cap_level = level;
    A.geo.cap_printed = c.cap_printed;
    // FP32 certification data (see geometry.cuh): margin tau = 1e-5 delta
    const double tau = 1e-5 * c.delta;
    double rin = c.delta, rout = c.delta;
    if (c.ball == NL_BALL_NGON) {
        const int N = c.ngon_n;
        const double *o = P->ngon_host.data();
        rin = INFINITY;
        rout = 0.0;
        for (int k = 0; k < N; k++) {
            const int k1 = (k + 1) % N;
            const double ex = o[2 * k1] - o[2 * k], ey = o[2 * k1 + 1] - o[2 * k + 1];
            const double el = sqrt(ex * ex + ey * ey);
            // distance from the centre to the line of edge k (polygon ccw around the centre)
            const double dk = (o[2 * k] * o[2 * k1 + 1] - o[2 * k + 1] * o[2 * k1]) / (el > 0.0 ? el : 1.0);
            rin = fmin(rin, dk);
            rout = fmax(rout, sqrt(o[2 * k] * o[2 * k] + o[2 * k + 1] * o[2 * k + 1]));
            A.geo.of[k][0] = (float)o[2 * k];
            A.geo.of[k][1] = (float)o[2 * k + 1];
            A.geo.ef[k][0] = (float)ex;
            A.geo.ef[k][1] = (float)ey;
            A.geo.mk[k] = (float)(el * tau);
        }
    }
    A.geo.tau = (float)tau;
    A.geo.inv_tau = (float)(1.0 / tau);
    if (c.ball == NL_BALL_NGON) {
        // regular polygon R (cos 2 pi k / N, sin 2 pi k / N)?  (enables the angular pass window)
        const int N = c.ngon_n;
        const double *o = P->ngon_host.data();
        const double R = sqrt(o[0] * o[0] + o[1] * o[1]);
        bool reg = R > 0.0;
        for (int k = 0; k < N && reg; k++) {
            const double th = 2.0 * M_PI * k / N;
            reg = fabs(o[2 * k] - R * cos(th)) <= 1e-12 * R && fabs(o[2 * k + 1] - R * sin(th)) <= 1e-12 * R;
        }
        A.geo.regular = reg ? 1 : 0;
        double m1 = 0.0;
        for (int k = 0; k < N; k++) m1 = fmax(m1, fabs(o[2 * k]) + fabs(o[2 * k + 1]));
        A.geo.r2 = (float)(2.0 * m1);
        A.geo.o1max = (float)m1;
        A.geo.sector = (float)(2.0 * M_PI / N);
        A.geo.rin_tau = (float)(rin - tau);
    }
    // FP32 local coordinates d = v - x: (v - bary_a) from FP32 hi + lo pairs (within 2u |v - bary_a|,
    // |v - bary_a| <= delta + 3 r_max), minus (x - bary_a) rounded from FP64 (within u r_max), rounded
    // (u |d|, |d| <= delta + 4 r_max): in all u (3 delta + 11 r_max) <= 4u (delta + 4 r_max)
    A.geo.err0 = (float)(4.0 * 5.9604644775390625e-8 * (c.delta + 4.0 * P->rmax));
    A.geo.rin_m2 = rin - tau > 0.0 ? (float)((rin - tau) * (rin - tau)) : -1.0f;
    A.geo.rout_p2 = (float)((rout + tau) * (rout + tau));
    A.geo.b_in2 = (float)((c.delta - tau) * (c.delta - tau));
    A.geo.b_out2 = (float)((c.delta + tau) * (c.delta + tau));
    for (int r = 0; r < A.inner.n; r++) {
        A.fin[r] = make_float4((float)A.inner.l[r][0], (float)A.inner.l[r][1], (float)A.inner.l[r][2],
                               (float)A.inner.w[r]);
    for (int q = 0; q < A.outer.n; q++)
        A.fout[q] = make_float4((float)A.outer.l[q][0], (float)A.outer.l[q][1], (float)A.outer.l[q][2],
                                (float)A.outer.w[q]);
    }
    A.flag = P->flag;
    A.blk = P->blk;
    A.mbb = P->mbb;
    A.maa = P->maa;
    A.qp_a = P->qp_a;
    A.cnt_a = P->cnt_a;
    A.hash_a = P->hash_a;
    A.stats = stats ? 1 : 0;
    A.err = P->err;
    A.defer = nullptr;
    A.dval = nullptr;
    A.defer_n = nullptr;
    A.defer_cap = 0;
    A.prob = 0;
    return NL_OK;
}

nl_status nl_alloc_numeric(nl_ctx *ctx, nl_plan *P)
{
    nl_status s;
    const size_t tsz = P->cfg.prec == NL_PREC_FP64 ? sizeof(double) : sizeof(float);
    if ((s = nl_alloc(ctx, &P->flag, (size_t)P->E)) != NL_OK) return s;
    unsigned char *blk = nullptr;
    if ((s = nl_alloc(ctx, &blk, tsz * 9 * (size_t)(P->E ? P->E : 1))) != NL_OK) return s;
    P->blk = blk;
    if ((s = nl_alloc(ctx, &P->mbb, 6 * (size_t)P->K)) != NL_OK) return s;
    if ((s = nl_alloc(ctx, &P->maa, 6 * (size_t)P->K)) != NL_OK) return s;
    if ((s = nl_alloc(ctx, &P->qp_a, (size_t)P->K)) != NL_OK) return s;
    if ((s = nl_alloc(ctx, &P->cnt_a, (size_t)P->K)) != NL_OK) return s;
    if ((s = nl_alloc(ctx, &P->hash_a, (size_t)P->K)) != NL_OK) return s;
    if ((s = nl_alloc(ctx, &P->err, 1)) != NL_OK) return s;
    NL_CK(cudaMemsetAsync(P->err, 0, sizeof(int), ctx->stream));
    return NL_OK;
}

namespace {

nl_status run_numeric(nl_ctx *ctx, nl_plan *P, bool stats, bool one_stream = false)
{
    nlq::NumArgs A;
    nl_status s = nl_fill_args(ctx, P, A, stats);
    if (s != NL_OK) return s;
    if (P->cfg.prec == NL_PREC_FP64) return nl_launch_numeric_f64(ctx, A, P->cfg.ball, one_stream);
    if (!P->defer) {
        const int cap = nl_defer_cap(P->E) > P->defer_min ? nl_defer_cap(P->E) : P->defer_min;
        nlq::DeferItem *q = nullptr;
        if ((s = nl_alloc(ctx, &q, nlq::defer_alloc_items(cap))) != NL_OK) return s;
        P->defer = q;
        if ((s = nl_alloc(ctx, &P->defer_n, 1)) != NL_OK) return s;
        P->defer_cap = cap;
    }
    A.defer = (nlq::DeferItem *)P->defer;
    A.dval = nlq::defer_values(A.defer, P->defer_cap);
    A.defer_n = P->defer_n;
    A.defer_cap = P->defer_cap;
    if (P->cfg.kernel == NL_KERNEL_INV_DIST) {
        if (!P->near_n) {
            const int cap = nl_near_cap(P->E) > P->near_min ? nl_near_cap(P->E) : P->near_min;
            nlq::DeferItem *q = nullptr;
            if (cap > 0 && (s = nl_alloc(ctx, &q, (size_t)cap)) != NL_OK) return s;
            P->nearq = q;
            nlq::OuterPt *ot = nullptr;
            if (cap > 0 && (s = nl_alloc(ctx, &ot, (size_t)P->K * A.outer.n)) != NL_OK) return s;
            P->otab = ot;
            if ((s = nl_alloc(ctx, &P->near_n, 1)) != NL_OK) return s;
            P->near_cap = cap;
        }
        if (P->near_cap > 0) {
            A.nearq = (nlq::DeferItem *)P->nearq;
            A.near_n = P->near_n;
            A.near_cap = P->near_cap;
            A.otab = (nlq::OuterPt *)P->otab;
        }
    }
    return nl_launch_numeric_f32(ctx, A, P->cfg.ball, one_stream);
}

}  // namespace

nl_status nl_run_numeric_one_stream(nl_ctx *ctx, nl_plan *P) { return run_numeric(ctx, P, false, true); }

// The steps of one assembly after the candidate count is known (stage C of the preparation):
// candidate lists, numeric phase, symbolic stage A; the counts of the queued items and the
// pattern size go to the host slot.  ev_num / ev_sym (may be null): recorded before and after
// the numeric phase.  one_stream: every numeric kernel on ctx->stream (the batch's problems).
nl_status nl_assemble_step_c(nl_ctx *ctx, nl_plan *P, nl_prep *T, nl_pat *Q, nl_host_slot *h, nl_csr *out,
                             bool one_stream, cudaEvent_t ev_num, cudaEvent_t ev_sym)
{
    nl_status s;
    if ((s = nl_prepare_c(ctx, P, T, h)) != NL_OK) return s;
    if ((s = nl_alloc_numeric(ctx, P)) != NL_OK) return s;
    if (ev_num) NL_CK(cudaEventRecord(ev_num, ctx->stream));
    if ((s = run_numeric(ctx, P, false, one_stream)) != NL_OK) return s;
    if (ev_sym) NL_CK(cudaEventRecord(ev_sym, ctx->stream));
    h->deferred = 0;
    h->near = 0;
    if (P->defer_n) NL_CK(cudaMemcpyAsync(&h->deferred, P->defer_n, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    if (P->near_n) NL_CK(cudaMemcpyAsync(&h->near, P->near_n, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    return nl_pattern_a(ctx, P, out, Q, h);
}

// The last steps, once the slot of step C has arrived: checks, a second numeric run if a queue
// overflowed, symbolic stage B and the scatter.  ev_sct (may be null): recorded before the scatter.
nl_status nl_assemble_step_d(nl_ctx *ctx, nl_plan *P, nl_pat *Q, const nl_host_slot *h, nl_csr *out,
                             bool one_stream, cudaEvent_t ev_sct)
{
    nl_status s;
    if ((s = nl_prepare_check(ctx, h)) != NL_OK) return s;
    // A full queue of FP64-decided or near-field items leaves the excess to the boundary
    // kernel's lanes, and which items those are depends on the scheduling.  Queues that hold
    // them all (kept for every re-assembly of this plan) make the values independent of it.
    const bool dfull = P->defer && h->deferred > P->defer_cap && !nl_defer_cap_fixed();
    const bool nfull = P->near_n && P->near_cap > 0 && h->near > P->near_cap && !nl_near_cap_fixed();
    if (dfull) {
        const int64_t want = (int64_t)h->deferred + h->deferred / 4;
        P->defer_min = (int)(want > (int64_t(1) << 24) ? (int64_t(1) << 24) : want);
        nl_free(P->defer, ctx->stream);
        nl_free(P->defer_n, ctx->stream);
    }
    if (nfull) {
        const int64_t want = (int64_t)h->near + h->near / 4;
        P->near_min = (int)(want > (int64_t(1) << 30) ? (int64_t(1) << 30) : want);
        nl_free(P->nearq, ctx->stream);
        nl_free(P->otab, ctx->stream);
        nl_free(P->near_n, ctx->stream);
    }
    if ((dfull || nfull) && (s = run_numeric(ctx, P, false, one_stream)) != NL_OK) return s;
    if ((s = nl_pattern_b(ctx, P, out, Q, h)) != NL_OK) return s;
    if (ev_sct) NL_CK(cudaEventRecord(ev_sct, ctx->stream));
    return nl_run_scatter(ctx, P, out);
}

void nl_plan_free(nl_plan *P, cudaStream_t s)
{
    if (!P) return;
    nl_free(P->tri, s); nl_free(P->tx, s); nl_free(P->ty, s); nl_free(P->bx, s); nl_free(P->by, s);
    nl_free(P->rad, s); nl_free(P->area, s); nl_free(P->akc, s); nl_free(P->hl, s); nl_free(P->ngon, s); nl_free(P->nbr_ptr, s); nl_free(P->nbr_idx, s);
    nl_free(P->nbr_split, s); nl_free(P->flag, s); nl_free(P->blk, s); nl_free(P->maa, s); nl_free(P->qp_a, s);
    nl_free(P->cnt_a, s); nl_free(P->hash_a, s); nl_free(P->lslot, s); nl_free(P->mbb, s); nl_free(P->tslot, s); nl_free(P->W, s);
    nl_free(P->val32, s); nl_free(P->x32, s); nl_free(P->err, s); nl_free(P->defer, s); nl_free(P->defer_n, s);
    nl_free(P->nearq, s); nl_free(P->near_n, s); nl_free(P->otab, s); nl_free(P->fxe, s);
}

nl_status nl_host_slots(nl_ctx *ctx, int n, nl_host_slot **out)
{
    if (n < 1) n = 1;
    if (ctx->nslots < n) {
        // the stream may still be copying into the old slots
        NL_CK(cudaStreamSynchronize(ctx->stream));
        if (ctx->slots) cudaFreeHost(ctx->slots);
        ctx->slots = nullptr;
        ctx->nslots = 0;
        const int cap = n < 64 ? 64 : n;
        cudaError_t e = cudaMallocHost((void **)&ctx->slots, sizeof(nl_host_slot) * (size_t)cap);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ctx->slots = nullptr;
            return nl_fail(ctx, NL_ENOMEM, "pinned host allocation failed");
        }
        ctx->nslots = cap;
    }
    memset(ctx->slots, 0, sizeof(nl_host_slot) * (size_t)n);
    *out = ctx->slots;
    return NL_OK;
}

// ---------------------------------------------------------------------------
// entry points
// ---------------------------------------------------------------------------
nl_status nl_side_streams(nl_ctx *ctx)
{
    for (int k = 0; k < nl_ctx::kSideStreams; k++)
        if (!ctx->side[k]) NL_CK(cudaStreamCreateWithFlags(&ctx->side[k], cudaStreamNonBlocking));
    for (int k = 0; k <= nl_ctx::kSideStreams; k++)
        if (!ctx->side_ev[k]) NL_CK(cudaEventCreateWithFlags(&ctx->side_ev[k], cudaEventDisableTiming));
    return NL_OK;
}

extern "C" {

nl_status nl_create(nl_ctx **out, int device, void *stream)
{
    if (!out) return NL_EINVAL;
    *out = nullptr;
    nl_ctx *ctx = new (std::nothrow) nl_ctx();
    if (!ctx) return NL_ENOMEM;
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess && stream) {
        ctx->stream = (cudaStream_t)stream;
    } else if (e == cudaSuccess) {
        e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        ctx->own_stream = (e == cudaSuccess);
    }
    for (int i = 0; e == cudaSuccess && i < 5; i++) e = cudaEventCreate(&ctx->ev[i]);
    // the side streams (the numeric phase's interior launch, the batch's stages) exist from the
    // start, so that no stream or event is created while the caller captures a graph
    for (int k = 0; e == cudaSuccess && k < nl_ctx::kSideStreams; k++)
        e = cudaStreamCreateWithFlags(&ctx->side[k], cudaStreamNonBlocking);
    for (int k = 0; e == cudaSuccess && k <= nl_ctx::kSideStreams; k++)
        e = cudaEventCreateWithFlags(&ctx->side_ev[k], cudaEventDisableTiming);
    if (e == cudaSuccess) {
        // keep freed pool memory cached by this process (up to 8 GiB) instead of handing it
        // back to the driver at every synchronisation: later assemblies allocate without
        // driver calls.  This is a property of the process's pool, not of the device.
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
            uint64_t thr = 0;
            if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr) == cudaSuccess &&
                thr < (uint64_t(8) << 30)) {
                thr = uint64_t(8) << 30;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
            }
        }
        cudaGetLastError();
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        nl_destroy(ctx);
        return NL_ECUDA;
    }
    *out = ctx;
    return NL_OK;
}

void nl_destroy(nl_ctx *ctx)
{
    if (!ctx) return;
    for (int i = 0; i < 5; i++)
        if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (int k = 0; k < nl_ctx::kSideStreams; k++)
        if (ctx->side[k]) {
            cudaStreamSynchronize(ctx->side[k]);
            cudaStreamDestroy(ctx->side[k]);
        }
    for (int k = 0; k <= nl_ctx::kSideStreams; k++)
        if (ctx->side_ev[k]) cudaEventDestroy(ctx->side_ev[k]);
    if (ctx->slots) cudaFreeHost(ctx->slots);
    nl_tune_cache_free(ctx->tune);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char *nl_last_error(nl_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t nl_last_fp64_items(nl_ctx *ctx) { return ctx ? ctx->last_fp64_items : -1; }

nl_status nl_assemble(nl_ctx *ctx, const nl_mesh *mesh, const nl_config *cfg, nl_csr *out)
{
    nl_status s = nl_validate(ctx, mesh, cfg);
    if (s != NL_OK) return s;
    if (!out) return nl_fail(ctx, NL_EINVAL, "null output");
    memset(out, 0, sizeof *out);
    NL_CK(cudaSetDevice(ctx->device));
    nl_plan *P = new (std::nothrow) nl_plan();
    if (!P) return nl_fail(ctx, NL_ENOMEM, "host allocation failed");
    out->priv = P;
    nl_host_slot *h = nullptr;
    nl_prep *T = nullptr;
    nl_pat *Q = nullptr;
    cudaError_t e;
    if ((s = nl_host_slots(ctx, 1, &h)) != NL_OK) goto fail;
    T = nl_prep_new();
    Q = nl_pat_new();
    if (!T || !Q) {
        s = nl_fail(ctx, NL_ENOMEM, "host allocation failed");
        goto fail;
    }
    // three host synchronisations: candidate-search grid, candidate count, pattern size
    if ((e = cudaEventRecord(ctx->ev[0], ctx->stream)) != cudaSuccess) goto cuda_fail;
    if ((s = nl_prepare_a(ctx, mesh, cfg, P, T, h)) != NL_OK) goto fail;
    if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) goto cuda_fail;
    if ((s = nl_prepare_b(ctx, P, T, h)) != NL_OK) goto fail;
    if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) goto cuda_fail;
    if ((s = nl_assemble_step_c(ctx, P, T, Q, h, out, false, ctx->ev[1], ctx->ev[2])) != NL_OK) goto fail;
    if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) goto cuda_fail;
    ctx->last_fp64_items = h->deferred;
    if ((s = nl_assemble_step_d(ctx, P, Q, h, out, false, ctx->ev[3])) != NL_OK) goto fail;
    if ((e = cudaEventRecord(ctx->ev[4], ctx->stream)) != cudaSuccess) goto cuda_fail;
    nl_prep_delete(T, ctx->stream);
    nl_pat_delete(Q, ctx->stream);
    return NL_OK;
cuda_fail:
    s = nl_cuda_fail(ctx, e, "stream operation");
fail:
    nl_prep_delete(T, ctx->stream);
    nl_pat_delete(Q, ctx->stream);
    nl_csr_free(ctx, out);
    return s;
}

nl_status nl_assemble_numeric(nl_ctx *ctx, nl_csr *m)
{
    if (!ctx) return NL_EINVAL;
    if (!m || !m->priv) return nl_fail(ctx, NL_EINVAL, "not an nl_assemble result");
    nl_plan *P = (nl_plan *)m->priv;
    if (!P->blk) return nl_fail(ctx, NL_EINVAL, "not an nl_assemble result");
    nl_status s;
    if ((s = run_numeric(ctx, P, false)) != NL_OK) return s;
    return nl_run_scatter(ctx, P, m);
}

nl_status nl_interactions(nl_ctx *ctx, const nl_mesh *mesh, const nl_config *cfg, uint64_t *hash_a,
                          int64_t *count_a, int64_t *qp_a)
{
    nl_status s = nl_validate(ctx, mesh, cfg);
    if (s != NL_OK) return s;
    NL_CK(cudaSetDevice(ctx->device));
    nl_plan P;
    if ((s = nl_prepare_mesh(ctx, mesh, cfg, &P)) == NL_OK && (s = nl_alloc_numeric(ctx, &P)) == NL_OK &&
        (s = run_numeric(ctx, &P, true)) == NL_OK) {
        cudaError_t e = cudaSuccess;
        if (hash_a && e == cudaSuccess)
            e = cudaMemcpyAsync(hash_a, P.hash_a, sizeof(uint64_t) * P.K, cudaMemcpyDeviceToHost, ctx->stream);
        if (count_a && e == cudaSuccess)
            e = cudaMemcpyAsync(count_a, P.cnt_a, sizeof(int64_t) * P.K, cudaMemcpyDeviceToHost, ctx->stream);
        if (qp_a && e == cudaSuccess)
            e = cudaMemcpyAsync(qp_a, P.qp_a, sizeof(int64_t) * P.K, cudaMemcpyDeviceToHost, ctx->stream);
        int deferred = 0;
        if (P.defer_n && e == cudaSuccess)
            e = cudaMemcpyAsync(&deferred, P.defer_n, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        ctx->last_fp64_items = deferred;
        if (e != cudaSuccess) s = nl_cuda_fail(ctx, e, "download of interaction statistics");
    }
    nl_plan_free(&P, ctx->stream);
    return s;
}

nl_status nl_csr_download(nl_ctx *ctx, const nl_csr *m, int64_t *row_ptr, int32_t *col_idx, double *val)
{
    if (!ctx) return NL_EINVAL;
    if (!m) return nl_fail(ctx, NL_EINVAL, "null matrix");
    if (row_ptr)
        NL_CK(cudaMemcpyAsync(row_ptr, m->row_ptr, sizeof(int64_t) * (m->n + 1), cudaMemcpyDeviceToHost, ctx->stream));
    if (col_idx && m->nnz)
        NL_CK(cudaMemcpyAsync(col_idx, m->col_idx, sizeof(int32_t) * m->nnz, cudaMemcpyDeviceToHost, ctx->stream));
    if (val && m->nnz)
        NL_CK(cudaMemcpyAsync(val, m->val, sizeof(double) * m->nnz, cudaMemcpyDeviceToHost, ctx->stream));
    // the error word of the last numeric phase and scatter, which ran after nl_assemble's last
    // host synchronisation (or in nl_assemble_numeric / nl_batch_run, which have none)
    const nl_plan *P = (const nl_plan *)m->priv;
    int herr = 0;
    if (P && P->err) NL_CK(cudaMemcpyAsync(&herr, P->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    NL_CK(cudaStreamSynchronize(ctx->stream));
    if (herr & 256)
        return nl_fail(ctx, NL_EUNSUPPORTED, "a fixed-point sum left its range (error word " +
                                                 std::to_string(herr) + ")");
    if (herr)
        return nl_fail(ctx, NL_EUNSUPPORTED, "the numeric phase or the scatter failed (error word " +
                                                 std::to_string(herr) + ")");
    return NL_OK;
}

void nl_csr_free(nl_ctx *ctx, nl_csr *m)
{
    if (!m) return;
    nl_plan *P = (nl_plan *)m->priv;
    // stream-ordered: work already queued on the context's stream finishes first
    cudaStream_t s = ctx ? ctx->stream : (P ? P->stream : nullptr);
    nl_free(m->row_ptr, s);
    nl_free(m->col_idx, s);
    nl_free(m->val, s);
    if (P) {
        nl_plan_free(P, s);
        delete P;
    }
    memset(m, 0, sizeof *m);
}

int64_t nl_launch_count(nl_ctx *ctx) { return ctx ? ctx->launches : 0; }

nl_status nl_last_timings(nl_ctx *ctx, double *ms4)
{
    if (!ctx || !ms4) return NL_EINVAL;
    NL_CK(cudaEventSynchronize(ctx->ev[4]));
    for (int i = 0; i < 4; i++) {
        float ms = 0.0f;
        cudaError_t e = cudaEventElapsedTime(&ms, ctx->ev[i], ctx->ev[i + 1]);
        if (e != cudaSuccess) return nl_cuda_fail(ctx, e, "cudaEventElapsedTime");
        ms4[i] = ms;
    }
    return NL_OK;
}

}  // extern "C"
