// numeric.cuh -- pair geometry + quadrature, one warp per outer triangle T_a.
//
// For the outer triangle T_a the warp stages its outer quadrature points x_q,
// weights W_q = w_q |T_a| and barycentric coordinates phi_a(x_q) in shared memory;
// each lane then takes candidate neighbours T_b in turn and, for every x_q, builds
// R(x_q, T_b) (geometry.cuh) and its inner sums
//     s0 = sum w psi,  s1 = sum w psi phi_b,  S2 = sum w psi phi_b phi_b^T
// over the fan subtriangles (inner rule) and caps (one centroid point), which
// gives the expansion of (phi_j(x)-phi_j(y))(phi_j'(x)-phi_j'(y)) psi of
// Eq. (bformhj) over the six local nodes (Sec. 7.2):
//     M_aa += W s0 phi_a phi_a^T,   M_bb += W S2,   M_ab += W phi_a s1^T
// (D receives +M_aa, +M_bb, -M_ab and -M_ab^T).  Per candidate pair the lane writes
// M_ab (9) to a pair buffer and a directed interaction flag, and adds the upper M_bb (6,
// symmetric) onto T_b's per-triangle sums (FP64 atomics); M_aa is summed over all
// candidates in FP64 and reduced across the warp.
//
// T = double: FP64 quadrature.  T = float: the inner sums run in FP32, the boundary
// kernel's per-pair sums in 32-bit fixed point (exact, order-free integer adds of values
// rounded to a per-pair grid), and the long sums (M_aa over all neighbours, M_bb over all
// pairs of T_b, and D over all pairs in the scatter) in FP64, which compensates the FP32
// rounding of the short sums.
#pragma once

#include <type_traits>

#include "geometry.cuh"

namespace nlq {

using nlg::D2;

struct RuleTab {
    int n, nsplit;            // nsplit: first point of the second rule (outer switch), else n
    double l[NL_MAXQ + 8][3];
    double w[NL_MAXQ + 8];
};

// An undecided (q, b) item of the FP32 path whose region the FP64 geometry has to build
// (an uncertified FP32 choice, the singular kernel's near field, a ball without an FP32
// region).  The boundary kernel queues it instead of running the FP64 code in one lane of
// an otherwise idle warp; k_deferred then integrates the queue with every lane busy.
struct DeferItem {
    int64_t e;     // candidate pair (T_a, T_b)
    int32_t a;     // outer triangle T_a
    int32_t qp;    // outer point q (bits 0-7) and problem index in a batched launch (bits 8-31)
};

// A queue of cap items is one allocation: the items, then the M_ab values (9 floats a slot,
// value-major: [9][cap]) that k_deferred computes and k_defer_merge adds onto the pairs.
constexpr int kDeferVals = 9;
inline size_t defer_alloc_items(int cap)
{
    return (size_t)cap + ((size_t)cap * kDeferVals * sizeof(float) + sizeof(DeferItem) - 1) / sizeof(DeferItem);
}
__host__ __device__ inline float *defer_values(DeferItem *q, int cap) { return q ? (float *)(q + cap) : nullptr; }

struct OuterPt;

struct NumArgs {
    int K;
    int64_t E;
    const double *tx, *ty;            // [3][K]
    const double *bx, *by, *area;     // [K]
    const float *akc;                 // [K] |T| kc in FP32
    const float *hl;                  // [16][K] coordinates as FP32 hi + lo pairs (k_hilo)
    const int64_t *nbr_ptr, *nbr_split;
    const int32_t *nbr_idx;
    RuleTab outer, inner;
    float4 fin[NL_MAXQ + 8];          // inner rule in FP32: barycentrics (x, y, z) and weight (w)
    float4 fout[NL_MAXQ + 8];         // outer rule in FP32 (the outer-support composite rule)
    double gl_x[8], gl_w[8];          // Gauss-Legendre on [0,1] with duffy_n points
    double gl2_x[2], gl2_w[2];
    float glf_x[8], glf_w[8];         // the same rules in FP32 (no FP64 conversions in the FP32 path)
    float glf_sh[8], glf_ch[8];       // sinh and cosh of the duffy_n nodes glf_x (FP32)
    float sh1f, ch1f;                 // sinh(1), cosh(1) (FP32)
    float gl2f_x[2], gl2f_w[2];
    float kcf;                        // kc in FP32
    int duffy_n;
    int switch47;                     // outer rule: 0..nsplit-1 if |bary_a - bary_b|^2 < thr2 else nsplit..n-1
    double thr2;                      // (delta - h_max)^2, or -1 when delta <= h_max
    int kernel;                       // nl_kernel
    int ball;                         // nl_ball (run-time dispatch of the batched kernel)
    int shifted;                      // every outer point's ball centred at bary_a (Sec. 4.3)
    int outer_support;                // barycenter ball with the outer integral over T_a n B(bary_b)
    double kc;
    nlg::GeoParams geo;
    uint8_t *flag;
    void *blk;                        // [9][E]: M_ab of every candidate pair (float or double)
    double *maa;                      // [6][K]
    double *mbb;                      // [6][K]: per-triangle sums of the pairs' upper M_bb (FP64 atomics;
                                      // zeroed before the numeric phase)
    int64_t *qp_a, *cnt_a;
    uint64_t *hash_a;
    int stats;
    int *err;                         // device error word: bit 0 = region buffer bound hit
    DeferItem *defer;                 // FP32 path: queue of the items the FP64 geometry decides (null: inline)
    float *dval;                      // [9][defer_cap]: each queued item's M_ab (k_deferred -> k_defer_merge)
    int *defer_n;                     // its fill count (zeroed before the boundary launch; may exceed the cap)
    int defer_cap;
    DeferItem *nearq;                 // FP32 path, singular kernel: queue of the near-field whole items that
                                      // k_near integrates (null: the boundary kernel integrates them itself)
    int *near_n;                      // its fill count (zeroed before the boundary launch; may exceed the cap)
    int near_cap;
    OuterPt *otab;                    // [K][outer.n] outer points as the boundary kernel staged them (read by
                                      // k_near; with the near-field queue only)
    int prob;                         // index of this problem in a batched launch's argument array
    float s0q_grid;                   // FP32 boundary kernel: scale of the fixed-point sums of s0 per
                                      // outer point (a power of two; the bound on a sum maps below 2^30)
};

template <typename T>
struct Sums {
    T s0, s1[3], S2[6];   // S2: 00 11 22 01 02 12
};

template <typename T>
__device__ __forceinline__ void sums_zero(Sums<T> &S)
{
    S.s0 = 0;
    for (int i = 0; i < 3; i++) S.s1[i] = 0;
    for (int i = 0; i < 6; i++) S.S2[i] = 0;
}

template <typename T>
__device__ __forceinline__ void sums_add(Sums<T> &S, T w, T p0, T p1, T p2)
{
    S.s0 += w;
    T w0 = w * p0, w1 = w * p1, w2 = w * p2;
    S.s1[0] += w0; S.s1[1] += w1; S.s1[2] += w2;
    S.S2[0] += w0 * p0; S.S2[1] += w1 * p1; S.S2[2] += w2 * p2;
    S.S2[3] += w0 * p1; S.S2[4] += w0 * p2; S.S2[5] += w1 * p2;
}

// affine map y -> barycentric coordinates in T_b (values only)
struct BaryMap {
    double ox, oy, e1x, e1y, e2x, e2y, inv;
};

__device__ __forceinline__ BaryMap bary_map(const D2 V[3])
{
    BaryMap m;
    m.ox = V[0].x; m.oy = V[0].y;
    m.e1x = V[1].x - V[0].x; m.e1y = V[1].y - V[0].y;
    m.e2x = V[2].x - V[0].x; m.e2y = V[2].y - V[0].y;
    m.inv = 1.0 / (m.e1x * m.e2y - m.e2x * m.e1y);
    return m;
}

__device__ __forceinline__ void bary_of(const BaryMap &m, double yx, double yy, double phi[3])
{
    double dx = yx - m.ox, dy = yy - m.oy;
    double l1 = (dx * m.e2y - m.e2x * dy) * m.inv;
    double l2 = (m.e1x * dy - dx * m.e1y) * m.inv;
    phi[0] = 1.0 - l1 - l2;
    phi[1] = l1;
    phi[2] = l2;
}

// The discrete choices of the near-singular rule for edge (P_a, P_b) and outer point x,
// in FP64 with the expression order of the rule's definition (no contraction): the foot
// distance d (a zero-area piece is skipped) and the signed positions tA, tB of the end
// points along the edge (a zero-length piece is skipped, ceil(asinh(|t| / d)) panels).
struct NearEdge64 {
    double d, tA, tB;
};

__device__ __forceinline__ NearEdge64 near_edge64(D2 pa, D2 pb, D2 x)
{
    using namespace nlg;
    double ex = sub(pb.x, pa.x), ey = sub(pb.y, pa.y);
    const double L = __dsqrt_rn(add(mul(ex, ex), mul(ey, ey)));
    NearEdge64 r;
    if (L == 0.0) { r.d = 0.0; r.tA = r.tB = 0.0; return r; }
    ex = dvd(ex, L);
    ey = dvd(ey, L);
    r.tA = add(mul(sub(pa.x, x.x), ex), mul(sub(pa.y, x.y), ey));
    r.tB = add(mul(sub(pb.x, x.x), ex), mul(sub(pb.y, x.y), ey));
    const double fx = sub(sub(pa.x, mul(r.tA, ex)), x.x), fy = sub(sub(pa.y, mul(r.tA, ey)), x.y);
    r.d = __dsqrt_rn(add(mul(fx, fx), mul(fy, fy)));
    return r;
}

__device__ __forceinline__ int near_panels64(double tau, double d)
{
    int n = (int)ceil(asinh(fabs(tau) / d));
    return n < 1 ? 1 : n;
}

// Near-singular rule for psi = c/|x - y| (signed apex-x decomposition with a Duffy
// collapse in s and the sinh substitution in u; dy/|x-y| = d ds du), FP64.
__device__ __forceinline__ void near_right_triangle(const NumArgs &A, const BaryMap &bm, D2 x, D2 F, double ex,
                                                    double ey, double d, double tau, double sign, int npan,
                                                    Sums<double> &S, int64_t &nqp)
{
    double sg = tau > 0.0 ? 1.0 : -1.0;
    double U = fmax(asinh(fabs(tau) / d), (double)(npan - 1));
    const int nu = A.duffy_n;
    for (int p = 0; p < npan; p++) {
        double u0 = (double)p, u1 = (p + 1 < npan) ? (double)(p + 1) : U;
        double hw = u1 - u0;
        for (int j = 0; j < nu; j++) {
            double u = u0 + hw * A.gl_x[j];
            double wu = hw * A.gl_w[j];
            double sh = sinh(u);
            double wx = (F.x - x.x) + sg * d * sh * ex;
            double wy = (F.y - x.y) + sg * d * sh * ey;
            for (int i = 0; i < 2; i++) {
                double sv = A.gl2_x[i];
                double phi[3];
                bary_of(bm, x.x + sv * wx, x.y + sv * wy, phi);
                sums_add<double>(S, sign * sg * d * A.gl2_w[i] * wu * A.kc, phi[0], phi[1], phi[2]);
                nqp++;
            }
        }
    }
}

__device__ __forceinline__ void near_polygon(const NumArgs &A, const BaryMap &bm, D2 x, const nlg::Region &R,
                                             Sums<double> &S, int64_t &nqp)
{
    const int n = R.nv;
    for (int i = 0; i < n; i++) {
        D2 a = R.P[i], b = R.P[(i + 1) % n];
        const NearEdge64 q = near_edge64(a, b, x);
        if (q.d == 0.0) continue;
        double ex = b.x - a.x, ey = b.y - a.y;
        double L = sqrt(ex * ex + ey * ey);
        if (L == 0.0) continue;
        ex /= L;
        ey /= L;
        double tA = (a.x - x.x) * ex + (a.y - x.y) * ey;
        double tB = (b.x - x.x) * ex + (b.y - x.y) * ey;
        D2 F;
        F.x = a.x - tA * ex;
        F.y = a.y - tA * ey;
        double fx = F.x - x.x, fy = F.y - x.y;
        double d = sqrt(fx * fx + fy * fy);
        double sigma = (fx * ey - fy * ex) > 0.0 ? 1.0 : -1.0;
        if (q.tB != 0.0) near_right_triangle(A, bm, x, F, ex, ey, d, tB, sigma, near_panels64(q.tB, q.d), S, nqp);
        if (q.tA != 0.0) near_right_triangle(A, bm, x, F, ex, ey, d, tA, -sigma, near_panels64(q.tA, q.d), S, nqp);
    }
}

// inner sums of the region R(x, T_b)
// one inner rule point: barycentrics and weight (FP32 path: one 128-bit load)
template <typename T>
__device__ __forceinline__ void rule_pt(const NumArgs &A, int r, T &p0, T &p1, T &p2, T &w)
{
    if (sizeof(T) == sizeof(float)) {
        const float4 f = A.fin[r];
        p0 = (T)f.x; p1 = (T)f.y; p2 = (T)f.z; w = (T)f.w;
    } else {
        p0 = (T)A.inner.l[r][0]; p1 = (T)A.inner.l[r][1]; p2 = (T)A.inner.l[r][2]; w = (T)A.inner.w[r];
    }
}

// inner sums over the whole triangle T_b: phi_b at the rule points are the rule's barycentrics.
// KIN: the kernel type when the caller knows it at compile time (0 constant, 1 c/|x - y|), else
// -1 (read from A.kernel)
template <typename T, int KIN = -1>
__device__ __forceinline__ void whole_sums(const NumArgs &A, const D2 V[3], T area_kc, D2 x, Sums<T> &S,
                                           int64_t &nqp, const nlg::F2 *dl = nullptr)
{
    sums_zero(S);
    const bool inv = KIN < 0 ? (A.kernel == NL_KERNEL_INV_DIST) : (KIN == 1);
    const int n = A.inner.n;
    T ar = area_kc;
    // Every (x_q, T_b) evaluates its inner points: for a constant kernel on a whole T_b
    // they do not depend on x, and the opaque barrier keeps the compiler from hoisting
    // them out of the outer-point loop (that hoist would skip counted work).
    if (sizeof(T) == sizeof(float)) asm volatile("" : "+f"(*(float *)&ar));
    else asm volatile("" : "+d"(*(double *)&ar));
    T lx[3], ly[3];
    if (inv) {
        if (sizeof(T) == sizeof(float) && dl)   // FP32 coordinates relative to x (no FP64 work)
            for (int i = 0; i < 3; i++) { lx[i] = (T)dl[i].x; ly[i] = (T)dl[i].y; }
        else
            for (int i = 0; i < 3; i++) { lx[i] = (T)(V[i].x - x.x); ly[i] = (T)(V[i].y - x.y); }
    }
    for (int r = 0; r < n; r++) {
        T p0, p1, p2, w;
        rule_pt<T>(A, r, p0, p1, p2, w);
        w *= ar;
        if (inv) {
            T dx = p0 * lx[0] + p1 * lx[1] + p2 * lx[2];
            T dy = p0 * ly[0] + p1 * ly[1] + p2 * ly[2];
            w = w / sqrt(dx * dx + dy * dy);
        }
        sums_add<T>(S, w, p0, p1, p2);
    }
    nqp += n;
}

template <typename T>
__device__ __forceinline__ void inner_sums(const NumArgs &A, const nlg::Region &R, const D2 V[3], double area_b,
                                           D2 x, Sums<T> &S, int64_t &nqp)
{
    sums_zero(S);
    const bool inv = (A.kernel == NL_KERNEL_INV_DIST);
    const RuleTab &ri = A.inner;
    if (inv && R.nv >= 3 && nlg::is_near(R, V, x)) {
        BaryMap bm = bary_map(V);
        Sums<double> Sd;
        sums_zero(Sd);
        near_polygon(A, bm, x, R, Sd, nqp);
        S.s0 = (T)Sd.s0;
        for (int i = 0; i < 3; i++) S.s1[i] = (T)Sd.s1[i];
        for (int i = 0; i < 6; i++) S.S2[i] = (T)Sd.S2[i];
    } else if (R.kind == nlg::KIND_WHOLE && R.ncap == 0) {
        // the region is T_b itself: phi_b at the rule points are the rule's barycentrics
        const T ar = (T)area_b;
        T lx[3], ly[3];
        if (inv)
            for (int i = 0; i < 3; i++) { lx[i] = (T)(V[i].x - x.x); ly[i] = (T)(V[i].y - x.y); }
        for (int r = 0; r < ri.n; r++) {
            T p0 = (T)ri.l[r][0], p1 = (T)ri.l[r][1], p2 = (T)ri.l[r][2];
            T w = (T)ri.w[r] * ar;
            if (inv) {
                T dx = p0 * lx[0] + p1 * lx[1] + p2 * lx[2];
                T dy = p0 * ly[0] + p1 * ly[1] + p2 * ly[2];
                w = w * (T)A.kc / sqrt(dx * dx + dy * dy);
            } else {
                w = w * (T)A.kc;
            }
            sums_add<T>(S, w, p0, p1, p2);
        }
        nqp += ri.n;
    } else {
        BaryMap bm = bary_map(V);
        if (R.nv >= 3) {
            double ph0[3];
            bary_of(bm, R.P[0].x, R.P[0].y, ph0);
            T f0[3] = {(T)ph0[0], (T)ph0[1], (T)ph0[2]};
            T l0x = (T)(R.P[0].x - x.x), l0y = (T)(R.P[0].y - x.y);
            double phk[3];
            bary_of(bm, R.P[1].x, R.P[1].y, phk);
            T fk[3] = {(T)phk[0], (T)phk[1], (T)phk[2]};
            T lkx = (T)(R.P[1].x - x.x), lky = (T)(R.P[1].y - x.y);
            for (int k = 1; k + 1 < R.nv; k++) {
                D2 s0p = R.P[0], s1p = R.P[k], s2p = R.P[k + 1];
                double ar = 0.5 * fabs((s1p.x - s0p.x) * (s2p.y - s0p.y) - (s2p.x - s0p.x) * (s1p.y - s0p.y));
                double phn[3];
                bary_of(bm, s2p.x, s2p.y, phn);
                T fn[3] = {(T)phn[0], (T)phn[1], (T)phn[2]};
                T lnx = (T)(s2p.x - x.x), lny = (T)(s2p.y - x.y);
                const T art = (T)ar;
                for (int r = 0; r < ri.n; r++) {
                    T m0, m1, m2, w;
                    rule_pt<T>(A, r, m0, m1, m2, w);
                    T p0 = m0 * f0[0] + m1 * fk[0] + m2 * fn[0];
                    T p1 = m0 * f0[1] + m1 * fk[1] + m2 * fn[1];
                    T p2 = m0 * f0[2] + m1 * fk[2] + m2 * fn[2];
                    w *= art;
                    if (inv) {
                        T dx = m0 * l0x + m1 * lkx + m2 * lnx;
                        T dy = m0 * l0y + m1 * lky + m2 * lny;
                        w = w * (T)A.kc / sqrt(dx * dx + dy * dy);
                    } else {
                        w = w * (T)A.kc;
                    }
                    sums_add<T>(S, w, p0, p1, p2);
                }
                nqp += ri.n;
                fk[0] = fn[0]; fk[1] = fn[1]; fk[2] = fn[2];
                lkx = lnx; lky = lny;
            }
        }
        for (int c = 0; c < R.ncap; c++) {
            double ph[3];
            bary_of(bm, R.cc[c].x, R.cc[c].y, ph);
            T w = (T)R.cw[c];
            if (inv) {
                double dx = R.cc[c].x - x.x, dy = R.cc[c].y - x.y;
                w = w * (T)(A.kc / sqrt(dx * dx + dy * dy));
            } else {
                w = w * (T)A.kc;
            }
            sums_add<T>(S, w, (T)ph[0], (T)ph[1], (T)ph[2]);
            nqp++;
        }
    }
}

// inner sums over a fanned polygon in FP32 coordinates relative to x, held in the lane's columns
// px / py of a shared buffer (FP32 path; KIN as for whole_sums)
template <int KIN = -1>
__device__ __forceinline__ void poly_sums_col(const NumArgs &A, nlg::Col px, nlg::Col py, int n, const nlg::F2 &d0,
                                              const nlg::F2 &e1, const nlg::F2 &e2, float inv_det,
                                              Sums<float> &S, int64_t &nqp)
{
    sums_zero(S);
    const int nr = A.inner.n;
    const float kc = A.kcf;
    auto phi = [&](float x, float y, float f[3]) {
        const float rx = x - d0.x, ry = y - d0.y;
        const float l1 = (rx * e2.y - e2.x * ry) * inv_det;
        const float l2 = (e1.x * ry - rx * e1.y) * inv_det;
        f[0] = 1.f - l1 - l2;
        f[1] = l1;
        f[2] = l2;
    };
    const float x0 = px[0], y0 = py[0];
    float xk = px[1], yk = py[1];
    float f0[3], fk[3];
    phi(x0, y0, f0);
    phi(xk, yk, fk);
    for (int k = 1; k + 1 < n; k++) {
        const float xn = px[k + 1], yn = py[k + 1];
        const float ar = 0.5f * fabsf((xk - x0) * (yn - y0) - (xn - x0) * (yk - y0)) * kc;
        float fn[3];
        phi(xn, yn, fn);
        for (int r = 0; r < nr; r++) {
            const float4 f = A.fin[r];
            const float m0 = f.x, m1 = f.y, m2 = f.z;
            const float p0 = m0 * f0[0] + m1 * fk[0] + m2 * fn[0];
            const float p1 = m0 * f0[1] + m1 * fk[1] + m2 * fn[1];
            const float p2 = m0 * f0[2] + m1 * fk[2] + m2 * fn[2];
            float w = f.w * ar;
            if (KIN < 0 ? A.kernel == NL_KERNEL_INV_DIST : KIN == 1) {   // psi = c / |y - x|, relative to x
                const float yx = m0 * x0 + m1 * xk + m2 * xn, yy = m0 * y0 + m1 * yk + m2 * yn;
                w *= rsqrtf(yx * yx + yy * yy);
            }
            sums_add<float>(S, w, p0, p1, p2);
        }
        nqp += nr;
        fk[0] = fn[0]; fk[1] = fn[1]; fk[2] = fn[2];
        xk = xn; yk = yn;
    }
}

// the same over buffer `which` of a clip buffer (the N-gon clip's output)
template <int KIN = -1>
__device__ __forceinline__ void poly_sums_sh(const NumArgs &A, const nlg::ClipBuf &cb, int which, int lane, int n,
                                             const nlg::F2 &d0, const nlg::F2 &e1, const nlg::F2 &e2, float inv_det,
                                             Sums<float> &S, int64_t &nqp)
{
    nlg::ClipBuf &c = const_cast<nlg::ClipBuf &>(cb);
    poly_sums_col<KIN>(A, nlg::Col{&c.x[which][0][lane]}, nlg::Col{&c.y[which][0][lane]}, n, d0, e1, e2, inv_det, S,
                       nqp);
}

// FP32 version of the near-singular rule (FP32-compensated path) for the whole triangle
// with FP32 vertices dl relative to x: the same signed apex-x decomposition, Duffy collapse
// and sinh substitution.  Its discrete choices are taken in FP64 (near_edge64) whenever
// FP32 is within 1e-4 of a threshold, so the evaluated points are those of the FP64 rule.
__device__ __forceinline__ void near_whole_f32(const NumArgs &A, const nlg::F2 dl[3], int tb, D2 x,
                                               const nlg::F2 &e1, const nlg::F2 &e2, float inv_det,
                                               Sums<float> &S, int64_t &nqp)
{
    sums_zero(S);
    const float kc = A.kcf;
    const int nu = A.duffy_n;
    for (int i = 0; i < 3; i++) {
        const nlg::F2 a = dl[i], b = dl[(i + 1) % 3];
        float ex = b.x - a.x, ey = b.y - a.y;
        const float L = sqrtf(ex * ex + ey * ey);
        ex /= L;
        ey /= L;
        const float tA = a.x * ex + a.y * ey, tB = b.x * ex + b.y * ey;
        const float Fx = a.x - tA * ex, Fy = a.y - tA * ey;
        const float d = sqrtf(Fx * Fx + Fy * Fy);
        const float UA = asinhf(fabsf(tA) / d), UB = asinhf(fabsf(tB) / d);
        const float th = 1e-4f * L;
        // U = asinh(|t| / d) moves by at most dt/|t| + dd/d; the FP32 coordinates carry an
        // absolute error below 1e-6 M (M = max(|a|, |b|) + L), asinhf a few ulp
        const float M = fmaxf(fmaxf(fabsf(a.x) + fabsf(a.y), fabsf(b.x) + fabsf(b.y)), L) + L;
        auto near_int = [&](float U, float t) {
            const float eps = 1e-6f * M * (1.f / d + 1.f / fabsf(t)) + 1e-5f * fmaxf(U, 1.f);
            return fabsf(U - rintf(U)) < eps;
        };
        bool skip_edge = false, skipA = false, skipB = false;
        int npA, npB;
        if (!(d >= th) || !(fabsf(tA) >= th) || !(fabsf(tB) >= th) || near_int(UA, tA) || near_int(UB, tB)) {
            // the FP64 vertices of T_b (edge i) from global memory
            const int i1 = (i + 1) % 3;
            const D2 Vi = {A.tx[i * A.K + tb], A.ty[i * A.K + tb]}, Vj = {A.tx[i1 * A.K + tb], A.ty[i1 * A.K + tb]};
            const NearEdge64 q = near_edge64(Vi, Vj, x);
            skip_edge = (q.d == 0.0);
            skipA = (q.tA == 0.0);
            skipB = (q.tB == 0.0);
            npA = skip_edge || skipA ? 0 : near_panels64(q.tA, q.d);
            npB = skip_edge || skipB ? 0 : near_panels64(q.tB, q.d);
        } else {
            npA = (int)ceilf(UA);
            npB = (int)ceilf(UB);
            npA = npA < 1 ? 1 : npA;
            npB = npB < 1 ? 1 : npB;
        }
        if (skip_edge || d == 0.f) continue;
        const float sigma = (Fx * ey - Fy * ex) > 0.f ? 1.f : -1.f;
        // The panels of both sides (B, then A) in one loop, so that lanes whose sides split their
        // panels differently still run the loop body together.  On a full panel [p, p + 1],
        // sinh(p + x_j) = sinh(p) cosh(x_j) + cosh(p) sinh(x_j), with sinh(p), cosh(p) carried from
        // panel to panel by the same addition theorem (sinh(1), cosh(1)); the last panel of a side,
        // [p, U], evaluates sinh directly.  The FP32 point y = s w - v_0 of T_b relative to its
        // first vertex is linear in s, and so are its barycentrics: l = s l_w - l_0.
        const int nB = skipB ? 0 : npB, nA = skipA ? 0 : npA;
        const float l10 = (dl[0].x * e2.y - e2.x * dl[0].y) * inv_det;
        const float l20 = (e1.x * dl[0].y - dl[0].x * e1.y) * inv_det;
        float sp = 0.f, cp = 1.f;   // sinh, cosh of the panel start
        for (int p = 0; p < nB + nA; p++) {
            const bool sideA = p >= nB;
            const int pnl = sideA ? p - nB : p, npan = sideA ? nA : nB;
            const float tau = sideA ? tA : tB, U = sideA ? UA : UB;
            const float sign = sideA ? -sigma : sigma;
            const float sg = tau > 0.f ? 1.f : -1.f;
            if (pnl == 0) {
                sp = 0.f;
                cp = 1.f;
            }
            const bool full = pnl + 1 < npan;
            const float u0 = (float)pnl, hw = full ? 1.f : fmaxf(U, u0) - u0;
            const float gdx = sg * d * ex, gdy = sg * d * ey, kcs = sign * sg * d * kc;
            // the Gauss points of the panel: sinh at the node, then the two points in s
            auto node = [&](int j, float sh) {
                const float wj = kcs * (hw * A.glf_w[j]);
                const float wx = fmaf(sh, gdx, Fx), wy = fmaf(sh, gdy, Fy);
                const float l1w = (wx * e2.y - e2.x * wy) * inv_det;
                const float l2w = (e1.x * wy - wx * e1.y) * inv_det;
                for (int k = 0; k < 2; k++) {
                    const float sv = A.gl2f_x[k];
                    const float l1 = sv * l1w - l10, l2 = sv * l2w - l20;
                    sums_add<float>(S, wj * A.gl2f_w[k], 1.f - l1 - l2, l1, l2);
                }
            };
            for (int j = 0; j < nu; j++)
                node(j, full ? fmaf(sp, A.glf_ch[j], cp * A.glf_sh[j]) : sinhf(u0 + hw * A.glf_x[j]));
            nqp += 2 * nu;
            if (full) {
                const float sn = fmaf(sp, A.ch1f, cp * A.sh1f);
                cp = fmaf(cp, A.ch1f, sp * A.sh1f);
                sp = sn;
            }
        }
    }
}

struct OuterPt {
    double x, y, W, l0, l1, l2;
    float lx, ly;     // x_q - bary_a in FP32
    float Wf, l0f, l1f, l2f;   // FP32 copies (no FP64 conversions in the FP32 path)
};

constexpr int kWarpsPerBlock = 4;

// Per-lane accumulators of one outer triangle: stats and the M_aa sum, in FP64 for double
// blocks and as compensated FP32 sums (Kahan: value mf, compensation mc) for float blocks.
struct LaneAcc {
    double maa[6];
    float mf[6], mc[6];
    uint32_t cnt, qp;   // per outer triangle and lane: far below 2^32
    uint64_t hsum;
};

__device__ __forceinline__ void acc_zero(LaneAcc &acc)
{
    for (int i = 0; i < 6; i++) {
        acc.maa[i] = 0.0;
        acc.mf[i] = 0.f;
        acc.mc[i] = 0.f;
    }
    acc.cnt = 0;
    acc.qp = 0;
    acc.hsum = 0;
}

// outer point q of T_a (vertices Va, area area_a)
__device__ __forceinline__ OuterPt outer_point(const NumArgs &A, int a, const D2 Va[3], double area_a, int q)
{
    double l0 = A.outer.l[q][0], l1 = A.outer.l[q][1], l2 = A.outer.l[q][2];
    OuterPt o;
    // x_q = l0 v0 + l1 v1 + l2 v2, left to right, round-to-nearest
    o.x = nlg::add(nlg::add(nlg::mul(l0, Va[0].x), nlg::mul(l1, Va[1].x)), nlg::mul(l2, Va[2].x));
    o.y = nlg::add(nlg::add(nlg::mul(l0, Va[0].y), nlg::mul(l1, Va[1].y)), nlg::mul(l2, Va[2].y));
    o.W = A.outer.w[q] * area_a;
    o.l0 = l0; o.l1 = l1; o.l2 = l2;
    o.lx = (float)(o.x - A.bx[a]);
    o.ly = (float)(o.y - A.by[a]);
    if (A.shifted) {
        // shifted-centre ball (Sec. 4.3): the region is built around bary_a for every outer
        // point; x_q keeps its weight and barycentrics (o.W, o.l*)
        o.x = A.bx[a];
        o.y = A.by[a];
        o.lx = 0.f;
        o.ly = 0.f;
    }
    o.Wf = (float)o.W;
    o.l0f = (float)l0; o.l1f = (float)l1; o.l2f = (float)l2;
    return o;
}

// outer points of T_a in shared memory (computed by the warp's lanes)
__device__ __forceinline__ void stage_outer(const NumArgs &A, int a, OuterPt *sq, int lane)
{
    const int K = A.K;
    D2 Va[3];
    for (int i = 0; i < 3; i++) { Va[i].x = A.tx[i * K + a]; Va[i].y = A.ty[i * K + a]; }
    const double area_a = A.area[a];
    for (int q = lane; q < A.outer.n; q += 32) sq[q] = outer_point(A, a, Va, area_a, q);
    __syncwarp();
}

// rule range of the pair (outer-rule switch of Sec. 8)
__device__ __forceinline__ void rule_range(const NumArgs &A, const D2 &ba, const D2 &bb, int &q0, int &q1)
{
    q0 = 0;
    q1 = A.outer.n;
    if (A.switch47) {
        double dx = nlg::sub(ba.x, bb.x), dy = nlg::sub(ba.y, bb.y);
        bool near4 = A.thr2 > 0.0 && nlg::add(nlg::mul(dx, dx), nlg::mul(dy, dy)) < A.thr2;
        if (near4) q1 = A.outer.nsplit; else q0 = A.outer.nsplit;
    }
}

// the per-(q, b) outer combination: M_bb += W S2, M_ab += W phi_a s1^T, M_aa += W s0 phi_a phi_a^T
template <typename T>
__device__ __forceinline__ void combine(const OuterPt &o, const Sums<T> &S, T *v)
{
    const bool f32 = sizeof(T) == sizeof(float);
    const T W = f32 ? (T)o.Wf : (T)o.W, la0 = f32 ? (T)o.l0f : (T)o.l0;
    const T la1 = f32 ? (T)o.l1f : (T)o.l1, la2 = f32 ? (T)o.l2f : (T)o.l2;
    const T wa0 = W * la0, wa1 = W * la1, wa2 = W * la2;
    v[0] += wa0 * S.s1[0]; v[1] += wa0 * S.s1[1]; v[2] += wa0 * S.s1[2];
    v[3] += wa1 * S.s1[0]; v[4] += wa1 * S.s1[1]; v[5] += wa1 * S.s1[2];
    v[6] += wa2 * S.s1[0]; v[7] += wa2 * S.s1[1]; v[8] += wa2 * S.s1[2];
    v[9] += W * S.S2[0]; v[10] += W * S.S2[1]; v[11] += W * S.S2[2];
    v[12] += W * S.S2[3]; v[13] += W * S.S2[4]; v[14] += W * S.S2[5];
    const T ws = W * S.s0;
    v[15] += ws * la0 * la0; v[16] += ws * la1 * la1; v[17] += ws * la2 * la2;
    v[18] += ws * la0 * la1; v[19] += ws * la0 * la2; v[20] += ws * la1 * la2;
}

// M_aa contributions m[0..5] into the lane's sums of its outer triangle
template <typename T>
__device__ __forceinline__ void maa_add(LaneAcc &acc, const T *m)
{
    if (sizeof(T) == sizeof(float)) {
        for (int i = 0; i < 6; i++) {
            const float y = (float)m[i] - acc.mc[i];
            const float t = acc.mf[i] + y;
            acc.mc[i] = (t - acc.mf[i]) - y;
            acc.mf[i] = t;
        }
    } else {
        for (int i = 0; i < 6; i++) acc.maa[i] += (double)m[i];
    }
}

// the pair's block: M_ab stored (v[0..8]), its upper M_bb (v[9..14]) added onto T_b's sums, its
// M_aa (v[15..20]) into the lane's sums of T_a (MAA = false: the caller sums M_aa itself)
template <typename T, bool MAA = true>
__device__ __forceinline__ void write_pair(const NumArgs &A, int64_t e, int b, bool any, const T *v, LaneAcc &acc)
{
    A.flag[e] = any ? 1 : 0;
    T *blk = (T *)A.blk;
    for (int i = 0; i < 9; i++) blk[(int64_t)i * A.E + e] = v[i];
    if (any)
        for (int i = 0; i < 6; i++) atomicAdd(&A.mbb[(int64_t)i * A.K + b], (double)v[9 + i]);
    if (MAA) maa_add<T>(acc, v + 15);
}

__device__ __forceinline__ void warp_reduce(LaneAcc &acc)
{
    for (int i = 0; i < 6; i++) acc.maa[i] += (double)acc.mf[i] - (double)acc.mc[i];
    for (int off = 16; off; off >>= 1) {
        for (int i = 0; i < 6; i++) acc.maa[i] += __shfl_xor_sync(0xffffffffu, acc.maa[i], off);
        acc.cnt += __shfl_xor_sync(0xffffffffu, acc.cnt, off);
        acc.qp += __shfl_xor_sync(0xffffffffu, acc.qp, off);
        acc.hsum += __shfl_xor_sync(0xffffffffu, acc.hsum, off);
    }
}

// whether the kernel accumulates the interaction statistics' record hashes: STS < 0 reads
// A.stats at run time; 0 / 1 fix it at compile time (the assembly's kernels leave the hash code
// out of their loops)
template <int STS>
__device__ __forceinline__ bool want_stats(const NumArgs &A)
{
    return STS < 0 ? A.stats != 0 : STS == 1;
}

// ---------------------------------------------------------------------------
// Interior pairs: T_b is whole for every outer point of T_a (certified when the
// candidate lists are built), so there is no per-point classification.  k_interior runs
// concurrently with k_boundary (it fills the boundary kernel's last wave): both add the
// per-triangle M_aa and statistics atomically onto zeroed outputs; the batched kernels run
// one after the other and store, then add.
// ---------------------------------------------------------------------------
template <typename T, int STS = -1, int KIN = -1>
__device__ __forceinline__ void interior_outer(const NumArgs &A, int a, const OuterPt *sq, int lane, LaneAcc &acc)
{
    const int K = A.K;
    const D2 ba = {A.bx[a], A.by[a]};
    const int64_t e0 = A.nbr_ptr[a], es = A.nbr_split[a];
    for (int64_t e = e0 + lane; e < es; e += 32) {
        const int b = A.nbr_idx[e];
#ifdef NL_CHECKS
        if (b < 0 || b >= K) {   // debug build: bad candidate recorded (bit 16) and skipped
            atomicOr(A.err, 16);
            continue;
        }
#endif
        const bool inv = KIN < 0 ? A.kernel == NL_KERNEL_INV_DIST : KIN == 1;
        // the FP64 vertices only where the quadrature uses them (singular kernel)
        D2 Vb[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
        if (inv)
            for (int i = 0; i < 3; i++) { Vb[i].x = A.tx[i * K + b]; Vb[i].y = A.ty[i * K + b]; }
        const T akc = sizeof(T) == sizeof(float) ? (T)A.akc[b] : (T)(A.area[b] * A.kc);
        int q0 = 0, q1 = A.outer.n;
        if (A.switch47) rule_range(A, ba, D2{A.bx[b], A.by[b]}, q0, q1);
        nlg::F2 vl[3];
        if (inv)
            for (int i = 0; i < 3; i++) { vl[i].x = (float)(Vb[i].x - ba.x); vl[i].y = (float)(Vb[i].y - ba.y); }
        T v[21];
        for (int i = 0; i < 21; i++) v[i] = 0;
        for (int q = q0; q < q1; q++) {
            const OuterPt o = sq[q];
            Sums<T> S;
            int64_t nq = 0;
            nlg::F2 dl[3];
            if (inv)
                for (int i = 0; i < 3; i++) { dl[i].x = vl[i].x - o.lx; dl[i].y = vl[i].y - o.ly; }
            whole_sums<T, KIN>(A, Vb, akc, D2{o.x, o.y}, S, nq, inv ? dl : nullptr);
            combine<T>(o, S, v);
            acc.qp += nq;
            if (!A.outer_support) {
                acc.cnt++;
                if (want_stats<STS>(A)) acc.hsum += nlg::record_hash(a, b, q - q0, nlg::KIND_WHOLE, 3, 0);
            }
        }
        if (A.outer_support && q1 > q0) {   // one record per pair: the support is all of T_a
            acc.cnt++;
            if (want_stats<STS>(A)) acc.hsum += nlg::record_hash(a, b, 0, nlg::KIND_WHOLE, 3, 0);
        }
        write_pair<T>(A, e, b, q1 > q0, v, acc);
    }
}

// warp reduction of the outer triangle's accumulators and their store: kStore (the first
// kernel of the triangle), kAdd (onto the values an earlier kernel stored, in stream order) or
// kAtomicAdd (onto zeroed outputs, from kernels that run concurrently).  Two atomic addends
// onto zero give the same sum in either order, so the result does not depend on the schedule.
enum FinishMode { kStore, kAdd, kAtomicAdd };

template <int STS = -1>
__device__ __forceinline__ void finish_outer(const NumArgs &A, int a, LaneAcc &acc, int lane, FinishMode mode)
{
    warp_reduce(acc);
    if (lane == 0) {
        const int K = A.K;
        if (mode == kAtomicAdd) {
            for (int i = 0; i < 6; i++) atomicAdd(&A.maa[(int64_t)i * K + a], acc.maa[i]);
            atomicAdd((unsigned long long *)&A.qp_a[a], (unsigned long long)acc.qp);
            atomicAdd((unsigned long long *)&A.cnt_a[a], (unsigned long long)acc.cnt);
            if (want_stats<STS>(A)) atomicAdd((unsigned long long *)&A.hash_a[a], (unsigned long long)acc.hsum);
        } else if (mode == kAdd) {
            for (int i = 0; i < 6; i++) A.maa[(int64_t)i * K + a] += acc.maa[i];
            A.qp_a[a] += acc.qp;
            A.cnt_a[a] += acc.cnt;
            if (want_stats<STS>(A)) A.hash_a[a] += acc.hsum;
        } else {
            for (int i = 0; i < 6; i++) A.maa[(int64_t)i * K + a] = acc.maa[i];
            A.qp_a[a] = acc.qp;
            A.cnt_a[a] = acc.cnt;
            if (want_stats<STS>(A)) A.hash_a[a] = acc.hsum;
        }
    }
}

// five resident 4-warp blocks per SM with float sums (96 registers); double sums unconstrained
template <typename T, int STS = -1, int KIN = -1>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, sizeof(T) == sizeof(float) ? 5 : 1) k_interior(const NumArgs A)
{
    __shared__ OuterPt sq_all[kWarpsPerBlock][NL_MAXQ + 8];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int a = blockIdx.x * kWarpsPerBlock + wib;
    if (a >= A.K) return;
    OuterPt *sq = sq_all[wib];
    stage_outer(A, a, sq, lane);
    __syncwarp();
    LaneAcc acc;
    acc_zero(acc);
    interior_outer<T, STS, KIN>(A, a, sq, lane, acc);
    finish_outer<STS>(A, a, acc, lane, kAtomicAdd);
}

// ---------------------------------------------------------------------------
// Boundary pairs.  32 candidates at a time (one per lane): every (q, b) is classified
// in FP32 in lockstep; whole items, near-field items (singular kernel) and undecided items
// go to warp queues that all 32 lanes then drain together (geometry + quadrature), adding
// their blocks into the owner lane's column of a shared accumulator.  Items whose region
// the FP64 geometry has to build are queued for k_deferred instead.
// ---------------------------------------------------------------------------
// FP32 data of a candidate T_b (64 bytes a lane, in shared memory); the rare FP64 paths
// read T_b's FP64 vertices, barycentre and area from global memory (cand_fp64).
struct CandData {
    float vlx[3], vly[3];      // T_b relative to bary_a
    float blx, bly;            // bary_b relative to bary_a
    float e1x, e1y, e2x, e2y, binv;
    float akcf;                // |T_b| times the kernel constant
    int b, q0;
};

struct CandFp64 {
    D2 V[3], bb;
    double area;
};

// bary_a as FP32 hi + lo pairs (x hi, x lo, y hi, y lo)
__device__ __forceinline__ float4 bary_hilo(const NumArgs &A, int a)
{
    const int64_t K = A.K;
    return make_float4(A.hl[12 * K + a], A.hl[13 * K + a], A.hl[14 * K + a], A.hl[15 * K + a]);
}

// FP32 data of candidate T_b relative to bary_a (ba, and bah its hi + lo pairs) and the
// outer-rule range [c.q0, q1) of the pair.  Each FP32 difference is (hi - hi) + (lo - lo): within
// 2u of the difference of the FP64 values (u = 2^-24), with no FP64 arithmetic.
__device__ __forceinline__ void load_cand(const NumArgs &A, int b, const D2 &ba, const float4 &bah, CandData &c,
                                          int &q1)
{
    const int64_t K = A.K;
    const float *H = A.hl;
    c.b = b;
    float xh[3], xl[3], yh[3], yl[3];
    for (int i = 0; i < 3; i++) {
        xh[i] = H[i * K + b];
        xl[i] = H[(3 + i) * K + b];
        yh[i] = H[(6 + i) * K + b];
        yl[i] = H[(9 + i) * K + b];
    }
    c.akcf = A.akc[b];
    for (int i = 0; i < 3; i++) {
        c.vlx[i] = (xh[i] - bah.x) + (xl[i] - bah.y);
        c.vly[i] = (yh[i] - bah.z) + (yl[i] - bah.w);
    }
    c.blx = (H[12 * K + b] - bah.x) + (H[13 * K + b] - bah.y);
    c.bly = (H[14 * K + b] - bah.z) + (H[15 * K + b] - bah.w);
    c.e1x = (xh[1] - xh[0]) + (xl[1] - xl[0]);
    c.e1y = (yh[1] - yh[0]) + (yl[1] - yl[0]);
    c.e2x = (xh[2] - xh[0]) + (xl[2] - xl[0]);
    c.e2y = (yh[2] - yh[0]) + (yl[2] - yl[0]);
    c.binv = 1.f / (c.e1x * c.e2y - c.e2x * c.e1y);
    int q0 = 0;
    q1 = A.outer.n;
    if (A.switch47) rule_range(A, ba, D2{A.bx[b], A.by[b]}, q0, q1);
    c.q0 = q0;
}

__device__ __forceinline__ CandFp64 cand_fp64(const NumArgs &A, int b)
{
    CandFp64 c;
    for (int i = 0; i < 3; i++) { c.V[i].x = A.tx[i * A.K + b]; c.V[i].y = A.ty[i * A.K + b]; }
    c.bb.x = A.bx[b];
    c.bb.y = A.by[b];
    c.area = A.area[b];
    return c;
}

// |T_b| kc in the quadrature type
template <typename T>
__device__ __forceinline__ T cand_akc(const NumArgs &A, const CandData &c)
{
    return sizeof(T) == sizeof(float) ? (T)c.akcf : (T)(A.area[c.b] * A.kc);
}

// longest edge of T_b in FP32 (the near field of the singular kernel)
__device__ __forceinline__ float cand_diam(const CandData &c)
{
    const float e3x = c.e2x - c.e1x, e3y = c.e2y - c.e1y;
    return sqrtf(fmaxf(fmaxf(c.e1x * c.e1x + c.e1y * c.e1y, c.e2x * c.e2x + c.e2y * c.e2y), e3x * e3x + e3y * e3y));
}

// Per-warp shared memory of the boundary kernel, sized for outer rules of at most NL_MAXQ
// points (14.2 KB with float sums: four 4-warp blocks fit an SM).
// fan triangles of a round of 32 polygon regions at most: a region has at most nlg::kBallCap = 16
// vertices (approxcaps with m <= 4 has 15, nocaps 6, an N-gon clip kClipCap = 8), 14 triangles
constexpr int kFanTasks = 32 * (nlg::kBallCap - 2);

template <typename T>
struct BoundaryShared {
    OuterPt sq[NL_MAXQ];
    CandData cand[32];
    T acc[16][32];             // M_ab (rows 0-8) and upper M_bb (9-14) of each lane's pair (FP32 sums: fixed
                               // point) and its non-empty flag (row 15), value-major: the owners of one
                               // atomic instruction hit distinct banks
    // per outer point x_q: the sum of s0 over the outer triangle's items, from which M_aa =
    // sum_q W_q phi_a(x_q) phi_a(x_q)^T s0q[q] (FP32 sums: fixed point on the grid s0q_grid)
    typename std::conditional<sizeof(T) == sizeof(float), int, T>::type s0q[NL_MAXQ];
    unsigned short queue[32 * NL_MAXQ];    // undecided items (owner lane << 8 | q)
    unsigned dmask[32];        // outer points of each lane's candidate whose item the deferred kernel takes
    // whole items from the front; whole items in the singular kernel's near field from the back
    // (a batch holds at most 32 x n_q items in all)
    unsigned short wqueue[32 * NL_MAXQ];
    int fstart[32];            // spread fans: first fan triangle of each lane's item in the round's list
    unsigned char fwhich[32];  // spread fans: the clip buffer that holds each lane's polygon
    unsigned char ftask[kFanTasks];   // spread fans: the lane whose item holds each fan triangle
    nlg::ClipBuf clip;         // per-lane FP32 clip buffers
};

constexpr int kQueueCap = 32 * NL_MAXQ;

template <int BALL, typename T>
__device__ __forceinline__ int classify_item(const NumArgs &A, const CandData &c, const OuterPt &o, nlg::F2 dl[3])
{
    for (int i = 0; i < 3; i++) { dl[i].x = c.vlx[i] - o.lx; dl[i].y = c.vly[i] - o.ly; }
    if (BALL == NL_BALL_BARYCENTER) {
        float bx = c.blx - o.lx, by = c.bly - o.ly, r2 = bx * bx + by * by;
        return r2 <= A.geo.b_in2 ? nlg::CLS_WHOLE : (r2 >= A.geo.b_out2 ? nlg::CLS_EMPTY : nlg::CLS_EXACT);
    }
    if (BALL == NL_BALL_OVERLAP) {
        float r0 = dl[0].x * dl[0].x + dl[0].y * dl[0].y, r1 = dl[1].x * dl[1].x + dl[1].y * dl[1].y;
        float r2 = dl[2].x * dl[2].x + dl[2].y * dl[2].y;
        if (fminf(r0, fminf(r1, r2)) <= A.geo.rin_m2) return nlg::CLS_WHOLE;
        if (nlg::dist2_origin_triangle(dl) > A.geo.rout_p2) return nlg::CLS_EMPTY;
        return nlg::CLS_EXACT;
    }
    return nlg::classify_vertices(dl, A.geo.rin_m2, A.geo.rout_p2);
}

// one undecided (q, b): build the region exactly as the FP64 geometry would and integrate it
template <int BALL, typename T>
__device__ __noinline__ bool exact_item_fp64(const NumArgs &A, const CandData &c, const OuterPt &o, Sums<T> &S,
                                             int64_t &nq, int &kind, int &nv, int &ncap, nlg::ClipBuf &cb,
                                             int lane);

// inner sums over fan triangle k (vertices 0, k, k + 1) of a polygon held in columns px / py, in
// FP32 coordinates relative to x (FP32 path; KIN as for whole_sums)
template <int KIN = -1>
__device__ __forceinline__ void fan_tri_sums(const NumArgs &A, nlg::Col px, nlg::Col py, int k, const nlg::F2 &d0,
                                             const nlg::F2 &e1, const nlg::F2 &e2, float inv_det, Sums<float> &S)
{
    sums_zero(S);
    const float kc = A.kcf;
    auto phi = [&](float x, float y, float f[3]) {
        const float rx = x - d0.x, ry = y - d0.y;
        const float l1 = (rx * e2.y - e2.x * ry) * inv_det;
        const float l2 = (e1.x * ry - rx * e1.y) * inv_det;
        f[0] = 1.f - l1 - l2;
        f[1] = l1;
        f[2] = l2;
    };
    const float x0 = px[0], y0 = py[0], xk = px[k], yk = py[k], xn = px[k + 1], yn = py[k + 1];
    float f0[3], fk[3], fn[3];
    phi(x0, y0, f0);
    phi(xk, yk, fk);
    phi(xn, yn, fn);
    const float ar = 0.5f * fabsf((xk - x0) * (yn - y0) - (xn - x0) * (yk - y0)) * kc;
    const int nr = A.inner.n;
    for (int r = 0; r < nr; r++) {
        const float4 f = A.fin[r];
        const float m0 = f.x, m1 = f.y, m2 = f.z;
        const float p0 = m0 * f0[0] + m1 * fk[0] + m2 * fn[0];
        const float p1 = m0 * f0[1] + m1 * fk[1] + m2 * fn[1];
        const float p2 = m0 * f0[2] + m1 * fk[2] + m2 * fn[2];
        float w = f.w * ar;
        if (KIN < 0 ? A.kernel == NL_KERNEL_INV_DIST : KIN == 1) {   // psi = c / |y - x|, relative to x
            const float yx = m0 * x0 + m1 * xk + m2 * xn, yy = m0 * y0 + m1 * yk + m2 * yn;
            w *= rsqrtf(yx * yx + yy * yy);
        }
        sums_add<float>(S, w, p0, p1, p2);
    }
}

// FP32 region of one undecided (q, b) of the balls whose region is a polygon (N-gon, nocaps,
// approxcaps), left in the lane's clip-buffer column (buffer *which): 1 with its vertex count n
// and kind, 0 empty, -1 the FP64 geometry decides (as exact_item_f32)
template <int BALL, bool INV>
__device__ __forceinline__ int exact_region_f32(const NumArgs &A, const CandData &c, const OuterPt &o,
                                                nlg::ClipBuf &cb, int lane, int &n, int &kind, int &which)
{
    nlg::F2 dl[3];
    for (int i = 0; i < 3; i++) { dl[i].x = c.vlx[i] - o.lx; dl[i].y = c.vly[i] - o.ly; }
    if (INV && nlg::near_f32(dl, cand_diam(c), A.geo.tau) != 0) return -1;
    which = 0;
    if (BALL == NL_BALL_NGON) {
        bool cut = false;
        n = nlg::clip_ngon_f32_sh<!INV>(dl, A.geo.err0, A.geo, cb, lane, &which, &cut);
        if (n < 0) return -1;
        if (n < 3) return 0;
        kind = cut ? nlg::KIND_PARTIAL : nlg::KIND_WHOLE;
        return 1;
    }
    kind = nlg::KIND_PARTIAL;
    n = nlg::ball_region_f32<BALL>(dl, A.geo, cb, lane, &kind);
    if (n < 0) return -1;
    return n >= 3 ? 1 : 0;
}

// FP32 region and quadrature of one undecided (q, b) of the balls the boundary kernel drains a
// lane per item (the N-gon's items go through exact_region_f32 and the spread fans): 1 done (S
// holds its sums), 0 empty region, -1 the FP64 geometry decides (the singular kernel's near
// field, an uncertified FP32 choice, FP64 sums or a ball without an FP32 region)
template <int BALL, typename T, bool INV>
__device__ __forceinline__ int exact_item_f32(const NumArgs &A, const CandData &c, const OuterPt &o, Sums<T> &S,
                                              int64_t &nq, int &kind, int &nv, int &ncap, nlg::ClipBuf &cb, int lane)
{
    if (sizeof(T) == sizeof(float) && (BALL == NL_BALL_NOCAPS || BALL == NL_BALL_APPROXCAPS)) {
        nlg::F2 dl[3];
        for (int i = 0; i < 3; i++) { dl[i].x = c.vlx[i] - o.lx; dl[i].y = c.vly[i] - o.ly; }
        if (INV && nlg::near_f32(dl, cand_diam(c), A.geo.tau) != 0)
            return -1;
        int k = nlg::KIND_PARTIAL;
        const int n = nlg::ball_region_f32<BALL>(dl, A.geo, cb, lane, &k);
        if (n >= 0) {
            // certified FP32 walk: same vertex count and kind as the FP64 walk
            if (n < 3) return 0;
            kind = k;
            nv = n;
            ncap = 0;
            if (k == nlg::KIND_WHOLE) {
                const D2 Vb[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};   // unused: FP32 coordinates dl
                whole_sums<T, INV>(A, Vb, cand_akc<T>(A, c), D2{o.x, o.y}, S, nq, dl);
            } else {
                const nlg::F2 e1 = {c.e1x, c.e1y}, e2 = {c.e2x, c.e2y};
                poly_sums_col<INV>(A, nlg::col(cb.x, lane), nlg::col(cb.y, lane), n, dl[0], e1, e2, c.binv,
                                   *(Sums<float> *)&S, nq);
            }
            return 1;
        }
    }
    if (sizeof(T) == sizeof(float) && BALL == NL_BALL_EXACTCAPS) {
        nlg::F2 dl[3];
        for (int i = 0; i < 3; i++) { dl[i].x = c.vlx[i] - o.lx; dl[i].y = c.vly[i] - o.ly; }
        if (INV && nlg::near_f32(dl, cand_diam(c), A.geo.tau) != 0)
            return -1;
        int nc = 0, k = nlg::KIND_PARTIAL;
        const int n = nlg::exactcaps_region_f32(dl, A.geo, cb, lane, &nc, &k);
        const nlg::Col px = nlg::col(cb.x, lane), py = nlg::col(cb.y, lane), pe = nlg::col(cb.e, lane);
        if (n >= 0) {
            // certified FP32 walk: the vertex count, the caps and the kind of the FP64 region
            if (n < 3 && nc == 0) return 0;
            kind = k;
            nv = n;
            ncap = nc;
            if (k == nlg::KIND_WHOLE) {
                const D2 Vb[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};   // unused: FP32 coordinates dl
                whole_sums<T, INV>(A, Vb, cand_akc<T>(A, c), D2{o.x, o.y}, S, nq, dl);
            } else {
                Sums<float> &Sf = *(Sums<float> *)&S;
                const nlg::F2 e1 = {c.e1x, c.e1y}, e2 = {c.e2x, c.e2y};
                if (n >= 3) poly_sums_col<INV>(A, px, py, n, dl[0], e1, e2, c.binv, Sf, nq);
                else sums_zero(Sf);
                for (int j = 0; j < nc; j++) {   // one point per cap: its centroid, weight its area
                    const float cx = px[8 + j], cy = py[8 + j];
                    const float rx = cx - dl[0].x, ry = cy - dl[0].y;
                    const float l1 = (rx * e2.y - e2.x * ry) * c.binv, l2 = (e1.x * ry - rx * e1.y) * c.binv;
                    float w = pe[j] * A.kcf;
                    if (INV) w *= rsqrtf(cx * cx + cy * cy);
                    sums_add<float>(Sf, w, 1.f - l1 - l2, l1, l2);
                    nq++;
                }
            }
            return 1;
        }
    }
    return -1;
}

// undecided item through the FP64 geometry (the region exactly as FP64 builds it)
template <int BALL, typename T>
__device__ __noinline__ bool exact_item_fp64(const NumArgs &A, const CandData &c, const OuterPt &o, Sums<T> &S,
                                             int64_t &nq, int &kind, int &nv, int &ncap, nlg::ClipBuf &cb,
                                             int lane)
{
    nlg::F2 dl[3];
    for (int i = 0; i < 3; i++) { dl[i].x = c.vlx[i] - o.lx; dl[i].y = c.vly[i] - o.ly; }
    const CandFp64 c64 = cand_fp64(A, c.b);
    const D2 *Vb = c64.V;
    const D2 x = {o.x, o.y};
    kind = nlg::KIND_WHOLE;
    nv = 3;
    ncap = 0;
    nlg::Region R;
    nlg::make_region<BALL>(Vb, dl, c64.bb, x, A.geo, R);
    if (R.overflow) atomicOr(A.err, 1);
    if (R.kind == nlg::KIND_NONE) return false;
    kind = R.kind;
    nv = R.nv;
    ncap = R.ncap;
    if (R.kind == nlg::KIND_WHOLE && R.ncap == 0 && A.kernel != NL_KERNEL_INV_DIST) {
        whole_sums<T>(A, Vb, (T)(c64.area * A.kc), x, S, nq);
    } else if (sizeof(T) == sizeof(float) && R.ncap == 0 && R.nv <= nlg::kClipCap &&
               (A.kernel == NL_KERNEL_CONST || !nlg::is_near(R, Vb, x))) {
        // FP32 quadrature on the FP64 polygon (coordinates relative to x)
        for (int i = 0; i < R.nv; i++) {
            cb.x[0][i][lane] = (float)(R.P[i].x - x.x);
            cb.y[0][i][lane] = (float)(R.P[i].y - x.y);
        }
        const nlg::F2 d0 = {(float)(Vb[0].x - x.x), (float)(Vb[0].y - x.y)};
        const nlg::F2 e1 = {c.e1x, c.e1y}, e2 = {c.e2x, c.e2y};
        poly_sums_sh(A, cb, 0, lane, R.nv, d0, e1, e2, c.binv, *(Sums<float> *)&S, nq);
    } else if (sizeof(T) == sizeof(float) && A.kernel == NL_KERNEL_INV_DIST && R.kind == nlg::KIND_WHOLE &&
               R.ncap == 0) {
        // a whole T_b in the singular kernel's near field (decided by the FP64 test): the FP32
        // near rule, as k_near integrates the near-field items that FP32 decides
        const nlg::F2 e1 = {c.e1x, c.e1y}, e2 = {c.e2x, c.e2y};
        near_whole_f32(A, dl, c.b, x, e1, e2, c.binv, *(Sums<float> *)&S, nq);
    } else {
        inner_sums<T>(A, R, Vb, c64.area, x, S, nq);
    }
    return true;
}

// ---------------------------------------------------------------------------
// Pair sums of the FP32 boundary kernel in fixed point.  The M_ab and upper M_bb sums of a pair
// (rows 0..14 of the shared accumulator) are 32-bit integers on a grid of 2^-p, a power of two
// per pair chosen from a bound on the pair's sums.  Every item rounds its 15 values to that
// grid and adds them with integer arithmetic (native shared-memory atomics), so a pair's sums do
// not depend on the order in which the lanes add them: the blocks are the same in every run.
// Bound: an item (x_q, T_b) adds W_q la_i s1_j to M_ab and W_q S2_jk to M_bb; with |la_i| <= L_q
// (the outer point's barycentrics) and 0 <= S2_jk, s1_j <= s0 (inner barycentrics in [0, 1] up to
// rounding) every sum of the pair is at most B_a s0max, B_a = sum_q |W_q| max(1, L_q).  The region
// lies in T_b, so s0max = kc |T_b| for a constant kernel; for c / |x - y| the integral over T_b is
// at most c 2 sqrt(pi |T_b|) (the disc of the same area centred at x), taken twice more for the
// quadrature's error.  The bound, rounded up to a power of two 2^e, maps to 2^29: a rounding error
// of at most 2^-30 of it per item, and sums far from the 2^31 range unless the bound is broken
// (|sum| >= 2^30 sets error bit 256).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float fx_outer_bound(const OuterPt *sq, int n)
{
    float b = 0.f;
    for (int q = 0; q < n; q++) {
        const float l = fmaxf(1.f, fmaxf(fabsf(sq[q].l0f), fmaxf(fabsf(sq[q].l1f), fabsf(sq[q].l2f))));
        b += fabsf(sq[q].Wf) * l;
    }
    return b * 1.0001f;   // above its own rounding
}

// grid scale 2^(29 - e) of a pair (outer bound bwa, |T_b| kc = akcf)
template <bool INV>
__device__ __forceinline__ float fx_scale(float bwa, float akcf, float kcf)
{
    const float r = INV ? bwa * 4.f * sqrtf(3.14159265f * kcf * akcf) : bwa * akcf;
    const int e = ((__float_as_int(fmaxf(r, 1e-25f)) >> 23) & 0xff) - 126;   // r < 2^e
    return __int_as_float((127 + 29 - e) << 23);
}

// rows 0..14 of an item's block w into owner own's column: integer atomics on the grid of scale
// fxs (FP32 sums), float atomics (FP64 sums)
template <typename T>
__device__ __forceinline__ void pair_add_atomic(T (*dst)[32], int own, const T *w, float fxs)
{
    if constexpr (sizeof(T) == sizeof(float)) {
        for (int k = 0; k < 15; k++) atomicAdd(reinterpret_cast<int *>(&dst[k][own]), __float2int_rn(w[k] * fxs));
    } else {
        (void)fxs;
        for (int k = 0; k < 15; k++) atomicAdd(&dst[k][own], w[k]);
    }
}

// the same by the owner lane itself, while no other lane adds to its column
template <typename T>
__device__ __forceinline__ void pair_add_owner(T (*dst)[32], int own, const T *w, float fxs)
{
    if constexpr (sizeof(T) == sizeof(float)) {
        for (int k = 0; k < 15; k++) *reinterpret_cast<int *>(&dst[k][own]) += __float2int_rn(w[k] * fxs);
    } else {
        (void)fxs;
        for (int k = 0; k < 15; k++) dst[k][own] += w[k];
    }
}

// An item's s0 onto its outer point's sum (M_aa of the outer triangle): fixed point (FP32 sums)
template <typename T, typename S0>
__device__ __forceinline__ void s0q_add(S0 *s0q, int q, T s0, float grid)
{
    if constexpr (sizeof(T) == sizeof(float)) atomicAdd(&s0q[q], __float2int_rn(s0 * grid));
    else atomicAdd(&s0q[q], s0);
}

// An item's block (combine of its sums S at outer point x_q = o) added as it is formed: rows
// 0..14 onto owner own's column (as pair_add_atomic), the flag, and s0 onto the outer point's
// sum.  No 21-value array stays live across the adds.
template <typename T, typename S0>
__device__ __forceinline__ void block_add(const OuterPt &o, const Sums<T> &S, T (*accum)[32], S0 *s0q, int own, int q,
                                          float fxs, float grid)
{
    const bool f32 = sizeof(T) == sizeof(float);
    const T W = f32 ? (T)o.Wf : (T)o.W, la0 = f32 ? (T)o.l0f : (T)o.l0;
    const T la1 = f32 ? (T)o.l1f : (T)o.l1, la2 = f32 ? (T)o.l2f : (T)o.l2;
    auto put = [&](int k, T v) {
        if constexpr (sizeof(T) == sizeof(float)) atomicAdd(reinterpret_cast<int *>(&accum[k][own]), __float2int_rn(v * fxs));
        else atomicAdd(&accum[k][own], v);
    };
    const T wa0 = W * la0, wa1 = W * la1, wa2 = W * la2;
    put(0, wa0 * S.s1[0]); put(1, wa0 * S.s1[1]); put(2, wa0 * S.s1[2]);
    put(3, wa1 * S.s1[0]); put(4, wa1 * S.s1[1]); put(5, wa1 * S.s1[2]);
    put(6, wa2 * S.s1[0]); put(7, wa2 * S.s1[1]); put(8, wa2 * S.s1[2]);
    put(9, W * S.S2[0]); put(10, W * S.S2[1]); put(11, W * S.S2[2]);
    put(12, W * S.S2[3]); put(13, W * S.S2[4]); put(14, W * S.S2[5]);
    accum[15][own] = (T)1;
    s0q_add<T>(s0q, q, S.s0, grid);
}

// Add rows 0..14 of a block w to owner own's column of the shared accumulator; am = the lanes
// that call this (all of them do; own < 0: a lane without a block).  Lanes with the same owner
// first sum their blocks by shuffles (the leader takes its peers' values one by one, in lane
// order), so one lane per owner adds: no shared atomics colliding on one address.  FP32 sums are
// rounded to the owner's grid first and summed as integers: the same sum for any grouping.
template <typename T>
__device__ __forceinline__ void warp_owner_add(T (*accum)[32], int own, int lane, const T *w, float fxs,
                                               unsigned am)
{
    using V = typename std::conditional<sizeof(T) == sizeof(float), int, T>::type;
    V x[15];
    for (int k = 0; k < 15; k++) {
        if constexpr (sizeof(T) == sizeof(float)) x[k] = __float2int_rn(w[k] * fxs);
        else x[k] = w[k];
    }
    __syncwarp(am);
    const unsigned peers = __match_any_sync(am, own);
    const int m = own >= 0 ? __popc(peers) : 0, leader = __ffs(peers) - 1;
    const int mmax = (int)__reduce_max_sync(am, (unsigned)m);
    for (int t = 1; t < mmax; t++) {
        unsigned rest = peers;
        for (int j = 0; j < t && rest; j++) rest &= rest - 1;
        const bool take = lane == leader && t < m;
        const int src = take ? __ffs(rest) - 1 : lane;
        for (int k = 0; k < 15; k++) {
            const V y = __shfl_sync(am, x[k], src);
            if (take) x[k] += y;
        }
    }
    if (own >= 0 && lane == leader) {
        for (int k = 0; k < 15; k++) atomicAdd(reinterpret_cast<V *>(&accum[k][own]), x[k]);
        accum[15][own] = (T)1;
    }
}

// Mark an item (owner own, outer point q) for k_deferred: false (the caller runs the FP64 code
// itself) for FP64 sums or without a queue.  The marks of a round are queued together by
// defer_flush, in (owner, q) order.
template <typename T>
__device__ __forceinline__ bool defer_mark(const NumArgs &A, BoundaryShared<T> &sh, int own, int q)
{
    if (sizeof(T) != sizeof(float) || !A.defer) return false;
    atomicOr(&sh.dmask[own], 1u << q);
    return true;
}

// Queue the round's marked items with one reservation for the warp, ordered by owner lane and
// outer point: the items of one pair are contiguous and in q order, so k_defer_merge adds them
// onto the pair in a fixed order (run-to-run identical FP32 values).  Items past the queue's
// capacity are integrated here, by their owner lane with the FP64 geometry, into its column of
// the accumulator.
template <int BALL, typename T>
__device__ __forceinline__ void defer_flush(const NumArgs &A, int a, int64_t base, BoundaryShared<T> &sh, int lane,
                                            float fxs, LaneAcc &acc)
{
    const unsigned m = sh.dmask[lane];
    const int cnt = __popc(m);
    int inc = cnt;
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    const int total = __shfl_sync(0xffffffffu, inc, 31);
    if (total == 0) return;
    sh.dmask[lane] = 0;
    int slot0 = 0;
    if (lane == 0) slot0 = atomicAdd(A.defer_n, total);
    slot0 = __shfl_sync(0xffffffffu, slot0, 0);
    int slot = slot0 + inc - cnt;
    for (unsigned rest = m; rest; rest &= rest - 1, slot++) {
        const int q = __ffs(rest) - 1;
        if (slot < A.defer_cap) {
            A.defer[slot] = DeferItem{base + lane, a, (A.prob << 8) | q};
            continue;
        }
        // queue full: this lane integrates its own item
        const CandData &cd = sh.cand[lane];
        const OuterPt &o = sh.sq[q];
        Sums<T> S;
        int64_t nq = 0;
        int kind, nv, ncap;
        if (!exact_item_fp64<BALL, T>(A, cd, o, S, nq, kind, nv, ncap, sh.clip, lane)) continue;
        T w[21];
        for (int k = 0; k < 21; k++) w[k] = 0;
        combine<T>(o, S, w);
        pair_add_owner<T>(sh.acc, lane, w, fxs);
        sh.acc[15][lane] = (T)1;
        s0q_add<T>(sh.s0q, q, S.s0, A.s0q_grid);
        acc.cnt++;
        acc.qp += nq;
        if (A.stats) acc.hsum += nlg::record_hash(a, cd.b, q - cd.q0, kind, nv, ncap);
    }
}

// A near-field whole item integrated by its owner lane into its own column of the shared
// accumulator (the near-field queue is full).  Not inlined: the boundary kernel's code stays
// free of the near rule, which runs in k_near.
template <typename T>
__device__ __noinline__ int64_t near_inline(const NumArgs &A, const CandData &cd, int q, BoundaryShared<T> &sh,
                                            int lane, float fxs)
{
    const OuterPt &o = sh.sq[q];
    nlg::F2 dl[3];
    for (int k = 0; k < 3; k++) { dl[k].x = cd.vlx[k] - o.lx; dl[k].y = cd.vly[k] - o.ly; }
    Sums<float> S;
    int64_t nq = 0;
    const nlg::F2 e1 = {cd.e1x, cd.e1y}, e2 = {cd.e2x, cd.e2y};
    near_whole_f32(A, dl, cd.b, D2{o.x, o.y}, e1, e2, cd.binv, S, nq);
    float w[21];
    for (int k = 0; k < 21; k++) w[k] = 0.f;
    combine<float>(o, S, w);
    T wt[21];
    for (int k = 0; k < 21; k++) wt[k] = (T)w[k];
    pair_add_owner<T>(sh.acc, lane, wt, fxs);
    sh.acc[15][lane] = (T)1;
    s0q_add<T>(sh.s0q, q, (T)S.s0, A.s0q_grid);
    return nq;
}

// Queue the near-field whole items of this lane's candidate (outer points m, bit q) for k_near,
// one reservation for the warp, in (owner, q) order; past the queue's capacity the lane
// integrates them itself.
template <typename T>
__device__ __forceinline__ void near_flush(const NumArgs &A, int a, int64_t base, unsigned m, BoundaryShared<T> &sh,
                                           float fxs, int lane, LaneAcc &acc)
{
    const int cnt = __popc(m);
    int inc = cnt;
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    const int total = __shfl_sync(0xffffffffu, inc, 31);
    if (total == 0) return;
    int slot0 = 0;
    if (lane == 0) slot0 = atomicAdd(A.near_n, total);
    slot0 = __shfl_sync(0xffffffffu, slot0, 0);
    int slot = slot0 + inc - cnt;
    for (unsigned rest = m; rest; rest &= rest - 1, slot++) {
        const int q = __ffs(rest) - 1;
        if (slot < A.near_cap) {
            A.nearq[slot] = DeferItem{base + lane, a, (A.prob << 8) | q};
            continue;
        }
        const CandData &cd = sh.cand[lane];
        acc.cnt++;
        acc.qp += near_inline<T>(A, cd, q, sh, lane, fxs);
        if (A.stats) acc.hsum += nlg::record_hash(a, cd.b, q - cd.q0, nlg::KIND_WHOLE, 3, 0);
    }
}

// The boundary candidates of outer triangle a (outer points staged in sh.sq).
// INV: the kernel is psi = c/|x - y| (near-field split), else the constant kernel.
template <int BALL, typename T, bool INV, bool NQ = false, int STS = -1>
__device__ __forceinline__ void boundary_outer(const NumArgs &A, int a, BoundaryShared<T> &sh, int lane,
                                               LaneAcc &acc)
{
    const int K = A.K;
    const D2 ba = {A.bx[a], A.by[a]};
    const float4 bah = bary_hilo(A, a);
    const int64_t es = A.nbr_split[a], e1 = A.nbr_ptr[a + 1];
    // M_aa belongs to the outer triangle, not to the pair: it is W_q phi_a phi_a^T times the sum of
    // s0 over all items of x_q, so the items only add their s0 onto their outer point's sum
    // (sh.s0q) and M_ab and M_bb (rows 0-14) onto the owner's column
    const int nq_all = A.outer.n;
    // FP32 sums: the outer bound of the pairs' fixed-point grids
    const float fx_bwa = sizeof(T) == sizeof(float) ? fx_outer_bound(sh.sq, nq_all) : 0.f;
    const bool inv = INV;
    for (int q = lane; q < NL_MAXQ; q += 32) sh.s0q[q] = 0;
    __syncwarp();
    for (int64_t base = es; base < e1; base += 32) {
        const int64_t e = base + lane;
        const bool valid = e < e1;
        int q0 = 0, q1 = 0;
        CandData c;
        if (valid) {
            int b = A.nbr_idx[e];
#ifdef NL_CHECKS
            if (b < 0 || b >= K) {   // debug build: bad candidate recorded (bit 16), replaced by a
                atomicOr(A.err, 16);
                b = a;
            }
#endif
            load_cand(A, b, ba, bah, c, q1);
            q0 = c.q0;
            sh.cand[lane] = c;
        }
        for (int i = 0; i < 16; i++) sh.acc[i][lane] = 0;
        sh.dmask[lane] = 0;
        int nqueue = 0;
        __syncwarp();
        // phase 1: classify every (q, b) in lockstep; queue whole and undecided items.  With a
        // near-field queue (FP32 singular kernel), the near-field whole items of this lane's
        // candidate are only marked (my_near, bit q) and handed to k_near after the round.
        constexpr bool split_near = INV && NQ && sizeof(T) == sizeof(float);
        unsigned my_near = 0;
        int nwhole = 0, nnear = 0;
        for (int q = 0; q < nq_all; q++) {
            const bool active = valid && q >= q0 && q < q1;
            int cls = nlg::CLS_EMPTY;
            if (active) {
                nlg::F2 dl[3];
                cls = classify_item<BALL, T>(A, c, sh.sq[q], dl);
                // singular kernel: whole items in the near field take the near rule (certified
                // in FP32; undecided ones the FP64 path)
                if (inv && cls == nlg::CLS_WHOLE) {
                    const int nr = nlg::near_f32(dl, cand_diam(c), A.geo.tau);
                    cls = nr == 0 ? nlg::CLS_WHOLE : (nr == 1 && sizeof(T) == sizeof(float) ? 3 : nlg::CLS_EXACT);
                    if (cls == 3 && split_near) {
                        my_near |= 1u << q;
                        cls = nlg::CLS_EMPTY;
                    }
                }
            }
            const unsigned mw = __ballot_sync(0xffffffffu, cls == nlg::CLS_WHOLE);
            const unsigned me = __ballot_sync(0xffffffffu, cls == nlg::CLS_EXACT);
            const unsigned mn = __ballot_sync(0xffffffffu, cls == 3);
            const unsigned below = (1u << lane) - 1u;
            const unsigned short item = (unsigned short)((lane << 8) | q);
            if (cls == nlg::CLS_WHOLE) sh.wqueue[nwhole + __popc(mw & below)] = item;
            if (cls == nlg::CLS_EXACT) sh.queue[nqueue + __popc(me & below)] = item;
            if (cls == 3) sh.wqueue[kQueueCap - 1 - (nnear + __popc(mn & below))] = item;
            nwhole += __popc(mw);
            nqueue += __popc(me);
            nnear += __popc(mn);
        }
        __syncwarp();
        // phase 2a: whole items with all lanes
        for (int i = lane; i < nwhole; i += 32) {
            const unsigned it = sh.wqueue[i];
            const int own = it >> 8, q = it & 0xff;
            const CandData &cd = sh.cand[own];
            const OuterPt &o = sh.sq[q];
            // FP64 vertices only where the FP64 quadrature of the singular kernel needs them
            D2 Vb[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
            if (INV && sizeof(T) == sizeof(double))
                for (int k = 0; k < 3; k++) { Vb[k].x = A.tx[k * K + cd.b]; Vb[k].y = A.ty[k * K + cd.b]; }
            Sums<T> S;
            int64_t nq = 0;
            nlg::F2 dl[3];
            if (INV)
                for (int k = 0; k < 3; k++) { dl[k].x = cd.vlx[k] - o.lx; dl[k].y = cd.vly[k] - o.ly; }
            whole_sums<T, INV>(A, Vb, cand_akc<T>(A, cd), D2{o.x, o.y}, S, nq, INV ? dl : nullptr);
            block_add<T>(o, S, sh.acc, sh.s0q, own, q, fx_scale<INV>(fx_bwa, cd.akcf, A.kcf), A.s0q_grid);
            acc.cnt++;
            acc.qp += nq;
            if (want_stats<STS>(A)) acc.hsum += nlg::record_hash(a, cd.b, q - cd.q0, nlg::KIND_WHOLE, 3, 0);
        }
        __syncwarp();
        // phase 2c: whole items in the singular kernel's near field (FP32 near rule)
        for (int i = lane; INV && !split_near && i < nnear; i += 32) {
            const int left = nnear - (i - lane);   // items of this round
            const unsigned rmask = left >= 32 ? 0xffffffffu : ((1u << left) - 1u);
            const unsigned it = sh.wqueue[kQueueCap - 1 - i];
            const int own = it >> 8, q = it & 0xff;
            const CandData &cd = sh.cand[own];
            const OuterPt &o = sh.sq[q];
            nlg::F2 dl[3];
            for (int k = 0; k < 3; k++) { dl[k].x = cd.vlx[k] - o.lx; dl[k].y = cd.vly[k] - o.ly; }
            Sums<T> S;
            int64_t nq = 0;
            const nlg::F2 e1 = {cd.e1x, cd.e1y}, e2 = {cd.e2x, cd.e2y};
            near_whole_f32(A, dl, cd.b, D2{o.x, o.y}, e1, e2, cd.binv, *(Sums<float> *)&S, nq);
            T w[21];
            for (int k = 0; k < 21; k++) w[k] = 0;
            combine<T>(o, S, w);
            // an owner lies in the near field of several outer points of one round: the lanes
            // with the same owner sum their blocks by shuffles, one lane per owner adds
            s0q_add<T>(sh.s0q, q, S.s0, A.s0q_grid);
            warp_owner_add<T>(sh.acc, own, lane, w, fx_scale<INV>(fx_bwa, cd.akcf, A.kcf), rmask);
            acc.cnt++;
            acc.qp += nq;
            if (want_stats<STS>(A)) acc.hsum += nlg::record_hash(a, cd.b, q - cd.q0, nlg::KIND_WHOLE, 3, 0);
        }
        // phase 2b: undecided items with all lanes.  The loop does not converge the warp between
        // items: lanes at different items run the same parts of the clip together.  So the order
        // in which their blocks reach an owner's column depends on the scheduling: FP32 sums are
        // integers there (the same for any order), FP64 blocks may differ in their last bits.
        // FP32 polygon regions of the N-gon (either kernel) and nocaps: a round of 32 items
        // builds its regions (a lane per item), then the warp spreads the fan triangles of all 32
        // polygons over its lanes, each adding its triangle's block onto the owner's column
        // (integer sums: any order), so the lanes stay busy although the fans have 1 to 4
        // triangles (nocaps boundary kernel of a K = 23328 problem 3.43 -> 2.20 ms; the N-gon's
        // numeric phase 5.63 -> 5.51 ms, with the singular kernel 15.9 -> 14.8 ms).  The fan is
        // the one the lane-per-item drain integrates (from the polygon's first vertex).  The
        // approxcaps fans (up to 13 triangles with the arc points) keep the lane-per-item drain:
        // a triangle's lookup and block add then cost about as much as its quadrature (2.68 ->
        // 3.08 ms spread, 2.95 ms with the owner table; tasks of two to five triangles of one fan
        // did not pay either).  The owner of each triangle comes from a per-round table
        // (`ftask`) instead of a binary search over the lanes' first triangles (the N-gon's
        // numeric phase 5.51 -> 5.38 ms).
        constexpr bool kSpread = sizeof(T) == sizeof(float) && (BALL == NL_BALL_NGON || (!INV && BALL == NL_BALL_NOCAPS));
        if constexpr (kSpread)
        for (int r0 = 0; r0 < nqueue; r0 += 32) {
            const int i = r0 + lane;
            int m = 0, which = 0;
            if (i < nqueue) {
                const unsigned it = sh.queue[i];
                const int own = it >> 8, q = it & 0xff;
                const CandData &cd = sh.cand[own];
                const OuterPt &o = sh.sq[q];
                int n = 0, kind = nlg::KIND_PARTIAL;
                const int r = exact_region_f32<BALL, INV>(A, cd, o, sh.clip, lane, n, kind, which);
                if (r > 0) {
                    m = n - 2;
                    acc.cnt++;
                    acc.qp += (uint32_t)(m * A.inner.n);
                    if (want_stats<STS>(A)) acc.hsum += nlg::record_hash(a, cd.b, q - cd.q0, kind, n, 0);
                } else if (r < 0 && !defer_mark<T>(A, sh, own, q)) {
                    Sums<T> S;
                    int64_t nq = 0;
                    int kd, nv, ncap;
                    if (exact_item_fp64<BALL, T>(A, cd, o, S, nq, kd, nv, ncap, sh.clip, lane)) {
                        block_add<T>(o, S, sh.acc, sh.s0q, own, q, fx_scale<INV>(fx_bwa, cd.akcf, A.kcf), A.s0q_grid);
                        acc.cnt++;
                        acc.qp += (uint32_t)nq;
                        if (want_stats<STS>(A)) acc.hsum += nlg::record_hash(a, cd.b, q - cd.q0, kd, nv, ncap);
                    }
                }
            }
            int incl = m;
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += y;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            sh.fstart[lane] = incl - m;
            sh.fwhich[lane] = (unsigned char)which;
            for (int j = incl - m; j < incl; j++) sh.ftask[j] = (unsigned char)lane;   // total <= kFanTasks
            __syncwarp();
            for (int t = lane; t < total; t += 32) {
                const int lo = sh.ftask[t];   // the lane whose item holds triangle t
                const int k = t - sh.fstart[lo] + 1;
                const unsigned it = sh.queue[r0 + lo];
                const int own = it >> 8, q = it & 0xff;
                const CandData &cd = sh.cand[own];
                const OuterPt &o = sh.sq[q];
                const int w = sh.fwhich[lo];
                const nlg::F2 d0 = {cd.vlx[0] - o.lx, cd.vly[0] - o.ly}, e1 = {cd.e1x, cd.e1y}, e2 = {cd.e2x, cd.e2y};
                Sums<float> S;
                fan_tri_sums<INV>(A, nlg::Col{&sh.clip.x[w][0][lo]}, nlg::Col{&sh.clip.y[w][0][lo]}, k, d0, e1, e2,
                                  cd.binv, S);
                block_add<float>(o, S, sh.acc, sh.s0q, own, q, fx_scale<INV>(fx_bwa, cd.akcf, A.kcf), A.s0q_grid);
            }
            __syncwarp();
        }
        if constexpr (!kSpread)
        for (int i = lane; i < nqueue; i += 32) {
            const unsigned it = sh.queue[i];
            const int own = it >> 8, q = it & 0xff;
            const CandData &cd = sh.cand[own];
            const OuterPt &o = sh.sq[q];
            Sums<T> S;
            int64_t nq = 0;
            int kind, nv, ncap;
            int r = exact_item_f32<BALL, T, INV>(A, cd, o, S, nq, kind, nv, ncap, sh.clip, lane);
            if (r < 0) {
                if (defer_mark<T>(A, sh, own, q)) continue;
                r = exact_item_fp64<BALL, T>(A, cd, o, S, nq, kind, nv, ncap, sh.clip, lane) ? 1 : 0;
            }
            if (r == 0) continue;
            block_add<T>(o, S, sh.acc, sh.s0q, own, q, fx_scale<INV>(fx_bwa, cd.akcf, A.kcf), A.s0q_grid);
            acc.cnt++;
            acc.qp += nq;
            if (want_stats<STS>(A)) acc.hsum += nlg::record_hash(a, cd.b, q - cd.q0, kind, nv, ncap);
        }
        __syncwarp();
        if (sizeof(T) == sizeof(float) && A.defer) {
            defer_flush<BALL, T>(A, a, base, sh, lane, fx_scale<INV>(fx_bwa, sh.cand[lane].akcf, A.kcf), acc);
            __syncwarp();
        }
        if constexpr (split_near) {
            near_flush<T>(A, a, base, my_near, sh, fx_scale<INV>(fx_bwa, sh.cand[lane].akcf, A.kcf), lane, acc);
            __syncwarp();
        }
        // phase 3: owners merge the queue's contributions and write their pair
        if (valid) {
            T v[15];
            if constexpr (sizeof(T) == sizeof(float)) {
                // back from the pair's grid (an exact power of two)
                const float inv_s = 1.f / fx_scale<INV>(fx_bwa, sh.cand[lane].akcf, A.kcf);
                bool big = false;
                for (int k = 0; k < 15; k++) {
                    const int iv = *reinterpret_cast<const int *>(&sh.acc[k][lane]);
                    big = big || iv >= (1 << 30) || iv <= -(1 << 30);
                    v[k] = (T)iv * inv_s;
                }
                if (big) atomicOr(A.err, 256);
            } else {
                for (int k = 0; k < 15; k++) v[k] = sh.acc[k][lane];
            }
            write_pair<T, false>(A, e, sh.cand[lane].b, sh.acc[15][lane] != (T)0, v, acc);
        }
        __syncwarp();
    }
    // M_aa = sum_q W_q phi_a(x_q) phi_a(x_q)^T s0q[q], in FP64, one outer point a lane
    for (int q = lane; q < nq_all; q += 32) {
        const OuterPt &o = sh.sq[q];
        if (sizeof(T) == sizeof(float) && (sh.s0q[q] >= (1 << 30) || sh.s0q[q] <= -(1 << 30))) atomicOr(A.err, 256);
        const double t = sizeof(T) == sizeof(float) ? (double)sh.s0q[q] / (double)A.s0q_grid : (double)sh.s0q[q];
        const double ws = o.W * t;
        acc.maa[0] += ws * o.l0 * o.l0; acc.maa[1] += ws * o.l1 * o.l1; acc.maa[2] += ws * o.l2 * o.l2;
        acc.maa[3] += ws * o.l0 * o.l1; acc.maa[4] += ws * o.l0 * o.l2; acc.maa[5] += ws * o.l1 * o.l2;
    }
}

// Boundary candidates of the outer-support barycenter balls (Sec. 6.2, barycenter case; the
// experiment of Table 3).  One lane per candidate T_b: the inner integral is over the whole T_b
// (the same sums for every outer point of the constant kernel), and the outer integrand lives on
// S = T_a n B_delta(bary_b), built by the disc walk of T_a around bary_b (nocaps / approxcaps;
// certified FP32 walk, else the FP64 walk), fanned from its first point; the outer rule runs on
// every subtriangle with phi_a taken at each outer point.  One record per pair with a non-empty S.
template <int BALL, typename T>
__device__ __forceinline__ void support_boundary(const NumArgs &A, int a, int lane, nlg::ClipBuf &cb, LaneAcc &acc)
{
    constexpr int DISC = (BALL == NL_BALL_BARY_NOCAPS) ? NL_BALL_NOCAPS : NL_BALL_APPROXCAPS;
    const int K = A.K;
    const D2 ba = {A.bx[a], A.by[a]};
    D2 Va[3];
    for (int i = 0; i < 3; i++) { Va[i].x = A.tx[i * K + a]; Va[i].y = A.ty[i * K + a]; }
    nlg::F2 va[3];   // T_a relative to bary_a
    for (int i = 0; i < 3; i++) { va[i].x = (float)(Va[i].x - ba.x); va[i].y = (float)(Va[i].y - ba.y); }
    const float f1x = va[1].x - va[0].x, f1y = va[1].y - va[0].y, f2x = va[2].x - va[0].x, f2y = va[2].y - va[0].y;
    const float finv = 1.f / (f1x * f2y - f2x * f1y);
    const BaryMap bma = bary_map(Va);
    const int64_t es = A.nbr_split[a], e1 = A.nbr_ptr[a + 1];
    for (int64_t e = es + lane; e < e1; e += 32) {
        const int b = A.nbr_idx[e];
        D2 Vb[3];
        for (int i = 0; i < 3; i++) { Vb[i].x = A.tx[i * K + b]; Vb[i].y = A.ty[i * K + b]; }
        const D2 bb = {A.bx[b], A.by[b]};
        int q0, q1;
        rule_range(A, ba, bb, q0, q1);
        Sums<T> S;
        int64_t nq_in = 0;
        whole_sums<T>(A, Vb, (T)(A.area[b] * A.kc), bb, S, nq_in);
        T v[21];
        for (int i = 0; i < 21; i++) v[i] = 0;
        int kind = nlg::KIND_NONE, nv = 0;
        int64_t nout = 0;
        bool done = false;
        if (sizeof(T) == sizeof(float)) {
            const float cbx = (float)(bb.x - ba.x), cby = (float)(bb.y - ba.y);
            nlg::F2 d[3];   // T_a relative to bary_b
            for (int i = 0; i < 3; i++) { d[i].x = va[i].x - cbx; d[i].y = va[i].y - cby; }
            int k = nlg::KIND_PARTIAL;
            const int n = nlg::ball_region_f32<DISC>(d, A.geo, cb, lane, &k);
            if (n >= 0) {
                done = true;
                if (n >= 3) {
                    kind = k;
                    nv = n;
                    const nlg::Col px = nlg::col(cb.x, lane), py = nlg::col(cb.y, lane);
                    for (int t = 1; t + 1 < n; t++) {
                        const nlg::F2 s0 = {px[0], py[0]}, s1 = {px[t], py[t]}, s2 = {px[t + 1], py[t + 1]};
                        const float ar = 0.5f * fabsf((s1.x - s0.x) * (s2.y - s0.y) - (s2.x - s0.x) * (s1.y - s0.y));
                        for (int q = q0; q < q1; q++) {
                            const float4 f = A.fout[q];
                            // the outer point relative to bary_a, and phi_a there
                            const float xr = f.x * s0.x + f.y * s1.x + f.z * s2.x + cbx - va[0].x;
                            const float yr = f.x * s0.y + f.y * s1.y + f.z * s2.y + cby - va[0].y;
                            const float l1 = (xr * f2y - f2x * yr) * finv, l2 = (f1x * yr - xr * f1y) * finv;
                            OuterPt o;
                            o.Wf = f.w * ar;
                            o.l0f = 1.f - l1 - l2;
                            o.l1f = l1;
                            o.l2f = l2;
                            combine<T>(o, S, v);
                            nout++;
                        }
                    }
                }
            }
        }
        if (!done) {
            nlg::Region R;
            const nlg::F2 dl_unused[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
            nlg::make_region<DISC>(Va, dl_unused, bb, bb, A.geo, R);
            if (R.overflow) atomicOr(A.err, 1);
            if (R.kind != nlg::KIND_NONE && R.nv >= 3) {
                kind = R.kind;
                nv = R.nv;
                for (int t = 1; t + 1 < R.nv; t++) {
                    const D2 s0 = R.P[0], s1 = R.P[t], s2 = R.P[t + 1];
                    const double ar = 0.5 * fabs((s1.x - s0.x) * (s2.y - s0.y) - (s2.x - s0.x) * (s1.y - s0.y));
                    for (int q = q0; q < q1; q++) {
                        const double l0 = A.outer.l[q][0], l1 = A.outer.l[q][1], l2 = A.outer.l[q][2];
                        const double x = l0 * s0.x + l1 * s1.x + l2 * s2.x, y = l0 * s0.y + l1 * s1.y + l2 * s2.y;
                        double phi[3];
                        bary_of(bma, x, y, phi);
                        OuterPt o;
                        o.W = A.outer.w[q] * ar;
                        o.l0 = phi[0];
                        o.l1 = phi[1];
                        o.l2 = phi[2];
                        o.Wf = (float)o.W;
                        o.l0f = (float)phi[0];
                        o.l1f = (float)phi[1];
                        o.l2f = (float)phi[2];
                        combine<T>(o, S, v);
                        nout++;
                    }
                }
            }
        }
        write_pair<T>(A, e, b, nout > 0, v, acc);
        if (nout > 0) {
            acc.cnt++;
            acc.qp += nout * nq_in;
            if (A.stats) acc.hsum += nlg::record_hash(a, b, 0, kind, nv, 0);
        }
    }
}

// boundary candidates of outer triangle a for the ball mode BALL (NQ: the singular kernel's
// near-field whole items go to the near-field queue)
template <int BALL, typename T, bool INV, bool NQ = false, int STS = -1>
__device__ __forceinline__ void boundary_any(const NumArgs &A, int a, BoundaryShared<T> &sh, int lane, LaneAcc &acc)
{
    if constexpr (BALL == NL_BALL_BARY_NOCAPS || BALL == NL_BALL_BARY_APPROXCAPS) {
        support_boundary<BALL, T>(A, a, lane, sh.clip, acc);
    } else {
        stage_outer(A, a, sh.sq, lane);
        __syncwarp();
        if (INV && A.otab)   // k_near reads the outer points from here (no FP64 arithmetic per item)
            for (int q = lane; q < A.outer.n; q += 32) A.otab[(int64_t)a * A.outer.n + q] = sh.sq[q];
        boundary_outer<BALL, T, INV, NQ, STS>(A, a, sh, lane, acc);
    }
}

// resident 4-warp blocks per SM: four with float sums (registers capped at 128, a few hundred
// bytes of spills), three with double sums
template <typename T, bool INV>
constexpr int kBoundaryBlocksPerSm = sizeof(T) == sizeof(float) ? 4 : 3;

template <int BALL, typename T, bool INV, bool NQ = false, int STS = -1>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, kBoundaryBlocksPerSm<T, INV>) k_boundary(const NumArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BoundaryShared<T> &sh = ((BoundaryShared<T> *)smem_raw)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int a = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (a >= A.K) return;
    LaneAcc acc;
    acc_zero(acc);
    boundary_any<BALL, T, INV, NQ, STS>(A, a, sh, lane, acc);
    // k_interior may be running: add atomically onto the zeroed outputs
    finish_outer<STS>(A, a, acc, lane, kAtomicAdd);
}

// ---------------------------------------------------------------------------
// Batched numeric phase: many independent problems in a few persistent launches: the
// interior candidates of every problem (k_interior_batch), then the boundary
// candidates of the problems of each ball mode (k_boundary_batch<BALL>), with the
// register and shared-memory budgets of k_interior and k_boundary.  A work item is a
// run of consecutive outer triangles of one problem; each warp takes the next item
// from the launch's global counter.  The outputs of every problem are those of
// k_interior + k_boundary: each triangle's values are produced by one warp in the same
// order, whatever the schedule.
// ---------------------------------------------------------------------------
struct BatchItem {
    int p;        // problem
    int a0, a1;   // outer triangles a0 .. a1-1
};

// next work item of the calling warp (lane 0 takes it from the counter)
__device__ __forceinline__ int next_item(int *counter, int lane)
{
    int it = 0;
    if (lane == 0) it = atomicAdd(counter, 1);
    return __shfl_sync(0xffffffffu, it, 0);
}

// interior candidates of every problem (stores M_aa and the statistics, as k_interior)
template <typename T>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, sizeof(T) == sizeof(float) ? 5 : 1)
    k_interior_batch(const NumArgs *__restrict__ As, const BatchItem *__restrict__ items, int n_items, int *counter)
{
    __shared__ OuterPt sq_all[kWarpsPerBlock][NL_MAXQ + 8];
    const int lane = threadIdx.x & 31;
    OuterPt *sq = sq_all[threadIdx.x >> 5];
    for (int it = next_item(counter, lane); it < n_items; it = next_item(counter, lane)) {
        const BatchItem w = items[it];
        const NumArgs &A = As[w.p];
#ifdef NL_CHECKS
        if (w.a0 < 0 || w.a1 > A.K || A.nbr_ptr[w.a0] < 0 || A.nbr_ptr[w.a1] > A.E) {
            atomicOr(A.err, 32);   // debug build: bad work item recorded (bit 32) and skipped
            continue;
        }
#endif
        for (int a = w.a0; a < w.a1; a++) {
            stage_outer(A, a, sq, lane);
            __syncwarp();
            LaneAcc acc;
            acc_zero(acc);
            interior_outer<T>(A, a, sq, lane, acc);
            finish_outer(A, a, acc, lane, kStore);
            __syncwarp();
        }
    }
}

// boundary candidates of the problems with ball mode BALL (adds onto k_interior_batch's
// values, as k_boundary adds onto k_interior's)
template <int BALL, typename T, bool INV>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, kBoundaryBlocksPerSm<T, INV>)
    k_boundary_batch(const NumArgs *__restrict__ As, const BatchItem *__restrict__ items, int n_items, int *counter)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BoundaryShared<T> &sh = ((BoundaryShared<T> *)smem_raw)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    for (int it = next_item(counter, lane); it < n_items; it = next_item(counter, lane)) {
        const BatchItem w = items[it];
        const NumArgs &A = As[w.p];
#ifdef NL_CHECKS
        if (w.a0 < 0 || w.a1 > A.K || A.nbr_ptr[w.a0] < 0 || A.nbr_ptr[w.a1] > A.E) {
            atomicOr(A.err, 32);   // debug build: bad work item recorded (bit 32) and skipped
            continue;
        }
#endif
        for (int a = w.a0; a < w.a1; a++) {
            LaneAcc acc;
            acc_zero(acc);
            boundary_any<BALL, T, INV>(A, a, sh, lane, acc);
            finish_outer(A, a, acc, lane, kAdd);
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------------------
// Deferred items of the FP32 path (after the boundary launch, in stream order): each
// thread takes one queued (q, b), builds its region with the FP64 geometry, integrates it
// in FP32, stores its M_ab in the queue's value slots (dv, column slot of [9][cap]) and adds
// its M_bb, M_aa (FP64 atomics) and statistics (integer atomics); k_defer_merge then adds
// the M_ab of each pair's items, which sit side by side in q order, onto the pair's values.
// ---------------------------------------------------------------------------
template <int BALL>
__device__ __forceinline__ void deferred_item(const NumArgs &A, const DeferItem &d, float *dv, int cap, int slot,
                                              nlg::ClipBuf &cb, int lane)
{
    const int K = A.K, a = d.a, q = d.qp & 0xff;
    const int64_t e = d.e;
#ifdef NL_CHECKS
    if (a < 0 || a >= K || e < 0 || e >= A.E || q >= A.outer.n) {   // debug build: bad item (bit 64), skipped
        atomicOr(A.err, 64);
        return;
    }
#endif
    const int b = A.nbr_idx[e];
    D2 Va[3];
    for (int i = 0; i < 3; i++) { Va[i].x = A.tx[i * K + a]; Va[i].y = A.ty[i * K + a]; }
    const OuterPt o = outer_point(A, a, Va, A.area[a], q);
    const D2 ba = {A.bx[a], A.by[a]};
    CandData c;
    int q1;
    load_cand(A, b, ba, bary_hilo(A, a), c, q1);
    Sums<float> S;
    int64_t nq = 0;
    int kind, nv, ncap;
    if (!exact_item_fp64<BALL, float>(A, c, o, S, nq, kind, nv, ncap, cb, lane)) {
        for (int k = 0; k < kDeferVals; k++) dv[(int64_t)k * cap + slot] = 0.f;
        return;
    }
    float w[21];
    for (int k = 0; k < 21; k++) w[k] = 0.f;
    combine<float>(o, S, w);
    for (int k = 0; k < kDeferVals; k++) dv[(int64_t)k * cap + slot] = w[k];
    for (int k = 0; k < 6; k++) atomicAdd(&A.mbb[(int64_t)k * K + b], (double)w[9 + k]);
    for (int k = 0; k < 6; k++) atomicAdd(&A.maa[(int64_t)k * K + a], (double)w[15 + k]);
    A.flag[e] = 1;
    atomicAdd((unsigned long long *)&A.qp_a[a], (unsigned long long)nq);
    atomicAdd((unsigned long long *)&A.cnt_a[a], 1ull);
    if (A.stats)
        atomicAdd((unsigned long long *)&A.hash_a[a],
                  (unsigned long long)nlg::record_hash(a, b, q - c.q0, kind, nv, ncap));
}

template <int BALL>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_deferred(const NumArgs A)
{
    __shared__ nlg::ClipBuf cb[kWarpsPerBlock];
    const int n = min(*A.defer_n, A.defer_cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        deferred_item<BALL>(A, A.defer[i], A.dval, A.defer_cap, i, cb[threadIdx.x >> 5], threadIdx.x & 31);
}

// the queue of one batched boundary launch (items of its problems, As indexed by qp >> 8)
template <int BALL>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_deferred_batch(const NumArgs *__restrict__ As, const DeferItem *__restrict__ items, const int *count, int cap)
{
    __shared__ nlg::ClipBuf cb[kWarpsPerBlock];
    const int n = min(*count, cap);
    float *dv = defer_values(const_cast<DeferItem *>(items), cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const DeferItem d = items[i];
        deferred_item<BALL>(As[d.qp >> 8], d, dv, cap, i, cb[threadIdx.x >> 5], threadIdx.x & 31);
    }
}

// Sum v (NV values) over each run of equal keys in lane order (runs of one key are contiguous
// in lane order; key < 0: a lane without values): the first lane of each run gets its run's sum,
// by a segmented tree of shuffles (five steps, a fixed order of additions), and the return value
// says which lanes lead a run.  All 32 lanes call this.
template <int NV, typename V>
__device__ __forceinline__ bool warp_run_sum(long long key, int lane, V *v)
{
    const long long prev = __shfl_up_sync(0xffffffffu, key, 1);
    const bool head = lane == 0 || prev != key;
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    // last lane of this lane's run: one before the next head (or lane 31)
    const unsigned later = heads & ~((2u << lane) - 1u);
    const int run_end = later ? __ffs(later) - 2 : 31;
    for (int off = 1; off < 32; off <<= 1)
        for (int k = 0; k < NV; k++) {
            const V x = __shfl_down_sync(0xffffffffu, v[k], off);
            if (lane + off <= run_end) v[k] += x;
        }
    return head && key >= 0;
}

// ---------------------------------------------------------------------------
// Near-field whole items of the FP32 singular kernel (after the boundary launch, in stream
// order): the boundary kernel queues every (x_q, T_b) whose whole T_b lies in the near field of
// x_q (certified in FP32), in (pair, outer point) order; here each warp takes 32 of them and
// runs the near-singular rule (signed apex-x decomposition, Duffy collapse, sinh substitution,
// as near_whole_f32) with its lanes spread over the items' panels instead of the items: the
// items have 3 to 30 panels (11 on average at the singular workload), so a lane per item left
// most lanes idle while the longest item ran.  A lane per item first sets up its six sides
// (two per edge: panel count, U, the scaled foot-point direction) in shared memory; the warp then
// takes the panels of all 32 items 32 at a time, sums each item's panels by a segmented shuffle
// tree and adds the sums onto the item's column; a lane per item finally combines its item.  The
// blocks are then summed over the lanes of one pair (M_ab onto the pair's stored values with
// FP32 atomics, M_bb onto T_b's sums) and of one outer triangle (M_aa, statistics), so a warp
// issues a few atomics per pair instead of one per item.
// ---------------------------------------------------------------------------
struct NearSide {              // one side (edge, end A or B) of a near-field item
    float gdx, gdy;            // sg d e: the foot point's scaled edge direction
    float fx, fy;              // foot point F of x on the edge's line, relative to x
    float kcs;                 // sign sg d kc
    float u;                   // U = asinh(|t| / d), the last panel's end
};

struct NearShared {            // per warp
    NearSide side[6][32];
    unsigned short npan[6][32];   // up to about 710 on a side (FP64 panel counts)
    float e1x[32], e1y[32], e2x[32], e2y[32], inv[32], l10[32], l20[32];
    int start[32];             // first panel of each lane's item in the warp's panel list
    float acc[10][32];         // each item's sums (s0, s1, S2) over its panels
};

// the six sides of an item (vertices dl relative to x): panel counts (0 for a degenerate side),
// by the same FP32 rule with FP64 fallback as near_whole_f32
__device__ __forceinline__ int near_setup_f32(const NumArgs &A, const nlg::F2 dl[3], int tb, D2 x, NearShared &sh,
                                              int lane)
{
    const float kc = A.kcf;
    int total = 0;
    for (int i = 0; i < 3; i++) {
        const nlg::F2 a = dl[i], b = dl[(i + 1) % 3];
        float ex = b.x - a.x, ey = b.y - a.y;
        const float L = sqrtf(ex * ex + ey * ey);
        ex /= L;
        ey /= L;
        const float tA = a.x * ex + a.y * ey, tB = b.x * ex + b.y * ey;
        const float Fx = a.x - tA * ex, Fy = a.y - tA * ey;
        const float d = sqrtf(Fx * Fx + Fy * Fy);
        const float UA = asinhf(fabsf(tA) / d), UB = asinhf(fabsf(tB) / d);
        const float th = 1e-4f * L;
        const float M = fmaxf(fmaxf(fabsf(a.x) + fabsf(a.y), fabsf(b.x) + fabsf(b.y)), L) + L;
        auto near_int = [&](float U, float t) {
            const float eps = 1e-6f * M * (1.f / d + 1.f / fabsf(t)) + 1e-5f * fmaxf(U, 1.f);
            return fabsf(U - rintf(U)) < eps;
        };
        bool skip_edge = false, skipA = false, skipB = false;
        int npA, npB;
        if (!(d >= th) || !(fabsf(tA) >= th) || !(fabsf(tB) >= th) || near_int(UA, tA) || near_int(UB, tB)) {
            const int i1 = (i + 1) % 3;
            const D2 Vi = {A.tx[i * A.K + tb], A.ty[i * A.K + tb]}, Vj = {A.tx[i1 * A.K + tb], A.ty[i1 * A.K + tb]};
            const NearEdge64 q = near_edge64(Vi, Vj, x);
            skip_edge = (q.d == 0.0);
            skipA = (q.tA == 0.0);
            skipB = (q.tB == 0.0);
            npA = skip_edge || skipA ? 0 : near_panels64(q.tA, q.d);
            npB = skip_edge || skipB ? 0 : near_panels64(q.tB, q.d);
        } else {
            npA = (int)ceilf(UA);
            npB = (int)ceilf(UB);
            npA = npA < 1 ? 1 : npA;
            npB = npB < 1 ? 1 : npB;
        }
        if (skip_edge || d == 0.f) npA = npB = 0;
        if (skipA) npA = 0;
        if (skipB) npB = 0;
        const float sigma = (Fx * ey - Fy * ex) > 0.f ? 1.f : -1.f;
        for (int sd = 0; sd < 2; sd++) {   // side B, then side A
            const bool sideA = sd == 1;
            const float tau = sideA ? tA : tB;
            const float sg = tau > 0.f ? 1.f : -1.f, sign = sideA ? -sigma : sigma;
            NearSide &S = sh.side[2 * i + sd][lane];
            S.gdx = sg * d * ex;
            S.gdy = sg * d * ey;
            S.fx = Fx;
            S.fy = Fy;
            S.kcs = sign * sg * d * kc;
            S.u = sideA ? UA : UB;
            const int np = sideA ? npA : npB;
            sh.npan[2 * i + sd][lane] = (unsigned short)np;
            total += np;
        }
    }
    return total;
}

// the item data of a near-field item that its panels use (barycentric frame of T_b)
struct NearItem {
    float e1x, e1y, e2x, e2y, inv, l10, l20;
};

// panel pnl of a side with npan panels (side data sd, item frame it) added onto S
__device__ __forceinline__ void near_panel_f32(const NumArgs &A, const NearSide &sd, int npan, const NearItem &it,
                                               int pnl, float S[10])
{
    const bool full = pnl + 1 < npan;
    const float u0 = (float)pnl, hw = full ? 1.f : fmaxf(sd.u, u0) - u0;
    // on a full panel [p, p + 1], sinh(p + x_j) = sinh(p) cosh(x_j) + cosh(p) sinh(x_j); the last
    // panel [p, U] evaluates sinh directly
    float sp = 0.f, cp = 1.f;
    if (full && pnl > 0) {
        const float ep = expf(u0), em = 1.f / ep;
        sp = 0.5f * (ep - em);
        cp = 0.5f * (ep + em);
    }
    const int nu = A.duffy_n;
    for (int j = 0; j < nu; j++) {
        const float sh_ = full ? fmaf(sp, A.glf_ch[j], cp * A.glf_sh[j]) : sinhf(u0 + hw * A.glf_x[j]);
        const float wj = sd.kcs * (hw * A.glf_w[j]);
        const float wx = fmaf(sh_, sd.gdx, sd.fx), wy = fmaf(sh_, sd.gdy, sd.fy);
        const float l1w = (wx * it.e2y - it.e2x * wy) * it.inv;
        const float l2w = (it.e1x * wy - wx * it.e1y) * it.inv;
        for (int k = 0; k < 2; k++) {
            const float sv = A.gl2f_x[k];
            const float l1 = sv * l1w - it.l10, l2 = sv * l2w - it.l20, l0 = 1.f - l1 - l2;
            const float w = wj * A.gl2f_w[k];
            const float w0 = w * l0, w1 = w * l1, w2 = w * l2;
            S[0] += w;
            S[1] += w0; S[2] += w1; S[3] += w2;
            S[4] += w0 * l0; S[5] += w1 * l1; S[6] += w2 * l2;
            S[7] += w0 * l1; S[8] += w0 * l2; S[9] += w1 * l2;
        }
    }
}

template <int BALL>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_near(const NumArgs A)
{
    __shared__ NearShared near_sh[kWarpsPerBlock];
    NearShared &sh = near_sh[threadIdx.x >> 5];
    const int n = min(*A.near_n, A.near_cap);
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int K = A.K;
    for (int64_t base = warp0 * 32; base < n; base += nwarps * 32) {
        const int64_t i = base + lane;
        long long ke = -1, ka = -1;
        int b = 0, q = 0, q0 = 0, np = 0;
        DeferItem d = {0, 0, 0};
        OuterPt o;
        if (i < n) {
            d = A.nearq[i];
            const int a = d.a;
            q = d.qp & 0xff;
#ifdef NL_CHECKS
            if (a < 0 || a >= K || d.e < 0 || d.e >= A.E || q >= A.outer.n) {   // debug build: bad item (bit 128)
                atomicOr(A.err, 128);
                ka = -2;
            }
#endif
            if (ka != -2) {
                b = A.nbr_idx[d.e];
                o = A.otab[(int64_t)a * A.outer.n + q];
                const D2 ba = {A.bx[a], A.by[a]};
                CandData c;
                int q1;
                load_cand(A, b, ba, bary_hilo(A, a), c, q1);
                q0 = c.q0;
                nlg::F2 dl[3];
                for (int k = 0; k < 3; k++) { dl[k].x = c.vlx[k] - o.lx; dl[k].y = c.vly[k] - o.ly; }
                sh.e1x[lane] = c.e1x;
                sh.e1y[lane] = c.e1y;
                sh.e2x[lane] = c.e2x;
                sh.e2y[lane] = c.e2y;
                sh.inv[lane] = c.binv;
                sh.l10[lane] = (dl[0].x * c.e2y - c.e2x * dl[0].y) * c.binv;
                sh.l20[lane] = (c.e1x * dl[0].y - dl[0].x * c.e1y) * c.binv;
                np = near_setup_f32(A, dl, b, D2{o.x, o.y}, sh, lane);
                ke = d.e;
                ka = a;
            }
        }
        // the warp's panel list: item j's panels start at start[j]
        int incl = np;
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        sh.start[lane] = incl - np;
        for (int k = 0; k < 10; k++) sh.acc[k][lane] = 0.f;
        __syncwarp();
        for (int t0 = 0; t0 < total; t0 += 32) {
            const int t = t0 + lane;
            float S[10];
            for (int k = 0; k < 10; k++) S[k] = 0.f;
            long long key = -1;
            int it = 0;
            if (t < total) {
                // the last item whose panels start at or before t (an item without panels shares
                // its start with the next one)
                int lo = 0, hi = 31;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (sh.start[mid] <= t) lo = mid; else hi = mid - 1;
                }
                it = lo;
                int r = t - sh.start[it], side = 0;
                while (side < 5 && r >= (int)sh.npan[side][it]) r -= (int)sh.npan[side++][it];
                const NearItem itd = {sh.e1x[it], sh.e1y[it], sh.e2x[it], sh.e2y[it], sh.inv[it], sh.l10[it],
                                      sh.l20[it]};
                near_panel_f32(A, sh.side[side][it], (int)sh.npan[side][it], itd, r, S);
                key = it;
            }
            // the panels of one item are adjacent: one shared add per item and pass
            if (warp_run_sum<10>(key, lane, S))
                for (int k = 0; k < 10; k++) sh.acc[k][it] += S[k];
            __syncwarp();
        }
        float w[21];
        for (int k = 0; k < 21; k++) w[k] = 0.f;
        int64_t nq = 0;
        if (ka >= 0) {
            Sums<float> S;
            S.s0 = sh.acc[0][lane];
            for (int k = 0; k < 3; k++) S.s1[k] = sh.acc[1 + k][lane];
            for (int k = 0; k < 6; k++) S.S2[k] = sh.acc[4 + k][lane];
            combine<float>(o, S, w);
            nq = 2 * (int64_t)A.duffy_n * np;
            A.flag[d.e] = 1;
        }
        __syncwarp();
        // M_ab onto the pair, M_bb onto T_b: one add per run of one pair in the warp (a warp's
        // items of one pair are adjacent: the queue holds them in (pair, outer point) order)
        if (warp_run_sum<15>(ke, lane, w)) {
            float *blk = (float *)A.blk;
            for (int k = 0; k < 9; k++) atomicAdd(&blk[(int64_t)k * A.E + ke], w[k]);
            for (int k = 0; k < 6; k++) atomicAdd(&A.mbb[(int64_t)k * K + b], (double)w[9 + k]);
        }
        // M_aa and the statistics onto T_a: one add per run of one outer triangle (the lanes' M_aa
        // summed in FP32, like every short sum of the FP32 path: FP64 arithmetic runs at 1/64 of
        // the FP32 rate here, and a warp-wide FP64 shuffle sum would occupy the FP64 pipe)
        float ma[6];
        for (int k = 0; k < 6; k++) ma[k] = w[15 + k];
        unsigned long long st[3] = {ka >= 0 ? 1ull : 0ull, (unsigned long long)nq,
                                    (ka >= 0 && A.stats) ? (unsigned long long)nlg::record_hash(
                                        (int)ka, b, q - q0, nlg::KIND_WHOLE, 3, 0) : 0ull};
        const long long kk = ka >= 0 ? ka : -1;
        const bool lead = warp_run_sum<6>(kk, lane, ma);
        warp_run_sum<3>(kk, lane, st);
        if (lead) {
            for (int k = 0; k < 6; k++) atomicAdd(&A.maa[(int64_t)k * K + kk], (double)ma[k]);
            atomicAdd((unsigned long long *)&A.cnt_a[kk], st[0]);
            atomicAdd((unsigned long long *)&A.qp_a[kk], st[1]);
            if (A.stats) atomicAdd((unsigned long long *)&A.hash_a[kk], st[2]);
        }
    }
}

// M_ab of the deferred items onto their pairs: the first slot of each run of one pair (same
// problem and pair index: a run is one warp's items of one candidate, in q order) sums the run
// in order and adds the sum once, so the values repeat exactly from run to run.  The pair's
// stored value is the boundary kernel's, final when this runs.  args(p): the arguments of
// problem p.
template <class Add>
__device__ __forceinline__ void defer_merge(Add add, const DeferItem *__restrict__ items, const int *count, int cap)
{
    const int n = min(*count, cap);
    const float *dv = defer_values(const_cast<DeferItem *>(items), cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const DeferItem d = items[i];
        if (i > 0) {
            const DeferItem p = items[i - 1];
            if (p.e == d.e && (p.qp >> 8) == (d.qp >> 8)) continue;   // inside a run
        }
        float sum[kDeferVals];
        for (int k = 0; k < kDeferVals; k++) sum[k] = dv[(int64_t)k * cap + i];
        for (int j = i + 1; j < n; j++) {
            const DeferItem r = items[j];
            if (r.e != d.e || (r.qp >> 8) != (d.qp >> 8)) break;
            for (int k = 0; k < kDeferVals; k++) sum[k] += dv[(int64_t)k * cap + j];
        }
        add(d.qp >> 8, d.e, sum);
    }
}

// the sum of one pair's run onto the pair's stored M_ab (problem arguments A)
__device__ __forceinline__ void defer_add(const NumArgs &A, int64_t e, const float *sum)
{
    float *blk = (float *)A.blk;
    for (int k = 0; k < kDeferVals; k++) blk[(int64_t)k * A.E + e] += sum[k];
}

// (templates on the value type, float: one kernel in every translation unit that launches it)
template <typename T>
__global__ void __launch_bounds__(256) k_defer_merge(const NumArgs A)
{
    defer_merge([&](int, int64_t e, const float *sum) { defer_add(A, e, sum); }, A.defer, A.defer_n, A.defer_cap);
}

template <typename T>
__global__ void __launch_bounds__(256)
    k_defer_merge_batch(const NumArgs *__restrict__ As, const DeferItem *__restrict__ items, const int *count, int cap)
{
    defer_merge([&](int p, int64_t e, const float *sum) { defer_add(As[p], e, sum); }, items, count, cap);
}

}  // namespace nlq

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// kernel arguments of one assembled problem (api.cu)
nl_status nl_fill_args(nl_ctx *ctx, const nl_plan *P, nlq::NumArgs &A, bool stats);

// persistent batched numeric launches over problems whose arguments are in dA (device
// array; items index it), of one value type (numeric_batch_f32/f64.cu); *counter must
// be zero when the launch starts
nl_status nl_launch_interior_batch_f32(nl_ctx *ctx, const nlq::NumArgs *dA, const nlq::BatchItem *items,
                                       int n_items, int *counter, int blocks);
nl_status nl_launch_interior_batch_f64(nl_ctx *ctx, const nlq::NumArgs *dA, const nlq::BatchItem *items,
                                       int n_items, int *counter, int blocks);
// single-problem numeric phase (numeric_f32/f64.cu); one_stream: every kernel on the context's
// stream (else the interior kernel runs on side stream 0, concurrently with the boundary kernel)
nl_status nl_launch_numeric_f64(nl_ctx *ctx, const nlq::NumArgs &A, int ball, bool one_stream = false);
nl_status nl_launch_numeric_f32(nl_ctx *ctx, const nlq::NumArgs &A, int ball, bool one_stream = false);

nl_status nl_launch_boundary_batch_f32(nl_ctx *ctx, int ball, bool inv, const nlq::NumArgs *dA,
                                       const nlq::BatchItem *items, int n_items, int *counter, int blocks,
                                       bool set_attr);
nl_status nl_launch_boundary_batch_f64(nl_ctx *ctx, int ball, bool inv, const nlq::NumArgs *dA,
                                       const nlq::BatchItem *items, int n_items, int *counter, int blocks,
                                       bool set_attr);
// the deferred items of one float boundary launch (queue `items`, fill count *count)
nl_status nl_launch_deferred_batch_f32(nl_ctx *ctx, int ball, const nlq::NumArgs *dA, const nlq::DeferItem *items,
                                       const int *count, int cap);
// grid of the deferred-item kernels: two blocks per SM (a grid-stride loop covers any count)
nl_status nl_deferred_blocks(nl_ctx *ctx, int *blocks);
// resident blocks per SM of the interior launch (ball < 0) or of a boundary launch
nl_status nl_batch_occupancy_f32(nl_ctx *ctx, int ball, bool inv, int *per_sm);
nl_status nl_batch_occupancy_f64(nl_ctx *ctx, int ball, bool inv, int *per_sm);

// Single-problem numeric phase: the per-triangle outputs are zeroed, k_boundary is launched on
// the context's stream and then k_interior on side stream 0 (both add their per-triangle values
// atomically), so that the interior kernel's blocks fill the boundary kernel's last wave; the
// context's stream waits for side stream 0 before anything that follows.
// the per-triangle outputs the numeric kernels add onto, zeroed on the context's stream
inline nl_status nl_numeric_zero(nl_ctx *ctx, const nlq::NumArgs &A)
{
    cudaStream_t st = ctx->stream;
    const size_t K = (size_t)A.K;
    NL_CK(cudaMemsetAsync(A.maa, 0, sizeof(double) * 6 * K, st));
    NL_CK(cudaMemsetAsync(A.qp_a, 0, sizeof(int64_t) * K, st));
    NL_CK(cudaMemsetAsync(A.cnt_a, 0, sizeof(int64_t) * K, st));
    NL_CK(cudaMemsetAsync(A.hash_a, 0, sizeof(uint64_t) * K, st));
    NL_CK(cudaMemsetAsync(A.mbb, 0, sizeof(double) * 6 * K, st));
    return NL_OK;
}

inline nl_status nl_numeric_fork(nl_ctx *ctx, const nlq::NumArgs &A)
{
    cudaStream_t st = ctx->stream;
    nl_status s = nl_numeric_zero(ctx, A);
    if (s != NL_OK) return s;
    s = nl_side_streams(ctx);
    if (s != NL_OK) return s;
    NL_CK(cudaEventRecord(ctx->side_ev[nl_ctx::kSideStreams], st));
    NL_CK(cudaStreamWaitEvent(ctx->side[0], ctx->side_ev[nl_ctx::kSideStreams], 0));
    return NL_OK;
}

// the interior kernel on the context's stream after the boundary kernel (no fork: the whole
// numeric phase of one problem on one stream, so that several problems can run side by side)
template <typename T, int STS = -1>
nl_status nl_numeric_interior_same(nl_ctx *ctx, const nlq::NumArgs &A, unsigned grid, unsigned threads, nl_status s)
{
    if (s != NL_OK) return s;
    if (A.kernel == NL_KERNEL_INV_DIST) nlq::k_interior<T, STS, 1><<<grid, threads, 0, ctx->stream>>>(A);
    else nlq::k_interior<T, STS, 0><<<grid, threads, 0, ctx->stream>>>(A);
    ++ctx->launches;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NL_OK : nl_cuda_fail(ctx, e, "k_interior launch");
}

// the interior kernel on side stream 0, then the join (always, so that nothing on the side
// stream outlives a failure); s: the status of the boundary launch
template <typename T, int STS = -1>
nl_status nl_numeric_interior_join(nl_ctx *ctx, const nlq::NumArgs &A, unsigned grid, unsigned threads, nl_status s)
{
    if (s == NL_OK) {
        if (A.kernel == NL_KERNEL_INV_DIST) nlq::k_interior<T, STS, 1><<<grid, threads, 0, ctx->side[0]>>>(A);
        else nlq::k_interior<T, STS, 0><<<grid, threads, 0, ctx->side[0]>>>(A);
        ++ctx->launches;
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) s = nl_cuda_fail(ctx, e, "k_interior launch");
    }
    cudaError_t e = cudaEventRecord(ctx->side_ev[0], ctx->side[0]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->side_ev[0], 0);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(ctx->side[0]);   // no ordering event: wait on the host instead
        if (s == NL_OK) s = nl_cuda_fail(ctx, e, "joining the interior launch");
    }
    return s;
}
