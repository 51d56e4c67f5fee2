// geometry.cuh -- pair geometry on the device: the region R(x, T_b) kept by the
// (approximate) ball centred at an outer point x (Sec. 4, Sec. 5.2, Sec. 7.1, Sec. 9).
//
// Every decision that shapes the interaction set (in-ball tests, edge roots,
// half-plane tests, clip vertices) is evaluated in FP64 with explicit
// round-to-nearest intrinsics (__dmul_rn / __dadd_rn / __dsub_rn / __ddiv_rn /
// __dsqrt_rn), which the compiler never contracts into fused multiply-adds, in
// the order the method's canonical expressions are written:
//   in-ball     dx = p - x;  dx*dx + dy*dy <= delta^2                (closed ball, Eq. (inter))
//   edge roots  q(l) = |p + l (q - p) - x|^2 - delta^2, disc = bh^2 - a c,
//               l = (-bh -/+ sqrt(disc)) / a, kept iff 0 < l < 1  (Sec. 7.1 task 5)
//   nocaps      walk edges i = 0, 1, 2: v_i if inside, then the edge's roots;
//               >= 3 points fanned from the first                   (Sec. 7.1 tasks 3-6)
//   approxcaps  arc points p = x + u delta / |u|, u = (e - x) + (n - x), by bisection (Sec. 4.2.2)
//   exactcaps   one centroid point per cap, weight = cap area       (Sec. 5.2, Eq. (areacap))
//   ngon        Sutherland-Hodgman against the polygon's half-planes, keep orient >= 0 (Sec. 9)
//   overlap     whole T_b iff T_b meets the closed ball             (Sec. 4.2.4)
// so that the set of (T_a, q, T_b) with a non-empty region, their kind and their
// vertex counts are bit-identical to a straightforward FP64 evaluation.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.cuh"

namespace nlg {

struct D2 {
    double x, y;
};

struct F2 {
    float x, y;
};

enum { KIND_NONE = 0, KIND_WHOLE = 1, KIND_PARTIAL = 2 };

__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dvd(double a, double b) { return __ddiv_rn(a, b); }

struct Region {
    int kind, nv, ncap;
    int overflow;      // a buffer bound was hit (never for convex input); reported as an error
    D2 P[NL_MAXV];     // polygon, counter-clockwise, fanned from P[0]
    D2 cc[3];          // exactcaps: cap centroids
    double cw[3];      // exactcaps: cap areas
};

struct GeoParams {
    double delta, d2;
    const double *ngon;   // [2 n] offsets (device)
    int ngon_n, cap_level, cap_printed;
    // FP32 certification data
    float tau;            // decision margin (1e-5 delta)
    float inv_tau;        // 1 / tau
    float rin_m2;         // (r_in - tau)^2: r_in = delta (disc balls) or the polygon's inradius
    float rout_p2;        // (delta + tau)^2
    float b_in2, b_out2;  // barycenter ball: (delta - tau)^2, (delta + tau)^2
    float of[64][2];      // polygon offsets o_k (FP32)
    float ef[64][2];      // edges o_{k+1} - o_k (FP32)
    float mk[64];         // |e_k| tau: margin of the FP32 orientation test of pass k
    float err0;           // bound on |dl - (v - x)| of the FP32 local coordinates
    int regular;          // offsets form the regular polygon R (cos 2 pi k / N, sin 2 pi k / N)
    float r2;             // 2 max_k |o_k|_1
    float o1max;          // max_k |o_k|_1
    float sector, rin_tau; // 2 pi / N; inradius - tau
    float deltaf;          // delta in FP32
};

// atan2 from the arctangent polynomial of Abramowitz & Stegun 4.4.49 (Hastings): on [0, 1]
// its error is at most 1e-5 rad; with the octant reduction and the FP32 rounding the
// angle is within 2e-5 rad of atan2(y, x).
__device__ __forceinline__ float atan2_poly(float y, float x)
{
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float a = mx > 0.f ? __fdividef(mn, mx) : 0.f, s = a * a;
    float r = a * (0.9998660f + s * (-0.3302995f + s * (0.1801410f + s * (-0.0851330f + s * 0.0208351f))));
    if (ay > ax) r = 1.57079632679f - r;
    if (x < 0.f) r = 3.14159265359f - r;
    return y < 0.f ? -r : r;
}

// Passes of the polygon clip that can change a triangle with FP32 coordinates d (relative to
// x), as a bit mask over k.  For a regular polygon, half-plane k (outward normal at angle
// (k + 1/2) 2pi/N, at distance r_in) holds every point p with |p| cos(angle(p) - phi_k) <=
// r_in - tau inside by tau; for a point of T_b (|p| <= r_max, angle within the triangle's
// angular extent when x is outside T_b) that holds whenever phi_k is farther than alpha,
// cos alpha = (r_in - tau) / r_max, from the extent.  Passes outside the extent widened by
// alpha (and 2e-3 rad for the angle errors, about 100x their bound) are the identity.
__device__ __forceinline__ uint64_t ngon_pass_mask(const F2 d[3], const GeoParams &g)
{
    const int N = g.ngon_n;
    const uint64_t full = (N >= 64) ? ~0ull : ((1ull << N) - 1ull);
    if (!g.regular) return full;
    const float o0 = d[0].x * d[1].y - d[0].y * d[1].x;
    const float o1 = d[1].x * d[2].y - d[1].y * d[2].x;
    const float o2 = d[2].x * d[0].y - d[2].y * d[0].x;
    if (fminf(o0, fminf(o1, o2)) > -1e-3f * (fabsf(o0) + fabsf(o1) + fabsf(o2))) return full;  // x inside or close
    float r2max = 0.f, t[3];
    for (int i = 0; i < 3; i++) {
        r2max = fmaxf(r2max, d[i].x * d[i].x + d[i].y * d[i].y);
        t[i] = atan2_poly(d[i].y, d[i].x);
    }
    if (r2max <= g.rin_tau * g.rin_tau) return 0ull;
    const float cz = g.rin_tau * rsqrtf(r2max);   // its few-ulp error is far inside the slack
    const float alpha = atan2_poly(sqrtf(fmaxf(1.f - cz * cz, 0.f)), cz);   // acos(cz)
    // sort the three angles, take the arc complementary to the largest gap
    float a0 = t[0], a1 = t[1], a2 = t[2], tmp;
    if (a0 > a1) { tmp = a0; a0 = a1; a1 = tmp; }
    if (a1 > a2) { tmp = a1; a1 = a2; a2 = tmp; }
    if (a0 > a1) { tmp = a0; a0 = a1; a1 = tmp; }
    const float two_pi = 6.28318530718f;
    const float g01 = a1 - a0, g12 = a2 - a1, g20 = a0 + two_pi - a2;
    float lo, hi;
    if (g20 >= g01 && g20 >= g12) { lo = a0; hi = a2; }
    else if (g01 >= g12) { lo = a1; hi = a0 + two_pi; }
    else { lo = a2; hi = a1 + two_pi; }
    if (hi - lo > 0.8f * 3.14159265f) return full;
    const float slack = alpha + 2e-3f;
    lo -= slack;
    hi += slack;
    if (hi - lo >= two_pi) return full;
    // passes k0..k1 (mod N) as a window of cnt bits rotated to k0 mod N
    const float isec = __fdividef(1.f, g.sector);
    const int k0 = (int)ceilf(lo * isec - 0.5f), k1 = (int)floorf(hi * isec - 0.5f);
    const int cnt = k1 - k0 + 1;
    if (cnt <= 0) return 0ull;
    if (cnt >= N) return full;
    int s = k0 % N;
    if (s < 0) s += N;
    const uint64_t w = (1ull << cnt) - 1ull;
    return ((w << s) | (s ? (w >> (N - s)) : 0ull)) & full;
}

__device__ __forceinline__ bool in_ball(D2 p, D2 x, double d2)
{
    double dx = sub(p.x, x.x), dy = sub(p.y, x.y);
    return add(mul(dx, dx), mul(dy, dy)) <= d2;
}

// roots of the edge p -> q with 0 < l < 1, increasing; ent[k]: walk enters the ball there
__device__ __forceinline__ int edge_roots(D2 p, D2 q, D2 x, double d2, bool p_in, double lam[2], bool ent[2])
{
    double dx = sub(q.x, p.x), dy = sub(q.y, p.y);
    double fx = sub(p.x, x.x), fy = sub(p.y, x.y);
    double a = add(mul(dx, dx), mul(dy, dy));
    double bh = add(mul(fx, dx), mul(fy, dy));
    double c = sub(add(mul(fx, fx), mul(fy, fy)), d2);
    double disc = sub(mul(bh, bh), mul(a, c));
    if (disc < 0.0) return 0;
    double s = __dsqrt_rn(disc);
    double l1 = dvd(sub(-bh, s), a);
    double l2 = dvd(add(-bh, s), a);
    bool k1 = (l1 > 0.0 && l1 < 1.0), k2 = (l2 > 0.0 && l2 < 1.0);
    if (k1 && k2) {
        lam[0] = l1; ent[0] = true;
        lam[1] = l2; ent[1] = false;
        return 2;
    }
    int n = 0;
    if (k1) { lam[n] = l1; ent[n] = !p_in; n++; }
    if (k2) { lam[n] = l2; ent[n] = !p_in; n++; }
    return n;
}

// boundary walk of T_b n B_delta(x); tag 0 = vertex, 1 = entry root, 2 = exit root
__device__ __forceinline__ int ball_walk(const D2 V[3], D2 x, double d2, D2 W[12], int tag[12], int *n_in)
{
    bool ins[3];
    int nin = 0;
#pragma unroll
    for (int i = 0; i < 3; i++) { ins[i] = in_ball(V[i], x, d2); nin += ins[i]; }
    *n_in = nin;
    int n = 0;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        D2 p = V[i], q = V[(i + 1) % 3];
        if (ins[i]) { W[n] = p; tag[n] = 0; n++; }
        double lam[2];
        bool ent[2];
        int nr = edge_roots(p, q, x, d2, ins[i], lam, ent);
        double ex = sub(q.x, p.x), ey = sub(q.y, p.y);
        for (int k = 0; k < nr; k++) {
            W[n].x = add(p.x, mul(lam[k], ex));
            W[n].y = add(p.y, mul(lam[k], ey));
            tag[n] = ent[k] ? 1 : 2;
            n++;
        }
    }
    return n;
}

__device__ __forceinline__ D2 arc_mid(D2 e, D2 n, D2 x, double delta)
{
    double ux = add(sub(e.x, x.x), sub(n.x, x.x));
    double uy = add(sub(e.y, x.y), sub(n.y, x.y));
    double s = dvd(delta, __dsqrt_rn(add(mul(ux, ux), mul(uy, uy))));
    D2 p;
    p.x = add(x.x, mul(ux, s));
    p.y = add(x.y, mul(uy, s));
    return p;
}

// 2^level - 1 arc points between e and n in counter-clockwise order (dyadic bisection)
__device__ __forceinline__ void arc_fill(D2 e, D2 n, D2 x, double delta, int level, D2 *out, int *cnt)
{
    D2 pts[17];
    int np = 2;
    pts[0] = e;
    pts[1] = n;
    for (int l = 0; l < level; l++) {
        // insert midpoints between consecutive points, from the back to keep indices valid
        for (int i = np - 1; i >= 1; i--) {
            pts[2 * i] = pts[i];
            pts[2 * i - 1] = arc_mid(pts[i - 1], pts[i], x, delta);
        }
        np = 2 * np - 1;
    }
    for (int i = 1; i + 1 < np; i++) out[(*cnt)++] = pts[i];
}

// exact circular cap between the chord end points e and n (values only)
__device__ __forceinline__ void cap_rule(D2 e, D2 n, D2 x, double delta, int printed, D2 *c, double *area)
{
    double cx = n.x - e.x, cy = n.y - e.y;
    double chord = sqrt(cx * cx + cy * cy);
    double th = asin(chord / (2.0 * delta));
    double tms;    // 2 theta - sin 2 theta
    if (th < 0.05) {
        double u = 2.0 * th, u2 = u * u, term = u * u2 / 6.0, sum = 0.0;
        for (int k = 1; k <= 6; k++) {
            sum += term;
            term *= -u2 / ((2.0 * k + 2.0) * (2.0 * k + 3.0));
        }
        tms = sum;
    } else {
        tms = 2.0 * th - sin(2.0 * th);
    }
    *area = delta * delta * tms / (printed ? 4.0 : 2.0);
    double st = sin(th);
    double d = (tms > 0.0) ? 4.0 * delta * st * st * st / (3.0 * tms) : delta;
    double mx = 0.5 * (e.x + n.x) - x.x, my = 0.5 * (e.y + n.y) - x.y;
    double ml = sqrt(mx * mx + my * my);
    c->x = x.x + d * mx / ml;
    c->y = x.y + d * my / ml;
}

__device__ __forceinline__ double orient(D2 a, D2 b, D2 p)
{
    return sub(mul(sub(b.x, a.x), sub(p.y, a.y)), mul(sub(b.y, a.y), sub(p.x, a.x)));
}

// Sutherland-Hodgman clip of the ccw triangle V by the regular polygon x + off_k.
// dl: FP32 coordinates of V relative to x; a pass whose every vertex is certified
// (FP32, margin mk[k]) to be on the kept side is the identity and is skipped.
__device__ __forceinline__ int clip_ngon(const D2 V[3], const F2 dl[3], D2 x, const GeoParams &g, D2 *out,
                                         int *overflow)
{
    D2 A[NL_MAXV], B[NL_MAXV];
    F2 Af[NL_MAXV];
    int n = 3;
    A[0] = V[0]; A[1] = V[1]; A[2] = V[2];
    Af[0] = dl[0]; Af[1] = dl[1]; Af[2] = dl[2];
    const int N = g.ngon_n;
    uint64_t mask = ngon_pass_mask(dl, g);
    while (mask && n > 0) {
        const int k = __ffsll((long long)mask) - 1;
        mask &= mask - 1;
        // certified identity pass: skip without FP64 work
        bool sure_in = true;
        {
            const float ox = g.of[k][0], oy = g.of[k][1], ex = g.ef[k][0], ey = g.ef[k][1], m = g.mk[k];
            for (int i = 0; i < n && sure_in; i++)
                sure_in = (ex * (Af[i].y - oy) - ey * (Af[i].x - ox)) > m;
        }
        if (sure_in) continue;
        const int k1 = (k + 1 < N) ? k + 1 : 0;
        D2 P0, P1;
        P0.x = add(x.x, g.ngon[2 * k]);
        P0.y = add(x.y, g.ngon[2 * k + 1]);
        P1.x = add(x.x, g.ngon[2 * k1]);
        P1.y = add(x.y, g.ngon[2 * k1 + 1]);
        double o[NL_MAXV];
        bool all_in = true;
        if (!sure_in)
            for (int i = 0; i < n; i++) {
                o[i] = orient(P0, P1, A[i]);
                all_in = all_in && (o[i] >= 0.0);
            }
        if (!sure_in && !all_in) {
            int m = 0;
            for (int i = 0; i < n; i++) {
                if (m + 2 > NL_MAXV) {
                    *overflow = 1;
                    break;
                }
                int ip = (i + n - 1) % n;
                D2 s = A[ip], e = A[i];
                double ds = o[ip], de = o[i];
                if (de >= 0.0) {
                    if (ds < 0.0) {
                        double t = dvd(ds, sub(ds, de));
                        B[m].x = add(s.x, mul(t, sub(e.x, s.x)));
                        B[m].y = add(s.y, mul(t, sub(e.y, s.y)));
                        m++;
                    }
                    B[m++] = e;
                } else if (ds >= 0.0) {
                    double t = dvd(ds, sub(ds, de));
                    B[m].x = add(s.x, mul(t, sub(e.x, s.x)));
                    B[m].y = add(s.y, mul(t, sub(e.y, s.y)));
                    m++;
                }
            }
            n = m;
            for (int i = 0; i < n; i++) {
                A[i] = B[i];
                Af[i].x = (float)(B[i].x - x.x);
                Af[i].y = (float)(B[i].y - x.y);
            }
        }
    }
    for (int i = 0; i < n; i++) out[i] = A[i];
    return n;
}

__device__ __forceinline__ bool overlaps(const D2 V[3], D2 x, double d2)
{
    for (int i = 0; i < 3; i++)
        if (in_ball(V[i], x, d2)) return true;
    for (int i = 0; i < 3; i++) {
        D2 p = V[i], q = V[(i + 1) % 3];
        double dx = sub(q.x, p.x), dy = sub(q.y, p.y);
        double fx = sub(p.x, x.x), fy = sub(p.y, x.y);
        double a = add(mul(dx, dx), mul(dy, dy));
        double bh = add(mul(fx, dx), mul(fy, dy));
        double c = sub(add(mul(fx, fx), mul(fy, fy)), d2);
        double disc = sub(mul(bh, bh), mul(a, c));
        if (disc >= 0.0) {
            double s = __dsqrt_rn(disc);
            double l1 = dvd(sub(-bh, s), a), l2 = dvd(add(-bh, s), a);
            if ((l1 >= 0.0 && l1 <= 1.0) || (l2 >= 0.0 && l2 <= 1.0)) return true;
        }
    }
    bool in = true;
    for (int i = 0; i < 3; i++)
        if (orient(V[i], V[(i + 1) % 3], x) < 0.0) in = false;
    return in;
}

// R(x, T_b) for the ball mode BALL
template <int BALL>
__device__ __forceinline__ void make_region(const D2 V[3], const F2 dl[3], D2 bary_b, D2 x, const GeoParams &g,
                                            Region &R)
{
    R.kind = KIND_NONE;
    R.nv = 0;
    R.ncap = 0;
    R.overflow = 0;
    if (BALL == NL_BALL_BARYCENTER || BALL == NL_BALL_OVERLAP) {
        bool keep = (BALL == NL_BALL_BARYCENTER) ? in_ball(bary_b, x, g.d2) : overlaps(V, x, g.d2);
        if (keep) {
            R.kind = KIND_WHOLE;
            R.nv = 3;
            R.P[0] = V[0]; R.P[1] = V[1]; R.P[2] = V[2];
        }
        return;
    }
    if (BALL == NL_BALL_NGON) {
        int n = clip_ngon(V, dl, x, g, R.P, &R.overflow);
        if (n >= 3) {
            R.nv = n;
            bool same = (n == 3);
            for (int i = 0; same && i < 3; i++) same = (R.P[i].x == V[i].x && R.P[i].y == V[i].y);
            R.kind = same ? KIND_WHOLE : KIND_PARTIAL;
        }
        return;
    }
    // nocaps / approxcaps / exactcaps
    D2 W[12];
    int tag[12], nin;
    int n = ball_walk(V, x, g.d2, W, tag, &nin);
    if (n < 2) return;
    if (BALL == NL_BALL_NOCAPS && n < 3) return;
    if (BALL == NL_BALL_NOCAPS || BALL == NL_BALL_EXACTCAPS) {
        if (n >= 3) {
            for (int i = 0; i < n; i++) R.P[i] = W[i];
            R.nv = n;
        }
        if (BALL == NL_BALL_EXACTCAPS) {
            for (int i = 0; i < n; i++) {
                int j = (i + 1) % n;
                if (tag[i] == 2 && tag[j] == 1 && R.ncap < 3) {
                    cap_rule(W[i], W[j], x, g.delta, g.cap_printed, &R.cc[R.ncap], &R.cw[R.ncap]);
                    R.ncap++;
                }
            }
        }
    } else {
        int m = 0;
        for (int i = 0; i < n; i++) {
            int j = (i + 1) % n;
            if (m + 1 > NL_MAXV) {
                R.overflow = 1;
                break;
            }
            R.P[m++] = W[i];
            if (tag[i] == 2 && tag[j] == 1) {
                if (m + (1 << g.cap_level) > NL_MAXV) {
                    R.overflow = 1;
                    break;
                }
                arc_fill(W[i], W[j], x, g.delta, g.cap_level, R.P, &m);
            }
        }
        R.nv = (m >= 3) ? m : 0;
    }
    if (R.nv >= 3 || R.ncap > 0) R.kind = (nin == 3 && n == 3) ? KIND_WHOLE : KIND_PARTIAL;
}

// ---------------------------------------------------------------------------
// Certified FP32 pre-classification.
//
// d[i] = v_i - x in FP32, each within eps_d of the exact difference (the inputs are
// rounded FP64 differences taken relative to the outer triangle's barycentre).  A
// decision is taken in FP32 only when the exact value clears the threshold by the
// margin tau (1e-5 delta, about 100x the FP32 error bound); then the FP64 predicates
// (whose own error is ~1e-16 delta) decide the same way, so the region equals the
// one the FP64 geometry would build:
//   whole  - every vertex at least tau inside the ball (or the polygon's inscribed
//            circle): every in-ball test is true, no edge root lies in (0, 1), every
//            polygon half-plane pass is the identity;
//   empty  - T_b at least tau outside the circle of radius delta (which contains
//            every approximate ball used here): no vertex inside, no edge root in
//            [0, 1], and no clip output vertex can survive.
// Anything else is undecided and goes to the FP64 geometry.
// ---------------------------------------------------------------------------
enum { CLS_EMPTY = 0, CLS_WHOLE = 1, CLS_EXACT = 2 };

__device__ __forceinline__ float dist2_origin_triangle(const F2 d[3])
{
    // 0 if the origin is inside the ccw triangle, else the squared distance to it
    float o0 = d[0].x * d[1].y - d[0].y * d[1].x;
    float o1 = d[1].x * d[2].y - d[1].y * d[2].x;
    float o2 = d[2].x * d[0].y - d[2].y * d[0].x;
    if (o0 >= 0.f && o1 >= 0.f && o2 >= 0.f) return 0.f;
    float best = INFINITY;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        F2 p = d[i], q = d[(i + 1) % 3];
        float ex = q.x - p.x, ey = q.y - p.y;
        float t = -(p.x * ex + p.y * ey) / (ex * ex + ey * ey);
        t = fminf(fmaxf(t, 0.f), 1.f);
        float cx = p.x + t * ex, cy = p.y + t * ey;
        best = fminf(best, cx * cx + cy * cy);
    }
    return best;
}

// rin: radius of the disc that lies inside the kept region for sure (delta, or the
// polygon's inradius); rout: radius of a disc containing it (delta)
// The triangle with vertices d (relative to the origin, every vertex farther than sqrt(r2))
// lies farther than sqrt(r2) from the origin: the origin is outside it and no edge comes closer.
// An edge p -> q whose closest point is interior (0 < n = -p.e < e.e) is at squared distance
// |p|^2 - n^2 / e.e; the test multiplies through by e.e (no division).
__device__ __forceinline__ bool triangle_beyond(const F2 d[3], float r2)
{
    const float o0 = d[0].x * d[1].y - d[0].y * d[1].x;
    const float o1 = d[1].x * d[2].y - d[1].y * d[2].x;
    const float o2 = d[2].x * d[0].y - d[2].y * d[0].x;
    if (o0 >= 0.f && o1 >= 0.f && o2 >= 0.f) return false;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const F2 p = d[i], q = d[(i + 1) % 3];
        const float ex = q.x - p.x, ey = q.y - p.y;
        const float n = -(p.x * ex + p.y * ey), ee = ex * ex + ey * ey;
        if (n > 0.f && n < ee && (p.x * p.x + p.y * p.y) * ee - n * n <= r2 * ee) return false;
    }
    return true;
}

__device__ __forceinline__ int classify_vertices(const F2 d[3], float rin_m2, float rout_p2)
{
    float r0 = d[0].x * d[0].x + d[0].y * d[0].y;
    float r1 = d[1].x * d[1].x + d[1].y * d[1].y;
    float r2 = d[2].x * d[2].x + d[2].y * d[2].y;
    if (fmaxf(r0, fmaxf(r1, r2)) <= rin_m2) return CLS_WHOLE;
    if (fminf(r0, fminf(r1, r2)) > rout_p2 && triangle_beyond(d, rout_p2)) return CLS_EMPTY;
    return CLS_EXACT;
}

// ---------------------------------------------------------------------------
// FP32 Sutherland-Hodgman clip with certified signs (FP32-compensated path).
//
// Each vertex carries an absolute bound err on its distance to the vertex the FP64
// clip holds at the same point of the algorithm.  An orientation o_k(v) computed in
// FP32 is trusted only if |o| > |e_k| (err + rounding allowance); then its sign is
// the FP64 sign, every branch of the clip matches the FP64 run, and so do the
// vertex count and the kind.  A new vertex p = s + t (e - s), t = o_s / (o_s - o_e),
// inherits err_p = max(err_s, err_e) + |e - s| (u_s + u_e) / (|o_s| + |o_e| - u_s - u_e)
// + rounding.  Returns the vertex count, or -1 when a sign is not certain (the
// caller then runs the FP64 clip).  Coordinates are relative to x.
// ---------------------------------------------------------------------------

// The same certified FP32 clip with its two vertex buffers in shared memory (one
// column per lane, [slot][lane]: no bank conflicts) and a capacity of kClipCap
// vertices (a triangle cut kClipCap - 3 times); more vertices return -1 and the
// caller takes the FP64 clip.  One loop per pass certifies every orientation and builds
// the clipped list at the same time; a pass that keeps every vertex is the identity and
// its copy is dropped.
//
// Error bound of o = e x (a - o_k) evaluated in FP32 (u = 2^-24), against the same
// expression on the FP64 vertex A*, offset O* and edge E*:
//   |o - E* x (A* - O*)| <= |e| (|a - A*| + |o_k - O*| + 1.5 u |a - o_k|_1 + 3 u |a - o_k|_1)
//                        <= |e| (err_a + 1.5 u |o_k|_1 + 4.5 u |r|_1),   r = a - o_k.
// The test uses twice that: |e| (err_a + 3 u |o_k|_1 + 9 u |r|_1).
constexpr int kClipCap = 8;

struct ClipBuf {
    float x[2][kClipCap][32], y[2][kClipCap][32], e[2][kClipCap][32];
};

// UNROLL: the vertex loop unrolled over the capacity (constant kernel: numeric phase 4.82 ->
// 4.69 ms; the singular kernel's larger boundary kernel lost more to instruction fetch)
template <bool UNROLL = false>
__device__ __forceinline__ int clip_ngon_f32_sh(const F2 dl[3], float err0, const GeoParams &g, ClipBuf &cb,
                                                int lane, int *which, bool *cut)
{
    const float kU9 = 9.0f * 5.9604645e-8f;    // 9 u
    const float kU3o = 3.0f * 5.9604645e-8f * g.o1max;   // 3 u max_k |o_k|_1
    int cur = 0, n = 3;
    for (int i = 0; i < 3; i++) {
        cb.x[0][i][lane] = dl[i].x;
        cb.y[0][i][lane] = dl[i].y;
        cb.e[0][i][lane] = err0;
    }
    *cut = false;
    uint64_t mask = ngon_pass_mask(dl, g);
    while (mask && n > 0) {
        const int k = __ffsll((long long)mask) - 1;
        mask &= mask - 1;
        const float ox = g.of[k][0], oy = g.of[k][1], ex = g.ef[k][0], ey = g.ef[k][1];
        const float el = g.mk[k] * g.inv_tau;   // |e_k|
        const float elu = el * kU9, elc = el * kU3o;
        // a pass over a convex polygon keeps at most n + 1 vertices (certified signs keep the exact
        // combinatorics), so a list of fewer than kClipCap vertices cannot outgrow the buffer
        if (n >= kClipCap) return -1;
        const int nxt = cur ^ 1;
        int m = 0;
        bool all_in = true;
        float sx = cb.x[cur][n - 1][lane], sy = cb.y[cur][n - 1][lane], se = cb.e[cur][n - 1][lane];
        float so = ex * (sy - oy) - ey * (sx - ox);
        float su = fmaf(el, se, fmaf(elu, fabsf(sx - ox) + fabsf(sy - oy), elc));
        // one vertex step: false when its sign is not certain
        auto step = [&](int i) -> bool {
            const float px = cb.x[cur][i][lane], py = cb.y[cur][i][lane], pe = cb.e[cur][i][lane];
            const float po = ex * (py - oy) - ey * (px - ox);
            // |e_k| (err + 3 u |o_k|_1 + 9 u |r|_1), the bound above
            const float pu = fmaf(el, pe, fmaf(elu, fabsf(px - ox) + fabsf(py - oy), elc));
            if (!(fabsf(po) > pu)) return false;
            const bool p_in = po > 0.f, s_in = so > 0.f;
            all_in = all_in && p_in;
            if (p_in != s_in) {
                // t by the fast division (within 2 ulp): its error is in the rounding term
                const float t = __fdividef(so, so - po);
                const float dx = px - sx, dy = py - sy;
                const float den = fabsf(so) + fabsf(po) - su - pu;   // > 0: both signs certified
                const float len = fabsf(dx) + fabsf(dy);
                cb.x[nxt][m][lane] = sx + t * dx;
                cb.y[nxt][m][lane] = sy + t * dy;
                // p = s + t (q - s): interpolated error, the error of t times |q - s| (its
                // quotient rounded up by 1e-6 relative), and rounding
                cb.e[nxt][m][lane] = fmaxf(se, pe) + __fdividef(len * (su + pu), den) * 1.000001f +
                                     6.f * 5.9604645e-8f * (fabsf(sx) + fabsf(sy) + len);
                m++;
            }
            if (p_in) {
                cb.x[nxt][m][lane] = px;
                cb.y[nxt][m][lane] = py;
                cb.e[nxt][m][lane] = pe;
                m++;
            }
            sx = px; sy = py; se = pe; so = po; su = pu;
            return true;
        };
        if constexpr (UNROLL) {
#pragma unroll
            for (int i = 0; i < kClipCap - 1; i++) {   // n < kClipCap
                if (i >= n) break;
                if (!step(i)) return -1;
            }
        } else {
            for (int i = 0; i < n; i++)
                if (!step(i)) return -1;
        }
        if (all_in) continue;   // identity pass: keep the current list
        *cut = true;
        cur = nxt;
        n = m;
    }
    *which = cur;
    return n;
}

// Near field of the singular kernel for a whole T_b: near iff dist(x, T_b) < diam(T_b).
// FP32 decides when the two differ by more than eta (1e-5 delta, far above the FP32
// ---------------------------------------------------------------------------
// FP32 region of the disc balls nocaps and approxcaps (Sec. 4.2.1, 4.2.2) with certified
// discrete choices.  d[i] = v_i - x in FP32 (within err0 of the exact differences).
// The FP64 walk (ball_walk) is decided by three kinds of predicates, each certified here
// with the margin tau = 1e-5 delta (rin_m2 = (delta - tau)^2, rout_p2 = (delta + tau)^2):
//   * vertex in the closed ball: |d|^2 <= rin_m2 -> in, > rout_p2 -> out;
//   * roots of an edge p -> q in (0, 1): with both end points certified, in -> in has none,
//     in -> out exactly one (the larger root, an exit), out -> in exactly one (the smaller
//     root, an entry); out -> out has two (entry, exit) when the segment passes within
//     delta - tau of x, none when it stays farther than delta + tau;
//   * anything closer to a threshold is undecided: return -1 (the FP64 walk decides).
// Then the walk emits the same points in the same order as the FP64 walk (vertex if
// inside, then the edge's roots by increasing parameter; approxcaps inserts the dyadic arc
// points between every exit and the next entry), so the vertex count and the kind equal
// the FP64 ones; the coordinates are FP32 values.  Returns the vertex count (0 when the
// region is empty or degenerate), writes P[0..n) and *kind.
// ---------------------------------------------------------------------------
constexpr int kBallCap = 16;   // FP32 region vertices (nocaps <= 6; approxcaps 6 + 3 (m - 1))

// Element k of the calling lane in a shared-memory array laid out [slot][32 lanes] (a column per
// lane: the lanes of a warp never share a bank).  The FP32 regions below keep their vertex lists
// in the lane's column of the clip buffer: arrays indexed by a run-time count would live in
// local memory, which the shared-memory carve-out leaves little L1 for.
struct Col {
    float *p;
    __device__ __forceinline__ float &operator[](int k) const { return p[k << 5]; }
};
// slot k of a ClipBuf coordinate array read flat (16 slots: [2][8])
__device__ __forceinline__ Col col(float (&a)[2][kClipCap][32], int lane) { return Col{&a[0][0][lane]}; }

// The certified FP32 walk itself: the walk points W (relative to x) into wx / wy, their tags (0
// vertex, 1 entry, 2 exit; two bits a point in *tags) and the count of vertices inside; returns the
// number of walk points (at most 6), or -1 when a choice is not certain.
__device__ __forceinline__ int ball_walk_f32(const F2 d[3], const GeoParams &g, Col wx, Col wy, unsigned *tags,
                                             int *n_in)
{
    const float delta = g.deltaf, d2f = delta * delta;
    bool ins[3];
    int nin = 0;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const float r = d[i].x * d[i].x + d[i].y * d[i].y;
        if (r <= g.rin_m2) ins[i] = true;
        else if (r > g.rout_p2) ins[i] = false;
        else return -1;
        nin += ins[i];
    }
    int n = 0;
    unsigned tg = 0;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const F2 p = d[i], q = d[(i + 1) % 3];
        if (ins[i]) { wx[n] = p.x; wy[n] = p.y; n++; }   // tag 0
        const bool qin = ins[(i + 1) % 3];
        if (ins[i] && qin) continue;
        const float ex = q.x - p.x, ey = q.y - p.y;
        const float a = ex * ex + ey * ey, b = p.x * ex + p.y * ey, c = p.x * p.x + p.y * p.y - d2f;
        int nr;
        if (!ins[i] && !qin) {
            // out -> out: the closest point of the segment to x is interior when 0 < -b < a, at
            // squared distance |p|^2 - b^2 / a (compared multiplied through by a); at an end
            // point it is that (outside) vertex
            const float pa = (p.x * p.x + p.y * p.y) * a - b * b;
            if (!(-b > 0.f && -b < a)) nr = 0;
            else if (pa <= g.rin_m2 * a) nr = 2;
            else if (pa > g.rout_p2 * a) nr = 0;
            else return -1;
        } else {
            nr = 1;
        }
        if (nr == 0) continue;
        // roots of a l^2 + 2 b l + c = 0 without cancellation (coordinates only: the fast
        // division's few-ulp error stays in the FP32 values)
        const float sq = sqrtf(fmaxf(b * b - a * c, 0.f));
        const float tt = b > 0.f ? -(b + sq) : (sq - b);
        float l1 = __fdividef(tt, a), l2 = __fdividef(c, tt);
        if (l1 > l2) { const float z = l1; l1 = l2; l2 = z; }
        if (nr == 2 || !ins[i]) {   // entry at the smaller root
            wx[n] = p.x + l1 * ex; wy[n] = p.y + l1 * ey; tg |= 1u << (2 * n); n++;
        }
        if (nr == 2 || ins[i]) {    // exit at the larger root
            wx[n] = p.x + l2 * ex; wy[n] = p.y + l2 * ey; tg |= 2u << (2 * n); n++;
        }
    }
    *tags = tg;
    *n_in = nin;
    return n;
}

__device__ __forceinline__ unsigned walk_tag(unsigned tags, int k) { return (tags >> (2 * k)) & 3u; }

// the unit-radius-delta point in the direction of u (the normalised sum of two arc points)
__device__ __forceinline__ F2 arc_dir(float ux, float uy, float delta)
{
    const float sc = delta * rsqrtf(ux * ux + uy * uy);
    return F2{ux * sc, uy * sc};
}

// FP32 region (nocaps, approxcaps) of T_b (d relative to x) in the lane's clip-buffer columns:
// the polygon's vertices in x / y slots 0 .. n-1 (approxcaps keeps the walk points in the e
// slots 0-5 and 8-13).  Returns n, 0 for an empty or degenerate region, -1 when a choice is not
// certain (or an approxcaps level above 2, left to the FP64 geometry).
template <int BALL>
__device__ __forceinline__ int ball_region_f32(const F2 d[3], const GeoParams &g, ClipBuf &cb, int lane, int *kind)
{
    const float delta = g.deltaf;
    const Col px = col(cb.x, lane), py = col(cb.y, lane);
    unsigned tags;
    int nin;
    if (BALL == NL_BALL_NOCAPS) {
        const int n = ball_walk_f32(d, g, px, py, &tags, &nin);
        if (n < 0) return -1;
        if (n < 3) return 0;
        *kind = (nin == 3 && n == 3) ? KIND_WHOLE : KIND_PARTIAL;
        return n;
    }
    // approxcaps: the walk, then the dyadic arc points between every exit and the next entry
    const Col ex = col(cb.e, lane);
    const Col wx = ex, wy = Col{ex.p + (8 << 5)};
    const int n = ball_walk_f32(d, g, wx, wy, &tags, &nin);
    if (n < 0) return -1;
    if (n < 2) return 0;
    const int level = g.cap_level;
    if (level > 2) return -1;
    const int per = (1 << level) - 1;
    int m = 0;
    for (int i = 0; i < n; i++) {
        const int j = i + 1 < n ? i + 1 : 0;
        if (m + 1 > kBallCap) return -1;
        const float x0 = wx[i], y0 = wy[i];
        px[m] = x0;
        py[m] = y0;
        m++;
        if (walk_tag(tags, i) == 2 && walk_tag(tags, j) == 1 && level > 0) {
            if (m + per > kBallCap) return -1;
            // dyadic bisection of the arc from W[i] to W[j]: each new point from its two
            // neighbours of the coarser level
            const float x1 = wx[j], y1 = wy[j];
            const F2 mid = arc_dir(x0 + x1, y0 + y1, delta);
            if (level == 1) {
                px[m] = mid.x; py[m] = mid.y; m++;
            } else {
                const F2 q1 = arc_dir(x0 + mid.x, y0 + mid.y, delta), q3 = arc_dir(mid.x + x1, mid.y + y1, delta);
                px[m] = q1.x; py[m] = q1.y; m++;
                px[m] = mid.x; py[m] = mid.y; m++;
                px[m] = q3.x; py[m] = q3.y; m++;
            }
        }
    }
    if (m < 3) return 0;
    *kind = (nin == 3 && n == 3) ? KIND_WHOLE : KIND_PARTIAL;
    return m;
}

// FP32 region of exactcaps (Sec. 5.2, Eq. (areacap)): the certified FP32 walk as for nocaps (a
// polygon when it has three points or more) and one cap for every exit followed by an entry,
// each integrated by one point at its centroid with weight its area, as the FP64 cap rule (the
// area delta^2 (2 th - sin 2 th) / 2, or / 4 with the printed weight, th = asin(chord / 2 delta);
// the series of 2 th - sin 2 th below 2 th = 0.5, where the difference loses FP32 digits).
// Coordinates relative to x, in the lane's clip-buffer columns: the polygon in x / y slots 0-5,
// the caps' centroids in x / y slots 8-10 and their areas in e slots 0-2.  Returns the polygon's
// vertex count (0 when under three points), -1 when the walk is not certain; *ncap caps.
__device__ __forceinline__ int exactcaps_region_f32(const F2 d[3], const GeoParams &g, ClipBuf &cb, int lane,
                                                    int *ncap, int *kind)
{
    const Col px = col(cb.x, lane), py = col(cb.y, lane), pe = col(cb.e, lane);
    unsigned tags;
    int nin;
    const int n = ball_walk_f32(d, g, px, py, &tags, &nin);
    *ncap = 0;
    if (n < 0) return -1;
    if (n < 2) return 0;
    const float delta = g.deltaf;
    int nc = 0;
    for (int i = 0; i < n; i++) {
        const int j = i + 1 < n ? i + 1 : 0;
        if (!(walk_tag(tags, i) == 2 && walk_tag(tags, j) == 1) || nc >= 3) continue;
        const F2 e = {px[i], py[i]}, f = {px[j], py[j]};
        const float cx = f.x - e.x, cy = f.y - e.y;
        const float chord = sqrtf(cx * cx + cy * cy);
        const float th = asinf(fminf(chord / (2.f * delta), 1.f));
        const float u = 2.f * th;
        float tms;   // 2 th - sin 2 th
        if (u < 0.5f) {
            const float u2 = u * u;
            float term = u * u2 / 6.f, sum = 0.f;
            for (int k = 1; k <= 6; k++) {
                sum += term;
                term *= -u2 / ((2.f * k + 2.f) * (2.f * k + 3.f));
            }
            tms = sum;
        } else {
            tms = u - sinf(u);
        }
        const float st = sinf(th);
        const float dc = tms > 0.f ? 4.f * delta * st * st * st / (3.f * tms) : delta;
        const float mx = 0.5f * (e.x + f.x), my = 0.5f * (e.y + f.y);
        const float im = rsqrtf(mx * mx + my * my);
        px[8 + nc] = dc * mx * im;
        py[8 + nc] = dc * my * im;
        pe[nc] = delta * delta * tms / (g.cap_printed ? 4.f : 2.f);
        nc++;
    }
    *ncap = nc;
    *kind = (nin == 3 && n == 3) ? KIND_WHOLE : KIND_PARTIAL;
    return n >= 3 ? n : 0;
}

// error of either); otherwise the FP64 test decides.  Returns 0 far, 1 near, -1 undecided.
__device__ __forceinline__ int near_f32(const F2 dl[3], float diamf, float eta)
{
    // dist = min over the edges of the distance from x (the origin) to the edge, 0 when x is
    // inside; each edge's squared distance is compared multiplied through by |e|^2 (no division)
    const float F = diamf + eta, Nr = diamf - eta, F2v = F * F, N2v = Nr > 0.f ? Nr * Nr : 0.f;
    const float o0 = dl[0].x * dl[1].y - dl[0].y * dl[1].x;
    const float o1 = dl[1].x * dl[2].y - dl[1].y * dl[2].x;
    const float o2 = dl[2].x * dl[0].y - dl[2].y * dl[0].x;
    if (o0 >= 0.f && o1 >= 0.f && o2 >= 0.f) return Nr > 0.f ? 1 : -1;   // x inside: dist 0
    bool all_far = true, any_near = false;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const F2 p = dl[i], q = dl[(i + 1) % 3];
        const float ex = q.x - p.x, ey = q.y - p.y;
        const float n = -(p.x * ex + p.y * ey), ee = ex * ex + ey * ey;
        float num, den;   // squared distance num / den
        if (n <= 0.f) { num = p.x * p.x + p.y * p.y; den = 1.f; }
        else if (n >= ee) { num = q.x * q.x + q.y * q.y; den = 1.f; }
        else { num = (p.x * p.x + p.y * p.y) * ee - n * n; den = ee; }
        all_far = all_far && num > F2v * den;
        any_near = any_near || num < N2v * den;
    }
    if (all_far) return 0;
    if (any_near) return 1;
    return -1;
}

// ---- near-singular test (values of psi = c/|x-y| need a special rule) ----
__device__ __forceinline__ D2 closest_on_seg(D2 a, D2 b, D2 x)
{
    double dx = sub(b.x, a.x), dy = sub(b.y, a.y);
    double t = dvd(add(mul(sub(x.x, a.x), dx), mul(sub(x.y, a.y), dy)), add(mul(dx, dx), mul(dy, dy)));
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    D2 p;
    p.x = add(a.x, mul(t, dx));
    p.y = add(a.y, mul(t, dy));
    return p;
}

// x within one diameter of T_b of the region (or inside it)
__device__ __forceinline__ bool is_near(const Region &R, const D2 V[3], D2 x)
{
    double diam2 = 0.0;
    for (int i = 0; i < 3; i++) {
        double dx = sub(V[(i + 1) % 3].x, V[i].x), dy = sub(V[(i + 1) % 3].y, V[i].y);
        double l = add(mul(dx, dx), mul(dy, dy));
        if (l > diam2) diam2 = l;
    }
    const int n = R.nv;
    bool inside = true;
    for (int i = 0; i < n; i++)
        if (orient(R.P[i], R.P[(i + 1) % n], x) < 0.0) inside = false;
    if (inside) return true;
    double best = INFINITY;
    for (int i = 0; i < n; i++) {
        D2 p = closest_on_seg(R.P[i], R.P[(i + 1) % n], x);
        double dx = sub(p.x, x.x), dy = sub(p.y, x.y);
        double d = add(mul(dx, dx), mul(dy, dy));
        if (d < best) best = d;
    }
    return best < diam2;
}

// splitmix64 finaliser (Steele, Lea, Flood 2014)
__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t record_hash(int a, int b, int q, int kind, int nv, int ncap)
{
    uint64_t h = mix64(((uint64_t)(uint32_t)a << 32) | (uint32_t)b);
    return mix64(h ^ (((uint64_t)q << 24) | ((uint64_t)kind << 16) | ((uint64_t)nv << 8) | (uint64_t)ncap));
}

}  // namespace nlg
