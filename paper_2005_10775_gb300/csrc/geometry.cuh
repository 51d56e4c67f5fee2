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
};

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

// Sutherland-Hodgman clip of the ccw triangle V by the regular polygon x + off_k
__device__ __forceinline__ int clip_ngon(const D2 V[3], D2 x, const GeoParams &g, D2 *out, int *overflow)
{
    D2 A[NL_MAXV], B[NL_MAXV];
    int n = 3;
    A[0] = V[0]; A[1] = V[1]; A[2] = V[2];
    const int N = g.ngon_n;
    D2 P0;
    P0.x = add(x.x, g.ngon[0]);
    P0.y = add(x.y, g.ngon[1]);
    const D2 first = P0;
    for (int k = 0; k < N && n > 0; k++) {
        D2 P1;
        if (k + 1 < N) {
            P1.x = add(x.x, g.ngon[2 * (k + 1)]);
            P1.y = add(x.y, g.ngon[2 * (k + 1) + 1]);
        } else {
            P1 = first;
        }
        // identity pass (every vertex on the kept side) is skipped: exact
        double o[NL_MAXV];
        bool all_in = true;
        for (int i = 0; i < n; i++) {
            o[i] = orient(P0, P1, A[i]);
            all_in = all_in && (o[i] >= 0.0);
        }
        if (!all_in) {
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
            for (int i = 0; i < n; i++) A[i] = B[i];
        }
        P0 = P1;
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
__device__ __forceinline__ void make_region(const D2 V[3], D2 bary_b, D2 x, const GeoParams &g, Region &R)
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
        int n = clip_ngon(V, x, g, R.P, &R.overflow);
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
