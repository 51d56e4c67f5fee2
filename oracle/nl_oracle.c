/*
 * nl_oracle.c -- plain, slow, FP64 CPU oracle for the P1 stiffness matrix of the
 * nonlocal diffusion operator with ball-supported kernels, following
 * D'Elia, Gunzburger, Vollmann, "A cookbook for finite element methods for
 * nonlocal problems, including quadrature rules and approximate Euclidean balls".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path; it is compiled with
 * -O2 -ffp-contract=off (no fused multiply-add, no fast-math) so that every
 * geometric predicate is evaluated exactly as written, left to right.
 *
 * What is computed (Sec. 7.2, Eq. (bformhj), with the fully discrete
 * quadrature of Sec. 7.3, Eq. (bformjqqh)):
 *
 *   D[j',j] = sum_{T_a} sum_{T_b} sum_q W_q sum_{S in R(x_q,T_b)} sum_r w_r |S|
 *             (phi_j(x)-phi_j(y)) (phi_j'(x)-phi_j'(y)) psi(x,y)
 *
 * over ALL K x K element pairs (the full (Omega u Omega_I)^2 matrix D of
 * Eq. (bform0)); A = D[Omega,Omega] and F = G - D[Omega,Omega_I] g follow from
 * the A-B-C assignment table of Sec. 7.2.  R(x,T_b) is the part of T_b that the
 * selected (approximate) ball keeps for the outer point x:
 *   barycenter  Sec. 4.2.3, Eq. (baryball)        whole T_b iff |x - bary_b| <= delta
 *   nocaps      Sec. 4.2.1 + Sec. 7.1 tasks 3-6   chord polygon of T_b n B_delta(x), fanned
 *   approxcaps  Sec. 4.2.2                        nocaps + each cap replaced by m-1 arc points
 *   exactcaps   Sec. 5.2                          nocaps triangles + one centroid point per cap
 *   ngon        Sec. 9 (regular inscribed polygon) T_b clipped by the regular N-gon
 *   overlap     Sec. 4.2.4, Eq. (overlap)          whole T_b iff T_b n B_delta(x) is non-empty
 *
 * Canonical geometry (all FP64, round-to-nearest, no contraction):
 *   G1 in-ball    dx=p.x-x.x; dy=p.y-x.y; (dx*dx + dy*dy) <= delta2   (closed ball, Eq. (inter))
 *   G2 barycentre ((v0+v1)+v2)/3.0                                    (Sec. 7.1 task 1)
 *   G3 edge roots q(l)=|p+l(q-p)-x|^2-delta^2 (Sec. 7.1 task 5), strict 0<l<1
 *   G4 nocaps     per edge i: emit v_i if inside, then the edge's roots by increasing l;
 *                 >= 3 points -> fan from the first (Sec. 7.1 task 6)
 *   G5 approxcaps recursive bisection of each exit->entry arc, p = x + u*(delta/sqrt(u.u))
 *   G6 exactcaps  cap area delta^2 (theta - sin theta cos theta) (Eq. (areacap)),
 *                 centroid at 4 delta sin^3 theta / (3 (2 theta - sin 2 theta)) (Sec. 5.2)
 *   G7 ngon       Sutherland-Hodgman against the N half-planes in order, keep orient >= 0
 *
 * The singular kernel psi = c / |x-y| (the paper names no rule, Sec. 2 and Sec. 3
 * remarks): when the outer point x lies within one diameter of T_b of the region
 * R (or inside it), R is integrated by the signed apex-x decomposition with a
 * Duffy collapse and a sinh substitution (near_polygon below), which makes the
 * integrand bounded; elsewhere the inner rule is used on the fan of R.
 *
 * Parity pins live in tests/test_oracle_pins.py (closed forms, paper Table 1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- enums (the oracle's own; mapped from strings by oracle/oracle.py) ---- */
enum { OR_BALL_BARYCENTER = 0, OR_BALL_NOCAPS = 1, OR_BALL_APPROXCAPS = 2,
       OR_BALL_EXACTCAPS = 3, OR_BALL_NGON = 4, OR_BALL_OVERLAP = 5,
       /* barycenter ball with the outer integral over T_a n B_delta(bary_b) only (Sec. 6.2,
          barycenter case; Table 3): that support approximated by nocaps / approxcaps */
       OR_BALL_BARY_NOCAPS = 6, OR_BALL_BARY_APPROXCAPS = 7 };
enum { OR_RULE_GAUSS3 = 0, OR_RULE_GAUSS4 = 1, OR_RULE_PAPER7 = 2,
       OR_RULE_DUNAVANT7 = 3, OR_RULE_DUNAVANT16 = 4, OR_RULE_SWITCH47 = 5 };
enum { OR_KERNEL_CONST = 0, OR_KERNEL_INV_DIST = 1 };
enum { OR_KIND_NONE = 0, OR_KIND_WHOLE = 1, OR_KIND_PARTIAL = 2 };

typedef struct {
    int32_t nv, nt;
    const double *vx, *vy;
    const int32_t *tri;             /* [3*nt], counter-clockwise */
} or_mesh;

typedef struct {
    double delta, kernel_c;
    int32_t kernel, ball, ngon_n, cap_m;
    const double *ngon_off;         /* [2*ngon_n] */
    int32_t outer, inner;
    int32_t duffy_n;                /* Gauss-Legendre points per direction of the Duffy rule */
    int32_t cap_printed;            /* 1: cap weight as printed in Sec. 5.2, (1/4) delta^2 (2t - sin 2t) */
    int32_t shifted;                /* 1: every outer point of T_a uses the ball centred at bary_a (Sec. 4.3,
                                       "shifted center approximate ball"); constant kernel only */
} or_cfg;

typedef struct {
    int32_t a, b;
    int8_t q, kind, nverts, ncaps;
} or_record;

typedef struct {
    /* COO of D restricted to the requested rows, sorted by (row, col), duplicates summed */
    int64_t nnz;
    int32_t *row, *col;
    double *val;
    int64_t n_pairs, n_qp_pairs, n_inter;
    or_record *rec;                 /* optional, n_inter records (sorted by a, b, q) */
    uint64_t *hash_a;               /* optional, [nt]: sum of record hashes per outer triangle */
    int64_t *count_a, *qp_a;        /* optional, [nt] */
} or_result;

#define MAXV 96
#define MAXCAP 8

/* ------------------------------------------------------------------------ */
/* Quadrature rules on the reference triangle: barycentric (l0,l1,l2) and a  */
/* weight; weights sum to 1 (multiply by the triangle area).                  */
/* ------------------------------------------------------------------------ */
typedef struct { int n; double p[16][4]; } or_rule;

static or_rule R_GAUSS3, R_GAUSS4, R_PAPER7, R_DUN7, R_DUN16;
static double GL_X[8][8], GL_W[8][8];   /* Gauss-Legendre on [0,1], n = 1..7 */
static int rules_ready = 0;

static void put(or_rule *r, double l0, double l1, double l2, double w)
{
    r->p[r->n][0] = l0; r->p[r->n][1] = l1; r->p[r->n][2] = l2; r->p[r->n][3] = w; r->n++;
}

static void put_s21(or_rule *r, double a, double w)  /* orbit (a, a, 1-2a) */
{
    double c = 1.0 - 2.0 * a;
    put(r, a, a, c, w); put(r, a, c, a, w); put(r, c, a, a, w);
}

static void put_s111(or_rule *r, double a, double b, double w) /* 6 permutations */
{
    double c = 1.0 - a - b;
    put(r, a, b, c, w); put(r, a, c, b, w); put(r, b, a, c, w);
    put(r, b, c, a, w); put(r, c, a, b, w); put(r, c, b, a, w);
}

static void gauss_legendre01(int n, double *x, double *w)
{
    /* Newton iteration on P_n over [-1,1], mapped to [0,1] (Golub-Welsch-free textbook form) */
    for (int i = 0; i < n; i++) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = 0.0;
            for (int k = 1; k <= n; k++) {
                double p2 = p1; p1 = p0;
                p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
            }
            pp = n * (z * p0 - p1) / (z * z - 1.0);
            double dz = p0 / pp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * pp * pp);   /* 2/((1-z^2)P'^2) on [-1,1], halved */
    }
}

static void init_rules(void)
{
    if (rules_ready) return;
    memset(&R_GAUSS3, 0, sizeof R_GAUSS3);
    memset(&R_GAUSS4, 0, sizeof R_GAUSS4);
    memset(&R_PAPER7, 0, sizeof R_PAPER7);
    memset(&R_DUN7, 0, sizeof R_DUN7);
    memset(&R_DUN16, 0, sizeof R_DUN16);
    /* three-point symmetric Gaussian rule, precision 2 (Sec. 5.3.1; interior points) */
    put_s21(&R_GAUSS3, 1.0 / 6.0, 1.0 / 3.0);
    /* four-point symmetric Gaussian rule, precision 3 (Sec. 6.1) */
    put(&R_GAUSS4, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0, -27.0 / 48.0);
    put_s21(&R_GAUSS4, 0.2, 25.0 / 48.0);
    /* seven-point vertex/mid-side/centroid rule, precision 3 (Sec. 6.3, Fig. 10):
       weights 27/60, 3/60, 8/60 relative to the area */
    put(&R_PAPER7, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0, 27.0 / 60.0);
    put(&R_PAPER7, 1.0, 0.0, 0.0, 3.0 / 60.0);
    put(&R_PAPER7, 0.0, 1.0, 0.0, 3.0 / 60.0);
    put(&R_PAPER7, 0.0, 0.0, 1.0, 3.0 / 60.0);
    put(&R_PAPER7, 0.5, 0.5, 0.0, 8.0 / 60.0);
    put(&R_PAPER7, 0.0, 0.5, 0.5, 8.0 / 60.0);
    put(&R_PAPER7, 0.5, 0.0, 0.5, 8.0 / 60.0);
    /* seven-point degree-5 rule (Radon 1948; Dunavant's degree-5 rule), closed form */
    {
        double s15 = sqrt(15.0);
        put(&R_DUN7, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0, 9.0 / 40.0);
        put_s21(&R_DUN7, (6.0 - s15) / 21.0, (155.0 - s15) / 1200.0);
        put_s21(&R_DUN7, (6.0 + s15) / 21.0, (155.0 + s15) / 1200.0);
    }
    /* sixteen-point degree-8 rule (Dunavant 1985), orbit structure 1 + 3*3 + 6;
       values solved from the moment equations by oracle/derive_dunavant16.py */
    put(&R_DUN16, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0, 0.1443156076777871682510911);
    put_s21(&R_DUN16, 0.4592925882927231560288155, 0.0950916342672846247938961);
    put_s21(&R_DUN16, 0.1705693077517602066222935, 0.1032173705347182502817916);
    put_s21(&R_DUN16, 0.05054722831703097545842355, 0.03245849762319808031092593);
    put_s111(&R_DUN16, 0.008394777409957605337213835, 0.2631128296346381134217858,
             0.02723031417443499426484469);
    for (int n = 1; n < 8; n++) gauss_legendre01(n, GL_X[n], GL_W[n]);
    rules_ready = 1;
}

static const or_rule *rule_of(int id)
{
    switch (id) {
    case OR_RULE_GAUSS3: return &R_GAUSS3;
    case OR_RULE_GAUSS4: return &R_GAUSS4;
    case OR_RULE_PAPER7: return &R_PAPER7;
    case OR_RULE_DUNAVANT7: return &R_DUN7;
    case OR_RULE_DUNAVANT16: return &R_DUN16;
    default: return NULL;
    }
}

/* ------------------------------------------------------------------------ */
/* Canonical geometry                                                        */
/* ------------------------------------------------------------------------ */
typedef struct { double x, y; } pt;

typedef struct {
    int kind, nverts, ncaps;
    pt P[MAXV];                     /* region polygon, counter-clockwise, fanned from P[0] */
    pt cap_c[MAXCAP];               /* exactcaps: cap centroids */
    double cap_w[MAXCAP];           /* exactcaps: cap areas */
} region;

/* G1: closed-ball membership */
static int in_ball(pt p, pt x, double d2)
{
    double dx = p.x - x.x;
    double dy = p.y - x.y;
    return (dx * dx + dy * dy) <= d2;
}

/* G2: barycentre */
static pt barycentre(pt v0, pt v1, pt v2)
{
    pt b;
    b.x = ((v0.x + v1.x) + v2.x) / 3.0;
    b.y = ((v0.y + v1.y) + v2.y) / 3.0;
    return b;
}

/* G3: roots of q(l) = |p + l (q - p) - x|^2 - delta^2 with 0 < l < 1 (strict),
   increasing; is_entry[k] = 1 if the boundary walk p->q enters the ball there. */
static int edge_roots(pt p, pt q, pt x, double d2, int p_inside, double *lam, int *is_entry)
{
    double dx = q.x - p.x, dy = q.y - p.y;
    double fx = p.x - x.x, fy = p.y - x.y;
    double a = dx * dx + dy * dy;
    double bh = fx * dx + fy * dy;
    double c = (fx * fx + fy * fy) - d2;
    double disc = bh * bh - a * c;
    int n = 0;
    if (disc < 0.0) return 0;
    double s = sqrt(disc);
    double l1 = (-bh - s) / a;
    double l2 = (-bh + s) / a;
    int k1 = (l1 > 0.0 && l1 < 1.0);
    int k2 = (l2 > 0.0 && l2 < 1.0);
    if (k1 && k2) {
        lam[0] = l1; is_entry[0] = 1;
        lam[1] = l2; is_entry[1] = 0;
        return 2;
    }
    if (k1) { lam[n] = l1; is_entry[n] = !p_inside; n++; }
    if (k2) { lam[n] = l2; is_entry[n] = !p_inside; n++; }
    return n;
}

/* G4 boundary walk of T_b n B_delta(x): vertices inside, then roots of each edge.
   Returns the count; tag[k] = 0 vertex, 1 entry root, 2 exit root. */
static int ball_walk(const pt *V, pt x, double d2, pt *out, int *tag, int *n_inside)
{
    int ins[3], n = 0;
    *n_inside = 0;
    for (int i = 0; i < 3; i++) { ins[i] = in_ball(V[i], x, d2); *n_inside += ins[i]; }
    for (int i = 0; i < 3; i++) {
        pt p = V[i], q = V[(i + 1) % 3];
        if (ins[i]) { out[n] = p; tag[n] = 0; n++; }
        double lam[2]; int ent[2];
        int nr = edge_roots(p, q, x, d2, ins[i], lam, ent);
        for (int k = 0; k < nr; k++) {
            out[n].x = p.x + lam[k] * (q.x - p.x);
            out[n].y = p.y + lam[k] * (q.y - p.y);
            tag[n] = ent[k] ? 1 : 2;
            n++;
        }
    }
    return n;
}

/* G5: arc point halfway (in angle) between e and n on the circle |y - x| = delta */
static pt arc_mid(pt e, pt n, pt x, double delta)
{
    double ux = (e.x - x.x) + (n.x - x.x);
    double uy = (e.y - x.y) + (n.y - x.y);
    double s = delta / sqrt(ux * ux + uy * uy);
    pt p;
    p.x = x.x + ux * s;
    p.y = x.y + uy * s;
    return p;
}

static void arc_fill(pt e, pt n, pt x, double delta, int level, pt *out, int *cnt)
{
    if (level == 0) return;
    pt m = arc_mid(e, n, x, delta);
    arc_fill(e, m, x, delta, level - 1, out, cnt);
    out[(*cnt)++] = m;
    arc_fill(m, n, x, delta, level - 1, out, cnt);
}

/* G6: exact circular cap between chord end points e and n */
static void cap_rule(pt e, pt n, pt x, double delta, int printed, pt *c, double *area)
{
    double cx = n.x - e.x, cy = n.y - e.y;
    double chord = sqrt(cx * cx + cy * cy);
    double th = asin(chord / (2.0 * delta));
    double two_th_minus_sin;      /* 2 theta - sin 2 theta */
    if (th < 0.05) {
        /* series of 2t - sin 2t = sum_{k>=1} (-1)^(k+1) (2t)^(2k+1) / (2k+1)! */
        double u = 2.0 * th, u2 = u * u, term = u * u2 / 6.0, sum = 0.0;
        for (int k = 1; k <= 6; k++) {
            sum += term;
            term *= -u2 / ((2.0 * k + 2.0) * (2.0 * k + 3.0));
        }
        two_th_minus_sin = sum;
    } else {
        two_th_minus_sin = 2.0 * th - sin(2.0 * th);
    }
    /* Eq. (areacap): delta^2 (theta - sin theta cos theta) = delta^2 (2 theta - sin 2 theta) / 2;
       the weight printed in Sec. 5.2 is half of that */
    *area = delta * delta * two_th_minus_sin / (printed ? 4.0 : 2.0);
    double st = sin(th);
    /* a tangent edge gives a zero chord: zero area, centroid on the circle (limit d -> delta) */
    double d = (two_th_minus_sin > 0.0) ? 4.0 * delta * st * st * st / (3.0 * two_th_minus_sin) : delta;
    double mx = (e.x + n.x) / 2.0 - x.x, my = (e.y + n.y) / 2.0 - x.y;
    double ml = sqrt(mx * mx + my * my);
    c->x = x.x + d * mx / ml;
    c->y = x.y + d * my / ml;
}

/* G7: orientation of p relative to the directed line a -> b */
static double orient(pt a, pt b, pt p)
{
    return (b.x - a.x) * (p.y - a.y) - (b.y - a.y) * (p.x - a.x);
}

static int clip_ngon(const pt *V, pt x, const or_cfg *cfg, pt *out)
{
    pt A[MAXV], B[MAXV];
    int n = 3;
    for (int i = 0; i < 3; i++) A[i] = V[i];
    int N = cfg->ngon_n;
    for (int k = 0; k < N && n > 0; k++) {
        int k1 = (k + 1) % N;
        pt P0, P1;
        P0.x = x.x + cfg->ngon_off[2 * k];  P0.y = x.y + cfg->ngon_off[2 * k + 1];
        P1.x = x.x + cfg->ngon_off[2 * k1]; P1.y = x.y + cfg->ngon_off[2 * k1 + 1];
        int m = 0;
        for (int i = 0; i < n; i++) {
            pt s = A[(i + n - 1) % n], e = A[i];
            double ds = orient(P0, P1, s), de = orient(P0, P1, e);
            if (m + 2 > MAXV) break;   /* never reached for convex input; bounds the buffer */
            if (de >= 0.0) {
                if (ds < 0.0) {
                    double t = ds / (ds - de);
                    B[m].x = s.x + t * (e.x - s.x); B[m].y = s.y + t * (e.y - s.y); m++;
                }
                B[m++] = e;
            } else if (ds >= 0.0) {
                double t = ds / (ds - de);
                B[m].x = s.x + t * (e.x - s.x); B[m].y = s.y + t * (e.y - s.y); m++;
            }
        }
        n = m;
        for (int i = 0; i < n; i++) A[i] = B[i];
    }
    for (int i = 0; i < n; i++) out[i] = A[i];
    return n;
}

/* distance-free overlap test T_b n B_delta(x) != empty (Eq. (overlap)):
   a vertex inside, an edge with a root in [0,1], or x inside T_b */
static int overlaps(const pt *V, pt x, double d2)
{
    for (int i = 0; i < 3; i++) if (in_ball(V[i], x, d2)) return 1;
    for (int i = 0; i < 3; i++) {
        pt p = V[i], q = V[(i + 1) % 3];
        double dx = q.x - p.x, dy = q.y - p.y;
        double fx = p.x - x.x, fy = p.y - x.y;
        double a = dx * dx + dy * dy;
        double bh = fx * dx + fy * dy;
        double c = (fx * fx + fy * fy) - d2;
        double disc = bh * bh - a * c;
        if (disc >= 0.0) {
            double s = sqrt(disc);
            double l1 = (-bh - s) / a, l2 = (-bh + s) / a;
            if ((l1 >= 0.0 && l1 <= 1.0) || (l2 >= 0.0 && l2 <= 1.0)) return 1;
        }
    }
    int in = 1;
    for (int i = 0; i < 3; i++) if (orient(V[i], V[(i + 1) % 3], x) < 0.0) in = 0;
    return in;
}

static void disc_region(const pt *V, pt x, const or_cfg *cfg, int ball, region *R);

/* R(x, T_b) for the selected ball (Sec. 4, Sec. 5.2, Sec. 9) */
static void make_region(const pt *V, pt x, const or_cfg *cfg, region *R)
{
    double delta = cfg->delta, d2 = delta * delta;
    R->kind = OR_KIND_NONE; R->nverts = 0; R->ncaps = 0;
    switch (cfg->ball) {
    case OR_BALL_BARYCENTER: {
        pt b = barycentre(V[0], V[1], V[2]);
        if (in_ball(b, x, d2)) {
            R->kind = OR_KIND_WHOLE; R->nverts = 3;
            for (int i = 0; i < 3; i++) R->P[i] = V[i];
        }
        return;
    }
    case OR_BALL_OVERLAP: {
        if (overlaps(V, x, d2)) {
            R->kind = OR_KIND_WHOLE; R->nverts = 3;
            for (int i = 0; i < 3; i++) R->P[i] = V[i];
        }
        return;
    }
    case OR_BALL_NOCAPS:
    case OR_BALL_APPROXCAPS:
    case OR_BALL_EXACTCAPS:
        disc_region(V, x, cfg, cfg->ball, R);
        return;
    case OR_BALL_NGON: {
        int n = clip_ngon(V, x, cfg, R->P);
        if (n >= 3) {
            R->nverts = n;
            int same = (n == 3);
            for (int i = 0; same && i < 3; i++)
                same = (R->P[i].x == V[i].x && R->P[i].y == V[i].y);
            R->kind = same ? OR_KIND_WHOLE : OR_KIND_PARTIAL;
        }
        return;
    }
    }
}

/* the nocaps / approxcaps / exactcaps region of triangle V around the ball B_delta(x) */
static void disc_region(const pt *V, pt x, const or_cfg *cfg, int ball, region *R)
{
    double delta = cfg->delta, d2 = delta * delta;
    R->kind = OR_KIND_NONE; R->nverts = 0; R->ncaps = 0;
    {
        pt W[12]; int tag[12], nin;
        int n = ball_walk(V, x, d2, W, tag, &nin);
        if (n < 3 && !(ball != OR_BALL_NOCAPS && n == 2)) return;
        if (n < 2) return;
        if (ball == OR_BALL_NOCAPS || ball == OR_BALL_EXACTCAPS) {
            if (n >= 3) {
                for (int i = 0; i < n; i++) R->P[i] = W[i];
                R->nverts = n;
            }
            if (ball == OR_BALL_EXACTCAPS) {
                for (int i = 0; i < n; i++) {
                    int j = (i + 1) % n;
                    if (tag[i] == 2 && tag[j] == 1) {
                        cap_rule(W[i], W[j], x, delta, cfg->cap_printed, &R->cap_c[R->ncaps], &R->cap_w[R->ncaps]);
                        R->ncaps++;
                    }
                }
            }
        } else {
            /* approxcaps: insert m-1 arc points between every exit and the next entry */
            int level = 0;
            while ((1 << level) < cfg->cap_m) level++;
            int m = 0;
            for (int i = 0; i < n; i++) {
                int j = (i + 1) % n;
                R->P[m++] = W[i];
                if (tag[i] == 2 && tag[j] == 1) arc_fill(W[i], W[j], x, delta, level, R->P, &m);
            }
            R->nverts = (m >= 3) ? m : 0;
        }
        if (R->nverts >= 3 || R->ncaps > 0)
            R->kind = (nin == 3 && n == 3) ? OR_KIND_WHOLE : OR_KIND_PARTIAL;
    }
}

/* The inputs the oracle's tables and buffers cover: the near rule's Gauss-Legendre tables hold
   1..7 points; a region holds at most MAXV vertices (3 + 64 for the N-gon, 6 + 3 (m - 1) for
   approxcaps with m arc segments, a power of two up to 16). */
static int cfg_ok(const or_cfg *cfg)
{
    if (cfg->kernel == OR_KERNEL_INV_DIST && (cfg->duffy_n < 1 || cfg->duffy_n > 7)) return 0;
    if (cfg->ball == OR_BALL_NGON && (cfg->ngon_n < 3 || cfg->ngon_n > 64 || !cfg->ngon_off)) return 0;
    if ((cfg->ball == OR_BALL_APPROXCAPS || cfg->ball == OR_BALL_BARY_APPROXCAPS) &&
        (cfg->cap_m < 1 || cfg->cap_m > 16 || (cfg->cap_m & (cfg->cap_m - 1)) != 0))
        return 0;
    return 1;
}

/* barycentric coordinates of y in triangle V (P1 basis functions phi_b(y)) */
static void barycentric(const pt *V, pt y, double *phi)
{
    double det = (V[1].x - V[0].x) * (V[2].y - V[0].y) - (V[2].x - V[0].x) * (V[1].y - V[0].y);
    double l1 = ((y.x - V[0].x) * (V[2].y - V[0].y) - (V[2].x - V[0].x) * (y.y - V[0].y)) / det;
    double l2 = ((V[1].x - V[0].x) * (y.y - V[0].y) - (y.x - V[0].x) * (V[1].y - V[0].y)) / det;
    phi[0] = 1.0 - l1 - l2;
    phi[1] = l1;
    phi[2] = l2;
}

static double tri_area(pt a, pt b, pt c)
{
    return 0.5 * fabs((b.x - a.x) * (c.y - a.y) - (c.x - a.x) * (b.y - a.y));
}

static double psi_of(const or_cfg *cfg, pt x, pt y)
{
    if (cfg->kernel == OR_KERNEL_CONST) return cfg->kernel_c;
    double dx = y.x - x.x, dy = y.y - x.y;
    return cfg->kernel_c / sqrt(dx * dx + dy * dy);
}

/* point of segment [a,b] closest to x */
static pt closest_on_seg(pt a, pt b, pt x)
{
    double dx = b.x - a.x, dy = b.y - a.y;
    double t = ((x.x - a.x) * dx + (x.y - a.y) * dy) / (dx * dx + dy * dy);
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    pt p; p.x = a.x + t * dx; p.y = a.y + t * dy;
    return p;
}

/* closest point of the convex polygon P (ccw) to x; returns 1 if x is inside */
static int closest_in_poly(const pt *P, int n, pt x, pt *c)
{
    int inside = 1;
    for (int i = 0; i < n; i++) if (orient(P[i], P[(i + 1) % n], x) < 0.0) inside = 0;
    if (inside) { *c = x; return 1; }
    double best = INFINITY;
    for (int i = 0; i < n; i++) {
        pt p = closest_on_seg(P[i], P[(i + 1) % n], x);
        double dx = p.x - x.x, dy = p.y - x.y, d = dx * dx + dy * dy;
        if (d < best) { best = d; *c = p; }
    }
    return 0;
}

typedef struct { double s0, s1[3], S2[3][3]; int64_t nqp; } inner_sums;

static void add_point(inner_sums *I, const pt *Vb, pt y, double omega)
{
    double phi[3];
    barycentric(Vb, y, phi);
    I->s0 += omega;
    for (int i = 0; i < 3; i++) {
        I->s1[i] += omega * phi[i];
        for (int k = 0; k < 3; k++) I->S2[i][k] += omega * phi[i] * phi[k];
    }
    I->nqp++;
}

/*
 * Near-singular rule for psi = c/|x - y| over the convex polygon P (ccw), for any x.
 * The polygon is the signed sum of the triangles (x, P_i, P_i+1).  Each one is split
 * at the foot F of the perpendicular from x onto the line of its edge (unit direction
 * e, distance d = |F - x|) into right triangles with legs d and tau (signed position of
 * P_i or P_i+1 along e relative to F).  On such a right triangle the collapsed (Duffy)
 * coordinate s in [0,1] and the sinh substitution tau t = d sinh(u) give
 *     y = x + s((F - x) + sgn(tau) d sinh(u) e),  dy / |x - y| = d ds du,
 * u in [0, asinh(|tau|/d)]: the integrand is bounded and smooth, so a Gauss-Legendre
 * rule with 2 points in s (exact: the P1 products are quadratic in s) and duffy_n
 * points on each unit panel in u integrates it.  (Duffy's collapse removes the 1/r at
 * the apex; the sinh substitution removes the near-singularity at the foot.)
 */
static void near_right_triangle(const or_cfg *cfg, const pt *Vb, pt x, pt F, double ex, double ey,
                                double d, double tau, double sign, inner_sums *I)
{
    if (tau == 0.0) return;
    double sg = tau > 0.0 ? 1.0 : -1.0;
    double U = asinh(fabs(tau) / d);
    int npan = (int)ceil(U);
    if (npan < 1) npan = 1;
    int nu = cfg->duffy_n;
    for (int p = 0; p < npan; p++) {
        double u0 = (double)p, u1 = (p + 1 < npan) ? (double)(p + 1) : U;
        double hw = u1 - u0;
        for (int j = 0; j < nu; j++) {
            double u = u0 + hw * GL_X[nu][j];
            double wu = hw * GL_W[nu][j];
            double sh = sinh(u);
            double wx = (F.x - x.x) + sg * d * sh * ex;
            double wy = (F.y - x.y) + sg * d * sh * ey;
            for (int i = 0; i < 2; i++) {
                double sv = GL_X[2][i], ws = GL_W[2][i];
                pt y;
                y.x = x.x + sv * wx;
                y.y = x.y + sv * wy;
                add_point(I, Vb, y, sign * sg * d * ws * wu * cfg->kernel_c);
            }
        }
    }
}

static void near_polygon(const or_cfg *cfg, const pt *Vb, pt x, const pt *P, int n, inner_sums *I)
{
    for (int i = 0; i < n; i++) {
        pt A = P[i], B = P[(i + 1) % n];
        double ex = B.x - A.x, ey = B.y - A.y;
        double L = sqrt(ex * ex + ey * ey);
        if (L == 0.0) continue;
        ex /= L; ey /= L;
        double tA = (A.x - x.x) * ex + (A.y - x.y) * ey;
        double tB = (B.x - x.x) * ex + (B.y - x.y) * ey;
        pt F;
        F.x = A.x - tA * ex;
        F.y = A.y - tA * ey;
        double fx = F.x - x.x, fy = F.y - x.y;
        double d = sqrt(fx * fx + fy * fy);
        if (d == 0.0) continue;                      /* x on the edge's line: zero-area piece */
        double sigma = (fx * ey - fy * ex) > 0.0 ? 1.0 : -1.0;
        near_right_triangle(cfg, Vb, x, F, ex, ey, d, tB, sigma, I);
        near_right_triangle(cfg, Vb, x, F, ex, ey, d, tA, -sigma, I);
    }
}

/* inner sums of the region: s0 = sum w psi, s1 = sum w psi phi_b, S2 = sum w psi phi_b phi_b^T */
static void inner_quadrature(const or_cfg *cfg, const pt *Vb, pt x, const region *R, inner_sums *I)
{
    memset(I, 0, sizeof *I);
    const or_rule *ri = rule_of(cfg->inner);
    int near = 0;
    if (cfg->kernel == OR_KERNEL_INV_DIST && R->nverts >= 3) {
        /* near: x within one diameter of T_b of the region (or inside it) */
        double diam2 = 0.0;
        for (int i = 0; i < 3; i++) {
            double dx = Vb[(i + 1) % 3].x - Vb[i].x, dy = Vb[(i + 1) % 3].y - Vb[i].y;
            double l = dx * dx + dy * dy;
            if (l > diam2) diam2 = l;
        }
        pt pc;
        closest_in_poly(R->P, R->nverts, x, &pc);
        double dx = pc.x - x.x, dy = pc.y - x.y;
        near = (dx * dx + dy * dy) < diam2;
    }
    if (near) {
        near_polygon(cfg, Vb, x, R->P, R->nverts, I);
    } else {
        for (int k = 1; k + 1 < R->nverts; k++) {
            pt S0 = R->P[0], S1 = R->P[k], S2p = R->P[k + 1];
            double area = tri_area(S0, S1, S2p);
            for (int r = 0; r < ri->n; r++) {
                const double *L = ri->p[r];
                pt y;
                y.x = L[0] * S0.x + L[1] * S1.x + L[2] * S2p.x;
                y.y = L[0] * S0.y + L[1] * S1.y + L[2] * S2p.y;
                add_point(I, Vb, y, L[3] * area * psi_of(cfg, x, y));
            }
        }
    }
    for (int c = 0; c < R->ncaps; c++)
        add_point(I, Vb, R->cap_c[c], R->cap_w[c] * psi_of(cfg, x, R->cap_c[c]));
}

/* ------------------------------------------------------------------------ */
/* Accumulation: open-addressing hash map (row, col) -> value                */
/* ------------------------------------------------------------------------ */
typedef struct { int64_t cap, n; int64_t *key; double *val; } hmap;

static void hm_init(hmap *h, int64_t cap)
{
    int64_t c = 1024;
    while (c < cap) c <<= 1;
    h->cap = c; h->n = 0;
    h->key = (int64_t *)malloc(sizeof(int64_t) * c);
    h->val = (double *)malloc(sizeof(double) * c);
    for (int64_t i = 0; i < c; i++) h->key[i] = -1;
}

static void hm_add(hmap *h, int64_t key, double v);

static void hm_grow(hmap *h)
{
    hmap g;
    hm_init(&g, h->cap * 2);
    for (int64_t i = 0; i < h->cap; i++) if (h->key[i] >= 0) hm_add(&g, h->key[i], h->val[i]);
    free(h->key); free(h->val);
    *h = g;
}

static void hm_add(hmap *h, int64_t key, double v)
{
    if (2 * (h->n + 1) > h->cap) hm_grow(h);
    uint64_t m = (uint64_t)h->cap - 1, i = ((uint64_t)key * 0x9E3779B97F4A7C15ULL) & m;
    while (h->key[i] >= 0 && h->key[i] != key) i = (i + 1) & m;
    if (h->key[i] < 0) { h->key[i] = key; h->val[i] = 0.0; h->n++; }
    h->val[i] += v;
}

/* splitmix64 finaliser (Steele, Lea, Flood 2014) */
static uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static uint64_t record_hash(int32_t a, int32_t b, int q, int kind, int nverts, int ncaps)
{
    uint64_t h = mix64(((uint64_t)(uint32_t)a << 32) | (uint32_t)b);
    return mix64(h ^ (((uint64_t)q << 24) | ((uint64_t)kind << 16) | ((uint64_t)nverts << 8) | (uint64_t)ncaps));
}

static int cmp_rec(const void *pa, const void *pb)
{
    const or_record *x = (const or_record *)pa, *y = (const or_record *)pb;
    if (x->a != y->a) return x->a < y->a ? -1 : 1;
    if (x->b != y->b) return x->b < y->b ? -1 : 1;
    return (x->q > y->q) - (x->q < y->q);
}

typedef struct { int64_t key; double val; } kv;

static int cmp_kv(const void *pa, const void *pb)
{
    int64_t x = ((const kv *)pa)->key, y = ((const kv *)pb)->key;
    return (x > y) - (x < y);
}

static pt vert(const or_mesh *m, int t, int i)
{
    pt p; int v = m->tri[3 * t + i];
    p.x = m->vx[v]; p.y = m->vy[v];
    return p;
}

/* largest triangle diameter (longest edge), used by the rule switch of Sec. 8 */
double or_hmax(const or_mesh *m)
{
    double h = 0.0;
    for (int t = 0; t < m->nt; t++)
        for (int i = 0; i < 3; i++) {
            pt p = vert(m, t, i), q = vert(m, t, (i + 1) % 3);
            double dx = q.x - p.x, dy = q.y - p.y, l = sqrt(dx * dx + dy * dy);
            if (l > h) h = l;
        }
    return h;
}

/* outer rule of the pair (a, b); Sec. 8: 4-point Gaussian rule if
   |bary_a - bary_b| < delta - h (h = largest triangle diameter), else 7-point rule */
static const or_rule *outer_rule(const or_mesh *m, const or_cfg *cfg, int a, int b, double hmax)
{
    if (cfg->outer != OR_RULE_SWITCH47) return rule_of(cfg->outer);
    pt ba = barycentre(vert(m, a, 0), vert(m, a, 1), vert(m, a, 2));
    pt bb = barycentre(vert(m, b, 0), vert(m, b, 1), vert(m, b, 2));
    double thr = cfg->delta - hmax;
    double dx = ba.x - bb.x, dy = ba.y - bb.y;
    if (thr > 0.0 && (dx * dx + dy * dy) < thr * thr) return &R_GAUSS4;
    return &R_PAPER7;
}

/*
 * Assemble D (or its rows selected by row_mask) by brute force over element pairs.
 *   a_list/n_a : outer triangles to visit (NULL = all)
 *   row_mask   : uint8 per node; if given, only pairs touching a masked node are
 *                visited and only masked rows are stored
 *   want_rec   : store every interaction record (a, q, b, kind, nverts, ncaps)
 *   want_hash  : per-outer-triangle record hash / count / qp-pair count
 */
int or_assemble(const or_mesh *m, const or_cfg *cfg, const int32_t *a_list, int32_t n_a,
                const uint8_t *row_mask, int32_t want_rec, int32_t want_hash,
                int32_t nthreads, or_result *res)
{
    init_rules();
    memset(res, 0, sizeof *res);
    if (!cfg_ok(cfg)) return -1;
    if (!rule_of(cfg->inner)) return -1;
    if (cfg->outer != OR_RULE_SWITCH47 && !rule_of(cfg->outer)) return -1;
    if (cfg->shifted && cfg->kernel != OR_KERNEL_CONST) return -1;
    const int bary_outer = (cfg->ball == OR_BALL_BARY_NOCAPS || cfg->ball == OR_BALL_BARY_APPROXCAPS);
    if (bary_outer && (cfg->kernel != OR_KERNEL_CONST || cfg->shifted)) return -1;
    int K = m->nt;
    int na = a_list ? n_a : K;
    double hmax = or_hmax(m);
    uint8_t *touch = NULL;
    int32_t *touch_list = NULL, n_touch = 0;
    if (row_mask) {
        touch = (uint8_t *)calloc(K, 1);
        touch_list = (int32_t *)malloc(sizeof(int32_t) * K);
        for (int t = 0; t < K; t++) {
            for (int i = 0; i < 3; i++) if (row_mask[m->tri[3 * t + i]]) touch[t] = 1;
            if (touch[t]) touch_list[n_touch++] = t;
        }
    }
    if (want_hash) {
        res->hash_a = (uint64_t *)calloc(K, sizeof(uint64_t));
        res->count_a = (int64_t *)calloc(K, sizeof(int64_t));
        res->qp_a = (int64_t *)calloc(K, sizeof(int64_t));
    }
    int nth = 1;
#ifdef _OPENMP
    nth = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
#endif
    hmap *maps = (hmap *)malloc(sizeof(hmap) * nth);
    or_record **recs = (or_record **)calloc(nth, sizeof(or_record *));
    int64_t *nrec = (int64_t *)calloc(nth, sizeof(int64_t)), *caprec = (int64_t *)calloc(nth, sizeof(int64_t));
    int64_t *npairs = (int64_t *)calloc(nth, sizeof(int64_t)), *nqp = (int64_t *)calloc(nth, sizeof(int64_t));
    for (int t = 0; t < nth; t++) hm_init(&maps[t], 1 << 16);

#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nth)
#endif
    for (int ia = 0; ia < na; ia++) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        int a = a_list ? a_list[ia] : ia;
        pt Va[3] = { vert(m, a, 0), vert(m, a, 1), vert(m, a, 2) };
        double area_a = tri_area(Va[0], Va[1], Va[2]);
        /* shifted ball (Sec. 4.3): the centre of every outer point's ball is T_a's barycentre */
        const pt centre_a = barycentre(Va[0], Va[1], Va[2]);
        int na_b = (row_mask && !touch[a]) ? n_touch : K;
        for (int ib = 0; ib < na_b; ib++) {
            int b = (row_mask && !touch[a]) ? touch_list[ib] : ib;
            pt Vb[3] = { vert(m, b, 0), vert(m, b, 1), vert(m, b, 2) };
            const or_rule *ro = outer_rule(m, cfg, a, b, hmax);
            double Maa[3][3] = {{0}}, Mbb[3][3] = {{0}}, Mab[3][3] = {{0}};
            int any = 0;
            if (bary_outer) {
                /* Sec. 6.2, barycenter case: the outer integrand is supported on
                   S = T_a n B_delta(bary_b) and the inner integral is over the whole T_b.  S is
                   approximated by nocaps / approxcaps around bary_b, fanned from its first point,
                   and the outer rule is applied on every subtriangle (the experiment of Table 3).
                   One interaction record per pair; qp-pairs = outer points x inner points. */
                const pt cb = barycentre(Vb[0], Vb[1], Vb[2]);
                region S;
                disc_region(Va, cb, cfg, cfg->ball == OR_BALL_BARY_NOCAPS ? OR_BALL_NOCAPS : OR_BALL_APPROXCAPS, &S);
                if (S.kind == OR_KIND_NONE || S.nverts < 3) continue;
                region Rb;
                Rb.kind = OR_KIND_WHOLE; Rb.nverts = 3; Rb.ncaps = 0;
                for (int i = 0; i < 3; i++) Rb.P[i] = Vb[i];
                inner_sums I;
                inner_quadrature(cfg, Vb, cb, &Rb, &I);   /* constant kernel: the same for every x */
                int64_t nout = 0;
                for (int k = 1; k + 1 < S.nverts; k++) {
                    const pt S0 = S.P[0], S1 = S.P[k], S2p = S.P[k + 1];
                    const double area = tri_area(S0, S1, S2p);
                    for (int q = 0; q < ro->n; q++) {
                        const double *L = ro->p[q];
                        pt x;
                        x.x = L[0] * S0.x + L[1] * S1.x + L[2] * S2p.x;
                        x.y = L[0] * S0.y + L[1] * S1.y + L[2] * S2p.y;
                        const double W = L[3] * area;
                        double la[3];
                        barycentric(Va, x, la);   /* phi_a at the outer point */
                        for (int i = 0; i < 3; i++)
                            for (int k2 = 0; k2 < 3; k2++) {
                                Maa[i][k2] += W * I.s0 * la[i] * la[k2];
                                Mbb[i][k2] += W * I.S2[i][k2];
                                Mab[i][k2] += W * la[i] * I.s1[k2];
                            }
                        nout++;
                    }
                }
                any = 1;
                nqp[tid] += nout * I.nqp;
                if (want_rec) {
                    if (nrec[tid] == caprec[tid]) {
                        caprec[tid] = caprec[tid] ? 2 * caprec[tid] : 4096;
                        recs[tid] = (or_record *)realloc(recs[tid], sizeof(or_record) * caprec[tid]);
                    }
                    or_record *r = &recs[tid][nrec[tid]++];
                    r->a = a; r->b = b; r->q = 0; r->kind = (int8_t)S.kind;
                    r->nverts = (int8_t)S.nverts; r->ncaps = 0;
                } else {
                    nrec[tid]++;
                }
                if (want_hash) {
                    res->hash_a[a] += record_hash(a, b, 0, S.kind, S.nverts, 0);
                    res->count_a[a] += 1;
                    res->qp_a[a] += nout * I.nqp;
                }
            }
            for (int q = 0; !bary_outer && q < ro->n; q++) {
                const double *L = ro->p[q];
                pt x;
                x.x = L[0] * Va[0].x + L[1] * Va[1].x + L[2] * Va[2].x;
                x.y = L[0] * Va[0].y + L[1] * Va[1].y + L[2] * Va[2].y;
                double W = L[3] * area_a;
                const pt xc = cfg->shifted ? centre_a : x;   /* centre of the ball */
                region R;
                make_region(Vb, xc, cfg, &R);
                if (R.kind == OR_KIND_NONE) continue;
                any = 1;
                inner_sums I;
                inner_quadrature(cfg, Vb, xc, &R, &I);
                nqp[tid] += I.nqp;
                if (want_rec) {
                    if (nrec[tid] == caprec[tid]) {
                        caprec[tid] = caprec[tid] ? 2 * caprec[tid] : 4096;
                        recs[tid] = (or_record *)realloc(recs[tid], sizeof(or_record) * caprec[tid]);
                    }
                    or_record *r = &recs[tid][nrec[tid]++];
                    r->a = a; r->b = b; r->q = (int8_t)q; r->kind = (int8_t)R.kind;
                    r->nverts = (int8_t)R.nverts; r->ncaps = (int8_t)R.ncaps;
                } else {
                    nrec[tid]++;
                }
                if (want_hash) {
                    res->hash_a[a] += record_hash(a, b, q, R.kind, R.nverts, R.ncaps);
                    res->count_a[a] += 1;
                    res->qp_a[a] += I.nqp;
                }
                /* (phi_j(x)-phi_j(y))(phi_j'(x)-phi_j'(y)) expanded over the local nodes:
                   aa: +W s0 phi_a phi_a^T, bb: +W S2, ab and ba: -W phi_a s1^T */
                for (int i = 0; i < 3; i++)
                    for (int k = 0; k < 3; k++) {
                        Maa[i][k] += W * I.s0 * L[i] * L[k];
                        Mbb[i][k] += W * I.S2[i][k];
                        Mab[i][k] += W * L[i] * I.s1[k];
                    }
            }
            if (!any) continue;
            npairs[tid]++;
            for (int i = 0; i < 3; i++) {
                int ai = m->tri[3 * a + i], bi = m->tri[3 * b + i];
                for (int k = 0; k < 3; k++) {
                    int ak = m->tri[3 * a + k], bk = m->tri[3 * b + k];
                    if (!row_mask || row_mask[ai]) hm_add(&maps[tid], (int64_t)ai * m->nv + ak, Maa[i][k]);
                    if (!row_mask || row_mask[bi]) hm_add(&maps[tid], (int64_t)bi * m->nv + bk, Mbb[i][k]);
                    if (!row_mask || row_mask[ai]) hm_add(&maps[tid], (int64_t)ai * m->nv + bk, -Mab[i][k]);
                    if (!row_mask || row_mask[bk]) hm_add(&maps[tid], (int64_t)bk * m->nv + ai, -Mab[i][k]);
                }
            }
        }
    }
    /* merge thread maps in thread order, then sort by (row, col) */
    hmap *all = &maps[0];
    for (int t = 1; t < nth; t++)
        for (int64_t i = 0; i < maps[t].cap; i++)
            if (maps[t].key[i] >= 0) hm_add(all, maps[t].key[i], maps[t].val[i]);
    kv *ent = (kv *)malloc(sizeof(kv) * (all->n + 1));
    int64_t ne = 0;
    for (int64_t i = 0; i < all->cap; i++)
        if (all->key[i] >= 0) { ent[ne].key = all->key[i]; ent[ne].val = all->val[i]; ne++; }
    qsort(ent, ne, sizeof(kv), cmp_kv);
    res->nnz = ne;
    res->row = (int32_t *)malloc(sizeof(int32_t) * (ne + 1));
    res->col = (int32_t *)malloc(sizeof(int32_t) * (ne + 1));
    res->val = (double *)malloc(sizeof(double) * (ne + 1));
    for (int64_t i = 0; i < ne; i++) {
        res->row[i] = (int32_t)(ent[i].key / m->nv);
        res->col[i] = (int32_t)(ent[i].key % m->nv);
        res->val[i] = ent[i].val;
    }
    free(ent);
    for (int t = 0; t < nth; t++) {
        res->n_pairs += npairs[t]; res->n_qp_pairs += nqp[t]; res->n_inter += nrec[t];
        free(maps[t].key); free(maps[t].val);
    }
    if (want_rec) {
        res->rec = (or_record *)malloc(sizeof(or_record) * (res->n_inter + 1));
        int64_t o = 0;
        for (int t = 0; t < nth; t++) {
            if (nrec[t]) memcpy(res->rec + o, recs[t], sizeof(or_record) * nrec[t]);
            o += nrec[t];
        }
        qsort(res->rec, res->n_inter, sizeof(or_record), cmp_rec);
    }
    for (int t = 0; t < nth; t++) free(recs[t]);
    free(recs); free(nrec); free(caprec); free(npairs); free(nqp); free(maps);
    free(touch); free(touch_list);
    return 0;
}

void or_free(or_result *r)
{
    free(r->row); free(r->col); free(r->val); free(r->rec);
    free(r->hash_a); free(r->count_a); free(r->qp_a);
    memset(r, 0, sizeof *r);
}

/* ---- single-region entry points for the geometry pins ---- */

/* region of T_b = (v[0..5]) for the outer point x: polygon and caps */
int or_region(const double *tri_xy, double x, double y, const or_cfg *cfg,
              int32_t *kind, int32_t *nverts, double *poly, int32_t *ncaps, double *caps)
{
    init_rules();
    if (!cfg_ok(cfg)) return -1;
    pt V[3] = { { tri_xy[0], tri_xy[1] }, { tri_xy[2], tri_xy[3] }, { tri_xy[4], tri_xy[5] } };
    pt X = { x, y };
    region R;
    make_region(V, X, cfg, &R);
    *kind = R.kind; *nverts = R.nverts; *ncaps = R.ncaps;
    for (int i = 0; i < R.nverts; i++) { poly[2 * i] = R.P[i].x; poly[2 * i + 1] = R.P[i].y; }
    for (int i = 0; i < R.ncaps; i++) {
        caps[3 * i] = R.cap_c[i].x; caps[3 * i + 1] = R.cap_c[i].y; caps[3 * i + 2] = R.cap_w[i];
    }
    return 0;
}

/* inner sums (s0, s1[3], S2[9]) of R(x, T_b) */
int or_inner(const double *tri_xy, double x, double y, const or_cfg *cfg, double *out, int64_t *nqp)
{
    init_rules();
    if (!cfg_ok(cfg)) return -1;
    pt V[3] = { { tri_xy[0], tri_xy[1] }, { tri_xy[2], tri_xy[3] }, { tri_xy[4], tri_xy[5] } };
    pt X = { x, y };
    region R;
    inner_sums I;
    make_region(V, X, cfg, &R);
    if (R.kind == OR_KIND_NONE) { memset(out, 0, sizeof(double) * 13); *nqp = 0; return 0; }
    inner_quadrature(cfg, V, X, &R, &I);
    out[0] = I.s0;
    for (int i = 0; i < 3; i++) out[1 + i] = I.s1[i];
    for (int i = 0; i < 3; i++) for (int k = 0; k < 3; k++) out[4 + 3 * i + k] = I.S2[i][k];
    *nqp = I.nqp;
    return 0;
}

/* quadrature rule table: returns the point count, fills [n][4] (l0, l1, l2, w) */
int or_rule_table(int32_t id, double *out)
{
    init_rules();
    const or_rule *r = rule_of(id);
    if (!r) return -1;
    memcpy(out, r->p, sizeof(double) * 4 * r->n);
    return r->n;
}

int or_gauss_legendre(int32_t n, double *x, double *w)
{
    init_rules();
    if (n < 1 || n > 7) return -1;
    for (int i = 0; i < n; i++) { x[i] = GL_X[n][i]; w[i] = GL_W[n][i]; }
    return n;
}

uint64_t or_record_hash(int32_t a, int32_t b, int32_t q, int32_t kind, int32_t nverts, int32_t ncaps)
{
    return record_hash(a, b, q, kind, nverts, ncaps);
}
