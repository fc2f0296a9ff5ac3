/*
 * creep_oracle.c -- FP64 reference evaluator of the per-receiver field of a
 * ray tracer with smooth-surface (creeping-wave) UTD diffraction.
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the CPU legs
 * of bench.py build, load or call this file.  It shares no code, header or
 * constant generator with the CUDA library; the Fock--Pekeris quadrature rule
 * and residue constants are passed in by oracle/fock.py (scipy Airy functions).
 *
 * What it computes (paper: "Indoor Wireless Signal Modeling with Smooth
 * Surface Diffraction Effects", Sec. II.B, Eqs. 1-4, Fig. 1):
 *   E(P) = U^i E^i(P) + sum_refl U^r E^r(P) + sum_creep E^d(P)
 * per receiver P and frequency, with
 *   E^i   the direct field of an isotropic source of polarisation p,
 *   E^r   planar PEC image reflections up to order 2 (Eq. 3 with R = -1/+1,
 *         flat faces) and the first-order reflection from each curved body
 *         (Eq. 3 with the Fock-uniform R and the curved-surface caustic
 *         distances),
 *   E^d   the first creeping ray in each direction around each body (Eq. 4),
 *         with T from the off-surface UTD of the references the paper cites,
 *         optionally with extra full turns round the body, and optionally
 *         fed by one planar reflection (the creeping rays of the source's
 *         image in a face, the wall->creeping paths).
 * The U's are the visibility bits of the straight sub-segments (Eqs. 1-2).
 *
 * Everything is plain double arithmetic in the order the formulas are written;
 * root finding is plain bisection; nothing is blocked or fused.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define C0_LIGHT 299792458.0
#define EPS_TRIM 1e-6
#define TWO_PI (2.0 * M_PI)

/* path type codes; a path is (type << 56) | (id1 << 28) | id2 */
enum { PT_LOS = 0, PT_R1 = 1, PT_R2 = 2, PT_RB = 3, PT_CP = 4, PT_CM = 5, PT_WCP = 6, PT_WCM = 7, PT_R3 = 8 };
/* receiver flags */
enum { FL_INSIDE = 1u, FL_CAUSTIC = 2u, FL_OVERFLOW = 8u };
/* enable mask */
enum { EN_LOS = 1, EN_PLANAR = 2, EN_BODYREFL = 4, EN_CREEP_SOFT = 8, EN_CREEP_HARD = 16, EN_WALL_CREEP = 32 };

/* -------------------------------------------------------------- vectors */
typedef struct { double x, y, z; } v3;
static inline v3 V(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static inline v3 add(v3 a, v3 b) { return V(a.x + b.x, a.y + b.y, a.z + b.z); }
static inline v3 sub(v3 a, v3 b) { return V(a.x - b.x, a.y - b.y, a.z - b.z); }
static inline v3 scl(v3 a, double s) { return V(a.x * s, a.y * s, a.z * s); }
static inline double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static inline v3 cross(v3 a, v3 b) {
    return V(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static inline double norm(v3 a) { return sqrt(dot(a, a)); }
static inline v3 unit(v3 a) { return scl(a, 1.0 / norm(a)); }

/* complex 3-vector */
typedef struct { cplx x, y, z; } c3;
static inline c3 CV(cplx x, cplx y, cplx z) { c3 r = {x, y, z}; return r; }
static inline c3 c3_from(v3 a) { return CV(a.x, a.y, a.z); }
static inline c3 c3_add(c3 a, c3 b) { return CV(a.x + b.x, a.y + b.y, a.z + b.z); }
static inline c3 c3_scl(c3 a, cplx s) { return CV(a.x * s, a.y * s, a.z * s); }
static inline cplx c3_dotr(c3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static inline c3 rscl(v3 a, cplx s) { return CV(a.x * s, a.y * s, a.z * s); }

/* ------------------------------------------------------ Fock functions */
typedef struct {
    const double *tau_re, *tau_im, *ws_re, *ws_im, *wh_re, *wh_im;
    const int *offsets;   /* n_buckets + 1 */
    int n_buckets;
    const double *res_alpha, *res_cs, *res_beta, *res_ch;
    int n_res;
    double xi_lo, xi_hi;
} fock_rule;

static cplx c_sing(void) { return cexp(-I * M_PI / 4.0) / (2.0 * sqrt(M_PI)); }

/* bucket 0: xi in [0, xi_hi]; bucket n >= 1: xi in [-n, -n+1) */
static int bucket_of(double xi) {
    if (xi >= 0.0) return 0;
    return (int)ceil(-xi);
}

/* Regular parts phat_s, phat_h = P + c/xi.  Quadrature inside [xi_lo, xi_hi],
 * residue series above xi_hi (Fock--Pekeris integrals). */
static void fock_phat(const fock_rule *R, double xi, cplx *ps, cplx *ph) {
    if (xi > R->xi_hi) {
        cplx e = cexp(-I * M_PI / 3.0);
        cplx ss = 0.0, sh = 0.0;
        for (int n = 0; n < R->n_res; ++n) {
            ss += cexp(-I * xi * R->res_alpha[n] * e) * R->res_cs[n];
            sh += cexp(-I * xi * R->res_beta[n] * e) * R->res_ch[n];
        }
        cplx pre = -cexp(-I * M_PI / 12.0) / (2.0 * sqrt(M_PI));
        *ps = pre * ss + c_sing() / xi;
        *ph = pre * sh + c_sing() / xi;
        return;
    }
    int b = bucket_of(xi);
    cplx ss = 0.0, sh = 0.0;
    for (int i = R->offsets[b]; i < R->offsets[b + 1]; ++i) {
        cplx tau = R->tau_re[i] + I * R->tau_im[i];
        cplx e = cexp(-I * xi * tau);
        ss += (R->ws_re[i] + I * R->ws_im[i]) * e;
        sh += (R->wh_re[i] + I * R->wh_im[i]) * e;
    }
    cplx pre = cexp(-I * M_PI / 4.0) / sqrt(M_PI);
    *ps = pre * ss;
    *ph = pre * sh;
}

/* Transition function F(X) = 2j sqrt(X) e^{jX} Int_{sqrt X}^inf e^{-j tau^2} dtau.
 * With tau = sqrt(X) + u and u = e^{-j pi/4} v the integral becomes
 *   F(X) = 2 sqrt(X) e^{j pi/4} Int_0^inf exp(-v^2 - 2 sqrt(X) e^{j pi/4} v) dv,
 * a smooth decaying integrand, done by composite 16-point Gauss-Legendre. */
static const double GL16_X[8] = {0.0950125098376374, 0.2816035507792589, 0.4580167776572274,
                                 0.6178762444026438, 0.7554044083550030, 0.8656312023878318,
                                 0.9445750230732326, 0.9894009349916499};
static const double GL16_W[8] = {0.1894506104550685, 0.1826034150449236, 0.1691565193950025,
                                 0.1495959888165767, 0.1246289712555339, 0.0951585116824928,
                                 0.0622535239386479, 0.0271524594117541};

static cplx transition_F(double X) {
    if (X <= 0.0) return 0.0;
    double sx = sqrt(X);
    cplx b = 2.0 * sx * cexp(I * M_PI / 4.0);
    /* decay rate of |integrand| ~ exp(-v^2 - sqrt(2X) v) */
    double rate = sqrt(2.0 * X);
    double vmax = (rate > 1.0) ? fmin(6.5, 44.0 / rate) : 6.5;
    double width = fmin(0.5, 1.0 / (1.0 + rate));
    int np = (int)ceil(vmax / width);
    double h = vmax / np;
    cplx s = 0.0;
    for (int p = 0; p < np; ++p) {
        double mid = (p + 0.5) * h, half = 0.5 * h;
        for (int i = 0; i < 8; ++i) {
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                double v = mid + sgn * half * GL16_X[i];
                s += half * GL16_W[i] * cexp(-v * v - b * v);
            }
        }
    }
    return b * s;
}

/* Fock bracket B = P + (c/xi)(1 - F(X)) = phat - c F(X)/xi, X = (K xi)^2. */
static void fock_bracket(const fock_rule *R, double xi, double K, cplx *Bs, cplx *Bh) {
    cplx ps, ph;
    fock_phat(R, xi, &ps, &ph);
    double X = (K * xi) * (K * xi);
    cplx cf = c_sing() * transition_F(X) / xi;
    *Bs = ps - cf;
    *Bh = ph - cf;
}

/* ------------------------------------------------------------ scene */
typedef struct { int type; v3 c; double a, h; } body;   /* type 0 sphere, 1 cylinder (axis +z, base c.z) */
typedef struct {
    v3 n; double d; int first, count;   /* plane n.x = d; triangles [first, first+count) in order list */
    int dielectric; cplx eps;           /* PEC, or a dielectric half-space of relative permittivity eps */
} face;

typedef struct {
    int n_tri; const double *tri; const int *tri_face; int *order; /* triangle ids grouped by face */
    int n_face; face *faces;
    const int *cand; int n_cand;        /* candidate face sequences [n_cand][3] (-1 padded), or none */
    int n_body; body *bodies;
    v3 tx, pol;
    int n_f; const double *freq;
    const fock_rule *fock;
    int max_order, enable;
    int max_enc;                        /* extra encirclements of the creeping rays (0: the first ray only) */
} scene;

static inline v3 tri_v(const scene *s, int t, int k) {
    const double *p = s->tri + 9 * t + 3 * k;
    return V(p[0], p[1], p[2]);
}

/* ---- op counters (algorithmic work model) ---- */
typedef struct {
    long long seg_tri, seg_body, inside_tri, image_cand, body_refl, creep_geom, paths, fock_evals;
} counters;

/* Segment A->B (trimmed to t in [EPS, 1-EPS]) against one closed triangle:
 * Moller-Trumbore with inclusive barycentric tests.  Parallel => no hit. */
static int seg_hits_tri(v3 A, v3 B, v3 v0, v3 v1, v3 v2) {
    v3 D = sub(B, A), e1 = sub(v1, v0), e2 = sub(v2, v0);
    v3 pv = cross(D, e2);
    double det = dot(e1, pv);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    v3 tv = sub(A, v0);
    double u = dot(tv, pv) * inv;
    if (u < 0.0 || u > 1.0) return 0;
    v3 qv = cross(tv, e1);
    double v = dot(D, qv) * inv;
    if (v < 0.0 || u + v > 1.0) return 0;
    double t = dot(e2, qv) * inv;
    return (t >= EPS_TRIM && t <= 1.0 - EPS_TRIM);
}

/* Segment vs open solid body.  A tangent touch does not obstruct. */
static int seg_hits_body(v3 A, v3 B, const body *b) {
    v3 D = sub(B, A);
    if (b->type == 0) {
        v3 w = sub(b->c, A);
        double t = dot(w, D) / dot(D, D);
        if (t < EPS_TRIM) t = EPS_TRIM;
        if (t > 1.0 - EPS_TRIM) t = 1.0 - EPS_TRIM;
        v3 q = sub(add(A, scl(D, t)), b->c);
        return dot(q, q) < b->a * b->a;
    }
    /* cylinder: rho(t) < a  and  cz < z(t) < cz + h  for some t in [EPS, 1-EPS] */
    double lo = EPS_TRIM, hi = 1.0 - EPS_TRIM;  /* closed range */
    double ox = A.x - b->c.x, oy = A.y - b->c.y;
    double qa = D.x * D.x + D.y * D.y, qb = 2.0 * (ox * D.x + oy * D.y), qc = ox * ox + oy * oy - b->a * b->a;
    double t1, t2;            /* open interval where rho < a */
    if (qa == 0.0) {
        if (!(qc < 0.0)) return 0;
        t1 = -INFINITY; t2 = INFINITY;
    } else {
        double disc = qb * qb - 4.0 * qa * qc;
        if (!(disc > 0.0)) return 0;
        double sq = sqrt(disc);
        t1 = (-qb - sq) / (2.0 * qa);
        t2 = (-qb + sq) / (2.0 * qa);
    }
    double t3, t4;            /* open interval where cz < z < cz + h */
    if (D.z == 0.0) {
        if (!(A.z > b->c.z && A.z < b->c.z + b->h)) return 0;
        t3 = -INFINITY; t4 = INFINITY;
    } else {
        double ta = (b->c.z - A.z) / D.z, tb = (b->c.z + b->h - A.z) / D.z;
        t3 = fmin(ta, tb); t4 = fmax(ta, tb);
    }
    double olo = fmax(t1, t3), ohi = fmin(t2, t4);   /* open (olo, ohi) */
    if (!(olo < ohi)) return 0;
    return (olo < hi) && (ohi > lo);
}

/* Visibility of the open segment A->B.  Triangles of faces skip_f1/skip_f2
 * (faces the endpoints lie on) and body skip_b are not tested. */
static int visible(const scene *s, v3 A, v3 B, int skip_f1, int skip_f2, int skip_b, counters *ct) {
    for (int t = 0; t < s->n_tri; ++t) {
        int f = s->tri_face[t];
        if (f == skip_f1 || f == skip_f2) continue;
        ct->seg_tri++;
        if (seg_hits_tri(A, B, tri_v(s, t, 0), tri_v(s, t, 1), tri_v(s, t, 2))) return 0;
    }
    for (int b = 0; b < s->n_body; ++b) {
        if (b == skip_b) continue;
        ct->seg_body++;
        if (seg_hits_body(A, B, &s->bodies[b])) return 0;
    }
    return 1;
}

static int inside_body(v3 P, const body *b) {
    if (b->type == 0) { v3 d = sub(P, b->c); return dot(d, d) <= b->a * b->a; }
    double dx = P.x - b->c.x, dy = P.y - b->c.y;
    return (dx * dx + dy * dy <= b->a * b->a) && P.z >= b->c.z && P.z <= b->c.z + b->h;
}

/* Closed point-in-triangle test for a point on the triangle's plane (edge functions). */
static int point_in_tri(v3 Q, v3 v0, v3 v1, v3 v2) {
    v3 n = cross(sub(v1, v0), sub(v2, v0));
    if (dot(cross(sub(v1, v0), sub(Q, v0)), n) < 0.0) return 0;
    if (dot(cross(sub(v2, v1), sub(Q, v1)), n) < 0.0) return 0;
    if (dot(cross(sub(v0, v2), sub(Q, v2)), n) < 0.0) return 0;
    return 1;
}

static int point_in_face(const scene *s, int f, v3 Q, counters *ct) {
    const face *F = &s->faces[f];
    for (int i = 0; i < F->count; ++i) {
        int t = s->order[F->first + i];
        ct->inside_tri++;
        if (point_in_tri(Q, tri_v(s, t, 0), tri_v(s, t, 1), tri_v(s, t, 2))) return 1;
    }
    return 0;
}

/* ------------------------------------------------------------ source */
/* Isotropic source of polarisation p: unit field vector along the part of p
 * transverse to the departure direction d, amplitude 1 at 1 m. */
static v3 source_pol(const scene *s, v3 d) {
    v3 pt = sub(s->pol, scl(d, dot(s->pol, d)));
    double n = norm(pt);
    if (n == 0.0) return V(0, 0, 0);
    return scl(pt, 1.0 / n);
}

/* PEC mirror of a field vector at a face with unit normal n: E -> -E + 2(n.E)n */
static c3 pec_mirror(c3 E, v3 n) {
    cplx en = c3_dotr(E, n);
    return CV(-E.x + 2.0 * en * n.x, -E.y + 2.0 * en * n.y, -E.z + 2.0 * en * n.z);
}

/* Reflection of a field vector E at face F, the ray arriving along si and
 * leaving along sr.  PEC: the image mirror above.  Dielectric half-space of
 * relative permittivity eps (e^{+jwt}: eps = eps' - j eps''): the Fresnel
 * coefficients at the incidence angle (cos = |si.n|)
 *   G_perp = (cos - r) / (cos + r),  G_par = (eps cos - r) / (eps cos + r),
 *   r = sqrt(eps - sin^2) (principal branch),
 * applied in the basis e_perp = unit(n x si), e_par = e_perp x si before and
 * e_perp x sr after the bounce (the basis in which the PEC mirror is
 * G_perp = -1, G_par = +1, the limit eps -> infinity).  At normal incidence
 * G_par = -G_perp and the reflection is G_perp E for any e_perp. */
static c3 reflect_at(const face *F, c3 E, v3 si, v3 sr) {
    if (!F->dielectric) return pec_mirror(E, F->n);
    double cth = fabs(dot(si, F->n));
    double s2 = 1.0 - cth * cth;
    cplx r = csqrt(F->eps - s2);
    cplx gs = (cth - r) / (cth + r);
    cplx gp = (F->eps * cth - r) / (F->eps * cth + r);
    v3 ep = cross(F->n, si);
    double ne = norm(ep);
    if (ne == 0.0) return c3_scl(E, gs);
    ep = scl(ep, 1.0 / ne);
    v3 epi = cross(ep, si), epr = cross(ep, sr);
    cplx a = c3_dotr(E, ep), b = c3_dotr(E, epi);
    return c3_add(rscl(ep, gs * a), rscl(epr, gp * b));
}

static v3 mirror_point(v3 X, const face *F) {
    double dist = dot(F->n, X) - F->d;
    return sub(X, scl(F->n, 2.0 * dist));
}

static inline uint64_t pcode(int type, int id1, int id2) {
    return ((uint64_t)type << 56) | ((uint64_t)id1 << 28) | (uint64_t)id2;
}

/* ------------------------------------------------------------ per-receiver */
typedef struct {
    c3 *E;             /* [n_f] accumulated field */
    double *Sabs;      /* [n_f] sum over paths of |E_path| (conditioning of the coherent sum) */
    double *pathE;     /* or NULL: [cap][n_f][3][2] each listed path's own field */
    int n_f;
    uint64_t *paths; int n_paths, cap;
    unsigned flags;
    counters ct;
} rx_state;

static void add_path(rx_state *st, uint64_t code) {
    if (st->n_paths < st->cap) st->paths[st->n_paths] = code;
    else st->flags |= FL_OVERFLOW;
    st->n_paths++;
    st->ct.paths++;
}

static double kwave(double f) { return TWO_PI * f / C0_LIGHT; }

static inline double c3_norm(c3 v) {
    return sqrt(creal(v.x) * creal(v.x) + cimag(v.x) * cimag(v.x) + creal(v.y) * creal(v.y) + cimag(v.y) * cimag(v.y) +
                creal(v.z) * creal(v.z) + cimag(v.z) * cimag(v.z));
}
/* add one path's field at frequency f */
static inline void accum(rx_state *st, int f, c3 v) {
    st->E[f] = c3_add(st->E[f], v);
    st->Sabs[f] += c3_norm(v);
    int idx = st->n_paths - 1;                 /* the path just listed */
    if (st->pathE && idx >= 0 && idx < st->cap) {
        double *o = st->pathE + ((size_t)idx * st->n_f + f) * 6;
        o[0] += creal(v.x); o[1] += cimag(v.x);
        o[2] += creal(v.y); o[3] += cimag(v.y);
        o[4] += creal(v.z); o[5] += cimag(v.z);
    }
}

/* Planar image path through the faces fs[0..k-1] in that order (k <= 3):
 * images S_m of the source in faces fs[0..m-1]; backwards from P, Q_m is
 * where S_{m+1} -> Q_{m+1} (Q_k = P) crosses face fs[m]'s plane (the two
 * strictly on opposite sides) and must lie in that face; then every leg
 * S -> Q_0 -> ... -> P clear of all triangles but those of the faces at its
 * ends.  Field: the source's polarisation reflected at each point in turn. */
static void seq_path(const scene *s, const int *fs, int k, v3 P, rx_state *st, uint64_t code) {
    v3 S = s->tx;
    v3 img[4];
    img[0] = S;
    for (int m = 0; m < k; ++m) img[m + 1] = mirror_point(img[m], &s->faces[fs[m]]);
    st->ct.image_cand++;
    v3 Q[3], X = P;
    for (int m = k - 1; m >= 0; --m) {
        const face *F = &s->faces[fs[m]];
        double di = dot(F->n, img[m + 1]) - F->d, dx = dot(F->n, X) - F->d;
        if (!(di * dx < 0.0)) return;
        Q[m] = add(img[m + 1], scl(sub(X, img[m + 1]), di / (di - dx)));
        if (!point_in_face(s, fs[m], Q[m], &st->ct)) return;
        X = Q[m];
    }
    if (!visible(s, S, Q[0], fs[0], -1, -1, &st->ct)) return;
    for (int m = 0; m + 1 < k; ++m)
        if (!visible(s, Q[m], Q[m + 1], fs[m], fs[m + 1], -1, &st->ct)) return;
    if (!visible(s, Q[k - 1], P, fs[k - 1], -1, -1, &st->ct)) return;
    add_path(st, code);
    double L = norm(sub(Q[0], S)) + norm(sub(P, Q[k - 1]));
    for (int m = 0; m + 1 < k; ++m) L += norm(sub(Q[m + 1], Q[m]));
    v3 din = unit(sub(Q[0], S));
    c3 e = c3_from(source_pol(s, din));
    for (int m = 0; m < k; ++m) {
        v3 dout = unit(sub(m + 1 < k ? Q[m + 1] : P, Q[m]));
        e = reflect_at(&s->faces[fs[m]], e, din, dout);
        din = dout;
    }
    for (int f = 0; f < s->n_f; ++f) {
        double kw = kwave(s->freq[f]);
        accum(st, f, c3_scl(e, cexp(-I * kw * L) / L));
    }
}

/* LOS and planar image paths (order 1 and 2 over all faces and face pairs,
 * or, with a candidate list, orders 1-3 over its sequences); PEC or
 * dielectric faces. */
static void planar_paths(const scene *s, v3 P, rx_state *st) {
    v3 S = s->tx;
    if (s->enable & EN_LOS) {
        if (visible(s, S, P, -1, -1, -1, &st->ct)) {
            add_path(st, pcode(PT_LOS, 0, 0));
            double R = norm(sub(P, S));
            v3 e = source_pol(s, unit(sub(P, S)));
            for (int f = 0; f < s->n_f; ++f) {
                double k = kwave(s->freq[f]);
                accum(st, f, rscl(e, cexp(-I * k * R) / R));
            }
        }
    }
    if (!(s->enable & EN_PLANAR)) return;
    if (s->cand) {
        /* candidate mode: orders 1 and 2 listed by their faces, order 3 by
         * the sequence's index in the list */
        for (int q = 0; q < s->n_cand; ++q) {
            const int *fs = s->cand + 3 * q;
            int k = (fs[0] >= 0) + (fs[1] >= 0) + (fs[2] >= 0);
            if (k < 1 || k > s->max_order) continue;
            uint64_t code = (k == 1) ? pcode(PT_R1, fs[0], 0) : (k == 2) ? pcode(PT_R2, fs[0], fs[1]) : pcode(PT_R3, q, 0);
            seq_path(s, fs, k, P, st, code);
        }
        return;
    }
    if (s->max_order >= 1) {
        for (int i = 0; i < s->n_face; ++i) {
            const face *Fi = &s->faces[i];
            st->ct.image_cand++;
            double dS = dot(Fi->n, S) - Fi->d, dP = dot(Fi->n, P) - Fi->d;
            if (!(dS * dP > 0.0)) continue;
            v3 S1 = mirror_point(S, Fi);
            double d1 = dot(Fi->n, S1) - Fi->d;
            double t = d1 / (d1 - dP);
            v3 Q = add(S1, scl(sub(P, S1), t));
            if (!point_in_face(s, i, Q, &st->ct)) continue;
            if (!visible(s, S, Q, i, -1, -1, &st->ct)) continue;
            if (!visible(s, Q, P, i, -1, -1, &st->ct)) continue;
            add_path(st, pcode(PT_R1, i, 0));
            double L = norm(sub(Q, S)) + norm(sub(P, Q));
            c3 e = reflect_at(Fi, c3_from(source_pol(s, unit(sub(Q, S)))), unit(sub(Q, S)), unit(sub(P, Q)));
            for (int f = 0; f < s->n_f; ++f) {
                double k = kwave(s->freq[f]);
                accum(st, f, c3_scl(e, cexp(-I * k * L) / L));
            }
        }
    }
    if (s->max_order >= 2) {
        for (int i = 0; i < s->n_face; ++i) {
            const face *Fi = &s->faces[i];
            v3 S1 = mirror_point(S, Fi);
            for (int j = 0; j < s->n_face; ++j) {
                if (j == i) continue;
                const face *Fj = &s->faces[j];
                st->ct.image_cand++;
                v3 S2 = mirror_point(S1, Fj);
                double d2 = dot(Fj->n, S2) - Fj->d, dP = dot(Fj->n, P) - Fj->d;
                if (!(d2 * dP < 0.0)) continue;          /* S2 -> P must cross plane j */
                double t2 = d2 / (d2 - dP);
                v3 Q2 = add(S2, scl(sub(P, S2), t2));
                if (!point_in_face(s, j, Q2, &st->ct)) continue;
                double e1 = dot(Fi->n, S1) - Fi->d, eq = dot(Fi->n, Q2) - Fi->d;
                if (!(e1 * eq < 0.0)) continue;          /* S1 -> Q2 must cross plane i */
                double t1 = e1 / (e1 - eq);
                v3 Q1 = add(S1, scl(sub(Q2, S1), t1));
                if (!point_in_face(s, i, Q1, &st->ct)) continue;
                if (!visible(s, S, Q1, i, -1, -1, &st->ct)) continue;
                if (!visible(s, Q1, Q2, i, j, -1, &st->ct)) continue;
                if (!visible(s, Q2, P, j, -1, -1, &st->ct)) continue;
                add_path(st, pcode(PT_R2, i, j));
                double L = norm(sub(Q1, S)) + norm(sub(Q2, Q1)) + norm(sub(P, Q2));
                c3 e = reflect_at(Fi, c3_from(source_pol(s, unit(sub(Q1, S)))), unit(sub(Q1, S)), unit(sub(Q2, Q1)));
                e = reflect_at(Fj, e, unit(sub(Q2, Q1)), unit(sub(P, Q2)));
                for (int f = 0; f < s->n_f; ++f) {
                    double k = kwave(s->freq[f]);
                    accum(st, f, c3_scl(e, cexp(-I * k * L) / L));
                }
            }
        }
    }
}

/* 2-D reflection point on a circle of radius a centred at the origin, for
 * points S and P (2-D, outside), lit geometry.  Q = a (cos psi u + sin psi v)
 * with u = S/|S|, v the in-plane unit normal towards P; psi in (0, gamma).
 * Found by bisection on d/dpsi (|S-Q| + |Q-P|) = 0 (law of reflection). */
static double refl_psi(double a, double dS, double px, double py, double gamma) {
    /* S = (dS, 0), P = (px, py) in the (u, v) frame */
    double lo = 0.0, hi = gamma;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;        /* interval at double resolution */
        double qx = a * cos(mid), qy = a * sin(mid);
        double tx = -a * sin(mid), ty = a * cos(mid);   /* dQ/dpsi */
        double sx = qx - dS, sy = qy;
        double rx = qx - px, ry = qy - py;
        double g = (sx * tx + sy * ty) / sqrt(sx * sx + sy * sy) + (rx * tx + ry * ty) / sqrt(rx * rx + ry * ry);
        if (g < 0.0) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* angle between two vectors in [0, pi] */
static double angle_between(v3 a, v3 b) { return atan2(norm(cross(a, b)), dot(a, b)); }

/* Geometry of the GO reflection point on a curved body. */
typedef struct {
    v3 Q, n;               /* reflection point, outward unit normal */
    double inv_f1, inv_f2; /* 1/rho^r = 1/s^i + inv_f (spherical incident wave) */
    double rho_g;          /* surface radius of curvature in the plane of incidence */
} refl_geom;

/* Geometry of one creeping ray (Fig. 1: attach Q1 = Q', shed Q2 = Q). */
typedef struct {
    v3 Q1, Q2, n1, n2;     /* attach/shed points and outward normals */
    double sp, t, sq;      /* s' (source->Q1), geodesic length, s (Q2->receiver) */
    double amp;            /* (1/s') * divergence * spreading, without T and phase */
    double rho_g;          /* geodesic radius of curvature (constant along the ray) */
    int caustic_j;         /* 1: the ray crossed the source axis (factor +j) */
    double dperp_P;        /* receiver distance from the source axis (sphere; 0 for cylinder) */
    int turns;             /* extra full encirclements */
} creep_geom;

/* Frame of a sphere/cylinder problem: u towards S, v in the (S, c, P) plane towards P. */
typedef struct { v3 u, v; double ds, dp, gam, bs, bp, pu, pv; } body_frame;

static void sphere_frame(const body *B, v3 S, v3 P, body_frame *F) {
    v3 ws = sub(S, B->c), wp = sub(P, B->c);
    F->ds = norm(ws); F->dp = norm(wp);
    F->u = scl(ws, 1.0 / F->ds);
    F->gam = angle_between(ws, wp);
    v3 vperp = sub(wp, scl(F->u, dot(wp, F->u)));
    double nv = norm(vperp);
    if (nv == 0.0) {
        v3 tmp = fabs(F->u.x) < 0.9 ? V(1, 0, 0) : V(0, 1, 0);
        F->v = unit(cross(F->u, tmp));
    } else {
        /* a second Gram-Schmidt pass: when P lies on (or within rounding of)
           the S-c axis, vperp is rounding noise and its normalisation alone
           need not be perpendicular to u */
        F->v = scl(vperp, 1.0 / nv);
        F->v = unit(sub(F->v, scl(F->u, dot(F->v, F->u))));
    }
    F->bs = acos(B->a / F->ds); F->bp = acos(B->a / F->dp);
    F->pu = dot(wp, F->u); F->pv = dot(wp, F->v);
}

/* horizontal frame of a vertical cylinder; returns 0 if S or P is over the footprint */
static int cylinder_frame(const body *B, v3 S, v3 P, body_frame *F) {
    double sx = S.x - B->c.x, sy = S.y - B->c.y, px = P.x - B->c.x, py = P.y - B->c.y;
    F->ds = sqrt(sx * sx + sy * sy); F->dp = sqrt(px * px + py * py);
    if (!(F->ds > B->a) || !(F->dp > B->a)) return 0;
    F->u = V(sx / F->ds, sy / F->ds, 0.0);
    F->gam = atan2(fabs(sx * py - sy * px), sx * px + sy * py);
    /* v = +-(z x u), the horizontal unit vector normal to u, turned toward P;
       side = (z x u).(P - c) >= 0 selects +.  (Normalising p - (p.u)u instead
       gives a v that is not normal to u when P lies on the S-c line in
       projection, where that vector is rounding noise.) */
    double side = F->u.x * py - F->u.y * px;
    F->v = (side < 0.0) ? V(F->u.y, -F->u.x, 0.0) : V(-F->u.y, F->u.x, 0.0);
    F->bs = acos(B->a / F->ds); F->bp = acos(B->a / F->dp);
    F->pu = px * F->u.x + py * F->u.y; F->pv = px * F->v.x + py * F->v.y;
    return 1;
}

/* Sphere: reflection point exists iff the receiver is strictly on the lit side
 * (gamma < beta_s + beta_p).  Caustic distances for a spherical wave on a
 * sphere: 1/rho1 = 1/s^i + 2/(a cos), 1/rho2 = 1/s^i + 2 cos/a. */
static int sphere_reflection(const body *B, v3 S, v3 P, refl_geom *G) {
    body_frame F;
    sphere_frame(B, S, P, &F);
    if (!(F.gam - F.bs - F.bp < 0.0)) return 0;
    double psi = refl_psi(B->a, F.ds, F.pu, F.pv, F.gam);
    G->n = add(scl(F.u, cos(psi)), scl(F.v, sin(psi)));
    G->Q = add(B->c, scl(G->n, B->a));
    double cth = -dot(unit(sub(G->Q, S)), G->n);
    G->inv_f1 = 2.0 / (B->a * cth);
    G->inv_f2 = 2.0 * cth / B->a;
    G->rho_g = B->a;
    return 1;
}

/* Vertical cylinder: 2-D reflection in the horizontal projection, height linear
 * in the unfolded horizontal length; valid iff projected-lit and the point is
 * on the lateral surface (cz <= z <= cz + h).  Curved-surface reflection
 * caustics with principal radii (a, inf): 1/f1 = 2 sin^2(theta_2)/(a cos),
 * 1/f2 = 0, theta_2 the angle between the incident ray and the axis. */
static int cylinder_reflection(const body *B, v3 S, v3 P, refl_geom *G) {
    body_frame F;
    if (!cylinder_frame(B, S, P, &F)) return 0;
    if (!(F.gam - F.bs - F.bp < 0.0)) return 0;
    double a = B->a;
    double psi = refl_psi(a, F.ds, F.pu, F.pv, F.gam);
    double qx = a * cos(psi), qy = a * sin(psi);
    double l1 = sqrt((qx - F.ds) * (qx - F.ds) + qy * qy);
    double l2 = sqrt((qx - F.pu) * (qx - F.pu) + (qy - F.pv) * (qy - F.pv));
    double zq = S.z + (P.z - S.z) * l1 / (l1 + l2);
    if (!(zq >= B->c.z && zq <= B->c.z + B->h)) return 0;
    G->n = add(scl(F.u, cos(psi)), scl(F.v, sin(psi)));
    G->Q = V(B->c.x + a * G->n.x, B->c.y + a * G->n.y, zq);
    v3 shi = unit(sub(G->Q, S));
    double cth = -dot(shi, G->n);
    G->inv_f1 = 2.0 * (1.0 - shi.z * shi.z) / (a * cth);
    G->inv_f2 = 0.0;
    v3 phi_hat = V(-G->n.y, G->n.x, 0.0);
    double sphi = dot(shi, phi_hat);
    G->rho_g = (sphi == 0.0) ? INFINITY : a * (1.0 - cth * cth) / (sphi * sphi);
    return 1;
}

/* Sphere creeping ray, dir 0 = short way (+), 1 = long way (-).  Great-circle
 * geodesic in the (S, c, P) plane; t = a (angle travelled); exists iff t > 0.
 * Divergence x spreading = sqrt(d_perp(Q1)/d_perp(P)) / sqrt(s), d_perp the
 * distance from the S-c axis; the long-way ray crosses that axis once. */
/* turns: extra full encirclements (the ray of the first one with its arc
 * lengthened by 2 pi a turns; it exists where the first one does). */
static int sphere_creeping(const body *B, v3 S, v3 P, int dir, int turns, creep_geom *G) {
    body_frame F;
    sphere_frame(B, S, P, &F);
    double a = B->a;
    double dpsi = (dir == 0) ? (F.gam - F.bs - F.bp) : (TWO_PI - F.gam - F.bs - F.bp);
    if (!(dpsi > 0.0)) return 0;
    dpsi += TWO_PI * turns;
    G->turns = turns;
    double psi1 = (dir == 0) ? F.bs : -F.bs;
    double psi2 = (dir == 0) ? F.gam - F.bp : F.gam + F.bp;
    G->n1 = add(scl(F.u, cos(psi1)), scl(F.v, sin(psi1)));
    G->n2 = add(scl(F.u, cos(psi2)), scl(F.v, sin(psi2)));
    G->Q1 = add(B->c, scl(G->n1, a));
    G->Q2 = add(B->c, scl(G->n2, a));
    G->sp = sqrt(F.ds * F.ds - a * a);
    G->sq = sqrt(F.dp * F.dp - a * a);
    G->t = a * dpsi;
    G->rho_g = a;
    G->dperp_P = F.dp * sin(F.gam);
    G->caustic_j = (dir == 1);
    double dperp_Q1 = a * sin(F.bs);
    G->amp = (G->dperp_P > 0.0) ? sqrt(dperp_Q1 / G->dperp_P) / sqrt(G->sq) / G->sp : 0.0;
    return 1;
}

/* Vertical finite cylinder creeping ray: helix; unrolled, the path is a straight
 * line of horizontal length H = d_s + a dphi + d_p and rise dz.  Valid iff
 * dphi > 0 and both Q1, Q2 lie within cz <= z <= cz + h.
 * Amplitude (1/s') sqrt(s'/(s'+t)) sqrt((s'+t)/(s (s'+t+s))) = 1/sqrt(s' s (s'+t+s)). */
static int cylinder_creeping(const body *B, v3 S, v3 P, int dir, int turns, creep_geom *G) {
    body_frame F;
    if (!cylinder_frame(B, S, P, &F)) return 0;
    double a = B->a;
    double dphi = (dir == 0) ? (F.gam - F.bs - F.bp) : (TWO_PI - F.gam - F.bs - F.bp);
    if (!(dphi > 0.0)) return 0;
    dphi += TWO_PI * turns;
    G->turns = turns;
    double ds_ = sqrt(F.ds * F.ds - a * a), dp_ = sqrt(F.dp * F.dp - a * a);
    double dz = P.z - S.z;
    double H = ds_ + a * dphi + dp_;
    double ell = sqrt(H * H + dz * dz);
    double sin0 = H / ell;
    double z1 = S.z + dz * ds_ / H, z2 = S.z + dz * (ds_ + a * dphi) / H;
    if (!(z1 >= B->c.z && z1 <= B->c.z + B->h && z2 >= B->c.z && z2 <= B->c.z + B->h)) return 0;
    double psi1 = (dir == 0) ? F.bs : -F.bs;
    double psi2 = (dir == 0) ? F.gam - F.bp : F.gam + F.bp;
    G->n1 = add(scl(F.u, cos(psi1)), scl(F.v, sin(psi1)));
    G->n2 = add(scl(F.u, cos(psi2)), scl(F.v, sin(psi2)));
    G->Q1 = V(B->c.x + a * G->n1.x, B->c.y + a * G->n1.y, z1);
    G->Q2 = V(B->c.x + a * G->n2.x, B->c.y + a * G->n2.y, z2);
    G->sp = ds_ / sin0; G->t = a * dphi / sin0; G->sq = dp_ / sin0;
    G->rho_g = a / (sin0 * sin0);
    G->caustic_j = 0;
    G->dperp_P = 0.0;
    G->amp = 1.0 / sqrt(G->sp * G->sq * (G->sp + G->t + G->sq));
    return 1;
}

/* Curved-body GO reflection field (Eq. 3) with the Fock-uniform reflection
 * coefficients R_s = R_perp, R_h = R_par:
 *   R = -sqrt(-4/xi) e^{-j xi^3/12} [P(xi) + (c/xi)(1 - F(X))],
 *   xi = -2 m cos(theta_i), m = (k rho_g/2)^{1/3}, X = 2 k L cos^2, L = s^i s^r/(s^i+s^r);
 * GO values -1 / +1 below XI_LO. */
static void add_body_reflection(const scene *s, const refl_geom *G, v3 P, rx_state *st) {
    v3 S = s->tx;
    v3 di = sub(G->Q, S), dr = sub(P, G->Q);
    double si = norm(di), sr = norm(dr);
    v3 shi = scl(di, 1.0 / si), shr = scl(dr, 1.0 / sr);
    double cth = -dot(shi, G->n);
    v3 eperp = cross(G->n, shi);
    double ne = norm(eperp);
    if (ne == 0.0) {                           /* normal incidence: any transverse direction */
        v3 tmp = fabs(G->n.x) < 0.9 ? V(1, 0, 0) : V(0, 1, 0);
        eperp = unit(cross(G->n, tmp));
    } else eperp = scl(eperp, 1.0 / ne);
    v3 epar_i = cross(eperp, shi), epar_r = cross(eperp, shr);
    v3 e0 = source_pol(s, shi);
    double Es = dot(e0, eperp), Eh = dot(e0, epar_i);
    double rho1 = 1.0 / (1.0 / si + G->inv_f1), rho2 = 1.0 / (1.0 / si + G->inv_f2);
    double A = sqrt(rho1 * rho2 / ((rho1 + sr) * (rho2 + sr)));
    double L = si * sr / (si + sr);
    for (int f = 0; f < s->n_f; ++f) {
        double k = kwave(s->freq[f]);
        double m = cbrt(k * G->rho_g / 2.0);
        double xi = -2.0 * m * cth;
        cplx Rs, Rh;
        if (xi < s->fock->xi_lo) { Rs = -1.0; Rh = 1.0; }
        else {
            cplx Bs, Bh;
            fock_bracket(s->fock, xi, sqrt(k * L / (2.0 * m * m)), &Bs, &Bh);
            st->ct.fock_evals++;
            cplx pre = -sqrt(-4.0 / xi) * cexp(-I * xi * xi * xi / 12.0);
            Rs = pre * Bs; Rh = pre * Bh;
        }
        cplx ph = A * cexp(-I * k * (si + sr)) / si;
        c3 Er = c3_add(rscl(eperp, Rs * Es * ph), rscl(epar_r, Rh * Eh * ph));
        accum(st, f, Er);
    }
}

/* Creeping field (Eq. 4):
 *   E^d = E^i(Q1) . [b1 b2 T_s + n1 n2 T_h] sqrt(deta1/deta2) sqrt(rho_d/(s(rho_d+s))) e^{-jks}
 *   T_{s,h} = -sqrt(m1 m2) sqrt(2/k) [P_{s,h}(xi) + (c/xi)(1 - F(X))] e^{-jkt},
 *   xi = m t / rho_g, X = k L xi^2/(2 m1 m2), L = s' s/(s'+s). */
static void add_creeping_from(const scene *s, const creep_geom *G, v3 S, c3 e0, v3 P, rx_state *st) {
    v3 t1 = unit(sub(G->Q1, S)), t2 = unit(sub(P, G->Q2));
    v3 b1 = cross(t1, G->n1), b2 = cross(t2, G->n2);
    cplx Es = c3_dotr(e0, b1), Eh = c3_dotr(e0, G->n1);
    double L = G->sp * G->sq / (G->sp + G->sq);
    cplx caus = G->caustic_j ? I : 1.0;
    /* a sphere's ray crosses the source axis twice per extra encirclement:
     * +j per crossing, -1 per turn */
    int sphere_turns = (G->dperp_P > 0.0) ? G->turns : 0;
    if (sphere_turns & 1) caus = -caus;
    for (int f = 0; f < s->n_f; ++f) {
        double k = kwave(s->freq[f]);
        double m = cbrt(k * G->rho_g / 2.0);
        double xi = m * G->t / G->rho_g;
        cplx Bs, Bh;
        fock_bracket(s->fock, xi, sqrt(k * L / (2.0 * m * m)), &Bs, &Bh);
        st->ct.fock_evals++;
        cplx Tpre = -m * sqrt(2.0 / k) * cexp(-I * k * G->t);
        cplx Ts = (s->enable & EN_CREEP_SOFT) ? Tpre * Bs : 0.0;
        cplx Th = (s->enable & EN_CREEP_HARD) ? Tpre * Bh : 0.0;
        cplx ph = caus * G->amp * cexp(-I * k * (G->sp + G->sq));
        c3 Ed = c3_add(rscl(b2, Ts * Es * ph), rscl(G->n2, Th * Eh * ph));
        accum(st, f, Ed);
    }
}
/* the creeping ray of the source itself: its polarisation along t1 */
static void add_creeping(const scene *s, const creep_geom *G, v3 P, rx_state *st) {
    v3 e0 = source_pol(s, unit(sub(G->Q1, s->tx)));
    add_creeping_from(s, G, s->tx, CV(e0.x, e0.y, e0.z), P, st);
}

static void body_paths(const scene *s, int b, v3 P, rx_state *st) {
    const body *B = &s->bodies[b];
    v3 S = s->tx;
    if (s->enable & EN_BODYREFL) {
        refl_geom G;
        st->ct.body_refl++;
        int ok = (B->type == 0) ? sphere_reflection(B, S, P, &G) : cylinder_reflection(B, S, P, &G);
        if (ok && visible(s, S, G.Q, -1, -1, b, &st->ct) && visible(s, G.Q, P, -1, -1, b, &st->ct)) {
            add_path(st, pcode(PT_RB, b, 0));
            add_body_reflection(s, &G, P, st);
        }
    }
    if (!(s->enable & (EN_CREEP_SOFT | EN_CREEP_HARD))) return;
    for (int turns = 0; turns <= s->max_enc; ++turns)
    for (int dir = 0; dir < 2; ++dir) {
        creep_geom G;
        st->ct.creep_geom++;
        int ok = (B->type == 0) ? sphere_creeping(B, S, P, dir, turns, &G)
                                : cylinder_creeping(B, S, P, dir, turns, &G);
        if (!ok) continue;
        if (!visible(s, S, G.Q1, -1, -1, b, &st->ct)) continue;
        if (!visible(s, G.Q2, P, -1, -1, b, &st->ct)) continue;
        add_path(st, pcode(dir == 0 ? PT_CP : PT_CM, b, turns));
        if (B->type == 0) {
            /* axial caustic of the sphere's creeping rays: flag k d_perp < pi */
            for (int f = 0; f < s->n_f; ++f)
                if (kwave(s->freq[f]) * G.dperp_P < M_PI) st->flags |= FL_CAUSTIC;
            if (!(G.dperp_P > 0.0)) continue;   /* exactly on the axis: no finite ray field */
        }
        add_creeping(s, &G, P, st);
    }
}

/* Wall -> creeping paths: S -> Qw (face f) -> Q1 -> surface ray -> Q2 -> P.
 * By the image method the reflected wave is the wave of the source's mirror
 * image Sf in the plane of face f, so the creeping ray is the one of Sf
 * (same geometry, spreading and length |Sf - Q1| = |S - Qw| + |Qw - Q1|)
 * with, at Q1, the source's polarisation reflected at Qw (reflect_at).
 * Valid iff Sf lies outside the body (a cylinder: its axis distance > a),
 * Q1 lies strictly on the source's side of the plane, Qw (where Sf -> Q1
 * crosses the plane) lies in face f, S -> Qw is visible (face f's triangles
 * not tested), Qw -> Q1 is visible (face f and body b not tested), and
 * Q2 -> P is visible (body b not tested).  Listed as (WCP or WCM, b,
 * 16 f + turns). */
static void wall_creep_paths(const scene *s, int b, v3 P, rx_state *st) {
    const body *B = &s->bodies[b];
    v3 S = s->tx;
    for (int f = 0; f < s->n_face; ++f) {
        const face *F = &s->faces[f];
        double dS = dot(F->n, S) - F->d;
        v3 Sf = mirror_point(S, F);
        v3 w = sub(Sf, B->c);
        if (B->type != 0) w.z = 0.0;
        if (!(norm(w) > B->a)) continue;
        for (int turns = 0; turns <= s->max_enc; ++turns)
        for (int dir = 0; dir < 2; ++dir) {
            creep_geom G;
            st->ct.creep_geom++;
            int ok = (B->type == 0) ? sphere_creeping(B, Sf, P, dir, turns, &G)
                                    : cylinder_creeping(B, Sf, P, dir, turns, &G);
            if (!ok) continue;
            double dQ = dot(F->n, G.Q1) - F->d;
            if (!(dS * dQ > 0.0)) continue;
            double dI = dot(F->n, Sf) - F->d;
            v3 Qw = add(Sf, scl(sub(G.Q1, Sf), dI / (dI - dQ)));
            if (!point_in_face(s, f, Qw, &st->ct)) continue;
            if (!visible(s, S, Qw, f, -1, -1, &st->ct)) continue;
            if (!visible(s, Qw, G.Q1, f, -1, b, &st->ct)) continue;
            if (!visible(s, G.Q2, P, -1, -1, b, &st->ct)) continue;
            add_path(st, pcode(dir == 0 ? PT_WCP : PT_WCM, b, 16 * f + turns));
            if (B->type == 0) {
                for (int k = 0; k < s->n_f; ++k)
                    if (kwave(s->freq[k]) * G.dperp_P < M_PI) st->flags |= FL_CAUSTIC;
                if (!(G.dperp_P > 0.0)) continue;
            }
            v3 si = unit(sub(Qw, S)), sr = unit(sub(G.Q1, Qw));
            v3 e0 = source_pol(s, si);
            c3 Er = reflect_at(F, CV(e0.x, e0.y, e0.z), si, sr);
            add_creeping_from(s, &G, Sf, Er, P, st);
        }
    }
}

/* ------------------------------------------------------------ entry points */

/* Build faces (planes) from the triangle->face map.  Face plane from the first
 * triangle of the face (unit normal of (v1-v0)x(v2-v0)). */
static int build_faces(scene *s) {
    int nf = 0;
    for (int t = 0; t < s->n_tri; ++t) if (s->tri_face[t] + 1 > nf) nf = s->tri_face[t] + 1;
    s->n_face = nf;
    s->faces = (face *)calloc(nf > 0 ? nf : 1, sizeof(face));
    s->order = (int *)malloc(sizeof(int) * (s->n_tri > 0 ? s->n_tri : 1));
    int *cnt = (int *)calloc(nf > 0 ? nf : 1, sizeof(int));
    for (int t = 0; t < s->n_tri; ++t) cnt[s->tri_face[t]]++;
    int acc = 0;
    for (int f = 0; f < nf; ++f) { s->faces[f].first = acc; s->faces[f].count = 0; acc += cnt[f]; }
    for (int t = 0; t < s->n_tri; ++t) {
        face *F = &s->faces[s->tri_face[t]];
        if (F->count == 0) {
            v3 n = unit(cross(sub(tri_v(s, t, 1), tri_v(s, t, 0)), sub(tri_v(s, t, 2), tri_v(s, t, 0))));
            F->n = n;
            F->d = dot(n, tri_v(s, t, 0));
        }
        s->order[F->first + F->count++] = t;
    }
    free(cnt);
    return 0;
}

/*
 * Evaluate the field at n_rx receivers.
 *   tri [n_tri][3][3], tri_face [n_tri] (face id per triangle; coplanar groups)
 *   bodies [n_body][6] = (type, cx, cy, cz, a, h)
 *   tx[3], pol[3], freq [n_f] (Hz)
 *   rx [n_rx][3]
 *   E_out [n_f][3][n_rx][2] (re, im), path_codes [n_rx][cap], path_count [n_rx],
 *   flags [n_rx], counters_out[8] (summed), sabs_out [n_f][n_rx] (sum of |E_path|, or NULL)
 * Returns 0.
 */
int oracle_eval(const double *tri, const int *tri_face, int n_tri,
                const double *bodies, int n_body,
                const double *tx, const double *pol,
                const double *freq, int n_f,
                const double *rx, int n_rx,
                const double *tau_re, const double *tau_im,
                const double *ws_re, const double *ws_im,
                const double *wh_re, const double *wh_im,
                const int *offsets, int n_buckets,
                const double *res_alpha, const double *res_cs,
                const double *res_beta, const double *res_ch, int n_res,
                double xi_lo, double xi_hi,
                int max_order, int enable,
                double *E_out, uint64_t *path_codes, int *path_count, int cap,
                unsigned *flags_out, long long *counters_out, int n_threads, double *sabs_out,
                double *path_E_out, const double *face_eps, int max_enc, const int *cand, int n_cand) {
    fock_rule R = {tau_re, tau_im, ws_re, ws_im, wh_re, wh_im, offsets, n_buckets,
                   res_alpha, res_cs, res_beta, res_ch, n_res, xi_lo, xi_hi};
    scene s;
    memset(&s, 0, sizeof(s));
    s.n_tri = n_tri; s.tri = tri; s.tri_face = tri_face;
    build_faces(&s);
    /* face materials: [n_face][3] = (dielectric flag, eps', eps'') or NULL (all PEC) */
    for (int f = 0; f < s.n_face; ++f) {
        s.faces[f].dielectric = face_eps ? face_eps[3 * f] != 0.0 : 0;
        s.faces[f].eps = face_eps ? face_eps[3 * f + 1] - I * face_eps[3 * f + 2] : 0.0;
    }
    s.n_body = n_body;
    s.bodies = (body *)malloc(sizeof(body) * (n_body > 0 ? n_body : 1));
    for (int b = 0; b < n_body; ++b) {
        const double *q = bodies + 6 * b;
        s.bodies[b].type = (int)q[0];
        s.bodies[b].c = V(q[1], q[2], q[3]);
        s.bodies[b].a = q[4];
        s.bodies[b].h = q[5];
    }
    s.tx = V(tx[0], tx[1], tx[2]);
    s.pol = V(pol[0], pol[1], pol[2]);
    s.n_f = n_f; s.freq = freq; s.fock = &R;
    s.max_order = max_order; s.enable = enable;
    s.max_enc = max_enc;
    s.cand = cand; s.n_cand = cand ? n_cand : 0;
    counters tot;
    memset(&tot, 0, sizeof(tot));
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    long long c0 = 0, c1 = 0, c2 = 0, c3v = 0, c4 = 0, c5 = 0, c6 = 0, c7 = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : c0, c1, c2, c3v, c4, c5, c6, c7)
    for (int r = 0; r < n_rx; ++r) {
        c3 Eacc[64];
        double Sacc[64];
        c3 *E = (n_f <= 64) ? Eacc : (c3 *)malloc(sizeof(c3) * n_f);
        double *Sa = (n_f <= 64) ? Sacc : (double *)malloc(sizeof(double) * n_f);
        for (int f = 0; f < n_f; ++f) { E[f] = CV(0, 0, 0); Sa[f] = 0.0; }
        rx_state st;
        memset(&st, 0, sizeof(st));
        st.E = E;
        st.Sabs = Sa;
        st.paths = path_codes ? path_codes + (size_t)r * cap : NULL;
        st.cap = path_codes ? cap : 0;
        st.n_f = n_f;
        st.pathE = (path_codes && path_E_out) ? path_E_out + (size_t)r * cap * n_f * 6 : NULL;
        v3 P = V(rx[3 * r], rx[3 * r + 1], rx[3 * r + 2]);
        int inside = 0;
        for (int b = 0; b < n_body; ++b) if (inside_body(P, &s.bodies[b])) inside = 1;
        if (inside) {
            st.flags |= FL_INSIDE;
        } else {
            planar_paths(&s, P, &st);
            for (int b = 0; b < n_body; ++b) body_paths(&s, b, P, &st);
            if (s.enable & EN_WALL_CREEP)
                for (int b = 0; b < n_body; ++b) wall_creep_paths(&s, b, P, &st);
        }
        for (int f = 0; f < n_f; ++f) {
            size_t base = ((size_t)f * 3) * n_rx + r;
            E_out[2 * (base)] = creal(E[f].x);            E_out[2 * (base) + 1] = cimag(E[f].x);
            E_out[2 * (base + n_rx)] = creal(E[f].y);     E_out[2 * (base + n_rx) + 1] = cimag(E[f].y);
            E_out[2 * (base + 2 * (size_t)n_rx)] = creal(E[f].z);
            E_out[2 * (base + 2 * (size_t)n_rx) + 1] = cimag(E[f].z);
        }
        if (path_count) path_count[r] = st.n_paths;
        if (flags_out) flags_out[r] = st.flags;
        c0 += st.ct.seg_tri; c1 += st.ct.seg_body; c2 += st.ct.inside_tri; c3v += st.ct.image_cand;
        c4 += st.ct.body_refl; c5 += st.ct.creep_geom; c6 += st.ct.paths; c7 += st.ct.fock_evals;
        if (sabs_out)
            for (int f = 0; f < n_f; ++f) sabs_out[(size_t)f * n_rx + r] = Sa[f];
        if (E != Eacc) free(E);
        if (Sa != Sacc) free(Sa);
    }
    if (counters_out) {
        counters_out[0] = c0; counters_out[1] = c1; counters_out[2] = c2; counters_out[3] = c3v;
        counters_out[4] = c4; counters_out[5] = c5; counters_out[6] = c6; counters_out[7] = c7;
    }
    free(s.faces); free(s.order); free(s.bodies);
    return 0;
}

/* ------------------------------------------------------------ candidates */
/* Ray hit with the closed triangle (v0, v1, v2) (Moller-Trumbore); returns
 * the ray parameter or -1. */
static double ray_tri(v3 o, v3 d, v3 v0, v3 v1, v3 v2) {
    v3 e1 = sub(v1, v0), e2 = sub(v2, v0);
    v3 p = cross(d, e2);
    double det = dot(e1, p);
    if (fabs(det) < 1e-14) return -1.0;
    double inv = 1.0 / det;
    v3 sv = sub(o, v0);
    double u = dot(sv, p) * inv;
    if (u < 0.0 || u > 1.0) return -1.0;
    v3 q = cross(sv, e1);
    double v = dot(d, q) * inv;
    if (v < 0.0 || u + v > 1.0) return -1.0;
    return dot(e2, q) * inv;
}

static int seq_cmp(const void *pa, const void *pb) {
    const int *x = (const int *)pa, *y = (const int *)pb;
    int kx = (x[0] >= 0) + (x[1] >= 0) + (x[2] >= 0), ky = (y[0] >= 0) + (y[1] >= 0) + (y[2] >= 0);
    if (kx != ky) return kx < ky ? -1 : 1;
    for (int m = 0; m < 3; ++m)
        if (x[m] != y[m]) return x[m] < y[m] ? -1 : 1;
    return 0;
}

/* Candidate face sequences of the large-scene mode, by a ray launch from the
 * transmitter: n_rays directions of the spherical Fibonacci lattice
 * (z_i = 1 - (2i + 1)/n, phi_i = i pi (3 - sqrt 5)), each ray reflected
 * specularly at the nearest triangle hit (parameter > 1e-9, the face it
 * leaves excluded; ties to the lower triangle index; bodies ignored) up to
 * max_order times; every prefix of its face sequence is a candidate.  The
 * distinct sequences, sorted (order, then faces), go to seq [cap][3] (-1
 * padded).  Returns their number (capped at cap). */
int oracle_candidates(const double *tri, const int *tri_face, int n_tri, const double *tx, int n_rays, int max_order,
                      int *seq, int cap) {
    scene s;
    memset(&s, 0, sizeof(s));
    s.n_tri = n_tri; s.tri = tri; s.tri_face = tri_face;
    build_faces(&s);
    /* ray i records its prefixes in slots i * max_order + k (unused slots
     * keep face -2 and are dropped), so the rays are independent */
    const int mo = max_order > 0 ? max_order : 1;
    const size_t n_slot = (size_t)(n_rays > 0 ? n_rays : 1) * mo;
    int *slot = (int *)malloc(sizeof(int) * 3 * n_slot);
    for (size_t q = 0; q < 3 * n_slot; ++q) slot[q] = -2;
    const double golden = M_PI * (3.0 - sqrt(5.0));
#pragma omp parallel for schedule(dynamic, 8)
    for (int i = 0; i < n_rays; ++i) {
        double z = 1.0 - (2.0 * i + 1.0) / n_rays;
        double r = sqrt(fmax(0.0, 1.0 - z * z));
        double ph = golden * i;
        v3 o = V(tx[0], tx[1], tx[2]), d = V(r * cos(ph), r * sin(ph), z);
        int fs[3] = {-1, -1, -1}, last = -1;
        for (int k = 0; k < max_order; ++k) {
            double best = INFINITY;
            int bt = -1;
            for (int t = 0; t < n_tri; ++t) {
                if (tri_face[t] == last) continue;
                double h = ray_tri(o, d, tri_v(&s, t, 0), tri_v(&s, t, 1), tri_v(&s, t, 2));
                if (h > 1e-9 && h < best) { best = h; bt = t; }
            }
            if (bt < 0) break;
            int f = tri_face[bt];
            fs[k] = f;
            int *q = slot + 3 * ((size_t)i * mo + k);
            for (int m = 0; m < 3; ++m) q[m] = (m <= k) ? fs[m] : -1;
            v3 n = s.faces[f].n;
            o = add(o, scl(d, best));
            d = sub(d, scl(n, 2.0 * dot(d, n)));
            last = f;
        }
    }
    int n_all = 0;
    int *all = (int *)malloc(sizeof(int) * 3 * n_slot);
    for (size_t q = 0; q < n_slot; ++q)
        if (slot[3 * q] != -2) { memcpy(all + 3 * n_all, slot + 3 * q, 3 * sizeof(int)); ++n_all; }
    free(slot);
    /* sort by (order, faces) and keep the distinct ones */
    qsort(all, (size_t)n_all, 3 * sizeof(int), seq_cmp);
    int n = 0;
    for (int a = 0; a < n_all; ++a) {
        if (a > 0 && !memcmp(all + 3 * a, all + 3 * (a - 1), 3 * sizeof(int))) continue;
        if (n < cap) memcpy(seq + 3 * n, all + 3 * a, 3 * sizeof(int));
        ++n;
    }
    free(all); free(s.faces); free(s.order);
    return n < cap ? n : cap;
}

/* Exposed for the oracle's own tests. */
void oracle_transition_F(const double *X, int n, double *out) {
    for (int i = 0; i < n; ++i) {
        cplx F = transition_F(X[i]);
        out[2 * i] = creal(F); out[2 * i + 1] = cimag(F);
    }
}

void oracle_fock_bracket(const double *tau_re, const double *tau_im,
                         const double *ws_re, const double *ws_im,
                         const double *wh_re, const double *wh_im,
                         const int *offsets, int n_buckets,
                         const double *res_alpha, const double *res_cs,
                         const double *res_beta, const double *res_ch, int n_res,
                         double xi_lo, double xi_hi,
                         const double *xi, const double *K, int n, double *out /* [n][4] */) {
    fock_rule R = {tau_re, tau_im, ws_re, ws_im, wh_re, wh_im, offsets, n_buckets,
                   res_alpha, res_cs, res_beta, res_ch, n_res, xi_lo, xi_hi};
    for (int i = 0; i < n; ++i) {
        cplx Bs, Bh;
        fock_bracket(&R, xi[i], K[i], &Bs, &Bh);
        out[4 * i] = creal(Bs); out[4 * i + 1] = cimag(Bs);
        out[4 * i + 2] = creal(Bh); out[4 * i + 3] = cimag(Bh);
    }
}

/* Geometry probes for the oracle's own tests (brute-force Fermat and ray-tube
 * checks).  body6 = (type, cx, cy, cz, a, h).
 * reflection: out = Q[3], n[3], inv_f1, inv_f2, rho_g; returns 1 if it exists.
 * creeping:   out = Q1[3], Q2[3], n1[3], n2[3], s', t, s, amp, rho_g, caustic_j, dperp_P. */
static body body_from(const double *q) {
    body B; B.type = (int)q[0]; B.c = V(q[1], q[2], q[3]); B.a = q[4]; B.h = q[5]; return B;
}
int oracle_body_reflection(const double *body6, const double *S, const double *P, double *out) {
    body B = body_from(body6);
    refl_geom G;
    v3 s_ = V(S[0], S[1], S[2]), p_ = V(P[0], P[1], P[2]);
    int ok = (B.type == 0) ? sphere_reflection(&B, s_, p_, &G) : cylinder_reflection(&B, s_, p_, &G);
    if (!ok) return 0;
    double v[9] = {G.Q.x, G.Q.y, G.Q.z, G.n.x, G.n.y, G.n.z, G.inv_f1, G.inv_f2, G.rho_g};
    memcpy(out, v, sizeof(v));
    return 1;
}
int oracle_body_creeping(const double *body6, const double *S, const double *P, int dir, int turns, double *out) {
    body B = body_from(body6);
    creep_geom G;
    v3 s_ = V(S[0], S[1], S[2]), p_ = V(P[0], P[1], P[2]);
    int ok = (B.type == 0) ? sphere_creeping(&B, s_, p_, dir, turns, &G) : cylinder_creeping(&B, s_, p_, dir, turns, &G);
    if (!ok) return 0;
    double v[19] = {G.Q1.x, G.Q1.y, G.Q1.z, G.Q2.x, G.Q2.y, G.Q2.z, G.n1.x, G.n1.y, G.n1.z,
                    G.n2.x, G.n2.y, G.n2.z, G.sp, G.t, G.sq, G.amp, G.rho_g, (double)G.caustic_j, G.dperp_P};
    memcpy(out, v, sizeof(v));
    return 1;
}
/* Segment visibility probe against one body (1 = obstructed). */
/* One reflection (reflect_at) of the complex field E[3] (re, im pairs) at a
 * face of unit normal n: dielectric != 0 with eps = eps_re - j eps_im. */
void oracle_reflect(const double *n, const double *si, const double *sr, const double *E, int dielectric,
                    double eps_re, double eps_im, double *out) {
    face F;
    memset(&F, 0, sizeof(F));
    F.n = V(n[0], n[1], n[2]);
    F.dielectric = dielectric;
    F.eps = eps_re - I * eps_im;
    c3 e = CV(E[0] + I * E[1], E[2] + I * E[3], E[4] + I * E[5]);
    c3 r = reflect_at(&F, e, V(si[0], si[1], si[2]), V(sr[0], sr[1], sr[2]));
    out[0] = creal(r.x); out[1] = cimag(r.x); out[2] = creal(r.y); out[3] = cimag(r.y);
    out[4] = creal(r.z); out[5] = cimag(r.z);
}

int oracle_seg_hits_body(const double *body6, const double *A, const double *Bp) {
    body B = body_from(body6);
    return seg_hits_body(V(A[0], A[1], A[2]), V(Bp[0], Bp[1], Bp[2]), &B);
}
