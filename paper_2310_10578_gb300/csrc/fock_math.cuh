// fock_math.cuh -- FP64 Airy functions and the Fock--Pekeris contour
// quadrature used to build the smooth-surface UTD table on the device.
//
// Functions (time convention e^{+j w t}), the soft/hard Fock--Pekeris
// integrals of the off-surface UTD that the paper uses for R and T
// (Sec. II.B, after Eq. 4):
//   P_s(xi) = e^{-j pi/4}/sqrt(pi) Int V(t)/W2(t)  e^{-j xi t} dt,
//   P_h(xi) = e^{-j pi/4}/sqrt(pi) Int V'(t)/W2'(t) e^{-j xi t} dt,
// V = sqrt(pi) Ai, W_{1,2} = sqrt(pi) (Bi +- j Ai).  Their regular parts
// phat = P + c/xi (c = e^{-j pi/4}/(2 sqrt(pi))) come from
//   phat = e^{-j pi/4}/sqrt(pi) [ Int_{-inf}^0 W1/(2j W2) e^{-j xi t} dt
//                                 + Int_0^inf V/W2 e^{-j xi t} dt ]
// (primes throughout for the hard case), with the negative half written in
// x = -t and deformed into the upper half x-plane where the integrand decays.
// W1, W2 are evaluated through Ai at rotated arguments:
//   W2(z) = 2 sqrt(pi) e^{-j pi/6} Ai(z e^{-2 pi j/3}),
//   W1(z) = 2 sqrt(pi) e^{+j pi/6} Ai(z e^{+2 pi j/3}).
//
// Ai(z) for complex z: Maclaurin series for |z| <= 4; the asymptotic
// expansion in zeta = (2/3) z^{3/2} for |z| >= 8 (|arg z| < pi); in between,
// Taylor steps of the Airy equation w'' = z w, integrated inward from |z| = 8
// where Ai decays outward (|arg z| < pi/3) and outward from |z| = 4
// elsewhere, the stable direction in each sector.
#pragma once
#include <math.h>

namespace creep {

struct cd {
    double x, y;
};

__host__ __device__ inline cd C(double x, double y = 0.0) { cd r; r.x = x; r.y = y; return r; }
__host__ __device__ inline cd operator+(cd a, cd b) { return C(a.x + b.x, a.y + b.y); }
__host__ __device__ inline cd operator-(cd a, cd b) { return C(a.x - b.x, a.y - b.y); }
__host__ __device__ inline cd operator-(cd a) { return C(-a.x, -a.y); }
__host__ __device__ inline cd operator*(cd a, cd b) { return C(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ inline cd operator*(cd a, double s) { return C(a.x * s, a.y * s); }
__host__ __device__ inline cd operator*(double s, cd a) { return C(a.x * s, a.y * s); }
__host__ __device__ inline cd operator/(cd a, cd b) {
    // scaled division (Smith)
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, d = b.x + b.y * r;
        return C((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    }
    double r = b.x / b.y, d = b.x * r + b.y;
    return C((a.x * r + a.y) / d, (a.y * r - a.x) / d);
}
__host__ __device__ inline cd operator/(cd a, double s) { return C(a.x / s, a.y / s); }
__host__ __device__ inline double cabs_(cd a) { return hypot(a.x, a.y); }
__host__ __device__ inline double carg_(cd a) { return atan2(a.y, a.x); }
__host__ __device__ inline cd cexp_(cd a) {
    double e = exp(a.x);
    return C(e * cos(a.y), e * sin(a.y));
}
__host__ __device__ inline cd cpolar(double r, double th) { return C(r * cos(th), r * sin(th)); }
// principal square root
__host__ __device__ inline cd csqrt_(cd a) {
    double r = cabs_(a);
    if (r == 0.0) return C(0.0, 0.0);
    double t = sqrt(0.5 * (r + fabs(a.x)));
    if (a.x >= 0.0) return C(t, a.y / (2.0 * t));
    return C(fabs(a.y) / (2.0 * t), (a.y >= 0.0) ? t : -t);
}

// Airy value and derivative, scaled: Ai(z) = ai * e^{-zeta}, Ai'(z) = aip * e^{-zeta}
struct airy_t {
    cd ai, aip, zeta;
};

// Ai(0) = 1/(3^{2/3} Gamma(2/3)), Ai'(0) = -1/(3^{1/3} Gamma(1/3))
__host__ __device__ inline double ai0() { return 1.0 / (pow(3.0, 2.0 / 3.0) * tgamma(2.0 / 3.0)); }
__host__ __device__ inline double aip0() { return -1.0 / (pow(3.0, 1.0 / 3.0) * tgamma(1.0 / 3.0)); }

// Maclaurin series: Ai = Ai(0) f + Ai'(0) g,  f = sum a_k z^{3k}, g = sum b_k z^{3k+1},
// a_k = a_{k-1}/((3k-1) 3k), b_k = b_{k-1}/(3k (3k+1)).
__host__ __device__ inline void airy_series(cd z, cd *ai, cd *aip) {
    if (z.x == 0.0 && z.y == 0.0) { *ai = C(ai0()); *aip = C(aip0()); return; }
    cd z2 = z * z, z3 = z2 * z;
    cd f = C(1.0), fp = C(0.0), g = z, gp = C(1.0);
    cd tf = C(1.0), tg = z;        // current terms a_k z^{3k}, b_k z^{3k+1}
    for (int k = 1; k < 80; ++k) {
        tf = tf * z3 / (double)((3 * k - 1) * (3 * k));
        tg = tg * z3 / (double)((3 * k) * (3 * k + 1));
        f = f + tf;
        g = g + tg;
        // derivatives: d/dz z^{3k} = 3k z^{3k-1}: term*3k/z ; d/dz z^{3k+1} = (3k+1) z^{3k}
        fp = fp + tf * (3.0 * k) / z;
        gp = gp + tg * (3.0 * k + 1.0) / z;
        if (cabs_(tf) < 1e-18 * cabs_(f) && cabs_(tg) < 1e-18 * cabs_(g) && k > 3) break;
    }
    double c1 = ai0(), c2 = aip0();
    *ai = c1 * f + c2 * g;
    *aip = c1 * fp + c2 * gp;
}

// Asymptotic expansion for large |z|, |arg z| < pi (A&S 10.4.59, 10.4.61):
//   Ai  ~ e^{-zeta} / (2 sqrt(pi) z^{1/4}) sum (-1)^k u_k zeta^{-k}
//   Ai' ~ -z^{1/4} e^{-zeta} / (2 sqrt(pi)) sum (-1)^k v_k zeta^{-k}
//   u_k = (6k-5)(6k-3)(6k-1) / ((2k-1) 216 k) u_{k-1}, v_k = -(6k+1)/(6k-1) u_k
__host__ __device__ inline airy_t airy_asym(cd z) {
    cd sz = csqrt_(z);
    cd z14 = csqrt_(sz);
    cd zeta = (2.0 / 3.0) * (z * sz);
    cd iz = C(1.0) / zeta;
    cd su = C(1.0), sv = C(1.0), pw = C(1.0);
    double u = 1.0, last = 1e300;
    for (int k = 1; k < 60; ++k) {
        u *= (double)((6 * k - 5) * (6 * k - 3) * (6 * k - 1)) / ((double)(2 * k - 1) * 216.0 * k);
        double v = -(6.0 * k + 1.0) / (6.0 * k - 1.0) * u;
        pw = pw * (-1.0) * iz;
        cd tu = u * pw, tv = v * pw;
        double mag = cabs_(tu);
        if (mag > last) break;            // asymptotic series: stop at the smallest term
        su = su + tu;
        sv = sv + tv;
        last = mag;
        if (mag < 1e-18) break;
    }
    double inv2sp = 0.5 / sqrt(M_PI);
    airy_t r;
    r.ai = su * inv2sp / z14;
    r.aip = -(sv * inv2sp) * z14;
    r.zeta = zeta;
    return r;
}

// Taylor step of w'' = z w from z0 to z0 + h
__host__ __device__ inline void airy_step(cd z0, cd h, cd *w, cd *wp) {
    cd c_prev = *w, c_cur = *wp;           // c0, c1
    cd c2 = z0 * c_prev / 2.0;
    // accumulate sum c_n h^n and sum n c_n h^{n-1}
    cd hn = h, val = c_prev + c_cur * h, der = c_cur;
    cd cm1 = c_prev, cm0 = c_cur, cn = c2;  // c_{n-2}, c_{n-1}, c_n for n = 2
    cd hnm1 = h;                            // h^{n-1}
    for (int n = 2; n < 60; ++n) {
        hn = hn * h;                        // h^n
        cd t = cn * hn;
        val = val + t;
        der = der + (double)n * cn * hnm1;
        hnm1 = hnm1 * h;
        // c_{n+1} = (z0 c_{n-1} + c_{n-2}) / ((n+1) n)
        cd cnext = (z0 * cm0 + cm1) / (double)((n + 1) * n);
        cm1 = cm0; cm0 = cn; cn = cnext;
        if (cabs_(t) < 1e-19 * cabs_(val) && n > 8) break;
    }
    (void)c2;
    *w = val;
    *wp = der;
}

__host__ __device__ inline void airy_integrate(cd z0, cd z1, cd *w, cd *wp) {
    double len = cabs_(z1 - z0);
    int ns = (int)ceil(len / 0.4);
    if (ns < 1) ns = 1;
    cd h = (z1 - z0) / (double)ns;
    cd z = z0;
    for (int i = 0; i < ns; ++i) {
        airy_step(z, h, w, wp);
        z = z + h;
    }
}

__host__ __device__ inline airy_t airy(cd z) {
    double r = cabs_(z);
    airy_t out;
    if (r >= 8.0) return airy_asym(z);
    out.zeta = C(0.0);
    if (r <= 4.0) {
        airy_series(z, &out.ai, &out.aip);
        return out;
    }
    double th = carg_(z);
    if (fabs(th) < M_PI / 3.0) {
        // recessive outward: start on |z| = 8 and integrate inward
        cd z8 = cpolar(8.0, th);
        airy_t a8 = airy_asym(z8);
        cd s = cexp_(-a8.zeta);
        cd w = a8.ai * s, wp = a8.aip * s;
        airy_integrate(z8, z, &w, &wp);
        out.ai = w; out.aip = wp;
    } else {
        cd z4 = cpolar(4.0, th);
        cd w, wp;
        airy_series(z4, &w, &wp);
        airy_integrate(z4, z, &w, &wp);
        out.ai = w; out.aip = wp;
    }
    return out;
}

// ratio Ai^(d)(z1) / Ai^(d)(z2) from scaled values
__host__ __device__ inline cd airy_ratio(const airy_t &a1, const airy_t &a2, bool deriv) {
    cd n = deriv ? a1.aip : a1.ai;
    cd d = deriv ? a2.aip : a2.ai;
    return (n / d) * cexp_(a2.zeta - a1.zeta);
}

// Integrands at tau.  pos: V/W2 and V'/W2' (used on tau >= 0);
// neg: W1/(2j W2) and W1'/(2j W2') (used on the deformed tau <= 0 branch).
__host__ __device__ inline void fock_integrands(cd tau, bool pos, cd *gs, cd *gh) {
    const cd wm = cpolar(1.0, -2.0 * M_PI / 3.0);   // e^{-2 pi j/3}
    const cd wp_ = cpolar(1.0, 2.0 * M_PI / 3.0);   // e^{+2 pi j/3}
    airy_t am = airy(tau * wm);
    if (pos) {
        airy_t a0 = airy(tau);
        // V/W2 = e^{j pi/6}/2 Ai(tau)/Ai(tau w^-1);  V'/W2' = e^{j 5pi/6}/2 Ai'(tau)/Ai'(tau w^-1)
        *gs = cpolar(0.5, M_PI / 6.0) * airy_ratio(a0, am, false);
        *gh = cpolar(0.5, 5.0 * M_PI / 6.0) * airy_ratio(a0, am, true);
    } else {
        airy_t ap = airy(tau * wp_);
        // W1/W2 = e^{j pi/3} Ai(tau w)/Ai(tau w^-1); W1'/W2' = e^{-j pi/3} Ai'(tau w)/Ai'(tau w^-1)
        cd inv2j = C(0.0, -0.5);
        *gs = inv2j * cpolar(1.0, M_PI / 3.0) * airy_ratio(ap, am, false);
        *gh = inv2j * cpolar(1.0, -M_PI / 3.0) * airy_ratio(ap, am, true);
    }
}

}  // namespace creep
