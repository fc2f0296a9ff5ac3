// devmath.cuh -- small vector, complex and double-float helpers for the field kernel.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace creep {

template <typename T>
struct v3t {
    T x, y, z;
};

template <typename T>
__device__ __forceinline__ v3t<T> mk3(T x, T y, T z) {
    v3t<T> r;
    r.x = x; r.y = y; r.z = z;
    return r;
}
template <typename T>
__device__ __forceinline__ v3t<T> operator+(v3t<T> a, v3t<T> b) { return mk3<T>(a.x + b.x, a.y + b.y, a.z + b.z); }
template <typename T>
__device__ __forceinline__ v3t<T> operator-(v3t<T> a, v3t<T> b) { return mk3<T>(a.x - b.x, a.y - b.y, a.z - b.z); }
template <typename T>
__device__ __forceinline__ v3t<T> operator*(v3t<T> a, T s) { return mk3<T>(a.x * s, a.y * s, a.z * s); }
template <typename T>
__device__ __forceinline__ T dot3(v3t<T> a, v3t<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename T>
__device__ __forceinline__ v3t<T> cross3(v3t<T> a, v3t<T> b) {
    return mk3<T>(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// IEEE double whose arithmetic the compiler may not contract (no fused
// multiply-add): every +, -, *, / rounds as written, so decisions taken in it
// reproduce a plain double evaluation of the same expression, tie for tie.
struct dx {
    double v;
    dx() = default;
    __host__ __device__ __forceinline__ dx(double a) : v(a) {}
};
__device__ __forceinline__ dx operator+(dx a, dx b) { return dx(__dadd_rn(a.v, b.v)); }
__device__ __forceinline__ dx operator-(dx a, dx b) { return dx(__dsub_rn(a.v, b.v)); }
__device__ __forceinline__ dx operator-(dx a) { return dx(-a.v); }
__device__ __forceinline__ dx operator*(dx a, dx b) { return dx(__dmul_rn(a.v, b.v)); }
__device__ __forceinline__ dx operator/(dx a, dx b) { return dx(__ddiv_rn(a.v, b.v)); }
__device__ __forceinline__ bool operator<(dx a, dx b) { return a.v < b.v; }
__device__ __forceinline__ bool operator>(dx a, dx b) { return a.v > b.v; }
__device__ __forceinline__ bool operator<=(dx a, dx b) { return a.v <= b.v; }
__device__ __forceinline__ bool operator>=(dx a, dx b) { return a.v >= b.v; }
__device__ __forceinline__ bool operator==(dx a, dx b) { return a.v == b.v; }
__device__ __forceinline__ bool operator!=(dx a, dx b) { return a.v != b.v; }
__device__ __forceinline__ dx Sqrt(dx x) { return dx(__dsqrt_rn(x.v)); }
__device__ __forceinline__ dx Acos(dx x) { return dx(acos(x.v)); }
__device__ __forceinline__ dx Atan2(dx y, dx x) { return dx(atan2(y.v, x.v)); }
__device__ __forceinline__ dx Cbrt(dx x) { return dx(cbrt(x.v)); }
__device__ __forceinline__ dx Exp(dx x) { return dx(exp(x.v)); }
__device__ __forceinline__ dx Fabs(dx x) { return dx(fabs(x.v)); }
__device__ __forceinline__ dx Floor(dx x) { return dx(floor(x.v)); }
__device__ __forceinline__ dx Fmin(dx a, dx b) { return dx(fmin(a.v, b.v)); }
__device__ __forceinline__ dx Fmax(dx a, dx b) { return dx(fmax(a.v, b.v)); }
__device__ __forceinline__ void SinCos(dx x, dx *s, dx *c) { double a, b; sincos(x.v, &a, &b); *s = dx(a); *c = dx(b); }
__device__ __forceinline__ float to_float(dx x) { return (float)x.v; }
__device__ __forceinline__ float to_float(float x) { return x; }
__device__ __forceinline__ double to_double(dx x) { return x.v; }
__device__ __forceinline__ double to_double(float x) { return (double)x; }

// precision-generic math
__device__ __forceinline__ float Sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double Sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float Acos(float x) { return acosf(x); }
__device__ __forceinline__ double Acos(double x) { return acos(x); }
__device__ __forceinline__ float Atan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double Atan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float Cbrt(float x) { return cbrtf(x); }
__device__ __forceinline__ double Cbrt(double x) { return cbrt(x); }
__device__ __forceinline__ float Exp(float x) { return expf(x); }
__device__ __forceinline__ double Exp(double x) { return exp(x); }
__device__ __forceinline__ float Fabs(float x) { return fabsf(x); }
__device__ __forceinline__ double Fabs(double x) { return fabs(x); }
__device__ __forceinline__ float Floor(float x) { return floorf(x); }
__device__ __forceinline__ double Floor(double x) { return floor(x); }
__device__ __forceinline__ void SinCos(float x, float *s, float *c) { sincosf(x, s, c); }
__device__ __forceinline__ void SinCos(double x, double *s, double *c) { sincos(x, s, c); }
__device__ __forceinline__ void SinCosPi(float x, float *s, float *c) { sincospif(x, s, c); }
__device__ __forceinline__ void SinCosPi(double x, double *s, double *c) { sincospi(x, s, c); }
__device__ __forceinline__ float Fmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double Fmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float Fmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double Fmax(double a, double b) { return fmax(a, b); }

template <typename T>
__device__ __forceinline__ T norm3(v3t<T> a) { return Sqrt(dot3(a, a)); }
template <typename T>
__device__ __forceinline__ v3t<T> unit3(v3t<T> a) { return a * (T(1) / norm3(a)); }

// complex
template <typename T>
struct cpx {
    T re, im;
};
template <typename T>
__device__ __forceinline__ cpx<T> mkc(T r, T i) {
    cpx<T> c;
    c.re = r; c.im = i;
    return c;
}
template <typename T>
__device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return mkc<T>(a.re + b.re, a.im + b.im); }
template <typename T>
__device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return mkc<T>(a.re - b.re, a.im - b.im); }
template <typename T>
__device__ __forceinline__ cpx<T> operator*(cpx<T> a, cpx<T> b) {
    return mkc<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T>
__device__ __forceinline__ cpx<T> operator*(cpx<T> a, T s) { return mkc<T>(a.re * s, a.im * s); }
template <typename T>
__device__ __forceinline__ cpx<T> cdiv(cpx<T> a, cpx<T> b) {
    T d = T(1) / (b.re * b.re + b.im * b.im);
    return mkc<T>((a.re * b.re + a.im * b.im) * d, (a.im * b.re - a.re * b.im) * d);
}
template <typename T>
__device__ __forceinline__ cpx<T> cexpi(T ph) {   // e^{j ph}
    T s, c;
    SinCos(ph, &s, &c);
    return mkc<T>(c, s);
}

// ---- double-float (unevaluated sum hi + lo of two floats) ----
struct dfl {
    float hi, lo;
};
__device__ __forceinline__ dfl two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    dfl r;
    r.hi = s; r.lo = e;
    return r;
}
__device__ __forceinline__ dfl quick_two_sum(float a, float b) {
    float s = a + b;
    float e = b - (s - a);
    dfl r;
    r.hi = s; r.lo = e;
    return r;
}
__device__ __forceinline__ dfl two_prod(float a, float b) {
    float p = a * b;
    float e = fmaf(a, b, -p);
    dfl r;
    r.hi = p; r.lo = e;
    return r;
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    dfl s = two_sum(a.hi, b.hi);
    float e = s.lo + (a.lo + b.lo);
    return quick_two_sum(s.hi, e);
}
__device__ __forceinline__ dfl df_addf(dfl a, float b) {
    dfl s = two_sum(a.hi, b);
    return quick_two_sum(s.hi, s.lo + a.lo);
}
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    dfl p = two_prod(a.hi, b.hi);
    float e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
    return quick_two_sum(p.hi, e);
}
__device__ __forceinline__ dfl df_sqrt(dfl a) {
    float s = sqrtf(a.hi);
    if (s == 0.0f) { dfl z; z.hi = 0.f; z.lo = 0.f; return z; }
    dfl ss = two_prod(s, s);
    float r = ((a.hi - ss.hi) - ss.lo + a.lo) / (2.0f * s);
    return quick_two_sum(s, r);
}
__device__ __forceinline__ dfl df_neg(dfl a) {
    dfl r;
    r.hi = -a.hi; r.lo = -a.lo;
    return r;
}
// double-float times float
__device__ __forceinline__ dfl df_mulf(dfl a, float b) {
    dfl p = two_prod(a.hi, b);
    return quick_two_sum(p.hi, fmaf(a.lo, b, p.lo));
}
// double-float quotient (two correction terms of the FP32 quotient)
__device__ __forceinline__ dfl df_div(dfl a, dfl b) {
    float q1 = a.hi / b.hi;
    dfl r = df_add(a, df_neg(df_mulf(b, q1)));
    float q2 = r.hi / b.hi;
    return quick_two_sum(q1, q2);
}
// square of an exact float difference b - a, as double-float
__device__ __forceinline__ dfl df_sq_diff(float b, float a) {
    dfl d = two_sum(b, -a);
    dfl s = two_prod(d.hi, d.hi);
    s.lo = fmaf(2.0f * d.hi, d.lo, s.lo);
    return quick_two_sum(s.hi, s.lo);
}
// square of a double-float
__device__ __forceinline__ dfl df_sq(dfl d) {
    dfl s = two_prod(d.hi, d.hi);
    s.lo = fmaf(2.0f * d.hi, d.lo, s.lo);
    return quick_two_sum(s.hi, s.lo);
}
// |P - X| for a double-float point X = (hi.xyz + lo.xyz) and a float point P
__device__ __forceinline__ dfl df_dist_df(float4 hi, float4 lo, v3t<float> P) {
    dfl dx = df_addf(two_sum(hi.x, -P.x), lo.x);
    dfl dy = df_addf(two_sum(hi.y, -P.y), lo.y);
    dfl dz = df_addf(two_sum(hi.z, -P.z), lo.z);
    return df_sqrt(df_add(df_add(df_sq(dx), df_sq(dy)), df_sq(dz)));
}
// |b - a| for float points, as double-float (~1e-14 relative)
__device__ __forceinline__ dfl df_dist(v3t<float> a, v3t<float> b) {
    dfl s = df_add(df_add(df_sq_diff(b.x, a.x), df_sq_diff(b.y, a.y)), df_sq_diff(b.z, a.z));
    return df_sqrt(s);
}

}  // namespace creep
