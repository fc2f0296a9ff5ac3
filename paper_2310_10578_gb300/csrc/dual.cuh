// dual.cuh -- dual numbers for the adjoint (reverse) pass.
//
// DualT<S> carries a value and its derivatives with respect to eight
// parameters of one path: slots 0-3 the centre (x, y, z) and radius of the
// path's body, 4-6 the transmitter position, 7 the frequency (Hz).  Each
// path's field depends on no other parameter once its visibility is fixed, so
// eight tangents give the whole Jacobian of one path's field; the adjoint
// kernel contracts it with the incoming gradient of the fields.  Every
// operation below applies the first-order chain rule to the operation in the
// value's own precision: F8 (float) is the adjoint's default, D8 (double)
// its FP64 form.
#pragma once
#include "devmath.cuh"

namespace creep {

constexpr int ND = 8;
enum { DS_CX = 0, DS_CY = 1, DS_CZ = 2, DS_A = 3, DS_SX = 4, DS_SY = 5, DS_SZ = 6, DS_F = 7 };

template <typename S>
struct DualT {
    S v;
    S d[ND];
    DualT() = default;
    __device__ __forceinline__ DualT(S a) : v(a) {
#pragma unroll
        for (int k = 0; k < ND; ++k) d[k] = S(0);
    }
};
typedef DualT<double> D8;
typedef DualT<float> F8;

// the value-precision math of a dual's scalar type
__device__ __forceinline__ void dsincos(double x, double *s, double *c) { sincos(x, s, c); }
__device__ __forceinline__ void dsincos(float x, float *s, float *c) { sincosf(x, s, c); }
__device__ __forceinline__ void dsincospi(double x, double *s, double *c) { sincospi(x, s, c); }
__device__ __forceinline__ void dsincospi(float x, float *s, float *c) { sincospif(x, s, c); }

// a parameter: value a, derivative 1 in slot k
template <typename S>
__device__ __forceinline__ DualT<S> dvar_t(S a, int k) {
    DualT<S> r(a);
    r.d[k] = S(1);
    return r;
}
__device__ __forceinline__ D8 dvar(double a, int k) { return dvar_t<double>(a, k); }
// y = f(x) with f'(x) = df: y.d = df x.d
template <typename S>
__device__ __forceinline__ DualT<S> dchain(S y, S df, const DualT<S> &x) {
    DualT<S> r;
    r.v = y;
#pragma unroll
    for (int k = 0; k < ND; ++k) r.d[k] = df * x.d[k];
    return r;
}
template <typename S>
__device__ __forceinline__ DualT<S> operator+(const DualT<S> &a, const DualT<S> &b) {
    DualT<S> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] + b.d[k];
    return r;
}
template <typename S>
__device__ __forceinline__ DualT<S> operator-(const DualT<S> &a, const DualT<S> &b) {
    DualT<S> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] - b.d[k];
    return r;
}
template <typename S>
__device__ __forceinline__ DualT<S> operator-(const DualT<S> &a) {
    DualT<S> r;
    r.v = -a.v;
#pragma unroll
    for (int k = 0; k < ND; ++k) r.d[k] = -a.d[k];
    return r;
}
template <typename S>
__device__ __forceinline__ DualT<S> operator*(const DualT<S> &a, const DualT<S> &b) {
    DualT<S> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
template <typename S>
__device__ __forceinline__ DualT<S> operator/(const DualT<S> &a, const DualT<S> &b) {
    DualT<S> r;
    const S ib = S(1) / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int k = 0; k < ND; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
    return r;
}
template <typename S> __device__ __forceinline__ bool operator<(const DualT<S> &a, const DualT<S> &b) { return a.v < b.v; }
template <typename S> __device__ __forceinline__ bool operator>(const DualT<S> &a, const DualT<S> &b) { return a.v > b.v; }
template <typename S> __device__ __forceinline__ bool operator<=(const DualT<S> &a, const DualT<S> &b) { return a.v <= b.v; }
template <typename S> __device__ __forceinline__ bool operator>=(const DualT<S> &a, const DualT<S> &b) { return a.v >= b.v; }
template <typename S> __device__ __forceinline__ bool operator==(const DualT<S> &a, const DualT<S> &b) { return a.v == b.v; }
template <typename S> __device__ __forceinline__ bool operator!=(const DualT<S> &a, const DualT<S> &b) { return a.v != b.v; }

template <typename S>
__device__ __forceinline__ DualT<S> Sqrt(const DualT<S> &x) {
    const S s = sqrt(x.v);
    return dchain<S>(s, s > S(0) ? S(0.5) / s : S(0), x);
}
template <typename S>
__device__ __forceinline__ DualT<S> Cbrt(const DualT<S> &x) {
    const S c = cbrt(x.v);
    return dchain<S>(c, c != S(0) ? S(1) / (S(3) * c * c) : S(0), x);
}
template <typename S>
__device__ __forceinline__ DualT<S> Acos(const DualT<S> &x) {
    const S s = sqrt(fmax(S(0), S(1) - x.v * x.v));
    return dchain<S>(acos(x.v), s > S(0) ? S(-1) / s : S(0), x);
}
template <typename S>
__device__ __forceinline__ DualT<S> Atan2(const DualT<S> &y, const DualT<S> &x) {
    DualT<S> r;
    r.v = atan2(y.v, x.v);
    const S q = x.v * x.v + y.v * y.v;
    const S iq = q > S(0) ? S(1) / q : S(0);
#pragma unroll
    for (int k = 0; k < ND; ++k) r.d[k] = (x.v * y.d[k] - y.v * x.d[k]) * iq;
    return r;
}
template <typename S>
__device__ __forceinline__ DualT<S> Exp(const DualT<S> &x) {
    const S e = exp(x.v);
    return dchain<S>(e, e, x);
}
template <typename S>
__device__ __forceinline__ DualT<S> Fabs(const DualT<S> &x) { return dchain<S>(fabs(x.v), x.v < S(0) ? S(-1) : S(1), x); }
template <typename S>
__device__ __forceinline__ DualT<S> Fmin(const DualT<S> &a, const DualT<S> &b) { return (b.v < a.v) ? b : a; }
template <typename S>
__device__ __forceinline__ DualT<S> Fmax(const DualT<S> &a, const DualT<S> &b) { return (b.v > a.v) ? b : a; }
template <typename S>
__device__ __forceinline__ void SinCos(const DualT<S> &x, DualT<S> *s, DualT<S> *c) {
    S sv, cv;
    dsincos(x.v, &sv, &cv);
    *s = dchain<S>(sv, cv, x);
    *c = dchain<S>(cv, -sv, x);
}
template <typename S>
__device__ __forceinline__ void SinCosPi(const DualT<S> &x, DualT<S> *s, DualT<S> *c) {
    S sv, cv;
    dsincospi(x.v, &sv, &cv);
    *s = dchain<S>(sv, S(M_PI) * cv, x);
    *c = dchain<S>(cv, -S(M_PI) * sv, x);
}
template <typename S>
__device__ __forceinline__ double to_double(const DualT<S> &x) { return (double)x.v; }
template <typename S>
__device__ __forceinline__ float to_float(const DualT<S> &x) { return (float)x.v; }

}  // namespace creep
