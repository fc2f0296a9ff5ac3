// dual.cuh -- FP64 dual numbers for the adjoint (reverse) pass.
//
// D8 carries a value and its derivatives with respect to eight parameters of
// one path: slots 0-3 the centre (x, y, z) and radius of the path's body,
// 4-6 the transmitter position, 7 the frequency (Hz).  Each path's field
// depends on no other parameter once its visibility is fixed, so eight
// tangents give the whole Jacobian of one path's field; the adjoint kernel
// contracts it with the incoming gradient of the fields.  Every operation
// below applies the first-order chain rule to the exact FP64 operation.
#pragma once
#include "devmath.cuh"

namespace creep {

constexpr int ND = 8;
enum { DS_CX = 0, DS_CY = 1, DS_CZ = 2, DS_A = 3, DS_SX = 4, DS_SY = 5, DS_SZ = 6, DS_F = 7 };

struct D8 {
    double v;
    double d[ND];
    D8() = default;
    __device__ __forceinline__ D8(double a) : v(a) {
#pragma unroll
        for (int k = 0; k < ND; ++k) d[k] = 0.0;
    }
};
// a parameter: value a, derivative 1 in slot k
__device__ __forceinline__ D8 dvar(double a, int k) {
    D8 r(a);
    r.d[k] = 1.0;
    return r;
}
// y = f(x) with f'(x) = df: y.d = df x.d
__device__ __forceinline__ D8 dchain(double y, double df, const D8 &x) {
    D8 r;
    r.v = y;
#pragma unroll
    for (int k = 0; k < ND; ++k) r.d[k] = df * x.d[k];
    return r;
}
__device__ __forceinline__ D8 operator+(const D8 &a, const D8 &b) {
    D8 r;
    r.v = a.v + b.v;
#pragma unroll
    for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] + b.d[k];
    return r;
}
__device__ __forceinline__ D8 operator-(const D8 &a, const D8 &b) {
    D8 r;
    r.v = a.v - b.v;
#pragma unroll
    for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] - b.d[k];
    return r;
}
__device__ __forceinline__ D8 operator-(const D8 &a) {
    D8 r;
    r.v = -a.v;
#pragma unroll
    for (int k = 0; k < ND; ++k) r.d[k] = -a.d[k];
    return r;
}
__device__ __forceinline__ D8 operator*(const D8 &a, const D8 &b) {
    D8 r;
    r.v = a.v * b.v;
#pragma unroll
    for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
__device__ __forceinline__ D8 operator/(const D8 &a, const D8 &b) {
    D8 r;
    const double ib = 1.0 / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int k = 0; k < ND; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
    return r;
}
__device__ __forceinline__ bool operator<(const D8 &a, const D8 &b) { return a.v < b.v; }
__device__ __forceinline__ bool operator>(const D8 &a, const D8 &b) { return a.v > b.v; }
__device__ __forceinline__ bool operator<=(const D8 &a, const D8 &b) { return a.v <= b.v; }
__device__ __forceinline__ bool operator>=(const D8 &a, const D8 &b) { return a.v >= b.v; }
__device__ __forceinline__ bool operator==(const D8 &a, const D8 &b) { return a.v == b.v; }
__device__ __forceinline__ bool operator!=(const D8 &a, const D8 &b) { return a.v != b.v; }

__device__ __forceinline__ D8 Sqrt(const D8 &x) {
    const double s = sqrt(x.v);
    return dchain(s, s > 0.0 ? 0.5 / s : 0.0, x);
}
__device__ __forceinline__ D8 Cbrt(const D8 &x) {
    const double c = cbrt(x.v);
    return dchain(c, c != 0.0 ? 1.0 / (3.0 * c * c) : 0.0, x);
}
__device__ __forceinline__ D8 Acos(const D8 &x) {
    const double s = sqrt(fmax(0.0, 1.0 - x.v * x.v));
    return dchain(acos(x.v), s > 0.0 ? -1.0 / s : 0.0, x);
}
__device__ __forceinline__ D8 Atan2(const D8 &y, const D8 &x) {
    D8 r;
    r.v = atan2(y.v, x.v);
    const double q = x.v * x.v + y.v * y.v;
    const double iq = q > 0.0 ? 1.0 / q : 0.0;
#pragma unroll
    for (int k = 0; k < ND; ++k) r.d[k] = (x.v * y.d[k] - y.v * x.d[k]) * iq;
    return r;
}
__device__ __forceinline__ D8 Exp(const D8 &x) {
    const double e = exp(x.v);
    return dchain(e, e, x);
}
__device__ __forceinline__ D8 Fabs(const D8 &x) { return dchain(fabs(x.v), x.v < 0.0 ? -1.0 : 1.0, x); }
__device__ __forceinline__ D8 Fmin(const D8 &a, const D8 &b) { return (b.v < a.v) ? b : a; }
__device__ __forceinline__ D8 Fmax(const D8 &a, const D8 &b) { return (b.v > a.v) ? b : a; }
__device__ __forceinline__ void SinCos(const D8 &x, D8 *s, D8 *c) {
    double sv, cv;
    sincos(x.v, &sv, &cv);
    *s = dchain(sv, cv, x);
    *c = dchain(cv, -sv, x);
}
__device__ __forceinline__ void SinCosPi(const D8 &x, D8 *s, D8 *c) {
    double sv, cv;
    sincospi(x.v, &sv, &cv);
    *s = dchain(sv, M_PI * cv, x);
    *c = dchain(cv, -M_PI * sv, x);
}
__device__ __forceinline__ double to_double(const D8 &x) { return x.v; }
__device__ __forceinline__ float to_float(const D8 &x) { return (float)x.v; }

}  // namespace creep
