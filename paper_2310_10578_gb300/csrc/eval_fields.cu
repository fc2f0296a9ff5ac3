// eval_fields.cu -- the per-receiver field kernels (sm_103a).
//
// For every receiver P the method enumerates the candidate ray paths (direct;
// planar image reflections of order 1 and 2, or the candidate face sequences
// of a large scene; per convex body the GO reflection and the creeping ray
// each way round, optionally with extra turns and fed by a wall reflection),
// decides each path's existence and visibility, and sums the coherent field
// of the valid ones over the frequencies (Eqs. 1-4 of the paper; the
// surface-ray geometry of Fig. 1).
//
// Work split.  One evaluation is a few class kernels k_eval<T, PATHS, CLS>
// on the caller's stream, one per path class (planar, body reflection,
// creeping, wall -> creeping), launched as programmatic dependents so that
// each one's geometry work overlaps the previous one's tail.  Blocks are
// persistent: they take work units of tiles of 32 consecutive receivers from
// an atomic queue; the warps of a tile split its candidates (warp p takes
// body b = p mod the tile's warps, planar candidate k = p mod ...) and their
// partial fields are summed in shared memory in warp order, so a result does
// not depend on timing.  The body classes (FP32 fields) run two passes per
// tile: a geometry pass that writes one record per valid path to shared
// memory, then, after a block barrier, a field pass over the records per
// frequency chunk.  Scene geometry, source images, body frames and the
// Fock--Pekeris table are staged in shared memory per block.
//
// Precision (RT_PREC_FP32): geometry and field math in FP32; every
// existence/visibility decision is computed with a margin in metres and is
// taken in FP32 only when the margin exceeds a band that bounds the FP32
// error; otherwise the whole candidate is re-evaluated in FP64 with exactly
// the decision rules of the FP64 definition (ties: triangles and face
// membership inclusive, bodies strict).  Path lengths are accumulated as
// double-float so that the phase 2 pi frac(L / lambda) keeps ~1e-7 rad at
// 28 GHz over tens of metres.  Reflection points near grazing incidence are
// refined in FP64.  RT_PREC_FP64 runs everything in FP64.
#include <cuda_runtime.h>
#include <stdint.h>

#include "devmath.cuh"
#include "dual.cuh"
#include "internal.h"

namespace creep {

#define EPS_TRIM 1e-6
enum { D_NO = 0, D_YES = 1, D_UNSURE = 2 };
enum { PT_LOS = 0, PT_R1 = 1, PT_R2 = 2, PT_RB = 3, PT_CP = 4, PT_CM = 5, PT_WCP = 6, PT_WCM = 7, PT_R3 = 8 };

constexpr int BLOCK = 128;
constexpr int SMEM_TRI_MAX = 256;
constexpr int SMEM_FACE_MAX = 512;
constexpr int SMEM_BODY_MAX = 256;
constexpr int BVH_TOP_NODES = 511;     // BVH nodes (the top 9 levels) staged in shared memory per block

__device__ __forceinline__ uint64_t pcode(int type, int a, int b) {
    return ((uint64_t)type << 56) | ((uint64_t)a << 28) | (uint64_t)b;
}

// "m > 0" with an uncertainty band (band == 0: exact, ties -> tie)
template <typename T>
__device__ __forceinline__ int decide(T m, T band, int tie) {
    if (m > band) return D_YES;
    if (m < -band) return D_NO;
    if (band > T(0)) return D_UNSURE;
    return (m > T(0)) ? D_YES : ((m < T(0)) ? D_NO : tie);
}


// scene view (pointers into shared or global memory)
struct Ctx {
    const float4 *tri, *tri_aux, *face32, *body;
    const dq4 *face64;
    const int2 *face_rng;
    const int *face_tris;
    const float4 *face_box;      // see DevScene
    int n_tri, n_face, n_body;
    float band;
    v3t<float> S, pol;
    const float4 *fock;          // [FOCK_N][2], then the P segment [FOCK_NP][2] (see DevScene)
    const float4 *res;           // [FOCK_NRES][2]
    const float *weid;
    float weid_L;
    const double2 *fock64;
    const dq4 *res64;
    const double *weid64;
    const float4 *img;           // source images (double-float), see DevScene
    int img_pairs;               // img holds the ordered face pairs too
    const float4 *txb;           // [n_body][2] source-side body frame, see DevScene
    const float4 *txw;           // [n_face][n_body][2] the same for each face's source image (or nullptr)
    const float4 *bvh;           // triangle BVH, see DevScene (nullptr: every triangle is tested)
    const int *bvh_tri;
    const float4 *bvh_top;       // its first bvh_top_n nodes (the top levels) staged in shared memory
    int bvh_top_n;
    const int4 *cand;            // candidate face sequences, see DevScene (n_cand = 0: every face and pair)
    const float4 *cimg;
    int n_cand;
    const float4 *face_mat;      // face materials, see DevScene (nullptr: all PEC)
    int enc;                     // this launch's creeping rays: extra full turns round the body
    // occluder masks (FP32 body kernels): occ_w words per body; word w of
    // body b's source-side mask has bit j set if body j may block a segment
    // from the source to a point of body b (occ_w = 0: no masks)
    const uint32_t *occ_src;
    int occ_w;
};

template <typename T>
__device__ __forceinline__ v3t<T> ld3(float4 q) { return mk3<T>(T((double)q.x), T((double)q.y), T((double)q.z)); }
template <>
__device__ __forceinline__ v3t<float> ld3<float>(float4 q) { return mk3<float>(q.x, q.y, q.z); }

// ------------------------------------------------------------------ visibility
// Segment A->B (t in [EPS, 1-EPS]) against a closed triangle.
__device__ int seg_tri(const Ctx &c, int t, v3t<float> A, v3t<float> B, float band) {
    float4 nq = c.tri_aux[3 * t];
    v3t<float> n = mk3(nq.x, nq.y, nq.z);
    float sA = dot3(n, A) - nq.w, sB = dot3(n, B) - nq.w;
    if ((sA > band && sB > band) || (sA < -band && sB < -band)) return D_NO;
    if (!((sA > band && sB < -band) || (sA < -band && sB > band))) return D_UNSURE;
    v3t<float> v0 = ld3<float>(c.tri[3 * t]), v1 = ld3<float>(c.tri[3 * t + 1]), v2 = ld3<float>(c.tri[3 * t + 2]);
    v3t<float> D = B - A, e1 = v1 - v0, e2 = v2 - v0;
    v3t<float> pv = cross3(D, e2);
    float inv = 1.0f / dot3(e1, pv);
    v3t<float> tv = A - v0;
    float u = dot3(tv, pv) * inv;
    v3t<float> qv = cross3(tv, e1);
    float v = dot3(D, qv) * inv;
    float tt = dot3(e2, qv) * inv;
    float4 alt = c.tri_aux[3 * t + 1];
    float Dl = norm3(D);
    float m = fminf(fminf(u * alt.y, v * alt.z), (1.0f - u - v) * alt.x);
    m = fminf(m, fminf((tt - (float)EPS_TRIM) * Dl, (1.0f - (float)EPS_TRIM - tt) * Dl));
    return decide(m, band, D_YES);
}
__device__ int seg_tri(const Ctx &c, int t, v3t<dx> A, v3t<dx> B, dx) {
    v3t<dx> v0 = ld3<dx>(c.tri[3 * t]), v1 = ld3<dx>(c.tri[3 * t + 1]), v2 = ld3<dx>(c.tri[3 * t + 2]);
    v3t<dx> D = B - A, e1 = v1 - v0, e2 = v2 - v0;
    v3t<dx> pv = cross3(D, e2);
    dx det = dot3(e1, pv);
    if (det == dx(0.0)) return D_NO;
    dx inv = dx(1.0) / det;
    v3t<dx> tv = A - v0;
    dx u = dot3(tv, pv) * inv;
    if (u < dx(0.0) || u > dx(1.0)) return D_NO;
    v3t<dx> qv = cross3(tv, e1);
    dx v = dot3(D, qv) * inv;
    if (v < dx(0.0) || u + v > dx(1.0)) return D_NO;
    dx tt = dot3(e2, qv) * inv;
    return (tt >= dx(EPS_TRIM) && tt <= dx(1.0) - dx(EPS_TRIM)) ? D_YES : D_NO;
}

// Segment vs open solid body (tangent touch does not obstruct)
__device__ int seg_body(const Ctx &c, int b, v3t<float> A, v3t<float> B, float band) {
    float4 q0 = c.body[2 * b], q1 = c.body[2 * b + 1];
    v3t<float> D = B - A;
    if (q1.y == 0.0f) {   // sphere
        v3t<float> w = mk3(q0.x - A.x, q0.y - A.y, q0.z - A.z);
        float t = dot3(w, D) / dot3(D, D);
        t = fminf(fmaxf(t, (float)EPS_TRIM), 1.0f - (float)EPS_TRIM);
        v3t<float> q = D * t - w;
        return decide(q0.w - norm3(q), band, D_NO);
    }
    float ox = A.x - q0.x, oy = A.y - q0.y;
    float qa = D.x * D.x + D.y * D.y;
    float od = ox * D.x + oy * D.y;
    float tc = (qa > 0.0f) ? fminf(fmaxf(-od / qa, (float)EPS_TRIM), 1.0f - (float)EPS_TRIM) : (float)EPS_TRIM;
    float hx = ox + tc * D.x, hy = oy + tc * D.y;
    float m2 = q0.w - sqrtf(hx * hx + hy * hy);
    if (m2 < -band) return D_NO;
    if (m2 <= band) return D_UNSURE;
    float t1 = -1e30f, t2 = 1e30f;
    if (qa > 0.0f) {
        float cr = ox * D.y - oy * D.x;
        float half = sqrtf(fmaxf(q0.w * q0.w - cr * cr / qa, 0.0f)) / sqrtf(qa);
        float tm = -od / qa;
        t1 = tm - half; t2 = tm + half;
    }
    float t3 = -1e30f, t4 = 1e30f;
    if (D.z == 0.0f) {
        float mz = fminf(A.z - q0.z, q0.z + q1.x - A.z);
        if (mz < -band) return D_NO;
        if (mz <= band) return D_UNSURE;
    } else {
        float ta = (q0.z - A.z) / D.z, tb = (q0.z + q1.x - A.z) / D.z;
        t3 = fminf(ta, tb); t4 = fmaxf(ta, tb);
    }
    float lo = fmaxf(fmaxf(t1, t3), (float)EPS_TRIM), hi = fminf(fminf(t2, t4), 1.0f - (float)EPS_TRIM);
    return decide((hi - lo) * norm3(D), band, D_NO);
}
__device__ int seg_body(const Ctx &c, int b, v3t<dx> A, v3t<dx> B, dx) {
    float4 q0 = c.body[2 * b], q1 = c.body[2 * b + 1];
    v3t<dx> D = B - A;
    dx a = (double)q0.w;
    if (q1.y == 0.0f) {
        v3t<dx> w = mk3<dx>((double)q0.x, (double)q0.y, (double)q0.z) - A;
        dx t = dot3(w, D) / dot3(D, D);
        if (t < dx(EPS_TRIM)) t = dx(EPS_TRIM);
        if (t > dx(1.0) - dx(EPS_TRIM)) t = dx(1.0) - dx(EPS_TRIM);
        v3t<dx> q = (A + D * t) - mk3<dx>((double)q0.x, (double)q0.y, (double)q0.z);
        return (dot3(q, q) < a * a) ? D_YES : D_NO;
    }
    dx lo = dx(EPS_TRIM), hi = dx(1.0) - dx(EPS_TRIM);
    dx ox = A.x - dx((double)q0.x), oy = A.y - dx((double)q0.y);
    dx qa = D.x * D.x + D.y * D.y, qb = dx(2.0) * (ox * D.x + oy * D.y), qc = ox * ox + oy * oy - a * a;
    dx t1, t2;
    if (qa == dx(0.0)) {
        if (!(qc < dx(0.0))) return D_NO;
        t1 = dx(-INFINITY); t2 = dx(INFINITY);
    } else {
        dx disc = qb * qb - dx(4.0) * qa * qc;
        if (!(disc > dx(0.0))) return D_NO;
        dx sq = Sqrt(disc);
        t1 = (-qb - sq) / (dx(2.0) * qa);
        t2 = (-qb + sq) / (dx(2.0) * qa);
    }
    dx cz = (double)q0.z, h = (double)q1.x;
    dx t3, t4;
    if (D.z == dx(0.0)) {
        if (!(A.z > cz && A.z < cz + h)) return D_NO;
        t3 = dx(-INFINITY); t4 = dx(INFINITY);
    } else {
        dx ta = (cz - A.z) / D.z, tb = (cz + h - A.z) / D.z;
        t3 = Fmin(ta, tb); t4 = Fmax(ta, tb);
    }
    dx olo = Fmax(t1, t3), ohi = Fmin(t2, t4);
    if (!(olo < ohi)) return D_NO;
    return (olo < hi && ohi > lo) ? D_YES : D_NO;
}

// The segment A + t D, t in [0, 1], meets the box [lo, hi] grown by m?
// (the host grows every box by more than the rounding of this test)
template <typename T>
__device__ __forceinline__ bool seg_box(v3t<T> A, v3t<T> D, const float4 &lo, const float4 &hi, T m) {
    T t0 = T(0), t1 = T(1);
    const T a[3] = {A.x, A.y, A.z}, d[3] = {D.x, D.y, D.z};
    const T l[3] = {T((double)lo.x) - m, T((double)lo.y) - m, T((double)lo.z) - m};
    const T h[3] = {T((double)hi.x) + m, T((double)hi.y) + m, T((double)hi.z) + m};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (d[k] == T(0)) {
            if (a[k] < l[k] || a[k] > h[k]) return false;
            continue;
        }
        T u = (l[k] - a[k]) / d[k], v = (h[k] - a[k]) / d[k];
        if (u > v) { T w = u; u = v; v = w; }
        t0 = Fmax(t0, u);
        t1 = Fmin(t1, v);
        if (t0 > t1) return false;
    }
    return true;
}
// Triangles (those of faces sf1/sf2 skipped) through the BVH: 0 none hit, 1
// hit, 2 unsure.  FP64: each triangle is tested in FP32 on the rounded
// endpoints first, in FP64 only where that is uncertain.
template <typename T>
__device__ __forceinline__ int tris_bvh(const Ctx &c, v3t<T> A, v3t<T> B, int sf1, int sf2, T band) {
    v3t<float> Af, Bf;
    float box_m = 0.0f;
    if constexpr (sizeof(T) == 4) {
        Af = A; Bf = B;
        box_m = band;
    } else {
        Af = mk3<float>(to_float(A.x), to_float(A.y), to_float(A.z));
        Bf = mk3<float>(to_float(B.x), to_float(B.y), to_float(B.z));
    }
    const v3t<float> Df = Bf - Af;
    int stk[32];
    int sp = 0, uns = 0;
    stk[sp++] = 0;
    while (sp > 0) {
        const int nd = stk[--sp];
        // the top levels from shared memory, the rest through L1/L2
        const float4 *nb = (nd < c.bvh_top_n) ? c.bvh_top : c.bvh;
        const float4 lo = nb[2 * nd], hi = nb[2 * nd + 1];
        // box test in FP32 in both precisions: on the rounded endpoints it
        // stays conservative (the boxes are padded by 1e-4 m plus 1e-6 of the
        // coordinate, far beyond the rounding of the endpoints and the test)
        if (!seg_box<float>(Af, Df, lo, hi, box_m)) continue;
        const int first = __float_as_int(lo.w), count = __float_as_int(hi.w);
        if (count == 0) {
            if (sp + 2 > 32) { uns = 1; continue; }    // (the host build is at most 32 deep)
            stk[sp++] = first + 1;
            stk[sp++] = first;
            continue;
        }
        for (int j = first; j < first + count; ++j) {
            const int t = c.bvh_tri[j];
            const int f = __float_as_int(c.tri[3 * t].w);
            if (f == sf1 || f == sf2) continue;
            int r;
            if constexpr (sizeof(T) == 4) {
                r = seg_tri(c, t, Af, Bf, c.band);
            } else {
                r = seg_tri(c, t, Af, Bf, c.band);
                if (r == D_UNSURE) r = seg_tri(c, t, A, B, band);
            }
            if (r == D_YES) return D_YES;
            uns |= (r == D_UNSURE);
        }
    }
    return uns ? D_UNSURE : D_NO;
}

// 0 visible, 1 blocked, 2 unsure.  Faces sf1/sf2 and body sb are skipped.
template <typename T>
__device__ __forceinline__ int blocked_impl(const Ctx &c, v3t<T> A, v3t<T> B, int sf1, int sf2, int sb, T band) {
    int uns = 0;
    if constexpr (sizeof(T) == 4) {
        // faces first: both ends clearly on one side of a face's plane => none of
        // its triangles can be hit (the plane tests of all faces are made
        // branch-free; only the faces left over are looked at); large scenes
        // through the BVH
        if (c.bvh) {
            const int r = tris_bvh(c, A, B, sf1, sf2, band);
            if (r == D_YES) return D_YES;
            uns = (r == D_UNSURE);
        }
        for (int f0 = 0; f0 < (c.bvh ? 0 : c.n_face); f0 += 32) {
            unsigned keep = 0;
            const int nfc = min(32, c.n_face - f0);
#pragma unroll 4
            for (int k = 0; k < nfc; ++k) {
                float4 q = c.face32[f0 + k];
                float sA = q.x * A.x + q.y * A.y + q.z * A.z - q.w, sB = q.x * B.x + q.y * B.y + q.z * B.z - q.w;
                bool cull = (sA > band && sB > band) || (sA < -band && sB < -band) || f0 + k == sf1 || f0 + k == sf2;
                keep |= cull ? 0u : (1u << k);
            }
            while (keep) {
                const int f = f0 + __ffs(keep) - 1;
                keep &= keep - 1;
                int2 rg = c.face_rng[f];
                for (int i = 0; i < rg.y; ++i) {
                    int r = seg_tri(c, c.face_tris[rg.x + i], A, B, band);
                    if (r == D_YES) return D_YES;
                    uns |= (r == D_UNSURE);
                }
            }
        }
    } else {
        // exact decisions, FP32-filtered: each primitive is first tested in FP32
        // on the rounded endpoints with the FP32 error band (which also covers
        // the rounding of the endpoints); only an uncertain one is tested in FP64
        v3t<float> Af = mk3<float>(to_float(A.x), to_float(A.y), to_float(A.z));
        v3t<float> Bf = mk3<float>(to_float(B.x), to_float(B.y), to_float(B.z));
        if (c.bvh) {
            // D_UNSURE here is a traversal-stack overflow (the FP64 triangle
            // tests are exact): the segment is then never reported visible.
            // The host build bounds the depth so that it cannot happen.
            const int rb = tris_bvh(c, A, B, sf1, sf2, band);
            if (rb != D_NO) return rb;
        }
        for (int t = 0; t < (c.bvh ? 0 : c.n_tri); ++t) {
            int f = __float_as_int(c.tri[3 * t].w);
            if (f == sf1 || f == sf2) continue;
            int r = seg_tri(c, t, Af, Bf, c.band);
            if (r == D_UNSURE) r = seg_tri(c, t, A, B, band);
            if (r == D_YES) return D_YES;
        }
#pragma unroll 1
        for (int b = 0; b < c.n_body; ++b) {
            if (b == sb) continue;
            int r = seg_body(c, b, Af, Bf, c.band);
            if (r == D_UNSURE) r = seg_body(c, b, A, B, band);
            if (r == D_YES) return D_YES;
        }
        return D_NO;
    }
    if constexpr (sizeof(T) == 4) {
        // bodies: a squared-distance test against the segment's closest point
        // to the centre (cylinders: to the axis, in projection) rejects the
        // bodies that are clearly apart -- distance above a + band, so the
        // margin of the full test would be below -band.  Four bodies at a
        // time without branches (sphere and cylinder differ by a select), so
        // their dependent chains overlap; the full test only for the rest.
        const v3t<float> D = B - A;
        const float qa = D.x * D.x + D.y * D.y;
        const float iqa = (qa > 0.0f) ? 1.0f / qa : 0.0f;
        const float idd = 1.0f / (qa + D.z * D.z);
        const float tlo = (float)EPS_TRIM, thi = 1.0f - (float)EPS_TRIM;
        const int nb = c.n_body;
        for (int b0 = 0; b0 < nb; b0 += 4) {
            unsigned near = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int b = min(b0 + k, nb - 1);
                const float4 q0 = c.body[2 * b];
                const bool sph = c.body[2 * b + 1].y == 0.0f;
                const float wx = q0.x - A.x, wy = q0.y - A.y, wz = sph ? q0.z - A.z : 0.0f;
                const float dz = sph ? D.z : 0.0f;
                const float t = fminf(fmaxf((wx * D.x + wy * D.y + wz * dz) * (sph ? idd : iqa), tlo), thi);
                const float hx = D.x * t - wx, hy = D.y * t - wy, hz = dz * t - wz;
                const float ab = q0.w + band;
                const bool n = (b0 + k < nb) && (b0 + k != sb) && (hx * hx + hy * hy + hz * hz <= ab * ab);
                near |= n ? (1u << k) : 0u;
            }
            while (near) {
                const int b = b0 + __ffs(near) - 1;
                near &= near - 1;
                int r = seg_body(c, b, A, B, band);
                if (r == D_YES) return D_YES;
                uns |= (r == D_UNSURE);
            }
        }
    }
    return uns ? D_UNSURE : D_NO;
}
// One out-of-line copy per precision: the visibility loop is called from ten
// places per receiver; inlining it everywhere overflows the instruction cache.
__device__ __noinline__ int blocked(const Ctx &c, v3t<float> A, v3t<float> B, int sf1, int sf2, int sb, float band) {
    return blocked_impl(c, A, B, sf1, sf2, sb, band);
}
// A leg with an occluder mask (FP32): the faces (but sf1, sf2) as in blocked;
// the bodies (but sb) are those of the mask occ, nw words (a superset of the
// bodies that can pass the distance test), or all of them without a mask.
__device__ __noinline__ int blocked_mask(const Ctx &c, v3t<float> A, v3t<float> B, int sf1, int sf2, int sb,
                                         float band, const uint32_t *occ, int nw) {
    if (!occ) return blocked_impl(c, A, B, sf1, sf2, sb, band);
    int uns = 0;
    if (c.bvh) {
        const int r = tris_bvh(c, A, B, sf1, sf2, band);
        if (r == D_YES) return D_YES;
        uns = (r == D_UNSURE);
    }
    for (int f0 = 0; f0 < (c.bvh ? 0 : c.n_face); f0 += 32) {
        unsigned keep = 0;
        const int nfc = min(32, c.n_face - f0);
#pragma unroll 4
        for (int k = 0; k < nfc; ++k) {
            float4 q = c.face32[f0 + k];
            float sA = q.x * A.x + q.y * A.y + q.z * A.z - q.w, sB = q.x * B.x + q.y * B.y + q.z * B.z - q.w;
            bool cull = (sA > band && sB > band) || (sA < -band && sB < -band) || f0 + k == sf1 || f0 + k == sf2;
            keep |= cull ? 0u : (1u << k);
        }
        while (keep) {
            const int f = f0 + __ffs(keep) - 1;
            keep &= keep - 1;
            int2 rg = c.face_rng[f];
            for (int i = 0; i < rg.y; ++i) {
                int r = seg_tri(c, c.face_tris[rg.x + i], A, B, band);
                if (r == D_YES) return D_YES;
                uns |= (r == D_UNSURE);
            }
        }
    }
    const v3t<float> D = B - A;
    const float qa = D.x * D.x + D.y * D.y;
    const float iqa = (qa > 0.0f) ? 1.0f / qa : 0.0f;
    const float idd = 1.0f / (qa + D.z * D.z);
    const float tlo = (float)EPS_TRIM, thi = 1.0f - (float)EPS_TRIM;
#pragma unroll 1
    for (int w = 0; w < nw; ++w) {
        unsigned cand = occ[w];
        if (sb >= 0 && sb >> 5 == w) cand &= ~(1u << (sb & 31));
        while (cand) {
            const int b = 32 * w + __ffs(cand) - 1;
            cand &= cand - 1;
            const float4 q0 = c.body[2 * b];
            const bool sph = c.body[2 * b + 1].y == 0.0f;
            const float wx = q0.x - A.x, wy = q0.y - A.y, wz = sph ? q0.z - A.z : 0.0f;
            const float dz = sph ? D.z : 0.0f;
            const float t = fminf(fmaxf((wx * D.x + wy * D.y + wz * dz) * (sph ? idd : iqa), tlo), thi);
            const float hx = D.x * t - wx, hy = D.y * t - wy, hz = dz * t - wz;
            const float ab = q0.w + band;
            if (hx * hx + hy * hy + hz * hz <= ab * ab) {
                int r = seg_body(c, b, A, B, band);
                if (r == D_YES) return D_YES;
                uns |= (r == D_UNSURE);
            }
        }
    }
    return uns ? D_UNSURE : D_NO;
}
__device__ __noinline__ int blocked(const Ctx &c, v3t<dx> A, v3t<dx> B, int sf1, int sf2, int sb, dx band) {
    return blocked_impl(c, A, B, sf1, sf2, sb, band);
}
// a leg from or to a point of body b; FP32 legs take the occluder mask occ
// (nullptr: every body)
template <typename T>
__device__ __forceinline__ int blocked_leg(const Ctx &c, v3t<T> A, v3t<T> B, int b, T band, const uint32_t *occ) {
    if constexpr (sizeof(T) == 4) return blocked_mask(c, A, B, -1, -1, b, band, occ, c.occ_w);
    else return blocked(c, A, B, -1, -1, b, band);
}
__device__ __forceinline__ const uint32_t *occ_of(const Ctx &c, const uint32_t *masks, int b) {
    return (masks && c.occ_w) ? masks + b * c.occ_w : nullptr;
}

// squared distance in the floor plane from p to the segment a b
__device__ __forceinline__ float seg_d2(float px, float py, float ax, float ay, float bx, float by) {
    const float dx = bx - ax, dy = by - ay, wx = px - ax, wy = py - ay;
    const float dd = dx * dx + dy * dy;
    const float t = dd > 0.0f ? fminf(fmaxf((wx * dx + wy * dy) / dd, 0.0f), 1.0f) : 0.0f;
    const float hx = wx - t * dx, hy = wy - t * dy;
    return hx * hx + hy * hy;
}

// ---- occluder masks of the planar legs (FP32 fields).  The lanes of a warp
// take the same planar candidate for the warp's receivers.  Its legs run
// between consecutive regions: the source point, the box of the lanes'
// reflection points on each face, the box of the lanes' receivers.  In
// projection on the floor every leg between two regions lies in the capsule
// of the segment joining the regions' centres, of radius the larger region's
// half-diagonal (a point of a leg is a convex combination of points of the
// two regions); a body whose disk, grown by the band and a margin for the
// FP32 arithmetic of this test, misses the capsule cannot pass the distance
// test of the visibility loop (projection shortens distances), and is left
// out of that leg's mask.

// a float's bits mapped to an unsigned integer of the same order
__device__ __forceinline__ unsigned ord_of(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float of_ord(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}
// the box in the floor plane of the points (x, y) of the lanes with v among
// the lanes `lanes` (all of which call this), as centre and half-diagonal;
// rad < 0 when no lane has v
__device__ __forceinline__ void lanes_box(unsigned lanes, bool v, float x, float y, float &cx, float &cy,
                                          float &rad) {
    const unsigned x0 = __reduce_min_sync(lanes, v ? ord_of(x) : 0xffffffffu);
    const unsigned x1 = __reduce_max_sync(lanes, v ? ord_of(x) : 0u);
    const unsigned y0 = __reduce_min_sync(lanes, v ? ord_of(y) : 0xffffffffu);
    const unsigned y1 = __reduce_max_sync(lanes, v ? ord_of(y) : 0u);
    if (x0 > x1) {
        cx = cy = 0.0f;
        rad = -1.0f;
        return;
    }
    const float fx0 = of_ord(x0), fx1 = of_ord(x1), fy0 = of_ord(y0), fy1 = of_ord(y1);
    cx = 0.5f * (fx0 + fx1);
    cy = 0.5f * (fy0 + fy1);
    // (rounded up by a relative 1e-6 for the centre's rounding)
    rad = 0.5f * sqrtf((fx1 - fx0) * (fx1 - fx0) + (fy1 - fy0) * (fy1 - fy0)) * 1.000001f;
}
// masks wm[l][nw] of the legs l = 0 .. LEGS - 1 between the disks (cx[l],
// cy[l], cr[l]) and (cx[l + 1], ...); the lanes `lanes` (all of which call
// this) share the bodies and set the bits by shared-memory atomics
template <int LEGS>
__device__ __forceinline__ void leg_masks(const Ctx &c, unsigned lanes, const float *cx, const float *cy,
                                          const float *cr, uint32_t *wm, int nw) {
    const int lane = threadIdx.x & 31;
    const int rank = __popc(lanes & ((1u << lane) - 1u)), nact = __popc(lanes);
    __syncwarp(lanes);                        // every lane is done with the previous masks
    for (int i = rank; i < LEGS * nw; i += nact) wm[i] = 0u;
    __syncwarp(lanes);
    const float margin = 1e-3f + 8.0f * c.band;
    float dx[LEGS], dy[LEGS], idd[LEGS], rl[LEGS];
#pragma unroll
    for (int l = 0; l < LEGS; ++l) {
        dx[l] = cx[l + 1] - cx[l];
        dy[l] = cy[l + 1] - cy[l];
        const float dd = dx[l] * dx[l] + dy[l] * dy[l];
        idd[l] = dd > 0.0f ? 1.0f / dd : 0.0f;
        rl[l] = fmaxf(cr[l], cr[l + 1]) + c.band + margin;
    }
#pragma unroll 1
    for (int b = rank; b < c.n_body; b += nact) {
        const float4 q = c.body[2 * b];
#pragma unroll
        for (int l = 0; l < LEGS; ++l) {
            // squared distance from the body's centre to the segment of centres
            const float wx = q.x - cx[l], wy = q.y - cy[l];
            const float t = fminf(fmaxf((wx * dx[l] + wy * dy[l]) * idd[l], 0.0f), 1.0f);
            const float hx = wx - t * dx[l], hy = wy - t * dy[l];
            const float lim = rl[l] + q.w;
            if (hx * hx + hy * hy <= lim * lim) atomicOr(&wm[l * nw + (b >> 5)], 1u << (b & 31));
        }
    }
    __syncwarp(lanes);
}

// point (on the triangle's plane) inside the closed triangle
__device__ int in_tri(const Ctx &c, int t, v3t<float> Q, float band) {
    float4 nq = c.tri_aux[3 * t], il = c.tri_aux[3 * t + 2];
    v3t<float> n = mk3(nq.x, nq.y, nq.z);
    v3t<float> v0 = ld3<float>(c.tri[3 * t]), v1 = ld3<float>(c.tri[3 * t + 1]), v2 = ld3<float>(c.tri[3 * t + 2]);
    float m0 = dot3(cross3(v1 - v0, Q - v0), n) * il.x;
    float m1 = dot3(cross3(v2 - v1, Q - v1), n) * il.y;
    float m2 = dot3(cross3(v0 - v2, Q - v2), n) * il.z;
    return decide(fminf(fminf(m0, m1), m2), band, D_YES);
}
__device__ int in_tri(const Ctx &c, int t, v3t<dx> Q, dx) {
    v3t<dx> v0 = ld3<dx>(c.tri[3 * t]), v1 = ld3<dx>(c.tri[3 * t + 1]), v2 = ld3<dx>(c.tri[3 * t + 2]);
    v3t<dx> n = cross3(v1 - v0, v2 - v0);
    if (dot3(cross3(v1 - v0, Q - v0), n) < dx(0.0)) return D_NO;
    if (dot3(cross3(v2 - v1, Q - v1), n) < dx(0.0)) return D_NO;
    if (dot3(cross3(v0 - v2, Q - v2), n) < dx(0.0)) return D_NO;
    return D_YES;
}
template <typename T>
__device__ int in_face(const Ctx &c, int f, v3t<T> Q, T band) {
    int2 r = c.face_rng[f];
    int uns = 0;
    for (int i = 0; i < r.y; ++i) {
        int d;
        if constexpr (sizeof(T) == 4) {
            d = in_tri(c, c.face_tris[r.x + i], Q, band);
        } else {
            d = in_tri(c, c.face_tris[r.x + i], mk3<float>(to_float(Q.x), to_float(Q.y), to_float(Q.z)), c.band);
            if (d == D_UNSURE) d = in_tri(c, c.face_tris[r.x + i], Q, band);
        }
        if (d == D_YES) return D_YES;
        uns |= (d == D_UNSURE);
    }
    return uns ? D_UNSURE : D_NO;
}

template <typename T> __device__ __forceinline__ void face_plane(const Ctx &c, int f, v3t<T> *n, T *d);
template <> __device__ __forceinline__ void face_plane<float>(const Ctx &c, int f, v3t<float> *n, float *d) {
    float4 q = c.face32[f]; *n = mk3(q.x, q.y, q.z); *d = q.w;
}
template <> __device__ __forceinline__ void face_plane<dx>(const Ctx &c, int f, v3t<dx> *n, dx *d) {
    dq4 q = c.face64[f]; *n = mk3<dx>(q.x, q.y, q.z); *d = dx(q.w);
}

// combine a new decision into a running conjunction; returns false to stop (definite NO)
__device__ __forceinline__ bool conj(int &acc, int d) {
    if (d == D_NO) { acc = D_NO; return false; }
    if (d == D_UNSURE) acc = D_UNSURE;
    return true;
}
__device__ __forceinline__ int vis_to_dec(int blk) { return blk == D_NO ? D_YES : (blk == D_YES ? D_NO : D_UNSURE); }

// ------------------------------------------------------------------ candidate geometry
template <typename T>
struct Geo {
    v3t<T> Q1, Q2, n1, n2;
    T sp, t, sq, amp, rho_g, inv_f1, inv_f2, dperp;
    int caus;
    dfl Lf;          // FP32 mode: total path length as double-float (reflection off a body)
    v3t<T> dr;       // reflection off a body: P - Q1, free of cancellation near the surface
};

template <typename T>
__device__ __forceinline__ v3t<T> mirror_pt(v3t<T> X, v3t<T> n, T d) {
    T dist = dot3(n, X) - d;
    return X - n * (T(2) * dist);
}

// signs of a and b strictly equal (want_same) or strictly opposite
template <typename T>
__device__ __forceinline__ int side_dec(T a, T b, T band, bool want_same) {
    if (band > T(0)) {
        if (Fabs(a) <= band || Fabs(b) <= band) return D_UNSURE;
        bool same = (a > 0) == (b > 0);
        return (same == want_same) ? D_YES : D_NO;
    }
    T p = a * b;
    return want_same ? (p > T(0) ? D_YES : D_NO) : (p < T(0) ? D_YES : D_NO);
}

template <typename T>
__device__ int cand_los(const Ctx &c, v3t<T> S, v3t<T> P, T band) {
    return vis_to_dec(blocked(c, S, P, -1, -1, -1, band));
}

// planar candidates: the geometric part (sides, reflection points in their
// faces; the points in g), then the visibility of the legs (FP32: with the
// legs' occluder masks wm, or none)
template <typename T>
__device__ __forceinline__ int cand_r1_geo(const Ctx &c, int i, v3t<T> S, v3t<T> P, T band, Geo<T> &g) {
    v3t<T> n; T d;
    face_plane<T>(c, i, &n, &d);
    T dS = dot3(n, S) - d, dP = dot3(n, P) - d;
    int acc = D_YES;
    if (!conj(acc, side_dec(dS, dP, band, true))) return D_NO;
    v3t<T> S1 = mirror_pt(S, n, d);
    T d1 = dot3(n, S1) - d;
    T t = d1 / (d1 - dP);
    g.Q1 = S1 + (P - S1) * t;
    if (!conj(acc, in_face(c, i, g.Q1, band))) return D_NO;
    return acc;
}
__device__ __forceinline__ int cand_r1_vis(const Ctx &c, int i, v3t<float> S, v3t<float> P, float band,
                                           const Geo<float> &g, int acc, const uint32_t *wm, int nw) {
    if (!conj(acc, vis_to_dec(blocked_mask(c, S, g.Q1, i, -1, -1, band, wm, nw)))) return D_NO;
    if (!conj(acc, vis_to_dec(blocked_mask(c, g.Q1, P, i, -1, -1, band, wm ? wm + nw : nullptr, nw)))) return D_NO;
    return acc;
}
template <typename T>
__device__ int cand_r1(const Ctx &c, int i, v3t<T> S, v3t<T> P, T band, Geo<T> &g) {
    int acc = cand_r1_geo<T>(c, i, S, P, band, g);
    if (acc == D_NO) return D_NO;
    if (!conj(acc, vis_to_dec(blocked(c, S, g.Q1, i, -1, -1, band)))) return D_NO;
    if (!conj(acc, vis_to_dec(blocked(c, g.Q1, P, i, -1, -1, band)))) return D_NO;
    return acc;
}

template <typename T>
__device__ __forceinline__ int cand_r2_geo(const Ctx &c, int i, int j, v3t<T> S, v3t<T> P, T band, Geo<T> &g) {
    v3t<T> ni, nj; T di, dj;
    face_plane<T>(c, i, &ni, &di);
    face_plane<T>(c, j, &nj, &dj);
    v3t<T> S1 = mirror_pt(S, ni, di);
    v3t<T> S2 = mirror_pt(S1, nj, dj);
    T d2 = dot3(nj, S2) - dj, dP = dot3(nj, P) - dj;
    int acc = D_YES;
    if (!conj(acc, side_dec(d2, dP, band, false))) return D_NO;
    T t2 = d2 / (d2 - dP);
    v3t<T> Q2 = S2 + (P - S2) * t2;
    if (!conj(acc, in_face(c, j, Q2, band))) return D_NO;
    T e1 = dot3(ni, S1) - di, eq = dot3(ni, Q2) - di;
    if (!conj(acc, side_dec(e1, eq, band, false))) return D_NO;
    T t1 = e1 / (e1 - eq);
    v3t<T> Q1 = S1 + (Q2 - S1) * t1;
    g.Q1 = Q1; g.Q2 = Q2;
    if (!conj(acc, in_face(c, i, Q1, band))) return D_NO;
    return acc;
}
__device__ __forceinline__ int cand_r2_vis(const Ctx &c, int i, int j, v3t<float> S, v3t<float> P, float band,
                                           const Geo<float> &g, int acc, const uint32_t *wm, int nw) {
    if (!conj(acc, vis_to_dec(blocked_mask(c, S, g.Q1, i, -1, -1, band, wm, nw)))) return D_NO;
    if (!conj(acc, vis_to_dec(blocked_mask(c, g.Q1, g.Q2, i, j, -1, band, wm ? wm + nw : nullptr, nw)))) return D_NO;
    if (!conj(acc, vis_to_dec(blocked_mask(c, g.Q2, P, j, -1, -1, band, wm ? wm + 2 * nw : nullptr, nw)))) return D_NO;
    return acc;
}
template <typename T>
__device__ int cand_r2(const Ctx &c, int i, int j, v3t<T> S, v3t<T> P, T band, Geo<T> &g) {
    int acc = cand_r2_geo<T>(c, i, j, S, P, band, g);
    if (acc == D_NO) return D_NO;
    if (!conj(acc, vis_to_dec(blocked(c, S, g.Q1, i, -1, -1, band)))) return D_NO;
    if (!conj(acc, vis_to_dec(blocked(c, g.Q1, g.Q2, i, j, -1, band)))) return D_NO;
    if (!conj(acc, vis_to_dec(blocked(c, g.Q2, P, j, -1, -1, band)))) return D_NO;
    return acc;
}

// candidate face sequence q of order k = sq.w (large-scene mode): the
// source's images after each reflection from the candidate table (FP32: hi;
// FP64: hi + lo); backwards from P, Q_m is where image m -> Q_{m+1} crosses
// face sq[m]'s plane (the two strictly on opposite sides) and lies in the
// face; then every leg clear but of the faces at its ends
template <typename T>
__device__ __forceinline__ v3t<T> cand_image(const Ctx &c, int q, int m) {
    const float4 h = c.cimg[6 * q + 2 * m];
    if constexpr (sizeof(T) == 4) {
        return mk3(h.x, h.y, h.z);
    } else {
        const float4 l = c.cimg[6 * q + 2 * m + 1];
        return mk3<T>(T((double)h.x + (double)l.x), T((double)h.y + (double)l.y), T((double)h.z + (double)l.z));
    }
}
// the geometric part: each reflection point on its face (no visibility)
template <typename T>
__device__ __forceinline__ int cand_seq_geom(const Ctx &c, int q, int4 sq, v3t<T> P, T band, v3t<T> Q[3]) {
    const int k = sq.w;
    const int fs[3] = {sq.x, sq.y, sq.z};
    int acc = D_YES;
    v3t<T> X = P;
#pragma unroll
    for (int m = 2; m >= 0; --m) {
        if (m >= k) continue;
        v3t<T> n; T d;
        face_plane<T>(c, fs[m], &n, &d);
        const v3t<T> I = cand_image<T>(c, q, m);
        const T di = dot3(n, I) - d, dX = dot3(n, X) - d;
        if (!conj(acc, side_dec(di, dX, band, false))) return D_NO;
        Q[m] = I + (X - I) * (di / (di - dX));
        if (!conj(acc, in_face(c, fs[m], Q[m], band))) return D_NO;
        X = Q[m];
    }
    return acc;
}
template <typename T>
__device__ int cand_seq(const Ctx &c, int q, int4 sq, v3t<T> S, v3t<T> P, T band, v3t<T> Q[3]) {
    const int k = sq.w;
    const int fs[3] = {sq.x, sq.y, sq.z};
    int acc = cand_seq_geom<T>(c, q, sq, P, band, Q);
    if (acc == D_NO) return D_NO;
    if (!conj(acc, vis_to_dec(blocked(c, S, Q[0], fs[0], -1, -1, band)))) return D_NO;
    if (k >= 2 && !conj(acc, vis_to_dec(blocked(c, Q[0], Q[1], fs[0], fs[1], -1, band)))) return D_NO;
    if (k >= 3 && !conj(acc, vis_to_dec(blocked(c, Q[1], Q[2], fs[1], fs[2], -1, band)))) return D_NO;
    const v3t<T> E = (k == 1) ? Q[0] : ((k == 2) ? Q[1] : Q[2]);
    if (!conj(acc, vis_to_dec(blocked(c, E, P, fs[k - 1], -1, -1, band)))) return D_NO;
    return acc;
}

// frame of the (S, c, P) problem: u towards S, v towards P (sphere: 3-D; cylinder: horizontal)
template <typename T>
struct Frame {
    v3t<T> u, v;
    T ds, dp, gam, bs, bp, pu, pv;
    T sps, sqp;     // tangent lengths sqrt(ds^2 - a^2), sqrt(dp^2 - a^2) (horizontal for cylinders)
    bool axis_ok;   // v well conditioned (P not near the S-c axis)
    int dec;        // D_YES: lateral paths possible; D_NO: source or receiver over a cylinder's footprint
    dfl dsq;        // FP32 mode: sqrt(ds^2 - a^2) as double-float (from the FP64 source precomputation)
    dfl dpq;        // FP32 mode: sqrt(dp^2 - a^2) as double-float
};

template <typename T>
__device__ void sphere_frame(v3t<T> S, v3t<T> P, v3t<T> cc, T a, Frame<T> &F, T band) {
    v3t<T> ws = S - cc, wp = P - cc;
    F.ds = norm3(ws); F.dp = norm3(wp);
    F.u = ws * (T(1) / F.ds);
    F.gam = Atan2(norm3(cross3(ws, wp)), dot3(ws, wp));
    v3t<T> vp = wp - F.u * dot3(wp, F.u);
    T nv = norm3(vp);
    F.axis_ok = (band > T(0)) ? (nv > T(1e-3) * F.dp) : true;
    if (nv == T(0)) {
        v3t<T> tmp = (Fabs(F.u.x) < T(0.9)) ? mk3<T>(1, 0, 0) : mk3<T>(0, 1, 0);
        F.v = unit3(cross3(F.u, tmp));
    } else {
        // second Gram-Schmidt pass: vp is rounding noise for P on the S-c axis
        F.v = vp * (T(1) / nv);
        F.v = unit3(F.v - F.u * dot3(F.v, F.u));
    }
    F.bs = Acos(a / F.ds); F.bp = Acos(a / F.dp);
    F.sps = Sqrt(F.ds * F.ds - a * a); F.sqp = Sqrt(F.dp * F.dp - a * a);
    F.pu = dot3(wp, F.u); F.pv = dot3(wp, F.v);
}

template <typename T>
__device__ void cyl_frame(v3t<T> S, v3t<T> P, T cx, T cy, T a, Frame<T> &F, T band) {
    T sx = S.x - cx, sy = S.y - cy, px = P.x - cx, py = P.y - cy;
    F.ds = Sqrt(sx * sx + sy * sy); F.dp = Sqrt(px * px + py * py);
    F.u = mk3<T>(sx / F.ds, sy / F.ds, T(0));
    F.gam = Atan2(Fabs(sx * py - sy * px), sx * px + sy * py);
    // in the horizontal plane v is +-(z x u), turned toward P; in FP32 its sign
    // is uncertain only for P within rounding of the S-c line
    T side = F.u.x * py - F.u.y * px;                 // (z x u).(P - c)
    F.v = (side < T(0)) ? mk3<T>(F.u.y, -F.u.x, T(0)) : mk3<T>(-F.u.y, F.u.x, T(0));
    if constexpr (sizeof(T) == 4) F.axis_ok = Fabs(side) > T(4e-6) * F.dp;
    else F.axis_ok = true;
    F.bs = Acos(a / F.ds); F.bp = Acos(a / F.dp);
    F.sps = Sqrt(F.ds * F.ds - a * a); F.sqp = Sqrt(F.dp * F.dp - a * a);
    F.pu = px * F.u.x + py * F.u.y; F.pv = px * F.v.x + py * F.v.y;
}

// The (S, c, P) frame of body b, shared by its reflection and both creeping
// rays.  FP32: the source-only quantities (u, |S - c|, beta_s, s' or d_s, and
// whether the source is over a cylinder's footprint) come precomputed in FP64
// per transmitter (Ctx::txb); FP64: computed here as the definition does.
__device__ __forceinline__ void body_frame_tb(const Ctx &c, const float4 *tb, int b, v3t<float> S, v3t<float> P,
                                              float band, Frame<float> &F) {
    float4 q0 = c.body[2 * b], q1 = c.body[2 * b + 1], t0 = tb[2 * b], t1 = tb[2 * b + 1];
    float a = q0.w;
    F.dec = D_YES;
    F.axis_ok = true;
    if (t1.w == 0.0f) { F.dec = D_NO; return; }      // source over the cylinder's footprint
    F.u = mk3(t0.x, t0.y, t0.z);
    F.ds = t0.w;
    F.bs = t1.x;
    F.dsq.hi = t1.y; F.dsq.lo = t1.z;
    if (q1.y == 0.0f) {
        v3t<float> wp = mk3(P.x - q0.x, P.y - q0.y, P.z - q0.z);
        F.pu = dot3(F.u, wp);
        v3t<float> cr = cross3(F.u, wp);
        F.pv = norm3(cr);
        F.dp = norm3(wp);
        F.axis_ok = F.pv > 1e-3f * F.dp;
        F.v = (F.pv > 0.0f) ? (wp - F.u * F.pu) * (1.0f / F.pv) : mk3(0.f, 0.f, 0.f);
    } else {
        float px = P.x - q0.x, py = P.y - q0.y;
        F.dp = sqrtf(px * px + py * py);
        int d = decide(F.dp - a, band, D_NO);
        if (d == D_NO) { F.dec = D_NO; return; }
        F.dec = d;
        F.pu = F.u.x * px + F.u.y * py;
        float side = F.u.x * py - F.u.y * px;             // (z x u).(P - c)
        F.pv = fabsf(side);
        F.axis_ok = F.pv > 4e-6f * F.dp;
        F.v = (side < 0.0f) ? mk3(F.u.y, -F.u.x, 0.0f) : mk3(-F.u.y, F.u.x, 0.0f);
    }
    F.gam = atan2f(F.pv, F.pu);
    // receiver tangent length and angle from d_p^2 - a^2 formed exactly in
    // double-float (X - c and a^2 are exact): well conditioned also for a
    // receiver within a few ulp of the surface, where acos(a / d_p) and
    // d_p^2 - a^2 in FP32 lose most of their digits
    dfl q2 = df_add(df_sq_diff(P.x, q0.x), df_sq_diff(P.y, q0.y));
    if (q1.y == 0.0f) q2 = df_add(q2, df_sq_diff(P.z, q0.z));
    dfl a2 = two_prod(a, a);
    a2.hi = -a2.hi; a2.lo = -a2.lo;
    q2 = df_add(q2, a2);
    if (q2.hi > 0.0f) {
        F.dpq = df_sqrt(q2);
    } else {
        F.dpq.hi = 0.0f; F.dpq.lo = 0.0f;
    }
    F.sqp = F.dpq.hi;
    F.sps = F.dsq.hi;
    F.bp = atan2f(F.sqp, a);
}
__device__ void body_frame(const Ctx &c, int b, v3t<float> S, v3t<float> P, float band, Frame<float> &F) {
    body_frame_tb(c, c.txb, b, S, P, band, F);
}
__device__ void body_frame(const Ctx &c, int b, v3t<dx> S, v3t<dx> P, dx band, Frame<dx> &F) {
    float4 q0 = c.body[2 * b], q1 = c.body[2 * b + 1];
    dx a = (double)q0.w;
    F.dec = D_YES;
    if (q1.y == 0.0f) {
        sphere_frame(S, P, mk3<dx>((double)q0.x, (double)q0.y, (double)q0.z), a, F, band);
        return;
    }
    dx rs = Sqrt((S.x - dx((double)q0.x)) * (S.x - dx((double)q0.x)) + (S.y - dx((double)q0.y)) * (S.y - dx((double)q0.y)));
    dx rp = Sqrt((P.x - dx((double)q0.x)) * (P.x - dx((double)q0.x)) + (P.y - dx((double)q0.y)) * (P.y - dx((double)q0.y)));
    if (!(rs > a) || !(rp > a)) { F.dec = D_NO; return; }
    cyl_frame(S, P, dx((double)q0.x), dx((double)q0.y), a, F, band);
}

// 2-D reflection point on the circle of radius a, S = (ds, 0), P = (pu, pv)
// with pv >= 0 and gam = the angle of P in [0, pi]: the root psi of dL/dpsi
// in (0, gam), returned as n = (cos psi, sin psi) with psi.
//   FP32: safeguarded Newton in x = psi / pi (sincospi needs no argument
// reduction), with the bracket (lo, hi) for bisection.  For Q = a n, t = a
// (-sin psi, cos psi):
//   dL/dpsi   = (Q - S).t / |Q - S| + (Q - P).t / |Q - P|,
//   d2L/dpsi2 = sum over X = S, P of (X.Q - ((Q - X).t / |Q - X|)^2) / |Q - X|,
// each term formed from the difference vector Q - X itself (well conditioned
// for X within microns of the surface).  The start is the bisector of the
// directions to S and P, psi = gam / 2, moved by the first-order shift of the
// reflection point towards the nearer end, delta = (a / 2) sin(gam / 2) (1/d_p
// - 1/d_s) (from expanding dL/dpsi = 0 to first order in a / d).  The
// iteration stops at a step below 2e-7 psi, or at a Newton step below the
// rounding noise of dL/dpsi over its slope -- the root's own error estimate
// *err_est, which no further step could improve on.
__device__ __forceinline__ float rsqrt1(float x) {      // 1/sqrt(x) with one Newton step on rsqrtf
    const float y = rsqrtf(x);
    return y * fmaf(-0.5f * x * y, y, 1.5f);
}
__device__ float refl_n32(float a, float ds, float pu, float pv, float gam, float *cs_out, float *sn_out,
                          float *err_est) {
    constexpr float EPS8 = 8.0f * 1.2e-7f;       // 8 ulp: the rounding noise of dL/dpsi, relative to gmag
    constexpr float PI_F = 3.14159265358979f, IPI_F = 0.318309886183791f;
    float gmag = 0.0f, curv = 1.0f;
    const float ip = rsqrt1(pu * pu + pv * pv);
    const float bx = 1.0f + pu * ip, by = pv * ip;          // u_S + u_P (bx >= 0)
    const float s_half = by * rsqrt1(bx * bx + by * by);    // sin(gam / 2)
    float dl = 0.5f * a * s_half * (ip - 1.0f / ds);
    dl = fminf(fmaxf(dl, -0.4f * gam), 0.4f * gam);
    const float xg = gam * IPI_F;
    float lo = 0.0f, hi = xg;
    float x = 0.5f * xg + dl * IPI_F;
    float s, c;
    sincospif(x, &s, &c);
    for (int it = 0; it < 24; ++it) {
        const float qx = a * c, qy = a * s;
        const float sx = qx - ds, sy = qy, rx = qx - pu, ry = qy - pv;
        const float ifs = rsqrt1(sx * sx + sy * sy), ifr = rsqrt1(rx * rx + ry * ry);
        const float gs = (sy * qx - sx * qy) * ifs, gr = (ry * qx - rx * qy) * ifr;    // (Q - X).t / |Q - X|
        const float g = gs + gr;
        const float g2 = (ds * qx - gs * gs) * ifs + (pu * qx + pv * qy - gr * gr) * ifr;
        gmag = fabsf(gs) + fabsf(gr) + a;
        curv = g2;
        if (g == 0.0f) break;
        if (g < 0.0f) lo = x; else hi = x;
        float nx = x - g / (PI_F * g2);
        const bool newton = g2 > 0.0f && nx >= lo && nx <= hi;   // (false for a NaN step)
        if (!newton) nx = 0.5f * (lo + hi);
        const float step = PI_F * fabsf(nx - x);
        x = nx;
        sincospif(x, &s, &c);
        if (step <= 2e-7f * fmaxf(PI_F * x, 1e-3f) || (newton && step <= EPS8 * gmag / g2)) break;
    }
    const float psi = PI_F * x;
    *err_est = (curv > 0.0f) ? EPS8 * gmag / curv + 2e-7f * psi : 1.0f;
    *cs_out = c;
    *sn_out = s;
    return psi;
}
// FP64 Newton steps for the reflection point, on the unit vector
// n = (cos psi, sin psi) itself and without trigonometric calls: for Q = a n
// on the circle, (Q - S).t = a ds sin(psi) and (Q - P).t = a (pu sin(psi) -
// pv cos(psi)), t the unit tangent, so
//   dL/dpsi   = a [ds s / |Q - S| + (pu s - pv c) / |Q - P|],
//   d2L/dpsi2 = (X.Q - (dL/dpsi)_X^2) / |Q - X| summed over X = S, P,
// and n is rotated by each step d with cos d, sin d from their Taylor series
// (|d| <= 1e-3), until a step is below tol (quadratic convergence: the next
// one would be of order tol^2).  Returns false (no result) if a step is too
// large, the curvature not positive or six steps do not converge; the caller
// then takes the safeguarded iteration below.
__device__ bool refl_newton64(double A, double Ds, double Pu, double Pv, double *c_io, double *s_io, double tol) {
    double c = *c_io, s = *s_io;
    const double dp2 = Pu * Pu + Pv * Pv;
    for (int it = 0; it < 6; ++it) {
        double ifs = rsqrt(A * A + Ds * Ds - 2.0 * A * Ds * c);
        double ifr = rsqrt(A * A + dp2 - 2.0 * A * (Pu * c + Pv * s));
        double gs = A * Ds * s * ifs, gr = A * (Pu * s - Pv * c) * ifr;
        double g = gs + gr;
        double g2 = (Ds * A * c - gs * gs) * ifs + (A * (Pu * c + Pv * s) - gr * gr) * ifr;
        if (!(g2 > 0.0)) return false;
        double d = -g / g2;
        if (!(fabs(d) <= 1e-3)) return false;
        double d2 = d * d;
        double cd = 1.0 - d2 * (0.5 - d2 * (1.0 / 24.0));
        double sd = d * (1.0 - d2 * ((1.0 / 6.0) - d2 * (1.0 / 120.0)));
        double cn = c * cd - s * sd, sn = s * cd + c * sd;
        c = cn; s = sn;
        if (fabs(d) <= tol) {
            *c_io = c; *s_io = s;
            return true;
        }
    }
    return false;
}

// Double-float refinement of an FP32 reflection point (near-grazing
// incidence, where the FP32 root of dL/dpsi is too coarse for cos(theta_i)).

// FP64 reflection point from a start n0 = (c, s): safeguarded Newton on the
// unit vector n itself, without trigonometric calls.  The bracket is kept as
// two unit vectors, n_lo (dL/dpsi < 0; initially psi = 0, the direction of S)
// and n_hi (dL/dpsi >= 0; initially psi = gam, the direction of P).  For Q =
// a n and t = a (-s, c),
//   dL/dpsi   = (Q - S).t / |Q - S| + (Q - P).t / |Q - P|,
//   d2L/dpsi2 = sum over X = S, P of (X.Q - ((Q - X).t / |Q - X|)^2) / |Q - X|,
// each from the difference vector Q - X.  A Newton step d turns n by the
// angle 2 atan(d / 2) (the rational rotation ((1 - u^2), 2u) / (1 + u^2), u =
// d / 2: a unit vector by construction, equal to the turn by d up to d^3/12,
// which only changes the step length); a step that leaves the bracket is
// replaced by its bisector normalise(n_lo + n_hi) (the bracket spans less than
// pi).  Stops at a Newton step below tol, or below the rounding of dL/dpsi
// over its slope (4 ulp of its two terms: near grazing, where the slope
// vanishes, no step can improve on it), or at a bracket narrower than tol;
// the result is the last n.
__device__ void refl_root64(double A, double Ds, double Pu, double Pv, double *c_io, double *s_io, double tol) {
    const double ip = rsqrt(Pu * Pu + Pv * Pv);
    double lc = 1.0, ls = 0.0, hc = Pu * ip, hs = Pv * ip;
    double c = *c_io, s = *s_io;
    {
        const double r = rsqrt(c * c + s * s);
        c *= r; s *= r;
    }
    // a start outside the bracket: its bisector
    if (!(ls * c - lc * s < 0.0 && c * hs - s * hc > 0.0)) {
        const double bc = lc + hc, bs = ls + hs, r = rsqrt(bc * bc + bs * bs);
        c = bc * r; s = bs * r;
    }
    for (int it = 0; it < 80; ++it) {
        const double qx = A * c, qy = A * s;
        const double sx = qx - Ds, sy = qy, rx = qx - Pu, ry = qy - Pv;
        const double ifs = rsqrt(sx * sx + sy * sy), ifr = rsqrt(rx * rx + ry * ry);
        const double gs = (sy * qx - sx * qy) * ifs, gr = (ry * qx - rx * qy) * ifr;
        const double g = gs + gr;
        const double g2 = (Ds * qx - gs * gs) * ifs + (Pu * qx + Pv * qy - gr * gr) * ifr;
        if (g == 0.0) break;
        if (g < 0.0) { lc = c; ls = s; } else { hc = c; hs = s; }
        const double d = -g / g2;
        bool ok = g2 > 0.0 && fabs(d) <= 0.5;
        double nc = c, ns = s;
        if (ok) {
            const double u = 0.5 * d, iu = 1.0 / (1.0 + u * u);
            const double cd = (1.0 - u * u) * iu, sd = 2.0 * u * iu;
            nc = c * cd - s * sd;
            ns = s * cd + c * sd;
            ok = (ls * nc - lc * ns < 0.0) && (nc * hs - ns * hc > 0.0);     // strictly inside the bracket
        }
        if (!ok) {
            const double bc = lc + hc, bs = ls + hs, r = rsqrt(bc * bc + bs * bs);
            nc = bc * r; ns = bs * r;
        }
        c = nc; s = ns;
        const double noise = 4.0 * 1.1102230246251565e-16 * (fabs(gs) + fabs(gr)) / g2;
        if ((ok && (fabs(d) <= tol || fabs(d) <= noise)) || fabs(lc * hs - ls * hc) <= tol) break;
    }
    *c_io = c;
    *s_io = s;
}

// Double-float refinement of an FP32 reflection point (near-grazing
// incidence, where the FP32 root of dL/dpsi is too coarse for cos(theta_i)).
// At n0 = (c0, s0), the FP32 root, normalised exactly (1/|n0| = 1 - delta/2,
// delta = |n0|^2 - 1 formed exactly), dL/dpsi in the closed form
//   dL/dpsi = a [ds s / |Q - S| + (pu s - pv c) / |Q - P|]
// (for Q = a n on the circle, (Q - S).t = a ds s and (Q - P).t = a (pu s -
// pv c), t the unit tangent) is evaluated in double-float -- its two terms
// cancel at the root, which is what limits the FP32 root -- and Newton steps
// rotate n; the FP32 slope is enough for the step.  Returns false if a step
// exceeds 1e-3 or the slope is not positive.
__device__ bool refl_polish_df(float a, float ds, float pu, float pv, float c0, float s0, float *cs_out,
                               float *sn_out) {
    for (int it = 0; it < 4; ++it) {
        dfl r2 = df_add(two_prod(c0, c0), two_prod(s0, s0));
        float delta = (r2.hi - 1.0f) + r2.lo;
        dfl c, s;
        c.hi = c0; c.lo = -0.5f * delta * c0;
        s.hi = s0; s.lo = -0.5f * delta * s0;
        // |Q - S|^2 = a^2 + ds^2 - 2 a ds c,  |Q - P|^2 = a^2 + pu^2 + pv^2 - 2 a (pu c + pv s)
        dfl a2 = two_prod(a, a);
        dfl fs2 = df_add(df_add(a2, two_prod(ds, ds)), df_neg(df_mul(c, two_prod(2.0f * a, ds))));
        dfl ps = df_add(df_mulf(c, pu), df_mulf(s, pv));
        dfl fr2 = df_add(df_add(a2, df_add(two_prod(pu, pu), two_prod(pv, pv))), df_neg(df_mulf(ps, 2.0f * a)));
        dfl fs = df_sqrt(fs2), fr = df_sqrt(fr2);
        dfl t1 = df_div(df_mulf(s, ds), fs);
        dfl t2 = df_div(df_add(df_mulf(s, pu), df_neg(df_mulf(c, pv))), fr);
        dfl g = df_add(t1, t2);                               // (dL/dpsi) / a
        // slope d2L/dpsi2 = a sum_X (u - a)(|X|^2 - a u) / |Q - X|^3, u = X.n: a
        // product form (the difference form cancels near grazing)
        float uS = ds * c0, uP = ps.hi;
        float g2 = a * ((uS - a) * (ds * ds - a * uS) / (fs.hi * fs.hi * fs.hi) +
                        (uP - a) * (pu * pu + pv * pv - a * uP) / (fr.hi * fr.hi * fr.hi));
        if (!(g2 > 0.0f)) return false;
        float d = -(a * (g.hi + g.lo)) / g2;
        if (!(fabsf(d) <= 1e-3f)) return false;
        // rotate by d (cos d = 1 - d^2/2, sin d = d - d^3/6 to FP32 resolution
        // at this size), one rounding
        const float d2 = d * d, d3 = d2 * d * (1.0f / 6.0f);
        float cn = c0 + (c.lo - s0 * d - 0.5f * c0 * d2 + s0 * d3);
        float sn = s0 + (s.lo + c0 * d - 0.5f * s0 * d2 - c0 * d3);
        c0 = cn; s0 = sn;
        if (fabsf(d) <= 1e-9f) break;
    }
    *cs_out = c0;
    *sn_out = s0;
    return true;
}

// FP64 refinement of an FP32 reflection point, for the cases the
// double-float step does not take: FP64 Newton steps, the safeguarded
// iteration when they do not converge.  Returns (cos psi, sin psi) in FP32.
__device__ __noinline__ void refl_polish(float a, float ds, float pu, float pv, float gam, float c0f, float s0f,
                                         float *cs_out, float *sn_out) {
    double c = c0f, s = s0f;
    double r = 1.0 / sqrt(c * c + s * s);
    c *= r; s *= r;
    if (!refl_newton64(a, ds, pu, pv, &c, &s, 1e-9)) {        // (the result is rounded to FP32)
        c = c0f; s = s0f;
        refl_root64(a, ds, pu, pv, &c, &s, 1e-9);
    }
    *cs_out = (float)c;
    *sn_out = (float)s;
}

// FP64 reflection point: the FP32 root refined by FP64 Newton steps to a step
// below 1e-13 (the next one would be of order 1e-26); the safeguarded
// iteration when they do not converge.
__device__ __noinline__ void refl_root(dx a, dx ds, dx pu, dx pv, dx gam, dx *cs_out, dx *sn_out) {
    float err, c0f, s0f;
    refl_n32(to_float(a), to_float(ds), to_float(pu), to_float(pv), to_float(gam), &c0f, &s0f, &err);
    double c = c0f, s = s0f;
    double r = 1.0 / sqrt(c * c + s * s);
    c *= r; s *= r;
    if (!refl_newton64(a.v, ds.v, pu.v, pv.v, &c, &s, 1e-13)) {
        c = c0f; s = s0f;
        refl_root64(a.v, ds.v, pu.v, pv.v, &c, &s, 1e-13);
    }
    *cs_out = dx(c);
    *sn_out = dx(s);
}

// X - (c + a n) per component as double-float, for FP32 X, c, n and radius a:
// X - c is exact, a n is exact, so the vector (and its length) is that of the
// FP32 surface point c + a n itself, also when X lies within a wavelength of
// the surface, where |X - c|^2 + a^2 - 2 a (X - c).n would cancel.  horiz:
// horizontal components only (vertical cylinders), z returned as zero.
__device__ __forceinline__ void df_to_surface(v3t<float> X, float4 c, float a, v3t<float> n, bool horiz, dfl w[3]) {
    dfl m;
    m = two_prod(a, n.x); m.hi = -m.hi; m.lo = -m.lo;
    w[0] = df_add(two_sum(X.x, -c.x), m);
    m = two_prod(a, n.y); m.hi = -m.hi; m.lo = -m.lo;
    w[1] = df_add(two_sum(X.y, -c.y), m);
    if (horiz) {
        w[2].hi = 0.0f; w[2].lo = 0.0f;
    } else {
        m = two_prod(a, n.z); m.hi = -m.hi; m.lo = -m.lo;
        w[2] = df_add(two_sum(X.z, -c.z), m);
    }
}
__device__ __forceinline__ dfl df_norm3(const dfl w[3]) {
    return df_sqrt(df_add(df_add(df_sq(w[0]), df_sq(w[1])), df_sq(w[2])));
}

// smallest incidence cosine of a reflection off a body (see cand_rb)
constexpr double COS_MIN = 1e-30;

// body reflection candidate (sphere or vertical cylinder)
template <typename T>
__device__ int cand_rb(const Ctx &c, int b, v3t<T> S, v3t<T> P, T band, const Frame<T> &F, Geo<T> &g,
                       const uint32_t *occ_rx = nullptr) {
    float4 q0 = c.body[2 * b], q1 = c.body[2 * b + 1];
    T a = q0.w;
    int acc = F.dec;
    bool sphere = (q1.y == 0.0f);
    if (acc == D_NO) return D_NO;
    if (!F.axis_ok) return D_UNSURE;       // frame ill-conditioned: decide in FP64
    T dplus = F.gam - F.bs - F.bp;
    if (!conj(acc, decide(-dplus * a, band, D_NO))) return D_NO;      // strictly lit
    T sn, cs;
    if constexpr (sizeof(T) == 4) {
        float psi_err = 0.0f;
        refl_n32(a, F.ds, F.pu, F.pv, F.gam, &cs, &sn, &psi_err);
        // incidence cosine (2-D, horizontal for cylinders): refine the root in FP64
        // when its FP32 error would exceed 1e-5 of cos(theta_i) (near grazing),
        // the amplitude budget of the FP32 path
        float c2 = (F.ds * cs - a) / sqrtf((a * cs - F.ds) * (a * cs - F.ds) + a * a * sn * sn);
        if (psi_err > 1e-5f * fmaxf(c2, 0.0f)) {
            if (!refl_polish_df(a, F.ds, F.pu, F.pv, cs, sn, &cs, &sn))
                refl_polish(a, F.ds, F.pu, F.pv, F.gam, cs, sn, &cs, &sn);
        }
    } else {
        refl_root(a, F.ds, F.pu, F.pv, F.gam, &cs, &sn);
    }
    v3t<T> n = F.u * cs + F.v * sn;
    v3t<T> Q;
    if (sphere) {
        Q = mk3<T>(T((double)q0.x), T((double)q0.y), T((double)q0.z)) + n * a;
    } else {
        T qx = a * cs, qy = a * sn;
        T l1 = Sqrt((qx - F.ds) * (qx - F.ds) + qy * qy);
        T l2 = Sqrt((qx - F.pu) * (qx - F.pu) + (qy - F.pv) * (qy - F.pv));
        T zq = S.z + (P.z - S.z) * l1 / (l1 + l2);
        if (!conj(acc, decide(zq - T((double)q0.z), band, D_YES))) return D_NO;
        if (!conj(acc, decide(T((double)q0.z) + T((double)q1.x) - zq, band, D_YES))) return D_NO;
        Q = mk3<T>(T((double)q0.x) + a * n.x, T((double)q0.y) + a * n.y, zq);
    }
    v3t<T> shi = unit3(Q - S);
    // incidence cosine, positive on the lit side; at grazing its rounding may
    // reach zero, where the divergence factor's zero and the Fock-uniform
    // coefficient's pole (both of order cos^(1/2)) would meet as 0 * inf: the
    // smallest positive value keeps their finite product
    const T cth = Fmax(-dot3(shi, n), T(COS_MIN));
    if (!conj(acc, vis_to_dec(blocked_leg(c, S, Q, b, band, occ_of(c, c.occ_src, b))))) return D_NO;
    if (!conj(acc, vis_to_dec(blocked_leg(c, Q, P, b, band, occ_of(c, occ_rx, b))))) return D_NO;
    if constexpr (sizeof(T) == 4) {
        // total length s^i + s^r to the FP32 surface point c + a n, each leg in
        // double-float (the length is stationary in psi, so the FP32 root and
        // the rounding of n enter at second order along the surface and by
        // about a ulp of a across it)
        dfl ws[3], wp[3];
        df_to_surface(S, q0, a, n, !sphere, ws);
        df_to_surface(P, q0, a, n, !sphere, wp);
        dfl si = df_norm3(ws), sr = df_norm3(wp);
        if (sphere) {
            g.Lf = df_add(si, sr);
            g.dr = mk3<T>(wp[0].hi + wp[0].lo, wp[1].hi + wp[1].lo, wp[2].hi + wp[2].lo);
        } else {
            // unrolled: horizontal run l1 + l2, vertical rise P.z - S.z
            dfl H = df_add(si, sr);
            g.Lf = df_sqrt(df_add(df_mul(H, H), df_sq_diff(P.z, S.z)));
            float l1 = si.hi, l2 = sr.hi;
            g.dr = mk3<T>(wp[0].hi + wp[0].lo, wp[1].hi + wp[1].lo, (P.z - S.z) * (l2 / (l1 + l2)));
        }
    } else {
        g.dr = P - Q;
    }
    g.Q1 = Q; g.n1 = n;
    if (sphere) {
        g.inv_f1 = T(2) / (a * cth);
        g.inv_f2 = T(2) * cth / a;
        g.rho_g = a;
    } else {
        g.inv_f1 = T(2) * (T(1) - shi.z * shi.z) / (a * cth);
        g.inv_f2 = T(0);
        T sphi = -shi.x * n.y + shi.y * n.x;     // s_i . phi_hat, phi_hat = z x n
        g.rho_g = (sphi == T(0)) ? T(INFINITY) : a * (T(1) - cth * cth) / (sphi * sphi);
    }
    return acc;
}

// creeping candidate, dir 0 short way, 1 long way (SRC_LEG false: the leg
// from the source S to Q1 is the caller's, e.g. S is a source image)
template <typename T, bool SRC_LEG = true>
__device__ int cand_creep(const Ctx &c, int b, int dir, v3t<T> S, v3t<T> P, T band, const Frame<T> &F, Geo<T> &g,
                          const uint32_t *occ_rx = nullptr) {
    float4 q0 = c.body[2 * b], q1 = c.body[2 * b + 1];
    T a = q0.w;
    bool sphere = (q1.y == 0.0f);
    int acc = F.dec;
    if (acc == D_NO) return D_NO;
    if (!F.axis_ok) return D_UNSURE;       // frame ill-conditioned: decide in FP64
    const T TWO_PI_T = T(6.283185307179586476925286766559);
    T dpsi = (dir == 0) ? (F.gam - F.bs - F.bp) : (TWO_PI_T - F.gam - F.bs - F.bp);
    if (!conj(acc, decide(dpsi * a, band, D_NO))) return D_NO;
    // extra encirclements: the same attachment and shedding points, the arc
    // 2 pi a longer per turn; on a sphere the ray crosses the source axis
    // twice per turn (+j each: -1 per turn)
    if (c.enc > 0) dpsi = dpsi + TWO_PI_T * T(c.enc);
    // the attachment and shedding directions psi1 = +-beta_s and psi2 = gam
    // -+ beta_p in closed form: cos beta_s = a / d_s, sin beta_s = s' / d_s,
    // (cos gam, sin gam) = (p_u, p_v) / d_p, cos beta_p = a / d_p, sin beta_p =
    // s'' / d_p (tangent lengths s', s'' from the frame)
    const T ids = T(1) / F.ds, idp2 = T(1) / (F.dp * F.dp);
    const T c1 = a * ids;
    const T s1 = (dir == 0) ? F.sps * ids : -(F.sps * ids);
    const T pa_u = F.pu * a, pa_v = F.pv * a, qs_u = F.pu * F.sqp, qs_v = F.pv * F.sqp;
    const T c2 = ((dir == 0) ? pa_u + qs_v : pa_u - qs_v) * idp2;
    const T s2 = ((dir == 0) ? pa_v - qs_u : pa_v + qs_u) * idp2;
    g.n1 = F.u * c1 + F.v * s1;
    g.n2 = F.u * c2 + F.v * s2;
    if (sphere) {
        v3t<T> cc = mk3<T>(q0.x, q0.y, q0.z);
        g.Q1 = cc + g.n1 * a;
        g.Q2 = cc + g.n2 * a;
        g.sp = F.sps;
        g.sq = F.sqp;
        g.t = a * dpsi;
        g.rho_g = a;
        g.caus = (dir == 1);
        g.dperp = F.pv;                          // distance of P from the S-c axis, d_p sin(gam)
        const T dq1 = a * (F.sps * ids);         // a sin(beta_s)
        g.amp = (g.dperp > T(0)) ? Sqrt(dq1 / g.dperp) / Sqrt(g.sq) / g.sp : T(0);
        if (c.enc & 1) g.amp = -g.amp;           // the (-1) of an odd number of extra turns
    } else {
        T ds_ = F.sps, dp_ = F.sqp;
        T dz = P.z - S.z;
        T H = ds_ + a * dpsi + dp_;
        T ell = Sqrt(H * H + dz * dz);
        T sin0 = H / ell;
        T z1 = S.z + dz * ds_ / H, z2 = S.z + dz * (ds_ + a * dpsi) / H;
        T cz = q0.z, top = (T)q0.z + (T)q1.x;
        if (!conj(acc, decide(z1 - cz, band, D_YES))) return D_NO;
        if (!conj(acc, decide(top - z1, band, D_YES))) return D_NO;
        if (!conj(acc, decide(z2 - cz, band, D_YES))) return D_NO;
        if (!conj(acc, decide(top - z2, band, D_YES))) return D_NO;
        g.Q1 = mk3<T>((T)q0.x + a * g.n1.x, (T)q0.y + a * g.n1.y, z1);
        g.Q2 = mk3<T>((T)q0.x + a * g.n2.x, (T)q0.y + a * g.n2.y, z2);
        g.sp = ds_ / sin0; g.t = a * dpsi / sin0; g.sq = dp_ / sin0;
        g.rho_g = a / (sin0 * sin0);
        g.caus = 0;
        g.dperp = T(0);
        g.amp = T(1) / Sqrt(g.sp * g.sq * (g.sp + g.t + g.sq));
    }
    if constexpr (SRC_LEG) {
        if (!conj(acc, vis_to_dec(blocked_leg(c, S, g.Q1, b, band, occ_of(c, c.occ_src, b))))) return D_NO;
    }
    if (!conj(acc, vis_to_dec(blocked_leg(c, g.Q2, P, b, band, occ_of(c, occ_rx, b))))) return D_NO;
    return acc;
}

// The planar leg of a wall -> creeping path: the source S reflects at face f
// towards Q1, the attachment point of the creeping ray of S's image Sw.
// Q1 strictly on S's side of the plane; Qw (where Sw -> Q1 crosses it) in
// the face; S -> Qw clear (face f not tested), Qw -> Q1 clear (face f and
// body b not tested).
template <typename T>
__device__ __forceinline__ v3t<T> wall_point(const Ctx &c, int f, v3t<T> Sw, v3t<T> Q1, T *dQ) {
    v3t<T> n; T d;
    face_plane<T>(c, f, &n, &d);
    T dI = dot3(n, Sw) - d;
    *dQ = dot3(n, Q1) - d;
    return Sw + (Q1 - Sw) * (dI / (dI - *dQ));
}
template <typename T>
__device__ int wall_legs(const Ctx &c, int f, int b, v3t<T> S, v3t<T> Sw, v3t<T> Q1, T band) {
    v3t<T> n; T d;
    face_plane<T>(c, f, &n, &d);
    T dQ;
    const v3t<T> Qw = wall_point(c, f, Sw, Q1, &dQ);
    int acc = D_YES;
    if (!conj(acc, side_dec(dot3(n, S) - d, dQ, band, true))) return D_NO;
    if (!conj(acc, in_face(c, f, Qw, band))) return D_NO;
    if (!conj(acc, vis_to_dec(blocked(c, S, Qw, f, -1, -1, band)))) return D_NO;
    if (!conj(acc, vis_to_dec(blocked(c, Qw, Q1, f, -1, b, band)))) return D_NO;
    return acc;
}

// ------------------------------------------------------------------ Fock functions
// Weideman's rational approximation of w(z) = e^{-z^2} erfc(-jz), Im z > 0:
// w ~ 2 p(Z)/(L - jz)^2 + 1/(sqrt(pi) (L - jz)), Z = (L + jz)/(L - jz).
template <typename T>
__device__ cpx<T> faddeeva(const Ctx &c, cpx<T> z);
template <>
__device__ cpx<float> faddeeva<float>(const Ctx &c, cpx<float> z) {
    float L = c.weid_L;
    cpx<float> lm = mkc(L + z.im, -z.re), lp = mkc(L - z.im, z.re);
    cpx<float> Z = cdiv(lp, lm);
    cpx<float> p = mkc(c.weid[WEIDEMAN_N - 1], 0.0f);
    for (int n = WEIDEMAN_N - 2; n >= 0; --n) p = p * Z + mkc(c.weid[n], 0.0f);
    cpx<float> r = cdiv(p * 2.0f, lm * lm) + cdiv(mkc(0.56418958354775628f, 0.0f), lm);
    return r;
}
// Fock--Pekeris functions at xi >= XI_LO.  regular = true returns phat = P + c/xi,
// false returns P itself (each computed without cancellation in its domain).
__device__ void pekeris(const Ctx &c, float xi, cpx<float> &ps, cpx<float> &ph, bool regular) {
    const float ci = 0.19947114f / xi;                 // c/xi = e^{-j pi/4}/(2 sqrt(pi) xi) = (ci, -ci)
    if (xi > (float)XI_HI && xi < (float)XI_P) {
        // the table's P segment: cubic Hermite in P itself
        const float u = (xi - (float)XI_HI) * (float)(1.0 / XI_STEP);
        const int j = min(max((int)u, 0), FOCK_NP - 2);
        const float t = u - (float)j, t2 = t * t, omt = 1.0f - t;
        const float h00 = (1.0f + 2.0f * t) * omt * omt, h10 = t * omt * omt, h01 = t2 * (3.0f - 2.0f * t),
                    h11 = t2 * (t - 1.0f);
        const float4 *tp = c.fock + 2 * FOCK_N;
        const float4 a0 = tp[2 * j], a1 = tp[2 * j + 2], b0 = tp[2 * j + 1], b1 = tp[2 * j + 3];
        ps = mkc(h00 * a0.x + h10 * a0.z + h01 * a1.x + h11 * a1.z, h00 * a0.y + h10 * a0.w + h01 * a1.y + h11 * a1.w);
        ph = mkc(h00 * b0.x + h10 * b0.z + h01 * b1.x + h11 * b1.z, h00 * b0.y + h10 * b0.w + h01 * b1.y + h11 * b1.w);
        if (regular) { ps = ps + mkc(ci, -ci); ph = ph + mkc(ci, -ci); }
        return;
    }
    if (xi > (float)XI_HI) {
        // residue series: term n decays as exp(-xi rs.x); the terms are summed
        // until one falls below 1e-8 of the first (exp2 and sincospi with the
        // constants scaled by log2(e) and 1/pi: no large-argument reduction)
        const float LOG2E = 1.4426950408889634f, INV_PI = 0.31830988618379067f;
        cpx<float> ss = mkc(0.f, 0.f), sh = mkc(0.f, 0.f);
        const float x0s = xi * c.res[0].x, x0h = xi * c.res[1].x;
        for (int n = 0; n < FOCK_NRES; ++n) {
            float4 rs = c.res[2 * n];
            float xs = xi * rs.x;
            if (xs - x0s > 18.5f) break;
            float sn, cs;
            sincospif(xi * (rs.y * INV_PI), &sn, &cs);
            float e = exp2f(-xs * LOG2E) * rs.z;
            ss = ss + mkc(e * cs, -e * sn);
        }
        for (int n = 0; n < FOCK_NRES; ++n) {
            float4 rh = c.res[2 * n + 1];
            float xh = xi * rh.x;
            if (xh - x0h > 18.5f) break;
            float sn, cs;
            sincospif(xi * (rh.y * INV_PI), &sn, &cs);
            float e = exp2f(-xh * LOG2E) * rh.z;
            sh = sh + mkc(e * cs, -e * sn);
        }
        const cpx<float> pre = mkc(-0.27248264483602590f, 0.07301150463530957f);   // -e^{-j pi/12}/(2 sqrt(pi))
        ps = pre * ss;
        ph = pre * sh;
        if (regular) { ps = ps + mkc(ci, -ci); ph = ph + mkc(ci, -ci); }
        return;
    }
    float u = (xi - (float)XI_LO) * (float)(1.0 / XI_STEP);
    int j = min(max((int)u, 0), FOCK_N - 2);
    float t = u - (float)j;
    float t2 = t * t, omt = 1.0f - t;
    float h00 = (1.0f + 2.0f * t) * omt * omt, h10 = t * omt * omt, h01 = t2 * (3.0f - 2.0f * t), h11 = t2 * (t - 1.0f);
    float4 a0 = c.fock[2 * j], a1 = c.fock[2 * j + 2];
    float4 b0 = c.fock[2 * j + 1], b1 = c.fock[2 * j + 3];
    cpx<float> Gs = mkc(h00 * a0.x + h10 * a0.z + h01 * a1.x + h11 * a1.z, h00 * a0.y + h10 * a0.w + h01 * a1.y + h11 * a1.w);
    cpx<float> Gh = mkc(h00 * b0.x + h10 * b0.z + h01 * b1.x + h11 * b1.z, h00 * b0.y + h10 * b0.w + h01 * b1.y + h11 * b1.w);
    float sn, cs;
    sincospif(xi * xi * xi * (float)(1.0 / (12.0 * M_PI)), &sn, &cs);   // e^{+j xi^3/12}
    cpx<float> rot = mkc(cs, sn);
    ps = Gs * rot;
    ph = Gh * rot;
    if (!regular) { ps = ps - mkc(ci, -ci); ph = ph - mkc(ci, -ci); }
}
__device__ void pekeris(const Ctx &c, dx xid, cpx<dx> &psd, cpx<dx> &phd, bool regular) {
    double xi = xid.v;
    const double ci = (0.5 / sqrt(M_PI)) * cos(M_PI / 4.0) / xi;
    cpx<double> ps, ph;
    if (xi > XI_HI) {
        cpx<double> ss = mkc(0.0, 0.0), sh = mkc(0.0, 0.0);
        for (int n = 0; n < FOCK_NRES; ++n) {
            dq4 rs = c.res64[2 * n], rh = c.res64[2 * n + 1];
            double sn, cs;
            sincos(xi * rs.y, &sn, &cs);
            double e = exp(-xi * rs.x) * rs.z;
            ss = ss + mkc(e * cs, -e * sn);
            sincos(xi * rh.y, &sn, &cs);
            e = exp(-xi * rh.x) * rh.z;
            sh = sh + mkc(e * cs, -e * sn);
        }
        cpx<double> pre = mkc(-cos(M_PI / 12.0), sin(M_PI / 12.0)) * (0.5 / sqrt(M_PI));
        ps = pre * ss;
        ph = pre * sh;
        if (regular) { ps = ps + mkc(ci, -ci); ph = ph + mkc(ci, -ci); }
    } else {
        double u = (xi - XI_LO) / XI_STEP;
        int j = min(max((int)u, 0), FOCK_N - 2);
        double t = u - j, t2 = t * t, omt = 1.0 - t;
        double h00 = (1 + 2 * t) * omt * omt, h10 = t * omt * omt * XI_STEP, h01 = t2 * (3 - 2 * t), h11 = t2 * (t - 1) * XI_STEP;
        cpx<double> G[2];
        for (int k = 0; k < 2; ++k) {
            double2 g0 = c.fock64[(j * 2 + k) * 2], d0 = c.fock64[(j * 2 + k) * 2 + 1];
            double2 g1 = c.fock64[((j + 1) * 2 + k) * 2], d1 = c.fock64[((j + 1) * 2 + k) * 2 + 1];
            G[k] = mkc(h00 * g0.x + h10 * d0.x + h01 * g1.x + h11 * d1.x, h00 * g0.y + h10 * d0.y + h01 * g1.y + h11 * d1.y);
        }
        double sn, cs;
        sincos(xi * xi * xi / 12.0, &sn, &cs);
        ps = G[0] * mkc(cs, sn);
        ph = G[1] * mkc(cs, sn);
        if (!regular) { ps = ps - mkc(ci, -ci); ph = ph - mkc(ci, -ci); }
    }
    psd = mkc<dx>(ps.re, ps.im);
    phd = mkc<dx>(ph.re, ph.im);
}

__device__ __forceinline__ cpx<dx> faddeeva_dx(const Ctx &c, cpx<dx> zd) {
    cpx<double> z = mkc(zd.re.v, zd.im.v);
    double L = c.weid_L;
    cpx<double> lm = mkc(L + z.im, -z.re), lp = mkc(L - z.im, z.re);
    cpx<double> Z = cdiv(lp, lm);
    cpx<double> p = mkc(c.weid64[WEIDEMAN_N - 1], 0.0);
    for (int n = WEIDEMAN_N - 2; n >= 0; --n) p = p * Z + mkc(c.weid64[n], 0.0);
    cpx<double> r = cdiv(p * 2.0, lm * lm) + cdiv(mkc(0.56418958354775628, 0.0), lm);
    return mkc<dx>(r.re, r.im);
}
__device__ __forceinline__ cpx<float> faddeeva_t(const Ctx &c, cpx<float> z) { return faddeeva<float>(c, z); }
__device__ __forceinline__ cpx<dx> faddeeva_t(const Ctx &c, cpx<dx> z) { return faddeeva_dx(c, z); }

// Fock bracket B = P + (c/xi)(1 - F(X)) = phat - c F(X)/xi with sqrt(X) = K |xi|.
// X <= 4: phat - c F/xi, F/xi = sgn(xi) sqrt(pi) K e^{j pi/4} w(e^{j 3pi/4} K |xi|).
// X > 4: P + (c/xi)(1 - F), 1 - F from w (X < 30) or from the asymptotic series
// 1 - F ~ -sum_{n>=1} (2n-1)!! (j/(2X))^n (X >= 30, 8 terms): no cancellation
// between two O(c/xi) terms.
template <typename T>
__device__ __forceinline__ void fock_bracket_impl(const Ctx &c, T xi, T K, cpx<T> &Bs, cpx<T> &Bh) {
    const T r2 = T(0.70710678118654752440), spi = T(1.7724538509055160273), cc = T(0.19947114020071633897);
    T sx = K * Fabs(xi);
    T X = sx * sx;
    cpx<T> ps, ph;
    if (!(X > T(4))) {
        pekeris(c, xi, ps, ph, true);
        cpx<T> w = faddeeva_t(c, mkc<T>(-(sx * r2), sx * r2));
        T s = (xi >= T(0) ? T(1) : T(-1)) * spi * K * r2;
        cpx<T> fx = w * mkc<T>(s, s);                      // F/xi
        cpx<T> cf = mkc<T>(cc * (fx.re + fx.im), cc * (fx.im - fx.re));   // (1 - j) cc * fx
        Bs = ps - cf;
        Bh = ph - cf;
        return;
    }
    pekeris(c, xi, ps, ph, false);
    cpx<T> omf;                                            // 1 - F(X)
    if (X >= T(30)) {
        T u = T(0.5) / X;                                  // j/(2X) = j u
        cpx<T> acc = mkc<T>(T(1), T(0));
        for (int n = 8; n >= 2; --n) {                     // 1 + (2n-1) j u (...)
            T f = T(2 * n - 1) * u;
            acc = mkc<T>(T(1) - f * acc.im, f * acc.re);
        }
        omf = mkc<T>(u * acc.im, -(u * acc.re));           // -(j u) acc
    } else {
        cpx<T> w = faddeeva_t(c, mkc<T>(-(sx * r2), sx * r2));
        T s = Sqrt(T(3.14159265358979323846) * X) * r2;   // sqrt(pi X) e^{j pi/4}
        cpx<T> F = w * mkc<T>(s, s);
        omf = mkc<T>(T(1) - F.re, -F.im);
    }
    T ci = cc / xi;
    cpx<T> cterm = mkc<T>(ci * (omf.re + omf.im), ci * (omf.im - omf.re));   // (1 - j) ci (1 - F)
    Bs = ps + cterm;
    Bh = ph + cterm;
}

struct Bpair {
    cpx<float> s, h;
};
__device__ __forceinline__ Bpair fock_bracket_f(const Ctx &c, float xi, float K) {
    Bpair b;
    fock_bracket_impl<float>(c, xi, K, b.s, b.h);
    return b;
}
// F32FOCK: evaluate the bracket in FP32 also for FP64 geometry (candidates
// re-decided in FP64: the bracket is a smooth function of xi and X, and its
// FP32 evaluation is accurate to ~1e-6, inside the FP32 path's budget)
template <typename T, bool F32FOCK = false>
__device__ __forceinline__ void fock_bracket(const Ctx &c, T xi, T K, cpx<T> &Bs, cpx<T> &Bh) {
    if constexpr (sizeof(T) == 4) {
        Bpair b = fock_bracket_f(c, xi, K);
        Bs = b.s; Bh = b.h;
    } else if constexpr (F32FOCK) {
        Bpair b = fock_bracket_f(c, to_float(xi), to_float(K));
        Bs = mkc<T>(T((double)b.s.re), T((double)b.s.im));
        Bh = mkc<T>(T((double)b.h.re), T((double)b.h.im));
    } else {
        fock_bracket_impl<T>(c, xi, K, Bs, Bh);
    }
}

// ------------------------------------------------------------------ field accumulation
template <typename T>
struct Acc {
    cpx<T> E[NFC][3];
};
// The same sums kept in shared memory (the kernel's per-warp partial-field
// array; entry j of this lane at p[32 j], j = 6 f + 2 q + {0: re, 1: im}):
// the receiver's sums are then not live registers across the calls of the
// candidate loop.
template <typename T>
struct AccS {
    T *p;
};

template <typename T>
__device__ __forceinline__ v3t<T> src_pol(const Ctx &c, v3t<T> d) {
    v3t<T> p = mk3<T>(c.pol.x, c.pol.y, c.pol.z);
    v3t<T> pt = p - d * dot3(p, d);
    T n = norm3(pt);
    return (n > T(0)) ? pt * (T(1) / n) : mk3<T>(0, 0, 0);
}
template <typename T>
__device__ __forceinline__ v3t<T> pec_mirror(v3t<T> e, v3t<T> n) {
    return n * (T(2) * dot3(n, e)) - e;
}

// path length representation: FP32 mode carries double-float
struct LenF { dfl L; };
struct LenD { dx L; };

__device__ __forceinline__ cpx<float> phasor(const FreqC &fq, int f, dfl L) {
    dfl il; il.hi = fq.il_hi[f]; il.lo = fq.il_lo[f];
    dfl cyc = df_mul(L, il);
    float n = floorf(cyc.hi);
    float fr = (cyc.hi - n) + cyc.lo;
    fr -= floorf(fr);
    float s, co;
    sincospif(2.0f * fr, &s, &co);
    return mkc(co, -s);
}
__device__ __forceinline__ cpx<dx> phasor(const FreqC &fq, int f, dx Ld) {
    double L = Ld.v;
    double cyc = L * fq.fc[f];
    double fr = cyc - floor(cyc);
    double s, co;
    sincospi(2.0 * fr, &s, &co);
    return mkc<dx>(co, -s);
}
__device__ __forceinline__ float len_val(dfl L) { return L.hi + L.lo; }
__device__ __forceinline__ dx len_val(dx L) { return L; }
__device__ __forceinline__ float kof(const FreqC &fq, int f, float) { return fq.k[f]; }
__device__ __forceinline__ dx kof(const FreqC &fq, int f, dx) { return dx(fq.kd[f]); }
__device__ __forceinline__ float khof(const FreqC &fq, int f, float) { return fq.kh[f]; }
__device__ __forceinline__ dx khof(const FreqC &fq, int f, dx) { return dx(cbrt(fq.kd[f] * 0.5)); }

// segment length helpers
__device__ __forceinline__ dfl seglen(v3t<float> a, v3t<float> b) { return df_dist(a, b); }
__device__ __forceinline__ dx seglen(v3t<dx> a, v3t<dx> b) { return norm3(b - a); }
__device__ __forceinline__ dfl ladd(dfl a, dfl b) { return df_add(a, b); }
__device__ __forceinline__ dx ladd(dx a, dx b) { return a + b; }
__device__ __forceinline__ dfl laddf(dfl a, float b) { return df_addf(a, b); }
__device__ __forceinline__ dx laddf(dx a, dx b) { return a + b; }
__device__ __forceinline__ dfl lsqrt_diff_sq(float d, float a) {    // sqrt(d^2 - a^2)
    dfl s = two_prod(d, d), t = two_prod(a, a);
    t.hi = -t.hi; t.lo = -t.lo;
    return df_sqrt(df_add(s, t));
}
__device__ __forceinline__ dx lsqrt_diff_sq(dx d, dx a) { return Sqrt(d * d - a * a); }

// acc.E[f] += (x, y, z) for a runtime f (registers stay registers)
template <typename T>
__device__ __forceinline__ void acc_put(Acc<T> &acc, int f, cpx<T> x, cpx<T> y, cpx<T> z) {
#pragma unroll
    for (int ff = 0; ff < NFC; ++ff) {
        if (ff == f) {
            acc.E[ff][0] = acc.E[ff][0] + x;
            acc.E[ff][1] = acc.E[ff][1] + y;
            acc.E[ff][2] = acc.E[ff][2] + z;
        }
    }
}

template <typename T>
__device__ __forceinline__ void acc_put(AccS<T> &acc, int f, cpx<T> x, cpx<T> y, cpx<T> z) {
    T *q = acc.p + f * 6 * 32;
    q[0] = q[0] + x.re; q[32] = q[32] + x.im;
    q[64] = q[64] + y.re; q[96] = q[96] + y.im;
    q[128] = q[128] + z.re; q[160] = q[160] + z.im;
}
template <typename T>
__device__ __forceinline__ void acc_zero(AccS<T> &acc) {
#pragma unroll
    for (int j = 0; j < NFC * 6; ++j) acc.p[32 * j] = T(0.0);
}

template <typename T, typename L, typename ACC>
__device__ __forceinline__ void add_ray(ACC &acc, const FreqC &fq, v3t<T> e, T amp, L len) {
#pragma unroll 1
    for (int f = 0; f < fq.nf; ++f) {
        cpx<T> ph = phasor(fq, f, len) * amp;
        acc_put(acc, f, ph * e.x, ph * e.y, ph * e.z);
    }
}
// the same ray for nfq frequency chunks fqs[0 .. nfq - 1], whose partial sums
// follow one another (NFC * 6 rows each)
template <typename T, typename L>
__device__ __forceinline__ void add_ray_chunks(AccS<T> &acc, const FreqC *fqs, int nfq, v3t<T> e, T amp, L len) {
#pragma unroll 1
    for (int k = 0; k < nfq; ++k) {
        AccS<T> a{acc.p + k * (NFC * 6 * 32)};
        add_ray(a, fqs[k], e, amp, len);
    }
}
// ---- dielectric faces (planar reflections): Fresnel coefficients of a
// half-space of relative permittivity eps = eps' - j eps'' (e^{+jwt}),
//   G_perp = (cos - r) / (cos + r),  G_par = (eps cos - r) / (eps cos + r),
//   r = sqrt(eps - sin^2) (principal branch), cos = |s_i . n|,
// in the basis e_perp = unit(n x s_i), e_par = e_perp x s_i before and
// e_perp x s_r after the bounce, the basis in which the PEC image mirror is
// G_perp = -1, G_par = +1.  At normal incidence the reflection is G_perp E.
template <typename T>
__device__ __forceinline__ cpx<T> csqrt_t(cpx<T> z) {     // principal branch, without cancellation
    T r = Sqrt(z.re * z.re + z.im * z.im);
    if (z.re >= T(0)) {
        T a = Sqrt((r + z.re) * T(0.5));
        return mkc<T>(a, a > T(0) ? z.im / (a * T(2)) : T(0));
    }
    T b = Sqrt((r - z.re) * T(0.5));
    return mkc<T>(Fabs(z.im) / (b * T(2)), z.im < T(0) ? -b : b);
}
template <typename T>
__device__ __forceinline__ cpx<T> c3dot(const cpx<T> E[3], v3t<T> u) { return E[0] * u.x + E[1] * u.y + E[2] * u.z; }
template <typename T>
__device__ void reflect_face(const Ctx &c, int f, cpx<T> E[3], v3t<T> si, v3t<T> sr) {
    v3t<T> n;
    T d;
    face_plane<T>(c, f, &n, &d);
    const float4 m = c.face_mat ? c.face_mat[f] : make_float4(0.f, 0.f, 0.f, 0.f);
    if (m.x == 0.0f) {                                   // PEC: E -> -E + 2 (n.E) n
        cpx<T> en = c3dot(E, n) * T(2);
        E[0] = en * n.x - E[0]; E[1] = en * n.y - E[1]; E[2] = en * n.z - E[2];
        return;
    }
    const T cth = Fabs(dot3(si, n));
    const cpx<T> eps = mkc<T>(T((double)m.y), T(-(double)m.z));
    const cpx<T> r = csqrt_t(mkc<T>(eps.re - (T(1) - cth * cth), eps.im));
    const cpx<T> gs = cdiv(mkc<T>(cth - r.re, -r.im), mkc<T>(cth + r.re, r.im));
    const cpx<T> ec = eps * cth;
    const cpx<T> gp = cdiv(ec - r, ec + r);
    v3t<T> ep = cross3(n, si);
    const T ne = norm3(ep);
    if (ne == T(0)) {
        E[0] = E[0] * gs; E[1] = E[1] * gs; E[2] = E[2] * gs;
        return;
    }
    ep = ep * (T(1) / ne);
    const v3t<T> epi = cross3(ep, si), epr = cross3(ep, sr);
    const cpx<T> a = gs * c3dot(E, ep), b = gp * c3dot(E, epi);
    E[0] = a * ep.x + b * epr.x; E[1] = a * ep.y + b * epr.y; E[2] = a * ep.z + b * epr.z;
}
// a ray of complex polarisation e (amplitude amp, length len) at every frequency of fq
template <typename T, typename L, typename ACC>
__device__ __forceinline__ void add_ray_cx(ACC &acc, const FreqC &fq, const cpx<T> e[3], T amp, L len) {
#pragma unroll 1
    for (int f = 0; f < fq.nf; ++f) {
        cpx<T> ph = phasor(fq, f, len) * amp;
        acc_put(acc, f, ph * e[0], ph * e[1], ph * e[2]);
    }
}
// planar image path S -> Q1 (face i) [-> Q2 (face j)] -> P with at least one
// dielectric face: its complex polarisation, then the ray at every chunk
template <typename T, typename L>
__device__ __noinline__ void add_planar_dielectric(const Ctx &c, AccS<T> &acc, const FreqC *fqs, int nfq, v3t<T> S,
                                                   v3t<T> Q1, v3t<T> Q2, v3t<T> P, int i, int j, T amp, L len) {
    const v3t<T> s1 = unit3(Q1 - S);
    const v3t<T> e0 = src_pol(c, s1);
    cpx<T> E[3] = {mkc<T>(e0.x, T(0)), mkc<T>(e0.y, T(0)), mkc<T>(e0.z, T(0))};
    if (j < 0) {
        reflect_face(c, i, E, s1, unit3(P - Q1));
    } else {
        const v3t<T> s2 = unit3(Q2 - Q1);
        reflect_face(c, i, E, s1, s2);
        reflect_face(c, j, E, s2, unit3(P - Q2));
    }
#pragma unroll 1
    for (int k = 0; k < nfq; ++k) {
        AccS<T> a{acc.p + k * (NFC * 6 * 32)};
        add_ray_cx(a, fqs[k], E, amp, len);
    }
}
__device__ __forceinline__ bool dielectric(const Ctx &c, int f) { return c.face_mat && f >= 0 && c.face_mat[f].x != 0.0f; }
// candidate sequence path S -> Q[0] .. Q[k-1] -> P (faces fs): the source's
// polarisation reflected at each point (PEC mirror or Fresnel), the ray at
// every chunk
template <typename T, typename L>
__device__ __noinline__ void add_seq_field(const Ctx &c, AccS<T> &acc, const FreqC *fqs, int nfq, v3t<T> S,
                                           const v3t<T> Q[3], v3t<T> P, int4 sq, T amp, L len) {
    const int k = sq.w;
    const int fs[3] = {sq.x, sq.y, sq.z};
    v3t<T> din = unit3(Q[0] - S);
    const v3t<T> e0 = src_pol(c, din);
    if (!dielectric(c, fs[0]) && !(k >= 2 && dielectric(c, fs[1])) && !(k >= 3 && dielectric(c, fs[2]))) {
        v3t<T> e = e0;
        for (int m = 0; m < k; ++m) {
            v3t<T> n; T d;
            face_plane<T>(c, fs[m], &n, &d);
            e = pec_mirror(e, n);
        }
        add_ray_chunks(acc, fqs, nfq, e, amp, len);
        return;
    }
    cpx<T> E[3] = {mkc<T>(e0.x, T(0)), mkc<T>(e0.y, T(0)), mkc<T>(e0.z, T(0))};
    for (int m = 0; m < k; ++m) {
        const v3t<T> dout = unit3((m + 1 < k ? Q[m + 1] : P) - Q[m]);
        reflect_face(c, fs[m], E, din, dout);
        din = dout;
    }
#pragma unroll 1
    for (int ch = 0; ch < nfq; ++ch) {
        AccS<T> a{acc.p + ch * (NFC * 6 * 32)};
        add_ray_cx(a, fqs[ch], E, amp, len);
    }
}

template <typename T>
__device__ __forceinline__ void acc_zero_rows(AccS<T> &acc, int rows) {
#pragma unroll 4
    for (int j = 0; j < rows; ++j) acc.p[32 * j] = T(0.0);
}

template <typename T, typename L, bool F32FOCK = false, typename ACC = Acc<T>>
__device__ void field_body_refl(const Ctx &c, ACC &acc, const FreqC &fq, v3t<T> S, v3t<T> P, const Geo<T> &g, L len) {
    v3t<T> Q = g.Q1, n = g.n1;
    v3t<T> di = Q - S;
    T si = norm3(di), sr = norm3(g.dr);
    v3t<T> shi = di * (T(1) / si);
    const T cth = Fmax(-dot3(shi, n), T(COS_MIN));       // (as in cand_rb)
    // reflected direction by the law of reflection: unlike (P - Q) / |P - Q|
    // it does not turn with a rounding-size shift of Q along the surface,
    // which matters when the receiver is within a wavelength of the body
    v3t<T> shr = unit3(shi + n * (T(2) * cth));
    v3t<T> ep = cross3(n, shi);
    T ne = norm3(ep);
    if (ne == T(0)) {
        v3t<T> tmp = (Fabs(n.x) < T(0.9)) ? mk3<T>(1, 0, 0) : mk3<T>(0, 1, 0);
        ep = unit3(cross3(n, tmp));
    } else {
        ep = ep * (T(1) / ne);
    }
    v3t<T> epi = cross3(ep, shi), epr = cross3(ep, shr);
    v3t<T> e0 = src_pol(c, shi);
    T Es = dot3(e0, ep), Eh = dot3(e0, epi);
    T rho1 = T(1) / (T(1) / si + g.inv_f1), rho2 = T(1) / (T(1) / si + g.inv_f2);
    T A = Sqrt(rho1 * rho2 / ((rho1 + sr) * (rho2 + sr))) / si;
    T Lp = si * sr / (si + sr);
    T rcb = Cbrt(g.rho_g);
#pragma unroll 1
    for (int f = 0; f < fq.nf; ++f) {
        {
            T k = kof(fq, f, T(0));
            T m = khof(fq, f, T(0)) * rcb;
            T xi = T(-2) * m * cth;
            cpx<T> Rs, Rh;
            if (!(xi >= T(XI_LO))) {
                Rs = mkc<T>(-1, 0); Rh = mkc<T>(1, 0);
            } else {
                cpx<T> Bs, Bh;
                fock_bracket<T, F32FOCK>(c, xi, Sqrt(k * Lp / (T(2) * m * m)), Bs, Bh);
                T sn, cs;
                if constexpr (sizeof(T) == 4) sincospif(-xi * xi * xi * (float)(1.0 / (12.0 * M_PI)), &sn, &cs);
                else SinCos(-xi * xi * xi / T(12), &sn, &cs);
                cpx<T> pre = mkc<T>(cs, sn) * (-Sqrt(T(-4) / xi));
                Rs = pre * Bs; Rh = pre * Bh;
            }
            cpx<T> ph = phasor(fq, f, len) * A;
            cpx<T> as = Rs * ph * Es, ah = Rh * ph * Eh;
            acc_put(acc, f, as * ep.x + ah * epr.x, as * ep.y + ah * epr.y, as * ep.z + ah * epr.z);
        }
    }
}

template <typename T, typename L, bool F32FOCK = false, typename ACC = Acc<T>>
__device__ void field_creep(const Ctx &c, ACC &acc, const FreqC &fq, v3t<T> S, v3t<T> P, const Geo<T> &g,
                            L len, unsigned enable) {
    v3t<T> t1 = unit3(g.Q1 - S), t2 = unit3(P - g.Q2);
    v3t<T> b1 = cross3(t1, g.n1), b2 = cross3(t2, g.n2);
    v3t<T> e0 = src_pol(c, t1);
    T Es = dot3(e0, b1), Eh = dot3(e0, g.n1);
    if (!(enable & RT_EN_CREEP_SOFT)) Es = T(0);
    if (!(enable & RT_EN_CREEP_HARD)) Eh = T(0);
    T Lp = g.sp * g.sq / (g.sp + g.sq);
    T rcb = Cbrt(g.rho_g);
    T tr = g.t / g.rho_g;
#pragma unroll 1
    for (int f = 0; f < fq.nf; ++f) {
        {
            T k = kof(fq, f, T(0));
            T m = khof(fq, f, T(0)) * rcb;
            T xi = m * tr;
            cpx<T> Bs, Bh;
            fock_bracket<T, F32FOCK>(c, xi, Sqrt(k * Lp / (T(2) * m * m)), Bs, Bh);
            // T = -m sqrt(2/k) B e^{-jkt}; e^{-jkt} is inside the path phasor (len includes t)
            T pre = -m * Sqrt(T(2) / k) * g.amp;
            cpx<T> ph = phasor(fq, f, len) * pre;
            if (g.caus) ph = mkc<T>(-ph.im, ph.re);          // x (+j)
            cpx<T> as = Bs * ph * Es, ah = Bh * ph * Eh;
            acc_put(acc, f, as * b2.x + ah * g.n2.x, as * b2.y + ah * g.n2.y, as * b2.z + ah * g.n2.z);
        }
    }
}

// wall -> creeping path: the creeping ray of the source's image Sw in face f,
// with the source's polarisation reflected at Qw (complex for a dielectric
// face) as the incident field at Q1
template <typename T, typename L, bool F32FOCK = false, typename ACC = Acc<T>>
__device__ void field_wcreep(const Ctx &c, ACC &acc, const FreqC &fq, int wf, v3t<T> S, v3t<T> Sw, v3t<T> P,
                             const Geo<T> &g, L len, unsigned enable) {
    T dQ;
    const v3t<T> Qw = wall_point(c, wf, Sw, g.Q1, &dQ);
    const v3t<T> si = unit3(Qw - S), t1 = unit3(g.Q1 - Sw), t2 = unit3(P - g.Q2);
    const v3t<T> e0 = src_pol(c, si);
    cpx<T> E[3] = {mkc<T>(e0.x, T(0)), mkc<T>(e0.y, T(0)), mkc<T>(e0.z, T(0))};
    reflect_face(c, wf, E, si, t1);
    const v3t<T> b1 = cross3(t1, g.n1), b2 = cross3(t2, g.n2);
    cpx<T> Es = c3dot(E, b1), Eh = c3dot(E, g.n1);
    if (!(enable & RT_EN_CREEP_SOFT)) Es = mkc<T>(T(0), T(0));
    if (!(enable & RT_EN_CREEP_HARD)) Eh = mkc<T>(T(0), T(0));
    T Lp = g.sp * g.sq / (g.sp + g.sq);
    T rcb = Cbrt(g.rho_g);
    T tr = g.t / g.rho_g;
#pragma unroll 1
    for (int f = 0; f < fq.nf; ++f) {
        T k = kof(fq, f, T(0));
        T m = khof(fq, f, T(0)) * rcb;
        T xi = m * tr;
        cpx<T> Bs, Bh;
        fock_bracket<T, F32FOCK>(c, xi, Sqrt(k * Lp / (T(2) * m * m)), Bs, Bh);
        T pre = -m * Sqrt(T(2) / k) * g.amp;
        cpx<T> ph = phasor(fq, f, len) * pre;
        if (g.caus) ph = mkc<T>(-ph.im, ph.re);          // x (+j)
        cpx<T> as = Bs * ph * Es, ah = Bh * ph * Eh;
        acc_put(acc, f, as * b2.x + ah * g.n2.x, as * b2.y + ah * g.n2.y, as * b2.z + ah * g.n2.z);
    }
}

// ---- path records (FP32): the frequency-independent factors of one path's
// field, written by the geometry pass and turned into fields, frequency by
// frequency, by the field pass; the two passes are separate loops so that
// each one's code stays in the instruction cache, and so that the geometry
// is reused for every frequency chunk.  14 floats, entry j of a lane at
// rec[32 j]:
//   0 Es, 1 Eh, 2-4 e1, 5-7 e2, 8 A (creeping: amplitude, negative for the
//   ray through the caustic), 9 L' (transition distance; its sign tells the
//   kind: > 0 reflection, < 0 creeping), 10 rho_g^(1/3), 11 cos(theta_i)
//   (reflection) or t / rho_g (creeping), 12-13 path length.
// A candidate decided in FP64 gets the record of its FP64 geometry when its
// field goes through the records (several frequency chunks).
constexpr int REC_N = 14;

__device__ __forceinline__ void rec_put(float *r, float Es, float Eh, v3t<float> e1, v3t<float> e2, float A,
                                        float Lp, float rcb, float x, dfl len) {
    r[0] = Es; r[32] = Eh;
    r[64] = e1.x; r[96] = e1.y; r[128] = e1.z;
    r[160] = e2.x; r[192] = e2.y; r[224] = e2.z;
    r[256] = A; r[288] = Lp; r[320] = rcb; r[352] = x; r[384] = len.hi; r[416] = len.lo;
}

// reflection off a body: as field_body_refl, up to the frequency loop, in
// the geometry's own precision (FP64 for a candidate decided in FP64: near
// grazing its incidence cosine and divergence factor must come from the same
// FP64 geometry, as their product is what stays finite)
template <typename T>
__device__ __forceinline__ void rb_prep(const Ctx &c, float *r, v3t<T> S, const Geo<T> &g, dfl len) {
    auto f3 = [](v3t<T> v) { return mk3<float>(to_float(v.x), to_float(v.y), to_float(v.z)); };
    v3t<T> Q = g.Q1, n = g.n1;
    v3t<T> di = Q - S;
    T si = norm3(di), sr = norm3(g.dr);
    v3t<T> shi = di * (T(1) / si);
    const T cth = Fmax(-dot3(shi, n), T(COS_MIN));    // (as in cand_rb)
    v3t<T> shr = unit3(shi + n * (T(2) * cth));
    v3t<T> ep = cross3(n, shi);
    T ne = norm3(ep);
    if (ne == T(0)) {
        v3t<T> tmp = (Fabs(n.x) < T(0.9)) ? mk3<T>(1, 0, 0) : mk3<T>(0, 1, 0);
        ep = unit3(cross3(n, tmp));
    } else {
        ep = ep * (T(1) / ne);
    }
    v3t<T> epi = cross3(ep, shi), epr = cross3(ep, shr);
    v3t<T> e0 = src_pol(c, shi);
    T rho1 = T(1) / (T(1) / si + g.inv_f1), rho2 = T(1) / (T(1) / si + g.inv_f2);
    T A = Sqrt(rho1 * rho2 / ((rho1 + sr) * (rho2 + sr))) / si;
    rec_put(r, to_float(dot3(e0, ep)), to_float(dot3(e0, epi)), f3(ep), f3(epr), to_float(A),
            to_float(si * sr / (si + sr)), to_float(Cbrt(g.rho_g)), to_float(cth), len);
}
__device__ __forceinline__ void rb_apply(const Ctx &c, AccS<float> &acc, const FreqC &fq, const float *r) {
    const float Es = r[0], Eh = r[32], A = r[256], Lp = r[288], rcb = r[320], cth = r[352];
    dfl len;
    len.hi = r[384]; len.lo = r[416];
    const float sLr = sqrtf(Lp) / rcb;            // (K = sk sqrt(L') / rcb, as in creep_apply)
#pragma unroll 1
    for (int f = 0; f < fq.nf; ++f) {
        float m = fq.kh[f] * rcb;
        float xi = -2.0f * m * cth;
        cpx<float> Rs, Rh;
        if (!(xi >= (float)XI_LO)) {
            Rs = mkc<float>(-1, 0); Rh = mkc<float>(1, 0);
        } else {
            cpx<float> Bs, Bh;
            fock_bracket<float>(c, xi, fq.sk[f] * sLr, Bs, Bh);
            float sn, cs;
            sincospif(-xi * xi * xi * (float)(1.0 / (12.0 * M_PI)), &sn, &cs);
            cpx<float> pre = mkc<float>(cs, sn) * (-sqrtf(-4.0f / xi));
            Rs = pre * Bs; Rh = pre * Bh;
        }
        cpx<float> ph = phasor(fq, f, len) * A;
        cpx<float> as = Rs * ph * Es, ah = Rh * ph * Eh;
        acc_put(acc, f, as * r[64] + ah * r[160], as * r[96] + ah * r[192], as * r[128] + ah * r[224]);
    }
}

// creeping ray: as field_creep, up to the frequency loop
// (in the geometry's own precision: FP64 for a candidate decided in FP64)
template <typename T>
__device__ __forceinline__ void creep_prep(const Ctx &c, float *r, v3t<T> S, v3t<T> P, const Geo<T> &g, dfl len,
                                           unsigned enable) {
    auto f3 = [](v3t<T> v) { return mk3<float>(to_float(v.x), to_float(v.y), to_float(v.z)); };
    v3t<T> t1 = unit3(g.Q1 - S), t2 = unit3(P - g.Q2);
    v3t<T> b1 = cross3(t1, g.n1), b2 = cross3(t2, g.n2);
    v3t<T> e0 = src_pol(c, t1);
    float Es = (enable & RT_EN_CREEP_SOFT) ? to_float(dot3(e0, b1)) : 0.0f;
    float Eh = (enable & RT_EN_CREEP_HARD) ? to_float(dot3(e0, g.n1)) : 0.0f;
    const float amp = to_float(g.amp);
    if (signbit(amp)) { Es = -Es; Eh = -Eh; }    // (the record's amplitude sign is the caustic flag)
    rec_put(r, Es, Eh, f3(b2), f3(g.n2), g.caus ? -fabsf(amp) : fabsf(amp), to_float(-(g.sp * g.sq / (g.sp + g.sq))),
            to_float(Cbrt(g.rho_g)), to_float(g.t / g.rho_g), len);
}
// wall -> creeping path (see field_wcreep): the real part of the reflected
// polarisation in one record; an imaginary part (a dielectric face) in a
// second one, its factor j taken by the record's caustic flag (j j = -1
// where the ray already has one).  Returns the number of records written.
__device__ __forceinline__ int wcreep_prep(const Ctx &c, float *r, int wf, v3t<float> S, v3t<float> Sw,
                                           v3t<float> P, const Geo<float> &g, dfl len, unsigned enable) {
    float dQ;
    const v3t<float> Qw = wall_point(c, wf, Sw, g.Q1, &dQ);
    const v3t<float> si = unit3(Qw - S), t1 = unit3(g.Q1 - Sw), t2 = unit3(P - g.Q2);
    const v3t<float> e0 = src_pol(c, si);
    cpx<float> E[3] = {mkc(e0.x, 0.0f), mkc(e0.y, 0.0f), mkc(e0.z, 0.0f)};
    reflect_face(c, wf, E, si, t1);
    const v3t<float> b1 = cross3(t1, g.n1), b2 = cross3(t2, g.n2);
    const cpx<float> Es = (enable & RT_EN_CREEP_SOFT) ? c3dot(E, b1) : mkc(0.0f, 0.0f);
    const cpx<float> Eh = (enable & RT_EN_CREEP_HARD) ? c3dot(E, g.n1) : mkc(0.0f, 0.0f);
    const float sg = signbit(g.amp) ? -1.0f : 1.0f, A = fabsf(g.amp);
    const float Lp = -(g.sp * g.sq / (g.sp + g.sq)), rcb = cbrtf(g.rho_g), tr = g.t / g.rho_g;
    rec_put(r, sg * Es.re, sg * Eh.re, b2, g.n2, g.caus ? -A : A, Lp, rcb, tr, len);
    if (!dielectric(c, wf)) return 1;
    const float si2 = g.caus ? -sg : sg;
    rec_put(r + REC_N * 32, si2 * Es.im, si2 * Eh.im, b2, g.n2, g.caus ? A : -A, Lp, rcb, tr, len);
    return 2;
}
__device__ __forceinline__ void creep_apply(const Ctx &c, AccS<float> &acc, const FreqC &fq, const float *r) {
    const float Es = r[0], Eh = r[32], Lp = -r[288], rcb = r[320], tr = r[352];
    const float amp = fabsf(r[256]);
    const bool caus = r[256] < 0.0f;
    dfl len;
    len.hi = r[384]; len.lo = r[416];
    // per frequency, K = sqrt(k L' / (2 m^2)) = sk sqrt(L') / rcb and the
    // amplitude m sqrt(2 / k) = pk rcb (m = kh rcb)
    const float sLr = sqrtf(Lp) / rcb, ra = rcb * amp;
#pragma unroll 1
    for (int f = 0; f < fq.nf; ++f) {
        float m = fq.kh[f] * rcb;
        float xi = m * tr;
        cpx<float> Bs, Bh;
        fock_bracket<float>(c, xi, fq.sk[f] * sLr, Bs, Bh);
        float pre = -fq.pk[f] * ra;
        cpx<float> ph = phasor(fq, f, len) * pre;
        if (caus) ph = mkc<float>(-ph.im, ph.re);          // x (+j)
        cpx<float> as = Bs * ph * Es, ah = Bh * ph * Eh;
        acc_put(acc, f, as * r[64] + ah * r[160], as * r[96] + ah * r[192], as * r[128] + ah * r[224]);
    }
}

// total creeping path length s' + t + s
__device__ __forceinline__ dfl creep_len(const Ctx &c, int b, v3t<float> S, v3t<float> P, const Geo<float> &g,
                                         const Frame<float> &F) {
    float4 q1 = c.body[2 * b + 1];
    if (q1.y == 0.0f) return df_addf(df_add(F.dsq, F.dpq), g.t);
    // cylinder: unrolled straight line, sqrt(H^2 + dz^2), H = d_s + a dphi + d_p
    dfl ds_ = F.dsq, dp_ = F.dpq;
    // a dphi = t sin(theta0), sin(theta0) = d_s / s'
    float adphi = g.t * (len_val(ds_) / g.sp);
    dfl H = df_addf(df_add(ds_, dp_), adphi);
    dfl dz2 = df_sq_diff(P.z, S.z);
    dfl H2 = df_mul(H, H);
    return df_sqrt(df_add(H2, dz2));
}
__device__ __forceinline__ dx creep_len(const Ctx &, int, v3t<dx>, v3t<dx>, const Geo<dx> &g, const Frame<dx> &) {
    return g.sp + g.t + g.sq;
}

__device__ __forceinline__ void len_from(double x, dfl *L) { L->hi = (float)x; L->lo = (float)(x - (double)L->hi); }
__device__ __forceinline__ void len_from(double x, dx *L) { *L = dx(x); }

template <typename T> struct LenOf;
template <> struct LenOf<float> { typedef dfl type; };
template <> struct LenOf<dx> { typedef dx type; };

// FP64 geometry -> FP32 (escalated candidates feed the FP32 field code)
__device__ __forceinline__ v3t<float> to_f3(v3t<dx> a) { return mk3<float>(to_float(a.x), to_float(a.y), to_float(a.z)); }
__device__ __forceinline__ Geo<float> to_f(const Geo<dx> &d) {
    Geo<float> g;
    g.Q1 = to_f3(d.Q1); g.Q2 = to_f3(d.Q2); g.n1 = to_f3(d.n1); g.n2 = to_f3(d.n2);
    g.sp = to_float(d.sp); g.t = to_float(d.t); g.sq = to_float(d.sq); g.amp = to_float(d.amp);
    g.rho_g = to_float(d.rho_g); g.inv_f1 = to_float(d.inv_f1); g.inv_f2 = to_float(d.inv_f2);
    g.dperp = to_float(d.dperp); g.caus = d.caus;
    g.dr = to_f3(d.dr);
    return g;
}
__device__ __forceinline__ dfl to_df(double x) {
    dfl r;
    r.hi = (float)x;
    r.lo = (float)(x - (double)r.hi);
    return r;
}

// ------------------------------------------------------------------ FP64 re-evaluation
// Out of line: these run for the few candidates whose FP32 margins fall inside
// the error band; keeping them out of the kernel body keeps the hot loop small.
struct Contrib {
    cpx<float> E[NFC][3];
};
__device__ __forceinline__ void contrib_from(Contrib *o, const Acc<dx> &a) {
#pragma unroll
    for (int f = 0; f < NFC; ++f)
#pragma unroll
        for (int q = 0; q < 3; ++q) o->E[f][q] = mkc<float>(to_float(a.E[f][q].re), to_float(a.E[f][q].im));
}
__device__ __forceinline__ void acc_add(AccS<float> &a, const Contrib &b, int nf) {
    for (int f = 0; f < nf; ++f) acc_put(a, f, b.E[f][0], b.E[f][1], b.E[f][2]);
}
__device__ __forceinline__ void acc_zero(Acc<dx> &a) {
#pragma unroll
    for (int f = 0; f < NFC; ++f)
#pragma unroll
        for (int q = 0; q < 3; ++q) a.E[f][q] = mkc<dx>(0.0, 0.0);
}
__device__ __forceinline__ v3t<dx> dxv(v3t<float> a) { return mk3<dx>((double)a.x, (double)a.y, (double)a.z); }

__device__ __noinline__ int esc_inside(const Ctx &c, int b, v3t<float> Pf) {
    float4 q0 = c.body[2 * b], q1 = c.body[2 * b + 1];
    dx ex = dx((double)Pf.x) - dx((double)q0.x), ey = dx((double)Pf.y) - dx((double)q0.y),
       ez = dx((double)Pf.z) - dx((double)q0.z), a = dx((double)q0.w);
    if (q1.y == 0.0f) return (ex * ex + ey * ey + ez * ez <= a * a) ? D_YES : D_NO;
    return (ex * ex + ey * ey <= a * a && dx((double)Pf.z) >= dx((double)q0.z) &&
            dx((double)Pf.z) <= dx((double)q0.z) + dx((double)q1.x)) ? D_YES : D_NO;
}
__device__ __noinline__ int esc_los(const Ctx &c, v3t<float> Pf) {
    return cand_los<dx>(c, dxv(c.S), dxv(Pf), dx(0.0));
}
__device__ __noinline__ int esc_r1(const Ctx &c, int i, v3t<float> Pf, v3t<float> *Q) {
    Geo<dx> g;
    int d = cand_r1<dx>(c, i, dxv(c.S), dxv(Pf), dx(0.0), g);
    if (d == D_YES) *Q = to_f3(g.Q1);
    return d;
}
__device__ __noinline__ int esc_r2(const Ctx &c, int i, int j, v3t<float> Pf, v3t<float> *Q1, v3t<float> *Q2) {
    Geo<dx> g;
    int d = cand_r2<dx>(c, i, j, dxv(c.S), dxv(Pf), dx(0.0), g);
    if (d == D_YES) { *Q1 = to_f3(g.Q1); *Q2 = to_f3(g.Q2); }
    return d;
}
__device__ __noinline__ int esc_seq(const Ctx &c, int q, int4 sq, v3t<float> Pf, v3t<float> Q[3]) {
    v3t<dx> Qd[3];
    int d = cand_seq<dx>(c, q, sq, dxv(c.S), dxv(Pf), dx(0.0), Qd);
    if (d == D_YES)
        for (int m = 0; m < sq.w; ++m) Q[m] = to_f3(Qd[m]);
    return d;
}
// body reflection decided and (field = true) evaluated in FP64
__device__ __noinline__ int esc_rb(const Ctx &c, int b, v3t<float> Pf, const FreqC &fq, bool field, Contrib *out,
                                   float *rec) {
    Geo<dx> g;
    v3t<dx> Sd = dxv(c.S), Pd = dxv(Pf);
    Frame<dx> F;
    body_frame(c, b, Sd, Pd, dx(0.0), F);
    int d = cand_rb<dx>(c, b, Sd, Pd, dx(0.0), F, g);
    if (d == D_YES && rec) {
        // the path record of the FP64 geometry (its field is summed with the
        // FP32 records, frequency chunk by frequency chunk)
        rb_prep<dx>(c, rec, Sd, g, to_df(to_double(seglen(Sd, g.Q1) + seglen(g.Q1, Pd))));
    } else if (d == D_YES && field) {
        Acc<dx> a;
        acc_zero(a);
        field_body_refl<dx, dx, true>(c, a, fq, Sd, Pd, g, seglen(Sd, g.Q1) + seglen(g.Q1, Pd));
        contrib_from(out, a);
    }
    return d;
}
// creeping ray decided, its caustic flag taken, and (field) evaluated in FP64
__device__ __noinline__ int esc_creep(const Ctx &c, int b, int dir, v3t<float> Pf, const FreqC &fq, bool field,
                                      double half_lambda_max, unsigned enable, Contrib *out, int *caustic,
                                      float *rec = nullptr, int *n_rec = nullptr) {
    Geo<dx> g;
    v3t<dx> Sd = dxv(c.S), Pd = dxv(Pf);
    Frame<dx> F;
    body_frame(c, b, Sd, Pd, dx(0.0), F);
    int d = cand_creep<dx>(c, b, dir, Sd, Pd, dx(0.0), F, g);
    *caustic = 0;
    if (d != D_YES) return d;
    bool sphere = c.body[2 * b + 1].y == 0.0f;
    if (sphere) {
        *caustic = half_lambda_max > g.dperp.v;
        if (!(g.dperp > dx(0.0))) {                  // exactly on the axis: no finite ray field
            if (field) {
                for (int f = 0; f < NFC; ++f)
                    for (int q = 0; q < 3; ++q) out->E[f][q] = mkc(0.0f, 0.0f);
            }
            return d;
        }
    }
    if (rec) {
        creep_prep<dx>(c, rec, Sd, Pd, g, to_df(to_double(g.sp + g.t + g.sq)), enable);
        *n_rec = 1;
    } else if (field) {
        Acc<dx> a;
        acc_zero(a);
        field_creep<dx, dx, true>(c, a, fq, Sd, Pd, g, g.sp + g.t + g.sq, enable);
        contrib_from(out, a);
    }
    return d;
}
// a source image outside body b (a cylinder: off its footprint), FP64
__device__ __forceinline__ bool img_outside(const Ctx &c, int b, v3t<dx> X) {
    const float4 q0 = c.body[2 * b], q1 = c.body[2 * b + 1];
    const dx ex = X.x - dx((double)q0.x), ey = X.y - dx((double)q0.y);
    const dx ez = (q1.y == 0.0f) ? X.z - dx((double)q0.z) : dx(0.0);
    return Sqrt(ex * ex + ey * ey + ez * ez) > dx((double)q0.w);
}
// the source's image in face wf: FP32 (hi) and FP64 (hi + lo)
__device__ __forceinline__ v3t<float> wall_img_f(const Ctx &c, int wf) {
    const float4 h = c.img[2 * wf];
    return mk3(h.x, h.y, h.z);
}
__device__ __forceinline__ v3t<dx> wall_img_d(const Ctx &c, int wf) {
    const float4 h = c.img[2 * wf], l = c.img[2 * wf + 1];
    return mk3<dx>(dx((double)h.x + (double)l.x), dx((double)h.y + (double)l.y), dx((double)h.z + (double)l.z));
}
// wall -> creeping candidate decided, its caustic flag taken, and (field)
// evaluated in FP64, or its records written (rec)
__device__ __noinline__ int esc_wcreep(const Ctx &c, int wf, int b, int dir, v3t<float> Pf, const FreqC &fq,
                                       bool field, double half_lambda_max, unsigned enable, Contrib *out,
                                       int *caustic, float *rec, int *n_rec) {
    Geo<dx> g;
    const v3t<dx> Sd = dxv(c.S), Pd = dxv(Pf), Sw = wall_img_d(c, wf);
    *caustic = 0;
    *n_rec = 0;
    if (!img_outside(c, b, Sw)) return D_NO;
    Frame<dx> F;
    body_frame(c, b, Sw, Pd, dx(0.0), F);
    int d = (F.dec == D_NO) ? D_NO : cand_creep<dx, false>(c, b, dir, Sw, Pd, dx(0.0), F, g);
    if (d == D_YES) d = wall_legs<dx>(c, wf, b, Sd, Sw, g.Q1, dx(0.0));
    if (d != D_YES) return d;
    if (c.body[2 * b + 1].y == 0.0f) {
        *caustic = half_lambda_max > g.dperp.v;
        if (!(g.dperp > dx(0.0))) {                  // exactly on the axis: no finite ray field
            if (field) {
                for (int f = 0; f < NFC; ++f)
                    for (int q = 0; q < 3; ++q) out->E[f][q] = mkc(0.0f, 0.0f);
            }
            return d;
        }
    }
    if (rec) {
        *n_rec = wcreep_prep(c, rec, wf, c.S, wall_img_f(c, wf), Pf, to_f(g), to_df(to_double(g.sp + g.t + g.sq)),
                             enable);
    } else if (field) {
        Acc<dx> a;
        acc_zero(a);
        field_wcreep<dx, dx, true>(c, a, fq, wf, Sd, Sw, Pd, g, g.sp + g.t + g.sq, enable);
        contrib_from(out, a);
    }
    return d;
}

// ------------------------------------------------------------------ kernel
// Path classes; one launch evaluates the classes of its CLS mask, so that each
// kernel carries only the code (and the live registers) of its classes.
enum { CLS_PLANAR = 1,        // direct ray and planar image reflections
       CLS_BODYREFL = 2,      // GO reflection off each curved body
       CLS_CREEP = 4,         // creeping rays round each curved body
       CLS_WCREEP = 8,        // creeping rays fed by a planar reflection (a work unit: face x body)
       CLS_SEQ = 16 };        // direct ray and the planar paths of the candidate list (large scenes)
constexpr bool is_planar(int cls) { return cls == CLS_PLANAR || cls == CLS_SEQ; }
constexpr int CLS_BODIES = CLS_BODYREFL | CLS_CREEP | CLS_WCREEP;
// Block shape.  The body classes run one block of 12 warps per SM: three
// tiles at a time, four warps per tile; a block barrier between the geometry
// pass and the field pass keeps all warps of the SM in the same pass, so the
// instruction cache holds one pass's code at a time.  The planar class, and
// the FP64 path, run 4-warp blocks, several per SM.
constexpr int blk_of(int cls, bool fp32) { return ((cls & CLS_BODIES) && fp32) ? 384 : BLOCK; }
constexpr int min_blocks(int cls, bool fp32) {
    return ((cls & CLS_BODIES) && fp32) ? 1 : (is_planar(cls) ? 4 : 3);
}
// records per work unit of a body class (FP32 fields)
constexpr int recs_per_unit(int cls) {
    return ((cls & CLS_CREEP) ? 2 : 0) + ((cls & CLS_BODYREFL) ? 1 : 0) + ((cls & CLS_WCREEP) ? 4 : 0);
}
constexpr int WARPS_PER_TILE = 4;
constexpr int MAX_CHUNKS = (RT_MAX_FREQS + NFC - 1) / NFC;
constexpr int PLANAR_CHUNKS = 4;       // frequency chunks per planar launch (FP32 fields)
constexpr int OCC_MAX_BODIES = 256;    // occluder masks up to this many bodies (FP32 body kernels)

// Field pass over one lane's records for the frequency chunk fq.
template <int CLS>
__device__ __forceinline__ void apply_records(const Ctx &c, AccS<float> &acc, const FreqC &fq, const float *rec,
                                              int nrec) {
    constexpr bool RB = (CLS & CLS_BODYREFL) != 0, CP = (CLS & (CLS_CREEP | CLS_WCREEP)) != 0;
#pragma unroll 1
    for (int j = 0; j < nrec; ++j) {
        const float *r = rec + j * REC_N * 32;
        if (RB && (!CP || r[288] > 0.0f)) rb_apply(c, acc, fq, r);
        else if (CP) creep_apply(c, acc, fq, r);
    }
}

// One receiver P = rx[r]: the paths of the classes in CLS among the
// candidates of share `part` of `nparts` -- the direct ray to share 0, the
// reflection off face i to share (1 + i) mod nparts, off faces (i, j) to
// share (1 + i n_face + j) mod nparts, the paths of body b to share
// b mod nparts -- summed into acc; the receiver's flags, the count of FP64
// re-decisions and (PATHS) the path codes from slot npath on.
// ---- candidate-list culling per tile.  A candidate (face sequence) can give
// a path to receiver P only if P and the source's last image lie strictly on
// opposite sides of the last face's plane and the last reflection point --
// where the segment image -> P crosses the plane -- lies on that face.  For a
// box holding the tile's receivers, both fail for every receiver at once if
// all eight corners lie on the image's side by more than twice the decision
// band, or, with all corners on the far side, if the box of the corners'
// crossing points misses the face's box (DevScene::face_box): the crossing
// points of the whole box lie in the hull of the corners' (the central
// projection keeps convexity on that half-space), and the face box is grown
// so that a point outside it is outside every triangle of the face by more
// than the band.  Such candidates are decided "no" for every receiver of the
// tile by the per-receiver test too (FP32 with its band, or FP64), so
// leaving them out changes no decision and no field.
constexpr int SEQ_MASK_WORDS = 512;      // culling up to 16384 candidates (a larger list is not culled)
__device__ __forceinline__ bool seq_may_hit(const Ctx &c, int q, int4 sq, const float lo[3], const float hi[3]) {
    const int k = sq.w;
    const int f = (k == 1) ? sq.x : ((k == 2) ? sq.y : sq.z);
    const float4 I = c.cimg[6 * q + 2 * (k - 1)];
    const float4 pl = c.face32[f];
    const float di = pl.x * I.x + pl.y * I.y + pl.z * I.z - pl.w;
    const float m = 2.0f * c.band;
    if (!(fabsf(di) > m)) return true;
    const float sg = di > 0.0f ? 1.0f : -1.0f;
    bool same = true, opp = true;
    float qlo[3] = {INFINITY, INFINITY, INFINITY}, qhi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
        const float px = (cc & 1) ? hi[0] : lo[0], py = (cc & 2) ? hi[1] : lo[1], pz = (cc & 4) ? hi[2] : lo[2];
        const float dp = pl.x * px + pl.y * py + pl.z * pz - pl.w;
        same = same && (dp * sg > m);
        opp = opp && (-dp * sg > m);
        const float t = di / (di - dp);
        const float x = I.x + (px - I.x) * t, y = I.y + (py - I.y) * t, z = I.z + (pz - I.z) * t;
        qlo[0] = fminf(qlo[0], x); qhi[0] = fmaxf(qhi[0], x);
        qlo[1] = fminf(qlo[1], y); qhi[1] = fmaxf(qhi[1], y);
        qlo[2] = fminf(qlo[2], z); qhi[2] = fmaxf(qhi[2], z);
    }
    if (same) return false;
    if (!opp) return true;
    const float4 b0 = c.face_box[2 * f], b1 = c.face_box[2 * f + 1];
    return qlo[0] <= b1.x && qhi[0] >= b0.x && qlo[1] <= b1.y && qhi[1] >= b0.y && qlo[2] <= b1.z && qhi[2] >= b0.z;
}
// All 32 lanes of a warp: the box of the tile's receivers (lanes with ok),
// then bit lane of word w set iff candidate 32 w + lane is in share part of
// nparts, within max_order, and not culled.  Returns false (no mask) when
// the list is too long to be culled.
__device__ __noinline__ bool seq_tile_mask(const Ctx &c, const float *rx, int n_rx, int r, bool ok, int part,
                                           int nparts, int max_order, uint32_t *mask) {
    if (c.n_cand > 32 * SEQ_MASK_WORDS) return false;
    const int lane = threadIdx.x & 31;
    float lo[3], hi[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float v = ok ? rx[k * n_rx + r] : 0.0f;
        lo[k] = ok ? v : INFINITY;
        hi[k] = ok ? v : -INFINITY;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
    }
    const int nw = (c.n_cand + 31) >> 5;
    for (int w = 0; w < nw; ++w) {
        const int q = 32 * w + lane;
        bool keep = false;
        if (q < c.n_cand && (1 + q) % nparts == part && lo[0] <= hi[0]) {
            const int4 sq = c.cand[q];
            if (sq.w <= max_order) keep = seq_may_hit(c, q, sq, lo, hi);
        }
        const unsigned word = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) mask[w] = word;
    }
    __syncwarp();
    return true;
}

// fields with the path list: the warps sharing a receiver take slots by
// atomics (the list is in no particular order); returns the overflow flag
__device__ __noinline__ uint32_t list_path(uint64_t *codes, int32_t *counts, int cap, int r, uint64_t code) {
    const int slot = atomicAdd(&counts[r], 1);
    if (slot < cap) {
        codes[(size_t)r * cap + slot] = code;
        return 0u;
    }
    return RT_FLAG_OVERFLOW;
}

template <typename T, bool PATHS, int CLS, bool LIST = false>
__device__ __forceinline__ void eval_receiver(const Ctx &c, const FreqC *fqs, int nfq, unsigned enable, int max_order,
                                              const float *__restrict__ rx, int n_rx, int r,
                                              uint64_t *__restrict__ codes, int32_t *__restrict__ counts, int cap,
                                              double half_lambda_max,
                                              int b_begin, int b_end, bool first_chunk, bool may_flush, int rcap,
                                              const uint32_t *occ_rx, int part, int nparts,
                                              AccS<T> acc, float *rec, uint32_t &fl, unsigned &nesc, int &npath,
                                              int &nrec_out, const uint32_t *qmask = nullptr, unsigned lanes = 0u,
                                              uint32_t *pwm = nullptr) {
    constexpr bool BODIES = (CLS & CLS_BODIES) != 0;
    const bool fp32 = sizeof(T) == 4;
    const T band = fp32 ? T(c.band) : T(0);
    // fqs[0]: the frequency chunk of the body classes' fields; the planar
    // rays take all nfq chunks (each with its own partial sums)
    const FreqC &fq = fqs[0];
    const int nf = fq.nf;
    v3t<float> Pf = mk3(rx[r], rx[n_rx + r], rx[2 * n_rx + r]);
    v3t<T> P = mk3<T>(T((double)Pf.x), T((double)Pf.y), T((double)Pf.z));
    v3t<T> Sx = mk3<T>(T((double)c.S.x), T((double)c.S.y), T((double)c.S.z));
    fl = 0;
    nesc = 0;
    nrec_out = 0;
    if (!PATHS) acc_zero_rows(acc, nfq * NFC * 6);
    typedef typename LenOf<T>::type LT;

    auto emit = [&](int type, int a, int b) {
        if (PATHS) {
            if (npath < cap) codes[(size_t)r * cap + npath] = pcode(type, a, b);
            else fl |= RT_FLAG_OVERFLOW;
        } else if constexpr (LIST) {
            fl |= list_path(codes, counts, cap, r, pcode(type, a, b));
        }
        ++npath;
    };
    auto escalated = [&]() {
        fl |= RT_FLAG_ESCALATED;
        ++nesc;
    };

    // receiver inside (or on) a body?  (every class kernel takes this decision
    // itself; it is the same in each)
    int inside = 0;
    for (int b = 0; b < c.n_body && !inside; ++b) {
        float4 q0 = c.body[2 * b], q1 = c.body[2 * b + 1];
        int d;
        T ex = P.x - T((double)q0.x), ey = P.y - T((double)q0.y), ez = P.z - T((double)q0.z), a = T((double)q0.w);
        if (fp32) {
            T m = (q1.y == 0.0f) ? a - Sqrt(ex * ex + ey * ey + ez * ez)
                                 : Fmin(Fmin(a - Sqrt(ex * ex + ey * ey), P.z - T((double)q0.z)),
                                        T((double)q0.z) + T((double)q1.x) - P.z);
            d = decide(m, band, D_YES);
            if (d == D_UNSURE) {
                if (part == 0 && first_chunk) escalated();   // every share and chunk takes it; one counts it
                else fl |= RT_FLAG_ESCALATED;
                d = esc_inside(c, b, Pf);
            }
        } else {
            d = esc_inside(c, b, Pf);
        }
        inside = (d == D_YES);
    }

    // planar occluder masks (FP32 fields, enumeration): the lanes `lanes`
    // (every lane of the warp that evaluates a receiver) share them; pnw mask
    // words per leg, 0 without masks
    constexpr bool PM = sizeof(T) == 4 && !PATHS && CLS == CLS_PLANAR;
    unsigned pl = 0u;
    int pnw = 0;
    float tcx = 0.0f, tcy = 0.0f, tcr = 0.0f;
    if constexpr (PM) {
        if (pwm && lanes && c.n_body > 0 && c.n_body <= OCC_MAX_BODIES) {
            pl = __ballot_sync(lanes, !inside);
            if (pl) {
                pnw = (c.n_body + 31) >> 5;
                if (!inside) lanes_box(pl, true, Pf.x, Pf.y, tcx, tcy, tcr);
            }
        }
    }
    if (inside) {
        fl |= RT_FLAG_INSIDE;
    } else {
        if constexpr ((CLS & (CLS_PLANAR | CLS_SEQ)) != 0) {
            // ---- direct ray (candidate 0)
            if ((enable & RT_EN_LOS) && part == 0) {
                int d = cand_los<T>(c, Sx, P, band);
                if (d == D_UNSURE) { escalated(); d = esc_los(c, Pf); }
                if (d == D_YES) {
                    emit(PT_LOS, 0, 0);
                    if (!PATHS) {
                        LT L = seglen(Sx, P);
                        add_ray_chunks(acc, fqs, nfq, src_pol(c, unit3(P - Sx)), T(1) / (T)len_val(L), L);
                    }
                }
            }
            // ---- planar image reflections: the candidate sequences (large
            // scenes), else every face and ordered face pair
            if constexpr (CLS == CLS_SEQ) {
              if ((enable & RT_EN_PLANAR) && max_order >= 1) {
                // the tile's mask (seq_tile_mask) lists this share's candidates
                // that survive culling; without one, every candidate of the share
                int w = 0, q = -1;
                uint32_t word = qmask ? qmask[0] : 0u;
                const int nw = (c.n_cand + 31) >> 5;
#pragma unroll 1
                for (;;) {
                    if (qmask) {
                        while (word == 0u && ++w < nw) word = qmask[w];
                        if (word == 0u) break;
                        q = 32 * w + __ffs(word) - 1;
                        word &= word - 1u;
                    } else {
                        if (++q >= c.n_cand) break;
                        if ((1 + q) % nparts != part) continue;
                    }
                    const int4 sq = c.cand[q];
                    if (sq.w > max_order) continue;
                    v3t<T> Q[3];
                    int d = cand_seq<T>(c, q, sq, Sx, P, band, Q);
                    if constexpr (sizeof(T) == 4) {
                        if (d == D_UNSURE) { escalated(); d = esc_seq(c, q, sq, Pf, Q); }
                    }
                    if (d != D_YES) continue;
                    if (sq.w == 1) emit(PT_R1, sq.x, 0);
                    else if (sq.w == 2) emit(PT_R2, sq.x, sq.y);
                    else emit(PT_R3, q, 0);
                    if (!PATHS) {
                        LT L;
                        if constexpr (sizeof(T) == 4) {
                            L = df_dist_df(c.cimg[6 * q + 2 * (sq.w - 1)], c.cimg[6 * q + 2 * (sq.w - 1) + 1], Pf);
                        } else {
                            L = seglen(Sx, Q[0]);
                            for (int m = 0; m + 1 < sq.w; ++m) L = ladd(L, seglen(Q[m], Q[m + 1]));
                            L = ladd(L, seglen(Q[sq.w - 1], P));
                        }
                        add_seq_field(c, acc, fqs, nfq, Sx, Q, P, sq, T(1) / (T)len_val(L), L);
                    }
                }
              }
            } else {
            if ((enable & RT_EN_PLANAR) && max_order >= 1) {
#pragma unroll 1
                for (int i = 0; i < c.n_face; ++i) {
                    if ((1 + i) % nparts != part) continue;      // candidates 1 .. n_face
                    Geo<T> g;
                    int d;
                    if constexpr (PM) {
                        if (pnw) {
                            d = cand_r1_geo<T>(c, i, Sx, P, band, g);
                            const bool v = d != D_NO;
                            float qx, qy, qr;
                            lanes_box(pl, v, g.Q1.x, g.Q1.y, qx, qy, qr);
                            if (qr < 0.0f) continue;                 // (no lane: the whole warp)
                            const float cx[3] = {c.S.x, qx, tcx}, cy[3] = {c.S.y, qy, tcy}, cr[3] = {0.0f, qr, tcr};
                            leg_masks<2>(c, pl, cx, cy, cr, pwm, pnw);
                            if (v) d = cand_r1_vis(c, i, Sx, P, band, g, d, pwm, pnw);
                        } else {
                            d = cand_r1<T>(c, i, Sx, P, band, g);
                        }
                    } else {
                        d = cand_r1<T>(c, i, Sx, P, band, g);
                    }
                    if constexpr (sizeof(T) == 4) {
                        if (d == D_UNSURE) { escalated(); d = esc_r1(c, i, Pf, &g.Q1); }
                    }
                    if (d == D_YES) {
                        emit(PT_R1, i, 0);
                        if (!PATHS) {
                            v3t<T> ni; T di;
                            face_plane<T>(c, i, &ni, &di);
                            LT L;
                            if constexpr (sizeof(T) == 4) L = df_dist_df(c.img[2 * i], c.img[2 * i + 1], Pf);
                            else L = ladd(seglen(Sx, g.Q1), seglen(g.Q1, P));
                            if (dielectric(c, i))
                                add_planar_dielectric(c, acc, fqs, nfq, Sx, g.Q1, g.Q1, P, i, -1,
                                                      T(1) / (T)len_val(L), L);
                            else
                                add_ray_chunks(acc, fqs, nfq, pec_mirror(src_pol(c, unit3(g.Q1 - Sx)), ni),
                                               T(1) / (T)len_val(L), L);
                        }
                    }
                }
            }
            if ((enable & RT_EN_PLANAR) && max_order >= 2) {
#pragma unroll 1
                for (int i = 0; i < c.n_face; ++i) {
#pragma unroll 1
                    for (int j = 0; j < c.n_face; ++j) {
                        if (j == i) continue;
                        if ((1 + i * c.n_face + j) % nparts != part) continue;   // then the ordered pairs
                        Geo<T> g;
                        int d;
                        if constexpr (PM) {
                            if (pnw) {
                                d = cand_r2_geo<T>(c, i, j, Sx, P, band, g);
                                const bool v = d != D_NO;
                                float ax, ay, ar, bx, by, br;
                                lanes_box(pl, v, g.Q1.x, g.Q1.y, ax, ay, ar);
                                lanes_box(pl, v, g.Q2.x, g.Q2.y, bx, by, br);
                                if (ar < 0.0f) continue;             // (no lane: the whole warp)
                                const float cx[4] = {c.S.x, ax, bx, tcx}, cy[4] = {c.S.y, ay, by, tcy},
                                            cr[4] = {0.0f, ar, br, tcr};
                                leg_masks<3>(c, pl, cx, cy, cr, pwm, pnw);
                                if (v) d = cand_r2_vis(c, i, j, Sx, P, band, g, d, pwm, pnw);
                            } else {
                                d = cand_r2<T>(c, i, j, Sx, P, band, g);
                            }
                        } else {
                            d = cand_r2<T>(c, i, j, Sx, P, band, g);
                        }
                        if constexpr (sizeof(T) == 4) {
                            if (d == D_UNSURE) { escalated(); d = esc_r2(c, i, j, Pf, &g.Q1, &g.Q2); }
                        }
                        if (d == D_YES) {
                            emit(PT_R2, i, j);
                            if (!PATHS) {
                                v3t<T> ni, nj; T di, dj;
                                face_plane<T>(c, i, &ni, &di);
                                face_plane<T>(c, j, &nj, &dj);
                                LT L;
                                if constexpr (sizeof(T) == 4) {
                                    int slot = c.n_face + i * c.n_face + j;
                                    L = df_dist_df(c.img[2 * slot], c.img[2 * slot + 1], Pf);
                                } else {
                                    L = ladd(ladd(seglen(Sx, g.Q1), seglen(g.Q1, g.Q2)), seglen(g.Q2, P));
                                }
                                if (dielectric(c, i) || dielectric(c, j)) {
                                    add_planar_dielectric(c, acc, fqs, nfq, Sx, g.Q1, g.Q2, P, i, j,
                                                          T(1) / (T)len_val(L), L);
                                } else {
                                    v3t<T> e = pec_mirror(pec_mirror(src_pol(c, unit3(g.Q1 - Sx)), ni), nj);
                                    add_ray_chunks(acc, fqs, nfq, e, T(1) / (T)len_val(L), L);
                                }
                            }
                        }
                    }
                }
            }
            }   // enumeration
        }
        // ---- curved bodies b_begin .. b_end - 1 (this share: every nparts-th)
        if constexpr (BODIES) {
            // FP32 fields: the geometry pass writes a record per valid path
            // (candidates decided in FP64 as tagged records too); the caller
            // turns them into fields, frequency chunk by frequency chunk, after
            // a block barrier.  The body range is sized so that the records fit.
            constexpr bool RECS = (sizeof(T) == 4) && !PATHS;
            constexpr int PER = recs_per_unit(CLS);
            int nrec = 0;
#pragma unroll 1
            for (int b = b_begin + part; b < b_end; b += nparts) {
                if constexpr (RECS) {
                    // one frequency chunk: records that could overflow are turned
                    // into fields here (with several chunks the caller sizes the
                    // body range so that they cannot)
                    if (may_flush && nrec > rcap - PER) {
                        apply_records<CLS>(c, acc, fq, rec, nrec);
                        nrec = 0;
                    }
                }
                if constexpr (CLS == CLS_WCREEP) {
                    // unit b: face wf, body bb; the creeping rays of the
                    // source's image in face wf, fed by the reflection there
                    if (!(enable & (RT_EN_CREEP_SOFT | RT_EN_CREEP_HARD))) continue;
                    const int wf = b / c.n_body, bb = b - wf * c.n_body;
                    const bool sphere = c.body[2 * bb + 1].y == 0.0f;
                    Frame<T> F;
                    v3t<T> Sw;
                    if constexpr (sizeof(T) == 4) {
                        Sw = wall_img_f(c, wf);
                        body_frame_tb(c, c.txw + 2 * (size_t)wf * c.n_body, bb, Sw, P, band, F);
                    } else {
                        Sw = wall_img_d(c, wf);
                        if (!img_outside(c, bb, Sw)) continue;
                        body_frame(c, bb, Sw, P, band, F);
                    }
#pragma unroll 1
                    for (int dir = 0; dir < 2; ++dir) {
                        Geo<T> g;
                        int d = cand_creep<T, false>(c, bb, dir, Sw, P, band, F, g);
                        if (d == D_YES) d = wall_legs<T>(c, wf, bb, Sx, Sw, g.Q1, band);
                        int cd = D_NO;
                        if (d == D_YES && sphere) {
                            if constexpr (sizeof(T) == 8) cd = (half_lambda_max > to_double(g.dperp)) ? D_YES : D_NO;
                            else cd = decide((T)half_lambda_max - g.dperp, band, D_NO);
                        }
                        if constexpr (sizeof(T) == 4) {
                            if (d == D_UNSURE || cd == D_UNSURE) {
                                escalated();
                                Contrib ct;
                                int caus = 0, added = 0;
                                const bool defer = RECS;
                                d = esc_wcreep(c, wf, bb, dir, Pf, fq, !PATHS && !defer, half_lambda_max, enable, &ct,
                                               &caus, defer ? rec + nrec * REC_N * 32 : nullptr, &added);
                                if (d == D_YES) {
                                    emit(dir == 0 ? PT_WCP : PT_WCM, bb, 16 * wf + c.enc);
                                    if (caus) fl |= RT_FLAG_CAUSTIC;
                                    if (defer) nrec += added;
                                    else if (!PATHS) acc_add(acc, ct, nf);
                                }
                                continue;
                            }
                        }
                        if (d != D_YES) continue;
                        emit(dir == 0 ? PT_WCP : PT_WCM, bb, 16 * wf + c.enc);
                        if (sphere) {
                            if (cd == D_YES) fl |= RT_FLAG_CAUSTIC;
                            if (!(g.dperp > T(0.0))) continue;        // exactly on the axis: no finite ray field
                        }
                        if constexpr (RECS) {
                            nrec += wcreep_prep(c, rec + nrec * REC_N * 32, wf, Sx, Sw, P, g,
                                                creep_len(c, bb, Sw, P, g, F), enable);
                        } else if constexpr (!PATHS) {
                            field_wcreep<T>(c, acc, fq, wf, Sx, Sw, P, g, creep_len(c, bb, Sw, P, g, F), enable);
                        }
                    }
                    continue;
                }
                Frame<T> F;
                body_frame(c, b, Sx, P, band, F);
                if constexpr ((CLS & CLS_BODYREFL) != 0) {
                    if (enable & RT_EN_BODYREFL) {
                        Geo<T> g;
                        int d = cand_rb<T>(c, b, Sx, P, band, F, g, occ_rx);
                        if constexpr (sizeof(T) == 4) {
                            if (d == D_UNSURE) {
                                // decided in FP64, and its geometry, length and amplitude
                                // too (they may be ill-conditioned in FP32, e.g. for a
                                // receiver at a surface); its record holds them, and the
                                // FP32 field pass evaluates it with the others
                                escalated();
                                Contrib ct;
                                const bool defer = RECS;
                                d = esc_rb(c, b, Pf, fq, !PATHS && !defer, &ct,
                                           defer ? rec + nrec * REC_N * 32 : nullptr);
                                if (d == D_YES) {
                                    emit(PT_RB, b, 0);
                                    if (defer) ++nrec;
                                    else if (!PATHS) acc_add(acc, ct, nf);
                                }
                                d = D_NO;
                            }
                        }
                        if (d == D_YES) {
                            emit(PT_RB, b, 0);
                            if constexpr (RECS) {
                                rb_prep(c, rec + (nrec++) * REC_N * 32, Sx, g, g.Lf);
                            } else if constexpr (!PATHS) {
                                field_body_refl<T>(c, acc, fq, Sx, P, g, ladd(seglen(Sx, g.Q1), seglen(g.Q1, P)));
                            }
                        }
                    }
                }
                if constexpr ((CLS & CLS_CREEP) != 0) {
                    if (enable & (RT_EN_CREEP_SOFT | RT_EN_CREEP_HARD)) {
                        bool sphere = c.body[2 * b + 1].y == 0.0f;
#pragma unroll 1
                        for (int dir = 0; dir < 2; ++dir) {
                            Geo<T> g;
                            int d = cand_creep<T>(c, b, dir, Sx, P, band, F, g, occ_rx);
                            int cd = D_NO;
                            if (d == D_YES && sphere) {
                                // axial caustic flag: k d_perp < pi for some frequency, i.e. d_perp < lambda_max / 2
                                if constexpr (sizeof(T) == 8) cd = (half_lambda_max > to_double(g.dperp)) ? D_YES : D_NO;
                                else cd = decide((T)half_lambda_max - g.dperp, band, D_NO);
                            }
                            if constexpr (sizeof(T) == 4) {
                                if (d == D_UNSURE || cd == D_UNSURE) {
                                    escalated();
                                    Contrib ct;
                                    int caus = 0;
                                    const bool defer = RECS;
                                    int added = 0;
                                    d = esc_creep(c, b, dir, Pf, fq, !PATHS && !defer, half_lambda_max, enable, &ct,
                                                  &caus, defer ? rec + nrec * REC_N * 32 : nullptr, &added);
                                    if (d == D_YES) {
                                        emit(dir == 0 ? PT_CP : PT_CM, b, c.enc);
                                        if (caus) fl |= RT_FLAG_CAUSTIC;
                                        if (defer) nrec += added;
                                        else if (!PATHS) acc_add(acc, ct, nf);
                                    }
                                    continue;
                                }
                            }
                            if (d != D_YES) continue;
                            emit(dir == 0 ? PT_CP : PT_CM, b, c.enc);
                            if (sphere) {
                                if (cd == D_YES) fl |= RT_FLAG_CAUSTIC;
                                if (!(g.dperp > T(0.0))) continue;        // exactly on the axis: no finite ray field
                            }
                            if constexpr (RECS) {
                                creep_prep(c, rec + (nrec++) * REC_N * 32, Sx, P, g, creep_len(c, b, Sx, P, g, F), enable);
                            } else if constexpr (!PATHS) {
                                field_creep<T>(c, acc, fq, Sx, P, g, creep_len(c, b, Sx, P, g, F), enable);
                            }
                        }
                    }
                }
            }
            nrec_out = nrec;
        }
    }
}

// ---- occluder masks.  A leg of a body path runs between a point of body b
// and the source or a receiver; in projection on the floor it lies in the
// convex hull of body b's disk (centre c_b, radius a_b) and of that end's
// region R, here a disk of radius rr round a segment T0 T1.  That hull lies
// within the triangle (T0, T1, c_b) grown by max(rr, a_b), so a body j whose
// disk (grown by the band and a margin for the FP32 arithmetic of this test)
// misses it cannot pass the distance test of the visibility loop for any
// such leg (projection shortens distances), and is left out of the mask.
// squared distance from p to the triangle (a, b, c); 0 inside or degenerate
__device__ __forceinline__ float tri_d2(float px, float py, float ax, float ay, float bx, float by, float cx,
                                        float cy) {
    const float d1 = (bx - ax) * (py - ay) - (by - ay) * (px - ax);
    const float d2 = (cx - bx) * (py - by) - (cy - by) * (px - bx);
    const float d3 = (ax - cx) * (py - cy) - (ay - cy) * (px - cx);
    const bool neg = d1 < 0.0f || d2 < 0.0f || d3 < 0.0f, pos = d1 > 0.0f || d2 > 0.0f || d3 > 0.0f;
    if (!(neg && pos)) return 0.0f;
    return fminf(seg_d2(px, py, ax, ay, bx, by), fminf(seg_d2(px, py, bx, by, cx, cy), seg_d2(px, py, cx, cy, ax, ay)));
}
// masks of every body for the region (T0, T1, rr): out[b * occ_w + w]; the
// calling warp (index wi of nwarps that share the work) takes bodies wi,
// wi + nwarps, ...; every lane of the warp takes part
__device__ __noinline__ void occ_masks(const Ctx &c, float t0x, float t0y, float t1x, float t1y, float rr, uint32_t *out, int wi,
                          int nwarps) {
    const int lane = threadIdx.x & 31, nb = c.n_body;
    const float margin = 1e-3f + 8.0f * c.band;
#pragma unroll 1
    for (int b = wi; b < nb; b += nwarps) {
        const float4 qb = c.body[2 * b];
        const float rad = fmaxf(rr, qb.w) + c.band + margin;
#pragma unroll 1
        for (int w = 0; w < c.occ_w; ++w) {
            const int j = 32 * w + lane;
            bool hit = false;
            if (j < nb && j != b) {
                const float4 qj = c.body[2 * j];
                const float lim = rad + qj.w;
                hit = tri_d2(qj.x, qj.y, t0x, t0y, t1x, t1y, qb.x, qb.y) <= lim * lim;
            }
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (lane == 0) out[b * c.occ_w + w] = m;
        }
    }
}

// the occluder masks of a tile's receivers: their bounding box as a disk of
// radius rr round the box's longer midline T0 T1; every lane of the warp
// takes part (rok: this lane's receiver exists)
__device__ __forceinline__ void tile_masks(const Ctx &c, const float *rx, int n_rx, int r, bool rok, uint32_t *out,
                                           int wi, int nwarps) {
    float x0 = rok ? rx[r] : INFINITY, y0 = rok ? rx[n_rx + r] : INFINITY;
    float x1 = rok ? x0 : -INFINITY, y1 = rok ? y0 : -INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x0 = fminf(x0, __shfl_xor_sync(0xffffffffu, x0, o));
        y0 = fminf(y0, __shfl_xor_sync(0xffffffffu, y0, o));
        x1 = fmaxf(x1, __shfl_xor_sync(0xffffffffu, x1, o));
        y1 = fmaxf(y1, __shfl_xor_sync(0xffffffffu, y1, o));
    }
    if (x0 <= x1) {
        const float xm = 0.5f * (x0 + x1), ym = 0.5f * (y0 + y1);
        const bool along_x = (x1 - x0) >= (y1 - y0);
        // (half the shorter side, rounded up by a relative 1e-6 for the midpoint's rounding)
        const float rr = (along_x ? 0.5f * (y1 - y0) : 0.5f * (x1 - x0)) * 1.000001f;
        occ_masks(c, along_x ? x0 : xm, along_x ? ym : y0, along_x ? x1 : xm, along_x ? ym : y1, rr, out, wi,
                  nwarps);
    }
}

// copy n bytes (a multiple of 4) from global to shared memory, all threads
__device__ __forceinline__ void stage_words(void *dst, const void *src, int n) {
    for (int i = threadIdx.x; i < n / 4; i += blockDim.x)
        static_cast<uint32_t *>(dst)[i] = static_cast<const uint32_t *>(src)[i];
}

template <typename T, bool PATHS, int CLS, bool LIST = false>
__global__ void __launch_bounds__(blk_of(CLS, sizeof(T) == 4), min_blocks(CLS, sizeof(T) == 4))
k_eval(DevScene S, FrameDev F1, const FrameDev *__restrict__ frames, int n_frames, unsigned long long n_tiles,
       const float *__restrict__ rx_base, const int32_t *__restrict__ perm, float *__restrict__ e_base,
       uint32_t *__restrict__ fl_base,
       uint64_t *__restrict__ codes, int32_t *__restrict__ counts, int cap, int ch0, int nch, int rcap,
       int nwt, int accumulate, int enc, unsigned long long *esc_counter, unsigned long long *queue) {
    constexpr bool BODIES = (CLS & CLS_BODIES) != 0;
    extern __shared__ float4 smem[];
    __shared__ Ctx s_ctx;
    __shared__ FreqC s_fqs[MAX_CHUNKS];        // frequency chunks ch0 .. ch0 + nch - 1
    // stage scene (and, for the body classes, the Fock--Pekeris table)
    const int n_fock = BODIES ? (FOCK_N + FOCK_NP) * 2 : 0, n_res = BODIES ? FOCK_NRES * 2 : 0;
    float4 *s_fock = smem;                                   // n_fock
    float4 *s_res = s_fock + n_fock;                         // n_res
    float4 *s_face = s_res + n_res;                          // n_face
    bool body_sm = S.n_body <= SMEM_BODY_MAX;
    const bool face_sm = S.n_face <= SMEM_FACE_MAX;
    float4 *s_body = s_face + (face_sm ? S.n_face : 0);      // n_body * 2 (if staged)
    bool tri_sm = S.n_tri <= SMEM_TRI_MAX;
    float4 *s_tri = s_body + (body_sm ? 2 * S.n_body : 0);   // n_tri * 3 (if staged)
    float4 *s_aux = s_tri + (tri_sm ? 3 * S.n_tri : 0);      // n_tri * 3 (if staged)
    float4 *s_txb = s_aux + (tri_sm ? 3 * S.n_tri : 0);      // n_body * 2 (if staged)
    const int n_top = S.bvh ? min(S.bvh_nodes, BVH_TOP_NODES) : 0;
    float4 *s_bvh = s_txb + (body_sm ? 2 * S.n_body : 0);    // n_top * 2: the BVH's top treelet
    float *s_weid = (float *)(s_bvh + 2 * n_top);
    float *s_rec = s_weid + WEIDEMAN_N;                      // path records (FP32 fields of the body classes)
    for (int i = threadIdx.x; i < 2 * n_top; i += blockDim.x) s_bvh[i] = S.bvh[i];
    for (int i = threadIdx.x; i < n_fock; i += blockDim.x) s_fock[i] = S.fock32[i];
    for (int i = threadIdx.x; i < n_res; i += blockDim.x) s_res[i] = S.res32[i];
    if (face_sm)
        for (int i = threadIdx.x; i < S.n_face; i += blockDim.x) s_face[i] = S.face32[i];
    // the frame's bodies, source-side body frames and frequency chunks (one
    // frame: F1; a batch: staged again whenever the block's next work unit is
    // in another frame)
    if (!frames) stage_words(s_fqs, F1.fqc + ch0, nch * sizeof(FreqC));
    if (body_sm && !frames)
        for (int i = threadIdx.x; i < 2 * F1.n_body; i += blockDim.x) {
            s_body[i] = F1.body[i];
            s_txb[i] = F1.txb[i];
        }
    if (tri_sm)
        for (int i = threadIdx.x; i < 3 * S.n_tri; i += blockDim.x) {
            s_tri[i] = S.tri[i];
            s_aux[i] = S.tri_alt[i];
        }
    if (BODIES)
        for (int i = threadIdx.x; i < WEIDEMAN_N; i += blockDim.x) s_weid[i] = S.weid[i];
    if (threadIdx.x == 0) {
        Ctx &c = s_ctx;
        c.tri = tri_sm ? s_tri : S.tri;
        c.tri_aux = tri_sm ? s_aux : S.tri_alt;
        c.face32 = face_sm ? s_face : S.face32;
        c.face64 = S.face64;
        c.face_rng = S.face_rng;
        c.face_tris = S.face_tris;
        c.face_box = S.face_box;
        c.body = body_sm ? s_body : F1.body;
        c.n_tri = S.n_tri; c.n_face = S.n_face; c.n_body = frames ? 0 : F1.n_body;
        c.band = S.band_len;
        c.S = mk3(S.tx[0], S.tx[1], S.tx[2]);
        c.pol = mk3(S.pol[0], S.pol[1], S.pol[2]);
        c.fock = s_fock; c.res = s_res; c.weid = s_weid; c.weid_L = S.weid_L;
        c.fock64 = S.fock64; c.res64 = S.res64; c.weid64 = S.weid64;
        c.img = S.img;
        c.img_pairs = S.img_pairs;
        c.face_mat = S.face_mat;
        c.txb = body_sm ? s_txb : F1.txb;
        c.occ_src = nullptr;
        c.occ_w = 0;
        c.enc = enc;
        c.txw = frames ? nullptr : S.txw;
        c.bvh = S.bvh; c.bvh_tri = S.bvh_tri;
        c.bvh_top = s_bvh; c.bvh_top_n = n_top;
        c.cand = S.cand; c.cimg = S.cimg;
        c.n_cand = S.cand ? (S.n_cand_dev ? *S.n_cand_dev : S.n_cand) : 0;
    }
    __syncthreads();
    // the next class kernel (launched as a programmatic dependent) may start
    // on SMs this grid leaves idle; it waits for this grid to complete before
    // it first touches the outputs (griddepcontrol.wait below)
    asm volatile("griddepcontrol.launch_dependents;");

    const Ctx &c = s_ctx;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = blk_of(CLS, sizeof(T) == 4) / 32;
    if constexpr (PATHS) {
        // (one frame only)
        const float *rx = rx_base;
        const int n_rx = F1.n_rx;
        const unsigned long long ntiles = ((unsigned long long)n_rx + 31ull) >> 5;
        // occluder masks (FP32 body kernels): the source side per block, the
        // receiver side per warp (each warp takes whole tiles)
        constexpr bool OCC = BODIES && sizeof(T) == 4 && CLS != CLS_WCREEP;
        const bool occ_on = OCC && S.n_body > 0 && S.n_body <= OCC_MAX_BODIES;
        const int occ_w = occ_on ? (S.n_body + 31) >> 5 : 0;
        uint32_t *s_occ_src = reinterpret_cast<uint32_t *>(s_rec);
        uint32_t *s_occ_mine = s_occ_src + (1 + warp) * S.n_body * occ_w;
        if (threadIdx.x == 0) {
            s_ctx.occ_src = occ_on ? s_occ_src : nullptr;
            s_ctx.occ_w = occ_w;
        }
        __syncthreads();
        if (occ_on) {
            occ_masks(c, c.S.x, c.S.y, c.S.x, c.S.y, 0.0f, s_occ_src, warp, NW);
            __syncthreads();
        }
        asm volatile("griddepcontrol.wait;" ::: "memory");   // the previous class kernel's lists are complete
        // path lists: each warp takes tiles of 32 consecutive receivers from
        // the launch's queue and lists every candidate itself (codes in the
        // canonical order)
        __shared__ uint32_t s_qmask_p[CLS == CLS_SEQ ? NW : 1][CLS == CLS_SEQ ? SEQ_MASK_WORDS : 1];
        for (;;) {
            unsigned long long t = 0;
            if (lane == 0) t = atomicAdd(queue, 1ull);
            t = __shfl_sync(0xffffffffu, t, 0);
            if (t >= ntiles) break;
            int r = (int)(t * 32ull) + lane;
            if (occ_on) {
                tile_masks(c, rx, n_rx, r, r < n_rx, s_occ_mine, 0, 1);
                __syncwarp();
            }
            bool qm_on = false;
            if constexpr (CLS == CLS_SEQ) {
                qm_on = seq_tile_mask(c, rx, n_rx, r < n_rx ? r : n_rx - 1, r < n_rx, 0, 1, S.max_order,
                                      &s_qmask_p[warp][0]);
            }
            if (r < n_rx) {
                AccS<T> acc{nullptr};                // no fields in this mode
                uint32_t fl;
                unsigned nesc;
                int npath = accumulate ? counts[r] : 0;
                int nrec;
                eval_receiver<T, PATHS, CLS, LIST>(c, s_fqs, 1, S.enable, S.max_order, rx, n_rx, r, codes, counts, cap,
                                                   F1.hl,
                                             0, CLS == CLS_WCREEP ? c.n_face * c.n_body : c.n_body, true, false, 0,
                                             occ_on ? s_occ_mine : nullptr, 0, 1, acc,
                                             nullptr, fl, nesc, npath, nrec, qm_on ? &s_qmask_p[warp][0] : nullptr);
                counts[r] = npath;
                if (fl_base) fl_base[r] = accumulate ? (fl_base[r] | fl) : fl;
                if (nesc) atomicAdd(esc_counter, (unsigned long long)nesc);
            }
        }
    } else {
        // fields: persistent blocks take tiles of 32 consecutive receivers
        // from the launch's queue, TPB tiles per step; the NWT warps of a
        // tile share its candidates (warp part p takes share p) and the
        // partial fields are summed in shared memory in warp order, so the
        // result does not depend on timing.  Sharing a tile among warps
        // shortens it, so the last tiles of the launch leave little of the GPU
        // idle.  Body classes (FP32): the bodies go in chunks sized for the
        // record buffer; per chunk all warps finish the geometry pass before
        // any starts the field pass, which runs once per frequency chunk on
        // the same records and adds its rows to the outputs.
        //   The tile shape: NWT = nwt warps share a tile (the launcher checks
        // that it divides the block's warps), TPB tiles per block.  A work
        // unit is TPB tiles of one frame; a batch's frames start at tile
        // indices that are multiples of TILE_ALIGN (the launcher checks that
        // TPB divides it), so unit u covers tiles u TPB .. u TPB + TPB - 1.  A
        // block's units come in increasing order, so its frame only moves on.
        const int NWT = nwt;
        const int TPB = NW / NWT;
        constexpr bool RECS = BODIES && sizeof(T) == 4;
        constexpr int PER = recs_per_unit(CLS);
        const unsigned long long n_units = (n_tiles + TPB - 1) / TPB;
        const int grp = warp / NWT, part = warp % NWT;
        // partial sums of each warp: NFC * 6 rows of 32 lanes; the FP32
        // planar kernel ("wide") keeps the rows of all nch chunks at once in
        // the dynamic region (it has no path records), so one geometry pass
        // serves every chunk
        constexpr bool WIDE = is_planar(CLS) && sizeof(T) == 4;
        __shared__ T s_part_st[NW][WIDE ? 1 : NFC * 6][32];
        const int prow = WIDE ? nch * NFC * 6 : NFC * 6;
        T *s_part = WIDE ? reinterpret_cast<T *>(s_rec) : &s_part_st[0][0][0];
        __shared__ uint32_t s_fl[NW][32];
        __shared__ uint32_t s_qmask[CLS == CLS_SEQ ? NW : 1][CLS == CLS_SEQ ? SEQ_MASK_WORDS : 1];
        __shared__ uint32_t s_pwm[CLS == CLS_PLANAR ? NW : 1][CLS == CLS_PLANAR ? 3 * (OCC_MAX_BODIES / 32) : 1];
        __shared__ unsigned long long s_unit;
        __shared__ int s_fi, s_new;
        __shared__ FrameDev s_fr;
        // occluder masks (FP32 body kernels): the source side per frame, the
        // receiver side per tile, after the path records
        constexpr bool OCC = BODIES && sizeof(T) == 4 && CLS != CLS_WCREEP;
        const bool occ_on = OCC && S.n_body > 0 && S.n_body <= OCC_MAX_BODIES;
        const int occ_w = occ_on ? (S.n_body + 31) >> 5 : 0;
        uint32_t *s_occ_src = reinterpret_cast<uint32_t *>(s_rec + (RECS ? NW * rcap * REC_N * 32 : 0));
        uint32_t *s_occ_rx = s_occ_src + S.n_body * occ_w;
        if (threadIdx.x == 0) {
            s_fi = -1;
            if (!frames) s_fr = F1;
            s_ctx.occ_src = occ_on ? s_occ_src : nullptr;
            s_ctx.occ_w = occ_w;
        }
        __syncthreads();
        if (occ_on && !frames) occ_masks(c, c.S.x, c.S.y, c.S.x, c.S.y, 0.0f, s_occ_src, warp, NW);
        for (;;) {
            if (threadIdx.x == 0) {
                const unsigned long long u = atomicAdd(queue, 1ull);
                int fi = 0, nw = 0;
                if (frames && u < n_units) {
                    fi = s_fi < 0 ? 0 : s_fi;
                    while (fi + 1 < n_frames && u * TPB >= frames[fi + 1].tile0) ++fi;
                    nw = fi != s_fi;
                    if (nw) s_fr = frames[fi];
                }
                s_unit = u;
                s_fi = fi;
                s_new = nw;
            }
            __syncthreads();
            if (s_unit >= n_units) break;
            if (s_new) {
                // this unit is the block's first in frame s_fi: stage its data
                if (body_sm)
                    for (int i = threadIdx.x; i < 2 * s_fr.n_body; i += blockDim.x) {
                        s_body[i] = s_fr.body[i];
                        s_txb[i] = s_fr.txb[i];
                    }
                stage_words(s_fqs, s_fr.fqc + ch0, nch * sizeof(FreqC));
                if (threadIdx.x == 0) {
                    s_ctx.body = body_sm ? s_body : s_fr.body;
                    s_ctx.txb = body_sm ? s_txb : s_fr.txb;
                    s_ctx.n_body = s_fr.n_body;
                    s_ctx.band = s_fr.band;
                }
                __syncthreads();
                if (occ_on) {
                    occ_masks(c, c.S.x, c.S.y, c.S.x, c.S.y, 0.0f, s_occ_src, warp, NW);
                    __syncthreads();
                }
            }
            const FrameDev &Fr = s_fr;
            const int n_rx = Fr.n_rx;
            const float *rx = rx_base + 3 * Fr.rx_off;
            float *e_out = e_base + Fr.e_off;
            uint32_t *flags_out = fl_base ? fl_base + Fr.rx_off : nullptr;
            const int n_b = BODIES ? (CLS == CLS_WCREEP ? c.n_face * c.n_body : c.n_body) : 0;
            // bodies per geometry pass: all of them with one frequency chunk (full
            // record buffers are flushed on the way), else as many as the buffer holds
            const int bc = (RECS && nch > 1) ? NWT * (rcap / PER) : (n_b > 0 ? n_b : 1);
            const unsigned long long t = s_unit * TPB - Fr.tile0 + grp;   // tile within the frame
            const long long r0 = (long long)(t * 32ull);
            const int r = r0 < n_rx ? (int)r0 + lane : n_rx;
            const bool rok = r < n_rx;
            if (occ_on) {
                // each warp makes the masks of the bodies of its own share
                // (b = part mod NWT), so no other warp waits for them
                tile_masks(c, rx, n_rx, r, rok, s_occ_rx + grp * S.n_body * occ_w, part, NWT);
                __syncwarp();
            }
            // candidate-list class: this warp's surviving candidates for the tile
            bool qm_on = false;
            if constexpr (CLS == CLS_SEQ) {
                if (n_rx > 0)
                    qm_on = seq_tile_mask(c, rx, n_rx, rok ? r : n_rx - 1, rok, part, NWT, S.max_order, &s_qmask[warp][0]);
            }
            AccS<T> acc{s_part + warp * prow * 32 + lane};     // the warp's partial sums, summed in place
            float *rec = s_rec + warp * (rcap * REC_N * 32) + lane;
            const unsigned lanes = __ballot_sync(0xffffffffu, rok);      // the lanes that evaluate a receiver
#pragma unroll 1
            for (int b0 = 0; b0 < (n_b > 0 ? n_b : 1); b0 += bc) {
                uint32_t fl = 0;
                unsigned nesc = 0;
                int npath = 0, nrec = 0;
                if (rok)
                    eval_receiver<T, PATHS, CLS, LIST>(c, s_fqs, WIDE ? nch : 1, S.enable, S.max_order, rx, n_rx, r,
                                                       codes, counts, cap,
                                                 Fr.hl, b0, min(b0 + bc, n_b), b0 == 0, nch == 1, rcap,
                                                 occ_on ? s_occ_rx + grp * S.n_body * occ_w : nullptr, part,
                                                 NWT, acc, rec, fl, nesc, npath, nrec,
                                                 qm_on ? &s_qmask[warp][0] : nullptr, lanes, &s_pwm[warp][0]);
                s_fl[warp][lane] = fl;
                if (nesc && ch0 == 0) atomicAdd(esc_counter, (unsigned long long)nesc);
#pragma unroll 1
                for (int ch = ch0; ch < ch0 + nch; ++ch) {
                    const FreqC &fqc = s_fqs[ch - ch0];
                    if constexpr (RECS) {
                        __syncthreads();              // geometry pass / previous reduction done
                        if (rok) {
                            if (ch > ch0) acc_zero(acc);      // the geometry pass zeroed it for the first chunk
                            apply_records<CLS>(c, acc, fqc, rec, nrec);
                        }
                    }
                    // the previous class kernel's fields and flags are complete (a
                    // no-op when this grid was not launched as a dependent, and
                    // after its first return)
                    asm volatile("griddepcontrol.wait;" ::: "memory");
                    __syncthreads();
                    // reduce the tile's NWT partials: part p writes the
                    // (frequency, component) pairs j = p, p + NWT, ... of chunk ch
                    if (rok) {
                        const int w0 = grp * NWT, f0 = ch * NFC;
                        const int ro = perm ? perm[Fr.rx_off + r] : r;       // the receiver's output slot
                        const bool add = accumulate || b0 > 0;
                        const T *pp = s_part + (WIDE ? (ch - ch0) * NFC * 6 * 32 : 0) + lane;
                        for (int j = part; j < fqc.nf * 3; j += NWT) {
                            T re = pp[(w0 * prow + 2 * j) * 32], im = pp[(w0 * prow + 2 * j + 1) * 32];
#pragma unroll
                            for (int w = 1; w < NW; ++w) {      // (unrolled to the block's warps, in order)
                                if (w < NWT) {
                                    re = re + pp[((w0 + w) * prow + 2 * j) * 32];
                                    im = im + pp[((w0 + w) * prow + 2 * j + 1) * 32];
                                }
                            }
                            size_t idx = ((size_t)(f0 + j / 3) * 3 + (j % 3)) * n_rx + ro;
                            float2 v;
                            v.x = to_float(re);
                            v.y = to_float(im);
                            if (add) {
                                float2 o = reinterpret_cast<float2 *>(e_out)[idx];
                                v.x += o.x;
                                v.y += o.y;
                            }
                            reinterpret_cast<float2 *>(e_out)[idx] = v;
                        }
                        if (ch == 0 && part == 0 && flags_out) {
                            uint32_t f_all = 0;
#pragma unroll
                            for (int w = 0; w < NW; ++w)
                                if (w < NWT) f_all |= s_fl[w0 + w][lane];
                            flags_out[ro] = add ? (flags_out[ro] | f_all) : f_all;
                        }
                    }
                }
                __syncthreads();                      // before the next geometry pass or tile
            }
        }
    }
}

// dynamic shared memory of a launch: scene, tables, then the path records
// (body classes) or the wide partial sums of wide_chunks chunks (planar)
static size_t smem_bytes(const DevScene &S, bool bodies, bool records, int blk, int rcap, int wide_chunks,
                         int occ_sets) {
    size_t n = (bodies ? (FOCK_N + FOCK_NP) * 2 + FOCK_NRES * 2 : 0) + (S.n_face <= SMEM_FACE_MAX ? S.n_face : 0) +
               (S.bvh ? 2 * (size_t)min(S.bvh_nodes, BVH_TOP_NODES) : 0);
    if (S.n_body <= SMEM_BODY_MAX) n += 4 * S.n_body;
    if (S.n_tri <= SMEM_TRI_MAX) n += 6 * S.n_tri;
    const int occ_w = (occ_sets > 0 && S.n_body > 0 && S.n_body <= OCC_MAX_BODIES) ? (S.n_body + 31) >> 5 : 0;
    return n * sizeof(float4) + WEIDEMAN_N * sizeof(float) + 16 +
           (records ? sizeof(float) * (blk / 32) * rcap * REC_N * 32 : 0) +
           sizeof(float) * (blk / 32) * wide_chunks * NFC * 6 * 32 +
           sizeof(uint32_t) * (size_t)S.n_body * occ_w * (1 + occ_sets);
}

// Launch state of one evaluation: the counters (escalations, one work queue
// per launch) and the launches queued so far.
struct LaunchCtx {
    unsigned long long *ctr;
    int n;
    cudaStream_t stream;
};

// What one evaluation covers: one frame (F1, frames == nullptr) or a batch
// of frames, and where its inputs and outputs are.
struct Work {
    FrameDev F1;
    const FrameDev *frames;
    int n_frames;
    unsigned long long n_tiles;
    const float *rx;
    const int32_t *perm;
    float *e;
    uint32_t *fl;
    uint64_t *codes;
    int32_t *counts;
    int cap;
    int nwt_planar, nwt_body, planar_chunks;   // tile shape and planar chunks per launch (FP32 fields)
};

template <typename T, bool PATHS, int CLS, bool LIST = false>
static cudaError_t launch_one(const DevScene &S, const Work &W, int ch0, int nch, int accumulate, LaunchCtx &L,
                              int enc = 0) {
    if (L.n >= CTR_QUEUES) return cudaErrorInvalidValue;
    constexpr bool bodies = (CLS & CLS_BODIES) != 0;
    constexpr int blk = blk_of(CLS, sizeof(T) == 4);
    constexpr int NW = blk / 32;
    // warps per tile (fields): the configured shape where it divides the
    // block (FP32), else the default (body kernels 4, planar the whole block)
    int nwt = bodies ? (sizeof(T) == 4 ? W.nwt_body : WARPS_PER_TILE) : (sizeof(T) == 4 ? W.nwt_planar : NW);
    if (nwt < 1 || NW % nwt != 0) nwt = bodies ? WARPS_PER_TILE : NW;
    if (W.frames && TILE_ALIGN % (NW / nwt) != 0) return cudaErrorInvalidValue;
    // records per lane: one frequency chunk flushes full buffers on the way
    // (5 is enough); several chunks size the body range by the capacity
    int rcap = (nch > 1) ? 6 : 5;
    const bool wide = is_planar(CLS) && sizeof(T) == 4 && !PATHS;
    if (nch < 1 || nch > MAX_CHUNKS || (!wide && !bodies && nch != 1)) return cudaErrorInvalidValue;
    // occluder masks (FP32 body kernels): one source-side set, and one
    // receiver-side set per tile in flight (fields) or per warp (path lists)
    const int occ_sets = (bodies && sizeof(T) == 4 && CLS != CLS_WCREEP) ? (PATHS ? NW : NW / nwt) : 0;
    const bool recs = bodies && sizeof(T) == 4 && !PATHS;
    size_t sm = smem_bytes(S, bodies, recs, blk, rcap, wide ? nch : 0, occ_sets);
    int dev = 0, nsm = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (recs) {
        // many bodies (their data and occluder masks in shared memory): fewer
        // records per lane -- fewer bodies per geometry pass, or earlier
        // flushes -- down to one work unit's, so that the block still fits
        int smax = 0;
        cudaFuncAttributes fa;
        if ((e = cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
        if ((e = cudaFuncGetAttributes(&fa, k_eval<T, PATHS, CLS, LIST>)) != cudaSuccess) return e;
        while (rcap > recs_per_unit(CLS) && fa.sharedSizeBytes + sm > (size_t)smax)
            sm = smem_bytes(S, bodies, recs, blk, --rcap, wide ? nch : 0, occ_sets);
    }
    e = cudaFuncSetAttribute(k_eval<T, PATHS, CLS, LIST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    // persistent grid: the blocks that fit on the device at once, at most
    // one per work unit
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_eval<T, PATHS, CLS, LIST>, blk, sm)) != cudaSuccess) return e;
    // (path lists: each warp takes whole tiles; up to one block per tile, so
    // that a few tiles spread over as many SMs)
    const int tiles_per_unit = PATHS ? 1 : NW / nwt;
    long long need = (long long)((W.n_tiles + tiles_per_unit - 1) / tiles_per_unit);
    long long cap_blocks = (long long)nsm * (occ > 0 ? occ : 1);
    int grid = (int)(need < cap_blocks ? need : cap_blocks);
    if (grid < 1) grid = 1;
    // every launch after the first of the evaluation is a programmatic
    // dependent of the one before: it may start while that one finishes
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(blk);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = L.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = L.n > 0 ? 1 : 0;
    e = cudaLaunchKernelEx(&cfg, k_eval<T, PATHS, CLS, LIST>, S, W.F1, W.frames, W.n_frames, W.n_tiles, W.rx, W.perm, W.e, W.fl,
                           W.codes, W.counts, W.cap, ch0, nch, rcap, nwt, accumulate, enc, L.ctr, L.ctr + 1 + L.n);
    ++L.n;
    return e != cudaSuccess ? e : cudaGetLastError();
}

// The class kernels of one evaluation.  Path lists and FP64 fields: the
// three classes per frequency chunk.  FP32 fields: the planar kernel per
// PLANAR_CHUNKS chunks, then each body kernel once for all chunks (the
// geometry of a pass serves every chunk it covers).
// The first launch writes the outputs, the later ones add to them.  Creeping
// rays with extra turns round the body: one more creeping launch per turn
// count (the geometry differs only in the arc length).
template <typename T, bool PATHS, bool LIST = false>
static cudaError_t launch_all(const DevScene &S, const Work &W, int nchunks, LaunchCtx &L) {
    cudaError_t e = cudaSuccess;
    const bool chunked_bodies = PATHS || sizeof(T) != 4;
    // wall -> creeping paths: single scenes with faces and bodies
    const bool wall = (S.enable & RT_EN_WALL_CREEP) && S.txw && !W.frames && S.n_face > 0 && S.n_body > 0;
    // FP32 fields: each planar launch takes up to PLANAR_CHUNKS chunks in one
    // geometry pass
    const int pstep = chunked_bodies ? 1 : (W.planar_chunks >= 1 && W.planar_chunks <= MAX_CHUNKS ? W.planar_chunks
                                                                                                  : PLANAR_CHUNKS);
    for (int ch = 0; ch < nchunks && e == cudaSuccess; ch += pstep) {
        const int n = nchunks - ch < pstep ? nchunks - ch : pstep;
        e = (S.cand && S.n_cand > 0) ? launch_one<T, PATHS, CLS_SEQ, LIST>(S, W, ch, n, 0, L)
                                     : launch_one<T, PATHS, CLS_PLANAR, LIST>(S, W, ch, n, 0, L);
        if (chunked_bodies && e == cudaSuccess) e = launch_one<T, PATHS, CLS_BODYREFL, LIST>(S, W, ch, 1, 1, L);
        for (int enc = 0; chunked_bodies && enc <= S.max_enc && e == cudaSuccess; ++enc)
            e = launch_one<T, PATHS, CLS_CREEP, LIST>(S, W, ch, 1, 1, L, enc);
        for (int enc = 0; chunked_bodies && wall && enc <= S.max_enc && e == cudaSuccess; ++enc)
            e = launch_one<T, PATHS, CLS_WCREEP, LIST>(S, W, ch, 1, 1, L, enc);
    }
    if (!chunked_bodies && e == cudaSuccess) e = launch_one<T, PATHS, CLS_BODYREFL, LIST>(S, W, 0, nchunks, 1, L);
    for (int enc = 0; !chunked_bodies && enc <= S.max_enc && e == cudaSuccess; ++enc)
        e = launch_one<T, PATHS, CLS_CREEP, LIST>(S, W, 0, nchunks, 1, L, enc);
    for (int enc = 0; !chunked_bodies && wall && enc <= S.max_enc && e == cudaSuccess; ++enc)
        e = launch_one<T, PATHS, CLS_WCREEP, LIST>(S, W, 0, nchunks, 1, L, enc);
    return e;
}

// paths: path lists only; list: fields and the path list (FP32: from the
// same kernels, unordered; FP64: the fields, then the path-list kernels)
static int run(const DevScene &S, const Work &W, int precision, bool paths, bool list, unsigned long long *ctr,
               cudaStream_t stream, int *n_launches) {
    LaunchCtx L{ctr, 0, stream};
    const int nchunks = paths ? 1 : (S.n_f + NFC - 1) / NFC;
    cudaError_t e;
    if (precision == RT_PREC_FP64) {
        e = paths ? launch_all<dx, true>(S, W, nchunks, L) : launch_all<dx, false>(S, W, nchunks, L);
        if (list && e == cudaSuccess) e = launch_all<dx, true>(S, W, 1, L);
    } else if (paths) {
        e = launch_all<float, true>(S, W, nchunks, L);
    } else {
        e = list ? launch_all<float, false, true>(S, W, nchunks, L) : launch_all<float, false>(S, W, nchunks, L);
    }
    *n_launches = L.n;
    if (e != cudaSuccess) {
        set_error(std::string("k_eval launch: ") + cudaGetErrorString(e));
        return RT_ERR_CUDA;
    }
    return RT_OK;
}

int launch_eval(const DevScene &S, const float *rx_soa, int n_rx, float *e_out, uint32_t *flags,
                uint64_t *codes, int32_t *counts, int cap, int precision, const int *shape, unsigned long long *ctr,
                cudaStream_t stream, int *n_launches) {
    *n_launches = 0;
    // fields and a path list (unordered): counts zeroed first
    const bool paths = codes != nullptr && e_out == nullptr;
    if (n_rx <= 0) return RT_OK;
    Work W = {};
    W.F1.body = S.body;
    W.F1.txb = S.txb;
    W.F1.fqc = S.fqc;
    W.F1.n_rx = n_rx;
    W.F1.n_body = S.n_body;
    W.F1.band = S.band_len;
    for (int f = 0; f < S.n_f; ++f) {
        double lam = 299792458.0 / S.freq[f];
        if (lam / 2.0 > W.F1.hl) W.F1.hl = lam / 2.0;
    }
    W.frames = nullptr;
    W.n_frames = 1;
    W.n_tiles = ((unsigned long long)n_rx + 31ull) >> 5;
    W.rx = rx_soa; W.e = e_out; W.fl = flags;
    W.codes = codes; W.counts = counts; W.cap = cap;
    W.nwt_planar = shape ? shape[0] : 4;
    W.nwt_body = shape ? shape[1] : WARPS_PER_TILE;
    W.planar_chunks = shape ? shape[2] : PLANAR_CHUNKS;
    if (codes && e_out) {
        cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)n_rx, stream);
        if (e != cudaSuccess) {
            set_error(std::string("launch_eval: ") + cudaGetErrorString(e));
            return RT_ERR_CUDA;
        }
    }
    return run(S, W, precision, paths, codes && e_out, ctr, stream, n_launches);
}

int launch_eval_batch(const DevScene &S, const FrameDev *frames_dev, const FrameDev *frames_host, int n_frames,
                      unsigned long long n_tiles, const float *rx_soa, const int32_t *perm, float *e_out,
                      uint32_t *flags, int precision, const int shape[3], unsigned long long *ctr,
                      cudaStream_t stream, int *n_launches) {
    *n_launches = 0;
    if (n_frames <= 0 || n_tiles == 0) return RT_OK;
    Work W = {};
    W.F1 = frames_host[0];      // (unused by the kernels when frames is set)
    W.frames = frames_dev;
    W.n_frames = n_frames;
    W.n_tiles = n_tiles;
    W.rx = rx_soa; W.perm = perm; W.e = e_out; W.fl = flags;
    W.nwt_planar = shape[0]; W.nwt_body = shape[1]; W.planar_chunks = shape[2];
    return run(S, W, precision, false, false, ctr, stream, n_launches);
}

// ============================================================== adjoint
// Gradient of a scalar loss through the fields (the vector-Jacobian product
// of the evaluation): given dLoss/dE (real and imaginary parts) at every
// receiver and frequency, the sums over the listed paths of each path's
// field derivative with respect to its body's centre and radius, the
// transmitter position and the frequency.  Visibility is held fixed: the
// paths are those of the forward path list (rt_paths), and each one's
// geometry and field are recomputed here in dual numbers (dual.cuh), by the
// same construction as the forward path: image points for planar
// reflections (Eq. 3), the specular point on the body (its derivative from
// one Newton step in dual arithmetic at the root, which is the
// implicit-function derivative), the tangent points and geodesic of the
// creeping ray (Eq. 4, Fig. 1), the Fock--Pekeris functions (table
// derivative from the cubic Hermite interpolant, residue series term by
// term), the transition function through w'(z) = -2 z w(z) + 2j/sqrt(pi).
//
// F8 (FP32 duals, the default): the forward FP32 construction -- FP32
// geometry, table and Faddeeva coefficients -- with each path's length for
// the phase as double-float from the same exact pieces the forward FP32
// kernel uses (the source's FP64 images, the tangent lengths from exact
// squares), so its phase keeps the forward's accuracy.  Direct, planar and
// creeping paths take F8; reflections off a body take D8 in both modes.
// D8 (FP64 duals, RT_PREC_FP64): the forward FP64 construction.

template <> __device__ __forceinline__ void face_plane<D8>(const Ctx &c, int f, v3t<D8> *n, D8 *d) {
    dq4 q = c.face64[f]; *n = mk3<D8>(q.x, q.y, q.z); *d = D8(q.w);
}
template <> __device__ __forceinline__ void face_plane<F8>(const Ctx &c, int f, v3t<F8> *n, F8 *d) {
    float4 q = c.face32[f]; *n = mk3<F8>(q.x, q.y, q.z); *d = F8(q.w);
}

// Fock--Pekeris functions of a dual xi: the residue series term by term
// above XI_HI, else the table's cubic Hermite interpolant and its slope
__device__ void pekeris(const Ctx &c, const D8 &xi, cpx<D8> &ps, cpx<D8> &ph, bool regular) {
    const double cc = (0.5 / sqrt(M_PI)) * cos(M_PI / 4.0);
    const D8 ci = D8(cc) / xi;
    if (xi.v > XI_HI) {
        cpx<D8> ss = mkc<D8>(0.0, 0.0), sh = mkc<D8>(0.0, 0.0);
        for (int n = 0; n < FOCK_NRES; ++n) {
            dq4 rs = c.res64[2 * n], rh = c.res64[2 * n + 1];
            D8 sn, cs;
            SinCos(xi * D8(rs.y), &sn, &cs);
            D8 e = Exp(-(xi * D8(rs.x))) * D8(rs.z);
            ss = ss + mkc<D8>(e * cs, -(e * sn));
            SinCos(xi * D8(rh.y), &sn, &cs);
            e = Exp(-(xi * D8(rh.x))) * D8(rh.z);
            sh = sh + mkc<D8>(e * cs, -(e * sn));
        }
        const cpx<D8> pre = mkc<D8>(-cos(M_PI / 12.0) * (0.5 / sqrt(M_PI)), sin(M_PI / 12.0) * (0.5 / sqrt(M_PI)));
        ps = pre * ss;
        ph = pre * sh;
        if (regular) { ps = ps + mkc<D8>(ci, -ci); ph = ph + mkc<D8>(ci, -ci); }
        return;
    }
    // cubic Hermite interpolant of G and its derivative in xi
    const double u = (xi.v - XI_LO) / XI_STEP;
    const int j = min(max((int)u, 0), FOCK_N - 2);
    const double t = u - j, t2 = t * t, omt = 1.0 - t;
    const double h00 = (1 + 2 * t) * omt * omt, h10 = t * omt * omt * XI_STEP, h01 = t2 * (3 - 2 * t),
                 h11 = t2 * (t - 1) * XI_STEP;
    // d/dxi = (d/dt) / XI_STEP
    const double d00 = (6 * t2 - 6 * t) / XI_STEP, d10 = 1 - 4 * t + 3 * t2, d01 = (6 * t - 6 * t2) / XI_STEP,
                 d11 = 3 * t2 - 2 * t;
    cpx<D8> G[2];
    for (int k = 0; k < 2; ++k) {
        double2 g0 = c.fock64[(j * 2 + k) * 2], q0 = c.fock64[(j * 2 + k) * 2 + 1];
        double2 g1 = c.fock64[((j + 1) * 2 + k) * 2], q1 = c.fock64[((j + 1) * 2 + k) * 2 + 1];
        const double gr = h00 * g0.x + h10 * q0.x + h01 * g1.x + h11 * q1.x;
        const double gi = h00 * g0.y + h10 * q0.y + h01 * g1.y + h11 * q1.y;
        const double dr = d00 * g0.x + d10 * q0.x + d01 * g1.x + d11 * q1.x;
        const double di = d00 * g0.y + d10 * q0.y + d01 * g1.y + d11 * q1.y;
        G[k] = mkc<D8>(dchain<double>(gr, dr, xi), dchain<double>(gi, di, xi));
    }
    const cpx<D8> rot = cexpi(xi * xi * xi / D8(12.0));
    ps = G[0] * rot;
    ph = G[1] * rot;
    if (!regular) { ps = ps - mkc<D8>(ci, -ci); ph = ph - mkc<D8>(ci, -ci); }
}
__device__ void pekeris(const Ctx &c, const F8 &xi, cpx<F8> &ps, cpx<F8> &ph, bool regular) {
    const F8 ci = F8(0.19947114f) / xi;               // c/xi = (ci, -ci)
    if (xi.v > (float)XI_HI) {
        // (the FP32 table's residue constants: alpha sqrt3/2, alpha/2, coefficient)
        cpx<F8> ss = mkc<F8>(0.0f, 0.0f), sh = mkc<F8>(0.0f, 0.0f);
        for (int n = 0; n < FOCK_NRES; ++n) {
            const float4 rs = c.res[2 * n], rh = c.res[2 * n + 1];
            F8 sn, cs;
            SinCos(xi * F8(rs.y), &sn, &cs);
            F8 e = Exp(-(xi * F8(rs.x))) * F8(rs.z);
            ss = ss + mkc<F8>(e * cs, -(e * sn));
            SinCos(xi * F8(rh.y), &sn, &cs);
            e = Exp(-(xi * F8(rh.x))) * F8(rh.z);
            sh = sh + mkc<F8>(e * cs, -(e * sn));
        }
        const cpx<F8> pre = mkc<F8>(-0.27248264483602590f, 0.07301150463530957f);   // -e^{-j pi/12}/(2 sqrt(pi))
        ps = pre * ss;
        ph = pre * sh;
        if (regular) { ps = ps + mkc<F8>(ci, -ci); ph = ph + mkc<F8>(ci, -ci); }
        return;
    }
    // the FP32 table holds G and XI_STEP G' per node
    const float u = (xi.v - (float)XI_LO) * (float)(1.0 / XI_STEP);
    const int j = min(max((int)u, 0), FOCK_N - 2);
    const float t = u - (float)j, t2 = t * t, omt = 1.0f - t;
    const float h00 = (1.0f + 2.0f * t) * omt * omt, h10 = t * omt * omt, h01 = t2 * (3.0f - 2.0f * t),
                h11 = t2 * (t - 1.0f);
    const float ih = (float)(1.0 / XI_STEP);
    const float d00 = (6.0f * t2 - 6.0f * t) * ih, d10 = (1.0f - 4.0f * t + 3.0f * t2) * ih,
                d01 = (6.0f * t - 6.0f * t2) * ih, d11 = (3.0f * t2 - 2.0f * t) * ih;
    cpx<F8> G[2];
    for (int k = 0; k < 2; ++k) {
        const float4 a0 = c.fock[2 * j + k], a1 = c.fock[2 * j + 2 + k];
        const float gr = h00 * a0.x + h10 * a0.z + h01 * a1.x + h11 * a1.z;
        const float gi = h00 * a0.y + h10 * a0.w + h01 * a1.y + h11 * a1.w;
        const float dr = d00 * a0.x + d10 * a0.z + d01 * a1.x + d11 * a1.z;
        const float di = d00 * a0.y + d10 * a0.w + d01 * a1.y + d11 * a1.w;
        G[k] = mkc<F8>(dchain<float>(gr, dr, xi), dchain<float>(gi, di, xi));
    }
    const cpx<F8> rot = cexpi(xi * xi * xi / F8(12.0f));
    ps = G[0] * rot;
    ph = G[1] * rot;
    if (!regular) { ps = ps - mkc<F8>(ci, -ci); ph = ph - mkc<F8>(ci, -ci); }
}

// w(z) of a dual z, with w'(z) = -2 z w + 2j / sqrt(pi)
template <typename S>
__device__ __forceinline__ cpx<DualT<S>> faddeeva_dual(const cpx<DualT<S>> &zd, cpx<S> w) {
    const cpx<S> z = mkc(zd.re.v, zd.im.v);
    const cpx<S> wp = z * w * S(-2) + mkc(S(0), S(1.1283791670955126));
    cpx<DualT<S>> r;
    r.re.v = w.re; r.im.v = w.im;
#pragma unroll
    for (int k = 0; k < ND; ++k) {
        r.re.d[k] = wp.re * zd.re.d[k] - wp.im * zd.im.d[k];
        r.im.d[k] = wp.re * zd.im.d[k] + wp.im * zd.re.d[k];
    }
    return r;
}
__device__ cpx<D8> faddeeva_t(const Ctx &c, const cpx<D8> &zd) {
    cpx<double> z = mkc(zd.re.v, zd.im.v);
    const double L = c.weid_L;
    cpx<double> lm = mkc(L + z.im, -z.re), lp = mkc(L - z.im, z.re);
    cpx<double> Z = cdiv(lp, lm);
    cpx<double> p = mkc(c.weid64[WEIDEMAN_N - 1], 0.0);
    for (int n = WEIDEMAN_N - 2; n >= 0; --n) p = p * Z + mkc(c.weid64[n], 0.0);
    cpx<double> w = cdiv(p * 2.0, lm * lm) + cdiv(mkc(0.56418958354775628, 0.0), lm);
    return faddeeva_dual<double>(zd, w);
}
__device__ cpx<F8> faddeeva_t(const Ctx &c, const cpx<F8> &zd) {
    return faddeeva_dual<float>(zd, faddeeva<float>(c, mkc(zd.re.v, zd.im.v)));
}

// wavenumber, (k/2)^{1/3} with the frequency as slot DS_F
__device__ __forceinline__ D8 kof(const FreqC &fq, int f, const D8 &) {
    D8 k(fq.kd[f]);
    k.d[DS_F] = 2.0 * M_PI / 299792458.0;
    return k;
}
__device__ __forceinline__ F8 kof(const FreqC &fq, int f, const F8 &) {
    F8 k(fq.k[f]);
    k.d[DS_F] = (float)(2.0 * M_PI / 299792458.0);
    return k;
}
__device__ __forceinline__ D8 khof(const FreqC &fq, int f, const D8 &x) { return Cbrt(kof(fq, f, x) * D8(0.5)); }
__device__ __forceinline__ F8 khof(const FreqC &fq, int f, const F8 &x) { return Cbrt(kof(fq, f, x) * F8(0.5f)); }

// the path phasor e^{-j k L}; FP64 duals: from the dual length itself
__device__ __forceinline__ cpx<D8> phasor(const FreqC &fq, int f, const D8 &L) {
    D8 fc(fq.fc[f]);
    fc.d[DS_F] = 1.0 / 299792458.0;
    D8 cyc = L * fc;
    cyc.v -= floor(cyc.v);                      // the integer cycles (no derivative)
    D8 s, co;
    SinCosPi(cyc * D8(2.0), &s, &co);
    return mkc<D8>(co, -s);
}
__device__ __forceinline__ D8 len_val(const D8 &L) { return L; }
// FP32 duals: the length's tangents from the dual, its value as double-float
// (the phase as the FP32 fraction of L / lambda, integer cycles dropped)
struct LenF8 {
    F8 l;           // tangents (and an FP32 value for amplitudes)
    dfl h;          // the value, for the phase
};
__device__ __forceinline__ cpx<F8> phasor(const FreqC &fq, int f, const LenF8 &L) {
    dfl il; il.hi = fq.il_hi[f]; il.lo = fq.il_lo[f];
    const dfl cyc = df_mul(L.h, il);
    float fr = (cyc.hi - floorf(cyc.hi)) + cyc.lo;
    fr -= floorf(fr);
    const float ilf = il.hi;
    F8 c;
    c.v = fr;
#pragma unroll
    for (int k = 0; k < ND; ++k) c.d[k] = L.l.d[k] * ilf;
    c.d[DS_F] += (L.h.hi + L.h.lo) * (float)(1.0 / 299792458.0);    // d(L f / c)/df
    F8 s, co;
    SinCosPi(c * F8(2.0f), &s, &co);
    return mkc<F8>(co, -s);
}
__device__ __forceinline__ F8 len_val(const LenF8 &L) { return L.l; }

template <typename DT> struct AdjLen;
template <> struct AdjLen<D8> { typedef D8 type; };
template <> struct AdjLen<F8> { typedef LenF8 type; };
__device__ __forceinline__ D8 mk_len(const D8 &l, dfl) { return l; }
__device__ __forceinline__ LenF8 mk_len(const F8 &l, dfl h) { return LenF8{l, h}; }

// contracts each path field's tangents with dLoss/dE of its receiver
struct AccAdj {
    const float *gE;        // [n_f][3][n_rx][2]
    int n_rx, r, f0;
    double g[ND - 1];       // body and transmitter slots
    double gf[NFC];         // frequency slot, per frequency of the chunk
};
template <typename S>
__device__ __forceinline__ void acc_put(AccAdj &a, int f, const cpx<DualT<S>> &x, const cpx<DualT<S>> &y,
                                        const cpx<DualT<S>> &z) {
    const cpx<DualT<S>> *e[3] = {&x, &y, &z};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const size_t idx = ((size_t)(a.f0 + f) * 3 + q) * a.n_rx + a.r;
        const S gr = a.gE[2 * idx], gi = a.gE[2 * idx + 1];
#pragma unroll
        for (int k = 0; k < ND - 1; ++k) a.g[k] += (double)(gr * e[q]->re.d[k] + gi * e[q]->im.d[k]);
        a.gf[f] += (double)(gr * e[q]->re.d[DS_F] + gi * e[q]->im.d[DS_F]);
    }
}

// body b's centre and radius as parameters (slots 0-3)
template <typename S>
__device__ __forceinline__ void adj_body(const Ctx &c, int b, v3t<DualT<S>> &cc, DualT<S> &a, bool &sphere) {
    float4 q0 = c.body[2 * b], q1 = c.body[2 * b + 1];
    cc = mk3<DualT<S>>(dvar_t<S>(q0.x, DS_CX), dvar_t<S>(q0.y, DS_CY), dvar_t<S>(q0.z, DS_CZ));
    a = dvar_t<S>(q0.w, DS_A);
    sphere = q1.y == 0.0f;
}

// the reflection point's angle as a dual: the root in the dual's precision
// (FP64: refined to the bisection root; FP32: the forward FP32 root, refined
// in double-float or FP64 near grazing), then one Newton step on dL/dpsi = 0
// in dual arithmetic (the implicit-function derivative)
__device__ __forceinline__ void refl_root_val(double a, double ds, double pu, double pv, double gam, double *c0,
                                              double *s0) {
    dx cc, ss;
    refl_root(dx(a), dx(ds), dx(pu), dx(pv), dx(gam), &cc, &ss);
    *c0 = cc.v; *s0 = ss.v;
}
__device__ __forceinline__ void refl_root_val(float a, float ds, float pu, float pv, float gam, float *c0, float *s0) {
    float err = 0.0f, sn, cs;
    refl_n32(a, ds, pu, pv, gam, &cs, &sn, &err);
    const float c2 = (ds * cs - a) / sqrtf((a * cs - ds) * (a * cs - ds) + a * a * sn * sn);
    if (err > 1e-5f * fmaxf(c2, 0.0f)) {
        if (!refl_polish_df(a, ds, pu, pv, cs, sn, &cs, &sn)) refl_polish(a, ds, pu, pv, gam, cs, sn, &cs, &sn);
    }
    *c0 = cs; *s0 = sn;
}
template <typename S>
__device__ __noinline__ void adj_refl_root(const DualT<S> &a, const DualT<S> &ds, const DualT<S> &pu,
                                           const DualT<S> &pv, const DualT<S> &gam, DualT<S> *cs, DualT<S> *sn) {
    typedef DualT<S> DT;
    S c0, s0;
    refl_root_val(a.v, ds.v, pu.v, pv.v, gam.v, &c0, &s0);
    const DT psi(atan2(s0, c0));
    DT s, c;
    SinCos(psi, &s, &c);
    const DT qx = a * c, qy = a * s;
    const DT lS = Sqrt((qx - ds) * (qx - ds) + qy * qy);
    const DT lP = Sqrt((qx - pu) * (qx - pu) + (qy - pv) * (qy - pv));
    const DT gS = a * ds * s / lS, gP = a * (pu * s - pv * c) / lP;
    DT h;
    if constexpr (sizeof(S) == 8) {
        h = (ds * qx - gS * gS) / lS + (pu * qx + pv * qy - gP * gP) / lP;
    } else {
        // d2L/dpsi2 in the product form a sum_X (u - a)(|X|^2 - a u) / |Q - X|^3,
        // u = X.n: the difference form above cancels near grazing incidence
        const DT uS = ds * c, uP = pu * c + pv * s;
        h = a * ((uS - a) * (ds * ds - a * uS) / (lS * lS * lS) +
                 (uP - a) * (pu * pu + pv * pv - a * uP) / (lP * lP * lP));
    }
    SinCos(psi - (gS + gP) / h, sn, cs);
}

// double-float lengths of the FP32 path pieces (no use for FP64 duals)
__device__ __forceinline__ v3t<float> vals(const v3t<F8> &a) { return mk3(a.x.v, a.y.v, a.z.v); }
__device__ __forceinline__ v3t<float> vals(const v3t<D8> &a) {
    return mk3((float)a.x.v, (float)a.y.v, (float)a.z.v);
}
// sqrt(|X - c|^2 - a^2) from the exact squares (horiz: horizontal distance)
__device__ __forceinline__ dfl df_tangent_len(v3t<float> X, float4 q0, bool horiz) {
    dfl q2 = df_add(df_sq_diff(X.x, q0.x), df_sq_diff(X.y, q0.y));
    if (!horiz) q2 = df_add(q2, df_sq_diff(X.z, q0.z));
    dfl a2 = two_prod(q0.w, q0.w);
    a2.hi = -a2.hi; a2.lo = -a2.lo;
    q2 = df_add(q2, a2);
    if (!(q2.hi > 0.0f)) { q2.hi = 0.0f; q2.lo = 0.0f; return q2; }
    return df_sqrt(q2);
}

// reflection off body b (the forward construction, without decisions)
template <typename DT>
__device__ __noinline__ void adj_rb(const Ctx &c, int b, v3t<DT> S, v3t<DT> P, const FreqC &fq, AccAdj &acc) {
    typedef decltype(DT().v) SC;
    v3t<DT> cc;
    DT a;
    bool sphere;
    adj_body<SC>(c, b, cc, a, sphere);
    Frame<DT> F;
    if (sphere) sphere_frame(S, P, cc, a, F, DT(0.0f));
    else cyl_frame(S, P, cc.x, cc.y, a, F, DT(0.0f));
    DT cs, sn;
    adj_refl_root<SC>(a, F.ds, F.pu, F.pv, F.gam, &cs, &sn);
    v3t<DT> n = F.u * cs + F.v * sn;
    v3t<DT> Q;
    if (sphere) {
        Q = cc + n * a;
    } else {
        DT qx = a * cs, qy = a * sn;
        DT l1 = Sqrt((qx - F.ds) * (qx - F.ds) + qy * qy);
        DT l2 = Sqrt((qx - F.pu) * (qx - F.pu) + (qy - F.pv) * (qy - F.pv));
        DT zq = S.z + (P.z - S.z) * l1 / (l1 + l2);
        Q = mk3<DT>(cc.x + a * n.x, cc.y + a * n.y, zq);
    }
    Geo<DT> g;
    v3t<DT> shi = unit3(Q - S);
    DT cth = -dot3(shi, n);
    g.dr = P - Q;
    g.Q1 = Q;
    g.n1 = n;
    if (sphere) {
        g.inv_f1 = DT(2.0f) / (a * cth);
        g.inv_f2 = DT(2.0f) * cth / a;
        g.rho_g = a;
    } else {
        g.inv_f1 = DT(2.0f) * (DT(1.0f) - shi.z * shi.z) / (a * cth);
        g.inv_f2 = DT(0.0f);
        DT sphi = -(shi.x * n.y) + shi.y * n.x;
        g.rho_g = (sphi == DT(0.0f)) ? DT(INFINITY) : a * (DT(1.0f) - cth * cth) / (sphi * sphi);
    }
    dfl Lh = {0.0f, 0.0f};
    if constexpr (sizeof(SC) == 4) {
        // the forward's length: both legs to the FP32 surface point c + a n, in double-float
        const float4 q0 = c.body[2 * b];
        dfl ws[3], wp[3];
        df_to_surface(vals(S), q0, q0.w, vals(n), !sphere, ws);
        df_to_surface(vals(P), q0, q0.w, vals(n), !sphere, wp);
        const dfl si = df_norm3(ws), sr = df_norm3(wp);
        if (sphere) {
            Lh = df_add(si, sr);
        } else {
            const dfl H = df_add(si, sr);
            Lh = df_sqrt(df_add(df_mul(H, H), df_sq_diff(P.z.v, S.z.v)));
        }
    }
    field_body_refl<DT, typename AdjLen<DT>::type, false, AccAdj>(c, acc, fq, S, P, g,
                                                                  mk_len(norm3(Q - S) + norm3(P - Q), Lh));
}

// creeping ray round body b, dir 0 short way, 1 long way, with enc extra
// turns; wall >= 0: fed by the reflection at face wall (the creeping ray of
// the source's image there); false: no finite field
template <typename DT>
__device__ __noinline__ bool adj_creep(const Ctx &c, int b, int dir, int enc, v3t<DT> S0, v3t<DT> P, const FreqC &fq,
                                       unsigned enable, AccAdj &acc, int wall = -1) {
    typedef decltype(DT().v) SC;
    v3t<DT> cc;
    DT a;
    bool sphere;
    adj_body<SC>(c, b, cc, a, sphere);
    v3t<DT> S = S0;
    v3t<float> Sval = vals(S0);            // (FP32 duals: the source point of the tangent length)
    if (wall >= 0) {
        v3t<DT> n;
        DT d;
        face_plane<DT>(c, wall, &n, &d);
        S = mirror_pt(S0, n, d);
        if constexpr (sizeof(SC) == 4) {
            // the image's value from the FP64 plane, as the forward's per-transmitter table has it
            const dq4 q = c.face64[wall];
            const double X[3] = {c.S.x, c.S.y, c.S.z};
            const double dist = q.x * X[0] + q.y * X[1] + q.z * X[2] - q.w;
            Sval = mk3((float)(X[0] - q.x * (2.0 * dist)), (float)(X[1] - q.y * (2.0 * dist)),
                       (float)(X[2] - q.z * (2.0 * dist)));
        }
    }
    Frame<DT> F;
    if (sphere) sphere_frame(S, P, cc, a, F, DT(0.0f));
    else cyl_frame(S, P, cc.x, cc.y, a, F, DT(0.0f));
    const DT TWO_PI(SC(6.283185307179586476925286766559));
    DT dpsi = (dir == 0) ? (F.gam - F.bs - F.bp) : (TWO_PI - F.gam - F.bs - F.bp);
    dpsi = dpsi + TWO_PI * DT(SC(enc));
    Geo<DT> g;
    DT psi1 = (dir == 0) ? F.bs : -F.bs;
    DT psi2 = (dir == 0) ? F.gam - F.bp : F.gam + F.bp;
    DT s1, c1, s2, c2;
    SinCos(psi1, &s1, &c1);
    SinCos(psi2, &s2, &c2);
    g.n1 = F.u * c1 + F.v * s1;
    g.n2 = F.u * c2 + F.v * s2;
    dfl Lh = {0.0f, 0.0f};
    if (sphere) {
        g.Q1 = cc + g.n1 * a;
        g.Q2 = cc + g.n2 * a;
        g.sp = F.sps;
        g.sq = F.sqp;
        g.t = a * dpsi;
        g.rho_g = a;
        g.caus = (dir == 1);
        DT sg, cg;
        SinCos(F.gam, &sg, &cg);
        g.dperp = F.dp * sg;
        if (!(g.dperp > DT(0.0f))) return false;
        DT sb, cb;
        SinCos(F.bs, &sb, &cb);
        g.amp = Sqrt(a * sb / g.dperp) / Sqrt(g.sq) / g.sp;
        if (enc & 1) g.amp = -g.amp;             // the (-1) of an odd number of extra turns
        if constexpr (sizeof(SC) == 4) {
            const float4 q0 = c.body[2 * b];
            Lh = df_addf(df_add(df_tangent_len(Sval, q0, false), df_tangent_len(vals(P), q0, false)), g.t.v);
        }
    } else {
        DT ds_ = F.sps, dp_ = F.sqp;
        DT dz = P.z - S.z;
        DT H = ds_ + a * dpsi + dp_;
        DT ell = Sqrt(H * H + dz * dz);
        DT sin0 = H / ell;
        DT z1 = S.z + dz * ds_ / H, z2 = S.z + dz * (ds_ + a * dpsi) / H;
        g.Q1 = mk3<DT>(cc.x + a * g.n1.x, cc.y + a * g.n1.y, z1);
        g.Q2 = mk3<DT>(cc.x + a * g.n2.x, cc.y + a * g.n2.y, z2);
        g.sp = ds_ / sin0;
        g.t = a * dpsi / sin0;
        g.sq = dp_ / sin0;
        g.rho_g = a / (sin0 * sin0);
        g.caus = 0;
        g.dperp = DT(0.0f);
        g.amp = DT(1.0f) / Sqrt(g.sp * g.sq * (g.sp + g.t + g.sq));
        if constexpr (sizeof(SC) == 4) {
            const float4 q0 = c.body[2 * b];
            const dfl Hh = df_addf(df_add(df_tangent_len(Sval, q0, true), df_tangent_len(vals(P), q0, true)),
                                   (a * dpsi).v);
            Lh = df_sqrt(df_add(df_mul(Hh, Hh), df_sq_diff(P.z.v, Sval.z)));
        }
    }
    typedef typename AdjLen<DT>::type LT;
    if (wall >= 0)
        field_wcreep<DT, LT, false, AccAdj>(c, acc, fq, wall, S0, S, P, g, mk_len(g.sp + g.t + g.sq, Lh), enable);
    else
        field_creep<DT, LT, false, AccAdj>(c, acc, fq, S, P, g, mk_len(g.sp + g.t + g.sq, Lh), enable);
    return true;
}

// the precise value of a planar path's length for FP32 duals: |P - image|,
// the image the source's FP64 mirror (double-float tables where they exist)
__device__ __forceinline__ dfl planar_len(const Ctx &c, int order, int i, int j, v3t<float> P) {
    if (order == 0) return df_dist(c.S, P);
    if (order == 1) return df_dist_df(c.img[2 * i], c.img[2 * i + 1], P);
    if (c.img_pairs) {
        const int slot = c.n_face + i * c.n_face + j;
        return df_dist_df(c.img[2 * slot], c.img[2 * slot + 1], P);
    }
    // (large scenes keep no pair table: the second mirror from the first image in FP64)
    const float4 h = c.img[2 * i], l = c.img[2 * i + 1];
    const double X[3] = {(double)h.x + (double)l.x, (double)h.y + (double)l.y, (double)h.z + (double)l.z};
    const dq4 q = c.face64[j];
    const double dist = q.x * X[0] + q.y * X[1] + q.z * X[2] - q.w;
    const double Y[3] = {X[0] - q.x * (2.0 * dist), X[1] - q.y * (2.0 * dist), X[2] - q.z * (2.0 * dist)};
    float4 yh, yl;
    yh.x = (float)Y[0]; yh.y = (float)Y[1]; yh.z = (float)Y[2]; yh.w = 0.0f;
    yl.x = (float)(Y[0] - (double)yh.x); yl.y = (float)(Y[1] - (double)yh.y); yl.z = (float)(Y[2] - (double)yh.z);
    yl.w = 0.0f;
    return df_dist_df(yh, yl, P);
}

// direct ray and planar image paths (faces i, j; -1: none)
template <typename DT>
__device__ __noinline__ void adj_planar(const Ctx &c, int order, int i, int j, v3t<DT> S, v3t<DT> P,
                                        const FreqC &fq, AccAdj &acc) {
    typedef decltype(DT().v) SC;
    dfl Lh = {0.0f, 0.0f};
    if constexpr (sizeof(SC) == 4) Lh = planar_len(c, order, i, j, vals(P));
    if (order == 0) {
        v3t<DT> d = P - S;
        DT L = norm3(d);
        add_ray(acc, fq, src_pol(c, d * (DT(1.0f) / L)), DT(1.0f) / L, mk_len(L, Lh));
        return;
    }
    v3t<DT> ni, nj;
    DT di, dj;
    face_plane<DT>(c, i, &ni, &di);
    v3t<DT> S1 = mirror_pt(S, ni, di);
    if (order == 1) {
        DT d1 = dot3(ni, S1) - di, dP = dot3(ni, P) - di;
        v3t<DT> Q = S1 + (P - S1) * (d1 / (d1 - dP));
        DT L = norm3(Q - S) + norm3(P - Q);
        if (dielectric(c, i)) {
            const v3t<DT> s1 = unit3(Q - S), e0 = src_pol(c, s1);
            cpx<DT> E[3] = {mkc<DT>(e0.x, DT(0.0f)), mkc<DT>(e0.y, DT(0.0f)), mkc<DT>(e0.z, DT(0.0f))};
            reflect_face(c, i, E, s1, unit3(P - Q));
            add_ray_cx(acc, fq, E, DT(1.0f) / L, mk_len(L, Lh));
        } else {
            add_ray(acc, fq, pec_mirror(src_pol(c, unit3(Q - S)), ni), DT(1.0f) / L, mk_len(L, Lh));
        }
        return;
    }
    face_plane<DT>(c, j, &nj, &dj);
    v3t<DT> S2 = mirror_pt(S1, nj, dj);
    DT d2 = dot3(nj, S2) - dj, dP = dot3(nj, P) - dj;
    v3t<DT> Q2 = S2 + (P - S2) * (d2 / (d2 - dP));
    DT e1 = dot3(ni, S1) - di, eq = dot3(ni, Q2) - di;
    v3t<DT> Q1 = S1 + (Q2 - S1) * (e1 / (e1 - eq));
    DT L = norm3(Q1 - S) + norm3(Q2 - Q1) + norm3(P - Q2);
    if (dielectric(c, i) || dielectric(c, j)) {
        const v3t<DT> s1 = unit3(Q1 - S), s2 = unit3(Q2 - Q1), e0 = src_pol(c, s1);
        cpx<DT> E[3] = {mkc<DT>(e0.x, DT(0.0f)), mkc<DT>(e0.y, DT(0.0f)), mkc<DT>(e0.z, DT(0.0f))};
        reflect_face(c, i, E, s1, s2);
        reflect_face(c, j, E, s2, unit3(P - Q2));
        add_ray_cx(acc, fq, E, DT(1.0f) / L, mk_len(L, Lh));
    } else {
        add_ray(acc, fq, pec_mirror(pec_mirror(src_pol(c, unit3(Q1 - S)), ni), nj), DT(1.0f) / L, mk_len(L, Lh));
    }
}

// order-3 candidate path (faces fs, the candidate list's sequence q): the
// images by mirroring the dual-number source, the points backwards from P
template <typename DT>
__device__ __noinline__ void adj_seq3(const Ctx &c, int q, int4 sq, v3t<DT> S, v3t<DT> P, const FreqC &fq,
                                      AccAdj &acc) {
    typedef decltype(DT().v) SC;
    v3t<DT> ni, nj, nk;
    DT di, dj, dk;
    face_plane<DT>(c, sq.x, &ni, &di);
    face_plane<DT>(c, sq.y, &nj, &dj);
    face_plane<DT>(c, sq.z, &nk, &dk);
    const v3t<DT> S1 = mirror_pt(S, ni, di);
    const v3t<DT> S2 = mirror_pt(S1, nj, dj);
    const v3t<DT> S3 = mirror_pt(S2, nk, dk);
    const DT e3 = dot3(nk, S3) - dk, p3 = dot3(nk, P) - dk;
    const v3t<DT> Q3 = S3 + (P - S3) * (e3 / (e3 - p3));
    const DT e2 = dot3(nj, S2) - dj, p2 = dot3(nj, Q3) - dj;
    const v3t<DT> Q2 = S2 + (Q3 - S2) * (e2 / (e2 - p2));
    const DT e1 = dot3(ni, S1) - di, p1 = dot3(ni, Q2) - di;
    const v3t<DT> Q1 = S1 + (Q2 - S1) * (e1 / (e1 - p1));
    const DT L = norm3(Q1 - S) + norm3(Q2 - Q1) + norm3(Q3 - Q2) + norm3(P - Q3);
    const v3t<DT> s1 = unit3(Q1 - S), s2 = unit3(Q2 - Q1), s3 = unit3(Q3 - Q2), s4 = unit3(P - Q3);
    const v3t<DT> e0 = src_pol(c, s1);
    cpx<DT> E[3] = {mkc<DT>(e0.x, DT(0.0f)), mkc<DT>(e0.y, DT(0.0f)), mkc<DT>(e0.z, DT(0.0f))};
    reflect_face(c, sq.x, E, s1, s2);
    reflect_face(c, sq.y, E, s2, s3);
    reflect_face(c, sq.z, E, s3, s4);
    dfl Lh = {0.0f, 0.0f};
    if constexpr (sizeof(SC) == 4) Lh = df_dist_df(c.cimg[6 * q + 4], c.cimg[6 * q + 5], vals(P));
    add_ray_cx(acc, fq, E, DT(1.0f) / L, mk_len(L, Lh));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One warp per receiver (persistent, from a queue), its lanes over the
// receiver's listed paths.  Body gradients by atomics per path; transmitter
// and frequency gradients summed over the warp first.
template <typename DT>
__global__ void __launch_bounds__(128) k_adjoint(DevScene S, const float *__restrict__ rx, int n_rx,
                                                 const uint64_t *__restrict__ codes,
                                                 const int32_t *__restrict__ counts, int cap,
                                                 const float *__restrict__ gE, double *g_body, double *g_tx,
                                                 double *g_f, unsigned long long *queue) {
    typedef decltype(DT().v) SC;
    Ctx c;
    c.tri = S.tri; c.tri_aux = S.tri_alt; c.face32 = S.face32; c.face64 = S.face64;
    c.face_rng = S.face_rng; c.face_tris = S.face_tris; c.face_box = S.face_box; c.body = S.body;
    c.n_tri = S.n_tri; c.n_face = S.n_face; c.n_body = S.n_body;
    c.band = 0.0f;
    c.S = mk3(S.tx[0], S.tx[1], S.tx[2]);
    c.pol = mk3(S.pol[0], S.pol[1], S.pol[2]);
    c.fock = S.fock32; c.res = S.res32; c.weid = S.weid; c.weid_L = S.weid_L;
    c.fock64 = S.fock64; c.res64 = S.res64; c.weid64 = S.weid64;
    c.img = S.img; c.img_pairs = S.img_pairs; c.txb = S.txb; c.occ_src = nullptr; c.occ_w = 0;
    c.face_mat = S.face_mat;
    c.txw = S.txw; c.bvh = S.bvh; c.bvh_tri = S.bvh_tri; c.bvh_top = nullptr; c.bvh_top_n = 0;
    c.cand = S.cand; c.cimg = S.cimg;
    c.n_cand = S.cand ? (S.n_cand_dev ? *S.n_cand_dev : S.n_cand) : 0;
    const int lane = threadIdx.x & 31;
    const int nch = (S.n_f + NFC - 1) / NFC;
    const v3t<DT> Sd = mk3<DT>(dvar_t<SC>(c.S.x, DS_SX), dvar_t<SC>(c.S.y, DS_SY), dvar_t<SC>(c.S.z, DS_SZ));
    double gtx[3] = {0.0, 0.0, 0.0};
    for (;;) {
        unsigned long long q = 0;
        if (lane == 0) q = atomicAdd(queue, 1ull);
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q >= (unsigned long long)n_rx) break;
        const int r = (int)q;
        const int np = min(counts[r], cap);
        const v3t<DT> Pd = mk3<DT>(DT(SC(rx[r])), DT(SC(rx[n_rx + r])), DT(SC(rx[2 * n_rx + r])));
        for (int j0 = 0; j0 < np; j0 += 32) {
            const int jj = j0 + lane;
            for (int ch = 0; ch < nch; ++ch) {
                const FreqC &fq = S.fqc[ch];
                AccAdj acc;
                acc.gE = gE; acc.n_rx = n_rx; acc.r = r; acc.f0 = ch * NFC;
                for (int k = 0; k < ND - 1; ++k) acc.g[k] = 0.0;
                for (int k = 0; k < NFC; ++k) acc.gf[k] = 0.0;
                int body = -1;
                if (jj < np) {
                    const uint64_t code = codes[(size_t)r * cap + jj];
                    const int type = (int)(code >> 56), id1 = (int)((code >> 28) & 0xFFFFFFFu),
                              id2 = (int)(code & 0xFFFFFFFu);
                    if (type == PT_LOS) adj_planar<DT>(c, 0, -1, -1, Sd, Pd, fq, acc);
                    else if (type == PT_R1) adj_planar<DT>(c, 1, id1, -1, Sd, Pd, fq, acc);
                    else if (type == PT_R2) adj_planar<DT>(c, 2, id1, id2, Sd, Pd, fq, acc);
                    else if (type == PT_R3 && c.cand && id1 < c.n_cand)
                        adj_seq3<DT>(c, id1, c.cand[id1], Sd, Pd, fq, acc);
                    else if (type == PT_RB) {
                        // reflection off a body: FP64 duals in both precisions (the
                        // FP32 chain through the specular point left errors of ~1e-3
                        // of the gradient on the test scenes)
                        const v3t<D8> S64 = mk3<D8>(dvar(c.S.x, DS_SX), dvar(c.S.y, DS_SY), dvar(c.S.z, DS_SZ));
                        const v3t<D8> P64 = mk3<D8>(D8((double)rx[r]), D8((double)rx[n_rx + r]),
                                                    D8((double)rx[2 * n_rx + r]));
                        adj_rb<D8>(c, id1, S64, P64, fq, acc);
                        body = id1;
                    }
                    else if (type == PT_CP || type == PT_CM) {
                        if (adj_creep<DT>(c, id1, type == PT_CM, id2, Sd, Pd, fq, S.enable, acc)) body = id1;
                    } else if (type == PT_WCP || type == PT_WCM) {
                        if (adj_creep<DT>(c, id1, type == PT_WCM, id2 & 15, Sd, Pd, fq, S.enable, acc, id2 >> 4))
                            body = id1;
                    }
                }
                if (body >= 0)
                    for (int k = 0; k < 4; ++k)
                        if (acc.g[k] != 0.0) atomicAdd(&g_body[4 * body + k], acc.g[k]);
                for (int k = 0; k < 3; ++k) gtx[k] += acc.g[DS_SX + k];
                for (int f = 0; f < fq.nf; ++f) {
                    const double v = warp_sum(acc.gf[f]);
                    if (lane == 0 && v != 0.0) atomicAdd(&g_f[ch * NFC + f], v);
                }
            }
        }
    }
    for (int k = 0; k < 3; ++k) {
        const double v = warp_sum(gtx[k]);
        if (lane == 0 && v != 0.0) atomicAdd(&g_tx[k], v);
    }
}

int launch_adjoint(const DevScene &S, const float *rx_soa, int n_rx, const uint64_t *codes, const int32_t *counts,
                   int cap, const float *grad_e, double *g_body, double *g_tx, double *g_f,
                   unsigned long long *queue, int precision, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess && S.n_body > 0) e = cudaMemsetAsync(g_body, 0, sizeof(double) * 4 * S.n_body, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g_tx, 0, sizeof(double) * 3, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g_f, 0, sizeof(double) * S.n_f, st);
    if (e == cudaSuccess && n_rx > 0) {
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        long long need = ((long long)n_rx + 3) / 4;
        int grid = (int)(need < 4LL * nsm ? need : 4LL * nsm);
        if (precision == RT_PREC_FP64)
            k_adjoint<D8><<<grid, 128, 0, st>>>(S, rx_soa, n_rx, codes, counts, cap, grad_e, g_body, g_tx, g_f, queue);
        else
            k_adjoint<F8><<<grid, 128, 0, st>>>(S, rx_soa, n_rx, codes, counts, cap, grad_e, g_body, g_tx, g_f, queue);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_error(std::string("adjoint: ") + cudaGetErrorString(e));
        return RT_ERR_CUDA;
    }
    return RT_OK;
}

}  // namespace creep
