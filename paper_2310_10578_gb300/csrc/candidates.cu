// candidates.cu -- the ray launch of the large-scene mode on the device.
//
// The paper's own path search is a ray tracer (Sec. III, BVH-accelerated);
// for order-3 reflections among ~100k faces this library takes candidate
// face sequences from a forward launch from the transmitter and validates
// each one exactly per receiver (the planar class kernel).  The launch rule
// (shared with the host launch in bvh.cu and with the oracle): n_rays
// directions of the spherical Fibonacci lattice; each ray is reflected
// specularly at the nearest triangle hit (Moller--Trumbore, parameter >
// 1e-9, the face it leaves excluded, equal parameters to the lower triangle
// index) up to max_order times; every prefix of its face sequence is a
// candidate; the distinct sequences sorted by (order, faces).
//
// Here: k_ray_launch, one thread per ray, walks the scene's triangle BVH
// (FP32 box tests, conservative on the padded boxes; FP64 triangle tests);
// this file is compiled without FMA contraction, so every FP64 operation
// rounds as in the host code (-ffp-contract=off) and both launches trace
// bit-identical rays from the same host-made directions and face normals.
// k_cand_finish, one block, sorts the (order, faces) keys in shared memory
// (bitonic), keeps the distinct ones in order (block scan) and writes the
// list with the source's FP64 images after each reflection, as
// rt_set_candidates would upload them.  Its length goes to device memory,
// where the class kernels read it: no host round trip.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace creep {

namespace {

constexpr int FINISH_THREADS = 1024;
constexpr unsigned long long KEY_NONE = ~0ull;

struct D3 { double x, y, z; };
__device__ __forceinline__ D3 d3(double x, double y, double z) { D3 r; r.x = x; r.y = y; r.z = z; return r; }
__device__ __forceinline__ D3 sub(D3 a, D3 b) { return d3(a.x - b.x, a.y - b.y, a.z - b.z); }
// the host's expression trees: ((a.x b.x + a.y b.y) + a.z b.z), a.y b.z - a.z b.y, ...
__device__ __forceinline__ double dotd(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 crossd(D3 a, D3 b) {
    return d3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// nearest-hit parameter of the ray o + t d with the closed triangle, or -1
__device__ double ray_tri_d(D3 o, D3 d, D3 v0, D3 v1, D3 v2) {
    D3 e1 = sub(v1, v0), e2 = sub(v2, v0);
    D3 p = crossd(d, e2);
    double det = dotd(e1, p);
    if (fabs(det) < 1e-14) return -1.0;
    double inv = 1.0 / det;
    D3 sv = sub(o, v0);
    double u = dotd(sv, p) * inv;
    if (u < 0.0 || u > 1.0) return -1.0;
    D3 q = crossd(sv, e1);
    double v = dotd(d, q) * inv;
    if (v < 0.0 || u + v > 1.0) return -1.0;
    return dotd(e2, q) * inv;
}

// the ray's parameter interval [0, tmax] meets the box?  In FP32 on the
// rounded ray: conservative, since the node
// boxes are padded outwards by 1e-4 m + 1e-6 of the coordinate, far beyond
// the rounding of the ray and of this test over the scene's extent; tmax is
// rounded up.  It only prunes the walk: every box holding a triangle whose
// FP64 hit parameter is <= tmax is kept, so the nearest hit is the FP64 one.
__device__ __forceinline__ bool ray_box_f(const float o[3], const float d[3], float4 lo, float4 hi, float tmax) {
    float t0 = 0.0f, t1 = tmax;
    const float bl[3] = {lo.x, lo.y, lo.z}, bh[3] = {hi.x, hi.y, hi.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (d[k] == 0.0f) {
            if (o[k] < bl[k] || o[k] > bh[k]) return false;
            continue;
        }
        const float inv = 1.0f / d[k];
        float a = (bl[k] - o[k]) * inv, b = (bh[k] - o[k]) * inv;
        if (a > b) { const float w = a; a = b; b = w; }
        t0 = fmaxf(t0, a);
        t1 = fminf(t1, b);
        if (t0 > t1) return false;
    }
    return true;
}

__device__ __forceinline__ D3 vtx(const float4 *tri, int t, int k) {
    const float4 v = tri[3 * t + k];
    return d3(v.x, v.y, v.z);
}

// key of a prefix: order (2 bits), then face + 1 of each slot (20 bits, 0 = none)
__device__ __forceinline__ unsigned long long seq_key(int k, const int fs[3]) {
    return ((unsigned long long)k << 60) | ((unsigned long long)(fs[0] + 1) << 40) |
           ((unsigned long long)(fs[1] + 1) << 20) | (unsigned long long)(fs[2] + 1);
}

__global__ void __launch_bounds__(32) k_ray_launch(const float4 *__restrict__ tri, const float4 *__restrict__ bvh,
                                                    const int *__restrict__ bvh_tri, const double *__restrict__ fn,
                                                    const double *__restrict__ dir, double ox, double oy, double oz,
                                                    int n_rays, int max_order, unsigned long long *__restrict__ keys,
                                                    int *__restrict__ overflow) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rays) return;
    for (int k = 0; k < max_order; ++k) keys[(size_t)i * max_order + k] = KEY_NONE;
    D3 o = d3(ox, oy, oz), d = d3(dir[3 * (size_t)i], dir[3 * (size_t)i + 1], dir[3 * (size_t)i + 2]);
    int fs[3] = {-1, -1, -1}, last = -1;
    int stack[64];
    for (int k = 0; k < max_order; ++k) {
        double best = INFINITY;
        int bt = -1, sp = 0;
        const float of[3] = {(float)o.x, (float)o.y, (float)o.z}, df[3] = {(float)d.x, (float)d.y, (float)d.z};
        stack[sp++] = 0;
        while (sp > 0) {
            const int nd = stack[--sp];
            const float4 lo = bvh[2 * nd], hi = bvh[2 * nd + 1];
            if (!ray_box_f(of, df, lo, hi, __double2float_ru(best))) continue;
            const int first = __float_as_int(lo.w), count = __float_as_int(hi.w);
            if (count == 0) {
                if (sp + 2 > 64) { atomicExch(overflow, 1); continue; }    // (the build is far shallower)
                stack[sp++] = first;
                stack[sp++] = first + 1;
                continue;
            }
            for (int j = first; j < first + count; ++j) {
                const int t = bvh_tri[j];
                if (__float_as_int(tri[3 * t].w) == last) continue;
                const double h = ray_tri_d(o, d, vtx(tri, t, 0), vtx(tri, t, 1), vtx(tri, t, 2));
                if (h > 1e-9 && (h < best || (h == best && t < bt))) { best = h; bt = t; }
            }
        }
        if (bt < 0) break;
        const int f = __float_as_int(tri[3 * bt].w);
        fs[k] = f;
        keys[(size_t)i * max_order + k] = seq_key(k + 1, fs);
        const D3 n = d3(fn[3 * (size_t)f], fn[3 * (size_t)f + 1], fn[3 * (size_t)f + 2]);
        o = d3(o.x + d.x * best, o.y + d.y * best, o.z + d.z * best);
        const double dn = 2.0 * dotd(d, n);
        d = d3(d.x - n.x * dn, d.y - n.y * dn, d.z - n.z * dn);
        last = f;
    }
}

// One block: sort n (a power of two, >= FINISH_THREADS) keys, keep the
// distinct valid ones in order, write the list and its images.
__global__ void __launch_bounds__(FINISH_THREADS) k_cand_finish(const unsigned long long *__restrict__ keys,
                                                                int n_keys, int n, const dq4 *__restrict__ face64,
                                                                double tx, double ty, double tz,
                                                                int4 *__restrict__ cand, float4 *__restrict__ cimg,
                                                                int *__restrict__ n_out) {
    extern __shared__ unsigned long long sk[];
    __shared__ int s_warp[FINISH_THREADS / 32];
    const int tid = threadIdx.x;
    for (int i = tid; i < n; i += FINISH_THREADS) sk[i] = i < n_keys ? keys[i] : KEY_NONE;
    __syncthreads();
    // bitonic sort, ascending
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < n; i += FINISH_THREADS) {
                const int l = i ^ j;
                if (l > i) {
                    const unsigned long long a = sk[i], b = sk[l];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) { sk[i] = b; sk[l] = a; }
                }
            }
            __syncthreads();
        }
    }
    // distinct valid keys: each thread a run of per consecutive slots
    const int per = n / FINISH_THREADS;
    const int b0 = tid * per;
    int mine = 0;
    for (int i = b0; i < b0 + per; ++i)
        mine += (sk[i] != KEY_NONE && (i == 0 || sk[i] != sk[i - 1])) ? 1 : 0;
    // exclusive block scan of the runs' counts
    const int lane = tid & 31, w = tid >> 5;
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_warp[w] = incl;
    __syncthreads();
    if (w == 0) {
        int v = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        s_warp[lane] = v;          // inclusive prefix of the warps' totals
    }
    __syncthreads();
    int pos = (w > 0 ? s_warp[w - 1] : 0) + incl - mine;
    if (tid == FINISH_THREADS - 1) *n_out = pos + mine;
    for (int i = b0; i < b0 + per; ++i) {
        const unsigned long long key = sk[i];
        if (key == KEY_NONE || (i > 0 && key == sk[i - 1])) continue;
        const int k = (int)(key >> 60);
        const int f[3] = {(int)((key >> 40) & 0xFFFFFull) - 1, (int)((key >> 20) & 0xFFFFFull) - 1,
                          (int)(key & 0xFFFFFull) - 1};
        cand[pos] = make_int4(f[0], f[1], f[2], k);
        // the source's image after each reflection (FP64, as hi + lo floats)
        double X[3] = {tx, ty, tz};
        for (int m = 0; m < 3; ++m) {
            float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
            if (m < k) {
                const dq4 F = face64[f[m]];
                const double dist = F.x * X[0] + F.y * X[1] + F.z * X[2] - F.w;
                X[0] = X[0] - F.x * (2.0 * dist);
                X[1] = X[1] - F.y * (2.0 * dist);
                X[2] = X[2] - F.z * (2.0 * dist);
                h = make_float4((float)X[0], (float)X[1], (float)X[2], 0.f);
                l = make_float4((float)(X[0] - (double)h.x), (float)(X[1] - (double)h.y), (float)(X[2] - (double)h.z), 0.f);
            }
            cimg[6 * (size_t)pos + 2 * m] = h;
            cimg[6 * (size_t)pos + 2 * m + 1] = l;
        }
        ++pos;
    }
}

}  // namespace

int launch_ray_candidates(const float4 *tri, const float4 *bvh, const int *bvh_tri, const dq4 *face64,
                          const double tx[3], int n_rays, int max_order, const DevCandBufs &B, cudaStream_t st) {
    const int n_keys = n_rays * max_order;
    int n = FINISH_THREADS;
    while (n < n_keys) n <<= 1;
    const size_t smem = sizeof(unsigned long long) * (size_t)n;
    cudaError_t e = cudaFuncSetAttribute(k_cand_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // B.n_cand[1]: set if a traversal stack overflowed (the build is far
    // shallower than the stack; reported by rt_get_candidates)
    if (e == cudaSuccess) e = cudaMemsetAsync(B.n_cand + 1, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        // one ray per thread, 32-thread blocks: a few thousand rays still
        // spread over most SMs
        k_ray_launch<<<(n_rays + 31) / 32, 32, 0, st>>>(tri, bvh, bvh_tri, B.fn, B.dir, tx[0], tx[1], tx[2], n_rays,
                                                         max_order, B.keys, B.n_cand + 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_cand_finish<<<1, FINISH_THREADS, smem, st>>>(B.keys, n_keys, n, face64, tx[0], tx[1], tx[2], B.cand, B.cimg,
                                                       B.n_cand);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_error(std::string("device ray launch: ") + cudaGetErrorString(e));
        return RT_ERR_CUDA;
    }
    return RT_OK;
}

}  // namespace creep
