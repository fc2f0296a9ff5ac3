// bvh.cu -- host side of the large-scene mode: the triangle BVH that the
// visibility tests traverse on the device, and the candidate face sequences
// of a ray launch from the transmitter (orders 1-3), which the planar class
// kernel then validates per receiver by the image method.
//
// BVH: binary, median split of the triangle centroids along the longest
// axis of their bounds, leaves of at most BVH_LEAF triangles (depth <=
// ceil(log2(n / BVH_LEAF)) + 1 <= 32 for any n < 2^31), nodes numbered
// breadth first (the top levels first).  Node i is two float4: (box min,
// first) and (box max, count); count > 0: a leaf over bvh_tri[first ..
// first + count); count == 0: an inner node with children first and
// first + 1.  The boxes are the triangles' float bounds widened
// outwards by 1e-4 m + 1e-6 of the coordinate, so an FP32 or FP64 slab test
// with its own rounding never drops a triangle that the exact test would hit.
//
// Ray launch: n_rays directions of the spherical Fibonacci lattice,
// z_i = 1 - (2 i + 1) / n, phi_i = i pi (3 - sqrt 5); each ray is reflected
// specularly at the nearest triangle hit (Moller-Trumbore, parameter > 1e-9,
// the face it leaves excluded, equal parameters to the lower triangle index,
// curved bodies ignored) up to max_order times, and every prefix of its face
// sequence is a candidate.  The distinct sequences are sorted by order, then
// faces.  Face normals for the bounce: the unit normal of each face's first
// triangle, (v1 - v0) x (v2 - v0) times the reciprocal of its length.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace creep {

namespace {

constexpr int BVH_LEAF = 4;

struct V3 { double x, y, z; };
inline V3 v3(double x, double y, double z) { return V3{x, y, z}; }
inline V3 operator-(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
inline double dotv(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 crossv(V3 a, V3 b) { return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }

inline float pad_lo(float v) { return nextafterf(v - (float)(1e-4 + 1e-6 * fabs((double)v)), -INFINITY); }
inline float pad_hi(float v) { return nextafterf(v + (float)(1e-4 + 1e-6 * fabs((double)v)), INFINITY); }

inline float int_bits(int i) {
    float f;
    memcpy(&f, &i, sizeof(f));
    return f;
}
inline int float_bits(float f) {
    int i;
    memcpy(&i, &f, sizeof(i));
    return i;
}

struct Builder {
    const float *tri;
    std::vector<int> idx;
    std::vector<float> cen;     // [n][3]
    std::vector<float4> nodes;

    void bounds(int lo, int hi, float bmin[3], float bmax[3]) const {
        for (int k = 0; k < 3; ++k) { bmin[k] = INFINITY; bmax[k] = -INFINITY; }
        for (int i = lo; i < hi; ++i) {
            const float *v = tri + 9 * (size_t)idx[i];
            for (int c = 0; c < 3; ++c)
                for (int k = 0; k < 3; ++k) {
                    bmin[k] = fminf(bmin[k], v[3 * c + k]);
                    bmax[k] = fmaxf(bmax[k], v[3 * c + k]);
                }
        }
    }
    void set(int node, int lo, int hi, int first, int count) {
        float bmin[3], bmax[3];
        bounds(lo, hi, bmin, bmax);
        nodes[2 * node] = make_float4(pad_lo(bmin[0]), pad_lo(bmin[1]), pad_lo(bmin[2]), int_bits(first));
        nodes[2 * node + 1] = make_float4(pad_hi(bmax[0]), pad_hi(bmax[1]), pad_hi(bmax[2]), int_bits(count));
    }
    // node covers idx[lo, hi)
    void build(int node, int lo, int hi) {
        if (hi - lo <= BVH_LEAF) {
            set(node, lo, hi, lo, hi - lo);
            return;
        }
        float cmin[3] = {INFINITY, INFINITY, INFINITY}, cmax[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int i = lo; i < hi; ++i)
            for (int k = 0; k < 3; ++k) {
                cmin[k] = fminf(cmin[k], cen[3 * (size_t)idx[i] + k]);
                cmax[k] = fmaxf(cmax[k], cen[3 * (size_t)idx[i] + k]);
            }
        int ax = 0;
        for (int k = 1; k < 3; ++k)
            if (cmax[k] - cmin[k] > cmax[ax] - cmin[ax]) ax = k;
        const int mid = lo + (hi - lo) / 2;
        std::nth_element(idx.begin() + lo, idx.begin() + mid, idx.begin() + hi, [&](int a, int b) {
            const float ca = cen[3 * (size_t)a + ax], cb = cen[3 * (size_t)b + ax];
            return ca < cb || (ca == cb && a < b);
        });
        const int left = (int)nodes.size() / 2;
        nodes.resize(nodes.size() + 4);
        set(node, lo, hi, left, 0);
        build(left, lo, mid);
        build(left + 1, mid, hi);
    }
};

// nearest hit of the ray o + t d with the closed triangle: parameter or -1
inline double ray_tri(V3 o, V3 d, V3 v0, V3 v1, V3 v2) {
    V3 e1 = v1 - v0, e2 = v2 - v0;
    V3 p = crossv(d, e2);
    double det = dotv(e1, p);
    if (fabs(det) < 1e-14) return -1.0;
    double inv = 1.0 / det;
    V3 sv = o - v0;
    double u = dotv(sv, p) * inv;
    if (u < 0.0 || u > 1.0) return -1.0;
    V3 q = crossv(sv, e1);
    double v = dotv(d, q) * inv;
    if (v < 0.0 || u + v > 1.0) return -1.0;
    return dotv(e2, q) * inv;
}

// the ray's parameter interval inside the box, or false
inline bool ray_box(V3 o, V3 d, const float4 &lo, const float4 &hi, double tmax) {
    double t0 = 0.0, t1 = tmax;
    const double os[3] = {o.x, o.y, o.z}, ds[3] = {d.x, d.y, d.z};
    const double bl[3] = {lo.x, lo.y, lo.z}, bh[3] = {hi.x, hi.y, hi.z};
    for (int k = 0; k < 3; ++k) {
        if (ds[k] == 0.0) {
            if (os[k] < bl[k] || os[k] > bh[k]) return false;
            continue;
        }
        double a = (bl[k] - os[k]) / ds[k], b = (bh[k] - os[k]) / ds[k];
        if (a > b) std::swap(a, b);
        t0 = std::max(t0, a);
        t1 = std::min(t1, b);
        if (t0 > t1) return false;
    }
    return true;
}

}  // namespace

void bvh_build(const float *tri, int n_tri, std::vector<float4> &nodes, std::vector<int> &order) {
    nodes.clear();
    order.clear();
    if (n_tri <= 0) return;
    Builder B;
    B.tri = tri;
    B.idx.resize(n_tri);
    B.cen.resize(3 * (size_t)n_tri);
    for (int t = 0; t < n_tri; ++t) {
        B.idx[t] = t;
        const float *v = tri + 9 * (size_t)t;
        for (int k = 0; k < 3; ++k) B.cen[3 * (size_t)t + k] = (v[k] + v[3 + k] + v[6 + k]) * (1.0f / 3.0f);
    }
    B.nodes.resize(2);
    B.build(0, 0, n_tri);
    // renumber the nodes breadth first (children pairs stay adjacent), so
    // that the top levels are the array's first nodes: the class kernels
    // stage that prefix (the top treelet) in shared memory
    const size_t n_nodes = B.nodes.size() / 2;
    std::vector<int> bfs;                   // bfs[new id] = old id
    bfs.reserve(n_nodes);
    std::vector<int> new_id(n_nodes, -1);
    bfs.push_back(0);
    new_id[0] = 0;
    for (size_t h = 0; h < bfs.size(); ++h) {
        const int old = bfs[h];
        if (float_bits(B.nodes[2 * (size_t)old + 1].w) == 0) {       // inner node: children first, first + 1
            const int c = float_bits(B.nodes[2 * (size_t)old].w);
            new_id[c] = (int)bfs.size();
            bfs.push_back(c);
            new_id[c + 1] = (int)bfs.size();
            bfs.push_back(c + 1);
        }
    }
    nodes.assign(2 * n_nodes, make_float4(0.f, 0.f, 0.f, 0.f));
    for (size_t k = 0; k < n_nodes; ++k) {
        float4 lo = B.nodes[2 * (size_t)bfs[k]], hi = B.nodes[2 * (size_t)bfs[k] + 1];
        if (float_bits(hi.w) == 0) lo.w = int_bits(new_id[float_bits(lo.w)]);
        nodes[2 * k] = lo;
        nodes[2 * k + 1] = hi;
    }
    order.swap(B.idx);
}

void ray_face_normals(const float *tri, const int *tri_face, int n_tri, int n_face, std::vector<double> &fn) {
    fn.assign(3 * (size_t)n_face, 0.0);
    std::vector<char> has(n_face, 0);
    for (int t = 0; t < n_tri; ++t) {
        int f = tri_face[t];
        if (has[f]) continue;
        has[f] = 1;
        const float *v = tri + 9 * (size_t)t;
        V3 c = crossv(v3(v[3], v[4], v[5]) - v3(v[0], v[1], v[2]), v3(v[6], v[7], v[8]) - v3(v[0], v[1], v[2]));
        double inv = 1.0 / sqrt(dotv(c, c));
        fn[3 * (size_t)f] = c.x * inv;
        fn[3 * (size_t)f + 1] = c.y * inv;
        fn[3 * (size_t)f + 2] = c.z * inv;
    }
}

void ray_directions(int n_rays, std::vector<double> &dir) {
    dir.resize(3 * (size_t)n_rays);
    const double golden = M_PI * (3.0 - sqrt(5.0));
    for (int i = 0; i < n_rays; ++i) {
        double z = 1.0 - (2.0 * i + 1.0) / n_rays;
        double r = sqrt(std::max(0.0, 1.0 - z * z));
        double ph = golden * i;
        dir[3 * (size_t)i] = r * cos(ph);
        dir[3 * (size_t)i + 1] = r * sin(ph);
        dir[3 * (size_t)i + 2] = z;
    }
}

int ray_launch(const float *tri, const int *tri_face, int n_tri, int n_face, const std::vector<float4> &nodes,
               const std::vector<int> &order, const double tx[3], int n_rays, int max_order,
               std::vector<int> &seq) {
    seq.clear();
    if (n_tri <= 0 || n_rays <= 0 || max_order < 1) return 0;
    // face normals from each face's first triangle
    std::vector<double> fnv;
    ray_face_normals(tri, tri_face, n_tri, n_face, fnv);
    std::vector<V3> fn(n_face);
    for (int f = 0; f < n_face; ++f) fn[f] = v3(fnv[3 * (size_t)f], fnv[3 * (size_t)f + 1], fnv[3 * (size_t)f + 2]);
    std::vector<double> dirs;
    ray_directions(n_rays, dirs);
    auto vert = [&](int t, int k) {
        const float *v = tri + 9 * (size_t)t + 3 * k;
        return v3(v[0], v[1], v[2]);
    };
    std::vector<int> all;
    all.reserve(3 * (size_t)n_rays * max_order);
    int stack[64];
    for (int i = 0; i < n_rays; ++i) {
        V3 o = v3(tx[0], tx[1], tx[2]), d = v3(dirs[3 * (size_t)i], dirs[3 * (size_t)i + 1], dirs[3 * (size_t)i + 2]);
        int fs[3] = {-1, -1, -1}, last = -1;
        for (int k = 0; k < max_order && k < 3; ++k) {
            double best = INFINITY;
            int bt = -1, sp = 0;
            stack[sp++] = 0;
            while (sp > 0) {
                const int nd = stack[--sp];
                const float4 lo = nodes[2 * nd], hi = nodes[2 * nd + 1];
                if (!ray_box(o, d, lo, hi, best)) continue;
                const int first = float_bits(lo.w), count = float_bits(hi.w);
                if (count == 0) {
                    stack[sp++] = first;
                    stack[sp++] = first + 1;
                    continue;
                }
                for (int j = first; j < first + count; ++j) {
                    const int t = order[j];
                    if (tri_face[t] == last) continue;
                    double h = ray_tri(o, d, vert(t, 0), vert(t, 1), vert(t, 2));
                    if (h > 1e-9 && (h < best || (h == best && t < bt))) { best = h; bt = t; }
                }
            }
            if (bt < 0) break;
            const int f = tri_face[bt];
            fs[k] = f;
            for (int m = 0; m < 3; ++m) all.push_back(m <= k ? fs[m] : -1);
            const V3 n = fn[f];
            o = v3(o.x + d.x * best, o.y + d.y * best, o.z + d.z * best);
            const double dn = 2.0 * dotv(d, n);
            d = v3(d.x - n.x * dn, d.y - n.y * dn, d.z - n.z * dn);
            last = f;
        }
    }
    const size_t n_all = all.size() / 3;
    std::vector<int> ix(n_all);
    for (size_t a = 0; a < n_all; ++a) ix[a] = (int)a;
    auto key = [&](int a) {
        const int *x = &all[3 * (size_t)a];
        return std::make_tuple((x[0] >= 0) + (x[1] >= 0) + (x[2] >= 0), x[0], x[1], x[2]);
    };
    std::sort(ix.begin(), ix.end(), [&](int a, int b) { return key(a) < key(b); });
    for (size_t a = 0; a < n_all; ++a) {
        if (a > 0 && key(ix[a]) == key(ix[a - 1])) continue;
        for (int m = 0; m < 3; ++m) seq.push_back(all[3 * (size_t)ix[a] + m]);
    }
    return (int)(seq.size() / 3);
}

}  // namespace creep
