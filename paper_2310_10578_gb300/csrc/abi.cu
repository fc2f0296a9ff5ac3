// abi.cu -- the C ABI (include/creep.h): scene management, argument checks,
// per-device Fock--Pekeris table cache, launches.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace creep {

static thread_local std::string g_err = "no error";
void set_error(const std::string &msg) { g_err = msg; }

// ---------------------------------------------------------------- table cache
struct DevTable {
    float4 *fock32 = nullptr;
    double2 *fock64 = nullptr;
    float4 *res32 = nullptr;
    dq4 *res64 = nullptr;
    float *weid = nullptr;
    double *weid64 = nullptr;
    float weid_L = 0.f;
    FockHost host;
};
static std::mutex g_table_mu;
static std::map<int, DevTable> g_tables;

// Weideman (1994) coefficients of w(z): a_n = (1/2M) sum_k f(t_k) cos(n k pi/M),
// t_k = L tan(k pi / 2M), f(t) = e^{-t^2} (L^2 + t^2), M = 2N, L = (N / sqrt 2)^{1/2}.
static void weideman(std::vector<double> &a, double *L) {
    const int N = WEIDEMAN_N, M = 2 * N;
    *L = sqrt(N / sqrt(2.0));
    a.assign(N, 0.0);
    for (int n = 1; n <= N; ++n) {
        double s = 0.0;
        for (int k = -M + 1; k <= M - 1; ++k) {
            double t = *L * tan(k * M_PI / (2.0 * M));
            s += exp(-t * t) * (*L * *L + t * t) * cos(n * k * M_PI / M);
        }
        a[n - 1] = s / (2.0 * M);
    }
}

static int get_table(DevTable **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e)); return RT_ERR_CUDA; }
    std::lock_guard<std::mutex> lk(g_table_mu);
    auto it = g_tables.find(dev);
    if (it != g_tables.end()) { *out = &it->second; return RT_OK; }
    DevTable T;
    int rc = build_fock_table(&T.host);
    if (rc != RT_OK) return rc;
    std::vector<float4> f32((FOCK_N + FOCK_NP) * 2);
    std::vector<double2> f64(FOCK_N * 4);
    for (int j = 0; j < FOCK_N; ++j)
        for (int k = 0; k < 2; ++k) {
            const double *q = &T.host.tab[(j * 2 + k) * 4];
            f32[j * 2 + k] = make_float4((float)q[0], (float)q[1], (float)(q[2] * XI_STEP), (float)(q[3] * XI_STEP));
            f64[(j * 2 + k) * 2] = make_double2(q[0], q[1]);
            f64[(j * 2 + k) * 2 + 1] = make_double2(q[2], q[3]);
        }
    for (int j = 0; j < FOCK_NP; ++j)              // the FP32 second segment: P, h P'
        for (int k = 0; k < 2; ++k) {
            const double *q = &T.host.tabp[(j * 2 + k) * 4];
            f32[(FOCK_N + j) * 2 + k] =
                make_float4((float)q[0], (float)q[1], (float)(q[2] * XI_STEP), (float)(q[3] * XI_STEP));
        }
    std::vector<float4> r32(FOCK_NRES * 2);
    std::vector<dq4> r64(FOCK_NRES * 2);
    const double s3 = sqrt(3.0) / 2.0;
    for (int n = 0; n < FOCK_NRES; ++n) {
        double al = T.host.res[n], cs = T.host.res[FOCK_NRES + n], be = T.host.res[2 * FOCK_NRES + n],
               ch = T.host.res[3 * FOCK_NRES + n];
        r32[2 * n] = make_float4((float)(al * s3), (float)(al / 2), (float)cs, 0.f);
        r32[2 * n + 1] = make_float4((float)(be * s3), (float)(be / 2), (float)ch, 0.f);
        r64[2 * n] = make_dq4(al * s3, al / 2, cs, 0.0);
        r64[2 * n + 1] = make_dq4(be * s3, be / 2, ch, 0.0);
    }
    std::vector<double> wa;
    double L;
    weideman(wa, &L);
    std::vector<float> wf(wa.begin(), wa.end());
    T.weid_L = (float)L;
#define CKT(x)                                                                         \
    do {                                                                               \
        cudaError_t e_ = (x);                                                          \
        if (e_ != cudaSuccess) { set_error(std::string(#x) + ": " + cudaGetErrorString(e_)); return RT_ERR_CUDA; } \
    } while (0)
    CKT(cudaMalloc(&T.fock32, sizeof(float4) * f32.size()));
    CKT(cudaMalloc(&T.fock64, sizeof(double2) * f64.size()));
    CKT(cudaMalloc(&T.res32, sizeof(float4) * r32.size()));
    CKT(cudaMalloc(&T.res64, sizeof(dq4) * r64.size()));
    CKT(cudaMalloc(&T.weid, sizeof(float) * WEIDEMAN_N));
    CKT(cudaMalloc(&T.weid64, sizeof(double) * WEIDEMAN_N));
    CKT(cudaMemcpy(T.fock32, f32.data(), sizeof(float4) * f32.size(), cudaMemcpyHostToDevice));
    CKT(cudaMemcpy(T.fock64, f64.data(), sizeof(double2) * f64.size(), cudaMemcpyHostToDevice));
    CKT(cudaMemcpy(T.res32, r32.data(), sizeof(float4) * r32.size(), cudaMemcpyHostToDevice));
    CKT(cudaMemcpy(T.res64, r64.data(), sizeof(dq4) * r64.size(), cudaMemcpyHostToDevice));
    CKT(cudaMemcpy(T.weid, wf.data(), sizeof(float) * WEIDEMAN_N, cudaMemcpyHostToDevice));
    CKT(cudaMemcpy(T.weid64, wa.data(), sizeof(double) * WEIDEMAN_N, cudaMemcpyHostToDevice));
    g_tables[dev] = T;
    *out = &g_tables[dev];
    return RT_OK;
}

}  // namespace creep

using namespace creep;

struct rt_scene {
    int device = 0;
    int n_tri = 0, n_face = 0, n_body = 0;
    std::vector<float> tri;             // [n_tri][9]
    std::vector<int> tri_face;
    std::vector<FaceHost> faces;
    std::vector<rt_body> bodies;
    // device copies
    float4 *d_tri = nullptr, *d_aux = nullptr, *d_face32 = nullptr, *d_body = nullptr;
    dq4 *d_face64 = nullptr;
    int2 *d_face_rng = nullptr;
    int *d_face_tris = nullptr;
    double *d_freq = nullptr;
    FreqC *d_fqc = nullptr;            // [RT_MAX_FREQS / NFC] per-chunk frequency constants
    float4 *d_img = nullptr;            // source images, see DevScene::img
    float4 *d_txb = nullptr;            // source-side body frames, see DevScene::txb
    float4 *d_txw = nullptr;            // the same for each face's source image, see DevScene::txw
    float4 *d_face_mat = nullptr;       // face materials, see DevScene::face_mat
    float4 *d_face_box = nullptr;       // per face its culling box, see DevScene::face_box
    bool any_dielectric = false;
    // large-scene mode: the triangle BVH (host copy for the ray launch; on the
    // device above BVH_MIN_TRI triangles) and the candidate face sequences
    std::vector<float4> h_bvh;
    std::vector<int> h_bvh_tri;
    float4 *d_bvh = nullptr;
    int *d_bvh_tri = nullptr;
    std::vector<int> cand;              // [n_cand][3]
    int4 *d_cand = nullptr;
    float4 *d_cimg = nullptr;           // [n_cand][3][2]
    int n_cand = 0;
    // a candidate list built on the device (rt_candidates_device): in use
    // while cand_dev is set (rt_set_tx and rt_set_candidates clear it); its
    // length lives in device memory (dcb.n_cand[0])
    bool cand_dev = false;
    DevCandBufs dcb = {};
    int dcb_rays = 0;                   // rays whose directions dcb.dir holds
    float4 *d_lbvh = nullptr;           // the BVH for the launch when the scene has too few triangles for d_bvh
    int *d_lbvh_tri = nullptr;
    cudaStream_t cand_stream = nullptr;
    // received power (rt_set_tx_power, rt_power_dbm): the transmitter's power
    // and per frequency P_t + 20 log10(lambda / 4 pi) on the device
    float power_dbm = 0.0f;
    float *d_pc0 = nullptr;             // [RT_MAX_FREQS]
    unsigned long long *d_esc = nullptr;   // [CTR_N]: FP64-decided candidates, then one work queue per launch
    DevTable *table = nullptr;
    // state
    bool tx_set = false, f_set = false;
    unsigned tx_version = 0;            // incremented by every rt_set_tx
    double tri_scale = 1.0;             // largest |coordinate| of the triangles (at least 1)
    float plan[4] = {0.f, 0.f, 0.f, 0.f};   // floor plan of the triangles: x min, x max, y min, y max
    float tx[3], pol[3];
    std::vector<double> freqs;
    float band_len = 0.f;
    // host-io scratch (rt_evaluate_host)
    float *io_rx = nullptr, *io_e = nullptr;
    uint32_t *io_fl = nullptr;
    size_t io_cap = 0;
    cudaStream_t last_stream = nullptr;
    int last_launches = 0;
    int shape[3] = {4, 4, 4};           // tile shape of rt_evaluate (rt_set_shape / rt_tune)
};

#define CK(x)                                                                              \
    do {                                                                                   \
        cudaError_t e_ = (x);                                                              \
        if (e_ != cudaSuccess) {                                                           \
            set_error(std::string(#x) + ": " + cudaGetErrorString(e_));                    \
            return RT_ERR_CUDA;                                                            \
        }                                                                                  \
    } while (0)

static bool fin32(float x) { return isfinite(x); }

static int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_error(buf);
    return code;
}

static void free_scene(rt_scene *s) {
    cudaFree(s->d_tri); cudaFree(s->d_aux); cudaFree(s->d_face32); cudaFree(s->d_body);
    cudaFree(s->d_face64); cudaFree(s->d_face_rng); cudaFree(s->d_face_tris); cudaFree(s->d_freq); cudaFree(s->d_fqc);
    cudaFree(s->d_esc); cudaFree(s->io_rx); cudaFree(s->io_e); cudaFree(s->io_fl); cudaFree(s->d_img); cudaFree(s->d_txb);
    cudaFree(s->d_txw); cudaFree(s->d_bvh); cudaFree(s->d_bvh_tri); cudaFree(s->d_cand); cudaFree(s->d_cimg);
    cudaFree(s->d_face_mat); cudaFree(s->d_face_box);
    cudaFree(s->dcb.dir); cudaFree(s->dcb.fn); cudaFree(s->dcb.keys); cudaFree(s->dcb.cand); cudaFree(s->dcb.cimg);
    cudaFree(s->dcb.n_cand); cudaFree(s->d_lbvh); cudaFree(s->d_lbvh_tri); cudaFree(s->d_pc0);
}

// distance from point p to the solid of body b (0 if inside)
static double dist_to_body(const double p[3], const rt_body &b) {
    if (b.type == RT_BODY_SPHERE) {
        double d = sqrt((p[0] - b.c[0]) * (p[0] - b.c[0]) + (p[1] - b.c[1]) * (p[1] - b.c[1]) + (p[2] - b.c[2]) * (p[2] - b.c[2]));
        return d > b.a ? d - b.a : 0.0;
    }
    double rho = sqrt((p[0] - b.c[0]) * (p[0] - b.c[0]) + (p[1] - b.c[1]) * (p[1] - b.c[1]));
    double dr = rho > b.a ? rho - b.a : 0.0;
    double dz = p[2] < b.c[2] ? b.c[2] - p[2] : (p[2] > b.c[2] + b.h ? p[2] - b.c[2] - b.h : 0.0);
    return sqrt(dr * dr + dz * dz);
}

static bool bodies_overlap(const rt_body &A, const rt_body &B) {
    if (A.type == RT_BODY_SPHERE && B.type == RT_BODY_SPHERE) {
        double c[3] = {A.c[0], A.c[1], A.c[2]};
        return dist_to_body(c, B) < A.a;
    }
    if (A.type == RT_BODY_SPHERE || B.type == RT_BODY_SPHERE) {
        const rt_body &S = A.type == RT_BODY_SPHERE ? A : B, &C = A.type == RT_BODY_SPHERE ? B : A;
        double c[3] = {S.c[0], S.c[1], S.c[2]};
        return dist_to_body(c, C) < S.a;
    }
    double dh = sqrt((A.c[0] - B.c[0]) * (A.c[0] - B.c[0]) + (A.c[1] - B.c[1]) * (A.c[1] - B.c[1]));
    bool zo = !(A.c[2] + A.h < B.c[2] || B.c[2] + B.h < A.c[2]);
    return zo && dh < (double)A.a + B.a;
}

// Check bodies (type, finite positive sizes, no two overlapping) and write
// their device form hb[2 n_body]; scale grows to cover them.
static int prep_bodies(const rt_body *bodies, int n_body, std::vector<float4> &hb, double &scale) {
    hb.assign(2 * (size_t)(n_body > 0 ? n_body : 1), make_float4(0.f, 0.f, 0.f, 0.f));
    for (int b = 0; b < n_body; ++b) {
        const rt_body &B = bodies[b];
        if (B.type != RT_BODY_SPHERE && B.type != RT_BODY_CYLINDER) return fail(RT_ERR_ARG, "body %d: bad type", b);
        if (!fin32(B.c[0]) || !fin32(B.c[1]) || !fin32(B.c[2]) || !fin32(B.a) || !fin32(B.h) || !(B.a > 0.f) ||
            (B.type == RT_BODY_CYLINDER && !(B.h > 0.f)))
            return fail(RT_ERR_ARG, "body %d: non-finite or non-positive size", b);
        for (int q = 0; q < b; ++q)
            if (bodies_overlap(bodies[q], B)) return fail(RT_ERR_GEOM, "bodies %d and %d overlap", q, b);
        hb[2 * b] = make_float4(B.c[0], B.c[1], B.c[2], B.a);
        hb[2 * b + 1] = make_float4(B.type == RT_BODY_CYLINDER ? B.h : 0.f, (float)B.type, 0.f, 0.f);
        for (int k = 0; k < 3; ++k) scale = fmax(scale, fabs((double)B.c[k]) + B.a + B.h);
    }
    return RT_OK;
}

// FP32 decision band: bounds the FP32 error of a margin (metres) built from
// a few dozen roundings of coordinates of magnitude <= scale: 32 ulp.
static float band_of(double scale) { return (float)(scale * 32.0 * 5.96e-8); }

// The transmitter p must lie outside every body.
static int check_tx_outside(const double p[3], const rt_body *bodies, int n_body, const char *who) {
    for (int b = 0; b < n_body; ++b)
        if (dist_to_body(p, bodies[b]) <= 0.0) return fail(RT_ERR_GEOM, "%s: transmitter inside or on body %d", who, b);
    return RT_OK;
}

// Per body, the source side of the (S, c, P) frame: the same for every
// receiver (FP64, rounded once).  txb[2 n_body].
static void prep_txb(const double p[3], const rt_body *bodies, int n_body, float4 *txb) {
    for (int b = 0; b < n_body; ++b) {
        const rt_body &B = bodies[b];
        double w[3] = {p[0] - B.c[0], p[1] - B.c[1], B.type == RT_BODY_SPHERE ? p[2] - B.c[2] : 0.0};
        double a = B.a;
        double ds = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        bool ok = ds > a;                      // cylinder: a source over the footprint has no lateral paths
        double u[3] = {0, 0, 0}, bs = 0, q = 0;
        if (ok) {
            for (int k = 0; k < 3; ++k) u[k] = w[k] / ds;
            bs = acos(a / ds);
            q = sqrt(ds * ds - a * a);
        }
        float qh = (float)q;
        txb[2 * b] = make_float4((float)u[0], (float)u[1], (float)u[2], (float)ds);
        txb[2 * b + 1] = make_float4((float)bs, qh, (float)(q - (double)qh), ok ? 1.f : 0.f);
    }
}

// Check n_f frequencies (Hz); fill the per-chunk constants fq[ceil(n_f /
// NFC)]: k, (k/2)^{1/3}, 1/lambda (double-float), FP64 k and f/c; and *hl,
// half the longest wavelength.
static int prep_freqs(const double *f_hz, int n_f, FreqC *fq, double *hl, const char *who) {
    if (n_f < 1 || n_f > RT_MAX_FREQS) return fail(RT_ERR_ARG, "%s: n_f = %d out of [1, %d]", who, n_f, RT_MAX_FREQS);
    for (int i = 0; i < n_f; ++i)
        if (!(f_hz[i] > 0.0) || !isfinite(f_hz[i])) return fail(RT_ERR_ARG, "%s: bad frequency", who);
    int nch = (n_f + NFC - 1) / NFC;
    for (int ch = 0; ch < nch; ++ch) {
        FreqC &q = fq[ch];
        memset(&q, 0, sizeof(q));
        q.nf = (n_f - ch * NFC) < NFC ? (n_f - ch * NFC) : NFC;
        for (int f = 0; f < NFC; ++f) {
            double fr = (f < q.nf) ? f_hz[ch * NFC + f] : f_hz[0];
            double k = 2.0 * M_PI * fr / 299792458.0;
            double il = fr / 299792458.0;
            q.k[f] = (float)k;
            q.kh[f] = (float)cbrt(k / 2.0);
            q.sk[f] = (float)sqrt(k / (2.0 * cbrt(k / 2.0) * cbrt(k / 2.0)));
            q.pk[f] = (float)(cbrt(k / 2.0) * sqrt(2.0 / k));
            q.il_hi[f] = (float)il;
            q.il_lo[f] = (float)(il - (double)q.il_hi[f]);
            q.kd[f] = k;
            q.fc[f] = il;
        }
    }
    *hl = 0.0;
    for (int i = 0; i < n_f; ++i) *hl = fmax(*hl, 299792458.0 / f_hz[i] / 2.0);
    return RT_OK;
}

static int noalloc_lookup(int dev);

extern "C" {

const char *rt_last_error(void) { return g_err.c_str(); }

int rt_scene_create(const float *tri_xyz, const int *tri_face, int n_tri, const rt_body *bodies, int n_body,
                    rt_scene **out) {
    if (!out) return fail(RT_ERR_ARG, "rt_scene_create: out is NULL");
    *out = nullptr;
    if (n_tri < 0 || n_body < 0) return fail(RT_ERR_ARG, "rt_scene_create: negative count");
    if ((n_tri > 0 && !tri_xyz) || (n_body > 0 && !bodies)) return fail(RT_ERR_ARG, "rt_scene_create: NULL array");
    if (n_tri > RT_MAX_TRIS) return fail(RT_ERR_OVERFLOW, "rt_scene_create: %d triangles > %d", n_tri, RT_MAX_TRIS);
    if (n_body > RT_MAX_BODIES) return fail(RT_ERR_OVERFLOW, "rt_scene_create: %d bodies > %d", n_body, RT_MAX_BODIES);
    rt_scene *s = new rt_scene();
    cudaGetDevice(&s->device);
    // the no-allocation entry point's fixed device array: its address is
    // looked up here, with the scene's device current, so that the module
    // holding it is loaded now and not by a later rt_evaluate_host_noalloc
    {
        int rcn = noalloc_lookup(s->device);
        if (rcn != RT_OK) { delete s; return rcn; }
    }
    s->n_tri = n_tri;
    s->n_body = n_body;
    s->tri.assign(tri_xyz, tri_xyz + 9 * (size_t)n_tri);
    for (size_t i = 0; i < s->tri.size(); ++i)
        if (!fin32(s->tri[i])) { delete s; return fail(RT_ERR_ARG, "rt_scene_create: non-finite vertex"); }
    s->tri_face.resize(n_tri);
    int nf = 0;
    for (int t = 0; t < n_tri; ++t) {
        int f = tri_face ? tri_face[t] : t;
        if (f < 0) { delete s; return fail(RT_ERR_ARG, "rt_scene_create: negative face id"); }
        s->tri_face[t] = f;
        if (f + 1 > nf) nf = f + 1;
    }
    if (nf > RT_MAX_FACES) { delete s; return fail(RT_ERR_OVERFLOW, "rt_scene_create: %d faces > %d", nf, RT_MAX_FACES); }
    s->n_face = nf;
    s->faces.assign(nf, FaceHost());
    std::vector<int> cnt(nf, 0);
    for (int t = 0; t < n_tri; ++t) cnt[s->tri_face[t]]++;
    int acc = 0;
    for (int f = 0; f < nf; ++f) {
        if (cnt[f] == 0) { delete s; return fail(RT_ERR_ARG, "rt_scene_create: face %d has no triangle", f); }
        s->faces[f].first = acc; s->faces[f].count = 0; acc += cnt[f];
    }
    std::vector<int> face_tris(n_tri > 0 ? n_tri : 1);
    std::vector<float4> htri(3 * (size_t)n_tri), haux(3 * (size_t)n_tri);
    for (int t = 0; t < n_tri; ++t) {
        const float *v = &s->tri[9 * (size_t)t];
        double v0[3] = {v[0], v[1], v[2]}, v1[3] = {v[3], v[4], v[5]}, v2[3] = {v[6], v[7], v[8]};
        double e1[3] = {v1[0] - v0[0], v1[1] - v0[1], v1[2] - v0[2]}, e2[3] = {v2[0] - v0[0], v2[1] - v0[1], v2[2] - v0[2]};
        double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(nn > 0.0)) { delete s; return fail(RT_ERR_ARG, "rt_scene_create: triangle %d is degenerate", t); }
        double u[3] = {n[0] / nn, n[1] / nn, n[2] / nn};
        double off = u[0] * v0[0] + u[1] * v0[1] + u[2] * v0[2];
        auto len = [](const double *a, const double *b) {
            return sqrt((a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) + (a[2] - b[2]) * (a[2] - b[2]));
        };
        double l01 = len(v0, v1), l12 = len(v1, v2), l20 = len(v2, v0);
        // altitudes: h0 of v0 over edge v1v2 = |n| / l12, etc.
        double h0 = nn / l12, h1 = nn / l20, h2 = nn / l01;
        int f = s->tri_face[t];
        FaceHost &F = s->faces[f];
        if (F.count == 0) {
            F.n[0] = u[0]; F.n[1] = u[1]; F.n[2] = u[2]; F.d = off;
        }
        face_tris[F.first + F.count++] = t;
        int fbits;
        memcpy(&fbits, &f, sizeof(int));
        float fw;
        memcpy(&fw, &fbits, sizeof(float));
        htri[3 * t] = make_float4(v[0], v[1], v[2], fw);
        htri[3 * t + 1] = make_float4(v[3], v[4], v[5], 0.f);
        htri[3 * t + 2] = make_float4(v[6], v[7], v[8], 0.f);
        haux[3 * t] = make_float4((float)u[0], (float)u[1], (float)u[2], (float)off);
        haux[3 * t + 1] = make_float4((float)h0, (float)h1, (float)h2, 0.f);
        haux[3 * t + 2] = make_float4((float)(1.0 / l01), (float)(1.0 / l12), (float)(1.0 / l20), 0.f);
    }
    // bodies
    s->bodies.assign(bodies, bodies + n_body);
    std::vector<float4> hb;
    double scale = 1.0;
    for (size_t i = 0; i < s->tri.size(); ++i) scale = fmax(scale, fabs((double)s->tri[i]));
    s->tri_scale = scale;
    if (n_tri > 0) {
        float bx0 = INFINITY, bx1 = -INFINITY, by0 = INFINITY, by1 = -INFINITY;
        for (int t = 0; t < 3 * n_tri; ++t) {
            bx0 = fminf(bx0, s->tri[3 * t]); bx1 = fmaxf(bx1, s->tri[3 * t]);
            by0 = fminf(by0, s->tri[3 * t + 1]); by1 = fmaxf(by1, s->tri[3 * t + 1]);
        }
        s->plan[0] = bx0; s->plan[1] = bx1; s->plan[2] = by0; s->plan[3] = by1;
    }
    int rcb = prep_bodies(s->bodies.data(), n_body, hb, scale);
    if (rcb != RT_OK) { delete s; return rcb; }
    s->band_len = band_of(scale);
    std::vector<float4> hf32(nf > 0 ? nf : 1);
    std::vector<dq4> hf64(nf > 0 ? nf : 1);
    std::vector<int2> hr(nf > 0 ? nf : 1);
    // per face the box of its triangles, grown by a margin that bounds the
    // FP32 face-membership decision: a point this far outside the box is
    // outside every triangle of the face by more than the decision band in
    // edge distance (the band over sin of half the smallest triangle angle),
    // plus the rounding of the culling test (1 mm)
    std::vector<float4> hbox(2 * (size_t)(nf > 0 ? nf : 1));
    {
        std::vector<double> bmin(3 * (size_t)nf, INFINITY), bmax(3 * (size_t)nf, -INFINITY), smin(nf, 1.0);
        for (int t = 0; t < n_tri; ++t) {
            const int f = s->tri_face[t];
            const float *v = &s->tri[9 * (size_t)t];
            for (int c = 0; c < 3; ++c)
                for (int k = 0; k < 3; ++k) {
                    bmin[3 * (size_t)f + k] = fmin(bmin[3 * (size_t)f + k], (double)v[3 * c + k]);
                    bmax[3 * (size_t)f + k] = fmax(bmax[3 * (size_t)f + k], (double)v[3 * c + k]);
                }
            for (int c = 0; c < 3; ++c) {        // the triangle's angle at vertex c
                const float *a = v + 3 * c, *b = v + 3 * ((c + 1) % 3), *e = v + 3 * ((c + 2) % 3);
                double u[3], w[3];
                for (int k = 0; k < 3; ++k) { u[k] = (double)b[k] - a[k]; w[k] = (double)e[k] - a[k]; }
                const double uu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                const double ww = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
                const double cs = (u[0] * w[0] + u[1] * w[1] + u[2] * w[2]) / (uu * ww);
                const double half = 0.5 * acos(fmax(-1.0, fmin(1.0, cs)));
                smin[f] = fmin(smin[f], sin(half));
            }
        }
        const double band = band_of(scale);
        for (int f = 0; f < nf; ++f) {
            const double m = 4.0 * band / fmax(smin[f], 1e-6) + 1e-3;
            hbox[2 * f] = make_float4((float)(bmin[3 * (size_t)f] - m), (float)(bmin[3 * (size_t)f + 1] - m),
                                      (float)(bmin[3 * (size_t)f + 2] - m), 0.f);
            hbox[2 * f + 1] = make_float4((float)(bmax[3 * (size_t)f] + m), (float)(bmax[3 * (size_t)f + 1] + m),
                                          (float)(bmax[3 * (size_t)f + 2] + m), 0.f);
        }
    }
    for (int f = 0; f < nf; ++f) {
        const FaceHost &F = s->faces[f];
        hf32[f] = make_float4((float)F.n[0], (float)F.n[1], (float)F.n[2], (float)F.d);
        hf64[f] = make_dq4(F.n[0], F.n[1], F.n[2], F.d);
        hr[f] = make_int2(F.first, F.count);
    }
    int rc = get_table(&s->table);
    if (rc != RT_OK) { delete s; return rc; }
#define CKS(x)                                                                  \
    do {                                                                        \
        cudaError_t e_ = (x);                                                   \
        if (e_ != cudaSuccess) {                                                \
            set_error(std::string(#x) + ": " + cudaGetErrorString(e_));         \
            free_scene(s); delete s; return RT_ERR_CUDA;                        \
        }                                                                       \
    } while (0)
    size_t ntr = n_tri > 0 ? n_tri : 1, nbd = n_body > 0 ? n_body : 1, nfc = nf > 0 ? nf : 1;
    CKS(cudaMalloc(&s->d_tri, sizeof(float4) * 3 * ntr));
    CKS(cudaMalloc(&s->d_aux, sizeof(float4) * 3 * ntr));
    CKS(cudaMalloc(&s->d_face32, sizeof(float4) * nfc));
    CKS(cudaMalloc(&s->d_face64, sizeof(dq4) * nfc));
    CKS(cudaMalloc(&s->d_face_rng, sizeof(int2) * nfc));
    CKS(cudaMalloc(&s->d_face_box, sizeof(float4) * 2 * nfc));
    CKS(cudaMalloc(&s->d_face_tris, sizeof(int) * ntr));
    CKS(cudaMalloc(&s->d_body, sizeof(float4) * 2 * nbd));
    CKS(cudaMalloc(&s->d_freq, sizeof(double) * RT_MAX_FREQS));
    CKS(cudaMalloc(&s->d_fqc, sizeof(FreqC) * ((RT_MAX_FREQS + NFC - 1) / NFC)));
    CKS(cudaMalloc(&s->d_esc, sizeof(unsigned long long) * CTR_N));
    // images of the source in every face and, for scenes the planar class
    // enumerates, in every ordered face pair
    const bool enum_faces = nf <= RT_MAX_ENUM_FACES;
    CKS(cudaMalloc(&s->d_img, sizeof(float4) * 2 * (nfc + (enum_faces ? nfc * nfc : 0))));
    CKS(cudaMalloc(&s->d_txb, sizeof(float4) * 2 * nbd));
    if (enum_faces) CKS(cudaMalloc(&s->d_txw, sizeof(float4) * 2 * nbd * nfc));
    bvh_build(s->tri.data(), n_tri, s->h_bvh, s->h_bvh_tri);
    if (n_tri > BVH_MIN_TRI) {
        CKS(cudaMalloc(&s->d_bvh, sizeof(float4) * s->h_bvh.size()));
        CKS(cudaMalloc(&s->d_bvh_tri, sizeof(int) * s->h_bvh_tri.size()));
        CKS(cudaMemcpy(s->d_bvh, s->h_bvh.data(), sizeof(float4) * s->h_bvh.size(), cudaMemcpyHostToDevice));
        CKS(cudaMemcpy(s->d_bvh_tri, s->h_bvh_tri.data(), sizeof(int) * s->h_bvh_tri.size(), cudaMemcpyHostToDevice));
    }
    if (n_tri > 0) {
        CKS(cudaMemcpy(s->d_tri, htri.data(), sizeof(float4) * 3 * n_tri, cudaMemcpyHostToDevice));
        CKS(cudaMemcpy(s->d_aux, haux.data(), sizeof(float4) * 3 * n_tri, cudaMemcpyHostToDevice));
        CKS(cudaMemcpy(s->d_face_tris, face_tris.data(), sizeof(int) * n_tri, cudaMemcpyHostToDevice));
    }
    if (nf > 0) {
        CKS(cudaMemcpy(s->d_face32, hf32.data(), sizeof(float4) * nf, cudaMemcpyHostToDevice));
        CKS(cudaMemcpy(s->d_face64, hf64.data(), sizeof(dq4) * nf, cudaMemcpyHostToDevice));
        CKS(cudaMemcpy(s->d_face_rng, hr.data(), sizeof(int2) * nf, cudaMemcpyHostToDevice));
        CKS(cudaMemcpy(s->d_face_box, hbox.data(), sizeof(float4) * 2 * nf, cudaMemcpyHostToDevice));
    }
    if (n_body > 0) CKS(cudaMemcpy(s->d_body, hb.data(), sizeof(float4) * 2 * n_body, cudaMemcpyHostToDevice));
    CKS(cudaMemset(s->d_esc, 0, sizeof(unsigned long long) * CTR_N));
    *out = s;
    return RT_OK;
}

void rt_scene_destroy(rt_scene *s) {
    if (!s) return;
    free_scene(s);
    delete s;
}

static int upload_candidates(rt_scene *s);

int rt_set_tx(rt_scene *s, const float tx[3], const float pol[3]) {
    if (!s || !tx || !pol) return fail(RT_ERR_ARG, "rt_set_tx: NULL argument");
    for (int k = 0; k < 3; ++k)
        if (!fin32(tx[k]) || !fin32(pol[k])) return fail(RT_ERR_ARG, "rt_set_tx: non-finite value");
    if (pol[0] == 0.f && pol[1] == 0.f && pol[2] == 0.f) return fail(RT_ERR_ARG, "rt_set_tx: zero polarisation");
    double p[3] = {tx[0], tx[1], tx[2]};
    int rc = check_tx_outside(p, s->bodies.data(), s->n_body, "rt_set_tx");
    if (rc != RT_OK) return rc;
    for (int f = 0; f < s->n_face; ++f) {
        const FaceHost &F = s->faces[f];
        if (F.n[0] * p[0] + F.n[1] * p[1] + F.n[2] * p[2] - F.d == 0.0)
            return fail(RT_ERR_GEOM, "rt_set_tx: transmitter on the plane of face %d", f);
    }
    memcpy(s->tx, tx, sizeof(s->tx));
    memcpy(s->pol, pol, sizeof(s->pol));
    // source images in every face and every ordered face pair (FP64), split
    // into float hi + lo: the planar path length is |P - image| (Eq. 3, image
    // method), exact to ~1e-14 for any receiver
    int nf = s->n_face;
    const bool enum_faces = nf <= RT_MAX_ENUM_FACES;
    std::vector<float4> img(2 * (size_t)(nf + (enum_faces ? nf * nf : 0)));
    auto mirror = [&](const double X[3], int f, double Y[3]) {
        const FaceHost &F = s->faces[f];
        double dist = F.n[0] * X[0] + F.n[1] * X[1] + F.n[2] * X[2] - F.d;
        for (int k = 0; k < 3; ++k) Y[k] = X[k] - F.n[k] * (2.0 * dist);
    };
    auto put = [&](size_t slot, const double Y[3]) {
        float h[3], l[3];
        for (int k = 0; k < 3; ++k) { h[k] = (float)Y[k]; l[k] = (float)(Y[k] - (double)h[k]); }
        img[2 * slot] = make_float4(h[0], h[1], h[2], 0.f);
        img[2 * slot + 1] = make_float4(l[0], l[1], l[2], 0.f);
    };
    for (int i = 0; i < nf; ++i) {
        double S1[3];
        mirror(p, i, S1);
        put(i, S1);
        for (int j = 0; j < nf && enum_faces; ++j) {
            double S2[3];
            mirror(S1, j, S2);
            put(nf + (size_t)i * nf + j, S2);
        }
    }
    if (nf > 0) CK(cudaMemcpy(s->d_img, img.data(), sizeof(float4) * img.size(), cudaMemcpyHostToDevice));
    // per body, the source side of the (S, c, P) frame: the same for every receiver
    std::vector<float4> txb(2 * (size_t)(s->n_body > 0 ? s->n_body : 1));
    prep_txb(p, s->bodies.data(), s->n_body, txb.data());
    if (s->n_body > 0) CK(cudaMemcpy(s->d_txb, txb.data(), sizeof(float4) * 2 * s->n_body, cudaMemcpyHostToDevice));
    // and per face, the same for the source's mirror image (wall -> creeping)
    if (s->n_body > 0 && nf > 0 && s->d_txw) {
        std::vector<float4> txw(2 * (size_t)s->n_body * nf);
        for (int f = 0; f < nf; ++f) {
            double S1[3];
            mirror(p, f, S1);
            prep_txb(S1, s->bodies.data(), s->n_body, txw.data() + 2 * (size_t)f * s->n_body);
        }
        CK(cudaMemcpy(s->d_txw, txw.data(), sizeof(float4) * txw.size(), cudaMemcpyHostToDevice));
    }
    s->tx_set = true;
    ++s->tx_version;
    s->cand_dev = false;                 // a device-built list belongs to the previous transmitter
    if (s->n_cand > 0) return upload_candidates(s);
    return RT_OK;
}

// The candidate list's device copy: the sequences and, per sequence, the
// source's images after each of its reflections (FP64, as hi + lo floats).
static int upload_candidates(rt_scene *s) {
    const int n = s->n_cand;
    cudaFree(s->d_cand); cudaFree(s->d_cimg);
    s->d_cand = nullptr; s->d_cimg = nullptr;
    if (n == 0) return RT_OK;
    std::vector<int4> hc(n);
    std::vector<float4> hi(6 * (size_t)n, make_float4(0.f, 0.f, 0.f, 0.f));
    const double p[3] = {s->tx[0], s->tx[1], s->tx[2]};
    for (int q = 0; q < n; ++q) {
        const int *f = &s->cand[3 * (size_t)q];
        const int k = (f[0] >= 0) + (f[1] >= 0) + (f[2] >= 0);
        hc[q] = make_int4(f[0], f[1], f[2], k);
        double X[3] = {p[0], p[1], p[2]};
        for (int m = 0; m < k; ++m) {
            const FaceHost &F = s->faces[f[m]];
            double dist = F.n[0] * X[0] + F.n[1] * X[1] + F.n[2] * X[2] - F.d;
            for (int c = 0; c < 3; ++c) X[c] = X[c] - F.n[c] * (2.0 * dist);
            float h[3], l[3];
            for (int c = 0; c < 3; ++c) { h[c] = (float)X[c]; l[c] = (float)(X[c] - (double)h[c]); }
            hi[6 * (size_t)q + 2 * m] = make_float4(h[0], h[1], h[2], 0.f);
            hi[6 * (size_t)q + 2 * m + 1] = make_float4(l[0], l[1], l[2], 0.f);
        }
    }
    CK(cudaMalloc(&s->d_cand, sizeof(int4) * n));
    CK(cudaMalloc(&s->d_cimg, sizeof(float4) * hi.size()));
    CK(cudaMemcpy(s->d_cand, hc.data(), sizeof(int4) * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(s->d_cimg, hi.data(), sizeof(float4) * hi.size(), cudaMemcpyHostToDevice));
    return RT_OK;
}

int rt_set_candidates(rt_scene *s, const int32_t *seq, int n) {
    if (!s || (n > 0 && !seq)) return fail(RT_ERR_ARG, "rt_set_candidates: NULL argument");
    if (n < 0 || n > RT_MAX_CANDIDATES) return fail(RT_ERR_ARG, "rt_set_candidates: n = %d out of range", n);
    for (int q = 0; q < n; ++q) {
        const int32_t *f = seq + 3 * (size_t)q;
        int k = 0;
        while (k < 3 && f[k] >= 0) ++k;
        if (k == 0) return fail(RT_ERR_ARG, "rt_set_candidates: sequence %d is empty", q);
        for (int m = 0; m < 3; ++m) {
            if (m < k && f[m] >= s->n_face) return fail(RT_ERR_ARG, "rt_set_candidates: bad face in sequence %d", q);
            if (m >= k && f[m] != -1) return fail(RT_ERR_ARG, "rt_set_candidates: sequence %d not -1 padded", q);
            if (m > 0 && m < k && f[m] == f[m - 1])
                return fail(RT_ERR_ARG, "rt_set_candidates: face twice in a row in sequence %d", q);
        }
    }
    s->cand.assign(seq, seq + 3 * (size_t)n);
    s->n_cand = n;
    s->cand_dev = false;
    if (!s->tx_set) return RT_OK;            // the images follow with the transmitter
    return upload_candidates(s);
}

int rt_candidates_mesh(const float *tri_xyz, const int *tri_face, int n_tri, const float tx[3], int n_rays,
                       int max_order, int32_t *seq, int cap, int *n_out) {
    if (!tri_xyz || !tx || !n_out || n_tri < 1) return fail(RT_ERR_ARG, "rt_candidates_mesh: NULL argument or no triangle");
    if (n_rays < 1 || n_rays > RT_MAX_RAYS || max_order < 1 || max_order > 3 || cap < 0 || (cap > 0 && !seq))
        return fail(RT_ERR_ARG, "rt_candidates_mesh: bad n_rays, max_order or cap");
    std::vector<int> tf(n_tri);
    int nf = 0;
    for (int t = 0; t < n_tri; ++t) {
        tf[t] = tri_face ? tri_face[t] : t;
        if (tf[t] < 0) return fail(RT_ERR_ARG, "rt_candidates_mesh: negative face id");
        if (tf[t] + 1 > nf) nf = tf[t] + 1;
    }
    std::vector<float4> nodes;
    std::vector<int> order, out;
    bvh_build(tri_xyz, n_tri, nodes, order);
    const double p[3] = {tx[0], tx[1], tx[2]};
    int n = ray_launch(tri_xyz, tf.data(), n_tri, nf, nodes, order, p, n_rays, max_order, out);
    for (int q = 0; q < n && q < cap; ++q)
        for (int m = 0; m < 3; ++m) seq[3 * (size_t)q + m] = out[3 * (size_t)q + m];
    *n_out = n;
    return RT_OK;
}

int rt_candidates(rt_scene *s, int n_rays, int max_order, int32_t *seq, int cap, int *n_out) {
    if (!s || !n_out) return fail(RT_ERR_ARG, "rt_candidates: NULL argument");
    if (n_rays < 1 || n_rays > RT_MAX_RAYS || max_order < 1 || max_order > 3 || cap < 0 || (cap > 0 && !seq))
        return fail(RT_ERR_ARG, "rt_candidates: bad n_rays, max_order or cap");
    if (!s->tx_set) return fail(RT_ERR_STATE, "rt_candidates: transmitter not set");
    const double p[3] = {s->tx[0], s->tx[1], s->tx[2]};
    std::vector<int> out;
    int n = ray_launch(s->tri.data(), s->tri_face.data(), s->n_tri, s->n_face, s->h_bvh, s->h_bvh_tri, p, n_rays,
                       max_order, out);
    for (int q = 0; q < n && q < cap; ++q)
        for (int m = 0; m < 3; ++m) seq[3 * (size_t)q + m] = out[3 * (size_t)q + m];
    *n_out = n;
    return RT_OK;
}

int rt_candidates_device(rt_scene *s, int n_rays, int max_order, void *stream) {
    if (!s) return fail(RT_ERR_ARG, "rt_candidates_device: NULL scene");
    if (n_rays < 1 || max_order < 1 || max_order > 3 || (long long)n_rays * max_order > RT_DEV_CAND_SLOTS)
        return fail(RT_ERR_ARG, "rt_candidates_device: n_rays x max_order = %lld not in [1, %d] (max_order 1-3)",
                    (long long)n_rays * max_order, RT_DEV_CAND_SLOTS);
    if (!s->tx_set) return fail(RT_ERR_STATE, "rt_candidates_device: transmitter not set");
    if (s->n_tri < 1) return fail(RT_ERR_STATE, "rt_candidates_device: no triangles");
    if (s->n_face >= (1 << 20) - 1) return fail(RT_ERR_OVERFLOW, "rt_candidates_device: %d faces", s->n_face);
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev != s->device) return fail(RT_ERR_STATE, "rt_candidates_device: the scene lives on device %d", s->device);
    cudaStream_t st = (cudaStream_t)stream;
    // set-up on first use (or for a new ray count): synchronous uploads of
    // the launch's inputs; later calls with the same ray count only queue
    // the two kernels
    if (!s->dcb.keys) {
        std::vector<double> fn;
        ray_face_normals(s->tri.data(), s->tri_face.data(), s->n_tri, s->n_face, fn);
        CK(cudaMalloc(&s->dcb.fn, sizeof(double) * fn.size()));
        CK(cudaMemcpy(s->dcb.fn, fn.data(), sizeof(double) * fn.size(), cudaMemcpyHostToDevice));
        CK(cudaMalloc(&s->dcb.keys, sizeof(unsigned long long) * RT_DEV_CAND_SLOTS));
        CK(cudaMalloc(&s->dcb.cand, sizeof(int4) * RT_DEV_CAND_SLOTS));
        CK(cudaMalloc(&s->dcb.cimg, sizeof(float4) * 6 * (size_t)RT_DEV_CAND_SLOTS));
        CK(cudaMalloc(&s->dcb.n_cand, sizeof(int) * 2));
        CK(cudaMemset(s->dcb.n_cand, 0, sizeof(int) * 2));
        if (!s->d_bvh) {
            CK(cudaMalloc(&s->d_lbvh, sizeof(float4) * s->h_bvh.size()));
            CK(cudaMalloc(&s->d_lbvh_tri, sizeof(int) * s->h_bvh_tri.size()));
            CK(cudaMemcpy(s->d_lbvh, s->h_bvh.data(), sizeof(float4) * s->h_bvh.size(), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(s->d_lbvh_tri, s->h_bvh_tri.data(), sizeof(int) * s->h_bvh_tri.size(), cudaMemcpyHostToDevice));
        }
    }
    if (s->dcb_rays != n_rays) {
        std::vector<double> dir;
        ray_directions(n_rays, dir);
        cudaFree(s->dcb.dir);
        s->dcb.dir = nullptr;
        s->dcb_rays = 0;
        CK(cudaMalloc(&s->dcb.dir, sizeof(double) * dir.size()));
        CK(cudaMemcpy(s->dcb.dir, dir.data(), sizeof(double) * dir.size(), cudaMemcpyHostToDevice));
        s->dcb_rays = n_rays;
    }
    const double p[3] = {s->tx[0], s->tx[1], s->tx[2]};
    int rc = launch_ray_candidates(s->d_tri, s->d_bvh ? s->d_bvh : s->d_lbvh, s->d_bvh ? s->d_bvh_tri : s->d_lbvh_tri,
                                   s->d_face64, p, n_rays, max_order, s->dcb, st);
    if (rc != RT_OK) return rc;
    s->cand_dev = true;
    s->cand_stream = st;
    return RT_OK;
}

int rt_get_candidates(rt_scene *s, int32_t *seq, int cap, int *n_out) {
    if (!s || !n_out || cap < 0 || (cap > 0 && !seq)) return fail(RT_ERR_ARG, "rt_get_candidates: bad argument");
    if (!s->cand_dev) {
        for (int q = 0; q < s->n_cand && q < cap; ++q)
            for (int m = 0; m < 3; ++m) seq[3 * (size_t)q + m] = s->cand[3 * (size_t)q + m];
        *n_out = s->n_cand;
        return RT_OK;
    }
    CK(cudaStreamSynchronize(s->cand_stream));
    int h[2] = {0, 0};
    CK(cudaMemcpy(h, s->dcb.n_cand, sizeof(h), cudaMemcpyDeviceToHost));
    if (h[1]) return fail(RT_ERR_OVERFLOW, "rt_get_candidates: a traversal stack of the device launch overflowed");
    std::vector<int4> c(h[0] > 0 ? h[0] : 1);
    if (h[0] > 0) CK(cudaMemcpy(c.data(), s->dcb.cand, sizeof(int4) * h[0], cudaMemcpyDeviceToHost));
    for (int q = 0; q < h[0] && q < cap; ++q) {
        seq[3 * (size_t)q] = c[q].x;
        seq[3 * (size_t)q + 1] = c[q].y;
        seq[3 * (size_t)q + 2] = c[q].z;
    }
    *n_out = h[0];
    return RT_OK;
}

// P_t + 20 log10(lambda / 4 pi) per frequency, to the device
static int upload_power(rt_scene *s) {
    if (!s->f_set) return RT_OK;
    std::vector<float> c0(s->freqs.size());
    for (size_t f = 0; f < c0.size(); ++f)
        c0[f] = (float)((double)s->power_dbm + 20.0 * log10(299792458.0 / s->freqs[f] / (4.0 * M_PI)));
    if (!s->d_pc0) CK(cudaMalloc(&s->d_pc0, sizeof(float) * RT_MAX_FREQS));
    CK(cudaMemcpy(s->d_pc0, c0.data(), sizeof(float) * c0.size(), cudaMemcpyHostToDevice));
    return RT_OK;
}

int rt_set_tx_power(rt_scene *s, float power_dbm) {
    if (!s) return fail(RT_ERR_ARG, "rt_set_tx_power: NULL scene");
    if (!fin32(power_dbm)) return fail(RT_ERR_ARG, "rt_set_tx_power: non-finite power");
    s->power_dbm = power_dbm;
    return upload_power(s);
}

int rt_power_dbm(rt_scene *s, const float *e_out, int n_rx, const float rx_pol[3], float *p_out, void *stream) {
    if (!s) return fail(RT_ERR_ARG, "rt_power_dbm: NULL scene");
    if (n_rx < 0) return fail(RT_ERR_ARG, "rt_power_dbm: n_rx < 0");
    if (!s->f_set) return fail(RT_ERR_STATE, "rt_power_dbm: frequencies not set");
    if (n_rx > 0 && (!e_out || !p_out)) return fail(RT_ERR_ARG, "rt_power_dbm: NULL buffer");
    if (rx_pol) {
        for (int k = 0; k < 3; ++k)
            if (!fin32(rx_pol[k])) return fail(RT_ERR_ARG, "rt_power_dbm: non-finite polarisation");
        if (rx_pol[0] == 0.f && rx_pol[1] == 0.f && rx_pol[2] == 0.f)
            return fail(RT_ERR_ARG, "rt_power_dbm: zero polarisation");
    }
    if (!s->d_pc0) {
        int rc = upload_power(s);
        if (rc != RT_OK) return rc;
    }
    return launch_power_dbm(e_out, (int)s->freqs.size(), n_rx, s->d_pc0, rx_pol, p_out, (cudaStream_t)stream);
}

int rt_set_face_materials(rt_scene *s, const float *mat, int n_face) {
    if (!s) return fail(RT_ERR_ARG, "rt_set_face_materials: NULL scene");
    if (!mat) {
        s->any_dielectric = false;
        return RT_OK;
    }
    if (n_face != s->n_face) return fail(RT_ERR_ARG, "rt_set_face_materials: %d faces, the scene has %d", n_face, s->n_face);
    std::vector<float4> m(n_face > 0 ? n_face : 1, make_float4(0.f, 0.f, 0.f, 0.f));
    bool any = false;
    for (int f = 0; f < n_face; ++f) {
        const float kind = mat[3 * f], er = mat[3 * f + 1], ei = mat[3 * f + 2];
        if (kind != 0.0f && kind != 1.0f) return fail(RT_ERR_ARG, "rt_set_face_materials: face %d: kind not 0 or 1", f);
        if (kind == 1.0f && (!fin32(er) || !fin32(ei) || !(er > 0.0f) || ei < 0.0f))
            return fail(RT_ERR_ARG, "rt_set_face_materials: face %d: eps' must be > 0 and eps'' >= 0", f);
        m[f] = make_float4(kind, kind == 1.0f ? er : 0.f, kind == 1.0f ? ei : 0.f, 0.f);
        any = any || kind == 1.0f;
    }
    if (!s->d_face_mat) CK(cudaMalloc(&s->d_face_mat, sizeof(float4) * (n_face > 0 ? n_face : 1)));
    if (n_face > 0) CK(cudaMemcpy(s->d_face_mat, m.data(), sizeof(float4) * n_face, cudaMemcpyHostToDevice));
    s->any_dielectric = any;
    return RT_OK;
}

int rt_set_freqs(rt_scene *s, const double *f_hz, int n_f) {
    if (!s || !f_hz) return fail(RT_ERR_ARG, "rt_set_freqs: NULL argument");
    std::vector<FreqC> fq((RT_MAX_FREQS + NFC - 1) / NFC);
    double hl;
    int rc = prep_freqs(f_hz, n_f, fq.data(), &hl, "rt_set_freqs");
    if (rc != RT_OK) return rc;
    s->freqs.assign(f_hz, f_hz + n_f);
    CK(cudaMemcpy(s->d_freq, f_hz, sizeof(double) * n_f, cudaMemcpyHostToDevice));
    int nch = (n_f + NFC - 1) / NFC;
    CK(cudaMemcpy(s->d_fqc, fq.data(), sizeof(FreqC) * nch, cudaMemcpyHostToDevice));
    s->f_set = true;
    if (s->d_pc0) return upload_power(s);
    return RT_OK;
}

static int make_dev(rt_scene *s, const rt_options *opt, DevScene &D, int *prec, bool need_freqs = true) {
    rt_options o = {2, RT_EN_ALL, RT_PREC_FP32, 0};
    if (opt) o = *opt;
    if (o.max_encirclements < 0 || o.max_encirclements > 4)
        return fail(RT_ERR_ARG, "max_encirclements %d not in [0, 4]", o.max_encirclements);
    // order 3 only through a candidate list
    const bool has_list = s->n_cand > 0 || s->cand_dev;
    const int top = has_list ? 3 : 2;
    if (o.max_order < 0 || o.max_order > top) return fail(RT_ERR_ARG, "max_order %d not in [0, %d]", o.max_order, top);
    if (o.precision != RT_PREC_FP32 && o.precision != RT_PREC_FP64) return fail(RT_ERR_ARG, "bad precision %d", o.precision);
    if (o.enable & ~(RT_EN_ALL | RT_EN_WALL_CREEP)) return fail(RT_ERR_ARG, "bad enable mask 0x%x", o.enable);
    if (s->n_face > RT_MAX_ENUM_FACES) {
        if ((o.enable & RT_EN_PLANAR) && o.max_order >= 1 && !has_list)
            return fail(RT_ERR_STATE, "%d faces: planar paths need a candidate list (rt_set_candidates)", s->n_face);
        if (o.enable & RT_EN_WALL_CREEP)
            return fail(RT_ERR_ARG, "wall -> creeping paths: at most %d faces", RT_MAX_ENUM_FACES);
    }
    if (!s->tx_set || (need_freqs && !s->f_set)) return fail(RT_ERR_STATE, "transmitter or frequencies not set");
    memset(&D, 0, sizeof(D));
    D.n_tri = s->n_tri; D.n_face = s->n_face; D.n_body = s->n_body; D.n_f = (int)s->freqs.size();
    D.tri = s->d_tri; D.tri_alt = s->d_aux; D.tri_nrm = s->d_aux;
    D.face32 = s->d_face32; D.face64 = s->d_face64; D.face_rng = s->d_face_rng; D.face_tris = s->d_face_tris;
    D.body = s->d_body;
    D.fock32 = s->table->fock32; D.fock64 = s->table->fock64;
    D.res32 = s->table->res32; D.res64 = s->table->res64;
    D.weid = s->table->weid; D.weid64 = s->table->weid64; D.weid_L = s->table->weid_L;
    D.freq = s->freqs.data();   // host pointer: read by the launcher only
    D.fqc = s->d_fqc;
    D.img = s->d_img;
    D.img_pairs = s->n_face <= RT_MAX_ENUM_FACES ? 1 : 0;
    D.txb = s->d_txb;
    D.txw = s->d_txw;
    D.bvh = s->d_bvh;
    D.bvh_tri = s->d_bvh_tri;
    D.bvh_nodes = s->d_bvh ? (int)(s->h_bvh.size() / 2) : 0;
    if (s->cand_dev) {
        D.cand = s->dcb.cand;
        D.cimg = s->dcb.cimg;
        D.n_cand = RT_DEV_CAND_SLOTS;           // an upper bound; the kernels read the length
        D.n_cand_dev = s->dcb.n_cand;
    } else {
        D.cand = s->n_cand > 0 ? s->d_cand : nullptr;
        D.cimg = s->d_cimg;
        D.n_cand = s->n_cand;
        D.n_cand_dev = nullptr;
    }
    D.face_mat = s->any_dielectric ? s->d_face_mat : nullptr;
    D.face_box = s->d_face_box;
    memcpy(D.tx, s->tx, sizeof(D.tx));
    memcpy(D.pol, s->pol, sizeof(D.pol));
    D.band_len = s->band_len;
    D.max_order = o.max_order;
    D.max_enc = o.max_encirclements;
    D.enable = o.enable;
    *prec = o.precision;
    return RT_OK;
}

int rt_evaluate(rt_scene *s, const float *rx_soa, int n_rx, float *e_out, uint32_t *flags, const rt_options *opt,
                void *stream) {
    if (!s) return fail(RT_ERR_ARG, "rt_evaluate: NULL scene");
    if (n_rx < 0) return fail(RT_ERR_ARG, "rt_evaluate: n_rx < 0");
    DevScene D;
    int prec;
    int rc = make_dev(s, opt, D, &prec);
    if (rc != RT_OK) return rc;
    if (n_rx > 0 && (!rx_soa || !e_out)) return fail(RT_ERR_ARG, "rt_evaluate: NULL buffer");
    if (n_rx == 0) return RT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemsetAsync(s->d_esc, 0, sizeof(unsigned long long) * CTR_N, st));
    s->last_stream = st;
    return launch_eval(D, rx_soa, n_rx, e_out, flags, nullptr, nullptr, 0, prec, s->shape, s->d_esc, st,
                       &s->last_launches);
}

int rt_paths(rt_scene *s, const float *rx_soa, int n_rx, uint64_t *codes, int32_t *counts, int cap, uint32_t *flags,
             const rt_options *opt, void *stream) {
    if (!s) return fail(RT_ERR_ARG, "rt_paths: NULL scene");
    if (n_rx < 0 || cap < 1) return fail(RT_ERR_ARG, "rt_paths: n_rx < 0 or cap < 1");
    DevScene D;
    int prec;
    int rc = make_dev(s, opt, D, &prec);
    if (rc != RT_OK) return rc;
    if (n_rx > 0 && (!rx_soa || !codes || !counts)) return fail(RT_ERR_ARG, "rt_paths: NULL buffer");
    if (n_rx == 0) return RT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemsetAsync(s->d_esc, 0, sizeof(unsigned long long) * CTR_N, st));
    s->last_stream = st;
    return launch_eval(D, rx_soa, n_rx, nullptr, flags, codes, counts, cap, prec, nullptr, s->d_esc, st,
                       &s->last_launches);
}

int rt_evaluate_with_paths(rt_scene *s, const float *rx_soa, int n_rx, float *e_out, uint64_t *codes, int32_t *counts,
                           int cap, uint32_t *flags, const rt_options *opt, void *stream) {
    if (!s) return fail(RT_ERR_ARG, "rt_evaluate_with_paths: NULL scene");
    if (n_rx < 0 || cap < 1) return fail(RT_ERR_ARG, "rt_evaluate_with_paths: n_rx < 0 or cap < 1");
    DevScene D;
    int prec;
    int rc = make_dev(s, opt, D, &prec);
    if (rc != RT_OK) return rc;
    if (n_rx > 0 && (!rx_soa || !e_out || !codes || !counts))
        return fail(RT_ERR_ARG, "rt_evaluate_with_paths: NULL buffer");
    if (n_rx == 0) return RT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemsetAsync(s->d_esc, 0, sizeof(unsigned long long) * CTR_N, st));
    s->last_stream = st;
    return launch_eval(D, rx_soa, n_rx, e_out, flags, codes, counts, cap, prec, s->shape, s->d_esc, st,
                       &s->last_launches);
}

int rt_backward(rt_scene *s, const float *rx_soa, int n_rx, const uint64_t *codes, const int32_t *counts, int cap,
                const float *grad_e, double *grad_bodies, double *grad_tx, double *grad_freqs, const rt_options *opt,
                void *stream) {
    if (!s) return fail(RT_ERR_ARG, "rt_backward: NULL scene");
    if (n_rx < 0 || cap < 1) return fail(RT_ERR_ARG, "rt_backward: n_rx < 0 or cap < 1");
    if (!grad_tx || !grad_freqs || (s->n_body > 0 && !grad_bodies))
        return fail(RT_ERR_ARG, "rt_backward: NULL gradient buffer");
    if (n_rx > 0 && (!rx_soa || !codes || !counts || !grad_e)) return fail(RT_ERR_ARG, "rt_backward: NULL buffer");
    DevScene D;
    int prec;
    int rc = make_dev(s, opt, D, &prec);
    if (rc != RT_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    s->last_stream = st;
    s->last_launches = n_rx > 0 ? 1 : 0;
    return launch_adjoint(D, rx_soa, n_rx, codes, counts, cap, grad_e, grad_bodies, grad_tx, grad_freqs, s->d_esc + 1,
                          prec, st);
}

int rt_evaluate_host(rt_scene *s, const float *rx_soa, int n_rx, float *e_out, uint32_t *flags, const rt_options *opt,
                     void *stream) {
    if (!s) return fail(RT_ERR_ARG, "rt_evaluate_host: NULL scene");
    if (n_rx < 0) return fail(RT_ERR_ARG, "rt_evaluate_host: n_rx < 0");
    if (n_rx == 0) return RT_OK;
    if (!rx_soa || !e_out) return fail(RT_ERR_ARG, "rt_evaluate_host: NULL buffer");
    if (!s->f_set) return fail(RT_ERR_STATE, "frequencies not set");
    cudaStream_t st = (cudaStream_t)stream;
    size_t nf = s->freqs.size();
    if ((size_t)n_rx > s->io_cap) {
        cudaFree(s->io_rx); cudaFree(s->io_e); cudaFree(s->io_fl);
        s->io_rx = nullptr; s->io_e = nullptr; s->io_fl = nullptr; s->io_cap = 0;
        CK(cudaMalloc(&s->io_rx, sizeof(float) * 3 * (size_t)n_rx));
        CK(cudaMalloc(&s->io_e, sizeof(float) * 2 * 3 * RT_MAX_FREQS * (size_t)n_rx));
        CK(cudaMalloc(&s->io_fl, sizeof(uint32_t) * (size_t)n_rx));
        s->io_cap = n_rx;
    }
    CK(cudaMemcpyAsync(s->io_rx, rx_soa, sizeof(float) * 3 * (size_t)n_rx, cudaMemcpyHostToDevice, st));
    int rc = rt_evaluate(s, s->io_rx, n_rx, s->io_e, flags ? s->io_fl : nullptr, opt, stream);
    if (rc != RT_OK) return rc;
    CK(cudaMemcpyAsync(e_out, s->io_e, sizeof(float) * 2 * 3 * nf * (size_t)n_rx, cudaMemcpyDeviceToHost, st));
    if (flags) CK(cudaMemcpyAsync(flags, s->io_fl, sizeof(uint32_t) * (size_t)n_rx, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return RT_OK;
}

int rt_get_stats(rt_scene *s, rt_stats *out) {
    if (!s || !out) return fail(RT_ERR_ARG, "rt_get_stats: NULL argument");
    CK(cudaStreamSynchronize(s->last_stream));
    unsigned long long v = 0;
    CK(cudaMemcpy(&v, s->d_esc, sizeof(v), cudaMemcpyDeviceToHost));
    out->escalated_candidates = v;
    out->kernel_launches = (unsigned long long)s->last_launches;
    return RT_OK;
}

int rt_fock_table(double *xi_lo, double *step, int *n, double *g, double *dg, double *res) {
    DevTable *T = nullptr;
    int rc = get_table(&T);
    if (rc != RT_OK) return rc;
    if (xi_lo) *xi_lo = XI_LO;
    if (step) *step = XI_STEP;
    if (n) *n = FOCK_N;
    for (int j = 0; j < FOCK_N; ++j)
        for (int k = 0; k < 2; ++k) {
            const double *q = &T->host.tab[(j * 2 + k) * 4];
            if (g) { g[(k * FOCK_N + j) * 2] = q[0]; g[(k * FOCK_N + j) * 2 + 1] = q[1]; }
            if (dg) { dg[(k * FOCK_N + j) * 2] = q[2]; dg[(k * FOCK_N + j) * 2 + 1] = q[3]; }
        }
    if (res) memcpy(res, T->host.res.data(), sizeof(double) * 4 * FOCK_NRES);
    return RT_OK;
}

int rt_fock_table_p(double *xi0, int *n, double *p, double *dp) {
    DevTable *T = nullptr;
    int rc = get_table(&T);
    if (rc != RT_OK) return rc;
    if (xi0) *xi0 = XI_HI;
    if (n) *n = FOCK_NP;
    for (int j = 0; j < FOCK_NP; ++j)
        for (int k = 0; k < 2; ++k) {
            const double *q = &T->host.tabp[(j * 2 + k) * 4];
            if (p) { p[(k * FOCK_NP + j) * 2] = q[0]; p[(k * FOCK_NP + j) * 2 + 1] = q[1]; }
            if (dp) { dp[(k * FOCK_NP + j) * 2] = q[2]; dp[(k * FOCK_NP + j) * 2 + 1] = q[3]; }
        }
    return RT_OK;
}

// ---- batched frames

}  // extern "C"

struct rt_batch {
    rt_scene *s = nullptr;
    int n_frames = 0, n_f = 0, max_body = 0, nch = 0;
    std::vector<FrameDev> fr;           // host copy of the device frame table
    std::vector<unsigned> fr_tx;        // scene transmitter version each frame was set with (0: never set)
    unsigned long long n_tiles = 0;
    float4 *d_body = nullptr, *d_txb = nullptr;   // [n_frames][max_body][2]
    FreqC *d_fqc = nullptr;                       // [n_frames][nch]
    FrameDev *d_frames = nullptr;                 // [n_frames]
    unsigned long long *d_ctr = nullptr;          // [CTR_N]
    // spatial ordering of the receivers: cell counts [n_frames][RX_CELLS],
    // ranks, the sorted receivers and the permutation [total receivers]
    uint32_t *d_cnt = nullptr, *d_rank = nullptr;
    float *d_rxs = nullptr;
    int32_t *d_perm = nullptr;
    long long total_rx = 0;
    int max_rx = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t last_stream = nullptr;
    int last_launches = 0;
    // tile shape: warps per tile of the planar and of the body kernels,
    // planar frequency chunks per launch (rt_batch_set_shape / rt_batch_tune)
    int shape[3] = {4, 4, 4};
};

static void free_batch(rt_batch *b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->d_body); cudaFree(b->d_txb); cudaFree(b->d_fqc); cudaFree(b->d_frames); cudaFree(b->d_ctr);
    cudaFree(b->d_cnt); cudaFree(b->d_rank); cudaFree(b->d_rxs); cudaFree(b->d_perm);
}

// queue one evaluation of the batch on st (no synchronisation)
static int batch_queue(rt_batch *b, const float *rx_soa, float *e_out, uint32_t *flags, const rt_options *opt,
                       cudaStream_t st) {
    rt_scene *s = b->s;
    for (int f = 0; f < b->n_frames; ++f)
        if (b->fr_tx[f] != s->tx_version)
            return fail(RT_ERR_STATE, "rt_batch: frame %d not set since the transmitter was last set", f);
    DevScene D;
    int prec;
    int rc = make_dev(s, opt, D, &prec, false);
    if (rc != RT_OK) return rc;
    if (b->n_tiles > 0 && (!rx_soa || !e_out)) return fail(RT_ERR_ARG, "rt_batch: NULL buffer");
    if (D.enable & RT_EN_WALL_CREEP) return fail(RT_ERR_ARG, "rt_batch: wall -> creeping paths are for single scenes");
    D.n_body = b->max_body;
    D.txw = nullptr;
    D.n_f = b->n_f;
    D.body = b->d_body; D.txb = b->d_txb; D.fqc = b->d_fqc;
    D.freq = nullptr;
    b->last_stream = st;
    b->last_launches = 0;
    if (b->n_tiles == 0) return RT_OK;
    CK(cudaMemsetAsync(b->d_ctr, 0, sizeof(unsigned long long) * CTR_N, st));
    // receivers in a spatial order (grid over the floor plan of the scene's
    // triangles, else a 100 m square round the origin), results in theirs
    float x0 = s->plan[0], x1 = s->plan[1], y0 = s->plan[2], y1 = s->plan[3];
    if (!(x1 > x0) || !(y1 > y0)) { x0 = -50.f; x1 = 50.f; y0 = -50.f; y1 = 50.f; }
    float4 grid = make_float4(x0, y0, (float)RX_GRID / (x1 - x0), (float)RX_GRID / (y1 - y0));
    rc = launch_rx_order(b->d_frames, b->n_frames, b->max_rx, rx_soa, grid, b->d_cnt, b->d_rank, b->d_rxs,
                         b->d_perm, st);
    if (rc != RT_OK) return rc;
    rc = launch_eval_batch(D, b->d_frames, b->fr.data(), b->n_frames, b->n_tiles, b->d_rxs, b->d_perm, e_out, flags,
                           prec, b->shape, b->d_ctr, st, &b->last_launches);
    if (rc == RT_OK) b->last_launches += 3;          // the ordering kernels
    return rc;
}

extern "C" {

int rt_batch_create(rt_scene *s, int n_frames, const int32_t *n_rx, int n_f, int max_body, rt_batch **out) {
    if (!out) return fail(RT_ERR_ARG, "rt_batch_create: out is NULL");
    *out = nullptr;
    if (!s || !n_rx) return fail(RT_ERR_ARG, "rt_batch_create: NULL argument");
    if (n_frames < 1) return fail(RT_ERR_ARG, "rt_batch_create: n_frames = %d < 1", n_frames);
    if (n_f < 1 || n_f > RT_MAX_FREQS) return fail(RT_ERR_ARG, "rt_batch_create: n_f = %d out of [1, %d]", n_f, RT_MAX_FREQS);
    if (max_body < 0) return fail(RT_ERR_ARG, "rt_batch_create: max_body < 0");
    if (max_body > RT_MAX_BODIES) return fail(RT_ERR_OVERFLOW, "rt_batch_create: max_body %d > %d", max_body, RT_MAX_BODIES);
    rt_batch *b = new rt_batch();
    b->s = s;
    b->n_frames = n_frames;
    b->n_f = n_f;
    b->max_body = max_body;
    b->nch = (n_f + NFC - 1) / NFC;
    b->fr.assign(n_frames, FrameDev());
    b->fr_tx.assign(n_frames, 0u);
    long long rx_off = 0;
    unsigned long long tile = 0;
    for (int f = 0; f < n_frames; ++f) {
        if (n_rx[f] < 0) { delete b; return fail(RT_ERR_ARG, "rt_batch_create: n_rx[%d] < 0", f); }
        FrameDev &F = b->fr[f];
        F.rx_off = rx_off;
        F.e_off = 6 * (long long)n_f * rx_off;
        F.tile0 = tile;
        F.n_rx = n_rx[f];
        F.n_body = 0;
        F.band = band_of(s->tri_scale);
        unsigned long long nt = ((unsigned long long)n_rx[f] + 31ull) >> 5;
        tile += (nt + TILE_ALIGN - 1) / TILE_ALIGN * TILE_ALIGN;
        rx_off += n_rx[f];
        if (n_rx[f] > b->max_rx) b->max_rx = n_rx[f];
    }
    b->n_tiles = tile;
    b->total_rx = rx_off;
    size_t nb = (size_t)n_frames * 2 * (max_body > 0 ? max_body : 1);
#define CKB(x)                                                                  \
    do {                                                                        \
        cudaError_t e_ = (x);                                                   \
        if (e_ != cudaSuccess) {                                                \
            set_error(std::string(#x) + ": " + cudaGetErrorString(e_));         \
            free_batch(b); delete b; return RT_ERR_CUDA;                        \
        }                                                                       \
    } while (0)
    CKB(cudaMalloc(&b->d_body, sizeof(float4) * nb));
    CKB(cudaMalloc(&b->d_txb, sizeof(float4) * nb));
    CKB(cudaMalloc(&b->d_fqc, sizeof(FreqC) * (size_t)n_frames * b->nch));
    CKB(cudaMalloc(&b->d_frames, sizeof(FrameDev) * (size_t)n_frames));
    CKB(cudaMalloc(&b->d_ctr, sizeof(unsigned long long) * CTR_N));
    {
        const size_t nr = (size_t)(rx_off > 0 ? rx_off : 1);
        CKB(cudaMalloc(&b->d_cnt, sizeof(uint32_t) * (size_t)n_frames * RX_CELLS));
        CKB(cudaMalloc(&b->d_rank, sizeof(uint32_t) * nr));
        CKB(cudaMalloc(&b->d_rxs, sizeof(float) * 3 * nr));
        CKB(cudaMalloc(&b->d_perm, sizeof(int32_t) * nr));
    }
    for (int f = 0; f < n_frames; ++f) {
        FrameDev &F = b->fr[f];
        F.body = b->d_body + (size_t)f * 2 * (max_body > 0 ? max_body : 1);
        F.txb = b->d_txb + (size_t)f * 2 * (max_body > 0 ? max_body : 1);
        F.fqc = b->d_fqc + (size_t)f * b->nch;
    }
    CKB(cudaMemcpy(b->d_frames, b->fr.data(), sizeof(FrameDev) * (size_t)n_frames, cudaMemcpyHostToDevice));
    CKB(cudaMemset(b->d_ctr, 0, sizeof(unsigned long long) * CTR_N));
#undef CKB
    *out = b;
    return RT_OK;
}

void rt_batch_destroy(rt_batch *b) {
    if (!b) return;
    free_batch(b);
    delete b;
}

int rt_batch_set_frame(rt_batch *b, int frame, const rt_body *bodies, int n_body, const double *f_hz) {
    if (!b || !f_hz || (n_body > 0 && !bodies)) return fail(RT_ERR_ARG, "rt_batch_set_frame: NULL argument");
    if (frame < 0 || frame >= b->n_frames) return fail(RT_ERR_ARG, "rt_batch_set_frame: frame %d out of range", frame);
    if (n_body < 0) return fail(RT_ERR_ARG, "rt_batch_set_frame: n_body < 0");
    if (n_body > b->max_body)
        return fail(RT_ERR_OVERFLOW, "rt_batch_set_frame: %d bodies > max_body %d", n_body, b->max_body);
    rt_scene *s = b->s;
    if (!s->tx_set) return fail(RT_ERR_STATE, "rt_batch_set_frame: transmitter not set");
    std::vector<float4> hb;
    double scale = s->tri_scale;
    int rc = prep_bodies(bodies, n_body, hb, scale);
    if (rc != RT_OK) return rc;
    double p[3] = {s->tx[0], s->tx[1], s->tx[2]};
    rc = check_tx_outside(p, bodies, n_body, "rt_batch_set_frame");
    if (rc != RT_OK) return rc;
    std::vector<float4> txb(hb.size());
    prep_txb(p, bodies, n_body, txb.data());
    std::vector<FreqC> fq(b->nch);
    double hl;
    rc = prep_freqs(f_hz, b->n_f, fq.data(), &hl, "rt_batch_set_frame");
    if (rc != RT_OK) return rc;
    FrameDev &F = b->fr[frame];
    F.n_body = n_body;
    F.hl = hl;
    F.band = band_of(scale);
    if (n_body > 0) {
        CK(cudaMemcpy((void *)F.body, hb.data(), sizeof(float4) * 2 * n_body, cudaMemcpyHostToDevice));
        CK(cudaMemcpy((void *)F.txb, txb.data(), sizeof(float4) * 2 * n_body, cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpy((void *)F.fqc, fq.data(), sizeof(FreqC) * b->nch, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b->d_frames + frame, &F, sizeof(FrameDev), cudaMemcpyHostToDevice));
    b->fr_tx[frame] = s->tx_version;
    return RT_OK;
}

int rt_batch_evaluate(rt_batch *b, const float *rx_soa, float *e_out, uint32_t *flags, const rt_options *opt,
                      void *stream) {
    if (!b) return fail(RT_ERR_ARG, "rt_batch_evaluate: NULL batch");
    return batch_queue(b, rx_soa, e_out, flags, opt, (cudaStream_t)stream);
}

int rt_batch_capture(rt_batch *b, const float *rx_soa, float *e_out, uint32_t *flags, const rt_options *opt,
                     void *stream) {
    if (!b) return fail(RT_ERR_ARG, "rt_batch_capture: NULL batch");
    if (!stream) return fail(RT_ERR_ARG, "rt_batch_capture: capture needs a stream other than the legacy default stream");
    cudaStream_t st = (cudaStream_t)stream;
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int rc = batch_queue(b, rx_soa, e_out, flags, opt, st);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (rc != RT_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(RT_ERR_CUDA, "rt_batch_capture: cudaStreamEndCapture: %s", cudaGetErrorString(e));
    b->graph = g;
    CK(cudaGraphInstantiate(&b->gexec, b->graph, 0));
    return RT_OK;
}

int rt_batch_replay(rt_batch *b, void *stream) {
    if (!b) return fail(RT_ERR_ARG, "rt_batch_replay: NULL batch");
    if (!b->gexec) return fail(RT_ERR_STATE, "rt_batch_replay: nothing captured");
    for (int f = 0; f < b->n_frames; ++f)
        if (b->fr_tx[f] != b->s->tx_version)
            return fail(RT_ERR_STATE, "rt_batch_replay: frame %d not set since the transmitter was last set", f);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaGraphLaunch(b->gexec, st));
    b->last_stream = st;
    return RT_OK;
}

static bool shape_ok(const int sh[3]) {
    const bool p = sh[0] == 1 || sh[0] == 2 || sh[0] == 4;
    const bool q = sh[1] >= 1 && sh[1] <= 12 && 12 % sh[1] == 0;
    return p && q && sh[2] >= 1 && sh[2] <= 4;
}

int rt_batch_set_shape(rt_batch *b, const int shape[3]) {
    if (!b || !shape) return fail(RT_ERR_ARG, "rt_batch_set_shape: NULL argument");
    if (!shape_ok(shape))
        return fail(RT_ERR_ARG, "rt_batch_set_shape: shape (%d, %d, %d) not in {1,2,4} x {1,2,3,4,6,12} x [1,4]",
                    shape[0], shape[1], shape[2]);
    memcpy(b->shape, shape, sizeof(b->shape));
    return RT_OK;
}

int rt_batch_get_shape(rt_batch *b, int shape[3]) {
    if (!b || !shape) return fail(RT_ERR_ARG, "rt_batch_get_shape: NULL argument");
    memcpy(shape, b->shape, sizeof(b->shape));
    return RT_OK;
}

}  // extern "C"

// Tile shapes chosen by the autotuner, per device, workload size and
// options: a later workload of the same size takes them without timing.
static std::mutex g_tune_mu;
static std::map<std::vector<long long>, std::vector<int>> g_tuned;

// Coordinate search over tile shapes from the default {4, 4, min(4, nch)}: body warps
// per tile, then planar warps per tile, then planar chunks per launch (up to
// nch), each timed as the faster of two evaluations after a warm-up.
// run(shape) queues one evaluation on st.  A shape that cannot launch is
// skipped; the default must run.
template <typename RUN>
static int tune_shape(RUN run, cudaStream_t st, int nch, const std::vector<long long> &key, int best[3]) {
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            for (int k = 0; k < 3; ++k) best[k] = it->second[k];
            return RT_OK;
        }
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    auto time_shape = [&](const int sh[3], float *ms) -> int {
        int rc = run(sh);
        float tb = 1e30f;
        for (int rep = 0; rep < 2 && rc == RT_OK; ++rep) {
            cudaEventRecord(e0, st);
            rc = run(sh);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) return fail(RT_ERR_CUDA, "autotuner: evaluation failed");
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (t < tb) tb = t;
        }
        *ms = tb;
        return rc;
    };
    best[0] = 4; best[1] = 4; best[2] = nch < 4 ? (nch > 0 ? nch : 1) : 4;
    float t_best = 0.f;
    int rc = time_shape(best, &t_best);
    const int cand_body[] = {2, 3, 4, 6, 12}, cand_planar[] = {1, 2, 4}, cand_chunks[] = {1, 2, 3, 4};
    auto trial = [&](int p, int q, int r) {
        const int sh[3] = {p, q, r};
        if (rc != RT_OK || !shape_ok(sh) || (sh[0] == best[0] && sh[1] == best[1] && sh[2] == best[2])) return;
        float t;
        if (time_shape(sh, &t) == RT_OK && t < t_best) { t_best = t; memcpy(best, sh, 3 * sizeof(int)); }
        cudaGetLastError();                  // a shape the device cannot launch is skipped
    };
    for (int q : cand_body) trial(best[0], q, best[2]);
    for (int p : cand_planar) trial(p, best[1], best[2]);
    for (int r : cand_chunks)
        if (r <= nch) trial(best[0], best[1], r);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != RT_OK) return rc;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = std::vector<int>(best, best + 3);
    return RT_OK;
}

extern "C" int rt_batch_tune(rt_batch *b, const float *rx_soa, float *e_out, uint32_t *flags, const rt_options *opt,
                             void *stream, int shape_out[3]) {
    if (!b) return fail(RT_ERR_ARG, "rt_batch_tune: NULL batch");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::vector<long long> key = {0, dev, b->n_frames, b->n_f, b->max_body, b->total_rx, b->max_rx,
                                  opt ? opt->max_order : 2, opt ? (long long)opt->enable : RT_EN_ALL,
                                  opt ? opt->precision : RT_PREC_FP32};
    int best[3];
    int rc = tune_shape([&](const int *sh) {
        memcpy(b->shape, sh, sizeof(b->shape));
        return batch_queue(b, rx_soa, e_out, flags, opt, st);
    }, st, (b->n_f + NFC - 1) / NFC, key, best);
    static const int kDefault[3] = {4, 4, 4};
    memcpy(b->shape, rc == RT_OK ? best : kDefault, sizeof(b->shape));
    if (rc == RT_OK && shape_out) memcpy(shape_out, best, sizeof(best));
    return rc;
}

extern "C" int rt_tune(rt_scene *s, const float *rx_soa, int n_rx, float *e_out, uint32_t *flags,
                       const rt_options *opt, void *stream, int shape_out[3]) {
    if (!s) return fail(RT_ERR_ARG, "rt_tune: NULL scene");
    if (n_rx <= 0) {
        if (shape_out) memcpy(shape_out, s->shape, sizeof(s->shape));
        return RT_OK;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::vector<long long> key = {1, dev, n_rx, (long long)s->freqs.size(), s->n_body, s->n_tri,
                                  opt ? opt->max_order : 2, opt ? (long long)opt->enable : RT_EN_ALL,
                                  opt ? opt->precision : RT_PREC_FP32};
    int best[3];
    int rc = tune_shape([&](const int *sh) {
        memcpy(s->shape, sh, sizeof(s->shape));
        return rt_evaluate(s, rx_soa, n_rx, e_out, flags, opt, stream);
    }, st, ((int)s->freqs.size() + NFC - 1) / NFC, key, best);
    static const int kDefault[3] = {4, 4, 4};
    memcpy(s->shape, rc == RT_OK ? best : kDefault, sizeof(s->shape));
    if (rc == RT_OK && shape_out) memcpy(shape_out, best, sizeof(best));
    return rc;
}

extern "C" int rt_set_shape(rt_scene *s, const int shape[3]) {
    if (!s || !shape) return fail(RT_ERR_ARG, "rt_set_shape: NULL argument");
    if (!shape_ok(shape))
        return fail(RT_ERR_ARG, "rt_set_shape: shape (%d, %d, %d) not in {1,2,4} x {1,2,3,4,6,12} x [1,4]",
                    shape[0], shape[1], shape[2]);
    memcpy(s->shape, shape, sizeof(s->shape));
    return RT_OK;
}

extern "C" int rt_get_shape(rt_scene *s, int shape[3]) {
    if (!s || !shape) return fail(RT_ERR_ARG, "rt_get_shape: NULL argument");
    memcpy(shape, s->shape, sizeof(s->shape));
    return RT_OK;
}

extern "C" {

int rt_batch_get_stats(rt_batch *b, rt_stats *out) {
    if (!b || !out) return fail(RT_ERR_ARG, "rt_batch_get_stats: NULL argument");
    CK(cudaStreamSynchronize(b->last_stream));
    unsigned long long v = 0;
    CK(cudaMemcpy(&v, b->d_ctr, sizeof(v), cudaMemcpyDeviceToHost));
    out->escalated_candidates = v;
    out->kernel_launches = (unsigned long long)b->last_launches;
    return RT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Evaluation from host buffers without device allocation (see creep.h).
// The staging buffers live in one file-scope device array; its device
// address is looked up once per device and then reused.
static __device__ __align__(256) unsigned char g_noalloc_scratch[RT_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[NOALLOC_MAX_DEVICES];   // device address per device (nullptr: not looked up yet)

size_t round256(size_t n) { return (n + 255) & ~(size_t)255; }
}  // namespace

// The array's device address on device dev (current), looked up once.  Called
// by rt_scene_create, so the lookup (and the lazy load of this file's module,
// which holds the array) happens when a scene is made, not inside an
// evaluation.
static int noalloc_lookup(int dev) {
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(RT_ERR_ARG, "device %d beyond the library's limit", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(RT_ERR_CUDA, "cudaGetSymbolAddress of the no-allocation array: %s", cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    return RT_OK;
}

extern "C" int rt_evaluate_host_noalloc(rt_scene *s, const float *rx_soa, int n_rx, float *e_out, uint32_t *flags,
                                        const rt_options *opt, void *stream) {
    if (!s) return fail(RT_ERR_ARG, "rt_evaluate_host_noalloc: NULL scene");
    if (n_rx < 0) return fail(RT_ERR_ARG, "rt_evaluate_host_noalloc: n_rx < 0");
    if (!s->f_set) return fail(RT_ERR_STATE, "frequencies not set");
    if (n_rx == 0) return RT_OK;
    if (!rx_soa || !e_out) return fail(RT_ERR_ARG, "rt_evaluate_host_noalloc: NULL buffer");
    size_t nf = s->freqs.size();
    size_t rx_bytes = round256(sizeof(float) * 3 * (size_t)n_rx);
    size_t e_bytes = round256(sizeof(float) * 2 * 3 * nf * (size_t)n_rx);
    size_t fl_bytes = round256(sizeof(uint32_t) * (size_t)n_rx);
    size_t need = rx_bytes + e_bytes + fl_bytes;
    if (need > (size_t)RT_NOALLOC_SCRATCH_BYTES)
        return fail(RT_ERR_OVERFLOW,
                    "rt_evaluate_host_noalloc: %d receivers x %d frequencies need %zu bytes of device scratch, "
                    "the fixed array holds %u; split the receivers into smaller calls",
                    n_rx, (int)nf, need, RT_NOALLOC_SCRATCH_BYTES);
    int dev = 0;
    CK(cudaGetDevice(&dev));
    // the scene's buffers live on s->device: pairing them with another
    // device's array would be a cross-device access
    if (dev != s->device)
        return fail(RT_ERR_STATE, "rt_evaluate_host_noalloc: device %d is current, the scene lives on device %d", dev,
                    s->device);
    void *base = nullptr;
    {
        int rcn = noalloc_lookup(dev);      // done by rt_scene_create; a no-op here
        if (rcn != RT_OK) return rcn;
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        base = g_noalloc_ptr[dev];
    }
    float *d_rx = (float *)base;
    float *d_e = (float *)((unsigned char *)base + rx_bytes);
    uint32_t *d_fl = (uint32_t *)((unsigned char *)base + rx_bytes + e_bytes);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(d_rx, rx_soa, sizeof(float) * 3 * (size_t)n_rx, cudaMemcpyHostToDevice, st));
    int rc = rt_evaluate(s, d_rx, n_rx, d_e, flags ? d_fl : nullptr, opt, stream);
    if (rc != RT_OK) return rc;
    CK(cudaMemcpyAsync(e_out, d_e, sizeof(float) * 2 * 3 * nf * (size_t)n_rx, cudaMemcpyDeviceToHost, st));
    if (flags) CK(cudaMemcpyAsync(flags, d_fl, sizeof(uint32_t) * (size_t)n_rx, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return RT_OK;
}
