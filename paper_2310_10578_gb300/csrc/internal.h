// internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/creep.h"

namespace creep {

// 4 doubles (the CUDA vector type of that shape is deprecated in CUDA 13)
struct __align__(16) dq4 {
    double x, y, z, w;
};
inline dq4 make_dq4(double x, double y, double z, double w) { dq4 r; r.x = x; r.y = y; r.z = z; r.w = w; return r; }

// Fock--Pekeris table domain (smooth-surface UTD coefficients).  Below XI_LO
// the reflection coefficients take their GO values -1 / +1; above XI_HI the
// residue (creeping-mode) series is summed instead of the table.
constexpr double XI_LO = -10.0;
constexpr double XI_HI = 1.5;
constexpr double XI_STEP = 1.0 / 64.0;
constexpr int FOCK_N = 737;            // (XI_HI - XI_LO) / XI_STEP + 1
// FP32 fields: a second segment of the table on [XI_HI, XI_P] holds P itself
// (not phat, and without the e^{-j xi^3/12} factor), where the residue series
// needs 4 to 16 terms (soft and hard) and phat = P + c/xi is mostly c/xi (so
// that P = phat - c/xi would lose FP32 digits); the series runs above XI_P.
// Its nodes come from the quadrature below XI_PRES and from the 8-term
// residue series (converged there to ~1e-11) from XI_PRES on.
constexpr double XI_P = 12.0;
constexpr double XI_PRES = 3.0;
constexpr int FOCK_NP = 673;           // (XI_P - XI_HI) / XI_STEP + 1
constexpr int FOCK_NBUCKET = 11;       // quadrature buckets: [0, XI_HI], [-1, 0), ..., [-10, -9)
constexpr int FOCK_NRES = 8;           // residue-series terms
constexpr int WEIDEMAN_N = 16;         // terms of the rational approximation of w(z)

struct FockHost {
    std::vector<double> tab;   // [FOCK_N][2][4]: G.re, G.im, G'.re, G'.im (soft, hard)
    std::vector<double> tabp;  // [FOCK_NP][2][4]: P.re, P.im, P'.re, P'.im (soft, hard) on [XI_HI, XI_P]
    std::vector<double> res;   // [4][FOCK_NRES]: alpha, 1/Ai'(-alpha)^2, beta, 1/(beta Ai(-beta)^2)
    int n_nodes = 0;
};

void set_error(const std::string &msg);
int build_fock_table(FockHost *T);

// Face (planar reflector) data
struct FaceHost {
    double n[3], d;            // unit normal and offset, from the face's first triangle
    int first, count;          // range in the face -> triangle index list
};

// Frequencies are evaluated in chunks of NFC (one accumulator set each).
constexpr int NFC = 4;
// Per-chunk frequency constants (built on the host at rt_set_freqs).
struct FreqC {
    float k[NFC], kh[NFC];       // wavenumber, (k/2)^{1/3}
    float sk[NFC], pk[NFC];      // sqrt(k / (2 kh^2)), kh sqrt(2 / k): the per-frequency factors of the
                                 // Fock distance parameter and of the creeping amplitude
    float il_hi[NFC], il_lo[NFC];// 1/lambda as double-float
    double kd[NFC], fc[NFC];     // FP64: wavenumber, f/c
    int nf;                      // frequencies in this chunk (0 for path lists)
};

// Device-side scene description passed to the field kernel by value.
struct DevScene {
    int n_tri, n_face, n_body, n_f;
    const float4 *tri;         // [n_tri][3]: v0 (w: face id bits), v1 (w: altitude over edge v1v2... see tri_alt), v2
    const float4 *tri_alt;     // [n_tri]: altitudes h0 (v0 over v1v2), h1, h2 and unit-normal inverse scale
    const float4 *tri_nrm;     // [n_tri]: unit normal (xyz), offset n.v0 (w)
    const float4 *face32;      // [n_face]: unit normal, offset (FP32)
    const dq4 *face64;     // [n_face]: unit normal, offset (FP64)
    const int2 *face_rng;      // [n_face]: first, count in face_tris
    const float4 *face_box;    // [n_face][2]: box of the face's triangles (min, max), grown by the margin
                               // beyond which the FP32 face-membership test is a certain no
    const int *face_tris;      // [n_tri]
    const float4 *body;        // [n_body][2]: (cx, cy, cz, a), (h, type, 0, 0)
    const float4 *fock32;      // [FOCK_N][2]: (G.re, G.im, h G'.re, h G'.im) soft, hard; then
                               // [FOCK_NP][2]: (P.re, P.im, h P'.re, h P'.im) on [XI_HI, XI_P]
    const double2 *fock64;     // [FOCK_N][2][2]: G, G' (soft, hard)
    const float4 *res32;       // [FOCK_NRES][2]: (alpha sqrt3/2, alpha/2, coef, 0) soft, hard
    const dq4 *res64;      // [FOCK_NRES][2]
    const float *weid;         // [WEIDEMAN_N]
    const double *weid64;      // [WEIDEMAN_N]
    float weid_L;
    const float4 *img;         // [n_face + n_face^2][2]: source images (hi, lo) as double-float:
                               // [f] mirror of Tx in face f; [n_face + i n_face + j] in i then j
    int img_pairs;             // img holds the pair slots (faces <= RT_MAX_ENUM_FACES)
    const float4 *face_mat;    // [n_face]: (dielectric ? 1 : 0, eps', eps'', 0), eps_r = eps' - j eps''; or
                               // nullptr when every face is PEC
    const float4 *txb;         // [n_body][2] per transmitter, FP64-computed: (u, |S - c|), (beta_s, sqrt(|S-c|^2 - a^2) hi, lo,
                               // lateral paths possible ? 1 : 0); cylinders use horizontal distances
    const float4 *bvh;         // triangle BVH (nullptr: small scene, every triangle is tested); node i:
                               // (box min, first), (box max, count); count > 0 leaf over bvh_tri[first ..
                               // first + count), else children first, first + 1 (ints as float bits)
    const int *bvh_tri;        // triangle ids in leaf order
    int bvh_nodes;             // nodes of the BVH (numbered breadth first: the top levels first)
    const int4 *cand;          // [n_cand] candidate face sequences (f0, f1, f2, order), -1 padded, or nullptr
    const float4 *cimg;        // [n_cand][3][2]: the source's image after 1, 2, 3 reflections (hi, lo)
    int n_cand;                // the list's length, or (n_cand_dev set) an upper bound of it
    const int *n_cand_dev;     // device-built list: its length in device memory (else nullptr)
    const float4 *txw;         // [n_face][n_body][2]: as txb, for the source's mirror image in each face
                               // (wall -> creeping paths); nullptr in batches
    const double *freq;        // [n_f] Hz (host copy, read by the launcher)
    const FreqC *fqc;          // [ceil(n_f / NFC)] per-chunk frequency constants (device)
    float tx[3], pol[3];
    float band_len;            // FP32 decision band (m)
    int max_order;
    unsigned enable;
    int max_enc;               // extra encirclements of the creeping rays
};

// One frame of an evaluation: its curved bodies, frequencies and receivers
// (the triangles and the transmitter belong to the scene).  A plain
// evaluation is one frame passed by value; a batch is a device array of them.
// Each frame's first tile index (32 receivers a tile) is a multiple of
// TILE_ALIGN, so that a work unit of any class kernel lies in one frame.
constexpr int TILE_ALIGN = 12;
struct FrameDev {
    const float4 *body;        // [n_body][2], as DevScene::body
    const float4 *txb;         // [n_body][2], as DevScene::txb
    const FreqC *fqc;          // [ceil(n_f / NFC)] frequency constants
    long long rx_off;          // first receiver: SoA block at rx + 3 rx_off, flags at flags + rx_off
    long long e_off;           // first output float
    unsigned long long tile0;  // first tile of the batch's tile range
    double hl;                 // half the longest wavelength (caustic flag threshold)
    int n_rx, n_body;
    float band;                // FP32 decision band (m) of the frame's geometry
};

// Device counters of one evaluation: [0] candidates decided in FP64, [1 + i]
// the work queue of launch i.  Zeroed by the caller before launch_eval.
// Host side of the large-scene mode (bvh.cu): the triangle BVH (layout of
// DevScene::bvh) and the candidate face sequences of a ray launch.
void bvh_build(const float *tri, int n_tri, std::vector<float4> &nodes, std::vector<int> &order);
int ray_launch(const float *tri, const int *tri_face, int n_tri, int n_face, const std::vector<float4> &nodes,
               const std::vector<int> &order, const double tx[3], int n_rays, int max_order, std::vector<int> &seq);
// The launch's inputs, shared by the host launch and the device one
// (candidates.cu), so that both trace bit-identical rays: per face the unit
// normal of its first triangle, (v1 - v0) x (v2 - v0) / |.|, [n_face][3];
// the n_rays directions of the spherical Fibonacci lattice, [n_rays][3].
void ray_face_normals(const float *tri, const int *tri_face, int n_tri, int n_face, std::vector<double> &fn);
void ray_directions(int n_rays, std::vector<double> &dir);
constexpr int BVH_MIN_TRI = 64;        // scenes with more triangles traverse the BVH on the device

// Device ray launch (candidates.cu): at most RT_DEV_CAND_SLOTS ray prefixes
// (n_rays x max_order); the finished list is sorted and made unique in one
// block's shared memory.
struct DevCandBufs {
    double *dir;               // [n_rays][3]
    double *fn;                // [n_face][3]
    unsigned long long *keys;  // [RT_DEV_CAND_SLOTS]
    int4 *cand;                // [RT_DEV_CAND_SLOTS]
    float4 *cimg;              // [RT_DEV_CAND_SLOTS][3][2]
    int *n_cand;               // [1]
};
int launch_ray_candidates(const float4 *tri, const float4 *bvh, const int *bvh_tri, const dq4 *face64,
                          const double tx[3], int n_rays, int max_order, const DevCandBufs &B, cudaStream_t st);

constexpr int CTR_QUEUES = 256;
constexpr int CTR_N = 1 + CTR_QUEUES;

// Evaluate (codes == nullptr), list paths (e_out == nullptr: canonical
// order), or both (the path list in no particular order); *n_launches
// receives the number of kernel launches queued.
// shape: the tile shape (see launch_eval_batch), or nullptr for the default.
int launch_eval(const DevScene &S, const float *rx_soa, int n_rx, float *e_out, uint32_t *flags,
                uint64_t *codes, int32_t *counts, int cap, int precision, const int *shape, unsigned long long *ctr,
                cudaStream_t stream, int *n_launches);

// Evaluate the n_frames frames of frames_dev (device copy of frames_host):
// every frame has S.n_f frequencies and at most S.n_body bodies; n_tiles is
// the end of the last frame's tile range.  perm (or nullptr): the receivers
// in rx_soa are in a reordered sequence; sorted position rx_off + p of a
// frame holds its receiver perm[rx_off + p], where that receiver's outputs go.
// shape = {warps per tile of the planar kernel (1, 2, 4), of the body
// kernels (1, 2, 3, 4, 6, 12), planar frequency chunks per launch (1-4)}.
int launch_eval_batch(const DevScene &S, const FrameDev *frames_dev, const FrameDev *frames_host, int n_frames,
                      unsigned long long n_tiles, const float *rx_soa, const int32_t *perm, float *e_out,
                      uint32_t *flags, int precision, const int shape[3], unsigned long long *ctr,
                      cudaStream_t stream, int *n_launches);

// Gradient of a loss through the fields (adjoint pass, eval_fields.cu): for
// the n_rx receivers' listed paths (codes/counts/cap as rt_paths wrote
// them), the sums of dLoss/dE (grad_e, as the fields) times each path's
// field derivative: g_body [n_body][4] (centre x, y, z, radius), g_tx [3],
// g_f [n_f]; all zeroed first.  queue: one device counter.  precision:
// RT_PREC_FP32 (FP32 dual numbers) or RT_PREC_FP64.
int launch_adjoint(const DevScene &S, const float *rx_soa, int n_rx, const uint64_t *codes, const int32_t *counts,
                   int cap, const float *grad_e, double *g_body, double *g_tx, double *g_f,
                   unsigned long long *queue, int precision, cudaStream_t st);

// Received power in dBm (power.cu): p_out [n_f][n_rx] from the field
// e_out [n_f][3][n_rx][2]; c0_dev [n_f] device floats P_t + 20 log10(lambda /
// 4 pi); pol host float[3] (normalised here) or nullptr for |E|.
int launch_power_dbm(const float *e_out, int n_f, int n_rx, const float *c0_dev, const float pol[3], float *p_out,
                     cudaStream_t st);

// Spatial ordering of a batch's receivers (rx_order.cu): a counting sort per
// frame on the RX_GRID x RX_GRID cells (Morton order) of the rectangle grid
// = (x0, y0, cells per metre in x, in y).  Scratch: cnt [n_frames][RX_CELLS],
// rank [total receivers]; results: rx_sorted (SoA per frame, as rx) and perm
// (see launch_eval_batch).  max_rx: the largest frame.
constexpr int RX_GRID = 128;
constexpr int RX_CELLS = RX_GRID * RX_GRID;
int launch_rx_order(const FrameDev *frames_dev, int n_frames, int max_rx, const float *rx, float4 grid,
                    uint32_t *cnt, uint32_t *rank, float *rx_sorted, int32_t *perm, cudaStream_t st);

}  // namespace creep
