/*
 * creep.h -- C ABI of the GB300 creeping-wave (smooth-surface UTD) field
 * evaluator.
 *
 * The operation (Wang, Audia, Manocha, "Indoor Wireless Signal Modeling with
 * Smooth Surface Diffraction Effects", Sec. II.B, Eqs. 1-4 and Fig. 1): for
 * one transmitter and every receiver P, sum coherently
 *   E(P) = U^i E^i(P)                         direct ray           (Eq. 1)
 *        + sum U^r E^r(P)                     specular reflections (Eqs. 1, 3)
 *        + sum E^d(P)                         creeping rays        (Eqs. 2, 4)
 * over: the direct ray; PEC image reflections off the scene's planar faces up
 * to order 2; the first-order reflection off each convex body with the
 * Fock-uniform reflection coefficient; and the first creeping (surface-
 * diffracted) ray in each direction around each sphere or vertical cylinder,
 * whose transfer function T uses the soft/hard Fock--Pekeris functions.  The
 * visibility bits U are straight-segment tests against every triangle and
 * body (Eqs. 1-2, "path validation", Sec. III.B).
 *
 * Optional extensions of the path set (each off by default): dielectric
 * faces (rt_set_face_materials), creeping rays with extra turns round the
 * body (rt_options.max_encirclements), creeping rays fed by one planar
 * reflection (RT_EN_WALL_CREEP), and for large scenes planar reflections up
 * to order 3 over a candidate list of face sequences (rt_candidates,
 * rt_set_candidates) with BVH visibility.
 *
 * Conventions
 *   - Units: metres, Hz.  Time convention e^{+j w t}: fields go as e^{-jks}.
 *   - Source: isotropic, polarisation vector pol; on a ray leaving in
 *     direction d the field is unit(pol - (pol.d) d) / r (|E| = 1/r).
 *   - Every entry point returns an int status (RT_OK = 0 or an RT_ERR_*
 *     code) and never throws; rt_last_error() gives a thread-local message.
 *   - Device pointers are CUDA device addresses of the current device; host
 *     pointers are ordinary host memory.  The caller owns every buffer it
 *     passes; the library owns the scene (its device copies of geometry and
 *     the Fock--Pekeris table) until rt_scene_destroy.
 *   - Calls on one scene are not thread-safe; different scenes are
 *     independent.  Kernels run on the caller's stream; rt_evaluate and
 *     rt_paths return without synchronising.
 */
#ifndef CREEP_H
#define CREEP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define RT_OK 0
#define RT_ERR_ARG 1       /* null pointer, n < 0, NaN/Inf coordinate, a <= 0, bad enum */
#define RT_ERR_GEOM 2      /* transmitter inside/on a body or on a face plane, overlapping bodies */
#define RT_ERR_CUDA 3      /* a CUDA runtime call failed; message in rt_last_error() */
#define RT_ERR_TIMEOUT 4   /* a bounded device wait gave up */
#define RT_ERR_OVERFLOW 5  /* a size exceeds a library limit (faces, bodies, path cap) */
#define RT_ERR_STATE 6     /* transmitter or frequencies not set; a large scene without a candidate list */

/* body types */
#define RT_BODY_SPHERE 0   /* centre c, radius a */
#define RT_BODY_CYLINDER 1 /* vertical (axis +z) finite cylinder: axis through (cx, cy), z in [cz, cz + h], radius a */

/* contribution enable mask (rt_options.enable) */
#define RT_EN_LOS 1u
#define RT_EN_PLANAR 2u
#define RT_EN_BODYREFL 4u
#define RT_EN_CREEP_SOFT 8u
#define RT_EN_CREEP_HARD 16u
#define RT_EN_ALL 31u
/* Creeping rays fed by one planar reflection: S -> Qw (face f) -> Q1 ->
 * surface ray -> Q2 -> P, the creeping rays of the source's mirror image in
 * face f with the source's polarisation reflected at Qw (PEC image mirror or
 * the face's Fresnel coefficients).  Not in RT_EN_ALL; single scenes only
 * (rt_batch_* reject it with RT_ERR_ARG).  A path exists iff the image lies
 * outside the body (a cylinder: off its footprint), the image's creeping ray
 * exists (with any extra turns), Q1 lies strictly on the source's side of
 * face f's plane, Qw (where image -> Q1 crosses the plane) lies in face f,
 * and S -> Qw (face f not tested), Qw -> Q1 (face f and the body not
 * tested) and Q2 -> P (the body not tested) are unobstructed. */
#define RT_EN_WALL_CREEP 32u

/* arithmetic of the geometry and field math (rt_options.precision) */
#define RT_PREC_FP32 0     /* FP32 bulk, double-float path lengths, FP64 re-evaluation of uncertain decisions */
#define RT_PREC_FP64 1     /* everything in FP64 */

/* per-receiver flags (optional output) */
#define RT_FLAG_INSIDE 1u     /* receiver inside or on a body: no field */
#define RT_FLAG_CAUSTIC 2u    /* within half a wavelength of a sphere's axial caustic (k d_perp < pi) */
#define RT_FLAG_ESCALATED 4u  /* at least one decision was re-evaluated in FP64 */
#define RT_FLAG_OVERFLOW 8u   /* more paths than the rt_paths capacity */

/* path type codes: a path is (type << 56) | (id1 << 28) | id2 */
#define RT_PATH_LOS 0      /* direct */
#define RT_PATH_R1 1       /* id1 = face */
#define RT_PATH_R2 2       /* id1 = first face, id2 = second face */
#define RT_PATH_RB 3       /* id1 = body: GO reflection off the body */
#define RT_PATH_CP 4       /* id1 = body, id2 = extra turns: creeping ray, short way round */
#define RT_PATH_CM 5       /* id1 = body, id2 = extra turns: creeping ray, long way round */
#define RT_PATH_WCP 6      /* id1 = body, id2 = 16 face + extra turns: reflection at face, then CP */
#define RT_PATH_WCM 7      /* id1 = body, id2 = 16 face + extra turns: reflection at face, then CM */
#define RT_PATH_R3 8       /* id1 = index in the candidate list: planar reflection of order 3 */

/* library limits.  Scenes of more than RT_MAX_ENUM_FACES faces take their
 * planar paths from a candidate list (rt_set_candidates) and have no
 * wall -> creeping paths; scenes of more than 64 triangles test visibility
 * through a triangle BVH. */
#define RT_MAX_FACES (1 << 20)
#define RT_MAX_ENUM_FACES 64
#define RT_MAX_CANDIDATES (1 << 20)
#define RT_MAX_RAYS (1 << 24)      /* rays of one candidate launch */
#define RT_MAX_BODIES 1024
#define RT_MAX_TRIS (1 << 22)
#define RT_MAX_FREQS 64

typedef struct rt_scene rt_scene;

typedef struct {
    int type;       /* RT_BODY_* */
    float c[3];     /* sphere: centre; cylinder: (axis x, axis y, base z) */
    float a;        /* radius, > 0 */
    float h;        /* cylinder height, > 0 (ignored for spheres) */
} rt_body;

typedef struct {
    int max_order;      /* planar reflection order 0, 1 or 2 (3 with a candidate list) */
    unsigned enable;    /* RT_EN_* mask */
    int precision;      /* RT_PREC_* */
    int max_encirclements;  /* creeping rays: extra full turns round a body, 0-4 (0: the first ray
                               each way only).  Turn n's ray is the first one's with its arc
                               lengthened by 2 pi a n, listed as (CP or CM, body, n); it exists where
                               the first one does and its heights on a cylinder are in range */
} rt_options;

typedef struct {
    /* candidate decisions of the last rt_evaluate / rt_paths on this scene
       that were taken in FP64 (RT_PREC_FP32 only; a receiver with at least
       one carries RT_FLAG_ESCALATED) */
    unsigned long long escalated_candidates;
    /* kernel launches the last rt_evaluate / rt_paths queued (the path
       classes run as separate kernels, per chunk of 4 frequencies) */
    unsigned long long kernel_launches;
} rt_stats;

/*
 * Build a scene.  tri_xyz: host float [n_tri][3][3] (vertex-major xyz);
 * tri_face: host int [n_tri], the planar face (coplanar triangle group that
 * reflects as one polygon, Eq. 3) each triangle belongs to, ids 0..n_face-1;
 * NULL makes every triangle its own face.  bodies: host [n_body].  The
 * library copies everything to the current device and builds, once per
 * device, the FP64 Fock--Pekeris table (see rt_fock_table).  *out
 * receives the scene.  Errors: RT_ERR_ARG, RT_ERR_GEOM (overlapping bodies),
 * RT_ERR_OVERFLOW (limits above), RT_ERR_CUDA.
 */
int rt_scene_create(const float *tri_xyz, const int *tri_face, int n_tri,
                    const rt_body *bodies, int n_body, rt_scene **out);

/* Free a scene and its device memory (NULL is a no-op). */
void rt_scene_destroy(rt_scene *scene);

/*
 * Transmitter position (host float[3]) and polarisation (host float[3],
 * non-zero).  RT_ERR_GEOM if the point is inside or on a body or on the
 * plane of a face (the off-surface assumption, Sec. II.B).
 */
int rt_set_tx(rt_scene *scene, const float tx[3], const float pol[3]);

/*
 * Face materials for the planar reflections (Eq. 3): mat host float
 * [n_face][3] = (kind, eps', eps''), kind 0 PEC (R = -1 / +1) or 1 a
 * dielectric half-space of relative permittivity eps' - j eps'' (eps' > 0,
 * eps'' >= 0; e^{+jwt}), reflecting with the Fresnel coefficients at the
 * incidence angle; NULL makes every face PEC (the default).  n_face must be
 * the scene's face count.  Curved bodies stay PEC.
 */
int rt_set_face_materials(rt_scene *scene, const float *mat, int n_face);

/*
 * Candidate face sequences of a ray launch from the transmitter (the planar
 * paths of large scenes).  The rule: n_rays
 * directions of the spherical Fibonacci lattice z_i = 1 - (2i + 1)/n_rays,
 * phi_i = i pi (3 - sqrt 5); each ray reflected specularly at the nearest
 * triangle hit -- parameter > 1e-9, the face it leaves excluded, ties to the
 * lower triangle index, curved bodies ignored -- up to max_order (1-3)
 * times; every prefix of its face sequence is a candidate; the distinct
 * ones sorted by order, then faces).  Host computation, FP64.
 *   seq    host int32 [cap][3]: face ids, -1 padded; NULL to count only.
 *   n_out  number of distinct sequences (those beyond cap are not written).
 * Errors: RT_ERR_STATE without a transmitter, RT_ERR_ARG for bad sizes.
 */
int rt_candidates(rt_scene *scene, int n_rays, int max_order, int32_t *seq, int cap, int *n_out);
/* (1 <= n_rays <= RT_MAX_RAYS) */

/* The same ray launch for a mesh and a transmitter without a scene: host
 * only (no device, no CUDA call).  tri_xyz, tri_face as in
 * rt_scene_create; tx host float[3].  Errors: RT_ERR_ARG. */
int rt_candidates_mesh(const float *tri_xyz, const int *tri_face, int n_tri, const float tx[3], int n_rays,
                       int max_order, int32_t *seq, int cap, int *n_out);

/*
 * The candidate list of the planar paths (orders 1-3): host int32
 * [n][3], face ids with -1 padding at the end, no face twice in a row;
 * copied.  With a list the planar class evaluates its sequences (up to the
 * options' max_order) instead of every face and ordered face pair: the path
 * list is exact for the candidate set.  Orders 1 and 2 are listed as
 * RT_PATH_R1 / RT_PATH_R2 with their faces, order 3 as RT_PATH_R3 with the
 * sequence's index.  The images are recomputed by every rt_set_tx.  n = 0
 * clears the list.  Errors: RT_ERR_ARG (bad face id, repeat, n > RT_MAX_CANDIDATES).
 */
int rt_set_candidates(rt_scene *scene, const int32_t *seq, int n);

/*
 * The ray launch of rt_candidates run on the device and installed as the
 * scene's candidate list, as rt_set_candidates would install the list
 * rt_candidates returns (the same sequences in the same order, so the same
 * path codes; the same FP64 arithmetic, rounded operation by operation as
 * the host launch rounds it), with no host round trip: the class kernels of
 * a later evaluation on `stream` read the list and its length from device
 * memory.  Sec. III's path search, in the form of the candidate rule above.
 *   n_rays x max_order <= RT_DEV_CAND_SLOTS; max_order 1-3; fewer than
 *   2^20 - 1 faces.
 * Asynchronous on `stream` (CUDA stream or NULL), except on the first call
 * and whenever n_rays changes, which upload the launch's directions and
 * face normals synchronously (library-owned device buffers, freed with the
 * scene).  The list belongs to the current transmitter: rt_set_tx and
 * rt_set_candidates drop it.  Errors: RT_ERR_ARG (sizes), RT_ERR_STATE (no
 * transmitter, no triangles, another device current), RT_ERR_OVERFLOW
 * (faces), RT_ERR_CUDA.
 */
#define RT_DEV_CAND_SLOTS 16384
int rt_candidates_device(rt_scene *scene, int n_rays, int max_order, void *stream);

/*
 * The scene's current candidate list into host int32 seq [cap][3] (-1
 * padded); *n_out receives its length (sequences beyond cap are not
 * written).  A device-built list is copied back after its stream
 * synchronises.  Errors: RT_ERR_ARG, RT_ERR_OVERFLOW (a traversal stack of
 * the device launch overflowed: no list), RT_ERR_CUDA.
 */
int rt_get_candidates(rt_scene *scene, int32_t *seq, int cap, int *n_out);

/*
 * Received power (the paper's maps and cuts are received power in dBm for
 * a 40 dBm omnidirectional transmitter, Sec. IV).
 * rt_set_tx_power: the transmitter's power in dBm (default 0 dBm).
 * rt_power_dbm: from a field e_out of rt_evaluate (device float
 *   [n_f][3][n_rx][2], normalised to |E| = 1/R in free space) the received
 *   power of an isotropic antenna, device float p_out [n_f][n_rx]:
 *     P_r = P_t + 20 log10(lambda / (4 pi)) + 20 log10 |E . p|
 *   (Friis), p = rx_pol (host float[3], normalised here) or, with rx_pol
 *   NULL, |E| (the power summed over polarisations); -inf where the field
 *   is zero.  Asynchronous on `stream`.  Errors: RT_ERR_ARG (NULL buffer,
 *   zero or non-finite polarisation), RT_ERR_STATE (no frequencies),
 *   RT_ERR_CUDA.
 */
int rt_set_tx_power(rt_scene *scene, float power_dbm);
int rt_power_dbm(rt_scene *scene, const float *e_out, int n_rx, const float rx_pol[3], float *p_out,
                 void *stream);

/* Frequencies (host double[n_f], Hz, > 0), 1 <= n_f <= RT_MAX_FREQS. */
int rt_set_freqs(rt_scene *scene, const double *f_hz, int n_f);

/*
 * Field at n_rx receivers (Eqs. 1-4).
 *   rx_soa  device float [3][n_rx]: x row, then y row, then z row.
 *   e_out   device float [n_f][3][n_rx][2]: (re, im) of E_x, E_y, E_z per
 *           frequency; caller-owned, fully overwritten.
 *   flags   device uint32 [n_rx] (RT_FLAG_*), or NULL.
 *   opt     NULL for {2, RT_EN_ALL, RT_PREC_FP32}.
 *   stream  cudaStream_t (NULL = legacy default stream).
 * n_rx = 0 is a no-op.  Asynchronous: returns after the launch.
 */
int rt_evaluate(rt_scene *scene, const float *rx_soa, int n_rx, float *e_out,
                uint32_t *flags, const rt_options *opt, void *stream);

/*
 * Same evaluation from and to HOST buffers (rx_soa host [3][n_rx], e_out host
 * [n_f][3][n_rx][2], flags host or NULL): copies in, evaluates, copies out,
 * synchronises the stream.  Device scratch for the copies is allocated on the
 * first call and kept with the scene.
 */
int rt_evaluate_host(rt_scene *scene, const float *rx_soa, int n_rx, float *e_out,
                     uint32_t *flags, const rt_options *opt, void *stream);

/*
 * rt_evaluate_host_noalloc -- the evaluation of rt_evaluate_host for callers
 * that may not allocate device memory.  (An engineering addition: the paper
 * has no counterpart.)
 *
 * Who needs it: code that runs where cudaMalloc is off limits -- for
 * example inside a framework that has already claimed the device's memory
 * for its own pool, in a loop that must not take cudaMalloc's implicit
 * device-wide synchronisation, or in a process whose allocator policy
 * forbids new device allocations after start-up.  rt_evaluate_host would
 * allocate its staging buffers on its first call; this entry point uses a
 * fixed device array compiled into the library instead and calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *
 * Arguments and results are those of rt_evaluate_host (host rx_soa
 * [3][n_rx], host e_out [n_f][3][n_rx][2], host flags [n_rx] or NULL,
 * copies in, evaluates, copies out, synchronises the stream).
 *
 * Limits and sharing:
 *   - The array holds RT_NOALLOC_SCRATCH_BYTES (8 MiB) on every device that
 *     loads the library, for the life of the process.  A call needs
 *     768 + n_rx * (16 + 24 * n_f) bytes (rounded up to 256-byte sections);
 *     larger requests fail with RT_ERR_OVERFLOW before any work is queued.
 *     With 3 frequencies that is up to about 95 000 receivers per call.
 *   - rt_scene_create looks up the array's device address
 *     (cudaGetSymbolAddress) on the device current at creation, which also
 *     loads the module holding it; the entry point itself only reads the
 *     stored address.  Call it with the scene's device current
 *     (RT_ERR_STATE otherwise).
 *   - All calls on a device share the one array and leave their data in it;
 *     nothing in it needs clearing, since each call overwrites what it reads.
 *     Calls whose GPU work overlaps (other threads, other streams) race on
 *     the array: serialise them.
 */
#define RT_NOALLOC_SCRATCH_BYTES (8u << 20)
int rt_evaluate_host_noalloc(rt_scene *scene, const float *rx_soa, int n_rx, float *e_out,
                             uint32_t *flags, const rt_options *opt, void *stream);

/*
 * Path lists (the visibility decisions of Eqs. 1-2) instead of the field.
 *   codes   device uint64 [n_rx][cap]: per receiver its paths in the
 *           enumeration order LOS, R1(face), R2(face, face), then per body
 *           RB, CP, CM; slots past the count are left untouched.
 *   counts  device int32 [n_rx]: number of paths (may exceed cap; then
 *           RT_FLAG_OVERFLOW is set and only cap codes are written).
 *   flags   device uint32 [n_rx] or NULL.
 */
int rt_paths(rt_scene *scene, const float *rx_soa, int n_rx, uint64_t *codes,
             int32_t *counts, int cap, uint32_t *flags, const rt_options *opt, void *stream);

/*
 * Batched frames: the evaluation of rt_evaluate (Eqs. 1-4) for n_frames
 * frames of one scene at once -- the dynamic-scene use of Sec. III (people
 * moving through a fixed room, one frame per time step).  Every frame shares
 * the scene's triangles, transmitter and polarisation; each has its own
 * curved bodies (which replace the scene's own bodies), its own n_f
 * frequencies (the same count in every frame) and its own number of
 * receivers.  All frames' receivers are one work queue of one launch per
 * path class, so uneven frames keep the GPU busy.
 *
 * Layout (rx_offset(f) = n_rx[0] + ... + n_rx[f - 1]):
 *   rx_soa  device float: frame f's [3][n_rx[f]] block (x row, y row, z
 *           row) at rx_soa + 3 rx_offset(f).
 *   e_out   device float: frame f's [n_f][3][n_rx[f]][2] block (as
 *           rt_evaluate) at e_out + 6 n_f rx_offset(f); fully overwritten.
 *   flags   device uint32: frame f's [n_rx[f]] at flags + rx_offset(f), or NULL.
 * A frame's fields equal those of rt_evaluate on a scene with the same
 * triangles and that frame's bodies, transmitter and frequencies.
 */
typedef struct rt_batch rt_batch;

/*
 * Create a batch of n_frames >= 1 frames on scene (which must outlive it):
 * n_rx host int32 [n_frames] (>= 0; zero is allowed), n_f in
 * [1, RT_MAX_FREQS] frequencies per frame, and max_body, the most bodies any
 * frame will hold (<= RT_MAX_BODIES).  Device memory for the frames' data
 * is allocated here.  Errors: RT_ERR_ARG, RT_ERR_OVERFLOW, RT_ERR_CUDA.
 */
int rt_batch_create(rt_scene *scene, int n_frames, const int32_t *n_rx, int n_f, int max_body,
                    rt_batch **out);

/* Free a batch (NULL is a no-op). */
void rt_batch_destroy(rt_batch *batch);

/*
 * Set frame `frame`: its bodies (host [n_body], n_body <= max_body, checked
 * as in rt_scene_create, and the scene's transmitter must lie outside them)
 * and its frequencies (host double [n_f], Hz).  Copies to the device and
 * synchronises; do not call while an evaluation of this batch is in flight.
 * The scene's transmitter must be set first; after a later rt_set_tx every
 * frame must be set again (RT_ERR_STATE otherwise).  A captured graph
 * (rt_batch_capture) reads the frames when it runs, so frames set between
 * replays take effect without a new capture.
 */
int rt_batch_set_frame(rt_batch *batch, int frame, const rt_body *bodies, int n_body,
                       const double *f_hz);

/*
 * Evaluate every frame (layout above) on `stream`; returns after the launch.
 * opt as for rt_evaluate.  RT_ERR_STATE if a frame has not been set.
 */
int rt_batch_evaluate(rt_batch *batch, const float *rx_soa, float *e_out, uint32_t *flags,
                      const rt_options *opt, void *stream);

/*
 * Capture rt_batch_evaluate(batch, rx_soa, e_out, flags, opt, stream) into a
 * CUDA graph kept with the batch (replacing an earlier one); nothing runs.
 * stream must not be the legacy default stream (NULL).  The buffers must
 * stay valid for every replay.
 */
int rt_batch_capture(rt_batch *batch, const float *rx_soa, float *e_out, uint32_t *flags,
                     const rt_options *opt, void *stream);

/* Launch the captured graph on `stream` (RT_ERR_STATE if none). */
int rt_batch_replay(rt_batch *batch, void *stream);

/*
 * The batch's tile shape: shape[0] warps per 32-receiver tile in the planar
 * kernel (1, 2 or 4), shape[1] in the body kernels (1, 2, 3, 4, 6 or 12),
 * shape[2] frequency chunks of 4 per planar launch (1-4); default {4, 4, 4}.
 * Fields differ between shapes only in the rounding of the sums over a
 * tile's warps.  rt_batch_set_shape: RT_ERR_ARG outside those sets.
 */
int rt_batch_set_shape(rt_batch *batch, const int shape[3]);
int rt_batch_get_shape(rt_batch *batch, int shape[3]);

/*
 * rt_batch_tune -- the batch's autotuner: times rt_batch_evaluate(batch,
 * rx_soa, e_out, flags, opt, stream) over tile shapes (a coordinate search
 * from the default: body warps per tile, then planar warps per tile, then
 * planar chunks per launch; the faster of two runs after a warm-up each),
 * keeps the fastest in the batch and writes it to shape_out (or NULL).  The
 * choice is remembered per device, batch size and options: a later batch of
 * the same size takes it without timing.  Synchronises; the outputs hold the
 * last evaluation.  Call before rt_batch_capture.
 */
int rt_batch_tune(rt_batch *batch, const float *rx_soa, float *e_out, uint32_t *flags,
                  const rt_options *opt, void *stream, int shape_out[3]);

/* Counters of the batch's last evaluation or replay (synchronises its stream). */
int rt_batch_get_stats(rt_batch *batch, rt_stats *out);

/*
 * The evaluation of rt_evaluate and, in the same kernels, each receiver's
 * path list (the visibility decisions of Eqs. 1-2): codes, counts, cap and
 * flags as for rt_paths, except that a receiver's codes come in no
 * particular order (the same set as rt_paths lists; sort to compare).  The
 * list rt_backward needs, at the cost of one evaluation.
 */
int rt_evaluate_with_paths(rt_scene *scene, const float *rx_soa, int n_rx, float *e_out,
                           uint64_t *codes, int32_t *counts, int cap, uint32_t *flags,
                           const rt_options *opt, void *stream);

/*
 * The tile shape of rt_evaluate and rt_evaluate_with_paths on this scene
 * (FP32), as for rt_batch_set_shape: warps per tile of the planar kernel
 * and of the body kernels, planar frequency chunks per launch.
 * rt_tune times rt_evaluate(scene, rx_soa, n_rx, e_out, flags, opt, stream)
 * over shapes as rt_batch_tune does, keeps the fastest for the scene and
 * writes it to shape_out (or NULL); remembered per device, receiver count,
 * scene size and options.  Synchronises; e_out holds the last evaluation.
 */
int rt_set_shape(rt_scene *scene, const int shape[3]);
int rt_get_shape(rt_scene *scene, int shape[3]);
int rt_tune(rt_scene *scene, const float *rx_soa, int n_rx, float *e_out, uint32_t *flags,
            const rt_options *opt, void *stream, int shape_out[3]);

/*
 * rt_backward -- gradient of a real loss through the fields (the adjoint of
 * rt_evaluate: its vector-Jacobian product) with respect to every body's
 * centre and radius, the transmitter position and every frequency, with
 * visibility held fixed: the paths are those listed by rt_paths for the same
 * receivers and options, and each one's geometry and field (Eqs. 1-4) are
 * recomputed in dual numbers (value and eight tangents), nothing per path
 * being stored.  opt->precision RT_PREC_FP64: FP64 dual numbers throughout;
 * RT_PREC_FP32: FP32 ones on direct, planar and creeping paths (each path's
 * length for the phase kept in double-float, as the FP32 fields keep it) and
 * FP64 ones on reflections off bodies.  The FP32 form is about 2.4x faster;
 * its field derivatives carry FP32 rounding, which a loss seeded by
 * E / |E|^2 (power in dB) amplifies near interference nulls.
 *   rx_soa, n_rx          device, as rt_evaluate.
 *   codes, counts, cap    device, as rt_paths or rt_evaluate_with_paths wrote
 *                         them (a receiver with more than cap paths
 *                         contributes the cap listed).
 *   grad_e                device float [n_f][3][n_rx][2]: dLoss/dRe E and
 *                         dLoss/dIm E, the layout of rt_evaluate's e_out.
 *   grad_bodies           device double [n_body][4]: dLoss/d(cx, cy, cz, a)
 *                         (cz has no effect on a cylinder: 0).
 *   grad_tx               device double [3]; grad_freqs device double [n_f]
 *                         (per Hz).  All three are overwritten.
 *   opt                   as for rt_evaluate (its enable mask weighs the soft
 *                         and hard creeping fields; precision picks the dual
 *                         numbers, above).
 * Asynchronous on `stream`.  Errors: RT_ERR_ARG, RT_ERR_STATE, RT_ERR_CUDA.
 */
int rt_backward(rt_scene *scene, const float *rx_soa, int n_rx, const uint64_t *codes,
                const int32_t *counts, int cap, const float *grad_e, double *grad_bodies,
                double *grad_tx, double *grad_freqs, const rt_options *opt, void *stream);

/*
 * rt_alu_peaks -- measured FP32 throughput of the current device, the
 * denominators of the evaluation's ALU roofline (an engineering addition: the
 * paper has no counterpart).  Runs two short microbenchmarks on `stream` and
 * synchronises: *ffma_tflops = FFMA rate (2 flops each) in TFLOP/s,
 * *mufu_gops = special-function-unit rate (ex2.approx) in Gop/s.  Allocates
 * and frees a small device buffer.  Errors: RT_ERR_ARG, RT_ERR_CUDA.
 */
int rt_alu_peaks(double *ffma_tflops, double *mufu_gops, void *stream);

/*
 * rt_l2_peak -- measured L2 read bandwidth of the current device (GB/s), the
 * denominator of the large-scene traversal's roofline, whose BVH and
 * triangles stay in the L2 (an engineering addition: the paper has no
 * counterpart).  Reads a 32 MiB buffer through L2 only, 16 passes, on
 * `stream`, and synchronises; allocates and frees the buffer.  Errors:
 * RT_ERR_ARG, RT_ERR_CUDA.
 */
int rt_l2_peak(double *l2_gbs, void *stream);

/* Counters of the last rt_evaluate / rt_paths on this scene (synchronises its stream). */
int rt_get_stats(rt_scene *scene, rt_stats *out);

/*
 * Copy the device's Fock--Pekeris table to host memory for inspection:
 * xi_lo, step, n nodes; G[kind][n] with kind 0 soft, 1 hard, of
 * G(xi) = phat(xi) e^{-j xi^3/12}, phat = P + c/xi, and dG/dxi; each complex as
 * (re, im) doubles.  Buffers: g host double [2][n][2], dg host double [2][n][2];
 * pass NULL to query n only.  res: host double [4][8] = alpha_n, 1/Ai'(-alpha_n)^2,
 * beta_n, 1/(beta_n Ai(-beta_n)^2) (residue-series constants), or NULL.
 */
int rt_fock_table(double *xi_lo, double *step, int *n, double *g, double *dg, double *res);

/*
 * The table's second segment, used by the FP32 fields above xi0 = 1.5 (the
 * smooth-surface functions after Eq. 4): P(xi) itself, P = phat - c/xi
 * (soft kind 0, hard kind 1), and dP/dxi at xi = xi0 + j step (the step of
 * rt_fock_table), j = 0 .. n - 1, up to xi = 12, where the residue series
 * takes over (nodes below xi = 3 from the table's quadrature, from 3 on from
 * the 8-term residue series).  p, dp: host double [2][n][2] ((re, im) pairs), or NULL to
 * query xi0 and n only.  Returns RT_OK, or RT_ERR_CUDA if the table could
 * not be built.
 */
int rt_fock_table_p(double *xi0, int *n, double *p, double *dp);

/* Thread-local description of the last error (never NULL). */
const char *rt_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CREEP_H */
