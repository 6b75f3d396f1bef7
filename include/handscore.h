/*
 * handscore.h -- C-ABI of the B300 hypothesis-scoring library (libhandscore.so)
 * for the model-based 26-DOF hand tracker of arxiv 2005.07068.
 *
 * One PSO generation is   pose_fk -> render_score_batch -> pso_step,
 * all asynchronous on the caller's stream.  The paper defines the problem as
 * argmin_h E(h, O) (Section III.A, Eq. 5) minimised by PSO (Section III.B).
 *
 * Conventions
 *  - Every data pointer is a DEVICE pointer owned by the caller, unless a
 *    parameter says "host".  Scoring calls allocate nothing: scratch memory
 *    is the caller's workspace (hs_workspace_size).
 *  - Every call returns an int status: HS_OK (0) or a negative HS_ERR_* code.
 *    Arguments are validated on the host before anything is launched; an
 *    invalid call launches nothing and never aborts or traps.
 *  - Kernels that meet bad data at run time (a non-finite pose, a wait that
 *    timed out) set bits of a device status word, readable with
 *    hs_get_device_status.
 *  - Units: mm and rad.  Pose layout (Eq. 1-3): [x, y, z, theta_x, theta_y,
 *    theta_z] of the wrist, then (MP_x, MP_z, PIP, DIP) for thumb, index,
 *    middle, ring, pinky: 26 floats, row-major [P][26].
 *  - Images are row-major with a row pitch in BYTES that must be a multiple
 *    of 16 (the observation tiles are fetched with TMA); base addresses must
 *    be 16-byte aligned.
 */
#ifndef HANDSCORE_H
#define HANDSCORE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* a CUDA stream (cudaStream_t); NULL is the legacy default stream */
typedef struct CUstream_st* hs_stream_t;

/* ---- status codes ------------------------------------------------------ */
#define HS_OK            0
#define HS_ERR_ARG      -1  /* NULL pointer, bad enum, non-finite parameter */
#define HS_ERR_ALIGN    -2  /* pointer not 16-B aligned or pitch not a multiple of 16 */
#define HS_ERR_SIZE     -3  /* size out of range or workspace too small */
#define HS_ERR_TIMEOUT  -4  /* a device wait ran out (see hs_get_device_status) */
#define HS_ERR_NOT_IMPL -5
#define HS_ERR_CUDA     -6  /* a CUDA runtime call failed (launch, copy, driver entry point) */

/* ---- device status bits (hs_get_device_status) ------------------------- */
#define HS_DEV_NONFINITE_POSE 0x1u /* pose_fk met a NaN/inf pose; that particle's E is NaN */
#define HS_DEV_TMA_TIMEOUT    0x2u /* an observation tile load did not arrive in time */
#define HS_DEV_BARRIER_TIMEOUT 0x4u /* track_frame(_multi): a wait for other CTAs ran out (the frame's results are void) */

/* ---- limits -------------------------------------------------------------- */
#define HS_NDOF            26
#define HS_MAX_BONES       32
#define HS_MAX_PRIMS       64
#define HS_MAX_DEPTH       7      /* bone chains: the palm at depth 0, its descendants at most this deep */
#define HS_MAX_PARTICLES   65535  /* particles per call (the render grid's y extent) */
#define HS_MAX_ROI         8192   /* W, H <= HS_MAX_ROI */

/* ---- hand model (Section II.A, Fig. 2) ----------------------------------- */
#define HS_PRIM_ELLIPSOID 0  /* dims = (sx, sy, sz, unused): semi-axes, mm      */
#define HS_PRIM_ECONE     1  /* dims = (ax, az, hl, kappa): capped elliptic truncated
                                cone along local y, |y| <= hl, section semi-axes
                                (ax, az) * (1 + kappa * y / hl), |kappa| < 1;
                                kappa = 0 is an elliptic cylinder                 */

/* Bone b > 0 has frame  parent * T(offset) * Rz(rest[2]) Ry(rest[1]) Rx(rest[0])
 * * Rz(pose[dof_z]) * Rx(pose[dof_x])  (a dof of -1 means none).  Bone 0 is the
 * palm: origin at the wrist pose[0..2], rotation diag(1,-1,-1) *
 * Rz(pose[5]) Ry(pose[4]) Rx(pose[3]).  Bones must be listed parents first. */
typedef struct {
    int32_t parent;     /* < own index; ignored for bone 0 */
    int32_t dof_z;      /* pose index driving Rz, or -1 */
    int32_t dof_x;      /* pose index driving Rx, or -1 */
    int32_t reserved;
    float offset[3];    /* bone origin in the parent frame, mm */
    float rest[3];      /* fixed rest rotation angles (x, y, z), rad */
} HsBoneDesc;

/* a primitive is axis-aligned with its bone, centred at `center` (bone frame) */
typedef struct {
    int32_t bone;
    int32_t kind;       /* HS_PRIM_ELLIPSOID or HS_PRIM_ECONE */
    float center[3];
    float dims[4];
} HsPrimDesc;

typedef struct {
    int32_t n_bones;            /* 1..HS_MAX_BONES */
    int32_t n_prims;            /* 1..HS_MAX_PRIMS */
    const HsBoneDesc* bones;    /* host [n_bones] */
    const HsPrimDesc* prims;    /* host [n_prims] */
    float lo[HS_NDOF];          /* joint limits (Tables 1-2, possibly narrowed), mm / rad */
    float hi[HS_NDOF];
} HsModelDesc;

/* opaque validated model; lives in host memory only (it is passed to the
 * kernels by value as a launch parameter) */
typedef struct HsModel HsModel;

/* pinhole camera; pixel (u, v) casts the ray ((u+0.5-cx)/fx, (v+0.5-cy)/fy, 1),
 * so depth = camera z (Kinect convention) */
typedef struct {
    float fx, fy, cx, cy;
} HsCamera;

#define HS_DEPTH_U16 0  /* uint16 mm, 0 = hole / undefined */
#define HS_DEPTH_F32 1  /* float32 mm, 0 = undefined */

/* observation O = (O_s, O_d) of Section II.B, one ROI */
typedef struct {
    const void* depth;      /* device [H][depth_pitch bytes] */
    const uint8_t* skin;    /* device [H][skin_pitch bytes], nonzero = skin */
    int32_t W, H;           /* ROI size, 1..HS_MAX_ROI */
    int32_t depth_pitch;    /* bytes, multiple of 16, >= W * element size */
    int32_t skin_pitch;     /* bytes, multiple of 16, >= W */
    int32_t depth_type;     /* HS_DEPTH_U16 or HS_DEPTH_F32 */
    uint32_t* stats;        /* device [2] (#valid depth pixels on skin, #skin pixels),
                               written by hs_obs_prepare, read by render_score_batch */
} HsObs;

/* Render kernels (all give the same E; they differ in how work is laid out):
 * the unit kernel walks pixels (16 x 4 blocks, primitives culled per 8 x 4
 * half), the tile kernels walk primitives (pixel-exact rectangles of each
 * primitive's box inside a TW x TH tile, nearest hit by a shared-memory
 * z-buffer), the strip kernels walk pixel strips 8 wide and 16 or 32 tall
 * (one warp per strip, each primitive's column terms formed once per strip,
 * nearest hit in registers).  HS_RENDER_AUTO picks by the number of
 * particles per call. */
#define HS_RENDER_AUTO        0
#define HS_RENDER_UNITS       1
#define HS_RENDER_TILES_32x16 2
#define HS_RENDER_TILES_32x32 3
#define HS_RENDER_TILES_64x32 4
#define HS_RENDER_TILES_64x64 5
#define HS_RENDER_STRIPS_8x16 6
#define HS_RENDER_STRIPS_8x32 7
/* the strip kernels as one persistent launch: one CTA per resident slot of
 * the GPU, each taking the next particle (of any swarm of a batch, largest
 * ROI first) from a counter in the workspace until all are scored;
 * ctas_per_particle is ignored */
#define HS_RENDER_PERSISTENT_8x16 8
#define HS_RENDER_PERSISTENT_8x32 9
#define HS_RENDER_VARIANTS    10

/* constants of Eq. 4-5 (paper: d_m = 1 cm, d_M = 4 cm, lambda = 20, lambda_k = 10),
 * in mm; 0 <= d_M < 127 (the depth sums are kept in 32-bit fixed point per pixel);
 * and the launch shape of the render (no effect on results): the kernel, and
 * the CTAs per particle (0 = about one resident wave in total, else 1..64) */
typedef struct {
    float d_m, d_M, lambda, lambda_k;
    int32_t variant;           /* HS_RENDER_* */
    int32_t ctas_per_particle;
} HsScoreParams;

/* per-particle sums of Eq. 4 (optional output of render_score_batch) */
typedef struct {
    float t_sum;        /* sum of the clamped depth term */
    uint32_t n_and;     /* sum(o_s AND r_m) */
    uint32_t n_or;      /* sum(o_s OR r_m) */
    uint32_t n_hit;     /* pixels where the hypothesis renders */
} HsParts;

/* 64-byte camera-space primitive record written by pose_fk (layout of float m[16]):
 *   m[0..8]  columns c0, c1, c2 of M = S^-1 R^T (R: primitive-to-camera rotation,
 *            S = diag of the primitive's scale), so a ray direction d = (a, b, 1)
 *            maps to h = a c0 + b c1 + c2 in scaled local coordinates
 *   m[9..11] C, the primitive centre in camera coordinates (mm); the renderer
 *            takes the ray point at depth t0 = C_z: g = M (t0 d - C)
 *   m[12]    bit mask (as uint32) of the cone caps to render (bit 0 at -hl,
 *            bit 1 at +hl); caps that the model hides inside a joint sphere or
 *            ellipsoid are left out, which does not change any depth
 *   m[13]    kappa for HS_PRIM_ECONE; 2.0 marks an ellipsoid
 *   m[14]    (int16 u0, int16 v0), m[15] (int16 u1, int16 v1): conservative
 *            inclusive pixel box of the primitive's projection; a primitive
 *            that reaches the plane z = 1 mm gets (-32767, -32767, 32767,
 *            32767).  The renderers take u0 != -32767 to mean that the whole
 *            solid lies beyond that plane (they then skip the far root and
 *            the tests of positive depth), so records made elsewhere than by
 *            pose_fk must keep that rule                                    */
typedef struct {
    float m[16];
} HsPrim;

/* swarm state, all device float arrays: x, v, pbest [P][26]; pbest_E [P];
 * gbest [26]; gbest_E [1]; E [P] = objective of x from render_score_batch */
typedef struct {
    float* x;
    float* v;
    float* pbest;
    float* pbest_E;
    float* gbest;
    float* gbest_E;
    const float* E;
} HsSwarm;

/* Section III.B: c1 = 2.8, c2 = 1.3; w = 2 / |2 - psi - sqrt(psi^2 - 4 psi)|,
 * psi = c1 + c2 > 4 (computed by pso_step); mutation every 3 generations of
 * the worst half (n_mutate = P / 2); mutate_every <= 0 disables it.
 * e_stop: Section III.B's stopping rule (the search ends once the best E
 * falls below a threshold; the paper uses 1.0), per swarm and on the device,
 * for the batch calls only (pso_step_fk_multi): 0 disables it, and the
 * single-swarm calls require 0. */
typedef struct {
    float c1, c2;
    int32_t mutate_every;
    int32_t n_mutate;
    float e_stop;
} HsPsoParams;

/* ---- kc variants (Section III.A, after Eq. 5) -----------------------------
 * The paper adds lambda_k kc(h) to E to rule out implausible poses such as
 * two fingers passing through each other, with kc the sum over the three
 * adjacent pairs of non-thumb fingers of -min(phi, 0), phi the abduction
 * difference of the pair (rad).  That only orders the abduction angles; the
 * variants below add a direct test of interpenetration between fingers:
 *   pen(h) = sum over pairs of collision proxies on different fingers of
 *            max(0, r_i + r_j - |c_i - c_j|)   (mm)
 * with the proxies the inscribed spheres of the model: one per ellipsoid
 * primitive (centre, smallest semi-axis) and three per cone primitive, on its
 * axis at y = -hl/2, 0, +hl/2, each the largest sphere about that point inside
 * the cone of circular section rho (1 + kappa y / hl), rho = min(ax, az):
 * radius min(rho (1 + kappa y / hl) / sqrt(1 + (rho kappa / hl)^2), hl - |y|).  A
 * primitive's finger is the child of the palm bone (bone 0) on its bone's
 * path to the palm; palm primitives (bone 0) take no part, nor do pairs of
 * two proxies centred at the origins of bones attached to the palm (knuckle
 * spheres: their distance is a constant of the model).  kc is then
 *   HS_KC_ABDUCTION : the paper's kc (default)
 *   HS_KC_ABD_PEN   : the paper's kc + pen_weight * pen
 *   HS_KC_PEN       : pen_weight * pen
 * (pen_weight in rad per mm, so that lambda_k applies to both).  pose_fk,
 * pso_step_fk, track_frame and the batch calls return this kc, and pose_grad
 * differentiates it (d pen / d pose: each penetrating pair contributes the
 * unit vector between its centres, moved by the bones' tangents). */
#define HS_KC_ABDUCTION 0
#define HS_KC_ABD_PEN   1
#define HS_KC_PEN       2
#define HS_MAX_PROXIES  128
#define HS_MAX_PROXY_PAIRS 2048
typedef struct {
    int32_t variant;    /* HS_KC_* */
    float pen_weight;   /* rad per mm of penetration, >= 0 */
} HsKcParams;

/* ---- calls ------------------------------------------------------------------ */

/* library version (major * 10000 + minor * 100 + patch) */
int hs_version(void);

/* static text for a status code */
const char* hs_status_string(int status);

/* Validate a model descriptor (Section II.A) and copy it into an opaque host
 * object.  Allocates host memory only.  Errors: HS_ERR_ARG (NULL, bad parent
 * order, bad dof index, bad kind, non-positive or non-finite dims, |kappa| >= 1,
 * lo > hi), HS_ERR_SIZE (counts out of range, a bone deeper than
 * HS_MAX_DEPTH). */
int hs_model_create(const HsModelDesc* desc, HsModel** out);
int hs_model_destroy(HsModel* model);
/* Select the kc variant of a model (see HsKcParams).  Errors: HS_ERR_ARG (NULL,
 * unknown variant, pen_weight negative or not finite), HS_ERR_SIZE (a variant
 * needs the proxies and the model has more than HS_MAX_PROXIES of them or more
 * than HS_MAX_PROXY_PAIRS pairs to test). */
int hs_model_set_kc(HsModel* model, const HsKcParams* kc);

/* Bytes of workspace render_score_batch needs for P particles (32 bytes per
 * particle: an exit count and fixed-point sums; then a 64-byte control block
 * holding the persistent launch's particle counter), rounded up to 256.  The
 * workspace must be zeroed once (hs_workspace_reset) before first use; every
 * call leaves it zeroed again.  Calls sharing one workspace must not overlap
 * on the GPU.
 * Errors: HS_ERR_ARG (bytes NULL), HS_ERR_SIZE (P out of range). */
int hs_workspace_size(int P, size_t* bytes);
int hs_workspace_reset(void* workspace, size_t bytes, hs_stream_t stream);

/* Per-frame preparation of an observation: counts the valid-depth skin pixels
 * and the skin pixels of the ROI into obs->stats.  Call once whenever the
 * observation changes, before render_score_batch.
 * Errors: HS_ERR_ARG, HS_ERR_ALIGN, HS_ERR_SIZE, HS_ERR_CUDA. */
int hs_obs_prepare(const HsObs* obs, hs_stream_t stream);

/* Forward kinematics (Eq. 1-3, Tables 1-2): clamp each pose to the model's
 * limits, build the bone frames and write P x n_prims camera-space records
 * (HsPrim) and kc[P] (the finger-crossing penalty after Eq. 5, rad).  A pose
 * with a NaN/inf entry gets kc = NaN and sets HS_DEV_NONFINITE_POSE.
 * poses [P][26], prims [P][n_prims], kc [P].  P = 0 is a no-op.
 * Errors: HS_ERR_ARG, HS_ERR_ALIGN (prims not 16-B aligned), HS_ERR_SIZE, HS_ERR_CUDA. */
int pose_fk(const HsModel* model, const float* poses, int P, const HsCamera* cam,
            HsPrim* prims, float* kc, hs_stream_t stream);

/* Render every hypothesis into the observation ROI by FP32 analytic ray casting
 * (depth map r_d, Section III.A) and reduce the per-pixel terms of Eq. 4 to
 * E[p] = D + lambda_k kc[p] (Eq. 5).  No rendered image is stored; parts [P]
 * (may be NULL) receives the sums.  dbg_depth [P][H][W] float (0 = no hit) and
 * dbg_mask [P][H][W] uint8 (bit 0 = hit, bit 1 = r_m) are optional test
 * outputs (NULL in production; when given they are cleared first).
 * workspace: hs_workspace_size(P) bytes, zeroed once before first use.
 * Errors: HS_ERR_ARG, HS_ERR_ALIGN, HS_ERR_SIZE, HS_ERR_CUDA. */
/* The render kernel (HS_RENDER_*, never AUTO) a call over P particles with these
 * parameters runs; HS_ERR_ARG for an invalid variant or P < 0. */
int hs_render_variant(const HsScoreParams* params, int P);

int render_score_batch(const HsModel* model, const HsObs* obs, const HsCamera* cam,
                       const HsPrim* prims, const float* kc, int P, const HsScoreParams* params,
                       void* workspace, size_t workspace_bytes, float* E, HsParts* parts,
                       float* dbg_depth, uint8_t* dbg_mask, hs_stream_t stream);

/* Tracking initialisation of a swarm (Section III.B: random positions, zero
 * velocity): particle 0 = clamped seed_pose, particle i > 0 = seed_pose +
 * (2u - 1) * scale[d] (u: Philox4x32-10 stream 3, counter (i, 3<<16 | d/4, 0,
 * frame), key = seed), clamped; pbest = x, pbest_E = gbest_E = +inf,
 * gbest = particle 0.  seed_pose: device [26]; scale: host [26].
 * Errors: HS_ERR_ARG, HS_ERR_SIZE, HS_ERR_CUDA. */
int pso_init(const HsModel* model, const HsSwarm* swarm, int P, const float* seed_pose,
             const float* scale, uint64_t seed, uint32_t frame, hs_stream_t stream);

/* One PSO generation after E = objective(x) (Section III.B, Eq. 6-7):
 * pbest where E < pbest_E; gbest = pbest[argmin pbest_E] (lowest index on
 * ties); v <- w (v + c1 r1 (pbest - x) + c2 r2 (gbest - x)), x <- clamp(x + v)
 * with r1/r2 = uniforms 2d / 2d+1 of Philox stream 1, counter (i, 1<<16 | k/4,
 * gen, frame); if mutate_every > 0 and gen % mutate_every == 0 the n_mutate
 * particles with the largest E (ties: higher index, NaN worst) re-draw dims
 * 6..25 uniformly in the limits (stream 2) with zero velocity there.
 * One CTA per swarm; P <= 4096.
 * Errors: HS_ERR_ARG, HS_ERR_SIZE, HS_ERR_CUDA. */
int pso_step(const HsModel* model, const HsSwarm* swarm, int P, const HsPsoParams* params,
             uint64_t seed, uint32_t frame, uint32_t gen, hs_stream_t stream);

/* render_score_batch for callers that cannot allocate device memory (a plugin
 * whose host owns every allocation, a real-time loop that must not allocate
 * after start-up, a layer without access to the application's allocator).
 * The paper has no counterpart: this is a deployment convenience.  Identical
 * to render_score_batch without the debug outputs, except that the scratch
 * workspace is a fixed array inside this library (HS_NOALLOC_SCRATCH_BYTES
 * bytes per GPU), so the call itself allocates nothing (no cudaMalloc, no
 * allocating library routine).
 *  - P is limited to what the array holds: calls with hs_workspace_size(P) >
 *    HS_NOALLOC_SCRATCH_BYTES (P > 8190 with the current 32-byte per-particle
 *    layout) return HS_ERR_SIZE and launch nothing.
 *  - The first call on a device looks up the array's device address (with
 *    cudaGetSymbolAddress) and caches it.  Under lazy module loading (the
 *    CUDA default) that first call is also when the driver loads the array
 *    onto the device, so it is the call that can fail for lack of device
 *    memory (HS_ERR_CUDA): make it at start-up, before any stream capture or
 *    allocation-free phase.  From then on the device holds the array until the
 *    process exits, and later calls allocate nothing.
 *  - Every call on a device shares the one array and clears the part it uses
 *    before launching, so calls that overlap on the GPU (different streams
 *    without ordering between them) race and give wrong results.
 * Errors: the arguments other than P are checked first, exactly as by
 * render_score_batch; then P (HS_ERR_SIZE when out of range or over the
 * array's limit). */
#define HS_NOALLOC_SCRATCH_BYTES (256 * 1024)
int render_score_batch_noalloc(const HsModel* model, const HsObs* obs, const HsCamera* cam,
                               const HsPrim* prims, const float* kc, int P, const HsScoreParams* params,
                               float* E, HsParts* parts, hs_stream_t stream);

/* One generation fused with the FK of the new positions: exactly pso_step
 * followed by pose_fk of the updated swarm, in one launch (one CTA per
 * particle), except that the new positions go to x_next [P][26] (a second
 * buffer; swarm->x is only read) so that no particle has to wait for another.
 * The caller alternates the two position buffers between generations.  prims
 * and kc receive the records of x_next for the next render_score_batch.
 * Tie rule of the fused step: when a particle's E equals its personal-best E
 * exactly and it is the global best, gbest takes its current position.
 * 1 <= P <= HS_FUSED_MAX_PARTICLES (every CTA scans the P objectives).
 * Errors: HS_ERR_ARG (NULL, x_next == swarm->x, bad constants), HS_ERR_ALIGN,
 * HS_ERR_SIZE, HS_ERR_CUDA. */
#define HS_FUSED_MAX_PARTICLES 4096  /* 2 x 4096 floats of shared memory per CTA */
int pso_step_fk(const HsModel* model, const HsSwarm* swarm, float* x_next, int P, const HsPsoParams* params,
                uint64_t seed, uint32_t frame, uint32_t gen, const HsCamera* cam, HsPrim* prims, float* kc,
                hs_stream_t stream);

/* ---- a whole tracking frame in one launch -------------------------------------------
 * Section III.B's per-frame loop -- initialise the swarm around the previous
 * frame's best pose, then `gens` generations of "score every particle (Section
 * III.A, Eq. 4-5), move the swarm (Eq. 6-7 and the mutation)" -- as one
 * cooperative launch whose `ctas` CTAs stay resident for the whole frame, with
 * one grid barrier per generation between scoring and the update.  The CTAs
 * are dealt evenly to the particles for the whole frame: particle p has CTAs
 * [ceil(p ctas / P), ceil((p + 1) ctas / P)).  The CTAs of a particle share
 * its 16x4-pixel work units and keep its state and FK records in their shared
 * memory.
 *
 * Results are exactly those of the step-by-step calls
 *     hs_obs_prepare(obs); pso_init(swarm, seed_pose, scale, seed, frame);
 *     pose_fk(x); for g = 1..gens: render_score_batch (any variant) on the
 *     records; pso_step_fk(gen = g) with swarm->x and x_next alternating
 * bit for bit, whatever `ctas`: E (swarm->E, written through the const
 * pointer: it must be a writable device array), pbest, pbest_E, gbest,
 * gbest_E, v, obs->stats, and the positions (generation g writes buffer g & 1
 * of {swarm->x, x_next}, so the final positions are in swarm->x when gens is
 * even, in x_next when odd).  prims (optional, may be NULL) and kc [P] receive
 * the records and kc of the final positions.
 *
 * ctas: CTAs of the grid, P <= ctas <= hs_frame_capacity(); 0 picks
 * min(capacity, 8 P).  workspace: hs_frame_workspace_size(P) bytes (a
 * control block and three generations of per-particle sums), zeroed once
 * before first use (every call leaves it zeroed).  Calls that share a
 * workspace must not overlap on the GPU.  If a grid barrier wait runs out
 * (about a second), the frame stops, HS_DEV_BARRIER_TIMEOUT is set and the
 * swarm's contents are void; the next call runs normally.  The workspace's
 * third 32-bit word is read as a number of arrivals every grid barrier waits
 * for beyond the grid's own: leave it zero (a test sets it to make the wait
 * run out).
 * Errors: HS_ERR_ARG (NULL, x_next == swarm->x, bad constants, gens < 0,
 * ctas < 0), HS_ERR_ALIGN, HS_ERR_SIZE (P out of range, ctas < P or over
 * capacity, workspace too small), HS_ERR_CUDA. */
#define HS_FRAME_MAX_PARTICLES 1024
int hs_frame_workspace_size(int P, size_t* bytes);
/* CTAs of track_frame that the current device keeps resident at once */
int hs_frame_capacity(int* ctas);
int track_frame(const HsModel* model, const HsObs* obs, const HsCamera* cam, const HsSwarm* swarm, float* x_next,
                int P, int gens, const HsScoreParams* score, const HsPsoParams* pso, const float* seed_pose,
                const float* scale, uint64_t seed, uint32_t frame, int ctas, void* workspace,
                size_t workspace_bytes, HsPrim* prims, float* kc, hs_stream_t stream);

/* ---- batches: many independent swarms per launch ----------------------------------
 * A batch binds S swarms (sequences), each with its own observation buffers,
 * camera, particle count, mutation count and Philox key, so that one launch
 * scores or updates every particle of every swarm (the paper's parallelism
 * "between particles" extended across sequences, Section IV).  Particle arrays
 * are concatenated over the swarms ([P_total][...], swarm s first at its
 * offset); per-swarm arrays are gbest [S][26], gbest_E [S], seed poses [S][26].
 * Random numbers use each particle's index within its swarm and the swarm's
 * key, so a batch reproduces S separate single-swarm runs exactly. */
#define HS_MAX_SWARMS 4096
typedef struct {
    HsObs obs;          /* this swarm's observation (buffers stay bound to the batch) */
    HsCamera cam;
    int32_t P;          /* particles, 1..HS_FUSED_MAX_PARTICLES */
    int32_t n_mutate;   /* particles mutated every mutate_every generations (paper: P / 2) */
    uint64_t seed;      /* Philox key of this swarm */
} HsSwarmDesc;

/* opaque host object describing a batch; its device part lives in the caller's buffer */
typedef struct HsBatch HsBatch;

/* Bytes of the device buffer a batch needs (views with TMA descriptors, the
 * particle-to-swarm table).  Errors: HS_ERR_ARG, HS_ERR_SIZE. */
int hs_batch_buffer_size(const HsSwarmDesc* swarms, int S, size_t* bytes);
/* Validate the swarms, encode their TMA descriptors and write the batch into
 * `buffer` (device, 256-byte aligned, hs_batch_buffer_size bytes; synchronous
 * on `stream`).  Allocates host memory for the handle only.  The observation
 * buffers must stay valid while the batch is used; new frames are copied into
 * them.  Errors: HS_ERR_ARG, HS_ERR_ALIGN, HS_ERR_SIZE, HS_ERR_CUDA. */
int hs_batch_create(const HsModel* model, const HsSwarmDesc* swarms, int S, void* buffer, size_t bytes,
                    hs_stream_t stream, HsBatch** out);
int hs_batch_destroy(HsBatch* batch);
int hs_batch_particles(const HsBatch* batch, int* P_total);
/* hs_obs_prepare for every swarm of the batch (two launches). */
int hs_obs_prepare_multi(const HsBatch* batch, hs_stream_t stream);
/* pose_fk over all P_total particles, each with its swarm's camera. */
int pose_fk_multi(const HsModel* model, const HsBatch* batch, const float* poses, HsPrim* prims, float* kc,
                  hs_stream_t stream);
/* render_score_batch over all particles of all swarms in one launch (each
 * particle against its swarm's observation); workspace: hs_workspace_size(P_total). */
int render_score_multi(const HsModel* model, const HsBatch* batch, const HsPrim* prims, const float* kc,
                       const HsScoreParams* params, void* workspace, size_t workspace_bytes, float* E,
                       HsParts* parts, hs_stream_t stream);
/* pso_init for every swarm: seed_poses device [S][26], scale host [26]. */
int pso_init_multi(const HsModel* model, const HsBatch* batch, const HsSwarm* swarm, const float* seed_poses,
                   const float* scale, uint32_t frame, hs_stream_t stream);
/* pso_step_fk for every swarm in one launch (n_mutate from each swarm's
 * descriptor; c1, c2 and mutate_every from params).  Device-side stop flags
 * (params->e_stop > 0): a swarm whose global best E, after this generation's
 * personal- and global-best update, is below e_stop stops -- this
 * generation's positions are kept (x_next = x, velocity unchanged, no FK),
 * and in the later generations of the frame render_score_multi does not
 * score its particles and pso_step_fk_multi only carries its positions over.
 * pso_init_multi starts every swarm running again. */
int pso_step_fk_multi(const HsModel* model, const HsBatch* batch, const HsSwarm* swarm, float* x_next,
                      const HsPsoParams* params, uint32_t frame, uint32_t gen, HsPrim* prims, float* kc,
                      hs_stream_t stream);

/* A whole frame of every swarm of the batch (Section III.B's per-frame loop,
 * Section IV's parallelism between particles, across sequences) as one
 * cooperative launch, after the observation totals (hs_obs_prepare_multi's
 * two launches, issued here first).  The resident CTAs take tasks from a
 * counter, generation by generation, each generation's particles largest ROI
 * first: a task is one particle's initialisation (generation 1) or step of the
 * previous generation, then its FK, render and E.  A particle's step waits
 * only until every particle of its own swarm has been scored at the previous
 * generation (a per-swarm count, awaited with a time limit), so the swarms
 * run generations apart and no CTA waits at a grid barrier.
 *
 * Results are exactly those of the step-by-step batch calls
 *     hs_obs_prepare_multi; pso_init_multi(seed_poses, scale, frame);
 *     pose_fk_multi(x); for g = 1..gens: render_score_multi (any variant);
 *     pso_step_fk_multi(gen = g) with swarm->x and x_next alternating
 * bit for bit, whatever `ctas`: E (written through the const pointer: it must
 * be a writable device array), pbest, pbest_E, gbest, gbest_E, v, the
 * positions (step g writes buffer g & 1 of {swarm->x, x_next}), and prims /
 * kc [P_total] (the records and kc of the final positions).  seed_poses:
 * device [S][26]; scale: host [26].
 *
 * ctas: CTAs of the grid, 1..hs_frame_multi_capacity(model, batch); 0 picks the capacity.
 * workspace: hs_frame_multi_workspace_size(batch) bytes (a 128-byte control
 * block, a count per swarm from byte 128 on, then two generations of E), zeroed
 * once before first use (every call leaves the control block and the counts
 * zeroed; the E part needs no initial value).  Calls that share a workspace must not
 * overlap on the GPU.  If a wait runs out (about a second) or an observation
 * load does not arrive, every CTA stops taking tasks, HS_DEV_BARRIER_TIMEOUT
 * (or HS_DEV_TMA_TIMEOUT) is set and the swarms' contents are void; the next
 * call runs normally.  The workspace's fourth 32-bit word is read as a number
 * of renders every wait expects beyond its swarm's own: leave it zero (a test
 * sets it to make the wait run out).  The stopping rule (params->e_stop) is
 * the step-by-step calls' only: e_stop must be 0 here.
 * Errors: HS_ERR_ARG (NULL, x_next == swarm->x, bad constants, e_stop != 0,
 * gens < 0, ctas < 0), HS_ERR_ALIGN, HS_ERR_SIZE (a swarm over
 * HS_FRAME_MAX_PARTICLES particles, (gens + 1) x P_total over 2^31 - 1 tasks,
 * ctas over capacity, workspace too small), HS_ERR_CUDA. */
int hs_frame_multi_workspace_size(const HsBatch* batch, size_t* bytes);
/* CTAs of track_frame_multi that the current device keeps resident at once for this model and batch (its
 * shared memory holds two values per particle of the batch's largest swarm, the records of the model's
 * primitives, and, for a model whose kc variant uses the interpenetration test, the model's collision data,
 * which leaves room for fewer CTAs); model NULL: for any model with the paper's kc (HS_MAX_PRIMS primitives);
 * batch NULL: for any batch (swarms of up to HS_FRAME_MAX_PARTICLES particles).
 * Errors: HS_ERR_ARG, HS_ERR_SIZE (a swarm over HS_FRAME_MAX_PARTICLES), HS_ERR_CUDA. */
int hs_frame_multi_capacity(const HsModel* model, const HsBatch* batch, int* ctas);
int track_frame_multi(const HsModel* model, const HsBatch* batch, const HsSwarm* swarm, float* x_next, int gens,
                      const HsScoreParams* score, const HsPsoParams* pso, const float* seed_poses,
                      const float* scale, uint32_t frame, int ctas, void* workspace, size_t workspace_bytes,
                      HsPrim* prims, float* kc, hs_stream_t stream);

/* ---- the smoothed objective E_s and its gradient (gradient polish) ---------------
 * E (Eq. 4-5) is piecewise constant in the pose at every silhouette and depth
 * threshold, so its gradient carries no silhouette information.  E_s keeps
 * E's terms (reading R1) and replaces each hard decision by a smooth one:
 *  - primitive coverage sigma(delta / tau_px), delta = Delta / |grad Delta| the
 *    first-order signed pixel distance to the primitive's silhouette from the
 *    ray-quadric discriminant; cones also fade at their end cut |Y| <= 1 over
 *    tau_px along the projected axis; the root uses a soft positive part of
 *    Delta (width tau_px in pixels);
 *  - the primitives touching a pixel are composited front to back in depth
 *    order (coverage c = 1 - prod(1 - alpha), depth z~ = sum T alpha z / c);
 *  - |O_d - z~| -> sqrt((O_d - z~)^2 + tau_mm^2), the d_M clamp -> a soft
 *    minimum, the d_m test -> a sigmoid, all of width tau_mm;
 *  - per pixel t = c t_hit + (1 - c) t_miss, r_m = c m; D_s and E_s as Eq. 4-5.
 * As tau_px, tau_mm -> 0, E_s -> E.  The paper optimises E with PSO alone; E_s
 * and its gradient serve the gradient polish of the best particles.  FP32. */
#define HS_SOFT_ADJ 13  /* per-primitive adjoint: M (9, record order), C (3), cone length in pixels (1) */
typedef struct {
    float tau_px;        /* silhouette softness, pixels (0.5) */
    float tau_mm;        /* depth softness, mm (0.5) */
    int32_t ctas_per_particle;  /* 0 = automatic */
    int32_t reserved;
} HsSoftParams;

/* E_s of P particles whose records came from pose_fk (FP32).  sums [P][3]
 * (may be NULL) receives (sum t, sum and, sum or), which the backward pass
 * needs.  workspace: hs_workspace_size(P) bytes, zeroed once (left zeroed).
 * obs->stats must be prepared (hs_obs_prepare).
 * Errors: HS_ERR_ARG, HS_ERR_ALIGN, HS_ERR_SIZE, HS_ERR_CUDA. */
int soft_score(const HsModel* model, const HsObs* obs, const HsCamera* cam, const HsPrim* prims, const float* kc,
               int P, const HsScoreParams* params, const HsSoftParams* soft, void* workspace,
               size_t workspace_bytes, float* E_s, float* sums, hs_stream_t stream);
/* dE_s / d(records): adds, for every particle and primitive, the adjoint of its
 * record (M in record order, C) and of the cone's pixel length to adj
 * [P][n_prims][HS_SOFT_ADJ] (device, 64-bit fixed point with 2^-40
 * resolution so that sums do not depend on scheduling; zero on entry,
 * pose_grad clears it).  sums: soft_score's output for the same inputs. */
int soft_score_backward(const HsModel* model, const HsObs* obs, const HsCamera* cam, const HsPrim* prims, int P,
                        const HsScoreParams* params, const HsSoftParams* soft, const float* sums, int64_t* adj,
                        hs_stream_t stream);
/* dE_s / d pose [P][26] from the record adjoints (the FK's tangents, Eq. 1-3:
 * each joint angle turns the bones below it about its world axis) plus
 * lambda_k dkc/dpose (and, with a kc variant, the interpenetration term's
 * derivative); zero for a parameter outside its
 * limits (the FK clamps it).  Rewrites prims/kc with pose_fk's values and
 * clears adj. */
int pose_grad(const HsModel* model, const float* poses, int P, const HsCamera* cam, const HsScoreParams* params,
              HsPrim* prims, float* kc, int64_t* adj, float* grad, hs_stream_t stream);

/* ---- gradient polish of the best particles (hybrid PSO) --------------------------
 * Not in the paper, which relies on PSO alone; the paper names fingers stuck in
 * local optima as its failure mode (Section III.B, V).  After a generation's E
 * is known: polish_select picks the k best particles (lowest E, lower index on
 * ties, NaN last), polish_gather copies their poses and E, polish_step moves
 * them down the gradient of E_s, and polish_keep_better writes a polished pose
 * (and its exact E) back only where it lowered E.  All device arrays. */
#define HS_POLISH_MAX 256
int polish_select(const float* E, int P, int k, int32_t* sel, hs_stream_t stream);
int polish_gather(const float* x, const float* E, const int32_t* sel, int k, float* x_sel, float* E_sel,
                  hs_stream_t stream);
/* x_sel [k][26] <- clamp(x_sel - eta S^2 g / |S g|) with S = scale (host [26],
 * > 0; e.g. 10 mm / 10 degrees) and the model's limits: a step of length eta
 * in scaled units along the preconditioned gradient grad [k][26]. */
int polish_step(const HsModel* model, float* x_sel, const float* grad, int k, float eta, const float* scale,
                hs_stream_t stream);
int polish_keep_better(float* x, float* E, const int32_t* sel, int k, const float* x_sel, const float* E_old,
                       const float* E_new, hs_stream_t stream);

/* ---- render autotuning -----------------------------------------------------------
 * Time every render kernel (HS_RENDER_UNITS .. HS_RENDER_VARIANTS - 1) with CTAs
 * per particle from {automatic, 1, 2, 3, 4, 6, 8, 16, 32} (more than 1 only while
 * K * P stays within about four resident waves; the persistent kernels take
 * none) on the caller's own inputs, and
 * write the fastest into params->variant and params->ctas_per_particle (the
 * Eq. 4-5 constants are kept).  The choice never changes results, only time.
 * Each candidate's `reps` calls are captured into a CUDA graph on a private
 * stream (after `stream` is synchronised), launched once untimed and once
 * between two CUDA events; the call synchronises and must not itself be
 * captured.
 * times_us (may be NULL) receives [HS_RENDER_VARIANTS][HS_TUNE_CTAS] average
 * microseconds per call, -1 where not tried.  E receives the last call's
 * objectives.  Errors: as render_score_batch / render_score_multi, and
 * HS_ERR_ARG for reps outside 1..1000.  The paper has no counterpart: its
 * render is a fixed OpenGL pipeline. */
#define HS_TUNE_CTAS 9
int render_score_batch_autotune(const HsModel* model, const HsObs* obs, const HsCamera* cam, const HsPrim* prims,
                                const float* kc, int P, HsScoreParams* params, void* workspace,
                                size_t workspace_bytes, float* E, int reps, float* times_us, hs_stream_t stream);
int render_score_multi_autotune(const HsModel* model, const HsBatch* batch, const HsPrim* prims, const float* kc,
                                HsScoreParams* params, void* workspace, size_t workspace_bytes, float* E, int reps,
                                float* times_us, hs_stream_t stream);

/* Read (and optionally clear) the device status word of the current device.
 * Synchronises the device.  out: host.  Errors: HS_ERR_ARG, HS_ERR_CUDA. */
int hs_get_device_status(uint32_t* out, int clear);

#ifdef __cplusplus
}
#endif
#endif /* HANDSCORE_H */
