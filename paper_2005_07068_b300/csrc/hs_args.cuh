// hs_args.cuh -- launch-argument structs and launcher prototypes shared by
// the C-ABI layer (api.cu) and the kernel translation units.
#pragma once

#include <cuda.h>

#include "hs_device.cuh"

namespace hs {

// One swarm of a batch (device memory, written by hs_batch_create): its
// observation (TMA tensor maps + raw pointers), camera, particle range,
// mutation count and Philox key.  Particles of swarm s are [offset, offset+P).
struct SwarmView {  // 128-byte aligned (CUtensorMap)
    CUtensorMap tm_depth;  // 2-D map of the depth image, 16 x 4 boxes
    CUtensorMap tm_skin;   // 2-D map of the skin mask, 16 x 4 boxes
    int32_t W, H, depth_f32, P;
    int32_t offset, n_mutate, depth_pitch, skin_pitch;
    float inv_fx, inv_fy, off_x, off_y;  // render rays: (u inv_fx + off_x, v inv_fy + off_y, 1)
    float fx, fy, cx, cy;                // FK projection
    const unsigned char* depth;
    const uint8_t* skin;
    uint32_t* stats;
    uint32_t key0, key1;
    uint32_t stop_gen;  // device state: 0 while the swarm runs, else the generation at which it stopped
                        // (e_stop); cleared by the batch init, set by the batch step
    uint32_t pad;
};

// header of a batch buffer: S views, then the swarm index of every particle
struct BatchDev {
    int32_t S, P_total;
    const SwarmView* views;  // [S]
    const int32_t* sid;      // [P_total]
};

// swarm s's stop word (SwarmView::stop_gen), read and written through
// volatile accesses: kernels of the same stream write it, so it must not be
// served from a read-only cache
__device__ __forceinline__ uint32_t swarm_stop_gen(const BatchDev& b, int s)
{
    return *reinterpret_cast<const volatile uint32_t*>(&b.views[s].stop_gen);
}
__device__ __forceinline__ void set_swarm_stop_gen(const BatchDev& b, int s, uint32_t gen)
{
    *reinterpret_cast<volatile uint32_t*>(const_cast<uint32_t*>(&b.views[s].stop_gen)) = gen;
}


struct FkArgs {
    const float* poses;  // [P][26]
    int P;
    float fx, fy, cx, cy;
    float4* prims;       // [P][n_prims][4]
    float* kc;           // [P]
    uint32_t* status;
    BatchDev batch;      // when set: the camera of particle p's swarm
};

// per-particle scratch of render_score_batch (32 bytes, zero between calls)
struct HsParticleWork {
    uint32_t next;                // unit queue ticket
    uint32_t exited;              // warps that have left the queue
    unsigned long long t_fix;     // sum of depth-term differences, fixed point 2^-24 mm
    uint32_t n_and, n_or, n_hit;  // sum(S and r_m), sum(r_m and not S), rendered pixels
    uint32_t tx_test;             // zero, except to test the observation wait's time limit: the particle's
                                  // first warp then arms its first load for this many bytes more than are
                                  // copied, so that wait runs out (no copy is left in flight); the kernels
                                  // only read it, and the last contributor clears the slot as usual
};

// control block of the persistent render launch, at the end of the render
// workspace (64 bytes, zero between calls)
struct RenderCtl {
    uint32_t next;    // the next particle (index into the call's order) to be taken
    uint32_t exited;  // CTAs that have left
    uint32_t pad[14];
};
static_assert(sizeof(RenderCtl) == 64, "64-byte control block");

struct RenderArgs {
    const float4* prims;  // [P][n_prims][4]
    const float* kc;      // [P]
    int P, n_prims, K;
    int W, H;
    float inv_fx, inv_fy, off_x, off_y;  // ray of pixel (u, v): (u inv_fx + off_x, v inv_fy + off_y, 1)
    float d_m, d_M, lambda, lambda_k;
    int depth_f32;
    const uint32_t* stats;  // [2]: #valid, #skin
    HsParticleWork* work;   // [P]
    float* E;
    HsParts* parts;
    float* dbg_depth;
    uint8_t* dbg_mask;
    uint32_t* status;
    BatchDev batch;  // batch.views == nullptr: one swarm described by the fields above
    const int32_t* order;  // CTA row y scores particle order[y] (nullptr: particle y)
    RenderCtl* ctl;        // the persistent launch's counters (after work[P] in the workspace)
};

struct PsoInitArgs {
    float *x, *v, *pbest, *pbest_E, *gbest, *gbest_E;
    const float* seed_pose;  // [26], or [S][26] for a batch
    float scale[kNdof];
    int P;
    uint32_t key0, key1, frame;
    BatchDev batch;  // when set: per-swarm seed pose, key and gbest slot
};

struct PsoStepArgs {
    float *x, *v, *pbest, *pbest_E, *gbest, *gbest_E;
    const float* E;
    int P;
    float c1, c2, w;
    int mutate, n_mutate;
    uint32_t key0, key1, frame, gen;
};

// the fused generation step: PSO update of every particle, then FK of its new pose
struct PsoFkArgs {
    const float* x;        // [P][26] current positions (read only)
    float* x_next;         // [P][26] new positions
    float *v, *pbest, *pbest_E, *gbest, *gbest_E;
    const float* E;
    int P;
    float c1, c2, w;
    int mutate, n_mutate;
    uint32_t key0, key1, frame, gen;
    float e_stop;          // batch only: a swarm stops once its global best E is below this (0: never)
    float4 cam;            // fx, fy, cx, cy
    float4* prims;         // [P][n_prims][4]
    float* kc;             // [P]
    uint32_t* status;
    BatchDev batch;        // when set: every particle works within its own swarm
};

// ---- one whole tracking frame in one cooperative launch (frame.cu) ----
// per-particle sums of one generation (32 bytes): the render's integer sums
// and the kc of the scored pose
struct FrameSums {
    unsigned long long t_fix;     // sum of depth-term differences, fixed point 2^-24 mm
    uint32_t n_and, n_or, n_hit;  // sum(S and r_m), sum(r_m and not S), rendered pixels
    float kc;
    uint32_t pad[2];
};
// control block at the start of the frame workspace (128 bytes)
struct FrameCtl {
    uint32_t barrier;  // grid-barrier arrivals of this launch
    uint32_t exited;   // CTAs that have finished
    uint32_t missing;  // arrivals every grid barrier waits for beyond the grid's own: zero, except to test the
                       // barrier's time limit (the wait then runs out); the kernel only reads it
    uint32_t pad[29];
};

struct FrameArgs {
    int W, H, depth_f32;
    float inv_fx, inv_fy, off_x, off_y;  // render rays
    float4 cam;                          // FK projection: fx, fy, cx, cy
    const unsigned char* depth;
    const uint8_t* skin;
    int depth_pitch, skin_pitch;
    uint32_t* stats;                     // obs stats [2], zero at launch
    float d_m, d_M, lambda, lambda_k;
    float* xbuf[2];                      // positions: generation g scores xbuf[(g - 1) & 1], writes xbuf[g & 1]
    float *v, *pbest, *pbest_E, *gbest, *gbest_E, *E;
    float4* prims_out;                   // [P][n_prims][4] records of the final positions, or nullptr
    float* kc;                           // [P] kc of the final positions
    const float* seed_pose;              // [26]
    float scale[kNdof];                  // initial spread per dimension
    float c1, c2, w;
    int mutate_every, n_mutate;
    uint32_t key0, key1, frame;
    int P, gens;
    FrameCtl* ctl;
    FrameSums* sums;                     // [3][P]
    uint32_t* status;
};

// ---- every swarm of a batch, a whole frame in one cooperative launch (frame.cu) ----
// control block at the start of the batch-frame workspace (128 bytes, zero between calls)
struct FrameMultiCtl {
    uint32_t next;     // the next task to be taken
    uint32_t exited;   // CTAs that have finished
    uint32_t abort;    // set when a wait ran out: no CTA takes another task
    uint32_t missing;  // renders every wait expects beyond its swarm's own: zero, except to test the wait's time
                       // limit (the wait then runs out); the kernel only reads it
    uint32_t pad[28];
};
static_assert(sizeof(FrameMultiCtl) == 128, "128-byte control block");

struct FrameMultiArgs {
    BatchDev batch;
    const int32_t* order;                // [P_total] the particles of a generation in task order
    float d_m, d_M, lambda, lambda_k;
    float* xbuf[2];                      // positions: step g reads xbuf[(g - 1) & 1], writes xbuf[g & 1]
    float *v, *pbest, *pbest_E, *gbest, *gbest_E, *E;
    float* Ebuf;                         // [2][P_total]: E of generation g at Ebuf[(g & 1) P_total + q]
    uint32_t* done;                      // [S] renders finished per swarm in this launch
    float4* prims_out;                   // [P_total][n_prims][4] records of the final positions
    float* kc;                           // [P_total] kc of the final positions
    const float* seed_poses;             // [S][26]
    float scale[kNdof];                  // initial spread per dimension
    float c1, c2, w;
    int mutate_every;
    uint32_t frame;
    int gens, P_max;
    FrameMultiCtl* ctl;
    uint32_t* status;
};

// ---- the smoothed objective and its gradient (soft.cu) ----
constexpr int kAdj = HS_SOFT_ADJ;  // per-primitive adjoint: record M (9), C (3), cone length L (1)

struct SoftWork {
    uint32_t exited, pad;
    long long t, a, o;  // fixed-point 2^-24: sum of t - t_miss, sum S r_m, sum (1 - S) r_m
};
static_assert(sizeof(SoftWork) == 32, "one 32-byte workspace slot per particle");

struct SoftArgs {
    const float4* prims;  // [P][n_prims][4]
    const float* kc;      // [P]
    int P, n_prims, K;
    int W, H;
    float inv_fx, inv_fy, off_x, off_y, fx, fy;
    float d_m, d_M, lambda, lambda_k, tau, tau_mm;
    const unsigned char* depth;
    const uint8_t* skin;
    int depth_pitch, skin_pitch, depth_f32;
    const uint32_t* stats;  // [2]: #valid, #skin
    SoftWork* work;         // forward: [P], zero between calls
    float* E;               // forward: [P]
    float* sums;            // forward output / backward input: [P][3] (sum t, sum and, sum or)
    long long* adj;         // backward: [P][n_prims][kAdj], fixed point 2^-40, accumulated
};

struct GradArgs {
    const float* poses;  // [P][26]
    int P;
    float fx, fy, cx, cy;
    float lambda_k;
    float4* prims;   // [P][n_prims][4] (rewritten by the FK, same values as pose_fk)
    float* kc;       // [P]
    long long* adj;  // [P][n_prims][kAdj], fixed point 2^-40, read then cleared
    float* grad;     // [P][26]
    uint32_t* status;
};

// one polish step: eta in scaled units, per-parameter scale and limits
struct PolishStep {
    float eta;
    float scale[kNdof];
    float lo[kNdof], hi[kNdof];
};
cudaError_t launch_select_best(const float* E, int P, int k, int32_t* sel, cudaStream_t s);
cudaError_t launch_gather(const float* x, const float* E, const int32_t* sel, int k, float* x_sel, float* E_sel,
                          cudaStream_t s);
cudaError_t launch_polish_step(float* x, const float* grad, int k, const PolishStep& st, cudaStream_t s);
cudaError_t launch_keep_better(float* x, float* E, const int32_t* sel, int k, const float* x_sel, const float* E_old,
                               const float* E_new, cudaStream_t s);

cudaError_t launch_soft(bool backward, const SoftArgs& args, cudaStream_t stream);
cudaError_t launch_pose_grad(const DevModel& model, const GradArgs& args, cudaStream_t stream);

cudaError_t launch_fk(const DevModel& model, const FkArgs& args, cudaStream_t stream);
cudaError_t launch_pso_step_fk(const DevModel& model, const PsoFkArgs& args, cudaStream_t stream);
cudaError_t launch_track_frame(const DevModel& model, const CUtensorMap& tm_depth, const CUtensorMap& tm_skin,
                               const FrameArgs& args, int ctas, cudaStream_t stream);
cudaError_t track_frame_capacity(int* ctas);  // co-resident CTAs of track_frame_kernel on the current device
cudaError_t launch_track_frame_multi(const DevModel& model, const FrameMultiArgs& args, int ctas, cudaStream_t stream);
// co-resident CTAs of track_frame_multi_kernel with shared memory for swarms of up to P_max particles and a model
// of n_prims primitives; collide: the kernel of a kc variant, which keeps the model's collision data in shared
// memory (fewer CTAs)
cudaError_t track_frame_multi_capacity(int* ctas, int P_max, int n_prims, bool collide);
// whether a model's kc variant needs its collision data in the kernels
inline bool frame_multi_needs_collide(const DevModelCore& m) { return m.kc_variant != HS_KC_ABDUCTION; }
cudaError_t launch_render_score(const CUtensorMap& tm_depth, const CUtensorMap& tm_skin, const RenderArgs& args,
                                cudaStream_t stream);
cudaError_t launch_render_tiles(int variant, const CUtensorMap& tm_depth, const CUtensorMap& tm_skin,
                                const RenderArgs& args, cudaStream_t stream);
cudaError_t launch_render_strips(int variant, const CUtensorMap& tm_depth, const CUtensorMap& tm_skin,
                                 const RenderArgs& args, cudaStream_t stream);
cudaError_t launch_obs_stats(const unsigned char* depth, int depth_pitch, int depth_f32, const uint8_t* skin,
                             int skin_pitch, int W, int H, uint32_t* stats, cudaStream_t stream);
cudaError_t launch_obs_stats_multi(const BatchDev& batch, int max_H, cudaStream_t stream);
cudaError_t launch_pso_init(const Limits& lim, const PsoInitArgs& args, cudaStream_t stream);
cudaError_t launch_pso_step(const Limits& lim, const PsoStepArgs& args, cudaStream_t stream);

}  // namespace hs
