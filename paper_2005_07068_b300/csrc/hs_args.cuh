// hs_args.cuh -- launch-argument structs and launcher prototypes shared by
// the C-ABI layer (api.cu) and the kernel translation units.
#pragma once

#include <cuda.h>

#include "hs_device.cuh"

namespace hs {

struct FkArgs {
    const float* poses;  // [P][26]
    int P;
    float fx, fy, cx, cy;
    float4* prims;       // [P][n_prims][4]
    float* kc;           // [P]
    uint32_t* status;
};

// per-particle scratch of render_score_batch (32 bytes, zero between calls)
struct HsParticleWork {
    uint32_t next;                // unit queue ticket
    uint32_t exited;              // warps that have left the queue
    unsigned long long t_fix;     // sum of depth-term differences, fixed point 2^-24 mm
    uint32_t n_and, n_or, n_hit;  // sum(S and r_m), sum(r_m and not S), rendered pixels
    uint32_t pad;
};

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
};

struct PsoInitArgs {
    float *x, *v, *pbest, *pbest_E, *gbest, *gbest_E;
    const float* seed_pose;
    float scale[kNdof];
    int P;
    uint32_t key0, key1, frame;
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
    float4 cam;            // fx, fy, cx, cy
    float4* prims;         // [P][n_prims][4]
    float* kc;             // [P]
    uint32_t* status;
};

cudaError_t launch_fk(const DevModel& model, const FkArgs& args, cudaStream_t stream);
cudaError_t launch_pso_step_fk(const DevModel& model, const PsoFkArgs& args, cudaStream_t stream);
cudaError_t launch_render_score(const CUtensorMap& tm_depth, const CUtensorMap& tm_skin, const RenderArgs& args,
                                cudaStream_t stream);
cudaError_t launch_obs_stats(const unsigned char* depth, int depth_pitch, int depth_f32, const uint8_t* skin,
                             int skin_pitch, int W, int H, uint32_t* stats, cudaStream_t stream);
cudaError_t launch_pso_init(const Limits& lim, const PsoInitArgs& args, cudaStream_t stream);
cudaError_t launch_pso_step(const Limits& lim, const PsoStepArgs& args, cudaStream_t stream);

}  // namespace hs
