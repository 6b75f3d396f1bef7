// pso.cu -- swarm initialisation and one PSO generation on the device
// (Section III.B, Eq. 6-7 and the mutation of the worst half).
//
// The paper runs the swarm on the CPU and reads D back every generation
// (Section IV, step 3).  Here the whole generation stays on the GPU: one CTA
// per swarm updates the personal bests, takes the argmin for the global best,
// applies Eq. 6-7 with per-dimension r1/r2 from a counter-based Philox4x32-10
// stream, clamps to the limits and, every `mutate_every` generations,
// re-draws the finger dims of the worst particles.
#include <algorithm>
#include <cfloat>
#include <climits>

#include "hs_step.cuh"

namespace hs {

constexpr int kPsoThreads = 512;

__global__ void __launch_bounds__(256) pso_init_kernel(const __grid_constant__ Limits lim, const PsoInitArgs a)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = g / kInitBlocks, j = g % kInitBlocks;
    if (i >= a.P) return;
    // a batch: particle i is number li of swarm s, with that swarm's key, seed pose and gbest slot
    int li = i, s = 0;
    uint32_t k0 = a.key0, k1 = a.key1;
    if (a.batch.views) {
        s = a.batch.sid[i];
        const SwarmView& v = a.batch.views[s];
        li = i - v.offset;
        k0 = v.key0;
        k1 = v.key1;
    }
    const float* seed_pose = a.seed_pose + (size_t)s * kNdof;
    if (a.batch.views && li == 0 && j == 0) set_swarm_stop_gen(a.batch, s, 0u);  // the swarm runs this frame
    const U4 r = philox4x32_10(U4{(uint32_t)li, (kStreamInit << 16) | (uint32_t)j, 0u, a.frame}, k0, k1);
    const uint32_t u[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        const int d = 4 * j + l;
        if (d >= kNdof) break;
        const float sp = seed_pose[d];
        float xv = li == 0 ? sp : fmaf(fmaf(2.f, u01(u[l]), -1.f), a.scale[d], sp);
        xv = fminf(fmaxf(xv, lim.lo[d]), lim.hi[d]);
        const size_t o = (size_t)i * kNdof + d;
        a.x[o] = xv;
        a.v[o] = 0.f;
        a.pbest[o] = xv;
        if (li == 0) a.gbest[(size_t)s * kNdof + d] = xv;
    }
    if (j == 0) {
        a.pbest_E[i] = INFINITY;
        if (li == 0) a.gbest_E[s] = INFINITY;
    }
}

__global__ void __launch_bounds__(kPsoThreads) pso_step_kernel(const __grid_constant__ Limits lim, const PsoStepArgs a)
{
    extern __shared__ float sE[];  // [P]
    __shared__ float s_gbest[kNdof];
    __shared__ float red_v[kPsoThreads / 32];
    __shared__ int red_i[kPsoThreads / 32];
    __shared__ int s_g;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int P = a.P;

    // 1. personal bests (strict improvement; NaN never improves)
    float bv = INFINITY;
    int bi = INT_MAX;
    for (int i = tid; i < P; i += kPsoThreads) {
        const float e = a.E[i];
        sE[i] = e;
        float pe = a.pbest_E[i];
        if (e < pe) {
            pe = e;
            a.pbest_E[i] = e;
            for (int d = 0; d < kNdof; ++d) a.pbest[(size_t)i * kNdof + d] = a.x[(size_t)i * kNdof + d];
        }
        if (bi == INT_MAX || pe < bv) {  // indices rise, so ties keep the lowest
            bv = pe;
            bi = i;
        }
    }
    // 2. global best = argmin pbest_E, lowest index on ties
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi != INT_MAX && (bi == INT_MAX || ov < bv || (ov == bv && oi < bi))) {
            bv = ov;
            bi = oi;
        }
    }
    if (lane == 0) {
        red_v[warp] = bv;
        red_i[warp] = bi;
    }
    __syncthreads();
    if (tid == 0) {
        float v = red_v[0];
        int g = red_i[0];
        for (int w = 1; w < kPsoThreads / 32; ++w) {
            const int oi = red_i[w];
            if (oi != INT_MAX && (g == INT_MAX || red_v[w] < v || (red_v[w] == v && oi < g))) {
                v = red_v[w];
                g = oi;
            }
        }
        s_g = g;
        a.gbest_E[0] = v;
    }
    __syncthreads();
    if (tid < kNdof) {
        const float gv = a.pbest[(size_t)s_g * kNdof + tid];
        s_gbest[tid] = gv;
        a.gbest[tid] = gv;
    }
    __syncthreads();

    // 3. Eq. 6-7 with per-dimension r1, r2, then clamp
    for (int q = tid; q < P * kPairBlocks; q += kPsoThreads) {
        const int i = q / kPairBlocks, j = q % kPairBlocks;
        const U4 r = philox4x32_10(U4{(uint32_t)i, (kStreamPso << 16) | (uint32_t)j, a.gen, a.frame}, a.key0, a.key1);
        const uint32_t u[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int d = 2 * j + h;
            if (d >= kNdof) break;
            const float r1 = u01(u[2 * h]), r2 = u01(u[2 * h + 1]);
            const size_t o = (size_t)i * kNdof + d;
            const float x = a.x[o];
            float acc = fmaf(a.c1 * r1, a.pbest[o] - x, a.v[o]);
            acc = fmaf(a.c2 * r2, s_gbest[d] - x, acc);
            const float vn = a.w * acc;
            a.v[o] = vn;
            a.x[o] = fminf(fmaxf(x + vn, lim.lo[d]), lim.hi[d]);
        }
    }

    // 4. mutation of the n_mutate worst particles (by this generation's E)
    if (a.mutate) {
        __syncthreads();
        for (int i = tid; i < P; i += kPsoThreads) {
            const float ei = sE[i];
            int rank = 0;
            for (int j = 0; j < P; ++j) rank += ranks_before(sE[j], j, ei, i);
            if (rank >= P - a.n_mutate) {
                for (int jb = 0; jb < kMutBlocks; ++jb) {
                    const U4 r = philox4x32_10(U4{(uint32_t)i, (kStreamMutate << 16) | (uint32_t)jb, a.gen, a.frame},
                                               a.key0, a.key1);
                    const uint32_t u[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
                    for (int l = 0; l < 4; ++l) {
                        const int d = 6 + 4 * jb + l;
                        if (d >= kNdof) break;
                        const size_t o = (size_t)i * kNdof + d;
                        a.x[o] = fmaf(u01(u[l]), lim.hi[d] - lim.lo[d], lim.lo[d]);
                        a.v[o] = 0.f;
                    }
                }
            }
        }
    }
}

// One generation of the swarm fused with the FK of the new positions: 64
// threads per particle, each CTA taking particles q = blockIdx.x, + gridDim.x,
// ... (the grid is what the device keeps resident, so the model is copied into
// shared memory once per CTA rather than once per particle: the copy reads the
// launch parameter with a different address in every lane, which the constant
// cache serves one address at a time).  Every particle's update reads the
// whole E / pbest_E vectors of its swarm (O(P)) to find the global best and its
// own mutation rank, so no particle waits for another: positions are
// double-buffered (x is read, x_next written) and a particle's personal best
// is judged improved when E <= pbest_E as read, which gives the same answer
// whether or not its owner has already stored the update.
template <class M>  // DevModelCore for the paper's kc, DevModel for a kc variant
__global__ void __launch_bounds__(64) pso_step_fk_kernel(const __grid_constant__ M model_param, const PsoFkArgs a)
{
    __shared__ FkShared sh;
    __shared__ CollideSmem<M> s_col;
    __shared__ float s_r[4 * kPairBlocks], s_m[4 * kMutBlocks];
    __shared__ float s_xn[kNdof];
    __shared__ float red_v[2];
    __shared__ int red_i[2], red_r[2];
    extern __shared__ float s_e[];  // E [P] then pbest_E [P] of this particle's swarm
    const int t = threadIdx.x;
    const int total = a.batch.views ? a.batch.P_total : a.P;
    pdl_launch_dependents();
    fk_load_model(sh, model_param);
    const CollideShared* col = collide_load(s_col, model_param);
    for (int q = blockIdx.x; q < total; q += gridDim.x) {
        // the swarm of particle q: particles [off, off + P), q is number i of them
        int off = 0, P = a.P, n_mutate = a.n_mutate, s = 0;
        uint32_t k0 = a.key0, k1 = a.key1;
        float4 cam = a.cam;
        if (a.batch.views) {
            s = a.batch.sid[q];
            const SwarmView& v = a.batch.views[s];
            off = v.offset;
            P = v.P;
            n_mutate = v.n_mutate;
            k0 = v.key0;
            k1 = v.key1;
            cam = make_float4(v.fx, v.fy, v.cx, v.cy);
        }
        const int i = q - off;
        float* s_pe = s_e + P;
        // this particle's random numbers depend only on (particle, generation, frame, seed):
        // the first are drawn while the previous kernel finishes
        draw_step_randoms(i, a.gen, a.frame, k0, k1, s_r, s_m, t);
        if (q == (int)blockIdx.x) pdl_wait();  // E comes from the previous kernel
        if (a.batch.views) {
            const uint32_t stopped = swarm_stop_gen(a.batch, s);
            if (stopped != 0u && stopped < a.gen) {  // stopped earlier in the frame: positions carried over
                if (t < kNdof) a.x_next[(size_t)q * kNdof + t] = a.x[(size_t)q * kNdof + t];
                __syncthreads();  // the shared random numbers are drawn anew for the next particle
                continue;
            }
        }
        float xi = 0.f, pbi = 0.f, vi = 0.f;
        if (t < kNdof) {  // this particle's own state, loaded before the global best is known
            xi = a.x[(size_t)q * kNdof + t];
            pbi = a.pbest[(size_t)q * kNdof + t];
            vi = a.v[(size_t)q * kNdof + t];
        }
        for (int j = t; j < P; j += 64) {
            s_e[j] = a.E[off + j];
            s_pe[j] = a.pbest_E[off + j];
        }
        __syncthreads();
        const SwarmRefs R{a.x, a.x_next, a.v, a.pbest, a.pbest_E, a.gbest, a.gbest_E, a.c1, a.c2, a.w, a.mutate};
        const StepOut o = swarm_update<64>(R, q, i, off, P, s, n_mutate, s_e, s_pe, s_r, s_m, sh.model.lo,
                                           sh.model.hi, xi, pbi, vi, s_pe[i], true, red_v, red_i, red_r);
        if (a.batch.views && a.e_stop > 0.f && o.gE < a.e_stop) {
            // Section III.B's stopping rule: the swarm's best is good enough.  This
            // generation's bests stand (stored above); the swarm stays where it was
            // (x_next = x, v as it was, the records of x kept), and the later
            // generations of the frame skip it
            if (t < kNdof) {
                a.x_next[(size_t)q * kNdof + t] = xi;
                a.v[(size_t)q * kNdof + t] = vi;
            }
            if (i == 0 && t == 0) set_swarm_stop_gen(a.batch, s, a.gen);
            __syncthreads();
            continue;
        }
        if (t < kNdof) s_xn[t] = o.xn;
        // FK of the new pose (fk_particle starts with a barrier that publishes s_xn)
        fk_particle(sh, col, s_xn, cam, a.prims + (size_t)q * sh.model.n_prims * 4, a.kc + q,
                    a.status);
        __syncthreads();  // this particle's shared state is no longer read
    }
}

// CTAs of pso_step_fk_kernel the current device keeps resident with `smem`
// bytes of dynamic shared memory
template <class M>
static int step_fk_resident(size_t smem)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pso_step_fk_kernel<M>, 64, smem) != cudaSuccess)
        return 0;
    return sms * per_sm;
}

cudaError_t launch_pso_step_fk(const DevModel& model, const PsoFkArgs& args, cudaStream_t stream)
{
    const bool core = model.kc_variant == HS_KC_ABDUCTION;
    static std::atomic<uint32_t> opted[2][64];
    const int smem_max = 2 * HS_FUSED_MAX_PARTICLES * (int)sizeof(float);
    const cudaError_t e = core ? opt_in_dynamic_smem(pso_step_fk_kernel<DevModelCore>, smem_max, opted[0])
                               : opt_in_dynamic_smem(pso_step_fk_kernel<DevModel>, smem_max, opted[1]);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    // every particle of all swarms of a batch, over at most the resident CTAs;
    // shared memory for the largest swarm
    const int total = args.batch.views ? args.batch.P_total : args.P;
    cfg.dynamicSmemBytes = 2 * (size_t)args.P * sizeof(float);
    const int resident = core ? step_fk_resident<DevModelCore>(cfg.dynamicSmemBytes)
                              : step_fk_resident<DevModel>(cfg.dynamicSmemBytes);
    cfg.gridDim = dim3(resident > 0 ? std::min(total, resident) : total);
    cfg.blockDim = dim3(64);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return core ? cudaLaunchKernelEx(&cfg, pso_step_fk_kernel<DevModelCore>, static_cast<const DevModelCore&>(model),
                                     args)
                : cudaLaunchKernelEx(&cfg, pso_step_fk_kernel<DevModel>, model, args);
}

cudaError_t launch_pso_init(const Limits& lim, const PsoInitArgs& args, cudaStream_t stream)
{
    const int n = args.P * kInitBlocks;
    pso_init_kernel<<<(n + 255) / 256, 256, 0, stream>>>(lim, args);
    return cudaGetLastError();
}

cudaError_t launch_pso_step(const Limits& lim, const PsoStepArgs& args, cudaStream_t stream)
{
    const size_t smem = (size_t)args.P * sizeof(float);
    pso_step_kernel<<<1, kPsoThreads, smem, stream>>>(lim, args);
    return cudaGetLastError();
}

}  // namespace hs
