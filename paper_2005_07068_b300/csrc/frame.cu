// frame.cu -- one whole tracking frame (Section III.B: initialise the swarm
// around the previous frame's best pose, then generations of "score every
// particle (Section III.A, Eq. 4-5), move the swarm (Eq. 6-7, mutation)") in
// a single cooperative launch.
//
// The graph path launches a kernel per step (observation totals, init, FK,
// then render + fused step per generation): about 16 us per generation at
// 64 particles, mostly launch gaps and the latency chains of short kernels.
// Here the grid's CTAs stay resident for the whole frame, dealt evenly to the
// particles (each gets floor(n / P) or ceil(n / P) of the n CTAs):
//
//  * every CTA keeps its particle's state (position, velocity, personal best)
//    and its FK records in shared memory; the CTAs of a particle run the
//    same FK and the same swarm update (identical inputs, identical results),
//    and the first of them (the primary) stores the particle's state;
//  * generation g: FK of the current pose -> raster records -> the CTA's share
//    of the particle's 16x4 units (the unit renderer of render_score_batch,
//    hs_units.cuh) -> integer sums added to the particle's slot of generation
//    g (three slots rotate, so a slot is cleared two generations before it is
//    reused) -> one grid barrier -> every CTA forms E of every particle of the
//    swarm from the sums (form_E, as the render kernels do) and takes its
//    particle's step (swarm_update, as pso_step_fk does);
//  * the observation totals are counted by all CTAs before the first barrier.
//
// Results equal the graph path bit for bit (unit kernel render + pso_step_fk),
// because every piece of arithmetic is the same code.  The barrier's wait is
// bounded (about a second): if it runs out, HS_DEV_BARRIER_TIMEOUT is set and
// the CTAs leave.  The last CTA to leave returns the workspace's counters and
// sums to zero for the next frame.
#include <atomic>

#include "hs_step.cuh"
#include "hs_units.cuh"

namespace hs {

constexpr int kFrameWarps = 8;
constexpr int kFrameThreads = kFrameWarps * 32;
constexpr unsigned long long kBarrierWaitNs = 1000000000ull;  // a grid barrier waits at most ~1 s (wall clock)
constexpr uint32_t kBarrierPolls = 1u << 26;  // and at most this many polls, should the clock not advance


// a particle's FK records, raster records and pixel boxes for up to MP primitives
template <int MP>
struct FramePrims {
    float4 rec[MP * 4];
    float4 rast[MP * kRastVec];
    int2 pbox[MP];
};
template <>
struct FramePrims<0> {};  // kept in dynamic shared memory, sized for the model

// NW: warps of the CTA; Col: the kc variants' collision data (CollideShared),
// or a placeholder byte for kernels launched only for the paper's kc; MP: see FramePrims
template <int NW, class Col = CollideShared, int MP = kMaxPrims>
struct FrameSharedT {
    FkShared fk;                      // model, pose, bone frames
    Col col;                          // the kc variants' collision data
    FramePrims<MP> pr;                // this particle's records
    alignas(128) unsigned char tile[NW][kStages][kSlot];
    uint64_t bar[NW][kStages];
    float x[kNdof], v[kNdof], pb[kNdof];  // the particle's state (identical in all its CTAs)
    float pe;                             // its personal-best E
    float kc;
    float r[4 * kPairBlocks], m[4 * kMutBlocks];
    long long red_t[NW];
    uint32_t red_c[NW][3];
    float red_v[NW];
    int red_i[NW], red_r[NW];
    int gprev;  // the swarm's global best after the previous generation
    uint32_t st[2];
    int4 wbox[2];  // union of the pixel boxes of primitives 0..31 and 32..63
};
using FrameShared = FrameSharedT<kFrameWarps>;

// all threads of every CTA: returns false if the wait ran out.  work() runs
// on every thread after this CTA has arrived, while the others are awaited
// (it must not touch what the barrier publishes).
template <class Work>
__device__ __forceinline__ bool grid_barrier(uint32_t* count, uint32_t target, uint32_t* status, const Work& work)
{
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        // release: this CTA's earlier writes (seen by thread 0 through the CTA
        // barrier) are visible to whoever acquires the count; no value returns,
        // so the thread goes on at once
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
    }
    work();
    if (threadIdx.x == 0) {
        uint32_t v;
        uint32_t polls = 0;
        unsigned long long t0;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
        for (;;) {
            asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
            if (v >= target) break;
            unsigned long long now;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
            if (now - t0 > kBarrierWaitNs || ++polls >= kBarrierPolls) {
                set_status(status, HS_DEV_BARRIER_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
    }
    return __syncthreads_and(ok) != 0;
}

__global__ void __launch_bounds__(kFrameThreads, 3)
    track_frame_kernel(const __grid_constant__ DevModel model, const __grid_constant__ CUtensorMap tm_depth,
                       const __grid_constant__ CUtensorMap tm_skin, const FrameArgs a)
{
    __shared__ FrameShared sh;
    extern __shared__ float s_dyn[];  // E [P], then pbest_E [P] as read
    float* s_e = s_dyn;
    float* s_pe = s_dyn + a.P;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t nblocks = gridDim.x;
    const uint32_t missing = a.ctl->missing;  // zero but in the test of the barrier's time limit
    // particle p has CTAs [ceil(p n / P), ceil((p + 1) n / P)) of the n in the grid
    const int P = a.P, p = (int)((unsigned long long)blockIdx.x * (unsigned)P / nblocks);
    const int first = (int)(((unsigned long long)p * nblocks + P - 1) / (unsigned)P);
    const int C = (int)(((unsigned long long)(p + 1) * nblocks + P - 1) / (unsigned)P) - first;
    const int c = (int)blockIdx.x - first;
    const bool primary = c == 0;
    const int n_prims = model.n_prims;

    fk_load_model(sh.fk, model);
    const CollideShared* col = collide_load(sh.col, model);
    if (lane < kStages) mbar_init(&sh.bar[warp][lane], 1);
    if (t == 0) {
        mbar_fence_init();
        sh.st[0] = sh.st[1] = 0u;
    }
    __syncthreads();

    // observation totals of the frame (#valid skin pixels, #skin pixels):
    // rows split over all CTAs, complete before the first barrier
    {
        uint32_t nv = 0, ns = 0;
        for (int y = blockIdx.x; y < a.H; y += nblocks) {
            for (int x = t; x < a.W; x += kFrameThreads) {
                const bool S = a.skin[(size_t)y * a.skin_pitch + x] != 0;
                const float od = a.depth_f32 ? reinterpret_cast<const float*>(a.depth + (size_t)y * a.depth_pitch)[x]
                                             : (float)reinterpret_cast<const uint16_t*>(
                                                   a.depth + (size_t)y * a.depth_pitch)[x];
                ns += S;
                nv += S && od > 0.f;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            nv += __shfl_xor_sync(0xffffffffu, nv, o);
            ns += __shfl_xor_sync(0xffffffffu, ns, o);
        }
        if (lane == 0 && (nv | ns)) {
            atomicAdd(&sh.st[0], nv);
            atomicAdd(&sh.st[1], ns);
        }
    }

    // tracking initialisation of this particle (as pso_init)
    if (t < kNdof) {
        const float xv = init_position(p, t, a.seed_pose[t], a.scale[t], sh.fk.model.lo[t], sh.fk.model.hi[t],
                                       a.frame, a.key0, a.key1);
        sh.x[t] = xv;
        sh.v[t] = 0.f;
        sh.pb[t] = xv;
        if (primary) {
            const size_t o = (size_t)p * kNdof + t;
            a.xbuf[0][o] = xv;
            a.v[o] = 0.f;
            a.pbest[o] = xv;
            if (p == 0) a.gbest[t] = xv;
        }
    }
    if (t == 0) {
        sh.pe = INFINITY;
        sh.gprev = 0;
        if (primary) {
            a.pbest_E[p] = INFINITY;
            if (p == 0) a.gbest_E[0] = INFINITY;
        }
    }
    __syncthreads();
    if (t == 0 && (sh.st[0] | sh.st[1])) {
        atomicAdd(&a.stats[0], sh.st[0]);
        atomicAdd(&a.stats[1], sh.st[1]);
    }

    const ParticleView pv{a.W, a.H, a.depth_f32, a.inv_fx, a.off_x, a.inv_fy, a.off_y, a.stats, &tm_depth, &tm_skin};
    RenderArgs ra = {};
    ra.d_m = a.d_m;
    ra.d_M = a.d_M;
    ra.status = a.status;
    const SwarmRefs R0{nullptr, nullptr, a.v, a.pbest, a.pbest_E, a.gbest, a.gbest_E, a.c1, a.c2, a.w, 0};
    uint32_t phases = 0u;
    uint32_t barriers = 0u;
    bool alive = true;
    for (int g = 1; g <= a.gens; ++g) {
        // FK of the current pose (fk_particle starts with a barrier that publishes
        // sh.x); each record's raster form is made by the thread that formed it
        fk_particle(sh.fk, col, sh.x, a.cam, sh.pr.rec, &sh.kc, a.status, [&](int j, const float* rec) {
            const float4 r4[4] = {make_float4(rec[0], rec[1], rec[2], rec[3]),
                                  make_float4(rec[4], rec[5], rec[6], rec[7]),
                                  make_float4(rec[8], rec[9], rec[10], rec[11]),
                                  make_float4(rec[12], rec[13], rec[14], rec[15])};
            store_raster(make_raster(r4, pv.inv_fx, pv.off_x, pv.inv_fy, pv.off_y), sh.pr.rast + kRastVec * j);
            sh.pr.pbox[j] = make_int2(__float_as_int(rec[14]), __float_as_int(rec[15]));
            // the union of the pixel boxes, per warp of record threads
            const int w = j >> 5;
            const uint32_t mask = n_prims >= 32 * (w + 1) ? 0xffffffffu : (1u << (n_prims - 32 * w)) - 1u;
            const int u0 = __reduce_min_sync(mask, lo_i16(rec[14])), v0 = __reduce_min_sync(mask, hi_i16(rec[14]));
            const int u1 = __reduce_max_sync(mask, lo_i16(rec[15])), v1 = __reduce_max_sync(mask, hi_i16(rec[15]));
            if ((j & 31) == 0) sh.wbox[w] = make_int4(u0, v0, u1, v1);
        });
        __syncthreads();
        // the particle's units (every thread forms the same box)
        int box[4];
        {
            int4 b = sh.wbox[0];
            if (n_prims > 32) {
                const int4 b1 = sh.wbox[1];
                b = make_int4(min(b.x, b1.x), min(b.y, b1.y), max(b.z, b1.z), max(b.w, b1.w));
            }
            unit_box_clip(b.x, b.y, b.z, b.w, a.W, a.H, box);
        }
        long long acc_t = 0;
        uint32_t acc_a = 0, acc_o = 0, acc_h = 0;
        if (box[3] > 0)
            render_units_warp(sh.pr.rast, sh.pr.pbox, n_prims, box, sh.tile[warp], sh.bar[warp], phases,
                              c * kFrameWarps + warp, C * kFrameWarps, pv, ra, p, lane, acc_t, acc_a, acc_o, acc_h);
        warp_sum(acc_t, acc_a, acc_o, acc_h);
        if (lane == 0) {
            sh.red_t[warp] = acc_t;
            sh.red_c[warp][0] = acc_a;
            sh.red_c[warp][1] = acc_o;
            sh.red_c[warp][2] = acc_h;
        }
        __syncthreads();
        FrameSums* slot = a.sums + (size_t)(g % 3) * P;
        if (t == 0) {
            for (int w = 1; w < kFrameWarps; ++w) {
                acc_t += sh.red_t[w];
                acc_a += sh.red_c[w][0];
                acc_o += sh.red_c[w][1];
                acc_h += sh.red_c[w][2];
            }
            if (acc_t) atomicAdd(&slot[p].t_fix, (unsigned long long)acc_t);
            if (acc_a) atomicAdd(&slot[p].n_and, acc_a);
            if (acc_o) atomicAdd(&slot[p].n_or, acc_o);
            if (acc_h) atomicAdd(&slot[p].n_hit, acc_h);
            if (primary) slot[p].kc = sh.kc;
        }
        // every particle's sums (and the frame's totals) are in; meanwhile this
        // particle's random numbers for the step
        ++barriers;
        if (!grid_barrier(&a.ctl->barrier, barriers * (nblocks + missing), a.status,
                          [&] { draw_step_randoms(p, (uint32_t)g, a.frame, a.key0, a.key1, sh.r, sh.m, t); })) {
            alive = false;
            break;
        }
        SwarmRefs R = R0;
        R.x = a.xbuf[(g - 1) & 1];
        R.x_next = a.xbuf[g & 1];
        R.mutate = a.mutate_every > 0 && g % a.mutate_every == 0 && a.n_mutate > 0;
        // the previous global best's position, read with the sums: it is most
        // often the global best again, and then needs no read after the argmin
        GbestGuess guess{sh.gprev, 0.f, 0.f};
        if (t < kNdof) {
            guess.x = __ldcg(R.x + (size_t)guess.g * kNdof + t);
            guess.pb = __ldcg(a.pbest + (size_t)guess.g * kNdof + t);
        }
        // E of every particle of the swarm, and the personal-best Es as read
        // (this particle's own from its copy)
        // (loads through L2: other CTAs wrote these during this launch)
        const uint32_t stats[2] = {__ldcg(a.stats), __ldcg(a.stats + 1)};
        for (int j = t; j < P; j += kFrameThreads) {
            const uint4 w0 = __ldcg(reinterpret_cast<const uint4*>(slot + j));
            const uint4 w1 = __ldcg(reinterpret_cast<const uint4*>(slot + j) + 1);
            const long long tf = (long long)(((unsigned long long)w0.y << 32) | w0.x);
            float t_sum;
            uint32_t so;
            s_e[j] = form_E(tf, w0.z, w0.w, stats, a.d_M, a.lambda, a.lambda_k, __uint_as_float(w1.y), t_sum, so);
            s_pe[j] = j == p ? sh.pe : __ldcg(a.pbest_E + j);
        }
        __syncthreads();
        float xi = 0.f, pbi = 0.f, vi = 0.f;
        if (t < kNdof) {
            xi = sh.x[t];
            pbi = sh.pb[t];
            vi = sh.v[t];
        }
        const StepOut o = swarm_update<kFrameThreads, true>(R, p, p, 0, P, 0, a.n_mutate, s_e, s_pe, sh.r, sh.m,
                                                      sh.fk.model.lo, sh.fk.model.hi, xi, pbi, vi, sh.pe, primary,
                                                      sh.red_v, sh.red_i, sh.red_r, guess);
        __syncthreads();  // every thread has read sh.x / sh.pe of this generation
        if (t < kNdof) {
            sh.x[t] = o.xn;
            sh.v[t] = o.vn;
            sh.pb[t] = o.pb;
        }
        if (t == 0) {
            if (o.imp) sh.pe = s_e[p];
            sh.gprev = o.g;
            if (primary) {
                a.E[p] = s_e[p];
                // the slot generation g + 2 will use: every CTA read it (as
                // generation g - 1's) before this barrier, none writes it before the next
                a.sums[(size_t)((g + 2) % 3) * P + p] = FrameSums{};
            }
        }
    }
    if (alive) {
        // the records and kc of the final positions
        fk_particle(sh.fk, col, sh.x, a.cam, sh.pr.rec, &sh.kc, a.status);
        __syncthreads();
        if (primary) {
            if (a.prims_out)
                for (int i = t; i < n_prims * 4; i += kFrameThreads)
                    a.prims_out[(size_t)p * n_prims * 4 + i] = sh.pr.rec[i];
            if (t == 0) a.kc[p] = sh.kc;
        }
    }
    // leave; the last CTA returns the workspace to zero
    __syncthreads();
    __shared__ uint32_t s_last;
    if (t == 0) {
        uint32_t done;
        asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(done) : "l"(&a.ctl->exited) : "memory");
        s_last = done == nblocks - 1;
    }
    __syncthreads();
    if (s_last) {
        for (int i = t; i < 3 * P; i += kFrameThreads) a.sums[i] = FrameSums{};
        if (t == 0) {
            a.ctl->barrier = 0u;
            a.ctl->exited = 0u;
        }
    }
}

// ---- every swarm of a batch: a whole frame in one cooperative launch ----
//
// The frame of S sequences at once (uneven ROIs and swarm sizes, Section IV's
// parallelism between particles): the work is a list of tasks, generation by
// generation, each generation's particles in the batch's order (largest ROI
// first).  A resident CTA takes the next task from a counter and does, for
// particle q (number i of swarm s) at generation g:
//
//  * g == 1: the tracking initialisation of q (as pso_init_multi);
//    g >= 2: once every particle of s has been rendered at generation g - 1
//    (a per-swarm count of finished renders, awaited with a time limit),
//    q's step of generation g - 1 (swarm_update: the global best and the
//    mutation rank from the swarm's E and pbest_E, then Eq. 6-7), as
//    pso_step_fk_multi does;
//  * g <= gens: FK of q's new pose, its raster records, the render of all its
//    16x4 units by the CTA's warps (the unit renderer, hs_units.cuh), and E
//    (form_E from the CTA's integer sums) into the generation's E buffer;
//    then the swarm's count goes up (release);
//  * g == gens + 1: q's final E, and the records and kc of its final pose.
//
// A task waits only for tasks of an earlier generation, and those were taken
// earlier by CTAs that are resident (the launch is cooperative), so the
// earliest unfinished task never waits: the frame always ends.  Swarms run
// generations apart from one another, so no CTA idles at a grid barrier.
// Every piece of arithmetic is the code of the step-by-step batch calls, so
// the results equal theirs bit for bit.  If a wait runs out (about a second),
// HS_DEV_BARRIER_TIMEOUT is set and every CTA stops taking tasks; the last CTA
// to leave returns the workspace's counters to zero.
// warps of a task's CTA: four, and registers (64) and shared memory (the
// particle's records sized for the model) for eight CTAs per SM, so that the
// latency of one task's serial phases (FK, the swarm scan) hides behind the
// others' (more CTAs of four warps measured faster than fewer of eight, and
// than CTAs of two warps)
constexpr int kMultiWarps = 4;
constexpr int kMultiThreads = kMultiWarps * 32;

// dynamic shared memory of track_frame_multi_kernel: E and pbest_E of the
// task's swarm [P_max] each, then the particle's FK records, raster records
// and pixel boxes [n_prims] (16-byte aligned)
__host__ __device__ inline size_t frame_multi_prims_offset(int P_max) { return ((size_t)P_max * 8 + 15) / 16 * 16; }
__host__ __device__ inline size_t frame_multi_dyn_bytes(int P_max, int n_prims)
{
    return frame_multi_prims_offset(P_max) + (size_t)n_prims * (sizeof(float4) * (4 + kRastVec) + sizeof(int2));
}

// Model: DevModelCore for the paper's kc (no collision data in shared memory,
// so more CTAs stay resident), DevModel for the kc variants
template <class Model>
__global__ void __launch_bounds__(kMultiThreads, 8)
    track_frame_multi_kernel(const __grid_constant__ Model model, const FrameMultiArgs a)
{
    __shared__ FrameSharedT<kMultiWarps, CollideSmem<Model>, 0> sh;
    __shared__ int s_task, s_go;
    extern __shared__ __align__(16) float s_dyn[];
    float* s_e = s_dyn;
    float* s_pe = s_dyn + a.P_max;
    float4* s_rec = reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(s_dyn) + frame_multi_prims_offset(a.P_max));
    float4* s_rast = s_rec + model.n_prims * 4;
    int2* s_pbox = reinterpret_cast<int2*>(s_rast + model.n_prims * kRastVec);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int n_prims = model.n_prims;
    const int P_total = a.batch.P_total, G = a.gens;
    const uint32_t total = (uint32_t)(G + 1) * (uint32_t)P_total;
    FrameMultiCtl* ctl = a.ctl;
    const uint32_t missing = ctl->missing;  // zero but in the test of the wait's time limit

    fk_load_model(sh.fk, model);
    const CollideShared* col = collide_load(sh.col, model);
    if (lane < kStages) mbar_init(&sh.bar[warp][lane], 1);
    if (t == 0) mbar_fence_init();
    __syncthreads();

    RenderArgs ra = {};
    ra.d_m = a.d_m;
    ra.d_M = a.d_M;
    ra.status = a.status;
    uint32_t phases = 0u;
    for (;;) {
        if (t == 0) {
            const uint32_t k = atomicAdd(&ctl->next, 1u);
            s_task = k < total && *reinterpret_cast<volatile uint32_t*>(&ctl->abort) == 0u ? (int)k : -1;
        }
        __syncthreads();  // also: the previous task's shared state is no longer read
        const int k = s_task;
        if (k < 0) break;
        const int g = k / P_total + 1;
        const int q = a.order[k - (g - 1) * P_total];
        const int s = a.batch.sid[q];
        const SwarmView& view = a.batch.views[s];
        const int off = view.offset, P = view.P, i = q - off;
        const uint32_t k0 = view.key0, k1 = view.key1;
        const float4 cam = make_float4(view.fx, view.fy, view.cx, view.cy);

        if (g == 1) {
            // the tracking initialisation of q (as pso_init_multi)
            if (t < kNdof) {
                const float xv = init_position(i, t, a.seed_poses[(size_t)s * kNdof + t], a.scale[t],
                                               sh.fk.model.lo[t], sh.fk.model.hi[t], a.frame, k0, k1);
                sh.x[t] = xv;
                const size_t o = (size_t)q * kNdof + t;
                a.xbuf[0][o] = xv;
                a.v[o] = 0.f;
                a.pbest[o] = xv;
                if (i == 0) a.gbest[(size_t)s * kNdof + t] = xv;
            }
            if (t == 0) {
                a.pbest_E[q] = INFINITY;
                if (i == 0) {
                    a.gbest_E[s] = INFINITY;
                    set_swarm_stop_gen(a.batch, s, 0u);  // the swarm runs this frame
                }
            }
        } else {
            // every particle of s rendered at generation g - 1 (acquire: their
            // E, positions and bests are visible)
            if (t == 0) {
                const uint32_t target = (uint32_t)(g - 1) * (uint32_t)P + missing;
                int go = 1;
                uint32_t polls = 0;
                const unsigned long long t0 = global_ns();
                for (;;) {
                    uint32_t v;
                    asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(a.done + s) : "memory");
                    if (v >= target) break;
                    if (*reinterpret_cast<volatile uint32_t*>(&ctl->abort) != 0u) {
                        go = 0;
                        break;
                    }
                    if (global_ns() - t0 > kBarrierWaitNs || ++polls >= kBarrierPolls) {
                        set_status(a.status, HS_DEV_BARRIER_TIMEOUT);
                        atomicExch(&ctl->abort, 1u);
                        go = 0;
                        break;
                    }
                    __nanosleep(64);
                }
                s_go = go;
            }
            draw_step_randoms(i, (uint32_t)(g - 1), a.frame, k0, k1, sh.r, sh.m, t);
            __syncthreads();
            if (!s_go) break;
            // q's step of generation g - 1 (as pso_step_fk_multi); loads through
            // L2: other CTAs wrote these during this launch
            const float* Eg = a.Ebuf + (size_t)((g - 1) & 1) * P_total;
            float xi = 0.f, pbi = 0.f, vi = 0.f;
            const float* x_cur = a.xbuf[(g - 2) & 1];
            if (t < kNdof) {
                xi = __ldcg(x_cur + (size_t)q * kNdof + t);
                pbi = __ldcg(a.pbest + (size_t)q * kNdof + t);
                vi = __ldcg(a.v + (size_t)q * kNdof + t);
            }
            for (int j = t; j < P; j += kMultiThreads) {
                s_e[j] = __ldcg(Eg + off + j);
                s_pe[j] = __ldcg(a.pbest_E + off + j);
            }
            __syncthreads();
            SwarmRefs R{x_cur, a.xbuf[(g - 1) & 1], a.v, a.pbest, a.pbest_E, a.gbest, a.gbest_E, a.c1, a.c2, a.w,
                        a.mutate_every > 0 && (g - 1) % a.mutate_every == 0};
            const StepOut o = swarm_update<kMultiThreads>(R, q, i, off, P, s, view.n_mutate, s_e, s_pe, sh.r, sh.m,
                                                          sh.fk.model.lo, sh.fk.model.hi, xi, pbi, vi, s_pe[i],
                                                          true, sh.red_v, sh.red_i, sh.red_r);
            if (t < kNdof) sh.x[t] = o.xn;
            if (g > G) {  // after the last generation: q's E, and the records and kc of its final pose
                if (t == 0) a.E[q] = s_e[i];
                fk_particle(sh.fk, col, sh.x, cam, a.prims_out + (size_t)q * n_prims * 4, a.kc + q, a.status);
                continue;
            }
        }
        if (g > G) {  // no generation at all: the records and kc of the initial pose
            fk_particle(sh.fk, col, sh.x, cam, a.prims_out + (size_t)q * n_prims * 4, a.kc + q, a.status);
            continue;
        }

        // generation g: FK of q's pose (fk_particle starts with a barrier that
        // publishes sh.x), raster records, the render of all q's units
        const ParticleView pv{view.W, view.H, view.depth_f32, view.inv_fx, view.off_x, view.inv_fy, view.off_y,
                              view.stats, &view.tm_depth, &view.tm_skin};
        fk_particle(sh.fk, col, sh.x, cam, s_rec, &sh.kc, a.status, [&](int j, const float* rec) {
            const float4 r4[4] = {make_float4(rec[0], rec[1], rec[2], rec[3]),
                                  make_float4(rec[4], rec[5], rec[6], rec[7]),
                                  make_float4(rec[8], rec[9], rec[10], rec[11]),
                                  make_float4(rec[12], rec[13], rec[14], rec[15])};
            store_raster(make_raster(r4, pv.inv_fx, pv.off_x, pv.inv_fy, pv.off_y), s_rast + kRastVec * j);
            s_pbox[j] = make_int2(__float_as_int(rec[14]), __float_as_int(rec[15]));
            const int w = j >> 5;
            const uint32_t mask = n_prims >= 32 * (w + 1) ? 0xffffffffu : (1u << (n_prims - 32 * w)) - 1u;
            const int u0 = __reduce_min_sync(mask, lo_i16(rec[14])), v0 = __reduce_min_sync(mask, hi_i16(rec[14]));
            const int u1 = __reduce_max_sync(mask, lo_i16(rec[15])), v1 = __reduce_max_sync(mask, hi_i16(rec[15]));
            if ((j & 31) == 0) sh.wbox[w] = make_int4(u0, v0, u1, v1);
        });
        __syncthreads();
        int box[4];
        {
            int4 b = sh.wbox[0];
            if (n_prims > 32) {
                const int4 b1 = sh.wbox[1];
                b = make_int4(min(b.x, b1.x), min(b.y, b1.y), max(b.z, b1.z), max(b.w, b1.w));
            }
            unit_box_clip(b.x, b.y, b.z, b.w, view.W, view.H, box);
        }
        long long acc_t = 0;
        uint32_t acc_a = 0, acc_o = 0, acc_h = 0;
        bool ok = true;
        if (box[3] > 0)
            ok = render_units_warp<false>(s_rast, s_pbox, n_prims, box, sh.tile[warp], sh.bar[warp], phases, warp,
                                   kMultiWarps, pv, ra, q, lane, acc_t, acc_a, acc_o, acc_h);
        warp_sum(acc_t, acc_a, acc_o, acc_h);
        if (lane == 0) {
            sh.red_t[warp] = acc_t;
            sh.red_c[warp][0] = acc_a;
            sh.red_c[warp][1] = acc_o;
            sh.red_c[warp][2] = acc_h;
        }
        // a warp whose observation wait ran out (status flagged) voids the frame
        if (!__syncthreads_and(ok)) {
            if (t == 0) atomicExch(&ctl->abort, 1u);
            break;
        }
        if (t == 0) {
            for (int w = 1; w < kMultiWarps; ++w) {
                acc_t += sh.red_t[w];
                acc_a += sh.red_c[w][0];
                acc_o += sh.red_c[w][1];
            }
            float t_sum;
            uint32_t so;
            a.Ebuf[(size_t)(g & 1) * P_total + q] =
                form_E(acc_t, acc_a, acc_o, view.stats, a.d_M, a.lambda, a.lambda_k, sh.kc, t_sum, so);
            // release: this task's E and q's step (stored by the CTA's threads
            // before the barriers above) are visible to whoever sees the count
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(a.done + s) : "memory");
        }
    }
    // leave; the last CTA returns the workspace to zero
    __syncthreads();
    __shared__ uint32_t s_last;
    if (t == 0) {
        uint32_t d;
        asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(d) : "l"(&ctl->exited) : "memory");
        s_last = d == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        for (int j = t; j < a.batch.S; j += kMultiThreads) a.done[j] = 0u;
        if (t == 0) {
            ctl->next = 0u;
            ctl->exited = 0u;
            ctl->abort = 0u;
        }
    }
}

// the dynamic shared memory of the largest swarm (2 P floats) on top of the
// static part passes the default 48 KB: opt in once per device
static std::atomic<uint32_t> g_frame_opted[64];
static cudaError_t frame_smem_opt_in()
{
    return opt_in_dynamic_smem(track_frame_kernel, 2 * HS_FRAME_MAX_PARTICLES * (int)sizeof(float), g_frame_opted);
}

cudaError_t track_frame_capacity(int* ctas)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = frame_smem_opt_in();
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // the dynamic part (2 P floats) is small next to the static part; size it for the largest P
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, track_frame_kernel, kFrameThreads,
                                                          2 * HS_FRAME_MAX_PARTICLES * sizeof(float));
    *ctas = e == cudaSuccess ? sms * per_sm : 0;
    return e;
}

cudaError_t launch_track_frame(const DevModel& model, const CUtensorMap& tm_depth, const CUtensorMap& tm_skin,
                               const FrameArgs& args, int ctas, cudaStream_t stream)
{
    const cudaError_t e = frame_smem_opt_in();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(kFrameThreads);
    cfg.dynamicSmemBytes = 2 * (size_t)args.P * sizeof(float);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident at once (the grid barrier needs it)
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, track_frame_kernel, model, tm_depth, tm_skin, args);
}


// the batch frame: its static part, then dynamic shared memory for the
// largest swarm of the batch and the model's primitives; one kernel per model type
static std::atomic<uint32_t> g_frame_multi_opted[2][64];
template <class Model>
static cudaError_t frame_multi_smem_opt_in()
{
    return opt_in_dynamic_smem(track_frame_multi_kernel<Model>,
                               (int)frame_multi_dyn_bytes(HS_FRAME_MAX_PARTICLES, kMaxPrims),
                               g_frame_multi_opted[std::is_same<Model, DevModel>::value ? 1 : 0]);
}

template <class Model>
static cudaError_t frame_multi_capacity_of(int* ctas, int P_max, int n_prims)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = frame_multi_smem_opt_in<Model>();
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, track_frame_multi_kernel<Model>, kMultiThreads,
                                                          frame_multi_dyn_bytes(P_max, n_prims));
    *ctas = e == cudaSuccess ? sms * per_sm : 0;
    return e;
}

cudaError_t track_frame_multi_capacity(int* ctas, int P_max, int n_prims, bool collide)
{
    return collide ? frame_multi_capacity_of<DevModel>(ctas, P_max, n_prims)
                   : frame_multi_capacity_of<DevModelCore>(ctas, P_max, n_prims);
}

template <class Model>
static cudaError_t launch_frame_multi_as(const Model& model, const FrameMultiArgs& args, int ctas, cudaStream_t stream)
{
    const cudaError_t e = frame_multi_smem_opt_in<Model>();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(kMultiThreads);
    cfg.dynamicSmemBytes = frame_multi_dyn_bytes(args.P_max, model.n_prims);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident at once (tasks wait on other CTAs' tasks)
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, track_frame_multi_kernel<Model>, model, args);
}

cudaError_t launch_track_frame_multi(const DevModel& model, const FrameMultiArgs& args, int ctas, cudaStream_t stream)
{
    if (frame_multi_needs_collide(model))
        return launch_frame_multi_as(model, args, ctas, stream);
    return launch_frame_multi_as(static_cast<const DevModelCore&>(model), args, ctas, stream);
}

}  // namespace hs
