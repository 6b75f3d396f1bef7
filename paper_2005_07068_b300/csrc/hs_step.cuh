// hs_step.cuh -- one particle's PSO generation (Section III.B: personal and
// global best, Eq. 6-7 with per-dimension r1/r2, clamping to Tables 1-2, and
// every few generations the re-draw of the worst particles' finger
// dimensions), shared by the fused swarm step (pso_step_fk) and the
// persistent frame kernel (track_frame), which therefore move a swarm
// identically.
//
// The update reads every particle's E and pbest_E of the swarm but writes only
// its own particle, so no particle waits for another.  It tolerates another
// particle's owner storing that particle's new pbest / pbest_E concurrently:
// the global best is argmin_j min(E_j, pbest_E_j as read) -- the same value
// whether or not pbest_E_j has been updated -- and its position is x_j when
// E_j <= pbest_E_j as read (then pbest_j is, or becomes, x_j), else pbest_j
// (which is then not being written).  On an exact tie E_j == pbest_E_j of the
// global best, gbest takes x_j.
#pragma once

#include <climits>

#include "hs_fk.cuh"

namespace hs {

constexpr int kInitBlocks = (kNdof + 3) / 4;      // Philox blocks per particle for 26 dims
constexpr int kPairBlocks = (2 * kNdof + 3) / 4;  // for r1/r2 of 26 dims
constexpr int kMutBlocks = (kNdof - 6 + 3) / 4;   // for the 20 finger dims

// (E_j, j) ranks before (E_i, i); NaN ranks after every number
__device__ __forceinline__ bool ranks_before(float ej, int j, float ei, int i)
{
    const bool nj = isnan(ej), ni = isnan(ei);
    if (nj != ni) return ni;
    if (!nj && ej != ei) return ej < ei;
    return j < i;
}

// Tracking initialisation of dimension d of particle number i of a swarm
// (random positions around the seed pose; particle 0 is the seed pose):
// Philox4x32-10 stream 3, counter (i, 3 << 16 | d / 4, 0, frame), word d % 4.
__device__ __forceinline__ float init_position(int i, int d, float seed_d, float scale_d, float lo_d, float hi_d,
                                               uint32_t frame, uint32_t k0, uint32_t k1)
{
    const U4 r = philox4x32_10(U4{(uint32_t)i, (kStreamInit << 16) | (uint32_t)(d / 4), 0u, frame}, k0, k1);
    const uint32_t u[4] = {r.x, r.y, r.z, r.w};
    const float xv = i == 0 ? seed_d : fmaf(fmaf(2.f, u01(u[d % 4]), -1.f), scale_d, seed_d);
    return fminf(fmaxf(xv, lo_d), hi_d);
}

// threads t < kPairBlocks: r1/r2 of particle number i (s_r [4 kPairBlocks]:
// number 2d is r1 of dimension d, 2d + 1 its r2); threads 32 .. 32 +
// kMutBlocks - 1: its mutation numbers (s_m [4 kMutBlocks], number d - 6 for
// finger dimension d).  They depend only on (particle, generation, frame, key).
__device__ __forceinline__ void draw_step_randoms(int i, uint32_t gen, uint32_t frame, uint32_t k0, uint32_t k1,
                                                  float* s_r, float* s_m, int t)
{
    if (t < kPairBlocks) {
        const U4 r = philox4x32_10(U4{(uint32_t)i, (kStreamPso << 16) | (uint32_t)t, gen, frame}, k0, k1);
        s_r[4 * t] = u01(r.x);
        s_r[4 * t + 1] = u01(r.y);
        s_r[4 * t + 2] = u01(r.z);
        s_r[4 * t + 3] = u01(r.w);
    } else if (t >= 32 && t < 32 + kMutBlocks) {
        const int b = t - 32;
        const U4 r = philox4x32_10(U4{(uint32_t)i, (kStreamMutate << 16) | (uint32_t)b, gen, frame}, k0, k1);
        s_m[4 * b] = u01(r.x);
        s_m[4 * b + 1] = u01(r.y);
        s_m[4 * b + 2] = u01(r.z);
        s_m[4 * b + 3] = u01(r.w);
    }
}

// the swarm arrays one update touches (particle rows are global indices)
struct SwarmRefs {
    const float* x;  // [.][26] positions that were scored (read only)
    float* x_next;   // [.][26] new positions
    float* v;
    float* pbest;
    float* pbest_E;
    float* gbest;    // [S][26]
    float* gbest_E;  // [S]
    float c1, c2, w;
    int mutate;      // this generation re-draws the worst n_mutate particles' finger dims
};

// what one update produces for the calling thread (t < 26: dimension t)
struct StepOut {
    float xn, vn, pb;  // new position, velocity and personal best of dimension t
    bool imp;          // the personal best improved (pbest_E becomes E_i)
    int g;             // the swarm's global best (index within the swarm)
    float gE;          // and its E
};

// a caller's early read of one particle's x and pbest (dimension t), taken
// after every particle's previous update was stored: if that particle turns
// out to be the global best, its position comes from here instead of a
// second read (the values are the same: x does not change during an update,
// and pbest_g is only rewritten when x_g becomes the best, in which case x_g
// is taken)
struct GbestGuess {
    int g;  // swarm index, or -1 for none
    float x, pb;
};

// The global best and the ranks: what every particle's update reads of the
// whole swarm.
struct SwarmBest {
    int g;     // argmin_j min(E_j, pbest_E_j as read): lowest index on ties, NaN never wins
    float gE;  // that minimum
    int rank;  // particles ranking before particle i by E (counted when mutating)
};

// NT threads (a multiple of 32) call it; s_e / s_pe [P] hold the swarm's E and
// pbest_E as read (the caller fills them and synchronises).  red_*: [NT / 32]
// shared scratch.  Every thread gets the result.
template <int NT>
__device__ __forceinline__ SwarmBest swarm_best(int P, int i, bool mutate, const float* s_e, const float* s_pe,
                                                float* red_v, int* red_i, int* red_r)
{
    static_assert(NT % 32 == 0, "whole warps");
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const float ei = s_e[i];
    float bv = INFINITY;
    int bi = INT_MAX, rank = 0;
    for (int j = t; j < P; j += NT) {
        const float ej = s_e[j], pj = s_pe[j];
        const float pe = ej < pj ? ej : pj;
        if (bi == INT_MAX || pe < bv) {
            bv = pe;
            bi = j;
        }
        if (mutate) rank += ranks_before(ej, j, ei, i);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi != INT_MAX && (bi == INT_MAX || ov < bv || (ov == bv && oi < bi))) {
            bv = ov;
            bi = oi;
        }
        rank += __shfl_xor_sync(0xffffffffu, rank, o);
    }
    if (lane == 0) {
        red_v[warp] = bv;
        red_i[warp] = bi;
        red_r[warp] = rank;
    }
    __syncthreads();
    SwarmBest b{red_i[0], red_v[0], red_r[0]};
#pragma unroll
    for (int w = 1; w < NT / 32; ++w) {
        if (red_i[w] != INT_MAX && (b.g == INT_MAX || red_v[w] < b.gE || (red_v[w] == b.gE && red_i[w] < b.g))) {
            b.g = red_i[w];
            b.gE = red_v[w];
        }
        b.rank += red_r[w];
    }
    return b;
}

// The same from one warp alone: every warp of the caller computes it over all
// P particles and every lane gets the result, with no shared memory and no
// barrier (the order is total -- pbest_E is never NaN, so min(E, pbest_E) is
// not either -- so every lane's reduction ends at the same argmin).
__device__ __forceinline__ SwarmBest swarm_best_warp(int P, int i, bool mutate, const float* s_e, const float* s_pe)
{
    const int lane = threadIdx.x & 31;
    const float ei = s_e[i];
    float bv = INFINITY;
    int bi = INT_MAX, rank = 0;
    for (int j = lane; j < P; j += 32) {
        const float ej = s_e[j], pj = s_pe[j];
        const float pe = ej < pj ? ej : pj;
        if (bi == INT_MAX || pe < bv) {
            bv = pe;
            bi = j;
        }
        if (mutate) rank += ranks_before(ej, j, ei, i);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi != INT_MAX && (bi == INT_MAX || ov < bv || (ov == bv && oi < bi))) {
            bv = ov;
            bi = oi;
        }
        rank += __shfl_xor_sync(0xffffffffu, rank, o);
    }
    return SwarmBest{bi, bv, rank};
}

// dimension t of the global best's position: its current x if that is its
// personal best now, else its pbest (read through L2: another CTA of a
// resident grid may have written them)
__device__ __forceinline__ float gbest_position(const float* x, const float* pbest, int row, bool x_is_best, int t)
{
    return x_is_best ? __ldcg(x + (size_t)row * kNdof + t) : __ldcg(pbest + (size_t)row * kNdof + t);
}

// Eq. 6-7 for dimension t of one particle (r1 = number 2t, r2 = number 2t+1 of
// s_r), then the clamp to the limits; a mutated particle re-draws its finger
// dimensions and zeroes their velocity.  imp: its personal best improved.
__device__ __forceinline__ StepOut swarm_move(float c1, float c2, float w, bool imp, bool mutated, int t, float xi,
                                              float pbi, float vi, float gv, const float* s_r, const float* s_m,
                                              const float* lo, const float* hi)
{
    StepOut out{0.f, 0.f, imp ? xi : pbi, imp, 0};
    float acc = fmaf(c1 * s_r[2 * t], out.pb - xi, vi);
    acc = fmaf(c2 * s_r[2 * t + 1], gv - xi, acc);
    float vn = w * acc;
    float xn = fminf(fmaxf(xi + vn, lo[t]), hi[t]);
    if (mutated && t >= 6) {
        xn = fmaf(s_m[t - 6], hi[t] - lo[t], lo[t]);
        vn = 0.f;
    }
    out.xn = xn;
    out.vn = vn;
    return out;
}

// One generation of particle number i (global row q) of a swarm of P
// particles starting at row off (swarm s), updated in place.  NT threads call
// it; s_e / s_pe as for swarm_best; xi, pbi, vi: the particle's own dimension
// t (t < 26) and own_pe its own pbest_E, from a copy no other thread writes.
// When `store`, writes the particle's v, x_next, pbest / pbest_E (on
// improvement) and, for i == 0, the swarm's gbest.  guess: see GbestGuess.
// kWarpBest: every warp finds the global best on its own (swarm_best_warp),
// else the NT threads share the scan (swarm_best); the result is the same.
template <int NT, bool kWarpBest = false>
__device__ __forceinline__ StepOut swarm_update(const SwarmRefs& R, int q, int i, int off, int P, int s, int n_mutate,
                                                const float* s_e, const float* s_pe, const float* s_r,
                                                const float* s_m, const float* lo, const float* hi, float xi,
                                                float pbi, float vi, float own_pe, bool store, float* red_v,
                                                int* red_i, int* red_r, const GbestGuess& guess = GbestGuess{-1, 0.f, 0.f})
{
    const int t = threadIdx.x;
    const SwarmBest b = kWarpBest ? swarm_best_warp(P, i, R.mutate, s_e, s_pe)
                                  : swarm_best<NT>(P, i, R.mutate, s_e, s_pe, red_v, red_i, red_r);
    const float ei = s_e[i];
    StepOut out{0.f, 0.f, 0.f, ei < own_pe, b.g, b.gE};  // strict improvement of this particle's personal best
    const bool mutated = R.mutate && b.rank >= P - n_mutate;
    if (t < kNdof) {
        const bool x_is_best = s_e[b.g] <= s_pe[b.g];
        const float gv = b.g == guess.g ? (x_is_best ? guess.x : guess.pb)
                                        : gbest_position(R.x, R.pbest, off + b.g, x_is_best, t);
        if (store && i == 0) R.gbest[(size_t)s * kNdof + t] = gv;
        if (store && out.imp) R.pbest[(size_t)q * kNdof + t] = xi;
        out = swarm_move(R.c1, R.c2, R.w, out.imp, mutated, t, xi, pbi, vi, gv, s_r, s_m, lo, hi);
        out.g = b.g;
        out.gE = b.gE;
        if (store) {
            R.v[(size_t)q * kNdof + t] = out.vn;
            R.x_next[(size_t)q * kNdof + t] = out.xn;
        }
    }
    if (store && t == 0) {
        if (out.imp) R.pbest_E[q] = ei;
        if (i == 0) R.gbest_E[s] = b.gE;
    }
    return out;
}

}  // namespace hs
