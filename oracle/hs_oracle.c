/*
 * hs_oracle.c -- FP64 CPU oracle for per-particle hypothesis scoring in the
 * model-based 26-DOF hand tracker of arxiv 2005.07068 (Quach et al.).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously correct
 * statement of what the scoring path computes.  Only the test-suite, the
 * package smoke check and the benchmark's CPU-baseline leg may load it.  It
 * shares no code, header, table or constant generator with the CUDA path.
 *
 * Every routine is written from the paper:
 *   pose layout ......... Eq. 1-3 (Section II.A)
 *   joint limits ........ Tables 1-2 (passed in as lo/hi)
 *   hand geometry ....... Section II.A and Fig. 2 (passed in as a descriptor)
 *   depth map r_d ....... Section III.A (projection with camera C)
 *   match map r_m ....... Section III.A, the rule before Eq. 4
 *   discrepancy D ....... Eq. 4;  objective E = D + lambda_k kc(h) ..... Eq. 5
 *   kc(h) ............... the definition after Eq. 5
 *   swarm update ........ Eq. 6-7 and the constants of Section III.B
 *   mutation ............ Section III.B (every 3 generations, worst half,
 *                         20 finger dims re-drawn)
 *   Philox4x32-10 ....... Salmon, Moraes, Dror, Shaw, "Parallel random
 *                         numbers: as easy as 1, 2, 3", SC'11
 * Readings where the paper is silent are those listed in the design notes:
 * camera model, kinematic conventions, cost branches for undefined depth,
 * kc pairs, mutation timing, the tracking initialisation and the stream
 * layout of the random numbers.
 *
 * Rendering is brute force: every pixel against every primitive, with the
 * textbook quadratic in FP64 and no culling.  Sums run in row-major pixel
 * order.  OpenMP is used only across independent particles.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <stdlib.h>

#define OR_NDOF 26
#define OR_MAXB 64
#define OR_MAXP 128

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11): 10 rounds of a multiply-xor Feistel network on a   */
/* 128-bit counter with a 64-bit key bumped by the Weyl constants.           */
/* ------------------------------------------------------------------ */
static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k[0];
    const uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
}

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
        philox_round(c, k);
    }
    memcpy(out, c, sizeof c);
}

/* U[0,1) from the top 24 bits: exact in both float and double */
double or_uniform(uint32_t u) { return (double)(u >> 8) * (1.0 / 16777216.0); }

/* uniform number `idx` of stream `stream` for particle i, generation gen,
 * frame `frame`: block idx/4 of counter (i, stream<<16 | block, gen, frame) */
static double rand_u(uint64_t seed, uint32_t stream, uint32_t i, uint32_t gen,
                     uint32_t frame, uint32_t idx)
{
    const uint32_t ctr[4] = {i, (stream << 16) | (idx >> 2), gen, frame};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    or_philox4x32_10(ctr, key, out);
    return or_uniform(out[idx & 3]);
}

/* ------------------------------------------------------------------ */
/* small 3x3 helpers, row-major                                          */
/* ------------------------------------------------------------------ */
static void mat_mul(const double a[9], const double b[9], double c[9])
{
    double t[9];
    for (int r = 0; r < 3; ++r)
        for (int col = 0; col < 3; ++col)
            t[3 * r + col] = a[3 * r] * b[col] + a[3 * r + 1] * b[3 + col] + a[3 * r + 2] * b[6 + col];
    memcpy(c, t, sizeof t);
}
static void mat_vec(const double a[9], const double v[3], double o[3])
{
    double t[3];
    for (int r = 0; r < 3; ++r) t[r] = a[3 * r] * v[0] + a[3 * r + 1] * v[1] + a[3 * r + 2] * v[2];
    memcpy(o, t, sizeof t);
}
static void mat_tvec(const double a[9], const double v[3], double o[3]) /* a^T v */
{
    double t[3];
    for (int r = 0; r < 3; ++r) t[r] = a[r] * v[0] + a[3 + r] * v[1] + a[6 + r] * v[2];
    memcpy(o, t, sizeof t);
}
static void rot_x(double a, double m[9])
{
    const double c = cos(a), s = sin(a);
    double t[9] = {1, 0, 0, 0, c, -s, 0, s, c};
    memcpy(m, t, sizeof t);
}
static void rot_y(double a, double m[9])
{
    const double c = cos(a), s = sin(a);
    double t[9] = {c, 0, s, 0, 1, 0, -s, 0, c};
    memcpy(m, t, sizeof t);
}
static void rot_z(double a, double m[9])
{
    const double c = cos(a), s = sin(a);
    double t[9] = {c, -s, 0, s, c, 0, 0, 0, 1};
    memcpy(m, t, sizeof t);
}
/* Rz(z) Ry(y) Rx(x) */
static void rot_zyx(double x, double y, double z, double m[9])
{
    double a[9], b[9];
    rot_z(z, a);
    rot_y(y, b);
    mat_mul(a, b, a);
    rot_x(x, b);
    mat_mul(a, b, m);
}

/* ------------------------------------------------------------------ */
/* Forward kinematics (Eq. 1-3, Section II.A)                           */
/* ------------------------------------------------------------------ */
/* clamp the pose to the joint limits (Tables 1-2); returns 0, or -1 if any
 * entry is not finite (the pose is then left untouched) */
int or_clamp_pose(const double* pose, const double* lo, const double* hi, double* out)
{
    for (int d = 0; d < OR_NDOF; ++d)
        if (!isfinite(pose[d])) return -1;
    for (int d = 0; d < OR_NDOF; ++d) {
        double v = pose[d];
        if (v < lo[d]) v = lo[d];
        if (v > hi[d]) v = hi[d];
        out[d] = v;
    }
    return 0;
}

/* kc(h) = sum over the 3 adjacent non-thumb finger pairs of -min(phi, 0),
 * phi = abduction of the radial finger minus that of the ulnar finger (rad) */
double or_kc(const double* q)
{
    static const int mpz[4] = {11, 15, 19, 23}; /* index, middle, ring, pinky */
    double kc = 0.0;
    for (int p = 0; p < 3; ++p) {
        const double phi = q[mpz[p]] - q[mpz[p + 1]];
        kc += -fmin(phi, 0.0);
    }
    return kc;
}

/*
 * Bone frames in camera coordinates.  Root (palm): origin at the wrist
 * (x, y, z), rotation Mount * Rz(tz) Ry(ty) Rx(tx) with Mount = diag(1,-1,-1)
 * (fingers point to image-up and the palm faces the camera at zero angles).
 * Bone b > 0: parent * T(offset) * Rz Ry Rx(rest angles) * Rz(q[dof_z]) *
 * Rx(q[dof_x]).  bone_R is [nb][9] row-major (columns = bone axes in camera
 * coordinates), bone_p [nb][3].
 */
int or_bone_frames(int nb, const int32_t* bones_i, const double* bones_f, const double* q,
                   double* bone_R, double* bone_p)
{
    if (nb < 1 || nb > OR_MAXB) return -1;
    double a[9], b[9];
    const double mount[9] = {1, 0, 0, 0, -1, 0, 0, 0, -1};
    rot_zyx(q[3], q[4], q[5], a);
    mat_mul(mount, a, bone_R);
    bone_p[0] = q[0]; bone_p[1] = q[1]; bone_p[2] = q[2];
    for (int k = 1; k < nb; ++k) {
        const int parent = bones_i[3 * k], dz = bones_i[3 * k + 1], dx = bones_i[3 * k + 2];
        if (parent < 0 || parent >= k) return -1;
        const double* f = bones_f + 6 * k;
        const double* Rp = bone_R + 9 * parent;
        double off[3];
        mat_vec(Rp, f, off);
        for (int i = 0; i < 3; ++i) bone_p[3 * k + i] = bone_p[3 * parent + i] + off[i];
        rot_zyx(f[3], f[4], f[5], a);
        mat_mul(Rp, a, a);
        rot_z(dz >= 0 ? q[dz] : 0.0, b);
        mat_mul(a, b, a);
        rot_x(dx >= 0 ? q[dx] : 0.0, b);
        mat_mul(a, b, bone_R + 9 * k);
    }
    return 0;
}

/* Primitive frames in camera coordinates: rotation = bone rotation (the
 * primitives are axis-aligned with their bone), centre = bone_R c + bone_p. */
int or_prim_frames(int np_, const int32_t* prims_i, const double* prims_f, int nb,
                   const double* bone_R, const double* bone_p, double* prim_R, double* prim_C)
{
    for (int k = 0; k < np_; ++k) {
        const int b = prims_i[2 * k];
        if (b < 0 || b >= nb) return -1;
        double c[3];
        mat_vec(bone_R + 9 * b, prims_f + 7 * k, c);
        for (int i = 0; i < 3; ++i) prim_C[3 * k + i] = c[i] + bone_p[3 * b + i];
        memcpy(prim_R + 9 * k, bone_R + 9 * b, 9 * sizeof(double));
    }
    return 0;
}

/* full FK: clamp, bones, primitives, kc.  Returns -1 on a non-finite pose. */
int or_fk(int nb, const int32_t* bones_i, const double* bones_f, int np_, const int32_t* prims_i,
          const double* prims_f, const double* lo, const double* hi, const double* pose,
          double* q_out, double* bone_R, double* bone_p, double* prim_R, double* prim_C, double* kc)
{
    double q[OR_NDOF];
    if (or_clamp_pose(pose, lo, hi, q) != 0) return -1;
    if (or_bone_frames(nb, bones_i, bones_f, q, bone_R, bone_p) != 0) return -2;
    if (or_prim_frames(np_, prims_i, prims_f, nb, bone_R, bone_p, prim_R, prim_C) != 0) return -2;
    if (q_out) memcpy(q_out, q, sizeof q);
    *kc = or_kc(q);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Ray casting (depth map r_d, Section III.A)                           */
/* ------------------------------------------------------------------ */
/* Ray from the camera centre through direction d (d_z = 1), so the ray
 * parameter t equals the camera-z depth.  Each primitive is intersected in
 * its local frame: o = R^T (0 - C), e = R^T d.  Returns the smallest t > 0
 * and the surface id (0 = quadric side, 1 = cap at -hl, 2 = cap at +hl), or
 * t = +inf for a miss. */
#define OR_INF (1.0 / 0.0)

static void consider(double t, int surf, double* best, int* best_surf)
{
    if (t > 0.0 && t < *best) { *best = t; *best_surf = surf; }
}

double or_intersect(int kind, const double* dims, const double* R, const double* C,
                    const double d[3], int* surface)
{
    double negC[3] = {-C[0], -C[1], -C[2]}, o[3], e[3];
    mat_tvec(R, negC, o);
    mat_tvec(R, d, e);
    double best = OR_INF;
    int bs = -1;
    if (kind == 0) { /* ellipsoid x^2/sx^2 + y^2/sy^2 + z^2/sz^2 = 1 */
        double os[3], es[3];
        for (int i = 0; i < 3; ++i) { os[i] = o[i] / dims[i]; es[i] = e[i] / dims[i]; }
        const double A = es[0] * es[0] + es[1] * es[1] + es[2] * es[2];
        const double B = 2.0 * (os[0] * es[0] + os[1] * es[1] + os[2] * es[2]);
        const double Cq = os[0] * os[0] + os[1] * os[1] + os[2] * os[2] - 1.0;
        const double disc = B * B - 4.0 * A * Cq;
        if (disc >= 0.0) {
            const double sq = sqrt(disc);
            consider((-B - sq) / (2.0 * A), 0, &best, &bs);
            consider((-B + sq) / (2.0 * A), 0, &best, &bs);
        }
    } else { /* capped elliptic truncated cone along y:
              * (x/ax)^2 + (z/az)^2 = (1 + kappa y / hl)^2, |y| <= hl */
        const double ax = dims[0], az = dims[1], hl = dims[2], kap = dims[3];
        const double oX = o[0] / ax, eX = e[0] / ax, oZ = o[2] / az, eZ = e[2] / az;
        const double oW = 1.0 + kap * o[1] / hl, eW = kap * e[1] / hl;
        const double A = eX * eX + eZ * eZ - eW * eW;
        const double B = 2.0 * (oX * eX + oZ * eZ - oW * eW);
        const double Cq = oX * oX + oZ * oZ - oW * oW;
        double roots[2];
        int nr = 0;
        if (fabs(A) > 1e-300) {
            const double disc = B * B - 4.0 * A * Cq;
            if (disc >= 0.0) {
                const double sq = sqrt(disc);
                roots[nr++] = (-B - sq) / (2.0 * A);
                roots[nr++] = (-B + sq) / (2.0 * A);
            }
        } else if (B != 0.0) {
            roots[nr++] = -Cq / B;
        }
        for (int i = 0; i < nr; ++i) {
            const double y = o[1] + roots[i] * e[1];
            if (fabs(y) <= hl) consider(roots[i], 0, &best, &bs);
        }
        if (e[1] != 0.0) {
            for (int s = 0; s < 2; ++s) {
                const double yc = s == 0 ? -hl : hl;
                const double t = (yc - o[1]) / e[1];
                const double X = (o[0] + t * e[0]) / ax, Z = (o[2] + t * e[2]) / az;
                const double w = 1.0 + kap * (s == 0 ? -1.0 : 1.0);
                if (X * X + Z * Z <= w * w) consider(t, 1 + s, &best, &bs);
            }
        }
    }
    if (surface) *surface = bs;
    return best;
}

static void pixel_dir(double u, double v, const double cam[4], double d[3])
{
    d[0] = (u + 0.5 - cam[2]) / cam[0];
    d[1] = (v + 0.5 - cam[3]) / cam[1];
    d[2] = 1.0;
}

/* nearest hit over all primitives along direction d; returns t (inf = miss),
 * the primitive id and surface id, and the second-nearest distinct-primitive
 * hit (for depth-tie detection). */
static double nearest_hit(int np_, const int32_t* prims_i, const double* prims_f, const double* prim_R,
                          const double* prim_C, const double d[3], int* prim, int* surf, double* second)
{
    double best = OR_INF, sec = OR_INF;
    int bp = -1, bsf = -1;
    for (int k = 0; k < np_; ++k) {
        int s;
        const double t = or_intersect(prims_i[2 * k + 1], prims_f + 7 * k + 3, prim_R + 9 * k,
                                      prim_C + 3 * k, d, &s);
        if (t < best) { sec = best; best = t; bp = k; bsf = s; }
        else if (t < sec) sec = t;
    }
    if (prim) *prim = bp;
    if (surf) *surf = bsf;
    if (second) *second = sec;
    return best;
}

/*
 * Render one hypothesis: depth [H][W] (camera z in mm, 0 where nothing is hit),
 * hit [H][W], and optionally prim id [H][W] and a boundary flag [H][W].
 * cam = (fx, fy, cx, cy).  A pixel is flagged as boundary when the outcome
 * (hit / primitive / surface) changes for a ray jittered by `jitter` pixels in
 * any of 8 directions, or when the two nearest hits of different primitives
 * lie within `tie_mm`.
 */
void or_render(int np_, const int32_t* prims_i, const double* prims_f, const double* prim_R,
               const double* prim_C, const double cam[4], int W, int H, double* depth, uint8_t* hit,
               int32_t* prim_id, uint8_t* boundary, double jitter, double tie_mm)
{
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            double d[3], sec;
            int pk, sf;
            pixel_dir(u, v, cam, d);
            const double t = nearest_hit(np_, prims_i, prims_f, prim_R, prim_C, d, &pk, &sf, &sec);
            const int h = t < OR_INF;
            depth[v * W + u] = h ? t : 0.0;
            hit[v * W + u] = (uint8_t)h;
            if (prim_id) prim_id[v * W + u] = h ? pk : -1;
            if (boundary) {
                int b = h && sec - t < tie_mm;
                static const int dir[8][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1},
                                              {1, 1}, {1, -1}, {-1, 1}, {-1, -1}};
                for (int j = 0; j < 8 && !b; ++j) {
                    double dj[3];
                    int pj, sj;
                    pixel_dir(u + jitter * dir[j][0], v + jitter * dir[j][1], cam, dj);
                    const double tj = nearest_hit(np_, prims_i, prims_f, prim_R, prim_C, dj, &pj, &sj, NULL);
                    const int hj = tj < OR_INF;
                    if (hj != h || (h && (pj != pk || sj != sf))) b = 1;
                }
                boundary[v * W + u] = (uint8_t)b;
            }
        }
}

/* ------------------------------------------------------------------ */
/* Cost (Section III.A, Eq. 4-5)                                        */
/* ------------------------------------------------------------------ */
/*
 * Per pixel, with S = skin mask, Od = observed depth (0 = hole / undefined):
 *   valid = S and Od > 0
 *   r_m   = hit and (not valid or |Z - Od| < d_m)
 *   t     = hit and valid     -> min(|Od - Z|, d_M)
 *           hit and S, Od = 0 -> 0        (undefined depth: unknown)
 *           hit and not S     -> d_M
 *           no hit and valid  -> d_M
 *           otherwise         -> 0
 * sums[0] = sum t, sums[1] = sum (S and r_m), sums[2] = sum (S or r_m),
 * D = sums[0]/sums[2] + lambda (1 - 2 sums[1] / (sums[1] + sums[2])),
 * and D = lambda when the union is empty.  rm_out (optional) gets r_m.
 * params = (d_m, d_M, lambda, lambda_k).
 */
double or_cost(int W, int H, const double* depth, const uint8_t* hit, const double* Od,
               const uint8_t* S, const double params[4], double sums[3], uint8_t* rm_out)
{
    const double dm = params[0], dM = params[1], lam = params[2];
    double st = 0.0, sa = 0.0, so = 0.0;
    for (int i = 0; i < W * H; ++i) {
        const int s = S[i] != 0, h = hit[i] != 0;
        const int valid = s && Od[i] > 0.0;
        const double diff = fabs(Od[i] - depth[i]);
        const int rm = h && (!valid || diff < dm);
        double t;
        if (h && valid) t = fmin(diff, dM);
        else if (h && s) t = 0.0;
        else if (h) t = dM;
        else if (valid) t = dM;
        else t = 0.0;
        st += t;
        sa += (s && rm);
        so += (s || rm);
        if (rm_out) rm_out[i] = (uint8_t)rm;
    }
    sums[0] = st; sums[1] = sa; sums[2] = so;
    if (so == 0.0) return lam;
    return st / so + lam * (1.0 - 2.0 * sa / (sa + so));
}

/*
 * Score P hypotheses: FK, render, Eq. 4-5.  poses [P][26]; outputs E [P],
 * D [P], kc [P], sums [P][3]; optional per-pixel depth/hit/rm/boundary
 * [P][H][W] (NULL to skip).  E is NaN for a non-finite pose.
 */
void or_score_batch(int P, const double* poses, int nb, const int32_t* bones_i, const double* bones_f,
                    int np_, const int32_t* prims_i, const double* prims_f, const double* lo,
                    const double* hi, const double cam[4], int W, int H, const double* Od,
                    const uint8_t* S, const double params[4], double* E, double* D, double* kc,
                    double* sums, double* depth_out, uint8_t* hit_out, uint8_t* rm_out,
                    uint8_t* boundary_out, double jitter, double tie_mm)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < P; ++p) {
        double bR[OR_MAXB * 9], bp[OR_MAXB * 3], pR[OR_MAXP * 9], pC[OR_MAXP * 3], k, s3[3];
        const size_t n = (size_t)W * H;
        double* depth = depth_out ? depth_out + p * n : (double*)malloc(n * sizeof(double));
        uint8_t* hit = hit_out ? hit_out + p * n : (uint8_t*)malloc(n);
        if (np_ > OR_MAXP || or_fk(nb, bones_i, bones_f, np_, prims_i, prims_f, lo, hi, poses + 26 * p,
                                   NULL, bR, bp, pR, pC, &k) != 0) {
            E[p] = D[p] = kc[p] = NAN;
            sums[3 * p] = sums[3 * p + 1] = sums[3 * p + 2] = NAN;
        } else {
            or_render(np_, prims_i, prims_f, pR, pC, cam, W, H, depth, hit, NULL,
                      boundary_out ? boundary_out + p * n : NULL, jitter, tie_mm);
            D[p] = or_cost(W, H, depth, hit, Od, S, params, s3, rm_out ? rm_out + p * n : NULL);
            kc[p] = k;
            E[p] = D[p] + params[3] * k;
            memcpy(sums + 3 * p, s3, sizeof s3);
        }
        if (!depth_out) free(depth);
        if (!hit_out) free(hit);
    }
}

/* ------------------------------------------------------------------ */
/* Particle swarm (Section III.B, Eq. 6-7)                              */
/* ------------------------------------------------------------------ */
/* constriction factor w = 2 / |2 - psi - sqrt(psi^2 - 4 psi)|, psi = c1 + c2 */
double or_pso_w(double c1, double c2)
{
    const double psi = c1 + c2;
    return 2.0 / fabs(2.0 - psi - sqrt(psi * psi - 4.0 * psi));
}

/* Eq. 6-7 for one particle with explicit r1, r2 [26]; x is clamped to the
 * limits after Eq. 7, the velocity is kept. */
void or_pso_update(const double* x, const double* v, const double* pbest, const double* gbest,
                   const double* r1, const double* r2, double c1, double c2, double w,
                   const double* lo, const double* hi, double* x_out, double* v_out)
{
    for (int d = 0; d < OR_NDOF; ++d) {
        const double vn = w * (v[d] + c1 * r1[d] * (pbest[d] - x[d]) + c2 * r2[d] * (gbest[d] - x[d]));
        double xn = x[d] + vn;
        if (xn < lo[d]) xn = lo[d];
        if (xn > hi[d]) xn = hi[d];
        v_out[d] = vn;
        x_out[d] = xn;
    }
}

/* rank key: NaN sorts last */
static int worse_than(double ea, int ia, double eb, int ib)
{
    const int na = isnan(ea), nb_ = isnan(eb);
    if (na != nb_) return na;
    if (!na && ea != eb) return ea > eb;
    return ia > ib;
}

/*
 * One generation after the evaluation of x (E [P] = objective of x):
 *  1. pbest_i <- x_i where E_i < pbestE_i (strict);
 *  2. gbest <- pbest of argmin pbestE (lowest index on ties);
 *  3. Eq. 6-7 for every particle, r1 = uniform 2d, r2 = uniform 2d+1 of
 *     stream 1, then clamp;
 *  4. if mutate_every > 0 and gen % mutate_every == 0: the n_mutate particles
 *     with the largest E (ties: larger index is worse, NaN worst) re-draw their
 *     20 finger dims (6..25) uniformly within the limits (stream 2, number
 *     d - 6) and zero their velocity there.
 * Arrays are updated in place.  gbest_E is a scalar.
 */
void or_pso_step(int P, double* x, double* v, double* pbest, double* pbest_E, double* gbest,
                 double* gbest_E, const double* E, const double* lo, const double* hi, double c1,
                 double c2, uint64_t seed, uint32_t frame, uint32_t gen, int mutate_every,
                 int n_mutate)
{
    const double w = or_pso_w(c1, c2);
    for (int i = 0; i < P; ++i)
        if (E[i] < pbest_E[i]) {
            pbest_E[i] = E[i];
            memcpy(pbest + 26 * i, x + 26 * i, 26 * sizeof(double));
        }
    int g = 0;
    for (int i = 1; i < P; ++i)
        if (pbest_E[i] < pbest_E[g]) g = i;
    memcpy(gbest, pbest + 26 * g, 26 * sizeof(double));
    *gbest_E = pbest_E[g];
    for (int i = 0; i < P; ++i) {
        double r1[26], r2[26];
        for (int d = 0; d < 26; ++d) {
            r1[d] = rand_u(seed, 1, (uint32_t)i, gen, frame, (uint32_t)(2 * d));
            r2[d] = rand_u(seed, 1, (uint32_t)i, gen, frame, (uint32_t)(2 * d + 1));
        }
        or_pso_update(x + 26 * i, v + 26 * i, pbest + 26 * i, gbest, r1, r2, c1, c2, w, lo, hi,
                      x + 26 * i, v + 26 * i);
    }
    if (mutate_every > 0 && gen % (uint32_t)mutate_every == 0) {
        for (int i = 0; i < P; ++i) {
            int rank = 0; /* number of particles better than i */
            for (int j = 0; j < P; ++j)
                if (j != i && worse_than(E[i], i, E[j], j)) ++rank;
            if (rank >= P - n_mutate) {
                for (int d = 6; d < 26; ++d) {
                    const double u = rand_u(seed, 2, (uint32_t)i, gen, frame, (uint32_t)(d - 6));
                    x[26 * i + d] = lo[d] + u * (hi[d] - lo[d]);
                    v[26 * i + d] = 0.0;
                }
            }
        }
    }
}

/*
 * Tracking initialisation (Section III.B: random positions, zero velocity):
 * particle 0 is the clamped seed pose; particle i > 0 is the seed pose plus
 * (2u - 1) * scale[d] with u = uniform d of stream 3, then clamped.  pbest = x,
 * pbest_E = +inf, gbest = particle 0, gbest_E = +inf.
 */
void or_pso_init(int P, const double* seed_pose, const double* scale, const double* lo,
                 const double* hi, uint64_t seed, uint32_t frame, double* x, double* v, double* pbest,
                 double* pbest_E, double* gbest, double* gbest_E)
{
    for (int i = 0; i < P; ++i) {
        for (int d = 0; d < 26; ++d) {
            double xv = seed_pose[d];
            if (i > 0) xv += (2.0 * rand_u(seed, 3, (uint32_t)i, 0, frame, (uint32_t)d) - 1.0) * scale[d];
            if (xv < lo[d]) xv = lo[d];
            if (xv > hi[d]) xv = hi[d];
            x[26 * i + d] = xv;
            v[26 * i + d] = 0.0;
            pbest[26 * i + d] = xv;
        }
        pbest_E[i] = OR_INF;
    }
    memcpy(gbest, x, 26 * sizeof(double));
    *gbest_E = OR_INF;
}

/* mean |angle error| in degrees over the 23 angular DOFs (wrist angles and
 * the 20 finger angles) */
double or_mean_joint_error_deg(const double* a, const double* b)
{
    double s = 0.0;
    for (int d = 3; d < 26; ++d) s += fabs(a[d] - b[d]);
    return s / 23.0 * 180.0 / M_PI;
}
