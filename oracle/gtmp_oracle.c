/*
 * CPU oracle for the layered-graph planner of "Anytime Global Tensor Motion
 * Planning" (GTMP with a straight-line local planner).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so, which
 * only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * load.  The CUDA library never links, calls or reads anything here, and this
 * file includes none of the CUDA sources: the two sides share no code.
 *
 * Precision: FP64 for everything the paper leaves in real arithmetic
 * (forward kinematics, distances, margins, edge costs).  The quantities that
 * the method *defines* through a floating-point formula and that decide an
 * integer (which sample is drawn, which waypoint configuration is checked,
 * whether a rejection-sampling attempt is accepted, which neighbour is the
 * nearest) are computed in FP32 with a stated operation order, because both
 * sides must take those decisions identically.  Build with
 * -ffp-contract=off so that the compiler fuses nothing behind our back.
 *
 * Citations are to the paper's sections, equations and algorithm.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <omp.h>

#define ORC_FREE 0
#define ORC_COLLIDE 1
#define ORC_AMBIGUOUS 2

#define TAG_UNIFORM 1u
#define TAG_INFORMED 2u
#define TAG_COIN 3u
#define TAG_FREE 5u

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,        */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of      */
/* two 32x32->64 multiplies with a Weyl-sequence key schedule.               */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    const uint32_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += weyl0;
            k1 += weyl1;
        }
        uint64_t p0 = (uint64_t)mul0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)mul1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* Philox word -> uniform float in [0, 1): the top 24 bits times 2^-24 (exact). */
static float word_to_unit(uint32_t w) { return (float)(w >> 8) * 0x1p-24f; }

static void philox_block(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                         uint32_t out[4]) {
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* Uniform layer sampling, Alg. 1 ("uniformly sample Q", gtmp) and the      */
/* layered sampling model of Sec. III-A: Q[r][l][i][k] is drawn from the     */
/* joint box with x = fma(u, hi_k - lo_k, lo_k) in FP32, u from word k&3 of  */
/* Philox block (i, l, r, TAG_UNIFORM<<24 | k>>2).                           */
/* ------------------------------------------------------------------------ */
void orc_sample_uniform(uint64_t seed, uint32_t restart, int L, int M, int dof,
                        const float* lo, const float* hi, float* Q /* [L][M][dof] */) {
    for (int l = 0; l < L; ++l)
        for (int i = 0; i < M; ++i)
            for (int k = 0; k < dof; ++k) {
                uint32_t w[4];
                philox_block(seed, (uint32_t)i, (uint32_t)l, restart, (TAG_UNIFORM << 24) | (uint32_t)(k >> 2), w);
                float u = word_to_unit(w[k & 3]);
                float width = hi[k] - lo[k];
                Q[((size_t)l * M + i) * dof + k] = fmaf(u, width, lo[k]);
            }
}

/* ------------------------------------------------------------------------ */
/* Scene: robot (point or DH serial arm with link spheres) and obstacles.   */
/* The free space C_free of Sec. III is the set of configurations whose     */
/* robot spheres overlap no obstacle.                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t kind;        /* 0 = point robot, 1 = DH serial arm */
    int32_t dof;
    const double* dh;    /* [dof][4]: d, a, alpha, theta offset */
    int32_t spl;         /* spheres per link */
    const double* link_sph; /* [dof][spl][4]: x, y, z, r in the link frame */
    double point_radius;
    int32_t n_s;
    const double* spheres; /* [n_s][4] */
    int32_t n_b;
    const double* boxes; /* [n_b][6]: lo xyz, hi xyz */
} orc_scene;

int orc_num_robot_spheres(const orc_scene* sc) { return sc->kind == 0 ? 1 : sc->dof * sc->spl; }

/* Forward kinematics: world centres and radii of all robot spheres.
 * Standard DH link transform A_i = Rz(q_i + theta_i) Tz(d_i) Tx(a_i) Rx(alpha_i),
 * chained from the base frame (the identity at the origin). */
void orc_fk_spheres(const orc_scene* sc, const double* q, double* out /* [S][4] */) {
    if (sc->kind == 0) {
        out[0] = q[0];
        out[1] = sc->dof > 1 ? q[1] : 0.0;
        out[2] = sc->dof > 2 ? q[2] : 0.0;
        out[3] = sc->point_radius;
        return;
    }
    double R[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    double t[3] = {0, 0, 0};
    for (int i = 0; i < sc->dof; ++i) {
        const double d = sc->dh[i * 4 + 0], a = sc->dh[i * 4 + 1];
        const double al = sc->dh[i * 4 + 2], th = q[i] + sc->dh[i * 4 + 3];
        const double ct = cos(th), st = sin(th), ca = cos(al), sa = sin(al);
        const double A[3][3] = {{ct, -st * ca, st * sa}, {st, ct * ca, -ct * sa}, {0.0, sa, ca}};
        const double p[3] = {a * ct, a * st, d};
        double tn[3], Rn[3][3];
        for (int r = 0; r < 3; ++r) {
            tn[r] = t[r] + R[r][0] * p[0] + R[r][1] * p[1] + R[r][2] * p[2];
            for (int c = 0; c < 3; ++c) Rn[r][c] = R[r][0] * A[0][c] + R[r][1] * A[1][c] + R[r][2] * A[2][c];
        }
        memcpy(t, tn, sizeof t);
        memcpy(R, Rn, sizeof R);
        for (int s = 0; s < sc->spl; ++s) {
            const double* ls = sc->link_sph + ((size_t)i * sc->spl + s) * 4;
            double* o = out + ((size_t)i * sc->spl + s) * 4;
            for (int r = 0; r < 3; ++r) o[r] = R[r][0] * ls[0] + R[r][1] * ls[1] + R[r][2] * ls[2] + t[r];
            o[3] = ls[3];
        }
    }
}

/* Signed distance from point c to an axis-aligned box (negative inside). */
static double box_signed_distance(const double* c, const double* box) {
    double e[3], outside2 = 0.0, emax = -INFINITY;
    for (int k = 0; k < 3; ++k) {
        double below = box[k] - c[k], above = c[k] - box[3 + k];
        e[k] = below > above ? below : above;
        if (e[k] > emax) emax = e[k];
        if (e[k] > 0.0) outside2 += e[k] * e[k];
    }
    if (emax <= 0.0) return emax;
    return sqrt(outside2);
}

/* Clearance of one configuration: min over (robot sphere, obstacle) of
 * signed distance minus radii.  Negative means the configuration is in
 * C_coll.  Returns +inf for an empty scene. */
double orc_config_margin(const orc_scene* sc, const double* q) {
    double cs[16 * 64 * 4];
    const int S = orc_num_robot_spheres(sc);
    orc_fk_spheres(sc, q, cs);
    double m = INFINITY;
    for (int s = 0; s < S; ++s) {
        const double* c = cs + 4 * s;
        for (int o = 0; o < sc->n_s; ++o) {
            const double* ob = sc->spheres + 4 * o;
            double dx = c[0] - ob[0], dy = c[1] - ob[1], dz = c[2] - ob[2];
            double v = sqrt(dx * dx + dy * dy + dz * dz) - ob[3] - c[3];
            if (v < m) m = v;
        }
        for (int o = 0; o < sc->n_b; ++o) {
            double v = box_signed_distance(c, sc->boxes + 6 * o) - c[3];
            if (v < m) m = v;
        }
    }
    return m;
}

static int label_of_margin(double m, double eps) {
    if (m < -eps) return ORC_COLLIDE;
    if (m <= eps) return ORC_AMBIGUOUS;
    return ORC_FREE;
}

void orc_config_labels(const orc_scene* sc, int n, const float* q, double eps, int8_t* labels,
                       double* margins) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) {
        double qd[64];
        for (int k = 0; k < sc->dof; ++k) qd[k] = (double)q[(size_t)i * sc->dof + k];
        double m = orc_config_margin(sc, qd);
        if (margins) margins[i] = m;
        labels[i] = (int8_t)label_of_margin(m, eps);
    }
}

/* ------------------------------------------------------------------------ */
/* Layer sampling on C_free (Sec. III: pi_m is a measure on C_m and C_free)  */
/* by rejection.  Sample (r, l, i), attempt a: attempt 0 is the uniform       */
/* sample of orc_sample_uniform; attempt a >= 1 takes word k & 3 of Philox    */
/* block (i, l, r, TAG_FREE<<24 | a<<2 | k>>2).  The first attempt whose      */
/* label is free is kept; if none of max_attempts is, the last one is kept    */
/* (its edges then collide through their endpoint).  used[] = the accepted    */
/* attempt or -1; undecided[] = 1 when an attempt before the accepted one     */
/* lay in the +-eps band (a float32 checker may decide it either way).        */
/* ------------------------------------------------------------------------ */
void orc_sample_free(const orc_scene* sc, uint64_t seed, uint32_t restart, int L, int M, const float* lo,
                     const float* hi, double eps, int max_attempts, float* Q, int32_t* used, int8_t* undecided) {
    const int dof = sc->dof;
#pragma omp parallel for schedule(dynamic, 8)
    for (int t = 0; t < L * M; ++t) {
        const int l = t / M, i = t % M;
        float* q = Q + (size_t)t * dof;
        double qd[64];
        int acc = -1;
        int8_t und = 0;
        for (int a = 0; a < max_attempts && acc < 0; ++a) {
            for (int k = 0; k < dof; ++k) {
                uint32_t w[4];
                const uint32_t word3 = a == 0 ? (TAG_UNIFORM << 24) | (uint32_t)(k >> 2)
                                              : (TAG_FREE << 24) | ((uint32_t)a << 2) | (uint32_t)(k >> 2);
                philox_block(seed, (uint32_t)i, (uint32_t)l, restart, word3, w);
                q[k] = fmaf(word_to_unit(w[k & 3]), hi[k] - lo[k], lo[k]);
                qd[k] = (double)q[k];
            }
            const int lab = label_of_margin(orc_config_margin(sc, qd), eps);
            if (lab == ORC_FREE) acc = a;
            else if (lab == ORC_AMBIGUOUS) und = 1;
        }
        used[t] = acc;
        undecided[t] = und;
    }
}

/* ------------------------------------------------------------------------ */
/* Straight-line local planner (SEV, Sec. VI; LP contract of Sec. III-B):    */
/* the segment u -> v is checked at H waypoints t_k = k/(H-1), k = 0..H-1.   */
/* Waypoint k is u for k = 0, v for k = H-1, else the FP32 configuration     */
/* fma(t_k, v - u, u) with t_k = (float)k / (float)(H-1).  Edge label:       */
/* collide if any waypoint collides, else ambiguous if any waypoint lies in  */
/* the +-eps band, else free.  Edge cost = ||v - u||_2 (path length, Sec.    */
/* IV-A), absent (collide) when it exceeds the edge-length limit.            */
/* ------------------------------------------------------------------------ */
int orc_edge_label(const orc_scene* sc, const float* u, const float* v, int H, double eps) {
    const int dof = sc->dof;
    int label = ORC_FREE;
    double q[64];
    for (int k = 0; k < H; ++k) {
        if (k == 0) {
            for (int d = 0; d < dof; ++d) q[d] = (double)u[d];
        } else if (k == H - 1) {
            for (int d = 0; d < dof; ++d) q[d] = (double)v[d];
        } else {
            const float t = (float)k / (float)(H - 1);
            for (int d = 0; d < dof; ++d) q[d] = (double)fmaf(t, v[d] - u[d], u[d]);
        }
        int w = label_of_margin(orc_config_margin(sc, q), eps);
        if (w == ORC_COLLIDE) return ORC_COLLIDE; /* the label can only stay "collide" */
        if (w == ORC_AMBIGUOUS) label = ORC_AMBIGUOUS;
    }
    return label;
}

double orc_edge_length(int dof, const float* u, const float* v) {
    double s = 0.0;
    for (int d = 0; d < dof; ++d) {
        double e = (double)v[d] - (double)u[d];
        s += e * e;
    }
    return sqrt(s);
}

/* ------------------------------------------------------------------------ */
/* Weighted length (App. "General Costs": any additive cost that dominates  */
/* length and is Lipschitz; a weighted length with 1 <= w <= W is the       */
/* example).  Weight field: w(q) = 1 + sum_b a_b max(0, 1 - |q - c_b|^2 /   */
/* s_b^2), bump b given as [c_b (dof values), s_b, a_b], a_b >= 0.  The     */
/* edge cost is the integral of w along the straight edge, taken by the     */
/* trapezoid rule on the planner's own H waypoints (the same float32        */
/* configurations that are collision-checked):                              */
/*   cost = |v - u| / (H - 1) * (w_0 / 2 + w_1 + ... + w_{H-2} + w_{H-1} / 2) */
/* With no bump (K = 0) the cost is the length itself.                      */
/* ------------------------------------------------------------------------ */
double orc_weight(int dof, const double* q, const double* bumps, int K) {
    double w = 1.0;
    for (int b = 0; b < K; ++b) {
        const double* c = bumps + (size_t)b * (dof + 2);
        double d2 = 0.0;
        for (int d = 0; d < dof; ++d) d2 += (q[d] - c[d]) * (q[d] - c[d]);
        const double s = c[dof], a = c[dof + 1];
        const double u = 1.0 - d2 / (s * s);
        if (u > 0.0) w += a * u;
    }
    return w;
}

double orc_weighted_length(int dof, const float* u, const float* v, int H, const double* bumps, int K) {
    const double len = orc_edge_length(dof, u, v);
    if (K == 0) return len;
    double q[64], sum = 0.0;
    for (int k = 0; k < H; ++k) {
        if (k == 0) {
            for (int d = 0; d < dof; ++d) q[d] = (double)u[d];
        } else if (k == H - 1) {
            for (int d = 0; d < dof; ++d) q[d] = (double)v[d];
        } else {
            const float t = (float)k / (float)(H - 1);
            for (int d = 0; d < dof; ++d) q[d] = (double)fmaf(t, v[d] - u[d], u[d]);
        }
        const double w = orc_weight(dof, q, bumps, K);
        sum += (k == 0 || k == H - 1) ? 0.5 * w : w;
    }
    return len * sum / (double)(H - 1);
}

/* All edges between vertex set A (na rows) and vertex set B (nb rows); the */
/* edge-length limit applies to the length, the cost is the weighted length */
/* (the length itself when K = 0).                                          */
void orc_edge_block(const orc_scene* sc, const float* A, int na, const float* B, int nb, int H,
                    double eps, double max_len, const double* bumps, int K, int8_t* labels /* [na][nb] */,
                    double* costs /* [na][nb] */) {
    const int dof = sc->dof;
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int a = 0; a < na; ++a)
        for (int b = 0; b < nb; ++b) {
            const float* u = A + (size_t)a * dof;
            const float* v = B + (size_t)b * dof;
            const size_t e = (size_t)a * nb + b;
            const double len = orc_edge_length(dof, u, v);
            costs[e] = K > 0 ? orc_weighted_length(dof, u, v, H, bumps, K) : len;
            if (len > max_len) {
                labels[e] = ORC_COLLIDE;
                continue;
            }
            labels[e] = (int8_t)orc_edge_label(sc, u, v, H, eps);
        }
}

/* Per-waypoint margins of one edge (for dense re-checks of returned paths). */
void orc_edge_margins(const orc_scene* sc, const float* u, const float* v, int H, double* margins) {
    const int dof = sc->dof;
    double q[64];
    for (int k = 0; k < H; ++k) {
        if (k == 0) {
            for (int d = 0; d < dof; ++d) q[d] = (double)u[d];
        } else if (k == H - 1) {
            for (int d = 0; d < dof; ++d) q[d] = (double)v[d];
        } else {
            const float t = (float)k / (float)(H - 1);
            for (int d = 0; d < dof; ++d) q[d] = (double)fmaf(t, v[d] - u[d], u[d]);
        }
        margins[k] = orc_config_margin(sc, q);
    }
}

/* ------------------------------------------------------------------------ */
/* Informed set X_f(c) = {x : ||x - q0|| + ||x - qg|| <= c} (Sec. IV-D): a   */
/* prolate hyperspheroid with foci q0, qg, semi-major axis c/2 along         */
/* a = (qg - q0)/c_min and semi-minor axes sqrt(c^2 - c_min^2)/2.  A uniform */
/* point of the unit ball z maps to x = centre + r2 z + (r1 - r2)(a.z) a.    */
/* The unit-ball point is drawn by rejection from the cube [-1, 1]^d and the */
/* image is rejected outside the joint box, so accepted points are uniform   */
/* in X_f(c) intersected with the box.  All steps FP32, in this order.       */
/* ------------------------------------------------------------------------ */
typedef struct {
    float centre[64];
    float axis[64];
    float r1, r2, cmin;
} orc_ellipsoid;

void orc_informed_params(int dof, const float* q0, const float* qg, float c, orc_ellipsoid* e) {
    float s = 0.0f;
    for (int k = 0; k < dof; ++k) {
        float dq = qg[k] - q0[k];
        s = fmaf(dq, dq, s);
    }
    e->cmin = sqrtf(s);
    for (int k = 0; k < dof; ++k) {
        float sum = q0[k] + qg[k];
        e->centre[k] = 0.5f * sum;
        if (e->cmin > 0.0f) {
            float dq = qg[k] - q0[k];
            e->axis[k] = dq / e->cmin;
        } else {
            e->axis[k] = (k == 0) ? 1.0f : 0.0f;
        }
    }
    e->r1 = 0.5f * c;
    float cc = c * c;
    float mm = e->cmin * e->cmin;
    float diff = cc - mm;
    if (diff < 0.0f) diff = 0.0f;
    e->r2 = 0.5f * sqrtf(diff);
}

/* One attempt of the informed sampler; returns 1 if accepted. */
int orc_informed_attempt(uint64_t seed, uint32_t i, uint32_t l, uint32_t attempt, int dof,
                         const orc_ellipsoid* e, const float* lo, const float* hi, float* x) {
    float z[64];
    uint32_t w[4];
    for (int k = 0; k < dof; ++k) {
        if ((k & 3) == 0) philox_block(seed, i, l, attempt, (TAG_INFORMED << 24) | (uint32_t)(k >> 2), w);
        float u = word_to_unit(w[k & 3]);
        z[k] = 2.0f * u - 1.0f;
    }
    float ss = 0.0f;
    for (int k = 0; k < dof; ++k) ss = fmaf(z[k], z[k], ss);
    if (!(ss <= 1.0f)) return 0;
    float dot = 0.0f;
    for (int k = 0; k < dof; ++k) dot = fmaf(e->axis[k], z[k], dot);
    float rdiff = e->r1 - e->r2;
    float coef = rdiff * dot;
    int inside = 1;
    for (int k = 0; k < dof; ++k) {
        x[k] = fmaf(coef, e->axis[k], fmaf(e->r2, z[k], e->centre[k]));
        if (!(x[k] >= lo[k] && x[k] <= hi[k])) inside = 0;
    }
    return inside;
}

/* ------------------------------------------------------------------------ */
/* expand-samples of Alg. 1 (AO-GTMP, Sec. IV-D).  Every layer l = 1..L is   */
/* topped up from M_old to M_new samples; new slot i of layer l is:          */
/*  - uniform in the joint box (the plain stream with restart 0) when        */
/*    c_best = +inf;                                                          */
/*  - else uniform in X_f(c_best) (informed sampler above) when the layer    */
/*    had no samples yet or the fair coin says so;                            */
/*  - else the midpoint 0.5 (u + v) of u = layer l-1 sample number           */
/*    (coin word 1 mod |layer l-1|) and its nearest layer l+1 sample v       */
/*    (FP32 squared distance, first index on ties).  Layer 0 is {q0} and      */
/*    layer L+1 is {qg}.                                                      */
/* The coin is bit 0 of word 0 of Philox block (i, l-1, 0, TAG_COIN<<24).    */
/* All new samples of one call see only the M_old samples present on entry. */
/* Returns 0, or -1 when an informed draw used up max_attempts.              */
/* ------------------------------------------------------------------------ */
int orc_expand_layers(uint64_t seed, int L, int M_old, int M_new, int dof, const float* lo,
                      const float* hi, const float* q0, const float* qg, float c_best,
                      int max_attempts, float* Q /* [L][M_new][dof] */) {
    orc_ellipsoid e;
    const int finite = isfinite(c_best);
    if (finite) orc_informed_params(dof, q0, qg, c_best, &e);
    int status = 0;
    for (int l = 0; l < L; ++l) {
        for (int i = M_old; i < M_new; ++i) {
            float* x = Q + ((size_t)l * M_new + i) * dof;
            if (!finite) {
                for (int k = 0; k < dof; ++k) {
                    uint32_t w[4];
                    philox_block(seed, (uint32_t)i, (uint32_t)l, 0u, (TAG_UNIFORM << 24) | (uint32_t)(k >> 2), w);
                    float width = hi[k] - lo[k];
                    x[k] = fmaf(word_to_unit(w[k & 3]), width, lo[k]);
                }
                continue;
            }
            uint32_t cw[4];
            philox_block(seed, (uint32_t)i, (uint32_t)l, 0u, TAG_COIN << 24, cw);
            const int heuristic = (cw[0] & 1u) != 0u;
            const int n_prev = (l == 0) ? 1 : M_old;
            const int n_next = (l == L - 1) ? 1 : M_old;
            if (!heuristic || n_prev == 0 || n_next == 0) {
                int ok = 0;
                for (int a = 0; a < max_attempts && !ok; ++a)
                    ok = orc_informed_attempt(seed, (uint32_t)i, (uint32_t)l, (uint32_t)a, dof, &e, lo, hi, x);
                if (!ok) {
                    status = -1;
                    for (int k = 0; k < dof; ++k) x[k] = NAN;
                }
                continue;
            }
            const uint32_t pick = cw[1] % (uint32_t)n_prev;
            const float* u = (l == 0) ? q0 : Q + ((size_t)(l - 1) * M_new + pick) * dof;
            const float* v = qg;
            if (l != L - 1) {
                float best = INFINITY;
                int bi = 0;
                for (int j = 0; j < n_next; ++j) {
                    const float* c = Q + ((size_t)(l + 1) * M_new + j) * dof;
                    float d2 = 0.0f;
                    for (int k = 0; k < dof; ++k) {
                        float dd = c[k] - u[k];
                        d2 = fmaf(dd, dd, d2);
                    }
                    if (d2 < best) {
                        best = d2;
                        bi = j;
                    }
                }
                v = Q + ((size_t)(l + 1) * M_new + bi) * dof;
            }
            for (int k = 0; k < dof; ++k) {
                float sum = u[k] + v[k];
                x[k] = 0.5f * sum;
            }
        }
    }
    return status;
}

/* Thread count of the OpenMP loops above (the timing of the CPU baseline at
 * one thread and at all threads); returns the count now in effect. */
int orc_set_threads(int n) {
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
}
