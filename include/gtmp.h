/*
 * gtmp.h — C ABI of a B300 (sm_103a) planner for Global Tensor Motion Planning
 * with the straight-line local planner, and its anytime policies.
 *
 * Paper: "Anytime Global Tensor Motion Planning" (Coumar, Le, Kingston).
 * The planning problem (Sec. III): configuration space C ⊆ R^d (here a joint
 * box), free space C_free (configurations whose robot spheres overlap no
 * obstacle), start q0 and goal qg.  The layered graph (Sec. III-A): layers
 * V_0 = {q0}, V_1..V_L of M sampled configurations each, V_{L+1} = {qg}; every
 * pair of vertices in adjacent layers is a candidate edge.  The local planner
 * (Sec. III-B; "SEV" of Sec. VI) realises edge (u, v) as the straight segment,
 * checked at H waypoints t_k = k/(H-1), k = 0..H-1; a realised edge costs its
 * length ||v - u|| (Sec. IV-A), an unrealised one +inf.  The graph search
 * (Sec. IV-B, Alg. 1 gtmp) is the backward value iteration
 *     J_{L+1}(qg) = 0,   J_l(u) = min_v c(u, v) + J_{l+1}(v)
 * and the path is obtained by following the minimisers from q0.
 * Anytime-GTMP (Sec. IV-C, Alg. 1 anytime-gtmp) repeats gtmp with fresh
 * samples; AO-GTMP (Sec. IV-D, Alg. 1 ao-gtmp / expand-samples) grows the
 * layers with informed and heuristic samples.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every function returns a gtmp_status; nothing throws across the ABI.
 *    On failure gtmp_last_error(ctx) holds a one-line message.
 *  - "host" pointers are read during the call and may be freed afterwards.
 *    "device" pointers are CUDA device memory owned by the caller; they must
 *    stay valid until the work enqueued by the call has completed.
 *  - All GPU work is enqueued on the context's stream (asynchronous); results
 *    in device buffers are valid after that stream has been synchronised
 *    (gtmp_synchronize does that and reports device-side error flags).
 *  - Floating-point data are IEEE float32, indices int32, row-major.
 *  - A context is not thread-safe; independent contexts may be used from
 *    different threads on different streams.
 *  - An infeasible problem is not an error: the cost is +inf and every path
 *    index is -1.
 *  - Precision: samples and waypoint configurations are defined in float32
 *    (the formulas below, correctly rounded); kinematics, distances, edge
 *    costs and values are computed in float32.
 */
#ifndef GTMP_H
#define GTMP_H

#include <stdint.h>

#if defined(__GNUC__)
#define GTMP_API __attribute__((visibility("default")))
#else
#define GTMP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gtmp_ctx gtmp_ctx; /* opaque, owned by the library */

typedef enum {
  GTMP_OK = 0,
  GTMP_ERR_INVALID_ARG = 1, /* argument out of range, NULL, NaN/Inf input; nothing was enqueued */
  GTMP_ERR_CUDA = 2,        /* a CUDA runtime call failed */
  GTMP_ERR_OOM = 3,         /* device allocation failed */
  GTMP_ERR_TIMEOUT = 4,     /* a bounded device-side wait or a bounded rejection sampler gave up */
  GTMP_ERR_UNSUPPORTED = 5, /* valid request this build does not implement */
  GTMP_ERR_NOT_READY = 6    /* a required earlier call is missing (e.g. solve before endpoints) */
} gtmp_status;

enum { GTMP_ROBOT_POINT = 0, GTMP_ROBOT_DH_ARM = 1 };

/* Edge evaluation mode of the fused solver.  All give the same values,
 * minimisers and paths, bit for bit.
 * EARLY_EXIT leaves an edge at its first colliding link, skips edges that
 * cannot lie on a finite chain and, for the uniform-radius 6/7-DoF arms,
 * tests each link only against the obstacles that can reach a ball enclosing
 * its spheres, found through a uniform grid over the obstacles built by
 * gtmp_set_obstacles (a conservative cull; results unchanged); FULL evaluates every
 * interior waypoint of every candidate edge against every obstacle
 * (data-independent work, used to measure the kernel);
 * LAZY checks an edge only if its cost c(u,v) + J_{l+1}(v) is below the best
 * realised edge of its row found so far, visiting each block of 32 columns in
 * ascending order of that bound (most edges are never realised). */
enum { GTMP_EVAL_EARLY_EXIT = 0, GTMP_EVAL_FULL = 1, GTMP_EVAL_LAZY = 2 };

/* Robot model (Sec. III: the map from a configuration to the robot's occupied
 * space that defines C_free).
 *  kind = GTMP_ROBOT_POINT: the configuration is the position of one sphere of
 *         radius point_radius (dof 1..3; missing coordinates are 0).
 *  kind = GTMP_ROBOT_DH_ARM: a serial arm in standard Denavit-Hartenberg form,
 *         link transform A_i = Rz(q_i + theta_i) Tz(d_i) Tx(a_i) Rx(alpha_i),
 *         base frame = world frame; link i carries spheres_per_link spheres
 *         given in the frame of link i (radius > 0).  Joint limits within
 *         +-4096 rad and theta offsets within +-2048 rad (the range of the
 *         kinematics' sine and cosine); gtmp_create, gtmp_batch_create and
 *         gtmp_solve_noalloc refuse other arms with GTMP_ERR_INVALID_ARG.
 * All pointers are host pointers, copied by gtmp_create. */
typedef struct {
  int32_t kind;
  int32_t dof;                 /* 1..16 */
  const float* dh;             /* [dof][4]: d, a, alpha, theta_offset (arm; ignored for point) */
  const float* link_spheres;   /* [dof][spheres_per_link][4]: x, y, z, r (arm) */
  int32_t spheres_per_link;    /* 1..8 (arm) */
  const float* q_lo;           /* [dof] joint-box lower bounds */
  const float* q_hi;           /* [dof] joint-box upper bounds, > q_lo */
  float point_radius;          /* point robot, >= 0 */
} gtmp_robot;

typedef struct {
  int32_t M;            /* capacity: samples per layer (1..16384) */
  int32_t L;            /* sample layers (1..64) */
  int32_t H;            /* waypoints per edge including both endpoints (2..1024) */
  int32_t R;            /* capacity: graphs solved together by gtmp_anytime (1..4096) */
  int32_t max_obstacles;/* capacity: spheres + boxes accepted by gtmp_set_obstacles (0..4096) */
  int32_t eval_mode;    /* GTMP_EVAL_EARLY_EXIT, GTMP_EVAL_FULL or GTMP_EVAL_LAZY */
  float max_edge_len;   /* edge-length limit l of Sec. III-B/IV-A; +INFINITY = none */
} gtmp_params;

/* Create a context on the current CUDA device; allocates all per-graph device
 * memory for the given capacities.  cuda_stream is a cudaStream_t (NULL = the
 * legacy default stream).  Source: problem statement of Sec. III. */
GTMP_API gtmp_status gtmp_create(const gtmp_robot* robot, const gtmp_params* params, void* cuda_stream, gtmp_ctx** out);

/* Free a context (synchronises its stream first).  NULL is accepted. */
GTMP_API gtmp_status gtmp_destroy(gtmp_ctx* ctx);

/* Last error message of this context ("" if none); valid until the next call. */
GTMP_API const char* gtmp_last_error(const gtmp_ctx* ctx);

/* Short name of a status code. */
GTMP_API const char* gtmp_status_string(gtmp_status s);

/* Change the stream later calls enqueue on. */
GTMP_API gtmp_status gtmp_set_stream(gtmp_ctx* ctx, void* cuda_stream);

/* Wait for the context's stream; returns GTMP_ERR_TIMEOUT if a kernel raised
 * a device-side error flag since the last call (the flag is then cleared). */
GTMP_API gtmp_status gtmp_synchronize(gtmp_ctx* ctx);

/* Obstacle region C_coll of Sec. III: spheres host [n_s][4] (centre x, y, z,
 * radius) and axis-aligned boxes host [n_b][6] (lo x, y, z, hi x, y, z).
 * Copied (the call returns after the copy).  n_s + n_b <= max_obstacles.
 * For the uniform-radius 6/7-DoF arms with at most 32 obstacle pairs it also
 * builds the early-exit cull grid (on the host, up to 16384 cells, sized so
 * the edge kernels keep two blocks per SM) and uploads it with the tables. */
GTMP_API gtmp_status gtmp_set_obstacles(gtmp_ctx* ctx, const float* spheres, int32_t n_s, const float* boxes, int32_t n_b);

/* Start q0 and goal qg (host [dof] each, inside the joint box).  Sec. III.
 * Resets the goal set to this single goal with terminal value 0. */
GTMP_API gtmp_status gtmp_set_endpoints(gtmp_ctx* ctx, const float* q_start, const float* q_goal);

/* Goal set of Alg. 1 (its G with terminal values V_g: the last layer's values
 * are min over goals of C_l + V_g): goals host [G][dof] inside the joint box,
 * values host [G] (finite, >= 0; NULL = all 0), 1 <= G <= M (capacity).
 * Replaces the goal of gtmp_set_endpoints, which must have set the start.
 * Every solve, restart and mode uses the set; informed expansion
 * (aogtmp_expand) and class sweeps (gtmp_solve_classes) need a single goal
 * and return GTMP_ERR_UNSUPPORTED otherwise. */
GTMP_API gtmp_status gtmp_set_goals(gtmp_ctx* ctx, const float* goals, const float* values, int32_t G);

/* Layer sampler of gtmp_sample_layers and gtmp_anytime.  GTMP_SAMPLER_UNIFORM
 * (default; Alg. 1 samples uniformly in the joint box): word k & 3 of Philox
 * block (i, l, restart, 1<<24 | k>>2) mapped to [lo, hi).  GTMP_SAMPLER_FREE
 * (Sec. III: pi_m is a measure on C_free): rejection on the exact checker;
 * attempt 0 is the uniform sample, attempt a >= 1 uses block (i, l, restart,
 * 5<<24 | a<<2 | k>>2); the first free attempt is kept, else the last of
 * max_attempts (its edges then collide through their endpoint).  Samples
 * that are free under the uniform sampler are unchanged.  Uses the current
 * obstacles (set them first). */
#define GTMP_SAMPLER_UNIFORM 0
#define GTMP_SAMPLER_FREE 1
GTMP_API gtmp_status gtmp_set_sampler(gtmp_ctx* ctx, int32_t sampler, int32_t max_attempts);

/* Weighted-length edge cost (App. "General Costs": any additive cost that
 * dominates length and is Lipschitz in the edge's endpoints keeps the
 * guarantees; a weighted length with 1 <= w <= W is the example).  Weight
 * field w(q) = 1 + sum_b a_b max(0, 1 - |q - c_b|^2 / s_b^2) of K bumps,
 * bumps host [K][dof + 2] = (c_b[0..dof-1], s_b, a_b) with c_b finite,
 * s_b > 0, a_b >= 0, 0 <= K <= GTMP_MAX_WEIGHT_BUMPS; K = 0 (bumps may be
 * NULL) restores the plain length.  The cost of a free edge u -> v is the
 * trapezoid rule of w on its H checked waypoints,
 *   |v - u| / (H - 1) * (w_0 / 2 + w_1 + ... + w_{H-2} + w_{H-1} / 2),
 * in float32, summed in waypoint order (the same bits in every mode).  The
 * edge-length limit still applies to |v - u|.  Copied (the call returns
 * after the copy); used by gtmp_solve (all modes), gtmp_solve_unfused,
 * gtmp_get_edge_costs, gtmp_anytime, aogtmp_expand (its informed set stays
 * valid: w >= 1), gtmp_solve_pruned and gtmp_solve_classes.  The batched and
 * allocation-free solvers keep the plain length. */
#define GTMP_MAX_WEIGHT_BUMPS 16
GTMP_API gtmp_status gtmp_set_cost_weight(gtmp_ctx* ctx, const float* bumps, int32_t K);

/* The goal vertex (index into the goal set) that graph `graph`'s best chain
 * reaches, -1 if infeasible: dev_goal device [1] int32.  Enqueued after the
 * solve on the context's stream. */
GTMP_API gtmp_status gtmp_get_goal_reached(gtmp_ctx* ctx, int32_t graph, int32_t* dev_goal);

/* Alg. 1 "uniformly sample Q": M samples per layer (M <= capacity) for graph 0.
 * Q[l][i][k] = fma(u, hi_k - lo_k, lo_k) in float32 with u = (w >> 8) * 2^-24,
 * w = word k&3 of Philox4x32-10(counter = (i, l, restart, 1<<24 | k>>2),
 * key = (seed lo 32 bits, seed hi 32 bits)), restart = 0 here; l is the
 * 0-based sample layer.  Asynchronous. */
GTMP_API gtmp_status gtmp_sample_layers(gtmp_ctx* ctx, uint64_t seed, int32_t M);

/* Alg. 1 optional input Q: device [L][M][dof] float32 samples for graph 0. */
GTMP_API gtmp_status gtmp_set_layers(gtmp_ctx* ctx, const float* dev_Q, int32_t M);

/* Copy graph 0's current samples to device [L][M][dof]. */
GTMP_API gtmp_status gtmp_get_layers(gtmp_ctx* ctx, float* dev_Q);

/* Exact configuration checker (membership in C_coll, Sec. III): dev_q device
 * [n][dof] float32 in, dev_labels device [n] uint8 out, 1 = in collision.
 * For an arm, a configuration with a coordinate beyond +-4096 rad (or NaN) is
 * labelled 1. */
GTMP_API gtmp_status gtmp_label_configs(gtmp_ctx* ctx, const float* dev_q, int32_t n, uint8_t* dev_labels);

/* gtmp of Alg. 1 on graph 0 with the fused edge + min-plus kernels (the edge
 * costs C_l are never stored).  dev_path device [L] int32: index of the chosen
 * vertex in each sample layer 1..L (-1 if infeasible); dev_cost device [1]
 * float32: J_0(q0) (+inf if infeasible).  Ties in the minimisation are broken
 * towards the smallest vertex index among exactly equal float32 values.
 * Requires endpoints and samples.  Asynchronous. */
GTMP_API gtmp_status gtmp_solve(gtmp_ctx* ctx, int32_t* dev_path, float* dev_cost);

/* Values and minimisers of the last solve of graph g: dev_V device
 * [L+2][M] float32 (row l = layer l; rows 0 and L+1 use column 0 only, other
 * columns +inf), dev_sigma device [L+2][M] int32 (minimiser in layer l+1, -1
 * if none or for the goal). */
GTMP_API gtmp_status gtmp_get_values(gtmp_ctx* ctx, int32_t g, float* dev_V, int32_t* dev_sigma);

/* Path-level lazy evaluation (a lazy variant of the kind Sec. VII leaves to
 * future work; no counterpart algorithm in the paper): on graph 0, repeat
 * (1) the min-plus sweep over optimistic edge costs -- each edge's cost as
 * gtmp_solve computes it, with no collision check, leaving out the edges found
 * colliding so far and the colliding vertices -- and (2) the exact check of
 * the chain it returns, at all H waypoints of its L + 1 edges, marking the
 * colliding ones; stop when a chain has no colliding edge (or no chain
 * exists).  Optimistic costs bound the true ones from below, so that chain is
 * optimal: its cost equals gtmp_solve's (the same float operations along the
 * same chain), its path may differ only between chains of equal cost.
 * dev_path device [L] int32, dev_cost device [1] float32 as gtmp_solve.
 * Synchronous: iterations are enqueued eight at a time, with the loop's
 * state on the device (the kernels of iterations past the last return at
 * once), and the state is read back after each group; allocates (L + 1) M^2
 * bits on first use.  stats (host, optional): iterations and colliding edges
 * found.  GTMP_ERR_TIMEOUT after max_iterations without a verified chain (the
 * outputs then hold the last, unverified chain). */
typedef struct {
  int32_t iterations;       /* sweeps run */
  int64_t colliding_edges;  /* edges the chain checks found colliding (and left out) */
} gtmp_lazy_stats;
GTMP_API gtmp_status gtmp_solve_lazy_path(gtmp_ctx* ctx, int32_t max_iterations, int32_t* dev_path, float* dev_cost,
                                          gtmp_lazy_stats* stats);

/* Unfused variant of gtmp_solve (same result): step 1 writes every edge cost
 * matrix C_l (float32, +inf = absent) into library-owned device memory,
 * step 2 runs the min-plus sweep reading it back.  The first call allocates
 * (2M + (L-1)M^2) floats (rows padded to a multiple of 4). */
GTMP_API gtmp_status gtmp_solve_unfused(gtmp_ctx* ctx, int32_t* dev_path, float* dev_cost);

/* Edge costs of one transition l -> l+1 (l = 0..L) of graph 0 as computed by
 * the unfused step 1: dev_C device [n_l][n_{l+1}] float32, +inf = absent.
 * Requires a previous gtmp_solve_unfused. */
GTMP_API gtmp_status gtmp_get_edge_costs(gtmp_ctx* ctx, int32_t l, float* dev_C);

/* Class-augmented value iteration (Prop. 1; the class-indexed archive of
 * Alg. 1 anytime-gtmp) on graph 0 of a planar point robot (GTMP_ROBOT_POINT,
 * dof 2, at most 16 obstacles): a minimum-cost chain in every realised class.
 * Class label of a start-to-goal chain: the winding numbers of the loop
 * (chain, then the straight segment qg -> q0) about each obstacle's centre
 * (sphere centres in input order, then box centres), one signed byte per
 * obstacle; edge (u, v) adds the winding numbers of the triangle u -> v -> qg,
 * decided by exact orientation tests.  Uses the unfused step-1 cost matrices
 * (allocated like gtmp_solve_unfused) and (L+2) M max_labels 24-byte table
 * entries.  max_labels (a power of two in [32, 4096]) bounds the labels of
 * one vertex: more gives GTMP_ERR_OOM.  Writes up to max_classes classes,
 * in no particular order: dev_paths device [max_classes][L] int32 (sample
 * indices of layers 1..L), dev_costs device [max_classes] float32, dev_labels
 * device [max_classes][16] int8 (entries past the obstacle count are 0);
 * *n_classes (host) = the number of classes found (may exceed max_classes).
 * Synchronous.  GTMP_ERR_UNSUPPORTED for other robots or more obstacles. */
GTMP_API gtmp_status gtmp_solve_classes(gtmp_ctx* ctx, int32_t max_labels, int32_t max_classes, int32_t* dev_paths,
                                        float* dev_costs, int8_t* dev_labels, int32_t* n_classes);

/* anytime-gtmp of Alg. 1 (single class): `restarts` independent graphs
 * (restart r uses Philox restart word r of gtmp_sample_layers' rule) solved
 * in one batch of launches.  dev_paths device [restarts][L], dev_costs device
 * [restarts], dev_best device [1] (restart with the lowest cost, first index
 * on ties, -1 if all infeasible).  restarts <= R. */
GTMP_API gtmp_status gtmp_anytime(gtmp_ctx* ctx, uint64_t seed, int32_t restarts, int32_t* dev_paths, float* dev_costs,
                         int32_t* dev_best);

/* One AO-GTMP stage (Alg. 1 ao-gtmp with expand-samples, Sec. IV-D) on
 * graph 0: top every layer up from the current M to M_new samples, then
 * solve; if the new cost is below *dev_best_cost, copy the path and cost into
 * dev_best_path / dev_best_cost.  The informed set uses c_best = *dev_best_cost
 * read on the device, so a sequence of stages needs no host round trip.
 * New slot i of 0-based layer l:
 *   c_best = +inf -> the uniform rule of gtmp_sample_layers (restart 0);
 *   else coin = bit 0 of word 0 of Philox(i, l, 0, 3<<24); if heads, or the
 *   graph had no samples yet: uniform in X_f(c_best) ∩ joint box, drawn by
 *   rejection (attempt a: z_k = 2u - 1 from Philox(i, l, a, 2<<24 | k>>2),
 *   accept if sum z_k^2 <= 1 and x = centre + r2 z + (r1 - r2)(a.z) a lies
 *   in the box; at most 65536 attempts, else GTMP_ERR_TIMEOUT at the next
 *   gtmp_synchronize); tails: midpoint of layer l-1 sample (word 1 mod M_old)
 *   and its nearest layer l+1 sample.  Only samples present on entry are used.
 * dev_stage_path device [L] and dev_stage_cost device [1] receive this
 * stage's own solution. */
GTMP_API gtmp_status aogtmp_expand(gtmp_ctx* ctx, uint64_t seed, int32_t M_new, int32_t* dev_stage_path,
                          float* dev_stage_cost, int32_t* dev_best_path, float* dev_best_cost);

/* Active layer count (Sec. IV-D: AO-GTMP runs in epochs, each with its own
 * number of layers): 1 <= L <= the L given to gtmp_create (the capacity).
 * Drops the current samples (the next solve needs new ones), re-places the
 * start and the goal set for the new layout and discards stored cost
 * matrices.  Synchronous. */
GTMP_API gtmp_status gtmp_set_num_layers(gtmp_ctx* ctx, int32_t L);

/* Edge-length limit l of later solves (Sec. III-B: edges longer than l are
 * rejected; Sec. V's l_M(r)): > 0, +INFINITY = none. */
GTMP_API gtmp_status gtmp_set_max_edge_len(gtmp_ctx* ctx, float max_edge_len);

/* AO-GTMP with epochs (Sec. IV-D).  Within an epoch the layer count L is
 * fixed and each stage doubles the samples per layer (M0, 2 M0, ... up to
 * M_max) through aogtmp_expand; the informed bound c (the best cost so far)
 * carries over from epoch to epoch.  A new epoch starts with fresh samples
 * (Philox seed + epoch) and
 *   L' = max(L + 1, ceil(c / (reach - 2 r - varsigma)) - 1)  if the layer rule
 *        L + 1 >= c / (reach - 2 r - varsigma) fails (finite c and reach),
 *   L' = L + 1                                                if M reached M_max,
 * clamped to the capacity (at the capacity only saturation starts an epoch,
 * again with fresh samples).  With limit_edges, a stage's edge-length limit is
 * l = min(l_0, c / (L + 1) + 2 r + varsigma) in double, rounded to float,
 * with the best cost c in place of the reference length (Sec. V's l_M(r);
 * l_0 = the limit on entry, restored on return); before the first solution
 * l = l_0. */
typedef struct {
  int32_t L0;          /* layers of the first epoch, 1..capacity */
  int32_t M0;          /* samples per layer at each epoch's first stage, >= 1 */
  int32_t M_max;       /* per-epoch sample cap, M0..capacity */
  int32_t stages;      /* stages in all, >= 1 */
  float reach;         /* Lambda_s(tau): the longest edge the planner connects reliably; +INFINITY: no layer rule */
  float r;             /* waypoint-ball radius r >= 0 */
  float varsigma;      /* margin varsigma >= 0; reach > 2 r + varsigma */
  int32_t limit_edges; /* 1: per-stage edge-length limit from the best cost (above); 0: keep the context's */
} gtmp_ao_schedule;

/* One stage of aogtmp_run: its epoch, layer count, samples per layer, edge
 * limit, own cost and the best cost after it (+inf while infeasible). */
typedef struct {
  int32_t epoch, L, M;
  float edge_limit, stage_cost, best_cost;
} gtmp_ao_stage;

/* Runs the schedule from scratch (c = +inf) on graph 0 (single goal).
 * dev_best_chain device [capacity + 2][dof] float32 receives the best chain
 * as configurations q0, ..., qg (rows past qg NaN; the epoch that found it
 * may have fewer layers than the last one), dev_best_cost device [1] its
 * cost, log host [stages] one record per stage, *best_layers host the layer
 * count of the best chain (0 if none).  Reads the best cost back after every
 * stage (the epoch rule needs it); leaves the context at the last epoch's
 * layer count and samples. */
GTMP_API gtmp_status aogtmp_run(gtmp_ctx* ctx, uint64_t seed, const gtmp_ao_schedule* schedule, float* dev_best_chain,
                                float* dev_best_cost, gtmp_ao_stage* log, int32_t* best_layers);

/* Launch accounting and kernel timing (library instrumentation; the paper
 * reports no such facility).  Every kernel the context enqueues increments
 * `launches`.  While timing is enabled, CUDA events bracket each fused
 * edge + min-plus launch on the context's stream; gtmp_profile_read
 * synchronises the stream, sums those launches' durations and resets the
 * counters.  The events add two event records per fused launch. */
typedef struct {
  int64_t launches;        /* kernels enqueued since the last read */
  int64_t fused_launches;  /* fused edge + min-plus launches timed */
  double fused_ms;         /* device time of their sweeps (ms): one event pair around each sweep of
                              L + 1 launches, which overlap as programmatic dependent launches */
  double fused_edges;      /* candidate edges those launches processed */
  int64_t minplus_launches;  /* min-plus launches of gtmp_solve_unfused timed */
  double minplus_ms;         /* device time of their sweeps (ms): one event pair around each
                                sweep of L + 1 launches, which overlap as programmatic
                                dependent launches */
  double minplus_bytes;      /* their algorithmic HBM bytes: 4 per stored edge cost read, 8 per
                                cost-to-go read and 8 per cost-to-go written */
} gtmp_profile;

GTMP_API gtmp_status gtmp_profile_enable(gtmp_ctx* ctx, int32_t enable);
GTMP_API gtmp_status gtmp_profile_read(gtmp_ctx* ctx, gtmp_profile* out);

/* Allocation-free solve.  The paper has no counterpart: this entry point
 * exists for callers that may not allocate device memory at solve time, such
 * as a control loop with a fixed real-time budget (cudaMalloc/cudaFree can
 * block and synchronise the whole device), a plugin running inside a host
 * application that owns every device allocation, or a process whose device
 * memory is fully reserved up front.  It plans one graph like gtmp_solve
 * (early-exit mode, same kernels, same result) from caller-supplied inputs:
 * robot, obstacles (host, as gtmp_set_obstacles, at most 256 in total),
 * endpoints (host [dof] each), samples dev_Q (device [L][M][dof] float32),
 * H and max_edge_len; it writes dev_path (device [L] int32), dev_cost (device
 * [1] float32) and, if dev_status is not NULL, the device error word (device
 * [1] int32; 0 = fine, else the bits gtmp_synchronize would report).
 * It calls no cudaMalloc, cudaFree or other allocating routine: all scratch
 * (samples in kernel layout, vertex flags, value/index keys, work counters,
 * the obstacle table) lives in one fixed 1 MiB device array inside the
 * library, which every GPU that loads the library holds until the process
 * exits.  Requests that need more than 1 MiB are rejected with
 * GTMP_ERR_INVALID_ARG and a message (scratch bytes = roughly (L+2) M
 * (4 dp + 9) with dp = 8 for 6/7-joint arms, so M = 1024, L = 8 fits).
 * The first call on a device resolves the array's device address and
 * queries launch limits for that device (the device must be current); make
 * that first call before any stream capture.  Every call on a device shares
 * the one array and overwrites it, so calls whose GPU work overlaps (other
 * streams, other threads) race and give wrong results; serialise them.
 * The host inputs (obstacle table, endpoints) travel inside the kernel
 * parameters of the call's first launch, so the call reads no host memory
 * after it returns and does not wait for earlier work on cuda_stream.
 * Work is enqueued on cuda_stream; outputs are valid after it completes.
 * On failure, err_msg (host, err_msg_len bytes, may be NULL) receives a
 * one-line reason. */
GTMP_API gtmp_status gtmp_solve_noalloc(const gtmp_robot* robot, const float* spheres, int32_t n_s,
                                        const float* boxes, int32_t n_b, const float* q_start,
                                        const float* q_goal, const float* dev_Q, int32_t M, int32_t L, int32_t H,
                                        float max_edge_len, void* cuda_stream, int32_t* dev_path, float* dev_cost,
                                        int32_t* dev_status, char* err_msg, int32_t err_msg_len);

/* ---------------------------------------------------------------------------
 * Batched planning (serving pattern; the paper plans one query at a time):
 * n independent problems, each gtmp of Alg. 1 with its own robot, obstacles,
 * endpoints, M, L and Philox seed, solved by one persistent launch.  Problem
 * p's samples are those gtmp_sample_layers(seed_p) draws, and its result is
 * the one gtmp_solve gives for that problem (same kernels and tie rule).
 * ------------------------------------------------------------------------- */
typedef struct {
  gtmp_robot robot;          /* host pointers, copied at create */
  const float* spheres;      /* host [n_s][4] */
  int32_t n_s;
  const float* boxes;        /* host [n_b][6] */
  int32_t n_b;
  const float* q_start;      /* host [dof] */
  const float* q_goal;       /* host [dof] */
  int32_t M;                 /* samples per layer, 1..16384 */
  int32_t L;                 /* sample layers, 1..64 */
  uint64_t seed;             /* Philox seed of this problem's samples */
} gtmp_problem;

typedef struct gtmp_batch gtmp_batch;

/* Copy n problems (H waypoints per edge for all) to the device and build the
 * work list (items of rows ordered by distance from the goal layer).
 * GTMP_ERR_INVALID_ARG for a problem outside the limits above (at most 4096
 * obstacles); GTMP_ERR_UNSUPPORTED when one problem's obstacle table and
 * cost-to-go row (16 B per obstacle float4, 4 B per sample) exceed the
 * 200 KB of shared memory an item stages them in. */
GTMP_API gtmp_status gtmp_batch_create(const gtmp_problem* problems, int32_t n, int32_t H, void* cuda_stream,
                                       gtmp_batch** out);
GTMP_API gtmp_status gtmp_batch_destroy(gtmp_batch* b);
GTMP_API const char* gtmp_batch_last_error(const gtmp_batch* b);
GTMP_API gtmp_status gtmp_batch_set_stream(gtmp_batch* b, void* cuda_stream);

/* L_max = max L over problems; nominal_checks = sum over problems of
 * H (2M + (L-1) M^2); work_items = items in the current work list;
 * kernels = kernel launches one gtmp_batch_solve enqueues (each output
 * optional, host). */
GTMP_API gtmp_status gtmp_batch_info(const gtmp_batch* b, int32_t* L_max, double* nominal_checks,
                                     int32_t* work_items, int32_t* kernels);

/* Sample, label and solve all problems: dev_paths device [n][L_max] int32
 * (problem p's layer indices in columns 0..L_p-1, -1 elsewhere or when
 * infeasible), dev_costs device [n] float32 (+inf when infeasible).  Enqueues
 * a memset, three set-up kernels, one persistent kernel per robot variant in
 * the batch (point robot, 6- and 7-joint uniform-radius arms, other arms)
 * and a path kernel on the batch stream; no host
 * synchronisation, so the call can be captured in a CUDA graph.  Every
 * device-side dependency wait is bounded (about 2 s without progress of the
 * awaited items); a wait that gives up abandons its item and sets the error
 * word that gtmp_batch_synchronize reports. */
GTMP_API gtmp_status gtmp_batch_solve(gtmp_batch* b, int32_t* dev_paths, float* dev_costs);
GTMP_API gtmp_status gtmp_batch_synchronize(gtmp_batch* b);

/* Tiling of the work list, per robot kind (kind = GTMP_ROBOT_POINT or
 * GTMP_ROBOT_DH_ARM; the two kinds run in separate persistent launches): about
 * target_edges candidate edges per item (an item smaller than a row is a
 * column piece of one row) and chunk columns per warp claim (point robots
 * take at least 32, one edge per lane).  gtmp_batch_set_tiling sets both
 * kinds; every setter synchronises the batch stream and rebuilds the work
 * list.  Defaults: 16384 edges for both kinds, chunk 32 (point) and 16
 * (arm).  gtmp_batch_autotune times each kind's persistent launches (CUDA
 * events around them; repeats solves per trial, into the given buffers)
 * first over four item sizes per kind, then over chunks 4, 8, 16 and 32 at
 * the best size, keeps each kind's fastest, and returns the time per solve
 * of the whole batch under the tilings kept in *best_ms (host, optional).
 * GTMP_ERR_INVALID_ARG for another kind, target_edges < 1 or a chunk outside
 * [1, 4096]. */
GTMP_API gtmp_status gtmp_batch_set_tiling(gtmp_batch* b, int32_t target_edges, int32_t chunk);
GTMP_API gtmp_status gtmp_batch_set_kind_tiling(gtmp_batch* b, int32_t kind, int32_t target_edges, int32_t chunk);
GTMP_API gtmp_status gtmp_batch_get_tiling(const gtmp_batch* b, int32_t kind, int32_t* target_edges, int32_t* chunk);
GTMP_API gtmp_status gtmp_batch_autotune(gtmp_batch* b, int32_t repeats, int32_t* dev_paths, float* dev_costs,
                                         float* best_ms);

/* Edge realisation of the batched solve: GTMP_EVAL_EARLY_EXIT (default) or
 * GTMP_EVAL_LAZY (the bound-ordered exact mode of gtmp_params.eval_mode; each
 * problem's result is unchanged bit for bit).  Takes effect at the next
 * gtmp_batch_solve; GTMP_ERR_INVALID_ARG for any other mode. */
GTMP_API gtmp_status gtmp_batch_set_eval_mode(gtmp_batch* b, int32_t eval_mode);

/* Fault injection for tests, no counterpart in the paper: makes depth `depth`
 * (0 <= depth < L of that problem) of problem `problem` unfinishable by
 * raising its completion target out of reach, so in the next
 * gtmp_batch_solve the items waiting on it give up after ~2 s without
 * progress, every other wait then stops at once, the waiting items are
 * abandoned and gtmp_batch_synchronize reports GTMP_ERR_TIMEOUT; nothing
 * faults and the GPU stays usable.  problem < 0 restores every target (the
 * next solve is exact again).  Synchronous; host-side only. */
GTMP_API gtmp_status gtmp_batch_inject_stall(gtmp_batch* b, int32_t problem, int32_t depth);

/* ---------------------------------------------------------------------------
 * Learned collision surrogate and surrogate-pruned solve (serving pattern; the
 * paper has no surrogate and names lazy edge realisation as future work,
 * Sec. VII).  Model: Fourier features [sin(Bq), cos(Bq)] (B: 64 x dof, drawn
 * N(0, sigma^2) per rad), three ReLU layers of 256 units, one logit; BF16 weights and
 * activations, FP32 accumulation on the tcgen05 tensor cores.
 * ------------------------------------------------------------------------- */
typedef struct {
  int32_t n_train;    /* training configurations, a multiple of 64 (uniform in the joint box, labelled by
                         the exact checker) */
  int32_t n_holdout;  /* held-out configurations for the reported rates */
  int32_t epochs;
  int32_t batch;      /* multiple of 64, <= n_train */
  float lr;           /* Adam step size */
  uint64_t seed;      /* Philox seed of the configurations and of the initial weights */
  float fourier_sigma;/* standard deviation of the Fourier frequencies per rad (<= 0: 1) */
} gtmp_surrogate_config;

typedef struct {
  float final_loss;       /* mean binary cross-entropy over the last epoch */
  float holdout_accuracy; /* at p = 1/2 */
  float holdout_fn_rate;  /* colliding held-out configurations predicted free */
  float holdout_fp_rate;  /* free held-out configurations predicted colliding */
  float train_ms;         /* device time of data generation, labelling and training */
} gtmp_surrogate_stats;

typedef struct {
  double edges;     /* candidate edges of the graph */
  double pruned;    /* live edges dropped before exact checking */
  float score_ms;   /* device time of the surrogate scoring kernels */
  float solve_ms;   /* device time of the exact fused transitions */
  double scored;    /* live edges scored by the surrogate (row and column live) */
  float band_ms;    /* device time of the protection-band passes (0 without a band) */
  float lists_ms;   /* device time of the live row / column lists the scoring reads */
} gtmp_prune_stats;

/* Train the context's surrogate for its robot and current obstacles
 * (synchronous; allocates its buffers on first use). */
GTMP_API gtmp_status gtmp_surrogate_train(gtmp_ctx* ctx, const gtmp_surrogate_config* cfg,
                                          gtmp_surrogate_stats* stats);

/* Logits of configurations dev_q device [n][dof] -> dev_logits device [n]. */
GTMP_API gtmp_status gtmp_surrogate_predict(gtmp_ctx* ctx, const float* dev_q, int32_t n, float* dev_logits);

/* FP32 master parameters (host [gtmp_surrogate_param_count()]: W1[256][128],
 * b1[256], W2[256][256], b2, W3[256][256], b3, w4[256], b4) and the Fourier
 * matrix (host [64][dof]). */
GTMP_API int64_t gtmp_surrogate_param_count(void);
GTMP_API gtmp_status gtmp_surrogate_get_params(gtmp_ctx* ctx, float* host_params, int64_t n, float* host_fourier,
                                               int64_t n_fourier);

/* Load FP32 parameters (layout of gtmp_surrogate_get_params) instead of
 * training, and the mean binary cross-entropy and its gradient (host
 * [gtmp_surrogate_param_count()]) at the current parameters for n labelled
 * configurations (dev_q device [n][dof], dev_labels device [n] uint8, n a
 * multiple of 64 up to 65536): one forward and backward pass of training,
 * without the update.  Synchronous. */
GTMP_API gtmp_status gtmp_surrogate_set_params(gtmp_ctx* ctx, const float* host_params, int64_t n,
                                               const float* host_fourier, int64_t n_fourier);
GTMP_API gtmp_status gtmp_surrogate_loss_grad(gtmp_ctx* ctx, const float* dev_q, const uint8_t* dev_labels, int32_t n,
                                              double* host_loss, float* host_grad, int64_t n_grad);

/* gtmp_solve on graph 0 in which an edge is dropped before exact checking when
 * the surrogate's collision probability at any of its scored waypoints
 * (score_waypoints = 1: t = 1/2; 3: t = 1/4, 1/2, 3/4) exceeds threshold and
 * the edge lies outside the protection band (gtmp_surrogate_set_protect);
 * scoring runs in one fused tensor-core kernel per transition and covers the
 * live edges only (row vertex free, column vertex free with a finite
 * cost-to-go: the exact solve skips every other edge anyway).  Every
 * surviving edge is realised by the exact checker (lazily when the context's
 * eval_mode is GTMP_EVAL_LAZY, else with early exit), so a returned path is
 * collision free at its H waypoints; the cost can exceed gtmp_solve's when a
 * free edge is dropped.  Synchronous (returns the stats); allocates an M x M
 * mask on first use. */
GTMP_API gtmp_status gtmp_solve_pruned(gtmp_ctx* ctx, float threshold, int32_t score_waypoints, int32_t* dev_path,
                                       float* dev_cost, gtmp_prune_stats* stats);

/* Protection band of the surrogate's pruning (no counterpart in the paper):
 * with band > 0, an edge (u, v) whose bound |v - u| + J(v) (its length plus
 * the cost-to-go of its head, a lower bound of what the edge can give the
 * row) is at most (1 + band) times the smallest such bound of its row (over
 * the live columns, edges beyond the edge limit left out) is never pruned,
 * whatever its score: the edges a row's best path most likely takes stay with
 * the exact checker, and the rest can be pruned at a lower threshold.  0 (the
 * default) turns the band off.  Takes effect at the next gtmp_solve_pruned or
 * gtmp_surrogate_score.  GTMP_ERR_INVALID_ARG outside [0, 16]. */
GTMP_API gtmp_status gtmp_surrogate_set_protect(gtmp_ctx* ctx, float band);

/* Inspection of the scoring step of gtmp_solve_pruned (no counterpart in the
 * paper): the fused scoring kernel's decision for every live edge of one
 * transition `layer` (0 = start row, L = the goal column) of graph 0, with
 * liveness taken from the context's current vertex labels and cost-to-go (so
 * call it after a gtmp_solve or gtmp_solve_pruned of the same samples):
 * rows whose vertex is free, columns whose vertex is free with a finite
 * cost-to-go.  dev_mask device [rows][cols] uint8 (rows = 1 for layer 0, else
 * M; cols = M, or the goal count for layer L): 1 = pruned (the largest
 * scored waypoint logit exceeds logit(threshold) and the edge lies outside
 * the protection band), 0 = kept, 2 = not live (not scored).  host_scored (may be NULL) receives the live-edge count.
 * Synchronous.  Errors: GTMP_ERR_NOT_READY before training or sampling,
 * GTMP_ERR_INVALID_ARG for a bad layer, threshold or waypoint count. */
GTMP_API gtmp_status gtmp_surrogate_score(gtmp_ctx* ctx, int32_t layer, float threshold, int32_t score_waypoints,
                                          uint8_t* dev_mask, int64_t* host_scored);

/* Inspection, no counterpart in the paper: the cull grid gtmp_set_obstacles
 * builds for the early-exit checker of the uniform-radius arms, computed on
 * the host for obstacles given as to gtmp_set_obstacles (n_s + n_b <= 4096)
 * and a link-ball radius R_link > 0, with at most max_cells <= 16384 cells.
 * masks host [max_cells] uint32: cell (ix, iy, iz) at
 * (iz * ny + iy) * nx + ix, bit p set when obstacle pair p (spheres 2p and
 * 2p + 1, then boxes in the same way after the sphere pairs) comes within
 * R_link + r (box: R_link) of the cell, plus a margin; dims host [3] = (nx,
 * ny, nz), all 0 when no grid is built (no obstacle, more than 32 pairs, or
 * max_cells < 64); origin_inv host [4] = lower corner x, y, z and 1 / cell
 * size.  A point whose float32 cell index (x - corner) * inv falls outside
 * the grid is farther than that from every obstacle.  Needs no GPU. */
GTMP_API gtmp_status gtmp_cull_grid(const float* spheres, int32_t n_s, const float* boxes, int32_t n_b, float R_link,
                                    int32_t max_cells, uint32_t* masks, int32_t* dims, float* origin_inv);

/* The sine and cosine the arm kinematics takes of each joint angle q_i +
 * theta_i (A_i above): Cody-Waite reduction by pi/2, then the Taylor series of
 * sin and cos on |r| <= pi/4; within 1e-7 absolute of the exact values for
 * |x| <= 6144 rad, the range the joint-limit and theta-offset bounds keep
 * every argument in.  dev_x device [n] float32 in, dev_s, dev_c device [n]
 * out; asynchronous on cuda_stream (NULL = legacy default stream).  Exposed
 * so that the kinematics' trigonometry can be checked against FP64.
 * GTMP_ERR_INVALID_ARG for n < 0 or a NULL pointer with n > 0. */
GTMP_API gtmp_status gtmp_joint_sincos(const float* dev_x, int32_t n, float* dev_s, float* dev_c, void* cuda_stream);

/* Calibration, no counterpart in the paper: the FP32 FMA throughput of the
 * current device in TFLOP/s (FMA = 2 flops), from a kernel of independent
 * FMA chains filling every SM, launched 8 times on cuda_stream (NULL = legacy
 * default stream); *tflops receives the best of the last 6.  Synchronises the
 * stream.  The fused edge kernels are FP32-pipe bound; this is the ceiling a
 * pure FMA stream reaches at the clocks and power state of the moment.
 * GTMP_ERR_CUDA if a launch fails. */
GTMP_API gtmp_status gtmp_fp32_fma_peak(void* cuda_stream, double* tflops);

/* The surrogate's tensor-core GEMM on its own: C[m][n] = sum_k A[m][k] B[n][k]
 * with A device [M][lda] and B device [N][ldb] bf16 (K contiguous; lda, ldb
 * multiples of 8, 16-byte aligned bases), C device [M][ldc] float32; N a
 * multiple of 16, K a multiple of 8.  Enqueued on cuda_stream; a timed-out
 * wait sets *dev_err (device int32). */
GTMP_API gtmp_status gtmp_umma_gemm_f32(const void* dev_A, int32_t lda, const void* dev_B, int32_t ldb, int32_t M,
                                        int32_t N, int32_t K, float* dev_C, int32_t ldc, void* cuda_stream,
                                        int32_t* dev_err);

/* Active samples per layer of graph 0 (after sample/set/expand). */
GTMP_API gtmp_status gtmp_get_M(const gtmp_ctx* ctx, int32_t* M);

#ifdef __cplusplus
}
#endif

#endif /* GTMP_H */
