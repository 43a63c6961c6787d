/*
 * plan.h -- C ABI of the GB300 (sm_103a) reachable-Bezier-polytope planner.
 *
 * The library builds the kinodynamic Bezier graph of arXiv 2411.13507 and
 * searches it on one GPU.  Every entry point is asynchronous on the stream
 * given to plan_create(); device-detected conditions (capacity, timeout, no
 * path) are written to a device status word that plan_wait() reads.  No entry
 * point throws across the ABI; each returns a plan_status code.
 *
 * Memory: every array argument documented "device" is caller-owned device
 * memory (e.g. a torch tensor); "host" arrays are read before the call
 * returns.  The library never frees caller memory.  It allocates only its own
 * context scratch (at plan_create and, when plan_wait reports that a call
 * needed more, at the next call).
 *
 * Notation (paper, Sec. II): m outputs, relative degree g (gamma), state
 * dimension n = m*g stacked x = [b; b'; ...; b^(g-1)] (Eq. BezDef), Bezier
 * degree p, durations T_t.  For one axis a, xi = [x_i^(0..g-1)_a ; x_j^(0..g-1)_a].
 */
#ifndef PLAN_H
#define PLAN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct plan_ctx plan_ctx;

typedef enum {
    PLAN_OK = 0,
    PLAN_ERR_INVALID_ARG = 1,  /* bad pointer, size or model parameter */
    PLAN_ERR_UNSUPPORTED = 2,  /* model outside the compiled set, or a polytope with > 16 rows */
    PLAN_ERR_CAPACITY = 3,     /* output buffer (or internal scratch) too small; see plan_info */
    PLAN_ERR_CUDA = 4,         /* a CUDA runtime call failed; see plan_last_error */
    PLAN_ERR_TIMEOUT = 5,      /* a bounded device loop ran out of iterations */
    PLAN_ERR_NO_PATH = 6,      /* goal vertex unreachable from the start vertex */
    PLAN_ERR_NO_MEMORY = 7     /* context scratch could not be allocated */
} plan_status;

/* Arithmetic of the edge-build margins. */
typedef enum {
    PLAN_F64 = 0,   /* FP64 results: bits of the canonical FP64 margins, costs in canonical FP64
                       (weights are doubles); see plan_set_tile for the two routes */
    PLAN_F32 = 1,   /* FP32 margins; any margin within its error band re-checked in FP64 */
    PLAN_TF32 = 2,  /* control-point products on tensor cores, TF32 inputs, FP32 accumulate, FP64 re-check;
                       2-D models only (m = 2; plan_create returns UNSUPPORTED otherwise) */
    PLAN_BF16 = 3   /* as TF32 with BF16 inputs (2-D models only) */
} plan_arith;

/* Storage type of states, A and b. */
typedef enum { PLAN_IN_F64 = 0, PLAN_IN_F32 = 1 } plan_input;

typedef enum { PLAN_COST_STATE = 0, PLAN_COST_POS = 1 } plan_cost_mode;

/*
 * Chain-of-integrators model (Eq. rom) and edge-test options.
 *   m, gamma, degree : compiled combinations (m,gamma,p) in
 *                      {(2,2,3),(2,2,5),(3,3,5),(3,3,7)}; others -> UNSUPPORTED.
 *   bound[k-1]       : per-axis bound c_k on the k-th derivative, k = 1..gamma
 *                      (k = gamma bounds the input u_d).  Theorem 1's F x <= G is
 *                      taken as |Q^(k)_j| <= c_k on every hodograph control point.
 *   tighten          : eps subtracted from every c_k and every b_r (Def. 1's
 *                      tracking-error margin; 0 by default).
 *   cost_mode        : PLAN_COST_STATE: polygon length of the n-row state-space
 *                      control points (Eq. BezDef, Property 2); PLAN_COST_POS:
 *                      position rows only.
 *   interior         : for degree > 2 gamma - 1 Lemma 1 fixes only the first and
 *                      last gamma control points.  PLAN_INTERIOR_ELEVATE (0): the
 *                      unique minimal-degree curve, degree-elevated (same curve);
 *                      PLAN_INTERIOR_MINSNAP (1): interior points minimising the
 *                      integral of |b^(gamma+1)|^2 over [0, T].
 */
typedef enum { PLAN_INTERIOR_ELEVATE = 0, PLAN_INTERIOR_MINSNAP = 1 } plan_interior;

typedef struct {
    int m;
    int gamma;
    int degree;
    int arith;      /* plan_arith */
    int input;      /* plan_input */
    int cost_mode;  /* plan_cost_mode */
    double bound[4];
    double tighten;
    int interior;   /* plan_interior */
} plan_model;

/*
 * Feasible-edge graph in CSR form, sorted by (i asc, j asc).  All pointers
 * are caller-owned device memory.
 *   row_off [N+1] int32   (always written)
 *   col     [cap] int32   end vertex j
 *   w       [cap]         edge cost: double when arith == PLAN_F64, else float;
 *                         min over feasible durations of the control-polygon
 *                         length (Sec. III-C), ties to the lower duration index
 *   tidx    [cap] uint8   index of that duration
 *   mask    [cap] uint32  bit t set iff (i -> j, T_t) passes the reach test and
 *                         fits a shared free polytope
 *   count   [1]   int64   number of edges E (written even when E > cap; the
 *                         CSR arrays are then left unwritten and the call
 *                         reports PLAN_ERR_CAPACITY)
 */
typedef struct {
    int32_t* row_off;
    int32_t* col;
    void* w;
    uint8_t* tidx;
    uint32_t* mask;
    int64_t cap;
    int64_t* count;
} plan_edges;

/* Counters of the last call, read by plan_wait (host struct). */
typedef struct {
    int32_t status;           /* plan_status of the device work */
    int32_t detail;           /* which check raised it (library-internal code) */
    int64_t memberships;      /* sum over polytopes of member counts */
    int64_t slots;            /* sum over polytopes of (member count)^2 */
    int64_t candidates;       /* distinct ordered pairs (i != j) sharing a polytope */
    int64_t checks;           /* candidates * nT */
    int64_t reach_pass;       /* (candidate, T) passing the reach test (owner block) */
    int64_t feasible;         /* feasible (candidate, T) bits in the output */
    int64_t rechecks;         /* (pair, T, polytope) evaluations re-done in FP64 */
    int64_t edges;            /* E */
    int64_t search_iters;     /* frontier sweeps of the last search */
    int32_t start, goal;      /* vertices chosen by the last search */
    int64_t need_slots, need_rechecks;  /* scratch sizes the last call needed */
    /* with plan_set_accounting(ctx, 1): algorithmic work of the last build under
     * short-circuit evaluation (reach rows up to the first violated one, free
     * rows of reach-passing checks, cost evaluations of feasible checks) */
    int64_t work_reach_rows, work_free_rows, work_costs;
    /* (pair, T) that the FP32 reach screen passed on to the full rows (the
     * screened pair kernel only; 0 otherwise) */
    int64_t screened;
    /* keep-out cut (plan_cut_edges): (edge, T) checked; (edge, T, obstacle)
     * screened; of those, missed by the obstacles' certified bounding boxes,
     * and the rest (the pair list); of the listed pairs, hit by a control
     * point inside and missed by one separating facet (FP32, decided within
     * error bands), matrix games solved in FP32; entries of the FP64 pass;
     * FP64 games that no certificate decided (|delta*| at rounding level) */
    int64_t cut_units, cut_tests, cut_box, cut_near, cut_step1, cut_step2, cut_games, cut_lp64, cut_ties;
    /* source rows [shard_lo, shard_hi) of the last plan_build_edges_shard
     * (0, N for a whole build; of the first query for a batch) */
    int32_t shard_lo, shard_hi;
} plan_info;

/* Create a context bound to the current CUDA device and the given stream
 * (cudaStream_t; NULL = legacy default stream).  Validates the model. */
int plan_create(plan_ctx** out, const plan_model* model, void* cuda_stream);

/* Release the context and its scratch (synchronises its stream first). */
void plan_destroy(plan_ctx* ctx);

/*
 * buildGraph + keep-in cut (Algorithm 1, Sec. III-A/B): for every ordered
 * pair of states sharing at least one free polytope and every duration T_t,
 * form the control points meeting the boundary conditions (Lemma 1, elevated
 * to degree p), test the hodograph control points against the bounds
 * (Theorem 1) and the control points against the shared polytope (Property 1),
 * reduce to the feasibility mask and the edge cost, and compact the graph.
 *
 *   N         number of states (0 <= N <= 1<<20)
 *   states    device [N][n], input type, x = [pos; vel; acc; ...] per state
 *   nT, T     host [nT] durations, 1 <= nT <= 32, all > 0 and finite
 *   K         number of free polytopes (0 <= K <= 1024)
 *   poly_off  device int32 [K+1], rows of polytope k are poly_off[k]..poly_off[k+1]-1,
 *             poly_off[0] = 0
 *   max_rows  host bound on the rows of any polytope, 1..16 (sizes shared
 *             memory; a polytope with more rows -> device status UNSUPPORTED)
 *   A, b      device [R][m] and [R], input type; polytope k = {x : A_r x <= b_r}
 *   out       caller-owned CSR (see plan_edges)
 * Errors: INVALID_ARG / UNSUPPORTED on the host; CAPACITY, UNSUPPORTED (row
 * count) on the device via plan_wait.  When internal scratch was too small,
 * plan_wait returns PLAN_ERR_CAPACITY with need_* set and grows the scratch, so
 * the caller simply repeats the call.
 */
int plan_build_edges(plan_ctx* ctx, int N, const void* states, int nT, const double* T, int K,
                     const int32_t* poly_off, int max_rows, const void* A, const void* b,
                     const plan_edges* out);

/*
 * One shard of plan_build_edges, for a build split over several GPUs
 * (Algorithm 1's buildGraph at a size one GPU would split): the source rows
 * are cut into nshard contiguous ranges of equal work, the work of row i
 * being the number of (i, j) pair slots it has in its polytopes (the sum of
 * the member counts of the polytopes holding state i; every duration costs
 * the same).  The cut points are computed on the device from the membership,
 * identically by every rank, so no exchange precedes the build.  This call
 * computes every candidate pair (i, j) of the rows i of shard `shard` over
 * every shared polytope and duration -- all polytopes, all columns j -- so its
 * rows are final: they equal the rows of plan_build_edges bit for bit.
 *   shard, nshard  0 <= shard < nshard <= 1024
 *   out            caller-owned CSR over all N rows: row_off [N+1] is written
 *                  for every row (rows outside the shard are empty), col / w /
 *                  tidx / mask hold the shard's edges only, count = their number
 * The rows of shard r precede those of shard r+1, so the whole graph is the
 * concatenation of the shards' edges in shard order, with row_off the sum of
 * the shards' row_off arrays.  plan_info.shard_lo / shard_hi report the rows;
 * candidates, checks and feasible count the shard's rows only.  Everything
 * else (arguments, errors, scratch growth) as plan_build_edges.
 */
int plan_build_edges_shard(plan_ctx* ctx, int N, const void* states, int nT, const double* T, int K,
                           const int32_t* poly_off, int max_rows, const void* A, const void* b, int shard,
                           int nshard, const plan_edges* out);

/* One query of a batched edge build (same fields as plan_build_edges). */
typedef struct {
    int N;
    const void* states;     /* device [N][n] */
    int nT;
    const double* T;        /* host [nT]; read by plan_prepare_batched */
    int K;
    const int32_t* poly_off; /* device [K+1] */
    const void* A;          /* device [R][m] */
    const void* b;          /* device [R] */
    plan_edges out;         /* caller-owned CSR of this query */
} plan_query;

/*
 * Batching form: many independent queries of uneven size in one pass.
 * plan_prepare_batched does the host work (argument checks, per-query
 * offsets, coefficient tables for every query's durations, scratch sizing,
 * descriptor upload; it may allocate and may wait for earlier uploads).
 * plan_build_edges_batched then launches the whole edge build of every
 * prepared query -- the pair work of all queries in ONE persistent launch --
 * without any host synchronisation or allocation, so it can be captured in a
 * CUDA graph and replayed (the device reads the queries' inputs at replay).
 * Results, statuses and counters are those of plan_build_edges, summed over
 * queries in plan_info; each query's edge count lands in its out.count.
 * Q <= 65535; max_rows bounds the rows of every polytope of every query.
 */
int plan_prepare_batched(plan_ctx* ctx, int Q, const plan_query* queries, int max_rows);
int plan_build_edges_batched(plan_ctx* ctx);

/* FP32 pair-kernel configuration: tile side (8..64, multiple of 4; 0 = 64),
 * CTAs per SM (0 = as many as fit), duration chunks per tile (work items are
 * tiles x chunks, longest durations first, largest tiles first; 0 = chosen
 * per build on the device once the tile count is known: enough chunks for
 * about eight items per SM, one to the most durations of any query) and
 * pipeline (0, the
 * default: one warp group that screens every 4x4 block of pairs on the few
 * reach rows that mix both boundary states and runs the surviving pairs,
 * compacted, through all rows; 1: the warp-specialised kernel -- producer
 * warps compute the next duration's halves while consumer warps reduce the
 * current one; used with 64-state tiles when its two stages fit in shared
 * memory; 2: one warp group, every 4x4 block through all rows).  Results do
 * not depend on the choice.  An FP64 model (PLAN_F64) runs these FP32
 * kernels too -- every margin within its rounding band of zero is re-checked
 * in canonical FP64, so the bits are the FP64 ones -- and then computes the
 * cost of every emitted edge and duration in canonical FP64 (the weight is
 * the cheapest, ties to the lower duration index); pipeline 3 (FP64 models
 * only) runs the canonical FP64 pair kernel instead (every margin and cost in
 * FP64, 32-state tiles).  Both FP64 routes give the same graph
 * bit for bit.  plan_autotune times every candidate on the prepared batch (reps launches
 * each, synchronising) and keeps the fastest; it reports the choice and its
 * mean pair-kernel time. */
int plan_set_tile(plan_ctx* ctx, int tile, int ctas_per_sm, int tchunks, int pipeline);
int plan_autotune(plan_ctx* ctx, int reps, int* best_tile, int* best_ctas, int* best_chunks, int* best_pipeline,
                  double* best_ms);

/*
 * findPath (Algorithm 1, Sec. III-C, Problem 2): the start and goal vertices
 * are the states nearest (Euclidean, positions only; ties to the lowest id) to
 * start_pos and goal_pos; then shortest paths with Dijkstra semantics (FP64
 * accumulation dist[u] + w; predecessor = the earliest-settled vertex that
 * attains dist[v], i.e. the minimum (dist[u], u)).
 *   states      device [N][n] (same array as the build)
 *   edges       device CSR from plan_build_edges (count must be <= cap)
 *   start_pos,
 *   goal_pos    host [m] doubles
 *   path        device int32 [path_cap]: vertex ids start..goal
 *   path_len    device int32 [1]: number of vertices (0 if no path)
 *   cost        device double [1]: path cost (+inf if no path)
 * Device status NO_PATH when the goal is unreachable, TIMEOUT if the frontier
 * loop exceeds N+1 sweeps, CAPACITY if the path is longer than path_cap.
 */
int plan_search(plan_ctx* ctx, int N, const void* states, const plan_edges* edges,
                const double* start_pos, const double* goal_pos, int32_t* path, int path_cap,
                int32_t* path_len, double* cost);

/*
 * plan_search with the start and goal positions read from device memory when
 * the search runs (not when it is issued), so that a replanning loop can
 * capture the search once in a CUDA graph and move start and goal between
 * replays.
 *   endpoints  device double [2][m]: start position, then goal position
 *              (finite; not checked on the host)
 * Everything else as plan_search.
 */
int plan_search_at(plan_ctx* ctx, int N, const void* states, const plan_edges* edges, const double* endpoints,
                   int32_t* path, int path_cap, int32_t* path_len, double* cost);

/*
 * Goal-rooted search for a replanning loop (Algorithm 1's findPath every tick; Sec.
 * III-C): start and goal vertices as plan_search_at (nearest to device
 * endpoints [2][m]); then the distance of every vertex TO the goal vertex, the
 * fixed point of d[u] = min over out-edges (u -> v) of (w + d[v]) in FP64,
 * and the path from the start along the successors (the out-neighbour v
 * minimising (w + d[v], v)); cost = d[start].  warm != 0: when the goal vertex
 * and N equal those of the previous plan_search_to call on this context, every
 * vertex whose successor chain to the goal still exists with weights no larger
 * than before keeps its previous distance and the rest restart from +inf; the
 * result equals a cold start (only the number of sweeps changes).  Rows of
 * the CSR must be sorted by column (as plan_build_edges and plan_cut_edges
 * write them).  One cooperative launch over every SM, like plan_search.
 * Among equal-cost paths it may return another one than plan_search, and the
 * cost may differ from plan_search's in the last bits (the path sum is
 * rounded from the goal end).  N, states, edges, path, path_cap, path_len
 * and cost as plan_search; endpoints as plan_search_at.  Device status as
 * plan_search (NO_PATH, CAPACITY, TIMEOUT).
 */
int plan_search_to(plan_ctx* ctx, int N, const void* states, const plan_edges* edges, const double* endpoints,
                   int warm, int32_t* path, int path_cap, int32_t* path_len, double* cost);

/* Bounds of the search kernel's device loops: at most max_sweeps frontier
 * sweeps (default N+1, the Bellman-Ford bound) and spin_limit polls of the
 * grid barrier (default 2^24).  0 keeps the default.  When a bound runs out
 * the kernel stops and plan_wait returns PLAN_ERR_TIMEOUT; the context stays
 * usable. */
int plan_set_search_limits(plan_ctx* ctx, int max_sweeps, int64_t spin_limit);

/* Convex obstacles in position space for the keep-out cut (Assumption 1):
 * obstacle o = {z in R^m : A_r z <= b_r, r = off[o] .. off[o+1]-1}. */
typedef struct {
    int n;                 /* number of obstacles, 0 .. 1<<20 */
    const int32_t* off;    /* device int32 [n+1], off[0] = 0, non-decreasing */
    int max_rows;          /* host bound on the rows of any obstacle, 1..16 */
    const void* A;         /* device [R][m], the model's input type (may be NULL when R = 0) */
    const void* b;         /* device [R], the model's input type (may be NULL when R = 0) */
} plan_obstacles;

/*
 * cutGraph (Algorithm 1, Sec. III-B, Algorithm 2 cutHeuristic, Cut-QP):
 * remove from a built graph every (edge, duration) whose curve may meet an
 * obstacle.  By Property 1 a curve is collision-free when the convex hull of
 * its control points P_0..P_p misses the obstacle; with the margins
 * G[l][r] = A_r . P_l - b_r the hull meets obstacle O iff
 *     delta* = min over lambda in the simplex of max_r (G^T lambda)_r <= 0,
 * the feasibility question that the Cut-QP's slack answers (touching counts as
 * meeting).  The control points are those of the edge build (Lemma 1, the
 * model's interior reading); the margins are defined in the canonical FP64
 * order (each half summed left to right, halves added, facet products summed
 * left to right, then b subtracted).  Algorithm 2's checks (a control point
 * with every margin <= 0: hit; a facet with every margin > 0: miss) and a
 * bounding-box screen decide most (edge, obstacle) pairs in FP32 within
 * proven error bands; the rest go through the matrix game solved in FP32, then
 * FP64, each answer accepted only with a weak-duality certificate.  A game that
 * no FP64 certificate decides (|delta*| at the FP64 rounding level) is decided
 * by the sign of its computed value and counted in plan_info.cut_ties.
 * The obstacles are taken as given (no tightening: inflate b to add a margin).
 *
 *   N, states  the states the graph was built on (device [N][n])
 *   nT, T      host [nT]: the durations the graph was built with (bit t of an
 *              edge mask refers to T[t])
 *   in         device CSR from plan_build_edges (read only; its count must be
 *              <= in->cap, else device status INVALID_ARG)
 *   obst       obstacles (see plan_obstacles); an obstacle with 0 rows is the
 *              whole space and cuts every edge
 *   out        caller-owned device CSR, no array shared with in: the edges with
 *              at least one duration left, sorted as in; mask = in.mask with the
 *              colliding durations cleared; w, tidx = the cheapest remaining
 *              duration (copied when in's best duration survives, else re-costed
 *              in canonical FP64, ties to the lower index); out->cap >= in's
 *              count always suffices
 * Errors: INVALID_ARG / UNSUPPORTED on the host; on the device (plan_wait):
 * CAPACITY with detail OUTPUT when out->cap is too small (count written), or
 * when the context's game lists were too small (they grow at plan_wait: repeat
 * the call); UNSUPPORTED if an obstacle has more than max_rows rows.
 */
int plan_cut_edges(plan_ctx* ctx, int N, const void* states, int nT, const double* T, const plan_edges* in,
                   const plan_obstacles* obst, const plan_edges* out);

/*
 * closestPoint and adjacentHyperplane (Algorithm 2; the separating hyperplane
 * between a node and an obstacle of Sec. III-D): for every point p and
 * obstacle o, the point z of o nearest to p (Euclidean projection onto
 * {z : A z <= b}), its distance d, and the hyperplane through z with unit
 * normal toward p, h = (p - z) / d, l = h . z (the obstacle lies in
 * {h . z <= l}, p at distance d on the other side).  A point inside its
 * obstacle: d = 0, z = p, h = 0, l = 0.  Also, per point, the nearest obstacle
 * (ties to the lower index).  The obstacle's faces and edges (edges as
 * segments) are computed in FP64 once per call; each (point, obstacle) then
 * takes, in FP32, the nearest of the face projections that land inside the
 * obstacle and of the edge segments' closest points.  Model: m = 2 or 3
 * (gamma and degree do not matter).
 *   P            number of points, 0 .. 1<<24
 *   points       device [P][m], the model's input type
 *   obst         obstacles (plan_obstacles, at most 16 rows each)
 *   closest      device float [P][n][m] or NULL
 *   plane        device float [P][n][m+1] (h, then l) or NULL
 *   dist         device float [P][n] or NULL
 *   nearest      device int32 [P] (-1 when n = 0) or NULL
 *   nearest_dist device float [P] (+inf when n = 0) or NULL
 * Errors: INVALID_ARG / UNSUPPORTED on the host; UNSUPPORTED on the device for
 * an obstacle above max_rows.
 */
int plan_obstacle_planes(plan_ctx* ctx, int P, const void* points, const plan_obstacles* obst, float* closest,
                         float* plane, float* dist, int32_t* nearest, float* nearest_dist);

/*
 * adjacentHyperplane for the nearest obstacle only (Sec. III-D: the MPC keeps
 * node k on its side of the plane between it and its closest obstacle): per
 * point the nearest obstacle as plan_obstacle_planes finds it, then that
 * pair's plane (h, l) with unit normal toward the point.  A point inside an
 * obstacle, or with no obstacle at all, gets h = 0, l = 0 (no constraint).
 *   nearest_plane  device float [P][m+1] (h, then l)
 *   nearest        device int32 [P] or NULL (-1 when n = 0)
 *   nearest_dist   device float [P] or NULL
 * Everything else, and the errors, as plan_obstacle_planes.
 */
int plan_nearest_planes(plan_ctx* ctx, int P, const void* points, const plan_obstacles* obst, float* nearest_plane,
                        int32_t* nearest, float* nearest_dist);

/* MPC refinement QP (Sec. III-D, Eq. (MPC)) of a batch of B problems on the
 * context's model (m <= 3, gamma <= 4, degree <= 9):
 *   min  sum_{k<H} (x_k - r_k)'Q(x_k - r_k) + (x_{k+1} - x_k)'F(x_{k+1} - x_k)
 *        + u_k'R u_k  +  (x_H - r_H)'V(x_H - r_H)
 *   s.t. x_{k+1} = A x_k + B u_k (exact discretisation of the chain of
 *        integrators, u the gamma-th derivative), x_0 = the given state,
 *        x_H = r_H, Theorem 1's reach rows of duration dt on every segment
 *        (the model's derivative bounds minus its tighten margin), every
 *        control point of segment k (not x_0 itself) on the side h.z >= l of
 *        plane k unless h = 0, and every control point but the first of a
 *        segment inside the keep-in polytope A_d z <= b_d.
 * x is derivative-major (positions, velocities, ...) as the graph's states.
 * Weights are diagonal; Q, F, V have n = m gamma entries, R has m.  The
 * problem is strictly convex; each is solved exactly (active-set method, in
 * FP64) on the GPU. */
typedef struct {
    int horizon;              /* H segments, gamma <= H <= 64 / m */
    double dt;                /* segment duration, > 0 */
    const double* Q;          /* host [n] > 0: distance to the reference */
    const double* F;          /* host [n] > 0: step between consecutive nodes (path length) */
    const double* R;          /* host [m] > 0: input */
    const double* V;          /* host [n] > 0: terminal */
    int keepin_rows;          /* 0 .. 16 */
    const double* keepin_A;   /* host [keepin_rows][m] or NULL */
    const double* keepin_b;   /* host [keepin_rows] or NULL */
} plan_mpc_params;

enum { PLAN_MPC_OK = 0, PLAN_MPC_INFEASIBLE = 1, PLAN_MPC_ITERATION_LIMIT = 2 };

/*
 *   B       problems, 0 .. 1<<24
 *   x0      device double [B][n]: measured state of every problem
 *   ref     device double [B][H+1][n]: reference nodes r_0 .. r_H
 *   planes  device float [B][H][m+1]: plane (h, l) of segment k (the output
 *           of plan_nearest_planes at the nodes x_0 .. x_{H-1} of the
 *           current iterate); h = 0 means no safety rows
 *   x       device double [B][H+1][n]: optimal nodes (x_0 = x0)
 *   u       device double [B][H][m]: optimal inputs
 *   obj     device double [B]: optimal objective value
 *   status  device int32 [B]: PLAN_MPC_OK, PLAN_MPC_INFEASIBLE or
 *           PLAN_MPC_ITERATION_LIMIT (x, u, obj then describe the last iterate)
 *   iters   device int32 [B] or NULL: active-set steps taken
 *   nodes   device double [B][H][m] or NULL: the positions of x_0 .. x_{H-1}
 *           (the points of the next round's plan_nearest_planes)
 * Asynchronous on the context stream; host errors INVALID_ARG (bad sizes or
 * weights) and UNSUPPORTED (model or problem size); per-problem outcomes go
 * to status, not to plan_wait.  An SQP refinement alternates
 * plan_nearest_planes at the new nodes and plan_mpc_qp.
 */
int plan_mpc_qp(plan_ctx* ctx, int B, const plan_mpc_params* prm, const double* x0, const double* ref,
                const float* planes, double* x, double* u, double* obj, int32_t* status, int32_t* iters,
                double* nodes);

/* Weights of the refinement objective (defaults 1, 1, 0.1). */
typedef struct {
    double w_snap;  /* weight of the snap energy */
    double mu;      /* weight of the barrier terms */
    double delta;   /* relaxation point of the log-barrier (> 0) */
} plan_refine_weights;

/*
 * Differentiable refinement of Bezier segments (one free polytope each): for
 * segment s with control points P_s (degree p = model degree, m axes), duration
 * T_s and polytope {x : A x <= b},
 *   loss_s = w_snap J_snap + mu sum phi_delta(margin)
 * where the margins are c_k -/+ Q^(k)_j on every hodograph control point
 * (Theorem 1 per axis, k = 1..gamma) and b_r - A_r P_l for the interior control
 * points (Property 1); phi_delta is the log-barrier -log m relaxed to its C^2
 * quadratic extension below delta; J_snap = integral over [0, T] of
 * ||b''''(t)||^2 (exact Gram form of the degree p-4 fourth-derivative curve).
 * Supported models: (m, gamma, p) in {(3,3,7), (2,2,5)}.
 *   S         number of segments
 *   P         device float [S][p+1][m]
 *   T         device float [S], > 0
 *   A, b      device float [S][rmax][m], [S][rmax]; rows >= nrows[s] ignored
 *   nrows     device int32 [S], 0..rmax
 *   weights   host (NULL: defaults)
 *   grad_loss device float [S] upstream gradient, or NULL for the forward pass only
 *   loss      device float [S] (may be NULL when grad_loss != NULL)
 *   dP, dT    device float [S][p+1][m], [S]: d(sum_s grad_loss_s loss_s) with
 *             respect to every control point and T (ignored when grad_loss is NULL)
 */
int plan_refine(plan_ctx* ctx, int S, const float* P, const float* T, const float* A, const float* b,
                const int32_t* nrows, int rmax, const plan_refine_weights* weights, const float* grad_loss,
                float* loss, float* dP, float* dT);

/* One query of a batched search. */
typedef struct {
    int N;
    const void* states;      /* device [N][n] */
    plan_edges edges;        /* device CSR of this query */
    double start_pos[4];     /* host, first m used */
    double goal_pos[4];
    int32_t* path;           /* device [path_cap] */
    int path_cap;
    int32_t* path_len;       /* device [1] */
    double* cost;            /* device [1] */
    int32_t* status;         /* device [1]: OK, NO_PATH, CAPACITY (path_len = needed), TIMEOUT, INVALID_ARG */
} plan_search_query;

/*
 * Batched findPath: the same computation as plan_search for many queries, one
 * 1024-thread block per query (block barriers, no grid barrier).  Per-query
 * outcomes go to each query's status word; NO_PATH is not a batch error.
 * plan_prepare_search_batched uploads the descriptors (may allocate/wait);
 * plan_search_batched only launches (capturable in a CUDA graph).
 */
int plan_prepare_search_batched(plan_ctx* ctx, int Q, const plan_search_query* queries);
int plan_search_batched(plan_ctx* ctx);

/*
 * plan_search_noalloc -- the search of plan_search for callers that cannot
 * allocate device memory while they plan.  The paper has no counterpart; it is
 * a deployment variant.  Typical callers: a replanning loop with a hard
 * per-tick deadline (cudaMalloc/cudaFree may block, and cudaFree synchronises
 * the whole device), and processes whose device memory belongs to a pool
 * allocator that the planner may not draw from.
 *
 * No context is needed and nothing is allocated: all scratch (status word,
 * grid-barrier counters, distance / predecessor / frontier arrays) lives in
 * one static device array sized for N <= 65536 vertices (about 1.9 MB:
 * 65536 x 28 bytes of per-vertex arrays plus 32 KB of per-block candidates
 * and the status block), held by every GPU that loads the library until the
 * process exits.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress, with that device current) and caches it for
 * the life of the process; make that first call before any stream capture.
 * The address belongs to the device's primary context (the CUDA runtime's):
 * after cudaDeviceReset, or with another context current, the cached address
 * is no longer valid, so do not call this entry point again in that process.
 * Every call on a device shares the array and it keeps the last call's
 * contents (the call clears the status and barrier words itself, and the
 * kernel initialises the per-vertex arrays), so calls whose work overlaps on
 * the GPU race: issue them on one stream or order them with events.
 * The device loops have fixed bounds: at most N+1 frontier sweeps (the
 * Bellman-Ford bound) and 2^24 polls of a grid barrier; when one runs out the
 * status is TIMEOUT (plan_set_search_limits does not apply here).
 *
 *   m, gamma     model (positions are the first m entries of each state)
 *   input        PLAN_IN_F64 / PLAN_IN_F32 storage of states
 *   w_f64        1 if edges->w holds doubles, 0 for floats
 *   N, states, edges, start_pos, goal_pos, path, path_cap, path_len, cost:
 *                as plan_search
 *   status       device int32 [1]: the device status (OK, NO_PATH, TIMEOUT,
 *                CAPACITY, INVALID_ARG), written on the stream
 *   cuda_stream  cudaStream_t (NULL = legacy default stream)
 * Returns PLAN_ERR_CAPACITY (before launching anything) when N > 65536,
 * PLAN_ERR_INVALID_ARG for bad arguments, PLAN_ERR_CUDA if a launch fails.
 */
int plan_search_noalloc(int m, int gamma, int input, int w_f64, int N, const void* states, const plan_edges* edges,
                        const double* start_pos, const double* goal_pos, int32_t* path, int path_cap,
                        int32_t* path_len, double* cost, int32_t* status, void* cuda_stream);

/* Synchronise the context stream, return the device status of the work
 * issued since the previous plan_wait, and fill *info (may be NULL). */
int plan_wait(plan_ctx* ctx, plan_info* info);

/*
 * Host-only: the library's FP64 coefficient tables for nT durations (no GPU
 * needed).  Each entry is the correctly rounded double of an exact rational
 * function of T.
 *   D [nT][p+1][2g]  control points (Lemma 1, degree-elevated to p)
 *   H [nT][Rax][2g]  reach rows, Rax = sum_{k=1..g} (p-k+1), k-major then j
 *   C [nT][g][p][2g] consecutive differences of the degree-p control points of
 *                    b^(d), d = 0..g-1 (rows of Eq. BezDef's state-space matrix)
 */
int plan_model_tables(const plan_model* model, int nT, const double* T, double* D, double* H, double* C);

/* Work accounting: when enabled, every plan_build_edges also launches an
 * (untimed, extra) counting kernel whose totals plan_wait reports in
 * plan_info.work_*.  Off by default. */
int plan_set_accounting(plan_ctx* ctx, int enable);

/* Per-kernel timing with CUDA events on the context stream (off by default).
 * plan_timing returns the accumulated milliseconds and launch counts since
 * the last reset (synchronises the stream). */
int plan_set_timing(plan_ctx* ctx, int enable);
int plan_timing(plan_ctx* ctx, double* pair_ms, int64_t* pair_launches, double* search_ms,
                int64_t* search_launches, int64_t* total_launches, int reset);

/* Timing of plan_cut_edges calls made while plan_set_timing is on: the
 * summed milliseconds of the first (screening) pass and of whole calls, and
 * the number of calls, since the last reset (synchronises the stream). */
int plan_cut_timing(plan_ctx* ctx, double* scan_ms, double* cut_ms, int64_t* cuts, int reset);

/* Measurement helper (no counterpart in the paper): the sustained issue rate
 * of the FP32 (or FP64) lane operations that make up the pair kernels' work, measured
 * on the current device by a full-occupancy kernel of independent register
 * chains timed with CUDA events (two launches; the second is timed).
 *   mix   0: one add and one max of an absolute value per step (a reach or
 *         free row of one pair); 1: one fused multiply-add per step; 2 and 3:
 *         the same in FP64 (the canonical FP64 pair kernel)
 *   iters chain steps per thread, 1 .. 2^24 (about 2^16 runs for milliseconds)
 *   lane_ops_per_s  host out: lane operations per second (an FMA counts one)
 *   ms    host out (may be NULL): duration of the timed launch
 * Synchronous; INVALID_ARG for bad arguments, CUDA if a launch fails. */
int plan_measure_lane_rate(int mix, int iters, double* lane_ops_per_s, double* ms);

const char* plan_status_string(int status);
const char* plan_last_error(plan_ctx* ctx);
const char* plan_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PLAN_H */
