// Internal definitions shared by the CUDA translation units of libplan.
#pragma once

#include <cstdint>

#include "../../include/plan.h"

namespace plan {

constexpr int RMAX = 16;        // rows per free polytope (ABI limit)
constexpr int NT_MAX = 32;      // durations per call (one bit each in the mask)
constexpr int TILE = 64;        // tile side of the FP32 pair kernel (states per side)
constexpr int TILE64 = 32;      // tile side of the FP64 pair kernel
constexpr int NK_MAX = 65535;   // members per polytope (16-bit local index in re-check entries)
constexpr int PIPE_FP64 = 3;    // plan_set_tile pipeline: the canonical FP64 pair kernel (FP64 models)

// Host: FP64 tables (see plan_tables.cpp).
int reach_rows(int g, int p);
void exact_tables(int g, int p, int interior, int nT, const double* T, double* D, double* H, double* C);

// Layout of the per-duration tables uploaded to the device (depends on g, p only).
struct TabLayout {
    int g, p, tg, rax, ni;
    // FP32 fast table (floats): reach rows scaled by 1/(c_k - eps) in kernel
    // order, interior control points, cost rows, column maxima for the bands.
    int f_H, f_D, f_C, f_HC, f_DC, f_stride;
    // FP64 canonical table (doubles): reach rows (k-major), all control points, cost rows.
    int e_H, e_D, e_C, e_stride;
};

inline TabLayout tab_layout(int g, int p) {
    TabLayout L;
    L.g = g;
    L.p = p;
    L.tg = 2 * g;
    L.rax = 0;
    for (int k = 1; k <= g; ++k) L.rax += p - k + 1;
    L.ni = p - 1;
    L.f_H = 0;
    L.f_D = L.f_H + L.rax * L.tg;
    L.f_C = L.f_D + L.ni * L.tg;
    L.f_HC = L.f_C + g * p * L.tg;
    L.f_DC = L.f_HC + 2 * g;
    L.f_stride = (L.f_DC + 2 * g + 3) & ~3;
    L.e_H = 0;
    L.e_D = L.e_H + L.rax * L.tg;
    L.e_C = L.e_D + (p + 1) * L.tg;
    L.e_stride = L.e_C + g * p * L.tg;
    return L;
}

// Device-side counters and status of the current call (mirrors plan_info).
struct DevInfo {
    int status;
    int detail;
    unsigned long long memberships;
    unsigned long long slots;
    unsigned long long candidates;
    unsigned long long checks;       // sum over queries of candidates * nT
    unsigned long long reach_pass;
    unsigned long long feasible;
    unsigned long long rechecks;
    unsigned long long edges;
    unsigned long long search_iters;
    unsigned long long need_slots;
    unsigned long long need_rechecks;
    unsigned long long items;
    unsigned long long screened;     // pairs the reach screen passed to the full rows
    unsigned int ticket;
    int max_rows_seen;
    int start;
    int goal;
    // search scratch
    unsigned long long near_d[2];
    unsigned long long bar[3];       // grid-barrier words, used in rotation: arrivals | raised flags << 32
    int path_len;
    unsigned long long work[3];
    // keep-out cut counters (contiguous: cleared together)
    unsigned long long cut_units;    // (edge, T) checked
    unsigned long long cut_tests;    // (edge, T, obstacle) screened
    unsigned long long cut_box;      // missed by the obstacles' certified boxes
    unsigned long long cut_near;     // entries of the pair list (the rest)
    unsigned long long cut_step1;    // hit: a control point inside (FP32, certain)
    unsigned long long cut_step2;    // missed: one separating facet (FP32, certain)
    unsigned long long cut_games;    // matrix games solved in FP32
    unsigned long long cut_lp64;     // entries settled in FP64
    unsigned long long cut_ties;     // FP64 games without a certificate either way
    int shard_lo, shard_hi;          // source rows [lo, hi) of the first query's shard
    int tchunks;                     // duration chunks per tile of the current edge build (k_batch)
};

enum Detail {
    DET_NONE = 0,
    DET_SLOTS = 1,
    DET_RECHECK = 2,
    DET_OUTPUT = 3,
    DET_ROWS = 4,
    DET_NK = 5,
    DET_PATHCAP = 6,
    DET_BARRIER = 7,
    DET_SWEEPS = 8,
    DET_WALK = 9,
    DET_CUTLIST = 10,
    DET_CUTIN = 11
};

// One query of a batch (device array; host-known offsets into the shared
// scratch, caller-owned input/output pointers).
struct QueryDesc {
    int N, K, nT, W;           // W: 32-bit words per membership mask
    int tabOff;                // first duration of this query in the table arrays
    int kOff;                  // per-polytope arrays (counts, centers, ...), K+1 entries each
    long long maskOff;         // memMask   [N][W]
    long long listOff;         // members / localIdx [K][N]
    long long rowsOff;         // row arrays [K * max_rows]
    long long rowOff;          // rowCount  [N]
    const void* states;
    const int* poly_off;
    const void* A;
    const void* b;
    int32_t* row_off;
    int32_t* col;
    void* w;
    uint8_t* tidx;
    uint32_t* mask;
    long long cap;
    int64_t* count;
    int shard, nshard;         // rows of shard `shard` of `nshard` (equal-work contiguous ranges); 0, 1: all rows
};

// Everything a build kernel needs, passed by value.
struct BuildParams {
    int Q;                     // queries in the batch
    int maxK;                  // max K over queries
    int maxN;                  // max N over queries
    int m, g, p;
    int cost_mode, in_f32, arith, max_rows;
    int tile;                  // tile side of the pair kernel (autotuned, <= TILE)
    int tchunks;               // duration chunks per tile (work items = tiles x tchunks)
    int itemTarget;            // > 0: k_batch picks the chunks per tile for about this many items
    int pipeline;              // FP32 pair kernel: 0 screened, 1 warp-specialised (64-state tiles), 2 unscreened
    int w64;                   // output weights are doubles (FP64 model)
    int cost64;                // FP64 model on the FP32 pair kernels: canonical FP64 cost pass after compaction
    int maxT;                  // most durations of any query
    double* half64;            // [totN][maxT][2][p * DR * m] FP64 cost halves (FP64 cost pass)
    double eps;
    const QueryDesc* qd;       // [Q]
    const long long* pfxMask;  // [Q+1] prefix of N*W        (membership threads)
    const long long* pfxPoly;  // [Q+1] prefix of K          (one CTA per polytope)
    const long long* pfxRows;  // [Q+1] prefix of K*max_rows (row threads)
    const long long* pfxN;     // [Q+1] prefix of N          (one warp per row)
    long long* qSlot;          // [Q+1] device-computed prefix of slots
    long long* qItem;          // [Q+1] device-computed prefix of tiles
    long long* qMem;           // [Q+1] device-computed prefix of memberships (row segments)
    long long totMask, totPoly, totRows, totN;
    const float* tab32;        // [nT_total][f_stride]
    const double* tab64;       // [nT_total][e_stride]
    double lim64[4];           // c_k - eps
    TabLayout L;
    // scratch (shared by all queries, indexed with the descriptor offsets)
    uint32_t* memMask;
    int* counts;
    int* members;
    int* localIdx;
    int* segKL;                // [memberships] row segment g -> polytope k << 16 | local index li
    float* centers;            // [kOff][4]
    double* blim64;
    float* A32;                // [rows][m]
    float* blim32;
    float* bc32;
    long long* resOff;         // [kOff] slot offset of each polytope, relative to qSlot[q]
    int* memOff;               // [kOff] membership offset of each polytope, relative to qMem[q]
    int* itemOff;              // [kOff + p] first item of the p-th polytope of the item order (prefix, + total)
    int* kPerm;                // [kOff + p] polytope at position p of the item order (tile area, largest first)
    int* ntile;                // j-tiles | i-tiles << 16 of each polytope
    int* tsize;                // j-tile side | i-tile side << 16
    int* iRange;               // members [a, b) of each polytope whose ids lie in the query's row range: a | b << 16
    int* rowRange;             // [Q][2] row range [lo, hi) of each query's shard (written by k_setup)
    uint32_t* resBits;
    unsigned long long* resKey;
    int* emitPre;
    unsigned long long* recheck;
    int* rowCount;
    long long slotCap, recheckCap;
    DevInfo* info;
};

struct SearchParams {
    int N, m, n, in_f32, w_f64;
    const void* states;
    const int32_t* row_off;
    const int32_t* col;
    const void* w;
    const int64_t* count;
    long long cap;
    double start[4], goal[4];
    const double* endpoints;   // device [2][m] start then goal, read at run time instead of start/goal (or null)
    unsigned long long* dist;  // [N] bit patterns of non-negative doubles
    unsigned long long* bestU; // [N]
    int* pred;                 // [N]
    unsigned long long* best16;  // [N][2] (dist[u] bits, u) of each vertex's predecessor, 16-byte aligned, or null
    unsigned long long* last;  // [N] distance each vertex last relaxed its out-edges from
    unsigned long long* near_blk;  // [4][blocks] per-block nearest candidates (bits, id) for start, goal
    int32_t* path;
    int path_cap;
    int32_t* path_len;
    double* cost;
    DevInfo* info;
    int max_sweeps;
    long long spin_limit;
    int walk_smem;             // vertices whose pred[] the walk stages in shared memory
};

// Shared-memory staging of pred[] for the walk (ints; 64 KB).
constexpr int SEARCH_WALK_SMEM = 16384;
// Blocks of the cooperative search (one per SM) that its scratch provides for.
constexpr int SEARCH_MAX_BLOCKS = 1024;
// Owned vertices per search block whose out-edge range and last-relaxed
// distance live in shared memory (the rest are read from global memory).
constexpr int SEARCH_OWN_CAP = 2048;

// One query of a batched search (device array).
struct SearchQueryDesc {
    int N, pad;
    long long off;             // scratch offset (prefix of N)
    const void* states;
    const int32_t* row_off;
    const int32_t* col;
    const void* w;
    const int64_t* count;
    long long cap;
    double start[4], goal[4];
    int32_t* path;
    int path_cap, pad2;
    int32_t* path_len;
    double* cost;
    int32_t* status;           // per-query plan_status (OK, NO_PATH, CAPACITY, TIMEOUT, INVALID_ARG)
};

struct BatchSearchParams {
    int Q, m, n, in_f32, w_f64, max_sweeps;
    const SearchQueryDesc* qd;
    unsigned long long* dist;
    unsigned long long* bestU;
    int* pred;
    unsigned char* front;      // [2 * total N]
    DevInfo* info;
};

struct RefineParams {
    long long S;
    int m, g, p, rmax;
    const float* P;        // [S][p+1][m]
    const float* T;        // [S]
    const float* A;        // [S][rmax][m]
    const float* b;        // [S][rmax]
    const int32_t* nrows;  // [S]
    float bound[4];
    float w_snap, mu, delta;
    const float* grad_loss;  // [S] or null (forward only)
    float* loss;           // [S] or null
    float* dP;             // [S][p+1][m]
    float* dT;             // [S]
};

// Keep-out cut of a built edge graph (plan_cut.cu).
constexpr int CUT_RMAX = 16;     // rows per obstacle
constexpr int CUT_CHUNK = 2048;  // edges per compaction chunk

struct CutParams {
    int m, g, p, nT, in_f32, w_f64, cost_mode;
    int N, n_obst, max_orows;
    const void* states;
    // input CSR (from the edge build) and its count on the device
    const int32_t* row_in;
    const int32_t* col_in;
    const void* w_in;
    const uint8_t* t_in;
    const uint32_t* mask_in;
    const int64_t* count_in;
    long long cap_in;
    // output CSR
    int32_t* row_out;
    int32_t* col_out;
    void* w_out;
    uint8_t* t_out;
    uint32_t* mask_out;
    int64_t* count_out;
    long long cap_out;
    // obstacles (caller arrays) and their FP32 copies, max_orows rows per obstacle
    const int32_t* obst_off;
    const void* A;
    const void* b;
    float* orow;               // [n_obst * max_orows][4] {A_0, A_1, A_2 (0 when m = 2), b}, 16-byte aligned
    float* okb;                // [n_obst * max_orows][2] band coefficients {K ||A_r||_1, K |b_r|}
    float* obox;               // [n_obst][8] certified bounds {lo_0, lo_1, lo_2, -, hi_0, hi_1, hi_2, -}
                               // (m = 2: {lo_0, lo_1, hi_0, hi_1} in the first four)
    int* ocount;               // [n_obst] rows of each obstacle
    const double* tab64;       // [nT][L.e_stride] canonical tables (control points, cost rows)
    const float* tab32;        // [nT][(p+1) * 2g] FP32 control-point table
    TabLayout L;
    int32_t* src;              // [cap_in] start vertex of each edge
    uint32_t* hit;             // [cap_in] durations whose curve meets an obstacle
    unsigned long long* list32;  // pair list: (edge * nT + T) << 20 | obstacle
    long long cap32;
    long long* chunk;          // [nchunks + 1] kept edges per chunk, then their exclusive prefix
    int32_t* pos;              // [cap_in + 1] output index of each edge (exclusive prefix of kept)
    long long nchunks;
    DevInfo* info;
};

// Goal-rooted search with a warm start (plan_search.cu).
struct GoalSearchParams {
    int N, m, n, in_f32, w_f64, warm, max_sweeps;
    long long spin_limit;      // grid-barrier poll bound
    const void* states;
    const int32_t* row_off;
    const int32_t* col;
    const void* w;
    const int64_t* count;
    long long cap;
    const double* endpoints;   // device [2][m]: start, goal positions
    double* d;                 // [N] distance to the goal vertex (kept for the next call)
    int* succ;                 // [N] next vertex toward the goal (kept)
    double* wsucc;             // [N] weight of that edge (kept)
    unsigned* anc;             // [2][N] pointer-jumping links, ancestor | chain ok << 31 (two buffers)
    unsigned long long* near_blk;  // [4 * blocks] per-block nearest start/goal candidates
    int* prev;                 // device [2]: goal vertex and N of the last call (-1 when none)
    int32_t* path;
    int path_cap;
    int32_t* path_len;
    double* cost;
    DevInfo* info;
};

// closestPoint / adjacentHyperplane (plan_planes.cu).
struct PlanesParams {
    int m, in_f32, P, n_obst, max_orows;
    const void* points;        // [P][m], input type
    const int32_t* obst_off;
    const void* A;
    const void* b;
    int max_edges;             // edge slots per obstacle (max_orows in 2-D, max_orows (max_orows - 1) / 2 in 3-D)
    float* orow;               // [n_obst * max_orows][4] {A_0, A_1, A_2, b}
    float* face;               // [n_obst * max_orows][4] unit normal, offset
    float* edge;               // [n_obst * max_edges][16] base point, t_lo; direction, t_hi; normals (see plan_planes.cu)
    int* nedge;                // [n_obst] edges found
    int* ocount;               // [n_obst]
    float* closest;            // [P][n_obst][m] or null
    float* plane;              // [P][n_obst][m+1] or null
    float* dist;               // [P][n_obst] or null
    int32_t* nearest;          // [P] or null
    float* nearest_dist;       // [P] or null
    unsigned long long* keys;  // [P] nearest keys (distance bits << 32 | obstacle), or null
    float* nearest_plane;      // [P][m+1] plane of the nearest obstacle (h = 0, l = 0 when none), or null
    const int32_t* pair_obst;  // pair mode: [P] one obstacle per point (-1: none); outputs indexed by point
    float* ub;                 // nearest-only mode: [P] upper bound of the nearest distance (prunes far pairs), or null
    DevInfo* info;
};

// MPC refinement QP (plan_mpc.cu): one warp per problem, FP64.
constexpr int MPC_OK = 0, MPC_INFEASIBLE = 1, MPC_MAXITER = 2;
constexpr int MPC_NV_MAX = 64;      // inputs per problem (m H)
constexpr int MPC_KEEP_MAX = 16;    // keep-in rows
struct MpcParams {
    int B, m, g, p, H, nv, rax, nkeep, warps, max_iter;
    const double* tab;      // device table: A, B, D, reach rows, their bounds, Q, F, V, R, keep-in rows
    const double* x0;       // [B][n]
    const double* ref;      // [B][H+1][n]
    const float* planes;    // [B][H][m+1]
    double* x;              // [B][H+1][n]
    double* u;              // [B][H][m]
    double* obj;            // [B]
    int32_t* status;        // [B]
    int32_t* iters;         // [B] or null
    double* nodes;          // [B][H][m] positions of x_0 .. x_{H-1}, or null
    double* J0;             // [nv][nv] scratch: L^-T of the batch's Hessian
    int j0_ready;           // J0 already holds the factor of this table (the setup kernel is skipped)
};
int mpc_table_size(int m, int g, int p, int rax, int nkeep);
size_t mpc_smem(int m, int g, int p, int rax, int nkeep, int H, int W);
size_t mpc_setup_smem(int m, int g, int p, int rax, int nkeep, int H);
int launch_mpc(const MpcParams& P, void* stream, int* launches);

// Launchers (plan_build.cu / plan_search.cu / plan_refine.cu); return cudaError_t as int.
int launch_build(const BuildParams& P, void* stream, int num_sms, int ctas_per_sm, void* ev_pair_begin,
                 void* ev_pair_end, int* launches);
int launch_search(const SearchParams& P, void* stream, int num_sms, int* launches);
int launch_search_batched(const BatchSearchParams& P, void* stream, int* launches);
int launch_search_to(const GoalSearchParams& G, void* stream, int num_sms, int* launches);
int launch_account(const BuildParams& P, void* stream, int num_sms, unsigned long long* work);
bool model_supported(int m, int g, int p);
bool tc_supported(int m, int g, int p);
bool refine_supported(int m, int g, int p);
int launch_refine(const RefineParams& R, void* stream, int* launches);
int launch_cut(const CutParams& C, void* stream, int num_sms, int* launches, void* ev_scan_begin, void* ev_scan_end);
int launch_planes(const PlanesParams& Q, void* stream, int num_sms, int* launches);

}  // namespace plan
