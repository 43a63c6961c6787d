// Keep-out cut kernels for sm_103a: remove from a built edge graph every
// (edge, duration) whose curve may meet an obstacle, then re-compact the CSR.
//
// Method (arXiv 2411.13507, Sec. III-B "Cut Graph", Algorithm 2, Cut-QP):
// Property 1 makes a curve collision-free when the convex hull of its control
// points misses every obstacle O = {z : A z <= b}.  With the margins
// G[l][r] = A_r . P_l - b_r of control point l against facet r, the hull meets
// O iff the value of the matrix game
//     delta* = min over lambda in the simplex of max_r (G^T lambda)_r
// is <= 0; that is the linear feasibility question whose slack the Cut-QP
// minimises.  Algorithm 2's first two checks are the game's cheapest
// certificates: a control point with every margin <= 0 is a hit, a facet
// with every margin > 0 a miss.  The result is defined on the canonical FP64
// margins (halves summed left to right without FMA, as in the edge build);
// the FP32 passes take only the decisions that their error bands prove.
//
//  Boxes (in k_cut_prep): a certified bounding box of every obstacle, each side
//    backed by a dual vector y >= 0 with A^T y = +-e_a (a certificate of the
//    game for every curve beyond that side).
//  Pass A (k_cut_scan): one lane per (edge, T); FP32 control points, their
//    box against every obstacle's box within error bounds; the pairs that no
//    box separates form the pair list.
//  Pass B (k_cut_pair): one thread per listed pair: FP32 margins with bands,
//    Algorithm 2's two checks (a point certainly inside -> hit, a facet
//    certainly separating -> miss), else the game by the simplex method in
//    registers.  Weak duality turns its solution into certificates: any
//    lambda >= 0 with G^T lambda < 0 proves a hit, any y >= 0 with G y > 0 a
//    miss; both are checked against G's error bands.
//  FP64 settling (in pass B, by the whole warp): canonical FP64 margins,
//    Algorithm 2's two checks exactly, the FP32 game's mixes as certificates,
//    then the game in FP64 with certificates against the rounding of the
//    check itself.  A game certified neither way has |delta*| at the rounding
//    level: a tie, decided by the sign of the computed value and counted.
//  Compaction: kept = mask & ~hit != 0; chunk counts, one scan, the fill (an
//    edge whose cheapest duration was cut is re-costed in canonical FP64 over
//    the durations left), the row offsets.
#include <cuda_runtime.h>

#include <cstdint>

#include "plan_internal.h"

namespace plan {

namespace {

#define CDEV __device__ __forceinline__

constexpr float U32 = 5.9604644775390625e-08f;  // 2^-24
constexpr double U64 = 1.1102230246251565e-16;  // 2^-53
// Band of an FP32 margin around the canonical FP64 one, per unit of
// (||A_r||_1 S + |b_r|), where S bounds every sum |D| . |x| of a control
// point: conversions of the table, the state and the facet (3 u), the
// control-point sums (g + 1 u), the facet products and the subtraction
// (m + 1 u) add up to at most 12 u for g, m <= 3; 32 u leaves room for the
// rounding of the band itself and of the comparisons built on it.
constexpr float KO = 32.f * U32;
constexpr int GAME_ITERS = 96;  // simplex pivots before an entry is handed on
constexpr unsigned long long OBST_BITS = 20;

CDEV void cut_status(DevInfo* info, int code, int detail) {
    if (atomicCAS(&info->status, 0, code) == 0) atomicExch(&info->detail, detail);
}
CDEV bool cut_failed(const DevInfo* info) { return *((volatile const int*)&info->status) != 0; }

CDEV float ld32(const void* p, long long i, int f32) {
    return f32 ? ((const float*)p)[i] : (float)((const double*)p)[i];
}
CDEV double ld64(const void* p, long long i, int f32) {
    return f32 ? (double)((const float*)p)[i] : ((const double*)p)[i];
}

// One global atomic per block for a per-thread count (every thread calls it).
CDEV void cut_block_add(unsigned long long* dst, unsigned long long v) {
    __shared__ unsigned long long s_acc;
    if (threadIdx.x == 0) s_acc = 0;
    __syncthreads();
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&s_acc, v);
    __syncthreads();
    if (threadIdx.x == 0 && s_acc) atomicAdd(dst, s_acc);
}

// The input edge count, read once per block; 0 after an earlier failure.
CDEV long long block_edges(const CutParams& C) {
    __shared__ long long s_e;
    if (threadIdx.x == 0) {
        long long E = (long long)*(volatile const int64_t*)C.count_in;
        if (E < 0 || E > C.cap_in) {
            cut_status(C.info, PLAN_ERR_INVALID_ARG, DET_CUTIN);
            E = 0;
        }
        if (cut_failed(C.info)) E = 0;
        s_e = E;
    }
    __syncthreads();
    return s_e;
}

// A list's entry count, read once per block, capped by its capacity.
CDEV long long block_count(const DevInfo* info, const unsigned long long* counter, long long cap) {
    __shared__ long long s_n;
    if (threadIdx.x == 0) {
        const long long n = (long long)*(volatile const unsigned long long*)counter;
        s_n = cut_failed(info) ? 0 : (n < cap ? n : cap);
    }
    __syncthreads();
    return s_n;
}

// ---------------------------------------------------------------------------
// FP32 control points of one (edge, T): P[l][a] = sum_c D[l][c] x_i^(c)_a +
// sum_c D[l][g+c] x_j^(c)_a, the magnitude bound S = max over (l, a) of the
// same sums of |D| |x|, and the points' bounding box.
// ---------------------------------------------------------------------------
template <int M, int G, int PD>
CDEV void unit_points(const CutParams& C, long long i, long long j, int t, float* P, float& S, float* lo, float* hi) {
    constexpr int N_ = M * G, NP = PD + 1, TG = 2 * G;
    float xi[N_], xj[N_];
#pragma unroll
    for (int c = 0; c < N_; ++c) {
        xi[c] = ld32(C.states, i * N_ + c, C.in_f32);
        xj[c] = ld32(C.states, j * N_ + c, C.in_f32);
    }
    const float* D = C.tab32 + (long long)t * NP * TG;
    S = 0.f;
#pragma unroll
    for (int a = 0; a < M; ++a) {
        lo[a] = __int_as_float(0x7f800000);
        hi[a] = -__int_as_float(0x7f800000);
    }
#pragma unroll
    for (int l = 0; l < NP; ++l) {
#pragma unroll
        for (int a = 0; a < M; ++a) {
            float sl = 0.f, sr = 0.f, ml = 0.f, mr = 0.f;
#pragma unroll
            for (int c = 0; c < G; ++c) {
                const float dl = __ldg(D + l * TG + c), dr = __ldg(D + l * TG + G + c);
                sl = fmaf(dl, xi[c * M + a], sl);
                sr = fmaf(dr, xj[c * M + a], sr);
                ml = fmaf(fabsf(dl), fabsf(xi[c * M + a]), ml);
                mr = fmaf(fabsf(dr), fabsf(xj[c * M + a]), mr);
            }
            const float v = sl + sr;
            P[l * M + a] = v;
            S = fmaxf(S, ml + mr);
            lo[a] = fminf(lo[a], v);
            hi[a] = fmaxf(hi[a], v);
        }
    }
}

// Facet row {A_0, A_1, A_2, b}: FP32 product A . z, margin A . z - b and band.
// The comparisons s > b + band and s <= b - band used by the screening pass
// round once more than s - b > band; the band's slack covers it.
template <int M>
CDEV float dot32(const float4& f, const float* z) {
    float s = f.x * z[0];
    s = fmaf(f.y, z[1], s);
    if (M == 3) s = fmaf(f.z, z[2], s);
    return s;
}
template <int M>
CDEV float margin32(const float4& f, const float* z) {
    float s = f.x * z[0];
    s = fmaf(f.y, z[1], s);
    if (M == 3) s = fmaf(f.z, z[2], s);
    return s - f.w;
}
template <int M>
CDEV float band32(const float4& f, float S) {
    float n1 = fabsf(f.x) + fabsf(f.y);
    if (M == 3) n1 += fabsf(f.z);
    return KO * fmaf(n1, S, fabsf(f.w));
}

// ---------------------------------------------------------------------------
// Certified bounding box of every obstacle (one warp per obstacle, in the prep).  For a
// direction d = +-e_a, any y >= 0 with A^T y = d bounds the obstacle:
// d . z <= b^T y on O (weak duality), and it turns into a certificate of the
// game: sum_r y_r G[l][r] = d . P_l - b^T y + (A^T y - d) . P_l.  The lanes
// search all m-row subsets in FP32 for the dual-feasible one with the lowest
// bound (the optimal vertex); lane d recomputes that subset's y in FP64,
// clamps it to y >= 0 and keeps
//   beta' = b^T y + 2^-48 sum_r y_r |b_r|                (rounded outward to FP32)
//   c     = ||A^T y - d||_1 + 2^-47 sum_r y_r ||A_r||_1  (must be <= 2^-30),
// which covers the residual, the rounding of b^T y and that of the canonical
// FP64 margins.  A unit whose control points satisfy d . P_l > beta' + c S
// for all l (checked as lo_a - e > hi bound, e = (16 u + 2^-29) S, in pass A)
// misses the obstacle: y is a certificate.  A direction without a usable y
// (unbounded obstacle, near-singular vertex) gets an infinite bound.
// ---------------------------------------------------------------------------
template <int M>
CDEV void obstacle_boxes(const CutParams& C, long long gw, long long nw) {
    const int lane = threadIdx.x & 31;
    const float finf = __int_as_float(0x7f800000);
    for (long long o = gw; o < C.n_obst; o += nw) {
        const int r0 = C.obst_off[o];
        int nr = C.obst_off[o + 1] - r0;
        // an obstacle the prep rejects (bad row count or arrays) keeps infinite bounds
        if (nr < 0 || nr > C.max_orows || r0 < 0 || (nr > 0 && (!C.A || !C.b))) nr = 0;
        float best[2 * M];
        int bsub[2 * M];
#pragma unroll
        for (int d = 0; d < 2 * M; ++d) {
            best[d] = finf;
            bsub[d] = -1;
        }
        int nsub = nr;
#pragma unroll
        for (int k = 1; k < M; ++k) nsub *= nr;
        for (int s = lane; s < nsub; s += 32) {
            int idx[M], q = s;
            bool inc = true;
#pragma unroll
            for (int k = 0; k < M; ++k) {
                idx[k] = q % nr;
                q /= nr;
                if (k > 0 && idx[k] <= idx[k - 1]) inc = false;
            }
            if (!inc) continue;
            float a[M][M], bs[M], nrm = 1.f;
#pragma unroll
            for (int k = 0; k < M; ++k) {
                float n1 = 0.f;
#pragma unroll
                for (int j = 0; j < M; ++j) {
                    a[k][j] = ld32(C.A, (long long)(r0 + idx[k]) * M + j, C.in_f32);
                    n1 += fabsf(a[k][j]);
                }
                bs[k] = ld32(C.b, r0 + idx[k], C.in_f32);
                nrm *= n1;
            }
            // y solves sum_k y_k a[k] = d: y = (a^T)^-1 d, i.e. row a of a^-1 ... via cofactors
            float inv[M][M], det;
            if (M == 2) {
                det = a[0][0] * a[1][1] - a[0][1] * a[1][0];
                inv[0][0] = a[1][1];
                inv[0][1] = -a[0][1];
                inv[1][0] = -a[1][0];
                inv[1][1] = a[0][0];
            } else {
#pragma unroll
                for (int i = 0; i < M; ++i)
#pragma unroll
                    for (int j = 0; j < M; ++j) {
                        const int i1 = (i + 1) % M, i2 = (i + 2) % M, j1 = (j + 1) % M, j2 = (j + 2) % M;
                        inv[j][i] = a[i1][j1] * a[i2][j2] - a[i1][j2] * a[i2][j1];  // adjugate
                    }
                det = a[0][0] * inv[0][0] + a[0][1] * inv[1][0] + a[0][M - 1] * inv[M - 1][0];
            }
            if (!(fabsf(det) > 1e-4f * nrm)) continue;
            const float rdet = 1.f / det;
            // a^T y = e_a  <=>  y_k = (a^-1)[a][k] = inv[a][k] / det
#pragma unroll
            for (int ax = 0; ax < M; ++ax)
#pragma unroll
                for (int sg = 0; sg < 2; ++sg) {
                    bool ok = true;
                    float bound = 0.f;
#pragma unroll
                    for (int k = 0; k < M; ++k) {
                        const float yk = (sg ? -1.f : 1.f) * inv[ax][k] * rdet;
                        ok = ok && yk >= -1e-6f;
                        bound = fmaf(yk, bs[k], bound);
                    }
                    const int d = 2 * ax + sg;
                    if (ok && bound < best[d]) {
                        best[d] = bound;
                        bsub[d] = s;
                    }
                }
        }
#pragma unroll
        for (int d = 0; d < 2 * M; ++d)
            for (int of = 16; of > 0; of >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best[d], of);
                const int os = __shfl_xor_sync(0xffffffffu, bsub[d], of);
                if (ob < best[d] || (ob == best[d] && os < bsub[d])) {
                    best[d] = ob;
                    bsub[d] = os;
                }
            }
        float out = 0.f;
        if (lane < 2 * M) {
            const int d = lane, ax = d >> 1;
            const double sgn = (d & 1) ? -1.0 : 1.0;
            int sub = -1;
#pragma unroll
            for (int k = 0; k < 2 * M; ++k) sub = (k == d) ? bsub[k] : sub;
            double bnd = __longlong_as_double(0x7FF0000000000000ll);  // +inf: no bound
            if (sub >= 0) {
                int idx[M], q = sub;
                double a[M][M], bs[M];
#pragma unroll
                for (int k = 0; k < M; ++k) {
                    idx[k] = q % nr;
                    q /= nr;
#pragma unroll
                    for (int j = 0; j < M; ++j) a[k][j] = ld64(C.A, (long long)(r0 + idx[k]) * M + j, C.in_f32);
                    bs[k] = ld64(C.b, r0 + idx[k], C.in_f32);
                }
                // solve a^T y = sgn e_ax by Cramer's rule in FP64
                double y[M];
                if (M == 2) {
                    const double det = a[0][0] * a[1][1] - a[0][1] * a[1][0];
                    const double e0 = ax == 0 ? sgn : 0.0, e1 = ax == 1 ? sgn : 0.0;
                    // [a00 a10; a01 a11] y = e
                    y[0] = (e0 * a[1][1] - a[1][0] * e1) / det;
                    y[1] = (a[0][0] * e1 - e0 * a[0][1]) / det;
                } else {
                    double adj[M][M];
#pragma unroll
                    for (int i = 0; i < M; ++i)
#pragma unroll
                        for (int j = 0; j < M; ++j) {
                            const int i1 = (i + 1) % M, i2 = (i + 2) % M, j1 = (j + 1) % M, j2 = (j + 2) % M;
                            adj[j][i] = a[i1][j1] * a[i2][j2] - a[i1][j2] * a[i2][j1];
                        }
                    const double det = a[0][0] * adj[0][0] + a[0][1] * adj[1][0] + a[0][M - 1] * adj[M - 1][0];
#pragma unroll
                    for (int k = 0; k < M; ++k) y[k] = sgn * adj[ax][k] / det;
                }
                double beta = 0.0, yb = 0.0, y1 = 0.0, rho = 0.0;
                bool fin = true;
#pragma unroll
                for (int k = 0; k < M; ++k) {
                    y[k] = y[k] > 0.0 ? y[k] : 0.0;
                    fin = fin && isfinite(y[k]);
                    beta += y[k] * bs[k];
                    yb += y[k] * fabs(bs[k]);
                    double n1 = 0.0;
#pragma unroll
                    for (int j = 0; j < M; ++j) n1 += fabs(a[k][j]);
                    y1 += y[k] * n1;
                }
#pragma unroll
                for (int j = 0; j < M; ++j) {
                    double w = 0.0;
#pragma unroll
                    for (int k = 0; k < M; ++k) w += y[k] * a[k][j];
                    rho += fabs(w - (j == ax ? sgn : 0.0));
                }
                const double c = rho + 0x1p-47 * y1;
                if (fin && isfinite(beta) && c <= 0x1p-30) bnd = beta + 0x1p-48 * yb;
            }
            // +e_ax: z_ax <= bnd (upper bound, rounded up); -e_ax: z_ax >= -bnd (rounded down)
            out = (d & 1) ? __double2float_rd(-bnd) : __double2float_ru(bnd);
        }
        // lanes 0..2M-1 hold hi_0, lo_0, hi_1, lo_1, ...
        float* ob = C.obox + o * 8;
        if (lane < 2 * M) {
            const int ax = lane >> 1;
            if (M == 2) ob[(lane & 1) ? ax : 2 + ax] = out;
            else ob[(lane & 1) ? ax : 4 + ax] = out;
        }
    }
}

// ---------------------------------------------------------------------------
// Prep, three kinds of blocks: start vertex of every edge and cleared hit bits
// (one warp per row); the obstacles' FP32 rows, max_orows per obstacle, with
// row-count checks; the obstacles' certified boxes (one warp per obstacle).
// ---------------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(256) k_cut_prep(CutParams C, int row_blocks, int copy_blocks) {
    if ((int)blockIdx.x >= row_blocks + copy_blocks) {  // certified boxes, one warp per obstacle
        const long long gw = ((long long)(blockIdx.x - row_blocks - copy_blocks) * blockDim.x + threadIdx.x) >> 5;
        const long long nw = ((long long)(gridDim.x - row_blocks - copy_blocks) * blockDim.x) >> 5;
        obstacle_boxes<M>(C, gw, nw);
        return;
    }
    if ((int)blockIdx.x < row_blocks) {
        const long long E = block_edges(C);
        const int lane = threadIdx.x & 31;
        const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const long long nw = ((long long)row_blocks * blockDim.x) >> 5;
        if (E == 0) return;
        // the CSR must cover exactly edges 0..E-1 with end vertices below N
        // (every later pass indexes states with them)
        if (w0 == 0 && lane == 0 && (C.row_in[0] != 0 || (long long)C.row_in[C.N] != E))
            cut_status(C.info, PLAN_ERR_INVALID_ARG, DET_CUTIN);
        for (long long i = w0; i < C.N; i += nw) {
            const long long a = C.row_in[i], b = C.row_in[i + 1];
            if (a < 0 || b < a || b > E) {
                if (lane == 0) cut_status(C.info, PLAN_ERR_INVALID_ARG, DET_CUTIN);
                continue;
            }
            for (long long e = a + lane; e < b; e += 32) {
                C.src[e] = (int32_t)i;
                C.hit[e] = 0u;
                if ((unsigned)C.col_in[e] >= (unsigned)C.N) cut_status(C.info, PLAN_ERR_INVALID_ARG, DET_CUTIN);
            }
        }
        return;
    }
    const long long u = ((long long)blockIdx.x - row_blocks) * blockDim.x + threadIdx.x;
    if (u >= (long long)C.n_obst * C.max_orows) return;
    const int o = (int)(u / C.max_orows), k = (int)(u % C.max_orows);
    const int r0 = C.obst_off[o], nr = C.obst_off[o + 1] - r0;
    if (nr < 0 || nr > C.max_orows || r0 < 0 || (nr > 0 && (!C.A || !C.b))) {
        if (k == 0) cut_status(C.info, nr > C.max_orows ? PLAN_ERR_UNSUPPORTED : PLAN_ERR_INVALID_ARG, DET_ROWS);
        if (k == 0) C.ocount[o] = 0;
        return;
    }
    if (k == 0) C.ocount[o] = nr;
    if (k < nr) {
        const long long r = r0 + k;
        float4 f;
        f.x = ld32(C.A, r * C.m, C.in_f32);
        f.y = ld32(C.A, r * C.m + 1, C.in_f32);
        f.z = C.m == 3 ? ld32(C.A, r * C.m + 2, C.in_f32) : 0.f;
        f.w = ld32(C.b, r, C.in_f32);
        reinterpret_cast<float4*>(C.orow)[u] = f;
        const float n1 = fabsf(f.x) + fabsf(f.y) + fabsf(f.z);
        reinterpret_cast<float2*>(C.okb)[u] = make_float2(KO * n1, KO * fabsf(f.w));
    }
}

// ---------------------------------------------------------------------------
// Pass A: a block of 8 warps takes 256 (edge, T) units (a lane each) and one
// stripe of the obstacles.  Each warp computes its units' FP32 control
// points (stripes of the same units repeat that small step); the block stages
// the obstacles' certified boxes in shared memory, SCAN_TILE at a time, and
// each lane tests its unit against them, eight per step: lo_a - e > hi_a(O)
// or hi_a + e < lo_a(O) for some axis a, with e = (16 u + 2^-29) S covering
// the FP32 control points and the bounds' own residual term.  Pairs that no
// box separates go to the pair list through a per-warp buffer in shared
// memory (one atomic per flush).
// ---------------------------------------------------------------------------
constexpr int SCAN_STEP = 8;
constexpr int SCAN_TILE = 1024;  // obstacle boxes staged per block step (half for m = 3)
constexpr int SCAN_BUF = 256;    // pair-list entries a warp gathers before one flush

// Appends a warp's buffered entries to the pair list with one atomic.
CDEV void flush_pairs(const CutParams& C, unsigned long long* buf, int n, int lane) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&C.info->cut_near, (unsigned long long)n);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int k = lane; k < n; k += 32)
        if (base + k < (unsigned long long)C.cap32) C.list32[base + k] = buf[k];
    __syncwarp();
}

template <int M, int G, int PD>
__global__ void __launch_bounds__(256) k_cut_scan(CutParams C, int target_items) {
    constexpr int NP = PD + 1, BW = M == 2 ? 1 : 2;  // float4 per staged box
    constexpr int TILE = SCAN_TILE / BW;  // a multiple of SCAN_STEP
    __shared__ float4 sbox[TILE * BW];
    __shared__ unsigned long long sbuf[8][SCAN_BUF];
    const long long E = block_edges(C);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long* buf = sbuf[warp];
    int nbuf = 0;
    const long long units = E * C.nT;
    const long long nbg = (units + 255) / 256;
    // stripes of the obstacles when the 256-unit groups alone are too few to
    // give every SM work (the same choice in every block)
    int stripes = (int)((target_items + nbg - 1) / (nbg > 0 ? nbg : 1));
    stripes = stripes < 1 ? 1 : (stripes > 16 ? 16 : stripes);
    if (stripes > C.n_obst) stripes = C.n_obst > 0 ? C.n_obst : 1;
    const int per = (C.n_obst + stripes - 1) / stripes;
    unsigned long long n_units = 0, n_tests = 0, n_near = 0;
    const float4* gbox = reinterpret_cast<const float4*>(C.obox);
    for (long long item = blockIdx.x; item < nbg * stripes; item += gridDim.x) {
        const long long bg = item / stripes;
        const int sidx = (int)(item - bg * stripes);
        const long long u = bg * 256 + threadIdx.x;
        float le[M], he[M];
        bool valid = false;
        if (u < units) {
            const long long e = u / C.nT;
            const int t = (int)(u - e * C.nT);
            if ((C.mask_in[e] >> t) & 1u) {
                float P[NP * M], S, lo[M], hi[M];
                unit_points<M, G, PD>(C, C.src[e], C.col_in[e], t, P, S, lo, hi);
                const float ebox = (16.f * U32 + 0x1p-29f) * S;
#pragma unroll
                for (int a = 0; a < M; ++a) {
                    le[a] = lo[a] - ebox;
                    he[a] = hi[a] + ebox;
                }
                valid = true;
                if (sidx == 0) ++n_units;
            }
        }
        if (!valid) {
#pragma unroll
            for (int a = 0; a < M; ++a) {
                le[a] = __int_as_float(0x7f800000);  // every box test says "far"
                he[a] = -__int_as_float(0x7f800000);
            }
        }
        const bool any_valid = __syncthreads_or(valid) != 0;
        const int o0 = sidx * per, o1 = min(C.n_obst, o0 + per);
        if (valid && any_valid) n_tests += (unsigned long long)max(0, o1 - o0);
        for (int t0 = o0; any_valid && t0 < o1; t0 += TILE) {
            const int nt = min(TILE, o1 - t0);
            const int ntp = (nt + SCAN_STEP - 1) / SCAN_STEP * SCAN_STEP;
            __syncthreads();  // the previous tile is consumed
            // the tile, padded to whole steps with empty boxes (lo = +inf,
            // hi = -inf: every test says "far")
            for (int k = threadIdx.x; k < ntp * BW; k += blockDim.x) {
                const int ob = k / BW, h = k - ob * BW;
                float4 v;
                if (ob < nt) {
                    v = __ldg(gbox + 2 * (long long)(t0 + ob) + (M == 2 ? 0 : h));
                } else {
                    const float pinf = __int_as_float(0x7f800000);
                    v = (M == 2) ? make_float4(pinf, pinf, -pinf, -pinf)
                                 : (h == 0 ? make_float4(pinf, pinf, pinf, 0.f) : make_float4(-pinf, -pinf, -pinf, 0.f));
                }
                sbox[k] = v;
            }
            __syncthreads();
            for (int ob = 0; ob < ntp; ob += SCAN_STEP) {
                unsigned need = 0;
#pragma unroll
                for (int k = 0; k < SCAN_STEP; ++k) {
                    const float4 b0 = sbox[(ob + k) * BW];
                    bool far;
                    if (M == 2) {
                        far = le[0] > b0.z || le[1] > b0.w || he[0] < b0.x || he[1] < b0.y;
                    } else {
                        const float4 b1 = sbox[(ob + k) * BW + 1];
                        far = le[0] > b1.x || le[1] > b1.y || le[M - 1] > b1.z || he[0] < b0.x || he[1] < b0.y ||
                              he[M - 1] < b0.z;
                    }
                    need |= far ? 0u : (1u << k);
                }
                if (__any_sync(0xffffffffu, need != 0u)) {
                    const int cnt = __popc(need);
                    int incl = cnt;
                    for (int of = 1; of < 32; of <<= 1) {
                        const int v = __shfl_up_sync(0xffffffffu, incl, of);
                        if (lane >= of) incl += v;
                    }
                    const int total = __shfl_sync(0xffffffffu, incl, 31);
                    if (nbuf + total > SCAN_BUF) {
                        flush_pairs(C, buf, nbuf, lane);
                        nbuf = 0;
                    }
                    int idx = nbuf + incl - cnt;
                    for (unsigned bits = need; bits; bits &= bits - 1u, ++idx)
                        buf[idx] = ((unsigned long long)u << OBST_BITS) |
                                   (unsigned long long)(t0 + ob + __ffs(bits) - 1);
                    __syncwarp();
                    nbuf += total;
                    n_near += cnt;
                }
            }
        }
    }
    // the block's buffered entries with one atomic for all eight warps
    __shared__ int s_n[8];
    __shared__ unsigned long long s_base;
    if (lane == 0) s_n[warp] = nbuf;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < 8; ++w) tot += s_n[w];
        s_base = tot ? atomicAdd(&C.info->cut_near, (unsigned long long)tot) : 0ull;
    }
    __syncthreads();
    unsigned long long base = s_base;
    for (int w = 0; w < warp; ++w) base += (unsigned long long)s_n[w];
    for (int k = lane; k < nbuf; k += 32)
        if (base + k < (unsigned long long)C.cap32) C.list32[base + k] = buf[k];
    cut_block_add(&C.info->cut_units, n_units);
    cut_block_add(&C.info->cut_tests, n_tests);
    cut_block_add(&C.info->cut_box, n_tests - n_near);
}

// ---------------------------------------------------------------------------
// The matrix game of G (NP rows l, nr <= RB columns r) by the simplex method.
// With c = 1 - min G every payoff M = G + c is >= 1; maximise sum_l u_l
// subject to sum_l M[l][r] u_l <= 1 for every r, u >= 0 (the slack basis is
// feasible).  At the optimum delta* = 1 / sum u - c, lambda = u (the row
// player's mix, unnormalised) and y_r = minus the reduced cost of slack r (the
// column player's mix).  Entering column: the largest reduced cost for the
// first GAME_DANTZIG pivots, then Bland's rule (lowest label; no cycling).
//
// Condensed tableau, one row per basic variable and one column per
// non-basic one (labels: u_l -> l, slack s_r -> NP + r), held in registers:
// every access with the pivot's row or column index is an unrolled select, so
// nothing goes to local memory.  T enters as M^T (rows r >= nr zero), rhs as
// 1 (0 for r >= nr, which never leave).  Returns false if GAME_ITERS pivots
// did not reach optimality; lambda and y are then those of the last basis
// (the caller uses them only as certificate candidates).
// ---------------------------------------------------------------------------
constexpr int GAME_DANTZIG = 24;

template <typename F>
CDEV F pos_part(F v) { return v > F(0) ? v : F(0); }

template <typename F, int NP, int RB>
CDEV bool game_reg(F (&T)[RB][NP], F (&rhs)[RB], F (&lam)[NP], F (&y)[RB], F tol) {
    F d[NP];
    int colLab[NP], rowLab[RB];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        d[j] = F(1);
        colLab[j] = j;
    }
#pragma unroll
    for (int i = 0; i < RB; ++i) rowLab[i] = NP + i;
    bool optimal = false;
    for (int it = 0; it < GAME_ITERS; ++it) {
        int c = -1, cl = 1 << 20;
        F dbest = tol;
        if (it < GAME_DANTZIG) {
#pragma unroll
            for (int j = 0; j < NP; ++j)
                if (d[j] > dbest) {
                    c = j;
                    dbest = d[j];
                }
            if (c >= 0) {
#pragma unroll
                for (int j = 0; j < NP; ++j) cl = (j == c) ? colLab[j] : cl;
            }
        } else {
#pragma unroll
            for (int j = 0; j < NP; ++j)
                if (d[j] > tol && colLab[j] < cl) {
                    c = j;
                    cl = colLab[j];
                }
        }
        if (c < 0) {
            optimal = true;
            break;
        }
        F colc[RB];
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            F v = T[i][0];
#pragma unroll
            for (int j = 1; j < NP; ++j) v = (j == c) ? T[i][j] : v;
            colc[i] = v;
        }
        int r = -1, rl = 1 << 20;
        F best = F(0);
#pragma unroll
        for (int i = 0; i < RB; ++i)
            if (colc[i] > tol) {
                const F ratio = rhs[i] / colc[i];
                if (r < 0 || ratio < best || (ratio == best && rowLab[i] < rl)) {
                    r = i;
                    best = ratio;
                    rl = rowLab[i];
                }
            }
        if (r < 0) break;  // unbounded: impossible with payoffs >= 1
        F rowr[NP], rhsr = rhs[0], p = colc[0];
#pragma unroll
        for (int j = 0; j < NP; ++j) rowr[j] = T[0][j];
#pragma unroll
        for (int i = 1; i < RB; ++i)
            if (i == r) {
#pragma unroll
                for (int j = 0; j < NP; ++j) rowr[j] = T[i][j];
                rhsr = rhs[i];
                p = colc[i];
            }
        const F inv = F(1) / p;
        F rs[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) rs[j] = (j == c) ? inv : rowr[j] * inv;
        const F rhs_s = rhsr * inv;
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            const bool isr = i == r;
            const F ci = colc[i];
#pragma unroll
            for (int j = 0; j < NP; ++j) T[i][j] = isr ? rs[j] : ((j == c) ? F(0) : T[i][j]) - ci * rs[j];
            rhs[i] = isr ? rhs_s : rhs[i] - ci * rhs_s;
        }
        F dc = d[0];
#pragma unroll
        for (int j = 1; j < NP; ++j) dc = (j == c) ? d[j] : dc;
#pragma unroll
        for (int j = 0; j < NP; ++j) d[j] = ((j == c) ? F(0) : d[j]) - dc * rs[j];
        int lr = rowLab[0];
#pragma unroll
        for (int i = 1; i < RB; ++i) lr = (i == r) ? rowLab[i] : lr;
#pragma unroll
        for (int i = 0; i < RB; ++i) rowLab[i] = (i == r) ? cl : rowLab[i];
#pragma unroll
        for (int j = 0; j < NP; ++j) colLab[j] = (j == c) ? lr : colLab[j];
    }
#pragma unroll
    for (int l = 0; l < NP; ++l) lam[l] = F(0);
#pragma unroll
    for (int i = 0; i < RB; ++i)
#pragma unroll
        for (int l = 0; l < NP; ++l)
            if (rowLab[i] == l) lam[l] = pos_part(rhs[i]);
#pragma unroll
    for (int i = 0; i < RB; ++i) y[i] = F(0);
#pragma unroll
    for (int j = 0; j < NP; ++j)
#pragma unroll
        for (int i = 0; i < RB; ++i)
            if (colLab[j] == NP + i) y[i] = pos_part(-d[j]);
    return optimal;
}

// Canonical FP64 half sum (left to right from 0, no FMA).
template <int G>
CDEV double half64(const double* coef, const double* x, int stride) {
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < G; ++c) s = __dadd_rn(s, __dmul_rn(coef[c], x[c * stride]));
    return s;
}

// ---------------------------------------------------------------------------
// FP64 settling of one (edge, T, obstacle), by the whole warp.  Canonical
// FP64 margins (the oracle's order: each control-point half summed left to
// right from 0, halves added; facet products summed left to right from 0,
// then b subtracted; no FMA): lane k computes control-point coordinate k, lane
// r then facet r's margins.  Algorithm 2's two checks exactly, then the FP32
// game's mixes (mix: lambda then y) as certificates, then the game itself with
// the warp as the tableau (lane r = basic row r) and exact-rounding
// certificates; a game certified neither way is a tie (|delta*| at rounding
// level), decided by the sign of its computed value.  GB300's FP64 pipe is
// narrow, so the FP64 instruction count stays low: the coordinates are
// computed once per warp, not once per lane, and the reciprocals come from an
// FP32 estimate and two Newton steps.  Returns 1 (hit) or -1 (miss).
// ---------------------------------------------------------------------------
CDEV double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// 1 / x for the pivots (|x| within FP32 range): FP32 estimate, two Newton
// steps (the pivot values only choose and scale pivots; the certificates
// re-check whatever comes out).
CDEV double rcp64(double x) {
    double r = (double)__frcp_rn((float)x);
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}

template <int M, int G, int PD>
CDEV int settle64(const CutParams& C, unsigned long long en, const float* mix, bool& tie) {
    constexpr int N_ = M * G, NP = PD + 1, TG = 2 * G;
    static_assert(NP * M <= 32, "one control-point coordinate per lane");
    const int lane = threadIdx.x & 31;
    const double inf = __longlong_as_double(0x7FF0000000000000ll);
    tie = false;
    const long long u = (long long)(en >> OBST_BITS);
    const int o = (int)(en & ((1ull << OBST_BITS) - 1ull));
    const long long e = u / C.nT;
    const int t = (int)(u - e * C.nT);
    const long long i = C.src[e], j = C.col_in[e];
    // lane k < NP * M: coordinate a = k % M of control point l = k / M
    double pk = 0.0;
    if (lane < NP * M) {
        const int l = lane / M, a = lane - l * M;
        const double* D = C.tab64 + (long long)t * C.L.e_stride + C.L.e_D + l * TG;
        double xi[G], xj[G];
#pragma unroll
        for (int c = 0; c < G; ++c) {
            xi[c] = ld64(C.states, i * N_ + c * M + a, C.in_f32);
            xj[c] = ld64(C.states, j * N_ + c * M + a, C.in_f32);
        }
        pk = __dadd_rn(half64<G>(D, xi, 1), half64<G>(D + G, xj, 1));
    }
    double P[NP * M];
#pragma unroll
    for (int q = 0; q < NP * M; ++q) P[q] = __shfl_sync(0xffffffffu, pk, q);
    const int r0 = C.obst_off[o], nr = C.ocount[o];
    const bool mine = lane < nr;
    double g[NP];
#pragma unroll
    for (int l = 0; l < NP; ++l) g[l] = 0.0;
    if (mine) {
        const double br = ld64(C.b, r0 + lane, C.in_f32);
        double Ar[M];
#pragma unroll
        for (int a = 0; a < M; ++a) Ar[a] = ld64(C.A, (long long)(r0 + lane) * M + a, C.in_f32);
#pragma unroll
        for (int l = 0; l < NP; ++l) {
            double sv = 0.0;
#pragma unroll
            for (int a = 0; a < M; ++a) sv = __dadd_rn(sv, __dmul_rn(Ar[a], P[l * M + a]));
            g[l] = __dsub_rn(sv, br);
        }
    }
    int verdict = 0;  // 1 hit, -1 miss
#pragma unroll
    for (int l = 0; l < NP; ++l)  // a control point with every margin <= 0
        if (__ballot_sync(0xffffffffu, mine && !(g[l] <= 0.0)) == 0u) verdict = 1;
    if (verdict == 0) {  // one facet with every margin > 0
        bool out = mine;
#pragma unroll
        for (int l = 0; l < NP; ++l) out = out && g[l] > 0.0;
        if (__ballot_sync(0xffffffffu, out) != 0u) verdict = -1;
    }
    if (verdict == 0 && mix) {  // the FP32 game's mixes on the canonical margins
        double L = 0.0, s = 0.0, a = 0.0;
#pragma unroll
        for (int l = 0; l < NP; ++l) {
            const double lm = (double)mix[l];
            L += lm;
            s += lm * g[l];
            a += lm * fabs(g[l]);
        }
        const double kh = 2.0 * (NP + 2) * U64, km = 2.0 * (32 + 2) * U64;
        if (L > 0.0 && __ballot_sync(0xffffffffu, mine && !(s + kh * a < 0.0)) == 0u) verdict = 1;
        if (verdict == 0) {
            const double yr = mine ? (double)mix[NP + lane] : 0.0;
            bool miss_ok = true;
#pragma unroll
            for (int l = 0; l < NP; ++l) {
                const double ks = warp_sum(yr * g[l]), ka = warp_sum(yr * fabs(g[l]));
                miss_ok = miss_ok && (ks - km * ka > 0.0);
            }
            if (miss_ok) verdict = -1;
        }
    }
        if (verdict == 0) {
            double gmin = inf;
#pragma unroll
            for (int l = 0; l < NP; ++l) gmin = mine ? fmin(gmin, g[l]) : gmin;
            for (int of = 16; of > 0; of >>= 1) gmin = fmin(gmin, __shfl_xor_sync(0xffffffffu, gmin, of));
            const double shift = 1.0 - gmin;
            double T[NP], rhs = mine ? 1.0 : 0.0, d[NP];
            int colLab[NP], rowLab = NP + lane;
#pragma unroll
            for (int l = 0; l < NP; ++l) {
                T[l] = mine ? g[l] + shift : 0.0;
                d[l] = 1.0;
                colLab[l] = l;
            }
            const double tol = 1e-13;
            for (int it = 0; it < GAME_ITERS; ++it) {
                int c = -1, cl = 1 << 20;
                double dbest = tol;
                if (it < GAME_DANTZIG) {
#pragma unroll
                    for (int l = 0; l < NP; ++l)
                        if (d[l] > dbest) {
                            c = l;
                            dbest = d[l];
                        }
                    if (c >= 0) {
#pragma unroll
                        for (int l = 0; l < NP; ++l) cl = (l == c) ? colLab[l] : cl;
                    }
                } else {
#pragma unroll
                    for (int l = 0; l < NP; ++l)
                        if (d[l] > tol && colLab[l] < cl) {
                            c = l;
                            cl = colLab[l];
                        }
                }
                if (c < 0) break;
                double colc = T[0];
#pragma unroll
                for (int l = 1; l < NP; ++l) colc = (l == c) ? T[l] : colc;
                const bool ok = mine && colc > tol;
                double best = ok ? rhs * rcp64(colc) : inf;
                int bl = ok ? rowLab : (1 << 20), bi = lane;
                for (int of = 16; of > 0; of >>= 1) {
                    const double ob = __shfl_xor_sync(0xffffffffu, best, of);
                    const int obl = __shfl_xor_sync(0xffffffffu, bl, of);
                    const int obi = __shfl_xor_sync(0xffffffffu, bi, of);
                    if (ob < best || (ob == best && obl < bl)) {
                        best = ob;
                        bl = obl;
                        bi = obi;
                    }
                }
                if (!(best < inf)) break;  // unbounded: impossible with payoffs >= 1
                const int r = bi;
                const double p = __shfl_sync(0xffffffffu, colc, r);
                const double inv = rcp64(p);
                double rs[NP];
#pragma unroll
                for (int l = 0; l < NP; ++l) {
                    const double v = __shfl_sync(0xffffffffu, T[l], r);
                    rs[l] = (l == c) ? inv : v * inv;
                }
                const double rhs_s = __shfl_sync(0xffffffffu, rhs, r) * inv;
                const int lr = __shfl_sync(0xffffffffu, rowLab, r);
                if (lane == r) {
#pragma unroll
                    for (int l = 0; l < NP; ++l) T[l] = rs[l];
                    rhs = rhs_s;
                    rowLab = cl;
                } else {
#pragma unroll
                    for (int l = 0; l < NP; ++l) T[l] = ((l == c) ? 0.0 : T[l]) - colc * rs[l];
                    rhs = rhs - colc * rhs_s;
                }
                double dc = d[0];
#pragma unroll
                for (int l = 1; l < NP; ++l) dc = (l == c) ? d[l] : dc;
#pragma unroll
                for (int l = 0; l < NP; ++l) {
                    d[l] = ((l == c) ? 0.0 : d[l]) - dc * rs[l];
                    colLab[l] = (l == c) ? lr : colLab[l];
                }
            }
            double lam[NP], L = 0.0;
#pragma unroll
            for (int l = 0; l < NP; ++l) {
                lam[l] = warp_sum(rowLab == l ? pos_part(rhs) : 0.0);
                L += lam[l];
            }
            double yr = 0.0;  // this lane's facet weight
#pragma unroll
            for (int l = 0; l < NP; ++l)
                if (colLab[l] == NP + lane) yr = pos_part(-d[l]);
            if (!mine) yr = 0.0;
            const double kh = 2.0 * (NP + 2) * U64, km = 2.0 * (32 + 2) * U64;
            double s = 0.0, a = 0.0;
#pragma unroll
            for (int l = 0; l < NP; ++l) {
                s += lam[l] * g[l];
                a += lam[l] * fabs(g[l]);
            }
            const bool hit_ok = L > 0.0 && __ballot_sync(0xffffffffu, mine && !(s + kh * a < 0.0)) == 0u;
            bool miss_ok = true;
#pragma unroll
            for (int l = 0; l < NP; ++l) {
                const double ks = warp_sum(yr * g[l]), ka = warp_sum(yr * fabs(g[l]));
                miss_ok = miss_ok && (ks - km * ka > 0.0);
            }
            if (hit_ok) verdict = 1;
            else if (miss_ok) verdict = -1;
            else {
                verdict = (L > 0.0 && 1.0 / L - shift <= 0.0) ? 1 : -1;
                tie = true;
            }
        }
    return verdict;
}

// ---------------------------------------------------------------------------
// Pass B: one lane per listed (edge, T, obstacle), the warp walking the list
// in steps of 32.  FP32 margins with their bands (b_r +- band_r against the
// products A_r . P_l):
//   a control point below every facet's b - band -> hit (Algorithm 2, first);
//   a facet above b + band at every control point -> miss (second);
// otherwise the game in registers (RB >= every obstacle's row count), then
// its certificates (weak duality; margins within band_r of the canonical):
//   hit:  lambda >= 0, L = sum lambda > 0, and for every r
//         sum_l lambda_l G[l][r] + L band_r + 2 (NP + 2) u sum_l lambda_l |G[l][r]| < 0;
//   miss: y >= 0 and for every l
//         sum_r y_r G[l][r] - sum_r y_r band_r - 2 (RB + 2) u sum_r y_r |G[l][r]| > 0.
// The margins are recomputed for the checks rather than kept in registers.
// Entries no FP32 certificate settles are then settled one by one by the
// whole warp in FP64 (settle64), with the lane's lambda and y passed through
// shared memory.
// ---------------------------------------------------------------------------
template <int M, int G, int PD, int RB>
__global__ void __launch_bounds__(128) k_cut_pair(CutParams C) {
    constexpr int NP = PD + 1;
    static_assert(NP + RB <= 32, "lambda and y fit one warp-sized buffer");
    __shared__ float s_mix[4][32];
    const long long n = block_count(C.info, &C.info->cut_near, C.cap32);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned long long n_s1 = 0, n_s2 = 0, n_games = 0, n_64 = 0, n_ties = 0;
    for (long long k0 = gw * 32; k0 < n; k0 += nw * 32) {
        const long long k = k0 + lane;
        unsigned long long en = 0;
        bool need64 = false;
        float lam[NP], y[RB];
        long long e = 0;
        int t = 0;
        if (k < n) {
            en = C.list32[k];
            const long long u = (long long)(en >> OBST_BITS);
            const int o = (int)(en & ((1ull << OBST_BITS) - 1ull));
            e = u / C.nT;
            t = (int)(u - e * C.nT);
            if (!((*(volatile const uint32_t*)(C.hit + e) >> t) & 1u)) {
                float P[NP * M], S, lo[M], hi[M];
                unit_points<M, G, PD>(C, C.src[e], C.col_in[e], t, P, S, lo, hi);
                const int nr = C.ocount[o];
                const long long rb = (long long)o * C.max_orows;
                const float4* rw = reinterpret_cast<const float4*>(C.orow) + rb;
                const float2* kw = reinterpret_cast<const float2*>(C.okb) + rb;
                float T[RB][NP], band[RB];
                bool inside[NP], sep = false;
#pragma unroll
                for (int l = 0; l < NP; ++l) inside[l] = true;
                float gmin = __int_as_float(0x7f800000);
#pragma unroll
                for (int i = 0; i < RB; ++i) {
                    float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
                    float bd = 0.f;
                    if (i < nr) {
                        f = __ldg(rw + i);
                        const float2 kb = __ldg(kw + i);
                        bd = fmaf(kb.x, S, kb.y);
                    }
                    band[i] = bd;
                    bool above = i < nr;
#pragma unroll
                    for (int l = 0; l < NP; ++l) {
                        const float sv = dot32<M>(f, P + l * M);
                        T[i][l] = sv - f.w;
                        if (i < nr) {
                            gmin = fminf(gmin, sv - f.w);
                            inside[l] = inside[l] && sv <= f.w - bd;
                            above = above && sv > f.w + bd;
                        }
                    }
                    sep = sep || above;
                }
                bool in = false;
#pragma unroll
                for (int l = 0; l < NP; ++l) in = in || inside[l];
                if (in) {
                    ++n_s1;
                    atomicOr(&C.hit[e], 1u << t);
                } else if (sep) {
                    ++n_s2;
                } else {
                    ++n_games;
                    const float shift = 1.f - gmin;
                    float rhs[RB];
#pragma unroll
                    for (int i = 0; i < RB; ++i) {
#pragma unroll
                        for (int l = 0; l < NP; ++l) T[i][l] = i < nr ? T[i][l] + shift : 0.f;
                        rhs[i] = i < nr ? 1.f : 0.f;
                    }
                    game_reg<float, NP, RB>(T, rhs, lam, y, 1e-6f);
                    float L = 0.f;
#pragma unroll
                    for (int l = 0; l < NP; ++l) L += lam[l];
                    bool hit_ok = L > 0.f;
                    float ks[NP], ka[NP], Y = 0.f;
#pragma unroll
                    for (int l = 0; l < NP; ++l) ks[l] = ka[l] = 0.f;
                    const float kh = 2.f * (NP + 2) * U32, km = 2.f * (RB + 2) * U32;
#pragma unroll
                    for (int i = 0; i < RB; ++i) {
                        if (i < nr) {
                            const float4 f = __ldg(rw + i);
                            float sm = 0.f, am = 0.f;
#pragma unroll
                            for (int l = 0; l < NP; ++l) {
                                const float gv = margin32<M>(f, P + l * M);
                                sm = fmaf(lam[l], gv, sm);
                                am = fmaf(lam[l], fabsf(gv), am);
                                ks[l] = fmaf(y[i], gv, ks[l]);
                                ka[l] = fmaf(y[i], fabsf(gv), ka[l]);
                            }
                            hit_ok = hit_ok && (sm + L * band[i] + kh * am < 0.f);
                            Y = fmaf(y[i], band[i], Y);
                        }
                    }
                    bool miss_ok = true;
#pragma unroll
                    for (int l = 0; l < NP; ++l) miss_ok = miss_ok && (ks[l] - Y - km * ka[l] > 0.f);
                    if (hit_ok) atomicOr(&C.hit[e], 1u << t);
                    else if (!miss_ok) {
                        need64 = true;
#pragma unroll
                        for (int r = 0; r < RB; ++r) y[r] = r < nr ? y[r] : 0.f;
                    }
                }
            }
        }
        // entries no FP32 certificate settled: the whole warp, one at a time
        for (unsigned todo = __ballot_sync(0xffffffffu, need64); todo; todo &= todo - 1u) {
            const int src = __ffs(todo) - 1;
            if (lane == src) {
#pragma unroll
                for (int l = 0; l < NP; ++l) s_mix[warp][l] = lam[l];
#pragma unroll
                for (int r = 0; r < RB; ++r) s_mix[warp][NP + r] = y[r];
            }
            __syncwarp();
            const unsigned long long en_s = __shfl_sync(0xffffffffu, en, src);
            bool tie;
            const int v = settle64<M, G, PD>(C, en_s, s_mix[warp], tie);
            if (lane == src) {
                ++n_64;
                n_ties += tie;
                if (v == 1) atomicOr(&C.hit[e], 1u << t);
            }
            __syncwarp();
        }
    }
    cut_block_add(&C.info->cut_step1, n_s1);
    cut_block_add(&C.info->cut_step2, n_s2);
    cut_block_add(&C.info->cut_games, n_games);
    cut_block_add(&C.info->cut_lp64, n_64);
    cut_block_add(&C.info->cut_ties, n_ties);
}

// ---------------------------------------------------------------------------
// Compaction.  Chunks of CUT_CHUNK edges, 8 consecutive edges per thread.
// ---------------------------------------------------------------------------
constexpr int FILL_THREADS = CUT_CHUNK / 8;

CDEV uint32_t kept_bits(const CutParams& C, long long e, long long E) {
    const uint32_t tmask = C.nT >= 32 ? 0xffffffffu : ((1u << C.nT) - 1u);  // bits of the given durations only
    return e < E ? (C.mask_in[e] & ~C.hit[e] & tmask) : 0u;
}

// Exclusive block scan of one value per thread (FILL_THREADS threads); also
// returns the block total.
CDEV int block_excl_scan(int v, int& total) {
    __shared__ int s_w[FILL_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < FILL_THREADS / 32 ? s_w[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < FILL_THREADS / 32) s_w[lane] = w;
    }
    __syncthreads();
    total = s_w[FILL_THREADS / 32 - 1];
    const int before = (warp > 0 ? s_w[warp - 1] : 0) + x - v;
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(FILL_THREADS) k_cut_count(CutParams C) {
    const long long E = block_edges(C);
    const long long nch = (E + CUT_CHUNK - 1) / CUT_CHUNK;
    for (long long c = blockIdx.x; c < nch; c += gridDim.x) {
        const long long e0 = c * CUT_CHUNK + (long long)threadIdx.x * 8;
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) cnt += kept_bits(C, e0 + k, E) != 0u;
        int total;
        block_excl_scan(cnt, total);
        if (threadIdx.x == 0) C.chunk[c] = total;
    }
}

// One block: exclusive prefix of the chunk counts, the output count, the
// capacity checks (output and both game lists).
__global__ void __launch_bounds__(1024) k_cut_offsets(CutParams C) {
    const long long E = block_edges(C);
    const long long nch = (E + CUT_CHUNK - 1) / CUT_CHUNK;
    __shared__ long long s_w[32];
    __shared__ long long s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long c0 = 0; c0 < nch; c0 += 1024) {
        const long long c = c0 + threadIdx.x;
        const long long v = c < nch ? C.chunk[c] : 0;
        long long x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        if (warp == 0) {
            long long w = s_w[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            s_w[lane] = w;
        }
        __syncthreads();
        const long long before = s_carry + (warp > 0 ? s_w[warp - 1] : 0) + x - v;
        if (c < nch) C.chunk[c] = before;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += s_w[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const long long total = s_carry;
        C.chunk[nch] = total;
        if (!cut_failed(C.info)) {
            *C.count_out = total;
            if (C.info->cut_near > (unsigned long long)C.cap32)
                cut_status(C.info, PLAN_ERR_CAPACITY, DET_CUTLIST);
            else if (total > C.cap_out)
                cut_status(C.info, PLAN_ERR_CAPACITY, DET_OUTPUT);
        }
    }
}

// Canonical FP64 cost of (i -> j, T_t), in the edge build's order: per
// control-polygon segment l the squares of its rows (derivative d, axis a)
// accumulated by FMA, then the square roots summed in l order.
template <int M, int G, int PD>
CDEV double edge_cost64(const CutParams& C, const double* xi, const double* xj, int t) {
    constexpr int TG = 2 * G;
    const int DR = C.cost_mode == 1 ? 1 : G;
    const double* tb = C.tab64 + (long long)t * C.L.e_stride + C.L.e_C;
    double cost = 0.0;
    for (int l = 0; l < PD; ++l) {
        double ss = 0.0;
        for (int d = 0; d < DR; ++d)
#pragma unroll
            for (int a = 0; a < M; ++a) {
                const double v = half64<G>(tb + (d * PD + l) * TG, xi + a, M) + half64<G>(tb + (d * PD + l) * TG + G, xj + a, M);
                ss = fma(v, v, ss);
            }
        cost += sqrt(ss);
    }
    return cost;
}

template <int M, int G, int PD>
__global__ void __launch_bounds__(FILL_THREADS) k_cut_fill(CutParams C) {
    constexpr int N_ = M * G;
    const long long E = block_edges(C);
    const long long nch = (E + CUT_CHUNK - 1) / CUT_CHUNK;
    __shared__ int s_ok;
    if (threadIdx.x == 0) s_ok = !cut_failed(C.info);
    __syncthreads();
    const bool write = s_ok != 0;
    for (long long c = blockIdx.x; c < nch; c += gridDim.x) {
        const long long e0 = c * CUT_CHUNK + (long long)threadIdx.x * 8;
        uint32_t nm[8];
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            nm[k] = kept_bits(C, e0 + k, E);
            cnt += nm[k] != 0u;
        }
        int total;
        long long q = C.chunk[c] + block_excl_scan(cnt, total);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const long long e = e0 + k;
            if (e >= E) break;
            C.pos[e] = (int32_t)q;
            if (nm[k] != 0u) {
                if (write) {
                    C.col_out[q] = C.col_in[e];
                    C.mask_out[q] = nm[k];
                    const int bt = C.t_in[e];
                    if ((nm[k] >> bt) & 1u) {
                        C.t_out[q] = (uint8_t)bt;
                        if (C.w_f64) ((double*)C.w_out)[q] = ((const double*)C.w_in)[e];
                        else ((float*)C.w_out)[q] = ((const float*)C.w_in)[e];
                    } else {
                        const long long i = C.src[e], j = C.col_in[e];
                        double xi[N_], xj[N_];
#pragma unroll
                        for (int s = 0; s < N_; ++s) {
                            xi[s] = ld64(C.states, i * N_ + s, C.in_f32);
                            xj[s] = ld64(C.states, j * N_ + s, C.in_f32);
                        }
                        double best = __longlong_as_double(0x7FF0000000000000ll);
                        int bt2 = 0;
                        for (uint32_t bits = nm[k]; bits; bits &= bits - 1u) {
                            const int t = __ffs(bits) - 1;
                            const double cst = edge_cost64<M, G, PD>(C, xi, xj, t);
                            if (cst < best) {
                                best = cst;
                                bt2 = t;
                            }
                        }
                        C.t_out[q] = (uint8_t)bt2;
                        if (C.w_f64) ((double*)C.w_out)[q] = best;
                        else ((float*)C.w_out)[q] = (float)best;
                    }
                }
                ++q;
            }
        }
    }
}

// Row offsets of the output: the output index of each row's first input edge.
__global__ void k_cut_rows(CutParams C) {
    const long long E = block_edges(C);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > C.N || cut_failed(C.info)) return;
    const long long a = C.row_in[i];
    const long long nch = (E + CUT_CHUNK - 1) / CUT_CHUNK;
    C.row_out[i] = (int32_t)(a >= E ? C.chunk[nch] : C.pos[a]);
}

template <int M, int G, int PD>
int launch_cut_t(const CutParams& C, cudaStream_t st, int num_sms, int* launches, cudaEvent_t e0, cudaEvent_t e1) {
    const long long rb = ((long long)C.N * 32 + 255) / 256;
    const int row_blocks = (int)(rb < num_sms * 8 ? (rb > 0 ? rb : 1) : num_sms * 8);
    const long long orows = (long long)C.n_obst * C.max_orows;
    const int obst_blocks = (int)((orows + 255) / 256);
    const int box_blocks = (C.n_obst + 7) / 8;
    k_cut_prep<M><<<row_blocks + obst_blocks + box_blocks, 256, 0, st>>>(C, row_blocks, obst_blocks);
    // pass A: a grid-stride loop over (256-unit group, obstacle stripe) items
    const int ga = num_sms * 8;
    if (e0) cudaEventRecord(e0, st);
    k_cut_scan<M, G, PD><<<ga, 256, 0, st>>>(C, num_sms * 6);
    if (e1) cudaEventRecord(e1, st);
    if (C.max_orows <= 8) k_cut_pair<M, G, PD, 8><<<num_sms * 4, 128, 0, st>>>(C);
    else k_cut_pair<M, G, PD, CUT_RMAX><<<num_sms * 4, 128, 0, st>>>(C);
    long long gc = C.nchunks < (long long)num_sms * 4 ? C.nchunks : (long long)num_sms * 4;
    if (gc < 1) gc = 1;
    k_cut_count<<<(int)gc, FILL_THREADS, 0, st>>>(C);
    k_cut_offsets<<<1, 1024, 0, st>>>(C);
    k_cut_fill<M, G, PD><<<(int)gc, FILL_THREADS, 0, st>>>(C);
    k_cut_rows<<<(int)((C.N + 1 + 255) / 256), 256, 0, st>>>(C);
    *launches += 7;
    return (int)cudaGetLastError();
}

}  // namespace

int launch_cut(const CutParams& C, void* stream, int num_sms, int* launches, void* ev_scan_begin, void* ev_scan_end) {
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = (cudaEvent_t)ev_scan_begin, e1 = (cudaEvent_t)ev_scan_end;
    if (C.m == 2 && C.g == 2 && C.p == 3) return launch_cut_t<2, 2, 3>(C, st, num_sms, launches, e0, e1);
    if (C.m == 2 && C.g == 2 && C.p == 5) return launch_cut_t<2, 2, 5>(C, st, num_sms, launches, e0, e1);
    if (C.m == 3 && C.g == 3 && C.p == 5) return launch_cut_t<3, 3, 5>(C, st, num_sms, launches, e0, e1);
    if (C.m == 3 && C.g == 3 && C.p == 7) return launch_cut_t<3, 3, 7>(C, st, num_sms, launches, e0, e1);
    return (int)cudaErrorInvalidValue;
}

}  // namespace plan
