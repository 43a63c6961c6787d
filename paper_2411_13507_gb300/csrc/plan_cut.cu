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
//  Pass A (k_cut_scan): one lane per (edge, T), the block's warps split the
//    obstacles; FP32 control points, then per obstacle (i) a facet whose
//    half-space misses the control points' bounding box -> miss, (ii) the
//    margins with bands: a point certainly inside -> hit, a facet certainly
//    separating -> miss, otherwise the entry joins the game list.
//  Pass B (k_cut_lp32): the game solved by the simplex method in FP32.  Weak
//    duality turns its solution into certificates: any lambda >= 0 with
//    G^T lambda < 0 proves a hit, any y >= 0 with G y > 0 a miss; both are
//    checked against G's error bands.  Uncertified entries go to pass C.
//  Pass C (k_cut_lp64): canonical FP64 margins, Algorithm 2's two checks
//    exactly, then the game in FP64 with certificates against the rounding of
//    the check itself.  A game certified neither way has |delta*| at the
//    rounding level: a tie, decided by the sign of the computed value and
//    counted.
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
constexpr int SCAN_WARPS = 8;   // obstacle stripes per block of pass A
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

// Facet row {A_0, A_1, A_2, b}: FP32 margin of point z and its band.
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
// Prep: start vertex of every edge, cleared hit bits (one warp per row), and
// the obstacles' FP32 rows, max_orows per obstacle, with row-count checks.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_cut_prep(CutParams C, int row_blocks) {
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
    }
}

// ---------------------------------------------------------------------------
// Pass A.  A block takes 32 (edge, T) units at a time (one per lane); warp 0
// computes their control points into shared memory, then warp w scans the
// obstacles w, w + 8, ... for all 32.  A unit found to hit stops every warp's
// scan of it (shared flag).  Entries that no band decides are appended to the
// game list (one atomic per warp and obstacle).
// ---------------------------------------------------------------------------
template <int M, int G, int PD>
__global__ void __launch_bounds__(256) k_cut_scan(CutParams C) {
    constexpr int NP = PD + 1, PS = NP * M + 1;  // odd stride: lane-strided reads hit distinct banks
    __shared__ float sP[32 * PS];
    __shared__ float sS[32], sLo[32 * 4], sHi[32 * 4];
    __shared__ int sState[32];  // 0 checking, 1 hit, 2 nothing to check
    const long long E = block_edges(C);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long units = E * C.nT;
    unsigned long long n_units = 0, n_tests = 0, n_box = 0, n_s1 = 0, n_s2 = 0;
    volatile int* vstate = sState;
    for (long long g0 = (long long)blockIdx.x * 32; g0 < units; g0 += (long long)gridDim.x * 32) {
        if (warp == 0) {
            const long long u = g0 + lane;
            int st = 2;
            if (u < units) {
                const long long e = u / C.nT;
                const int t = (int)(u - e * C.nT);
                if ((C.mask_in[e] >> t) & 1u) {
                    float P[NP * M], S, lo[M], hi[M];
                    unit_points<M, G, PD>(C, C.src[e], C.col_in[e], t, P, S, lo, hi);
#pragma unroll
                    for (int k = 0; k < NP * M; ++k) sP[lane * PS + k] = P[k];
                    sS[lane] = S;
#pragma unroll
                    for (int a = 0; a < M; ++a) {
                        sLo[lane * 4 + a] = lo[a];
                        sHi[lane * 4 + a] = hi[a];
                    }
                    st = 0;
                    ++n_units;
                }
            }
            sState[lane] = st;
        }
        __syncthreads();
        bool done = sState[lane] != 0;
        float P[NP * M], lo[M], hi[M], S = 0.f;
#pragma unroll
        for (int k = 0; k < NP * M; ++k) P[k] = sP[lane * PS + k];
#pragma unroll
        for (int a = 0; a < M; ++a) {
            lo[a] = sLo[lane * 4 + a];
            hi[a] = sHi[lane * 4 + a];
        }
        S = sS[lane];
        for (int o = warp; o < C.n_obst; o += SCAN_WARPS) {
            done = done || vstate[lane] != 0;
            if (__all_sync(0xffffffffu, done)) break;
            bool want = false;
            if (!done) {
                ++n_tests;
                const int nr = __ldg(C.ocount + o);
                const float4* rw = reinterpret_cast<const float4*>(C.orow) + (long long)o * C.max_orows;
                // (i) bounding-box screen: the box corner lowest along A_r
                bool sep = false;
                for (int r = 0; r < nr && !sep; ++r) {
                    const float4 f = __ldg(rw + r);
                    float z[M];
                    z[0] = f.x >= 0.f ? lo[0] : hi[0];
                    z[1] = f.y >= 0.f ? lo[1] : hi[1];
                    if (M == 3) z[M - 1] = f.z >= 0.f ? lo[M - 1] : hi[M - 1];
                    sep = margin32<M>(f, z) > band32<M>(f, S);
                }
                if (sep) {
                    ++n_box;
                } else {
                    // (ii) the margins: a facet above every band separates; a
                    // point below every band is inside
                    float gmax[NP];
#pragma unroll
                    for (int l = 0; l < NP; ++l) gmax[l] = -__int_as_float(0x7f800000);
                    bool sep2 = false;
                    for (int r = 0; r < nr; ++r) {
                        const float4 f = __ldg(rw + r);
                        const float band = band32<M>(f, S);
                        float mn = __int_as_float(0x7f800000);
#pragma unroll
                        for (int l = 0; l < NP; ++l) {
                            const float gv = margin32<M>(f, P + l * M);
                            mn = fminf(mn, gv);
                            gmax[l] = fmaxf(gmax[l], gv + band);
                        }
                        if (mn > band) {
                            sep2 = true;
                            break;
                        }
                    }
                    if (sep2) {
                        ++n_s2;
                    } else {
                        bool in = false;
#pragma unroll
                        for (int l = 0; l < NP; ++l) in = in || gmax[l] <= 0.f;
                        if (in) {
                            ++n_s1;
                            done = true;
                            vstate[lane] = 1;
                        } else {
                            want = true;
                        }
                    }
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, want);
            if (bal) {
                const int leader = __ffs(bal) - 1;
                unsigned long long base = 0;
                if (lane == leader) base = atomicAdd(&C.info->cut_lp, (unsigned long long)__popc(bal));
                base = __shfl_sync(0xffffffffu, base, leader);
                if (want) {
                    const unsigned long long idx = base + __popc(bal & ((1u << lane) - 1u));
                    if (idx < (unsigned long long)C.cap32)
                        C.list32[idx] = ((unsigned long long)(g0 + lane) << OBST_BITS) | (unsigned long long)o;
                }
            }
        }
        __syncthreads();
        if (warp == 0 && sState[lane] == 1) {
            const long long u = g0 + lane, e = u / C.nT;
            atomicOr(&C.hit[e], 1u << (int)(u - e * C.nT));
        }
        __syncthreads();
    }
    cut_block_add(&C.info->cut_units, n_units);
    cut_block_add(&C.info->cut_tests, n_tests);
    cut_block_add(&C.info->cut_box, n_box);
    cut_block_add(&C.info->cut_step1, n_s1);
    cut_block_add(&C.info->cut_step2, n_s2);
}

// ---------------------------------------------------------------------------
// The matrix game of G (NP rows l, nr columns r, G[l * nr + r]) by the
// simplex method with Bland's rule: with c = 1 - min G every payoff
// M = G + c is >= 1; maximise sum_l u_l subject to sum_l M[l][r] u_l <= 1 for
// every r, u >= 0 (the slack basis is feasible).  At the optimum
// delta* = 1 / sum u - c, lambda = u (the row player's mix, unnormalised) and
// y_r = minus the reduced cost of slack r (the column player's mix).  The
// tableau lives in local memory with the row stride of the actual nr.
// Returns false if GAME_ITERS pivots did not reach optimality; lambda and y
// are then whatever the last basis gives (the caller only uses them as
// certificate candidates).
// ---------------------------------------------------------------------------
template <typename F, int NP>
CDEV bool game_solve(const F* G, int nr, F* lam, F* y, F& value, F tol) {
    constexpr int NCMAX = NP + CUT_RMAX + 1;
    F tab[CUT_RMAX * NCMAX];
    F obj[NCMAX];
    int basis[CUT_RMAX];
    const int nc = NP + nr + 1, rhs = NP + nr;
    F gmin = G[0];
    for (int k = 1; k < NP * nr; ++k) gmin = G[k] < gmin ? G[k] : gmin;
    const F shift = F(1) - gmin;
    for (int r = 0; r < nr; ++r) {
        F* row = tab + r * nc;
        for (int l = 0; l < NP; ++l) row[l] = G[l * nr + r] + shift;
        for (int k = 0; k < nr; ++k) row[NP + k] = k == r ? F(1) : F(0);
        row[rhs] = F(1);
        basis[r] = NP + r;
    }
    for (int j = 0; j < nc; ++j) obj[j] = j < NP ? F(1) : F(0);
    bool optimal = false;
    for (int it = 0; it < GAME_ITERS; ++it) {
        int enter = -1;
        for (int j = 0; j < NP + nr; ++j)
            if (obj[j] > tol) {
                enter = j;
                break;
            }
        if (enter < 0) {
            optimal = true;
            break;
        }
        int leave = -1;
        F best = F(0);
        for (int r = 0; r < nr; ++r) {
            const F a = tab[r * nc + enter];
            if (a > tol) {
                const F ratio = tab[r * nc + rhs] / a;
                if (leave < 0 || ratio < best || (ratio == best && basis[r] < basis[leave])) {
                    best = ratio;
                    leave = r;
                }
            }
        }
        if (leave < 0) break;  // unbounded: impossible with payoffs >= 1
        F* prow = tab + leave * nc;
        const F inv = F(1) / prow[enter];
        for (int j = 0; j < nc; ++j) prow[j] *= inv;
        prow[enter] = F(1);
        for (int r = 0; r < nr; ++r) {
            if (r == leave) continue;
            F* row = tab + r * nc;
            const F f = row[enter];
            if (f != F(0)) {
                for (int j = 0; j < nc; ++j) row[j] -= f * prow[j];
                row[enter] = F(0);
            }
        }
        const F f = obj[enter];
        for (int j = 0; j < nc; ++j) obj[j] -= f * prow[j];
        obj[enter] = F(0);
        basis[leave] = enter;
    }
    for (int l = 0; l < NP; ++l) lam[l] = F(0);
    F z = F(0);
    for (int r = 0; r < nr; ++r)
        if (basis[r] < NP) {
            const F v = tab[r * nc + rhs];
            lam[basis[r]] = v > F(0) ? v : F(0);
        }
    for (int l = 0; l < NP; ++l) z += lam[l];
    for (int r = 0; r < nr; ++r) {
        const F v = -obj[NP + r];
        y[r] = v > F(0) ? v : F(0);
    }
    value = z > F(0) ? F(1) / z - shift : F(0);
    return optimal;
}

// Certificates from a game solution, for margins known to within band[r] of
// the canonical ones (band = 0 for the canonical margins themselves) and
// evaluated with unit roundoff uu.  hit: lambda >= 0 with every
// (G^T lambda)_r + (sum lambda) band_r below zero beyond the evaluation's own
// rounding.  miss: y >= 0 with every (G y)_l - sum_r y_r band_r above zero.
template <typename F, int NP>
CDEV bool certify_hit(const F* G, int nr, const F* band, const F* lam, F uu) {
    F L = F(0);
    for (int l = 0; l < NP; ++l) L += lam[l];
    if (!(L > F(0))) return false;
    const F k = F(2 * (NP + 2)) * uu;
    for (int r = 0; r < nr; ++r) {
        F s = F(0), a = F(0);
        for (int l = 0; l < NP; ++l) {
            s += lam[l] * G[l * nr + r];
            a += lam[l] * (G[l * nr + r] < F(0) ? -G[l * nr + r] : G[l * nr + r]);
        }
        if (!(s + L * band[r] + k * a < F(0))) return false;
    }
    return true;
}
template <typename F, int NP>
CDEV bool certify_miss(const F* G, int nr, const F* band, const F* y, F uu) {
    F Y = F(0);
    for (int r = 0; r < nr; ++r) Y += y[r] * band[r];
    const F k = F(2 * (nr + 2)) * uu;
    for (int l = 0; l < NP; ++l) {
        F s = F(0), a = F(0);
        for (int r = 0; r < nr; ++r) {
            s += y[r] * G[l * nr + r];
            a += y[r] * (G[l * nr + r] < F(0) ? -G[l * nr + r] : G[l * nr + r]);
        }
        if (!(s - Y - k * a > F(0))) return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// Pass B: one thread per game-list entry.
// ---------------------------------------------------------------------------
template <int M, int G, int PD>
__global__ void __launch_bounds__(128) k_cut_lp32(CutParams C) {
    constexpr int NP = PD + 1;
    const long long n = block_count(C.info, &C.info->cut_lp, C.cap32);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const unsigned long long en = C.list32[k];
        const long long u = (long long)(en >> OBST_BITS);
        const int o = (int)(en & ((1ull << OBST_BITS) - 1ull));
        const long long e = u / C.nT;
        const int t = (int)(u - e * C.nT);
        if ((*(volatile const uint32_t*)(C.hit + e) >> t) & 1u) continue;
        float P[NP * M], S, lo[M], hi[M];
        unit_points<M, G, PD>(C, C.src[e], C.col_in[e], t, P, S, lo, hi);
        const int nr = C.ocount[o];
        const float4* rw = reinterpret_cast<const float4*>(C.orow) + (long long)o * C.max_orows;
        float Gm[NP * CUT_RMAX], band[CUT_RMAX];
        for (int r = 0; r < nr; ++r) {
            const float4 f = rw[r];
            band[r] = band32<M>(f, S);
#pragma unroll
            for (int l = 0; l < NP; ++l) Gm[l * nr + r] = margin32<M>(f, P + l * M);
        }
        float lam[NP], y[CUT_RMAX], val;
        game_solve<float, NP>(Gm, nr, lam, y, val, 1e-6f);
        if (certify_hit<float, NP>(Gm, nr, band, lam, U32)) {
            atomicOr(&C.hit[e], 1u << t);
        } else if (!certify_miss<float, NP>(Gm, nr, band, y, U32)) {
            const unsigned long long idx = atomicAdd(&C.info->cut_lp64, 1ull);
            if (idx < (unsigned long long)C.cap64) C.list64[idx] = en;
        }
    }
}

// ---------------------------------------------------------------------------
// Pass C: canonical FP64 margins (the oracle's order: each control-point half
// summed left to right from 0, halves added; facet products summed left to
// right from 0, then b subtracted; no FMA), Algorithm 2's two checks, the
// game with exact-rounding certificates, ties by the value's sign.
// ---------------------------------------------------------------------------
template <int G>
CDEV double half64(const double* coef, const double* x, int stride) {
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < G; ++c) s = __dadd_rn(s, __dmul_rn(coef[c], x[c * stride]));
    return s;
}

template <int M, int G, int PD>
__global__ void __launch_bounds__(128) k_cut_lp64(CutParams C) {
    constexpr int N_ = M * G, NP = PD + 1, TG = 2 * G;
    const long long n = block_count(C.info, &C.info->cut_lp64, C.cap64);
    const long long stride = (long long)gridDim.x * blockDim.x;
    unsigned long long n_ties = 0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const unsigned long long en = C.list64[k];
        const long long u = (long long)(en >> OBST_BITS);
        const int o = (int)(en & ((1ull << OBST_BITS) - 1ull));
        const long long e = u / C.nT;
        const int t = (int)(u - e * C.nT);
        if ((*(volatile const uint32_t*)(C.hit + e) >> t) & 1u) continue;
        const long long i = C.src[e], j = C.col_in[e];
        double xi[N_], xj[N_];
#pragma unroll
        for (int c = 0; c < N_; ++c) {
            xi[c] = ld64(C.states, i * N_ + c, C.in_f32);
            xj[c] = ld64(C.states, j * N_ + c, C.in_f32);
        }
        const double* D = C.tab64 + (long long)t * C.L.e_stride + C.L.e_D;
        double P[NP * M];
#pragma unroll
        for (int l = 0; l < NP; ++l)
#pragma unroll
            for (int a = 0; a < M; ++a)
                P[l * M + a] = __dadd_rn(half64<G>(D + l * TG, xi + a, M), half64<G>(D + l * TG + G, xj + a, M));
        const int r0 = C.obst_off[o], nr = C.ocount[o];
        double Gm[NP * CUT_RMAX], zero[CUT_RMAX];
        for (int r = 0; r < nr; ++r) {
            zero[r] = 0.0;
            const double br = ld64(C.b, r0 + r, C.in_f32);
            double Ar[M];
#pragma unroll
            for (int a = 0; a < M; ++a) Ar[a] = ld64(C.A, (long long)(r0 + r) * M + a, C.in_f32);
#pragma unroll
            for (int l = 0; l < NP; ++l) {
                double s = 0.0;
#pragma unroll
                for (int a = 0; a < M; ++a) s = __dadd_rn(s, __dmul_rn(Ar[a], P[l * M + a]));
                Gm[l * nr + r] = __dsub_rn(s, br);
            }
        }
        int verdict = 0;  // 1 hit, -1 miss
        for (int l = 0; l < NP && verdict == 0; ++l) {  // a control point inside
            bool in = true;
            for (int r = 0; r < nr; ++r) in = in && Gm[l * nr + r] <= 0.0;
            if (in) verdict = 1;
        }
        for (int r = 0; r < nr && verdict == 0; ++r) {  // one separating facet
            bool out = true;
            for (int l = 0; l < NP; ++l) out = out && Gm[l * nr + r] > 0.0;
            if (out) verdict = -1;
        }
        if (verdict == 0) {
            double lam[NP], y[CUT_RMAX], val;
            game_solve<double, NP>(Gm, nr, lam, y, val, 1e-13);
            if (certify_hit<double, NP>(Gm, nr, zero, lam, U64)) verdict = 1;
            else if (certify_miss<double, NP>(Gm, nr, zero, y, U64)) verdict = -1;
            else {
                verdict = val <= 0.0 ? 1 : -1;
                ++n_ties;
            }
        }
        if (verdict == 1) atomicOr(&C.hit[e], 1u << t);
    }
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
            if (C.info->cut_lp > (unsigned long long)C.cap32 || C.info->cut_lp64 > (unsigned long long)C.cap64)
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
int launch_cut_t(const CutParams& C, cudaStream_t st, int num_sms, int* launches) {
    const int row_blocks = (int)((((long long)C.N * 32 + 255) / 256) < num_sms * 8 ? ((long long)C.N * 32 + 255) / 256
                                                                                   : num_sms * 8);
    const long long orows = (long long)C.n_obst * C.max_orows;
    const int obst_blocks = (int)((orows + 255) / 256);
    const int prep_blocks = (row_blocks > 0 ? row_blocks : 1) + obst_blocks;
    k_cut_prep<<<prep_blocks, 256, 0, st>>>(C, row_blocks > 0 ? row_blocks : 1);
    const long long units = C.cap_in * C.nT;
    long long ga = (units + 31) / 32;
    if (ga > (long long)num_sms * 8) ga = (long long)num_sms * 8;
    if (ga < 1) ga = 1;
    k_cut_scan<M, G, PD><<<(int)ga, 256, 0, st>>>(C);
    k_cut_lp32<M, G, PD><<<num_sms * 4, 128, 0, st>>>(C);
    k_cut_lp64<M, G, PD><<<num_sms, 128, 0, st>>>(C);
    long long gc = C.nchunks < (long long)num_sms * 4 ? C.nchunks : (long long)num_sms * 4;
    if (gc < 1) gc = 1;
    k_cut_count<<<(int)gc, FILL_THREADS, 0, st>>>(C);
    k_cut_offsets<<<1, 1024, 0, st>>>(C);
    k_cut_fill<M, G, PD><<<(int)gc, FILL_THREADS, 0, st>>>(C);
    k_cut_rows<<<(int)((C.N + 1 + 255) / 256), 256, 0, st>>>(C);
    *launches += 8;
    return (int)cudaGetLastError();
}

}  // namespace

int launch_cut(const CutParams& C, void* stream, int num_sms, int* launches) {
    cudaStream_t st = (cudaStream_t)stream;
    if (C.m == 2 && C.g == 2 && C.p == 3) return launch_cut_t<2, 2, 3>(C, st, num_sms, launches);
    if (C.m == 2 && C.g == 2 && C.p == 5) return launch_cut_t<2, 2, 5>(C, st, num_sms, launches);
    if (C.m == 3 && C.g == 3 && C.p == 5) return launch_cut_t<3, 3, 5>(C, st, num_sms, launches);
    if (C.m == 3 && C.g == 3 && C.p == 7) return launch_cut_t<3, 3, 7>(C, st, num_sms, launches);
    return (int)cudaErrorInvalidValue;
}

}  // namespace plan
