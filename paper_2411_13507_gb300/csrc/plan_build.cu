// Edge-build kernels for sm_103a: membership, per-polytope member lists, the
// pair kernels (FP32 fast path with error bands, FP64 canonical path), the
// FP64 re-check of ambiguous margins and the CSR compaction.
//
// Method (arXiv 2411.13507):
//  * Sec. III-A buildGraph: e_ij exists iff F [v_i; v_j] <= G (Theorem 1),
//    taken per axis as |Q^(k)_j| <= c_k on the hodograph control points of
//    every derivative order k = 1..gamma of the Lemma-1 curve.
//  * Property 1 + keep-in polytope: the curve stays in a shared free polytope
//    when every control point satisfies A P_l <= b (interior l; the end points
//    are the states, which are members).
//  * Sec. III-C: edge cost = control-polygon length of the state-space
//    control points (Property 2); one edge weight = min over feasible T.
//
// All four tests are linear in xi = [x_i; x_j], so every row value splits
// into a start half (depends on x_i only) and an end half (x_j only).  The
// halves of a tile of states are computed once per duration into shared
// memory and each pair costs one add per row ("outer sum"), reduced with a
// max in registers.  Canonical FP64 order (the definition of a bit-exact
// result) is: each half summed left to right without FMA, then the two
// halves added; see the FP64 kernel and the re-check kernel.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "plan_internal.h"

namespace plan {

#define DEVI __device__ __forceinline__

// Error-band constants (multiples of the FP32 unit roundoff u = 2^-24).
// Reach row: x~ (1) + coefficient (1) + product (1) + g-1 sums + final add
// <= 7 roundings for g <= 4; factor 2 margin -> 16u.  Free row: adds the
// control-point products, the polytope products (m-1 sums) and the bound:
// <= 12 roundings -> 24u.  Membership: m products and sums + bound -> 16u.
// The FP64 canonical value is within 4 * 2^-53 of the exact value, far inside
// the margin.  A margin whose computed value is within band of zero is
// re-evaluated in canonical FP64.
constexpr float KU = 5.9604644775390625e-08f;  // 2^-24
constexpr float KR = 16.f * KU;
// (The screened kernel forms P = start half + end half of each interior
// control point and then A_r . P - b_r: the halves' chains, one add, m
// products and sums and the bound -- fewer roundings than the bound below
// allows, over the same magnitude.)
constexpr float KF = 24.f * KU;
constexpr float KMEM = 16.f * KU;
// Half-precision screen.  The screen row-axes of the reach halves are rounded
// to FP16 and summed in FP16.  Each of those three roundings errs by at most
// 2^-11 of its result (2^-25 absolute below the normal range), so the FP16 sum
// is within 2^-10 (1 + 2^-11) (|u| + |w|) + 3 * 2^-25 of the exact sum u + w of
// the FP32 halves, and the reach band already bounds that sum's distance to
// the exact margin; |u| <= magR of its state (the band magnitude bounds every
// reach row-axis).
// The screen therefore widens the reach band by KH = 2^-9 times the magnitude
// sum (1.999 times the bound) plus EH = 2^-20, and rejects nothing whose magnitude
// sum exceeds MAGH (there the FP16 values could overflow).
constexpr float KH = 1.953125e-03f;         // 2^-9
constexpr float EH = 9.5367431640625e-07f;  // 2^-20
constexpr float MAGH = 16384.f;
// FP32 cost conditioning.  A cost is a sum of segment norms of (start half +
// end half) rows; its rounding error stays below about 1.2 u times the sum of
// |half| over all rows (measured over every feasible check of the 2-D and 3-D
// workloads, both interior readings), so a cost whose half-magnitude sum
// exceeds COST_RHO times the cost (error bound ~3.5e-6 relative, e.g. two
// nearly equal states whose halves cancel) is recomputed in FP64 instead.
constexpr float COST_RHO = 48.f;
constexpr unsigned long long KEY_NONE = ~0ull;
constexpr unsigned long long DINF_BITS = 0x7FF0000000000000ull;

DEVI void set_status(DevInfo* info, int code, int detail) {
    if (atomicCAS(&info->status, 0, code) == 0) atomicExch(&info->detail, detail);
}
DEVI bool has_failed(const DevInfo* info) { return *((volatile const int*)&info->status) != 0; }

// The call's status and one of its counters, read by one thread per block and
// shared: thousands of warps reading the same word would all queue at one L2
// slice.  Every thread of the block must call it (it holds a barrier).
DEVI bool block_failed(const DevInfo* info, const unsigned long long* counter, long long* n) {
    __shared__ int s_fail;
    __shared__ long long s_n;
    if (threadIdx.x == 0) {
        s_fail = has_failed(info);
        s_n = counter ? (long long)*(volatile const unsigned long long*)counter : 0;
    }
    __syncthreads();
    if (n) *n = s_n;
    return s_fail != 0;
}

// Adds every thread's v to *dst with one global atomic per block (shared
// atomics first).  Every thread of the block must call it.
DEVI void block_add(unsigned long long* dst, unsigned long long v) {
    __shared__ unsigned long long s_acc;
    if (threadIdx.x == 0) s_acc = 0;
    __syncthreads();
    if ((blockDim.x & 31) == 0) {  // whole warps: reduce in registers first
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&s_acc, v);
    } else if (v) {
        atomicAdd(&s_acc, v);
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_acc) atomicAdd(dst, s_acc);
}

DEVI double ldv(const void* p, long long i, int f32) {
    return f32 ? (double)((const float*)p)[i] : ((const double*)p)[i];
}
DEVI float ldf(const void* p, long long i, int f32) {
    return f32 ? ((const float*)p)[i] : (float)((const double*)p)[i];
}

DEVI unsigned long long key_f32(float cost, int t) {
    return ((unsigned long long)__float_as_uint(cost) << 32) | (unsigned)t;
}
DEVI unsigned long long key_f64(double cost, int t) {
    return ((unsigned long long)__double_as_longlong(cost) & ~31ull) | (unsigned)t;
}

template <int G, int PD>
struct Shape {
    static constexpr int RAX = (G >= 1 ? PD : 0) + (G >= 2 ? PD - 1 : 0) + (G >= 3 ? PD - 2 : 0) + (G >= 4 ? PD - 3 : 0);
    static constexpr int NI = PD - 1;
    static constexpr int TG = 2 * G;
};

// Member-list entries carry the state id in bits 0..30 and, in bit 31, whether
// the state lies in more than one polytope (only then can a pair be shared by
// several polytopes).
constexpr int MULTI_BIT = (int)0x80000000u;
DEVI int mem_id(int v) { return v & 0x7fffffff; }
DEVI bool mem_multi(int v) { return v < 0; }

// First position in an ascending member list whose state id is >= j.
DEVI int lower_bound_members(const int* mem, int n, int j) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (mem_id(mem[mid]) < j) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Largest q with pfx[q] <= x (pfx ascending, pfx[Q] > x): query of a global index.
DEVI int find_q(const long long* pfx, int Q, long long x) {
    int lo = 0, hi = Q;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pfx[mid] <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Rows of every polytope: FP32 copies, b - eps, row-count checks.
// ---------------------------------------------------------------------------
__global__ void k_prep(BuildParams P) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= P.totRows) return;
    const int q = find_q(P.pfxRows, P.Q, t);
    const QueryDesc& Q = P.qd[q];
    const long long loc = t - P.pfxRows[q];
    const int k = (int)(loc / P.max_rows), rr = (int)(loc % P.max_rows);
    const int r0 = Q.poly_off[k], r1 = Q.poly_off[k + 1];
    if (rr == 0) {
        const int nr = r1 - r0;
        if (nr < 0 || nr > P.max_rows || (k == 0 && r0 != 0)) set_status(P.info, PLAN_ERR_UNSUPPORTED, DET_ROWS);
        atomicMax(&P.info->max_rows_seen, nr);
    }
    const int r = r0 + rr;
    if (r >= r1 || r < 0 || r >= Q.K * P.max_rows) return;
    const long long rg = Q.rowsOff + r;
    const double bl = __dsub_rn(ldv(Q.b, r, P.in_f32), P.eps);
    P.blim64[rg] = bl;
    P.blim32[rg] = (float)bl;
    for (int a = 0; a < P.m; ++a) P.A32[rg * P.m + a] = ldf(Q.A, (long long)r * P.m + a, P.in_f32);
}

// ---------------------------------------------------------------------------
// A1 membership: bit k of state i set iff A_k x_i^(0) <= b_k - eps on every
// row (canonical FP64 decision; FP32 first, FP64 only inside the band).
// ---------------------------------------------------------------------------
DEVI void member_word(const BuildParams& P, long long t, int lane) {
    const int q = find_q(P.pfxMask, P.Q, t);
    const QueryDesc& Q = P.qd[q];
    const float* A32 = P.A32 + Q.rowsOff * P.m;
    const float* lim32 = P.blim32 + Q.rowsOff;
    const int* poff = Q.poly_off;
    const long long loc = t - P.pfxMask[q];
    const int i = (int)(loc / Q.W), w = (int)(loc % Q.W);
    const int m = P.m, n = P.m * P.g;
    double x64[4];
    float x32[4];
    for (int a = 0; a < m; ++a) {
        x64[a] = ldv(Q.states, (long long)i * n + a, P.in_f32);
        x32[a] = (float)x64[a];
    }
    const int k = w * 32 + lane;  // this lane's polytope
    bool in = k < Q.K;
    if (in) {
        const int r0 = poff[k], r1 = poff[k + 1];
        if (r1 - r0 > P.max_rows || r1 > Q.K * P.max_rows || r0 < 0) in = false;
        // four rows per step: their loads are issued together
        for (int rb = r0; rb < r1 && in; rb += 4) {
            float av[4][4], lim[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool ok = rb + u < r1;
#pragma unroll
                for (int a = 0; a < 4; ++a) av[u][a] = (ok && a < m) ? A32[(long long)(rb + u) * m + a] : 0.f;
                lim[u] = ok ? lim32[rb + u] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (rb + u >= r1 || !in) break;
                const long long rg = Q.rowsOff + rb + u;
                float s = 0.f, mag = 0.f;
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    if (a < m) {
                        s = fmaf(av[u][a], x32[a], s);
                        mag = fmaf(fabsf(av[u][a]), fabsf(x32[a]), mag);
                    }
                }
                const float d = s - lim[u];
                const float band = KMEM * (mag + fabsf(lim[u]));
                if (!(d < -band)) {
                    if (d > band) {
                        in = false;
                    } else {  // within the band (or NaN): canonical FP64 row
                        double sd = 0.0;
                        for (int a = 0; a < m; ++a)
                            sd = __dadd_rn(sd, __dmul_rn(ldv(Q.A, (long long)(rb + u) * m + a, P.in_f32), x64[a]));
                        if (!(sd <= P.blim64[rg])) in = false;
                    }
                }
            }
        }
    }
    const uint32_t word = __ballot_sync(0xffffffffu, in);
    if (lane == 0) P.memMask[Q.maskOff + (long long)i * Q.W + w] = word;
}

__global__ void __launch_bounds__(256, 4) k_member(BuildParams P) {
    const int lane = threadIdx.x & 31;
    if (block_failed(P.info, nullptr, nullptr)) return;
    // one warp per (state, word), persistent: a single wave of CTAs loops
    // over the items (each is a short chain of dependent loads)
    for (long long t = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; t < P.totMask;
         t += ((long long)gridDim.x * blockDim.x) >> 5)
        member_word(P, t, lane);
}

// ---------------------------------------------------------------------------
// Ordered member list of each polytope (ascending state id), local indices,
// block centre (first member's position) and centred FP32 bounds.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_lists(BuildParams P) {
    const int q = find_q(P.pfxPoly, P.Q, blockIdx.x);
    const QueryDesc& Q = P.qd[q];
    const int k = (int)(blockIdx.x - P.pfxPoly[q]);
    __shared__ int warpTot[32];
    __shared__ int s_base, s_step;
    __shared__ float s_c[4];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    const int w = k >> 5;
    const uint32_t bit = 1u << (k & 31);
    int* members = P.members + Q.listOff + (long long)k * Q.N;
    int* localIdx = P.localIdx + Q.listOff + (long long)k * Q.N;
    constexpr int PER = 8;  // consecutive states per thread: one block step covers 8192 states
    for (int i0 = 0; i0 < Q.N; i0 += blockDim.x * PER) {
        const int ib = i0 + threadIdx.x * PER;
        unsigned mine = 0;  // bit u: state ib + u is a member
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int i = ib + u;
            if (i < Q.N && (P.memMask[Q.maskOff + (long long)i * Q.W + w] & bit)) mine |= 1u << u;
        }
        const int cnt = __popc(mine);
        int inc = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) warpTot[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            int v = lane < nw ? warpTot[lane] : 0;
            int wi = v;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            if (lane < nw) warpTot[lane] = wi - v;
            if (lane == nw - 1) s_step = wi;  // the step's total
        }
        __syncthreads();
        int pos = s_base + warpTot[wid] + inc - cnt;
        for (unsigned bits = mine; bits; bits &= bits - 1u, ++pos) {
            const int i = ib + __ffs(bits) - 1;
            int npoly = 0;
            for (int w2 = 0; w2 < Q.W; ++w2) npoly += __popc(P.memMask[Q.maskOff + (long long)i * Q.W + w2]);
            members[pos] = i | (npoly > 1 ? MULTI_BIT : 0);
            localIdx[i] = pos;
        }
        __syncthreads();
        if (threadIdx.x == 0) s_base += s_step;
        __syncthreads();
    }
    const int nk = s_base;
    if (threadIdx.x == 0) {
        P.counts[Q.kOff + k] = nk;
        const int n = P.m * P.g;
        for (int a = 0; a < 4; ++a) {
            float c = 0.f;
            if (nk > 0 && a < P.m) c = ldf(Q.states, (long long)mem_id(members[0]) * n + a, P.in_f32);
            s_c[a] = c;
            P.centers[(long long)(Q.kOff + k) * 4 + a] = c;
        }
    }
    __syncthreads();
    const int r0 = Q.poly_off[k], r1 = Q.poly_off[k + 1];
    for (int r = r0 + threadIdx.x; r < r1 && r < Q.K * P.max_rows; r += blockDim.x) {
        double sacc = 0.0;
        for (int a = 0; a < P.m; ++a) sacc += ldv(Q.A, (long long)r * P.m + a, P.in_f32) * (double)s_c[a];
        P.bc32[Q.rowsOff + r] = (float)(P.blim64[Q.rowsOff + r] - sacc);
    }
}

// ---------------------------------------------------------------------------
// Work decomposition: per polytope, balanced square tiles of <= tile states;
// prefix sums of slots (n_k^2) and tiles; capacity checks.
// ---------------------------------------------------------------------------
template <typename T>
DEVI T block_exclusive_scan(T v, T* warpbuf, T* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warpbuf[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        T s = lane < nw ? warpbuf[lane] : (T)0;
        T si = s;
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += y;
        }
        if (lane < nw) warpbuf[lane] = si - s;
        if (lane == 31) *total = si;
    }
    __syncthreads();
    T r = warpbuf[wid] + inc - v;
    __syncthreads();
    return r;
}

// Source-row range of a query's shard: the rows are cut into nshard
// contiguous ranges of equal work, the work of row i being its pair slots
// sum_{k holds i} n_k.  With S_i the work of rows < i and W the total, shard
// r starts at the number of rows with S_i * nshard < W * r (S is
// non-decreasing, so those rows form a prefix); the last shard ends at N.
// Every rank computes the same cut points from the same membership.  One CTA
// per query; every thread must call it.
DEVI void shard_rows(const BuildParams& P, const QueryDesc& Q, int* s_counts, long long* wb, long long* tot,
                     int& lo, int& hi) {
    lo = 0;
    hi = Q.N;
    if (Q.nshard <= 1) return;
    for (int k = threadIdx.x; k < Q.K; k += blockDim.x) s_counts[k] = P.counts[Q.kOff + k];
    __syncthreads();
    const uint32_t* mask = P.memMask + Q.maskOff;
    auto row_work = [&](int i) -> long long {
        long long w = 0;
        if (i < Q.N)
            for (int wd = 0; wd < Q.W; ++wd) {
                uint32_t x = mask[(long long)i * Q.W + wd];
                while (x) {
                    w += s_counts[wd * 32 + __ffs(x) - 1];
                    x &= x - 1u;
                }
            }
        return w;
    };
    long long W = 0;
    for (int i0 = 0; i0 < Q.N; i0 += blockDim.x) {
        block_exclusive_scan<long long>(row_work(i0 + threadIdx.x), wb, tot);
        W += *tot;
        __syncthreads();
    }
    const long long tlo = W * Q.shard, thi = W * (Q.shard + 1);
    long long carry = 0, nlo = 0, nhi = 0;
    for (int i0 = 0; i0 < Q.N; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        const long long ex = block_exclusive_scan<long long>(row_work(i), wb, tot);
        const long long S = carry + ex;
        const int blo = (i < Q.N && S * Q.nshard < tlo) ? 1 : 0;
        const int bhi = (i < Q.N && S * Q.nshard < thi) ? 1 : 0;
        carry += *tot;
        __syncthreads();
        block_exclusive_scan<long long>(blo, wb, tot);
        nlo += *tot;
        __syncthreads();
        block_exclusive_scan<long long>(bhi, wb, tot);
        nhi += *tot;
        __syncthreads();
    }
    lo = (int)nlo;
    hi = Q.shard + 1 == Q.nshard ? Q.N : (int)nhi;
}

// One CTA per query: the shard's row range, then balanced tiles and slot
// offsets of its polytopes.  Every polytope keeps its full n_k x n_k slot
// block; the i-tiles cover only the members whose ids lie in the row range
// (a contiguous part of the ascending member list), the j-tiles all members.
__global__ void __launch_bounds__(1024) k_setup(BuildParams P) {
    __shared__ long long wb[32];
    __shared__ long long tot;
    __shared__ int s_counts[1024];
    __shared__ int s_items[1024];
    const int q = blockIdx.x;
    const QueryDesc& Q = P.qd[q];
    const int tile = P.tile;
    int rlo, rhi;
    shard_rows(P, Q, s_counts, wb, &tot, rlo, rhi);
    if (threadIdx.x == 0) {
        P.rowRange[2 * q] = rlo;
        P.rowRange[2 * q + 1] = rhi;
        if (q == 0) {
            P.info->shard_lo = rlo;
            P.info->shard_hi = rhi;
        }
    }
    long long slots = 0, items = 0, mem = 0;
    long long carry_s = 0, carry_i = 0, carry_m = 0;
    int my_key = 0, my_items = 0;  // tile area and items of this thread's polytope (K <= blockDim.x)
    for (int k0 = 0; k0 < Q.K; k0 += blockDim.x) {
        const int k = k0 + threadIdx.x;
        const long long nk = (k < Q.K) ? P.counts[Q.kOff + k] : 0;
        if (nk > NK_MAX) set_status(P.info, PLAN_ERR_UNSUPPORTED, DET_NK);
        int a = 0, b = (int)nk;
        if (Q.nshard > 1 && k < Q.K && nk <= NK_MAX) {
            const int* ml = P.members + Q.listOff + (long long)k * Q.N;
            a = lower_bound_members(ml, (int)nk, rlo);
            b = lower_bound_members(ml, (int)nk, rhi);
        }
        const int nt = nk > 0 ? (int)((nk + tile - 1) / tile) : 0;
        const int ts = nt ? (int)((nk + nt - 1) / nt) : 0;
        const int ni = b - a;
        const int nti = ni > 0 ? (ni + tile - 1) / tile : 0;
        const int tsi = nti ? (ni + nti - 1) / nti : 0;
        const long long so = block_exclusive_scan<long long>(nk * nk, wb, &tot);
        slots = tot;
        const long long io = block_exclusive_scan<long long>((long long)nti * nt, wb, &tot);
        items = tot;
        const long long mo = block_exclusive_scan<long long>(nk, wb, &tot);
        mem = tot;
        if (k < Q.K) {
            P.memOff[Q.kOff + k] = (int)(carry_m + mo);
            P.resOff[Q.kOff + k] = carry_s + so;
            P.itemOff[Q.kOff + k] = (int)(carry_i + io);
            P.ntile[Q.kOff + k] = nt | (nti << 16);
            P.tsize[Q.kOff + k] = ts | (tsi << 16);
            P.iRange[Q.kOff + k] = a | (b << 16);
            my_items = nti * nt;
            my_key = my_items > 0 ? ts * tsi : 0;
        }
        carry_s += slots;
        carry_i += items;
        carry_m += mem;
    }
    // Item order: polytopes by tile area, largest first (ties by index), so
    // that the last items the blocks take are the smallest ones; itemOff is
    // the prefix of the items in that order.  More polytopes than threads
    // keep the index order.
    if (Q.K <= (int)blockDim.x) {
        const int k = threadIdx.x;
        __syncthreads();  // s_counts is free again (shard_rows)
        if (k < Q.K) s_counts[k] = my_key;
        __syncthreads();
        if (k < Q.K) {
            int rank = 0;
            for (int k2 = 0; k2 < Q.K; ++k2) {
                const int o = s_counts[k2];
                rank += (o > my_key || (o == my_key && k2 < k)) ? 1 : 0;
            }
            P.kPerm[Q.kOff + rank] = k;
            s_items[rank] = my_items;
        }
        __syncthreads();
        const long long io = block_exclusive_scan<long long>(k < Q.K ? (long long)s_items[k] : 0ll, wb, &tot);
        if (k < Q.K) P.itemOff[Q.kOff + k] = (int)io;
    } else {
        for (int k = threadIdx.x; k < Q.K; k += blockDim.x) P.kPerm[Q.kOff + k] = k;
    }
    if (threadIdx.x == 0) {
        P.resOff[Q.kOff + Q.K] = carry_s;
        P.itemOff[Q.kOff + Q.K] = (int)carry_i;
        P.memOff[Q.kOff + Q.K] = (int)carry_m;
        P.qSlot[q + 1] = carry_s;   // per-query totals; k_batch turns them into prefixes
        P.qItem[q + 1] = carry_i;
        P.qMem[q + 1] = carry_m;
        atomicAdd(&P.info->memberships, (unsigned long long)carry_m);
    }
}

// Prefix sums of the per-query slot and tile totals; scratch capacity check.
__global__ void __launch_bounds__(1024) k_batch(BuildParams P) {
    __shared__ long long wb[32];
    __shared__ long long tot;
    long long cs = 0, ci = 0, cm = 0;
    for (int q0 = 0; q0 < P.Q; q0 += blockDim.x) {
        const int q = q0 + threadIdx.x;
        const long long vs = q < P.Q ? P.qSlot[q + 1] : 0;
        const long long vi = q < P.Q ? P.qItem[q + 1] : 0;
        const long long vm = q < P.Q ? P.qMem[q + 1] : 0;
        __syncthreads();
        const long long es = block_exclusive_scan<long long>(vs, wb, &tot);
        const long long ts = tot;
        const long long ei = block_exclusive_scan<long long>(vi, wb, &tot);
        const long long ti = tot;
        const long long em = block_exclusive_scan<long long>(vm, wb, &tot);
        const long long tmm = tot;
        if (q < P.Q) {
            P.qSlot[q + 1] = cs + es + vs;
            P.qItem[q + 1] = ci + ei + vi;
            P.qMem[q + 1] = cm + em + vm;
        }
        cs += ts;
        ci += ti;
        cm += tmm;
    }
    if (threadIdx.x == 0) {
        P.qSlot[0] = 0;
        P.qItem[0] = 0;
        P.qMem[0] = 0;
        P.info->slots = cs;
        // chunks per tile: the set value, or by default enough for about
        // itemTarget items -- one to the most durations of any query
        int tch = P.tchunks;
        if (P.itemTarget > 0) {
            const long long want = ci > 0 ? (P.itemTarget + ci - 1) / ci : 1;
            const int most = P.maxT > 0 ? P.maxT : 1;
            tch = (int)(want < 1 ? 1 : (want > most ? most : want));
        }
        P.info->tchunks = tch;
        P.info->items = ci * tch;
        if (cs > P.slotCap) {
            P.info->need_slots = cs;
            set_status(P.info, PLAN_ERR_CAPACITY, DET_SLOTS);
        }
        if (ci > 0x7fffffffLL) set_status(P.info, PLAN_ERR_UNSUPPORTED, DET_NK);
    }
}

struct Item {
    int q, k, i0, j0, TI, TJ, nk;
    long long base;   // slot of member pair (0, 0) of polytope k
};

DEVI Item item_decode(const BuildParams& P, long long item) {
    Item it;
    it.q = find_q(P.qItem, P.Q, item);
    const QueryDesc& Q = P.qd[it.q];
    const int local = (int)(item - P.qItem[it.q]);
    const int* io = P.itemOff + Q.kOff;
    int lo = 0, hi = Q.K;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (io[mid] <= local) lo = mid;
        else hi = mid;
    }
    const int k = P.kPerm[Q.kOff + lo];  // position lo of the item order
    it.k = k;
    const int loc = local - io[lo];
    const int nt = P.ntile[Q.kOff + k] & 0xffff, tsp = P.tsize[Q.kOff + k];
    const int ts = tsp & 0xffff, tsi = tsp >> 16;
    const unsigned ir = (unsigned)P.iRange[Q.kOff + k];
    const int a = (int)(ir & 0xffffu), b = (int)(ir >> 16);
    it.nk = P.counts[Q.kOff + k];
    const int ti = loc / nt, tj = loc % nt;
    it.i0 = a + ti * tsi;
    it.j0 = tj * ts;
    it.TI = min(tsi, b - it.i0);
    it.TJ = min(ts, it.nk - it.j0);
    it.base = P.qSlot[it.q] + P.resOff[Q.kOff + k];
    return it;
}

// Work item of the FP32 / tensor-core kernels: a tile and a chunk of
// durations [t0, t1).  Chunks of the longest durations (where pairs survive
// the reach test and the free and cost rows run) come first, so the costly
// items start early and the short ones fill the tail.
struct ItemT {
    Item it;
    int t0, t1;
};

DEVI ItemT item_decode_chunk(const BuildParams& P, long long item) {
    const long long tiles = P.qItem[P.Q];
    const int tch = P.itemTarget > 0 ? P.info->tchunks : P.tchunks;  // chunks of this build (k_batch)
    const int c = tch - 1 - (int)(item / tiles);
    ItemT r;
    r.it = item_decode(P, item % tiles);
    const int nT = P.qd[r.it.q].nT;
    r.t0 = (c * nT) / tch;
    r.t1 = ((c + 1) * nT) / tch;
    return r;
}

// Slots start empty (no feasible duration, no key); the pair kernels merge
// into them with atomics.
// Clears the pair slots and writes the row-segment table (segment g -> its
// polytope and local index), one warp per polytope.
__global__ void k_zero_slots(BuildParams P) {
    long long n = 0;
    if (block_failed(P.info, &P.info->slots, &n)) return;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        P.resBits[s] = 0u;
        P.resKey[s] = KEY_NONE;
    }
    const int lane = threadIdx.x & 31;
    for (long long gp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; gp < P.totPoly;
         gp += ((long long)gridDim.x * blockDim.x) >> 5) {
        const int q = find_q(P.pfxPoly, P.Q, gp);
        const QueryDesc& Q = P.qd[q];
        const int k = (int)(gp - P.pfxPoly[q]);
        const long long start = P.qMem[q] + P.memOff[Q.kOff + k];
        const int nk = P.counts[Q.kOff + k];
        for (int li = lane; li < nk; li += 32) P.segKL[start + li] = (k << 16) | li;
    }
}

constexpr int RECHECK_THREADS = 128;  // four warps (one FP64 unit each) per re-check entry

// Re-check entry: cost-only flag (1 bit) | query (16 bits) | polytope (10) | li (16) | lj (16) | T (5).
// Bit 63 marks a check that is certainly feasible and needs only its cost in
// FP64 (an ill-conditioned FP32 cost).
DEVI void append_recheck(const BuildParams& P, int q, int k, int li, int lj, int t, bool cost_only = false) {
    const unsigned long long idx = atomicAdd(&P.info->rechecks, 1ull);
    if ((long long)idx < P.recheckCap) {
        P.recheck[idx] = ((unsigned long long)cost_only << 63) | ((unsigned long long)q << 47) |
                         ((unsigned long long)k << 37) | ((unsigned long long)li << 21) |
                         ((unsigned long long)lj << 5) | (unsigned long long)t;
    } else {
        atomicMax(&P.info->need_rechecks, idx + 1);
        set_status(P.info, PLAN_ERR_CAPACITY, DET_RECHECK);
    }
}

// ---------------------------------------------------------------------------
// A2/A3 FP32 pair kernel.  Persistent CTAs pull (polytope, i-tile, j-tile)
// items; per duration the tile's halves go to shared memory and each thread
// reduces a 4x4 micro-tile of pairs.  Reach rows are ordered so that the
// rows most likely to fail (highest derivative, interior) come first, and a
// thread stops the reach loop once all its pairs have definitely failed.
// ---------------------------------------------------------------------------
// Pair phase of one duration for a thread's 4x4 micro-tile (shared by the
// FP32 kernel and the tensor-core kernel): reach rows (add, |.|, max) with an
// early stop once all 16 pairs definitely fail, free rows (add, max), cost of
// the feasible pairs; ambiguous pairs go to the FP64 re-check.
template <int M, int G, int PD>
DEVI void pair_phase(const BuildParams& P, const Item& itd, int t, int T, int gi, int gj, uint32_t vmask, uint32_t dmask,
                     int nr, int DR, const float* UL, const float* UR, const float* FL, const float* FR,
                     const float* CL, const float* CRr, const float* magR, const float* magF, float KRb, float KFb,
                     unsigned long long& rp_cnt) {
    using S = Shape<G, PD>;
    constexpr int RAX = S::RAX, NI = S::NI;
    const int k = itd.k, i0 = itd.i0, j0 = itd.j0;
    const float KR = KRb, KF = KFb;
    {
        float mRi[4], mRj[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            mRi[q] = magR[4 * gi + q];
            mRj[q] = magR[T + 4 * gj + q];
        }
        const float bmx = KR * (fmaxf(fmaxf(mRi[0], mRi[1]), fmaxf(mRi[2], mRi[3])) +
                                fmaxf(fmaxf(mRj[0], mRj[1]), fmaxf(mRj[2], mRj[3])));
        float rm[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) rm[q] = ((vmask >> q) & 1u) && !((dmask >> q) & 1u) ? 0.f : __int_as_float(0x7f800000);
        const float* ulp = UL + 4 * gi;
        const float* urp = UR + 4 * gj;
        bool dead = false;
        for (int r = 0; r < RAX; ++r) {
#pragma unroll
            for (int a = 0; a < M; ++a) {
                const float4 u = *reinterpret_cast<const float4*>(ulp + (r * M + a) * T);
                const float4 w = *reinterpret_cast<const float4*>(urp + (r * M + a) * T);
                const float uu[4] = {u.x, u.y, u.z, u.w};
                const float ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int qa = 0; qa < 4; ++qa)
#pragma unroll
                    for (int qb = 0; qb < 4; ++qb) rm[qa * 4 + qb] = fmaxf(rm[qa * 4 + qb], fabsf(uu[qa] + ww[qb]));
            }
            if ((r & 1) == 1) {
                float mn = rm[0];
#pragma unroll
                for (int q = 1; q < 16; ++q) mn = fminf(mn, rm[q]);
                if (mn > 1.f + bmx) {
                    dead = true;
                    break;
                }
            }
        }
        if (!dead) {
            uint32_t rfail = 0, rpass = 0;
#pragma unroll
            for (int qa = 0; qa < 4; ++qa)
#pragma unroll
                for (int qb = 0; qb < 4; ++qb) {
                    const int q = qa * 4 + qb;
                    const float band = KR * (mRi[qa] + mRj[qb]);
                    if (!(rm[q] <= 1.f + band)) rfail |= 1u << q;
                    else if (rm[q] <= 1.f - band) rpass |= 1u << q;
                }
            rpass &= vmask & ~dmask;
            rfail |= ~vmask | dmask;
            rfail &= 0xFFFFu;
            rp_cnt += __popc(rpass);
            if (rfail != 0xFFFFu) {
                float fm[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) fm[q] = -__int_as_float(0x7f800000);
                const float* flp = FL + 4 * gi;
                const float* frp = FR + 4 * gj;
                const int FRk = NI * nr;
                for (int r = 0; r < FRk; ++r) {
                    const float4 u = *reinterpret_cast<const float4*>(flp + r * T);
                    const float4 w = *reinterpret_cast<const float4*>(frp + r * T);
                    const float uu[4] = {u.x, u.y, u.z, u.w};
                    const float ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                    for (int qa = 0; qa < 4; ++qa)
#pragma unroll
                        for (int qb = 0; qb < 4; ++qb) fm[qa * 4 + qb] = fmaxf(fm[qa * 4 + qb], uu[qa] + ww[qb]);
                }
                uint32_t ffail = 0, fpass = 0;
                float mFi[4], mFj[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    mFi[q] = magF[4 * gi + q];
                    mFj[q] = magF[T + 4 * gj + q];
                }
#pragma unroll
                for (int qa = 0; qa < 4; ++qa)
#pragma unroll
                    for (int qb = 0; qb < 4; ++qb) {
                        const int q = qa * 4 + qb;
                        const float band = KF * (mFi[qa] + mFj[qb]);
                        if (!(fm[q] <= band)) ffail |= 1u << q;
                        else if (fm[q] <= -band) fpass |= 1u << q;
                    }
                const uint32_t feas = rpass & fpass & ~rfail & ~ffail & 0xFFFFu;
                const uint32_t amb = ~(rfail | ffail) & ~feas & 0xFFFFu;
                if (feas) {
                    float cs[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) cs[q] = 0.f;
                    const float* clp = CL + 4 * gi;
                    const float* crp = CRr + 4 * gj;
                    const int per_l = DR * M;
                    float mL[4] = {0.f, 0.f, 0.f, 0.f}, mR[4] = {0.f, 0.f, 0.f, 0.f};  // sum |half| per state
                    for (int l = 0; l < PD; ++l) {
                        float ss[16];
#pragma unroll
                        for (int q = 0; q < 16; ++q) ss[q] = 0.f;
                        for (int e = 0; e < per_l; ++e) {
                            const int row = l * per_l + e;
                            const float4 u = *reinterpret_cast<const float4*>(clp + row * T);
                            const float4 w = *reinterpret_cast<const float4*>(crp + row * T);
                            const float uu[4] = {u.x, u.y, u.z, u.w};
                            const float ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                            for (int qa = 0; qa < 4; ++qa) {
                                mL[qa] += fabsf(uu[qa]);
                                mR[qa] += fabsf(ww[qa]);
#pragma unroll
                                for (int qb = 0; qb < 4; ++qb) {
                                    const float d = uu[qa] + ww[qb];
                                    ss[qa * 4 + qb] = fmaf(d, d, ss[qa * 4 + qb]);
                                }
                            }
                        }
#pragma unroll
                        for (int q = 0; q < 16; ++q) cs[q] += sqrtf(ss[q]);
                    }
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        if ((feas >> q) & 1u) {
                            const int li = i0 + 4 * gi + (q >> 2), lj = j0 + 4 * gj + (q & 3);
                            if (P.cost64 || mL[q >> 2] + mR[q & 3] <= COST_RHO * cs[q]) {
                                const long long slot = itd.base + (long long)li * itd.nk + lj;
                                atomicOr(&P.resBits[slot], 1u << t);
                                atomicMin(&P.resKey[slot], key_f32(cs[q], t));
                            } else {
                                append_recheck(P, itd.q, k, li, lj, t, true);  // ill-conditioned FP32 cost
                            }
                        }
                    }
                }
                if (amb) {
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if ((amb >> q) & 1u) append_recheck(P, itd.q, k, i0 + 4 * gi + (q >> 2), j0 + 4 * gj + (q & 3), t);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Reach screen.  Whether a pair fails the reach test is decided, for most
// pairs, by a few reach rows: the rows whose control points depend on both
// boundary states.  Rows fixed by one end state alone only restate that
// state's own derivatives (which satisfy the bounds for states drawn inside
// them), so they seldom fail.  The screen takes the middle first-derivative
// row and the first and last second-derivative rows that mix both ends.  It
// only orders the work: a pair that passes the screen still sees every row.
// ---------------------------------------------------------------------------
template <int G, int PD>
struct Screen {
    static constexpr int NS = 3;
    // reach-row index (k-major canonical layout): k = 2, j = G-2 and j = PD-G; k = 1, j = (PD-1)/2
    static constexpr int row(int s) { return s == 0 ? PD + (G - 2) : (s == 1 ? PD + (PD - G) : (PD - 1) / 2); }
    static constexpr int index(int rr) { return rr == row(0) ? 0 : (rr == row(1) ? 1 : (rr == row(2) ? 2 : -1)); }
};

// The screen of one 4x4 micro-tile on the screen row-axes in FP16, stored
// [row][state]: start states as (h, h) pairs, end states as single halves, so
// one packed add gives two pairs' sums.  Returns the live pairs that do not
// certainly fail there (the band of the FP32 sum widened by the FP16 error).
template <int M, int G, int PD>
DEVI uint32_t screen_tile(int T, int gi, int gj, uint32_t live, const __half2* SCL, const __half* SCR, const float* magR) {
    __half2 rm[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) rm[q] = __float2half2_rn(0.f);
#pragma unroll
    for (int r = 0; r < Screen<G, PD>::NS * M; ++r) {
        const uint4 ul = *reinterpret_cast<const uint4*>(SCL + r * T + 4 * gi);
        const uint2 wr = *reinterpret_cast<const uint2*>(SCR + r * T + 4 * gj);
        const unsigned uw[4] = {ul.x, ul.y, ul.z, ul.w};
        const unsigned ww[2] = {wr.x, wr.y};
#pragma unroll
        for (int qa = 0; qa < 4; ++qa)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                __half2 u2, w2;
                __builtin_memcpy(&u2, &uw[qa], 4);
                __builtin_memcpy(&w2, &ww[h], 4);
                rm[qa * 2 + h] = __hmax2(rm[qa * 2 + h], __habs2(__hadd2(u2, w2)));
            }
    }
    uint32_t fail = 0;
#pragma unroll
    for (int qa = 0; qa < 4; ++qa)
#pragma unroll
        for (int qb = 0; qb < 4; ++qb) {
            const int q = qa * 4 + qb;
            const __half2 m2 = rm[qa * 2 + (qb >> 1)];
            const float r = (qb & 1) ? __high2float(m2) : __low2float(m2);
            const float ms = magR[4 * gi + qa] + magR[T + 4 * gj + qb];
            if (!(r <= 1.f + (KR + KH) * ms + EH) && ms <= MAGH) fail |= 1u << q;
        }
    return live & ~fail;
}

// Rows of the per-duration FP32 table as the one-group kernel stages it in
// shared memory: every table row (reach rows, interior control points, cost
// rows, the two band rows) padded to [side][4] so that one 16-byte load
// fetches the G coefficients a half needs.
template <int G, int PD>
struct PadTab {
    using S = Shape<G, PD>;
    static constexpr int ROW_D = S::RAX, ROW_C = S::RAX + S::NI, ROW_HC = ROW_C + G * PD, ROW_DC = ROW_HC + 1;
    static constexpr int NROW = ROW_DC + 1;
    static constexpr int FLOATS = NROW * 8;
};

template <int G, int PD>
DEVI void stage_table(float* dst, const float* src, int tid, int nthr) {
    constexpr int TG = 2 * G;
    for (int u = tid; u < PadTab<G, PD>::FLOATS; u += nthr) {
        const int row = u >> 3, side = (u >> 2) & 1, c = u & 3;
        dst[u] = c < G ? src[row * TG + side * G + c] : 0.f;
    }
}

// The same staging with asynchronous 4-byte copies (cp.async): the issuing
// thread does not wait for the global loads; cp.async.wait_all before the
// block barrier that precedes the table's first use completes them.
template <int G, int PD>
DEVI void stage_table_async(float* dst, const float* src, int tid, int nthr) {
    constexpr int TG = 2 * G;
    for (int u = tid; u < PadTab<G, PD>::FLOATS; u += nthr) {
        const int row = u >> 3, side = (u >> 2) & 1, c = u & 3;
        if (c < G) {
            const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst + u);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src + row * TG + side * G + c)
                         : "memory");
        } else {
            dst[u] = 0.f;
        }
    }
}
DEVI void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int M, int G, int PD>
__global__ void __launch_bounds__(256, 2) k_pairs_fast(BuildParams P) {
    using S = Shape<G, PD>;
    using PT = PadTab<G, PD>;
    constexpr int N_ = M * G, RAX = S::RAX, RR = M * RAX, NI = S::NI;
    static_assert(G <= 4 && M <= 3, "padded rows hold at most four coefficients");
    const int T = P.tile;  // shared-memory stride = tile side (multiple of 4, <= TILE)
    extern __shared__ __align__(16) float sm[];
    const int FRm = NI * P.max_rows;
    const int DR = P.cost_mode == 1 ? 1 : G;
    const int CRW = G * PD * M;
    float* UL = sm;
    float* UR = UL + RR * T;
    float* FL = UR + RR * T;
    float* FR = FL + FRm * T;
    float* CL = FR + FRm * T;
    float* CRr = CL + CRW * T;
    float* magR = CRr + CRW * T;
    float* magF = magR + 2 * T;
    float* xs = magF + 2 * T;
    float* xab = xs + 2 * T * N_;
    float* tabs = xab + 2 * T * G;       // two padded duration tables (double buffer)
    float* Ab = tabs + 2 * PT::FLOATS;   // [RMAX][4]: A_r (M entries), then b_r
    __shared__ long long s_item;
    __shared__ float s_rown1, s_bmax;

    const int tid = threadIdx.x, nthr = blockDim.x;
    const long long nitems = (long long)P.info->items;
    const int fst = P.L.f_stride;
    unsigned long long rp_cnt = 0;

    for (;;) {
        if (tid == 0) {
            const long long it = (long long)atomicAdd(&P.info->ticket, 1u);
            s_item = has_failed(P.info) ? 0x7fffffffffffLL : it;  // one decision for the whole block
        }
        __syncthreads();
        const long long item = s_item;
        if (item >= nitems) break;
        const ItemT itc = item_decode_chunk(P, item);
        const Item& itd = itc.it;
        if (itc.t0 >= itc.t1) {  // empty chunk (nT < number of chunks)
            __syncthreads();     // everyone has read s_item before it is rewritten
            continue;
        }
        const QueryDesc& Qd = P.qd[itd.q];
        const int k = itd.k, i0 = itd.i0, j0 = itd.j0, TI = itd.TI, TJ = itd.TJ;
        const int ni4 = (TI + 3) & ~3, nj4 = (TJ + 3) & ~3;
        const int S2 = ni4 + nj4;
        const int r0 = Qd.poly_off[k], nr = Qd.poly_off[k + 1] - r0;
        const long long rg0 = Qd.rowsOff + r0;
        for (int u = tid; u < nr * 4; u += nthr) {
            const int r = u >> 2, c = u & 3;
            Ab[u] = c < M ? P.A32[(rg0 + r) * M + c] : (c == M ? P.bc32[rg0 + r] : 0.f);
        }
        const int* members = P.members + Qd.listOff + (long long)k * Qd.N;
        float cx[M];
#pragma unroll
        for (int a = 0; a < M; ++a) cx[a] = P.centers[(long long)(Qd.kOff + k) * 4 + a];
        for (int u = tid; u < S2 * N_; u += nthr) {
            const int s = u / N_, e = u % N_;
            const bool right = s >= ni4;
            const int ls = right ? s - ni4 : s;
            const int lidx = (right ? j0 : i0) + ls;
            float v = 0.f;
            if (ls < (right ? TJ : TI)) {
                const long long id = mem_id(members[lidx]);
                if (e < M) {
                    if (P.in_f32) v = ((const float*)Qd.states)[id * N_ + e] - cx[e];
                    else v = (float)(((const double*)Qd.states)[id * N_ + e] - (double)cx[e]);
                } else {
                    v = ldf(Qd.states, id * N_ + e, P.in_f32);
                }
            }
            xs[(right ? T + ls : ls) * N_ + e] = v;
        }
        stage_table<G, PD>(tabs, P.tab32 + (long long)(Qd.tabOff + itc.t0) * fst, tid, nthr);
        __syncthreads();
        for (int s = tid; s < S2; s += nthr) {
            const bool right = s >= ni4;
            const int ls = right ? s - ni4 : s;
            const float* x = xs + (right ? T + ls : ls) * N_;
            float* xa = xab + (right ? T + ls : ls) * G;
#pragma unroll
            for (int c = 0; c < G; ++c) {
                float mx = 0.f;
#pragma unroll
                for (int a = 0; a < M; ++a) mx = fmaxf(mx, fabsf(x[c * M + a]));
                xa[c] = mx;
            }
        }
        if (tid == 0) {
            float rn = 0.f, bm = 0.f;
            for (int r = 0; r < nr; ++r) {
                float s1 = 0.f;
                for (int a = 0; a < M; ++a) s1 += fabsf(Ab[r * 4 + a]);
                rn = fmaxf(rn, s1);
                bm = fmaxf(bm, fabsf(Ab[r * 4 + M]));
            }
            s_rown1 = rn * 1.0001f;
            s_bmax = bm;
        }
        __syncthreads();

        const int ngi = ni4 >> 2, ngj = nj4 >> 2;
        const bool act = tid < ngi * ngj;
        const int gi = act ? tid / ngj : 0, gj = act ? tid % ngj : 0;
        uint32_t vmask = 0, dmask = 0;  // valid pairs, diagonal pairs
#pragma unroll
        for (int qa = 0; qa < 4; ++qa)
#pragma unroll
            for (int qb = 0; qb < 4; ++qb) {
                const int li = 4 * gi + qa, lj = 4 * gj + qb;
                if (act && li < TI && lj < TJ) vmask |= 1u << (qa * 4 + qb);
                if (i0 + li == j0 + lj) dmask |= 1u << (qa * 4 + qb);  // a state paired with itself
            }
        for (int t = itc.t0; t < itc.t1; ++t) {
            const float* tab = tabs + ((t - itc.t0) & 1) * PT::FLOATS;
            // Halves.  Work units are balanced over the block: (state, axis,
            // section) with section = the RAX reach rows or the DR*PD cost
            // rows, then (state, interior control point) for the free rows.
            // Every row is one 16-byte coefficient load and G FMAs (the same
            // operation order as the reference formula h_0 x_0 + h_1 x_1 + ...).
            const int nRC = S2 * M;
            for (int u = tid; u < 2 * nRC; u += nthr) {
                const bool cost = u >= nRC;
                const int v = cost ? u - nRC : u;
                const int s = v / M, a = v - s * M;
                const bool right = s >= ni4;
                const int ls = right ? s - ni4 : s;
                const float* x = xs + (right ? T + ls : ls) * N_;
                float xc[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) xc[c] = c < G ? x[c * M + a] : 0.f;
                const float* trow = tab + (right ? 4 : 0);
                if (!cost) {
                    float* dU = (right ? UR : UL) + a * T + ls;
#pragma unroll
                    for (int r = 0; r < RAX; ++r) {
                        const float4 h = *reinterpret_cast<const float4*>(trow + r * 8);
                        float w = h.x * xc[0];
                        w = fmaf(h.y, xc[1], w);
                        if (G > 2) w = fmaf(h.z, xc[2], w);
                        if (G > 3) w = fmaf(h.w, xc[3], w);
                        dU[r * M * T] = w;
                    }
                } else {
                    float* dC = (right ? CRr : CL) + a * T + ls;
#pragma unroll
                    for (int d = 0; d < G; ++d) {
                        if (d < DR) {
#pragma unroll
                            for (int l = 0; l < PD; ++l) {
                                const float4 h = *reinterpret_cast<const float4*>(trow + (PT::ROW_C + d * PD + l) * 8);
                                float w = h.x * xc[0];
                                w = fmaf(h.y, xc[1], w);
                                if (G > 2) w = fmaf(h.z, xc[2], w);
                                if (G > 3) w = fmaf(h.w, xc[3], w);
                                dC[(l * DR + d) * M * T] = w;
                            }
                        }
                    }
                }
            }
            for (int u = tid; u < S2 * NI; u += nthr) {
                const int s = u / NI, l = u - s * NI;
                const bool right = s >= ni4;
                const int ls = right ? s - ni4 : s;
                const float* x = xs + (right ? T + ls : ls) * N_;
                const float4 dd = *reinterpret_cast<const float4*>(tab + (PT::ROW_D + l) * 8 + (right ? 4 : 0));
                float pt[M];
#pragma unroll
                for (int a = 0; a < M; ++a) {
                    float w = dd.x * x[a];
                    w = fmaf(dd.y, x[M + a], w);
                    if (G > 2) w = fmaf(dd.z, x[2 * M + a], w);
                    if (G > 3) w = fmaf(dd.w, x[3 * M + a], w);
                    pt[a] = w;
                }
                float* dF = (right ? FR : FL) + l * nr * T + ls;
#pragma unroll 4
                for (int r = 0; r < nr; ++r) {
                    const float4 ab = *reinterpret_cast<const float4*>(Ab + r * 4);
                    float w = ab.x * pt[0];
                    w = fmaf(ab.y, pt[1], w);
                    if (M > 2) w = fmaf(ab.z, pt[2], w);
                    if (!right) w -= (M > 2 ? ab.w : ab.z);
                    dF[r * T] = w;
                }
            }
            // band magnitudes
            for (int s = tid; s < S2; s += nthr) {
                const bool right = s >= ni4;
                const int ls = right ? s - ni4 : s;
                const float* xa = xab + (right ? T + ls : ls) * G;
                const float* hc = tab + PT::ROW_HC * 8 + (right ? 4 : 0);
                const float* dc = tab + PT::ROW_DC * 8 + (right ? 4 : 0);
                float mr = 0.f, md = 0.f;
#pragma unroll
                for (int c = 0; c < G; ++c) {
                    mr = fmaf(hc[c], xa[c], mr);
                    md = fmaf(dc[c], xa[c], md);
                }
                magR[(right ? T : 0) + ls] = mr;
                magF[(right ? T : 0) + ls] = md * s_rown1 + (right ? 0.f : s_bmax);
            }
            __syncthreads();

            // the next duration's table goes to the other buffer while the pairs run
            if (t + 1 < itc.t1)
                stage_table<G, PD>(tabs + ((t + 1 - itc.t0) & 1) * PT::FLOATS,
                                   P.tab32 + (long long)(Qd.tabOff + t + 1) * fst, tid, nthr);
            if (act) {
                pair_phase<M, G, PD>(P, itd, t, T, gi, gj, vmask, dmask, nr, DR, UL, UR, FL, FR, CL, CRr, magR, magF, KR, KF,
                                     rp_cnt);
            }
            __syncthreads();
        }
    }
    block_add(&P.info->reach_pass, rp_cnt);
}

// ---------------------------------------------------------------------------
// Screened FP32 pair kernel (the default one).  Same persistent item loop as
// the one-group kernel, in four phases per duration:
//   1. reach halves, stored per state ([state][row], rows padded to 16-byte
//      quads, per-state stride = 4 mod 8 floats so that quad loads of
//      different states fall in different bank groups); the screen row-axes
//      also in FP16, stored [row][state] for the micro-tile screen; the
//      interior control points' halves; the cost rows' magnitudes;
//   2. screen of every 4x4 micro-tile; pairs that do not certainly fail are
//      appended to list 1 (shared memory);
//   3. every reach row of the list-1 pairs (four per 16-byte load) and, for
//      those that pass, every polytope row at every interior control point,
//      one pair per thread; feasible pairs go to list 2, ambiguous ones to
//      the FP64 re-check;
//   4. costs of the list-2 pairs from their two staged states and the atomic
//      merge into the pair slots.
// Maxima are order-free and the reach sums and costs keep the reference
// order, so slots and costs equal those of the other FP32 kernels; the free
// margins take fewer roundings within the same band, so only the set of
// ambiguous margins re-checked in FP64 can differ.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int pad_odd4(int n) { return ((n + 3) / 8) * 8 + 4; }  // >= n, = 4 mod 8

// per-state stride of the interior control points' halves
__host__ __device__ inline int sc_free_stride(int NI, int M) {
    return pad_odd4((NI * M + 3) & ~3);  // the interior control points' halves
}

template <int M, int G, int PD>
struct ScShape {
    using S = Shape<G, PD>;
    static constexpr int RR = M * S::RAX;        // reach row-axes
    static constexpr int RQ = (RR + 3) / 4;      // their 16-byte quads
    static constexpr int RH = (RQ + 1) / 2;      // quads of the first half-unit
    static constexpr int SU = pad_odd4(4 * RQ);  // per-state stride of the reach halves
    static constexpr int NS = Screen<G, PD>::NS * M;
    static constexpr int XS = pad_odd4(M * G);   // per-state stride of the staged states
};

// Reach halves of one state for quads [Q0, Q1): row-axis q = rr*M + a holds
// sum_c H[rr][side][c] x[c][a]; rows past RR are 0 (neutral in max |u + w|).
// The screen row-axes also go, rounded to FP16, to the screen arrays dS.
template <int M, int G, int PD, int Q0, int Q1>
DEVI void reach_quads(const float (&x)[M * G], const float* trow, float* dU, void* dS, int ls, bool right, int T) {
    constexpr int RR = ScShape<M, G, PD>::RR;
#pragma unroll
    for (int qd = Q0; qd < Q1; ++qd) {
        float w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = 4 * qd + j;
            w[j] = 0.f;
            if (q < RR) {
                const int rr = q / M, a = q % M;
                const float4 h = *reinterpret_cast<const float4*>(trow + rr * 8);
                float v = h.x * x[a];
                if (G > 1) v = fmaf(h.y, x[M + a], v);
                if (G > 2) v = fmaf(h.z, x[2 * M + a], v);
                if (G > 3) v = fmaf(h.w, x[3 * M + a], v);
                w[j] = v;
                const int si = Screen<G, PD>::index(rr);
                if (si >= 0) {  // screen row-axis in FP16: (h, h) for start states, h for end states
                    const __half hv = __float2half_rn(v);
                    if (right) reinterpret_cast<__half*>(dS)[(si * M + a) * T + ls] = hv;
                    else reinterpret_cast<__half2*>(dS)[(si * M + a) * T + ls] = __halves2half2(hv, hv);
                }
            }
        }
        *reinterpret_cast<float4*>(dU + 4 * qd) = make_float4(w[0], w[1], w[2], w[3]);
    }
}

template <int M, int G, int PD>
DEVI void load_state(float (&x)[M * G], const float* xr) {
    constexpr int XS = ScShape<M, G, PD>::XS;
    float v[XS];
#pragma unroll
    for (int e = 0; e < XS; e += 4) {
        const float4 f = *reinterpret_cast<const float4*>(xr + e);
        v[e] = f.x;
        v[e + 1] = f.y;
        v[e + 2] = f.z;
        v[e + 3] = f.w;
    }
#pragma unroll
    for (int e = 0; e < M * G; ++e) x[e] = v[e];
}

// Interior control-point halves of one state for points [L0, L1): point l's
// coordinate a, sum_c D[l][side][c] x[c][a], at dP[l * M + a]; the unit that
// ends at NI also zeroes the padding up to the next 16-byte quad.
template <int M, int G, int PD, int L0, int L1>
DEVI void point_halves(const float (&x)[M * G], const float* tab, bool right, float* dP) {
    constexpr int NI = Shape<G, PD>::NI, NP = (NI * M + 3) & ~3;
#pragma unroll
    for (int l = L0; l < L1; ++l) {
        const float4 dd = *reinterpret_cast<const float4*>(tab + (PadTab<G, PD>::ROW_D + l) * 8 + (right ? 4 : 0));
#pragma unroll
        for (int a = 0; a < M; ++a) {
            float w = dd.x * x[a];
            if (G > 1) w = fmaf(dd.y, x[M + a], w);
            if (G > 2) w = fmaf(dd.z, x[2 * M + a], w);
            if (G > 3) w = fmaf(dd.w, x[3 * M + a], w);
            dP[l * M + a] = w;
        }
    }
    if (L1 == NI) {
#pragma unroll
        for (int e = NI * M; e < NP; ++e) dP[e] = 0.f;
    }
}

// Sum of |cost half| of one state over the floats [F0, F1) of its packed
// cost rows (row e = d*M + a, d < DR, of segment l at float l * DR * M + e:
// sum_c C[d][l][side][c] x[c][a]), in float order; nothing is stored.
template <int M, int G, int PD, int DR, int F0, int F1>
DEVI float cost_mag(const float (&x)[M * G], const float* tab, bool right) {
    constexpr int DRM = DR * M, NF = PD * DRM;
    static_assert(F1 > F0, "each unit takes some of the cost rows");
    float mag = 0.f;
#pragma unroll
    for (int f = F0; f < F1; ++f) {
        if (f < NF) {
            const int l = f / DRM, e = f % DRM, d = e / M, a = e % M;
            const float4 h =
                *reinterpret_cast<const float4*>(tab + (PadTab<G, PD>::ROW_C + d * PD + l) * 8 + (right ? 4 : 0));
            float w = h.x * x[a];
            if (G > 1) w = fmaf(h.y, x[M + a], w);
            if (G > 2) w = fmaf(h.z, x[2 * M + a], w);
            if (G > 3) w = fmaf(h.w, x[3 * M + a], w);
            mag += fabsf(w);
        }
    }
    return mag;
}

// The split of a state's cost rows (counted as packed floats) between its
// two units for the magnitude sums: at the segment boundary (PD + 1) / 2
// rounded down to a quad, the rest to the end of the padding.
template <int M, int PD, int DR>
struct CostSplit {
    static constexpr int NP = (PD * DR * M + 3) & ~3;
    static constexpr int FS0 = (((PD + 1) / 2) * DR * M) & ~3;
    static constexpr int FS = FS0 > 0 ? FS0 : (NP > 4 ? 4 : NP);
};

// The next item for a block, or past the end once the build has failed.
DEVI long long take_item(DevInfo* info) {
    const long long it = (long long)atomicAdd(&info->ticket, 1u);
    return has_failed(info) ? 0x7fffffffffffLL : it;
}

// Half H of one staged state: elements [H*EH, (H+1)*EH) of the XS-float row
// (positions centred on the polytope, FP32; zero for padding states and
// padding elements), and the maxima over the axes of the derivatives whose
// M elements lie in this half.
template <int M, int G, int XS, int H>
DEVI void stage_state_half(const void* states, bool in_f32, long long id, bool valid, const float (&cx)[M],
                           float* xrow, float* xa) {
    constexpr int N_ = M * G, EH = XS / 2;
    static_assert(XS % 2 == 0 && EH % M == 0, "a derivative's axes lie in one half of the staged state");
    float v[EH];
#pragma unroll
    for (int q = 0; q < EH; ++q) {
        const int e = H * EH + q;
        float x = 0.f;
        if (valid && e < N_) {
            if (e < M) {
                if (in_f32) x = ((const float*)states)[id * N_ + e] - cx[e < M ? e : 0];
                else x = (float)(((const double*)states)[id * N_ + e] - (double)cx[e < M ? e : 0]);
            } else {
                x = ldf(states, id * N_ + e, in_f32);
            }
        }
        v[q] = x;
    }
#pragma unroll
    for (int q = 0; q < EH; ++q) xrow[H * EH + q] = v[q];
#pragma unroll
    for (int c = 0; c < G; ++c) {
        if (c * M >= H * EH && c * M < (H + 1) * EH) {
            float mx = 0.f;
#pragma unroll
            for (int a = 0; a < M; ++a) {
                const int q = c * M + a - H * EH;  // in [0, EH) inside this branch
                mx = fmaxf(mx, fabsf(v[q >= 0 && q < EH ? q : 0]));
            }
            xa[c] = mx;
        }
    }
}

// Control-polygon length of one pair from its two staged states: per
// segment l the root of the sum of squares, over rows e = d*M + a (d < DR) in
// order, of start half + end half (each sum_c C[d][l][side][c] x[c][a], the
// table rows broadcast), summed over the PD segments in order.
template <int M, int G, int PD, int DR>
DEVI float pair_cost_states(const float* xi, const float* xj, const float* tab) {
    float a[M * G], b[M * G];
    load_state<M, G, PD>(a, xi);
    load_state<M, G, PD>(b, xj);
    float cs = 0.f;
#pragma unroll
    for (int l = 0; l < PD; ++l) {
        float ss = 0.f;
#pragma unroll
        for (int d = 0; d < DR; ++d) {
            const float4 hl = *reinterpret_cast<const float4*>(tab + (PadTab<G, PD>::ROW_C + d * PD + l) * 8);
            const float4 hr = *reinterpret_cast<const float4*>(tab + (PadTab<G, PD>::ROW_C + d * PD + l) * 8 + 4);
#pragma unroll
            for (int q = 0; q < M; ++q) {
                float cl = hl.x * a[q];
                if (G > 1) cl = fmaf(hl.y, a[M + q], cl);
                if (G > 2) cl = fmaf(hl.z, a[2 * M + q], cl);
                if (G > 3) cl = fmaf(hl.w, a[3 * M + q], cl);
                float cr = hr.x * b[q];
                if (G > 1) cr = fmaf(hr.y, b[M + q], cr);
                if (G > 2) cr = fmaf(hr.z, b[2 * M + q], cr);
                if (G > 3) cr = fmaf(hr.w, b[3 * M + q], cr);
                const float dv = cl + cr;
                ss = fmaf(dv, dv, ss);
            }
        }
        cs += sqrtf(ss);
    }
    return cs;
}

template <int M, int G, int PD>
__global__ void __launch_bounds__(256, 3) k_pairs_sc(BuildParams P) {
    using S = Shape<G, PD>;
    using PT = PadTab<G, PD>;
    using SS = ScShape<M, G, PD>;
    constexpr int N_ = M * G, NI = S::NI, RQ = SS::RQ, RH = SS::RH, SU = SS::SU, NS = SS::NS, XS = SS::XS;
    static_assert(G <= 4 && M <= 3, "padded rows hold at most four coefficients");
    const int T = P.tile;  // tile side (multiple of 4, <= TILE)
    extern __shared__ __align__(16) float sm[];
    const int DR = P.cost_mode == 1 ? 1 : G;
    const int SF = sc_free_stride(NI, M);
    float* UL = sm;                  // [T][SU] reach halves, start states
    float* UR = UL + T * SU;         //          end states
    float* FL = UR + T * SU;         // [T][SF] interior control-point halves
    float* FR = FL + T * SF;
    __half2* SCL = reinterpret_cast<__half2*>(FR + T * SF);       // [NS][T] screen row-axes, start states: (h, h)
    __half* SCR = reinterpret_cast<__half*>(FR + T * SF + NS * T);  // [NS][T] end states (half of the space used)
    float* magR = FR + T * SF + 2 * NS * T;                          // [2T] band magnitudes
    float* magF = magR + 2 * T;
    float* magC = magF + 2 * T;      // [2T] sum of |cost half| per state-side (cost conditioning):
    float* magC2 = magC + 2 * T;     //      first unit's rows, second unit's rows
    float* xs = magC2 + 2 * T;       // [2T][XS] centred states
    float* xab = xs + 2 * T * XS;    // [2T][G] per-derivative maxima over the axes
    float* tabs = xab + 2 * T * G;   // two padded duration tables
    float* Ab = tabs + 2 * PT::FLOATS;  // [RMAX][4]: A_r, then b_r
    uint16_t* list1 = reinterpret_cast<uint16_t*>(Ab + RMAX * 4);  // screened pairs (li << 8 | lj)
    uint16_t* list2 = list1 + T * T;                                 // feasible pairs
    __shared__ long long s_item;
    __shared__ float s_rown1, s_bmax;
    __shared__ int s_n1[2], s_n2[2];  // list lengths, by duration parity

    const int tid = threadIdx.x, nthr = blockDim.x;
    const long long nitems = (long long)P.info->items;
    const int fst = P.L.f_stride;
    unsigned long long rp_cnt = 0, nscreened = 0;
    const float NEG_INF = -__int_as_float(0x7f800000);

    for (;;) {
        if (tid == 0) s_item = take_item(P.info);
        __syncthreads();
        const long long item = s_item;
        if (item >= nitems) break;
        const ItemT itc = item_decode_chunk(P, item);
        const Item& itd = itc.it;
        if (itc.t0 >= itc.t1) {  // empty chunk (nT < number of chunks)
            __syncthreads();     // everyone has read s_item before it is rewritten
            continue;
        }
        const QueryDesc& Qd = P.qd[itd.q];
        const int k = itd.k, i0 = itd.i0, j0 = itd.j0, TI = itd.TI, TJ = itd.TJ;
        const int ni4 = (TI + 3) & ~3, nj4 = (TJ + 3) & ~3;
        const int S2 = ni4 + nj4;
        const int r0 = Qd.poly_off[k], nr = Qd.poly_off[k + 1] - r0;
        const long long rg0 = Qd.rowsOff + r0;
        for (int u = tid; u < nr * 4; u += nthr) {
            const int r = u >> 2, c = u & 3;
            Ab[u] = c < M ? P.A32[(rg0 + r) * M + c] : (c == M ? P.bc32[rg0 + r] : 0.f);
        }
        const int* members = P.members + Qd.listOff + (long long)k * Qd.N;
        float cx[M];
#pragma unroll
        for (int a = 0; a < M; ++a) cx[a] = P.centers[(long long)(Qd.kOff + k) * 4 + a];
        // two threads per state (the second S2 threads take the second
        // halves), each loading the member id once and half of the state's
        // elements, all of its loads in flight together; each also writes the
        // per-derivative maxima over the axes of its half
        for (int u = tid; u < 2 * S2; u += nthr) {
            const bool hi = u >= S2;  // warp-uniform halves for whole tiles
            const int s = hi ? u - S2 : u;
            const bool right = s >= ni4;
            const int ls = right ? s - ni4 : s;
            const bool valid = ls < (right ? TJ : TI);
            const long long id = valid ? mem_id(members[(right ? j0 : i0) + ls]) : 0;
            const int row = right ? T + ls : ls;
            if (hi) stage_state_half<M, G, XS, 1>(Qd.states, P.in_f32, id, valid, cx, xs + row * XS, xab + row * G);
            else stage_state_half<M, G, XS, 0>(Qd.states, P.in_f32, id, valid, cx, xs + row * XS, xab + row * G);
        }
        if (tid < 32) {  // band scalars of the polytope's rows (warp 0, rows from global memory)
            float rn = 0.f, bm = 0.f;
            for (int r = tid; r < nr; r += 32) {
                float s1 = 0.f;
#pragma unroll
                for (int a = 0; a < M; ++a) s1 += fabsf(P.A32[(rg0 + r) * M + a]);
                rn = fmaxf(rn, s1);
                bm = fmaxf(bm, fabsf(P.bc32[rg0 + r]));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                rn = fmaxf(rn, __shfl_xor_sync(0xffffffffu, rn, o));
                bm = fmaxf(bm, __shfl_xor_sync(0xffffffffu, bm, o));
            }
            if (tid == 0) {
                s_rown1 = rn * 1.0001f;
                s_bmax = bm;
            }
        }
        stage_table_async<G, PD>(tabs, P.tab32 + (long long)(Qd.tabOff + itc.t0) * fst, tid, nthr);
        if (tid == 0) {
            s_n1[0] = s_n1[1] = 0;
            s_n2[0] = s_n2[1] = 0;
        }
        cp_async_wait_all();
        __syncthreads();

        const int ngi = ni4 >> 2, ngj = nj4 >> 2;
        const bool act = tid < ngi * ngj;
        const int gi = act ? tid / ngj : 0, gj = act ? tid % ngj : 0;
        uint32_t live = 0;  // valid, off-diagonal pairs of this thread's micro-tile
#pragma unroll
        for (int qa = 0; qa < 4; ++qa)
#pragma unroll
            for (int qb = 0; qb < 4; ++qb) {
                const int li = 4 * gi + qa, lj = 4 * gj + qb;
                if (act && li < TI && lj < TJ && i0 + li != j0 + lj) live |= 1u << (qa * 4 + qb);
            }
        for (int t = itc.t0; t < itc.t1; ++t) {
            // Three block barriers per duration.  The costs of duration t
            // (phase 4) read only the staged states, table t, the cost
            // magnitudes and list 2, which duration t+1 rewrites only after
            // its first barrier (magnitudes in phase 2, the table buffer by the
            // prefetch for t+2, list 2 in phase 3) -- so duration t+1's halves
            // overlap the slowest warps' costs of duration t.
            const int par = (t - itc.t0) & 1;
            const float* tab = tabs + par * PT::FLOATS;
            // 1. halves: two units per state, each loading the state once --
            // the first takes reach quads [0, RH), interior points [0, NI/2)
            // and the band magnitudes, the second the rest
            for (int u = tid; u < 2 * S2; u += nthr) {
                const bool second = u >= S2;
                const int s = second ? u - S2 : u;
                const bool right = s >= ni4;
                const int ls = right ? s - ni4 : s;
                float x[N_];
                load_state<M, G, PD>(x, xs + (right ? T + ls : ls) * XS);
                const float* trow = tab + (right ? 4 : 0);
                float* dU = (right ? UR : UL) + ls * SU;
                void* dS = right ? (void*)SCR : (void*)SCL;
                float* dF = (right ? FR : FL) + ls * SF;
                if (!second) {
                    reach_quads<M, G, PD, 0, RH>(x, trow, dU, dS, ls, right, T);
                    point_halves<M, G, PD, 0, NI / 2>(x, tab, right, dF);
                    const float* xa = xab + (right ? T + ls : ls) * G;
                    const float* hc = tab + PT::ROW_HC * 8 + (right ? 4 : 0);
                    const float* dc = tab + PT::ROW_DC * 8 + (right ? 4 : 0);
                    float mr = 0.f, md = 0.f;
#pragma unroll
                    for (int c = 0; c < G; ++c) {
                        mr = fmaf(hc[c], xa[c], mr);
                        md = fmaf(dc[c], xa[c], md);
                    }
                    magR[(right ? T : 0) + ls] = mr;
                    magF[(right ? T : 0) + ls] = md * s_rown1 + (right ? 0.f : s_bmax);
                } else {
                    reach_quads<M, G, PD, RH, RQ>(x, trow, dU, dS, ls, right, T);
                    point_halves<M, G, PD, NI / 2, NI>(x, tab, right, dF);
                }
            }
            __syncthreads();

            // the next duration's table goes to the other buffer meanwhile (its
            // last reader, the costs of duration t-1, finished before the barrier
            // above); the list lengths of duration t+1 are cleared
            if (t + 1 < itc.t1)
                stage_table_async<G, PD>(tabs + ((t + 1 - itc.t0) & 1) * PT::FLOATS,
                                         P.tab32 + (long long)(Qd.tabOff + t + 1) * fst, tid, nthr);
            if (tid == 0) {
                s_n1[par ^ 1] = 0;
                s_n2[par ^ 1] = 0;
            }
            // the cost rows' magnitudes of this duration (cost conditioning), one
            // part per unit
            for (int u = tid; u < 2 * S2; u += nthr) {
                const bool second = u >= S2;
                const int s = second ? u - S2 : u;
                const bool right = s >= ni4;
                const int ls = right ? s - ni4 : s;
                float x[N_];
                load_state<M, G, PD>(x, xs + (right ? T + ls : ls) * XS);
                using CSG = CostSplit<M, PD, G>;
                using CS1 = CostSplit<M, PD, 1>;
                const float mg = DR == G ? (!second ? cost_mag<M, G, PD, G, 0, CSG::FS>(x, tab, right)
                                                    : cost_mag<M, G, PD, G, CSG::FS, CSG::NP>(x, tab, right))
                                         : (!second ? cost_mag<M, G, PD, 1, 0, CS1::FS>(x, tab, right)
                                                    : cost_mag<M, G, PD, 1, CS1::FS, CS1::NP>(x, tab, right));
                (second ? magC2 : magC)[(right ? T : 0) + ls] = mg;
            }

            // 2. screen and list 1 (positions by a warp prefix of the survivor
            // counts and one shared atomic per warp; the block is whole warps)
            {
                uint32_t surv = act ? screen_tile<M, G, PD>(T, gi, gj, live, SCL, SCR, magR) : 0u;
                const int cnt = __popc(surv);
                int inc = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, inc, o);
                    if ((tid & 31) >= o) inc += y;
                }
                int wbase = 0;
                if ((tid & 31) == 31 && inc) wbase = atomicAdd(&s_n1[par], inc);
                int pos = __shfl_sync(0xffffffffu, wbase, 31) + inc - cnt;
                while (surv) {
                    const int q = __ffs(surv) - 1;
                    surv &= surv - 1;
                    list1[pos++] = (uint16_t)(((4 * gi + (q >> 2)) << 8) | (4 * gj + (q & 3)));
                }
            }
            __syncthreads();

            // 3. every reach and free row of the screened pairs
            const int n1 = s_n1[par];
            if (tid == 0) nscreened += (unsigned long long)n1;
            for (int e = tid; e < n1; e += nthr) {
                const int v = list1[e];
                const int li = v >> 8, lj = v & 255;
                const float* ul = UL + li * SU;
                const float* ur = UR + lj * SU;
                float r4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int qd = 0; qd < RQ; ++qd) {
                    const float4 a = *reinterpret_cast<const float4*>(ul + 4 * qd);
                    const float4 b = *reinterpret_cast<const float4*>(ur + 4 * qd);
                    r4[0] = fmaxf(r4[0], fabsf(a.x + b.x));
                    r4[1] = fmaxf(r4[1], fabsf(a.y + b.y));
                    r4[2] = fmaxf(r4[2], fabsf(a.z + b.z));
                    r4[3] = fmaxf(r4[3], fabsf(a.w + b.w));
                }
                const float rm = fmaxf(fmaxf(r4[0], r4[1]), fmaxf(r4[2], r4[3]));
                const float bandR = KR * (magR[li] + magR[T + lj]);
                int outcome = 0;  // 0 certain failure, 1 certainly feasible, 2 ambiguous
                if (rm <= 1.f + bandR) {
                    const bool rpass = rm <= 1.f - bandR;
                    rp_cnt += rpass ? 1u : 0u;
                    // interior control points P_l = start half + end half, then
                    // every polytope row A_r . P_l - b_r (rows broadcast from Ab)
                    constexpr int NPQ = (NI * M + 3) / 4;
                    const float* pl_ = FL + li * SF;
                    const float* pr_ = FR + lj * SF;
                    float pt[4 * NPQ];
#pragma unroll
                    for (int q = 0; q < NPQ; ++q) {
                        const float4 a = *reinterpret_cast<const float4*>(pl_ + 4 * q);
                        const float4 c = *reinterpret_cast<const float4*>(pr_ + 4 * q);
                        pt[4 * q] = a.x + c.x;
                        pt[4 * q + 1] = a.y + c.y;
                        pt[4 * q + 2] = a.z + c.z;
                        pt[4 * q + 3] = a.w + c.w;
                    }
                    float f2[2] = {NEG_INF, NEG_INF};
                    for (int r = 0; r < nr; ++r) {
                        const float4 ab = *reinterpret_cast<const float4*>(Ab + r * 4);
                        const float br = M > 2 ? ab.w : ab.z;
#pragma unroll
                        for (int l = 0; l < NI; ++l) {
                            float w = ab.x * pt[l * M];
                            w = fmaf(ab.y, pt[l * M + 1], w);
                            if (M > 2) w = fmaf(ab.z, pt[l * M + 2], w);
                            f2[l & 1] = fmaxf(f2[l & 1], w - br);
                        }
                    }
                    const float fm = fmaxf(f2[0], f2[1]);
                    const float bandF = KF * (magF[li] + magF[T + lj]);
                    if (fm <= bandF) outcome = (rpass && fm <= -bandF) ? 1 : 2;
                }
                // list 2 positions: one shared atomic per warp
                const unsigned am = __activemask();
                const unsigned fb = __ballot_sync(am, outcome == 1);
                if (fb) {
                    const int lane = tid & 31, leader = __ffs(fb) - 1;
                    int b2 = 0;
                    if (lane == leader) b2 = atomicAdd(&s_n2[par], __popc(fb));
                    b2 = __shfl_sync(am, b2, leader);
                    if (outcome == 1) list2[b2 + __popc(fb & ((1u << lane) - 1u))] = (uint16_t)v;
                }
                if (outcome == 2) append_recheck(P, itd.q, k, i0 + li, j0 + lj, t);
            }
            cp_async_wait_all();  // the next duration's table, visible after this barrier
            __syncthreads();

            const int n2 = s_n2[par];
            // 4. costs of the feasible pairs from their two staged states (per
            // segment the sum of squares in row order)
            for (int e = tid; e < n2; e += nthr) {
                const int v = list2[e];
                const int li = v >> 8, lj = v & 255;
                const float* xi = xs + li * XS;
                const float* xj = xs + (T + lj) * XS;
                const float cs = DR == G ? pair_cost_states<M, G, PD, G>(xi, xj, tab)
                                         : pair_cost_states<M, G, PD, 1>(xi, xj, tab);
                const float mc = (magC[li] + magC2[li]) + (magC[T + lj] + magC2[T + lj]);
                if (P.cost64 || mc <= COST_RHO * cs) {  // FP64 models re-cost every edge anyway
                    const long long slot = itd.base + (long long)(i0 + li) * itd.nk + (j0 + lj);
                    atomicOr(&P.resBits[slot], 1u << t);
                    atomicMin(&P.resKey[slot], key_f32(cs, t));
                } else {
                    append_recheck(P, itd.q, k, i0 + li, j0 + lj, t, true);  // ill-conditioned FP32 cost
                }
            }
        }
    }
    block_add(&P.info->reach_pass, rp_cnt);
    block_add(&P.info->screened, nscreened);
}

// ---------------------------------------------------------------------------
// Warp-specialised FP32 pair kernel.  Eight producer warps stage an item's
// states and compute the halves of one duration into one of two shared-memory
// stages; eight consumer warps (one 4x4 micro-tile per thread, 64x64 tiles)
// reduce the pairs of the other stage.  Stages change hands through mbarriers
// (producers: "stage s holds duration t", consumers: "stage s is free"), so the
// groups never meet at a CTA-wide barrier and consumers that finish a duration
// early move on instead of waiting for the slowest warp.  Every wait is
// bounded; on expiry the kernel records PLAN_ERR_TIMEOUT and stops.
// ---------------------------------------------------------------------------
struct StageMeta {
    int end;
    int q, k, i0, j0, TI, TJ, nk, nr, t;
    long long base;
};

namespace ws {
DEVI uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
DEVI void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
DEVI void mbar_arrive(uint64_t* bar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n}\n" ::"r"(saddr(bar)) : "memory");
}
DEVI bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait; false (and PLAN_ERR_TIMEOUT recorded) if the phase never completes
DEVI bool mbar_wait(uint64_t* bar, uint32_t parity, DevInfo* info) {
    long long spins = 0;
    while (!mbar_try(bar, parity)) {
        if (++spins > (1LL << 22)) {
            set_status(info, PLAN_ERR_TIMEOUT, DET_BARRIER);
            return false;
        }
    }
    return true;
}
DEVI void bar_producers() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
}  // namespace ws

template <int M, int G, int PD>
__global__ void __launch_bounds__(512, 1) k_pairs_ws(BuildParams P) {
    using S = Shape<G, PD>;
    constexpr int N_ = M * G, RAX = S::RAX, RR = M * RAX, NI = S::NI, TG = S::TG;
    constexpr int T = TILE;
    constexpr int NCW = 8;  // consumer warps (warps 8..15); warps 0..7 produce
    extern __shared__ __align__(16) float sm[];
    const int FRm = NI * P.max_rows;
    const int DR = P.cost_mode == 1 ? 1 : G;
    const int CRW = G * PD * M;
    const int stage_floats = (2 * RR + 2 * FRm + 2 * CRW + 4) * T;
    float* xs = sm + 2 * stage_floats;
    float* xab = xs + 2 * T * N_;
    float* tabs = xab + 2 * T * G;
    float* Ap = tabs + 2 * P.L.f_stride;
    float* bp = Ap + RMAX * M;
    __shared__ StageMeta meta[2];
    __shared__ __align__(8) uint64_t full[2];
    __shared__ __align__(8) uint64_t empty[2];
    __shared__ long long s_item;
    __shared__ float s_rown1, s_bmax;
    __shared__ int s_stop;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long nitems = (long long)P.info->items;
    const TabLayout L = P.L;
    if (tid == 0) {
        ws::mbar_init(&full[0], 1);
        ws::mbar_init(&full[1], 1);
        ws::mbar_init(&empty[0], NCW);
        ws::mbar_init(&empty[1], NCW);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_stop = 0;
    }
    __syncthreads();

    auto stage_ptr = [&](int st, float*& UL, float*& UR, float*& FL, float*& FR, float*& CL, float*& CRr,
                         float*& magR, float*& magF) {
        float* b = sm + st * stage_floats;
        UL = b;
        UR = UL + RR * T;
        FL = UR + RR * T;
        FR = FL + FRm * T;
        CL = FR + FRm * T;
        CRr = CL + CRW * T;
        magR = CRr + CRW * T;
        magF = magR + 2 * T;
    };

    if (warp < 8) {
        // ------------------------------ producers ------------------------------
        const int ptid = tid, pn = 256;
        int stage = 0;
        uint32_t uses[2] = {0u, 0u};
        bool ok = true;
        for (;;) {
            if (ptid == 0) {
                const long long it = (long long)atomicAdd(&P.info->ticket, 1u);
                s_item = (has_failed(P.info) || *(volatile int*)&s_stop) ? 0x7fffffffffffLL : it;
            }
            ws::bar_producers();
            const long long item = s_item;
            if (item >= nitems) break;
            const ItemT itc = item_decode_chunk(P, item);
            const Item& itd = itc.it;
            if (itc.t0 >= itc.t1) {
                ws::bar_producers();
                continue;
            }
            const QueryDesc& Qd = P.qd[itd.q];
            const int k = itd.k, i0 = itd.i0, j0 = itd.j0, TI = itd.TI, TJ = itd.TJ;
            const int ni4 = (TI + 3) & ~3, nj4 = (TJ + 3) & ~3;
            const int r0 = Qd.poly_off[k], nr = Qd.poly_off[k + 1] - r0;
            const long long rg0 = Qd.rowsOff + r0;
            for (int u = ptid; u < nr * M; u += pn) Ap[u] = P.A32[rg0 * M + u];
            for (int u = ptid; u < nr; u += pn) bp[u] = P.bc32[rg0 + u];
            const int* members = P.members + Qd.listOff + (long long)k * Qd.N;
            float cx[M];
#pragma unroll
            for (int a = 0; a < M; ++a) cx[a] = P.centers[(long long)(Qd.kOff + k) * 4 + a];
            for (int u = ptid; u < (ni4 + nj4) * N_; u += pn) {
                const int s = u / N_, e = u % N_;
                const bool right = s >= ni4;
                const int ls = right ? s - ni4 : s;
                const int lidx = (right ? j0 : i0) + ls;
                float v = 0.f;
                if (ls < (right ? TJ : TI)) {
                    const long long id = mem_id(members[lidx]);
                    if (e < M) {
                        if (P.in_f32) v = ((const float*)Qd.states)[id * N_ + e] - cx[e];
                        else v = (float)(((const double*)Qd.states)[id * N_ + e] - (double)cx[e]);
                    } else {
                        v = ldf(Qd.states, id * N_ + e, P.in_f32);
                    }
                }
                xs[(right ? T + ls : ls) * N_ + e] = v;
            }
            for (int u = ptid; u < L.f_stride; u += pn) tabs[u] = P.tab32[(long long)(Qd.tabOff + itc.t0) * L.f_stride + u];
            ws::bar_producers();
            for (int s = ptid; s < ni4 + nj4; s += pn) {
                const bool right = s >= ni4;
                const int ls = right ? s - ni4 : s;
                const float* x = xs + (right ? T + ls : ls) * N_;
                float* xa = xab + (right ? T + ls : ls) * G;
#pragma unroll
                for (int c = 0; c < G; ++c) {
                    float mx = 0.f;
#pragma unroll
                    for (int a = 0; a < M; ++a) mx = fmaxf(mx, fabsf(x[c * M + a]));
                    xa[c] = mx;
                }
            }
            if (ptid == 0) {
                float rn = 0.f, bm = 0.f;
                for (int r = 0; r < nr; ++r) {
                    float s1 = 0.f;
                    for (int a = 0; a < M; ++a) s1 += fabsf(Ap[r * M + a]);
                    rn = fmaxf(rn, s1);
                    bm = fmaxf(bm, fabsf(bp[r]));
                }
                s_rown1 = rn * 1.0001f;
                s_bmax = bm;
            }
            ws::bar_producers();
            for (int t = itc.t0; t < itc.t1 && ok; ++t) {
                const float* tab = tabs + ((t - itc.t0) & 1) * L.f_stride;
                if (uses[stage] > 0 && !ws::mbar_wait(&empty[stage], (uses[stage] - 1) & 1u, P.info)) {
                    ok = false;
                    break;
                }
                float *UL, *UR, *FL, *FR, *CL, *CRr, *magR, *magF;
                stage_ptr(stage, UL, UR, FL, FR, CL, CRr, magR, magF);
                for (int u = ptid; u < (ni4 + nj4) * M; u += pn) {
                    const int s = u / M, a = u % M;
                    const bool right = s >= ni4;
                    const int ls = right ? s - ni4 : s;
                    const float* x = xs + (right ? T + ls : ls) * N_;
                    float xc[G];
#pragma unroll
                    for (int c = 0; c < G; ++c) xc[c] = x[c * M + a];
                    const int co = right ? G : 0;
                    float* dU = right ? UR : UL;
#pragma unroll 3
                    for (int r = 0; r < RAX; ++r) {
                        const float* h = tab + L.f_H + r * TG + co;
                        float v = h[0] * xc[0];
#pragma unroll
                        for (int c = 1; c < G; ++c) v = fmaf(h[c], xc[c], v);
                        dU[(r * M + a) * T + ls] = v;
                    }
                    float* dC = right ? CRr : CL;
                    for (int d = 0; d < DR; ++d)
                        for (int l = 0; l < PD; ++l) {
                            const float* cc = tab + L.f_C + (d * PD + l) * TG + co;
                            float v = cc[0] * xc[0];
#pragma unroll
                            for (int c = 1; c < G; ++c) v = fmaf(cc[c], xc[c], v);
                            dC[((l * DR + d) * M + a) * T + ls] = v;
                        }
                }
                for (int u = ptid; u < (ni4 + nj4) * NI; u += pn) {
                    const int s = u / NI, l = u % NI;
                    const bool right = s >= ni4;
                    const int ls = right ? s - ni4 : s;
                    const float* x = xs + (right ? T + ls : ls) * N_;
                    const float* dd = tab + L.f_D + l * TG + (right ? G : 0);
                    float pt[M];
#pragma unroll
                    for (int a = 0; a < M; ++a) {
                        float v = dd[0] * x[a];
#pragma unroll
                        for (int c = 1; c < G; ++c) v = fmaf(dd[c], x[c * M + a], v);
                        pt[a] = v;
                    }
                    float* dF = right ? FR : FL;
                    for (int r = 0; r < nr; ++r) {
                        float v = Ap[r * M] * pt[0];
#pragma unroll
                        for (int a = 1; a < M; ++a) v = fmaf(Ap[r * M + a], pt[a], v);
                        if (!right) v -= bp[r];
                        dF[(l * nr + r) * T + ls] = v;
                    }
                }
                for (int s = ptid; s < ni4 + nj4; s += pn) {
                    const bool right = s >= ni4;
                    const int ls = right ? s - ni4 : s;
                    const float* xa = xab + (right ? T + ls : ls) * G;
                    float mr = 0.f, md = 0.f;
#pragma unroll
                    for (int c = 0; c < G; ++c) {
                        mr = fmaf(tab[L.f_HC + (right ? G : 0) + c], xa[c], mr);
                        md = fmaf(tab[L.f_DC + (right ? G : 0) + c], xa[c], md);
                    }
                    magR[(right ? T : 0) + ls] = mr;
                    magF[(right ? T : 0) + ls] = md * s_rown1 + (right ? 0.f : s_bmax);
                }
                if (t + 1 < itc.t1) {
                    float* nxt = tabs + ((t + 1 - itc.t0) & 1) * L.f_stride;
                    for (int u = ptid; u < L.f_stride; u += pn) nxt[u] = P.tab32[(long long)(Qd.tabOff + t + 1) * L.f_stride + u];
                }
                if (ptid == 0) {
                    StageMeta& mt = meta[stage];
                    mt.end = 0;
                    mt.q = itd.q;
                    mt.k = k;
                    mt.i0 = i0;
                    mt.j0 = j0;
                    mt.TI = TI;
                    mt.TJ = TJ;
                    mt.nk = itd.nk;
                    mt.nr = nr;
                    mt.t = t;
                    mt.base = itd.base;
                }
                ws::bar_producers();  // halves, next table and metadata written
                if (ptid == 0) ws::mbar_arrive(&full[stage]);
                ++uses[stage];
                stage ^= 1;
            }
            if (!ok) break;
        }
        // end of work: hand the consumers an end marker
        if (ptid == 0) {
            bool wok = true;
            if (uses[stage] > 0) wok = ws::mbar_wait(&empty[stage], (uses[stage] - 1) & 1u, P.info);
            meta[stage].end = 1;
            (void)wok;
            ws::mbar_arrive(&full[stage]);
        }
    } else {
        // ------------------------------ consumers ------------------------------
        const int ctid = tid - 256;
        int stage = 0;
        uint32_t uses[2] = {0u, 0u};
        unsigned long long rp_cnt = 0;
        for (;;) {
            if (!ws::mbar_wait(&full[stage], uses[stage] & 1u, P.info)) {
                s_stop = 1;
                break;
            }
            const StageMeta mt = meta[stage];
            if (mt.end) break;
            float *UL, *UR, *FL, *FR, *CL, *CRr, *magR, *magF;
            stage_ptr(stage, UL, UR, FL, FR, CL, CRr, magR, magF);
            const int ni4 = (mt.TI + 3) & ~3, nj4 = (mt.TJ + 3) & ~3;
            const int ngi = ni4 >> 2, ngj = nj4 >> 2;
            const bool act = ctid < ngi * ngj;
            const int gi = act ? ctid / ngj : 0, gj = act ? ctid % ngj : 0;
            uint32_t vmask = 0, dmask = 0;
#pragma unroll
            for (int qa = 0; qa < 4; ++qa)
#pragma unroll
                for (int qb = 0; qb < 4; ++qb) {
                    const int li = 4 * gi + qa, lj = 4 * gj + qb;
                    if (act && li < mt.TI && lj < mt.TJ) vmask |= 1u << (qa * 4 + qb);
                    if (mt.i0 + li == mt.j0 + lj) dmask |= 1u << (qa * 4 + qb);  // a state paired with itself
                }
            if (act) {
                Item itd;
                itd.q = mt.q;
                itd.k = mt.k;
                itd.i0 = mt.i0;
                itd.j0 = mt.j0;
                itd.TI = mt.TI;
                itd.TJ = mt.TJ;
                itd.nk = mt.nk;
                itd.base = mt.base;
                pair_phase<M, G, PD>(P, itd, mt.t, T, gi, gj, vmask, dmask, mt.nr, DR, UL, UR, FL, FR, CL, CRr, magR,
                                     magF, KR, KF, rp_cnt);
            }
            __syncwarp();
            if (lane == 0) ws::mbar_arrive(&empty[stage]);
            ++uses[stage];
            stage ^= 1;
        }
        for (int o = 16; o > 0; o >>= 1) rp_cnt += __shfl_down_sync(0xffffffffu, rp_cnt, o);
        if (lane == 0 && rp_cnt) atomicAdd(&P.info->reach_pass, rp_cnt);
    }
}

// ---------------------------------------------------------------------------
// Precision form: the per-state products H xi and A p (the halves of the reach
// rows and of the polytope rows of the control points) on the 5th-generation
// tensor cores; the cost halves stay FP32 FMAs (computed while the MMA runs).
// Per item and duration one CTA builds, in shared memory, the operand
//   A [128 x K] : rows 0..63 the centred start states x~_i, rows 64..127 the
//                 end states x~_j, features (c, a) and a constant 1,
//   B [N x K]   : row n < NRp the start-half coefficients of output row n,
//                 row NRp + n the end-half coefficients,
// both TF32 (kind::tf32) or BF16 (kind::f16) and K-major without swizzle
// (8-row x 16-byte core matrices; LBO = K-chunk stride, SBO = row-group
// stride), and one thread issues tcgen05.mma (M = 128, N <= 256, FP32
// accumulators in tensor memory) and commits to an mbarrier.  The warps read
// the accumulators back with tcgen05.ld (warp w reads lanes 32 (w % 4) ..) and
// scatter the halves into the same shared-memory arrays the FP32 kernel uses;
// the pair phase is shared.  The error bands grow with the input rounding
// (2^-11 TF32, 2^-8 BF16) and every ambiguous margin is re-checked in FP64.
// ---------------------------------------------------------------------------
namespace tc {

DEVI uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

DEVI void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(slot)), "r"(ncols)
                 : "memory");
}
DEVI void tmem_relinquish() { asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory"); }
DEVI void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
DEVI void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
DEVI bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
DEVI void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
DEVI void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
DEVI void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
DEVI void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <bool BF>
DEVI void mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accumulate) {
    if (BF)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
}
DEVI void commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}
DEVI void ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}
// Shared-memory matrix descriptor: start >> 4 (bits 0-13), LBO >> 4 (16-29),
// SBO >> 4 (32-45), descriptor version 1 (46-47), no swizzle (61-63 = 0).
DEVI uint64_t desc(uint32_t saddr_bytes, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr_bytes >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// Instruction descriptor (kind::f16 / kind::tf32): D = F32 (bits 4-5 = 1),
// A/B format (bits 7-9, 10-12: BF16 = 1, TF32 = 2), both K-major (bits 15,
// 16 = 0), N >> 3 (bits 17-22), M >> 4 (bits 24-28).
DEVI uint32_t idesc(int Mdim, int Ndim, bool bf) {
    const uint32_t fmt = bf ? 1u : 2u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(Ndim >> 3) << 17) | ((uint32_t)(Mdim >> 4) << 24);
}
}  // namespace tc

template <int M, int G, int PD, bool BF>
__global__ void __launch_bounds__(256, 2) k_pairs_tc(BuildParams P) {
    using S = Shape<G, PD>;
    constexpr int N_ = M * G, RAX = S::RAX, RR = M * RAX, NI = S::NI, TG = S::TG;
    constexpr int KFEAT = N_ + 1;
    constexpr int KI = BF ? 16 : 8;
    constexpr int KP = (KFEAT + KI - 1) / KI * KI;
    constexpr int ESZ = BF ? 2 : 4;
    constexpr int CHUNKS = KP * ESZ / 16;
    constexpr uint32_t LBO = 128, SBO = CHUNKS * 128;
    constexpr int KSTEPS = KP / KI;
    constexpr uint32_t TMEM_COLS = 256;
    const int T = P.tile;
    extern __shared__ __align__(1024) float sm[];
    const int FRm = NI * P.max_rows;
    const int DR = P.cost_mode == 1 ? 1 : G;
    const int CRW = G * PD * M;
    // operands first (1024-byte aligned), then the FP32 kernel's arrays
    unsigned char* Aop = reinterpret_cast<unsigned char*>(sm);
    const int NRcap = RR + FRm;  // reach and free rows go through the tensor cores
    const int NRp_cap = (NRcap + 7) & ~7;
    const int Ncap = (2 * NRp_cap + 15) & ~15;
    unsigned char* Bop = Aop + ((128 * KP * ESZ + 1023) & ~1023);
    float* UL = reinterpret_cast<float*>(Bop + ((Ncap * KP * ESZ + 1023) & ~1023));
    float* UR = UL + RR * T;
    float* FL = UR + RR * T;
    float* FR = FL + FRm * T;
    float* CL = FR + FRm * T;
    float* CRr = CL + CRW * T;
    float* magR = CRr + CRW * T;
    float* magF = magR + 2 * T;
    float* xs = magF + 2 * T;
    float* xab = xs + 2 * T * N_;
    float* tab = xab + 2 * T * G;
    float* Ap = tab + P.L.f_stride;
    float* bp = Ap + RMAX * M;
    __shared__ long long s_item;
    __shared__ float s_rown1, s_bmax;
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ int s_abort;

    const int tid = threadIdx.x, nthr = blockDim.x, warp = tid >> 5, lane = tid & 31;
    const long long nitems = (long long)P.info->items;
    const TabLayout L = P.L;
    const float kin = BF ? 0.00390625f : 0.00048828125f;  // 2^-8, 2^-11
    // input rounding of both factors (2 kin; 3 kin for the A (x) D coefficient)
    // plus a generous allowance for the tensor core's FP32 accumulation
    const float KRt = 2.f * (2.f * kin + 64.f * KU);
    const float KFt = 2.f * (3.f * kin + 64.f * KU);
    unsigned long long rp_cnt = 0;
    uint32_t phase = 0;

    if (warp == 0) {
        tc::tmem_alloc(&s_tmem, TMEM_COLS);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&s_mbar, 1);
        tc::fence_mbar_init();
        s_abort = 0;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = s_tmem;

    auto put = [&](unsigned char* base, int row, int k, float v) {
        const int chunk = (k * ESZ) >> 4, within = (k * ESZ) & 15;
        unsigned char* p = base + (row >> 3) * SBO + chunk * LBO + (row & 7) * 16 + within;
        if (BF) {
            *reinterpret_cast<__nv_bfloat16*>(p) = __float2bfloat16_rn(v);
        } else {
            uint32_t r;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
            *reinterpret_cast<uint32_t*>(p) = r;
        }
    };

    for (;;) {
        if (tid == 0) {
            const long long it = (long long)atomicAdd(&P.info->ticket, 1u);
            s_item = (has_failed(P.info) || s_abort) ? 0x7fffffffffffLL : it;
        }
        __syncthreads();
        const long long item = s_item;
        if (item >= nitems) break;
        const ItemT itc = item_decode_chunk(P, item);
        const Item& itd = itc.it;
        if (itc.t0 >= itc.t1) {
            __syncthreads();
            continue;
        }
        const QueryDesc& Qd = P.qd[itd.q];
        const int k = itd.k, i0 = itd.i0, j0 = itd.j0, TI = itd.TI, TJ = itd.TJ, nk = itd.nk;
        const int ni4 = (TI + 3) & ~3, nj4 = (TJ + 3) & ~3;
        const int r0 = Qd.poly_off[k], nr = Qd.poly_off[k + 1] - r0;
        const int NR = RR + NI * nr;
        const int NRp = (NR + 7) & ~7;
        const int Ntot = (2 * NRp + 15) & ~15;
        const long long rg0 = Qd.rowsOff + r0;
        for (int u = tid; u < nr * M; u += nthr) Ap[u] = P.A32[rg0 * M + u];
        for (int u = tid; u < nr; u += nthr) bp[u] = P.bc32[rg0 + u];
        const int* members = P.members + Qd.listOff + (long long)k * Qd.N;
        float cx[M];
#pragma unroll
        for (int a = 0; a < M; ++a) cx[a] = P.centers[(long long)(Qd.kOff + k) * 4 + a];
        for (int u = tid; u < (ni4 + nj4) * N_; u += nthr) {
            const int s = u / N_, e = u % N_;
            const bool right = s >= ni4;
            const int ls = right ? s - ni4 : s;
            const int lidx = (right ? j0 : i0) + ls;
            float v = 0.f;
            if (ls < (right ? TJ : TI)) {
                const long long id = mem_id(members[lidx]);
                if (e < M) {
                    if (P.in_f32) v = ((const float*)Qd.states)[id * N_ + e] - cx[e];
                    else v = (float)(((const double*)Qd.states)[id * N_ + e] - (double)cx[e]);
                } else {
                    v = ldf(Qd.states, id * N_ + e, P.in_f32);
                }
            }
            xs[(right ? T + ls : ls) * N_ + e] = v;
        }
        __syncthreads();
        for (int s = tid; s < ni4 + nj4; s += nthr) {
            const bool right = s >= ni4;
            const int ls = right ? s - ni4 : s;
            const float* x = xs + (right ? T + ls : ls) * N_;
            float* xa = xab + (right ? T + ls : ls) * G;
#pragma unroll
            for (int c = 0; c < G; ++c) {
                float mx = 0.f;
#pragma unroll
                for (int a = 0; a < M; ++a) mx = fmaxf(mx, fabsf(x[c * M + a]));
                xa[c] = mx;
            }
        }
        // operand A: 64 start rows, 64 end rows, features x~ then the constant 1
        for (int u = tid; u < 128 * KP; u += nthr) {
            const int row = u / KP, f = u % KP;
            const bool right = row >= 64;
            const int ls = right ? row - 64 : row;
            float v = 0.f;
            if (ls < (right ? nj4 : ni4)) {
                if (f < N_) v = xs[(right ? T + ls : ls) * N_ + f];
                else if (f == N_) v = 1.f;
            }
            put(Aop, row, f, v);
        }
        if (tid == 0) {
            float rn = 0.f, bm = 0.f;
            for (int r = 0; r < nr; ++r) {
                float s1 = 0.f;
                for (int a = 0; a < M; ++a) s1 += fabsf(Ap[r * M + a]);
                rn = fmaxf(rn, s1);
                bm = fmaxf(bm, fabsf(bp[r]));
            }
            s_rown1 = rn * 1.0001f;
            s_bmax = bm;
        }
        __syncthreads();

        const int ngi = ni4 >> 2, ngj = nj4 >> 2;
        const bool act = tid < ngi * ngj;
        const int gi = act ? tid / ngj : 0, gj = act ? tid % ngj : 0;
        uint32_t vmask = 0, dmask = 0;
#pragma unroll
        for (int qa = 0; qa < 4; ++qa)
#pragma unroll
            for (int qb = 0; qb < 4; ++qb) {
                const int li = 4 * gi + qa, lj = 4 * gj + qb;
                if (act && li < TI && lj < TJ) vmask |= 1u << (qa * 4 + qb);
                if (i0 + li == j0 + lj) dmask |= 1u << (qa * 4 + qb);  // a state paired with itself
            }
        for (int t = itc.t0; t < itc.t1; ++t) {
            for (int u = tid; u < L.f_stride; u += nthr) tab[u] = P.tab32[(long long)(Qd.tabOff + t) * L.f_stride + u];
            __syncthreads();
            // operand B: coefficient rows (start halves, then end halves)
            for (int u = tid; u < Ntot * KP; u += nthr) {
                const int n = u / KP, f = u % KP;
                const bool right = n >= NRp;
                const int o = right ? n - NRp : n;
                const int co = right ? G : 0;
                float v = 0.f;
                if (o < NR && f <= N_) {
                    const int c = f / M, a = f % M;
                    if (o < RR) {  // reach row (r, axis)
                        const int r = o / M, ra = o % M;
                        if (f < N_ && a == ra) v = tab[L.f_H + r * TG + co + c];
                    } else {  // free row (l, polytope row)
                        const int q = o - RR, l = q / nr, rr = q % nr;
                        if (f < N_) v = Ap[rr * M + a] * tab[L.f_D + l * TG + co + c];
                        else if (!right) v = -bp[rr];
                    }
                }
                put(Bop, n, f, v);
            }
            for (int s = tid; s < ni4 + nj4; s += nthr) {
                const bool right = s >= ni4;
                const int ls = right ? s - ni4 : s;
                const float* xa = xab + (right ? T + ls : ls) * G;
                float mr = 0.f, md = 0.f;
#pragma unroll
                for (int c = 0; c < G; ++c) {
                    mr = fmaf(tab[L.f_HC + (right ? G : 0) + c], xa[c], mr);
                    md = fmaf(tab[L.f_DC + (right ? G : 0) + c], xa[c], md);
                }
                magR[(right ? T : 0) + ls] = mr;
                magF[(right ? T : 0) + ls] = md * s_rown1 + (right ? 0.f : s_bmax);
            }
            tc::fence_async_smem();
            tc::fence_before();
            __syncthreads();
            tc::fence_after();
            if (tid == 0) {
                const uint32_t id = tc::idesc(128, Ntot, BF);
#pragma unroll
                for (int st = 0; st < KSTEPS; ++st) {
                    const uint64_t ad = tc::desc(tc::saddr(Aop) + st * 2 * LBO, LBO, SBO);
                    const uint64_t bd = tc::desc(tc::saddr(Bop) + st * 2 * LBO, LBO, SBO);
                    tc::mma<BF>(tbase, ad, bd, id, st > 0 ? 1u : 0u);
                }
                tc::commit(&s_mbar);
            }
            // cost halves stay FP32 (FMA), computed while the MMA runs
            for (int u = tid; u < (ni4 + nj4) * M; u += nthr) {
                const int s = u / M, a = u % M;
                const bool right = s >= ni4;
                const int ls = right ? s - ni4 : s;
                const float* x = xs + (right ? T + ls : ls) * N_;
                float xc[G];
#pragma unroll
                for (int c = 0; c < G; ++c) xc[c] = x[c * M + a];
                const int co = right ? G : 0;
                float* dC = right ? CRr : CL;
                for (int d = 0; d < DR; ++d)
                    for (int l = 0; l < PD; ++l) {
                        const float* cc = tab + L.f_C + (d * PD + l) * TG + co;
                        float v = cc[0] * xc[0];
#pragma unroll
                        for (int c = 1; c < G; ++c) v = fmaf(cc[c], xc[c], v);
                        dC[((l * DR + d) * M + a) * T + ls] = v;
                    }
            }
            {
                long long spins = 0;
                while (!tc::mbar_try_wait(&s_mbar, phase)) {
                    if (++spins > (1LL << 22)) {
                        set_status(P.info, PLAN_ERR_TIMEOUT, DET_BARRIER);
                        s_abort = 1;
                        break;
                    }
                }
                phase ^= 1u;
            }
            tc::fence_after();
            // accumulators -> halves: warp w reads lanes 32 (w % 4) + lane
            {
                const int quarter = warp & 3;
                const int row = quarter * 32 + lane;
                const bool right = row >= 64;
                const int ls = right ? row - 64 : row;
                const bool live = ls < (right ? nj4 : ni4);
                const int c0 = right ? NRp : 0;
                const int nchunk = (NR + 15) >> 4;
                for (int ch = (warp >> 2); ch < nchunk; ch += (nthr >> 7)) {
                    float v[16];
                    tc::ld16(tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(c0 + ch * 16), v);
                    if (live) {
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const int o = ch * 16 + q;
                            if (o >= NR) break;
                            if (o < RR) (right ? UR : UL)[o * T + ls] = v[q];
                            else (right ? FR : FL)[(o - RR) * T + ls] = v[q];
                        }
                    }
                }
            }
            tc::fence_before();
            __syncthreads();
            if (act)
                pair_phase<M, G, PD>(P, itd, t, T, gi, gj, vmask, dmask, nr, DR, UL, UR, FL, FR, CL, CRr, magR, magF,
                                     KRt, KFt, rp_cnt);
            __syncthreads();
        }
    }
    block_add(&P.info->reach_pass, rp_cnt);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tbase, TMEM_COLS);
}

// ---------------------------------------------------------------------------
// Canonical FP64 helpers (must match the oracle's operation order exactly).
// ---------------------------------------------------------------------------
template <int G>
DEVI double half_sum(const double* coef, const double* x, int stride) {
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < G; ++c) s = __dadd_rn(s, __dmul_rn(coef[c], x[c * stride]));
    return s;
}

template <int G, int PD>
DEVI int reach_order(int r) {  // derivative order k of canonical reach row r (k-major)
    int k = 1, acc = PD;
    while (r >= acc && k < G) {
        ++k;
        acc += PD - k + 1;
    }
    return k;
}

// A2/A3 FP64 canonical pair kernel: every decision is made in the canonical
// order, so no re-check is needed.
template <int M, int G, int PD>
__global__ void __launch_bounds__(256) k_pairs_f64(BuildParams P) {
    using S = Shape<G, PD>;
    constexpr int N_ = M * G, RAX = S::RAX, RR = M * RAX, NI = S::NI, TG = S::TG;
    constexpr int T = TILE64;
    extern __shared__ __align__(16) double smd[];
    const int DR = P.cost_mode == 1 ? 1 : G;
    const int CRW = G * PD * M;
    double* hL = smd;
    double* hR = hL + RR * T;
    double* cL = hR + RR * T;
    double* cR = cL + NI * M * T;
    double* kL = cR + NI * M * T;
    double* kR = kL + CRW * T;
    double* xs = kR + CRW * T;
    double* tab = xs + 2 * T * N_;
    double* Ap = tab + P.L.e_stride;
    double* bl = Ap + RMAX * M;
    double* limr = bl + RMAX;
    double* bcs = limr + RAX;         // [T*T] best cost
    uint32_t* bbits = (uint32_t*)(bcs + T * T);
    uint8_t* bts = (uint8_t*)(bbits + T * T);
    __shared__ long long s_item;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const long long nitems = (long long)P.info->items;
    const TabLayout L = P.L;
    unsigned long long rp_cnt = 0;
    for (int r = tid; r < RAX; r += nthr) limr[r] = P.lim64[reach_order<G, PD>(r) - 1];
    for (;;) {
        if (tid == 0) {
            const long long it = (long long)atomicAdd(&P.info->ticket, 1u);
            s_item = has_failed(P.info) ? 0x7fffffffffffLL : it;  // one decision for the whole block
        }
        __syncthreads();
        const long long item = s_item;
        if (item >= nitems) break;
        const ItemT itc = item_decode_chunk(P, item);
        const Item& itd = itc.it;
        if (itc.t0 >= itc.t1) {  // empty chunk (nT < number of chunks)
            __syncthreads();     // everyone has read s_item before it is rewritten
            continue;
        }
        const QueryDesc& Qd = P.qd[itd.q];
        const int k = itd.k, i0 = itd.i0, j0 = itd.j0, TI = itd.TI, TJ = itd.TJ, nk = itd.nk;
        const int r0 = Qd.poly_off[k], nr = Qd.poly_off[k + 1] - r0;
        for (int u = tid; u < nr * M; u += nthr) Ap[u] = ldv(Qd.A, (long long)r0 * M + u, P.in_f32);
        for (int u = tid; u < nr; u += nthr) bl[u] = P.blim64[Qd.rowsOff + r0 + u];
        const int* members = P.members + Qd.listOff + (long long)k * Qd.N;
        for (int u = tid; u < (TI + TJ) * N_; u += nthr) {
            const int s = u / N_, e = u % N_;
            const bool right = s >= TI;
            const int ls = right ? s - TI : s;
            const long long id = mem_id(members[(right ? j0 : i0) + ls]);
            xs[(right ? T + ls : ls) * N_ + e] = ldv(Qd.states, id * N_ + e, P.in_f32);
        }
        for (int u = tid; u < T * T; u += nthr) {
            bcs[u] = __longlong_as_double(DINF_BITS);
            bbits[u] = 0;
            bts[u] = 0;
        }
        __syncthreads();
        for (int t = itc.t0; t < itc.t1; ++t) {
            for (int u = tid; u < L.e_stride; u += nthr) tab[u] = P.tab64[(long long)(Qd.tabOff + t) * L.e_stride + u];
            __syncthreads();
            for (int u = tid; u < (TI + TJ) * M; u += nthr) {
                const int s = u / M, a = u % M;
                const bool right = s >= TI;
                const int ls = right ? s - TI : s;
                const double* x = xs + (right ? T + ls : ls) * N_ + a;
                const int co = right ? G : 0;
                double* dh = right ? hR : hL;
                for (int r = 0; r < RAX; ++r) dh[(r * M + a) * T + ls] = half_sum<G>(tab + L.e_H + r * TG + co, x, M);
                double* dc = right ? cR : cL;
                for (int l = 1; l <= NI; ++l)
                    dc[((l - 1) * M + a) * T + ls] = half_sum<G>(tab + L.e_D + l * TG + co, x, M);
                double* dk = right ? kR : kL;
                for (int d = 0; d < DR; ++d)
                    for (int l = 0; l < PD; ++l)
                        dk[((l * DR + d) * M + a) * T + ls] = half_sum<G>(tab + L.e_C + (d * PD + l) * TG + co, x, M);
            }
            __syncthreads();
            for (int pp = tid; pp < TI * TJ; pp += nthr) {
                const int li = pp / TJ, lj = pp % TJ;
                if (i0 + li == j0 + lj) continue;
                bool ok = true;
                for (int r = 0; r < RAX && ok; ++r) {
                    const double lim = limr[r];
#pragma unroll
                    for (int a = 0; a < M; ++a) {
                        const double s = __dadd_rn(hL[(r * M + a) * T + li], hR[(r * M + a) * T + lj]);
                        if (!(fabs(s) <= lim)) ok = false;
                    }
                }
                if (!ok) continue;
                ++rp_cnt;
                for (int l = 0; l < NI && ok; ++l) {
                    double pt[M];
#pragma unroll
                    for (int a = 0; a < M; ++a) pt[a] = __dadd_rn(cL[(l * M + a) * T + li], cR[(l * M + a) * T + lj]);
                    for (int r = 0; r < nr; ++r) {
                        double s = 0.0;
#pragma unroll
                        for (int a = 0; a < M; ++a) s = __dadd_rn(s, __dmul_rn(Ap[r * M + a], pt[a]));
                        if (!(s <= bl[r])) {
                            ok = false;
                            break;
                        }
                    }
                }
                if (!ok) continue;
                double cost = 0.0;
                const int per_l = DR * M;
                for (int l = 0; l < PD; ++l) {
                    double ss = 0.0;
                    for (int e = 0; e < per_l; ++e) {
                        const int row = l * per_l + e;
                        const double d = kL[row * T + li] + kR[row * T + lj];
                        ss = fma(d, d, ss);
                    }
                    cost += sqrt(ss);
                }
                const int q = li * T + lj;
                bbits[q] |= 1u << t;
                if (cost < bcs[q]) {
                    bcs[q] = cost;
                    bts[q] = (uint8_t)t;
                }
            }
            __syncthreads();
        }
        // merge this chunk of durations into the pair slots (other chunks of
        // the same tile merge theirs: OR of the bits, min of cost | T)
        const long long base = itd.base;
        for (int pp = tid; pp < TI * TJ; pp += nthr) {
            const int li = pp / TJ, lj = pp % TJ;
            const int q = li * T + lj;
            if (!bbits[q]) continue;
            const long long slot = base + (long long)(i0 + li) * nk + (j0 + lj);
            atomicOr(&P.resBits[slot], bbits[q]);
            atomicMin(&P.resKey[slot], key_f64(bcs[q], bts[q]));
        }
        __syncthreads();
    }
    block_add(&P.info->reach_pass, rp_cnt);
}

// ---------------------------------------------------------------------------
// A4 re-check: ambiguous (polytope, pair, T) entries evaluated in canonical
// FP64 (reach rows, then the interior control points against polytope k).
// ---------------------------------------------------------------------------
template <int M, int G, int PD>
__global__ void __launch_bounds__(RECHECK_THREADS) k_recheck(BuildParams P) {
    // one entry per block of four warps, blocks spread over all SMs: every
    // sub-partition of an SM has its own FP64 unit and GB300's FP64 rate is
    // low, so an entry's rows are split over the four (threads take the rows,
    // each row in canonical order); the control-polygon segments' squared
    // norms are then summed in canonical order by one thread per segment
    using S = Shape<G, PD>;
    constexpr int N_ = M * G, RAX = S::RAX, NI = S::NI, TG = S::TG;
    __shared__ double s_v[PD * G * M];
    __shared__ double s_seg[PD];
    long long n = 0;
    if (block_failed(P.info, &P.info->rechecks, &n)) return;
    n = min(n, P.recheckCap);
    const int DR = P.cost_mode == 1 ? 1 : G;
    const TabLayout L = P.L;
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (long long e = blockIdx.x; e < n; e += gridDim.x) {
        const unsigned long long en = P.recheck[e];
        const int t = (int)(en & 31ull), lj = (int)((en >> 5) & 0xFFFFull), li = (int)((en >> 21) & 0xFFFFull);
        const int k = (int)((en >> 37) & 0x3FFull), q = (int)((en >> 47) & 0xFFFFull);
        const bool cost_only = (en >> 63) != 0;  // feasible for certain: only the cost in FP64
        const QueryDesc& Q = P.qd[q];
        const int nk = P.counts[Q.kOff + k];
        const int* members = P.members + Q.listOff + (long long)k * Q.N;
        const long long i = mem_id(members[li]), j = mem_id(members[lj]);
        double xi[N_], xj[N_];
#pragma unroll
        for (int c = 0; c < N_; ++c) {
            xi[c] = ldv(Q.states, i * N_ + c, P.in_f32);
            xj[c] = ldv(Q.states, j * N_ + c, P.in_f32);
        }
        const double* tb = P.tab64 + (long long)(Q.tabOff + t) * L.e_stride;
        int ok = 1;
        for (int u = cost_only ? RAX * M : tid; u < RAX * M; u += nthr) {
            const int r = u / M, a = u % M;
            const double s = __dadd_rn(half_sum<G>(tb + L.e_H + r * TG, xi + a, M),
                                       half_sum<G>(tb + L.e_H + r * TG + G, xj + a, M));
            if (!(fabs(s) <= P.lim64[reach_order<G, PD>(r) - 1])) ok = 0;
        }
        if (!__syncthreads_and(ok)) continue;
        const int r0 = Q.poly_off[k], nr = Q.poly_off[k + 1] - r0;
        for (int u = cost_only ? NI * nr : tid; u < NI * nr; u += nthr) {
            const int l = 1 + u / nr, r = r0 + u % nr;
            double s = 0.0;
            for (int a = 0; a < M; ++a) {
                const double pa = __dadd_rn(half_sum<G>(tb + L.e_D + l * TG, xi + a, M),
                                            half_sum<G>(tb + L.e_D + l * TG + G, xj + a, M));
                s = __dadd_rn(s, __dmul_rn(ldv(Q.A, (long long)r * M + a, P.in_f32), pa));
            }
            if (!(s <= P.blim64[Q.rowsOff + r])) ok = 0;
        }
        if (!__syncthreads_and(ok)) continue;
        // cost rows: value (l, d, a) of segment l, then each segment's squared
        // norm summed in (d, a) order and its root, then the segments in order
        for (int u = tid; u < PD * DR * M; u += nthr) {
            const int l = u / (DR * M), d = (u / M) % DR, a = u % M;
            s_v[u] = half_sum<G>(tb + L.e_C + (d * PD + l) * TG, xi + a, M) +
                     half_sum<G>(tb + L.e_C + (d * PD + l) * TG + G, xj + a, M);
        }
        __syncthreads();
        if (tid < PD) {
            double ss = 0.0;
            for (int w = 0; w < DR * M; ++w) {
                const double v = s_v[tid * DR * M + w];
                ss = fma(v, v, ss);
            }
            s_seg[tid] = sqrt(ss);
        }
        __syncthreads();
        if (tid == 0) {
            double cost = 0.0;
            for (int l = 0; l < PD; ++l) cost += s_seg[l];
            const long long slot = P.qSlot[q] + P.resOff[Q.kOff + k] + (long long)li * nk + lj;
            atomicOr(&P.resBits[slot], 1u << t);
            atomicMin(&P.resKey[slot], key_f32((float)cost, t));
        }
        __syncthreads();  // s_v and s_seg are rewritten by the next entry
    }
}

// ---------------------------------------------------------------------------
// A5 compaction.  The pair (i, j) is emitted by its lowest shared polytope
// (its "owner"); bits are OR-ed and keys min-ed over all shared polytopes.
// Pass 1 counts per row and stores, for each slot, the inclusive count of
// emitted entries in its (row, polytope) segment; pass 2 places every entry
// at its rank among the row's emitted ids (sorted by j).
// ---------------------------------------------------------------------------
struct QView {  // per-query pointers into the shared scratch
    const QueryDesc* Q;
    const uint32_t* mask;
    const int* counts;
    const int* members;
    const int* localIdx;
    const long long* resOff;
    long long slot0;
    __device__ QView(const BuildParams& P, int q) {
        Q = &P.qd[q];
        mask = P.memMask + Q->maskOff;
        counts = P.counts + Q->kOff;
        members = P.members + Q->listOff;
        localIdx = P.localIdx + Q->listOff;
        resOff = P.resOff + Q->kOff;
        slot0 = P.qSlot[q];
    }
    __device__ long long seg(int k, int i) const {  // slot of (member i, member 0) in polytope k
        return slot0 + resOff[k] + (long long)localIdx[(long long)k * Q->N + i] * counts[k];
    }
};

DEVI int owner_of(const QView& V, int i, int j, int& nshared) {
    int owner = -1;
    nshared = 0;
    const int W = V.Q->W;
    for (int w = 0; w < W; ++w) {
        const uint32_t x = V.mask[(long long)i * W + w] & V.mask[(long long)j * W + w];
        if (x && owner < 0) owner = w * 32 + __ffs(x) - 1;
        nshared += __popc(x);
    }
    return owner;
}

DEVI void combine(const BuildParams& P, const QView& V, int i, int j, int k, uint32_t& bits, unsigned long long& key) {
    const int W = V.Q->W;
    for (int w = k >> 5; w < W; ++w) {
        uint32_t x = V.mask[(long long)i * W + w] & V.mask[(long long)j * W + w];
        if (w == (k >> 5)) x &= ~((2u << (k & 31)) - 1u);  // polytopes above k
        while (x) {
            const int k2 = w * 32 + __ffs(x) - 1;
            x &= x - 1u;
            const long long s2 = V.seg(k2, i) + V.localIdx[(long long)k2 * V.Q->N + j];
            bits |= P.resBits[s2];
            const unsigned long long k2v = P.resKey[s2];
            if (k2v < key) key = k2v;
        }
    }
}

// Segment of the flat membership index g: query, polytope k and the state's
// local index li in it.
struct SegRef {
    int q, k, li;
};
DEVI SegRef seg_of(const BuildParams& P, long long g) {
    SegRef r;
    r.q = P.Q == 1 ? 0 : find_q(P.qMem, P.Q, g);
    const int v = P.segKL[g];
    r.k = v >> 16;
    r.li = v & 0xffff;
    return r;
}

// Pass 1, one warp per row segment (state i in polytope k, its slots (i, j)
// for the polytope's members j): is each slot the pair's owner (the lowest
// polytope both states contain -- only pairs of states that both lie in
// several polytopes can be shared), and is the pair feasible for some
// duration?  The owner slot receives the pair's result combined over all
// shared polytopes; emitPre gets the inclusive prefix of the emitted flags
// within the segment, and the segment total adds to row i's count.
__global__ void __launch_bounds__(256, 4) k_emit(BuildParams P) {
    long long nseg = 0;
    if (block_failed(P.info, &P.info->memberships, &nseg)) return;
    const int lane = threadIdx.x & 31;
    unsigned long long cand = 0, chk = 0, feas = 0;
    for (long long g = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; g < nseg;
         g += ((long long)gridDim.x * blockDim.x) >> 5) {
        const SegRef sr = seg_of(P, g);
        const QView V(P, sr.q);
        const QueryDesc& Q = *V.Q;
        const int k = sr.k, nk = V.counts[k];
        const int* mem = V.members + (long long)k * Q.N;
        const int im = mem[sr.li];
        const int i = mem_id(im);
        if (i < P.rowRange[2 * sr.q] || i >= P.rowRange[2 * sr.q + 1]) continue;  // another shard's row
        const long long base = V.slot0 + V.resOff[k] + (long long)sr.li * nk;
        int running = 0;
        for (int lg = 0; lg < nk; lg += 128) {
            // four chunks of 32 slots: every load of the group is issued first
            int jv[4];
            uint32_t bv[4];
            unsigned long long kv[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int lj = lg + 32 * c + lane;
                const bool in = lj < nk;
                jv[c] = in ? mem[lj] : 0;
                bv[c] = in ? P.resBits[base + lj] : 0u;
                kv[c] = in ? P.resKey[base + lj] : 0ull;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int lj = lg + 32 * c + lane;
                if (lg + 32 * c >= nk) break;  // warp-uniform
                int flag = 0;
                if (lj < nk) {
                    const int jm = jv[c], j = mem_id(jm);
                    if (i != j) {
                        int ns = 1;
                        if (!(mem_multi(im) && mem_multi(jm)) || owner_of(V, i, j, ns) == k) {
                            ++cand;
                            chk += Q.nT;
                            uint32_t bits = bv[c];
                            if (ns > 1) {
                                unsigned long long key = kv[c];
                                combine(P, V, i, j, k, bits, key);
                                P.resBits[base + lj] = bits;
                                P.resKey[base + lj] = key;
                            }
                            flag = bits != 0;
                            feas += __popc(bits);
                        }
                    }
                }
                const unsigned bal = __ballot_sync(0xffffffffu, flag != 0);
                if (lj < nk) P.emitPre[base + lj] = running + __popc(bal & ((2u << lane) - 1u));
                running += __popc(bal);
            }
        }
        if (lane == 0 && running) atomicAdd(&P.rowCount[Q.rowOff + i], running);
    }
    block_add(&P.info->candidates, cand);
    block_add(&P.info->checks, chk);
    block_add(&P.info->feasible, feas);
}

// One CTA per query: exclusive scan of the row counts into row_off, E, capacity.
__global__ void __launch_bounds__(1024) k_scan(BuildParams P) {
    __shared__ long long wb[32];
    __shared__ long long tot;
    if (has_failed(P.info)) return;
    const QueryDesc& Q = P.qd[blockIdx.x];
    const int N = Q.N;
    const int* rc = P.rowCount + Q.rowOff;
    const int per = (N + blockDim.x - 1) / blockDim.x;
    const int s0 = threadIdx.x * per, s1 = min(N, s0 + per);
    long long local = 0;
    for (int i = s0; i < s1; ++i) local += rc[i];
    long long run = block_exclusive_scan<long long>(local, wb, &tot);
    const long long total = tot;
    for (int i = s0; i < s1; ++i) {
        Q.row_off[i] = (int32_t)run;
        run += rc[i];
    }
    if (threadIdx.x == 0) {
        Q.row_off[N] = (int32_t)total;
        atomicAdd(&P.info->edges, (unsigned long long)total);
        *Q.count = total;
        if (total > Q.cap || total > 0x7fffffffLL) set_status(P.info, PLAN_ERR_CAPACITY, DET_OUTPUT);
    }
}

DEVI void write_edge(const BuildParams& P, const QueryDesc& Q, long long o, int j, uint32_t bits,
                      unsigned long long key) {
    Q.col[o] = j;
    Q.mask[o] = bits;
    Q.tidx[o] = (uint8_t)(key & 31ull);
    if (P.arith == PLAN_F64) ((double*)Q.w)[o] = __longlong_as_double((long long)(key & ~31ull));
    else if (P.w64) ((double*)Q.w)[o] = (double)__uint_as_float((unsigned)(key >> 32));  // replaced by k_cost64
    else ((float*)Q.w)[o] = __uint_as_float((unsigned)(key >> 32));
}

// Output pass.  Work items [0, memberships) are row segments: a state that
// lies in one polytope only has its whole row there, so an emitted entry's
// rank in the row is the segment prefix -- one warp per segment.  Items
// [memberships, memberships + rows) are rows of states in several polytopes:
// one warp per row merges its segments' emitted ids (each segment already in
// ascending order) by rank, with the segments' ids staged in shared memory,
// or, when they do not fit, by binary searches in the other segments' member
// lists.
__global__ void __launch_bounds__(256, 4) k_compact_fill(BuildParams P, int run_cap) {
    extern __shared__ uint32_t bmem[];
    __shared__ int s_meta[8][32 * 4 + 1];
    __shared__ long long s_metab[8][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    long long nseg = 0;
    if (block_failed(P.info, &P.info->memberships, &nseg)) return;
    const long long nitem = nseg + P.totN;
    int* runs = reinterpret_cast<int*>(bmem) + (size_t)wib * run_cap;  // this warp's staged ids
    for (long long it0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; it0 < nitem;
         it0 += ((long long)gridDim.x * blockDim.x) >> 5) {
        // rows first: the long multi-polytope rows start early instead of
        // forming the tail
        const long long it = it0 < P.totN ? nseg + it0 : it0 - P.totN;
        if (it < nseg) {
            const SegRef sr = seg_of(P, it);
            const QView V(P, sr.q);
            const QueryDesc& Q = *V.Q;
            const int* mem = V.members + (long long)sr.k * Q.N;
            const int im = mem[sr.li];
            if (mem_multi(im)) continue;  // the row item handles it
            if (mem_id(im) < P.rowRange[2 * sr.q] || mem_id(im) >= P.rowRange[2 * sr.q + 1]) continue;
            const int nk = V.counts[sr.k];
            const long long base = V.slot0 + V.resOff[sr.k] + (long long)sr.li * nk;
            const long long rbase = Q.row_off[mem_id(im)];
            for (int lg = 0; lg < nk; lg += 128) {
                int pv[4], pp[4], jv[4];
                uint32_t bv[4];
                unsigned long long kv[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {  // every load of the group first
                    const int lj = lg + 32 * c + lane;
                    const bool in = lj < nk;
                    pv[c] = in ? P.emitPre[base + lj] : 0;
                    pp[c] = in && lj > 0 ? P.emitPre[base + lj - 1] : 0;
                    jv[c] = in ? mem[lj] : 0;
                    bv[c] = in ? P.resBits[base + lj] : 0u;
                    kv[c] = in ? P.resKey[base + lj] : 0ull;
                }
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (pv[c] != pp[c]) write_edge(P, Q, rbase + pp[c], mem_id(jv[c]), bv[c], kv[c]);
            }
            continue;
        }
        const long long row = it - nseg;
        const int q = find_q(P.pfxN, P.Q, row);
        const QView V(P, q);
        const QueryDesc& Q = *V.Q;
        const int i = (int)(row - P.pfxN[q]);
        if (i < P.rowRange[2 * q] || i >= P.rowRange[2 * q + 1]) continue;  // another shard's row
        const int W = Q.W;
        int npoly = 0;
        for (int w = 0; w < W; ++w) npoly += __popc(V.mask[(long long)i * W + w]);
        if (npoly < 2) continue;  // a segment item handled it
        const long long rbase = Q.row_off[i];
        // Segment metadata (lane t: the row's t-th polytope): base slot, size,
        // emitted count (the segment prefix at its last slot), run offset.
        int* s_k = s_meta[wib];
        int* s_nk = s_k + 32;
        int* s_e = s_k + 64;
        int* s_off = s_k + 96;  // 33 entries
        long long* s_base = s_metab[wib];
        int total = 0x7fffffff;
        if (npoly <= 32) {
            if (lane == 0) {
                int t = 0;
                for (int w = 0; w < W; ++w) {
                    uint32_t mw = V.mask[(long long)i * W + w];
                    while (mw) {
                        s_k[t++] = w * 32 + __ffs(mw) - 1;
                        mw &= mw - 1u;
                    }
                }
            }
            __syncwarp();
            if (lane < npoly) {
                const int k = s_k[lane], nk = V.counts[k];
                const long long base = V.seg(k, i);
                s_nk[lane] = nk;
                s_base[lane] = base;
                s_e[lane] = nk > 0 ? P.emitPre[base + nk - 1] : 0;
            }
            __syncwarp();
            if (lane == 0) {
                int run = 0;
                for (int t = 0; t < npoly; ++t) {
                    s_off[t] = run;
                    run += s_e[t];
                }
                s_off[npoly] = run;
            }
            __syncwarp();
            total = s_off[npoly];
        }
        if (total <= run_cap / 2) {
            // Runs: each segment's emitted ids, in slot order (ascending ids), in
            // shared memory; an entry's rank in the row is its segment prefix
            // plus, for every other segment, the number of its ids below it
            // (binary search in shared memory).
            int* runj = runs + run_cap / 2;  // slot index (within its segment) of each staged id
            for (int t = 0; t < npoly; ++t) {
                const int nk = s_nk[t];
                const long long base = s_base[t];
                const int* mem = V.members + (long long)s_k[t] * Q.N;
                const int off = s_off[t];
                for (int lg = 0; lg < nk; lg += 128) {
                    int pv[4], pp[4], jv[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {  // every load of the group first
                        const int lj = lg + 32 * c + lane;
                        const bool in = lj < nk;
                        pv[c] = in ? P.emitPre[base + lj] : 0;
                        pp[c] = in && lj > 0 ? P.emitPre[base + lj - 1] : 0;
                        jv[c] = in ? mem[lj] : 0;
                    }
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (pv[c] != pp[c]) {
                            runs[off + pp[c]] = mem_id(jv[c]);
                            runj[off + pp[c]] = lg + 32 * c + lane;
                        }
                }
            }
            __syncwarp();
            // every staged entry: rank = its segment prefix + the other
            // segments' ids below it; then its result slot is copied out
            for (int e0 = 0; e0 < total; e0 += 64) {
                long long rk[2], slot[2];
                int jj[2];
                uint32_t bv[2];
                unsigned long long kv[2];
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int e = e0 + 32 * c + lane;
                    rk[c] = -1;
                    if (e < total) {
                        int t = 0;
                        while (t + 1 < npoly && s_off[t + 1] <= e) ++t;
                        const int j = runs[e];
                        long long rank = e - s_off[t];
                        for (int b = 0; b < npoly; ++b) {
                            if (b == t) continue;
                            const int* rb = runs + s_off[b];
                            int lo = 0, hi = s_e[b];
                            while (lo < hi) {
                                const int mid = (lo + hi) >> 1;
                                if (rb[mid] < j) lo = mid + 1;
                                else hi = mid;
                            }
                            rank += lo;
                        }
                        rk[c] = rank;
                        jj[c] = j;
                        slot[c] = s_base[t] + runj[e];
                    }
                }
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    bv[c] = rk[c] >= 0 ? P.resBits[slot[c]] : 0u;
                    kv[c] = rk[c] >= 0 ? P.resKey[slot[c]] : 0ull;
                }
#pragma unroll
                for (int c = 0; c < 2; ++c)
                    if (rk[c] >= 0) write_edge(P, Q, rbase + rk[c], jj[c], bv[c], kv[c]);
            }
        } else {
            // too many polytopes or entries for the shared-memory runs: count
            // the other segments' ids below j by binary search in their member
            // lists (global memory)
            for (int w = 0; w < W; ++w) {
                uint32_t mw = V.mask[(long long)i * W + w];
                while (mw) {
                    const int k = w * 32 + __ffs(mw) - 1;
                    mw &= mw - 1u;
                    const int nk = V.counts[k];
                    const long long base = V.seg(k, i);
                    const int* mem = V.members + (long long)k * Q.N;
                    for (int lj = lane; lj < nk; lj += 32) {
                        const int pre = P.emitPre[base + lj];
                        const int prev = lj > 0 ? P.emitPre[base + lj - 1] : 0;
                        if (pre == prev) continue;  // not emitted here
                        const int j = mem_id(mem[lj]);
                        long long rank = prev;
                        for (int w2 = 0; w2 < W; ++w2) {
                            uint32_t m2 = V.mask[(long long)i * W + w2];
                            while (m2) {
                                const int k2 = w2 * 32 + __ffs(m2) - 1;
                                m2 &= m2 - 1u;
                                if (k2 == k) continue;
                                const int n2 = V.counts[k2];
                                const int pos = lower_bound_members(V.members + (long long)k2 * Q.N, n2, j);
                                if (pos > 0) rank += P.emitPre[V.seg(k2, i) + pos - 1];
                            }
                        }
                        write_edge(P, Q, rbase + rank, j, P.resBits[base + lj], P.resKey[base + lj]);
                    }
                }
            }
        }
        __syncwarp();  // the runs are rebuilt by this warp's next row
    }
}

// ---------------------------------------------------------------------------
// Canonical FP64 costs of an FP64 model built by the FP32 pair kernels: for
// every emitted edge (i, j) and every duration t of its mask, the control-
// polygon length in the FP64 kernel's order -- each cost row (segment l,
// derivative d, axis a) the start half plus the end half, each half summed
// left to right without FMA; per segment the squared norm in (d, a) order
// with FMA, its root; the segments summed in order -- and the weight = the
// cheapest duration by the key (cost bits with the low five cleared | t),
// as the FP64 kernel's slot merge takes it.  The halves depend on one state
// and one duration only, so k_halves64 computes both halves of every state
// and duration once (half64 [state][t][side][row]); k_cost64 then adds,
// squares and takes roots per (edge, duration), one thread per edge.
// ---------------------------------------------------------------------------
template <int M, int G, int PD>
__global__ void __launch_bounds__(256) k_halves64(BuildParams P) {
    constexpr int N_ = M * G, TG = 2 * G;
    if (block_failed(P.info, nullptr, nullptr)) return;
    const TabLayout L = P.L;
    const int DR = P.cost_mode == 1 ? 1 : G;
    const int E = PD * DR * M;
    const long long per = (long long)P.maxT * 2 * E;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < P.totN * per;
         u += (long long)gridDim.x * blockDim.x) {
        const long long row = u / per;
        const int rem = (int)(u % per), t = rem / (2 * E), side = (rem / E) & 1, r = rem % E;
        const int q = find_q(P.pfxN, P.Q, row);
        const QueryDesc& Q = P.qd[q];
        if (t >= Q.nT) continue;
        const long long i = row - P.pfxN[q];
        const int l = r / (DR * M), d = (r / M) % DR, a = r % M;
        double x[N_];
#pragma unroll
        for (int c = 0; c < N_; ++c) x[c] = ldv(Q.states, i * N_ + c, P.in_f32);
        const double* tb = P.tab64 + (long long)(Q.tabOff + t) * L.e_stride;
        P.half64[u] = half_sum<G>(tb + L.e_C + (d * PD + l) * TG + side * G, x + a, M);
    }
}

template <int M, int G, int PD>
__global__ void __launch_bounds__(256) k_cost64(BuildParams P) {
    if (block_failed(P.info, nullptr, nullptr)) return;
    const int DR = P.cost_mode == 1 ? 1 : G;
    const int E = PD * DR * M;
    const long long per = (long long)P.maxT * 2 * E;
    // one thread per edge (blocks of query blockIdx.y): full warps, since the
    // narrow FP64 pipe is what bounds this pass
    const int q = blockIdx.y;
    const QueryDesc& Q = P.qd[q];
    const long long E_q = *Q.count;
    const int N = Q.N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < E_q; e += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = N;  // the row of edge e: largest i with row_off[i] <= e
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (Q.row_off[mid] <= e) lo = mid;
            else hi = mid;
        }
        const int i = lo, j = Q.col[e];
        const double* hi64 = P.half64 + (P.pfxN[q] + i) * per;
        const double* hj64 = P.half64 + (P.pfxN[q] + j) * per;
        uint32_t bits = Q.mask[e];
        unsigned long long best = KEY_NONE;
        while (bits) {
            const int t = __ffs(bits) - 1;
            bits &= bits - 1u;
            const double* kl = hi64 + (long long)t * 2 * E;      // start half (side 0) of state i
            const double* kr = hj64 + (long long)t * 2 * E + E;  // end half (side 1) of state j
            double cost = 0.0;
            for (int l = 0; l < PD; ++l) {
                double ss = 0.0;
                for (int w = 0; w < DR * M; ++w) {
                    const double v = kl[l * DR * M + w] + kr[l * DR * M + w];
                    ss = fma(v, v, ss);
                }
                cost += sqrt(ss);
            }
            const unsigned long long key = key_f64(cost, t);
            if (key < best) best = key;
        }
        ((double*)Q.w)[e] = __longlong_as_double((long long)(best & ~31ull));
        Q.tidx[e] = (uint8_t)(best & 31ull);
    }
}

// ---------------------------------------------------------------------------
// Work accounting (untimed, on request): the algorithmic work of the edge
// build under short-circuit evaluation in the pair kernel's row order.  For
// every distinct check (owner pair, T): reach rows (row, axis) are counted up
// to and including the first violated one (all of them when the check passes
// the reach test); a reach-passing check then counts free rows (control point
// l, polytope row r) up to the first violated one for each shared polytope in
// turn, stopping at the first polytope that contains the hull; a feasible
// check counts one cost evaluation.  Margins use FP32 like the fast kernel.
// ---------------------------------------------------------------------------
template <int M, int G, int PD>
__global__ void k_account(BuildParams P, unsigned long long* work) {
    using S = Shape<G, PD>;
    constexpr int N_ = M * G, RAX = S::RAX, NI = S::NI, TG = S::TG;
    if (has_failed(P.info)) return;
    const TabLayout L = P.L;
    const long long total = (long long)P.info->slots;
    unsigned long long wr = 0, wf = 0, wc = 0;
    for (long long sidx = blockIdx.x * (long long)blockDim.x + threadIdx.x; sidx < total;
         sidx += (long long)gridDim.x * blockDim.x) {
        const int q = find_q(P.qSlot, P.Q, sidx);
        const QView V(P, q);
        const QueryDesc& Q = *V.Q;
        const long long ls = sidx - V.slot0;
        int lo = 0, hi = Q.K;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (V.resOff[mid] <= ls) lo = mid;
            else hi = mid;
        }
        const int k = lo, nk = V.counts[k];
        if (nk == 0) continue;
        const long long loc = ls - V.resOff[k];
        const int li = (int)(loc / nk), lj = (int)(loc % nk);
        const int i = mem_id(V.members[(long long)k * Q.N + li]), j = mem_id(V.members[(long long)k * Q.N + lj]);
        if (i == j || i < P.rowRange[2 * q] || i >= P.rowRange[2 * q + 1]) continue;
        int ns;
        if (owner_of(V, i, j, ns) != k) continue;
        float xi[N_], xj[N_];
        for (int c = 0; c < N_; ++c) {
            xi[c] = ldf(Q.states, (long long)i * N_ + c, P.in_f32);
            xj[c] = ldf(Q.states, (long long)j * N_ + c, P.in_f32);
        }
        for (int t = 0; t < Q.nT; ++t) {
            const float* tb = P.tab32 + (long long)(Q.tabOff + t) * L.f_stride;
            bool ok = true;
            for (int r = 0; r < RAX && ok; ++r)
                for (int a = 0; a < M && ok; ++a) {
                    float s = 0.f;
                    for (int c = 0; c < G; ++c) s += tb[L.f_H + r * TG + c] * xi[c * M + a] + tb[L.f_H + r * TG + G + c] * xj[c * M + a];
                    ++wr;
                    if (fabsf(s) > 1.f) ok = false;
                }
            if (!ok) continue;
            float pt[NI][M];
            for (int l = 0; l < NI; ++l)
                for (int a = 0; a < M; ++a) {
                    float s = 0.f;
                    for (int c = 0; c < G; ++c) s += tb[L.f_D + l * TG + c] * xi[c * M + a] + tb[L.f_D + l * TG + G + c] * xj[c * M + a];
                    pt[l][a] = s;
                }
            bool feas = false;
            for (int w = 0; w < Q.W && !feas; ++w) {
                uint32_t x = V.mask[(long long)i * Q.W + w] & V.mask[(long long)j * Q.W + w];
                while (x && !feas) {
                    const int k2 = w * 32 + __ffs(x) - 1;
                    x &= x - 1u;
                    bool fok = true;
                    for (int l = 0; l < NI && fok; ++l)
                        for (int r = Q.poly_off[k2]; r < Q.poly_off[k2 + 1] && fok; ++r) {
                            float s = 0.f;
                            for (int a = 0; a < M; ++a) s += P.A32[(Q.rowsOff + r) * M + a] * pt[l][a];
                            ++wf;
                            if (s > P.blim32[Q.rowsOff + r]) fok = false;
                        }
                    feas = fok;
                }
            }
            if (feas) ++wc;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        wr += __shfl_down_sync(0xffffffffu, wr, o);
        wf += __shfl_down_sync(0xffffffffu, wf, o);
        wc += __shfl_down_sync(0xffffffffu, wc, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&work[0], wr);
        atomicAdd(&work[1], wf);
        atomicAdd(&work[2], wc);
    }
}

int launch_account(const BuildParams& P, void* stream, int num_sms, unsigned long long* work) {
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = num_sms * 8;
    if (P.m == 2 && P.g == 2 && P.p == 3) k_account<2, 2, 3><<<nb, 256, 0, st>>>(P, work);
    else if (P.m == 2 && P.g == 2 && P.p == 5) k_account<2, 2, 5><<<nb, 256, 0, st>>>(P, work);
    else if (P.m == 3 && P.g == 3 && P.p == 5) k_account<3, 3, 5><<<nb, 256, 0, st>>>(P, work);
    else if (P.m == 3 && P.g == 3 && P.p == 7) k_account<3, 3, 7><<<nb, 256, 0, st>>>(P, work);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Launch sequence.
// ---------------------------------------------------------------------------
template <int M, int G, int PD>
size_t smem_fast(const BuildParams& P) {
    using S = Shape<G, PD>;
    const int RR = M * S::RAX, FRm = S::NI * P.max_rows, CRW = G * PD * M;
    const size_t T = (size_t)P.tile;
    size_t f = (size_t)(2 * RR + 2 * FRm + 2 * CRW + 4) * T + 2 * T * (M * G + G) + 2 * P.L.f_stride + RMAX * (M + 1);
    return f * sizeof(float);
}

// unscreened one-group FP32 kernel: halves, states, two padded tables, A|b rows
template <int M, int G, int PD>
size_t smem_one(const BuildParams& P) {
    using S = Shape<G, PD>;
    const int RR = M * S::RAX, FRm = S::NI * P.max_rows, CRW = G * PD * M;
    const size_t T = (size_t)P.tile;
    size_t f = (size_t)(2 * RR + 2 * FRm + 2 * CRW + 4) * T + 2 * T * (M * G + G) + 2 * PadTab<G, PD>::FLOATS + RMAX * 4;
    return f * sizeof(float);
}

// screened FP32 kernel: transposed halves, screen rows, band and cost
// magnitudes, states, two padded tables, A|b rows and the two pair lists
template <int M, int G, int PD>
size_t smem_sc(const BuildParams& P) {
    using SS = ScShape<M, G, PD>;
    const int DR = P.cost_mode == 1 ? 1 : G;
    const size_t T = (size_t)P.tile;
    const size_t SF = (size_t)sc_free_stride(Shape<G, PD>::NI, M);
    size_t f = T * (2 * SS::SU + 2 * SF + 2 * SS::NS + 8) + 2 * T * (SS::XS + G) + 2 * PadTab<G, PD>::FLOATS + RMAX * 4;
    return f * sizeof(float) + 2 * T * T * sizeof(uint16_t);
}

template <int M, int G, int PD>
size_t smem_ws(const BuildParams& P) {
    using S = Shape<G, PD>;
    const int RR = M * S::RAX, FRm = S::NI * P.max_rows, CRW = G * PD * M;
    const size_t T = TILE;
    size_t f = 2 * (size_t)(2 * RR + 2 * FRm + 2 * CRW + 4) * T + 2 * T * (M * G + G) + 2 * P.L.f_stride + RMAX * (M + 1);
    return f * sizeof(float);
}

template <int M, int G, int PD>
size_t smem_f64(const BuildParams& P) {
    using S = Shape<G, PD>;
    const int RR = M * S::RAX, CRW = G * PD * M;
    size_t d = (size_t)(2 * RR + 2 * S::NI * M + 2 * CRW) * TILE64 + 2 * TILE64 * M * G + P.L.e_stride + RMAX * (M + 1) +
               S::RAX + TILE64 * TILE64;
    return d * sizeof(double) + TILE64 * TILE64 * (sizeof(uint32_t) + 1) + 16;
}

template <int M, int G, int PD, bool BF>
size_t smem_tc(const BuildParams& P) {
    using S = Shape<G, PD>;
    constexpr int N_ = M * G, KI = BF ? 16 : 8, KP = (N_ + 1 + KI - 1) / KI * KI, ESZ = BF ? 2 : 4;
    const int RR = M * S::RAX, FRm = S::NI * P.max_rows;
    const int NRp = (RR + FRm + 7) & ~7, Ncap = (2 * NRp + 15) & ~15;
    const size_t ops = (size_t)((128 * KP * ESZ + 1023) & ~1023) + (size_t)((Ncap * KP * ESZ + 1023) & ~1023);
    return ops + smem_fast<M, G, PD>(P);
}

template <int M, int G, int PD, bool BF>
int launch_tc(const BuildParams& P, cudaStream_t st, int num_sms, int ctas_per_sm, cudaEvent_t e0, cudaEvent_t e1,
              int* launches) {
    const size_t sm = smem_tc<M, G, PD, BF>(P);
    cudaFuncSetAttribute(k_pairs_tc<M, G, PD, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pairs_tc<M, G, PD, BF>, 256, sm);
    if (occ < 1) occ = 1;
    if (occ > 2) occ = 2;  // two 256-column tensor-memory allocations per SM
    if (ctas_per_sm > 0 && ctas_per_sm < occ) occ = ctas_per_sm;
    if (e0) cudaEventRecord(e0, st);
    k_pairs_tc<M, G, PD, BF><<<num_sms * occ, 256, sm, st>>>(P);
    if (e1) cudaEventRecord(e1, st);
    ++*launches;
    k_recheck<M, G, PD><<<num_sms * 8, RECHECK_THREADS, 0, st>>>(P);
    ++*launches;
    return (int)cudaGetLastError();
}

template <int M, int G, int PD>
int launch_pairs(const BuildParams& P, cudaStream_t st, int num_sms, int ctas_per_sm, cudaEvent_t e0, cudaEvent_t e1,
                 int* launches) {
    if (P.arith == PLAN_TF32 || P.arith == PLAN_BF16) {
        if constexpr (M == 2 && G == 2) {
            if (P.arith == PLAN_BF16) return launch_tc<M, G, PD, true>(P, st, num_sms, ctas_per_sm, e0, e1, launches);
            return launch_tc<M, G, PD, false>(P, st, num_sms, ctas_per_sm, e0, e1, launches);
        }
        return (int)cudaErrorInvalidValue;
    }
    if (P.arith == PLAN_F64) {
        const size_t sm = smem_f64<M, G, PD>(P);
        cudaFuncSetAttribute(k_pairs_f64<M, G, PD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pairs_f64<M, G, PD>, 256, sm);
        if (occ < 1) occ = 1;
        if (e0) cudaEventRecord(e0, st);
        k_pairs_f64<M, G, PD><<<num_sms * occ, 256, sm, st>>>(P);
        if (e1) cudaEventRecord(e1, st);
        ++*launches;
    } else if (P.pipeline == 1 && P.tile == TILE && smem_ws<M, G, PD>(P) <= 227 * 1024) {
        const size_t sm = smem_ws<M, G, PD>(P);
        cudaFuncSetAttribute(k_pairs_ws<M, G, PD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e0) cudaEventRecord(e0, st);
        k_pairs_ws<M, G, PD><<<num_sms, 512, sm, st>>>(P);
        if (e1) cudaEventRecord(e1, st);
        ++*launches;
        k_recheck<M, G, PD><<<num_sms * 8, RECHECK_THREADS, 0, st>>>(P);
        ++*launches;
    } else {
        // pipeline 0: screened kernel; 2: every pair through all rows
        const bool sc = P.pipeline != 2;
        auto kern = sc ? k_pairs_sc<M, G, PD> : k_pairs_fast<M, G, PD>;
        const size_t sm = sc ? smem_sc<M, G, PD>(P) : smem_one<M, G, PD>(P);
        int threads = (P.tile / 4) * (P.tile / 4);  // one thread per 4x4 micro-tile
        if (sc) threads = (threads + 31) & ~31;      // whole warps (warp-level list positions)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, sm);
        if (occ < 1) occ = 1;
        if (ctas_per_sm > 0 && ctas_per_sm < occ) occ = ctas_per_sm;
        if (e0) cudaEventRecord(e0, st);
        kern<<<num_sms * occ, threads, sm, st>>>(P);
        if (e1) cudaEventRecord(e1, st);
        ++*launches;
        k_recheck<M, G, PD><<<num_sms * 8, RECHECK_THREADS, 0, st>>>(P);
        ++*launches;
    }
    return (int)cudaGetLastError();
}

bool model_supported(int m, int g, int p) {
    return (m == 2 && g == 2 && (p == 3 || p == 5)) || (m == 3 && g == 3 && (p == 5 || p == 7));
}

// Tensor-core precision form: the start and end halves share one M=128 x
// N<=256 accumulator, which the 2-D models fit.
bool tc_supported(int m, int g, int p) { return m == 2 && g == 2 && (p == 3 || p == 5); }

template <int M, int G, int PD>
int launch_cost64(const BuildParams& P, cudaStream_t st, int num_sms) {
    const int DR = P.cost_mode == 1 ? 1 : G;
    const long long n = P.totN * (long long)P.maxT * 2 * PD * DR * M;
    const long long hb = (n + 255) / 256;
    k_halves64<M, G, PD><<<(unsigned)(hb < (long long)num_sms * 8 ? (hb > 0 ? hb : 1) : (long long)num_sms * 8), 256, 0, st>>>(P);
    // blocks per query: about eight two-warp CTAs per SM over the batch, at
    // least one; small CTAs spread a small graph's edges over every SM's
    // FP64 units (the CTAs past the edges exit at once)
    const int bx = (int)((long long)num_sms * 8 / P.Q > 0 ? (long long)num_sms * 8 / P.Q : 1);
    k_cost64<M, G, PD><<<dim3((unsigned)bx, (unsigned)P.Q), 64, 0, st>>>(P);
    return (int)cudaGetLastError();
}

int launch_build(const BuildParams& P, void* stream, int num_sms, int ctas_per_sm, void* ev0, void* ev1, int* launches) {
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = (cudaEvent_t)ev0, e1 = (cudaEvent_t)ev1;
    if (P.Q <= 0) return 0;
    if (P.totRows > 0) {
        k_prep<<<(unsigned)((P.totRows + 255) / 256), 256, 0, st>>>(P);
        ++*launches;
    }
    if (P.totMask > 0) {  // also writes the (zero) masks of queries without polytopes
        const long long need = (P.totMask * 32 + 255) / 256;
        k_member<<<(unsigned)(need < num_sms * 4 ? need : num_sms * 4), 256, 0, st>>>(P);
        ++*launches;
    }
    if (P.totPoly > 0) {
        k_lists<<<(unsigned)P.totPoly, 1024, 0, st>>>(P);
        ++*launches;
    }
    k_setup<<<P.Q, 1024, 0, st>>>(P);
    k_batch<<<1, 1024, 0, st>>>(P);
    *launches += 2;
    if (P.totN > 0 && P.totPoly > 0) {
        k_zero_slots<<<num_sms * 8, 256, 0, st>>>(P);
        ++*launches;
        int rc = 0;
        if (P.m == 2 && P.g == 2 && P.p == 3) rc = launch_pairs<2, 2, 3>(P, st, num_sms, ctas_per_sm, e0, e1, launches);
        else if (P.m == 2 && P.g == 2 && P.p == 5) rc = launch_pairs<2, 2, 5>(P, st, num_sms, ctas_per_sm, e0, e1, launches);
        else if (P.m == 3 && P.g == 3 && P.p == 5) rc = launch_pairs<3, 3, 5>(P, st, num_sms, ctas_per_sm, e0, e1, launches);
        else if (P.m == 3 && P.g == 3 && P.p == 7) rc = launch_pairs<3, 3, 7>(P, st, num_sms, ctas_per_sm, e0, e1, launches);
        if (rc) return rc;
    }
    if (P.totN > 0) {
        cudaMemsetAsync(P.rowCount, 0, sizeof(int) * (size_t)P.totN, st);
        if (P.totPoly > 0) {
            k_emit<<<num_sms * 16, 256, 0, st>>>(P);
            ++*launches;
        }
    }
    k_scan<<<P.Q, 1024, 0, st>>>(P);
    ++*launches;
    if (P.totN > 0 && P.totPoly > 0) {
        // staged ids and slot indices per warp (a row holds fewer than N
        // entries; rows with more than run_cap / 2 use the binary-search
        // path): at most 32 KB a CTA, so that four CTAs (the register
        // bound) fit on an SM
        const int run_cap = 2 * (P.maxN < 512 ? (P.maxN > 32 ? P.maxN : 32) : 512);
        const size_t smem = ((size_t)8 * run_cap * sizeof(int) + 1023) & ~(size_t)1023;
        const cudaError_t ea = cudaFuncSetAttribute(k_compact_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (ea != cudaSuccess) return (int)ea;
        k_compact_fill<<<num_sms * 4, 256, smem, st>>>(P, run_cap);
        ++*launches;
        if (P.cost64) {
            int rc = 0;
            if (P.m == 2 && P.g == 2 && P.p == 3) rc = launch_cost64<2, 2, 3>(P, st, num_sms);
            else if (P.m == 2 && P.g == 2 && P.p == 5) rc = launch_cost64<2, 2, 5>(P, st, num_sms);
            else if (P.m == 3 && P.g == 3 && P.p == 5) rc = launch_cost64<3, 3, 5>(P, st, num_sms);
            else if (P.m == 3 && P.g == 3 && P.p == 7) rc = launch_cost64<3, 3, 7>(P, st, num_sms);
            if (rc) return rc;
            *launches += 2;
        }
    }
    return (int)cudaGetLastError();
}

}  // namespace plan
