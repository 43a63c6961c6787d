// findPath for sm_103a (Sec. III-C, Problem 2): nearest start/goal vertices,
// then single-source shortest paths with Dijkstra's semantics, all in one
// cooperative kernel with a bounded software grid barrier.
//
// Distances are FP64 bit patterns (non-negative doubles order like unsigned
// integers), relaxed with atomicMin by frontier sweeps (Bellman-Ford).  With
// non-negative weights and round-to-nearest, fl(d + w) is monotone in d and
// >= d, so the sweep's fixed point is the minimum over paths of the
// left-to-right rounded path sum -- the same value Dijkstra produces.  The
// predecessor of v is then the in-neighbour u attaining dist[v] that Dijkstra
// (heap keyed (dist, id), strict-improvement relaxation) settles first: the
// minimum (dist[u], u).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cmath>
#include <cstring>
#include <mutex>

#include "plan_internal.h"

namespace plan {

#define DEVI __device__ __forceinline__

namespace {
constexpr unsigned long long DINF = 0x7FF0000000000000ull;

DEVI void set_status_s(DevInfo* info, int code, int detail) {
    if (atomicCAS(&info->status, 0, code) == 0) atomicExch(&info->detail, detail);
}
DEVI bool failed_s(const DevInfo* info) {
    const int s = *((volatile const int*)&info->status);
    return s != 0 && s != PLAN_ERR_NO_PATH;
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident): one
// release-add per block on a 64-bit word -- 1 for the arrival, plus 2^32 when
// the block raises its flag -- and an acquire-load poll until the low half
// counts every block; the high half then tells every block how many raised
// the flag.  Three words are used in rotation (round r uses word r mod 3):
// once round r completes, every block has left the poll of round r-1, so
// block 0 clears that word, which round r+2 uses next.  All three start at
// zero (cleared before the launch).  The spin is bounded: on expiry the block
// records PLAN_ERR_TIMEOUT and returns false instead of waiting forever; it
// also returns false when a failure was recorded before the barrier.
DEVI bool grid_sync(DevInfo* info, unsigned nblocks, long long spin_limit, int& round, bool raise = false,
                    unsigned* raised = nullptr) {
    __shared__ int s_ok;
    __shared__ unsigned s_raised;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned long long* word = &info->bar[round % 3];
        const unsigned long long inc = 1ull | (raise ? (1ull << 32) : 0ull);
        unsigned long long cur = 0;
        asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(word), "l"(inc) : "memory");
        long long it = 0;
        for (;;) {
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(cur) : "l"(word) : "memory");
            if ((unsigned)(cur & 0xffffffffull) >= nblocks) break;
            if (++it > spin_limit) {
                set_status_s(info, PLAN_ERR_TIMEOUT, DET_BARRIER);
                ok = 0;
                break;
            }
        }
        if (ok && blockIdx.x == 0) info->bar[(round + 2) % 3] = 0ull;
        if (ok && failed_s(info)) ok = 0;  // a failure recorded before the barrier stops every block
        s_ok = ok;
        s_raised = (unsigned)(cur >> 32);
    }
    __syncthreads();
    ++round;
    if (raised) *raised = s_raised;
    return s_ok != 0;
}

DEVI double ldd(const void* p, long long i, int f32) {
    return f32 ? (double)((const float*)p)[i] : ((const double*)p)[i];
}
}  // namespace

// check-and-relax rounds of the cooperative search per grid barrier
#ifndef PLAN_SEARCH_ROUNDS
#define PLAN_SEARCH_ROUNDS 4
#endif
constexpr int SWEEP_ROUNDS = PLAN_SEARCH_ROUNDS;

// A vertex's predecessor candidate: the bits of dist[u] and u, ordered
// lexicographically (the nearer in-neighbour, ties to the lower id).
struct alignas(16) DistPred {
    unsigned long long d, u;
};

// Lowers *a to (d, u) if that pair is smaller: a compare-and-swap loop that
// retries only when another thread changed *a in between (lock-free: every
// failed swap means a smaller pair was stored by someone else).
DEVI void min_dist_pred(DistPred* a, unsigned long long d, unsigned long long u) {
    const volatile unsigned long long* va = reinterpret_cast<const volatile unsigned long long*>(a);
    DistPred cur{va[0], va[1]};  // a torn read only costs one failed swap
    while (d < cur.d || (d == cur.d && u < cur.u)) {
        const DistPred want{d, u};
        const DistPred old = atomicCAS(a, cur, want);
        if (old.d == cur.d && old.u == cur.u) return;
        cur = old;
    }
}

// (bits, id) pairs ordered lexicographically: the nearest vertex, ties to the lowest id
DEVI void keep_min(unsigned long long& kb, int& ki, unsigned long long ob, int oi) {
    if (ob < kb || (ob == kb && oi < ki)) {
        kb = ob;
        ki = oi;
    }
}

// Exclusive prefix of cnt[0..n) in place (n <= blockDim.x = 1024); cnt[n] =
// the total, which is returned to every thread.
DEVI int block_scan_degrees(int* cnt, int n, int* wsum) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int x = tid < n ? cnt[tid] : 0;
    int incl = x;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        int t = lane < nw ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        wsum[lane] = t;  // inclusive per-warp totals
        if (lane == 31) wsum[32] = t;
    }
    __syncthreads();
    const int excl = incl - x + (wid > 0 ? wsum[wid - 1] : 0);
    if (tid < n) cnt[tid] = excl;
    if (tid == 0) cnt[n] = wsum[32];
    __syncthreads();
    return cnt[n];
}

// Largest i in [0, n) with pre[i] <= q (pre strictly increasing: every listed
// vertex has at least one out-edge).
DEVI int find_entry(const int* pre, int n, int q) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= q) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The search kernel launches one 1024-thread block per SM.  Phases:
//   0. every block initialises its share of the per-vertex arrays and finds
//      its nearest candidates for the start and goal; after one grid barrier
//      every block reduces the candidates of all blocks itself;
//   1. frontier sweeps.  A vertex is on the frontier when its distance is
//      below the value it last relaxed its out-edges from (kept in last[]),
//      so no frontier flags are written or read.  The sweep that relaxes
//      nothing ends the loop;
//   2. predecessors in two passes (minimum dist[u], then minimum u);
//   3. block 0 stages pred[] in shared memory and walks goal -> start.
__global__ void __launch_bounds__(1024, 1) k_search(SearchParams P) {
    extern __shared__ int s_pred[];
    __shared__ unsigned long long s_kb[2][32];
    __shared__ int s_ki[2][32];
    __shared__ int s_nf;                        // listed vertices of this round
    __shared__ unsigned long long s_gd;         // the goal's distance as this block last read it
    __shared__ int s_v[1024], s_e0[1024];       // vertex, first out-edge
    __shared__ int s_pre[1025];                 // out-degree, then its exclusive prefix
    __shared__ unsigned long long s_dv[1024];   // distance the vertex relaxes from
    __shared__ int s_wsum[33];
    __shared__ int s_ro[2 * SEARCH_OWN_CAP];                   // out-edge range of owned vertex k
    __shared__ unsigned long long s_last[SEARCH_OWN_CAP];      // distance it last relaxed from
    const unsigned nb = gridDim.x;
    int bar_round = 0;
    const long long gtid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    DevInfo* info = P.info;
    const int N = P.N;

    // phase 0: per-vertex arrays; every block's nearest candidates (A6:
    // canonical FP64 squared distance summed left to right, ties to the
    // lowest id) go to near_blk, and after the barrier every block reduces
    // them to the same start and goal
    if (gtid == 0) {
        const long long E = *P.count;
        if (E < 0 || E > P.cap) set_status_s(info, PLAN_ERR_INVALID_ARG, DET_OUTPUT);
    }
    const int tid = threadIdx.x, nt = blockDim.x;
    const long long nown = N > (int)blockIdx.x ? (N - 1 - (long long)blockIdx.x) / nb + 1 : 0;  // owned vertices
    const int ncache = (int)(nown < SEARCH_OWN_CAP ? nown : SEARCH_OWN_CAP);
    for (int k = tid; k < ncache; k += nt) {
        const long long v = blockIdx.x + (long long)k * nb;
        s_ro[2 * k] = __ldg(&P.row_off[v]);
        s_ro[2 * k + 1] = __ldg(&P.row_off[v + 1]);
        s_last[k] = DINF;
    }
    unsigned long long kb[2] = {~0ull, ~0ull};
    int ki[2] = {0x7fffffff, 0x7fffffff};
    double spos[4], gpos[4];
    for (int a = 0; a < 4; ++a) {
        spos[a] = P.endpoints ? (a < P.m ? P.endpoints[a] : 0.0) : P.start[a];
        gpos[a] = P.endpoints ? (a < P.m ? P.endpoints[P.m + a] : 0.0) : P.goal[a];
    }
    for (long long k = tid; k < nown; k += nt) {  // owned vertices: the FP64 work spreads over every SM
        const long long v = blockIdx.x + k * nb;
        P.dist[v] = DINF;
        P.last[v] = DINF;
        if (P.best16) {
            P.best16[2 * v] = ~0ull;
            P.best16[2 * v + 1] = ~0ull;
        } else {
            P.bestU[v] = ~0ull;
            P.pred[v] = 0x7fffffff;
        }
        double ds = 0.0, dg = 0.0;
        for (int a = 0; a < P.m; ++a) {
            const double x = ldd(P.states, v * P.n + a, P.in_f32);
            const double ts = __dsub_rn(x, spos[a]);
            const double tg = __dsub_rn(x, gpos[a]);
            ds = __dadd_rn(ds, __dmul_rn(ts, ts));
            dg = __dadd_rn(dg, __dmul_rn(tg, tg));
        }
        keep_min(kb[0], ki[0], (unsigned long long)__double_as_longlong(ds), (int)v);
        keep_min(kb[1], ki[1], (unsigned long long)__double_as_longlong(dg), (int)v);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ob = __shfl_down_sync(0xffffffffu, kb[h], o);
            const int oi = __shfl_down_sync(0xffffffffu, ki[h], o);
            keep_min(kb[h], ki[h], ob, oi);
        }
        if (lane == 0) {
            s_kb[h][wid] = kb[h];
            s_ki[h][wid] = ki[h];
        }
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        const int h = threadIdx.x;
        unsigned long long b0 = ~0ull;
        int i0 = 0x7fffffff;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) keep_min(b0, i0, s_kb[h][w], s_ki[h][w]);
        P.near_blk[4 * blockIdx.x + 2 * h] = b0;
        P.near_blk[4 * blockIdx.x + 2 * h + 1] = (unsigned long long)(unsigned)i0;
    }
    if (!grid_sync(info, nb, P.spin_limit, bar_round)) return;
    if (threadIdx.x < 64) {  // warp 0: start (h = 0) from lanes' blocks; warp 1: goal
        const int h = threadIdx.x >> 5;
        unsigned long long b0 = ~0ull;
        int i0 = 0x7fffffff;
        volatile unsigned long long* nbk = P.near_blk;
        for (unsigned q = lane; q < nb; q += 32) keep_min(b0, i0, nbk[4 * q + 2 * h], (int)nbk[4 * q + 2 * h + 1]);
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ob = __shfl_down_sync(0xffffffffu, b0, o);
            const int oi = __shfl_down_sync(0xffffffffu, i0, o);
            keep_min(b0, i0, ob, oi);
        }
        if (lane == 0) {
            s_ki[h][0] = i0;
            if (blockIdx.x == 0) {
                info->near_d[h] = b0;
                if (h == 0) info->start = i0;
                else info->goal = i0;
            }
        }
    }
    __syncthreads();
    const int s = s_ki[0][0], g = s_ki[1][0];
    if (s < 0 || s >= N || g < 0 || g >= N) {
        if (gtid == 0) set_status_s(info, PLAN_ERR_INVALID_ARG, DET_WALK);
        return;
    }

    // phase 1 (A7).  Block b owns the vertices b, b + B, b + 2B, ... (B =
    // blocks), so that vertices with neighbouring ids -- often neighbours in
    // the graph, hence on the frontier together -- land in different blocks.
    // Per round of up to 1024 owned vertices: each thread checks one vertex
    // (on the frontier when its distance is below last[v]); the block lists
    // the frontier vertices with their out-degrees, scans the degrees, and
    // then relaxes the listed out-edges edge-parallel (thread q takes edge q
    // of the concatenated lists, found by binary search), with
    // non-returning atomicMin.
    // A vertex whose distance is not below the goal's current distance does
    // not relax its out-edges: nothing reached through it can improve a
    // vertex closer than the goal (weights are non-negative), and those --
    // every vertex of a shortest path to the goal and its predecessors -- are
    // exactly what the path needs (Dijkstra stops once the goal is settled).
    volatile unsigned long long* vdist = P.dist;
    int it = 0;
    for (;;) {
        bool relaxed = false;  // block-uniform
        // SWEEP_ROUNDS check-and-relax rounds per barrier: the later rounds
        // pick up what other blocks relaxed meanwhile
        for (int rep = 0; rep < SWEEP_ROUNDS; ++rep)
        for (long long k0 = 0; k0 < nown; k0 += nt) {
            if (tid == 0) {
                s_nf = 0;
                s_gd = vdist[g];  // one read per block: same-address reads queue at one L2 slice
            }
            __syncthreads();
            const long long k = k0 + tid;
            const unsigned long long gd = s_gd;
            if (k < nown) {
                const long long v = blockIdx.x + k * nb;
                const bool cached = k < SEARCH_OWN_CAP;
                const unsigned long long dvb = v == s ? 0ull : vdist[v];
                if (dvb < (cached ? s_last[k] : P.last[v]) && dvb < gd) {
                    if (cached) s_last[k] = dvb;
                    else P.last[v] = dvb;
                    if (v == s) vdist[v] = 0ull;
                    const int e0 = cached ? s_ro[2 * k] : __ldg(&P.row_off[v]);
                    const int e1 = cached ? s_ro[2 * k + 1] : __ldg(&P.row_off[v + 1]);
                    if (e1 > e0) {
                        const int i = atomicAdd(&s_nf, 1);
                        s_v[i] = (int)v;
                        s_e0[i] = e0;
                        s_pre[i] = e1 - e0;
                        s_dv[i] = dvb;
                    }
                }
            }
            __syncthreads();
            const int nf = s_nf;
            if (nf == 0) continue;
            relaxed = true;
            const int tot = block_scan_degrees(s_pre, nf, s_wsum);
            // four edges per thread per pass: their loads are issued together
            for (int q0 = tid; q0 < tot; q0 += 4 * nt) {
                int uu[4], ei[4];
                double ww[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int q = q0 + c * nt;
                    uu[c] = -1;
                    ei[c] = 0;
                    ww[c] = 0.0;
                    if (q < tot) {
                        const int i = find_entry(s_pre, nf, q);
                        const int e = s_e0[i] + (q - s_pre[i]);
                        ei[c] = i;
                        uu[c] = __ldg(&P.col[e]);
                        ww[c] = P.w_f64 ? __ldg(&((const double*)P.w)[e]) : (double)__ldg(&((const float*)P.w)[e]);
                    }
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (uu[c] < 0 || uu[c] >= N) continue;
                    const double dv = __longlong_as_double((long long)s_dv[ei[c]]);
                    atomicMin(&P.dist[uu[c]], (unsigned long long)__double_as_longlong(__dadd_rn(dv, ww[c])));
                }
            }
            __syncthreads();  // the lists are rebuilt by the next round
        }
        // the barrier counts the blocks that relaxed: none means a fixed point
        unsigned nrelaxed = 0;
        if (!grid_sync(info, nb, P.spin_limit, bar_round, relaxed, &nrelaxed)) return;
        ++it;
        if (nrelaxed == 0) break;
        if (it > P.max_sweeps) {
            if (gtid == 0) set_status_s(info, PLAN_ERR_TIMEOUT, DET_SWEEPS);
            return;
        }
    }

    // phase 2: predecessor = minimum (dist[u], u) over in-neighbours attaining
    // dist[v], over the out-edges of every vertex closer than the goal (the
    // only possible predecessors on a path to it; same ownership and
    // edge-parallel layout as the sweeps): one pass of 16-byte lexicographic
    // minima when best16 is given, else two passes (minimum dist[u], then
    // minimum u among those attaining it)
    if (tid == 0) s_gd = vdist[g];
    __syncthreads();
    const unsigned long long dgoal = s_gd;
    const int npass = P.best16 ? 1 : 2;
    for (int pass = 0; pass < npass; ++pass) {
        for (long long k0 = 0; k0 < nown; k0 += nt) {
            if (tid == 0) s_nf = 0;
            __syncthreads();
            const long long k = k0 + tid;
            if (k < nown) {
                const long long v = blockIdx.x + k * nb;
                const bool cached = k < SEARCH_OWN_CAP;
                const unsigned long long dvb = vdist[v];
                const int e0 = cached ? s_ro[2 * k] : __ldg(&P.row_off[v]);
                const int e1 = cached ? s_ro[2 * k + 1] : __ldg(&P.row_off[v + 1]);
                if (dvb < dgoal && e1 > e0) {
                    const int i = atomicAdd(&s_nf, 1);
                    s_v[i] = (int)v;
                    s_e0[i] = e0;
                    s_pre[i] = e1 - e0;
                    s_dv[i] = dvb;
                }
            }
            __syncthreads();
            const int nf = s_nf;
            if (nf == 0) continue;
            const int tot = block_scan_degrees(s_pre, nf, s_wsum);
            for (int q = tid; q < tot; q += nt) {
                const int i = find_entry(s_pre, nf, q);
                const int e = s_e0[i] + (q - s_pre[i]);
                const int u = __ldg(&P.col[e]);
                if (u < 0 || u >= N || u == s) continue;
                const double w = P.w_f64 ? __ldg(&((const double*)P.w)[e]) : (double)__ldg(&((const float*)P.w)[e]);
                const unsigned long long dvb = s_dv[i];
                const unsigned long long nd =
                    (unsigned long long)__double_as_longlong(__dadd_rn(__longlong_as_double((long long)dvb), w));
                if (nd != vdist[u]) continue;
                if (P.best16) min_dist_pred(reinterpret_cast<DistPred*>(P.best16 + 2LL * u), dvb, (unsigned long long)s_v[i]);
                else if (pass == 0) atomicMin(&P.bestU[u], dvb);
                else if (((volatile unsigned long long*)P.bestU)[u] == dvb) atomicMin(&P.pred[u], s_v[i]);
            }
            __syncthreads();
        }
        if (!grid_sync(info, nb, P.spin_limit, bar_round)) return;
    }

    // phase 3: walk goal -> start (block 0; pred[] staged in shared memory when it fits)
    if (blockIdx.x != 0) return;
    const bool staged = N <= P.walk_smem;
    if (staged) {
        for (int v = threadIdx.x; v < N; v += blockDim.x)
            s_pred[v] = P.best16 ? (int)((volatile unsigned long long*)P.best16)[2 * v + 1] : ((volatile int*)P.pred)[v];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // the predecessor of v (an unset one reads as -1 or INT_MAX, out of range)
        auto pr = [&](int v) -> int {
            if (staged) return s_pred[v];
            return P.best16 ? (int)P.best16[2LL * v + 1] : P.pred[v];
        };
        info->search_iters = (unsigned long long)it;
        const unsigned long long dg = vdist[g];
        if (dg >= DINF) {
            *P.path_len = 0;
            *P.cost = __longlong_as_double((long long)DINF);
            set_status_s(info, PLAN_ERR_NO_PATH, DET_NONE);
        } else {
            int len = 1, v = g;
            bool okw = true;
            while (v != s) {
                v = pr(v);
                if (v < 0 || v >= N || len > N) {
                    okw = false;
                    break;
                }
                ++len;
            }
            if (!okw) {
                set_status_s(info, PLAN_ERR_INVALID_ARG, DET_WALK);
                *P.path_len = 0;
            } else if (len > P.path_cap) {
                set_status_s(info, PLAN_ERR_CAPACITY, DET_PATHCAP);
                *P.path_len = len;
            } else {
                v = g;
                for (int q = len - 1; q >= 0; --q) {
                    P.path[q] = v;
                    if (q) v = pr(v);
                }
                *P.path_len = len;
            }
            *P.cost = __longlong_as_double((long long)dg);
        }
        info->path_len = *P.path_len;
    }
}

// ---------------------------------------------------------------------------
// Batched search: one 1024-thread CTA per query; the same phases as k_search
// with block barriers in place of the grid barrier.  Per-query status: OK,
// NO_PATH (path_len 0, cost +inf), CAPACITY (path longer than path_cap;
// path_len = the length needed), TIMEOUT (sweep bound), INVALID_ARG.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_search_batched(BatchSearchParams B) {
    const SearchQueryDesc& Q = B.qd[blockIdx.x];
    const int N = Q.N;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    unsigned long long* dist = B.dist + Q.off;
    unsigned long long* best = B.bestU + Q.off;
    int* pred = B.pred + Q.off;
    unsigned char* front = B.front + 2 * Q.off;
    __shared__ unsigned long long s_nd[2];
    __shared__ int s_id[2];
    __shared__ int s_changed;
    __shared__ int s_bad;
    if (tid == 0) {
        s_nd[0] = s_nd[1] = ~0ull;
        s_id[0] = s_id[1] = 0x7fffffff;
        s_bad = 0;
        const long long E = *Q.count;
        if (N < 1 || E < 0 || E > Q.cap) s_bad = 1;
    }
    for (int v = tid; v < N; v += blockDim.x) {
        dist[v] = DINF;
        best[v] = ~0ull;
        pred[v] = 0x7fffffff;
        front[v] = 0;
        front[N + v] = 0;
    }
    __syncthreads();
    if (s_bad) {
        if (tid == 0) {
            *Q.status = PLAN_ERR_INVALID_ARG;
            if (N >= 1) *Q.path_len = 0;
        }
        return;
    }
    for (int pass = 0; pass < 2; ++pass) {
        for (int v = tid; v < N; v += blockDim.x) {
            double ds = 0.0, dg = 0.0;
            for (int a = 0; a < B.m; ++a) {
                const double x = ldd(Q.states, (long long)v * B.n + a, B.in_f32);
                const double ts = __dsub_rn(x, Q.start[a]);
                const double tg = __dsub_rn(x, Q.goal[a]);
                ds = __dadd_rn(ds, __dmul_rn(ts, ts));
                dg = __dadd_rn(dg, __dmul_rn(tg, tg));
            }
            const unsigned long long bs = (unsigned long long)__double_as_longlong(ds);
            const unsigned long long bg = (unsigned long long)__double_as_longlong(dg);
            if (pass == 0) {
                atomicMin(&s_nd[0], bs);
                atomicMin(&s_nd[1], bg);
            } else {
                if (bs == s_nd[0]) atomicMin(&s_id[0], v);
                if (bg == s_nd[1]) atomicMin(&s_id[1], v);
            }
        }
        __syncthreads();
    }
    const int s = s_id[0], g = s_id[1];
    if (tid == 0) {
        dist[s] = 0ull;
        front[s] = 1;
    }
    int cur = 0, it = 0;
    volatile unsigned long long* vdist = dist;
    for (;;) {
        if (tid == 0) s_changed = 0;
        __syncthreads();
        bool my_change = false;
        const unsigned long long gd = vdist[g];   // vertices not closer than the goal do not relax
        for (int v = wid; v < N; v += nw) {
            if (!front[cur * N + v]) continue;
            __syncwarp();
            if (lane == 0) front[cur * N + v] = 0;
            if (vdist[v] >= gd) continue;
            const double dv = __longlong_as_double((long long)vdist[v]);
            const long long e0 = Q.row_off[v], e1 = Q.row_off[v + 1];
            for (long long e = e0 + lane; e < e1; e += 32) {
                const int u = Q.col[e];
                if (u < 0 || u >= N) continue;
                const double w = B.w_f64 ? ((const double*)Q.w)[e] : (double)((const float*)Q.w)[e];
                const unsigned long long nd = (unsigned long long)__double_as_longlong(__dadd_rn(dv, w));
                const unsigned long long old = atomicMin(&dist[u], nd);
                if (nd < old) {
                    front[(cur ^ 1) * N + u] = 1;
                    my_change = true;
                }
            }
        }
        if (__any_sync(0xffffffffu, my_change) && lane == 0) s_changed = 1;
        __syncthreads();
        const int ch = s_changed;
        ++it;
        if (!ch) break;
        if (it > B.max_sweeps) {
            if (tid == 0) {
                *Q.status = PLAN_ERR_TIMEOUT;
                *Q.path_len = 0;
            }
            return;
        }
        cur ^= 1;
        __syncthreads();
    }
    const unsigned long long dgoal = vdist[g];
    for (int pass = 0; pass < 2; ++pass) {
        for (int v = wid; v < N; v += nw) {
            const unsigned long long dvb = vdist[v];
            if (dvb >= dgoal) continue;   // only vertices closer than the goal can precede path vertices
            const double dv = __longlong_as_double((long long)dvb);
            const long long e0 = Q.row_off[v], e1 = Q.row_off[v + 1];
            for (long long e = e0 + lane; e < e1; e += 32) {
                const int u = Q.col[e];
                if (u < 0 || u >= N || u == s) continue;
                const double w = B.w_f64 ? ((const double*)Q.w)[e] : (double)((const float*)Q.w)[e];
                const unsigned long long nd = (unsigned long long)__double_as_longlong(__dadd_rn(dv, w));
                if (nd != vdist[u]) continue;
                if (pass == 0) atomicMin(&best[u], dvb);
                else if (best[u] == dvb) atomicMin(&pred[u], v);
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        const unsigned long long dg = vdist[g];
        int st = PLAN_OK;
        if (dg >= DINF) {
            *Q.path_len = 0;
            *Q.cost = __longlong_as_double((long long)DINF);
            st = PLAN_ERR_NO_PATH;
        } else {
            int len = 1, v = g;
            bool okw = true;
            while (v != s) {
                v = pred[v];
                if (v < 0 || v >= N || len > N) {
                    okw = false;
                    break;
                }
                ++len;
            }
            if (!okw) {
                st = PLAN_ERR_INVALID_ARG;
                *Q.path_len = 0;
            } else if (len > Q.path_cap) {
                st = PLAN_ERR_CAPACITY;
                *Q.path_len = len;
            } else {
                v = g;
                for (int q = len - 1; q >= 0; --q) {
                    Q.path[q] = v;
                    if (q) v = pred[v];
                }
                *Q.path_len = len;
            }
            *Q.cost = __longlong_as_double((long long)dg);
        }
        *Q.status = st;
        atomicAdd(&B.info->search_iters, (unsigned long long)it);
    }
}

// ---------------------------------------------------------------------------
// Goal-rooted search with a warm start (the replanning loop of Algorithm 1:
// findPath every tick on a graph that changes only where obstacles moved;
// Sec. III-C distances and path).  One cooperative launch, one 1024-thread block per SM.
//
// d[u] = distance from u to the goal vertex: the fixed point of
// d[u] = min over out-edges (u -> v) of fl(w + d[v]), d[goal] = 0, reached by
// pull sweeps over the out-edges (no reverse graph); succ[u] = the
// out-neighbour minimising (w + d[v], v).  With non-negative weights fl(w + x)
// is monotone in x and >= x, so iterating from +inf converges to the greatest
// fixed point, the minimum over paths of the right-to-left rounded path sum.
//
// Warm start: when the goal vertex and N are those of the previous call, a
// vertex keeps its previous d when its successor chain to the goal still
// exists with weights no larger than before; every other vertex restarts from
// +inf.  A kept value was fl(old weight + old d of the successor) down the
// whole chain, so it is at least the new chain's rounded sum, an upper bound
// of the new fixed point; iterating the monotone sweep from any upper bound
// reaches the same greatest fixed point, so the result equals a cold start and
// only the number of sweeps changes.  The chains are checked by pointer
// jumping (log rounds) on links packed as anc | ok << 31.  A call that stops
// early leaves no warm state behind.
//
// Phases:
//   0. every thread takes vertices v = gtid, gtid + threads, ...: nearest
//      start/goal candidates and, when a warm start is possible, the link of v
//      (ok when the out-edge (v, succ[v]) is still in v's row -- rows sorted by
//      column, binary search -- with a weight <= the kept one and d[v] finite;
//      the previous goal is its own ok ancestor);  grid barrier;
//   1. every block reduces the candidates; warm start: pointer jumping in each
//      block's shared memory (N <= TO_SMEM_N; else in global memory, one grid
//      barrier per round) and d reset off the valid chains; cold: d = +inf,
//      d[goal] = 0;  grid barrier;
//   2. sweeps: one warp per vertex u (u = warp, warp + warps, ...), lanes over
//      u's out-edges; each lane keeps its first edge of its first TO_KC
//      vertices in registers across sweeps; grid barrier per sweep, whose
//      raised count says whether any block lowered a distance;
//   3. successors, same layout;  grid barrier;
//   4. block 0 walks start -> goal along succ.
// ---------------------------------------------------------------------------
constexpr int TO_KC = 2;            // owned vertices per warp held in registers
constexpr int TO_CLUSTER_MAX_N = 12288;   // on-chip variant (one cluster) up to this N
constexpr int TO_SMEM_N = 24576;    // pointer jumping in shared memory up to this N (8 bytes a vertex)
constexpr unsigned TO_OK = 0x80000000u;

namespace {
DEVI double ldw(const GoalSearchParams& G, long long e) {
    return G.w_f64 ? __ldg(&((const double*)G.w)[e]) : (double)__ldg(&((const float*)G.w)[e]);
}

// (c, v, w) lexicographic minimum (successor choice; w only breaks exact ties of duplicate columns)
DEVI void keep_succ(double& c, int& v, double& w, double oc, int ov, double ow) {
    if (oc < c || (oc == c && (ov < v || (ov == v && ow < w)))) {
        c = oc;
        v = ov;
        w = ow;
    }
}

// One pointer-jumping round over v = begin, begin + step, ... on packed links.
template <bool GLOBAL>
DEVI int jump_round(const unsigned* a0, unsigned* a1, int begin, int step, int N) {
    int changed = 0;
    for (int v = begin; v < N; v += step) {
        const unsigned x = GLOBAL ? ((const volatile unsigned*)a0)[v] : a0[v];
        const int a = (int)(x & ~TO_OK);
        const unsigned y = GLOBAL ? ((const volatile unsigned*)a0)[a] : a0[a];
        const unsigned z = (y & ~TO_OK) | (x & y & TO_OK);
        if (GLOBAL) ((volatile unsigned*)a1)[v] = z;
        else a1[v] = z;
        changed |= z != x;
    }
    return changed;
}
}  // namespace

__global__ void __launch_bounds__(1024, 1) k_search_to(GoalSearchParams G) {
    extern __shared__ unsigned s_link[];   // [2][N] packed links (warm start, N <= TO_SMEM_N)
    __shared__ unsigned long long s_kb[2][32];
    __shared__ int s_ki[2][32];
    __shared__ int s_prev[2];
    const int N = G.N, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const unsigned nb = gridDim.x;
    const int nthreads = (int)(nb * blockDim.x), gtid = (int)(blockIdx.x * blockDim.x) + tid;
    const int nwarps = (int)(nb * (blockDim.x >> 5)), gw = gtid >> 5;
    DevInfo* info = G.info;
    int bar_round = 0;
    const double inf = __longlong_as_double(DINF);
    if (gtid == 0) {
        const long long E = *G.count;
        if (E < 0 || E > G.cap) set_status_s(info, PLAN_ERR_INVALID_ARG, DET_OUTPUT);
    }
    if (tid == 0) {
        s_prev[0] = ((volatile int*)G.prev)[0];
        s_prev[1] = ((volatile int*)G.prev)[1];
    }
    __syncthreads();
    const int pg = s_prev[0];
    const bool may_warm = G.warm && s_prev[1] == N && pg >= 0 && pg < N;

    // phase 0
    double sp[4], gp[4];
    for (int a = 0; a < 4; ++a) {
        sp[a] = a < G.m ? G.endpoints[a] : 0.0;
        gp[a] = a < G.m ? G.endpoints[G.m + a] : 0.0;
    }
    unsigned long long kb[2] = {~0ull, ~0ull};
    int ki[2] = {0x7fffffff, 0x7fffffff};
    for (int v = gtid; v < N; v += nthreads) {
        double ds = 0.0, dg = 0.0;
        for (int a = 0; a < G.m; ++a) {
            const double x = ldd(G.states, (long long)v * G.n + a, G.in_f32);
            const double ts = __dsub_rn(x, sp[a]), tg = __dsub_rn(x, gp[a]);
            ds = __dadd_rn(ds, __dmul_rn(ts, ts));
            dg = __dadd_rn(dg, __dmul_rn(tg, tg));
        }
        keep_min(kb[0], ki[0], (unsigned long long)__double_as_longlong(ds), v);
        keep_min(kb[1], ki[1], (unsigned long long)__double_as_longlong(dg), v);
        if (may_warm) {
            unsigned link = (unsigned)v;
            if (v == pg) {
                link |= TO_OK;
            } else {
                const int sv = G.succ[v];
                if (sv >= 0 && sv < N && G.d[v] < inf) {
                    const int r1 = __ldg(&G.row_off[v + 1]);
                    int lo = __ldg(&G.row_off[v]), hi = r1;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (__ldg(&G.col[mid]) < sv) lo = mid + 1;
                        else hi = mid;
                    }
                    if (lo < r1 && __ldg(&G.col[lo]) == sv && ldw(G, lo) <= G.wsucc[v]) link = (unsigned)sv | TO_OK;
                }
            }
            G.anc[v] = link;
        }
    }
    for (int h = 0; h < 2; ++h) {
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ob = __shfl_down_sync(0xffffffffu, kb[h], o);
            const int oi = __shfl_down_sync(0xffffffffu, ki[h], o);
            keep_min(kb[h], ki[h], ob, oi);
        }
        if (lane == 0) {
            s_kb[h][wid] = kb[h];
            s_ki[h][wid] = ki[h];
        }
    }
    __syncthreads();
    if (tid < 2) {
        unsigned long long b0 = ~0ull;
        int i0 = 0x7fffffff;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) keep_min(b0, i0, s_kb[tid][w], s_ki[tid][w]);
        G.near_blk[4 * blockIdx.x + 2 * tid] = b0;
        G.near_blk[4 * blockIdx.x + 2 * tid + 1] = (unsigned long long)(unsigned)i0;
    }
    if (!grid_sync(info, nb, G.spin_limit, bar_round)) return;

    // phase 1
    if (tid < 64) {  // warp 0: start over the blocks' candidates; warp 1: goal
        const int h = tid >> 5;
        unsigned long long b0 = ~0ull;
        int i0 = 0x7fffffff;
        volatile unsigned long long* nbk = G.near_blk;
        for (unsigned q = lane; q < nb; q += 32) keep_min(b0, i0, nbk[4 * q + 2 * h], (int)nbk[4 * q + 2 * h + 1]);
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ob = __shfl_down_sync(0xffffffffu, b0, o);
            const int oi = __shfl_down_sync(0xffffffffu, i0, o);
            keep_min(b0, i0, ob, oi);
        }
        if (lane == 0) s_ki[h][0] = i0;
    }
    __syncthreads();
    const int start = s_ki[0][0], goal = s_ki[1][0];
    if (start < 0 || start >= N || goal < 0 || goal >= N) {
        if (gtid == 0) set_status_s(info, PLAN_ERR_INVALID_ARG, DET_WALK);
        return;
    }
    if (gtid == 0) ((volatile int*)G.prev)[0] = -1;  // d and succ are consistent again only when this call completes
    const bool warm = may_warm && pg == goal;
    if (warm) {
        const unsigned* fin;
        if (N <= TO_SMEM_N) {
            unsigned* a0 = s_link;
            unsigned* a1 = s_link + N;
            for (int v = tid; v < N; v += blockDim.x) a0[v] = ((const volatile unsigned*)G.anc)[v];
            __syncthreads();
            for (int r = 0; r < 64; ++r) {
                const int any = __syncthreads_or(jump_round<false>(a0, a1, tid, blockDim.x, N));
                unsigned* t = a0;
                a0 = a1;
                a1 = t;
                if (!any) break;
            }
            fin = a0;
        } else {
            unsigned* a0 = (unsigned*)G.anc;
            unsigned* a1 = (unsigned*)G.anc + N;
            for (int r = 0; r < 64; ++r) {
                const int ch = __syncthreads_or(jump_round<true>(a0, a1, gtid, nthreads, N));
                unsigned nraised = 0;
                if (!grid_sync(info, nb, G.spin_limit, bar_round, ch != 0, &nraised)) return;
                unsigned* t = a0;
                a0 = a1;
                a1 = t;
                if (nraised == 0) break;
            }
            fin = a0;
        }
        const bool shared_fin = N <= TO_SMEM_N;
        for (int v = gtid; v < N; v += nthreads) {
            const unsigned x = shared_fin ? fin[v] : ((const volatile unsigned*)fin)[v];
            if (v == goal) G.d[v] = 0.0;
            else if (x != ((unsigned)goal | TO_OK)) G.d[v] = inf;
        }
    } else {
        for (int v = gtid; v < N; v += nthreads) G.d[v] = v == goal ? 0.0 : inf;
    }
    if (!grid_sync(info, nb, G.spin_limit, bar_round)) return;

    // phase 2: sweeps
    volatile double* d = G.d;
    int r_e1[TO_KC], r_col[TO_KC], r_next[TO_KC];
    double r_w[TO_KC];
#pragma unroll
    for (int k = 0; k < TO_KC; ++k) {
        const int u = gw + k * nwarps;
        r_col[k] = -1;
        r_w[k] = 0.0;
        r_e1[k] = 0;
        r_next[k] = 0;
        if (u < N) {
            const int e0 = __ldg(&G.row_off[u]);
            r_e1[k] = __ldg(&G.row_off[u + 1]);
            r_next[k] = e0 + 32 + lane;
            if (e0 + lane < r_e1[k]) {
                r_col[k] = __ldg(&G.col[e0 + lane]);
                r_w[k] = ldw(G, e0 + lane);
            }
        }
    }
    int sweeps = 0;
    for (;;) {
        if (sweeps >= G.max_sweeps) {
            if (gtid == 0) set_status_s(info, PLAN_ERR_TIMEOUT, DET_SWEEPS);
            return;
        }
        ++sweeps;
        int changed = 0;
        for (int k = 0, u = gw; u < N; ++k, u += nwarps) {
            double best = inf;
            int e = 0, e1 = 0;
            if (k < TO_KC) {
                int c = -1;
                double w = 0.0;
#pragma unroll
                for (int q = 0; q < TO_KC; ++q)
                    if (q == k) {
                        c = r_col[q];
                        w = r_w[q];
                        e = r_next[q];
                        e1 = r_e1[q];
                    }
                if (c >= 0 && c < N) best = __dadd_rn(w, d[c]);
            } else {
                e = __ldg(&G.row_off[u]) + lane;
                e1 = __ldg(&G.row_off[u + 1]);
            }
            for (; e < e1; e += 32) {
                const int c = __ldg(&G.col[e]);
                if (c < 0 || c >= N) continue;
                const double x = __dadd_rn(ldw(G, e), d[c]);
                if (x < best) best = x;
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double y = __shfl_xor_sync(0xffffffffu, best, o);
                if (y < best) best = y;
            }
            if (lane == 0 && u != goal && best < d[u]) {
                d[u] = best;
                changed = 1;
            }
        }
        const int ch = __syncthreads_or(changed);
        unsigned nraised = 0;
        if (!grid_sync(info, nb, G.spin_limit, bar_round, ch != 0, &nraised)) return;
        if (nraised == 0) break;
    }

    // phase 3: successors (ties to the lowest id) for the path and the next warm start
    for (int k = 0, u = gw; u < N; ++k, u += nwarps) {
        double bc = inf, bw = 0.0;
        int bv = 0x7fffffff;
        if (u != goal) {
            int e = 0, e1 = 0;
            if (k < TO_KC) {
                int c = -1;
                double w = 0.0;
#pragma unroll
                for (int q = 0; q < TO_KC; ++q)
                    if (q == k) {
                        c = r_col[q];
                        w = r_w[q];
                        e = r_next[q];
                        e1 = r_e1[q];
                    }
                if (c >= 0 && c < N) keep_succ(bc, bv, bw, __dadd_rn(w, d[c]), c, w);
            } else {
                e = __ldg(&G.row_off[u]) + lane;
                e1 = __ldg(&G.row_off[u + 1]);
            }
            for (; e < e1; e += 32) {
                const int c = __ldg(&G.col[e]);
                if (c < 0 || c >= N) continue;
                const double w = ldw(G, e);
                keep_succ(bc, bv, bw, __dadd_rn(w, d[c]), c, w);
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double oc = __shfl_xor_sync(0xffffffffu, bc, o);
            const int ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const double ow = __shfl_xor_sync(0xffffffffu, bw, o);
            keep_succ(bc, bv, bw, oc, ov, ow);
        }
        if (lane == 0) {
            G.succ[u] = bc < inf ? bv : -1;
            G.wsucc[u] = bc < inf ? bw : 0.0;
        }
    }
    if (!grid_sync(info, nb, G.spin_limit, bar_round)) return;

    // phase 4: the path (block 0, thread 0)
    if (gtid == 0) {
        const volatile int* succ = G.succ;
        info->start = start;
        info->goal = goal;
        info->search_iters = (unsigned long long)sweeps;
        const double ds = d[start];
        if (!(ds < inf)) {
            *G.path_len = 0;
            *G.cost = inf;
            set_status_s(info, PLAN_ERR_NO_PATH, DET_NONE);
        } else {
            int v = start, L = 0;
            bool ok = true;
            for (;;) {
                if (L < G.path_cap) G.path[L] = v;
                ++L;
                if (v == goal) break;
                v = succ[v];
                if (v < 0 || v >= N || L > N) {
                    ok = false;
                    break;
                }
            }
            *G.path_len = L;
            *G.cost = ds;
            if (!ok) set_status_s(info, PLAN_ERR_TIMEOUT, DET_WALK);
            else if (L > G.path_cap) set_status_s(info, PLAN_ERR_CAPACITY, DET_PATHCAP);
        }
        info->path_len = *G.path_len;
        ((volatile int*)G.prev)[1] = N;
        __threadfence();
        ((volatile int*)G.prev)[0] = goal;
    }
}

// ---------------------------------------------------------------------------
// The same goal-rooted search on chip, for graphs whose distances and rows fit
// in the shared memory of one thread-block cluster (replanning graphs of some
// thousands of vertices).  A dependent L2 round trip costs about 2 us on this
// part and a software grid barrier about 1.3 us, against about 0.3 us for the
// cluster barrier and tens of cycles for a shared-memory load, so every sweep
// stays inside the cluster:
//   - CTA r of the cluster owns the vertices [r V, (r+1) V), V = ceil(N / C),
//     and holds their rows (columns, weights) in its shared memory (edges past
//     its capacity are read from global memory);
//   - every CTA holds a copy of all N distances; the owner of u writes each
//     improvement of d[u] into every copy with distributed-shared-memory
//     stores (one writer per entry; readers see the old or the new value, both
//     upper bounds, as in the global kernel);
//   - one cluster barrier per sweep, after every CTA has stored its
//     "changed" flag into every CTA's flag slots (two slot sets by sweep
//     parity: a CTA overwrites the set of sweep s only after the barrier of
//     sweep s + 1, which every CTA passes only once it has read them).
// The warm start computes the links of owned vertices (rows in shared
// memory), broadcasts them, and every CTA runs the pointer jumping in its own
// shared memory.  Every exit and every cluster barrier is reached by all CTAs
// alike: each decision is taken from values identical in every CTA (the edge
// count, the start and goal, the sweep count, the gathered flags).
// A sweep is edge-parallel inside a CTA: every thread takes owned edges
// (u -> c) and lowers best[u] (the bits of fl(w + d[c]); non-negative doubles
// order like unsigned integers) with a shared-memory atomicMin; a vertex pass
// then compares best[u] with d[u] and broadcasts the improvements.
// Shared memory: d [N] doubles, links / successors [2N] u32, best [V] u64,
// owned row offsets [V+1], owned columns [cap], their local source vertex
// [cap] u16 and weights [cap].
// ---------------------------------------------------------------------------
namespace {
DEVI unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
DEVI unsigned cl_map(unsigned a, unsigned rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
DEVI void cl_st_f64(unsigned a, double v) { asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory"); }
DEVI void cl_st_u32(unsigned a, unsigned v) { asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory"); }
DEVI void cl_st_u64(unsigned a, unsigned long long v) {
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}
DEVI void cl_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
DEVI unsigned cl_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
DEVI unsigned cl_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
}  // namespace

constexpr int TO_CL_MAX = 16;

__global__ void __launch_bounds__(1024, 1) k_search_to_cluster(GoalSearchParams G, int ecap) {
    extern __shared__ __align__(16) unsigned char s_raw[];
    __shared__ unsigned long long s_near[TO_CL_MAX][4];   // per CTA: start bits, id, goal bits, id
    __shared__ int s_flag[2][TO_CL_MAX];
    __shared__ unsigned s_rb_d[TO_CL_MAX];                 // d copy of every CTA (cluster addresses)
    __shared__ unsigned long long s_kb[2][32];
    __shared__ int s_ki[2][32];
    __shared__ int s_prev[2], s_se[2];
    const int N = G.N, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nt = blockDim.x;
    const unsigned rank = cl_rank(), C = cl_size();
    const int V = (N + (int)C - 1) / (int)C;
    const int v0 = min(N, (int)rank * V), v1 = min(N, v0 + V), nv = v1 - v0;
    double* s_d = (double*)s_raw;
    unsigned* s_link = (unsigned*)(s_d + N);
    unsigned long long* s_best = (unsigned long long*)(s_link + 2 * N);
    int* s_ro = (int*)(s_best + V);
    int* s_col = s_ro + (V + 1);
    unsigned short* s_src = (unsigned short*)(s_col + ecap);
    double* s_w = (double*)(((uintptr_t)(s_src + ecap) + 7) & ~(uintptr_t)7);
    DevInfo* info = G.info;
    const double inf = __longlong_as_double(DINF);
    volatile double* vd = s_d;

    cl_sync();  // every CTA of the cluster is running before any remote store
    if (tid < (int)C) s_rb_d[tid] = cl_map(smem_addr(s_d), tid);
    if (tid == 0) {
        s_prev[0] = ((volatile int*)G.prev)[0];
        s_prev[1] = ((volatile int*)G.prev)[1];
        const long long E = *G.count;
        s_se[0] = (E < 0 || E > G.cap) ? 1 : 0;
        if (s_se[0] && rank == 0) set_status_s(info, PLAN_ERR_INVALID_ARG, DET_OUTPUT);
    }
    __syncthreads();
    if (s_se[0]) {  // the same edge count in every CTA: all leave here
        cl_sync();
        return;
    }
    const int pg = s_prev[0];
    const bool may_warm = G.warm && s_prev[1] == N && pg >= 0 && pg < N;

    // phase 0: owned rows into shared memory; nearest candidates; links
    const int eb = __ldg(&G.row_off[v0]), ee = __ldg(&G.row_off[v1]);
    const int nloc = min(ee - eb, ecap);
    for (int k = tid; k <= nv; k += nt) s_ro[k] = __ldg(&G.row_off[v0 + k]) - eb;
    for (int i = tid; i < nloc; i += nt) {
        s_col[i] = __ldg(&G.col[eb + i]);
        s_w[i] = ldw(G, eb + i);
    }
    if (may_warm)
        for (int v = tid; v < N; v += nt) s_d[v] = ((const volatile double*)G.d)[v];
    double sp[4], gp[4];
    for (int a = 0; a < 4; ++a) {
        sp[a] = a < G.m ? G.endpoints[a] : 0.0;
        gp[a] = a < G.m ? G.endpoints[G.m + a] : 0.0;
    }
    unsigned long long kb[2] = {~0ull, ~0ull};
    int ki[2] = {0x7fffffff, 0x7fffffff};
    for (int v = v0 + tid; v < v1; v += nt) {
        double ds = 0.0, dg = 0.0;
        for (int a = 0; a < G.m; ++a) {
            const double x = ldd(G.states, (long long)v * G.n + a, G.in_f32);
            const double ts = __dsub_rn(x, sp[a]), tg = __dsub_rn(x, gp[a]);
            ds = __dadd_rn(ds, __dmul_rn(ts, ts));
            dg = __dadd_rn(dg, __dmul_rn(tg, tg));
        }
        keep_min(kb[0], ki[0], (unsigned long long)__double_as_longlong(ds), v);
        keep_min(kb[1], ki[1], (unsigned long long)__double_as_longlong(dg), v);
    }
    for (int h = 0; h < 2; ++h) {
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ob = __shfl_down_sync(0xffffffffu, kb[h], o);
            const int oi = __shfl_down_sync(0xffffffffu, ki[h], o);
            keep_min(kb[h], ki[h], ob, oi);
        }
        if (lane == 0) {
            s_kb[h][wid] = kb[h];
            s_ki[h][wid] = ki[h];
        }
    }
    __syncthreads();  // also: owned rows loaded
    for (int k = tid; k < nv; k += nt) {   // local source vertex of every on-chip edge
        const int r1 = min(s_ro[k + 1], nloc);
        for (int i = s_ro[k]; i < r1; ++i) s_src[i] = (unsigned short)k;
    }
    if (tid < 2) {
        unsigned long long b0 = ~0ull;
        int i0 = 0x7fffffff;
        for (int w = 0; w < (nt >> 5); ++w) keep_min(b0, i0, s_kb[tid][w], s_ki[tid][w]);
        const unsigned a = smem_addr(&s_near[rank][2 * tid]);
        for (unsigned q = 0; q < C; ++q) {
            const unsigned ra = cl_map(a, q);
            cl_st_u64(ra, b0);
            cl_st_u64(ra + 8, (unsigned long long)(unsigned)i0);
        }
    }
    if (may_warm) {
        const unsigned la = smem_addr(s_link);
        for (int v = v0 + tid; v < v1; v += nt) {
            unsigned link = (unsigned)v;
            if (v == pg) {
                link |= TO_OK;
            } else {
                const int sv = G.succ[v];
                if (sv >= 0 && sv < N && G.d[v] < inf) {
                    const int k = v - v0, r1 = s_ro[k + 1];
                    int lo = s_ro[k], hi = r1;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        const int cm = mid < ecap ? s_col[mid] : __ldg(&G.col[eb + mid]);
                        if (cm < sv) lo = mid + 1;
                        else hi = mid;
                    }
                    if (lo < r1) {
                        const int cl = lo < ecap ? s_col[lo] : __ldg(&G.col[eb + lo]);
                        const double wl = lo < ecap ? s_w[lo] : ldw(G, eb + lo);
                        if (cl == sv && wl <= G.wsucc[v]) link = (unsigned)sv | TO_OK;
                    }
                }
            }
            for (unsigned q = 0; q < C; ++q) cl_st_u32(cl_map(la + 4u * v, q), link);
        }
    }
    cl_sync();

    // phase 1: start and goal (every CTA alike); warm: pointer jumping here; d
    if (tid < 2) {
        unsigned long long b0 = ~0ull;
        int i0 = 0x7fffffff;
        for (unsigned q = 0; q < C; ++q) keep_min(b0, i0, s_near[q][2 * tid], (int)s_near[q][2 * tid + 1]);
        s_se[tid] = i0;
    }
    __syncthreads();
    const int start = s_se[0], goal = s_se[1];
    if (start < 0 || start >= N || goal < 0 || goal >= N) {
        if (rank == 0 && tid == 0) set_status_s(info, PLAN_ERR_INVALID_ARG, DET_WALK);
        cl_sync();
        return;
    }
    if (rank == 0 && tid == 0) ((volatile int*)G.prev)[0] = -1;
    const bool warm = may_warm && pg == goal;
    if (warm) {
        unsigned* a0 = s_link;
        unsigned* a1 = s_link + N;
        for (int r = 0; r < 64; ++r) {
            const int any = __syncthreads_or(jump_round<false>(a0, a1, tid, nt, N));
            unsigned* t = a0;
            a0 = a1;
            a1 = t;
            if (!any) break;
        }
        for (int v = tid; v < N; v += nt)
            if (v == goal) s_d[v] = 0.0;
            else if (a0[v] != ((unsigned)goal | TO_OK)) s_d[v] = inf;
    } else {
        for (int v = tid; v < N; v += nt) s_d[v] = v == goal ? 0.0 : inf;
    }
    cl_sync();  // no copy is written by a sweep before every CTA has set it

    // phase 2: sweeps
    int sweeps = 0;
    for (;;) {
        if (sweeps >= G.max_sweeps) {
            if (rank == 0 && tid == 0) set_status_s(info, PLAN_ERR_TIMEOUT, DET_SWEEPS);
            return;  // the same count in every CTA; no remote access follows the last barrier
        }
        const int par = sweeps & 1;
        ++sweeps;
        int changed = 0;
        for (int k = tid; k < nv; k += nt) s_best[k] = (unsigned long long)__double_as_longlong(vd[v0 + k]);
        __syncthreads();
        for (int i = tid; i < nloc; i += nt) {   // on-chip edges
            const int c = s_col[i];
            if (c < 0 || c >= N) continue;
            const unsigned long long x = (unsigned long long)__double_as_longlong(__dadd_rn(s_w[i], vd[c]));
            const int k = s_src[i];
            if (x < ((volatile unsigned long long*)s_best)[k]) atomicMin(&s_best[k], x);
        }
        __syncthreads();
        for (int k = tid; k < nv; k += nt) {
            const int u = v0 + k;
            if (u == goal) continue;
            const double cur = vd[u];
            double best = __longlong_as_double((long long)s_best[k]);
            const int r1 = s_ro[k + 1];
            for (int i = max(s_ro[k], nloc); i < r1; ++i) {   // edges past the on-chip capacity
                const int c = __ldg(&G.col[eb + i]);
                if (c < 0 || c >= N) continue;
                const double x = __dadd_rn(ldw(G, eb + i), vd[c]);
                if (x < best) best = x;
            }
            if (best < cur) {
                for (unsigned q = 0; q < C; ++q) cl_st_f64(s_rb_d[q] + 8u * (unsigned)u, best);
                changed = 1;
            }
        }
        const int ch = __syncthreads_or(changed);
        if (tid < (int)C) cl_st_u32(cl_map(smem_addr(&s_flag[par][rank]), tid), (unsigned)ch);
        cl_sync();
        int any = 0;
        for (unsigned q = 0; q < C; ++q) any |= s_flag[par][q];
        if (!any) break;
    }

    // phase 3: successors of owned vertices; d, succ, wsucc kept for the next
    // call; successors also into CTA 0's link area for the walk
    const unsigned succ0 = cl_map(smem_addr(s_link), 0);
    for (int k = tid; k < nv; k += nt) {
        const int u = v0 + k;
        double bc = inf, bw = 0.0;
        int bv = 0x7fffffff;
        if (u != goal) {
            const int r1 = s_ro[k + 1];
            for (int i = s_ro[k]; i < r1; ++i) {
                const int c = i < ecap ? s_col[i] : __ldg(&G.col[eb + i]);
                if (c < 0 || c >= N) continue;
                const double w = i < ecap ? s_w[i] : ldw(G, eb + i);
                keep_succ(bc, bv, bw, __dadd_rn(w, vd[c]), c, w);
            }
        }
        const int sv = bc < inf ? bv : -1;
        G.succ[u] = sv;
        G.wsucc[u] = bc < inf ? bw : 0.0;
        G.d[u] = vd[u];
        cl_st_u32(succ0 + 4u * (unsigned)u, (unsigned)sv);
    }
    cl_sync();

    // phase 4: the path (CTA 0, thread 0)
    if (rank == 0 && tid == 0) {
        const volatile int* succ = (const volatile int*)s_link;
        info->start = start;
        info->goal = goal;
        info->search_iters = (unsigned long long)sweeps;
        const double ds = vd[start];
        if (!(ds < inf)) {
            *G.path_len = 0;
            *G.cost = inf;
            set_status_s(info, PLAN_ERR_NO_PATH, DET_NONE);
        } else {
            int v = start, L = 0;
            bool ok = true;
            for (;;) {
                if (L < G.path_cap) G.path[L] = v;
                ++L;
                if (v == goal) break;
                v = succ[v];
                if (v < 0 || v >= N || L > N) {
                    ok = false;
                    break;
                }
            }
            *G.path_len = L;
            *G.cost = ds;
            if (!ok) set_status_s(info, PLAN_ERR_TIMEOUT, DET_WALK);
            else if (L > G.path_cap) set_status_s(info, PLAN_ERR_CAPACITY, DET_PATHCAP);
        }
        info->path_len = *G.path_len;
        ((volatile int*)G.prev)[1] = N;
        __threadfence();
        ((volatile int*)G.prev)[0] = goal;
    }
}

namespace {
// Shared memory of the on-chip kernel for N vertices, cluster size C and ecap
// edges a CTA.
size_t cluster_smem(int N, int C, int ecap) {
    const int V = (N + C - 1) / C;
    size_t b = (size_t)8 * N + (size_t)8 * N + (size_t)8 * V + (size_t)4 * (V + 1) + (size_t)6 * ecap;
    b = (b + 7) & ~(size_t)7;
    return b + (size_t)8 * ecap;
}

struct ClusterChoice {
    int dev = -1, optin = 0;
    int ok16 = -1, ok8 = -1;   // -1 unknown, 0 no, 1 yes (at the largest shared memory)
};
std::mutex g_cl_mu;
ClusterChoice g_cl[64];

// Cluster size usable at the device's largest shared-memory size (16, 8 or 0).
int cluster_size_for(int dev) {
    std::lock_guard<std::mutex> lock(g_cl_mu);
    if (dev < 0 || dev >= 64) return 0;
    ClusterChoice& c = g_cl[dev];
    if (c.dev != dev) {
        c.dev = dev;
        cudaDeviceGetAttribute(&c.optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        const int dyn = c.optin - 4096;   // room for the static shared memory
        cudaFuncSetAttribute(k_search_to_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        cudaFuncSetAttribute(k_search_to_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        for (int C : {16, 8}) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(C);
            cfg.blockDim = dim3(1024);
            cfg.dynamicSmemBytes = dyn;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = C;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int ncl = 0;
            const cudaError_t e = cudaOccupancyMaxActiveClusters(&ncl, k_search_to_cluster, &cfg);
            if (e != cudaSuccess) cudaGetLastError();
            (C == 16 ? c.ok16 : c.ok8) = (e == cudaSuccess && ncl >= 1) ? 1 : 0;
        }
    }
    return c.ok16 == 1 ? 16 : c.ok8 == 1 ? 8 : 0;
}
}  // namespace

int launch_search_to(const GoalSearchParams& G, void* stream, int num_sms, int* launches) {
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    cudaGetDevice(&dev);
    const int C = G.N <= TO_CLUSTER_MAX_N ? cluster_size_for(dev) : 0;
    if (C > 0) {
        // owned edges a CTA keeps on chip: twice the even share of the CSR's
        // capacity, within the device's shared memory (the rest from global memory)
        const int dyn = g_cl[dev].optin - 4096;
        const long long even = (G.cap + C - 1) / C;
        long long ecap = 2 * even + 64;
        const size_t base = cluster_smem(G.N, C, 0);
        const long long fit = ((long long)dyn - (long long)base - 16) / 14;
        if (ecap > fit) ecap = fit;
        if (ecap >= even / 2 && ecap >= 64) {
            const int ec = (int)ecap;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(C);
            cfg.blockDim = dim3(1024);
            cfg.dynamicSmemBytes = cluster_smem(G.N, C, ec);
            cfg.stream = st;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = C;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            GoalSearchParams Q = G;
            cudaError_t e = cudaLaunchKernelEx(&cfg, k_search_to_cluster, Q, ec);
            ++*launches;
            return (int)e;
        }
    }
    const size_t smem_max = (size_t)2 * TO_SMEM_N * sizeof(unsigned);
    const size_t smem = G.warm && G.N <= TO_SMEM_N ? (size_t)2 * G.N * sizeof(unsigned) : 0;
    cudaFuncSetAttribute(k_search_to, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_search_to, 1024, smem_max);
    if (occ < 1) return (int)cudaErrorCooperativeLaunchTooLarge;
    GoalSearchParams Q = G;
    void* args[] = {&Q};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_search_to, dim3(num_sms), dim3(1024), args, smem, st);
    ++*launches;
    return (int)e;
}

int launch_search_batched(const BatchSearchParams& P, void* stream, int* launches) {
    if (P.Q <= 0) return 0;
    k_search_batched<<<P.Q, 1024, 0, (cudaStream_t)stream>>>(P);
    ++*launches;
    return (int)cudaGetLastError();
}

int launch_search(const SearchParams& P, void* stream, int num_sms, int* launches) {
    cudaStream_t st = (cudaStream_t)stream;
    // one block per SM: fewer arrivals per grid barrier; the walk's staging
    // buffer (block 0) holds pred[] for up to SEARCH_WALK_SMEM vertices
    const size_t smem = (size_t)SEARCH_WALK_SMEM * sizeof(int);
    cudaFuncSetAttribute(k_search, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_search, 1024, smem);
    if (occ < 1) return (int)cudaErrorCooperativeLaunchTooLarge;
    SearchParams Q = P;
    Q.walk_smem = SEARCH_WALK_SMEM;
    void* args[] = {&Q};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_search, dim3(num_sms), dim3(1024), args, smem, st);
    ++*launches;
    return (int)e;
}

// ---------------------------------------------------------------------------
// Search that allocates nothing (plan_search_noalloc).
//
// Some callers cannot allocate device memory when they plan: a replanning
// loop that must answer within a few milliseconds (cudaMalloc and cudaFree
// can block and cudaFree synchronises the device), or a process whose device
// memory is owned entirely by a pool allocator.  This variant of the search
// keeps all of its scratch -- the status word and grid-barrier counters, the
// distance, predecessor and last-relaxed arrays -- in one file-scope __device__
// array sized for NOALLOC_MAX_N vertices (about 1.9 MB), which every GPU that
// loads the library holds until the process exits.  The caller passes only
// inputs and outputs.
// ---------------------------------------------------------------------------
constexpr int NOALLOC_MAX_N = 65536;
constexpr int NOALLOC_MAX_DEVICES = 64;

struct NoAllocScratch {
    DevInfo info;
    unsigned long long dist[NOALLOC_MAX_N];
    unsigned long long best[NOALLOC_MAX_N];
    int pred[NOALLOC_MAX_N];
    unsigned long long last[NOALLOC_MAX_N];
    unsigned long long near_blk[4 * SEARCH_MAX_BLOCKS];
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on the current device.  The symbol's
// name is only a host-side stand-in; the address is looked up once per device
// (with that device current) and cached.
cudaError_t noalloc_scratch(NoAllocScratch** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = p;
    }
    *out = reinterpret_cast<NoAllocScratch*>(g_noalloc_addr[dev]);
    return cudaSuccess;
}
}  // namespace

}  // namespace plan

extern "C" int plan_search_noalloc(int m, int gamma, int input, int w_f64, int N, const void* states,
                                   const plan_edges* edges, const double* start_pos, const double* goal_pos,
                                   int32_t* path, int path_cap, int32_t* path_len, double* cost, int32_t* status,
                                   void* cuda_stream) {
    using namespace plan;
    if (m < 1 || m > 4 || gamma < 1 || gamma > 4 || (input != PLAN_IN_F64 && input != PLAN_IN_F32)) return PLAN_ERR_INVALID_ARG;
    if (N < 1 || !states || !edges || !edges->row_off || !edges->count || edges->cap < 0 ||
        (edges->cap > 0 && (!edges->col || !edges->w)))
        return PLAN_ERR_INVALID_ARG;
    if (!start_pos || !goal_pos || !path || path_cap < 1 || !path_len || !cost || !status) return PLAN_ERR_INVALID_ARG;
    for (int a = 0; a < m; ++a)
        if (!std::isfinite(start_pos[a]) || !std::isfinite(goal_pos[a])) return PLAN_ERR_INVALID_ARG;
    if (N > NOALLOC_MAX_N) return PLAN_ERR_CAPACITY;  // more vertices than the static scratch holds
    NoAllocScratch* scr = nullptr;
    if (noalloc_scratch(&scr) != cudaSuccess) return PLAN_ERR_CUDA;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PLAN_ERR_CUDA;
    if (sms > SEARCH_MAX_BLOCKS) return PLAN_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the status word and the grid-barrier counters must start at zero; the
    // kernel initialises the per-vertex arrays itself
    if (cudaMemsetAsync(&scr->info, 0, sizeof(DevInfo), st) != cudaSuccess) return PLAN_ERR_CUDA;
    SearchParams S;
    memset(&S, 0, sizeof(S));
    S.N = N;
    S.m = m;
    S.n = m * gamma;
    S.in_f32 = input == PLAN_IN_F32;
    S.w_f64 = w_f64 != 0;
    S.states = states;
    S.row_off = edges->row_off;
    S.col = edges->col;
    S.w = edges->w;
    S.count = edges->count;
    S.cap = edges->cap;
    for (int a = 0; a < m; ++a) {
        S.start[a] = start_pos[a];
        S.goal[a] = goal_pos[a];
    }
    S.dist = scr->dist;
    S.bestU = scr->best;
    S.pred = scr->pred;
    S.last = scr->last;
    S.near_blk = scr->near_blk;
    S.path = path;
    S.path_cap = path_cap;
    S.path_len = path_len;
    S.cost = cost;
    S.info = &scr->info;
    S.max_sweeps = N + 1;
    S.spin_limit = 1LL << 24;
    int launches = 0;
    if (launch_search(S, st, sms, &launches) != 0) return PLAN_ERR_CUDA;
    if (cudaMemcpyAsync(status, &scr->info.status, sizeof(int32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return PLAN_ERR_CUDA;
    return PLAN_OK;
}
