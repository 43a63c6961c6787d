// findPath for sm_103a (Sec. III-C, Problem 2): nearest start/goal vertices,
// then single-source shortest paths with Dijkstra's semantics, all in one
// cooperative kernel with a bounded software grid barrier.
//
// Distances are FP64 bit patterns (non-negative doubles order like unsigned
// integers), relaxed with atomicMin by a frontier sweep (Bellman-Ford).  With
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

// Grid-wide barrier for a cooperative launch (all blocks co-resident).  The
// spin is bounded: on expiry the block records PLAN_ERR_TIMEOUT and returns
// false instead of waiting forever.
DEVI bool grid_sync(DevInfo* info, unsigned nblocks, long long spin_limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* genp = &info->bar_gen;
        const unsigned gen = *genp;
        __threadfence();
        const unsigned arrived = atomicAdd(&info->bar_count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&info->bar_count, 0u);
            __threadfence();
            atomicAdd(&info->bar_gen, 1u);
        } else {
            long long it = 0;
            while (*genp == gen) {
                if (++it > spin_limit) {
                    set_status_s(info, PLAN_ERR_TIMEOUT, DET_BARRIER);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

DEVI double ldd(const void* p, long long i, int f32) {
    return f32 ? (double)((const float*)p)[i] : ((const double*)p)[i];
}
}  // namespace

__global__ void __launch_bounds__(1024) k_search(SearchParams P) {
    const unsigned nb = gridDim.x;
    const long long gtid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const long long gwarp = gtid >> 5, nwarps = nthr >> 5;
    DevInfo* info = P.info;
    const int N = P.N;

    // phase 0: initialise scratch
    if (gtid == 0) {
        info->near_d[0] = ~0ull;
        info->near_d[1] = ~0ull;
        info->start = 0x7fffffff;
        info->goal = 0x7fffffff;
        info->changed[0] = 0;
        info->changed[1] = 0;
        info->changed[2] = 0;
        const long long E = *P.count;
        if (E < 0 || E > P.cap) set_status_s(info, PLAN_ERR_INVALID_ARG, DET_OUTPUT);
    }
    for (long long v = gtid; v < N; v += nthr) {
        P.dist[v] = DINF;
        P.bestU[v] = ~0ull;
        P.pred[v] = 0x7fffffff;
        P.front[v] = 0;
        P.front[N + v] = 0;
    }
    if (!grid_sync(info, nb, P.spin_limit)) return;
    if (failed_s(info)) return;

    // A6: nearest vertex to the start and goal positions (canonical FP64
    // squared distance summed left to right; ties to the lowest id)
    for (long long v = gtid; v < N; v += nthr) {
        double ds = 0.0, dg = 0.0;
        for (int a = 0; a < P.m; ++a) {
            const double x = ldd(P.states, v * P.n + a, P.in_f32);
            const double ts = __dsub_rn(x, P.start[a]);
            const double tg = __dsub_rn(x, P.goal[a]);
            ds = __dadd_rn(ds, __dmul_rn(ts, ts));
            dg = __dadd_rn(dg, __dmul_rn(tg, tg));
        }
        atomicMin(&info->near_d[0], (unsigned long long)__double_as_longlong(ds));
        atomicMin(&info->near_d[1], (unsigned long long)__double_as_longlong(dg));
    }
    if (!grid_sync(info, nb, P.spin_limit)) return;
    for (long long v = gtid; v < N; v += nthr) {
        double ds = 0.0, dg = 0.0;
        for (int a = 0; a < P.m; ++a) {
            const double x = ldd(P.states, v * P.n + a, P.in_f32);
            const double ts = __dsub_rn(x, P.start[a]);
            const double tg = __dsub_rn(x, P.goal[a]);
            ds = __dadd_rn(ds, __dmul_rn(ts, ts));
            dg = __dadd_rn(dg, __dmul_rn(tg, tg));
        }
        if ((unsigned long long)__double_as_longlong(ds) == info->near_d[0]) atomicMin(&info->start, (int)v);
        if ((unsigned long long)__double_as_longlong(dg) == info->near_d[1]) atomicMin(&info->goal, (int)v);
    }
    if (!grid_sync(info, nb, P.spin_limit)) return;
    const int s = *((volatile int*)&info->start), g = *((volatile int*)&info->goal);
    if (s < 0 || s >= N || g < 0 || g >= N) {
        if (gtid == 0) set_status_s(info, PLAN_ERR_INVALID_ARG, DET_WALK);
        return;
    }
    if (gtid == 0) {
        P.dist[s] = 0ull;
        P.front[s] = 1;
    }
    if (!grid_sync(info, nb, P.spin_limit)) return;

    // A7: frontier sweeps until no distance changes.  A relaxation reads the
    // current dist[u] first and only then issues a non-returning atomicMin,
    // so a warp's edge chunks need no round trip through the atomic unit.
    int cur = 0, it = 0;
    volatile unsigned long long* vdist = P.dist;
    for (;;) {
        bool my_change = false;
        for (long long v = gwarp; v < N; v += nwarps) {
            if (!*((volatile unsigned char*)&P.front[cur * N + v])) continue;
            __syncwarp();
            if (lane == 0) P.front[cur * N + v] = 0;
            const double dv = __longlong_as_double((long long)vdist[v]);
            const long long e0 = P.row_off[v], e1 = P.row_off[v + 1];
            for (long long eb = e0; eb < e1; eb += 128) {
                int uu[4];
                double ww[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const long long e = eb + c * 32 + lane;
                    uu[c] = -1;
                    if (e < e1) {
                        uu[c] = P.col[e];
                        ww[c] = P.w_f64 ? ((const double*)P.w)[e] : (double)((const float*)P.w)[e];
                    }
                }
                unsigned long long cu[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) cu[c] = (uu[c] >= 0 && uu[c] < N) ? vdist[uu[c]] : 0ull;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (uu[c] < 0 || uu[c] >= N) continue;
                    const unsigned long long nd = (unsigned long long)__double_as_longlong(__dadd_rn(dv, ww[c]));
                    if (nd < cu[c]) {
                        atomicMin(&P.dist[uu[c]], nd);
                        P.front[(cur ^ 1) * N + uu[c]] = 1;
                        my_change = true;
                    }
                }
            }
        }
        // flag of sweep j is changed[j % 3]: written during sweep j, read after
        // its barrier, cleared during sweep j+2 (after every block has read it)
        if (__any_sync(0xffffffffu, my_change) && lane == 0) atomicExch(&info->changed[it % 3], 1);
        if (gtid == 0) info->changed[(it + 1) % 3] = 0;
        if (!grid_sync(info, nb, P.spin_limit)) return;
        const int ch = *((volatile int*)&info->changed[it % 3]);
        ++it;
        if (!ch) break;
        if (it > P.max_sweeps) {
            if (gtid == 0) set_status_s(info, PLAN_ERR_TIMEOUT, DET_SWEEPS);
            return;
        }
        cur ^= 1;
    }

    // predecessor: minimum (dist[u], u) over in-neighbours attaining dist[v]
    for (int pass = 0; pass < 2; ++pass) {
        for (long long v = gwarp; v < N; v += nwarps) {
            const unsigned long long dvb = vdist[v];
            if (dvb >= DINF) continue;
            const double dv = __longlong_as_double((long long)dvb);
            const long long e0 = P.row_off[v], e1 = P.row_off[v + 1];
            for (long long e = e0 + lane; e < e1; e += 32) {
                const int u = P.col[e];
                if (u < 0 || u >= N || u == s) continue;
                const double w = P.w_f64 ? ((const double*)P.w)[e] : (double)((const float*)P.w)[e];
                const unsigned long long nd = (unsigned long long)__double_as_longlong(__dadd_rn(dv, w));
                if (nd != vdist[u]) continue;
                if (pass == 0) atomicMin(&P.bestU[u], dvb);
                else if (P.bestU[u] == dvb) atomicMin(&P.pred[u], (int)v);
            }
        }
        if (!grid_sync(info, nb, P.spin_limit)) return;
    }

    // walk goal -> start
    if (gtid == 0) {
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
                v = P.pred[v];
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
                    if (q) v = P.pred[v];
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
        for (int v = wid; v < N; v += nw) {
            if (!front[cur * N + v]) continue;
            __syncwarp();
            if (lane == 0) front[cur * N + v] = 0;
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
    for (int pass = 0; pass < 2; ++pass) {
        for (int v = wid; v < N; v += nw) {
            const unsigned long long dvb = vdist[v];
            if (dvb >= DINF) continue;
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

int launch_search_batched(const BatchSearchParams& P, void* stream, int* launches) {
    if (P.Q <= 0) return 0;
    k_search_batched<<<P.Q, 1024, 0, (cudaStream_t)stream>>>(P);
    ++*launches;
    return (int)cudaGetLastError();
}

int launch_search(const SearchParams& P, void* stream, int num_sms, int* launches) {
    cudaStream_t st = (cudaStream_t)stream;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_search, 1024, 0);
    if (occ < 1) occ = 1;
    if (occ > 2) occ = 2;
    const int nb = num_sms * occ;
    SearchParams Q = P;
    void* args[] = {&Q};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_search, dim3(nb), dim3(1024), args, 0, st);
    ++*launches;
    return (int)e;
}

// ---------------------------------------------------------------------------
// Search that allocates nothing (plan_search_noalloc).
//
// Some callers cannot allocate device memory when they plan: a replanning
// loop that must answer within a few milliseconds (cudaMalloc and cudaFree
// can block and cudaFree synchronises the device), code that runs while a
// stream is being captured into a CUDA graph, or a process whose device
// memory is owned entirely by a pool allocator.  This variant of the search
// keeps all of its scratch -- the status word and grid-barrier counters, the
// distance, predecessor and frontier arrays -- in one file-scope __device__
// array sized for NOALLOC_MAX_N vertices (about 1.4 MB), which every GPU that
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
    unsigned char front[2 * NOALLOC_MAX_N];
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
    S.front = scr->front;
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
