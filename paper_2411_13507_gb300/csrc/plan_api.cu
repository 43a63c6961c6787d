// C ABI of libplan: context, scratch management, table upload and launches.
// Every entry point validates its arguments on the host, issues work on the
// context stream and returns; device-side conditions land in a status word
// that plan_wait reads.  No exception crosses the ABI.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "plan_internal.h"

using namespace plan;

struct plan_ctx {
    plan_model model;
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;
    TabLayout L;
    std::string last_error;
    // tables
    std::vector<double> Tcache;
    int tab_nT_cap = 0;
    double* d_tab64 = nullptr;
    float* d_tab32 = nullptr;
    double* h_tab64 = nullptr;
    float* h_tab32 = nullptr;
    cudaEvent_t tab_ev = nullptr;
    bool tab_ev_live = false;
    double lim64[4] = {0, 0, 0, 0};
    // status
    DevInfo* d_info = nullptr;
    DevInfo* h_info = nullptr;
    int last_nT = 0;
    // host-sized scratch
    long long capN = -1, capK = -1, capR = -1, capW = -1;
    uint32_t* memMask = nullptr;
    int* counts = nullptr;
    int* members = nullptr;
    int* localIdx = nullptr;
    float* centers = nullptr;
    double* blim64 = nullptr;
    float* A32 = nullptr;
    float* blim32 = nullptr;
    float* bc32 = nullptr;
    long long* resOff = nullptr;
    int* itemOff = nullptr;
    int* ntile = nullptr;
    int* tsize = nullptr;
    int* rowCount = nullptr;
    // device-sized scratch
    long long slotCap = 0, recheckCap = 0;
    long long want_slots = 0, want_rechecks = 0;
    uint32_t* resBits = nullptr;
    unsigned long long* resKey = nullptr;
    int* emitPre = nullptr;
    unsigned long long* recheck = nullptr;
    // search scratch
    long long capS = -1;
    unsigned long long* sdist = nullptr;
    unsigned long long* sbest = nullptr;
    int* spred = nullptr;
    unsigned char* sfront = nullptr;
    // timing
    bool timing = false;
    bool accounting = false;
    int max_sweeps = 0;
    long long spin_limit = 0;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pair, ev_search;
    long long launches = 0;
};

namespace {

const char* kVersion = "libplan 0.1 (sm_103a)";

int fail(plan_ctx* c, int code, const std::string& msg) {
    if (c) c->last_error = msg;
    return code;
}

int cuda_fail(plan_ctx* c, cudaError_t e, const char* where) {
    return fail(c, PLAN_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

template <typename T>
bool dalloc(plan_ctx* c, T** p, long long count) {
    if (*p) cudaFree(*p);
    *p = nullptr;
    if (count <= 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (size_t)count);
    if (e != cudaSuccess) {
        *p = nullptr;
        c->last_error = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        cudaGetLastError();
        return false;
    }
    return true;
}

int check_model(const plan_model* m) {
    if (!m) return PLAN_ERR_INVALID_ARG;
    if (m->m < 1 || m->m > 4 || m->gamma < 1 || m->gamma > 4) return PLAN_ERR_INVALID_ARG;
    if (m->degree < 2 * m->gamma - 1 || m->degree > 15) return PLAN_ERR_INVALID_ARG;
    if (m->arith < PLAN_F64 || m->arith > PLAN_BF16) return PLAN_ERR_INVALID_ARG;
    if (m->input != PLAN_IN_F64 && m->input != PLAN_IN_F32) return PLAN_ERR_INVALID_ARG;
    if (m->cost_mode != PLAN_COST_STATE && m->cost_mode != PLAN_COST_POS) return PLAN_ERR_INVALID_ARG;
    if (!std::isfinite(m->tighten) || m->tighten < 0) return PLAN_ERR_INVALID_ARG;
    for (int k = 0; k < m->gamma; ++k)
        if (!std::isfinite(m->bound[k]) || !(m->bound[k] - m->tighten > 0)) return PLAN_ERR_INVALID_ARG;
    if (!model_supported(m->m, m->gamma, m->degree) && !refine_supported(m->m, m->gamma, m->degree))
        return PLAN_ERR_UNSUPPORTED;
    if (m->arith == PLAN_TF32 || m->arith == PLAN_BF16) return PLAN_ERR_UNSUPPORTED;
    return PLAN_OK;
}

// Build the per-duration device tables (FP64 canonical and FP32 fast) and
// upload them asynchronously.
int upload_tables(plan_ctx* c, int nT, const double* T) {
    bool same = (int)c->Tcache.size() == nT;
    for (int t = 0; same && t < nT; ++t) same = c->Tcache[t] == T[t];
    if (same) return PLAN_OK;
    const TabLayout& L = c->L;
    const int g = c->model.gamma, p = c->model.degree, tg = L.tg;
    if (nT > c->tab_nT_cap) {
        if (c->tab_ev_live) cudaEventSynchronize(c->tab_ev);
        if (c->h_tab64) cudaFreeHost(c->h_tab64);
        if (c->h_tab32) cudaFreeHost(c->h_tab32);
        c->h_tab64 = nullptr;
        c->h_tab32 = nullptr;
        if (!dalloc(c, &c->d_tab64, (long long)NT_MAX * L.e_stride) || !dalloc(c, &c->d_tab32, (long long)NT_MAX * L.f_stride))
            return PLAN_ERR_NO_MEMORY;
        if (cudaMallocHost((void**)&c->h_tab64, sizeof(double) * NT_MAX * L.e_stride) != cudaSuccess ||
            cudaMallocHost((void**)&c->h_tab32, sizeof(float) * NT_MAX * L.f_stride) != cudaSuccess)
            return fail(c, PLAN_ERR_NO_MEMORY, "cudaMallocHost tables");
        c->tab_nT_cap = NT_MAX;
    }
    if (c->tab_ev_live) cudaEventSynchronize(c->tab_ev);  // staging buffer free again
    std::vector<double> D((size_t)(p + 1) * tg), H((size_t)L.rax * tg), C((size_t)g * p * tg);
    std::vector<int> Hk;
    for (int k = 1; k <= g; ++k)
        for (int j = 0; j <= p - k; ++j) Hk.push_back(k);
    // kernel row order for the fast path: highest derivative first, interior
    // control points before the end points (the rows most likely to fail)
    std::vector<int> order;
    int base = L.rax;
    for (int k = g; k >= 1; --k) {
        base -= p - k + 1;
        for (int j = 1; j < p - k; ++j) order.push_back(base + j);
        order.push_back(base);
        if (p - k > 0) order.push_back(base + p - k);
    }
    for (int t = 0; t < nT; ++t) {
        exact_tables(g, p, 1, &T[t], D.data(), H.data(), C.data());
        double* e = c->h_tab64 + (size_t)t * L.e_stride;
        float* f = c->h_tab32 + (size_t)t * L.f_stride;
        memset(f, 0, sizeof(float) * L.f_stride);
        for (int i = 0; i < L.rax * tg; ++i) e[L.e_H + i] = H[i];
        for (int i = 0; i < (p + 1) * tg; ++i) e[L.e_D + i] = D[i];
        for (int i = 0; i < g * p * tg; ++i) e[L.e_C + i] = C[i];
        for (int rr = 0; rr < L.rax; ++rr) {
            const int r = order[rr];
            const double s = 1.0 / c->lim64[Hk[r] - 1];
            for (int col = 0; col < tg; ++col) {
                const float v = (float)(H[(size_t)r * tg + col] * s);
                f[L.f_H + rr * tg + col] = v;
                float& mx = f[L.f_HC + col];
                mx = fmaxf(mx, fabsf(v));
            }
        }
        for (int l = 1; l < p; ++l)
            for (int col = 0; col < tg; ++col) {
                const float v = (float)D[(size_t)l * tg + col];
                f[L.f_D + (l - 1) * tg + col] = v;
                float& mx = f[L.f_DC + col];
                mx = fmaxf(mx, fabsf(v));
            }
        for (int i = 0; i < g * p * tg; ++i) f[L.f_C + i] = (float)C[i];
    }
    cudaError_t e1 = cudaMemcpyAsync(c->d_tab64, c->h_tab64, sizeof(double) * (size_t)nT * L.e_stride,
                                     cudaMemcpyHostToDevice, c->stream);
    cudaError_t e2 = cudaMemcpyAsync(c->d_tab32, c->h_tab32, sizeof(float) * (size_t)nT * L.f_stride,
                                     cudaMemcpyHostToDevice, c->stream);
    if (e1 != cudaSuccess || e2 != cudaSuccess) return cuda_fail(c, e1 != cudaSuccess ? e1 : e2, "table upload");
    cudaEventRecord(c->tab_ev, c->stream);
    c->tab_ev_live = true;
    c->Tcache.assign(T, T + nT);
    return PLAN_OK;
}

int ensure_host_sized(plan_ctx* c, long long N, long long K, long long R, long long W) {
    if (N > c->capN || K > c->capK || W > c->capW) {
        const long long n2 = N > c->capN ? N : c->capN, k2 = K > c->capK ? K : c->capK;
        const long long w2 = W > c->capW ? W : c->capW;
        if (!dalloc(c, &c->memMask, n2 * w2) || !dalloc(c, &c->members, k2 * n2) ||
            !dalloc(c, &c->localIdx, k2 * n2) || !dalloc(c, &c->rowCount, n2 + 1))
            return PLAN_ERR_NO_MEMORY;
        if (K > c->capK) {
            if (!dalloc(c, &c->counts, k2 + 1) || !dalloc(c, &c->centers, 4 * (k2 + 1)) ||
                !dalloc(c, &c->resOff, k2 + 1) || !dalloc(c, &c->itemOff, k2 + 1) ||
                !dalloc(c, &c->ntile, k2 + 1) || !dalloc(c, &c->tsize, k2 + 1))
                return PLAN_ERR_NO_MEMORY;
        }
        c->capN = n2;
        c->capK = k2;
        c->capW = w2;
    }
    if (R > c->capR) {
        if (!dalloc(c, &c->blim64, R) || !dalloc(c, &c->A32, 4 * R) || !dalloc(c, &c->blim32, R) ||
            !dalloc(c, &c->bc32, R))
            return PLAN_ERR_NO_MEMORY;
        c->capR = R;
    }
    return PLAN_OK;
}

int ensure_device_sized(plan_ctx* c, long long slots, long long rechecks) {
    if (slots > c->slotCap) {
        if (!dalloc(c, &c->resBits, slots) || !dalloc(c, &c->resKey, slots) || !dalloc(c, &c->emitPre, slots)) {
            c->slotCap = 0;
            return PLAN_ERR_NO_MEMORY;
        }
        c->slotCap = slots;
    }
    if (rechecks > c->recheckCap) {
        if (!dalloc(c, &c->recheck, rechecks)) {
            c->recheckCap = 0;
            return PLAN_ERR_NO_MEMORY;
        }
        c->recheckCap = rechecks;
    }
    return PLAN_OK;
}

cudaEvent_t take_event(plan_ctx* c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

}  // namespace

extern "C" {

const char* plan_version(void) { return kVersion; }

const char* plan_status_string(int s) {
    switch (s) {
        case PLAN_OK: return "ok";
        case PLAN_ERR_INVALID_ARG: return "invalid argument";
        case PLAN_ERR_UNSUPPORTED: return "unsupported model or polytope";
        case PLAN_ERR_CAPACITY: return "capacity exceeded";
        case PLAN_ERR_CUDA: return "CUDA error";
        case PLAN_ERR_TIMEOUT: return "device loop timed out";
        case PLAN_ERR_NO_PATH: return "no path";
        case PLAN_ERR_NO_MEMORY: return "out of device memory";
        default: return "unknown status";
    }
}

const char* plan_last_error(plan_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

int plan_model_tables(const plan_model* model, int nT, const double* T, double* D, double* H, double* C) {
    if (!model || model->gamma < 1 || model->gamma > 4 || model->degree < 2 * model->gamma - 1 || model->degree > 15)
        return PLAN_ERR_INVALID_ARG;
    if (nT < 0 || (nT > 0 && (!T || !D || !H || !C))) return PLAN_ERR_INVALID_ARG;
    for (int t = 0; t < nT; ++t)
        if (!std::isfinite(T[t]) || !(T[t] > 0)) return PLAN_ERR_INVALID_ARG;
    try {
        exact_tables(model->gamma, model->degree, nT, T, D, H, C);
    } catch (...) {
        return PLAN_ERR_NO_MEMORY;
    }
    return PLAN_OK;
}

int plan_create(plan_ctx** out, const plan_model* model, void* cuda_stream) {
    if (!out) return PLAN_ERR_INVALID_ARG;
    *out = nullptr;
    int rc = check_model(model);
    if (rc != PLAN_OK) return rc;
    plan_ctx* c = new (std::nothrow) plan_ctx();
    if (!c) return PLAN_ERR_NO_MEMORY;
    c->model = *model;
    c->stream = (cudaStream_t)cuda_stream;
    c->L = tab_layout(model->gamma, model->degree);
    for (int k = 0; k < model->gamma; ++k) c->lim64[k] = model->bound[k] - model->tighten;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_info, sizeof(DevInfo));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_info, sizeof(DevInfo));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->tab_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        plan_destroy(c);
        return PLAN_ERR_CUDA;
    }
    memset(c->h_info, 0, sizeof(DevInfo));
    *out = c;
    return PLAN_OK;
}

void plan_destroy(plan_ctx* c) {
    if (!c) return;
    if (c->stream || c->d_info) cudaStreamSynchronize(c->stream);
    void* dev[] = {c->d_tab64, c->d_tab32, c->d_info, c->memMask, c->counts, c->members, c->localIdx, c->centers,
                   c->blim64, c->A32, c->blim32, c->bc32, c->resOff, c->itemOff, c->ntile, c->tsize, c->rowCount,
                   c->resBits, c->resKey, c->emitPre, c->recheck, c->sdist, c->sbest, c->spred, c->sfront};
    for (void* p : dev)
        if (p) cudaFree(p);
    if (c->h_tab64) cudaFreeHost(c->h_tab64);
    if (c->h_tab32) cudaFreeHost(c->h_tab32);
    if (c->h_info) cudaFreeHost(c->h_info);
    if (c->tab_ev) cudaEventDestroy(c->tab_ev);
    for (auto& pr : c->ev_pair) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (auto& pr : c->ev_search) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    delete c;
}

int plan_build_edges(plan_ctx* c, int N, const void* states, int nT, const double* T, int K,
                     const int32_t* poly_off, int max_rows, const void* A, const void* b, const plan_edges* out) {
    if (!c) return PLAN_ERR_INVALID_ARG;
    if (!model_supported(c->model.m, c->model.gamma, c->model.degree))
        return fail(c, PLAN_ERR_UNSUPPORTED, "edge build not compiled for this (m, gamma, p)");
    if (N < 0 || N > (1 << 20)) return fail(c, PLAN_ERR_INVALID_ARG, "N out of range");
    if (nT < 1 || nT > NT_MAX || !T) return fail(c, PLAN_ERR_INVALID_ARG, "nT must be 1..32 with a host T array");
    for (int t = 0; t < nT; ++t)
        if (!std::isfinite(T[t]) || !(T[t] > 0)) return fail(c, PLAN_ERR_INVALID_ARG, "durations must be finite and > 0");
    if (K < 0 || K > 1024) return fail(c, PLAN_ERR_INVALID_ARG, "K must be 0..1024");
    if (K > 0 && (max_rows < 1 || max_rows > RMAX)) return fail(c, PLAN_ERR_INVALID_ARG, "max_rows must be 1..16");
    if ((N > 0 && !states) || (K > 0 && (!poly_off || !A || !b)))
        return fail(c, PLAN_ERR_INVALID_ARG, "null input array");
    if (!out || !out->row_off || !out->count || out->cap < 0 ||
        (out->cap > 0 && (!out->col || !out->w || !out->tidx || !out->mask)))
        return fail(c, PLAN_ERR_INVALID_ARG, "bad output CSR");
    if ((long long)K * N > (1LL << 31)) return fail(c, PLAN_ERR_INVALID_ARG, "K*N too large");
    int rc = upload_tables(c, nT, T);
    if (rc != PLAN_OK) return rc;
    const long long W = K > 0 ? (K + 31) / 32 : 1;
    const long long R = (long long)(K > 0 ? K : 1) * (max_rows > 0 ? max_rows : 1);
    rc = ensure_host_sized(c, N, K, R, W);
    if (rc != PLAN_OK) return rc;
    long long want_s = c->want_slots, want_r = c->want_rechecks;
    if (want_s == 0) want_s = (long long)3 * N * (long long)N / (K > 0 ? K : 1) + 4096;
    if (want_r == 0) want_r = (1 << 16);
    rc = ensure_device_sized(c, want_s, want_r);
    if (rc != PLAN_OK) return rc;
    cudaError_t e = cudaMemsetAsync(c->d_info, 0, sizeof(DevInfo), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset info");
    c->last_nT = nT;

    BuildParams P;
    memset(&P, 0, sizeof(P));
    P.N = N;
    P.K = K;
    P.nT = nT;
    P.W = (int)W;
    P.R = (int)R;
    P.m = c->model.m;
    P.g = c->model.gamma;
    P.p = c->model.degree;
    P.cost_mode = c->model.cost_mode;
    P.in_f32 = c->model.input == PLAN_IN_F32;
    P.arith = c->model.arith;
    P.max_rows = K > 0 ? max_rows : 1;
    P.eps = c->model.tighten;
    P.states = states;
    P.poly_off = poly_off;
    P.A = A;
    P.b = b;
    P.tab32 = c->d_tab32;
    P.tab64 = c->d_tab64;
    for (int k = 0; k < 4; ++k) P.lim64[k] = c->lim64[k];
    P.L = c->L;
    P.memMask = c->memMask;
    P.counts = c->counts;
    P.members = c->members;
    P.localIdx = c->localIdx;
    P.centers = c->centers;
    P.blim64 = c->blim64;
    P.A32 = c->A32;
    P.blim32 = c->blim32;
    P.bc32 = c->bc32;
    P.resOff = c->resOff;
    P.itemOff = c->itemOff;
    P.ntile = c->ntile;
    P.tsize = c->tsize;
    P.resBits = c->resBits;
    P.resKey = c->resKey;
    P.emitPre = c->emitPre;
    P.recheck = c->recheck;
    P.rowCount = c->rowCount;
    P.slotCap = c->slotCap;
    P.recheckCap = c->recheckCap;
    P.info = c->d_info;
    P.row_off = out->row_off;
    P.col = out->col;
    P.w = out->w;
    P.tidx = out->tidx;
    P.mask = out->mask;
    P.cap = out->cap;
    P.count = out->count;

    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->timing) {
        e0 = take_event(c);
        e1 = take_event(c);
        c->ev_pair.emplace_back(e0, e1);
    }
    int launches = 0;
    int ce = launch_build(P, c->stream, c->num_sms, e0, e1, &launches);
    c->launches += launches;
    if (ce != 0) return cuda_fail(c, (cudaError_t)ce, "build launch");
    if (c->accounting && N > 0 && K > 0) {
        ce = launch_account(P, c->stream, c->num_sms, c->d_info->work);
        if (ce != 0) return cuda_fail(c, (cudaError_t)ce, "accounting launch");
    }
    return PLAN_OK;
}

int plan_search(plan_ctx* c, int N, const void* states, const plan_edges* edges, const double* start_pos,
                const double* goal_pos, int32_t* path, int path_cap, int32_t* path_len, double* cost) {
    if (!c) return PLAN_ERR_INVALID_ARG;
    if (N < 1 || N > (1 << 20) || !states) return fail(c, PLAN_ERR_INVALID_ARG, "need N >= 1 states");
    if (!edges || !edges->row_off || !edges->count || edges->cap < 0 || (edges->cap > 0 && (!edges->col || !edges->w)))
        return fail(c, PLAN_ERR_INVALID_ARG, "bad CSR");
    if (!start_pos || !goal_pos || !path || path_cap < 1 || !path_len || !cost)
        return fail(c, PLAN_ERR_INVALID_ARG, "bad search output");
    for (int a = 0; a < c->model.m; ++a)
        if (!std::isfinite(start_pos[a]) || !std::isfinite(goal_pos[a]))
            return fail(c, PLAN_ERR_INVALID_ARG, "start/goal must be finite");
    if (N > c->capS) {
        if (!dalloc(c, &c->sdist, N) || !dalloc(c, &c->sbest, N) || !dalloc(c, &c->spred, N) ||
            !dalloc(c, &c->sfront, 2LL * N))
            return PLAN_ERR_NO_MEMORY;
        c->capS = N;
    }
    SearchParams S;
    memset(&S, 0, sizeof(S));
    S.N = N;
    S.m = c->model.m;
    S.n = c->model.m * c->model.gamma;
    S.in_f32 = c->model.input == PLAN_IN_F32;
    S.w_f64 = c->model.arith == PLAN_F64;
    S.states = states;
    S.row_off = edges->row_off;
    S.col = edges->col;
    S.w = edges->w;
    S.count = edges->count;
    S.cap = edges->cap;
    for (int a = 0; a < c->model.m; ++a) {
        S.start[a] = start_pos[a];
        S.goal[a] = goal_pos[a];
    }
    S.dist = c->sdist;
    S.bestU = c->sbest;
    S.pred = c->spred;
    S.front = c->sfront;
    S.path = path;
    S.path_cap = path_cap;
    S.path_len = path_len;
    S.cost = cost;
    S.info = c->d_info;
    S.max_sweeps = c->max_sweeps > 0 ? c->max_sweeps : N + 1;
    S.spin_limit = c->spin_limit > 0 ? c->spin_limit : (1LL << 24);
    cudaError_t e = cudaMemsetAsync(&c->d_info->bar_count, 0, sizeof(unsigned) * 2, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset barrier");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->timing) {
        e0 = take_event(c);
        e1 = take_event(c);
        c->ev_search.emplace_back(e0, e1);
        cudaEventRecord(e0, c->stream);
    }
    int launches = 0;
    int ce = launch_search(S, c->stream, c->num_sms, &launches);
    if (c->timing) cudaEventRecord(e1, c->stream);
    c->launches += launches;
    if (ce != 0) return cuda_fail(c, (cudaError_t)ce, "search launch");
    return PLAN_OK;
}

int plan_refine(plan_ctx* c, int S, const float* P, const float* T, const float* A, const float* b,
                const int32_t* nrows, int rmax, const plan_refine_weights* weights, const float* grad_loss,
                float* loss, float* dP, float* dT) {
    if (!c) return PLAN_ERR_INVALID_ARG;
    if (!refine_supported(c->model.m, c->model.gamma, c->model.degree))
        return fail(c, PLAN_ERR_UNSUPPORTED, "refine needs (m,gamma,p) = (3,3,7) or (2,2,5)");
    if (S < 0 || rmax < 0 || rmax > 64) return fail(c, PLAN_ERR_INVALID_ARG, "bad S or rmax");
    if (S > 0 && (!P || !T || !nrows || (rmax > 0 && (!A || !b))))
        return fail(c, PLAN_ERR_INVALID_ARG, "null input array");
    if (S > 0 && ((!grad_loss && !loss) || (grad_loss && (!dP || !dT))))
        return fail(c, PLAN_ERR_INVALID_ARG, "null output array");
    plan_refine_weights w = {1.0, 1.0, 0.1};
    if (weights) w = *weights;
    if (!(w.delta > 0) || !std::isfinite(w.mu) || !std::isfinite(w.w_snap))
        return fail(c, PLAN_ERR_INVALID_ARG, "bad weights");
    RefineParams R;
    memset(&R, 0, sizeof(R));
    R.S = S;
    R.m = c->model.m;
    R.g = c->model.gamma;
    R.p = c->model.degree;
    R.rmax = rmax;
    R.P = P;
    R.T = T;
    R.A = A;
    R.b = b;
    R.nrows = nrows;
    for (int k = 0; k < 4; ++k) R.bound[k] = (float)c->lim64[k];
    R.w_snap = (float)w.w_snap;
    R.mu = (float)w.mu;
    R.delta = (float)w.delta;
    R.grad_loss = grad_loss;
    R.loss = loss;
    R.dP = dP;
    R.dT = dT;
    int launches = 0;
    int ce = launch_refine(R, c->stream, &launches);
    c->launches += launches;
    if (ce != 0) return cuda_fail(c, (cudaError_t)ce, "refine launch");
    return PLAN_OK;
}

int plan_wait(plan_ctx* c, plan_info* info) {
    if (!c) return PLAN_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream sync");
    e = cudaMemcpy(c->h_info, c->d_info, sizeof(DevInfo), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "read status");
    const DevInfo& d = *c->h_info;
    if (d.status == PLAN_ERR_CAPACITY) {
        if (d.detail == DET_SLOTS) c->want_slots = (long long)(d.need_slots + d.need_slots / 4 + 1024);
        if (d.detail == DET_RECHECK) {
            long long need = (long long)(d.need_rechecks > d.rechecks ? d.need_rechecks : d.rechecks);
            c->want_rechecks = need + need / 4 + 1024;
        }
    }
    if (info) {
        memset(info, 0, sizeof(*info));
        info->status = d.status;
        info->detail = d.detail;
        info->memberships = (int64_t)d.memberships;
        info->slots = (int64_t)d.slots;
        info->candidates = (int64_t)d.candidates;
        info->checks = (int64_t)d.candidates * c->last_nT;
        info->reach_pass = (int64_t)d.reach_pass;
        info->feasible = (int64_t)d.feasible;
        info->rechecks = (int64_t)d.rechecks;
        info->edges = (int64_t)d.edges;
        info->search_iters = (int64_t)d.search_iters;
        info->start = d.start;
        info->goal = d.goal;
        info->need_slots = (int64_t)d.need_slots;
        info->need_rechecks = (int64_t)d.need_rechecks;
        info->work_reach_rows = (int64_t)d.work[0];
        info->work_free_rows = (int64_t)d.work[1];
        info->work_costs = (int64_t)d.work[2];
    }
    return d.status;
}

int plan_set_search_limits(plan_ctx* c, int max_sweeps, int64_t spin_limit) {
    if (!c || max_sweeps < 0 || spin_limit < 0) return PLAN_ERR_INVALID_ARG;
    c->max_sweeps = max_sweeps;
    c->spin_limit = spin_limit;
    return PLAN_OK;
}

int plan_set_accounting(plan_ctx* c, int enable) {
    if (!c) return PLAN_ERR_INVALID_ARG;
    c->accounting = enable != 0;
    return PLAN_OK;
}

int plan_set_timing(plan_ctx* c, int enable) {
    if (!c) return PLAN_ERR_INVALID_ARG;
    c->timing = enable != 0;
    return PLAN_OK;
}

int plan_timing(plan_ctx* c, double* pair_ms, int64_t* pair_launches, double* search_ms, int64_t* search_launches,
                int64_t* total_launches, int reset) {
    if (!c) return PLAN_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream sync");
    double pm = 0, sm = 0;
    for (auto& pr : c->ev_pair) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) pm += ms;
    }
    for (auto& pr : c->ev_search) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) sm += ms;
    }
    cudaGetLastError();
    if (pair_ms) *pair_ms = pm;
    if (search_ms) *search_ms = sm;
    if (pair_launches) *pair_launches = (int64_t)c->ev_pair.size();
    if (search_launches) *search_launches = (int64_t)c->ev_search.size();
    if (total_launches) *total_launches = c->launches;
    if (reset) {
        for (auto& pr : c->ev_pair) {
            c->ev_pool.push_back(pr.first);
            c->ev_pool.push_back(pr.second);
        }
        for (auto& pr : c->ev_search) {
            c->ev_pool.push_back(pr.first);
            c->ev_pool.push_back(pr.second);
        }
        c->ev_pair.clear();
        c->ev_search.clear();
        c->launches = 0;
    }
    return PLAN_OK;
}

}  // extern "C"
