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
    // batch state (host) and its device copies
    int bQ = 0, b_max_rows = 1, b_tile = 0;
    std::vector<QueryDesc> hq;
    std::vector<long long> pfx;       // 4 x (Q+1): mask, poly, rows, N
    long long totMask = 0, totPoly = 0, totRows = 0, totN = 0, totList = 0, totK1 = 0;
    int maxK = 0, maxN = 0, maxT = 0;
    std::vector<double> Tall;
    QueryDesc* d_qd = nullptr;
    long long* d_pfx = nullptr;
    long long* d_qSlot = nullptr;
    long long* d_qItem = nullptr;
    long long* d_qMem = nullptr;
    int* d_rowRange = nullptr;
    long long capQ = -1;
    char* h_stage = nullptr;
    size_t stage_cap = 0;
    cudaEvent_t stage_ev = nullptr;
    bool stage_live = false;
    std::vector<char> last_stage;
    int tile = 0, ctas_per_sm = 0;    // pair-kernel configuration (0 = default)
    int tchunks = 0;                  // duration chunks per tile (0 = chosen per build)
    int pipeline = 0;                 // screened one-group FP32 pair kernel
    // batched search
    int sQ = 0;
    long long sTotN = 0;
    int sMaxN = 0;
    SearchQueryDesc* d_sqd = nullptr;
    long long capSQ = -1;
    char* h_sstage = nullptr;
    size_t sstage_cap = 0;
    cudaEvent_t sstage_ev = nullptr;
    bool sstage_live = false;
    std::vector<char> last_sstage;
    // host-sized scratch
    long long capN = -1, capK = -1, capR = -1, capW = -1, capL = -1;
    uint32_t* memMask = nullptr;
    int* counts = nullptr;
    int* members = nullptr;
    int* localIdx = nullptr;
    int* segKL = nullptr;
    float* centers = nullptr;
    double* blim64 = nullptr;
    float* A32 = nullptr;
    float* blim32 = nullptr;
    float* bc32 = nullptr;
    long long* resOff = nullptr;
    int* itemOff = nullptr;
    int* kPerm = nullptr;
    int* ntile = nullptr;
    int* tsize = nullptr;
    int* iRange = nullptr;
    int* memOff = nullptr;
    int* rowCount = nullptr;
    // device-sized scratch
    long long slotCap = 0, recheckCap = 0;
    long long want_slots = 0, want_rechecks = 0;
    uint32_t* resBits = nullptr;
    unsigned long long* resKey = nullptr;
    int* emitPre = nullptr;
    unsigned long long* recheck = nullptr;
    double* half64 = nullptr;         // FP64 cost halves of every state, duration and side (FP64 cost pass)
    long long half64Cap = 0;
    // search scratch
    long long capS = -1;
    unsigned long long* sdist = nullptr;
    unsigned long long* sbest = nullptr;
    unsigned long long* sbest16 = nullptr;  // [N][2] predecessor pairs of plan_search
    long long capS16 = -1;
    int* spred = nullptr;
    unsigned char* sfront = nullptr;
    long long capLast = -1;
    unsigned long long* slast = nullptr;
    unsigned long long* snear = nullptr;   // [4][SEARCH_MAX_BLOCKS]
    // keep-out cut
    std::vector<double> cutT;
    int cut_nT_cap = 0;
    double* d_cut64 = nullptr;
    float* d_cut32 = nullptr;
    double* h_cut64 = nullptr;
    float* h_cut32 = nullptr;
    cudaEvent_t cut_ev = nullptr;
    bool cut_ev_live = false;
    // MPC refinement QP
    double* d_mpc = nullptr;
    double* h_mpc = nullptr;
    int mpc_cap = 0;
    double* d_mpcJ = nullptr;
    long long mpc_jcap = 0;
    std::vector<double> mpc_last;   // table and horizon whose factor d_mpcJ holds
    cudaEvent_t mpc_ev = nullptr;
    bool mpc_ev_live = false;
    int smem_optin = 0;
    long long capCutE = -1, capCutO = -1, capCutR = -1;
    int32_t* cut_src = nullptr;
    uint32_t* cut_hit = nullptr;
    int32_t* cut_pos = nullptr;
    long long* cut_chunk = nullptr;
    float* cut_orow = nullptr;
    float* cut_okb = nullptr;
    float* cut_obox = nullptr;
    int* cut_ocount = nullptr;
    long long cut32Cap = 0, want_cut32 = 0;
    unsigned long long* cut_list32 = nullptr;
    // goal-rooted search (kept between calls for the warm start)
    long long capGoal = -1;
    double* g_d = nullptr;
    int* g_succ = nullptr;
    double* g_wsucc = nullptr;
    unsigned* g_anc = nullptr;
    int* g_prev = nullptr;
    // closest points / planes
    long long capPlO = -1, capPlR = -1, capPlE = -1, capPlP = -1;
    float* pl_orow = nullptr;
    float* pl_face = nullptr;
    float* pl_edge = nullptr;
    int* pl_nedge = nullptr;
    int* pl_ocount = nullptr;
    unsigned long long* pl_keys = nullptr;
    int32_t* pl_near = nullptr;
    float* pl_ub = nullptr;
    // timing
    bool timing = false;
    bool accounting = false;
    int max_sweeps = 0;
    long long spin_limit = 0;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pair, ev_search, ev_scan, ev_cut;
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
    if (m->interior != PLAN_INTERIOR_ELEVATE && m->interior != PLAN_INTERIOR_MINSNAP) return PLAN_ERR_INVALID_ARG;
    if (!std::isfinite(m->tighten) || m->tighten < 0) return PLAN_ERR_INVALID_ARG;
    for (int k = 0; k < m->gamma; ++k)
        if (!std::isfinite(m->bound[k]) || !(m->bound[k] - m->tighten > 0)) return PLAN_ERR_INVALID_ARG;
    if (!model_supported(m->m, m->gamma, m->degree) && !refine_supported(m->m, m->gamma, m->degree))
        return PLAN_ERR_UNSUPPORTED;
    if ((m->arith == PLAN_TF32 || m->arith == PLAN_BF16) && !tc_supported(m->m, m->gamma, m->degree))
        return PLAN_ERR_UNSUPPORTED;
    return PLAN_OK;
}

// Build the per-duration device tables (FP64 canonical and FP32 fast) for the
// concatenated durations of all queries and upload them asynchronously.
int upload_tables(plan_ctx* c, const std::vector<double>& Tall) {
    if (Tall == c->Tcache) return PLAN_OK;
    const TabLayout& L = c->L;
    const int g = c->model.gamma, p = c->model.degree, tg = L.tg;
    const int nT = (int)Tall.size();
    if (c->tab_ev_live) cudaEventSynchronize(c->tab_ev);  // staging buffers free again
    if (nT > c->tab_nT_cap) {
        if (c->h_tab64) cudaFreeHost(c->h_tab64);
        if (c->h_tab32) cudaFreeHost(c->h_tab32);
        c->h_tab64 = nullptr;
        c->h_tab32 = nullptr;
        c->tab_nT_cap = 0;
        const int cap = nT < NT_MAX ? NT_MAX : nT;
        if (!dalloc(c, &c->d_tab64, (long long)cap * L.e_stride) || !dalloc(c, &c->d_tab32, (long long)cap * L.f_stride))
            return PLAN_ERR_NO_MEMORY;
        if (cudaMallocHost((void**)&c->h_tab64, sizeof(double) * (size_t)cap * L.e_stride) != cudaSuccess ||
            cudaMallocHost((void**)&c->h_tab32, sizeof(float) * (size_t)cap * L.f_stride) != cudaSuccess)
            return fail(c, PLAN_ERR_NO_MEMORY, "cudaMallocHost tables");
        c->tab_nT_cap = cap;
    }
    std::vector<double> D((size_t)nT * (p + 1) * tg), H((size_t)nT * L.rax * tg), C((size_t)nT * g * p * tg);
    exact_tables(g, p, c->model.interior, nT, Tall.data(), D.data(), H.data(), C.data());
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
        const double* Dt = D.data() + (size_t)t * (p + 1) * tg;
        const double* Ht = H.data() + (size_t)t * L.rax * tg;
        const double* Ct = C.data() + (size_t)t * g * p * tg;
        double* e = c->h_tab64 + (size_t)t * L.e_stride;
        float* f = c->h_tab32 + (size_t)t * L.f_stride;
        memset(f, 0, sizeof(float) * L.f_stride);
        for (int i = 0; i < L.rax * tg; ++i) e[L.e_H + i] = Ht[i];
        for (int i = 0; i < (p + 1) * tg; ++i) e[L.e_D + i] = Dt[i];
        for (int i = 0; i < g * p * tg; ++i) e[L.e_C + i] = Ct[i];
        for (int rr = 0; rr < L.rax; ++rr) {
            const int r = order[rr];
            const double s = 1.0 / c->lim64[Hk[r] - 1];
            for (int col = 0; col < tg; ++col) {
                const float v = (float)(Ht[(size_t)r * tg + col] * s);
                f[L.f_H + rr * tg + col] = v;
                float& mx = f[L.f_HC + col];
                mx = fmaxf(mx, fabsf(v));
            }
        }
        for (int l = 1; l < p; ++l)
            for (int col = 0; col < tg; ++col) {
                const float v = (float)Dt[(size_t)l * tg + col];
                f[L.f_D + (l - 1) * tg + col] = v;
                float& mx = f[L.f_DC + col];
                mx = fmaxf(mx, fabsf(v));
            }
        for (int i = 0; i < g * p * tg; ++i) f[L.f_C + i] = (float)Ct[i];
    }
    cudaError_t e1 = cudaMemcpyAsync(c->d_tab64, c->h_tab64, sizeof(double) * (size_t)nT * L.e_stride,
                                     cudaMemcpyHostToDevice, c->stream);
    cudaError_t e2 = cudaMemcpyAsync(c->d_tab32, c->h_tab32, sizeof(float) * (size_t)nT * L.f_stride,
                                     cudaMemcpyHostToDevice, c->stream);
    if (e1 != cudaSuccess || e2 != cudaSuccess) return cuda_fail(c, e1 != cudaSuccess ? e1 : e2, "table upload");
    cudaEventRecord(c->tab_ev, c->stream);
    c->tab_ev_live = true;
    c->Tcache = Tall;
    return PLAN_OK;
}

int ensure_host_sized(plan_ctx* c, long long mask, long long list, long long k1, long long rows, long long nrow) {
    if (mask > c->capW) {
        if (!dalloc(c, &c->memMask, mask)) return PLAN_ERR_NO_MEMORY;
        c->capW = mask;
    }
    if (list > c->capL) {
        if (!dalloc(c, &c->members, list) || !dalloc(c, &c->localIdx, list) || !dalloc(c, &c->segKL, list))
            return PLAN_ERR_NO_MEMORY;
        c->capL = list;
    }
    if (k1 > c->capK) {
        if (!dalloc(c, &c->counts, k1) || !dalloc(c, &c->centers, 4 * k1) || !dalloc(c, &c->resOff, k1) ||
            !dalloc(c, &c->itemOff, k1) || !dalloc(c, &c->kPerm, k1) || !dalloc(c, &c->ntile, k1) || !dalloc(c, &c->tsize, k1) ||
            !dalloc(c, &c->iRange, k1) || !dalloc(c, &c->memOff, k1))
            return PLAN_ERR_NO_MEMORY;
        c->capK = k1;
    }
    if (rows > c->capR) {
        if (!dalloc(c, &c->blim64, rows) || !dalloc(c, &c->A32, 4 * rows) || !dalloc(c, &c->blim32, rows) ||
            !dalloc(c, &c->bc32, rows))
            return PLAN_ERR_NO_MEMORY;
        c->capR = rows;
    }
    if (nrow > c->capN) {
        if (!dalloc(c, &c->rowCount, nrow)) return PLAN_ERR_NO_MEMORY;
        c->capN = nrow;
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
    // the minimum-energy solve stays within exact 128-bit rationals up to degree 9
    if (model->interior != PLAN_INTERIOR_ELEVATE &&
        (model->interior != PLAN_INTERIOR_MINSNAP || model->degree > 9))
        return PLAN_ERR_INVALID_ARG;
    if (nT < 0 || (nT > 0 && (!T || !D || !H || !C))) return PLAN_ERR_INVALID_ARG;
    for (int t = 0; t < nT; ++t)
        if (!std::isfinite(T[t]) || !(T[t] > 0)) return PLAN_ERR_INVALID_ARG;
    try {
        exact_tables(model->gamma, model->degree, model->interior, nT, T, D, H, C);
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
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->stage_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->sstage_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->cut_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->mpc_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
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
    void* dev[] = {c->d_tab64, c->d_tab32, c->d_info, c->memMask, c->counts, c->members, c->localIdx, c->segKL, c->centers,
                   c->blim64, c->A32, c->blim32, c->bc32, c->resOff, c->itemOff, c->kPerm, c->ntile, c->tsize, c->iRange, c->rowCount,
                   c->resBits, c->resKey, c->emitPre, c->recheck, c->half64, c->sdist, c->sbest, c->sbest16, c->spred, c->sfront, c->slast, c->snear,
                   c->d_qd, c->d_pfx, c->d_qSlot, c->d_qItem, c->d_qMem, c->d_rowRange, c->d_sqd, c->memOff,
                   c->d_cut64, c->d_cut32, c->cut_src, c->cut_hit, c->cut_pos, c->cut_chunk, c->cut_orow,
                   c->cut_ocount, c->cut_list32, c->cut_okb, c->cut_obox, c->pl_orow, c->pl_face, c->pl_edge, c->pl_nedge, c->pl_ocount, c->pl_keys, c->pl_near, c->pl_ub, c->d_mpc, c->d_mpcJ, c->g_d, c->g_succ, c->g_wsucc, c->g_anc, c->g_prev};
    for (void* p : dev)
        if (p) cudaFree(p);
    if (c->h_tab64) cudaFreeHost(c->h_tab64);
    if (c->h_tab32) cudaFreeHost(c->h_tab32);
    if (c->h_info) cudaFreeHost(c->h_info);
    if (c->h_cut64) cudaFreeHost(c->h_cut64);
    if (c->h_mpc) cudaFreeHost(c->h_mpc);
    if (c->mpc_ev) cudaEventDestroy(c->mpc_ev);
    if (c->h_cut32) cudaFreeHost(c->h_cut32);
    if (c->cut_ev) cudaEventDestroy(c->cut_ev);
    if (c->h_stage) cudaFreeHost(c->h_stage);
    if (c->stage_ev) cudaEventDestroy(c->stage_ev);
    if (c->h_sstage) cudaFreeHost(c->h_sstage);
    if (c->sstage_ev) cudaEventDestroy(c->sstage_ev);
    if (c->tab_ev) cudaEventDestroy(c->tab_ev);
    for (auto& pr : c->ev_pair) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (auto& pr : c->ev_search) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (auto* lst : {&c->ev_scan, &c->ev_cut})
        for (auto& pr : *lst) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    delete c;
}

}  // extern "C"

namespace {

int check_query(plan_ctx* c, const plan_query& q) {
    if (q.N < 0 || q.N > (1 << 20)) return fail(c, PLAN_ERR_INVALID_ARG, "N out of range");
    if (q.nT < 1 || q.nT > NT_MAX || !q.T) return fail(c, PLAN_ERR_INVALID_ARG, "nT must be 1..32 with a host T array");
    for (int t = 0; t < q.nT; ++t)
        if (!std::isfinite(q.T[t]) || !(q.T[t] > 0)) return fail(c, PLAN_ERR_INVALID_ARG, "durations must be finite and > 0");
    if (q.K < 0 || q.K > 1024) return fail(c, PLAN_ERR_INVALID_ARG, "K must be 0..1024");
    if ((q.N > 0 && !q.states) || (q.K > 0 && (!q.poly_off || !q.A || !q.b)))
        return fail(c, PLAN_ERR_INVALID_ARG, "null input array");
    const plan_edges& o = q.out;
    if (!o.row_off || !o.count || o.cap < 0 || (o.cap > 0 && (!o.col || !o.w || !o.tidx || !o.mask)))
        return fail(c, PLAN_ERR_INVALID_ARG, "bad output CSR");
    if ((long long)q.K * q.N > (1LL << 31)) return fail(c, PLAN_ERR_INVALID_ARG, "K*N too large");
    return PLAN_OK;
}

// Host work of a batch: validation, offsets, tables, scratch, descriptor upload.
int prepare(plan_ctx* c, int Q, const plan_query* qs, int max_rows, int shard = 0, int nshard = 1) {
    if (!model_supported(c->model.m, c->model.gamma, c->model.degree))
        return fail(c, PLAN_ERR_UNSUPPORTED, "edge build not compiled for this (m, gamma, p)");
    if (Q < 1 || Q > 65535 || !qs) return fail(c, PLAN_ERR_INVALID_ARG, "need 1..65535 queries");
    int anyK = 0;
    for (int q = 0; q < Q; ++q) {
        int rc = check_query(c, qs[q]);
        if (rc != PLAN_OK) return rc;
        anyK |= qs[q].K > 0;
    }
    if (anyK && (max_rows < 1 || max_rows > RMAX)) return fail(c, PLAN_ERR_INVALID_ARG, "max_rows must be 1..16");
    if (!anyK) max_rows = 1;
    std::vector<QueryDesc> hq(Q);
    std::vector<long long> pfx(4 * (size_t)(Q + 1), 0);
    std::vector<double> Tall;
    long long mask = 0, poly = 0, rows = 0, nrow = 0, list = 0, k1 = 0;
    int maxK = 0, maxN = 0, maxT = 0;
    for (int q = 0; q < Q; ++q) {
        const plan_query& in = qs[q];
        if (in.nT > maxT) maxT = in.nT;
        QueryDesc& d = hq[q];
        memset(&d, 0, sizeof(d));
        d.N = in.N;
        d.K = in.K;
        d.nT = in.nT;
        d.W = in.K > 0 ? (in.K + 31) / 32 : 1;
        d.tabOff = (int)Tall.size();
        d.kOff = (int)k1;
        d.maskOff = mask;
        d.listOff = list;
        d.rowsOff = rows;
        d.rowOff = nrow;
        d.states = in.states;
        d.poly_off = in.poly_off;
        d.A = in.A;
        d.b = in.b;
        d.row_off = in.out.row_off;
        d.col = in.out.col;
        d.w = in.out.w;
        d.tidx = in.out.tidx;
        d.mask = in.out.mask;
        d.cap = in.out.cap;
        d.count = in.out.count;
        d.shard = shard;
        d.nshard = nshard;
        Tall.insert(Tall.end(), in.T, in.T + in.nT);
        pfx[0 * (Q + 1) + q] = mask;
        pfx[1 * (Q + 1) + q] = poly;
        pfx[2 * (Q + 1) + q] = rows;
        pfx[3 * (Q + 1) + q] = nrow;
        mask += (long long)in.N * d.W;
        poly += in.K;
        rows += (long long)in.K * max_rows;
        nrow += in.N;
        list += (long long)in.K * in.N;
        k1 += in.K + 1;
        if (in.K > maxK) maxK = in.K;
        if (in.N > maxN) maxN = in.N;
    }
    pfx[0 * (Q + 1) + Q] = mask;
    pfx[1 * (Q + 1) + Q] = poly;
    pfx[2 * (Q + 1) + Q] = rows;
    pfx[3 * (Q + 1) + Q] = nrow;
    if (Tall.size() > (size_t)(1 << 20)) return fail(c, PLAN_ERR_INVALID_ARG, "too many durations in the batch");
    int rc = upload_tables(c, Tall);
    if (rc != PLAN_OK) return rc;
    rc = ensure_host_sized(c, mask, list, k1, rows, nrow);
    if (rc != PLAN_OK) return rc;
    if (Q > c->capQ) {
        if (c->stage_live) cudaEventSynchronize(c->stage_ev);
        if (!dalloc(c, &c->d_qd, Q) || !dalloc(c, &c->d_pfx, 4LL * (Q + 1)) || !dalloc(c, &c->d_qSlot, Q + 1) ||
            !dalloc(c, &c->d_qItem, Q + 1) || !dalloc(c, &c->d_qMem, Q + 1) || !dalloc(c, &c->d_rowRange, 2LL * Q))
            return PLAN_ERR_NO_MEMORY;
        c->capQ = Q;
        c->last_stage.clear();
    }
    long long want_s = c->want_slots, want_r = c->want_rechecks;
    if (want_s == 0) {
        for (int q = 0; q < Q; ++q)
            want_s += 3LL * qs[q].N * (long long)qs[q].N / (qs[q].K > 0 ? qs[q].K : 1) + 1024;
    }
    if (want_r == 0) want_r = 1 << 16;
    rc = ensure_device_sized(c, want_s, want_r);
    if (rc != PLAN_OK) return rc;
    if (c->model.arith == PLAN_F64) {
        // the FP64 cost pass: both cost halves of every state and duration
        const int DR = c->model.cost_mode == PLAN_COST_POS ? 1 : c->model.gamma;
        const long long need = nrow * (long long)maxT * 2 * c->model.degree * DR * c->model.m;
        if (need > c->half64Cap) {
            if (c->stage_live) cudaEventSynchronize(c->stage_ev);
            if (!dalloc(c, &c->half64, need)) {
                c->half64Cap = 0;
                return PLAN_ERR_NO_MEMORY;
            }
            c->half64Cap = need;
        }
    }
    // descriptors + prefixes, uploaded only when they changed
    const size_t bytes = sizeof(QueryDesc) * Q + sizeof(long long) * pfx.size();
    std::vector<char> blob(bytes);
    memcpy(blob.data(), hq.data(), sizeof(QueryDesc) * Q);
    memcpy(blob.data() + sizeof(QueryDesc) * Q, pfx.data(), sizeof(long long) * pfx.size());
    if (blob != c->last_stage) {
        if (c->stage_live) cudaEventSynchronize(c->stage_ev);
        if (bytes > c->stage_cap) {
            if (c->h_stage) cudaFreeHost(c->h_stage);
            c->h_stage = nullptr;
            c->stage_cap = 0;
            if (cudaMallocHost((void**)&c->h_stage, bytes) != cudaSuccess) return fail(c, PLAN_ERR_NO_MEMORY, "stage");
            c->stage_cap = bytes;
        }
        memcpy(c->h_stage, blob.data(), bytes);
        cudaError_t e1 = cudaMemcpyAsync(c->d_qd, c->h_stage, sizeof(QueryDesc) * Q, cudaMemcpyHostToDevice, c->stream);
        cudaError_t e2 = cudaMemcpyAsync(c->d_pfx, c->h_stage + sizeof(QueryDesc) * Q, sizeof(long long) * pfx.size(),
                                         cudaMemcpyHostToDevice, c->stream);
        if (e1 != cudaSuccess || e2 != cudaSuccess) return cuda_fail(c, e1 != cudaSuccess ? e1 : e2, "descriptor upload");
        cudaEventRecord(c->stage_ev, c->stream);
        c->stage_live = true;
        c->last_stage.swap(blob);
    }
    c->bQ = Q;
    c->b_max_rows = max_rows;
    c->hq.swap(hq);
    c->pfx.swap(pfx);
    c->totMask = mask;
    c->totPoly = poly;
    c->totRows = rows;
    c->totN = nrow;
    c->totList = list;
    c->totK1 = k1;
    c->maxK = maxK;
    c->maxN = maxN;
    c->maxT = maxT;
    c->last_nT = Q == 1 ? qs[0].nT : 0;
    return PLAN_OK;
}

int default_tile(const plan_ctx* c) { return c->model.arith == PLAN_F64 ? TILE64 : TILE; }

// Launch the prepared batch (no host synchronisation, no allocation).
int issue(plan_ctx* c) {
    if (c->bQ < 1) return fail(c, PLAN_ERR_INVALID_ARG, "no prepared batch");
    cudaError_t e = cudaMemsetAsync(c->d_info, 0, sizeof(DevInfo), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset info");
    const int Q = c->bQ;
    BuildParams P;
    memset(&P, 0, sizeof(P));
    P.Q = Q;
    P.maxK = c->maxK;
    P.maxN = c->maxN;
    P.m = c->model.m;
    P.g = c->model.gamma;
    P.p = c->model.degree;
    P.cost_mode = c->model.cost_mode;
    P.in_f32 = c->model.input == PLAN_IN_F32;
    // FP64 model: by default the FP32 pair kernels decide the bits (banded
    // margins re-checked in canonical FP64, so the bits are the FP64 ones) and
    // a canonical FP64 pass computes the costs of the emitted edges; pipeline
    // PLAN_PIPE_FP64 runs the canonical FP64 pair kernel instead
    const bool canonical64 = c->model.arith == PLAN_F64 && c->pipeline == PIPE_FP64;
    P.arith = (c->model.arith == PLAN_F64 && !canonical64) ? PLAN_F32 : c->model.arith;
    P.w64 = c->model.arith == PLAN_F64;
    P.cost64 = c->model.arith == PLAN_F64 && !canonical64;
    P.maxT = c->maxT;
    P.half64 = c->half64;
    P.max_rows = c->b_max_rows;
    P.tile = (P.arith == PLAN_F64) ? TILE64
             : (P.arith == PLAN_F32) ? (c->tile > 0 ? c->tile : TILE)
                                     : TILE;  // tensor-core form: 64-state tiles, 256 threads
    // the canonical FP64 kernel: one duration per item by default (it is bound
    // by the narrow FP64 pipe; small problems need the items to fill every SM)
    P.tchunks = c->tchunks > 0 ? c->tchunks : (P.arith == PLAN_F64 ? 8 : 2);
    // default chunking: about eight items per SM once the tile count is known
    P.itemTarget = c->tchunks > 0 ? 0 : 8 * c->num_sms;
    P.pipeline = canonical64 ? 0 : c->pipeline;
    P.eps = c->model.tighten;
    P.qd = c->d_qd;
    P.pfxMask = c->d_pfx;
    P.pfxPoly = c->d_pfx + (Q + 1);
    P.pfxRows = c->d_pfx + 2 * (Q + 1);
    P.pfxN = c->d_pfx + 3 * (Q + 1);
    P.qSlot = c->d_qSlot;
    P.qItem = c->d_qItem;
    P.qMem = c->d_qMem;
    P.totMask = c->totMask;
    P.totPoly = c->totPoly;
    P.totRows = c->totRows;
    P.totN = c->totN;
    P.tab32 = c->d_tab32;
    P.tab64 = c->d_tab64;
    for (int k = 0; k < 4; ++k) P.lim64[k] = c->lim64[k];
    P.L = c->L;
    P.memMask = c->memMask;
    P.counts = c->counts;
    P.members = c->members;
    P.localIdx = c->localIdx;
    P.segKL = c->segKL;
    P.centers = c->centers;
    P.blim64 = c->blim64;
    P.A32 = c->A32;
    P.blim32 = c->blim32;
    P.bc32 = c->bc32;
    P.resOff = c->resOff;
    P.itemOff = c->itemOff;
    P.kPerm = c->kPerm;
    P.ntile = c->ntile;
    P.tsize = c->tsize;
    P.iRange = c->iRange;
    P.rowRange = c->d_rowRange;
    P.memOff = c->memOff;
    P.resBits = c->resBits;
    P.resKey = c->resKey;
    P.emitPre = c->emitPre;
    P.recheck = c->recheck;
    P.rowCount = c->rowCount;
    P.slotCap = c->slotCap;
    P.recheckCap = c->recheckCap;
    P.info = c->d_info;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->timing) {
        e0 = take_event(c);
        e1 = take_event(c);
        c->ev_pair.emplace_back(e0, e1);
    }
    int launches = 0;
    int ce = launch_build(P, c->stream, c->num_sms, c->ctas_per_sm, e0, e1, &launches);
    c->launches += launches;
    if (ce != 0) return cuda_fail(c, (cudaError_t)ce, "build launch");
    if (c->accounting && c->totN > 0 && c->totPoly > 0) {
        ce = launch_account(P, c->stream, c->num_sms, c->d_info->work);
        if (ce != 0) return cuda_fail(c, (cudaError_t)ce, "accounting launch");
    }
    return PLAN_OK;
}

}  // namespace

extern "C" {

int plan_build_edges(plan_ctx* c, int N, const void* states, int nT, const double* T, int K,
                     const int32_t* poly_off, int max_rows, const void* A, const void* b, const plan_edges* out) {
    if (!c) return PLAN_ERR_INVALID_ARG;
    if (!out) return fail(c, PLAN_ERR_INVALID_ARG, "bad output CSR");
    plan_query q;
    q.N = N;
    q.states = states;
    q.nT = nT;
    q.T = T;
    q.K = K;
    q.poly_off = poly_off;
    q.A = A;
    q.b = b;
    q.out = *out;
    int rc = prepare(c, 1, &q, max_rows);
    if (rc != PLAN_OK) return rc;
    return issue(c);
}

int plan_build_edges_shard(plan_ctx* c, int N, const void* states, int nT, const double* T, int K,
                           const int32_t* poly_off, int max_rows, const void* A, const void* b, int shard, int nshard,
                           const plan_edges* out) {
    if (!c) return PLAN_ERR_INVALID_ARG;
    if (!out) return fail(c, PLAN_ERR_INVALID_ARG, "bad output CSR");
    if (nshard < 1 || nshard > 1024 || shard < 0 || shard >= nshard)
        return fail(c, PLAN_ERR_INVALID_ARG, "need 0 <= shard < nshard <= 1024");
    plan_query q;
    q.N = N;
    q.states = states;
    q.nT = nT;
    q.T = T;
    q.K = K;
    q.poly_off = poly_off;
    q.A = A;
    q.b = b;
    q.out = *out;
    int rc = prepare(c, 1, &q, max_rows, shard, nshard);
    if (rc != PLAN_OK) return rc;
    return issue(c);
}

int plan_prepare_batched(plan_ctx* c, int Q, const plan_query* queries, int max_rows) {
    if (!c) return PLAN_ERR_INVALID_ARG;
    return prepare(c, Q, queries, max_rows);
}

int plan_build_edges_batched(plan_ctx* c) {
    if (!c) return PLAN_ERR_INVALID_ARG;
    return issue(c);
}

int plan_set_tile(plan_ctx* c, int tile, int ctas_per_sm, int tchunks, int pipeline) {
    if (!c || tile < 0 || ctas_per_sm < 0 || ctas_per_sm > 8 || tchunks < 0 || tchunks > NT_MAX || pipeline < 0 ||
        pipeline > PIPE_FP64 || (pipeline == PIPE_FP64 && c->model.arith != PLAN_F64))
        return PLAN_ERR_INVALID_ARG;
    c->pipeline = pipeline;
    if (tile != 0 && (tile < 8 || tile > TILE || (tile & 3))) return fail(c, PLAN_ERR_INVALID_ARG, "tile must be 8..64, multiple of 4");
    c->tile = tile;
    c->ctas_per_sm = ctas_per_sm;
    c->tchunks = tchunks;
    return PLAN_OK;
}

int plan_autotune(plan_ctx* c, int reps, int* best_tile, int* best_ctas, int* best_chunks, int* best_pipeline,
                  double* best_ms) {
    if (!c || reps < 1) return PLAN_ERR_INVALID_ARG;
    if (c->bQ < 1) return fail(c, PLAN_ERR_INVALID_ARG, "prepare a batch first");
    if (c->model.arith != PLAN_F32 && c->model.arith != PLAN_F64) {  // the tensor-core kernel has fixed tiles
        if (best_tile) *best_tile = TILE;
        if (best_ctas) *best_ctas = 0;
        if (best_chunks) *best_chunks = 2;
        if (best_pipeline) *best_pipeline = 0;
        return PLAN_OK;
    }
    const bool was_timing = c->timing;
    // candidates: the screened one-group kernel over tile sides, the
    // unscreened one and the warp-specialised one (64-state tiles); every one
    // over duration chunks
    struct Cand { int pipe, tile, ctas; };
    const Cand cands[] = {{0, 64, 0}, {0, 48, 0}, {0, 32, 0}, {2, 64, 0}, {1, 64, 0}};
    const int chunks[] = {1, 2, 4, 8};
    double best = 1e30;
    int bt = TILE, bc = 0, bk = 2, bp = 0;
    for (const Cand& cd : cands)
        for (int ch : chunks) {
            const int cc = cd.ctas, t = cd.tile;
            c->pipeline = cd.pipe;
            c->tile = t;
            c->ctas_per_sm = cc;
            c->tchunks = ch;
            // one untimed run sizes the scratch for this configuration
            for (int tries = 0; tries < 4; ++tries) {
                int rc = issue(c);
                if (rc != PLAN_OK) return rc;
                plan_info info;
                rc = plan_wait(c, &info);
                if (rc == PLAN_OK) break;
                if (rc != PLAN_ERR_CAPACITY || info.detail == DET_OUTPUT) {
                    c->timing = was_timing;
                    return rc;
                }
            }
            c->timing = true;
            double pm = 0;
            int64_t pl = 0;
            plan_timing(c, nullptr, nullptr, nullptr, nullptr, nullptr, 1);
            for (int r = 0; r < reps; ++r) {
                int rc = issue(c);
                if (rc != PLAN_OK) return rc;
            }
            plan_timing(c, &pm, &pl, nullptr, nullptr, nullptr, 1);
            c->timing = was_timing;
            const double ms = pl ? pm / pl : 1e30;
            if (ms < best) {
                best = ms;
                bt = t;
                bc = cc;
                bk = ch;
                bp = cd.pipe;
            }
        }
    c->tile = bt;
    c->ctas_per_sm = bc;
    c->tchunks = bk;
    c->pipeline = bp;
    if (best_tile) *best_tile = bt;
    if (best_ctas) *best_ctas = bc;
    if (best_chunks) *best_chunks = bk;
    if (best_pipeline) *best_pipeline = bp;
    if (best_ms) *best_ms = best;
    return PLAN_OK;
}

}  // extern "C"

namespace {

// plan_search and plan_search_at: start/goal from the host (start_pos,
// goal_pos) or from device memory at run time (endpoints).
int search_common(plan_ctx* c, int N, const void* states, const plan_edges* edges, const double* start_pos,
                  const double* goal_pos, const double* endpoints, int32_t* path, int path_cap, int32_t* path_len,
                  double* cost) {
    if (!c) return PLAN_ERR_INVALID_ARG;
    if (N < 1 || N > (1 << 20) || !states) return fail(c, PLAN_ERR_INVALID_ARG, "need N >= 1 states");
    if (!edges || !edges->row_off || !edges->count || edges->cap < 0 || (edges->cap > 0 && (!edges->col || !edges->w)))
        return fail(c, PLAN_ERR_INVALID_ARG, "bad CSR");
    if ((!endpoints && (!start_pos || !goal_pos)) || !path || path_cap < 1 || !path_len || !cost)
        return fail(c, PLAN_ERR_INVALID_ARG, "bad search output");
    if (!endpoints)
        for (int a = 0; a < c->model.m; ++a)
            if (!std::isfinite(start_pos[a]) || !std::isfinite(goal_pos[a]))
                return fail(c, PLAN_ERR_INVALID_ARG, "start/goal must be finite");
    if (N > c->capS) {
        if (!dalloc(c, &c->sdist, N) || !dalloc(c, &c->sbest, N) || !dalloc(c, &c->spred, N) ||
            !dalloc(c, &c->sfront, 2LL * N))
            return PLAN_ERR_NO_MEMORY;
        c->capS = N;
    }
    if (N > c->capS16) {
        if (!dalloc(c, &c->sbest16, 2LL * N)) return PLAN_ERR_NO_MEMORY;
        c->capS16 = N;
    }
    if (N > c->capLast) {
        if (!dalloc(c, &c->slast, N)) return PLAN_ERR_NO_MEMORY;
        c->capLast = N;
    }
    if (!c->snear && !dalloc(c, &c->snear, 4LL * SEARCH_MAX_BLOCKS)) return PLAN_ERR_NO_MEMORY;
    if (c->num_sms > SEARCH_MAX_BLOCKS) return fail(c, PLAN_ERR_UNSUPPORTED, "more SMs than the search scratch holds");
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
    if (!endpoints)
        for (int a = 0; a < c->model.m; ++a) {
            S.start[a] = start_pos[a];
            S.goal[a] = goal_pos[a];
        }
    S.endpoints = endpoints;
    S.dist = c->sdist;
    S.bestU = c->sbest;
    S.best16 = c->sbest16;
    S.pred = c->spred;
    S.last = c->slast;
    S.near_blk = c->snear;
    S.path = path;
    S.path_cap = path_cap;
    S.path_len = path_len;
    S.cost = cost;
    S.info = c->d_info;
    S.max_sweeps = c->max_sweeps > 0 ? c->max_sweeps : N + 1;
    S.spin_limit = c->spin_limit > 0 ? c->spin_limit : (1LL << 24);
    cudaError_t e = cudaMemsetAsync(&c->d_info->bar[0], 0, sizeof(unsigned long long) * 3, c->stream);
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

}  // namespace

extern "C" {

int plan_search(plan_ctx* c, int N, const void* states, const plan_edges* edges, const double* start_pos,
                const double* goal_pos, int32_t* path, int path_cap, int32_t* path_len, double* cost) {
    return search_common(c, N, states, edges, start_pos, goal_pos, nullptr, path, path_cap, path_len, cost);
}

int plan_search_at(plan_ctx* c, int N, const void* states, const plan_edges* edges, const double* endpoints,
                   int32_t* path, int path_cap, int32_t* path_len, double* cost) {
    if (!endpoints) return fail(c, PLAN_ERR_INVALID_ARG, "null endpoints");
    return search_common(c, N, states, edges, nullptr, nullptr, endpoints, path, path_cap, path_len, cost);
}

}  // extern "C"

namespace {

// FP64 canonical tables (control points, cost rows; the edge build's layout)
// and the FP32 control-point table of the cut's durations, uploaded once per
// distinct duration list.
int upload_cut_tables(plan_ctx* c, int nT, const double* T) {
    std::vector<double> Tv(T, T + nT);
    if (Tv == c->cutT) return PLAN_OK;
    const TabLayout& L = c->L;
    const int g = c->model.gamma, p = c->model.degree, tg = L.tg;
    const int f_stride = (p + 1) * tg;
    if (c->cut_ev_live) cudaEventSynchronize(c->cut_ev);
    if (nT > c->cut_nT_cap) {
        if (c->h_cut64) cudaFreeHost(c->h_cut64);
        if (c->h_cut32) cudaFreeHost(c->h_cut32);
        c->h_cut64 = nullptr;
        c->h_cut32 = nullptr;
        c->cut_nT_cap = 0;
        if (!dalloc(c, &c->d_cut64, (long long)NT_MAX * L.e_stride) || !dalloc(c, &c->d_cut32, (long long)NT_MAX * f_stride))
            return PLAN_ERR_NO_MEMORY;
        if (cudaMallocHost((void**)&c->h_cut64, sizeof(double) * (size_t)NT_MAX * L.e_stride) != cudaSuccess ||
            cudaMallocHost((void**)&c->h_cut32, sizeof(float) * (size_t)NT_MAX * f_stride) != cudaSuccess)
            return fail(c, PLAN_ERR_NO_MEMORY, "cudaMallocHost cut tables");
        c->cut_nT_cap = NT_MAX;
    }
    std::vector<double> D((size_t)nT * (p + 1) * tg), H((size_t)nT * L.rax * tg), C((size_t)nT * g * p * tg);
    exact_tables(g, p, c->model.interior, nT, T, D.data(), H.data(), C.data());
    for (int t = 0; t < nT; ++t) {
        const double* Dt = D.data() + (size_t)t * (p + 1) * tg;
        const double* Ht = H.data() + (size_t)t * L.rax * tg;
        const double* Ct = C.data() + (size_t)t * g * p * tg;
        double* e = c->h_cut64 + (size_t)t * L.e_stride;
        float* f = c->h_cut32 + (size_t)t * f_stride;
        for (int i = 0; i < L.rax * tg; ++i) e[L.e_H + i] = Ht[i];
        for (int i = 0; i < (p + 1) * tg; ++i) e[L.e_D + i] = Dt[i];
        for (int i = 0; i < g * p * tg; ++i) e[L.e_C + i] = Ct[i];
        for (int i = 0; i < (p + 1) * tg; ++i) f[i] = (float)Dt[i];
    }
    cudaError_t e1 = cudaMemcpyAsync(c->d_cut64, c->h_cut64, sizeof(double) * (size_t)nT * L.e_stride,
                                     cudaMemcpyHostToDevice, c->stream);
    cudaError_t e2 = cudaMemcpyAsync(c->d_cut32, c->h_cut32, sizeof(float) * (size_t)nT * f_stride,
                                     cudaMemcpyHostToDevice, c->stream);
    if (e1 != cudaSuccess || e2 != cudaSuccess) return cuda_fail(c, e1 != cudaSuccess ? e1 : e2, "cut table upload");
    cudaEventRecord(c->cut_ev, c->stream);
    c->cut_ev_live = true;
    c->cutT = Tv;
    return PLAN_OK;
}

}  // namespace

extern "C" {

int plan_cut_edges(plan_ctx* c, int N, const void* states, int nT, const double* T, const plan_edges* in,
                   const plan_obstacles* obst, const plan_edges* out) {
    if (!c) return PLAN_ERR_INVALID_ARG;
    if (!model_supported(c->model.m, c->model.gamma, c->model.degree) || c->model.m < 2 || c->model.m > 3)
        return fail(c, PLAN_ERR_UNSUPPORTED, "keep-out cut not compiled for this (m, gamma, p)");
    if (N < 0 || N > (1 << 20) || (N > 0 && !states)) return fail(c, PLAN_ERR_INVALID_ARG, "N out of range");
    if (nT < 1 || nT > NT_MAX || !T) return fail(c, PLAN_ERR_INVALID_ARG, "nT must be 1..32 with a host T array");
    for (int t = 0; t < nT; ++t)
        if (!std::isfinite(T[t]) || !(T[t] > 0)) return fail(c, PLAN_ERR_INVALID_ARG, "durations must be finite and > 0");
    if (!in || !in->row_off || !in->count || in->cap < 0 ||
        (in->cap > 0 && (!in->col || !in->w || !in->tidx || !in->mask)))
        return fail(c, PLAN_ERR_INVALID_ARG, "bad input CSR");
    if (!out || !out->row_off || !out->count || out->cap < 0 ||
        (out->cap > 0 && (!out->col || !out->w || !out->tidx || !out->mask)))
        return fail(c, PLAN_ERR_INVALID_ARG, "bad output CSR");
    if (out->row_off == in->row_off || (out->cap > 0 && in->cap > 0 && (out->col == in->col || out->w == in->w ||
                                                                         out->tidx == in->tidx || out->mask == in->mask)))
        return fail(c, PLAN_ERR_INVALID_ARG, "input and output CSR must not share arrays");
    if (in->cap > (1LL << 31) - 2) return fail(c, PLAN_ERR_INVALID_ARG, "input CSR capacity above 2^31 - 2");
    // A and b may be null when no obstacle has rows (the device checks it per obstacle)
    if (!obst || obst->n < 0 || obst->n > (1 << 20) || (obst->n > 0 && !obst->off))
        return fail(c, PLAN_ERR_INVALID_ARG, "bad obstacles");
    if (obst->n > 0 && (obst->max_rows < 1 || obst->max_rows > CUT_RMAX))
        return fail(c, PLAN_ERR_INVALID_ARG, "obstacle max_rows must be 1..16");
    int rc = upload_cut_tables(c, nT, T);
    if (rc != PLAN_OK) return rc;
    const long long capE = in->cap > 0 ? in->cap : 1;
    const long long nchunks = (capE + CUT_CHUNK - 1) / CUT_CHUNK;
    if (capE > c->capCutE) {
        if (!dalloc(c, &c->cut_src, capE) || !dalloc(c, &c->cut_hit, capE) || !dalloc(c, &c->cut_pos, capE + 1) ||
            !dalloc(c, &c->cut_chunk, nchunks + 1)) {
            c->capCutE = -1;
            return PLAN_ERR_NO_MEMORY;
        }
        c->capCutE = capE;
    }
    const int maxr = obst->n > 0 ? obst->max_rows : 1;
    const long long nob = obst->n > 0 ? obst->n : 1;
    if (nob > c->capCutO || nob * maxr > c->capCutR) {
        if (!dalloc(c, &c->cut_ocount, nob) || !dalloc(c, &c->cut_orow, 4 * nob * maxr) ||
            !dalloc(c, &c->cut_okb, 2 * nob * maxr) || !dalloc(c, &c->cut_obox, 8 * nob)) {
            c->capCutO = c->capCutR = -1;
            return PLAN_ERR_NO_MEMORY;
        }
        c->capCutO = nob;
        c->capCutR = nob * maxr;
    }
    const long long w32 = c->want_cut32 > 0 ? c->want_cut32 : (1LL << 18);
    if (w32 > c->cut32Cap) {
        if (!dalloc(c, &c->cut_list32, w32)) {
            c->cut32Cap = 0;
            return PLAN_ERR_NO_MEMORY;
        }
        c->cut32Cap = w32;
    }
    CutParams C;
    memset(&C, 0, sizeof(C));
    C.m = c->model.m;
    C.g = c->model.gamma;
    C.p = c->model.degree;
    C.nT = nT;
    C.in_f32 = c->model.input == PLAN_IN_F32;
    C.w_f64 = c->model.arith == PLAN_F64;
    C.cost_mode = c->model.cost_mode;
    C.N = N;
    C.n_obst = obst->n;
    C.max_orows = maxr;
    C.states = states;
    C.row_in = in->row_off;
    C.col_in = in->col;
    C.w_in = in->w;
    C.t_in = in->tidx;
    C.mask_in = in->mask;
    C.count_in = in->count;
    C.cap_in = in->cap;
    C.row_out = out->row_off;
    C.col_out = out->col;
    C.w_out = out->w;
    C.t_out = out->tidx;
    C.mask_out = out->mask;
    C.count_out = out->count;
    C.cap_out = out->cap;
    C.obst_off = obst->off;
    C.A = obst->A;
    C.b = obst->b;
    C.orow = c->cut_orow;
    C.okb = c->cut_okb;
    C.obox = c->cut_obox;
    C.ocount = c->cut_ocount;
    C.tab64 = c->d_cut64;
    C.tab32 = c->d_cut32;
    C.L = c->L;
    C.src = c->cut_src;
    C.hit = c->cut_hit;
    C.list32 = c->cut_list32;
    C.cap32 = c->cut32Cap;
    C.chunk = c->cut_chunk;
    C.pos = c->cut_pos;
    C.nchunks = nchunks;
    C.info = c->d_info;
    cudaError_t e = cudaMemsetAsync(&c->d_info->cut_units, 0, 9 * sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset cut counters");
    cudaEvent_t s0 = nullptr, s1 = nullptr, c0 = nullptr, c1 = nullptr;
    if (c->timing) {
        s0 = take_event(c);
        s1 = take_event(c);
        c0 = take_event(c);
        c1 = take_event(c);
        c->ev_scan.emplace_back(s0, s1);
        c->ev_cut.emplace_back(c0, c1);
        cudaEventRecord(c0, c->stream);
    }
    int launches = 0;
    int ce = launch_cut(C, c->stream, c->num_sms, &launches, s0, s1);
    if (c->timing) cudaEventRecord(c1, c->stream);
    c->launches += launches;
    if (ce != 0) return cuda_fail(c, (cudaError_t)ce, "cut launch");
    return PLAN_OK;
}

int plan_search_to(plan_ctx* c, int N, const void* states, const plan_edges* edges, const double* endpoints, int warm,
                   int32_t* path, int path_cap, int32_t* path_len, double* cost) {
    if (!c) return PLAN_ERR_INVALID_ARG;
    if (N < 1 || N > (1 << 20) || !states) return fail(c, PLAN_ERR_INVALID_ARG, "need N >= 1 states");
    if (!edges || !edges->row_off || !edges->count || edges->cap < 0 || (edges->cap > 0 && (!edges->col || !edges->w)))
        return fail(c, PLAN_ERR_INVALID_ARG, "bad CSR");
    if (!endpoints || !path || path_cap < 1 || !path_len || !cost) return fail(c, PLAN_ERR_INVALID_ARG, "bad search output");
    if (N > c->capGoal) {
        if (!dalloc(c, &c->g_d, N) || !dalloc(c, &c->g_succ, N) || !dalloc(c, &c->g_wsucc, N) ||
            !dalloc(c, &c->g_anc, 2LL * N) || !dalloc(c, &c->g_prev, 2)) {
            c->capGoal = -1;
            return PLAN_ERR_NO_MEMORY;
        }
        c->capGoal = N;
        cudaError_t e = cudaMemsetAsync(c->g_prev, 0xff, 2 * sizeof(int), c->stream);  // no previous call
        if (e != cudaSuccess) return cuda_fail(c, e, "memset search state");
    }
    if (!c->snear && !dalloc(c, &c->snear, 4LL * SEARCH_MAX_BLOCKS)) return PLAN_ERR_NO_MEMORY;
    if (c->num_sms > SEARCH_MAX_BLOCKS) return fail(c, PLAN_ERR_UNSUPPORTED, "more SMs than the search scratch holds");
    GoalSearchParams G;
    memset(&G, 0, sizeof(G));
    G.N = N;
    G.m = c->model.m;
    G.n = c->model.m * c->model.gamma;
    G.in_f32 = c->model.input == PLAN_IN_F32;
    G.w_f64 = c->model.arith == PLAN_F64;
    G.warm = warm != 0;
    G.max_sweeps = c->max_sweeps > 0 ? c->max_sweeps : N + 1;
    G.states = states;
    G.row_off = edges->row_off;
    G.col = edges->col;
    G.w = edges->w;
    G.count = edges->count;
    G.cap = edges->cap;
    G.endpoints = endpoints;
    G.d = c->g_d;
    G.succ = c->g_succ;
    G.wsucc = c->g_wsucc;
    G.anc = c->g_anc;
    G.near_blk = c->snear;
    G.prev = c->g_prev;
    G.spin_limit = c->spin_limit > 0 ? c->spin_limit : (1LL << 24);
    G.path = path;
    G.path_cap = path_cap;
    G.path_len = path_len;
    G.cost = cost;
    G.info = c->d_info;
    cudaError_t e = cudaMemsetAsync(&c->d_info->bar[0], 0, sizeof(unsigned long long) * 3, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset barrier");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->timing) {
        e0 = take_event(c);
        e1 = take_event(c);
        c->ev_search.emplace_back(e0, e1);
        cudaEventRecord(e0, c->stream);
    }
    int launches = 0;
    int ce = launch_search_to(G, c->stream, c->num_sms, &launches);
    if (c->timing) cudaEventRecord(e1, c->stream);
    c->launches += launches;
    if (ce != 0) return cuda_fail(c, (cudaError_t)ce, "search launch");
    return PLAN_OK;
}

static int planes_common(plan_ctx* c, int P, const void* points, const plan_obstacles* obst, float* closest,
                         float* plane, float* dist, int32_t* nearest, float* nearest_dist, float* nearest_plane) {
    if (!c) return PLAN_ERR_INVALID_ARG;
    const int m = c->model.m;
    if (m < 2 || m > 3) return fail(c, PLAN_ERR_UNSUPPORTED, "closest points for m = 2 or 3 only");
    if (P < 0 || P > (1 << 24) || (P > 0 && !points)) return fail(c, PLAN_ERR_INVALID_ARG, "bad points");
    if (!obst || obst->n < 0 || obst->n > (1 << 20) || (obst->n > 0 && !obst->off))
        return fail(c, PLAN_ERR_INVALID_ARG, "bad obstacles");
    if (obst->n > 0 && (obst->max_rows < 1 || obst->max_rows > CUT_RMAX))
        return fail(c, PLAN_ERR_INVALID_ARG, "obstacle max_rows must be 1..16");
    if ((long long)P * obst->n > (1LL << 40)) return fail(c, PLAN_ERR_INVALID_ARG, "too many (point, obstacle) pairs");
    const int maxr = obst->n > 0 ? obst->max_rows : 1;
    const long long nob = obst->n > 0 ? obst->n : 1;
    const int max_edges = m == 2 ? maxr : (maxr * (maxr - 1)) / 2 > 0 ? (maxr * (maxr - 1)) / 2 : 1;
    if (nob > c->capPlO || nob * maxr > c->capPlR || nob * max_edges > c->capPlE) {
        if (!dalloc(c, &c->pl_ocount, nob) || !dalloc(c, &c->pl_orow, 4 * nob * maxr) ||
            !dalloc(c, &c->pl_face, 4 * nob * maxr) || !dalloc(c, &c->pl_edge, 16 * nob * max_edges) ||
            !dalloc(c, &c->pl_nedge, nob)) {
            c->capPlO = c->capPlR = c->capPlE = -1;
            return PLAN_ERR_NO_MEMORY;
        }
        c->capPlO = nob;
        c->capPlR = nob * maxr;
        c->capPlE = nob * max_edges;
    }
    const bool want_near = nearest || nearest_dist || nearest_plane;
    if (want_near && P > c->capPlP) {
        if (!dalloc(c, &c->pl_keys, P) || !dalloc(c, &c->pl_near, P) || !dalloc(c, &c->pl_ub, P)) {
            c->capPlP = -1;
            return PLAN_ERR_NO_MEMORY;
        }
        c->capPlP = P;
    }
    if (nearest_plane && !nearest) nearest = c->pl_near;   // the pair pass needs the indices
    PlanesParams Q;
    memset(&Q, 0, sizeof(Q));
    Q.m = m;
    Q.in_f32 = c->model.input == PLAN_IN_F32;
    Q.P = P;
    Q.n_obst = obst->n;
    Q.max_orows = maxr;
    Q.points = points;
    Q.obst_off = obst->off;
    Q.A = obst->A;
    Q.b = obst->b;
    Q.orow = c->pl_orow;
    Q.max_edges = max_edges;
    Q.face = c->pl_face;
    Q.edge = c->pl_edge;
    Q.nedge = c->pl_nedge;
    Q.ocount = c->pl_ocount;
    Q.closest = closest;
    Q.plane = plane;
    Q.dist = dist;
    Q.nearest = nearest;
    Q.nearest_dist = nearest_dist;
    Q.keys = want_near ? c->pl_keys : nullptr;
    // nearest only (no per-pair output): prune pairs by distance bounds
    Q.ub = want_near && !closest && !plane && !dist ? c->pl_ub : nullptr;
    Q.nearest_plane = nearest_plane;
    Q.info = c->d_info;
    cudaError_t e = cudaSuccess;
    if (want_near && P > 0) e = cudaMemsetAsync(c->pl_keys, 0xff, sizeof(unsigned long long) * (size_t)P, c->stream);
    if (e == cudaSuccess && Q.ub && P > 0) e = cudaMemsetAsync(c->pl_ub, 0x7f, sizeof(float) * (size_t)P, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset planes scratch");
    int launches = 0;
    int ce = launch_planes(Q, c->stream, c->num_sms, &launches);
    c->launches += launches;
    if (ce != 0) return cuda_fail(c, (cudaError_t)ce, "planes launch");
    return PLAN_OK;
}

int plan_obstacle_planes(plan_ctx* c, int P, const void* points, const plan_obstacles* obst, float* closest,
                         float* plane, float* dist, int32_t* nearest, float* nearest_dist) {
    return planes_common(c, P, points, obst, closest, plane, dist, nearest, nearest_dist, nullptr);
}

int plan_nearest_planes(plan_ctx* c, int P, const void* points, const plan_obstacles* obst, float* nearest_plane,
                        int32_t* nearest, float* nearest_dist) {
    if (c && P > 0 && !nearest_plane) return fail(c, PLAN_ERR_INVALID_ARG, "null nearest_plane");
    return planes_common(c, P, points, obst, nullptr, nullptr, nullptr, nearest, nearest_dist, nearest_plane);
}

int plan_mpc_qp(plan_ctx* c, int B, const plan_mpc_params* prm, const double* x0, const double* ref,
                const float* planes, double* x, double* u, double* obj, int32_t* status, int32_t* iters,
                double* nodes) {
    if (!c) return PLAN_ERR_INVALID_ARG;
    const int m = c->model.m, g = c->model.gamma, p = c->model.degree, n = m * g;
    if (m < 1 || m > 3 || g < 1 || g > 4 || p < 2 * g - 1 || p > 9)
        return fail(c, PLAN_ERR_UNSUPPORTED, "MPC QP for m <= 3, gamma <= 4, degree <= 9");
    if (!prm) return fail(c, PLAN_ERR_INVALID_ARG, "null MPC parameters");
    const int H = prm->horizon;
    if (H < g || (long long)m * H > MPC_NV_MAX) return fail(c, PLAN_ERR_INVALID_ARG, "horizon must be gamma .. 64/m");
    if (!std::isfinite(prm->dt) || !(prm->dt > 0.0)) return fail(c, PLAN_ERR_INVALID_ARG, "dt must be finite and > 0");
    if (!prm->Q || !prm->F || !prm->R || !prm->V) return fail(c, PLAN_ERR_INVALID_ARG, "null weights");
    for (int i = 0; i < n; ++i)
        if (!(prm->Q[i] > 0.0) || !(prm->F[i] > 0.0) || !(prm->V[i] > 0.0) || !std::isfinite(prm->Q[i]) ||
            !std::isfinite(prm->F[i]) || !std::isfinite(prm->V[i]))
            return fail(c, PLAN_ERR_INVALID_ARG, "weights must be finite and > 0");
    for (int i = 0; i < m; ++i)
        if (!(prm->R[i] > 0.0) || !std::isfinite(prm->R[i])) return fail(c, PLAN_ERR_INVALID_ARG, "weights must be finite and > 0");
    const int nk = prm->keepin_rows;
    if (nk < 0 || nk > MPC_KEEP_MAX || (nk > 0 && (!prm->keepin_A || !prm->keepin_b)))
        return fail(c, PLAN_ERR_INVALID_ARG, "keep-in rows must be 0..16 with host arrays");
    for (int i = 0; i < nk * m; ++i)
        if (!std::isfinite(prm->keepin_A[i])) return fail(c, PLAN_ERR_INVALID_ARG, "keep-in rows must be finite");
    for (int i = 0; i < nk; ++i)
        if (!std::isfinite(prm->keepin_b[i])) return fail(c, PLAN_ERR_INVALID_ARG, "keep-in rows must be finite");
    if (B < 0 || B > (1 << 24)) return fail(c, PLAN_ERR_INVALID_ARG, "B out of range");
    if (B > 0 && (!x0 || !ref || !planes || !x || !u || !obj || !status))
        return fail(c, PLAN_ERR_INVALID_ARG, "null MPC array");
    const int rax = reach_rows(g, p);
    // one warp (problem) per CTA: the FP64 pipe of every SM is the bound, and
    // small CTAs let the scheduler spread the problems evenly over the SMs
    const int W = 1;
    if (mpc_smem(m, g, p, rax, nk, H, W) > (size_t)c->smem_optin ||
        mpc_setup_smem(m, g, p, rax, nk, H) > (size_t)c->smem_optin)
        return fail(c, PLAN_ERR_UNSUPPORTED, "MPC problem too large for shared memory");
    // the table: per-axis transition A[c][c'] = dt^(c'-c)/(c'-c)!, input
    // column B[c] = dt^(g-c)/(g-c)!, D and reach rows of duration dt, the
    // bound of every reach row, weights, keep-in rows
    const int ts = mpc_table_size(m, g, p, rax, nk);
    if ((long long)m * H * m * H > c->mpc_jcap) {
        c->mpc_last.clear();
        if (!dalloc(c, &c->d_mpcJ, (long long)m * H * m * H)) return PLAN_ERR_NO_MEMORY;
        c->mpc_jcap = (long long)m * H * m * H;
    }
    if (ts > c->mpc_cap) {
        if (c->mpc_ev_live) cudaEventSynchronize(c->mpc_ev);
        if (c->h_mpc) cudaFreeHost(c->h_mpc);
        c->h_mpc = nullptr;
        c->mpc_cap = 0;
        if (!dalloc(c, &c->d_mpc, ts)) return PLAN_ERR_NO_MEMORY;
        if (cudaMallocHost((void**)&c->h_mpc, sizeof(double) * (size_t)ts) != cudaSuccess)
            return fail(c, PLAN_ERR_NO_MEMORY, "pinned MPC table");
        c->mpc_cap = ts;
    }
    if (c->mpc_ev_live) cudaEventSynchronize(c->mpc_ev);   // the previous upload has left the pinned buffer
    std::vector<double> D((size_t)(p + 1) * 2 * g), Hr((size_t)rax * 2 * g), Cc((size_t)g * p * 2 * g);
    const double dt = prm->dt;
    exact_tables(g, p, c->model.interior, 1, &dt, D.data(), Hr.data(), Cc.data());
    double* t = c->h_mpc;
    int o = 0;
    auto taylor = [&](int k) {  // dt^k / k!
        double v = 1.0;
        for (int i = 1; i <= k; ++i) v = v * dt / (double)i;
        return v;
    };
    for (int r = 0; r < g; ++r)
        for (int cc = 0; cc < g; ++cc) t[o++] = cc >= r ? taylor(cc - r) : 0.0;
    for (int r = 0; r < g; ++r) t[o++] = taylor(g - r);
    for (double v : D) t[o++] = v;
    for (double v : Hr) t[o++] = v;
    for (int ord = 1, r = 0; ord <= g; ++ord)
        for (int j = 0; j <= p - ord; ++j, ++r) t[o++] = c->lim64[ord - 1];
    for (int i = 0; i < n; ++i) t[o++] = prm->Q[i];
    for (int i = 0; i < n; ++i) t[o++] = prm->F[i];
    for (int i = 0; i < n; ++i) t[o++] = prm->V[i];
    for (int i = 0; i < m; ++i) t[o++] = prm->R[i];
    for (int i = 0; i < nk * m; ++i) t[o++] = prm->keepin_A[i];
    for (int i = 0; i < nk; ++i) t[o++] = prm->keepin_b[i];
    if (o != ts) return fail(c, PLAN_ERR_INVALID_ARG, "internal: MPC table size");
    cudaError_t e = cudaMemcpyAsync(c->d_mpc, c->h_mpc, sizeof(double) * (size_t)ts, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "MPC table upload");
    cudaEventRecord(c->mpc_ev, c->stream);
    c->mpc_ev_live = true;
    MpcParams M;
    memset(&M, 0, sizeof(M));
    M.B = B;
    M.m = m;
    M.g = g;
    M.p = p;
    M.H = H;
    M.nv = m * H;
    M.rax = rax;
    M.nkeep = nk;
    M.warps = W;
    const long long rows = (long long)H * m * rax * 2 + (long long)H * (p + 1) + (long long)H * p * nk;
    M.max_iter = (int)(4 * (rows + m * H) + 64);
    M.tab = c->d_mpc;
    M.x0 = x0;
    M.ref = ref;
    M.planes = planes;
    M.x = x;
    M.u = u;
    M.obj = obj;
    M.status = status;
    M.iters = iters;
    M.nodes = nodes;
    M.J0 = c->d_mpcJ;
    // the factor depends on the table (model, dt, weights, keep-in rows
    // included, a superset) and the horizon only
    std::vector<double> key(c->h_mpc, c->h_mpc + ts);
    key.push_back((double)H);
    key.push_back((double)m);
    key.push_back((double)g);
    key.push_back((double)p);
    M.j0_ready = key == c->mpc_last ? 1 : 0;
    int launches = 0;
    int ce = launch_mpc(M, c->stream, &launches);
    c->launches += launches;
    if (ce != 0) {
        c->mpc_last.clear();
        return cuda_fail(c, (cudaError_t)ce, "MPC launch");
    }
    c->mpc_last.swap(key);
    return PLAN_OK;
}

int plan_prepare_search_batched(plan_ctx* c, int Q, const plan_search_query* qs) {
    if (!c) return PLAN_ERR_INVALID_ARG;
    if (Q < 1 || Q > 65535 || !qs) return fail(c, PLAN_ERR_INVALID_ARG, "need 1..65535 queries");
    std::vector<SearchQueryDesc> hq(Q);
    long long tot = 0;
    int maxN = 0;
    for (int q = 0; q < Q; ++q) {
        const plan_search_query& in = qs[q];
        if (in.N < 1 || in.N > (1 << 20) || !in.states) return fail(c, PLAN_ERR_INVALID_ARG, "need N >= 1 states");
        const plan_edges& e = in.edges;
        if (!e.row_off || !e.count || e.cap < 0 || (e.cap > 0 && (!e.col || !e.w)))
            return fail(c, PLAN_ERR_INVALID_ARG, "bad CSR");
        if (!in.path || in.path_cap < 1 || !in.path_len || !in.cost || !in.status)
            return fail(c, PLAN_ERR_INVALID_ARG, "bad search output");
        for (int a2 = 0; a2 < c->model.m; ++a2)
            if (!std::isfinite(in.start_pos[a2]) || !std::isfinite(in.goal_pos[a2]))
                return fail(c, PLAN_ERR_INVALID_ARG, "start/goal must be finite");
        SearchQueryDesc& d = hq[q];
        memset(&d, 0, sizeof(d));
        d.N = in.N;
        d.off = tot;
        d.states = in.states;
        d.row_off = e.row_off;
        d.col = e.col;
        d.w = e.w;
        d.count = e.count;
        d.cap = e.cap;
        for (int a2 = 0; a2 < 4; ++a2) {
            d.start[a2] = a2 < c->model.m ? in.start_pos[a2] : 0.0;
            d.goal[a2] = a2 < c->model.m ? in.goal_pos[a2] : 0.0;
        }
        d.path = in.path;
        d.path_cap = in.path_cap;
        d.path_len = in.path_len;
        d.cost = in.cost;
        d.status = in.status;
        tot += in.N;
        if (in.N > maxN) maxN = in.N;
    }
    if (tot > c->capS) {
        if (!dalloc(c, &c->sdist, tot) || !dalloc(c, &c->sbest, tot) || !dalloc(c, &c->spred, tot) ||
            !dalloc(c, &c->sfront, 2LL * tot))
            return PLAN_ERR_NO_MEMORY;
        c->capS = tot;
    }
    if (Q > c->capSQ) {
        if (c->sstage_live) cudaEventSynchronize(c->sstage_ev);
        if (!dalloc(c, &c->d_sqd, Q)) return PLAN_ERR_NO_MEMORY;
        c->capSQ = Q;
        c->last_sstage.clear();
    }
    const size_t bytes = sizeof(SearchQueryDesc) * Q;
    std::vector<char> blob(bytes);
    memcpy(blob.data(), hq.data(), bytes);
    if (blob != c->last_sstage) {
        if (c->sstage_live) cudaEventSynchronize(c->sstage_ev);
        if (bytes > c->sstage_cap) {
            if (c->h_sstage) cudaFreeHost(c->h_sstage);
            c->h_sstage = nullptr;
            c->sstage_cap = 0;
            if (cudaMallocHost((void**)&c->h_sstage, bytes) != cudaSuccess) return fail(c, PLAN_ERR_NO_MEMORY, "stage");
            c->sstage_cap = bytes;
        }
        memcpy(c->h_sstage, blob.data(), bytes);
        cudaError_t e = cudaMemcpyAsync(c->d_sqd, c->h_sstage, bytes, cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "search descriptor upload");
        cudaEventRecord(c->sstage_ev, c->stream);
        c->sstage_live = true;
        c->last_sstage.swap(blob);
    }
    c->sQ = Q;
    c->sTotN = tot;
    c->sMaxN = maxN;
    return PLAN_OK;
}

int plan_search_batched(plan_ctx* c) {
    if (!c) return PLAN_ERR_INVALID_ARG;
    if (c->sQ < 1) return fail(c, PLAN_ERR_INVALID_ARG, "no prepared search batch");
    BatchSearchParams B;
    memset(&B, 0, sizeof(B));
    B.Q = c->sQ;
    B.m = c->model.m;
    B.n = c->model.m * c->model.gamma;
    B.in_f32 = c->model.input == PLAN_IN_F32;
    B.w_f64 = c->model.arith == PLAN_F64;
    B.max_sweeps = c->max_sweeps > 0 ? c->max_sweeps : c->sMaxN + 1;
    B.qd = c->d_sqd;
    B.dist = c->sdist;
    B.bestU = c->sbest;
    B.pred = c->spred;
    B.front = c->sfront;
    B.info = c->d_info;
    int launches = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->timing) {
        e0 = take_event(c);
        e1 = take_event(c);
        c->ev_search.emplace_back(e0, e1);
        cudaEventRecord(e0, c->stream);
    }
    int ce = launch_search_batched(B, c->stream, &launches);
    if (c->timing) cudaEventRecord(e1, c->stream);
    c->launches += launches;
    if (ce != 0) return cuda_fail(c, (cudaError_t)ce, "batched search launch");
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
    // the status covers the work issued since the previous plan_wait: clear it
    e = cudaMemset(c->d_info, 0, 2 * sizeof(int));
    if (e != cudaSuccess) return cuda_fail(c, e, "clear status");
    const DevInfo& d = *c->h_info;
    if (d.status == PLAN_ERR_CAPACITY) {
        if (d.detail == DET_SLOTS) c->want_slots = (long long)(d.need_slots + d.need_slots / 4 + 1024);
        if (d.detail == DET_RECHECK) {
            long long need = (long long)(d.need_rechecks > d.rechecks ? d.need_rechecks : d.rechecks);
            c->want_rechecks = need + need / 4 + 1024;
        }
        if (d.detail == DET_CUTLIST) {
            c->want_cut32 = (long long)(d.cut_near + d.cut_near / 4 + 4096);
        }
    }
    if (info) {
        memset(info, 0, sizeof(*info));
        info->status = d.status;
        info->detail = d.detail;
        info->memberships = (int64_t)d.memberships;
        info->slots = (int64_t)d.slots;
        info->candidates = (int64_t)d.candidates;
        info->checks = (int64_t)d.checks;
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
        info->screened = (int64_t)d.screened;
        info->cut_units = (int64_t)d.cut_units;
        info->cut_tests = (int64_t)d.cut_tests;
        info->cut_box = (int64_t)d.cut_box;
        info->cut_near = (int64_t)d.cut_near;
        info->cut_step1 = (int64_t)d.cut_step1;
        info->cut_step2 = (int64_t)d.cut_step2;
        info->cut_games = (int64_t)d.cut_games;
        info->cut_lp64 = (int64_t)d.cut_lp64;
        info->cut_ties = (int64_t)d.cut_ties;
        info->shard_lo = d.shard_lo;
        info->shard_hi = d.shard_hi;
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

int plan_cut_timing(plan_ctx* c, double* scan_ms, double* cut_ms, int64_t* cuts, int reset) {
    if (!c) return PLAN_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream sync");
    double a = 0, b = 0;
    for (auto& pr : c->ev_scan) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) a += ms;
    }
    for (auto& pr : c->ev_cut) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) b += ms;
    }
    cudaGetLastError();
    if (scan_ms) *scan_ms = a;
    if (cut_ms) *cut_ms = b;
    if (cuts) *cuts = (int64_t)c->ev_cut.size();
    if (reset) {
        for (auto* lst : {&c->ev_scan, &c->ev_cut}) {
            for (auto& pr : *lst) {
                c->ev_pool.push_back(pr.first);
                c->ev_pool.push_back(pr.second);
            }
            lst->clear();
        }
    }
    return PLAN_OK;
}

}  // extern "C"
