// Measured issue rate of the FP32 (and FP64) lane operations the pair kernels
// are made of, for the roofline of the edge build (the paper has no counterpart: this
// is a measurement helper).  A reach or free row costs one add and one
// max (of an absolute value, for reach rows) per pair; a cost segment is
// mostly fused multiply-adds.  Each kernel below runs independent chains of
// one of these mixes in registers, with every thread of a full-occupancy
// grid busy, and the host times it with CUDA events.
#include <cuda_runtime.h>

#include "plan.h"

namespace {

constexpr int CHAINS = 8;

// add then |.|-max per chain step: the reach-row pattern (2 lane ops)
__global__ void __launch_bounds__(256) k_lane_addmax(float* out, float x, int iters) {
    float a[CHAINS], m[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) {
        a[i] = (float)(threadIdx.x & 7) * 1e-3f + (float)i;
        m[i] = 0.f;
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < CHAINS; ++i) {
            a[i] = a[i] + x;
            m[i] = fmaxf(m[i], fabsf(a[i]));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) s += m[i];
    if (s == -1.f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never true; keeps the chains live
}

// fused multiply-add per chain step (1 lane op)
__global__ void __launch_bounds__(256) k_lane_fma(float* out, float x, float y, int iters) {
    float a[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) a[i] = (float)(threadIdx.x & 7) * 1e-3f + (float)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < CHAINS; ++i) a[i] = fmaf(a[i], y, x);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) s += a[i];
    if (s == -1.f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// the FP64 counterparts (the canonical FP64 pair kernel and the re-check)
__global__ void __launch_bounds__(256) k_lane_addmax64(double* out, double x, int iters) {
    double a[CHAINS], m[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) {
        a[i] = (double)(threadIdx.x & 7) * 1e-3 + (double)i;
        m[i] = 0.0;
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < CHAINS; ++i) {
            a[i] = a[i] + x;
            m[i] = fmax(m[i], fabs(a[i]));
        }
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) s += m[i];
    if (s == -1.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_lane_fma64(double* out, double x, double y, int iters) {
    double a[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) a[i] = (double)(threadIdx.x & 7) * 1e-3 + (double)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < CHAINS; ++i) a[i] = fma(a[i], y, x);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) s += a[i];
    if (s == -1.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int plan_measure_lane_rate(int mix, int iters, double* lane_ops_per_s, double* ms) {
    if (mix < 0 || mix > 3 || iters < 1 || iters > (1 << 24) || !lane_ops_per_s) return PLAN_ERR_INVALID_ARG;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PLAN_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PLAN_ERR_CUDA;
    if (cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess) return PLAN_ERR_CUDA;
    const int threads = 256;
    const int blocks = sms * (per_sm / threads);
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = PLAN_ERR_CUDA;
    float t = 0.f;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return PLAN_ERR_CUDA;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) goto done;
    for (int rep = 0; rep < 2; ++rep) {  // the first launch warms up
        cudaEventRecord(e0, st);
        if (mix == 0) k_lane_addmax<<<blocks, threads, 0, st>>>(nullptr, 1e-7f, iters);
        else if (mix == 1) k_lane_fma<<<blocks, threads, 0, st>>>(nullptr, 1e-7f, 0.999999f, iters);
        else if (mix == 2) k_lane_addmax64<<<blocks, threads, 0, st>>>(nullptr, 1e-7, iters);
        else k_lane_fma64<<<blocks, threads, 0, st>>>(nullptr, 1e-7, 0.999999, iters);
        cudaEventRecord(e1, st);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) goto done;
    }
    if (cudaEventElapsedTime(&t, e0, e1) != cudaSuccess || t <= 0.f) goto done;
    *lane_ops_per_s = (double)blocks * threads * (double)iters * CHAINS * (mix % 2 == 0 ? 2.0 : 1.0) / (t * 1e-3);
    if (ms) *ms = t;
    rc = PLAN_OK;
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    return rc;
}
