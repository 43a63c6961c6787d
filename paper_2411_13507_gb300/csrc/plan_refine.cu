// Differentiable refinement objective for sm_103a: one thread per Bezier
// segment (the axes one after the other), forward (loss) and hand-written backward (d loss / d control points
// and d loss / d T) of
//
//   loss = w_snap J_snap + mu sum_r phi_delta(margin_r)
//
// with the reach margins c_k -/+ Q^(k)_j (Theorem 1 read per axis on the
// hodograph control points Q^(k)_j = p!/(p-k)! T^-k Delta^k P_j), the free
// margins b_r - A_r P_l of the interior control points (Property 1), the
// relaxed log-barrier phi_delta (-log m above delta, its C^2 quadratic
// extension below) and the snap energy
//   J_snap = (p!/(p-4)!)^2 T^-7 sum_jl G_jl <Delta^4 P_j, Delta^4 P_l>,
//   G_jl = C(q,j) C(q,l) / ((2q+1) C(2q,j+l)),  q = p-4,
// the exact integral of ||b''''||^2 over [0, T].  The backward pass applies
// the adjoint of the forward-difference operator (x_l = g_{l-1} - g_l) to the
// margin and snap gradients.
#include <cuda_runtime.h>

#include <cstdint>

#include "plan_internal.h"

namespace plan {

#define DEVI __device__ __forceinline__

namespace {

DEVI float phi_f(float m, float delta, float log_delta) {
    if (m >= delta) return -logf(m);
    const float z = (m - 2.f * delta) / delta;
    return -log_delta + 0.5f * z * z - 0.5f;
}
DEVI float dphi_f(float m, float delta) { return m >= delta ? -1.f / m : (m - 2.f * delta) / (delta * delta); }

constexpr float fact_f(int n) { return n <= 1 ? 1.f : n * fact_f(n - 1); }
constexpr int comb_i(int n, int k) { return (k < 0 || k > n) ? 0 : (k == 0 || k == n ? 1 : comb_i(n - 1, k - 1) + comb_i(n - 1, k)); }

template <int M, int L>
DEVI void fwd_diff(float (&d)[8][M], int len) {  // d[0..len-2] = d[j+1] - d[j]
#pragma unroll
    for (int j = 0; j < L - 1; ++j)
        if (j < len - 1)
#pragma unroll
            for (int a = 0; a < M; ++a) d[j][a] = d[j + 1][a] - d[j][a];
}

// adjoint of the forward difference: g has `len` entries -> len+1 entries
template <int M, int L>
DEVI void adj_diff(float (&g)[8][M], int len) {
    float out[8][M];
#pragma unroll
    for (int l = 0; l < L; ++l)
#pragma unroll
        for (int a = 0; a < M; ++a) {
            float v = 0.f;
            if (l >= 1 && l - 1 < len) v += g[l - 1][a];
            if (l < len) v -= g[l][a];
            out[l][a] = (l <= len) ? v : 0.f;
        }
#pragma unroll
    for (int l = 0; l < L; ++l)
#pragma unroll
        for (int a = 0; a < M; ++a) g[l][a] = out[l][a];
}

}  // namespace

template <int M, int G, int PD, bool GRAD>
__global__ void __launch_bounds__(128) k_refine(RefineParams R) {
    constexpr int L = PD + 1;
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= R.S) return;
    const float* Ps = R.P + s * L * M;
    const float T = R.T[s];
    const float Ti = 1.f / T;
    const float mu = R.mu, delta = R.delta, ld = logf(R.delta), ws = R.w_snap;
    const float up = GRAD ? R.grad_loss[s] : 1.f;
    float loss = 0.f, dT = 0.f;
    float* dPs = GRAD ? R.dP + s * L * M : nullptr;

    // Reach margins and snap energy separate over the axes (Theorem 1 per
    // axis; the snap integral is the sum of the axes' integrals): one axis
    // at a time keeps few values live.  Its gradient goes straight to dP.
#pragma unroll 1
    for (int a = 0; a < M; ++a) {
        float Pa[8][1];
#pragma unroll
        for (int l = 0; l < 8; ++l) Pa[l][0] = l < L ? Ps[l * M + a] : 0.f;
        float ga[8];
#pragma unroll
        for (int l = 0; l < 8; ++l) ga[l] = 0.f;
#pragma unroll
        for (int k = 1; k <= G; ++k) {
            float d[8][1];
#pragma unroll
            for (int l = 0; l < 8; ++l) d[l][0] = Pa[l][0];
#pragma unroll
            for (int it = 0; it < k; ++it) fwd_diff<1, L>(d, L - it);
            float sk = fact_f(PD) / fact_f(PD - k);
#pragma unroll
            for (int it = 0; it < k; ++it) sk *= Ti;
            const float ck = R.bound[k - 1];
            const int nk = L - k;
            float g[8][1];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                g[j][0] = 0.f;
                if (j < nk) {
                    const float Q = sk * d[j][0];
                    const float m1 = ck - Q, m2 = ck + Q;
                    loss += mu * (phi_f(m1, delta, ld) + phi_f(m2, delta, ld));
                    if (GRAD) {
                        const float gQ = mu * (dphi_f(m2, delta) - dphi_f(m1, delta)) * up;
                        g[j][0] = gQ * sk;
                        dT += gQ * Q * (-(float)k) * Ti;
                    }
                }
            }
            if (GRAD) {
#pragma unroll
                for (int it = k; it >= 1; --it) adj_diff<1, L>(g, L - it);
#pragma unroll
                for (int l = 0; l < L; ++l) ga[l] += g[l][0];
            }
        }
        {
            constexpr int q = PD - 4;
            float d4[8][1];
#pragma unroll
            for (int l = 0; l < 8; ++l) d4[l][0] = Pa[l][0];
#pragma unroll
            for (int it = 0; it < 4; ++it) fwd_diff<1, L>(d4, L - it);
            float c = fact_f(PD) / fact_f(PD - 4);
            c = c * c;
            float t7 = Ti * Ti * Ti;
            t7 = t7 * t7 * Ti;
            c *= t7;
            float quad = 0.f;
            float gd[8][1];
#pragma unroll
            for (int j = 0; j < 8; ++j) gd[j][0] = 0.f;
#pragma unroll
            for (int j = 0; j <= q; ++j)
#pragma unroll
                for (int l = 0; l <= q; ++l) {
                    const float Gjl = (float)(comb_i(q, j) * comb_i(q, l)) / (float)((2 * q + 1) * comb_i(2 * q, j + l));
                    quad = fmaf(Gjl * d4[j][0], d4[l][0], quad);
                    if (GRAD) gd[j][0] = fmaf(Gjl, d4[l][0], gd[j][0]);
                }
            const float J = c * quad;
            loss += ws * J;
            if (GRAD) {
                const float f = ws * c * 2.f * up;
#pragma unroll
                for (int j = 0; j < 8; ++j) gd[j][0] = (j <= q) ? gd[j][0] * f : 0.f;
#pragma unroll
                for (int it = 4; it >= 1; --it) adj_diff<1, L>(gd, L - it);
#pragma unroll
                for (int l = 0; l < L; ++l) ga[l] += gd[l][0];
                dT += ws * (-7.f) * J * Ti * up;
            }
        }
        if (GRAD) {
#pragma unroll
            for (int l = 0; l < L; ++l) dPs[l * M + a] = ga[l];
        }
    }
    // free-space margins of the interior control points (every axis)
    float P[8][M];
#pragma unroll
    for (int l = 1; l < PD; ++l)
#pragma unroll
        for (int a = 0; a < M; ++a) P[l][a] = Ps[l * M + a];
    float df[8][M];
#pragma unroll
    for (int l = 0; l < 8; ++l)
#pragma unroll
        for (int a = 0; a < M; ++a) df[l][a] = 0.f;
    const int nr = min(R.nrows[s], R.rmax);
    for (int r = 0; r < nr; ++r) {
        float Ar[M];
#pragma unroll
        for (int a = 0; a < M; ++a) Ar[a] = R.A[(s * R.rmax + r) * M + a];
        const float br = R.b[s * R.rmax + r];
#pragma unroll
        for (int l = 1; l < PD; ++l) {
            float dot = 0.f;
#pragma unroll
            for (int a = 0; a < M; ++a) dot = fmaf(Ar[a], P[l][a], dot);
            const float mg = br - dot;
            loss += mu * phi_f(mg, delta, ld);
            if (GRAD) {
                const float gm = mu * dphi_f(mg, delta) * up;
#pragma unroll
                for (int a = 0; a < M; ++a) df[l][a] -= gm * Ar[a];
            }
        }
    }
    if (R.loss) R.loss[s] = loss;
    if (GRAD) {
#pragma unroll
        for (int l = 1; l < PD; ++l)
#pragma unroll
            for (int a = 0; a < M; ++a) dPs[l * M + a] += df[l][a];
        R.dT[s] = dT;
    }
}

bool refine_supported(int m, int g, int p) { return (m == 3 && g == 3 && p == 7) || (m == 2 && g == 2 && p == 5); }

int launch_refine(const RefineParams& R, void* stream, int* launches) {
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned nb = (unsigned)((R.S + 127) / 128);
    if (R.S == 0) return 0;
    const bool grad = R.grad_loss != nullptr;
    if (R.m == 3 && R.g == 3 && R.p == 7) {
        if (grad) k_refine<3, 3, 7, true><<<nb, 128, 0, st>>>(R);
        else k_refine<3, 3, 7, false><<<nb, 128, 0, st>>>(R);
    } else if (R.m == 2 && R.g == 2 && R.p == 5) {
        if (grad) k_refine<2, 2, 5, true><<<nb, 128, 0, st>>>(R);
        else k_refine<2, 2, 5, false><<<nb, 128, 0, st>>>(R);
    } else {
        return (int)cudaErrorInvalidValue;
    }
    ++*launches;
    return (int)cudaGetLastError();
}

}  // namespace plan
