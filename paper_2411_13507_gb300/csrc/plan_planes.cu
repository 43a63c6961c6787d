// closestPoint and adjacentHyperplane for sm_103a (arXiv 2411.13507,
// Algorithm 2; Sec. III-D: the separating hyperplane between an MPC node and
// an obstacle).
//
// For a point v outside a convex obstacle O = {z : A z <= b} the closest
// point (the Euclidean projection onto O) lies in the relative interior of a
// face, on an edge, or at a vertex.  A prep step computes, in FP64 once per
// obstacle, every facet's unit normal and offset and every edge of O as a
// segment: a base point, a unit direction and the parameter interval the
// other facets leave (a facet or pair of facets with an empty interval is not
// a face or an edge; an unbounded edge keeps an infinite end).  Per (point,
// obstacle), in FP32: inside O (every row <= 0) -> distance 0; otherwise the
// nearest of the projections onto the faces that land inside O (m = 3; in 2-D
// the faces are the edges) and of the closest points of the edge segments
// (parameter clamped to its interval, which also covers the vertices).  Every
// candidate is a point of O, so the nearest one is the projection.  The
// segments come rounded from FP64, so the FP32 error does not grow with how
// sharp a vertex is (no linear solve happens per pair).  The plane:
// h = (v - z) / |v - z|, l = h . z.
#include <cuda_runtime.h>

#include <cstdint>

#include "plan_internal.h"

namespace plan {

namespace {

#define PDEV __device__ __forceinline__

constexpr float U32P = 5.9604644775390625e-08f;  // 2^-24
constexpr int EDGE_F4 = 4;  // float4 per edge record

PDEV void p_status(DevInfo* info, int code, int detail) {
    if (atomicCAS(&info->status, 0, code) == 0) atomicExch(&info->detail, detail);
}
PDEV bool p_failed(const DevInfo* info) { return *((volatile const int*)&info->status) != 0; }
PDEV float pld32(const void* p, long long i, int f32) {
    return f32 ? ((const float*)p)[i] : (float)((const double*)p)[i];
}

// Obstacle rows as {A_0, A_1, A_2, b} (FP32, for the inside test), max_orows
// per obstacle, with row-count checks.
__global__ void k_planes_prep(PlanesParams Q) {
    const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= (long long)Q.n_obst * Q.max_orows) return;
    const int o = (int)(u / Q.max_orows), k = (int)(u % Q.max_orows);
    const int r0 = Q.obst_off[o], nr = Q.obst_off[o + 1] - r0;
    if (nr < 0 || nr > Q.max_orows || r0 < 0 || (nr > 0 && (!Q.A || !Q.b))) {
        if (k == 0) p_status(Q.info, nr > Q.max_orows ? PLAN_ERR_UNSUPPORTED : PLAN_ERR_INVALID_ARG, DET_ROWS);
        if (k == 0) Q.ocount[o] = 0;
        return;
    }
    if (k == 0) Q.ocount[o] = nr;
    if (k < nr) {
        const long long r = r0 + k;
        float4 f;
        f.x = pld32(Q.A, r * Q.m, Q.in_f32);
        f.y = pld32(Q.A, r * Q.m + 1, Q.in_f32);
        f.z = Q.m == 3 ? pld32(Q.A, r * Q.m + 2, Q.in_f32) : 0.f;
        f.w = pld32(Q.b, r, Q.in_f32);
        reinterpret_cast<float4*>(Q.orow)[u] = f;
    }
}

PDEV double pld64(const void* p, long long i, int f32) {
    return f32 ? (double)((const float*)p)[i] : ((const double*)p)[i];
}

// The interval of t along z0 + t d that every row leaves (t_lo > t_hi: none)
// and the rows that set its ends (-1 for an infinite end).
template <int M>
PDEV void clip_line(const PlanesParams& Q, int r0, int nr, const double* z0, const double* d, double& tlo, double& thi,
                    int& rlo, int& rhi) {
    const double inf = __longlong_as_double(0x7FF0000000000000ll);
    tlo = -inf;
    thi = inf;
    rlo = rhi = -1;
    for (int r = 0; r < nr; ++r) {
        double ad = 0.0, az = 0.0;
#pragma unroll
        for (int a = 0; a < M; ++a) {
            const double A = pld64(Q.A, (long long)(r0 + r) * M + a, Q.in_f32);
            ad = fma(A, d[a], ad);
            az = fma(A, z0[a], az);
        }
        const double slack = pld64(Q.b, r0 + r, Q.in_f32) - az;
        const double scale = fabs(pld64(Q.b, r0 + r, Q.in_f32)) + 1.0;
        if (fabs(ad) <= 1e-12) {
            if (slack < -1e-12 * scale) {  // parallel to the line and excluding it
                tlo = inf;
                thi = -inf;
            }
        } else if (ad > 0.0) {
            if (slack / ad < thi) {
                thi = slack / ad;
                rhi = r;
            }
        } else {
            if (slack / ad > tlo) {
                tlo = slack / ad;
                rlo = r;
            }
        }
    }
}

// Unit normal and offset of row r (FP64).
template <int M>
PDEV void unit_row(const PlanesParams& Q, int r0, int r, double* n, double& c) {
    double n2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) n[a] = 0.0;
#pragma unroll
    for (int a = 0; a < M; ++a) {
        n[a] = pld64(Q.A, (long long)(r0 + r) * M + a, Q.in_f32);
        n2 = fma(n[a], n[a], n2);
    }
    const double rn = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
#pragma unroll
    for (int a = 0; a < M; ++a) n[a] *= rn;
    c = pld64(Q.b, r0 + r, Q.in_f32) * rn;
}

// One warp per obstacle: faces (unit normal, offset) and edges, compacted;
// FP64, rounded to FP32 at the end.  Edge record (4 float4): base point and
// t_lo; unit direction and t_hi; then in 2-D the unit normals of the rows
// that end the segment at t_lo and t_hi (zero at an infinite end) and the
// edge's own unit normal and offset, in 3-D the unit normals of its two
// facets.
template <int M>
__global__ void __launch_bounds__(128) k_planes_geom(PlanesParams Q) {
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long o = gw; o < Q.n_obst; o += nw) {
        const int r0 = Q.obst_off[o];
        int nr = Q.obst_off[o + 1] - r0;
        if (nr < 0 || nr > Q.max_orows || r0 < 0 || (nr > 0 && (!Q.A || !Q.b))) nr = 0;
        float4* face = reinterpret_cast<float4*>(Q.face) + o * Q.max_orows;
        float4* edge = reinterpret_cast<float4*>(Q.edge) + EDGE_F4 * o * Q.max_edges;
        // faces
        for (int r = lane; r < Q.max_orows; r += 32) {
            float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r < nr) {
                double A[3] = {0.0, 0.0, 0.0}, n2 = 0.0;
#pragma unroll
                for (int a = 0; a < M; ++a) {
                    A[a] = pld64(Q.A, (long long)(r0 + r) * M + a, Q.in_f32);
                    n2 = fma(A[a], A[a], n2);
                }
                const double rn = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
                f = make_float4((float)(A[0] * rn), (float)(A[1] * rn), (float)(A[2] * rn),
                                (float)(pld64(Q.b, r0 + r, Q.in_f32) * rn));
            }
            face[r] = f;
        }
        // edges: a facet's line (2-D) or a pair of facets' line (3-D)
        const int ncand = M == 2 ? nr : nr * nr;
        int count = 0;
        for (int c0 = 0; c0 < ncand; c0 += 32) {
            const int c = c0 + lane;
            bool ok = false;
            double z0[3] = {0.0, 0.0, 0.0}, d[3] = {0.0, 0.0, 0.0}, tlo = 0.0, thi = 0.0;
            int ra = -1, rb = -1, rlo = -1, rhi = -1;  // the edge's own facets, the rows at its ends
            if (c < ncand) {
                if (M == 2) {
                    const double a0 = pld64(Q.A, (long long)(r0 + c) * 2, Q.in_f32);
                    const double a1 = pld64(Q.A, (long long)(r0 + c) * 2 + 1, Q.in_f32);
                    const double n2 = a0 * a0 + a1 * a1;
                    if (n2 > 0.0) {
                        const double rn = 1.0 / sqrt(n2), bb = pld64(Q.b, r0 + c, Q.in_f32);
                        d[0] = -a1 * rn;
                        d[1] = a0 * rn;
                        z0[0] = a0 * bb / n2;   // the line's point nearest the origin
                        z0[1] = a1 * bb / n2;
                        ra = c;
                        ok = true;
                    }
                } else {
                    const int r1 = c / nr, r2 = c - r1 * nr;
                    if (r1 < r2) {
                        double a[3], bq[3], b1, b2;
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            a[k] = pld64(Q.A, (long long)(r0 + r1) * 3 + k, Q.in_f32);
                            bq[k] = pld64(Q.A, (long long)(r0 + r2) * 3 + k, Q.in_f32);
                        }
                        b1 = pld64(Q.b, r0 + r1, Q.in_f32);
                        b2 = pld64(Q.b, r0 + r2, Q.in_f32);
                        double x[3] = {a[1] * bq[2] - a[2] * bq[1], a[2] * bq[0] - a[0] * bq[2], a[0] * bq[1] - a[1] * bq[0]};
                        const double xx = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
                        const double aa = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
                        const double bbq = bq[0] * bq[0] + bq[1] * bq[1] + bq[2] * bq[2];
                        if (xx > 1e-20 * aa * bbq) {
                            // z0 = alpha a + beta bq with a . z0 = b1, bq . z0 = b2
                            const double ab = a[0] * bq[0] + a[1] * bq[1] + a[2] * bq[2];
                            const double det = aa * bbq - ab * ab;
                            const double al = (b1 * bbq - b2 * ab) / det, be = (b2 * aa - b1 * ab) / det;
                            const double rx = 1.0 / sqrt(xx);
#pragma unroll
                            for (int k = 0; k < 3; ++k) {
                                z0[k] = al * a[k] + be * bq[k];
                                d[k] = x[k] * rx;
                            }
                            ra = r1;
                            rb = r2;
                            ok = true;
                        }
                    }
                }
                if (ok) {
                    clip_line<M>(Q, r0, nr, z0, d, tlo, thi, rlo, rhi);
                    ok = tlo <= thi;
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, ok);
            const int slot = count + __popc(bal & ((1u << lane) - 1u));
            if (ok && slot < Q.max_edges) {
                float4* ed = edge + EDGE_F4 * slot;
                ed[0] = make_float4((float)z0[0], (float)z0[1], (float)z0[2], __double2float_rd(tlo));
                ed[1] = make_float4((float)d[0], (float)d[1], (float)d[2], __double2float_ru(thi));
                double na[3], nb[3], ca = 0.0, cb = 0.0;
                if (M == 2) {
                    // the normals of the rows at the two ends (zero at an infinite end), own normal and offset
                    double nl[3] = {0.0, 0.0, 0.0}, nh[3] = {0.0, 0.0, 0.0}, cl = 0.0, ch = 0.0;
                    if (rlo >= 0) unit_row<M>(Q, r0, rlo, nl, cl);
                    if (rhi >= 0) unit_row<M>(Q, r0, rhi, nh, ch);
                    unit_row<M>(Q, r0, ra, na, ca);
                    ed[2] = make_float4((float)nl[0], (float)nl[1], (float)nh[0], (float)nh[1]);
                    ed[3] = make_float4((float)na[0], (float)na[1], (float)ca, 0.f);
                } else {
                    unit_row<M>(Q, r0, ra, na, ca);
                    unit_row<M>(Q, r0, rb, nb, cb);
                    ed[2] = make_float4((float)na[0], (float)na[1], (float)na[2], 0.f);
                    ed[3] = make_float4((float)nb[0], (float)nb[1], (float)nb[2], 0.f);
                }
            }
            count += __popc(bal);
        }
        if (lane == 0) {
            Q.nedge[o] = count < Q.max_edges ? count : Q.max_edges;
            if (count > Q.max_edges) p_status(Q.info, PLAN_ERR_UNSUPPORTED, DET_ROWS);
        }
    }
}

template <int M>
PDEV float pdot(const float4& f, const float* z) {
    float s = f.x * z[0];
    s = fmaf(f.y, z[1], s);
    if (M == 3) s = fmaf(f.z, z[2], s);
    return s;
}

// Nearest-only mode, pass A: per point an upper bound of its nearest
// obstacle's distance -- the distance to one vertex (the first edge's start)
// of every obstacle, min-reduced (non-negative floats order as their bits).
template <int M>
__global__ void __launch_bounds__(256) k_planes_ub(PlanesParams Q) {
    const long long total = (long long)Q.P * Q.n_obst;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < total; base += stride) {
        const long long k = base + threadIdx.x;
        const bool act = k < total;
        long long p = 0;
        unsigned ub = 0x7f7f7f7fu;
        if (act) {
            p = k / Q.n_obst;
            const int o = (int)(k - p * Q.n_obst);
            const float4* ew = reinterpret_cast<const float4*>(Q.edge) + EDGE_F4 * (long long)o * Q.max_edges;
            if (Q.nedge[o] >= 1) {
                const float4 e0 = __ldg(ew), e1 = __ldg(ew + 1);
                if (fabsf(e0.w) < 3.0e38f) {   // an unbounded edge has no start vertex
                    float d2 = 0.f;
#pragma unroll
                    for (int a = 0; a < M; ++a) {
                        const float c = fmaf(e0.w, a == 0 ? e1.x : (a == 1 ? e1.y : e1.z),
                                             a == 0 ? e0.x : (a == 1 ? e0.y : e0.z));
                        const float t = pld32(Q.points, p * M + a, Q.in_f32) - c;
                        d2 = fmaf(t, t, d2);
                    }
                    ub = __float_as_uint(sqrtf(d2));
                }
            }
        }
        // lanes of one point are consecutive obstacles: one atomic per run
        const long long p0 = __shfl_sync(0xffffffffu, p, 0), p31 = __shfl_sync(0xffffffffu, p, 31);
        if (p0 == p31 && __all_sync(0xffffffffu, act)) {
            for (int of = 16; of > 0; of >>= 1) ub = min(ub, __shfl_xor_sync(0xffffffffu, ub, of));
            if (lane == 0) atomicMin(reinterpret_cast<unsigned*>(Q.ub) + p, ub);
        } else if (act && ub != 0x7f7f7f7fu) {
            atomicMin(reinterpret_cast<unsigned*>(Q.ub) + p, ub);
        }
    }
}

// One thread per (point, obstacle), the obstacle index fastest (coalesced
// stores of the point-major outputs); per point the nearest obstacle as a
// 64-bit key (distance bits << 32 | obstacle), min-reduced per warp first.
template <int M>
__global__ void __launch_bounds__(256) k_planes(PlanesParams Q) {
    __shared__ int s_fail;
    if (threadIdx.x == 0) s_fail = p_failed(Q.info);
    __syncthreads();
    if (s_fail) return;
    const long long total = Q.pair_obst ? (long long)Q.P : (long long)Q.P * Q.n_obst;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const float inf = __int_as_float(0x7f800000);
    for (long long base = (long long)blockIdx.x * blockDim.x; base < total; base += stride) {
        const long long k = base + threadIdx.x;
        const bool act = k < total;
        long long p = 0;
        int o = 0;
        unsigned long long key = ~0ull;
        if (act && Q.pair_obst) {  // pair mode (no keys): the given obstacle of point k
            p = k;
            o = Q.pair_obst[k];
            if (o < 0 || o >= Q.n_obst) {
                if (Q.plane)
                    for (int a = 0; a <= M; ++a) Q.plane[k * (M + 1) + a] = 0.f;
                if (Q.dist) Q.dist[k] = inf;
                continue;
            }
        } else if (act) {
            p = k / Q.n_obst;
            o = (int)(k - p * Q.n_obst);
        }
        bool pruned = false;
        if (act && Q.ub) {
            // nearest-only mode: an obstacle whose distance lower bound (the
            // largest signed distance to one of its facet planes) exceeds the
            // point's upper bound (with room for float rounding) cannot be
            // the nearest, nor tie with it
            float v[M], vs = 1.f;
#pragma unroll
            for (int a = 0; a < M; ++a) {
                v[a] = pld32(Q.points, p * M + a, Q.in_f32);
                vs += fabsf(v[a]);
            }
            const int nr = Q.ocount[o];
            const float4* fw = reinterpret_cast<const float4*>(Q.face) + (long long)o * Q.max_orows;
            float lb = -inf;
            for (int r = 0; r < nr; ++r) {
                const float4 f = __ldg(fw + r);
                lb = fmaxf(lb, pdot<M>(f, v) - f.w);
            }
            const float ub = Q.ub[p];
            pruned = lb > fmaf(ub, 1.00001f, 1e-5f * vs);
        }
        if (act && !pruned) {
            float v[M];
#pragma unroll
            for (int a = 0; a < M; ++a) v[a] = pld32(Q.points, p * M + a, Q.in_f32);
            const int nr = Q.ocount[o];
            const float4* rw = reinterpret_cast<const float4*>(Q.orow) + (long long)o * Q.max_orows;
            bool in = true;
            for (int r = 0; r < nr; ++r) {
                const float4 f = __ldg(rw + r);
                in = in && pdot<M>(f, v) - f.w <= 0.f;
            }
            float z[M], d2 = 0.f;
#pragma unroll
            for (int a = 0; a < M; ++a) z[a] = v[a];
            if (!in) {
                d2 = inf;
                if (M == 3) {  // faces whose projection lands inside the obstacle
                    const float4* fw = reinterpret_cast<const float4*>(Q.face) + (long long)o * Q.max_orows;
                    for (int r = 0; r < nr; ++r) {
                        const float4 f = __ldg(fw + r);
                        const float sd = pdot<M>(f, v) - f.w;
                        if (!(sd > 0.f) || sd * sd >= d2) continue;
                        float c[M];
#pragma unroll
                        for (int a = 0; a < M; ++a) c[a] = fmaf(-sd, a == 0 ? f.x : (a == 1 ? f.y : f.z), v[a]);
                        bool ok = true;
                        for (int q = 0; q < nr; ++q) {
                            if (q == r) continue;
                            const float4 g = __ldg(rw + q);
                            const float sv = pdot<M>(g, c) - g.w;
                            const float mag = fabsf(g.x * c[0]) + fabsf(g.y * c[1]) + fabsf(g.z * c[M - 1]) + fabsf(g.w);
                            ok = ok && sv <= 8.f * U32P * mag;
                        }
                        if (ok) {
                            d2 = sd * sd;
#pragma unroll
                            for (int a = 0; a < M; ++a) z[a] = c[a];
                        }
                    }
                }
                // edge segments (and their end points, the vertices).  The
                // candidate is chosen by sign tests, not by comparing nearly
                // equal distances: a segment whose parameter needs no clamping
                // (and, in 2-D, whose facet v lies outside of) holds the
                // projection; in 2-D a vertex does when v - vertex lies in the
                // cone of its two facet normals.  The nearest candidate is the
                // fallback for what rounding leaves undecided.
                const float4* ew = reinterpret_cast<const float4*>(Q.edge) + EDGE_F4 * (long long)o * Q.max_edges;
                const int ne = Q.nedge[o];
                bool found = false;
                float fb_d2 = inf, fb[M];
#pragma unroll
                for (int a = 0; a < M; ++a) fb[a] = v[a];
                for (int e = 0; e < ne && !found && !(M == 3 && d2 < inf); ++e) {
                    const float4 e0 = __ldg(ew + EDGE_F4 * e), e1 = __ldg(ew + EDGE_F4 * e + 1);
                    float w[M];
                    w[0] = v[0] - e0.x;
                    w[1] = v[1] - e0.y;
                    if (M == 3) w[M - 1] = v[M - 1] - e0.z;
                    float t = e1.x * w[0];
                    t = fmaf(e1.y, w[1], t);
                    if (M == 3) t = fmaf(e1.z, w[M - 1], t);
                    const float tc = fminf(fmaxf(t, e0.w), e1.w);
                    float c[M], dd = 0.f;
                    c[0] = fmaf(tc, e1.x, e0.x);
                    c[1] = fmaf(tc, e1.y, e0.y);
                    if (M == 3) c[M - 1] = fmaf(tc, e1.z, e0.z);
#pragma unroll
                    for (int a = 0; a < M; ++a) dd = fmaf(v[a] - c[a], v[a] - c[a], dd);
                    bool hit;
                    if (M == 2) {
                        const float4 e2 = __ldg(ew + EDGE_F4 * e + 2), e3 = __ldg(ew + EDGE_F4 * e + 3);
                        const float sd = fmaf(e3.y, v[1], e3.x * v[0]) - e3.z;  // outside this facet?
                        if (tc == t) {
                            hit = sd > 0.f;
                        } else {
                            // a clamped end: the vertex; v - c in the cone of the two normals
                            const float wx = v[0] - c[0], wy = v[1] - c[1];
                            const float nx = t < e0.w ? e2.x : e2.z, ny = t < e0.w ? e2.y : e2.w;
                            float k1 = e3.x * wy - e3.y * wx, k2 = wx * ny - wy * nx, kk = e3.x * ny - e3.y * nx;
                            if (kk < 0.f) {
                                k1 = -k1;
                                k2 = -k2;
                                kk = -kk;
                            }
                            hit = (nx != 0.f || ny != 0.f) && kk > 0.f && k1 >= 0.f && k2 >= 0.f;
                        }
                    } else {
                        // 3-D: an unclamped point of an edge whose two facet normals span v - c
                        hit = false;
                        if (tc == t) {
                            const float4 e2 = __ldg(ew + EDGE_F4 * e + 2), e3 = __ldg(ew + EDGE_F4 * e + 3);
                            const float wx = v[0] - c[0], wy = v[1] - c[1], wz = v[M - 1] - c[M - 1];
                            // signs of (n_a x w) . d, (w x n_b) . d and (n_a x n_b) . d
                            const float k1 = (e2.y * wz - e2.z * wy) * e1.x + (e2.z * wx - e2.x * wz) * e1.y +
                                             (e2.x * wy - e2.y * wx) * e1.z;
                            const float k2 = (wy * e3.z - wz * e3.y) * e1.x + (wz * e3.x - wx * e3.z) * e1.y +
                                             (wx * e3.y - wy * e3.x) * e1.z;
                            float kk = (e2.y * e3.z - e2.z * e3.y) * e1.x + (e2.z * e3.x - e2.x * e3.z) * e1.y +
                                       (e2.x * e3.y - e2.y * e3.x) * e1.z;
                            float s1 = k1, s2 = k2;
                            if (kk < 0.f) {
                                s1 = -s1;
                                s2 = -s2;
                                kk = -kk;
                            }
                            hit = kk > 0.f && s1 >= 0.f && s2 >= 0.f;
                        }
                    }
                    if (hit) {
                        found = true;
                        d2 = dd;
#pragma unroll
                        for (int a = 0; a < M; ++a) z[a] = c[a];
                    } else if (dd < fb_d2) {
                        fb_d2 = dd;
#pragma unroll
                        for (int a = 0; a < M; ++a) fb[a] = c[a];
                    }
                }
                if (!found && !(d2 < inf && M == 3)) {
                    d2 = fb_d2;
#pragma unroll
                    for (int a = 0; a < M; ++a) z[a] = fb[a];
                } else if (!found && M == 3 && fb_d2 < d2) {
                    d2 = fb_d2;
#pragma unroll
                    for (int a = 0; a < M; ++a) z[a] = fb[a];
                }
            }
            const float d = sqrtf(d2);
            if (Q.closest)
#pragma unroll
                for (int a = 0; a < M; ++a) Q.closest[k * M + a] = d2 < inf ? z[a] : __int_as_float(0x7fc00000);
            if (Q.dist) Q.dist[k] = d;
            if (Q.plane) {
                const float rdn = (d > 0.f && d < inf) ? 1.f / d : 0.f;
                float l = 0.f;
#pragma unroll
                for (int a = 0; a < M; ++a) {
                    const float h = (v[a] - z[a]) * rdn;
                    Q.plane[k * (M + 1) + a] = h;
                    l = fmaf(h, z[a], l);
                }
                Q.plane[k * (M + 1) + M] = l;
            }
            key = ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)o;
        }
        if (Q.keys) {
            // lanes of one point are consecutive obstacles: reduce runs of the same point
            const long long p0 = __shfl_sync(0xffffffffu, p, 0), p31 = __shfl_sync(0xffffffffu, p, 31);
            if (p0 == p31 && __all_sync(0xffffffffu, act)) {
                unsigned long long kk = key;
                for (int of = 16; of > 0; of >>= 1) {
                    const unsigned long long ok = __shfl_xor_sync(0xffffffffu, kk, of);
                    kk = ok < kk ? ok : kk;
                }
                if (lane == 0) atomicMin(Q.keys + p, kk);
            } else if (act && !pruned) {
                atomicMin(Q.keys + p, key);
            }
        }
    }
}

__global__ void k_planes_nearest(PlanesParams Q) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= Q.P || p_failed(Q.info)) return;
    const unsigned long long key = Q.keys[p];
    const bool none = key == ~0ull;
    if (Q.nearest) Q.nearest[p] = none ? -1 : (int32_t)(key & 0xffffffffu);
    if (Q.nearest_dist) Q.nearest_dist[p] = none ? __int_as_float(0x7f800000) : __uint_as_float((unsigned)(key >> 32));
}

}  // namespace

int launch_planes(const PlanesParams& Q, void* stream, int num_sms, int* launches) {
    cudaStream_t st = (cudaStream_t)stream;
    const long long orows = (long long)Q.n_obst * Q.max_orows;
    if (orows > 0) {
        k_planes_prep<<<(int)((orows + 255) / 256), 256, 0, st>>>(Q);
        if (Q.m == 2) k_planes_geom<2><<<(Q.n_obst + 3) / 4, 128, 0, st>>>(Q);
        else k_planes_geom<3><<<(Q.n_obst + 3) / 4, 128, 0, st>>>(Q);
        *launches += 2;
    }
    const long long total = (long long)Q.P * Q.n_obst;
    if (total > 0) {
        long long grid = (total + 255) / 256;
        if (grid > (long long)num_sms * 16) grid = (long long)num_sms * 16;
        if (Q.ub) {
            if (Q.m == 2) k_planes_ub<2><<<(int)grid, 256, 0, st>>>(Q);
            else k_planes_ub<3><<<(int)grid, 256, 0, st>>>(Q);
            ++*launches;
        }
        if (Q.m == 2) k_planes<2><<<(int)grid, 256, 0, st>>>(Q);
        else k_planes<3><<<(int)grid, 256, 0, st>>>(Q);
        ++*launches;
    }
    if (Q.P > 0 && (Q.nearest || Q.nearest_dist)) {
        k_planes_nearest<<<(int)((Q.P + 255) / 256), 256, 0, st>>>(Q);
        ++*launches;
    }
    if (Q.P > 0 && Q.nearest_plane && Q.nearest) {
        // the plane of each point's nearest obstacle: the same per-pair work
        // for the pairs (p, nearest[p]) only
        PlanesParams Q2 = Q;
        Q2.pair_obst = Q.nearest;
        Q2.closest = nullptr;
        Q2.dist = nullptr;
        Q2.plane = Q.nearest_plane;
        Q2.keys = nullptr;
        Q2.ub = nullptr;
        Q2.nearest = nullptr;
        Q2.nearest_dist = nullptr;
        long long grid = (Q.P + 255) / 256;
        if (grid > (long long)num_sms * 16) grid = (long long)num_sms * 16;
        if (Q.m == 2) k_planes<2><<<(int)grid, 256, 0, st>>>(Q2);
        else k_planes<3><<<(int)grid, 256, 0, st>>>(Q2);
        ++*launches;
    }
    return (int)cudaGetLastError();
}

}  // namespace plan
