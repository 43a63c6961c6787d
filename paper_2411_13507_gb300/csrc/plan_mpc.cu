// MPC refinement QP for sm_103a (Sec. III-D, Eq. (MPC)): one quadratic
// program per problem of a batch, one warp per problem, FP64.
//
// The problem (x_k in R^n derivative-major, n = m g; u_k in R^m the g-th
// derivative of every axis; horizon H, step dt):
//   min sum_{k<H} (x_k - r_k)'Q(x_k - r_k) + (x_{k+1} - x_k)'F(x_{k+1} - x_k)
//       + u_k'R u_k + (x_H - r_H)'V(x_H - r_H)
//   s.t. x_{k+1} = A x_k + B u_k, x_0 fixed, x_H = r_H,
//        |H_r xi_{k,a}| <= c_ord(r) (Theorem 1 rows of duration dt per axis
//        and segment), h_k . P_l(k) >= l_k for the control points of segment
//        k (l >= 1 when k = 0) unless h_k = 0, and A_d P_l(k) <= b_d for
//        l = 1..p (keep-in rows, optional).
// Q, F, V, R diagonal and positive.
//
// GPU formulation.  The dynamics are condensed away: per axis a the chain is
// the same, so x_{k,a}^(c) = phi_{k,a,c} + sum_{j<k} Gam[k][c][j] u_{j,a}
// with Gam[k][c][j] = (A^{k-1-j} B)_c and phi_{k,a} = A^k x0_a.  The
// variables are the inputs, axis-major (index a H + j), so the Hessian is
// block-diagonal over the axes.  The QP is solved by the dual active-set
// method of Goldfarb and Idnani (1983): start at the unconstrained minimum
// with no active constraint, add the terminal equalities, then repeatedly
// add the most violated inequality (ties to the lowest row id), taking a
// partial step that drops an active inequality whenever its multiplier would
// turn negative; the factorisation J = L^-T (G = L L') and the triangular R
// with J' N_active = [R; 0] are updated by a Householder reflection when a
// constraint enters and by Givens rotations when one leaves.  Constraint rows
// are never stored: the scan evaluates every row from the node states, and
// the row chosen to enter is expanded into input space through Gam.
//
// A reach row met twice -- the hodograph control point of a derivative of
// order < g at a node two segments share is that derivative itself -- is
// scanned once (the first such row of every segment k >= 1 is skipped).
//
// The Hessian and its factor J0 = L^-T depend on the model, dt and the
// weights only: a small kernel (one CTA per axis block) computes them when
// those change (the host compares the table with the last call's) and every
// problem starts from a copy of J0.
//
// One warp per problem: lanes own variable indices (two each up to 64) for
// the dense steps and strided row ids for the scan; the warp synchronises
// with __syncwarp only.  The scan screens every row in float and decides in
// double only the rows the float rounding leaves open (the narrow FP64 pipe
// of this part is the bound).  Shared memory: the table (double and float)
// and Gam per CTA; per warp G (then L), J, R, the working vectors and the
// float copies of the states and planes.
#include <cuda_runtime.h>

#include <cstdint>

#include "plan_internal.h"

namespace plan {

#define MDEV __device__ __forceinline__

namespace {

struct MpcLayout {  // offsets into the table of doubles
    int A, Bv, D, Hr, hb, Q, F, V, R, KA, Kb, total;
    MDEV void init(int m, int g, int p, int rax, int nkeep) {
        const int n = m * g;
        A = 0;
        Bv = A + g * g;
        D = Bv + g;
        Hr = D + (p + 1) * 2 * g;
        hb = Hr + rax * 2 * g;
        Q = hb + rax;
        F = Q + n;
        V = F + n;
        R = V + n;
        KA = R + m;
        Kb = KA + nkeep * m;
        total = Kb + nkeep;
    }
};

// Row ids of the scan: reach rows (k, a, r, sign), then safety rows (k, l),
// then keep-in rows (k, l >= 1, r).
struct RowSpace {
    int H, m, g, p, rax, nkeep;
    int n_reach, n_safe, n_keep, total;
    MDEV void init(int H_, int m_, int g_, int p_, int rax_, int nkeep_) {
        H = H_;
        m = m_;
        g = g_;
        p = p_;
        rax = rax_;
        nkeep = nkeep_;
        n_reach = H * m * rax * 2;
        n_safe = H * (p + 1);
        n_keep = H * p * nkeep;
        total = n_reach + n_safe + n_keep;
    }
};

// First reach row of derivative order o (1-based): orders have p - o + 1 rows.
MDEV int first_row_of_order(int o, int p) { return (o - 1) * p - ((o - 1) * (o - 2)) / 2; }

// Coefficients of one row on the states of its segment: value = sum over
// axes a and derivatives c of alpha0[a][c] x_{k,a}^(c) + alpha1[a][c]
// x_{k+1,a}^(c); the row reads value <= bound.  Returns false for a row
// that is not scanned (duplicate or absent).
struct RowCoef {
    int k;
    double a0[3][4], a1[3][4];
    double bound;
};

MDEV bool row_coef(const RowSpace& S, const double* tab, const MpcLayout& L, const double* planes_w, int id,
                   RowCoef& rc) {
    const int g = S.g, m = S.m, p = S.p;
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 4; ++c) {
            rc.a0[a][c] = 0.0;
            rc.a1[a][c] = 0.0;
        }
    if (id < S.n_reach) {
        const int sg = id & 1;
        int t = id >> 1;
        const int r = t % S.rax;
        t /= S.rax;
        const int a = t % m;
        const int k = t / m;
        // order of row r and the duplicate rule
        int o = 1;
        while (o < g && r >= first_row_of_order(o + 1, p)) ++o;
        if (k >= 1 && o < g && r == first_row_of_order(o, p)) return false;
        const double sgn = sg ? -1.0 : 1.0;
        for (int c = 0; c < g; ++c) {
            rc.a0[a][c] = sgn * tab[L.Hr + r * 2 * g + c];
            rc.a1[a][c] = sgn * tab[L.Hr + r * 2 * g + g + c];
        }
        rc.k = k;
        rc.bound = tab[L.hb + r];
        return true;
    }
    id -= S.n_reach;
    if (id < S.n_safe) {
        const int k = id / (p + 1), l = id % (p + 1);
        if (k == 0 && l == 0) return false;
        const double* pl = planes_w + k * (m + 1);
        bool any = false;
        for (int a = 0; a < m; ++a) any |= pl[a] != 0.0;
        if (!any) return false;
        for (int a = 0; a < m; ++a)
            for (int c = 0; c < g; ++c) {
                rc.a0[a][c] = -pl[a] * tab[L.D + l * 2 * g + c];
                rc.a1[a][c] = -pl[a] * tab[L.D + l * 2 * g + g + c];
            }
        rc.k = k;
        rc.bound = -pl[m];
        return true;
    }
    id -= S.n_safe;
    const int r = id % S.nkeep;
    const int t = id / S.nkeep;
    const int l = 1 + t % p, k = t / p;
    for (int a = 0; a < m; ++a)
        for (int c = 0; c < g; ++c) {
            const double ka = tab[L.KA + r * m + a];
            rc.a0[a][c] = ka * tab[L.D + l * 2 * g + c];
            rc.a1[a][c] = ka * tab[L.D + l * 2 * g + g + c];
        }
    rc.k = k;
    rc.bound = tab[L.Kb + r];
    return true;
}

// slack = bound - value and its magnitude (sum of |terms| + |bound|) of row
// id, evaluated by row type in arithmetic T (float for the screen, double
// for the decision); false for a row that is not scanned.
template <typename T>
MDEV bool row_eval(const RowSpace& S, const T* tab, const MpcLayout& L, const T* pw, const T* xs, int id, T& slack,
                   T& mag) {
    const int g = S.g, m = S.m, p = S.p, n = m * g;
    T v = 0, s = 0, bound;
    if (id < S.n_reach) {
        const int sg = id & 1;
        int t = id >> 1;
        const int r = t % S.rax;
        t /= S.rax;
        const int a = t % m, k = t / m;
        int o = 1;
        while (o < g && r >= first_row_of_order(o + 1, p)) ++o;
        if (k >= 1 && o < g && r == first_row_of_order(o, p)) return false;
        const T* hr = tab + L.Hr + r * 2 * g;
        for (int c = 0; c < g; ++c) {
            const T t0 = hr[c] * xs[k * n + c * m + a], t1 = hr[g + c] * xs[(k + 1) * n + c * m + a];
            v += t0 + t1;
            s += fabs(t0) + fabs(t1);
        }
        if (sg) v = -v;
        bound = tab[L.hb + r];
    } else if (id < S.n_reach + S.n_safe) {
        id -= S.n_reach;
        const int k = id / (p + 1), l = id % (p + 1);
        if (k == 0 && l == 0) return false;
        const T* pl = pw + k * (m + 1);
        bool any = false;
        for (int a = 0; a < m; ++a) any |= pl[a] != T(0);
        if (!any) return false;
        const T* d = tab + L.D + l * 2 * g;
        for (int a = 0; a < m; ++a) {
            T P = 0, Pm = 0;
            for (int c = 0; c < g; ++c) {
                const T t0 = d[c] * xs[k * n + c * m + a], t1 = d[g + c] * xs[(k + 1) * n + c * m + a];
                P += t0 + t1;
                Pm += fabs(t0) + fabs(t1);
            }
            v -= pl[a] * P;
            s += fabs(pl[a]) * Pm;
        }
        bound = -pl[m];
    } else {
        id -= S.n_reach + S.n_safe;
        const int r = id % S.nkeep, t = id / S.nkeep;
        const int l = 1 + t % p, k = t / p;
        const T* d = tab + L.D + l * 2 * g;
        for (int a = 0; a < m; ++a) {
            T P = 0, Pm = 0;
            for (int c = 0; c < g; ++c) {
                const T t0 = d[c] * xs[k * n + c * m + a], t1 = d[g + c] * xs[(k + 1) * n + c * m + a];
                P += t0 + t1;
                Pm += fabs(t0) + fabs(t1);
            }
            const T ka = tab[L.KA + r * m + a];
            v += ka * P;
            s += fabs(ka) * Pm;
        }
        bound = tab[L.Kb + r];
    }
    slack = bound - v;
    mag = s + fabs(bound);
    return true;
}

// The row in input space in the form nvec . u >= bnd (GI convention):
// nvec = -(alpha Gam), bnd = alpha . phi - bound.  Lanes fill their indices.
MDEV void row_in_u(const RowCoef& rc, const double* Gam, const double* phi, int H, int m, int g, int nv, int lane,
                   double* nvec, double& bnd) {
    for (int i = lane; i < nv; i += 32) {
        const int a = i / H, j = i % H;
        double s = 0.0;
        for (int c = 0; c < g; ++c) {
            s += rc.a0[a][c] * Gam[(rc.k * g + c) * H + j];
            s += rc.a1[a][c] * Gam[((rc.k + 1) * g + c) * H + j];
        }
        nvec[i] = -s;
    }
    double b = 0.0;
    for (int a = 0; a < m; ++a)
        for (int c = 0; c < g; ++c)
            b += rc.a0[a][c] * phi[(rc.k * m + a) * g + c] + rc.a1[a][c] * phi[((rc.k + 1) * m + a) * g + c];
    bnd = b - rc.bound;
}

MDEV double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace

// Gam[k][c][j] = (A^{k-1-j} B)_c for j < k, by the whole block: column j = 0
// holds A^{k-1} B (one thread, by repeated products), every other column
// copies it from row k - j (reads column 0 only, writes the others).
MDEV void mpc_gam(const double* tab, const MpcLayout& L, double* Gam, int H, int g) {
    for (int i = threadIdx.x; i < (H + 1) * g * H; i += blockDim.x) Gam[i] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v[4], t[4];
        for (int c = 0; c < g; ++c) v[c] = tab[L.Bv + c];
        for (int s = 0; s < H; ++s) {
            for (int c = 0; c < g; ++c) Gam[((s + 1) * g + c) * H] = v[c];
            for (int c = 0; c < g; ++c) {
                double acc = 0.0;
                for (int cc = 0; cc < g; ++cc) acc += tab[L.A + c * g + cc] * v[cc];
                t[c] = acc;
            }
            for (int c = 0; c < g; ++c) v[c] = t[c];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < (H + 1) * g * H; i += blockDim.x) {
        const int j = i % H, kc = i / H, c = kc % g, k = kc / g;
        if (j >= 1 && j < k) Gam[i] = Gam[((k - j) * g + c) * H];
    }
    __syncthreads();
}

// One axis block of the Hessian G of the condensed objective (G is
// block-diagonal over the axes and depends on the model, dt and the weights
// only, so one factorisation serves every problem of a batch): G_a [H][H] by
// the whole block, then by warp 0 its Cholesky factor G_a = L L' (in place)
// and J_a = L^-T [H][H] (rd [H] scratch).
MDEV void mpc_factor_axis(const double* tab, const MpcLayout& L, const double* Gam, int H, int m, int g, int a,
                          double* G, double* J, double* rd) {
    for (int i = threadIdx.x; i < H * H; i += blockDim.x) {
        const int j = i / H, j2 = i % H;
        double s = 0.0;
        for (int k = 0; k <= H; ++k)
            for (int c = 0; c < g; ++c) {
                const double gk = Gam[(k * g + c) * H + j], gk2 = Gam[(k * g + c) * H + j2];
                if (k < H) {
                    const double q = tab[L.Q + c * m + a], f = tab[L.F + c * m + a];
                    const double d1 = Gam[((k + 1) * g + c) * H + j] - gk, d2 = Gam[((k + 1) * g + c) * H + j2] - gk2;
                    s += q * gk * gk2 + f * d1 * d2;
                } else {
                    s += tab[L.V + c * m + a] * gk * gk2;
                }
            }
        if (j == j2) s += tab[L.R + a];
        G[j * H + j2] = 2.0 * s;
    }
    __syncthreads();
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    // Cholesky in place (lower triangle), column by column
    for (int j = 0; j < H; ++j) {
        double dsum = 0.0;
        for (int k = lane; k < j; k += 32) dsum += G[j * H + k] * G[j * H + k];
        dsum = warp_sum(dsum);
        const double djj = sqrt(G[j * H + j] - dsum);
        __syncwarp();
        for (int i = j + 1 + lane; i < H; i += 32) {
            double s = G[i * H + j];
            for (int k = 0; k < j; ++k) s -= G[i * H + k] * G[j * H + k];
            G[i * H + j] = s / djj;
        }
        __syncwarp();
        if (lane == 0) G[j * H + j] = djj;
        __syncwarp();
    }
    // J = L^-T: column c of L^-1 by forward substitution, written as row c of J
    for (int i = lane; i < H * H; i += 32) J[i] = 0.0;
    for (int i = lane; i < H; i += 32) rd[i] = 1.0 / G[i * H + i];
    __syncwarp();
    for (int c = lane; c < H; c += 32) {
        for (int i = c; i < H; ++i) {
            double s = i == c ? 1.0 : 0.0;
            for (int k = c; k < i; ++k) s -= G[i * H + k] * J[c * H + k];
            J[c * H + i] = s * rd[i];
        }
    }
    __syncwarp();
}

// J0 = L^-T of the batch's Hessian: CTA a factors the block of axis a and
// writes rows a H .. a H + H - 1 of J0 (zero outside the block).
__global__ void __launch_bounds__(128) k_mpc_setup(MpcParams P) {
    extern __shared__ __align__(16) double s_set[];
    const int m = P.m, g = P.g, H = P.H, nv = P.nv, a = blockIdx.x;
    MpcLayout L;
    L.init(m, g, P.p, P.rax, P.nkeep);
    double* tab = s_set;
    double* Gam = tab + L.total;
    double* G = Gam + (H + 1) * g * H;
    double* J = G + H * H;
    double* rd = J + H * H;
    for (int i = threadIdx.x; i < L.total; i += blockDim.x) tab[i] = P.tab[i];
    __syncthreads();
    mpc_gam(tab, L, Gam, H, g);
    mpc_factor_axis(tab, L, Gam, H, m, g, a, G, J, rd);
    if (threadIdx.x < 32)
        for (int i = threadIdx.x; i < H * nv; i += 32) {
            const int r = i / nv, c = i % nv;
            P.J0[(a * H + r) * nv + c] = (c >= a * H && c < a * H + H) ? J[r * H + (c - a * H)] : 0.0;
        }
}

__global__ void __launch_bounds__(256) k_mpc(MpcParams P) {
    extern __shared__ __align__(16) double s_mpc[];
    const int m = P.m, g = P.g, p = P.p, H = P.H, nv = P.nv, n = m * g;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, W = blockDim.x >> 5;
    MpcLayout L;
    L.init(m, g, p, P.rax, P.nkeep);
    double* tab = s_mpc;
    double* Gam = tab + L.total;                      // [(H+1) g][H]
    double* wbase = Gam + (H + 1) * g * H;
    const int per_warp = 2 * nv * nv + 8 * nv + (H + 1) * m * g + (H + 1) * n + H * (m + 1);
    double* J = wbase + w * per_warp;                 // [nv][nv], from J0
    double* Rm = J + nv * nv;                         // [nv][nv] upper triangle of R (column q: Rm[i * nv + q])
    double* uv = Rm + nv * nv;
    double* gv = uv + nv;
    double* dv = gv + nv;
    double* zv = dv + nv;
    double* rv = zv + nv;
    double* npv = rv + nv;
    double* mult = npv + nv;
    double* rdR = mult + nv;                          // [nv] reciprocals of R's diagonal
    double* phi = rdR + nv;                           // [(H+1) m][g]
    double* xs = phi + (H + 1) * m * g;               // [(H+1)][n]
    double* pw = xs + (H + 1) * n;                    // [H][m+1] planes of this problem
    int* act = reinterpret_cast<int*>(wbase + W * per_warp) + w * nv;
    float* tab32 = reinterpret_cast<float*>(reinterpret_cast<int*>(wbase + W * per_warp) + W * nv);  // [L.total]
    const int per_warp32 = (H + 1) * n + H * (m + 1);
    float* xs32 = tab32 + L.total + w * per_warp32;   // [(H+1)][n]
    float* pw32 = xs32 + (H + 1) * n;                 // [H][m+1]

    // CTA: the table (double and float) and Gam
    for (int i = threadIdx.x; i < L.total; i += blockDim.x) {
        tab[i] = P.tab[i];
        tab32[i] = (float)P.tab[i];
    }
    __syncthreads();
    mpc_gam(tab, L, Gam, H, g);

    const long long b = (long long)blockIdx.x * W + w;
    if (b >= P.B) return;  // whole warps leave together; no block barrier follows
    const double* x0 = P.x0 + b * n;
    const double* ref = P.ref + b * (H + 1) * n;
    const float* planes = P.planes + b * H * (m + 1);
    for (int i = lane; i < H * (m + 1); i += 32) {
        pw32[i] = planes[i];
        pw[i] = (double)planes[i];
    }
    // free response phi_{k,a} = A^k x0_a
    for (int i = lane; i < m * g; i += 32) {
        const int a = i / g, c = i % g;
        phi[(0 * m + a) * g + c] = x0[c * m + a];
    }
    __syncwarp();
    for (int k = 0; k < H; ++k) {
        double val = 0.0;
        int a = 0, c = 0;
        if (lane < m * g) {
            a = lane / g;
            c = lane % g;
            for (int cc = 0; cc < g; ++cc) val += tab[L.A + c * g + cc] * phi[(k * m + a) * g + cc];
        }
        __syncwarp();
        if (lane < m * g) phi[((k + 1) * m + a) * g + c] = val;
        __syncwarp();
    }
    // J = L^-T of the batch's Hessian (from the setup kernel), gradient at u = 0
    for (int i = lane; i < nv * nv; i += 32) J[i] = P.J0[i];
    for (int row = lane; row < nv; row += 32) {
        const int a = row / H, j = row % H;
        double s = 0.0;
        for (int k = 0; k <= H; ++k)
            for (int c = 0; c < g; ++c) {
                const double gk = Gam[(k * g + c) * H + j];
                const double ph = phi[(k * m + a) * g + c];
                const double rf = ref[k * n + c * m + a];
                if (k < H) {
                    const double d1 = Gam[((k + 1) * g + c) * H + j] - gk;
                    const double dph = phi[((k + 1) * m + a) * g + c] - ph;
                    s += tab[L.Q + c * m + a] * gk * (ph - rf) + tab[L.F + c * m + a] * d1 * dph;
                } else {
                    s += tab[L.V + c * m + a] * gk * (ph - rf);
                }
            }
        gv[row] = 2.0 * s;
    }
    __syncwarp();
    // unconstrained minimum u = -J J' g
    for (int i = lane; i < nv; i += 32) {
        double s = 0.0;
        for (int k = 0; k < nv; ++k) s += J[k * nv + i] * gv[k];
        dv[i] = s;
    }
    __syncwarp();
    for (int i = lane; i < nv; i += 32) {
        double s = 0.0;
        for (int k = i; k < nv; ++k) s += J[i * nv + k] * dv[k];
        uv[i] = -s;
    }
    __syncwarp();

    RowSpace S;
    S.init(H, m, g, p, P.rax, P.nkeep);
    const int neq = n;                    // terminal equalities (a, c)
    int q = 0, status = MPC_OK, iters = 0;
    int next_eq = 0;
    const int max_iter = P.max_iter;
    for (;;) {
        // node states from u (and their float copy for the screen)
        for (int i = lane; i < (H + 1) * n; i += 32) {
            const int k = i / n, cm = i % n, c = cm / m, a = cm % m;
            double s = phi[(k * m + a) * g + c];
            for (int j = 0; j < k; ++j) s += Gam[(k * g + c) * H + j] * uv[a * H + j];
            xs[i] = s;
            xs32[i] = (float)s;
        }
        __syncwarp();
        // the constraint to add: the next terminal equality, else the most violated row
        int pid = -1;
        double sp = 0.0, bnd = 0.0;
        RowCoef rc;
        bool is_eq = false;
        if (next_eq < neq) {
            const int a = next_eq / g, c = next_eq % g;
            is_eq = true;
            pid = next_eq;
            for (int i = lane; i < nv; i += 32) {
                const int aa = i / H, j = i % H;
                npv[i] = aa == a ? Gam[(H * g + c) * H + j] : 0.0;
            }
            bnd = ref[H * n + c * m + a] - phi[(H * m + a) * g + c];
            ++next_eq;
        } else {
            double best = 0.0;
            int bid = 0x7fffffff;
            // screen in float: a row whose float slack exceeds the float
            // rounding band (at most (4g + 2m + 8) 2^-24 of the magnitude,
            // taken as 64 2^-24) holds in exact arithmetic and is skipped;
            // every other row is decided in double
            for (int id = lane; id < S.total; id += 32) {
                float s32, m32;
                if (!row_eval<float>(S, tab32, L, pw32, xs32, id, s32, m32)) continue;
                if (s32 > 3.814697265625e-06f * m32) continue;   // 64 * 2^-24
                double sl, mag;
                row_eval<double>(S, tab, L, pw, xs, id, sl, mag);
                if (sl < -1e-11 * mag && (sl < best || (sl == best && id < bid))) {
                    best = sl;
                    bid = id;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bid, o);
                if (ob < best || (ob == best && oi < bid)) {
                    best = ob;
                    bid = oi;
                }
            }
            if (bid == 0x7fffffff) break;  // every row holds: optimal
            pid = neq + bid;
            row_coef(S, tab, L, pw, bid, rc);
            row_in_u(rc, Gam, phi, H, m, g, nv, lane, npv, bnd);
        }
        __syncwarp();
        // s_p = n_p . u - b_p; an equality is oriented so that s_p <= 0
        double spv = 0.0;
        for (int i = lane; i < nv; i += 32) spv += npv[i] * uv[i];
        sp = warp_sum(spv) - bnd;
        if (is_eq && sp > 0.0) {
            for (int i = lane; i < nv; i += 32) npv[i] = -npv[i];
            bnd = -bnd;
            sp = -sp;
        }
        __syncwarp();
        double mult_p = 0.0;
        bool added = false;
        while (!added) {
            if (++iters > max_iter) {
                status = MPC_MAXITER;
                break;
            }
            // d = J' n_p
            for (int i = lane; i < nv; i += 32) {
                double s = 0.0;
                for (int k = 0; k < nv; ++k) s += J[k * nv + i] * npv[k];
                dv[i] = s;
            }
            __syncwarp();
            // z = J2 d2 (columns q..nv-1), r = R^-1 d1
            double zz = 0.0, dd = 0.0;
            for (int i = lane; i < nv; i += 32) {
                double s = 0.0;
                for (int k = q; k < nv; ++k) s += J[i * nv + k] * dv[k];
                zv[i] = s;
                dd += dv[i] * dv[i];
                if (i >= q) zz += dv[i] * dv[i];
            }
            zz = warp_sum(zz);
            dd = warp_sum(dd);
            // r = R^-1 d[0..q) by a column sweep over the lanes
            for (int i = lane; i < q; i += 32) rv[i] = dv[i];
            __syncwarp();
            for (int i = q - 1; i >= 0; --i) {
                const double ri = rv[i] * rdR[i];
                __syncwarp();
                for (int k = lane; k < i; k += 32) rv[k] -= Rm[k * nv + i] * ri;
                if (lane == 0) rv[i] = ri;
                __syncwarp();
            }
            // step lengths: t1 (an active inequality's multiplier reaches 0;
            // lowest position on ties), t2 (full)
            double rmax = 0.0;
            for (int j = lane; j < q; j += 32) rmax = fmax(rmax, fabs(rv[j]));
            for (int o = 16; o > 0; o >>= 1) rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
            double t1 = __longlong_as_double(0x7ff0000000000000ll);
            int l = 0x7fffffff;
            for (int j = lane; j < q; j += 32) {
                if (act[j] >= neq && rv[j] > 1e-13 * rmax) {
                    const double ratio = mult[j] / rv[j];
                    if (ratio < t1) {
                        t1 = ratio;
                        l = j;
                    }
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ot = __shfl_xor_sync(0xffffffffu, t1, o);
                const int ol = __shfl_xor_sync(0xffffffffu, l, o);
                if (ot < t1 || (ot == t1 && ol < l)) {
                    t1 = ot;
                    l = ol;
                }
            }
            if (l == 0x7fffffff) l = -1;
            const bool zero_z = zz <= 1e-22 * dd;
            const double t2 = zero_z ? __longlong_as_double(0x7ff0000000000000ll) : -sp / zz;
            const double t = fmin(t1, t2);
            if (!(t < __longlong_as_double(0x7ff0000000000000ll))) {
                status = MPC_INFEASIBLE;
                break;
            }
            if (!zero_z)
                for (int i = lane; i < nv; i += 32) uv[i] += t * zv[i];
            if (lane == 0)
                for (int j = 0; j < q; ++j) mult[j] -= t * rv[j];
            mult_p += t;
            __syncwarp();
            if (!zero_z && t == t2) {
                // add p: one Householder reflection of the columns q..nv-1 of J
                // maps d[q..] onto alpha e_q (alpha = -sign(d_q) |d[q..]|, no
                // cancellation); then R's new column is d[0..q]
                if (q < nv - 1) {
                    double ss = 0.0;
                    for (int i = q + lane; i < nv; i += 32) ss += dv[i] * dv[i];
                    ss = warp_sum(ss);
                    const double dq = dv[q];
                    const double alpha = dq >= 0.0 ? -sqrt(ss) : sqrt(ss);
                    const double v0 = dq - alpha;
                    const double beta = 1.0 / (ss - alpha * dq);   // 2 / (v'v)
                    for (int r = lane; r < nv; r += 32) {
                        double wv = J[r * nv + q] * v0;
                        for (int k = q + 1; k < nv; ++k) wv += J[r * nv + k] * dv[k];
                        wv *= beta;
                        J[r * nv + q] -= wv * v0;
                        for (int k = q + 1; k < nv; ++k) J[r * nv + k] -= wv * dv[k];
                    }
                    __syncwarp();
                    if (lane == 0) dv[q] = alpha;
                    __syncwarp();
                }
                if (lane == 0) {
                    for (int i = 0; i <= q; ++i) Rm[i * nv + q] = dv[i];
                    rdR[q] = 1.0 / dv[q];
                    act[q] = pid;
                    mult[q] = mult_p;
                }
                ++q;
                added = true;
                __syncwarp();
            } else {
                // drop the inequality at position l: remove its column, restore
                // the triangle by rotations of rows (R) and columns (J)
                if (lane == 0) {
                    for (int j = l; j < q - 1; ++j) {
                        for (int i = 0; i <= j + 1; ++i) Rm[i * nv + j] = Rm[i * nv + j + 1];
                        act[j] = act[j + 1];
                        mult[j] = mult[j + 1];
                    }
                }
                __syncwarp();
                for (int j = l; j < q - 1; ++j) {
                    const double a0 = Rm[j * nv + j], a1 = Rm[(j + 1) * nv + j];
                    const double h = hypot(a0, a1);
                    const double c = h > 0.0 ? a0 / h : 1.0, s = h > 0.0 ? a1 / h : 0.0;
                    __syncwarp();
                    for (int k = j + lane; k < q - 1; k += 32) {
                        const double r0 = Rm[j * nv + k], r1 = Rm[(j + 1) * nv + k];
                        Rm[j * nv + k] = c * r0 + s * r1;
                        Rm[(j + 1) * nv + k] = -s * r0 + c * r1;
                    }
                    for (int k = lane; k < nv; k += 32) {
                        const double j0 = J[k * nv + j], j1 = J[k * nv + j + 1];
                        J[k * nv + j] = c * j0 + s * j1;
                        J[k * nv + j + 1] = -s * j0 + c * j1;
                    }
                    __syncwarp();
                }
                --q;
                for (int j = l + lane; j < q; j += 32) rdR[j] = 1.0 / Rm[j * nv + j];
                if (lane == 0) Rm[q * nv + q] = 0.0;
                // s_p at the new point
                double s2 = 0.0;
                for (int i = lane; i < nv; i += 32) s2 += npv[i] * uv[i];
                sp = warp_sum(s2) - bnd;
                __syncwarp();
            }
        }
        if (status != MPC_OK) break;
    }
    // outputs: states, inputs (node-major), objective
    for (int i = lane; i < (H + 1) * n; i += 32) {
        const int k = i / n, cm = i % n, c = cm / m, a = cm % m;
        double s = phi[(k * m + a) * g + c];
        for (int j = 0; j < k; ++j) s += Gam[(k * g + c) * H + j] * uv[a * H + j];
        xs[i] = s;
        P.x[b * (H + 1) * n + i] = s;
        if (P.nodes && k < H && cm < m) P.nodes[(b * H + k) * m + cm] = s;   // positions of x_0 .. x_{H-1}
    }
    for (int i = lane; i < nv; i += 32) {
        const int a = i / H, j = i % H;
        P.u[b * nv + j * m + a] = uv[i];
    }
    __syncwarp();
    double o = 0.0;
    for (int i = lane; i < (H + 1) * n; i += 32) {
        const int k = i / n, cm = i % n;
        const double e = xs[i] - ref[i];
        if (k < H) {
            const double d = xs[i + n] - xs[i];
            o += tab[L.Q + cm] * e * e + tab[L.F + cm] * d * d;
        } else {
            o += tab[L.V + cm] * e * e;
        }
    }
    for (int i = lane; i < nv; i += 32) o += tab[L.R + i / H] * uv[i] * uv[i];
    o = warp_sum(o);
    if (lane == 0) {
        P.obj[b] = o;
        P.status[b] = status;
        if (P.iters) P.iters[b] = iters;
    }
}

int mpc_table_size(int m, int g, int p, int rax, int nkeep) {
    const int n = m * g;
    return g * g + g + (p + 1) * 2 * g + rax * 2 * g + rax + 3 * n + m + nkeep * m + nkeep;
}

size_t mpc_smem(int m, int g, int p, int rax, int nkeep, int H, int W) {
    const int n = m * g, nv = m * H;
    const size_t per_warp = (size_t)2 * nv * nv + 8 * nv + (H + 1) * m * g + (H + 1) * n + H * (m + 1);
    const size_t per_warp32 = (size_t)(H + 1) * n + H * (m + 1);
    const size_t ts = (size_t)mpc_table_size(m, g, p, rax, nkeep);
    return sizeof(double) * (ts + (size_t)(H + 1) * g * H + W * per_warp) + sizeof(int) * (size_t)W * nv +
           sizeof(float) * (ts + W * per_warp32);
}

size_t mpc_setup_smem(int m, int g, int p, int rax, int nkeep, int H) {
    return sizeof(double) * ((size_t)mpc_table_size(m, g, p, rax, nkeep) + (size_t)(H + 1) * g * H +
                             (size_t)2 * H * H + H);
}

int launch_mpc(const MpcParams& P, void* stream, int* launches) {
    if (P.B <= 0) return 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (!P.j0_ready) {
        const size_t s0 = mpc_setup_smem(P.m, P.g, P.p, P.rax, P.nkeep, P.H);
        cudaFuncSetAttribute(k_mpc_setup, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s0);
        k_mpc_setup<<<P.m, 128, s0, st>>>(P);
        ++*launches;
    }
    const size_t smem = mpc_smem(P.m, P.g, P.p, P.rax, P.nkeep, P.H, P.warps);
    cudaFuncSetAttribute(k_mpc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int grid = (P.B + P.warps - 1) / P.warps;
    k_mpc<<<grid, 32 * P.warps, smem, st>>>(P);
    ++*launches;
    return (int)cudaGetLastError();
}

}  // namespace plan
