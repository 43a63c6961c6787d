/*
 * Plain FP64 CPU oracle for the batched Bezier edge build and the graph search.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header or table generator with the CUDA path: its coefficient tables come
 * from oracle/tables.py (exact rationals), its inputs from the seeded
 * generator.
 *
 * Build: cc -O2 -ffp-contract=off -fno-fast-math -fPIC -shared [-fopenmp].
 * -ffp-contract=off matters: every product and sum below is rounded on its
 * own, in the order written, which is the canonical evaluation order that
 * makes "bit-exact feasibility" well defined:
 *   reach row   S = (sum_c HL_c x_i^(c)) + (sum_c HR_c x_j^(c)),  ok iff |S| <= c_k - eps
 *   free row    P_l = (sum_c DL_lc x_i^(c)) + (sum_c DR_lc x_j^(c))  per axis,
 *               S = sum_a A_ra P_la,                                ok iff S <= b_r - eps
 *   membership  S = sum_a A_ra x^(0)_a,                              in iff S <= b_r - eps
 * (each sum left to right, starting from the first product).
 *
 * Paper passages followed:
 *   Sec. III-A, buildGraph: an edge e_ij exists iff F [v_i; v_j] <= G
 *     (Theorem 1), read here as per-axis bounds on the hodograph control
 *     points of every derivative order k = 1..gamma.
 *   Property 1 (convex hull) with the keep-in polytope: the curve stays in a
 *     shared free polytope if all control points satisfy A P_l <= b.
 *   Sec. III-C, findPath: nearest vertices to the start and goal positions,
 *     edge cost sum_l ||P_{l+1} - P_l||_2 (Property 2), Dijkstra.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int m, gamma, p, nT, N, K, cost_mode; /* cost_mode 0: all state rows, 1: position rows */
    const double* states;                 /* [N][m*gamma], stacked [pos; vel; acc; ...] */
    const int* poly_off;                  /* [K+1] */
    const double* A;                      /* [R][m] */
    const double* b;                      /* [R] */
    double eps;                           /* tightening of every bound */
    const double* bounds;                 /* [gamma]: c_1 .. c_gamma */
    const double* D;                      /* [nT][p+1][2g] */
    const double* H;                      /* [nT][Rax][2g] */
    const double* C;                      /* [nT][g][p][2g] */
} orc_problem;

static int orc_rax(const orc_problem* P) {
    int r = 0;
    for (int k = 1; k <= P->gamma; ++k) r += P->p - k + 1;
    return r;
}

/* Membership of state i in polytope k (canonical order). */
static int orc_in(const orc_problem* P, int i, int k) {
    const int m = P->m, n = P->m * P->gamma;
    const double* x = P->states + (size_t)i * n;
    for (int r = P->poly_off[k]; r < P->poly_off[k + 1]; ++r) {
        double s = 0.0;
        for (int a = 0; a < m; ++a) s = s + P->A[(size_t)r * m + a] * x[a];
        double lim = P->b[r] - P->eps;
        if (!(s <= lim)) return 0;
    }
    return 1;
}

void orc_membership(const orc_problem* P, uint8_t* in /* [N][K] */) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < P->N; ++i)
        for (int k = 0; k < P->K; ++k) in[(size_t)i * P->K + k] = (uint8_t)orc_in(P, i, k);
}

static int orc_shares(const orc_problem* P, const uint8_t* in, int i, int j) {
    for (int k = 0; k < P->K; ++k)
        if (in[(size_t)i * P->K + k] && in[(size_t)j * P->K + k]) return 1;
    return 0;
}

/* Number of candidate partners of each row (j != i sharing a polytope). */
void orc_candidate_counts(const orc_problem* P, const uint8_t* in, int nrows, const int* rows,
                          int64_t* counts) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int t = 0; t < nrows; ++t) {
        int i = rows[t];
        int64_t c = 0;
        for (int j = 0; j < P->N; ++j)
            if (j != i && orc_shares(P, in, i, j)) ++c;
        counts[t] = c;
    }
}

/*
 * Evaluate one candidate pair (i -> j) for every duration.
 *   mask      bit t set iff (pair, T_t) is feasible
 *   costs     [nT] control-polygon length for every T (feasible or not)
 *   rmarg     [nT] min over reach rows of (c_k - eps) - |S|
 *   fmarg     [nT] max over shared polytopes of min over rows and l of (b_r - eps) - S
 * Returns the best duration index (lowest cost among feasible T, ties to the
 * lower index) or -1.
 */
static int orc_eval_pair(const orc_problem* P, const uint8_t* in, int i, int j, uint32_t* mask,
                         double* costs, double* rmarg, double* fmarg, double* best_w) {
    const int m = P->m, g = P->gamma, p = P->p, n = m * g, twog = 2 * g;
    const int rax = orc_rax(P);
    const double* xi = P->states + (size_t)i * n;
    const double* xj = P->states + (size_t)j * n;
    double Pc[64 * 4]; /* control points [p+1][m], p <= 63, m <= 4 */
    uint32_t msk = 0;
    int best = -1;
    double bw = INFINITY;
    for (int t = 0; t < P->nT; ++t) {
        const double* D = P->D + (size_t)t * (p + 1) * twog;
        const double* H = P->H + (size_t)t * rax * twog;
        const double* C = P->C + (size_t)t * g * p * twog;
        /* reach rows, per axis */
        double rmin = INFINITY;
        int reach_ok = 1;
        for (int a = 0; a < m; ++a) {
            int row = 0;
            for (int k = 1; k <= g; ++k) {
                double lim = P->bounds[k - 1] - P->eps;
                for (int jj = 0; jj <= p - k; ++jj, ++row) {
                    const double* h = H + (size_t)row * twog;
                    double sl = 0.0, sr = 0.0;
                    for (int c = 0; c < g; ++c) sl = sl + h[c] * xi[c * m + a];
                    for (int c = 0; c < g; ++c) sr = sr + h[g + c] * xj[c * m + a];
                    double s = sl + sr;
                    double mg = lim - fabs(s);
                    if (mg < rmin) rmin = mg;
                    if (!(fabs(s) <= lim)) reach_ok = 0;
                }
            }
        }
        /* control points (Lemma 1), all l = 0..p */
        for (int l = 0; l <= p; ++l)
            for (int a = 0; a < m; ++a) {
                const double* d = D + (size_t)l * twog;
                double sl = 0.0, sr = 0.0;
                for (int c = 0; c < g; ++c) sl = sl + d[c] * xi[c * m + a];
                for (int c = 0; c < g; ++c) sr = sr + d[g + c] * xj[c * m + a];
                Pc[l * m + a] = sl + sr;
            }
        /* free-space test against every shared polytope (Property 1, keep-in) */
        int free_ok = 0;
        double fbest = -INFINITY;
        for (int k = 0; k < P->K; ++k) {
            if (!(in[(size_t)i * P->K + k] && in[(size_t)j * P->K + k])) continue;
            int ok = 1;
            double fmin = INFINITY;
            for (int r = P->poly_off[k]; r < P->poly_off[k + 1]; ++r) {
                double lim = P->b[r] - P->eps;
                for (int l = 0; l <= p; ++l) {
                    double s = 0.0;
                    for (int a = 0; a < m; ++a) s = s + P->A[(size_t)r * m + a] * Pc[l * m + a];
                    double mg = lim - s;
                    if (mg < fmin) fmin = mg;
                    if (!(s <= lim)) ok = 0;
                }
            }
            if (ok) free_ok = 1;
            if (fmin > fbest) fbest = fmin;
        }
        /* cost: length of the state-space control polygon (Property 2) */
        int drows = (P->cost_mode == 1) ? 1 : g;
        double cost = 0.0;
        for (int l = 0; l < p; ++l) {
            double ss = 0.0;
            for (int dd = 0; dd < drows; ++dd) {
                const double* cr = C + ((size_t)dd * p + l) * twog;
                for (int a = 0; a < m; ++a) {
                    double sl = 0.0, sr = 0.0;
                    for (int c = 0; c < g; ++c) sl = sl + cr[c] * xi[c * m + a];
                    for (int c = 0; c < g; ++c) sr = sr + cr[g + c] * xj[c * m + a];
                    double v = sl + sr;
                    ss = ss + v * v;
                }
            }
            cost = cost + sqrt(ss);
        }
        if (costs) costs[t] = cost;
        if (rmarg) rmarg[t] = rmin;
        if (fmarg) fmarg[t] = fbest;
        if (reach_ok && free_ok) {
            msk |= (1u << t);
            if (cost < bw) { bw = cost; best = t; }
        }
    }
    *mask = msk;
    *best_w = bw;
    return best;
}

/*
 * Candidate pairs of the given rows, in (row order, j ascending).  Output
 * arrays must hold sum(counts) entries (see orc_candidate_counts); costs,
 * rmarg, fmarg hold [pairs][nT] and may be NULL.
 */
void orc_edges_rows(const orc_problem* P, const uint8_t* in, int nrows, const int* rows,
                    const int64_t* offsets /* [nrows] start of each row's output */,
                    int32_t* out_i, int32_t* out_j, uint32_t* out_mask, double* out_w,
                    int32_t* out_t, double* out_costs, double* out_rmarg, double* out_fmarg) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int t = 0; t < nrows; ++t) {
        int i = rows[t];
        int64_t o = offsets[t];
        for (int j = 0; j < P->N; ++j) {
            if (j == i || !orc_shares(P, in, i, j)) continue;
            uint32_t msk;
            double bw;
            int bt = orc_eval_pair(P, in, i, j, &msk, out_costs ? out_costs + o * P->nT : NULL,
                                   out_rmarg ? out_rmarg + o * P->nT : NULL,
                                   out_fmarg ? out_fmarg + o * P->nT : NULL, &bw);
            out_i[o] = i;
            out_j[o] = j;
            out_mask[o] = msk;
            out_w[o] = bw;
            out_t[o] = bt;
            ++o;
        }
    }
}

/* Nearest vertex to a position (Sec. III-C): squared distance summed left to
 * right, ties to the lowest id. */
int orc_nearest(const orc_problem* P, const double* pos) {
    const int m = P->m, n = P->m * P->gamma;
    int best = -1;
    double bd = INFINITY;
    for (int i = 0; i < P->N; ++i) {
        const double* x = P->states + (size_t)i * n;
        double d = 0.0;
        for (int a = 0; a < m; ++a) {
            double t = x[a] - pos[a];
            d = d + t * t;
        }
        if (d < bd) { bd = d; best = i; }
    }
    return best;
}

/* ---- Dijkstra with a binary heap keyed (dist, id), lazy deletion ---- */
typedef struct { double d; int v; } orc_item;

static int orc_less(orc_item a, orc_item b) { return a.d < b.d || (a.d == b.d && a.v < b.v); }

static void orc_push(orc_item* h, int64_t* n, orc_item x) {
    int64_t i = (*n)++;
    h[i] = x;
    while (i > 0) {
        int64_t par = (i - 1) / 2;
        if (!orc_less(h[i], h[par])) break;
        orc_item t = h[i]; h[i] = h[par]; h[par] = t;
        i = par;
    }
}

static orc_item orc_pop(orc_item* h, int64_t* n) {
    orc_item top = h[0];
    h[0] = h[--(*n)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, s = i;
        if (l < *n && orc_less(h[l], h[s])) s = l;
        if (r < *n && orc_less(h[r], h[s])) s = r;
        if (s == i) break;
        orc_item t = h[i]; h[i] = h[s]; h[s] = t;
        i = s;
    }
    return top;
}

/* Single-source shortest paths on a CSR graph with non-negative weights.
 * dist accumulated as dist[u] + w in FP64; relax only on strict improvement.
 * Returns 0, or -1 if the heap could not be allocated. */
int orc_dijkstra(int N, const int64_t* row_off, const int32_t* col, const double* w, int s,
                 double* dist, int32_t* pred) {
    for (int v = 0; v < N; ++v) { dist[v] = INFINITY; pred[v] = -1; }
    if (s < 0 || s >= N) return 0;
    int64_t E = row_off[N];
    orc_item* h = (orc_item*)malloc(sizeof(orc_item) * (size_t)(E + 2));
    uint8_t* done = (uint8_t*)calloc((size_t)N, 1);
    if (!h || !done) { free(h); free(done); return -1; }
    int64_t hn = 0;
    dist[s] = 0.0;
    orc_item st = {0.0, s};
    orc_push(h, &hn, st);
    while (hn > 0) {
        orc_item it = orc_pop(h, &hn);
        int u = it.v;
        if (done[u] || it.d != dist[u]) continue;
        done[u] = 1;
        for (int64_t e = row_off[u]; e < row_off[u + 1]; ++e) {
            int v = col[e];
            double nd = dist[u] + w[e];
            if (nd < dist[v]) {
                dist[v] = nd;
                pred[v] = u;
                orc_item x = {nd, v};
                orc_push(h, &hn, x);
            }
        }
    }
    free(h);
    free(done);
    return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
