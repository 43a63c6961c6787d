// Coefficient tables of the reachable Bezier polytope, computed on the host.
//
// Every coefficient is rho * T^e, where rho is an exact rational that does
// not depend on T and e is an integer exponent.  rho comes from the Bezier
// recurrences below, evaluated in exact int128 rational arithmetic; the value
// rho * T^e is then rounded once to the nearest double (ties to even) by an
// exact big-integer division, so each table entry is the correctly rounded
// value of its exact definition.
//
//  * Lemma 1 (minimal degree q = 2g-1): with y_c = T^c x^(c),
//      beta_k     = (q-k)!/q! y_L,k - sum_{s<k} (-1)^{k-s} C(k,s) beta_s
//      beta_{q-k} = (-1)^k [ (q-k)!/q! y_R,k - sum_{s<k} (-1)^s C(k,s) beta_{q-s} ]
//    (the derivative of a Bezier curve at an end point is a scaled forward or
//    backward difference of its first or last control points), then degree
//    elevation to p: P_l = sum_s C(q,s) C(p-q,l-s) / C(p,l) beta_s.
//  * Theorem 1 read per axis: reach rows are the hodograph control points
//      Q^(k)_j = p!/(p-k)! T^-k sum_s (-1)^{k-s} C(k,s) P_{j+s},  k = 1..g.
//  * Eq. (BezDef) / Property 2: the degree-p control points of b^(d) are Q^(d)
//    elevated by d; cost rows are their consecutive differences.
//  * Interior points for p > 2g-1 (Lemma 1 fixes only the first and last g
//    control points of a degree-p curve): either the elevated minimal-degree
//    curve (default) or the points minimising int_0^T |b^(g+1)|^2 dt with the
//    2g end points fixed (PLAN_INTERIOR_MINSNAP).  The energy is a quadratic
//    form in Delta^(g+1) P with the Bernstein Gram matrix of degree p-g-1, so
//    the minimiser is free = S fixed for a rational S independent of T.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "plan_internal.h"

namespace plan {
namespace {

typedef __int128 i128;

i128 gcd128(i128 a, i128 b) {
    if (a < 0) a = -a;
    if (b < 0) b = -b;
    while (b != 0) {
        i128 t = a % b;
        a = b;
        b = t;
    }
    return a;
}

struct Rat {
    i128 n = 0, d = 1;
    Rat() {}
    Rat(i128 num, i128 den = 1) : n(num), d(den) { norm(); }
    void norm() {
        if (d < 0) { n = -n; d = -d; }
        i128 g = gcd128(n, d);
        if (g > 1) { n /= g; d /= g; }
        if (n == 0) d = 1;
    }
};
Rat operator+(const Rat& a, const Rat& b) { return Rat(a.n * b.d + b.n * a.d, a.d * b.d); }
Rat operator-(const Rat& a, const Rat& b) { return Rat(a.n * b.d - b.n * a.d, a.d * b.d); }
Rat operator*(const Rat& a, const Rat& b) { return Rat(a.n * b.n, a.d * b.d); }

int64_t binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}
int64_t fact(int n) {
    int64_t r = 1;
    for (int i = 2; i <= n; ++i) r *= i;
    return r;
}

// ---- minimal unsigned big integer (little-endian 32-bit limbs) ----
struct Big {
    static const int L = 24;
    uint32_t w[L];
    Big() { memset(w, 0, sizeof(w)); }
    explicit Big(unsigned __int128 x) {
        memset(w, 0, sizeof(w));
        for (int i = 0; i < 4; ++i) { w[i] = (uint32_t)x; x >>= 32; }
    }
    int bitlen() const {
        for (int i = L - 1; i >= 0; --i)
            if (w[i]) return i * 32 + (32 - __builtin_clz(w[i]));
        return 0;
    }
    void mul(uint64_t m) {
        unsigned __int128 carry = 0;
        for (int i = 0; i < L; ++i) {
            unsigned __int128 v = (unsigned __int128)w[i] * m + carry;
            w[i] = (uint32_t)v;
            carry = v >> 32;
        }
    }
    Big shl(int s) const {
        Big r;
        int q = s / 32, b = s % 32;
        for (int i = L - 1; i >= 0; --i) {
            uint64_t v = 0;
            int src = i - q;
            if (src >= 0) v = (uint64_t)w[src] << b;
            if (b && src - 1 >= 0) v |= (uint64_t)w[src - 1] >> (32 - b);
            r.w[i] = (uint32_t)v;
        }
        return r;
    }
    static int cmp(const Big& a, const Big& b) {
        for (int i = L - 1; i >= 0; --i)
            if (a.w[i] != b.w[i]) return a.w[i] < b.w[i] ? -1 : 1;
        return 0;
    }
    void sub(const Big& b) {  // requires *this >= b
        int64_t borrow = 0;
        for (int i = 0; i < L; ++i) {
            int64_t v = (int64_t)w[i] - (int64_t)b.w[i] - borrow;
            borrow = v < 0;
            w[i] = (uint32_t)(v + (borrow ? ((int64_t)1 << 32) : 0));
        }
    }
};

// floor(X / Y) for a quotient known to be < 2^56; X becomes the remainder.
uint64_t divmod_small(Big& X, const Big& Y) {
    uint64_t q = 0;
    for (int bit = 56; bit >= 0; --bit) {
        Big Yb = Y.shl(bit);
        if (Big::cmp(Yb, X) <= 0) {
            X.sub(Yb);
            q |= (uint64_t)1 << bit;
        }
    }
    return q;
}

// Correctly rounded double of (num/den) * T^e, T > 0 finite.
double round_rho_pow(const Rat& rho, double T, int e) {
    if (rho.n == 0) return 0.0;
    bool neg = rho.n < 0;
    unsigned __int128 an = (unsigned __int128)(neg ? -rho.n : rho.n);
    unsigned __int128 ad = (unsigned __int128)rho.d;
    int ex;
    double f = std::frexp(T, &ex);
    uint64_t M = (uint64_t)std::ldexp(f, 53);
    long shift = (long)e * (long)(ex - 53);
    Big A(an), B(ad);
    for (int i = 0; i < (e >= 0 ? e : -e); ++i) {
        if (e > 0) A.mul(M);
        else B.mul(M);
    }
    int s = 53 - (A.bitlen() - B.bitlen());
    uint64_t q;
    Big X, Y;
    for (;;) {
        X = s >= 0 ? A.shl(s) : A;
        Y = s >= 0 ? B : B.shl(-s);
        Big Xr = X;
        q = divmod_small(Xr, Y);
        if (q >= ((uint64_t)1 << 53)) { --s; continue; }
        if (q < ((uint64_t)1 << 52)) { ++s; continue; }
        X = Xr;  // remainder
        break;
    }
    Big twoR = X.shl(1);
    int c = Big::cmp(twoR, Y);
    if (c > 0 || (c == 0 && (q & 1))) {
        ++q;
        if (q == ((uint64_t)1 << 53)) { q >>= 1; --s; }
    }
    double v = std::ldexp((double)q, (int)(shift - s));
    return neg ? -v : v;
}

struct RhoTables {
    int g, p, twog, rax;
    // D: [p+1][2g]; H: [rax][2g] (exponent c-k); C: [g][p][2g] (exponent c-d)
    std::vector<Rat> D, H, C;
    std::vector<int> Hk;  // derivative order of each reach row
};

// Solves A X = B in place for square A (exact rationals, partial pivoting on
// non-zero); B has ncol columns.
void solve_rat(std::vector<std::vector<Rat>>& A, std::vector<std::vector<Rat>>& B) {
    const int n = (int)A.size(), ncol = n ? (int)B[0].size() : 0;
    for (int col = 0; col < n; ++col) {
        int piv = col;
        while (piv < n && A[piv][col].n == 0) ++piv;
        std::swap(A[col], A[piv]);
        std::swap(B[col], B[piv]);
        const Rat inv(A[col][col].d, A[col][col].n);
        for (int c = 0; c < n; ++c) A[col][c] = A[col][c] * inv;
        for (int c = 0; c < ncol; ++c) B[col][c] = B[col][c] * inv;
        for (int r = 0; r < n; ++r) {
            if (r == col || A[r][col].n == 0) continue;
            const Rat f = A[r][col];
            for (int c = 0; c < n; ++c) A[r][c] = A[r][c] - f * A[col][c];
            for (int c = 0; c < ncol; ++c) B[r][c] = B[r][c] - f * B[col][c];
        }
    }
}

// Control points of the degree-p curve with interior points of minimal
// (g+1)-th-derivative energy: first g and last g points from the end
// conditions (the end-point difference relations at degree p), the rest from
// the normal equations of the energy.
std::vector<std::vector<Rat>> minsnap_points(int g, int p) {
    const int tg = 2 * g;
    std::vector<std::vector<Rat>> P(p + 1, std::vector<Rat>(tg));
    for (int k = 0; k < g; ++k) {  // start side
        std::vector<Rat> v(tg);
        v[k] = Rat(fact(p - k), fact(p));
        for (int s = 0; s < k; ++s) {
            Rat w(((k - s) % 2 ? -1 : 1) * binom(k, s));
            for (int c = 0; c < tg; ++c) v[c] = v[c] - w * P[s][c];
        }
        P[k] = v;
    }
    for (int k = 0; k < g; ++k) {  // end side
        std::vector<Rat> v(tg);
        v[g + k] = Rat(fact(p - k), fact(p));
        for (int s = 0; s < k; ++s) {
            Rat w((s % 2 ? -1 : 1) * binom(k, s));
            for (int c = 0; c < tg; ++c) v[c] = v[c] - w * P[p - s][c];
        }
        Rat sg(k % 2 ? -1 : 1);
        for (int c = 0; c < tg; ++c) v[c] = sg * v[c];
        P[p - k] = v;
    }
    const int nf = p - 2 * g + 1, qd = p - g - 1;  // free points g..p-g; Delta^(g+1) P has qd+1 rows
    if (nf <= 0) return P;
    // E: Delta^(g+1) as a (qd+1) x (p+1) matrix; Gram of the degree-qd Bernstein basis
    std::vector<std::vector<Rat>> E(qd + 1, std::vector<Rat>(p + 1)), Gm(qd + 1, std::vector<Rat>(qd + 1));
    for (int j = 0; j <= qd; ++j)
        for (int s = 0; s <= g + 1; ++s) E[j][j + s] = Rat(((g + 1 - s) % 2 ? -1 : 1) * binom(g + 1, s));
    for (int j = 0; j <= qd; ++j)
        for (int l = 0; l <= qd; ++l)
            Gm[j][l] = Rat(binom(qd, j) * binom(qd, l), (2 * qd + 1) * binom(2 * qd, j + l));
    // (E_z^T G E_z) z = -E_z^T G (E_f f), f = the fixed points (as maps of xi)
    std::vector<std::vector<Rat>> GE(qd + 1, std::vector<Rat>(p + 1));  // G E
    for (int j = 0; j <= qd; ++j)
        for (int c = 0; c <= p; ++c)
            for (int l = 0; l <= qd; ++l) GE[j][c] = GE[j][c] + Gm[j][l] * E[l][c];
    std::vector<std::vector<Rat>> Az(nf, std::vector<Rat>(nf)), Bz(nf, std::vector<Rat>(tg));
    for (int a = 0; a < nf; ++a) {
        const int za = g + a;
        for (int b = 0; b < nf; ++b) {
            const int zb = g + b;
            for (int j = 0; j <= qd; ++j) Az[a][b] = Az[a][b] + E[j][za] * GE[j][zb];
        }
        for (int c = 0; c <= p; ++c) {
            if (c >= g && c <= p - g) continue;  // fixed points only
            Rat m;  // (E_z^T G E)[a][c]
            for (int j = 0; j <= qd; ++j) m = m + E[j][za] * GE[j][c];
            for (int x = 0; x < tg; ++x) Bz[a][x] = Bz[a][x] - m * P[c][x];
        }
    }
    solve_rat(Az, Bz);
    for (int a = 0; a < nf; ++a) P[g + a] = Bz[a];
    return P;
}

RhoTables rho_tables(int g, int p, int interior) {
    RhoTables R;
    R.g = g;
    R.p = p;
    R.twog = 2 * g;
    const int q = 2 * g - 1, tg = 2 * g;
    std::vector<std::vector<Rat>> beta(q + 1, std::vector<Rat>(tg));
    for (int k = 0; k < g; ++k) {  // start side
        std::vector<Rat> v(tg);
        v[k] = Rat(fact(q - k), fact(q));
        for (int s = 0; s < k; ++s) {
            Rat w(((k - s) % 2 ? -1 : 1) * binom(k, s));
            for (int c = 0; c < tg; ++c) v[c] = v[c] - w * beta[s][c];
        }
        beta[k] = v;
    }
    for (int k = 0; k < g; ++k) {  // end side
        std::vector<Rat> v(tg);
        v[g + k] = Rat(fact(q - k), fact(q));
        for (int s = 0; s < k; ++s) {
            Rat w((s % 2 ? -1 : 1) * binom(k, s));
            for (int c = 0; c < tg; ++c) v[c] = v[c] - w * beta[q - s][c];
        }
        Rat sg(k % 2 ? -1 : 1);
        for (int c = 0; c < tg; ++c) v[c] = sg * v[c];
        beta[q - k] = v;
    }
    // degree elevation q -> p, or the minimum-energy interior points
    std::vector<std::vector<Rat>> P(p + 1, std::vector<Rat>(tg));
    if (interior == 1 && p > q) {
        P = minsnap_points(g, p);
    } else {
        for (int l = 0; l <= p; ++l)
            for (int s = 0; s <= q; ++s) {
                int64_t num = binom(q, s) * binom(p - q, l - s);
                if (!num) continue;
                Rat w(num, binom(p, l));
                for (int c = 0; c < tg; ++c) P[l][c] = P[l][c] + w * beta[s][c];
            }
    }
    R.D.resize((size_t)(p + 1) * tg);
    for (int l = 0; l <= p; ++l)
        for (int c = 0; c < tg; ++c) R.D[(size_t)l * tg + c] = P[l][c];
    // hodographs Q^(k), k = 0..g (Q^(0) = P)
    std::vector<std::vector<std::vector<Rat>>> Q(g + 1);
    Q[0] = P;
    for (int k = 1; k <= g; ++k) {
        Q[k].assign(p - k + 1, std::vector<Rat>(tg));
        Rat scale(fact(p), fact(p - k));
        for (int j = 0; j <= p - k; ++j)
            for (int s = 0; s <= k; ++s) {
                Rat w(((k - s) % 2 ? -1 : 1) * binom(k, s));
                for (int c = 0; c < tg; ++c) Q[k][j][c] = Q[k][j][c] + scale * w * P[j + s][c];
            }
    }
    R.rax = 0;
    for (int k = 1; k <= g; ++k) {
        for (int j = 0; j <= p - k; ++j) {
            for (int c = 0; c < tg; ++c) R.H.push_back(Q[k][j][c]);
            R.Hk.push_back(k);
        }
        R.rax += p - k + 1;
    }
    // cost rows: degree-p control points of b^(d) = Q^(d) elevated by d
    R.C.assign((size_t)g * p * tg, Rat());
    for (int d = 0; d < g; ++d) {
        std::vector<std::vector<Rat>> W(p + 1, std::vector<Rat>(tg));
        for (int l = 0; l <= p; ++l)
            for (int j = 0; j <= p - d; ++j) {
                int64_t num = binom(p - d, j) * binom(d, l - j);
                if (!num) continue;
                Rat w(num, binom(p, l));
                for (int c = 0; c < tg; ++c) W[l][c] = W[l][c] + w * Q[d][j][c];
            }
        for (int l = 0; l < p; ++l)
            for (int c = 0; c < tg; ++c) R.C[((size_t)d * p + l) * tg + c] = W[l + 1][c] - W[l][c];
    }
    return R;
}

}  // namespace

int reach_rows(int g, int p) {
    int r = 0;
    for (int k = 1; k <= g; ++k) r += p - k + 1;
    return r;
}

void exact_tables(int g, int p, int interior, int nT, const double* T, double* D, double* H, double* C) {
    RhoTables R = rho_tables(g, p, interior);
    const int tg = 2 * g;
    for (int t = 0; t < nT; ++t) {
        double Tv = T[t];
        for (int l = 0; l <= p; ++l)
            for (int c = 0; c < tg; ++c)
                D[((size_t)t * (p + 1) + l) * tg + c] = round_rho_pow(R.D[(size_t)l * tg + c], Tv, c % g);
        for (int r = 0; r < R.rax; ++r)
            for (int c = 0; c < tg; ++c)
                H[((size_t)t * R.rax + r) * tg + c] =
                    round_rho_pow(R.H[(size_t)r * tg + c], Tv, (c % g) - R.Hk[r]);
        for (int d = 0; d < g; ++d)
            for (int l = 0; l < p; ++l)
                for (int c = 0; c < tg; ++c)
                    C[(((size_t)t * g + d) * p + l) * tg + c] =
                        round_rho_pow(R.C[((size_t)d * p + l) * tg + c], Tv, (c % g) - d);
    }
}

}  // namespace plan
