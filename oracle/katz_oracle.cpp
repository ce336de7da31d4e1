// CPU ORACLE for certified Katz ranking (van der Grinten, Bergamini,
// Green, Bader, Meyerhenke: "Scalable Katz Ranking Computation in Large
// Static and Dynamic Graphs", ESA 2018).
//
// TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the benchmark's
// CPU-baseline leg may load this library.  The CUDA library never links,
// includes or calls anything here, and this file includes nothing of it.
//
// Plain, slow, obviously correct: every step follows the paper's text in its
// own notation (omega_i = walk counts, c_r = Katz partial sum, l_r / u_r =
// per-node bounds, M = active set).  Floating point is IEEE FP64 (the paper
// states no precision; its comparison against CG at residual 1e-15 implies
// FP64).  Exact walk counts use unsigned __int128.  Build with
// -ffp-contract=off so that no multiply-add is fused on any host.
//
// Row loops of the walk recurrence may run under OpenMP; each row is summed
// sequentially in CSR order, so results do not depend on the thread count.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

enum { OK = 0, EINVAL_ = 1, EALPHA_ = 2, ENOTCONV_ = 3, EOVERFLOW_ = 4 };

// Stopping criteria of Sec. 3.1.  The ranking criterion is the top-k
// criterion with k = n (the paper says so), so it reuses converged().
enum { CRIT_TOPK = 0, CRIT_RANKING = 1, CRIT_SCORE = 2, CRIT_PAIR = 3 };

typedef unsigned __int128 u128;

// Theorem 1: gamma = deg_max / (1 - alpha deg_max), valid for alpha < 1/deg_max.
double theorem1_gamma(double alpha, double D) { return D / (1.0 - alpha * D); }

struct Bounds {
    std::vector<double> c, l, u;  // c_r (Eq. 1 partial sum), l_r, u_r
};

// l_r and u_r from c_r and omega_r (Alg. 1; undirected improvement of Sec. 3.1).
void bounds_from(const std::vector<double>& c, const std::vector<double>& omega_r, double alpha_r1,
                 double gamma, bool undirected, std::vector<double>& l, std::vector<double>& u) {
    const size_t n = c.size();
    l.resize(n);
    u.resize(n);
    for (size_t v = 0; v < n; ++v) {
        double tail = alpha_r1 * omega_r[v];  // alpha^{r+1} omega_r(v)
        l[v] = undirected ? c[v] + tail : c[v];
        u[v] = c[v] + tail * gamma;
    }
}

// The decreasing order used by partialSort: larger l first, ties by smaller id.
struct ByLowerDesc {
    const double* l;
    bool operator()(int32_t a, int32_t b) const {
        if (l[a] != l[b]) return l[a] > l[b];
        return a < b;
    }
};

// converged() of Algorithm 1 (top-k criterion).  M is the active set; on
// return its first min(|M|, k) entries are the current top-k in order.
bool converged(std::vector<int32_t>& M, int64_t k, const std::vector<double>& l,
               const std::vector<double>& u, double eps) {
    const int64_t kk = std::min<int64_t>(k, (int64_t)M.size());
    if (kk == 0) return true;
    std::partial_sort(M.begin(), M.begin() + kk, M.end(), ByLowerDesc{l.data()});
    const double theta = l[M[kk - 1]];  // l_r(M[k])
    // Deactivate M[i], i > k, if u_r(M[i]) - eps < l_r(M[k]); iterate over the
    // sorted snapshot, keep the rest.
    std::vector<int32_t> keep(M.begin(), M.begin() + kk);
    for (size_t i = (size_t)kk; i < M.size(); ++i) {
        const int32_t v = M[i];
        if (!(u[v] - eps < theta)) keep.push_back(v);
    }
    M.swap(keep);
    if ((int64_t)M.size() > k) return false;
    const int64_t top = std::min<int64_t>((int64_t)M.size(), k);
    for (int64_t i = 1; i < top; ++i)
        if (u[M[i]] - eps >= l[M[i - 1]]) return false;
    return true;
}

// Score criterion (Sec. 3.1): the upper and lower bound of every node differ
// by less than eps.
bool score_done(const std::vector<double>& l, const std::vector<double>& u, double eps) {
    for (size_t v = 0; v < l.size(); ++v)
        if (!(u[v] - l[v] < eps)) return false;
    return true;
}

// Pair criterion (Sec. 3.1): nodes a and b are eps-separated (Eq. 3); w is the
// one with the larger lower bound (ties: smaller id), v the other.
bool pair_done(int32_t a, int32_t b, const std::vector<double>& l, const std::vector<double>& u, double eps) {
    const bool a_first = l[a] > l[b] || (l[a] == l[b] && a < b);
    const int32_t w = a_first ? a : b, v = a_first ? b : a;
    return l[w] > u[v] - eps;
}

// Eq. (5): omega_i(v) = sum over arcs v->x of omega_{i-1}(x), in CSR order.
void walk_step(int64_t n, const int64_t* rowptr, const int32_t* col, const std::vector<double>& prev,
               std::vector<double>& next) {
    next.assign((size_t)n, 0.0);
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t v = 0; v < n; ++v) {
        double s = 0.0;
        for (int64_t j = rowptr[v]; j < rowptr[v + 1]; ++j) s += prev[(size_t)col[j]];
        next[(size_t)v] = s;
    }
}

int64_t max_degree(int64_t n, const int64_t* rowptr) {
    int64_t d = 0;
    for (int64_t v = 0; v < n; ++v) d = std::max<int64_t>(d, rowptr[v + 1] - rowptr[v]);
    return d;
}

// ---------------------------------------------------------------------------
// A mutable graph and the state the dynamic algorithm keeps (Sec. 4).
// ---------------------------------------------------------------------------
struct Session {
    int64_t n = 0;
    bool undirected = true;
    int64_t D = 0;  // degree bound used for gamma (>= deg_max of every state)
    std::vector<std::vector<int32_t>> adj;  // out-neighbours, kept sorted
    // state of the last ranking
    double alpha = 0, gamma = 0, eps = 0;
    int64_t k = 0;
    int r = 0, r_max = 0;
    bool conv = false;
    std::vector<std::vector<double>> omega;  // omega[i][v], i = 0..r (omega[0] = 1)
    std::vector<double> apow;                // apow[i] = alpha^i
    Bounds b;
    std::vector<int32_t> M;
    int crit = CRIT_TOPK;
    int32_t pa = 0, pb = 0;  // the pair of the pair criterion

    // the stopping criterion of this ranking, after iteration r
    bool check() {
        if (crit == CRIT_SCORE) return score_done(b.l, b.u, eps);
        if (crit == CRIT_PAIR) return pair_done(pa, pb, b.l, b.u, eps);
        return converged(M, k, b.l, b.u, eps);
    }

    void csr(std::vector<int64_t>& rp, std::vector<int32_t>& cl) const {
        rp.assign((size_t)n + 1, 0);
        for (int64_t v = 0; v < n; ++v) rp[v + 1] = rp[v] + (int64_t)adj[v].size();
        cl.clear();
        cl.reserve((size_t)rp[n]);
        for (int64_t v = 0; v < n; ++v) cl.insert(cl.end(), adj[v].begin(), adj[v].end());
    }

    // Iteration r -> r+1 of Alg. 1: omega_{r+1}, c_{r+1}, l_{r+1}, u_{r+1}.
    int iterate(const std::vector<int64_t>& rp, const std::vector<int32_t>& cl) {
        std::vector<double> next;
        walk_step(n, rp.data(), cl.data(), omega[(size_t)r], next);
        for (double x : next)
            if (!std::isfinite(x)) return EOVERFLOW_;
        ++r;
        omega.push_back(std::move(next));
        apow.push_back(apow.back() * alpha);
        const std::vector<double>& w = omega[(size_t)r];
        for (int64_t v = 0; v < n; ++v) b.c[v] = b.c[v] + apow[(size_t)r] * w[v];
        bounds_from(b.c, w, apow[(size_t)r] * alpha, gamma, undirected, b.l, b.u);
        return OK;
    }

    // Algorithm 1.  The bounds are defined for r >= 1 (Theorem 1), so the
    // first convergence check follows the first iteration.
    int rank_static(double alpha_, int64_t k_, double eps_, int r_max_) {
        return rank_criterion(alpha_, CRIT_TOPK, k_, 0, 0, eps_, r_max_);
    }

    // Algorithm 1 with any criterion of Sec. 3.1.
    int rank_criterion(double alpha_, int crit_, int64_t k_, int32_t a, int32_t b2, double eps_, int r_max_) {
        if (crit_ < CRIT_TOPK || crit_ > CRIT_PAIR) return EINVAL_;
        if (crit_ == CRIT_RANKING) k_ = n;
        if (crit_ == CRIT_PAIR && (a < 0 || b2 < 0 || a >= n || b2 >= n || a == b2)) return EINVAL_;
        if (crit_ == CRIT_SCORE || crit_ == CRIT_PAIR) k_ = 1;
        if (!(eps_ > 0.0) || k_ < 1 || r_max_ < 1) return EINVAL_;
        crit = crit_;
        pa = a;
        pb = b2;
        const int64_t dmax = [&] {
            int64_t d = 0;
            for (auto& a : adj) d = std::max<int64_t>(d, (int64_t)a.size());
            return d;
        }();
        if (D < dmax) D = dmax;
        alpha = alpha_ > 0.0 ? alpha_ : 1.0 / (double)(D + 1);
        if (!(alpha * (double)D < 1.0)) return EALPHA_;
        gamma = theorem1_gamma(alpha, (double)D);
        eps = eps_;
        k = std::min<int64_t>(k_, n);
        r_max = r_max_;
        r = 0;
        omega.assign(1, std::vector<double>((size_t)n, 1.0));  // omega_0 = 1
        apow.assign(1, 1.0);
        b.c.assign((size_t)n, 0.0);                            // c_0 = 0
        M.resize((size_t)n);
        std::iota(M.begin(), M.end(), 0);                      // M = V
        std::vector<int64_t> rp;
        std::vector<int32_t> cl;
        csr(rp, cl);
        conv = false;
        do {
            if (r >= r_max) return ENOTCONV_;
            int st = iterate(rp, cl);
            if (st) return st;
        } while (!(conv = check()));
        return OK;
    }

    // The loop body of Algorithm 1 exactly R times, without converged():
    // omega_R, c_R and the bounds l_R, u_R (used to inspect every iteration).
    int run_fixed(double alpha_, int R) {
        if (R < 0) return EINVAL_;
        int st = rank_static(alpha_, 1, 1.0, 1);  // validates alpha, sets gamma, one iteration
        if (st != OK && st != ENOTCONV_) return st;
        r = 0;
        omega.resize(1);
        apow.assign(1, 1.0);
        b.c.assign((size_t)n, 0.0);
        b.l.assign((size_t)n, 0.0);
        b.u.assign((size_t)n, 0.0);
        std::vector<int64_t> rp;
        std::vector<int32_t> cl;
        csr(rp, cl);
        while (r < R) {
            st = iterate(rp, cl);
            if (st) return st;
        }
        conv = false;
        return OK;
    }

    bool has(int32_t a, int32_t x) const {
        return std::binary_search(adj[a].begin(), adj[a].end(), x);
    }

    // Preconditions of Alg. 2: I and E disjoint, D a subset of E; the batch
    // itself names each edge at most once (an unordered pair when undirected,
    // an ordered one when directed, Sec. 2.1) and no self-loops; no row may
    // exceed the degree bound the bounds were built with (the out-degree of
    // the source when directed).
    int validate(int64_t m, const int32_t* src, const int32_t* dst, const uint8_t* ins) const {
        std::vector<std::pair<int32_t, int32_t>> seen;
        std::vector<int64_t> dd((size_t)n, 0);
        for (int64_t e = 0; e < m; ++e) {
            int32_t a = src[e], x = dst[e];
            if (a < 0 || x < 0 || a >= n || x >= n || a == x) return EINVAL_;
            seen.push_back(undirected ? std::make_pair(std::min(a, x), std::max(a, x)) : std::make_pair(a, x));
            bool present = has(a, x);
            if (ins[e] ? present : !present) return EINVAL_;
            int delta = ins[e] ? 1 : -1;
            dd[a] += delta;
            if (undirected) dd[x] += delta;
        }
        std::sort(seen.begin(), seen.end());
        if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) return EINVAL_;
        for (int64_t v = 0; v < n; ++v)
            if ((int64_t)adj[v].size() + dd[v] > D) return EALPHA_;
        return OK;
    }

    void mutate(int64_t m, const int32_t* src, const int32_t* dst, const uint8_t* ins) {
        auto arc = [&](int32_t a, int32_t x, bool add) {
            auto& row = adj[a];
            auto it = std::lower_bound(row.begin(), row.end(), x);
            if (add) row.insert(it, x); else row.erase(it);
        };
        for (int64_t e = 0; e < m; ++e) {
            arc(src[e], dst[e], ins[e] != 0);
            if (undirected) arc(dst[e], src[e], ins[e] != 0);
        }
    }

    // Sec. 4: after the batch, omega'_1..omega'_r equal the static values on
    // the modified graph (the paper's correctness statement), so the oracle
    // recomputes them directly; the literal Alg. 2 lives in
    // oracle_alg2_update_u128 and is checked against this recomputation.
    // Then bounds, reactivation with threshold min_{x in M} l_r(x) - eps,
    // and further static iterations until converged().
    int apply_update(int64_t m, const int32_t* src, const int32_t* dst, const uint8_t* ins) {
        if (r < 1) return EINVAL_;
        int st = validate(m, src, dst, ins);
        if (st) return st;
        mutate(m, src, dst, ins);
        std::vector<int64_t> rp;
        std::vector<int32_t> cl;
        csr(rp, cl);
        const int r_keep = r;
        omega.resize(1);
        apow.assign(1, 1.0);
        b.c.assign((size_t)n, 0.0);
        r = 0;
        while (r < r_keep) {
            st = iterate(rp, cl);
            if (st) return st;
        }
        double lmin = INFINITY;
        for (int32_t x : M) lmin = std::min(lmin, b.l[x]);
        std::vector<char> in((size_t)n, 0);
        for (int32_t x : M) in[x] = 1;
        for (int64_t w = 0; w < n; ++w)
            if (!in[w] && b.u[w] >= lmin - eps) M.push_back((int32_t)w);  // reactivation
        conv = false;
        while (!(conv = check())) {
            if (r >= r_max) return ENOTCONV_;
            st = iterate(rp, cl);
            if (st) return st;
        }
        return OK;
    }
};

bool fits(u128 a, u128 b, u128* out) {
    u128 s = a + b;
    if (s < a) return false;
    *out = s;
    return true;
}

}  // namespace

extern "C" {

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

// Exact walk counts omega_1..omega_r of Eq. (5) from omega_0 = 1, as
// unsigned 128-bit integers: out[(i-1)*n*2 + 2*v] = low 64 bits,
// out[... + 1] = high 64 bits.  Returns EOVERFLOW_ if a count exceeds 2^128-1.
int oracle_walks_u128(int64_t n, const int64_t* rowptr, const int32_t* col, int r, uint64_t* out) {
    std::vector<u128> prev((size_t)n, 1), next((size_t)n);
    for (int i = 1; i <= r; ++i) {
        for (int64_t v = 0; v < n; ++v) {
            u128 s = 0;
            for (int64_t j = rowptr[v]; j < rowptr[v + 1]; ++j)
                if (!fits(s, prev[(size_t)col[j]], &s)) return EOVERFLOW_;
            next[(size_t)v] = s;
        }
        for (int64_t v = 0; v < n; ++v) {
            out[((size_t)(i - 1) * n + v) * 2] = (uint64_t)next[v];
            out[((size_t)(i - 1) * n + v) * 2 + 1] = (uint64_t)(next[v] >> 64);
        }
        prev.swap(next);
    }
    return OK;
}

// Algorithm 2 taken literally, in exact arithmetic, for checking that the
// paper's delta update reproduces the static walk counts.  Inputs: the graph
// E before the batch, omega_1..omega_r on E (layout as oracle_walks_u128),
// the batch (directed arcs src->dst, ins = 1 insert / 0 delete).  Output:
// omega'_1..omega'_r.  The garbled parts are read as follows: omega' starts
// as a copy of omega (so omega'_i(x) = omega_i(x) wherever it is not
// written); S is expanded level-synchronously (the loop at level i visits S
// as it stood after level i-1); E means E \ D while the levels run.
// Returns EOVERFLOW_ on overflow or a negative intermediate.
int oracle_alg2_update_u128(int64_t n, const int64_t* rowptr, const int32_t* col, int r,
                            const uint64_t* omega_in, int64_t m, const int32_t* src,
                            const int32_t* dst, const uint8_t* ins, uint64_t* omega_out) {
    // E \ D as reverse adjacency: for each v, the w with w->v in E \ D
    std::vector<std::vector<int32_t>> pred((size_t)n);
    std::vector<std::pair<int32_t, int32_t>> Dset;
    for (int64_t e = 0; e < m; ++e)
        if (!ins[e]) Dset.push_back({src[e], dst[e]});
    std::sort(Dset.begin(), Dset.end());
    for (int64_t w = 0; w < n; ++w)
        for (int64_t j = rowptr[w]; j < rowptr[w + 1]; ++j) {
            std::pair<int32_t, int32_t> a{(int32_t)w, col[j]};
            if (!std::binary_search(Dset.begin(), Dset.end(), a)) pred[(size_t)col[j]].push_back((int32_t)w);
        }
    typedef __int128 s128;
    auto get = [&](const uint64_t* base, int i, int64_t v) -> s128 {  // i >= 1
        size_t o = ((size_t)(i - 1) * n + v) * 2;
        return (s128)(((u128)base[o + 1] << 64) | base[o]);
    };
    std::vector<std::vector<s128>> om((size_t)r + 1, std::vector<s128>((size_t)n, 1));
    std::vector<std::vector<s128>> omp((size_t)r + 1, std::vector<s128>((size_t)n, 1));
    for (int i = 1; i <= r; ++i)
        for (int64_t v = 0; v < n; ++v) om[i][v] = omp[i][v] = get(omega_in, i, v);
    std::vector<char> inS((size_t)n, 0);
    std::vector<int32_t> S;
    for (int64_t e = 0; e < m; ++e)
        if (!inS[src[e]]) { inS[src[e]] = 1; S.push_back(src[e]); }
    for (int i = 1; i <= r; ++i) {
        const std::vector<int32_t> snap = S;  // S after level i-1
        for (int32_t v : snap) {
            const s128 delta = omp[i - 1][v] - om[i - 1][v];
            for (int32_t w : pred[v]) {
                if (!inS[w]) { inS[w] = 1; S.push_back(w); }
                omp[i][w] += delta;
            }
        }
        for (int64_t e = 0; e < m; ++e) {
            if (ins[e]) omp[i][src[e]] += omp[i - 1][dst[e]];
            else omp[i][src[e]] -= om[i - 1][dst[e]];
        }
    }
    for (int i = 1; i <= r; ++i)
        for (int64_t v = 0; v < n; ++v) {
            if (omp[i][v] < 0) return EOVERFLOW_;
            u128 x = (u128)omp[i][v];
            size_t o = ((size_t)(i - 1) * n + v) * 2;
            omega_out[o] = (uint64_t)x;
            omega_out[o + 1] = (uint64_t)(x >> 64);
        }
    return OK;
}

// ---- session API: a graph plus the state Algorithm 2 keeps -----------------

void* oracle_session_create(int64_t n, const int64_t* rowptr, const int32_t* col, int undirected,
                            int64_t deg_bound) {
    if (n < 1) return nullptr;
    Session* s = new Session();
    s->n = n;
    s->undirected = undirected != 0;
    s->adj.resize((size_t)n);
    for (int64_t v = 0; v < n; ++v) {
        s->adj[v].assign(col + rowptr[v], col + rowptr[v + 1]);
        std::sort(s->adj[v].begin(), s->adj[v].end());
    }
    s->D = std::max<int64_t>(deg_bound, max_degree(n, rowptr));
    return s;
}

void oracle_session_free(void* p) { delete (Session*)p; }

int oracle_session_rank(void* p, double alpha, int64_t k, double eps, int r_max) {
    return ((Session*)p)->rank_static(alpha, k, eps, r_max);
}

int oracle_session_rank_criterion(void* p, double alpha, int crit, int64_t k, int32_t a, int32_t b, double eps,
                                   int r_max) {
    return ((Session*)p)->rank_criterion(alpha, crit, k, a, b, eps, r_max);
}

int oracle_session_update(void* p, int64_t m, const int32_t* src, const int32_t* dst,
                          const uint8_t* ins) {
    return ((Session*)p)->apply_update(m, src, dst, ins);
}

// r, |M|, converged, alpha, gamma, degree bound
void oracle_session_info(void* p, int* r, int64_t* active, int* conv, double* alpha, double* gamma,
                         int64_t* D) {
    Session* s = (Session*)p;
    *r = s->r;
    *active = (int64_t)s->M.size();
    *conv = s->conv ? 1 : 0;
    *alpha = s->alpha;
    *gamma = s->gamma;
    *D = s->D;
}

// The first min(k, |M|) entries of M (the ranking once converged).
int64_t oracle_session_ranking(void* p, int32_t* ids, int64_t cap) {
    Session* s = (Session*)p;
    if (s->crit == CRIT_SCORE) return 0;  // certifies scores, not an order
    if (s->crit == CRIT_PAIR) {            // the pair in its certified order
        if (cap < 2) return 0;
        const bool a_first = s->b.l[s->pa] > s->b.l[s->pb] || (s->b.l[s->pa] == s->b.l[s->pb] && s->pa < s->pb);
        ids[0] = a_first ? s->pa : s->pb;
        ids[1] = a_first ? s->pb : s->pa;
        return 2;
    }
    int64_t kk = std::min<int64_t>({s->k, (int64_t)s->M.size(), cap});
    for (int64_t i = 0; i < kk; ++i) ids[i] = s->M[i];
    return kk;
}

void oracle_session_bounds(void* p, double* c, double* l, double* u) {
    Session* s = (Session*)p;
    for (int64_t v = 0; v < s->n; ++v) {
        if (c) c[v] = s->b.c[v];
        if (l) l[v] = s->b.l[v];
        if (u) u[v] = s->b.u[v];
    }
}

// omega_i (unscaled walk counts as FP64), 0 <= i <= r
int oracle_session_omega(void* p, int i, double* out) {
    Session* s = (Session*)p;
    if (i < 0 || i > s->r) return EINVAL_;
    std::memcpy(out, s->omega[(size_t)i].data(), (size_t)s->n * sizeof(double));
    return OK;
}

// alpha^i as the oracle accumulated it
double oracle_session_alpha_pow(void* p, int i) {
    Session* s = (Session*)p;
    return (i >= 0 && i < (int)s->apow.size()) ? s->apow[(size_t)i] : NAN;
}

int64_t oracle_session_active(void* p, int32_t* ids, int64_t cap) {
    Session* s = (Session*)p;
    int64_t m = std::min<int64_t>(cap, (int64_t)s->M.size());
    for (int64_t i = 0; i < m; ++i) ids[i] = s->M[i];
    return (int64_t)s->M.size();
}

// converged() of Algorithm 1 on given bounds l[v] <= c(v) <= u[v] with
// M = V: writes the first min(k, n) entries of the sorted M to top (the
// ranking when certified) and returns 1 if the top-k criterion holds, else 0.
int oracle_converged_bounds(int64_t n, const double* l, const double* u, int64_t k, double eps, int32_t* top) {
    std::vector<double> lv(l, l + n), uv(u, u + n);
    std::vector<int32_t> M((size_t)n);
    std::iota(M.begin(), M.end(), 0);
    std::vector<int32_t> all(M);
    const int64_t kk = std::min<int64_t>(k, n);
    std::partial_sort(all.begin(), all.begin() + kk, all.end(), ByLowerDesc{lv.data()});
    for (int64_t i = 0; i < kk; ++i) top[i] = all[(size_t)i];
    return converged(M, k, lv, uv, eps) ? 1 : 0;
}

int oracle_session_run_fixed(void* p, double alpha, int R) {
    return ((Session*)p)->run_fixed(alpha, R);
}

// Run only the walk recurrence for `iters` iterations plus converged() after
// each one (Algorithm 1 with a fixed iteration budget).  Used to time a bounded
// sample of a large workload.  Returns the number of iterations run.
int oracle_session_iterations(void* p, double alpha, int64_t k, double eps, int iters) {
    Session* s = (Session*)p;
    int st = s->rank_static(alpha, k, eps, iters);
    return st == ENOTCONV_ || st == OK ? s->r : -st;
}

}  // extern "C"
