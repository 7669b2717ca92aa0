// SF-GRASS oracle: a plain, slow, single-threaded FP64 CPU restatement of the method.
//
// TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the CPU-baseline leg of the
// benchmark may load this library. The product path (the CUDA library) shares no code with it.
//
// Every function follows the paper (Zhang, Zhao, Feng, "SF-GRASS: Solver-Free Graph Spectral
// Sparsification", ICCAD 2020) step by step, in its order and notation, with no blocking, fusion
// or reordering. Where the paper is silent the reading used is named in the comment.
//
// Parity status: every function here is pinned by the CPU tests (closed-form spectra, invariants,
// brute force on tiny graphs, the effective-resistance identity of Eq. formula_Reff), except the
// end-to-end sparsifier edge set, which the paper gives no worked example for ("parity unpinned"
// against the paper; pinned only through kappa and the unit pins of its steps).
//
// Build: g++ -O2 -std=c++17 -shared -fPIC -ffp-contract=off sfg_oracle.cpp -o liboracle_sfg.so
// (-ffp-contract=off: no fused multiply-add, so every FP64 expression rounds as written.)

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <utility>
#include <vector>

namespace {

// ---------------------------------------------------------------------------------------------
// Counter-based Gaussian generator (reading of Sec. 3.2 "K initial random vectors"; the paper
// does not fix a distribution or generator). SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the
// generator adds the golden gamma to its state and returns the 64-bit finaliser of the new state;
// splitmix64(x) below is that finaliser applied to x + gamma, i.e. the output of a generator in
// state x. The stream starts in state s0 = splitmix64(seed), so its output number p + 1 is
// o_p = splitmix64(s0 + p * gamma) and any output is reachable directly from its index.
// Output o_p feeds entries 2p and 2p+1 of the row-major N x K block (entry j = i*K + k) through
// both branches of Box-Muller: u1 = ((o_p >> 32) + 1) 2^-32 in (0,1], u2 = ((o_p >> 8) mod 2^24)
// 2^-24 in [0,1), r = sqrt(-2 ln u1), x_2p = r cos(2 pi u2), x_2p+1 = r sin(2 pi u2).
// ---------------------------------------------------------------------------------------------
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + kGamma;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double gaussian_draw(uint64_t seed, uint64_t j) {
    const uint64_t o = splitmix64(splitmix64(seed) + (j >> 1) * kGamma);
    const double u1 = (double)((o >> 32) + 1) * 0x1.0p-32;
    const double u2 = (double)((o >> 8) & 0xffffffull) * 0x1.0p-24;
    const double two_pi = 6.283185307179586;
    const double r = std::sqrt(-2.0 * std::log(u1));
    return (j & 1) ? r * std::sin(two_pi * u2) : r * std::cos(two_pi * u2);
}

// Seed of the level-l embedding in the multilevel method (reading: each level re-embeds its own
// graph, Algorithm 1 "Embed G_{l-1}"; the same level seed is reused for G_l and P_l).
uint64_t level_seed(uint64_t seed, int level) {
    return level == 0 ? seed : splitmix64(seed ^ (uint64_t)level);
}

// Canonical, de-duplicated, weighted undirected edge list (Sec. 2.1): u < v, sorted by (u, v),
// parallel edges merged by adding weights (Laplacians add), self-loops dropped (D sums t != p).
struct Graph {
    int32_t n = 0;
    std::vector<int32_t> u, v;
    std::vector<float> w;  // canonical weights: the FP64 sum of the merged inputs, rounded once
    int64_t m() const { return (int64_t)u.size(); }
};

// Laplacian L = D - A in CSR form (Eq. formula_adjacency and the definition of D below it).
struct Laplacian {
    int32_t n = 0;
    std::vector<int64_t> row_ptr;
    std::vector<int32_t> col;
    std::vector<double> a;    // A(p,q) = w(p,q)
    std::vector<int32_t> eid; // canonical edge id of each stored entry
    std::vector<double> deg;  // D(p,p) = sum_{t != p} w(p,t)
};

int canonicalize(int32_t n, int64_t m, const int32_t* u, const int32_t* v, const float* w,
                 Graph& g) {
    if (n < 0 || m < 0) return 1;
    for (int64_t e = 0; e < m; ++e) {
        if (u[e] < 0 || u[e] >= n || v[e] < 0 || v[e] >= n) return 1;
        if (!std::isfinite(w[e]) || !(w[e] > 0.0f)) return 1;
    }
    struct Item { int32_t a, b; int64_t idx; };
    std::vector<Item> items;
    items.reserve((size_t)m);
    for (int64_t e = 0; e < m; ++e) {
        if (u[e] == v[e]) continue;  // self-loop: no contribution to L
        items.push_back({std::min(u[e], v[e]), std::max(u[e], v[e]), e});
    }
    std::stable_sort(items.begin(), items.end(), [](const Item& x, const Item& y) {
        return x.a != y.a ? x.a < y.a : x.b < y.b;
    });
    g.n = n;
    g.u.clear(); g.v.clear(); g.w.clear();
    size_t i = 0;
    while (i < items.size()) {
        size_t j = i;
        double sum = 0.0;  // duplicates summed in input order, in FP64
        while (j < items.size() && items[j].a == items[i].a && items[j].b == items[i].b) {
            sum += (double)w[items[j].idx];
            ++j;
        }
        g.u.push_back(items[i].a);
        g.v.push_back(items[i].b);
        g.w.push_back((float)sum);
        i = j;
    }
    return 0;
}

Laplacian build_laplacian(const Graph& g) {
    Laplacian L;
    L.n = g.n;
    std::vector<std::vector<std::pair<int32_t, int32_t>>> rows((size_t)g.n);  // (col, edge id)
    for (int64_t e = 0; e < g.m(); ++e) {
        rows[(size_t)g.u[e]].push_back({g.v[e], (int32_t)e});
        rows[(size_t)g.v[e]].push_back({g.u[e], (int32_t)e});
    }
    L.row_ptr.assign((size_t)g.n + 1, 0);
    L.deg.assign((size_t)g.n, 0.0);
    for (int32_t p = 0; p < g.n; ++p) {
        auto& r = rows[(size_t)p];
        std::sort(r.begin(), r.end());
        for (auto& ce : r) {
            L.col.push_back(ce.first);
            L.a.push_back((double)g.w[(size_t)ce.second]);
            L.eid.push_back(ce.second);
            L.deg[(size_t)p] += (double)g.w[(size_t)ce.second];
        }
        L.row_ptr[(size_t)p + 1] = (int64_t)L.col.size();
    }
    return L;
}

Graph subgraph(const Graph& g, const uint8_t* mask) {
    Graph s;
    s.n = g.n;
    for (int64_t e = 0; e < g.m(); ++e)
        if (mask[e]) { s.u.push_back(g.u[e]); s.v.push_back(g.v[e]); s.w.push_back(g.w[e]); }
    return s;
}

// y = L x for an N x K row-major block: (L x)_p = D(p,p) x_p - sum_q A(p,q) x_q.
void laplacian_apply(const Laplacian& L, int K, const std::vector<double>& x,
                     std::vector<double>& y) {
    y.assign(x.size(), 0.0);
    for (int32_t p = 0; p < L.n; ++p)
        for (int k = 0; k < K; ++k) {
            double s = L.deg[(size_t)p] * x[(size_t)p * K + k];
            for (int64_t j = L.row_ptr[(size_t)p]; j < L.row_ptr[(size_t)p + 1]; ++j)
                s -= L.a[(size_t)j] * x[(size_t)L.col[(size_t)j] * K + k];
            y[(size_t)p * K + k] = s;
        }
}

// Sec. 3.2: K random vectors, made orthogonal to the all-one vector by removing each column's mean.
void init_vectors(int32_t n, int K, uint64_t seed, std::vector<double>& x) {
    x.assign((size_t)n * K, 0.0);
    for (int32_t i = 0; i < n; ++i)
        for (int k = 0; k < K; ++k)
            x[(size_t)i * K + k] = gaussian_draw(seed, (uint64_t)i * (uint64_t)K + (uint64_t)k);
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int32_t i = 0; i < n; ++i) s += x[(size_t)i * K + k];
        const double mean = n > 0 ? s / n : 0.0;
        for (int32_t i = 0; i < n; ++i) x[(size_t)i * K + k] -= mean;
    }
}

// Sec. 3.2 relaxation sweeps on L x = 0, in the weighted-Jacobi form x <- x - omega D^-1 L x
// (reading: the paper names Gauss-Seidel; the data-parallel weighted-Jacobi smoother with a fixed
// omega is used). A node with D(p,p) = 0 has (L x)_p = 0 and is left unchanged.
void jacobi(const Laplacian& L, int K, int steps, double omega, std::vector<double>& x) {
    std::vector<double> y;
    for (int t = 0; t < steps; ++t) {
        laplacian_apply(L, K, x, y);
        for (int32_t p = 0; p < L.n; ++p) {
            const double d = L.deg[(size_t)p];
            if (d == 0.0) continue;
            for (int k = 0; k < K; ++k) x[(size_t)p * K + k] -= omega * y[(size_t)p * K + k] / d;
        }
    }
}

// Reading: after smoothing, remove each column's mean again (Jacobi keeps the D-weighted mean,
// not the plain mean) and scale each column to unit RMS (||x||_2 = sqrt(N)).
void project(int32_t n, int K, std::vector<double>& x) {
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int32_t i = 0; i < n; ++i) s += x[(size_t)i * K + k];
        const double mean = n > 0 ? s / n : 0.0;
        for (int32_t i = 0; i < n; ++i) x[(size_t)i * K + k] -= mean;
        double q = 0.0;
        for (int32_t i = 0; i < n; ++i) q += x[(size_t)i * K + k] * x[(size_t)i * K + k];
        const double rms = n > 0 ? std::sqrt(q / n) : 0.0;
        if (rms > 0.0)
            for (int32_t i = 0; i < n; ++i) x[(size_t)i * K + k] /= rms;
    }
}

void smooth(const Laplacian& L, int K, int steps, double omega, uint64_t seed,
            std::vector<double>& x) {
    init_vectors(L.n, K, seed, x);
    jacobi(L, K, steps, omega, x);
    project(L.n, K, x);
}

// Union-find with path halving; used by Kruskal and by component labelling.
struct DSU {
    std::vector<int32_t> parent;
    explicit DSU(int32_t n) : parent((size_t)n) { std::iota(parent.begin(), parent.end(), 0); }
    int32_t find(int32_t a) {
        while (parent[(size_t)a] != a) {
            parent[(size_t)a] = parent[(size_t)parent[(size_t)a]];
            a = parent[(size_t)a];
        }
        return a;
    }
    bool unite(int32_t a, int32_t b) {
        a = find(a); b = find(b);
        if (a == b) return false;
        parent[(size_t)std::max(a, b)] = std::min(a, b);
        return true;
    }
};

// Sec. 3.4: the spanning-tree backbone is approximated by a maximum-weight spanning tree. Kruskal
// over the strict order (weight descending, edge id ascending), so the forest is unique. Only
// edges with allow[e] != 0 take part (allow == nullptr: all edges).
void kruskal_max(const Graph& g, const uint8_t* allow, uint8_t* mask) {
    std::vector<int32_t> order;
    for (int64_t e = 0; e < g.m(); ++e)
        if (!allow || allow[e]) order.push_back((int32_t)e);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return g.w[(size_t)a] > g.w[(size_t)b]; });
    DSU dsu(g.n);
    for (int64_t e = 0; e < g.m(); ++e) mask[e] = 0;
    for (int32_t e : order)
        if (dsu.unite(g.u[(size_t)e], g.v[(size_t)e])) mask[e] = 1;
}

int32_t count_components(const Graph& g) {
    DSU dsu(g.n);
    int32_t c = g.n;
    for (int64_t e = 0; e < g.m(); ++e)
        if (dsu.unite(g.u[(size_t)e], g.v[(size_t)e])) --c;
    return c;
}

// Eqs. formula_eig_perturb1_conclusion / formula_eig_perturb1_conclusion2 with U replaced by the
// smoothed block X (end of Sec. 3.5): s(p,q) = w(p,q) ||X^T e_pq||^2 = w(p,q) sum_k (X_pk - X_qk)^2.
// Modes (reading): 0 = s_P / (s_G + eta), 1 = s_G (Algorithm 1 embeds G), 2 = s_P (Sec. 3.5
// perturbs L_P).
double edge_distance(const std::vector<double>& x, int K, int32_t p, int32_t q) {
    double s = 0.0;
    for (int k = 0; k < K; ++k) {
        const double d = x[(size_t)p * K + k] - x[(size_t)q * K + k];
        s += d * d;
    }
    return s;
}

void score_edges(const Graph& g, const std::vector<double>& xg, const std::vector<double>& xp,
                 int K, const int32_t* ids, int64_t ne, int mode, double eta, double* out) {
    for (int64_t i = 0; i < ne; ++i) {
        const int32_t e = ids[i];
        const double w = (double)g.w[(size_t)e];
        const double sg = w * edge_distance(xg, K, g.u[(size_t)e], g.v[(size_t)e]);
        const double sp = w * edge_distance(xp, K, g.u[(size_t)e], g.v[(size_t)e]);
        out[i] = mode == 1 ? sg : (mode == 2 ? sp : sp / (sg + eta));
    }
}

// Algorithm 1, selection step (keep the candidates of largest distortion): the k largest by (score descending,
// id ascending); returned ids ascending.
void topk(const double* scores, const int32_t* ids, int64_t ne, int64_t k, int32_t* out) {
    std::vector<int64_t> order((size_t)ne);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        if (scores[a] != scores[b]) return scores[a] > scores[b];
        return ids[a] < ids[b];
    });
    std::vector<int32_t> sel;
    for (int64_t i = 0; i < k; ++i) sel.push_back(ids[order[(size_t)i]]);
    std::sort(sel.begin(), sel.end());
    for (int64_t i = 0; i < k; ++i) out[i] = sel[(size_t)i];
}

// Sec. 3.2 (the algebraic-distance affinity of Livne & Brandt quoted there):
// a_pq = (X_p . X_q)^2 / (||X_p||^2 ||X_q||^2); the aggregation distance is delta_pq = 1 - a_pq.
// A zero row makes a_pq undefined; delta is then 1 (no affinity).
void affinity(const Graph& g, const std::vector<double>& x, int K, double* delta) {
    std::vector<double> nn((size_t)g.n, 0.0);
    for (int32_t p = 0; p < g.n; ++p) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += x[(size_t)p * K + k] * x[(size_t)p * K + k];
        nn[(size_t)p] = s;
    }
    for (int64_t e = 0; e < g.m(); ++e) {
        const int32_t p = g.u[(size_t)e], q = g.v[(size_t)e];
        double dot = 0.0;
        for (int k = 0; k < K; ++k) dot += x[(size_t)p * K + k] * x[(size_t)q * K + k];
        const double den = nn[(size_t)p] * nn[(size_t)q];
        delta[e] = den > 0.0 ? 1.0 - (dot * dot) / den : 1.0;
    }
}

// Sec. 3.2 aggregation (reading: the paper asks for connected sets of nodes that are close in the
// embedding). Each node hooks to the neighbour with the smallest delta (ties: smaller neighbour
// id); aggregation sets are the connected components of the hook graph; aggregate ids are
// numbered by increasing smallest member. A node without neighbours is a singleton.
int32_t aggregate(const Graph& g, const Laplacian& L, const double* delta, int32_t* agg) {
    DSU dsu(g.n);
    for (int32_t p = 0; p < g.n; ++p) {
        int32_t best = -1;
        double bd = 0.0;
        for (int64_t j = L.row_ptr[(size_t)p]; j < L.row_ptr[(size_t)p + 1]; ++j) {
            const double d = delta[L.eid[(size_t)j]];
            const int32_t q = L.col[(size_t)j];
            if (best < 0 || d < bd || (d == bd && q < best)) { best = q; bd = d; }
        }
        if (best >= 0) dsu.unite(p, best);
    }
    std::vector<int32_t> label((size_t)g.n, -1);
    int32_t nc = 0;
    for (int32_t p = 0; p < g.n; ++p) {  // increasing p: a set's first visit is its smallest member
        const int32_t r = dsu.find(p);
        if (label[(size_t)r] < 0) label[(size_t)r] = nc++;
        agg[p] = label[(size_t)r];
    }
    return nc;
}

// Sec. 3.2 Galerkin coarse Laplacian L_l = H^{-T} L_{l-1} H^+ with H^+(p,i) = 1 for p in S_i:
// the coarse weight between aggregates I and J is the sum of the fine weights between them and
// intra-aggregate edges vanish. That is the canonical form of the list (agg[u], agg[v], w) taken in
// fine edge-id order. fine2coarse[e] = coarse edge id of fine edge e, or -1 inside an aggregate.
void galerkin(const Graph& g, const int32_t* agg, int32_t nc, Graph& c, int32_t* fine2coarse) {
    std::vector<int32_t> cu((size_t)g.m()), cv((size_t)g.m());
    for (int64_t e = 0; e < g.m(); ++e) { cu[(size_t)e] = agg[g.u[(size_t)e]]; cv[(size_t)e] = agg[g.v[(size_t)e]]; }
    canonicalize(nc, g.m(), cu.data(), cv.data(), g.w.data(), c);
    for (int64_t e = 0; e < g.m(); ++e) {
        int32_t a = std::min(cu[(size_t)e], cv[(size_t)e]), b = std::max(cu[(size_t)e], cv[(size_t)e]);
        if (a == b) { fine2coarse[e] = -1; continue; }
        int64_t lo = 0, hi = c.m();  // binary search (a, b) in the sorted coarse list
        while (lo < hi) {
            int64_t mid = (lo + hi) / 2;
            if (c.u[(size_t)mid] < a || (c.u[(size_t)mid] == a && c.v[(size_t)mid] < b)) lo = mid + 1;
            else hi = mid;
        }
        fine2coarse[e] = (int32_t)lo;
    }
}

// Sec. 3.4 / Algorithm 1 backward mapping. Inner-cluster: a maximum spanning tree of the subgraph
// induced by each aggregation set. Inter-cluster: for every edge (I, J) of P_l, the fine edge of
// largest weight between S_I and S_J (ties: smallest fine id).
void backward_map(const Graph& g, const int32_t* agg, const int32_t* fine2coarse,
                  const Graph& c, const uint8_t* pmask_c, uint8_t* pmask_f) {
    std::vector<uint8_t> inner((size_t)g.m());
    for (int64_t e = 0; e < g.m(); ++e) inner[(size_t)e] = agg[g.u[(size_t)e]] == agg[g.v[(size_t)e]];
    kruskal_max(g, inner.data(), pmask_f);
    std::vector<int32_t> best((size_t)c.m(), -1);
    for (int64_t e = 0; e < g.m(); ++e) {
        const int32_t ce = fine2coarse[e];
        if (ce < 0 || !pmask_c[ce]) continue;
        const int32_t b = best[(size_t)ce];
        if (b < 0 || g.w[(size_t)e] > g.w[(size_t)b]) best[(size_t)ce] = (int32_t)e;
    }
    for (int64_t ce = 0; ce < c.m(); ++ce)
        if (best[(size_t)ce] >= 0) pmask_f[best[(size_t)ce]] = 1;
}

int64_t round_half_up(double x) { return (int64_t)std::floor(x + 0.5); }

struct Params {
    int K, steps, levels;
    double omega;
    uint64_t seed;
    int mode;
    double budget_frac;
    int budget_unit;  // 0: k = round(beta * N_l); 1: k = round(beta * #off-tree edges of G_l)
    double eta;
};

// Add spectrally critical off-subgraph edges to the sparsifier mask of one level (Sec. 3.5,
// Algorithm 1, scoring and selection steps: score every edge outside the subgraph, add the top ones).
// Budget (reading): the level's sparsifier ends with round(beta * base) edges beyond a spanning
// forest (N_l - c_l edges); edges already present count; nothing is added if already over.
int64_t recover_edges(const Graph& g, const std::vector<double>& xg,
                      const Params& P, uint64_t seed, uint8_t* mask) {
    const int32_t comps = count_components(g);
    const int64_t forest = (int64_t)g.n - comps;
    const int64_t base = P.budget_unit == 0 ? (int64_t)g.n : g.m() - forest;
    const int64_t target = round_half_up(P.budget_frac * (double)base);
    int64_t in_p = 0;
    for (int64_t e = 0; e < g.m(); ++e) in_p += mask[e];
    std::vector<int32_t> cand;
    for (int64_t e = 0; e < g.m(); ++e)
        if (!mask[e]) cand.push_back((int32_t)e);
    int64_t k = target - (in_p - forest);
    if (k < 0) k = 0;
    if (k > (int64_t)cand.size()) k = (int64_t)cand.size();
    if (k == 0) return 0;
    Graph pg = subgraph(g, mask);
    Laplacian LP = build_laplacian(pg);
    std::vector<double> xp;
    smooth(LP, P.K, P.steps, P.omega, seed, xp);
    std::vector<double> sc(cand.size());
    score_edges(g, xg, xp, P.K, cand.data(), (int64_t)cand.size(), P.mode, P.eta, sc.data());
    std::vector<int32_t> sel((size_t)k);
    topk(sc.data(), cand.data(), (int64_t)cand.size(), k, sel.data());
    for (int32_t e : sel) mask[e] = 1;
    return k;
}

// Flat sparsifier of one graph: maximum spanning tree, then recovered off-tree edges.
void sparsify_flat(const Graph& g, const Params& P, uint64_t seed, uint8_t* mask) {
    kruskal_max(g, nullptr, mask);
    Laplacian LG = build_laplacian(g);
    std::vector<double> xg;
    smooth(LG, P.K, P.steps, P.omega, seed, xg);
    recover_edges(g, xg, P, seed, mask);
}

// Distance-1 colouring by Jones-Plassmann rounds (the Gauss-Seidel smoother's parallel order).
// Node priority: splitmix64(0x636f6c6f72 xor v), ties by the larger id. In each round every
// uncoloured node whose priority beats all its uncoloured neighbours is selected; all selected
// nodes then take the smallest colour not used by an already coloured neighbour. Selected nodes
// are never adjacent, so the order inside a round does not matter.
int32_t jp_coloring(const Laplacian& L, std::vector<int32_t>& color) {
    const int32_t n = L.n;
    color.assign((size_t)n, -1);
    auto prio = [](int32_t v) { return splitmix64(0x636f6c6f72ull ^ (uint64_t)(uint32_t)v); };
    auto beats = [&](int32_t a, int32_t b) {  // a outranks b
        const uint64_t pa = prio(a), pb = prio(b);
        return pa > pb || (pa == pb && a > b);
    };
    int32_t left = n, ncolors = 0;
    std::vector<int32_t> sel;
    while (left > 0) {
        sel.clear();
        for (int32_t v = 0; v < n; ++v) {
            if (color[(size_t)v] >= 0) continue;
            bool top = true;
            for (int64_t j = L.row_ptr[(size_t)v]; j < L.row_ptr[(size_t)v + 1] && top; ++j) {
                const int32_t u = L.col[(size_t)j];
                if (color[(size_t)u] < 0 && beats(u, v)) top = false;
            }
            if (top) sel.push_back(v);
        }
        for (int32_t v : sel) {
            std::vector<char> used;
            for (int64_t j = L.row_ptr[(size_t)v]; j < L.row_ptr[(size_t)v + 1]; ++j) {
                const int32_t c = color[(size_t)L.col[(size_t)j]];
                if (c >= 0) {
                    if ((size_t)c >= used.size()) used.resize((size_t)c + 1, 0);
                    used[(size_t)c] = 1;
                }
            }
            int32_t c = 0;
            while ((size_t)c < used.size() && used[(size_t)c]) ++c;
            color[(size_t)v] = c;
            ncolors = std::max(ncolors, c + 1);
        }
        left -= (int32_t)sel.size();
    }
    return ncolors;
}

// Gauss-Seidel sweeps on L x = 0 (Sec. 3.2 names Gauss-Seidel relaxation), over the nodes in
// colour order: x_p <- x_p - omega (L x)_p / D(p,p) with the current values of all neighbours
// (omega = 1: plain Gauss-Seidel). A node with D(p,p) = 0 is left unchanged.
void gauss_seidel(const Laplacian& L, const std::vector<int32_t>& color, int32_t ncolors, int K,
                  int steps, double omega, std::vector<double>& x) {
    std::vector<double> lx((size_t)K);
    for (int t = 0; t < steps; ++t)
        for (int32_t c = 0; c < ncolors; ++c)
            for (int32_t p = 0; p < L.n; ++p) {
                if (color[(size_t)p] != c) continue;
                const double d = L.deg[(size_t)p];
                if (d == 0.0) continue;
                for (int k = 0; k < K; ++k) lx[(size_t)k] = d * x[(size_t)p * K + k];
                for (int64_t j = L.row_ptr[(size_t)p]; j < L.row_ptr[(size_t)p + 1]; ++j) {
                    const int32_t q = L.col[(size_t)j];
                    for (int k = 0; k < K; ++k) lx[(size_t)k] -= L.a[(size_t)j] * x[(size_t)q * K + k];
                }
                for (int k = 0; k < K; ++k) x[(size_t)p * K + k] -= omega * lx[(size_t)k] / d;
            }
}

}  // namespace

extern "C" {

// Returns 0 on success, 1 on invalid input (ids out of range, non-finite or non-positive weight).
int orc_canonicalize(int32_t n, int64_t m, const int32_t* u, const int32_t* v, const float* w,
                     int32_t* cu, int32_t* cv, float* cw, int64_t* m_out) {
    Graph g;
    if (canonicalize(n, m, u, v, w, g)) return 1;
    for (int64_t e = 0; e < g.m(); ++e) { cu[e] = g.u[(size_t)e]; cv[e] = g.v[(size_t)e]; cw[e] = g.w[(size_t)e]; }
    *m_out = g.m();
    return 0;
}

static Graph make_graph(int32_t n, int64_t m, const int32_t* cu, const int32_t* cv, const float* cw) {
    Graph g;
    g.n = n;
    g.u.assign(cu, cu + m); g.v.assign(cv, cv + m); g.w.assign(cw, cw + m);
    return g;
}

// CSR of L from a canonical edge list: row_ptr[n+1], col/val/eid[2m], deg[n].
void orc_laplacian(int32_t n, int64_t m, const int32_t* cu, const int32_t* cv, const float* cw,
                   int64_t* row_ptr, int32_t* col, double* val, int32_t* eid, double* deg) {
    Laplacian L = build_laplacian(make_graph(n, m, cu, cv, cw));
    std::copy(L.row_ptr.begin(), L.row_ptr.end(), row_ptr);
    std::copy(L.col.begin(), L.col.end(), col);
    std::copy(L.a.begin(), L.a.end(), val);
    std::copy(L.eid.begin(), L.eid.end(), eid);
    std::copy(L.deg.begin(), L.deg.end(), deg);
}

void orc_laplacian_apply(int32_t n, int64_t m, const int32_t* cu, const int32_t* cv,
                         const float* cw, int K, const double* x, double* y) {
    Laplacian L = build_laplacian(make_graph(n, m, cu, cv, cw));
    std::vector<double> xv(x, x + (size_t)n * K), yv;
    laplacian_apply(L, K, xv, yv);
    std::copy(yv.begin(), yv.end(), y);
}

double orc_gaussian(uint64_t seed, uint64_t j) { return gaussian_draw(seed, j); }
uint64_t orc_splitmix64(uint64_t x) { return splitmix64(x); }

void orc_init_vectors(int32_t n, int K, uint64_t seed, double* x) {
    std::vector<double> xv;
    init_vectors(n, K, seed, xv);
    std::copy(xv.begin(), xv.end(), x);
}

// x (n x K, in/out): `steps` weighted-Jacobi sweeps, no initialisation, no projection.
void orc_jacobi(int32_t n, int64_t m, const int32_t* cu, const int32_t* cv, const float* cw,
                int K, int steps, double omega, double* x) {
    Laplacian L = build_laplacian(make_graph(n, m, cu, cv, cw));
    std::vector<double> xv(x, x + (size_t)n * K);
    jacobi(L, K, steps, omega, xv);
    std::copy(xv.begin(), xv.end(), x);
}

void orc_project(int32_t n, int K, double* x) {
    std::vector<double> xv(x, x + (size_t)n * K);
    project(n, K, xv);
    std::copy(xv.begin(), xv.end(), x);
}

// The whole local spectral embedding: seeded init, mean removal, Jacobi sweeps, projection.
void orc_smooth(int32_t n, int64_t m, const int32_t* cu, const int32_t* cv, const float* cw,
                int K, int steps, double omega, uint64_t seed, double* x) {
    Laplacian L = build_laplacian(make_graph(n, m, cu, cv, cw));
    std::vector<double> xv;
    smooth(L, K, steps, omega, seed, xv);
    std::copy(xv.begin(), xv.end(), x);
}

int32_t orc_coloring(int32_t n, int64_t m, const int32_t* cu, const int32_t* cv, const float* cw,
                     int32_t* color) {
    Laplacian L = build_laplacian(make_graph(n, m, cu, cv, cw));
    std::vector<int32_t> c;
    const int32_t nc = jp_coloring(L, c);
    std::copy(c.begin(), c.end(), color);
    return nc;
}

void orc_gauss_seidel(int32_t n, int64_t m, const int32_t* cu, const int32_t* cv, const float* cw,
                      int K, int steps, double omega, double* x) {
    Laplacian L = build_laplacian(make_graph(n, m, cu, cv, cw));
    std::vector<int32_t> c;
    const int32_t nc = jp_coloring(L, c);
    std::vector<double> xv(x, x + (size_t)n * K);
    gauss_seidel(L, c, nc, K, steps, omega, xv);
    std::copy(xv.begin(), xv.end(), x);
}

// Seeded vectors, Gauss-Seidel sweeps in colour order, projection.
void orc_smooth_gs(int32_t n, int64_t m, const int32_t* cu, const int32_t* cv, const float* cw,
                   int K, int steps, double omega, uint64_t seed, double* x) {
    Laplacian L = build_laplacian(make_graph(n, m, cu, cv, cw));
    std::vector<int32_t> c;
    const int32_t nc = jp_coloring(L, c);
    std::vector<double> xv;
    init_vectors(n, K, seed, xv);
    gauss_seidel(L, c, nc, K, steps, omega, xv);
    project(n, K, xv);
    std::copy(xv.begin(), xv.end(), x);
}

// Gauss-Seidel smoothing in a given colour order (a proper colouring of the graph, e.g. the
// colouring of a supergraph on the same nodes).
void orc_smooth_gs_colored(int32_t n, int64_t m, const int32_t* cu, const int32_t* cv,
                           const float* cw, const int32_t* color, int32_t ncolors, int K,
                           int steps, double omega, uint64_t seed, double* x) {
    Laplacian L = build_laplacian(make_graph(n, m, cu, cv, cw));
    std::vector<int32_t> c(color, color + n);
    std::vector<double> xv;
    init_vectors(n, K, seed, xv);
    gauss_seidel(L, c, ncolors, K, steps, omega, xv);
    project(n, K, xv);
    std::copy(xv.begin(), xv.end(), x);
}

void orc_score_edges(int32_t n, int64_t m, const int32_t* cu, const int32_t* cv, const float* cw,
                     const double* xg, const double* xp, int K, const int32_t* ids, int64_t ne,
                     int mode, double eta, double* out) {
    Graph g = make_graph(n, m, cu, cv, cw);
    std::vector<double> XG(xg, xg + (size_t)n * K), XP(xp, xp + (size_t)n * K);
    score_edges(g, XG, XP, K, ids, ne, mode, eta, out);
}

void orc_topk(const double* scores, const int32_t* ids, int64_t ne, int64_t k, int32_t* out) {
    topk(scores, ids, ne, k, out);
}

void orc_mst(int32_t n, int64_t m, const int32_t* cu, const int32_t* cv, const float* cw,
             const uint8_t* allow, uint8_t* mask) {
    kruskal_max(make_graph(n, m, cu, cv, cw), allow, mask);
}

int32_t orc_components(int32_t n, int64_t m, const int32_t* cu, const int32_t* cv) {
    std::vector<float> w((size_t)m, 1.0f);
    return count_components(make_graph(n, m, cu, cv, w.data()));
}

void orc_affinity(int32_t n, int64_t m, const int32_t* cu, const int32_t* cv, const float* cw,
                  const double* x, int K, double* delta) {
    std::vector<double> xv(x, x + (size_t)n * K);
    affinity(make_graph(n, m, cu, cv, cw), xv, K, delta);
}

int32_t orc_aggregate(int32_t n, int64_t m, const int32_t* cu, const int32_t* cv, const float* cw,
                      const double* delta, int32_t* agg) {
    Graph g = make_graph(n, m, cu, cv, cw);
    Laplacian L = build_laplacian(g);
    return aggregate(g, L, delta, agg);
}

// Coarse canonical edge list into cu_out/cv_out/cw_out (capacity m), count in *mc_out.
void orc_galerkin(int32_t n, int64_t m, const int32_t* cu, const int32_t* cv, const float* cw,
                  const int32_t* agg, int32_t nc, int32_t* cu_out, int32_t* cv_out, float* cw_out,
                  int64_t* mc_out, int32_t* fine2coarse) {
    Graph g = make_graph(n, m, cu, cv, cw), c;
    galerkin(g, agg, nc, c, fine2coarse);
    for (int64_t e = 0; e < c.m(); ++e) { cu_out[e] = c.u[(size_t)e]; cv_out[e] = c.v[(size_t)e]; cw_out[e] = c.w[(size_t)e]; }
    *mc_out = c.m();
}

void orc_backward_map(int32_t n, int64_t m, const int32_t* cu, const int32_t* cv, const float* cw,
                      const int32_t* agg, const int32_t* fine2coarse, int32_t nc, int64_t mc,
                      const int32_t* ccu, const int32_t* ccv, const float* ccw,
                      const uint8_t* pmask_c, uint8_t* pmask_f) {
    Graph g = make_graph(n, m, cu, cv, cw), c = make_graph(nc, mc, ccu, ccv, ccw);
    backward_map(g, agg, fine2coarse, c, pmask_c, pmask_f);
}

// Algorithm 1. levels == 0: flat (spanning tree + recovered off-tree edges). levels >= 1: the
// multilevel method (coarsen levels times, sparsify the coarsest graph flat, map back and recover
// edges at each finer level). Writes the sparsifier mask over G's canonical edges; returns the
// number of levels actually built (coarsening stops early when a level has no edges left).
// stats (may be NULL; 5 entries per level l = 0..levels): N_l, M_l, c_l (components of G_l), the
// edges of P_l before edge recovery at that level (the mapped backbone; the spanning forest at the
// coarsest level) and after it. agg_all (may be NULL; levels blocks of n entries): block l - 1
// holds the map from G_{l-1} to G_l. pmask_all (may be NULL; levels + 1 blocks of m entries):
// block l holds P_l over G_l's edges.
int orc_sparsify_levels(int32_t n, int64_t m, const int32_t* cu, const int32_t* cv, const float* cw,
                        int K, int steps, int levels, double omega, uint64_t seed, int mode,
                        double budget_frac, int budget_unit, double eta, uint8_t* mask_out,
                        int64_t* stats, int32_t* agg_all = nullptr, uint8_t* pmask_all = nullptr);

int orc_sparsify(int32_t n, int64_t m, const int32_t* cu, const int32_t* cv, const float* cw,
                 int K, int steps, int levels, double omega, uint64_t seed, int mode,
                 double budget_frac, int budget_unit, double eta, uint8_t* mask_out) {
    return orc_sparsify_levels(n, m, cu, cv, cw, K, steps, levels, omega, seed, mode, budget_frac,
                               budget_unit, eta, mask_out, nullptr);
}

int orc_sparsify_levels(int32_t n, int64_t m, const int32_t* cu, const int32_t* cv, const float* cw,
                        int K, int steps, int levels, double omega, uint64_t seed, int mode,
                        double budget_frac, int budget_unit, double eta, uint8_t* mask_out,
                        int64_t* stats, int32_t* agg_all, uint8_t* pmask_all) {
    Params P{K, steps, levels, omega, seed, mode, budget_frac, budget_unit, eta};
    std::vector<Graph> G(1, make_graph(n, m, cu, cv, cw));
    std::vector<std::vector<int32_t>> AGG(1), F2C(1);
    std::vector<std::vector<double>> XG;
    int lf = 0;
    for (int l = 1; l <= levels; ++l) {  // Algorithm 1, coarsening phase: multilevel spectral reduction
        const Graph& f = G.back();
        if (f.m() == 0) break;
        Laplacian L = build_laplacian(f);
        std::vector<double> x;
        smooth(L, K, steps, omega, level_seed(seed, l - 1), x);
        std::vector<double> delta((size_t)f.m());
        affinity(f, x, K, delta.data());
        std::vector<int32_t> agg((size_t)f.n);
        const int32_t nc = aggregate(f, L, delta.data(), agg.data());
        Graph c;
        std::vector<int32_t> f2c((size_t)f.m());
        galerkin(f, agg.data(), nc, c, f2c.data());
        XG.push_back(std::move(x));
        AGG.push_back(std::move(agg));
        F2C.push_back(std::move(f2c));
        G.push_back(std::move(c));
        lf = l;
    }
    auto count = [](const std::vector<uint8_t>& mk) {
        int64_t c = 0;
        for (uint8_t b : mk) c += b;
        return c;
    };
    auto record = [&](int l, int64_t before, int64_t after, const std::vector<uint8_t>& mk) {
        if (pmask_all) std::copy(mk.begin(), mk.end(), pmask_all + (size_t)l * (size_t)m);
        if (agg_all && l >= 1)
            std::copy(AGG[(size_t)l].begin(), AGG[(size_t)l].end(), agg_all + (size_t)(l - 1) * (size_t)n);
        if (!stats) return;
        const Graph& gl = G[(size_t)l];
        int64_t* s = stats + 5 * l;
        s[0] = gl.n; s[1] = gl.m(); s[2] = count_components(gl); s[3] = before; s[4] = after;
    };
    std::vector<uint8_t> pm((size_t)G[(size_t)lf].m());
    {
        kruskal_max(G[(size_t)lf], nullptr, pm.data());
        const int64_t before = count(pm);
        sparsify_flat(G[(size_t)lf], P, level_seed(seed, lf), pm.data());
        record(lf, before, count(pm), pm);
    }
    for (int l = lf; l >= 1; --l) {  // Algorithm 1, level loop
        const Graph& f = G[(size_t)l - 1];
        std::vector<uint8_t> pf((size_t)f.m());
        backward_map(f, AGG[(size_t)l].data(), F2C[(size_t)l].data(), G[(size_t)l], pm.data(), pf.data());
        const int64_t before = count(pf);
        recover_edges(f, XG[(size_t)l - 1], P, level_seed(seed, l - 1), pf.data());
        record(l - 1, before, count(pf), pf);
        pm.swap(pf);
    }
    std::copy(pm.begin(), pm.end(), mask_out);
    return lf;
}

}  // extern "C"
