// Contraction-path optimisation on the host (tn_path_optimize, declared in tn.h).
//
// Simulated annealing over the contraction tree (Sec. 3.2).  A state is a binary tree whose
// leaves are the network's tensors; its energy is the score
//     log2(T_cc + alpha T_mc) + beta log2(T_sc)
// with T_cc the multiply-add count of all pairwise steps (8 real flops each), T_mc the elements
// the steps read and write, and T_sc the largest intermediate.  The local update exchanges the
// three nearest descendants of a vertex: a vertex X = (A, Q) with Q = (B, C) becomes
// X = ((A, C), B) or X = ((A, B), C), the two possible directions.  A sweep visits every internal
// vertex from the root towards the leaves and tries one update at each, accepted by the
// Metropolis rule at the current temperature (score units, log2).
//
// Dynamic slicing (Sec. 3.2): while the largest intermediate exceeds the target, the bond whose
// removal gives the lowest score (over all slices) is sliced and the tree is re-tuned by further
// sweeps, so the order adapts to the sliced network.
//
// Every dimension is 2 and every label lies on two tensors (or on one tensor and the output), so
// the label set of a contraction result is the symmetric difference of its operands' sets and a
// step's multiply-add count is 2^|union of the operands' labels|; sliced labels are masked out.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <queue>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tn.h"

namespace tn {
tn_status report(tn_status s, const char *msg);  // records the thread's error message
void clear_error();                               // clears it (every entry point)
}

namespace {

// splitmix64-seeded xoshiro256** (published definitions), for reproducible chains
struct Rng {
    uint64_t s[4];
    explicit Rng(uint64_t seed) {
        for (int i = 0; i < 4; ++i) {
            seed += 0x9e3779b97f4a7c15ull;
            uint64_t z = seed;
            z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
            z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
            s[i] = z ^ (z >> 31);
        }
    }
    static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
    uint64_t next() {
        const uint64_t r = rotl(s[1] * 5, 7) * 9;
        const uint64_t t = s[1] << 17;
        s[2] ^= s[0];
        s[3] ^= s[1];
        s[1] ^= s[2];
        s[0] ^= s[3];
        s[2] ^= t;
        s[3] = rotl(s[3], 45);
        return r;
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

struct Problem {
    int n = 0;                      // leaves
    int W = 0;                      // 64-bit words per label set
    std::vector<uint64_t> leaf;     // n * W
    std::vector<uint64_t> openm;    // W: open labels (never sliced)
    std::vector<int32_t> value;     // dense label id -> label
};

struct Tree {
    int n = 0, W = 0, root = -1;
    std::vector<int> lc, rc, par;   // 2n - 1 nodes; leaves 0..n-1
    std::vector<uint64_t> L;        // label sets, (2n - 1) * W
    std::vector<int> sz, cc;        // |L \ S| and |(L_l | L_r) \ S| (internal nodes)
    std::vector<uint64_t> S;        // sliced mask
    int nsl = 0;
    // histograms over internal nodes: cc exponents, T_mc terms, sizes (index = log2)
    std::vector<int64_t> hcc, hmc, hsz;
    // balanced indices (App. A.2): cc exponents of the unbalanced internal nodes, whose
    // multiply-adds count 2^gb times in the score (gb = 0: off)
    std::vector<int64_t> hub;
    int gb = 0;
    int emax = 0;  // histogram length: number of labels + 1

    // a step with children of su and sw labels and cc labels in their union, as a GEMM:
    // k = su + sw - cc contracted labels, m = su - k and n = sw - k free ones; unbalanced when
    // k < 2^6 or min(m, n) < 2^5 elements
    static bool unbalanced(int su, int sw, int c) {
        const int k = su + sw - c;
        return k < 6 || std::min(su - k, sw - k) < 5;
    }

    const uint64_t *set(int v) const { return &L[(size_t)v * W]; }
    uint64_t *set(int v) { return &L[(size_t)v * W]; }
    int pc_masked(const uint64_t *a) const {
        int c = 0;
        for (int w = 0; w < W; ++w) c += __builtin_popcountll(a[w] & ~S[w]);
        return c;
    }
    int pc_union(const uint64_t *a, const uint64_t *b) const {
        int c = 0;
        for (int w = 0; w < W; ++w) c += __builtin_popcountll((a[w] | b[w]) & ~S[w]);
        return c;
    }

    // recompute every set, size and histogram from the structure (post-order)
    void rebuild() {
        hcc.assign(emax, 0);
        hmc.assign(emax, 0);
        hsz.assign(emax, 0);
        hub.assign(emax, 0);
        std::vector<int> order;
        order.reserve(2 * n);
        std::vector<int> st{root};
        while (!st.empty()) {
            const int v = st.back();
            st.pop_back();
            order.push_back(v);
            if (v >= n) {
                st.push_back(lc[v]);
                st.push_back(rc[v]);
            }
        }
        for (auto it = order.rbegin(); it != order.rend(); ++it) {
            const int v = *it;
            if (v < n) {
                sz[v] = pc_masked(set(v));
                continue;
            }
            const uint64_t *a = set(lc[v]), *b = set(rc[v]);
            uint64_t *o = set(v);
            for (int w = 0; w < W; ++w) o[w] = a[w] ^ b[w];
            sz[v] = pc_masked(o);
            cc[v] = pc_union(a, b);
            hcc[cc[v]] += 1;
            if (gb > 0 && unbalanced(sz[lc[v]], sz[rc[v]], cc[v])) hub[cc[v]] += 1;
            hmc[sz[lc[v]]] += 1;
            hmc[sz[rc[v]]] += 1;
            hmc[sz[v]] += 1;
            hsz[sz[v]] += 1;
        }
    }

    int max_size() const { return hist_top(hsz); }
    static int hist_top(const std::vector<int64_t> &h) {
        for (int e = (int)h.size() - 1; e >= 0; --e)
            if (h[e]) return e;
        return 0;
    }
    // log2 of sum_e h[e] 2^e, evaluated relative to the top exponent (no overflow); terms more
    // than 2^-80 below the top are dropped
    static double log2_sum(const std::vector<int64_t> &h) {
        const int top = hist_top(h);
        double s = 0.0;
        for (int e = top; e >= 0 && e > top - 80; --e)
            if (h[e]) s += std::ldexp((double)h[e], e - top);
        return s > 0.0 ? top + std::log2(s) : 0.0;
    }
    // score over all slices: nsl + log2(T_cc + alpha T_mc) + beta log2(T_sc); T_cc counted in
    // multiply-adds (the factor 8 of real flops is a constant offset)
    double score(double alpha, double beta) const {
        double l = log2_sum(hcc);
        if (gb > 0 && std::any_of(hub.begin(), hub.end(), [](int64_t x) { return x != 0; })) {
            // T_cc + (2^gb - 1) T_unbalanced
            const double y = std::log2(std::exp2((double)gb) - 1.0) + log2_sum(hub);
            const double m = std::max(l, y);
            l = m + std::log2(std::exp2(l - m) + std::exp2(y - m));
        }
        if (alpha > 0) {
            const double y = std::log2(alpha) + log2_sum(hmc);
            const double m = std::max(l, y);
            l = m + std::log2(std::exp2(l - m) + std::exp2(y - m));
        }
        return nsl + l + beta * max_size();
    }
};

// Tree from a pair path (a, b): the result takes id a, id b is retired.
bool tree_from_path(const Problem &P, const int32_t *path, Tree &T, std::string &err) {
    const int n = P.n;
    T.n = n;
    T.W = P.W;
    T.lc.assign(2 * n - 1, -1);
    T.rc.assign(2 * n - 1, -1);
    T.par.assign(2 * n - 1, -1);
    T.L.assign((size_t)(2 * n - 1) * P.W, 0);
    T.sz.assign(2 * n - 1, 0);
    T.cc.assign(2 * n - 1, 0);
    T.S.assign(P.W, 0);
    T.emax = (int)P.value.size() + 1;
    std::copy(P.leaf.begin(), P.leaf.end(), T.L.begin());
    std::vector<int> node(n);
    std::vector<char> alive(n, 1);
    for (int i = 0; i < n; ++i) node[i] = i;
    for (int s = 0; s < n - 1; ++s) {
        const int a = path[2 * s], b = path[2 * s + 1];
        if (a < 0 || b < 0 || a >= n || b >= n || a == b || !alive[a] || !alive[b]) {
            err = "path step " + std::to_string(s) + " uses a retired or invalid id";
            return false;
        }
        const int v = n + s;
        T.lc[v] = node[a];
        T.rc[v] = node[b];
        T.par[node[a]] = v;
        T.par[node[b]] = v;
        node[a] = v;
        alive[b] = 0;
    }
    T.root = n == 1 ? 0 : 2 * n - 2;
    return true;
}

// Post-order pairs of the tree: each internal vertex contracts the representatives (lowest
// leaf id reached first) of its two subtrees; the result keeps the left representative.
void path_from_tree(const Tree &T, int32_t *out) {
    const int n = T.n;
    if (n == 1) return;
    std::vector<int> rep(2 * n - 1, -1);
    for (int i = 0; i < n; ++i) rep[i] = i;
    std::vector<int> order;
    std::vector<int> st{T.root};
    while (!st.empty()) {
        const int v = st.back();
        st.pop_back();
        if (v < n) continue;
        order.push_back(v);
        st.push_back(T.lc[v]);
        st.push_back(T.rc[v]);
    }
    int k = 0;
    for (auto it = order.rbegin(); it != order.rend(); ++it) {
        const int v = *it;
        int a = rep[T.lc[v]], b = rep[T.rc[v]];
        if (b < a) std::swap(a, b);
        out[2 * k] = a;
        out[2 * k + 1] = b;
        rep[v] = a;
        ++k;
    }
}

struct Params {
    double alpha, beta, t_start, t_end;
    int sweeps, sweeps_per_slice, sweeps_final, max_log2_size, max_sliced, greedy_trials;
};

// Random greedy tree: repeatedly contract the connected pair with the lowest perturbed cost
// log2 size(result) - g * log2(size(a) + size(b)) (sizes in elements, every dim 2); the
// perturbation subtracts 8 * temp * G with G a Gumbel(0, 1) draw, so temp = 0 is a plain greedy
// rule.  (In log units a large result is charged by its width, not its element count, which
// keeps the rule from contracting every small pair before the first large one.)  Tensors left
// without a shared label at the end are paired smallest first.
void random_greedy(const Problem &P, Rng &rng, double g, double temp, Tree &T) {
    const int n = P.n, W = P.W;
    T.n = n;
    T.W = W;
    T.lc.assign(2 * n - 1, -1);
    T.rc.assign(2 * n - 1, -1);
    T.par.assign(2 * n - 1, -1);
    T.L.assign((size_t)(2 * n - 1) * W, 0);
    T.sz.assign(2 * n - 1, 0);
    T.cc.assign(2 * n - 1, 0);
    if (T.S.size() != (size_t)W) T.S.assign(W, 0);
    T.emax = (int)P.value.size() + 1;
    std::copy(P.leaf.begin(), P.leaf.end(), T.L.begin());
    const int nl = (int)P.value.size();
    std::vector<int> holder((size_t)nl * 2, -1);   // the (at most two) active holders of a label
    std::vector<int> version((size_t)(2 * n - 1), 0);
    std::vector<char> alive((size_t)(2 * n - 1), 0);
    std::vector<int> pc((size_t)(2 * n - 1), 0);   // label counts
    auto add_holder = [&](int l, int v) {
        if (holder[2 * l] < 0) holder[2 * l] = v;
        else holder[2 * l + 1] = v;
    };
    auto drop_holder = [&](int l, int v) {
        if (holder[2 * l] == v) holder[2 * l] = -1;
        else if (holder[2 * l + 1] == v) holder[2 * l + 1] = -1;
    };
    for (int v = 0; v < n; ++v) {
        alive[v] = 1;
        const uint64_t *lv = T.set(v);
        for (int w = 0; w < W; ++w) {
            uint64_t b = lv[w];
            pc[v] += __builtin_popcountll(b);
            while (b) {
                add_holder(w * 64 + __builtin_ctzll(b), v);
                b &= b - 1;
            }
        }
    }
    struct Cand {
        double key;
        int a, b, va, vb;
        bool operator<(const Cand &o) const { return key > o.key; }  // min-heap
    };
    std::priority_queue<Cand> q;
    auto push_pair = [&](int a, int b) {
        const uint64_t *la = T.set(a), *lb = T.set(b);
        int x = 0;
        for (int w = 0; w < W; ++w) x += __builtin_popcountll(la[w] ^ lb[w]);
        const double cost = (double)x - g * std::log2(std::ldexp(1.0, pc[a]) + std::ldexp(1.0, pc[b]));
        double key = cost;
        if (temp > 0) {
            double u = rng.uniform();
            if (u < 1e-300) u = 1e-300;
            key -= 8.0 * temp * (-std::log(-std::log(u)));
        }
        q.push(Cand{key, a, b, version[a], version[b]});
    };
    auto push_neighbours = [&](int v) {
        const uint64_t *lv = T.set(v);
        for (int w = 0; w < W; ++w) {
            uint64_t b = lv[w];
            while (b) {
                const int l = w * 64 + __builtin_ctzll(b);
                b &= b - 1;
                for (int h = 0; h < 2; ++h) {
                    const int u = holder[2 * l + h];
                    if (u >= 0 && u != v && u < v) push_pair(u, v);
                    else if (u >= 0 && u != v) push_pair(v, u);
                }
            }
        }
    };
    for (int v = 0; v < n; ++v) push_neighbours(v);
    int next = n, remaining = n;
    auto merge = [&](int a, int b) {
        const int c = next++;
        T.lc[c] = a;
        T.rc[c] = b;
        T.par[a] = c;
        T.par[b] = c;
        const uint64_t *la = T.set(a), *lb = T.set(b);
        uint64_t *lc = T.set(c);
        for (int w = 0; w < W; ++w) {
            lc[w] = la[w] ^ lb[w];
            for (uint64_t x = la[w]; x; x &= x - 1) drop_holder(w * 64 + __builtin_ctzll(x), a);
            for (uint64_t x = lb[w]; x; x &= x - 1) drop_holder(w * 64 + __builtin_ctzll(x), b);
        }
        for (int w = 0; w < W; ++w)
            for (uint64_t x = lc[w]; x; x &= x - 1) {
                add_holder(w * 64 + __builtin_ctzll(x), c);
                pc[c] += 1;
            }
        alive[a] = alive[b] = 0;
        version[a]++;
        version[b]++;
        alive[c] = 1;
        --remaining;
        return c;
    };
    while (!q.empty()) {
        const Cand t = q.top();
        q.pop();
        if (!alive[t.a] || !alive[t.b] || version[t.a] != t.va || version[t.b] != t.vb) continue;
        const int c = merge(t.a, t.b);
        push_neighbours(c);
    }
    // no shared label left: pair the remaining tensors, smallest first
    while (remaining > 1) {
        int a = -1, b = -1;
        for (int v = 0; v < next; ++v) {
            if (!alive[v]) continue;
            if (a < 0 || pc[v] < pc[a]) {
                b = a;
                a = v;
            } else if (b < 0 || pc[v] < pc[b]) {
                b = v;
            }
        }
        merge(a, b);
    }
    T.root = n == 1 ? 0 : next - 1;
}

struct Chain {
    Tree T;
    Rng rng;
    int64_t tried = 0, accepted = 0;
    std::vector<uint64_t> scratch;  // the candidate label set of a local update
    Chain(const Tree &t, uint64_t seed) : T(t), rng(seed), scratch(t.W) {}

    // one local update at internal vertex x (Metropolis at temperature temp)
    void update(int x, double temp, const Params &p, double &cur) {
        Tree &t = T;
        const int n = t.n;
        const int c0 = t.lc[x], c1 = t.rc[x];
        const bool i0 = c0 >= n, i1 = c1 >= n;
        if (!i0 && !i1) return;
        const int q = (i0 && i1) ? ((rng.next() >> 63) ? c0 : c1) : (i0 ? c0 : c1);
        const int a = q == c0 ? c1 : c0;
        const bool keep_left = (rng.next() >> 63) != 0;  // which grandchild pairs with a
        const int k = keep_left ? t.lc[q] : t.rc[q];
        const int m = keep_left ? t.rc[q] : t.lc[q];
        ++tried;
        // new set of q: L_a ^ L_k
        uint64_t *lq = t.set(q);
        const uint64_t *la = t.set(a), *lk = t.set(k), *lm = t.set(m);
        const int W = t.W;
        uint64_t *nqp = scratch.data();
        for (int w = 0; w < W; ++w) nqp[w] = la[w] ^ lk[w];
        const int sz_q_old = t.sz[q], cc_q_old = t.cc[q], cc_x_old = t.cc[x];
        const int sz_q_new = t.pc_masked(nqp);
        const int cc_q_new = t.pc_union(la, lk);
        const int cc_x_new = t.pc_union(nqp, lm);
        // balance of q and x before (q = (k, m), x = (q, a)) and after (q = (a, k), x = (q, m))
        bool ub_old_q = false, ub_old_x = false, ub_new_q = false, ub_new_x = false;
        if (t.gb > 0) {
            ub_old_q = Tree::unbalanced(t.sz[k], t.sz[m], cc_q_old);
            ub_old_x = Tree::unbalanced(sz_q_old, t.sz[a], cc_x_old);
            ub_new_q = Tree::unbalanced(t.sz[a], t.sz[k], cc_q_new);
            ub_new_x = Tree::unbalanced(sz_q_new, t.sz[m], cc_x_new);
        }
        auto apply = [&](int sq_rm, int cq_rm, int cx_rm, int sq_add, int cq_add, int cx_add,
                         bool uq_rm, bool ux_rm, bool uq_add, bool ux_add) {
            t.hcc[cq_rm] -= 1;
            t.hcc[cx_rm] -= 1;
            t.hcc[cq_add] += 1;
            t.hcc[cx_add] += 1;
            if (t.gb > 0) {
                t.hub[cq_rm] -= uq_rm;
                t.hub[cx_rm] -= ux_rm;
                t.hub[cq_add] += uq_add;
                t.hub[cx_add] += ux_add;
            }
            t.hmc[sq_rm] -= 2;
            t.hmc[sq_add] += 2;
            t.hsz[sq_rm] -= 1;
            t.hsz[sq_add] += 1;
        };
        apply(sz_q_old, cc_q_old, cc_x_old, sz_q_new, cc_q_new, cc_x_new, ub_old_q, ub_old_x,
              ub_new_q, ub_new_x);
        const double nxt = t.score(p.alpha, p.beta);
        const double d = nxt - cur;
        if (d <= 0.0 || (temp > 0.0 && rng.uniform() < std::exp(-d / temp))) {
            // q = (a, k), x = (q, m)
            t.lc[q] = a;
            t.rc[q] = k;
            t.par[a] = q;
            t.par[k] = q;
            t.lc[x] = q;
            t.rc[x] = m;
            t.par[m] = x;
            std::memcpy(lq, nqp, sizeof(uint64_t) * W);
            t.sz[q] = sz_q_new;
            t.cc[q] = cc_q_new;
            t.cc[x] = cc_x_new;
            cur = nxt;
            ++accepted;
        } else {
            apply(sz_q_new, cc_q_new, cc_x_new, sz_q_old, cc_q_old, cc_x_old, ub_new_q, ub_new_x,
                  ub_old_q, ub_old_x);
        }
    }

    // sweeps from the root to the leaves, temperature geometric from t0 to t1
    void anneal(int sweeps, double t0, double t1, const Params &p) {
        if (sweeps <= 0 || T.n < 3) return;
        double cur = T.score(p.alpha, p.beta);
        std::vector<int> order;
        for (int s = 0; s < sweeps; ++s) {
            const double temp = sweeps == 1 ? t1 : t0 * std::pow(t1 / t0, (double)s / (sweeps - 1));
            order.clear();
            order.push_back(T.root);
            for (size_t h = 0; h < order.size(); ++h) {
                const int v = order[h];
                if (T.lc[v] >= T.n) order.push_back(T.lc[v]);
                if (T.rc[v] >= T.n) order.push_back(T.rc[v]);
            }
            for (int v : order) update(v, temp, p, cur);
            // exact re-evaluation once per sweep keeps the running score honest
            cur = T.score(p.alpha, p.beta);
        }
    }

    // slice the bond whose removal gives the lowest score; false when none is left
    bool slice_one(const Problem &P, const Params &p) {
        const int W = T.W;
        const int mx = T.max_size();
        std::vector<uint64_t> cand(W, 0);
        for (int v = T.n; v < 2 * T.n - 1; ++v)
            if (T.sz[v] == mx) {
                const uint64_t *l = T.set(v);
                for (int w = 0; w < W; ++w) cand[w] |= l[w];
            }
        double best = 0.0;
        int best_id = -1;
        for (int w = 0; w < W; ++w) {
            uint64_t bits = cand[w] & ~T.S[w] & ~P.openm[w];
            while (bits) {
                const int b = __builtin_ctzll(bits);
                bits &= bits - 1;
                const int id = w * 64 + b;
                T.S[w] |= 1ull << b;
                T.nsl += 1;
                T.rebuild();
                const double s = T.score(p.alpha, p.beta);
                T.S[w] &= ~(1ull << b);
                T.nsl -= 1;
                if (best_id < 0 || s < best ||
                    (s == best && P.value[id] < P.value[best_id])) {
                    best = s;
                    best_id = id;
                }
            }
        }
        if (best_id < 0) {
            T.rebuild();
            return false;
        }
        T.S[best_id / 64] |= 1ull << (best_id % 64);
        T.nsl += 1;
        T.rebuild();
        return true;
    }

    // random greedy trees with sampled cost weight and temperature; keep the best by score
    void greedy_start(const Problem &P, const Params &p) {
        T.rebuild();
        double best = T.score(p.alpha, p.beta);
        Tree cand = T;
        for (int k = 0; k < p.greedy_trials; ++k) {
            const double g = 0.5 + rng.uniform();                      // size weight in [0.5, 1.5)
            const double temp = std::exp2(-8.0 + 8.0 * rng.uniform());  // in [2^-8, 1)
            random_greedy(P, rng, g, temp, cand);
            cand.rebuild();
            const double sc = cand.score(p.alpha, p.beta);
            if (sc < best) {
                best = sc;
                T = cand;
            }
        }
    }

    void run(const Problem &P, const Params &p) {
        if (p.greedy_trials > 0) greedy_start(P, p);
        T.rebuild();
        anneal(p.sweeps, p.t_start, p.t_end, p);
        if (p.max_log2_size > 0) {
            while (T.max_size() > p.max_log2_size && T.nsl < p.max_sliced) {
                if (!slice_one(P, p)) break;
                anneal(p.sweeps_per_slice, p.t_end * 4.0, p.t_end, p);
            }
        }
        anneal(p.sweeps_final, p.t_end * 4.0, p.t_end, p);
        T.rebuild();
    }
};

}  // namespace

static tn_status path_optimize_impl(int32_t num_tensors, const int32_t *ranks,
                                    const int32_t *const *labels, int32_t num_open,
                                    const int32_t *open_labels, const int32_t *path_in,
                                    const tn_path_options *opts, int32_t *path_out,
                                    int32_t *sliced_out, int32_t sliced_capacity,
                                    tn_path_info *info);

extern "C" tn_status tn_path_optimize(int32_t num_tensors, const int32_t *ranks,
                                      const int32_t *const *labels, int32_t num_open,
                                      const int32_t *open_labels, const int32_t *path_in,
                                      const tn_path_options *opts, int32_t *path_out,
                                      int32_t *sliced_out, int32_t sliced_capacity,
                                      tn_path_info *info) {
    tn::clear_error();
    try {
        return path_optimize_impl(num_tensors, ranks, labels, num_open, open_labels, path_in,
                                  opts, path_out, sliced_out, sliced_capacity, info);
    } catch (const std::bad_alloc &) {
        return tn::report(TN_ERR_OOM, "tn_path_optimize: host memory exhausted");
    } catch (...) {
        return tn::report(TN_ERR_INVALID_ARG, "tn_path_optimize: internal error");
    }
}

static tn_status path_optimize_impl(int32_t num_tensors, const int32_t *ranks,
                                    const int32_t *const *labels, int32_t num_open,
                                    const int32_t *open_labels, const int32_t *path_in,
                                    const tn_path_options *opts, int32_t *path_out,
                                    int32_t *sliced_out, int32_t sliced_capacity,
                                    tn_path_info *info) {
    if (num_tensors < 1 || !ranks || !labels || num_open < 0 || (num_open > 0 && !open_labels) ||
        (num_tensors > 1 && (!path_in || !path_out)) || sliced_capacity < 0 ||
        (sliced_capacity > 0 && !sliced_out) || !info)
        return tn::report(TN_ERR_INVALID_ARG, "tn_path_optimize: invalid argument");
    tn_path_options o{};
    o.sweeps = 200;
    o.sweeps_per_slice = 40;
    o.sweeps_final = 200;
    o.t_start = 0.05;
    o.t_end = 0.001;
    o.max_sliced = 64;
    o.chains = 1;
    if (opts) {
        o.seed = opts->seed;
        if (opts->sweeps >= 0) o.sweeps = opts->sweeps;
        if (opts->sweeps_per_slice >= 0) o.sweeps_per_slice = opts->sweeps_per_slice;
        if (opts->sweeps_final >= 0) o.sweeps_final = opts->sweeps_final;
        if (opts->t_start > 0) o.t_start = opts->t_start;
        if (opts->t_end > 0) o.t_end = opts->t_end;
        o.alpha = opts->alpha;
        o.beta = opts->beta;
        o.max_log2_size = opts->max_log2_size;
        if (opts->max_sliced > 0) o.max_sliced = opts->max_sliced;
        if (opts->chains > 0) o.chains = opts->chains;
        if (opts->greedy_trials > 0) o.greedy_trials = opts->greedy_trials;
        o.balance_log2 = opts->balance_log2;
    }
    if (o.alpha < 0 || o.beta < 0 || o.max_log2_size < 0 || o.chains > 256 || o.t_end > o.t_start ||
        o.balance_log2 < 0 || o.balance_log2 > 16)
        return tn::report(TN_ERR_INVALID_ARG, "tn_path_optimize: invalid option");
    o.max_sliced = std::min(o.max_sliced, sliced_capacity);

    // dense label ids; every label on two tensors, or on one tensor and the output
    Problem P;
    P.n = num_tensors;
    std::unordered_map<int32_t, int> id;
    std::vector<int> count;
    auto get = [&](int32_t l) {
        auto it = id.find(l);
        if (it != id.end()) return it->second;
        const int k = (int)P.value.size();
        id.emplace(l, k);
        P.value.push_back(l);
        count.push_back(0);
        return k;
    };
    std::vector<std::vector<int>> lab(num_tensors);
    for (int i = 0; i < num_tensors; ++i) {
        if (ranks[i] < 0 || (ranks[i] > 0 && !labels[i]))
            return tn::report(TN_ERR_INVALID_ARG, "tn_path_optimize: invalid rank or labels");
        for (int r = 0; r < ranks[i]; ++r) {
            const int k = get(labels[i][r]);
            for (int q : lab[i])
                if (q == k)
                    return tn::report(TN_ERR_SHAPE, "tn_path_optimize: label repeated on a tensor");
            lab[i].push_back(k);
            count[k] += 1;
        }
    }
    std::vector<char> is_open(P.value.size(), 0);
    for (int j = 0; j < num_open; ++j) {
        auto it = id.find(open_labels[j]);
        if (it == id.end() || is_open[it->second])
            return tn::report(TN_ERR_SHAPE, "tn_path_optimize: open label not on a tensor");
        is_open[it->second] = 1;
    }
    for (size_t k = 0; k < P.value.size(); ++k) {
        const int need = is_open[k] ? 1 : 2;
        if (count[k] > 2)
            return tn::report(TN_ERR_UNSUPPORTED,
                              "tn_path_optimize: hyperedge (label on three or more tensors)");
        if (count[k] != need)
            return tn::report(TN_ERR_SHAPE, "tn_path_optimize: dangling or over-used label");
    }
    P.W = std::max(1, (int)((P.value.size() + 63) / 64));
    P.leaf.assign((size_t)num_tensors * P.W, 0);
    P.openm.assign(P.W, 0);
    for (int i = 0; i < num_tensors; ++i)
        for (int k : lab[i]) P.leaf[(size_t)i * P.W + k / 64] |= 1ull << (k % 64);
    for (size_t k = 0; k < P.value.size(); ++k)
        if (is_open[k]) P.openm[k / 64] |= 1ull << (k % 64);

    Tree T0;
    std::string err;
    if (num_tensors > 1 && !tree_from_path(P, path_in, T0, err))
        return tn::report(TN_ERR_PATH, ("tn_path_optimize: " + err).c_str());
    if (num_tensors == 1) {
        *info = tn_path_info{};
        return TN_OK;
    }
    T0.gb = o.balance_log2;
    T0.rebuild();
    const Params prm{o.alpha, o.beta, o.t_start, o.t_end, o.sweeps, o.sweeps_per_slice,
                     o.sweeps_final, o.max_log2_size, o.max_sliced, o.greedy_trials};
    tn_path_info out{};
    out.initial_log2_tcc = 3.0 + Tree::log2_sum(T0.hcc);
    out.initial_max_log2_size = T0.max_size();

    // independent chains (one thread each), the lowest final score wins, ties to the first
    std::vector<Chain> chains;
    chains.reserve(o.chains);
    for (int c = 0; c < o.chains; ++c)
        chains.emplace_back(T0, o.seed * 0x9e3779b97f4a7c15ull + (uint64_t)c + 1);
    // chains that get no thread (thread creation refused) run on the calling thread; nothing
    // is thrown across the C ABI
    std::vector<std::thread> th;
    std::vector<char> started((size_t)o.chains, 0);
    for (int c = 1; c < o.chains; ++c) {
        try {
            th.emplace_back([&, c] { chains[c].run(P, prm); });
            started[(size_t)c] = 1;
        } catch (...) {
            break;
        }
    }
    for (int c = 0; c < o.chains; ++c)
        if (!started[(size_t)c]) chains[c].run(P, prm);
    for (auto &t : th) t.join();
    int best = 0;
    double best_score = chains[0].T.score(o.alpha, o.beta);
    for (int c = 1; c < o.chains; ++c) {
        const double s = chains[c].T.score(o.alpha, o.beta);
        if (s < best_score) {
            best_score = s;
            best = c;
        }
    }
    const Tree &T = chains[best].T;
    path_from_tree(T, path_out);
    int ns = 0;
    for (size_t k = 0; k < P.value.size(); ++k)
        if (T.S[k / 64] >> (k % 64) & 1) sliced_out[ns++] = P.value[k];
    out.log2_tcc = 3.0 + Tree::log2_sum(T.hcc);
    out.log2_tcc_total = out.log2_tcc + ns;
    out.log2_tmc = Tree::log2_sum(T.hmc);
    out.max_log2_size = T.max_size();
    out.num_sliced = ns;
    out.score = best_score;
    for (const auto &c : chains) {
        out.moves_tried += c.tried;
        out.moves_accepted += c.accepted;
    }
    *info = out;
    return TN_OK;
}
