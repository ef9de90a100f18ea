// Sparse-state contraction (tn_sparse_plan / tn_sparse_contract / tn_sparse_get_info, tn.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <iterator>
#include <new>
#include <unordered_map>
#include <utility>
#include <vector>

#include "../../include/tn.h"
#include "tn_internal.h"

namespace {

template <typename... Args>
tn_status fail(tn_status s, const char *fmt, Args... args) {
    return tn::reportf(s, fmt, args...);
}

#define TN_CUDA(call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(e_ == cudaErrorMemoryAllocation ? TN_ERR_OOM : TN_ERR_CUDA,            \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);  \
    } while (0)

tn_status check_net(const tn_network *n) {
    if (!n || n->magic != tn::kNetMagic)
        return fail(TN_ERR_INVALID_ARG, "not a tn network handle");
    return TN_OK;
}

void fill_pos(int8_t *dst, int n, int value) {
    for (int i = 0; i < n; ++i) dst[i] = (int8_t)value;
}

}  // namespace

// ------------------------------------------------------------------ sparse-state contraction
// Sec. 3.3: the amplitudes of a list of sampled bitstrings.  Every tensor keeps, for the open
// labels it carries, only the configurations of those labels that occur among the samples (its
// merged sparse bond); a step pairs each configuration of its result with the projections onto
// its operands' open labels (gather tables) and contracts the dense labels per configuration.

namespace {

using tn::kSparseMagic;

// a dense subtree gets an ordinary plan when its steps hold at least this many flops
constexpr double kSparseDenseMinFlops = 268435456.0;

uint64_t pext64(uint64_t x, uint64_t mask) {  // bits of x at the set bits of mask, packed
    uint64_t r = 0;
    int k = 0;
    while (mask) {
        const int b = __builtin_ctzll(mask);
        mask &= mask - 1;
        r |= ((x >> b) & 1ull) << k++;
    }
    return r;
}

}  // namespace

struct tn_sparse_plan {
    uint32_t magic = kSparseMagic;
    const tn_network *net = nullptr;
    int device = 0;
    int64_t num_samples = 0;
    struct Ten {
        std::vector<int> open;       // indices into the network's open labels, ascending
        std::vector<int> dense;      // the other labels, most significant first
        std::vector<uint64_t> cfg;   // sampled configurations (bit r = value of open[r]), sorted
        int64_t off = 0;             // complex64 element offset in the arena
    };
    std::vector<Ten> ten;            // leaves, then one result per step
    struct St {
        int a = -1, b = -1, c = -1;
        int64_t ga = 0, gb = 0;      // offsets of the gather tables in `gather`
        int ln = 0;                  // B-only dense labels (the low bits of C's dense index)
        bool gemm = false;           // tiled GEMM per configuration
        bool thin = false;           // at most 16 columns: thread per row (else element-wise)
        bool grouped = false;        // grouped GEMM over configurations sharing an operand entry
        int64_t g_members = 0, g_off = 0, g_len = 0, g_tiles = 0;  // offsets in `gather`
        tn::SparseGroupDesc g{};
        tn::GenericDesc d{};
    };
    std::vector<St> steps;
    // maximal subtrees without open labels, contracted by ordinary dense plans (layout pass,
    // tensor cores in the low-precision modes); their results are converted into the arena
    struct Sub {
        tn_network *net = nullptr;
        tn_plan_t *plan = nullptr;
        int node = -1;               // the sparse tensor the subtree produces
        double2 *out = nullptr;      // its complex128 result
        int64_t n = 0;
    };
    std::vector<Sub> subs;
    std::vector<char> skip;          // per step: computed inside a dense subtree
    std::vector<tn::SparseLeafDesc> convs;
    tn::SparseLeafDesc *conv_dev = nullptr;
    int64_t *zero_off = nullptr;
    tn_precision mode = TN_PREC_C64;
    std::vector<tn::SparseLeafDesc> leaves;
    int max_leaf_rank = 0;
    int root = -1;
    float2 *arena = nullptr;
    int32_t *gather = nullptr;
    int64_t *cfg_off = nullptr;
    int32_t *sample_idx = nullptr;
    tn::SparseLeafDesc *leaves_dev = nullptr;
    double tcc = 0;
    int64_t arena_elems = 0, total_configs = 0, distinct = 0, launches = 0;
};

namespace {

void sparse_free(tn_sparse_plan_t *p) {
    for (auto &sb : p->subs) {
        if (sb.plan) tn_destroy(sb.plan);
        if (sb.net) tn_destroy(sb.net);
        if (sb.out) cudaFree(sb.out);
    }
    if (p->conv_dev) cudaFree(p->conv_dev);
    if (p->zero_off) cudaFree(p->zero_off);
    if (p->arena) cudaFree(p->arena);
    if (p->gather) cudaFree(p->gather);
    if (p->cfg_off) cudaFree(p->cfg_off);
    if (p->sample_idx) cudaFree(p->sample_idx);
    if (p->leaves_dev) cudaFree(p->leaves_dev);
    p->magic = 0;
    delete p;
}

// distinct projections of the sample keys onto the open labels in `mask`, sorted
std::vector<uint64_t> sample_configs(const std::vector<uint64_t> &keys, uint64_t mask) {
    std::vector<uint64_t> v;
    v.reserve(keys.size());
    for (uint64_t k : keys) v.push_back(pext64(k, mask));
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    return v;
}

uint64_t open_mask(const std::vector<int> &open) {
    uint64_t m = 0;
    for (int o : open) m |= 1ull << o;
    return m;
}

int dense_bit(const std::vector<int> &dense, int label) {  // bit position, or -1
    for (size_t q = 0; q < dense.size(); ++q)
        if (dense[q] == label) return (int)(dense.size() - 1 - q);
    return -1;
}

}  // namespace

extern "C" {

static tn_status sparse_plan_impl(const tn_network_t *net, int32_t path_len,
                                  const int32_t *path, int64_t num_samples,
                                  const uint8_t *samples, tn_precision mode,
                                  tn_sparse_plan_t **out);

tn_status tn_sparse_plan(const tn_network_t *net, int32_t path_len, const int32_t *path,
                         int64_t num_samples, const uint8_t *samples, tn_precision mode,
                         tn_sparse_plan_t **out) {
    tn::clear_error();
    try {
        return sparse_plan_impl(net, path_len, path, num_samples, samples, mode, out);
    } catch (const std::bad_alloc &) {
        return fail(TN_ERR_OOM, "tn_sparse_plan: host memory exhausted");
    } catch (...) {
        return fail(TN_ERR_INVALID_ARG, "tn_sparse_plan: internal error");
    }
}

static tn_status sparse_plan_impl(const tn_network_t *net, int32_t path_len,
                                  const int32_t *path, int64_t num_samples,
                                  const uint8_t *samples, tn_precision mode,
                                  tn_sparse_plan_t **out) {
    tn_status cs = check_net(net);
    if (cs != TN_OK) return cs;
    if (!out || num_samples < 1 || !samples || path_len < 0 || (path_len > 0 && !path))
        return fail(TN_ERR_INVALID_ARG, "tn_sparse_plan: invalid argument");
    *out = nullptr;
    const int n = (int)net->labels.size();
    const int nopen = (int)net->open.size();
    if (nopen > 64) return fail(TN_ERR_UNSUPPORTED, "sparse-state: more than 64 open labels");
    if (path_len != n - 1)
        return fail(TN_ERR_PATH, "path has %d pairs, the network needs %d", path_len, n - 1);
    if (num_samples > (int64_t)0x7fffffff)
        return fail(TN_ERR_INVALID_ARG, "too many samples");
    std::unordered_map<int, int> open_index, count;
    for (int j = 0; j < nopen; ++j) open_index[net->open[j]] = j;
    for (const auto &ls : net->labels)
        for (int l : ls) count[l] += 1;
    for (const auto &kv : count)
        if (!open_index.count(kv.first) && kv.second != 2)
            return fail(TN_ERR_UNSUPPORTED, "sparse-state: label %d lies on %d tensors",
                        kv.first, kv.second);
    if ((int)mode < (int)TN_PREC_C64 || (int)mode > (int)TN_PREC_MIXED)
        return fail(TN_ERR_INVALID_ARG, "tn_sparse_plan: unknown precision mode");
    auto *p = new tn_sparse_plan_t;
    p->mode = mode;
    p->net = net;
    p->device = net->device;
    p->num_samples = num_samples;
    // sample keys: bit j = value of open label j
    std::vector<uint64_t> keys((size_t)num_samples);
    for (int64_t i = 0; i < num_samples; ++i) {
        uint64_t k = 0;
        for (int j = 0; j < nopen; ++j) {
            const uint8_t v = samples[i * nopen + j];
            if (v > 1) {
                sparse_free(p);
                return fail(TN_ERR_INVALID_ARG, "sample %lld: bit %d is neither 0 nor 1",
                            (long long)i, j);
            }
            k |= (uint64_t)v << j;
        }
        keys[(size_t)i] = k;
    }
    // leaves
    std::vector<int64_t> cfg_off_host, cfg_first((size_t)n);
    p->ten.resize((size_t)(2 * n - 1));
    for (int t = 0; t < n; ++t) {
        auto &T = p->ten[t];
        const auto &ls = net->labels[t];
        const int R = (int)ls.size();
        std::vector<int> axis_of_open;
        for (int r = 0; r < R; ++r) {
            auto it = open_index.find(ls[r]);
            if (it == open_index.end()) T.dense.push_back(ls[r]);
        }
        for (int j = 0; j < nopen; ++j)
            for (int r = 0; r < R; ++r)
                if (ls[r] == net->open[j]) {
                    T.open.push_back(j);
                    axis_of_open.push_back(r);
                }
        if ((int)T.dense.size() > TN_MAXR - 1) {
            sparse_free(p);
            return fail(TN_ERR_UNSUPPORTED, "sparse-state: leaf rank too large");
        }
        T.cfg = sample_configs(keys, open_mask(T.open));
        tn::SparseLeafDesc d{};
        d.src = net->data + net->offset[t];
        d.nconf = (int64_t)T.cfg.size();
        d.rank_d = (int)T.dense.size();
        fill_pos(d.pos_d, TN_MAXR, -1);
        for (int i = 0; i < d.rank_d; ++i) {
            const int l = T.dense[d.rank_d - 1 - i];
            const int r = (int)(std::find(ls.begin(), ls.end(), l) - ls.begin());
            d.pos_d[i] = (int8_t)(R - 1 - r);
        }
        cfg_first[(size_t)t] = (int64_t)cfg_off_host.size();  // pointer set after the upload
        for (uint64_t c : T.cfg) {
            int64_t o = 0;
            for (size_t q = 0; q < T.open.size(); ++q)
                if ((c >> q) & 1ull) o |= 1ll << (R - 1 - axis_of_open[q]);
            cfg_off_host.push_back(o);
        }
        p->leaves.push_back(d);
        p->max_leaf_rank = std::max(p->max_leaf_rank, d.rank_d);
    }
    // steps: replay the path (the result keeps id a, id b is retired)
    std::vector<int> node(n);
    std::vector<char> alive(n, 1);
    for (int i = 0; i < n; ++i) node[i] = i;
    std::vector<int32_t> gather_host;
    for (int s = 0; s < path_len; ++s) {
        const int a = path[2 * s], b = path[2 * s + 1];
        if (a < 0 || b < 0 || a >= n || b >= n || a == b || !alive[a] || !alive[b]) {
            sparse_free(p);
            return fail(TN_ERR_PATH, "path step %d uses a retired or invalid id", s);
        }
        const int c = n + s;
        const auto &A = p->ten[node[a]];
        const auto &B = p->ten[node[b]];
        auto &C = p->ten[c];
        std::merge(A.open.begin(), A.open.end(), B.open.begin(), B.open.end(),
                   std::back_inserter(C.open));
        std::vector<int> shared;
        for (int l : A.dense)
            if (std::find(B.dense.begin(), B.dense.end(), l) != B.dense.end()) shared.push_back(l);
        for (int l : A.dense)
            if (std::find(shared.begin(), shared.end(), l) == shared.end()) C.dense.push_back(l);
        for (int l : B.dense)
            if (std::find(shared.begin(), shared.end(), l) == shared.end()) C.dense.push_back(l);
        if ((int)C.dense.size() > TN_MAXR - 1 || (int)shared.size() > 62) {
            sparse_free(p);
            return fail(TN_ERR_UNSUPPORTED, "sparse-state: step %d is too large", s);
        }
        C.cfg = sample_configs(keys, open_mask(C.open));
        // projections of C's configurations onto A's and B's open labels
        uint64_t ma = 0, mb = 0;
        for (size_t r = 0; r < C.open.size(); ++r) {
            if (std::binary_search(A.open.begin(), A.open.end(), C.open[r])) ma |= 1ull << r;
            else mb |= 1ull << r;
        }
        tn_sparse_plan_t::St st;
        st.a = node[a];
        st.b = node[b];
        st.c = c;
        st.ga = (int64_t)gather_host.size();
        for (uint64_t k : C.cfg)
            gather_host.push_back((int32_t)(std::lower_bound(A.cfg.begin(), A.cfg.end(),
                                                             pext64(k, ma)) - A.cfg.begin()));
        st.gb = (int64_t)gather_host.size();
        for (uint64_t k : C.cfg)
            gather_host.push_back((int32_t)(std::lower_bound(B.cfg.begin(), B.cfg.end(),
                                                             pext64(k, mb)) - B.cfg.begin()));
        tn::GenericDesc &d = st.d;
        d.rank_c = (int)C.dense.size();
        d.nk = (int)shared.size();
        fill_pos(d.posA_c, TN_MAXR, -1);
        fill_pos(d.posB_c, TN_MAXR, -1);
        fill_pos(d.posA_k, TN_MAXR, -1);
        fill_pos(d.posB_k, TN_MAXR, -1);
        for (int i = 0; i < d.rank_c; ++i) {
            const int l = C.dense[d.rank_c - 1 - i];
            d.posA_c[i] = (int8_t)dense_bit(A.dense, l);
            d.posB_c[i] = (int8_t)dense_bit(B.dense, l);
        }
        for (int j = 0; j < d.nk; ++j) {
            const int l = shared[d.nk - 1 - j];
            d.posA_k[j] = (int8_t)dense_bit(A.dense, l);
            d.posB_k[j] = (int8_t)dense_bit(B.dense, l);
        }
        {
            int nb = 0;
            for (int l : B.dense)
                if (std::find(shared.begin(), shared.end(), l) == shared.end()) ++nb;
            st.ln = nb;
            st.gemm = d.rank_c - nb >= 3 && nb >= 3 && d.nk >= 3;
            st.thin = !st.gemm && nb <= 4 && d.rank_c - nb >= 5 && d.nk >= 2;
        }
        if (d.nk >= 3) {
            // group the result configurations by the operand entry they share (the operand with
            // fewer distinct entries): one GEMM per group over the stacked other operand
            const int64_t nc = (int64_t)C.cfg.size();
            const int32_t *ga = gather_host.data() + st.ga, *gb = gather_host.data() + st.gb;
            std::vector<int32_t> ka(ga, ga + nc), kb(gb, gb + nc);
            std::sort(ka.begin(), ka.end());
            std::sort(kb.begin(), kb.end());
            const int64_t na = std::unique(ka.begin(), ka.end()) - ka.begin();
            const int64_t nbk = std::unique(kb.begin(), kb.end()) - kb.begin();
            const bool by_a = na <= nbk;
            const int32_t *key = by_a ? ga : gb;
            std::vector<int32_t> order((size_t)nc);
            for (int64_t i = 0; i < nc; ++i) order[(size_t)i] = (int32_t)i;
            std::stable_sort(order.begin(), order.end(),
                             [&](int32_t x, int32_t y) { return key[x] < key[y]; });
            const int lmv = d.rank_c - st.ln;
            const int64_t M = 1ll << lmv, N = 1ll << st.ln;
            std::vector<int32_t> goff, glen, tiles;
            double useful = 0, padded = 0;
            for (int64_t i = 0; i < nc;) {
                int64_t j = i;
                while (j < nc && key[order[(size_t)j]] == key[order[(size_t)i]]) ++j;
                const int64_t len = j - i;
                const int64_t rows = by_a ? M : len * M, cols = by_a ? len * N : N;
                const int64_t tr = (rows + 63) / 64, tc = (cols + 63) / 64;
                const int gi = (int)goff.size();
                goff.push_back((int32_t)i);
                glen.push_back((int32_t)len);
                for (int64_t a2 = 0; a2 < tr; ++a2)
                    for (int64_t b2 = 0; b2 < tc; ++b2) {
                        tiles.push_back(gi);
                        tiles.push_back((int32_t)a2);
                        tiles.push_back((int32_t)b2);
                    }
                useful += (double)rows * (double)cols;
                padded += (double)(tr * tc) * 4096.0;
                i = j;
            }
            if (useful >= 0.25 * padded && (int64_t)tiles.size() / 3 < 0x7fffffffll) {
                st.grouped = true;
                st.g.by_a = by_a ? 1 : 0;
                st.g.ntiles = (int64_t)tiles.size() / 3;
                st.g_members = (int64_t)gather_host.size();
                gather_host.insert(gather_host.end(), order.begin(), order.end());
                st.g_off = (int64_t)gather_host.size();
                gather_host.insert(gather_host.end(), goff.begin(), goff.end());
                st.g_len = (int64_t)gather_host.size();
                gather_host.insert(gather_host.end(), glen.begin(), glen.end());
                st.g_tiles = (int64_t)gather_host.size();
                gather_host.insert(gather_host.end(), tiles.begin(), tiles.end());
            }
        }
        p->tcc += 8.0 * (double)C.cfg.size() * std::ldexp(1.0, d.rank_c + d.nk);
        p->steps.push_back(st);
        node[a] = c;
        alive[b] = 0;
    }
    p->root = n == 1 ? 0 : node[path[2 * (path_len - 1)]];
    {
        const auto &R = p->ten[p->root];
        bool all = (int)R.open.size() == nopen;
        for (int j = 0; all && j < nopen; ++j) all = R.open[j] == j;
        if (!R.dense.empty() || !all) {
            sparse_free(p);
            return fail(TN_ERR_PATH, "the path does not reduce to the open labels");
        }
        p->distinct = (int64_t)R.cfg.size();
    }
    // maximal dense subtrees (no open label below them) worth an ordinary plan
    p->skip.assign(p->steps.size(), 0);
    std::vector<int> step_of((size_t)(2 * n - 1), -1), parent((size_t)(2 * n - 1), -1);
    for (size_t k = 0; k < p->steps.size(); ++k) {
        step_of[(size_t)p->steps[k].c] = (int)k;
        parent[(size_t)p->steps[k].a] = p->steps[k].c;
        parent[(size_t)p->steps[k].b] = p->steps[k].c;
    }
    std::vector<std::pair<int, std::vector<int>>> dense_roots;  // root node, its steps
    for (size_t k = 0; k < p->steps.size(); ++k) {
        const int c = p->steps[k].c;
        const int par = parent[(size_t)c];
        if (!p->ten[c].open.empty() || (par >= 0 && p->ten[par].open.empty())) continue;
        // c is the root of a maximal dense subtree: gather its steps (path order) and work
        std::vector<int> sub_steps, stack{c};
        double work = 0;
        while (!stack.empty()) {
            const int v = stack.back();
            stack.pop_back();
            const int sk = step_of[(size_t)v];
            if (sk < 0) continue;
            sub_steps.push_back(sk);
            work += 8.0 * std::ldexp(1.0, p->steps[sk].d.rank_c + p->steps[sk].d.nk);
            stack.push_back(p->steps[sk].a);
            stack.push_back(p->steps[sk].b);
        }
        if (work < kSparseDenseMinFlops || p->ten[c].dense.size() > 30) continue;
        std::sort(sub_steps.begin(), sub_steps.end());
        dense_roots.emplace_back(c, sub_steps);
    }
    for (auto &dr : dense_roots) {
        const int c = dr.first;
        const std::vector<int> &sub_steps = dr.second;
        // local ids of the subtree's leaves (original tensor ids), in increasing order
        std::vector<int> lv;
        for (int sk : sub_steps)
            for (int side = 0; side < 2; ++side) {
                const int id = path[2 * sk + side];
                if (std::find(lv.begin(), lv.end(), id) == lv.end()) lv.push_back(id);
            }
        std::sort(lv.begin(), lv.end());
        std::vector<int32_t> lpath;
        for (int sk : sub_steps)
            for (int side = 0; side < 2; ++side)
                lpath.push_back((int32_t)(std::lower_bound(lv.begin(), lv.end(),
                                                           path[2 * sk + side]) - lv.begin()));
        tn_sparse_plan_t::Sub sb;
        sb.node = c;
        sb.net = new tn_network();
        sb.net->device = net->device;
        for (int id : lv) {
            sb.net->labels.push_back(net->labels[id]);
            sb.net->offset.push_back(sb.net->total);
            sb.net->total += (int64_t)1 << net->labels[id].size();
        }
        sb.net->open = p->ten[c].dense;
        cudaError_t e = cudaMalloc(&sb.net->data, sizeof(double2) * (size_t)sb.net->total);
        for (size_t q = 0; e == cudaSuccess && q < lv.size(); ++q)
            e = cudaMemcpy(sb.net->data + sb.net->offset[q], net->data + net->offset[lv[q]],
                           sizeof(double2) * ((size_t)1 << net->labels[lv[q]].size()),
                           cudaMemcpyDeviceToDevice);
        sb.n = (int64_t)1 << p->ten[c].dense.size();
        if (e == cudaSuccess) e = cudaMalloc(&sb.out, sizeof(double2) * (size_t)sb.n);
        p->subs.push_back(sb);  // owned by the plan from here on
        if (e != cudaSuccess) {
            sparse_free(p);
            return fail(e == cudaErrorMemoryAllocation ? TN_ERR_OOM : TN_ERR_CUDA,
                        "sparse-state dense subtree: %s", cudaGetErrorString(e));
        }
        tn_status ps = tn_plan(sb.net, (int32_t)sub_steps.size(), lpath.data(), 0, nullptr, mode,
                               nullptr, &p->subs.back().plan);
        if (ps != TN_OK) {
            sparse_free(p);
            return ps;
        }
        for (int sk : sub_steps) p->skip[(size_t)sk] = 1;
    }
    // arena: every tensor its own range (configurations x dense elements)
    int64_t off = 0;
    for (auto &T : p->ten) {
        T.off = off;
        const int64_t elems = (int64_t)T.cfg.size() << T.dense.size();
        off += (elems + 31) / 32 * 32;
        p->total_configs += (int64_t)T.cfg.size();
    }
    p->arena_elems = off;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != p->device) cudaSetDevice(p->device);
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e == cudaSuccess && (double)off * 8.0 > 0.6 * (double)free_b) {
        if (dev != p->device) cudaSetDevice(dev);
        sparse_free(p);
        return fail(TN_ERR_OOM, "sparse-state arena needs %lld bytes", (long long)(off * 8));
    }
    std::vector<int32_t> idx((size_t)num_samples);
    {
        const auto &R = p->ten[p->root];
        for (int64_t i = 0; i < num_samples; ++i)
            idx[(size_t)i] = (int32_t)(std::lower_bound(R.cfg.begin(), R.cfg.end(), keys[(size_t)i]) -
                                       R.cfg.begin());
    }
    auto upload = [&](void **dst, const void *src, size_t bytes) -> cudaError_t {
        cudaError_t r = cudaMalloc(dst, bytes ? bytes : 8);
        if (r != cudaSuccess || !bytes) return r;
        return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    };
    e = cudaMalloc(&p->arena, (size_t)std::max<int64_t>(off, 1) * sizeof(float2));
    if (e == cudaSuccess)
        e = upload(reinterpret_cast<void **>(&p->gather), gather_host.data(),
                   gather_host.size() * sizeof(int32_t));
    if (e == cudaSuccess)
        e = upload(reinterpret_cast<void **>(&p->cfg_off), cfg_off_host.data(),
                   cfg_off_host.size() * sizeof(int64_t));
    if (e == cudaSuccess)
        e = upload(reinterpret_cast<void **>(&p->sample_idx), idx.data(),
                   idx.size() * sizeof(int32_t));
    if (e == cudaSuccess && !p->subs.empty()) {
        const int64_t zero = 0;
        e = upload(reinterpret_cast<void **>(&p->zero_off), &zero, sizeof(int64_t));
        for (auto &sb : p->subs) {
            tn::SparseLeafDesc cd{};
            cd.src = sb.out;
            cd.dst = p->arena + p->ten[sb.node].off;
            cd.cfg_off = p->zero_off;
            cd.nconf = 1;
            cd.rank_d = (int)p->ten[sb.node].dense.size();
            fill_pos(cd.pos_d, TN_MAXR, -1);
            for (int i = 0; i < cd.rank_d; ++i) cd.pos_d[i] = (int8_t)i;
            p->convs.push_back(cd);
        }
        if (e == cudaSuccess)
            e = upload(reinterpret_cast<void **>(&p->conv_dev), p->convs.data(),
                       p->convs.size() * sizeof(tn::SparseLeafDesc));
    }
    if (e == cudaSuccess) {
        for (int t = 0; t < n; ++t) {
            auto &d = p->leaves[t];
            d.cfg_off = p->cfg_off + cfg_first[(size_t)t];
            d.dst = p->arena + p->ten[t].off;
        }
        e = upload(reinterpret_cast<void **>(&p->leaves_dev), p->leaves.data(),
                   p->leaves.size() * sizeof(tn::SparseLeafDesc));
    }
    if (dev != p->device) cudaSetDevice(dev);
    if (e != cudaSuccess) {
        sparse_free(p);
        return fail(e == cudaErrorMemoryAllocation ? TN_ERR_OOM : TN_ERR_CUDA,
                    "sparse-state plan: %s", cudaGetErrorString(e));
    }
    for (auto &st : p->steps) {
        if (st.grouped) {
            st.g.gA = p->gather + st.ga;
            st.g.gB = p->gather + st.gb;
            st.g.members = p->gather + st.g_members;
            st.g.grp_off = p->gather + st.g_off;
            st.g.grp_len = p->gather + st.g_len;
            st.g.tiles = p->gather + st.g_tiles;
        }
        st.d.A = p->arena + p->ten[st.a].off;
        st.d.B = p->arena + p->ten[st.b].off;
        st.d.C = p->arena + p->ten[st.c].off;
        st.d.sA = (int64_t)1 << p->ten[st.a].dense.size();
        st.d.sB = (int64_t)1 << p->ten[st.b].dense.size();
        st.d.sC = (int64_t)1 << p->ten[st.c].dense.size();
    }
    *out = p;
    return TN_OK;
}

tn_status tn_sparse_contract(tn_sparse_plan_t *p, void *amps_dev, void *stream_) {
    tn::clear_error();
    if (!p || p->magic != kSparseMagic)
        return fail(TN_ERR_INVALID_ARG, "not a sparse-state plan handle");
    if (!amps_dev) return fail(TN_ERR_INVALID_ARG, "amps_dev is NULL");
    cudaStream_t stream = (cudaStream_t)stream_;
    int dev = 0;
    TN_CUDA(cudaGetDevice(&dev));
    if (dev != p->device) TN_CUDA(cudaSetDevice(p->device));
    // dense subtrees first: ordinary plans into their complex128 buffers, then into the arena
    int max_conv = 0;
    for (auto &sb : p->subs) {
        TN_CUDA(cudaMemsetAsync(sb.out, 0, sizeof(double2) * (size_t)sb.n, stream));
        tn_plan_info pi{};
        tn_status ps = tn_plan_get_info(sb.plan, &pi);
        if (ps == TN_OK) ps = tn_contract(sb.plan, 0, pi.num_slices, sb.out, stream);
        if (ps != TN_OK) return ps;
        max_conv = std::max(max_conv, (int)(63 - __builtin_clzll((uint64_t)sb.n)));
    }
    if (!p->subs.empty()) {
        TN_CUDA(tn::launch_sparse_leaves(p->conv_dev, (int32_t)p->convs.size(), max_conv, stream));
        p->launches += 1;
    }
    TN_CUDA(tn::launch_sparse_leaves(p->leaves_dev, (int32_t)p->leaves.size(), p->max_leaf_rank,
                                     stream));
    p->launches += 1;
    for (size_t k = 0; k < p->steps.size(); ++k) {
        const auto &st = p->steps[k];
        if (p->skip[k]) continue;
        const int64_t nconf = (int64_t)p->ten[st.c].cfg.size();
        if (st.grouped)
            TN_CUDA(tn::launch_sparse_group(st.d, st.ln, st.g, stream));
        else if (st.gemm)
            TN_CUDA(tn::launch_sparse_gemm(st.d, st.ln, p->gather + st.ga, p->gather + st.gb,
                                           nconf, stream));
        else if (st.thin)
            TN_CUDA(tn::launch_sparse_thin(st.d, st.ln, p->gather + st.ga, p->gather + st.gb,
                                           nconf, stream));
        else
            TN_CUDA(tn::launch_sparse_step(st.d, p->gather + st.ga, p->gather + st.gb, nconf,
                                           stream));
        p->launches += 1;
    }
    TN_CUDA(tn::launch_sparse_amps(p->arena + p->ten[p->root].off, p->sample_idx,
                                   p->num_samples, reinterpret_cast<double2 *>(amps_dev), stream));
    p->launches += 1;
    if (dev != p->device) cudaSetDevice(dev);
    return TN_OK;
}

tn_status tn_sparse_get_info(const tn_sparse_plan_t *p, tn_sparse_info *out) {
    tn::clear_error();
    if (!p || p->magic != kSparseMagic || !out)
        return fail(TN_ERR_INVALID_ARG, "not a sparse-state plan handle");
    *out = tn_sparse_info{};
    out->num_steps = (int64_t)p->steps.size();
    out->num_samples = p->num_samples;
    out->distinct_samples = p->distinct;
    out->total_configs = p->total_configs;
    out->arena_bytes = p->arena_elems * (int64_t)sizeof(float2);
    out->tcc = p->tcc;
    out->kernel_launches = p->launches;
    int mx = 0;
    for (const auto &T : p->ten) mx = std::max(mx, (int)T.dense.size());
    out->max_log2_dense = mx;
    out->dense_subtrees = (int64_t)p->subs.size();
    for (size_t k = 0; k < p->skip.size(); ++k) out->dense_subtree_steps += p->skip[k] ? 1 : 0;
    for (const auto &st : p->steps) {
        out->gemm_steps += !st.grouped && st.gemm ? 1 : 0;
        out->thin_steps += !st.grouped && !st.gemm && st.thin ? 1 : 0;
        out->grouped_steps += st.grouped ? 1 : 0;
    }
    return TN_OK;
}

}  // extern "C"

void tn::sparse_destroy(void *handle) { sparse_free(reinterpret_cast<tn_sparse_plan_t *>(handle)); }
