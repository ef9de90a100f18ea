// Host runtime and C ABI of the contraction engine (declared in include/tn.h).
//
// tn_plan() turns (network, path, sliced bonds, precision) into a list of device operations:
//   1. replay of the path (Sec. 3.1: pairs (a, b), the result keeps id a) with the sliced labels
//      removed (Sec. 3.2), giving for every step its contracted (K), free (M, N) and batch
//      labels (Sec. 2.4, Eq. chap2_einsum) and its T_cc / T_mc (Eq. T_cc, Eq. T_mc);
//   2. routing of every step to a kernel (tensor-core GEMM, CUDA-core GEMM, element-wise) by
//      its GEMM extents, following the balanced-index thresholds of App. A.2;
//   3. a layout pass from the root back to the leaves (Sec. 4.1, index reordering): each operand
//      of a step is stored as [its free labels in the order of the step's result][the contracted
//      labels], so every step reads its operands as GEMM matrices and every producer writes
//      directly in its consumer's order; no separate transpose pass exists;
//   4. slice-independent steps are hoisted into a prologue that runs once per tn_contract call;
//   5. a liveness-based first-fit placement of every tensor in one device workspace, with as
//      many slices per launch as the workspace allows.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/tn.h"
#include "tn_internal.h"

namespace {

using tn::kNetMagic;
constexpr uint32_t kPlanMagic = 0x544e504cu;  // "TNPL"
constexpr int kMaxLabel = 1 << 20;
constexpr int kMaxRank = 62;

thread_local std::string g_err;

tn_status fail(tn_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define TN_CUDA(call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(e_ == cudaErrorMemoryAllocation ? TN_ERR_OOM : TN_ERR_CUDA,            \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);  \
    } while (0)

}  // namespace

tn_status tn::report(tn_status s, const char *msg) { return fail(s, "%s", msg); }

void tn::clear_error() { g_err.clear(); }

tn_status tn::reportf(tn_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return fail(s, "%s", buf);
}


namespace {

enum Kernel { K_GENERIC = 0, K_STREAM = 1, K_GEMM = 2, K_TC = 3 };

// Complex form of a tensor-core step: TN_GEMM_4M, TN_GEMM_3M, or 4M with compensated hi/lo
// operand planes (Sec. 4.2: x = hi + lo, xy ~ hi hi + hi lo + lo hi).
constexpr int kFormSplit = 3;

bool bf16_mode(tn_precision m) {
    return m == TN_PREC_BF16_SCALED || m == TN_PREC_SPLIT_BF16;
}

bool tf32_mode(tn_precision m) { return m == TN_PREC_TF32 || m == TN_PREC_SPLIT_TF32; }

// Stored type of the tensor-core operands: 0 FP16, 1 BF16, 2 FP32 rounded to TF32.
int operand_dtype(tn_precision m) { return tf32_mode(m) ? 2 : (bf16_mode(m) ? 1 : 0); }

// Modes whose dense steps run single-pass unless the precision policy demotes some of them.
bool single_pass_mode(tn_precision m) {
    return m == TN_PREC_FP16_SCALED || m == TN_PREC_BF16_SCALED || m == TN_PREC_TF32;
}

// Error model of the precision policy (Sec. 4.3; stated in full in tn.h).  A single-pass step
// rounds both operands to nearest in a type of unit roundoff u; for significands uniform in
// [1, 2) the relative Frobenius error of that rounding is u / sqrt(7) per operand, so a step
// adds about sqrt(2/7) u to the relative error of its result, which carries to the amplitudes
// with a gain near 1 (the rest of the network is a product of unitaries and projections).
// Steps round independently, so their errors add in quadrature.
constexpr double kErrSafety = 1.5;       // over the ~1.15 measured on circuits
constexpr double kErrSplitStep = 4e-6;   // compensated step with accumulator promotion
constexpr double kErrFloor = 1e-5;       // complex64 leaves and FP32 steps
constexpr double kBf16DefaultBudget = 5e-3;

double unit_roundoff(tn_precision m) {
    return bf16_mode(m) ? std::ldexp(1.0, -8) : std::ldexp(1.0, -11);  // FP16, TF32: 2^-11
}

double predicted_eps(tn_precision m, int single, int split) {
    if (m == TN_PREC_C64) return kErrFloor;
    const double cu = kErrSafety * std::sqrt(2.0 / 7.0) * unit_roundoff(m);
    return std::sqrt(single * cu * cu + split * kErrSplitStep * kErrSplitStep +
                     kErrFloor * kErrFloor);
}

struct Tensor {
    std::vector<int> order;  // memory order of the labels, most significant first
    bool dep = false;        // depends on the slice id
    int producer = -1;       // step index, or -1 for a leaf
    int leaf = -1;           // network tensor index for a leaf
    int64_t off = -1;        // complex64 element offset in the arena
    int t0 = 0, t1 = 0;      // lifetime on the op timeline
    int meta = -1;           // block of per-slice (max-abs, exponent) if some step needs them
    bool direct = false;     // produced directly as a planar 16-bit copy (no complex64 storage)
    int rank() const { return (int)order.size(); }
    int pos(int label) const {  // bit position of a label in this tensor's memory index
        for (int i = 0; i < rank(); ++i)
            if (order[i] == label) return rank() - 1 - i;
        return -1;
    }
};

struct Planar {              // planar 16-bit copy of a tensor feeding a tensor-core step
    int tensor = -1;
    int planes = 2;          // planes written: re, im (4M) or re, im, re + im (3M)
    int cap_planes = 2;      // planes allocated (3 while the autotuner may still pick 3M)
    bool direct = false;     // written by its producer's epilogue (no conversion pass)
    int64_t off = -1;        // byte offset in the arena
    int64_t bytes_per_slice = 0;
    int t = 0;               // time of the consuming step
    int meta = -1;           // index of its (amax, exps) block
    int t0 = 0;              // first op that writes it
};

struct Step {
    int a = -1, b = -1, c = -1;  // tensor indices
    std::vector<int> la, lb, lc; // replayed label lists (before layout)
    std::vector<int> K, M, N, batch;
    int kernel = K_GENERIC;
    bool dep = false;
    double tcc = 0, tmc = 0;
    int t = 0;                   // op time
    int pa = -1, pb = -1;        // planar copies for K_TC
    int form = TN_GEMM_4M;
    int splits = 1;              // K_GEMM split-K factor
    bool tune_form = false;      // autotune: 3M is still a candidate for this K_TC step
    bool thin_tc = false;        // K_STREAM on the tensor cores (k_gemm_thin_tc)
    // K_STREAM on the tensor cores: the output stage's swizzle (thin_choose_swizzle), chosen at
    // the first launch
    mutable int8_t thin_phi[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    mutable bool thin_phi_set = false;
    mutable bool thin_tc_off = false;  // its result order does not fit the 128-row tile
    int variant = -1;            // K_TC kernel variant
    int out_meta = -1;           // meta block whose per-slice max-abs this step's epilogue records
    int direct_planar = -1;      // planar copy this step writes directly instead of complex64
    int64_t part_off = -1;       // K_GEMM split-K partials (byte offset in the arena)
    int chain = -1;              // run of small element-wise steps launched together (k_generic_chain)
    bool chain_head = false;     // first step of its run: launches the whole run
    // profile mode: recorded (start, stop) event pairs not yet read, and the running totals
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending, pending_prep;
    double time_ms = 0, prep_ms = 0;
    int64_t timed = 0;
};

struct Op {
    int kind;   // 0 bind invariant, 1 step, 2 bind sliced, 3 convert, 4 accumulate
    int index;  // step or planar index
};

}  // namespace

struct tn_plan {
    uint32_t magic = kPlanMagic;
    const tn_network *net = nullptr;
    int device = 0;
    tn_precision mode = TN_PREC_C64;
    tn_plan_options opts{};
    std::vector<int> sliced;
    std::vector<int> root_open;  // the open labels the root keeps (open minus sliced), in order
    tn::AccMap acc;              // where root elements and slices go in amps
    std::vector<Tensor> tensors;
    std::vector<Step> steps;
    std::vector<Planar> planars;
    int root = -1;
    int64_t num_slices = 1;
    int64_t sb = 1;              // slices per launch
    int64_t arena_elems = 0;     // complex64 elements
    int64_t arena_bytes = 0;
    char *arena = nullptr;
    bool own_arena = false;
    std::vector<tn::BindItem> bind_inv, bind_sl;
    std::vector<tn::BindTiled> tiled_inv, tiled_sl;  // leaves bound by the tiled permutation
    tn::BindItem *bind_inv_dev = nullptr, *bind_sl_dev = nullptr;
    std::vector<std::vector<int>> chains;  // step indices of each run of chained steps
    std::vector<int64_t> chain_first;      // first descriptor of each run in chain_dev
    tn::GenericDesc *chain_dev = nullptr;
    int max_rank_inv = 0, max_rank_sl = 0;
    unsigned int *meta = nullptr;  // per meta block: amax[sb] then exps[sb]
    int nmeta = 0;
    double *partial = nullptr;     // readout partials
    double2 *amps_tmp = nullptr;   // tn_contract_host accumulator
    int n_partial = 64;
    int max_log = 0;
    bool tc_ok = false;
    int single_pass = 0, compensated = 0;  // precision policy: dense steps of each kind
    double eps_pred = 0;                   // the error model's amplitude error of the plan
    std::vector<tn::TcGemmDesc> tc_desc;  // per step (only K_TC entries used)
    int64_t launches = 0;                 // kernels launched by this plan
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> event_pool;
    bool tuned = false;                   // autotune done (first full batch)
    // CUDA graph of the slice-dependent steps of one full batch (use_graph)
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int64_t graph_launches = 0;           // kernels inside one replay
    // profile mode: leaf-binding launches bracketed by events, and their running total
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending_bind;
    double bind_ms = 0;
    int64_t bind_timed = 0;
};

namespace {

int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

tn_status check_net(const tn_network *n) {
    if (!n || n->magic != kNetMagic) return fail(TN_ERR_INVALID_ARG, "not a tn network handle");
    return TN_OK;
}

tn_status check_plan(const tn_plan_t *p) {
    if (!p || p->magic != kPlanMagic) return fail(TN_ERR_INVALID_ARG, "not a tn plan handle");
    return TN_OK;
}

// Pick the kernel of a step from its GEMM extents (log2).  Dense steps go to the tensor cores
// when the mode asks for them; the thresholds follow App. A.2 (k >= 64, m, n >= 32 keep the
// tensor cores busy) rounded up to the tcgen05 tile (M 128, N 128, K 64).
int route(const Step &s, tn_precision mode, bool tc_ok) {
    const int lm = (int)s.M.size(), ln = (int)s.N.size(), lk = (int)s.K.size();
    const bool tc_mode = mode != TN_PREC_C64;
    if (s.batch.empty() && tc_mode && tc_ok && lm >= 7 && ln >= 7 && lk >= 6) return K_TC;
    // large outputs of short contractions (8 <= k < 64) also go to the tensor cores: the short-K
    // variant's tensor map zero-fills the K tile past k, and its epilogue writes 2 CTAs per SM
    if (s.batch.empty() && tc_mode && tc_ok && lm >= 7 && ln >= 7 && lk >= 3 && lm + ln >= 20)
        return K_TC;
    // a narrow side of 32 or 64 (App. A.2's m, n >= 32 threshold): the 32- or 64-column tile,
    // the wide side as M, when that side has at least 2^12 rows to spread over the SMs
    if (s.batch.empty() && tc_mode && tc_ok && (std::min(lm, ln) == 5 || std::min(lm, ln) == 6) &&
        std::max(lm, ln) >= 12 && lk >= 3)
        return K_TC;
    // thin steps: a contraction (k <= 1024) of a large operand with a small one (at most 16
    // free elements), streamed on the CUDA cores at memory speed
    if (s.batch.empty() && lk >= 1 && lk <= 10 && std::min(lm, ln) <= 4 && std::max(lm, ln) >= 10)
        return K_STREAM;
    // register-tiled GEMM (split along K when the output is small); a contraction of fewer than
    // 16 elements is cheaper as an element-wise pass with coalesced stores
    if (s.batch.empty() && lk >= 2 && lm >= 3 && ln >= 3 && lm + ln + lk >= 14) return K_GEMM;
    // a long contraction (k >= 1024) into a small result: the CUDA-core GEMM splits K over many
    // CTAs where the element-wise kernel would give each output one serial sum
    if (s.batch.empty() && lk >= 10 && lm + ln >= 1) return K_GEMM;
    return K_GENERIC;
}

void fill_pos(int8_t *dst, int n, int value) {
    for (int i = 0; i < n; ++i) dst[i] = (int8_t)value;
}

}  // namespace

extern "C" {

const char *tn_status_string(tn_status s) {
    switch (s) {
        case TN_OK: return "ok";
        case TN_ERR_INVALID_ARG: return "invalid argument";
        case TN_ERR_SHAPE: return "inconsistent shape or labels";
        case TN_ERR_PATH: return "invalid contraction path";
        case TN_ERR_OOM: return "out of device memory";
        case TN_ERR_CUDA: return "CUDA error";
        case TN_ERR_TIMEOUT: return "device wait timed out";
        case TN_ERR_UNSUPPORTED: return "unsupported input";
        case TN_ERR_NUMERIC: return "scaled storage overflow";
    }
    return "unknown status";
}

tn_status tn_last_error_detail(char *buf, size_t len) {
    if (!buf || len == 0) return TN_ERR_INVALID_ARG;
    size_t n = std::min(len - 1, g_err.size());
    memcpy(buf, g_err.data(), n);
    buf[n] = 0;
    return TN_OK;
}

tn_status tn_network_load(int32_t num_tensors, const int32_t *ranks,
                          const int32_t *const *labels, const int64_t *const *dims,
                          const double *const *data, int32_t num_open,
                          const int32_t *open_labels, tn_network_t **out) {
    g_err.clear();
    if (!out) return fail(TN_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (num_tensors < 1 || !ranks || !labels || !dims || !data)
        return fail(TN_ERR_INVALID_ARG, "need at least one tensor and non-NULL arrays");
    if (num_open < 0 || (num_open > 0 && !open_labels))
        return fail(TN_ERR_INVALID_ARG, "bad open labels");
    if (num_open > 40) return fail(TN_ERR_UNSUPPORTED, "at most 40 open labels");
    std::map<int, int> count;
    auto *net = new tn_network();
    for (int i = 0; i < num_tensors; ++i) {
        if (ranks[i] < 0 || ranks[i] > kMaxRank) {
            delete net;
            return fail(TN_ERR_INVALID_ARG, "tensor %d: rank %d out of range", i, ranks[i]);
        }
        if (ranks[i] > 0 && (!labels[i] || !dims[i])) {
            delete net;
            return fail(TN_ERR_INVALID_ARG, "tensor %d: NULL labels or dims", i);
        }
        if (!data[i]) {
            delete net;
            return fail(TN_ERR_INVALID_ARG, "tensor %d: NULL data", i);
        }
        std::vector<int> ls;
        for (int r = 0; r < ranks[i]; ++r) {
            int l = labels[i][r];
            if (l < 0 || l >= kMaxLabel) {
                delete net;
                return fail(TN_ERR_INVALID_ARG, "tensor %d: label %d out of range", i, l);
            }
            if (dims[i][r] != 2) {
                delete net;
                return fail(TN_ERR_UNSUPPORTED, "tensor %d: dim %lld (only 2 is supported)", i,
                            (long long)dims[i][r]);
            }
            if (std::find(ls.begin(), ls.end(), l) != ls.end()) {
                delete net;
                return fail(TN_ERR_SHAPE, "tensor %d: label %d repeated", i, l);
            }
            ls.push_back(l);
            count[l]++;
        }
        net->labels.push_back(ls);
        net->offset.push_back(net->total);
        net->total += (int64_t)1 << ranks[i];
    }
    for (int j = 0; j < num_open; ++j) {
        int l = open_labels[j];
        if (count.find(l) == count.end()) {
            delete net;
            return fail(TN_ERR_SHAPE, "open label %d is on no tensor", l);
        }
        if (std::find(net->open.begin(), net->open.end(), l) != net->open.end()) {
            delete net;
            return fail(TN_ERR_SHAPE, "open label %d repeated", l);
        }
        net->open.push_back(l);
        count[l]++;
    }
    for (auto &kv : count)
        if (kv.second < 2) {
            delete net;
            return fail(TN_ERR_SHAPE, "label %d is on one tensor only and not open", kv.first);
        }
    if (cudaGetDevice(&net->device) != cudaSuccess) {
        delete net;
        return fail(TN_ERR_CUDA, "no CUDA device");
    }
    cudaError_t e = cudaMalloc(&net->data, sizeof(double2) * (size_t)net->total);
    if (e != cudaSuccess) {
        delete net;
        return fail(e == cudaErrorMemoryAllocation ? TN_ERR_OOM : TN_ERR_CUDA,
                    "cudaMalloc network: %s", cudaGetErrorString(e));
    }
    *out = net;
    tn_status s = tn_network_set_data(net, data);
    if (s != TN_OK) {
        tn_destroy(net);
        *out = nullptr;
    }
    return s;
}

tn_status tn_network_set_data(tn_network_t *net, const double *const *data) {
    g_err.clear();
    if (check_net(net) != TN_OK) return TN_ERR_INVALID_ARG;
    if (!data) return fail(TN_ERR_INVALID_ARG, "data is NULL");
    std::vector<double2> host((size_t)net->total);
    for (size_t i = 0; i < net->labels.size(); ++i) {
        if (!data[i]) return fail(TN_ERR_INVALID_ARG, "tensor %d: NULL data", (int)i);
        memcpy(&host[(size_t)net->offset[i]], data[i],
               sizeof(double2) * ((size_t)1 << net->labels[i].size()));
    }
    TN_CUDA(cudaMemcpy(net->data, host.data(), sizeof(double2) * host.size(),
                       cudaMemcpyHostToDevice));
    return TN_OK;
}

}  // extern "C"

namespace {

// First-fit placement of intervals [t0, t1] with sizes, returns the peak (in units).
int64_t place(std::vector<std::pair<int64_t, std::pair<int, int>>> items,
              std::vector<int64_t> &offsets) {
    // items: (size, (t0, t1)); offsets out in input order
    struct Live { int64_t off, size; int t0, t1; };
    std::vector<Live> placed;
    std::vector<int> order(items.size());
    for (size_t i = 0; i < items.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        if (items[x].second.first != items[y].second.first)
            return items[x].second.first < items[y].second.first;
        return items[x].first > items[y].first;
    });
    offsets.assign(items.size(), 0);
    int64_t peak = 0;
    for (int idx : order) {
        const int64_t sz = items[idx].first;
        const int t0 = items[idx].second.first, t1 = items[idx].second.second;
        std::vector<std::pair<int64_t, int64_t>> busy;
        for (auto &p : placed)
            if (!(p.t1 < t0 || p.t0 > t1)) busy.push_back({p.off, p.off + p.size});
        std::sort(busy.begin(), busy.end());
        int64_t cand = 0;
        for (auto &bz : busy) {
            if (cand + sz <= bz.first) break;
            cand = std::max(cand, bz.second);
        }
        offsets[idx] = cand;
        placed.push_back({cand, sz, t0, t1});
        peak = std::max(peak, cand + sz);
    }
    return peak;
}

// Layout, allocation and descriptors for a given number of slices per launch.
int64_t layout_bytes(tn_plan_t *p, int64_t sb, bool commit) {
    std::vector<std::pair<int64_t, std::pair<int, int>>> items;
    std::vector<int> who;  // >= 0 tensor, < 0: -(planar + 1)
    for (size_t i = 0; i < p->tensors.size(); ++i) {
        const Tensor &t = p->tensors[i];
        if (t.direct) continue;  // lives only as its planar copy
        int64_t bytes = (int64_t)8 << t.rank();
        if (t.dep) bytes *= sb;
        items.push_back({align_up(bytes, 256), {t.t0, t.t1}});
        who.push_back((int)i);
    }
    for (size_t i = 0; i < p->planars.size(); ++i) {
        const Planar &q = p->planars[i];
        const Tensor &t = p->tensors[q.tensor];
        int64_t bytes = q.bytes_per_slice * (t.dep ? sb : 1);
        items.push_back({align_up(bytes, 1024), {q.t0, q.t}});
        who.push_back(-(int)i - 1);
    }
    const int npl = (int)p->planars.size();
    for (size_t i = 0; i < p->steps.size(); ++i) {
        Step &st = p->steps[i];
        if (st.kernel != K_GEMM) continue;
        const int64_t sl = st.dep ? sb : 1;
        const int sp = st.direct_planar >= 0
                           ? 1
                           : tn::gemm_simt_splits((int)st.M.size(), (int)st.N.size(),
                                                  (int)st.K.size(), sl);
        if (commit) st.splits = sp;
        if (sp <= 1) continue;
        const int64_t bytes = (int64_t)sp * sl * ((int64_t)8 << (st.M.size() + st.N.size()));
        items.push_back({align_up(bytes, 256), {st.t, st.t}});
        who.push_back(-(npl + (int)i) - 1);
    }
    std::vector<int64_t> offs;
    int64_t peak = place(items, offs);
    if (commit) {
        for (size_t i = 0; i < who.size(); ++i) {
            if (who[i] >= 0) p->tensors[who[i]].off = offs[i] / 8;
            else if (-who[i] - 1 < npl) p->planars[-who[i] - 1].off = offs[i];
            else p->steps[-who[i] - 1 - npl].part_off = offs[i];
        }
    }
    return align_up(peak, 1024);
}

tn_status build_descriptors(tn_plan_t *p);

}  // namespace

static tn_status plan_impl(const tn_network_t *net, int32_t path_len, const int32_t *path,
                           int32_t num_sliced, const int32_t *sliced_labels, tn_precision mode,
                           const tn_plan_options *opts, tn_plan_t **out);

// host allocations of the planners may throw; nothing crosses the C ABI
extern "C" tn_status tn_plan(const tn_network_t *net, int32_t path_len, const int32_t *path,
                             int32_t num_sliced, const int32_t *sliced_labels, tn_precision mode,
                             const tn_plan_options *opts, tn_plan_t **out) {
    try {
        return plan_impl(net, path_len, path, num_sliced, sliced_labels, mode, opts, out);
    } catch (const std::bad_alloc &) {
        return fail(TN_ERR_OOM, "tn_plan: host memory exhausted");
    } catch (...) {
        return fail(TN_ERR_INVALID_ARG, "tn_plan: internal error");
    }
}

static tn_status plan_impl(const tn_network_t *net, int32_t path_len, const int32_t *path,
                           int32_t num_sliced, const int32_t *sliced_labels, tn_precision mode,
                           const tn_plan_options *opts, tn_plan_t **out) {
    g_err.clear();
    if (!out) return fail(TN_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (check_net(net) != TN_OK) return TN_ERR_INVALID_ARG;
    const int nt = (int)net->labels.size();
    if (path_len != nt - 1) return fail(TN_ERR_PATH, "path has %d pairs, need %d", path_len, nt - 1);
    if (path_len > 0 && !path) return fail(TN_ERR_INVALID_ARG, "path is NULL");
    if (num_sliced < 0 || num_sliced > 40 || (num_sliced > 0 && !sliced_labels))
        return fail(TN_ERR_INVALID_ARG, "bad sliced labels");
    if ((int)mode < 0 || (int)mode > (int)TN_PREC_MIXED)
        return fail(TN_ERR_INVALID_ARG, "bad precision mode");

    auto *p = new tn_plan_t();
    p->net = net;
    p->mode = mode;
    p->device = net->device;
    if (opts) p->opts = *opts;
    p->tc_ok = tn::tc_available() && tn::tc_prepare() == cudaSuccess;
    if (tn::simt_prepare() != cudaSuccess) {
        delete p;
        return fail(TN_ERR_CUDA, "setting the CUDA-core kernels' shared-memory limit failed");
    }

    std::map<int, int> cnt;  // holders of each label (tensors + output)
    for (auto &ls : net->labels)
        for (int l : ls) cnt[l]++;
    for (int l : net->open) cnt[l]++;
    for (int j = 0; j < num_sliced; ++j) {
        int l = sliced_labels[j];
        if (cnt.find(l) == cnt.end()) {
            delete p;
            return fail(TN_ERR_INVALID_ARG, "sliced label %d is not in the network", l);
        }
        if (std::find(p->sliced.begin(), p->sliced.end(), l) != p->sliced.end()) {
            delete p;
            return fail(TN_ERR_INVALID_ARG, "sliced label %d repeated", l);
        }
        p->sliced.push_back(l);
    }
    p->num_slices = (int64_t)1 << num_sliced;
    auto is_sliced = [&](int l) {
        return std::find(p->sliced.begin(), p->sliced.end(), l) != p->sliced.end();
    };
    for (int l : p->sliced) cnt[l] = 0;

    // leaves, with sliced labels removed
    std::vector<int> cur(nt);
    std::vector<std::vector<int>> lab(nt);
    for (int i = 0; i < nt; ++i) {
        Tensor t;
        t.leaf = i;
        for (int l : net->labels[i]) {
            if (is_sliced(l)) t.dep = true;
            else lab[i].push_back(l);
        }
        if (num_sliced == 0) t.dep = true;  // one slice: everything runs in the slice loop
        p->tensors.push_back(t);
        cur[i] = i;
    }
    std::vector<bool> alive(nt, true);
    // 1. replay
    for (int s = 0; s < path_len; ++s) {
        int a = path[2 * s], b = path[2 * s + 1];
        if (a < 0 || a >= nt || b < 0 || b >= nt || a == b || !alive[a] || !alive[b]) {
            delete p;
            return fail(TN_ERR_PATH, "step %d: pair (%d, %d) invalid or retired", s, a, b);
        }
        Step st;
        st.a = cur[a];
        st.b = cur[b];
        st.la = lab[a];
        st.lb = lab[b];
        auto inb = [&](int l) { return std::find(st.lb.begin(), st.lb.end(), l) != st.lb.end(); };
        auto ina = [&](int l) { return std::find(st.la.begin(), st.la.end(), l) != st.la.end(); };
        for (int l : st.la) {
            if (inb(l)) {
                if (cnt[l] > 2) { st.batch.push_back(l); st.lc.push_back(l); }
                else st.K.push_back(l);
            } else {
                st.M.push_back(l);
                st.lc.push_back(l);
            }
        }
        for (int l : st.lb)
            if (!ina(l)) { st.N.push_back(l); st.lc.push_back(l); }
        if ((int)st.lc.size() > kMaxRank || (int)st.lc.size() > TN_MAXR - 1) {
            delete p;
            return fail(TN_ERR_UNSUPPORTED, "step %d: result rank %d too large", s,
                        (int)st.lc.size());
        }
        for (int l : st.batch) cnt[l]--;
        for (int l : st.K) cnt[l] = 0;
        const double la_ = (double)st.la.size(), lb_ = (double)st.lb.size();
        st.tcc = 8.0 * std::ldexp(1.0, (int)(la_ + lb_) - (int)st.K.size());
        st.tmc = 8.0 * (std::ldexp(1.0, (int)la_) + std::ldexp(1.0, (int)lb_) +
                        std::ldexp(1.0, (int)st.lc.size()));
        Tensor t;
        t.producer = s;
        t.dep = p->tensors[st.a].dep || p->tensors[st.b].dep;
        st.dep = t.dep;
        st.c = (int)p->tensors.size();
        p->tensors.push_back(t);
        cur[a] = st.c;
        lab[a] = st.lc;
        alive[b] = false;
        p->max_log = std::max(p->max_log, (int)st.lc.size());
        p->steps.push_back(st);
    }
    int root_id = -1;
    for (int i = 0; i < nt; ++i)
        if (alive[i]) { root_id = i; break; }
    p->root = cur[root_id];
    // the root keeps the open labels that are not sliced; sliced open labels select the block
    // of the amplitudes a slice is added to
    for (int l : net->open)
        if (!is_sliced(l)) p->root_open.push_back(l);
    {
        const int no = (int)net->open.size();
        auto open_bit = [&](int l) {
            return no - 1 - (int)(std::find(net->open.begin(), net->open.end(), l) -
                                  net->open.begin());
        };
        const int nr = (int)p->root_open.size();
        p->acc.nroot = nr;
        for (int r = 0; r < nr; ++r) p->acc.root_pos[r] = (int8_t)open_bit(p->root_open[nr - 1 - r]);
        for (int j = 0; j < (int)p->sliced.size(); ++j)
            if (std::find(net->open.begin(), net->open.end(), p->sliced[j]) != net->open.end()) {
                p->acc.bj[p->acc.nb] = (int8_t)j;
                p->acc.bpos[p->acc.nb] = (int8_t)open_bit(p->sliced[j]);
                p->acc.nb++;
            }
    }
    {
        std::vector<int> rl = lab[root_id], ol = p->root_open;
        std::sort(rl.begin(), rl.end());
        std::sort(ol.begin(), ol.end());
        if (rl != ol) {
            delete p;
            return fail(TN_ERR_PATH, "the path does not reduce to a tensor of the open labels");
        }
    }
    for (int i = 0; i < nt; ++i) p->max_log = std::max(p->max_log, (int)lab[i].size());

    // 2. routing
    for (auto &st : p->steps) {
        st.kernel = route(st, mode, p->tc_ok);
        // slice-independent steps run once per call; they stay on the CUDA cores
        if (!st.dep && st.kernel == K_TC) st.kernel = K_GEMM;
        // a streaming step with K = 16, or with 16 columns and K = 8, takes the tensor cores
        // (compensated TF32, FP32-level accuracy) in the tensor-core modes: on the CUDA cores
        // its 4 * NT * K multiply-adds per row and their operand reads keep it below memory
        // speed (measured on GB300 at 2^24-2^26 rows: K = 16 with 4, 8, 16 columns 3.6, 2.9,
        // 3.3 TB/s there against 3.6, 3.9, 4.6 on the tensor cores; 16 columns and K = 8 3.9
        // against 4.6); the other shapes are faster on the CUDA cores (4.2-6.7 TB/s against
        // 2.4-3.9).  opts.thin_tc > 0 sends every step that fits, < 0 none
        if (st.kernel == K_STREAM && mode != TN_PREC_C64 && p->tc_ok && st.dep) {
            const int wide = (int)std::max(st.M.size(), st.N.size());
            const int narrow = (int)std::min(st.M.size(), st.N.size());
            const int lk = (int)st.K.size();
            st.thin_tc = tn::thin_tc_fits(wide, narrow, lk) &&
                         (p->opts.thin_tc > 0 ||
                          (p->opts.thin_tc == 0 && (lk == 4 || (narrow == 4 && lk == 3))));
        }
        if (mode == TN_PREC_SPLIT_FP16 || mode == TN_PREC_SPLIT_BF16 ||
            mode == TN_PREC_SPLIT_TF32 || mode == TN_PREC_MIXED)
            st.form = kFormSplit;
        else
            st.form = (p->opts.gemm_form == TN_GEMM_3M) ? TN_GEMM_3M : TN_GEMM_4M;
    }

    if (mode == TN_PREC_MIXED || single_pass_mode(mode)) {
        // Sec. 4.3 / Table 3: the dense steps with the largest T_cc run single-pass, the others
        // with compensated hi/lo products of the same type; k from the mode, mixed_topk and
        // the error budget (precision policy in tn.h)
        std::vector<int> tc;
        for (int s = 0; s < path_len; ++s)
            if (p->steps[s].kernel == K_TC && p->steps[s].dep) tc.push_back(s);
        std::stable_sort(tc.begin(), tc.end(), [&](int x, int y) {
            return p->steps[x].tcc > p->steps[y].tcc;
        });
        const int ntc = (int)tc.size(), topk = p->opts.mixed_topk;
        const double budget = p->opts.eps_budget > 0 ? p->opts.eps_budget
                              : (mode == TN_PREC_BF16_SCALED ? kBf16DefaultBudget : 0.0);
        int k = ntc;
        if (mode == TN_PREC_MIXED) k = topk > 0 ? std::min(topk, ntc) : (budget > 0 ? ntc : 1);
        else if (topk > 0) k = std::min(topk, ntc);
        k = std::min(k, ntc);
        if (budget > 0)
            while (k > 0 && predicted_eps(mode, k, ntc - k) > budget) --k;
        const int split_form_default =
            (p->opts.gemm_form == TN_GEMM_3M) ? TN_GEMM_3M : TN_GEMM_4M;
        for (int i = 0; i < ntc; ++i) {
            Step &st = p->steps[tc[i]];
            st.form = i < k ? (mode == TN_PREC_MIXED ? TN_GEMM_4M : split_form_default)
                            : kFormSplit;
        }
        p->single_pass = k;
        p->compensated = ntc - k;
        p->eps_pred = predicted_eps(mode, k, ntc - k);
    } else {
        int ntc = 0;
        for (auto &st : p->steps) ntc += st.kernel == K_TC && st.dep;
        p->single_pass = 0;  // c64 (no dense steps) or a compensated mode
        p->compensated = mode == TN_PREC_C64 ? 0 : ntc;
        p->eps_pred = predicted_eps(mode, 0, p->compensated);
    }
    for (auto &st : p->steps)
        st.tune_form = p->opts.autotune && p->opts.gemm_form == TN_GEMM_AUTO &&
                       st.kernel == K_TC && st.form != kFormSplit;

    // 3. layout: root first, then every step's operands from its result's order
    p->tensors[p->root].order = p->root_open;
    for (int s = path_len - 1; s >= 0; --s) {
        Step &st = p->steps[s];
        const std::vector<int> &co = p->tensors[st.c].order;
        auto pos_in = [&](const std::vector<int> &v, int l) {
            return (int)(std::find(v.begin(), v.end(), l) - v.begin());
        };
        // Operand roles of a GEMM step: the tensor-core epilogue maps consecutive lanes to
        // consecutive rows (m), the CUDA-core one maps them to consecutive columns (n); give the
        // label at bit 0 of the result to the side whose stores are then contiguous.
        if (st.kernel == K_TC && std::min(st.M.size(), st.N.size()) < 7) {
            // the 32- or 64-column tile: the wide side must be M (tiles of 128 rows)
            if (st.M.size() < st.N.size()) {
                std::swap(st.a, st.b);
                std::swap(st.la, st.lb);
                std::swap(st.M, st.N);
            }
        } else if ((st.kernel == K_TC || st.kernel == K_GEMM) && !co.empty()) {
            const int low = co.back();
            const bool low_in_m = std::find(st.M.begin(), st.M.end(), low) != st.M.end();
            const bool want_m = st.kernel == K_TC;
            if (low_in_m != want_m) {
                std::swap(st.a, st.b);
                std::swap(st.la, st.lb);
                std::swap(st.M, st.N);
            }
        }
        std::vector<int> oa, ob;
        for (int l : co) {
            if (std::find(st.la.begin(), st.la.end(), l) != st.la.end()) oa.push_back(l);
            if (std::find(st.lb.begin(), st.lb.end(), l) != st.lb.end()) ob.push_back(l);
        }
        for (int l : st.K) { oa.push_back(l); ob.push_back(l); }
        // M and N in the order of the result (used by the GEMM descriptors)
        std::sort(st.M.begin(), st.M.end(), [&](int x, int y) { return pos_in(co, x) < pos_in(co, y); });
        std::sort(st.N.begin(), st.N.end(), [&](int x, int y) { return pos_in(co, x) < pos_in(co, y); });
        p->tensors[st.a].order = oa;
        p->tensors[st.b].order = ob;
    }
    if (path_len == 0) p->tensors[p->root].order = p->root_open;

    // 4. tensor-core operands get planar 16-bit copies.  When the operand's producer is a GEMM
    //    step of the slice loop (with whole 64 x 64 tiles to spare), that producer writes the
    //    copy directly, with an exponent bounded from its own inputs' max-abs; otherwise a
    //    conversion pass makes it from complex64 just before the step.
    for (int s = 0; s < path_len; ++s) {
        Step &st = p->steps[s];
        if (!st.dep || st.kernel != K_TC) continue;
        for (int side = 0; side < 2; ++side) {
            Planar q;
            q.tensor = side ? st.b : st.a;
            q.planes = st.form == TN_GEMM_3M ? 3 : (st.form == kFormSplit ? 4 : 2);
            if (st.tune_form) q.planes = 3;  // the tuner may pick 3M for this step
            q.cap_planes = q.planes;
            q.bytes_per_slice = (int64_t)((tf32_mode(mode) ? 4 : 2) * q.cap_planes)
                                << p->tensors[q.tensor].rank();
            const Tensor &X = p->tensors[q.tensor];
            // TF32 operands (FP32 storage) are always made by the conversion pass
            if (X.producer >= 0 && st.form != kFormSplit && !tf32_mode(mode)) {
                // A producer's direct output takes its exponent from a bound (2 K max|a| max|b|)
                // that can exceed the true maximum by many binades, which leaves the stored
                // values low in FP16's range; single-pass operands keep their 11 significant
                // bits there, but the lo planes of compensated operands would fall into the
                // subnormals, so those are split from complex64 with their measured max-abs.
                // A CUDA-core producer writes directly only with whole 64 x 64 tiles, and then
                // never splits K (its epilogue must hold final sums).
                // A CUDA-core producer that would split K (judged at one slice in flight, its
                // fewest tiles) writes complex64 instead: a long contraction over few tiles
                // needs the split more than the saved conversion pass.
                const Step &pr = p->steps[X.producer];
                q.direct = pr.dep && (pr.kernel == K_TC || pr.kernel == K_STREAM ||
                                      (pr.kernel == K_GEMM && pr.M.size() >= 6 &&
                                       pr.N.size() >= 6 &&
                                       tn::gemm_simt_splits((int)pr.M.size(), (int)pr.N.size(),
                                                            (int)pr.K.size(), 1) == 1));
            }
            (side ? st.pb : st.pa) = (int)p->planars.size();
            p->planars.push_back(q);
        }
    }
    {
        auto need_meta = [&](int ti) {
            if (p->tensors[ti].meta < 0) p->tensors[ti].meta = p->nmeta++;
        };
        for (auto &q : p->planars) need_meta(q.tensor);
        for (auto &q : p->planars)
            if (q.direct) {
                const Step &pr = p->steps[p->tensors[q.tensor].producer];
                if (pr.kernel == K_GEMM || pr.kernel == K_STREAM) {
                    need_meta(pr.a);
                    need_meta(pr.b);
                }
            }
        for (auto &q : p->planars) {
            q.meta = p->tensors[q.tensor].meta;
            if (q.direct) {
                p->tensors[q.tensor].direct = true;
                p->steps[p->tensors[q.tensor].producer].direct_planar = (int)(&q - &p->planars[0]);
            }
        }
        // a tensor's max-abs is recorded by its producer's epilogue; leaves get an amax pass
        for (auto &x : p->tensors)
            if (x.meta >= 0 && x.producer >= 0) p->steps[x.producer].out_meta = x.meta;
    }
    // runs of consecutive small element-wise steps are launched together, one block per slice
    // (k_generic_chain): runs of the slice-independent prologue and runs of the slice loop,
    // each in its own execution order; not in profile mode, which times every step on its own
    if (!p->opts.profile) {
        std::vector<int> run[2];  // [0] prologue, [1] slice loop
        auto close_run = [&](std::vector<int> &r) {
            if (r.size() >= 2) {
                const int id = (int)p->chains.size();
                for (int k : r) p->steps[k].chain = id;
                p->steps[r[0]].chain_head = true;
                p->chains.push_back(r);
            }
            r.clear();
        };
        for (int s = 0; s < path_len; ++s) {
            const Step &st = p->steps[s];
            const int rc = p->tensors[st.c].rank(), nk = (int)st.K.size();
            const bool small = st.kernel == K_GENERIC && st.out_meta < 0 &&
                               rc <= tn::kChainMaxRankC && nk <= tn::kChainMaxNk &&
                               rc + nk <= tn::kChainMaxWork;
            std::vector<int> &r = run[st.dep ? 1 : 0];
            if (small) r.push_back(s);
            else close_run(r);
        }
        close_run(run[0]);
        close_run(run[1]);
    }
    // op timeline: invariant leaves, invariant steps, sliced leaves, dependent steps (each
    // tensor-core step preceded by its conversions; a run of chained steps is one op, so every
    // tensor it touches is live at that op and no two of them share memory), accumulate
    std::vector<Op> ops;
    ops.push_back({0, -1});
    for (int s = 0; s < path_len; ++s)
        if (!p->steps[s].dep && (p->steps[s].chain < 0 || p->steps[s].chain_head))
            ops.push_back({1, s});
    ops.push_back({2, -1});
    for (int s = 0; s < path_len; ++s)
        if (p->steps[s].dep) {
            Step &st = p->steps[s];
            if (st.chain >= 0 && !st.chain_head) continue;  // part of its run's op
            if (st.kernel == K_TC) {
                ops.push_back({3, st.pa});
                ops.push_back({3, st.pb});
            }
            ops.push_back({1, s});
        }
    ops.push_back({4, -1});
    const int tend = (int)ops.size() - 1;
    for (int t = 0; t < (int)ops.size(); ++t) {
        const Op &op = ops[t];
        if (op.kind == 0 || op.kind == 2) {
            for (auto &x : p->tensors)
                if (x.producer < 0 && x.dep == (op.kind == 2)) x.t0 = x.t1 = t;
        } else if (op.kind == 1) {
            const Step &head = p->steps[op.index];
            const std::vector<int> one{op.index};
            for (int k : head.chain_head ? p->chains[head.chain] : one) {
                Step &st = p->steps[k];
                st.t = t;
                p->tensors[st.c].t0 = p->tensors[st.c].t1 = t;
                p->tensors[st.a].t1 = t;
                p->tensors[st.b].t1 = t;
            }
        }
    }
    for (auto &st : p->steps) {
        if (st.kernel != K_TC) continue;
        for (int side = 0; side < 2; ++side) {
            Planar &q = p->planars[side ? st.pb : st.pa];
            q.t = st.t;  // last use
            q.t0 = q.direct ? p->steps[p->tensors[q.tensor].producer].t : st.t - 2;
        }
    }
    // invariant tensors read by the slice loop stay live through all batches
    for (auto &st : p->steps)
        if (st.dep) {
            if (!p->tensors[st.a].dep) p->tensors[st.a].t1 = tend;
            if (!p->tensors[st.b].dep) p->tensors[st.b].t1 = tend;
        }
    p->tensors[p->root].t1 = tend;

    // 5. slices per launch under the workspace limit
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        delete p;
        return fail(TN_ERR_CUDA, "cudaMemGetInfo failed");
    }
    int64_t limit = p->opts.workspace_limit > 0 ? p->opts.workspace_limit
                                                : (int64_t)((double)free_b * 0.6);
    int64_t sb = p->num_slices;
    if (p->opts.max_slices_in_flight > 0) sb = std::min(sb, p->opts.max_slices_in_flight);
    sb = std::min<int64_t>(sb, 65535);
    while (sb > 1 && layout_bytes(p, sb, false) > limit) sb = (sb + 1) / 2;
    const int64_t need = layout_bytes(p, sb, true);
    if (need > limit) {
        delete p;
        return fail(TN_ERR_OOM, "workspace needs %lld bytes for one slice, limit %lld",
                    (long long)need, (long long)limit);
    }
    p->sb = sb;
    p->arena_bytes = need;
    if (p->opts.workspace) {
        if (reinterpret_cast<uintptr_t>(p->opts.workspace) % 256 != 0) {
            delete p;
            return fail(TN_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
        }
        p->arena = (char *)p->opts.workspace;
    } else {
        cudaError_t e = cudaMalloc(&p->arena, (size_t)need);
        if (e != cudaSuccess) {
            delete p;
            return fail(TN_ERR_OOM, "cudaMalloc workspace (%lld bytes): %s", (long long)need,
                        cudaGetErrorString(e));
        }
        p->own_arena = true;
    }
    tn_status s = build_descriptors(p);
    if (s != TN_OK) {
        tn_destroy(p);
        return s;
    }
    *out = p;
    return TN_OK;
}

namespace {

tn::BindItem make_bind(const tn_plan_t *p, const Tensor &t) {
    tn::BindItem it{};
    const std::vector<int> &src = p->net->labels[t.leaf];
    it.dst_off = t.off;
    it.dst_sstride = t.dep ? ((int64_t)1 << t.rank()) : 0;
    if (p->sliced.empty()) it.dst_sstride = 0;
    it.src_off = p->net->offset[t.leaf];
    it.rank = t.rank();
    const int rs = (int)src.size();
    fill_pos(it.pos_src, TN_MAXR, -1);
    for (int i = 0; i < t.rank(); ++i) {
        const int l = t.order[t.rank() - 1 - i];
        const int j = (int)(std::find(src.begin(), src.end(), l) - src.begin());
        it.pos_src[i] = (int8_t)(rs - 1 - j);
    }
    it.nsl = 0;
    for (int j = 0; j < (int)p->sliced.size(); ++j) {
        auto f = std::find(src.begin(), src.end(), p->sliced[j]);
        if (f == src.end()) continue;
        it.sl_bit[it.nsl] = (int8_t)j;
        it.sl_pos[it.nsl] = (int8_t)(rs - 1 - (int)(f - src.begin()));
        it.nsl++;
    }
    return it;
}

// Leaves of at least this rank are bound by the tiled permutation kernel (k_bind_tiled); smaller
// ones (gates, projectors) are gathered many per launch by k_bind.
constexpr int kTiledBindMinRank = 12;

// Tile tables of a large leaf (see tn::BindTiled) from its gather description.  The tile holds
// destination bits 0-5 and the destination bits of the six lowest unsliced source bits (runs
// of 1 KiB in the source); while it has fewer than 11 bits (the two sets overlap) it grows by
// the next destination bit and the next source bit in turn.  A block reads the tile with its
// bits in source order, so consecutive threads read consecutive source addresses.
tn::BindTiled make_bind_tiled(const tn::BindItem &it) {
    tn::BindTiled b{};
    b.dst_off = it.dst_off;
    b.dst_sstride = it.dst_sstride;
    b.src_off = it.src_off;
    b.nsl = it.nsl;
    for (int j = 0; j < 8; ++j) {
        b.sl_bit[j] = it.sl_bit[j];
        b.sl_pos[j] = it.sl_pos[j];
    }
    const int r = it.rank;
    // destination bits ordered by their source bit
    std::vector<std::pair<int, int>> by_src;
    for (int i = 0; i < r; ++i) by_src.push_back({it.pos_src[i], i});
    std::sort(by_src.begin(), by_src.end());
    std::vector<bool> in(r, false);
    int nd = 0, ns = 0, t = 0;
    auto add = [&](int d) {
        if (!in[d]) {
            in[d] = true;
            t++;
        }
    };
    for (; nd < 6 && nd < r; ++nd) add(nd);
    for (; ns < 6 && ns < r; ++ns) add(by_src[ns].second);
    for (bool dst_turn = true; t < 11 && (nd < r || ns < r); dst_turn = !dst_turn) {
        if (dst_turn && nd < r) add(nd++);
        else if (!dst_turn && ns < r) add(by_src[ns++].second);
    }
    // tile bits: destination bits 0-5 first, then the others in destination order
    std::vector<int> tile_d;
    for (int d = 0; d < r; ++d)
        if (in[d]) tile_d.push_back(d);
    b.t = (int)tile_d.size();
    auto tile_bit = [&](int d) {
        return (int)(std::find(tile_d.begin(), tile_d.end(), d) - tile_d.begin());
    };
    for (int q = 0; q < 12; ++q) b.t2d[q] = q < b.t ? (int8_t)tile_d[q] : (int8_t)-1;
    // read order: the tile's bits by increasing source bit
    std::vector<int> order;
    for (auto &x : by_src)
        if (in[x.second]) order.push_back(x.second);
    for (int q = 0; q < 12; ++q) {
        b.e2t[q] = q < b.t ? (int8_t)tile_bit(order[q]) : (int8_t)-1;
        b.e2s[q] = q < b.t ? it.pos_src[order[q]] : (int8_t)-1;
    }
    fill_pos(b.rest_d, TN_MAXR, -1);
    fill_pos(b.rest_s, TN_MAXR, -1);
    int u = 0;
    for (int d = 0; d < r; ++d)
        if (!in[d]) {
            b.rest_d[u] = (int8_t)d;
            b.rest_s[u] = it.pos_src[d];
            u++;
        }
    b.nrest = u;
    b.ntiles = (int64_t)1 << u;
    return b;
}

// Direct planar output of step st (see tn::PlanarOut): the consumer's planar buffer, the
// exponents of its meta block, and the max-abs of st's inputs for the bound.
void fill_planar_out(const tn_plan_t *p, const Step &st, tn::PlanarOut &o) {
    const Planar &q = p->planars[st.direct_planar];
    const Tensor &C = p->tensors[st.c], &A = p->tensors[st.a], &B = p->tensors[st.b];
    const int64_t n = (int64_t)1 << C.rank();
    o.base = p->arena + q.off;
    o.sstride = C.dep ? n : 0;
    o.plane_stride = n * (C.dep ? p->sb : 1);
    o.planes = q.planes;
    o.bf16 = bf16_mode(p->mode);
    o.exps = reinterpret_cast<int32_t *>(p->meta + 2 * p->sb * q.meta + p->sb);
    o.amax_a = p->meta + 2 * p->sb * A.meta;
    o.amax_b = p->meta + 2 * p->sb * B.meta;
    o.a_sliced = A.dep ? 1 : 0;
    o.b_sliced = B.dep ? 1 : 0;
    o.log2_k = (int)st.K.size();
}

// Descriptor of tensor-core step st with kernel variant `variant` (tile shape and form).
tn_status make_tc_desc(const tn_plan_t *p, const Step &st, int variant, tn::TcGemmDesc &d) {
    memset(&d, 0, sizeof d);
    const Tensor &A = p->tensors[st.a], &B = p->tensors[st.b], &C = p->tensors[st.c];
    const int bf = operand_dtype(p->mode);
    const int64_t Kx = (int64_t)1 << st.K.size();
    const Planar &qa = p->planars[st.pa], &qb = p->planars[st.pb];
    const int64_t sa = A.dep ? p->sb : 1, sbb = B.dep ? p->sb : 1;
    if (tn::tc_variant_tf32(variant) != (bf == 2))
        return fail(TN_ERR_UNSUPPORTED, "kernel variant %d does not take this operand type",
                    variant);
    d.variant = variant;
    d.bk = tn::tc_variant_bk(variant);
    d.form = tn::tc_variant_form(variant);
    if (d.form == 2 && (qa.planes != 3 || qb.planes != 3))
        return fail(TN_ERR_UNSUPPORTED, "3M needs the operands' sum planes");
    if (d.form == 3 && (qa.planes != 4 || qb.planes != 4))
        return fail(TN_ERR_UNSUPPORTED, "compensated products need the operands' lo planes");
    const int bn = tn::tc_variant_bn(variant);
    if (tn::encode_tmap_planar(&d.tmA, p->arena + qa.off, Kx, (int64_t)1 << st.M.size(),
                                 qa.cap_planes * sa, bf, d.bk, 128) != 0 ||
        tn::encode_tmap_planar(&d.tmB, p->arena + qb.off, Kx, (int64_t)1 << st.N.size(),
                                 qb.cap_planes * sbb, bf, d.bk, bn) != 0)
        return fail(TN_ERR_CUDA, "cuTensorMapEncodeTiled failed for step %d",
                    (int)(&st - &p->steps[0]));
    d.C = reinterpret_cast<float2 *>(p->arena) + C.off;
    d.sC = C.dep ? ((int64_t)1 << C.rank()) : 0;
    d.lm = (int)st.M.size();
    d.ln = (int)st.N.size();
    d.lk = (int)st.K.size();
    d.a_sliced = A.dep ? 1 : 0;
    d.b_sliced = B.dep ? 1 : 0;
    d.slices_a = sa;
    d.slices_b = sbb;
    d.expA = reinterpret_cast<const int32_t *>(p->meta + 2 * p->sb * qa.meta + p->sb);
    d.expB = reinterpret_cast<const int32_t *>(p->meta + 2 * p->sb * qb.meta + p->sb);
    d.dtype = bf;
    d.amax_out = st.out_meta >= 0 ? p->meta + 2 * p->sb * st.out_meta : nullptr;
    if (st.direct_planar >= 0) {
        d.planar_out = 1;
        fill_planar_out(p, st, d.pout);
    }
    fill_pos(d.posC_m, TN_MAXR, -1);
    fill_pos(d.posC_n, TN_MAXR, -1);
    for (int i = 0; i < d.lm; ++i) d.posC_m[i] = (int8_t)C.pos(st.M[st.M.size() - 1 - i]);
    for (int i = 0; i < d.ln; ++i) d.posC_n[i] = (int8_t)C.pos(st.N[st.N.size() - 1 - i]);
    // epilogue chunk: 7 row bits and 6 column bits, sorted by position in C; the first three
    // are always positions 0-2 (C's three lowest labels are among the lowest three of M and
    // of N), which the epilogue's 8-element stores rely on
    // (the persistent short-K variants stage 32-column chunks: 7 row and 5 column bits)
    const bool pers = tn::tc_variant_is_pers(variant);
    tn::sort_tile_bits(7, pers || bn == 32 ? 5 : 6, d.posC_m, d.posC_n, 128, d.tb_src, d.tb_pos);
    if (pers) {
        tn::tc_choose_swizzle(d.tb_src, d.phi, 4);
        tn::tc_choose_swizzle(d.tb_src, d.phi5, 5);
    }
    if (d.tb_pos[0] != 0 || d.tb_pos[1] != 1 || d.tb_pos[2] != 2)
        return fail(TN_ERR_UNSUPPORTED, "step %d: result bits 0-2 outside the epilogue chunk",
                    (int)(&st - &p->steps[0]));
    return TN_OK;
}

tn::GenericDesc make_generic_desc(const tn_plan_t *p, const Step &st, unsigned int *amax_out) {
    const Tensor &A = p->tensors[st.a], &B = p->tensors[st.b], &C = p->tensors[st.c];
    float2 *arena = reinterpret_cast<float2 *>(p->arena);
    tn::GenericDesc d{};
    d.A = arena + A.off;
    d.B = arena + B.off;
    d.C = arena + C.off;
    d.sA = A.dep ? ((int64_t)1 << A.rank()) : 0;
    d.sB = B.dep ? ((int64_t)1 << B.rank()) : 0;
    d.sC = C.dep ? ((int64_t)1 << C.rank()) : 0;
    d.rank_c = C.rank();
    d.nk = (int)st.K.size();
    d.amax_out = amax_out;
    fill_pos(d.posA_c, TN_MAXR, -1);
    fill_pos(d.posB_c, TN_MAXR, -1);
    fill_pos(d.posA_k, TN_MAXR, -1);
    fill_pos(d.posB_k, TN_MAXR, -1);
    for (int i = 0; i < C.rank(); ++i) {
        const int l = C.order[C.rank() - 1 - i];
        d.posA_c[i] = (int8_t)A.pos(l);
        d.posB_c[i] = (int8_t)B.pos(l);
    }
    const int nk = (int)st.K.size();
    for (int j = 0; j < nk; ++j) {
        const int l = st.K[nk - 1 - j];
        d.posA_k[j] = (int8_t)A.pos(l);
        d.posB_k[j] = (int8_t)B.pos(l);
    }
    return d;
}

tn_status build_descriptors(tn_plan_t *p) {
    for (auto &t : p->tensors) {
        if (t.leaf < 0) continue;
        if (t.rank() > TN_MAXR - 1) return fail(TN_ERR_UNSUPPORTED, "leaf rank too large");
        int nsl = 0;
        for (int l : p->net->labels[t.leaf])
            if (std::find(p->sliced.begin(), p->sliced.end(), l) != p->sliced.end()) nsl++;
        if (nsl > 8) return fail(TN_ERR_UNSUPPORTED, "a leaf carries more than 8 sliced labels");
        tn::BindItem it = make_bind(p, t);
        if (t.rank() >= kTiledBindMinRank) {
            (t.dep ? p->tiled_sl : p->tiled_inv).push_back(make_bind_tiled(it));
            continue;
        }
        if (t.dep) {
            p->bind_sl.push_back(it);
            p->max_rank_sl = std::max(p->max_rank_sl, t.rank());
        } else {
            p->bind_inv.push_back(it);
            p->max_rank_inv = std::max(p->max_rank_inv, t.rank());
        }
    }
    auto upload = [&](std::vector<tn::BindItem> &v, tn::BindItem **dst) -> tn_status {
        if (v.empty()) return TN_OK;
        TN_CUDA(cudaMalloc(dst, sizeof(tn::BindItem) * v.size()));
        TN_CUDA(cudaMemcpy(*dst, v.data(), sizeof(tn::BindItem) * v.size(),
                           cudaMemcpyHostToDevice));
        return TN_OK;
    };
    tn_status s = upload(p->bind_inv, &p->bind_inv_dev);
    if (s != TN_OK) return s;
    s = upload(p->bind_sl, &p->bind_sl_dev);
    if (s != TN_OK) return s;
    if (p->nmeta > 0)
        TN_CUDA(cudaMalloc(&p->meta, sizeof(unsigned int) * 2 * p->sb * p->nmeta));
    TN_CUDA(cudaMalloc(&p->partial, sizeof(double) * 2 * p->n_partial));
    TN_CUDA(cudaMalloc(&p->amps_tmp, sizeof(double2) << p->net->open.size()));

    if (!p->chains.empty()) {
        std::vector<tn::GenericDesc> all;
        for (const auto &run : p->chains) {
            p->chain_first.push_back((int64_t)all.size());
            for (int k : run) all.push_back(make_generic_desc(p, p->steps[k], nullptr));
        }
        TN_CUDA(cudaMalloc(&p->chain_dev, sizeof(tn::GenericDesc) * all.size()));
        TN_CUDA(cudaMemcpy(p->chain_dev, all.data(), sizeof(tn::GenericDesc) * all.size(),
                           cudaMemcpyHostToDevice));
    }
    p->tc_desc.resize(p->steps.size());
    for (auto &st : p->steps) {
        if (st.kernel != K_TC) continue;
        st.variant = tn::tc_pick_variant(st.form == TN_GEMM_3M ? 2 : (st.form == kFormSplit ? 3 : 1),
                                         (int)st.K.size(), (int)st.N.size(), p->opts.tc_bk,
                                         p->opts.tc_bn, tf32_mode(p->mode));
        tn_status s = make_tc_desc(p, st, st.variant, p->tc_desc[&st - &p->steps[0]]);
        if (s != TN_OK) return s;
    }
    return TN_OK;
}

using EventPair = std::pair<cudaEvent_t, cudaEvent_t>;

tn_status run_step_inner(tn_plan_t *p, const Step &st, int64_t slices, cudaStream_t stream,
                         const EventPair *ev, const EventPair *prep);

tn_status take_events(tn_plan_t *p, EventPair &ev) {
    if (!p->event_pool.empty()) {
        ev = p->event_pool.back();
        p->event_pool.pop_back();
        return TN_OK;
    }
    TN_CUDA(cudaEventCreate(&ev.first));
    TN_CUDA(cudaEventCreate(&ev.second));
    return TN_OK;
}

tn_status make_tc_desc(const tn_plan_t *p, const Step &st, int variant, tn::TcGemmDesc &d);

// Bind the invariant leaves (sliced = false, once per call) or the sliced leaves of slices
// [s0, s0 + ns): small leaves in one gather launch, each large leaf by the tiled permutation.
// Profile mode brackets them with one event pair.
tn_status bind_leaves(tn_plan_t *p, bool sliced, int64_t s0, int64_t ns, cudaStream_t stream) {
    const auto &items = sliced ? p->bind_sl : p->bind_inv;
    const auto &tiled = sliced ? p->tiled_sl : p->tiled_inv;
    if (items.empty() && tiled.empty()) return TN_OK;
    float2 *arena = reinterpret_cast<float2 *>(p->arena);
    const double2 *src = p->net->data;
    EventPair ev{};
    if (p->opts.profile) {
        tn_status s = take_events(p, ev);
        if (s != TN_OK) return s;
        TN_CUDA(cudaEventRecord(ev.first, stream));
    }
    if (!items.empty()) {
        TN_CUDA(tn::launch_bind(sliced ? p->bind_sl_dev : p->bind_inv_dev, (int32_t)items.size(),
                                src, arena, s0, ns, sliced ? p->max_rank_sl : p->max_rank_inv,
                                stream));
        p->launches++;
    }
    for (const auto &b : tiled) {
        TN_CUDA(tn::launch_bind_tiled(b, src, arena, s0, ns, stream));
        p->launches++;
    }
    if (p->opts.profile) {
        TN_CUDA(cudaEventRecord(ev.second, stream));
        p->pending_bind.push_back(ev);
    }
    return TN_OK;
}

// Autotune a tensor-core step (first full batch): run it once as planned, then launch every
// applicable kernel variant (tile shape, K tile, 4M or 3M) between CUDA events and keep the
// fastest.  All variants compute the same result; when 4M wins, the operands' sum planes are
// no longer written.
tn_status tune_tc_step(tn_plan_t *p, Step &st, int64_t slices, cudaStream_t stream) {
    const int si = (int)(&st - &p->steps[0]);
    tn_status s = run_step_inner(p, st, slices, stream, nullptr, nullptr);
    if (s != TN_OK) return s;
    const int lk = (int)st.K.size(), ln = (int)st.N.size();
    const bool three_planes = p->planars[st.pa].planes == 3 && p->planars[st.pb].planes == 3;
    std::vector<int> cands;
    std::vector<tn::TcGemmDesc> descs;
    std::vector<EventPair> evs;
    for (int v = 0; v < tn::tc_num_variants(); ++v) {
        if (!tn::tc_variant_fits(v, lk, ln)) continue;
        const int form = tn::tc_variant_form(v);
        if ((st.form == kFormSplit) != (form == 3)) continue;  // split steps stay split
        if (tn::tc_variant_tf32(v) != tf32_mode(p->mode)) continue;
        if (form == 2 && !three_planes) continue;
        if (p->opts.gemm_form == TN_GEMM_4M && form == 2) continue;
        if (p->opts.gemm_form == TN_GEMM_3M && form == 1) continue;
        tn::TcGemmDesc d;
        s = make_tc_desc(p, st, v, d);
        if (s != TN_OK) return s;
        EventPair ev;
        TN_CUDA(cudaEventCreate(&ev.first));
        TN_CUDA(cudaEventCreate(&ev.second));
        cands.push_back(v);
        descs.push_back(d);
        evs.push_back(ev);
    }
    for (size_t i = 0; i < cands.size(); ++i) {
        TN_CUDA(cudaEventRecord(evs[i].first, stream));
        TN_CUDA(tn::launch_gemm_tc(descs[i], slices, stream));
        TN_CUDA(cudaEventRecord(evs[i].second, stream));
        p->launches += 1;
    }
    TN_CUDA(cudaStreamSynchronize(stream));
    int best = -1;
    float best_ms = 0.f;
    for (size_t i = 0; i < cands.size(); ++i) {
        float ms = 0.f;
        TN_CUDA(cudaEventElapsedTime(&ms, evs[i].first, evs[i].second));
        if (best < 0 || ms < best_ms) {
            best = (int)i;
            best_ms = ms;
        }
        cudaEventDestroy(evs[i].first);
        cudaEventDestroy(evs[i].second);
    }
    if (best < 0) return TN_OK;
    st.variant = cands[best];
    {
        const int f = tn::tc_variant_form(st.variant);
        st.form = f == 2 ? TN_GEMM_3M : (f == 3 ? kFormSplit : TN_GEMM_4M);
    }
    p->tc_desc[si] = descs[best];
    if (st.form == TN_GEMM_4M && st.tune_form) {
        // the sum planes are not read: their producers stop writing them
        for (int side = 0; side < 2; ++side) {
            Planar &q = p->planars[side ? st.pb : st.pa];
            q.planes = 2;
            const Tensor &X = p->tensors[q.tensor];
            if (q.direct && p->steps[X.producer].kernel == K_TC)
                p->tc_desc[X.producer].pout.planes = 2;
        }
    }
    st.tune_form = false;
    return TN_OK;
}

// Launch one step; in profile mode its main kernel (and, for a tensor-core step, its operand
// conversions) are bracketed by CUDA events on the contraction stream.
tn_status run_step(tn_plan_t *p, Step &st, int64_t slices, cudaStream_t stream) {
    if (st.chain >= 0) {
        // the run's first step launches the whole run; the others are part of that launch
        if (!st.chain_head) return TN_OK;
        const cudaError_t e = tn::launch_generic_chain(
            p->chain_dev + p->chain_first[st.chain], (int32_t)p->chains[st.chain].size(), slices,
            stream);
        if (e != cudaSuccess)
            return fail(TN_ERR_CUDA, "step %d chain launch: %s", (int)(&st - &p->steps[0]),
                        cudaGetErrorString(e));
        p->launches += 1;
        return TN_OK;
    }
    if (!p->opts.profile) return run_step_inner(p, st, slices, stream, nullptr, nullptr);
    EventPair ev{nullptr, nullptr}, prep{nullptr, nullptr};
    tn_status s = take_events(p, ev);
    if (s != TN_OK) return s;
    if (st.kernel == K_TC) {
        s = take_events(p, prep);
        if (s != TN_OK) return s;
    }
    s = run_step_inner(p, st, slices, stream, &ev, st.kernel == K_TC ? &prep : nullptr);
    st.pending.push_back(ev);
    if (st.kernel == K_TC) st.pending_prep.push_back(prep);
    return s;
}

tn_status run_step_inner(tn_plan_t *p, const Step &st, int64_t slices, cudaStream_t stream,
                         const EventPair *ev, const EventPair *prep) {
    const Tensor &A = p->tensors[st.a], &B = p->tensors[st.b], &C = p->tensors[st.c];
    float2 *arena = reinterpret_cast<float2 *>(p->arena);
    const int64_t sA = A.dep ? ((int64_t)1 << A.rank()) : 0;
    const int64_t sB = B.dep ? ((int64_t)1 << B.rank()) : 0;
    const int64_t sC = C.dep ? ((int64_t)1 << C.rank()) : 0;
    cudaError_t e = cudaSuccess;
    unsigned int *amax_out = nullptr;
    if (st.out_meta >= 0) {
        amax_out = p->meta + 2 * p->sb * st.out_meta;
        TN_CUDA(cudaMemsetAsync(amax_out, 0, sizeof(unsigned int) * (C.dep ? slices : 1),
                                stream));
    }
    // a direct CUDA-core or streaming producer bounds its output from its inputs' max-abs;
    // inputs that are leaves (no producer epilogue records it) get an amax pass here
    if ((st.kernel == K_GEMM || st.kernel == K_STREAM) && st.direct_planar >= 0) {
        for (int side = 0; side < 2; ++side) {
            const Tensor &X = side ? B : A;
            if (X.producer >= 0) continue;
            tn::ConvertDesc cd{};
            cd.src = arena + X.off;
            cd.n = (int64_t)1 << X.rank();
            cd.src_sstride = X.dep ? cd.n : 0;
            cd.amax = p->meta + 2 * p->sb * X.meta;
            const int64_t sx = X.dep ? slices : 1;
            TN_CUDA(cudaMemsetAsync(cd.amax, 0, sizeof(unsigned int) * sx, stream));
            TN_CUDA(tn::launch_amax(cd, sx, stream));
            p->launches += 1;
        }
    }
    if (st.kernel == K_TC) {
        const int si = (int)(&st - &p->steps[0]);
        if (prep) TN_CUDA(cudaEventRecord(prep->first, stream));
        for (int side = 0; side < 2; ++side) {
            const Planar &q = p->planars[side ? st.pb : st.pa];
            const Tensor &X = side ? B : A;
            if (q.direct) continue;  // written by its producer
            tn::ConvertDesc cd{};
            cd.src = arena + X.off;
            cd.dst = p->arena + q.off;
            cd.n = (int64_t)1 << X.rank();
            cd.src_sstride = X.dep ? cd.n : 0;
            const int64_t sx = X.dep ? slices : 1;
            cd.plane_stride = cd.n * (X.dep ? p->sb : 1);
            cd.dst_sstride = cd.n;
            cd.amax = p->meta + 2 * p->sb * q.meta;
            cd.exps = reinterpret_cast<int32_t *>(p->meta + 2 * p->sb * q.meta + p->sb);
            cd.dtype = operand_dtype(p->mode);
            cd.planes = q.planes;
            if (X.producer < 0) {  // a leaf: no producer epilogue recorded its max-abs
                TN_CUDA(cudaMemsetAsync(cd.amax, 0, sizeof(unsigned int) * sx, stream));
                TN_CUDA(tn::launch_amax(cd, sx, stream));
                p->launches += 1;
            }
            TN_CUDA(tn::launch_convert16(cd, sx, stream));
            p->launches += 1;
        }
        if (prep) TN_CUDA(cudaEventRecord(prep->second, stream));
        if (ev) TN_CUDA(cudaEventRecord(ev->first, stream));
        e = tn::launch_gemm_tc(p->tc_desc[si], slices, stream);
        if (ev) TN_CUDA(cudaEventRecord(ev->second, stream));
        p->launches += 1;
    } else if (st.kernel == K_STREAM) {
        // the operand with more free bits streams (one thread per row), the other is held in
        // shared memory; A * B = B * A, so the roles follow the sizes
        const bool swap = st.N.size() > st.M.size();
        const Tensor &R = swap ? B : A, &Q = swap ? A : B;
        const std::vector<int> &Rl = swap ? st.N : st.M, &Ql = swap ? st.M : st.N;
        tn::GemmDesc d{};
        d.A = arena + R.off;
        d.B = arena + Q.off;
        d.C = arena + C.off;
        d.sA = swap ? sB : sA;
        d.sB = swap ? sA : sB;
        d.sC = sC;
        d.lm = (int)Rl.size();
        d.ln = (int)Ql.size();
        d.lk = (int)st.K.size();
        d.splits = 1;
        d.amax_out = amax_out;
        if (st.direct_planar >= 0) {
            d.planar_out = 1;
            fill_planar_out(p, st, d.pout);
        }
        fill_pos(d.posC_m, TN_MAXR, -1);
        fill_pos(d.posC_n, TN_MAXR, -1);
        for (int i = 0; i < d.lm; ++i) d.posC_m[i] = (int8_t)C.pos(Rl[Rl.size() - 1 - i]);
        for (int i = 0; i < d.ln; ++i) d.posC_n[i] = (int8_t)C.pos(Ql[Ql.size() - 1 - i]);
        // tiles of 256 rows on the CUDA cores, of 128 rows on the tensor cores; C's three lowest
        // positions must lie in the tile (else the step stays on the CUDA cores)
        bool on_tc = st.thin_tc && !st.thin_tc_off;
        if (on_tc) {
            d.tile_bits = 7 + d.ln;
            tn::sort_tile_bits(7, d.ln, d.posC_m, d.posC_n, 128, d.tb_src, d.tb_pos);
            if (d.tb_pos[0] != 0 || d.tb_pos[1] != 1 || d.tb_pos[2] != 2) {
                st.thin_tc_off = true;
                on_tc = false;
            }
        }
        if (!on_tc) {
            d.tile_bits = 8 + d.ln;
            tn::sort_tile_bits(8, d.ln, d.posC_m, d.posC_n, 128, d.tb_src, d.tb_pos);
            if (d.tb_pos[0] != 0 || d.tb_pos[1] != 1 || d.tb_pos[2] != 2)
                return fail(TN_ERR_UNSUPPORTED, "step %d: result bits 0-2 outside the thin tile",
                            (int)(&st - &p->steps[0]));
        }
        if (on_tc && !st.thin_phi_set) {
            tn::thin_choose_swizzle(d.tb_src, d.ln, d.planar_out != 0, st.thin_phi);
            st.thin_phi_set = true;
        }
        memcpy(d.phi, st.thin_phi, sizeof d.phi);
        if (on_tc) {
            tn::ThinTcDesc td;
            memset(&td, 0, sizeof td);
            td.g = d;
            if (tn::encode_tmap_thin(&td.tmA, d.A, d.lm, d.lk, d.sA ? slices : 1) != 0)
                return fail(TN_ERR_CUDA, "step %d: tensor map of the thin operand",
                            (int)(&st - &p->steps[0]));
            if (ev) TN_CUDA(cudaEventRecord(ev->first, stream));
            e = tn::launch_gemm_thin_tc(td, slices, stream);
            if (ev) TN_CUDA(cudaEventRecord(ev->second, stream));
        } else {
            if (ev) TN_CUDA(cudaEventRecord(ev->first, stream));
            e = tn::launch_gemm_thin(d, slices, stream);
            if (ev) TN_CUDA(cudaEventRecord(ev->second, stream));
        }
        p->launches += 1;
    } else if (st.kernel == K_GEMM) {
        tn::GemmDesc d{};
        d.A = arena + A.off;
        d.B = arena + B.off;
        d.C = arena + C.off;
        d.sA = sA;
        d.sB = sB;
        d.sC = sC;
        d.lm = (int)st.M.size();
        d.ln = (int)st.N.size();
        d.lk = (int)st.K.size();
        d.splits = st.splits;
        d.partial = st.part_off >= 0 ? reinterpret_cast<float2 *>(p->arena + st.part_off) : nullptr;
        d.amax_out = amax_out;
        if (st.direct_planar >= 0) {
            d.planar_out = 1;
            fill_planar_out(p, st, d.pout);
        }
        fill_pos(d.posC_m, TN_MAXR, -1);
        fill_pos(d.posC_n, TN_MAXR, -1);
        for (int i = 0; i < d.lm; ++i) d.posC_m[i] = (int8_t)C.pos(st.M[st.M.size() - 1 - i]);
        for (int i = 0; i < d.ln; ++i) d.posC_n[i] = (int8_t)C.pos(st.N[st.N.size() - 1 - i]);
        {
            const int tm = std::min(d.lm, 6), tnb = std::min(d.ln, 6);
            d.tile_bits = tm + tnb;
            tn::sort_tile_bits(tm, tnb, d.posC_m, d.posC_n, 64, d.tb_src, d.tb_pos);
            // the staging index of row i, column j is 64 * i + j: row bit i is index bit 6 + i
            for (int q = 0; q < d.tile_bits; ++q)
                if (d.tb_src[q] & 64) d.tb_src[q] = (int8_t)(6 + (d.tb_src[q] & 63));
            if (d.tb_pos[0] != 0)
                return fail(TN_ERR_UNSUPPORTED, "step %d: result bit 0 outside the GEMM tile",
                            (int)(&st - &p->steps[0]));
        }
        if (ev) TN_CUDA(cudaEventRecord(ev->first, stream));
        e = tn::launch_gemm_simt(d, slices, stream);
        if (st.splits > 1) p->launches += 1;
        if (ev) TN_CUDA(cudaEventRecord(ev->second, stream));
        p->launches += 1;
    } else {
        const tn::GenericDesc d = make_generic_desc(p, st, amax_out);
        if (ev) TN_CUDA(cudaEventRecord(ev->first, stream));
        e = tn::launch_generic(d, slices, stream);
        if (ev) TN_CUDA(cudaEventRecord(ev->second, stream));
        p->launches += 1;
    }
    if (e != cudaSuccess)
        return fail(TN_ERR_CUDA, "step %d launch: %s", (int)(&st - &p->steps[0]),
                    cudaGetErrorString(e));
    return TN_OK;
}

}  // namespace

extern "C" {

tn_status tn_plan_get_info(const tn_plan_t *p, tn_plan_info *out) {
    g_err.clear();
    if (check_plan(p) != TN_OK) return TN_ERR_INVALID_ARG;
    if (!out) return fail(TN_ERR_INVALID_ARG, "out is NULL");
    memset(out, 0, sizeof *out);
    out->num_steps = (int64_t)p->steps.size();
    out->num_slices = p->num_slices;
    out->slices_in_flight = p->sb;
    out->workspace_bytes = p->arena_bytes;
    out->num_open = (int32_t)p->net->open.size();
    out->max_log2_size = p->max_log;
    for (auto &st : p->steps) {
        if (st.dep) {
            out->tcc_per_slice += st.tcc;
            out->tmc_per_slice += st.tmc;
        } else {
            out->tcc_invariant += st.tcc;
        }
        switch (st.kernel) {
            case K_TC: out->num_tc_steps++; break;
            case K_GEMM: out->num_gemm_steps++; break;
            case K_STREAM: out->num_stream_steps++; break;
            default: out->num_generic_steps++; break;
        }
    }
    out->kernel_launches = p->launches;
    tn_plan_t *mp = const_cast<tn_plan_t *>(p);
    for (auto &ev : mp->pending_bind) {
        float ms_ = 0.f;
        TN_CUDA(cudaEventSynchronize(ev.second));
        TN_CUDA(cudaEventElapsedTime(&ms_, ev.first, ev.second));
        mp->bind_ms += ms_;
        mp->bind_timed += 1;
        mp->event_pool.push_back(ev);
    }
    mp->pending_bind.clear();
    out->bind_ms = p->bind_ms;
    out->bind_launches = p->bind_timed;
    out->num_open_sliced = p->acc.nb;
    out->num_single_pass = p->single_pass;
    out->num_compensated = p->compensated;
    out->eps_predicted = p->eps_pred;
    return TN_OK;
}

tn_status tn_plan_get_step_info(const tn_plan_t *p, int64_t step, tn_step_info *out) {
    g_err.clear();
    if (check_plan(p) != TN_OK) return TN_ERR_INVALID_ARG;
    if (!out || step < 0 || step >= (int64_t)p->steps.size())
        return fail(TN_ERR_INVALID_ARG, "bad step index");
    const Step &st = p->steps[(size_t)step];
    memset(out, 0, sizeof *out);
    out->kernel = st.thin_tc && !st.thin_tc_off ? 4 : st.kernel;
    out->slice_dependent = st.dep ? 1 : 0;
    out->log2_m = (int)st.M.size();
    out->log2_n = (int)st.N.size();
    out->log2_k = (int)st.K.size();
    out->log2_batch = (int)st.batch.size();
    out->log2_a = (int)st.la.size();
    out->log2_b = (int)st.lb.size();
    out->log2_c = (int)st.lc.size();
    out->gemm_form = st.kernel == K_TC ? st.form : 0;
    out->tc_variant = st.kernel == K_TC ? st.variant : -1;
    {
        // sorted chunk bits that are C's lowest positions: 0, 1, 2, ...
        const Tensor &C = p->tensors[st.c];
        int8_t pm[TN_MAXR], pn[TN_MAXR], src[32], pos[32];
        const std::vector<int> *Ms = &st.M, *Ns = &st.N;
        int tm = 0, tn_ = 0;
        if (st.kernel == K_TC) {
            tm = 7;
            tn_ = 6;
        } else if (st.kernel == K_GEMM) {
            tm = std::min((int)st.M.size(), 6);
            tn_ = std::min((int)st.N.size(), 6);
        } else if (st.kernel == K_STREAM) {
            if (st.N.size() > st.M.size()) std::swap(Ms, Ns);
            tm = st.thin_tc && !st.thin_tc_off ? 7 : 8;
            tn_ = (int)Ns->size();
        }
        int run = 0;
        if (tm + tn_ > 0) {
            for (int i = 0; i < (int)Ms->size(); ++i) pm[i] = (int8_t)C.pos((*Ms)[Ms->size() - 1 - i]);
            for (int i = 0; i < (int)Ns->size(); ++i) pn[i] = (int8_t)C.pos((*Ns)[Ns->size() - 1 - i]);
            tn::sort_tile_bits(tm, tn_, pm, pn, 64, src, pos);
            while (run < tm + tn_ && pos[run] == run) run++;
        } else {
            run = std::min(C.rank(), 10);  // element-wise kernel: consecutive threads, C order
        }
        out->store_run_log2 = run;
    }
    {
        const Tensor &A = p->tensors[st.a], &B = p->tensors[st.b], &C = p->tensors[st.c];
        const double esz = tf32_mode(p->mode) ? 4.0 : 2.0;
        auto operand = [&](const Tensor &X, int planar) {
            const double n = std::ldexp(1.0, X.rank());
            if (st.kernel == K_TC && planar >= 0) return n * esz * p->planars[planar].planes;
            return n * 8.0;
        };
        double bytes = operand(A, st.kernel == K_TC ? st.pa : -1) +
                       operand(B, st.kernel == K_TC ? st.pb : -1);
        const double nc = std::ldexp(1.0, C.rank());
        bytes += st.direct_planar >= 0 ? nc * esz * p->planars[st.direct_planar].planes : nc * 8.0;
        out->tmc_bytes = bytes;
    }
    out->tcc = st.tcc;
    Step &ms = const_cast<Step &>(st);
    tn_plan_t *mp = const_cast<tn_plan_t *>(p);
    for (auto &ev : ms.pending) {
        float ms_ = 0.f;
        TN_CUDA(cudaEventSynchronize(ev.second));
        TN_CUDA(cudaEventElapsedTime(&ms_, ev.first, ev.second));
        ms.time_ms += ms_;
        ms.timed += 1;
        mp->event_pool.push_back(ev);
    }
    ms.pending.clear();
    for (auto &ev : ms.pending_prep) {
        float ms_ = 0.f;
        TN_CUDA(cudaEventSynchronize(ev.second));
        TN_CUDA(cudaEventElapsedTime(&ms_, ev.first, ev.second));
        ms.prep_ms += ms_;
        mp->event_pool.push_back(ev);
    }
    ms.pending_prep.clear();
    out->time_ms = st.time_ms;
    out->launches = st.timed;
    out->prep_ms = st.prep_ms;
    return TN_OK;
}

// FP64 sum of the ns slices in flight (ids s0..) into the amplitudes (Sec. 5: the answer is the
// sum of the sub-task results); with sliced open labels each slice goes to its own block.
static cudaError_t accumulate(tn_plan_t *p, const Tensor &R, int64_t nout, int64_t ns, int64_t s0,
                              void *amps_dev, cudaStream_t stream) {
    float2 *arena = reinterpret_cast<float2 *>(p->arena);
    double2 *amps = reinterpret_cast<double2 *>(amps_dev);
    if (p->acc.nb == 0)
        return tn::launch_accumulate(arena + R.off, R.dep ? nout : 0, nout, R.dep ? ns : 1, amps,
                                     stream);
    // a root that does not depend on the slice (possible only when nothing below it is sliced)
    // is still added once per slice: each slice id names its own block
    return tn::launch_accumulate_batched(arena + R.off, R.dep ? nout : 0, nout, ns, s0, p->acc,
                                         amps, stream);
}

tn_status tn_contract(tn_plan_t *p, int64_t slice_begin, int64_t slice_end, void *amps_dev,
                      void *stream_) {
    g_err.clear();
    if (check_plan(p) != TN_OK) return TN_ERR_INVALID_ARG;
    if (!amps_dev) return fail(TN_ERR_INVALID_ARG, "amps_dev is NULL");
    if (slice_begin < 0 || slice_end > p->num_slices || slice_begin > slice_end)
        return fail(TN_ERR_INVALID_ARG, "slice range [%lld, %lld) outside [0, %lld)",
                    (long long)slice_begin, (long long)slice_end, (long long)p->num_slices);
    cudaStream_t stream = (cudaStream_t)stream_;
    {
        cudaError_t pending = cudaPeekAtLastError();
        if (pending != cudaSuccess)
            return fail(TN_ERR_CUDA, "pending CUDA error: %s", cudaGetErrorString(pending));
    }
    if (slice_begin == slice_end) return TN_OK;
    int dev = 0;
    TN_CUDA(cudaGetDevice(&dev));
    if (dev != p->device) TN_CUDA(cudaSetDevice(p->device));
    float2 *arena = reinterpret_cast<float2 *>(p->arena);
    // prologue: slice-independent leaves and steps, once per call
    {
        tn_status s = bind_leaves(p, false, 0, 1, stream);
        if (s != TN_OK) return s;
    }
    for (auto &st : p->steps)
        if (!st.dep) {
            tn_status s = run_step(p, st, 1, stream);
            if (s != TN_OK) return s;
        }
    const Tensor &R = p->tensors[p->root];
    const int64_t nout = (int64_t)1 << R.rank();
    for (int64_t s0 = slice_begin; s0 < slice_end; s0 += p->sb) {
        const int64_t ns = std::min(p->sb, slice_end - s0);
        {
            tn_status s = bind_leaves(p, true, s0, ns, stream);
            if (s != TN_OK) return s;
        }
        if (p->opts.autotune && !p->tuned && ns == p->sb) {
            // first full batch: tune the tensor-core steps while running it
            for (auto &st : p->steps)
                if (st.dep) {
                    tn_status s = st.kernel == K_TC ? tune_tc_step(p, st, ns, stream)
                                                    : run_step(p, st, ns, stream);
                    if (s != TN_OK) return s;
                }
            p->tuned = true;
            TN_CUDA(accumulate(p, R, nout, ns, s0, amps_dev, stream));
            p->launches++;
            continue;
        }
        const bool graph = p->opts.use_graph && !p->opts.profile && ns == p->sb;
        if (graph && !p->graph_exec) {
            // capture the dependent steps once, on a plan-owned stream
            if (!p->cap_stream)
                TN_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
            const int64_t l0 = p->launches;
            TN_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
            tn_status cs = TN_OK;
            for (auto &st : p->steps)
                if (st.dep && cs == TN_OK) cs = run_step(p, st, ns, p->cap_stream);
            cudaGraph_t g = nullptr;
            cudaError_t ce = cudaStreamEndCapture(p->cap_stream, &g);
            if (cs != TN_OK) {
                if (g) cudaGraphDestroy(g);
                return cs;
            }
            if (ce != cudaSuccess) return fail(TN_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
            p->graph = g;
            TN_CUDA(cudaGraphInstantiate(&p->graph_exec, p->graph, 0));
            p->graph_launches = p->launches - l0;
            p->launches = l0;
        }
        if (graph) {
            TN_CUDA(cudaGraphLaunch(p->graph_exec, stream));
            p->launches += p->graph_launches;
        } else {
            for (auto &st : p->steps)
                if (st.dep) {
                    tn_status s = run_step(p, st, ns, stream);
                    if (s != TN_OK) return s;
                }
        }
        TN_CUDA(accumulate(p, R, nout, ns, s0, amps_dev, stream));
        p->launches++;
    }
    if (p->opts.sync_each_call) {
        TN_CUDA(cudaStreamSynchronize(stream));
        if (!p->planars.empty() && tn::tc_status_read_and_clear() != 0)
            return fail(TN_ERR_TIMEOUT, "a tensor-core kernel gave up a bounded wait");
    }
    if (dev != p->device) cudaSetDevice(dev);
    return TN_OK;
}

tn_status tn_contract_host(tn_plan_t *p, int64_t slice_begin, int64_t slice_end,
                           double *amps_host, void *stream_) {
    g_err.clear();
    if (check_plan(p) != TN_OK) return TN_ERR_INVALID_ARG;
    if (!amps_host) return fail(TN_ERR_INVALID_ARG, "amps_host is NULL");
    cudaStream_t stream = (cudaStream_t)stream_;
    const int64_t n = (int64_t)1 << p->net->open.size();
    TN_CUDA(tn::launch_zero_f64(p->amps_tmp, n, stream));
    tn_status s = tn_contract(p, slice_begin, slice_end, p->amps_tmp, stream_);
    if (s != TN_OK) return s;
    TN_CUDA(cudaMemcpyAsync(amps_host, p->amps_tmp, sizeof(double2) * (size_t)n,
                            cudaMemcpyDeviceToHost, stream));
    TN_CUDA(cudaStreamSynchronize(stream));
    if (!p->planars.empty() && tn::tc_status_read_and_clear() != 0)
        return fail(TN_ERR_TIMEOUT, "a tensor-core kernel gave up a bounded wait");
    return TN_OK;
}

tn_status tn_selftest_wait_timeout(int32_t limit_ms, void *stream) {
    g_err.clear();
    return tn::tc_selftest_wait_timeout(limit_ms, (cudaStream_t)stream);
}

tn_status tn_readout(const tn_plan_t *p, const void *amps_dev, int32_t n_qubits, double out[4],
                     void *stream_) {
    g_err.clear();
    if (check_plan(p) != TN_OK) return TN_ERR_INVALID_ARG;
    if (!amps_dev || !out || n_qubits < 0 || n_qubits > 1000)
        return fail(TN_ERR_INVALID_ARG, "bad readout arguments");
    cudaStream_t stream = (cudaStream_t)stream_;
    const int64_t m = (int64_t)1 << p->net->open.size();
    TN_CUDA(tn::launch_readout(reinterpret_cast<const double2 *>(amps_dev), m, p->partial,
                               p->n_partial, stream));
    double h[2];
    TN_CUDA(cudaMemcpyAsync(h, p->partial, sizeof h, cudaMemcpyDeviceToHost, stream));
    TN_CUDA(cudaStreamSynchronize(stream));
    const double D = std::ldexp(1.0, n_qubits);
    out[0] = h[0];
    out[1] = h[1];
    out[2] = D * h[0] / (double)m - 1.0;
    out[3] = h[0] > 0.0 ? D * h[1] / h[0] - 1.0 : 0.0;
    return TN_OK;
}

}  // extern "C"

extern "C" {

void tn_destroy(void *handle) {
    if (!handle) return;
    const uint32_t magic = *reinterpret_cast<const uint32_t *>(handle);
    if (magic == kNetMagic) {
        auto *n = reinterpret_cast<tn_network *>(handle);
        if (n->data) cudaFree(n->data);
        n->magic = 0;
        delete n;
    } else if (magic == tn::kSparseMagic) {
        tn::sparse_destroy(handle);
    } else if (magic == kPlanMagic) {
        auto *p = reinterpret_cast<tn_plan_t *>(handle);
        if (p->own_arena && p->arena) cudaFree(p->arena);
        if (p->bind_inv_dev) cudaFree(p->bind_inv_dev);
        if (p->bind_sl_dev) cudaFree(p->bind_sl_dev);
        if (p->chain_dev) cudaFree(p->chain_dev);
        if (p->meta) cudaFree(p->meta);
        if (p->partial) cudaFree(p->partial);
        if (p->amps_tmp) cudaFree(p->amps_tmp);
        for (auto &ev : p->pending_bind) p->event_pool.push_back(ev);
        for (auto &st : p->steps) {
            for (auto &ev : st.pending) p->event_pool.push_back(ev);
            for (auto &ev : st.pending_prep) p->event_pool.push_back(ev);
        }
        for (auto &ev : p->event_pool) {
            cudaEventDestroy(ev.first);
            cudaEventDestroy(ev.second);
        }
        if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
        if (p->graph) cudaGraphDestroy(p->graph);
        if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
        p->magic = 0;
        delete p;
    }
}

}  // extern "C"
