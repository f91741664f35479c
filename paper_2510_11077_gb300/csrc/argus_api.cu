// C ABI of the batched Kalman-filter likelihood (declared in include/argus.h).
//
// Host side only: validation, the device copy of the TOA data (the per-TOA
// pre-stage), the schedule (work items sorted by TOA count, persistent grid
// size, scratch slots), CUDA-graph capture and replay, and host-pointer
// staging.  Every arithmetic step of the likelihood runs in kf_kernels.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/argus.h"
#include "kf_few.cuh"
#include "kf_internal.cuh"
#include "kf_scan_grad.cuh"
#include "lib_internal.cuh"

using namespace argus;

namespace {

thread_local std::string g_last_error;

argus_status fail(argus_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

}  // namespace

// the last-error record shared by every entry point of the library
int argus::record_error(int status, const char* msg) {
    g_last_error = msg ? msg : "";
    return status;
}

// Host validation of pulsar data shared by every handle constructor: sorted
// finite TOAs, positive errors, unit positions, EQUAD >= 0, a positive
// semi-definite prior.  Returns ARGUS_OK and the TOA count, or the status.
int argus::validate_pulsars(const argus_pulsar* psrs, int32_t n_pulsars, int64_t* total_out) {
    int64_t total = 0;
    for (int p = 0; p < n_pulsars; ++p) {
        const argus_pulsar& ps = psrs[p];
        char buf[160];
        if (ps.n_toa < 0 || ps.n_toa > INT32_MAX) {
            snprintf(buf, sizeof buf, "pulsar %d: n_toa out of range", p);
            return fail(ARGUS_ERR_INVALID_ARG, buf);
        }
        if (ps.n_toa > 0 && (!ps.t || !ps.r || !ps.sigma)) {
            snprintf(buf, sizeof buf, "pulsar %d: NULL data", p);
            return fail(ARGUS_ERR_INVALID_ARG, buf);
        }
        for (int64_t k = 0; k < ps.n_toa; ++k) {
            if (!std::isfinite(ps.t[k]) || !std::isfinite(ps.r[k]) || !std::isfinite(ps.sigma[k]) ||
                !(ps.sigma[k] > 0.0) || (k > 0 && ps.t[k] < ps.t[k - 1])) {
                snprintf(buf, sizeof buf, "pulsar %d TOA %lld: non-finite, unsorted or sigma <= 0", p,
                         (long long)k);
                return fail(ARGUS_ERR_INVALID_ARG, buf);
            }
        }
        const double nrm = std::sqrt(ps.pos[0] * ps.pos[0] + ps.pos[1] * ps.pos[1] + ps.pos[2] * ps.pos[2]);
        if (!(std::fabs(nrm - 1.0) <= 1e-6)) {
            snprintf(buf, sizeof buf, "pulsar %d: position is not a unit vector", p);
            return fail(ARGUS_ERR_INVALID_ARG, buf);
        }
        if (!(ps.equad >= 0.0) || !std::isfinite(ps.equad)) {
            snprintf(buf, sizeof buf, "pulsar %d: EQUAD must be finite and >= 0", p);
            return fail(ARGUS_ERR_INVALID_ARG, buf);
        }
        if (!(ps.p0[0] >= 0.0 && ps.p0[2] >= 0.0 && ps.p0[0] * ps.p0[2] >= ps.p0[1] * ps.p0[1]) ||
            !std::isfinite(ps.p0[1])) {
            snprintf(buf, sizeof buf, "pulsar %d: prior covariance is not positive semi-definite", p);
            return fail(ARGUS_ERR_INVALID_ARG, buf);
        }
        total += ps.n_toa;
    }
    *total_out = total;
    return ARGUS_OK;
}

namespace {

argus_status cuda_fail(cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(e == cudaErrorMemoryAllocation ? ARGUS_ERR_OOM : ARGUS_ERR_CUDA, m);
}

#define CK(call)                                         \
    do {                                                 \
        cudaError_t _e = (call);                         \
        if (_e != cudaSuccess) return cuda_fail(_e, #call); \
    } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <class T>
argus_status grow(T** p, size_t* cap, size_t need) {
    if (need <= *cap && *p) return ARGUS_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (need == 0) return ARGUS_OK;
    CK(cudaMalloc(reinterpret_cast<void**>(p), need * sizeof(T)));
    *cap = need;
    return ARGUS_OK;
}

struct GraphKey {
    const double* theta;
    int64_t B;
    double* ll;
    double* grad;
    double* lane;
    bool operator==(const GraphKey& o) const {
        return theta == o.theta && B == o.B && ll == o.ll && grad == o.grad && lane == o.lane;
    }
};

struct GraphEntry {
    GraphKey key;
    cudaGraphExec_t exec;
    uint64_t last_use;
};

constexpr int kMaxGraphs = 8;

}  // namespace

struct argus_array {
    int device = 0;
    int n_sm = 0;
    int P = 0;
    int32_t model = kRandomWalk;   // red-noise model (argus.h: ARGUS_NOISE_*)
    int32_t flags = 0;             // kFlagOU | kFlagPulsarTerm (argus.h model flags)
    int32_t nq = 2;                // parameters per pulsar
    int64_t total_toa = 0;
    int32_t stride_max = 1;   // for the current plan
    int32_t nseg_max = 0;
    int32_t n_max = 0;        // most TOAs of any pulsar
    std::vector<PulsarDev> h_psr;
    PulsarDev* d_psr = nullptr;
    double* d_rec = nullptr;
    argus_plan plan{};
    // per-batch buffers
    double* d_lc = nullptr;        size_t cap_lc = 0;
    double* d_lane = nullptr;      size_t cap_lane = 0;
    WorkItem* d_items = nullptr;   size_t cap_items = 0;
    int64_t items_B = -1;
    int items_W = 0;
    int n_items = 0;
    // adjoint scratch, one slot per resident block of the persistent grid
    double* d_ckpt = nullptr;      size_t cap_ckpt = 0;
    double* d_tape = nullptr;      size_t cap_tape = 0;
    int* d_counter = nullptr;
    int* d_any2 = nullptr;         // host-pointer calls: some walker's filter met a bad variance
    // time-parallel filter (ARGUS_MODE_SCAN)
    ScanItem* d_sitems = nullptr;  size_t cap_sitems = 0;
    int32_t* d_lane_first = nullptr; size_t cap_lane_first = 0;
    double* d_tpre = nullptr;      size_t cap_tpre = 0;
    double* d_bagg = nullptr;      size_t cap_bagg = 0;
    double* d_bpre = nullptr;      size_t cap_bpre = 0;
    double* d_part = nullptr;      size_t cap_part = 0;
    int64_t scan_B = -1;
    int32_t scan_E = 0;
    int32_t n_sitems = 0;
    double* d_phase_tab = nullptr;
    // time-parallel adjoint (ARGUS_MODE_SCAN with a gradient)
    double* d_stape = nullptr;     size_t cap_stape = 0;
    double* d_tsuf = nullptr;      size_t cap_tsuf = 0;
    double* d_ragg = nullptr;      size_t cap_ragg = 0;
    double* d_rpre = nullptr;      size_t cap_rpre = 0;
    double* d_partg = nullptr;     size_t cap_partg = 0;
    unsigned long long* d_rdone = nullptr; size_t cap_rdone = 0;
    // host staging
    double* d_stage = nullptr;     size_t cap_stage = 0;
    // graphs
    cudaStream_t cap_stream = nullptr;
    std::vector<GraphEntry> graphs;
    uint64_t use_clock = 0;
    // stage timing (argus_array_set_timing)
    bool timing = false;
    bool timed_once = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace {

void drop_graphs(argus_array* h) {
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
}

argus_plan default_plan() {
    argus_plan p{};
    p.mode = ARGUS_MODE_BATCHED;
    p.walkers_per_cta = 128;
    p.ctas_per_sm = 4;
    p.ckpt_stride = 0;
    p.use_graph = 1;
    return p;
}

argus_status validate_plan(const argus_plan* p) {
    if (!p) return fail(ARGUS_ERR_INVALID_ARG, "plan is NULL");
    if (p->mode != ARGUS_MODE_BATCHED && p->mode != ARGUS_MODE_PLAIN && p->mode != ARGUS_MODE_SCAN)
        return fail(ARGUS_ERR_INVALID_ARG, "plan.mode must be BATCHED, PLAIN or SCAN");
    const int w = p->walkers_per_cta;
    if (w != 32 && w != 64 && w != 128 && w != 256)
        return fail(ARGUS_ERR_INVALID_ARG, "plan.walkers_per_cta must be 32, 64, 128 or 256");
    if (p->ctas_per_sm < 1 || p->ctas_per_sm > 16)
        return fail(ARGUS_ERR_INVALID_ARG, "plan.ctas_per_sm must be in 1..16");
    if (p->ckpt_stride < 0 || p->ckpt_stride > kMaxStride)
        return fail(ARGUS_ERR_INVALID_ARG, "plan.ckpt_stride must be in 0..256");
    if (p->use_graph != 0 && p->use_graph != 1)
        return fail(ARGUS_ERR_INVALID_ARG, "plan.use_graph must be 0 or 1");
    if (p->tape_cache != 0 && p->tape_cache != 1)
        return fail(ARGUS_ERR_INVALID_ARG, "plan.tape_cache must be 0 or 1");
    if (p->scan_elems < 0 || p->scan_elems > 4096)
        return fail(ARGUS_ERR_INVALID_ARG, "plan.scan_elems must be in 0..4096");
    if (p->reserved != 0) return fail(ARGUS_ERR_INVALID_ARG, "plan.reserved must be 0");
    return ARGUS_OK;
}

// Segment length of the adjoint for a pulsar with n TOAs.
int stride_for(int64_t n, int ckpt_stride) {
    int c = ckpt_stride;
    if (c == 0) c = int(std::ceil(std::sqrt(double(std::max<int64_t>(n, 1)))));
    return std::max(1, std::min(c, kMaxStride));
}

// Re-derive per-pulsar strides for the plan and upload the pulsar table.
argus_status apply_plan(argus_array* h) {
    h->stride_max = 1;
    h->nseg_max = 0;
    h->n_max = 0;
    for (auto& ps : h->h_psr) {
        h->n_max = std::max(h->n_max, ps.n);
        ps.stride = stride_for(ps.n, h->plan.ckpt_stride);
        ps.nseg = int((ps.n + ps.stride - 1) / ps.stride);
        h->stride_max = std::max(h->stride_max, ps.stride);
        h->nseg_max = std::max(h->nseg_max, ps.nseg);
    }
    CK(cudaMemcpy(h->d_psr, h->h_psr.data(), sizeof(PulsarDev) * h->P, cudaMemcpyHostToDevice));
    drop_graphs(h);
    h->items_B = -1;
    h->scan_B = -1;
    // the adjoint scratch is sized by the plan (blocks x walkers x segment or
    // tape length): release it so a new plan allocates what it needs rather
    // than keeping the largest buffer any earlier plan used
    cudaFree(h->d_ckpt);
    cudaFree(h->d_tape);
    h->d_ckpt = nullptr;
    h->d_tape = nullptr;
    h->cap_ckpt = 0;
    h->cap_tape = 0;
    return ARGUS_OK;
}

// Work items (pulsar, walker tile), pulsars with the most TOAs first.
argus_status ensure_items(argus_array* h, int64_t B, int W) {
    if (h->items_B == B && h->items_W == W) return ARGUS_OK;
    std::vector<int> order(h->P);
    for (int p = 0; p < h->P; ++p) order[p] = p;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return h->h_psr[a].n > h->h_psr[b].n; });
    std::vector<WorkItem> items;
    const int64_t tiles = (B + W - 1) / W;
    items.reserve(size_t(tiles) * h->P);
    for (int p : order)
        for (int64_t t = 0; t < tiles; ++t) items.push_back(WorkItem{p, int32_t(t * W)});
    if (items.size() > size_t(INT32_MAX)) return fail(ARGUS_ERR_UNSUPPORTED, "too many work items");
    argus_status st = grow(&h->d_items, &h->cap_items, items.size());
    if (st) return st;
    if (!items.empty())
        CK(cudaMemcpy(h->d_items, items.data(), sizeof(WorkItem) * items.size(),
                      cudaMemcpyHostToDevice));
    h->n_items = int(items.size());
    h->items_B = B;
    h->items_W = W;
    drop_graphs(h);
    return ARGUS_OK;
}

int grid_for(const argus_array* h, int n_items) {
    const int g = h->n_sm * h->plan.ctas_per_sm;
    return std::max(1, std::min(g, n_items));
}

// Buffers for a batch of B walkers; reallocation invalidates captured graphs.
argus_status ensure_batch(argus_array* h, int64_t B, int W, int grid, bool grad) {
    const size_t lanes = size_t(B) * h->P;
    void* before[4] = {h->d_lc, h->d_lane, h->d_ckpt, h->d_tape};
    argus_status st;
    if ((st = grow(&h->d_lc, &h->cap_lc, lanes * kLaneConsts))) return st;
    if ((st = grow(&h->d_lane, &h->cap_lane, lanes * (1 + kLaneGrads)))) return st;
    if (grad) {
        // the cached tape needs no checkpoints (K3 writes none with it)
        const size_t ck = h->plan.tape_cache ? 1 : size_t(h->nseg_max) * kCkptDoubles * W * grid;
        const size_t tp_len = h->plan.tape_cache ? size_t(std::max(h->n_max, 1)) : size_t(h->stride_max);
        const size_t tp = tp_len * tape_doubles(h->model) * W * grid;
        if ((st = grow(&h->d_ckpt, &h->cap_ckpt, std::max<size_t>(ck, 1)))) return st;
        if ((st = grow(&h->d_tape, &h->cap_tape, std::max<size_t>(tp, 1)))) return st;
    }
    void* after[4] = {h->d_lc, h->d_lane, h->d_ckpt, h->d_tape};
    if (memcmp(before, after, sizeof(before)) != 0) drop_graphs(h);
    return ARGUS_OK;
}

FilterArgs make_args(argus_array* h, int64_t B, int W, int grid, bool persistent) {
    FilterArgs a{};
    a.rec = h->d_rec;
    a.psr = h->d_psr;
    a.items = h->d_items;
    a.n_items = h->n_items;
    a.P = h->P;
    a.B = B;
    a.lc = h->d_lc;
    a.lane_out = h->d_lane;
    a.ckpt = h->d_ckpt;
    a.tape = h->d_tape;
    a.ckpt_slot = int64_t(h->nseg_max) * kCkptDoubles * W;
    const int64_t tp_len = h->plan.tape_cache ? std::max(h->n_max, 1) : h->stride_max;
    a.tape_slot = tp_len * tape_doubles(h->model) * W;
    a.stride_max = h->stride_max;
    a.tape_cache = h->plan.tape_cache;
    a.counter = persistent ? h->d_counter : nullptr;
    a.model = h->model;
    (void)grid;
    return a;
}

// Chunks of the time-parallel filter for a batch of B walkers: lanes in
// lane_out order (p * B + b), each cut into chunks of 32 E TOAs.
argus_status ensure_scan(argus_array* h, int64_t B) {
    int64_t E = h->plan.scan_elems;
    if (E == 0) {
        const int64_t work = B * h->total_toa;
        const int64_t warps = int64_t(std::max(h->n_sm, 1)) * 4;
        E = std::max<int64_t>(1, (work + 32 * warps - 1) / (32 * warps));
        // no more TOAs per thread than the longest pulsar spreads over one
        // chunk's 32 threads: a larger E only pads every chunk (and the
        // adjoint's tape) with idle threads
        E = std::min<int64_t>(E, std::max<int64_t>(1, (int64_t(h->n_max) + 31) / 32));
        E = std::min<int64_t>(E, 4096);
    }
    if (h->scan_B == B && h->scan_E == E) return ARGUS_OK;
    const int64_t lanes = B * h->P;
    std::vector<ScanItem> items;
    std::vector<int32_t> first(size_t(lanes) + 1, 0);
    const int64_t chunk = 32 * E;
    for (int p = 0; p < h->P; ++p) {
        const int64_t n = h->h_psr[p].n;
        for (int64_t b = 0; b < B; ++b) {
            const int64_t lane = int64_t(p) * B + b;
            first[lane] = int32_t(items.size());
            for (int64_t k0 = 0; k0 < n; k0 += chunk) {
                if (items.size() >= size_t(INT32_MAX / 32))
                    return fail(ARGUS_ERR_UNSUPPORTED, "too many scan chunks: use a batched plan");
                items.push_back(ScanItem{int32_t(lane), int32_t(k0)});
            }
        }
    }
    first[lanes] = int32_t(items.size());
    const size_t ni = std::max<size_t>(items.size(), 1);
    argus_status st;
    if ((st = grow(&h->d_sitems, &h->cap_sitems, ni))) return st;
    if ((st = grow(&h->d_lane_first, &h->cap_lane_first, first.size()))) return st;
    if ((st = grow(&h->d_tpre, &h->cap_tpre, ni * 32 * kScanElem))) return st;
    if ((st = grow(&h->d_bagg, &h->cap_bagg, ni * kScanElem))) return st;
    if ((st = grow(&h->d_bpre, &h->cap_bpre, ni * kScanElem))) return st;
    // chunk sums [ni][2], then one 8-byte counter per lane (kf_scan.cu's S3
    // finds the lane's last chunk with it)
    if ((st = grow(&h->d_part, &h->cap_part, ni * 2 + size_t(lanes)))) return st;
    if (!items.empty())
        CK(cudaMemcpy(h->d_sitems, items.data(), sizeof(ScanItem) * items.size(),
                      cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_lane_first, first.data(), sizeof(int32_t) * first.size(),
                  cudaMemcpyHostToDevice));
    h->n_sitems = int32_t(items.size());
    h->scan_B = B;
    h->scan_E = int32_t(E);
    drop_graphs(h);
    return ARGUS_OK;
}

// Scratch of the time-parallel adjoint for the current chunking (after
// ensure_scan); reallocation invalidates captured graphs.
argus_status ensure_scan_grad(argus_array* h, int64_t B) {
    const size_t ni = std::max<size_t>(size_t(h->n_sitems), 1);
    const size_t lanes = std::max<size_t>(size_t(B) * h->P, 1);
    const size_t tape = ni * 32 * size_t(h->scan_E) * size_t(scan_tape_doubles(h->model));
    void* before[6] = {h->d_stape, h->d_tsuf, h->d_ragg, h->d_rpre, h->d_partg, h->d_rdone};
    argus_status st;
    if ((st = grow(&h->d_stape, &h->cap_stape, tape))) return st;
    if ((st = grow(&h->d_tsuf, &h->cap_tsuf, ni * 32 * kAdjElem))) return st;
    if ((st = grow(&h->d_ragg, &h->cap_ragg, ni * kAdjElem))) return st;
    if ((st = grow(&h->d_rpre, &h->cap_rpre, ni * kAdjElem))) return st;
    if ((st = grow(&h->d_partg, &h->cap_partg, ni * kLaneGrads))) return st;
    if ((st = grow(&h->d_rdone, &h->cap_rdone, lanes))) return st;
    void* after[6] = {h->d_stape, h->d_tsuf, h->d_ragg, h->d_rpre, h->d_partg, h->d_rdone};
    if (memcmp(before, after, sizeof(before)) != 0) drop_graphs(h);
    return ARGUS_OK;
}

// Enqueue one time-parallel evaluation: K1 -> S1..S3 (and, with a gradient,
// G3, R2, R3 in place of S3) -> K4.
argus_status enqueue_scan(argus_array* h, const double* theta, int64_t B, double* ll, double* grad,
                          double* lane, cudaStream_t s) {
    // a few walkers: K1 and K4 with one block of four warps per walker
    const bool few = few_walkers(B, h->P);
    if (h->timing) CK(cudaEventRecordWithFlags(h->ev[0], s, cudaEventRecordExternal));
    if (few) launch_project_few(theta, B, h->P, h->flags, h->d_psr, h->d_lc, s);
    else launch_project(theta, B, h->P, h->flags, h->d_psr, h->d_lc, s);
    if (h->timing) CK(cudaEventRecordWithFlags(h->ev[1], s, cudaEventRecordExternal));
    ScanArgs a{};
    a.rec = h->d_rec;
    a.psr = h->d_psr;
    a.lc = h->d_lc;
    a.P = h->P;
    a.B = B;
    a.items = h->d_sitems;
    a.n_items = h->n_sitems;
    a.E = h->scan_E;
    a.lane_first = h->d_lane_first;
    a.tpre = h->d_tpre;
    a.bagg = h->d_bagg;
    a.bpre = h->d_bpre;
    a.part = h->d_part;
    a.lane_out = h->d_lane;
    a.phase_table = h->d_phase_tab;
    a.model = h->model;
    if (grad) {
        ScanGradArgs g{};
        g.s = a;
        g.tape = h->d_stape;
        g.tsuf = h->d_tsuf;
        g.ragg = h->d_ragg;
        g.rpre = h->d_rpre;
        g.partg = h->d_partg;
        g.rdone = h->d_rdone;
        launch_filter_scan_grad(g, s);
    } else {
        launch_filter_scan(a, s);
    }
    if (h->timing) CK(cudaEventRecordWithFlags(h->ev[2], s, cudaEventRecordExternal));
    if (few && grad) launch_reduce_few(theta, B, h->P, h->flags, h->d_psr, h->d_lane, ll, grad, lane, s);
    else launch_reduce(theta, B, h->P, h->flags, h->d_psr, h->d_lane, ll, grad, lane, s);
    if (h->timing) {
        CK(cudaEventRecordWithFlags(h->ev[3], s, cudaEventRecordExternal));
        h->timed_once = true;
    }
    CK(cudaGetLastError());
    return ARGUS_OK;
}

// Enqueue one batched evaluation: K1 -> K2 or K3 -> K4.
argus_status enqueue_batched(argus_array* h, const double* theta, int64_t B, double* ll,
                             double* grad, double* lane, cudaStream_t s) {
    const bool want_grad = grad != nullptr;
    const int W = h->plan.walkers_per_cta;
    const int grid = grid_for(h, h->n_items);
    CK(cudaMemsetAsync(h->d_counter, 0, sizeof(int), s));
    if (h->timing) CK(cudaEventRecordWithFlags(h->ev[0], s, cudaEventRecordExternal));
    launch_project(theta, B, h->P, h->flags, h->d_psr, h->d_lc, s);
    if (h->timing) CK(cudaEventRecordWithFlags(h->ev[1], s, cudaEventRecordExternal));
    FilterArgs a = make_args(h, B, W, grid, true);
    if (want_grad) launch_filter_grad(a, W, grid, s);
    else launch_filter_fwd(a, W, grid, s);
    if (h->timing) CK(cudaEventRecordWithFlags(h->ev[2], s, cudaEventRecordExternal));
    launch_reduce(theta, B, h->P, h->flags, h->d_psr, h->d_lane, ll, grad, lane, s);
    if (h->timing) {
        CK(cudaEventRecordWithFlags(h->ev[3], s, cudaEventRecordExternal));
        h->timed_once = true;
    }
    CK(cudaGetLastError());
    return ARGUS_OK;
}

argus_status run_batched(argus_array* h, const double* theta, int64_t B, double* ll, double* grad,
                         double* lane, cudaStream_t s) {
    const int W = h->plan.walkers_per_cta;
    const bool scan = h->plan.mode == ARGUS_MODE_SCAN;
    argus_status st;
    if (scan) {
        if ((st = ensure_batch(h, B, W, 1, false))) return st;
        if ((st = ensure_scan(h, B))) return st;
        if (grad && (st = ensure_scan_grad(h, B))) return st;
    } else {
        if ((st = ensure_items(h, B, W))) return st;
        const int grid = grid_for(h, h->n_items);
        if ((st = ensure_batch(h, B, W, grid, grad != nullptr))) return st;
    }
    auto enqueue = [&](cudaStream_t st_) {
        return scan ? enqueue_scan(h, theta, B, ll, grad, lane, st_)
                    : enqueue_batched(h, theta, B, ll, grad, lane, st_);
    };
    if (!h->plan.use_graph) return enqueue(s);

    GraphKey key{theta, B, ll, grad, lane};
    for (auto& g : h->graphs) {
        if (g.key == key) {
            g.last_use = ++h->use_clock;
            CK(cudaGraphLaunch(g.exec, s));
            return ARGUS_OK;
        }
    }
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    st = enqueue(h->cap_stream);
    cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &graph);
    if (st) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate");
    if (int(h->graphs.size()) >= kMaxGraphs) {
        auto old = std::min_element(h->graphs.begin(), h->graphs.end(),
                                    [](const GraphEntry& a, const GraphEntry& b) {
                                        return a.last_use < b.last_use;
                                    });
        cudaGraphExecDestroy(old->exec);
        h->graphs.erase(old);
    }
    h->graphs.push_back(GraphEntry{key, exec, ++h->use_clock});
    CK(cudaGraphLaunch(exec, s));
    return ARGUS_OK;
}

// The comparison point: the same kernels, one parameter vector per launch.
argus_status run_plain(argus_array* h, const double* theta, int64_t B, double* ll, double* grad,
                       double* lane, cudaStream_t s) {
    const int W = 32;
    const int D = kNgw + h->nq * h->P;
    argus_status st;
    if ((st = ensure_items(h, 1, W))) return st;
    const int grid = h->n_items;
    if ((st = ensure_batch(h, 1, W, grid, grad != nullptr))) return st;
    FilterArgs a = make_args(h, 1, W, grid, false);
    for (int64_t b = 0; b < B; ++b) {
        const double* th = theta + b * D;
        launch_project(th, 1, h->P, h->flags, h->d_psr, h->d_lc, s);
        if (grad) launch_filter_grad(a, W, grid, s);
        else launch_filter_fwd(a, W, grid, s);
        launch_reduce(th, 1, h->P, h->flags, h->d_psr, h->d_lane, ll ? ll + b : nullptr,
                      grad ? grad + b * D : nullptr, lane ? lane + b * h->P : nullptr, s);
    }
    CK(cudaGetLastError());
    return ARGUS_OK;
}

bool is_device_ptr(const void* p) {
    if (!p) return true;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();   // clear the sticky-free error of an unknown pointer
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Evaluate with any mix of host and device pointers.
argus_status evaluate(argus_array* h, const double* theta, int64_t B, double* ll, double* grad,
                      double* lane, void* stream) {
    if (!h) return fail(ARGUS_ERR_INVALID_ARG, "array handle is NULL");
    if (B < 0) return fail(ARGUS_ERR_INVALID_ARG, "B must be >= 0");
    if (B == 0) return ARGUS_OK;
    if (!theta) return fail(ARGUS_ERR_INVALID_ARG, "theta is NULL");
    if (B > (int64_t(1) << 31) / std::max(1, h->P))
        return fail(ARGUS_ERR_UNSUPPORTED, "B x P exceeds 2^31 lanes");
    DeviceGuard guard(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int D = kNgw + h->nq * h->P;
    const bool dev_in = is_device_ptr(theta);
    const bool dev_ll = is_device_ptr(ll), dev_g = is_device_ptr(grad), dev_l = is_device_ptr(lane);
    const bool staged = !(dev_in && dev_ll && dev_g && dev_l);
    const double* th_d = theta;
    double *ll_d = ll, *g_d = grad, *lane_d = lane;
    if (staged) {
        const size_t need = size_t(B) * (2 * D + 1 + h->P);
        argus_status st = grow(&h->d_stage, &h->cap_stage, need);
        if (st) return st;
        double* base = h->d_stage;
        if (!dev_in) {
            CK(cudaMemcpyAsync(base, theta, sizeof(double) * B * D, cudaMemcpyHostToDevice, s));
            th_d = base;
        }
        base += size_t(B) * D;
        if (ll && !dev_ll) ll_d = base;
        base += B;
        if (grad && !dev_g) g_d = base;
        base += size_t(B) * D;
        if (lane && !dev_l) lane_d = base;
    }
    argus_status st = (h->plan.mode == ARGUS_MODE_PLAIN)
                          ? run_plain(h, th_d, B, ll_d, g_d, lane_d, s)
                          : run_batched(h, th_d, B, ll_d, g_d, lane_d, s);
    if (st) return st;
    if (staged) {
        // a synchronous call can report the filter's numerical failures as a status
        int any2 = 0;
        const bool report = ll != nullptr;
        if (report) {
            CK(cudaMemsetAsync(h->d_any2, 0, sizeof(int), s));
            launch_walker_flags(th_d, B, h->P, h->flags, ll_d, nullptr, h->d_any2, s);
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(&any2, h->d_any2, sizeof(int), cudaMemcpyDeviceToHost, s));
        }
        if (ll && !dev_ll)
            CK(cudaMemcpyAsync(ll, ll_d, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
        if (grad && !dev_g)
            CK(cudaMemcpyAsync(grad, g_d, sizeof(double) * B * D, cudaMemcpyDeviceToHost, s));
        if (lane && !dev_l)
            CK(cudaMemcpyAsync(lane, lane_d, sizeof(double) * B * h->P, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (any2)
            return fail(ARGUS_ERR_NONFINITE,
                        "a walker's filter met an innovation variance that is not a positive normal "
                        "finite number: its loglik is -inf and its gradient 0; the other walkers' "
                        "results are valid");
    }
    return ARGUS_OK;
}

}  // namespace

extern "C" {

argus_status argus_array_create(const argus_pulsar* psrs, int32_t n_pulsars, int32_t device,
                                argus_array** out) {
    return argus_array_create_ex(psrs, n_pulsars, device, ARGUS_NOISE_RANDOM_WALK, out);
}

argus_status argus_array_create_ex(const argus_pulsar* psrs, int32_t n_pulsars, int32_t device,
                                   int32_t model, argus_array** out) {
    if (!out) return fail(ARGUS_ERR_INVALID_ARG, "out is NULL");
    if ((model & ~int32_t(ARGUS_NOISE_OU | ARGUS_PULSAR_TERM)) != 0)
        return fail(ARGUS_ERR_INVALID_ARG,
                    "model must be ARGUS_NOISE_RANDOM_WALK or ARGUS_NOISE_OU, optionally | ARGUS_PULSAR_TERM");
    if (!psrs || n_pulsars < 1) return fail(ARGUS_ERR_INVALID_ARG, "need at least one pulsar");
    if (device < 0) return fail(ARGUS_ERR_INVALID_ARG, "device must be >= 0");
    int64_t total = 0;
    if (argus_status st = argus_status(validate_pulsars(psrs, n_pulsars, &total))) return st;
    // host validation is complete; now the device
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device >= ndev) return fail(ARGUS_ERR_INVALID_ARG, "no such device");
    cudaDeviceProp prop{};
    CK(cudaGetDeviceProperties(&prop, device));
    if (prop.major != 10 || prop.minor != 3)
        return fail(ARGUS_ERR_UNSUPPORTED, std::string("built for sm_103a, device is ") + prop.name);

    DeviceGuard guard(device);
    argus_array* h = new argus_array();
    h->device = device;
    h->n_sm = prop.multiProcessorCount;
    h->P = n_pulsars;
    h->model = (model & ARGUS_NOISE_OU) ? kOrnsteinUhlenbeck : kRandomWalk;
    h->flags = ((model & ARGUS_NOISE_OU) ? kFlagOU : 0) | ((model & ARGUS_PULSAR_TERM) ? kFlagPulsarTerm : 0);
    h->nq = params_per_pulsar(h->flags);
    h->total_toa = total;
    h->plan = default_plan();
    h->h_psr.resize(n_pulsars);

    // A0 pre-stage: per-TOA records [t, dt, dt^2/2, dt^3/3, r, sigma^2, dt^2, 2 dt]
    std::vector<double> rec(size_t(std::max<int64_t>(total, 1)) * kRecDoubles, 0.0);
    int64_t off = 0;
    for (int p = 0; p < n_pulsars; ++p) {
        const argus_pulsar& ps = psrs[p];
        PulsarDev& d = h->h_psr[p];
        d.off = off;
        d.n = int32_t(ps.n_toa);
        for (int i = 0; i < 3; ++i) d.pos[i] = ps.pos[i];
        d.equad2 = ps.equad * ps.equad;
        for (int i = 0; i < 3; ++i) d.p0[i] = ps.p0[i];
        for (int64_t k = 0; k < ps.n_toa; ++k) {
            double* q = rec.data() + (off + k) * kRecDoubles;
            const double dt = (k == 0) ? 0.0 : ps.t[k] - ps.t[k - 1];
            q[0] = ps.t[k];
            q[1] = dt;
            q[2] = dt * dt / 2.0;
            q[3] = dt * dt * dt / 3.0;
            q[4] = ps.r[k];
            q[5] = ps.sigma[k] * ps.sigma[k];
            q[6] = dt * dt;
            q[7] = 2.0 * dt;
        }
        off += ps.n_toa;
    }
    auto cleanup = [&](argus_status st) {
        argus_array_destroy(h);
        return st;
    };
    cudaError_t e;
    // (one record's room even for an array without TOAs: no kernel reads it then)
    if ((e = cudaMalloc(&h->d_rec, std::max<size_t>(rec.size(), kRecDoubles) * sizeof(double))) !=
        cudaSuccess)
        return cleanup(cuda_fail(e, "cudaMalloc(records)"));
    if (!rec.empty() &&
        (e = cudaMemcpy(h->d_rec, rec.data(), rec.size() * sizeof(double), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
        return cleanup(cuda_fail(e, "cudaMemcpy(records)"));
    if ((e = cudaMalloc(&h->d_psr, sizeof(PulsarDev) * n_pulsars)) != cudaSuccess)
        return cleanup(cuda_fail(e, "cudaMalloc(pulsars)"));
    if ((e = cudaMalloc(&h->d_counter, sizeof(int))) != cudaSuccess)
        return cleanup(cuda_fail(e, "cudaMalloc(counter)"));
    if ((e = cudaMalloc(&h->d_any2, sizeof(int))) != cudaSuccess)
        return cleanup(cuda_fail(e, "cudaMalloc(status flag)"));
    if ((e = cudaMalloc(&h->d_phase_tab, sizeof(double) * kPhaseTableDoubles)) != cudaSuccess)
        return cleanup(cuda_fail(e, "cudaMalloc(phase table)"));
    launch_fill_phase_table(h->d_phase_tab, nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaDeviceSynchronize()) != cudaSuccess)
        return cleanup(cuda_fail(e, "phase table"));
    if ((e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cleanup(cuda_fail(e, "cudaStreamCreate"));
    argus_status st = apply_plan(h);
    if (st) return cleanup(st);
    *out = h;
    return ARGUS_OK;
}

void argus_array_destroy(argus_array* h) {
    if (!h) return;
    DeviceGuard guard(h->device);
    cudaDeviceSynchronize();
    drop_graphs(h);
    for (auto& e : h->ev)
        if (e) cudaEventDestroy(e);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    cudaFree(h->d_rec);
    cudaFree(h->d_psr);
    cudaFree(h->d_lc);
    cudaFree(h->d_lane);
    cudaFree(h->d_items);
    cudaFree(h->d_ckpt);
    cudaFree(h->d_tape);
    cudaFree(h->d_counter);
    cudaFree(h->d_any2);
    cudaFree(h->d_stage);
    cudaFree(h->d_sitems);
    cudaFree(h->d_lane_first);
    cudaFree(h->d_tpre);
    cudaFree(h->d_bagg);
    cudaFree(h->d_bpre);
    cudaFree(h->d_part);
    cudaFree(h->d_phase_tab);
    cudaFree(h->d_stape);
    cudaFree(h->d_tsuf);
    cudaFree(h->d_ragg);
    cudaFree(h->d_rpre);
    cudaFree(h->d_partg);
    cudaFree(h->d_rdone);
    delete h;
}

int32_t argus_array_dim(const argus_array* h) { return h ? kNgw + h->nq * h->P : -1; }

int32_t argus_array_device(const argus_array* h) { return h ? h->device : -1; }

int32_t argus_array_model(const argus_array* h) {
    if (!h) return -1;
    return ((h->flags & kFlagOU) ? ARGUS_NOISE_OU : ARGUS_NOISE_RANDOM_WALK) |
           ((h->flags & kFlagPulsarTerm) ? ARGUS_PULSAR_TERM : 0);
}

argus_status argus_array_set_plan(argus_array* h, const argus_plan* plan) {
    if (!h) return fail(ARGUS_ERR_INVALID_ARG, "array handle is NULL");
    argus_status st = validate_plan(plan);
    if (st) return st;
    DeviceGuard guard(h->device);
    CK(cudaDeviceSynchronize());
    h->plan = *plan;
    return apply_plan(h);
}

argus_status argus_array_get_plan(const argus_array* h, argus_plan* plan) {
    if (!h || !plan) return fail(ARGUS_ERR_INVALID_ARG, "NULL argument");
    *plan = h->plan;
    return ARGUS_OK;
}

argus_status argus_loglik(argus_array* h, const double* theta, int64_t B, double* loglik,
                          void* stream) {
    if (B > 0 && !loglik) return fail(ARGUS_ERR_INVALID_ARG, "loglik is NULL");
    return evaluate(h, theta, B, loglik, nullptr, nullptr, stream);
}

argus_status argus_loglik_grad(argus_array* h, const double* theta, int64_t B, double* loglik,
                               double* grad, void* stream) {
    if (B > 0 && (!loglik || !grad)) return fail(ARGUS_ERR_INVALID_ARG, "loglik or grad is NULL");
    return evaluate(h, theta, B, loglik, grad, nullptr, stream);
}

argus_status argus_walker_flags(argus_array* h, const double* theta, int64_t B, const double* loglik,
                                int32_t* flags, void* stream) {
    if (!h) return fail(ARGUS_ERR_INVALID_ARG, "array handle is NULL");
    if (B < 0) return fail(ARGUS_ERR_INVALID_ARG, "B must be >= 0");
    if (B == 0) return ARGUS_OK;
    if (!theta || !loglik || !flags) return fail(ARGUS_ERR_INVALID_ARG, "NULL theta, loglik or flags");
    DeviceGuard guard(h->device);
    if (!is_device_ptr(theta) || !is_device_ptr(loglik) || !is_device_ptr(flags))
        return fail(ARGUS_ERR_INVALID_ARG, "argus_walker_flags needs device pointers");
    launch_walker_flags(theta, B, h->P, h->flags, loglik, flags, nullptr,
                        reinterpret_cast<cudaStream_t>(stream));
    CK(cudaGetLastError());
    return ARGUS_OK;
}

argus_status argus_lane_loglik(argus_array* h, const double* theta, int64_t B, double* lane_ll,
                               void* stream) {
    if (B > 0 && !lane_ll) return fail(ARGUS_ERR_INVALID_ARG, "lane_ll is NULL");
    return evaluate(h, theta, B, nullptr, nullptr, lane_ll, stream);
}

argus_status argus_array_set_timing(argus_array* h, int32_t enable) {
    if (!h) return fail(ARGUS_ERR_INVALID_ARG, "array handle is NULL");
    DeviceGuard guard(h->device);
    if (enable && !h->ev[0])
        for (auto& e : h->ev) CK(cudaEventCreate(&e));
    h->timing = enable != 0;
    h->timed_once = false;
    drop_graphs(h);
    return ARGUS_OK;
}

argus_status argus_array_get_timing(argus_array* h, float* ms) {
    if (!h || !ms) return fail(ARGUS_ERR_INVALID_ARG, "NULL argument");
    if (!h->timing || !h->timed_once)
        return fail(ARGUS_ERR_INVALID_ARG, "no timed call since timing was enabled");
    DeviceGuard guard(h->device);
    CK(cudaEventSynchronize(h->ev[3]));
    for (int i = 0; i < 3; ++i) CK(cudaEventElapsedTime(&ms[i], h->ev[i], h->ev[i + 1]));
    return ARGUS_OK;
}

argus_status argus_cw_signal(argus_array* h, const double* theta_gw, double* s) {
    if (!h || !theta_gw || !s) return fail(ARGUS_ERR_INVALID_ARG, "NULL argument");
    for (int j = 0; j < kNgw; ++j)
        if (!std::isfinite(theta_gw[j])) return fail(ARGUS_ERR_INVALID_ARG, "non-finite theta_gw");
    if (h->total_toa == 0) return ARGUS_OK;
    DeviceGuard guard(h->device);
    double* d = nullptr;
    CK(cudaMalloc(&d, sizeof(double) * (kNgw + h->total_toa)));
    cudaError_t e = cudaMemcpy(d, theta_gw, sizeof(double) * kNgw, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        launch_cw_signal(d, h->P, h->d_psr, h->d_rec, h->n_max, d + kNgw, nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMemcpy(s, d + kNgw, sizeof(double) * h->total_toa, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "argus_cw_signal");
    return ARGUS_OK;
}

const char* argus_status_string(argus_status s) {
    switch (s) {
        case ARGUS_OK: return "ARGUS_OK";
        case ARGUS_ERR_INVALID_ARG: return "ARGUS_ERR_INVALID_ARG";
        case ARGUS_ERR_CUDA: return "ARGUS_ERR_CUDA";
        case ARGUS_ERR_OOM: return "ARGUS_ERR_OOM";
        case ARGUS_ERR_NONFINITE: return "ARGUS_ERR_NONFINITE";
        case ARGUS_ERR_TIMEOUT: return "ARGUS_ERR_TIMEOUT";
        case ARGUS_ERR_UNSUPPORTED: return "ARGUS_ERR_UNSUPPORTED";
    }
    return "ARGUS_ERR_UNKNOWN";
}

const char* argus_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free log-likelihood + gradient (argus_loglik_grad_noalloc).
//
// For callers that must not allocate device memory while they run: code
// embedded in a framework that has already reserved (nearly) all of the GPU's
// memory for its own pool, so a cudaMalloc from this library would fail or
// fragment that pool, and code in a hot loop where a cudaMalloc/cudaFree (which
// can synchronise the device) is not acceptable.  The handle is still created
// once, up front, by argus_array_create.  Each call then takes all of its
// scratch -- work counter, work items, lane constants, per-lane results,
// adjoint checkpoints and tape -- from one file-scope device array of
// kNoAllocBytes, and allocates nothing.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr size_t kNoAllocBytes = size_t(64) << 20;   // 64 MiB, held by every GPU that loads the library
constexpr int kNoAllocW = 64;                        // walkers per block in this variant
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};
void* g_noalloc_ctx[kNoAllocMaxDevices] = {};   // the context each address was looked up in

__global__ void k_noalloc_items(WorkItem* items, int n_items, int64_t tiles, int W) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_items) return;
    items[i] = WorkItem{int32_t(i / tiles), int32_t((i % tiles) * W)};
}

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

// The current CUDA context (driver entry point, looked up once), or nullptr.
void* current_context() {
    using GetCtx = int (*)(void**);
    static GetCtx fn = []() -> GetCtx {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<GetCtx>(f);
    }();
    void* ctx = nullptr;
    if (!fn || fn(&ctx) != 0) return nullptr;
    return ctx;
}

// Device address of the scratch array on the current device (the array's name
// in host code is only a host-side stand-in).  Looked up once per device, and
// again if the device's context has changed since (a device reset destroys the
// primary context, and the module, with the array, loads again elsewhere).
argus_status noalloc_scratch(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return fail(ARGUS_ERR_UNSUPPORTED, "device ordinal beyond the no-alloc table");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    void* ctx = current_context();
    if (!g_noalloc_addr[dev] || !ctx || ctx != g_noalloc_ctx[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_noalloc_addr[dev] = p;
        g_noalloc_ctx[dev] = ctx;
    }
    *out = static_cast<unsigned char*>(g_noalloc_addr[dev]);
    return ARGUS_OK;
}

}  // namespace

extern "C" argus_status argus_loglik_grad_noalloc(argus_array* h, const double* theta, int64_t B,
                                                  double* loglik, double* grad, void* stream) {
    if (!h) return fail(ARGUS_ERR_INVALID_ARG, "array handle is NULL");
    if (B < 0) return fail(ARGUS_ERR_INVALID_ARG, "B must be >= 0");
    if (B == 0) return ARGUS_OK;
    if (!theta || !loglik || !grad) return fail(ARGUS_ERR_INVALID_ARG, "NULL theta, loglik or grad");
    DeviceGuard guard(h->device);
    if (!is_device_ptr(theta) || !is_device_ptr(loglik) || !is_device_ptr(grad))
        return fail(ARGUS_ERR_INVALID_ARG, "argus_loglik_grad_noalloc needs device pointers");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int W = kNoAllocW;
    const int64_t tiles = (B + W - 1) / W;
    const int64_t n_items64 = tiles * h->P;
    if (n_items64 > INT32_MAX) return fail(ARGUS_ERR_UNSUPPORTED, "too many work items");
    const int n_items = int(n_items64);
    const size_t lanes = size_t(B) * h->P;
    // carve the array: counter | items | lane constants | lane results | slots
    const size_t off_items = 256;
    const size_t off_lc = off_items + align256(size_t(n_items) * sizeof(WorkItem));
    const size_t off_lane = off_lc + align256(lanes * kLaneConsts * sizeof(double));
    const size_t off_slots = off_lane + align256(lanes * (1 + kLaneGrads) * sizeof(double));
    const size_t ck_slot = size_t(h->nseg_max) * kCkptDoubles * W;     // doubles
    const size_t tp_slot = size_t(h->stride_max) * tape_doubles(h->model) * W;   // doubles
    const size_t slot_bytes = align256(ck_slot * sizeof(double)) + align256(tp_slot * sizeof(double));
    if (off_slots + slot_bytes > kNoAllocBytes) {
        char buf[200];
        snprintf(buf, sizeof buf,
                 "argus_loglik_grad_noalloc: B x P = %zu lanes with %d-TOA segments needs %zu bytes "
                 "of static scratch; the maximum is %zu",
                 lanes, h->stride_max, off_slots + slot_bytes, kNoAllocBytes);
        return fail(ARGUS_ERR_UNSUPPORTED, buf);
    }
    const int fit = int(std::min<size_t>((kNoAllocBytes - off_slots) / slot_bytes, INT32_MAX));
    const int grid = std::max(1, std::min({n_items, 4 * h->n_sm, fit}));
    unsigned char* base = nullptr;
    argus_status st = noalloc_scratch(h->device, &base);
    if (st) return st;
    int* counter = reinterpret_cast<int*>(base);
    WorkItem* items = reinterpret_cast<WorkItem*>(base + off_items);
    double* lc = reinterpret_cast<double*>(base + off_lc);
    double* lane = reinterpret_cast<double*>(base + off_lane);
    double* ckpt = reinterpret_cast<double*>(base + off_slots);
    double* tape = reinterpret_cast<double*>(base + off_slots + align256(ck_slot * sizeof(double)) * grid);
    // the work counter must start at zero; everything else is written before it is read
    CK(cudaMemsetAsync(counter, 0, sizeof(int), s));
    k_noalloc_items<<<(n_items + 255) / 256, 256, 0, s>>>(items, n_items, tiles, W);
    launch_project(theta, B, h->P, h->flags, h->d_psr, lc, s);
    FilterArgs a{};
    a.rec = h->d_rec;
    a.psr = h->d_psr;
    a.items = items;
    a.n_items = n_items;
    a.P = h->P;
    a.B = B;
    a.lc = lc;
    a.lane_out = lane;
    a.ckpt = ckpt;
    a.tape = tape;
    a.ckpt_slot = int64_t(align256(ck_slot * sizeof(double)) / sizeof(double));
    a.tape_slot = int64_t(align256(tp_slot * sizeof(double)) / sizeof(double));
    a.stride_max = h->stride_max;
    a.counter = counter;
    a.model = h->model;
    launch_filter_grad(a, W, grid, s);
    launch_reduce(theta, B, h->P, h->flags, h->d_psr, lane, loglik, grad, nullptr, s);
    CK(cudaGetLastError());
    return ARGUS_OK;
}
