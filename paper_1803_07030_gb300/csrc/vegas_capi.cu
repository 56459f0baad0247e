// C-ABI of the Metropolis sweep: context creation (packing samples into device memory),
// the schedule driver (one CUDA graph per MCS, replayed), history and spin I/O.
// See include/vegas.h for the contract of every entry point.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "vegas_internal.h"

using namespace vegas;

namespace {

thread_local std::string g_create_error;

// An NVTX range for the lifetime of the object (tracing: a profiler shows every vegas_run
// and every temperature/field step it enqueues; without a profiler attached NVTX does nothing).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

struct SampleInfo {
    int32_t n = 0, n_colours = 0, uniform_degree = 0;
    int32_t site_off = 0;      // first global site
    int64_t edge_off = 0;      // first global edge
    std::vector<int32_t> cstart, lower_mode, orig;
    bool uniform_params = false, has_anisotropy = false;
    bool has_policy = false, has_adaptive = false;
    double sigma0 = 0.0;
    SiteParams64 u{};
    std::vector<int32_t> type;  // per site (new numbering)
};

struct PassLaunch {
    PassArgs args;
    int grid;
    int threads = kThreads;    // threads per block (FP64 passes of small classes use fewer)
    int32_t sample, group;     // partial slots are grouped by (sample, type group)
    int32_t col;               // colour class
    int64_t slot = 0;          // first block slot
};

// One sweep launch of an MCS of the per-class sweep: a single pass, or the direct FP32 passes
// of one colour class of several samples (or type groups) merged into one launch.
struct LaunchGroup {
    std::vector<int> passes;     // indices into the context's passes
    int grid = 0;                // merged: the passes' blocks together
    PassArgs *d_args = nullptr;  // merged: the passes' arguments
    int32_t *d_first = nullptr;  // merged: first block of each pass, and the total
};

}  // namespace

struct vegas_ctx {
    vegas_options opt{};
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    bool own_stream = false;
    int precision = 32, R = 1, log2R = 0, n_samples = 0, n_inst = 0, max_colours = 0;
    int64_t n_sites = 0, n_edges = 0;
    std::vector<SampleInfo> samples;
    std::vector<PassLaunch> passes;
    // device buffers
    void *d_spins = nullptr, *d_edges = nullptr, *d_p0 = nullptr, *d_p1 = nullptr, *d_pk = nullptr;
    int2 *d_ell = nullptr;  // links as fixed rows of kEllRow (spins-in-shared-memory sweeps)
    int64_t *d_rowptr = nullptr, *d_slot_base = nullptr;
    uint32_t *d_pass_tickets = nullptr;  // [passes] block counters of the R = 32 staged kernel
    int32_t n_groups = 1;      // type groups of the partial slots (n_types with type_stats)
    int32_t n_types = 0;       // tracked site types (type_stats), else 0
    double *d_type_hist = nullptr;
    size_t type_hist_cap = 0;
    void *d_snap = nullptr;
    size_t snap_cap = 0;       // bytes
    int4 *d_segs = nullptr;
    int32_t *d_orig = nullptr, *d_slot_count = nullptr;
    double *d_norm = nullptr, *d_partial = nullptr, *d_sched = nullptr, *d_hist = nullptr;
    size_t sched_cap = 0, hist_cap = 0;
    // acceptance counts and update policies
    uint32_t *d_acc = nullptr, *d_acc_hist = nullptr;
    size_t acc_hist_cap = 0;
    PolicySite *d_pol = nullptr;      // FP64 contexts
    PolicySite32 *d_pol32 = nullptr;  // FP32 contexts
    int32_t *d_qis = nullptr;         // [global site] 1 for qIsing sites, or NULL
    double *d_sigma = nullptr;
    int32_t *d_adapt_n = nullptr;
    bool any_adaptive = false;
    RunState *d_run = nullptr;
    uint32_t *d_err = nullptr;
    uint8_t *d_alog = nullptr;
    int64_t alog_bytes = 0;
    int64_t device_bytes = 0;
    // resident (persistent) sweep
    ResidentInst *d_insts = nullptr;
    int32_t *d_cstart = nullptr;
    uint32_t *d_queue = nullptr;
    ResidentArgs res{};
    int res_threads = 256, res_grid = 1;
    bool res_smem_eligible = false;  // every instance's spins fit the shared-memory form
    bool res_smem = false;           // the resident sweep keeps spins in shared memory
    bool cluster_smem = false;       // the cluster sweep keeps copies of the spins in shared memory
    int res_items = 0;          // instances of the resident and cluster sweeps
    bool res_policy = false;    // some sample has a policy table (kernel choice for the shapes)
    bool res_eligible = false, tuned = false;
    int32_t max_instance_sites = 0, min_instance_sites = 0;
    double tune_ms[4] = {0.0, 0.0, 0.0, 0.0};  // per-MCS time of each sweep when tuned
    // cluster sweep: clusters of cluster_cs blocks, cluster_n of them at once
    bool cluster_eligible = false;
    int cluster_cs = 0, cluster_n = 0, cluster_threads = 256;
    // cooperative sweep
    bool coop_eligible = false;
    CoopArgs coop{};
    int coop_grid = 1;
    int coop_grid_max = 1;  // every block the GPU holds at once, capped by the widest class and max_blocks
    GridBarrier *d_bar = nullptr;
    double *d_coop_partial = nullptr;
    // wavefront sweep: both classes of an MCS in one launch
    WaveArgs wave{};
    int wave_grid = 1;
    int32_t *d_tasks = nullptr;
    int32_t *d_deps = nullptr;  // wavefront sweep: distinct class-0 blocks of each class-1 block
    std::vector<LaunchGroup> launches;  // the per-class sweep's launches of one MCS, in class order
    // renormalisation folded into the step's last class-1 pass (per-class sweep, R = 32)
    bool fold_ok = false;
    PassArgs fold_args{};       // the class-1 pass's arguments with the fold's fields
    int32_t fold_nb0 = 0;       // class-0 blocks
    int32_t *d_fold_deps = nullptr, *d_fold_deg = nullptr;
    uint32_t *d_fold_cnt = nullptr;
    uint32_t *d_done = nullptr, *d_ticket = nullptr;
    double *d_wave_partial = nullptr;
    int64_t *d_wave_slot_base = nullptr;
    int32_t *d_wave_slot_count = nullptr;
    // graph of one MCS (per-class sweep), and graphs of a whole temperature/field step
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<std::pair<int64_t, cudaGraphExec_t>> step_graphs;  // key: mcs * 2 + variant
    // run graphs of the per-class and resident sweeps: a conditional while node over
    // temperature/field steps whose body is one whole step; key: mcs * 4 + variant
    std::vector<std::pair<int64_t, cudaGraphExec_t>> run_graphs;
    std::vector<cudaGraph_t> run_graph_defs;
    bool run_graph_failed = false;
    // host state
    std::vector<std::vector<double>> hist;  // per instance: records * 4
    std::vector<std::vector<uint32_t>> acc_hist;  // per instance: accepted attempts per record
    std::vector<std::vector<double>> type_hist;   // per instance: records * n_types * 3
    std::vector<std::vector<double>> snaps;       // per instance: steps * n_sites * 3 (caller order)
    int64_t snapshot_steps = 0;
    int64_t records = 0;
    uint32_t t = 0;
    uint32_t device_error = 0;
    int64_t kernel_launches = 0, sweep_launches = 0, graph_launches = 0;
    double sweep_ms = 0.0, last_run_ms = 0.0;
    int variant = 0;
    bool poisoned = false;
    std::string err;
};

namespace {

vegas_status fail(vegas_ctx *c, vegas_status st, const std::string &msg) {
    if (c) {
        c->err = msg;
        if (st == VEGAS_ECUDA || st == VEGAS_EDEVICE || st == VEGAS_ETIMEOUT) c->poisoned = true;
    } else {
        g_create_error = msg;
    }
    return st;
}

// A host exception caught at an entry point, as a status (called inside a catch block).
vegas_status host_exception(vegas_ctx *c) {
    std::string m;
    const vegas_status st = status_of_current_exception(m);
    return fail(c, st, m);
}

#define CK(ctx, call)                                                                                     \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess)                                                                            \
            return fail((ctx), e_ == cudaErrorMemoryAllocation ? VEGAS_ENOMEM : VEGAS_ECUDA,              \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                              \
    } while (0)

template <typename T>
cudaError_t dalloc(vegas_ctx *c, T **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e == cudaSuccess) c->device_bytes += (int64_t)bytes;
    return e;
}

void free_all(vegas_ctx *c) {
    for (auto &kv : c->step_graphs) cudaGraphExecDestroy(kv.second);
    for (auto &kv : c->run_graphs) cudaGraphExecDestroy(kv.second);
    for (cudaGraph_t g : c->run_graph_defs) cudaGraphDestroy(g);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    void *bufs[] = {c->d_spins, c->d_edges, c->d_ell, c->d_p0, c->d_p1, c->d_pk, c->d_rowptr, c->d_slot_base, c->d_orig,
                    c->d_slot_count, c->d_norm, c->d_partial, c->d_sched, c->d_hist, c->d_run, c->d_err, c->d_alog,
                    c->d_insts, c->d_cstart, c->d_queue, c->d_bar, c->d_coop_partial, c->d_acc, c->d_acc_hist,
                    c->d_pol, c->d_pol32, c->d_qis, c->d_sigma, c->d_adapt_n, c->d_type_hist, c->d_snap, c->d_segs,
                    c->d_tasks, c->d_deps, c->d_done, c->d_ticket, c->d_pass_tickets, c->d_wave_partial, c->d_wave_slot_base, c->d_wave_slot_count,
                    c->d_fold_deps, c->d_fold_deg, c->d_fold_cnt};
    for (void *b : bufs)
        if (b) cudaFree(b);
    for (LaunchGroup &lg : c->launches) {
        if (lg.d_args) cudaFree(lg.d_args);
        if (lg.d_first) cudaFree(lg.d_first);
    }
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

int32_t float_bits(float f) {
    int32_t i;
    std::memcpy(&i, &f, sizeof i);
    return i;
}

int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

// Block shape of the resident sweep: threads per block, as many blocks as fit (at most one
// per instance), and the grouping of small instances (group_threads threads per instance of
// at most group_sites sites, several per block; 0 = one instance per block).
// smem: each instance's spins in shared memory for the whole launch (512 or 1024 threads; a
// group's region is then at most kResSmemBytes / (12 x groups) sites). Returns false, leaving
// the spins in global memory, when that form does not fit the device.
constexpr int64_t kResSmemBytes = 200 * 1024;  // spins in shared memory: 12 bytes per site

bool set_resident_shape(vegas_ctx *c, int threads, int group_threads = 0, int group_sites = 0, bool smem = false) {
    const bool grouped = group_threads > 0 && group_threads < threads && threads % group_threads == 0 &&
                         threads / group_threads <= 15;
    c->res.group_threads = grouped ? group_threads : 0;
    c->res.group_sites = grouped ? group_sites : 0;
    c->res_smem = false;
    if (smem && c->res_smem_eligible) {
        ResidentArgs a = c->res;
        if (grouped)  // an even cap: the groups' regions then keep the budget with even starts
            a.group_sites = (int)std::min<int64_t>(group_sites, (kResSmemBytes / (12 * (threads / group_threads))) & ~1);
        a.smem_sites = c->max_instance_sites;
        const int bps = resident_blocks_per_sm(threads, c->res_policy, resident_smem_bytes(a, threads));
        cudaGetLastError();
        if (bps > 0) {
            c->res.group_sites = a.group_sites;
            c->res_smem = true;
            c->res_threads = threads;
            c->res_grid = (int)std::min<int64_t>((int64_t)c->res_items, (int64_t)c->sm_count * bps);
            return true;
        }
        threads = std::min(threads, 512);
    }
    c->res_threads = threads;
    c->res_grid = (int)std::min<int64_t>((int64_t)c->res_items,
                                         (int64_t)c->sm_count * resident_blocks_per_sm(threads, c->res_policy));
    return !smem;
}

// Shape of the cluster sweep: cs blocks of `threads` per cluster, as many clusters as fit,
// instances of at most `split` sites swept by one block each (0: all by clusters), those of at
// most group_sites sites several to a block in groups of group_threads threads (-1: the
// grouping already set), and with smem every block's copy of the spins in shared memory;
// false (shape unchanged) if no such cluster fits.
bool set_cluster_shape(vegas_ctx *c, int cs, int threads, int split = 0, int group_threads = -1, int group_sites = 0,
                       bool smem = false) {
    if (smem && !c->res_smem_eligible) return false;
    ResidentArgs a = c->res;
    if (group_threads >= 0) {
        a.group_threads = group_threads > 0 && group_threads < threads ? group_threads : 0;
        a.group_sites = a.group_threads > 0 ? group_sites : 0;
    }
    if (smem && a.group_threads > 0)
        a.group_sites = (int)std::min<int64_t>(a.group_sites, (kResSmemBytes / (12 * (threads / a.group_threads))) & ~1);
    a.smem_sites = smem ? c->max_instance_sites : 0;
    const int cap = cluster_capacity(cs, threads, c->res_policy, cluster_smem_bytes(a, threads));
    cudaGetLastError();
    if (cap <= 0) return false;
    c->cluster_cs = cs;
    c->cluster_threads = threads;
    c->cluster_n = (int)std::min<int64_t>((int64_t)c->res_items, cap);
    c->cluster_smem = smem;
    c->res.split_sites = split;
    c->res.group_threads = a.group_threads;
    c->res.group_sites = a.group_sites;
    return true;
}

// The step's last class-1 pass renormalises the spins (per-class sweep of a sample that
// allows it; option renorm_fold).
bool fold_active(const vegas_ctx *c) { return c->fold_ok && c->variant == 0; }

// The cooperative sweep's grid: bps blocks per SM, within coop_grid_max. Every grid barrier
// takes one arrival per block, so more blocks than the sample needs cost time: on the 64^3
// lattice 2 blocks per SM ran 12.5 G attempts/s, 1 ran 12.1 and 3 ran 10.6.
void set_coop_shape(vegas_ctx *c, int bps) { c->coop_grid = std::max(1, std::min(c->coop_grid_max, c->sm_count * bps)); }

// Launch one MCS: every colour class of every sample, then the reduction. last: the step's
// last MCS, whose class-1 pass then renormalises every spin when fold_active.
void enqueue_mcs(vegas_ctx *c, cudaStream_t st, std::vector<cudaEvent_t> *ev, bool last = false) {
    const bool fold = last && fold_active(c);
    if (fold) cudaMemsetAsync(c->d_fold_cnt, 0, sizeof(uint32_t) * (size_t)c->fold_nb0, st);
    int k = 0;
    for (const LaunchGroup &lg : c->launches) {
        const PassLaunch &p = c->passes[(size_t)lg.passes[0]];
        if (ev) cudaEventRecord((*ev)[2 * k], st);
        if (lg.d_args) {
            launch_pass32_multi(p.args, lg.d_args, lg.d_first, (int32_t)lg.passes.size(), lg.grid, st);
        } else if (c->precision == 64) {
            launch_pass64(p.args, p.grid, p.threads, st);
        } else if (fold && lg.passes[0] == 1) {
            launch_pass32(c->fold_args, p.grid, st);
        } else {
            launch_pass32(p.args, p.grid, st);
        }
        if (ev) cudaEventRecord((*ev)[2 * k + 1], st);
        ++k;
    }
    // the reduction also zeroes the R = 32 kernel's block counters for the next MCS
    ReduceArgs ra{c->d_partial, c->d_slot_base, c->d_slot_count, c->d_run, c->d_adapt_n, c->R, c->n_inst,
                  c->n_groups, c->n_types, c->d_pass_tickets, (int32_t)c->passes.size()};
    launch_reduce(ra, st);
}

// One persistent launch for n MCS of the current step; the run state advances afterwards.
void enqueue_resident(vegas_ctx *c, cudaStream_t st, int32_t n) {
    cudaMemsetAsync(c->d_queue, 0, sizeof(uint32_t), st);
    ResidentArgs a = c->res;
    a.mcs = n;
    a.smem_sites = c->res_smem ? c->max_instance_sites : 0;
    launch_resident(a, c->res_grid, c->res_threads, st);
    launch_advance(c->d_run, n, st);
}

// One cooperative launch for n MCS of the current step; the run state advances afterwards.
void enqueue_coop(vegas_ctx *c, cudaStream_t st, int32_t n) {
    cudaMemsetAsync(c->d_bar, 0, sizeof(GridBarrier), st);
    CoopArgs a = c->coop;
    a.mcs = n;
    launch_coop(a, c->coop_grid, st);
    launch_advance(c->d_run, n, st);
}

// One cluster-sweep launch for n MCS of the current step; the run state advances afterwards.
void enqueue_cluster(vegas_ctx *c, cudaStream_t st, int32_t n) {
    cudaMemsetAsync(c->d_queue, 0, sizeof(uint32_t), st);
    ResidentArgs a = c->res;
    a.mcs = n;
    a.smem_sites = c->cluster_smem ? c->max_instance_sites : 0;
    launch_cluster(a, c->cluster_n, c->cluster_cs, c->cluster_threads, st);
    launch_advance(c->d_run, n, st);
}

// One MCS of the wavefront sweep (both colour classes in one launch), then the reduction;
// returns the CUDA error of the sweep launch.
int enqueue_wave(vegas_ctx *c, cudaStream_t st) {
    cudaMemsetAsync(c->d_ticket, 0, sizeof(uint32_t), st);
    const int e = launch_wave(c->wave, c->wave_grid, st);
    ReduceArgs ra{c->d_wave_partial, c->d_wave_slot_base, c->d_wave_slot_count, c->d_run, c->d_adapt_n, c->R,
                  c->n_inst, 1, 0, nullptr, 0};
    launch_reduce(ra, st);
    return e;
}

// Renormalisation at the end of a step (unless the step's last pass did it: folded), then
// (option snapshots) the copy of the final state.
void enqueue_renorm(vegas_ctx *c, cudaStream_t st, bool folded = false) {
    RenormArgs ra{c->d_spins, c->d_norm, c->n_sites * c->R, c->log2R, c->d_qis};
    const int grid = (int)std::min<int64_t>((ra.n_work + 255) / 256, (int64_t)c->sm_count * 8);
    if (c->precision == 64)
        launch_renorm64(ra, grid, st);
    else if (!folded)
        launch_renorm32(ra, grid, st);
    if (c->opt.snapshots) {
        const int64_t n16 = c->n_sites * c->R * (c->precision == 64 ? 2 : 1);
        const int g2 = (int)std::min<int64_t>((n16 + 255) / 256, (int64_t)c->sm_count * 8);
        launch_snapshot(c->d_spins, c->d_snap, n16, c->d_run, g2, st);
    }
}

constexpr int64_t kMaxStepGraphNodes = 20000;

// Launches of one whole step (mcs MCS and the renormalisation) for the chosen variant, or
// -1 when such a graph would be too large.
int64_t step_graph_nodes(const vegas_ctx *c, int32_t mcs) {
    const int64_t sweep = c->variant == 4 ? 3 * (int64_t)mcs
                                         : (c->variant >= 1 ? 3 : (int64_t)mcs * ((int64_t)c->launches.size() + 1));
    const int64_t n = sweep + 1 + (c->opt.snapshots ? 1 : 0);
    return n <= kMaxStepGraphNodes ? n : -1;
}

// Graph of one temperature/field step; every kernel reads the step from the run state, so
// the same graph serves every step with this MCS count.
vegas_status step_graph(vegas_ctx *c, int32_t mcs, cudaGraphExec_t *out) {
    const int64_t key = (int64_t)mcs * 4 + c->variant;
    for (auto &kv : c->step_graphs)
        if (kv.first == key) {
            *out = kv.second;
            return VEGAS_OK;
        }
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    CK(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    if (c->variant == 1) {
        enqueue_resident(c, c->cap_stream, mcs);
    } else if (c->variant == 2) {
        enqueue_coop(c, c->cap_stream, mcs);
    } else {
        for (int32_t m = 0; m < mcs; ++m) enqueue_mcs(c, c->cap_stream, nullptr, m == mcs - 1);
    }
    enqueue_renorm(c, c->cap_stream, fold_active(c));
    CK(c, cudaStreamEndCapture(c->cap_stream, &g));
    cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    CK(c, e);
    c->step_graphs.emplace_back(key, ge);
    *out = ge;
    return VEGAS_OK;
}

// Graph of a whole run of a sweep: a conditional while node whose body is one
// temperature/field step (mcs MCS, the renormalisation, the snapshot) followed by the loop
// control kernel, so one launch runs every step of the schedule (the step index, schedule
// and record count come from the run state). Returns false, leaving no capture open, when
// the device or driver cannot build it; the caller then falls back to one graph per step
// (per-class and resident sweeps) or direct launches.
bool run_graph(vegas_ctx *c, int32_t mcs, cudaGraphExec_t *out) {
    const int64_t key = (int64_t)mcs * 4 + c->variant;
    for (auto &kv : c->run_graphs)
        if (kv.first == key) {
            *out = kv.second;
            return true;
        }
    if (c->run_graph_failed) return false;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    bool capturing = false;
    auto give_up = [&]() {
        if (capturing) {  // the graph it returns is the conditional node's body, owned by g
            cudaGraph_t body_out = nullptr;
            cudaStreamEndCapture(c->cap_stream, &body_out);
        }
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        c->run_graph_failed = true;
        return false;
    };
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return give_up();
    cudaGraphConditionalHandle loop;
    if (cudaGraphConditionalHandleCreate(&loop, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) return give_up();
    cudaGraphNodeParams wp = {cudaGraphNodeTypeConditional};  // the other members zero
    wp.conditional.handle = loop;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wn;
    if (cudaGraphAddNode(&wn, g, nullptr, nullptr, 0, &wp) != cudaSuccess) return give_up();
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(c->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
        return give_up();
    capturing = true;
    if (c->variant == 1) {
        enqueue_resident(c, c->cap_stream, mcs);
    } else if (c->variant == 2) {
        enqueue_coop(c, c->cap_stream, mcs);
    } else if (c->variant == 3) {
        enqueue_cluster(c, c->cap_stream, mcs);
    } else if (c->variant == 4) {
        for (int32_t m = 0; m < mcs; ++m) enqueue_wave(c, c->cap_stream);
    } else {
        for (int32_t m = 0; m < mcs; ++m) enqueue_mcs(c, c->cap_stream, nullptr, m == mcs - 1);
    }
    enqueue_renorm(c, c->cap_stream, fold_active(c));
    launch_run_ctrl(c->d_run, (unsigned long long)loop, c->cap_stream);
    cudaGraph_t captured = nullptr;
    capturing = false;
    if (cudaStreamEndCapture(c->cap_stream, &captured) != cudaSuccess) return give_up();
    if (cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) return give_up();
    c->run_graph_defs.push_back(g);
    c->run_graphs.emplace_back(key, ge);
    *out = ge;
    return true;
}

vegas_status build_graph(vegas_ctx *c) {
    if (c->graph_exec) return VEGAS_OK;
    CK(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    enqueue_mcs(c, c->cap_stream, nullptr);
    CK(c, cudaStreamEndCapture(c->cap_stream, &c->graph));
    CK(c, cudaGraphInstantiate(&c->graph_exec, c->graph, 0));
    return VEGAS_OK;
}

vegas_status check_usable(vegas_ctx *c) {
    if (!c) return VEGAS_EINVAL;
    if (c->poisoned) {
        if (c->err.rfind("context poisoned", 0) != 0) c->err = "context poisoned by an earlier error: " + c->err;
        return VEGAS_ESTATE;
    }
    return VEGAS_OK;
}

vegas_status set_device(vegas_ctx *c) {
    CK(c, cudaSetDevice(c->device));
    return VEGAS_OK;
}

// The distinct class-0 blocks (bs sites each, counted from the sample's first site) that each
// block of bs class-1 sites links to: ascending, -1 padded, width per block; last[q] is the
// largest of block q's (0 when it has none). False when a block links to more than width.
bool class1_block_deps(const SampleInfo &si, const LoadedSample &l, int bs, int width, std::vector<int32_t> &deps,
                       std::vector<int32_t> &last) {
    const int32_t n1 = si.cstart[2] - si.cstart[1], nb1 = (n1 + bs - 1) / bs;
    deps.assign((size_t)nb1 * width, -1);
    last.assign((size_t)nb1, 0);
    for (int32_t q = 0; q < nb1; ++q) {
        int32_t *dq = &deps[(size_t)q * width];
        int nd = 0;
        const int32_t g0 = si.cstart[1] + q * bs, g1 = std::min(g0 + bs, si.cstart[2]);
        for (int32_t g = g0; g < g1; ++g)
            for (int64_t e = l.row_ptr[(size_t)g]; e < l.row_ptr[(size_t)g + 1]; ++e) {
                const int32_t b = l.col[(size_t)e] / bs;
                if (std::find(dq, dq + nd, b) != dq + nd) continue;
                if (nd == width) return false;
                dq[nd++] = b;
            }
        std::sort(dq, dq + nd);
        last[(size_t)q] = nd > 0 ? dq[nd - 1] : 0;
    }
    return true;
}

}  // namespace

extern "C" void vegas_default_options(vegas_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->precision = 32;
    o->replicas = 1;
    o->seed = 1;
    o->inst_base = 0;
    o->device = -1;
    o->cuda_stream = nullptr;
    o->variant = -1;
    o->accept_log_mcs = 0;
    o->timing = 0;
    o->graphs = 1;
    o->max_blocks = 0;
    o->pipeline_depth = 0;
    o->timeout_ns = 0;
    o->fault_inject = 0;
    o->type_stats = 0;
    o->snapshots = 0;
    o->cluster_blocks = 0;
    o->cluster_threads = 0;
    o->cluster_split = 0;
    o->group_threads = 0;
    o->group_sites = 0;
    o->wave_lag = 0;
    o->wave_slab = 0;
    o->resident_smem = 0;
    o->renorm_fold = 0;
}

// vegas_create without the exception guard; *made is the context under construction.
static vegas_status create_context(const vegas_sample *samples, int32_t n_samples, const vegas_options *opt,
                                   vegas_ctx **out, vegas_ctx **made) {
    if (!out) return fail(nullptr, VEGAS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!samples || n_samples < 1) return fail(nullptr, VEGAS_EINVAL, "need at least one sample");
    vegas_options o;
    vegas_default_options(&o);
    if (opt) o = *opt;
    if (o.precision != 32 && o.precision != 64) return fail(nullptr, VEGAS_EINVAL, "precision must be 32 or 64");
    if (o.replicas < 1 || o.replicas > 32 || (o.replicas & (o.replicas - 1)))
        return fail(nullptr, VEGAS_EINVAL, "replicas must be 1, 2, 4, 8, 16 or 32");
    if (o.accept_log_mcs < 0 || o.inst_base < 0 || o.max_blocks < 0) return fail(nullptr, VEGAS_EINVAL, "negative option");
    if (o.variant < -1 || o.variant > 4) return fail(nullptr, VEGAS_EINVAL, "variant must be -1, 0, 1, 2, 3 or 4");
    if (o.variant == 4 && (o.precision != 32 || n_samples != 1 || o.replicas != 32 || o.type_stats))
        return fail(nullptr, VEGAS_EINVAL,
                    "the wavefront sweep (variant 4) is FP32 with one sample, 32 replicas and no per-type statistics");
    if (o.wave_lag < 0) return fail(nullptr, VEGAS_EINVAL, "wave_lag must be >= 0");
    if (o.wave_slab < -1) return fail(nullptr, VEGAS_EINVAL, "wave_slab must be >= -1");
    if (o.resident_smem < -1 || o.resident_smem > 1) return fail(nullptr, VEGAS_EINVAL, "resident_smem must be -1, 0 or 1");
    if (o.renorm_fold < -1 || o.renorm_fold > 0) return fail(nullptr, VEGAS_EINVAL, "renorm_fold must be -1 or 0");
    if (o.resident_smem == 1 && o.variant != 1 && o.variant != 3 && o.variant != -1)
        return fail(nullptr, VEGAS_EINVAL, "resident_smem = 1 needs the resident or cluster sweep (variant 1, 3 or automatic)");
    if (o.cluster_split < 0) return fail(nullptr, VEGAS_EINVAL, "cluster_split must be >= 0");
    if (o.group_threads != 0 && o.group_threads != 64 && o.group_threads != 128 && o.group_threads != 256)
        return fail(nullptr, VEGAS_EINVAL, "group_threads must be 0, 64, 128 or 256");
    if (o.group_sites < 0) return fail(nullptr, VEGAS_EINVAL, "group_sites must be >= 0");
    if (o.cluster_blocks != 0 && (o.cluster_blocks < 2 || o.cluster_blocks > 16))
        return fail(nullptr, VEGAS_EINVAL, "cluster_blocks must be 0 or 2 .. 16");
    if (o.cluster_threads != 0 && o.cluster_threads != 256 && o.cluster_threads != 512)
        return fail(nullptr, VEGAS_EINVAL, "cluster_threads must be 0, 256 or 512");
    if (o.variant == 3 && o.precision != 32)
        return fail(nullptr, VEGAS_EINVAL, "the cluster sweep (variant 3) is FP32 only");
    if (o.timeout_ns < 0 || o.fault_inject < 0 || o.fault_inject > 1) return fail(nullptr, VEGAS_EINVAL, "bad timeout or fault_inject");
    if (o.graphs < 0 || o.graphs > 2) return fail(nullptr, VEGAS_EINVAL, "graphs must be 0, 1 or 2");
    if (o.type_stats < 0 || o.type_stats > 1 || o.snapshots < 0 || o.snapshots > 1)
        return fail(nullptr, VEGAS_EINVAL, "type_stats and snapshots must be 0 or 1");
    if (o.variant == 2 && o.type_stats)
        return fail(nullptr, VEGAS_EINVAL, "the cooperative sweep (variant 2) does not record per-type statistics");
    if (o.variant == 2 && n_samples != 1)
        return fail(nullptr, VEGAS_EINVAL, "the cooperative sweep (variant 2) runs one sample");
    if (o.pipeline_depth < 0 || o.pipeline_depth > 3) return fail(nullptr, VEGAS_EINVAL, "pipeline_depth must be 0..3");
    if (o.variant == 1 && o.precision != 32)
        return fail(nullptr, VEGAS_EINVAL, "the resident sweep (variant 1) is FP32 only");
    if ((int64_t)o.inst_base + (int64_t)n_samples * o.replicas > (int64_t)UINT32_MAX)
        return fail(nullptr, VEGAS_EINVAL, "instance ids exceed 32 bits");

    // validate and renumber every sample before touching the device
    std::vector<LoadedSample> L((size_t)n_samples);
    int64_t n_sites = 0, n_edges = 0;
    for (int32_t s = 0; s < n_samples; ++s) {
        std::string e;
        if (!load_sample(samples[s], L[(size_t)s], e, o.type_stats != 0, o.variant == 4, (double)o.wave_slab))
            return fail(nullptr, VEGAS_EINVAL, "sample " + std::to_string(s) + ": " + e);
        n_sites += L[(size_t)s].n;
        n_edges += L[(size_t)s].n_edges + (L[(size_t)s].n_edges & 1);  // keep every sample 16-byte aligned
    }
    if (n_sites * o.replicas > ((int64_t)1 << 40) || n_sites > INT32_MAX - (1 << 24) || n_edges >= INT32_MAX)
        return fail(nullptr, VEGAS_EINVAL, "too many sites or links for one context");
    if (o.variant == 4) {
        const LoadedSample &l = L[0];
        if (l.n_colours != 2 || l.uniform_degree != 6 || !l.policy.empty() || l.lower_mode[0] != 0 ||
            l.lower_mode[1] != 1)
            return fail(nullptr, VEGAS_EINVAL,
                        "the wavefront sweep (variant 4) needs two colour classes, six links per site and no "
                        "policy table");
    }
    int32_t n_types = 0;
    if (o.type_stats)
        for (auto &l : L) n_types = std::max(n_types, l.n_types);

    vegas_ctx *c = new (std::nothrow) vegas_ctx();
    if (!c) return fail(nullptr, VEGAS_ENOMEM, "host allocation failed");
    *made = c;
    c->opt = o;
    c->precision = o.precision;
    c->R = o.replicas;
    c->log2R = ilog2(o.replicas);
    c->n_samples = n_samples;
    c->n_inst = n_samples * o.replicas;
    c->n_sites = n_sites;
    c->n_edges = n_edges;
    c->variant = 0;
    c->n_types = n_types;
    c->n_groups = n_types > 0 ? n_types : 1;

    auto bail = [&](vegas_status st) {
        g_create_error = c->err;
        free_all(c);
        delete c;
        *made = nullptr;
        return st;
    };
    int ndev = 0;
    cudaError_t ce = cudaGetDeviceCount(&ndev);
    if (ce != cudaSuccess || ndev == 0) {
        c->err = std::string("no CUDA device: ") + cudaGetErrorString(ce);
        return bail(VEGAS_ECUDA);
    }
    if (o.device >= 0) {
        c->device = o.device;
    } else if (cudaGetDevice(&c->device) != cudaSuccess) {
        c->err = "cudaGetDevice failed";
        return bail(VEGAS_ECUDA);
    }
    vegas_status st;
#define TRY(x)                         \
    do {                               \
        if ((st = (x)) != VEGAS_OK) return bail(st); \
    } while (0)
    TRY(set_device(c));
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, c->device) != cudaSuccess) {
        c->err = "cudaGetDeviceProperties failed";
        return bail(VEGAS_ECUDA);
    }
    c->sm_count = prop.multiProcessorCount;
    if (o.cuda_stream) {
        c->stream = (cudaStream_t)o.cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            c->err = "cudaStreamCreate failed";
            return bail(VEGAS_ECUDA);
        }
        c->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        c->err = "cudaStreamCreate failed";
        return bail(VEGAS_ECUDA);
    }

    // ---- pack samples (host staging)
    const int R = c->R;
    const bool p64 = c->precision == 64;
    bool any_site_params = false, any_policy = false;
    for (auto &l : L) {
        any_site_params |= !l.uniform_params;
        any_policy |= !l.policy.empty();
    }
    std::vector<PolicySite> h_pol(any_policy && p64 ? (size_t)n_sites : 0, PolicySite{0.0, kPolRandom, 0});
    std::vector<PolicySite32> h_pol32(any_policy && !p64 ? (size_t)n_sites : 0, PolicySite32{0.f, kPolRandom});
    std::vector<int32_t> h_qis;  // filled only when some site is qIsing
    std::vector<int32_t> h_orig((size_t)n_sites);
    std::vector<int64_t> h_rowptr((size_t)n_sites + 1);
    std::vector<double> h_norm((size_t)n_sites);
    std::vector<int2> h_e32;
    std::vector<Edge64> h_e64;
    if (p64)
        h_e64.resize((size_t)n_edges, Edge64{0.0, 0, 0});
    else
        h_e32.resize((size_t)n_edges, make_int2(0, 0));
    std::vector<float4> h_p0f, h_p1f;
    std::vector<float> h_pkf;
    std::vector<double4_32a> h_p0d, h_p1d;
    std::vector<double> h_pkd;
    if (any_site_params) {
        if (p64) {
            h_p0d.resize((size_t)n_sites);
            h_p1d.resize((size_t)n_sites);
            h_pkd.resize((size_t)n_sites);
        } else {
            h_p0f.resize((size_t)n_sites);
            h_p1f.resize((size_t)n_sites);
            h_pkf.resize((size_t)n_sites);
        }
    }
    c->samples.resize((size_t)n_samples);
    int64_t site_off = 0, edge_off = 0;
    for (int32_t s = 0; s < n_samples; ++s) {
        LoadedSample &l = L[(size_t)s];
        SampleInfo &si = c->samples[(size_t)s];
        si.n = l.n;
        si.n_colours = l.n_colours;
        si.uniform_degree = l.uniform_degree;
        si.site_off = (int32_t)site_off;
        si.edge_off = edge_off;
        si.cstart = l.cstart;
        si.lower_mode = l.lower_mode;
        si.orig = l.orig;
        si.uniform_params = l.uniform_params;
        si.has_anisotropy = l.has_anisotropy;
        if (o.type_stats) si.type = l.type;
        si.has_policy = !l.policy.empty();
        si.has_adaptive = l.has_adaptive;
        si.sigma0 = l.sigma0;
        c->any_adaptive |= l.has_adaptive;
        if (si.has_policy)
            for (int32_t g = 0; g < l.n; ++g) {
                const double par = l.policy_param[(size_t)g];
                const int32_t code = l.policy[(size_t)g];
                if (p64)
                    h_pol[(size_t)(site_off + g)] = PolicySite{par, code, 0};
                else
                    h_pol32[(size_t)(site_off + g)] = PolicySite32{(float)par, code};
                if (code == kPolQIsing) {
                    if (h_qis.empty()) h_qis.assign((size_t)n_sites, 0);
                    h_qis[(size_t)(site_off + g)] = 1;
                }
            }
        si.u = SiteParams64{l.field_axis[0], l.field_axis[1], l.field_axis[2], l.spin_norm[0],
                            l.e_uni[0],      l.e_uni[1],      l.e_uni[2],      l.k_uni[0], l.k_cub[0]};
        c->max_colours = std::max(c->max_colours, l.n_colours);
        for (int32_t g = 0; g < l.n; ++g) {
            const size_t G = (size_t)(site_off + g);
            h_orig[G] = l.orig[(size_t)g];
            h_rowptr[G] = edge_off + l.row_ptr[(size_t)g];
            h_norm[G] = l.spin_norm[(size_t)g];
            if (any_site_params) {
                const double *fa = &l.field_axis[3 * (size_t)g], *ea = &l.e_uni[3 * (size_t)g];
                if (p64) {
                    h_p0d[G] = make_double4_32a(fa[0], fa[1], fa[2], l.spin_norm[(size_t)g]);
                    h_p1d[G] = make_double4_32a(ea[0], ea[1], ea[2], l.k_uni[(size_t)g]);
                    h_pkd[G] = l.k_cub[(size_t)g];
                } else {
                    h_p0f[G] = make_float4((float)fa[0], (float)fa[1], (float)fa[2], (float)l.spin_norm[(size_t)g]);
                    h_p1f[G] = make_float4((float)ea[0], (float)ea[1], (float)ea[2], (float)l.k_uni[(size_t)g]);
                    h_pkf[G] = (float)l.k_cub[(size_t)g];
                }
            }
        }
        for (int64_t e = 0; e < l.n_edges; ++e) {
            const int32_t colg = (int32_t)(site_off + l.col[(size_t)e]);
            if (p64)
                h_e64[(size_t)(edge_off + e)] = Edge64{l.J[(size_t)e], colg, 0};
            else
                h_e32[(size_t)(edge_off + e)] = make_int2(colg, float_bits((float)l.J[(size_t)e]));
        }
        site_off += l.n;
        edge_off += l.n_edges + (l.n_edges & 1);
    }
    h_rowptr[(size_t)n_sites] = edge_off;

    // ---- device buffers
    const size_t vbytes = p64 ? sizeof(double4_32a) : sizeof(float4);
#define DALLOC(ptr, bytes)                                                              \
    do {                                                                                \
        cudaError_t e_ = dalloc(c, &(ptr), (bytes));                                    \
        if (e_ != cudaSuccess) {                                                        \
            c->err = std::string("cudaMalloc ") + #ptr + ": " + cudaGetErrorString(e_); \
            return bail(e_ == cudaErrorMemoryAllocation ? VEGAS_ENOMEM : VEGAS_ECUDA);  \
        }                                                                               \
    } while (0)
#define H2D(dst, src, bytes)                                                                  \
    do {                                                                                      \
        cudaError_t e_ = cudaMemcpyAsync((dst), (src), (bytes), cudaMemcpyHostToDevice, c->stream); \
        if (e_ != cudaSuccess) {                                                              \
            c->err = std::string("upload: ") + cudaGetErrorString(e_);                        \
            return bail(VEGAS_ECUDA);                                                         \
        }                                                                                     \
    } while (0)
    DALLOC(c->d_spins, (size_t)n_sites * R * vbytes);
    DALLOC(c->d_orig, sizeof(int32_t) * (size_t)n_sites);
    DALLOC(c->d_rowptr, sizeof(int64_t) * ((size_t)n_sites + 1));
    DALLOC(c->d_norm, sizeof(double) * (size_t)n_sites);
    DALLOC(c->d_edges, (p64 ? sizeof(Edge64) : sizeof(int2)) * (size_t)std::max<int64_t>(n_edges, 1));
    DALLOC(c->d_run, sizeof(RunState));
    DALLOC(c->d_err, 4 * sizeof(uint32_t));
    H2D(c->d_orig, h_orig.data(), sizeof(int32_t) * (size_t)n_sites);
    H2D(c->d_rowptr, h_rowptr.data(), sizeof(int64_t) * ((size_t)n_sites + 1));
    H2D(c->d_norm, h_norm.data(), sizeof(double) * (size_t)n_sites);
    if (n_edges > 0) {
        if (p64)
            H2D(c->d_edges, h_e64.data(), sizeof(Edge64) * (size_t)n_edges);
        else
            H2D(c->d_edges, h_e32.data(), sizeof(int2) * (size_t)n_edges);
    }
    if (any_site_params) {
        const size_t pv = p64 ? sizeof(double4_32a) : sizeof(float4), ps = p64 ? sizeof(double) : sizeof(float);
        DALLOC(c->d_p0, pv * (size_t)n_sites);
        DALLOC(c->d_p1, pv * (size_t)n_sites);
        DALLOC(c->d_pk, ps * (size_t)n_sites);
        H2D(c->d_p0, p64 ? (const void *)h_p0d.data() : (const void *)h_p0f.data(), pv * (size_t)n_sites);
        H2D(c->d_p1, p64 ? (const void *)h_p1d.data() : (const void *)h_p1f.data(), pv * (size_t)n_sites);
        H2D(c->d_pk, p64 ? (const void *)h_pkd.data() : (const void *)h_pkf.data(), ps * (size_t)n_sites);
    }
    if (!h_qis.empty()) {
        DALLOC(c->d_qis, sizeof(int32_t) * (size_t)n_sites);
        H2D(c->d_qis, h_qis.data(), sizeof(int32_t) * (size_t)n_sites);
    }
    if (any_policy && p64) {
        DALLOC(c->d_pol, sizeof(PolicySite) * (size_t)n_sites);
        H2D(c->d_pol, h_pol.data(), sizeof(PolicySite) * (size_t)n_sites);
    } else if (any_policy) {
        DALLOC(c->d_pol32, sizeof(PolicySite32) * (size_t)n_sites);
        H2D(c->d_pol32, h_pol32.data(), sizeof(PolicySite32) * (size_t)n_sites);
    }
    {  // accepted-attempt counters; widths of the adaptive policy and the sites they divide by
        DALLOC(c->d_acc, sizeof(uint32_t) * (size_t)c->n_inst);
        DALLOC(c->d_sigma, sizeof(double) * (size_t)c->n_inst);
        DALLOC(c->d_adapt_n, sizeof(int32_t) * (size_t)c->n_inst);
        std::vector<double> h_sigma((size_t)c->n_inst, 0.0);
        std::vector<int32_t> h_an((size_t)c->n_inst, 0);
        for (int32_t s = 0; s < n_samples; ++s)
            for (int32_t r = 0; r < R; ++r) {
                const SampleInfo &si = c->samples[(size_t)s];
                h_sigma[(size_t)(s * R + r)] = si.has_adaptive ? si.sigma0 : 0.0;
                h_an[(size_t)(s * R + r)] = si.has_adaptive ? si.n : 0;
            }
        H2D(c->d_sigma, h_sigma.data(), sizeof(double) * (size_t)c->n_inst);
        H2D(c->d_adapt_n, h_an.data(), sizeof(int32_t) * (size_t)c->n_inst);
        if (cudaMemsetAsync(c->d_acc, 0, sizeof(uint32_t) * (size_t)c->n_inst, c->stream) != cudaSuccess) {
            c->err = "memset failed";
            return bail(VEGAS_ECUDA);
        }
    }
    if (cudaMemsetAsync(c->d_err, 0, 4 * sizeof(uint32_t), c->stream) != cudaSuccess) {
        c->err = "memset failed";
        return bail(VEGAS_ECUDA);
    }
    if (o.accept_log_mcs > 0) {
        c->alog_bytes = (int64_t)o.accept_log_mcs * n_sites * R;
        DALLOC(c->d_alog, (size_t)c->alog_bytes);
        if (cudaMemsetAsync(c->d_alog, 0, (size_t)c->alog_bytes, c->stream) != cudaSuccess) {
            c->err = "memset failed";
            return bail(VEGAS_ECUDA);
        }
    }

    // ---- sweep launches, one per non-empty colour class of each sample (per type segment of a
    // class with per-type statistics: sites are stored type by type inside each class)
    int64_t alog_base = 0;
    for (int32_t s = 0; s < n_samples; ++s) {
        SampleInfo &si = c->samples[(size_t)s];
        for (int32_t col = 0; col < si.n_colours; ++col)
          for (int32_t sb = si.cstart[(size_t)col]; sb < si.cstart[(size_t)col + 1];) {
            int32_t se = si.cstart[(size_t)col + 1];
            const int32_t ty = si.type.empty() ? 0 : si.type[(size_t)sb];
            if (!si.type.empty())
                for (int32_t g = sb; g < se; ++g)
                    if (si.type[(size_t)g] != ty) {
                        se = g;
                        break;
                    }
            const int32_t nc = se - sb;
            PassLaunch pl;
            pl.sample = s;
            pl.group = ty;
            pl.col = col;
            PassArgs &a = pl.args;
            std::memset(&a, 0, sizeof a);
            a.spins = c->d_spins;
            a.edges = c->d_edges;
            a.row_ptr = c->d_rowptr;
            a.orig = c->d_orig;
            a.p0 = si.uniform_params ? nullptr : c->d_p0;
            a.p1 = si.uniform_params ? nullptr : c->d_p1;
            a.pk = si.uniform_params ? nullptr : c->d_pk;
            a.pol = si.has_policy ? c->d_pol : nullptr;
            a.pol32 = si.has_policy ? c->d_pol32 : nullptr;
            a.pol_fixed = -1;
            if (a.pol32 && nc > 0) {  // one policy over the whole pass: a specialised kernel
                const int32_t g0 = si.site_off + sb, code = h_pol32[(size_t)g0].code;
                bool same = true;
                for (int32_t g = g0 + 1; g < si.site_off + se && same; ++g) same = h_pol32[(size_t)g].code == code;
                if (same) a.pol_fixed = code;
            }
            a.run = c->d_run;
            a.err = c->d_err;
            a.alog = c->d_alog;
            a.seed = o.seed;
            a.edge_base = si.edge_off;
            a.site_off = si.site_off;
            a.g_begin = si.site_off + sb;
            a.g_end = si.site_off + se;
            a.lower_end = si.site_off + si.cstart[(size_t)col];  // the class start: lower colours below
            a.log2R = c->log2R;
            a.inst0 = o.inst_base + s * R;
            a.inst_local0 = s * R;
            a.n_inst = c->n_inst;
            a.n_sample_sites = si.n;
            a.alog_stride = (int64_t)n_sites * R;
            a.alog_base = alog_base;
            a.alog_mcs = (uint32_t)o.accept_log_mcs;
            a.deg = si.uniform_degree;
            a.n_sites_total = (int32_t)n_sites;
            a.n_edges_total = n_edges;
            a.lower_mode = si.lower_mode[(size_t)col];
            a.params_mode = si.uniform_params ? (si.has_anisotropy ? 1 : 0) : 2;
            // measured on the 32 x 256^3 spin glass: depth 2 keeps 3 blocks per SM for R >= 16
            // (2.93 ms per class vs 3.07 ms at depth 3 and 4.32 ms at depth 4, which fits only
            // one block per SM); with fewer replicas the deeper pipeline was marginally faster
            a.depth = (o.pipeline_depth == 0) ? (c->R >= 16 ? 2 : 3) : (o.pipeline_depth == 1 ? 0 : o.pipeline_depth);
            a.u64 = si.u;
            a.u32 = SiteParams32{(float)si.u.nx, (float)si.u.ny, (float)si.u.nz, (float)si.u.s, (float)si.u.ex,
                                 (float)si.u.ey, (float)si.u.ez, (float)si.u.k,  (float)si.u.kc};
            const int64_t work = (int64_t)nc * R;
            if (c->precision == 64) {
                // an SM runs few FP64 operations per clock: spread a small class over many SMs
                // (blocks of 32 .. kThreads threads, about one block per SM)
                const int64_t per_sm = (work + c->sm_count - 1) / c->sm_count;
                pl.threads = (int)std::min<int64_t>(kThreads, std::max<int64_t>(32, (per_sm + 31) / 32 * 32));
            }
            if (c->precision != 64) pl.threads = pass32_threads(a);  // the R = 32 kernel runs 7-warp blocks
            const int64_t need = (work + pl.threads - 1) / pl.threads;
            int64_t cap = (int64_t)c->sm_count * pass_blocks_per_sm(c->precision, a);
            if (o.max_blocks > 0) cap = std::min<int64_t>(cap, o.max_blocks);
            pl.grid = (int)std::max<int64_t>(1, std::min(need, cap));
            a.partial = nullptr;  // set below, once the slot buffer exists
            c->passes.push_back(pl);
            sb = se;
          }
        alog_base += (int64_t)si.n * R;
    }
    // block slots grouped by (sample, type group), passes of a group in sweep order
    const int32_t NG = c->n_groups;
    std::vector<int64_t> h_sb((size_t)n_samples * NG, 0);
    std::vector<int32_t> h_sc((size_t)n_samples * NG, 0);
    int64_t slots = 0;
    for (int32_t s = 0; s < n_samples; ++s)
        for (int32_t k = 0; k < NG; ++k) {
            h_sb[(size_t)(s * NG + k)] = slots;
            for (PassLaunch &pl : c->passes)
                if (pl.sample == s && (NG == 1 || pl.group == k)) {
                    pl.slot = slots;
                    h_sc[(size_t)(s * NG + k)] += pl.grid;
                    slots += pl.grid;
                }
        }
    DALLOC(c->d_partial, sizeof(double) * 4 * (size_t)std::max<int64_t>(slots, 1) * R);
    for (PassLaunch &pl : c->passes) pl.args.partial = c->d_partial + pl.slot * R * 4;
    DALLOC(c->d_pass_tickets, sizeof(uint32_t) * std::max<size_t>(c->passes.size(), 1));
    if (cudaMemsetAsync(c->d_pass_tickets, 0, sizeof(uint32_t) * std::max<size_t>(c->passes.size(), 1), c->stream) !=
        cudaSuccess) {
        c->err = "memset failed";
        return bail(VEGAS_ECUDA);
    }
    for (size_t k = 0; k < c->passes.size(); ++k) c->passes[k].args.ticket = c->d_pass_tickets + k;
    // the sweep's launches of one MCS, class by class: the direct FP32 passes of a class that
    // share a kernel go out as one launch, every other pass alone
    {
        int32_t n_col = 0;
        for (const PassLaunch &pl : c->passes) n_col = std::max(n_col, pl.col + 1);
        for (int32_t col = 0; col < n_col; ++col) {
            std::vector<LaunchGroup> merged;  // by kernel: params mode, lower mode, policy table
            std::vector<int> keys;
            for (size_t k = 0; k < c->passes.size(); ++k) {
                const PassLaunch &pl = c->passes[k];
                if (pl.col != col) continue;
                const PassArgs &a = pl.args;
                if (c->precision == 64 || !pass32_direct(a)) {
                    LaunchGroup lg;
                    lg.passes.push_back((int)k);
                    c->launches.push_back(lg);
                    continue;
                }
                const int key = (a.params_mode * 3 + a.lower_mode) * 2 + (a.pol32 ? 1 : 0);
                size_t q = 0;
                while (q < keys.size() && keys[q] != key) ++q;
                if (q == keys.size()) {
                    keys.push_back(key);
                    merged.emplace_back();
                }
                merged[q].passes.push_back((int)k);
            }
            for (LaunchGroup &lg : merged) {
                if (lg.passes.size() > 1) {
                    std::vector<PassArgs> args;
                    std::vector<int32_t> first(1, 0);
                    for (int k : lg.passes) {
                        args.push_back(c->passes[(size_t)k].args);
                        first.push_back(first.back() + c->passes[(size_t)k].grid);
                    }
                    lg.grid = first.back();
                    c->launches.push_back(lg);  // owns the buffers from here (freed with the context)
                    LaunchGroup &own = c->launches.back();
                    DALLOC(own.d_args, sizeof(PassArgs) * args.size());
                    DALLOC(own.d_first, sizeof(int32_t) * first.size());
                    H2D(own.d_args, args.data(), sizeof(PassArgs) * args.size());
                    H2D(own.d_first, first.data(), sizeof(int32_t) * first.size());
                    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {  // the host vectors go out of scope
                        c->err = "upload of the merged passes failed";
                        return bail(VEGAS_ECUDA);
                    }
                } else {
                    c->launches.push_back(lg);
                }
            }
        }
    }
    DALLOC(c->d_slot_base, sizeof(int64_t) * h_sb.size());
    DALLOC(c->d_slot_count, sizeof(int32_t) * h_sc.size());
    H2D(c->d_slot_base, h_sb.data(), sizeof(int64_t) * h_sb.size());
    H2D(c->d_slot_count, h_sc.data(), sizeof(int32_t) * h_sc.size());
    RunState rs0{};
    rs0.mcs = 1;
    H2D(c->d_run, &rs0, sizeof rs0);

    // ---- resident sweep: one entry per instance, largest first
    if (!p64) {
        std::vector<ResidentInst> insts;
        int32_t any_aniso = 0;  // some instance with anisotropy or per-site parameters
        std::vector<int32_t> h_cs;  // class starts (cooperative sweep)
        std::vector<int4> h_segs;   // sweep segments (resident sweep)
        int64_t alog_off = 0;
        for (int32_t s = 0; s < n_samples; ++s) {
            const SampleInfo &si = c->samples[(size_t)s];
            const int32_t seg_off = (int32_t)h_segs.size();
            for (int32_t q = 0; q <= si.n_colours; ++q) h_cs.push_back(si.site_off + si.cstart[(size_t)q]);
            for (const PassLaunch &pl : c->passes)  // the passes of this sample, in sweep order
                if (pl.sample == s) {
                    const bool last = pl.args.g_end == si.site_off + si.cstart[(size_t)pl.col + 1];
                    h_segs.push_back(make_int4(pl.args.g_begin, pl.args.g_end, pl.args.lower_end,
                                               pl.group | ((last ? 1 : 0) << 16)));
                }
            const int32_t n_segs = (int32_t)h_segs.size() - seg_off;
            c->max_instance_sites = std::max(c->max_instance_sites, si.n);
            c->min_instance_sites = c->min_instance_sites == 0 ? si.n : std::min(c->min_instance_sites, si.n);
            for (int32_t r = 0; r < R; ++r) {
                ResidentInst I;
                std::memset(&I, 0, sizeof I);
                I.g_begin = si.site_off;
                I.g_end = si.site_off + si.n;
                I.seg_off = seg_off;
                I.n_segs = n_segs;
                I.inst_id = o.inst_base + s * R + r;
                I.inst_local = s * R + r;
                I.r = r;
                I.params_mode = si.uniform_params ? (si.has_anisotropy ? 1 : 0) : 2;
                if (I.params_mode != 0) any_aniso = 1;
                I.n_sample_sites = si.n;
                I.adaptive = si.has_adaptive ? 1 : 0;
                I.alog_base = alog_off;
                I.u = SiteParams32{(float)si.u.nx, (float)si.u.ny, (float)si.u.nz, (float)si.u.s, (float)si.u.ex,
                                   (float)si.u.ey, (float)si.u.ez, (float)si.u.k,  (float)si.u.kc};
                insts.push_back(I);
            }
            alog_off += (int64_t)si.n * R;
        }
        std::stable_sort(insts.begin(), insts.end(), [](const ResidentInst &x, const ResidentInst &y) {
            return (x.g_end - x.g_begin) > (y.g_end - y.g_begin);
        });
        DALLOC(c->d_insts, sizeof(ResidentInst) * insts.size());
        DALLOC(c->d_cstart, sizeof(int32_t) * h_cs.size());
        DALLOC(c->d_segs, sizeof(int4) * std::max<size_t>(h_segs.size(), 1));
        DALLOC(c->d_queue, sizeof(uint32_t));
        H2D(c->d_insts, insts.data(), sizeof(ResidentInst) * insts.size());
        H2D(c->d_cstart, h_cs.data(), sizeof(int32_t) * h_cs.size());
        if (!h_segs.empty()) H2D(c->d_segs, h_segs.data(), sizeof(int4) * h_segs.size());
        c->res_items = (int)insts.size();
        c->res_policy = any_policy;
        ResidentArgs &ra = c->res;
        std::memset(&ra, 0, sizeof ra);
        ra.any_aniso = any_aniso;
        // spins in shared memory: every instance fits at 12 bytes per site and every row in a
        // fixed row of kEllRow links (the form reads links without row offsets)
        int64_t max_deg = 0;
        for (int64_t g = 0; g < n_sites; ++g) max_deg = std::max(max_deg, h_rowptr[(size_t)g + 1] - h_rowptr[(size_t)g]);
        c->res_smem_eligible = o.resident_smem >= 0 && 12 * (int64_t)c->max_instance_sites <= kResSmemBytes &&
                               max_deg <= kEllRow;
        if (c->res_smem_eligible) {
            std::vector<int2> h_ell((size_t)n_sites * kEllRow, make_int2(-1, 0));
            for (int64_t g = 0; g < n_sites; ++g)
                for (int64_t e = h_rowptr[(size_t)g]; e < h_rowptr[(size_t)g + 1]; ++e)
                    h_ell[(size_t)g * kEllRow + (size_t)(e - h_rowptr[(size_t)g])] = h_e32[(size_t)e];
            DALLOC(c->d_ell, sizeof(int2) * h_ell.size());
            H2D(c->d_ell, h_ell.data(), sizeof(int2) * h_ell.size());
        }
        if (o.resident_smem == 1 && !c->res_smem_eligible) {
            c->err = "resident_smem = 1: the largest instance does not fit in shared memory (12 bytes per site, at "
                     "most " + std::to_string(kResSmemBytes / 12) + " sites)";
            return bail(VEGAS_EINVAL);
        }
        if (o.resident_smem == 1)
            set_resident_shape(c, 512, o.group_threads, o.group_sites, true);
        else
            set_resident_shape(c, c->max_instance_sites >= 4096 ? 512 : 256, o.group_threads, o.group_sites);
        ra.spins = c->d_spins;
        ra.edges = c->d_edges;
        ra.ell = (const int4 *)c->d_ell;
        ra.row_ptr = c->d_rowptr;
        ra.orig = c->d_orig;
        ra.p0 = c->d_p0;
        ra.p1 = c->d_p1;
        ra.pk = c->d_pk;
        ra.pol = any_policy ? c->d_pol32 : nullptr;
        ra.insts = c->d_insts;
        ra.segs = c->d_segs;
        ra.n_types = c->n_types;
        ra.queue = c->d_queue;
        ra.run = c->d_run;
        ra.err = c->d_err;
        ra.alog = c->d_alog;
        ra.seed = o.seed;
        ra.alog_stride = (int64_t)n_sites * R;
        ra.alog_mcs = (uint32_t)o.accept_log_mcs;
        ra.n_items = (int32_t)insts.size();
        ra.n_inst = c->n_inst;
        ra.log2R = c->log2R;
        // one block per instance only pays while instances are small; the resident sweep keeps
        // per-type sums for at most 8 types
        c->res_eligible = c->max_instance_sites <= (1 << 18) && c->n_types <= 8;
        // cluster sweep: about 2048 sites per block of the cluster, 2 .. 16 blocks of 256 threads
        // (measured on the 29k-site core/shell particle: 0.63 G attempts/s with 16 x 256 threads,
        // 0.54 with 16 x 512)
        if (c->n_types <= 8) {
            int cs = 2;
            while (cs < 16 && (int64_t)cs * 2048 < c->max_instance_sites) cs *= 2;
            const int nt = o.cluster_threads > 0 ? o.cluster_threads : 256;
            if (o.cluster_blocks > 0) cs = o.cluster_blocks;
            int cap = cluster_capacity(cs, nt, any_policy);
            if (cap == 0 && cs == 16 && o.cluster_blocks == 0) {
                cs = 8;
                cap = cluster_capacity(cs, nt, any_policy);
            }
            c->cluster_threads = nt;
            if (cap > 0) {
                c->cluster_eligible = set_cluster_shape(c, cs, nt, o.cluster_split, -1, 0,
                                                        o.variant == 3 && o.resident_smem == 1);
            }
            cudaGetLastError();  // an unsupported cluster shape only makes the sweep ineligible
        }
    }
    // ---- cooperative sweep: one sample, every block on every class
    if (n_samples == 1 && !c->passes.empty() && !c->any_adaptive && !o.type_stats) {
        const int nt = kCoopThreads;
        // FP32 rows of at most kEllRow links other than the sc lattices' six: fixed padded rows
        // (the resident sweep's, or built here), read without row offsets
        const int deg0 = c->passes[0].args.deg;
        bool use_ell = false;
        if (!p64 && deg0 != 6) {
            int64_t max_deg = 0;
            for (int64_t g = 0; g < n_sites; ++g)
                max_deg = std::max(max_deg, h_rowptr[(size_t)g + 1] - h_rowptr[(size_t)g]);
            if (max_deg <= kEllRow) {
                if (!c->d_ell) {
                    std::vector<int2> h_ell((size_t)n_sites * kEllRow, make_int2(-1, 0));
                    for (int64_t g = 0; g < n_sites; ++g)
                        for (int64_t e = h_rowptr[(size_t)g]; e < h_rowptr[(size_t)g + 1]; ++e)
                            h_ell[(size_t)g * kEllRow + (size_t)(e - h_rowptr[(size_t)g])] = h_e32[(size_t)e];
                    DALLOC(c->d_ell, sizeof(int2) * h_ell.size());
                    H2D(c->d_ell, h_ell.data(), sizeof(int2) * h_ell.size());
                    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {  // h_ell goes out of scope
                        c->err = "upload of the fixed link rows failed";
                        return bail(VEGAS_ECUDA);
                    }
                }
                use_ell = true;
            }
        }
        const int form = p64 ? 0 : (deg0 == 6 ? 6 : (use_ell ? kEllRow : 0));
        c->coop_grid_max = c->sm_count * coop_blocks_per_sm(any_policy, form, p64);
        if (o.max_blocks > 0) c->coop_grid_max = std::min(c->coop_grid_max, o.max_blocks);
        const SampleInfo &si = c->samples[0];
        {  // no more blocks than one thread per site and replica of the largest class: a small
           // sample's grid barriers then wait on the blocks that have work only
            int64_t widest = 0;
            for (int32_t q = 0; q < si.n_colours; ++q)
                widest = std::max<int64_t>(widest, (int64_t)(si.cstart[(size_t)q + 1] - si.cstart[(size_t)q]) * R);
            // FP64: down to one site and replica group per block (a block's FP64 work is what bounds it)
            const int64_t per_block = p64 ? R : nt;
            c->coop_grid_max =
                (int)std::max<int64_t>(1, std::min<int64_t>(c->coop_grid_max, (widest + per_block - 1) / per_block));
        }
        if (p64) {  // the class starts (FP32 contexts built them with the resident sweep's tables)
            std::vector<int32_t> h_cs;
            for (int32_t q = 0; q <= si.n_colours; ++q) h_cs.push_back(si.site_off + si.cstart[(size_t)q]);
            DALLOC(c->d_cstart, sizeof(int32_t) * h_cs.size());
            H2D(c->d_cstart, h_cs.data(), sizeof(int32_t) * h_cs.size());
            if (cudaStreamSynchronize(c->stream) != cudaSuccess) {  // h_cs goes out of scope
                c->err = "upload of the class starts failed";
                return bail(VEGAS_ECUDA);
            }
        }
        set_coop_shape(c, 2);
        DALLOC(c->d_bar, sizeof(GridBarrier));
        DALLOC(c->d_coop_partial, sizeof(double) * 4 * 2 * (size_t)c->coop_grid_max * R);  // two MCS in turn
        CoopArgs &ca = c->coop;
        std::memset(&ca, 0, sizeof ca);
        ca.pass = c->passes[0].args;
        ca.pass.lower_mode = 2;
        ca.cstart = c->d_cstart;
        ca.n_colours = c->samples[0].n_colours;
        ca.bar = c->d_bar;
        ca.partial = c->d_coop_partial;
        ca.timeout_ns = o.timeout_ns > 0 ? o.timeout_ns : 2000000000LL;
        ca.skip_block = o.fault_inject == 1 ? 0 : -1;
        ca.fp64 = p64 ? 1 : 0;
        ca.ell = use_ell ? c->d_ell : nullptr;
        c->coop_eligible = true;
    }
    // ---- renormalisation folded into the step's last class-1 pass: one sample of two colour
    // classes swept by the R = 32 kernel without a policy table (every class-1 link to class 0),
    // no discrete-valued sites, every class-0 block read by some class-1 block
    if (c->precision == 32 && o.renorm_fold == 0 && n_samples == 1 && c->R == 32 && c->passes.size() == 2 &&
        !c->d_qis && c->samples[0].n_colours == 2) {
        const SampleInfo &si = c->samples[0];
        const PassArgs &p0 = c->passes[0].args, &p1 = c->passes[1].args;
        const bool whole = p0.g_begin == si.site_off && p0.g_end == si.site_off + si.cstart[1] &&
                           p1.g_begin == si.site_off + si.cstart[1] && p1.g_end == si.site_off + si.cstart[2];
        std::vector<int32_t> deps, last;
        if (whole && p1.lower_mode == 1 && pass32_kind(p0) == VEGAS_KERNEL_PASS32_R32 &&
            pass32_kind(p1) == VEGAS_KERNEL_PASS32_R32 &&
            class1_block_deps(si, L[0], kFoldBlockSites, kFoldDeps, deps, last)) {
            const int32_t nb0 = (si.cstart[1] + kFoldBlockSites - 1) / kFoldBlockSites;
            std::vector<int32_t> deg((size_t)nb0, 0);
            for (int32_t d : deps)
                if (d >= 0) deg[(size_t)d]++;
            if (nb0 > 0 && std::find(deg.begin(), deg.end(), 0) == deg.end()) {
                DALLOC(c->d_fold_deps, sizeof(int32_t) * deps.size());
                DALLOC(c->d_fold_deg, sizeof(int32_t) * deg.size());
                DALLOC(c->d_fold_cnt, sizeof(uint32_t) * deg.size());
                H2D(c->d_fold_deps, deps.data(), sizeof(int32_t) * deps.size());
                H2D(c->d_fold_deg, deg.data(), sizeof(int32_t) * deg.size());
                if (cudaMemsetAsync(c->d_fold_cnt, 0, sizeof(uint32_t) * deg.size(), c->stream) != cudaSuccess ||
                    cudaStreamSynchronize(c->stream) != cudaSuccess) {  // the host vectors go out of scope
                    c->err = "upload of the class-1 block reads failed";
                    return bail(VEGAS_ECUDA);
                }
                PassArgs &fa = c->fold_args;
                fa = p1;
                fa.fold_deps = c->d_fold_deps;
                fa.fold_deg = c->d_fold_deg;
                fa.fold_cnt = c->d_fold_cnt;
                fa.fold_norm = c->d_norm;
                fa.fold_c0_begin = p0.g_begin;
                fa.fold_c0_end = p0.g_end;
                // sets the kernel's shared-memory limit; the same block shape as the plain pass
                const bool same_shape = pass_blocks_per_sm(32, fa) == pass_blocks_per_sm(32, p1) &&
                                        pass32_threads(fa) == pass32_threads(p1) && pass32_smem(fa) == pass32_smem(p1);
                if (cudaGetLastError() != cudaSuccess || !same_shape) {
                    c->err = "the renormalising class-1 pass does not fit beside the plain one";
                    return bail(VEGAS_ECUDA);
                }
                c->fold_nb0 = nb0;
                c->fold_ok = true;
            }
        }
    }
    // ---- wavefront sweep: task order and completion flags
    if (o.variant == 4) {
        const SampleInfo &si = c->samples[0];
        const LoadedSample &l = L[0];
        const PassArgs &p0 = c->passes[0].args;
        const int bps = wave_blocks_per_sm(p0.params_mode);
        if (bps < 1) {
            c->err = "the wavefront sweep kernel does not fit on this device";
            return bail(VEGAS_ECUDA);
        }
        c->wave_grid = c->sm_count * bps;
        if (o.max_blocks > 0) c->wave_grid = std::min(c->wave_grid, o.max_blocks);
        const int64_t W = (int64_t)c->wave_grid * (kThreads / 32);
        const int32_t n0 = si.cstart[1], n1 = si.cstart[2] - si.cstart[1];
        constexpr int BS = kWaveBlockSites;
        const int32_t nb0 = (n0 + BS - 1) / BS, nb1 = (n1 + BS - 1) / BS;
        // the class-0 blocks that class-1 block q links to (distinct, ascending; D: the last)
        std::vector<int32_t> D, deps;
        if (!class1_block_deps(si, l, BS, kWaveDeps, deps, D)) {
            c->err = "the wavefront sweep needs every block of " + std::to_string(BS) +
                     " class-1 sites to link to at most " + std::to_string(kWaveDeps) + " blocks of class-0 sites";
            return bail(VEGAS_EINVAL);
        }
        // class-0 blocks in memory order; each class-1 block after class-0 block
        // min(D + lag, nb0 - 1), so every dependency comes earlier in the list
        const int64_t lag = o.wave_lag > 0 ? o.wave_lag : W;
        std::vector<int32_t> first((size_t)nb0 + 1, 0), after((size_t)nb1);
        for (int32_t q = 0; q < nb1; ++q) {
            after[(size_t)q] = (int32_t)std::min<int64_t>((int64_t)D[(size_t)q] + lag, nb0 - 1);
            first[(size_t)after[(size_t)q] + 1]++;
        }
        for (int32_t j = 0; j < nb0; ++j) first[(size_t)j + 1] += first[(size_t)j];
        std::vector<int32_t> byj((size_t)nb1), fill(first.begin(), first.end() - 1);
        for (int32_t q = 0; q < nb1; ++q) byj[(size_t)fill[(size_t)after[(size_t)q]]++] = q;
        std::vector<int32_t> tasks;
        tasks.reserve((size_t)nb0 + nb1);
        std::vector<int64_t> pos0((size_t)nb0);
        for (int32_t j = 0; j < nb0; ++j) {
            pos0[(size_t)j] = (int64_t)tasks.size();
            tasks.push_back(j);
            for (int32_t k = first[(size_t)j]; k < first[(size_t)j + 1]; ++k) tasks.push_back(nb0 + byj[(size_t)k]);
        }
        for (int64_t m = 0; m < (int64_t)tasks.size(); ++m)  // the order the progress argument needs
            if (tasks[(size_t)m] >= nb0 && pos0[(size_t)D[(size_t)(tasks[(size_t)m] - nb0)]] >= m) {
                c->err = "wavefront task order: a class-1 block before one of its dependencies";
                return bail(VEGAS_EINVAL);
            }
        DALLOC(c->d_tasks, sizeof(int32_t) * tasks.size());
        DALLOC(c->d_deps, sizeof(int32_t) * std::max<size_t>(deps.size(), 1));
        DALLOC(c->d_done, sizeof(uint32_t) * (size_t)nb0);
        DALLOC(c->d_ticket, sizeof(uint32_t));
        DALLOC(c->d_wave_partial, sizeof(double) * 4 * (size_t)c->wave_grid * R);
        DALLOC(c->d_wave_slot_base, sizeof(int64_t));
        DALLOC(c->d_wave_slot_count, sizeof(int32_t));
        H2D(c->d_tasks, tasks.data(), sizeof(int32_t) * tasks.size());
        if (!deps.empty()) H2D(c->d_deps, deps.data(), sizeof(int32_t) * deps.size());
        const int64_t zero = 0;
        const int32_t gcount = c->wave_grid;
        H2D(c->d_wave_slot_base, &zero, sizeof zero);
        H2D(c->d_wave_slot_count, &gcount, sizeof gcount);
        if (cudaMemsetAsync(c->d_done, 0, sizeof(uint32_t) * (size_t)nb0, c->stream) != cudaSuccess) {
            c->err = "memset failed";
            return bail(VEGAS_ECUDA);
        }
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) {  // the host vectors above go out of scope
            c->err = "upload of the wavefront task order failed";
            return bail(VEGAS_ECUDA);
        }
        WaveArgs &wa = c->wave;
        std::memset(&wa, 0, sizeof wa);
        wa.pass = p0;
        wa.pass.partial = c->d_wave_partial;
        wa.tasks = c->d_tasks;
        wa.deps = c->d_deps;
        wa.ticket = c->d_ticket;
        wa.done = c->d_done;
        wa.n_tasks = (int32_t)tasks.size();
        wa.nb0 = nb0;
        wa.c1_begin = si.site_off + si.cstart[1];
        wa.c1_end = si.site_off + si.cstart[2];
        wa.timeout_ns = o.timeout_ns > 0 ? o.timeout_ns : 2000000000LL;
        wa.skip_block = o.fault_inject == 1 ? 0 : -1;
        c->variant = 4;
        c->tuned = true;
    } else if (o.variant == 2) {
        if (!c->coop_eligible) {
            c->err = "variant 2 (cooperative) does not run samples with the adaptive policy";
            return bail(VEGAS_EINVAL);
        }
        c->variant = 2;
        c->tuned = true;
    } else if (o.variant == 3) {
        if (!c->cluster_eligible) {
            c->err = "variant 3 (cluster) needs FP32, at most 8 tracked types and a device with thread-block clusters";
            return bail(VEGAS_EINVAL);
        }
        c->variant = 3;
        c->tuned = true;
    } else if (o.variant == 1) {
        if (!c->res_eligible) {
            c->err = "variant 1 (resident) needs FP32, samples of at most 262144 sites and at most 8 tracked types";
            return bail(VEGAS_EINVAL);
        }
        c->variant = 1;
        c->tuned = true;
    } else if (o.variant == 0 || (!c->res_eligible && !c->coop_eligible && !c->cluster_eligible)) {
        c->variant = 0;
        c->tuned = true;
    } else {
        // automatic: timed on the first run; until then, the shape suggests one
        c->variant = (c->res_eligible && c->n_inst >= 2 && c->max_instance_sites <= 16384) ? 1 : 0;
    }

    // ---- initial state
    for (int32_t s = 0; s < n_samples; ++s) {
        const SampleInfo &si = c->samples[(size_t)s];
        double *d_given = nullptr;
        const LoadedSample &l = L[(size_t)s];
        if (!l.init_spins.empty()) {
            if (cudaMalloc(&d_given, sizeof(double) * l.init_spins.size()) != cudaSuccess) {
                c->err = "cudaMalloc for initial spins failed";
                return bail(VEGAS_ENOMEM);
            }
            H2D(d_given, l.init_spins.data(), sizeof(double) * l.init_spins.size());
        }
        InitArgs ia{c->d_spins, c->d_orig, c->d_norm, d_given, c->d_err, o.seed, si.site_off, si.site_off + si.n,
                    o.inst_base + s * R, c->log2R, c->d_qis};
        const int64_t work = (int64_t)si.n * R;
        const int grid = (int)std::min<int64_t>((work + 255) / 256, (int64_t)c->sm_count * 8);
        if (p64)
            launch_init64(ia, grid, c->stream);
        else
            launch_init32(ia, grid, c->stream);
        c->kernel_launches++;
        if (d_given) {
            cudaError_t e = cudaStreamSynchronize(c->stream);
            cudaFree(d_given);
            if (e != cudaSuccess) {
                c->err = std::string("initial state: ") + cudaGetErrorString(e);
                return bail(VEGAS_ECUDA);
            }
        }
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->err = std::string("create: ") + cudaGetErrorString(e);
        return bail(VEGAS_ECUDA);
    }
    c->hist.assign((size_t)c->n_inst, std::vector<double>());
    c->acc_hist.assign((size_t)c->n_inst, std::vector<uint32_t>());
    c->type_hist.assign((size_t)c->n_inst, std::vector<double>());
    c->snaps.assign((size_t)c->n_inst, std::vector<double>());
#undef TRY
#undef DALLOC
#undef H2D
    *out = c;
    return VEGAS_OK;
}

extern "C" vegas_status vegas_create(const vegas_sample *samples, int32_t n_samples, const vegas_options *opt,
                                     vegas_ctx **out) {
    vegas_ctx *made = nullptr;
    try {
        return create_context(samples, n_samples, opt, out, &made);
    } catch (...) {
        const vegas_status st = host_exception(nullptr);
        if (made) {
            free_all(made);
            delete made;
        }
        if (out) *out = nullptr;
        return st;
    }
}

extern "C" vegas_status vegas_run(vegas_ctx *c, const double *T, const double *B, int32_t n_steps, int32_t mcs) {
    try {
        vegas_status st = check_usable(c);
        if (st != VEGAS_OK) return st;
        if (n_steps < 0 || mcs < 0) return fail(c, VEGAS_EINVAL, "n_steps and mcs_per_step must be >= 0");
        if (n_steps == 0 || mcs == 0) return VEGAS_OK;
        if (!T || !B) return fail(c, VEGAS_EINVAL, "T or B is NULL");
        const int64_t NI = c->n_inst;
        if ((int64_t)c->t + (int64_t)n_steps * mcs >= (int64_t)UINT32_MAX)
            return fail(c, VEGAS_EINVAL, "global MCS counter would exceed 32 bits");
        std::vector<double> sched((size_t)n_steps * NI * 2);
        for (int64_t i = 0; i < NI; ++i)
            for (int32_t s = 0; s < n_steps; ++s) {
                const double Ti = T[i * n_steps + s], Bi = B[i * n_steps + s];
                if (!(Ti > 0.0) || !std::isfinite(Ti)) return fail(c, VEGAS_EINVAL, "T must be finite and > 0");
                if (!std::isfinite(Bi)) return fail(c, VEGAS_EINVAL, "B must be finite");
                sched[((size_t)s * NI + i) * 2] = 1.0 / Ti;
                sched[((size_t)s * NI + i) * 2 + 1] = Bi;
            }
        if ((st = set_device(c)) != VEGAS_OK) return st;
        NvtxRange run_range("vegas_run");
        const int64_t nrec = (int64_t)n_steps * mcs;
        if (sched.size() > c->sched_cap) {
            if (c->d_sched) {
                cudaFree(c->d_sched);
                c->device_bytes -= (int64_t)(c->sched_cap * sizeof(double));
            }
            c->sched_cap = 0;
            CK(c, dalloc(c, &c->d_sched, sizeof(double) * sched.size()));
            c->sched_cap = sched.size();
        }
        const size_t hneed = (size_t)nrec * NI * 4;
        if (hneed > c->hist_cap) {
            if (c->d_hist) {
                cudaFree(c->d_hist);
                c->device_bytes -= (int64_t)(c->hist_cap * sizeof(double));
            }
            c->hist_cap = 0;
            CK(c, dalloc(c, &c->d_hist, sizeof(double) * hneed));
            c->hist_cap = hneed;
        }
        const size_t aneed = (size_t)nrec * NI;
        if (aneed > c->acc_hist_cap) {
            if (c->d_acc_hist) {
                cudaFree(c->d_acc_hist);
                c->device_bytes -= (int64_t)(c->acc_hist_cap * sizeof(uint32_t));
            }
            c->acc_hist_cap = 0;
            CK(c, dalloc(c, &c->d_acc_hist, sizeof(uint32_t) * aneed));
            c->acc_hist_cap = aneed;
        }
        const size_t tneed = (size_t)nrec * NI * (size_t)c->n_types * 3;
        if (tneed > c->type_hist_cap) {
            if (c->d_type_hist) {
                cudaFree(c->d_type_hist);
                c->device_bytes -= (int64_t)(c->type_hist_cap * sizeof(double));
            }
            c->type_hist_cap = 0;
            CK(c, dalloc(c, &c->d_type_hist, sizeof(double) * tneed));
            c->type_hist_cap = tneed;
        }
        const int64_t vbytes = c->precision == 64 ? 32 : 16;
        const size_t sneed = c->opt.snapshots ? (size_t)n_steps * (size_t)(c->n_sites * c->R * vbytes) : 0;
        if (sneed > c->snap_cap) {
            if (c->d_snap) {
                cudaFree(c->d_snap);
                c->device_bytes -= (int64_t)c->snap_cap;
            }
            c->snap_cap = 0;
            CK(c, dalloc(c, &c->d_snap, sneed));
            c->snap_cap = sneed;
        }
        CK(c, cudaMemcpyAsync(c->d_sched, sched.data(), sizeof(double) * sched.size(), cudaMemcpyHostToDevice, c->stream));
        RunState rs{};
        rs.t = c->t;
        rs.rec = 0;
        rs.ticket = 0;
        rs.mcs = (uint32_t)mcs;
        rs.sched = c->d_sched;
        rs.hist = c->d_hist;
        rs.acc = c->d_acc;
        rs.acc_hist = c->d_acc_hist;
        rs.sigma = c->d_sigma;
        rs.type_hist = c->n_types > 0 ? c->d_type_hist : nullptr;
        rs.rec_end = (uint32_t)nrec;
        CK(c, cudaMemcpyAsync(c->d_run, &rs, sizeof rs, cudaMemcpyHostToDevice, c->stream));

        const bool use_graph = c->opt.graphs != 0 && !c->opt.timing;
        if (use_graph && (st = build_graph(c)) != VEGAS_OK) return st;
        std::vector<cudaEvent_t> ev;
        if (c->opt.timing) {
            ev.resize(2 * c->launches.size() * (size_t)mcs + 2);
            for (auto &x : ev) CK(c, cudaEventCreate(&x));
        }
        cudaEvent_t e0, e1;
        CK(c, cudaEventCreate(&e0));
        CK(c, cudaEventCreate(&e1));
        CK(c, cudaEventRecord(e0, c->stream));
        double sweep_ms = 0.0;
        bool folded = false;  // this step's last class-1 pass renormalised the spins
        // the kernels read the MCS counter, record index and schedule from the run state, which
        // the reductions (per-class sweep) and the advance kernel (resident sweep) move forward
        auto stream_mcs = [&](int32_t m0, int32_t n) -> vegas_status {
            for (int32_t m = m0; m < m0 + n; ++m) {
                const bool last = m == mcs - 1;
                folded = folded || (last && fold_active(c));
                if (use_graph && !(last && fold_active(c))) {
                    CK(c, cudaGraphLaunch(c->graph_exec, c->stream));
                    c->graph_launches++;
                } else if (c->opt.timing) {
                    std::vector<cudaEvent_t> sub(ev.begin() + (size_t)m * 2 * c->launches.size(),
                                                 ev.begin() + (size_t)(m + 1) * 2 * c->launches.size());
                    enqueue_mcs(c, c->stream, &sub, last);
                } else {
                    enqueue_mcs(c, c->stream, nullptr, last);
                }
                c->kernel_launches += (int64_t)c->launches.size() + 1;
                c->sweep_launches += (int64_t)c->launches.size();
            }
            return VEGAS_OK;
        };
        auto resident = [&](int32_t n) -> vegas_status {
            if (n <= 0) return VEGAS_OK;
            if (c->opt.timing) CK(c, cudaEventRecord(ev[ev.size() - 2], c->stream));
            enqueue_resident(c, c->stream, n);
            if (c->opt.timing) CK(c, cudaEventRecord(ev[ev.size() - 1], c->stream));
            CK(c, cudaGetLastError());
            c->kernel_launches += 2;
            c->sweep_launches++;
            return VEGAS_OK;
        };
        auto coop = [&](int32_t n) -> vegas_status {
            if (n <= 0) return VEGAS_OK;
            if (c->opt.timing) CK(c, cudaEventRecord(ev[ev.size() - 2], c->stream));
            enqueue_coop(c, c->stream, n);
            if (c->opt.timing) CK(c, cudaEventRecord(ev[ev.size() - 1], c->stream));
            CK(c, cudaGetLastError());
            c->kernel_launches += 2;
            c->sweep_launches++;
            return VEGAS_OK;
        };
        auto cluster = [&](int32_t n) -> vegas_status {
            if (n <= 0) return VEGAS_OK;
            if (c->opt.timing) CK(c, cudaEventRecord(ev[ev.size() - 2], c->stream));
            enqueue_cluster(c, c->stream, n);
            if (c->opt.timing) CK(c, cudaEventRecord(ev[ev.size() - 1], c->stream));
            CK(c, cudaGetLastError());
            c->kernel_launches += 2;
            c->sweep_launches++;
            return VEGAS_OK;
        };
        auto wave = [&](int32_t m0, int32_t n) -> vegas_status {
            for (int32_t m = m0; m < m0 + n; ++m) {
                if (c->opt.timing) CK(c, cudaEventRecord(ev[2 * (size_t)m], c->stream));
                const int e = enqueue_wave(c, c->stream);
                if (e != 0)
                    return fail(c, VEGAS_ECUDA, std::string("wavefront sweep launch: ") + cudaGetErrorString((cudaError_t)e));
                if (c->opt.timing) CK(c, cudaEventRecord(ev[2 * (size_t)m + 1], c->stream));
                CK(c, cudaGetLastError());
                c->kernel_launches += 2;
                c->sweep_launches++;
            }
            return VEGAS_OK;
        };
        auto run_variant = [&](int v, int32_t m0, int32_t n) -> vegas_status {
            if (v == 4) return wave(m0, n);
            if (v == 1) return resident(n);
            if (v == 2) return coop(n);
            if (v == 3) return cluster(n);
            return stream_mcs(m0, n);
        };
        for (int32_t s = 0; s < n_steps; ++s) {
            // one range per step; when the rest of the schedule goes out as one run graph, this
            // step's range covers that launch
            char step_name[48];
            std::snprintf(step_name, sizeof step_name, "vegas_run step %d/%d", (int)s + 1, (int)n_steps);
            NvtxRange step_range(step_name);
            int32_t m0 = 0;
            folded = false;
            if (!c->tuned && mcs >= 2) {
                // autotune: time a few MCS of each eligible sweep and block shape on the real chain
                // (all give the same spins) and keep the fastest for this context. Shapes: threads
                // per block of the resident sweep (so sites per thread), blocks per cluster of the
                // cluster sweep.
                struct Cand {
                    int v, a, b, split, group;  // sweep; threads (resident) or blocks per cluster,
                                                // threads; cluster split; threads per small instance
                    int sm = 0;                 // resident: spins in shared memory
                };
                std::vector<Cand> cand{{0, 0, 0, 0, 0}};
                // instances of very different sizes (split and grouping candidates)
                const bool uneven = c->res_items > 1 && 4 * (int64_t)c->min_instance_sites < c->max_instance_sites;
                if (c->res_eligible && c->opt.resident_smem != 1) {
                    cand.push_back({1, 256, 0, 0, 0});
                    cand.push_back({1, 512, 0, 0, 0});
                    if (uneven) {  // small instances several to a block
                        cand.push_back({1, 512, 0, 0, 128});
                        cand.push_back({1, 512, 0, 0, 256});
                    }
                }
                if (c->res_eligible && c->res_smem_eligible) {  // spins in shared memory
                    cand.push_back({1, 512, 0, 0, 0, 1});
                    if (uneven) {
                        cand.push_back({1, 512, 0, 0, 128, 1});
                        cand.push_back({1, 512, 0, 0, 256, 1});
                    }
                }
                if (c->coop_eligible)  // blocks per SM
                    for (int bps = 1; bps <= 3 && c->sm_count * (bps - 1) < c->coop_grid_max; ++bps)
                        cand.push_back({2, bps, 0, 0, 0});
                if (c->cluster_eligible) {
                    const int cs0 = c->cluster_cs, big = c->max_instance_sites;
                    cand.push_back({3, cs0, 256, 0, 0});
                    if (cs0 / 2 >= 2) cand.push_back({3, cs0 / 2, 256, 0, 0});
                    // batches of uneven instances: clusters for the largest, blocks (and groups of a
                    // block) for the rest
                    if (uneven)
                        for (int sp : {big / 2, big / 4})
                            if (sp > 0) {
                                cand.push_back({3, 2, 512, sp, 128});
                                cand.push_back({3, 4, 256, sp, 0});
                            }
                    if (c->res_smem_eligible) {  // every block's copy of the spins in shared memory
                        cand.push_back({3, 2, 512, uneven ? big / 2 : 0, 0, 1});
                        cand.push_back({3, 4, 512, uneven ? big / 4 : 0, 0, 1});
                        if (uneven) {
                            cand.push_back({3, 2, 512, big / 2, 128, 1});
                            cand.push_back({3, 4, 512, big / 4, 128, 1});
                            // clusters for the largest only: they set the launch's length (on the
                            // 256 nanoparticles: 23.0, 24.4, 23.9 and 23.2 G attempts/s at 3/4,
                            // 4/5, 17/20 and 7/8 of the largest; 20.7 with no cluster)
                            for (int f : {75, 80, 85}) cand.push_back({3, 2, 512, big * f / 100, 256, 1});
                        }
                    }
                }
                // longer probes when the step allows (less noise between close candidates), at most
                // a quarter of the step
                const int32_t probe = std::max(1, std::min(16, mcs / (4 * (int32_t)cand.size())));
                if (probe * (int32_t)cand.size() <= mcs) {
                    float best = 0.f;
                    int best_v = c->variant;
                    Cand best_c = cand[0];
                    const int cs_rule = c->cluster_cs, ct_rule = c->cluster_threads, rt_rule = c->res_threads;
                    for (const Cand &vc : cand) {
                        const int v = vc.v;
                        // grouped instances: group_threads threads for up to 16 sites each per thread
                        if (v == 1 && !set_resident_shape(c, vc.a, vc.group, vc.group * 16, vc.sm != 0)) continue;
                        if (v == 2) set_coop_shape(c, vc.a);
                        if (v == 3 && !set_cluster_shape(c, vc.a, vc.b, vc.split, vc.group, vc.group * 16, vc.sm != 0))
                            continue;
                        cudaEvent_t x0, x1;
                        CK(c, cudaEventCreate(&x0));
                        CK(c, cudaEventCreate(&x1));
                        CK(c, cudaEventRecord(x0, c->stream));
                        if ((st = run_variant(v, m0, probe)) != VEGAS_OK) return st;
                        CK(c, cudaEventRecord(x1, c->stream));
                        CK(c, cudaStreamSynchronize(c->stream));
                        float ms = 0.f;
                        CK(c, cudaEventElapsedTime(&ms, x0, x1));
                        cudaEventDestroy(x0);
                        cudaEventDestroy(x1);
                        if (c->tune_ms[v] == 0.0 || ms / probe < c->tune_ms[v]) c->tune_ms[v] = ms / probe;
                        sweep_ms += ms;
                        if (v == cand[0].v || ms < best) {
                            best = ms;
                            best_v = v;
                            best_c = vc;
                        }
                        m0 += probe;
                        uint32_t e4 = 0;
                        CK(c, cudaMemcpy(&e4, c->d_err, sizeof e4, cudaMemcpyDeviceToHost));
                        if (e4) break;  // report the device error below
                    }
                    c->variant = best_v;
                    // the shape of the sweep kept goes last: the two persistent sweeps share the
                    // grouping of small instances
                    if (c->cluster_eligible && best_v != 3) set_cluster_shape(c, cs_rule, ct_rule, 0, 0, 0);
                    set_coop_shape(c, best_v == 2 ? best_c.a : 2);
                    if (best_v == 1)
                        set_resident_shape(c, best_c.a, best_c.group, best_c.group * 16, best_c.sm != 0);
                    else
                        set_resident_shape(c, rt_rule);
                    if (best_v == 3)
                        set_cluster_shape(c, best_c.a, best_c.b, best_c.split, best_c.group, best_c.group * 16,
                                          best_c.sm != 0);
                }
                c->tuned = true;
            }

            if (m0 == 0 && c->tuned && use_graph && c->opt.graphs == 1 && step_graph_nodes(c, mcs) > 0) {
                // every remaining step in one launch of the run graph
                cudaGraphExec_t ge;
                if (run_graph(c, mcs, &ge)) {
                    CK(c, cudaGraphLaunch(ge, c->stream));
                    c->graph_launches++;
                    const int64_t left = n_steps - s;
                    // kernels per step: the sweep's (a persistent launch + advance; mcs x (wavefront +
                    // reduction); or mcs x (passes + reduction)), the renormalisation, the snapshot,
                    // the loop control
                    const int64_t sweep_k = c->variant == 4 ? 2 * (int64_t)mcs
                                            : (c->variant >= 1 ? 2 : (int64_t)mcs * ((int64_t)c->launches.size() + 1));
                    c->kernel_launches += left * (sweep_k + (fold_active(c) ? 1 : 2) + (c->opt.snapshots ? 1 : 0));
                    c->sweep_launches += c->variant == 4 ? left * (int64_t)mcs
                                         : (c->variant >= 1 ? left : left * (int64_t)mcs * (int64_t)c->launches.size());
                    break;
                }
            }
            if (m0 == 0 && c->tuned && use_graph && c->variant < 2 && step_graph_nodes(c, mcs) > 0) {
                // the whole step as one graph (the cooperative and cluster launches stay direct launches)
                cudaGraphExec_t ge;
                if ((st = step_graph(c, mcs, &ge)) != VEGAS_OK) return st;
                CK(c, cudaGraphLaunch(ge, c->stream));
                c->graph_launches++;
                const int64_t nodes = step_graph_nodes(c, mcs);
                c->kernel_launches += c->variant >= 1 ? 3 + (c->opt.snapshots ? 1 : 0) : nodes - (fold_active(c) ? 1 : 0);
                c->sweep_launches += c->variant >= 1 ? 1 : (int64_t)mcs * (int64_t)c->launches.size();
                continue;
            }
            if ((st = run_variant(c->variant, m0, mcs - m0)) != VEGAS_OK) return st;
            enqueue_renorm(c, c->stream, folded);
            c->kernel_launches += (folded ? 0 : 1) + (c->opt.snapshots ? 1 : 0);
            if (c->opt.timing) {  // read this step's sweep timings before the events are reused
                CK(c, cudaStreamSynchronize(c->stream));
                if (c->variant == 4) {
                    for (int32_t m = m0; m < mcs; ++m) {
                        float ms = 0.f;
                        CK(c, cudaEventElapsedTime(&ms, ev[2 * (size_t)m], ev[2 * (size_t)m + 1]));
                        sweep_ms += ms;
                    }
                } else if (c->variant >= 1) {
                    float ms = 0.f;
                    CK(c, cudaEventElapsedTime(&ms, ev[ev.size() - 2], ev[ev.size() - 1]));
                    sweep_ms += ms;
                } else {
                    for (size_t k = (size_t)m0 * 2 * c->launches.size(); k + 1 < ev.size() - 2; k += 2) {
                        float ms = 0.f;
                        CK(c, cudaEventElapsedTime(&ms, ev[k], ev[k + 1]));
                        sweep_ms += ms;
                    }
                }
            }
        }
        CK(c, cudaEventRecord(e1, c->stream));
        CK(c, cudaGetLastError());
        CK(c, cudaStreamSynchronize(c->stream));
        float run_ms = 0.f;
        CK(c, cudaEventElapsedTime(&run_ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        for (auto &x : ev) cudaEventDestroy(x);
        c->last_run_ms = run_ms;
        c->sweep_ms += sweep_ms;
        uint32_t derr4[4] = {0, 0, 0, 0};
        CK(c, cudaMemcpy(derr4, c->d_err, sizeof derr4, cudaMemcpyDeviceToHost));
        const uint32_t derr = derr4[0];
        // history: device [rec][inst][4] -> host per instance, appended
        std::vector<double> h(hneed);
        CK(c, cudaMemcpy(h.data(), c->d_hist, sizeof(double) * hneed, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < NI; ++i) {
            auto &v = c->hist[(size_t)i];
            const size_t old = v.size();
            v.resize(old + (size_t)nrec * 4);
            for (int64_t r = 0; r < nrec; ++r)
                std::memcpy(&v[old + (size_t)r * 4], &h[((size_t)r * NI + i) * 4], 4 * sizeof(double));
        }
        std::vector<uint32_t> ha(aneed);
        CK(c, cudaMemcpy(ha.data(), c->d_acc_hist, sizeof(uint32_t) * aneed, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < NI; ++i) {
            auto &v = c->acc_hist[(size_t)i];
            const size_t old = v.size();
            v.resize(old + (size_t)nrec);
            for (int64_t r = 0; r < nrec; ++r) v[old + (size_t)r] = ha[(size_t)r * NI + i];
        }
        if (tneed > 0) {  // [rec][inst][type][3] -> per instance, appended
            std::vector<double> ht(tneed);
            CK(c, cudaMemcpy(ht.data(), c->d_type_hist, sizeof(double) * tneed, cudaMemcpyDeviceToHost));
            const size_t per = (size_t)c->n_types * 3;
            for (int64_t i = 0; i < NI; ++i) {
                auto &v = c->type_hist[(size_t)i];
                const size_t old = v.size();
                v.resize(old + (size_t)nrec * per);
                for (int64_t r = 0; r < nrec; ++r)
                    std::memcpy(&v[old + (size_t)r * per], &ht[((size_t)r * NI + i) * per], per * sizeof(double));
            }
        }
        if (sneed > 0) {  // [step][site][replica] in the device layout -> per instance, caller order
            std::vector<unsigned char> hs(sneed);
            CK(c, cudaMemcpy(hs.data(), c->d_snap, sneed, cudaMemcpyDeviceToHost));
            const size_t step_bytes = (size_t)(c->n_sites * c->R * vbytes);
            for (int32_t sm = 0; sm < c->n_samples; ++sm) {
                const SampleInfo &si = c->samples[(size_t)sm];
                for (int32_t r = 0; r < c->R; ++r) {
                    auto &v = c->snaps[(size_t)(sm * c->R + r)];
                    const size_t old = v.size();
                    v.resize(old + (size_t)n_steps * (size_t)si.n * 3);
                    for (int32_t st = 0; st < n_steps; ++st)
                        for (int32_t g = 0; g < si.n; ++g) {
                            const unsigned char *p =
                                hs.data() + (size_t)st * step_bytes + ((size_t)(si.site_off + g) * c->R + r) * vbytes;
                            double *o3 = &v[old + ((size_t)st * si.n + (size_t)si.orig[(size_t)g]) * 3];
                            if (c->precision == 64) {
                                std::memcpy(o3, p, 3 * sizeof(double));
                            } else {
                                float f[3];
                                std::memcpy(f, p, sizeof f);
                                for (int q = 0; q < 3; ++q) o3[q] = f[q];
                            }
                        }
                }
            }
            c->snapshot_steps += n_steps;
        }
        c->records += nrec;
        c->t += (uint32_t)nrec;
        c->device_error |= derr;
        if (derr & kErrTimeout)
            return fail(c, VEGAS_ETIMEOUT,
                        c->variant == 4 ? "a warp of the wavefront sweep waited longer than timeout_ns for the class-0 "
                                          "blocks that a class-1 block links to"
                                        : "a grid barrier of the cooperative sweep waited longer than timeout_ns");
        if (derr) {
            char msg[200];
            std::snprintf(msg, sizeof msg,
                          "device error flags 0x%x (1: NaN energy change, 2: sphere sampler cap, 4: index check; "
                          "check code %u, value %u)",
                          derr, derr4[1], derr4[2]);
            return fail(c, VEGAS_EDEVICE, msg);
        }
        return VEGAS_OK;
    } catch (...) {
        return host_exception(c);
    }
}

extern "C" vegas_status vegas_history(const vegas_ctx *cc, double *out, size_t capacity, size_t *n_written) {
    try {
        vegas_ctx *c = const_cast<vegas_ctx *>(cc);
        vegas_status st = check_usable(c);
        if (st != VEGAS_OK) return st;
        const size_t need = (size_t)c->n_inst * (size_t)c->records * 4;
        if (n_written) *n_written = need;
        if (!out) return VEGAS_OK;
        if (capacity < need) return fail(c, VEGAS_EINVAL, "history buffer too small");
        for (int i = 0; i < c->n_inst; ++i)
            std::memcpy(out + (size_t)i * c->records * 4, c->hist[(size_t)i].data(), sizeof(double) * c->records * 4);
        return VEGAS_OK;
    } catch (...) {
        return host_exception(const_cast<vegas_ctx *>(cc));
    }
}

extern "C" vegas_status vegas_accept_history(const vegas_ctx *cc, uint32_t *out, size_t capacity, size_t *n_written) {
    try {
        vegas_ctx *c = const_cast<vegas_ctx *>(cc);
        vegas_status st = check_usable(c);
        if (st != VEGAS_OK) return st;
        const size_t need = (size_t)c->n_inst * (size_t)c->records;
        if (n_written) *n_written = need;
        if (!out) return VEGAS_OK;
        if (capacity < need) return fail(c, VEGAS_EINVAL, "acceptance buffer too small");
        for (int i = 0; i < c->n_inst; ++i)
            std::memcpy(out + (size_t)i * c->records, c->acc_hist[(size_t)i].data(), sizeof(uint32_t) * c->records);
        return VEGAS_OK;
    } catch (...) {
        return host_exception(const_cast<vegas_ctx *>(cc));
    }
}

extern "C" vegas_status vegas_type_history(const vegas_ctx *cc, double *out, size_t capacity, size_t *n_written) {
    try {
        vegas_ctx *c = const_cast<vegas_ctx *>(cc);
        vegas_status st = check_usable(c);
        if (st != VEGAS_OK) return st;
        if (c->n_types == 0) return fail(c, VEGAS_EINVAL, "per-type statistics need the option type_stats");
        const size_t per = (size_t)c->records * (size_t)c->n_types * 3;
        const size_t need = (size_t)c->n_inst * per;
        if (n_written) *n_written = need;
        if (!out) return VEGAS_OK;
        if (capacity < need) return fail(c, VEGAS_EINVAL, "type history buffer too small");
        for (int i = 0; i < c->n_inst; ++i)
            std::memcpy(out + (size_t)i * per, c->type_hist[(size_t)i].data(), sizeof(double) * per);
        return VEGAS_OK;
    } catch (...) {
        return host_exception(const_cast<vegas_ctx *>(cc));
    }
}

extern "C" vegas_status vegas_get_snapshot(const vegas_ctx *cc, int32_t inst, int64_t step, double *out) {
    try {
        vegas_ctx *c = const_cast<vegas_ctx *>(cc);
        vegas_status st = check_usable(c);
        if (st != VEGAS_OK) return st;
        if (!c->opt.snapshots) return fail(c, VEGAS_EINVAL, "snapshots need the option snapshots");
        if (inst < 0 || inst >= c->n_inst) return fail(c, VEGAS_EINVAL, "instance out of range");
        if (step < 0 || step >= c->snapshot_steps) return fail(c, VEGAS_EINVAL, "no snapshot for this step");
        if (!out) return fail(c, VEGAS_EINVAL, "out is NULL");
        const size_t n3 = (size_t)c->samples[(size_t)(inst / c->R)].n * 3;
        std::memcpy(out, c->snaps[(size_t)inst].data() + (size_t)step * n3, sizeof(double) * n3);
        return VEGAS_OK;
    } catch (...) {
        return host_exception(const_cast<vegas_ctx *>(cc));
    }
}

extern "C" vegas_status vegas_adaptive_width(const vegas_ctx *cc, double *out) {
    try {
        vegas_ctx *c = const_cast<vegas_ctx *>(cc);
        vegas_status st = check_usable(c);
        if (st != VEGAS_OK) return st;
        if (!out) return fail(c, VEGAS_EINVAL, "out is NULL");
        if ((st = set_device(c)) != VEGAS_OK) return st;
        CK(c, cudaMemcpy(out, c->d_sigma, sizeof(double) * (size_t)c->n_inst, cudaMemcpyDeviceToHost));
        return VEGAS_OK;
    } catch (...) {
        return host_exception(const_cast<vegas_ctx *>(cc));
    }
}

extern "C" vegas_status vegas_set_adaptive_width(vegas_ctx *c, const double *in) {
    try {
        vegas_status st = check_usable(c);
        if (st != VEGAS_OK) return st;
        if (!in) return fail(c, VEGAS_EINVAL, "in is NULL");
        std::vector<double> h((size_t)c->n_inst, 0.0);
        for (int32_t i = 0; i < c->n_inst; ++i) {
            if (!c->samples[(size_t)(i / c->R)].has_adaptive) continue;
            if (!(in[i] > 0.0) || !std::isfinite(in[i])) return fail(c, VEGAS_EINVAL, "width must be finite and > 0");
            h[(size_t)i] = in[i];
        }
        if ((st = set_device(c)) != VEGAS_OK) return st;
        CK(c, cudaMemcpy(c->d_sigma, h.data(), sizeof(double) * (size_t)c->n_inst, cudaMemcpyHostToDevice));
        return VEGAS_OK;
    } catch (...) {
        return host_exception(c);
    }
}

extern "C" vegas_status vegas_set_mcs_counter(vegas_ctx *c, uint32_t t) {
    try {
        vegas_status st = check_usable(c);
        if (st != VEGAS_OK) return st;
        if (t == UINT32_MAX) return fail(c, VEGAS_EINVAL, "MCS counter must be below 2^32 - 1");
        if (c->d_done) {
            // the wavefront sweep's completion words hold t + 1 of past MCS; cleared, none can
            // match an MCS of the new count before its class-0 block has finished
            if ((st = set_device(c)) != VEGAS_OK) return st;
            CK(c, cudaMemsetAsync(c->d_done, 0, sizeof(uint32_t) * (size_t)c->wave.nb0, c->stream));
            CK(c, cudaStreamSynchronize(c->stream));
        }
        c->t = t;
        return VEGAS_OK;
    } catch (...) {
        return host_exception(c);
    }
}

namespace {

vegas_status spins_io(vegas_ctx *c, int32_t inst, double *out, const double *in) {
    vegas_status st = check_usable(c);
    if (st != VEGAS_OK) return st;
    if (inst < 0 || inst >= c->n_inst) return fail(c, VEGAS_EINVAL, "instance out of range");
    if (!out && !in) return fail(c, VEGAS_EINVAL, "buffer is NULL");
    if ((st = set_device(c)) != VEGAS_OK) return st;
    const SampleInfo &si = c->samples[(size_t)(inst / c->R)];
    const int32_t r = inst % c->R;
    const size_t n = (size_t)si.n;
    double *d = nullptr;
    CK(c, cudaMalloc(&d, sizeof(double) * 3 * n));
    std::vector<double> h(3 * n);
    const int grid = (int)std::min<int64_t>(((int64_t)n + 255) / 256, (int64_t)c->sm_count * 8);
    cudaError_t e = cudaSuccess;
    if (out) {
        launch_gather(c->d_spins, c->precision, si.site_off, (int64_t)n, c->log2R, r, d, grid, c->stream);
        e = cudaMemcpyAsync(h.data(), d, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e == cudaSuccess)
            for (size_t g = 0; g < n; ++g)
                for (int q = 0; q < 3; ++q) out[3 * (size_t)si.orig[g] + q] = h[3 * g + q];
    } else {
        for (size_t g = 0; g < n; ++g)
            for (int q = 0; q < 3; ++q) {
                const double v = in[3 * (size_t)si.orig[g] + q];
                if (!std::isfinite(v)) {
                    cudaFree(d);
                    return fail(c, VEGAS_EINVAL, "non-finite spin component");
                }
                h[3 * g + q] = v;
            }
        e = cudaMemcpyAsync(d, h.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) launch_scatter(c->d_spins, c->precision, si.site_off, (int64_t)n, c->log2R, r, d, grid, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    c->kernel_launches++;
    cudaFree(d);
    if (e == cudaSuccess) e = cudaGetLastError();
    CK(c, e);
    return VEGAS_OK;
}

}  // namespace

extern "C" vegas_status vegas_get_spins(const vegas_ctx *c, int32_t inst, double *out) {
    try {
        if (!out) return fail(const_cast<vegas_ctx *>(c), VEGAS_EINVAL, "out is NULL");
        return spins_io(const_cast<vegas_ctx *>(c), inst, out, nullptr);
    } catch (...) {
        return host_exception(const_cast<vegas_ctx *>(c));
    }
}

extern "C" vegas_status vegas_set_spins(vegas_ctx *c, int32_t inst, const double *in) {
    try {
        if (!in) return fail(c, VEGAS_EINVAL, "in is NULL");
        return spins_io(c, inst, nullptr, in);
    } catch (...) {
        return host_exception(c);
    }
}

extern "C" vegas_status vegas_accept_log(const vegas_ctx *cc, uint8_t *out, size_t capacity, size_t *n_written) {
    try {
        vegas_ctx *c = const_cast<vegas_ctx *>(cc);
        vegas_status st = check_usable(c);
        if (st != VEGAS_OK) return st;
        if (n_written) *n_written = (size_t)c->alog_bytes;
        if (!out || c->alog_bytes == 0) return VEGAS_OK;
        if (capacity < (size_t)c->alog_bytes) return fail(c, VEGAS_EINVAL, "accept log buffer too small");
        if ((st = set_device(c)) != VEGAS_OK) return st;
        CK(c, cudaMemcpy(out, c->d_alog, (size_t)c->alog_bytes, cudaMemcpyDeviceToHost));
        return VEGAS_OK;
    } catch (...) {
        return host_exception(const_cast<vegas_ctx *>(cc));
    }
}

extern "C" vegas_status vegas_stats(const vegas_ctx *c, vegas_stats_t *o) {
    try {
        if (!c || !o) return VEGAS_EINVAL;
        std::memset(o, 0, sizeof *o);
        o->n_samples = c->n_samples;
        o->n_instances = c->n_inst;
        o->replicas = c->R;
        o->precision = c->precision;
        o->max_colours = c->max_colours;
        o->variant = c->variant;
        o->n_sites = c->n_sites;
        o->n_edges = c->n_edges;
        o->records = c->records;
        o->mcs_done = c->t;
        o->device_error = c->device_error;
        o->kernel_launches = c->kernel_launches;
        o->sweep_launches = c->sweep_launches;
        o->sweep_ms = c->sweep_ms;
        o->last_run_ms = c->last_run_ms;
        o->device_bytes = c->device_bytes;
        o->n_types = c->n_types;
        o->snapshot_steps = c->snapshot_steps;
        o->block_threads = c->variant == 1 ? c->res_threads : (c->variant == 3 ? c->cluster_threads : kThreads);
        o->cluster_blocks = c->variant == 3 ? c->cluster_cs : 0;
        o->split_sites = c->variant == 3 ? c->res.split_sites : 0;
        o->group_threads = (c->variant == 1 || c->variant == 3) ? c->res.group_threads : 0;
        o->group_sites = (c->variant == 1 || c->variant == 3) ? c->res.group_sites : 0;
        o->graph_launches = c->graph_launches;
        uint32_t kinds = 0;
        if (c->variant == 1)
            kinds = c->res_smem ? VEGAS_KERNEL_RESIDENT32_SMEM : VEGAS_KERNEL_RESIDENT32;
        else if (c->variant == 2)
            kinds = c->precision == 64 ? VEGAS_KERNEL_COOP64 : VEGAS_KERNEL_COOP32;
        else if (c->variant == 3)
            kinds = c->cluster_smem ? VEGAS_KERNEL_CLUSTER32_SMEM : VEGAS_KERNEL_CLUSTER32;
        else if (c->variant == 4)
            kinds = VEGAS_KERNEL_WAVE32;
        else
            for (const PassLaunch &p : c->passes)
                kinds |= c->precision == 64 ? VEGAS_KERNEL_PASS64 : pass32_kind(p.args);
        if (fold_active(c)) kinds |= VEGAS_KERNEL_PASS32_R32_RENORM;
        o->sweep_kernels = kinds;
        return VEGAS_OK;
    } catch (...) {
        return host_exception(const_cast<vegas_ctx *>(c));
    }
}

extern "C" const char *vegas_last_error(const vegas_ctx *c) {
    if (!c) return g_create_error.c_str();
    return c->err.c_str();
}

extern "C" void vegas_destroy(vegas_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}
