// Internal declarations shared by the loader, the kernels and the C-ABI driver.
#pragma once

#include <cstddef>
#include <cstdint>
#include <exception>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include <vector_types.h>  // int4 (CUDA headers; also used by the host-only loader)

#include "../../include/vegas.h"

namespace vegas {

// Status and message of the exception being handled (call it inside a catch block only): the
// entry points turn host exceptions, such as a failed allocation, into a status instead of
// letting them cross the C boundary.
inline vegas_status status_of_current_exception(std::string &msg) {
    try {
        throw;
    } catch (const std::bad_alloc &) {
        msg = "host allocation failed";
        return VEGAS_ENOMEM;
    } catch (const std::length_error &) {
        msg = "host allocation failed (size out of range)";
        return VEGAS_ENOMEM;
    } catch (const std::exception &e) {
        msg = std::string("host error: ") + e.what();
        return VEGAS_EINVAL;
    } catch (...) {
        msg = "host error";
        return VEGAS_EINVAL;
    }
}

constexpr int kMaxColours = 64;
constexpr int kMaxTypes = 64;   // site types tracked by the per-type statistics
constexpr int kThreads = 256;  // threads per block of the sweep kernels
constexpr int kCoopThreads = 256;  // threads per block of the cooperative sweep
constexpr int kCoop64Threads = 32; // the same in FP64: small blocks spread a class over many SMs

// Random-number purposes (fourth Philox counter word; low 16 bits hold a candidate index).
constexpr uint32_t kPurposeTrial64 = 0x00000u;   // FP64 sphere candidates
constexpr uint32_t kPurposeAccept64 = 0x10000u;  // FP64 acceptance uniform
constexpr uint32_t kPurposeInit = 0x20000u;      // initial spins (t = 0xFFFFFFFF)
constexpr uint32_t kPurposeTrial32 = 0x40000u;   // FP32 trial (z, azimuth) + acceptance
constexpr uint32_t kPurposeGauss2 = 0x08000u;    // FP64 Gaussian: second pair of normals (| k)
constexpr uint32_t kPurposeChoice = 0x0C000u;    // FP64 Hinzke-Nowak choice
constexpr uint32_t kInitT = 0xFFFFFFFFu;

// Update policies (vegas_policy in the C-ABI).
constexpr int32_t kPolRandom = 0, kPolFlip = 1, kPolSmallStep = 2, kPolGaussian = 3, kPolHinzkeNowak = 4,
                  kPolAdaptive = 5, kPolQIsing = 6;

// Error bits set by kernels in the device error word.
constexpr uint32_t kErrNaN = 1u;
constexpr uint32_t kErrSphere = 2u;
constexpr uint32_t kErrIndex = 4u;  // debug builds: an index or alignment check failed
constexpr uint32_t kErrTimeout = 8u;  // a bounded wait (grid barrier, wavefront dependency) ran out

// ------------------------------------------------------------------ host-side sample

// A validated sample renumbered colour-major: sites of colour 0 first, then colour 1, ...;
// inside a colour class, increasing caller id. Neighbour order inside a row is the caller's.
struct LoadedSample {
    int32_t n = 0;
    int32_t n_colours = 0;
    int64_t n_edges = 0;
    int32_t uniform_degree = 0;  // > 0 when every row has this many links
    std::vector<int32_t> orig;   // new index -> caller id
    std::vector<int32_t> inv;    // caller id -> new index
    std::vector<int32_t> cstart; // [n_colours + 1] class boundaries (new numbering)
    std::vector<int64_t> row_ptr;  // new numbering
    std::vector<int32_t> col;      // new numbering, sample-local
    std::vector<double> J;
    // per-site parameters in new numbering (always filled; defaults where NULL)
    std::vector<double> spin_norm, field_axis, k_uni, e_uni, k_cub;
    std::vector<double> init_spins;  // empty: Philox initial state
    std::vector<int32_t> type;       // per site (new numbering); all 0 without a type array
    int32_t n_types = 1;             // 1 + the largest type
    bool uniform_params = false;     // every site has the same (s, n, k, e, kc)
    double slab_width = 0.0;         // wavefront order: slab width along x (0: whole planes)
    bool has_anisotropy = false;     // some k or kc is non-zero
    // update policy per site (new numbering): code and parameter (cap height 1 - cos theta
    // for small step and Hinzke-Nowak, width for Gaussian and adaptive); empty when every
    // site is random
    std::vector<int32_t> policy;
    std::vector<double> policy_param;
    bool has_adaptive = false;
    double sigma0 = 0.0;             // starting width: the first adaptive type's parameter
    // per colour class: 0 = no neighbour of a lower colour, 1 = every neighbour lower,
    // 2 = mixed (tested per link)
    std::vector<int32_t> lower_mode;
};

// Validates and renumbers; on failure returns false and sets err. type_major: inside each
// colour class, sites are ordered by type first (then Morton order or caller id). plane_order:
// inside each class, positions are ordered by z, then y, then x (instead of the Morton curve),
// so that every neighbour of a site lies within about one plane of it in memory order.
// wave_slab (with plane_order): the sites are first cut into slabs along x, and ordered slab
// by slab, each slab plane by plane (z, y, x): > 0 the slab width in position units, 0 an
// automatic width (slabs of about 16384 sites per plane), < 0 no slabs.
bool load_sample(const vegas_sample &s, LoadedSample &out, std::string &err, bool type_major = false,
                 bool plane_order = false, double wave_slab = -1.0);

// ------------------------------------------------------------------ device-side layouts

struct SiteParams32 {  // uniform parameters of a sample, FP32 kernels
    float nx, ny, nz, s;
    float ex, ey, ez, k;
    float kc;
};

struct SiteParams64 {
    double nx, ny, nz, s;
    double ex, ey, ez, k;
    double kc;
};

struct PolicySite {  // update policy of one site (samples with a policy table), FP64 path
    double par;      // cap height 1 - cos theta (small step, Hinzke-Nowak) or width (Gaussian)
    int32_t code;    // kPolRandom .. kPolAdaptive
    int32_t pad;
};

struct PolicySite32 {  // the same for the FP32 path (8 bytes: staged with the links)
    float par;
    int32_t code;
};

struct Edge64 {  // one directed link, FP64 path
    double J;
    int32_t col;  // global (packed) site index
    int32_t pad;
};

// Mutable run state kept in device memory so that captured launches need no new
// arguments between MCS or between calls.
struct RunState {
    uint32_t t;       // global MCS counter (Philox counter word 1)
    uint32_t rec;     // records written in the current run
    uint32_t ticket;  // last-block-done counter of the reduction
    uint32_t mcs;     // MCS per temperature/field step of the current run
    const double *sched;  // [n_steps][n_inst][2] = (beta, B)
    double *hist;         // [records][n_inst][4]
    uint32_t *acc;        // [n_inst] accepted attempts of the current MCS, or NULL (not counted)
    uint32_t *acc_hist;   // [records][n_inst] accepted attempts per MCS
    double *sigma;        // [n_inst] width of the adaptive policy, or NULL
    double *type_hist;    // [records][n_inst][n_types][3] magnetization per site type, or NULL
    uint32_t rec_end;     // records of the current run (n_steps * mcs): where the run graph stops
    uint32_t pad_;
};

// One colour class of one sample: everything a sweep launch needs.
struct PassArgs {
    void *spins;               // float4 or double4_32a, [global site][replica]
    const void *edges;         // int2 (col, J float bits) or Edge64, global edge index
    const int64_t *row_ptr;    // [global site + 1] global edge offsets
    const int32_t *orig;       // [global site] caller id
    const void *p0;            // per-site (n, s): float4/double4_32a, or NULL when uniform
    const void *p1;            // per-site (e, k)
    const void *pk;            // per-site kc (float/double)
    const PolicySite *pol;     // FP64: per-site update policy, or NULL (every site random)
    const PolicySite32 *pol32; // FP32: the same
    RunState *run;
    double *partial;           // [block][replica][4] of this pass
    uint32_t *err;
    uint8_t *alog;             // accept log or NULL
    uint64_t seed;
    int64_t edge_base;         // first edge of the sample (uniform degree indexing)
    int32_t site_off;          // first global site of the sample
    int32_t g_begin, g_end;    // global site range of the class
    int32_t lower_end;         // sites with global index < lower_end have a lower colour
    int32_t log2R;
    int32_t inst0;             // instance id of the sample's replica 0 (Philox)
    int32_t inst_local0;       // ctx-local index of replica 0 (schedule column)
    int32_t n_inst;            // ctx-local instances (schedule row length)
    int32_t n_sample_sites;    // sites of the sample (accept log indexing)
    int64_t alog_stride;       // bytes per MCS of the accept log
    int64_t alog_base;         // offset of replica 0 of this sample inside one MCS
    uint32_t alog_mcs;
    int32_t deg;               // uniform degree or 0
    int32_t n_sites_total;     // sites over all samples (debug index checks)
    int64_t n_edges_total;
    int32_t lower_mode;        // 0: no link to a lower colour, 1: every link, 2: test each
    int32_t params_mode;       // 0: uniform, no anisotropy; 1: uniform; 2: per site
    int32_t depth;             // staged FP32 kernel: cp.async pipeline depth (2..4); 0 = direct kernel
    uint32_t *ticket;          // R = 32 staged kernel: next block of 8 sites of this pass (zeroed
                               // by the MCS's reduction); unused by the other kernels
    int32_t pol_fixed;         // FP32 with a policy table: the one policy of every site of the
                               // pass, or -1 (mixed, or no table)
    // The step's last class-1 pass of a two-class sample (R = 32 kernel) with the
    // renormalisation folded in, else NULL: class-1 spins are stored renormalised, and each
    // class-0 block of kFoldBlockSites sites is renormalised by the warp whose class-1 block is
    // the last of its readers to finish.
    const int32_t *fold_deps;  // [class-1 block][kFoldDeps] distinct class-0 blocks read, -1 padded
    const int32_t *fold_deg;   // [class-0 block] class-1 blocks that read it
    uint32_t *fold_cnt;        // [class-0 block] of those finished (zeroed before the pass)
    const double *fold_norm;   // [global site] s_i
    int32_t fold_c0_begin, fold_c0_end;  // global sites of class 0
    SiteParams32 u32;
    SiteParams64 u64;
};

// Block slots are grouped by sample and, with per-type statistics, by site type: group
// (s, k) holds the partials of every pass over type-k sites of sample s.
struct ReduceArgs {
    const double *partial;     // all passes
    const int64_t *slot_base;  // [n_samples][n_groups] first block slot of the group
    const int32_t *slot_count; // [n_samples][n_groups] block slots of the group
    RunState *run;
    const int32_t *adapt_n;    // [n_inst] sites of the instance's sample if it adapts a width, else 0
    int32_t R, n_inst;
    int32_t n_groups;          // type groups per sample (1 without per-type statistics)
    int32_t n_types;           // > 0: write the magnetization of each group to run->type_hist
    uint32_t *tickets;         // block counters of the MCS's passes, zeroed here for the next MCS, or NULL
    int32_t n_tickets;
};

struct RenormArgs {
    void *spins;
    const double *norm;      // [global site] spin norm s_i
    int64_t n_work;          // global sites * R
    int32_t log2R;
    const int32_t *qis;      // [global site] 1 for qIsing sites (left as they are), or NULL
};

struct InitArgs {
    void *spins;
    const int32_t *orig;
    const double *norm;      // [global site] spin norm s_i
    const double *given;     // [sample site][3] caller initial state (new numbering) or NULL
    uint32_t *err;
    uint64_t seed;
    int32_t g_begin, g_end;  // global sites of the sample
    int32_t inst0;           // instance id of replica 0
    int32_t log2R;
    const int32_t *qis;      // [global site] 1 for qIsing sites (a uniform value along z), or NULL
};

// One instance of the resident sweep: a sample's sites and one of its replicas.
struct ResidentInst {
    int32_t g_begin, g_end;    // the sample's global sites
    int32_t seg_off;           // first segment of the sample in ResidentArgs::segs
    int32_t n_segs;
    int32_t inst_id;           // Philox instance id
    int32_t inst_local;        // schedule and history column
    int32_t r;                 // replica within the sample
    int32_t params_mode;       // 0, 1, 2 as for PassArgs
    int32_t n_sample_sites;
    int32_t adaptive;          // 1: the sample adapts the width of its adaptive sites
    int64_t alog_base;         // accept-log offset of replica 0 of the sample
    SiteParams32 u;
};

constexpr int kEllRow = 12;  // links per fixed row of the spins-in-shared-memory sweeps

// Persistent sweep: every block takes instances from a queue (largest first) and runs all
// MCS of one temperature/field step on each, colour class after colour class.
struct ResidentArgs {
    void *spins;
    const void *edges;         // int2 (col, J float bits)
    const int64_t *row_ptr;
    const int32_t *orig;
    const void *p0, *p1, *pk;  // per-site parameters (samples with params_mode 2)
    const PolicySite32 *pol;   // per-site update policy, or NULL (every site random)
    const ResidentInst *insts; // [n_items], largest first
    // segments of a sample in sweep order: {begin, end, class begin, type | last-of-class << 16}
    // (global sites); one per colour class, or per (class, type) with per-type statistics
    const int4 *segs;
    uint32_t *queue;           // work counter, zero before the launch
    uint32_t *err;
    uint8_t *alog;
    uint64_t seed;
    int64_t alog_stride;
    uint32_t alog_mcs;
    int32_t n_items, n_inst, log2R;
    int32_t n_types;           // > 0: per-type magnetization into run->type_hist
    RunState *run;             // MCS counter t, record index, MCS per step, schedule, history
    int32_t mcs;               // MCS in this launch (all inside one temperature/field step)
    int32_t split_sites;       // cluster sweep: instances of at most this many sites are swept by
                               // one block each (0: every instance by a whole cluster)
    int32_t group_threads;     // > 0: a block sweeps instances of at most group_sites sites
    int32_t group_sites;       // NT / group_threads at a time, group_threads threads each
    const int4 *ell;           // spins in shared memory: every site's links as a fixed row of
                               // 12 (neighbour, J float bits) pairs in row order, padded with
                               // neighbour -1 ([global site][6] int4)
    int32_t any_aniso;         // 0: no instance has anisotropy or per-site parameters
    int32_t smem_sites;        // resident sweep: > 0 keeps each instance's spins in shared memory
                               // for the whole launch (room for this many sites per block, or
                               // group_sites per group); 0 reads and writes them in global memory
};

// Grid barrier of the cooperative sweep (zeroed before every launch).
// Grid barrier: the arrival counter and the generation word the waiting blocks poll sit on
// separate 128-byte lines, so the polling loads do not queue with the arrivals' atomics.
struct GridBarrier {
    uint32_t count;  // blocks arrived at the current barrier
    uint32_t pad0_[31];
    uint32_t gen;    // completed barriers
    uint32_t abort;  // set when a wait timed out: every block leaves
    uint32_t pad1_[30];
};

// Cooperative sweep of one sample (R replicas): all blocks sweep each colour class together
// and meet at a bounded grid barrier between classes; every MCS of the step in one launch.
struct CoopArgs {
    PassArgs pass;             // site range of class 0 .. per class below, links, parameters
    const int32_t *cstart;     // class starts (global sites), n_colours + 1
    int32_t n_colours;
    int32_t mcs;               // MCS in this launch
    GridBarrier *bar;
    double *partial;           // [2][block][R][4]: the partials of two MCS in turn
    int64_t timeout_ns;        // longest wait at one barrier
    int32_t skip_block;        // fault injection: this block never arrives (-1: none)
    int32_t fp64;              // 1: FP64 spins (coop64_kernel)
    const int2 *ell;           // FP32 rows of at most kEllRow links as fixed padded rows, or NULL
};

// Wavefront sweep of one two-colour sample with R = 32 replicas: both colour classes of an
// MCS in one launch. The sites of each class are cut into blocks of 8; tasks[] lists the
// blocks in sweep order, and every warp draws its next task from a ticket counter. A block
// of class 1 starts once every class-0 block holding one of its neighbours has finished this
// MCS (done[b] == t + 1, published with release semantics). Every class-1 block comes after
// all of its class-0 dependencies in tasks[], and the holder of a ticket is a running warp,
// which makes the waits finite; each wait is still bounded by timeout_ns.
constexpr int kWaveBlockSites = 8;   // sites per task of the wavefront sweep
constexpr int kWaveDeps = 32;        // class-0 blocks a class-1 block may link to
constexpr int kFoldBlockSites = 8;   // the R = 32 kernel's blocks of sites
constexpr int kFoldDeps = 32;        // class-0 blocks a class-1 block may read (one per lane)

struct WaveArgs {
    PassArgs pass;             // class 0: links, parameters, spins, run state; partial = [block][32][4]
    const int32_t *tasks;      // [n_tasks]: b < nb0 is block b of class 0, else block b - nb0 of class 1
    const int32_t *deps;       // [nb1][kWaveDeps]: the distinct class-0 blocks each class-1 block
                               // links to, padded with -1
    uint32_t *ticket;          // next task of the launch (zeroed before every launch)
    uint32_t *done;            // [nb0] MCS counter + 1 of the MCS in which class-0 block b last finished
    int32_t n_tasks, nb0;
    int32_t c1_begin, c1_end;  // global sites of class 1 (class 0 is pass.g_begin .. pass.g_end)
    int64_t timeout_ns;        // longest wait for one block's dependencies
    int32_t skip_block;        // fault injection: this class-0 block is never published (-1: none)
};

// ------------------------------------------------------------------ launchers

using PassFn = void (*)(PassArgs);
// FP32 colour-pass kernel for a pass (staged for rows of six links, else direct) and its
// dynamic shared memory; the direct kernel for a parameter mode, lower mode and policy flag.
PassFn select_pass32(const PassArgs &a);
int pass32_smem(const PassArgs &a);
int pass32_threads(const PassArgs &a);  // threads per block of that kernel
// The kernel select_pass32 picks, as a VEGAS_KERNEL_* bit of include/vegas.h.
// The direct FP32 passes of one colour class of several samples (same kernel, key's template
// fields) in one launch; passes[p] runs blocks first[p] .. first[p + 1] - 1 of the grid.
void launch_pass32_multi(const PassArgs &key, const PassArgs *passes, const int32_t *first, int32_t n, int grid,
                         void *stream);
bool pass32_direct(const PassArgs &a);  // the pass runs the direct (plain-load) kernel
uint32_t pass32_kind(const PassArgs &a);
PassFn select_direct(int pm, int lm, bool pol);

// Sweep launch of one colour class; lower_mode, params_mode and deg pick the compiled variant.
void launch_pass32(const PassArgs &a, int grid, void *stream);
void launch_pass64(const PassArgs &a, int grid, int threads, void *stream);  // threads: 32 .. kThreads
void launch_reduce(const ReduceArgs &a, void *stream);
void launch_renorm32(const RenormArgs &a, int grid, void *stream);
void launch_renorm64(const RenormArgs &a, int grid, void *stream);
void launch_init32(const InitArgs &a, int grid, void *stream);
void launch_init64(const InitArgs &a, int grid, void *stream);
void launch_gather(void *spins, int precision, int64_t site_off, int64_t n, int32_t log2R, int32_t r, double *out3,
                   int grid, void *stream);
void launch_scatter(void *spins, int precision, int64_t site_off, int64_t n, int32_t log2R, int32_t r,
                    const double *in3, int grid, void *stream);

// Blocks per SM the pass kernels reach at kThreads threads (occupancy query).
int pass_blocks_per_sm(int precision, const PassArgs &a);

// Resident sweep with `threads` per block (256 or 512).
void launch_resident(const ResidentArgs &a, int grid, int threads, void *stream);
// Adds n to the run state's MCS counter and record index (after a resident launch).
void launch_advance(RunState *run, int32_t n, void *stream);
// Loop control of the run graph (a conditional while node over temperature/field steps):
// sets the node's handle to 1 while the run has records left (run->rec < run->rec_end).
void launch_run_ctrl(const RunState *run, unsigned long long loop_handle, void *stream);
// Copies the spins into the snapshot slot of the step that just ended (read from the run state).
void launch_snapshot(const void *spins, void *snap, int64_t n16, const RunState *run, int grid, void *stream);

// Cooperative launch (all blocks co-resident); returns the CUDA error of the launch.
int launch_coop(const CoopArgs &a, int grid, void *stream);
int coop_blocks_per_sm(bool pol, int form, bool fp64);  // form: 6 (rows of six links), kEllRow (padded rows) or 0
// Blocks of the resident sweep per SM (smem_bytes > 0: the shared-memory form, whose limit
// is raised here; 0 when it does not fit).
int resident_blocks_per_sm(int threads, bool pol, size_t smem_bytes = 0);
size_t resident_smem_bytes(const ResidentArgs &a, int threads);
// Cluster sweep: n_clusters clusters of cs blocks of `threads` (256 or 512); returns the CUDA
// error of the launch.
int launch_cluster(const ResidentArgs &a, int n_clusters, int cs, int threads, void *stream);
// Clusters of cs blocks of `threads` that fit on the device at once (0 when none or on error).
// Clusters of cs blocks that fit at once (smem_bytes > 0: the form with spins in shared
// memory, whose limit is raised here); 0 when none fits.
int cluster_capacity(int cs, int threads, bool pol, size_t smem_bytes = 0);
size_t cluster_smem_bytes(const ResidentArgs &a, int threads);

// Wavefront sweep: launch of `grid` blocks of kThreads; returns the CUDA error of the launch.
// wave_blocks_per_sm is the occupancy of its kernel for a parameter mode.
int launch_wave(const WaveArgs &a, int grid, void *stream);
int wave_blocks_per_sm(int params_mode);

}  // namespace vegas
