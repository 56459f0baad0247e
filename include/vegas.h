/*
 * vegas.h - C-ABI of the GB300 Metropolis sweep of the classical Heisenberg model.
 *
 * The library runs the Monte Carlo Metropolis method of Sec. III.B (Eq. 4) on the spin
 * Hamiltonian of Sec. III.A (Eq. 1-3) for many independent instances on one GPU, and
 * records energy and magnetization after every Monte Carlo step (MCS) of every
 * temperature/field step (Sec. II, first feature). Every entry point is plain C: host
 * pointers and sizes in, status codes out. Nothing here throws, aborts, exits or traps.
 *
 * Model (Eq. 1-3), with each undirected bond counted once:
 *   E = -1/2 sum_i sum_{j in N(i)} J_ij S_i.S_j - B sum_i S_i.n_i
 *       - sum_i k_i (S_i.e_i)^2 - sum_i kc_i (Sx^2 Sy^2 + Sy^2 Sz^2 + Sx^2 Sz^2)_i
 *   S_i = s_i * (unit vector); B is a scalar field intensity and n_i the per-site field
 *   axis (Sec. III.C material file); k > 0 is an easy axis. k_B = 1.
 * Update policies (Sec. II; Sec. IV.C), chosen per site type through a table in the sample
 *   (a policy per magnetic phase). Each proposes S_i' = s_i * (unit vector u') from the
 *   current direction u = S_i/|S_i|; the proposal density depends only on the angle between
 *   u and u', so Metropolis acceptance (Eq. 4) is unchanged:
 *   VEGAS_POLICY_RANDOM        u' uniform on the sphere (the default, Sec. III.B)
 *   VEGAS_POLICY_SPIN_FLIP     u' = -u
 *   VEGAS_POLICY_SMALL_STEP    u' uniform in the cap of half-angle theta (param) around u
 *   VEGAS_POLICY_GAUSSIAN      u' = direction of u + sigma g, g three standard normals,
 *                              sigma = param
 *   VEGAS_POLICY_HINZKE_NOWAK  spin flip, random or small step (cap half-angle = param),
 *                              each with probability 1/3 (Hinzke & Nowak's combination)
 *   VEGAS_POLICY_QISING        mixed-spin Ising: S_i = (0, 0, m), m in {-s_i, -s_i + 1, ..., s_i}
 *                              (2 s_i a whole number from 1 to 64); the trial is one of the 2 s_i
 *                              other values, uniformly; such sites start at a uniform value and
 *                              are not renormalised (their length is |m|)
 *   VEGAS_POLICY_ADAPTIVE      Gaussian with one width sigma per instance (starting at the
 *                              param of the first adaptive type); after each MCS of the
 *                              first fifth of every temperature/field step, sigma <-
 *                              sigma * 0.5 / max(1 - R, 0.01), R the MCS's acceptance rate
 *                              over all sites of the instance, clamped to [1e-4, 100]; then
 *                              frozen, so the rest of the step is a plain Metropolis chain
 *                              whose acceptance rate sits near 1/2.
 * Sweep order: one MCS visits every site once, colour class by colour class of a proper
 *   colouring (greedy in site order unless the caller gives one). Sites of one class
 *   share no link, so they are updated in parallel with exactly the result of any
 *   sequential order.
 *
 * Instances: n_samples samples, each run as `replicas` independent replicas; instance
 *   id = inst_base + sample * replicas + replica. Random numbers are Philox4x32-10 keyed
 *   by the seed, with counter (site id in the caller's numbering, global MCS index,
 *   instance id, purpose), so a result does not depend on how instances are batched.
 *
 * Ownership: every pointer passed in stays owned by the caller and is only read during
 *   the call. The library owns all device memory and frees it in vegas_destroy.
 * Errors: a call that fails returns a non-zero vegas_status and stores a message
 *   readable with vegas_last_error(ctx) (vegas_last_error(NULL) for vegas_create).
 *   After VEGAS_ECUDA, VEGAS_EDEVICE or VEGAS_ETIMEOUT the context is poisoned: later calls return
 *   VEGAS_ESTATE, except vegas_last_error, vegas_stats and vegas_destroy.
 * Threads: one context must not be used from two threads at once.
 */
#ifndef VEGAS_H
#define VEGAS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vegas_ctx vegas_ctx;

typedef enum {
    VEGAS_OK = 0,
    VEGAS_EINVAL = 1,   /* invalid argument or sample (message says which) */
    VEGAS_ENOMEM = 2,   /* host or device allocation failed */
    VEGAS_ECUDA = 3,    /* a CUDA runtime call failed (no device, launch error, ...) */
    VEGAS_ETIMEOUT = 4, /* a bounded device wait ran out (grid barrier of the cooperative sweep,
                           dependency wait of the wavefront sweep) */
    VEGAS_EDEVICE = 5,  /* a kernel flagged an error: NaN energy change, sampler cap */
    VEGAS_ESTATE = 6    /* context poisoned by an earlier ECUDA/EDEVICE/ETIMEOUT */
} vegas_status;

/*
 * One sample: the material file of Sec. III.C (sites, spin norms, field axes, types and
 * exchange links) plus the anisotropy file, as arrays. Links are a directed CSR in which
 * every link appears in both directions with equal J (J[i->j] == J[j->i]); no self-links,
 * no duplicate links, col in [0, n_sites). Optional arrays may be NULL (default noted).
 * The order of a row is kept: the local field sums neighbours in that order.
 */
typedef enum {
    VEGAS_POLICY_RANDOM = 0,
    VEGAS_POLICY_SPIN_FLIP = 1,
    VEGAS_POLICY_SMALL_STEP = 2,
    VEGAS_POLICY_GAUSSIAN = 3,
    VEGAS_POLICY_HINZKE_NOWAK = 4,
    VEGAS_POLICY_ADAPTIVE = 5,
    VEGAS_POLICY_QISING = 6
} vegas_policy;

typedef struct {
    int32_t n_sites;           /* >= 1 and < 2^31 */
    int32_t n_policy_types;    /* entries of type_policy and type_param; 0: every site random */
    int64_t n_edges;           /* == row_ptr[n_sites] */
    const int64_t *row_ptr;    /* [n_sites + 1], row_ptr[0] == 0, non-decreasing */
    const int32_t *col;        /* [n_edges] neighbour site */
    const double *J;           /* [n_edges] exchange J_ij (Eq. 1) */
    const int32_t *type;       /* [n_sites] or NULL (all 0); selects the update policy */
    const double *spin_norm;   /* [n_sites] s_i > 0, or NULL (all 1) */
    const double *field_axis;  /* [n_sites][3] n_i, or NULL (all +z) */
    const double *k_uni;       /* [n_sites] uniaxial constant k_i (Eq. 2), or NULL (0) */
    const double *e_uni;       /* [n_sites][3] uniaxial axis e_i, or NULL (all +z) */
    const double *k_cub;       /* [n_sites] cubic constant (Eq. 3), or NULL (0) */
    const int32_t *color;      /* [n_sites] proper colouring, or NULL (greedy) */
    const double *init_spins;  /* [n_sites][3] initial state for every replica, or NULL:
                                  S_i = s_i * uniform-on-sphere from Philox */
    const double *positions;   /* [n_sites][3] site coordinates, or NULL. Used only to order
                                  sites in device memory (a Morton curve inside each colour
                                  class) so that a sweep's neighbour reads stay in L2; results
                                  do not depend on it. */
    const int32_t *type_policy; /* [n_policy_types] vegas_policy of each site type, or NULL
                                   when n_policy_types == 0. With a table, every type must
                                   lie in [0, n_policy_types). */
    const double *type_param;   /* [n_policy_types]: cap half-angle theta in (0, pi] radians
                                   (small step, Hinzke-Nowak), width sigma > 0 (Gaussian,
                                   adaptive), ignored (random, spin flip, qIsing) */
} vegas_sample;

typedef struct {
    int32_t precision;      /* 64: FP64 spins and arithmetic; 32: FP32 spins and energy
                               changes with FP64 history sums. Default 32. */
    int32_t replicas;       /* replicas per sample: 1, 2, 4, 8, 16 or 32. Default 1. */
    uint64_t seed;          /* Philox key. Default 1. */
    int32_t inst_base;      /* id of the first instance. Default 0. */
    int32_t device;         /* CUDA device ordinal, -1 = current. Default -1. */
    void *cuda_stream;      /* cudaStream_t to run on, NULL = a stream of the library */
    int32_t variant;        /* -1 automatic: the first run times each eligible sweep and block
                               shape on a few MCS of the real chain and keeps the fastest
                               (vegas_stats reports the choice); 0 one launch per colour
                               class, 1 resident: one persistent launch per step, a block per
                               instance (FP32), 2 cooperative: one launch per step, all blocks
                               sweep one sample class by class (FP32 or FP64, one sample, no
                               adaptive policy), 3 cluster: one persistent launch per step, a thread-
                               block cluster of 2 .. 16 blocks per instance, the blocks meeting at
                               the hardware cluster barrier between colour classes (FP32),
                               4 wavefront: one launch per MCS runs both colour classes,
                               a block of class-1 sites starting once the class-0 blocks
                               it links to have finished (FP32, one sample, 32
                               replicas, two colour classes, six links per site, no policy
                               table, no per-type statistics; sites are stored plane by plane
                               when positions are given). Variant 4 is used only when asked
                               for. Default -1. */
    int32_t accept_log_mcs; /* > 0: keep the accept/reject bit of every attempt of the
                               first accept_log_mcs MCS (debugging and parity). Default 0. */
    int32_t timing;         /* 1: time every sweep launch with CUDA events. Default 0. */
    int32_t graphs;         /* 1: launch a whole run as one CUDA graph (a conditional while
                               node over its temperature/field steps; the launches of one step
                               as its body), falling back to the next form if the device or
                               driver cannot build it;
                               2: one graph per step (per-class and resident sweeps; the others
                               launch directly); 0: no graphs. Default 1. */
    int32_t max_blocks;     /* > 0: at most this many thread blocks per sweep launch (tests,
                               tuning); 0 = as many as fit on the device. Default 0. */
    int32_t pipeline_depth; /* FP32 sweeps of rows with six links: groups of rows kept in
                               flight per warp, 2 or 3; 1 = no staging (direct kernel);
                               0 = automatic. Default 0. */
    int64_t timeout_ns;     /* longest wait of a block at a grid barrier of the cooperative
                               sweep, or of a warp for the dependencies of one block of the
                               wavefront sweep, before the run fails with VEGAS_ETIMEOUT;
                               0 = 2 s. */
    int32_t fault_inject;   /* testing only: 1 = in the cooperative sweep one block leaves
                               before its first grid barrier, and in the wavefront sweep the
                               first block of class-0 sites is never reported finished, so the
                               blocks that wait for it time out. Default 0. */
    int32_t type_stats;     /* 1: also record the magnetization of every site type (magnetic
                               phase, Sec. II) after every MCS (vegas_type_history). Sites are
                               then stored type by type inside each colour class, and the
                               cooperative sweep is not used. Default 0. */
    int32_t snapshots;      /* 1: keep every instance's spins at the end of every
                               temperature/field step (after the renormalisation; Sec. II, the
                               final state per step), read with vegas_get_snapshot. Costs a
                               device copy of the spins per step and host memory for all of
                               them. Default 0. */
    int32_t cluster_blocks; /* cluster sweep (variant 3): blocks per cluster, 2 .. 16;
                               0 = by instance size (about 2048 sites per block) */
    int32_t cluster_threads;/* cluster sweep: threads per block, 256 or 512; 0 = 256 */
    int32_t group_threads;  /* resident sweep (variant 1) and the single-block phase of the
                               cluster sweep: instances of at most group_sites sites are swept
                               several to a block, group_threads threads (64, 128 or 256) each,
                               each group meeting at its own named barrier; 0 = one instance
                               per block. The automatic choice picks its own. Default 0. */
    int32_t group_sites;    /* see group_threads. Default 0. */
    int32_t cluster_split;  /* cluster sweep (variant 3): instances of at most this many sites
                               are swept by one block each, larger ones by a whole cluster;
                               0 = every instance by a cluster. The automatic choice (variant
                               -1) picks its own. Default 0. */
    int32_t wave_lag;       /* wavefront sweep: a class-1 block is queued this many class-0
                               blocks after the last class-0 block it links to, so that its
                               dependencies have usually finished when a warp reaches it;
                               0 = the number of warps of the launch. Default 0. */
    int32_t wave_slab;      /* wavefront sweep with positions: sites are stored slab by slab
                               along x, each slab plane by plane (z, then y, then x), so the
                               planes in flight stay a few MB at any cross-section; > 0 the slab
                               width in position units, 0 automatic (slabs of about 16384 sites
                               per plane; whole planes when they are no larger), -1 whole planes.
                               Default 0. */
    int32_t resident_smem;  /* resident and cluster sweeps (variants 1, 3): 1 keeps the spins
                               in shared memory for all MCS of a step (12 bytes per site; instances
                               of at most 17066 sites): the resident sweep holds each instance in its
                               block (512 threads), the cluster sweep a copy of it in every
                               block of the cluster, an accepted spin written to every copy through
                               distributed shared memory; -1 never; 0 the automatic choice times it
                               beside the other shapes (with variant 1 or 3 fixed: global memory).
                               Default 0. */
    int32_t renorm_fold;    /* FP32, one sample of two colour classes swept by the kernel of 32
                               replicas per site (per-class sweep): 0 renormalises the spins to
                               their norms s_i inside the step's last class-1 pass instead of in
                               a pass of their own (the same arithmetic at the same point of the
                               step, so the same bits); -1 always in a pass of their own.
                               Default 0. */
} vegas_options;

typedef struct {
    int32_t n_samples, n_instances, replicas, precision;
    int32_t max_colours;        /* largest colour count over samples */
    int32_t variant;            /* variant used by the last run */
    int64_t n_sites;            /* sites over all samples (one replica) */
    int64_t n_edges;            /* directed links over all samples */
    int64_t records;            /* history records per instance so far */
    uint32_t mcs_done;          /* global MCS counter t */
    uint32_t device_error;      /* error bits set by kernels (1 NaN dE, 2 sampler cap,
                                   4 index check failed in a debug build, 8 bounded wait timed out) */
    int64_t kernel_launches;    /* kernels launched by the library so far */
    int64_t sweep_launches;     /* colour-pass (or resident) sweep launches so far */
    double sweep_ms;            /* summed event time of sweep launches (timing = 1) */
    double last_run_ms;         /* event time of the last vegas_run on the device */
    int64_t device_bytes;       /* device memory held by the context */
    int32_t n_types;            /* site types tracked per instance (type_stats), else 0 */
    int32_t pad_;
    int64_t snapshot_steps;     /* steps with a stored final state per instance (snapshots) */
    int32_t block_threads;      /* threads per block of the sweep in use (the resident sweep's
                                   is chosen by the autotuner: 256 or 512) */
    int32_t cluster_blocks;     /* blocks per cluster of the cluster sweep when it is in use
                                   (chosen by the autotuner), else 0 */
    int64_t graph_launches;     /* CUDA graph launches so far: with graphs = 1 a run is one
                                   launch of a graph whose conditional while node repeats one
                                   temperature/field step */
    int32_t split_sites;        /* cluster sweep in use: instances of at most this many sites
                                   are swept by one block each, larger ones by a whole cluster
                                   (chosen by the autotuner; 0 = every instance by a cluster) */
    int32_t group_threads;      /* resident or cluster sweep in use: threads per small instance
                                   swept several to a block (0 = one instance per block) */
    int32_t group_sites;        /* the largest instance swept that way */
    uint32_t sweep_kernels;     /* the kernels of the sweep in use (the variant of the last run),
                                   one VEGAS_KERNEL_* bit each */
} vegas_stats_t;

/* Bits of vegas_stats_t.sweep_kernels: which sweep kernels a run launches. */
#define VEGAS_KERNEL_PASS64 0x1u               /* FP64 colour pass */
#define VEGAS_KERNEL_PASS32_DIRECT 0x2u        /* FP32 colour pass, plain loads, any rows */
#define VEGAS_KERNEL_PASS32_STAGED 0x4u        /* FP32 colour pass, staged rows of six links */
#define VEGAS_KERNEL_PASS32_R32 0x8u           /* FP32 colour pass, 32 replicas per site */
#define VEGAS_KERNEL_PASS32_R32_POLICY 0x10u   /* the same with an update-policy table */
#define VEGAS_KERNEL_RESIDENT32 0x20u          /* resident (persistent) sweep */
#define VEGAS_KERNEL_COOP32 0x40u              /* cooperative sweep, FP32 */
#define VEGAS_KERNEL_CLUSTER32 0x80u           /* cluster sweep */
#define VEGAS_KERNEL_WAVE32 0x100u             /* wavefront sweep */
#define VEGAS_KERNEL_PASS32_R32_ONE_POLICY 0x200u /* 32 replicas per site, compiled for the one
                                                     update policy of every site of the class */
#define VEGAS_KERNEL_RESIDENT32_SMEM 0x400u    /* resident sweep, spins in shared memory */
#define VEGAS_KERNEL_CLUSTER32_SMEM 0x800u     /* cluster sweep, spins copied in every block's
                                                  shared memory */
#define VEGAS_KERNEL_PASS32_R32_RENORM 0x1000u /* 32 replicas per site, the step's last class-1
                                                  pass renormalising every spin (renorm_fold) */
#define VEGAS_KERNEL_COOP64 0x2000u            /* cooperative sweep, FP64 */

/* Fills *opt with the defaults listed above. */
void vegas_default_options(vegas_options *opt);

/*
 * Build a context: validate every sample, colour it (greedy in site order when no
 * colouring is given), renumber sites colour-major (colour 0 first) while keeping the
 * caller's ids for random-number keys and the caller's neighbour order inside each row,
 * upload topology and parameters, and set the initial spins (Sec. III.C material file;
 * Sec. III.B "an initial state is chosen"). opt may be NULL (defaults).
 * Returns VEGAS_EINVAL for: n_samples < 1; a NULL required array; row_ptr not starting
 * at 0, decreasing, or not ending at n_edges; col out of range; a self-link; a duplicate
 * link; J not symmetric; a non-finite parameter; spin_norm <= 0; a colouring
 * that is not proper; a policy table with an unknown policy, a parameter out of range or
 * a site type outside it; bad options. On failure *out is NULL.
 */
vegas_status vegas_create(const vegas_sample *samples, int32_t n_samples, const vegas_options *opt,
                          vegas_ctx **out);

/*
 * Continue the Markov chain of every instance through n_steps temperature/field steps
 * of mcs_per_step MCS each (Sec. III.C parameters; Sec. II history). T and B are
 * [n_instances][n_steps] host arrays (row-major), T > 0 and finite, B finite. The state
 * carries over between steps and between calls; one call with n_steps = a + b gives the
 * same spins and history as a call with the first a steps followed by a call with the
 * remaining b. After every MCS one history record (E, Mx, My, Mz) per instance is kept,
 * with the number of accepted attempts (and, with type_stats, the magnetization of every
 * site type); after the last MCS of every step each spin is rescaled to its norm s_i in
 * FP64 (and, with snapshots, the spins are kept).
 * Blocking: returns when the device work is done.
 */
vegas_status vegas_run(vegas_ctx *ctx, const double *T, const double *B, int32_t n_steps, int32_t mcs_per_step);

/*
 * Copy the history into out as [n_instances][records][4] doubles (E, Mx, My, Mz; totals
 * over the instance's sites, FP64), records in run order. With out == NULL only
 * *n_written is set (to the number of doubles). Returns VEGAS_EINVAL if capacity_doubles
 * is too small.
 */
vegas_status vegas_history(const vegas_ctx *ctx, double *out, size_t capacity_doubles, size_t *n_written);

/* Spins of one instance as [n_sites][3] doubles in the caller's site order. */
vegas_status vegas_get_spins(const vegas_ctx *ctx, int32_t instance, double *out);

/* Replace the spins of one instance ([n_sites][3] doubles, caller's site order; each
 * vector is used as given, FP32 contexts round it). For checkpoint/resume. */
vegas_status vegas_set_spins(vegas_ctx *ctx, int32_t instance, const double *in);

/*
 * Set the global MCS counter t that keys the random numbers of the next MCS (the value
 * vegas_stats reports as mcs_done). With the spins (vegas_set_spins) and, for adaptive
 * policies, the widths (vegas_set_adaptive_width) of a checkpoint, a new context continues
 * the chain bit for bit where the checkpointed one stopped. t < 2^32 - 1; VEGAS_EINVAL
 * otherwise.
 */
vegas_status vegas_set_mcs_counter(vegas_ctx *ctx, uint32_t t);

/*
 * Accept/reject bits of the first accept_log_mcs MCS (option), as
 * [mcs][n_instances][n_sites] bytes (1 = accepted) in the caller's site order.
 * out == NULL: size query.
 */
vegas_status vegas_accept_log(const vegas_ctx *ctx, uint8_t *out, size_t capacity, size_t *n_written);

/*
 * Accepted attempts of every MCS, as [n_instances][records] counts (one per history
 * record, same order); acceptance rate = count / n_sites of the instance's sample.
 * out == NULL: size query (*n_written = number of counts).
 */
vegas_status vegas_accept_history(const vegas_ctx *ctx, uint32_t *out, size_t capacity, size_t *n_written);

/*
 * Width sigma of the adaptive policy of every instance ([n_instances] doubles; 0 for
 * instances whose sample has no adaptive type). _set replaces them (checkpoint/resume);
 * values must be finite and > 0 where the sample adapts, and are ignored elsewhere.
 */
vegas_status vegas_adaptive_width(const vegas_ctx *ctx, double *out);
vegas_status vegas_set_adaptive_width(vegas_ctx *ctx, const double *in);

/*
 * Magnetization of every site type after every MCS (option type_stats), as
 * [n_instances][records][n_types][3] doubles: the sum of S_i over the instance's sites of
 * type k (types 0 .. n_types-1, n_types = 1 + the largest type over all samples; a sample
 * without types has every site in type 0). Summed over k it equals the history's
 * (Mx, My, Mz). out == NULL: size query. VEGAS_EINVAL without type_stats.
 */
vegas_status vegas_type_history(const vegas_ctx *ctx, double *out, size_t capacity, size_t *n_written);

/*
 * Spins of one instance at the end of temperature/field step `step` (0 = the first step
 * ever run on this context; option snapshots), as [n_sites][3] doubles in the caller's site
 * order. VEGAS_EINVAL without snapshots or for a step not yet run.
 */
vegas_status vegas_get_snapshot(const vegas_ctx *ctx, int32_t instance, int64_t step, double *out);

/* ---------------------------------------------------------------- history analysis
 * Stand-alone (no context): host arrays in and out, device temporaries allocated and freed
 * inside the call, FP64 throughout. Errors: the status and vegas_analysis_last_error().
 */

/* Fields per series of vegas_thermal_averages, in this order. */
#define VEGAS_AVG_FIELDS 16
/*   0 e     = <E>/N            1 e_err  (binned standard error)
 *   2 m     = <|M|>/N          3 m_err  (binned)
 *   4 c     = (<E^2> - <E>^2) / (N T^2)      5 c_err   (jackknife over the bins)
 *   6 chi   = (<M^2> - <|M|>^2) / (N T)      7 chi_err (jackknife)
 *   8 u4    = 1 - <M^4> / (3 <M^2>^2)        9 u4_err  (jackknife; Binder cumulant)
 *  10 v1    = <E> - <|M| E> / <|M|>         11 v2 = <E> - <M^2 E> / <M^2>
 *           (v_j = d ln<|M|^j> / d beta, the cumulants of finite-size scaling, Sec. IV.B)
 *  12 tau_e, 13 tau_m: integrated autocorrelation times of E and |M| in MCS (Sec. II), with
 *           Sokal's automatic window (the smallest W >= 6 tau(W), at most n/2)
 *  14 n (records used), 15 n_bins. k_B = 1; E, M are the totals of a history record. */

/*
 * Thermal averages of n_series histories (one temperature/field step of one instance each),
 * series = [n_series][len][4] (E, Mx, My, Mz after every MCS, as from vegas_history), the
 * first `cut` records of each dropped (thermalisation). Bins: b = (len - cut) / n_bins
 * records each over the first b * n_bins records after the cut. T[s] and n_sites[s] are the
 * series' temperature and site count. out = [n_series][VEGAS_AVG_FIELDS]. cuda_stream: a
 * cudaStream_t or NULL. Returns VEGAS_EINVAL for 0 > cut >= len, n_bins outside [2, 64],
 * fewer records than bins, T or n_sites <= 0 or non-finite.
 */
vegas_status vegas_thermal_averages(const double *series, int64_t n_series, int64_t len, int64_t cut,
                                    int32_t n_bins, const double *T, const double *n_sites, double *out,
                                    void *cuda_stream);

/*
 * Single and multiple histogram reweighting (Sec. IV.E; Ferrenberg & Swendsen 1988, 1989):
 * K runs at inverse temperatures betas_k with n samples each, energies E = [K][n] and
 * observables O = [K][n][n_obs] (n_obs <= 8, may be 0). The free energies g_k = ln Z_k -
 * ln Z_0 solve g_k = ln sum_i exp(-beta_k E_i - D_i), D_i = ln sum_j n exp(-beta_j E_i -
 * g_j), iterated from g = 0 until max |change| < tol or max_iter iterations; then
 * out[b][q] = <O_q> at betas_out[b]. K = 1 is the single-histogram method. g_out ([K]) and
 * iters_out may be NULL.
 */
vegas_status vegas_reweight(const double *E, const double *O, int32_t K, int64_t n, int32_t n_obs,
                            const double *betas_k, const double *betas_out, int32_t n_out, int32_t max_iter,
                            double tol, double *out, double *g_out, int32_t *iters_out, void *cuda_stream);

/* Message of the last failed analysis call on this thread. */
const char *vegas_analysis_last_error(void);

/* ---------------------------------------------------------------- Ising model
 * Ising systems with the spin-flip policy (Sec. II; the 2D Ising workloads of Sec. IV.B and
 * IV.E): s = +-1 on a periodic square (dims 2) or simple cubic (dims 3) lattice of side L,
 * E = -J sum_<ij> s_i s_j - h sum_i s_i (each bond once), site id i = x + L (y + L z).
 * One MCS = every site of colour 0 ((x + y + z) even), then every site of colour 1, each
 * with one flip attempt: dE = 2 s_i (J sum_j s_j + h); accepted iff dE <= 0 or
 * u < exp(-dE / T), u = w 2^-32 with w the word (inst & 3) of Philox4x32-10(seed; i, t,
 * inst >> 2, 0x80000), t the global MCS counter. Initial state: s_i = +1 iff bit 31 of word
 * (inst & 3) of Philox(seed; i, 0xFFFFFFFF, inst >> 2, 0x90000) is set (or all +1).
 * Device layout: 32 sites of one replica per 32-bit word (multi-spin coding along x, one
 * array per colour); acceptance by integer thresholds computed on the host, so the result
 * is the same bit for bit as the definition above. Replicas are independent instances with
 * their own temperature and field.
 */
typedef struct vegas_ising vegas_ising;

typedef struct {
    int32_t dims;        /* 2 or 3 */
    int32_t L;           /* side: a multiple of 64, L^dims < 2^31 */
    double J;            /* exchange (finite) */
    int32_t replicas;    /* a multiple of 4, at most 512 */
    int32_t inst_base;   /* id of replica 0: a multiple of 4 */
    uint64_t seed;       /* Philox key */
    int32_t device;      /* CUDA device ordinal, -1 = current */
    void *cuda_stream;   /* cudaStream_t, NULL = a stream of the library */
    int32_t init_up;     /* 1: every spin +1; 0: the Philox initial state */
    int32_t timing;      /* 1: time every sweep launch with CUDA events */
} vegas_ising_options;

void vegas_ising_default_options(vegas_ising_options *opt);
vegas_status vegas_ising_create(const vegas_ising_options *opt, vegas_ising **out);
/* T, h: [replicas][n_steps] (T > 0); records (E, M) after every MCS. Blocking. */
vegas_status vegas_ising_run(vegas_ising *ctx, const double *T, const double *h, int32_t n_steps,
                             int32_t mcs_per_step);
/* History as [replicas][records][2] doubles (E, M); out == NULL: size query. */
vegas_status vegas_ising_history(const vegas_ising *ctx, double *out, size_t capacity, size_t *n_written);
/* Spins of one replica as L^dims int8 (+1 / -1) in site-id order. */
vegas_status vegas_ising_get_spins(const vegas_ising *ctx, int32_t replica, int8_t *out);
vegas_status vegas_ising_set_spins(vegas_ising *ctx, int32_t replica, const int8_t *in);
/* Global MCS counter of the next MCS, as vegas_set_mcs_counter (checkpoint/resume). */
vegas_status vegas_ising_set_mcs_counter(vegas_ising *ctx, uint32_t t);
/* n_instances, n_sites, records, mcs_done, kernel_launches, sweep_launches, sweep_ms,
 * last_run_ms, device_bytes are filled; the other fields are 0. */
vegas_status vegas_ising_stats(const vegas_ising *ctx, vegas_stats_t *out);
const char *vegas_ising_last_error(const vegas_ising *ctx);
void vegas_ising_destroy(vegas_ising *ctx);

/* Counters and sizes of the context (valid also on a poisoned context). */
vegas_status vegas_stats(const vegas_ctx *ctx, vegas_stats_t *out);

/*
 * Greedy colouring used by vegas_create when a sample has no colouring: sites in index
 * order, each takes the smallest colour not used by an already coloured neighbour.
 * Host only (no device needed). Returns the number of colours, or -1 on invalid input
 * (n_sites < 0, a NULL array, row_ptr not starting at 0 or decreasing, col out of range);
 * row_ptr must hold n_sites + 1 entries and col row_ptr[n_sites].
 */
int32_t vegas_greedy_colour(int32_t n_sites, const int64_t *row_ptr, const int32_t *col, int32_t *color_out);

/*
 * One MCS on device memory the caller owns; the library allocates nothing.
 *
 * The paper has no counterpart: this entry point exists for callers that cannot let a
 * library call cudaMalloc (programs that manage every device byte in their own pool or
 * arena, loops that cannot afford the implicit device synchronisation of an allocation,
 * plug-in hosts that hand out fixed buffers). They cannot create a context, so the data
 * comes as device pointers, and the sweep keeps its scratch (partial sums of E and M for
 * at most 1024 thread blocks x 32 replicas, the run state, the error word: about 1 MB) in
 * a static device array of the library that every GPU loading the library holds until
 * the process exits.
 *
 * Layout (the library's own): sites numbered colour-major, colour class c being sites
 * [colour_start[c], colour_start[c+1]); no link joins two sites of one class.
 *   spins     device, [n_sites][replicas] x (x, y, z, unused) float32, 16-byte aligned;
 *             updated in place
 *   links     device, 8-byte aligned, [n_edges] x (neighbour index as int32, J as float32
 *             bits), every link present in both directions with equal J; every neighbour
 *             index in [0, n_sites)
 *   row_ptr   device, 8-byte aligned, [n_sites + 1] int64 link offsets: row_ptr[0] == 0,
 *             non-decreasing, row_ptr[n_sites] == n_edges (the links array's length)
 *   site_id   device, 4-byte aligned, [n_sites] int32 ids used as Philox keys (the caller's
 *             numbering)
 *   colour_start  host, [n_colours + 1], from 0 to n_sites, n_colours <= 64
 *   replicas  1, 2, 4, ..., 32 (larger values are rejected: the scratch holds 32)
 *   beta, field   host, [replicas]: 1/T > 0 and B of each replica
 *   site_params   host, 9 doubles (nx, ny, nz, s, ex, ey, ez, k, kc) shared by all
 *             sites, or NULL (field axis +z, s = 1, no anisotropy)
 *   seed, inst0, t  Philox key, instance id of replica 0, global MCS index
 *   out       device, 8-byte aligned, [replicas][4] doubles: (E, Mx, My, Mz) after the MCS
 *   stream    cudaStream_t or NULL (legacy default stream)
 * The device arrays are not validated (the library cannot read them without copies):
 * neighbour indices outside [0, n_sites) or row offsets past the links array are undefined
 * behaviour. A debug build of the library (build(debug=True)) checks every row and
 * neighbour index in the kernel and reports a bad one as VEGAS_EDEVICE (flag 4) instead of
 * reading through it.
 * Computes what vegas_run computes for one MCS of an FP32 context with these replicas
 * (same random numbers for the same seed, ids, instances and t); no renormalisation.
 * Set-up: the first call on a device (and the first after that device's context has been
 * replaced, e.g. by cudaDeviceReset) looks up the device address of the static scratch
 * (cudaGetSymbolAddress) with that device current; make that first call before any stream
 * capture begins. Blocking: every call waits for the sweep to finish on `stream` and reads
 * the error word back with a blocking copy before it returns. Every call uses the same
 * scratch and rewrites it; calls whose GPU work overlaps (other threads, other streams)
 * race on it. Errors: VEGAS_EINVAL for bad sizes, NULL or misaligned pointers (message from
 * vegas_noalloc_last_error), VEGAS_ECUDA, VEGAS_EDEVICE (1: NaN energy change; 4: a bad
 * index seen by a debug build).
 */
vegas_status vegas_sweep_noalloc(void *spins, const void *links, const int64_t *row_ptr, const int32_t *site_id,
                                 int32_t n_sites, const int32_t *colour_start, int32_t n_colours, int32_t replicas,
                                 const double *beta, const double *field, const double *site_params, uint64_t seed,
                                 int32_t inst0, uint32_t t, double *out, void *stream);

/* Message of the last failed vegas_sweep_noalloc call of this thread. Never NULL. */
const char *vegas_noalloc_last_error(void);

/* Message of the last failed call on ctx (ctx == NULL: last failed vegas_create of this
 * thread). Valid until the next call on ctx. Never NULL. */
const char *vegas_last_error(const vegas_ctx *ctx);

/* Free the context and its device memory. NULL is accepted. */
void vegas_destroy(vegas_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* VEGAS_H */
