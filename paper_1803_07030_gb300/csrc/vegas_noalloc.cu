// vegas_sweep_noalloc: one Metropolis MCS on memory the caller owns, with no device
// allocation by the library.
//
// Who needs this: programs that own every byte of device memory themselves and do not
// let a library call cudaMalloc: engines with their own memory pool or arena, code that
// must not trigger the implicit device synchronisation of cudaMalloc/cudaFree in a
// latency-critical loop, and hosts that give a plug-in fixed device buffers only. They
// cannot create a vegas context (vegas_create allocates), so this entry point takes the
// spins, links and caller ids as device pointers and keeps the only scratch it needs (the
// per-block partial sums of energy and magnetization, the run state and the error word)
// in one statically allocated device array of this file.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "vegas_internal.h"

using namespace vegas;

namespace {

constexpr int kNoAllocMaxBlocks = 1024;   // thread blocks over all colour classes of one MCS
constexpr int kNoAllocMaxReplicas = 32;
constexpr int kNoAllocMaxDevices = 64;

struct NoAllocHeader {
    RunState run;
    uint32_t err[4];
    int64_t slot_base[1];
    int32_t slot_count[1];
    int32_t pad_;
    double sched[2 * kNoAllocMaxReplicas];
};

constexpr size_t kHeaderBytes = (sizeof(NoAllocHeader) + 255) / 256 * 256;
constexpr size_t kPartialBytes = sizeof(double) * 4 * (size_t)kNoAllocMaxBlocks * kNoAllocMaxReplicas;

// The scratch: header, then the partial sums. Every GPU that loads the library holds these
// ~1 MB until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kHeaderBytes + kPartialBytes];

struct SetupArgs {
    NoAllocHeader *h;
    double *out;
    uint32_t t;
    int32_t R;
    int32_t blocks;
    double beta[kNoAllocMaxReplicas];
    double B[kNoAllocMaxReplicas];
};

// Writes the run state of one call; everything that must start at zero is cleared here.
__global__ void noalloc_setup(const SetupArgs s) {
    NoAllocHeader *h = s.h;
    const int i = threadIdx.x;
    if (i < s.R) {
        h->sched[2 * i] = s.beta[i];
        h->sched[2 * i + 1] = s.B[i];
    }
    if (i == 0) {
        h->run.t = s.t;
        h->run.rec = 0;
        h->run.ticket = 0;
        h->run.mcs = 1;
        h->run.sched = h->sched;
        h->run.hist = s.out;
        h->run.acc = nullptr;  // no acceptance counts, no adaptive policy here
        h->run.acc_hist = nullptr;
        h->run.sigma = nullptr;
        h->run.type_hist = nullptr;
        for (int q = 0; q < 4; ++q) h->err[q] = 0;
        h->slot_base[0] = 0;
        h->slot_count[0] = s.blocks;
    }
}

// Device address of the scratch, looked up once per CUDA context. The address belongs to the
// context that loaded this module, not to the device ordinal: after the device's primary
// context is reset (cudaDeviceReset) the module is loaded again and the array may sit
// elsewhere, so the cache is keyed by the context's process-unique id (cuCtxGetId).
struct ScratchSlot {
    unsigned long long ctx_id;  // 0: not looked up yet
    void *addr;
};
std::mutex g_mu;
ScratchSlot g_slot[kNoAllocMaxDevices] = {};
thread_local std::string g_err;

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// The unique id of the calling thread's current context, or 0 when there is none yet or the
// driver does not offer the query (the scratch address is then looked up on every call).
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (CtxGetCurrentFn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (CtxGetIdFn)f;
        cudaGetLastError();
    });
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

vegas_status fail(vegas_status st, const std::string &m) {
    g_err = m;
    return st;
}

// A host exception caught at the entry point, as a status (called inside a catch block).
vegas_status noalloc_host_exception() {
    std::string m;
    const vegas_status st = status_of_current_exception(m);
    return fail(st, m);
}

}  // namespace

extern "C" const char *vegas_noalloc_last_error(void) { return g_err.c_str(); }

extern "C" vegas_status vegas_sweep_noalloc(void *spins, const void *links, const int64_t *row_ptr,
                                            const int32_t *site_id, int32_t n_sites, const int32_t *colour_start,
                                            int32_t n_colours, int32_t replicas, const double *beta,
                                            const double *field, const double *site_params, uint64_t seed,
                                            int32_t inst0, uint32_t t, double *out, void *stream) {
    try {
        if (!spins || !links || !row_ptr || !site_id || !colour_start || !beta || !field || !out)
            return fail(VEGAS_EINVAL, "a required pointer is NULL");
        // the kernels load spins as float4, links, row offsets and sums as 8-byte words: a
        // misaligned device pointer would fault the GPU, so it is refused here
        if ((uintptr_t)spins % 16 != 0) return fail(VEGAS_EINVAL, "spins must be 16-byte aligned");
        if ((uintptr_t)links % 8 != 0 || (uintptr_t)row_ptr % 8 != 0 || (uintptr_t)out % 8 != 0)
            return fail(VEGAS_EINVAL, "links, row_ptr and out must be 8-byte aligned");
        if ((uintptr_t)site_id % 4 != 0) return fail(VEGAS_EINVAL, "site_id must be 4-byte aligned");
        if (n_sites < 1) return fail(VEGAS_EINVAL, "n_sites must be >= 1");
        if (replicas < 1 || replicas > kNoAllocMaxReplicas || (replicas & (replicas - 1)))
            return fail(VEGAS_EINVAL, "replicas must be a power of two no larger than 32 (the static scratch holds the "
                                      "partial sums of at most 32 replicas)");
        if (n_colours < 1 || n_colours > kMaxColours) return fail(VEGAS_EINVAL, "n_colours must be in [1, 64]");
        if (colour_start[0] != 0 || colour_start[n_colours] != n_sites)
            return fail(VEGAS_EINVAL, "colour_start must run from 0 to n_sites");
        for (int c = 0; c < n_colours; ++c)
            if (colour_start[c + 1] < colour_start[c]) return fail(VEGAS_EINVAL, "colour_start must not decrease");
        for (int r = 0; r < replicas; ++r)
            if (!(beta[r] > 0.0) || !std::isfinite(beta[r]) || !std::isfinite(field[r]))
                return fail(VEGAS_EINVAL, "beta must be finite and > 0, field finite");

        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return fail(VEGAS_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(VEGAS_EINVAL, "device ordinal too large");
        void *base = nullptr;
        {
            // set-up, once per device and CUDA context, with the device current: the device
            // address of the static scratch (in host code its name is only a host-side handle)
            std::lock_guard<std::mutex> lk(g_mu);
            ScratchSlot &sl = g_slot[dev];
            unsigned long long id = current_context_id();
            if (id == 0 || sl.ctx_id != id) {
                void *addr = nullptr;
                e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
                if (e != cudaSuccess) {
                    sl = ScratchSlot{0, nullptr};
                    return fail(VEGAS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
                }
                if (id == 0) id = current_context_id();  // the lookup made the primary context current
                sl = ScratchSlot{id, addr};
            }
            base = sl.addr;
        }
        NoAllocHeader *hdr = (NoAllocHeader *)base;
        double *partial = (double *)((unsigned char *)base + kHeaderBytes);

        int sm = 0;
        e = cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return fail(VEGAS_ECUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
        int log2R = 0;
        while ((1 << log2R) < replicas) ++log2R;

        // uniform site parameters: (nx, ny, nz, s, ex, ey, ez, k, kc); default +z field axis, s = 1
        double p[9] = {0.0, 0.0, 1.0, 1.0, 0.0, 0.0, 1.0, 0.0, 0.0};
        if (site_params) std::memcpy(p, site_params, sizeof p);
        for (double v : p)
            if (!std::isfinite(v)) return fail(VEGAS_EINVAL, "non-finite site parameter");
        if (!(p[3] > 0.0)) return fail(VEGAS_EINVAL, "spin norm must be > 0");

        // one direct-kernel launch per colour class; their blocks share the scratch's slots
        PassArgs a;
        std::memset(&a, 0, sizeof a);
        a.spins = spins;
        a.edges = links;
        a.row_ptr = row_ptr;
        a.orig = site_id;
        a.run = &hdr->run;
        a.err = hdr->err;
        a.seed = seed;
        a.site_off = 0;
        a.log2R = log2R;
        a.inst0 = inst0;
        a.inst_local0 = 0;
        a.n_inst = replicas;
        a.n_sample_sites = n_sites;
        a.n_sites_total = n_sites;  // debug builds check neighbour indices against it
        a.n_edges_total = 0;        // unknown here: debug builds check rows for order only
        a.deg = 0;
        a.depth = 0;
        a.lower_mode = 2;
        a.params_mode = (p[7] != 0.0 || p[8] != 0.0) ? 1 : 0;
        a.u32 = SiteParams32{(float)p[0], (float)p[1], (float)p[2], (float)p[3], (float)p[4],
                             (float)p[5], (float)p[6], (float)p[7], (float)p[8]};
        a.u64 = SiteParams64{p[0], p[1], p[2], p[3], p[4], p[5], p[6], p[7], p[8]};
        const int per_class = std::max(1, kNoAllocMaxBlocks / n_colours);
        const int occ = sm * pass_blocks_per_sm(32, a);
        int grids[kMaxColours];
        int total = 0;
        for (int c = 0; c < n_colours; ++c) {
            const int64_t work = (int64_t)(colour_start[c + 1] - colour_start[c]) << log2R;
            const int64_t need = (work + kThreads - 1) / kThreads;
            grids[c] = (int)std::max<int64_t>(1, std::min<int64_t>({need, (int64_t)per_class, (int64_t)occ}));
            total += grids[c];
        }
        if (total > kNoAllocMaxBlocks) return fail(VEGAS_EINVAL, "too many colour classes for the static scratch");

        SetupArgs sa;
        std::memset(&sa, 0, sizeof sa);
        sa.h = hdr;
        sa.out = out;
        sa.t = t;
        sa.R = replicas;
        sa.blocks = total;
        for (int r = 0; r < replicas; ++r) {
            sa.beta[r] = beta[r];
            sa.B[r] = field[r];
        }
        cudaStream_t st = (cudaStream_t)stream;
        noalloc_setup<<<1, 32, 0, st>>>(sa);
        int slot = 0;
        for (int c = 0; c < n_colours; ++c) {  // an empty class runs one block that writes zeros
            a.g_begin = colour_start[c];
            a.g_end = colour_start[c + 1];
            a.lower_end = colour_start[c];
            a.partial = partial + (int64_t)slot * replicas * 4;
            launch_pass32(a, grids[c], st);
            slot += grids[c];
        }
        ReduceArgs ra{partial, hdr->slot_base, hdr->slot_count, &hdr->run, nullptr, replicas, replicas, 1, 0, nullptr, 0};
        launch_reduce(ra, st);
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail(VEGAS_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(VEGAS_ECUDA, std::string("sweep: ") + cudaGetErrorString(e));
        uint32_t err = 0;
        e = cudaMemcpy(&err, hdr->err, sizeof err, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail(VEGAS_ECUDA, std::string("error word: ") + cudaGetErrorString(e));
        if (err)
            return fail(VEGAS_EDEVICE, "device error flags " + std::to_string(err) +
                                           " (1: NaN energy change, 4: bad row or neighbour index seen by a debug build)");
        return VEGAS_OK;
    } catch (...) {
        return noalloc_host_exception();
    }
}
