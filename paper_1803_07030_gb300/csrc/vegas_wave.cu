// Wavefront sweep (R = 32 replicas, rows of six links, two colour classes): one launch runs
// both colour classes of an MCS (Sec. II, Eq. 4), so the rows that the class-0 half of the
// sweep reads are still in L2 when the class-1 half needs them.
//
// Each class is cut into blocks of 8 consecutive sites. The host lists the blocks in sweep
// order: class-0 blocks in memory order, and each class-1 block some distance after the
// last class-0 block that holds one of its neighbours, and gives every class-1 block the row
// of distinct class-0 blocks it links to. Every warp draws the index of its next task from a
// ticket counter (so the tasks in flight are always about one per warp, consecutive in the
// list: a narrow window that L2 holds), and runs it as eight groups of one site x 32
// replicas with the depth-2 cp.async pipeline of the batched per-class kernel. A class-0
// block publishes done[b] = t + 1 when its spins are stored; a class-1 block reads its
// neighbours' rows only after every class-0 block of its row has published (one acquire
// load per lane). Since class-1
// sites link only to class-0 sites, this gives every attempt the same neighbour values as
// the per-class sweep (class 0 from the previous MCS, class 1 after class 0 of this MCS),
// and the same Philox counters, so the spins are bit for bit those of that sweep.
//
// Progress: the lowest unfinished ticket is held by a running warp whose earlier task is
// finished (it was a lower ticket), and the task's dependencies have lower tickets, so it
// can always proceed; no co-residency of the grid is needed. Each wait is
// still bounded by timeout_ns; a warp that gives up sets kErrTimeout, which makes every
// other waiting warp give up too, and all warps still meet at the block reduction.
#include <cuda_runtime.h>

#include <cstdint>

#include "vegas_device.cuh"
#include "vegas_internal.h"
#include "vegas_staged.cuh"

namespace vegas {
namespace {

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t *p) { return *(const volatile uint32_t *)p; }

__device__ __forceinline__ uint64_t wave_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr int kWaveBS = kWaveBlockSites;                    // sites per block (task)
constexpr int kWaveRows = 2 * 7 * 32 * 16;                  // two groups of 7 rows of 32 replicas
constexpr int kWaveLinkBytes = kWaveBS * 6 * 8;             // the block's links (col, J)
constexpr int kWaveSlot = kWaveLinkBytes + kWaveBS * 4;     // links + caller ids
constexpr int kWaveWarpBytes = kWaveRows + 2 * kWaveSlot;
constexpr int kWaveSmem = (kThreads / 32) * kWaveWarpBytes;

template <int PM>
__global__ void __launch_bounds__(kThreads, 3) wave32_r32(const WaveArgs w) {
    constexpr int DEG = 6, BS = kWaveBS, R = 32;
    extern __shared__ __align__(16) unsigned char smem[];
    const PassArgs &a = w.pass;
    const RunState *rs_ = a.run;
    const uint32_t t = rs_->t, tag = t + 1u;
    const uint32_t step_idx = rs_->rec / rs_->mcs;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = lane;
    unsigned char *wbase = smem + warp * kWaveWarpBytes;
    float4 *rows = (float4 *)wbase;
    unsigned char *lslots = wbase + kWaveRows;
    float4 *S = (float4 *)a.spins;
    const float4 *Sr = S + r;
    const int2 *E = (const int2 *)a.edges;
    const uint32_t inst = (uint32_t)(a.inst0 + r);
    const double *sc = rs_->sched + ((int64_t)step_idx * a.n_inst + a.inst_local0 + r) * 2;
    const float beta = (float)sc[0], B = (float)sc[1];
    uint32_t rk0[10], rk1[10];
    {
        uint32_t x = (uint32_t)a.seed, y = (uint32_t)(a.seed >> 32);
#pragma unroll
        for (int q = 0; q < 10; ++q) {
            rk0[q] = x;
            rk1[q] = y;
            x += 0x9E3779B9u;
            y += 0xBB67AE85u;
        }
    }
    // first site and end of block b
    auto block_range = [&](int b, int &sb, int &se) {
        if (b < w.nb0) {
            sb = a.g_begin + b * BS;
            se = min(sb + BS, a.g_end);
        } else {
            sb = w.c1_begin + (b - w.nb0) * BS;
            se = min(sb + BS, w.c1_end);
        }
    };
    auto issue_links = [&](int sb, int se, int slot) {
        const int ns = se - sb;
        unsigned char *dst = lslots + slot * kWaveSlot;
        const unsigned char *src = (const unsigned char *)(E + a.edge_base + (int64_t)(sb - a.site_off) * DEG);
        VEGAS_CHECK(ns >= 1 && ns <= BS && sb >= a.g_begin && se <= w.c1_end, 21, sb);
        VEGAS_CHECK(a.edge_base + (int64_t)(se - a.site_off) * DEG <= a.n_edges_total, 22, sb);
        VEGAS_CHECK(((uintptr_t)src & 15) == 0, 23, sb);
        for (int k = lane; k < ns * (DEG / 2); k += 32) cp16(dst + 16 * k, src + 16 * k);
        if (lane < ns) cp4(dst + kWaveLinkBytes + 4 * lane, a.orig + sb + lane);
    };
    auto issue_rows = [&](int g, int se, int lslot, int j, int rslot) {
        if (g >= se) return;
        const int4 *lk = (const int4 *)(lslots + lslot * kWaveSlot) + j * (DEG / 2);
        float4 *dst = rows + rslot * (DEG + 1) * 32 + lane;
        VEGAS_CHECK(g < a.n_sites_total, 24, g);
#pragma unroll
        for (int q = 0; q < DEG / 2; ++q) {
            const int4 l = lk[q];
            VEGAS_CHECK(l.x >= 0 && l.x < a.n_sites_total && l.z >= 0 && l.z < a.n_sites_total, 25, l.x);
            cp16(dst + (2 * q) * 32, Sr + (int64_t)l.x * R);
            cp16(dst + (2 * q + 1) * 32, Sr + (int64_t)l.z * R);
        }
        cp16(dst + DEG * 32, Sr + (int64_t)g * R);
    };
    // every class-0 block that class-1 block b links to (its row of distinct blocks, one per
    // lane) has finished this MCS (warp-uniform)
    auto deps_ready = [&](int b) -> bool {
        static_assert(kWaveDeps == 32, "one dependency per lane");
        const int d = __ldg(w.deps + (size_t)(b - w.nb0) * kWaveDeps + lane);
#ifdef VEGAS_DEBUG_CHECKS
        if (d >= w.nb0) {
            atomicOr(a.err, kErrIndex);
            atomicCAS(a.err + 1, 0u, 26u);
            a.err[2] = (uint32_t)d;
        }
#endif
        const bool ok = d < 0 || d >= w.nb0 || ld_acquire(w.done + d) == tag;
        return __all_sync(0xFFFFFFFFu, ok);
    };
    // bounded wait for deps_ready; false when this warp or another one gave up
    auto wait_deps = [&](int b) -> bool {
        if (deps_ready(b)) return true;
        const uint64_t t0 = __shfl_sync(0xFFFFFFFFu, wave_ns(), 0);
        for (;;) {
            __nanosleep(128);
            if (deps_ready(b)) return true;
            int give_up = 0;
            if (lane == 0) {
                if (ld_volatile(a.err) & kErrTimeout) {
                    give_up = 1;
                } else if ((int64_t)(wave_ns() - t0) > w.timeout_ns) {
                    atomicOr(a.err, kErrTimeout);
                    give_up = 1;
                }
            }
            if (__shfl_sync(0xFFFFFFFFu, give_up, 0)) return false;
        }
    };

    Acc32 acc;
    bool nan_seen = false;
    const bool log_accepts = a.alog && t < a.alog_mcs;
    int b = 0, sb = 0, se = 0, ls = 0;
    bool pre = false;  // rows of groups 0 and 1 of task m already issued
    uint32_t tk = 0;
    if (lane == 0) tk = atomicAdd(w.ticket, 1u);
    int m = (int)min(__shfl_sync(0xFFFFFFFFu, tk, 0), (uint32_t)w.n_tasks);
    if (m < w.n_tasks) {
        b = __ldg(w.tasks + m);
        block_range(b, sb, se);
        issue_links(sb, se, 0);
        cp_commit();
        cp_wait<0>();
        __syncwarp();
    }
    while (m < w.n_tasks) {
        const bool c1 = b >= w.nb0;
        if (!pre) {
            if (c1 && !wait_deps(b)) break;
            __syncwarp();  // orders the lanes' acquire loads before every lane's row copies
            issue_rows(sb, se, ls, 0, 0);
            cp_commit();
            issue_rows(sb + 1, se, ls, 1, 1);
            cp_commit();
        }
        int m2 = w.n_tasks, b2 = 0, sb2 = 0, se2 = 0;
        bool has2 = false, ready2 = false;
        const unsigned char *slot = lslots + ls * kWaveSlot;
        // unrolled by two (the row slot j & 1 stays a constant): eight copies of the attempt
        // overflow the instruction cache once the dependency and ticket code is added
#pragma unroll 2
        for (int j = 0; j < BS; ++j) {
            cp_wait<1>();
            __syncwarp();
            const int g = sb + j;
            if (g < se) {
                const uint32_t orig = ((const uint32_t *)(slot + kWaveLinkBytes))[j];
                const int4 *lk = (const int4 *)slot + j * (DEG / 2);
                const float4 *row = rows + (j & 1) * (DEG + 1) * 32 + lane;
                // one code path for both classes (class 0: no lower links, lower sums 0)
                staged_attempt_rw<DEG, PM, 3>(a, lk, row, orig, g, r, R, t, trial_block32(orig, t, inst, rk0, rk1), beta,
                                              B, S, acc, nan_seen, log_accepts, nullptr, 0.f, c1);
            }
            __syncwarp();
            // the next ticket: drawn at j = 0, read at j = 2, its links copied at j = 3 (they
            // land by the wait at the top of j = 5)
            if (j == 0 && lane == 0) tk = atomicAdd(w.ticket, 1u);
            if (j == 2) {
                m2 = (int)min(__shfl_sync(0xFFFFFFFFu, tk, 0), (uint32_t)w.n_tasks);
                has2 = m2 < w.n_tasks;
                if (has2) b2 = __ldg(w.tasks + m2);
            }
            if (j == 3 && has2) {
                block_range(b2, sb2, se2);
                issue_links(sb2, se2, ls ^ 1);
            }
            // rows of the next block's first two groups go out at j = BS - 2, BS - 1, after the
            // __syncwarp that follows the wait at the top of those groups
            if (j == BS - 3 && has2) ready2 = b2 < w.nb0 || deps_ready(b2);
            if (j + 2 < BS)
                issue_rows(sb + j + 2, se, ls, j + 2, j & 1);
            else if (ready2)
                issue_rows(sb2 + j + 2 - BS, se2, ls ^ 1, j + 2 - BS, j & 1);
            cp_commit();
        }
        if (!c1) {  // publish: the release by lane 0 orders the stores of every lane before it
            __syncwarp();
            if (lane == 0 && b != w.skip_block) st_release(w.done + b, tag);
        }
        m = m2;
        b = b2;
        sb = sb2;
        se = se2;
        ls ^= 1;
        pre = ready2;
    }
    cp_wait<0>();
    if (nan_seen) atomicOr(a.err, kErrNaN);
    acc.flush();
    block_partials(acc.d, acc.nacc, R, a.partial + (int64_t)blockIdx.x * R * 4, acc_counters(rs_, a.inst_local0));
}

using WaveFn = void (*)(WaveArgs);

WaveFn select_wave(int pm) {
    static const WaveFn tab[3] = {wave32_r32<0>, wave32_r32<1>, wave32_r32<2>};
    return tab[pm < 0 ? 0 : (pm > 2 ? 2 : pm)];
}

}  // namespace

int launch_wave(const WaveArgs &a, int grid, void *stream) {
    const WaveFn k = select_wave(a.pass.params_mode);  // its shared-memory limit is raised by wave_blocks_per_sm
    k<<<grid, kThreads, kWaveSmem, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

int wave_blocks_per_sm(int params_mode) {
    const WaveFn k = select_wave(params_mode);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kWaveSmem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kThreads, kWaveSmem) != cudaSuccess) return 0;
    return nb;
}

}  // namespace vegas
