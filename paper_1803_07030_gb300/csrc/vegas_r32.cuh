// The replica-batched FP32 colour pass (R = 32, rows of six links): shared by the translation
// unit of the staged kernels (no policy table, or a table read per site) and the one of the
// kernels specialised to a single update policy.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "vegas_device.cuh"
#include "vegas_internal.h"
#include "vegas_staged.cuh"

namespace vegas {
namespace {

// Replica-batched sweep (R = 32): one warp = one site x 32 replicas, depth-2 pipeline. A
// warp takes blocks of eight consecutive sites from the pass's ticket counter, so the blocks
// in flight stay about one per warp and consecutive in memory order however unevenly the
// warps progress: the neighbour rows they share are still in L2 when the last of them reads
// them. The eight groups of a block are unrolled, so every ring slot and offset is a
// constant: group j of a block computes from row slot j & 1 and its link slot; the next
// ticket is drawn at j = 0 and its block's links copied at j = 4; rows of group j + 2 (the
// next block's first two at j = 6, 7) are copied at the end of group j.
// POL = 1 adds the sites' update policies (8 bytes each, staged with the caller ids); POL =
// 2 + c does the same for a pass whose sites all have policy c, with the trial of that policy
// alone compiled in (each site's parameter still comes from its entry).
// Without a policy table the kernel runs in blocks of 7 warps, four blocks per SM (72
// registers, 56 KB of shared memory each: 28 warps per SM); with one, in blocks of 8 warps,
// three per SM. The block's partial sums are formed in each warp's own shared-memory area
// once its sweep is done, so the block needs no other shared memory.
template <int POL>
struct R32Shape {
    static constexpr int DEG = 6, D = 2, BS = 8;
    static constexpr int WARPS = POL ? 8 : 7, MIN_BLOCKS = POL ? 3 : 4;
    static constexpr int ROWS = D * (DEG + 1) * 32 * 16;
    static constexpr int LINK_BYTES = BS * DEG * 8;
    static constexpr int POL_OFF = LINK_BYTES + BS * 4;
    static constexpr int SLOT = POL_OFF + (POL ? BS * 8 : 0);
    static constexpr int WARP_BYTES = ROWS + 2 * SLOT;
};

// Fixed-order block sums of (E, Mx, My, Mz) per replica and the accepted counts, through the
// warps' own areas of the dynamic shared memory (the same order as block_partials: a butterfly
// inside the warp, then the warps in order).
__device__ __forceinline__ void block_partials_r32(double v[4], uint32_t nacc, unsigned char *smem, int warp_bytes,
                                                   double *out, uint32_t *acc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double *mine = (double *)(smem + (size_t)warp * warp_bytes);
#pragma unroll
    for (int q = 0; q < 4; ++q) mine[lane * 4 + q] = v[q];
    ((uint32_t *)(mine + 32 * 4))[lane] = nacc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double a4[4] = {0.0, 0.0, 0.0, 0.0};
        uint32_t na = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            const double *o = (const double *)(smem + (size_t)w * warp_bytes);
#pragma unroll
            for (int q = 0; q < 4; ++q) a4[q] += o[threadIdx.x * 4 + q];
            na += ((const uint32_t *)(o + 32 * 4))[threadIdx.x];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) out[threadIdx.x * 4 + q] = a4[q];
        if (acc && na) atomicAdd(acc + threadIdx.x, na);
    }
}

__device__ __forceinline__ uint32_t atom_add_acq_rel(uint32_t *p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Renormalise class-0 block b (its sites x 32 replicas, lane = replica), four rows in flight.
__device__ __forceinline__ void renorm_block32(const PassArgs &a, float4 *S, int b, int lane) {
    const int g0 = a.fold_c0_begin + b * kFoldBlockSites;
    const int n = min(kFoldBlockSites, a.fold_c0_end - g0);
#pragma unroll
    for (int h = 0; h < kFoldBlockSites; h += 4) {
        float4 v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (h + k < n) v[k] = __ldcg(S + (int64_t)(g0 + h + k) * 32 + lane);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (h + k < n) S[(int64_t)(g0 + h + k) * 32 + lane] = renorm_spin32(v[k], __ldg(a.fold_norm + g0 + h + k));
    }
}

// RN = 1 (the step's last class-1 pass of a two-class sample, POL = 0): every attempt stores
// its spin renormalised, and once a block's eight groups are done the warp counts the block
// finished for each class-0 block it read (one per lane, an acquire-release add after the
// block's copies have landed); the warp whose add completes a class-0 block's count of readers
// renormalises that block. No class-1 block reads it afterwards in this pass and nothing else
// reads spins before the pass ends, so every spin is renormalised after its last use of the
// step: the same values as a renormalisation pass after the sweep.
template <int PM, int LM, int POL, int RN = 0>
__global__ void __launch_bounds__(R32Shape<POL>::WARPS * 32, R32Shape<POL>::MIN_BLOCKS) pass32_r32(const PassArgs a) {
    static_assert(RN == 0 || POL == 0, "the folded renormalisation runs without a policy table");
    using Sh = R32Shape<POL>;
    constexpr int DEG = Sh::DEG, D = Sh::D, BS = Sh::BS, R = 32;
    constexpr int ROWS = Sh::ROWS;
    constexpr int LINK_BYTES = Sh::LINK_BYTES;
    constexpr int POL_OFF = Sh::POL_OFF;
    constexpr int SLOT = Sh::SLOT;
    constexpr int WARP_BYTES = Sh::WARP_BYTES;
    static_assert(BS == kFoldBlockSites && kFoldDeps == 32, "the host's blocks of class sites; one per lane");
    extern __shared__ __align__(16) unsigned char smem[];
    const RunState *rs_ = a.run;
    const uint32_t t = rs_->t;
    const uint32_t step_idx = rs_->rec / rs_->mcs;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = lane;
    unsigned char *wbase = smem + warp * WARP_BYTES;
    float4 *rows = (float4 *)wbase;
    unsigned char *lslots = wbase + ROWS;
    float4 *S = (float4 *)a.spins;
    const float4 *Sr = S + r;
    const int2 *E = (const int2 *)a.edges;
    const uint32_t inst = (uint32_t)(a.inst0 + r);
    const double *sc = rs_->sched + ((int64_t)step_idx * a.n_inst + a.inst_local0 + r) * 2;
    const float beta = (float)sc[0], B = (float)sc[1];
    const float sigma = (POL && rs_->sigma) ? (float)rs_->sigma[a.inst_local0 + r] : 0.f;
    const int g_end = a.g_end;
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
    auto issue_links = [&](int sb, int slot) {
        if (sb >= g_end) return;
        const int ns = min(BS, g_end - sb);
        unsigned char *dst = lslots + slot * SLOT;
        const unsigned char *src = (const unsigned char *)(E + a.edge_base + (int64_t)(sb - a.site_off) * DEG);
        VEGAS_CHECK(sb >= a.g_begin && sb + ns <= a.n_sites_total, 11, sb);
        VEGAS_CHECK(a.edge_base + (int64_t)(sb - a.site_off + ns) * DEG <= a.n_edges_total, 12, sb);
        VEGAS_CHECK(((uintptr_t)src & 15) == 0, 13, sb);
        if (lane < ns * (DEG / 2)) cp16(dst + 16 * lane, src + 16 * lane);
        if (lane < ns) cp4(dst + LINK_BYTES + 4 * lane, a.orig + sb + lane);
        if (POL && lane < ns) cp8(dst + POL_OFF + 8 * lane, a.pol32 + sb + lane);
    };
    auto issue_rows = [&](int g, int lslot, int j, int rslot) {
        if (g >= g_end) return;
        const int4 *lk = (const int4 *)(lslots + lslot * SLOT) + j * (DEG / 2);
        float4 *dst = rows + rslot * (DEG + 1) * 32 + lane;
        VEGAS_CHECK(g < a.n_sites_total, 14, g);
#pragma unroll
        for (int q = 0; q < DEG / 2; ++q) {
            const int4 l = lk[q];
            VEGAS_CHECK(l.x >= 0 && l.x < a.n_sites_total && l.z >= 0 && l.z < a.n_sites_total, 15, l.x);
            cp16(dst + (2 * q) * 32, Sr + (int64_t)l.x * R);
            cp16(dst + (2 * q + 1) * 32, Sr + (int64_t)l.z * R);
        }
        cp16(dst + DEG * 32, Sr + (int64_t)g * R);
    };

    const uint32_t n_blocks = (uint32_t)(g_end - a.g_begin + BS - 1) / BS;  // a ticket past them ends the warp
    uint32_t tk = 0;
    if (lane == 0) tk = atomicAdd(a.ticket, 1u);
    int sb = a.g_begin + (int)min(__shfl_sync(0xFFFFFFFFu, tk, 0), n_blocks) * BS;
    issue_links(sb, 0);
    cp_commit();
    cp_wait<0>();
    __syncwarp();
    issue_rows(sb, 0, 0, 0);
    cp_commit();
    issue_rows(sb + 1, 0, 1, 1);
    cp_commit();
    Acc32 acc;
    bool nan_seen = false;
    const bool log_accepts = a.alog && t < a.alog_mcs;
    int ls = 0;
    while (sb < g_end) {
        int sb2 = g_end;  // the next block (drawn at j = 0, known from j = 4)
#pragma unroll
        for (int j = 0; j < BS; ++j) {
            cp_wait<D - 1>();
            __syncwarp();
            const int g = sb + j;
            if (g < g_end) {
                const unsigned char *slot = lslots + ls * SLOT;
                const uint32_t orig = ((const uint32_t *)(slot + LINK_BYTES))[j];
                staged_attempt<DEG, PM, LM, POL, RN != 0>(a, (const int4 *)slot + j * (DEG / 2),
                                                 rows + (j & 1) * (DEG + 1) * 32 + lane, orig, g, r, R, t, inst, rk0, rk1,
                                                 beta, B, S, acc, nan_seen, log_accepts,
                                                 (const PolicySite32 *)(slot + POL_OFF) + j, sigma);
            }
            __syncwarp();
            if (j == 0 && lane == 0) tk = atomicAdd(a.ticket, 1u);
            if (j == 4) {
                sb2 = a.g_begin + (int)min(__shfl_sync(0xFFFFFFFFu, tk, 0), n_blocks) * BS;
                issue_links(sb2, ls ^ 1);
            }
            if (j + 2 < BS)
                issue_rows(sb + j + 2, ls, j + 2, j & 1);
            else
                issue_rows(sb2 + j + 2 - BS, ls ^ 1, j + 2 - BS, j & 1);
            cp_commit();
        }
        if (RN) {
            const int dep = a.fold_deps[(int64_t)((sb - a.g_begin) / BS) * kFoldDeps + lane];
            __syncwarp();  // every lane's copies of this block have landed and been read
            const bool last = dep >= 0 && atom_add_acq_rel(a.fold_cnt + dep, 1u) + 1u == (uint32_t)__ldg(a.fold_deg + dep);
            for (uint32_t m = __ballot_sync(0xFFFFFFFFu, last); m; m &= m - 1)
                renorm_block32(a, S, __shfl_sync(0xFFFFFFFFu, dep, __ffs(m) - 1), lane);
        }
        sb = sb2;
        ls ^= 1;
    }
    cp_wait<0>();
    if (nan_seen) atomicOr(a.err, kErrNaN);
    acc.flush();
    __syncwarp();  // every lane's copies have landed and been read: the warp's area is free
    block_partials_r32(acc.d, acc.nacc, smem, WARP_BYTES, a.partial + (int64_t)blockIdx.x * R * 4,
                       acc_counters(rs_, a.inst_local0));
}

}  // namespace

// The R = 32 kernels specialised to one update policy (code 1 .. 6), built in their own
// translation unit.
PassFn select_r32_fixed(int pm, int lm, int code);
// The R = 32 kernel of the step's last class-1 pass with the renormalisation folded in
// (lower mode 1: every link of class 1 goes to class 0), in the same unit.
PassFn select_r32_renorm(int pm);

}  // namespace vegas
