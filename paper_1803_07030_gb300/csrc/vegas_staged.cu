// Staged FP32 sweep kernels for rows of six links (simple cubic lattices): a cp.async pipeline
// in shared memory per warp, for any replica count (pass32_staged) and the replica-batched
// R = 32 case (pass32_r32), and the choice between them and the direct kernel.
#include <cuda_runtime.h>

#include <cstdint>

#include "vegas_device.cuh"
#include "vegas_internal.h"
#include "vegas_staged.cuh"
#include "vegas_r32.cuh"

namespace vegas {
namespace {

// ------------------------------------------------------------------ FP32 colour pass (staged)
// Rows of exactly DEG links. Each warp walks its share of the class in "groups" of 32
// work items (32/R sites x R replicas) and keeps a software pipeline in shared memory:
// the links and caller ids of group k+2D and the neighbour and own spin rows of group k+D
// are copied with cp.async while group k is computed, so DRAM latency overlaps compute
// instead of stalling the warp. Group k's rows are complete once all but the last D-1
// committed copy groups have landed (cp.async.wait_group D-1).

// Geometry of the staged kernel. A group is 32 work items (spg = 32/R sites x R replicas);
// a block is NB consecutive groups (BS = NB * spg >= 8 consecutive sites) whose links and
// caller ids are staged together. NLS block slots cover the 2D-group lookahead of links.
struct StagedGeom {
    int spg, BS, NB, NLS, link_bytes, slot_bytes, rows_bytes, warp_bytes;
};

__host__ __device__ inline StagedGeom staged_geom(int deg, int D, int log2R) {
    StagedGeom g;
    g.spg = 32 >> log2R;
    g.BS = g.spg > 8 ? g.spg : 8;
    g.NB = g.BS / g.spg;
    g.NLS = (2 * D + g.NB - 1) / g.NB + 1;
    g.link_bytes = ((g.BS * deg * 8 + 15) / 16) * 16;
    g.slot_bytes = g.link_bytes + ((g.BS * 4 + 15) / 16) * 16;
    g.rows_bytes = D * (deg + 1) * 32 * 16;
    g.warp_bytes = g.rows_bytes + g.NLS * g.slot_bytes;
    return g;
}

// Position of one group in the warp's sequence: first site, index inside its block, and
// the slot holding its block's links. Groups are visited in increasing site order.
struct GroupPos {
    int sbase, j, lslot;
    __device__ __forceinline__ void next(const StagedGeom &G, int bstride) {
        if (++j == G.NB) {
            j = 0;
            sbase += bstride - (G.NB - 1) * G.spg;
            lslot = (lslot + 1 == G.NLS) ? 0 : lslot + 1;
        } else {
            sbase += G.spg;
        }
    }
};

// LOG2R >= 0 fixes the replica count at compile time (the batched case R = 32); -1 reads it
// from the arguments.
// Depth 2 fits three blocks per SM in shared memory; the register cap keeps them resident.
template <int DEG, int PM, int LM, int D, int LOG2R>
__global__ void __launch_bounds__(kThreads, D == 2 ? 3 : 2) pass32_staged(const PassArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const RunState *rs_ = a.run;
    const uint32_t t = rs_->t;
    const uint32_t step_idx = rs_->rec / rs_->mcs;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int log2R = LOG2R >= 0 ? LOG2R : a.log2R, R = 1 << log2R;
    const StagedGeom G = staged_geom(DEG, D, log2R);
    const int r = lane & (R - 1), my = lane >> log2R;  // replica, site within the group
    unsigned char *wbase = smem + (size_t)warp * G.warp_bytes;
    float4 *rows = (float4 *)wbase;                     // [D][DEG+1][32]
    unsigned char *lslots = wbase + G.rows_bytes;       // [NLS][links | caller ids]
    float4 *S = (float4 *)a.spins;
    const float4 *Sr = S + r;
    const int2 *E = (const int2 *)a.edges;
    const uint32_t inst = (uint32_t)(a.inst0 + r);
    const double *sc = rs_->sched + ((int64_t)step_idx * a.n_inst + a.inst_local0 + r) * 2;
    const float beta = (float)sc[0], B = (float)sc[1];
    const int g_end = a.g_end;
    const int nwarps = blockDim.x >> 5;
    const int W = blockIdx.x * nwarps + warp;
    const int bstride = gridDim.x * nwarps * G.BS;  // sites between this warp's blocks
    uint32_t rk0[10], rk1[10];                      // Philox round keys, kept in registers
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

    auto issue_links = [&](int sb, int slot) {  // links and caller ids of the block at sb
        if (sb >= g_end) return;
        const int ns = min(G.BS, g_end - sb);
        unsigned char *dst = lslots + slot * G.slot_bytes;
        const unsigned char *src = (const unsigned char *)(E + a.edge_base + (int64_t)(sb - a.site_off) * DEG);
        const int nch = ns * (DEG / 2);
        VEGAS_CHECK(sb >= a.g_begin && slot >= 0 && slot < G.NLS, 1, sb);
        VEGAS_CHECK(a.edge_base + (int64_t)(sb - a.site_off) * DEG + (int64_t)ns * DEG <= a.n_edges_total, 2, sb);
        VEGAS_CHECK(((uintptr_t)src & 15) == 0 && ((uintptr_t)dst & 15) == 0, 3, sb);
        VEGAS_CHECK(sb + ns <= a.n_sites_total, 4, sb);
        for (int c = lane; c < nch; c += 32) cp16(dst + 16 * c, src + 16 * c);
        if (lane < ns) cp4(dst + G.link_bytes + 4 * lane, a.orig + sb + lane);
    };
    auto issue_rows = [&](const GroupPos &p, int rslot) {  // rows of a group (its links have landed)
        const int g = p.sbase + my;
        if (g >= g_end) return;
        const int4 *lk = (const int4 *)(lslots + p.lslot * G.slot_bytes) + (p.j * G.spg + my) * (DEG / 2);
        float4 *dst = rows + rslot * (DEG + 1) * 32 + lane;
        VEGAS_CHECK(p.lslot >= 0 && p.lslot < G.NLS && rslot >= 0 && rslot < D, 5, p.lslot * 16 + rslot);
        VEGAS_CHECK(g < a.n_sites_total, 6, g);
#pragma unroll
        for (int j = 0; j < DEG / 2; ++j) {
            const int4 q = lk[j];
            VEGAS_CHECK(q.x >= 0 && q.x < a.n_sites_total && q.z >= 0 && q.z < a.n_sites_total, 7, q.x);
            cp16(dst + (2 * j) * 32, Sr + (int64_t)q.x * R);
            cp16(dst + (2 * j + 1) * 32, Sr + (int64_t)q.z * R);
        }
        cp16(dst + DEG * 32, Sr + (int64_t)g * R);
    };

    // prologue: links of every block whose first group is among the first 2D, then the
    // rows of the first D groups
    const int g0 = a.g_begin + W * G.BS;
    const int nb_pro = (2 * D + G.NB - 1) / G.NB;
    for (int b = 0; b < nb_pro; ++b) issue_links(g0 + b * bstride, b);
    cp_commit();
    cp_wait<0>();
    __syncwarp();
    GroupPos pk{g0, 0, 0};  // group k (computed now)
    GroupPos pd = pk;       // group k + D (rows issued at the end of this iteration)
    for (int q = 0; q < D; ++q) {
        issue_rows(pd, q);
        cp_commit();
        pd.next(G, bstride);
    }
    int k_issue = nb_pro * G.NB - 2 * D;  // iteration whose end issues the next block's links
    int sb_next = g0 + nb_pro * bstride, ls_next = nb_pro;
    int rsl = 0;
    Acc32 acc;
    bool nan_seen = false;
    const bool log_accepts = a.alog && t < a.alog_mcs;
    for (int k = 0; pk.sbase < g_end; ++k) {
        cp_wait<D - 1>();
        __syncwarp();
        const int g = pk.sbase + my;
        if (g < g_end) {
            const unsigned char *slot = lslots + pk.lslot * G.slot_bytes;
            const int li = pk.j * G.spg + my;
            const int4 *lk = (const int4 *)slot + li * (DEG / 2);
            const float4 *row = rows + rsl * (DEG + 1) * 32 + lane;
            const uint32_t orig = ((const uint32_t *)(slot + G.link_bytes))[li];
            bool skip = false;
#ifdef VEGAS_DEBUG_CHECKS
            if (orig >= (uint32_t)a.n_sample_sites || g >= a.n_sites_total) {
                atomicOr(a.err, kErrIndex);
                atomicCAS(a.err + 1, 0u, 8u);
                a.err[2] = orig;
                skip = true;
            }
#endif
            if (!skip) staged_attempt<DEG, PM, LM>(a, lk, row, orig, g, r, R, t, inst, rk0, rk1, beta, B, S, acc, nan_seen,
                                              log_accepts);
        }
        __syncwarp();
        if (k == k_issue) {
            issue_links(sb_next, ls_next);
            k_issue += G.NB;
            sb_next += bstride;
            ls_next = (ls_next + 1 == G.NLS) ? 0 : ls_next + 1;
        }
        issue_rows(pd, rsl);
        cp_commit();
        pk.next(G, bstride);
        pd.next(G, bstride);
        rsl = (rsl + 1 == D) ? 0 : rsl + 1;
    }
    cp_wait<0>();
    if (nan_seen) atomicOr(a.err, kErrNaN);
    acc.flush();
    block_partials(acc.d, acc.nacc, R, a.partial + (int64_t)blockIdx.x * R * 4, acc_counters(rs_, a.inst_local0));
}

// ------------------------------------------------------------------ variant table
template <int D>
PassFn select_staged6(int pm, int lm) {
    static const PassFn tab[3][3] = {
        {pass32_staged<6, 0, 0, D, -1>, pass32_staged<6, 0, 1, D, -1>, pass32_staged<6, 0, 2, D, -1>},
        {pass32_staged<6, 1, 0, D, -1>, pass32_staged<6, 1, 1, D, -1>, pass32_staged<6, 1, 2, D, -1>},
        {pass32_staged<6, 2, 0, D, -1>, pass32_staged<6, 2, 1, D, -1>, pass32_staged<6, 2, 2, D, -1>},
    };
    return tab[pm][lm];
}

PassFn select_r32_table(int pm, int lm, bool pol) {
    static const PassFn tab[2][3][3] = {
        {
            {pass32_r32<0, 0, 0>, pass32_r32<0, 1, 0>, pass32_r32<0, 2, 0>},
            {pass32_r32<1, 0, 0>, pass32_r32<1, 1, 0>, pass32_r32<1, 2, 0>},
            {pass32_r32<2, 0, 0>, pass32_r32<2, 1, 0>, pass32_r32<2, 2, 0>},
        },
        {
            {pass32_r32<0, 0, 1>, pass32_r32<0, 1, 1>, pass32_r32<0, 2, 1>},
            {pass32_r32<1, 0, 1>, pass32_r32<1, 1, 1>, pass32_r32<1, 2, 1>},
            {pass32_r32<2, 0, 1>, pass32_r32<2, 1, 1>, pass32_r32<2, 2, 1>},
        },
    };
    return tab[pol ? 1 : 0][pm][lm];
}

// R = 32 kernel of a pass: with a policy table, specialised to the one policy of the class
// when it has one (random: the kernel without a table, which draws the same trial).
PassFn select_r32(const PassArgs &a) {
    if (a.fold_deps) return select_r32_renorm(a.params_mode);
    if (a.pol32 && a.pol_fixed == kPolRandom) return select_r32_table(a.params_mode, a.lower_mode, false);
    if (a.pol32 && a.pol_fixed > kPolRandom) return select_r32_fixed(a.params_mode, a.lower_mode, a.pol_fixed);
    return select_r32_table(a.params_mode, a.lower_mode, a.pol32 != nullptr);
}

bool staged_shape(const PassArgs &a) { return a.deg == 6 && a.depth >= 2; }
bool use_r32(const PassArgs &a) { return staged_shape(a) && a.log2R == 5 && a.depth == 2; }
// Samples with a policy table take the staged path only through the R = 32 kernel.
bool use_staged(const PassArgs &a) { return staged_shape(a) && (!a.pol32 || use_r32(a)); }

int staged_smem(const PassArgs &a) {
    if (use_r32(a)) {
        const bool table = a.pol32 && a.pol_fixed != kPolRandom;  // policy entries staged with the links
        return table ? R32Shape<1>::WARPS * R32Shape<1>::WARP_BYTES : R32Shape<0>::WARPS * R32Shape<0>::WARP_BYTES;
    }
    return (kThreads / 32) * staged_geom(6, a.depth, a.log2R).warp_bytes;
}

PassFn select_staged(const PassArgs &a) {
    if (use_r32(a)) return select_r32(a);
    return a.depth == 2 ? select_staged6<2>(a.params_mode, a.lower_mode) : select_staged6<3>(a.params_mode, a.lower_mode);
}

}  // namespace

PassFn select_pass32(const PassArgs &a) {
    return use_staged(a) ? select_staged(a) : select_direct(a.params_mode, a.lower_mode, a.pol32 != nullptr);
}

int pass32_smem(const PassArgs &a) { return use_staged(a) ? staged_smem(a) : 0; }

bool pass32_direct(const PassArgs &a) { return !use_staged(a); }

int pass32_threads(const PassArgs &a) {
    if (!use_r32(a)) return kThreads;
    const bool table = a.pol32 && a.pol_fixed != kPolRandom;
    return 32 * (table ? R32Shape<1>::WARPS : R32Shape<0>::WARPS);
}

uint32_t pass32_kind(const PassArgs &a) {
    if (!use_staged(a)) return VEGAS_KERNEL_PASS32_DIRECT;
    if (use_r32(a)) {
        if (a.fold_deps) return VEGAS_KERNEL_PASS32_R32_RENORM;
        if (!a.pol32 || a.pol_fixed == kPolRandom) return VEGAS_KERNEL_PASS32_R32;
        return a.pol_fixed > kPolRandom ? VEGAS_KERNEL_PASS32_R32_ONE_POLICY : VEGAS_KERNEL_PASS32_R32_POLICY;
    }
    return VEGAS_KERNEL_PASS32_STAGED;
}

}  // namespace vegas
