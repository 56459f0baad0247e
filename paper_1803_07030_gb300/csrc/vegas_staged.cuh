// Pieces shared by the staged FP32 sweep kernels: cp.async copies into shared memory, one
// attempt computed from rows already staged there, and the index checks of debug builds.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "vegas_device.cuh"
#include "vegas_internal.h"

namespace vegas {
namespace {

__device__ __forceinline__ void cp16(void *smem, const void *gmem) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp4(void *smem, const void *gmem) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp8(void *smem, const void *gmem) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Philox4x32-10 block of one attempt (counter: caller id, MCS, instance, purpose) with the
// round keys precomputed in registers.
__device__ __forceinline__ uint4 trial_block32(uint32_t orig, uint32_t t, uint32_t inst, const uint32_t *rk0,
                                               const uint32_t *rk1) {
    uint4 c = make_uint4(orig, t, inst, kPurposeTrial32);
#pragma unroll
    for (int q = 0; q < 10; ++q) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ rk0[q], lo1, hi0 ^ c.w ^ rk1[q], lo0);
    }
    return c;
}

// One staged attempt with its random block c already drawn: links lk (int4 pairs), rows
// row[j*32] (neighbour j) and row[DEG*32] (own) in shared memory; with POL, the site's
// update policy *ps too (POL 1: the policy from the entry; POL 2 + c: every site has policy
// c). LM 3 takes the lower sums as all (lower_all) or none at run time. RN stores the spin
// after the attempt renormalised, accepted or not (the step's last pass over the site).
template <int DEG, int PM, int LM, int POL = 0, bool RN = false>
__device__ __forceinline__ void staged_attempt_rw(const PassArgs &a, const int4 *lk, const float4 *row, uint32_t orig,
                                                  int g, int r, int R, uint32_t t, uint4 c, float beta, float B,
                                                  float4 *S, Acc32 &acc, bool &nan_seen, bool log_accepts,
                                                  const PolicySite32 *ps = nullptr, float sigma = 0.f,
                                                  bool lower_all = true) {
    const Site32 p = site_params32(a, PM, g);
    float2 hxy = make_float2(0.f, 0.f), lxy = make_float2(0.f, 0.f);
    float hz = 0.f, lz = 0.f;
#pragma unroll
    for (int j = 0; j < DEG / 2; ++j) {
        const int4 q = lk[j];
        link32(row[(2 * j) * 32], __int_as_float(q.y), LM == 2 && q.x < a.lower_end, hxy, hz, lxy, lz);
        link32(row[(2 * j + 1) * 32], __int_as_float(q.w), LM == 2 && q.z < a.lower_end, hxy, hz, lxy, lz);
    }
    if (LM == 1 || (LM == 3 && lower_all)) {
        lxy = hxy;
        lz = hz;
    }
    const float4 Si = row[DEG * 32];
    float4 Sn;
    bool ok, bad;
    float e_i;
    const float3 P =
        POL ? policy_trial32<(POL >= 2 ? POL - 2 : -1)>(*ps, sigma, Si, p.sn, c) : trial_random32(c, p.sn);
    attempt32<PM, LM == 3 ? 1 : LM>(Si, hxy, hz, lxy, lz, p, beta, B, P, c.z, Sn, ok, e_i, bad);
    nan_seen |= bad;
    if (RN)
        S[(int64_t)g * R + r] = renorm_spin32(Sn, __ldg(a.fold_norm + g));
    else if (ok)
        S[(int64_t)g * R + r] = Sn;
    if (log_accepts)
        a.alog[(int64_t)t * a.alog_stride + a.alog_base + (int64_t)r * a.n_sample_sites + orig] = ok ? 1 : 0;
    acc.add(e_i, Sn, ok);
}

// The same, drawing the random block first.
template <int DEG, int PM, int LM, int POL = 0, bool RN = false>
__device__ __forceinline__ void staged_attempt(const PassArgs &a, const int4 *lk, const float4 *row, uint32_t orig,
                                               int g, int r, int R, uint32_t t, uint32_t inst, const uint32_t *rk0,
                                               const uint32_t *rk1, float beta, float B, float4 *S, Acc32 &acc,
                                               bool &nan_seen, bool log_accepts, const PolicySite32 *ps = nullptr,
                                               float sigma = 0.f) {
    staged_attempt_rw<DEG, PM, LM, POL, RN>(a, lk, row, orig, g, r, R, t, trial_block32(orig, t, inst, rk0, rk1), beta,
                                            B, S, acc, nan_seen, log_accepts, ps, sigma);
}

}  // namespace
}  // namespace vegas

// Debug builds (VEGAS_DEBUG_CHECKS) check every staged copy: a failed check sets
// kErrIndex, records a code and a value, and skips the access.
#ifdef VEGAS_DEBUG_CHECKS
#define VEGAS_CHECK(cond, code, val)                   \
    if (!(cond)) {                                     \
        atomicOr(a.err, kErrIndex);                    \
        atomicCAS(a.err + 1, 0u, (uint32_t)(code));    \
        a.err[2] = (uint32_t)(val);                    \
        return;                                        \
    }
#else
#define VEGAS_CHECK(cond, code, val)
#endif
