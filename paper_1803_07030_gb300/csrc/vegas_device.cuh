// Device helpers shared by the sweep kernels (the FP32 attempt and its trials, Philox,
// the block partials). Included by vegas_kernels.cu and vegas_staged.cu; everything here has
// internal linkage in each translation unit.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "vegas_internal.h"

namespace vegas {
namespace {

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11:
// ten rounds of two 32x32->64 multiplies (M0 = 0xD2511F53, M1 = 0xCD9E8D57) with the key
// bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85) between rounds.
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ float cub32(float x, float y, float z) {
    const float xx = x * x, yy = y * y, zz = z * z;
    return fmaf(xx, yy, fmaf(yy, zz, xx * zz));
}

// ------------------------------------------------------------------ block partials
// Per-block sums of (E, Mx, My, Mz) for each replica. Lanes whose index agrees modulo R
// hold the same replica; a fixed butterfly and a fixed warp order make the result
// deterministic. out points at this block's [R][4] slot. The accepted attempts of the block
// are added to acc[replica] (integers: the order does not matter), when acc is not NULL.
__device__ __forceinline__ void block_partials(double v[4], uint32_t nacc, int R, double *out, uint32_t *acc) {
    __shared__ double sm[kThreads / 32][32][4];
    __shared__ uint32_t sn[kThreads / 32][32];
    for (int off = 16; off >= R; off >>= 1) {
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] += __shfl_xor_sync(0xFFFFFFFFu, v[q], off);
        nacc += __shfl_xor_sync(0xFFFFFFFFu, nacc, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane < R) {
#pragma unroll
        for (int q = 0; q < 4; ++q) sm[warp][lane][q] = v[q];
        sn[warp][lane] = nacc;
    }
    __syncthreads();
    if ((int)threadIdx.x < R) {
        double a4[4] = {0.0, 0.0, 0.0, 0.0};
        uint32_t na = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
#pragma unroll
            for (int q = 0; q < 4; ++q) a4[q] += sm[w][threadIdx.x][q];
            na += sn[w][threadIdx.x];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) out[threadIdx.x * 4 + q] = a4[q];
        if (acc && na) atomicAdd(acc + threadIdx.x, na);
    }
}

// Accepted-attempt counters of replica 0 of a pass's sample (NULL when not counted).
__device__ __forceinline__ uint32_t *acc_counters(const RunState *rs, int inst_local0) {
    return rs->acc ? rs->acc + inst_local0 : nullptr;
}

// ------------------------------------------------------------------ FP32 attempt
// One Metropolis attempt in FP32, written with explicit roundings (fmaf where a fused
// multiply-add is meant, __fmul_rn / __fadd_rn elsewhere) so that every kernel that calls
// it computes bit-identical results for the same inputs, whatever the surrounding code.
// h is the exchange field sum_j J_ij S_j (row order), l its part over lower colours.
struct Site32 {
    float nx, ny, nz, sn, ex, ey, ez, k, kc;
};

// Random trial (Sec. III.B): z uniform in (-1, 1), azimuth uniform in (-pi, pi): by
// Archimedes' theorem (sqrt(1-z^2) cos phi, sqrt(1-z^2) sin phi, z) is uniform on the sphere.
// Each uniform takes 23 random bits as the mantissa of a float in [1, 2): f = 1 + k 2^-23,
// so z = 2 (f - 1.5) + 2^-23 = (2k + 1) 2^-23 - 1 exactly (midpoints of 2^23 cells).
__device__ __forceinline__ float3 trial_random32(uint4 rw, float sn) {
    const float fz = __uint_as_float(0x3F800000u | (rw.x >> 9));
    const float fp = __uint_as_float(0x3F800000u | (rw.y >> 9));
    const float z = fmaf(__fsub_rn(fz, 1.5f), 2.0f, 0x1p-23f);
    const float phi = fmaf(__fsub_rn(fp, 1.5f), 6.28318530717959f, 3.14159265358979f * 0x1p-23f);
    float sphi, cphi;
    __sincosf(phi, &sphi, &cphi);
    const float rho2 = fmaf(-z, z, 1.0f);
    const float rho = __fmul_rn(rho2, rsqrtf(rho2));
    // x and y in packed pairs (each lane of a pair rounds as the scalar operation does)
    const float2 xy = __fmul2_rn(make_float2(sn, sn), __fmul2_rn(make_float2(rho, rho), make_float2(cphi, sphi)));
    return make_float3(xy.x, xy.y, __fmul_rn(sn, z));
}

// One Metropolis attempt in FP32 on the trial P, written with explicit roundings (fmaf
// where a fused multiply-add is meant, __fmul_rn / __fadd_rn elsewhere) so that every
// kernel that calls it computes bit-identical results for the same inputs, whatever the
// surrounding code. h is the exchange field sum_j J_ij S_j (row order), l its part over
// lower colours (x and y of each as a packed pair: the packed FP32 instructions of sm_100+
// round each lane as the scalar operation does, so the results are the same bits); wacc is
// the random word of the acceptance uniform.
template <int PM, int LM>
__device__ __forceinline__ void attempt32(const float4 Si, float2 hxy, float hz, float2 lxy, float lz,
                                          const Site32 &p, float beta, float B, const float3 P, uint32_t wacc,
                                          float4 &Sn, bool &acc, float &e_i, bool &nan_seen) {
    const float2 Hxy = __ffma2_rn(make_float2(B, B), make_float2(p.nx, p.ny), hxy);
    const float Hz = fmaf(B, p.nz, hz);
    const float Hx = Hxy.x, Hy = Hxy.y, lx = lxy.x, ly = lxy.y;
    const float px = P.x, py = P.y, pz = P.z;
    // P - S as P + (-S): the same rounding
    const float2 dxy = __fadd2_rn(make_float2(px, py), make_float2(-Si.x, -Si.y));
    const float dx = dxy.x, dy = dxy.y, dz = __fsub_rn(pz, Si.z);
    float dE = -fmaf(dx, Hx, fmaf(dy, Hy, __fmul_rn(dz, Hz)));
    if (PM != 0) {
        const float pn = fmaf(px, p.ex, fmaf(py, p.ey, __fmul_rn(pz, p.ez)));
        const float po = fmaf(Si.x, p.ex, fmaf(Si.y, p.ey, __fmul_rn(Si.z, p.ez)));
        dE = fmaf(-p.k, __fmul_rn(__fsub_rn(pn, po), __fadd_rn(pn, po)), dE);
        dE = fmaf(-p.kc, __fsub_rn(cub32(px, py, pz), cub32(Si.x, Si.y, Si.z)), dE);
    }
    // Metropolis acceptance (Eq. 4) with the uniform u = wacc 2^-32 (all 32 random bits):
    // u < p  <=>  wacc < p 2^32, so the test is wacc < floor(p 2^32) (p 2^32 is exact in FP32,
    // the conversion truncates) and P(accept) = floor(p 2^32) 2^-32 lies in (p - 2^-32, p].
    // p >= 1 accepts outright (floor(2^32) does not fit 32 bits). NaN rejects.
    const float pacc = __expf(__fmul_rn(-beta, dE));
    acc = (dE <= 0.f) || (pacc >= 1.0f) || (wacc < __float2uint_rz(__fmul_rn(pacc, 0x1p32f)));
    nan_seen = (dE != dE);
    if (nan_seen) acc = false;
    const float qx = acc ? px : Si.x, qy = acc ? py : Si.y, qz = acc ? pz : Si.z;
    Sn = make_float4(qx, qy, qz, 0.f);
    // this site's share of the energy after the MCS: -S.l - B S.n - k (S.e)^2 - kc cub(S)
    float e = __fmul_rn(-B, fmaf(qx, p.nx, fmaf(qy, p.ny, __fmul_rn(qz, p.nz))));
    if (LM != 0) e = __fsub_rn(e, fmaf(qx, lx, fmaf(qy, ly, __fmul_rn(qz, lz))));
    if (PM != 0) {
        const float pe = fmaf(qx, p.ex, fmaf(qy, p.ey, __fmul_rn(qz, p.ez)));
        e = __fsub_rn(e, fmaf(__fmul_rn(p.k, pe), pe, __fmul_rn(p.kc, cub32(qx, qy, qz))));
    }
    e_i = e;
}

// ------------------------------------------------------------------ FP32 update policies
// The same proposals as the FP64 path, drawn from the attempt's one Philox block: words x and
// y are the two uniforms, z the acceptance uniform, w the Hinzke-Nowak choice or, for the
// Gaussian, the third normal (inverse error function of a 23-bit uniform; the first two
// come from Box-Muller on x and y).
__device__ __forceinline__ float u23(uint32_t w) {  // k 2^-23 in [0, 1)
    return __fsub_rn(__uint_as_float(0x3F800000u | (w >> 9)), 1.0f);
}

__device__ __forceinline__ float3 unit32(float x, float y, float z) {
    const float q = rsqrtf(fmaf(x, x, fmaf(y, y, __fmul_rn(z, z))));
    return make_float3(__fmul_rn(x, q), __fmul_rn(y, q), __fmul_rn(z, q));
}

constexpr int kPolCapSphere = 6;  // internal: the random third of Hinzke-Nowak, as a cap of height 2

// PC >= 0: every site of the pass has policy PC (the kernel is specialised: the other
// policies' code is not compiled in); -1: the policy of each site from its table entry.
template <int PC = -1>
__device__ __forceinline__ float3 policy_trial32(const PolicySite32 ps, float sigma, const float4 Si, float sn,
                                                 uint4 rw) {
    int code = PC >= 0 ? PC : ps.code;
    if (code == kPolQIsing) {  // another of the 2 s + 1 values along z, uniformly
        const int n2 = (int)(2.0f * sn);
        const int idx = (int)(Si.z + sn + 0.5f);
        int k = min((int)(u23(rw.x) * (float)n2), n2 - 1);
        if (k >= idx) k += 1;
        return make_float3(0.f, 0.f, (float)k - sn);
    }
    if (code == kPolHinzkeNowak) {
        // a uniform point on the sphere is the cap of height 2 around any axis, so the random
        // and small-step thirds share one code path (no divergence between them in a warp)
        const float v = __fmul_rn(u23(rw.w), 3.0f);
        code = v < 1.0f ? kPolFlip : (v < 2.0f ? kPolCapSphere : kPolSmallStep);
    }
    if (code == kPolFlip) return make_float3(-Si.x, -Si.y, -Si.z);
    if (code == kPolRandom) return trial_random32(rw, sn);
    const float3 u = unit32(Si.x, Si.y, Si.z);
    float sphi, cphi;
    const float phi = fmaf(__fsub_rn(__uint_as_float(0x3F800000u | (rw.y >> 9)), 1.5f), 6.28318530717959f,
                           3.14159265358979f * 0x1p-23f);
    __sincosf(phi, &sphi, &cphi);
    if (code == kPolSmallStep || code == kPolCapSphere) {  // uniform in the cap of height h around u
        const float h = code == kPolCapSphere ? 2.0f : ps.par;
        const float sh = __fmul_rn(u23(rw.x), h);
        const float z = __fsub_rn(1.0f, sh);
        const float r = sqrtf(fmaxf(__fmul_rn(sh, __fsub_rn(2.0f, sh)), 0.0f));
        // orthonormal frame (e1, e2, u) without branches (Duff, Burgess, Christensen, Hery,
        // Kensler, Liani, Villemin, "Building an orthonormal basis, revisited", JCGT 6(1),
        // 2017): with s = sign(u_z) and a = -1 / (s + u_z), e1 = (1 + s a u_x^2, s a u_x u_y,
        // -s u_x), e2 = (a u_x u_y, s + a u_y^2, -u_y); |s + u_z| >= 1, so nothing diverges
        // between the lanes of a warp. The azimuth is uniform, so the frame's orientation
        // about u does not change the law of the trial.
        const float sgn = copysignf(1.0f, u.z);
        const float am = __fdividef(-1.0f, __fadd_rn(sgn, u.z));
        const float b = __fmul_rn(__fmul_rn(u.x, u.y), am);
        const float3 e1 = make_float3(fmaf(__fmul_rn(sgn, __fmul_rn(u.x, u.x)), am, 1.0f), __fmul_rn(sgn, b),
                                      -__fmul_rn(sgn, u.x));
        const float3 e2 = make_float3(b, fmaf(__fmul_rn(u.y, u.y), am, sgn), -u.y);
        const float x = __fmul_rn(r, cphi), y = __fmul_rn(r, sphi);
        return make_float3(__fmul_rn(sn, fmaf(x, e1.x, fmaf(y, e2.x, __fmul_rn(z, u.x)))),
                           __fmul_rn(sn, fmaf(x, e1.y, fmaf(y, e2.y, __fmul_rn(z, u.y)))),
                           __fmul_rn(sn, fmaf(x, e1.z, fmaf(y, e2.z, __fmul_rn(z, u.z)))));
    }
    // Gaussian (fixed width) or adaptive (the instance's width): direction of u + sigma g
    const float sg = code == kPolAdaptive ? sigma : ps.par;
    const float rad = sqrtf(__fmul_rn(-2.0f, __logf(__fsub_rn(1.0f, u23(rw.x)))));  // 1 - u in (0, 1]
    // (2k + 1) 2^-23 - 1 lies strictly inside (-1, 1); sqrt 2 erfinv of it is standard normal
    const float g2 = __fmul_rn(1.41421356237310f, erfinvf(fmaf(u23(rw.w), 2.0f, -1.0f + 0x1p-23f)));
    const float3 v = unit32(fmaf(sg, __fmul_rn(rad, cphi), u.x), fmaf(sg, __fmul_rn(rad, sphi), u.y), fmaf(sg, g2, u.z));
    return make_float3(__fmul_rn(sn, v.x), __fmul_rn(sn, v.y), __fmul_rn(sn, v.z));
}

// Per-thread sums of E and M: runs of at most 64 attempts in FP32, then FP64 (a run's
// rounding error is below 64 * 2^-24 of its absolute sum, < 1e-5 of E/N).
// Also counts the accepted attempts.
struct Acc32 {
    double d[4] = {0.0, 0.0, 0.0, 0.0};
    float2 fem = make_float2(0.f, 0.f);  // E and Mz
    float2 fxy = make_float2(0.f, 0.f);  // Mx and My
    int n = 0;
    uint32_t nacc = 0;
    __device__ __forceinline__ void add(float e, float4 q, bool ok) {
        nacc += ok ? 1u : 0u;
        fem = __fadd2_rn(fem, make_float2(e, q.z));
        fxy = __fadd2_rn(fxy, make_float2(q.x, q.y));
        if (++n == 64) flush();
    }

    __device__ __forceinline__ void flush() {
        d[0] += (double)fem.x;
        d[1] += (double)fxy.x;
        d[2] += (double)fxy.y;
        d[3] += (double)fem.y;
        fem = make_float2(0.f, 0.f);
        fxy = make_float2(0.f, 0.f);
        n = 0;
    }
};

// One link's share of the field: x and y as a packed pair (one instruction, the same two
// roundings), z alone; with `lower`, also of the part over lower colours.
__device__ __forceinline__ void link32(const float4 Sj, float J, bool lower, float2 &hxy, float &hz, float2 &lxy,
                                       float &lz) {
    const float2 jj = make_float2(J, J), sxy = make_float2(Sj.x, Sj.y);
    hxy = __ffma2_rn(jj, sxy, hxy);
    hz = fmaf(J, Sj.z, hz);
    if (lower) {
        lxy = __ffma2_rn(jj, sxy, lxy);
        lz = fmaf(J, Sj.z, lz);
    }
}

__device__ __forceinline__ Site32 site_params32(const PassArgs &a, int PMv, int g) {
    Site32 p{a.u32.nx, a.u32.ny, a.u32.nz, a.u32.s, a.u32.ex, a.u32.ey, a.u32.ez, a.u32.k, a.u32.kc};
    if (PMv == 2) {
        const float4 p0 = __ldg((const float4 *)a.p0 + g), p1 = __ldg((const float4 *)a.p1 + g);
        p = Site32{p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w, __ldg((const float *)a.pk + g)};
    }
    return p;
}

// ------------------------------------------------------------------ FP32 renormalisation
// u = |S|^2 - 1 of a float spin with no FP64 operation (GB300 runs two of those per SM and
// clock): each square split into its rounded value and its exact rounding error (Dekker's
// product, the error from one FMA), the rounded squares summed with Knuth's TwoSum (both
// parts exact), 1 taken off exactly (Sterbenz: the sum lies in [1/2, 2] whenever |u| <= 1/2)
// and the five error terms added in. The tail's own roundings stay below 2^-44, so for |u|
// <= 1/2 the result is u + delta, |delta| < 2^-44, rounded once to a float; further out it
// is only a rough value. The _rn intrinsics keep the products out of the sums.
__device__ __forceinline__ float norm2_minus1_f32(float x, float y, float z) {
    const float px = __fmul_rn(x, x), py = __fmul_rn(y, y), pz = __fmul_rn(z, z);
    const float ex = fmaf(x, x, -px), ey = fmaf(y, y, -py), ez = fmaf(z, z, -pz);
    const float s1 = __fadd_rn(px, py), b1 = __fsub_rn(s1, px);
    const float t1 = __fadd_rn(__fsub_rn(px, __fsub_rn(s1, b1)), __fsub_rn(py, b1));
    const float s2 = __fadd_rn(s1, pz), b2 = __fsub_rn(s2, s1);
    const float t2 = __fadd_rn(__fsub_rn(s1, __fsub_rn(s2, b2)), __fsub_rn(pz, b2));
    const float tail = __fadd_rn(__fadd_rn(t1, t2), __fadd_rn(__fadd_rn(ex, ey), ez));
    return __fadd_rn(__fsub_rn(s2, 1.0f), tail);
}

// The FP64 formula s / sqrt(1 + u), u from three FP64 FMAs; not inlined, so that the rare
// call costs the callers' common path no registers.
__device__ __noinline__ float4 renorm_spin32_fp64(const float4 v, double s) {
    const double x = v.x, y = v.y, z = v.z;
    const double f = s / sqrt(fma(x, x, fma(y, y, fma(z, z, -1.0))) + 1.0);
    return make_float4((float)(x * f), (float)(y * f), (float)(z * f), 0.f);
}

// S <- s S / |S| for one float spin. For s = 1 (tested on its bits) and |u| < 2^-16, u = |S|^2
// - 1 (every spin a Metropolis step leaves has |u| ~ 1e-7): S + S d with d = -u/2 + 3u^2/8,
// the first terms of (1 + u)^(-1/2) - 1, in one FMA per component and no FP64 operation;
// otherwise the FP64 formula.
__device__ __forceinline__ float4 renorm_spin32(const float4 v, double s) {
    const float uf = norm2_minus1_f32(v.x, v.y, v.z);
    if (__double_as_longlong(s) == 0x3FF0000000000000LL && fabsf(uf) < 0x1p-16f) {
        const float d = __fmul_rn(uf, fmaf(0.375f, uf, -0.5f));
        return make_float4(fmaf(v.x, d, v.x), fmaf(v.y, d, v.y), fmaf(v.z, d, v.z), 0.f);
    }
    return renorm_spin32_fp64(v, s);
}

}  // namespace
}  // namespace vegas
