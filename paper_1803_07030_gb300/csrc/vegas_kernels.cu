// Device kernels of the Metropolis sweep (Sec. III.B, Eq. 4) on the Heisenberg
// Hamiltonian (Sec. III.A, Eq. 1-3), for sm_103a.
//
// Layout in HBM: spins are [global site][replica] (float4 or double4_32a; w unused), so the R
// replicas of one site sit next to each other; sites are numbered colour-major per sample,
// samples packed one after the other. A warp of 32 threads covers 32/R sites x R
// replicas: with R = 32 one warp is one site, its neighbour rows are contiguous 512-byte
// lines and each link (col, J) is one broadcast load shared by the replicas.
//
// One launch sweeps one colour class: no site of the class links to another, so every
// thread updates its site from neighbours that this launch never writes. While it
// gathers the local field, a thread also sums the links to lower colours; those
// neighbours are already final for this MCS, so -S_i.h_i(lower) - B S_i.n_i - anisotropy
// summed over all sites is the exact energy after the MCS (each bond is counted once, at
// its higher-coloured end) without a second pass over the links.
//
// The FP64 kernel evaluates every step exactly as the CPU oracle does (no FMA, the same
// operation order, Marsaglia sampler, correctly rounded sqrt and divide), so its spins and
// accept decisions match the oracle bit for bit. The FP32 kernels draw one Philox block per
// attempt (uniform z and azimuth, the acceptance uniform) and use FMA.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "vegas_device.cuh"
#include "vegas_internal.h"

namespace vegas {
namespace {

// ------------------------------------------------------------------ FP64 helpers
// Explicit round-to-nearest operations: the compiler may not fuse them, which keeps the
// FP64 path identical to the CPU oracle built without contraction.
__device__ __forceinline__ double dm(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double da(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double ds(double a, double b) { return __dsub_rn(a, b); }

// Uniform in [0, 1) with 53 bits: (hi * 2^21 + (lo >> 11)) * 2^-53 (exact).
__device__ __forceinline__ double u53(uint32_t hi, uint32_t lo) {
    const unsigned long long m = ((unsigned long long)hi << 21) | (unsigned long long)(lo >> 11);
    return __dmul_rn(__ull2double_rn(m), 0x1p-53);
}

// Point on the unit sphere by Marsaglia's method (Ann. Math. Stat. 43, 1972): draw
// (u1, u2) uniform in the square [-1, 1)^2 until s = u1^2 + u2^2 < 1, then
// (2 u1 sqrt(1-s), 2 u2 sqrt(1-s), 1 - 2 s). Candidate k uses counter word 3 = purpose|k.
__device__ double3 sphere64(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t purpose, uint32_t k0, uint32_t k1,
                            uint32_t *err) {
    for (uint32_t k = 0; k < 64; ++k) {
        const uint4 w = philox10(make_uint4(c0, c1, c2, purpose | k), k0, k1);
        const double u1 = ds(dm(2.0, u53(w.x, w.y)), 1.0);
        const double u2 = ds(dm(2.0, u53(w.z, w.w)), 1.0);
        const double s = da(dm(u1, u1), dm(u2, u2));
        if (s >= 1.0) continue;
        const double q = __dsqrt_rn(ds(1.0, s));
        return make_double3(dm(dm(2.0, u1), q), dm(dm(2.0, u2), q), ds(1.0, dm(2.0, s)));
    }
    atomicOr(err, kErrSphere);
    return make_double3(0.0, 0.0, 1.0);
}

__device__ __forceinline__ double cub64(double x, double y, double z) {
    const double xx = dm(x, x), yy = dm(y, y), zz = dm(z, z);
    return da(da(dm(xx, yy), dm(yy, zz)), dm(xx, zz));
}

// ------------------------------------------------------------------ FP64 update policies
// Trial generators of the policies other than "random" (Sec. II), evaluated with the same
// operations in the same order as the CPU oracle, so that the FP64 path stays bit-exact.

// ln x for a normal x > 0: x = m 2^e with m in [sqrt(1/2), sqrt 2), ln m = 2 atanh t for
// t = (m - 1)/(m + 1), atanh t = sum_j t^(2j+1)/(2j+1) up to j = 13 (Abramowitz & Stegun
// 4.1.27; |t| <= 0.172, so the remainder is below 1e-20).
__device__ double log_series64(double x) {
    unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    int e = (int)((bits >> 52) & 0x7FFull) - 1023;
    bits = (bits & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull;
    double m = __longlong_as_double((long long)bits);
    if (m > 1.4142135623730951) {
        m = dm(m, 0.5);
        e += 1;
    }
    const double t = __ddiv_rn(ds(m, 1.0), da(m, 1.0));
    const double t2 = dm(t, t);
    double p = 1.0 / 27.0;
#pragma unroll
    for (int k = 25; k >= 1; k -= 2) p = da(dm(p, t2), 1.0 / (double)k);
    return da(dm(dm(2.0, t), p), dm((double)e, 0.6931471805599453));
}

// Two standard normals by the polar method (Marsaglia & Bray 1964): (u1, u2) uniform in the
// unit disk (candidate k uses counter word 3 = purpose|k), f = sqrt(-2 ln s / s).
__device__ bool normal_pair64(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t purpose, uint32_t k0, uint32_t k1,
                              double &g0, double &g1) {
    for (uint32_t k = 0; k < 64; ++k) {
        const uint4 w = philox10(make_uint4(c0, c1, c2, purpose | k), k0, k1);
        const double u1 = ds(dm(2.0, u53(w.x, w.y)), 1.0);
        const double u2 = ds(dm(2.0, u53(w.z, w.w)), 1.0);
        const double s = da(dm(u1, u1), dm(u2, u2));
        if (s >= 1.0 || s == 0.0) continue;
        const double f = __dsqrt_rn(__ddiv_rn(dm(-2.0, log_series64(s)), s));
        g0 = dm(u1, f);
        g1 = dm(u2, f);
        return true;
    }
    g0 = g1 = 0.0;
    return false;
}

__device__ __forceinline__ double3 unit64(double x, double y, double z) {
    const double q = __dsqrt_rn(da(da(dm(x, x), dm(y, y)), dm(z, z)));
    return make_double3(__ddiv_rn(x, q), __ddiv_rn(y, q), __ddiv_rn(z, q));
}

// Orthonormal frame around the unit vector u: e1 = unit(a x u) with a the coordinate axis of
// the smallest |u_k| (the first on ties), e2 = u x e1.
__device__ __forceinline__ void frame64(const double3 u, double3 &e1, double3 &e2) {
    const double ax = fabs(u.x), ay = fabs(u.y), az = fabs(u.z);
    if (ax <= ay && ax <= az)
        e1 = unit64(0.0, -u.z, u.y);
    else if (ay <= az)
        e1 = unit64(u.z, 0.0, -u.x);
    else
        e1 = unit64(-u.y, u.x, 0.0);
    e2 = make_double3(ds(dm(u.y, e1.z), dm(u.z, e1.y)), ds(dm(u.z, e1.x), dm(u.x, e1.z)),
                      ds(dm(u.x, e1.y), dm(u.y, e1.x)));
}

// Point uniform in the cap of height h = 1 - cos(theta) around the unit vector u: a disk
// point (u1, u2) gives s = u1^2 + u2^2 uniform in [0, 1) and the azimuth; z = 1 - s h and
// (x, y) = (u1, u2) sqrt(h (2 - s h)).
__device__ double3 cap64(const double3 u, double h, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t purpose,
                         uint32_t k0, uint32_t k1, uint32_t *err) {
    for (uint32_t k = 0; k < 64; ++k) {
        const uint4 w = philox10(make_uint4(c0, c1, c2, purpose | k), k0, k1);
        const double u1 = ds(dm(2.0, u53(w.x, w.y)), 1.0);
        const double u2 = ds(dm(2.0, u53(w.z, w.w)), 1.0);
        const double s = da(dm(u1, u1), dm(u2, u2));
        if (s >= 1.0) continue;
        const double sh = dm(s, h);
        const double z = ds(1.0, sh);
        const double r = __dsqrt_rn(dm(h, ds(2.0, sh)));
        const double x = dm(u1, r), y = dm(u2, r);
        double3 e1, e2;
        frame64(u, e1, e2);
        return make_double3(da(da(dm(x, e1.x), dm(y, e2.x)), dm(z, u.x)), da(da(dm(x, e1.y), dm(y, e2.y)), dm(z, u.y)),
                            da(da(dm(x, e1.z), dm(y, e2.z)), dm(z, u.z)));
    }
    atomicOr(err, kErrSphere);
    return u;
}

// Trial direction (unit vector) of a site under its policy; the caller scales it by s_i.
__device__ double3 policy_trial64(const PolicySite ps, double sigma, const double4_32a Si, double sn, uint32_t orig,
                                  uint32_t t, uint32_t inst, uint32_t k0, uint32_t k1, uint32_t *err) {
    int code = ps.code;
    if (code == kPolHinzkeNowak) {  // flip, random or small step with probability 1/3 each
        const uint4 w = philox10(make_uint4(orig, t, inst, kPurposeChoice), k0, k1);
        const double v = dm(u53(w.x, w.y), 3.0);
        code = v < 1.0 ? kPolFlip : (v < 2.0 ? kPolRandom : kPolSmallStep);
    }
    if (code == kPolFlip) return make_double3(__ddiv_rn(-Si.x, sn), __ddiv_rn(-Si.y, sn), __ddiv_rn(-Si.z, sn));
    if (code == kPolSmallStep) return cap64(unit64(Si.x, Si.y, Si.z), ps.par, orig, t, inst, kPurposeTrial64, k0, k1, err);
    if (code == kPolGaussian || code == kPolAdaptive) {
        const double sg = code == kPolAdaptive ? sigma : ps.par;
        const double3 u = unit64(Si.x, Si.y, Si.z);
        double g0, g1, g2, g3;
        if (!normal_pair64(orig, t, inst, kPurposeTrial64, k0, k1, g0, g1)) atomicOr(err, kErrSphere);
        if (!normal_pair64(orig, t, inst, kPurposeTrial64 | kPurposeGauss2, k0, k1, g2, g3)) atomicOr(err, kErrSphere);
        return unit64(da(u.x, dm(sg, g0)), da(u.y, dm(sg, g1)), da(u.z, dm(sg, g2)));
    }
    return sphere64(orig, t, inst, kPurposeTrial64, k0, k1, err);
}

// Adaptive width after an MCS with `accepted` of n attempts accepted: sigma * 0.5 / max(1 - R,
// 0.01) clamped to [1e-4, 100], R = accepted / n (the oracle's control law, same roundings).
__device__ __forceinline__ double adapt_width(double sigma, uint32_t accepted, int32_t n) {
    const double rate = __ddiv_rn((double)accepted, (double)n);
    double f = ds(1.0, rate);
    if (f < 0.01) f = 0.01;
    double sg = dm(sigma, __ddiv_rn(0.5, f));
    if (sg < 1e-4) sg = 1e-4;
    if (sg > 100.0) sg = 100.0;
    return sg;
}

// ------------------------------------------------------------------ FP64 colour pass
// A spin through L2 only (ld.global.cg): other blocks of the same launch write spins.
__device__ __forceinline__ double4_32a ldcg_spin64(const double4_32a *p) {
    const double2 lo = __ldcg((const double2 *)p), hi = __ldcg((const double2 *)p + 1);
    return make_double4_32a(lo.x, lo.y, hi.x, hi.y);
}

// One FP64 attempt at site g, replica r (Eq. 1-4, the oracle's order of operations) at MCS t
// of step `step`, adding the site's share of E and M to acc4 and the decision to nacc. Links to
// sites below lower_end count as lower colours when lower_mode is 2 (1: every link). CG = 1
// reads the neighbour spins through L2 only (the cooperative sweep, whose other blocks write
// them within the launch).
template <int CG = 0>
__device__ __forceinline__ void site64(const PassArgs &a, int g, int r, int R, uint32_t t, uint32_t step,
                                       int lower_mode, int lower_end, double4_32a *S, const Edge64 *E, uint32_t k0,
                                       uint32_t k1, double acc4[4], uint32_t &nacc) {
    const RunState *rs = a.run;
    const double *sched = rs->sched;
    const uint32_t inst = (uint32_t)(a.inst0 + r);
    const double *sc = sched + ((int64_t)step * a.n_inst + a.inst_local0 + r) * 2;
    const double beta = sc[0], B = sc[1];
    const uint32_t orig = (uint32_t)a.orig[g];
    double nx, ny, nz, sn, ex, ey, ez, k, kc;
    if (a.params_mode == 2) {
        const double4_32a p0 = ((const double4_32a *)a.p0)[g], p1 = ((const double4_32a *)a.p1)[g];
        nx = p0.x; ny = p0.y; nz = p0.z; sn = p0.w;
        ex = p1.x; ey = p1.y; ez = p1.z; k = p1.w;
        kc = ((const double *)a.pk)[g];
    } else {
        nx = a.u64.nx; ny = a.u64.ny; nz = a.u64.nz; sn = a.u64.s;
        ex = a.u64.ex; ey = a.u64.ey; ez = a.u64.ez; k = a.u64.k; kc = a.u64.kc;
    }
    const int64_t si = (int64_t)g * R + r;
    const double4_32a Si = S[si];
    // local field in the caller's row order, plus the links to lower colours
    double hx = 0.0, hy = 0.0, hz = 0.0, lx = 0.0, ly = 0.0, lz = 0.0;
    for (int64_t e = a.row_ptr[g]; e < a.row_ptr[g + 1]; ++e) {
        const Edge64 ed = E[e];
        const double4_32a Sj = CG ? ldcg_spin64(S + (int64_t)ed.col * R + r) : S[(int64_t)ed.col * R + r];
        hx = da(hx, dm(ed.J, Sj.x));
        hy = da(hy, dm(ed.J, Sj.y));
        hz = da(hz, dm(ed.J, Sj.z));
        if (lower_mode == 1 || (lower_mode == 2 && ed.col < lower_end)) {
            lx = da(lx, dm(ed.J, Sj.x));
            ly = da(ly, dm(ed.J, Sj.y));
            lz = da(lz, dm(ed.J, Sj.z));
        }
    }
    hx = da(hx, dm(B, nx));
    hy = da(hy, dm(B, ny));
    hz = da(hz, dm(B, nz));
    // trial: uniform on the sphere of radius s_i, or the site's update policy
    double px, py, pz;
    if (a.pol && a.pol[g].code == kPolQIsing) {  // another of the 2 s + 1 values along z
        const int n2 = (int)dm(2.0, sn);
        const int idx = (int)da(da(Si.z, sn), 0.5);
        const uint4 w = philox10(make_uint4(orig, t, inst, kPurposeTrial64), k0, k1);
        int k = (int)dm(u53(w.x, w.y), (double)n2);
        if (k >= n2) k = n2 - 1;
        if (k >= idx) k += 1;
        px = 0.0;
        py = 0.0;
        pz = ds((double)k, sn);
    } else {
        const double3 u = a.pol ? policy_trial64(a.pol[g], rs->sigma ? rs->sigma[a.inst_local0 + r] : 0.0, Si, sn,
                                                 orig, t, inst, k0, k1, a.err)
                                : sphere64(orig, t, inst, kPurposeTrial64, k0, k1, a.err);
        px = dm(sn, u.x);
        py = dm(sn, u.y);
        pz = dm(sn, u.z);
    }
    // energy change (Eq. 1-3) in a fixed order
    const double dx = ds(px, Si.x), dy = ds(py, Si.y), dz = ds(pz, Si.z);
    const double dEex = -da(da(dm(dx, hx), dm(dy, hy)), dm(dz, hz));
    double dE = dEex;
    if (a.params_mode != 0) {
        const double pn = da(da(dm(px, ex), dm(py, ey)), dm(pz, ez));
        const double po = da(da(dm(Si.x, ex), dm(Si.y, ey)), dm(Si.z, ez));
        const double dEan = -dm(k, ds(dm(pn, pn), dm(po, po)));
        const double dEcub = -dm(kc, ds(cub64(px, py, pz), cub64(Si.x, Si.y, Si.z)));
        dE = da(da(dEex, dEan), dEcub);
    }
    // Metropolis acceptance (Eq. 4), k_B = 1
    bool acc;
    if (dE <= 0.0) {
        acc = true;
    } else {
        const uint4 wa = philox10(make_uint4(orig, t, inst, kPurposeAccept64), k0, k1);
        acc = u53(wa.x, wa.y) < exp(-dm(beta, dE));
    }
    if (isnan(dE)) {
        atomicOr(a.err, kErrNaN);
        acc = false;
    }
    if (acc) S[si] = make_double4_32a(px, py, pz, 0.0);
    if (a.alog && t < a.alog_mcs)
        a.alog[(int64_t)t * a.alog_stride + a.alog_base + (int64_t)r * a.n_sample_sites + orig] = acc ? 1 : 0;
    // this site's share of E and M after the MCS
    const double qx = acc ? px : Si.x, qy = acc ? py : Si.y, qz = acc ? pz : Si.z;
    double e_i = -(qx * lx + qy * ly + qz * lz) - B * (qx * nx + qy * ny + qz * nz);
    if (a.params_mode != 0) {
        const double pe = qx * ex + qy * ey + qz * ez;
        e_i -= k * pe * pe + kc * cub64(qx, qy, qz);
    }
    acc4[0] += e_i;
    acc4[1] += qx;
    acc4[2] += qy;
    acc4[3] += qz;
    nacc += acc ? 1u : 0u;
}

__global__ void __launch_bounds__(kThreads) pass64_kernel(const PassArgs a) {
    const RunState *rs = a.run;
    const uint32_t t = rs->t;
    const uint32_t step = rs->rec / rs->mcs;
    const int R = 1 << a.log2R;
    const int64_t n_work = (int64_t)(a.g_end - a.g_begin) << a.log2R;
    double4_32a *S = (double4_32a *)a.spins;
    const Edge64 *E = (const Edge64 *)a.edges;
    const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
    double acc4[4] = {0.0, 0.0, 0.0, 0.0};
    uint32_t nacc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n_work; w += stride)
        site64(a, a.g_begin + (int)(w >> a.log2R), (int)(w & (R - 1)), R, t, step, a.lower_mode, a.lower_end, S, E, k0,
               k1, acc4, nacc);
    block_partials(acc4, nacc, R, a.partial + (int64_t)blockIdx.x * R * 4, acc_counters(rs, a.inst_local0));
}

constexpr int kDirectRow = 12;  // rows up to this length gather all neighbours at once

// One attempt of the direct path: gathers the neighbour rows with plain loads (row order),
// draws the trial, decides, writes, and adds the site's share of E and M. Returns the
// decision.
// POL = 1: the sample has an update-policy table (pol[g], the instance's width sigma).
// CG = 1: neighbour spins are read with ld.global.cg (L2 only) because other blocks of the same
// launch write them (cooperative and cluster sweeps); otherwise through the read-only path.
// UD > 0: every row has UD links and site g's start at ud_e0 (a sample of uniform degree), so
// row_ptr is not read and all UD neighbour rows are in flight together. UD = kEllRow: E holds
// fixed rows of kEllRow links in row order, padded with col = -1 entries, which are skipped.
template <int PM, int LM, int POL, int CG = 0, int UD = 0>
__device__ __forceinline__ bool direct_attempt(float4 *S, const int2 *E, const int64_t *row_ptr, int g, int r, int R,
                                               int lower_end, uint32_t orig, const Site32 &p, float beta, float B,
                                               uint32_t t, uint32_t inst, uint32_t k0, uint32_t k1, Acc32 &acc,
                                               bool &nan_seen, const PolicySite32 *pol, float sigma, float4 &Sq,
                                               int64_t ud_e0 = 0) {
    const int64_t si = (int64_t)g * R + r;
    const float4 Si = S[si];
    float2 hxy = make_float2(0.f, 0.f), lxy = make_float2(0.f, 0.f);
    float hz = 0.f, lz = 0.f;
    const int64_t e0 = UD > 0 ? ud_e0 : __ldg(row_ptr + g);
    const int deg = UD > 0 ? UD : (int)(__ldg(row_ptr + g + 1) - e0);
    if (UD > 0) {
        constexpr bool PAD = UD == kEllRow;
        int2 ed[UD > 0 ? UD : 1];
        float4 Sj[UD > 0 ? UD : 1];
#pragma unroll
        for (int k = 0; k < UD; ++k) ed[k] = __ldg(E + e0 + k);
#pragma unroll
        for (int k = 0; k < UD; ++k)
            if (!PAD || ed[k].x >= 0) {
                const float4 *q = S + (int64_t)ed[k].x * R + r;
                Sj[k] = CG ? __ldcg(q) : __ldg(q);
            }
#pragma unroll
        for (int k = 0; k < UD; ++k)
            if (!PAD || ed[k].x >= 0)
                link32(Sj[k], __int_as_float(ed[k].y), LM == 2 && ed[k].x < lower_end, hxy, hz, lxy, lz);
    } else if (deg <= kDirectRow) {
        // all links first, then the neighbour rows with every load in flight together; the
        // field still sums in row order
        int2 ed[kDirectRow];
#pragma unroll
        for (int k = 0; k < kDirectRow; ++k)
            if (k < deg) ed[k] = __ldg(E + e0 + k);
#pragma unroll
        for (int k0 = 0; k0 < kDirectRow; k0 += 4) {  // neighbour rows four at a time
            if (k0 >= deg) break;
            float4 Sj[4];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (k0 + k < deg) {
                    const float4 *q = S + (int64_t)ed[k0 + k].x * R + r;
                    Sj[k] = CG ? __ldcg(q) : __ldg(q);
                }
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (k0 + k < deg)
                    link32(Sj[k], __int_as_float(ed[k0 + k].y), LM == 2 && ed[k0 + k].x < lower_end, hxy, hz, lxy, lz);
        }
    } else {
        for (int64_t e = e0; e < e0 + deg; ++e) {
            const int2 ed = __ldg(E + e);
            const float4 *q = S + (int64_t)ed.x * R + r;
            link32(CG ? __ldcg(q) : __ldg(q), __int_as_float(ed.y), LM == 2 && ed.x < lower_end, hxy, hz, lxy, lz);
        }
    }
    if (LM == 1) {
        lxy = hxy;
        lz = hz;
    }
    const uint4 rw = philox10(make_uint4(orig, t, inst, kPurposeTrial32), k0, k1);
    const float3 P = POL ? policy_trial32(pol[g], sigma, Si, p.sn, rw) : trial_random32(rw, p.sn);
    float4 Sn;
    bool ok, bad;
    float e_i;
    attempt32<PM, LM>(Si, hxy, hz, lxy, lz, p, beta, B, P, rw.z, Sn, ok, e_i, bad);
    nan_seen |= bad;
    if (ok) S[si] = Sn;
    acc.add(e_i, Sn, ok);
    Sq = Sn;
    return ok;
}

#ifdef VEGAS_DEBUG_CHECKS
// Debug builds: the row of site g and every neighbour index in it, and the caller id, are
// checked before the attempt reads through them; a bad one sets kErrIndex, records a code
// and the value, and the attempt is skipped. n_edges_total == 0 means the link count is not
// known (the allocation-free entry point): rows are then checked for order only.
__device__ bool direct_row_ok(const PassArgs &a, int g, uint32_t orig) {
    uint32_t code = 0;
    int64_t val = 0;
    const int64_t e0 = a.row_ptr[g], e1 = a.row_ptr[g + 1];
    if (orig >= (uint32_t)a.n_sample_sites) {
        code = 31;
        val = orig;
    } else if (e0 < 0 || e1 < e0 || (a.n_edges_total > 0 && e1 > a.n_edges_total)) {
        code = 32;
        val = g;
    } else {
        const int2 *E = (const int2 *)a.edges;
        for (int64_t e = e0; e < e1; ++e) {
            const int j = E[e].x;
            if (j < 0 || j >= a.n_sites_total) {
                code = 33;
                val = j;
                break;
            }
        }
    }
    if (code == 0) return true;
    atomicOr(a.err, kErrIndex);
    atomicCAS(a.err + 1, 0u, code);
    a.err[2] = (uint32_t)val;
    return false;
}
#endif

// Spins in shared memory (the resident and cluster sweeps): a region of 3 cap floats holds x and
// y of site i as one 8-byte pair at pair index i and z at float 2 cap + i, so a neighbour takes
// two loads; regions start at multiples of 3 cap floats with cap even, so the pairs are 8-byte
// aligned.
__device__ __forceinline__ float4 sm_spin(const float *sp, int cap, int i) {
    const float2 xy = ((const float2 *)sp)[i];
    return make_float4(xy.x, xy.y, sp[2 * cap + i], 0.f);
}
__device__ __forceinline__ void sm_set(float *sp, int cap, int i, float x, float y, float z) {
    ((float2 *)sp)[i] = make_float2(x, y);
    sp[2 * cap + i] = z;
}

// The same attempt with the instance's spins in shared memory (resident sweep with spins kept
// on chip for the whole step): sp holds the instance's sites in the layout of sm_spin, site g
// at g - g0. The site's links come as a fixed row of kEllRow (neighbour,
// J) pairs in row order, padded with neighbour -1 (erow, 16-byte aligned), so no row offset is
// read before them. Neighbour values, the field's row order and every rounding are those of
// direct_attempt, so the results are bit for bit the same.
// AN = 0: no instance has anisotropy or per-site parameters, so the anisotropy terms (zeros
// there) are left out; the spins and decisions are those of the general form.
template <int POL, int AN = 1>
__device__ __forceinline__ bool smem_attempt(float *sp, int cap, int g0, const int4 *erow, int g, int lower_end,
                                             uint32_t orig, const Site32 &p, float beta, float B, uint32_t t,
                                             uint32_t inst, uint32_t k0, uint32_t k1, Acc32 &acc, bool &nan_seen,
                                             const PolicySite32 *pol, float sigma, float4 &Sq) {
    const int i = g - g0;
    const float4 Si = sm_spin(sp, cap, i);
    float2 hxy = make_float2(0.f, 0.f), lxy = make_float2(0.f, 0.f);
    float hz = 0.f, lz = 0.f;
    int4 q[kEllRow / 2];
#pragma unroll
    for (int k = 0; k < kEllRow / 2; ++k) q[k] = __ldg(erow + k);
#pragma unroll
    for (int k = 0; k < kEllRow / 2; ++k) {
        if (q[k].x >= 0) {
            const int j = q[k].x - g0;
            link32(sm_spin(sp, cap, j), __int_as_float(q[k].y), q[k].x < lower_end,
                   hxy, hz, lxy, lz);
        }
        if (q[k].z >= 0) {
            const int j = q[k].z - g0;
            link32(sm_spin(sp, cap, j), __int_as_float(q[k].w), q[k].z < lower_end,
                   hxy, hz, lxy, lz);
        }
    }
    const uint4 rw = philox10(make_uint4(orig, t, inst, kPurposeTrial32), k0, k1);
    const float3 P = POL ? policy_trial32(pol[g], sigma, Si, p.sn, rw) : trial_random32(rw, p.sn);
    float4 Sn;
    bool ok, bad;
    float e_i;
    attempt32<AN ? 2 : 0, 2>(Si, hxy, hz, lxy, lz, p, beta, B, P, rw.z, Sn, ok, e_i, bad);
    nan_seen |= bad;
    if (ok) sm_set(sp, cap, i, Sn.x, Sn.y, Sn.z);
    acc.add(e_i, Sn, ok);
    Sq = Sn;
    return ok;
}

// One fixed row of links (96 bytes: at most two 128-byte lines) and the caller id of a site
// into L1 ahead of use.
__device__ __forceinline__ void prefetch_site_l1(const int4 *ell, const int32_t *orig, int g) {
    const char *p0 = (const char *)(ell + (size_t)g * (kEllRow / 2));
    const char *p1 = p0 + kEllRow * sizeof(int2) - 1;
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p0));
    if (((uintptr_t)p0 >> 7) != ((uintptr_t)p1 >> 7)) asm volatile("prefetch.global.L1 [%0];" ::"l"(p1));
    asm volatile("prefetch.global.L1 [%0];" ::"l"(orig + g));
}

// The sites of one colour segment that a thread sweeps with the spins in shared memory: g,
// g + stride, ... below end; the next site's links are prefetched into L1 while the current
// one is computed, and after the last one the thread's first site of the next segment
// (next_g, if below next_end), whose class comes after the barrier.
template <typename F>
__device__ __forceinline__ void smem_segment(const int4 *ell, const int32_t *orig, int g, int end, int stride,
                                             int next_g, int next_end, F &&visit) {
    for (; g < end; g += stride) {
        if (g + stride < end)
            prefetch_site_l1(ell, orig, g + stride);
        else if (next_g < next_end)
            prefetch_site_l1(ell, orig, next_g);
        visit(g);
    }
}

// ------------------------------------------------------------------ FP32 colour pass (direct)
// Any row length: reads row_ptr and gathers neighbours with plain loads.
// PM: params_mode (0 uniform without anisotropy, 1 uniform, 2 per site).
// LM: lower_mode (0 no lower links, 1 all links lower, 2 test each link).
// block / grid: the block's index in the pass and the pass's block count (blockIdx.x and
// gridDim.x in the pass's own launch).
template <int PM, int LM, int POL>
__device__ __forceinline__ void pass32_body(const PassArgs &a, int block, int grid) {
    const RunState *rs = a.run;
    const uint32_t t = rs->t;
    const uint32_t step = rs->rec / rs->mcs;
    const int R = 1 << a.log2R;
    const int64_t n_work = (int64_t)(a.g_end - a.g_begin) << a.log2R;
    float4 *S = (float4 *)a.spins;
    const int2 *E = (const int2 *)a.edges;
    const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
    const int64_t stride = (int64_t)grid * blockDim.x;
    const int64_t w0 = (int64_t)block * blockDim.x + threadIdx.x;
    // a thread always serves the same replica (the stride is a multiple of 32 >= R)
    const int r = (int)(w0 & (R - 1));
    const uint32_t inst = (uint32_t)(a.inst0 + r);
    const double *sc = rs->sched + ((int64_t)step * a.n_inst + a.inst_local0 + r) * 2;
    const float beta = (float)sc[0], B = (float)sc[1];
    const float sigma = (POL && rs->sigma) ? (float)rs->sigma[a.inst_local0 + r] : 0.f;
    Acc32 acc;
    for (int64_t w = w0; w < n_work; w += stride) {
        const int g = a.g_begin + (int)(w >> a.log2R);
        const uint32_t orig = (uint32_t)__ldg(a.orig + g);
#ifdef VEGAS_DEBUG_CHECKS
        if (!direct_row_ok(a, g, orig)) continue;
#endif
        bool nan_seen = false;
        float4 Sq;
        const bool ok = direct_attempt<PM, LM, POL>(S, E, a.row_ptr, g, r, R, a.lower_end, orig, site_params32(a, PM, g),
                                                    beta, B, t, inst, k0, k1, acc, nan_seen, a.pol32, sigma, Sq);
        if (nan_seen) atomicOr(a.err, kErrNaN);
        if (a.alog && t < a.alog_mcs)
            a.alog[(int64_t)t * a.alog_stride + a.alog_base + (int64_t)r * a.n_sample_sites + orig] = ok ? 1 : 0;
    }
    acc.flush();
    block_partials(acc.d, acc.nacc, R, a.partial + (int64_t)block * R * 4, acc_counters(rs, a.inst_local0));
}

template <int PM, int LM, int POL>
__global__ void __launch_bounds__(kThreads, 2) pass32_kernel(const PassArgs a) {
    pass32_body<PM, LM, POL>(a, blockIdx.x, gridDim.x);
}

// Several passes of one colour class with the same kernel (the samples of a batch) in one
// launch: block b runs block b - first[p] of pass p, first[p] <= b < first[p + 1], with that
// pass's arguments (copied to shared memory) and block count, so every block does what it does
// in the pass's own launch and writes the same partial sums.
template <int PM, int LM, int POL>
__global__ void __launch_bounds__(kThreads, 2) pass32_multi_kernel(const PassArgs *passes, const int32_t *first,
                                                                   int32_t n) {
    static_assert(sizeof(PassArgs) % 8 == 0, "copied as 8-byte words");
    __shared__ PassArgs s_a;
    __shared__ int s_p;
    if (threadIdx.x == 0) {  // the last pass whose first block is <= blockIdx.x
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(first + mid) <= (int32_t)blockIdx.x)
                lo = mid;
            else
                hi = mid - 1;
        }
        s_p = lo;
    }
    __syncthreads();
    const int p = s_p;
    const uint64_t *src = (const uint64_t *)(passes + p);
    for (int i = threadIdx.x; i < (int)(sizeof(PassArgs) / 8); i += blockDim.x) ((uint64_t *)&s_a)[i] = __ldg(src + i);
    __syncthreads();
    const int f = __ldg(first + p);
    pass32_body<PM, LM, POL>(s_a, (int)blockIdx.x - f, __ldg(first + p + 1) - f);
}

// ------------------------------------------------------------------ resident (persistent) sweep
// Every block takes instances from a queue (largest first; an atomic ticket, no waiting)
// and runs all MCS of the step on it: colour class after colour class with __syncthreads
// in between, then a fixed-order block sum of E and M written straight into the history.
// Used for batches of many small, uneven samples, where one launch per colour class of
// every sample would cost far more than the sweep itself.
__device__ __forceinline__ Site32 resident_params(const ResidentArgs &a, const ResidentInst &I, int g) {
    if (I.params_mode == 2) {
        const float4 p0 = __ldg((const float4 *)a.p0 + g), p1 = __ldg((const float4 *)a.p1 + g);
        return Site32{p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w, __ldg((const float *)a.pk + g)};
    }
    return Site32{I.u.nx, I.u.ny, I.u.nz, I.u.s, I.u.ex, I.u.ey, I.u.ez, I.u.k, I.u.kc};
}

constexpr int kResidentMaxTypes = 8;  // per-type statistics in the resident sweep

// Every MCS of the current step on instance I by a group of gthreads threads of the block
// (the whole block: gbar = 0; else warps gtid / 32 .. of a group meeting at named barrier
// gbar): colour class after colour class with a barrier between them, then a fixed-order
// sum of the group's warps' E and M (and per-type magnetization, s_tm zeroed by the caller)
// written into the history.
__device__ __forceinline__ void group_sync(int bar, int nthreads) {
    if (bar == 0)
        __syncthreads();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nthreads) : "memory");
}


// SM = 1: the instance's spins are copied into shared memory (sp, three arrays of cap floats)
// before the first MCS, every attempt reads and writes them there, and they are copied back
// after the last MCS of the launch; only the links and parameters come from L2 and HBM.
template <int NT, int POL, int SM = 0, int AN = 1>
__device__ __forceinline__ void resident_sweep_block(const ResidentArgs &a, const ResidentInst &I, double (*s_red)[4], uint32_t *s_acc,
                                     double (*s_tm)[kResidentMaxTypes][3], double (*s_part)[4], bool &nan_seen,
                                     int gtid, int gthreads, int gbar, float *sp = nullptr, int cap = 0) {
    float4 *S = (float4 *)a.spins;
    const int2 *E = (const int2 *)a.edges;
    const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
    const int R = 1 << a.log2R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n_types = a.n_types;
    RunState *rs = a.run;
    const int gw0 = (threadIdx.x - gtid) >> 5;  // the group's first warp
    const uint32_t t0 = rs->t, rec0 = rs->rec;
    const uint32_t step = rec0 / rs->mcs;
    const double *sc = rs->sched + ((int64_t)step * a.n_inst + I.inst_local) * 2;
    const float beta = (float)sc[0], B = (float)sc[1];
    const uint32_t inst = (uint32_t)I.inst_id;
    if (SM) {  // the instance's spins into shared memory
        for (int g = I.g_begin + gtid; g < I.g_end; g += gthreads) {
            const float4 v = S[(int64_t)g * R + I.r];
            sm_set(sp, cap, g - I.g_begin, v.x, v.y, v.z);
        }
        group_sync(gbar, gthreads);
    }
    for (int m = 0; m < a.mcs; ++m) {
        const uint32_t t = t0 + (uint32_t)m;
        const bool log_accepts = a.alog && t < a.alog_mcs;
        // the width is read after the barrier that ends the previous MCS (thread 0 wrote it)
        const float sigma = (POL && rs->sigma) ? (float)rs->sigma[I.inst_local] : 0.f;
        Acc32 acc;
        for (int q = 0; q < I.n_segs; ++q) {
            const int4 sg = a.segs[I.seg_off + q];  // {begin, end, class begin, type | last << 16}
            float tm[3] = {0.f, 0.f, 0.f};
            // the attempt of site g: one code path for every parameter mode (with k = kc = 0 the
            // anisotropy terms add signed zeros only, so spins and decisions equal the specialised
            // paths'); SM: row given, spins in shared memory
            auto visit = [&](int g) {
                const uint32_t orig = (uint32_t)__ldg(a.orig + g);
                const Site32 p = resident_params(a, I, g);
                float4 Sq;
                const bool ok =
                    SM ? smem_attempt<POL, AN>(sp, cap, I.g_begin, a.ell + (size_t)g * (kEllRow / 2), g, sg.z, orig,
                                               p, beta, B, t, inst, k0, k1, acc, nan_seen, a.pol, sigma, Sq)
                       : direct_attempt<2, 2, POL>(S, E, a.row_ptr, g, I.r, R, sg.z, orig, p, beta, B, t, inst, k0, k1,
                                                   acc, nan_seen, a.pol, sigma, Sq);
                tm[0] = __fadd_rn(tm[0], Sq.x);
                tm[1] = __fadd_rn(tm[1], Sq.y);
                tm[2] = __fadd_rn(tm[2], Sq.z);
                if (log_accepts)
                    a.alog[(int64_t)t * a.alog_stride + I.alog_base + (int64_t)I.r * I.n_sample_sites + orig] =
                        ok ? 1 : 0;
            };
            if (SM) {
                const int4 nx = q + 1 < I.n_segs ? a.segs[I.seg_off + q + 1] : make_int4(0, 0, 0, 0);
                smem_segment(a.ell, a.orig, sg.x + gtid, sg.y, gthreads, nx.x + gtid, nx.y, visit);
            } else {
                for (int g = sg.x + gtid; g < sg.y; g += gthreads) visit(g);
            }
            if (n_types > 0) {  // this segment's magnetization into its type (fixed order)
                double d[3] = {(double)tm[0], (double)tm[1], (double)tm[2]};
                for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) d[c] += __shfl_xor_sync(0xFFFFFFFFu, d[c], off);
                }
                const int ty = sg.w & 0xFFFF;
                if (lane == 0 && ty < kResidentMaxTypes) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) s_tm[warp][ty][c] += d[c];
                }
            }
            if (sg.w >> 16) group_sync(gbar, gthreads);  // the last segment of a colour class
        }
        // the MCS's totals in FP64 with few FP64 operations (GB300 runs two per SM and clock):
        // every thread leaves its four sums in shared memory, then warp q of the group adds
        // quantity q over the group's threads (each lane a fixed stride, then a butterfly),
        // so the order, and the result, is fixed
        acc.flush();
        uint32_t na = acc.nacc;
        for (int off = 16; off > 0; off >>= 1) na += __shfl_xor_sync(0xFFFFFFFFu, na, off);
#pragma unroll
        for (int q = 0; q < 4; ++q) s_part[threadIdx.x][q] = acc.d[q];
        if (lane == 0) s_acc[warp] = na;
        group_sync(gbar, gthreads);
        {
            const int gw = gtid >> 5, nw = gthreads >> 5, t0 = (int)threadIdx.x - gtid;
            for (int q = gw; q < 4; q += nw) {
                double x = 0.0;
                for (int k = lane; k < gthreads; k += 32) x += s_part[t0 + k][q];
                for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, off);
                if (lane == 0) s_red[gw0][q] = x;
            }
        }
        group_sync(gbar, gthreads);
        if (gtid == 0) {
            double sum[4];
            uint32_t nsum = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) sum[q] = s_red[gw0][q];
            for (int w = gw0; w < gw0 + (gthreads >> 5); ++w) nsum += s_acc[w];
            const int64_t rec = (int64_t)rec0 + m;
            double *h = rs->hist + (rec * a.n_inst + I.inst_local) * 4;
#pragma unroll
            for (int q = 0; q < 4; ++q) h[q] = sum[q];
            if (rs->acc_hist) rs->acc_hist[rec * a.n_inst + I.inst_local] = nsum;
            if (I.adaptive && rs->sigma && (uint32_t)(rec % rs->mcs) < rs->mcs / 5)
                rs->sigma[I.inst_local] = adapt_width(rs->sigma[I.inst_local], nsum, I.n_sample_sites);
            if (n_types > 0 && rs->type_hist) {
                double *th = rs->type_hist + (rec * a.n_inst + I.inst_local) * n_types * 3;
                for (int k = 0; k < n_types; ++k)
                    for (int c = 0; c < 3; ++c) {
                        double x = 0.0;
                        for (int w = gw0; w < gw0 + (gthreads >> 5); ++w) {
                            x += s_tm[w][k][c];
                            s_tm[w][k][c] = 0.0;
                        }
                        th[k * 3 + c] = x;
                    }
            }
        }
        group_sync(gbar, gthreads);
    }
    if (SM)  // the last MCS ended at a barrier: its spins go back to global memory
        for (int g = I.g_begin + gtid; g < I.g_end; g += gthreads) {
            const int i = g - I.g_begin;
            S[(int64_t)g * R + I.r] = sm_spin(sp, cap, i);
        }
}

// Draws instances from the queue and sweeps them until it is empty (first >= 0: start with
// that one). An instance of at most group_sites sites comes with NT / group_threads - 1 more
// (the queue is largest first, so they are no larger), and the block sweeps them at once,
// a group of group_threads threads each; larger instances take the whole block.
// SM = 1: spins in shared memory, dyn: the block's dynamic shared memory (a group gi of ng
// takes region gi of a.group_sites sites, a whole-block instance all a.smem_sites).
template <int NT, int POL, int SM = 0, int AN = 1>
__device__ __forceinline__ void resident_loop(const ResidentArgs &a, int first, double (*s_red)[4], uint32_t *s_acc,
                                              double (*s_tm)[kResidentMaxTypes][3], double (*s_part)[4], int *s_items,
                                              bool &nan_seen, float *dyn = nullptr) {
    const int GT = a.group_threads;
    for (;;) {
        if (threadIdx.x == 0) {
            const int it = first >= 0 ? first : (int)atomicAdd(a.queue, 1u);
            int ng = 1;
            if (GT > 0 && GT < NT && it < a.n_items && a.insts[it].g_end - a.insts[it].g_begin <= a.group_sites) {
                ng = NT / GT;
                const int more = (int)atomicAdd(a.queue, (uint32_t)(ng - 1));
                for (int k = 1; k < ng; ++k) s_items[k] = more + k - 1;
            }
            s_items[0] = it;
            s_items[NT / 32] = ng;
        }
        first = -1;
        for (int q = threadIdx.x; q < (NT / 32) * kResidentMaxTypes * 3; q += NT) (&s_tm[0][0][0])[q] = 0.0;
        __syncthreads();
        const int ng = s_items[NT / 32];
        if (s_items[0] >= a.n_items) break;
        // one group per instance drawn (the whole block when ng = 1, named barrier 0)
        const int gt = NT / ng, gi = (int)threadIdx.x / gt, item = s_items[gi];
        if (item < a.n_items) {
            const ResidentInst I = a.insts[item];
            const int cap = ng == 1 ? a.smem_sites : a.group_sites;
            resident_sweep_block<NT, POL, SM, AN>(a, I, s_red, s_acc, s_tm, s_part, nan_seen, (int)threadIdx.x - gi * gt,
                                              gt, ng == 1 ? 0 : 1 + gi,
                                              SM ? dyn + (size_t)gi * 3 * (size_t)((cap + 1) & ~1) : nullptr, cap);
        }
        __syncthreads();  // every group is done before the items are drawn again
    }
}

// The same, for the cluster sweep's second phase (inlined: a call kept its registers apart from
// the cluster phase's but made the phase slower than the resident kernel).
template <int NT, int POL, int SM = 0>
__device__ __forceinline__ void resident_loop_call(const ResidentArgs &a, int first, double (*s_red)[4], uint32_t *s_acc,
                                                double (*s_tm)[kResidentMaxTypes][3], double (*s_part)[4],
                                                int *s_items, bool &nan_seen, float *dyn = nullptr) {
    resident_loop<NT, POL, SM>(a, first, s_red, s_acc, s_tm, s_part, s_items, nan_seen, dyn);
}

template <int NT, int POL, int SM = 0, int AN = 1>
__global__ void __launch_bounds__(NT) resident32_kernel(const ResidentArgs a) {
    __shared__ int s_items[NT / 32 + 1];  // the instances drawn (one per group) and their count
    __shared__ double s_red[NT / 32][4];
    __shared__ uint32_t s_acc[NT / 32];
    __shared__ double s_tm[NT / 32][kResidentMaxTypes][3];  // per warp and type, segment order
    __shared__ double s_part[NT][4];                         // every thread's MCS totals
    extern __shared__ __align__(16) float res_dyn[];         // SM: the instances' spins
    bool nan_seen = false;
    resident_loop<NT, POL, SM, AN>(a, -1, s_red, s_acc, s_tm, s_part, s_items, nan_seen, res_dyn);
    if (nan_seen) atomicOr(a.err, kErrNaN);
}

// ------------------------------------------------------------------ cluster sweep
// As the resident sweep, but a thread-block cluster of CS blocks (on CS SMs) takes each
// instance: the blocks split every colour segment, meet at the hardware cluster barrier
// between classes, and rank 0 sums the blocks' per-MCS totals from their shared memory in
// rank order. For instances too large for one block and too small to fill the GPU per class.
// Every block of a cluster runs the same loop (rank 0 fetches the instance and the others
// read it from rank 0's shared memory), so all of them reach every barrier. Instances are
// queued largest first: from the first one with at most split_sites sites on, the blocks of
// a cluster leave the loop together and sweep instances alone, as the resident sweep does
// (rank 0 keeps the one just drawn), so small instances do not hold a whole cluster.
// SM = 1: every block of the cluster keeps a full copy of the instance's spins in its shared
// memory; an attempt reads its own copy, and an accepted spin is written to every block's
// copy (distributed shared memory). No block reads a site of the class being swept, and the
// cluster barrier at the end of the class orders those writes before the next class reads
// them, so every copy holds the same values at every barrier. The blocks then sweep small
// instances alone, each in its own shared memory as the resident sweep does.
template <int NT, int POL, int SM = 0>
__global__ void __launch_bounds__(NT, 512 / NT) cluster32_kernel(const ResidentArgs a) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int CS = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    constexpr int NB = 5 + kResidentMaxTypes * 3;  // E, Mx, My, Mz, accepted, per-type M
    __shared__ int s_item;
    __shared__ double s_red[NT / 32][4];
    __shared__ uint32_t s_acc[NT / 32];
    __shared__ double s_tm[NT / 32][kResidentMaxTypes][3];
    __shared__ double s_blk[NB];  // this block's totals of the MCS
    __shared__ double s_tot[NB];  // rank 0: the cluster's totals
    float4 *S = (float4 *)a.spins;
    const int2 *E = (const int2 *)a.edges;
    const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
    const int R = 1 << a.log2R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n_types = a.n_types;
    RunState *rs = a.run;
    bool nan_seen = false;
    extern __shared__ __align__(16) float cl_dyn[];  // SM: this block's copy of the instance's spins
    const int cap = a.smem_sites;
    int alone = -2;  // >= -1: the blocks sweep alone from now on (-1: draw the next instance)
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) s_item = (int)atomicAdd(a.queue, 1u);
        for (int q = threadIdx.x; q < (NT / 32) * kResidentMaxTypes * 3; q += NT) (&s_tm[0][0][0])[q] = 0.0;
        cl.sync();
        const int item = *cl.map_shared_rank(&s_item, 0);
        cl.sync();  // every block has read the item before rank 0 fetches the next
        if (item >= a.n_items) break;
        const ResidentInst I = a.insts[item];
        if (a.split_sites > 0 && I.g_end - I.g_begin <= a.split_sites) {
            alone = rank == 0 ? item : -1;
            break;
        }
        const uint32_t t0 = rs->t, rec0 = rs->rec;
        const uint32_t step = rec0 / rs->mcs;
        const double *sc = rs->sched + ((int64_t)step * a.n_inst + I.inst_local) * 2;
        const float beta = (float)sc[0], B = (float)sc[1];
        const uint32_t inst = (uint32_t)I.inst_id;
        if (SM) {  // every block: the whole instance into its own shared memory
            for (int g = I.g_begin + (int)threadIdx.x; g < I.g_end; g += NT) {
                const float4 v = S[(int64_t)g * R + I.r];
                sm_set(cl_dyn, cap, g - I.g_begin, v.x, v.y, v.z);
            }
            cl.sync();  // no block writes into a copy that is still being loaded
        }
        for (int m = 0; m < a.mcs; ++m) {
            const uint32_t t = t0 + (uint32_t)m;
            const bool log_accepts = a.alog && t < a.alog_mcs;
            const float sigma = (POL && rs->sigma) ? (float)rs->sigma[I.inst_local] : 0.f;
            Acc32 acc;
            for (int q = 0; q < I.n_segs; ++q) {
                const int4 sg = a.segs[I.seg_off + q];  // {begin, end, class begin, type | last << 16}
                float tm[3] = {0.f, 0.f, 0.f};
                auto visit = [&](int g) {
                    const uint32_t orig = (uint32_t)__ldg(a.orig + g);
                    const Site32 p = resident_params(a, I, g);
                    float4 Sq;
                    bool ok;
                    if (SM) {
                        ok = smem_attempt<POL>(cl_dyn, cap, I.g_begin, a.ell + (size_t)g * (kEllRow / 2), g, sg.z,
                                               orig, p, beta, B, t, inst, k0, k1, acc, nan_seen, a.pol, sigma, Sq);
                        if (ok) {  // the new spin into the other blocks' copies
                            const int i = g - I.g_begin;
                            for (int b = 1; b < CS; ++b) {
                                sm_set(cl.map_shared_rank(cl_dyn, (rank + b) % CS), cap, i, Sq.x, Sq.y, Sq.z);
                            }
                        }
                    } else {
                        ok = direct_attempt<2, 2, POL, 1>(S, E, a.row_ptr, g, I.r, R, sg.z, orig, p, beta, B, t, inst,
                                                          k0, k1, acc, nan_seen, a.pol, sigma, Sq);
                    }
                    tm[0] = __fadd_rn(tm[0], Sq.x);
                    tm[1] = __fadd_rn(tm[1], Sq.y);
                    tm[2] = __fadd_rn(tm[2], Sq.z);
                    if (log_accepts)
                        a.alog[(int64_t)t * a.alog_stride + I.alog_base + (int64_t)I.r * I.n_sample_sites + orig] =
                            ok ? 1 : 0;
                };
                const int off = rank * NT + (int)threadIdx.x;
                if (SM) {
                    const int4 nx = q + 1 < I.n_segs ? a.segs[I.seg_off + q + 1] : make_int4(0, 0, 0, 0);
                    smem_segment(a.ell, a.orig, sg.x + off, sg.y, CS * NT, nx.x + off, nx.y, visit);
                } else {
                    for (int g = sg.x + off; g < sg.y; g += CS * NT) visit(g);
                }
                if (n_types > 0) {
                    double d[3] = {(double)tm[0], (double)tm[1], (double)tm[2]};
                    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) d[c] += __shfl_xor_sync(0xFFFFFFFFu, d[c], off);
                    }
                    const int ty = sg.w & 0xFFFF;
                    if (lane == 0 && ty < kResidentMaxTypes) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) s_tm[warp][ty][c] += d[c];
                    }
                }
                if (sg.w >> 16) cl.sync();  // a colour class ends: its spins are final for the cluster
            }
            acc.flush();
            double v[4] = {acc.d[0], acc.d[1], acc.d[2], acc.d[3]};
            uint32_t na = acc.nacc;
            for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] += __shfl_xor_sync(0xFFFFFFFFu, v[q], off);
                na += __shfl_xor_sync(0xFFFFFFFFu, na, off);
            }
            if (lane == 0) {
#pragma unroll
                for (int q = 0; q < 4; ++q) s_red[warp][q] = v[q];
                s_acc[warp] = na;
            }
            __syncthreads();
            if (threadIdx.x == 0) {  // this block's totals, warps in order
                double sum[4] = {0.0, 0.0, 0.0, 0.0};
                uint32_t nsum = 0;
                for (int w = 0; w < NT / 32; ++w) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) sum[q] += s_red[w][q];
                    nsum += s_acc[w];
                }
                for (int q = 0; q < 4; ++q) s_blk[q] = sum[q];
                s_blk[4] = (double)nsum;
                // per-type magnetization only with per-type statistics (a serial chain on one
                // thread while the cluster waits)
                for (int k = 0; k < n_types && k < kResidentMaxTypes; ++k)
                    for (int c = 0; c < 3; ++c) {
                        double x = 0.0;
                        for (int w = 0; w < NT / 32; ++w) {
                            x += s_tm[w][k][c];
                            s_tm[w][k][c] = 0.0;
                        }
                        s_blk[5 + k * 3 + c] = x;
                    }
            }
            cl.sync();
            if (rank == 0) {  // the cluster's totals: thread q sums quantity q over the blocks in rank order
                if ((int)threadIdx.x < NB) {
                    double x = 0.0;
                    for (int b = 0; b < CS; ++b) x += cl.map_shared_rank(s_blk, b)[threadIdx.x];
                    s_tot[threadIdx.x] = x;
                }
                __syncthreads();
            }
            if (rank == 0 && threadIdx.x == 0) {
                const double *tot = s_tot;
                const int64_t rec = (int64_t)rec0 + m;
                double *h = rs->hist + (rec * a.n_inst + I.inst_local) * 4;
                for (int q = 0; q < 4; ++q) h[q] = tot[q];
                const uint32_t nsum = (uint32_t)tot[4];
                if (rs->acc_hist) rs->acc_hist[rec * a.n_inst + I.inst_local] = nsum;
                if (I.adaptive && rs->sigma && (uint32_t)(rec % rs->mcs) < rs->mcs / 5)
                    rs->sigma[I.inst_local] = adapt_width(rs->sigma[I.inst_local], nsum, I.n_sample_sites);
                if (n_types > 0 && rs->type_hist) {
                    double *th = rs->type_hist + (rec * a.n_inst + I.inst_local) * n_types * 3;
                    for (int k = 0; k < n_types && k < kResidentMaxTypes; ++k)
                        for (int c = 0; c < 3; ++c) th[k * 3 + c] = tot[5 + k * 3 + c];
                }
            }
            cl.sync();  // the width and the totals' buffers are ready for the next MCS
        }
        if (SM)  // each block's own sites back to global memory (the copies agree after the last barrier)
            for (int q = 0; q < I.n_segs; ++q) {
                const int4 sg = a.segs[I.seg_off + q];
                for (int g = sg.x + rank * NT + (int)threadIdx.x; g < sg.y; g += CS * NT) {
                    const int i = g - I.g_begin;
                    S[(int64_t)g * R + I.r] = sm_spin(cl_dyn, cap, i);
                }
            }
    }
    // small instances: no shared memory of another block is read or written from here on
    if (alone >= -1) {
        __shared__ int s_items[NT / 32 + 1];
        __shared__ double s_part[NT][4];
        resident_loop_call<NT, POL, SM>(a, alone, s_red, s_acc, s_tm, s_part, s_items, nan_seen, cl_dyn);
    }
    if (nan_seen) atomicOr(a.err, kErrNaN);
}

// ------------------------------------------------------------------ cooperative sweep
// One sample, all blocks: class c of MCS m is swept by the whole grid, then the grid meets
// at a barrier. The barrier's wait is bounded by the global timer: a block that waits
// longer than timeout_ns sets kErrTimeout and the abort flag, and every block returns at
// its next barrier (or while waiting), so a lost block never hangs the GPU.
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ bool grid_barrier(GridBarrier *b, uint32_t nblocks, int64_t timeout_ns, uint32_t *err, bool skip) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile GridBarrier *vb = b;
        const uint32_t gen = vb->gen;
        __threadfence();
        if (!skip) {
            const uint32_t arrived = atomicAdd(&b->count, 1u);
            if (arrived == nblocks - 1) {
                atomicExch(&b->count, 0u);
                __threadfence();
                atomicAdd(&b->gen, 1u);
            } else {
                const uint64_t t0 = global_ns();
                while (vb->gen == gen) {
                    if (vb->abort) {
                        ok = 0;
                        break;
                    }
                    if ((int64_t)(global_ns() - t0) > timeout_ns) {
                        atomicOr(err, kErrTimeout);
                        atomicExch(&b->abort, 1u);
                        ok = 0;
                        break;
                    }
                }
            }
        } else {
            ok = 0;  // fault injection: leave without arriving
        }
        __threadfence();
        if (vb->abort) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// The grid barrier in two halves, so that a block can do work between arriving and waiting
// that no other block's writes affect. Arrival: every thread of the block is done, thread 0
// notes the generation and adds the block to the count (the last block advances the
// generation). Wait: thread 0 waits, bounded as in grid_barrier, until the generation moves.
struct BarrierTicket {
    uint32_t gen;
    bool released;
};
__device__ __forceinline__ BarrierTicket grid_arrive(GridBarrier *b, uint32_t nblocks, bool skip) {
    BarrierTicket tk{0u, false};
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile GridBarrier *vb = b;
        tk.gen = vb->gen;
        __threadfence();
        if (!skip && atomicAdd(&b->count, 1u) == nblocks - 1) {
            atomicExch(&b->count, 0u);
            __threadfence();
            atomicAdd(&b->gen, 1u);
            tk.released = true;
        }
    }
    return tk;  // meaningful in thread 0 only
}
__device__ bool grid_wait(GridBarrier *b, BarrierTicket tk, int64_t timeout_ns, uint32_t *err, bool skip) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = skip ? 0 : 1;  // fault injection: the block left without arriving
        volatile GridBarrier *vb = b;
        if (ok && !tk.released) {
            const uint64_t t0 = global_ns();
            while (vb->gen == tk.gen) {
                if (vb->abort) {
                    ok = 0;
                    break;
                }
                if ((int64_t)(global_ns() - t0) > timeout_ns) {
                    atomicOr(err, kErrTimeout);
                    atomicExch(&b->abort, 1u);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        if (vb->abort) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// One attempt on a fixed row of UD links (6: rows of six links; kEllRow: padded rows, col = -1
// entries skipped) split in two: prep_attempt takes everything that no other block writes
// during a class (caller id, parameters, the site's own spin, which only its own thread
// writes, the links, the Philox block and the trial), finish_attempt the neighbour spins
// (through L2), the field in row order and the decision. Together they compute what
// direct_attempt<2, 2, POL, 1, UD> computes, operation for operation.
template <int UD>
struct PrepU {
    uint32_t orig, wacc;
    Site32 p;
    float4 Si;
    int2 ed[UD > 0 ? UD : 1];
    float3 P;
};
template <int UD, int POL>
__device__ __forceinline__ void prep_attempt(const PassArgs &a, const int2 *E, int64_t e0, int g, int r, int R,
                                             uint32_t t, uint32_t inst, uint32_t k0, uint32_t k1, const float4 *S,
                                             PrepU<UD> &q) {
    q.orig = (uint32_t)__ldg(a.orig + g);
    q.p = Site32{a.u32.nx, a.u32.ny, a.u32.nz, a.u32.s, a.u32.ex, a.u32.ey, a.u32.ez, a.u32.k, a.u32.kc};
    if (a.params_mode == 2) q.p = site_params32(a, 2, g);
    q.Si = S[(int64_t)g * R + r];
#pragma unroll
    for (int k = 0; k < UD; ++k) q.ed[k] = __ldg(E + e0 + k);
    const uint4 rw = philox10(make_uint4(q.orig, t, inst, kPurposeTrial32), k0, k1);
    q.P = POL ? policy_trial32(a.pol32[g], 0.f, q.Si, q.p.sn, rw) : trial_random32(rw, q.p.sn);
    q.wacc = rw.z;
}
template <int UD>
__device__ __forceinline__ bool finish_attempt(const PrepU<UD> &q, int g, int r, int R, int lower_end, float beta,
                                               float B, float4 *S, Acc32 &acc, bool &nan_seen, float4 &Sq) {
    constexpr bool PAD = UD == kEllRow;
    float2 hxy = make_float2(0.f, 0.f), lxy = make_float2(0.f, 0.f);
    float hz = 0.f, lz = 0.f;
    float4 Sj[UD > 0 ? UD : 1];
#pragma unroll
    for (int k = 0; k < UD; ++k)
        if (!PAD || q.ed[k].x >= 0) Sj[k] = __ldcg(S + (int64_t)q.ed[k].x * R + r);
#pragma unroll
    for (int k = 0; k < UD; ++k)
        if (!PAD || q.ed[k].x >= 0)
            link32(Sj[k], __int_as_float(q.ed[k].y), q.ed[k].x < lower_end, hxy, hz, lxy, lz);
    float4 Sn;
    bool ok, bad;
    float e_i;
    attempt32<2, 2>(q.Si, hxy, hz, lxy, lz, q.p, beta, B, q.P, q.wacc, Sn, ok, e_i, bad);
    nan_seen |= bad;
    if (ok) S[(int64_t)g * R + r] = Sn;
    acc.add(e_i, Sn, ok);
    Sq = Sn;
    return ok;
}

// UD > 0: a sample whose every row has UD links (direct_attempt's uniform-degree path); UD =
// kEllRow: rows of at most kEllRow links read as fixed, padded rows (ca.ell).
template <int NT, int POL, int UD = 0>
__global__ void __launch_bounds__(NT) coop32_kernel(const CoopArgs ca) {
    const PassArgs &a = ca.pass;
    RunState *rs = a.run;
    const uint32_t t0 = rs->t, rec0 = rs->rec;
    const uint32_t step = rec0 / rs->mcs;
    const int R = 1 << a.log2R;
    float4 *S = (float4 *)a.spins;
    const int2 *E = (const int2 *)a.edges;
    const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
    const int64_t stride = (int64_t)gridDim.x * NT;
    const int64_t w0 = (int64_t)blockIdx.x * NT + threadIdx.x;
    const int r = (int)(w0 & (R - 1));  // fixed per thread (the stride is a multiple of 32 >= R)
    const uint32_t inst = (uint32_t)(a.inst0 + r);
    const double *sc = rs->sched + ((int64_t)step * a.n_inst + a.inst_local0 + r) * 2;
    const float beta = (float)sc[0], B = (float)sc[1];
    const bool skip = (int)blockIdx.x == ca.skip_block;
    bool nan_seen = false;
    // block 0 adds the block partials of MCS mm (buffer mm & 1) into the history: one warp per
    // replica, lanes striding over the blocks, a fixed tree
    auto record = [&](int mm) {
        if (blockIdx.x != 0) return;
        const double *part = ca.partial + (int64_t)(mm & 1) * gridDim.x * R * 4;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int rr = warp; rr < R; rr += NT / 32) {
            double v[4] = {0.0, 0.0, 0.0, 0.0};
            for (int b = lane; b < (int)gridDim.x; b += 32) {
                const double *p = part + ((int64_t)b * R + rr) * 4;
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] += p[q];
            }
            for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] += __shfl_xor_sync(0xFFFFFFFFu, v[q], off);
            }
            if (lane == 0) {
                double *h = rs->hist + ((int64_t)(rec0 + mm) * a.n_inst + a.inst_local0 + rr) * 4;
#pragma unroll
                for (int q = 0; q < 4; ++q) h[q] = v[q];
                if (rs->acc) {
                    const uint32_t n = rs->acc[a.inst_local0 + rr];
                    rs->acc[a.inst_local0 + rr] = 0;
                    if (rs->acc_hist) rs->acc_hist[(int64_t)(rec0 + mm) * a.n_inst + a.inst_local0 + rr] = n;
                }
            }
        }
    };
    // With two or more classes the record of MCS m is taken after the first class barrier of
    // MCS m + 1: every block wrote its partials and counts of MCS m before reaching it, and
    // none adds the counts of MCS m + 1 before the next barrier, which block 0 reaches only
    // after recording. That saves one grid barrier per MCS.
    const bool deferred = ca.n_colours >= 2;
    if (UD > 0 && deferred) {
        // Split-phase barriers: after arriving at the end of a class, a block prepares its
        // first attempt of the next class (prep_attempt) and only then waits. The MCS's partial sums
        // go out after its last wait, so every block adds the MCS's accepted counts only
        // after block 0 has recorded the previous MCS (which it does after the next class-0
        // wait, and before arriving at the class-1 barrier the other blocks then wait on).
        Acc32 acc;
        BarrierTicket tk{0u, false};
        bool pending = false;  // an arrival not yet waited for
        for (int m = 0; m < ca.mcs; ++m) {
            const uint32_t t = t0 + (uint32_t)m;
            const bool log_accepts = a.alog && t < a.alog_mcs;
            for (int c = 0; c < ca.n_colours; ++c) {
                const int cb = ca.cstart[c], ce = ca.cstart[c + 1];
                const int64_t n_work = (int64_t)(ce - cb) << a.log2R;
                const bool has = w0 < n_work;
                PrepU<UD> q;
                if (has) {
                    const int g = cb + (int)(w0 >> a.log2R);
                    prep_attempt<UD, POL>(a, UD == kEllRow ? ca.ell : E,
                                          UD == kEllRow ? (int64_t)g * kEllRow : a.edge_base + (int64_t)(g - a.site_off) * UD,
                                          g, r, R, t, inst, k0, k1, S, q);
                }
                if (pending) {
                    if (!grid_wait(ca.bar, tk, ca.timeout_ns, a.err, skip)) return;
                    pending = false;
                    if (c == 0) {  // MCS m - 1 is over everywhere: its partial sums
                        acc.flush();
                        block_partials(acc.d, acc.nacc, R,
                                       ca.partial + ((int64_t)((m - 1) & 1) * gridDim.x + blockIdx.x) * R * 4,
                                       acc_counters(rs, a.inst_local0));
                        acc = Acc32();
                    }
                    if (c == 1 && m > 0) record(m - 1);
                }
                if (has) {
                    const int g = cb + (int)(w0 >> a.log2R);
                    float4 Sq;
                    const bool ok = finish_attempt<UD>(q, g, r, R, cb, beta, B, S, acc, nan_seen, Sq);
                    if (log_accepts)
                        a.alog[(int64_t)t * a.alog_stride + a.alog_base + (int64_t)r * a.n_sample_sites + q.orig] =
                            ok ? 1 : 0;
                }
                for (int64_t w = w0 + stride; w < n_work; w += stride) {
                    const int g = cb + (int)(w >> a.log2R);
                    const uint32_t orig = (uint32_t)__ldg(a.orig + g);
                    Site32 p{a.u32.nx, a.u32.ny, a.u32.nz, a.u32.s, a.u32.ex, a.u32.ey, a.u32.ez, a.u32.k, a.u32.kc};
                    if (a.params_mode == 2) p = site_params32(a, 2, g);
                    float4 Sq;
                    const bool ok = direct_attempt<2, 2, POL, 1, UD>(
                        S, UD == kEllRow ? ca.ell : E, a.row_ptr, g, r, R, cb, orig, p, beta, B, t, inst, k0, k1, acc,
                        nan_seen, a.pol32, 0.f, Sq,
                        UD == kEllRow ? (int64_t)g * kEllRow : a.edge_base + (int64_t)(g - a.site_off) * UD);
                    if (log_accepts)
                        a.alog[(int64_t)t * a.alog_stride + a.alog_base + (int64_t)r * a.n_sample_sites + orig] = ok ? 1 : 0;
                }
                tk = grid_arrive(ca.bar, gridDim.x, skip);
                pending = true;
            }
        }
        if (pending) {
            if (!grid_wait(ca.bar, tk, ca.timeout_ns, a.err, skip)) return;
            acc.flush();
            block_partials(acc.d, acc.nacc, R, ca.partial + ((int64_t)((ca.mcs - 1) & 1) * gridDim.x + blockIdx.x) * R * 4,
                           acc_counters(rs, a.inst_local0));
            if (!grid_barrier(ca.bar, gridDim.x, ca.timeout_ns, a.err, skip)) return;
            record(ca.mcs - 1);
        }
        if (nan_seen) atomicOr(a.err, kErrNaN);
        return;
    }
    for (int m = 0; m < ca.mcs; ++m) {
        const uint32_t t = t0 + (uint32_t)m;
        const bool log_accepts = a.alog && t < a.alog_mcs;
        Acc32 acc;
        for (int c = 0; c < ca.n_colours; ++c) {
            const int cb = ca.cstart[c], ce = ca.cstart[c + 1];
            const int64_t n_work = (int64_t)(ce - cb) << a.log2R;
            for (int64_t w = w0; w < n_work; w += stride) {
                const int g = cb + (int)(w >> a.log2R);
                const uint32_t orig = (uint32_t)__ldg(a.orig + g);
                Site32 p{a.u32.nx, a.u32.ny, a.u32.nz, a.u32.s, a.u32.ex, a.u32.ey, a.u32.ez, a.u32.k, a.u32.kc};
                if (a.params_mode == 2) p = site_params32(a, 2, g);
                // one code path for every parameter mode (zero constants add signed zeros)
                float4 Sq;
                const bool ok = direct_attempt<2, 2, POL, 1, UD>(
                    S, UD == kEllRow ? ca.ell : E, a.row_ptr, g, r, R, cb, orig, p, beta, B, t, inst, k0, k1, acc,
                    nan_seen, a.pol32, 0.f, Sq,
                    UD == kEllRow ? (int64_t)g * kEllRow : a.edge_base + (int64_t)(g - a.site_off) * UD);
                if (log_accepts)
                    a.alog[(int64_t)t * a.alog_stride + a.alog_base + (int64_t)r * a.n_sample_sites + orig] = ok ? 1 : 0;
            }
            if (!grid_barrier(ca.bar, gridDim.x, ca.timeout_ns, a.err, skip)) return;
            if (deferred && c == 0 && m > 0) record(m - 1);
        }
        // per-MCS sums: block partials per replica into buffer m & 1
        acc.flush();
        block_partials(acc.d, acc.nacc, R, ca.partial + ((int64_t)(m & 1) * gridDim.x + blockIdx.x) * R * 4,
                       acc_counters(rs, a.inst_local0));
        if (!deferred) {
            if (!grid_barrier(ca.bar, gridDim.x, ca.timeout_ns, a.err, skip)) return;
            record(m);
        }
    }
    if (deferred && ca.mcs > 0) {
        if (!grid_barrier(ca.bar, gridDim.x, ca.timeout_ns, a.err, skip)) return;
        record(ca.mcs - 1);
    }
    if (nan_seen) atomicOr(a.err, kErrNaN);
}

// The cooperative sweep in FP64 (the attempt of pass64_kernel, so the oracle's spins bit for
// bit): blocks of NT threads, every block on every class, the same bounded grid barrier and
// deferred record as coop32_kernel. GB300 runs about two FP64 operations per SM and clock, so
// the host spreads a class over many SMs with small blocks (about one thread per site of the
// widest class) instead of filling a few.
template <int NT>
__global__ void __launch_bounds__(NT) coop64_kernel(const CoopArgs ca) {
    const PassArgs &a = ca.pass;
    RunState *rs = a.run;
    const uint32_t t0 = rs->t, rec0 = rs->rec;
    const uint32_t step = rec0 / rs->mcs;
    const int R = 1 << a.log2R;
    double4_32a *S = (double4_32a *)a.spins;
    const Edge64 *E = (const Edge64 *)a.edges;
    const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
    // lane l serves replica l mod R (as block_partials needs); site v of a class goes to block
    // v mod grid, so a class's sites spread over every block (over as many SMs' FP64 units as
    // the grid has blocks) before any block takes two
    const int r = (int)threadIdx.x & (R - 1);
    const int64_t v0 = (int64_t)(threadIdx.x >> a.log2R) * gridDim.x + blockIdx.x;
    const int64_t vstride = (int64_t)gridDim.x * (NT >> a.log2R);
    const bool skip = (int)blockIdx.x == ca.skip_block;
    // block 0 adds the block partials of MCS mm (buffer mm & 1) into the history: one warp per
    // replica, lanes striding over the blocks, a fixed tree
    auto record = [&](int mm) {
        if (blockIdx.x != 0) return;
        const double *part = ca.partial + (int64_t)(mm & 1) * gridDim.x * R * 4;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int rr = warp; rr < R; rr += NT / 32) {
            double v[4] = {0.0, 0.0, 0.0, 0.0};
            for (int b = lane; b < (int)gridDim.x; b += 32) {
                const double *p = part + ((int64_t)b * R + rr) * 4;
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] += __ldcg(p + q);
            }
            for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] += __shfl_xor_sync(0xFFFFFFFFu, v[q], off);
            }
            if (lane == 0) {
                double *h = rs->hist + ((int64_t)(rec0 + mm) * a.n_inst + a.inst_local0 + rr) * 4;
#pragma unroll
                for (int q = 0; q < 4; ++q) h[q] = v[q];
                if (rs->acc) {
                    const uint32_t n = atomicExch(rs->acc + a.inst_local0 + rr, 0u);
                    if (rs->acc_hist) rs->acc_hist[(int64_t)(rec0 + mm) * a.n_inst + a.inst_local0 + rr] = n;
                }
            }
        }
    };
    const bool deferred = ca.n_colours >= 2;
    for (int m = 0; m < ca.mcs; ++m) {
        const uint32_t t = t0 + (uint32_t)m;
        double acc4[4] = {0.0, 0.0, 0.0, 0.0};
        uint32_t nacc = 0;
        for (int c = 0; c < ca.n_colours; ++c) {
            const int cb = ca.cstart[c], ce = ca.cstart[c + 1];
            for (int64_t v = v0; v < ce - cb; v += vstride)
                site64<1>(a, cb + (int)v, r, R, t, step, 2, cb, S, E, k0, k1, acc4, nacc);
            if (!grid_barrier(ca.bar, gridDim.x, ca.timeout_ns, a.err, skip)) return;
            if (deferred && c == 0 && m > 0) record(m - 1);
        }
        block_partials(acc4, nacc, R, ca.partial + ((int64_t)(m & 1) * gridDim.x + blockIdx.x) * R * 4,
                       acc_counters(rs, a.inst_local0));
        if (!deferred) {
            if (!grid_barrier(ca.bar, gridDim.x, ca.timeout_ns, a.err, skip)) return;
            record(m);
        }
    }
    if (deferred && ca.mcs > 0) {
        if (!grid_barrier(ca.bar, gridDim.x, ca.timeout_ns, a.err, skip)) return;
        record(ca.mcs - 1);
    }
}

// ------------------------------------------------------------------ per-MCS reduction
// One block per instance sums its sample's block partials over every colour class in a fixed
// order (thread k takes slots k, k + 256, ... in turn, then a butterfly inside each warp and
// the warps in order) and appends the record; the last block to finish advances the MCS
// counter and the record index (no waiting: a ticket counter, not a barrier). Block 0 also
// zeroes the passes' block counters: every pass of this MCS has finished.
__global__ void __launch_bounds__(256) reduce_kernel(const ReduceArgs a) {
    __shared__ double red[8][4];
    RunState *rs = a.run;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int il = blockIdx.x;
    const uint32_t rec = rs->rec;
    if (blockIdx.x == 0 && a.tickets)
        for (int k = threadIdx.x; k < a.n_tickets; k += blockDim.x) a.tickets[k] = 0u;
    const int s = il / a.R, r = il % a.R;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = 0; k < a.n_groups; ++k) {  // type groups in order, then their total
        const int64_t base = a.slot_base[s * a.n_groups + k];
        const int32_t cnt = a.slot_count[s * a.n_groups + k];
        double u[4] = {0.0, 0.0, 0.0, 0.0};
        for (int32_t j = threadIdx.x; j < cnt; j += blockDim.x) {
            const double4_32a p = *(const double4_32a *)(a.partial + ((base + j) * a.R + r) * 4);
            u[0] += p.x;
            u[1] += p.y;
            u[2] += p.z;
            u[3] += p.w;
        }
        for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
            for (int q = 0; q < 4; ++q) u[q] += __shfl_xor_sync(0xFFFFFFFFu, u[q], off);
        }
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < 4; ++q) red[warp][q] = u[q];
        __syncthreads();
        if (threadIdx.x == 0) {
            double t4[4] = {0.0, 0.0, 0.0, 0.0};
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
#pragma unroll
                for (int q = 0; q < 4; ++q) t4[q] += red[w][q];
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] += t4[q];
            if (a.n_types > 0 && rs->type_hist) {
                double *th = rs->type_hist + (((int64_t)rec * a.n_inst + il) * a.n_types + k) * 3;
#pragma unroll
                for (int c = 0; c < 3; ++c) th[c] = t4[c + 1];
            }
        }
        __syncthreads();  // red is reused by the next group
    }
    if (threadIdx.x == 0) {
        double *h = rs->hist + ((int64_t)rec * a.n_inst + il) * 4;
#pragma unroll
        for (int q = 0; q < 4; ++q) h[q] = v[q];
        if (rs->acc) {  // accepted attempts of this MCS; the adaptive width follows them
            const uint32_t n = rs->acc[il];
            rs->acc[il] = 0;
            if (rs->acc_hist) rs->acc_hist[(int64_t)rec * a.n_inst + il] = n;
            if (a.adapt_n && a.adapt_n[il] > 0 && rs->sigma && rec % rs->mcs < rs->mcs / 5)
                rs->sigma[il] = adapt_width(rs->sigma[il], n, a.adapt_n[il]);
        }
        __threadfence();
        const uint32_t done = atomicAdd(&rs->ticket, 1u);
        if (done == gridDim.x - 1) {
            rs->ticket = 0;
            rs->t = rs->t + 1;
            rs->rec = rec + 1;
            __threadfence();
        }
    }
}

// ------------------------------------------------------------------ renormalisation
// S_i <- s_i S_i / |S_i| with FP64 arithmetic (the FP64 form matches the oracle's
// f = s / sqrt((x^2 + y^2) + z^2), then x f, y f, z f).
__global__ void renorm64_kernel(const RenormArgs a) {
    double4_32a *S = (double4_32a *)a.spins;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < a.n_work; w += (int64_t)gridDim.x * blockDim.x) {
        if (a.qis && a.qis[w >> a.log2R]) continue;  // discrete values keep their length
        const double4_32a v = S[w];
        const double n2 = da(da(dm(v.x, v.x), dm(v.y, v.y)), dm(v.z, v.z));
        const double f = __ddiv_rn(a.norm[w >> a.log2R], __dsqrt_rn(n2));
        S[w] = make_double4_32a(dm(v.x, f), dm(v.y, f), dm(v.z, f), 0.0);
    }
}

// FP32 spins (renorm_spin32): in the common case (s = 1 and |S|^2 within 2^-16 of 1, which
// every spin drawn or kept by a Metropolis step is: |u| ~ 1e-7) no FP64 operation at all.
// u = |S|^2 - 1 comes from FP32 products and sums with their exact errors, within 2^-44 of
// the exact value; 1/sqrt(1 + u) - 1 = -u/2 + 3u^2/8 - (5/16) u^3 + ..., and S' = S + S d with
// d the first two terms in FP32, one FMA per component. d is off by at most (5/16)|u|^3 +
// 2^-24 |u| + 2^-45, so S + S d is within 5e-13 |S| of S s/|S| at |u| = 2^-16 and within
// 5e-14 |S| at the usual |u| ~ 1e-7: it rounds to the same float as the exact product unless
// that product lies that close to a rounding boundary (half a float ulp is 3e-8 |S|). Other
// spins take the FP64 formula s / sqrt(|S|^2).
__global__ void renorm32_kernel(const RenormArgs a) {
    float4 *S = (float4 *)a.spins;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < a.n_work; w += (int64_t)gridDim.x * blockDim.x) {
        if (a.qis && a.qis[w >> a.log2R]) continue;  // discrete values keep their length
        S[w] = renorm_spin32(S[w], a.norm[w >> a.log2R]);
    }
}

// ------------------------------------------------------------------ initial state
// S_i = s_i * sphere(counter = (caller id, 0xFFFFFFFF, instance, 0x20000|k)), in FP64 for
// both precisions (FP32 contexts round it), or the caller's state.
template <typename V>
__global__ void init_kernel(const InitArgs a) {
    V *S = (V *)a.spins;
    const int R = 1 << a.log2R;
    const int64_t n_work = (int64_t)(a.g_end - a.g_begin) << a.log2R;
    const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n_work; w += (int64_t)gridDim.x * blockDim.x) {
        const int g = a.g_begin + (int)(w >> a.log2R);
        const int r = (int)(w & (R - 1));
        double x, y, z;
        if (a.given) {
            const double *p = a.given + (int64_t)(g - a.g_begin) * 3;
            x = p[0];
            y = p[1];
            z = p[2];
        } else if (a.qis && a.qis[g]) {  // qIsing: a uniform value of {-s, ..., s} along z
            const double s = a.norm[g];
            const int nv = (int)dm(2.0, s) + 1;
            const uint4 wq = philox10(make_uint4((uint32_t)a.orig[g], kInitT, (uint32_t)(a.inst0 + r), kPurposeInit), k0, k1);
            int k = (int)dm(u53(wq.x, wq.y), (double)nv);
            if (k >= nv) k = nv - 1;
            x = 0.0;
            y = 0.0;
            z = ds((double)k, s);
        } else {
            const double s = a.norm[g];
            const double3 u = sphere64((uint32_t)a.orig[g], kInitT, (uint32_t)(a.inst0 + r), kPurposeInit, k0, k1, a.err);
            x = dm(s, u.x);
            y = dm(s, u.y);
            z = dm(s, u.z);
        }
        V v;
        v.x = x;
        v.y = y;
        v.z = z;
        v.w = 0;
        S[(int64_t)g * R + r] = v;
    }
}

// ------------------------------------------------------------------ gather / scatter
__global__ void gather_kernel(const void *spins, int precision, int64_t site_off, int64_t n, int32_t log2R, int32_t r,
                              double *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t w = ((site_off + i) << log2R) + r;
        if (precision == 64) {
            const double4_32a v = ((const double4_32a *)spins)[w];
            out[3 * i] = v.x;
            out[3 * i + 1] = v.y;
            out[3 * i + 2] = v.z;
        } else {
            const float4 v = ((const float4 *)spins)[w];
            out[3 * i] = v.x;
            out[3 * i + 1] = v.y;
            out[3 * i + 2] = v.z;
        }
    }
}

__global__ void scatter_kernel(void *spins, int precision, int64_t site_off, int64_t n, int32_t log2R, int32_t r,
                               const double *in) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t w = ((site_off + i) << log2R) + r;
        if (precision == 64)
            ((double4_32a *)spins)[w] = make_double4_32a(in[3 * i], in[3 * i + 1], in[3 * i + 2], 0.0);
        else
            ((float4 *)spins)[w] = make_float4((float)in[3 * i], (float)in[3 * i + 1], (float)in[3 * i + 2], 0.f);
    }
}

}  // namespace

// Direct FP32 sweep kernel for a parameter mode, lower mode and policy flag.
PassFn select_direct(int pm, int lm, bool pol) {
    static const PassFn tab[2][3][3] = {
        {
            {pass32_kernel<0, 0, 0>, pass32_kernel<0, 1, 0>, pass32_kernel<0, 2, 0>},
            {pass32_kernel<1, 0, 0>, pass32_kernel<1, 1, 0>, pass32_kernel<1, 2, 0>},
            {pass32_kernel<2, 0, 0>, pass32_kernel<2, 1, 0>, pass32_kernel<2, 2, 0>},
        },
        {
            {pass32_kernel<0, 0, 1>, pass32_kernel<0, 1, 1>, pass32_kernel<0, 2, 1>},
            {pass32_kernel<1, 0, 1>, pass32_kernel<1, 1, 1>, pass32_kernel<1, 2, 1>},
            {pass32_kernel<2, 0, 1>, pass32_kernel<2, 1, 1>, pass32_kernel<2, 2, 1>},
        },
    };
    return tab[pol ? 1 : 0][pm][lm];
}

using MultiFn = void (*)(const PassArgs *, const int32_t *, int32_t);

void launch_pass32_multi(const PassArgs &key, const PassArgs *passes, const int32_t *first, int32_t n, int grid,
                         void *stream) {
    static const MultiFn tab[2][3][3] = {
        {
            {pass32_multi_kernel<0, 0, 0>, pass32_multi_kernel<0, 1, 0>, pass32_multi_kernel<0, 2, 0>},
            {pass32_multi_kernel<1, 0, 0>, pass32_multi_kernel<1, 1, 0>, pass32_multi_kernel<1, 2, 0>},
            {pass32_multi_kernel<2, 0, 0>, pass32_multi_kernel<2, 1, 0>, pass32_multi_kernel<2, 2, 0>},
        },
        {
            {pass32_multi_kernel<0, 0, 1>, pass32_multi_kernel<0, 1, 1>, pass32_multi_kernel<0, 2, 1>},
            {pass32_multi_kernel<1, 0, 1>, pass32_multi_kernel<1, 1, 1>, pass32_multi_kernel<1, 2, 1>},
            {pass32_multi_kernel<2, 0, 1>, pass32_multi_kernel<2, 1, 1>, pass32_multi_kernel<2, 2, 1>},
        },
    };
    tab[key.pol32 ? 1 : 0][key.params_mode][key.lower_mode]<<<grid, kThreads, 0, (cudaStream_t)stream>>>(passes, first,
                                                                                                            n);
}

void launch_pass32(const PassArgs &a, int grid, void *stream) {
    select_pass32(a)<<<grid, pass32_threads(a), pass32_smem(a), (cudaStream_t)stream>>>(a);
}

void launch_pass64(const PassArgs &a, int grid, int threads, void *stream) {
    pass64_kernel<<<grid, threads, 0, (cudaStream_t)stream>>>(a);
}

void launch_reduce(const ReduceArgs &a, void *stream) {
    reduce_kernel<<<a.n_inst, 256, 0, (cudaStream_t)stream>>>(a);
}

void launch_renorm32(const RenormArgs &a, int grid, void *stream) {
    renorm32_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(a);
}

void launch_renorm64(const RenormArgs &a, int grid, void *stream) {
    renorm64_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(a);
}

void launch_init32(const InitArgs &a, int grid, void *stream) {
    init_kernel<float4><<<grid, 256, 0, (cudaStream_t)stream>>>(a);
}

void launch_init64(const InitArgs &a, int grid, void *stream) {
    init_kernel<double4_32a><<<grid, 256, 0, (cudaStream_t)stream>>>(a);
}

void launch_gather(void *spins, int precision, int64_t site_off, int64_t n, int32_t log2R, int32_t r, double *out3,
                   int grid, void *stream) {
    gather_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(spins, precision, site_off, n, log2R, r, out3);
}

void launch_scatter(void *spins, int precision, int64_t site_off, int64_t n, int32_t log2R, int32_t r,
                    const double *in3, int grid, void *stream) {
    scatter_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(spins, precision, site_off, n, log2R, r, in3);
}

__global__ void advance_kernel(RunState *run, int32_t n) {
    run->t += (uint32_t)n;
    run->rec += (uint32_t)n;
}

void launch_advance(RunState *run, int32_t n, void *stream) { advance_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(run, n); }

// Runs after a step's last MCS and renormalisation inside the run graph: another step while
// records are left in the run.
__global__ void run_ctrl_kernel(const RunState *run, cudaGraphConditionalHandle loop) {
    cudaGraphSetConditional(loop, run->rec < run->rec_end ? 1u : 0u);
}

void launch_run_ctrl(const RunState *run, unsigned long long loop_handle, void *stream) {
    run_ctrl_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(run, (cudaGraphConditionalHandle)loop_handle);
}

// Copies the spins (n16 16-byte words) into slot (rec / mcs - 1) of the snapshot buffer: the
// step whose last MCS and renormalisation just ran.
__global__ void snapshot_kernel(const uint4 *spins, uint4 *snap, int64_t n16, const RunState *run) {
    const int64_t step = (int64_t)(run->rec / run->mcs) - 1;
    uint4 *dst = snap + step * n16;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n16; w += (int64_t)gridDim.x * blockDim.x)
        dst[w] = spins[w];
}

void launch_snapshot(const void *spins, void *snap, int64_t n16, const RunState *run, int grid, void *stream) {
    snapshot_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>((const uint4 *)spins, (uint4 *)snap, n16, run);
}


using CoopFn = void (*)(CoopArgs);

// rows of six links (the simple cubic lattices) take the uniform-degree form, other rows of at
// most kEllRow links the padded fixed rows when the host built them (form = kEllRow)
CoopFn select_coop(bool pol, int form) {
    if (form == 6) return pol ? coop32_kernel<kCoopThreads, 1, 6> : coop32_kernel<kCoopThreads, 0, 6>;
    if (form == kEllRow) return pol ? coop32_kernel<kCoopThreads, 1, kEllRow> : coop32_kernel<kCoopThreads, 0, kEllRow>;
    return pol ? coop32_kernel<kCoopThreads, 1> : coop32_kernel<kCoopThreads, 0>;
}

int launch_coop(const CoopArgs &a, int grid, void *stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kCoopThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = (cudaStream_t)stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (a.fp64) {
        cfg.blockDim = dim3(kCoop64Threads);
        return (int)cudaLaunchKernelEx(&cfg, coop64_kernel<kCoop64Threads>, a);
    }
    return (int)cudaLaunchKernelEx(&cfg, select_coop(a.pass.pol32 != nullptr, a.pass.deg == 6 ? 6 : (a.ell ? kEllRow : 0)),
                                   a);
}

int coop_blocks_per_sm(bool pol, int form, bool fp64) {
    int nb = 0;
    if (fp64)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, coop64_kernel<kCoop64Threads>, kCoop64Threads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, select_coop(pol, form), kCoopThreads, 0);
    return nb > 0 ? nb : 1;
}

using ResFn = void (*)(ResidentArgs);

// Spins in global memory: 256 or 512 threads; in shared memory (smem = 1): 512 (1024 threads
// would leave 64 registers per thread and spill).
ResFn select_resident(int threads, bool pol, bool smem, bool aniso = true) {
    if (smem && !aniso) return pol ? resident32_kernel<512, 1, 1, 0> : resident32_kernel<512, 0, 1, 0>;
    if (smem) return pol ? resident32_kernel<512, 1, 1> : resident32_kernel<512, 0, 1>;
    if (threads >= 512) return pol ? resident32_kernel<512, 1> : resident32_kernel<512, 0>;
    return pol ? resident32_kernel<256, 1> : resident32_kernel<256, 0>;
}

int resident_threads(int threads, bool smem) {
    if (smem) return 512;
    return threads >= 512 ? 512 : 256;
}

// Dynamic shared memory of the resident sweep: three floats per site of the largest region
// (a whole-block instance, or all groups' regions together).
size_t resident_smem_bytes(const ResidentArgs &a, int threads) {
    if (a.smem_sites <= 0) return 0;
    const int nt = resident_threads(threads, true);
    const int ng = a.group_threads > 0 && a.group_threads < nt ? nt / a.group_threads : 1;
    // groups' regions start at even site counts (sm_spin's pairs stay 8-byte aligned)
    const int64_t sites = std::max<int64_t>(a.smem_sites, ng > 1 ? (int64_t)ng * ((a.group_sites + 1) & ~1) : 0);
    return (size_t)sites * 3 * sizeof(float);
}

void launch_resident(const ResidentArgs &a, int grid, int threads, void *stream) {
    const bool smem = a.smem_sites > 0;
    const int nt = resident_threads(threads, smem);
    select_resident(nt, a.pol != nullptr, smem, a.any_aniso != 0)<<<grid, nt, resident_smem_bytes(a, threads),
                                                                     (cudaStream_t)stream>>>(a);
}

using ClusterFn = void (*)(ResidentArgs);

ClusterFn select_cluster(int threads, bool pol, bool smem) {
    if (smem) {
        if (threads >= 512) return pol ? cluster32_kernel<512, 1, 1> : cluster32_kernel<512, 0, 1>;
        return pol ? cluster32_kernel<256, 1, 1> : cluster32_kernel<256, 0, 1>;
    }
    if (threads >= 512) return pol ? cluster32_kernel<512, 1> : cluster32_kernel<512, 0>;
    return pol ? cluster32_kernel<256, 1> : cluster32_kernel<256, 0>;
}

// Dynamic shared memory of the cluster sweep with spins in shared memory: a copy of the
// largest instance per block, or the groups' regions of its single-block phase.
size_t cluster_smem_bytes(const ResidentArgs &a, int threads) {
    if (a.smem_sites <= 0) return 0;
    const int nt = threads >= 512 ? 512 : 256;
    const int ng = a.group_threads > 0 && a.group_threads < nt ? nt / a.group_threads : 1;
    // groups' regions start at even site counts (sm_spin's pairs stay 8-byte aligned)
    const int64_t sites = std::max<int64_t>(a.smem_sites, ng > 1 ? (int64_t)ng * ((a.group_sites + 1) & ~1) : 0);
    return (size_t)sites * 3 * sizeof(float);
}

int launch_cluster(const ResidentArgs &a, int n_clusters, int cs, int threads, void *stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_clusters * cs);
    cfg.blockDim = dim3(threads >= 512 ? 512 : 256);
    cfg.dynamicSmemBytes = cluster_smem_bytes(a, threads);
    cfg.stream = (cudaStream_t)stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return (int)cudaLaunchKernelEx(&cfg, select_cluster(threads, a.pol != nullptr, a.smem_sites > 0), a);
}

int cluster_capacity(int cs, int threads, bool pol, size_t smem_bytes) {
    ClusterFn k = select_cluster(threads, pol, smem_bytes > 0);
    if (cs > 8 && cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) return 0;
    if (smem_bytes > 0 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes) != cudaSuccess)
        return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(threads >= 512 ? 512 : 256);
    cfg.dynamicSmemBytes = smem_bytes;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) return 0;
    return n;
}

int resident_blocks_per_sm(int threads, bool pol, size_t smem_bytes) {
    int nb = 0;
    const bool smem = smem_bytes > 0;
    const int nt = resident_threads(threads, smem);
    const ResFn k = select_resident(nt, pol, smem);
    if (smem && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes) != cudaSuccess)
        return 0;
    // the form without anisotropy terms takes the same shared memory
    if (smem && cudaFuncSetAttribute(select_resident(nt, pol, smem, false), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem_bytes) != cudaSuccess)
        return 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, nt, smem_bytes);
    return nb > 0 ? nb : (smem ? 0 : 1);
}

int pass_blocks_per_sm(int precision, const PassArgs &a) {
    int nb = 0;
    if (precision == 64)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pass64_kernel, kThreads, 0);
    else {
        const int sm = pass32_smem(a);
        if (sm > 0) cudaFuncSetAttribute(select_pass32(a), cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, select_pass32(a), pass32_threads(a), sm);
    }
    return nb > 0 ? nb : 1;
}

}  // namespace vegas
