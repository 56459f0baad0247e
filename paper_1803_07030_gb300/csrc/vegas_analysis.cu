// Analysis of a simulation history on the GPU: thermal averages with binned and jackknife
// errors, the Binder cumulant and the cumulants V1, V2, integrated autocorrelation times
// (Sec. II, Sec. IV.A-B), and single/multiple histogram reweighting (Sec. IV.E; Ferrenberg
// & Swendsen 1988, 1989). FP64 throughout; every sum is a fixed-order block reduction, so
// results do not change between runs.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "vegas_internal.h"

using namespace vegas;

namespace {

constexpr int kAnaThreads = 256;
constexpr int kMaxObs = 8;  // observables per reweighting call

thread_local std::string g_ana_err;

vegas_status ana_fail(vegas_status st, const std::string &m) {
    g_ana_err = m;
    return st;
}

// A host exception caught at an entry point, as a status (called inside a catch block).
vegas_status analysis_host_exception() {
    std::string m;
    const vegas_status st = status_of_current_exception(m);
    return ana_fail(st, m);
}

// Sum of v over the block, in a fixed order; every thread gets the result.
__device__ double block_sum(double v, double *sm) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();  // sm may still be read by the previous call
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sm[w];
    return s;
}

// Sums over records [i0, i1) of one series: the eight shifted moments
//   e' = E - Eref, a' = |M| - Aref:  e', e'^2, a', a'^2, a' e', M^2, M^4, M^2 e'.
__device__ void moment_sums(const double *h, int64_t i0, int64_t i1, double Eref, double Aref, double *sm,
                            double out[8]) {
    double v[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const double *r = h + i * 4;
        const double m2 = r[1] * r[1] + r[2] * r[2] + r[3] * r[3];
        const double e = r[0] - Eref, a = sqrt(m2) - Aref;
        v[0] += e;
        v[1] += e * e;
        v[2] += a;
        v[3] += a * a;
        v[4] += a * e;
        v[5] += m2;
        v[6] += m2 * m2;
        v[7] += m2 * e;
    }
    for (int q = 0; q < 8; ++q) out[q] = block_sum(v[q], sm);
}

// (c, chi, u4) from moment sums over n samples.
__device__ void estimates(const double S[8], double n, double N, double T, double out[3]) {
    const double me = S[0] / n, ma = S[2] / n, m2 = S[5] / n;
    out[0] = (S[1] / n - me * me) / (N * T * T);
    out[1] = (S[3] / n - ma * ma) / (N * T);
    out[2] = 1.0 - (S[6] / n) / (3.0 * m2 * m2);
}

// Integrated autocorrelation time of x_i = (E or |M|) - mean, Sokal's window (c = 6).
__device__ double tau_window(const double *h, int64_t cut, int64_t n, int which, double mean, double *sm) {
    auto x = [&](int64_t i) {
        const double *r = h + (cut + i) * 4;
        return (which == 0 ? r[0] : sqrt(r[1] * r[1] + r[2] * r[2] + r[3] * r[3])) - mean;
    };
    double c0 = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double d = x(i);
        c0 += d * d;
    }
    c0 = block_sum(c0, sm) / (double)n;
    if (c0 == 0.0) return 0.5;
    double tau = 0.5;
    for (int64_t t = 1; t <= n / 2; ++t) {
        double c = 0.0;
        for (int64_t i = threadIdx.x; i < n - t; i += blockDim.x) c += x(i) * x(i + t);
        c = block_sum(c, sm) / (double)(n - t);
        tau += c / c0;
        if ((double)t >= 6.0 * tau) break;
    }
    return tau;
}

// One block per series: point estimates over all records after the cut, errors from n_bins
// equal bins over the first b * n_bins of them.
__global__ void __launch_bounds__(kAnaThreads) thermal_kernel(const double *series, int64_t len, int64_t cut,
                                                              int32_t n_bins, const double *T, const double *Nsites,
                                                              double *out) {
    __shared__ double sm[kAnaThreads / 32];
    __shared__ double s_bin[64][8];  // n_bins <= 64
    const int64_t sid = blockIdx.x;
    const double *h = series + sid * len * 4;
    const int64_t n = len - cut;
    const double Tt = T[sid], N = Nsites[sid];
    // reference shifts: the plain means of E and |M|
    double s0 = 0.0, s1 = 0.0;
    for (int64_t i = cut + threadIdx.x; i < len; i += blockDim.x) {
        const double *r = h + i * 4;
        s0 += r[0];
        s1 += sqrt(r[1] * r[1] + r[2] * r[2] + r[3] * r[3]);
    }
    const double Eref = block_sum(s0, sm) / (double)n;
    const double Aref = block_sum(s1, sm) / (double)n;
    double S[8];
    moment_sums(h, cut, len, Eref, Aref, sm, S);
    const int64_t b = n / n_bins;
    for (int k = 0; k < n_bins; ++k) {
        double Sk[8];
        moment_sums(h, cut + k * b, cut + (k + 1) * b, Eref, Aref, sm, Sk);
        if (threadIdx.x == 0)
            for (int q = 0; q < 8; ++q) s_bin[k][q] = Sk[q];
    }
    const double dn = (double)n;
    const double meanE = Eref + S[0] / dn, meanA = Aref + S[2] / dn, meanM2 = S[5] / dn;
    const double tau_e = tau_window(h, cut, n, 0, meanE, sm);
    const double tau_m = tau_window(h, cut, n, 1, meanA, sm);
    if (threadIdx.x != 0) return;
    double est[3];
    estimates(S, dn, N, Tt, est);
    const double covAE = S[4] / dn - (S[2] / dn) * (S[0] / dn);
    const double covM2E = S[7] / dn - meanM2 * (S[0] / dn);
    // the bin means' spread, and leave-one-bin-out (jackknife) estimates
    const double nb = (double)n_bins;
    double Tot[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    double mbe = 0.0, mba = 0.0;
    for (int k = 0; k < n_bins; ++k) {
        for (int q = 0; q < 8; ++q) Tot[q] += s_bin[k][q];
        mbe += s_bin[k][0] / (double)b;
        mba += s_bin[k][2] / (double)b;
    }
    mbe /= nb;
    mba /= nb;
    double vbe = 0.0, vba = 0.0;
    for (int k = 0; k < n_bins; ++k) {
        const double de = s_bin[k][0] / (double)b - mbe, da = s_bin[k][2] / (double)b - mba;
        vbe += de * de;
        vba += da * da;
    }
    const double e_err = sqrt(vbe / (nb - 1.0)) / sqrt(nb) / N;
    const double m_err = sqrt(vba / (nb - 1.0)) / sqrt(nb) / N;
    double jm[3] = {0.0, 0.0, 0.0}, jv[3] = {0.0, 0.0, 0.0};
    const double nj = (double)((n_bins - 1) * b);
    for (int pass = 0; pass < 2; ++pass)  // mean of the jackknife estimates, then their spread
        for (int k = 0; k < n_bins; ++k) {
            double R[8], jk[3];
            for (int q = 0; q < 8; ++q) R[q] = Tot[q] - s_bin[k][q];
            estimates(R, nj, N, Tt, jk);  // shift-invariant forms: the sample's own means enter
            for (int q = 0; q < 3; ++q) {
                if (pass == 0)
                    jm[q] += jk[q] / nb;
                else
                    jv[q] += (jk[q] - jm[q]) * (jk[q] - jm[q]);
            }
        }
    double *o = out + sid * VEGAS_AVG_FIELDS;
    o[0] = meanE / N;
    o[1] = e_err;
    o[2] = meanA / N;
    o[3] = m_err;
    o[4] = est[0];
    o[5] = sqrt((nb - 1.0) / nb * jv[0]);
    o[6] = est[1];
    o[7] = sqrt((nb - 1.0) / nb * jv[1]);
    o[8] = est[2];
    o[9] = sqrt((nb - 1.0) / nb * jv[2]);
    o[10] = -covAE / meanA;
    o[11] = -covM2E / meanM2;
    o[12] = tau_e;
    o[13] = tau_m;
    o[14] = dn;
    o[15] = nb;
}

// ------------------------------------------------------------------ reweighting
// D_i = ln sum_j n exp(-beta_j E_i - g_j) for every sample i.
__global__ void denom_kernel(const double *E, int64_t n_tot, const double *beta, const double *g, int32_t K,
                             double logn, double *D) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_tot; i += (int64_t)gridDim.x * blockDim.x) {
        const double e = E[i];
        double m = -INFINITY;
        for (int j = 0; j < K; ++j) m = fmax(m, -beta[j] * e - g[j]);
        double s = 0.0;
        for (int j = 0; j < K; ++j) s += exp(-beta[j] * e - g[j] - m);
        D[i] = logn + m + log(s);
    }
}

// Partial log-sum-exp of x_i = -beta E_i - D_i (and the x-weighted observables) per block:
// (max, sum of exp(x - max), sums of O exp(x - max)).
__global__ void __launch_bounds__(kAnaThreads) lse_kernel(const double *E, const double *D, const double *O,
                                                          int32_t n_obs, int64_t n_tot, const double *betas,
                                                          double *part) {
    __shared__ double sm[kAnaThreads / 32];
    const double beta = betas[blockIdx.y];
    const int64_t chunk = (n_tot + gridDim.x - 1) / gridDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * chunk, i1 = min(n_tot, i0 + chunk);
    double m = -INFINITY;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) m = fmax(m, -beta * E[i] - D[i]);
    // block max (fixed order)
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xFFFFFFFFu, m, off));
    __shared__ double smax[kAnaThreads / 32];
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = m;
    __syncthreads();
    double M = -INFINITY;
    for (int w = 0; w < kAnaThreads / 32; ++w) M = fmax(M, smax[w]);
    double s = 0.0, so[kMaxObs];
    for (int q = 0; q < kMaxObs; ++q) so[q] = 0.0;
    if (M > -INFINITY) {
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            const double w = exp(-beta * E[i] - D[i] - M);
            s += w;
            for (int q = 0; q < n_obs; ++q) so[q] += w * O[i * n_obs + q];
        }
    }
    double *p = part + ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * (2 + kMaxObs);
    const double ts = block_sum(s, sm);
    double to[kMaxObs];
    for (int q = 0; q < n_obs; ++q) to[q] = block_sum(so[q], sm);
    if (threadIdx.x == 0) {
        p[0] = M;
        p[1] = ts;
        for (int q = 0; q < n_obs; ++q) p[2 + q] = to[q];
    }
}

// Combines the per-block partials of each row y in block order: lse[y] = M + ln S and, when
// obs is not NULL, obs[y][q] = sum O exp(x) / sum exp(x).
__global__ void combine_kernel(const double *part, int32_t n_parts, int32_t n_rows, int32_t n_obs, double *lse,
                               double *obs) {
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= n_rows) return;
    const double *p = part + (int64_t)y * n_parts * (2 + kMaxObs);
    double M = -INFINITY;
    for (int b = 0; b < n_parts; ++b) M = fmax(M, p[b * (2 + kMaxObs)]);
    double s = 0.0, so[kMaxObs];
    for (int q = 0; q < kMaxObs; ++q) so[q] = 0.0;
    for (int b = 0; b < n_parts; ++b) {
        const double *pb = p + b * (2 + kMaxObs);
        if (pb[0] == -INFINITY) continue;
        const double f = exp(pb[0] - M);
        s += pb[1] * f;
        for (int q = 0; q < n_obs; ++q) so[q] += pb[2 + q] * f;
    }
    lse[y] = M + log(s);
    if (obs)
        for (int q = 0; q < n_obs; ++q) obs[(int64_t)y * n_obs + q] = so[q] / s;
}

struct DevBuf {
    std::vector<void *> ptrs;
    ~DevBuf() {
        for (void *p : ptrs) cudaFree(p);
    }
    template <typename T>
    cudaError_t alloc(T **p, size_t bytes) {
        cudaError_t e = cudaMalloc((void **)p, bytes > 0 ? bytes : 8);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
};

#define ACK(call)                                                                                        \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess)                                                                           \
            return ana_fail(e_ == cudaErrorMemoryAllocation ? VEGAS_ENOMEM : VEGAS_ECUDA,                \
                            std::string(#call) + ": " + cudaGetErrorString(e_));                         \
    } while (0)

vegas_status have_device() {
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) return ana_fail(VEGAS_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    return VEGAS_OK;
}

}  // namespace

extern "C" const char *vegas_analysis_last_error(void) { return g_ana_err.c_str(); }

extern "C" vegas_status vegas_thermal_averages(const double *series, int64_t n_series, int64_t len, int64_t cut,
                                               int32_t n_bins, const double *T, const double *n_sites, double *out,
                                               void *cuda_stream) {
    try {
        if (!series || !T || !n_sites || !out) return ana_fail(VEGAS_EINVAL, "a required pointer is NULL");
        if (n_series < 1 || len < 1 || cut < 0 || cut >= len) return ana_fail(VEGAS_EINVAL, "need n_series >= 1 and 0 <= cut < len");
        if (n_bins < 2 || n_bins > 64) return ana_fail(VEGAS_EINVAL, "n_bins must be in [2, 64]");
        if ((len - cut) / n_bins < 1) return ana_fail(VEGAS_EINVAL, "fewer records after the cut than bins");
        if (n_series > INT32_MAX) return ana_fail(VEGAS_EINVAL, "too many series");
        for (int64_t s = 0; s < n_series; ++s)
            if (!(T[s] > 0.0) || !std::isfinite(T[s]) || !(n_sites[s] > 0.0))
                return ana_fail(VEGAS_EINVAL, "T and n_sites must be finite and > 0");
        vegas_status st = have_device();
        if (st != VEGAS_OK) return st;
        cudaStream_t stream = (cudaStream_t)cuda_stream;
        DevBuf b;
        double *d_h, *d_T, *d_N, *d_out;
        const size_t hb = sizeof(double) * 4 * (size_t)n_series * (size_t)len;
        ACK(b.alloc(&d_h, hb));
        ACK(b.alloc(&d_T, sizeof(double) * n_series));
        ACK(b.alloc(&d_N, sizeof(double) * n_series));
        ACK(b.alloc(&d_out, sizeof(double) * VEGAS_AVG_FIELDS * n_series));
        ACK(cudaMemcpyAsync(d_h, series, hb, cudaMemcpyHostToDevice, stream));
        ACK(cudaMemcpyAsync(d_T, T, sizeof(double) * n_series, cudaMemcpyHostToDevice, stream));
        ACK(cudaMemcpyAsync(d_N, n_sites, sizeof(double) * n_series, cudaMemcpyHostToDevice, stream));
        thermal_kernel<<<(unsigned)n_series, kAnaThreads, 0, stream>>>(d_h, len, cut, n_bins, d_T, d_N, d_out);
        ACK(cudaGetLastError());
        ACK(cudaMemcpyAsync(out, d_out, sizeof(double) * VEGAS_AVG_FIELDS * n_series, cudaMemcpyDeviceToHost, stream));
        ACK(cudaStreamSynchronize(stream));
        return VEGAS_OK;
    } catch (...) {
        return analysis_host_exception();
    }
}

extern "C" vegas_status vegas_reweight(const double *E, const double *O, int32_t K, int64_t n, int32_t n_obs,
                                       const double *betas_k, const double *betas_out, int32_t n_out,
                                       int32_t max_iter, double tol, double *out, double *g_out, int32_t *iters_out,
                                       void *cuda_stream) {
    try {
        if (!E || !betas_k || (n_out > 0 && (!betas_out || !out)) || (n_obs > 0 && !O))
            return ana_fail(VEGAS_EINVAL, "a required pointer is NULL");
        if (K < 1 || n < 1 || n_obs < 0 || n_obs > kMaxObs || n_out < 0 || max_iter < 1 || !(tol > 0.0))
            return ana_fail(VEGAS_EINVAL, "need K >= 1, n >= 1, 0 <= n_obs <= 8, n_out >= 0, max_iter >= 1, tol > 0");
        const int64_t n_tot = (int64_t)K * n;
        for (int32_t k = 0; k < K; ++k)
            if (!std::isfinite(betas_k[k])) return ana_fail(VEGAS_EINVAL, "non-finite beta");
        for (int64_t i = 0; i < n_tot; ++i)
            if (!std::isfinite(E[i])) return ana_fail(VEGAS_EINVAL, "non-finite energy");
        vegas_status st = have_device();
        if (st != VEGAS_OK) return st;
        cudaStream_t stream = (cudaStream_t)cuda_stream;
        DevBuf b;
        double *d_E, *d_O, *d_D, *d_bk, *d_bo, *d_g, *d_lse, *d_part, *d_obs;
        const int parts = (int)std::min<int64_t>(256, (n_tot + kAnaThreads - 1) / kAnaThreads);
        const int rows = std::max<int32_t>(K, n_out);
        ACK(b.alloc(&d_E, sizeof(double) * n_tot));
        ACK(b.alloc(&d_O, sizeof(double) * n_tot * std::max(n_obs, 1)));
        ACK(b.alloc(&d_D, sizeof(double) * n_tot));
        ACK(b.alloc(&d_bk, sizeof(double) * K));
        ACK(b.alloc(&d_bo, sizeof(double) * std::max(n_out, 1)));
        ACK(b.alloc(&d_g, sizeof(double) * K));
        ACK(b.alloc(&d_lse, sizeof(double) * rows));
        ACK(b.alloc(&d_part, sizeof(double) * (2 + kMaxObs) * (size_t)parts * rows));
        ACK(b.alloc(&d_obs, sizeof(double) * (size_t)std::max(n_out, 1) * std::max(n_obs, 1)));
        ACK(cudaMemcpyAsync(d_E, E, sizeof(double) * n_tot, cudaMemcpyHostToDevice, stream));
        if (n_obs > 0) ACK(cudaMemcpyAsync(d_O, O, sizeof(double) * n_tot * n_obs, cudaMemcpyHostToDevice, stream));
        ACK(cudaMemcpyAsync(d_bk, betas_k, sizeof(double) * K, cudaMemcpyHostToDevice, stream));
        if (n_out > 0) ACK(cudaMemcpyAsync(d_bo, betas_out, sizeof(double) * n_out, cudaMemcpyHostToDevice, stream));
        std::vector<double> g((size_t)K, 0.0), gn((size_t)K);
        ACK(cudaMemcpyAsync(d_g, g.data(), sizeof(double) * K, cudaMemcpyHostToDevice, stream));
        const double logn = std::log((double)n);
        const int dgrid = (int)std::min<int64_t>((n_tot + 255) / 256, 4096);
        int32_t it = 0;
        for (it = 1; it <= max_iter; ++it) {
            denom_kernel<<<dgrid, 256, 0, stream>>>(d_E, n_tot, d_bk, d_g, K, logn, d_D);
            lse_kernel<<<dim3(parts, K), kAnaThreads, 0, stream>>>(d_E, d_D, d_O, 0, n_tot, d_bk, d_part);
            combine_kernel<<<(K + 127) / 128, 128, 0, stream>>>(d_part, parts, K, 0, d_lse, nullptr);
            ACK(cudaGetLastError());
            ACK(cudaMemcpyAsync(gn.data(), d_lse, sizeof(double) * K, cudaMemcpyDeviceToHost, stream));
            ACK(cudaStreamSynchronize(stream));
            double diff = 0.0;
            const double g0 = gn[0];
            for (int32_t k = 0; k < K; ++k) {
                gn[(size_t)k] -= g0;  // gauge: g_0 = 0
                diff = std::max(diff, std::fabs(gn[(size_t)k] - g[(size_t)k]));
            }
            g = gn;
            ACK(cudaMemcpyAsync(d_g, g.data(), sizeof(double) * K, cudaMemcpyHostToDevice, stream));
            if (!std::isfinite(diff)) return ana_fail(VEGAS_EDEVICE, "reweighting iteration produced a non-finite value");
            if (diff < tol) break;
        }
        if (it > max_iter) it = max_iter;
        if (g_out) std::memcpy(g_out, g.data(), sizeof(double) * K);
        if (iters_out) *iters_out = it;
        if (n_out > 0) {
            denom_kernel<<<dgrid, 256, 0, stream>>>(d_E, n_tot, d_bk, d_g, K, logn, d_D);
            lse_kernel<<<dim3(parts, n_out), kAnaThreads, 0, stream>>>(d_E, d_D, d_O, n_obs, n_tot, d_bo, d_part);
            combine_kernel<<<(n_out + 127) / 128, 128, 0, stream>>>(d_part, parts, n_out, n_obs, d_lse, d_obs);
            ACK(cudaGetLastError());
            if (n_obs > 0)
                ACK(cudaMemcpyAsync(out, d_obs, sizeof(double) * n_out * n_obs, cudaMemcpyDeviceToHost, stream));
            ACK(cudaStreamSynchronize(stream));
        }
        return VEGAS_OK;
    } catch (...) {
        return analysis_host_exception();
    }
}
