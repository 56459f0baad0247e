// Ising model with the spin-flip policy (Sec. II) on periodic square and simple cubic
// lattices, multi-spin coded: one 32-bit word holds 32 consecutive sites of one colour of
// one row (x direction) of one replica. A thread takes one word position for a group of four
// replicas (the four words of one Philox block per site): it builds, bit-sliced, the count
// of neighbours aligned with each spin, draws one Philox block per site, and decides 128
// flips against integer thresholds. Magnetization and bond sums are popcounts.
//
// Threshold: accept iff dE <= 0 or w < ceil(exp(-beta dE) 2^32), which for an integer w is
// exactly w 2^-32 < exp(-beta dE). The host computes exp in FP64 with the same expression
// as the definition, so the chain is the definition's bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "vegas_device.cuh"
#include "vegas_internal.h"

namespace vegas {
namespace {

constexpr uint32_t kPurposeIsing = 0x80000u;
constexpr uint32_t kPurposeIsingInit = 0x90000u;
constexpr int kIsingThreads = 256;
constexpr int kMaxIsingReplicas = 512;

struct IsingThr {          // one replica at one temperature/field step
    uint32_t thr[14];      // class s * (z + 1) + a: accept iff w < thr (when not always)
    uint32_t always;       // bit per class: dE <= 0
    uint32_t pad;
};

struct IsingRun {
    uint32_t t, rec, mcs, pad;
    const IsingThr *thr;          // [n_steps][R]
    const double *h;              // [n_steps][R]
    double *hist;                 // [records][R][2]
    unsigned long long *acc;      // [R][2]: up spins, aligned bonds (colour-1 ends)
};

struct IsingPassArgs {
    uint32_t *spins;
    IsingRun *run;
    uint64_t seed;
    int64_t rows;        // L^(dims-1)
    int32_t L, KW, R, c, inst_base;
};

__host__ __device__ inline int64_t word_index(int r, int c, int64_t row, int kw, int64_t rows, int KW) {
    return ((int64_t)(r * 2 + c) * rows + row) * KW + kw;
}

// Adds the bit vector x to the bit-sliced counter (p0, p1, p2) (counts up to 7).
__device__ __forceinline__ void slice_add(uint32_t x, uint32_t &p0, uint32_t &p1, uint32_t &p2) {
    const uint32_t c0 = p0 & x;
    p0 ^= x;
    const uint32_t c1 = p1 & c0;
    p1 ^= c0;
    p2 ^= c1;
}

template <int DIMS>
__global__ void __launch_bounds__(kIsingThreads) ising_pass_kernel(const IsingPassArgs a) {
    constexpr int Z = 2 * DIMS;
    __shared__ IsingThr s_thr[kMaxIsingReplicas];
    IsingRun *rs = a.run;
    const uint32_t t = rs->t;
    const uint32_t step = rs->rec / rs->mcs;
    for (int i = threadIdx.x; i < a.R; i += blockDim.x) s_thr[i] = rs->thr[(int64_t)step * a.R + i];
    __syncthreads();
    const int L = a.L, KW = a.KW, c = a.c, oc = 1 - c;
    const int64_t rows = a.rows, per_g = rows * KW, n_items = (int64_t)(a.R / 4) * per_g;
    const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
    const int lane = threadIdx.x & 31;
    uint32_t *S = a.spins;
    unsigned long long up[4] = {0, 0, 0, 0}, al[4] = {0, 0, 0, 0};
    int g_cur = -1;
    auto flush = [&]() {  // warp-uniform: all lanes share g_cur
        for (int j = 0; j < 4; ++j) {
            unsigned long long u = up[j], v = al[j];
            for (int off = 16; off > 0; off >>= 1) {
                u += __shfl_xor_sync(0xFFFFFFFFu, u, off);
                v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
            }
            if (lane == 0 && g_cur >= 0) {
                atomicAdd(&rs->acc[(g_cur * 4 + j) * 2], u);
                atomicAdd(&rs->acc[(g_cur * 4 + j) * 2 + 1], v);
            }
            up[j] = 0;
            al[j] = 0;
        }
    };
    // n_items and the stride are multiples of 32, and so is per_g: a warp's items share g
    for (int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; item < n_items;
         item += (int64_t)gridDim.x * blockDim.x) {
        const int g = (int)(item / per_g);
        if (g != g_cur) {
            flush();
            g_cur = g;
        }
        const int64_t rem = item - (int64_t)g * per_g;
        const int64_t row = rem / KW;
        const int kw = (int)(rem - row * KW);
        const int y = (int)(row % L), zc = DIMS == 3 ? (int)(row / L) : 0;
        const int off = (y + zc + c) & 1;
        const int64_t rym = (int64_t)((y + L - 1) % L) + (int64_t)L * zc, ryp = (int64_t)((y + 1) % L) + (int64_t)L * zc;
        const int64_t rzm = DIMS == 3 ? (int64_t)y + (int64_t)L * ((zc + L - 1) % L) : 0;
        const int64_t rzp = DIMS == 3 ? (int64_t)y + (int64_t)L * ((zc + 1) % L) : 0;
        const int kws = off == 0 ? (kw + KW - 1) % KW : (kw + 1) % KW;
        uint32_t own[4], nb[4][Z], p0[4], p1[4], p2[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = g * 4 + j;
            own[j] = S[word_index(r, c, row, kw, rows, KW)];
            const uint32_t xa = S[word_index(r, oc, row, kw, rows, KW)];
            const uint32_t xb = S[word_index(r, oc, row, kws, rows, KW)];
            nb[j][0] = xa;                                                      // x neighbour at the same k
            nb[j][1] = off == 0 ? (xa << 1) | (xb >> 31) : (xa >> 1) | (xb << 31);  // k - 1 or k + 1
            nb[j][2] = S[word_index(r, oc, rym, kw, rows, KW)];
            nb[j][3] = S[word_index(r, oc, ryp, kw, rows, KW)];
            if (DIMS == 3) {
                nb[j][4] = S[word_index(r, oc, rzm, kw, rows, KW)];
                nb[j][5] = S[word_index(r, oc, rzp, kw, rows, KW)];
            }
            p0[j] = p1[j] = p2[j] = 0u;
#pragma unroll
            for (int q = 0; q < Z; ++q) slice_add(~(own[j] ^ nb[j][q]), p0[j], p1[j], p2[j]);
        }
        uint32_t flip[4] = {0u, 0u, 0u, 0u};
        const uint32_t group = (uint32_t)(a.inst_base >> 2) + (uint32_t)g;
        const int64_t site0 = (int64_t)L * row + off + (int64_t)kw * 64;  // x = 2 (32 kw + b) + off
        for (int b = 0; b < 32; ++b) {
            const uint32_t site = (uint32_t)(site0 + 2 * b);
            const uint4 w = philox10(make_uint4(site, t, group, kPurposeIsing), k0, k1);
            const uint32_t wj[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int cls = (int)((own[j] >> b) & 1u) * (Z + 1) + (int)((p0[j] >> b) & 1u) +
                                2 * (int)((p1[j] >> b) & 1u) + 4 * (int)((p2[j] >> b) & 1u);
                const IsingThr &T = s_thr[g * 4 + j];
                const bool acc = ((T.always >> cls) & 1u) || wj[j] < T.thr[cls];
                flip[j] |= (uint32_t)acc << b;
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t nw = own[j] ^ flip[j];
            if (flip[j]) S[word_index(g * 4 + j, c, row, kw, rows, KW)] = nw;
            up[j] += (unsigned long long)__popc(nw);
            if (c == 1) {  // each bond counted at its colour-1 end, after the update
#pragma unroll
                for (int q = 0; q < Z; ++q) al[j] += (unsigned long long)__popc(~(nw ^ nb[j][q]));
            }
        }
    }
    flush();
}

// After both passes: (E, M) of every replica into the history; the counters are cleared and
// the MCS counter and record index advance. One block, one thread per replica.
__global__ void ising_reduce_kernel(IsingRun *rs, int32_t R, int64_t n, int32_t Z, double J) {
    const uint32_t rec = rs->rec, step = rec / rs->mcs;
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        const unsigned long long upc = rs->acc[r * 2], alc = rs->acc[r * 2 + 1];
        const int64_t M = 2 * (int64_t)upc - n;
        const int64_t bsum = 2 * (int64_t)alc - (int64_t)Z * (n / 2);
        const double h = rs->h[(int64_t)step * R + r];
        double *o = rs->hist + ((int64_t)rec * R + r) * 2;
        o[0] = __dsub_rn(__dmul_rn(-J, (double)bsum), __dmul_rn(h, (double)M));
        o[1] = (double)M;
        rs->acc[r * 2] = 0;
        rs->acc[r * 2 + 1] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        rs->t = rs->t + 1;
        rs->rec = rec + 1;
    }
}

// Initial state: bit 31 of the replica's word of Philox(seed; site, 0xFFFFFFFF, group, 0x90000).
__global__ void ising_init_kernel(uint32_t *S, uint64_t seed, int64_t rows, int32_t L, int32_t KW, int32_t R,
                                  int32_t dims, int32_t inst_base, int32_t all_up) {
    const int64_t per_g = rows * KW, n_items = 2 * (int64_t)(R / 4) * per_g;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; item < n_items;
         item += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(item / ((int64_t)(R / 4) * per_g));
        const int64_t rest = item - (int64_t)c * (R / 4) * per_g;
        const int g = (int)(rest / per_g);
        const int64_t rem = rest - (int64_t)g * per_g;
        const int64_t row = rem / KW;
        const int kw = (int)(rem - row * KW);
        const int y = (int)(row % L), zc = dims == 3 ? (int)(row / L) : 0;
        const int off = (y + zc + c) & 1;
        uint32_t wd[4] = {0u, 0u, 0u, 0u};
        for (int b = 0; b < 32; ++b) {
            const uint32_t site = (uint32_t)((int64_t)L * row + off + (int64_t)kw * 64 + 2 * b);
            const uint4 w = philox10(make_uint4(site, 0xFFFFFFFFu, (uint32_t)(inst_base >> 2) + (uint32_t)g,
                                                kPurposeIsingInit),
                                     k0, k1);
            const uint32_t wj[4] = {w.x, w.y, w.z, w.w};
            for (int j = 0; j < 4; ++j) wd[j] |= (all_up ? 1u : (wj[j] >> 31)) << b;
        }
        for (int j = 0; j < 4; ++j) S[word_index(g * 4 + j, c, row, kw, rows, KW)] = wd[j];
    }
}

std::string g_ising_create_error;

}  // namespace
}  // namespace vegas

using namespace vegas;

struct vegas_ising {
    vegas_ising_options opt{};
    int device = 0, sm_count = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int64_t n = 0, rows = 0;
    int32_t KW = 0, Z = 0;
    uint32_t *d_spins = nullptr;
    IsingRun *d_run = nullptr;
    IsingThr *d_thr = nullptr;
    double *d_h = nullptr, *d_hist = nullptr;
    unsigned long long *d_acc = nullptr;
    size_t thr_cap = 0, hist_cap = 0;
    int grid = 1;
    std::vector<std::vector<double>> hist;  // per replica: records * 2
    int64_t records = 0;
    uint32_t t = 0;
    int64_t kernel_launches = 0, sweep_launches = 0, device_bytes = 0;
    double sweep_ms = 0.0, last_run_ms = 0.0;
    bool poisoned = false;
    std::string err;
};

namespace vegas {
namespace {

vegas_status ifail(vegas_ising *c, vegas_status st, const std::string &m) {
    if (c) {
        c->err = m;
        if (st == VEGAS_ECUDA || st == VEGAS_EDEVICE) c->poisoned = true;
    } else {
        g_ising_create_error = m;
    }
    return st;
}

// A host exception caught at an entry point, as a status (called inside a catch block).
vegas_status ising_host_exception(vegas_ising *c) {
    std::string m;
    const vegas_status st = status_of_current_exception(m);
    return ifail(c, st, m);
}

#define ICK(ctx, call)                                                                                 \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            return ifail((ctx), e_ == cudaErrorMemoryAllocation ? VEGAS_ENOMEM : VEGAS_ECUDA,          \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                          \
    } while (0)

void ising_free(vegas_ising *c) {
    void *bufs[] = {c->d_spins, c->d_run, c->d_thr, c->d_h, c->d_hist, c->d_acc};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

vegas_status ising_usable(vegas_ising *c) {
    if (!c) return VEGAS_EINVAL;
    if (c->poisoned) return VEGAS_ESTATE;
    return VEGAS_OK;
}

void launch_ising_pass(vegas_ising *c, int colour, cudaStream_t st) {
    IsingPassArgs a{c->d_spins, c->d_run, c->opt.seed, c->rows, c->opt.L, c->KW, c->opt.replicas, colour,
                    c->opt.inst_base};
    if (c->opt.dims == 3)
        ising_pass_kernel<3><<<c->grid, kIsingThreads, 0, st>>>(a);
    else
        ising_pass_kernel<2><<<c->grid, kIsingThreads, 0, st>>>(a);
}

}  // namespace
}  // namespace vegas

extern "C" void vegas_ising_default_options(vegas_ising_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->dims = 2;
    o->L = 64;
    o->J = 1.0;
    o->replicas = 32;
    o->inst_base = 0;
    o->seed = 1;
    o->device = -1;
    o->cuda_stream = nullptr;
    o->init_up = 0;
    o->timing = 0;
}

// vegas_ising_create without the exception guard; *made is the context under construction.
static vegas_status ising_create(const vegas_ising_options *opt, vegas_ising **out, vegas_ising **made) {
    if (!out) return ifail(nullptr, VEGAS_EINVAL, "out is NULL");
    *out = nullptr;
    vegas_ising_options o;
    vegas_ising_default_options(&o);
    if (opt) o = *opt;
    if (o.dims != 2 && o.dims != 3) return ifail(nullptr, VEGAS_EINVAL, "dims must be 2 or 3");
    if (o.L < 64 || o.L % 64) return ifail(nullptr, VEGAS_EINVAL, "L must be a positive multiple of 64");
    const int64_t n = o.dims == 3 ? (int64_t)o.L * o.L * o.L : (int64_t)o.L * o.L;
    if (n >= ((int64_t)1 << 31)) return ifail(nullptr, VEGAS_EINVAL, "L^dims must be below 2^31");
    if (o.replicas < 4 || o.replicas > kMaxIsingReplicas || o.replicas % 4)
        return ifail(nullptr, VEGAS_EINVAL, "replicas must be a multiple of 4 in [4, 512]");
    if (o.inst_base < 0 || o.inst_base % 4) return ifail(nullptr, VEGAS_EINVAL, "inst_base must be a multiple of 4");
    if (!std::isfinite(o.J)) return ifail(nullptr, VEGAS_EINVAL, "J must be finite");
    if (o.init_up < 0 || o.init_up > 1 || o.timing < 0 || o.timing > 1)
        return ifail(nullptr, VEGAS_EINVAL, "init_up and timing must be 0 or 1");
    vegas_ising *c = new (std::nothrow) vegas_ising();
    if (!c) return ifail(nullptr, VEGAS_ENOMEM, "host allocation failed");
    *made = c;
    c->opt = o;
    c->n = n;
    c->rows = o.dims == 3 ? (int64_t)o.L * o.L : o.L;
    c->KW = o.L / 64;
    c->Z = 2 * o.dims;
    auto bail = [&](vegas_status st) {
        g_ising_create_error = c->err;
        ising_free(c);
        delete c;
        *made = nullptr;
        return st;
    };
    int ndev = 0;
    cudaError_t ce = cudaGetDeviceCount(&ndev);
    if (ce != cudaSuccess || ndev == 0) {
        c->err = std::string("no CUDA device: ") + cudaGetErrorString(ce);
        return bail(VEGAS_ECUDA);
    }
    if (o.device >= 0)
        c->device = o.device;
    else if (cudaGetDevice(&c->device) != cudaSuccess) {
        c->err = "cudaGetDevice failed";
        return bail(VEGAS_ECUDA);
    }
    vegas_status st;
    if ((st = [&]() -> vegas_status {
             ICK(c, cudaSetDevice(c->device));
             ICK(c, cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device));
             if (o.cuda_stream) {
                 c->stream = (cudaStream_t)o.cuda_stream;
             } else {
                 ICK(c, cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
                 c->own_stream = true;
             }
             const size_t words = (size_t)o.replicas * 2 * (size_t)c->rows * (size_t)c->KW;
             ICK(c, cudaMalloc(&c->d_spins, words * sizeof(uint32_t)));
             ICK(c, cudaMalloc(&c->d_run, sizeof(IsingRun)));
             ICK(c, cudaMalloc(&c->d_acc, sizeof(unsigned long long) * 2 * o.replicas));
             c->device_bytes = (int64_t)(words * 4 + sizeof(IsingRun) + 16 * (size_t)o.replicas);
             ICK(c, cudaMemsetAsync(c->d_acc, 0, sizeof(unsigned long long) * 2 * o.replicas, c->stream));
             int nb = 0;
             ICK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                        &nb, o.dims == 3 ? ising_pass_kernel<3> : ising_pass_kernel<2>, kIsingThreads, 0));
             const int64_t items = (int64_t)(o.replicas / 4) * c->rows * c->KW;
             c->grid = (int)std::max<int64_t>(1, std::min<int64_t>((items + kIsingThreads - 1) / kIsingThreads,
                                                                   (int64_t)c->sm_count * std::max(nb, 1)));
             const int64_t init_items = 2 * items;
             const int ig = (int)std::min<int64_t>((init_items + 255) / 256, (int64_t)c->sm_count * 8);
             ising_init_kernel<<<ig, 256, 0, c->stream>>>(c->d_spins, o.seed, c->rows, o.L, c->KW, o.replicas, o.dims,
                                                          o.inst_base, o.init_up);
             ICK(c, cudaGetLastError());
             ICK(c, cudaStreamSynchronize(c->stream));
             c->kernel_launches = 1;
             return VEGAS_OK;
         }()) != VEGAS_OK)
        return bail(st);
    c->hist.assign((size_t)o.replicas, std::vector<double>());
    *out = c;
    return VEGAS_OK;
}

extern "C" vegas_status vegas_ising_create(const vegas_ising_options *opt, vegas_ising **out) {
    vegas_ising *made = nullptr;
    try {
        return ising_create(opt, out, &made);
    } catch (...) {
        const vegas_status st = ising_host_exception(nullptr);
        if (made) {
            ising_free(made);
            delete made;
        }
        if (out) *out = nullptr;
        return st;
    }
}

extern "C" vegas_status vegas_ising_run(vegas_ising *c, const double *T, const double *h, int32_t n_steps,
                                        int32_t mcs) {
    try {
        vegas_status st = ising_usable(c);
        if (st != VEGAS_OK) return st;
        if (n_steps < 0 || mcs < 0) return ifail(c, VEGAS_EINVAL, "n_steps and mcs_per_step must be >= 0");
        if (n_steps == 0 || mcs == 0) return VEGAS_OK;
        if (!T || !h) return ifail(c, VEGAS_EINVAL, "T or h is NULL");
        if ((int64_t)c->t + (int64_t)n_steps * mcs >= (int64_t)UINT32_MAX)
            return ifail(c, VEGAS_EINVAL, "global MCS counter would exceed 32 bits");
        const int R = c->opt.replicas, Z = c->Z;
        std::vector<IsingThr> thr((size_t)n_steps * R);
        std::vector<double> hv((size_t)n_steps * R);
        for (int r = 0; r < R; ++r)
            for (int s = 0; s < n_steps; ++s) {
                const double Tv = T[(int64_t)r * n_steps + s], hh = h[(int64_t)r * n_steps + s];
                if (!(Tv > 0.0) || !std::isfinite(Tv)) return ifail(c, VEGAS_EINVAL, "T must be finite and > 0");
                if (!std::isfinite(hh)) return ifail(c, VEGAS_EINVAL, "h must be finite");
                const double beta = 1.0 / Tv;
                IsingThr &e = thr[(size_t)s * R + r];
                std::memset(&e, 0, sizeof e);
                for (int sb = 0; sb < 2; ++sb)
                    for (int al = 0; al <= Z; ++al) {
                        const double si = sb ? 1.0 : -1.0;
                        const double sum = sb ? (double)(2 * al - Z) : (double)(Z - 2 * al);
                        const double dE = 2.0 * si * (c->opt.J * sum + hh);
                        const int cls = sb * (Z + 1) + al;
                        if (dE <= 0.0) {
                            e.always |= 1u << cls;
                            continue;
                        }
                        // accept iff w < x = exp(-beta dE) 2^32 (w integer): iff w < ceil(x)
                        const double x = std::ceil(std::exp(-(beta * dE)) * 4294967296.0);
                        if (x >= 4294967296.0)
                            e.always |= 1u << cls;
                        else
                            e.thr[cls] = (uint32_t)x;
                    }
                hv[(size_t)s * R + r] = hh;
            }
        ICK(c, cudaSetDevice(c->device));
        const int64_t nrec = (int64_t)n_steps * mcs;
        if (thr.size() > c->thr_cap) {
            if (c->d_thr) cudaFree(c->d_thr);
            if (c->d_h) cudaFree(c->d_h);
            c->d_thr = nullptr;
            c->d_h = nullptr;
            c->thr_cap = 0;
            ICK(c, cudaMalloc(&c->d_thr, sizeof(IsingThr) * thr.size()));
            ICK(c, cudaMalloc(&c->d_h, sizeof(double) * thr.size()));
            c->thr_cap = thr.size();
        }
        const size_t hneed = (size_t)nrec * R * 2;
        if (hneed > c->hist_cap) {
            if (c->d_hist) cudaFree(c->d_hist);
            c->d_hist = nullptr;
            c->hist_cap = 0;
            ICK(c, cudaMalloc(&c->d_hist, sizeof(double) * hneed));
            c->hist_cap = hneed;
        }
        ICK(c, cudaMemcpyAsync(c->d_thr, thr.data(), sizeof(IsingThr) * thr.size(), cudaMemcpyHostToDevice, c->stream));
        ICK(c, cudaMemcpyAsync(c->d_h, hv.data(), sizeof(double) * hv.size(), cudaMemcpyHostToDevice, c->stream));
        IsingRun rs{c->t, 0u, (uint32_t)mcs, 0u, c->d_thr, c->d_h, c->d_hist, c->d_acc};
        ICK(c, cudaMemcpyAsync(c->d_run, &rs, sizeof rs, cudaMemcpyHostToDevice, c->stream));
        std::vector<cudaEvent_t> ev;
        if (c->opt.timing) {
            ev.resize((size_t)nrec * 4);
            for (auto &x : ev) ICK(c, cudaEventCreate(&x));
        }
        cudaEvent_t e0, e1;
        ICK(c, cudaEventCreate(&e0));
        ICK(c, cudaEventCreate(&e1));
        ICK(c, cudaEventRecord(e0, c->stream));
        const int rthreads = std::min(std::max(32, (R + 31) / 32 * 32), 512);
        for (int64_t m = 0; m < nrec; ++m) {
            for (int colour = 0; colour < 2; ++colour) {
                if (c->opt.timing) ICK(c, cudaEventRecord(ev[(size_t)m * 4 + 2 * colour], c->stream));
                launch_ising_pass(c, colour, c->stream);
                if (c->opt.timing) ICK(c, cudaEventRecord(ev[(size_t)m * 4 + 2 * colour + 1], c->stream));
            }
            ising_reduce_kernel<<<1, rthreads, 0, c->stream>>>(c->d_run, R, c->n, Z, c->opt.J);
        }
        ICK(c, cudaGetLastError());
        ICK(c, cudaEventRecord(e1, c->stream));
        ICK(c, cudaStreamSynchronize(c->stream));
        float ms = 0.f;
        ICK(c, cudaEventElapsedTime(&ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        double sw = 0.0;
        for (size_t k = 0; k + 1 < ev.size(); k += 2) {
            float x = 0.f;
            ICK(c, cudaEventElapsedTime(&x, ev[k], ev[k + 1]));
            sw += x;
        }
        for (auto &x : ev) cudaEventDestroy(x);
        c->last_run_ms = ms;
        c->sweep_ms += sw;
        c->kernel_launches += nrec * 3;
        c->sweep_launches += nrec * 2;
        std::vector<double> hh(hneed);
        ICK(c, cudaMemcpy(hh.data(), c->d_hist, sizeof(double) * hneed, cudaMemcpyDeviceToHost));
        for (int r = 0; r < R; ++r) {
            auto &v = c->hist[(size_t)r];
            const size_t old = v.size();
            v.resize(old + (size_t)nrec * 2);
            for (int64_t k = 0; k < nrec; ++k) {
                v[old + (size_t)k * 2] = hh[((size_t)k * R + r) * 2];
                v[old + (size_t)k * 2 + 1] = hh[((size_t)k * R + r) * 2 + 1];
            }
        }
        c->records += nrec;
        c->t += (uint32_t)nrec;
        return VEGAS_OK;
    } catch (...) {
        return ising_host_exception(c);
    }
}

extern "C" vegas_status vegas_ising_history(const vegas_ising *cc, double *out, size_t capacity, size_t *n_written) {
    try {
        vegas_ising *c = const_cast<vegas_ising *>(cc);
        vegas_status st = ising_usable(c);
        if (st != VEGAS_OK) return st;
        const size_t need = (size_t)c->opt.replicas * (size_t)c->records * 2;
        if (n_written) *n_written = need;
        if (!out) return VEGAS_OK;
        if (capacity < need) return ifail(c, VEGAS_EINVAL, "history buffer too small");
        for (int r = 0; r < c->opt.replicas; ++r)
            std::memcpy(out + (size_t)r * c->records * 2, c->hist[(size_t)r].data(), sizeof(double) * c->records * 2);
        return VEGAS_OK;
    } catch (...) {
        return ising_host_exception(const_cast<vegas_ising *>(cc));
    }
}

namespace vegas {
namespace {

// Copies one replica's words (both colours) between device and host, then (un)packs them.
vegas_status ising_spins_io(vegas_ising *c, int32_t replica, int8_t *out, const int8_t *in) {
    vegas_status st = ising_usable(c);
    if (st != VEGAS_OK) return st;
    if (replica < 0 || replica >= c->opt.replicas) return ifail(c, VEGAS_EINVAL, "replica out of range");
    ICK(c, cudaSetDevice(c->device));
    const int L = c->opt.L, KW = c->KW;
    const int64_t rows = c->rows;
    std::vector<uint32_t> w((size_t)2 * rows * KW);
    uint32_t *dev = c->d_spins + word_index(replica, 0, 0, 0, rows, KW);
    if (in)
        for (int64_t i = 0; i < c->n; ++i)
            if (in[i] != 1 && in[i] != -1) return ifail(c, VEGAS_EINVAL, "spins must be +1 or -1");
    if (out) ICK(c, cudaMemcpy(w.data(), dev, sizeof(uint32_t) * w.size(), cudaMemcpyDeviceToHost));
    for (int col = 0; col < 2; ++col)
        for (int64_t row = 0; row < rows; ++row) {
            const int y = (int)(row % L), zc = c->opt.dims == 3 ? (int)(row / L) : 0;
            const int off = (y + zc + col) & 1;
            for (int kw = 0; kw < KW; ++kw) {
                uint32_t &word = w[(size_t)(((int64_t)col * rows + row) * KW + kw)];
                for (int b = 0; b < 32; ++b) {
                    const int64_t site = (int64_t)L * row + off + 64 * kw + 2 * b;
                    if (out)
                        out[site] = ((word >> b) & 1u) ? 1 : -1;
                    else if (in[site] > 0)
                        word |= 1u << b;
                }
            }
        }
    if (in) {
        ICK(c, cudaMemcpy(dev, w.data(), sizeof(uint32_t) * w.size(), cudaMemcpyHostToDevice));
    }
    return VEGAS_OK;
}

}  // namespace
}  // namespace vegas

extern "C" vegas_status vegas_ising_get_spins(const vegas_ising *c, int32_t replica, int8_t *out) {
    try {
        if (!out) return ifail(const_cast<vegas_ising *>(c), VEGAS_EINVAL, "out is NULL");
        return ising_spins_io(const_cast<vegas_ising *>(c), replica, out, nullptr);
    } catch (...) {
        return ising_host_exception(const_cast<vegas_ising *>(c));
    }
}

extern "C" vegas_status vegas_ising_set_spins(vegas_ising *c, int32_t replica, const int8_t *in) {
    try {
        if (!in) return ifail(c, VEGAS_EINVAL, "in is NULL");
        return ising_spins_io(c, replica, nullptr, in);
    } catch (...) {
        return ising_host_exception(c);
    }
}

extern "C" vegas_status vegas_ising_set_mcs_counter(vegas_ising *c, uint32_t t) {
    try {
        vegas_status st = ising_usable(c);
        if (st != VEGAS_OK) return st;
        if (t == UINT32_MAX) return ifail(c, VEGAS_EINVAL, "MCS counter must be below 2^32 - 1");
        c->t = t;
        return VEGAS_OK;
    } catch (...) {
        return ising_host_exception(c);
    }
}

extern "C" vegas_status vegas_ising_stats(const vegas_ising *c, vegas_stats_t *o) {
    try {
        if (!c || !o) return VEGAS_EINVAL;
        std::memset(o, 0, sizeof *o);
        o->n_samples = 1;
        o->n_instances = c->opt.replicas;
        o->replicas = c->opt.replicas;
        o->max_colours = 2;
        o->n_sites = c->n;
        o->n_edges = c->n * c->Z;
        o->records = c->records;
        o->mcs_done = c->t;
        o->kernel_launches = c->kernel_launches;
        o->sweep_launches = c->sweep_launches;
        o->sweep_ms = c->sweep_ms;
        o->last_run_ms = c->last_run_ms;
        o->device_bytes = c->device_bytes;
        return VEGAS_OK;
    } catch (...) {
        return ising_host_exception(const_cast<vegas_ising *>(c));
    }
}

extern "C" const char *vegas_ising_last_error(const vegas_ising *c) {
    if (!c) return g_ising_create_error.c_str();
    return c->err.c_str();
}

extern "C" void vegas_ising_destroy(vegas_ising *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    ising_free(c);
    delete c;
}
