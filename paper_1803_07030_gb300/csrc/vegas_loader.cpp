// Sample loader (host): validation, greedy colouring and colour-major renumbering.
//
// The sample is the paper's material file (Sec. III.C: per-site spin norm, field axis and
// type; links with exchange J_ij) plus its anisotropy file, given as arrays. The loader
// rejects anything the sweep cannot treat exactly: asymmetric or duplicate links,
// self-links, out-of-range neighbours, non-finite parameters, an improper colouring.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <unordered_map>

#include "vegas_internal.h"

namespace vegas {

namespace {

bool finite_all(const double *p, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

std::string at(const char *what, int64_t i) { return std::string(what) + " at index " + std::to_string(i); }

// Spread the low 21 bits of v so that bit b lands on bit 3b (Morton interleave helper).
uint64_t spread3(uint64_t v) {
    v &= 0x1FFFFFull;
    v = (v | (v << 32)) & 0x1F00000000FFFFull;
    v = (v | (v << 16)) & 0x1F0000FF0000FFull;
    v = (v | (v << 8)) & 0x100F00F00F00F00Full;
    v = (v | (v << 4)) & 0x10C30C30C30C30C3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

// Morton (Z-order) keys of the site positions on a 2^21 grid spanning their bounding box.
std::vector<uint64_t> morton_keys(const double *pos, int32_t n) {
    double lo[3] = {pos[0], pos[1], pos[2]}, hi[3] = {pos[0], pos[1], pos[2]};
    for (int32_t i = 0; i < n; ++i)
        for (int q = 0; q < 3; ++q) {
            lo[q] = std::min(lo[q], pos[3 * (int64_t)i + q]);
            hi[q] = std::max(hi[q], pos[3 * (int64_t)i + q]);
        }
    const double ext = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]});
    const double scale = ext > 0.0 ? 2097151.0 / ext : 0.0;
    std::vector<uint64_t> key((size_t)n);
    for (int32_t i = 0; i < n; ++i) {
        uint64_t k = 0;
        for (int q = 0; q < 3; ++q) {
            double c = (pos[3 * (int64_t)i + q] - lo[q]) * scale;
            c = std::min(std::max(c, 0.0), 2097151.0);
            k |= spread3((uint64_t)c) << q;
        }
        key[(size_t)i] = k;
    }
    return key;
}


}  // namespace

}  // namespace vegas

extern "C" int32_t vegas_greedy_colour(int32_t n, const int64_t *row_ptr, const int32_t *col, int32_t *color) {
    try {
        if (n < 0 || (n > 0 && (!row_ptr || !color))) return -1;
        if (n > 0 && row_ptr[0] != 0) return -1;
        for (int32_t i = 0; i < n; ++i)
            if (row_ptr[i + 1] < row_ptr[i]) return -1;
        if (n > 0 && row_ptr[n] > 0 && !col) return -1;
        std::vector<int32_t> seen;  // seen[c] == i  <=>  colour c is used by a coloured neighbour of i
        int32_t nc = 0;
        for (int32_t i = 0; i < n; ++i) color[i] = -1;
        for (int32_t i = 0; i < n; ++i) {
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                const int32_t j = col[e];
                if (j < 0 || j >= n) return -1;
                const int32_t cj = color[j];
                if (cj >= 0) {
                    if ((size_t)cj >= seen.size()) seen.resize((size_t)cj + 1, -1);
                    seen[(size_t)cj] = i;
                }
            }
            int32_t c = 0;
            while ((size_t)c < seen.size() && seen[(size_t)c] == i) ++c;
            color[i] = c;
            nc = std::max(nc, c + 1);
        }
        return nc;
    } catch (...) {
        return -1;  // a host exception never crosses the C boundary
    }
}

namespace vegas {

namespace {

// Slab width along x of the wavefront order: the planes (distinct z) of a sample with many
// sites per plane are cut into slabs of about 16384 sites per plane, so that the window of
// planes a wavefront keeps in flight stays a few MB whatever the lattice's cross-section.
// Returns 0 for no slabs.
double auto_slab_width(const double *P, int32_t n) {
    std::vector<double> z((size_t)n);
    double xmin = P[0], xmax = P[0];
    for (int32_t i = 0; i < n; ++i) {
        z[(size_t)i] = P[3 * (size_t)i + 2];
        xmin = std::min(xmin, P[3 * (size_t)i]);
        xmax = std::max(xmax, P[3 * (size_t)i]);
    }
    std::sort(z.begin(), z.end());
    const int64_t planes = std::unique(z.begin(), z.end()) - z.begin();
    const int64_t per_plane = (n + planes - 1) / planes;
    const int64_t n_slabs = (per_plane + 16383) / 16384;
    if (n_slabs <= 1 || !(xmax > xmin)) return 0.0;
    return (xmax - xmin) / (double)n_slabs * (1.0 + 1e-9);
}

}  // namespace

bool load_sample(const vegas_sample &s, LoadedSample &L, std::string &err, bool type_major, bool plane_order,
                 double wave_slab) {
    const int32_t n = s.n_sites;
    if (n < 1) { err = "n_sites must be >= 1"; return false; }
    if (!s.row_ptr) { err = "row_ptr is NULL"; return false; }
    if (s.n_edges < 0) { err = "n_edges < 0"; return false; }
    if (s.n_edges > 0 && (!s.col || !s.J)) { err = "col or J is NULL"; return false; }
    if (s.row_ptr[0] != 0) { err = "row_ptr[0] != 0"; return false; }
    for (int32_t i = 0; i < n; ++i)
        if (s.row_ptr[i + 1] < s.row_ptr[i]) { err = at("row_ptr decreases", i); return false; }
    if (s.row_ptr[n] != s.n_edges) { err = "row_ptr[n_sites] != n_edges"; return false; }
    if (s.n_edges > (int64_t)INT32_MAX) { err = "more than 2^31-1 links in one sample"; return false; }
    const int64_t E = s.n_edges;
    for (int64_t e = 0; e < E; ++e)
        if (s.col[e] < 0 || s.col[e] >= n) { err = at("col out of range", e); return false; }
    if (!finite_all(s.J, E)) { err = "non-finite J"; return false; }

    // self-links, duplicates and symmetry: short rows are scanned, long rows use a sorted copy
    constexpr int64_t kScan = 32;
    // sorted (col, J) copies of the rows too long to scan
    std::unordered_map<int32_t, std::vector<std::pair<int32_t, double>>> sorted;
    for (int32_t i = 0; i < n; ++i) {
        const int64_t b = s.row_ptr[i], d = s.row_ptr[i + 1] - b;
        if (d > kScan) {
            auto &v = sorted[i];
            v.reserve((size_t)d);
            for (int64_t e = b; e < b + d; ++e) v.emplace_back(s.col[e], s.J[e]);
            std::sort(v.begin(), v.end());
        }
    }
    auto find_in_row = [&](int32_t j, int32_t i, double *Jout) -> int {
        const int64_t b = s.row_ptr[j], d = s.row_ptr[j + 1] - b;
        if (d > kScan) {
            const auto &v = sorted.at(j);
            auto it = std::lower_bound(v.begin(), v.end(), std::make_pair(i, -(double)INFINITY));
            if (it == v.end() || it->first != i) return 0;
            *Jout = it->second;
            return 1;
        }
        for (int64_t e = b; e < b + d; ++e)
            if (s.col[e] == i) { *Jout = s.J[e]; return 1; }
        return 0;
    };
    for (int32_t i = 0; i < n; ++i) {
        const int64_t b = s.row_ptr[i], d = s.row_ptr[i + 1] - b;
        if (d > kScan) {
            const auto &v = sorted.at(i);
            for (size_t q = 0; q < v.size(); ++q) {
                if (v[q].first == i) { err = at("self-link at site", i); return false; }
                if (q > 0 && v[q].first == v[q - 1].first) { err = at("duplicate link at site", i); return false; }
            }
        } else {
            for (int64_t e = b; e < b + d; ++e) {
                if (s.col[e] == i) { err = at("self-link at site", i); return false; }
                for (int64_t f = b; f < e; ++f)
                    if (s.col[f] == s.col[e]) { err = at("duplicate link at site", i); return false; }
            }
        }
        for (int64_t e = b; e < b + d; ++e) {
            double Jr = 0.0;
            if (!find_in_row(s.col[e], i, &Jr)) { err = at("link without its reverse, edge", e); return false; }
            if (Jr != s.J[e]) { err = at("J not symmetric, edge", e); return false; }
        }
    }
    sorted.clear();

    // parameters (defaults: s = 1, n = +z, k = 0, e = +z, kc = 0)
    const double *prm[5] = {s.spin_norm, s.field_axis, s.k_uni, s.e_uni, s.k_cub};
    const int64_t len[5] = {n, 3 * (int64_t)n, n, 3 * (int64_t)n, n};
    const char *name[5] = {"spin_norm", "field_axis", "k_uni", "e_uni", "k_cub"};
    for (int q = 0; q < 5; ++q)
        if (prm[q] && !finite_all(prm[q], len[q])) { err = std::string("non-finite ") + name[q]; return false; }
    if (s.spin_norm)
        for (int32_t i = 0; i < n; ++i)
            if (!(s.spin_norm[i] > 0.0)) { err = at("spin_norm <= 0", i); return false; }
    if (s.init_spins && !finite_all(s.init_spins, 3 * (int64_t)n)) { err = "non-finite init_spins"; return false; }
    if (s.positions && !finite_all(s.positions, 3 * (int64_t)n)) { err = "non-finite positions"; return false; }

    // colouring
    std::vector<int32_t> colour((size_t)n);
    int32_t nc = 0;
    if (s.color) {
        for (int32_t i = 0; i < n; ++i) {
            if (s.color[i] < 0 || s.color[i] >= kMaxColours) { err = at("colour outside [0, 64)", i); return false; }
            colour[(size_t)i] = s.color[i];
            nc = std::max(nc, s.color[i] + 1);
        }
        for (int32_t i = 0; i < n; ++i)
            for (int64_t e = s.row_ptr[i]; e < s.row_ptr[i + 1]; ++e)
                if (colour[(size_t)s.col[e]] == colour[(size_t)i]) { err = at("colouring not proper at site", i); return false; }
    } else {
        nc = vegas_greedy_colour(n, s.row_ptr, s.col, colour.data());
        if (nc > kMaxColours) { err = "greedy colouring needs more than 64 colours"; return false; }
    }

    // colour-major renumbering, increasing caller id inside a class
    L.n = n;
    L.n_colours = nc;
    L.n_edges = E;
    L.cstart.assign((size_t)nc + 1, 0);
    for (int32_t i = 0; i < n; ++i) L.cstart[(size_t)colour[(size_t)i] + 1]++;
    for (int32_t c = 0; c < nc; ++c) L.cstart[(size_t)c + 1] += L.cstart[(size_t)c];
    std::vector<int32_t> fill(L.cstart.begin(), L.cstart.end() - 1);
    L.orig.resize((size_t)n);
    L.inv.resize((size_t)n);
    for (int32_t i = 0; i < n; ++i) L.orig[(size_t)fill[(size_t)colour[(size_t)i]]++] = i;
    if (s.positions && plane_order) {  // memory order inside each class: slab, then z, y, x
        const double *P = s.positions;
        const double width = wave_slab > 0.0 ? wave_slab : (wave_slab == 0.0 ? auto_slab_width(P, n) : 0.0);
        double xmin = P[0];
        for (int32_t i = 1; i < n; ++i) xmin = std::min(xmin, P[3 * (size_t)i]);
        std::vector<int64_t> slab((size_t)n, 0);
        if (width > 0.0)
            for (int32_t i = 0; i < n; ++i) slab[(size_t)i] = (int64_t)std::floor((P[3 * (size_t)i] - xmin) / width);
        L.slab_width = width;
        for (int32_t c = 0; c < nc; ++c)
            std::stable_sort(L.orig.begin() + L.cstart[(size_t)c], L.orig.begin() + L.cstart[(size_t)c + 1],
                             [&](int32_t x, int32_t y) {
                                 if (slab[(size_t)x] != slab[(size_t)y]) return slab[(size_t)x] < slab[(size_t)y];
                                 for (int q = 2; q >= 0; --q)
                                     if (P[3 * (size_t)x + q] != P[3 * (size_t)y + q])
                                         return P[3 * (size_t)x + q] < P[3 * (size_t)y + q];
                                 return false;
                             });
    } else if (s.positions) {  // memory order inside each class: Morton curve of the positions
        const std::vector<uint64_t> key = morton_keys(s.positions, n);
        for (int32_t c = 0; c < nc; ++c)
            std::stable_sort(L.orig.begin() + L.cstart[(size_t)c], L.orig.begin() + L.cstart[(size_t)c + 1],
                             [&](int32_t x, int32_t y) { return key[(size_t)x] < key[(size_t)y]; });
    }
    L.n_types = 1;
    if (s.type)
        for (int32_t i = 0; i < n; ++i) {
            if (type_major && (s.type[i] < 0 || s.type[i] >= kMaxTypes)) {
                err = at("site type outside [0, 64) (per-type statistics) at site", i);
                return false;
            }
            L.n_types = std::max(L.n_types, s.type[i] + 1);
        }
    if (type_major && s.type)  // type by type inside each class, keeping the order above
        for (int32_t c = 0; c < nc; ++c)
            std::stable_sort(L.orig.begin() + L.cstart[(size_t)c], L.orig.begin() + L.cstart[(size_t)c + 1],
                             [&](int32_t x, int32_t y) { return s.type[x] < s.type[y]; });
    for (int32_t g = 0; g < n; ++g) L.inv[(size_t)L.orig[(size_t)g]] = g;
    L.type.assign((size_t)n, 0);
    if (s.type)
        for (int32_t g = 0; g < n; ++g) L.type[(size_t)g] = s.type[L.orig[(size_t)g]];
    L.row_ptr.resize((size_t)n + 1);
    L.col.resize((size_t)E);
    L.J.resize((size_t)E);
    L.row_ptr[0] = 0;
    int32_t deg0 = (int32_t)(s.row_ptr[1] - s.row_ptr[0]);
    bool uni_deg = true;
    for (int32_t g = 0; g < n; ++g) {
        const int32_t i = L.orig[(size_t)g];
        const int64_t b = s.row_ptr[i], d = s.row_ptr[i + 1] - b;
        if (d != deg0) uni_deg = false;
        const int64_t o = L.row_ptr[(size_t)g];
        for (int64_t k = 0; k < d; ++k) {
            L.col[(size_t)(o + k)] = L.inv[(size_t)s.col[b + k]];
            L.J[(size_t)(o + k)] = s.J[b + k];
        }
        L.row_ptr[(size_t)g + 1] = o + d;
    }
    L.uniform_degree = (uni_deg && deg0 > 0) ? deg0 : 0;

    // which classes see lower colours
    L.lower_mode.assign((size_t)nc, 0);
    for (int32_t c = 0; c < nc; ++c) {
        int64_t lo = 0, all = 0;
        for (int32_t g = L.cstart[(size_t)c]; g < L.cstart[(size_t)c + 1]; ++g)
            for (int64_t e = L.row_ptr[(size_t)g]; e < L.row_ptr[(size_t)g + 1]; ++e) {
                ++all;
                if (L.col[(size_t)e] < L.cstart[(size_t)c]) ++lo;
            }
        L.lower_mode[(size_t)c] = (lo == 0) ? 0 : (lo == all ? 1 : 2);
    }

    // parameters in the new numbering
    L.spin_norm.resize((size_t)n);
    L.field_axis.resize(3 * (size_t)n);
    L.k_uni.resize((size_t)n);
    L.e_uni.resize(3 * (size_t)n);
    L.k_cub.resize((size_t)n);
    for (int32_t g = 0; g < n; ++g) {
        const int64_t i = L.orig[(size_t)g];
        L.spin_norm[(size_t)g] = s.spin_norm ? s.spin_norm[i] : 1.0;
        for (int q = 0; q < 3; ++q) {
            L.field_axis[3 * (size_t)g + q] = s.field_axis ? s.field_axis[3 * i + q] : (q == 2 ? 1.0 : 0.0);
            L.e_uni[3 * (size_t)g + q] = s.e_uni ? s.e_uni[3 * i + q] : (q == 2 ? 1.0 : 0.0);
        }
        L.k_uni[(size_t)g] = s.k_uni ? s.k_uni[i] : 0.0;
        L.k_cub[(size_t)g] = s.k_cub ? s.k_cub[i] : 0.0;
    }
    bool uni = true, ani = false;
    for (int32_t g = 0; g < n && (uni || !ani); ++g) {
        if (L.k_uni[(size_t)g] != 0.0 || L.k_cub[(size_t)g] != 0.0) ani = true;
        if (L.spin_norm[(size_t)g] != L.spin_norm[0] || L.k_uni[(size_t)g] != L.k_uni[0] ||
            L.k_cub[(size_t)g] != L.k_cub[0])
            uni = false;
        for (int q = 0; q < 3; ++q)
            if (L.field_axis[3 * (size_t)g + q] != L.field_axis[(size_t)q] ||
                L.e_uni[3 * (size_t)g + q] != L.e_uni[(size_t)q])
                uni = false;
    }
    L.uniform_params = uni;
    L.has_anisotropy = ani;
    // update policies per type (Sec. II): per-site code and parameter in the new numbering
    L.policy.clear();
    L.policy_param.clear();
    L.has_adaptive = false;
    L.sigma0 = 0.0;
    if (s.n_policy_types < 0) { err = "n_policy_types < 0"; return false; }
    if (s.n_policy_types > 0) {
        const int32_t nt = s.n_policy_types;
        if (!s.type_policy || !s.type_param) { err = "type_policy or type_param is NULL"; return false; }
        std::vector<double> par((size_t)nt);
        bool any = false;
        for (int32_t q = 0; q < nt; ++q) {
            const int32_t code = s.type_policy[q];
            const double v = s.type_param[q];
            if (code < kPolRandom || code > kPolQIsing) { err = at("unknown update policy for type", q); return false; }
            if ((code == kPolSmallStep || code == kPolHinzkeNowak) && !(v > 0.0 && v <= 3.141592653589793))
                { err = at("cap half-angle outside (0, pi] for type", q); return false; }
            if ((code == kPolGaussian || code == kPolAdaptive) && !(v > 0.0 && std::isfinite(v)))
                { err = at("Gaussian width not finite and > 0 for type", q); return false; }
            // the cap height 1 - cos(theta) is computed once here, in FP64 with the host libm
            par[(size_t)q] = (code == kPolSmallStep || code == kPolHinzkeNowak) ? 1.0 - std::cos(v) : v;
            if (code != kPolRandom) any = true;
            if (code == kPolAdaptive && !L.has_adaptive) {
                L.has_adaptive = true;
                L.sigma0 = v;
            }
        }
        for (int32_t i = 0; i < n; ++i) {
            const int32_t ty = s.type ? s.type[i] : 0;
            if (ty < 0 || ty >= nt) { err = at("site type outside the policy table at site", i); return false; }
            if (s.type_policy[ty] == kPolQIsing) {  // 2 s must be a whole number of values, 1 .. 64
                const double two_s = 2.0 * (s.spin_norm ? s.spin_norm[i] : 1.0);
                if (two_s != std::floor(two_s) || two_s < 1.0 || two_s > 64.0) {
                    err = at("qIsing site needs a spin norm in {1/2, 1, ..., 32} at site", i);
                    return false;
                }
            }
        }
        if (any) {
            L.policy.resize((size_t)n);
            L.policy_param.resize((size_t)n);
            for (int32_t g = 0; g < n; ++g) {
                const int32_t ty = s.type ? s.type[L.orig[(size_t)g]] : 0;
                L.policy[(size_t)g] = s.type_policy[ty];
                L.policy_param[(size_t)g] = par[(size_t)ty];
            }
        }
    }
    if (s.init_spins) {
        L.init_spins.resize(3 * (size_t)n);
        for (int32_t g = 0; g < n; ++g)
            for (int q = 0; q < 3; ++q) L.init_spins[3 * (size_t)g + q] = s.init_spins[3 * (int64_t)L.orig[(size_t)g] + q];
    }
    return true;
}

}  // namespace vegas
