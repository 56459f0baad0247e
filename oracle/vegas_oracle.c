/*
 * CPU FP64 oracle of the Metropolis sweep of the classical Heisenberg model.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library's product path links, loads or calls
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline leg do.
 * It shares no code with the CUDA library: its Philox generator, sphere sampler, greedy
 * colouring and energy are written here again, from their published definitions.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no -ffast-math). FMA contraction must
 * stay off: the FP64 GPU path is compared with this code bit for bit.
 *
 * What it computes, with the paper's notation (Sec. III.A-B):
 *   Energy (Eq. 1-3), S_i = s_i * unit vector, each undirected bond counted once:
 *     E = -1/2 sum_i sum_{j in N(i)} J_ij S_i.S_j - B sum_i S_i.n_i
 *         - sum_i k_i (S_i.e_i)^2 - sum_i kc_i (Sx^2 Sy^2 + Sy^2 Sz^2 + Sx^2 Sz^2)_i
 *     The anisotropy enters Eq. 1 with a minus sign, so k > 0 is an easy axis.
 *   Metropolis step (Eq. 4): trial S' uniform on the sphere of radius s_i ("random"
 *     update policy); accept when dE <= 0, else when u < exp(-dE / T), k_B = 1.
 *   One MCS = one attempt per spin. Mode 0 sweeps the colour classes of a proper
 *     colouring in colour order (sites of one class are not linked, so any order inside a
 *     class gives the same result; increasing site id is used). Mode 1 is the paper's
 *     literal form: N attempts on uniformly drawn sites.
 *   History: after every MCS, E from the definition above and M = sum_i S_i (Sec. II).
 *   After the last MCS of each temperature/field step every spin is rescaled to its norm
 *     s_i (periodic renormalisation of |S|).
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key = (seed low 32
 * bits, seed high 32 bits), counter = (site, MCS t, instance, purpose | k):
 *   purpose 0x00000|k  trial candidate k of the sphere sampler
 *   purpose 0x10000    acceptance uniform
 *   purpose 0x20000|k  initial spin candidate k (with t = 0xFFFFFFFF)
 *   purposes 0x50000 (site pick), 0x60000|k (trial), 0x70000 (acceptance) in mode 1,
 *     where the first counter word is the attempt index instead of the site.
 * Sphere sampler: Marsaglia, Ann. Math. Stat. 43 (1972) 645: a, b uniform in [0,1) from
 *   53-bit words, u1 = 2a-1, u2 = 2b-1, s = u1^2+u2^2, reject s >= 1, then
 *   (2 u1 sqrt(1-s), 2 u2 sqrt(1-s), 1-2s). Uses only correctly rounded operations.
 *
 * Update policies (Sec. II, Sec. III.B, Sec. IV.C; the paper names them without formulas,
 * these are the readings; every proposal depends only on the angle between S and S', so it
 * is symmetric and plain Metropolis acceptance stays exact):
 *   0 random        S' uniform on the sphere (Marsaglia, above)
 *   1 spin flip     S' = -S
 *   2 small step    S' uniform in the cap of half-angle theta around S: a disk point
 *                   (u1, u2) as in Marsaglia gives s uniform in [0,1) and an azimuth, and
 *                   z = 1 - s h, (x, y) = (u1, u2) sqrt(h (2 - s h)) with h = 1 - cos theta,
 *                   placed in an orthonormal frame (e1, e2, S/|S|)
 *   3 Gaussian      S' = s_i (S/|S| + sigma g)/|...|, g three standard normals by the polar
 *                   method (Marsaglia & Bray 1964) with candidates of purpose 0x00000|k and
 *                   0x08000|k
 *   4 Hinzke-Nowak  one of spin flip, random, small step with probability 1/3 each, chosen by
 *                   the uniform of purpose 0x0C000 (Hinzke & Nowak 1999 combinational move)
 *   6 qIsing        mixed-spin Ising (Sec. II): S = (0, 0, m) with m in {-s, -s + 1, ..., s}
 *                   (s = the spin norm, 2 s a positive integer); the trial m' is uniform over
 *                   the 2 s other values: k = floor(u * 2 s) from the uniform of purpose
 *                   0x00000, m' = k - s if k < index(m) else k + 1 - s. Such sites start at a
 *                   uniform value (the init uniform u, index floor(u (2 s + 1))) and are never
 *                   renormalised.
 *   5 adaptive      Gaussian whose width sigma (one per instance) is rescaled after each MCS by
 *                   0.5 / max(1 - R, 0.01), R the MCS's acceptance rate, clamped to
 *                   [1e-4, 100], during the first fifth of every temperature/field step only;
 *                   it is then frozen, so the measured part is a plain Metropolis chain.
 * The policy of a site comes from its type through a table (a policy per magnetic phase).
 * Logarithms are computed here with the atanh series (Abramowitz & Stegun 4.1.27), not libm,
 * so that any implementation of the same series gives the same bits.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t n;
    int32_t pad_;
    const int64_t *row_ptr;
    const int32_t *col;
    const double *J;
    const double *spin_norm;  /* NULL: all 1 */
    const double *field_axis; /* NULL: all +z */
    const double *k_uni;      /* NULL: all 0 */
    const double *e_uni;      /* NULL: all +z */
    const double *k_cub;      /* NULL: all 0 */
    const int32_t *type;      /* NULL: all 0 */
    const int32_t *type_policy; /* [n_policy_types] or NULL: every site random */
    const double *type_param;   /* [n_policy_types]: theta (2, 4) or sigma (3, 5) */
    int32_t n_policy_types;
    int32_t pad2_;
} vo_sample;

enum { VO_RANDOM = 0, VO_FLIP = 1, VO_SMALL_STEP = 2, VO_GAUSSIAN = 3, VO_HINZKE_NOWAK = 4, VO_ADAPTIVE = 5,
       VO_QISING = 6 };

enum { VO_ERR_NAN = 1, VO_ERR_SPHERE = 2 };

/* ---------------------------------------------------------------- Philox4x32-10 */

static void philox_round(uint32_t c[4], uint32_t k0, uint32_t k1) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k0;
    const uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

void vo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        philox_round(c, k0, k1);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    memcpy(out, c, sizeof c);
}

static void philox(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t w[4]) {
    const uint32_t ctr[4] = {c0, c1, c2, c3};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    vo_philox4x32_10(ctr, key, w);
}

/* 53-bit uniform in [0, 1) from two words: (hi * 2^21 + lo >> 11) * 2^-53. */
static double u53(uint32_t hi, uint32_t lo) {
    const uint64_t m = ((uint64_t)hi << 21) | (uint64_t)(lo >> 11);
    return (double)m * 0x1p-53;
}

/* Marsaglia (1972) point on the unit sphere; returns candidates used, or -1 past 64. */
int vo_sphere(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t purpose, double out[3]) {
    for (uint32_t k = 0; k < 64; ++k) {
        uint32_t w[4];
        philox(seed, c0, c1, c2, purpose | k, w);
        const double a = u53(w[0], w[1]);
        const double b = u53(w[2], w[3]);
        const double u1 = 2.0 * a - 1.0;
        const double u2 = 2.0 * b - 1.0;
        const double s = u1 * u1 + u2 * u2;
        if (s >= 1.0) continue;
        const double q = sqrt(1.0 - s);
        out[0] = (2.0 * u1) * q;
        out[1] = (2.0 * u2) * q;
        out[2] = 1.0 - 2.0 * s;
        return (int)k + 1;
    }
    out[0] = 0.0;
    out[1] = 0.0;
    out[2] = 1.0;
    return -1;
}

/* Uniform in [0, 1) from one Philox block (the acceptance draw of Eq. 4). */
double vo_uniform(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3) {
    uint32_t w[4];
    philox(seed, c0, c1, c2, c3, w);
    return u53(w[0], w[1]);
}

/* ---------------------------------------------------------------- policy helpers */

/* ln x for finite x > 0 (normal): x = m 2^e with m in [sqrt(1/2), sqrt 2), ln m = 2 atanh t,
 * t = (m-1)/(m+1), atanh t = sum t^(2j+1)/(2j+1) to j = 13 (|t| <= 0.172: error < 1e-20). */
double vo_log(double x) {
    uint64_t bits;
    memcpy(&bits, &x, sizeof bits);
    int32_t e = (int32_t)((bits >> 52) & 0x7FF) - 1023;
    bits = (bits & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull;
    double m;
    memcpy(&m, &bits, sizeof m);
    if (m > 1.4142135623730951) {
        m = m * 0.5;
        e = e + 1;
    }
    const double t = (m - 1.0) / (m + 1.0);
    const double t2 = t * t;
    double p = 1.0 / 27.0;
    for (int32_t k = 25; k >= 1; k -= 2) p = p * t2 + 1.0 / (double)k;
    return (2.0 * t) * p + (double)e * 0.6931471805599453;
}

/* Two standard normals by the polar method; candidates k use counter word 3 = purpose|k.
 * Returns 0 past 64 candidates (then both are 0). */
static int normal_pair(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t purpose, double g[2]) {
    for (uint32_t k = 0; k < 64; ++k) {
        uint32_t w[4];
        philox(seed, c0, c1, c2, purpose | k, w);
        const double u1 = 2.0 * u53(w[0], w[1]) - 1.0;
        const double u2 = 2.0 * u53(w[2], w[3]) - 1.0;
        const double s = u1 * u1 + u2 * u2;
        if (s >= 1.0 || s == 0.0) continue;
        const double f = sqrt((-2.0 * vo_log(s)) / s);
        g[0] = u1 * f;
        g[1] = u2 * f;
        return 1;
    }
    g[0] = g[1] = 0.0;
    return 0;
}

/* u = v / |v|. */
static void unit_of(const double v[3], double u[3]) {
    const double q = sqrt((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2]);
    u[0] = v[0] / q;
    u[1] = v[1] / q;
    u[2] = v[2] / q;
}

/* Orthonormal frame around the unit vector u: e1 = unit(a x u) with a the coordinate axis of
 * the smallest |u_k| (first on ties), e2 = u x e1. */
static void frame_of(const double u[3], double e1[3], double e2[3]) {
    const double ax = fabs(u[0]), ay = fabs(u[1]), az = fabs(u[2]);
    double c[3];
    if (ax <= ay && ax <= az) {
        c[0] = 0.0; c[1] = -u[2]; c[2] = u[1];
    } else if (ay <= az) {
        c[0] = u[2]; c[1] = 0.0; c[2] = -u[0];
    } else {
        c[0] = -u[1]; c[1] = u[0]; c[2] = 0.0;
    }
    unit_of(c, e1);
    e2[0] = u[1] * e1[2] - u[2] * e1[1];
    e2[1] = u[2] * e1[0] - u[0] * e1[2];
    e2[2] = u[0] * e1[1] - u[1] * e1[0];
}

/* Point uniform in the cap of height h = 1 - cos(theta) around the unit vector u. */
static int cap_point(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t purpose, const double u[3],
                     double h, double out[3]) {
    for (uint32_t k = 0; k < 64; ++k) {
        uint32_t w[4];
        philox(seed, c0, c1, c2, purpose | k, w);
        const double u1 = 2.0 * u53(w[0], w[1]) - 1.0;
        const double u2 = 2.0 * u53(w[2], w[3]) - 1.0;
        const double s = u1 * u1 + u2 * u2;
        if (s >= 1.0) continue;
        const double sh = s * h;
        const double z = 1.0 - sh;
        const double r = sqrt(h * (2.0 - sh));
        const double x = u1 * r, y = u2 * r;
        double e1[3], e2[3];
        frame_of(u, e1, e2);
        for (int q = 0; q < 3; ++q) out[q] = (x * e1[q] + y * e2[q]) + z * u[q];
        return 1;
    }
    out[0] = u[0];
    out[1] = u[1];
    out[2] = u[2];
    return 0;
}

double vo_cap_height(double theta) { return 1.0 - cos(theta); }

/* ---------------------------------------------------------------- colouring */

/* Greedy colouring: visit sites in index order, give each the smallest colour not used by
 * an already coloured neighbour. Returns the number of colours. */
int32_t vo_greedy_colour(int32_t n, const int64_t *row_ptr, const int32_t *col, int32_t *colour) {
    int32_t nc = 0;
    int32_t cap = 64;
    int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    for (int32_t c = 0; c < cap; ++c) mark[c] = -1;
    for (int32_t i = 0; i < n; ++i) colour[i] = -1;
    for (int32_t i = 0; i < n; ++i) {
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int32_t j = col[e];
            const int32_t cj = colour[j];
            if (cj >= 0) mark[cj] = i; /* every assigned colour is < cap */
        }
        int32_t c = 0;
        while (c < cap && mark[c] == i) ++c;
        if (c == cap) {
            int32_t ncap = cap * 2;
            mark = (int32_t *)realloc(mark, sizeof(int32_t) * (size_t)ncap);
            for (int32_t q = cap; q < ncap; ++q) mark[q] = -1;
            cap = ncap;
        }
        colour[i] = c;
        if (c + 1 > nc) nc = c + 1;
    }
    free(mark);
    return nc;
}

/* ---------------------------------------------------------------- energy */

/* Spin norm s_i of the material file (Sec. III.C); 1 when not given. */
static double norm_of(const vo_sample *s, int32_t i) { return s->spin_norm ? s->spin_norm[i] : 1.0; }

/* Per-site axis (field axis n_i or anisotropy axis e_i); +z when not given. */
static void axis_of(const double *a, int32_t i, double v[3]) {
    if (a) {
        v[0] = a[3 * (int64_t)i];
        v[1] = a[3 * (int64_t)i + 1];
        v[2] = a[3 * (int64_t)i + 2];
    } else {
        v[0] = 0.0;
        v[1] = 0.0;
        v[2] = 1.0;
    }
}

/* Cubic anisotropy form of Eq. 3: x^2 y^2 + y^2 z^2 + x^2 z^2 of the spin's components. */
static double cubic_form(const double v[3]) {
    const double xx = v[0] * v[0], yy = v[1] * v[1], zz = v[2] * v[2];
    return (xx * yy + yy * zz) + xx * zz;
}

/* Energy of site i's own terms plus half of its bonds (Eq. 1-3). */
static double site_energy(const vo_sample *s, const double *S, int32_t i, double B) {
    const double *Si = S + 3 * (int64_t)i;
    double ex = 0.0;
    for (int64_t e = s->row_ptr[i]; e < s->row_ptr[i + 1]; ++e) {
        const double *Sj = S + 3 * (int64_t)s->col[e];
        ex += s->J[e] * ((Si[0] * Sj[0] + Si[1] * Sj[1]) + Si[2] * Sj[2]);
    }
    double n[3], ea[3];
    axis_of(s->field_axis, i, n);
    axis_of(s->e_uni, i, ea);
    const double k = s->k_uni ? s->k_uni[i] : 0.0;
    const double kc = s->k_cub ? s->k_cub[i] : 0.0;
    const double zee = (Si[0] * n[0] + Si[1] * n[1]) + Si[2] * n[2];
    const double pe = (Si[0] * ea[0] + Si[1] * ea[1]) + Si[2] * ea[2];
    return -0.5 * ex - B * zee - k * (pe * pe) - kc * cubic_form(Si);
}

/* Total energy (Eq. 1-3): the sum of the site energies, so every bond counts once. */
double vo_energy(const vo_sample *s, const double *S, double B) {
    double E = 0.0;
    for (int32_t i = 0; i < s->n; ++i) E += site_energy(s, S, i, B);
    return E;
}

/* M = sum_i S_i, the magnetization recorded after every MCS (Sec. II). */
void vo_magnetisation(int32_t n, const double *S, double M[3]) {
    M[0] = M[1] = M[2] = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        M[0] += S[3 * (int64_t)i];
        M[1] += S[3 * (int64_t)i + 1];
        M[2] += S[3 * (int64_t)i + 2];
    }
}

/* Energy change of replacing S_i by Sp (Eq. 1-3), evaluated in a fixed order:
 * h = sum_j J_ij S_j (row order) + B n_i; d = Sp - S_i;
 * dE = (-(d.h) - k((Sp.e)^2 - (S.e)^2)) - kc(cub(Sp) - cub(S)). */
double vo_delta_e(const vo_sample *s, const double *S, int32_t i, const double Sp[3], double B) {
    double hx = 0.0, hy = 0.0, hz = 0.0;
    for (int64_t e = s->row_ptr[i]; e < s->row_ptr[i + 1]; ++e) {
        const double *Sj = S + 3 * (int64_t)s->col[e];
        const double J = s->J[e];
        hx = hx + J * Sj[0];
        hy = hy + J * Sj[1];
        hz = hz + J * Sj[2];
    }
    double n[3], ea[3];
    axis_of(s->field_axis, i, n);
    axis_of(s->e_uni, i, ea);
    hx = hx + B * n[0];
    hy = hy + B * n[1];
    hz = hz + B * n[2];
    const double *Si = S + 3 * (int64_t)i;
    const double dx = Sp[0] - Si[0], dy = Sp[1] - Si[1], dz = Sp[2] - Si[2];
    const double dEex = -((dx * hx + dy * hy) + dz * hz);
    const double k = s->k_uni ? s->k_uni[i] : 0.0;
    const double kc = s->k_cub ? s->k_cub[i] : 0.0;
    const double pn = (Sp[0] * ea[0] + Sp[1] * ea[1]) + Sp[2] * ea[2];
    const double po = (Si[0] * ea[0] + Si[1] * ea[1]) + Si[2] * ea[2];
    const double dEan = -(k * (pn * pn - po * po));
    const double dEcub = -(kc * (cubic_form(Sp) - cubic_form(Si)));
    return (dEex + dEan) + dEcub;
}

/* 1 when site i follows the qIsing policy (discrete values along z). */
static int is_qising(const vo_sample *s, int32_t i) {
    if (!s->type_policy) return 0;
    const int32_t ty = s->type ? s->type[i] : 0;
    return ty >= 0 && ty < s->n_policy_types && s->type_policy[ty] == VO_QISING;
}

/* Renormalisation once per temperature/field step: S_i <- s_i * S_i / |S_i|, with
 * f = s_i / sqrt((x^2 + y^2) + z^2); qIsing sites keep their length. */
void vo_renormalise(const vo_sample *s, double *S) {
    for (int32_t i = 0; i < s->n; ++i) {
        if (is_qising(s, i)) continue;  /* discrete values keep their length */
        double *v = S + 3 * (int64_t)i;
        const double n2 = (v[0] * v[0] + v[1] * v[1]) + v[2] * v[2];
        const double f = norm_of(s, i) / sqrt(n2);
        v[0] = v[0] * f;
        v[1] = v[1] * f;
        v[2] = v[2] * f;
    }
}

/* Initial state: S_i = s_i * sphere(counter = (i, 0xFFFFFFFF, inst, 0x20000 | k)). */
int vo_init_spins(const vo_sample *s, uint64_t seed, int32_t inst, double *S) {
    int err = 0;
    for (int32_t i = 0; i < s->n; ++i) {
        const double sn = norm_of(s, i);
        if (is_qising(s, i)) {  /* a uniform value of {-s, ..., s} along z */
            const int32_t nv = (int32_t)(2.0 * sn) + 1;
            int32_t k = (int32_t)(vo_uniform(seed, (uint32_t)i, 0xFFFFFFFFu, (uint32_t)inst, 0x20000u) * (double)nv);
            if (k >= nv) k = nv - 1;
            S[3 * (int64_t)i] = 0.0;
            S[3 * (int64_t)i + 1] = 0.0;
            S[3 * (int64_t)i + 2] = (double)k - sn;
            continue;
        }
        double u[3];
        if (vo_sphere(seed, (uint32_t)i, 0xFFFFFFFFu, (uint32_t)inst, 0x20000u, u) < 0) err |= VO_ERR_SPHERE;
        S[3 * (int64_t)i] = sn * u[0];
        S[3 * (int64_t)i + 1] = sn * u[1];
        S[3 * (int64_t)i + 2] = sn * u[2];
    }
    return err;
}

/* ---------------------------------------------------------------- the Markov chain */

typedef struct {
    const vo_sample *s;
    const int32_t *order;   /* sites in sweep order: colour 0 by id, colour 1 by id, ... */
    uint64_t seed;
    int32_t inst;
    const double *T, *B;    /* this instance's schedule, n_steps entries */
    int32_t n_steps, mcs;
    uint32_t t0;
    double *S;              /* n*3 */
    double *hist;           /* n_steps*mcs*4 */
    uint8_t *accept_log;    /* log_mcs*n or NULL */
    int32_t log_mcs;
    int32_t mode;
    int err;
    int64_t *acc_hist;      /* n_steps*mcs accepted attempts, or NULL */
    double sigma;           /* adaptive width of this instance */
    int has_adaptive;
    double *type_hist;      /* n_steps*mcs*n_types*3 magnetization per site type, or NULL */
    int32_t n_types;
    double *snaps;          /* n_steps*n*3 spins after every step, or NULL */
} vo_job;

/* Optional outputs of vo_run_ex (any pointer may be NULL). */
typedef struct {
    int64_t *acc_hist;      /* [n_inst][n_steps*mcs] accepted attempts per MCS */
    double *sigma_inout;    /* [n_inst] adaptive widths: in (<= 0: the policy's parameter), out */
    double *type_hist;      /* [n_inst][n_steps*mcs][n_types][3] sum of S_i over the sites of each type */
    int32_t n_types;
    int32_t pad_;
    double *snaps;          /* [n_inst][n_steps][n][3] spins at the end of every step (after the
                               renormalisation): the final state per temperature/field step */
} vo_extra;

static void policy_of(const vo_sample *s, int32_t i, int32_t *pol, double *par) {
    *pol = VO_RANDOM;
    *par = 0.0;
    if (!s->type_policy) return;
    const int32_t ty = s->type ? s->type[i] : 0;
    if (ty >= 0 && ty < s->n_policy_types) {
        *pol = s->type_policy[ty];
        *par = s->type_param[ty];
    }
}

/* Trial state of site i under its update policy (unit vector before the spin norm). */
static void trial_of(vo_job *jb, int32_t i, uint32_t c0, uint32_t t, uint32_t p_trial, double out[3]) {
    const vo_sample *s = jb->s;
    const uint32_t inst = (uint32_t)jb->inst;
    int32_t pol;
    double par;
    policy_of(s, i, &pol, &par);
    const double *Si = jb->S + 3 * (int64_t)i;
    if (pol == VO_HINZKE_NOWAK) {
        const double v = vo_uniform(jb->seed, c0, t, inst, 0x0C000u) * 3.0;
        pol = v < 1.0 ? VO_FLIP : (v < 2.0 ? VO_RANDOM : VO_SMALL_STEP);
    }
    if (pol == VO_FLIP) {
        const double sn = norm_of(s, i);
        out[0] = -Si[0] / sn;
        out[1] = -Si[1] / sn;
        out[2] = -Si[2] / sn;
        return;
    }
    if (pol == VO_SMALL_STEP) {
        double u[3];
        unit_of(Si, u);
        if (!cap_point(jb->seed, c0, t, inst, p_trial, u, vo_cap_height(par), out)) jb->err |= VO_ERR_SPHERE;
        return;
    }
    if (pol == VO_GAUSSIAN || pol == VO_ADAPTIVE) {
        const double sigma = pol == VO_ADAPTIVE ? jb->sigma : par;
        double u[3], g0[2], g1[2];
        unit_of(Si, u);
        if (!normal_pair(jb->seed, c0, t, inst, p_trial, g0)) jb->err |= VO_ERR_SPHERE;
        if (!normal_pair(jb->seed, c0, t, inst, p_trial | 0x08000u, g1)) jb->err |= VO_ERR_SPHERE;
        const double v[3] = {u[0] + sigma * g0[0], u[1] + sigma * g0[1], u[2] + sigma * g1[0]};
        unit_of(v, out);
        return;
    }
    if (vo_sphere(jb->seed, c0, t, inst, p_trial, out) < 0) jb->err |= VO_ERR_SPHERE;
}

/* Trial state of site i (unit vector) for the given spins and adaptive width, counters
 * (i, t, inst, purpose 0): the sampler attempts use, exposed for the distribution pins. */
int vo_trial(const vo_sample *s, const double *S, int32_t i, uint64_t seed, uint32_t t, int32_t inst, double sigma,
             double *out) {
    vo_job jb;
    memset(&jb, 0, sizeof jb);
    jb.s = s;
    jb.S = (double *)S;
    jb.seed = seed;
    jb.inst = inst;
    jb.sigma = sigma;
    trial_of(&jb, i, (uint32_t)i, t, 0x00000u, out);
    return jb.err;
}

/* One Metropolis attempt on site i (Eq. 4). Trial and acceptance counters are
 * (c0, t, inst, purpose). Returns 1 when accepted. */
static int attempt(vo_job *jb, int32_t i, uint32_t c0, uint32_t t, double beta, double B, uint32_t p_trial,
                   uint32_t p_accept) {
    const vo_sample *s = jb->s;
    const double sn = norm_of(s, i);
    double Sp[3];
    if (is_qising(s, i)) {  /* another of the 2 s + 1 values along z, uniformly */
        const int32_t n2 = (int32_t)(2.0 * sn);
        const int32_t idx = (int32_t)(jb->S[3 * (int64_t)i + 2] + sn + 0.5);
        int32_t k = (int32_t)(vo_uniform(jb->seed, c0, t, (uint32_t)jb->inst, p_trial) * (double)n2);
        if (k >= n2) k = n2 - 1;
        if (k >= idx) k += 1;
        Sp[0] = 0.0;
        Sp[1] = 0.0;
        Sp[2] = (double)k - sn;
    } else {
        double u[3];
        trial_of(jb, i, c0, t, p_trial, u);
        Sp[0] = sn * u[0];
        Sp[1] = sn * u[1];
        Sp[2] = sn * u[2];
    }
    const double dE = vo_delta_e(s, jb->S, i, Sp, B);
    int acc;
    if (dE <= 0.0) {
        acc = 1;
    } else {
        const double r = vo_uniform(jb->seed, c0, t, (uint32_t)jb->inst, p_accept);
        acc = r < exp(-(beta * dE));
    }
    if (isnan(dE)) {
        jb->err |= VO_ERR_NAN;
        acc = 0;
    }
    if (acc) {
        double *Si = jb->S + 3 * (int64_t)i;
        Si[0] = Sp[0];
        Si[1] = Sp[1];
        Si[2] = Sp[2];
    }
    return acc;
}

static void *run_job(void *arg) {
    vo_job *jb = (vo_job *)arg;
    const vo_sample *s = jb->s;
    const int32_t n = s->n;
    uint32_t t = jb->t0;
    int64_t rec = 0;
    for (int32_t st = 0; st < jb->n_steps; ++st) {
        const double beta = 1.0 / jb->T[st];
        const double B = jb->B[st];
        for (int32_t m = 0; m < jb->mcs; ++m) {
            const int64_t mrun = (int64_t)st * jb->mcs + m;
            uint8_t *log = (jb->accept_log && mrun < jb->log_mcs) ? jb->accept_log + mrun * n : NULL;
            int64_t accepted = 0;
            if (jb->mode == 0) {
                for (int32_t q = 0; q < n; ++q) {
                    const int32_t i = jb->order[q];
                    const int a = attempt(jb, i, (uint32_t)i, t, beta, B, 0x00000u, 0x10000u);
                    accepted += a;
                    if (log) log[i] = (uint8_t)a;
                }
            } else {
                for (int32_t a = 0; a < n; ++a) {
                    const double r = vo_uniform(jb->seed, (uint32_t)a, t, (uint32_t)jb->inst, 0x50000u);
                    int32_t i = (int32_t)(r * (double)n);
                    if (i >= n) i = n - 1;
                    accepted += attempt(jb, i, (uint32_t)a, t, beta, B, 0x60000u, 0x70000u);
                }
            }
            if (jb->acc_hist) jb->acc_hist[rec] = accepted;
            if (jb->has_adaptive && m < jb->mcs / 5) {  /* adapt during the first fifth of the step */
                const double rate = (double)accepted / (double)n;
                double f = 1.0 - rate;
                if (f < 0.01) f = 0.01;
                double sg = jb->sigma * (0.5 / f);
                if (sg < 1e-4) sg = 1e-4;
                if (sg > 100.0) sg = 100.0;
                jb->sigma = sg;
            }
            double M[3];
            vo_magnetisation(n, jb->S, M);
            double *h = jb->hist + rec * 4;
            h[0] = vo_energy(s, jb->S, B);
            h[1] = M[0];
            h[2] = M[1];
            h[3] = M[2];
            if (jb->type_hist) {  /* statistics of each magnetic phase (Sec. II): M per type */
                double *th = jb->type_hist + rec * jb->n_types * 3;
                for (int32_t k = 0; k < 3 * jb->n_types; ++k) th[k] = 0.0;
                for (int32_t i = 0; i < n; ++i) {
                    const int32_t ty = s->type ? s->type[i] : 0;
                    if (ty < 0 || ty >= jb->n_types) continue;
                    for (int q = 0; q < 3; ++q) th[3 * ty + q] += jb->S[3 * (int64_t)i + q];
                }
            }
            ++rec;
            ++t;
        }
        vo_renormalise(s, jb->S);
        if (jb->snaps) memcpy(jb->snaps + (int64_t)st * n * 3, jb->S, sizeof(double) * 3 * (size_t)n);
    }
    return NULL;
}

/*
 * Run n_inst instances of one sample (replicas inst_base .. inst_base+n_inst-1) through
 * n_steps temperature/field steps of mcs MCS each, starting at global MCS counter t0.
 *   colour    NULL: greedy colouring; else a colouring (not checked for properness here)
 *   T, B      [n_inst][n_steps]
 *   spins     [n_inst][n][3], in/out; when init != 0 it is first filled by vo_init_spins
 *   history   [n_inst][n_steps*mcs][4] = (E, Mx, My, Mz) after every MCS
 *   accept_log NULL or [n_inst][log_mcs][n] bytes, 1 where the attempt at that site in
 *             that MCS was accepted (mode 0 only)
 * Returns the OR of VO_ERR_* over instances, or -1 on invalid arguments.
 */
int vo_run_ex(const vo_sample *s, const int32_t *colour, uint64_t seed, int32_t n_inst, int32_t inst_base,
              const double *T, const double *B, int32_t n_steps, int32_t mcs, uint32_t t0, double *spins,
              int32_t init, double *history, uint8_t *accept_log, int32_t log_mcs, int32_t mode, int32_t n_threads,
              const vo_extra *x);

int vo_run(const vo_sample *s, const int32_t *colour, uint64_t seed, int32_t n_inst, int32_t inst_base,
           const double *T, const double *B, int32_t n_steps, int32_t mcs, uint32_t t0, double *spins, int32_t init,
           double *history, uint8_t *accept_log, int32_t log_mcs, int32_t mode, int32_t n_threads) {
    return vo_run_ex(s, colour, seed, n_inst, inst_base, T, B, n_steps, mcs, t0, spins, init, history, accept_log,
                     log_mcs, mode, n_threads, NULL);
}

/* As vo_run, plus the optional outputs of x (see vo_extra). */
int vo_run_ex(const vo_sample *s, const int32_t *colour, uint64_t seed, int32_t n_inst, int32_t inst_base,
              const double *T, const double *B, int32_t n_steps, int32_t mcs, uint32_t t0, double *spins,
              int32_t init, double *history, uint8_t *accept_log, int32_t log_mcs, int32_t mode, int32_t n_threads,
              const vo_extra *x) {
    int64_t *acc_hist = x ? x->acc_hist : NULL;
    double *sigma_inout = x ? x->sigma_inout : NULL;
    if (!s || s->n < 0 || n_inst < 1 || n_steps < 0 || mcs < 0 || !T || !B || !spins || !history) return -1;
    const int32_t n = s->n;
    int32_t *col_own = NULL;
    const int32_t *cl = colour;
    int32_t nc = 0;
    if (!cl) {
        col_own = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        nc = vo_greedy_colour(n, s->row_ptr, s->col, col_own);
        cl = col_own;
    } else {
        for (int32_t i = 0; i < n; ++i)
            if (cl[i] + 1 > nc) nc = cl[i] + 1;
    }
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t q = 0;
    for (int32_t c = 0; c < nc; ++c)
        for (int32_t i = 0; i < n; ++i)
            if (cl[i] == c) order[q++] = i;

    vo_job *jobs = (vo_job *)calloc((size_t)n_inst, sizeof(vo_job));
    int err = 0;
    for (int32_t r = 0; r < n_inst; ++r) {
        vo_job *jb = &jobs[r];
        jb->s = s;
        jb->order = order;
        jb->seed = seed;
        jb->inst = inst_base + r;
        jb->T = T + (int64_t)r * n_steps;
        jb->B = B + (int64_t)r * n_steps;
        jb->n_steps = n_steps;
        jb->mcs = mcs;
        jb->t0 = t0;
        jb->S = spins + (int64_t)r * n * 3;
        jb->hist = history + (int64_t)r * n_steps * mcs * 4;
        jb->accept_log = accept_log ? accept_log + (int64_t)r * log_mcs * n : NULL;
        jb->log_mcs = log_mcs;
        jb->mode = mode;
        jb->acc_hist = acc_hist ? acc_hist + (int64_t)r * n_steps * mcs : NULL;
        jb->n_types = x ? x->n_types : 0;
        jb->type_hist = (x && x->type_hist && x->n_types > 0)
                            ? x->type_hist + (int64_t)r * n_steps * mcs * x->n_types * 3 : NULL;
        jb->snaps = (x && x->snaps) ? x->snaps + (int64_t)r * n_steps * s->n * 3 : NULL;
        jb->has_adaptive = 0;
        jb->sigma = 0.0;
        if (s->type_policy)
            for (int32_t ty = 0; ty < s->n_policy_types; ++ty)
                if (s->type_policy[ty] == VO_ADAPTIVE && !jb->has_adaptive) {
                    jb->has_adaptive = 1;
                    jb->sigma = s->type_param[ty];
                }
        if (sigma_inout && sigma_inout[r] > 0.0) jb->sigma = sigma_inout[r];
        if (init) err |= vo_init_spins(s, seed, jb->inst, jb->S);
    }
    if (n_threads < 1) n_threads = 1;
    if (n_threads > n_inst) n_threads = n_inst;
    /* instances r, r + n_threads, ... run on thread r */
    for (int32_t base = 0; base < n_inst; base += n_threads) {
        pthread_t th[256];
        int32_t cnt = 0;
        for (int32_t r = base; r < n_inst && cnt < n_threads && cnt < 256; ++r, ++cnt) {
            if (n_threads == 1) {
                run_job(&jobs[r]);
            } else {
                pthread_create(&th[cnt], NULL, run_job, &jobs[r]);
            }
        }
        if (n_threads > 1)
            for (int32_t k = 0; k < cnt; ++k) pthread_join(th[k], NULL);
    }
    for (int32_t r = 0; r < n_inst; ++r) {
        err |= jobs[r].err;
        if (sigma_inout) sigma_inout[r] = jobs[r].sigma;
    }
    free(jobs);
    free(order);
    free(col_own);
    return err;
}

/* ---------------------------------------------------------------- Ising model (spin flip)
 * The Ising limit of Eq. 1 (Sec. II: Ising systems updated with the spin-flip policy):
 * s_i = +-1 on a periodic square (dims 2) or simple cubic (dims 3) lattice of even side L,
 * site id i = x + L (y + L z), E = -J sum_<ij> s_i s_j - h sum_i s_i (each bond once).
 * One MCS: every site of colour 0 ((x + y + z) even) in increasing id, then colour 1.
 * Attempt (Eq. 4): dE = 2 s_i (J sum_j s_j + h); accept iff dE <= 0 or u < exp(-(beta dE)),
 * where u = w 2^-32 and w is word (inst & 3) of Philox(seed; i, t, inst >> 2, 0x80000).
 * Initial state: s_i = +1 iff bit 31 of word (inst & 3) of Philox(seed; i, 0xFFFFFFFF,
 * inst >> 2, 0x90000) is set.
 */
static void ising_coords(int32_t dims, int32_t L, int32_t i, int32_t c[3]) {
    c[0] = i % L;
    c[1] = (i / L) % L;
    c[2] = dims == 3 ? i / (L * L) : 0;
}

static int32_t ising_id(int32_t dims, int32_t L, const int32_t c[3]) {
    (void)dims;
    return c[0] + L * (c[1] + L * c[2]);
}

/* Neighbour ids of site i: -x, +x, -y, +y (, -z, +z); returns the count. */
static int ising_neighbours(int32_t dims, int32_t L, int32_t i, int32_t nb[6]) {
    int32_t c[3];
    ising_coords(dims, L, i, c);
    int k = 0;
    for (int d = 0; d < dims; ++d)
        for (int sgn = -1; sgn <= 1; sgn += 2) {
            int32_t q[3] = {c[0], c[1], c[2]};
            q[d] = (q[d] + sgn + L) % L;
            nb[k++] = ising_id(dims, L, q);
        }
    return k;
}

int vo_ising_run(int32_t dims, int32_t L, double J, uint64_t seed, int32_t n_rep, int32_t inst_base,
                 const double *T, const double *h, int32_t n_steps, int32_t mcs, uint32_t t0, int8_t *spins,
                 int32_t init, double *history) {
    if ((dims != 2 && dims != 3) || L < 4 || (L & 1) || n_rep < 1 || inst_base < 0) return -1;
    const int32_t n = dims == 3 ? L * L * L : L * L;
    for (int32_t r = 0; r < n_rep; ++r) {
        const uint32_t inst = (uint32_t)(inst_base + r);
        int8_t *s = spins + (int64_t)r * n;
        if (init)
            for (int32_t i = 0; i < n; ++i) {
                uint32_t w[4];
                philox(seed, (uint32_t)i, 0xFFFFFFFFu, inst >> 2, 0x90000u, w);
                s[i] = (w[inst & 3u] >> 31) ? 1 : -1;
            }
        uint32_t t = t0;
        int64_t rec = 0;
        for (int32_t st = 0; st < n_steps; ++st) {
            const double beta = 1.0 / T[(int64_t)r * n_steps + st];
            const double hh = h[(int64_t)r * n_steps + st];
            for (int32_t m = 0; m < mcs; ++m) {
                for (int32_t colour = 0; colour < 2; ++colour)
                    for (int32_t i = 0; i < n; ++i) {
                        int32_t c[3], nb[6];
                        ising_coords(dims, L, i, c);
                        if (((c[0] + c[1] + c[2]) & 1) != colour) continue;
                        const int z = ising_neighbours(dims, L, i, nb);
                        int32_t sum = 0;
                        for (int k = 0; k < z; ++k) sum += s[nb[k]];
                        const double si = (double)s[i];
                        const double dE = 2.0 * si * (J * (double)sum + hh);
                        int acc = dE <= 0.0;
                        if (!acc) {
                            uint32_t w[4];
                            philox(seed, (uint32_t)i, t, inst >> 2, 0x80000u, w);
                            acc = (double)w[inst & 3u] * 0x1p-32 < exp(-(beta * dE));
                        }
                        if (acc) s[i] = (int8_t)(-s[i]);
                    }
                /* E and M after the MCS: bonds along +x, +y (, +z) from every site */
                int64_t bsum = 0, msum = 0;
                for (int32_t i = 0; i < n; ++i) {
                    int32_t nb[6];
                    ising_neighbours(dims, L, i, nb);
                    for (int d = 0; d < dims; ++d) bsum += (int64_t)s[i] * s[nb[2 * d + 1]];
                    msum += s[i];
                }
                double *hr = history + ((int64_t)r * n_steps * mcs + rec) * 2;
                hr[0] = -J * (double)bsum - hh * (double)msum;
                hr[1] = (double)msum;
                ++rec;
                ++t;
            }
        }
    }
    return 0;
}
