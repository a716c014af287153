/*
 * kmc_oracle.c -- plain, slow, obviously-correct CPU oracle of one timestep of
 * the test-particle kinetic Monte Carlo method of Sagert et al. (arXiv:1210.8084).
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check and the CPU-baseline leg of the
 * benchmark).  It shares no code, header or constant generator with the CUDA
 * library.  Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -shared -fPIC.
 *
 * Which passage each function follows:
 *   orc_philox4x32_10   Philox4x32-10 (Salmon et al., SC'11, Sect. 4.2 and Table 2)
 *   orc_contact_R2      Eq. 7 (lambda = 1/(sigma n)) and Eq. reff_lambda
 *   orc_adaptive_dt     Sect. "Simulation setup": dt(t) = dx / v_max(t)
 *   orc_cell_keys       Sect. "Simulation setup": spatial binning into c-bins
 *   orc_pair_test       Sect. "Point of Closest Approach Method", Eqs. 5-6
 *                       (crossing number chi), Eqs. collision_time/collision_time2
 *                       (real overlap times), scattering-detection criteria 1-2
 *   orc_best_partners   criterion 3 (closest candidate) over the 3^D neighbourhood
 *                       (8 neighbours in 2-D, 26 in 3-D)
 *   orc_mutual_pairs    "only unambiguously determined interaction partners"
 *   orc_collide_move    CM-frame scattering with random opposite directions,
 *                       t_poca (Eq. 12) and the split position update (Eqs. 13-14),
 *                       reflective walls (Sod test set-up), absorbing walls (Sedov test)
 *   orc_collide_move_ids  the same on a subset of a larger system (one domain and
 *                       its halo), the pair's random direction keyed by global ids
 *   orc_moments         n = N/V, bulk velocity (Eq. vel_b), stress tensor with
 *                       kinetic and collisional parts (Eq. stress), pressure
 *                       (Eq. 18), v_rms and T = m v_rms^2 / f (Eq. 19)
 * Readings of silent or garbled passages are listed in the design notes; the
 * ones that shape this file are restated at the point of use.
 */
#include "kmc_oracle.h"

#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ Philox */

/* Philox4x32 with 10 rounds.  Round: two 32x32->64 multiplies by the
 * published multipliers; the high halves are xor-ed with the other two counter
 * words and the round key, the low halves pass through; the words are
 * permuted.  The key is bumped by the Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform deviates in (0, 1) from Philox words.  binary32 path: 24-bit odd
 * mantissa, (2m+1) 2^-24.  binary64 path: 53-bit odd mantissa from two words. */
static double uniform32(uint32_t x) { return (double)((x >> 8) | 1u) * 0x1p-24; }
static double uniform64(uint32_t hi, uint32_t lo)
{
    uint64_t m = ((uint64_t)hi << 20) | (uint64_t)(lo >> 12); /* 52 bits */
    return (double)(2u * m + 1u) * 0x1p-53;
}

int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Absorbing walls (Sect. "Sedov test"): a particle that left the box through
 * one is no longer evolved; it is marked by a NaN position (and velocity). */
static int gone(const double* r) { return isnan(r[0]); }

/* ------------------------------------------------------------ parameters */

double orc_contact_R2(double lambda, double sigma, double nbar)
{
    /* Eq. 7: lambda = 1/(sigma n)  =>  sigma = 1/(lambda n).
     * Eq. reff_lambda: lambda = 1/(4 pi r_eff^2 n)  =>  4 pi r_eff^2 = sigma.
     * Contact distance r_eff,A + r_eff,B = 2 r_eff  =>  R^2 = 4 r_eff^2 = sigma/pi. */
    double s = sigma > 0.0 ? sigma : 1.0 / (lambda * nbar);
    return s / M_PI;
}

/* Sect. "Simulation setup": the timestep follows the fastest particle,
 * dt(t) = dx / v_max(t), so that no particle leaves its scattering
 * neighbourhood within a step.  dx: the smallest c-bin width. */
double orc_adaptive_dt(const orc_params* P, int64_t n, const double* vel, double dt_rest)
{
    double v2max = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double* v = vel + 3 * i;
        double v2;
        if (P->decide32) {
            float x = (float)v[0], y = (float)v[1], z = (float)v[2];
            float xx = x * x;
            v2 = (double)fmaf(z, z, fmaf(y, y, xx));
        } else {
            v2 = fma(v[2], v[2], fma(v[1], v[1], v[0] * v[0]));
        }
        if (v2 > v2max) v2max = v2;
    }
    if (!(v2max > 0.0)) return dt_rest;
    double dx = INFINITY;
    for (int d = 0; d < P->dim; ++d) {
        double w = (P->hi[d] - P->lo[d]) / P->n_cells[d];
        if (w < dx) dx = w;
    }
    return dx / sqrt(v2max);
}

/* ------------------------------------------------------------------- keys */

/* c_d = floor((x_d - lo_d) * (n_d / (hi_d - lo_d))), clamped to [0, n_d - 1];
 * evaluated in the decision precision. */
static int cell_1d(const orc_params* P, int d, double x)
{
    int n = P->n_cells[d];
    double inv = (double)n / (P->hi[d] - P->lo[d]);
    if (P->decide32) {
        float t = ((float)x - (float)P->lo[d]) * (float)inv;
        if (t < 0.0f) return 0;
        if (t >= (float)n) return n - 1;
        return (int)t;
    } else {
        double t = (x - P->lo[d]) * inv;
        if (t < 0.0) return 0;
        if (t >= (double)n) return n - 1;
        return (int)t;
    }
}

static int32_t linear_key(const orc_params* P, const int c[3])
{
    if (P->dim == 2) return c[0] + P->n_cells[0] * c[1];
    return c[0] + P->n_cells[0] * (c[1] + P->n_cells[1] * c[2]);
}

static int n_bins(const orc_params* P)
{
    int C = P->n_cells[0] * P->n_cells[1];
    if (P->dim == 3) C *= P->n_cells[2];
    return C;
}

void orc_cell_keys(const orc_params* P, int64_t n, const double* pos,
                   int32_t* key_out, int32_t* cidx_out)
{
    for (int64_t i = 0; i < n; ++i) {
        int c[3] = {0, 0, 0};
        if (gone(pos + 3 * i)) {   /* absorbed: in no c-bin */
            if (key_out) key_out[i] = -1;
            if (cidx_out) for (int d = 0; d < 3; ++d) cidx_out[3 * i + d] = 0;
            continue;
        }
        for (int d = 0; d < P->dim; ++d) c[d] = cell_1d(P, d, pos[3 * i + d]);
        if (key_out) key_out[i] = linear_key(P, c);
        if (cidx_out) for (int d = 0; d < 3; ++d) cidx_out[3 * i + d] = c[d];
    }
}

/* --------------------------------------------------------- PoCA pair test */

/* Relative coordinates of the pair, minimum image in periodic dimensions:
 * shift by one box length when the separation exceeds half of it. */
static float min_image_f(const orc_params* P, int d, float x)
{
    if (P->bc[d] != 0) return x;
    float L = (float)(P->hi[d] - P->lo[d]);
    float h = 0.5f * L;
    if (x > h) return x - L;
    if (x < -h) return x + L;
    return x;
}

static double min_image_d(const orc_params* P, int d, double x)
{
    if (P->bc[d] != 0) return x;
    double L = P->hi[d] - P->lo[d];
    double h = 0.5 * L;
    if (x > h) return x - L;
    if (x < -h) return x + L;
    return x;
}

/* The acceptance test, written once per precision with the same operation
 * order and the same fused multiply-adds:
 *   r_rel = r_i - r_j,  v_rel = v_i - v_j                      (Eq. 5)
 *   a = r_rel . v_rel,  b = |v_rel|^2,  r2 = |r_rel|^2
 *   chi = (r_rel(t).v_rel)(r_rel(t+dt).v_rel) = a (a + b dt)   (Eq. c_value)
 *     -> chi < 0 is evaluated by the signs of its two factors: a < 0 and
 *        a + b dt > 0 (b >= 0, so a > 0 forces a + b dt > 0).
 *   overlap times real  <=>  discriminant of Eq. collision_time
 *     disc = a^2 - b (r2 - R^2) >= 0                           (Eq. collision_time2,
 *     whose printed numerator "-(v.r)^2" is read as -(v.r); only the reality
 *     of the roots is used, tangency counts as real)
 *   distance of closest approach d^2 = r2 - a^2 / b            (criterion 3)  */
static int pair_test_f(const orc_params* P, const double* ri, const double* vi,
                       const double* rj, const double* vj, float q[5])
{
    float dr[3] = {0, 0, 0}, dv[3] = {0, 0, 0};
    for (int d = 0; d < P->dim; ++d) {
        dr[d] = min_image_f(P, d, (float)ri[d] - (float)rj[d]);
        dv[d] = (float)vi[d] - (float)vj[d];
    }
    float a = dr[0] * dv[0];
    a = fmaf(dr[1], dv[1], a);
    float b = dv[0] * dv[0];
    b = fmaf(dv[1], dv[1], b);
    float r2 = dr[0] * dr[0];
    r2 = fmaf(dr[1], dr[1], r2);
    if (P->dim == 3) {
        a = fmaf(dr[2], dv[2], a);
        b = fmaf(dv[2], dv[2], b);
        r2 = fmaf(dr[2], dr[2], r2);
    }
    float dt = (float)P->dt, R2 = (float)P->R2;
    float disc = fmaf(a, a, -(b * (r2 - R2)));
    float d2 = (b > 0.0f) ? r2 - (a * a) / b : INFINITY;
    if (q) { q[0] = a; q[1] = b; q[2] = r2; q[3] = disc; q[4] = d2; }
    if (!(b > 0.0f)) return 0;
    if (!(a < 0.0f && fmaf(b, dt, a) > 0.0f)) return 0;   /* criterion 1 */
    return disc >= 0.0f;                                     /* criterion 2 */
}

static int pair_test_d(const orc_params* P, const double* ri, const double* vi,
                       const double* rj, const double* vj, double q[5])
{
    double dr[3] = {0, 0, 0}, dv[3] = {0, 0, 0};
    for (int d = 0; d < P->dim; ++d) {
        dr[d] = min_image_d(P, d, ri[d] - rj[d]);
        dv[d] = vi[d] - vj[d];
    }
    double a = dr[0] * dv[0];
    a = fma(dr[1], dv[1], a);
    double b = dv[0] * dv[0];
    b = fma(dv[1], dv[1], b);
    double r2 = dr[0] * dr[0];
    r2 = fma(dr[1], dr[1], r2);
    if (P->dim == 3) {
        a = fma(dr[2], dv[2], a);
        b = fma(dv[2], dv[2], b);
        r2 = fma(dr[2], dr[2], r2);
    }
    double disc = fma(a, a, -(b * (r2 - P->R2)));
    double d2 = (b > 0.0) ? r2 - (a * a) / b : INFINITY;
    if (q) { q[0] = a; q[1] = b; q[2] = r2; q[3] = disc; q[4] = d2; }
    if (!(b > 0.0)) return 0;
    if (!(a < 0.0 && fma(b, P->dt, a) > 0.0)) return 0;   /* criterion 1 */
    return disc >= 0.0;                                      /* criterion 2 */
}

int orc_pair_test(const orc_params* P, const double* ri, const double* vi,
                  const double* rj, const double* vj, double* quant5)
{
    if (P->decide32) {
        float q[5];
        int ok = pair_test_f(P, ri, vi, rj, vj, q);
        if (quant5) for (int k = 0; k < 5; ++k) quant5[k] = (double)q[k];
        return ok;
    }
    return pair_test_d(P, ri, vi, rj, vj, quant5);
}

/* ------------------------------------------------------ neighbourhood */

/* Distinct neighbour indices c-1, c, c+1 along one dimension: wrapped when
 * periodic (duplicates dropped when n <= 2), cut at the box when walled. */
static int neighbours_1d(const orc_params* P, int d, int c, int out[3])
{
    int n = P->n_cells[d], m = 0;
    for (int o = -1; o <= 1; ++o) {
        int cc = c + o;
        if (P->bc[d] == 0) cc = ((cc % n) + n) % n;
        else if (cc < 0 || cc >= n) continue;
        int dup = 0;
        for (int k = 0; k < m; ++k) if (out[k] == cc) dup = 1;
        if (!dup) out[m++] = cc;
    }
    return m;
}

/* Is c-bin cj in the neighbourhood of ci?  (|dc| <= 1 per dimension, cyclic
 * in periodic dimensions.) */
static int in_neighbourhood(const orc_params* P, const int ci[3], const int cj[3])
{
    for (int d = 0; d < P->dim; ++d) {
        int dc = abs(ci[d] - cj[d]);
        if (P->bc[d] == 0 && P->n_cells[d] - dc < dc) dc = P->n_cells[d] - dc;
        if (dc > 1) return 0;
    }
    return 1;
}

/* Keep the better of two candidates: smaller d^2, ties to the lower id. */
static int better_f(float d2, int32_t j, float bd, int32_t bj)
{
    return d2 < bd || (d2 == bd && j < bj);
}
static int better_d(double d2, int32_t j, double bd, int32_t bj)
{
    return d2 < bd || (d2 == bd && j < bj);
}

/* c-bin lists in (key, id) order: counting sort by key, ids ascending. */
typedef struct { int32_t* key; int32_t* cidx; int64_t* start; int32_t* list; } bins_t;

static void bins_build(const orc_params* P, int64_t n, const double* pos, bins_t* B)
{
    int C = n_bins(P);
    B->key = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    B->cidx = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(n > 0 ? n : 1));
    B->start = (int64_t*)calloc((size_t)C + 1, sizeof(int64_t));
    B->list = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    orc_cell_keys(P, n, pos, B->key, B->cidx);
    for (int64_t i = 0; i < n; ++i)
        if (B->key[i] >= 0) B->start[B->key[i] + 1]++;
    for (int c = 0; c < C; ++c) B->start[c + 1] += B->start[c];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)C);
    for (int c = 0; c < C; ++c) fill[c] = B->start[c];
    for (int64_t i = 0; i < n; ++i)
        if (B->key[i] >= 0) B->list[fill[B->key[i]]++] = (int32_t)i;
    free(fill);
}

static void bins_free(bins_t* B)
{
    free(B->key); free(B->cidx); free(B->start); free(B->list);
}

/* Visit every particle j != i in the neighbourhood of i's c-bin. */
#define FOR_NEIGHBOURHOOD(P, B, i, j, BODY)                                        \
    do {                                                                           \
        int nx_[3], ny_[3], nz_[3] = {0, 0, 0};                                    \
        int mx_ = neighbours_1d(P, 0, (B)->cidx[3 * (i) + 0], nx_);                \
        int my_ = neighbours_1d(P, 1, (B)->cidx[3 * (i) + 1], ny_);                \
        int mz_ = (P)->dim == 3 ? neighbours_1d(P, 2, (B)->cidx[3 * (i) + 2], nz_) \
                                : 1;                                               \
        for (int a_ = 0; a_ < mx_; ++a_)                                           \
            for (int b_ = 0; b_ < my_; ++b_)                                       \
                for (int c_ = 0; c_ < mz_; ++c_) {                                 \
                    int cc_[3] = {nx_[a_], ny_[b_], nz_[c_]};                      \
                    int32_t k_ = linear_key(P, cc_);                               \
                    for (int64_t s_ = (B)->start[k_]; s_ < (B)->start[k_ + 1];     \
                         ++s_) {                                                   \
                        int32_t j = (B)->list[s_];                                 \
                        if (j == (i)) continue;                                    \
                        BODY                                                       \
                    }                                                              \
                }                                                                  \
    } while (0)

int64_t orc_best_partners(const orc_params* P, int64_t n, const double* pos,
                          const double* vel, int32_t* best)
{
    bins_t B;
    bins_build(P, n, pos, &B);
    int64_t found = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : found)
    for (int64_t i = 0; i < n; ++i) {
        int32_t bj = -1;
        if (B.key[i] < 0) {   /* absorbed */
            best[i] = -1;
            continue;
        }
        if (P->decide32) {
            float bd = INFINITY, q[5];
            FOR_NEIGHBOURHOOD(P, &B, i, j, {
                if (pair_test_f(P, pos + 3 * i, vel + 3 * i, pos + 3 * j, vel + 3 * j, q)
                    && better_f(q[4], j, bd, bj)) { bd = q[4]; bj = j; }
            });
        } else {
            double bd = INFINITY, q[5];
            FOR_NEIGHBOURHOOD(P, &B, i, j, {
                if (pair_test_d(P, pos + 3 * i, vel + 3 * i, pos + 3 * j, vel + 3 * j, q)
                    && better_d(q[4], j, bd, bj)) { bd = q[4]; bj = j; }
            });
        }
        best[i] = bj;
        found += (bj >= 0);
    }
    bins_free(&B);
    return found;
}

int64_t orc_candidate_count(const orc_params* P, int64_t n, const double* pos)
{
    bins_t B;
    bins_build(P, n, pos, &B);
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (B.key[i] < 0) continue;
        FOR_NEIGHBOURHOOD(P, &B, i, j, { total += 1; (void)j; });
    }
    bins_free(&B);
    return total;
}

int64_t orc_best_partners_brute(const orc_params* P, int64_t n, const double* pos,
                                const double* vel, int32_t* best)
{
    int32_t* cidx = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(n > 0 ? n : 1));
    orc_cell_keys(P, n, pos, NULL, cidx);
    int64_t found = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t bj = -1;
        double bd = INFINITY;
        float bdf = INFINITY;
        for (int64_t j = 0; j < n && !gone(pos + 3 * i); ++j) {
            if (j == i || gone(pos + 3 * j) || !in_neighbourhood(P, cidx + 3 * i, cidx + 3 * j)) continue;
            double q[5];
            if (!orc_pair_test(P, pos + 3 * i, vel + 3 * i, pos + 3 * j, vel + 3 * j, q))
                continue;
            if (P->decide32) {
                if (better_f((float)q[4], (int32_t)j, bdf, bj)) { bdf = (float)q[4]; bj = (int32_t)j; }
            } else {
                if (better_d(q[4], (int32_t)j, bd, bj)) { bd = q[4]; bj = (int32_t)j; }
            }
        }
        best[i] = bj;
        found += (bj >= 0);
    }
    free(cidx);
    return found;
}

int64_t orc_mutual_pairs(int64_t n, const int32_t* best, int32_t* pairs_out)
{
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t j = best[i];
        if (j > i && best[j] == (int32_t)i) {
            if (pairs_out) { pairs_out[2 * m] = (int32_t)i; pairs_out[2 * m + 1] = j; }
            ++m;
        }
    }
    return m;
}

/* ------------------------------------------------- scatter, move, walls */

/* Specular reflection: fold the end-of-step coordinate back into [lo, hi]
 * and flip the velocity component once per fold.  Periodic: shift into
 * [lo, hi).  Absorbing: the coordinate is left as it is (the caller removes a
 * particle that ends outside). */
static void boundary_1d(const orc_params* P, int d, double* x, double* v)
{
    double lo = P->lo[d], hi = P->hi[d];
    if (P->bc[d] == 2) return;
    if (P->bc[d] == 1) {
        for (int it = 0; it < 64 && (*x < lo || *x > hi); ++it) {
            if (*x < lo) *x = 2.0 * lo - *x;
            else *x = 2.0 * hi - *x;
            *v = -*v;
        }
        if (*x < lo) *x = lo;
        if (*x > hi) *x = hi;
    } else {
        double L = hi - lo;
        if (*x >= hi) *x -= L;
        else if (*x < lo) *x += L;
        if (*x < lo || *x >= hi) *x = lo + (*x - lo) - L * floor((*x - lo) / L);
        if (*x >= hi) *x = lo;
    }
}

void orc_collide_move(const orc_params* P, int64_t n, const double* pos,
                      const double* vel, const int32_t* best, double* pos_out,
                      double* vel_out, double* virial_out, int32_t* paired_out)
{
    orc_collide_move_ids(P, n, pos, vel, best, NULL, pos_out, vel_out, virial_out, paired_out);
}

void orc_collide_move_ids(const orc_params* P, int64_t n, const double* pos,
                          const double* vel, const int32_t* best, const int64_t* ids,
                          double* pos_out, double* vel_out, double* virial_out,
                          int32_t* paired_out)
{
    const uint32_t key[2] = {(uint32_t)(P->seed & 0xffffffffu), (uint32_t)(P->seed >> 32)};
    for (int64_t i = 0; i < n; ++i) {
        const double* r = pos + 3 * i;
        const double* v = vel + 3 * i;
        double* ro = pos_out + 3 * i;
        double* vo = vel_out + 3 * i;
        int32_t j = best ? best[i] : -1;
        int paired = (j >= 0 && best[j] == (int32_t)i);
        double W = 0.0;
        for (int d = 0; d < 3; ++d) { ro[d] = r[d]; vo[d] = v[d]; }
        if (paired) {
            const double* rj = pos + 3 * j;
            const double* vj = vel + 3 * j;
            int64_t lo = i < j ? i : j;
            double sgn = (i == lo) ? 1.0 : -1.0;
            /* relative coordinates oriented (self - partner) */
            double dr[3] = {0, 0, 0}, dv[3];
            for (int d = 0; d < P->dim; ++d) dr[d] = min_image_d(P, d, r[d] - rj[d]);
            for (int d = 0; d < 3; ++d) dv[d] = v[d] - vj[d];
            double a = 0.0, b = 0.0;
            for (int d = 0; d < P->dim; ++d) { a += dr[d] * dv[d]; b += dv[d] * dv[d]; }
            double tp = -a / b;                                        /* Eq. 12 */
            double g = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
            /* random isotropic direction for the pair, drawn once per pair from
             * Philox keyed by (lower id, step) */
            uint32_t id_lo = ids ? (uint32_t)ids[lo] : (uint32_t)lo;
            uint32_t ctr[4] = {id_lo, P->step, 0u, 0u}, x[4];
            orc_philox4x32_10(ctr, key, x);
            double u1 = P->decide32 ? uniform32(x[0]) : uniform64(x[0], x[1]);
            double u2 = P->decide32 ? uniform32(x[2]) : uniform64(x[2], x[3]);
            double cth = 1.0 - 2.0 * u1;
            double sth = 2.0 * sqrt(u1 * (1.0 - u1));
            double phi = 2.0 * M_PI * u2;
            double nhat[3] = {sth * cos(phi), sth * sin(phi), cth};
            if (P->vel_dim == 2) {   /* isotropic in the plane: azimuth only */
                nhat[0] = cos(phi);
                nhat[1] = sin(phi);
                nhat[2] = 0.0;
            }
            /* CM frame: outgoing velocities opposite, |v_rel| preserved */
            for (int d = 0; d < 3; ++d) {
                double vcm = 0.5 * (v[d] + vj[d]);
                vo[d] = vcm + sgn * 0.5 * g * nhat[d];
            }
            /* Eq. 13: r + v_old t_poca + v_new (dt - t_poca) */
            for (int d = 0; d < P->dim; ++d)
                ro[d] = r[d] + v[d] * tp + vo[d] * (P->dt - tp);
            /* collisional virial: r_ij at closest approach dotted with dp_i */
            for (int d = 0; d < P->dim; ++d) W += (dr[d] + dv[d] * tp) * (vo[d] - v[d]);
        } else {
            for (int d = 0; d < P->dim; ++d) ro[d] = r[d] + v[d] * P->dt;  /* Eq. 14 */
        }
        int out = gone(r);
        for (int d = 0; d < P->dim; ++d) {
            boundary_1d(P, d, &ro[d], &vo[d]);
            if (P->bc[d] == 2 && (ro[d] < P->lo[d] || ro[d] > P->hi[d])) out = 1;
        }
        if (out) {   /* absorbed (now or earlier): NaN state */
            for (int d = 0; d < 3; ++d) ro[d] = vo[d] = NAN;
            W = 0.0;
        }
        if (virial_out) virial_out[i] = W;
        if (paired_out) paired_out[i] = paired ? j : -1;
    }
}

/* ------------------------------------------------------------ DSMC variant */

/* The classic DSMC collision step the paper contrasts with its method (Sect.
 * "Direct Simulation Monte Carlo Technique": collisions only between particles
 * of the same scattering cell, partners picked at random), in Bird's
 * no-time-counter form with the cross-section of Eq. 7.  Cells are the
 * c-bins; a cell's particles are taken in increasing id.  Per cell with N >= 2
 * particles and volume V_c:
 *   M = floor(1/2 N (N - 1) sigma g_max dt / V_c + u_0) candidate pairs, with
 *       sigma = pi R^2 and g_max = 2 v_max (v_max the largest speed of the
 *       state, so g_max bounds every relative speed);
 *   candidate k: i, j distinct positions in the cell drawn uniformly, accepted
 *       with probability g / g_max (g = |v_i - v_j|; sigma is the same for all
 *       pairs), then scattered as the PoCA pairs are: isotropic in the CM
 *       frame, v' = v_cm +- g/2 n.
 * Collisions are applied in candidate order, each to the current velocities.
 * Random numbers: Philox4x32-10 with key = seed and counter (cell, step, k,
 * 0x44534D43) for the pair and the acceptance, (cell, step, k, 0x44534D44) for
 * the direction, (cell, step, 0xFFFFFFFF, 0x44534D43) for u_0; cell = the
 * c-bin's index with x slowest, (c_x n_y + c_y) n_z + c_z.  Position indices:
 * i = floor(w0 N / 2^32), j = floor(w1 (N - 1) / 2^32), j += 1 when j >= i.
 * All of it in binary64; with decide32 the new velocities are rounded to
 * binary32 after every collision (the state precision).  Velocities are
 * updated in place; collided[i] = 1 for a particle in at least one accepted
 * pair.  Returns the number of accepted collisions. */
int64_t orc_dsmc_collide(const orc_params* P, int64_t n, const double* pos, double* vel, int32_t* collided)
{
    const uint32_t key[2] = {(uint32_t)(P->seed & 0xffffffffu), (uint32_t)(P->seed >> 32)};
    const uint32_t TAG_PAIR = 0x44534D43u, TAG_DIR = 0x44534D44u;
    int C = n_bins(P);
    int32_t* cidx = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(n > 0 ? n : 1));
    int32_t* kk = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    orc_cell_keys(P, n, pos, kk, cidx);
    /* cell of every particle in the search order (x slowest); -1 when absorbed */
    int64_t* cnt = (int64_t*)calloc((size_t)C + 1, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        if (kk[i] < 0) continue;
        const int32_t* c = cidx + 3 * i;
        int32_t s = P->dim == 3 ? (c[0] * P->n_cells[1] + c[1]) * P->n_cells[2] + c[2] : c[0] * P->n_cells[1] + c[1];
        kk[i] = s;
        cnt[s + 1] += 1;
    }
    for (int c = 0; c < C; ++c) cnt[c + 1] += cnt[c];
    /* ids of every cell in increasing order (a stable counting sort over ids) */
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(C > 0 ? C : 1));
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int c = 0; c < C; ++c) fill[c] = cnt[c];
    for (int64_t i = 0; i < n; ++i)
        if (kk[i] >= 0) order[fill[kk[i]]++] = i;
    /* largest speed, |v|^2 as the adaptive timestep takes it */
    double v2max = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (kk[i] < 0) continue;
        const double* v = vel + 3 * i;
        double v2;
        if (P->decide32) {
            float x = (float)v[0], y = (float)v[1], z = (float)v[2];
            float xx = x * x;
            v2 = (double)fmaf(z, z, fmaf(y, y, xx));
        } else {
            v2 = fma(v[2], v[2], fma(v[1], v[1], v[0] * v[0]));
        }
        if (v2 > v2max) v2max = v2;
    }
    const double gmax = 2.0 * sqrt(v2max);
    const double sigma = M_PI * P->R2;
    double Vc = 1.0;
    for (int d = 0; d < P->dim; ++d) Vc *= (P->hi[d] - P->lo[d]) / P->n_cells[d];
    for (int64_t i = 0; i < n; ++i) collided[i] = 0;
    int64_t accepted = 0;
    for (int c = 0; c < C; ++c) {
        const int64_t N = cnt[c + 1] - cnt[c];
        if (N < 2) continue;
        const int64_t* ids = order + cnt[c];
        uint32_t w[4];
        uint32_t ctr0[4] = {(uint32_t)c, P->step, 0xFFFFFFFFu, TAG_PAIR};
        orc_philox4x32_10(ctr0, key, w);
        const double Nd = (double)N;
        const double m_real = 0.5 * Nd * (Nd - 1.0) * sigma * gmax * P->dt / Vc;
        const double m = floor(m_real + uniform64(w[0], w[1]));
        const uint32_t M = m > 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)m;
        for (uint32_t k = 0; k < M; ++k) {
            uint32_t ctr[4] = {(uint32_t)c, P->step, k, TAG_PAIR};
            orc_philox4x32_10(ctr, key, w);
            uint32_t pi = (uint32_t)(((uint64_t)w[0] * (uint64_t)N) >> 32);
            uint32_t pj = (uint32_t)(((uint64_t)w[1] * (uint64_t)(N - 1)) >> 32);
            if (pj >= pi) pj += 1u;
            double* va = vel + 3 * ids[pi];
            double* vb = vel + 3 * ids[pj];
            double dv0 = va[0] - vb[0], dv1 = va[1] - vb[1], dv2 = va[2] - vb[2];
            double g = sqrt(dv0 * dv0 + dv1 * dv1 + dv2 * dv2);
            if (!(uniform64(w[2], w[3]) * gmax < g)) continue;
            uint32_t ctr2[4] = {(uint32_t)c, P->step, k, TAG_DIR};
            orc_philox4x32_10(ctr2, key, w);
            double u1 = uniform64(w[0], w[1]), u2 = uniform64(w[2], w[3]);
            double cth = 1.0 - 2.0 * u1;
            double sth = 2.0 * sqrt(u1 * (1.0 - u1));
            double phi = 2.0 * M_PI * u2;
            double nhat[3] = {sth * cos(phi), sth * sin(phi), cth};
            if (P->vel_dim == 2) {
                nhat[0] = cos(phi);
                nhat[1] = sin(phi);
                nhat[2] = 0.0;
            }
            double h = 0.5 * g;
            for (int d = 0; d < 3; ++d) {
                double vcm = 0.5 * (va[d] + vb[d]);
                double a = vcm + h * nhat[d], b = vcm - h * nhat[d];
                va[d] = P->decide32 ? (double)(float)a : a;
                vb[d] = P->decide32 ? (double)(float)b : b;
            }
            collided[ids[pi]] = 1;
            collided[ids[pj]] = 1;
            ++accepted;
        }
    }
    free(cidx); free(kk); free(cnt); free(fill); free(order);
    return accepted;
}

/* ---------------------------------------------------------------- moments */

void orc_moments(const orc_params* P, int64_t n, const double* pos, const double* vel,
                 const double* virial, double* raw, double* derived, double* glob)
{
    int C = n_bins(P);
    double* acc = (double*)calloc((size_t)C * 8, sizeof(double));
    double G[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int32_t* key = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    orc_cell_keys(P, n, pos, key, NULL);
    for (int64_t i = 0; i < n; ++i) {
        if (key[i] < 0) continue;   /* absorbed */
        const double* v = vel + 3 * i;
        double W = virial ? virial[i] : 0.0;
        double* m = acc + 8 * (size_t)key[i];
        m[0] += 1.0;
        for (int d = 0; d < 3; ++d) { m[1 + d] += v[d]; m[4 + d] += v[d] * v[d]; }
        m[7] += W;
        G[0] += 1.0;
        G[1] += 0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        for (int d = 0; d < 3; ++d) G[2 + d] += v[d];
        G[5] += W;
    }
    free(key);
    double Vc = 1.0;
    for (int d = 0; d < P->dim; ++d) Vc *= (P->hi[d] - P->lo[d]) / P->n_cells[d];
    for (int c = 0; c < C; ++c) {
        const double* m = acc + 8 * (size_t)c;
        if (raw) for (int k = 0; k < 8; ++k) raw[8 * (size_t)c + k] = m[k];
        if (!derived) continue;
        double* o = derived + 8 * (size_t)c;
        for (int k = 0; k < 8; ++k) o[k] = 0.0;
        if (m[0] <= 0.0) continue;
        double N = m[0];
        double u[3] = {m[1] / N, m[2] / N, m[3] / N};
        /* mean square peculiar speed: <|v|^2> - |u|^2, i.e. v_rms^2 of Eq. 19
         * read as (1/N) Sum |v_i - v_b|^2 */
        double c2 = (m[4] + m[5] + m[6]) / N - (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        double T = c2 / (P->vel_dim == 2 ? 2.0 : 3.0);   /* f velocity degrees of freedom, m = 1 */
        double nd = N / Vc;
        double pkin = nd * T;           /* kinetic part of Eq. stress: -trace/3V */
        /* collisional part: (1/2)(1/dt) Sum_i Sum_j r_ij . dp_i, trace over the
         * position dimensions, divided by dim V */
        double pvir = m[7] / (2.0 * P->dim * Vc * P->dt);
        o[0] = nd; o[1] = u[0]; o[2] = u[1]; o[3] = u[2];
        o[4] = T; o[5] = pkin; o[6] = pvir; o[7] = pkin + pvir;
    }
    if (glob) for (int k = 0; k < 8; ++k) glob[k] = G[k];
    free(acc);
}

void orc_radial(const orc_params* P, int64_t n, const double* pos, const double* vel,
                const double* center, double* out)
{
    int C = n_bins(P);
    for (int c = 0; c < 2 * C; ++c) out[c] = 0.0;
    double* cnt = (double*)calloc((size_t)C, sizeof(double));
    int32_t* key = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    orc_cell_keys(P, n, pos, key, NULL);
    for (int64_t i = 0; i < n; ++i) {
        if (key[i] < 0) continue;   /* absorbed */
        double r[3] = {0.0, 0.0, 0.0};
        double r2 = 0.0;
        for (int d = 0; d < P->dim; ++d) {
            r[d] = pos[3 * i + d] - center[d];
            r2 += r[d] * r[d];
        }
        cnt[key[i]] += 1.0;
        if (r2 <= 0.0) continue;
        double len = sqrt(r2), vr = 0.0;
        for (int d = 0; d < P->dim; ++d) vr += vel[3 * i + d] * (r[d] / len);
        out[2 * (size_t)key[i]] += vr;
    }
    for (int c = 0; c < C; ++c)
        if (cnt[c] > 0.0) out[2 * (size_t)c + 1] = out[2 * (size_t)c] / cnt[c];
    free(cnt);
    free(key);
}

/* ------------------------------------------------------------------- step */

int64_t orc_step(const orc_params* P, int64_t n, double* pos, double* vel,
                 int32_t* best_out, int32_t* paired_out, double* raw,
                 double* derived, double* glob)
{
    size_t nn = (size_t)(n > 0 ? n : 1);
    int32_t* best = (int32_t*)malloc(sizeof(int32_t) * nn);
    int32_t* paired = (int32_t*)malloc(sizeof(int32_t) * nn);
    double* p2 = (double*)malloc(sizeof(double) * 3 * nn);
    double* v2 = (double*)malloc(sizeof(double) * 3 * nn);
    double* W = (double*)malloc(sizeof(double) * nn);
    orc_best_partners(P, n, pos, vel, best);                          /* search */
    orc_collide_move(P, n, pos, vel, best, p2, v2, W, paired);        /* scatter + move */
    int64_t npairs = 0;
    for (int64_t i = 0; i < n; ++i) npairs += (paired[i] > (int32_t)i);
    memcpy(pos, p2, sizeof(double) * 3 * (size_t)n);
    memcpy(vel, v2, sizeof(double) * 3 * (size_t)n);
    if (raw || derived || glob) orc_moments(P, n, pos, vel, W, raw, derived, glob);
    if (best_out) memcpy(best_out, best, sizeof(int32_t) * (size_t)n);
    if (paired_out) memcpy(paired_out, paired, sizeof(int32_t) * (size_t)n);
    free(best); free(paired); free(p2); free(v2); free(W);
    return npairs;
}
