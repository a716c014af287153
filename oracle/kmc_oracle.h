/*
 * kmc_oracle.h -- plain CPU oracle for the test-particle kinetic Monte Carlo step
 * of Sagert et al., "Hydrodynamic Shock Wave Studies within a Kinetic Monte Carlo
 * Approach" (arXiv:1210.8084).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this code: only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no source with the CUDA library.
 *
 * Everything is FP64 except the optional binary32 "decision" mode: when
 * decide32 != 0 the quantities that decide an integer result (cell index, the
 * crossing-number sign, the real-root test, the argmin distance) are evaluated in
 * IEEE binary32 so that an FP32 device path can be compared bit-for-bit on those
 * integers.  Both modes use the same operation order and the same fused
 * multiply-adds (fma/fmaf), compiled with -ffp-contract=off.
 *
 * Particle identity is the array index (0..n-1).  Positions and velocities are
 * n x 3 row-major doubles; in 2-D position mode (dim == 2) the z position is
 * carried but ignored, while velocities stay 3-D.
 */
#ifndef KMC_ORACLE_H
#define KMC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int dim;            /* position dimensions used for binning and PoCA: 2 or 3 */
    int n_cells[3];     /* c-bins per dimension (n_cells[2] ignored when dim == 2) */
    double lo[3], hi[3];/* box */
    int bc[3];          /* 0 = periodic, 1 = specular (reflective) wall */
    double R2;          /* (r_eff,A + r_eff,B)^2, Eq. (reff_lambda) */
    double dt;          /* timestep */
    uint64_t seed;      /* Philox key: (low 32 bits, high 32 bits) */
    uint32_t step;      /* Philox counter word 1 */
    int decide32;       /* 1: decisions in binary32; 0: binary64 */
    int vel_dim;        /* velocity components: 3, or 2 (x, y; the paper's 2-D runs, f = 2) */
} orc_params;

/* Threads of the OpenMP loops (closest-candidate search); <= 0 keeps the default.
 * Returns the number in use. */
int orc_set_threads(int n);

/* Philox4x32-10 block function (Salmon, Moraes, Dror, Shaw, SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* sigma from lambda = (sigma n)^-1 (Eq. 7) unless sigma > 0 is given, then the
 * squared contact distance R2 = (2 r_eff)^2 with lambda = (4 pi r_eff^2 n)^-1
 * (Eq. reff_lambda), i.e. R2 = sigma / pi.  nbar = N / V. */
double orc_contact_R2(double lambda, double sigma, double nbar);

/* Adaptive timestep (Sect. "Simulation setup"): dt = dx / v_max with dx the
 * smallest c-bin width over the position dimensions and v_max the largest
 * speed of the state.  |v|^2 = fma(vz, vz, fma(vy, vy, vx * vx)) in the
 * decision precision, the root and the quotient in binary64.  Returns dt_rest
 * when every particle is at rest. */
double orc_adaptive_dt(const orc_params* P, int64_t n, const double* vel, double dt_rest);

/* Cell index (per dim, clamped) and linear c-bin key c_x + n_x (c_y + n_y c_z). */
void orc_cell_keys(const orc_params* P, int64_t n, const double* pos,
                   int32_t* key_out, int32_t* cidx_out /* n x 3, may be NULL */);

/* The PoCA acceptance test for the ordered pair (i, j) (Eqs. 5-6, 8-9,
 * criteria 1-2 of the scattering detection).  Returns 1 if j is a collision
 * candidate for i; writes a, b, r2, disc, d2 (as doubles) when non-NULL. */
int orc_pair_test(const orc_params* P, const double* ri, const double* vi,
                  const double* rj, const double* vj, double* quant5);

/* Criterion 3: for every particle the closest candidate (smallest d_min^2,
 * ties to the lower id) among particles in its 3^D neighbourhood of c-bins.
 * best[i] = id or -1.  Returns the number of particles with a candidate. */
int64_t orc_best_partners(const orc_params* P, int64_t n, const double* pos,
                          const double* vel, int32_t* best);

/* Same result by brute force over all pairs filtered by the neighbourhood
 * predicate (tiny n only). */
int64_t orc_best_partners_brute(const orc_params* P, int64_t n, const double* pos,
                                const double* vel, int32_t* best);

/* Number of candidates examined (neighbourhood size sum) for the cost model. */
int64_t orc_candidate_count(const orc_params* P, int64_t n, const double* pos);

/* Unambiguous pairs: i <-> j iff best[i] == j and best[j] == i.
 * pairs_out gets (lo, hi) id pairs sorted by lo; returns the pair count. */
int64_t orc_mutual_pairs(int64_t n, const int32_t* best, int32_t* pairs_out);

/* Scatter in the CM frame, split move, walls.  Reads start-of-step state,
 * writes end-of-step state; virial_out[i] = r_ij(t_poca) . dp_i for paired
 * particles (0 otherwise); paired_out[i] = partner id or -1. */
void orc_collide_move(const orc_params* P, int64_t n, const double* pos,
                      const double* vel, const int32_t* best, double* pos_out,
                      double* vel_out, double* virial_out, int32_t* paired_out);

/* The same for a subset of a larger system (one domain plus its halo): ids[i]
 * is the global identity of entry i, which keys the pair's random direction.
 * The entries must be in increasing id order, so that "lower index" and "lower
 * id" agree.  ids == NULL means ids[i] = i. */
void orc_collide_move_ids(const orc_params* P, int64_t n, const double* pos,
                          const double* vel, const int32_t* best, const int64_t* ids,
                          double* pos_out, double* vel_out, double* virial_out,
                          int32_t* paired_out);

/* The DSMC comparison variant's collisions (random partners inside a c-bin,
 * Bird's no-time-counter scheme with sigma of Eq. 7): velocities updated in
 * place, collided[i] = 1 for particles in an accepted pair; returns the number
 * of accepted collisions.  The definition is restated in kmc_oracle.c.  The
 * move that follows is orc_collide_move with no pairs (free flight, walls). */
int64_t orc_dsmc_collide(const orc_params* P, int64_t n, const double* pos, double* vel, int32_t* collided);

/* Per-c-bin moments of the given state.  raw: C x 8 =
 * [N, Sum vx, Sum vy, Sum vz, Sum vx^2, Sum vy^2, Sum vz^2, Sum W];
 * derived: C x 8 = [n, ux, uy, uz, T, p_kin, p_vir, p];
 * glob: 8 = [N, E, Px, Py, Pz, Sum W, 0, 0].  Any output may be NULL. */
void orc_moments(const orc_params* P, int64_t n, const double* pos, const double* vel,
                 const double* virial, double* raw, double* derived, double* glob);

/* Radial velocity per c-bin (Eq. vel_r, the Noh and Sedov tests):
 * v_r = (1/N) Sum_i v_i . r_hat_i, r_hat_i the unit vector from `center` to
 * particle i over the position dimensions (a particle at the centre adds 0).
 * out: C x 2 = [Sum v . r_hat, v_r] (v_r = 0 in an empty c-bin). */
void orc_radial(const orc_params* P, int64_t n, const double* pos, const double* vel,
                const double* center, double* out);

/* One full step in place.  best_out (n), paired_out (n), raw/derived/glob
 * as in orc_moments; any may be NULL.  Returns the number of pairs. */
int64_t orc_step(const orc_params* P, int64_t n, double* pos, double* vel,
                 int32_t* best_out, int32_t* paired_out, double* raw,
                 double* derived, double* glob);

#ifdef __cplusplus
}
#endif
#endif
