/*
 * kmc.h -- C ABI of the GB300 (sm_103a) test-particle kinetic Monte Carlo step
 * of Sagert et al., "Hydrodynamic Shock Wave Studies within a Kinetic Monte Carlo
 * Approach" (arXiv:1210.8084).
 *
 * One step (Sect. "Simulation setup", Fig. 2 flow chart):
 *   1. bin particles by cell key (c-bins, Sect. "Simulation setup");
 *   2. for every particle, the closest collision candidate in its 3^D
 *      neighbourhood of c-bins that passes the PoCA acceptance test
 *      (negative crossing number chi, Eq. c_value; real overlap times,
 *      Eqs. collision_time/collision_time2; minimum distance, criterion 3);
 *   3. keep only unambiguous (mutually closest) pairs;
 *   4. isotropic elastic scattering in the pair's centre-of-mass frame;
 *   5. split free flight r + v_old t_poca + v_new (dt - t_poca) (Eqs. 12-14),
 *      plain free flight r + v dt for the others, reflective walls / periodic wrap;
 *   6. per-c-bin moments n, v_b, T, p (Eqs. vel_b, stress, 18, 19).
 *
 * Conventions: m = 1, k_B = 1, velocities 3-D.  Particle ids are the input
 * indices (instance-local in batched mode).  Every call returns KMC_OK (0) or a
 * negative KMC_E* code; kmc_last_error() gives a message.  All device work runs
 * on the stream given in kmc_config.stream (a private stream when NULL), in
 * order; calls that return host data synchronise that stream.
 *
 * Precision: precision = 32 holds particle state in binary32, precision = 64 in
 * binary64.  The decision quantities of the acceptance test are evaluated with a
 * fixed operation order (fused multiply-adds included) in the state precision.
 * Per-c-bin moment sums are exact 64-bit integer sums of every particle's
 * contribution rounded once to a grid of 2^-e (e per instance and field, set
 * each step from the largest speed so that no sum can overflow; far finer than
 * binary32 at every size the library accepts), returned as binary64: they do not
 * depend on the order in which particles are summed, so reruns, and a batched
 * run against the same instances run alone, give the same bits.
 */
#ifndef KMC_H
#define KMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define KMC_API __attribute__((visibility("default")))
#else
#define KMC_API
#endif

#define KMC_OK 0
#define KMC_EINVAL (-1)   /* invalid argument or configuration */
#define KMC_ENOMEM (-2)   /* device or host allocation failed */
#define KMC_ECUDA (-3)    /* a CUDA runtime call failed */
#define KMC_ETIMEOUT (-4) /* a bounded device-side wait gave up (state invalid) */
#define KMC_ERANGE (-5)   /* a size exceeds an internal limit */
#define KMC_ESTATE (-6)   /* call not valid in the handle's current state */

#define KMC_WHERE_HOST 0   /* pointer is host memory (pageable or pinned) */
#define KMC_WHERE_DEVICE 1 /* pointer is device memory of the current device */

#define KMC_BC_PERIODIC 0
#define KMC_BC_WALL 1      /* specular (reflective) wall, Sect. "Sod test" */
#define KMC_BC_ABSORB 2    /* absorbing wall, Sect. "Sedov test": a particle whose step ends outside the box
                            * leaves the simulation (no longer searched, moved or counted in the moments;
                            * kmc_get_state returns NaN position and velocity for it; a NaN position in the
                            * input of kmc_init / kmc_set_state marks a particle already absorbed) */

#define KMC_FLAG_RECORD 1   /* keep each particle's closest candidate and partner of the last step */
#define KMC_FLAG_NO_GRAPH 2 /* launch kernels directly instead of replaying a captured CUDA graph (by default
                             * kmc_step launches one graph that loops over all its steps on the device) */
#define KMC_FLAG_STAGED_SEARCH 4 /* stage tile neighbourhoods in shared memory (3-D; same results as the direct search) */
#define KMC_FLAG_NO_TILE_SEARCH 8 /* search unsubdivided grids per particle too (default: one block per c-bin; same results) */
#define KMC_FLAG_VELOCITY_2D 32  /* dim_pos = 2 only: velocities in the (x, y) plane (the paper's 2-D runs, f = 2,
                                  * gamma = 2): v_z must be 0, outgoing directions isotropic in the plane
                                  * (azimuth 2 pi u2 of the pair's draw), T = m v_rms^2 / 2 */
#define KMC_FLAG_DSMC 64   /* comparison variant, not the paper's method: the classic random-partner DSMC
                            * collisions the paper contrasts with PoCA (Sect. "Direct Simulation Monte Carlo
                            * Technique"), in Bird's no-time-counter form, instead of the closest-approach search:
                            * per c-bin of N particles and volume V_c, floor(N (N-1) sigma g_max dt / (2 V_c) + u)
                            * random candidate pairs (sigma of Eq. 7, g_max = 2 v_max), each accepted with
                            * probability |v_i - v_j| / g_max and scattered as the PoCA pairs are, one after
                            * another, then free flight for all.  The collision cells are the c-bins (sub_cells
                            * must be 0 or 1).  Collided particles count as paired in the moments (zero virial);
                            * kmc_get_partners reports -1 */
#define KMC_FLAG_RADIAL_MOMENT 128 /* also accumulate the radial velocity per c-bin (KMC_MOM_RADIAL, Eq. vel_r) */
#define KMC_FLAG_NO_TILE_PRUNE 256 /* binary32: no pruned tile search.  By default an instance whose automatic
                                    * search cells would be its c-bins (the reach exceeds half a c-bin), whose contact
                                    * distance R is at most half the narrowest c-bin and whose periodic dimensions
                                    * have 6 c-bins or more searches on half c-bins (sub_cells 2 per position
                                    * dimension) with one block per c-bin, where each group of 32 homes skips every
                                    * cluster of 4 candidates whose swept box (positions over the step) stays farther
                                    * than R, plus a rounding margin, from the group's, and each home then every
                                    * remaining cluster that stays as far from its own; same results */
#define KMC_FLAG_ADAPTIVE_DT 16  /* timestep dt(t) = dx_min / v_max(t) of each step's start state (Sect. "Simulation
                                  * setup"; dx_min the smallest c-bin width, v_max the largest speed of the instance,
                                  * |v|^2 = fma(vz, vz, fma(vy, vy, vx vx)) in the state precision, the quotient in
                                  * binary64, rounded to binary32 for binary32 state); the configured dt is used only
                                  * while every particle is at rest */

#define KMC_MOM_RAW 1       /* per c-bin: N, Sum vx, Sum vy, Sum vz, Sum vx^2, Sum vy^2, Sum vz^2, Sum W */
#define KMC_MOM_DERIVED 2   /* per c-bin: n, ux, uy, uz, T, p_kin, p_vir, p */
#define KMC_MOM_GLOBAL 4    /* per instance: N, E = 1/2 Sum |v|^2, Px, Py, Pz, Sum W, pairs, 0 */
#define KMC_MOM_RADIAL 8    /* per c-bin (handles with KMC_FLAG_RADIAL_MOMENT; KMC_ESTATE otherwise):
                             * Sum v.r_hat, v_r = Sum v.r_hat / N (Eq. vel_r; the Noh and Sedov tests),
                             * r_hat the unit vector from kmc_config.radial_center to the particle over the
                             * position dimensions (no periodic image; 0 for a particle at the centre) */

typedef struct kmc_handle kmc_handle;

/* One independent problem of a batched run (kmc_config.n_instances > 1).
 * Instances share geometry and precision; their particles are consecutive
 * blocks of the pos/vel arrays, in instance order. */
typedef struct kmc_instance {
    int64_t n_particles;
    double lambda;   /* mean free path (Eq. 7); used when sigma <= 0 */
    double sigma;    /* cross-section; > 0 overrides lambda */
    double dt;       /* timestep, > 0 */
    uint64_t seed;   /* Philox-4x32-10 key (low word, high word) */
} kmc_instance;

typedef struct kmc_config {
    int dim_pos;        /* position dimensions: 2 (x, y) or 3 (x, y, z) */
    int n_cells[3];     /* c-bins per dimension, each >= 1 (n_cells[2] ignored if dim_pos == 2) */
    double lo[3];       /* box lower corner */
    double hi[3];       /* box upper corner, hi > lo */
    int bc[3];          /* KMC_BC_PERIODIC or KMC_BC_WALL per dimension */
    double lambda;      /* single run: mean free path (used when sigma <= 0) */
    double sigma;       /* single run: cross-section (> 0 overrides lambda) */
    double dt;          /* single run: timestep */
    uint64_t seed;      /* single run: Philox key */
    int precision;      /* 32 or 64 */
    int n_instances;    /* 0 or 1: single run from the fields above; > 1: batched from instances[] */
    const kmc_instance* instances; /* n_instances entries when batched; read during kmc_init only */
    void* stream;       /* cudaStream_t; NULL = a stream owned by the handle */
    int sub_cells[3];   /* search-grid subdivision of each c-bin per dimension; 0 = automatic */
    double occupancy_target; /* automatic subdivision: particles per search cell aimed at (0 = 0.5) */
    int flags;          /* KMC_FLAG_* */
    double radial_center[3]; /* centre of the radial velocity moment (KMC_MOM_RADIAL), finite */
    int tile_threads;   /* search of unsubdivided grids (one block per c-bin): threads per block, a
                         * multiple of 32 from 64 to 256 (0 = 256); speed only, never results */
    int tile_cap;       /* the same: candidates staged in shared memory at once, even, 64 ... 6144 in
                         * binary32, 64 ... 3072 in binary64 (0 = 1536 / 768, 48 KiB); speed only */
    int tile_split;     /* the same, binary32: blocks that share one c-bin's candidates, 1 ... 8 (0 = 1);
                         * speed only */
} kmc_config;

/* Mean number of candidates a particle of the current state examines in the
 * search (the size of its search window; the paper's 3^D c-bin neighbourhood
 * restricted to the search cells that can hold a candidate).  Synchronises. */
KMC_API int kmc_window_size(kmc_handle* h, double* mean_candidates);

/* Pair tests the binary32 tile search has evaluated since kmc_init with its
 * pruning (KMC_FLAG_NO_TILE_PRUNE unset): 4 for every (home, cluster of 4
 * staged candidates) pair whose boxes meet (padding slots of a window row's
 * last cluster included).  0 for handles without that search.
 * The plain tile search tests (C_p - 1) / 2 pairs per particle, C_p from
 * kmc_window_size.  Synchronises the handle's stream. */
KMC_API int kmc_tile_tests(kmc_handle* h, double* tests);

/* Read-only description of a handle (kmc_get_info). */
typedef struct kmc_info {
    int64_t n_particles;     /* total over instances */
    int64_t n_bins;          /* c-bins over all instances (moment rows) */
    int64_t n_search_cells;  /* search-grid cells over all instances */
    int n_instances;
    int precision;
    uint32_t step;           /* steps taken since init (Philox counter word 1 of the next step) */
    int sub_cells[3];        /* subdivision of instance 0 */
    double R2;               /* instance 0: squared contact distance (2 r_eff)^2 = sigma / pi */
    double sigma;            /* instance 0 */
    double dt;               /* instance 0: timestep of the next step */
    double vmax;             /* instance 0: largest speed of the current state */
    int window[3];           /* instance 0: search half-width in search cells for the next step */
    int64_t bytes_device;    /* device memory held by the handle */
    int64_t stage_tiles;     /* tiles of the shared-memory staged search (0: direct search only) */
    int tile_rows;           /* instance 0: y-rows per staged tile (0: searched directly) */
    int stage_cap;           /* candidates a staged tile holds in shared memory */
    double time;             /* instance 0: simulated time since kmc_init or the last kmc_set_state */
    int n_scan_tiles;        /* tiles of the key scan (kmc_test_hold_scan) */
    int kernels_per_step;    /* kernels one kmc_step launches per step without moments */
    int kernels_moments;     /* kernels added per step when moments are wanted */
    int tile_threads;        /* tile search threads per c-bin block */
    int tile_cap;            /* tile search staging capacity (candidates) */
    int tile_split;          /* tile search blocks per c-bin */
    int graph_mode;          /* how the last kmc_step ran: 2 = one CUDA graph for all its steps (a device-side
                              * loop counter drives a conditional while node), 1 = one graph per step,
                              * 0 = kernel by kernel (KMC_FLAG_NO_GRAPH, or before the first kmc_step) */
    int tile_prune;          /* 1: the binary32 tile search skips candidate clusters out of reach (for some
                              * instance) */
} kmc_info;

/* Create a simulation.  pos and vel are n x 3 row-major arrays of float
 * (precision 32) or double (precision 64), in host or device memory per
 * `where`; in 2-D mode the z column of pos is carried unchanged.  The data are
 * copied (the caller keeps ownership).  Single run: n particles, ids 0..n-1.
 * Batched: n must equal the sum of instances[].n_particles.  Positions must be
 * finite and inside the box (walls: [lo, hi]; periodic: [lo, hi)), velocities
 * finite; violations give KMC_EINVAL.  *out is set only on success. */
KMC_API int kmc_init(const kmc_config* cfg, int64_t n, const void* pos, const void* vel,
             int where, kmc_handle** out);

/* Advance every instance by nsteps >= 0 steps (asynchronous on the handle's
 * stream).  want_moments != 0 accumulates the per-c-bin moments of each step's
 * end state (kmc_moments then returns those of the last step).  Returns
 * KMC_ETIMEOUT / KMC_ECUDA for failures detected so far (launch errors now,
 * device-side flags at the next synchronising call). */
KMC_API int kmc_step(kmc_handle* h, int nsteps, int want_moments);

/* Phases of one step, in launch order, for kmc_step_profiled. */
#define KMC_PHASE_SEARCH 0   /* closest candidate per particle (criteria 1-3), one thread per particle */
#define KMC_PHASE_TILE 1     /* the same, one block per c-bin, for grids whose search cells are the c-bins */
#define KMC_PHASE_MOVE 2     /* pairs, scattering, free flight, walls, next key and histogram */
#define KMC_PHASE_SCAN 3     /* exclusive scan of the key histogram */
#define KMC_PHASE_SCATTER 4  /* counting-sort scatter into (key, id) order */
#define KMC_PHASE_MOMENTS 5  /* per-c-bin moment sums of the new state (want_moments only) */
#define KMC_PHASE_FINALIZE 6 /* derived moments and per-instance totals (want_moments only) */
#define KMC_NPHASES 7

/* Same work as kmc_step, launched kernel by kernel (no graph) with a CUDA
 * event recorded on the handle's stream before and after every phase.
 * Synchronises the stream, then writes ms_out[KMC_NPHASES + 1]: the device
 * time of each phase summed over the nsteps steps, and the total from the
 * first to the last event.  Used to measure per-kernel durations. */
KMC_API int kmc_step_profiled(kmc_handle* h, int nsteps, int want_moments, double* ms_out);

/* Copy moments into out (caller-allocated doubles): the blocks selected by
 * fields_mask, in the order RAW (n_bins x 8), DERIVED (n_bins x 8),
 * GLOBAL (n_instances x 8), RADIAL (n_bins x 2).  Rows are c-bins with key c_x + n_x (c_y + n_y c_z),
 * instance-major.  Moments are those accumulated by the last kmc_step with
 * want_moments != 0, or, if none since the state was last set, of the current
 * state with zero virial.  Synchronises the stream when where == HOST. */
KMC_API int kmc_moments(kmc_handle* h, double* out, int where, int fields_mask);

/* Number of doubles kmc_moments writes for fields_mask. */
KMC_API int64_t kmc_moments_size(const kmc_handle* h, int fields_mask);

/* Release all device and host memory of the handle.  NULL-safe. */
KMC_API void kmc_free(kmc_handle* h);

/* Wait for the handle's stream; report device-side error flags. */
KMC_API int kmc_sync(kmc_handle* h);

/* Message of the last error on h (or of the last failed kmc_init if h is NULL). */
KMC_API const char* kmc_last_error(const kmc_handle* h);

KMC_API int kmc_get_info(kmc_handle* h, kmc_info* info);

/* Current state in id order (n x 3 each, state precision).  Synchronises
 * the stream when where == HOST.  Either pointer may be NULL. */
KMC_API int kmc_get_state(kmc_handle* h, void* pos, void* vel, int where);

/* Replace the state (same layout and checks as kmc_init) and set the step
 * counter; used for checkpoint/resume.  Discards pending moments. */
KMC_API int kmc_set_state(kmc_handle* h, const void* pos, const void* vel, int where, uint32_t step);

/* c-bin key c_x + n_x (c_y + n_y c_z) of every particle of the current state,
 * id order (int32, instance-local keys). */
KMC_API int kmc_get_cell_keys(kmc_handle* h, int32_t* keys, int where);

/* The sort permutation of the current state (Sect. "Simulation setup": particles
 * sorted into bins every step): perm[p] = index in the pos/vel arrays of
 * kmc_init (instance offset + instance-local id) of the particle at sorted
 * position p.  Sorted order is the search-grid key (instance, then search cell
 * with x slowest and the last position dimension fastest; a search cell is a
 * c-bin or, when kmc_info.sub_cells > 1, a subdivision of one), then id: the
 * particles of a search cell appear in increasing id.  Particles absorbed by a
 * wall come last, in no particular order; so do the particles of a search cell
 * holding more than 16384 (their cell is kept together, in no particular order
 * inside it).  int32[n]; synchronises the stream when where == HOST. */
KMC_API int kmc_get_perm(kmc_handle* h, int32_t* perm, int where);

/* Requires KMC_FLAG_RECORD.  best: closest candidate (instance-local id) of
 * each particle in the last step, -1 if none; partner: collision partner of the
 * last step (mutually closest), -1 if none.  Either pointer may be NULL. */
KMC_API int kmc_get_partners(kmc_handle* h, int32_t* best, int32_t* partner, int where);

/* Pick the implementation parameters of the search for a configuration by
 * measurement (the paper has no counterpart: these parameters change speed
 * only, never results).  For each candidate setting -- automatic subdivision
 * at several occupancy targets, the per-c-bin tile search (with several
 * threads per c-bin block and staging capacities) or the per-particle search
 * where the grid is not subdivided, and the shared-memory staged search for
 * 3-D grids -- a handle is created from (cfg, n, pos, vel, where) as in
 * kmc_init, warmed up for one step and timed over trial_steps >= 1 steps with
 * CUDA events on its stream, then freed; the caller's data are only read.
 * *best receives a copy of *cfg with occupancy_target, tile_threads, tile_cap,
 * tile_split and flags (the KMC_FLAG_NO_TILE_SEARCH / KMC_FLAG_STAGED_SEARCH / KMC_FLAG_NO_TILE_PRUNE bits) of the
 * fastest setting and sub_cells = 0 (automatic); *ms_per_step (may be NULL)
 * its time.
 * Device memory: one handle at a time.  Synchronises cfg->stream.  Returns
 * KMC_EINVAL for an invalid configuration or state; a setting whose handle
 * cannot be created (e.g. KMC_ENOMEM) is skipped, and its error is returned
 * only when no setting could be timed. */
KMC_API int kmc_autotune(const kmc_config* cfg, int64_t n, const void* pos, const void* vel, int where,
                         int trial_steps, kmc_config* best, double* ms_per_step);

/* Test hook of the failure detection (the paper has no counterpart).  The only
 * device-side wait of a step is the key scan's look-back on a predecessor
 * tile's status word, bounded by a poll cap (2^22 by default).  This call
 * lowers the cap to spin_cap >= 1 polls and, for tile >= 0 (a tile of the
 * handle's scan, kmc_info.n_scan_tiles), makes that tile withhold its status
 * in every following scan, so that the tiles after it run out of polls, give
 * up and return.  The step then completes with a wrong sort, and the next
 * synchronising call returns KMC_ETIMEOUT; kmc_set_state (or kmc_init) clears
 * the hold, the cap and the error.  tile = -1 only sets the cap.  Synchronises. */
KMC_API int kmc_test_hold_scan(kmc_handle* h, int tile, uint32_t spin_cap);

/* Closest-candidate search without any allocation.  The paper has no
 * counterpart: this entry point exists for callers that may not allocate
 * device memory themselves or through this library, e.g. a host framework
 * that owns all device memory through its own pool, code under a fixed
 * device-memory budget, or a loop where cudaMalloc's implicit device
 * synchronisation is not acceptable.  It computes, for one state, the
 * same closest candidate per particle (criteria 1-3) as the first step of a
 * kmc_init handle, writing best[id] = instance-local id of the candidate or -1.
 *
 * cfg: single instance only (n_instances <= 1; lambda/sigma, dt, box, cells,
 * walls, precision and KMC_FLAG_ADAPTIVE_DT / KMC_FLAG_VELOCITY_2D used as
 * kmc_init uses them, other flags accepted and without effect; sub_cells > 0
 * selects the search subdivision, 0 means plain c-bins (the results are the
 * same either way); stream as in kmc_init, NULL = legacy default stream).
 * The configuration is checked as kmc_init checks it.
 * pos, vel: device arrays n x 3 of float/double per cfg.precision; best:
 * device int32[n].  All scratch (packed state, keys, histogram, scan tiles)
 * lives in one file-scope __device__ array of KMC_STATIC_SCRATCH_BYTES that
 * every GPU loading the library holds until exit; n above
 * KMC_STATIC_MAX_PARTICLES or a search grid above KMC_STATIC_MAX_CELLS gives
 * KMC_ERANGE.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  Calls share the array and keep the last call's
 * contents: calls whose work overlaps on the GPU race, so issue them in order
 * on one stream.  Asynchronous on the stream; returns KMC_EINVAL / KMC_ERANGE /
 * KMC_ECUDA for argument, size or launch errors.  Validity of the particles is
 * not checked (unlike kmc_init), and failures detected on the device (the
 * scan's bounded wait giving up) are not reported: such a call returns KMC_OK
 * with unreliable best[]. */
#define KMC_STATIC_MAX_PARTICLES 262144
#define KMC_STATIC_MAX_CELLS 1048576
#define KMC_STATIC_SCRATCH_BYTES (48u << 20)
KMC_API int kmc_find_partners_noalloc(const kmc_config* cfg, int64_t n, const void* pos, const void* vel,
                                      int32_t* best);

#ifdef __cplusplus
}
#endif
#endif
