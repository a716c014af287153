// kmc_internal.h -- shared declarations of the sm_103a kinetic Monte Carlo library
// (device tables, handle, kernel launchers).  Host code and kernels include it;
// nothing outside csrc/ does.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/kmc.h"

namespace kmc {

constexpr int kThreads = 256;          // threads per block of the particle kernels
constexpr int kScanThreads = 256;      // scan: threads per tile
constexpr int kScanItems = 16;         // scan: keys per thread (4 x uint4)
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr uint32_t kSpinCap = 1u << 22;  // bounded waits: iterations before giving up
constexpr int kFoldCap = 64;           // wall folds per coordinate per step
constexpr int kAccFields = 10;         // per c-bin accumulator: N, Sum v (3), Sum v^2 (3), Sum W, collided
constexpr int kTestSlots = 256;        // counters of the pruned tile search's pair tests (blocks spread over them)
constexpr int kCbinRows = 4;           // rows of search cells per c-bin up to which moments go one warp per c-bin
constexpr int kPrunedCap = 1888;       // default staging capacity of the pruned tile search (28 B per slot)
                                       // count, Sum v.r_hat
constexpr int kMomStride = 18;         // per c-bin output: 8 raw, 8 derived, Sum v.r_hat, v_r
constexpr uint32_t kCanonMax = 16384;  // search cells up to this many particles are put in id order

// device error flags (DevState::error)
constexpr uint32_t kErrScanTimeout = 1u;
constexpr uint32_t kErrKeyRange = 2u;

constexpr unsigned long long kNoPartner = ~0ull;  // partner key of a particle without candidate
constexpr int kMomItems = 4;           // moments: consecutive particles per thread
constexpr int kStageThreads = 256;     // staged search: threads per tile

// Per-instance constants.  Geometry (box, c-bins, walls) is shared; the search
// grid subdivision s[] and the interaction constants are per instance.
struct InstDev {
    int64_t p_off;       // first particle of the instance (global index)
    int64_t n;           // particles of the instance
    uint32_t key_base;   // first search-grid key of the instance
    uint32_t bin_base;   // first c-bin (moment row) of the instance
    int s[3];            // subdivision of a c-bin into search cells per dimension
    int M[3];            // search cells per dimension = n_cells * s
    double R2;           // squared contact distance
    double dt;           // timestep
    float R2f, dtf;      // the same rounded to binary32 (binary32 kernels use these)
    uint32_t seed_lo, seed_hi;
    double w[3];         // search-cell width per dimension
    // staged search (3-D, sparse search cells): tiles of tile_rows consecutive
    // y-rows of one x-slab; the tile's neighbourhood rows are copied to
    // shared memory before the search
    int staged;
    int tiled;           // search cells are the c-bins: one block per cell (tile_search_kernel)
    int prune;           // tiled, binary32: candidate clusters out of a warp's reach are skipped
    int adaptive;        // timestep dx_min / v_max(t) per step (Sect. "Simulation setup")
    double dx_min;       // smallest c-bin width over the position dimensions
    int tile_rows;
    int tiles_per_x;     // ceil(M[1] / tile_rows)
    uint32_t tile_base;  // first tile of the instance in the staged launch
};

// Per-instance quantities that change every step (written on the device).
struct InstDyn {
    unsigned long long vmax2_cur;   // bits of the largest |v|^2 (binary64) of the current state
    unsigned long long vmax2_next;  // accumulated by the step's move kernel
    double dt;                      // timestep of the next step (the configured one unless adaptive)
    double dt_prev;                 // timestep of the step just taken (virial pressure)
    double time;                    // simulated time since the state was set
    float dtf;                      // dt rounded to binary32
    int k[3];                       // search half-window in search cells
    int mom_e[3];                   // moment sums: fixed-point exponents of v, v^2 and W
};

struct Geo {
    int dim;
    int vdim;   // velocity components: 3, or 2 (x, y only: the paper's 2-D runs)
    int n[3];
    int bc[3];
    double lo[3], hi[3], L[3], inv_dx[3];
    double rc[3];   // centre of the radial velocity moment
};

struct DevState {
    uint32_t step;        // Philox counter word 1 of the step being taken
    uint32_t error;       // kErr* bits
    uint32_t spin_cap;    // bounded waits: polls before giving up (0: kSpinCap)
    uint32_t hold_tile1;  // test of the bounded wait: scan tile hold_tile1 - 1 never publishes its
                          // status (0: none); set only through kmc_test_hold_scan
    uint32_t steps_left;  // steps still to take in the current graph-resident step loop
    uint32_t pad;
};

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    using type = float4;
};
struct __align__(32) dvec4 {
    double x, y, z, w;
};
template <>
struct Vec4<double> {
    using type = dvec4;
};

// Pointers and sizes of one simulation, passed by value to every launcher.
template <typename T>
struct Bufs {
    using V = typename Vec4<T>::type;
    int64_t n;
    int n_inst;
    const InstDev* inst;     // [n_inst]
    InstDyn* dyn;            // [n_inst]
    DevState* st;
    Geo geo;
    V* posA; V* velA;        // sorted state (search-grid key order)
    V* posB; V* velB;        // staging / unsorted end-of-step state
    unsigned long long* bkey;  // [n] partner key of A[p] (tag of the closest candidate, kNoPartner)
    uint32_t* slot_of;       // [n] by global id: sorted position in A (written by the search);
                             // the scatter reuses it for the tags of shared search cells
    uint32_t* key;           // [n] search key of B
    uint32_t* tagB;          // [n] tag of B[p], written with B (read coalesced by the scatter)
    uint32_t* slot;          // [n] rank of B[p] within its search cell
    uint32_t* count;         // [n_keys + 1] histogram (zero outside the step)
    uint32_t* start;         // [n_keys + 1] exclusive scan of count
    unsigned long long* scan_status;  // [1 + n_tiles]: ticket + tile descriptors
    uint32_t n_keys;
    uint32_t n_tiles;
    unsigned long long* acc; // [n_bins * kAccFields] moment sums, fixed point (two's complement)
    double* mom;             // [n_bins * kMomStride] raw, derived, radial
    double* glob;            // [n_inst * 8]
    int64_t n_bins;
    int32_t* rec_best;       // RECORD: [n] by global id
    int32_t* rec_partner;    // RECORD: [n] by global id
    int record;
    // staged search launch
    uint32_t n_stage_tiles;  // tiles over all staged instances (0: none)
    int stage_cap;           // candidate vectors a tile can stage
    int stage_rows;          // row slots of the staged start table
    int stage_stride;        // entries per row slot (max M[2] + 1, even)
    int stage_pair_cap;      // entries of the binary32 pair list
    int any_direct;          // some instance uses the direct (per-thread) search
    int any_tiled;           // some instance uses the tile search (one block per c-bin)
    int any_plain_tiled;     // some tiled instance searches on its c-bins (not pruned)
    int dsmc;                // the random-partner comparison variant instead of the PoCA search
    int radial;              // accumulate Sum v.r_hat (KMC_FLAG_RADIAL_MOMENT)
    int cbin_moments;        // every c-bin is at most kCbinRows runs of search cells: moments per c-bin
    int tile_threads;        // tile search: threads per c-bin block (a multiple of 32, 64 ... 256)
    int tile_cap;            // tile search: candidates staged in shared memory at once (even)
    int tile_split;          // tile search: blocks sharing one c-bin's window (binary32)
    int tile_prune;          // some instance uses the pruned tile search (binary32, half c-bins)
    unsigned long long* tile_tests;  // [kTestSlots] pair tests made by the pruned tile search (cumulative; may be null)
    // particle tag = (instance << id_bits) | instance-local id
    uint32_t id_bits;        // 32 when there is one instance
    uint32_t id_mask;
};

// Launchers (defined in kmc_kernels.cuh, instantiated per precision).
template <typename T>
cudaError_t launch_pack(const Bufs<T>& b, const T* pos3, const T* vel3, uint32_t* bad, cudaStream_t s);
template <typename T>
cudaError_t launch_bin_init(const Bufs<T>& b, cudaStream_t s);
template <typename T>
cudaError_t launch_search(const Bufs<T>& b, cudaStream_t s);       // staged + per-particle search
template <typename T>
cudaError_t launch_tile_search(const Bufs<T>& b, cudaStream_t s);  // one block per c-bin (tiled instances)
template <typename T>
cudaError_t prepare_staged(const Bufs<T>& b);
template <typename T>
size_t stage_smem_bytes(const Bufs<T>& b);
template <typename T>
cudaError_t prepare_tile(const Bufs<T>& b);
template <typename T>
size_t tile_smem_bytes(const Bufs<T>& b);
template <typename T>
cudaError_t launch_move(const Bufs<T>& b, cudaStream_t s);
template <typename T>
cudaError_t launch_scatter(const Bufs<T>& b, cudaStream_t s);
template <typename T>
cudaError_t launch_gather_state(const Bufs<T>& b, T* pos3, T* vel3, cudaStream_t s);
template <typename T>
cudaError_t launch_cell_keys(const Bufs<T>& b, int32_t* keys, cudaStream_t s);
template <typename T>
cudaError_t launch_moments(const Bufs<T>& b, int use_virial, cudaStream_t s);
template <typename T>
cudaError_t launch_window_count(const Bufs<T>& b, unsigned long long* total, cudaStream_t s);
template <typename T>
cudaError_t launch_perm(const Bufs<T>& b, int32_t* perm, cudaStream_t s);
template <typename T>
cudaError_t launch_dsmc(const Bufs<T>& b, cudaStream_t s);     // random-partner collisions per c-bin
template <typename T>
cudaError_t launch_cbin_hist(const Bufs<T>& b, uint32_t* hist, unsigned long long* vmax2, cudaStream_t s);

// precision-independent
cudaError_t launch_scan(uint32_t* count, uint32_t* start, uint32_t n_keys, uint32_t n_tiles,
                        unsigned long long* status, InstDyn* dyn, const InstDev* inst,
                        int n_inst, DevState* st, Geo geo, int bump_step, cudaStream_t s);
// gacc: [n_inst * 8] integer totals, zero between calls (the launch leaves it zero)
cudaError_t launch_finalize(const InstDev* inst, const InstDyn* dyn, int n_inst, Geo geo,
                            const unsigned long long* acc, double* mom, double* glob, unsigned long long* gacc,
                            int64_t n_bins, cudaStream_t s);

}  // namespace kmc
