// kmc_api.cu -- host side of the C ABI declared in include/kmc.h: validation,
// derived constants, search-grid choice, device memory, launch sequence of one
// step, CUDA-graph replay, getters.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "kmc_internal.h"

using namespace kmc;

namespace {

thread_local std::string g_init_error;

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct kmc_handle {
    kmc_config cfg;
    int precision = 32;
    int dim = 3;
    int64_t n = 0;
    int n_inst = 1;
    std::vector<InstDev> inst_h;
    Geo geo{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // device memory
    std::vector<DevBuf> allocs;
    void *posA = nullptr, *velA = nullptr, *posB = nullptr, *velB = nullptr;
    unsigned long long* bkey = nullptr;
    uint32_t* slot_of = nullptr;
    uint32_t *key = nullptr, *slot = nullptr, *tagB = nullptr, *count = nullptr, *start = nullptr, *bad = nullptr;
    unsigned long long* scan_status = nullptr;
    InstDev* inst_d = nullptr;
    InstDyn* dyn_d = nullptr;
    DevState* st_d = nullptr;
    unsigned long long* acc = nullptr;
    unsigned long long* gacc = nullptr;   // per-instance integer totals (zero between reductions)
    unsigned long long* tile_tests = nullptr;   // [kTestSlots] pair tests of the pruned tile search, cumulative
    double *mom = nullptr, *glob = nullptr;
    int32_t *rec_best = nullptr, *rec_partner = nullptr;
    uint32_t n_keys = 0, n_tiles = 0;
    uint32_t id_bits = 32;
    uint32_t n_stage_tiles = 0;
    int stage_cap = 0, stage_rows = 0, stage_stride = 0, stage_pair_cap = 0, any_direct = 1, any_tiled = 0;
    int any_plain_tiled = 0;
    int cbin_moments = 0;   // moments one warp per c-bin (every c-bin: at most kCbinRows runs of search cells)
    int tile_threads = 256, tile_cap = 1536, tile_split = 1, tile_prune = 1;
    int64_t n_bins = 0, bins_per_inst = 0;
    int64_t bytes = 0;
    int mom_state = 0;  // 1: acc/mom/glob describe the current state
    cudaGraphExec_t graph[2] = {nullptr, nullptr};       // one step (per want_moments)
    cudaGraphExec_t loop_graph[2] = {nullptr, nullptr};  // all steps of a call: device-side loop
    bool graph_failed = false;
    bool loop_failed = false;
    std::string err;
};

namespace {

#define KMC_CUDA(h, call)                                                                 \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            (h)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                \
            return KMC_ECUDA;                                                             \
        }                                                                                 \
    } while (0)

int fail(kmc_handle* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    else g_init_error = msg;
    return code;
}

size_t elem_size(const kmc_handle* h) { return h->precision == 64 ? sizeof(double) : sizeof(float); }
size_t vec_size(const kmc_handle* h) { return h->precision == 64 ? sizeof(dvec4) : sizeof(float4); }

int dev_alloc(kmc_handle* h, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(h, KMC_ENOMEM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
    h->allocs.push_back({*p, bytes});
    h->bytes += (int64_t)bytes;
    return KMC_OK;
}

template <typename T>
Bufs<T> make_bufs(const kmc_handle* h) {
    using V = typename Vec4<T>::type;
    Bufs<T> b;
    b.n = h->n;
    b.n_inst = h->n_inst;
    b.inst = h->inst_d;
    b.dyn = h->dyn_d;
    b.st = h->st_d;
    b.geo = h->geo;
    b.posA = (V*)h->posA;
    b.velA = (V*)h->velA;
    b.posB = (V*)h->posB;
    b.velB = (V*)h->velB;
    b.bkey = h->bkey;
    b.slot_of = h->slot_of;
    b.key = h->key;
    b.slot = h->slot;
    b.tagB = h->tagB;
    b.count = h->count;
    b.start = h->start;
    b.scan_status = h->scan_status;
    b.n_keys = h->n_keys;
    b.n_tiles = h->n_tiles;
    b.acc = h->acc;
    b.mom = h->mom;
    b.glob = h->glob;
    b.n_bins = h->n_bins;
    b.rec_best = h->rec_best;
    b.rec_partner = h->rec_partner;
    b.record = (h->cfg.flags & KMC_FLAG_RECORD) ? 1 : 0;
    b.n_stage_tiles = h->n_stage_tiles;
    b.stage_cap = h->stage_cap;
    b.stage_rows = h->stage_rows;
    b.stage_stride = h->stage_stride;
    b.stage_pair_cap = h->stage_pair_cap;
    b.any_direct = h->any_direct;
    b.any_tiled = h->any_tiled;
    b.any_plain_tiled = h->any_plain_tiled;
    b.dsmc = (h->cfg.flags & KMC_FLAG_DSMC) ? 1 : 0;
    b.radial = (h->cfg.flags & KMC_FLAG_RADIAL_MOMENT) ? 1 : 0;
    b.tile_threads = h->tile_threads;
    b.tile_cap = h->tile_cap;
    b.tile_split = h->tile_split;
    b.tile_prune = h->tile_prune;
    b.cbin_moments = h->cbin_moments;
    b.tile_tests = h->tile_tests;
    b.id_bits = h->id_bits;
    b.id_mask = h->id_bits >= 32 ? 0xffffffffu : ((1u << h->id_bits) - 1u);
    return b;
}

// One step: search, move (+ key, histogram), scan, scatter, moments and
// finalize (when wanted).  When `ev` is given, ev[k] is recorded before phase k
// and ev[KMC_NPHASES] at the end.
template <typename T>
cudaError_t enqueue_step(kmc_handle* h, int want_moments, cudaEvent_t* ev = nullptr) {
    const Bufs<T> b = make_bufs<T>(h);
    cudaStream_t s = h->stream;
    cudaError_t e;
    auto mark = [&](int k) { return ev ? cudaEventRecord(ev[k], s) : cudaSuccess; };
    if ((e = mark(KMC_PHASE_SEARCH)) != cudaSuccess) return e;
    if (b.dsmc) {   // random partners inside each c-bin instead of the closest-approach search
        if ((e = launch_dsmc<T>(b, s)) != cudaSuccess) return e;
    } else if ((e = launch_search<T>(b, s)) != cudaSuccess) {
        return e;
    }
    if ((e = mark(KMC_PHASE_TILE)) != cudaSuccess) return e;
    if (!b.dsmc && (e = launch_tile_search<T>(b, s)) != cudaSuccess) return e;
    if ((e = mark(KMC_PHASE_MOVE)) != cudaSuccess) return e;
    if ((e = launch_move<T>(b, s)) != cudaSuccess) return e;
    if ((e = mark(KMC_PHASE_SCAN)) != cudaSuccess) return e;
    if ((e = launch_scan(h->count, h->start, h->n_keys, h->n_tiles, h->scan_status, h->dyn_d, h->inst_d,
                         h->n_inst, h->st_d, h->geo, 1, s)) != cudaSuccess)
        return e;
    if ((e = mark(KMC_PHASE_SCATTER)) != cudaSuccess) return e;
    if ((e = launch_scatter<T>(b, s)) != cudaSuccess) return e;
    if ((e = mark(KMC_PHASE_MOMENTS)) != cudaSuccess) return e;
    if (want_moments) {
        e = cudaMemsetAsync(h->acc, 0, sizeof(unsigned long long) * kAccFields * (size_t)h->n_bins, s);
        if (e != cudaSuccess) return e;
        if ((e = launch_moments<T>(b, 1, s)) != cudaSuccess) return e;
    }
    if ((e = mark(KMC_PHASE_FINALIZE)) != cudaSuccess) return e;
    if (want_moments) {
        if ((e = launch_finalize(h->inst_d, h->dyn_d, h->n_inst, h->geo, h->acc, h->mom, h->glob, h->gacc, h->n_bins,
                                  s)) !=
            cudaSuccess)
            return e;
    }
    return mark(KMC_NPHASES);
}

cudaError_t enqueue_step_any(kmc_handle* h, int want_moments, cudaEvent_t* ev = nullptr) {
    return h->precision == 64 ? enqueue_step<double>(h, want_moments, ev)
                              : enqueue_step<float>(h, want_moments, ev);
}

// Sort the packed state in B into A (keys, histogram, scan, scatter).
template <typename T>
cudaError_t enqueue_bin(kmc_handle* h) {
    const Bufs<T> b = make_bufs<T>(h);
    cudaStream_t s = h->stream;
    cudaError_t e;
    if ((e = launch_bin_init<T>(b, s)) != cudaSuccess) return e;
    if ((e = launch_scan(h->count, h->start, h->n_keys, h->n_tiles, h->scan_status, h->dyn_d, h->inst_d,
                         h->n_inst, h->st_d, h->geo, 0, s)) != cudaSuccess)
        return e;
    return launch_scatter<T>(b, s);
}

// Validate and pack user arrays (already on the device) into B; returns the
// number of rejected particles through *bad_host.
int pack_inputs(kmc_handle* h, const void* pos_d, const void* vel_d, uint32_t* bad_host) {
    KMC_CUDA(h, cudaMemsetAsync(h->bad, 0, sizeof(uint32_t), h->stream));
    cudaError_t e;
    if (h->precision == 64)
        e = launch_pack<double>(make_bufs<double>(h), (const double*)pos_d, (const double*)vel_d, h->bad, h->stream);
    else
        e = launch_pack<float>(make_bufs<float>(h), (const float*)pos_d, (const float*)vel_d, h->bad, h->stream);
    KMC_CUDA(h, e);
    KMC_CUDA(h, cudaMemcpyAsync(bad_host, h->bad, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream));
    KMC_CUDA(h, cudaStreamSynchronize(h->stream));
    return KMC_OK;
}

// Bring user pos/vel onto the device: device pointers are used in place, host
// arrays are staged in the raw bytes of A (n x 3 x 2 elements fit in A).
int stage_inputs(kmc_handle* h, const void* pos, const void* vel, int where, const void** pos_d,
                 const void** vel_d) {
    const size_t bytes3 = (size_t)h->n * 3 * elem_size(h);
    if (where == KMC_WHERE_DEVICE) {
        *pos_d = pos;
        *vel_d = vel;
        return KMC_OK;
    }
    // each n x 3 array fits in the n vectors of posA / velA
    KMC_CUDA(h, cudaMemcpyAsync(h->posA, pos, bytes3, cudaMemcpyHostToDevice, h->stream));
    KMC_CUDA(h, cudaMemcpyAsync(h->velA, vel, bytes3, cudaMemcpyHostToDevice, h->stream));
    *pos_d = h->posA;
    *vel_d = h->velA;
    return KMC_OK;
}

int check_device_error(kmc_handle* h) {
    DevState st;
    KMC_CUDA(h, cudaMemcpyAsync(&st, h->st_d, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    KMC_CUDA(h, cudaStreamSynchronize(h->stream));
    if (st.error & kErrScanTimeout) return fail(h, KMC_ETIMEOUT, "device: a bounded wait in the key scan gave up");
    if (st.error) return fail(h, KMC_ETIMEOUT, "device: sort slot out of range (error flag " + std::to_string(st.error) + ")");
    return KMC_OK;
}

// Search-grid subdivision of instance i: cells of width >= D' (so the first
// step searches +-1 cell) and about `target` particles per cell in the
// densest c-bin, capped so the key count stays within a few times N.
void choose_subdivision(const kmc_handle* h, InstDev& I, double vmax, uint32_t max_bin_occ) {
    const double dt0 = (I.adaptive && vmax > 0.0) ? I.dx_min / vmax : I.dt;   // timestep of step 0
    const double D = sqrt(I.R2) + 2.0 * vmax * dt0;
    int smax[3] = {1, 1, 1};
    int nsub = 0;
    for (int d = 0; d < h->dim; ++d) {
        const double dx = h->geo.L[d] / h->geo.n[d];
        // cells 10% wider than the step-0 reach, so the window stays +-1 cell
        // while v_max drifts up with the sampled Maxwell tail
        const double Dp = 1.1 * (D * 1.001 + 1e-5 * h->geo.L[d]);
        double r = dx / Dp;
        if (!(r >= 1.0)) r = 1.0;
        if (r > 4096.0) r = 4096.0;
        smax[d] = (int)floor(r);
        if (smax[d] >= 2) ++nsub;
    }
    int s[3] = {1, 1, 1};
    const double target = h->cfg.occupancy_target > 0 ? h->cfg.occupancy_target : 0.5;
    if (nsub > 0 && max_bin_occ > 0) {
        const double m = (double)max_bin_occ / target;  // search cells wanted per c-bin
        const double per_dim = pow(m > 1.0 ? m : 1.0, 1.0 / nsub);
        for (int d = 0; d < h->dim; ++d) {
            if (smax[d] >= 2) {
                int v = (int)ceil(per_dim);
                s[d] = std::max(1, std::min(v, smax[d]));
            }
        }
        // keep the key count within 8 N + 4 C for this instance
        const double C = (double)h->bins_per_inst;
        const double cap = 8.0 * (double)I.n + 4.0 * C;
        for (int guard = 0; guard < 64; ++guard) {
            double keys = C;
            for (int d = 0; d < h->dim; ++d) keys *= s[d];
            if (keys <= cap) break;
            int dmax = 0;
            for (int d = 1; d < h->dim; ++d)
                if (s[d] > s[dmax]) dmax = d;
            if (s[dmax] <= 1) break;
            s[dmax] = std::max(1, (int)(s[dmax] * 0.9));
        }
    }
    bool forced = false;
    for (int d = 0; d < 3; ++d) {
        if (d < h->dim && h->cfg.sub_cells[d] > 0) {
            s[d] = h->cfg.sub_cells[d];
            forced = true;
        }
        if (d >= h->dim || (h->cfg.flags & KMC_FLAG_DSMC)) s[d] = 1;   // DSMC: collision cells are the c-bins
    }
    // Pruned tile search (binary32): where the search cells would be the c-bins
    // (the reach exceeds half a c-bin) but the contact distance is at most half
    // the narrowest c-bin, search on half c-bins with one block per c-bin that
    // skips the candidate clusters out of reach.  Periodic dimensions need 6
    // c-bins or more (a window of 6 half c-bins that never meets its own image)
    // and the key count stays within the cap above.
    I.prune = 0;
    if (!forced && h->tile_prune && s[0] == 1 && s[1] == 1 && s[2] == 1 &&
        !(h->cfg.flags & (KMC_FLAG_DSMC | KMC_FLAG_NO_TILE_SEARCH | KMC_FLAG_STAGED_SEARCH))) {
        double wmin = h->geo.L[0] / h->geo.n[0];
        bool ok = true;
        double keys = (double)h->bins_per_inst;
        for (int d = 0; d < h->dim; ++d) {
            wmin = std::min(wmin, h->geo.L[d] / h->geo.n[d]);
            if (h->geo.bc[d] == KMC_BC_PERIODIC && h->geo.n[d] < 6) ok = false;
            keys *= 2.0;
        }
        ok = ok && sqrt(I.R2) <= 0.5 * wmin && keys <= 8.0 * (double)I.n + 4.0 * (double)h->bins_per_inst;
        if (ok) {
            for (int d = 0; d < h->dim; ++d) s[d] = 2;
            I.prune = 1;
        }
    }
    for (int d = 0; d < 3; ++d) {
        I.s[d] = s[d];
        I.M[d] = h->geo.n[d] * s[d];
        I.w[d] = h->geo.L[d] / (double)I.M[d];
    }
}

// Staged search plan (3-D only): a tile is tile_rows y-rows of one x-slab,
// sized for about one block of home particles in the densest rows; the tile's
// neighbourhood (3 x-slabs by tile_rows + 2 y-rows at the first step) must
// fit the shared-memory budget, otherwise the instance is searched directly.
void plan_staged_search(kmc_handle* h, const std::vector<uint32_t>& max_occ) {
    const size_t vbytes = vec_size(h);
    const size_t budget = 160 * 1024;
    uint32_t tiles = 0;
    int cap = 0, rows = 0, stride = 0, pcap = 0, direct = 0;
    for (int i = 0; i < h->n_inst; ++i) {
        InstDev& I = h->inst_h[i];
        I.staged = 0;
        I.tile_rows = 1;
        I.tiles_per_x = 1;
        I.tile_base = tiles;
        bool ok = h->dim == 3 && I.n > 0 && (h->cfg.flags & KMC_FLAG_STAGED_SEARCH);
        double ppr = 1.0;   // particles per y-row (all z) in the densest c-bins
        if (ok) {
            ppr = std::max(1.0, (double)max_occ[i] * h->geo.n[2] / ((double)I.s[0] * I.s[1]));
            int R = (int)std::floor(0.9 * kStageThreads / ppr);
            R = std::max(1, std::min(R, I.M[1]));
            const int nxs = std::min(3, I.M[0]);
            const int rows_i = nxs * (R + 4);
            const int cap_i = ((int)std::ceil(nxs * (R + 2) * ppr * 1.3) + 64 + 31) / 32 * 32;
            // pair list: home particles x candidates (27 search cells of the window)
            const double cand = 27.0 * ppr / I.M[2];
            const int pcap_i = h->precision == 32 ? ((int)std::ceil(R * ppr * cand * 1.5) + 512 + 31) / 32 * 32 : 0;
            const size_t bytes = (size_t)cap_i * 2 * vbytes + (size_t)rows_i * (I.M[2] + 2) * sizeof(uint32_t) +
                                 (size_t)pcap_i * 4 + 2 * kStageThreads * 12 + 4;
            ok = I.s[0] == 1 && R + 4 < I.M[1] && rows_i <= 64 && bytes <= budget && cap_i < 65536 &&
                 R * ppr * 1.3 < 2 * kStageThreads;
            if (ok) {
                I.staged = 1;
                I.tile_rows = R;
                I.tiles_per_x = (I.M[1] + R - 1) / R;
                tiles += (uint32_t)(I.M[0] * I.tiles_per_x);
                cap = std::max(cap, cap_i);
                rows = std::max(rows, rows_i);
                stride = std::max(stride, (I.M[2] + 2) / 2 * 2);
                pcap = std::max(pcap, pcap_i);
            }
        }
        if (!ok) direct = 1;
    }
    const size_t total = (size_t)cap * 2 * vbytes + (size_t)rows * stride * sizeof(uint32_t) + (size_t)pcap * 4 +
                         2 * kStageThreads * 12 + 4;
    if (tiles > 0 && total > budget) {   // instances disagree too much: search all directly
        for (auto& I : h->inst_h) I.staged = 0;
        tiles = 0;
        direct = 1;
    }
    h->n_stage_tiles = tiles;
    h->stage_cap = cap;
    h->stage_rows = rows;
    h->stage_stride = stride;
    h->stage_pair_cap = pcap;
    h->any_direct = direct;
}

int validate_config(const kmc_config* c, int64_t n) {
    if (!c) return fail(nullptr, KMC_EINVAL, "cfg is NULL");
    if (c->dim_pos != 2 && c->dim_pos != 3) return fail(nullptr, KMC_EINVAL, "dim_pos must be 2 or 3");
    if (c->precision != 32 && c->precision != 64) return fail(nullptr, KMC_EINVAL, "precision must be 32 or 64");
    if (n < 0) return fail(nullptr, KMC_EINVAL, "n < 0");
    if (n >= (int64_t)INT32_MAX) return fail(nullptr, KMC_ERANGE, "n must be below 2^31 - 1");
    for (int d = 0; d < c->dim_pos; ++d) {
        if (c->n_cells[d] < 1) return fail(nullptr, KMC_EINVAL, "n_cells must be >= 1");
        if (!(c->hi[d] > c->lo[d]) || !isfinite(c->lo[d]) || !isfinite(c->hi[d]))
            return fail(nullptr, KMC_EINVAL, "box must satisfy lo < hi, finite");
        if (!isfinite(c->radial_center[d])) return fail(nullptr, KMC_EINVAL, "radial_center must be finite");
        if (c->bc[d] != KMC_BC_PERIODIC && c->bc[d] != KMC_BC_WALL && c->bc[d] != KMC_BC_ABSORB)
            return fail(nullptr, KMC_EINVAL, "bc must be KMC_BC_PERIODIC or KMC_BC_WALL");
        if (c->sub_cells[d] < 0) return fail(nullptr, KMC_EINVAL, "sub_cells must be >= 0");
    }
    if (c->n_instances < 0) return fail(nullptr, KMC_EINVAL, "n_instances < 0");
    if (c->n_instances > 1 && !c->instances) return fail(nullptr, KMC_EINVAL, "instances is NULL");
    if (c->flags &
        ~(KMC_FLAG_RECORD | KMC_FLAG_NO_GRAPH | KMC_FLAG_STAGED_SEARCH | KMC_FLAG_NO_TILE_SEARCH | KMC_FLAG_ADAPTIVE_DT |
          KMC_FLAG_VELOCITY_2D | KMC_FLAG_DSMC | KMC_FLAG_RADIAL_MOMENT | KMC_FLAG_NO_TILE_PRUNE))
        return fail(nullptr, KMC_EINVAL, "unknown flags");
    if (c->tile_threads != 0 && (c->tile_threads < 64 || c->tile_threads > 256 || (c->tile_threads & 31)))
        return fail(nullptr, KMC_EINVAL, "tile_threads must be 0 or a multiple of 32 from 64 to 256");
    if (c->tile_split < 0 || c->tile_split > 8) return fail(nullptr, KMC_EINVAL, "tile_split must be 0 ... 8");
    if (c->tile_cap != 0 && (c->tile_cap < 64 || (c->tile_cap & 1) || c->tile_cap > (c->precision == 64 ? 3072 : 6144)))
        return fail(nullptr, KMC_EINVAL, "tile_cap must be 0 or even, 64 ... 6144 (binary32) / 3072 (binary64)");
    if (c->flags & KMC_FLAG_DSMC) {
        for (int d = 0; d < c->dim_pos; ++d)
            if (c->sub_cells[d] > 1) return fail(nullptr, KMC_EINVAL, "KMC_FLAG_DSMC: the collision cells are the c-bins");
        if (c->flags & KMC_FLAG_STAGED_SEARCH) return fail(nullptr, KMC_EINVAL, "KMC_FLAG_DSMC has no search to stage");
    }
    if ((c->flags & KMC_FLAG_VELOCITY_2D) && c->dim_pos != 2)
        return fail(nullptr, KMC_EINVAL, "2-D velocities need dim_pos = 2");
    return KMC_OK;
}

int check_instance(const kmc_instance& I) {
    if (I.n_particles < 0) return fail(nullptr, KMC_EINVAL, "instance n_particles < 0");
    if (!(I.dt > 0) || !isfinite(I.dt)) return fail(nullptr, KMC_EINVAL, "dt must be finite and > 0");
    if (!(I.sigma > 0) && !(I.lambda > 0))
        return fail(nullptr, KMC_EINVAL, "need lambda > 0 (may be +inf) or sigma > 0");
    if (I.sigma > 0 && !isfinite(I.sigma)) return fail(nullptr, KMC_EINVAL, "sigma must be finite");
    return KMC_OK;
}

void release(kmc_handle* h) {
    if (!h) return;
    for (int g = 0; g < 2; ++g)
        if (h->graph[g]) cudaGraphExecDestroy(h->graph[g]);
    for (int g = 0; g < 2; ++g)
        if (h->loop_graph[g]) cudaGraphExecDestroy(h->loop_graph[g]);
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (auto& a : h->allocs) cudaFree(a.p);
    h->allocs.clear();
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

// Place the packed state of B into A and reset the per-step state.
int sort_packed(kmc_handle* h, uint32_t step) {
    DevState st{};
    st.step = step;
    KMC_CUDA(h, cudaMemcpyAsync(h->st_d, &st, sizeof(DevState), cudaMemcpyHostToDevice, h->stream));
    KMC_CUDA(h, cudaMemsetAsync(h->dyn_d, 0, sizeof(InstDyn) * h->n_inst, h->stream));
    KMC_CUDA(h, cudaMemsetAsync(h->count, 0, sizeof(uint32_t) * (size_t)h->n_tiles * kScanTile, h->stream));
    cudaError_t e = h->precision == 64 ? enqueue_bin<double>(h) : enqueue_bin<float>(h);
    KMC_CUDA(h, e);
    h->mom_state = 0;
    return check_device_error(h);
}

// Device side of the graph-resident step loop: the body of a conditional
// while node is one step followed by this kernel, which counts the step and
// clears the loop's condition after the last one.
__global__ void loop_control(DevState* st, cudaGraphConditionalHandle loop) {
    const uint32_t left = st->steps_left > 0u ? st->steps_left - 1u : 0u;
    st->steps_left = left;
    cudaGraphSetConditional(loop, left > 0u ? 1u : 0u);
}

__global__ void set_steps_left(DevState* st, uint32_t n) { st->steps_left = n; }

// One executable graph that runs steps_left steps of the handle: a while node
// (condition 1 at every launch) whose body is the step's launch sequence plus
// loop_control.  Returns an error (the caller falls back to one graph per
// step) where conditional nodes are not available.
cudaError_t build_loop_graph(kmc_handle* h, int want_moments, cudaGraphExec_t* out) {
    *out = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle loop;
    e = cudaGraphConditionalHandleCreate(&loop, g, 1u, cudaGraphCondAssignDefault);
    cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};   // the rest zero
    p.conditional.handle = loop;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &p);
    if (e == cudaSuccess) {
        cudaGraph_t body = p.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 = enqueue_step_any(h, want_moments);
            if (e1 == cudaSuccess) {
                loop_control<<<1, 1, 0, h->stream>>>(h->st_d, loop);
                e1 = cudaGetLastError();
            }
            cudaError_t e2 = cudaStreamEndCapture(h->stream, &body);
            e = e1 != cudaSuccess ? e1 : e2;
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (e != cudaSuccess) *out = nullptr;
    cudaGraphDestroy(g);
    return e;
}

}  // namespace

extern "C" {

const char* kmc_last_error(const kmc_handle* h) { return h ? h->err.c_str() : g_init_error.c_str(); }

int kmc_init(const kmc_config* cfg, int64_t n, const void* pos, const void* vel, int where, kmc_handle** out) {
    g_init_error.clear();
    if (!out) return fail(nullptr, KMC_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate_config(cfg, n);
    if (rc) return rc;
    if (n > 0 && (!pos || !vel)) return fail(nullptr, KMC_EINVAL, "pos/vel is NULL");
    if (where != KMC_WHERE_HOST && where != KMC_WHERE_DEVICE) return fail(nullptr, KMC_EINVAL, "bad where");

    std::vector<kmc_instance> insts;
    if (cfg->n_instances <= 1) {
        kmc_instance I{n, cfg->lambda, cfg->sigma, cfg->dt, cfg->seed};
        insts.push_back(I);
    } else {
        int64_t tot = 0;
        for (int i = 0; i < cfg->n_instances; ++i) {
            insts.push_back(cfg->instances[i]);
            tot += cfg->instances[i].n_particles;
        }
        if (tot != n) return fail(nullptr, KMC_EINVAL, "sum of instance particle counts differs from n");
    }
    for (auto& I : insts)
        if ((rc = check_instance(I))) return rc;

    kmc_handle* h = new kmc_handle();
    h->cfg = *cfg;
    h->cfg.instances = nullptr;
    h->precision = cfg->precision;
    h->dim = cfg->dim_pos;
    h->n = n;
    h->n_inst = (int)insts.size();
    h->tile_threads = cfg->tile_threads > 0 ? cfg->tile_threads : 256;
    h->tile_cap = cfg->tile_cap > 0 ? cfg->tile_cap : (h->precision == 64 ? 768 : 1536);
    h->tile_split = h->precision == 64 ? 1 : (cfg->tile_split > 0 ? cfg->tile_split : 1);
    h->tile_prune = h->precision == 32 && !(cfg->flags & KMC_FLAG_NO_TILE_PRUNE) ? 1 : 0;

    Geo& g = h->geo;
    g.dim = h->dim;
    g.vdim = (cfg->flags & KMC_FLAG_VELOCITY_2D) ? 2 : 3;
    for (int d = 0; d < 3; ++d) {
        const bool used = d < h->dim;
        g.rc[d] = used ? cfg->radial_center[d] : 0.0;
        g.n[d] = used ? cfg->n_cells[d] : 1;
        g.bc[d] = used ? cfg->bc[d] : KMC_BC_PERIODIC;
        g.lo[d] = used ? cfg->lo[d] : 0.0;
        g.hi[d] = used ? cfg->hi[d] : 1.0;
        g.L[d] = g.hi[d] - g.lo[d];
        g.inv_dx[d] = (double)g.n[d] / (g.hi[d] - g.lo[d]);
    }
    h->bins_per_inst = (int64_t)g.n[0] * g.n[1] * g.n[2];
    h->n_bins = h->bins_per_inst * h->n_inst;
    if (h->n_bins > (int64_t)UINT32_MAX / 2) {
        delete h;
        return fail(nullptr, KMC_ERANGE, "too many c-bins");
    }
    double V = 1.0;
    for (int d = 0; d < h->dim; ++d) V *= g.L[d];
    // particle tag: instance index above the local id
    {
        uint32_t inst_bits = 0;
        while ((1ll << inst_bits) < (long long)h->n_inst) ++inst_bits;
        h->id_bits = 32 - inst_bits;
        int64_t nmax = 0;
        for (auto& I : insts) nmax = std::max(nmax, I.n_particles);
        if (inst_bits > 0 && nmax > (int64_t)(1ll << h->id_bits)) {
            delete h;
            return fail(nullptr, KMC_ERANGE, "instance too large for the particle tag: fewer instances or particles");
        }
    }

    int64_t off = 0;
    for (int i = 0; i < h->n_inst; ++i) {
        InstDev I{};
        I.p_off = off;
        I.n = insts[i].n_particles;
        off += I.n;
        I.bin_base = (uint32_t)(i * h->bins_per_inst);
        // Eq. 7 and Eq. reff_lambda: sigma = 1/(lambda n), R^2 = (2 r_eff)^2 = sigma/pi
        const double nbar = (double)I.n / V;
        const double sigma = insts[i].sigma > 0 ? insts[i].sigma : 1.0 / (insts[i].lambda * nbar);
        I.R2 = I.n > 0 ? sigma / M_PI : 0.0;
        I.dt = insts[i].dt;
        I.R2f = (float)I.R2;
        I.dtf = (float)I.dt;
        I.adaptive = (cfg->flags & KMC_FLAG_ADAPTIVE_DT) ? 1 : 0;
        I.dx_min = INFINITY;
        for (int d = 0; d < h->dim; ++d) I.dx_min = std::min(I.dx_min, g.L[d] / g.n[d]);
        I.seed_lo = (uint32_t)(insts[i].seed & 0xffffffffu);
        I.seed_hi = (uint32_t)(insts[i].seed >> 32);
        for (int d = 0; d < 3; ++d) {
            I.s[d] = 1;
            I.M[d] = g.n[d];
            I.w[d] = g.L[d] / g.n[d];
        }
        h->inst_h.push_back(I);
    }

    // stream
    if (cfg->stream) {
        h->stream = (cudaStream_t)cfg->stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            g_init_error = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
            delete h;
            return KMC_ECUDA;
        }
        h->own_stream = true;
    }

    auto bail = [&](int code) {
        std::string m = h->err;
        release(h);
        delete h;
        g_init_error = m;
        return code;
    };

    // particle buffers
    const size_t nv = (size_t)std::max<int64_t>(n, 1);
    if ((rc = dev_alloc(h, &h->posA, nv * vec_size(h)))) return bail(rc);
    if ((rc = dev_alloc(h, &h->velA, nv * vec_size(h)))) return bail(rc);
    if ((rc = dev_alloc(h, &h->posB, nv * vec_size(h)))) return bail(rc);
    if ((rc = dev_alloc(h, &h->velB, nv * vec_size(h)))) return bail(rc);
    if ((rc = dev_alloc(h, (void**)&h->bkey, nv * sizeof(unsigned long long)))) return bail(rc);
    if ((rc = dev_alloc(h, (void**)&h->slot_of, nv * sizeof(uint32_t)))) return bail(rc);
    if ((rc = dev_alloc(h, (void**)&h->key, nv * sizeof(uint32_t)))) return bail(rc);
    if ((rc = dev_alloc(h, (void**)&h->slot, nv * sizeof(uint32_t)))) return bail(rc);
    if ((rc = dev_alloc(h, (void**)&h->tagB, nv * sizeof(uint32_t)))) return bail(rc);
    if ((rc = dev_alloc(h, (void**)&h->inst_d, sizeof(InstDev) * h->n_inst))) return bail(rc);
    if ((rc = dev_alloc(h, (void**)&h->dyn_d, sizeof(InstDyn) * h->n_inst))) return bail(rc);
    if ((rc = dev_alloc(h, (void**)&h->st_d, sizeof(DevState)))) return bail(rc);
    if ((rc = dev_alloc(h, (void**)&h->bad, sizeof(uint32_t) * 4))) return bail(rc);
    if ((rc = dev_alloc(h, (void**)&h->acc, sizeof(unsigned long long) * kAccFields * (size_t)h->n_bins)))
        return bail(rc);
    if ((rc = dev_alloc(h, (void**)&h->mom, sizeof(double) * kMomStride * (size_t)h->n_bins))) return bail(rc);
    if ((rc = dev_alloc(h, (void**)&h->glob, sizeof(double) * 8 * (size_t)h->n_inst))) return bail(rc);
    if ((rc = dev_alloc(h, (void**)&h->gacc, sizeof(unsigned long long) * 8 * (size_t)h->n_inst))) return bail(rc);
    if ((rc = dev_alloc(h, (void**)&h->tile_tests, sizeof(unsigned long long) * kTestSlots))) return bail(rc);
    if (cudaMemsetAsync(h->tile_tests, 0, sizeof(unsigned long long) * kTestSlots, h->stream) != cudaSuccess)
        return bail(fail(h, KMC_ECUDA, "memset of the tile-search test counters failed"));
    if (cudaMemsetAsync(h->gacc, 0, sizeof(unsigned long long) * 8 * (size_t)h->n_inst, h->stream) != cudaSuccess)
        return bail(fail(h, KMC_ECUDA, "memset of the moment totals failed"));
    if (cfg->flags & KMC_FLAG_RECORD) {
        if ((rc = dev_alloc(h, (void**)&h->rec_best, nv * sizeof(int32_t)))) return bail(rc);
        if ((rc = dev_alloc(h, (void**)&h->rec_partner, nv * sizeof(int32_t)))) return bail(rc);
        if (cudaMemsetAsync(h->rec_best, 0xff, nv * sizeof(int32_t), h->stream) != cudaSuccess ||
            cudaMemsetAsync(h->rec_partner, 0xff, nv * sizeof(int32_t), h->stream) != cudaSuccess)
            return bail(fail(h, KMC_ECUDA, "memset of record buffers failed"));
    }
    if (cudaMemcpyAsync(h->inst_d, h->inst_h.data(), sizeof(InstDev) * h->n_inst, cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess)
        return bail(fail(h, KMC_ECUDA, "upload of instance table failed"));

    // inputs -> B, validation
    const void *pos_d = nullptr, *vel_d = nullptr;
    if ((rc = stage_inputs(h, pos, vel, where, &pos_d, &vel_d))) return bail(rc);
    uint32_t bad = 0;
    if (n > 0 && (rc = pack_inputs(h, pos_d, vel_d, &bad))) return bail(rc);
    if (bad) return bail(fail(h, KMC_EINVAL, std::to_string(bad) + " particle(s) non-finite or outside the box"));

    // search grid: per-instance vmax and densest c-bin of the initial state
    {
        uint32_t* hist = nullptr;
        unsigned long long* vm = nullptr;
        if ((rc = dev_alloc(h, (void**)&hist, sizeof(uint32_t) * (size_t)h->n_bins))) return bail(rc);
        if ((rc = dev_alloc(h, (void**)&vm, sizeof(unsigned long long) * h->n_inst))) return bail(rc);
        std::vector<uint32_t> hist_h((size_t)h->n_bins, 0u);
        std::vector<unsigned long long> vm_h(h->n_inst, 0ull);
        bool okc = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (size_t)h->n_bins, h->stream) == cudaSuccess &&
                   cudaMemsetAsync(vm, 0, sizeof(unsigned long long) * h->n_inst, h->stream) == cudaSuccess;
        if (okc && n > 0) {
            const cudaError_t e = h->precision == 64
                                      ? launch_cbin_hist<double>(make_bufs<double>(h), hist, vm, h->stream)
                                      : launch_cbin_hist<float>(make_bufs<float>(h), hist, vm, h->stream);
            okc = e == cudaSuccess;
        }
        okc = okc &&
              cudaMemcpyAsync(hist_h.data(), hist, sizeof(uint32_t) * (size_t)h->n_bins, cudaMemcpyDeviceToHost,
                              h->stream) == cudaSuccess &&
              cudaMemcpyAsync(vm_h.data(), vm, sizeof(unsigned long long) * h->n_inst, cudaMemcpyDeviceToHost,
                              h->stream) == cudaSuccess &&
              cudaStreamSynchronize(h->stream) == cudaSuccess;
        if (!okc) return bail(fail(h, KMC_ECUDA, "search-grid statistics failed"));
        uint64_t keys = 0;
        std::vector<uint32_t> max_occ(h->n_inst, 0u);
        for (int i = 0; i < h->n_inst; ++i) {
            uint32_t mx = 0;
            for (int64_t b = 0; b < h->bins_per_inst; ++b) mx = std::max(mx, hist_h[(size_t)(i * h->bins_per_inst + b)]);
            max_occ[i] = mx;
            double v2;
            memcpy(&v2, &vm_h[i], sizeof(double));
            choose_subdivision(h, h->inst_h[i], sqrt(v2), mx);
            h->inst_h[i].key_base = (uint32_t)keys;
            keys += (uint64_t)h->inst_h[i].M[0] * h->inst_h[i].M[1] * h->inst_h[i].M[2];
            if (keys >= (uint64_t)UINT32_MAX - 2 * (uint64_t)kScanTile)
                return bail(fail(h, KMC_ERANGE, "search grid exceeds 2^32 keys; set sub_cells"));
        }
        h->n_keys = (uint32_t)keys;
        h->cbin_moments = 1;
        for (const InstDev& I : h->inst_h)
            if ((h->dim == 3 ? I.s[0] * I.s[1] : I.s[0]) > kCbinRows) h->cbin_moments = 0;
        // keys of the cells, one key after them for absorbed particles, and the end offset
        h->n_tiles = (uint32_t)((keys + 2 + kScanTile - 1) / kScanTile);
        plan_staged_search(h, max_occ);
        // search cells that are the c-bins themselves: one block per cell
        h->any_tiled = 0;
        h->any_plain_tiled = 0;
        h->any_direct = 0;
        int prune_any = 0;
        const bool dsmc = (h->cfg.flags & KMC_FLAG_DSMC) != 0;
        for (auto& I : h->inst_h) {
            if (dsmc) {   // no closest-approach search at all
                I.staged = I.tiled = 0;
                continue;
            }
            I.tiled = !I.staged && I.n > 0 && ((I.s[0] == 1 && I.s[1] == 1 && I.s[2] == 1) || I.prune) &&
                      !(h->cfg.flags & KMC_FLAG_NO_TILE_SEARCH);
            I.prune = I.prune && I.tiled;
            h->any_tiled |= I.tiled;
            h->any_plain_tiled |= I.tiled && !I.prune;
            h->any_direct |= !I.tiled && !I.staged;   // searched one thread per particle
            prune_any |= I.prune;
        }
        h->tile_prune = prune_any;
        // the pruned search's default staging capacity fills 4 blocks per SM
        if (prune_any && h->cfg.tile_cap == 0 && !h->any_plain_tiled) h->tile_cap = kPrunedCap;
        if (cudaMemcpyAsync(h->inst_d, h->inst_h.data(), sizeof(InstDev) * h->n_inst, cudaMemcpyHostToDevice,
                            h->stream) != cudaSuccess)
            return bail(fail(h, KMC_ECUDA, "upload of instance table failed"));
    }
    const size_t padded = (size_t)h->n_tiles * kScanTile;
    if ((rc = dev_alloc(h, (void**)&h->count, padded * sizeof(uint32_t)))) return bail(rc);
    if ((rc = dev_alloc(h, (void**)&h->start, padded * sizeof(uint32_t)))) return bail(rc);
    if ((rc = dev_alloc(h, (void**)&h->scan_status, (1 + (size_t)h->n_tiles) * sizeof(unsigned long long))))
        return bail(rc);
    if (h->n_stage_tiles > 0) {
        const cudaError_t e = h->precision == 64 ? prepare_staged<double>(make_bufs<double>(h))
                                                 : prepare_staged<float>(make_bufs<float>(h));
        if (e != cudaSuccess) return bail(fail(h, KMC_ECUDA, std::string("staged search set-up: ") + cudaGetErrorString(e)));
    }
    if (h->any_tiled) {
        const cudaError_t e = h->precision == 64 ? prepare_tile<double>(make_bufs<double>(h))
                                                 : prepare_tile<float>(make_bufs<float>(h));
        if (e != cudaSuccess) return bail(fail(h, KMC_ECUDA, std::string("tile search set-up: ") + cudaGetErrorString(e)));
    }
    if ((rc = sort_packed(h, 0u))) return bail(rc);
    *out = h;
    return KMC_OK;
}

int kmc_step(kmc_handle* h, int nsteps, int want_moments) {
    if (!h) return fail(nullptr, KMC_EINVAL, "handle is NULL");
    if (nsteps < 0) return fail(h, KMC_EINVAL, "nsteps < 0");
    want_moments = want_moments ? 1 : 0;
    if (nsteps == 0) return KMC_OK;
    if (h->n == 0) {
        // nothing moves; keep the step counter in step with the request
        DevState st;
        KMC_CUDA(h, cudaMemcpyAsync(&st, h->st_d, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
        KMC_CUDA(h, cudaStreamSynchronize(h->stream));
        st.step += (uint32_t)nsteps;
        KMC_CUDA(h, cudaMemcpyAsync(h->st_d, &st, sizeof(st), cudaMemcpyHostToDevice, h->stream));
        h->mom_state = 0;
        return KMC_OK;
    }
    const bool use_graph = !(h->cfg.flags & KMC_FLAG_NO_GRAPH) && !h->graph_failed;
    // all steps in one graph launch: the loop runs on the device
    if (use_graph && !h->loop_failed) {
        if (!h->loop_graph[want_moments] && build_loop_graph(h, want_moments, &h->loop_graph[want_moments]) != cudaSuccess) {
            cudaGetLastError();
            h->loop_failed = true;
        }
        if (h->loop_graph[want_moments]) {
            set_steps_left<<<1, 1, 0, h->stream>>>(h->st_d, (uint32_t)nsteps);
            KMC_CUDA(h, cudaGetLastError());
            KMC_CUDA(h, cudaGraphLaunch(h->loop_graph[want_moments], h->stream));
            h->mom_state = want_moments;
            return KMC_OK;
        }
    }
    if (use_graph && !h->graph[want_moments]) {
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 = enqueue_step_any(h, want_moments);
            cudaError_t e2 = cudaStreamEndCapture(h->stream, &graph);
            if (e1 == cudaSuccess && e2 == cudaSuccess) {
                e = cudaGraphInstantiate(&h->graph[want_moments], graph, 0);
                if (e != cudaSuccess) h->graph[want_moments] = nullptr;
            }
            if (graph) cudaGraphDestroy(graph);
        }
        if (!h->graph[want_moments]) {
            cudaGetLastError();
            h->graph_failed = true;
        }
    }
    for (int s = 0; s < nsteps; ++s) {
        if (use_graph && h->graph[want_moments]) {
            KMC_CUDA(h, cudaGraphLaunch(h->graph[want_moments], h->stream));
        } else {
            KMC_CUDA(h, enqueue_step_any(h, want_moments));
        }
    }
    h->mom_state = want_moments;
    return KMC_OK;
}

int kmc_step_profiled(kmc_handle* h, int nsteps, int want_moments, double* ms_out) {
    if (!h || !ms_out) return fail(h, KMC_EINVAL, "NULL argument");
    if (nsteps < 0) return fail(h, KMC_EINVAL, "nsteps < 0");
    want_moments = want_moments ? 1 : 0;
    for (int k = 0; k <= KMC_NPHASES; ++k) ms_out[k] = 0.0;
    if (nsteps == 0 || h->n == 0) return kmc_step(h, nsteps, want_moments);
    const int per = KMC_NPHASES + 1;
    std::vector<cudaEvent_t> ev((size_t)nsteps * per, nullptr);
    int rc = KMC_OK;
    for (auto& e : ev) {
        if (cudaEventCreate(&e) != cudaSuccess) {
            e = nullptr;
            rc = fail(h, KMC_ECUDA, "cudaEventCreate failed");
            break;
        }
    }
    for (int s = 0; rc == KMC_OK && s < nsteps; ++s) {
        cudaError_t e = enqueue_step_any(h, want_moments, ev.data() + (size_t)s * per);
        if (e != cudaSuccess) rc = fail(h, KMC_ECUDA, std::string("profiled step: ") + cudaGetErrorString(e));
    }
    if (rc == KMC_OK && cudaStreamSynchronize(h->stream) != cudaSuccess)
        rc = fail(h, KMC_ECUDA, "cudaStreamSynchronize failed");
    for (int s = 0; rc == KMC_OK && s < nsteps; ++s) {
        const cudaEvent_t* e = ev.data() + (size_t)s * per;
        for (int k = 0; k < KMC_NPHASES; ++k) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e[k], e[k + 1]);
            ms_out[k] += ms;
        }
    }
    if (rc == KMC_OK) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev.front(), ev.back());
        ms_out[KMC_NPHASES] = ms;
        h->mom_state = want_moments;
    }
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    if (rc == KMC_OK) rc = check_device_error(h);
    return rc;
}

int64_t kmc_moments_size(const kmc_handle* h, int mask) {
    if (!h) return 0;
    int64_t s = 0;
    if (mask & KMC_MOM_RAW) s += 8 * h->n_bins;
    if (mask & KMC_MOM_DERIVED) s += 8 * h->n_bins;
    if (mask & KMC_MOM_GLOBAL) s += 8 * (int64_t)h->n_inst;
    if (mask & KMC_MOM_RADIAL) s += 2 * h->n_bins;
    return s;
}

int kmc_moments(kmc_handle* h, double* out, int where, int mask) {
    if (!h) return fail(nullptr, KMC_EINVAL, "handle is NULL");
    if (!out) return fail(h, KMC_EINVAL, "out is NULL");
    if (where != KMC_WHERE_HOST && where != KMC_WHERE_DEVICE) return fail(h, KMC_EINVAL, "bad where");
    if (mask & ~(KMC_MOM_RAW | KMC_MOM_DERIVED | KMC_MOM_GLOBAL | KMC_MOM_RADIAL))
        return fail(h, KMC_EINVAL, "bad fields_mask");
    if (!h->mom_state) {
        KMC_CUDA(h, cudaMemsetAsync(h->acc, 0, sizeof(unsigned long long) * kAccFields * (size_t)h->n_bins,
                                    h->stream));
        cudaError_t e = h->precision == 64 ? launch_moments<double>(make_bufs<double>(h), 0, h->stream)
                                           : launch_moments<float>(make_bufs<float>(h), 0, h->stream);
        KMC_CUDA(h, e);
        KMC_CUDA(h, launch_finalize(h->inst_d, h->dyn_d, h->n_inst, h->geo, h->acc, h->mom, h->glob, h->gacc,
                                    h->n_bins, h->stream));
        h->mom_state = 1;
    }
    const cudaMemcpyKind kind = where == KMC_WHERE_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    double* o = out;
    if (h->n_bins > 0 && (mask & KMC_MOM_RAW)) {
        KMC_CUDA(h, cudaMemcpy2DAsync(o, 8 * sizeof(double), h->mom, kMomStride * sizeof(double), 8 * sizeof(double),
                                      (size_t)h->n_bins, kind, h->stream));
        o += 8 * h->n_bins;
    }
    if (h->n_bins > 0 && (mask & KMC_MOM_DERIVED)) {
        KMC_CUDA(h, cudaMemcpy2DAsync(o, 8 * sizeof(double), h->mom + 8, kMomStride * sizeof(double), 8 * sizeof(double),
                                      (size_t)h->n_bins, kind, h->stream));
        o += 8 * h->n_bins;
    }
    if (mask & KMC_MOM_GLOBAL) {
        KMC_CUDA(h, cudaMemcpyAsync(o, h->glob, sizeof(double) * 8 * h->n_inst, kind, h->stream));
        o += 8 * h->n_inst;
    }
    if ((mask & KMC_MOM_RADIAL) && !(h->cfg.flags & KMC_FLAG_RADIAL_MOMENT))
        return fail(h, KMC_ESTATE, "KMC_MOM_RADIAL needs a handle created with KMC_FLAG_RADIAL_MOMENT");
    if (h->n_bins > 0 && (mask & KMC_MOM_RADIAL)) {
        KMC_CUDA(h, cudaMemcpy2DAsync(o, 2 * sizeof(double), h->mom + 16, kMomStride * sizeof(double),
                                      2 * sizeof(double), (size_t)h->n_bins, kind, h->stream));
    }
    if (where == KMC_WHERE_HOST) return check_device_error(h);
    return KMC_OK;
}

int kmc_autotune(const kmc_config* cfg, int64_t n, const void* pos, const void* vel, int where, int trial_steps,
                 kmc_config* best, double* ms_per_step) {
    if (!cfg || !best) return fail(nullptr, KMC_EINVAL, "NULL argument");
    if (trial_steps < 1) return fail(nullptr, KMC_EINVAL, "trial_steps < 1");
    struct Trial {
        double occ;
        int flags;
        int tile_threads, tile_cap, tile_split;
    };
    const int keep = cfg->flags & ~(KMC_FLAG_NO_TILE_SEARCH | KMC_FLAG_STAGED_SEARCH | KMC_FLAG_NO_TILE_PRUNE);
    const int cap0 = cfg->precision == 64 ? 768 : 1536;
    std::vector<Trial> trials;
    for (double occ : {0.25, 0.35, 0.5, 0.7, 1.0, 1.5}) trials.push_back({occ, keep, 0, 0, 0});
    // threads per c-bin block and staging capacity of the tile search (these
    // trials are skipped as duplicates where the grid is subdivided)
    const int tile_opts[][3] = {{128, cap0, 1}, {256, 2 * cap0, 1}, {128, cap0 / 2, 1}, {256, cap0 / 2, 1},
                                {64, cap0 / 2, 1},   {256, cap0, 2},     {256, cap0, 3},      {128, cap0 / 2, 2}};
    for (const auto& t : tile_opts) trials.push_back({0.0, keep, t[0], t[1], t[2]});
    if (cfg->precision == 32) trials.push_back({0.0, keep | KMC_FLAG_NO_TILE_PRUNE, 0, 0, 0});
    trials.push_back({0.0, keep | KMC_FLAG_NO_TILE_SEARCH, 0, 0, 0});
    if (cfg->dim_pos == 3 && !(cfg->flags & KMC_FLAG_DSMC)) trials.push_back({0.0, keep | KMC_FLAG_STAGED_SEARCH, 0, 0, 0});
    double best_ms = -1.0;
    kmc_config pick = *cfg;
    int first_rc = KMC_OK;
    std::vector<std::vector<int>> tried;   // search set-up of every timed trial
    for (const Trial& t : trials) {
        kmc_config c = *cfg;
        c.sub_cells[0] = c.sub_cells[1] = c.sub_cells[2] = 0;
        c.occupancy_target = t.occ;
        c.flags = t.flags;
        c.tile_threads = t.tile_threads;
        c.tile_cap = t.tile_cap;
        c.tile_split = t.tile_split;
        kmc_handle* h = nullptr;
        const int rc = kmc_init(&c, n, pos, vel, where, &h);
        if (rc != KMC_OK) {
            if (rc == KMC_EINVAL) return rc;   // the configuration or the data are invalid
            if (first_rc == KMC_OK) first_rc = rc;
            continue;                          // e.g. out of memory for this subdivision
        }
        // settings that end in an already timed set-up (same subdivision and
        // search kernel for every instance) are not timed again
        std::vector<int> setup;
        for (const InstDev& I : h->inst_h) setup.insert(setup.end(), {I.s[0], I.s[1], I.s[2], I.tiled, I.staged});
        setup.push_back(h->any_tiled ? h->tile_threads : 0);
        setup.push_back(h->any_tiled ? h->tile_cap : 0);
        setup.push_back(h->any_tiled ? h->tile_split : 0);
        setup.push_back(h->any_tiled ? h->tile_prune : 0);
        if (std::find(tried.begin(), tried.end(), setup) != tried.end()) {
            kmc_free(h);
            continue;
        }
        tried.push_back(setup);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        float ms = 0.f;
        bool ok = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
        ok = ok && kmc_step(h, 1, 1) == KMC_OK && cudaEventRecord(e0, h->stream) == cudaSuccess &&
             kmc_step(h, trial_steps, 1) == KMC_OK && cudaEventRecord(e1, h->stream) == cudaSuccess &&
             kmc_sync(h) == KMC_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        kmc_free(h);
        if (!ok) return fail(nullptr, KMC_ECUDA, "autotune trial failed");
        const double per = (double)ms / trial_steps;
        if (best_ms < 0.0 || per < best_ms) {
            best_ms = per;
            pick = c;
        }
    }
    if (best_ms < 0.0) return first_rc != KMC_OK ? first_rc : fail(nullptr, KMC_ECUDA, "no autotune trial ran");
    *best = pick;
    if (ms_per_step) *ms_per_step = best_ms;
    return KMC_OK;
}

void kmc_free(kmc_handle* h) {
    if (!h) return;
    release(h);
    delete h;
}

int kmc_sync(kmc_handle* h) {
    if (!h) return fail(nullptr, KMC_EINVAL, "handle is NULL");
    return check_device_error(h);
}

int kmc_get_info(kmc_handle* h, kmc_info* info) {
    if (!h || !info) return fail(h, KMC_EINVAL, "NULL argument");
    DevState st;
    InstDyn dy;
    KMC_CUDA(h, cudaMemcpyAsync(&st, h->st_d, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
    KMC_CUDA(h, cudaMemcpyAsync(&dy, h->dyn_d, sizeof(dy), cudaMemcpyDeviceToHost, h->stream));
    KMC_CUDA(h, cudaStreamSynchronize(h->stream));
    memset(info, 0, sizeof(*info));
    info->n_particles = h->n;
    info->n_bins = h->n_bins;
    info->n_search_cells = h->n_keys;
    info->n_instances = h->n_inst;
    info->precision = h->precision;
    info->step = st.step;
    const InstDev& I = h->inst_h[0];
    for (int d = 0; d < 3; ++d) {
        info->sub_cells[d] = I.s[d];
        info->window[d] = dy.k[d];
    }
    info->R2 = I.R2;
    info->sigma = I.R2 * M_PI;
    info->dt = dy.dt;
    info->time = dy.time;
    double v2;
    memcpy(&v2, &dy.vmax2_cur, sizeof(double));
    info->vmax = sqrt(v2);
    info->bytes_device = h->bytes;
    info->stage_tiles = h->n_stage_tiles;
    info->tile_rows = I.staged ? I.tile_rows : 0;
    info->stage_cap = h->stage_cap;
    info->n_scan_tiles = (int)h->n_tiles;
    // per-particle search (also records slot_of outside tiled instances), tile
    // search, staged search, move, scan, two scatter passes,
    // then moments and two finalize kernels when moments are wanted
    info->kernels_per_step = ((h->any_direct || h->n_stage_tiles > 0) ? 1 : 0) + (h->any_plain_tiled ? 1 : 0) +
                             (h->tile_prune ? 1 : 0) +
                             (h->n_stage_tiles > 0 ? 1 : 0) + ((h->cfg.flags & KMC_FLAG_DSMC) ? 1 : 0) + 4;
    info->kernels_moments = 3;
    info->tile_threads = h->tile_threads;
    info->tile_cap = h->tile_cap;
    info->tile_split = h->tile_split;
    info->tile_prune = h->tile_prune;
    info->graph_mode = (h->cfg.flags & KMC_FLAG_NO_GRAPH) || h->graph_failed
                           ? 0
                           : ((h->loop_graph[0] || h->loop_graph[1]) ? 2 : (h->loop_failed ? 1 : 0));
    return KMC_OK;
}

int kmc_window_size(kmc_handle* h, double* mean_candidates) {
    if (!h || !mean_candidates) return fail(h, KMC_EINVAL, "NULL argument");
    *mean_candidates = 0.0;
    if (h->n == 0) return KMC_OK;
    // the scan-status words are free between steps: use one as the counter
    unsigned long long* total = h->scan_status;
    KMC_CUDA(h, cudaMemsetAsync(total, 0, sizeof(unsigned long long), h->stream));
    cudaError_t e = h->precision == 64 ? launch_window_count<double>(make_bufs<double>(h), total, h->stream)
                                       : launch_window_count<float>(make_bufs<float>(h), total, h->stream);
    KMC_CUDA(h, e);
    unsigned long long t = 0;
    KMC_CUDA(h, cudaMemcpyAsync(&t, total, sizeof(t), cudaMemcpyDeviceToHost, h->stream));
    KMC_CUDA(h, cudaStreamSynchronize(h->stream));
    *mean_candidates = (double)t / (double)h->n;
    return KMC_OK;
}

int kmc_tile_tests(kmc_handle* h, double* tests) {
    if (!h || !tests) return fail(h, KMC_EINVAL, "NULL argument");
    unsigned long long t[kTestSlots];
    KMC_CUDA(h, cudaMemcpyAsync(t, h->tile_tests, sizeof(t), cudaMemcpyDeviceToHost, h->stream));
    KMC_CUDA(h, cudaStreamSynchronize(h->stream));
    double sum = 0.0;
    for (int i = 0; i < kTestSlots; ++i) sum += (double)t[i];
    *tests = sum;
    return KMC_OK;
}

int kmc_get_state(kmc_handle* h, void* pos, void* vel, int where) {
    if (!h) return fail(nullptr, KMC_EINVAL, "handle is NULL");
    if (where != KMC_WHERE_HOST && where != KMC_WHERE_DEVICE) return fail(h, KMC_EINVAL, "bad where");
    if (h->n == 0) return KMC_OK;
    const size_t bytes3 = (size_t)h->n * 3 * elem_size(h);
    // B is free between steps; each n x 3 array fits in the n vectors of posB / velB
    void* pd = where == KMC_WHERE_DEVICE ? pos : (pos ? h->posB : nullptr);
    void* vd = where == KMC_WHERE_DEVICE ? vel : (vel ? h->velB : nullptr);
    cudaError_t e = h->precision == 64
                        ? launch_gather_state<double>(make_bufs<double>(h), (double*)pd, (double*)vd, h->stream)
                        : launch_gather_state<float>(make_bufs<float>(h), (float*)pd, (float*)vd, h->stream);
    KMC_CUDA(h, e);
    if (where == KMC_WHERE_HOST) {
        if (pos) KMC_CUDA(h, cudaMemcpyAsync(pos, h->posB, bytes3, cudaMemcpyDeviceToHost, h->stream));
        if (vel) KMC_CUDA(h, cudaMemcpyAsync(vel, h->velB, bytes3, cudaMemcpyDeviceToHost, h->stream));
        return check_device_error(h);
    }
    return KMC_OK;
}

int kmc_set_state(kmc_handle* h, const void* pos, const void* vel, int where, uint32_t step) {
    if (!h) return fail(nullptr, KMC_EINVAL, "handle is NULL");
    if (where != KMC_WHERE_HOST && where != KMC_WHERE_DEVICE) return fail(h, KMC_EINVAL, "bad where");
    if (h->n > 0 && (!pos || !vel)) return fail(h, KMC_EINVAL, "pos/vel is NULL");
    const void *pos_d = nullptr, *vel_d = nullptr;
    int rc;
    if ((rc = stage_inputs(h, pos, vel, where, &pos_d, &vel_d))) return rc;
    uint32_t bad = 0;
    if (h->n > 0 && (rc = pack_inputs(h, pos_d, vel_d, &bad))) return rc;
    if (bad) return fail(h, KMC_EINVAL, std::to_string(bad) + " particle(s) non-finite or outside the box");
    return sort_packed(h, step);
}

int kmc_get_cell_keys(kmc_handle* h, int32_t* keys, int where) {
    if (!h || !keys) return fail(h, KMC_EINVAL, "NULL argument");
    if (where != KMC_WHERE_HOST && where != KMC_WHERE_DEVICE) return fail(h, KMC_EINVAL, "bad where");
    if (h->n == 0) return KMC_OK;
    int32_t* dst = where == KMC_WHERE_DEVICE ? keys : (int32_t*)h->key;  // key[] is free between steps
    cudaError_t e = h->precision == 64 ? launch_cell_keys<double>(make_bufs<double>(h), dst, h->stream)
                                       : launch_cell_keys<float>(make_bufs<float>(h), dst, h->stream);
    KMC_CUDA(h, e);
    if (where == KMC_WHERE_HOST) {
        KMC_CUDA(h, cudaMemcpyAsync(keys, dst, sizeof(int32_t) * (size_t)h->n, cudaMemcpyDeviceToHost, h->stream));
        return check_device_error(h);
    }
    return KMC_OK;
}

int kmc_get_perm(kmc_handle* h, int32_t* perm, int where) {
    if (!h || !perm) return fail(h, KMC_EINVAL, "NULL argument");
    if (where != KMC_WHERE_HOST && where != KMC_WHERE_DEVICE) return fail(h, KMC_EINVAL, "bad where");
    if (h->n == 0) return KMC_OK;
    int32_t* dst = where == KMC_WHERE_DEVICE ? perm : (int32_t*)h->key;  // key[] is free between steps
    cudaError_t e = h->precision == 64 ? launch_perm<double>(make_bufs<double>(h), dst, h->stream)
                                       : launch_perm<float>(make_bufs<float>(h), dst, h->stream);
    KMC_CUDA(h, e);
    if (where == KMC_WHERE_HOST) {
        KMC_CUDA(h, cudaMemcpyAsync(perm, dst, sizeof(int32_t) * (size_t)h->n, cudaMemcpyDeviceToHost, h->stream));
        return check_device_error(h);
    }
    return KMC_OK;
}

int kmc_test_hold_scan(kmc_handle* h, int tile, uint32_t spin_cap) {
    if (!h) return fail(nullptr, KMC_EINVAL, "handle is NULL");
    if (tile < -1 || (tile >= 0 && (uint32_t)tile >= h->n_tiles))
        return fail(h, KMC_EINVAL, "tile must be -1 or a scan tile of the handle");
    if (spin_cap < 1) return fail(h, KMC_EINVAL, "spin_cap must be >= 1");
    // both words in one copy: spin_cap, then hold_tile1
    const uint32_t w[2] = {spin_cap, (uint32_t)(tile + 1)};
    static_assert(offsetof(DevState, hold_tile1) == offsetof(DevState, spin_cap) + sizeof(uint32_t),
                  "spin_cap and hold_tile1 are adjacent");
    KMC_CUDA(h, cudaMemcpyAsync((char*)h->st_d + offsetof(DevState, spin_cap), w, sizeof(w), cudaMemcpyHostToDevice,
                                h->stream));
    KMC_CUDA(h, cudaStreamSynchronize(h->stream));
    return KMC_OK;
}

int kmc_get_partners(kmc_handle* h, int32_t* best, int32_t* partner, int where) {
    if (!h) return fail(nullptr, KMC_EINVAL, "handle is NULL");
    if (!(h->cfg.flags & KMC_FLAG_RECORD)) return fail(h, KMC_ESTATE, "handle was created without KMC_FLAG_RECORD");
    if (where != KMC_WHERE_HOST && where != KMC_WHERE_DEVICE) return fail(h, KMC_EINVAL, "bad where");
    if (h->n == 0) return KMC_OK;
    const cudaMemcpyKind kind = where == KMC_WHERE_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const size_t bytes = sizeof(int32_t) * (size_t)h->n;
    if (best) KMC_CUDA(h, cudaMemcpyAsync(best, h->rec_best, bytes, kind, h->stream));
    if (partner) KMC_CUDA(h, cudaMemcpyAsync(partner, h->rec_partner, bytes, kind, h->stream));
    if (where == KMC_WHERE_HOST) return check_device_error(h);
    return KMC_OK;
}

}  // extern "C"
