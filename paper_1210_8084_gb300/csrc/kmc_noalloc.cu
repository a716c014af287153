// kmc_noalloc.cu -- closest-candidate search that allocates nothing.
//
// For callers that may not allocate device memory (a host framework that owns
// all device memory, a fixed device-memory budget, loops where cudaMalloc's
// implicit synchronisation is not acceptable): all scratch of the search lives
// in one file-scope __device__ array, reused by every call.  The kernels are
// the library's own (pack, bin, scan, scatter, search); only the buffers
// differ.  Calls share the array, so calls whose work overlaps on the GPU race.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "kmc_internal.h"

using namespace kmc;

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[KMC_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device with that device current (the array's name in host code is only
// a host-side stand-in).
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Particle tag stored in the w lane of a position vector.
__device__ __forceinline__ uint32_t tag_of(float w) { return __float_as_uint(w); }
__device__ __forceinline__ uint32_t tag_of(double w) {
    return (uint32_t)(unsigned long long)__double_as_longlong(w);
}

// The instance table, passed by value (kernel parameters live with the launch,
// so no host buffer has to outlive the call).
__global__ void put_instance(InstDev* dst, InstDev I) { *dst = I; }

// Closest candidate per particle (its tag is the low half of the partner
// key; one instance, so tag = id), by id.
template <typename T>
__global__ void __launch_bounds__(kThreads) best_by_id(Bufs<T> b, int32_t* __restrict__ out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= b.n) return;
    const uint32_t id = tag_of(b.posA[p].w);
    const unsigned long long k = b.bkey[p];
    out[id] = k != kNoPartner ? (int32_t)(uint32_t)k : -1;
}

template <typename T>
int run(const kmc_config* cfg, int64_t n, const void* pos, const void* vel, int32_t* best, void* base) {
    using V = typename Vec4<T>::type;
    cudaStream_t s = (cudaStream_t)cfg->stream;
    // geometry and the single instance (Eq. 7 and Eq. reff_lambda for R^2)
    Geo g{};
    g.dim = cfg->dim_pos;
    g.vdim = (cfg->flags & KMC_FLAG_VELOCITY_2D) ? 2 : 3;
    double V3 = 1.0;
    for (int d = 0; d < 3; ++d) {
        const bool used = d < g.dim;
        g.n[d] = used ? cfg->n_cells[d] : 1;
        g.bc[d] = used ? cfg->bc[d] : KMC_BC_PERIODIC;
        g.lo[d] = used ? cfg->lo[d] : 0.0;
        g.hi[d] = used ? cfg->hi[d] : 1.0;
        g.L[d] = g.hi[d] - g.lo[d];
        g.inv_dx[d] = (double)g.n[d] / (g.hi[d] - g.lo[d]);
        if (used) V3 *= g.L[d];
    }
    InstDev I{};
    I.p_off = 0;
    I.n = n;
    const double nbar = (double)n / V3;
    const double sigma = cfg->sigma > 0 ? cfg->sigma : 1.0 / (cfg->lambda * nbar);
    I.R2 = n > 0 ? sigma / M_PI : 0.0;
    I.dt = cfg->dt;
    I.R2f = (float)I.R2;
    I.dtf = (float)I.dt;
    I.seed_lo = (uint32_t)(cfg->seed & 0xffffffffu);
    I.seed_hi = (uint32_t)(cfg->seed >> 32);
    // adaptive timestep as a handle's first step takes it (set by the scan's step bookkeeping)
    I.adaptive = (cfg->flags & KMC_FLAG_ADAPTIVE_DT) ? 1 : 0;
    I.dx_min = INFINITY;
    for (int d = 0; d < g.dim; ++d) I.dx_min = fmin(I.dx_min, g.L[d] / g.n[d]);
    uint64_t keys = 1;
    for (int d = 0; d < 3; ++d) {
        I.s[d] = (d < g.dim && cfg->sub_cells[d] > 0) ? cfg->sub_cells[d] : 1;
        I.M[d] = g.n[d] * I.s[d];
        I.w[d] = g.L[d] / (double)I.M[d];
        keys *= (uint64_t)I.M[d];
    }
    if (keys > (uint64_t)KMC_STATIC_MAX_CELLS) return KMC_ERANGE;
    const uint32_t n_keys = (uint32_t)keys;
    const uint32_t n_tiles = (uint32_t)((keys + 2 + kScanTile - 1) / kScanTile);   // + absorbed key, end
    // carve the scratch array
    unsigned char* p = (unsigned char*)base;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char* q = p + off;
        off += align256(bytes);
        return q;
    };
    const size_t nv = (size_t)(n > 0 ? n : 1);
    Bufs<T> b{};
    b.n = n;
    b.n_inst = 1;
    b.st = (DevState*)take(sizeof(DevState));
    b.inst = (const InstDev*)take(sizeof(InstDev));
    b.dyn = (InstDyn*)take(sizeof(InstDyn));
    uint32_t* bad = (uint32_t*)take(sizeof(uint32_t));
    b.geo = g;
    b.posA = (V*)take(nv * sizeof(V));
    b.velA = (V*)take(nv * sizeof(V));
    b.posB = (V*)take(nv * sizeof(V));
    b.velB = (V*)take(nv * sizeof(V));
    b.bkey = (unsigned long long*)take(nv * sizeof(unsigned long long));
    b.slot_of = (uint32_t*)take(nv * sizeof(uint32_t));
    b.key = (uint32_t*)take(nv * sizeof(uint32_t));
    b.slot = (uint32_t*)take(nv * sizeof(uint32_t));
    b.tagB = (uint32_t*)take(nv * sizeof(uint32_t));
    b.count = (uint32_t*)take((size_t)n_tiles * kScanTile * sizeof(uint32_t));
    b.start = (uint32_t*)take((size_t)n_tiles * kScanTile * sizeof(uint32_t));
    b.scan_status = (unsigned long long*)take((1 + (size_t)n_tiles) * sizeof(unsigned long long));
    if (off > (size_t)KMC_STATIC_SCRATCH_BYTES) return KMC_ERANGE;
    b.n_keys = n_keys;
    b.n_tiles = n_tiles;
    b.any_direct = 1;
    b.tile_threads = 256;   // no instance here is tiled
    b.tile_cap = 1536;
    b.id_bits = 32;
    b.id_mask = 0xffffffffu;
    // the array keeps the last call's contents: clear what must start at zero
    put_instance<<<1, 1, 0, s>>>((InstDev*)b.inst, I);
    if (cudaGetLastError() != cudaSuccess) return KMC_ECUDA;
    if (cudaMemsetAsync(b.st, 0, sizeof(DevState), s) != cudaSuccess) return KMC_ECUDA;
    if (cudaMemsetAsync(b.dyn, 0, sizeof(InstDyn), s) != cudaSuccess) return KMC_ECUDA;
    if (cudaMemsetAsync(bad, 0, sizeof(uint32_t), s) != cudaSuccess) return KMC_ECUDA;
    if (cudaMemsetAsync(b.count, 0, (size_t)n_tiles * kScanTile * sizeof(uint32_t), s) != cudaSuccess)
        return KMC_ECUDA;
    if (n == 0) return KMC_OK;
    if (launch_pack<T>(b, (const T*)pos, (const T*)vel, bad, s) != cudaSuccess) return KMC_ECUDA;
    if (launch_bin_init<T>(b, s) != cudaSuccess) return KMC_ECUDA;
    if (launch_scan(b.count, b.start, n_keys, n_tiles, b.scan_status, b.dyn, b.inst, 1, b.st, g, 0, s) != cudaSuccess)
        return KMC_ECUDA;
    if (launch_scatter<T>(b, s) != cudaSuccess) return KMC_ECUDA;
    if (launch_search<T>(b, s) != cudaSuccess) return KMC_ECUDA;   // per particle (no instance is tiled here)
    best_by_id<T><<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, s>>>(b, best);
    return cudaGetLastError() == cudaSuccess ? KMC_OK : KMC_ECUDA;
}

}  // namespace

extern "C" KMC_API int kmc_find_partners_noalloc(const kmc_config* cfg, int64_t n, const void* pos,
                                                 const void* vel, int32_t* best) {
    if (!cfg) return KMC_EINVAL;
    if (cfg->dim_pos != 2 && cfg->dim_pos != 3) return KMC_EINVAL;
    if (cfg->precision != 32 && cfg->precision != 64) return KMC_EINVAL;
    if (cfg->n_instances > 1) return KMC_EINVAL;
    if (n < 0) return KMC_EINVAL;
    if (n > KMC_STATIC_MAX_PARTICLES) return KMC_ERANGE;
    if (n > 0 && (!pos || !vel || !best)) return KMC_EINVAL;
    // the checks of kmc_init
    if (!(cfg->dt > 0) || !isfinite(cfg->dt)) return KMC_EINVAL;
    if (!(cfg->sigma > 0) && !(cfg->lambda > 0)) return KMC_EINVAL;
    if (cfg->sigma > 0 && !isfinite(cfg->sigma)) return KMC_EINVAL;
    if (cfg->flags & ~(KMC_FLAG_RECORD | KMC_FLAG_NO_GRAPH | KMC_FLAG_STAGED_SEARCH | KMC_FLAG_NO_TILE_SEARCH |
                       KMC_FLAG_ADAPTIVE_DT | KMC_FLAG_VELOCITY_2D | KMC_FLAG_RADIAL_MOMENT))
        return KMC_EINVAL;   // KMC_FLAG_DSMC included: that variant has no closest candidates
    if ((cfg->flags & KMC_FLAG_VELOCITY_2D) && cfg->dim_pos != 2) return KMC_EINVAL;
    for (int d = 0; d < cfg->dim_pos; ++d) {
        if (cfg->n_cells[d] < 1 || !(cfg->hi[d] > cfg->lo[d])) return KMC_EINVAL;
        if (!isfinite(cfg->lo[d]) || !isfinite(cfg->hi[d])) return KMC_EINVAL;
        if (cfg->bc[d] != KMC_BC_PERIODIC && cfg->bc[d] != KMC_BC_WALL && cfg->bc[d] != KMC_BC_ABSORB)
            return KMC_EINVAL;
        if (cfg->sub_cells[d] < 0) return KMC_EINVAL;
    }
    void* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return KMC_ECUDA;
    return cfg->precision == 64 ? run<double>(cfg, n, pos, vel, best, base)
                                : run<float>(cfg, n, pos, vel, best, base);
}
