// kmc_scan.cu -- single-pass exclusive scan of the search-key histogram
// (decoupled look-back) and the moment finalisation kernels.
//
// The scan turns count[k] (particles per search cell) into start[k], the first
// sorted position of cell k, and clears count for the next step.  Tiles are
// claimed with an atomic ticket, so every predecessor of a tile has already
// started when the tile looks back; each wait is bounded (kSpinCap) and sets
// kErrScanTimeout instead of hanging.
//
// The block holding tile 0 also rolls the per-instance step bookkeeping: the
// largest speed of the new state becomes current and the search half-window
// k_d = ceil(D' / w_d) with D' = 1.001 (R + 2 v_max dt) + 1e-5 L_d is derived
// from it.  Any pair that passes the acceptance test is closer than
// R + |v_rel| t_poca <= R + 2 v_max dt at the start of the step, so the window
// never drops a candidate of the 3^D c-bin neighbourhood.  The same block sets
// the fixed-point exponents of the moment sums from the largest speed.
#include <math.h>

#include "kmc_internal.h"

namespace kmc {

namespace {

constexpr unsigned long long kFlagAgg = 1ull << 32;
constexpr unsigned long long kFlagInc = 2ull << 32;

__device__ __forceinline__ unsigned long long load_status(const unsigned long long* p) {
    return *reinterpret_cast<const volatile unsigned long long*>(p);
}

// Largest e (within [-120, 120]) with m 2^e < 2^62: a sum of terms bounded by
// m in total stays inside a signed 64-bit integer with a factor 2 to spare.
__device__ __forceinline__ int fixed_exponent(double m) {
    if (!(m > 0.0) || !isfinite(m)) return 0;
    const int e = 61 - ilogb(m);
    return e < -120 ? -120 : (e > 120 ? 120 : e);
}

__device__ void step_bookkeeping(InstDyn* dyn, const InstDev* inst, int n_inst, DevState* st, const Geo& geo,
                                 int bump) {
    for (int i = threadIdx.x; i < n_inst; i += blockDim.x) {
        const unsigned long long nx = dyn[i].vmax2_next;
        dyn[i].vmax2_cur = nx;
        dyn[i].vmax2_next = 0ull;
        const double vmax = sqrt(__longlong_as_double((long long)nx));
        // timestep of the next step: the configured one, or dx_min / v_max(t)
        // (adaptive; the previous one while every particle is at rest)
        const double prev = dyn[i].dt;
        double dt = inst[i].dt;
        if (inst[i].adaptive) dt = vmax > 0.0 ? inst[i].dx_min / vmax : (prev > 0.0 ? prev : inst[i].dt);
        if (bump) {
            dyn[i].dt_prev = prev;
            dyn[i].time += prev;
        } else {   // state set: no step taken yet
            dyn[i].dt_prev = dt;
        }
        dyn[i].dt = dt;
        dyn[i].dtf = (float)dt;
        const double D = sqrt(inst[i].R2) + 2.0 * vmax * dt;
        for (int d = 0; d < 3; ++d) {
            const double Dp = D * 1.001 + 1e-5 * geo.L[d];
            const double r = Dp / inst[i].w[d];
            int k = inst[i].M[d];
            if (r < (double)inst[i].M[d]) k = (int)ceil(r);
            dyn[i].k[d] = k < 1 ? 1 : k;
        }
        // Moment sums (fixed point): over the instance's n particles |v_d| <= v_max,
        // v_d^2 <= v_max^2, and a collided particle's |W| = |r_ij(t_poca) . dv| <=
        // R (1 + sqrt 2) v_max (the pair's PoCA distance is at most R, and the
        // pair's energy bounds the pre-collision speed by sqrt 2 v_max); the
        // factors 1 + 1e-6 and 4 cover the rounding of |v|^2 and of W.
        const double nn = (double)(inst[i].n > 0 ? inst[i].n : 1);
        const double vm = vmax * (1.0 + 1e-6);
        dyn[i].mom_e[0] = vm > 0.0 ? fixed_exponent(nn * vm) : 120;
        dyn[i].mom_e[1] = vm > 0.0 ? fixed_exponent(nn * vm * vm) : 120;
        const double wm = nn * 4.0 * sqrt(inst[i].R2) * vm;
        dyn[i].mom_e[2] = wm > 0.0 ? fixed_exponent(wm) : 120;
    }
    if (threadIdx.x == 0 && bump) st->step += 1u;
}

__global__ void __launch_bounds__(kScanThreads) scan_kernel(uint32_t* __restrict__ count,
                                                            uint32_t* __restrict__ start,
                                                            unsigned long long* status, InstDyn* dyn,
                                                            const InstDev* inst, int n_inst, DevState* st,
                                                            Geo geo, int bump) {
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_warp[kScanThreads / 32];
    __shared__ uint32_t s_prefix;
    if (threadIdx.x == 0) s_tile = (uint32_t)atomicAdd(&status[0], 1ull);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile == 0) step_bookkeeping(dyn, inst, n_inst, st, geo, bump);
    // the test of the bounded wait lowers the cap and holds back one tile's status
    const uint32_t cap = st->spin_cap ? st->spin_cap : kSpinCap;
    const bool publish = st->hold_tile1 != tile + 1u;

    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const size_t base = (size_t)tile * kScanTile + (size_t)threadIdx.x * kScanItems;
    uint32_t it[kScanItems];
    const uint4* src = reinterpret_cast<const uint4*>(count + base);
#pragma unroll
    for (int q = 0; q < kScanItems / 4; ++q) {
        const uint4 v = src[q];
        it[4 * q + 0] = v.x; it[4 * q + 1] = v.y; it[4 * q + 2] = v.z; it[4 * q + 3] = v.w;
    }
    uint32_t total = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const uint32_t c = it[i];
        it[i] = total;          // exclusive within the thread
        total += c;
    }
    // block-wide exclusive scan of the thread totals
    uint32_t inc = total;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if ((int)lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kScanThreads / 32 ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if ((int)lane >= o) wi += y;
        }
        const uint32_t aggregate = __shfl_sync(0xffffffffu, wi, kScanThreads / 32 - 1);
        if (lane < kScanThreads / 32) s_warp[lane] = wi - w;  // exclusive warp offsets
        // decoupled look-back
        uint32_t prefix = 0;
        if (tile == 0) {
            if (lane == 0 && publish) atomicExch(&status[1], kFlagInc | (unsigned long long)aggregate);
        } else {
            if (lane == 0 && publish) atomicExch(&status[1 + tile], kFlagAgg | (unsigned long long)aggregate);
            long long pred = (long long)tile - 1;
            bool done = false;
            while (!done) {
                const long long t = pred - (long long)lane;
                unsigned long long sv = kFlagInc;
                if (t >= 0) {
                    uint32_t spins = 0;
                    for (;;) {
                        sv = load_status(&status[1 + t]);
                        if ((sv >> 32) != 0ull) break;
                        if (++spins > cap) {
                            atomicOr(&st->error, kErrScanTimeout);
                            sv = kFlagInc;
                            break;
                        }
                        if (spins > 16) __nanosleep(64);
                    }
                }
                const uint32_t flag = (uint32_t)(sv >> 32);
                const uint32_t val = (uint32_t)sv;
                const unsigned incl = __ballot_sync(0xffffffffu, flag == 2u);
                uint32_t contrib;
                if (incl) {
                    const int first = __ffs(incl) - 1;
                    contrib = ((int)lane <= first) ? val : 0u;
                    done = true;
                } else {
                    contrib = val;
                    pred -= 32;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
                prefix += contrib;
            }
            if (lane == 0 && publish)
                atomicExch(&status[1 + tile], kFlagInc | (unsigned long long)(prefix + aggregate));
        }
        if (lane == 0) s_prefix = prefix;
    }
    __syncthreads();
    const uint32_t off = s_prefix + s_warp[warp] + (inc - total);
    uint4* dst = reinterpret_cast<uint4*>(start + base);
    uint4* clr = reinterpret_cast<uint4*>(count + base);
#pragma unroll
    for (int q = 0; q < kScanItems / 4; ++q) {
        dst[q] = make_uint4(off + it[4 * q], off + it[4 * q + 1], off + it[4 * q + 2], off + it[4 * q + 3]);
        clr[q] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// Fixed-point sum -> binary64 (exact below 2^53, correctly rounded above).
__device__ __forceinline__ double unfix(unsigned long long a, int e) { return ldexp((double)(long long)a, -e); }

// Derived per-c-bin moments (Eqs. vel_b, stress, 18, 19 with the readings
// u = Sum v / N, v_rms^2 = <|v - u|^2>, T = v_rms^2 / 3, p = n T + virial),
// and the per-instance integer totals of the fixed-point sums (exact, so the
// order of the atomics does not matter): a warp whose bins belong to one
// instance reduces with shuffles and adds once.
__global__ void __launch_bounds__(256) finalize_bins_kernel(const InstDev* __restrict__ inst,
                                                            const InstDyn* __restrict__ dyn, Geo geo,
                                                            const unsigned long long* __restrict__ acc,
                                                            double* __restrict__ mom, unsigned long long* gacc,
                                                            int64_t n_bins, int64_t bins_per_inst) {
    const int64_t bidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = bidx < n_bins;
    const int i = valid ? (int)(bidx / bins_per_inst) : 0;
    unsigned long long t[7] = {0, 0, 0, 0, 0, 0, 0};
    if (valid) {
        const InstDyn& D = dyn[i];
        const unsigned long long* a = acc + bidx * kAccFields;
        unsigned long long ai[kAccFields];
        for (int k = 0; k < kAccFields; ++k) ai[k] = a[k];
        t[0] = ai[0];
        t[1] = ai[4] + ai[5] + ai[6];
        t[2] = ai[1];
        t[3] = ai[2];
        t[4] = ai[3];
        t[5] = ai[7];
        t[6] = ai[8];
        double* o = mom + bidx * kMomStride;
        double r[8];
        r[0] = (double)(long long)ai[0];
        for (int k = 1; k <= 3; ++k) r[k] = unfix(ai[k], D.mom_e[0]);
        for (int k = 4; k <= 6; ++k) r[k] = unfix(ai[k], D.mom_e[1]);
        r[7] = unfix(ai[7], D.mom_e[2]);
        for (int k = 0; k < 8; ++k) o[k] = r[k];
        double Vc = 1.0;
        for (int d = 0; d < geo.dim; ++d) Vc *= geo.L[d] / (double)geo.n[d];
        const double N = r[0];
        const double svr = unfix(ai[9], D.mom_e[0]);
        o[16] = svr;
        o[17] = N > 0.0 ? svr / N : 0.0;   // Eq. vel_r
        if (N <= 0.0) {
            for (int k = 8; k < 16; ++k) o[k] = 0.0;
        } else {
            const double dt = D.dt_prev;   // the step whose collisions W sums
            const double ux = r[1] / N, uy = r[2] / N, uz = r[3] / N;
            const double c2 = (r[4] + r[5] + r[6]) / N - (ux * ux + uy * uy + uz * uz);
            const double T = c2 / (geo.vdim == 2 ? 2.0 : 3.0);   // f velocity degrees of freedom
            const double nd = N / Vc;
            const double pkin = nd * T;
            const double pvir = r[7] / (2.0 * geo.dim * Vc * dt);
            o[8] = nd; o[9] = ux; o[10] = uy; o[11] = uz;
            o[12] = T; o[13] = pkin; o[14] = pvir; o[15] = pkin + pvir;
        }
    }
    const int i0 = __shfl_sync(0xffffffffu, i, 0);
    if (__all_sync(0xffffffffu, !valid || i == i0)) {
#pragma unroll
        for (int k = 0; k < 7; ++k) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t[k] += __shfl_xor_sync(0xffffffffu, t[k], o);
        }
        if ((threadIdx.x & 31u) == 0 && __shfl_sync(0xffffffffu, (int)valid, 0))
            for (int k = 0; k < 7; ++k)
                if (t[k]) atomicAdd(gacc + (size_t)i0 * 8 + k, t[k]);
    } else if (valid) {
        for (int k = 0; k < 7; ++k)
            if (t[k]) atomicAdd(gacc + (size_t)i * 8 + k, t[k]);
    }
}

// Per-instance totals (N, energy, momentum, virial, pairs) from the integer
// totals, converted once; the totals are cleared for the next reduction.
__global__ void finalize_glob_kernel(const InstDyn* __restrict__ dyn, unsigned long long* gacc,
                                     double* __restrict__ glob, int n_inst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_inst) return;
    const InstDyn& D = dyn[i];
    unsigned long long* t = gacc + (size_t)i * 8;
    double* g = glob + (int64_t)i * 8;
    g[0] = (double)(long long)t[0];
    g[1] = 0.5 * unfix(t[1], D.mom_e[1]);
    g[2] = unfix(t[2], D.mom_e[0]);
    g[3] = unfix(t[3], D.mom_e[0]);
    g[4] = unfix(t[4], D.mom_e[0]);
    g[5] = unfix(t[5], D.mom_e[2]);
    g[6] = 0.5 * (double)(long long)t[6];  // collided particles / 2 = pairs
    g[7] = 0.0;
    for (int k = 0; k < 8; ++k) t[k] = 0ull;
}

}  // namespace

cudaError_t launch_scan(uint32_t* count, uint32_t* start, uint32_t n_keys, uint32_t n_tiles,
                        unsigned long long* status, InstDyn* dyn, const InstDev* inst, int n_inst,
                        DevState* st, Geo geo, int bump_step, cudaStream_t s) {
    (void)n_keys;
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(unsigned long long) * (1 + (size_t)n_tiles), s);
    if (e != cudaSuccess) return e;
    scan_kernel<<<n_tiles, kScanThreads, 0, s>>>(count, start, status, dyn, inst, n_inst, st, geo, bump_step);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const InstDev* inst, const InstDyn* dyn, int n_inst, Geo geo,
                            const unsigned long long* acc, double* mom, double* glob, unsigned long long* gacc,
                            int64_t n_bins, cudaStream_t s) {
    if (n_bins == 0 || n_inst == 0) return cudaSuccess;
    const int64_t per = n_bins / n_inst;
    finalize_bins_kernel<<<(unsigned)((n_bins + 255) / 256), 256, 0, s>>>(inst, dyn, geo, acc, mom, gacc, n_bins,
                                                                         per);
    finalize_glob_kernel<<<(n_inst + 127) / 128, 128, 0, s>>>(dyn, gacc, glob, n_inst);
    return cudaGetLastError();
}

}  // namespace kmc
