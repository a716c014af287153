// kmc_kernels.cuh -- sm_103a kernels of one kinetic Monte Carlo step, templated on
// the state precision T (float or double) and the position dimension DIM.
//
// Step structure (Sagert et al., Sect. "Simulation setup" and Fig. 2):
//   search  : closest PoCA candidate per particle over its c-bin neighbourhood
//             (per particle, or per c-bin block on unsubdivided grids)
//   move    : unambiguous pairs, CM scattering, split free flight, walls,
//             next search key + histogram
//   scan    : exclusive scan of the key histogram (kmc_scan.cu)
//   scatter : counting-sort scatter into search-key order
//   moments : per-c-bin sums of the new state (finalised in kmc_scan.cu)
//
// Layout: SoA of 16-byte (binary32) or 32-byte (binary64) vectors,
//   pos = (x, y, z, tag bits), vel = (vx, vy, vz, W),
// tag = (instance << id_bits) | instance-local id, W = collisional virial of the
// particle's last step (+inf when it did not collide, -inf once absorbed),
// sorted by search key = key_base + (gx * My + gy) * Mz + gz where g is the
// search cell (a c-bin subdivided s_d times per dimension, x slowest).
#pragma once

#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "kmc_internal.h"

namespace kmc {

// ---------------------------------------------------------------- arithmetic
// Decision arithmetic uses explicitly rounded operations so the compiler cannot
// contract or reorder them; the fused multiply-adds are the explicit fma calls.
template <typename T>
struct R;
template <>
struct R<float> {
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
    static __device__ __forceinline__ float sqrt_(float a) { return sqrtf(a); }
    static __device__ __forceinline__ uint32_t bits(float a) { return __float_as_uint(a); }
    static __device__ __forceinline__ float from_bits(uint32_t u) { return __uint_as_float(u); }
    static __device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }
    static __device__ __forceinline__ float qnan() { return __int_as_float(0x7fc00000); }
};
template <>
struct R<double> {
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ double sqrt_(double a) { return sqrt(a); }
    static __device__ __forceinline__ uint32_t bits(double a) {
        return (uint32_t)(unsigned long long)__double_as_longlong(a);
    }
    static __device__ __forceinline__ double from_bits(uint32_t u) {
        return __longlong_as_double((long long)(unsigned long long)u);
    }
    static __device__ __forceinline__ double inf() { return __longlong_as_double(0x7ff0000000000000LL); }
    static __device__ __forceinline__ double qnan() { return __longlong_as_double(0x7ff8000000000000LL); }
};

// Timestep of the current step (constant unless adaptive; set on the device by
// the step bookkeeping) and squared contact distance, in the state precision
// (binary32 copies are rounded once from binary64, as the oracle rounds them).
__device__ __forceinline__ float step_dt(const InstDyn& D, float) { return D.dtf; }
__device__ __forceinline__ double step_dt(const InstDyn& D, double) { return D.dt; }
__device__ __forceinline__ float inst_R2(const InstDev& I, float) { return I.R2f; }
__device__ __forceinline__ double inst_R2(const InstDev& I, double) { return I.R2; }

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32 multiplies with
// the published multipliers; the key advances by the Weyl increments.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Uniform deviates in (0, 1) with an odd mantissa: binary32 from one word,
// binary64 from two.
template <typename T>
__device__ __forceinline__ void uniforms(uint4 x, T& u1, T& u2);
template <>
__device__ __forceinline__ void uniforms<float>(uint4 x, float& u1, float& u2) {
    u1 = (float)((x.x >> 8) | 1u) * 0x1p-24f;
    u2 = (float)((x.z >> 8) | 1u) * 0x1p-24f;
}
template <>
__device__ __forceinline__ void uniforms<double>(uint4 x, double& u1, double& u2) {
    const unsigned long long m1 = ((unsigned long long)x.x << 20) | (x.y >> 12);
    const unsigned long long m2 = ((unsigned long long)x.z << 20) | (x.w >> 12);
    u1 = (double)(2ull * m1 + 1ull) * 0x1p-53;
    u2 = (double)(2ull * m2 + 1ull) * 0x1p-53;
}

__device__ __forceinline__ void sincos_2pi(float u, float* s, float* c) { sincospif(2.0f * u, s, c); }
__device__ __forceinline__ void sincos_2pi(double u, double* s, double* c) { sincospi(2.0 * u, s, c); }

// ------------------------------------------------------------- geometry
// Per-dimension constants in the state precision.  For walled dimensions the
// half length is +inf so the minimum-image shift never fires.
template <typename T>
struct GeoT {
    T lo[3], hi[3], inv[3], L[3], hL[3], rc[3];
    int n[3];
    bool wall[3];     // no periodic wrap: reflective or absorbing
    bool absorb[3];   // absorbing: a particle that ends a step outside is removed
    int vdim;
    __device__ __forceinline__ void load(const Geo& g) {
        vdim = g.vdim;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            lo[d] = (T)g.lo[d];
            hi[d] = (T)g.hi[d];
            inv[d] = (T)g.inv_dx[d];
            L[d] = (T)g.L[d];
            wall[d] = g.bc[d] != 0;
            absorb[d] = g.bc[d] == 2;
            hL[d] = wall[d] ? R<T>::inf() : (T)0.5 * L[d];
            rc[d] = (T)g.rc[d];
            n[d] = g.n[d];
        }
    }
};

// c-bin index c = floor((x - lo) * n / (hi - lo)) clamped to [0, n-1], and the
// search cell g = c * s + floor(frac * s) inside it.
template <typename T>
__device__ __forceinline__ void cell_and_search(T x, T lo, T inv, int n, int s, int& c, int& g) {
    const T t = R<T>::mul(R<T>::sub(x, lo), inv);
    int ci;
    if (t < (T)0) ci = 0;
    else if (t >= (T)n) ci = n - 1;
    else ci = (int)t;
    c = ci;
    if (s == 1) { g = ci; return; }
    const T fs = R<T>::mul(R<T>::sub(t, (T)ci), (T)s);
    int si;
    if (fs < (T)0) si = 0;
    else if (fs >= (T)s) si = s - 1;
    else si = (int)fs;
    g = ci * s + si;
}

template <typename T>
__device__ __forceinline__ T min_image(T x, T hL, T L) {
    if (x > hL) return R<T>::sub(x, L);
    if (x < -hL) return R<T>::add(x, L);
    return x;
}

// Keys of a position: search key (global) and c-bin (global row).
template <typename T, int DIM>
__device__ __forceinline__ void keys_of(const GeoT<T>& G, const InstDev& I, const T x[3],
                                        uint32_t& skey, uint32_t& bin) {
    int c[3] = {0, 0, 0}, g[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < DIM; ++d) cell_and_search<T>(x[d], G.lo[d], G.inv[d], G.n[d], I.s[d], c[d], g[d]);
    if (DIM == 3) {
        skey = I.key_base + ((uint32_t)g[0] * (uint32_t)I.M[1] + (uint32_t)g[1]) * (uint32_t)I.M[2] + (uint32_t)g[2];
        bin = I.bin_base + (uint32_t)c[0] + (uint32_t)G.n[0] * ((uint32_t)c[1] + (uint32_t)G.n[1] * (uint32_t)c[2]);
    } else {
        skey = I.key_base + (uint32_t)g[0] * (uint32_t)I.M[1] + (uint32_t)g[1];
        bin = I.bin_base + (uint32_t)c[0] + (uint32_t)G.n[0] * (uint32_t)c[1];
    }
}

// Instance of a global particle index (instances are consecutive blocks).
__device__ __forceinline__ int instance_of(const InstDev* inst, int n_inst, int64_t gidx) {
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (inst[mid].p_off <= gidx) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Instance and local id of a particle tag.
template <typename T>
__device__ __forceinline__ int tag_inst(const Bufs<T>& b, uint32_t tag) {
    return b.id_bits >= 32u ? 0 : (int)(tag >> b.id_bits);
}
template <typename T>
__device__ __forceinline__ uint32_t tag_id(const Bufs<T>& b, uint32_t tag) {
    return tag & b.id_mask;
}

// ------------------------------------------------------------ warp helpers
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Histogram increment aggregated over lanes with the same key; returns the
// lane's rank within its key (the counting-sort slot).
__device__ __forceinline__ uint32_t aggregated_increment(uint32_t* count, uint32_t key, unsigned active) {
    const unsigned peers = __match_any_sync(active, key);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if ((int)lane_id() == leader) base = atomicAdd(count + key, (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    const unsigned lt = (1u << lane_id()) - 1u;
    return base + (uint32_t)__popc(peers & lt);
}

// Largest |v|^2 per instance: a warp maximum on the bit patterns (non-negative
// floats order like their bits, so the reduction is integer work), then one
// atomicMax per warp on the binary64 bits, skipped when it cannot raise the
// stored value.  A warp that straddles two instances falls back to one atomic
// per lane.
__device__ __forceinline__ unsigned long long vmax_bits(float v2) {
    return (unsigned long long)__double_as_longlong((double)v2);
}
__device__ __forceinline__ unsigned long long vmax_bits(double v2) {
    return (unsigned long long)__double_as_longlong(v2);
}
__device__ __forceinline__ unsigned long long warp_max_bits(float v2, bool valid) {
    const unsigned m = __reduce_max_sync(kFull, valid ? __float_as_uint(v2) : 0u);
    return vmax_bits(__uint_as_float(m));
}
__device__ __forceinline__ unsigned long long warp_max_bits(double v2, bool valid) {
    unsigned long long m = valid ? (unsigned long long)__double_as_longlong(v2) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(kFull, m, o);
        m = y > m ? y : m;
    }
    return m;
}

// A particle absorbed by a wall carries vel.w = -inf (W is finite or +inf otherwise).
template <typename T>
__device__ __forceinline__ bool absorbed(T w) {
    return w == -R<T>::inf();
}

// |v|^2 in a fixed operation order (the adaptive timestep depends on its bits)
template <typename T>
__device__ __forceinline__ T speed2(T vx, T vy, T vz) {
    return R<T>::fma(vz, vz, R<T>::fma(vy, vy, R<T>::mul(vx, vx)));
}

template <typename T>
__device__ __forceinline__ void warp_vmax(InstDyn* dyn, bool valid, int inst, T v2) {
    const int inst0 = __shfl_sync(kFull, inst, 0);
    if (__all_sync(kFull, !valid || inst == inst0)) {
        const unsigned long long m = warp_max_bits(v2, valid);
        if (lane_id() == 0) {
            unsigned long long* dst = &dyn[inst0].vmax2_next;
            if (m > *((volatile unsigned long long*)dst)) atomicMax(dst, m);
        }
    } else if (valid) {
        atomicMax(&dyn[inst].vmax2_next, vmax_bits(v2));
    }
}

// Moment sums per c-bin in fixed point.  Every particle's contribution (v,
// v^2, W) is rounded once to an integer multiple of 2^-e, with e chosen per
// instance and field so that the sum over all of the instance's particles
// stays below 2^62 in magnitude (step bookkeeping in kmc_scan.cu); the sums
// are then exact 64-bit integer sums, so they do not depend on the order in
// which particles are visited or on how they are grouped into threads, warps
// and blocks: reruns, batched and plain runs give the same bits.  Aggregation
// has three levels so that few atomics reach any one bin: lanes with the same
// bin are reduced with warp shuffles; each warp group's totals go to a
// shared-memory slot list; after a block barrier the first slot of every
// distinct bin adds up its duplicates and issues the global atomics.  All
// threads of the block must call this; a lane contributes its partial sums
// (v, v^2, W, v.r_hat), particle count and collided count.
constexpr int kMomSums = 8;
// accumulator index of partial sum k: Sum v (3), Sum v^2 (3), Sum W, then Sum v.r_hat after the collided count
__device__ __forceinline__ int acc_field(int k) { return k < 7 ? 1 + k : 9; }

struct MomentSlots {
    uint32_t bin[kThreads];
    long long f[kMomSums][kThreads];
    int cnt[kThreads];
    int coll[kThreads];
    int n;
};

__device__ __forceinline__ float pow2_of(int e, float) { return __int_as_float((127 + e) << 23); }
__device__ __forceinline__ double pow2_of(int e, double) {
    return __longlong_as_double((long long)(1023 + e) << 52);
}
// x 2^e rounded to the nearest integer (2^e scales exactly; |x 2^e| < 2^62 by the choice of e)
__device__ __forceinline__ long long fixed_of(float x, float scale) { return __float2ll_rn(x * scale); }
__device__ __forceinline__ long long fixed_of(double x, double scale) { return __double2ll_rn(x * scale); }

__device__ __forceinline__ void block_moment_partials(MomentSlots& S, unsigned long long* acc, bool valid,
                                                      uint32_t bin, const long long fl[kMomSums], int cnt_l,
                                                      int coll_l) {
    // runs of lanes with the same bin (a lane without particles is a run of its
    // own): a segmented sum over the warp in five shuffle steps, whatever the
    // number of runs; the last lane of each run adds a slot
    const unsigned lane = lane_id();
    const uint32_t key = valid ? bin : 0xffffffffu;
    const uint32_t prev = __shfl_up_sync(kFull, key, 1);
    const unsigned heads = __ballot_sync(kFull, lane == 0 || !valid || key != prev);
    const int seg = __popc(heads & (0xffffffffu >> (31 - lane)));   // run index of this lane
    long long f[kMomSums];
#pragma unroll
    for (int k = 0; k < kMomSums; ++k) f[k] = valid ? fl[k] : 0ll;
    int c = valid ? cnt_l : 0, cc = valid ? coll_l : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int so = __shfl_up_sync(kFull, seg, o);
        const bool add = lane >= (unsigned)o && so == seg;
#pragma unroll
        for (int k = 0; k < kMomSums; ++k) {
            const long long y = __shfl_up_sync(kFull, f[k], o);
            if (add) f[k] += y;
        }
        const int yc = __shfl_up_sync(kFull, c, o), ycc = __shfl_up_sync(kFull, cc, o);
        if (add) {
            c += yc;
            cc += ycc;
        }
    }
    const int seg_next = __shfl_down_sync(kFull, seg, 1);
    if (valid && (lane == 31 || seg_next != seg)) {
        const int slot = atomicAdd(&S.n, 1);
        S.bin[slot] = bin;
#pragma unroll
        for (int k = 0; k < kMomSums; ++k) S.f[k][slot] = f[k];
        S.cnt[slot] = c;
        S.coll[slot] = cc;
    }
    __syncthreads();
    const int ns = S.n;
    for (int t = threadIdx.x; t < ns; t += blockDim.x) {
        const uint32_t mb = S.bin[t];
        bool first = true;
        for (int u = 0; u < t; ++u)
            if (S.bin[u] == mb) { first = false; break; }
        if (!first) continue;
        long long tot[kMomSums] = {0, 0, 0, 0, 0, 0, 0, 0};
        long long c = 0, cc = 0;
        for (int u = t; u < ns; ++u) {
            if (S.bin[u] != mb) continue;
#pragma unroll
            for (int k = 0; k < kMomSums; ++k) tot[k] += S.f[k][u];
            c += S.cnt[u];
            cc += S.coll[u];
        }
        unsigned long long* a = acc + (size_t)mb * kAccFields;
        atomicAdd(a + 0, (unsigned long long)c);
#pragma unroll
        for (int k = 0; k < kMomSums; ++k)
            if (tot[k]) atomicAdd(a + acc_field(k), (unsigned long long)tot[k]);
        if (cc) atomicAdd(a + 8, (unsigned long long)cc);
    }
}

// --------------------------------------------------------------- kernels

// Pack n x 3 input arrays into (pos, id) / (vel, instance) vectors of B and
// count particles that are non-finite or outside the box.
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) pack_kernel(Bufs<T> b, const T* __restrict__ pos3,
                                                        const T* __restrict__ vel3, uint32_t* bad) {
    using V = typename Vec4<T>::type;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= b.n) return;
    const int inst = instance_of(b.inst, b.n_inst, p);
    const uint32_t id = (uint32_t)(p - b.inst[inst].p_off);
    T x[3], v[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        x[d] = pos3[3 * p + d];
        v[d] = vel3[3 * p + d];
    }
    bool any_absorb = false;
#pragma unroll
    for (int d = 0; d < DIM; ++d) any_absorb = any_absorb || b.geo.bc[d] == 2;
    // a particle already absorbed (a state read back from an absorbing run) has a NaN position
    const bool gone = any_absorb && isnan(x[0]);
    bool ok = true;
    if (!gone) {
#pragma unroll
        for (int d = 0; d < 3; ++d) ok = ok && isfinite(x[d]) && isfinite(v[d]);
        if (b.geo.vdim == 2) ok = ok && v[2] == (T)0;   // 2-D velocities: no z component
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const T lo = (T)b.geo.lo[d], hi = (T)b.geo.hi[d];
            if (b.geo.bc[d] != 0) ok = ok && x[d] >= lo && x[d] <= hi;
            else ok = ok && x[d] >= lo && x[d] < hi;
        }
    }
    if (!ok) atomicAdd(bad, 1u);
    V P, Q;
    const uint32_t tag = (b.id_bits >= 32u ? 0u : ((uint32_t)inst << b.id_bits)) | id;
    P.x = gone ? (T)0 : x[0]; P.y = gone ? (T)0 : x[1]; P.z = gone ? (T)0 : x[2]; P.w = R<T>::from_bits(tag);
    Q.x = gone ? (T)0 : v[0]; Q.y = gone ? (T)0 : v[1]; Q.z = gone ? (T)0 : v[2];
    Q.w = gone ? -R<T>::inf() : R<T>::inf();
    b.posB[p] = P;
    b.velB[p] = Q;
}

// Keys, counting-sort slots, histogram and |v|max of the packed state in B
// (used after packing: at init and when the state is replaced).
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) bin_kernel(Bufs<T> b) {
    using V = typename Vec4<T>::type;
    __shared__ GeoT<T> G;
    if (threadIdx.x == 0) G.load(b.geo);
    __syncthreads();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = p < b.n;
    V P = {}, Q = {};
    int inst = 0;
    if (valid) {
        P = b.posB[p];
        Q = b.velB[p];
        inst = tag_inst(b, R<T>::bits(P.w));
    }
    const InstDev I = b.inst[inst];
    const T x[3] = {P.x, P.y, P.z};
    uint32_t skey = 0, bin = 0;
    keys_of<T, DIM>(G, I, x, skey, bin);
    const bool gone = absorbed(Q.w);
    if (gone) skey = b.n_keys;   // the key after every cell: no search window reaches it
    const unsigned active = __ballot_sync(kFull, valid);
    if (valid) {
        const uint32_t slot = aggregated_increment(b.count, skey, active);
        b.key[p] = skey;
        b.slot[p] = slot;
        b.tagB[p] = R<T>::bits(P.w);
    }
    warp_vmax<T>(b.dyn, valid && !gone, inst, speed2<T>(Q.x, Q.y, Q.z));
}

// The PoCA acceptance test of the ordered pair (i, j) and its closest-approach
// distance, in the operation order shared with the CPU oracle:
//   a = r.v, b = |v|^2, r2 = |r|^2 (first product rounded, then fused adds),
//   chi < 0  <=>  a < 0 and fma(b, dt, a) > 0           (Eq. c_value)
//   disc = fma(a, a, -(b * (r2 - R^2))) >= 0             (Eq. collision_time2)
//   d2 = r2 - (a * a) / b                                (criterion 3)
template <typename T, int DIM>
__device__ __forceinline__ bool poca_test(const GeoT<T>& G, const T xi[3], const T vi[3], const T xj[3],
                                          const T vj[3], T dt, T R2, T& d2) {
    T dr[3], dv[3];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        dr[d] = min_image<T>(R<T>::sub(xi[d], xj[d]), G.hL[d], G.L[d]);
        dv[d] = R<T>::sub(vi[d], vj[d]);
    }
    T a = R<T>::mul(dr[0], dv[0]);
    a = R<T>::fma(dr[1], dv[1], a);
    T bb = R<T>::mul(dv[0], dv[0]);
    bb = R<T>::fma(dv[1], dv[1], bb);
    if (DIM == 3) {
        a = R<T>::fma(dr[2], dv[2], a);
        bb = R<T>::fma(dv[2], dv[2], bb);
    }
    if (!(bb > (T)0 && a < (T)0 && R<T>::fma(bb, dt, a) > (T)0)) return false;
    T r2 = R<T>::mul(dr[0], dr[0]);
    r2 = R<T>::fma(dr[1], dr[1], r2);
    if (DIM == 3) r2 = R<T>::fma(dr[2], dr[2], r2);
    const T disc = R<T>::fma(a, a, -R<T>::mul(bb, R<T>::sub(r2, R2)));
    if (!(disc >= (T)0)) return false;
    d2 = R<T>::sub(r2, R<T>::div(R<T>::mul(a, a), bb));
    return true;
}

// Candidate data through the read-only path.
__device__ __forceinline__ float4 ldg_vec(const float4* p) { return __ldg(p); }
__device__ __forceinline__ dvec4 ldg_vec(const dvec4* p) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 c = __ldg(reinterpret_cast<const double2*>(p) + 1);
    dvec4 r;
    r.x = a.x; r.y = a.y; r.z = c.x; r.w = c.y;
    return r;
}

// Order-preserving 32-bit image of a binary32 distance (-0 folded into +0):
// unsigned comparison of the images is the floating-point comparison.
__device__ __forceinline__ uint32_t ordered_bits(float d2) {
    const uint32_t u = __float_as_uint(d2 + 0.0f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Partner key of a particle: the tag of its closest candidate in the low 32
// bits; in binary32 the high 32 bits hold the ordered image of d2, so that
// the minimum key is the closest candidate with ties to the lower id (tags of
// one instance order as their ids); the symmetric search combines keys with
// atomicMin.  Binary64 searches store the key of a full window directly and
// leave the high bits zero.
template <typename T>
__device__ __forceinline__ unsigned long long partner_key(T d2, uint32_t tag) {
    if (sizeof(T) == 4) return ((unsigned long long)ordered_bits((float)d2) << 32) | (unsigned long long)tag;
    return (unsigned long long)tag;
}

// The acceptance test with the separation r_i - r_j formed as
// (x_i - x_j) + shift_d: the shift is the periodic image of the candidate's
// row (0, +L or -L) when MINIMG is false, and the per-candidate minimum image
// of every periodic dimension when MINIMG is true.  Both give the same bits as
// the oracle's minimum image: inside a window narrower than half the box the
// image of a row is the same for all its candidates.
template <typename T, int DIM, bool MINIMG, bool SHIFT = true>
__device__ __forceinline__ bool poca_test_sh(const GeoT<T>& G, const T xi[3], const T vi[3], const T xj[3],
                                             const T vj[3], const T sh[3], T dt, T R2, T& d2) {
    T dr[3], dv[3];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        const T x = R<T>::sub(xi[d], xj[d]);
        // SHIFT = false: a row without periodic image (x + 0 = x)
        dr[d] = MINIMG ? min_image<T>(x, G.hL[d], G.L[d]) : (SHIFT ? R<T>::add(x, sh[d]) : x);
        dv[d] = R<T>::sub(vi[d], vj[d]);
    }
    T a = R<T>::mul(dr[0], dv[0]);
    a = R<T>::fma(dr[1], dv[1], a);
    T bb = R<T>::mul(dv[0], dv[0]);
    bb = R<T>::fma(dv[1], dv[1], bb);
    if (DIM == 3) {
        a = R<T>::fma(dr[2], dv[2], a);
        bb = R<T>::fma(dv[2], dv[2], bb);
    }
    if (!(bb > (T)0 && a < (T)0 && R<T>::fma(bb, dt, a) > (T)0)) return false;
    T r2 = R<T>::mul(dr[0], dr[0]);
    r2 = R<T>::fma(dr[1], dr[1], r2);
    if (DIM == 3) r2 = R<T>::fma(dr[2], dr[2], r2);
    const T disc = R<T>::fma(a, a, -R<T>::mul(bb, R<T>::sub(r2, R2)));
    if (!(disc >= (T)0)) return false;
    d2 = R<T>::sub(r2, R<T>::div(R<T>::mul(a, a), bb));
    return true;
}

// Search window of one dimension in search-cell coordinates: within k cells of
// g and inside the c-bins c-1 .. c+1; cut at walls.  A periodic window is kept
// unwrapped (t in (-M, 2M); image shift +L below 0, -L above M-1).  When every
// cell of the window lies less than half a box (minus half a cell) from the
// particle's cell, all candidates of a row share one image and the shift is
// exact; otherwise (`amb`) the candidates take the per-candidate minimum image,
// and a window as wide as the row becomes the row itself.
struct Win {
    int lo, hi;
    bool amb;   // per-candidate minimum image needed
};
__device__ __forceinline__ Win window_1d(int g, int c, int s, int M, int k, bool wall) {
    Win w;
    w.lo = max(g - k, (c - 1) * s);
    w.hi = min(g + k, (c + 2) * s - 1);
    w.amb = false;
    if (wall) {
        w.lo = max(w.lo, 0);
        w.hi = min(w.hi, M - 1);
    } else if (w.hi - w.lo + 1 >= M) {
        w.lo = 0;
        w.hi = M - 1;
        w.amb = true;
    } else {
        const int m = max(g - w.lo, w.hi - g) + 1;
        w.amb = 2 * m + 1 > M;
    }
    return w;
}

// Test the candidates [q, qe) of one range and keep the closest (smaller d2,
// ties to the lower id).  The next candidate is loaded before the current one
// is tested.
template <typename T, int DIM, bool MINIMG, bool SYM = false>
__device__ __forceinline__ void scan_range(const Bufs<T>& b, const GeoT<T>& G, int32_t q, int32_t qe,
                                           const T sh[3], const T xi[3], const T vi[3], T dt, T R2, T& bd,
                                           uint32_t& bid, int32_t& bq, int32_t self = 0, uint32_t tag = 0) {
    using V = typename Vec4<T>::type;
    if (SYM) q = max(q, self + 1);
    if (q >= qe) return;
    V Pn = ldg_vec(b.posA + q);
    V Qn = ldg_vec(b.velA + q);
    for (; q < qe; ++q) {
        const V Pj = Pn, Qj = Qn;
        if (q + 1 < qe) {
            Pn = ldg_vec(b.posA + q + 1);
            Qn = ldg_vec(b.velA + q + 1);
        }
        const T xj[3] = {Pj.x, Pj.y, Pj.z};
        const T vj[3] = {Qj.x, Qj.y, Qj.z};
        T d2;
        // the particle itself has v_rel = 0 and fails b > 0
        if (poca_test_sh<T, DIM, MINIMG>(G, xi, vi, xj, vj, sh, dt, R2, d2)) {
            const uint32_t idj = R<T>::bits(Pj.w);
            if (d2 < bd || (d2 == bd && idj < bid)) {
                bd = d2;
                bid = idj;
                bq = q;
            }
            if (SYM) atomicMin(&b.bkey[q], partner_key<T>(d2, tag));
        }
    }
}

// Unwrapped window index -> (cell, image shift) of a periodic or walled dimension.
template <typename T>
__device__ __forceinline__ int unwrap(int t, int M, T L, T& shift) {
    shift = (T)0;
    if (t < 0) { shift = L; return t + M; }
    if (t >= M) { shift = -L; return t - M; }
    return t;
}

// Every candidate range of one particle.  The last position dimension is the
// fastest of the key, so a window is a set of rows (x, or x and y) each with
// one or two contiguous key ranges.  Common case (at most 3 cells per row
// dimension, one range per row): all row ranges are fetched first so their
// loads overlap, then the rows are scanned in turn.  Otherwise rows are
// visited one at a time.
// Walk the non-empty row ranges of one particle as one sequence: the ranges
// sit in shared memory (`rng`, one slot per row, stride kThreads), `mask`
// marks the non-empty rows, and the next candidate is loaded while the current
// one is tested.  A lane with short rows goes on to its next row instead of
// idling until the longest row of its warp is done.  `code` holds the periodic
// image of every row: two bits per x row (bits 0-5) and per y row (bits 6-11),
// 1 = +L, 2 = -L; `sf` is the image of the fast dimension.
template <typename T>
__device__ __forceinline__ T image_of(uint32_t c, T L) {
    return c == 1u ? L : (c == 2u ? -L : (T)0);
}

template <typename T, int DIM, bool MINIMG, bool SYM, bool SHIFT = true>
__device__ __forceinline__ void walk_rows(const Bufs<T>& b, const GeoT<T>& G, const int2* rng, uint32_t mask,
                                          uint32_t code, T sf, const T xi[3], const T vi[3], T dt, T R2, T& bd,
                                          uint32_t& bid, int32_t& bq, uint32_t tag) {
    using V = typename Vec4<T>::type;
    if (mask == 0u) return;
    int r = __ffs(mask) - 1;
    mask &= mask - 1u;
    int2 rg = rng[r * kThreads];
    int32_t q = rg.x, qe = rg.y;
    auto row_shift = [&](int row, T& s0, T& s1) {
        const int ix = (DIM == 3) ? row / 3 : row;
        const int iy = (DIM == 3) ? row - 3 * ix : 0;
        s0 = image_of<T>((code >> (2 * ix)) & 3u, G.L[0]);
        s1 = (DIM == 3) ? image_of<T>((code >> (6 + 2 * iy)) & 3u, G.L[1]) : sf;
    };
    T s0, s1;
    row_shift(r, s0, s1);
    V Pn = ldg_vec(b.posA + q);
    V Qn = ldg_vec(b.velA + q);
    for (;;) {
        const V Pj = Pn, Qj = Qn;
        const int32_t qj = q;
        T sh[3];
        sh[0] = s0;
        sh[1] = s1;
        sh[2] = sf;
        bool more = true;
        if (++q >= qe) {
            if (mask != 0u) {
                r = __ffs(mask) - 1;
                mask &= mask - 1u;
                rg = rng[r * kThreads];
                q = rg.x;
                qe = rg.y;
                row_shift(r, s0, s1);
            } else {
                more = false;
            }
        }
        if (more) {
            Pn = ldg_vec(b.posA + q);
            Qn = ldg_vec(b.velA + q);
        }
        const T xj[3] = {Pj.x, Pj.y, Pj.z};
        const T vj[3] = {Qj.x, Qj.y, Qj.z};
        T d2;
        // the particle itself has v_rel = 0 and fails b > 0
        if (poca_test_sh<T, DIM, MINIMG, SHIFT>(G, xi, vi, xj, vj, sh, dt, R2, d2)) {
            const uint32_t idj = R<T>::bits(Pj.w);
            if (d2 < bd || (d2 == bd && idj < bid)) {
                bd = d2;
                bid = idj;
                bq = qj;
            }
            if (SYM) atomicMin(&b.bkey[qj], partner_key<T>(d2, tag));
        }
        if (!more) break;
    }
}

template <typename T, int DIM, bool MINIMG, bool WALK = false, bool SYM = false>
__device__ __forceinline__ void scan_window(const Bufs<T>& b, const GeoT<T>& G, const InstDev& I, const Win w[3],
                                            const T xi[3], const T vi[3], T dt, T R2, T& bd, uint32_t& bid,
                                            int32_t& bq, int2* rng = nullptr, int32_t self = 0,
                                            uint32_t tag = 0, uint32_t self_key = 0) {
    constexpr int F = DIM - 1;   // fast (contiguous) dimension
    const int MF = I.M[F];
    const uint32_t nmax = (uint32_t)b.n;
    // fast-dimension parts: unwrapped window -> 1 or 2 key ranges with shifts
    int fa[2], fb[2];
    T fs[2] = {(T)0, (T)0};
    int nf = 1;
    if (w[F].lo < 0) {
        fa[0] = w[F].lo + MF; fb[0] = MF - 1; fs[0] = G.L[F];
        fa[1] = 0; fb[1] = w[F].hi;
        nf = 2;
    } else if (w[F].hi >= MF) {
        fa[0] = w[F].lo; fb[0] = MF - 1;
        fa[1] = 0; fb[1] = w[F].hi - MF; fs[1] = -G.L[F];
        nf = 2;
    } else {
        fa[0] = w[F].lo; fb[0] = w[F].hi;
    }
    const int nx = w[0].hi - w[0].lo + 1;
    const int ny = (DIM == 3) ? w[1].hi - w[1].lo + 1 : 1;
    const uint32_t My = (DIM == 3) ? (uint32_t)I.M[1] : 1u;
    const uint32_t Mf = (uint32_t)MF;
    if (nf == 1 && nx <= 3 && ny <= 3) {
        constexpr int NR = (DIM == 3) ? 9 : 3;
        int32_t q0[NR], q1[NR];
        T sx[3], sy[3];
        int gxs[3], gys[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            gxs[i] = unwrap<T>(w[0].lo + i, I.M[0], G.L[0], sx[i]);
            gys[i] = (DIM == 3) ? unwrap<T>(w[1].lo + i, I.M[1], G.L[1], sy[i]) : 0;
            if (DIM != 3) sy[i] = (T)0;
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int ix = (DIM == 3) ? r / 3 : r;
            const int iy = (DIM == 3) ? r % 3 : 0;
            q0[r] = 0;
            q1[r] = 0;
            if (ix < nx && iy < ny) {
                const uint32_t row = I.key_base + ((uint32_t)gxs[ix] * My + (uint32_t)gys[iy]) * Mf;
                // symmetric search: a row that ends before the particle's own cell
                // holds only lower positions, whose particles test this one
                if (SYM && row + (uint32_t)fb[0] < self_key) continue;
                // clamped so that a corrupted scan (flagged on the host) cannot read outside A
                q0[r] = (int32_t)min(b.start[row + (uint32_t)fa[0]], nmax);
                q1[r] = (int32_t)min(b.start[row + (uint32_t)fb[0] + 1u], nmax);
            }
        }
        if constexpr (WALK) {
            uint32_t mask = 0u, code = 0u;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                if (SYM) q0[r] = max(q0[r], self + 1);
                if (q1[r] > q0[r]) {
                    rng[r * kThreads] = make_int2(q0[r], q1[r]);
                    mask |= 1u << r;
                }
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                code |= (sx[i] > (T)0 ? 1u : (sx[i] < (T)0 ? 2u : 0u)) << (2 * i);
                if (DIM == 3) code |= (sy[i] > (T)0 ? 1u : (sy[i] < (T)0 ? 2u : 0u)) << (6 + 2 * i);
            }
            // no row of the window has a periodic image (the common case): skip the image additions
            if (code == 0u && fs[0] == (T)0)
                walk_rows<T, DIM, MINIMG, SYM, false>(b, G, rng, mask, code, fs[0], xi, vi, dt, R2, bd, bid, bq, tag);
            else
                walk_rows<T, DIM, MINIMG, SYM, true>(b, G, rng, mask, code, fs[0], xi, vi, dt, R2, bd, bid, bq, tag);
        } else {
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int ix = (DIM == 3) ? r / 3 : r;
                const int iy = (DIM == 3) ? r % 3 : 0;
                T sh[3];
                sh[0] = sx[ix];
                sh[1] = (DIM == 3) ? sy[iy] : fs[0];
                sh[2] = fs[0];
                scan_range<T, DIM, MINIMG, SYM>(b, G, q0[r], q1[r], sh, xi, vi, dt, R2, bd, bid, bq, self, tag);
            }
        }
        return;
    }
    for (int tx = w[0].lo; tx <= w[0].hi; ++tx) {
        T sx;
        const int gx = unwrap<T>(tx, I.M[0], G.L[0], sx);
        for (int ty = (DIM == 3 ? w[1].lo : 0); ty <= (DIM == 3 ? w[1].hi : 0); ++ty) {
            T sy = (T)0;
            const int gy = (DIM == 3) ? unwrap<T>(ty, I.M[1], G.L[1], sy) : 0;
            const uint32_t row = I.key_base + ((uint32_t)gx * My + (uint32_t)gy) * Mf;
            for (int part = 0; part < nf; ++part) {
                const int32_t q = (int32_t)min(b.start[row + (uint32_t)fa[part]], nmax);
                const int32_t qe = (int32_t)min(b.start[row + (uint32_t)fb[part] + 1u], nmax);
                T sh[3];
                sh[0] = sx;
                sh[1] = (DIM == 3) ? sy : fs[part];
                sh[2] = fs[part];
                scan_range<T, DIM, MINIMG, SYM>(b, G, q, qe, sh, xi, vi, dt, R2, bd, bid, bq, self, tag);
            }
        }
    }
}

// Closest candidate of every particle (criterion 3 over the 3^D c-bin
// neighbourhood, restricted to the search cells that can hold a candidate).
// One thread per particle in sorted order; candidates are read through L1.
// Binary32: the pair test is symmetric (swapping i and j negates dr and dv
// exactly, which leaves a, b, |r|^2, disc and d2 bit for bit unchanged), so
// every pair is tested once, by its lower sorted position, and the outcome
// goes to both partners: to the tester's running minimum and, with
// atomicMin, to the candidate's key.  Keys start at kNoPartner.  Binary64
// tests every candidate of a full window and stores its key.  Every particle
// records its sorted position by id (slot_of) for the move kernel.
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 4 : 2) search_kernel(Bufs<T> b) {
    using V = typename Vec4<T>::type;
    constexpr bool kSym = sizeof(T) == 4;
    __shared__ GeoT<T> G;
    __shared__ int2 rng[(DIM == 3 ? 9 : 3) * kThreads];
    if (threadIdx.x == 0) G.load(b.geo);
    __syncthreads();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= b.n) return;
    const V P = b.posA[p];
    const V Q = b.velA[p];
    const uint32_t tag = R<T>::bits(P.w);
    const int inst = tag_inst(b, tag);
    const InstDev& I = b.inst[inst];
    if (I.tiled) return;   // searched, and its slot_of recorded, by the tile search
    // sorted position by id, read by the move kernel to find a partner
    b.slot_of[I.p_off + (int64_t)tag_id(b, tag)] = (uint32_t)p;
    if (I.staged || absorbed(Q.w)) return;   // searched by the staged kernel, or gone
    const int* kk = b.dyn[inst].k;
    const T xi[3] = {P.x, P.y, P.z};
    const T vi[3] = {Q.x, Q.y, Q.z};
    const T dt = step_dt(b.dyn[inst], T()), R2 = inst_R2(I, T());
    int c[3] = {0, 0, 0}, g[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < DIM; ++d) cell_and_search<T>(xi[d], G.lo[d], G.inv[d], G.n[d], I.s[d], c[d], g[d]);
    T bd = R<T>::inf();
    uint32_t bid = 0xffffffffu;
    int32_t bq = -1;
    if (kSym && DIM == 3) {
        // Common case: c-bins not split in x, half-window 1 in y and z, and a
        // search cell at least one cell from the y and z faces.  The window is
        // then the z-ranges [g_z - 1, g_z + 1] of the rows (c_x + {-1, 0, 1},
        // g_y + {-1, 0, 1}), none with a periodic image; the symmetric search
        // keeps the own row from p + 1 on and the four rows after it.
        const int My = I.M[1], Mz = I.M[2];
        const bool x_ok = G.wall[0] || (G.n[0] >= 5 && c[0] >= 1 && c[0] <= G.n[0] - 2);
        if (I.s[0] == 1 && kk[1] == 1 && kk[2] == 1 && My >= 5 && Mz >= 5 && g[1] >= 1 && g[1] <= My - 2 &&
            g[2] >= 1 && g[2] <= Mz - 2 && x_ok) {
            const uint32_t own = I.key_base + ((uint32_t)g[0] * (uint32_t)My + (uint32_t)g[1]) * (uint32_t)Mz +
                                 (uint32_t)g[2];
            const uint32_t dy = (uint32_t)Mz, dx = (uint32_t)My * (uint32_t)Mz;
            // the next x row: cut at a wall, wrapped when periodic (c_x <= n_x - 2 there)
            const bool has_x = c[0] + 1 < G.n[0];
            const uint32_t nxt = own + dx;
            const uint32_t rows[5] = {own - 1u, own + dy - 1u, nxt - dy - 1u, nxt - 1u, nxt + dy - 1u};
            const uint32_t nmax = (uint32_t)b.n;
            int2* rng_t = rng + threadIdx.x;
            uint32_t mask = 0u;
#pragma unroll
            for (int r = 0; r < 5; ++r) {
                if (r >= 2 && !has_x) break;
                int32_t q0 = (int32_t)min(b.start[rows[r]], nmax);
                const int32_t q1 = (int32_t)min(b.start[rows[r] + 3u], nmax);
                if (r == 0) q0 = max(q0, (int32_t)p + 1);
                if (q1 > q0) {
                    rng_t[r * kThreads] = make_int2(q0, q1);
                    mask |= 1u << r;
                }
            }
            walk_rows<T, DIM, false, true, false>(b, G, rng_t, mask, 0u, (T)0, xi, vi, dt, R2, bd, bid, bq, tag);
            if (bq >= 0) atomicMin(&b.bkey[p], partner_key<T>(bd, bid));
            return;
        }
    }
    Win w[3];
    bool amb = false;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        w[d] = window_1d(g[d], c[d], I.s[d], I.M[d], kk[d], G.wall[d]);
        amb = amb || w[d].amb;
    }
    uint32_t self_key = 0;
    if (kSym) {
        self_key = (DIM == 3) ? I.key_base + ((uint32_t)g[0] * (uint32_t)I.M[1] + (uint32_t)g[1]) * (uint32_t)I.M[2] +
                                    (uint32_t)g[2]
                              : I.key_base + (uint32_t)g[0] * (uint32_t)I.M[1] + (uint32_t)g[1];
    }
    if (amb)
        scan_window<T, DIM, true, true, kSym>(b, G, I, w, xi, vi, dt, R2, bd, bid, bq, rng + threadIdx.x,
                                              (int32_t)p, tag, self_key);
    else
        scan_window<T, DIM, false, true, kSym>(b, G, I, w, xi, vi, dt, R2, bd, bid, bq, rng + threadIdx.x,
                                               (int32_t)p, tag, self_key);
    if (kSym) {
        if (bq >= 0) atomicMin(&b.bkey[p], partner_key<T>(bd, bid));
    } else {
        b.bkey[p] = bq >= 0 ? partner_key<T>(bd, bid) : kNoPartner;
    }
}

// ------------------------------------------------------ paired binary32 test
// A home particle of the paired test (its coordinates and the step's
// constants) and the periodic image shift of the candidates' range, each value
// in both halves of a float2.
struct PairHome {
    float2 x0, x1, x2, v0, v1, v2, dt2, mR2;
};
struct PairShift {
    float2 s0, s1, s2;
};

__device__ __forceinline__ PairHome pair_home(const float xi[3], const float vi[3], float dt, float R2) {
    PairHome h;
    h.x0 = make_float2(xi[0], xi[0]);
    h.x1 = make_float2(xi[1], xi[1]);
    h.x2 = make_float2(xi[2], xi[2]);
    h.v0 = make_float2(vi[0], vi[0]);
    h.v1 = make_float2(vi[1], vi[1]);
    h.v2 = make_float2(vi[2], vi[2]);
    h.dt2 = make_float2(dt, dt);
    h.mR2 = make_float2(-R2, -R2);   // r2 - R^2 as r2 + (-R^2): the same rounding
    return h;
}

__device__ __forceinline__ PairShift pair_shift(const float sh[3]) {
    return PairShift{make_float2(sh[0], sh[0]), make_float2(sh[1], sh[1]), make_float2(sh[2], sh[2])};
}

// The arithmetic of criteria 1-2 (Eqs. 5-6, 8-9) for one home against the two
// candidates of a staged pair in the negated layout A = (-x, -x', -y, -y'),
// B = (-z, -z', -vx, -vx'), C = (-vy, -vy', -vz, -vz'): a = dr.dv, b = |dv|^2,
// |dr|^2, f = fma(b, dt, a) and disc = a^2 - b (|dr|^2 - R^2).  Each component
// of __fadd2_rn / __fmul2_rn / __ffma2_rn rounds exactly as the scalar
// operation, and x - y is x + (-y) in IEEE arithmetic, so every quantity is bit
// for bit that of poca_test_sh.
template <int DIM, bool SH>
__device__ __forceinline__ void paired_core(const PairHome& h, const PairShift& sh, const float4 A, const float4 B,
                                            const float4 C, float2& rr, float2& a, float2& bb, float2& f,
                                            float2& disc) {
    float2 d0 = __fadd2_rn(h.x0, make_float2(A.x, A.y));
    float2 d1 = __fadd2_rn(h.x1, make_float2(A.z, A.w));
    float2 d2v = make_float2(0.f, 0.f);
    if (DIM == 3) d2v = __fadd2_rn(h.x2, make_float2(B.x, B.y));
    if (SH) {
        d0 = __fadd2_rn(d0, sh.s0);
        d1 = __fadd2_rn(d1, sh.s1);
        if (DIM == 3) d2v = __fadd2_rn(d2v, sh.s2);
    }
    const float2 u0 = __fadd2_rn(h.v0, make_float2(B.z, B.w));
    const float2 u1 = __fadd2_rn(h.v1, make_float2(C.x, C.y));
    a = __fmul2_rn(d0, u0);
    a = __ffma2_rn(d1, u1, a);
    bb = __fmul2_rn(u0, u0);
    bb = __ffma2_rn(u1, u1, bb);
    rr = __fmul2_rn(d0, d0);
    rr = __ffma2_rn(d1, d1, rr);
    if (DIM == 3) {
        const float2 u2 = __fadd2_rn(h.v2, make_float2(C.z, C.w));
        a = __ffma2_rn(d2v, u2, a);
        bb = __ffma2_rn(u2, u2, bb);
        rr = __ffma2_rn(d2v, d2v, rr);
    }
    f = __ffma2_rn(bb, h.dt2, a);
    const float2 y = __fmul2_rn(bb, __fadd2_rn(rr, h.mR2));
    disc = __ffma2_rn(a, a, make_float2(-y.x, -y.y));
}

// Criteria 1-2 for the two candidates: bit 0 / 1 of the result is set when the
// first / second passes (the real-root test is evaluated for both, so that no
// lane branches off for criterion 2; b > 0 needs no test of its own: a < 0 and
// fma(b, dt, a) > 0 give b dt > -a > 0 exactly).  rr, a, bb give d^2 of a
// passing candidate.
template <int DIM, bool SH>
__device__ __forceinline__ unsigned paired_test(const PairHome& h, const PairShift& sh, const float4 A,
                                                const float4 B, const float4 C, float2& rr, float2& a, float2& bb) {
    float2 f, disc;
    paired_core<DIM, SH>(h, sh, A, B, C, rr, a, bb, f, disc);
    return ((a.x < 0.f && f.x > 0.f && disc.x >= 0.f) ? 1u : 0u) | ((a.y < 0.f && f.y > 0.f && disc.y >= 0.f) ? 2u : 0u);
}

// The same test with its decisions left in sign bits, for the pruned tile
// search: bit 31 of w.x / w.y is set when a < 0, f > 0 and disc >= 0 may all
// hold for the first / second candidate.  It is set for every candidate that
// passes (a < 0 sets the sign of a; f > 0 and disc >= 0 leave theirs clear:
// disc = fma(a, a, -y) is never -0, as an exact zero sum rounds to +0 and
// a * a is never -0) and also for a = -0, f = +0 or a NaN, so the caller
// re-tests a set bit exactly (pair_passes).  Four candidates' conditions then
// cost four LOP3s and one compare.
template <int DIM, bool SH>
__device__ __forceinline__ uint2 paired_signs(const PairHome& h, const PairShift& sh, const float4 A, const float4 B,
                                              const float4 C, float2& rr, float2& a, float2& bb) {
    float2 f, disc;
    paired_core<DIM, SH>(h, sh, A, B, C, rr, a, bb, f, disc);
    return make_uint2(__float_as_uint(a.x) & ~__float_as_uint(f.x) & ~__float_as_uint(disc.x),
                      __float_as_uint(a.y) & ~__float_as_uint(f.y) & ~__float_as_uint(disc.y));
}

// Criteria 1-2 for one candidate from its a, b, |dr|^2, rounded as in the
// paired test (each paired component rounds as these scalar operations).
__device__ __forceinline__ bool pair_passes(const PairHome& h, float rr, float a, float bb) {
    const float f = __fmaf_rn(bb, h.dt2.x, a);
    const float y = __fmul_rn(bb, __fadd_rn(rr, h.mR2.x));
    const float disc = __fmaf_rn(a, a, -y);
    return a < 0.f && f > 0.f && disc >= 0.f;
}

// ------------------------------------------------------ tile search
// Instances whose search cells are the c-bins themselves (no subdivision):
// every particle of a cell has the same window, the 3^D c-bin neighbourhood
// (criterion 3), so one block per cell reads the window's candidates once
// into shared memory and every home particle of the cell runs the same loop
// over them (broadcast reads, no divergence between lanes).  Same decisions as
// the direct search: rows of the window as key ranges with their periodic
// images, binary32 symmetric (a home tests only candidates at higher sorted
// positions and offers the outcome to both keys), binary64 full window.
constexpr int kTileThreads = 256;   // largest block of the tile search (the launch may use fewer)
constexpr int kTileRanges = 18;   // 3 x 3 rows x 2 parts (a periodic fast dimension may split)

// Default staging capacity: candidates (pos + vel) held in shared memory at
// once, 48 KiB in either precision; a handle may choose another (tile_cap).
template <typename T>
struct TileCap {
    static constexpr int value = 1536;
};
template <>
struct TileCap<double> {
    static constexpr int value = 768;
};

// The rows of c-bin kc's window as key ranges of sorted positions (one per
// row and part of the fast dimension, with the row's periodic image shift):
// range r is [rq0[r], rq0[r] + rlen[r]), at offset rpre[r] of the ranges'
// concatenation; nr_s ranges, tot_s candidates.  Binary32 (symmetric) keeps
// only positions from the cell's own first one h0 on.  Block-wide (syncs).
template <typename T, int DIM>
__device__ __forceinline__ void tile_window_ranges(const Bufs<T>& b, const GeoT<T>& G, const InstDev& I, int inst,
                                                   uint32_t kc, int64_t h0, int* rq0, int* rlen, int* rpre,
                                                   T (*rsh)[3], int& nr_s, int& tot_s) {
    constexpr bool kSym = sizeof(T) == 4;
    const int tid = threadIdx.x;
    // cell coordinates from the key (x slowest)
    uint32_t rel = kc - I.key_base;
    int g[3] = {0, 0, 0};
    if (DIM == 3) {
        g[2] = (int)(rel % (uint32_t)I.M[2]);
        rel /= (uint32_t)I.M[2];
    }
    g[1] = (int)(rel % (uint32_t)I.M[1]);
    g[0] = (int)(rel / (uint32_t)I.M[1]);
    const int* kk = b.dyn[inst].k;
    Win w[3];
#pragma unroll
    for (int d = 0; d < DIM; ++d) w[d] = window_1d(g[d], g[d], 1, I.M[d], kk[d], G.wall[d]);
    constexpr int F = DIM - 1;
    const int MF = I.M[F];
    // fast-dimension parts of the window
    int fa[2], fb[2];
    T fs[2] = {(T)0, (T)0};
    int nf = 1;
    if (w[F].lo < 0) {
        fa[0] = w[F].lo + MF; fb[0] = MF - 1; fs[0] = G.L[F];
        fa[1] = 0; fb[1] = w[F].hi;
        nf = 2;
    } else if (w[F].hi >= MF) {
        fa[0] = w[F].lo; fb[0] = MF - 1;
        fa[1] = 0; fb[1] = w[F].hi - MF; fs[1] = -G.L[F];
        nf = 2;
    } else {
        fa[0] = w[F].lo; fb[0] = w[F].hi;
    }
    const int nx = w[0].hi - w[0].lo + 1;
    const int ny = (DIM == 3) ? w[1].hi - w[1].lo + 1 : 1;
    // one range per (row, part); thread r fills entry r
    const int nrange = nx * ny * nf;
    if (tid < kTileRanges) {
        rq0[tid] = 0;
        rlen[tid] = 0;
    }
    if (tid < nrange) {
        const int part = tid % nf;
        const int row = tid / nf;
        const int ix = (DIM == 3) ? row / ny : row;
        const int iy = (DIM == 3) ? row % ny : 0;
        T sx, sy = (T)0;
        const int gx = unwrap<T>(w[0].lo + ix, I.M[0], G.L[0], sx);
        const int gy = (DIM == 3) ? unwrap<T>(w[1].lo + iy, I.M[1], G.L[1], sy) : 0;
        const uint32_t My = (DIM == 3) ? (uint32_t)I.M[1] : 1u;
        const uint32_t rk = I.key_base + ((uint32_t)gx * My + (uint32_t)gy) * (uint32_t)MF;
        const uint32_t nmax = (uint32_t)b.n;
        int32_t q0 = (int32_t)min(b.start[rk + (uint32_t)fa[part]], nmax);
        const int32_t q1 = (int32_t)min(b.start[rk + (uint32_t)fb[part] + 1u], nmax);
        if (kSym) q0 = max(q0, (int32_t)h0);   // lower positions test this cell's particles
        rq0[tid] = q0;
        rlen[tid] = max(q1 - q0, 0);
        rsh[tid][0] = sx;
        rsh[tid][1] = (DIM == 3) ? sy : fs[part];
        rsh[tid][2] = fs[part];
    }
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int r = 0; r < nrange; ++r) {
            rpre[r] = acc;
            acc += rlen[r];
        }
        nr_s = nrange;
        tot_s = acc;
    }
    __syncthreads();
}

template <typename T, int DIM, bool MINIMG>
__device__ __forceinline__ void tile_search_cell(const Bufs<T>& b, const GeoT<T>& G, const InstDev& I, int inst,
                                                 uint32_t kc, int64_t h0, int64_t h1, typename Vec4<T>::type* sp,
                                                 typename Vec4<T>::type* sv, int* rq0, int* rlen, int* rpre,
                                                 T (*rsh)[3], int& nr_s, int& tot_s) {
    using V = typename Vec4<T>::type;
    constexpr bool kSym = sizeof(T) == 4;
    const int CAP = b.tile_cap;   // even
    const int tid = threadIdx.x;
    tile_window_ranges<T, DIM>(b, G, I, inst, kc, h0, rq0, rlen, rpre, rsh, nr_s, tot_s);
    const int nr = nr_s, total = tot_s;
    // The window may be split between tile_split blocks of the same c-bin
    // (blockIdx.y = part), each taking every tile_split-th chunk of `per`
    // candidates (binary32 only: the blocks combine their minima with the
    // keys' atomicMin).  A block with a single chunk stages it once for all its
    // home chunks.
    const int split = kSym ? (int)gridDim.y : 1;
    const int part = kSym ? (int)blockIdx.y : 0;
    int per = CAP;
    if (split > 1) per = min(CAP, ((total + split - 1) / split + 1) & ~1);
    if (part * per >= total) return;   // nothing left for this block (block-uniform)
    const bool once = part * per + split * per >= total;
    // Binary32 without per-candidate minimum image: candidates are staged in
    // pairs (staged entries 2k and 2k + 1 side by side, negated so that
    // x_i - x_j is one paired addition) and every home tests two candidates at
    // once with the paired binary32 instructions of sm_100+.  Each component of
    // __fadd2_rn / __fmul2_rn / __ffma2_rn rounds exactly as the scalar
    // operation, and x - y is x + (-y) in IEEE arithmetic, so the decisions and
    // d^2 are bit for bit those of poca_test_sh.
    constexpr bool kPair = std::is_same<T, float>::value && !MINIMG;
    float4* pA = reinterpret_cast<float4*>(sp);          // (-x, -x', -y, -y')
    float4* pB = pA + CAP / 2;                            // (-z, -z', -vx, -vx')
    float4* pC = reinterpret_cast<float4*>(sv);          // (-vy, -vy', -vz, -vz')
    uint2* pT = reinterpret_cast<uint2*>(pC + CAP / 2);  // (tag, tag')
    auto stage = [&](int c0) {
        const int cn = min(per, total - c0);
        for (int e = tid; e < cn; e += blockDim.x) {
            const int ge = c0 + e;
            int r = 0;
            while (r + 1 < nr && rpre[r + 1] <= ge) ++r;
            const int64_t q = (int64_t)rq0[r] + (ge - rpre[r]);
            if constexpr (kPair) {
                const float4 P = ldg_vec(b.posA + q), Q = ldg_vec(b.velA + q);
                const int k = e >> 1, s = e & 1;
                float* a = reinterpret_cast<float*>(pA + k);
                float* bz = reinterpret_cast<float*>(pB + k);
                float* c = reinterpret_cast<float*>(pC + k);
                a[s] = -P.x;
                a[2 + s] = -P.y;
                bz[s] = -P.z;
                bz[2 + s] = -Q.x;
                c[s] = -Q.y;
                c[2 + s] = -Q.z;
                reinterpret_cast<uint32_t*>(pT + k)[s] = __float_as_uint(P.w);
            } else {
                sp[e] = ldg_vec(b.posA + q);
                sv[e] = ldg_vec(b.velA + q);
            }
        }
    };
    if (once) {
        stage(part * per);
        __syncthreads();
    }
    const T dt = step_dt(b.dyn[inst], T()), R2 = inst_R2(I, T());
    for (int32_t hc = (int32_t)h0; hc < (int32_t)h1; hc += (int32_t)blockDim.x) {
        const int32_t p = hc + tid;
        const bool home = p < (int32_t)h1;
        V P = {}, Q = {};
        if (home) {
            P = b.posA[p];
            Q = b.velA[p];
        }
        const T xi[3] = {P.x, P.y, P.z};
        const T vi[3] = {Q.x, Q.y, Q.z};
        const uint32_t tag = R<T>::bits(P.w);
        // sorted position by id, read by the move kernel to find a partner (every
        // home is visited in exactly one chunk of homes of part 0)
        if (home && part == 0) b.slot_of[I.p_off + (int64_t)tag_id(b, tag)] = (uint32_t)p;
        T bd = R<T>::inf();
        uint32_t bid = 0xffffffffu;
        // binary32: a home tests only higher positions; binary64: the whole
        // window (the particle itself fails b > 0)
        const int32_t lim = kSym ? p : -1;
        // the candidates [e0, e1) of one range; SH: the range has a periodic image;
        // CHK: the range may hold positions at or below the home's (own c-bin)
        auto scan = [&](auto has_shift, auto check, int e0, int e1, int c0, int32_t qoff, const T sh[3]) {
            constexpr bool SH = decltype(has_shift)::value;
            constexpr bool CHK = decltype(check)::value;
#pragma unroll 2
            for (int e = e0; e < e1; ++e) {
                const int32_t q = qoff + e;
                if (CHK && q <= lim) continue;
                const V Pj = sp[e - c0];
                const V Qj = sv[e - c0];
                const T xj[3] = {Pj.x, Pj.y, Pj.z};
                const T vj[3] = {Qj.x, Qj.y, Qj.z};
                T d2;
                const bool pass = SH || MINIMG ? poca_test_sh<T, DIM, MINIMG>(G, xi, vi, xj, vj, sh, dt, R2, d2)
                                               : poca_test_sh<T, DIM, false, false>(G, xi, vi, xj, vj, sh, dt, R2, d2);
                if (pass) {
                    const uint32_t idj = R<T>::bits(Pj.w);
                    if (d2 < bd || (d2 == bd && idj < bid)) {
                        bd = d2;
                        bid = idj;
                    }
                    if (kSym) atomicMin(&b.bkey[q], partner_key<T>(d2, tag));
                }
            }
        };
        // paired layout: candidates [e0, e1) of one range, two per step; an
        // entry without its pair (odd start or end of the range) alone
        auto scan2 = [&](auto has_shift, auto check, int e0, int e1, int c0, int32_t qoff, const T sh[3]) {
            if constexpr (kPair) {
                constexpr bool SH = decltype(has_shift)::value;
                constexpr bool CHK = decltype(check)::value;
                // the closest-candidate bookkeeping of one passing candidate
                auto take = [&](float d2, uint32_t idj, int32_t q) {
                    if (d2 < bd || (d2 == bd && idj < bid)) {
                        bd = d2;
                        bid = idj;
                    }
                    atomicMin(&b.bkey[q], partner_key<float>(d2, tag));
                };
                auto one = [&](int e) {
                    const int32_t q = qoff + e;
                    if (CHK && q <= lim) return;
                    const int l = e - c0, k = l >> 1, s = l & 1;
                    const float* a = reinterpret_cast<const float*>(pA + k);
                    const float* bz = reinterpret_cast<const float*>(pB + k);
                    const float* c = reinterpret_cast<const float*>(pC + k);
                    const float xj[3] = {-a[s], -a[2 + s], -bz[s]};
                    const float vj[3] = {-bz[2 + s], -c[s], -c[2 + s]};
                    float d2;
                    if (poca_test_sh<float, DIM, false, SH>(G, xi, vi, xj, vj, sh, dt, R2, d2))
                        take(d2, reinterpret_cast<const uint32_t*>(pT + k)[s], q);
                };
                // d^2 of a candidate that passed criteria 1-2, in poca_test_sh's order
                auto close = [&](float rr, float a, float bb, uint32_t idj, int32_t q) {
                    take(R<float>::sub(rr, R<float>::div(R<float>::mul(a, a), bb)), idj, q);
                };
                const PairHome ph = pair_home(xi, vi, dt, R2);
                const PairShift ps = pair_shift(sh);
                int e = e0;
                if ((e - c0) & 1) one(e++);
                // Only a candidate that passes all of criteria 1-2 (about one test
                // in a thousand) leaves the paired path, for d^2.  The whole test
                // of staged pair k (candidates 2k, 2k + 1 of the chunk); bit 0 / 1
                // of the result: candidate passes criteria 1-2
                auto test2 = [&](int k, int32_t q, float2& rr, float2& a, float2& bb) -> unsigned {
                    unsigned ok = paired_test<DIM, SH>(ph, ps, pA[k], pB[k], pC[k], rr, a, bb);
                    if (CHK) ok &= (q > lim ? 1u : 0u) | (q + 1 > lim ? 2u : 0u);
                    return ok;
                };
                auto take2 = [&](unsigned ok, int k, int32_t q, float2 rr, float2 a, float2 bb) {
                    const uint2 tg = pT[k];
                    if (ok & 1u) close(rr.x, a.x, bb.x, tg.x, q);
                    if (ok & 2u) close(rr.y, a.y, bb.y, tg.y, q + 1);
                };
                // two staged pairs (four candidates) per step of the loop: the two
                // tests interleave, and one branch covers all four
                for (; e + 3 < e1; e += 4) {
                    const int k = (e - c0) >> 1;
                    const int32_t q = qoff + e;
                    float2 rr0, a0, b0, rr1, a1, b1;
                    const unsigned ok0 = test2(k, q, rr0, a0, b0);
                    const unsigned ok1 = test2(k + 1, q + 2, rr1, a1, b1);
                    if (ok0 | ok1) {
                        if (ok0) take2(ok0, k, q, rr0, a0, b0);
                        if (ok1) take2(ok1, k + 1, q + 2, rr1, a1, b1);
                    }
                }
                if (e + 1 < e1) {
                    const int k = (e - c0) >> 1;
                    float2 rr0, a0, b0;
                    const unsigned ok0 = test2(k, qoff + e, rr0, a0, b0);
                    if (ok0) take2(ok0, k, qoff + e, rr0, a0, b0);
                    e += 2;
                }
                if (e < e1) one(e);
            }
        };
        for (int c0 = part * per; c0 < total; c0 += split * per) {
            if (!once) {
                __syncthreads();
                stage(c0);
                __syncthreads();
            }
            if (!home) continue;
            const int c1 = min(total, c0 + per);
            for (int r = 0; r < nr; ++r) {
                const int e0 = max(rpre[r], c0), e1 = min(rpre[r] + rlen[r], c1);
                if (e0 >= e1) continue;
                const T sh[3] = {rsh[r][0], rsh[r][1], rsh[r][2]};
                const int32_t qoff = rq0[r] - rpre[r];
                // binary32: a range that starts after the cell's last particle needs no position check
                // (binary64 tests the whole window: the particle itself fails b > 0)
                const bool chk = kSym && qoff + e0 <= (int32_t)h1 - 1;
                const bool shifted = sh[0] != (T)0 || sh[1] != (T)0 || sh[2] != (T)0;
                if constexpr (kPair) {
                    if (shifted) {
                        if (chk) scan2(std::true_type{}, std::true_type{}, e0, e1, c0, qoff, sh);
                        else scan2(std::true_type{}, std::false_type{}, e0, e1, c0, qoff, sh);
                    } else {
                        if (chk) scan2(std::false_type{}, std::true_type{}, e0, e1, c0, qoff, sh);
                        else scan2(std::false_type{}, std::false_type{}, e0, e1, c0, qoff, sh);
                    }
                } else if (shifted) {
                    if (chk) scan(std::true_type{}, std::true_type{}, e0, e1, c0, qoff, sh);
                    else scan(std::true_type{}, std::false_type{}, e0, e1, c0, qoff, sh);
                } else {
                    if (chk) scan(std::false_type{}, std::true_type{}, e0, e1, c0, qoff, sh);
                    else scan(std::false_type{}, std::false_type{}, e0, e1, c0, qoff, sh);
                }
            }
        }
        if (home) {
            if (kSym) {
                if (bid != 0xffffffffu) atomicMin(&b.bkey[p], partner_key<T>(bd, bid));
            } else {
                b.bkey[p] = bid != 0xffffffffu ? partner_key<T>(bd, bid) : kNoPartner;
            }
        }
    }
}

// ------------------------------------------------------ pruned tile search (binary32)
// In a dense window almost every (home, candidate) pair of the tile search is
// too far apart to meet within the step: a pair can pass criteria 1-2 only if,
// at some time t in [0, dt], the two particles are within R of each other in
// every coordinate.  So every particle is bounded by its swept box (the box of
// the segment x .. x + v dt), and each cluster of kCluster staged candidates and
// each group of 32 homes by the union of theirs.  Two filters, both with boxes
// widened by R and a rounding margin: a warp first checks 32 clusters against
// its group's box (a lane per cluster), then every cluster that meets it
// against each lane's own home box; the (home, cluster) pairs that meet go to
// a per-warp queue, and the warp tests 32 queued pairs at a time (a lane per
// pair: about one in seven of the group's pairs).  For small boxes these
// instances search on half c-bins (2 search cells per c-bin and dimension):
// the canonical (search cell, id) order then groups every c-bin's particles by
// half c-bin, so consecutive homes and consecutive candidates are close in
// space without any sort in the block.  The window is still the 3^D c-bin
// neighbourhood (criterion 3), as rows of half c-bins.  The order of the tests
// changes nothing: every home's key and every candidate's key take the minimum
// of theirs by atomicMin.
//
// Rounding margin.  For a pair that the binary32 test accepts, exact arithmetic
// on its rounded differences gives d^2 <= R^2 + 15 u |dr|^2 (u = 2^-24; the
// error of disc is at most 14 u b |dr|^2), a crossing time within
// 3 u |dr| / |dv| + 6 u dt of [0, dt], and differences within 6 u C of the
// exact ones (C bounds every coordinate plus an image shift).  So at a time in
// [0, dt] the two particles are within R + sqrt(15 u) |dr| + 3 u |dr| +
// 7 u |dv| dt + 6 u C of each other in every coordinate.  With |dr| <=
// 2 sqrt(3) w (w the widest c-bin: both lie in one 3^D neighbourhood) that is
// below R (1 + 2^-10) + 2^-7 w + 2^-16 C, the widening of a home's or a
// group's box, plus 2^-12 of each particle's |v dt|_1, the widening of every
// swept box.
constexpr int kSub = 2;          // search cells per c-bin and position dimension of a pruned instance
constexpr int kSubRanges = 72;   // window rows (6 x 6 in 3-D) x 2 parts of the fast dimension
constexpr int kCluster = 4;      // staged candidates per cluster (two staged pairs: one step of the loop)
constexpr int kBatch = 64;       // clusters of one work item (a home group against them)
constexpr int kMaxBatches = 96;  // batches of one staged chunk: 6144 / kCluster / kBatch + kSubRanges = 96
constexpr int kQueue = 64;       // (home, cluster) pairs a warp holds before testing them (a power of two)
constexpr int32_t kNoHome = 0x7fffffff;   // sorted position of a lane without a home: above every cluster's

// Swept box of one particle over the step, widened by 2^-12 |v dt|_1.
template <int DIM>
__device__ __forceinline__ void swept_box(const float x[3], const float v[3], float dt, float lo[3], float hi[3]) {
    float s[3], e = 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        s[d] = v[d] * dt;
        e += fabsf(s[d]);
    }
    e *= 0x1p-12f;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        lo[d] = x[d] + fminf(0.f, s[d]) - e;
        hi[d] = x[d] + fmaxf(0.f, s[d]) + e;
    }
}

// One cluster of kCluster staged candidates: its box per dimension in the
// block's frame in the form (lo, -hi) (two halves, c-bin units; the bits of a
// __half2), and the sorted position of its first slot (slot j holds position
// q0 + j; a pad slot holds NaN).
struct __align__(16) ClusterBox {
    uint32_t x, y, z;
    int q0;
};

__device__ __forceinline__ uint32_t half2_bits(__half2 h) {
    uint32_t u;
    memcpy(&u, &h, sizeof(u));
    return u;
}

// Dynamic shared memory of the pruned search for a capacity of `cap` staged
// candidates (cap rounded down to a multiple of 16): six floats per staged
// candidate and one ClusterBox per cluster.
__host__ __device__ constexpr size_t pruned_smem_bytes(int cap) {
    return (size_t)(24 + 16 / kCluster) * (size_t)(cap & ~15);
}

// Conservative half-precision bounds of a box [lo, hi] in c-bin units of the
// block's frame, widened by eps (the rounding of the float map into those
// units), in the two forms of one test: (lo, -hi) rounded down and (hi, -lo)
// rounded up.  Boxes a and b meet in a dimension when both halves of a as
// (lo, -hi) are at most those of b as (hi, -lo): lo_a <= hi_b and lo_b <= hi_a.
__device__ __forceinline__ uint32_t box_lo_neghi(float lo, float hi, float eps) {
    return half2_bits(__halves2half2(__float2half_rd(lo - eps), __float2half_rd(-(hi + eps))));
}
__device__ __forceinline__ uint32_t box_hi_neglo(float lo, float hi, float eps) {
    return half2_bits(__halves2half2(__float2half_ru(hi + eps), __float2half_ru(eps - lo)));
}

// 1 when the boxes meet in all three dimensions (a: (lo, -hi), b: (hi, -lo)
// per dimension), else 0: paired half-precision compares, no branch.
__device__ __forceinline__ uint32_t boxes_meet3(uint32_t ax, uint32_t ay, uint32_t az, uint32_t bx, uint32_t by,
                                                uint32_t bz) {
    uint32_t r;
    asm("{\n\t.reg .pred p0, p1, p2, p3, p4, p5;\n\t"
        "setp.le.f16x2 p0|p1, %1, %4;\n\t"
        "setp.le.f16x2 p2|p3, %2, %5;\n\t"
        "setp.le.f16x2 p4|p5, %3, %6;\n\t"
        "and.pred p0, p0, p1;\n\t"
        "and.pred p2, p2, p3;\n\t"
        "and.pred p4, p4, p5;\n\t"
        "and.pred p0, p0, p2;\n\t"
        "and.pred p0, p0, p4;\n\t"
        "selp.u32 %0, 1, 0, p0;\n\t}"
        : "=r"(r)
        : "r"(ax), "r"(ay), "r"(az), "r"(bx), "r"(by), "r"(bz));
    return r;
}

// Cluster c meets the box b (hi, -lo) per dimension and may hold a position
// above q (in 2-D the third halves are 0 <= 0).
__device__ __forceinline__ bool cluster_meets(const ClusterBox& c, const uint32_t b[3], int32_t q) {
    return ((uint32_t)(c.q0 > q - (kCluster - 1)) & boxes_meet3(c.x, c.y, c.z, b[0], b[1], b[2])) != 0u;
}

// Exclusive prefix sums of v(0) ... v(n - 1), n <= 96, by one whole warp: lane
// l sums entries 3l ... 3l + 2, the lanes scan their sums; out[i] = v(0) + ... +
// v(i - 1) for i <= n.
template <typename Fn>
__device__ __forceinline__ void warp_exclusive_scan96(int n, Fn v, int* out) {
    const int lane = threadIdx.x & 31;
    int x[3], own = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int i = 3 * lane + j;
        x[j] = i < n ? v(i) : 0;
        own += x[j];
    }
    int inc = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
    }
    int acc = inc - own;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int i = 3 * lane + j;
        if (i <= n) out[i] = acc;
        acc += x[j];
    }
}

// Search key of search cell (gx, gy, gz) of instance I.
template <int DIM>
__device__ __forceinline__ uint32_t cell_key(const InstDev& I, int gx, int gy, int gz) {
    if (DIM == 3) return I.key_base + ((uint32_t)gx * (uint32_t)I.M[1] + (uint32_t)gy) * (uint32_t)I.M[2] + (uint32_t)gz;
    return I.key_base + (uint32_t)gx * (uint32_t)I.M[1] + (uint32_t)gy;
}

// One block per c-bin c of a pruned instance.
template <int DIM, int CAPC>
__device__ __forceinline__ void tile_search_pruned(const Bufs<float>& b, const GeoT<float>& G, const InstDev& I,
                                                   int inst, const int c[3], unsigned char* smem) {
    constexpr int F = DIM - 1;   // fastest key dimension
    // staged slots per chunk (a multiple of kCluster): for the default launch a
    // compile-time constant (the shared-memory offsets become immediates), else
    // the handle's
    const int CAP = CAPC ? CAPC : (b.tile_cap & ~15);
    // the default launch (CAPC != 0) has kTileThreads threads
    const int tid = threadIdx.x, lane = tid & 31, nthr = CAPC ? kTileThreads : (int)blockDim.x;
    const int warp = tid >> 5, nwarps = nthr >> 5;
    // staged pair k (slots 2k, 2k + 1): pA (-x, -x', -y, -y'), pB (-z, -z', -vx, -vx'),
    // pC (-vy, -vy', -vz, -vz')
    float4* pA = reinterpret_cast<float4*>(smem);
    float4* pB = pA + CAP / 2;
    float4* pC = pB + CAP / 2;
    // cluster c: its box in the block's frame (c-bin units from the c-bin's low
    // corner, its range's image shift applied) and its largest sorted position
    ClusterBox* cbox = reinterpret_cast<ClusterBox*>(pC + CAP / 2);
    __shared__ int rq0[kSubRanges], rlen[kSubRanges], ppre[kSubRanges + 1], pb0[kSubRanges], pb1[kSubRanges];
    __shared__ float rsh[kSubRanges][3];
    __shared__ int hq0[4], hpre[5];                       // the c-bin's own rows (homes)
    __shared__ uint32_t gbox[kTileThreads / 32][3];       // home group boxes (hi, -lo), widened
    __shared__ int gminp[kTileThreads / 32];              // lowest sorted position of each home group
    __shared__ int gnext[kTileThreads / 32];              // next batch of each home group
    __shared__ int batch[kMaxBatches];                    // batch i: range << 18 | (clusters - 1) << 12 | first
    __shared__ int bpre[kSubRanges + 1];                  // first batch of each segment (at its first range)
    __shared__ unsigned short wqueue[kTileThreads / 32][kQueue];   // per warp: cluster << 5 | home lane
    __shared__ int nr_s;
    __shared__ unsigned long long blk_tests;

    // the homes: rows (2 c_x + i, 2 c_y + j) of the c-bin, each with its two
    // search cells along the fast dimension (consecutive keys)
    constexpr int kHomeRows = DIM == 3 ? 4 : 2;
    if (tid < kHomeRows) {
        const int gx = kSub * c[0] + (DIM == 3 ? tid >> 1 : tid);
        const int gy = DIM == 3 ? kSub * c[1] + (tid & 1) : kSub * c[1];
        const uint32_t k0 = DIM == 3 ? cell_key<3>(I, gx, gy, kSub * c[2]) : cell_key<2>(I, gx, gy, 0);
        const uint32_t nmax = (uint32_t)b.n;
        const int32_t q0 = (int32_t)min(b.start[k0], nmax), q1 = (int32_t)min(b.start[k0 + kSub], nmax);
        hq0[tid] = q0;
        hpre[tid + 1] = max(q1 - q0, 0);
    }
    __syncthreads();
    if (tid == 0) {
        hpre[0] = 0;
        for (int i = 1; i <= kHomeRows; ++i) hpre[i] += hpre[i - 1];
    }
    __syncthreads();
    const int nh_all = hpre[kHomeRows];
    if (nh_all == 0) return;   // block-uniform
    const int32_t h0 = hq0[0];   // the c-bin's lowest sorted position (its first row comes first)

    // the window: rows of the c-bin neighbourhood in search cells, each cut to
    // positions from h0 on (binary32 symmetric search: the lower sorted position
    // of a pair tests it)
    {
        int wlo[3], whi[3], nw[3] = {1, 1, 1};
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            wlo[d] = kSub * c[d] - kSub;
            whi[d] = kSub * c[d] + 2 * kSub - 1;
            if (G.wall[d]) {
                wlo[d] = max(wlo[d], 0);
                whi[d] = min(whi[d], I.M[d] - 1);
            }
            nw[d] = whi[d] - wlo[d] + 1;
        }
        // fast-dimension parts (a periodic window may wrap)
        const int MF = I.M[F];
        int fa[2], fb[2];
        float fs[2] = {0.f, 0.f};
        int nf = 1;
        if (wlo[F] < 0) {
            fa[0] = wlo[F] + MF; fb[0] = MF - 1; fs[0] = G.L[F];
            fa[1] = 0; fb[1] = whi[F];
            nf = 2;
        } else if (whi[F] >= MF) {
            fa[0] = wlo[F]; fb[0] = MF - 1;
            fa[1] = 0; fb[1] = whi[F] - MF; fs[1] = -G.L[F];
            nf = 2;
        } else {
            fa[0] = wlo[F]; fb[0] = whi[F];
        }
        const int ny = DIM == 3 ? nw[1] : 1;
        const int nrange = nw[0] * ny * nf;
        for (int t = tid; t < nrange; t += nthr) {
            const int part = t % nf, row = t / nf;
            const int ix = DIM == 3 ? row / ny : row, iy = DIM == 3 ? row % ny : 0;
            float sx, sy = 0.f;
            const int gx = unwrap<float>(wlo[0] + ix, I.M[0], G.L[0], sx);
            const int gy = DIM == 3 ? unwrap<float>(wlo[1] + iy, I.M[1], G.L[1], sy) : 0;
            const uint32_t rk = DIM == 3 ? cell_key<3>(I, gx, gy, 0) : cell_key<2>(I, gx, 0, 0);
            const uint32_t nmax = (uint32_t)b.n;
            const int32_t q0 = max((int32_t)min(b.start[rk + (uint32_t)fa[part]], nmax), h0);
            const int32_t q1 = (int32_t)min(b.start[rk + (uint32_t)fb[part] + 1u], nmax);
            rq0[t] = q0;
            rlen[t] = max(q1 - q0, 0);
            rsh[t][0] = sx;
            rsh[t][1] = DIM == 3 ? sy : fs[part];
            rsh[t][2] = DIM == 3 ? fs[part] : 0.f;
        }
        if (tid == 0) nr_s = nrange;
    }
    __syncthreads();
    const int nr = nr_s;
    // every range padded to whole clusters: range r occupies [ppre[r], ppre[r + 1])
    if (warp == 0) warp_exclusive_scan96(nr, [&](int r) { return (rlen[r] + kCluster - 1) / kCluster * kCluster; }, ppre);
    if (tid == 0) blk_tests = 0ull;
    __syncthreads();
    const int ptot = ppre[nr];
    // window split between gridDim.y blocks of the c-bin, as in the plain tile search
    const int split = (int)gridDim.y, part = (int)blockIdx.y;
    int per = CAP;
    if (split > 1) per = min(CAP, ((ptot + split - 1) / split + kCluster - 1) / kCluster * kCluster);
    if (part * per >= ptot) return;   // nothing left for this block (block-uniform)
    const bool once = part * per + split * per >= ptot;
    const float dt = step_dt(b.dyn[inst], 0.f), R2 = inst_R2(I, 0.f);
    float wmax = 0.f, cmax = 0.f, lmax = 0.f;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        wmax = fmaxf(wmax, G.L[d] / (float)G.n[d]);
        cmax = fmaxf(cmax, fmaxf(fabsf(G.lo[d]), fabsf(G.hi[d])));
        lmax = fmaxf(lmax, G.L[d]);
    }
    const float margin = sqrtf(R2) * (1.f + 0x1p-10f) + 0x1p-7f * wmax + 0x1p-16f * (cmax + lmax);
    // Boxes go to c-bin units of this block's frame, u = (x - lo) n / L - c: three
    // binary32 roundings of terms up to (cmax + lmax) n / L, covered by eps
    float ueps[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int d = 0; d < DIM; ++d) ueps[d] = 0x1p-10f + 0x1p-21f * (cmax + lmax) * G.inv[d];
    const float qnan = __int_as_float(0x7fc00000);
    // a swept box [lo, hi], widened by the margin, as (hi, -lo) in the block's frame
    auto home_box = [&](const float lo[3], const float hi[3], uint32_t hb[3]) {
#pragma unroll
        for (int d = 0; d < 3; ++d)
            hb[d] = d < DIM ? box_hi_neglo((lo[d] - margin - G.lo[d]) * G.inv[d] - (float)c[d],
                                           (hi[d] + margin - G.lo[d]) * G.inv[d] - (float)c[d], ueps[d])
                            : 0u;
    };

    // Stage chunk [c0, c0 + per) of the padded ranges: a warp per range part,
    // each slot gathers its candidate (a pad: NaN, position -1) with the next
    // slot's loads already in flight, and the kCluster lanes of a cluster
    // combine their swept boxes and positions.  Then the batches of kBatch
    // clusters of every part.
    auto stage = [&](int c0) {
        const int cn = min(per, ptot - c0);
        for (int r = tid; r < nr; r += nthr) {   // up to kSubRanges ranges, blocks from 64 threads
            const int a = max(ppre[r], c0);
            const int e = max(a, min(ppre[r + 1], c0 + cn));
            pb0[r] = a - c0;
            pb1[r] = e - c0;
        }
        __syncthreads();
        for (int r = warp; r < nr; r += nwarps) {
            const int s0 = pb0[r], s1 = pb1[r];
            if (s0 >= s1) continue;   // warp-uniform
            const int32_t qb = rq0[r] + c0 - ppre[r];   // sorted position of slot s: qb + s
            const int sv = min(s1, ppre[r] + rlen[r] - c0);   // slots below sv hold candidates
            auto fetch = [&](int sl, float4& P, float4& Q) {
                P = make_float4(qnan, qnan, qnan, qnan);
                Q = P;
                if (sl < sv) {
                    P = ldg_vec(b.posA + qb + sl);
                    Q = ldg_vec(b.velA + qb + sl);
                }
            };
            float4 P, Q;
            fetch(s0 + lane, P, Q);
            for (int e0 = s0; e0 < s1; e0 += 32) {   // the same trip count on the warp's lanes (shuffles)
                const int sl = e0 + lane;
                float4 Pn, Qn;
                fetch(sl + 32, Pn, Qn);
                if (sl < s1) {
                    const int k = sl >> 1, h = sl & 1;
                    float* pa = reinterpret_cast<float*>(pA + k);
                    float* pbz = reinterpret_cast<float*>(pB + k);
                    float* pc = reinterpret_cast<float*>(pC + k);
                    pa[h] = -P.x;
                    pa[2 + h] = -P.y;
                    pbz[h] = -P.z;
                    pbz[2 + h] = -Q.x;
                    pc[h] = -Q.y;
                    pc[2 + h] = -Q.z;
                }
                const float x[3] = {P.x, P.y, P.z}, v[3] = {Q.x, Q.y, Q.z};
                float lo[3], hi[3];
                swept_box<DIM>(x, v, dt, lo, hi);
#pragma unroll
                for (int o = 1; o < kCluster; o <<= 1) {   // a pad's NaN drops out of fminf / fmaxf
#pragma unroll
                    for (int d = 0; d < DIM; ++d) {
                        lo[d] = fminf(lo[d], __shfl_xor_sync(kFull, lo[d], o));
                        hi[d] = fmaxf(hi[d], __shfl_xor_sync(kFull, hi[d], o));
                    }
                }
                if ((lane & (kCluster - 1)) == 0 && sl < s1) {
                    // the test takes x_i - (x_j - shift): the box of x_j - shift, in c-bin
                    // units from the block's c-bin corner
                    float ul[3], uh[3];
#pragma unroll
                    for (int d = 0; d < DIM; ++d) {
                        ul[d] = (lo[d] - rsh[r][d] - G.lo[d]) * G.inv[d] - (float)c[d];
                        uh[d] = (hi[d] - rsh[r][d] - G.lo[d]) * G.inv[d] - (float)c[d];
                    }
                    ClusterBox cb;
                    cb.x = box_lo_neghi(ul[0], uh[0], ueps[0]);
                    cb.y = box_lo_neghi(ul[1], uh[1], ueps[1]);
                    cb.z = DIM == 3 ? box_lo_neghi(ul[2], uh[2], ueps[2]) : 0u;
                    cb.q0 = qb + sl;   // sl is the cluster's first slot (s0 and e0 are multiples of kCluster)
                    cbox[sl / kCluster] = cb;
                }
                P = Pn;
                Q = Qn;
            }
        }
        if (warp == 0) {
            // Segments: runs of consecutive ranges with the same image shift, whose
            // clusters lie consecutively in the chunk.  Batches of up to kBatch
            // clusters of one segment: range (the shift's) << 18 | (clusters - 1) << 12
            // | first cluster.
            auto starts = [&](int r) {   // range r starts a segment
                return r < nr && (r == 0 || rsh[r][0] != rsh[r - 1][0] || rsh[r][1] != rsh[r - 1][1] ||
                                  rsh[r][2] != rsh[r - 1][2]);
            };
            // bit r of the 96-bit word (m0, m1, m2): range r starts a segment
            const unsigned m0 = __ballot_sync(kFull, starts(lane)), m1 = __ballot_sync(kFull, starts(32 + lane)),
                           m2 = __ballot_sync(kFull, starts(64 + lane));
            auto is_start = [&](int r) { return ((r < 32 ? m0 : r < 64 ? m1 : m2) >> (r & 31)) & 1u; };
            auto seg_end = [&](int r) {   // the first range after segment start r that starts another, or nr
                const int f = r + 1;
                const unsigned w0 = f < 32 ? m0 & (~0u << f) : 0u;
                const unsigned w1 = f < 32 ? m1 : f < 64 ? m1 & (~0u << (f - 32)) : 0u;
                const unsigned w2 = f < 64 ? m2 : f < 96 ? m2 & (~0u << (f - 64)) : 0u;
                const int e = w0 ? __ffs(w0) - 1 : w1 ? 31 + __ffs(w1) : w2 ? 63 + __ffs(w2) : nr;
                return min(e, nr);
            };
            // clusters [a, z) of the segment starting at range r: ranges wholly before
            // the chunk have pb0 = pb1 = 0, those wholly after it pb0 = pb1 >= cn
            auto seg_span = [&](int r, int& a, int& z) {
                a = min(pb0[r], cn) / kCluster;
                z = min(pb1[seg_end(r) - 1], cn) / kCluster;
            };
            auto seg_batches = [&](int r) {
                if (!is_start(r)) return 0;
                int a, z;
                seg_span(r, a, z);
                return (z - a + kBatch - 1) / kBatch;
            };
            warp_exclusive_scan96(nr, seg_batches, bpre);
            __syncwarp();
            for (int r = lane; r < nr; r += 32) {
                if (!is_start(r)) continue;
                int a, z;
                seg_span(r, a, z);
                for (int j = bpre[r], cl = a; cl < z; ++j, cl += kBatch)
                    batch[j] = (r << 18) | ((min(kBatch, z - cl) - 1) << 12) | cl;
            }
        }
    };

    // Work of a chunk: every home group (32 homes) against every batch of
    // kBatch clusters of the staged rows.  A warp starts on its own group and
    // takes its batches from the group's counter; once that is exhausted it
    // helps another group, so that no warp idles at the chunk's barrier while
    // others work.  Results go straight to the keys (atomicMin on both sides of
    // a passing pair), so a group's batches may run on any warp.
    if (once) {
        stage(part * per);
        __syncthreads();
    }
    unsigned wtests = 0;   // this warp's (home, staged slot) tests
    // position of home i (0 ... nh_all - 1) of the c-bin's rows
    auto home_pos = [&](int i) -> int32_t {
        int k = 0;
        while (k + 1 < kHomeRows && hpre[k + 1] <= i) ++k;
        return hq0[k] + (i - hpre[k]);
    };
    unsigned short* queue = wqueue[warp];
    for (int hc = 0; hc < nh_all; hc += nthr) {
        const int nh = min(nthr, nh_all - hc);
        const int ngroups = (nh + 31) >> 5;
        // group boxes: warp g bounds the swept boxes of group g, widened by the margin
        if (warp < ngroups) {
            const int hi = warp * 32 + lane;
            float wlo[3] = {R<float>::inf(), R<float>::inf(), R<float>::inf()};
            float whi[3] = {-R<float>::inf(), -R<float>::inf(), -R<float>::inf()};
            int32_t pmin = 0x7fffffff;
            if (hi < nh) {
                const int32_t p = home_pos(hc + hi);
                const float4 P = b.posA[p], Q = b.velA[p];
                // sorted position by id, read by the move kernel (part 0 visits every home once)
                if (part == 0) b.slot_of[I.p_off + (int64_t)tag_id(b, __float_as_uint(P.w))] = (uint32_t)p;
                const float x[3] = {P.x, P.y, P.z}, v[3] = {Q.x, Q.y, Q.z};
                swept_box<DIM>(x, v, dt, wlo, whi);
                pmin = p;
            }
            for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    wlo[d] = fminf(wlo[d], __shfl_xor_sync(kFull, wlo[d], o));
                    whi[d] = fmaxf(whi[d], __shfl_xor_sync(kFull, whi[d], o));
                }
                pmin = min(pmin, __shfl_xor_sync(kFull, pmin, o));
            }
            if (lane == 0) {
                uint32_t gb[3];
                home_box(wlo, whi, gb);
#pragma unroll
                for (int d = 0; d < 3; ++d) gbox[warp][d] = gb[d];
                gminp[warp] = pmin;
            }
        }
        for (int c0 = part * per; c0 < ptot; c0 += split * per) {
            if (!once) {
                __syncthreads();
                stage(c0);
            }
            if (tid < ngroups) gnext[tid] = 0;   // fresh group counters
            __syncthreads();
            const int nbatch = bpre[nr];
            int g = warp % ngroups, loaded = -1;
            float hx[3], hv[3];          // this lane's home
            uint32_t hb[3];              // its box, (hi, -lo)
            int32_t p = kNoHome;
            uint32_t tag = 0;
            // The warp's queue: (home lane, cluster) pairs whose boxes meet, n from
            // qhead on (a ring of kQueue entries)
            int qhead = 0, qn = 0;
            // d^2 of a candidate that passed criteria 1-2, offered to both keys
            auto close = [&](float rr, float a, float bb, int32_t hp, uint32_t htag, int32_t q, uint32_t qtag) {
                const float d2 = R<float>::sub(rr, R<float>::div(R<float>::mul(a, a), bb));
                atomicMin(&b.bkey[hp], partner_key<float>(d2, qtag));
                atomicMin(&b.bkey[q], partner_key<float>(d2, htag));
            };
            // Test n (<= 32) queued pairs from qhead on: lane l takes entry qhead + l,
            // the home of the entry's lane (by shuffles) against the entry's cluster
            // (two staged pairs).  A home tests only candidates at higher sorted
            // positions (each pair once).
            auto test_queued = [&](auto has_shift, int n, const PairShift& ps) {
                constexpr bool SH = decltype(has_shift)::value;
                __syncwarp();   // the entries written by other lanes
                const unsigned e = lane < n ? queue[(qhead + lane) & (kQueue - 1)] : 0u;
                const int src = (int)(e & 31u), k = (int)(e >> 5) * (kCluster / 2);
                const int32_t q = cbox[e >> 5].q0;   // candidate j at q + j (a pad never passes: NaN)
                float xi[3], vi[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    xi[d] = __shfl_sync(kFull, hx[d], src);
                    vi[d] = __shfl_sync(kFull, hv[d], src);
                }
                const int32_t hp = __shfl_sync(kFull, p, src);
                const uint32_t htag = __shfl_sync(kFull, tag, src);
                if (lane >= n) xi[0] = qnan;   // an empty lane fails every test
                const PairHome h = pair_home(xi, vi, dt, R2);
                float2 rr0, a0, b0, rr1, a1, b1;
                const uint2 w0 = paired_signs<DIM, SH>(h, ps, pA[k], pB[k], pC[k], rr0, a0, b0);
                const uint2 w1 = paired_signs<DIM, SH>(h, ps, pA[k + 1], pB[k + 1], pC[k + 1], rr1, a1, b1);
                if ((int)(w0.x | w0.y | w1.x | w1.y) < 0) {   // some candidate may pass: exact tests
                    unsigned pm = (w0.x >> 31) | (w0.y >> 31 << 1) | (w1.x >> 31 << 2) | (w1.y >> 31 << 3);
                    const int32_t dj = hp - q;   // candidates j <= dj lie at or below the home
                    if (dj >= 0) pm &= dj >= 3 ? 0u : 0xfu << (dj + 1);
                    while (pm) {   // this lane's flagged candidates, one at a time
                        const int j = __ffs(pm) - 1;
                        pm &= pm - 1;
                        const float rr = j == 0 ? rr0.x : j == 1 ? rr0.y : j == 2 ? rr1.x : rr1.y;
                        const float a = j == 0 ? a0.x : j == 1 ? a0.y : j == 2 ? a1.x : a1.y;
                        const float bb = j == 0 ? b0.x : j == 1 ? b0.y : j == 2 ? b1.x : b1.y;
                        if (pair_passes(h, rr, a, bb))
                            close(rr, a, bb, hp, htag, q + j, __float_as_uint(__ldg(&b.posA[q + j].w)));
                    }
                }
                wtests += (unsigned)(n * kCluster);
                qhead += n;
                __syncwarp();   // the entries are read before they are written again
            };
            // clusters [cb0, cb1) of one range part: 32 checks against the group's box
            // per ballot, then each overlapping cluster against every lane's own box;
            // the pairs that meet go to the queue, which is tested 32 at a time.  A
            // cluster whose positions all lie at or below a home holds no pair the
            // home tests.
            auto scan_batch = [&](auto has_shift, int cb0, int cb1, const float sh[3]) {
                const PairShift ps = pair_shift(sh);
                for (int cb = cb0; cb < cb1; cb += 32) {
                    const int cl = cb + lane;
                    bool ov = false;
                    if (cl < cb1) ov = cluster_meets(cbox[cl], gbox[g], gminp[g]);
                    for (unsigned m = __ballot_sync(kFull, ov); m; m &= m - 1) {
                        const int cm = cb + __ffs(m) - 1;
                        const bool hit = cluster_meets(cbox[cm], hb, p);
                        const unsigned hm = __ballot_sync(kFull, hit);
                        if (hit) queue[(qhead + qn + __popc(hm & ((1u << lane) - 1u))) & (kQueue - 1)] =
                            (unsigned short)((cm << 5) | lane);
                        qn += __popc(hm);
                        if (qn >= 32) {
                            test_queued(has_shift, 32, ps);
                            qn -= 32;
                        }
                    }
                }
                if (qn > 0) {   // the batch's shift and positions end here
                    test_queued(has_shift, qn, ps);
                    qn = 0;
                }
            };
            while (true) {
                int bi = 0;
                if (lane == 0) {
                    bi = atomicAdd(&gnext[g], 1);
                    if (bi >= nbatch) {   // this group is done: the next one with batches left
                        volatile int* gv = gnext;
                        int ng = -1;
                        for (int j = 1; j < ngroups && ng < 0; ++j) {
                            const int gg = (g + j) % ngroups;
                            if (gv[gg] < nbatch) ng = gg;
                        }
                        bi = ng < 0 ? -1 : -2 - ng;
                    }
                }
                bi = __shfl_sync(kFull, bi, 0);
                if (bi == -1) break;
                if (bi < 0) {
                    g = -2 - bi;
                    continue;
                }
                if (g != loaded) {   // this group's homes (a lane without one meets no cluster)
                    loaded = g;
                    const int hi = g * 32 + lane;
                    float4 P = make_float4(qnan, qnan, qnan, qnan), Q = P;
                    p = kNoHome;
                    if (hi < nh) {
                        p = home_pos(hc + hi);
                        P = b.posA[p];
                        Q = b.velA[p];
                    }
                    hx[0] = P.x; hx[1] = P.y; hx[2] = P.z;
                    hv[0] = Q.x; hv[1] = Q.y; hv[2] = Q.z;
                    tag = __float_as_uint(P.w);
                    float lo[3], hi_[3];
                    swept_box<DIM>(hx, hv, dt, lo, hi_);
                    home_box(lo, hi_, hb);
                }
                const int be = batch[bi], r = be >> 18, cb0 = be & 0xfff, cb1 = cb0 + ((be >> 12) & 63) + 1;
                const float sh[3] = {rsh[r][0], rsh[r][1], rsh[r][2]};
                if (sh[0] != 0.f || sh[1] != 0.f || sh[2] != 0.f) scan_batch(std::true_type{}, cb0, cb1, sh);
                else scan_batch(std::false_type{}, cb0, cb1, sh);
            }
        }
        __syncthreads();   // the next home chunk rewrites the group boxes and counters
    }
    if (b.tile_tests) {   // one counter update per block, the blocks spread over kTestSlots counters
        if (lane == 0 && wtests) atomicAdd(&blk_tests, (unsigned long long)wtests);
        __syncthreads();
        if (tid == 0 && blk_tests) atomicAdd(&b.tile_tests[(blockIdx.x + blockIdx.y) % kTestSlots], blk_tests);
    }
}

// Instance of c-bin bc (instances own consecutive c-bin ranges) and the
// c-bin's coordinates in key order (x slowest).
template <int DIM>
__device__ __forceinline__ int cbin_of_block(const Bufs<float>& b, const Geo& geo, uint32_t bc, int c[3]) {
    int lo = 0, hi = b.n_inst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.inst[mid].bin_base <= bc) lo = mid;
        else hi = mid - 1;
    }
    uint32_t rel = bc - b.inst[lo].bin_base;
    c[2] = 0;
    if (DIM == 3) {
        c[2] = (int)(rel % (uint32_t)geo.n[2]);
        rel /= (uint32_t)geo.n[2];
    }
    c[1] = (int)(rel % (uint32_t)geo.n[1]);
    c[0] = (int)(rel / (uint32_t)geo.n[1]);
    return lo;
}

// The pruned tile search: one block per c-bin of the pruned instances (grid:
// every c-bin; the others' blocks return at once).  A kernel of its own, so
// that its registers are allocated apart from the plain tile search's.
template <int DIM, int CAPC>
__global__ void __launch_bounds__(kTileThreads, 4) tile_pruned_kernel(Bufs<float> b) {
    extern __shared__ __align__(32) unsigned char tile_smem[];
    __shared__ GeoT<float> G;
    __shared__ int inst_s, c_s[3];
    if (threadIdx.x == 0) {
        G.load(b.geo);
        int c[3];
        inst_s = cbin_of_block<DIM>(b, b.geo, blockIdx.x, c);
        c_s[0] = c[0];
        c_s[1] = c[1];
        c_s[2] = c[2];
    }
    __syncthreads();
    const InstDev& I = b.inst[inst_s];
    if (!I.prune) return;   // block-uniform
    const int c[3] = {c_s[0], c_s[1], c_s[2]};
    tile_search_pruned<DIM, CAPC>(b, G, I, inst_s, c, tile_smem);
}

// The plain tile search: one block per c-bin of the tiled instances whose
// search cells are the c-bins (grid: every c-bin, in key order inside each
// instance; other blocks return at once).
template <typename T, int DIM>
__global__ void __launch_bounds__(kTileThreads, sizeof(T) == 4 ? 4 : 1) tile_search_kernel(Bufs<T> b) {
    using V = typename Vec4<T>::type;
    extern __shared__ __align__(32) unsigned char tile_smem[];   // 2 x tile_cap vectors
    V* sp = reinterpret_cast<V*>(tile_smem);
    V* sv = sp + b.tile_cap;
    __shared__ GeoT<T> G;
    __shared__ int rq0[kTileRanges], rlen[kTileRanges], rpre[kTileRanges];
    __shared__ T rsh[kTileRanges][3];
    __shared__ int nr_s, tot_s, inst_s;
    __shared__ int64_t h0_s, h1_s;
    const uint32_t bc = blockIdx.x;
    if (threadIdx.x == 0) {
        G.load(b.geo);
        // instance of the c-bin (instances own consecutive c-bin ranges)
        int lo = 0, hi = b.n_inst - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (b.inst[mid].bin_base <= bc) lo = mid;
            else hi = mid - 1;
        }
        inst_s = lo;
    }
    __syncthreads();
    const InstDev& I = b.inst[inst_s];
    if (!I.tiled || I.prune) return;   // block-uniform
    // search cells are the c-bins: the c-bin's key (x slowest, as the c-bin order here)
    const uint32_t kc = I.key_base + (bc - I.bin_base);
    if (threadIdx.x == 0) {
        h0_s = min(b.start[kc], (uint32_t)b.n);
        h1_s = min(b.start[kc + 1], (uint32_t)b.n);
    }
    __syncthreads();
    if (h0_s >= h1_s) return;   // block-uniform
    bool amb = false;
    {
        // ambiguity of the periodic images is a property of the cell's window
        uint32_t rel = kc - I.key_base;
        int g[3] = {0, 0, 0};
        if (DIM == 3) {
            g[2] = (int)(rel % (uint32_t)I.M[2]);
            rel /= (uint32_t)I.M[2];
        }
        g[1] = (int)(rel % (uint32_t)I.M[1]);
        g[0] = (int)(rel / (uint32_t)I.M[1]);
        const int* kk = b.dyn[inst_s].k;
#pragma unroll
        for (int d = 0; d < DIM; ++d) amb = amb || window_1d(g[d], g[d], 1, I.M[d], kk[d], G.wall[d]).amb;
    }
    if (amb)
        tile_search_cell<T, DIM, true>(b, G, I, inst_s, kc, h0_s, h1_s, sp, sv, rq0, rlen, rpre, rsh, nr_s, tot_s);
    else
        tile_search_cell<T, DIM, false>(b, G, I, inst_s, kc, h0_s, h1_s, sp, sv, rq0, rlen, rpre, rsh, nr_s, tot_s);
}

// Direct search of one particle (global loads), used by the staged kernel for
// particles whose window it cannot serve from shared memory.
template <typename T, int DIM>
__device__ __noinline__ unsigned long long search_one_direct(const Bufs<T>& b, const GeoT<T>& G, int64_t p) {
    using V = typename Vec4<T>::type;
    const V P = b.posA[p];
    const V Q = b.velA[p];
    const int inst = tag_inst(b, R<T>::bits(P.w));
    const InstDev& I = b.inst[inst];
    const int* kk = b.dyn[inst].k;
    const T xi[3] = {P.x, P.y, P.z};
    const T vi[3] = {Q.x, Q.y, Q.z};
    const T dt = step_dt(b.dyn[inst], T()), R2 = inst_R2(I, T());
    int c[3] = {0, 0, 0}, g[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < DIM; ++d) cell_and_search<T>(xi[d], G.lo[d], G.inv[d], G.n[d], I.s[d], c[d], g[d]);
    Win w[3];
    bool amb = false;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        w[d] = window_1d(g[d], c[d], I.s[d], I.M[d], kk[d], G.wall[d]);
        amb = amb || w[d].amb;
    }
    T bd = R<T>::inf();
    uint32_t bid = 0xffffffffu;
    int32_t bq = -1;
    if (amb) scan_window<T, DIM, true>(b, G, I, w, xi, vi, dt, R2, bd, bid, bq);
    else scan_window<T, DIM, false>(b, G, I, w, xi, vi, dt, R2, bd, bid, bq);
    return bq >= 0 ? partner_key<T>(bd, bid) : kNoPartner;
}

// Staged search (3-D, sparse search cells).  A block owns a tile: tile_rows
// consecutive y-rows of one x-slab, i.e. one contiguous range of A.  Every
// row of the tile's neighbourhood (x-slabs of the window, y-rows of the
// union of the windows) is a contiguous range of A too; those rows and their
// search-cell offsets are copied to shared memory with coalesced loads, then
// each thread walks its own window there: same candidates, same test, same
// tie rule as the direct search, without dependent global loads.  A tile
// whose neighbourhood does not fit, or a particle whose window is not a plain
// unwrapped window, takes the direct path.
constexpr int kStageMaxRows = 64;
constexpr int kStageMaxHome = 2 * kStageThreads;

// Ranges [q0, q1) (shared-memory indices) of one home particle's window
// inside the staged rows; calls f(q0, q1) for each.  Returns false when the
// window is not a plain unwrapped window inside the staged union.
template <typename T, typename F>
__device__ __forceinline__ bool for_each_staged_range(const GeoT<T>& G, const InstDev& I, const int* kk,
                                                      const uint32_t* loc, int stride, int xlo, int nx, int ylo,
                                                      int ny, const T xi[3], F&& f) {
    int c[3], g[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) cell_and_search<T>(xi[d], G.lo[d], G.inv[d], G.n[d], I.s[d], c[d], g[d]);
    Win w[3];
    bool amb = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        w[d] = window_1d(g[d], c[d], I.s[d], I.M[d], kk[d], G.wall[d]);
        amb = amb || w[d].amb;
    }
    if (amb || w[0].lo < xlo || w[0].hi >= xlo + nx || w[1].lo < ylo || w[1].hi >= ylo + ny) return false;
    const int MZ = I.M[2];
    int fa0 = w[2].lo, fb0 = w[2].hi, fa1 = 1, fb1 = 0;
    if (w[2].lo < 0) { fa0 = w[2].lo + MZ; fb0 = MZ - 1; fa1 = 0; fb1 = w[2].hi; }
    else if (w[2].hi >= MZ) { fb0 = MZ - 1; fa1 = 0; fb1 = w[2].hi - MZ; }
    for (int tx = w[0].lo; tx <= w[0].hi; ++tx) {
        for (int ty = w[1].lo; ty <= w[1].hi; ++ty) {
            const uint32_t* lr = loc + ((tx - xlo) * ny + (ty - ylo)) * stride;
            f((int)lr[fa0], (int)lr[fb0 + 1]);
            if (fa1 <= fb1) f((int)lr[fa1], (int)lr[fb1 + 1]);
        }
    }
    return true;
}

// Pair-list search over the staged rows (binary32).  Phase A: every home
// particle writes its candidates as (home ordinal, staged index) entries at
// its offset of a block-wide exclusive scan.  Phase B: the block tests the
// entries round-robin, so every lane has work whatever the window sizes; a
// passing candidate lowers the home particle's 64-bit key (ordered d2, tag)
// with a shared-memory atomicMin, which keeps the smaller distance and, on a
// tie, the lower id.  Phase C: each home particle stores its key (the same
// format as the direct search).  Periodic images come from the
// per-candidate minimum image, equal to the row image inside these windows.
template <typename T>
__device__ __noinline__ void staged_pairs(const Bufs<T>& b, const GeoT<T>& G, const InstDev& I, const int* kk,
                                          const typename Vec4<T>::type* sp, const typename Vec4<T>::type* sv,
                                          unsigned char* scratch, const int32_t* rowA0, const int32_t* rowL0,
                                          int nr, int xlo, int nx, int ylo, int ny, int32_t h0, int32_t h1,
                                          int stride, T dt, T R2) {
    using V = typename Vec4<T>::type;
    __shared__ int s_total;
    __shared__ int s_warp[kStageThreads / 32];
    unsigned long long* bkey = reinterpret_cast<unsigned long long*>(scratch);
    int* hoff = reinterpret_cast<int*>(bkey + kStageMaxHome);            // [kStageMaxHome + 1]
    uint32_t* pairs = reinterpret_cast<uint32_t*>(hoff + kStageMaxHome + 1);
    const uint32_t* ltab = reinterpret_cast<const uint32_t*>(sv + b.stage_cap);
    const int tid = threadIdx.x;
    const int H = h1 - h0;
    // home particles sit contiguously in the staged rows, in A order, from
    // the staged row holding h0
    int hbase = 0;
    for (int r = 0; r < nr; ++r) {
        if (rowA0[r] <= h0 && h0 < rowA0[r] + (rowL0[r + 1] - rowL0[r])) {
            hbase = rowL0[r] + (h0 - rowA0[r]);
            break;
        }
    }
    const bool fits = H <= kStageMaxHome;
    // phase A1: candidate counts
    int cnt[2] = {0, 0};
    bool direct[2] = {!fits, !fits};
    if (fits) {
        for (int k = 0; k < 2; ++k) {
            const int i = tid + k * kStageThreads;
            if (i >= H) break;
            const V P = sp[hbase + i];
            const T xi[3] = {P.x, P.y, P.z};
            int c = 0;
            const bool ok = for_each_staged_range<T>(G, I, kk, ltab, stride, xlo, nx, ylo, ny, xi,
                                                     [&](int q0, int q1) { c += max(q1 - q0, 0); });
            cnt[k] = ok ? c : 0;
            direct[k] = !ok;
        }
    }
    // block exclusive scan of the per-thread totals
    int mine = cnt[0] + cnt[1];
    int inc = mine;
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = lane < kStageThreads / 32 ? s_warp[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < kStageThreads / 32) s_warp[lane] = wi - w;
        if (lane == kStageThreads / 32 - 1) s_total = wi;
    }
    __syncthreads();
    const int base = s_warp[warp] + inc - mine;
    const bool list_ok = fits && s_total <= b.stage_pair_cap;
    // phase A2: write the entries, reset the keys
    if (list_ok) {
        int off = base;
        for (int k = 0; k < 2; ++k) {
            const int i = tid + k * kStageThreads;
            if (i >= H) break;
            hoff[i] = off;
            bkey[i] = ~0ull;
            if (direct[k]) continue;
            const V P = sp[hbase + i];
            const T xi[3] = {P.x, P.y, P.z};
            const uint32_t hi16 = (uint32_t)i << 16;
            for_each_staged_range<T>(G, I, kk, ltab, stride, xlo, nx, ylo, ny, xi, [&](int q0, int q1) {
                for (int q = q0; q < q1; ++q) pairs[off++] = hi16 | (uint32_t)q;
            });
        }
        if (tid == 0) hoff[min(H, kStageMaxHome)] = s_total;
    }
    __syncthreads();
    if (!list_ok) {   // too many entries for the list: direct search for the whole tile
        for (int64_t p = h0 + tid; p < h1; p += blockDim.x) b.bkey[p] = search_one_direct<T, 3>(b, G, p);
        return;
    }
    // phase B: balanced pair tests
    const T sh0[3] = {(T)0, (T)0, (T)0};
    for (int t = tid; t < s_total; t += blockDim.x) {
        const uint32_t e = pairs[t];
        const int i = (int)(e >> 16);
        const int q = (int)(e & 0xffffu);
        const V Pi = sp[hbase + i], Qi = sv[hbase + i];
        const V Pj = sp[q], Qj = sv[q];
        const T xi[3] = {Pi.x, Pi.y, Pi.z}, vi[3] = {Qi.x, Qi.y, Qi.z};
        const T xj[3] = {Pj.x, Pj.y, Pj.z}, vj[3] = {Qj.x, Qj.y, Qj.z};
        T d2;
        if (poca_test_sh<T, 3, true>(G, xi, vi, xj, vj, sh0, dt, R2, d2)) {
            const unsigned long long key = ((unsigned long long)ordered_bits((float)d2) << 32) |
                                           (unsigned long long)R<T>::bits(Pj.w);
            atomicMin(&bkey[i], key);
        }
    }
    __syncthreads();
    // phase C: the keys to global memory
    for (int k = 0; k < 2; ++k) {
        const int i = tid + k * kStageThreads;
        if (i >= H) break;
        const int64_t p = h0 + i;
        if (direct[k]) {
            b.bkey[p] = search_one_direct<T, 3>(b, G, p);
            continue;
        }
        b.bkey[p] = bkey[i];
    }
}

template <typename T>
__global__ void __launch_bounds__(kStageThreads) search_staged_kernel(Bufs<T> b) {
    using V = typename Vec4<T>::type;
    extern __shared__ __align__(32) unsigned char smem[];
    V* sp = reinterpret_cast<V*>(smem);
    V* sv = sp + b.stage_cap;
    uint32_t* loc = reinterpret_cast<uint32_t*>(sv + b.stage_cap);
    __shared__ GeoT<T> G;
    __shared__ int s_inst, s_gx, s_y0, s_y1, s_xlo, s_nx, s_ylo, s_ny, s_ok;
    __shared__ int32_t s_h0, s_h1;
    __shared__ int32_t s_rowA0[kStageMaxRows];
    __shared__ int32_t s_rowL0[kStageMaxRows + 1];
    __shared__ uint32_t s_rowK[kStageMaxRows];
    const int tid = threadIdx.x;
    const uint32_t tile = blockIdx.x;
    if (tid == 0) {
        G.load(b.geo);
        int lo = 0, hi = b.n_inst - 1;   // last instance with tile_base <= tile
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (b.inst[mid].tile_base <= tile) lo = mid;
            else hi = mid - 1;
        }
        const InstDev& I = b.inst[lo];
        const uint32_t t = tile - I.tile_base;
        s_inst = lo;
        s_gx = (int)(t / (uint32_t)I.tiles_per_x);
        s_y0 = (int)(t % (uint32_t)I.tiles_per_x) * I.tile_rows;
        s_y1 = min(s_y0 + I.tile_rows, I.M[1]);
        const uint32_t Mz = (uint32_t)I.M[2], My = (uint32_t)I.M[1];
        const uint32_t k0 = I.key_base + ((uint32_t)s_gx * My + (uint32_t)s_y0) * Mz;
        const uint32_t k1 = I.key_base + ((uint32_t)s_gx * My + (uint32_t)s_y1) * Mz;
        s_h0 = (int32_t)min(b.start[k0], (uint32_t)b.n);
        s_h1 = (int32_t)min(b.start[k1], (uint32_t)b.n);
        const int* kk = b.dyn[lo].k;
        // x-slabs of the (common) x-window, union of the y-windows
        const Win wx = window_1d(s_gx, s_gx / I.s[0], I.s[0], I.M[0], kk[0], G.wall[0]);
        const Win wy0 = window_1d(s_y0, s_y0 / I.s[1], I.s[1], I.M[1], kk[1], G.wall[1]);
        const Win wy1 = window_1d(s_y1 - 1, (s_y1 - 1) / I.s[1], I.s[1], I.M[1], kk[1], G.wall[1]);
        s_xlo = wx.lo;
        s_nx = wx.hi - wx.lo + 1;
        s_ylo = wy0.lo;
        s_ny = wy1.hi - wy0.lo + 1;
        s_ok = !wx.amb && !wy0.amb && !wy1.amb && s_ny < I.M[1] && s_nx * s_ny <= min(b.stage_rows, kStageMaxRows);
    }
    __syncthreads();
    if (s_h0 >= s_h1) return;
    const InstDev& I = b.inst[s_inst];
    const uint32_t Mz = (uint32_t)I.M[2], My = (uint32_t)I.M[1];
    const int nr = s_nx * s_ny;
    if (s_ok) {
        // row ranges of A
        for (int r = tid; r < nr; r += blockDim.x) {
            T sh;
            const int gx = unwrap<T>(s_xlo + r / s_ny, I.M[0], G.L[0], sh);
            const int gy = unwrap<T>(s_ylo + r % s_ny, I.M[1], G.L[1], sh);
            const uint32_t rk = I.key_base + ((uint32_t)gx * My + (uint32_t)gy) * Mz;
            const int32_t a0 = (int32_t)min(b.start[rk], (uint32_t)b.n);
            const int32_t a1 = (int32_t)min(b.start[rk + Mz], (uint32_t)b.n);
            s_rowK[r] = rk;
            s_rowA0[r] = a0;
            s_rowL0[r + 1] = max(a1 - a0, 0);
        }
        __syncthreads();
        if (tid == 0) {
            s_rowL0[0] = 0;
            for (int r = 0; r < nr; ++r) s_rowL0[r + 1] += s_rowL0[r];
            if (s_rowL0[nr] > b.stage_cap) s_ok = 0;
        }
        __syncthreads();
    }
    if (!s_ok) {   // neighbourhood too large for this tile: direct search
        for (int64_t p = s_h0 + tid; p < s_h1; p += blockDim.x) b.bkey[p] = search_one_direct<T, 3>(b, G, p);
        return;
    }
    // copy the rows and their search-cell offsets: one warp per row, lanes
    // along the row (coalesced)
    const int stride = b.stage_stride;
    const int lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    for (int r = warp; r < nr; r += nwarps) {
        const int32_t a0 = s_rowA0[r], l0 = s_rowL0[r], cnt = s_rowL0[r + 1] - l0;
        for (int t = lane; t < cnt; t += 32) {
            sp[l0 + t] = ldg_vec(b.posA + a0 + t);
            sv[l0 + t] = ldg_vec(b.velA + a0 + t);
        }
        const uint32_t rk = s_rowK[r];
        uint32_t* lr = loc + r * stride;
        for (int z = lane; z <= (int)Mz; z += 32) {
            const int32_t a = (int32_t)min(b.start[rk + (uint32_t)z], (uint32_t)b.n);
            lr[z] = (uint32_t)(l0 + (a - a0));
        }
    }
    __syncthreads();

    const int* kk = b.dyn[s_inst].k;
    const T dt = step_dt(b.dyn[s_inst], T()), R2 = inst_R2(I, T());
    if constexpr (sizeof(T) == 4) {
        staged_pairs(b, G, I, kk, sp, sv, reinterpret_cast<unsigned char*>(loc + (size_t)b.stage_rows * stride),
                     s_rowA0, s_rowL0, nr, s_xlo, s_nx, s_ylo, s_ny, s_h0, s_h1, stride, dt, R2);
    } else {
        for (int64_t p = s_h0 + tid; p < s_h1; p += blockDim.x) {
            const V P = b.posA[p];
            const V Q = b.velA[p];
            const T xi[3] = {P.x, P.y, P.z};
            const T vi[3] = {Q.x, Q.y, Q.z};
            int c[3], g[3];
    #pragma unroll
            for (int d = 0; d < 3; ++d) cell_and_search<T>(xi[d], G.lo[d], G.inv[d], G.n[d], I.s[d], c[d], g[d]);
            Win w[3];
            bool amb = false;
    #pragma unroll
            for (int d = 0; d < 3; ++d) {
                w[d] = window_1d(g[d], c[d], I.s[d], I.M[d], kk[d], G.wall[d]);
                amb = amb || w[d].amb;
            }
            if (amb || w[0].lo < s_xlo || w[0].hi >= s_xlo + s_nx || w[1].lo < s_ylo || w[1].hi >= s_ylo + s_ny) {
                b.bkey[p] = search_one_direct<T, 3>(b, G, p);
                continue;
            }
            // z parts of the window (z is the fastest key dimension)
            const int MZ = I.M[2];
            int fa[2], fb[2];
            T fs[2] = {(T)0, (T)0};
            int nf = 1;
            if (w[2].lo < 0) {
                fa[0] = w[2].lo + MZ; fb[0] = MZ - 1; fs[0] = G.L[2];
                fa[1] = 0; fb[1] = w[2].hi;
                nf = 2;
            } else if (w[2].hi >= MZ) {
                fa[0] = w[2].lo; fb[0] = MZ - 1;
                fa[1] = 0; fb[1] = w[2].hi - MZ; fs[1] = -G.L[2];
                nf = 2;
            } else {
                fa[0] = w[2].lo; fb[0] = w[2].hi;
            }
            T bd = R<T>::inf();
            uint32_t bid = 0xffffffffu;
            int32_t bq = -1;
            int tx = w[0].lo, ty = w[1].lo, part = 0;
            int32_t q = 0, qe = 0, off = 0;
            T sh[3] = {(T)0, (T)0, (T)0};
            for (;;) {
                if (q >= qe) {
                    bool more = false;
                    while (tx <= w[0].hi) {
                        T sx, sy;
                        unwrap<T>(tx, I.M[0], G.L[0], sx);
                        unwrap<T>(ty, I.M[1], G.L[1], sy);
                        const int r = (tx - s_xlo) * s_ny + (ty - s_ylo);
                        q = (int32_t)loc[r * stride + fa[part]];
                        qe = (int32_t)loc[r * stride + fb[part] + 1];
                        off = s_rowA0[r] - s_rowL0[r];
                        sh[0] = sx;
                        sh[1] = sy;
                        sh[2] = part == 0 ? fs[0] : fs[1];
                        if (++part == nf) {
                            part = 0;
                            if (++ty > w[1].hi) { ty = w[1].lo; ++tx; }
                        }
                        if (q < qe) { more = true; break; }
                    }
                    if (!more) break;
                }
                const V Pj = sp[q];
                const V Qj = sv[q];
                const T xj[3] = {Pj.x, Pj.y, Pj.z};
                const T vj[3] = {Qj.x, Qj.y, Qj.z};
                T d2;
                // the particle itself has v_rel = 0 and fails b > 0
                if (poca_test_sh<T, 3, false>(G, xi, vi, xj, vj, sh, dt, R2, d2)) {
                    const uint32_t idj = R<T>::bits(Pj.w);
                    if (d2 < bd || (d2 == bd && idj < bid)) {
                        bd = d2;
                        bid = idj;
                        bq = q + off;
                    }
                }
                ++q;
            }
            b.bkey[p] = bq >= 0 ? partner_key<T>(bd, bid) : kNoPartner;
        }
    }
}

// Unambiguous pairs, CM-frame scattering, split free flight, walls, then the
// next step's search key / slot / histogram.  The particle's collisional
// virial goes to vel.w for the moment pass.
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 8 : 1) move_kernel(Bufs<T> b) {
    using V = typename Vec4<T>::type;
    __shared__ GeoT<T> G;
    if (threadIdx.x == 0) G.load(b.geo);
    __syncthreads();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = p < b.n;
    V P = {}, Q = {};
    int inst = 0;
    unsigned long long kp = kNoPartner;
    if (valid) {
        P = b.posA[p];
        Q = b.velA[p];
        inst = tag_inst(b, R<T>::bits(P.w));
        kp = b.bkey[p];
    }
    const InstDev I = b.inst[inst];
    const uint32_t tag = R<T>::bits(P.w);   // ordering of tags = ordering of local ids
    const T x[3] = {P.x, P.y, P.z};
    const T v[3] = {Q.x, Q.y, Q.z};
    const T dt = step_dt(b.dyn[inst], T());
    T xn[3] = {x[0], x[1], x[2]}, vn[3] = {v[0], v[1], v[2]};
    T W = (T)0;
    bool paired = false;
    bool gone = valid && absorbed(Q.w);   // absorbed in an earlier step: stays as it is
    uint32_t tagj = 0xffffffffu;
    int64_t j = -1;
    V Pj = {}, Qj = {};
    if (kp != kNoPartner) {
        tagj = (uint32_t)kp;
        const int64_t lid = (int64_t)tag_id(b, tagj);
        // A candidate of another instance, or a position outside A, comes only
        // from a step whose sort failed (flagged as KMC_ETIMEOUT): slot_of then
        // still holds the scatter's tags for some ids.  Both are skipped.
        if (tag_inst(b, tagj) == inst && lid < I.n) {
            j = b.slot_of[I.p_off + lid];
            if (j >= b.n) j = -1;
        }
    }
    if (j >= 0) {
        // the candidate's key and state in one round trip; the state is used if the pair is mutual
        const unsigned long long kj = b.bkey[j];
        Pj = b.posA[j];
        Qj = b.velA[j];
        paired = kj != kNoPartner && (uint32_t)kj == tag;
    }
    if (paired) {
        const T xj[3] = {Pj.x, Pj.y, Pj.z};
        const T vj[3] = {Qj.x, Qj.y, Qj.z};
        T dr[3] = {0, 0, 0}, dv[3];
#pragma unroll
        for (int d = 0; d < DIM; ++d) dr[d] = min_image<T>(R<T>::sub(x[d], xj[d]), G.hL[d], G.L[d]);
#pragma unroll
        for (int d = 0; d < 3; ++d) dv[d] = R<T>::sub(v[d], vj[d]);
        T a = R<T>::mul(dr[0], dv[0]);
        a = R<T>::fma(dr[1], dv[1], a);
        T bb = R<T>::mul(dv[0], dv[0]);
        bb = R<T>::fma(dv[1], dv[1], bb);
        if (DIM == 3) {
            a = R<T>::fma(dr[2], dv[2], a);
            bb = R<T>::fma(dv[2], dv[2], bb);
        }
        const T b3 = (DIM == 3) ? bb : R<T>::fma(dv[2], dv[2], bb);
        const T tp = R<T>::div(-a, bb);                         // Eq. 12
        const uint32_t lo_id = tag_id(b, tag < tagj ? tag : tagj);
        const T sgn = tag < tagj ? (T)1 : (T)-1;
        const uint4 rnd = philox4x32_10(make_uint4(lo_id, b.st->step, 0u, 0u), I.seed_lo, I.seed_hi);
        T u1, u2;
        uniforms<T>(rnd, u1, u2);
        const T cth = (T)1 - (T)2 * u1;
        const T sth = (T)2 * R<T>::sqrt_(u1 * ((T)1 - u1));
        T sphi, cphi;
        sincos_2pi(u2, &sphi, &cphi);
        // isotropic opposite directions: on the sphere, or in the plane for 2-D velocities
        const T nh[3] = {G.vdim == 2 ? cphi : sth * cphi, G.vdim == 2 ? sphi : sth * sphi,
                         G.vdim == 2 ? (T)0 : cth};
        const T h = (T)0.5 * R<T>::sqrt_(b3);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const T vcm = (T)0.5 * (v[d] + vj[d]);
            vn[d] = vcm + sgn * (h * nh[d]);
        }
        const T rest = R<T>::sub(dt, tp);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            xn[d] = R<T>::add(R<T>::add(x[d], R<T>::mul(v[d], tp)), R<T>::mul(vn[d], rest));  // Eq. 13
            W += (dr[d] + dv[d] * tp) * (vn[d] - v[d]);
        }
    } else if (!gone) {
#pragma unroll
        for (int d = 0; d < DIM; ++d) xn[d] = R<T>::add(x[d], R<T>::mul(v[d], dt));  // Eq. 14
    }
    // absorbing walls (the particle leaves the simulation), reflective walls
    // (fold) and periodic wrap
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        const T lo = G.lo[d], hi = G.hi[d];
        if (G.absorb[d]) {
            if (xn[d] < lo || xn[d] > hi) gone = true;
        } else if (G.wall[d]) {
            for (int it = 0; it < kFoldCap && (xn[d] < lo || xn[d] > hi); ++it) {
                xn[d] = (xn[d] < lo) ? R<T>::sub((T)2 * lo, xn[d]) : R<T>::sub((T)2 * hi, xn[d]);
                vn[d] = -vn[d];
            }
            if (xn[d] < lo) xn[d] = lo;
            if (xn[d] > hi) xn[d] = hi;
        } else {
            const T L = G.L[d];
            if (xn[d] >= hi) xn[d] = R<T>::sub(xn[d], L);
            else if (xn[d] < lo) xn[d] = R<T>::add(xn[d], L);
            if (xn[d] < lo || xn[d] >= hi) {
                const T f = floor(R<T>::div(R<T>::sub(xn[d], lo), L));
                xn[d] = R<T>::sub(R<T>::add(lo, R<T>::sub(xn[d], lo)), R<T>::mul(L, f));
            }
            if (xn[d] >= hi) xn[d] = lo;
        }
    }
    uint32_t skey = 0, bin = 0;
    keys_of<T, DIM>(G, I, xn, skey, bin);
    if (gone) skey = b.n_keys;   // absorbed: the key after every cell
    const unsigned active = __ballot_sync(kFull, valid);
    if (valid) {
        const uint32_t slot = aggregated_increment(b.count, skey, active);
        V Pn, Qn;
        Pn.x = xn[0]; Pn.y = xn[1]; Pn.z = xn[2]; Pn.w = P.w;
        Qn.x = vn[0]; Qn.y = vn[1]; Qn.z = vn[2];
        // W of the step (+inf: no collision); the random-partner variant marked its
        // collided particles with 0 (point collisions carry no virial)
        const bool hit = paired || (b.dsmc && Q.w == (T)0);
        Qn.w = gone ? -R<T>::inf() : (hit ? W : R<T>::inf());
        b.posB[p] = Pn;
        b.velB[p] = Qn;
        b.key[p] = skey;
        b.slot[p] = slot;
        b.tagB[p] = tag;
        if (b.record) {
            const int64_t gid = I.p_off + (int64_t)tag_id(b, tag);
            b.rec_best[gid] = (kp != kNoPartner) ? (int32_t)tag_id(b, tagj) : -1;
            b.rec_partner[gid] = paired ? (int32_t)tag_id(b, tagj) : -1;
        }
    }
    (void)bin;
    warp_vmax<T>(b.dyn, valid && !gone, inst, speed2<T>(vn[0], vn[1], vn[2]));
}

// Counting-sort scatter B -> A in canonical order: search key, then particle
// tag (instance, then id) inside a search cell.  The histogram atomics of the
// move kernel gave every particle an arbitrary rank inside its cell (slot);
// pass 1 writes the tag of every particle that shares its cell at that rank,
// pass 2 counts the cell's tags below its own, which is its rank in id order,
// and moves the particle there.  A cell of more than kCanonMax particles keeps
// the atomic order (the count is quadratic in the cell's size), and so do the
// absorbed particles collected after the last cell.  The tags go to slot_of,
// which is free between the move and the next search.
// The tag pass takes kScatterItems particles per thread, a block's items apart
// (coalesced), with every item's loads issued before any is used: a particle
// costs two dependent round trips (its key, then its cell's range), so a
// thread keeps several in flight.  The moving pass (one particle per thread)
// issues its state loads first.
constexpr int kScatterItems = 4;

template <typename T>
__global__ void __launch_bounds__(kThreads) scatter_tags_kernel(Bufs<T> b) {
    const int64_t p0 = (int64_t)blockIdx.x * blockDim.x * kScatterItems + threadIdx.x;
    uint32_t k[kScatterItems], s0[kScatterItems], s1[kScatterItems];
#pragma unroll
    for (int i = 0; i < kScatterItems; ++i) {
        const int64_t p = p0 + (int64_t)i * blockDim.x;
        k[i] = p < b.n ? b.key[p] : b.n_keys;
    }
#pragma unroll
    for (int i = 0; i < kScatterItems; ++i) {
        s0[i] = s1[i] = 0u;
        if (k[i] < b.n_keys) {
            s0[i] = b.start[k[i]];
            s1[i] = b.start[k[i] + 1];
        }
    }
#pragma unroll
    for (int i = 0; i < kScatterItems; ++i) {
        const int64_t p = p0 + (int64_t)i * blockDim.x;
        // alone in its cell (most cells of a fine grid), or outside every cell
        if (s1[i] <= s0[i] + 1u || s1[i] - s0[i] > kCanonMax) continue;
        const uint32_t dst = s0[i] + b.slot[p];
        if (dst >= s1[i] || dst >= (uint32_t)b.n) continue;   // only after a failed scan (flagged by the scatter)
        b.slot_of[dst] = b.tagB[p];
    }
}

// Tags of [q, q1) below `tag`: scalar up to a 16-byte boundary, then four per load.
__device__ __forceinline__ uint32_t tags_below(const uint32_t* __restrict__ t, uint32_t q, uint32_t q1,
                                               uint32_t tag) {
    uint32_t r = 0;
    for (; q < q1 && (q & 3u); ++q) r += t[q] < tag ? 1u : 0u;
    const uint4* t4 = reinterpret_cast<const uint4*>(t + q);
    const uint32_t n4 = (q1 - q) >> 2;
#pragma unroll 4
    for (uint32_t i = 0; i < n4; ++i) {
        const uint4 v = t4[i];
        r += (v.x < tag ? 1u : 0u) + (v.y < tag ? 1u : 0u) + (v.z < tag ? 1u : 0u) + (v.w < tag ? 1u : 0u);
    }
    for (q += n4 << 2; q < q1; ++q) r += t[q] < tag ? 1u : 0u;
    return r;
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 8) scatter_kernel(Bufs<T> b) {
    using V = typename Vec4<T>::type;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= b.n) return;
    // the particle's own words and state first (independent loads), then its cell's range
    const uint32_t k = b.key[p], slot = b.slot[p], tag = b.tagB[p];
    const V P = b.posB[p], Q = b.velB[p];
    const uint32_t s0 = b.start[k];
    const uint32_t s1 = k < b.n_keys ? b.start[k + 1] : s0;
    uint32_t rank = slot;
    if (s1 > s0 + 1u && s1 - s0 <= kCanonMax && s1 <= (uint32_t)b.n) rank = tags_below(b.slot_of, s0, s1, tag);
    const uint32_t dst = s0 + rank;
    if (dst >= (uint32_t)b.n) {  // only after a failed scan; reported as a device error
        atomicOr(&b.st->error, kErrKeyRange);
        return;
    }
    b.posA[dst] = P;
    b.velA[dst] = Q;
    b.bkey[dst] = kNoPartner;   // the next search starts from no partner
}

// Index (position in the input arrays, p_off + local id) of every particle of
// A, in sorted order: the sort permutation.
template <typename T>
__global__ void __launch_bounds__(kThreads) perm_kernel(Bufs<T> b, int32_t* __restrict__ perm) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= b.n) return;
    const uint32_t tag = R<T>::bits(b.posA[p].w);
    perm[p] = (int32_t)(b.inst[tag_inst(b, tag)].p_off + (int64_t)tag_id(b, tag));
}

// ------------------------------------------------------------ DSMC variant
// The classic random-partner collisions the paper contrasts with PoCA (Sect.
// "Direct Simulation Monte Carlo Technique"), in Bird's no-time-counter form:
// collision cells are the c-bins (the search grid of a DSMC handle is the
// c-bins, so a cell is one contiguous range of A, its particles in id order).
// Per cell of N >= 2 particles: M = floor(1/2 N (N - 1) sigma g_max dt / V_c
// + u_0) candidate pairs, sigma = pi R^2 (Eq. 7), g_max = 2 v_max; candidate k
// takes positions i != j of the cell from Philox (cell, step, k, kDsmcPairTag)
// and is accepted when u g_max < g = |v_i - v_j|; an accepted pair scatters
// isotropically in its CM frame with the direction from (cell, step, k,
// kDsmcDirTag).  Candidates are applied one after another by one thread per
// cell; arithmetic in binary64 in a fixed order, new velocities stored in the
// state precision after every collision, collided particles marked with
// vel.w = 0 for the move and the moments.
constexpr uint32_t kDsmcPairTag = 0x44534D43u;
constexpr uint32_t kDsmcDirTag = 0x44534D44u;

__device__ __forceinline__ double uniform53(uint32_t hi, uint32_t lo) {
    const unsigned long long m = ((unsigned long long)hi << 20) | (unsigned long long)(lo >> 12);
    return (double)(2ull * m + 1ull) * 0x1p-53;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) dsmc_kernel(Bufs<T> b) {
    using V = typename Vec4<T>::type;
    const int64_t kc64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (kc64 >= (int64_t)b.n_keys) return;
    const uint32_t kc = (uint32_t)kc64;
    const uint32_t nmax = (uint32_t)b.n;
    const uint32_t s0 = min(b.start[kc], nmax), s1 = min(b.start[kc + 1], nmax);
    if (s1 <= s0) return;
    for (uint32_t q = s0; q < s1; ++q) b.velA[q].w = R<T>::inf();   // not collided (yet)
    const uint32_t N = s1 - s0;
    if (N < 2) return;
    int lo = 0, hi = b.n_inst - 1;   // instance of the cell (consecutive key ranges)
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.inst[mid].key_base <= kc) lo = mid;
        else hi = mid - 1;
    }
    const InstDev& I = b.inst[lo];
    const InstDyn& D = b.dyn[lo];
    const uint32_t cell = kc - I.key_base;
    const uint32_t step = b.st->step;
    const double gmax = __dmul_rn(2.0, __dsqrt_rn(__longlong_as_double((long long)D.vmax2_cur)));
    const double sigma = __dmul_rn(M_PI, I.R2);
    double Vc = 1.0;
    for (int d = 0; d < b.geo.dim; ++d) Vc = __dmul_rn(Vc, __ddiv_rn(b.geo.L[d], (double)b.geo.n[d]));
    const double Nd = (double)N;
    double m = __dmul_rn(__dmul_rn(0.5, Nd), __dsub_rn(Nd, 1.0));
    m = __ddiv_rn(__dmul_rn(__dmul_rn(__dmul_rn(m, sigma), gmax), D.dt), Vc);
    uint4 w = philox4x32_10(make_uint4(cell, step, 0xFFFFFFFFu, kDsmcPairTag), I.seed_lo, I.seed_hi);
    m = floor(__dadd_rn(m, uniform53(w.x, w.y)));
    const uint32_t M = m > 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)m;
    V* vel = b.velA + s0;
    for (uint32_t k = 0; k < M; ++k) {
        w = philox4x32_10(make_uint4(cell, step, k, kDsmcPairTag), I.seed_lo, I.seed_hi);
        const uint32_t pi = (uint32_t)(((unsigned long long)w.x * (unsigned long long)N) >> 32);
        uint32_t pj = (uint32_t)(((unsigned long long)w.y * (unsigned long long)(N - 1u)) >> 32);
        if (pj >= pi) pj += 1u;
        V A = vel[pi], B = vel[pj];
        const double va[3] = {(double)A.x, (double)A.y, (double)A.z};
        const double vb[3] = {(double)B.x, (double)B.y, (double)B.z};
        const double d0 = __dsub_rn(va[0], vb[0]), d1 = __dsub_rn(va[1], vb[1]), d2 = __dsub_rn(va[2], vb[2]);
        const double g = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2)));
        if (!(__dmul_rn(uniform53(w.z, w.w), gmax) < g)) continue;
        w = philox4x32_10(make_uint4(cell, step, k, kDsmcDirTag), I.seed_lo, I.seed_hi);
        const double u1 = uniform53(w.x, w.y), u2 = uniform53(w.z, w.w);
        double sphi, cphi;
        sincospi(__dmul_rn(2.0, u2), &sphi, &cphi);
        const double cth = __dsub_rn(1.0, __dmul_rn(2.0, u1));
        const double sth = __dmul_rn(2.0, __dsqrt_rn(__dmul_rn(u1, __dsub_rn(1.0, u1))));
        const bool plane = b.geo.vdim == 2;
        const double nh[3] = {plane ? cphi : __dmul_rn(sth, cphi), plane ? sphi : __dmul_rn(sth, sphi),
                              plane ? 0.0 : cth};
        const double h = __dmul_rn(0.5, g);
        double na[3], nb[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double vcm = __dmul_rn(0.5, __dadd_rn(va[d], vb[d]));
            const double t = __dmul_rn(h, nh[d]);
            na[d] = __dadd_rn(vcm, t);
            nb[d] = __dsub_rn(vcm, t);
        }
        A.x = (T)na[0]; A.y = (T)na[1]; A.z = (T)na[2]; A.w = (T)0;
        B.x = (T)nb[0]; B.y = (T)nb[1]; B.z = (T)nb[2]; B.w = (T)0;
        vel[pi] = A;
        vel[pj] = B;
    }
}

// State of A in id order.
template <typename T>
__global__ void __launch_bounds__(kThreads) gather_kernel(Bufs<T> b, T* __restrict__ pos3, T* __restrict__ vel3) {
    using V = typename Vec4<T>::type;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= b.n) return;
    const V P = b.posA[p];
    const V Q = b.velA[p];
    const int inst = tag_inst(b, R<T>::bits(P.w));
    const int64_t gid = b.inst[inst].p_off + (int64_t)tag_id(b, R<T>::bits(P.w));
    const bool gone = absorbed(Q.w);   // absorbed by a wall: NaN position and velocity
    const T nan = R<T>::qnan();
    if (pos3) {
        pos3[3 * gid] = gone ? nan : P.x;
        pos3[3 * gid + 1] = gone ? nan : P.y;
        pos3[3 * gid + 2] = gone ? nan : P.z;
    }
    if (vel3) {
        vel3[3 * gid] = gone ? nan : Q.x;
        vel3[3 * gid + 1] = gone ? nan : Q.y;
        vel3[3 * gid + 2] = gone ? nan : Q.z;
    }
}

// c-bin key (instance-local) of every particle of A, id order.
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) cellkey_kernel(Bufs<T> b, int32_t* __restrict__ keys) {
    using V = typename Vec4<T>::type;
    __shared__ GeoT<T> G;
    if (threadIdx.x == 0) G.load(b.geo);
    __syncthreads();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= b.n) return;
    const V P = b.posA[p];
    const V Q = b.velA[p];
    const int inst = tag_inst(b, R<T>::bits(P.w));
    const InstDev& I = b.inst[inst];
    const T x[3] = {P.x, P.y, P.z};
    uint32_t skey, bin;
    keys_of<T, DIM>(G, I, x, skey, bin);
    keys[I.p_off + (int64_t)tag_id(b, R<T>::bits(P.w))] = absorbed(Q.w) ? -1 : (int32_t)(bin - I.bin_base);
}

// Moment sums per c-bin of the sorted state A (Eqs. vel_b, stress, 18, 19):
// N, Sum v, Sum v^2, Sum W and the collided count, in fixed point (see
// block_moment_partials).  Each thread reduces kMomItems consecutive particles
// (consecutive particles of A share a c-bin almost always), then warp and
// block aggregation.  use_virial = 0 ignores vel.w (state not produced by a step).
template <typename T, int DIM, bool RADIAL>
__global__ void __launch_bounds__(kThreads) moments_kernel(Bufs<T> b, int use_virial) {
    using V = typename Vec4<T>::type;
    __shared__ GeoT<T> G;
    __shared__ MomentSlots S;
    if (threadIdx.x == 0) {
        G.load(b.geo);
        S.n = 0;
    }
    __syncthreads();
    const int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kMomItems;
    uint32_t cur = 0xffffffffu;
    long long f[kMomSums] = {0, 0, 0, 0, 0, 0, 0, 0};
    int cnt = 0, coll = 0;
    V Ps[kMomItems], Qs[kMomItems];   // all loads in flight before the sums
#pragma unroll
    for (int k = 0; k < kMomItems; ++k) {
        if (base + k < b.n) {
            Ps[k] = b.posA[base + k];
            Qs[k] = b.velA[base + k];
        }
    }
    int inst_c = -1;
    uint32_t bin_base = 0;
    T sv = (T)0, s2 = (T)0, sw = (T)0;   // 2^e of the instance's three fields
#pragma unroll
    for (int k = 0; k < kMomItems; ++k) {
        const int64_t p = base + k;
        if (p >= b.n) break;
        const V P = Ps[k];
        const V Q = Qs[k];
        if (absorbed(Q.w)) continue;   // left through an absorbing wall
        const int inst = tag_inst(b, R<T>::bits(P.w));
        if (inst != inst_c) {   // the instance's constants, once per run of one instance
            inst_c = inst;
            bin_base = b.inst[inst].bin_base;
            sv = pow2_of(b.dyn[inst].mom_e[0], T());
            s2 = pow2_of(b.dyn[inst].mom_e[1], T());
            sw = pow2_of(b.dyn[inst].mom_e[2], T());
        }
        const T x[3] = {P.x, P.y, P.z};
        // the c-bin (the search cell is not needed here)
        int c[3] = {0, 0, 0}, g[3];
#pragma unroll
        for (int d = 0; d < DIM; ++d) cell_and_search<T>(x[d], G.lo[d], G.inv[d], G.n[d], 1, c[d], g[d]);
        const uint32_t bin = bin_base + (uint32_t)c[0] +
                             (uint32_t)G.n[0] * ((uint32_t)c[1] + (DIM == 3 ? (uint32_t)G.n[1] * (uint32_t)c[2] : 0u));
        if (bin != cur && cnt > 0) {   // rare: the thread's particles span two bins
            unsigned long long* a = b.acc + (size_t)cur * kAccFields;
            atomicAdd(a + 0, (unsigned long long)cnt);
#pragma unroll
            for (int q = 0; q < kMomSums; ++q) atomicAdd(a + acc_field(q), (unsigned long long)f[q]);
            if (coll) atomicAdd(a + 8, (unsigned long long)coll);
#pragma unroll
            for (int q = 0; q < kMomSums; ++q) f[q] = 0ll;
            cnt = coll = 0;
        }
        cur = bin;
        const bool collided = use_virial && Q.w != R<T>::inf();
        f[0] += fixed_of(Q.x, sv); f[1] += fixed_of(Q.y, sv); f[2] += fixed_of(Q.z, sv);
        f[3] += fixed_of(Q.x * Q.x, s2); f[4] += fixed_of(Q.y * Q.y, s2); f[5] += fixed_of(Q.z * Q.z, s2);
        if (collided) f[6] += fixed_of(Q.w, sw);
        // radial velocity (Eq. vel_r): v . r_hat, r_hat from the configured centre
        // over the position dimensions (0 at the centre itself); |v . r_hat| <= v_max
        if (RADIAL) {
            const T v3[3] = {Q.x, Q.y, Q.z};
            T r2 = (T)0, vd = (T)0;
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                const T dx = x[d] - G.rc[d];
                r2 += dx * dx;
                vd += v3[d] * dx;
            }
            if (r2 > (T)0) f[7] += fixed_of(vd / R<T>::sqrt_(r2), sv);
        }
        cnt += 1;
        coll += collided ? 1 : 0;
    }
    block_moment_partials(S, b.acc, cnt > 0, cur, f, cnt, coll);
}

// The same sums where every c-bin of every instance is at most kCbinRows runs
// of consecutive search cells (the search cells are the c-bins or their
// halves): one warp per c-bin reads its runs of the sorted state A and stores
// its sums, with no atomics (fixed-point sums do not depend on their order).
template <typename T, int DIM, bool RADIAL>
__global__ void __launch_bounds__(kThreads) moments_cbin_kernel(Bufs<T> b, int use_virial) {
    using V = typename Vec4<T>::type;
    __shared__ GeoT<T> G;
    if (threadIdx.x == 0) G.load(b.geo);
    __syncthreads();
    const int64_t bc = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    if (bc >= b.n_bins) return;   // warp-uniform
    const int lane = (int)lane_id();
    int inst = 0;
    {
        int hi = b.n_inst - 1;
        while (inst < hi) {
            const int mid = (inst + hi + 1) >> 1;
            if ((int64_t)b.inst[mid].bin_base <= bc) inst = mid;
            else hi = mid - 1;
        }
    }
    const InstDev& I = b.inst[inst];
    // c-bin coordinates in moment order (x fastest)
    uint32_t rel = (uint32_t)(bc - I.bin_base);
    const int cx = (int)(rel % (uint32_t)G.n[0]);
    rel /= (uint32_t)G.n[0];
    const int cy = DIM == 3 ? (int)(rel % (uint32_t)G.n[1]) : (int)rel;
    const int cz = DIM == 3 ? (int)(rel / (uint32_t)G.n[1]) : 0;
    const T sv = pow2_of(b.dyn[inst].mom_e[0], T()), s2 = pow2_of(b.dyn[inst].mom_e[1], T());
    const T sw = pow2_of(b.dyn[inst].mom_e[2], T());
    long long f[kMomSums] = {0, 0, 0, 0, 0, 0, 0, 0};
    int cnt = 0, coll = 0;
    // rows of search cells inside the c-bin: (x, y) in 3-D, x in 2-D; each row's
    // cells along the fast dimension are consecutive keys.  Lane r < rows reads
    // row r's range, then the lanes stride over the rows' particles together.
    const int rows = DIM == 3 ? I.s[0] * I.s[1] : I.s[0];
    const int sf = DIM == 3 ? I.s[2] : I.s[1];
    uint32_t r0 = 0, rl = 0;
    if (lane < rows) {
        const int gx = cx * I.s[0] + (DIM == 3 ? lane / I.s[1] : lane);
        uint32_t key;
        if (DIM == 3)
            key = I.key_base + ((uint32_t)gx * (uint32_t)I.M[1] + (uint32_t)(cy * I.s[1] + lane % I.s[1])) *
                                   (uint32_t)I.M[2] + (uint32_t)(cz * sf);
        else
            key = I.key_base + (uint32_t)gx * (uint32_t)I.M[1] + (uint32_t)(cy * sf);
        r0 = min(b.start[key], (uint32_t)b.n);
        rl = min(b.start[key + (uint32_t)sf], (uint32_t)b.n) - r0;
    }
    uint32_t rs[kCbinRows], re[kCbinRows];   // row r: particles [rs, re) of the c-bin's concatenation
    uint32_t base[kCbinRows];
    uint32_t total = 0;
#pragma unroll
    for (int r = 0; r < kCbinRows; ++r) {
        base[r] = __shfl_sync(kFull, r0, r);
        rs[r] = total;
        total += r < rows ? __shfl_sync(kFull, rl, r) : 0u;
        re[r] = total;
    }
    auto pos_of = [&](uint32_t i) -> int64_t {   // sorted position of the c-bin's particle i
        int64_t p = 0;
#pragma unroll
        for (int r = 0; r < kCbinRows; ++r)
            if (i >= rs[r] && i < re[r]) p = (int64_t)base[r] + (i - rs[r]);
        return p;
    };
    auto add = [&](const V& P, const V& Q) {
        const bool collided = use_virial && Q.w != R<T>::inf();
        f[0] += fixed_of(Q.x, sv); f[1] += fixed_of(Q.y, sv); f[2] += fixed_of(Q.z, sv);
        f[3] += fixed_of(Q.x * Q.x, s2); f[4] += fixed_of(Q.y * Q.y, s2); f[5] += fixed_of(Q.z * Q.z, s2);
        if (collided) f[6] += fixed_of(Q.w, sw);
        if (RADIAL) {   // Eq. vel_r, as in moments_kernel
            const T x[3] = {P.x, P.y, P.z};
            const T v3[3] = {Q.x, Q.y, Q.z};
            T r2 = (T)0, vd = (T)0;
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                const T dx = x[d] - G.rc[d];
                r2 += dx * dx;
                vd += v3[d] * dx;
            }
            if (r2 > (T)0) f[7] += fixed_of(vd / R<T>::sqrt_(r2), sv);
        }
        cnt += 1;
        coll += collided ? 1 : 0;
    };
    for (uint32_t i = lane; i < total; i += 64) {   // two particles per lane with their loads in flight
        const bool two = i + 32 < total;
        const int64_t p0 = pos_of(i), p1 = two ? pos_of(i + 32) : p0;
        const V P0 = b.posA[p0], Q0 = b.velA[p0];
        V P1 = P0, Q1 = Q0;
        if (two) {
            P1 = b.posA[p1];
            Q1 = b.velA[p1];
        }
        add(P0, Q0);
        if (two) add(P1, Q1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < kMomSums; ++k) f[k] += __shfl_xor_sync(kFull, f[k], o);
    }
    cnt = (int)__reduce_add_sync(kFull, (unsigned)cnt);
    coll = (int)__reduce_add_sync(kFull, (unsigned)coll);
    if (lane == 0) {
        unsigned long long* a = b.acc + (size_t)bc * kAccFields;
        a[0] = (unsigned long long)cnt;
#pragma unroll
        for (int k = 0; k < kMomSums; ++k) a[acc_field(k)] = (unsigned long long)f[k];
        a[8] = (unsigned long long)coll;
    }
}

// Candidates each particle of A examines (the sizes of its search window), summed
// over the particles: a diagnostic for the arithmetic roofline of the search.
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) window_count_kernel(Bufs<T> b, unsigned long long* total) {
    using V = typename Vec4<T>::type;
    __shared__ GeoT<T> G;
    if (threadIdx.x == 0) G.load(b.geo);
    __syncthreads();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long cnt = 0;
    if (p < b.n && !absorbed(b.velA[p].w)) {
        const V P = b.posA[p];
        const int inst = tag_inst(b, R<T>::bits(P.w));
        const InstDev& I = b.inst[inst];
        const int* kk = b.dyn[inst].k;
        const T xi[3] = {P.x, P.y, P.z};
        int c[3] = {0, 0, 0}, g[3] = {0, 0, 0};
#pragma unroll
        for (int d = 0; d < DIM; ++d) cell_and_search<T>(xi[d], G.lo[d], G.inv[d], G.n[d], I.s[d], c[d], g[d]);
        Win w[3] = {{0, 0, false}, {0, 0, false}, {0, 0, false}};
#pragma unroll
        for (int d = 0; d < DIM; ++d) w[d] = window_1d(g[d], c[d], I.s[d], I.M[d], kk[d], G.wall[d]);
        constexpr int F = DIM - 1;
        const int MF = I.M[F];
        const uint32_t My = (DIM == 3) ? (uint32_t)I.M[1] : 1u, Mf = (uint32_t)MF;
        for (int tx = w[0].lo; tx <= w[0].hi; ++tx) {
            T s0;
            const int gx = unwrap<T>(tx, I.M[0], G.L[0], s0);
            for (int ty = (DIM == 3 ? w[1].lo : 0); ty <= (DIM == 3 ? w[1].hi : 0); ++ty) {
                T s1;
                const int gy = (DIM == 3) ? unwrap<T>(ty, I.M[1], G.L[1], s1) : 0;
                const uint32_t row = I.key_base + ((uint32_t)gx * My + (uint32_t)gy) * Mf;
                for (int tz = w[F].lo; tz <= w[F].hi; ++tz) {
                    T s2;
                    const int gz = unwrap<T>(tz, MF, G.L[F], s2);
                    cnt += b.start[row + (uint32_t)gz + 1u] - b.start[row + (uint32_t)gz];
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
    if (lane_id() == 0 && cnt) atomicAdd(total, cnt);
}

// Particles per c-bin and largest |v|^2 per instance of the packed state in B
// (statistics for the host's choice of search grid at init).
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) cbin_hist_kernel(Bufs<T> b, uint32_t* __restrict__ hist,
                                                             unsigned long long* vmax2) {
    using V = typename Vec4<T>::type;
    __shared__ GeoT<T> G;
    if (threadIdx.x == 0) G.load(b.geo);
    __syncthreads();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = p < b.n;
    V P = {}, Q = {};
    int inst = 0;
    if (valid) {
        P = b.posB[p];
        Q = b.velB[p];
        inst = tag_inst(b, R<T>::bits(P.w));
    }
    const InstDev I = b.inst[inst];
    const T x[3] = {P.x, P.y, P.z};
    uint32_t skey = 0, bin = 0;
    keys_of<T, DIM>(G, I, x, skey, bin);
    const bool live = valid && !absorbed(Q.w);
    const unsigned active = __ballot_sync(kFull, live);
    if (live) {
        const unsigned peers = __match_any_sync(active, bin);
        if ((int)lane_id() == __ffs(peers) - 1) atomicAdd(hist + bin, (uint32_t)__popc(peers));
    }
    const double v2 = (double)Q.x * Q.x + (double)Q.y * Q.y + (double)Q.z * Q.z;
    double m = live ? v2 : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(kFull, m, o));
    const int inst0 = __shfl_sync(kFull, inst, 0);
    const bool same = __all_sync(kFull, !valid || inst == inst0);
    if (same) {
        if (lane_id() == 0 && valid) atomicMax(vmax2 + inst0, (unsigned long long)__double_as_longlong(m));
    } else if (valid) {
        atomicMax(vmax2 + inst, (unsigned long long)__double_as_longlong(v2));
    }
}

// ------------------------------------------------------------- launchers
inline unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

#define KMC_DIM_DISPATCH(dim, KERNEL, ...)                                      \
    do {                                                                        \
        if ((dim) == 3) KERNEL<T, 3><<<blocks_for(b.n), kThreads, 0, s>>>(__VA_ARGS__); \
        else KERNEL<T, 2><<<blocks_for(b.n), kThreads, 0, s>>>(__VA_ARGS__);    \
    } while (0)

template <typename T>
cudaError_t launch_pack(const Bufs<T>& b, const T* pos3, const T* vel3, uint32_t* bad, cudaStream_t s) {
    if (b.n == 0) return cudaSuccess;
    KMC_DIM_DISPATCH(b.geo.dim, pack_kernel, b, pos3, vel3, bad);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bin_init(const Bufs<T>& b, cudaStream_t s) {
    if (b.n == 0) return cudaSuccess;
    KMC_DIM_DISPATCH(b.geo.dim, bin_kernel, b);
    return cudaGetLastError();
}

template <typename T>
size_t stage_smem_bytes(const Bufs<T>& b) {
    size_t bytes = (size_t)b.stage_cap * 2 * sizeof(typename Vec4<T>::type) +
                   (size_t)b.stage_rows * (size_t)b.stage_stride * sizeof(uint32_t);
    if (sizeof(T) == 4)   // pair list: keys, offsets, entries
        bytes += (size_t)kStageMaxHome * 8 + (size_t)(kStageMaxHome + 1) * 4 + (size_t)b.stage_pair_cap * 4;
    return bytes;
}

template <typename T>
cudaError_t launch_search(const Bufs<T>& b, cudaStream_t s) {
    if (b.n == 0) return cudaSuccess;
    if (b.n_stage_tiles > 0) {
        search_staged_kernel<T><<<b.n_stage_tiles, kStageThreads, stage_smem_bytes(b), s>>>(b);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // besides the direct search it records slot_of for the particles of every
    // instance that is not tiled (staged ones included)
    if (b.any_direct || b.n_stage_tiles > 0) KMC_DIM_DISPATCH(b.geo.dim, search_kernel, b);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tile_search(const Bufs<T>& b, cudaStream_t s) {
    if (b.n == 0 || !b.any_tiled || b.n_keys == 0) return cudaSuccess;
    const dim3 grid((unsigned)b.n_bins, sizeof(T) == 4 ? (unsigned)b.tile_split : 1u);   // split: binary32 only
    if (b.any_plain_tiled) {
        const size_t smem = tile_smem_bytes(b);
        if (b.geo.dim == 3) tile_search_kernel<T, 3><<<grid, b.tile_threads, smem, s>>>(b);
        else tile_search_kernel<T, 2><<<grid, b.tile_threads, smem, s>>>(b);
    }
    if constexpr (sizeof(T) == 4) {
        if (b.tile_prune) {
            const size_t smem = pruned_smem_bytes(b.tile_cap);
            const bool dflt = (b.tile_cap & ~15) == kPrunedCap && b.tile_threads == kTileThreads;
            if (b.geo.dim == 3) {
                if (dflt) tile_pruned_kernel<3, kPrunedCap><<<grid, b.tile_threads, smem, s>>>(b);
                else tile_pruned_kernel<3, 0><<<grid, b.tile_threads, smem, s>>>(b);
            } else {
                if (dflt) tile_pruned_kernel<2, kPrunedCap><<<grid, b.tile_threads, smem, s>>>(b);
                else tile_pruned_kernel<2, 0><<<grid, b.tile_threads, smem, s>>>(b);
            }
        }
    }
    return cudaGetLastError();
}

template <typename T>
size_t tile_smem_bytes(const Bufs<T>& b) {
    return (size_t)b.tile_cap * 2 * sizeof(typename Vec4<T>::type);
}

// Dynamic shared memory beyond 48 KiB must be allowed per kernel.
template <typename T>
cudaError_t prepare_tile(const Bufs<T>& b) {
    const int bytes = (int)tile_smem_bytes(b);
    cudaError_t e = cudaFuncSetAttribute(tile_search_kernel<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tile_search_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if constexpr (sizeof(T) == 4) {
        const int pb = (int)pruned_smem_bytes(b.tile_cap);
        const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
        if (e == cudaSuccess) e = cudaFuncSetAttribute(tile_pruned_kernel<3, kPrunedCap>, attr, pb);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(tile_pruned_kernel<3, 0>, attr, pb);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(tile_pruned_kernel<2, kPrunedCap>, attr, pb);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(tile_pruned_kernel<2, 0>, attr, pb);
    }
    return e;
}

template <typename T>
cudaError_t prepare_staged(const Bufs<T>& b) {
    const size_t bytes = stage_smem_bytes(b);
    return cudaFuncSetAttribute(search_staged_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T>
cudaError_t launch_move(const Bufs<T>& b, cudaStream_t s) {
    if (b.n == 0) return cudaSuccess;
    KMC_DIM_DISPATCH(b.geo.dim, move_kernel, b);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scatter(const Bufs<T>& b, cudaStream_t s) {
    if (b.n == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((b.n + (int64_t)kThreads * kScatterItems - 1) / ((int64_t)kThreads * kScatterItems));
    scatter_tags_kernel<T><<<blocks, kThreads, 0, s>>>(b);
    scatter_kernel<T><<<blocks_for(b.n), kThreads, 0, s>>>(b);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dsmc(const Bufs<T>& b, cudaStream_t s) {
    if (b.n == 0 || b.n_keys == 0) return cudaSuccess;
    dsmc_kernel<T><<<(unsigned)((b.n_keys + kThreads - 1) / kThreads), kThreads, 0, s>>>(b);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_perm(const Bufs<T>& b, int32_t* perm, cudaStream_t s) {
    if (b.n == 0) return cudaSuccess;
    perm_kernel<T><<<blocks_for(b.n), kThreads, 0, s>>>(b, perm);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather_state(const Bufs<T>& b, T* pos3, T* vel3, cudaStream_t s) {
    if (b.n == 0) return cudaSuccess;
    gather_kernel<T><<<blocks_for(b.n), kThreads, 0, s>>>(b, pos3, vel3);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cell_keys(const Bufs<T>& b, int32_t* keys, cudaStream_t s) {
    if (b.n == 0) return cudaSuccess;
    KMC_DIM_DISPATCH(b.geo.dim, cellkey_kernel, b, keys);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_moments(const Bufs<T>& b, int use_virial, cudaStream_t s) {
    if (b.n == 0) return cudaSuccess;
    if (b.cbin_moments) {   // one warp per c-bin
        const unsigned blocks = (unsigned)((b.n_bins + kThreads / 32 - 1) / (kThreads / 32));
        if (b.radial) {
            if (b.geo.dim == 3) moments_cbin_kernel<T, 3, true><<<blocks, kThreads, 0, s>>>(b, use_virial);
            else moments_cbin_kernel<T, 2, true><<<blocks, kThreads, 0, s>>>(b, use_virial);
        } else {
            if (b.geo.dim == 3) moments_cbin_kernel<T, 3, false><<<blocks, kThreads, 0, s>>>(b, use_virial);
            else moments_cbin_kernel<T, 2, false><<<blocks, kThreads, 0, s>>>(b, use_virial);
        }
        return cudaGetLastError();
    }
    const int64_t threads = (b.n + kMomItems - 1) / kMomItems;
    const unsigned blocks = (unsigned)((threads + kThreads - 1) / kThreads);
    if (b.radial) {
        if (b.geo.dim == 3) moments_kernel<T, 3, true><<<blocks, kThreads, 0, s>>>(b, use_virial);
        else moments_kernel<T, 2, true><<<blocks, kThreads, 0, s>>>(b, use_virial);
    } else {
        if (b.geo.dim == 3) moments_kernel<T, 3, false><<<blocks, kThreads, 0, s>>>(b, use_virial);
        else moments_kernel<T, 2, false><<<blocks, kThreads, 0, s>>>(b, use_virial);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cbin_hist(const Bufs<T>& b, uint32_t* hist, unsigned long long* vmax2, cudaStream_t s) {
    if (b.n == 0) return cudaSuccess;
    KMC_DIM_DISPATCH(b.geo.dim, cbin_hist_kernel, b, hist, vmax2);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_window_count(const Bufs<T>& b, unsigned long long* total, cudaStream_t s) {
    if (b.n == 0) return cudaSuccess;
    KMC_DIM_DISPATCH(b.geo.dim, window_count_kernel, b, total);
    return cudaGetLastError();
}

#define KMC_INSTANTIATE(T)                                                                        \
    template cudaError_t launch_pack<T>(const Bufs<T>&, const T*, const T*, uint32_t*, cudaStream_t); \
    template cudaError_t launch_bin_init<T>(const Bufs<T>&, cudaStream_t);                         \
    template cudaError_t launch_search<T>(const Bufs<T>&, cudaStream_t);                           \
    template cudaError_t launch_tile_search<T>(const Bufs<T>&, cudaStream_t);                      \
    template cudaError_t prepare_staged<T>(const Bufs<T>&);                                        \
    template cudaError_t prepare_tile<T>(const Bufs<T>&);                                          \
    template size_t tile_smem_bytes<T>(const Bufs<T>&);                                            \
    template size_t stage_smem_bytes<T>(const Bufs<T>&);                                           \
    template cudaError_t launch_move<T>(const Bufs<T>&, cudaStream_t);                             \
    template cudaError_t launch_scatter<T>(const Bufs<T>&, cudaStream_t);                          \
    template cudaError_t launch_gather_state<T>(const Bufs<T>&, T*, T*, cudaStream_t);             \
    template cudaError_t launch_cell_keys<T>(const Bufs<T>&, int32_t*, cudaStream_t);              \
    template cudaError_t launch_moments<T>(const Bufs<T>&, int, cudaStream_t);                     \
    template cudaError_t launch_cbin_hist<T>(const Bufs<T>&, uint32_t*, unsigned long long*, cudaStream_t); \
    template cudaError_t launch_window_count<T>(const Bufs<T>&, unsigned long long*, cudaStream_t);   \
    template cudaError_t launch_perm<T>(const Bufs<T>&, int32_t*, cudaStream_t);                   \
    template cudaError_t launch_dsmc<T>(const Bufs<T>&, cudaStream_t);

}  // namespace kmc
