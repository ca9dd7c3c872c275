// gdi_device.cuh -- device helpers shared by the CTA-resident and the grid-scale kernels of
// libgdi.so: Philox4x32-10, the digest hash, the threshold search and the flip threshold of one
// spin, and block-level reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gdi {

constexpr int32_t GAM_INF = 1 << 30;      // |threshold| sentinel: flips always / never
constexpr int32_t ES_NONE = INT32_MIN;    // the draw accepts no energy change
constexpr int32_t ES_ALL = INT32_MAX;     // the draw accepts every energy change

// ---------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, multipliers 0xD2511F53 and
// 0xCD9E8D57, Weyl key increments 0x9E3779B9 and 0xBB67AE85.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint32_t word_of(const uint4 &v, int i)
{
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// splitmix64 finaliser (Steele, Lea, Flood 2014) -- state digest only
__device__ __forceinline__ uint64_t splitmix64_fin(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ int32_t floor_div_pos(int32_t a, int32_t b)  // b > 0
{
    int32_t q = a / b;
    if ((a % b) != 0 && a < 0) --q;
    return q;
}

// E*(u): number of table entries > u for a Metropolis row (entries are thr(dE = 1..len),
// non-increasing), i.e. the largest dE >= 0 the draw accepts.  thr(dE) > u exactly when
// dE <= T ln(2^32 / (u + 1)); that float estimate is corrected against the row itself, so the
// result is the exact count whatever the rounding of the estimate.  Paper rows hold thr(-1, 0, +1).
__device__ __forceinline__ int32_t estar_of(const uint32_t *row, int len, int mode, uint32_t u,
                                            float T)
{
    if (mode == 0) {
        float est = T * (22.18070977791825f - __logf((float)u + 1.0f));
        int e = est <= 0.f ? 0 : (est >= (float)len ? len : (int)est);
        while (e < len && row[e] > u) ++e;
        while (e > 0 && row[e - 1] <= u) --e;
        return e;
    }
    if (row[0] <= u) return ES_NONE;
    if (row[1] <= u) return -1;
    if (row[2] <= u) return 0;
    return ES_ALL;
}

__device__ __forceinline__ int32_t gamma_of(int sg, int32_t h, int32_t es, int32_t A, int32_t B)
{
    if (sg > 0) {
        if (es == ES_NONE) return GAM_INF;
        if (es == ES_ALL) return -GAM_INF;
        if (A == 0) return (B * h <= es) ? -GAM_INF : GAM_INF;
        return -floor_div_pos(-(B * h + 4 * A - es), 4 * A);     // ceil
    }
    if (es == ES_NONE) return -GAM_INF;
    if (es == ES_ALL) return GAM_INF;
    if (A == 0) return (-B * h <= es) ? GAM_INF : -GAM_INF;
    return floor_div_pos(es + B * h - 4 * A, 4 * A);
}

// gamma_of when 4A = 2^sh: floor division by a power of two is an arithmetic shift
__device__ __forceinline__ int32_t gamma_of_shift(int sg, int32_t h, int32_t es, int32_t A, int32_t B, int sh)
{
    if (sg > 0) {
        if (es == ES_NONE) return GAM_INF;
        if (es == ES_ALL) return -GAM_INF;
        return -((-(B * h + 4 * A - es)) >> sh);          // ceil((B h + 4A - E*) / 4A)
    }
    if (es == ES_NONE) return -GAM_INF;
    if (es == ES_ALL) return GAM_INF;
    return (es + B * h - 4 * A) >> sh;                    // floor((E* + B h - 4A) / 4A)
}

// ---------------------------------------------------------------------------------------------
// block primitives (BS threads, red: shared scratch of >= BS/32 + 1 words of T)
template <int BS, typename T>
__device__ __forceinline__ T block_sum(T v, T *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    T s = 0;
#pragma unroll
    for (int i = 0; i < BS / 32; ++i) s += red[i];
    return s;
}

// exclusive scan of one int32 per thread; returns the prefix, *total gets the block sum
template <int BS>
__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t *red, int32_t *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) red[wid] = x;
    __syncthreads();
    int32_t base = 0, tot = 0;
#pragma unroll
    for (int i = 0; i < BS / 32; ++i) {
        const int32_t r = red[i];
        if (i < wid) base += r;
        tot += r;
    }
    *total = tot;
    return base + x - v;
}


// warp sum
template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

}  // namespace gdi
