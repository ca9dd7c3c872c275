// gdi_window.cuh -- sorted-window building blocks of libgdi.so, shared by the grid-scale kernels
// (gdi_grid.cu) and the CTA-resident sorted-window kernel (gdi_kernels.cu).
//
// A window is W consecutive ranks of one colour class.  Inside it the +1 group, in order of flip
// threshold gamma ascending (then position), and the -1 group, by gamma descending, each see the
// exact running G (reading R2 of Algorithm 3).  Sorting a group once gives every member k the value
// rel = a_k - c (+1: a_k = gamma_(k) + 2k; -1: b_k = gamma_(k) - 2k) relative to a reference G c,
// after which member k flips iff rel <= x (+1) or rel >= x (-1) for the x = G - c entering the
// group: one comparison per member.  Stage maps summarise a window on the lattice x = -64 .. 62.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gdi_device.cuh"

namespace gdi {
namespace win {

constexpr int KC = 31;                  // flips per group the exact counting histogram covers at once
constexpr int HA = 2 * KC + 1;          // histogram bins of the exact counting replay
constexpr int NT = 64;                  // lattice points of a stage map
constexpr int32_t KEY_D = 1 << 22;      // threshold distances are clamped to [-KEY_D, KEY_D)
constexpr int32_t REL_CAP = 32767;      // rel values are stored clamped to +-REL_CAP
constexpr int32_t FAST_X = 32000;       // |G - c| up to which the stored rel values decide exactly
constexpr unsigned long long STEP_MASK = (1ull << (NT - 1)) - 1ull;

struct StageMap {
    unsigned long long mask;            // bit j: the step from lattice point j to j + 1 rises
    int32_t ylo;                        // output index of lattice point 0
    int32_t narrow;                     // 1: the window's rel values are exact on the lattice only
};

// In-place cumulative counts of bins[0, nb) by one warp: forward (bins[x] = base + sum_{b <= x})
// or backward (bins[x] = base + sum_{b >= x}); each lane scans a contiguous chunk.
__device__ inline void warp_cumulate(int32_t *bins, int nb, int32_t base, bool forward)
{
    const int lane = threadIdx.x & 31;
    const int ch = (nb + 31) / 32;
    const int l = forward ? lane : 31 - lane;          // chunk order along the scan direction
    const int b0 = l * ch, b1 = min(b0 + ch, nb);
    int32_t loc = 0;
    for (int b = b0; b < b1; ++b) loc += bins[b];
    // lanes in increasing order hold the chunks in scan order (backward: lane 0 owns the top
    // chunk), so an inclusive scan over lane order gives the sum up to and including my chunk
    int32_t x = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    int32_t run = base + x - loc;                       // everything before my chunk
    if (forward) {
        for (int b = b0; b < b1; ++b) { run += bins[b]; bins[b] = run; }
    } else {
        for (int b = b1 - 1; b >= b0; --b) { run += bins[b]; bins[b] = run; }
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------------------------
// Exact decision of one group of one window for one replica, by one warp.
// Members are window positions i in [ws, we) whose start sign (bit r of s0[i]) is the group's;
// gam[i * gs + r] are their thresholds.  +1 group: the k-th member in (gamma asc, position asc)
// order flips iff g - 2k >= gamma_(k).  -1 group: (gamma desc, position asc), flips iff
// g + 2k <= gamma_(k).  Returns the number of flips K; marks them in fm (if fm != null).
__device__ inline int32_t warp_count(const int32_t *gam, int gs, int gc, const uint8_t *s0, int r, int ws,
                              int we, bool plus, int64_t v)
{
    const int lane = threadIdx.x & 31;
    int32_t c = 0;
    for (int i = ws + lane; i < we; i += 32) {
        const bool neg = (s0[i] >> r) & 1;
        if (plus != !neg) continue;
        const int64_t gm = gam[(size_t)i * gs + gc];
        c += plus ? (gm <= v) : (gm >= v);
    }
    return warp_sum(c);
}

__device__ inline int32_t warp_group(const int32_t *gam, int gs, int gc, const uint8_t *s0, int r, int ws,
                              int we, int32_t g, bool plus, int32_t *bins, uint32_t *fm)
{
    const int lane = threadIdx.x & 31;
    // histogram of thresholds over [g - 2KC, g] (+) or [g, g + 2KC] (-); beyond: "deep" members
    const int64_t base = plus ? (int64_t)g - 2 * KC : (int64_t)g;
    for (int b = lane; b < HA; b += 32) bins[b] = 0;
    __syncwarp();
    int32_t deep = 0;
    for (int i = ws + lane; i < we; i += 32) {
        const bool neg = (s0[i] >> r) & 1;
        if (plus == neg) continue;
        const int64_t gm = gam[(size_t)i * gs + gc];
        const int64_t b = gm - base;
        if (plus) {
            if (b < 0) ++deep;
            else if (b < HA) atomicAdd(&bins[b], 1);
        } else {
            if (b >= HA) ++deep;
            else if (b >= 0) atomicAdd(&bins[b], 1);
        }
    }
    deep = warp_sum(deep);
    __syncwarp();
    // cumulative counts toward the deep side: plus: C(base + x) = deep + sum_{b <= x};
    // minus: D(base + x) = deep + sum_{b >= x}
    warp_cumulate(bins, HA, deep, plus);
    // K = #{k : count(g -/+ 2k) >= k + 1}, k in [0, KC] (one lane per k)
    int32_t K;
    int64_t vstar = 0;
    int32_t t = 0;
    bool slow;
    {
        const int k = lane;   // KC + 1 == 32 lanes
        const int x = plus ? (HA - 1) - 2 * k : 2 * k;
        const bool pred = bins[x] >= k + 1;
        const unsigned m = __ballot_sync(0xFFFFFFFFu, pred);
        K = __popc(m);
        slow = (m >> 31) & 1;   // K may exceed KC
    }
    if (!slow) {
        if (K == 0) return 0;
        if (K <= deep) {
            // all K flips are deep members (K == deep here: K >= min(deep, KC + 1))
            vstar = plus ? base : base + HA - 1;   // flips: exactly the deep members
            t = 0;
        } else {
            // v* = the K-th value in group order; t = ties at v* that flip
            int first = -1;
            for (int x0 = 0; x0 < HA; x0 += 32) {
                const int x = x0 + lane;
                bool pred = false;
                if (x < HA) pred = plus ? (bins[x] >= K) : (bins[HA - 1 - x] >= K);
                const unsigned m = __ballot_sync(0xFFFFFFFFu, pred);
                if (m) { first = x0 + __ffs(m) - 1; break; }
            }
            if (plus) {
                vstar = base + first;
                const int32_t before = first > 0 ? bins[first - 1] : deep;
                t = K - before;
            } else {
                const int xb = HA - 1 - first;
                vstar = base + xb;
                const int32_t before = xb < HA - 1 ? bins[xb + 1] : deep;
                t = K - before;
            }
        }
    } else {
        // exact counting path: K = max{k + 1 : count(g -/+ 2k) >= k + 1}
        const int32_t n0 = warp_count(gam, gs, gc, s0, r, ws, we, plus, g);
        int32_t lo = 0, hi = n0;   // K in [0, n0]
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;   // test k = mid - 1
            const int64_t v = plus ? (int64_t)g - 2 * (int64_t)(mid - 1) : (int64_t)g + 2 * (int64_t)(mid - 1);
            if (warp_count(gam, gs, gc, s0, r, ws, we, plus, v) >= mid) lo = mid; else hi = mid - 1;
        }
        K = lo;
        if (K == 0) return 0;
        // v*: plus: smallest v with C(v) >= K; minus: largest v with D(v) >= K
        int64_t a = -((int64_t)1 << 31), b = (int64_t)1 << 31;
        if (plus) {
            b = (int64_t)g - 2 * (int64_t)(K - 1);
            while (a < b) {
                const int64_t mid = a + ((b - a) >> 1);
                if (warp_count(gam, gs, gc, s0, r, ws, we, true, mid) >= K) b = mid; else a = mid + 1;
            }
            vstar = a;
            t = K - warp_count(gam, gs, gc, s0, r, ws, we, true, vstar - 1);
        } else {
            a = (int64_t)g + 2 * (int64_t)(K - 1);
            while (a < b) {
                const int64_t mid = a + ((b - a + 1) >> 1);
                if (warp_count(gam, gs, gc, s0, r, ws, we, false, mid) >= K) a = mid; else b = mid - 1;
            }
            vstar = a;
            t = K - warp_count(gam, gs, gc, s0, r, ws, we, false, vstar + 1);
        }
    }
    if (fm) {
        int32_t run = 0;
        for (int i0 = ws; i0 < we; i0 += 32) {
            const int i = i0 + lane;
            bool mem = false, strict = false, tie = false;
            if (i < we) {
                const bool neg = (s0[i] >> r) & 1;
                mem = (plus != neg);
                if (mem) {
                    const int64_t gm = gam[(size_t)i * gs + gc];
                    strict = plus ? (gm < vstar) : (gm > vstar);
                    tie = (gm == vstar);
                }
            }
            const unsigned tm = __ballot_sync(0xFFFFFFFFu, tie);
            const int32_t idx = run + __popc(tm & ((1u << lane) - 1u));
            run += __popc(tm);
            if (strict || (tie && idx < t)) atomicOr(&fm[i >> 2], 1u << (8 * (i & 3) + r));
        }
    }
    return K;
}

// ascending sort of 32 * S keys held as key[s] of lane l = element l * S + s: a bitonic network in
// its all-ascending form (every merge starts with a "flip" stage that pairs element e with
// e ^ (size - 1), then half-cleaners pair e with e ^ j), so that a compare-exchange always sends
// the minimum to the lower element -- in-register steps are a plain min/max pair
template <int S>
__device__ __forceinline__ void warp_bitonic(uint32_t (&key)[S])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int size = 2; size <= 32 * S; size <<= 1) {
        if (size <= S) {
#pragma unroll
            for (int s = 0; s < S; ++s) {
                if ((s & (size >> 1)) == 0) {
                    const int q = s ^ (size - 1);
                    const uint32_t a = key[s], b = key[q];
                    key[s] = min(a, b);
                    key[q] = max(a, b);
                }
            }
        } else {
            const bool lower = ((lane * S) & (size >> 1)) == 0;
            uint32_t o[S];
#pragma unroll
            for (int s = 0; s < S; ++s) o[s] = __shfl_xor_sync(0xFFFFFFFFu, key[S - 1 - s], size / S - 1);
#pragma unroll
            for (int s = 0; s < S; ++s) key[s] = lower ? min(key[s], o[s]) : max(key[s], o[s]);
        }
#pragma unroll
        for (int j = size >> 2; j >= 1; j >>= 1) {
            if (j >= S) {
                const bool keep_min = ((lane * S) & j) == 0;
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    const uint32_t o = __shfl_xor_sync(0xFFFFFFFFu, key[s], j / S);
                    key[s] = keep_min ? min(key[s], o) : max(key[s], o);
                }
            } else {
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    if ((s & j) == 0) {
                        const uint32_t a = key[s], b = key[s + j];
                        key[s] = min(a, b);
                        key[s + j] = max(a, b);
                    }
                }
            }
        }
    }
}

// The same ascending network on 16-bit keys packed two to a register: register t of a lane holds
// its element t (low half) and element t + S/2 (high half), so a compare-exchange of two registers
// in the same half does two element pairs at once (__vminu2 / __vmaxu2) and a cross-lane stage
// moves two keys per shuffle.  Pairs that meet inside one register (the top bit of the in-lane
// index) are swapped into place with a byte permute.  S >= 2.
static __device__ __forceinline__ uint32_t swap16(uint32_t v) { return __byte_perm(v, 0, 0x1032); }

// compare-exchange of the two halves of v: the minimum to the low half
static __device__ __forceinline__ uint32_t ce_halves(uint32_t v)
{
    const uint32_t w = swap16(v);
    return __byte_perm(__vminu2(v, w), __vmaxu2(v, w), 0x7610);
}

template <int S>
__device__ __forceinline__ void warp_bitonic16(uint32_t (&P)[S / 2])
{
    constexpr int H = S / 2;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int size = 2; size <= 32 * S; size <<= 1) {
        // flip stage: element e meets e ^ (size - 1), the minimum goes to the lower one
        if (size <= H) {
#pragma unroll
            for (int t = 0; t < H; ++t) {
                if ((t & (size >> 1)) == 0) {
                    const int q = t ^ (size - 1);
                    const uint32_t a = P[t], b = P[q];
                    P[t] = __vminu2(a, b);
                    P[q] = __vmaxu2(a, b);
                }
            }
        } else if (size == S) {
            // element t (low half of P[t]) meets S-1-t (high half of P[H-1-t]), and element t + H
            // (high half of P[t]) meets H-1-t (low half of P[H-1-t])
#pragma unroll
            for (int t = 0; t < H; ++t) {
                const int q = H - 1 - t;
                if (q == t) {
                    P[t] = ce_halves(P[t]);
                } else if (t < q) {
                    const uint32_t a = P[t], b = swap16(P[q]);
                    const uint32_t mn = __vminu2(a, b), mx = __vmaxu2(a, b);
                    P[t] = __byte_perm(mn, mx, 0x7610);
                    P[q] = __byte_perm(mn, mx, 0x5432);
                }
            }
        } else {
            const bool lower = ((lane * S) & (size >> 1)) == 0;
            uint32_t o[H];
#pragma unroll
            for (int t = 0; t < H; ++t) o[t] = swap16(__shfl_xor_sync(0xFFFFFFFFu, P[H - 1 - t], size / S - 1));
#pragma unroll
            for (int t = 0; t < H; ++t) P[t] = lower ? __vminu2(P[t], o[t]) : __vmaxu2(P[t], o[t]);
        }
        // half-cleaners: element e meets e ^ j
#pragma unroll
        for (int j = size >> 2; j >= 1; j >>= 1) {
            if (j >= S) {
                const bool keep_min = ((lane * S) & j) == 0;
#pragma unroll
                for (int t = 0; t < H; ++t) {
                    const uint32_t o = __shfl_xor_sync(0xFFFFFFFFu, P[t], j / S);
                    P[t] = keep_min ? __vminu2(P[t], o) : __vmaxu2(P[t], o);
                }
            } else if (j == H) {
#pragma unroll
                for (int t = 0; t < H; ++t) P[t] = ce_halves(P[t]);
            } else {
#pragma unroll
                for (int t = 0; t < H; ++t) {
                    if ((t & j) == 0) {
                        const uint32_t a = P[t], b = P[t + j];
                        P[t] = __vminu2(a, b);
                        P[t + j] = __vmaxu2(a, b);
                    }
                }
            }
        }
    }
}

// rel values and the two stage maps of one window (positions [ws, ws + wlen), wlen <= 32 * S) for
// replica r, by one warp.  out[0] = +1 group, out[1] = -1 group.
//
// Narrow keys: when every member has d >= -62 (d = the threshold's distance from c in sort
// direction), the window sorts 16-bit keys (group, d clamped to [-62, 65] in 7 bits, position).
// With d >= -62 a window entered at x = G - c in the lattice [-64, 62] keeps x in [-64, 64]
// through both of its groups (the +1 group cannot take x below -64, the -1 group not above 64), and
// a member clamped at the top cannot flip at any such x (+1: rel = d + 2k >= 65 > 64; -1:
// rel = -d - 2k <= -65 < -64) and sorts after every other member of its group either way.  So the
// stage maps and the replay of a window entered on the lattice are exact; the stored rel values of
// clamped members are not, so the replay uses a narrow window's rel values only when it is entered
// on the lattice (StageMap.narrow) and replays it exactly otherwise.
template <int S>
__device__ __forceinline__ void window_maps(const int32_t *gam_r, const uint8_t *s0, int16_t *rel_r, int ws,
                                            int wlen, int r, int32_t c, StageMap *out)
{
    const int lane = threadIdx.x & 31;
    int32_t dv[S];
    uint32_t ng = 0;                      // bit s: member s is in the -1 group
    int32_t np = 0;
    bool wide = false;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int pos = s * 32 + lane;
        dv[s] = 0;
        if (pos < wlen) {
            const int32_t g = gam_r[ws + pos];
            const uint32_t neg = (s0[ws + pos] >> r) & 1u;
            int32_t d = neg ? c - g : g - c;
            d = min(max(d, -KEY_D), KEY_D - 1);
            dv[s] = d;
            ng |= neg << s;
            np += neg ? 0 : 1;
            wide |= d < -62;
        }
    }
    np = __reduce_add_sync(0xFFFFFFFFu, np);
    const bool narrow = S >= 2 && !__any_sync(0xFFFFFFFFu, wide);
    unsigned long long kp = 0, km = 0;
    int32_t cle = 0, cge = 0;
    // element e of the sorted order: group, d and position -> rel value and lattice bits, without
    // branches (the lanes of a warp hold members of both groups at every distance)
    auto take = [&](int e, bool neg, int32_t d, int pos) {
        const int32_t rel = neg ? -d - 2 * (e - np) : d + 2 * e;
        rel_r[ws + pos] = (int16_t)min(max(rel, -REL_CAP), REL_CAP);
        // +1 group: an a_k at or below the lattice start counts into ylo, one in (-64, 62] clears
        // the step of its lattice interval; -1 group: b_k >= -64 counts, b_k in [-64, 61] clears
        const bool pos_grp = !neg;
        cle += (pos_grp && rel <= -NT) ? 1 : 0;
        const bool p_in = pos_grp && rel > -NT && rel <= NT - 2;
        kp |= p_in ? 1ull << (((uint32_t)(rel + NT - 1) >> 1) & 63u) : 0ull;
        const bool m_ge = neg && rel >= -NT;
        cge += m_ge ? 1 : 0;
        km |= (m_ge && rel <= NT - 3) ? 1ull << (((uint32_t)(rel + NT) >> 1) & 63u) : 0ull;
    };
    if constexpr (S >= 2) {
        if (narrow) {
            constexpr int H = S / 2;
            uint32_t P[H];
#pragma unroll
            for (int t = 0; t < H; ++t) {
                uint32_t k2[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int s = t + h * H;
                    const int pos = s * 32 + lane;
                    uint32_t k = 0xFFFFu;
                    if (pos < wlen) {
                        const uint32_t neg = (ng >> s) & 1u;
                        const int32_t dq = min(dv[s], 65) + 62;
                        k = (neg << 15) | ((uint32_t)dq << 8) | (uint32_t)pos;
                    }
                    k2[h] = k;
                }
                P[t] = k2[0] | (k2[1] << 16);
            }
            warp_bitonic16<S>(P);
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const int e = lane * S + s;
                if (e < wlen) {
                    const uint32_t k = (s < H ? P[s] : (P[s - H] >> 16)) & 0xFFFFu;
                    const bool neg = (k >> 15) != 0;
                    const int32_t d = (int32_t)((k >> 8) & 0x7Fu) - 62;
                    take(e, neg, d, (int)(k & 0xFFu));
                }
            }
        }
    }
    if (!narrow) {
        uint32_t key[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int pos = s * 32 + lane;
            key[s] = pos < wlen ? (((ng >> s) & 1u) << 31) | ((uint32_t)(dv[s] + KEY_D) << 8) | (uint32_t)pos
                                : 0xFFFFFFFFu;
        }
        warp_bitonic<S>(key);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int e = lane * S + s;
            if (e < wlen) {
                const uint32_t k = key[s];
                take(e, (k >> 31) != 0, (int32_t)((k >> 8) & 0x7FFFFFu) - KEY_D, (int)(k & 0xFFu));
            }
        }
    }
    const uint32_t kp0 = __reduce_or_sync(0xFFFFFFFFu, (uint32_t)kp);
    const uint32_t kp1 = __reduce_or_sync(0xFFFFFFFFu, (uint32_t)(kp >> 32));
    const uint32_t km0 = __reduce_or_sync(0xFFFFFFFFu, (uint32_t)km);
    const uint32_t km1 = __reduce_or_sync(0xFFFFFFFFu, (uint32_t)(km >> 32));
    cle = __reduce_add_sync(0xFFFFFFFFu, cle);
    cge = __reduce_add_sync(0xFFFFFFFFu, cge);
    if (lane == 0) {
        out[0].mask = ~(((unsigned long long)kp1 << 32) | kp0) & STEP_MASK;
        out[0].ylo = -cle;
        out[0].narrow = narrow ? 1 : 0;
        out[1].mask = ~(((unsigned long long)km1 << 32) | km0) & STEP_MASK;
        out[1].ylo = cge;
        out[1].narrow = narrow ? 1 : 0;
    }
}

static __device__ __forceinline__ int stage_apply(const StageMap &m, int t)
{
    if (t < 0) return -1;
    const int y = m.ylo + __popcll(m.mask & ((1ull << t) - 1ull));
    return (y >= 0 && y < NT) ? y : -1;
}

// the exact replay of one window by counting (|G - c| beyond the stored values), kept out of line
static __device__ __noinline__ int32_t window_replay_exact(const int32_t *gr, const uint8_t *s0, int r, int ws, int we,
                                                    int32_t g, bool plus_first, int32_t *bins, uint32_t *fm)
{
    const int32_t K1 = warp_group(gr, 1, 0, s0, r, ws, we, g, plus_first, bins, fm);
    g = plus_first ? g - 2 * K1 : g + 2 * K1;
    const int32_t K2 = warp_group(gr, 1, 0, s0, r, ws, we, g, !plus_first, bins, fm);
    return plus_first ? g + 2 * K2 : g - 2 * K2;
}

// Replay of one window (positions [ws, we)) of replica r from x = G - c with its rel values, by one
// warp: both groups in order, each member deciding by one comparison; the flips go into the
// replica's flip bitmap fb.  With W a multiple of 32 every window owns whole words; otherwise
// windows share words and OR their bits in atomically, so windows may be replayed concurrently.
// Returns x after the window.
template <int SL>
__device__ __forceinline__ int32_t replay_window(const int16_t *rr, const uint8_t *s0, int r, int ws, int we,
                                                 int32_t x, bool plus_first, uint32_t *fb, int W)
{
    const int lane = threadIdx.x & 31;
    // members of the window in registers (slot s = positions ws + 32 s + lane)
    int32_t rv[SL];
    uint32_t ng = 0, vd = 0;            // bit s: member is -1 / exists
#pragma unroll
    for (int s = 0; s < SL; ++s) {
        const int i = ws + 32 * s + lane;
        rv[s] = 0;
        if (i < we) {
            rv[s] = rr[i];
            vd |= 1u << s;
            ng |= ((uint32_t)(s0[i] >> r) & 1u) << s;
        }
    }
    uint32_t wbits[SL];
#pragma unroll
    for (int s = 0; s < SL; ++s) wbits[s] = 0;
#pragma unroll
    for (int ph = 0; ph < 2; ++ph) {
        const bool plus = plus_first == (ph == 0);
        int32_t cnt = 0;
#pragma unroll
        for (int s = 0; s < SL; ++s) {
            const bool mem = ((vd >> s) & 1u) && (((ng >> s) & 1u) != (plus ? 1u : 0u));
            const bool f = mem && (plus ? rv[s] <= x : rv[s] >= x);
            const unsigned bm = __ballot_sync(0xFFFFFFFFu, f);
            cnt += __popc(bm);
            wbits[s] |= bm;
        }
        x = plus ? x - 2 * cnt : x + 2 * cnt;
    }
    // flip words: slot s covers positions [ws + 32 s, ws + 32 s + 32)
    if ((W & 31) == 0) {
#pragma unroll
        for (int s = 0; s < SL; ++s)
            if (lane == s && ws + 32 * s < we) fb[(ws >> 5) + s] = wbits[s];
    } else if (lane == 0) {
        const int sh = ws & 31;
#pragma unroll
        for (int s = 0; s < SL; ++s) {
            if (!wbits[s]) continue;
            const int q = (ws >> 5) + s;
            atomicOr(&fb[q], wbits[s] << sh);
            if (sh) atomicOr(&fb[q + 1], wbits[s] >> (32 - sh));
        }
    }
    return x;
}


}  // namespace win
}  // namespace gdi
