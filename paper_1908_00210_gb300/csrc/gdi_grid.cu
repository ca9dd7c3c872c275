// gdi_grid.cu -- grid-scale GDI anneal for graphs too large for one block (e.g. 10^6 vertices).
//
// Semantics are those of the CTA-resident kernel (Algorithm 3 of arXiv:1908.00210, serialised:
// colour classes in order, windows of W ranks, inside a window the +1 group by threshold ascending
// then the -1 group by threshold descending, each seeing the exact running G).  What changes is
// how the chain of windows is evaluated when a class holds thousands of windows spread over every
// SM.  Common to both variants below: up to 8 replicas share one byte per vertex (bit r set = spin
// of replica r is -1), so one gather of a neighbour byte feeds all of them (SWAR byte-lane
// counters); every block owns a contiguous run of windows of each class; the map "G at window
// start -> G at window end" is monotone and is tabulated around c, the G at class start.
//
// Sorted-window variant (W <= 256, gdi_grid_sorted_kernel): a warp sorts each (window, replica)
// group once, after which every member decides its own flip by one comparison; block tables are
// published with the class parity in every byte and each block finds its entering G by looking
// them up, so only one grid barrier per class remains (described before the kernel).  The local
// fields are kept across classes and updated by the flips (atomic adds to the neighbours).
//
// Tabulated variant (W > 256, gdi_grid_anneal_kernel):
//   * every window tabulates its map for G in [c - RT, c + RT] from two small histograms of its
//     thresholds, and each block composes the maps of its consecutive windows;
//   * after a grid barrier one block per replica walks the P block maps (a few hundred
//     shared-memory lookups) and publishes every block's exact input G; an entry that left the
//     tabulated range is recomputed exactly from the spins (fallback);
//   * after a second barrier every block replays its windows with the exact input, flips, and a
//     third barrier makes the class's spins visible to the next class.
//
// Grid barriers are sense/generation barriers on global counters with a bounded spin, and every
// other wait (tables, exact G words) is bounded too: a block that waits too long sets the error word and the kernel returns
// (GDI_ERR_TIMEOUT on the host).
#include <cuda_runtime.h>
#include <stdint.h>

#include "gdi_device.cuh"
#include "gdi_internal.h"
#include "gdi_window.cuh"

using namespace gdi;
using namespace gdi::win;

namespace {

constexpr int GB = 768;                 // threads per block
constexpr int NWARP = GB / 32;
static_assert(GB % 32 == 0, "whole warps; the threshold loop keeps one replica per thread");
constexpr int RT = 64;                  // tables cover G in [c - RT, c + RT]
constexpr int TW = 2 * RT + 1;
static_assert(TW == GDI_GRID_TW, "table width mismatch");
constexpr int HB = 2 * RT + 4 * KC + 1; // histogram bins for building a window table (KC: gdi_window.cuh)
constexpr int16_t TINV = INT16_MIN;
constexpr int LONG_ROW = 48;

__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }

__device__ __forceinline__ uint64_t spread8(uint32_t b)
{
    return (((uint64_t)(b & 0x7Fu) * 0x0002040810204081ull) & 0x0101010101010101ull) |
           ((uint64_t)(b >> 7) << 56);
}

struct GridLayout {
    int spc, wpc, P, max_row;
    size_t off_h, off_gam, off_s0, off_fm, off_longq, off_wtab, off_win, off_hist, off_ctab, off_row,
        off_misc, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline GridLayout grid_layout(int spc, int wpc, int P, int max_row)
{
    GridLayout L;
    L.spc = spc;
    L.wpc = wpc;
    L.P = P;
    L.max_row = max_row;
    size_t o = 0;
    L.off_h = o; o = align16(o + (size_t)spc * 8 * sizeof(int16_t));
    L.off_gam = o; o = align16(o + (size_t)spc * 8 * sizeof(int32_t));
    L.off_s0 = o; o = align16(o + (size_t)spc);
    L.off_fm = o; o = align16(o + (size_t)((spc + 3) / 4) * sizeof(uint32_t));
    L.off_longq = o; o = align16(o + (size_t)spc * sizeof(int32_t));
    L.off_wtab = o; o = align16(o + (size_t)wpc * 8 * TW * sizeof(int16_t));
    L.off_win = o; o = align16(o + (size_t)wpc * 8 * sizeof(int32_t));
    L.off_hist = o; o = align16(o + (size_t)NWARP * 2 * HB * sizeof(int32_t));
    L.off_ctab = o; o = align16(o + (size_t)P * TW * sizeof(int16_t));
    L.off_row = o; o = align16(o + (size_t)(max_row + 4) * sizeof(uint32_t));
    L.off_misc = o; o = align16(o + 64 * sizeof(int64_t));
    L.total = o;
    return L;
}

struct GridArgs {
    GdiDevProblem P;
    GdiDevRun R;
    GdiGridScratch X;
    int rep_base, nrep;
    int spc, wpc;
    const int32_t *wbnd;    // [classes][blocks + 1] first window of every block, or null (even split)
    unsigned long long *hf; // maintained fields (X.hfield) when this kernel keeps them, else null
    bool es_pre;            // sorted path: E* of the next class drawn ahead into shared memory
};

// ---------------------------------------------------------------------------------------------
// bounded grid barrier; returns false (and the caller must return) if any block timed out.  The
// arrival counter only grows: barrier k of a launch completes when it reaches k * gridDim.x, so the
// last arrival has nothing left to do (no reset, no generation word) and the waiters see the count
// one round trip after it lands.  bar[2] is a gate the failure-detection hook closes: while it is
// set no barrier completes and every wait runs into its bound.
__device__ bool grid_sync(const GdiGridScratch &X)
{
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        unsigned long long *cnt = reinterpret_cast<unsigned long long *>(X.bar);
        volatile unsigned int *gate = X.bar + 2;
        __threadfence();
        const unsigned long long old = atomicAdd(cnt, 1ull);
        const unsigned long long target = (old / gridDim.x + 1) * gridDim.x;
        int good = 1;
        long long spins = 0;
        while (*(volatile unsigned long long *)cnt < target || *gate) {
            if (++spins > X.spin_limit) {
                atomicExch(X.err, GDI_DEVERR_TIMEOUT);
                good = 0;
                break;
            }
            if (*(volatile int *)X.err) { good = 0; break; }
            __nanosleep(64);
        }
        __threadfence();
        if (*(volatile int *)X.err) good = 0;
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// local fields of one rank (row entries [e0, e1)) for all 8 replicas, thread-serial over the row,
// written to hout[0..7] (all replicas) or hout[0] (replica `one` only)
__device__ __forceinline__ void field8_thread(const GdiDevProblem &P, int64_t base, int64_t e0, int64_t e1,
                                              const uint8_t *packed, int16_t *hout, int one)
{
    uint64_t aP = 0, aN = 0;
    int32_t nN = 0, cnt = 0;
    int32_t cP0 = 0, cP1 = 0, cP2 = 0, cP3 = 0, cP4 = 0, cP5 = 0, cP6 = 0, cP7 = 0;
    int32_t cN0 = 0, cN1 = 0, cN2 = 0, cN3 = 0, cN4 = 0, cN5 = 0, cN6 = 0, cN7 = 0;
#define GDI_FLUSH()                                                                               \
    do {                                                                                          \
        cP0 += (int32_t)(aP & 0xFF); cP1 += (int32_t)((aP >> 8) & 0xFF);                          \
        cP2 += (int32_t)((aP >> 16) & 0xFF); cP3 += (int32_t)((aP >> 24) & 0xFF);                 \
        cP4 += (int32_t)((aP >> 32) & 0xFF); cP5 += (int32_t)((aP >> 40) & 0xFF);                 \
        cP6 += (int32_t)((aP >> 48) & 0xFF); cP7 += (int32_t)((aP >> 56) & 0xFF);                 \
        cN0 += (int32_t)(aN & 0xFF); cN1 += (int32_t)((aN >> 8) & 0xFF);                          \
        cN2 += (int32_t)((aN >> 16) & 0xFF); cN3 += (int32_t)((aN >> 24) & 0xFF);                 \
        cN4 += (int32_t)((aN >> 32) & 0xFF); cN5 += (int32_t)((aN >> 40) & 0xFF);                 \
        cN6 += (int32_t)((aN >> 48) & 0xFF); cN7 += (int32_t)((aN >> 56) & 0xFF);                 \
        aP = aN = 0;                                                                              \
    } while (0)
    // predicated batches of 8 entries: every load of a batch is in flight at once (rows of up to 8
    // entries cost one round trip for the columns and one for the spins)
    for (int64_t e = e0; e < e1; e += 8) {
        const int nb = (int)min((int64_t)8, e1 - e);
        uint32_t c[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) c[k] = k < nb ? __ldg(P.col + e + k) : 0u;
        uint8_t b[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) b[k] = k < nb ? __ldcg(packed + base + (c[k] & 0x7FFFFFFFu)) : (uint8_t)0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint64_t sv = spread8(b[k]);
            if (c[k] >> 31) { aN += sv; ++nN; } else aP += sv;
        }
        cnt += 8;
        if (cnt >= 248) { GDI_FLUSH(); cnt = 0; }
    }
    GDI_FLUSH();
#undef GDI_FLUSH
    const int32_t sw = (int32_t)(e1 - e0) - 2 * nN;     // sum of weights
    // h = sum w (1 - 2 bit) = sum w - 2 sum w bit
    if (one < 0) {
        hout[0] = (int16_t)(sw - 2 * (cP0 - cN0)); hout[1] = (int16_t)(sw - 2 * (cP1 - cN1));
        hout[2] = (int16_t)(sw - 2 * (cP2 - cN2)); hout[3] = (int16_t)(sw - 2 * (cP3 - cN3));
        hout[4] = (int16_t)(sw - 2 * (cP4 - cN4)); hout[5] = (int16_t)(sw - 2 * (cP5 - cN5));
        hout[6] = (int16_t)(sw - 2 * (cP6 - cN6)); hout[7] = (int16_t)(sw - 2 * (cP7 - cN7));
    } else {
        const int32_t cp = one == 0 ? cP0 : one == 1 ? cP1 : one == 2 ? cP2 : one == 3 ? cP3
                         : one == 4 ? cP4 : one == 5 ? cP5 : one == 6 ? cP6 : cP7;
        const int32_t cn = one == 0 ? cN0 : one == 1 ? cN1 : one == 2 ? cN2 : one == 3 ? cN3
                         : one == 4 ? cN4 : one == 5 ? cN5 : one == 6 ? cN6 : cN7;
        hout[0] = (int16_t)(sw - 2 * (cp - cn));
    }
}

// Partial sums of one chunk [c0, c1) of a long row (c1 - c0 <= LCHUNK), by one warp: sw = sum of
// weights, sb[k] = sum of w * bit_k (bit_k set = replica k is -1); valid in every lane.  Lanes take
// entries c0 + lane + 32 t in predicated batches of 8 (every load of a batch in flight at once).
constexpr int LCHUNK = 512;
__device__ __forceinline__ void chunk8_warp(const GdiDevProblem &P, int64_t base, int64_t c0, int64_t c1,
                            const uint8_t *packed, int32_t &sw, int32_t sb[8])
{
    const int lane = threadIdx.x & 31;
    uint64_t aP = 0, aN = 0;
    int32_t nN = 0, n = 0;
    // at most LCHUNK / 32 = 16 entries per lane: byte lanes cannot overflow
    for (int64_t e0 = c0 + lane; e0 < c1; e0 += 32 * 8) {
        uint32_t x[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = e0 + 32 * k < c1 ? __ldg(P.col + e0 + 32 * k) : 0u;
        uint8_t b[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            b[k] = e0 + 32 * k < c1 ? __ldcg(packed + base + (x[k] & 0x7FFFFFFFu)) : (uint8_t)0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (e0 + 32 * k >= c1) continue;
            const uint64_t sv = spread8(b[k]);
            if (x[k] >> 31) { aN += sv; ++nN; } else aP += sv;
            ++n;
        }
    }
    sw = warp_sum(n - 2 * nN);
#pragma unroll
    for (int k = 0; k < 8; ++k)
        sb[k] = warp_sum((int32_t)((aP >> (8 * k)) & 0xFF) - (int32_t)((aN >> (8 * k)) & 0xFF));
}

// Maintained local fields.  The fields of rank rk for the 8 replicas of a group live in two 64-bit
// words, H[2 rk + q] = sum_k h_{4q+k} 2^(16 k) mod 2^64.  Every |h| <= max degree < 2^15, so a word
// decodes exactly, and a flip adds its field changes to every neighbour's words with 64-bit atomic
// adds: the spins of a colour class change only at the class end, and the next class reads fields
// that are exact for the spins after the flips.
__device__ __forceinline__ unsigned long long field_word(const int16_t *h)
{
    unsigned long long w = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) w += (unsigned long long)(long long)h[k] << (16 * k);
    return w;
}

// decode one field word into four fields, returned as two pairs of 16-bit lanes
__device__ __forceinline__ uint2 field_unword(unsigned long long w)
{
    long long v = (long long)w;
    uint32_t o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int32_t x = (int16_t)(v & 0xFFFF);
        o[k] = (uint32_t)x & 0xFFFFu;
        v = (v - x) >> 16;
    }
    return make_uint2(o[0] | (o[1] << 16), o[2] | (o[3] << 16));
}

// the field changes that flipping replicas f (bit k) of a rank with group bits s (bit k set: -1
// before the flip) makes at a neighbour joined by weight +1: -2 where +1 -> -1, +2 where -1 -> +1
__device__ __forceinline__ void flip_words(uint32_t f, uint32_t s, unsigned long long &d0, unsigned long long &d1)
{
    d0 = d1 = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (!((f >> k) & 1u)) continue;
        const unsigned long long d = ((s >> k) & 1u) ? 2ull : ~1ull;        // +2 or -2 mod 2^64
        if (k < 4) d0 += d << (16 * k); else d1 += d << (16 * (k - 4));
    }
}

// ---------------------------------------------------------------------------------------------
struct GSmem {
    int16_t *h;        // [spc][8]
    int32_t *gam;      // [spc][8]
    uint8_t *s0;       // [spc]
    uint32_t *fm;      // [spc/4]
    int32_t *longq;    // [spc]
    int16_t *wtab;     // [wpc][8][TW]
    int32_t *win;      // [wpc][8]
    int32_t *hist;     // [NWARP][2][HB] (tabulated path) or [NWARP][HA] (sorted path)
    int32_t *nchunk;   // [spc] chunk counts of the long rows
    int16_t *ctab;     // [P][TW]
    uint32_t *row;     // [max_row]
    int64_t *misc;     // scratch
};

__device__ inline void class_partition(int32_t lo, int32_t hi, int W, int p, int P, int32_t &a0,
                                       int32_t &a1, int &nwin)
{
    const int32_t nw = (hi - lo + W - 1) / W;
    const int32_t k0 = (int32_t)(((int64_t)p * nw) / P);
    const int32_t k1 = (int32_t)(((int64_t)(p + 1) * nw) / P);
    a0 = lo + k0 * W;
    a1 = min(lo + k1 * W, hi);
    if (a1 < a0) a1 = a0;
    nwin = k1 - k0;
}

// Entry check of a launch's plan, by every block before it writes shared memory: the class bounds
// run monotonically from 0 to n, this block's share of every class fits the plan's spc ranks and
// wpc windows, and every table row of the sweep range fits max_row.  gdi_anneal derives these sizes
// itself; a caller of the allocation-free entry point passes them.  A failed check -- or an input
// check that failed before the launch and left the error word set -- makes the launch return: the
// failing block sets the error word, the others see it at their first barrier.
__device__ bool plan_fits(const GridArgs &A)
{
    const GdiDevProblem &P = A.P;
    const GdiDevRun &R = A.R;
    const int64_t base = P.node_off[0];
    const int32_t n = (int32_t)(P.node_off[1] - base);
    const int32_t *cls = P.class_ptr + P.class_off[0];
    const int32_t ncls = P.class_off[1] - P.class_off[0] - 1;
    const int Pb = gridDim.x, p = blockIdx.x;
    int bad = *(volatile int32_t *)A.X.err != 0 || ncls < 1;
    if (!bad) {
        if (threadIdx.x == 0 && (cls[0] != 0 || cls[ncls] != n)) bad = 1;
        for (int c = threadIdx.x; c < ncls; c += GB) {
            const int32_t lo = cls[c], hi = cls[c + 1];
            if (lo < 0 || hi < lo || hi > n) { bad = 1; continue; }
            int32_t x0, x1;
            int nw;
            if (A.wbnd) {
                const int32_t *bd = A.wbnd + (size_t)c * (Pb + 1);
                x0 = min(lo + bd[p] * P.W, hi);
                x1 = min(lo + bd[p + 1] * P.W, hi);
                nw = bd[p + 1] - bd[p];
            } else {
                class_partition(lo, hi, P.W, p, Pb, x0, x1, nw);
            }
            if (nw < 0 || nw > A.wpc || x1 - x0 > A.spc || x1 < x0) bad = 1;
        }
        for (int s = R.s_begin + threadIdx.x; s < R.s_end; s += GB) {
            const int32_t len = R.tab_off[s + 1] - R.tab_off[s];
            if (R.tab_off[s] < 0 || len < 0 || len > R.max_row) bad = 1;
        }
    }
    bad = __syncthreads_or(bad);
    if (bad && threadIdx.x == 0) atomicCAS(A.X.err, 0, GDI_DEVERR_INPUT);
    return !bad;
}

// E* in 16 bits: the sentinels at the ends of the range (values are 0..max_row < 32000 or -1)
__device__ __forceinline__ int16_t es_encode(int32_t e)
{
    return e == ES_NONE ? (int16_t)INT16_MIN : (e == ES_ALL ? (int16_t)INT16_MAX : (int16_t)e);
}
__device__ __forceinline__ int32_t es_decode(int16_t v)
{
    return v == INT16_MIN ? ES_NONE : (v == INT16_MAX ? ES_ALL : (int32_t)v);
}

// E*(u) of every (rank, replica) of [a0, a1) at sweep sw (table row `row` of length rlen) into rows
// es_out[r * es_s + 4 qq + j] for rank 4 (q0 + qq) + j (q0 = a0 / 4), by the threads t of 0 .. nth - 1
// (nth a multiple of 8).  The draws
// depend on (rank, sweep, replica) and the table row only, so they can be made before the spins of
// the range are known.
__device__ void estar_ahead(const GridArgs &A, const uint32_t *row, int32_t a0, int32_t a1, int sw, int16_t *es_out,
                            int es_s, int32_t rlen, float Tsw, int t, int nth)
{
    if (a1 <= a0) return;
    const int32_t q0 = a0 >> 2, q1 = (a1 - 1) >> 2, nq = q1 - q0 + 1;
    const int r = t & 7;
    if (r >= A.nrep) return;
    for (int32_t qq = t >> 3; qq < nq; qq += nth >> 3) {
        const int32_t qd = q0 + qq;
        const uint4 u4 = philox4x32_10(make_uint4((uint32_t)qd, (uint32_t)sw, 0u, (uint32_t)(A.rep_base + r)),
                                       A.R.key0, A.R.key1);
        uint32_t e[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            e[j] = (uint16_t)es_encode(estar_of(row, rlen, A.R.mode, word_of(u4, j), Tsw));
        *reinterpret_cast<uint2 *>(es_out + (size_t)r * es_s + 4 * qq) = make_uint2(e[0] | (e[1] << 16), e[2] | (e[3] << 16));
    }
}

// Thresholds of the spin range [a0, a1).  all_reps: every replica, threshold of (i, r) stored at
// gam_out[i * gis + r * grs] (fields in hbuf [i*8 + r], rows longer than LONG_ROW summed by a
// warp).  Otherwise only replica `one`, stored at gam_out[i * gis] with fields [i] (thread-serial
// rows; used by the rare exact fallback).  gam_out must hold 8 ints per rank either way (the
// long-row partial sums live there before the thresholds are written).
__device__ void range_thresholds(const GridArgs &A, const GSmem &S, int32_t a0, int32_t a1, int sw,
                                 bool all_reps, int one, int32_t *gam_out, int gis, int grs, uint8_t *s0_out,
                                 int16_t *hbuf, int32_t rlen, float Tsw, bool quad_rows = false,
                                 const int16_t *es_in = nullptr, int es_s = 0, int32_t *gc_out = nullptr,
                                 int32_t gc_val = 0)
{
    const GdiDevProblem &P = A.P;
    const int64_t base = P.node_off[0];
    const uint8_t *packed = A.X.packed;
    const int32_t ns = a1 - a0;
    const int hs = all_reps ? 8 : 1;
    __shared__ int nlong;
    if (threadIdx.x == 0) nlong = 0;
    __syncthreads();
    const bool kept = all_reps && A.hf != nullptr;
    if (kept) {
        // kept fields: the start signs and field words of up to KU ranks per thread are all in
        // flight before any is used (one L2 round trip instead of one per rank)
        constexpr int KU = 2;
        const ulonglong2 *hf2 = reinterpret_cast<const ulonglong2 *>(A.hf) + base + a0;
        for (int32_t i0 = threadIdx.x; i0 < ns; i0 += KU * GB) {
            uint8_t b[KU];
            ulonglong2 v[KU];
#pragma unroll
            for (int u = 0; u < KU; ++u) {
                const int32_t i = i0 + u * GB;
                if (i < ns) {
                    b[u] = __ldcg(packed + base + a0 + i);
                    v[u] = __ldcg(hf2 + i);
                }
            }
#pragma unroll
            for (int u = 0; u < KU; ++u) {
                const int32_t i = i0 + u * GB;
                if (i < ns) {
                    s0_out[i] = b[u];
                    const uint2 lo = field_unword(v[u].x), hi = field_unword(v[u].y);
                    *reinterpret_cast<uint4 *>(hbuf + (size_t)i * 8) = make_uint4(lo.x, lo.y, hi.x, hi.y);
                }
            }
        }
    }
    if (gc_out) gc_out[threadIdx.x] = gc_val;       // the caller's thread t < replicas stores word t
    for (int32_t i = threadIdx.x; i < ns && !kept; i += GB) {
        const int32_t rk = a0 + i;
        s0_out[i] = __ldcg(packed + base + rk);
        const int64_t e0 = P.row_ptr[base + rk], e1 = P.row_ptr[base + rk + 1];
        if (all_reps && e1 - e0 > LONG_ROW) {
            S.longq[atomicAdd(&nlong, 1)] = i;
        } else {
            field8_thread(P, base, e0, e1, packed, all_reps ? hbuf + (size_t)i * 8 : hbuf + i, all_reps ? -1 : one);
        }
    }
    __syncthreads();
    if (all_reps && !kept) {
        // long rows: chunks of LCHUNK entries are warp tasks; partial sums meet in shared memory.
        // acc[i*8 + k] = sum_j w_ij bit_k(j) lives in the threshold array (free until the
        // thresholds are written below); sum_j w_ij lives in the first 4 bytes of the row's
        // field slots; the chunk count of long row t is kept in the histogram area.
        const int nl = nlong;
        int32_t *acc = gam_out;
        int32_t *nchunk = S.nchunk;              // [nl]
        for (int t = threadIdx.x; t < nl; t += GB) {
            const int32_t i = S.longq[t];
            const int64_t deg = P.row_ptr[base + a0 + i + 1] - P.row_ptr[base + a0 + i];
            nchunk[t] = (int32_t)((deg + LCHUNK - 1) / LCHUNK);
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[(size_t)i * 8 + k] = 0;
            *reinterpret_cast<int32_t *>(hbuf + (size_t)i * 8) = 0;
        }
        __syncthreads();
        {
            int task = 0;
            for (int t = 0; t < nl; ++t) {
                const int nc = nchunk[t];
                for (int c = 0; c < nc; ++c, ++task) {
                    if (task % NWARP != warp_id()) continue;
                    const int32_t i = S.longq[t];
                    const int64_t r0 = P.row_ptr[base + a0 + i], r1 = P.row_ptr[base + a0 + i + 1];
                    const int64_t c0 = r0 + (int64_t)c * LCHUNK, c1 = min(r1, c0 + LCHUNK);
                    int32_t swv, sb[8];
                    chunk8_warp(P, base, c0, c1, packed, swv, sb);
                    if ((threadIdx.x & 31) == 0) {
#pragma unroll
                        for (int k = 0; k < 8; ++k) atomicAdd(&acc[(size_t)i * 8 + k], sb[k]);
                        atomicAdd(reinterpret_cast<int32_t *>(hbuf + (size_t)i * 8), swv);
                    }
                }
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nl; t += GB) {
            const int32_t i = S.longq[t];
            const int32_t swv = *reinterpret_cast<const int32_t *>(hbuf + (size_t)i * 8);
#pragma unroll
            for (int k = 0; k < 8; ++k) hbuf[(size_t)i * 8 + k] = (int16_t)(swv - 2 * acc[(size_t)i * 8 + k]);
        }
        __syncthreads();
    }
    if (ns > 0) {
        const int32_t q0 = a0 >> 2, q1 = (a1 - 1) >> 2;
        const int nr = all_reps ? A.nrep : 1;
        const int a_shift = (P.A > 0 && (P.A & (P.A - 1)) == 0) ? 2 + __ffs(P.A) - 1 : -1;   // log2(4A)
        // one Philox block per (quad of ranks, replica)
        auto quad = [&](int32_t qd, int r) {
            const uint4 u4 = philox4x32_10(make_uint4((uint32_t)qd, (uint32_t)sw, 0u,
                                                      (uint32_t)(A.rep_base + r)),
                                           A.R.key0, A.R.key1);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int32_t rk = 4 * qd + j;
                if (rk < a0 || rk >= a1) continue;
                const int32_t i = rk - a0;
                const int sg = ((s0_out[i] >> r) & 1) ? -1 : 1;
                const int32_t h = hbuf[(size_t)i * hs + (all_reps ? r : 0)];
                const int32_t es = estar_of(S.row, rlen, A.R.mode, word_of(u4, j), Tsw);
                gam_out[(size_t)i * gis + (size_t)(all_reps ? r : 0) * grs] =
                    a_shift >= 0 ? gamma_of_shift(sg, h, es, P.A, P.B, a_shift) : gamma_of(sg, h, es, P.A, P.B);
            }
        };
        const int32_t nq = q1 - q0 + 1;
        if (nr == 8 && quad_rows) {
            // rows of stride grs = 4 mod 32 whose element a0 - (a0 mod 4) is 16-byte aligned: the four
            // thresholds of a quad go out in one 16-byte store (ranks outside [a0, a1) store 0)
            const int r = threadIdx.x & 7;
            int32_t *row = gam_out - (a0 & 3) + (size_t)r * grs;
            for (int32_t qq = threadIdx.x >> 3; qq < nq; qq += GB / 8) {
                const int32_t qd = q0 + qq;
                int32_t ev[4];
                if (es_in) {
                    // E* drawn ahead (same rows layout: quad qq at 4 qq)
                    const uint2 w = *reinterpret_cast<const uint2 *>(es_in + (size_t)r * es_s + 4 * qq);
                    ev[0] = es_decode((int16_t)(w.x & 0xFFFFu));
                    ev[1] = es_decode((int16_t)(w.x >> 16));
                    ev[2] = es_decode((int16_t)(w.y & 0xFFFFu));
                    ev[3] = es_decode((int16_t)(w.y >> 16));
                } else {
                    const uint4 u4 = philox4x32_10(make_uint4((uint32_t)qd, (uint32_t)sw, 0u,
                                                              (uint32_t)(A.rep_base + r)),
                                                   A.R.key0, A.R.key1);
#pragma unroll
                    for (int j = 0; j < 4; ++j) ev[j] = estar_of(S.row, rlen, A.R.mode, word_of(u4, j), Tsw);
                }
                int32_t g[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int32_t rk = 4 * qd + j;
                    g[j] = 0;
                    if (rk < a0 || rk >= a1) continue;
                    const int32_t i = rk - a0;
                    const int sg = ((s0_out[i] >> r) & 1) ? -1 : 1;
                    const int32_t h = hbuf[(size_t)i * 8 + r];
                    const int32_t es = ev[j];
                    g[j] = a_shift >= 0 ? gamma_of_shift(sg, h, es, P.A, P.B, a_shift) : gamma_of(sg, h, es, P.A, P.B);
                }
                *reinterpret_cast<int4 *>(row + 4 * qq) = make_int4(g[0], g[1], g[2], g[3]);
            }
        } else if (nr == 8) {
            // a thread keeps one replica (GB is a multiple of 8): no division in the task loop
            const int r = threadIdx.x & 7;
            for (int32_t qq = threadIdx.x >> 3; qq < nq; qq += GB / 8) quad(q0 + qq, r);
        } else {
            for (int32_t t = threadIdx.x; t < nq * nr; t += GB) quad(q0 + t / nr, all_reps ? t % nr : one);
        }
    }
    __syncthreads();
}

// table of one window (positions [ws, we)) for replica r over G in [c - RT, c + RT], by one warp
__device__ void window_table(const GSmem &S, int ws, int we, int r, int32_t c, bool plus_first,
                             int32_t *hp, int32_t *hm, int16_t *tab)
{
    const int lane = threadIdx.x & 31;
    const int64_t base = (int64_t)c - RT - 2 * KC;
    for (int b = lane; b < HB; b += 32) { hp[b] = 0; hm[b] = 0; }
    __syncwarp();
    int32_t under = 0, over = 0;
    for (int i = ws + lane; i < we; i += 32) {
        const bool neg = (S.s0[i] >> r) & 1;
        const int64_t b = (int64_t)S.gam[(size_t)i * 8 + r] - base;
        if (!neg) {
            if (b < 0) ++under;
            else if (b < HB) atomicAdd(&hp[b], 1);
        } else {
            if (b >= HB) ++over;
            else if (b >= 0) atomicAdd(&hm[b], 1);
        }
    }
    under = warp_sum(under);
    over = warp_sum(over);
    __syncwarp();
    warp_cumulate(hp, HB, under, true);     // C(base + b)
    warp_cumulate(hm, HB, over, false);     // D(base + b)
    for (int e = lane; e < TW; e += 32) {
        int64_t g = (int64_t)c - RT + e;
        bool valid = true;
        for (int ph = 0; ph < 2 && valid; ++ph) {
            const bool plus = plus_first ? (ph == 0) : (ph == 1);
            // K = #{k in [0, KC] : count(g -/+ 2k) >= k + 1}; the predicate holds for a prefix of
            // k, so K is found by binary search; K = KC + 1 means the table cannot represent it
            int32_t lo = 0, hi = KC + 1;
            while (lo < hi) {
                const int32_t mid = (lo + hi + 1) >> 1;          // does k = mid - 1 hold?
                const int64_t v = plus ? g - 2 * (mid - 1) : g + 2 * (mid - 1);
                const int32_t cnt = plus ? hp[v - base] : hm[v - base];
                if (cnt >= mid) lo = mid; else hi = mid - 1;
            }
            const int32_t K = lo;
            if (K > KC) valid = false;
            g = plus ? g - 2 * K : g + 2 * K;
        }
        tab[e] = valid ? (int16_t)(g - ((int64_t)c - RT)) : TINV;
    }
    __syncwarp();
}

// exact output G of a window (both groups), by one warp
__device__ int32_t window_exact(const int32_t *gam, int gs, int gc, const uint8_t *s0, int r, int ws,
                                int we, int32_t g, bool plus_first, int32_t *bins)
{
    const int32_t K1 = warp_group(gam, gs, gc, s0, r, ws, we, g, plus_first, bins, nullptr);
    g = plus_first ? g - 2 * K1 : g + 2 * K1;
    const int32_t K2 = warp_group(gam, gs, gc, s0, r, ws, we, g, !plus_first, bins, nullptr);
    return plus_first ? g + 2 * K2 : g - 2 * K2;
}

// G of every replica: n - 2 #(-1), accumulated into X.Gcls (zeroed by the host)
__device__ __noinline__ void init_G(const GridArgs &A, int p, int Pb, int32_t n, int64_t base)
{
    const GdiGridScratch &X = A.X;
    const int lane = threadIdx.x & 31;
    const int nrep = A.nrep;
    int32_t cntm[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int32_t r0 = (int32_t)(((int64_t)p * n) / Pb), r1 = (int32_t)(((int64_t)(p + 1) * n) / Pb);
    for (int32_t i = r0 + threadIdx.x; i < r1; i += GB) {
        const uint8_t b = __ldcg(X.packed + base + i);
#pragma unroll
        for (int k = 0; k < 8; ++k) cntm[k] += (b >> k) & 1;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int32_t m = warp_sum(cntm[k]);
        if (k < nrep && lane == 0 && m) atomicAdd(&X.Gcls[k], -2 * m);
    }
    if (p == 0 && threadIdx.x < nrep) atomicAdd(&X.Gcls[threadIdx.x], n);
}

// digest and cut of every replica after sweep sw (grid-wide atomics), and G after the sweep
// maintained fields of every rank from the packed spins at launch start
__device__ __noinline__ void init_fields(const GridArgs &A, int p, int Pb, int32_t n, int64_t base)
{
    const GdiDevProblem &P = A.P;
    unsigned long long *H = A.hf;
    for (int32_t rk = p * GB + threadIdx.x; rk < n; rk += Pb * GB) {
        const int64_t e0 = P.row_ptr[base + rk], e1 = P.row_ptr[base + rk + 1];
        if (e1 - e0 > LONG_ROW) continue;
        int16_t h[8];
        field8_thread(P, base, e0, e1, A.X.packed, h, -1);
        H[2 * (base + rk)] = field_word(h);
        H[2 * (base + rk) + 1] = field_word(h + 4);
    }
    // rows longer than LONG_ROW: one warp per row, chunk by chunk
    const int lane = threadIdx.x & 31;
    for (int32_t rk = p * NWARP + warp_id(); rk < n; rk += Pb * NWARP) {
        const int64_t e0 = P.row_ptr[base + rk], e1 = P.row_ptr[base + rk + 1];
        if (e1 - e0 <= LONG_ROW) continue;
        int32_t swt = 0, sbt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int64_t c0 = e0; c0 < e1; c0 += LCHUNK) {
            int32_t swv, sb[8];
            chunk8_warp(P, base, c0, min(e1, c0 + (int64_t)LCHUNK), A.X.packed, swv, sb);
            swt += swv;
#pragma unroll
            for (int k = 0; k < 8; ++k) sbt[k] += sb[k];
        }
        if (lane == 0) {
            int16_t h[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) h[k] = (int16_t)(swt - 2 * sbt[k]);
            H[2 * (base + rk)] = field_word(h);
            H[2 * (base + rk) + 1] = field_word(h + 4);
        }
    }
}

__device__ __noinline__ void sweep_trace(const GridArgs &A, int p, int Pb, int32_t n, int64_t base, int sw)
{
    const GdiDevProblem &P = A.P;
    const GdiDevRun &R = A.R;
    const GdiGridScratch &X = A.X;
    const int lane = threadIdx.x & 31;
    const int nrep = A.nrep;
    const int32_t r0 = (int32_t)(((int64_t)p * n) / Pb), r1 = (int32_t)(((int64_t)(p + 1) * n) / Pb);
    uint64_t dg[8];
    int64_t ct[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) { dg[k] = 0; ct[k] = 0; }
    for (int32_t i = r0 + threadIdx.x; i < r1; i += GB) {
        const uint8_t b = __ldcg(X.packed + base + i);
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (k < nrep && !((b >> k) & 1))
                dg[k] += splitmix64_fin((uint64_t)(uint32_t)i | ((uint64_t)(sw & 0xFFFF) << 32) |
                                        ((uint64_t)((A.rep_base + k) & 0xFFFF) << 48));
        const int64_t e0 = P.row_ptr[base + i], e1 = P.row_ptr[base + i + 1];
        for (int64_t e = e0; e < e1; ++e) {
            const uint32_t cc = __ldg(P.col + e);
            const uint32_t j = cc & 0x7FFFFFFFu;
            if ((int32_t)j <= i) continue;
            const uint8_t d = b ^ __ldcg(X.packed + base + j);
            if (!d) continue;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if ((d >> k) & 1) ct[k] += (cc >> 31) ? -1 : 1;
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint64_t a = warp_sum(dg[k]);
        const int64_t b = warp_sum(ct[k]);
        const int64_t o = (int64_t)(A.rep_base + k) * R.sweeps + sw;
        if (k < nrep && lane == 0) {
            if (a) atomicAdd((unsigned long long *)(R.tr_digest + o), (unsigned long long)a);
            if (b) atomicAdd((unsigned long long *)(R.tr_cut + o), (unsigned long long)b);
        }
    }
    if (p == 0 && threadIdx.x < nrep)
        R.tr_G[(int64_t)(A.rep_base + threadIdx.x) * R.sweeps + sw] =
            *(volatile int32_t *)&X.Gcls[threadIdx.x];
}

__global__ void __launch_bounds__(GB, 1) gdi_grid_anneal_kernel(GridArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int chain_pp;
    __shared__ int32_t chain_g;
    const GdiDevProblem &P = A.P;
    const GdiDevRun &R = A.R;
    const GdiGridScratch &X = A.X;
    const int Pb = gridDim.x, p = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const GridLayout L = grid_layout(A.spc, A.wpc, Pb, R.max_row);
    GSmem S;
    S.h = reinterpret_cast<int16_t *>(smem_raw + L.off_h);
    S.gam = reinterpret_cast<int32_t *>(smem_raw + L.off_gam);
    S.s0 = reinterpret_cast<uint8_t *>(smem_raw + L.off_s0);
    S.fm = reinterpret_cast<uint32_t *>(smem_raw + L.off_fm);
    S.longq = reinterpret_cast<int32_t *>(smem_raw + L.off_longq);
    S.wtab = reinterpret_cast<int16_t *>(smem_raw + L.off_wtab);
    S.win = reinterpret_cast<int32_t *>(smem_raw + L.off_win);
    S.hist = reinterpret_cast<int32_t *>(smem_raw + L.off_hist);
    S.nchunk = S.hist;   // spc <= NWARP * 2 * HB, checked by the plan
    S.ctab = reinterpret_cast<int16_t *>(smem_raw + L.off_ctab);
    S.row = reinterpret_cast<uint32_t *>(smem_raw + L.off_row);
    S.misc = reinterpret_cast<int64_t *>(smem_raw + L.off_misc);
    int32_t *Gc = reinterpret_cast<int32_t *>(S.misc);   // [8] class-start G of each replica
    const int64_t base = P.node_off[0];
    const int32_t n = (int32_t)(P.node_off[1] - base);
    const int32_t *cls = P.class_ptr + P.class_off[0];
    const int32_t ncls = P.class_off[1] - P.class_off[0] - 1;
    const int W = P.W;
    const int nrep = A.nrep;

    if (!plan_fits(A)) return;
    init_G(A, p, Pb, n, base);
    if (!grid_sync(X)) return;

    for (int sw = R.s_begin; sw < R.s_end; ++sw) {
        const int32_t roff = R.tab_off[sw];
        const int32_t rlen = R.tab_off[sw + 1] - roff;
        for (int k = threadIdx.x; k < rlen; k += GB) S.row[k] = R.tab[roff + k];
        const float Tsw = R.temp ? R.temp[sw] : 0.f;
        const bool plus_first = (sw & 1) == 0;
        __syncthreads();
        for (int c = 0; c < ncls; ++c) {
            const int32_t lo = cls[c], hi = cls[c + 1];
            int32_t a0, a1;
            int nwin;
            class_partition(lo, hi, W, p, Pb, a0, a1, nwin);
            if (threadIdx.x < nrep) Gc[threadIdx.x] = *(volatile int32_t *)&X.Gcls[threadIdx.x];
            // ---- phase A: thresholds of my windows, window tables, block table
            range_thresholds(A, S, a0, a1, sw, true, 0, S.gam, 8, 1, S.s0, S.h, rlen, Tsw);
            for (int task = warp; task < nwin * nrep; task += NWARP) {
                const int kk = task / nrep, r = task % nrep;
                const int ws = kk * W, we = min(ws + W, a1 - a0);
                window_table(S, ws, we, r, Gc[r], plus_first, S.hist + (size_t)warp * 2 * HB,
                             S.hist + (size_t)warp * 2 * HB + HB, S.wtab + ((size_t)kk * 8 + r) * TW);
            }
            __syncthreads();
            if (warp < nrep) {
                const int r = warp;
                for (int e = lane; e < TW; e += 32) {
                    int32_t idx = e;
                    for (int kk = 0; kk < nwin; ++kk) {
                        if (idx < 0 || idx >= TW) { idx = TINV; break; }
                        const int16_t v = S.wtab[((size_t)kk * 8 + r) * TW + idx];
                        if (v == TINV) { idx = TINV; break; }
                        idx = v;
                    }
                    X.tables[((size_t)p * 8 + r) * TW + e] = (int16_t)idx;
                }
            }
            if (!grid_sync(X)) return;
            // ---- phase C: one block per replica chains the block tables
            if (p < nrep) {
                const int r = p;
                for (int pp = warp; pp < Pb; pp += NWARP) {
                    const int16_t *src = X.tables + ((size_t)pp * 8 + r) * TW;
                    int16_t v[(TW + 31) / 32];
#pragma unroll
                    for (int j = 0; j < (TW + 31) / 32; ++j)
                        v[j] = (lane + 32 * j < TW) ? __ldcg(src + lane + 32 * j) : (int16_t)0;
#pragma unroll
                    for (int j = 0; j < (TW + 31) / 32; ++j)
                        if (lane + 32 * j < TW) S.ctab[(size_t)pp * TW + lane + 32 * j] = v[j];
                }
                const int32_t c0 = Gc[r];
                if (threadIdx.x == 0) { chain_pp = 0; chain_g = c0; }
                __syncthreads();
                while (true) {
                    if (threadIdx.x == 0) {
                        int pp = chain_pp;
                        int32_t g = chain_g;
                        while (pp < Pb) {
                            const int64_t idx = (int64_t)g - ((int64_t)c0 - RT);
                            if (idx < 0 || idx >= TW) break;
                            const int16_t v = S.ctab[(size_t)pp * TW + idx];
                            if (v == TINV) break;
                            X.gin[(size_t)pp * 8 + r] = g;
                            g = (int32_t)((int64_t)c0 - RT + v);
                            ++pp;
                        }
                        chain_pp = pp;
                        chain_g = g;
                    }
                    __syncthreads();
                    const int pp = chain_pp;
                    const int32_t g = chain_g;
                    __syncthreads();
                    if (pp >= Pb) break;
                    // exact fallback for block pp: its thresholds for replica r, recomputed into the
                    // histogram area (free during this phase)
                    if (threadIdx.x == 0) X.gin[(size_t)pp * 8 + r] = g;
                    int32_t b0, b1;
                    int nw2;
                    class_partition(lo, hi, W, pp, Pb, b0, b1, nw2);
                    const int32_t nb = b1 - b0;
                    int32_t *fg = S.hist;
                    int16_t *fh = reinterpret_cast<int16_t *>(fg + nb);
                    uint8_t *fs = reinterpret_cast<uint8_t *>(fh + ((nb + 7) & ~7));
                    int32_t *fbins = reinterpret_cast<int32_t *>(fs + ((nb + 15) & ~15));
                    range_thresholds(A, S, b0, b1, sw, false, r, fg, 1, 0, fs, fh, rlen, Tsw);
                    if (warp == 0) {
                        int32_t gg = g;
                        for (int kk = 0; kk < nw2; ++kk) {
                            const int ws = kk * W, we = min(ws + W, nb);
                            gg = window_exact(fg, 1, 0, fs, r, ws, we, gg, plus_first, fbins);
                        }
                        if (lane == 0) {
                            chain_pp = pp + 1;
                            chain_g = gg;
                            atomicAdd(X.status + r, 1);
                        }
                    }
                    __syncthreads();
                }
                if (threadIdx.x == 0) X.Gcls[r] = chain_g;
            }
            if (!grid_sync(X)) return;
            // ---- phase D: inputs of my windows, then the exact flips of every (window, replica)
            for (int i = threadIdx.x; i < (a1 - a0 + 3) / 4; i += GB) S.fm[i] = 0;
            if (warp < nrep) {
                const int r = warp;
                int32_t g = __ldcg(X.gin + (size_t)p * 8 + r);
                const int32_t cbase = Gc[r] - RT;
                int32_t *bins = S.hist + (size_t)warp * 2 * HB;
                for (int kk = 0; kk < nwin; ++kk) {
                    if (lane == 0) S.win[kk * 8 + r] = g;
                    const int64_t idx = (int64_t)g - cbase;
                    int16_t v = TINV;
                    if (idx >= 0 && idx < TW) v = S.wtab[((size_t)kk * 8 + r) * TW + idx];
                    if (v != TINV) {
                        g = cbase + v;
                    } else {
                        const int ws = kk * W, we = min(ws + W, a1 - a0);
                        g = window_exact(S.gam, 8, r, S.s0, r, ws, we, g, plus_first, bins);
                    }
                }
            }
            __syncthreads();
            for (int task = warp; task < nwin * nrep; task += NWARP) {
                const int kk = task / nrep, r = task % nrep;
                const int ws = kk * W, we = min(ws + W, a1 - a0);
                int32_t *bins = S.hist + (size_t)warp * 2 * HB;
                int32_t g = S.win[kk * 8 + r];
                const int32_t K1 = warp_group(S.gam, 8, r, S.s0, r, ws, we, g, plus_first, bins, S.fm);
                g = plus_first ? g - 2 * K1 : g + 2 * K1;
                warp_group(S.gam, 8, r, S.s0, r, ws, we, g, !plus_first, bins, S.fm);
            }
            __syncthreads();
            for (int32_t i = threadIdx.x; i < a1 - a0; i += GB) {
                const uint8_t f = (uint8_t)(S.fm[i >> 2] >> (8 * (i & 3)));
                if (f) X.packed[base + a0 + i] = S.s0[i] ^ f;
            }
            if (!grid_sync(X)) return;
        }
        if (R.flags & GDI_DEV_TRACE) sweep_trace(A, p, Pb, n, base, sw);
    }
}

// =============================================================================================
// Sorted-window path (1 <= W <= 256).
//
// One warp takes one (window, replica): lanes hold the window's members (up to 8 per lane) with
// keys (group, threshold distance from the class-start G c, position), and a bitonic sort puts
// each group in its flip order.  The k-th member of the +1 group (gamma ascending) flips iff
// G - 2k >= gamma_(k), i.e. iff a_k = gamma_(k) + 2k <= G; a_k is strictly increasing, so for any
// entering G the flips are exactly the members with a_k <= G -- one comparison per member, no
// histogram.  The -1 group likewise flips iff b_k = gamma'_(k) - 2k >= G.  Every member keeps
// rel = a_k - c (or b_k - c) in shared memory; the exact replay of a window is then two warp
// counts.
//
// Block maps: on the lattice x = G - c in {-64, -62, ..., 62} (64 points; G - c is always even) a
// group is a staircase: index j -> ylo + popcount(mask & bits below j), read from where the a_k
// (b_k) fall.  The maps of a block's windows are composed per replica into a 64-entry byte table
// (two lattice points per lane; -1 = leaves the lattice) and published byte by byte with the class
// parity in every byte, so a reader needs no flag.  The last block of every run of 16 blocks also
// composes the run's tables into a run table.  Every block then fetches the run tables before it
// and the block tables of its own run (one poll of all of them per round trip) and looks its exact
// entering G up from c: at most 160 / 16 + 15 byte lookups, without a grid barrier.  Where the walk leaves the lattice, the block whose table failed publishes its exact
// outgoing G (it knows its own entering G and replays exactly), and the walk continues from it.
// One grid barrier per class remains: the next class reads this class's spins.
constexpr int SMAXW = 256;
constexpr int RUN = 16;                 // blocks per run table
__host__ __device__ inline int nruns(int P) { return (P + RUN - 1) / RUN; }
// per replica warp: run tables [nruns] + own-run block tables [RUN] + descent tables [RUN]
__host__ __device__ inline int walk_slots(int P) { return nruns(P) + 2 * RUN; }


struct SortedLayout {
    size_t off_h, off_gam, off_es, off_s0, off_fm, off_fbits, off_longq, off_smap, off_hist, off_walk, off_row,
        off_misc, total;
    int fw;                             // words of one replica's flip bitmap
    int gs;                             // threshold row stride (ints): >= spc + 7, 4 mod 32
    int es;                             // E* row stride (int16): >= spc + 7, 16 mod 32; 0 = no E* rows
};

__host__ __device__ inline SortedLayout sorted_layout(int spc, int wpc, int max_row, int P, bool es_rows)
{
    SortedLayout L;
    size_t o = 0;
    L.off_h = o; o = align16(o + (size_t)spc * 8 * sizeof(int16_t));      // fields, then rel
    // thresholds [r][gs]: a row starts 4 words (16 banks' worth of bytes) after the previous
    // one's bank, so the 8 replicas' 16-byte stores of one quad of ranks hit disjoint banks
    L.gs = ((spc + 3 + 31) & ~31) + 4;
    L.off_gam = o; o = align16(o + (size_t)L.gs * 8 * sizeof(int32_t));
    // E* of the next class's ranks [r][es], drawn ahead by the warps that do not walk
    L.es = es_rows ? ((spc + 3 + 31) & ~31) + 16 : 0;
    L.off_es = o; o = align16(o + (size_t)L.es * 8 * sizeof(int16_t));
    L.off_s0 = o; o = align16(o + (size_t)spc);
    L.off_fm = o; o = align16(o + (size_t)((spc + 3) / 4) * sizeof(uint32_t));
    L.fw = spc / 32 + 2;
    L.off_fbits = o; o = align16(o + (size_t)8 * L.fw * sizeof(uint32_t));
    L.off_longq = o; o = align16(o + (size_t)2 * spc * sizeof(int32_t));   // long rows, chunk counts
    L.off_smap = o; o = align16(o + (size_t)wpc * 8 * 2 * sizeof(StageMap));
    L.off_hist = o; o = align16(o + (size_t)NWARP * HA * sizeof(int32_t));    // exact-replay bins
    L.off_walk = o; o = align16(o + (size_t)8 * walk_slots(P) * NT);
    L.off_row = o; o = align16(o + (size_t)(max_row + 4) * sizeof(uint32_t));
    L.off_misc = o; o = align16(o + 64 * sizeof(int64_t));
    L.total = o;
    return L;
}

// chain buffers carved from the scratch table area: exact outgoing G [P][8] (epoch << 32 | G),
// block tables [P][8][64], run tables [NR][8][64]
__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
__host__ __device__ inline size_t chain_off_tab(int P) { return align256((size_t)P * 8 * sizeof(uint64_t)); }
__host__ __device__ inline size_t chain_off_rtab(int P) { return chain_off_tab(P) + (size_t)P * 8 * NT; }
__host__ __device__ inline size_t chain_bytes(int P) { return chain_off_rtab(P) + (size_t)nruns(P) * 8 * NT; }

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// bounded wait for an exact G word of this epoch: false (error word set) after X.spin_limit polls
// or when another block failed
__device__ __forceinline__ bool wait_exact(const unsigned long long *f, uint32_t epoch, const GdiGridScratch &X,
                                           int32_t &g)
{
    long long spins = 0;
    unsigned long long v;
    while (((v = ld_acquire_u64(f)) >> 32) != epoch) {
        if (++spins > X.spin_limit) { atomicExch(X.err, GDI_DEVERR_TIMEOUT); return false; }
        if ((spins & 63) == 0 && *(volatile int *)X.err) return false;
        __nanosleep(32);
    }
    g = (int32_t)(uint32_t)v;
    return true;
}

// Published tables carry the class parity in bit 7 of every byte and the entry (-1 .. 63, -1 as
// 0x7F) in the low 7 bits.  A byte is atomic on its own, so a reader that sees the parity of the
// current class in all 64 bytes has the whole table: no flag, and one round trip per poll.  The
// bytes of the previous class hold the other parity, and the chain area is zeroed at launch
// (parity 0) while the first class has parity 1.
__device__ __forceinline__ void st_tab_byte(int8_t *p, int v, uint32_t par)
{
    const uint32_t b = ((uint32_t)v & 0x7Fu) | par;
    asm volatile("st.relaxed.gpu.global.u8 [%0], %1;" ::"l"(p), "r"(b) : "memory");
}

__device__ __forceinline__ uint4 ld_tab16(const int8_t *p)
{
    uint4 v;
    // no memory clobber: the four loads of a table may be in flight together; volatile keeps
    // every poll's loads
    asm volatile("ld.relaxed.gpu.global.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// four table bytes: the low 7 bits, 0x7F mapped to 0xFF (-1)
__device__ __forceinline__ uint32_t tab_decode(uint32_t w)
{
    const uint32_t v = w & 0x7F7F7F7Fu;
    return v | ((v + 0x01010101u) & 0x80808080u);
}

// warp: copies the tables a + k * stride (k < na) to da + k * NT and b + k * stride (k < nb) to
// db + k * NT, decoded, once every byte of them carries the parity `par` (lane k < na + nb <= 32
// reads one table per poll).  Bounded wait; false on timeout or when another block failed.
__device__ bool fetch_valid(const int8_t *a, int na, int8_t *da, const int8_t *b, int nb, int8_t *db,
                            size_t stride, uint32_t par, const GdiGridScratch &X)
{
    const int lane = threadIdx.x & 31;
    const int8_t *src = nullptr;
    int8_t *dst = nullptr;
    if (lane < na) {
        src = a + (size_t)lane * stride;
        dst = da + (size_t)lane * NT;
    } else if (lane < na + nb) {
        src = b + (size_t)(lane - na) * stride;
        dst = db + (size_t)(lane - na) * NT;
    }
    const uint32_t want = par ? 0x80808080u : 0u;
    long long spins = 0;
    bool ok = true;
    for (;;) {
        // every poll copies the decoded bytes; the last poll, where all are current, stays
        bool good = true;
        if (src) {
            const uint4 v0 = ld_tab16(src), v1 = ld_tab16(src + 16), v2 = ld_tab16(src + 32),
                        v3 = ld_tab16(src + 48);
            const uint32_t m = (v0.x & v0.y & v0.z & v0.w & v1.x & v1.y & v1.z & v1.w & v2.x & v2.y & v2.z &
                                v2.w & v3.x & v3.y & v3.z & v3.w) & 0x80808080u;
            const uint32_t o = (v0.x | v0.y | v0.z | v0.w | v1.x | v1.y | v1.z | v1.w | v2.x | v2.y | v2.z |
                                v2.w | v3.x | v3.y | v3.z | v3.w) & 0x80808080u;
            good = par ? m == want : o == want;
            uint4 *d4 = reinterpret_cast<uint4 *>(dst);
            d4[0] = make_uint4(tab_decode(v0.x), tab_decode(v0.y), tab_decode(v0.z), tab_decode(v0.w));
            d4[1] = make_uint4(tab_decode(v1.x), tab_decode(v1.y), tab_decode(v1.z), tab_decode(v1.w));
            d4[2] = make_uint4(tab_decode(v2.x), tab_decode(v2.y), tab_decode(v2.z), tab_decode(v2.w));
            d4[3] = make_uint4(tab_decode(v3.x), tab_decode(v3.y), tab_decode(v3.z), tab_decode(v3.w));
        }
        if (__all_sync(0xFFFFFFFFu, good)) break;
        if (++spins > X.spin_limit) {
            if (lane == 0) atomicExch(X.err, GDI_DEVERR_TIMEOUT);
            ok = false;
            break;
        }
        if ((spins & 63) == 0 && __any_sync(0xFFFFFFFFu, *(volatile int *)X.err != 0)) {
            ok = false;
            break;
        }
        __nanosleep(20);
    }
    __syncwarp();
    return ok;
}

// SL = members per lane of a window sort (1, 2, 4 or 8): one instantiation per window size class
template <int SL>
__global__ void __launch_bounds__(GB, 1) gdi_grid_sorted_kernel(GridArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const GdiDevProblem &P = A.P;
    const GdiDevRun &R = A.R;
    const GdiGridScratch &X = A.X;
    const int Pb = gridDim.x, p = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int spc = A.spc;
    const SortedLayout L = sorted_layout(spc, A.wpc, R.max_row, Pb, A.es_pre);
    int16_t *hb = reinterpret_cast<int16_t *>(smem_raw + L.off_h);   // fields [i*8 + r], then rel [r*spc + i]
    int32_t *gam = reinterpret_cast<int32_t *>(smem_raw + L.off_gam);
    int16_t *esb = reinterpret_cast<int16_t *>(smem_raw + L.off_es);   // E* drawn ahead [r][L.es]
    uint8_t *s0 = smem_raw + L.off_s0;
    uint32_t *fm = reinterpret_cast<uint32_t *>(smem_raw + L.off_fm);
    StageMap *smap = reinterpret_cast<StageMap *>(smem_raw + L.off_smap);
    int32_t *hist = reinterpret_cast<int32_t *>(smem_raw + L.off_hist);
    int8_t *walk = reinterpret_cast<int8_t *>(smem_raw + L.off_walk);
    uint32_t *fbits = reinterpret_cast<uint32_t *>(smem_raw + L.off_fbits);   // [r][fw] fast-path flips
    GSmem S = {};
    S.longq = reinterpret_cast<int32_t *>(smem_raw + L.off_longq);
    S.hist = hist;
    S.nchunk = S.longq + spc;
    S.row = reinterpret_cast<uint32_t *>(smem_raw + L.off_row);
    S.misc = reinterpret_cast<int64_t *>(smem_raw + L.off_misc);
    int32_t *Gc = reinterpret_cast<int32_t *>(S.misc);   // [8] class-start G of each replica
    unsigned char *cb = reinterpret_cast<unsigned char *>(X.tables);
    unsigned long long *exg = reinterpret_cast<unsigned long long *>(cb);
    int8_t *tabs = reinterpret_cast<int8_t *>(cb + chain_off_tab(Pb));
    int8_t *rtabs = reinterpret_cast<int8_t *>(cb + chain_off_rtab(Pb));
    const int NR = nruns(Pb);
    const int run = p / RUN, run0 = run * RUN;
    const bool leader = (p % RUN == RUN - 1) || p == Pb - 1;
    const int64_t base = P.node_off[0];
    const int32_t n = (int32_t)(P.node_off[1] - base);
    const int32_t *cls = P.class_ptr + P.class_off[0];
    const int32_t ncls = P.class_off[1] - P.class_off[0] - 1;
    const int W = P.W;
    const int nrep = A.nrep;

    if (!plan_fits(A)) return;
    init_G(A, p, Pb, n, base);
    if (A.hf) init_fields(A, p, Pb, n, base);
    if (!grid_sync(X)) return;
    __shared__ int npush;

    // my ranks [x0, x1) of class cc (kept in shared memory for the first CB_MAX classes, so that a
    // class starts without a global round trip for its bounds)
    auto class_range_g = [&](int cc, int32_t &x0, int32_t &x1, int &nw) {
        const int32_t lo = cls[cc], hi = cls[cc + 1];
        if (A.wbnd) {
            const int32_t *bd = A.wbnd + (size_t)cc * (Pb + 1);
            x0 = min(lo + bd[p] * W, hi);
            x1 = min(lo + bd[p + 1] * W, hi);
            nw = bd[p + 1] - bd[p];
        } else {
            class_partition(lo, hi, W, p, Pb, x0, x1, nw);
        }
    };
    constexpr int CB_MAX = 64;
    __shared__ int32_t cbnd[3 * CB_MAX];
    for (int cc = threadIdx.x; cc < ncls && cc < CB_MAX; cc += GB) {
        int32_t x0, x1;
        int nw;
        class_range_g(cc, x0, x1, nw);
        cbnd[3 * cc] = x0;
        cbnd[3 * cc + 1] = x1;
        cbnd[3 * cc + 2] = nw;
    }
    auto class_range = [&](int cc, int32_t &x0, int32_t &x1, int &nw) {
        if (cc < CB_MAX) {
            x0 = cbnd[3 * cc];
            x1 = cbnd[3 * cc + 1];
            nw = cbnd[3 * cc + 2];
        } else {
            class_range_g(cc, x0, x1, nw);
        }
    };
    uint32_t epoch = 0;
    bool have_es = false;                      // esb holds E* of the current class's ranks
    for (int sw = R.s_begin; sw < R.s_end; ++sw) {
        const int32_t roff = R.tab_off[sw];
        const int32_t rlen = R.tab_off[sw + 1] - roff;
        for (int k = threadIdx.x; k < rlen; k += GB) S.row[k] = R.tab[roff + k];
        const float Tsw = R.temp ? R.temp[sw] : 0.f;
        const bool plus_first = (sw & 1) == 0;
        __syncthreads();
        for (int c = 0; c < ncls; ++c) {
            ++epoch;
            const uint32_t par = (epoch & 1u) << 7;        // parity of this class's table bytes
            int32_t a0, a1;
            int nwin;
            class_range(c, a0, a1, nwin);
            const int32_t ns = a1 - a0;
            // the class-start G (written by the last block of the previous class) is loaded here
            // and stored inside the threshold phase, so its round trip overlaps the field loads
            const int32_t gcl = threadIdx.x < nrep ? *(volatile int32_t *)&X.Gcls[threadIdx.x] : 0;
            // ---- thresholds of my ranks (ends with a block barrier)
            // thresholds of rank a0 + i for replica r at gamc[r * gs + i]
            int32_t *gamc = gam + (a0 & 3);
            range_thresholds(A, S, a0, a1, sw, true, 0, gamc, 1, L.gs, s0, hb, rlen, Tsw, true,
                             have_es ? esb : nullptr, L.es, threadIdx.x < nrep ? Gc : nullptr, gcl);
            // ---- sorted groups: rel values and stage maps of every (window, replica)
            for (int task = warp; task < nwin * nrep; task += NWARP) {
                const int kk = task / nrep, r = task % nrep;
                const int ws = kk * W, wlen = min(W, ns - ws);
                const int32_t *gr = gamc + (size_t)r * L.gs;
                int16_t *rr = hb + (size_t)r * spc;
                StageMap *o = smap + ((size_t)kk * 8 + r) * 2;
                window_maps<SL>(gr, s0, rr, ws, wlen, r, Gc[r], o);
            }
            for (int i = threadIdx.x; i < (ns + 3) / 4; i += GB) fm[i] = 0;
            for (int i = threadIdx.x; i < 8 * L.fw; i += GB) fbits[i] = 0;
            if (threadIdx.x == 0) npush = 0;
            __syncthreads();
            // ---- block table per replica: lanes hold lattice points lane and lane + 32
            int t0 = lane, t1 = lane + 32;
            if (warp < nrep) {
                const int r = warp;
                for (int kk = 0; kk < nwin; ++kk) {
#pragma unroll
                    for (int ph = 0; ph < 2; ++ph) {
                        const StageMap m = smap[((size_t)kk * 8 + r) * 2 + (plus_first ? ph : 1 - ph)];
                        t0 = stage_apply(m, t0);
                        t1 = stage_apply(m, t1);
                    }
                }
                int8_t *dst = tabs + ((size_t)p * 8 + r) * NT;
                st_tab_byte(dst + lane, t0, par);
                st_tab_byte(dst + lane + 32, t1, par);
            }
            // ---- the last block of a run composes the run's block tables into the run table
            bool ok = true;
            if (leader) {
                if (warp < nrep) {
                    const int r = warp;
                    int8_t *dt = walk + ((size_t)r * walk_slots(Pb) + NR + RUN) * NT;   // descent slots
                    const int cnt = p - run0;                 // blocks of the run before me
                    ok = fetch_valid(tabs + ((size_t)run0 * 8 + r) * NT, cnt, dt, nullptr, 0, nullptr,
                                     (size_t)8 * NT, par, X);
                    if (ok) {
                        int u0 = lane, u1 = lane + 32;
                        for (int k = 0; k < cnt; ++k) {
                            if (u0 >= 0) u0 = dt[k * NT + u0];
                            if (u1 >= 0) u1 = dt[k * NT + u1];
                        }
                        // then my own table (lane l holds T[l], T[l + 32])
                        const int x00 = __shfl_sync(0xFFFFFFFFu, t0, u0 & 31);
                        const int x01 = __shfl_sync(0xFFFFFFFFu, t1, u0 & 31);
                        const int x10 = __shfl_sync(0xFFFFFFFFu, t0, u1 & 31);
                        const int x11 = __shfl_sync(0xFFFFFFFFu, t1, u1 & 31);
                        u0 = u0 < 0 ? -1 : (u0 >= 32 ? x01 : x00);
                        u1 = u1 < 0 ? -1 : (u1 >= 32 ? x11 : x10);
                        int8_t *rd = rtabs + ((size_t)run * 8 + r) * NT;
                        st_tab_byte(rd + lane, u0, par);
                        st_tab_byte(rd + lane + 32, u1, par);
                    }
                }
            }
            // ---- entering G: run tables of the runs before mine, then the block tables of my run
            if (warp < nrep) {
                const int r = warp;
                const int32_t c0 = Gc[r];
                int8_t *ws_run = walk + (size_t)r * walk_slots(Pb) * NT;    // [NR][64]
                int8_t *ws_own = ws_run + (size_t)NR * NT;                   // [RUN][64]
                int8_t *ws_dsc = ws_own + (size_t)RUN * NT;                  // [RUN][64]
                const int nown = p - run0;
                if (ok) {
                    const int8_t *ra = rtabs + (size_t)r * NT, *ob = tabs + ((size_t)run0 * 8 + r) * NT;
                    if (run + nown <= 32) {
                        ok = fetch_valid(ra, run, ws_run, ob, nown, ws_own, (size_t)8 * NT, par, X);
                    } else {
                        ok = fetch_valid(ra, run, ws_run, nullptr, 0, nullptr, (size_t)8 * NT, par, X) &&
                             fetch_valid(ob, nown, ws_own, nullptr, 0, nullptr, (size_t)8 * NT, par, X);
                    }
                }
                int idx = NT / 2;          // lattice index of the running G, or -1 when off the lattice
                int32_t gx = c0;           // the running G when off the lattice
                // one block step: its table, or its exact outgoing G where the table cannot map
                auto block_step = [&](const int8_t *t, int j) {
                    const int nidx = idx >= 0 ? (int)t[idx] : -1;
                    if (nidx >= 0) { idx = nidx; return; }
                    int32_t v = 0;
                    ok = wait_exact(exg + (size_t)j * 8 + r, epoch, X, v);
                    gx = v;
                    const int32_t xr = gx - c0;
                    idx = (xr >= -NT && xr <= NT - 2) ? (xr + NT) >> 1 : -1;
                };
                for (int q = 0; q < run && ok; ++q) {
                    const int nidx = idx >= 0 ? (int)ws_run[q * NT + idx] : -1;
                    if (nidx >= 0) { idx = nidx; continue; }
                    // the run table cannot map the running G: walk the run block by block
                    ok = fetch_valid(tabs + ((size_t)q * RUN * 8 + r) * NT, RUN, ws_dsc, nullptr, 0, nullptr,
                                     (size_t)8 * NT, par, X);
                    for (int k = 0; k < RUN && ok; ++k) block_step(ws_dsc + k * NT, q * RUN + k);
                    __syncwarp();
                }
                for (int k = 0; k < nown && ok; ++k) block_step(ws_own + k * NT, run0 + k);
                ok = __all_sync(0xFFFFFFFFu, ok);
                if (ok) {
                    const int32_t gin = idx >= 0 ? c0 - NT + 2 * idx : gx;
                    const int own = __shfl_sync(0xFFFFFFFFu, (idx >= 0 && idx < 32) ? t0 : t1, idx & 31);
                    const bool need_exact = idx < 0 || own < 0;
                    uint32_t *fb = fbits + (size_t)r * L.fw;
                    int32_t x = gin - c0;
                    const int32_t *gr = gamc + (size_t)r * L.gs;
                    const int16_t *rr = hb + (size_t)r * spc;
                    int32_t *bins = hist + (size_t)warp * HA;
                    for (int kk = 0; kk < nwin; ++kk) {
                        const int ws = kk * W, we = min(ws + W, ns);
                        // a narrow window's rel values hold on the lattice only (see window_maps)
                        const bool on = smap[((size_t)kk * 8 + r) * 2].narrow ? (x >= -NT && x <= NT - 2)
                                                                            : (x >= -FAST_X && x <= FAST_X);
                        x = on ? replay_window<SL>(rr, s0, r, ws, we, x, plus_first, fb, W)
                               : window_replay_exact(gr, s0, r, ws, we, c0 + x, plus_first, bins, fm) - c0;
                    }
                    const int32_t gout = c0 + x;
                    if (lane == 0) {
                        if (need_exact) {
                            st_release_u64(exg + (size_t)p * 8 + r,
                                           ((unsigned long long)epoch << 32) | (uint32_t)gout);
                            atomicAdd(X.status + r, 1);
                        }
                        if (p == Pb - 1) X.Gcls[r] = gout;
                    }
                }
            } else if (A.es_pre && (c + 1 < ncls || sw + 1 < R.s_end)) {
                // the warps that do not walk draw the next class's E* meanwhile (after the last
                // class: the next sweep's first class, from that sweep's table row)
                const bool same = c + 1 < ncls;
                const int sn = same ? sw : sw + 1;
                int32_t b0, b1;
                int nwb;
                class_range(same ? c + 1 : 0, b0, b1, nwb);
                const int32_t ro = R.tab_off[sn];
                estar_ahead(A, same ? S.row : R.tab + ro, b0, b1, sn, esb, L.es,
                            same ? rlen : R.tab_off[sn + 1] - ro, same ? Tsw : (R.temp ? R.temp[sn] : 0.f),
                            threadIdx.x - nrep * 32, GB - nrep * 32);
            }
            have_es = A.es_pre && (c + 1 < ncls || sw + 1 < R.s_end);
            __syncthreads();
            // ---- write the flips; with maintained fields, push their field changes to the
            // neighbours: a warp takes 32 consecutive ranks and walks the concatenated rows of its
            // flipping ones lane by lane (rows longer than LONG_ROW go to a block queue instead)
            uint32_t *pq = reinterpret_cast<uint32_t *>(S.longq);
            // row bounds of the next chunk are loaded while the current one is pushed
            int64_t nrow0 = 0, nrow1 = 0;
            if (A.hf && warp * 32 + lane < ns) {
                nrow0 = __ldg(P.row_ptr + base + a0 + warp * 32 + lane);
                nrow1 = __ldg(P.row_ptr + base + a0 + warp * 32 + lane + 1);
            }
            for (int32_t i0 = warp * 32; i0 < ns; i0 += GB) {
                const int32_t i = i0 + lane;
                const int64_t row0 = nrow0, row1 = nrow1;
                if (A.hf && i + GB < ns) {
                    nrow0 = __ldg(P.row_ptr + base + a0 + i + GB);
                    nrow1 = __ldg(P.row_ptr + base + a0 + i + GB + 1);
                }
                uint32_t f = 0;
                if (i < ns) {
                    f = (fm[i >> 2] >> (8 * (i & 3))) & 0xFFu;
                    for (int r = 0; r < nrep; ++r) f |= ((fbits[(size_t)r * L.fw + (i >> 5)] >> (i & 31)) & 1u) << r;
                }
                if (f) X.packed[base + a0 + i] = (uint8_t)(s0[i] ^ f);
                if (!A.hf || !__any_sync(0xFFFFFFFFu, f != 0)) continue;
                int64_t e0 = 0;
                int32_t d = 0;
                unsigned long long d0 = 0, d1 = 0;
                if (f) {
                    e0 = row0;
                    d = (int32_t)(row1 - row0);
                    if (d > LONG_ROW) {
                        pq[atomicAdd(&npush, 1)] = (uint32_t)i | (f << 24);
                        d = 0;
                    } else {
                        flip_words(f, s0[i], d0, d1);
                    }
                }
                int32_t incl = d;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                    if (lane >= o) incl += t;
                }
                const int32_t excl = incl - d;
                const int32_t tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
                for (int32_t k0 = 0; k0 < tot; k0 += 4 * 32) {
                    uint32_t cc[4];
                    unsigned long long w0[4], w1[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        // owner of entry k: the last lane whose rows start at or before k
                        const int32_t k = k0 + 32 * u + lane;
                        int src = 0;
#pragma unroll
                        for (int st = 16; st > 0; st >>= 1)
                            if (__shfl_sync(0xFFFFFFFFu, excl, src + st) <= k) src += st;
                        const int64_t oe = __shfl_sync(0xFFFFFFFFu, e0, src);
                        const int32_t ox = __shfl_sync(0xFFFFFFFFu, excl, src);
                        w0[u] = __shfl_sync(0xFFFFFFFFu, d0, src);
                        w1[u] = __shfl_sync(0xFFFFFFFFu, d1, src);
                        cc[u] = k < tot ? __ldg(P.col + oe + (k - ox)) : 0u;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (k0 + 32 * u + lane >= tot) continue;
                        unsigned long long *w = A.hf + 2 * (base + (int64_t)(cc[u] & 0x7FFFFFFFu));
                        const bool neg = (cc[u] >> 31) != 0;
                        if (w0[u]) atomicAdd(w, neg ? 0ull - w0[u] : w0[u]);
                        if (w1[u]) atomicAdd(w + 1, neg ? 0ull - w1[u] : w1[u]);
                    }
                }
            }
            if (A.hf) {
                __syncthreads();
                const int nq = npush;
                for (int t = warp; t < nq; t += NWARP) {
                    const uint32_t q = pq[t];
                    const int32_t i = (int32_t)(q & 0xFFFFFFu);
                    unsigned long long d0, d1;
                    flip_words(q >> 24, s0[i], d0, d1);
                    const int64_t e0 = P.row_ptr[base + a0 + i], e1 = P.row_ptr[base + a0 + i + 1];
                    for (int64_t eb = e0; eb < e1; eb += 4 * 32) {
                        uint32_t cc[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int64_t e = eb + 32 * u + lane;
                            cc[u] = e < e1 ? __ldg(P.col + e) : 0u;
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            if (eb + 32 * u + lane >= e1) continue;
                            unsigned long long *w = A.hf + 2 * (base + (int64_t)(cc[u] & 0x7FFFFFFFu));
                            const bool neg = (cc[u] >> 31) != 0;
                            if (d0) atomicAdd(w, neg ? 0ull - d0 : d0);
                            if (d1) atomicAdd(w + 1, neg ? 0ull - d1 : d1);
                        }
                    }
                }
            }
            if (!grid_sync(X)) return;
        }
        if (R.flags & GDI_DEV_TRACE) {
            sweep_trace(A, p, Pb, n, base, sw);
            // a block may start writing the next sweep's spins before every block has read this
            // sweep's (it waits only for the blocks before it), so the trace gets its own barrier
            if (!grid_sync(X)) return;
        }
    }
}

// Algorithm 3 as printed (GDI_FLAG_RACY): inside a colour class every spin decides at once on the
// G it reads at that moment -- +1 flips iff G >= gamma, -1 iff G <= gamma', the same thresholds
// (and Philox draws) as the serialised path -- and adds its change to G with an atomic, so a spin
// sees the flips whose atomics landed before its read and not the others.  Not deterministic;
// the windows play no part (W only sizes the blocks' shares).  One grid barrier per class.
__global__ void __launch_bounds__(GB, 1) gdi_grid_racy_kernel(GridArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const GdiDevProblem &P = A.P;
    const GdiDevRun &R = A.R;
    const GdiGridScratch &X = A.X;
    const int Pb = gridDim.x, p = blockIdx.x;
    const int spc = A.spc;
    const SortedLayout L = sorted_layout(spc, A.wpc, R.max_row, Pb, A.es_pre);
    int16_t *hb = reinterpret_cast<int16_t *>(smem_raw + L.off_h);
    int32_t *gam = reinterpret_cast<int32_t *>(smem_raw + L.off_gam);
    uint8_t *s0 = smem_raw + L.off_s0;
    uint32_t *fm = reinterpret_cast<uint32_t *>(smem_raw + L.off_fm);
    GSmem S = {};
    S.longq = reinterpret_cast<int32_t *>(smem_raw + L.off_longq);
    S.hist = reinterpret_cast<int32_t *>(smem_raw + L.off_hist);
    S.nchunk = S.longq + spc;
    S.row = reinterpret_cast<uint32_t *>(smem_raw + L.off_row);
    S.misc = reinterpret_cast<int64_t *>(smem_raw + L.off_misc);
    const int64_t base = P.node_off[0];
    const int32_t n = (int32_t)(P.node_off[1] - base);
    const int32_t *cls = P.class_ptr + P.class_off[0];
    const int32_t ncls = P.class_off[1] - P.class_off[0] - 1;
    const int nrep = A.nrep;

    if (!plan_fits(A)) return;
    init_G(A, p, Pb, n, base);
    if (!grid_sync(X)) return;
    for (int sw = R.s_begin; sw < R.s_end; ++sw) {
        const int32_t roff = R.tab_off[sw];
        const int32_t rlen = R.tab_off[sw + 1] - roff;
        for (int k = threadIdx.x; k < rlen; k += GB) S.row[k] = R.tab[roff + k];
        const float Tsw = R.temp ? R.temp[sw] : 0.f;
        __syncthreads();
        for (int c = 0; c < ncls; ++c) {
            int32_t a0, a1;
            int nwin;
            if (A.wbnd) {
                const int32_t *bd = A.wbnd + (size_t)c * (Pb + 1);
                a0 = min(cls[c] + bd[p] * P.W, cls[c + 1]);
                a1 = min(cls[c] + bd[p + 1] * P.W, cls[c + 1]);
            } else {
                class_partition(cls[c], cls[c + 1], P.W, p, Pb, a0, a1, nwin);
            }
            const int32_t ns = a1 - a0;
            range_thresholds(A, S, a0, a1, sw, true, 0, gam, 1, spc, s0, hb, rlen, Tsw);
            for (int i = threadIdx.x; i < (ns + 3) / 4; i += GB) fm[i] = 0;
            __syncthreads();
            for (int r = 0; r < nrep; ++r) {
                for (int32_t i = threadIdx.x; i < ns; i += GB) {
                    const int32_t gm = gam[(size_t)r * spc + i];
                    const bool neg = (s0[i] >> r) & 1;
                    const int32_t g = *(volatile int32_t *)&X.Gcls[r];
                    if (neg ? g <= gm : g >= gm) {
                        atomicAdd(&X.Gcls[r], neg ? 2 : -2);
                        atomicOr(&fm[i >> 2], 1u << (8 * (i & 3) + r));
                    }
                }
            }
            __syncthreads();
            for (int32_t i = threadIdx.x; i < ns; i += GB) {
                const uint32_t f = (fm[i >> 2] >> (8 * (i & 3))) & 0xFFu;
                if (f) X.packed[base + a0 + i] = (uint8_t)(s0[i] ^ f);
            }
            if (!grid_sync(X)) return;
        }
        if (R.flags & GDI_DEV_TRACE) {
            sweep_trace(A, p, Pb, n, base, sw);
            if (!grid_sync(X)) return;
        }
    }
}

__global__ void set_word_kernel(unsigned int *p, unsigned int v) { *p = v; }


// ---------------------------------------------------------------------------------------------
// replica group <-> int8 spins in rank space
__global__ void pack_kernel(int8_t *spins, int64_t N, int rep_base, int nrep, uint8_t *packed)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t b = 0;
        for (int r = 0; r < nrep; ++r) b |= (spins[(int64_t)(rep_base + r) * N + i] < 0 ? 1u : 0u) << r;
        packed[i] = (uint8_t)b;
    }
}

__global__ void unpack_kernel(int8_t *spins, int64_t N, int rep_base, int nrep, const uint8_t *packed)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t b = packed[i];
        for (int r = 0; r < nrep; ++r) spins[(int64_t)(rep_base + r) * N + i] = ((b >> r) & 1) ? -1 : 1;
    }
}

// cut of every replica of a group from the packed spins, in one pass over the CSR: for an entry
// (i, j > i), d = b_i ^ b_j has bit r set where replica r cuts the edge; SWAR byte lanes count the
// cut weights (flushed before they can overflow)
__global__ void packed_cut_kernel(GdiDevProblem P, const uint8_t *packed, int nrep, int64_t *cut)
{
    const int64_t base = P.node_off[0];
    const int64_t n = P.node_off[1] - base;
    int64_t acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t b = packed[base + i];
        uint64_t aP = 0, aN = 0;
        int cnt = 0;
        const int64_t e1 = P.row_ptr[base + i + 1];
        for (int64_t e = P.row_ptr[base + i]; e < e1; ++e) {
            const uint32_t c = __ldg(P.col + e);
            const uint32_t j = c & 0x7FFFFFFFu;
            if ((int64_t)j <= i) continue;
            const uint64_t sv = spread8((uint32_t)(b ^ packed[base + j]));
            if (c >> 31) aN += sv; else aP += sv;
            if (++cnt == 255) {
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    acc[k] += (int64_t)((aP >> (8 * k)) & 0xFF) - (int64_t)((aN >> (8 * k)) & 0xFF);
                aP = aN = 0;
                cnt = 0;
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += (int64_t)((aP >> (8 * k)) & 0xFF) - (int64_t)((aN >> (8 * k)) & 0xFF);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int64_t v = warp_sum(acc[k]);
        if (k < nrep && (threadIdx.x & 31) == 0 && v) atomicAdd((unsigned long long *)(cut + k), (unsigned long long)v);
    }
}

// ---------------------------------------------------------------------------------------------
// exact-balance repair of a single large instance, replica by replica (int8 spins)
__device__ __forceinline__ int32_t field_i8(const GdiDevProblem &P, const int8_t *s, int64_t r)
{
    int32_t h = 0;
    for (int64_t e = P.row_ptr[r]; e < P.row_ptr[r + 1]; ++e) {
        const uint32_t c = __ldg(P.col + e);
        const int32_t v = s[c & 0x7FFFFFFFu];
        h += (c >> 31) ? -v : v;
    }
    return h;
}

// per replica: k = (|G| - n mod 2) / 2 majority spins with the smallest (s h, rank) keys flip.
// rp[r*4 + 0..3] = k, majority sign, kappa (smallest key with count(key <= kappa) >= k), t (ties)
__global__ void repair_hist_kernel(GdiDevProblem P, const int8_t *spins, int nrep, const int32_t *G,
                                   int32_t *hist, int32_t D)
{
    const int64_t N = P.N;
    for (int r = 0; r < nrep; ++r) {
        const int32_t g = G[r];
        const int32_t tgt = (int32_t)(N & 1);
        if ((g < 0 ? -g : g) <= tgt) continue;
        const int8_t maj = g > 0 ? 1 : -1;
        const int8_t *s = spins + (int64_t)r * N;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
            if (s[i] != maj) continue;
            const int32_t key = maj * field_i8(P, s, i);
            atomicAdd(&hist[(int64_t)r * (2 * D + 1) + key + D], 1);
        }
    }
}

__global__ void repair_select_kernel(const int32_t *G, int64_t N, const int32_t *hist, int32_t D, int32_t *rp)
{
    const int r = blockIdx.x;
    if (threadIdx.x != 0) return;
    const int32_t g = G[r];
    const int32_t tgt = (int32_t)(N & 1);
    const int32_t ag = g < 0 ? -g : g;
    int32_t k = ag > tgt ? (ag - tgt) / 2 : 0;
    rp[r * 4 + 0] = k;
    rp[r * 4 + 1] = g > 0 ? 1 : -1;
    rp[r * 4 + 2] = 0;
    rp[r * 4 + 3] = 0;
    if (k == 0) return;
    int32_t run = 0;
    for (int32_t b = 0; b < 2 * D + 1; ++b) {
        const int32_t hb = hist[(int64_t)r * (2 * D + 1) + b];
        if (run + hb >= k) {
            rp[r * 4 + 2] = b - D;
            rp[r * 4 + 3] = k - run;
            return;
        }
        run += hb;
    }
}

// ties (key == kappa) per block in rank order, then the flip flags
__global__ void repair_ties_kernel(GdiDevProblem P, const int8_t *spins, int nrep, const int32_t *rp,
                                   int32_t *ties, int64_t chunk)
{
    const int64_t N = P.N;
    const int64_t i0 = (int64_t)blockIdx.x * chunk, i1 = min(N, i0 + chunk);
    for (int r = 0; r < nrep; ++r) {
        if (rp[r * 4] == 0) { if (threadIdx.x == 0) ties[(int64_t)r * gridDim.x + blockIdx.x] = 0; continue; }
        const int8_t maj = (int8_t)rp[r * 4 + 1];
        const int32_t kappa = rp[r * 4 + 2];
        const int8_t *s = spins + (int64_t)r * N;
        int32_t c = 0;
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x)
            if (s[i] == maj && maj * field_i8(P, s, i) == kappa) ++c;
        c = warp_sum(c);
        __shared__ int32_t acc;
        if (threadIdx.x == 0) acc = 0;
        __syncthreads();
        if ((threadIdx.x & 31) == 0) atomicAdd(&acc, c);
        __syncthreads();
        if (threadIdx.x == 0) ties[(int64_t)r * gridDim.x + blockIdx.x] = acc;
        __syncthreads();
    }
}

__global__ void repair_mark_kernel(GdiDevProblem P, const int8_t *spins, int nrep, const int32_t *rp,
                                   const int32_t *ties, int64_t chunk, uint8_t *flags)
{
    // blockDim.x == 256; ranks of the chunk are visited in rounds of 256 in rank order
    const int64_t N = P.N;
    const int64_t i0 = (int64_t)blockIdx.x * chunk, i1 = min(N, i0 + chunk);
    __shared__ int32_t before;
    __shared__ int32_t wsum[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = 0; r < nrep; ++r) {
        if (rp[r * 4] == 0) continue;
        const int8_t maj = (int8_t)rp[r * 4 + 1];
        const int32_t kappa = rp[r * 4 + 2], t = rp[r * 4 + 3];
        const int8_t *s = spins + (int64_t)r * N;
        if (threadIdx.x == 0) {
            int32_t b = 0;
            for (int q = 0; q < (int)blockIdx.x; ++q) b += ties[(int64_t)r * gridDim.x + q];
            before = b;
        }
        __syncthreads();
        int32_t run = before;
        for (int64_t j0 = i0; j0 < i1; j0 += 256) {
            const int64_t i = j0 + threadIdx.x;
            bool strict = false, tie = false;
            if (i < i1 && s[i] == maj) {
                const int32_t key = maj * field_i8(P, s, i);
                strict = key < kappa;
                tie = key == kappa;
            }
            const unsigned m = __ballot_sync(0xFFFFFFFFu, tie);
            if (lane == 0) wsum[warp] = __popc(m);
            __syncthreads();
            int32_t off = run;
            for (int w = 0; w < warp; ++w) off += wsum[w];
            const int32_t idx = off + __popc(m & ((1u << lane) - 1u));
            int32_t tot = 0;
            for (int w = 0; w < 8; ++w) tot += wsum[w];
            if (strict || (tie && idx < t)) flags[i] |= (uint8_t)(1u << r);
            run += tot;
            __syncthreads();
        }
    }
}

__global__ void repair_apply_kernel(int8_t *spins, int64_t N, int nrep, const uint8_t *flags, const int32_t *rp,
                                    int32_t *G)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t f = flags[i];
        if (!f) continue;
        for (int r = 0; r < nrep; ++r)
            if ((f >> r) & 1) spins[(int64_t)r * N + i] = (int8_t)(-spins[(int64_t)r * N + i]);
    }
    if (blockIdx.x == 0 && threadIdx.x < nrep) {
        const int r = threadIdx.x;
        G[r] = G[r] - 2 * rp[r * 4 + 1] * rp[r * 4 + 0];
    }
}

}  // namespace

// ---------------------------------------------------------------------------------------------
int gdi_grid_plan(const GdiDevProblem &P, int max_row, int sms, size_t smem_limit, int *spc, int *wpc,
                  size_t *smem)
{
    if (P.num_instances != 1 || P.W < 1) return -1;
    // the kernels' static shared memory (class bounds, a few words) counts against the same limit
    smem_limit = smem_limit > 2048 ? smem_limit - 2048 : 0;
    // windows per block under an even split: the largest class decides
    const int wp = (int)((P.max_class + P.W - 1) / P.W);
    const int w = (wp + sms - 1) / sms;
    *wpc = w < 1 ? 1 : w;
    *spc = *wpc * P.W;
    if (P.W <= SMAXW) {
        // the cost-weighted split stays within the even share of windows per block: more shared
        // memory per block (less L1) costs more than the finer balance gains
        // with rows for the E* drawn ahead when they fit, else without
        *smem = sorted_layout(*spc, *wpc, max_row, sms, true).total;
        if (*smem <= smem_limit) return 0;
        *smem = sorted_layout(*spc, *wpc, max_row, sms, false).total;
        return *smem <= smem_limit ? 0 : -1;
    }
    // the tabulated path keeps the long rows' chunk counts in the histogram area, and its exact
    // chain fallback the thresholds, fields, start signs and bins of one block's windows (one
    // replica)
    if ((size_t)*spc > (size_t)NWARP * 2 * HB) return -1;
    if ((size_t)*spc * 7 + 64 + HA * sizeof(int32_t) > (size_t)NWARP * 2 * HB * sizeof(int32_t)) return -1;
    *smem = grid_layout(*spc, *wpc, sms, max_row).total;
    return *smem <= smem_limit ? 0 : -1;
}

constexpr double LAST_SHARE = 0.6;

void gdi_grid_window_bounds(const int64_t *cost, const int64_t *cost_off, int num_classes, int blocks,
                            int wpc, int32_t *bnd)
{
    for (int c = 0; c < num_classes; ++c) {
        const int64_t *w = cost + cost_off[c];
        const int nw = (int)(cost_off[c + 1] - cost_off[c]);
        int32_t *K = bnd + (size_t)c * (blocks + 1);
        int64_t total = 0;
        for (int k = 0; k < nw; ++k) total += w[k];
        // ideal cut before block p: the window boundary nearest to p shares of the class's cost,
        // where the last block takes LAST_SHARE of a share: it walks last, so its replay and push
        // end the class
        int k = 0;
        int64_t pre = 0;
        K[0] = 0;
        for (int p = 1; p < blocks; ++p) {
            const double target = (double)total * p / (blocks - 1 + LAST_SHARE);
            while (k < nw && (double)(pre + w[k]) <= target) pre += w[k++];
            int cut = k;
            if (k < nw && (double)(pre + w[k]) - target < target - (double)pre) cut = k + 1;
            K[p] = cut;
        }
        K[blocks] = nw;
        // at most wpc windows per block: clamp to what the blocks before and after can hold
        for (int p = 0; p <= blocks; ++p) {
            const int64_t lo = (int64_t)nw - (int64_t)(blocks - p) * wpc;
            const int64_t hi = (int64_t)p * wpc;
            int64_t v = K[p];
            if (v < lo) v = lo;
            if (v > hi) v = hi;
            if (p > 0 && v < K[p - 1]) v = K[p - 1];
            K[p] = (int32_t)v;
        }
        for (int p = 0; p < blocks; ++p)
            if (K[p + 1] > K[p] + wpc) K[p + 1] = K[p] + wpc;
    }
}

int gdi_launch_grid_anneal(const GdiDevProblem &P, const GdiDevRun &R, const GdiGridScratch &X,
                           int8_t *spins, int sms, int spc, int wpc, size_t smem, const int32_t *wbnd,
                           GdiKernelTimer *timer, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    const bool racy = (R.flags & GDI_DEV_RACY) != 0;
    const bool sorted = P.W <= SMAXW && !racy;
    if (racy) smem = sorted_layout(spc, wpc, R.max_row, sms, false).total;
    const void *kern = racy ? (const void *)gdi_grid_racy_kernel
                     : !sorted ? (const void *)gdi_grid_anneal_kernel
                     : P.W <= 32 ? (const void *)gdi_grid_sorted_kernel<1>
                     : P.W <= 64 ? (const void *)gdi_grid_sorted_kernel<2>
                     : P.W <= 128 ? (const void *)gdi_grid_sorted_kernel<4>
                                  : (const void *)gdi_grid_sorted_kernel<8>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, GB, smem);
    if (e != cudaSuccess) return (int)e;
    if (per_sm < 1) return (int)cudaErrorCooperativeLaunchTooLarge;
    // the sorted path's chain buffers (exact G, flags, byte tables) live in the table area
    if (sorted && chain_bytes(sms) > (size_t)sms * 8 * TW * sizeof(int16_t)) return (int)cudaErrorInvalidValue;
    const int pg = (int)((P.N + 255) / 256) < 4096 ? (int)((P.N + 255) / 256) : 4096;
    for (int g0 = 0; g0 < P.replicas; g0 += 8) {
        const int nrep = P.replicas - g0 < 8 ? P.replicas - g0 : 8;
        pack_kernel<<<pg, 256, 0, st>>>(spins, P.N, g0, nrep, X.packed);
        cudaMemsetAsync(X.Gcls, 0, 8 * sizeof(int32_t), st);
        cudaMemsetAsync(X.bar, 0, 4 * sizeof(unsigned int), st);
        if (X.bar_start) set_word_kernel<<<1, 1, 0, st>>>(X.bar + 2, 1u);
        if (sorted) cudaMemsetAsync(X.tables, 0, chain_bytes(sms), st);
        GridArgs A;
        A.P = P;
        A.R = R;
        A.X = X;
        A.rep_base = g0;
        A.nrep = nrep;
        A.spc = spc;
        A.wpc = wpc;
        A.wbnd = (sorted || racy) ? wbnd : nullptr;
        A.hf = sorted ? X.hfield : nullptr;
        A.es_pre = sorted && R.max_row < 32000 && smem >= sorted_layout(spc, wpc, R.max_row, sms, true).total;
        void *args[] = {&A};
        const bool timed = timer && timer->ev && timer->n < timer->cap;
        if (timed) cudaEventRecord(timer->ev[2 * timer->n], st);
        e = cudaLaunchCooperativeKernel(kern, dim3(sms), dim3(GB), args, smem, st);
        if (e != cudaSuccess) return (int)e;
        if (timed) cudaEventRecord(timer->ev[2 * timer->n++ + 1], st);
        if (R.raw_cut) {
            cudaMemsetAsync(R.raw_cut + g0, 0, nrep * sizeof(int64_t), st);
            packed_cut_kernel<<<152 * 4, 256, 0, st>>>(P, X.packed, nrep, R.raw_cut + g0);
        }
        unpack_kernel<<<pg, 256, 0, st>>>(spins, P.N, g0, nrep, X.packed);
        e = cudaMemcpyAsync(R.raw_G + g0, X.Gcls, nrep * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return (int)e;
    }
    return (int)cudaGetLastError();
}

// raw cut, repair, final cut, final G of a single instance (all replicas)
int gdi_launch_grid_finish(const GdiDevProblem &P, const GdiDevRun &R, const GdiGridScratch &X,
                           int8_t *spins, int do_repair, void *stream)
{
    // the raw cut was taken from the packed spins right after each group's anneal launch
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = 152 * 4;
    const int64_t N = P.N;
    const int D = P.max_degree;
    cudaError_t e = cudaMemcpyAsync(R.final_G, R.raw_G, P.replicas * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return (int)e;
    if (!do_repair) {
        e = cudaMemcpyAsync(R.final_cut, R.raw_cut, P.replicas * sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
        return e != cudaSuccess ? (int)e : (int)cudaGetLastError();
    }
    const int pg = (int)((N + 255) / 256) < 4096 ? (int)((N + 255) / 256) : 4096;
    for (int g0 = 0; g0 < P.replicas; g0 += 8) {
        const int nrep = P.replicas - g0 < 8 ? P.replicas - g0 : 8;
        int8_t *sp = spins + (int64_t)g0 * N;
        GdiDevProblem Q = P;
        cudaMemsetAsync(X.rhist, 0, (size_t)nrep * (2 * D + 1) * sizeof(int32_t), st);
        cudaMemsetAsync(X.rflags, 0, (size_t)N, st);
        repair_hist_kernel<<<nb, 256, 0, st>>>(Q, sp, nrep, R.final_G + g0, X.rhist, D);
        repair_select_kernel<<<nrep, 32, 0, st>>>(R.final_G + g0, N, X.rhist, D, X.rparams);
        const int64_t chunk = (N + nb - 1) / nb;
        repair_ties_kernel<<<nb, 256, 0, st>>>(Q, sp, nrep, X.rparams, X.rties, chunk);
        repair_mark_kernel<<<nb, 256, 0, st>>>(Q, sp, nrep, X.rparams, X.rties, chunk, X.rflags);
        repair_apply_kernel<<<nb, 256, 0, st>>>(sp, N, nrep, X.rflags, X.rparams, R.final_G + g0);
        // final cut of the group from its repaired spins, packed again
        pack_kernel<<<pg, 256, 0, st>>>(spins, N, g0, nrep, X.packed);
        cudaMemsetAsync(R.final_cut + g0, 0, nrep * sizeof(int64_t), st);
        packed_cut_kernel<<<nb, 256, 0, st>>>(P, X.packed, nrep, R.final_cut + g0);
    }
    return (int)cudaGetLastError();
}

