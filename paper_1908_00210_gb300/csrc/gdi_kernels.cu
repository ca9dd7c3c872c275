// gdi_kernels.cu -- sm_103a kernels of libgdi.so: the GDI annealing sweep (Algorithm 3 of
// Cook, Jin, Tan, arXiv:1908.00210), its initial state, the exact-balance repair and the cut.
//
// CTA-resident path: one thread block anneals one (instance, replica) at a time with the whole
// spin vector in shared memory (int8 per vertex); the rank-space CSR streams from L2/HBM.  The
// block loops over its work items (persistent), sweeps, colour classes and windows without
// leaving the kernel, so an anneal of M sweeps is one launch.
//
// Work items are taken from a size-sorted queue (an atomic counter over the largest-first order),
// so long instances start first and short ones fill the tail.
//
// Per window (a chunk of W consecutive ranks of one colour class):
//   1. thresholds: for every spin, the local field h_i = sum_j w_ij s_j over its CSR row (Eq. 2),
//      a Philox4x32-10 draw u_i, the largest energy change E*(u_i) that the draw accepts (binary
//      search of the table row), and from it the flip threshold in G:
//        s_i = +1 flips iff G >= gamma_i = ceil((B h_i + 4A - E*) / 4A)
//        s_i = -1 flips iff G <= gamma_i = floor((E* + B h_i - 4A) / 4A)
//      (dE = B s_i h_i + 4A (1 - s_i G), Eq. 4-6 with G counting the other spins).
//   2. the +1 group and the -1 group of the window each see the exact running G in threshold
//      order (Algorithm 3's atomically updated G, serialised): with d_i = G - gamma_i (+1 group) or
//      gamma_i - G (-1 group), the k-th spin in d-descending order flips iff d_(k) >= 2k.  The
//      number of flips K and the cut-off d* come from a shared-memory histogram of d with suffix
//      sums; ties at d* are resolved by rank with a block prefix count.
//   3. G changes by -2K (+1 group) or +2K (-1 group): one shared-memory update per group, the
//      block-level analogue of the paper's atomicAdd on G.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gdi_device.cuh"
#include "gdi_internal.h"
#include "gdi_window.cuh"

namespace {

using namespace gdi;
using namespace gdi::win;

// ---------------------------------------------------------------------------------------------
struct Smem {
    int8_t *sig;        // [max_n] spins of the current item, rank order
    int8_t *s0;         // [max_window] group (sign at window start) of each window position
    int8_t *flag;       // [max_n] repair decisions
    int32_t *gam;       // [max_window] flip thresholds
    int32_t *hist;      // [H] histogram of d / suffix counts
    uint32_t *row;      // [max_row] table row of the current sweep
    int32_t *red32;     // [BS/32 + 2]
    int64_t *red64;     // [BS/32 + 2]
    int32_t *G;         // running magnetisation of the item
};

// h_i = sum_j w_ij s_j over the CSR row of local rank r (Eq. 2)
__device__ __forceinline__ int32_t local_field(const GdiDevProblem &P, int64_t base, int32_t r,
                                               const int8_t *sig)
{
    const int64_t e0 = P.row_ptr[base + r], e1 = P.row_ptr[base + r + 1];
    int32_t h = 0;
    for (int64_t e = e0; e < e1; ++e) {
        const uint32_t c = __ldg(P.col + e);
        const int32_t s = sig[c & 0x7FFFFFFFu];
        h += (c >> 31) ? -s : s;
    }
    return h;
}

// the same sum over the 16-bit column copy (instances of at most 32,767 vertices)
__device__ __forceinline__ int32_t local_field16(const GdiDevProblem &P, int64_t base, int32_t r,
                                                 const int8_t *sig)
{
    const int64_t e0 = P.row_ptr[base + r], e1 = P.row_ptr[base + r + 1];
    int32_t h = 0;
    for (int64_t e = e0; e < e1; ++e) {
        const uint32_t c = __ldg(P.col16 + e);
        const int32_t s = sig[c & 0x7FFFu];
        h += (c >> 15) ? -s : s;
    }
    return h;
}

// count of members of group grp with d >= x (exact d), block-wide
template <int BS>
__device__ int32_t count_ge(const Smem &S, int32_t Wn, int grp, int32_t Gc, int64_t x)
{
    int32_t c = 0;
    for (int32_t p = threadIdx.x; p < Wn; p += BS) {
        if (S.s0[p] != grp) continue;
        const int64_t d = grp > 0 ? (int64_t)Gc - S.gam[p] : (int64_t)S.gam[p] - Gc;
        c += (d >= x);
    }
    return block_sum<BS, int32_t>(c, S.red32);
}

// Decide the flips of one group of a window and apply them (see file header, step 2).
template <int BS>
__device__ void select_and_flip(const Smem &S, int32_t wlo, int32_t Wn, int grp, int H)
{
    __syncthreads();
    const int32_t Gc = *S.G;
    for (int32_t b = threadIdx.x; b < H; b += BS) S.hist[b] = 0;
    __syncthreads();
    for (int32_t p = threadIdx.x; p < Wn; p += BS) {
        if (S.s0[p] != grp) continue;
        const int32_t d = grp > 0 ? Gc - S.gam[p] : S.gam[p] - Gc;
        if (d >= 0) atomicAdd(&S.hist[d < H - 1 ? d : H - 1], 1);
    }
    __syncthreads();
    // suffix sums in place: hist[x] := #{members with min(d, H-1) >= x}
    {
        const int32_t c = (H + BS - 1) / BS;
        const int32_t b0 = threadIdx.x * c;
        const int32_t b1 = min(b0 + c, H);
        int32_t loc = 0;
        for (int32_t b = b0; b < b1; ++b) loc += S.hist[b];
        int32_t total;
        const int32_t before = block_excl_scan<BS>(loc, S.red32, &total);
        int32_t run = total - before;
        for (int32_t b = b0; b < b1; ++b) {
            const int32_t hb = S.hist[b];
            S.hist[b] = run;
            run -= hb;
        }
    }
    __syncthreads();
    const int32_t n_top = S.hist[H - 1];
    const bool safe = n_top <= (H - 1) / 2 + 1;
    int32_t K, t;
    int64_t dstar;
    if (safe) {
        int32_t cnt = 0;
        for (int32_t k = threadIdx.x; 2 * k <= H - 1; k += BS) cnt += (S.hist[2 * k] >= k + 1);
        K = block_sum<BS, int32_t>(cnt, S.red32);
        if (K == 0) return;
        int32_t cx = 0;
        for (int32_t x = threadIdx.x; x < H; x += BS) cx += (S.hist[x] >= K);
        dstar = block_sum<BS, int32_t>(cx, S.red32) - 1;
        const int32_t above = (dstar + 1 <= H - 1) ? S.hist[dstar + 1] : 0;
        t = K - above;
    } else {
        // exact counting passes (rare: more than H/2 members far above the running G)
        const int32_t n0 = count_ge<BS>(S, Wn, grp, Gc, 0);
        int32_t lo = 0, hi = n0 - 1;
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (count_ge<BS>(S, Wn, grp, Gc, 2 * (int64_t)mid) >= mid + 1) lo = mid; else hi = mid - 1;
        }
        K = lo + 1;
        int64_t dl = 2 * (int64_t)(K - 1), dh = (int64_t)1 << 32;
        while (dl < dh) {
            const int64_t mid = (dl + dh + 1) >> 1;
            if (count_ge<BS>(S, Wn, grp, Gc, mid) >= K) dl = mid; else dh = mid - 1;
        }
        dstar = dl;
        t = K - count_ge<BS>(S, Wn, grp, Gc, dstar + 1);
    }
    // apply: contiguous position chunks so that the tie prefix follows rank order
    const int32_t chunk = (Wn + BS - 1) / BS;
    const int32_t p0 = threadIdx.x * chunk;
    const int32_t p1 = min(p0 + chunk, Wn);
    int32_t ties = 0;
    for (int32_t p = p0; p < p1; ++p) {
        if (S.s0[p] != grp) continue;
        int64_t d = grp > 0 ? (int64_t)Gc - S.gam[p] : (int64_t)S.gam[p] - Gc;
        if (safe && d > H - 1) d = H - 1;
        ties += (d == dstar);
    }
    int32_t total;
    int32_t idx = block_excl_scan<BS>(ties, S.red32, &total);
    for (int32_t p = p0; p < p1; ++p) {
        if (S.s0[p] != grp) continue;
        int64_t d = grp > 0 ? (int64_t)Gc - S.gam[p] : (int64_t)S.gam[p] - Gc;
        if (safe && d > H - 1) d = H - 1;
        bool flip = d > dstar;
        if (d == dstar) flip = (idx++ < t);
        if (flip) S.sig[wlo + p] = (int8_t)(-grp);
    }
    __syncthreads();
    if (threadIdx.x == 0) *S.G = Gc - 2 * grp * K;
}

// Algorithm 2 (the paper's standard annealer, GDI_FLAG_STANDARD): every spin of the window forms
// the balance term from the complete graph of Eq. 5, i.e. sums all n spins itself (an O(n) read per
// spin, which is what the decoupled G of Algorithm 3 removes), on the state at the window start,
// and flips iff its draw accepts dE = B s h + 4A (1 - s G) -- the same test as "G >= gamma" with
// the threshold gamma of step 1.  All decisions are taken before any spin of the window changes.
template <int BS>
__device__ void standard_window(const Smem &S, int32_t wlo, int32_t Wn, int32_t n)
{
    __syncthreads();
    int32_t dG = 0;
    // the spin vector is read in 4-byte words from its first 4-byte boundary on (the shared
    // layout aligns it to 8 bytes only); the bytes before and after are read one by one
    const int32_t head = (int32_t)((4 - (reinterpret_cast<uintptr_t>(S.sig) & 3)) & 3) < n
                             ? (int32_t)((4 - (reinterpret_cast<uintptr_t>(S.sig) & 3)) & 3) : n;
    const int32_t nwords = (n - head) >> 2;
    const int32_t *sw = reinterpret_cast<const int32_t *>(S.sig + head);
    for (int32_t p = threadIdx.x; p < Wn; p += BS) {
        int32_t G = 0;                              // sum of all spins, read by this spin
        for (int32_t j = 0; j < head; ++j) G += S.sig[j];
        for (int32_t k = 0; k < nwords; ++k) G += __dp4a(sw[k], 0x01010101, 0);
        for (int32_t j = head + 4 * nwords; j < n; ++j) G += S.sig[j];
        const int sg = S.s0[p];
        const bool flip = sg > 0 ? G >= S.gam[p] : G <= S.gam[p];
        S.flag[wlo + p] = flip ? 1 : 0;
        dG += flip ? -2 * sg : 0;
    }
    dG = block_sum<BS, int32_t>(dG, S.red32);
    for (int32_t p = threadIdx.x; p < Wn; p += BS)
        if (S.flag[wlo + p]) S.sig[wlo + p] = (int8_t)(-S.s0[p]);
    __syncthreads();
    if (threadIdx.x == 0) *S.G += dG;
}

// cut of the item: (1/2) sum_i sum_j w_ij [s_i != s_j]
template <int BS>
__device__ int64_t item_cut(const GdiDevProblem &P, int64_t base, int32_t n, const Smem &S)
{
    int64_t c = 0;
    for (int32_t r = threadIdx.x; r < n; r += BS) {
        const int8_t sr = S.sig[r];
        const int64_t e0 = P.row_ptr[base + r], e1 = P.row_ptr[base + r + 1];
        for (int64_t e = e0; e < e1; ++e) {
            const uint32_t cc = __ldg(P.col + e);
            if (S.sig[cc & 0x7FFFFFFFu] != sr) c += (cc >> 31) ? -1 : 1;
        }
    }
    return block_sum<BS, int64_t>(c, S.red64) / 2;
}

// #majority spins with repair key (s_i h_i) <= x, and with key == x (when eq != null)
template <int BS>
__device__ int32_t repair_count(const GdiDevProblem &P, int64_t base, int32_t n, const Smem &S,
                                int maj, int64_t x, bool strict)
{
    int32_t c = 0;
    for (int32_t r = threadIdx.x; r < n; r += BS) {
        if (S.sig[r] != maj) continue;
        const int64_t key = (int64_t)maj * local_field(P, base, r, S.sig);
        c += strict ? (key < x) : (key <= x);
    }
    return block_sum<BS, int32_t>(c, S.red32);
}

// Exact-balance repair: flip the k majority spins with the smallest (s_i h_i, rank) keys.
template <int BS>
__device__ void repair(const GdiDevProblem &P, int64_t base, int32_t n, const Smem &S)
{
    __syncthreads();
    const int32_t G = *S.G;
    const int32_t target = n & 1;
    const int32_t aG = G < 0 ? -G : G;
    if (aG <= target) return;
    const int32_t k = (aG - target) / 2;
    const int maj = G > 0 ? 1 : -1;
    // kappa = smallest key value with count(key <= kappa) >= k ; keys lie in [-deg, deg]
    int64_t lo = -(int64_t)P.max_degree - 1, hi = (int64_t)P.max_degree + 1;
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (repair_count<BS>(P, base, n, S, maj, mid, false) >= k) hi = mid; else lo = mid + 1;
    }
    const int64_t kappa = lo;
    const int32_t less = repair_count<BS>(P, base, n, S, maj, kappa, true);
    const int32_t t = k - less;
    const int32_t chunk = (n + BS - 1) / BS;
    const int32_t p0 = threadIdx.x * chunk, p1 = min(p0 + chunk, n);
    // keys of my chunk are recomputed below before any spin of the item changes: compute flags first
    int32_t ties = 0;
    for (int32_t r = p0; r < p1; ++r) {
        if (S.sig[r] != maj) continue;
        ties += ((int64_t)maj * local_field(P, base, r, S.sig) == kappa);
    }
    int32_t total;
    int32_t idx = block_excl_scan<BS>(ties, S.red32, &total);
    // decide every flip before writing any spin (keys are defined on the pre-repair state)
    for (int32_t r = p0; r < p1; ++r) {
        int8_t f = 0;
        if (S.sig[r] == maj) {
            const int64_t key = (int64_t)maj * local_field(P, base, r, S.sig);
            bool flip = key < kappa;
            if (key == kappa) flip = (idx++ < t);
            f = flip ? 1 : 0;
        }
        S.flag[r] = f;
    }
    __syncthreads();
    for (int32_t r = threadIdx.x; r < n; r += BS)
        if (S.flag[r]) S.sig[r] = (int8_t)(-maj);
    __syncthreads();
    if (threadIdx.x == 0) *S.G = G - 2 * maj * k;
    __syncthreads();
}

template <int BS>
__global__ void __launch_bounds__(BS) gdi_cta_anneal_kernel(GdiDevProblem P, GdiDevRun R, int H)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem S;
    {
        unsigned char *p = smem_raw;
        S.red64 = reinterpret_cast<int64_t *>(p); p += sizeof(int64_t) * (BS / 32 + 2);
        S.red32 = reinterpret_cast<int32_t *>(p); p += sizeof(int32_t) * (BS / 32 + 2);
        S.G = reinterpret_cast<int32_t *>(p); p += 16;
        S.hist = reinterpret_cast<int32_t *>(p); p += sizeof(int32_t) * H;
        S.gam = reinterpret_cast<int32_t *>(p); p += sizeof(int32_t) * ((P.max_window + 3) & ~3);
        S.row = reinterpret_cast<uint32_t *>(p); p += sizeof(uint32_t) * ((R.max_row + 3) & ~3);
        S.s0 = reinterpret_cast<int8_t *>(p); p += (P.max_window + 15) & ~15;
        S.sig = reinterpret_cast<int8_t *>(p); p += (P.max_n + 15) & ~15;
        S.flag = reinterpret_cast<int8_t *>(p);
    }
    const int32_t items = P.num_instances * P.replicas;
    __shared__ int32_t next_item;
    while (true) {
        // persistent blocks take (instance, replica) items from a queue sorted by size, largest
        // first; items are independent, so the assignment does not change any result
        __syncthreads();
        if (threadIdx.x == 0) next_item = atomicAdd(R.item_counter, 1);
        __syncthreads();
        const int32_t slot = next_item;
        if (slot >= items) break;
        const int32_t item = R.item_order[slot];
        const int32_t q = item / P.replicas;
        const int32_t rep = item - q * P.replicas;
        const int64_t base = P.node_off[q];
        const int32_t n = (int32_t)(P.node_off[q + 1] - base);
        const int32_t *cls = P.class_ptr + P.class_off[q];
        const int32_t ncls = P.class_off[q + 1] - P.class_off[q] - 1;
        int8_t *gsig = R.spins + (int64_t)rep * P.N + base;

        int32_t g = 0;
        for (int32_t r = threadIdx.x; r < n; r += BS) {
            const int8_t s = gsig[r];
            S.sig[r] = s;
            g += s;
        }
        g = block_sum<BS, int32_t>(g, S.red32);
        if (threadIdx.x == 0) *S.G = g;
        __syncthreads();

        for (int32_t sw = R.s_begin; sw < R.s_end; ++sw) {
            const int32_t roff = R.tab_off[sw];
            const int32_t rlen = R.tab_off[sw + 1] - roff;
            for (int32_t k = threadIdx.x; k < rlen; k += BS) S.row[k] = R.tab[roff + k];
            const float Tsw = R.temp ? R.temp[sw] : 0.f;
            __syncthreads();
            for (int32_t c = 0; c < ncls; ++c) {
                const int32_t clo = cls[c], chi = cls[c + 1];
                const int32_t Wn0 = P.W > 0 ? P.W : (chi - clo);
                for (int32_t wlo = clo; wlo < chi; wlo += Wn0) {
                    const int32_t whi = min(wlo + Wn0, chi);
                    const int32_t Wn = whi - wlo;
                    // step 1: thresholds, one Philox call per aligned quad of ranks
                    const int32_t q0 = wlo >> 2, q1 = (whi - 1) >> 2;
                    for (int32_t qd = q0 + threadIdx.x; qd <= q1; qd += BS) {
                        const uint4 u4 = philox4x32_10(
                            make_uint4((uint32_t)qd, (uint32_t)sw, (uint32_t)q, (uint32_t)rep),
                            R.key0, R.key1);
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int32_t r = 4 * qd + j;
                            if (r < wlo || r >= whi) continue;
                            const int sg = S.sig[r];
                            const int32_t h = local_field(P, base, r, S.sig);
                            const int32_t es = estar_of(S.row, rlen, R.mode, word_of(u4, j), Tsw);
                            S.gam[r - wlo] = gamma_of(sg, h, es, P.A, P.B);
                            S.s0[r - wlo] = (int8_t)sg;
                        }
                    }
                    if (R.flags & GDI_DEV_STANDARD) {
                        standard_window<BS>(S, wlo, Wn, n);
                        continue;
                    }
                    // step 2/3: the two groups in the canonical order (+1 first on even sweeps)
                    const int first = (sw & 1) ? -1 : 1;
                    select_and_flip<BS>(S, wlo, Wn, first, H);
                    select_and_flip<BS>(S, wlo, Wn, -first, H);
                    __syncthreads();
                }
            }
            if (R.flags & GDI_DEV_TRACE) {
                uint64_t dg = 0;
                for (int32_t r = threadIdx.x; r < n; r += BS)
                    if (S.sig[r] > 0)
                        dg += splitmix64_fin((uint64_t)(uint32_t)r | ((uint64_t)(sw & 0xFFFF) << 32) |
                                             ((uint64_t)(rep & 0xFFFF) << 48));
                dg = block_sum<BS, uint64_t>(dg, reinterpret_cast<uint64_t *>(S.red64));
                const int64_t ct = item_cut<BS>(P, base, n, S);
                if (threadIdx.x == 0) {
                    const int64_t o = (int64_t)item * R.sweeps + sw;
                    R.tr_digest[o] = dg;
                    R.tr_G[o] = *S.G;
                    R.tr_cut[o] = ct;
                }
            }
            __syncthreads();
        }
        // outputs before and after the exact-balance repair
        const int64_t raw_cut = item_cut<BS>(P, base, n, S);
        __syncthreads();
        const int32_t raw_G = *S.G;
        if (!(R.flags & GDI_DEV_NO_REPAIR)) repair<BS>(P, base, n, S);
        const int64_t fin_cut = item_cut<BS>(P, base, n, S);
        __syncthreads();
        if (threadIdx.x == 0) {
            R.raw_G[item] = raw_G;
            R.raw_cut[item] = raw_cut;
            R.final_G[item] = *S.G;
            R.final_cut[item] = fin_cut;
        }
        for (int32_t r = threadIdx.x; r < n; r += BS) gsig[r] = S.sig[r];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------------
// CTA-resident sorted-window kernel (1 <= W <= 256): the same results as gdi_cta_anneal_kernel with
// far fewer block barriers per window.  Per colour class: the thresholds of the class's ranks
// (fields gathered from the shared spins); every warp sorts whole windows of the class
// (window_maps: one comparison value per member, valid for any G entering the window, and the
// window's stage maps on the lattice, gdi_window.cuh); one thread walks the stage maps from the
// class-start G, every window entered on the lattice is replayed at once by its own warp -- two
// rounds of ballots -- and the rest in rank order; then the flips are applied.  The windows of a
// class share no edge, so only the running G passes from one window to the next.  SL = members per
// lane of a window.
struct SortedCta {
    int32_t *gam;       // [max_class] flip thresholds of the class
    int16_t *rel;       // [max_class] comparison values
    uint8_t *s0;        // [max_class] 1 = the member was -1 at window start
    uint8_t *narrow;    // [windows of the largest class] window sorted with 16-bit keys
    uint32_t *fbits;    // [2][max_class / 32 + 2] flips of the fast replay (two class buffers)
    uint32_t *fm;       // [2][max_class / 4 + 2] flips of the exact replay (byte per member)
    int32_t *bins;      // [HA] exact-replay histogram
    StageMap *maps;     // [warps][2] stage maps of the window a warp sorts (classes of many windows)
    StageMap *wmaps;    // [nwm][2] stage maps of every window (classes of at most nwm windows)
    int32_t *tin;       // [nwm + 2] entering lattice index of every window; then the walk's
                        // first failing window and its last lattice index
};

// windows per class whose stage maps are kept for the walk (more: one warp replays them in order)
constexpr int CTA_WALK_MAX = 128;
static_assert(sizeof(StageMap) == 16, "a pair copies stage maps as 16-byte words");

__host__ __device__ inline int cta_walk_windows(int32_t max_class, int W)
{
    const int32_t nw = (max_class + W - 1) / W;
    return nw < CTA_WALK_MAX ? (int)nw : CTA_WALK_MAX;
}

__host__ __device__ inline size_t align16c(size_t x) { return (x + 15) & ~(size_t)15; }

// Shared-memory layout of the sorted CTA kernel, one function for the kernel's carving and the
// host's size: the common part (reductions, G, table row, spins, repair flags), then the class
// buffers.  Every array starts on a 16-byte boundary.
struct CtaSortedLayout {
    size_t red64, red32, G, row, sig, flag, gam, rel, s0, narrow, fbits, fm, bins, maps, wmaps, tin, total;
};

__host__ __device__ inline CtaSortedLayout cta_sorted_layout(int32_t max_n, int32_t max_class, int32_t max_row,
                                                             int W, int BS)
{
    CtaSortedLayout L;
    const size_t mc = (size_t)max_class + 8;
    size_t o = 0;
    L.red64 = o; o = align16c(o + sizeof(int64_t) * (BS / 32 + 2));
    L.red32 = o; o = align16c(o + sizeof(int32_t) * (BS / 32 + 2));
    L.G = o; o = align16c(o + 16);
    L.row = o; o = align16c(o + sizeof(uint32_t) * (size_t)(max_row + 4));
    L.sig = o; o = align16c(o + (size_t)max_n + 16);
    L.flag = o; o = align16c(o + (size_t)max_n + 16);
    L.gam = o; o = align16c(o + 4 * mc);
    L.rel = o; o = align16c(o + 2 * mc);
    L.s0 = o; o = align16c(o + mc);
    L.narrow = o; o = align16c(o + (size_t)((max_class + W - 1) / W) + 4);
    L.fbits = o; o = align16c(o + 2 * 4 * (mc / 32 + 2));
    L.fm = o; o = align16c(o + 2 * 4 * (mc / 4 + 2));
    L.bins = o; o = align16c(o + 4 * (size_t)win::HA);
    L.maps = o; o = align16c(o + sizeof(StageMap) * 2 * (size_t)(BS / 32));
    const int nwm = cta_walk_windows(max_class, W);
    L.wmaps = o; o = align16c(o + sizeof(StageMap) * 2 * (size_t)nwm);
    L.tin = o; o = align16c(o + sizeof(int32_t) * (size_t)(nwm + 2));
    L.total = o;
    return L;
}

__host__ __device__ inline size_t cta_sorted_smem(int32_t max_n, int32_t max_class, int32_t max_row, int W, int BS)
{
    return cta_sorted_layout(max_n, max_class, max_row, W, BS).total;
}

// PAIR: a cluster of two blocks anneals each item.  Both keep all spins and G; a class of 3 to
// nwm windows is split in two halves of windows (thresholds, sorts and replays each block's own),
// each block copies the other's stage maps in through distributed shared memory and walks all of
// them, and each block applies the whole class's flips from both blocks' bitmaps.  Other classes
// are done by block 0 alone.  Flip bitmaps alternate between two buffers from class to class, so a block may clear
// the next class's buffer while its partner still reads the current one.
template <int BS, int SL, bool PAIR>
__global__ void __launch_bounds__(BS, 1024 / BS) gdi_cta_sorted_kernel(GdiDevProblem P, GdiDevRun R)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem S = {};
    SortedCta C;
    {
        const CtaSortedLayout L = cta_sorted_layout(P.max_n, P.max_class, R.max_row, P.W, BS);
        S.red64 = reinterpret_cast<int64_t *>(smem_raw + L.red64);
        S.red32 = reinterpret_cast<int32_t *>(smem_raw + L.red32);
        S.G = reinterpret_cast<int32_t *>(smem_raw + L.G);
        S.row = reinterpret_cast<uint32_t *>(smem_raw + L.row);
        S.sig = reinterpret_cast<int8_t *>(smem_raw + L.sig);
        S.flag = reinterpret_cast<int8_t *>(smem_raw + L.flag);
        C.gam = reinterpret_cast<int32_t *>(smem_raw + L.gam);
        C.rel = reinterpret_cast<int16_t *>(smem_raw + L.rel);
        C.s0 = smem_raw + L.s0;
        C.narrow = smem_raw + L.narrow;
        C.fbits = reinterpret_cast<uint32_t *>(smem_raw + L.fbits);
        C.fm = reinterpret_cast<uint32_t *>(smem_raw + L.fm);
        C.bins = reinterpret_cast<int32_t *>(smem_raw + L.bins);
        C.maps = reinterpret_cast<StageMap *>(smem_raw + L.maps);
        C.wmaps = reinterpret_cast<StageMap *>(smem_raw + L.wmaps);
        C.tin = reinterpret_cast<int32_t *>(smem_raw + L.tin);
        // the launch must have given the whole layout (the host sizes it with the same function)
        uint32_t dyn;
        asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
        if ((size_t)dyn < L.total) {
            if (threadIdx.x == 0 && blockIdx.x == 0) atomicCAS(R.err, 0, GDI_DEVERR_INPUT);
            return;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int W = P.W;
    const int nwm = cta_walk_windows(P.max_class, W);
    const int32_t items = P.num_instances * P.replicas;
    const size_t fbw = ((size_t)P.max_class + 8) / 32 + 2, fmw = ((size_t)P.max_class + 8) / 4 + 2;
    __shared__ int32_t next_item;
    unsigned crank = 0;                                  // block rank in the cluster
    if constexpr (PAIR) crank = cooperative_groups::this_cluster().block_rank();
    // the partner block's copy of a shared-memory object (same layout in both blocks)
    auto peer = [&](auto *ptr) { return cooperative_groups::this_cluster().map_shared_rank(ptr, crank ^ 1u); };
    auto pair_sync = [&]() {
        if constexpr (PAIR) cooperative_groups::this_cluster().sync();
        else __syncthreads();
    };
    while (true) {
        pair_sync();
        if (crank == 0 && threadIdx.x == 0) {
            const int32_t t = atomicAdd(R.item_counter, 1);
            next_item = t;
            if constexpr (PAIR) *peer(&next_item) = t;
        }
        pair_sync();
        const int32_t slot = next_item;
        if (slot >= items) break;
        const int32_t item = R.item_order[slot];
        const int32_t q = item / P.replicas;
        const int32_t rep = item - q * P.replicas;
        const int64_t base = P.node_off[q];
        const int32_t n = (int32_t)(P.node_off[q + 1] - base);
        const int32_t *cls = P.class_ptr + P.class_off[q];
        const int32_t ncls = P.class_off[q + 1] - P.class_off[q] - 1;
        int8_t *gsig = R.spins + (int64_t)rep * P.N + base;
        const int64_t nnz_item = P.row_ptr[base + n] - P.row_ptr[base];
        const int32_t mean_deg = n > 0 ? (int32_t)min((nnz_item + n - 1) / n, (int64_t)64) : 1;

        int32_t g = 0;
        for (int32_t r = threadIdx.x; r < n; r += BS) {
            const int8_t sv = gsig[r];
            S.sig[r] = sv;
            g += sv;
        }
        g = block_sum<BS, int32_t>(g, S.red32);
        if (threadIdx.x == 0) *S.G = g;
        __syncthreads();
        uint32_t cc = 0;                                 // classes annealed so far (buffer parity)

        for (int32_t sw = R.s_begin; sw < R.s_end; ++sw) {
            const int32_t roff = R.tab_off[sw];
            const int32_t rlen = R.tab_off[sw + 1] - roff;
            for (int32_t k = threadIdx.x; k < rlen; k += BS) S.row[k] = R.tab[roff + k];
            const float Tsw = R.temp ? R.temp[sw] : 0.f;
            const bool plus_first = (sw & 1) == 0;
            __syncthreads();
            for (int32_t c = 0; c < ncls; ++c) {
                const int32_t lo = cls[c], hi = cls[c + 1];
                const int32_t ns = hi - lo;
                const int32_t nwin = (ns + W - 1) / W;
                const int32_t c0 = *S.G;                 // G at class start (the reference c)
                uint32_t *fb = C.fbits + (PAIR ? (cc & 1u) * fbw : 0);
                uint32_t *fmm = C.fm + (PAIR ? (cc & 1u) * fmw : 0);
                ++cc;
                // a class of 3 to nwm windows keeps every window's stage maps for the walk below
                // (one or two windows replay in order at the cost of the walk's extra barrier);
                // a pair splits such a class: windows [0, kmid) are block 0's, the rest block 1's
                const bool walk = nwin >= 3 && nwin <= nwm;
                const bool split = PAIR && walk;
                const int32_t kmid = split ? (nwin + 1) / 2 : nwin;
                const int32_t kb = crank ? kmid : 0, ke = crank ? nwin : kmid;
                const int32_t rb = min(kb * W, ns), re = min(ke * W, ns);     // my ranks in the class
                const int32_t nown = re - rb;
                // the field sums' longest chain of dependent reads decides the layout: one thread
                // per aligned quad of ranks (one Philox call per quad; per round 4 rows), or a team
                // of T lanes per rank (T a power of two; per round a row / T); a round also costs
                // about 4 reads of draw and reduction latency, and the team layout, which draws
                // per rank, must shorten the chain by a quarter
                int T = 0;
                {
                    const int32_t nq = (nown + 3) / 4 + 1;
                    int32_t best = ((nq + BS - 1) / BS) * (4 * mean_deg + 4) * 3 / 4;
                    for (int t = 1; t <= 32; t <<= 1) {
                        const int32_t chain = ((nown * t + BS - 1) / BS) * ((mean_deg + t - 1) / t + 4);
                        if (chain < best) { best = chain; T = t; }
                    }
                }
                if (T == 0) {
                    for (int32_t qd = ((lo + rb) >> 2) + threadIdx.x; nown > 0 && qd <= ((lo + re - 1) >> 2); qd += BS) {
                        const uint4 u4 = philox4x32_10(
                            make_uint4((uint32_t)qd, (uint32_t)sw, (uint32_t)q, (uint32_t)rep), R.key0, R.key1);
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int32_t r = 4 * qd + j;
                            if (r < lo + rb || r >= lo + re) continue;
                            const int sg = S.sig[r];
                            const int32_t h = P.col16 ? local_field16(P, base, r, S.sig) : local_field(P, base, r, S.sig);
                            const int32_t es = estar_of(S.row, rlen, R.mode, word_of(u4, j), Tsw);
                            C.gam[r - lo] = gamma_of(sg, h, es, P.A, P.B);
                            C.s0[r - lo] = sg < 0 ? 1 : 0;
                        }
                    }
                } else {
                    // teams are aligned lane groups of one warp; every lane takes part in every
                    // round's shuffles (the round count is the same for the whole block)
                    const int sub = threadIdx.x & (T - 1);
                    for (int32_t k0 = rb; k0 < re; k0 += BS / T) {
                        const int32_t i = k0 + (int32_t)threadIdx.x / T;
                        int32_t h = 0;
                        if (i < re) {
                            const int64_t e0 = P.row_ptr[base + lo + i], e1 = P.row_ptr[base + lo + i + 1];
                            if (P.col16) {
                                for (int64_t e = e0 + sub; e < e1; e += T) {
                                    const uint32_t cc = __ldg(P.col16 + e);
                                    const int32_t sv = S.sig[cc & 0x7FFFu];
                                    h += (cc >> 15) ? -sv : sv;
                                }
                            } else {
                                for (int64_t e = e0 + sub; e < e1; e += T) {
                                    const uint32_t cc = __ldg(P.col + e);
                                    const int32_t sv = S.sig[cc & 0x7FFFFFFFu];
                                    h += (cc >> 31) ? -sv : sv;
                                }
                            }
                        }
                        for (int o = T >> 1; o >= 1; o >>= 1) h += __shfl_xor_sync(0xFFFFFFFFu, h, o);
                        if (i < re && sub == 0) {
                            const int32_t r = lo + i;
                            const uint4 u4 = philox4x32_10(
                                make_uint4((uint32_t)(r >> 2), (uint32_t)sw, (uint32_t)q, (uint32_t)rep), R.key0,
                                R.key1);
                            const int sg = S.sig[r];
                            const int32_t es = estar_of(S.row, rlen, R.mode, word_of(u4, r & 3), Tsw);
                            C.gam[i] = gamma_of(sg, h, es, P.A, P.B);
                            C.s0[i] = sg < 0 ? 1 : 0;
                        }
                    }
                }
                for (int32_t i = threadIdx.x; i < ns / 32 + 2; i += BS) fb[i] = 0;
                for (int32_t i = threadIdx.x; i < ns / 4 + 2; i += BS) fmm[i] = 0;
                __syncthreads();
                // every window of mine sorted by one warp
                for (int32_t kk = kb + warp; kk < ke; kk += BS / 32) {
                    const int32_t ws = kk * W, wlen = min(W, ns - ws);
                    StageMap *o = walk ? C.wmaps + 2 * kk : C.maps + 2 * warp;
                    window_maps<SL>(C.gam, C.s0, C.rel, ws, wlen, 0, c0, o);
                    __syncwarp();
                    if (lane == 0) C.narrow[kk] = (uint8_t)o[0].narrow;
                }
                // (a pair meets here for every class: the tail below may write the partner's G,
                // which the partner must have read as this class's c0 first)
                pair_sync();
                int32_t k_seq = 0;                       // first window the ordered tail replays
                if (split) {
                    // the partner's stage maps copied in at once (one remote round trip), into the
                    // slots of its windows, which this block does not use itself
                    const int32_t pkb = crank ? 0 : kmid, pke = crank ? kmid : nwin;
                    const uint4 *src = reinterpret_cast<const uint4 *>(peer(C.wmaps) + 2 * pkb);
                    uint4 *dst = reinterpret_cast<uint4 *>(C.wmaps + 2 * pkb);
                    for (int32_t i = threadIdx.x; i < 2 * (pke - pkb); i += BS) dst[i] = src[i];
                    __syncthreads();
                }
                if (walk) {
                    // one thread follows x = G - c0 from 0 through the windows' stage maps (lattice
                    // index t: x = 2 t - NT) up to the first window that leaves the lattice (in a
                    // pair both blocks walk, to the same result)
                    if (threadIdx.x == 0) {
                        int t = NT / 2;
                        int32_t kf = nwin;
                        for (int32_t kk = 0; kk < nwin; ++kk) {
                            C.tin[kk] = t;
                            const StageMap *wm = C.wmaps;
                            const int u = stage_apply(wm[2 * kk + (plus_first ? 1 : 0)],
                                                      stage_apply(wm[2 * kk + (plus_first ? 0 : 1)], t));
                            if (u < 0) { kf = kk; break; }
                            t = u;
                        }
                        C.tin[nwm] = kf;
                        C.tin[nwm + 1] = t;
                        if (kf == nwin) *S.G = c0 + 2 * t - NT;
                    }
                    __syncthreads();
                    k_seq = C.tin[nwm];
                    // my windows before it were entered on the lattice: all replayed at once
                    for (int32_t kk = kb + warp; kk < min(ke, k_seq); kk += BS / 32) {
                        const int32_t ws = kk * W, we = min(ws + W, ns);
                        replay_window<SL>(C.rel, C.s0, 0, ws, we, 2 * C.tin[kk] - NT, plus_first, fb, W);
                    }
                }
                // the rest in rank order by one warp of block 0, each window entered with the G its
                // predecessors left; a window of block 1 is read, and its flips written, remotely
                if (crank == 0 && warp == 0 && k_seq < nwin) {
                    int32_t x = walk ? 2 * C.tin[k_seq] - NT : 0;
                    for (int32_t kk = k_seq; kk < nwin; ++kk) {
                        const bool mine = kk < kmid;
                        const int16_t *rel = C.rel;
                        const uint8_t *s0 = C.s0, *nar = C.narrow;
                        const int32_t *gam = C.gam;
                        uint32_t *fbo = fb, *fmo = fmm;
                        if constexpr (PAIR) {
                            if (!mine) {
                                rel = peer(C.rel); s0 = peer(C.s0); nar = peer(C.narrow);
                                gam = peer(C.gam); fbo = peer(fb); fmo = peer(fmm);
                            }
                        }
                        const int32_t ws = kk * W, we = min(ws + W, ns);
                        const bool on = nar[kk] ? (x >= -NT && x <= NT - 2) : (x >= -FAST_X && x <= FAST_X);
                        x = on ? replay_window<SL>(rel, s0, 0, ws, we, x, plus_first, fbo, W)
                               : window_replay_exact(gam, s0, 0, ws, we, c0 + x, plus_first, C.bins, fmo) - c0;
                    }
                    if (lane == 0) {
                        *S.G = c0 + x;
                        if constexpr (PAIR) *peer(S.G) = c0 + x;
                    }
                }
                if constexpr (PAIR) pair_sync(); else __syncthreads();
                // every block applies the whole class's flips to its copy of the spins
                for (int part = 0; part < (PAIR ? 2 : 1); ++part) {
                    const int32_t i0 = part == 0 ? 0 : min(kmid * W, ns), i1 = part == 0 ? min(kmid * W, ns) : ns;
                    const uint32_t *fbr = fb, *fmr = fmm;
                    if constexpr (PAIR) {
                        if ((unsigned)part != crank) { fbr = peer(fb); fmr = peer(fmm); }
                    }
                    for (int32_t i = i0 + threadIdx.x; i < i1; i += BS) {
                        const uint32_t f = ((fbr[i >> 5] >> (i & 31)) | (fmr[i >> 2] >> (8 * (i & 3)))) & 1u;
                        if (f) S.sig[lo + i] = (int8_t)-S.sig[lo + i];
                    }
                }
                __syncthreads();
            }
            if (R.flags & GDI_DEV_TRACE) {
                uint64_t dg = 0;
                for (int32_t r = threadIdx.x; r < n; r += BS)
                    if (S.sig[r] > 0)
                        dg += splitmix64_fin((uint64_t)(uint32_t)r | ((uint64_t)(sw & 0xFFFF) << 32) |
                                             ((uint64_t)(rep & 0xFFFF) << 48));
                dg = block_sum<BS, uint64_t>(dg, reinterpret_cast<uint64_t *>(S.red64));
                const int64_t ct = item_cut<BS>(P, base, n, S);
                if (threadIdx.x == 0 && crank == 0) {
                    const int64_t o = (int64_t)item * R.sweeps + sw;
                    R.tr_digest[o] = dg;
                    R.tr_G[o] = *S.G;
                    R.tr_cut[o] = ct;
                }
            }
            __syncthreads();
        }
        const int64_t raw_cut = item_cut<BS>(P, base, n, S);
        __syncthreads();
        const int32_t raw_G = *S.G;
        if (!(R.flags & GDI_DEV_NO_REPAIR)) repair<BS>(P, base, n, S);
        const int64_t fin_cut = item_cut<BS>(P, base, n, S);
        __syncthreads();
        if (crank == 0) {
            if (threadIdx.x == 0) {
                R.raw_G[item] = raw_G;
                R.raw_cut[item] = raw_cut;
                R.final_G[item] = *S.G;
                R.final_cut[item] = fin_cut;
            }
            for (int32_t r = threadIdx.x; r < n; r += BS) gsig[r] = S.sig[r];
        }
        __syncthreads();
    }
}

// Initial state (Alg. 3 "initialize all s_i"): balanced random pairs from Philox, or the caller's
// spins scattered from original order to rank order.
__global__ void gdi_init_kernel(GdiDevProblem P, int8_t *spins, const int8_t *init_orig, int kind,
                                uint32_t key0, uint32_t key1)
{
    const int64_t total = (int64_t)P.replicas * P.N;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t rep = (int32_t)(t / P.N);
        const int64_t v = t - (int64_t)rep * P.N;
        if (kind == 1) {            // caller spins, original vertex v
            spins[(int64_t)rep * P.N + P.rank_of[v]] = init_orig[t] > 0 ? 1 : -1;
            continue;
        }
        // random: v is a global rank; find its instance by binary search of node_off
        int32_t lo = 0, hi = P.num_instances - 1;
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (P.node_off[mid] <= v) lo = mid; else hi = mid - 1;
        }
        const int64_t base = P.node_off[lo];
        const int32_t n = (int32_t)(P.node_off[lo + 1] - base);
        const int32_t r = (int32_t)(v - base);
        int8_t s;
        if ((n & 1) && r == n - 1) {
            s = -1;
        } else {
            const int32_t pr = r >> 1;
            const uint4 u4 = philox4x32_10(make_uint4((uint32_t)(pr >> 2), 0xFFFFFFFFu, (uint32_t)lo,
                                                      (uint32_t)rep), key0, key1);
            const int8_t a = (word_of(u4, pr & 3) >> 31) ? -1 : 1;
            s = (r & 1) ? (int8_t)-a : a;
        }
        spins[t] = s;
    }
}

__global__ void gdi_gather_kernel(GdiDevProblem P, const int8_t *spins, int8_t *out)
{
    const int64_t total = (int64_t)P.replicas * P.N;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t rep = (int32_t)(t / P.N);
        const int64_t v = t - (int64_t)rep * P.N;
        out[t] = spins[(int64_t)rep * P.N + P.rank_of[v]];
    }
}

size_t cta_smem(const GdiDevProblem &P, const GdiDevRun &R, int BS, int H)
{
    size_t b = sizeof(int64_t) * (BS / 32 + 2) + sizeof(int32_t) * (BS / 32 + 2) + 16;
    b += sizeof(int32_t) * (size_t)H;
    b += sizeof(int32_t) * (size_t)((P.max_window + 3) & ~3);
    b += sizeof(uint32_t) * (size_t)((R.max_row + 3) & ~3);
    b += (size_t)((P.max_window + 15) & ~15);
    b += (size_t)((P.max_n + 15) & ~15);
    b += (size_t)P.max_n;
    return b;
}

int hist_bins(const GdiDevProblem &P)
{
    int H = 64;
    while (H < 2 * P.max_window + 2 && H < 256) H <<= 1;
    return H;
}

// the sorted-window kernel serves every window size 1 .. 256 (one instantiation per members per
// lane) of the running-G method when its whole-class buffers fit in a block's shared memory;
// Algorithm 2 (GDI_DEV_STANDARD), larger windows and larger classes take gdi_cta_anneal_kernel
inline bool cta_sorted(const GdiDevProblem &P, const GdiDevRun &R, int BS)
{
    if (P.W < 1 || P.W > 256 || (R.flags & GDI_DEV_STANDARD)) return false;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return cta_sorted_smem(P.max_n, P.max_class, R.max_row, P.W, BS) <= (size_t)optin;
}

// a pair of blocks per item when the items fill at most half of the SMs and the largest class
// has enough windows (8 to the walk's limit) for two halves
inline bool cta_pair(const GdiDevProblem &P, const GdiDevRun &R, int BS)
{
    if (!cta_sorted(P, R, BS)) return false;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t items = (int64_t)P.num_instances * P.replicas;
    const int32_t nw = (P.max_class + P.W - 1) / P.W;
    return 2 * items <= sms && nw >= 8 && nw <= CTA_WALK_MAX;
}

template <int BS, bool PAIR>
const void *cta_sorted_kernel_for(int W)
{
    return W <= 32 ? (const void *)gdi_cta_sorted_kernel<BS, 1, PAIR>
         : W <= 64 ? (const void *)gdi_cta_sorted_kernel<BS, 2, PAIR>
         : W <= 128 ? (const void *)gdi_cta_sorted_kernel<BS, 4, PAIR>
                    : (const void *)gdi_cta_sorted_kernel<BS, 8, PAIR>;
}

template <int BS>
const void *cta_kernel(const GdiDevProblem &P, const GdiDevRun &R)
{
    if (!cta_sorted(P, R, BS)) return (const void *)gdi_cta_anneal_kernel<BS>;
    return cta_pair(P, R, BS) ? cta_sorted_kernel_for<BS, true>(P.W) : cta_sorted_kernel_for<BS, false>(P.W);
}

template <int BS>
size_t cta_kernel_smem(const GdiDevProblem &P, const GdiDevRun &R)
{
    return cta_sorted(P, R, BS) ? cta_sorted_smem(P.max_n, P.max_class, R.max_row, P.W, BS)
                         : cta_smem(P, R, BS, hist_bins(P));
}

template <int BS>
int launch_cta(const GdiDevProblem &P, const GdiDevRun &R, int grid_limit, cudaStream_t st,
               int *grid_used, size_t *smem_used)
{
    const void *kern = cta_kernel<BS>(P, R);
    const size_t smem = cta_kernel_smem<BS>(P, R);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BS, smem);
    if (e != cudaSuccess) return (int)e;
    if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
    const int items = P.num_instances * P.replicas;
    int grid = sms * per_sm;
    if (grid > items) grid = items;
    if (grid_limit > 0 && grid > grid_limit) grid = grid_limit;
    if (cta_pair(P, R, BS)) {
        // clusters of two blocks, one item per cluster
        void *args[] = {const_cast<GdiDevProblem *>(&P), const_cast<GdiDevRun *>(&R)};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * items);
        cfg.blockDim = dim3(BS);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int ncl = 0;
        e = cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg);
        if (e != cudaSuccess) return (int)e;
        if (ncl < 1) return (int)cudaErrorInvalidConfiguration;
        grid = 2 * (items < ncl ? items : ncl);
        if (grid_limit > 0 && grid > grid_limit) grid = grid_limit >= 2 ? (grid_limit & ~1) : 2;
        cfg.gridDim = dim3(grid);
        e = cudaLaunchKernelExC(&cfg, kern, args);
        if (e != cudaSuccess) return (int)e;
    } else if (cta_sorted(P, R, BS)) {
        void *args[] = {const_cast<GdiDevProblem *>(&P), const_cast<GdiDevRun *>(&R)};
        e = cudaLaunchKernel(kern, dim3(grid), dim3(BS), args, smem, st);
        if (e != cudaSuccess) return (int)e;
    } else {
        gdi_cta_anneal_kernel<BS><<<grid, BS, smem, st>>>(P, R, hist_bins(P));
    }
    if (grid_used) *grid_used = grid;
    if (smem_used) *smem_used = smem;
    return (int)cudaGetLastError();
}

template <int BS>
int cta_occupancy(const GdiDevProblem &P, const GdiDevRun &R, int *per_sm)
{
    const void *kern = cta_kernel<BS>(P, R);
    const size_t smem = cta_kernel_smem<BS>(P, R);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, BS, smem);
    return (int)e;
}

}  // namespace

int gdi_cta_blocks_per_sm(const GdiDevProblem &P, const GdiDevRun &R, int block, int *per_sm)
{
    *per_sm = 0;
    switch (block) {
    case 128: return cta_occupancy<128>(P, R, per_sm);
    case 256: return cta_occupancy<256>(P, R, per_sm);
    case 512: return cta_occupancy<512>(P, R, per_sm);
    case 1024: return cta_occupancy<1024>(P, R, per_sm);
    default: return (int)cudaErrorInvalidValue;
    }
}

int gdi_cta_smem_bytes(const GdiDevProblem &P, const GdiDevRun &R, int block, size_t *bytes, int *hist)
{
    const int H = hist_bins(P);
    if (hist) *hist = H;
    if (bytes) *bytes = cta_sorted(P, R, block) ? cta_sorted_smem(P.max_n, P.max_class, R.max_row, P.W, block)
                                      : cta_smem(P, R, block, H);
    return 0;
}

int gdi_launch_cta_anneal(const GdiDevProblem &P, const GdiDevRun &R, int block, int grid_limit,
                          void *stream, int *grid_used, size_t *smem_used)
{
    cudaStream_t st = (cudaStream_t)stream;
    switch (block) {
    case 128: return launch_cta<128>(P, R, grid_limit, st, grid_used, smem_used);
    case 256: return launch_cta<256>(P, R, grid_limit, st, grid_used, smem_used);
    case 512: return launch_cta<512>(P, R, grid_limit, st, grid_used, smem_used);
    case 1024: return launch_cta<1024>(P, R, grid_limit, st, grid_used, smem_used);
    default: return (int)cudaErrorInvalidValue;
    }
}

int gdi_launch_init(const GdiDevProblem &P, int8_t *spins, const int8_t *init_orig, int init_kind,
                    uint32_t key0, uint32_t key1, void *stream)
{
    const int64_t total = (int64_t)P.replicas * P.N;
    int grid = (int)((total + 255) / 256);
    if (grid > 152 * 32) grid = 152 * 32;
    if (grid < 1) grid = 1;
    gdi_init_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(P, spins, init_orig, init_kind, key0, key1);
    return (int)cudaGetLastError();
}

int gdi_launch_gather_spins(const GdiDevProblem &P, const int8_t *spins_rank, int8_t *out_orig,
                            void *stream)
{
    const int64_t total = (int64_t)P.replicas * P.N;
    int grid = (int)((total + 255) / 256);
    if (grid > 152 * 32) grid = 152 * 32;
    if (grid < 1) grid = 1;
    gdi_gather_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(P, spins_rank, out_orig);
    return (int)cudaGetLastError();
}
