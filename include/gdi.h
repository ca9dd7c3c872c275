/*
 * gdi.h -- C ABI of libgdi.so, a GB300 (sm_103a) implementation of the Globally Decoupled Ising
 * (GDI) annealer for balanced min-cut graph bisection (Cook, Jin, Tan, arXiv:1908.00210).
 *
 * Problem (Section 4.1): split the vertices of G(V, E) into V1 (spin +1) and V2 (spin -1) with
 * |V1| = |V2| and the smallest total weight of crossing edges.  The annealer minimises
 *     H = A (sum_i s_i)^2 + B sum_<ij> w_ij (1 - s_i s_j) / 2              (Eq. 4, 5, 6)
 * with Algorithm 3: the balance term reads one global magnetisation G = sum_i s_i that is updated
 * by every flip, instead of the complete graph that Eq. 5 implies.
 *
 * Conventions shared by every entry point:
 *   - Return value: 0 on success, a negative GDI_ERR_* code on failure.  No call aborts the
 *     process; gdi_last_error() gives a one-line message for the calling thread's last failure.
 *   - Ownership: gdi_create copies every input into buffers owned by the context; the caller may
 *     free its own buffers when the call returns.  Outputs are written into caller buffers.
 *   - Memory kind: arguments named *_mem say whether a pointer is host (GDI_MEM_HOST) or device
 *     (GDI_MEM_DEVICE, a CUDA device pointer on the context's device).
 *   - Streams: gdi_anneal enqueues all device work on the given CUDA stream and returns without
 *     waiting; the getters synchronise that stream before reading.
 *   - Vertex numbering: graphs are given in original vertex ids; spins come back in that order.
 *   - Threads: a context may be used by one host thread at a time.
 */
#ifndef GDI_H
#define GDI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define GDI_OK 0
#define GDI_ERR_INVALID_ARG   -1   /* null pointer, bad size, bad schedule, weight not +-1      */
#define GDI_ERR_NOT_SYMMETRIC -2   /* (i,j,w) present without (j,i,w)                           */
#define GDI_ERR_SELF_LOOP     -3
#define GDI_ERR_DUP_EDGE      -4
#define GDI_ERR_BAD_COLORING  -5   /* negative colour or two adjacent vertices share a colour    */
#define GDI_ERR_OVERFLOW      -6   /* a size or an energy term would not fit the integer ranges  */
#define GDI_ERR_OOM           -7
#define GDI_ERR_CUDA          -8   /* a CUDA runtime call failed (message in gdi_last_error)     */
#define GDI_ERR_TIMEOUT       -9   /* a bounded device wait gave up; the context stays usable    */
#define GDI_ERR_NOT_ANNEALED  -10  /* a getter was called before any gdi_anneal                  */
#define GDI_ERR_TOO_LARGE     -11  /* no kernel variant supports this size                        */

/* memory kinds */
#define GDI_MEM_HOST   0
#define GDI_MEM_DEVICE 1

/* schedule modes */
#define GDI_METROPOLIS 0   /* accept with min(1, exp(-dE/T_s)), T_s geometric from t0 to t1          */
#define GDI_PAPER_PF   1   /* Alg. 2/3: argmin, then flip with probability P_f; P_f geometric pf0->pf1 */

/* kernel paths (gdi_configure) */
#define GDI_PATH_AUTO 0   /* several instances: CTA-resident.  One instance (W >= 1): the path a
                             cost model fitted on GB300 predicts faster (per colour class and per
                             vertex + edge): the grid-scale path for a few replicas of a graph
                             above a few thousand vertices, or whenever the CTA path's shared
                             memory does not fit; CTA-resident otherwise                         */
#define GDI_PATH_CTA  1   /* one thread block anneals one (instance, replica), spins in shared
                             memory; with 1 <= W <= 256, when the items fill at most half of the
                             SMs and the largest class has 8 to 128 windows, a cluster of two
                             blocks anneals each item (gdi_last_launch counts both blocks)       */
#define GDI_PATH_GRID 2   /* one instance over every SM (needs W >= 1); up to 8 replicas per pass;
                             W <= 256: sorted-window kernel, W > 256: tabulated-window kernel */

/* gdi_run.flags */
#define GDI_FLAG_TRACE     1  /* record per-sweep G, cut and state digest (slower; for parity)     */
#define GDI_FLAG_NO_REPAIR 2  /* skip the exact-balance repair after the last sweep                */
#define GDI_FLAG_CONTINUE  4  /* start from the spins the previous gdi_anneal left (resume)        */
#define GDI_FLAG_RACY      8  /* Algorithm 3 as printed: inside a colour class every spin decides on
                                 the G it reads at that moment and adds its change with an atomic;
                                 not deterministic, W ignored; grid-scale path (one instance) only */
#define GDI_FLAG_STANDARD 16  /* Algorithm 2, the paper's "standard" annealer (Section 5.2): every
                                 spin forms the balance term of Eq. 5 by reading all n spins (the
                                 complete graph) instead of the decoupled G, and the spins of a
                                 window decide on the state at the window start (W = 1: one spin at
                                 a time).  Deterministic; CTA-resident path only */

typedef struct gdi_ctx gdi_ctx;  /* opaque; owned by the library */

/* A graph, or a batch of independent graphs given as one disjoint union.  Host pointers. */
typedef struct {
    int32_t num_instances;     /* >= 1                                                          */
    const int64_t *inst_ptr;   /* [num_instances + 1] vertex offsets of the instances; may be
                                  NULL when num_instances == 1                                  */
    int64_t num_vertices;      /* N, total over instances                                       */
    const int64_t *row_ptr;    /* [N + 1] CSR offsets                                           */
    const int32_t *col;        /* [row_ptr[N]] neighbour ids (0..N-1, inside the same instance) */
    const int32_t *weight;     /* [row_ptr[N]] edge weights, each +1 or -1; NULL = all +1       */
    const int32_t *color;      /* [N] proper colouring (values >= 0, per instance); NULL = greedy
                                  first-fit colouring in vertex-id order                        */
} gdi_graph;

/* Model constants of Eq. 4-6 and the decoupling window. */
typedef struct {
    int32_t A;          /* balance-penalty weight, >= 0 (Eq. 5)                                   */
    int32_t B;          /* cut weight, >= 1 (Eq. 6)                                              */
    int32_t W;          /* window: a colour class is updated in chunks of W consecutive ranks, each
                           chunk seeing the exact running G in threshold order; 0 = whole class  */
    int32_t replicas;   /* independent replicas per instance, >= 1                              */
} gdi_model;

/* Annealing schedule (Section 5.2; "reduce P_f" of Alg. 2/3 is the per-sweep table row). */
typedef struct {
    int32_t mode;       /* GDI_METROPOLIS or GDI_PAPER_PF                                         */
    double t0, t1;      /* Metropolis temperatures at the first and last sweep, > 0              */
    double pf0, pf1;    /* paper mode flip probabilities at the first and last sweep, in [0, 0.5) */
    int32_t sweeps;     /* M >= 1                                                                 */
} gdi_schedule;

/* One annealing call. */
typedef struct {
    uint64_t seed;          /* Philox key; replica r of instance q draws counters (rank/4, sweep, q, r) */
    int32_t first_sweep;    /* anneal sweeps [first_sweep, last_sweep) of the schedule            */
    int32_t last_sweep;     /* <= 0 means schedule.sweeps                                         */
    int32_t flags;          /* GDI_FLAG_*                                                         */
    const int8_t *init_spins; /* [replicas][N] spins (+1/-1) in original order, or NULL: balanced
                                 random start (ignored with GDI_FLAG_CONTINUE)                    */
    int32_t init_mem;       /* GDI_MEM_HOST or GDI_MEM_DEVICE for init_spins                       */
    void *stream;           /* cudaStream_t for all device work; NULL = the legacy default stream */
} gdi_run;

/* Build a context: validate the CSR (symmetric, no self-loops, no duplicates, weights +-1),
 * colour it (or check the given colouring), relabel every instance into rank order, and copy it to
 * the current CUDA device.  Rank order: the vertices of an instance sorted by colour ascending,
 * then inside each colour class by splitmix64(local vertex id) ascending (splitmix64 = the
 * finaliser of Steele, Lea and Flood, OOPSLA'14: z += 0x9E3779B97F4A7C15; z = (z ^ z>>30) *
 * 0xBF58476D1CE4E5B9; z = (z ^ z>>27) * 0x94D049BB133111EB; z ^= z>>31), a fixed pseudo-random
 * order inside the class; gdi_rank_space returns it.  This is the update order of the deterministic
 * reading of Algorithm 3 (Section 5.3): classes in order, each class in windows of W consecutive
 * ranks.  Device memory: the rank-space CSR (8 B per vertex + 4 B per directed edge), plus a
 * 16-bit copy of the columns (2 B per directed edge) when every instance has at most 32,767
 * vertices, and the spins (1 B per vertex per replica).  Host-side preprocessing; blocking. */
int gdi_create(gdi_ctx **out, const gdi_graph *graph, const gdi_model *model);

/* Anneal every replica of every instance with Algorithm 3, serialised deterministically: colour
 * classes in order, windows of W ranks, and inside a window the exact running G seen in threshold
 * order (+1 group first on even sweeps); then repair to exact balance |G| = n mod 2 and compute
 * the cut.
 * Enqueued on run->stream; returns without waiting.  Host pointers in `run` are read before the
 * call returns. */
int gdi_anneal(gdi_ctx *ctx, const gdi_schedule *schedule, const gdi_run *run);

/* Spins after the last gdi_anneal, [replicas][N] in original vertex order (+1 = V1, -1 = V2,
 * Section 4.1).  Synchronises the run stream. */
int gdi_get_spins(gdi_ctx *ctx, int8_t *out, int32_t out_mem);

/* Per (instance, replica), index q * replicas + r: raw G after the last sweep, G after repair,
 * cut before and after repair (cut = sum of crossing edge weights, Section 6.2).  Any pointer may be
 * NULL.  Host pointers.  Synchronises the run stream. */
int gdi_get_results(gdi_ctx *ctx, int32_t *raw_G, int32_t *final_G, int64_t *raw_cut,
                    int64_t *final_cut);

/* Cut after repair of one (instance, replica): the sum of w_ij over the edges whose ends lie on
 * different sides, i.e. the cut term of Eq. 6 without its factor B (Section 4.1), which for unit
 * weights is the number of crossing edges that Table 1 reports (Section 6.2).  Host pointer;
 * GDI_ERR_INVALID_ARG for an index out of range, GDI_ERR_NOT_ANNEALED before any anneal.
 * Synchronises the run stream. */
int gdi_cut(gdi_ctx *ctx, int32_t instance, int32_t replica, int64_t *cut_out);

/* Magnetisation G = sum_i s_i = |V1| - |V2| of one (instance, replica) before (raw) and after the
 * repair: the quantity Eq. 5 penalises and the balance column of Table 1 (Section 6.2).  After the
 * repair |G| = n mod 2.  Host pointers, either may be NULL; errors as gdi_cut.  Synchronises. */
int gdi_balance(gdi_ctx *ctx, int32_t instance, int32_t replica, int32_t *raw_G, int32_t *final_G);

/* Per-sweep trace of the last gdi_anneal with GDI_FLAG_TRACE: [q * replicas + r][sweeps] arrays of
 * the state digest, G and cut after each sweep (entries outside the annealed range are 0).
 * digest = sum over ranks i with s_i = +1 of splitmix64(i | sweep << 32 | replica << 48) mod 2^64.
 * Any pointer may be NULL.  Host pointers. */
int gdi_get_trace(gdi_ctx *ctx, uint64_t *digest, int32_t *G, int64_t *cut);

/* Launch configuration of later gdi_anneal calls: kernel path (GDI_PATH_*), threads per block of
 * the CTA-resident path (0 = keep, else 128/256/512/1024) and a cap on the number of blocks
 * (0 = one wave on every SM).  Results do not depend on any of these (the autotuner relies on it). */
int gdi_configure(gdi_ctx *ctx, int32_t path, int32_t block, int32_t grid_limit);

/* Autotuner: anneals the first probe_sweeps sweeps of `schedule` (random start, no repair) under
 * each candidate launch configuration -- threads per block 128/256/512/1024 x one or several
 * blocks per SM on the CTA path, 100/75/50 % of the SMs on the grid path -- times each with CUDA
 * events on a private stream, and keeps the fastest for later calls (as gdi_configure would).
 * Results never depend on the configuration, so tuning is free of side effects on correctness;
 * it does overwrite the context's spins and results.  Blocking.  Outputs may be NULL. */
int gdi_autotune(gdi_ctx *ctx, const gdi_schedule *schedule, int32_t probe_sweeps,
                 int32_t *block_out, int32_t *grid_out, float *ms_out);

/* What the last gdi_anneal launched: path, blocks, dynamic shared memory per block, and how many
 * times the grid-scale path took its exact fallback -- a block whose G-map could not carry the
 * running magnetisation and replayed its windows exactly instead (0 on the CTA path; a count of
 * events, summed over replicas).  Synchronises. */
int gdi_last_launch(gdi_ctx *ctx, int32_t *path, int32_t *grid, int64_t *smem_bytes,
                    int32_t *fallbacks);

/* Failure-detection test hook (the paper has no counterpart).  The next gdi_anneal that takes the
 * grid-scale path starts with its grid barrier's gate word closed, set from the host, so no
 * barrier can complete -- a flag that no block will ever clear.  Every block's
 * bounded wait then gives up after spin_limit polls (>= 1; each poll sleeps tens of ns), sets the
 * device error word and returns; the anneal reports GDI_ERR_TIMEOUT (from gdi_get_results and
 * the other synchronising calls).  Nothing faults, traps or hangs, the context stays usable, and
 * the following anneal runs normally.  The CTA-resident path has no cross-block waits and ignores
 * the hook, which stays armed until a grid-scale anneal consumes it. */
int gdi_inject_wait_failure(gdi_ctx *ctx, int64_t spin_limit);

/* Device time of the anneal kernel launches of the last gdi_anneal (the sweep kernels alone,
 * without the initialisation, packing, cut and repair kernels around them), measured with CUDA
 * events recorded on the anneal's stream around every launch: *ms = their sum, *launches = how
 * many (one per group of 8 replicas on the grid-scale path, one on the CTA path; may be NULL).
 * GDI_ERR_NOT_ANNEALED if there was no anneal, or if it was captured into a CUDA graph (no
 * events are recorded while a stream is being captured).  Synchronises. */
int gdi_kernel_time(gdi_ctx *ctx, float *ms, int32_t *launches);

/* Context facts: number of colour classes per instance (host [num_instances], may be NULL),
 * the largest degree, and the E_cap of the last schedule (0 before any anneal). */
int gdi_info(gdi_ctx *ctx, int32_t *num_classes, int32_t *max_degree, int32_t *ecap);

/* Rank-space layout of one graph (num_instances = 1), computed on the host exactly as gdi_create
 * computes it, in the form gdi_anneal_static takes: validation and colouring as gdi_create (greedy
 * first-fit when graph->color is NULL), then
 *   vert_of   [n]      the original vertex at rank r (rank order as described at gdi_create);
 *   row_ptr   [n + 1]  CSR offsets of the relabelled graph;
 *   col       [nnz]    neighbour rank | 0x80000000 when the edge weight is -1;
 *   class_ptr [num_classes + 1] rank boundaries of the colour classes (room for n + 1 entries);
 *   max_class, max_degree (may be NULL).
 * All host arrays owned by the caller.  Errors as gdi_create.  No device work. */
int gdi_rank_space(const gdi_graph *graph, int32_t *vert_of, int64_t *row_ptr, uint32_t *col,
                   int32_t *class_ptr, int32_t *num_classes, int32_t *max_class,
                   int32_t *max_degree);

/* Threshold table of a schedule, built on the host as gdi_anneal builds it ("reduce P_f" of
 * Algorithms 2 and 3 becomes one table row per sweep, Section 5.2), in the form gdi_anneal_static
 * takes.  Metropolis row s holds floor(exp(-dE / T_s) 2^32) for dE = 1, 2, ... while non-zero,
 * T_s = t0 (t1/t0)^(s/(M-1)), temp[s] = T_s; paper row s holds 2^32 - p_s, 2^31, p_s with
 * p_s = floor(P_f,s 2^32) + 1 (a flip iff u <= P_f) and temp[s] = 0.  With tab == NULL only *tab_len
 * and *max_row are returned (a size query); otherwise tab [tab_cap >= *tab_len], tab_off
 * [sweeps + 1] and temp [sweeps] are filled.  Host arrays owned by the caller. */
int gdi_build_table(const gdi_schedule *schedule, uint32_t *tab, int64_t tab_cap, int64_t *tab_len,
                    int32_t *tab_off, float *temp, int32_t *max_row);

/* ---- Allocation-free sweep (the paper has no counterpart) -----------------------------------
 * For callers that cannot allocate device memory while they run: code whose device memory belongs
 * to another allocator (a framework's caching pool or a fixed arena) or that must not grow its
 * device footprint after start-up.  gdi_anneal allocates its table, staging and scratch buffers on
 * first use; gdi_anneal_static calls no cudaMalloc, cudaFree or allocating library routine.  It
 * runs the grid-scale sweep kernel of GDI_PATH_GRID on one graph whose arrays the caller already
 * holds on the device, in the rank-space layout below, with its scratch in one fixed-size static
 * device array of about 1.4 MB that every GPU which loads libgdi.so keeps until the process exits.
 *
 * Inputs (device pointers, current device, read only):
 *   row_ptr   [n + 1] int64 CSR offsets of the graph relabelled in rank order (the order described
 *             at gdi_create: colour, then splitmix64 of the vertex id -- gdi_rank_space computes
 *             it; any other order anneals in a different order and gives different results from
 *             gdi_anneal); col [row_ptr[n]] neighbour rank | 0x80000000 when the weight is -1.
 *   class_ptr [num_classes + 1] rank boundaries of the colour classes (0 ... n); max_class is the
 *             largest class, max_degree the largest row length.
 *   tab, tab_off [sweeps + 1], temp [sweeps]: the threshold table as gdi_build_table returns it,
 *             max_row its longest row.
 *   A, B, W, mode, sweeps, [first_sweep, last_sweep) (last_sweep <= 0 = sweeps), seed: as in
 *   gdi_model / gdi_schedule / gdi_run; replicas 1..8 draw Philox counters (rank/4, sweep, 0, r).
 * In/out: spins [replicas][n] int8 (+1/-1) in rank order, annealed in place (no repair).
 * Out: G_out [replicas] int32, the magnetisation after the last sweep.
 * Limits: n <= GDI_STATIC_MAX_VERTICES, replicas <= 8, W >= 1 and small enough for the per-block
 * plan, at most GDI_STATIC_MAX_BLOCKS blocks; beyond them the call returns GDI_ERR_TOO_LARGE and
 * launches nothing.  Enqueued on `stream`; returns without waiting.
 * The first call on a device looks up the device address of the static array
 * (cudaGetSymbolAddress), so make that first call before any stream capture.  Every call shares
 * the one array, which keeps the previous call's contents (the call clears what must start at
 * zero): calls whose work overlaps on the GPU race with each other, so serialise them (one stream,
 * or events).  If a grid barrier wait ever ran out, the kernel stops early and the spins are those
 * of the interrupted sweep.
 * Input checks: the sizes and arrays above come from the caller, so before the anneal the call
 * enqueues checks that row_ptr starts at 0 with rows of at most max_degree entries, that every
 * neighbour rank is below n and outside its row's colour class, that class_ptr runs monotonically
 * from 0 to n with no class above max_class, and that every table row of the sweep range fits
 * max_row.  A failed check launches no sweep work: spins stay as they were and G_out is undefined.
 * Symmetry of the CSR is not checked.  gdi_anneal_static_status reports the outcome. */
#define GDI_STATIC_MAX_VERTICES (1 << 20)
#define GDI_STATIC_MAX_BLOCKS 160
int gdi_anneal_static(int32_t n, const int64_t *row_ptr, const uint32_t *col, int32_t num_classes,
                      const int32_t *class_ptr, int32_t max_class, int32_t max_degree, int32_t A,
                      int32_t B, int32_t W, int32_t mode, const uint32_t *tab,
                      const int32_t *tab_off, const float *temp, int32_t max_row, int32_t sweeps,
                      int32_t first_sweep, int32_t last_sweep, uint64_t seed, int32_t replicas,
                      int8_t *spins, int32_t *G_out, void *stream);

/* Outcome of the last gdi_anneal_static on the current device, enqueued on `stream` after it: a
 * one-thread kernel writes GDI_OK, GDI_ERR_INVALID_ARG (an input check failed) or GDI_ERR_TIMEOUT
 * (a bounded device wait ran out) into *status, which must be device-accessible memory (device
 * memory, or mapped pinned host memory).  Allocates nothing; the paper has no counterpart. */
int gdi_anneal_static_status(int32_t *status, void *stream);

/* Free the context and its device buffers (synchronises the run stream first).  Library
 * housekeeping: the paper has no counterpart.  NULL is allowed and does nothing. */
void gdi_destroy(gdi_ctx *ctx);

/* Static description of an error code. */
const char *gdi_strerror(int code);

/* Message of the calling thread's last failed call ("" if none). */
const char *gdi_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GDI_H */
