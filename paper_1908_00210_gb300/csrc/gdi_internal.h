// gdi_internal.h -- device-side data layout shared by the host API (gdi_api.cpp) and the kernels
// (gdi_kernels.cu) of libgdi.so.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

// Rank space: every instance q is relabelled so that its vertices are sorted by (colour, id);
// colour classes are then contiguous rank ranges [class_ptr[k], class_ptr[k+1]).  Rank-space ids
// are global over the batch (instance q owns [node_off[q], node_off[q+1])).
struct GdiDevProblem {
    int32_t num_instances;
    int32_t replicas;
    int64_t N;                       // total vertices
    const int64_t *node_off;         // [Q+1]
    const int32_t *class_off;        // [Q+1] offsets into class_ptr
    const int32_t *class_ptr;        // per instance: C_q + 1 class boundaries in local ranks
    const int64_t *row_ptr;          // [N+1] rank-space CSR offsets
    const uint32_t *col;             // [nnz] local neighbour rank | (weight < 0) << 31
    const uint16_t *col16;           // [nnz] the same in 16 bits (rank | (weight < 0) << 15) when
                                     // every instance has at most 32,767 vertices, else null
    const int32_t *rank_of;          // [N] original vertex -> global rank
    int32_t A, B, W;
    int32_t max_n;                   // largest instance
    int32_t max_window;              // largest window (W or class size) over instances
    int32_t max_degree;
    int32_t max_class;               // largest colour class
};

// Global scratch of the grid-scale path (single large instance).
struct GdiGridScratch {
    uint8_t *packed;                 // [N] spins of one replica group: bit r set = replica r is -1
    int16_t *tables;                 // [P][8][TW] composed window tables of every block (W > 256);
                                     // for W <= 256 the same bytes hold the sorted path's exact-G
                                     // words and [P][8][64] byte block and run tables
    int32_t *gin;                    // [P][8] exact G entering every block's windows
    int32_t *Gcls;                   // [8] G at class start / after the class
    unsigned int *bar;               // [4] grid barrier: 64-bit arrival count, gate, unused
    int32_t *err;                    // [1] device error word
    int32_t *status;                 // [16] diagnostics: exact fallbacks per replica
    int32_t *rhist;                  // [8][2*max_degree+1] repair key histogram
    uint8_t *rflags;                 // [N] repair flips (bit per replica)
    int32_t *rties;                  // [8][blocks] repair ties per block
    int32_t *rparams;                // [8][4] repair k, majority, kappa, ties to take
    unsigned long long *hfield;      // [N][2] maintained local fields of the replica group (the
                                     // sorted-window path), or null: fields gathered every class
    long long spin_limit;            // polls before a device wait gives up (error word set)
    unsigned int bar_start;          // nonzero: the barrier's gate starts closed (test hook)
};

// One annealing call.
struct GdiDevRun {
    int8_t *spins;                   // [R][N] spins in rank space
    const uint32_t *tab;             // threshold rows (see gdi_api.cpp: build_table)
    const int32_t *tab_off;          // [M+1] row offsets into tab
    const float *temp;               // [M] T_s (Metropolis; only guides the E* search)
    int32_t mode;                    // 0 Metropolis, 1 paper P_f
    int32_t sweeps;                  // M
    int32_t s_begin, s_end;
    int32_t max_row;                 // longest table row
    uint32_t key0, key1;             // Philox key = (seed low, seed high)
    int32_t flags;
    int32_t *raw_G, *final_G;        // [Q*R]
    int64_t *raw_cut, *final_cut;    // [Q*R]
    uint64_t *tr_digest;             // [Q*R][M] or null
    int32_t *tr_G;
    int64_t *tr_cut;
    int32_t *err;                    // device error word (0 = ok)
    const int32_t *item_order;       // [Q*R] items, largest instance first (CTA path)
    int32_t *item_counter;           // [1] next item to take (zeroed before the launch)
};

// record a failure for gdi_last_error() (gdi_api.cpp); returns code
#ifdef __cplusplus
#include <string>
int gdi_set_error(int code, const std::string &msg);
#endif

// kernel launch wrappers (gdi_kernels.cu); return a cudaError_t as int
int gdi_launch_init(const GdiDevProblem &P, int8_t *spins, const int8_t *init_orig, int init_kind,
                    uint32_t key0, uint32_t key1, void *stream);
int gdi_launch_cta_anneal(const GdiDevProblem &P, const GdiDevRun &R, int block, int grid_limit,
                          void *stream, int *grid_used, size_t *smem_used);
int gdi_cta_smem_bytes(const GdiDevProblem &P, const GdiDevRun &R, int block, size_t *bytes, int *hist);
// resident CTA-path blocks per SM for this problem and block size (0 when the block does not fit)
int gdi_cta_blocks_per_sm(const GdiDevProblem &P, const GdiDevRun &R, int block, int *per_sm);
// Grid plan for `sms` blocks: spans of ranks (spc) and windows (wpc) per block and per class, and
// the dynamic shared memory; -1 if the instance does not fit smem_limit.
int gdi_grid_plan(const GdiDevProblem &P, int max_row, int sms, size_t smem_limit, int *spc, int *wpc,
                  size_t *smem);
// Host: first window of every block, per class, for the sorted-window grid path.  cost[k] is the
// cost of window k of the class (windows of one class consecutive, class c starting at
// cost_off[c]); every block gets at most wpc windows.  bnd has num_classes * (blocks + 1) entries.
void gdi_grid_window_bounds(const int64_t *cost, const int64_t *cost_off, int num_classes, int blocks,
                            int wpc, int32_t *bnd);
// Event pairs recorded around every anneal kernel launch (timing of the kernel alone).
struct GdiKernelTimer {
    cudaEvent_t *ev;                 // [2 * cap] begin/end events, or null (not timed)
    int cap;                         // pairs available
    int n;                           // pairs recorded
};
int gdi_launch_grid_anneal(const GdiDevProblem &P, const GdiDevRun &R, const GdiGridScratch &X,
                           int8_t *spins, int sms, int spc, int wpc, size_t smem, const int32_t *wbnd,
                           GdiKernelTimer *timer, void *stream);
int gdi_launch_grid_finish(const GdiDevProblem &P, const GdiDevRun &R, const GdiGridScratch &X,
                           int8_t *spins, int do_repair, void *stream);
int gdi_launch_gather_spins(const GdiDevProblem &P, const int8_t *spins_rank, int8_t *out_orig,
                            void *stream);

// flags mirrored from gdi.h
#define GDI_DEV_TRACE 1
#define GDI_DEV_NO_REPAIR 2
#define GDI_DEV_RACY 4
#define GDI_DEV_STANDARD 8

// device error codes written to GdiDevRun::err
#define GDI_DEVERR_RANGE 1
#define GDI_DEVERR_TIMEOUT 2
#define GDI_DEVERR_INPUT 3     // an input check of the launch failed (sizes the caller passed)

#define GDI_GRID_TW 129   // entries of a window table (2 * 64 + 1)
