// gdi_static.cu -- gdi_anneal_static: the grid-scale sweep without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while device memory is owned by another
// allocator (a framework's caching pool or a fixed arena), or a process that must not grow its
// device footprint after start-up.  gdi_anneal allocates its table, staging and grid scratch on
// first use, so those callers cannot use it.  This entry point runs the same grid-scale sweep
// kernel, but its scratch (packed spins of one 8-replica group, the per-block window tables, the
// chain inputs, the class-start magnetisations, the barrier counters and the error word) lives in
// one file-scope __device__ array of fixed size, which every GPU that loads the library holds
// until the process exits.  The caller passes every input and output as device pointers.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "gdi.h"
#include "gdi_internal.h"

namespace {

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr size_t ST_MAX_N = (size_t)GDI_STATIC_MAX_VERTICES;
constexpr size_t ST_MAX_BLOCKS = (size_t)GDI_STATIC_MAX_BLOCKS;
constexpr size_t OFF_PACKED = 0;
constexpr size_t OFF_TABLES = OFF_PACKED + align256(ST_MAX_N);
constexpr size_t OFF_GIN = OFF_TABLES + align256(ST_MAX_BLOCKS * 8 * GDI_GRID_TW * sizeof(int16_t));
constexpr size_t OFF_GCLS = OFF_GIN + align256(ST_MAX_BLOCKS * 8 * sizeof(int32_t));
constexpr size_t OFF_BAR = OFF_GCLS + 256;
constexpr size_t OFF_ERR = OFF_BAR + 256;
constexpr size_t OFF_STATUS = OFF_ERR + 256;
constexpr size_t OFF_META = OFF_STATUS + 256;   // node_off int64[2], class_off int32[2]
constexpr size_t ST_TOTAL = OFF_META + 256;

// The scratch.  Host code must not take its address directly (the name is a host-side stand-in);
// it uses the device address from cudaGetSymbolAddress, fetched once per device.
__device__ __align__(256) unsigned char g_gdi_static_scratch[ST_TOTAL];

struct DeviceSlot {
    std::once_flag once;
    cudaError_t err = cudaSuccess;
    unsigned char *ptr = nullptr;
};
constexpr int ST_MAX_DEVICES = 64;
DeviceSlot g_slots[ST_MAX_DEVICES];

__global__ void static_meta_kernel(int64_t *node_off, int32_t *class_off, int64_t n, int32_t nbounds)
{
    node_off[0] = 0;
    node_off[1] = n;
    class_off[0] = 0;
    class_off[1] = nbounds;
}

// Input checks, enqueued before the anneal (the sizes and arrays come from the caller, and the
// kernel's shared-memory plan trusts them).  Rows: row_ptr starts at 0 and every row holds 0 ..
// max_degree entries, so every row lies inside [0, row_ptr[n]).
__global__ void static_rows_check_kernel(int32_t n, const int64_t *row_ptr, int32_t max_degree, int32_t *err)
{
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = row_ptr[i + 1] - row_ptr[i];
        if (d < 0 || d > max_degree) bad = 1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && row_ptr[0] != 0) bad = 1;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(err, 0, GDI_DEVERR_INPUT);
}

// Columns (only once the rows passed): every neighbour rank lies in [0, n) and outside the row's
// own colour class (a proper colouring, which also rules out self-loops).
__global__ void static_cols_check_kernel(int32_t n, const int64_t *row_ptr, const uint32_t *col,
                                         const int32_t *class_ptr, int32_t num_classes, int32_t *err)
{
    if (*(volatile int32_t *)err) return;
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = 0, hi = num_classes;          // class k of rank i: class_ptr[k] <= i < class_ptr[k + 1]
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (class_ptr[mid] <= i) lo = mid; else hi = mid;
        }
        const int64_t c0 = class_ptr[lo], c1 = class_ptr[lo + 1];
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int64_t j = (int64_t)(col[e] & 0x7FFFFFFFu);
            if (j >= n || (j >= c0 && j < c1)) bad = 1;
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(err, 0, GDI_DEVERR_INPUT);
}

__global__ void static_status_kernel(const int32_t *err, int32_t *out)
{
    const int32_t e = *(volatile const int32_t *)err;
    *out = e == 0 ? GDI_OK : e == GDI_DEVERR_TIMEOUT ? GDI_ERR_TIMEOUT
         : e == GDI_DEVERR_INPUT ? GDI_ERR_INVALID_ARG : GDI_ERR_CUDA;
}

// the device address of the static array on the current device (looked up once per device)
int static_base(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return gdi_set_error(GDI_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= ST_MAX_DEVICES)
        return gdi_set_error(GDI_ERR_TOO_LARGE, "gdi_anneal_static: device ordinal above 63");
    DeviceSlot &slot = g_slots[dev];
    std::call_once(slot.once, [&slot]() {
        slot.err = cudaGetSymbolAddress((void **)&slot.ptr, g_gdi_static_scratch);
    });
    if (slot.err != cudaSuccess || !slot.ptr)
        return gdi_set_error(GDI_ERR_CUDA, std::string("cudaGetSymbolAddress(static scratch): ") +
                                               cudaGetErrorString(slot.err));
    *out = slot.ptr;
    return GDI_OK;
}

}  // namespace

extern "C" int gdi_anneal_static_status(int32_t *status, void *stream)
{
    if (!status) return gdi_set_error(GDI_ERR_INVALID_ARG, "gdi_anneal_static_status: null pointer");
    unsigned char *base = nullptr;
    const int rc = static_base(&base);
    if (rc) return rc;
    static_status_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(reinterpret_cast<const int32_t *>(base + OFF_ERR), status);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return gdi_set_error(GDI_ERR_CUDA, std::string("gdi_anneal_static_status: ") + cudaGetErrorString(e));
    return GDI_OK;
}

extern "C" int gdi_anneal_static(int32_t n, const int64_t *row_ptr, const uint32_t *col,
                                 int32_t num_classes, const int32_t *class_ptr, int32_t max_class,
                                 int32_t max_degree, int32_t A, int32_t B, int32_t W, int32_t mode,
                                 const uint32_t *tab, const int32_t *tab_off, const float *temp,
                                 int32_t max_row, int32_t sweeps, int32_t first_sweep,
                                 int32_t last_sweep, uint64_t seed, int32_t replicas, int8_t *spins,
                                 int32_t *G_out, void *stream)
{
    if (!row_ptr || !col || !class_ptr || !tab || !tab_off || !spins || !G_out)
        return gdi_set_error(GDI_ERR_INVALID_ARG, "gdi_anneal_static: null device pointer");
    if (n < 1 || (int64_t)n > GDI_STATIC_MAX_VERTICES)
        return gdi_set_error(GDI_ERR_TOO_LARGE, "gdi_anneal_static: n = " + std::to_string(n) +
                                                    " outside [1, " + std::to_string(GDI_STATIC_MAX_VERTICES) +
                                                    "], the size of its static scratch");
    if (replicas < 1 || replicas > 8)
        return gdi_set_error(GDI_ERR_TOO_LARGE, "gdi_anneal_static: replicas must be 1..8");
    if (num_classes < 1 || max_class < 1 || max_class > n || W < 1 || A < 0 || B < 1 || sweeps < 1 ||
        max_row < 0 || (mode != GDI_METROPOLIS && mode != GDI_PAPER_PF) || max_degree < 0)
        return gdi_set_error(GDI_ERR_INVALID_ARG, "gdi_anneal_static: bad size or model argument");
    const int32_t s_end = last_sweep > 0 ? last_sweep : sweeps;
    if (first_sweep < 0 || s_end > sweeps || first_sweep > s_end)
        return gdi_set_error(GDI_ERR_INVALID_ARG, "gdi_anneal_static: sweep range outside the schedule");
    if (max_degree > 32767)
        return gdi_set_error(GDI_ERR_TOO_LARGE, "gdi_anneal_static: degree above 32767");
    if ((int64_t)B * max_degree + 4LL * A + max_row + 1 >= ((int64_t)1 << 29))
        return gdi_set_error(GDI_ERR_OVERFLOW, "gdi_anneal_static: B * max_degree + 4A + E_cap >= 2^29");

    unsigned char *base = nullptr;
    int rcb = static_base(&base);
    if (rcb) return rcb;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return gdi_set_error(GDI_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));

    int sms = 0, optin = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int nblk = sms < (int)ST_MAX_BLOCKS ? sms : (int)ST_MAX_BLOCKS;

    GdiDevProblem P;
    P.num_instances = 1;
    P.replicas = replicas;
    P.N = n;
    P.node_off = reinterpret_cast<const int64_t *>(base + OFF_META);
    P.class_off = reinterpret_cast<const int32_t *>(base + OFF_META + 16);
    P.class_ptr = class_ptr;
    P.row_ptr = row_ptr;
    P.col = col;
    P.col16 = nullptr;
    P.rank_of = nullptr;
    P.A = A;
    P.B = B;
    P.W = W;
    P.max_n = n;
    P.max_window = W < max_class ? W : max_class;
    P.max_degree = max_degree;
    P.max_class = max_class;
    int spc = 0, wpc = 0;
    size_t smem = 0;
    if (gdi_grid_plan(P, max_row, nblk, (size_t)optin, &spc, &wpc, &smem) != 0)
        return gdi_set_error(GDI_ERR_TOO_LARGE, "gdi_anneal_static: the plan needs " + std::to_string(smem) +
                                                    " bytes of shared memory per block; use a smaller W");

    GdiGridScratch X;
    X.packed = base + OFF_PACKED;
    X.tables = reinterpret_cast<int16_t *>(base + OFF_TABLES);
    X.gin = reinterpret_cast<int32_t *>(base + OFF_GIN);
    X.Gcls = reinterpret_cast<int32_t *>(base + OFF_GCLS);
    X.bar = reinterpret_cast<unsigned int *>(base + OFF_BAR);
    X.err = reinterpret_cast<int32_t *>(base + OFF_ERR);
    X.status = reinterpret_cast<int32_t *>(base + OFF_STATUS);
    X.rhist = nullptr;
    X.rflags = nullptr;
    X.rties = nullptr;
    X.rparams = nullptr;
    X.hfield = nullptr;
    X.spin_limit = 1ll << 26;
    X.bar_start = 0;

    GdiDevRun R;
    R.spins = spins;
    R.tab = tab;
    R.tab_off = tab_off;
    R.temp = temp;
    R.mode = mode;
    R.sweeps = sweeps;
    R.s_begin = first_sweep;
    R.s_end = s_end;
    R.max_row = max_row;
    R.key0 = (uint32_t)seed;
    R.key1 = (uint32_t)(seed >> 32);
    R.flags = 0;
    R.raw_G = G_out;
    R.final_G = nullptr;
    R.raw_cut = nullptr;
    R.final_cut = nullptr;
    R.tr_digest = nullptr;
    R.tr_G = nullptr;
    R.tr_cut = nullptr;
    R.err = X.err;

    cudaStream_t st = (cudaStream_t)stream;
    // the array keeps the previous call's contents: clear the words that must start at zero
    // (the launcher clears the barrier and the magnetisations of every replica group itself)
    static_meta_kernel<<<1, 1, 0, st>>>(reinterpret_cast<int64_t *>(base + OFF_META),
                                         reinterpret_cast<int32_t *>(base + OFF_META + 16), n,
                                         num_classes + 1);
    e = cudaMemsetAsync(X.err, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(X.status, 0, 16 * sizeof(int32_t), st);
    if (e != cudaSuccess) return gdi_set_error(GDI_ERR_CUDA, std::string("gdi_anneal_static: ") + cudaGetErrorString(e));
    // input checks; a failure leaves the error word set and the anneal kernel returns at entry
    {
        const int cb = (int)std::min<int64_t>(((int64_t)n + 255) / 256, (int64_t)nblk * 8);
        static_rows_check_kernel<<<cb, 256, 0, st>>>(n, row_ptr, max_degree, X.err);
        static_cols_check_kernel<<<cb, 256, 0, st>>>(n, row_ptr, col, class_ptr, num_classes, X.err);
    }
    const int ke = gdi_launch_grid_anneal(P, R, X, spins, nblk, spc, wpc, smem, nullptr, nullptr, st);
    if (ke) return gdi_set_error(GDI_ERR_CUDA, std::string("gdi_anneal_static launch: ") +
                                                   cudaGetErrorString((cudaError_t)ke));
    return GDI_OK;
}
