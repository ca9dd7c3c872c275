// gdi_mpnn.cu -- kernels of the learned warm start: a 3-layer message-passing network over a batch
// of graphs (disjoint union CSR), its training (loss, backward, Adam) and the rounding of its
// logits to an exactly balanced initial spin assignment for gdi_anneal.
//
// Layer l: H_l = ReLU(H_{l-1} Ws_l + (A_mean H_{l-1}) Wn_l + b_l), A_mean = D^-1 A (mean over
// neighbours).  Output z = H_3 wo + bo.  Weights are BF16 (round-to-nearest-even copies of FP32
// master weights); activations, accumulations and gradients are FP32.  The dense layers of the
// network (din = 16 and 64), forward and backward, run on the tensor cores (mma.sync m16n8k16,
// BF16 operands, FP32 accumulation) with the FP32 activations split into two BF16 parts; the
// neighbour aggregations are CSR gathers with one warp per vertex and lanes over channels.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gdi_device.cuh"
#include "gdi_mpnn.h"

using namespace gdi;

namespace {

constexpr int HID = GDI_MPNN_HIDDEN;   // 64
constexpr int FIN = GDI_MPNN_FEATURES; // 16
constexpr int NRAND = 8;               // random positional channels

inline bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

__device__ __forceinline__ float bf16_to_f(uint16_t b)
{
    return __uint_as_float((uint32_t)b << 16);
}

__device__ __forceinline__ int64_t graph_of(const int64_t *graph_ptr, int G, int64_t i)
{
    int lo = 0, hi = G - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (graph_ptr[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------------------------
// Aggregation, one warp per destination vertex, lanes over channels (d <= 64):
//   mode 0: Y_i = (1/deg_i) sum_{j in N(i)} X_j               (A_mean X)
//   mode 1: Y_j = sum_{i in N(j)} X_i / deg_i                 (A_mean^T X, graph symmetric)
//   mode 2: Y_i = 0.5 X_i + 0.5 sum_{j in N(i)} X_j / sqrt(deg_i deg_j)   (lazy normalised walk)
// accumulate: Y += result instead of Y = result.
__global__ void aggregate_kernel(int64_t N, const int64_t *row_ptr, const int32_t *col, const float *X,
                                 int d, float *Y, int mode, int accumulate)
{
    const int lane = threadIdx.x & 31;
    const int64_t wglob = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = wglob; i < N; i += nw) {
        const int64_t e0 = row_ptr[i], e1 = row_ptr[i + 1];
        const float degi = (float)(e1 - e0);
        float a0 = 0.f, a1 = 0.f;
        for (int64_t e = e0; e < e1; ++e) {
            const int64_t j = col[e];
            float wgt = 1.f;
            if (mode == 1) {
                const float dj = (float)(row_ptr[j + 1] - row_ptr[j]);
                wgt = 1.f / dj;
            } else if (mode == 2) {
                const float dj = (float)(row_ptr[j + 1] - row_ptr[j]);
                wgt = rsqrtf(degi * dj);
            }
            if (lane < d) a0 += wgt * X[j * d + lane];
            if (lane + 32 < d) a1 += wgt * X[j * d + lane + 32];
        }
        if (mode == 0 && e1 > e0) { a0 /= degi; a1 /= degi; }
        if (mode == 2) {
            if (lane < d) a0 = 0.5f * X[i * d + lane] + 0.5f * a0;
            if (lane + 32 < d) a1 = 0.5f * X[i * d + lane + 32] + 0.5f * a1;
        }
        if (lane < d) Y[i * d + lane] = accumulate ? Y[i * d + lane] + a0 : a0;
        if (lane + 32 < d) Y[i * d + lane + 32] = accumulate ? Y[i * d + lane + 32] + a1 : a1;
    }
}

// ---------------------------------------------------------------------------------------------
// Dense forward: H = ReLU(X Ws + AGG Wn + b), X/AGG: N x din, Ws/Wn: din x 64 (BF16), H: N x 64.
__global__ void dense_fwd_kernel(int64_t N, const float *X, const float *AGG, int din, const uint16_t *Ws,
                                 const uint16_t *Wn, const float *b, float *H, int relu)
{
    extern __shared__ float sm[];
    float *ws = sm, *wn = sm + din * HID;
    for (int t = threadIdx.x; t < din * HID; t += blockDim.x) { ws[t] = bf16_to_f(Ws[t]); wn[t] = bf16_to_f(Wn[t]); }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t wglob = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = wglob; i < N; i += nw) {
        const float x0 = lane < din ? X[i * din + lane] : 0.f;
        const float x1 = lane + 32 < din ? X[i * din + lane + 32] : 0.f;
        const float g0 = lane < din ? AGG[i * din + lane] : 0.f;
        const float g1 = lane + 32 < din ? AGG[i * din + lane + 32] : 0.f;
        float o0 = b[lane], o1 = b[lane + 32];
        for (int k = 0; k < din; ++k) {
            const float xk = __shfl_sync(0xFFFFFFFFu, k < 32 ? x0 : x1, k & 31);
            const float gk = __shfl_sync(0xFFFFFFFFu, k < 32 ? g0 : g1, k & 31);
            o0 += xk * ws[k * HID + lane] + gk * wn[k * HID + lane];
            o1 += xk * ws[k * HID + lane + 32] + gk * wn[k * HID + lane + 32];
        }
        if (relu) { o0 = fmaxf(o0, 0.f); o1 = fmaxf(o1, 0.f); }
        H[i * HID + lane] = o0;
        H[i * HID + lane + 32] = o1;
    }
}

// Dense backward (data): dPRE = dH * [H > 0]; dXs = dPRE Ws^T; T = dPRE Wn^T  (N x din each).
__global__ void dense_bwd_kernel(int64_t N, int din, const uint16_t *Ws, const uint16_t *Wn, const float *H,
                                 const float *dH, float *dPRE, float *dXs, float *T)
{
    extern __shared__ float sm[];
    float *wsT = sm, *wnT = sm + din * HID;   // transposed: [c][k]
    for (int t = threadIdx.x; t < din * HID; t += blockDim.x) {
        const int k = t / HID, c = t % HID;
        wsT[c * din + k] = bf16_to_f(Ws[t]);
        wnT[c * din + k] = bf16_to_f(Wn[t]);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t wglob = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = wglob; i < N; i += nw) {
        const float p0 = H[i * HID + lane] > 0.f ? dH[i * HID + lane] : 0.f;
        const float p1 = H[i * HID + lane + 32] > 0.f ? dH[i * HID + lane + 32] : 0.f;
        dPRE[i * HID + lane] = p0;
        dPRE[i * HID + lane + 32] = p1;
        float s0 = 0.f, s1 = 0.f, t0 = 0.f, t1 = 0.f;   // outputs k = lane, lane + 32
        for (int c = 0; c < HID; ++c) {
            const float pc = __shfl_sync(0xFFFFFFFFu, c < 32 ? p0 : p1, c & 31);
            if (lane < din) { s0 += pc * wsT[c * din + lane]; t0 += pc * wnT[c * din + lane]; }
            if (lane + 32 < din) { s1 += pc * wsT[c * din + lane + 32]; t1 += pc * wnT[c * din + lane + 32]; }
        }
        if (lane < din) { dXs[i * din + lane] = s0; T[i * din + lane] = t0; }
        if (lane + 32 < din) { dXs[i * din + lane + 32] = s1; T[i * din + lane + 32] = t1; }
    }
}

// ---------------------------------------------------------------------------------------------
// Tensor-core dense layers (din = 16 or 64): mma.sync m16n8k16 with BF16 operands and FP32
// accumulation, one warp per tile of 16 vertices.  The weights are BF16 already; an FP32
// activation x is split into two BF16 parts hi = bf16(x), lo = bf16(x - hi), and hi W + lo W is
// accumulated in FP32: each product of BF16 values is exact in FP32, so the only rounding beyond
// the FP32 sums is the part of x below lo (about 2^-17 of |x|).
// Fragment layout of m16n8k16 (PTX ISA): g = lane / 4, q = lane % 4; A (16 x 16, row major) regs
// a0..a3 = rows g, g + 8, g, g + 8 at columns 2q, 2q + 1 (a0, a1) and 2q + 8, 2q + 9 (a2, a3);
// B (16 x 8, column major) regs b0, b1 = rows 2q, 2q + 1 and 2q + 8, 2q + 9 of column g;
// C/D (16 x 8) c0, c1 = row g, columns 2q, 2q + 1; c2, c3 = row g + 8, same columns.  The lower
// 16 bits of a register hold the element with the smaller index.
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                 "{%8, %9}, {%0, %1, %2, %3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// two FP32 values (element k, k + 1) -> packed BF16 high parts and packed BF16 residuals
__device__ __forceinline__ void split_bf16x2(float x0, float x1, uint32_t &hi, uint32_t &lo)
{
    const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
    const __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
    const __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
    hi = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
    lo = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
}

// H = ReLU([X | AGG] [Ws; Wn] + b): K = 2 DIN, 64 outputs = 8 column tiles.
template <int DIN>
__global__ void __launch_bounds__(256) dense_fwd_mma_kernel(int64_t N, const float *X, const float *AGG,
                                                            const uint16_t *Ws, const uint16_t *Wn,
                                                            const float *b, float *H)
{
    constexpr int K = 2 * DIN, KP = K / 2 + 4;           // pairs per output column (+4: banks)
    __shared__ uint32_t wt[HID * KP];                     // [n][k pair]: (k, k+1) of output n
    for (int t = threadIdx.x; t < HID * (K / 2); t += blockDim.x) {
        const int n = t / (K / 2), kp = t % (K / 2), k = 2 * kp;
        const uint16_t w0 = k < DIN ? Ws[k * HID + n] : Wn[(k - DIN) * HID + n];
        const uint16_t w1 = k + 1 < DIN ? Ws[(k + 1) * HID + n] : Wn[(k + 1 - DIN) * HID + n];
        wt[n * KP + kp] = (uint32_t)w0 | ((uint32_t)w1 << 16);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const int64_t wglob = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float bias[8][2];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) { bias[nt][0] = b[nt * 8 + 2 * q]; bias[nt][1] = b[nt * 8 + 2 * q + 1]; }
    for (int64_t tile = wglob; tile * 16 < N; tile += nw) {
        const int64_t r0 = tile * 16 + g, r1 = r0 + 8;
        float acc[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            acc[nt][0] = acc[nt][2] = bias[nt][0];
            acc[nt][1] = acc[nt][3] = bias[nt][1];
        }
#pragma unroll
        for (int ks = 0; ks < K / 16; ++ks) {
            const float *src = ks * 16 < DIN ? X : AGG;     // a k-step never straddles the two
            const int kk = (ks * 16) % DIN + 2 * q;
            const float2 z = make_float2(0.f, 0.f);
            const float2 v00 = r0 < N ? *reinterpret_cast<const float2 *>(src + r0 * DIN + kk) : z;
            const float2 v10 = r1 < N ? *reinterpret_cast<const float2 *>(src + r1 * DIN + kk) : z;
            const float2 v01 = r0 < N ? *reinterpret_cast<const float2 *>(src + r0 * DIN + kk + 8) : z;
            const float2 v11 = r1 < N ? *reinterpret_cast<const float2 *>(src + r1 * DIN + kk + 8) : z;
            uint32_t ah[4], al[4];
            split_bf16x2(v00.x, v00.y, ah[0], al[0]);
            split_bf16x2(v10.x, v10.y, ah[1], al[1]);
            split_bf16x2(v01.x, v01.y, ah[2], al[2]);
            split_bf16x2(v11.x, v11.y, ah[3], al[3]);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const uint32_t *wr = wt + (nt * 8 + g) * KP + ks * 8 + q;
                const uint32_t b0 = wr[0], b1 = wr[4];
                mma_bf16_16816(acc[nt], ah, b0, b1);
                mma_bf16_16816(acc[nt], al, b0, b1);
            }
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int c = nt * 8 + 2 * q;
            if (r0 < N) *reinterpret_cast<float2 *>(H + r0 * HID + c) = make_float2(fmaxf(acc[nt][0], 0.f), fmaxf(acc[nt][1], 0.f));
            if (r1 < N) *reinterpret_cast<float2 *>(H + r1 * HID + c) = make_float2(fmaxf(acc[nt][2], 0.f), fmaxf(acc[nt][3], 0.f));
        }
    }
}

// Backward (data) of one layer: dPRE = dH * [H > 0] (written out), then dXs = dPRE Ws^T and
// T = dPRE Wn^T: K = 64, DIN outputs each, one pass per weight matrix.
template <int DIN>
__global__ void __launch_bounds__(256) dense_bwd_mma_kernel(int64_t N, const uint16_t *Ws, const uint16_t *Wn,
                                                            const float *H, const float *dH, float *dPRE,
                                                            float *dXs, float *T)
{
    constexpr int KP = HID / 2 + 4;
    __shared__ uint32_t wt[2][DIN * KP];                  // [m][j][c pair]: W_m[j][c], W_m[j][c+1]
    for (int t = threadIdx.x; t < DIN * (HID / 2); t += blockDim.x) {
        const int j = t / (HID / 2), cp = t % (HID / 2);
        wt[0][j * KP + cp] = reinterpret_cast<const uint32_t *>(Ws)[t];
        wt[1][j * KP + cp] = reinterpret_cast<const uint32_t *>(Wn)[t];
    }
    __syncthreads();
    constexpr int NT = DIN / 8;
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const int64_t wglob = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t tile = wglob; tile * 16 < N; tile += nw) {
        const int64_t r0 = tile * 16 + g, r1 = r0 + 8;
        // A fragments of dPRE for the 4 k-steps (c = 16 ks + ...), hi and lo parts
        uint32_t ah[4][4], al[4][4];
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int64_t r = (h & 1) ? r1 : r0;
                const int c = ks * 16 + 2 * q + ((h & 2) ? 8 : 0);
                float2 p = make_float2(0.f, 0.f);
                if (r < N) {
                    const float2 hv = *reinterpret_cast<const float2 *>(H + r * HID + c);
                    const float2 dv = *reinterpret_cast<const float2 *>(dH + r * HID + c);
                    p = make_float2(hv.x > 0.f ? dv.x : 0.f, hv.y > 0.f ? dv.y : 0.f);
                    *reinterpret_cast<float2 *>(dPRE + r * HID + c) = p;
                }
                split_bf16x2(p.x, p.y, ah[ks][h], al[ks][h]);
            }
        }
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            float *out = m == 0 ? dXs : T;
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint32_t *wr = wt[m] + (nt * 8 + g) * KP + ks * 8 + q;
                    const uint32_t b0 = wr[0], b1 = wr[4];
                    mma_bf16_16816(acc, ah[ks], b0, b1);
                    mma_bf16_16816(acc, al[ks], b0, b1);
                }
                const int j = nt * 8 + 2 * q;
                if (r0 < N) *reinterpret_cast<float2 *>(out + r0 * DIN + j) = make_float2(acc[0], acc[1]);
                if (r1 < N) *reinterpret_cast<float2 *>(out + r1 * DIN + j) = make_float2(acc[2], acc[3]);
            }
        }
    }
}

// out[din x dout] += A^T B over the rows of a chunk; A: N x din, B: N x dout (dout <= 64).
// Also colsum[dout] += sum of the rows of B when colsum != null.
__global__ void wgrad_kernel(int64_t N, const float *A, int din, const float *B, int dout, float *out,
                             float *colsum, int64_t chunk)
{
    extern __shared__ float sm[];
    float *sa = sm;                      // [32][din]
    float *sb = sm + 32 * din;           // [32][dout]
    const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(N, r0 + chunk);
    const int outs = din * dout;
    float acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.f;
    float cs = 0.f;
    for (int64_t t0 = r0; t0 < r1; t0 += 32) {
        const int rows = (int)min((int64_t)32, r1 - t0);
        __syncthreads();
        for (int t = threadIdx.x; t < 32 * din; t += blockDim.x) {
            const int rr = t / din, k = t % din;
            sa[t] = rr < rows ? A[(t0 + rr) * din + k] : 0.f;
        }
        for (int t = threadIdx.x; t < 32 * dout; t += blockDim.x) {
            const int rr = t / dout, c = t % dout;
            sb[t] = rr < rows ? B[(t0 + rr) * dout + c] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int o = threadIdx.x + q * blockDim.x;
            if (o < outs) {
                const int k = o / dout, c = o % dout;
                float s = 0.f;
                for (int rr = 0; rr < 32; ++rr) s += sa[rr * din + k] * sb[rr * dout + c];
                acc[q] += s;
            }
        }
        if (colsum && threadIdx.x < dout)
            for (int rr = 0; rr < 32; ++rr) cs += sb[rr * dout + threadIdx.x];
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int o = threadIdx.x + q * blockDim.x;
        if (o < outs && acc[q] != 0.f) atomicAdd(&out[o], acc[q]);
    }
    if (colsum && threadIdx.x < dout && cs != 0.f) atomicAdd(&colsum[threadIdx.x], cs);
}

// z = H wo + bo
__global__ void out_fwd_kernel(int64_t N, const float *H, const uint16_t *wo, const float *bo, float *z)
{
    const int lane = threadIdx.x & 31;
    const int64_t wglob = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float w0 = bf16_to_f(wo[lane]), w1 = bf16_to_f(wo[lane + 32]);
    for (int64_t i = wglob; i < N; i += nw) {
        float s = H[i * HID + lane] * w0 + H[i * HID + lane + 32] * w1;
        s = warp_sum(s);
        if (lane == 0) z[i] = s + bo[0];
    }
}

// dH = dz wo^T
__global__ void out_bwd_kernel(int64_t N, const uint16_t *wo, const float *dz, float *dH)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N * HID; t += (int64_t)gridDim.x * blockDim.x)
        dH[t] = dz[t / HID] * bf16_to_f(wo[t % HID]);
}

// Per graph (one block): L1 = mean softplus(-y z), L2 = mean softplus(y z), m = mean tanh z;
// loss_g = min(L1, L2) + lambda m^2; dz for the chosen sign; loss += loss_g / G.
__device__ __forceinline__ float softplus_f(float x) { return x > 20.f ? x : log1pf(expf(x)); }
__device__ __forceinline__ float sigmoid_f(float x) { return 1.f / (1.f + expf(-x)); }

__global__ void loss_kernel(int G, const int64_t *graph_ptr, const float *z, const int8_t *y, float lambda,
                            float *stats, float *dz, float *loss)
{
    const int g = blockIdx.x;
    const int64_t v0 = graph_ptr[g], v1 = graph_ptr[g + 1];
    const float n = (float)(v1 - v0);
    float l1 = 0.f, l2 = 0.f, th = 0.f;
    for (int64_t i = v0 + threadIdx.x; i < v1; i += blockDim.x) {
        const float yz = (float)y[i] * z[i];
        l1 += softplus_f(-yz);
        l2 += softplus_f(yz);
        th += tanhf(z[i]);
    }
    __shared__ float red[3][32];
    l1 = warp_sum(l1); l2 = warp_sum(l2); th = warp_sum(th);
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = l1; red[1][threadIdx.x >> 5] = l2; red[2][threadIdx.x >> 5] = th; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f, b = 0.f, c = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += red[0][w]; b += red[1][w]; c += red[2][w]; }
        red[0][0] = a / n; red[1][0] = b / n; red[2][0] = c / n;
    }
    __syncthreads();
    const float L1 = red[0][0], L2 = red[1][0], m = red[2][0];
    const float sgn = L1 <= L2 ? 1.f : -1.f;   // target y (sgn = 1) or -y
    const float lg = fminf(L1, L2) + lambda * m * m;
    if (threadIdx.x == 0) {
        stats[g * 4 + 0] = L1; stats[g * 4 + 1] = L2; stats[g * 4 + 2] = m; stats[g * 4 + 3] = lg;
        atomicAdd(loss, lg / (float)G);
    }
    for (int64_t i = v0 + threadIdx.x; i < v1; i += blockDim.x) {
        const float t = sgn * (float)y[i];
        const float th_i = tanhf(z[i]);
        dz[i] = (-t * sigmoid_f(-t * z[i]) + lambda * 2.f * m * (1.f - th_i * th_i)) / (n * (float)G);
    }
}

__global__ void adam_kernel(int64_t P, float *p, const float *g, float *m, float *v, uint16_t *pb, float lr,
                            float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < P; t += (int64_t)gridDim.x * blockDim.x) {
        const float gt = g[t];
        const float mt = b1 * m[t] + (1.f - b1) * gt;
        const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
        m[t] = mt;
        v[t] = vt;
        const float pt = p[t] - lr * (mt / c1) / (sqrtf(vt / c2) + eps);
        p[t] = pt;
        pb[t] = __bfloat16_as_ushort(__float2bfloat16_rn(pt));
    }
}

__global__ void to_bf16_kernel(int64_t P, const float *p, uint16_t *pb)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < P; t += (int64_t)gridDim.x * blockDim.x)
        pb[t] = __bfloat16_as_ushort(__float2bfloat16_rn(p[t]));
}

// ---------------------------------------------------------------------------------------------
// Features: 8 channels of +-1 Philox noise, diffused by `steps` lazy normalised-walk steps, then
// centred and scaled to unit RMS per graph; channel 8 = log(1 + deg), channel 9 = deg / mean deg
// of the graph; channels 10..15 = 0.
__global__ void feat_init_kernel(int64_t N, int G, const int64_t *graph_ptr, const uint32_t *graph_id,
                                 uint32_t k0, uint32_t k1, float *R)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N * NRAND; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / NRAND;
        const int c = (int)(t % NRAND);
        const int g = (int)graph_of(graph_ptr, G, i);
        const uint32_t il = (uint32_t)(i - graph_ptr[g]);
        const uint4 u = philox4x32_10(make_uint4(il, (uint32_t)c, graph_id[g], 0x4D504E4Eu), k0, k1);
        R[t] = (u.x >> 31) ? -1.f : 1.f;
    }
}

// per graph (one block): centre and scale channels of R, write X (N x 16) with degree features.
// flags & GDI_MPNN_ALIGN: channel c >= 1 is multiplied by the sign of its inner product with
// channel 0 (after centring), so that the channels' low-frequency components point the same way
// inside a graph; flags & GDI_MPNN_NO_NOISE: the noise channels are written as 0.
__global__ void feat_finish_kernel(int G, const int64_t *graph_ptr, const int64_t *row_ptr, const float *R,
                                   float *X, int flags)
{
    const int g = blockIdx.x;
    const int64_t v0 = graph_ptr[g], v1 = graph_ptr[g + 1];
    const float n = (float)(v1 - v0);
    __shared__ float red[NRAND + 1][32];
    __shared__ float mean[NRAND + 1], rms[NRAND], sgn[NRAND];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    float s[NRAND + 1];
#pragma unroll
    for (int c = 0; c <= NRAND; ++c) s[c] = 0.f;
    for (int64_t i = v0 + threadIdx.x; i < v1; i += blockDim.x) {
#pragma unroll
        for (int c = 0; c < NRAND; ++c) s[c] += R[i * NRAND + c];
        s[NRAND] += (float)(row_ptr[i + 1] - row_ptr[i]);
    }
#pragma unroll
    for (int c = 0; c <= NRAND; ++c) {
        const float a = warp_sum(s[c]);
        if (lane == 0) red[c][w] = a;
    }
    __syncthreads();
    if (threadIdx.x <= NRAND) {
        float a = 0.f;
        for (int q = 0; q < nwarp; ++q) a += red[threadIdx.x][q];
        mean[threadIdx.x] = a / n;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NRAND; ++c) s[c] = 0.f;
    for (int64_t i = v0 + threadIdx.x; i < v1; i += blockDim.x)
#pragma unroll
        for (int c = 0; c < NRAND; ++c) {
            const float x = R[i * NRAND + c] - mean[c];
            s[c] += x * x;
        }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NRAND; ++c) {
        const float a = warp_sum(s[c]);
        if (lane == 0) red[c][w] = a;
    }
    __syncthreads();
    if (threadIdx.x < NRAND) {
        float a = 0.f;
        for (int q = 0; q < nwarp; ++q) a += red[threadIdx.x][q];
        rms[threadIdx.x] = sqrtf(a / n) + 1e-12f;
    }
    __syncthreads();
    // inner products of the centred channels with channel 0
#pragma unroll
    for (int c = 0; c < NRAND; ++c) s[c] = 0.f;
    if (flags & GDI_MPNN_ALIGN)
        for (int64_t i = v0 + threadIdx.x; i < v1; i += blockDim.x) {
            const float x0 = R[i * NRAND] - mean[0];
#pragma unroll
            for (int c = 1; c < NRAND; ++c) s[c] += x0 * (R[i * NRAND + c] - mean[c]);
        }
    __syncthreads();
#pragma unroll
    for (int c = 1; c < NRAND; ++c) {
        const float a = warp_sum(s[c]);
        if (lane == 0) red[c][w] = a;
    }
    __syncthreads();
    if (threadIdx.x < NRAND) {
        float a = 0.f;
        if (threadIdx.x > 0 && (flags & GDI_MPNN_ALIGN))
            for (int q = 0; q < nwarp; ++q) a += red[threadIdx.x][q];
        sgn[threadIdx.x] = (flags & GDI_MPNN_NO_NOISE) ? 0.f : (a < 0.f ? -1.f : 1.f);
    }
    __syncthreads();
    for (int64_t i = v0 + threadIdx.x; i < v1; i += blockDim.x) {
        const float deg = (float)(row_ptr[i + 1] - row_ptr[i]);
#pragma unroll
        for (int c = 0; c < NRAND; ++c) X[i * FIN + c] = sgn[c] * ((R[i * NRAND + c] - mean[c]) / rms[c]);
        X[i * FIN + NRAND] = log1pf(deg);
        X[i * FIN + NRAND + 1] = mean[NRAND] > 0.f ? deg / mean[NRAND] : 0.f;
#pragma unroll
        for (int c = NRAND + 2; c < FIN; ++c) X[i * FIN + c] = 0.f;
    }
}

// ---------------------------------------------------------------------------------------------
// Rounding (one block per graph): the floor(n/2) largest logits (ties: smaller vertex id first)
// become +1, the rest -1.  Bitonic sort of 64-bit keys in shared memory (n <= 8192).
__device__ __forceinline__ uint32_t float_order_desc(float f)
{
    // map float to uint32 so that larger floats give smaller keys
    uint32_t u = __float_as_uint(f);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);   // ascending order of floats
    return ~u;                                          // descending
}

__global__ void round_kernel(const int64_t *graph_ptr, const float *z, int8_t *spins)
{
    extern __shared__ unsigned long long keys[];
    const int g = blockIdx.x;
    const int64_t v0 = graph_ptr[g];
    const int n = (int)(graph_ptr[g + 1] - v0);
    int P2 = 1;
    while (P2 < n) P2 <<= 1;
    for (int t = threadIdx.x; t < P2; t += blockDim.x)
        keys[t] = t < n ? (((unsigned long long)float_order_desc(z[v0 + t]) << 32) | (unsigned)t)
                        : ~0ull;
    __syncthreads();
    for (int k = 2; k <= P2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < P2; t += blockDim.x) {
                const int p = t ^ j;
                if (p > t) {
                    const bool up = (t & k) == 0;
                    const unsigned long long a = keys[t], b = keys[p];
                    if ((a > b) == up) { keys[t] = b; keys[p] = a; }
                }
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int v = (int)(keys[t] & 0xFFFFFFFFu);
        spins[v0 + v] = t < n / 2 ? 1 : -1;
    }
}

int grid_for(int64_t work, int per_block)
{
    int64_t g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > 152 * 16) g = 152 * 16;
    return (int)g;
}

}  // namespace

extern "C" {

int gdi_mpnn_features(int64_t N, int32_t G, const int64_t *graph_ptr, const uint32_t *graph_id,
                      const int64_t *row_ptr, const int32_t *col, uint64_t seed, int32_t steps,
                      int32_t flags, float *X, float *scratch, void *stream)
{
    if (N < 1 || G < 1 || steps < 0 || !graph_ptr || !graph_id || !row_ptr || !col || !X || !scratch ||
        (flags & ~(GDI_MPNN_ALIGN | GDI_MPNN_NO_NOISE)))
        return GDI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    float *R0 = scratch, *R1 = scratch + N * NRAND;
    feat_init_kernel<<<grid_for(N * NRAND, 256), 256, 0, st>>>(N, G, graph_ptr, graph_id, (uint32_t)seed,
                                                                (uint32_t)(seed >> 32), R0);
    for (int s = 0; s < steps; ++s) {
        aggregate_kernel<<<grid_for(N * 32, 256), 256, 0, st>>>(N, row_ptr, col, R0, NRAND, R1, 2, 0);
        float *t = R0; R0 = R1; R1 = t;
    }
    feat_finish_kernel<<<G, 256, 0, st>>>(G, graph_ptr, row_ptr, R0, X, flags);
    return cudaGetLastError() == cudaSuccess ? GDI_OK : GDI_ERR_CUDA;
}

int gdi_mpnn_aggregate(int64_t N, const int64_t *row_ptr, const int32_t *col, const float *X, int32_t d,
                       float *Y, int32_t mode, int32_t accumulate, void *stream)
{
    if (N < 1 || d < 1 || d > 64 || mode < 0 || mode > 2) return GDI_ERR_INVALID_ARG;
    aggregate_kernel<<<grid_for(N * 32, 256), 256, 0, (cudaStream_t)stream>>>(N, row_ptr, col, X, d, Y, mode,
                                                                              accumulate);
    return cudaGetLastError() == cudaSuccess ? GDI_OK : GDI_ERR_CUDA;
}

int gdi_mpnn_dense_fwd(int64_t N, const float *X, const float *AGG, int32_t din, const uint16_t *Ws,
                       const uint16_t *Wn, const float *b, float *H, void *stream)
{
    if (N < 1 || din < 1 || din > 64) return GDI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int tb = (int)min((N + 15) / 16 * 32 / 256 + 1, (int64_t)152 * 16);   // tiles of 16 rows, 8 warps a block
    // the tensor-core kernels move activations in pairs (8-byte accesses)
    const bool pairs = aligned(X, 8) && aligned(AGG, 8) && aligned(H, 8);
    if (din == 64 && pairs) {
        dense_fwd_mma_kernel<64><<<tb, 256, 0, st>>>(N, X, AGG, Ws, Wn, b, H);
    } else if (din == 16 && pairs) {
        dense_fwd_mma_kernel<16><<<tb, 256, 0, st>>>(N, X, AGG, Ws, Wn, b, H);
    } else {
        const size_t smem = 2 * (size_t)din * HID * sizeof(float);
        dense_fwd_kernel<<<grid_for(N * 32, 256), 256, smem, st>>>(N, X, AGG, din, Ws, Wn, b, H, 1);
    }
    return cudaGetLastError() == cudaSuccess ? GDI_OK : GDI_ERR_CUDA;
}

int gdi_mpnn_dense_bwd(int64_t N, int32_t din, const uint16_t *Ws, const uint16_t *Wn, const float *H,
                       const float *dH, float *dPRE, float *dXs, float *T, void *stream)
{
    if (N < 1 || din < 1 || din > 64) return GDI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int tb = (int)min((N + 15) / 16 * 32 / 256 + 1, (int64_t)152 * 16);
    // pairs of activations (8-byte accesses) and pairs of BF16 weights (4-byte accesses)
    const bool pairs = aligned(H, 8) && aligned(dH, 8) && aligned(dPRE, 8) && aligned(dXs, 8) && aligned(T, 8) &&
                       aligned(Ws, 4) && aligned(Wn, 4);
    if (din == 64 && pairs) {
        dense_bwd_mma_kernel<64><<<tb, 256, 0, st>>>(N, Ws, Wn, H, dH, dPRE, dXs, T);
    } else if (din == 16 && pairs) {
        dense_bwd_mma_kernel<16><<<tb, 256, 0, st>>>(N, Ws, Wn, H, dH, dPRE, dXs, T);
    } else {
        const size_t smem = 2 * (size_t)din * HID * sizeof(float);
        dense_bwd_kernel<<<grid_for(N * 32, 256), 256, smem, st>>>(N, din, Ws, Wn, H, dH, dPRE, dXs, T);
    }
    return cudaGetLastError() == cudaSuccess ? GDI_OK : GDI_ERR_CUDA;
}

int gdi_mpnn_wgrad(int64_t N, const float *A, int32_t din, const float *B, int32_t dout, float *out,
                   float *colsum, void *stream)
{
    if (N < 1 || din < 1 || din > 64 || dout < 1 || dout > 64) return GDI_ERR_INVALID_ARG;
    const int64_t chunk = 1024;
    const int grid = (int)((N + chunk - 1) / chunk);
    const size_t smem = 32 * (size_t)(din + dout) * sizeof(float);
    wgrad_kernel<<<grid, 256, smem, (cudaStream_t)stream>>>(N, A, din, B, dout, out, colsum, chunk);
    return cudaGetLastError() == cudaSuccess ? GDI_OK : GDI_ERR_CUDA;
}

int gdi_mpnn_out_fwd(int64_t N, const float *H, const uint16_t *wo, const float *bo, float *z, void *stream)
{
    if (N < 1) return GDI_ERR_INVALID_ARG;
    out_fwd_kernel<<<grid_for(N * 32, 256), 256, 0, (cudaStream_t)stream>>>(N, H, wo, bo, z);
    return cudaGetLastError() == cudaSuccess ? GDI_OK : GDI_ERR_CUDA;
}

int gdi_mpnn_out_bwd(int64_t N, const uint16_t *wo, const float *dz, float *dH, void *stream)
{
    if (N < 1) return GDI_ERR_INVALID_ARG;
    out_bwd_kernel<<<grid_for(N * HID, 256), 256, 0, (cudaStream_t)stream>>>(N, wo, dz, dH);
    return cudaGetLastError() == cudaSuccess ? GDI_OK : GDI_ERR_CUDA;
}

int gdi_mpnn_loss(int32_t G, const int64_t *graph_ptr, const float *z, const int8_t *y, float lambda,
                  float *stats, float *dz, float *loss, void *stream)
{
    if (G < 1) return GDI_ERR_INVALID_ARG;
    loss_kernel<<<G, 256, 0, (cudaStream_t)stream>>>(G, graph_ptr, z, y, lambda, stats, dz, loss);
    return cudaGetLastError() == cudaSuccess ? GDI_OK : GDI_ERR_CUDA;
}

int gdi_mpnn_adam(int64_t P, float *params, const float *grads, float *m, float *v, uint16_t *params_bf16,
                  float lr, float beta1, float beta2, float eps, int32_t step, void *stream)
{
    if (P < 1 || step < 1) return GDI_ERR_INVALID_ARG;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    adam_kernel<<<grid_for(P, 256), 256, 0, (cudaStream_t)stream>>>(P, params, grads, m, v, params_bf16, lr, beta1,
                                                                     beta2, eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? GDI_OK : GDI_ERR_CUDA;
}

int gdi_mpnn_to_bf16(int64_t P, const float *params, uint16_t *params_bf16, void *stream)
{
    if (P < 1) return GDI_ERR_INVALID_ARG;
    to_bf16_kernel<<<grid_for(P, 256), 256, 0, (cudaStream_t)stream>>>(P, params, params_bf16);
    return cudaGetLastError() == cudaSuccess ? GDI_OK : GDI_ERR_CUDA;
}

int gdi_mpnn_round(int32_t G, const int64_t *graph_ptr, int32_t max_n, const float *z, int8_t *spins,
                   void *stream)
{
    if (G < 1 || max_n < 1 || max_n > 8192) return GDI_ERR_INVALID_ARG;
    int P2 = 1;
    while (P2 < max_n) P2 <<= 1;
    const size_t smem = (size_t)P2 * sizeof(unsigned long long);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(round_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    round_kernel<<<G, 512, smem, (cudaStream_t)stream>>>(graph_ptr, z, spins);
    return cudaGetLastError() == cudaSuccess ? GDI_OK : GDI_ERR_CUDA;
}

}  // extern "C"
