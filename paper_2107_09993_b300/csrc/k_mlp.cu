// k_mlp.cu -- the learned proposal (a project addition; the paper has none).
//
// A small perceptron reads distribution features of a point set and proposes
// (1) the grid layer of step (a) and (2) 16 filter points that pre-filter
// step (d). The plain path still decides the result: proposals are snapped to
// real data points inside sky_skyline, so a bad proposal only costs time.
//
//   k_features   per-dimension 32-bin histograms of the min/max-normalised
//                values and all pairwise Pearson correlations, over a strided
//                sample of at most 65,536 rows (one CTA)
//   k_dense      y = act(x W^T + b), bf16 weights, fp32 accumulation
//   k_loss       cross-entropy over the admissible layers + lambda x masked
//                MSE of the filter points; writes dL/dy
//   k_dense_bwd_data / k_dense_bwd_weight   backward of k_dense
//   k_adamw      decoupled-weight-decay Adam on fp32 master weights, then the
//                bf16 copy used by the forward pass
//   k_decode     layer = argmax of the admissible logits; filter points back
//                to data units
#include <cuda_bf16.h>

#include <cstdint>
#include <cstdio>

#include "../../include/sky.h"
#include "sky_common.cuh"
#include "sky_internal.h"

namespace sky {
namespace mlp {

constexpr int DMAX = 16, BINS = 32, NL = 8, NF = 16;
constexpr int F_IN = DMAX * BINS + DMAX * (DMAX - 1) / 2 + 4;   // 636
constexpr int HID = 64;
constexpr int OUT = NL + NF * DMAX;                             // 264
constexpr int64_t SAMPLE = 65536;
constexpr int kTileRows = 1024;
static_assert(F_IN == SKY_MLP_FEATURES && OUT == SKY_MLP_OUTPUTS, "header constants");

// parameter offsets (W1, b1, W2, b2, W3, b3), row-major W[n][k]
constexpr int64_t oW1 = 0, ob1 = oW1 + HID * F_IN, oW2 = ob1 + HID, ob2 = oW2 + HID * HID, oW3 = ob2 + HID,
                  ob3 = oW3 + OUT * HID, P = ob3 + OUT;
static_assert(P == SKY_MLP_PARAMS, "parameter count");

__device__ __forceinline__ bool layer_ok(int c, int d) { return (c + 1) * d <= 24; }

// ------------------------------------------------------------- features ---
// The sample: every stride-th row, stride = ceil(n / 65,536), so at most
// 65,536 rows in 64 tiles of 1,024. Three launches:
//   k_feat_minmax  one CTA per tile: per-dimension min / max of the tile
//   k_feat_tile    one CTA per tile: reduces the tile minima / maxima (in
//                  tile order), normalises its rows to [0, 1], and writes
//                  the tile's 32-bin histogram counts and its first and
//                  second moment sums (binary32 over the tile's rows, stored
//                  as binary64)
//   k_feat_final   one CTA: sums the tiles' counts and moments in tile order
//                  and writes the 636 features and the sample range
// The fixed tile decomposition makes the result independent of the GPU's
// SM count and of scheduling.
constexpr int kTiles = (int)(SAMPLE / kTileRows);            // 64
constexpr int kNPair = DMAX * (DMAX + 1) / 2;                 // 136 (k <= l)
constexpr int kNSum = kNPair + DMAX;                          // 152
// per-tile partials in the work buffer, in floats
constexpr int64_t kWorkMM = 0;                                          // [kTiles][2 * DMAX]
constexpr int64_t kWorkHist = kWorkMM + (int64_t)kTiles * 2 * DMAX;     // [kTiles][DMAX * BINS] u32
constexpr int64_t kWorkSum = kWorkHist + (int64_t)kTiles * DMAX * BINS; // [kTiles][kNSum] f64
constexpr int64_t kWorkFeat = kWorkSum + (int64_t)kTiles * kNSum * 2;
static_assert(kWorkSum % 2 == 0, "f64 partials 8-byte aligned");

__device__ __forceinline__ int64_t sample_stride(int64_t n)
{
    const int64_t t = (n + SAMPLE - 1) / SAMPLE;
    return t > 1 ? t : 1;
}

__global__ void __launch_bounds__(kTileRows) k_feat_minmax(const float* __restrict__ pts, int64_t n, int d,
                                                           int64_t ld, float* __restrict__ mm)
{
    __shared__ float s_mn[32][DMAX], s_mx[32][DMAX];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t stride = sample_stride(n), s = (n + stride - 1) / stride;
    const int64_t i = (int64_t)blockIdx.x * kTileRows + tid;
    float mn[DMAX], mx[DMAX];
#pragma unroll
    for (int k = 0; k < DMAX; ++k) { mn[k] = INFINITY; mx[k] = -INFINITY; }
    if (i < s) {
        const float* r = pts + i * stride * ld;
#pragma unroll
        for (int k = 0; k < DMAX; ++k)
            if (k < d) { const float v = __ldg(r + k); mn[k] = v; mx[k] = v; }
    }
#pragma unroll
    for (int k = 0; k < DMAX; ++k) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[k] = fminf(mn[k], __shfl_xor_sync(kFull, mn[k], o));
            mx[k] = fmaxf(mx[k], __shfl_xor_sync(kFull, mx[k], o));
        }
        if (lane == 0) { s_mn[warp][k] = mn[k]; s_mx[warp][k] = mx[k]; }
    }
    __syncthreads();
    if (tid < DMAX) {
        float lo = INFINITY, hi = -INFINITY;
        for (int w = 0; w < kTileRows / 32; ++w) { lo = fminf(lo, s_mn[w][tid]); hi = fmaxf(hi, s_mx[w][tid]); }
        mm[blockIdx.x * 2 * DMAX + tid] = lo;
        mm[blockIdx.x * 2 * DMAX + DMAX + tid] = hi;
    }
}

__global__ void __launch_bounds__(kTileRows) k_feat_tile(const float* __restrict__ pts, int64_t n, int d, int64_t ld,
                                                         const float* __restrict__ mm, int tiles,
                                                         uint32_t* __restrict__ hist_out,
                                                         double* __restrict__ sum_out, float* __restrict__ range)
{
    extern __shared__ float s_x[];                  // [kTileRows][DMAX]
    __shared__ float s_lo[DMAX], s_inv[DMAX];
    __shared__ uint32_t s_hist[DMAX * BINS];
    const int tid = threadIdx.x;
    const int64_t stride = sample_stride(n), s = (n + stride - 1) / stride;
    if (tid < DMAX) {
        float lo = INFINITY, hi = -INFINITY;
        for (int t = 0; t < tiles; ++t) { lo = fminf(lo, mm[t * 2 * DMAX + tid]); hi = fmaxf(hi, mm[t * 2 * DMAX + DMAX + tid]); }
        if (tid >= d) { lo = 0.0f; hi = 0.0f; }
        const float rg = __fsub_rn(hi, lo);
        s_lo[tid] = lo;
        s_inv[tid] = rg > 0.0f ? __fdiv_rn(1.0f, rg) : 0.0f;
        if (blockIdx.x == 0) { range[tid] = lo; range[DMAX + tid] = hi; }
    }
    for (int t = tid; t < DMAX * BINS; t += kTileRows) s_hist[t] = 0u;
    __syncthreads();
    const int64_t t0 = (int64_t)blockIdx.x * kTileRows;
    const int rows = (int)((s - t0) < kTileRows ? (s - t0) : kTileRows);
    if (tid < rows) {
        const float* r = pts + (t0 + tid) * stride * ld;
#pragma unroll
        for (int k = 0; k < DMAX; ++k) {
            float x = 0.0f;
            if (k < d) {
                x = __fmul_rn(__fsub_rn(__ldg(r + k), s_lo[k]), s_inv[k]);
                x = fminf(fmaxf(x, 0.0f), 1.0f);
                const int b = min(BINS - 1, (int)floorf(__fmul_rn(x, (float)BINS)));
                atomicAdd(&s_hist[k * BINS + b], 1u);
            }
            s_x[tid * DMAX + k] = x;
        }
    }
    __syncthreads();
    for (int t = tid; t < DMAX * BINS; t += kTileRows) hist_out[(int64_t)blockIdx.x * DMAX * BINS + t] = s_hist[t];
    if (tid < kNPair) {               // pair index -> (k, l), k <= l
        int pk = 0, t = tid;
        while (t >= DMAX - pk) { t -= DMAX - pk; ++pk; }
        const int pl = pk + t;
        float acc = 0.0f;
        for (int i = 0; i < rows; ++i) acc = fmaf(s_x[i * DMAX + pk], s_x[i * DMAX + pl], acc);
        sum_out[(int64_t)blockIdx.x * kNSum + tid] = (double)acc;
    } else if (tid < kNSum) {
        const int k = tid - kNPair;
        float acc = 0.0f;
        for (int i = 0; i < rows; ++i) acc += s_x[i * DMAX + k];
        sum_out[(int64_t)blockIdx.x * kNSum + tid] = (double)acc;
    }
}

__global__ void __launch_bounds__(512) k_feat_final(int64_t n, int d, int tiles, const uint32_t* __restrict__ hist,
                                                    const double* __restrict__ sums, float* __restrict__ feat)
{
    __shared__ double s_sum[kNSum];
    const int tid = threadIdx.x;
    const int64_t stride = sample_stride(n), s = (n + stride - 1) / stride;
    if (tid < kNSum) {
        double a = 0.0;
        for (int t = 0; t < tiles; ++t) a += sums[(int64_t)t * kNSum + tid];
        s_sum[tid] = a;
    }
    for (int b = tid; b < DMAX * BINS; b += blockDim.x) {
        uint32_t c = 0;
        for (int t = 0; t < tiles; ++t) c += hist[(int64_t)t * DMAX * BINS + b];
        feat[b] = (float)((double)c / (double)s);
    }
    __syncthreads();
    if (tid < DMAX * (DMAX - 1) / 2) {
        int k = 0, t = tid;
        while (t >= DMAX - 1 - k) { t -= DMAX - 1 - k; ++k; }
        const int l = k + 1 + t;
        auto pair = [&](int a, int b) {   // index of (a, b), a <= b, in the pair list
            return a * DMAX - a * (a - 1) / 2 + (b - a);
        };
        const double ek = s_sum[kNPair + k] / s, el = s_sum[kNPair + l] / s;
        const double vk = s_sum[pair(k, k)] / s - ek * ek;
        const double vl = s_sum[pair(l, l)] / s - el * el;
        const double cv = s_sum[pair(k, l)] / s - ek * el;
        double c = 0.0;
        if (k < d && l < d && vk > 1e-12 && vl > 1e-12) c = cv / sqrt(vk * vl);
        feat[DMAX * BINS + tid] = (float)c;
    }
    if (tid == 0) {
        feat[F_IN - 4] = (float)d / 16.0f;
        feat[F_IN - 3] = (float)(log2((double)s) / 32.0);
        feat[F_IN - 2] = 0.0f;
        feat[F_IN - 1] = 0.0f;
    }
}

// ------------------------------------------------------------------ MLP ---
__global__ void __launch_bounds__(128) k_dense(const float* __restrict__ x, int K, const __nv_bfloat16* __restrict__ W,
                                               const __nv_bfloat16* __restrict__ bias, int N, float* y, int relu)
{
    const int b = blockIdx.x;
    const int nn = blockIdx.y * blockDim.x + threadIdx.x;
    if (nn >= N) return;
    const float* xr = x + (int64_t)b * K;
    const __nv_bfloat16* wr = W + (int64_t)nn * K;
    float acc = __bfloat162float(bias[nn]);
    for (int k = 0; k < K; ++k) acc = fmaf(xr[k], __bfloat162float(wr[k]), acc);
    y[(int64_t)b * N + nn] = relu ? fmaxf(acc, 0.0f) : acc;
}

__global__ void k_loss(const float* __restrict__ y, const int32_t* __restrict__ dims,
                       const int32_t* __restrict__ labels, const float* __restrict__ target,
                       const float* __restrict__ mask, int B, float lam, float* dy, float* loss)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float* yr = y + (int64_t)b * OUT;
    float* dr = dy + (int64_t)b * OUT;
    const int d = dims[b];
    const int lab = labels[b];
    float zmax = -INFINITY;
    for (int c = 0; c < NL; ++c) if (layer_ok(c, d)) zmax = fmaxf(zmax, yr[c]);
    float se = 0.0f;
    for (int c = 0; c < NL; ++c) if (layer_ok(c, d)) se += expf(yr[c] - zmax);
    float L = 0.0f;
    for (int c = 0; c < NL; ++c) {
        const float p = layer_ok(c, d) ? expf(yr[c] - zmax) / se : 0.0f;
        dr[c] = (p - (c == lab ? 1.0f : 0.0f)) / (float)B;
        if (c == lab) L -= logf(p);
    }
    const float* tr = target + (int64_t)b * NF * DMAX;
    const float* mr = mask + (int64_t)b * NF * DMAX;
    float cnt = 0.0f;
    for (int j = 0; j < NF * DMAX; ++j) cnt += mr[j];
    cnt = fmaxf(cnt, 1.0f);
    float mse = 0.0f;
    for (int j = 0; j < NF * DMAX; ++j) {
        const float r = (yr[NL + j] - tr[j]) * mr[j];
        mse += r * r;
        dr[NL + j] = lam * 2.0f * r / cnt / (float)B;
    }
    atomicAdd(loss, (L + lam * mse / cnt) / (float)B);
}

// dx[b][k] = sum_n dy[b][n] W[n][k], times the ReLU mask of act[b][k] (if given)
__global__ void __launch_bounds__(128) k_dense_bwd_data(const float* __restrict__ dy, int N,
                                                        const __nv_bfloat16* __restrict__ W, int K,
                                                        const float* __restrict__ act, float* dx)
{
    const int b = blockIdx.x;
    const int k = blockIdx.y * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const float* dr = dy + (int64_t)b * N;
    float acc = 0.0f;
    for (int nn = 0; nn < N; ++nn) acc = fmaf(dr[nn], __bfloat162float(W[(int64_t)nn * K + k]), acc);
    if (act && !(act[(int64_t)b * K + k] > 0.0f)) acc = 0.0f;
    dx[(int64_t)b * K + k] = acc;
}

// gW[n][k] = sum_b dy[b][n] x[b][k]; column k == K holds the bias gradient
__global__ void __launch_bounds__(256) k_dense_bwd_weight(const float* __restrict__ dy, int N,
                                                          const float* __restrict__ x, int K, int B, float* gW,
                                                          float* gb)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * (K + 1)) return;
    const int nn = (int)(t / (K + 1)), k = (int)(t % (K + 1));
    float acc = 0.0f;
    for (int b = 0; b < B; ++b) acc = fmaf(dy[(int64_t)b * N + nn], k < K ? x[(int64_t)b * K + k] : 1.0f, acc);
    if (k < K) gW[(int64_t)nn * K + k] = acc;
    else gb[nn] = acc;
}

__global__ void __launch_bounds__(256) k_adamw(float* w, const float* __restrict__ g, float* m, float* v,
                                               __nv_bfloat16* wb, int64_t count, float lr, float wd, float b1,
                                               float b2, float eps, float c1, float c2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / c1, vh = vi / c2;
    const float wi = w[i] - lr * (mh / (sqrtf(vh) + eps) + wd * w[i]);
    w[i] = wi;
    wb[i] = __float2bfloat16_rn(wi);
}

__global__ void __launch_bounds__(256) k_round(const float* __restrict__ w, __nv_bfloat16* wb, int64_t count)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) wb[i] = __float2bfloat16_rn(w[i]);
}

// layer and filter points from one output row
__global__ void k_decode(const float* __restrict__ y, int d, const float* __restrict__ range, float inflate,
                         float* prop, int32_t* layer)
{
    const int t = threadIdx.x;
    if (t == 0) {
        int best = 0;
        float bv = -INFINITY;
        for (int c = 0; c < NL; ++c)
            if (layer_ok(c, d) && y[c] > bv) { bv = y[c]; best = c; }
        *layer = best + 1;
    }
    if (t < NF * DMAX) {
        const int j = t / DMAX, k = t % DMAX;
        if (k < d) {
            const float v = fminf(fmaxf(y[NL + j * DMAX + k], 0.0f), 1.0f);
            const float lo = range[k], hi = range[DMAX + k];
            prop[j * d + k] = lo + (v + inflate) * (hi - lo);
        }
    }
}

}  // namespace mlp
}  // namespace sky

// ============================================================ C ABI ======
using namespace sky;
using namespace sky::mlp;

namespace {

thread_local char t_merr[256];

sky_status mfail(sky_status s, const char* m, cudaError_t e = cudaSuccess)
{
    snprintf(t_merr, sizeof(t_merr), "%s%s%s", m, e != cudaSuccess ? ": " : "", e != cudaSuccess ? cudaGetErrorString(e) : "");
    return s;
}

cudaError_t forward_impl(const __nv_bfloat16* w, const float* feat, int B, float* out, float* work, cudaStream_t s)
{
    float* h1 = work;
    float* h2 = work + (int64_t)B * HID;
    k_dense<<<dim3(B, (HID + 127) / 128), 128, 0, s>>>(feat, F_IN, w + oW1, w + ob1, HID, h1, 1);
    k_dense<<<dim3(B, (HID + 127) / 128), 128, 0, s>>>(h1, HID, w + oW2, w + ob2, HID, h2, 1);
    k_dense<<<dim3(B, (OUT + 127) / 128), 128, 0, s>>>(h2, HID, w + oW3, w + ob3, OUT, out, 0);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

const char* sky_mlp_last_error(void) { return t_merr; }

size_t sky_mlp_work_floats(int32_t batch)
{
    return (size_t)batch * (size_t)(2 * HID + OUT + OUT + 2 * HID) + 64;
}

size_t sky_features_work_floats(void) { return (size_t)kWorkFeat; }

sky_status sky_features(const float* d_pts, int64_t n, int32_t d, int64_t ld, float* d_feat, float* d_range,
                        float* d_work, void* stream)
{
    if (d < 1 || d > DMAX || n < 1 || ld < d || !d_pts || !d_feat || !d_range || !d_work)
        return mfail(SKY_ERR_INVALID_ARGUMENT, "bad features arguments");
    if (reinterpret_cast<uintptr_t>(d_work) % 8 != 0) return mfail(SKY_ERR_INVALID_ARGUMENT, "work not 8-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t stride = (n + SAMPLE - 1) / SAMPLE > 1 ? (n + SAMPLE - 1) / SAMPLE : 1;
    const int64_t s = (n + stride - 1) / stride;
    const int tiles = (int)((s + kTileRows - 1) / kTileRows);
    float* mm = d_work + kWorkMM;
    uint32_t* hist = reinterpret_cast<uint32_t*>(d_work + kWorkHist);
    double* sums = reinterpret_cast<double*>(d_work + kWorkSum);
    k_feat_minmax<<<tiles, kTileRows, 0, st>>>(d_pts, n, d, ld, mm);
    const int smem = kTileRows * DMAX * (int)sizeof(float);
    cudaFuncSetAttribute(k_feat_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_feat_tile<<<tiles, kTileRows, smem, st>>>(d_pts, n, d, ld, mm, tiles, hist, sums, d_range);
    k_feat_final<<<1, 512, 0, st>>>(n, d, tiles, hist, sums, d_feat);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SKY_OK : mfail(SKY_ERR_CUDA, "features launch", e);
}

sky_status sky_mlp_forward(const uint16_t* d_params_bf16, const float* d_feat, int32_t batch, float* d_out,
                           float* d_work, void* stream)
{
    if (!d_params_bf16 || !d_feat || !d_out || !d_work || batch < 1)
        return mfail(SKY_ERR_INVALID_ARGUMENT, "bad forward arguments");
    const cudaError_t e = forward_impl(reinterpret_cast<const __nv_bfloat16*>(d_params_bf16), d_feat, batch, d_out,
                                       d_work, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SKY_OK : mfail(SKY_ERR_CUDA, "forward launch", e);
}

sky_status sky_mlp_round(const float* d_master, uint16_t* d_bf16, int64_t count, void* stream)
{
    if (!d_master || !d_bf16 || count < 0) return mfail(SKY_ERR_INVALID_ARGUMENT, "bad round arguments");
    if (count == 0) return SKY_OK;
    k_round<<<(unsigned)((count + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        d_master, reinterpret_cast<__nv_bfloat16*>(d_bf16), count);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SKY_OK : mfail(SKY_ERR_CUDA, "round launch", e);
}

sky_status sky_mlp_backward(const uint16_t* d_params_bf16, const float* d_feat, const int32_t* d_dims,
                            const int32_t* d_labels, const float* d_targets, const float* d_masks, int32_t batch,
                            float lam, float* d_grad, float* d_work, float* d_loss, void* stream)
{
    if (!d_params_bf16 || !d_feat || !d_dims || !d_labels || !d_targets || !d_masks || !d_grad || !d_work ||
        !d_loss || batch < 1)
        return mfail(SKY_ERR_INVALID_ARGUMENT, "bad backward arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const __nv_bfloat16* w = reinterpret_cast<const __nv_bfloat16*>(d_params_bf16);
    const int B = batch;
    float* h1 = d_work;
    float* h2 = h1 + (int64_t)B * HID;
    float* y = h2 + (int64_t)B * HID;
    float* dy = y + (int64_t)B * OUT;
    float* dh2 = dy + (int64_t)B * OUT;
    float* dh1 = dh2 + (int64_t)B * HID;
    cudaMemsetAsync(d_loss, 0, sizeof(float), s);
    forward_impl(w, d_feat, B, y, d_work, s);
    k_loss<<<(B + 127) / 128, 128, 0, s>>>(y, d_dims, d_labels, d_targets, d_masks, B, lam, dy, d_loss);
    k_dense_bwd_weight<<<(unsigned)(((int64_t)OUT * (HID + 1) + 255) / 256), 256, 0, s>>>(dy, OUT, h2, HID, B,
                                                                                         d_grad + oW3, d_grad + ob3);
    k_dense_bwd_data<<<dim3(B, (HID + 127) / 128), 128, 0, s>>>(dy, OUT, w + oW3, HID, h2, dh2);
    k_dense_bwd_weight<<<(unsigned)(((int64_t)HID * (HID + 1) + 255) / 256), 256, 0, s>>>(dh2, HID, h1, HID, B,
                                                                                         d_grad + oW2, d_grad + ob2);
    k_dense_bwd_data<<<dim3(B, (HID + 127) / 128), 128, 0, s>>>(dh2, HID, w + oW2, HID, h1, dh1);
    k_dense_bwd_weight<<<(unsigned)(((int64_t)HID * (F_IN + 1) + 255) / 256), 256, 0, s>>>(dh1, HID, d_feat, F_IN, B,
                                                                                          d_grad + oW1, d_grad + ob1);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SKY_OK : mfail(SKY_ERR_CUDA, "backward launch", e);
}

sky_status sky_mlp_adamw(float* d_master, uint16_t* d_bf16, float* d_m, float* d_v, const float* d_grad,
                         int32_t step, float lr, float wd, void* stream)
{
    if (!d_master || !d_bf16 || !d_m || !d_v || !d_grad || step < 1)
        return mfail(SKY_ERR_INVALID_ARGUMENT, "bad adamw arguments");
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    k_adamw<<<(unsigned)((P + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        d_master, d_grad, d_m, d_v, reinterpret_cast<__nv_bfloat16*>(d_bf16), P, lr, wd, b1, b2, eps, c1, c2);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SKY_OK : mfail(SKY_ERR_CUDA, "adamw launch", e);
}

sky_status sky_propose(const float* d_pts, int64_t n, int32_t d, int64_t ld, const uint16_t* d_params_bf16,
                       float inflate, int64_t n_ref, float* d_prop, int32_t* h_log2g, float* d_work, void* stream)
{
    if (!d_params_bf16 || !d_prop || !h_log2g || !d_work || n_ref < 0)
        return mfail(SKY_ERR_INVALID_ARGUMENT, "bad propose arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float* feat = d_work + kWorkFeat;
    float* range = feat + F_IN;
    float* y = range + 2 * DMAX;
    float* act = y + OUT;
    int32_t* layer = reinterpret_cast<int32_t*>(act + 2 * HID);
    sky_status st = sky_features(d_pts, n, d, ld, feat, range, d_work, stream);
    if (st != SKY_OK) return st;
    cudaError_t e = forward_impl(reinterpret_cast<const __nv_bfloat16*>(d_params_bf16), feat, 1, y, act, s);
    if (e == cudaSuccess) {
        k_decode<<<1, 256, 0, s>>>(y, d, range, inflate, d_prop, layer);
        e = cudaGetLastError();
    }
    int32_t lg = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&lg, layer, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return mfail(SKY_ERR_CUDA, "propose", e);
    if (n_ref > 0) {
        // The network's layer is the best layer for a set of n_ref rows with
        // these features; the automatic policy's change from n_ref to n rows
        // carries it to this set's size.
        lg += auto_log2g(n, d) - auto_log2g(n_ref, d);
        int top = 24 / d > 1 ? 24 / d : 1;
        if (top > kMaxAutoLayer) top = kMaxAutoLayer;
        lg = lg < 1 ? 1 : (lg > top ? top : lg);
    }
    *h_log2g = lg;
    return SKY_OK;
}

size_t sky_propose_work_floats(void) { return (size_t)(kWorkFeat + F_IN + 2 * DMAX + OUT + 2 * HID + 8); }

}  // extern "C"
