// cnn.cu -- the per-patch refinement-flag predictor: a learned stand-in for
// the b-cell flag buffer of Sec. 3.2 (regridding).  Three 3x3 convolutions of
// 16 channels with ReLU and a 1x1 head to one logit per cell, over the dense
// planes of a level (5 input features per cell), zero padding at the plane
// edge.  Forward in FP32 (training) or with FP16 activations and weights and
// FP32 accumulation (inference); hand-written backward (binary cross-entropy
// with logits, averaged over masked cells) and Adam, all on the device.
//
// Flat parameter vector: for each layer, W (C_out, C_in, k, k) then b (C_out);
// layers (5->16, 3x3), (16->16, 3x3), (16->16, 3x3), (16->1, 1x1).
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include "cnn.h"

namespace tsu {

namespace {

constexpr int HID = kCnnHidden;

struct LayerSpec {
    int cin, cout, k, woff, boff;
};

__host__ __device__ inline LayerSpec layer_spec(int l)
{
    const int cin[4] = {kCnnIn, HID, HID, HID}, cout[4] = {HID, HID, HID, 1}, k[4] = {3, 3, 3, 1};
    int off = 0;
    for (int i = 0; i < l; i++) off += cout[i] * cin[i] * k[i] * k[i] + cout[i];
    LayerSpec s{cin[l], cout[l], k[l], off, off + cout[l] * cin[l] * k[l] * k[l]};
    return s;
}

// y[n, o, i, j] = b[o] + sum_c sum_taps w[o, c, di, dj] x[n, c, i+di-1, j+dj-1]; one thread per output
// pixel computes all C_out channels.  TIN: float or __half storage.
template <typename TIN, typename TOUT, int CIN, int COUT, int K, bool RELU>
__global__ void conv_fwd_kernel(const TIN *__restrict__ x, const float *__restrict__ theta, int off_w, int off_b,
                                TOUT *__restrict__ y, int n, int H, int W, bool half_weights)
{
    __shared__ float sw[COUT * CIN * K * K];
    __shared__ float sb[COUT];
    for (int k = threadIdx.x; k < COUT * CIN * K * K; k += blockDim.x) {
        float v = theta[off_w + k];
        sw[k] = half_weights ? __half2float(__float2half_rn(v)) : v;
    }
    for (int k = threadIdx.x; k < COUT; k += blockDim.x) sb[k] = theta[off_b + k];
    __syncthreads();
    const long long plane = (long long)H * W;
    const long long total = (long long)n * plane;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total; p += (long long)gridDim.x * blockDim.x) {
        const int img = (int)(p / plane);
        const int rem = (int)(p - (long long)img * plane);
        const int i = rem / W, j = rem % W;
        float acc[COUT];
#pragma unroll
        for (int o = 0; o < COUT; o++) acc[o] = sb[o];
        const TIN *xi = x + (long long)img * CIN * plane;
        for (int c = 0; c < CIN; c++) {
#pragma unroll
            for (int di = 0; di < K; di++) {
                const int ii = i + di - K / 2;
                if (ii < 0 || ii >= H) continue;
#pragma unroll
                for (int dj = 0; dj < K; dj++) {
                    const int jj = j + dj - K / 2;
                    if (jj < 0 || jj >= W) continue;
                    const float v = (float)xi[(long long)c * plane + (long long)ii * W + jj];
#pragma unroll
                    for (int o = 0; o < COUT; o++) acc[o] = fmaf(sw[((o * CIN + c) * K + di) * K + dj], v, acc[o]);
                }
            }
        }
        TOUT *yo = y + (long long)img * COUT * plane + rem;
#pragma unroll
        for (int o = 0; o < COUT; o++) {
            float v = RELU ? fmaxf(acc[o], 0.0f) : acc[o];
            yo[(long long)o * plane] = (TOUT)v;
        }
    }
}

// dL/dz of the head and the loss: g = (sigmoid(z) - t) m / M
__global__ void bce_grad_kernel(const float *z, const float *t, const float *m, long long total, float inv_count,
                                float *g, double *loss)
{
    double part = 0.0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total; p += (long long)gridDim.x * blockDim.x) {
        float zz = z[p], tt = t[p], mm = m[p];
        float s = 1.0f / (1.0f + __expf(-zz));
        g[p] = (s - tt) * mm * inv_count;
        float l = fmaxf(zz, 0.0f) - zz * tt + log1pf(__expf(-fabsf(zz)));
        part += (double)(l * mm);
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, part * (double)inv_count);
}

// weight and bias gradients of one layer: dW[o,c,di,dj] = sum g[n,o,i,j] a[n,c,i+di-1,j+dj-1].
// Each block reduces a slice of the pixels for every weight entry (threads over entries) and adds its
// partial sums with one atomic per entry.
template <int CIN, int COUT, int K>
__global__ void conv_wgrad_kernel(const float *__restrict__ g, const float *__restrict__ a, int n, int H, int W,
                                  float *gw, float *gb, int pix_per_block)
{
    constexpr int NW = COUT * CIN * K * K;
    const long long plane = (long long)H * W;
    const long long total = (long long)n * plane;
    const long long p0 = (long long)blockIdx.x * pix_per_block;
    const long long p1 = p0 + pix_per_block < total ? p0 + pix_per_block : total;
    for (int e = threadIdx.x; e < NW + COUT; e += blockDim.x) {
        float acc = 0.0f;
        if (e < NW) {
            const int dj = e % K, di = (e / K) % K, c = (e / (K * K)) % CIN, o = e / (K * K * CIN);
            for (long long p = p0; p < p1; p++) {
                const int img = (int)(p / plane);
                const int rem = (int)(p - (long long)img * plane);
                const int i = rem / W, j = rem % W;
                const int ii = i + di - K / 2, jj = j + dj - K / 2;
                if (ii < 0 || ii >= H || jj < 0 || jj >= W) continue;
                acc = fmaf(g[((long long)img * COUT + o) * plane + rem],
                           a[((long long)img * CIN + c) * plane + (long long)ii * W + jj], acc);
            }
            atomicAdd(gw + e, acc);
        } else {
            const int o = e - NW;
            for (long long p = p0; p < p1; p++) {
                const int img = (int)(p / plane);
                const int rem = (int)(p - (long long)img * plane);
                acc += g[((long long)img * COUT + o) * plane + rem];
            }
            atomicAdd(gb + o, acc);
        }
    }
}

// gradient with respect to the layer input, times ReLU' of that input:
// ga[n,c,i,j] = relu'(a) * sum_o sum_taps w[o,c,di,dj] g[n,o,i-di+1,j-dj+1]
template <int CIN, int COUT, int K>
__global__ void conv_dgrad_kernel(const float *__restrict__ g, const float *__restrict__ theta, int off_w,
                                  const float *__restrict__ a, int n, int H, int W, float *ga)
{
    __shared__ float sw[COUT * CIN * K * K];
    for (int k = threadIdx.x; k < COUT * CIN * K * K; k += blockDim.x) sw[k] = theta[off_w + k];
    __syncthreads();
    const long long plane = (long long)H * W;
    const long long total = (long long)n * plane;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total; p += (long long)gridDim.x * blockDim.x) {
        const int img = (int)(p / plane);
        const int rem = (int)(p - (long long)img * plane);
        const int i = rem / W, j = rem % W;
        float acc[CIN];
#pragma unroll
        for (int c = 0; c < CIN; c++) acc[c] = 0.0f;
        for (int o = 0; o < COUT; o++) {
#pragma unroll
            for (int di = 0; di < K; di++) {
                const int ii = i - di + K / 2;
                if (ii < 0 || ii >= H) continue;
#pragma unroll
                for (int dj = 0; dj < K; dj++) {
                    const int jj = j - dj + K / 2;
                    if (jj < 0 || jj >= W) continue;
                    const float gv = g[((long long)img * COUT + o) * plane + (long long)ii * W + jj];
#pragma unroll
                    for (int c = 0; c < CIN; c++) acc[c] = fmaf(sw[((o * CIN + c) * K + di) * K + dj], gv, acc[c]);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < CIN; c++) {
            const long long q = ((long long)img * CIN + c) * plane + rem;
            ga[q] = a[q] > 0.0f ? acc[c] : 0.0f;
        }
    }
}

__global__ void adam_kernel(float *theta, const float *grad, float *m, float *v, int np, float lr, float b1, float b2,
                            float eps, float c1, float c2)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
        float gk = grad[k];
        float mk = b1 * m[k] + (1.0f - b1) * gk;
        float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        theta[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    }
}

__global__ void to_half_kernel(const float *x, __half *y, long long n)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
        y[p] = __float2half_rn(x[p]);
}

int blocks_for(long long n, int threads)
{
    long long b = (n + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

int cnn_n_params()
{
    LayerSpec s = layer_spec(3);
    return s.boff + s.cout;
}

size_t cnn_workspace_floats(int n, int H, int W)
{
    const size_t px = (size_t)n * H * W;
    return px * (size_t)(3 * HID + 1) /* activations a1..a3, logits */ + px * (size_t)(2 * HID) /* two grad planes */ +
           px /* head grad */;
}

int cnn_forward(const float *theta, const float *x, int n, int H, int W, bool fp16, float *act, float *logits,
                void *half_ws, cudaStream_t st)
{
    const long long px = (long long)n * H * W;
    const int th = 128, bl = blocks_for(px, th);
    float *a1 = act, *a2 = act + px * HID, *a3 = act + 2 * px * HID;
    LayerSpec L0 = layer_spec(0), L1 = layer_spec(1), L2 = layer_spec(2), L3 = layer_spec(3);
    if (!fp16) {
        conv_fwd_kernel<float, float, kCnnIn, HID, 3, true><<<bl, th, 0, st>>>(x, theta, L0.woff, L0.boff, a1, n, H, W, false);
        conv_fwd_kernel<float, float, HID, HID, 3, true><<<bl, th, 0, st>>>(a1, theta, L1.woff, L1.boff, a2, n, H, W, false);
        conv_fwd_kernel<float, float, HID, HID, 3, true><<<bl, th, 0, st>>>(a2, theta, L2.woff, L2.boff, a3, n, H, W, false);
        conv_fwd_kernel<float, float, HID, 1, 1, false><<<bl, th, 0, st>>>(a3, theta, L3.woff, L3.boff, logits, n, H, W, false);
    } else {
        // FP16 activations and weights, FP32 accumulation
        __half *hx = reinterpret_cast<__half *>(half_ws);
        __half *h1 = hx + px * kCnnIn, *h2 = h1 + px * HID, *h3 = h2 + px * HID;
        to_half_kernel<<<blocks_for(px * kCnnIn, 256), 256, 0, st>>>(x, hx, px * kCnnIn);
        conv_fwd_kernel<__half, __half, kCnnIn, HID, 3, true><<<bl, th, 0, st>>>(hx, theta, L0.woff, L0.boff, h1, n, H, W, true);
        conv_fwd_kernel<__half, __half, HID, HID, 3, true><<<bl, th, 0, st>>>(h1, theta, L1.woff, L1.boff, h2, n, H, W, true);
        conv_fwd_kernel<__half, __half, HID, HID, 3, true><<<bl, th, 0, st>>>(h2, theta, L2.woff, L2.boff, h3, n, H, W, true);
        conv_fwd_kernel<__half, float, HID, 1, 1, false><<<bl, th, 0, st>>>(h3, theta, L3.woff, L3.boff, logits, n, H, W, true);
    }
    return (int)cudaGetLastError();
}

size_t cnn_half_workspace_bytes(int n, int H, int W)
{
    return (size_t)n * H * W * (kCnnIn + 3 * HID) * sizeof(__half);
}

int cnn_loss_grad(const float *theta, const float *x, const float *t, const float *m, int n, int H, int W, float mcount,
                  float *ws, float *grad, double *loss, cudaStream_t st)
{
    const long long px = (long long)n * H * W;
    float *act = ws, *logits = ws + px * 3 * HID;
    float *ga = logits + px, *gb = ga + px * HID, *gz = gb + px * HID;
    int e = cnn_forward(theta, x, n, H, W, false, act, logits, nullptr, st);
    if (e) return e;
    const int th = 128, bl = blocks_for(px, th);
    float *a1 = act, *a2 = act + px * HID, *a3 = act + 2 * px * HID;
    LayerSpec L0 = layer_spec(0), L1 = layer_spec(1), L2 = layer_spec(2), L3 = layer_spec(3);
    cudaMemsetAsync(grad, 0, cnn_n_params() * sizeof(float), st);
    cudaMemsetAsync(loss, 0, sizeof(double), st);
    bce_grad_kernel<<<bl, th, 0, st>>>(logits, t, m, px, mcount > 0 ? 1.0f / mcount : 0.0f, gz, loss);
    const int ppb = 1024;
    const int wb = (int)((px + ppb - 1) / ppb);
    // head (1x1, 16 -> 1)
    conv_wgrad_kernel<HID, 1, 1><<<wb, 128, 0, st>>>(gz, a3, n, H, W, grad + L3.woff, grad + L3.boff, ppb);
    conv_dgrad_kernel<HID, 1, 1><<<bl, th, 0, st>>>(gz, theta, L3.woff, a3, n, H, W, ga);
    // layer 3 (3x3, 16 -> 16): input a2
    conv_wgrad_kernel<HID, HID, 3><<<wb, 256, 0, st>>>(ga, a2, n, H, W, grad + L2.woff, grad + L2.boff, ppb);
    conv_dgrad_kernel<HID, HID, 3><<<bl, th, 0, st>>>(ga, theta, L2.woff, a2, n, H, W, gb);
    // layer 2: input a1
    conv_wgrad_kernel<HID, HID, 3><<<wb, 256, 0, st>>>(gb, a1, n, H, W, grad + L1.woff, grad + L1.boff, ppb);
    conv_dgrad_kernel<HID, HID, 3><<<bl, th, 0, st>>>(gb, theta, L1.woff, a1, n, H, W, ga);
    // layer 1: input x (no ReLU before it, no input gradient needed)
    conv_wgrad_kernel<kCnnIn, HID, 3><<<wb, 256, 0, st>>>(ga, x, n, H, W, grad + L0.woff, grad + L0.boff, ppb);
    return (int)cudaGetLastError();
}

int cnn_adam(float *theta, const float *grad, float *m, float *v, int np, float lr, int t, cudaStream_t st)
{
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    adam_kernel<<<blocks_for(np, 256), 256, 0, st>>>(theta, grad, m, v, np, lr, b1, b2, 1e-8f, c1, c2);
    return (int)cudaGetLastError();
}

}  // namespace tsu
