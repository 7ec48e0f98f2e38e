// cnn.cu -- the per-patch refinement-flag predictor: a learned stand-in for
// the b-cell flag buffer of Sec. 3.2 (regridding).  Three 3x3 convolutions of
// 16 channels with ReLU and a 1x1 head to one logit per cell, over the dense
// planes of a level (5 input features per cell), zero padding at the plane
// edge.  Forward in FP32 (training) or, for inference, one fused kernel on
// the tensor cores with FP16 activations and weights and FP32 accumulation;
// hand-written backward (binary cross-entropy
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


int blocks_for(long long n, int threads)
{
    long long b = (n + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

// ---------------------------------------------------------------- inference on tensor cores
// The FP16 inference path fused into one kernel.  A CTA produces the logits
// of a TH x TW tile of one plane; the tile's inputs and the two hidden
// activations it needs (the tile grown by 2 and by 1 cells) live in shared
// memory as FP16, channels last (24-half pixel stride: ldmatrix rows of 16
// bytes fall on distinct banks).  Each 3x3 layer is an implicit GEMM on the
// warp-level tensor-core MMA (m16n8k16, FP16 inputs, FP32 accumulation): an
// M-block is 16 consecutive pixels of the output region, K runs over the 9
// taps x 16 channels (the 5 input features padded with zeros), N = 16
// channels in two 8-wide blocks.  Activations outside the plane are zero, as
// zero padding of every layer's input requires.  The 1x1 head is a shuffle
// reduction of the last layer's accumulators.

namespace tc {
constexpr int TH = 16, TW = 32;            // output tile
constexpr int PS = 24;                     // halves per pixel in shared memory
constexpr int H0 = TH + 6, W0 = TW + 6;    // input region (3-cell margin)
constexpr int H1 = TH + 4, W1 = TW + 4;    // first hidden layer
constexpr int H2 = TH + 2, W2 = TW + 2;    // second hidden layer
constexpr int N0 = H0 * W0, N1 = H1 * W1, N2 = H2 * W2;
constexpr int NWARP = 4;
// per layer: 9 taps x 2 n-blocks x 32 lanes x 2 registers of packed FP16 weights
constexpr int WFRAG = 9 * 2 * 32 * 2;
constexpr size_t smem_bytes()
{
    return (size_t)(N0 > N2 ? N0 : N2) * PS * 2 + (size_t)N1 * PS * 2 + 3 * WFRAG * 4 + 3 * 16 * 4 + 16 * 4 + 16;
}
}  // namespace tc

__device__ __forceinline__ uint32_t pack_half2(float lo, float hi)
{
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

// One 3x3 layer over an output region of ho x wo pixels (top-left at plane
// row gy, column gx) from an input region of (ho+2) x (wo+2) pixels.  LAST:
// apply the head and write logits instead of storing activations.
template <bool LAST>
__device__ __forceinline__ void tc_layer(const __half *in, int wi, __half *out, int ho, int wo, int gy, int gx, int H,
                                         int W, const uint32_t *wf, const float *bias, const float *whead, float bhead,
                                         float *logits)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const int npx = ho * wo, nblk = (npx + 15) / 16;
    const uint32_t in_s = (uint32_t)__cvta_generic_to_shared(in);
    // ldmatrix row of this lane: matrix m = lane / 8 -> pixel rows 0-7 / 8-15, channel half 0 / 1
    const int m = lane >> 3, prow = (m & 1) * 8 + (lane & 7), chalf = (m >> 1) * 8;
    for (int blk = warp; blk < nblk; blk += tc::NWARP) {
        int p = blk * 16 + prow;
        p = p < npx ? p : npx - 1;
        const int r = p / wo, c = p - r * wo;
        float acc[2][4];
#pragma unroll
        for (int nb = 0; nb < 2; nb++) {
            const float b0 = bias[nb * 8 + 2 * t4], b1 = bias[nb * 8 + 2 * t4 + 1];
            acc[nb][0] = b0; acc[nb][1] = b1; acc[nb][2] = b0; acc[nb][3] = b1;
        }
#pragma unroll
        for (int tap = 0; tap < 9; tap++) {
            const int di = tap / 3, dj = tap % 3;
            const uint32_t addr = in_s + (uint32_t)(((r + di) * wi + (c + dj)) * tc::PS + chalf) * 2u;
            uint32_t a0, a1, a2, a3;
            ldsm_x4(addr, a0, a1, a2, a3);
#pragma unroll
            for (int nb = 0; nb < 2; nb++) {
                const uint32_t *f = wf + ((tap * 2 + nb) * 32 + lane) * 2;
                mma16816(acc[nb], a0, a1, a2, a3, f[0], f[1]);
            }
        }
        // rows g and g+8 of the block, channels nb*8 + 2*t4, +1
#pragma unroll
        for (int half = 0; half < 2; half++) {
            const int pp = blk * 16 + g + half * 8;
            if (pp >= npx) continue;
            const int rr = pp / wo, cc = pp - rr * wo;
            const int yy = gy + rr, xx = gx + cc;
            const bool inside = yy >= 0 && yy < H && xx >= 0 && xx < W;
            if (!LAST) {
#pragma unroll
                for (int nb = 0; nb < 2; nb++) {
                    const float v0 = inside ? fmaxf(acc[nb][2 * half], 0.0f) : 0.0f;
                    const float v1 = inside ? fmaxf(acc[nb][2 * half + 1], 0.0f) : 0.0f;
                    *reinterpret_cast<uint32_t *>(out + pp * tc::PS + nb * 8 + 2 * t4) = pack_half2(v0, v1);
                }
            }
        }
        if (LAST) {
            // head: activations rounded to FP16 as stored activations are, FP32 dot product
            float part[2] = {0.0f, 0.0f};
#pragma unroll
            for (int half = 0; half < 2; half++)
#pragma unroll
                for (int nb = 0; nb < 2; nb++)
#pragma unroll
                    for (int e = 0; e < 2; e++) {
                        const float v = __half2float(__float2half_rn(fmaxf(acc[nb][2 * half + e], 0.0f)));
                        part[half] = fmaf(whead[nb * 8 + 2 * t4 + e], v, part[half]);
                    }
#pragma unroll
            for (int half = 0; half < 2; half++) {
                part[half] += __shfl_xor_sync(0xffffffffu, part[half], 1);
                part[half] += __shfl_xor_sync(0xffffffffu, part[half], 2);
            }
            if (t4 == 0) {
#pragma unroll
                for (int half = 0; half < 2; half++) {
                    const int pp = blk * 16 + g + half * 8;
                    if (pp >= npx) continue;
                    const int rr = pp / wo, cc = pp - rr * wo;
                    const int yy = gy + rr, xx = gx + cc;
                    if (yy < H && xx < W) logits[(long long)yy * W + xx] = part[half] + bhead;
                }
            }
        }
    }
}

__global__ void __launch_bounds__(tc::NWARP * 32) cnn_infer_tc_kernel(const float *__restrict__ theta,
                                                                      const float *__restrict__ x, int H, int W,
                                                                      float *__restrict__ logits)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __half *s0 = reinterpret_cast<__half *>(smem);                               // inputs, then layer 2
    __half *s1 = s0 + (size_t)(tc::N0 > tc::N2 ? tc::N0 : tc::N2) * tc::PS;      // layer 1
    uint32_t *wf = reinterpret_cast<uint32_t *>(s1 + (size_t)tc::N1 * tc::PS);    // weight fragments, 3 layers
    float *bias = reinterpret_cast<float *>(wf + 3 * tc::WFRAG);                 // 3 x 16
    float *whead = bias + 48;                                                     // 16, then its bias
    const int img = blockIdx.z;
    const int ty0 = blockIdx.y * tc::TH, tx0 = blockIdx.x * tc::TW;
    const long long plane = (long long)H * W;
    const float *xi = x + (long long)img * kCnnIn * plane;
    // weight fragments: b0 = (W[o][2t][tap], W[o][2t+1][tap]), b1 = channels 2t+8, 2t+9; o = nb*8 + lane/4
    for (int e = threadIdx.x; e < 3 * 9 * 2 * 32; e += blockDim.x) {
        const int l = e / (9 * 2 * 32), rem = e % (9 * 2 * 32);
        const int tap = rem / 64, nb = (rem / 32) % 2, ln = rem % 32;
        const LayerSpec S = layer_spec(l);
        const int o = nb * 8 + ln / 4, k0 = 2 * (ln % 4);
        float w[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int cch = k0 + (q & 1) + (q >> 1) * 8;
            w[q] = cch < S.cin ? theta[S.woff + (o * S.cin + cch) * 9 + tap] : 0.0f;
        }
        uint32_t *f = wf + l * tc::WFRAG + ((tap * 2 + nb) * 32 + ln) * 2;
        f[0] = pack_half2(w[0], w[1]);
        f[1] = pack_half2(w[2], w[3]);
    }
    for (int e = threadIdx.x; e < 48; e += blockDim.x) bias[e] = theta[layer_spec(e / 16).boff + e % 16];
    if (threadIdx.x < 16) {
        const LayerSpec S = layer_spec(3);
        whead[threadIdx.x] = __half2float(__float2half_rn(theta[S.woff + threadIdx.x]));
        if (threadIdx.x == 0) whead[16] = theta[S.boff];
    }
    // inputs of the 3-cell grown tile, FP16, zero outside the plane and in channels 5..15
    for (int e = threadIdx.x; e < tc::N0 * 16; e += blockDim.x) {
        const int p = e / 16, ch = e % 16;
        const int r = p / tc::W0, c = p - r * tc::W0;
        const int yy = ty0 - 3 + r, xx = tx0 - 3 + c;
        float v = 0.0f;
        if (ch < kCnnIn && yy >= 0 && yy < H && xx >= 0 && xx < W) v = xi[(long long)ch * plane + (long long)yy * W + xx];
        s0[p * tc::PS + ch] = __float2half_rn(v);
    }
    __syncthreads();
    tc_layer<false>(s0, tc::W0, s1, tc::H1, tc::W1, ty0 - 2, tx0 - 2, H, W, wf, bias, nullptr, 0.0f, nullptr);
    __syncthreads();
    tc_layer<false>(s1, tc::W1, s0, tc::H2, tc::W2, ty0 - 1, tx0 - 1, H, W, wf + tc::WFRAG, bias + 16, nullptr, 0.0f,
                    nullptr);
    __syncthreads();
    tc_layer<true>(s0, tc::W2, nullptr, tc::TH, tc::TW, ty0, tx0, H, W, wf + 2 * tc::WFRAG, bias + 32, whead,
                   whead[16], logits + (long long)img * plane);
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
        // FP16 activations and weights, FP32 accumulation: one fused tensor-core kernel
        (void)half_ws;
        static bool configured = false;
        const size_t sm = tc::smem_bytes();
        if (!configured) {
            cudaError_t e = cudaFuncSetAttribute(cnn_infer_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return (int)e;
            configured = true;
        }
        dim3 grid((W + tc::TW - 1) / tc::TW, (H + tc::TH - 1) / tc::TH, n);
        cnn_infer_tc_kernel<<<grid, tc::NWARP * 32, sm, st>>>(theta, x, H, W, logits);
    }
    return (int)cudaGetLastError();
}

size_t cnn_half_workspace_bytes(int, int, int)
{
    return 16;   // the fused inference kernel keeps its activations in shared memory
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
