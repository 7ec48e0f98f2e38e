// cnn_api.cpp -- C ABI of the refinement-flag predictor's kernels (forward,
// loss gradient, training) on host buffers.  The network and its use inside
// regridding are described in include/tsunami.h.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <random>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/tsunami.h"
#include "cnn.h"

using namespace tsu;

namespace {

struct Buf {
    void *p = nullptr;
    ~Buf() { if (p) cudaFree(p); }
    cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, bytes < 16 ? 16 : bytes); }
    template <typename T> T *as() { return reinterpret_cast<T *>(p); }
};

#define CKR(x) do { if ((x) != cudaSuccess) return TSU_ERR_CUDA; } while (0)

}  // namespace

extern "C" int tsu_cnn_num_params(void) { return cnn_n_params(); }

extern "C" int tsu_cnn_forward(const float *theta, const float *x, int n, int h, int w, int fp16, float *logits)
{
    if (!theta || !x || !logits || n < 1 || h < 1 || w < 1) return TSU_ERR_ARG;
    const size_t px = (size_t)n * h * w;
    const int np = cnn_n_params();
    Buf dth, dx, dact, dlog, dhalf;
    CKR(dth.alloc(np * sizeof(float)));
    CKR(dx.alloc(px * kCnnIn * sizeof(float)));
    CKR(dact.alloc(px * 3 * kCnnHidden * sizeof(float)));
    CKR(dlog.alloc(px * sizeof(float)));
    CKR(dhalf.alloc(cnn_half_workspace_bytes(n, h, w)));
    CKR(cudaMemcpy(dth.p, theta, np * sizeof(float), cudaMemcpyHostToDevice));
    CKR(cudaMemcpy(dx.p, x, px * kCnnIn * sizeof(float), cudaMemcpyHostToDevice));
    if (cnn_forward(dth.as<float>(), dx.as<float>(), n, h, w, fp16 != 0, dact.as<float>(), dlog.as<float>(), dhalf.p, 0))
        return TSU_ERR_CUDA;
    CKR(cudaMemcpy(logits, dlog.p, px * sizeof(float), cudaMemcpyDeviceToHost));
    return TSU_OK;
}

extern "C" int tsu_cnn_loss_grad(const float *theta, const float *x, const float *t, const float *m, int n, int h,
                                 int w, double *loss, float *grad)
{
    if (!theta || !x || !t || !m || !loss || !grad || n < 1 || h < 1 || w < 1) return TSU_ERR_ARG;
    const size_t px = (size_t)n * h * w;
    const int np = cnn_n_params();
    double cnt = 0.0;
    for (size_t k = 0; k < px; k++) cnt += m[k];
    Buf dth, dx, dt, dm, dws, dg, dl;
    CKR(dth.alloc(np * sizeof(float)));
    CKR(dx.alloc(px * kCnnIn * sizeof(float)));
    CKR(dt.alloc(px * sizeof(float)));
    CKR(dm.alloc(px * sizeof(float)));
    CKR(dws.alloc(cnn_workspace_floats(n, h, w) * sizeof(float)));
    CKR(dg.alloc(np * sizeof(float)));
    CKR(dl.alloc(sizeof(double)));
    CKR(cudaMemcpy(dth.p, theta, np * sizeof(float), cudaMemcpyHostToDevice));
    CKR(cudaMemcpy(dx.p, x, px * kCnnIn * sizeof(float), cudaMemcpyHostToDevice));
    CKR(cudaMemcpy(dt.p, t, px * sizeof(float), cudaMemcpyHostToDevice));
    CKR(cudaMemcpy(dm.p, m, px * sizeof(float), cudaMemcpyHostToDevice));
    if (cnn_loss_grad(dth.as<float>(), dx.as<float>(), dt.as<float>(), dm.as<float>(), n, h, w, (float)cnt,
                      dws.as<float>(), dg.as<float>(), dl.as<double>(), 0))
        return TSU_ERR_CUDA;
    CKR(cudaMemcpy(grad, dg.p, np * sizeof(float), cudaMemcpyDeviceToHost));
    CKR(cudaMemcpy(loss, dl.p, sizeof(double), cudaMemcpyDeviceToHost));
    return TSU_OK;
}

// Mini-batch Adam on the GPU over a host dataset of n planes; batches of
// `batch` planes drawn with a Mersenne twister seeded by `seed`.
extern "C" int tsu_cnn_train(float *theta, const float *x, const float *t, const float *m, int n, int h, int w,
                             int steps, int batch, float lr, unsigned seed, double *loss_first, double *loss_last)
{
    if (!theta || !x || !t || !m || n < 1 || h < 1 || w < 1 || steps < 1 || batch < 1 || !(lr > 0)) return TSU_ERR_ARG;
    if (batch > n) batch = n;
    const size_t plane = (size_t)h * w;
    const int np = cnn_n_params();
    Buf dth, dx, dt, dm, dws, dg, dl, dmo, dv, bx, bt, bm;
    CKR(dth.alloc(np * sizeof(float)));
    CKR(dx.alloc((size_t)n * plane * kCnnIn * sizeof(float)));
    CKR(dt.alloc((size_t)n * plane * sizeof(float)));
    CKR(dm.alloc((size_t)n * plane * sizeof(float)));
    CKR(dws.alloc(cnn_workspace_floats(batch, h, w) * sizeof(float)));
    CKR(dg.alloc(np * sizeof(float)));
    CKR(dl.alloc(sizeof(double)));
    CKR(dmo.alloc(np * sizeof(float)));
    CKR(dv.alloc(np * sizeof(float)));
    CKR(bx.alloc((size_t)batch * plane * kCnnIn * sizeof(float)));
    CKR(bt.alloc((size_t)batch * plane * sizeof(float)));
    CKR(bm.alloc((size_t)batch * plane * sizeof(float)));
    CKR(cudaMemcpy(dth.p, theta, np * sizeof(float), cudaMemcpyHostToDevice));
    CKR(cudaMemcpy(dx.p, x, (size_t)n * plane * kCnnIn * sizeof(float), cudaMemcpyHostToDevice));
    CKR(cudaMemcpy(dt.p, t, (size_t)n * plane * sizeof(float), cudaMemcpyHostToDevice));
    CKR(cudaMemcpy(dm.p, m, (size_t)n * plane * sizeof(float), cudaMemcpyHostToDevice));
    CKR(cudaMemset(dmo.p, 0, np * sizeof(float)));
    CKR(cudaMemset(dv.p, 0, np * sizeof(float)));
    std::vector<double> cnt(n, 0.0);
    for (int k = 0; k < n; k++)
        for (size_t q = 0; q < plane; q++) cnt[k] += m[(size_t)k * plane + q];
    std::mt19937 rng(seed);
    std::vector<int> order(n);
    for (int k = 0; k < n; k++) order[k] = k;
    size_t pos = n;
    for (int s = 1; s <= steps; s++) {
        double bc = 0.0;
        for (int b = 0; b < batch; b++) {
            if (pos >= (size_t)n) { std::shuffle(order.begin(), order.end(), rng); pos = 0; }
            int k = order[pos++];
            bc += cnt[k];
            CKR(cudaMemcpyAsync(bx.as<float>() + (size_t)b * plane * kCnnIn, dx.as<float>() + (size_t)k * plane * kCnnIn,
                                plane * kCnnIn * sizeof(float), cudaMemcpyDeviceToDevice, 0));
            CKR(cudaMemcpyAsync(bt.as<float>() + (size_t)b * plane, dt.as<float>() + (size_t)k * plane,
                                plane * sizeof(float), cudaMemcpyDeviceToDevice, 0));
            CKR(cudaMemcpyAsync(bm.as<float>() + (size_t)b * plane, dm.as<float>() + (size_t)k * plane,
                                plane * sizeof(float), cudaMemcpyDeviceToDevice, 0));
        }
        if (cnn_loss_grad(dth.as<float>(), bx.as<float>(), bt.as<float>(), bm.as<float>(), batch, h, w, (float)bc,
                          dws.as<float>(), dg.as<float>(), dl.as<double>(), 0))
            return TSU_ERR_CUDA;
        if (s == 1 && loss_first) CKR(cudaMemcpy(loss_first, dl.p, sizeof(double), cudaMemcpyDeviceToHost));
        if (cnn_adam(dth.as<float>(), dg.as<float>(), dmo.as<float>(), dv.as<float>(), np, lr, s, 0)) return TSU_ERR_CUDA;
        if (s == steps && loss_last) CKR(cudaMemcpy(loss_last, dl.p, sizeof(double), cudaMemcpyDeviceToHost));
    }
    CKR(cudaMemcpy(theta, dth.p, np * sizeof(float), cudaMemcpyDeviceToHost));
    return TSU_OK;
}
