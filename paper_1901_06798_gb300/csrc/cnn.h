// cnn.h -- device side of the refinement-flag predictor (see cnn.cu).
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

namespace tsu {

constexpr int kCnnIn = 5;       // input features per cell
constexpr int kCnnHidden = 16;  // channels of the three 3x3 layers

int cnn_n_params();
// FP32 activations + gradient planes needed by cnn_loss_grad for n planes of H x W
size_t cnn_workspace_floats(int n, int H, int W);
// workspace bytes of the inference path (its activations stay in shared memory)
size_t cnn_half_workspace_bytes(int n, int H, int W);
// logits (n, H, W) of inputs x (n, 5, H, W); act: >= 3*16*n*H*W floats (FP32 path)
int cnn_forward(const float *theta, const float *x, int n, int H, int W, bool fp16, float *act, float *logits,
                void *half_ws, cudaStream_t st);
// mean binary cross-entropy over mask (count mcount) and its gradient (flat, cnn_n_params floats)
int cnn_loss_grad(const float *theta, const float *x, const float *t, const float *m, int n, int H, int W, float mcount,
                  float *ws, float *grad, double *loss, cudaStream_t st);
int cnn_adam(float *theta, const float *grad, float *m, float *v, int np, float lr, int t, cudaStream_t st);

}  // namespace tsu
