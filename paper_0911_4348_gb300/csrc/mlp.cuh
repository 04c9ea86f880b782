// Warm-start network kernels (mlp.cu): layout and launchers.
#pragma once

#include "common.cuh"

namespace fedvr {

// Parameter layout of the per-pair network: W1 [din][H], b1 [H], W2 [H][H],
// b2 [H], W3 [H][dout], b3 [dout]; din = 2M+3, dout = M.
struct MlpNet {
  int din = 0, H = 0, dout = 0;
  long o_W1 = 0, o_b1 = 0, o_W2 = 0, o_b2 = 0, o_W3 = 0, o_b3 = 0, nparam = 0;
};

MlpNet mlp_layout(int M, int H);
// act: 4 * rows * H floats (Z1, H1, Z2, H2); Y: rows * dout.
cudaError_t mlp_forward_f32(const MlpNet &L, const float *W, int rows, const float *X, float *act,
                            float *Y, cudaStream_t s);
cudaError_t mlp_forward_bf16(const MlpNet &L, const void *Wbf, const float *W, int rows,
                             const float *X, float *act, float *Y, cudaStream_t s);
// dbuf: 2 * rows * max(H, dout) floats; part: 256 doubles of loss partials.
cudaError_t mlp_loss_grad(const MlpNet &L, const float *W, int rows, const float *X,
                          const float *T, float *act, float *Y, float *dbuf, float *grad,
                          double *part, cudaStream_t s);
cudaError_t mlp_adam(long count, float lr, int t, const float *g, float *m, float *v, float *w,
                     cudaStream_t s);
cudaError_t mlp_to_bf16(long count, const float *w, void *wbf, cudaStream_t s);
cudaError_t mlp_gather(int rows, int cols, const int *idx, const float *src, float *dst,
                       cudaStream_t s);
// Features (and targets if Sstar != NULL) of every pair a >= b; s_dev receives
// s = max|S1|.
cudaError_t mlp_features(int n, int M, double L, const double *S1, const double *G0,
                         const double *V, const double *X, double *s_dev, const double *Sstar,
                         float *F, float *T, cudaStream_t s);
cudaError_t mlp_scatter(int n, int M, const double *S1, const double *s_dev, const float *Y,
                        double *out, cudaStream_t s);

}  // namespace fedvr
