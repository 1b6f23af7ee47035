// mlp.h - launchers of the cost-model kernels (mlp.cu).
#pragma once

#include <cuda_runtime.h>

#define JACC_MLP_NPARAM 8705

namespace jacc {
size_t mlp_smem_bytes();
cudaError_t mlp_setup();
int mlp_nparts(int n);
cudaError_t mlp_fwd_bwd(const float* P, const float* X, const float* Y, int n, float* partial, float* loss_partial,
                        unsigned* step, cudaStream_t s);
cudaError_t mlp_adam(float* P, float* M, float* V, const float* partial, int nparts, const float* loss_partial, int n,
                     float* loss_out, const unsigned* step, float lr, float b1, float b2, float eps, float* grad_out,
                     cudaStream_t s);
cudaError_t mlp_forward(const float* P, const float* X, int n, float* Y, cudaStream_t s);
cudaError_t mlp_pick(const float* pred, const int* valid, int nq, int ntile, int* pick, float* gap, cudaStream_t s);
}  // namespace jacc
