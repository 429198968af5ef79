// Learned warm start of the fine-level subspace iteration (not part of the
// paper's method; the paper starts ARPACK without a learned guess).  A small
// MLP maps a subdomain's log10-kappa patch to NN_NVEC vectors on an
// NN_GRID x NN_GRID node grid over its Neumann box; they are interpolated to
// the box's nodes and used as the first start columns of Eq. theGEVP's
// subspace iteration.  Layer sizes, parameter packing and the loss are given
// in include/msdd.h (msdd_nn_*).
#pragma once
#include "common.cuh"
#include "q1.cuh"

namespace msdd {

constexpr int NN_PATCH = 24, NN_IN = NN_PATCH * NN_PATCH, NN_H = 48, NN_GRID = 13, NN_G2 = NN_GRID * NN_GRID,
              NN_NVEC = 12, NN_OUT = NN_NVEC * NN_G2;
constexpr long long NN_W1 = 0, NN_B1 = NN_W1 + (long long)NN_H * NN_IN, NN_W2 = NN_B1 + NN_H,
                    NN_B2 = NN_W2 + (long long)NN_H * NN_H, NN_W3 = NN_B2 + NN_H,
                    NN_B3 = NN_W3 + (long long)NN_OUT * NN_H, NN_NPARAM = NN_B3 + NN_OUT;

// workspace floats for a batch of S samples
size_t nn_workspace_floats(int S);
// log10-kappa patches of the given boxes (scalar 2D coefficient), P x NN_IN
void nn_patches(const Geom& g, const ProbBox* d_boxes, int P, float* X, cudaStream_t s);
// out = net(params, X) (S x NN_OUT); work: nn_workspace_floats(S) floats
void nn_forward(const float* params, int S, const float* X, float* out, float* work, cudaStream_t s);
// mean loss over the batch (device double) and the parameter gradient (device float)
void nn_loss_grad(const float* params, int S, const float* X, const float* T, const int* m, double* loss,
                  float* grad, float* work, cudaStream_t s);
void nn_adam(float* params, const float* grad, float* m1, float* m2, int t, float lr, cudaStream_t s);
// grid vectors Y (P x NN_OUT) -> node values on each box (row offsets off[i]), rows x NN_NVEC doubles
void nn_start_vectors(const ProbBox* d_boxes, const long long* d_off, int P, int dim, const float* Y, double* out,
                      cudaStream_t s);
// training targets from eigenvectors X (rows roff[i], leading dim ldx, first m[i] columns) of the boxes
void nn_targets(const ProbBox* d_boxes, const long long* d_roff, const int* d_m, int P, int dim, const double* X,
                int ldx, float* T, int* mout, cudaStream_t s);

}  // namespace msdd
