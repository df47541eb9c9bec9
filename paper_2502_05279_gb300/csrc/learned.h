// Learned interpolation: network shape and launchers (k_learned.cu).
#pragma once

#include <cuda_runtime.h>

namespace bmg {

constexpr int MLP_IN = 18, MLP_HID = 64, MLP_OUT = 4;
constexpr int MLP_PARAMS = MLP_IN * MLP_HID + MLP_HID + MLP_HID * MLP_HID + MLP_HID + MLP_HID * MLP_OUT + MLP_OUT;

void launch_features(int n, const double* st, float* X, cudaStream_t s);
void launch_mlp_infer(const float* X, int M, const float* par, float* out, cudaStream_t s);
void launch_learned_ci(int n, const double* st, const float* delta, double* ci, double* aux, cudaStream_t s);
void launch_uniform_pm1(int n, unsigned long long seed, double* x, cudaStream_t s);
void launch_tv_energies(int n, const double* st, const double* ci, int K, const double* vecs, double* errs,
                        double* Aes, double* partials, double* energies, cudaStream_t s);
void launch_tv_grad(int n, const double* st, int K, const double* vecs, const double* Aes, const double* scale,
                    const double* aux, double* dW, double* tx, double* ty, float* ddelta, cudaStream_t s);
void launch_mlp_fwd(const float* X, int M, const float* par, float* Z1, float* Z2, float* out, cudaStream_t s);
void launch_mlp_bwd(const float* X, int M, const float* par, const float* Z1, const float* Z2, const float* dout,
                    float* partial, float* grad, cudaStream_t s);
void launch_adam(float* par, const float* grad, float* m, float* v, float lr, int step, cudaStream_t s);
int mlp_backward_blocks(int M);
// Two-grid training loss on crops (k_twogrid.cu): n = 7, 15 or 31.
bool twogrid_size_ok(int n);
int launch_twogrid(int n, int ncrop, int K, const double* coefs, const double* vecs, const float* delta,
                   const double* eref, double weight, double* energies, float* ddelta, int* err, cudaStream_t s);
void launch_features_crops(int n, int ncrop, const double* coefs, float* X, cudaStream_t s);

}  // namespace bmg
