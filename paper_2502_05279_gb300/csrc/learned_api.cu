// C ABI of the learned interpolation: network parameters and optimiser state
// on the device, one loss/gradient evaluation per training problem, Adam,
// tensor-core inference and the learned weights.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "learned.h"

using namespace bmg;

struct bmg_mlp {
  float* par = nullptr;
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  int step = 0;
  // training workspace, sized for the largest problem seen
  int cap_n = 0, cap_k = 0;
  float *X = nullptr, *Z1 = nullptr, *Z2 = nullptr, *out = nullptr, *dout = nullptr, *partial = nullptr;
  float* zero_delta = nullptr;
  double *ci = nullptr, *aux = nullptr, *errs = nullptr, *Aes = nullptr, *dW = nullptr, *tx = nullptr, *ty = nullptr;
  double *partials = nullptr, *energies = nullptr, *scale = nullptr;
  // two-grid training workspace (rows = crops x coarse points)
  size_t tg_rows = 0;
  float *tg_X = nullptr, *tg_Z1 = nullptr, *tg_Z2 = nullptr, *tg_out = nullptr, *tg_dout = nullptr,
        *tg_partial = nullptr;
  int* tg_err = nullptr;
};

#define CK(call)                               \
  do {                                         \
    int _rc = cuda_check((call), #call);       \
    if (_rc != BMG_OK) return _rc;             \
  } while (0)

namespace {

void free_ws(bmg_mlp* m) {
  void* ptrs[] = {m->X, m->Z1, m->Z2, m->out, m->dout, m->partial, m->zero_delta, m->ci, m->aux, m->errs,
                  m->Aes, m->dW, m->tx, m->ty, m->partials, m->energies, m->scale};
  for (void* p : ptrs) cudaFree(p);
  m->X = m->Z1 = m->Z2 = m->out = m->dout = m->partial = m->zero_delta = nullptr;
  m->ci = m->aux = m->errs = m->Aes = m->dW = m->tx = m->ty = m->partials = m->energies = m->scale = nullptr;
  m->cap_n = m->cap_k = 0;
}

template <typename T>
int alloc0(T** p, size_t count) {
  CK(dev_malloc((void**)p, count * sizeof(T)));
  CK(cudaMemset(*p, 0, count * sizeof(T)));
  return BMG_OK;
}

int ensure_ws(bmg_mlp* m, int n, int K) {
  if (n <= m->cap_n && K <= m->cap_k) return BMG_OK;
  free_ws(m);
  int nc = (n - 1) / 2;
  size_t M = (size_t)nc * nc, ps = plane_size(n), psc = plane_size(nc);
  int rc;
  if ((rc = alloc0(&m->X, M * MLP_IN)) || (rc = alloc0(&m->Z1, M * MLP_HID)) || (rc = alloc0(&m->Z2, M * MLP_HID)) ||
      (rc = alloc0(&m->out, M * MLP_OUT)) || (rc = alloc0(&m->dout, M * MLP_OUT)) ||
      (rc = alloc0(&m->zero_delta, M * MLP_OUT)) ||
      (rc = alloc0(&m->partial, (size_t)mlp_backward_blocks((int)M) * MLP_PARAMS)) ||
      (rc = alloc0(&m->ci, 8 * psc)) || (rc = alloc0(&m->aux, 4 * psc)) || (rc = alloc0(&m->errs, K * ps)) ||
      (rc = alloc0(&m->Aes, K * ps)) || (rc = alloc0(&m->dW, 8 * psc)) || (rc = alloc0(&m->tx, psc)) ||
      (rc = alloc0(&m->ty, psc)) || (rc = alloc0(&m->partials, 1024)) || (rc = alloc0(&m->energies, K)) ||
      (rc = alloc0(&m->scale, K)))
    return rc;
  m->cap_n = n;
  m->cap_k = K;
  return BMG_OK;
}

bool level_size_ok(int n) { return n >= 3 && ((n + 1) & n) == 0; }

void free_tg(bmg_mlp* m) {
  void* ptrs[] = {m->tg_X, m->tg_Z1, m->tg_Z2, m->tg_out, m->tg_dout, m->tg_partial, m->tg_err};
  for (void* p : ptrs) cudaFree(p);
  m->tg_X = m->tg_Z1 = m->tg_Z2 = m->tg_out = m->tg_dout = m->tg_partial = nullptr;
  m->tg_err = nullptr;
  m->tg_rows = 0;
}

int ensure_tg(bmg_mlp* m, size_t rows) {
  if (rows <= m->tg_rows) return BMG_OK;
  free_tg(m);
  int rc;
  if ((rc = alloc0(&m->tg_X, rows * MLP_IN)) || (rc = alloc0(&m->tg_Z1, rows * MLP_HID)) ||
      (rc = alloc0(&m->tg_Z2, rows * MLP_HID)) || (rc = alloc0(&m->tg_out, rows * MLP_OUT)) ||
      (rc = alloc0(&m->tg_dout, rows * MLP_OUT)) ||
      (rc = alloc0(&m->tg_partial, (size_t)mlp_backward_blocks((int)rows) * MLP_PARAMS)) ||
      (rc = alloc0(&m->tg_err, 1))) {
    free_tg(m);
    return rc;
  }
  m->tg_rows = rows;
  return BMG_OK;
}

}  // namespace

namespace bmg {
// Level-0 learned weights for bmg_setup: features, tensor-core inference, weights.
int mlp_level0_interp(const void* mp, int n, const double* st, double* ci, cudaStream_t s) {
  const bmg_mlp* m = (const bmg_mlp*)mp;
  int nc = (n - 1) / 2;
  size_t M = (size_t)nc * nc;
  float *X = nullptr, *delta = nullptr;
  CK(cudaMallocAsync((void**)&X, M * MLP_IN * sizeof(float), s));
  CK(cudaMallocAsync((void**)&delta, M * MLP_OUT * sizeof(float), s));
  launch_features(n, st, X, s);
  launch_mlp_infer(X, (int)M, m->par, delta, s);
  launch_learned_ci(n, st, delta, ci, nullptr, s);
  CK(cudaFreeAsync(X, s));
  CK(cudaFreeAsync(delta, s));
  return cuda_check(cudaGetLastError(), "learned interpolation");
}
}  // namespace bmg

extern "C" {

int bmg_mlp_create(bmg_mlp** out) {
  if (!out) return set_error(BMG_EINVAL, "bmg_mlp_create: out is NULL");
  *out = nullptr;
  bmg_mlp* m = new bmg_mlp();
  int rc;
  if ((rc = alloc0(&m->par, MLP_PARAMS)) || (rc = alloc0(&m->grad, MLP_PARAMS)) || (rc = alloc0(&m->m, MLP_PARAMS)) ||
      (rc = alloc0(&m->v, MLP_PARAMS))) {
    bmg_mlp_free(m);
    return rc;
  }
  *out = m;
  return BMG_OK;
}

int bmg_mlp_set_params(bmg_mlp* m, const float* host, int count) {
  if (!m || !host || count != MLP_PARAMS) return set_error(BMG_EINVAL, "bmg_mlp_set_params: need %d floats", MLP_PARAMS);
  CK(cudaMemcpy(m->par, host, sizeof(float) * MLP_PARAMS, cudaMemcpyHostToDevice));
  CK(cudaMemset(m->m, 0, sizeof(float) * MLP_PARAMS));
  CK(cudaMemset(m->v, 0, sizeof(float) * MLP_PARAMS));
  m->step = 0;
  return BMG_OK;
}

int bmg_mlp_get_params(const bmg_mlp* m, float* host, int count) {
  if (!m || !host || count != MLP_PARAMS) return set_error(BMG_EINVAL, "bmg_mlp_get_params: need %d floats", MLP_PARAMS);
  CK(cudaMemcpy(host, m->par, sizeof(float) * MLP_PARAMS, cudaMemcpyDeviceToHost));
  return BMG_OK;
}

int bmg_mlp_get_adam(const bmg_mlp* m, float* moment1, float* moment2, int* step, int count) {
  if (!m || !moment1 || !moment2 || !step || count != MLP_PARAMS)
    return set_error(BMG_EINVAL, "bmg_mlp_get_adam: need two arrays of %d floats and a step", MLP_PARAMS);
  CK(cudaMemcpy(moment1, m->m, sizeof(float) * MLP_PARAMS, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(moment2, m->v, sizeof(float) * MLP_PARAMS, cudaMemcpyDeviceToHost));
  *step = m->step;
  return BMG_OK;
}

int bmg_mlp_set_adam(bmg_mlp* m, const float* moment1, const float* moment2, int step, int count) {
  if (!m || !moment1 || !moment2 || step < 0 || count != MLP_PARAMS)
    return set_error(BMG_EINVAL, "bmg_mlp_set_adam: need two arrays of %d floats and a step >= 0", MLP_PARAMS);
  CK(cudaMemcpy(m->m, moment1, sizeof(float) * MLP_PARAMS, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(m->v, moment2, sizeof(float) * MLP_PARAMS, cudaMemcpyHostToDevice));
  m->step = step;
  return BMG_OK;
}

int bmg_mlp_loss_grad(bmg_mlp* m, int n, const double* coef, int K, const double* vecs, const double* eref,
                      double* loss, float* grad, double* eref_out, void* stream) {
  if (!m || !level_size_ok(n) || !coef || K < 1 || !vecs || !loss)
    return set_error(BMG_EINVAL, "bmg_mlp_loss_grad: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  if ((rc = ensure_ws(m, n, K))) return rc;
  int nc = (n - 1) / 2;
  int M = nc * nc;
  std::vector<double> ref(K), e(K), sc(K);
  if (eref) {
    for (int k = 0; k < K; ++k) ref[k] = eref[k];
  } else {
    launch_learned_ci(n, coef, m->zero_delta, m->ci, nullptr, s);
    launch_tv_energies(n, coef, m->ci, K, vecs, m->errs, m->Aes, m->partials, m->energies, s);
    CK(cudaMemcpyAsync(ref.data(), m->energies, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (eref_out)
      for (int k = 0; k < K; ++k) eref_out[k] = ref[k];
  }
  launch_features(n, coef, m->X, s);
  launch_mlp_fwd(m->X, M, m->par, m->Z1, m->Z2, m->out, s);
  launch_learned_ci(n, coef, m->out, m->ci, m->aux, s);
  launch_tv_energies(n, coef, m->ci, K, vecs, m->errs, m->Aes, m->partials, m->energies, s);
  CK(cudaMemcpyAsync(e.data(), m->energies, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double L = 0.0;
  for (int k = 0; k < K; ++k) {
    L += e[k] / ref[k] / K;
    sc[k] = -2.0 / (ref[k] * K);
  }
  *loss = L;
  CK(cudaMemcpyAsync(m->scale, sc.data(), sizeof(double) * K, cudaMemcpyHostToDevice, s));
  launch_tv_grad(n, coef, K, vecs, m->Aes, m->scale, m->aux, m->dW, m->tx, m->ty, m->dout, s);
  launch_mlp_bwd(m->X, M, m->par, m->Z1, m->Z2, m->dout, m->partial, m->grad, s);
  if (grad) CK(cudaMemcpyAsync(grad, m->grad, sizeof(float) * MLP_PARAMS, cudaMemcpyDeviceToHost, s));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return std::isfinite(L) ? BMG_OK : set_error(BMG_ENAN, "bmg_mlp_loss_grad: loss is not finite");
}

int bmg_mlp_twogrid(bmg_mlp* m, int ncrop, int n, const double* coefs, int K, const double* vecs,
                    const double* eref, double* energies, double* loss, float* grad, void* stream) {
  if (!m || ncrop < 1 || !twogrid_size_ok(n) || !coefs || K < 1 || !vecs || !energies || (eref && !loss))
    return set_error(BMG_EINVAL, "bmg_mlp_twogrid: bad argument (n must be 7, 15 or 31)");
  cudaStream_t s = (cudaStream_t)stream;
  const int nc = (n - 1) / 2;
  const size_t rows = (size_t)ncrop * nc * nc;
  if (rows > (size_t)1 << 30) return set_error(BMG_EINVAL, "bmg_mlp_twogrid: too many crops");
  int rc;
  if ((rc = ensure_tg(m, rows))) return rc;
  CK(cudaMemsetAsync(m->tg_err, 0, sizeof(int), s));
  const float* delta = nullptr;
  if (eref) {
    launch_features_crops(n, ncrop, coefs, m->tg_X, s);
    launch_mlp_fwd(m->tg_X, (int)rows, m->par, m->tg_Z1, m->tg_Z2, m->tg_out, s);
    delta = m->tg_out;
  }
  if ((rc = launch_twogrid(n, ncrop, K, coefs, vecs, delta, eref, 1.0 / ncrop, energies, m->tg_dout, m->tg_err, s)))
    return rc;
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, m->tg_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (bad) return set_error(BMG_ESINGULAR, "bmg_mlp_twogrid: a crop's coarse operator has a non-positive pivot");
  if (!eref) return BMG_OK;
  std::vector<double> e((size_t)ncrop * K), r((size_t)ncrop * K);
  CK(cudaMemcpyAsync(e.data(), energies, sizeof(double) * e.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(r.data(), eref, sizeof(double) * r.size(), cudaMemcpyDeviceToHost, s));
  launch_mlp_bwd(m->tg_X, (int)rows, m->par, m->tg_Z1, m->tg_Z2, m->tg_dout, m->tg_partial, m->grad, s);
  if (grad) CK(cudaMemcpyAsync(grad, m->grad, sizeof(float) * MLP_PARAMS, cudaMemcpyDeviceToHost, s));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  double L = 0.0;
  for (size_t k = 0; k < e.size(); ++k) L += e[k] / r[k];
  L /= (double)e.size();
  *loss = L;
  return std::isfinite(L) ? BMG_OK : set_error(BMG_ENAN, "bmg_mlp_twogrid: loss is not finite");
}

int bmg_mlp_adam(bmg_mlp* m, float lr, void* stream) {
  if (!m || !(lr > 0.0f)) return set_error(BMG_EINVAL, "bmg_mlp_adam: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  m->step += 1;
  launch_adam(m->par, m->grad, m->m, m->v, lr, m->step, s);
  CK(cudaGetLastError());
  return cuda_check(cudaStreamSynchronize(s), "bmg_mlp_adam");
}

int bmg_mlp_infer(const bmg_mlp* m, int n, const double* coef, float* delta, void* stream) {
  if (!m || !level_size_ok(n) || !coef || !delta) return set_error(BMG_EINVAL, "bmg_mlp_infer: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  int nc = (n - 1) / 2;
  size_t M = (size_t)nc * nc;
  float* X = nullptr;
  CK(cudaMallocAsync((void**)&X, M * MLP_IN * sizeof(float), s));
  launch_features(n, coef, X, s);
  launch_mlp_infer(X, (int)M, m->par, delta, s);
  CK(cudaFreeAsync(X, s));
  CK(cudaGetLastError());
  return cuda_check(cudaStreamSynchronize(s), "bmg_mlp_infer");
}

int bmg_mlp_features(int n, const double* coef, float* X, void* stream) {
  if (!level_size_ok(n) || !coef || !X) return set_error(BMG_EINVAL, "bmg_mlp_features: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  launch_features(n, coef, X, s);
  CK(cudaGetLastError());
  return cuda_check(cudaStreamSynchronize(s), "bmg_mlp_features");
}

int bmg_learned_interp(int n, const double* coef, const float* delta, double* ci, void* stream) {
  if (!level_size_ok(n) || !coef || !delta || !ci) return set_error(BMG_EINVAL, "bmg_learned_interp: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  launch_learned_ci(n, coef, delta, ci, nullptr, s);
  CK(cudaGetLastError());
  return cuda_check(cudaStreamSynchronize(s), "bmg_learned_interp");
}

int bmg_fill_uniform(int n, unsigned long long seed, double* x, void* stream) {
  if (n < 1 || !x) return set_error(BMG_EINVAL, "bmg_fill_uniform: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  launch_uniform_pm1(n, seed, x, s);
  CK(cudaGetLastError());
  return cuda_check(cudaStreamSynchronize(s), "bmg_fill_uniform");
}

void bmg_mlp_free(bmg_mlp* m) {
  if (!m) return;
  free_ws(m);
  free_tg(m);
  cudaFree(m->par);
  cudaFree(m->grad);
  cudaFree(m->m);
  cudaFree(m->v);
  delete m;
}

}  // extern "C"
