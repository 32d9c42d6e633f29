// C ABI of the learned-start model (Sec. 5.A.4, SCF initialisation): create / destroy, parameters,
// BF16 inference, FP32 loss and gradient, Adam training steps.  The start density itself
// (descriptors of a grid's atoms, SAD + correction) is in xls_api.cu beside the grid.
#include <string>
#include <vector>

#include "xls_internal.h"

using namespace xls;

#define XLS_TRY(expr)            \
  do {                           \
    xls_status _s = (expr);      \
    if (_s != XLS_OK) return _s; \
  } while (0)

namespace {

xls_status err(xls_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

#define MLP_CUDA(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) return err(XLS_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
xls_status dalloc(T** p, size_t bytes) {
  if (cudaMalloc((void**)p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return err(XLS_ENOMEM, "model: device allocation of " + std::to_string(bytes) + " B failed");
  }
  return XLS_OK;
}

void free_work(xls_mlp m) {
  float* fs[] = {m->A, m->D, m->e, m->X, m->y, m->yp};
  for (float* f : fs) cudaFree(f);
  cudaFree(m->loss_partial);
  m->A = m->D = m->e = m->X = m->y = m->yp = nullptr;
  m->loss_partial = nullptr;
  m->cap = 0;
}

// inputs on the host are staged into the work arrays; device inputs are used in place
xls_status stage(xls_mlp m, const float* X, const float* y, long long n, int on_device, const float** dX,
                 const float** dy) {
  XLS_TRY(mlp_reserve(m, n));
  if (on_device) {
    *dX = X;
    if (dy) *dy = y;
    return XLS_OK;
  }
  MLP_CUDA(cudaMemcpyAsync(m->X, X, (size_t)n * 32 * sizeof(float), cudaMemcpyHostToDevice, m->st));
  *dX = m->X;
  if (dy) {
    MLP_CUDA(cudaMemcpyAsync(m->y, y, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, m->st));
    *dy = m->y;
  }
  return XLS_OK;
}

}  // namespace

namespace xls {
xls_status mlp_reserve(xls_mlp_s* m, long long n) {
  if (n <= m->cap) return XLS_OK;
  free_work(m);
  const size_t nn = (size_t)n;
  XLS_TRY(dalloc(&m->A, nn * 192 * sizeof(float)));
  XLS_TRY(dalloc(&m->D, nn * 192 * sizeof(float)));
  XLS_TRY(dalloc(&m->e, nn * sizeof(float)));
  XLS_TRY(dalloc(&m->X, nn * 32 * sizeof(float)));
  XLS_TRY(dalloc(&m->y, nn * sizeof(float)));
  XLS_TRY(dalloc(&m->yp, nn * sizeof(float)));
  XLS_TRY(dalloc(&m->loss_partial, ((nn + 127) / 128) * sizeof(double)));
  m->cap = n;
  return XLS_OK;
}
}  // namespace xls

extern "C" {

xls_status xls_mlp_create(const double* params, int n_params, void* cuda_stream, xls_mlp* out) {
  if (!params || !out || n_params != mlp_param_count())
    return err(XLS_EINVAL, "xls_mlp_create: params must hold " + std::to_string(mlp_param_count()) + " values");
  xls_mlp m = new xls_mlp_s();
  m->st = (cudaStream_t)cuda_stream;
  m->n_params = n_params;
  xls_status s = XLS_OK;
  if ((s = dalloc(&m->theta, n_params * sizeof(float))) != XLS_OK || (s = dalloc(&m->m, n_params * sizeof(float))) != XLS_OK ||
      (s = dalloc(&m->v, n_params * sizeof(float))) != XLS_OK || (s = dalloc(&m->grad, n_params * sizeof(float))) != XLS_OK ||
      (s = dalloc(&m->wpartial, mlp_wpartial_floats() * sizeof(float))) != XLS_OK ||
      (s = dalloc(&m->loss, sizeof(double))) != XLS_OK) {
    xls_mlp_destroy(m);
    return s;
  }
  std::vector<float> f(params, params + n_params);
  cudaMemcpy(m->theta, f.data(), n_params * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemset(m->m, 0, n_params * sizeof(float));
  cudaMemset(m->v, 0, n_params * sizeof(float));
  *out = m;
  return XLS_OK;
}

xls_status xls_mlp_destroy(xls_mlp m) {
  if (!m) return XLS_OK;
  if (m->st) cudaStreamSynchronize(m->st);
  else cudaDeviceSynchronize();
  free_work(m);
  float* fs[] = {m->theta, m->m, m->v, m->grad, m->wpartial};
  for (float* f : fs) cudaFree(f);
  cudaFree(m->loss);
  delete m;
  return XLS_OK;
}

xls_status xls_mlp_get_params(xls_mlp m, double* params_out) {
  if (!m || !params_out) return err(XLS_EINVAL, "xls_mlp_get_params: bad arguments");
  std::vector<float> f(m->n_params);
  MLP_CUDA(cudaStreamSynchronize(m->st));
  MLP_CUDA(cudaMemcpy(f.data(), m->theta, m->n_params * sizeof(float), cudaMemcpyDeviceToHost));
  for (int i = 0; i < m->n_params; ++i) params_out[i] = f[i];
  return XLS_OK;
}

xls_status xls_mlp_infer(xls_mlp m, const float* X, long long n, float* y_out, int on_device) {
  if (!m || !X || !y_out || n < 0) return err(XLS_EINVAL, "xls_mlp_infer: bad arguments");
  if (n == 0) return XLS_OK;
  const float* dX = nullptr;
  XLS_TRY(stage(m, X, nullptr, n, on_device, &dX, nullptr));
  float* dy = on_device ? y_out : m->yp;
  launch_mlp_infer(n, m->theta, dX, dy, m->st);
  MLP_CUDA(cudaGetLastError());
  if (!on_device) MLP_CUDA(cudaMemcpyAsync(y_out, m->yp, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, m->st));
  MLP_CUDA(cudaStreamSynchronize(m->st));
  return XLS_OK;
}

xls_status xls_mlp_loss_grad(xls_mlp m, const float* X, const float* y, long long n, double* loss_out,
                             double* grad_out, int on_device) {
  if (!m || !X || !y || n < 1) return err(XLS_EINVAL, "xls_mlp_loss_grad: bad arguments");
  const float *dX = nullptr, *dy = nullptr;
  XLS_TRY(stage(m, X, y, n, on_device, &dX, &dy));
  launch_mlp_grad(n, m->theta, dX, dy, m->A, m->D, m->e, m->loss_partial, m->wpartial, m->grad, m->loss, m->st);
  MLP_CUDA(cudaGetLastError());
  double l = 0.0;
  MLP_CUDA(cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->st));
  std::vector<float> g;
  if (grad_out) {
    g.resize(m->n_params);
    MLP_CUDA(cudaMemcpyAsync(g.data(), m->grad, m->n_params * sizeof(float), cudaMemcpyDeviceToHost, m->st));
  }
  MLP_CUDA(cudaStreamSynchronize(m->st));
  if (loss_out) *loss_out = l / (double)n;
  if (grad_out)
    for (int i = 0; i < m->n_params; ++i) grad_out[i] = g[i];
  return XLS_OK;
}

xls_status xls_mlp_train_step(xls_mlp m, const float* X, const float* y, long long n, double lr, double* loss_out,
                              int on_device) {
  if (!m || !X || !y || n < 1 || !(lr > 0)) return err(XLS_EINVAL, "xls_mlp_train_step: bad arguments");
  const float *dX = nullptr, *dy = nullptr;
  XLS_TRY(stage(m, X, y, n, on_device, &dX, &dy));
  launch_mlp_grad(n, m->theta, dX, dy, m->A, m->D, m->e, m->loss_partial, m->wpartial, m->grad, m->loss, m->st);
  m->t += 1;
  launch_adam(m->n_params, m->theta, m->m, m->v, m->grad, (float)lr, m->t, m->st);
  MLP_CUDA(cudaGetLastError());
  double l = 0.0;
  MLP_CUDA(cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->st));
  MLP_CUDA(cudaStreamSynchronize(m->st));
  if (loss_out) *loss_out = l / (double)n;
  return XLS_OK;
}

}  // extern "C"
