// C entry points of the screening network (include/ftp.h, ftp_mlp_*): a
// handle that owns the FP32 master parameters, the Adam moments and the
// per-CTA gradient partials on one device, and drives the tcgen05 forward and
// backward kernels of ftp_mlp.cu.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "ftp.h"
#include "ftp_internal.cuh"
#include "ftp_screen.cuh"

using namespace ftp;

struct ftp_mlp_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int nfeat = 0;
  int64_t np = 0;
  int num_sms = 0;
  int64_t step = 0;  // Adam steps taken
  float* d_params = nullptr;
  float* d_m = nullptr;
  float* d_v = nullptr;
  float* d_partial = nullptr;  // [num_sms][np + 1]
  float* d_grad = nullptr;
  float* d_loss = nullptr;     // one per step of the last ftp_mlp_train
  int64_t loss_cap = 0;
  int* d_status = nullptr;
  int* h_status = nullptr;
  // staging of host arrays
  void* d_stage = nullptr;
  size_t stage_cap = 0;
};

namespace ftp {
const float* mlp_params_dev(const ::ftp_mlp_s* h) { return h->d_params; }
int mlp_nfeat(const ::ftp_mlp_s* h) { return h->nfeat; }
int mlp_device(const ::ftp_mlp_s* h) { return h->device; }
}  // namespace ftp

namespace {

bool on_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

struct DeviceGuard {
  int prev = 0;
  explicit DeviceGuard(int d) {
    cudaGetDevice(&prev);
    cudaSetDevice(d);
  }
  ~DeviceGuard() { cudaSetDevice(prev); }
};

#define MLP_CK(x)                          \
  do {                                     \
    if ((x) != cudaSuccess) {              \
      cudaGetLastError();                  \
      return FTP_ERR_CUDA;                 \
    }                                      \
  } while (0)

// Staging area of at least `bytes` (grow-only).
ftp_status stage(ftp_mlp_t h, size_t bytes) {
  if (h->stage_cap >= bytes) return FTP_OK;
  if (h->d_stage) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->d_stage);
  }
  h->d_stage = nullptr;
  h->stage_cap = 0;
  if (cudaMalloc(&h->d_stage, bytes) != cudaSuccess) {
    cudaGetLastError();
    return FTP_ERR_OOM;
  }
  h->stage_cap = bytes;
  return FTP_OK;
}

ftp_status finish(ftp_mlp_t h) {
  MLP_CK(cudaMemcpyAsync(h->h_status, h->d_status, sizeof(int) * ST_WORDS,
                         cudaMemcpyDeviceToHost, h->stream));
  MLP_CK(cudaStreamSynchronize(h->stream));
  return (ftp_status)h->h_status[ST_CODE];
}

uint64_t splitmix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

}  // namespace

extern "C" {

int64_t ftp_mlp_param_count(int nfeat) {
  return nfeat >= 1 && nfeat <= kMlpMaxFeat ? mlp_param_count(nfeat) : -1;
}

void ftp_mlp_destroy(ftp_mlp_t h) {
  if (!h) return;
  DeviceGuard g(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  cudaFree(h->d_params);
  cudaFree(h->d_m);
  cudaFree(h->d_v);
  cudaFree(h->d_partial);
  cudaFree(h->d_grad);
  cudaFree(h->d_loss);
  cudaFree(h->d_status);
  cudaFree(h->d_stage);
  if (h->h_status) cudaFreeHost(h->h_status);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

ftp_status ftp_mlp_set_params(ftp_mlp_t h, const float* params) {
  if (!h || !params) return FTP_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  MLP_CK(cudaMemcpyAsync(h->d_params, params, sizeof(float) * h->np, cudaMemcpyDefault,
                         h->stream));
  MLP_CK(cudaMemsetAsync(h->d_m, 0, sizeof(float) * h->np, h->stream));
  MLP_CK(cudaMemsetAsync(h->d_v, 0, sizeof(float) * h->np, h->stream));
  MLP_CK(cudaStreamSynchronize(h->stream));
  h->step = 0;
  return FTP_OK;
}

ftp_status ftp_mlp_get_params(ftp_mlp_t h, float* params) {
  if (!h || !params) return FTP_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  MLP_CK(cudaMemcpyAsync(params, h->d_params, sizeof(float) * h->np, cudaMemcpyDefault,
                         h->stream));
  MLP_CK(cudaStreamSynchronize(h->stream));
  return FTP_OK;
}

ftp_status ftp_mlp_get_state(ftp_mlp_t h, float* params, float* adam_m, float* adam_v,
                             int64_t* steps) {
  if (!h || !params || !adam_m || !adam_v || !steps) return FTP_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  const size_t pb = sizeof(float) * (size_t)h->np;
  MLP_CK(cudaMemcpyAsync(params, h->d_params, pb, cudaMemcpyDefault, h->stream));
  MLP_CK(cudaMemcpyAsync(adam_m, h->d_m, pb, cudaMemcpyDefault, h->stream));
  MLP_CK(cudaMemcpyAsync(adam_v, h->d_v, pb, cudaMemcpyDefault, h->stream));
  MLP_CK(cudaStreamSynchronize(h->stream));
  *steps = h->step;
  return FTP_OK;
}

ftp_status ftp_mlp_set_state(ftp_mlp_t h, const float* params, const float* adam_m,
                             const float* adam_v, int64_t steps) {
  // the step count keys the minibatch draws and Adam's bias correction (an
  // int in the update kernel)
  if (!h || !params || !adam_m || !adam_v || steps < 0 || steps > (int64_t)INT32_MAX - (1 << 20))
    return FTP_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  const size_t pb = sizeof(float) * (size_t)h->np;
  MLP_CK(cudaMemcpyAsync(h->d_params, params, pb, cudaMemcpyDefault, h->stream));
  MLP_CK(cudaMemcpyAsync(h->d_m, adam_m, pb, cudaMemcpyDefault, h->stream));
  MLP_CK(cudaMemcpyAsync(h->d_v, adam_v, pb, cudaMemcpyDefault, h->stream));
  MLP_CK(cudaStreamSynchronize(h->stream));
  h->step = steps;
  return FTP_OK;
}

ftp_status ftp_mlp_create(ftp_mlp_t* out, int nfeat, const float* params, uint64_t seed,
                          int device, void* cuda_stream) {
  if (!out) return FTP_ERR_INVALID_ARG;
  *out = nullptr;
  if (nfeat < 1 || nfeat > kMlpMaxFeat) return FTP_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return FTP_ERR_CUDA;
  }
  DeviceGuard g(device);
  ftp_mlp_s* h = new ftp_mlp_s();
  h->device = device;
  h->nfeat = nfeat;
  h->np = mlp_param_count(nfeat);
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (h->num_sms < 1) h->num_sms = 1;
  if (cuda_stream) {
    h->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return FTP_ERR_CUDA;
    }
    h->own_stream = true;
  }
  const size_t pb = sizeof(float) * (size_t)h->np;
  if (cudaMalloc(&h->d_params, pb) != cudaSuccess || cudaMalloc(&h->d_m, pb) != cudaSuccess ||
      cudaMalloc(&h->d_v, pb) != cudaSuccess || cudaMalloc(&h->d_grad, pb) != cudaSuccess ||
      cudaMalloc(&h->d_partial, sizeof(float) * (size_t)h->num_sms * (h->np + 1)) !=
          cudaSuccess ||
      cudaMalloc(&h->d_status, sizeof(int) * ST_WORDS) != cudaSuccess ||
      cudaMallocHost(&h->h_status, sizeof(int) * ST_WORDS) != cudaSuccess) {
    cudaGetLastError();
    ftp_mlp_destroy(h);
    return FTP_ERR_OOM;
  }
  if (cudaMemset(h->d_status, 0, sizeof(int) * ST_WORDS) != cudaSuccess) {
    ftp_mlp_destroy(h);
    return FTP_ERR_CUDA;
  }
  ftp_status st;
  if (params) {
    st = ftp_mlp_set_params(h, params);
  } else {
    // U(-1/sqrt(fan_in), 1/sqrt(fan_in)) for the weights and biases of each
    // layer, from a counter-based generator
    std::vector<float> p((size_t)h->np);
    const int H = kMlpHidden;
    uint64_t ctr = seed * 0x9E3779B97F4A7C15ull;
    auto uni = [&](double a) {
      const double u = (double)(splitmix(ctr++) >> 11) * (1.0 / 9007199254740992.0);
      return (float)((2.0 * u - 1.0) * a);
    };
    size_t o = 0;
    const double a1 = 1.0 / sqrt((double)nfeat), a2 = 1.0 / sqrt((double)H);
    for (int i = 0; i < H * nfeat + H; ++i) p[o++] = uni(a1);       // W1, b1
    for (int i = 0; i < H * H + H; ++i) p[o++] = uni(a2);           // W2, b2
    for (int i = 0; i < H + 1; ++i) p[o++] = uni(a2);               // w3, b3
    st = ftp_mlp_set_params(h, p.data());
  }
  if (st != FTP_OK) {
    ftp_mlp_destroy(h);
    return st;
  }
  *out = h;
  return FTP_OK;
}

ftp_status ftp_mlp_forward(ftp_mlp_t h, const float* X, int64_t n, float* scores) {
  if (!h || n < 0 || (n > 0 && (!X || !scores))) return FTP_ERR_INVALID_ARG;
  if (n == 0) return FTP_OK;
  DeviceGuard g(h->device);
  const bool xd = on_device(X), sd = on_device(scores);
  const size_t xb = sizeof(float) * (size_t)n * h->nfeat, sb = sizeof(float) * (size_t)n;
  ftp_status st = stage(h, (xd ? 0 : xb) + (sd ? 0 : sb) + 256);
  if (st != FTP_OK) return st;
  const float* dX = X;
  float* dS = scores;
  unsigned char* sp = (unsigned char*)h->d_stage;
  if (!xd) {
    MLP_CK(cudaMemcpyAsync(sp, X, xb, cudaMemcpyHostToDevice, h->stream));
    dX = (const float*)sp;
    sp += (xb + 255) / 256 * 256;
  }
  if (!sd) dS = (float*)sp;
  MLP_CK(cudaMemsetAsync(h->d_status, 0, sizeof(int) * ST_WORDS, h->stream));
  if (launch_mlp_forward(h->d_params, h->nfeat, dX, n, dS, h->d_status, h->num_sms, h->stream) <
      0)
    return FTP_ERR_CUDA;
  MLP_CK(cudaGetLastError());
  if (!sd) MLP_CK(cudaMemcpyAsync(scores, dS, sb, cudaMemcpyDeviceToHost, h->stream));
  return finish(h);
}

ftp_status ftp_mlp_gradient(ftp_mlp_t h, const float* X, const float* target, int64_t rows,
                            const int64_t* idx, int64_t n, float* grad, float* loss) {
  if (!h || !X || !target || rows < 1 || n < 1) return FTP_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  const bool xd = on_device(X), td = on_device(target), id = !idx || on_device(idx);
  const size_t xb = sizeof(float) * (size_t)rows * h->nfeat, tb = sizeof(float) * (size_t)rows,
               ib = idx ? sizeof(int64_t) * (size_t)n : 0;
  auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
  ftp_status st = stage(h, (xd ? 0 : r256(xb)) + (td ? 0 : r256(tb)) + (id ? 0 : r256(ib)) + 256);
  if (st != FTP_OK) return st;
  unsigned char* sp = (unsigned char*)h->d_stage;
  const float* dX = X;
  const float* dT = target;
  const int64_t* dI = idx;
  if (!xd) {
    MLP_CK(cudaMemcpyAsync(sp, X, xb, cudaMemcpyHostToDevice, h->stream));
    dX = (const float*)sp;
    sp += r256(xb);
  }
  if (!td) {
    MLP_CK(cudaMemcpyAsync(sp, target, tb, cudaMemcpyHostToDevice, h->stream));
    dT = (const float*)sp;
    sp += r256(tb);
  }
  if (!id) {
    MLP_CK(cudaMemcpyAsync(sp, idx, ib, cudaMemcpyHostToDevice, h->stream));
    dI = (const int64_t*)sp;
  }
  if (!h->d_loss) {
    if (cudaMalloc(&h->d_loss, sizeof(float) * 1024) != cudaSuccess) return FTP_ERR_OOM;
    h->loss_cap = 1024;
  }
  MLP_CK(cudaMemsetAsync(h->d_status, 0, sizeof(int) * ST_WORDS, h->stream));
  const int gridn = launch_mlp_grad(h->d_params, h->nfeat, dX, dT, dI, 0, rows, n, h->d_partial,
                                    h->num_sms, h->d_status, h->num_sms, h->stream);
  if (gridn < 1) return FTP_ERR_CUDA;
  launch_mlp_reduce_adam(h->d_params, h->d_m, h->d_v, h->d_partial, gridn, h->nfeat, n, h->d_grad,
                         h->d_loss, 0, 0.f, 0.f, 0.f, 0.f, 1, h->stream);
  MLP_CK(cudaGetLastError());
  if (grad)
    MLP_CK(cudaMemcpyAsync(grad, h->d_grad, sizeof(float) * h->np, cudaMemcpyDefault, h->stream));
  if (loss) MLP_CK(cudaMemcpyAsync(loss, h->d_loss, sizeof(float), cudaMemcpyDefault, h->stream));
  return finish(h);
}

ftp_status ftp_mlp_train(ftp_mlp_t h, const float* X, const float* target, int64_t rows,
                         int64_t steps, int64_t batch, float lr, uint64_t seed, float* losses) {
  if (!h || !X || !target || rows < 1 || steps < 0 || batch < 1 || !(lr > 0.f))
    return FTP_ERR_INVALID_ARG;
  if (!on_device(X) || !on_device(target)) return FTP_ERR_INVALID_ARG;
  if (steps == 0) return FTP_OK;
  DeviceGuard g(h->device);
  if (h->loss_cap < steps) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->d_loss);
    h->d_loss = nullptr;
    h->loss_cap = 0;
    if (cudaMalloc(&h->d_loss, sizeof(float) * (size_t)steps) != cudaSuccess) {
      cudaGetLastError();
      return FTP_ERR_OOM;
    }
    h->loss_cap = steps;
  }
  MLP_CK(cudaMemsetAsync(h->d_status, 0, sizeof(int) * ST_WORDS, h->stream));
  for (int64_t it = 0; it < steps; ++it) {
    // minibatch rows drawn with replacement by a counter-based generator
    const uint64_t key = splitmix(seed ^ splitmix((uint64_t)(h->step + 1))) | 1ull;
    const int gridn = launch_mlp_grad(h->d_params, h->nfeat, X, target, nullptr, key, rows, batch,
                                      h->d_partial, h->num_sms, h->d_status, h->num_sms,
                                      h->stream);
    if (gridn < 1) return FTP_ERR_CUDA;
    h->step += 1;
    launch_mlp_reduce_adam(h->d_params, h->d_m, h->d_v, h->d_partial, gridn, h->nfeat, batch,
                           nullptr, h->d_loss + it, 1, lr, 0.9f, 0.999f, 1e-8f, (int)h->step,
                           h->stream);
  }
  MLP_CK(cudaGetLastError());
  if (losses)
    MLP_CK(cudaMemcpyAsync(losses, h->d_loss, sizeof(float) * (size_t)steps, cudaMemcpyDefault,
                           h->stream));
  return finish(h);
}

}  // extern "C"

extern "C" ftp_status ftp_training_rows(const double* power, const float* features, int nfeat,
                                        int64_t ncurves, const int64_t* row_off, double top_frac,
                                        int neighbours, double rand_frac, uint64_t seed,
                                        float* X_out, float* y_out, int64_t cap, int64_t* count,
                                        int device, void* cuda_stream) {
  if (!power || !features || !row_off || !X_out || !y_out || !count || ncurves < 1 ||
      nfeat < 1 || cap < 0 || *count < 0 || !(top_frac > 0.0) || !(top_frac <= 1.0) ||
      neighbours < 0 || !(rand_frac >= 0.0) || !(rand_frac <= 1.0))
    return FTP_ERR_INVALID_ARG;
  for (int64_t c = 0; c < ncurves; ++c)
    if (row_off[c] < 0 || row_off[c + 1] <= row_off[c]) return FTP_ERR_INVALID_ARG;
  DeviceGuard g(device);
  if (!on_device(power) || !on_device(features) || !on_device(X_out) || !on_device(y_out))
    return FTP_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int64_t r0 = row_off[0], rows = row_off[ncurves] - r0;
  std::vector<int64_t> rel((size_t)ncurves + 1);
  for (int64_t c = 0; c <= ncurves; ++c) rel[(size_t)c] = row_off[c] - r0;
  const int64_t nblocks = (rows + 4095) / 4096 + 1;
  int64_t *d_rowoff = nullptr, *d_blocks = nullptr;
  uint8_t* d_sel = nullptr;
  unsigned long long* d_count = nullptr;
  int* d_status = nullptr;
  ftp_status st = FTP_OK;
  if (cudaMalloc(&d_rowoff, sizeof(int64_t) * rel.size()) != cudaSuccess ||
      cudaMalloc(&d_blocks, sizeof(int64_t) * (size_t)nblocks) != cudaSuccess ||
      cudaMalloc(&d_sel, (size_t)rows) != cudaSuccess ||
      cudaMalloc(&d_count, sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&d_status, sizeof(int) * ST_WORDS) != cudaSuccess) {
    cudaGetLastError();
    st = FTP_ERR_OOM;
  }
  unsigned long long hc = (unsigned long long)*count;
  int hs[ST_WORDS] = {};
  if (st == FTP_OK) {
    cudaMemcpyAsync(d_rowoff, rel.data(), sizeof(int64_t) * rel.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_count, &hc, sizeof(hc), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(d_status, 0, sizeof(int) * ST_WORDS, s);
    SelectArgs a{};
    a.ncurves = (int)ncurves;
    a.row_off = d_rowoff;
    a.top_frac = top_frac;
    a.nbr = neighbours;
    a.rand_threshold = rand_frac >= 1.0 ? ~0ull : (uint64_t)(rand_frac * 18446744073709551616.0);
    a.seed = splitmix(seed);
    a.row_global0 = r0;
    a.sel = d_sel;
    a.status = d_status;
    launch_select(a, power + r0, true, s);
    launch_gather_rows(d_sel, rows, features + r0 * nfeat, nfeat, power + r0, X_out, y_out, cap,
                       d_count, d_blocks, d_status, s);
    cudaMemcpyAsync(&hc, d_count, sizeof(hc), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(hs, d_status, sizeof(hs), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
      st = FTP_ERR_CUDA;
    else if (hs[ST_CODE] != 0)
      st = (ftp_status)hs[ST_CODE];
    else
      *count = (int64_t)hc;
  }
  cudaFree(d_rowoff);
  cudaFree(d_blocks);
  cudaFree(d_sel);
  cudaFree(d_count);
  cudaFree(d_status);
  return st;
}
