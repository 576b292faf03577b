// Allocation-free entry point: steps (b)-(c) on trigonometric sums the caller
// already holds in device memory, with every piece of scratch the kernel
// needs taken from a fixed array in the library's own device memory.
//
// Who needs it: code that must not allocate device memory - a host process
// whose device memory is owned by another runtime's pool allocator, a
// latency-bound loop where cudaMalloc/cudaFree (which can synchronise the
// device) are not acceptable, or a service running under a hard device-memory
// cap - can still call the periodogram's root stage; it passes the sums
// (e.g. from ftp_sums), the moments and device output arrays.
//
// The scratch lives in one file-scope __device__ array: every GPU that loads
// the library holds it until the process exits.  Host code cannot use the
// array's name as a device address (it is a host-side stand-in), so the first
// call on each device, with that device current, looks the address up with
// cudaGetSymbolAddress and caches it; make that first call before any stream
// capture.  All calls share the one array and it keeps the last call's
// contents, so everything the kernel counts on is cleared or written at the
// start of each call, and calls whose work overlaps on the GPU (other
// streams, other host threads) race on it.
//
// It cannot re-solve anything (it never sees the observations): an item whose
// Aberth iteration hit its cap keeps FTP_FLAG_NONCONVERGED, and an item whose
// estimated error of P from the sums exceeds the path's threshold (clustered
// phases) gets FTP_FLAG_UNRESOLVED.  The flags array is the only per-item
// report of either, so pass one when such items matter.
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "../../include/ftp.h"
#include "ftp_internal.cuh"

namespace {

using namespace ftp;

// Layout of the scratch array (bytes).
constexpr size_t kOffStatus = 0;                       // int[ST_WORDS]
constexpr size_t kOffCounters = 64;                    // unsigned long long[CNT_WORDS]
constexpr size_t kOffQueue = 128;                      // unsigned long long[2]
constexpr size_t kOffMoments = 192;                    // double[MO_WORDS]
constexpr size_t kOffRows = 256;                       // int[FTP_NOALLOC_MAX_TEMPLATES]
constexpr size_t kOffAlpha = 512;                      // double2[max templates][kMaxH]
constexpr size_t kScratchBytes =
    kOffAlpha + (size_t)FTP_NOALLOC_MAX_TEMPLATES * kMaxH * sizeof(double2);

static_assert(kOffRows + FTP_NOALLOC_MAX_TEMPLATES * sizeof(int) <= kOffAlpha, "layout");
static_assert(kOffCounters + CNT_WORDS * sizeof(unsigned long long) <= kOffQueue, "layout");
static_assert(kOffStatus + ST_WORDS * sizeof(int) <= kOffCounters, "layout");
static_assert(kScratchBytes == FTP_NOALLOC_SCRATCH_BYTES, "header states the scratch size");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device `dev`.
cudaError_t scratch_address(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// True for device memory of `device` and for managed memory; host memory,
// unknown pointers and another GPU's memory (which the kernels could only
// reach through peer mappings this call does not set up) are rejected.
bool on_device(const void* p, int device) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == device;
}

}  // namespace

extern "C" ftp_status ftp_periodogram_sums_noalloc(
    const void* sums, int64_t row_stride, ftp_precision prec, int64_t nf, int H_sums, double ybar,
    double YY, const ftp_template* tpl, int ntemplates, double* power, double* theta1,
    double* theta2, double* theta3, uint8_t* flags, int device, void* cuda_stream) {
  // ---- arguments (no device work yet)
  if (!sums || !tpl || !power || !theta1 || !theta2 || !theta3) return FTP_ERR_INVALID_ARG;
  if (prec != FTP_MIXED && prec != FTP_FP64) return FTP_ERR_INVALID_ARG;
  if (nf < 1 || H_sums < 1 || H_sums > FTP_MAX_H || ntemplates < 1) return FTP_ERR_INVALID_ARG;
  if (ntemplates > FTP_NOALLOC_MAX_TEMPLATES) return FTP_ERR_UNSUPPORTED;
  if (!(YY > 0.0) || !isfinite(YY) || !isfinite(ybar)) return FTP_ERR_INVALID_ARG;
  const size_t esz = (prec == FTP_MIXED) ? sizeof(float2) : sizeof(double2);
  const int64_t need = (nf + 63) / 64 * 64;  // rows are read in whole work units
  if (row_stride < need || (row_stride * (int64_t)esz) % 16 != 0 ||
      ((uintptr_t)sums & 15) != 0)
    return FTP_ERR_INVALID_ARG;
  for (int i = 0; i < ntemplates; ++i) {
    if (tpl[i].H < 1 || tpl[i].H > H_sums || !tpl[i].c || !tpl[i].s) return FTP_ERR_INVALID_ARG;
    for (int n = 0; n < tpl[i].H; ++n)
      if (!isfinite(tpl[i].c[n]) || !isfinite(tpl[i].s[n])) return FTP_ERR_NONFINITE;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev ||
      device >= kMaxDevices) {
    cudaGetLastError();
    return FTP_ERR_INVALID_ARG;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return FTP_ERR_CUDA;
  struct Restore {
    int d;
    ~Restore() { cudaSetDevice(d); }
  } restore{prev};
  if (!on_device(sums, device) || !on_device(power, device) || !on_device(theta1, device) ||
      !on_device(theta2, device) || !on_device(theta3, device) ||
      (flags && !on_device(flags, device)))
    return FTP_ERR_INVALID_ARG;

  unsigned char* scratch = nullptr;
  if (scratch_address(device, &scratch) != cudaSuccess) return FTP_ERR_CUDA;
  int* status = reinterpret_cast<int*>(scratch + kOffStatus);
  auto* counters = reinterpret_cast<unsigned long long*>(scratch + kOffCounters);
  auto* queue = reinterpret_cast<unsigned long long*>(scratch + kOffQueue);
  double* moments = reinterpret_cast<double*>(scratch + kOffMoments);
  int* rows = reinterpret_cast<int*>(scratch + kOffRows);
  double2* alpha = reinterpret_cast<double2*>(scratch + kOffAlpha);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

  // ---- templates grouped by H (insertion order within a group), host side
  double2 h_alpha[FTP_NOALLOC_MAX_TEMPLATES * kMaxH];
  int h_rows[FTP_NOALLOC_MAX_TEMPLATES];
  int group_H[FTP_NOALLOC_MAX_TEMPLATES], group_first[FTP_NOALLOC_MAX_TEMPLATES],
      group_count[FTP_NOALLOC_MAX_TEMPLATES];
  int ngroups = 0, q = 0;
  for (int H = 1; H <= FTP_MAX_H; ++H) {
    const int first = q;
    for (int i = 0; i < ntemplates; ++i) {
      if (tpl[i].H != H) continue;
      for (int n = 0; n < kMaxH; ++n)
        h_alpha[q * kMaxH + n] = (n < H) ? make_double2(0.5 * tpl[i].c[n], 0.5 * tpl[i].s[n])
                                         : make_double2(0.0, 0.0);
      h_rows[q++] = i;
    }
    if (q > first) {
      group_H[ngroups] = H;
      group_first[ngroups] = first;
      group_count[ngroups++] = q - first;
    }
  }
  const double h_moments[MO_WORDS] = {ybar, YY, 1.0, 0.0};

  // ---- everything the kernel reads is written here: nothing carries over
#define FTP_NA(x)                                              \
  do {                                                         \
    if ((x) != cudaSuccess) {                                  \
      cudaGetLastError();                                      \
      return FTP_ERR_CUDA;                                     \
    }                                                          \
  } while (0)
  FTP_NA(cudaMemsetAsync(status, 0, sizeof(int) * ST_WORDS, s));
  FTP_NA(cudaMemsetAsync(counters, 0, sizeof(unsigned long long) * CNT_WORDS, s));
  FTP_NA(cudaMemcpyAsync(moments, h_moments, sizeof(h_moments), cudaMemcpyHostToDevice, s));
  FTP_NA(cudaMemcpyAsync(rows, h_rows, sizeof(int) * ntemplates, cudaMemcpyHostToDevice, s));
  FTP_NA(cudaMemcpyAsync(alpha, h_alpha, sizeof(double2) * kMaxH * ntemplates,
                         cudaMemcpyHostToDevice, s));
  int num_sms = 0;
  FTP_NA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device));
  for (int g = 0; g < ngroups; ++g) {
    RootsArgs a{};
    a.sums = sums;
    a.sums_elems = (int64_t)3 * H_sums * row_stride;
    a.out_elems = (int64_t)ntemplates * nf;
    a.nf = nf;
    a.nf_pad = row_stride;
    a.Hs = H_sums;
    a.H = group_H[g];
    a.ntpl = group_count[g];
    a.alpha = alpha + (size_t)group_first[g] * kMaxH;
    a.rows = rows + group_first[g];
    a.moments = moments;
    a.power = power;
    a.theta1 = theta1;
    a.theta2 = theta2;
    a.theta3 = theta3;
    a.flags = flags;
    a.out_stride = nf;
    a.status = status;
    a.counters = counters;
    a.queue = queue;
    a.maxit = (prec == FTP_MIXED) ? 60 : 80;
    a.polish_steps = 1;
    a.wait_polls = kWaitPolls;
    // the a-posteriori error estimate of P runs without a re-solve list:
    // items above the threshold get FTP_FLAG_UNRESOLVED instead
    a.sum_err = (prec == FTP_MIXED) ? kSumErrF32 : kSumErrF64;
    a.redo_tol = (prec == FTP_MIXED) ? kRedoTolF32 : kRedoTolF64;
    FTP_NA(cudaMemsetAsync(queue, 0, sizeof(unsigned long long), s));
    const int r = launch_roots(prec == FTP_MIXED ? ROOTS_MIXED : ROOTS_FP64, a, num_sms, s);
    if (r == -1) return FTP_ERR_UNSUPPORTED;
    if (r < 0) return FTP_ERR_CUDA;
    FTP_NA(cudaGetLastError());
  }
  int h_status[ST_WORDS] = {};
  FTP_NA(cudaMemcpyAsync(h_status, status, sizeof(h_status), cudaMemcpyDeviceToHost, s));
  FTP_NA(cudaStreamSynchronize(s));
#undef FTP_NA
  return (ftp_status)h_status[ST_CODE];
}
