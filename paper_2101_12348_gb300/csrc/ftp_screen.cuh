// Internal declarations of the screening path: features from the NFFT sums,
// the BF16 surrogate network (tcgen05 tensor cores), per-curve top-K
// selection and the list of work units the exact solver runs on.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ftp_internal.cuh"

struct ftp_mlp_s;  // the screening network handle of the C ABI

namespace ftp {

constexpr uint8_t FTP_SCREENED_OUT_FLAG = 32u;  // mirrors FTP_FLAG_SCREENED_OUT
constexpr int kFeatMaxH = 8;                    // features of at most 8 harmonics
constexpr int kMlpHidden = 128;
constexpr int kMlpMaxFeat = 2 * kFeatMaxH + 2;  // 18 inputs (K padded to 32)

// One lightcurve as the feature, selection and fill kernels see it.
struct ScreenCurve {
  int64_t sums_off;   // element offset of its sum rows
  int64_t nf_pad;     // row stride of those rows
  int64_t nf;         // frequencies
  int64_t row_base;   // first row of its frequencies in the chunk's per-frequency arrays
  int64_t out_row;    // first row of its features in the features output
  int64_t nobs;       // observations
  int64_t item_base;  // first of its (template, frequency) items in the chunk
  int64_t out_off;    // element offset of its output block [templates][nf]
  int32_t Hs;         // harmonics its sums were computed for
  int32_t curve;      // index of its moments block (MO_WORDS doubles each)
};
static_assert(sizeof(ScreenCurve) == 72, "ScreenCurve layout");

struct FeatArgs {
  const void* sums;         // float2 (mixed) or double2 (FP64) sum rows
  const double* moments;    // MO_WORDS doubles per curve
  const ScreenCurve* curves;
  int ncurves;
  int Hf;                   // feature harmonics (<= every curve's Hs)
  int64_t nrows;            // rows of the chunk (sum of nf)
  float* out;               // [rows][2 Hf + 2]
  const int* status;
};
// Returns the launches issued (1), 0 for no rows, -1 for an unsupported Hf.
int launch_features(const FeatArgs& a, bool fp64, cudaStream_t s);

struct SelectArgs {
  int ncurves;
  const int64_t* row_off;   // [ncurves + 1] curve c owns rows row_off[c] .. row_off[c+1]-1
  double top_frac;          // K = ceil(top_frac * nf), 1 <= K <= nf
  int nbr;                  // dilation: +- nbr neighbours
  uint64_t rand_threshold;  // 0: none; else also rows whose hash < threshold
  uint64_t seed;
  int64_t row_global0;      // global index of row 0 (hash counter)
  uint8_t* sel;             // [rows] out: 1 selected
  const int* status;
};
void launch_select(const SelectArgs& a, const void* score, bool score_fp64, cudaStream_t s);

void launch_unit_list(const RootsSeg* segs, const int64_t* seg_units, int nseg, int64_t nunits,
                      int ngw, const uint8_t* sel, int64_t* list, unsigned long long* count,
                      const int* status, cudaStream_t s);

void launch_fill(const ScreenCurve* curves, int ncurves, int64_t nitems, double* p, double* t1,
                 double* t2, double* t3, uint8_t* flags, const int* status, cudaStream_t s);

// ------------------------------------------------------------------ network
// Flat FP32 parameters: W1 [128][nfeat], b1 [128], W2 [128][128] (W2[j][i]:
// output j, input i), b2 [128], w3 [128], b3.
__host__ __device__ constexpr int64_t mlp_param_count(int nfeat) {
  return (int64_t)kMlpHidden * nfeat + 3 * kMlpHidden + (int64_t)kMlpHidden * kMlpHidden + 1;
}

// Scores of n rows of X [n][nfeat] (FP32).  Returns launches (1) or -1.
int launch_mlp_forward(const float* params, int nfeat, const float* X, int64_t n, float* score,
                       int* status, int num_sms, cudaStream_t s);

// Per-CTA partial gradients of the mean squared error over a minibatch of n
// rows of X [rows][nfeat] / target [rows] into partial
// [grid][mlp_param_count + 1] (the last entry the partial sum of squared
// residuals).  Row i of the minibatch is idx[i] when idx is given, else
// splitmix64(sample_key + i) mod rows when sample_key != 0, else i.  Returns
// the grid size used (>= 1), or -1.
int launch_mlp_grad(const float* params, int nfeat, const float* X, const float* target,
                    const int64_t* idx, uint64_t sample_key, int64_t rows, int64_t n,
                    float* partial, int max_grid, int* status, int num_sms, cudaStream_t s);

// Rows whose sel byte is set, in order, appended to X_out / y_out starting at
// row *count (device counter, updated); rows beyond cap are counted but not
// written.  score (double) is the target.  Uses block_counts scratch of
// ceil(rows / 4096) + 1 int64.  Returns launches.
int launch_gather_rows(const uint8_t* sel, int64_t rows, const float* X, int nfeat,
                       const double* score, float* X_out, float* y_out, int64_t cap,
                       unsigned long long* count, int64_t* block_counts, const int* status,
                       cudaStream_t s);

// The screening network handle (defined with the C entry points).
const float* mlp_params_dev(const ::ftp_mlp_s* h);
int mlp_nfeat(const ::ftp_mlp_s* h);
int mlp_device(const ::ftp_mlp_s* h);

// Sums the partials into grad (nullable) and loss (nullable, mean squared
// error), then (adam != 0) one Adam step on params with moments m, v.
void launch_mlp_reduce_adam(float* params, float* m, float* v, const float* partial, int grid,
                            int nfeat, int64_t n, float* grad, float* loss, int adam, float lr,
                            float beta1, float beta2, float eps, int step, cudaStream_t s);

}  // namespace ftp
