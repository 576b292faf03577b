// Instantiations of the root-stage kernels for float2 sums from the FP32 NFFT, FP32 Aberth (mixed
// path), H = 1..16: the first kernel and the one-lane-per-item evaluation kernel.
#include "ftp_eval.cuh"

namespace ftp {

namespace {
// Lanes per item: the smallest power of two that keeps the per-lane root
// count (and so the register footprint) small; a unit row must stay a
// multiple of 16 bytes for the bulk copies.
constexpr int pick_g(int H) {
  const int D = 6 * H - 2;
  const int maxrr = sizeof(float) == 4 ? 5 : 4;
  const int gmax = sizeof(float2) == 8 ? 16 : 32;
  int g = 4;
  while (g < gmax && (D + g - 1) / g > maxrr) g *= 2;
  return g;
}
}  // namespace

int roots_lanes_mixed(int H) { return (H >= 1 && H <= kMaxH) ? pick_g(H) : 0; }

int launch_roots_mixed(const RootsArgs& a, int num_sms, cudaStream_t s) {
  switch (a.H) {
#define FTP_CASE(h) \
  case h:           \
    return roots::launch_h_mixed<h, pick_g(h)>(a, num_sms, s);
    FTP_CASE(1) FTP_CASE(2) FTP_CASE(3) FTP_CASE(4) FTP_CASE(5) FTP_CASE(6) FTP_CASE(7) FTP_CASE(8)
    FTP_CASE(9) FTP_CASE(10) FTP_CASE(11) FTP_CASE(12) FTP_CASE(13) FTP_CASE(14) FTP_CASE(15)
    FTP_CASE(16)
#undef FTP_CASE
    default:
      return -1;
  }
}

}  // namespace ftp
