// Instantiations of the assembly + roots kernel for mixed precision (FP32 sums and Aberth, FP64 assembly and polish), H = 1..16.
#include "ftp_roots.cuh"

namespace ftp {

int launch_roots_mixed(const RootsArgs& a, int num_sms, cudaStream_t s) {
  switch (a.H) {
#define FTP_CASE(h) \
  case h:           \
    return roots::launch_h<true, h>(a, num_sms, s);
    FTP_CASE(1) FTP_CASE(2) FTP_CASE(3) FTP_CASE(4) FTP_CASE(5) FTP_CASE(6) FTP_CASE(7) FTP_CASE(8)
    FTP_CASE(9) FTP_CASE(10) FTP_CASE(11) FTP_CASE(12) FTP_CASE(13) FTP_CASE(14) FTP_CASE(15)
    FTP_CASE(16)
#undef FTP_CASE
    default:
      return -1;
  }
}

size_t roots_smem_mixed(int H) {
  switch (H) {
#define FTP_CASE(h) \
  case h:           \
    return roots::Cfg<true, h>::SMEM;
    FTP_CASE(1) FTP_CASE(2) FTP_CASE(3) FTP_CASE(4) FTP_CASE(5) FTP_CASE(6) FTP_CASE(7) FTP_CASE(8)
    FTP_CASE(9) FTP_CASE(10) FTP_CASE(11) FTP_CASE(12) FTP_CASE(13) FTP_CASE(14) FTP_CASE(15)
    FTP_CASE(16)
#undef FTP_CASE
    default:
      return 0;
  }
}

}  // namespace ftp
