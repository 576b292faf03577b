// The screening surrogate: a 2H+2 -> 128 -> 128 -> 1 ReLU network with BF16
// weights and activations and FP32 accumulation, on the fifth-generation
// tensor cores (tcgen05 MMA, accumulators in tensor memory).  Not part of the
// paper: it ranks trial frequencies so that the exact template periodogram
// runs only on the most promising ones.
//
// Network (per row m):
//   Z1 = bf16(x) W1b^T + b1,  A1 = bf16(relu(Z1))
//   Z2 = A1 W2b^T + b2,       A2 = bf16(relu(Z2))
//   s  = A2 . w3b + b3
// Training minimises mean((s - target)^2).  Backward, per minibatch:
//   ds = 2 (s - target) / n,  dZ2 = ds w3b * [Z2 > 0]
//   g_w3 = sum A2 ds, g_b3 = sum ds, g_b2 = sum dZ2
//   g_W2 = bf16(dZ2)^T A1, dA1 = bf16(dZ2) W2b, dZ1 = dA1 * [Z1 > 0]
//   g_b1 = sum dZ1, g_W1 = bf16(dZ1)^T bf16(x)
//
// The forward kernel adds b1 and b2 on the tensor core: W1's operand tile
// carries both as three-term BF16 splits (b to about 24 bits, so Z1 and Z2
// are the same FP32 sums), b1 against ones in the X tile and b2 against an
// indicator operand, which keeps the shared-memory pipe, the forward's
// bound, free of per-tile bias loads.
//
// Tiles of 128 rows.  One thread owns one row (its TMEM lane).  Every
// operand tile is written once to shared memory in the core-matrix layout of
// ftp_tc.cuh; the products that need a transposed operand read the same bytes
// with the MN-major descriptor bit, so nothing is ever transposed.  TMEM
// columns (gradient kernel): [0,128) Z1 then dA1, [128,256) Z2,
// [256,384) g_W2 accumulated over all tiles of the CTA, [384,384+KP) g_W1.
#include <math.h>
#include <stdint.h>

#include "ftp_internal.cuh"
#include "ftp_screen.cuh"
#include "ftp_tc.cuh"

namespace ftp {

namespace {

constexpr int HID = kMlpHidden;
constexpr int T128 = HID * HID * 2;  // bytes of a 128 x 128 BF16 tile

template <int KP> struct FwdL {
  static constexpr int W1 = 0;
  static constexpr int W2 = W1 + HID * KP * 2;
  static constexpr int X = W2 + T128;
  static constexpr int A1 = X + HID * KP * 2;
  static constexpr int IND = A1 + T128;  // 8 x KP indicator rows (b2 selector)
  static constexpr int VEC = IND + 8 * KP * 2;  // b1, b2, bf16(w3): [3][128] FP32
  static constexpr int BAR = VEC + 3 * HID * 4;
  static constexpr int SLOT = BAR + 16;
  static constexpr int BYTES = SLOT + 16;
};

template <int KP> struct GradL {
  static constexpr int W1 = 0;
  static constexpr int W2 = W1 + HID * KP * 2;
  static constexpr int X = W2 + T128;
  static constexpr int A1 = X + HID * KP * 2;
  static constexpr int DZ2 = A1 + T128;
  static constexpr int DZ1 = DZ2 + T128;
  static constexpr int VEC = DZ1 + T128;     // b1, b2, bf16(w3)
  static constexpr int RED = VEC + 3 * HID * 4;  // [4 warps][3][128] FP32
  static constexpr int SCAL = RED + 4 * 3 * HID * 4;  // [4 warps][2]
  static constexpr int BAR = SCAL + 64;
  static constexpr int SLOT = BAR + 16;
  static constexpr int BYTES = SLOT + 16;
};

// Sync point between MMA issue and the other threads: shared-memory operands
// written by the threads become visible to the tensor core, and TMEM reads of
// the threads are ordered before the next MMA.
__device__ __forceinline__ void mma_sync_point() {
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
}

// Weights into shared memory as BF16 operand tiles, vectors as FP32.
// With `fold` (the forward kernel), W1's operand tile also carries the
// biases as three-term BF16 splits b = hi + mid + lo (hi = bf16(b), mid =
// bf16(b - hi), lo = bf16(b - hi - mid): b to about 24 bits): b1 in columns
// nfeat .. nfeat + 2, which meet ones in the X tile, and b2 in columns
// nfeat + 3 .. nfeat + 5, which meet ones in the indicator rows; so the
// tensor core adds both, in FP32, and no thread loads a bias per tile.
__device__ __forceinline__ float bias_part(float b, int part) {
  const float hi = tc::bf16_round(b);
  const float mid = tc::bf16_round(b - hi);
  return part == 0 ? hi : part == 1 ? mid : tc::bf16_round(b - hi - mid);
}

template <int KP>
__device__ void load_weights(const float* __restrict__ P, int nfeat, unsigned char* sW1,
                             unsigned char* sW2, float* vec, bool fold = false) {
  const float* W1 = P;
  const float* b1 = P + HID * nfeat;
  const float* W2 = b1 + HID;
  const float* b2 = W2 + HID * HID;
  const float* w3 = b2 + HID;
  for (int idx = threadIdx.x; idx < HID * (KP / 8); idx += blockDim.x) {
    const int r = idx / (KP / 8), q = idx % (KP / 8);
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = q * 8 + e, f = k - nfeat;
      v[e] = k < nfeat              ? W1[r * nfeat + k]
             : fold && f < 3        ? bias_part(b1[r], f)
             : fold && f < 6        ? bias_part(b2[r], f - 3)
                                    : 0.f;
    }
    *reinterpret_cast<uint4*>(sW1 + tc::core_off(r, q * 8, KP)) = tc::pack8(v);
  }
  for (int idx = threadIdx.x; idx < HID * (HID / 8); idx += blockDim.x) {
    const int r = idx / (HID / 8), q = idx % (HID / 8);
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = W2[r * HID + q * 8 + e];
    *reinterpret_cast<uint4*>(sW2 + tc::core_off(r, q * 8, HID)) = tc::pack8(v);
  }
  for (int i = threadIdx.x; i < HID; i += blockDim.x) {
    vec[i] = b1[i];
    vec[HID + i] = b2[i];
    vec[2 * HID + i] = tc::bf16_round(w3[i]);
  }
}

// splitmix64: a counter-based generator (Steele, Lea & Flood 2014).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Row of X behind minibatch entry i.
struct RowMap {
  const int64_t* idx;
  uint64_t key;
  int64_t rows;
  __device__ __forceinline__ int64_t operator()(int64_t i) const {
    return idx ? idx[i] : key ? (int64_t)(splitmix64(key + (uint64_t)i) % (uint64_t)rows) : i;
  }
};

// Minibatch entries r0.. into the X tile; entries past n are 0.
template <int KP>
__device__ void stage_x(const float* __restrict__ X, RowMap map, int64_t n, int64_t r0, int nfeat,
                        unsigned char* sX) {
  for (int t = threadIdx.x; t < HID * (KP / 8); t += blockDim.x) {
    const int r = t / (KP / 8), q = t % (KP / 8);
    const int64_t i = r0 + r;
    float v[8];
    if (i < n) {
      const int64_t row = map(i);
      const float* x = X + row * nfeat;
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = q * 8 + e < nfeat ? x[q * 8 + e] : 0.f;
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = 0.f;
    }
    *reinterpret_cast<uint4*>(sX + tc::core_off(r, q * 8, KP)) = tc::pack8(v);
  }
}

// After it, lane l of the warp holds the sum over the warp's lanes of v[l].
__device__ __forceinline__ float transpose_reduce(float (&v)[32], int lane) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const float send = up ? v[i] : v[i + o];
      const float keep = up ? v[i + o] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0];
}

__device__ __forceinline__ void store_row(unsigned char* tile, int row, int col0, const float* v) {
#pragma unroll
  for (int q = 0; q < 4; ++q)
    *reinterpret_cast<uint4*>(tile + tc::core_off(row, col0 + q * 8, HID)) = tc::pack8(v + q * 8);
}

// The forward kernel's X tiles, prefetched into registers: thread t holds
// the chunks (row, 8 features) c = t + 128 u, u < KP / 8, of a tile, loaded
// while the previous tile is in the tensor cores and epilogues.
template <int KP> struct XChunks {
  float v[KP / 8][8];
};
template <int KP>
__device__ __forceinline__ void load_x(const float* __restrict__ X, int64_t n, int64_t r0,
                                       int nfeat, XChunks<KP>& c) {
#pragma unroll
  for (int u = 0; u < KP / 8; ++u) {
    const int t = threadIdx.x + HID * u;
    const int r = t / (KP / 8), q = t % (KP / 8);
    const int64_t i = r0 + r;
    const float* x = X + i * nfeat;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = q * 8 + e;
      c.v[u][e] = k < nfeat ? (i < n ? x[k] : 0.f) : k < nfeat + 3 ? 1.f : 0.f;
    }
  }
}
template <int KP>
__device__ __forceinline__ void store_x(const XChunks<KP>& c, unsigned char* sX) {
#pragma unroll
  for (int u = 0; u < KP / 8; ++u) {
    const int t = threadIdx.x + HID * u;
    const int r = t / (KP / 8), q = t % (KP / 8);
    *reinterpret_cast<uint4*>(sX + tc::core_off(r, q * 8, KP)) = tc::pack8(c.v[u]);
  }
}

// bf16(relu(Z)) of this thread's TMEM lane (128 FP32 columns, biases already
// in Z) into its row of a 128 x 128 operand tile: ReLU and rounding in one
// conversion per pair; the next 32 columns load from TMEM while this chunk
// is converted.
__device__ __forceinline__ void relu_epilogue(uint32_t tl, unsigned char* tile, int row) {
  uint32_t rb[2][32];
  tc::tmem_ld32_issue(tl, rb[0]);
#pragma unroll
  for (int ch = 0; ch < 4; ++ch) {
    tc::tmem_wait_ld(rb[ch & 1]);
    if (ch < 3) tc::tmem_ld32_issue(tl + (ch + 1) * 32, rb[(ch + 1) & 1]);
    const float* v = reinterpret_cast<const float*>(rb[ch & 1]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint4 w;
      uint32_t* wp = reinterpret_cast<uint32_t*>(&w);
#pragma unroll
      for (int e = 0; e < 4; ++e) wp[e] = tc::pack2_relu(v[q * 8 + 2 * e], v[q * 8 + 2 * e + 1]);
      *reinterpret_cast<uint4*>(tile + tc::core_off(row, ch * 32 + q * 8, HID)) = w;
    }
  }
}

template <int KP>
__global__ void __launch_bounds__(128) mlp_forward_kernel(const float* __restrict__ P, int nfeat,
                                                          const float* __restrict__ X, int64_t n,
                                                          float* __restrict__ score,
                                                          int* status) {
  using L = FwdL<KP>;
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char *sW1 = sm + L::W1, *sW2 = sm + L::W2, *sX = sm + L::X, *sA1 = sm + L::A1;
  float* vec = reinterpret_cast<float*>(sm + L::VEC);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::BAR);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + L::SLOT);
  const int tid = threadIdx.x, warp = tid >> 5;
  if (status[ST_CODE] != DEV_OK) return;
  if (warp == 0) tc::tmem_alloc(slot, 128);
  load_weights<KP>(P, nfeat, sW1, sW2, vec, true);
  // indicator rows: ones in the b2 columns of W1's tile; the descriptor
  // repeats these 8 rows over all 128 (row-group stride 0)
  unsigned char* sI = sm + L::IND;
  for (int c = tid; c < 8 * (KP / 8); c += blockDim.x) {
    const int r = c % 8, q = c / 8;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int f = q * 8 + e - nfeat;
      v[e] = f >= 3 && f < 6 ? 1.f : 0.f;
    }
    *reinterpret_cast<uint4*>(sI + tc::core_off(r, q * 8, KP)) = tc::pack8(v);
  }
  const float b3 = P[mlp_param_count(nfeat) - 1];
  if (tid == 0) tc::bar_init(bar);
  mma_sync_point();
  const uint32_t tmem = *slot;
  const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
  constexpr uint32_t id = tc::idesc_bf16(128, 128, false, false);
  const uint32_t aX = tc::sa(sX), aW1 = tc::sa(sW1), aA1 = tc::sa(sA1), aW2 = tc::sa(sW2);
  const uint32_t aI = tc::sa(sI);
  uint32_t phase = 0;
  bool ok = true;
  const int64_t ntiles = (n + HID - 1) / HID;
  XChunks<KP> xc;
  if (blockIdx.x < ntiles) load_x<KP>(X, n, (int64_t)blockIdx.x * HID, nfeat, xc);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * HID;
    store_x<KP>(xc, sX);
    // the next tile's features load while this one is in flight
    if (tile + gridDim.x < ntiles) load_x<KP>(X, n, (tile + gridDim.x) * HID, nfeat, xc);
    mma_sync_point();
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < KP / 16; ++ks)
        tc::mma_bf16(tmem, tc::sdesc(aX + ks * 256, 128, (KP / 8) * 128),
                     tc::sdesc(aW1 + ks * 256, 128, (KP / 8) * 128), id, ks > 0);
      tc::mma_commit(bar);
    }
    ok = __syncthreads_and(tc::bar_wait(bar, phase));
    phase ^= 1u;
    if (!ok) break;
    tc::fence_after();
    // A1 = bf16(relu(Z1)) into its operand tile (b1 came with the MMA)
    relu_epilogue(tl, sA1, tid);
    mma_sync_point();
    if (tid == 0) {
      // Z2 = b2 (indicator rows x W1's tile), then += A1 W2^T
#pragma unroll
      for (int ks = 0; ks < KP / 16; ++ks)
        tc::mma_bf16(tmem, tc::sdesc(aI + ks * 256, 128, 0),
                     tc::sdesc(aW1 + ks * 256, 128, (KP / 8) * 128), id, ks > 0);
#pragma unroll
      for (int ks = 0; ks < HID / 16; ++ks)
        tc::mma_bf16(tmem, tc::sdesc(aA1 + ks * 256, 128, 2048),
                     tc::sdesc(aW2 + ks * 256, 128, 2048), id, 1);
      tc::mma_commit(bar);
    }
    ok = __syncthreads_and(tc::bar_wait(bar, phase));
    phase ^= 1u;
    if (!ok) break;
    tc::fence_after();
    // s = A2 . w3 + b3 with A2 = bf16(relu(Z2)): ReLU and rounding in one
    // conversion per pair, FP32 accumulation of the even and the odd columns
    // in the two halves of a packed pair
    uint64_t s2 = 0ull;
    {
      uint32_t rb[2][32];
      tc::tmem_ld32_issue(tl, rb[0]);
#pragma unroll
      for (int ch = 0; ch < 4; ++ch) {
        tc::tmem_wait_ld(rb[ch & 1]);
        if (ch < 3) tc::tmem_ld32_issue(tl + (ch + 1) * 32, rb[(ch + 1) & 1]);
        const float* v = reinterpret_cast<const float*>(rb[ch & 1]);
        const ulonglong2* wq = reinterpret_cast<const ulonglong2*>(vec + 2 * HID + ch * 32);
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
          const ulonglong2 w = wq[j / 4];  // a 16-byte broadcast load: two w3 pairs
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const uint32_t a2 = tc::pack2_relu(v[j + 2 * e], v[j + 2 * e + 1]);
            s2 = tc::fma2(tc::pk(tc::bf16_lo(a2), tc::bf16_hi(a2)), e ? w.y : w.x, s2);
          }
        }
      }
    }
    const float s = tc::pk_sum(s2);
    if (r0 + tid < n) score[r0 + tid] = s + b3;
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
  }
  if (!ok && tid == 0) atomicCAS(&status[ST_CODE], DEV_OK, DEV_TIMEOUT);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, 128);
}

template <int KP>
__global__ void __launch_bounds__(128, 1) mlp_grad_kernel(const float* __restrict__ P, int nfeat,
                                                          const float* __restrict__ X,
                                                          const float* __restrict__ target,
                                                          RowMap map, int64_t n,
                                                          float* __restrict__ partial,
                                                          int* status) {
  using L = GradL<KP>;
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char *sW1 = sm + L::W1, *sW2 = sm + L::W2, *sX = sm + L::X, *sA1 = sm + L::A1;
  unsigned char *sD2 = sm + L::DZ2, *sD1 = sm + L::DZ1;
  float* vec = reinterpret_cast<float*>(sm + L::VEC);
  float* red = reinterpret_cast<float*>(sm + L::RED);
  float* scal = reinterpret_cast<float*>(sm + L::SCAL);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::BAR);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + L::SLOT);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (status[ST_CODE] != DEV_OK) return;
  if (warp == 0) tc::tmem_alloc(slot, 512);
  load_weights<KP>(P, nfeat, sW1, sW2, vec);
  const float b3 = P[mlp_param_count(nfeat) - 1];
  if (tid == 0) tc::bar_init(bar);
  mma_sync_point();
  const uint32_t tmem = *slot;
  const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
  constexpr uint32_t idKK = tc::idesc_bf16(128, 128, false, false);
  constexpr uint32_t idKM = tc::idesc_bf16(128, 128, false, true);
  constexpr uint32_t idMM = tc::idesc_bf16(128, 128, true, true);
  constexpr uint32_t idW1 = tc::idesc_bf16(128, KP, true, true);
  constexpr uint32_t XKS = (KP / 8) * 128;  // X tile: core stride along its rows
  const uint32_t aX = tc::sa(sX), aW1 = tc::sa(sW1), aA1 = tc::sa(sA1), aW2 = tc::sa(sW2);
  const uint32_t aD2 = tc::sa(sD2), aD1 = tc::sa(sD1);
  const float inv_n2 = 2.0f / (float)n;
  float acc_w3[4] = {0, 0, 0, 0}, acc_b2[4] = {0, 0, 0, 0}, acc_b1[4] = {0, 0, 0, 0};
  float acc_b3 = 0.f, acc_loss = 0.f;
  uint32_t phase = 0;
  bool ok = true, first = true;
  const int64_t ntiles = (n + HID - 1) / HID;
  auto wait_mma = [&]() -> bool {
    const bool r = __syncthreads_and(tc::bar_wait(bar, phase));
    phase ^= 1u;
    tc::fence_after();
    return r;
  };
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * HID;
    const bool valid = r0 + tid < n;
    const float tgt = valid ? target[map(r0 + tid)] : 0.f;
    stage_x<KP>(X, map, n, r0, nfeat, sX);
    mma_sync_point();
    // ---- Z1 = X W1^T
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < KP / 16; ++ks)
        tc::mma_bf16(tmem, tc::sdesc(aX + ks * 256, 128, XKS), tc::sdesc(aW1 + ks * 256, 128, XKS),
                     idKK, ks > 0);
      tc::mma_commit(bar);
    }
    if (!(ok = wait_mma())) break;
    uint32_t mask1[4];
#pragma unroll 1
    for (int ch = 0; ch < 4; ++ch) {
      float v[32];
      tc::tmem_ld32(tl + ch * 32, v);
      uint32_t m = 0;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const float z = v[j] + vec[ch * 32 + j];
        m |= (z > 0.f ? 1u : 0u) << j;
        v[j] = fmaxf(z, 0.f);
      }
      mask1[ch] = m;
      store_row(sA1, tid, ch * 32, v);
    }
    mma_sync_point();
    // ---- Z2 = A1 W2^T (columns 128..255)
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < HID / 16; ++ks)
        tc::mma_bf16(tmem + 128, tc::sdesc(aA1 + ks * 256, 128, 2048),
                     tc::sdesc(aW2 + ks * 256, 128, 2048), idKK, ks > 0);
      tc::mma_commit(bar);
    }
    if (!(ok = wait_mma())) break;
    float s = 0.f;
#pragma unroll 1
    for (int ch = 0; ch < 4; ++ch) {
      float v[32];
      tc::tmem_ld32(tl + 128 + ch * 32, v);
#pragma unroll
      for (int j = 0; j < 32; ++j)
        s = fmaf(tc::bf16_round(fmaxf(v[j] + vec[HID + ch * 32 + j], 0.f)),
                 vec[2 * HID + ch * 32 + j], s);
    }
    const float r = s + b3 - tgt;
    const float ds = valid ? r * inv_n2 : 0.f;
    acc_loss += valid ? r * r : 0.f;
    acc_b3 += ds;
#pragma unroll 1
    for (int ch = 0; ch < 4; ++ch) {
      float v[32], g3[32];
      tc::tmem_ld32(tl + 128 + ch * 32, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const float z = v[j] + vec[HID + ch * 32 + j];
        g3[j] = tc::bf16_round(fmaxf(z, 0.f)) * ds;
        v[j] = z > 0.f ? ds * vec[2 * HID + ch * 32 + j] : 0.f;  // dZ2
      }
      store_row(sD2, tid, ch * 32, v);
      acc_b2[ch] += transpose_reduce(v, lane);
      acc_w3[ch] += transpose_reduce(g3, lane);
    }
    mma_sync_point();
    // ---- dA1 = dZ2 W2 (columns 0..127), g_W2 += dZ2^T A1 (columns 256..383)
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < HID / 16; ++ks)
        tc::mma_bf16(tmem, tc::sdesc(aD2 + ks * 256, 128, 2048),
                     tc::sdesc(aW2 + ks * 4096, 2048, 128), idKM, ks > 0);
#pragma unroll
      for (int ks = 0; ks < HID / 16; ++ks)
        tc::mma_bf16(tmem + 256, tc::sdesc(aD2 + ks * 4096, 2048, 128),
                     tc::sdesc(aA1 + ks * 4096, 2048, 128), idMM, (!first || ks > 0) ? 1u : 0u);
      tc::mma_commit(bar);
    }
    if (!(ok = wait_mma())) break;
#pragma unroll 1
    for (int ch = 0; ch < 4; ++ch) {
      float v[32];
      tc::tmem_ld32(tl + ch * 32, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = (mask1[ch] >> j) & 1u ? v[j] : 0.f;  // dZ1
      store_row(sD1, tid, ch * 32, v);
      acc_b1[ch] += transpose_reduce(v, lane);
    }
    mma_sync_point();
    // ---- g_W1 += dZ1^T X (columns 384..)
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < HID / 16; ++ks)
        tc::mma_bf16(tmem + 384, tc::sdesc(aD1 + ks * 4096, 2048, 128),
                     tc::sdesc(aX + ks * 2 * XKS, XKS, 128), idW1, (!first || ks > 0) ? 1u : 0u);
      tc::mma_commit(bar);
    }
    if (!(ok = wait_mma())) break;
    first = false;
  }
  // ---- this CTA's partial gradient
  const int64_t PC = mlp_param_count(nfeat);
  float* out = partial + (size_t)blockIdx.x * (PC + 1);
  float* oW1 = out;
  float* ob1 = out + HID * nfeat;
  float* oW2 = ob1 + HID;
  float* ob2 = oW2 + HID * HID;
  float* ow3 = ob2 + HID;
  if (ok) {
#pragma unroll 1
    for (int ch = 0; ch < 4; ++ch) {
      float v[32];
      if (!first) tc::tmem_ld32(tl + 256 + ch * 32, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) oW2[tid * HID + ch * 32 + j] = first ? 0.f : v[j];
    }
    float v[32];
    if (!first) tc::tmem_ld32(tl + 384, v);
    for (int k = 0; k < nfeat; ++k) oW1[tid * nfeat + k] = first ? 0.f : v[k];
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
      red[(warp * 3 + 0) * HID + ch * 32 + lane] = acc_b1[ch];
      red[(warp * 3 + 1) * HID + ch * 32 + lane] = acc_b2[ch];
      red[(warp * 3 + 2) * HID + ch * 32 + lane] = acc_w3[ch];
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      acc_b3 += __shfl_xor_sync(0xffffffffu, acc_b3, o);
      acc_loss += __shfl_xor_sync(0xffffffffu, acc_loss, o);
    }
    if (lane == 0) {
      scal[warp * 2] = acc_b3;
      scal[warp * 2 + 1] = acc_loss;
    }
  }
  __syncthreads();
  if (ok) {
    float b1s = 0.f, b2s = 0.f, w3s = 0.f;
    for (int w = 0; w < 4; ++w) {
      b1s += red[(w * 3 + 0) * HID + tid];
      b2s += red[(w * 3 + 1) * HID + tid];
      w3s += red[(w * 3 + 2) * HID + tid];
    }
    ob1[tid] = b1s;
    ob2[tid] = b2s;
    ow3[tid] = w3s;
    if (tid == 0) {
      out[PC - 1] = scal[0] + scal[2] + scal[4] + scal[6];
      out[PC] = scal[1] + scal[3] + scal[5] + scal[7];
    }
  } else if (tid == 0) {
    atomicCAS(&status[ST_CODE], DEV_OK, DEV_TIMEOUT);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, 512);
}

__global__ void __launch_bounds__(256) mlp_reduce_adam_kernel(
    float* __restrict__ params, float* __restrict__ m, float* __restrict__ v,
    const float* __restrict__ partial, int grid, int64_t PC, int64_t n, float* __restrict__ grad,
    float* __restrict__ loss, int adam, float lr, float beta1, float beta2, float eps, float c1,
    float c2) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p <= PC; p += stride) {
    float g = 0.f;
    for (int c = 0; c < grid; ++c) g += partial[(size_t)c * (PC + 1) + p];
    if (p == PC) {
      if (loss) *loss = g / (float)n;
      continue;
    }
    if (grad) grad[p] = g;
    if (adam) {
      const float mm = beta1 * m[p] + (1.f - beta1) * g;
      const float vv = beta2 * v[p] + (1.f - beta2) * g * g;
      m[p] = mm;
      v[p] = vv;
      params[p] -= lr * (mm * c1) / (sqrtf(vv * c2) + eps);
    }
  }
}

template <typename Kern>
int set_smem(Kern k, int bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) ==
                 cudaSuccess
             ? 0
             : -1;
}

}  // namespace

int launch_mlp_forward(const float* params, int nfeat, const float* X, int64_t n, float* score,
                       int* status, int num_sms, cudaStream_t s) {
  if (n <= 0) return 0;
  if (nfeat < 1 || nfeat > kMlpMaxFeat) return -1;
  const int64_t ntiles = (n + HID - 1) / HID;
  // three CTAs per SM (128 TMEM columns each) so one CTA's epilogue overlaps
  // another's MMA
  const int64_t grid = ntiles < 3 * (int64_t)num_sms ? ntiles : 3 * (int64_t)num_sms;
  if (nfeat + 6 <= 16) {  // the biases take six columns of W1's tile
    static int once = set_smem(mlp_forward_kernel<16>, FwdL<16>::BYTES);
    if (once) return -1;
    mlp_forward_kernel<16><<<(unsigned)grid, 128, FwdL<16>::BYTES, s>>>(params, nfeat, X, n,
                                                                        score, status);
  } else {
    static int once = set_smem(mlp_forward_kernel<32>, FwdL<32>::BYTES);
    if (once) return -1;
    mlp_forward_kernel<32><<<(unsigned)grid, 128, FwdL<32>::BYTES, s>>>(params, nfeat, X, n,
                                                                        score, status);
  }
  return 1;
}

int launch_mlp_grad(const float* params, int nfeat, const float* X, const float* target,
                    const int64_t* idx, uint64_t sample_key, int64_t rows, int64_t n,
                    float* partial, int max_grid, int* status, int num_sms, cudaStream_t s) {
  if (n <= 0 || rows <= 0 || nfeat < 1 || nfeat > kMlpMaxFeat || max_grid < 1) return -1;
  const RowMap map{idx, sample_key, rows};
  const int64_t ntiles = (n + HID - 1) / HID;
  int64_t grid = ntiles < num_sms ? ntiles : num_sms;
  if (grid > max_grid) grid = max_grid;
  if (nfeat <= 16) {
    static int once = set_smem(mlp_grad_kernel<16>, GradL<16>::BYTES);
    if (once) return -1;
    mlp_grad_kernel<16><<<(unsigned)grid, 128, GradL<16>::BYTES, s>>>(params, nfeat, X, target,
                                                                      map, n, partial, status);
  } else {
    static int once = set_smem(mlp_grad_kernel<32>, GradL<32>::BYTES);
    if (once) return -1;
    mlp_grad_kernel<32><<<(unsigned)grid, 128, GradL<32>::BYTES, s>>>(params, nfeat, X, target,
                                                                      map, n, partial, status);
  }
  return (int)grid;
}

void launch_mlp_reduce_adam(float* params, float* m, float* v, const float* partial, int grid,
                            int nfeat, int64_t n, float* grad, float* loss, int adam, float lr,
                            float beta1, float beta2, float eps, int step, cudaStream_t s) {
  const int64_t PC = mlp_param_count(nfeat);
  const float c1 = 1.f / (1.f - powf(beta1, (float)step));
  const float c2 = 1.f / (1.f - powf(beta2, (float)step));
  mlp_reduce_adam_kernel<<<(unsigned)((PC + 256) / 256), 256, 0, s>>>(
      params, m, v, partial, grid, PC, n, grad, loss, adam, lr, beta1, beta2, eps, c1, c2);
}

}  // namespace ftp
