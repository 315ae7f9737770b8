// Exclusive prefix sum of a u32 array: per-block totals, a single-block scan
// of the totals, then a per-block scan that adds its offset.  Integer and
// order-fixed, so the result is exact and deterministic.  All three kernels
// return at once unless the control block says the lists are being rebuilt.
#include "dem_internal.cuh"

namespace dem {

namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;  // per thread
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_tot,
                                                         uint32_t* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    uint32_t w = lane < nw ? warp_tot[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < nw) warp_tot[lane] = wi - w;
    if (lane == nw - 1) *total = wi;
  }
  __syncthreads();
  return incl - v + warp_tot[wid];
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_reduce(const Ctl* ctl, const uint32_t* in, int64_t n, uint32_t* block_sums) {
  if (!ctl->rebuild || ctl->status) return;
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t total;
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
    if (i < n) s += in[i];
  }
  block_exclusive_scan(s, warp_tot, &total);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_partials(const Ctl* ctl, uint32_t* block_sums, int64_t nblocks) {
  if (!ctl->rebuild || ctl->status) return;
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t total;
  uint32_t carry = 0;
  for (int64_t b0 = 0; b0 < nblocks; b0 += kScanThreads) {
    int64_t i = b0 + threadIdx.x;
    uint32_t v = i < nblocks ? block_sums[i] : 0u;
    uint32_t ex = block_exclusive_scan(v, warp_tot, &total);
    if (i < nblocks) block_sums[i] = carry + ex;
    __syncthreads();
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) block_sums[nblocks] = carry;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_down(const Ctl* ctl, const uint32_t* in, uint32_t* out, int64_t n,
            const uint32_t* block_sums, int64_t nblocks) {
  if (!ctl->rebuild || ctl->status) return;
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t total;
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
    v[k] = i < n ? in[i] : 0u;
    s += v[k];
  }
  uint32_t ex = block_exclusive_scan(s, warp_tot, &total) + block_sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
    if (i < n) out[i] = ex;
    ex += v[k];
  }
  if (blockIdx.x == nblocks - 1 && threadIdx.x == 0) out[n] = block_sums[nblocks];
}

}  // namespace

int64_t scan_block_sums_size(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

// out has n + 1 entries; out[n] is the total.
void launch_scan(cudaStream_t st, const Ctl* ctl, const uint32_t* in, uint32_t* out, int64_t n,
                 uint32_t* block_sums) {
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, st>>>(ctl, in, n, block_sums);
  k_scan_partials<<<1, kScanThreads, 0, st>>>(ctl, block_sums, nb);
  k_scan_down<<<(unsigned)nb, kScanThreads, 0, st>>>(ctl, in, out, n, block_sums, nb);
}

}  // namespace dem
