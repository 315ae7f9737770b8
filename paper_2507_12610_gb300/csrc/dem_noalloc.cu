// dem_contact_forces_noalloc: contact force and torque sums of a particle
// state with no friction history, computed without allocating any memory.
//
// Its scratch (cell keys, arrival slots, cell counts and offsets, the sorted
// order) lives in one file-scope device array of fixed size, so the call needs
// neither cudaMalloc nor any other allocator.  Host code only ever sees that
// array's name as a host-side stand-in, never a device address: the device
// address is obtained once per device with cudaGetSymbolAddress and passed to
// the kernels.
//
// The arithmetic is the same as the FP64 step of the library for a first
// step (zero springs, particle pairs only, partners summed in ascending index),
// and this file is compiled without multiply-add contraction like that step.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "dem_internal.cuh"
#include "dem_law.cuh"
#include "dem_math.cuh"

namespace dem {
namespace {

constexpr int64_t kNoAllocMaxParticles = 131072;  // 2^17
constexpr int64_t kNoAllocMaxCells = 262144;      // 2^18
constexpr int kTile = 4096;                       // scan tile (elements per block)
constexpr int64_t kMaxTiles = kNoAllocMaxCells / kTile + 1;
constexpr int kMaxTouching = 64;                  // touching partners per particle
constexpr uint32_t kMaxPerCell = 64;              // particles per grid cell

// scratch layout (u32 words)
constexpr int64_t kOffKey = 0;
constexpr int64_t kOffLocal = kOffKey + kNoAllocMaxParticles;
constexpr int64_t kOffOrder = kOffLocal + kNoAllocMaxParticles;
constexpr int64_t kOffCount = kOffOrder + kNoAllocMaxParticles;
constexpr int64_t kOffStart = kOffCount + kNoAllocMaxCells;
constexpr int64_t kOffTiles = kOffStart + kNoAllocMaxCells + 1;
constexpr int64_t kOffStatus = kOffTiles + kMaxTiles + 1;
constexpr int64_t kScratchWords = kOffStatus + 1;

// ~3.5 MB, held by every device that loads the library until the process exits
__device__ __align__(256) uint32_t g_noalloc_scratch[kScratchWords];

struct Grid {
  double lo[3], hi[3];
  double inv_h;
  int32_t nc[3];
  int32_t ncells;
};

__device__ __forceinline__ uint32_t cell_of(const Grid& g, double x, double y, double z) {
  int c[3];
  const double p[3] = {x, y, z};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double f = floor((p[a] - g.lo[a]) * g.inv_h);
    int ci = f < 0.0 ? 0 : (f >= (double)g.nc[a] ? g.nc[a] - 1 : (int)f);
    c[a] = ci;
  }
  return (uint32_t)((c[2] * g.nc[1] + c[1]) * g.nc[0] + c[0]);
}

__global__ void na_clear(uint32_t* s, int64_t ncells) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ncells;
       i += (int64_t)gridDim.x * blockDim.x)
    s[kOffCount + i] = 0u;
  if (blockIdx.x == 0 && threadIdx.x == 0) s[kOffStatus] = 0u;
}

__device__ __forceinline__ void na_fail(uint32_t* s, uint32_t code) {
  atomicCAS(&s[kOffStatus], 0u, code);
}

// Cell of each particle.  A radius outside (0, r_max], a non-finite or
// out-of-domain position (DEM_ERR_INVALID) or a cell holding more than
// kMaxPerCell particles (DEM_ERR_CAPACITY) sets the status word; the later
// kernels then return at once, so a wrong domain or radius bound cannot make
// the call walk one crowded cell for a long time.
__global__ void na_bin(uint32_t* s, Grid g, const double* R, const double* x, int64_t n,
                       double r_max) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double px = x[3 * i], py = x[3 * i + 1], pz = x[3 * i + 2], r = R[i];
  const double p3[3] = {px, py, pz};
  bool ok = r > 0.0 && r <= r_max;
#pragma unroll
  for (int a = 0; a < 3; ++a) ok = ok && p3[a] >= g.lo[a] && p3[a] <= g.hi[a];  // false for NaN
  uint32_t c = 0;
  if (ok) {
    c = cell_of(g, px, py, pz);
    const uint32_t k = atomicAdd(&s[kOffCount + c], 1u);
    if (k >= kMaxPerCell) na_fail(s, (uint32_t)DEM_ERR_CAPACITY);
    s[kOffLocal + i] = k;
  } else {
    na_fail(s, (uint32_t)DEM_ERR_INVALID);
    s[kOffLocal + i] = 0u;
  }
  s[kOffKey + i] = c;
}

// Exclusive scan of the cell counts: tile totals (one block per tile of
// kTile cells), an exclusive scan of the totals (one warp), then every tile
// scanned in shared memory (256 threads, kTile / 256 consecutive cells each).
// The result is the same whatever the launch shape (integer sums).
constexpr int kScanThreads = 256;
constexpr int kPerThread = kTile / kScanThreads;

__device__ __forceinline__ uint32_t warp_excl_scan(uint32_t v, uint32_t& total) {
  const int lane = threadIdx.x & 31;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  total = __shfl_sync(0xffffffffu, incl, 31);
  return incl - v;
}

__global__ void __launch_bounds__(kScanThreads) na_scan_tiles(uint32_t* s, int64_t ncells) {
  __shared__ uint32_t part[kScanThreads];
  const int64_t base = (int64_t)blockIdx.x * kTile;
  uint32_t sum = 0;
  for (int k = threadIdx.x; k < kTile; k += blockDim.x) {
    const int64_t i = base + k;
    if (i < ncells) sum += s[kOffCount + i];
  }
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) s[kOffTiles + blockIdx.x] = part[0];
}

// one warp: exclusive scan of the tile totals, 32 at a time with a carry
__global__ void na_scan_top(uint32_t* s, int64_t ntiles) {
  uint32_t carry = 0;
  for (int64_t t0 = 0; t0 < ntiles; t0 += 32) {
    const int64_t t = t0 + threadIdx.x;
    const uint32_t v = t < ntiles ? s[kOffTiles + t] : 0u;
    uint32_t total;
    const uint32_t ex = warp_excl_scan(v, total);
    if (t < ntiles) s[kOffTiles + t] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) s[kOffTiles + ntiles] = carry;
}

__global__ void __launch_bounds__(kScanThreads) na_scan_down(uint32_t* s, int64_t ncells,
                                                             int64_t ntiles) {
  __shared__ uint32_t wsum[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kPerThread;
  uint32_t v[kPerThread];
  uint32_t mine = 0;
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    v[k] = base + k < ncells ? s[kOffCount + base + k] : 0u;
    mine += v[k];
  }
  // exclusive prefix of the threads' sums within the block
  uint32_t wtotal;
  const uint32_t ex = warp_excl_scan(mine, wtotal);
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) wsum[warp] = wtotal;
  __syncthreads();
  uint32_t before = 0;
  for (int k = 0; k < warp; ++k) before += wsum[k];
  uint32_t acc = s[kOffTiles + blockIdx.x] + before + ex;
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    if (base + k < ncells) s[kOffStart + base + k] = acc;
    acc += v[k];
  }
  if (blockIdx.x == ntiles - 1 && threadIdx.x == 0) s[kOffStart + ncells] = s[kOffTiles + ntiles];
}

__global__ void na_scatter(uint32_t* s, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || s[kOffStatus] != 0u) return;
  s[kOffOrder + s[kOffStart + s[kOffKey + i]] + s[kOffLocal + i]] = (uint32_t)i;
}

// within a cell, ascending particle index
__global__ void na_cell_sort(uint32_t* s, int64_t ncells) {
  if (s[kOffStatus] != 0u) return;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncells;
       c += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t a = s[kOffStart + c], b = s[kOffStart + c + 1];
    uint32_t* o = s + kOffOrder;
    for (uint32_t i = a + 1; i < b; ++i) {
      const uint32_t v = o[i];
      uint32_t j = i;
      while (j > a && o[j - 1] > v) {
        o[j] = o[j - 1];
        --j;
      }
      o[j] = v;
    }
  }
}

struct ForceArgs {
  const double* R;
  const double* x;
  const double* v;
  const double* w;
  double* F;
  double* T;
  int64_t n;
  double rho;
  LawConst<double> c;
};

__device__ __forceinline__ V3<double> ld3(const double* a, int64_t i) {
  return mk(a[3 * i], a[3 * i + 1], a[3 * i + 2]);
}

// One thread per particle: touching partners from the 27 cells, sorted by
// index, each pair evaluated in canonical orientation with zero springs.
__global__ void __launch_bounds__(128) na_forces(uint32_t* s, Grid g, ForceArgs a) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.n || s[kOffStatus] != 0u) return;
  const double Rt = a.R[t];
  const uint32_t ct = s[kOffKey + t];
  const int cx = (int)(ct % (uint32_t)g.nc[0]);
  const int cy = (int)((ct / (uint32_t)g.nc[0]) % (uint32_t)g.nc[1]);
  const int cz = (int)(ct / ((uint32_t)g.nc[0] * (uint32_t)g.nc[1]));
  uint32_t touch[kMaxTouching];
  int nt = 0;
  bool over = false;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int x0 = cx + dx, y0 = cy + dy, z0 = cz + dz;
        if (x0 < 0 || y0 < 0 || z0 < 0 || x0 >= g.nc[0] || y0 >= g.nc[1] || z0 >= g.nc[2])
          continue;
        const uint32_t c = (uint32_t)((z0 * g.nc[1] + y0) * g.nc[0] + x0);
        for (uint32_t k = s[kOffStart + c]; k < s[kOffStart + c + 1]; ++k) {
          const uint32_t u = s[kOffOrder + k];
          if ((int64_t)u == t) continue;
          const int64_t lo = t < (int64_t)u ? t : (int64_t)u, hi = t < (int64_t)u ? (int64_t)u : t;
          const V3<double> d = ld3(a.x, lo) - ld3(a.x, hi);
          const double S = a.R[lo] + a.R[hi];
          const double d2 = dot(d, d);
          if (d2 > S * S * (1.0 + 1e-10)) continue;
          const double dist = sqrt(d2);
          if (S - dist < 0.0 || !(dist > 0.0)) continue;
          if (nt < kMaxTouching) {
            int j = nt++;
            while (j > 0 && touch[j - 1] > u) {
              touch[j] = touch[j - 1];
              --j;
            }
            touch[j] = u;
          } else {
            over = true;
          }
        }
      }
  if (over) atomicCAS(&s[kOffStatus], 0u, (uint32_t)DEM_ERR_CAPACITY);
  V3<double> F = mk(0.0, 0.0, 0.0), T = mk(0.0, 0.0, 0.0);
  const double mt = 4.0 / 3.0 * M_PI * a.rho * Rt * Rt * Rt;
  for (int k = 0; k < nt; ++k) {
    const int64_t u = touch[k];
    const bool t_is_i = t < u;
    const int64_t i = t_is_i ? t : u, j = t_is_i ? u : t;
    const V3<double> d = ld3(a.x, i) - ld3(a.x, j);
    const double Ri = a.R[i], Rj = a.R[j];
    const double S = Ri + Rj;
    const double dist = sqrt(dot(d, d));
    const double delta = S - dist;
    const V3<double> nh = (1.0 / dist) * d;
    const double mu_ = 4.0 / 3.0 * M_PI * a.rho * a.R[u] * a.R[u] * a.R[u];
    const double mi = t_is_i ? mt : mu_, mj = t_is_i ? mu_ : mt;
    const double Rs = 1.0 / (1.0 / Ri + 1.0 / Rj);
    const double ms = 1.0 / (1.0 / mi + 1.0 / mj);
    const double ri = Ri - delta / 2.0, rj = Rj - delta / 2.0;
    const V3<double> wi = ld3(a.w, i), wj = ld3(a.w, j);
    V3<double> us = mk(0.0, 0.0, 0.0), ur = us;
    double ut = 0.0;
    const LawOut<double> o =
        contact_law(a.c, nh, delta, Rs, ms, ri, rj, 1.0 / (1.0 / ri + 1.0 / rj),
                    ld3(a.v, i) - ld3(a.v, j), ri * wi + rj * wj, wi - wj, us, ur, ut);
    if (t_is_i) {
      F = F + o.f;
      T = T + o.ti;
    } else {
      F = F - o.f;
      T = T + o.tj;
    }
  }
  a.F[3 * t] = F.x; a.F[3 * t + 1] = F.y; a.F[3 * t + 2] = F.z;
  a.T[3 * t] = T.x; a.T[3 * t + 1] = T.y; a.T[3 * t + 2] = T.z;
}

std::mutex g_setup_mutex;
constexpr int kMaxDevices = 64;
uint32_t* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set-up on the
// first call per device).
int scratch_for_current_device(uint32_t** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return DEM_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return DEM_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_scratch_ptr[dev];
  return DEM_OK;
}

double beta_host(double e_n) {
  if (e_n <= 0.0) return 1.0;
  if (e_n >= 1.0) return 0.0;
  const double l = std::log(e_n);
  const double r = M_PI / l;
  return 1.0 / std::sqrt(1.0 + r * r);
}

}  // namespace
}  // namespace dem

using namespace dem;

extern "C" int dem_contact_forces_noalloc(const dem_params* params, int64_t n, double r_max,
                                          const double* R, const double* x, const double* v,
                                          const double* w, double* F, double* T,
                                          void* stream) {
  if (!params || !R || !x || !v || !w || !F || !T) return DEM_ERR_INVALID;
  if (n < 1 || n > kNoAllocMaxParticles) return DEM_ERR_INVALID;
  if (!(r_max > 0) || !std::isfinite(r_max)) return DEM_ERR_INVALID;
  const double E = params->E, nu = params->nu;
  if (!(E > 0) || !(nu > -1.0 && nu <= 0.5) || !(params->rho > 0) || !(params->e_n >= 0) ||
      !(params->e_n <= 1) || params->mu_s < 0 || params->mu_r < 0 || params->mu_t < 0 ||
      !(params->dt > 0))
    return DEM_ERR_INVALID;
  Grid g{};
  const double h = 2.0 * r_max;
  int64_t ncells = 1;
  for (int a = 0; a < 3; ++a) {
    const double lo = params->domain_lo[a], hi = params->domain_hi[a];
    if (!(lo < hi) || !std::isfinite(lo) || !std::isfinite(hi)) return DEM_ERR_INVALID;
    const double c = std::ceil((hi - lo) / h);
    if (!(c >= 1) || c > (double)kNoAllocMaxCells) return DEM_ERR_INVALID;
    g.lo[a] = lo;
    g.hi[a] = hi;
    g.nc[a] = (int32_t)c;
    ncells *= (int64_t)c;
    if (ncells > kNoAllocMaxCells) return DEM_ERR_INVALID;
  }
  g.inv_h = 1.0 / h;
  g.ncells = (int32_t)ncells;
  uint32_t* s = nullptr;
  int rc = scratch_for_current_device(&s);
  if (rc != DEM_OK) return rc;
  ForceArgs fa;
  fa.R = R; fa.x = x; fa.v = v; fa.w = w; fa.F = F; fa.T = T; fa.n = n;
  fa.rho = params->rho;
  const double G = E / (2.0 * (1.0 + nu));
  fa.c = LawConst<double>{1.0 / ((1.0 - nu * nu) / E + (1.0 - nu * nu) / E),
                          1.0 / ((2.0 - nu) / G + (2.0 - nu) / G), beta_host(params->e_n),
                          params->mu_s, params->mu_r, params->mu_t, params->dt, 0.0};
  fa.c.cs_cn = std::sqrt(fa.c.Gs / (5.0 * fa.c.Es));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t ntiles = (ncells + kTile - 1) / kTile;
  const unsigned nb = (unsigned)((n + 127) / 128);
  na_clear<<<(unsigned)std::min<int64_t>((ncells + 255) / 256, 1024), 256, 0, st>>>(s, ncells);
  na_bin<<<nb, 128, 0, st>>>(s, g, R, x, n, r_max);
  na_scan_tiles<<<(unsigned)ntiles, kScanThreads, 0, st>>>(s, ncells);
  na_scan_top<<<1, 32, 0, st>>>(s, ntiles);
  na_scan_down<<<(unsigned)ntiles, kScanThreads, 0, st>>>(s, ncells, ntiles);
  na_scatter<<<nb, 128, 0, st>>>(s, n);
  na_cell_sort<<<(unsigned)std::min<int64_t>((ncells + 255) / 256, 1024), 256, 0, st>>>(s,
                                                                                      ncells);
  na_forces<<<nb, 128, 0, st>>>(s, g, fa);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return DEM_ERR_CUDA;
  uint32_t status = 0;
  if (cudaMemcpyAsync(&status, s + kOffStatus, sizeof status, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return DEM_ERR_CUDA;
  }
  return (int)status;
}
