// Kernels of the message-passing surrogate (declared in include/mpnn.h).
//
// Dense layers run on the tensor cores through mma.sync m16n8k16 with bf16
// operands and fp32 accumulation; graph gathers and segment sums follow a
// CSR order, so every sum is taken in a fixed order and results do not depend
// on thread scheduling (no floating-point atomics).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/dem.h"
#include "../../include/mpnn.h"

namespace {

int launch_status() {
  return cudaGetLastError() == cudaSuccess ? DEM_OK : DEM_ERR_CUDA;
}

__device__ __forceinline__ uint32_t ld_pair(const uint16_t* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

__device__ __forceinline__ uint16_t to_bf16(float x) {
  const __nv_bfloat16 b = __float2bfloat16_rn(x);
  return *reinterpret_cast<const uint16_t*>(&b);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// One 64 x 64 output tile per block of 4 warps; warp w owns rows
// 32 (w / 2) .. +32 and columns 32 (w % 2) .. +32: 2 x 4 tiles of 16 x 8.
// Fragments come straight from global memory (32-bit pairs; the operands of
// these layers are small and stay in L1/L2).  Block z of a split covers the
// k range [z kc, (z + 1) kc) and writes its partial tile to work[z].
__global__ void __launch_bounds__(128)
k_gemm(int64_t M, int64_t N, int64_t K, int64_t kc, const uint16_t* __restrict__ A,
       const uint16_t* __restrict__ Bt, float* __restrict__ C, uint16_t* __restrict__ Cb,
       const float* __restrict__ bias, int epi, int accumulate, float* __restrict__ work) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int64_t row0 = (int64_t)blockIdx.y * 64 + (warp >> 1) * 32;
  const int64_t col0 = (int64_t)blockIdx.x * 64 + (warp & 1) * 32;
  const int64_t k_begin = (int64_t)blockIdx.z * kc;
  const int64_t k_end = k_begin + kc < K ? k_begin + kc : K;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
  for (int64_t k = k_begin; k < k_end; k += 16) {
    uint32_t a[2][4], b[4][2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const uint16_t* r0 = A + (row0 + 16 * i + g) * K + k + 2 * t;
      const uint16_t* r8 = r0 + 8 * K;
      a[i][0] = ld_pair(r0);
      a[i][1] = ld_pair(r8);
      a[i][2] = ld_pair(r0 + 8);
      a[i][3] = ld_pair(r8 + 8);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint16_t* c = Bt + (col0 + 8 * j + g) * K + k + 2 * t;
      b[j][0] = ld_pair(c);
      b[j][1] = ld_pair(c + 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        mma_bf16(acc[i][j], a[i][0], a[i][1], a[i][2], a[i][3], b[j][0], b[j][1]);
  }
  float* dst = work ? work + (int64_t)blockIdx.z * M * N : C;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int64_t row = row0 + 16 * i + g + (r >= 2 ? 8 : 0);
        const int64_t col = col0 + 8 * j + 2 * t + (r & 1);
        float v = acc[i][j][r];
        if (!work) {
          if (accumulate) v += C[row * N + col];
          if (epi >= 1) v += bias[col];
          if (epi == 2) v = fmaxf(v, 0.f);
          if (Cb) Cb[row * N + col] = to_bf16(v);
        }
        dst[row * N + col] = v;
      }
}

// Sum of split partials in ascending split order, then the epilogue.
__global__ void k_split_reduce(int64_t MN, int64_t N, int splits, const float* __restrict__ work,
                               float* __restrict__ C, uint16_t* __restrict__ Cb,
                               const float* __restrict__ bias, int epi, int accumulate) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < MN;
       i += (int64_t)gridDim.x * blockDim.x) {
    float v = 0.f;
    for (int z = 0; z < splits; ++z) v += work[(int64_t)z * MN + i];
    if (accumulate) v += C[i];
    if (epi >= 1) v += bias[i % N];
    if (epi == 2) v = fmaxf(v, 0.f);
    C[i] = v;
    if (Cb) Cb[i] = to_bf16(v);
  }
}

__global__ void k_transpose(int64_t R, int64_t Cn, const uint16_t* __restrict__ in,
                            uint16_t* __restrict__ out) {
  __shared__ uint16_t tile[32][33];
  const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
  // in is [Cn][R]: read rows c of in, columns r
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t c = c0 + k, r = r0 + threadIdx.x;
    tile[k][threadIdx.x] = (c < Cn && r < R) ? in[c * R + r] : 0;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t r = r0 + k, c = c0 + threadIdx.x;
    if (r < R && c < Cn) out[r * Cn + c] = tile[threadIdx.x][k];
  }
}

__global__ void k_to_bf16(int64_t n, const float* __restrict__ in, uint16_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = to_bf16(in[i]);
}

constexpr uint32_t kOnePair = 0x3F80u;  // bf16 1.0 in the low half, 0 in the high half

// Out[e] = [H[dst[e]], H[src[e]], Ef[e], 1, 0 x 15] in 32-bit pairs (the
// constant 1 carries the layer's bias); zero rows past E.
__global__ void k_gather_edges(int64_t E, int64_t Epad, int H, int F, const int32_t* __restrict__ dst,
                               const int32_t* __restrict__ src, const uint16_t* __restrict__ Hn,
                               const uint16_t* __restrict__ Ef, uint16_t* __restrict__ out) {
  const int W2 = (2 * H + F + 16) / 2;  // pairs per row
  const int64_t total = Epad * W2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i / W2;
    const int c = (int)(i - e * W2) * 2;
    uint32_t v = 0;
    if (e < E) {
      if (c < H) v = ld_pair(Hn + (int64_t)dst[e] * H + c);
      else if (c < 2 * H) v = ld_pair(Hn + (int64_t)src[e] * H + (c - H));
      else if (c < 2 * H + F) v = ld_pair(Ef + e * F + (c - 2 * H));
      else if (c == 2 * H + F) v = kOnePair;
    }
    reinterpret_cast<uint32_t*>(out)[i] = v;
  }
}

// Out[i] = [A[i] (bf16, WA), bf16(B[i]) (fp32, WB), 1, 0 x 15]; zero rows past n.
__global__ void k_concat_rows(int64_t n, int64_t npad, int WA, int WB, const uint16_t* __restrict__ A,
                              const float* __restrict__ B, uint16_t* __restrict__ out) {
  const int W = WA + WB + 16;
  const int64_t total = npad * W;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / W;
    const int c = (int)(idx - i * W);
    uint16_t v = 0;
    if (i < n) {
      if (c < WA) v = A[i * WA + c];
      else if (c < WA + WB) v = to_bf16(B[i * WB + (c - WA)]);
      else if (c == WA + WB) v = 0x3F80u;
    }
    out[idx] = v;
  }
}

// h += u (fp32) and its bf16 copy, n values.
__global__ void k_residual(int64_t n, float* __restrict__ h, const float* __restrict__ u,
                           uint16_t* __restrict__ hb) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float v = h[i] + u[i];
    h[i] = v;
    hb[i] = to_bf16(v);
  }
}

// Out[e][c] = In[idx[e]][c] (fp32, width W); zero rows past E.
__global__ void k_gather_rows(int64_t E, int64_t Epad, int W, const int32_t* __restrict__ idx,
                              const float* __restrict__ in, float* __restrict__ out) {
  const int64_t total = Epad * W;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = k / W;
    const int c = (int)(k - e * W);
    out[k] = e < E ? in[(int64_t)idx[e] * W + c] : 0.f;
  }
}

// Out[i][c] = sum_{k in [off[i], off[i+1])} In[perm ? perm[k] : k][c0 + c], ascending k.
__global__ void k_segment_sum(int64_t n, int64_t npad, int W, int64_t stride, int c0,
                              const int64_t* __restrict__ off, const int32_t* __restrict__ perm,
                              const float* __restrict__ in, float* __restrict__ out) {
  const int64_t total = npad * W;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / W;
    const int c = (int)(idx - i * W);
    float s = 0.f;
    if (i < n)
      for (int64_t k = off[i]; k < off[i + 1]; ++k) {
        const int64_t e = perm ? (int64_t)perm[k] : k;
        s += in[e * stride + c0 + c];
      }
    out[i * W + c] = s;
  }
}

__global__ void k_relu_backward(int64_t n, const float* __restrict__ Y, float* __restrict__ G) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (!(Y[i] > 0.f)) G[i] = 0.f;
}

__global__ void k_adam(int64_t n, float* __restrict__ W, float* __restrict__ m,
                       float* __restrict__ v, const float* __restrict__ G, float lr, float b1,
                       float b2, float eps, float c1, float c2, uint16_t* __restrict__ Wb,
                       uint16_t* __restrict__ Wt, int rows, int cols, int kin) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float g = G[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float w = W[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    W[i] = w;
    if (Wb) Wb[i] = to_bf16(w);
    if (Wt && rows > 0) {
      const int64_t r = i / cols, c = i - r * cols;
      if (r < kin) Wt[c * (int64_t)kin + r] = to_bf16(w);
    }
  }
}

// One block: sum of squares in a fixed order (block-strided, then a tree).
__global__ void k_mse(int64_t n, const float* __restrict__ a, const float* __restrict__ b,
                      float scale, float* __restrict__ G, float* __restrict__ out) {
  __shared__ float part[256];
  float s = 0.f;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const float d = a[i] - b[i];
    s += d * d;
    G[i] = 2.f * d * scale;
  }
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = part[0];
}

// ---- neighbour graph within a cutoff (all pairs, tiled through shared memory)

// pass 0 counts, pass 1 writes: for node i, its neighbours j != i with
// |x_j - x_i| < cut in ascending j (the loop order), and dst of each edge.
__global__ void __launch_bounds__(256)
k_graph(int64_t n, const float* __restrict__ x, float cut2, int pass,
        int64_t* __restrict__ cnt_or_off, int32_t* __restrict__ nbr, int32_t* __restrict__ dst) {
  __shared__ float sx[256], sy[256], sz[256];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float xi = 0.f, yi = 0.f, zi = 0.f;
  if (i < n) {
    xi = x[3 * i];
    yi = x[3 * i + 1];
    zi = x[3 * i + 2];
  }
  int64_t k = 0;
  const int64_t base = (pass == 1 && i < n) ? cnt_or_off[i] : 0;
  for (int64_t j0 = 0; j0 < n; j0 += 256) {
    const int64_t jl = j0 + threadIdx.x;
    __syncthreads();
    if (jl < n) {
      sx[threadIdx.x] = x[3 * jl];
      sy[threadIdx.x] = x[3 * jl + 1];
      sz[threadIdx.x] = x[3 * jl + 2];
    }
    __syncthreads();
    const int m = (int)(n - j0 < 256 ? n - j0 : 256);
    if (i < n)
      for (int jj = 0; jj < m; ++jj) {
        const float dx = sx[jj] - xi, dy = sy[jj] - yi, dz = sz[jj] - zi;
        if (j0 + jj != i && dx * dx + dy * dy + dz * dz < cut2) {
          if (pass == 1) {
            nbr[base + k] = (int32_t)(j0 + jj);
            dst[base + k] = (int32_t)i;
          }
          ++k;
        }
      }
  }
  if (pass == 0 && i < n) cnt_or_off[i] = k;
}

// ---- neighbour graph from cell lists (cells of edge = cutoff) ---------------

constexpr int kMaxDegree = 128;  // neighbours of one node within the cutoff

// Bounding box of the nodes (one block): box = (lo xyz, hi xyz).
__global__ void __launch_bounds__(1024) k_box(int64_t n, const float* __restrict__ x,
                                              float* __restrict__ box) {
  __shared__ float s[6][1024];
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
    for (int a = 0; a < 3; ++a) {
      lo[a] = fminf(lo[a], x[3 * i + a]);
      hi[a] = fmaxf(hi[a], x[3 * i + a]);
    }
  for (int a = 0; a < 3; ++a) {
    s[a][threadIdx.x] = lo[a];
    s[3 + a][threadIdx.x] = hi[a];
  }
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int a = 0; a < 3; ++a) {
        s[a][threadIdx.x] = fminf(s[a][threadIdx.x], s[a][threadIdx.x + o]);
        s[3 + a][threadIdx.x] = fmaxf(s[3 + a][threadIdx.x], s[3 + a][threadIdx.x + o]);
      }
    __syncthreads();
  }
  if (threadIdx.x < 6) box[threadIdx.x] = s[threadIdx.x][0];
}

struct CellGrid {
  float lo[3];
  float inv_h;
  int32_t nc[3];
};

__device__ __forceinline__ int3 grid_cell(const CellGrid& g, float x, float y, float z) {
  const float p[3] = {x, y, z};
  int c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int ci = (int)floorf((p[a] - g.lo[a]) * g.inv_h);
    c[a] = ci < 0 ? 0 : (ci >= g.nc[a] ? g.nc[a] - 1 : ci);
  }
  return make_int3(c[0], c[1], c[2]);
}

// cell of every node and its arrival index in the cell
__global__ void k_cells_count(int64_t n, const float* __restrict__ x, CellGrid g,
                              unsigned long long* __restrict__ ccount,
                              int64_t* __restrict__ keyloc) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int3 c = grid_cell(g, x[3 * i], x[3 * i + 1], x[3 * i + 2]);
    const int64_t key = ((int64_t)c.z * g.nc[1] + c.y) * g.nc[0] + c.x;
    const unsigned long long loc = atomicAdd(&ccount[key], 1ull);
    keyloc[i] = (key << 24) | (int64_t)loc;
  }
}

__global__ void k_cells_scatter(int64_t n, const int64_t* __restrict__ keyloc,
                                const int64_t* __restrict__ cstart, int32_t* __restrict__ order) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t kl = keyloc[i];
    order[cstart[kl >> 24] + (kl & 0xffffff)] = (int32_t)i;
  }
}

// pass 0 counts (and records the largest degree), pass 1 writes: for node i,
// its neighbours j != i with |x_j - x_i| < cut from the 27 cells around it,
// in ascending j, and dst of each edge.
__global__ void __launch_bounds__(128)
k_graph_cells(int64_t n, const float* __restrict__ x, CellGrid g, float cut2, int pass,
              const int64_t* __restrict__ cstart, const int32_t* __restrict__ order,
              int64_t* __restrict__ cnt_or_off, int32_t* __restrict__ nbr,
              int32_t* __restrict__ dst, unsigned int* __restrict__ max_degree) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
  const int3 c = grid_cell(g, xi, yi, zi);
  int32_t found[kMaxDegree];
  int k = 0;
  for (int dz = -1; dz <= 1; ++dz) {
    const int cz = c.z + dz;
    if (cz < 0 || cz >= g.nc[2]) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int cy = c.y + dy;
      if (cy < 0 || cy >= g.nc[1]) continue;
      const int x0 = c.x > 0 ? c.x - 1 : 0, x1 = c.x + 1 < g.nc[0] ? c.x + 1 : g.nc[0] - 1;
      const int64_t row = ((int64_t)cz * g.nc[1] + cy) * g.nc[0];
      for (int64_t s = cstart[row + x0]; s < cstart[row + x1 + 1]; ++s) {
        const int32_t j = order[s];
        if ((int64_t)j == i) continue;
        const float dx = x[3 * j] - xi, dy2 = x[3 * j + 1] - yi, dz2 = x[3 * j + 2] - zi;
        if (dx * dx + dy2 * dy2 + dz2 * dz2 >= cut2) continue;
        if (pass == 1 && k < kMaxDegree) {  // sorted insertion (ascending j)
          int m = k;
          while (m > 0 && found[m - 1] > j) {
            found[m] = found[m - 1];
            --m;
          }
          found[m] = j;
        }
        ++k;
      }
    }
  }
  if (pass == 0) {
    cnt_or_off[i] = k;
    atomicMax(max_degree, (unsigned int)k);
  } else {
    const int64_t base = cnt_or_off[i];
    for (int m = 0; m < k && m < kMaxDegree; ++m) {
      nbr[base + m] = found[m];
      dst[base + m] = (int32_t)i;
    }
  }
}

// Exclusive scan of n counts into off[0..n] by one block (ascending).
__global__ void k_scan_counts(int64_t n, const int64_t* __restrict__ cnt, int64_t* __restrict__ off) {
  __shared__ int64_t part[1024];
  const int64_t chunk = (n + 1023) / 1024;
  const int64_t a = threadIdx.x * chunk, b = a + chunk < n ? a + chunk : n;
  int64_t s = 0;
  for (int64_t i = a; i < b; ++i) s += cnt[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t run = 0;
    for (int t = 0; t < 1024; ++t) {
      const int64_t v = part[t];
      part[t] = run;
      run += v;
    }
    off[n] = run;
  }
  __syncthreads();
  int64_t run = part[threadIdx.x];
  for (int64_t i = a; i < b; ++i) {
    off[i] = run;
    run += cnt[i];
  }
}

// perm[k] for k in node j's row (edges received by j, neighbour i = nbr[k]):
// the index of the reverse edge (received by i, sent by j), found by binary
// search in i's sorted row.  Grouped this way, the edges sent by j are
// perm[off[j] .. off[j+1]) in ascending receiver.
__global__ void k_reverse_edges(int64_t E, const int64_t* __restrict__ off,
                                const int32_t* __restrict__ nbr, const int32_t* __restrict__ dst,
                                int32_t* __restrict__ perm) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < E;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t j = dst[k], i = nbr[k];
    int64_t lo = off[i], hi = off[i + 1];
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (nbr[mid] < j) lo = mid + 1;
      else hi = mid;
    }
    perm[k] = (int32_t)lo;
  }
}

// Node and edge inputs of the network (16 columns each, bf16; column 7 holds
// the constant 1 that carries the first layer's bias):
//   node: v / vs, R w / vs, R / Rs - 1
//   edge (received by i from j): (x_j - x_i) / Rs, (|x_j - x_i| - R_i - R_j) / Rs,
//         (v_j - v_i) / vs
__global__ void k_features(int64_t n, int64_t npad, int64_t E, int64_t Epad,
                           const int32_t* __restrict__ dst, const int32_t* __restrict__ nbr,
                           const float* __restrict__ x, const float* __restrict__ v,
                           const float* __restrict__ w, const float* __restrict__ R, float vs,
                           float Rs, uint16_t* __restrict__ nf, uint16_t* __restrict__ ef) {
  const int64_t total = npad + Epad;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    float f[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) f[c] = 0.f;
    uint16_t* out;
    if (k < npad) {
      const int64_t i = k;
      out = nf + i * 16;
      if (i < n) {
        for (int c = 0; c < 3; ++c) {
          f[c] = v[3 * i + c] / vs;
          f[3 + c] = R[i] * w[3 * i + c] / vs;
        }
        f[6] = R[i] / Rs - 1.f;
        f[7] = 1.f;
      }
    } else {
      const int64_t e = k - npad;
      out = ef + e * 16;
      if (e < E) {
        const int64_t i = dst[e], j = nbr[e];
        float d2 = 0.f;
        for (int c = 0; c < 3; ++c) {
          const float d = x[3 * j + c] - x[3 * i + c];
          f[c] = d / Rs;
          d2 += d * d;
          f[4 + c] = (v[3 * j + c] - v[3 * i + c]) / vs;
        }
        f[3] = (sqrtf(d2) - R[i] - R[j]) / Rs;
        f[7] = 1.f;
      }
    }
#pragma unroll
    for (int c = 0; c < 16; ++c) out[c] = to_bf16(f[c]);
  }
}

unsigned grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 152 * 32) b = 152 * 32;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

extern "C" {

int mpnn_gemm(int64_t M, int64_t N, int64_t K, const uint16_t* A, const uint16_t* Bt, float* C,
              uint16_t* Cb, const float* bias, int32_t epi, int32_t accumulate, void* stream) {
  if (M <= 0 || N <= 0 || K <= 0 || M % 64 || N % 64 || K % 16 || !A || !Bt || !C)
    return DEM_ERR_INVALID;
  if (epi < 0 || epi > 2 || (epi >= 1 && !bias) || (accumulate && epi)) return DEM_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  dim3 grid((unsigned)(N / 64), (unsigned)(M / 64), 1);
  k_gemm<<<grid, 128, 0, st>>>(M, N, K, K, A, Bt, C, Cb, bias, epi, accumulate, nullptr);
  return launch_status();
}

// Split-k variant for a long reduction (the weight gradients): `splits`
// partial products go to work[splits][M][N] and are summed in order.
int mpnn_gemm_split(int64_t M, int64_t N, int64_t K, int32_t splits, const uint16_t* A,
                    const uint16_t* Bt, float* C, int32_t accumulate, float* work, void* stream) {
  if (M <= 0 || N <= 0 || K <= 0 || M % 64 || N % 64 || K % 16 || splits < 1 || !A || !Bt ||
      !C || !work)
    return DEM_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int64_t kc = (K + splits - 1) / splits;
  kc = (kc + 15) / 16 * 16;
  const int64_t z = (K + kc - 1) / kc;
  dim3 grid((unsigned)(N / 64), (unsigned)(M / 64), (unsigned)z);
  k_gemm<<<grid, 128, 0, st>>>(M, N, K, kc, A, Bt, C, nullptr, nullptr, 0, 0, work);
  k_split_reduce<<<grid_for(M * N, 256), 256, 0, st>>>(M * N, N, (int)z, work, C, nullptr,
                                                       nullptr, 0, accumulate);
  return launch_status();
}

int mpnn_transpose_bf16(int64_t R, int64_t Cn, const uint16_t* in, uint16_t* out, void* stream) {
  if (R <= 0 || Cn <= 0 || !in || !out) return DEM_ERR_INVALID;
  dim3 grid((unsigned)((Cn + 31) / 32), (unsigned)((R + 31) / 32));
  k_transpose<<<grid, dim3(32, 8), 0, static_cast<cudaStream_t>(stream)>>>(R, Cn, in, out);
  return launch_status();
}

int mpnn_to_bf16(int64_t n, const float* in, uint16_t* out, void* stream) {
  if (n < 0 || (n > 0 && (!in || !out))) return DEM_ERR_INVALID;
  if (n == 0) return DEM_OK;
  k_to_bf16<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(n, in, out);
  return launch_status();
}

int mpnn_gather_edges(int64_t E, int64_t Epad, int32_t H, int32_t F, const int32_t* dst,
                      const int32_t* src, const uint16_t* Hn, const uint16_t* Ef, uint16_t* out,
                      void* stream) {
  if (E < 0 || Epad < E || H <= 0 || F <= 0 || H % 2 || F % 2 || !out) return DEM_ERR_INVALID;
  if (E > 0 && (!dst || !src || !Hn || !Ef)) return DEM_ERR_INVALID;
  if (Epad == 0) return DEM_OK;
  k_gather_edges<<<grid_for(Epad * (2 * H + F + 16) / 2, 256), 256, 0,
                   static_cast<cudaStream_t>(stream)>>>(E, Epad, H, F, dst, src, Hn, Ef, out);
  return launch_status();
}

int mpnn_concat_rows(int64_t n, int64_t npad, int32_t WA, int32_t WB, const uint16_t* A,
                     const float* B, uint16_t* out, void* stream) {
  if (n < 0 || npad < n || WA <= 0 || WB < 0 || !A || (WB > 0 && !B) || !out)
    return DEM_ERR_INVALID;
  if (npad == 0) return DEM_OK;
  k_concat_rows<<<grid_for(npad * (WA + WB + 16), 256), 256, 0,
                  static_cast<cudaStream_t>(stream)>>>(n, npad, WA, WB, A, B, out);
  return launch_status();
}

int mpnn_residual(int64_t n, float* h, const float* u, uint16_t* hb, void* stream) {
  if (n <= 0 || !h || !u || !hb) return DEM_ERR_INVALID;
  k_residual<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(n, h, u, hb);
  return launch_status();
}

int mpnn_gather_rows(int64_t E, int64_t Epad, int32_t W, const int32_t* idx, const float* in,
                     float* out, void* stream) {
  if (E < 0 || Epad < E || W <= 0 || !out || (E > 0 && (!idx || !in))) return DEM_ERR_INVALID;
  if (Epad == 0) return DEM_OK;
  k_gather_rows<<<grid_for(Epad * W, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      E, Epad, W, idx, in, out);
  return launch_status();
}

int mpnn_segment_sum(int64_t n, int64_t npad, int32_t W, const int64_t* off, const float* in,
                     float* out, void* stream) {
  if (n < 0 || npad < n || W <= 0 || !off || !in || !out) return DEM_ERR_INVALID;
  if (npad == 0) return DEM_OK;
  k_segment_sum<<<grid_for(npad * W, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      n, npad, W, W, 0, off, nullptr, in, out);
  return launch_status();
}

// Strided form: columns [c0, c0 + W) of rows of width `stride`.
int mpnn_segment_sum_cols(int64_t n, int64_t npad, int32_t W, int64_t stride, int32_t c0,
                          const int64_t* off, const int32_t* perm, const float* in, float* out,
                          void* stream) {
  if (n < 0 || npad < n || W <= 0 || c0 < 0 || c0 + W > stride || !off || !in || !out)
    return DEM_ERR_INVALID;
  if (npad == 0) return DEM_OK;
  k_segment_sum<<<grid_for(npad * W, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      n, npad, W, stride, c0, off, perm, in, out);
  return launch_status();
}

int mpnn_segment_sum_perm(int64_t n, int64_t npad, int32_t W, const int64_t* off,
                          const int32_t* perm, const float* in, float* out, void* stream) {
  if (n < 0 || npad < n || W <= 0 || !off || !perm || !in || !out) return DEM_ERR_INVALID;
  if (npad == 0) return DEM_OK;
  k_segment_sum<<<grid_for(npad * W, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      n, npad, W, W, 0, off, perm, in, out);
  return launch_status();
}

int mpnn_relu_backward(int64_t n, const float* Y, float* G, void* stream) {
  if (n < 0 || (n > 0 && (!Y || !G))) return DEM_ERR_INVALID;
  if (n == 0) return DEM_OK;
  k_relu_backward<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(n, Y, G);
  return launch_status();
}

int mpnn_adam(int64_t n, float* W, float* m, float* v, const float* G, float lr, float beta1,
               float beta2, float eps, int64_t t, uint16_t* Wb, uint16_t* Wt, int32_t rows,
               int32_t cols, int32_t kin, void* stream) {
  if (n <= 0 || !W || !m || !v || !G || t < 1 || (Wt && (rows <= 0 || cols <= 0 || kin > rows)))
    return DEM_ERR_INVALID;
  const float c1 = 1.f / (1.f - powf(beta1, (float)t));
  const float c2 = 1.f / (1.f - powf(beta2, (float)t));
  k_adam<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      n, W, m, v, G, lr, beta1, beta2, eps, c1, c2, Wb, Wt, rows, cols, kin);
  return launch_status();
}

int mpnn_graph(int64_t n, const float* x, float cutoff, int64_t* cnt, int64_t* off,
               int32_t* nbr, int32_t* dst, int64_t max_edges, int64_t* n_edges_host,
               void* stream) {
  if (n <= 0 || !x || !(cutoff > 0) || !cnt || !off) return DEM_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned nb = (unsigned)((n + 255) / 256);
  const float c2 = cutoff * cutoff;
  k_graph<<<nb, 256, 0, st>>>(n, x, c2, 0, cnt, nullptr, nullptr);
  k_scan_counts<<<1, 1024, 0, st>>>(n, cnt, off);
  int64_t E = 0;
  if (cudaMemcpyAsync(&E, off + n, sizeof E, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return DEM_ERR_CUDA;
  if (n_edges_host) *n_edges_host = E;
  if (E > max_edges || !nbr || !dst) return E > max_edges ? DEM_ERR_CAPACITY : DEM_ERR_INVALID;
  k_graph<<<nb, 256, 0, st>>>(n, x, c2, 1, off, nbr, dst);
  return launch_status();
}

int mpnn_graph_cells(int64_t n, const float* x, float cutoff, int64_t max_cells, int64_t* work,
                     float* box, int64_t* cnt, int64_t* off, int32_t* nbr, int32_t* dst,
                     int64_t max_edges, int64_t* n_edges_host, void* stream) {
  if (n <= 0 || n >= ((int64_t)1 << 24) || !x || !(cutoff > 0) || max_cells <= 0 || !work ||
      !box || !cnt || !off)
    return DEM_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_box<<<1, 1024, 0, st>>>(n, x, box);
  float hb[6];
  if (cudaMemcpyAsync(hb, box, sizeof hb, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return DEM_ERR_CUDA;
  CellGrid g;
  int64_t ncells = 1;
  for (int a = 0; a < 3; ++a) {
    if (!(hb[a] <= hb[3 + a])) return DEM_ERR_INVALID;  // non-finite positions
    g.lo[a] = hb[a];
    const double ext = (double)hb[3 + a] - (double)hb[a];
    const int64_t c = (int64_t)(ext / cutoff) + 1;
    g.nc[a] = (int32_t)(c < (1 << 20) ? c : (1 << 20));
    ncells *= g.nc[a];
    if (ncells > max_cells) return DEM_ERR_CAPACITY;
  }
  g.inv_h = 1.f / cutoff;
  // workspace: cell counts [ncells + 1], cell starts [ncells + 1], key|local [n], order [n]
  unsigned long long* ccount = reinterpret_cast<unsigned long long*>(work);
  int64_t* cstart = work + (max_cells + 1);
  int64_t* keyloc = cstart + (max_cells + 1);
  int32_t* order = reinterpret_cast<int32_t*>(keyloc + n);
  unsigned int* maxdeg = reinterpret_cast<unsigned int*>(order + n);
  if (cudaMemsetAsync(ccount, 0, sizeof(int64_t) * (ncells + 1), st) != cudaSuccess ||
      cudaMemsetAsync(maxdeg, 0, sizeof(unsigned int), st) != cudaSuccess)
    return DEM_ERR_CUDA;
  const unsigned nb = grid_for(n, 256);
  k_cells_count<<<nb, 256, 0, st>>>(n, x, g, ccount, keyloc);
  k_scan_counts<<<1, 1024, 0, st>>>(ncells, reinterpret_cast<const int64_t*>(ccount), cstart);
  k_cells_scatter<<<nb, 256, 0, st>>>(n, keyloc, cstart, order);
  const float c2 = cutoff * cutoff;
  const unsigned nb128 = (unsigned)((n + 127) / 128);
  k_graph_cells<<<nb128, 128, 0, st>>>(n, x, g, c2, 0, cstart, order, cnt, nullptr, nullptr,
                                       maxdeg);
  k_scan_counts<<<1, 1024, 0, st>>>(n, cnt, off);
  int64_t E = 0;
  unsigned int md = 0;
  if (cudaMemcpyAsync(&E, off + n, sizeof E, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&md, maxdeg, sizeof md, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return DEM_ERR_CUDA;
  if (n_edges_host) *n_edges_host = E;
  if (md > (unsigned)kMaxDegree) return DEM_ERR_CAPACITY;
  if (E > max_edges || !nbr || !dst) return E > max_edges ? DEM_ERR_CAPACITY : DEM_ERR_INVALID;
  k_graph_cells<<<nb128, 128, 0, st>>>(n, x, g, c2, 1, cstart, order, off, nbr, dst, maxdeg);
  return launch_status();
}

int mpnn_reverse_edges(int64_t E, const int64_t* off, const int32_t* nbr, const int32_t* dst,
                       int32_t* perm, void* stream) {
  if (E < 0 || (E > 0 && (!off || !nbr || !dst || !perm))) return DEM_ERR_INVALID;
  if (E == 0) return DEM_OK;
  k_reverse_edges<<<grid_for(E, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(E, off, nbr,
                                                                                  dst, perm);
  return launch_status();
}

int mpnn_features(int64_t n, int64_t npad, int64_t E, int64_t Epad, const int32_t* dst,
                  const int32_t* nbr, const float* x, const float* v, const float* w,
                  const float* R, float vs, float Rs, uint16_t* nf, uint16_t* ef, void* stream) {
  if (n <= 0 || npad < n || E < 0 || Epad < E || !x || !v || !w || !R || !nf || !ef ||
      (E > 0 && (!dst || !nbr)) || !(vs > 0) || !(Rs > 0))
    return DEM_ERR_INVALID;
  k_features<<<grid_for(npad + Epad, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      n, npad, E, Epad, dst, nbr, x, v, w, R, vs, Rs, nf, ef);
  return launch_status();
}

int mpnn_mse(int64_t n, const float* a, const float* b, float scale, float* G, float* out,
             void* stream) {
  if (n <= 0 || !a || !b || !G || !out) return DEM_ERR_INVALID;
  k_mse<<<1, 256, 0, static_cast<cudaStream_t>(stream)>>>(n, a, b, scale, G, out);
  return launch_status();
}

}  // extern "C"
