/*
 * mpnn.h -- C ABI of the message-passing surrogate kernels in libdem.so.
 *
 * The surrogate is a learned stand-in for the DEM force evaluation over a
 * stride of time steps: a message-passing network over the particle
 * neighbour graph that predicts each particle's mean linear and angular
 * acceleration over the stride.  This header exposes its building blocks;
 * the network, its training loop and the DEM fallback are assembled by the
 * Python module paper_2507_12610_gb300/surrogate.py.  The paper has no
 * learned component; these entry points are the project's own.
 *
 * Conventions: every pointer is a DEVICE pointer unless stated; matrices are
 * row-major; bf16 is IEEE bfloat16 stored as uint16_t; `stream` is a
 * cudaStream_t (NULL = legacy default stream).  Calls enqueue work and return
 * without waiting (except mpnn_graph, which reads the edge count back); they
 * return DEM_OK (0), DEM_ERR_INVALID (1) for bad sizes or NULL pointers,
 * DEM_ERR_CAPACITY (2) if the edge buffers are too small, or DEM_ERR_CUDA (4)
 * if a launch fails.  No call allocates device memory.  Every sum is taken in
 * a fixed order: results do not depend on the launch shape or on timing.
 */
#ifndef MPNN_H_
#define MPNN_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* C[M][N] (fp32) = A[M][K] (bf16) * B, B given transposed as Bt[N][K] (bf16),
 * then, by `epi`: 0 plain, 1 + bias[N] (fp32), 2 relu(+ bias).  If Cb is not
 * NULL the result is also written as bf16 to Cb[M][N].  With `accumulate`
 * nonzero, C += A * B (epi must be 0).  Tensor cores (mma m16n8k16, bf16
 * inputs, fp32 accumulation).  Requires M % 64 == 0, N % 64 == 0, K % 16 == 0. */
int mpnn_gemm(int64_t M, int64_t N, int64_t K, const uint16_t* A, const uint16_t* Bt,
              float* C, uint16_t* Cb, const float* bias, int32_t epi, int32_t accumulate,
              void* stream);

/* As mpnn_gemm (epi 0) with the k range split in `splits` parts whose partial
 * products go to work[splits][M][N] (caller-owned) and are then summed in
 * ascending part order; for long reductions (weight gradients). */
int mpnn_gemm_split(int64_t M, int64_t N, int64_t K, int32_t splits, const uint16_t* A,
                    const uint16_t* Bt, float* C, int32_t accumulate, float* work, void* stream);

/* Out[R][C] (bf16) = In[C][R] transposed. */
int mpnn_transpose_bf16(int64_t R, int64_t C, const uint16_t* in, uint16_t* out, void* stream);

/* fp32 -> bf16 (round to nearest even) of n values. */
int mpnn_to_bf16(int64_t n, const float* in, uint16_t* out, void* stream);

/* Neighbour graph: for each of n nodes at x (fp32 [n][3]) the nodes j != i
 * with |x_j - x_i| < cutoff, in ascending j: cnt[n] (work), off[n+1] (CSR
 * offsets, int64), nbr[E] (sender j), dst[E] (receiver i).  Writes the edge
 * count E to *n_edges_host (host pointer; the call waits for it) and returns
 * DEM_ERR_CAPACITY without writing edges if E > max_edges.  All pairs are
 * tested (O(n^2), tiled through shared memory). */
int mpnn_graph(int64_t n, const float* x, float cutoff, int64_t* cnt, int64_t* off,
               int32_t* nbr, int32_t* dst, int64_t max_edges, int64_t* n_edges_host,
               void* stream);

/* The same graph from cell lists (cells of edge `cutoff` over the nodes'
 * bounding box, 27 cells searched per node; O(n)), in ascending j per node.
 * work: device workspace of 2 (max_cells + 1) + 2 n int64 words + 1; box:
 * 6 floats of device memory (the bounding box, written).  The call waits for
 * the bounding box and the edge count.  Errors: DEM_ERR_INVALID (n < 1 or
 * n >= 2^24, non-finite positions, cutoff <= 0), DEM_ERR_CAPACITY (more than
 * max_cells cells, more than max_edges edges, or a node with more than 128
 * neighbours; nothing written then). */
int mpnn_graph_cells(int64_t n, const float* x, float cutoff, int64_t max_cells, int64_t* work,
                     float* box, int64_t* cnt, int64_t* off, int32_t* nbr, int32_t* dst,
                     int64_t max_edges, int64_t* n_edges_host, void* stream);

/* perm[k] = index of the reverse of edge k (the graph is symmetric); grouped
 * by off, perm lists the edges each node sends, in ascending receiver. */
int mpnn_reverse_edges(int64_t E, const int64_t* off, const int32_t* nbr, const int32_t* dst,
                       int32_t* perm, void* stream);

/* Network inputs, 16 bf16 columns per node / edge, column 7 = 1 (bias):
 * node i: v_i / vs, R_i w_i / vs, R_i / Rs - 1; edge (i <- j):
 * (x_j - x_i) / Rs, (|x_j - x_i| - R_i - R_j) / Rs, (v_j - v_i) / vs.  Rows
 * past n (up to npad) and past E (up to Epad) are zero.  x, v, w fp32 [n][3],
 * R fp32 [n]. */
int mpnn_features(int64_t n, int64_t npad, int64_t E, int64_t Epad, const int32_t* dst,
                  const int32_t* nbr, const float* x, const float* v, const float* w,
                  const float* R, float vs, float Rs, uint16_t* nf, uint16_t* ef, void* stream);

/* Message-layer input: row e of Out (bf16, width 2H + F + 16) =
 * [Hn[dst[e]], Hn[src[e]], Ef[e], 1, 0 x 15]; rows past E (up to Epad) zero. */
int mpnn_gather_edges(int64_t E, int64_t Epad, int32_t H, int32_t F, const int32_t* dst,
                      const int32_t* src, const uint16_t* Hn, const uint16_t* Ef, uint16_t* out,
                      void* stream);

/* Out[i] = [A[i] (bf16, WA columns), bf16(B[i]) (fp32, WB columns), 1, 0 x 15];
 * rows past n (up to npad) zero. */
int mpnn_concat_rows(int64_t n, int64_t npad, int32_t WA, int32_t WB, const uint16_t* A,
                     const float* B, uint16_t* out, void* stream);

/* h += u (fp32, n values) and hb = bf16(h). */
int mpnn_residual(int64_t n, float* h, const float* u, uint16_t* hb, void* stream);

/* Out[e] = In[idx[e]] (fp32 rows of width W); rows past E (up to Epad) zero. */
int mpnn_gather_rows(int64_t E, int64_t Epad, int32_t W, const int32_t* idx, const float* in,
                     float* out, void* stream);

/* Out[i][:] = sum over e in [off[i], off[i+1]) of In[e][:] (fp32, width W),
 * ascending e; rows past n (up to npad) zero. */
int mpnn_segment_sum(int64_t n, int64_t npad, int32_t W, const int64_t* off, const float* in,
                     float* out, void* stream);

/* As mpnn_segment_sum over columns [c0, c0 + W) of rows of width `stride`,
 * through perm when not NULL (In row perm[k] for k in the segment). */
int mpnn_segment_sum_cols(int64_t n, int64_t npad, int32_t W, int64_t stride, int32_t c0,
                          const int64_t* off, const int32_t* perm, const float* in, float* out,
                          void* stream);

/* As mpnn_segment_sum through perm. */
int mpnn_segment_sum_perm(int64_t n, int64_t npad, int32_t W, const int64_t* off,
                          const int32_t* perm, const float* in, float* out, void* stream);

/* ReLU backward: G[i] = 0 where Y[i] <= 0 (fp32, n values). */
int mpnn_relu_backward(int64_t n, const float* Y, float* G, void* stream);

/* Adam step (bias-corrected, step t >= 1) on n fp32 parameters W with
 * moments m, v and gradient G.  Also writes the bf16 copy Wb (same layout,
 * may be NULL) and, if Wt is not NULL, the transposed bf16 copy of the
 * [rows][cols] matrix's first kin rows: Wt[cols][kin]. */
int mpnn_adam(int64_t n, float* W, float* m, float* v, const float* G, float lr, float beta1,
              float beta2, float eps, int64_t t, uint16_t* Wb, uint16_t* Wt, int32_t rows,
              int32_t cols, int32_t kin, void* stream);

/* out[0] = sum of (a - b)^2 over n values (one block, fixed order), and
 * G = 2 (a - b) * scale. */
int mpnn_mse(int64_t n, const float* a, const float* b, float scale, float* G, float* out,
             void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MPNN_H_ */
