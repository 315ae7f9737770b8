// Geometry shared by the list build and the step kernels: cell coordinates of
// a shifted float position, and the closest point on a mesh element.
#pragma once

#include "dem_internal.cuh"
#include "dem_math.cuh"

namespace dem {

// Cell coordinates of a shifted position X (X = x - origin), clamped to the
// grid.  Clamping keeps neighbouring particles in neighbouring cells, so a
// particle that leaves the binning box is still found (only less efficiently).
__device__ __forceinline__ int3 cell_coords(const Params& p, float X, float Y, float Z) {
  int cx = (int)floorf((X - (float)p.base[0]) * p.inv_h);
  int cy = (int)floorf((Y - (float)p.base[1]) * p.inv_h);
  int cz = (int)floorf((Z - (float)p.base[2]) * p.inv_h);
  cx = min(max(cx, 0), p.nc[0] - 1);
  cy = min(max(cy, 0), p.nc[1] - 1);
  cz = min(max(cz, 0), p.nc[2] - 1);
  return make_int3(cx, cy, cz);
}

__device__ __forceinline__ uint32_t cell_index(const Params& p, int3 c) {
  return (uint32_t)((c.z * p.nc[1] + c.y) * p.nc[0] + c.x);
}

// Nearest feature of an element, reported with the closest point so that a
// caller can redo the distance to that feature in higher precision: a vertex
// (its slot, 0-3), an edge (feat_edge of its two slots) or the face.
constexpr int kFeatFace = 32;
__host__ __device__ constexpr int feat_edge(int i, int j) { return 4 + 4 * i + j; }

// Closest point on triangle (a, b, c) to point q, by Voronoi regions of the
// vertices, edges and face (Ericson, Real-Time Collision Detection, Sec. 5.1.5,
// the reference the paper gives for its distance routines).
template <typename T>
__device__ __forceinline__ V3<T> closest_point_triangle(V3<T> q, V3<T> a, V3<T> b, V3<T> c,
                                                        int& feat) {
  const V3<T> ab = b - a, ac = c - a, aq = q - a;
  const T d1 = dot(ab, aq), d2 = dot(ac, aq);
  if (d1 <= T(0) && d2 <= T(0)) {
    feat = 0;
    return a;
  }
  const V3<T> bq = q - b;
  const T d3 = dot(ab, bq), d4 = dot(ac, bq);
  if (d3 >= T(0) && d4 <= d3) {
    feat = 1;
    return b;
  }
  const T vc = d1 * d4 - d3 * d2;
  if (vc <= T(0) && d1 >= T(0) && d3 <= T(0)) {
    feat = feat_edge(0, 1);
    const T t = d1 / (d1 - d3);
    return a + t * ab;
  }
  const V3<T> cq = q - c;
  const T d5 = dot(ab, cq), d6 = dot(ac, cq);
  if (d6 >= T(0) && d5 <= d6) {
    feat = 2;
    return c;
  }
  const T vb = d5 * d2 - d1 * d6;
  if (vb <= T(0) && d2 >= T(0) && d6 <= T(0)) {
    feat = feat_edge(0, 2);
    const T t = d2 / (d2 - d6);
    return a + t * ac;
  }
  const T va = d3 * d6 - d5 * d4;
  if (va <= T(0) && (d4 - d3) >= T(0) && (d5 - d6) >= T(0)) {
    feat = feat_edge(1, 2);
    const T t = (d4 - d3) / ((d4 - d3) + (d5 - d6));
    return b + t * (c - b);
  }
  feat = kFeatFace;
  const T den = T(1) / (va + vb + vc);
  const T v = vb * den, w = vc * den;
  return a + v * ab + w * ac;
}

// Closest point on segment ab to q (a zero-length segment is its end point).
template <typename T>
__device__ __forceinline__ V3<T> closest_point_segment(V3<T> q, V3<T> a, V3<T> b, int& feat) {
  const V3<T> ab = b - a;
  const T l2 = dot(ab, ab);
  feat = 0;
  if (!(l2 > T(0))) return a;
  const T t = dot(q - a, ab) / l2;
  if (t <= T(0)) return a;
  if (t >= T(1)) {
    feat = 1;
    return b;
  }
  feat = feat_edge(0, 1);
  return a + t * ab;
}

// Closest point on the rectangle a-b-c-d (right angles; edges a->b and a->d):
// the two edge coordinates of q select the face, an edge or a corner; the
// edges and corners are those of the given vertices.
template <typename T>
__device__ __forceinline__ V3<T> closest_point_rectangle(V3<T> q, V3<T> a, V3<T> b, V3<T> c,
                                                         V3<T> d, int& feat) {
  const V3<T> u = b - a, w = d - a, aq = q - a;
  const T s = dot(aq, u) / dot(u, u);
  const T t = dot(aq, w) / dot(w, w);
  const bool s0 = s <= T(0), s1 = s >= T(1), t0 = t <= T(0), t1 = t >= T(1);
  int f;
  if (!(s0 || s1 || t0 || t1)) {
    feat = kFeatFace;
    return a + s * u + t * w;
  }
  if (s0 && t0) {
    feat = 0;
    return a;
  }
  if (s1 && t0) {
    feat = 1;
    return b;
  }
  if (s1 && t1) {
    feat = 2;
    return c;
  }
  if (s0 && t1) {
    feat = 3;
    return d;
  }
  if (t0) {
    feat = feat_edge(0, 1);
    return closest_point_segment(q, a, b, f);
  }
  if (s1) {
    feat = feat_edge(1, 2);
    return closest_point_segment(q, b, c, f);
  }
  if (t1) {
    feat = feat_edge(3, 2);
    return closest_point_segment(q, d, c, f);
  }
  feat = feat_edge(0, 3);
  return closest_point_segment(q, a, d, f);
}

// Closest point on a mesh element of nv vertices (Sec. 3.3): 1 point,
// 2 segment, 3 triangle, 4 rectangle (vertices a, b, c, d in order).
template <typename T>
__device__ __forceinline__ V3<T> closest_point_element(V3<T> q, V3<T> a, V3<T> b, V3<T> c,
                                                       V3<T> d, int nv, int& feat) {
  if (nv == 3) return closest_point_triangle(q, a, b, c, feat);
  if (nv == 4) return closest_point_rectangle(q, a, b, c, d, feat);
  if (nv == 2) return closest_point_segment(q, a, b, feat);
  feat = 0;
  return a;
}
template <typename T>
__device__ __forceinline__ V3<T> closest_point_element(V3<T> q, V3<T> a, V3<T> b, V3<T> c,
                                                       V3<T> d, int nv) {
  int feat;
  return closest_point_element(q, a, b, c, d, nv, feat);
}

}  // namespace dem
