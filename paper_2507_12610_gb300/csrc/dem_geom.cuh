// Geometry shared by the list build and the step kernels: cell coordinates of
// a shifted float position, and the closest point on a triangle.
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

// Closest point on triangle (a, b, c) to point q, by Voronoi regions of the
// vertices, edges and face (Ericson, Real-Time Collision Detection, Sec. 5.1.5,
// the reference the paper gives for its distance routines).
template <typename T>
__device__ __forceinline__ V3<T> closest_point_triangle(V3<T> q, V3<T> a, V3<T> b, V3<T> c) {
  const V3<T> ab = b - a, ac = c - a, aq = q - a;
  const T d1 = dot(ab, aq), d2 = dot(ac, aq);
  if (d1 <= T(0) && d2 <= T(0)) return a;
  const V3<T> bq = q - b;
  const T d3 = dot(ab, bq), d4 = dot(ac, bq);
  if (d3 >= T(0) && d4 <= d3) return b;
  const T vc = d1 * d4 - d3 * d2;
  if (vc <= T(0) && d1 >= T(0) && d3 <= T(0)) {
    const T t = d1 / (d1 - d3);
    return a + t * ab;
  }
  const V3<T> cq = q - c;
  const T d5 = dot(ab, cq), d6 = dot(ac, cq);
  if (d6 >= T(0) && d5 <= d6) return c;
  const T vb = d5 * d2 - d1 * d6;
  if (vb <= T(0) && d2 >= T(0) && d6 <= T(0)) {
    const T t = d2 / (d2 - d6);
    return a + t * ac;
  }
  const T va = d3 * d6 - d5 * d4;
  if (va <= T(0) && (d4 - d3) >= T(0) && (d5 - d6) >= T(0)) {
    const T t = (d4 - d3) / ((d4 - d3) + (d5 - d6));
    return b + t * (c - b);
  }
  const T den = T(1) / (va + vb + vc);
  const T v = vb * den, w = vc * den;
  return a + v * ab + w * ac;
}

// Closest point on segment ab to q.
template <typename T>
__device__ __forceinline__ V3<T> closest_point_segment(V3<T> q, V3<T> a, V3<T> b) {
  const V3<T> ab = b - a;
  const T l2 = dot(ab, ab);
  if (!(l2 > T(0))) return a;
  T t = dot(q - a, ab) / l2;
  t = t < T(0) ? T(0) : (t > T(1) ? T(1) : t);
  return a + t * ab;
}

// Closest point on the rectangle with corner a and perpendicular edges a->b,
// a->d: clamp the two edge coordinates of q (exact for right angles).
template <typename T>
__device__ __forceinline__ V3<T> closest_point_rectangle(V3<T> q, V3<T> a, V3<T> b, V3<T> d) {
  const V3<T> u = b - a, w = d - a, aq = q - a;
  T s = dot(aq, u) / dot(u, u);
  T t = dot(aq, w) / dot(w, w);
  s = s < T(0) ? T(0) : (s > T(1) ? T(1) : s);
  t = t < T(0) ? T(0) : (t > T(1) ? T(1) : t);
  return a + s * u + t * w;
}

// Closest point on a mesh element of nv vertices (Sec. 3.3): 1 point,
// 2 segment, 3 triangle, 4 rectangle (vertices a, b, c, d in order).
template <typename T>
__device__ __forceinline__ V3<T> closest_point_element(V3<T> q, V3<T> a, V3<T> b, V3<T> c,
                                                       V3<T> d, int nv) {
  if (nv == 3) return closest_point_triangle(q, a, b, c);
  if (nv == 4) return closest_point_rectangle(q, a, b, d);
  if (nv == 2) return closest_point_segment(q, a, b);
  return a;
}

}  // namespace dem
