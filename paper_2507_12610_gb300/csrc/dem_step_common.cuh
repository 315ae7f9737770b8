// Helpers shared by the step kernels of both precisions.
#pragma once

#include "dem_internal.cuh"
#include "dem_math.cuh"

namespace dem {

__device__ __forceinline__ void set_status(Ctl* ctl, uint32_t code) {
  atomicCAS(&ctl->status, 0u, code);
}

__device__ __forceinline__ V3<double> xyz(D4 a) { return mk(a.x, a.y, a.z); }

__device__ __forceinline__ void count_and_flag(Ctl* ctl, uint32_t npair, uint32_t nmesh, bool disp,
                                               bool bad) {
  const unsigned full = 0xffffffffu;
  const uint32_t sp = __reduce_add_sync(full, npair);
  const uint32_t sm = __reduce_add_sync(full, nmesh);
  const bool anyd = __any_sync(full, disp);
  const bool anyb = __any_sync(full, bad);
  if ((threadIdx.x & 31) == 0) {
    if (sp) atomicAdd(&ctl->pair_contacts, sp);
    if (sm) atomicAdd(&ctl->mesh_contacts, sm);
    if (anyd) atomicOr(&ctl->disp_flag, 1u);
    if (anyb) set_status(ctl, DEM_ERR_NONFINITE);
  }
}

// Hamilton product (Sec. 2.3).
template <typename T>
__device__ __forceinline__ void qmul(const T a[4], const T b[4], T out[4]) {
  out[0] = a[0] * b[0] - (a[1] * b[1] + a[2] * b[2] + a[3] * b[3]);
  const V3<T> av = mk(a[1], a[2], a[3]), bv = mk(b[1], b[2], b[3]);
  const V3<T> r = a[0] * bv + b[0] * av + cross(av, bv);
  out[1] = r.x;
  out[2] = r.y;
  out[3] = r.z;
}

// The rotation factor of the SPIRAL update (Sec. 2.3, Eq. spiral): the unit
// quaternion (cos phi, sin phi a / |a|) with phi = h |a|, returned as
// r = (cos phi - 1, sin phi a / |a|) (the scalar part minus one, so a caller
// adding the increment q r to q keeps the small terms).  For phi^2 < 1/256
// both parts come from |a|^2 alone as Taylor series of the angle:
//   cos phi - 1 = -(p/2) (1 - (p/12) (1 - (p/30) (1 - (p/56) (1 - p/90)))),
//   sin phi / phi = 1 - (p/6) (1 - (p/20) (1 - (p/42) (1 - (p/72) (1 - p/110)))),
// p = phi^2, and sin phi a / |a| = (sin phi / phi) h a.  Truncated after the
// p^5 terms the first omitted term is below 1e-23 of the result (double);
// float keeps the first three levels (omitted terms below 1e-11).  No root,
// division or sine is taken.  Larger angles take sin and cos.  Returns false
// if a = 0 (no rotation).
__device__ __forceinline__ bool rot_factor(double h, V3<double> a, double r[4]) {
  const double a2 = dot(a, a);
  if (!(a2 > 0.0)) return false;
  const double p = (h * h) * a2;
  if (p < 1.0 / 256.0) {
    const double cm1 =
        -(p * 0.5) *
        (1.0 - (p * (1.0 / 12.0)) *
                   (1.0 - (p * (1.0 / 30.0)) * (1.0 - (p * (1.0 / 56.0)) * (1.0 - p * (1.0 / 90.0)))));
    const double sc =
        1.0 - (p * (1.0 / 6.0)) *
                  (1.0 - (p * (1.0 / 20.0)) *
                             (1.0 - (p * (1.0 / 42.0)) * (1.0 - (p * (1.0 / 72.0)) * (1.0 - p * (1.0 / 110.0)))));
    const double sh = sc * h;
    r[0] = cm1;
    r[1] = sh * a.x;
    r[2] = sh * a.y;
    r[3] = sh * a.z;
  } else {
    const double an = sqrt(a2);
    double sp, cp;
    sincos(h * an, &sp, &cp);
    r[0] = cp - 1.0;
    r[1] = sp * a.x / an;
    r[2] = sp * a.y / an;
    r[3] = sp * a.z / an;
  }
  return true;
}
__device__ __forceinline__ bool rot_factor(float h, V3<float> a, float r[4]) {
  const float a2 = dot(a, a);
  if (!(a2 > 0.f)) return false;
  const float p = (h * h) * a2;
  if (p < 1.f / 256.f) {
    r[0] = -(p * 0.5f) * (1.f - (p * (1.f / 12.f)) * (1.f - p * (1.f / 30.f)));
    const float sh = (1.f - (p * (1.f / 6.f)) * (1.f - (p * (1.f / 20.f)) * (1.f - p * (1.f / 42.f)))) * h;
    r[1] = sh * a.x;
    r[2] = sh * a.y;
    r[3] = sh * a.z;
  } else {
    const float an = sqrtf(a2);
    const float phi = h * an;
    const float s2 = sinf(0.5f * phi);
    const float sp = sinf(phi);
    r[0] = -2.f * s2 * s2;
    r[1] = sp * a.x / an;
    r[2] = sp * a.y / an;
    r[3] = sp * a.z / an;
  }
  return true;
}

void launch_step_fp64(cudaStream_t st, Ctl* ctl, const Params& p, StateBufs sb, Lists L,
                      MeshDev mesh, double* forces);

}  // namespace dem
