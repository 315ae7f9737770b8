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

void launch_step_fp64(cudaStream_t st, Ctl* ctl, const Params& p, StateBufs sb, Lists L,
                      MeshDev mesh, double* forces);

}  // namespace dem
