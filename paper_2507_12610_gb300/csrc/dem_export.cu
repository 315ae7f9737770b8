// State read-back on the device: the current records (slot order, shifted,
// hi/lo in DEM_MIXED) converted to absolute double values in caller order,
// into a staging buffer that the host then copies out in one transfer per
// array.  Inactive rows (awaiting spawning) read as zero vectors and the
// identity quaternion.  Additions only (compiled without contraction), so the
// values are those of the same sums taken on the host.
#include <type_traits>

#include "dem_internal.cuh"

namespace dem {

namespace {

__device__ __forceinline__ double sum2(float hi, float lo) { return (double)hi + (double)lo; }

template <typename Rec>
__global__ void k_export_state(const Ctl* ctl, Params p, StateBufs sb, Lists L, int64_t n,
                               double* out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const uint32_t ph = ctl->phase & 1u;
  const ListBuf lb = list_of(L, ctl->lphase & 1u);
  const Rec* P = static_cast<const Rec*>(buf_of(sb.P, ph));
  const Rec* V = static_cast<const Rec*>(buf_of(sb.V, ph));
  const Rec* W = static_cast<const Rec*>(buf_of(sb.W, ph));
  const Rec* Q = static_cast<const Rec*>(buf_of(sb.Q, ph));
  const int64_t i = lb.gid[t];
  double* x = out + 3 * i;
  double* v = out + 3 * n + 3 * i;
  double* w = out + 6 * n + 3 * i;
  double* q = out + 9 * n + 4 * i;
  const Rec Pt = P[t];
  bool inactive;
  double xs[3], vs[3], ws[3], qs[4];
  if constexpr (std::is_same<Rec, F8>::value) {
    const F8 Vt = V[t], Wt = W[t], Qt = Q[t];
    inactive = Pt.hi.w == 0.f;
    xs[0] = p.origin[0] + sum2(Pt.hi.x, Pt.lo.x);
    xs[1] = p.origin[1] + sum2(Pt.hi.y, Pt.lo.y);
    xs[2] = p.origin[2] + sum2(Pt.hi.z, Pt.lo.z);
    vs[0] = sum2(Vt.hi.x, Vt.lo.x); vs[1] = sum2(Vt.hi.y, Vt.lo.y); vs[2] = sum2(Vt.hi.z, Vt.lo.z);
    ws[0] = sum2(Wt.hi.x, Wt.lo.x); ws[1] = sum2(Wt.hi.y, Wt.lo.y); ws[2] = sum2(Wt.hi.z, Wt.lo.z);
    qs[0] = sum2(Qt.hi.x, Qt.lo.x); qs[1] = sum2(Qt.hi.y, Qt.lo.y);
    qs[2] = sum2(Qt.hi.z, Qt.lo.z); qs[3] = sum2(Qt.hi.w, Qt.lo.w);
  } else {
    const D4 Vt = V[t], Wt = W[t], Qt = Q[t];
    inactive = Pt.w == 0.0;
    xs[0] = Pt.x; xs[1] = Pt.y; xs[2] = Pt.z;
    vs[0] = Vt.x; vs[1] = Vt.y; vs[2] = Vt.z;
    ws[0] = Wt.x; ws[1] = Wt.y; ws[2] = Wt.z;
    qs[0] = Qt.x; qs[1] = Qt.y; qs[2] = Qt.z; qs[3] = Qt.w;
  }
  if (inactive) {
    for (int a = 0; a < 3; ++a) xs[a] = vs[a] = ws[a] = 0.0;
    qs[0] = 1.0;
    qs[1] = qs[2] = qs[3] = 0.0;
  }
  for (int a = 0; a < 3; ++a) {
    x[a] = xs[a];
    v[a] = vs[a];
    w[a] = ws[a];
  }
  for (int a = 0; a < 4; ++a) q[a] = qs[a];
}

}  // namespace

void launch_export_state(cudaStream_t st, const Ctl* ctl, const Params& p, StateBufs sb,
                         Lists L, int64_t n, double* out) {
  if (n <= 0) return;
  const unsigned nb = (unsigned)((n + 255) / 256);
  if (p.mixed)
    k_export_state<F8><<<nb, 256, 0, st>>>(ctl, p, sb, L, n, out);
  else
    k_export_state<D4><<<nb, 256, 0, st>>>(ctl, p, sb, L, n, out);
}

}  // namespace dem
