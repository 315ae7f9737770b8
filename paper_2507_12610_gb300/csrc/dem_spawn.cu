// Particle spawning (arXiv 2507.12610, Sec. 3.1, "Particle generation").
//
// One warp per spawn event.  The attempts of an event depend on each other
// (a kept sphere blocks later ones, a failed attempt hands its radius to the
// next), so they run in sequence; the lanes share the overlap test of each
// attempt: the particles of the 27 cells around the centre (binned at the
// last list rebuild; they have moved less than the skin since, and a cell is
// wider than two radii plus the skin), the spheres kept earlier in the event,
// and the mesh elements listed for the centre's cell.  Kept particles take the
// next inactive caller index, whose slot is its caller index (inactive
// particles sit at the end of the slot order in caller order, see the
// binning), and the control block asks for a list rebuild at the next step.
// A new particle cannot touch anything at the positions of this step, so it
// needs no list entries before that rebuild.
//
// Compiled without FMA contraction: the centre and radius of a kept sphere
// are the same bits as those of the plain evaluation of the same formulas.
#include "dem_geom.cuh"
#include "dem_internal.cuh"
#include "dem_math.cuh"
#include "dem_step_common.cuh"

namespace dem {

namespace {

// k-th uniform in [0, 1) of the spawn stream: SplitMix64 (Steele, Lea & Flood,
// "Fast splittable pseudorandom number generators", OOPSLA 2014) evaluated at
// seed + (k + 1) * 0x9E3779B97F4A7C15, top 53 bits.
__device__ __forceinline__ double spawn_uniform(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ double lerp_box(double lo, double hi, double u) {
  return lo + u * (hi - lo);
}

__device__ __forceinline__ void split_ff(double a, float& hi, float& lo) {
  hi = (float)a;
  lo = (float)(a - (double)hi);
}

struct Sphere {
  double x, y, z, r;
};

__device__ __forceinline__ Sphere sphere_of(const Params&, const D4& P) {
  return Sphere{P.x, P.y, P.z, P.w};
}
__device__ __forceinline__ Sphere sphere_of(const Params& p, const F8& P) {
  return Sphere{p.origin[0] + ((double)P.hi.x + (double)P.lo.x),
                p.origin[1] + ((double)P.hi.y + (double)P.lo.y),
                p.origin[2] + ((double)P.hi.z + (double)P.lo.z),
                (double)P.hi.w + (double)P.lo.w};
}

// |c - x_j| < r + R_j, written as the plain squared comparison
__device__ __forceinline__ bool overlaps(double cx, double cy, double cz, double r,
                                         const Sphere& o) {
  const double dx = cx - o.x, dy = cy - o.y, dz = cz - o.z;
  const double s = r + o.r;
  return dx * dx + dy * dy + dz * dz < s * s;
}

__device__ __forceinline__ void put_new(const Params& p, D4* P, D4* V, D4* W, D4* Q, uint32_t i,
                                        double cx, double cy, double cz, double r) {
  const double m = 4.0 / 3.0 * M_PI * p.rho * r * r * r;
  P[i] = make_D4(cx, cy, cz, r);
  V[i] = make_D4(p.sp_v0[0], p.sp_v0[1], p.sp_v0[2], m);
  W[i] = make_D4(p.sp_w0[0], p.sp_w0[1], p.sp_w0[2], 0.0);
  Q[i] = make_D4(1.0, 0.0, 0.0, 0.0);
}

__device__ __forceinline__ void put_new(const Params& p, F8* P, F8* V, F8* W, F8* Q, uint32_t i,
                                        double cx, double cy, double cz, double r) {
  const double m = 4.0 / 3.0 * M_PI * p.rho * r * r * r;
  F8 a, b, c, d;
  split_ff(cx - p.origin[0], a.hi.x, a.lo.x);
  split_ff(cy - p.origin[1], a.hi.y, a.lo.y);
  split_ff(cz - p.origin[2], a.hi.z, a.lo.z);
  split_ff(r, a.hi.w, a.lo.w);
  split_ff(p.sp_v0[0], b.hi.x, b.lo.x);
  split_ff(p.sp_v0[1], b.hi.y, b.lo.y);
  split_ff(p.sp_v0[2], b.hi.z, b.lo.z);
  b.hi.w = (float)m;
  b.lo.w = (float)(1.0 / m);
  split_ff(p.sp_w0[0], c.hi.x, c.lo.x);
  split_ff(p.sp_w0[1], c.hi.y, c.lo.y);
  split_ff(p.sp_w0[2], c.hi.z, c.lo.z);
  c.hi.w = (float)(1.0 / r);
  c.lo.w = 0.f;
  d.hi = make_float4(1.f, 0.f, 0.f, 0.f);
  d.lo = make_float4(0.f, 0.f, 0.f, 0.f);
  P[i] = a;
  V[i] = b;
  W[i] = c;
  Q[i] = d;
}

template <typename Rec>
__global__ void __launch_bounds__(32)
k_spawn(Ctl* ctl, Params p, StateBufs sb, BinBuf bb, MeshDev mesh) {
  __shared__ double kx[kSpawnMaxAttempts], ky[kSpawnMaxAttempts], kz[kSpawnMaxAttempts],
      kr[kSpawnMaxAttempts];
  if (ctl->status) return;
  if (ctl->step % p.sp_every != 0) return;
  const uint32_t A = ctl->n_active;
  if (A >= (uint32_t)p.n) return;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x;
  const uint32_t ph = ctl->phase & 1u;
  Rec* P = static_cast<Rec*>(buf_of(sb.P, ph));
  Rec* V = static_cast<Rec*>(buf_of(sb.V, ph));
  Rec* W = static_cast<Rec*>(buf_of(sb.W, ph));
  Rec* Q = static_cast<Rec*>(buf_of(sb.Q, ph));
  uint64_t draws = ctl->spawn_draws;
  double carry = ctl->spawn_carry;
  uint32_t kept = 0;
  for (int a = 0; a < p.sp_attempts && A + kept < (uint32_t)p.n; ++a) {
    double r = carry;
    if (r < 0.0) r = lerp_box(p.sp_rmin, p.sp_rmax, spawn_uniform(p.sp_seed, draws++));
    const double cx = lerp_box(p.sp_lo[0], p.sp_hi[0], spawn_uniform(p.sp_seed, draws++));
    const double cy = lerp_box(p.sp_lo[1], p.sp_hi[1], spawn_uniform(p.sp_seed, draws++));
    const double cz = lerp_box(p.sp_lo[2], p.sp_hi[2], spawn_uniform(p.sp_seed, draws++));
    bool ov = false;
    const int3 cc = cell_coords(p, (float)(cx - p.origin[0]), (float)(cy - p.origin[1]),
                                (float)(cz - p.origin[2]));
    if (lane < 27) {
      const int x = cc.x + lane % 3 - 1, y = cc.y + (lane / 3) % 3 - 1, z = cc.z + lane / 9 - 1;
      if (x >= 0 && x < p.nc[0] && y >= 0 && y < p.nc[1] && z >= 0 && z < p.nc[2]) {
        const uint32_t cell = cell_index(p, make_int3(x, y, z));
        const uint32_t e = bb.cell_start[cell + 1];
        for (uint32_t u = bb.cell_start[cell]; u < e && !ov; ++u)
          ov = overlaps(cx, cy, cz, r, sphere_of(p, P[u]));
      }
    }
    for (uint32_t k = lane; k < kept && !ov; k += 32)
      ov = overlaps(cx, cy, cz, r, Sphere{kx[k], ky[k], kz[k], kr[k]});
    if (mesh.nt > 0) {
      // the element lists are in the mesh's frame: the centre turned back by
      // the rotation of this step selects the list (the test itself is made
      // against the elements at their current pose)
      int3 cm = cc;
      if (p.omega_norm > 0.0) {
        const double th = p.omega_norm * ((double)ctl->step * p.dt);
        const double co = cos(th), si = sin(th);
        const V3<double> ax = (1.0 / p.omega_norm) *
                              mk(p.mesh_omega[0], p.mesh_omega[1], p.mesh_omega[2]);
        const V3<double> cen = mk(p.mesh_center[0], p.mesh_center[1], p.mesh_center[2]);
        const V3<double> rr = mk(cx, cy, cz) - cen;
        const V3<double> qm =
            cen + (co * rr - si * cross(ax, rr) + (dot(ax, rr) * (1.0 - co)) * ax);
        cm = cell_coords(p, (float)(qm.x - p.origin[0]), (float)(qm.y - p.origin[1]),
                         (float)(qm.z - p.origin[2]));
      }
      const uint32_t cell = cell_index(p, cm);
      const uint32_t e = min(bb.tcell_start[cell + 1], bb.tcap);
      for (uint32_t i = bb.tcell_start[cell] + lane; i < e && !ov; i += 32) {
        const uint32_t k = bb.tcell_tri[i];
        const V3<double> q = mk(cx, cy, cz);
        const V3<double> y = closest_point_element(
            q, xyz(mesh.cur[4 * k]), xyz(mesh.cur[4 * k + 1]), xyz(mesh.cur[4 * k + 2]),
            xyz(mesh.cur[4 * k + 3]), (int)mesh.curf[4 * k].w);
        ov = overlaps(cx, cy, cz, r, Sphere{y.x, y.y, y.z, mesh.rad[k]});
      }
    }
    if (__any_sync(full, ov)) {
      carry = r;
      continue;
    }
    if (lane == 0) {
      put_new(p, P, V, W, Q, A + kept, cx, cy, cz, r);
      kx[kept] = cx;
      ky[kept] = cy;
      kz[kept] = cz;
      kr[kept] = r;
    }
    __syncwarp();
    ++kept;
    carry = -1.0;
  }
  if (lane == 0) {
    ctl->n_active = A + kept;
    ctl->spawn_carry = carry;
    ctl->spawn_draws = draws;
    if (kept) ctl->force_rebuild = 1u;
  }
}

}  // namespace

void launch_spawn(cudaStream_t st, Ctl* ctl, const Params& p, StateBufs sb, BinBuf bb,
                  MeshDev mesh) {
  if (p.sp_attempts <= 0) return;
  if (p.mixed)
    k_spawn<F8><<<1, 32, 0, st>>>(ctl, p, sb, bb, mesh);
  else
    k_spawn<D4><<<1, 32, 0, st>>>(ctl, p, sb, bb, mesh);
}

}  // namespace dem
