// One DEM time step on the device: mesh pose, contact forces from the Verlet
// list (particle pairs and particle-triangle candidates), the per-particle
// force/torque gather, and the semi-implicit Euler + SPIRAL integration
// (arXiv 2507.12610, Sec. 2.1-2.3).
//
// One thread per particle slot.  A thread walks its list in ascending partner
// caller index, then its triangle candidates in ascending triangle index, and
// sums the contributions in exactly that order: the result is deterministic
// and independent of the launch shape, the skin and the rebuild schedule (no
// floating-point atomics anywhere).  Each touching pair is evaluated by both
// of its particles in the canonical orientation (lower caller index = body i),
// which gives both the same bits; each keeps its own copy of the friction
// history, so no thread ever reads what another thread writes in this step.
// Reading the old state and writing the new one to the other buffer keeps all
// contacts of a step at the state of t_n (as in the paper's loop).
#include "dem_geom.cuh"
#include "dem_internal.cuh"
#include "dem_law.cuh"
#include "dem_math.cuh"
#include "dem_step_common.cuh"
#include "dem_step_pairs.cuh"
#include "dem_step_warp.cuh"

namespace dem {

namespace {

// ---- mesh pose: reference vertices rotated by |Omega| t about the axis ------

// One thread per element: its vertices at the pose of step ctl->step + ahead
// (absolute in FP64; shifted as hi + lo floats), and for triangles and
// rectangles the unit normal (the reference normal, rotated) and offset of
// its plane, split the same way.  The rotation's cosine and sine are taken
// once per block.
constexpr int kPoseThreads = 128;

__global__ void __launch_bounds__(kPoseThreads)
k_mesh_pose(const Ctl* ctl, Params p, MeshDev mesh, int ahead) {
  __shared__ double s_cs[2];
  if (ctl->status) return;  // the same for every thread of the block
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t step = ctl->step + ahead;
  if (threadIdx.x == 0) {
    // the pose of this step: the same expression, so the same bits, as
    // k_set_pose, which keeps the one-thread step kernels free of FP64
    // transcendentals
    const double th = p.omega_norm * ((double)step * p.dt);
    s_cs[0] = p.omega_norm > 0.0 ? cos(th) : 1.0;
    s_cs[1] = p.omega_norm > 0.0 ? sin(th) : 0.0;
  }
  __syncthreads();
  if (k >= mesh.nt) return;
  const int4 tv = mesh.tri[k];
  const int nvk = tv.w >= 0 ? 4 : (tv.z >= 0 ? 3 : (tv.y >= 0 ? 2 : 1));
  const double rad = mesh.rad[k];
  const double wn = p.omega_norm;
  const double c = s_cs[0], s = s_cs[1];
  const V3<double> ax =
      wn > 0.0 ? (1.0 / wn) * mk(p.mesh_omega[0], p.mesh_omega[1], p.mesh_omega[2])
               : mk(0.0, 0.0, 0.0);
  const V3<double> ctr = mk(p.mesh_center[0], p.mesh_center[1], p.mesh_center[2]);
  const V3<double> org = mk(p.origin[0], p.origin[1], p.origin[2]);
  V3<double> X[4];  // shifted vertices
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int vi = j == 0 ? tv.x : (j == 1 ? tv.y : (j == 2 ? tv.z : tv.w));
    V3<double> pos = xyz(mesh.ref[j < nvk ? vi : tv.x]);
    if (wn > 0.0) {
      const V3<double> r = pos - ctr;
      pos = ctr + (c * r + s * cross(ax, r) + (dot(ax, r) * (1.0 - c)) * ax);
    }
    mesh.cur[4 * k + j] = make_D4(pos.x, pos.y, pos.z, j == 0 ? rad : 0.0);
    X[j] = pos - org;
    const float hx = (float)X[j].x, hy = (float)X[j].y, hz = (float)X[j].z;
    const float rw = j == 0 ? (float)rad : (j == 1 ? (float)(rad - (double)(float)rad) : 0.f);
    mesh.curf[4 * k + j] = make_float4(hx, hy, hz, j == 0 ? (float)nvk : 0.f);
    mesh.curl[4 * k + j] = make_float4((float)(X[j].x - hx), (float)(X[j].y - hy),
                                       (float)(X[j].z - hz), rw);
  }
  // the face normal: the reference one, rotated like the vertices
  float4 ph = make_float4(0.f, 0.f, 0.f, 0.f), pl = ph;
  if (nvk >= 3) {
    V3<double> nrm = xyz(mesh.nref[k]);
    if (wn > 0.0) nrm = c * nrm + s * cross(ax, nrm) + (dot(ax, nrm) * (1.0 - c)) * ax;
    const double off = dot(nrm, X[0]);
    ph = make_float4((float)nrm.x, (float)nrm.y, (float)nrm.z, (float)off);
    pl = make_float4((float)(nrm.x - ph.x), (float)(nrm.y - ph.y), (float)(nrm.z - ph.z),
                     (float)(off - ph.w));
  }
  mesh.plane[2 * k] = ph;
  mesh.plane[2 * k + 1] = pl;
}

// Rotation of the mesh at the control block's step (after a host upload); the
// same expression k_advance uses, so a resumed run sees the same bits.
__global__ void k_set_pose(Ctl* ctl, Params p) {
  const double th = p.omega_norm * ((double)ctl->step * p.dt);
  ctl->rot_c = cos(th);
  ctl->rot_s = sin(th);
}

// ---- graph condition: run the rebuild body of this step or skip it ----------

__global__ void k_decide(const Ctl* ctl, cudaGraphConditionalHandle h) {
  cudaGraphSetConditional(h, (ctl->rebuild != 0u && ctl->status == 0u) ? 1u : 0u);
}

// ---- end of step: flip buffers, count, decide the next rebuild -------------

__global__ void k_advance(Ctl* ctl, Params p) {
  if (ctl->status) return;
  ctl->phase ^= 1u;
  ctl->step += 1;
  ctl->pair_contacts_last = ctl->pair_contacts;
  ctl->mesh_contacts_last = ctl->mesh_contacts;
  ctl->pair_contacts = 0;
  ctl->mesh_contacts = 0;
  // mesh displacement since the last rebuild: a point at distance r from the
  // axis moves by the chord 2 r |sin(dtheta / 2)|
  bool mesh_moved = false;
  if (p.omega_norm > 0.0) {
    // the chord 2 r |sin(dtheta / 2)| is at most r |dtheta|: a bound that
    // asks for the rebuild no later than the chord itself would
    const double th = p.omega_norm * ((double)ctl->step * p.dt);
    mesh_moved = p.mesh_rmax * fabs(th - ctl->mesh_angle_ref) >= (double)p.half_skin_trigger;
  }
  ctl->rebuild = (ctl->disp_flag || ctl->force_rebuild || mesh_moved) ? 1u : 0u;
  ctl->disp_flag = 0u;
  ctl->force_rebuild = 0u;
}

// ============================================================================
// DEM_MIXED: contact arithmetic in FP32, state as compensated hi/lo pairs
// ============================================================================

__device__ __forceinline__ V3<float> hi3(float4 a) { return mk(a.x, a.y, a.z); }
// r_i w_i + r_j w_j with rounded products and a commutative sum (no
// contraction): the same bits whichever body comes first
__device__ __forceinline__ V3<float> sym_sum(float ri, V3<float> wi, float rj, V3<float> wj) {
  return mk(__fadd_rn(__fmul_rn(ri, wi.x), __fmul_rn(rj, wj.x)),
            __fadd_rn(__fmul_rn(ri, wi.y), __fmul_rn(rj, wj.y)),
            __fadd_rn(__fmul_rn(ri, wi.z), __fmul_rn(rj, wj.z)));
}
// accurate difference of two hi/lo 3-vectors, rounded once
__device__ __forceinline__ V3<float> diff3(const F8& a, const F8& b) {
  return mk((a.hi.x - b.hi.x) + (a.lo.x - b.lo.x), (a.hi.y - b.hi.y) + (a.lo.y - b.lo.y),
            (a.hi.z - b.hi.z) + (a.lo.z - b.lo.z));
}
__device__ __forceinline__ V3<float> sum3(const F8& a) {
  return mk(a.hi.x + a.lo.x, a.hi.y + a.lo.y, a.hi.z + a.lo.z);
}
// (hi, lo) + b, renormalised
__device__ __forceinline__ void acc(float& hi, float& lo, float b) {
  const ff s = ff_add_f(ff{hi, lo}, b);
  hi = s.hi;
  lo = s.lo;
}

// Resident 4-warp blocks per SM of the mixed step kernel: 8 caps it at 64
// registers (a few spilled words).  With the phase-B sums kept in shared
// memory this measured 3 % faster than 7 blocks of 72 registers; before, the
// spills of 64 registers made 8 blocks slower.
#ifndef DEM_MIXED_MIN_BLOCKS
#define DEM_MIXED_MIN_BLOCKS 8
#endif

// Overlap and unit normal (from the element to the particle) of particle
// record Pt with feature `feat` of mesh element kt, in compensated FP32: the
// element's vertices and plane are hi + lo floats in the same shifted frame as
// the particle, so q - vertex is formed exactly (same binade) and the distance
// keeps ~1e-14 m; the feature comes from the FP32 closest-point search (a
// feature chosen wrongly by rounding is off by a second-order amount, since
// neighbouring features meet with a common closest point).  Al, Bl: low words
// of the element's first two vertex slots (their .w carry the element radius).
__device__ __forceinline__ bool mesh_gap(const MeshDev& mesh, uint32_t kt, int feat,
                                         const F8& Pt, const float4& Al, const float4& Bl,
                                         float& delta, V3<float>& nh) {
  ff dist;
  if (feat == kFeatFace) {
    // signed distance n . q - c with q = hi + lo, n = hi + lo, c = hi + lo
    const float4 ph = mesh.plane[2 * kt], pl = mesh.plane[2 * kt + 1];
    ff sd = two_prod(ph.x, Pt.hi.x);
    sd = ff_add(sd, two_prod(ph.y, Pt.hi.y));
    sd = ff_add(sd, two_prod(ph.z, Pt.hi.z));
    sd = ff_add(sd, ff{-ph.w, -pl.w});
    sd = ff_add_f(sd, (ph.x * Pt.lo.x + ph.y * Pt.lo.y + ph.z * Pt.lo.z) +
                          (pl.x * Pt.hi.x + pl.y * Pt.hi.y + pl.z * Pt.hi.z));
    const float sg = sd.hi >= 0.f ? 1.f : -1.f;
    dist = ff{sg * sd.hi, sg * sd.lo};
    nh = mk(sg * ph.x, sg * ph.y, sg * ph.z);
  } else {
    // e = q - (nearest point of the vertex or edge), each component hi + lo
    const int i = feat < 4 ? feat : ((feat - 4) >> 2);
    const float4 Vh = mesh.curf[4 * kt + i];
    const float4 Vl = i == 0 ? Al : (i == 1 ? Bl : mesh.curl[4 * kt + i]);
    ff ex = two_sum(Pt.hi.x - Vh.x, Pt.lo.x - Vl.x);
    ff ey = two_sum(Pt.hi.y - Vh.y, Pt.lo.y - Vl.y);
    ff ez = two_sum(Pt.hi.z - Vh.z, Pt.lo.z - Vl.z);
    if (feat >= 4) {
      const int j = (feat - 4) & 3;
      const float4 Wh = mesh.curf[4 * kt + j];
      const float4 Wl = j == 1 ? Bl : mesh.curl[4 * kt + j];
      // edge direction u = W - V (hi part exact) and the foot parameter t in
      // FP32, then once more from the residual: an error in t moves the foot
      // along the edge, which changes the distance only to second order but
      // would tilt the normal to first order (by the error over the distance)
      const float uhx = Wh.x - Vh.x, uhy = Wh.y - Vh.y, uhz = Wh.z - Vh.z;
      const float ulx = Wl.x - Vl.x, uly = Wl.y - Vl.y, ulz = Wl.z - Vl.z;
      const V3<float> u = mk(uhx + ulx, uhy + uly, uhz + ulz);
      const float uu = dot(u, u);
      const float iuu = uu > 0.f ? 1.f / uu : 0.f;
      float tt = dot(mk(ex.hi + ex.lo, ey.hi + ey.lo, ez.hi + ez.lo), u) * iuu;
      tt = fminf(fmaxf(tt, 0.f), 1.f);
      ex = ff_add(ex, ff_add_f(two_prod(-tt, uhx), -tt * ulx));
      ey = ff_add(ey, ff_add_f(two_prod(-tt, uhy), -tt * uly));
      ez = ff_add(ez, ff_add_f(two_prod(-tt, uhz), -tt * ulz));
      if (tt > 0.f && tt < 1.f) {
        const float t2 = dot(mk(ex.hi + ex.lo, ey.hi + ey.lo, ez.hi + ez.lo), u) * iuu;
        ex = ff_add_f(ex, -t2 * u.x);
        ey = ff_add_f(ey, -t2 * u.y);
        ez = ff_add_f(ez, -t2 * u.z);
      }
    }
    // |e| = sqrt(e.e), e.e in hi + lo, one correction step for the root
    ff s2 = two_prod(ex.hi, ex.hi);
    s2.lo = __fmaf_rn(2.f * ex.hi, ex.lo, s2.lo);
    ff sy = two_prod(ey.hi, ey.hi);
    sy.lo = __fmaf_rn(2.f * ey.hi, ey.lo, sy.lo);
    ff sz = two_prod(ez.hi, ez.hi);
    sz.lo = __fmaf_rn(2.f * ez.hi, ez.lo, sz.lo);
    s2 = ff_add(ff_add(s2, sy), sz);
    const float r0 = sqrtf(s2.hi);
    if (!(r0 > 0.f)) return false;
    const float r1 = (__fmaf_rn(-r0, r0, s2.hi) + s2.lo) / (2.f * r0);
    dist = fast_two_sum(r0, r1);
    const float ir = 1.f / r0;
    nh = mk((ex.hi + ex.lo) * ir, (ey.hi + ey.lo) * ir, (ez.hi + ez.lo) * ir);
  }
  if (!(dist.hi > 0.f)) return false;
  // delta = R_i + R_j - |e|
  ff d = two_sum(Pt.hi.w, Al.w);
  d.lo += Pt.lo.w + Bl.w;
  d = ff_add(d, ff{-dist.hi, -dist.lo});
  delta = d.hi + d.lo;
  return delta >= 0.f;
}

struct MixedPolicy {
  static constexpr int kMinBlocks = DEM_MIXED_MIN_BLOCKS;  // resident blocks per SM
  using Rec = F8;
  using Hist = HistM;
  using T = float;
  using Aux = NoAux;  // the records carry 1/R and 1/m
  static __device__ __forceinline__ Aux aux(const ListBuf&, uint32_t) { return Aux{}; }

  struct Acc {
    Acc3 F, T;
    __device__ __forceinline__ void zero() {
      F.zero();
      T.zero();
    }
    __device__ __forceinline__ void add(const float* c) {
      F.add(mk(c[0], c[1], c[2]));
      T.add(mk(c[3], c[4], c[5]));
    }
    // one component at a time (h, l: that component's sum and compensation)
    static __device__ __forceinline__ void add1(float& h, float& l, float v) { kahan(h, l, v); }
    __device__ __forceinline__ void set(const float* h, const float* l) {
      F.hx = h[0]; F.hy = h[1]; F.hz = h[2]; F.lx = l[0]; F.ly = l[1]; F.lz = l[2];
      T.hx = h[3]; T.hy = h[4]; T.hz = h[5]; T.lx = l[3]; T.ly = l[4]; T.lz = l[5];
    }
  };

  struct Geo {
    float delta, dist;
    V3<float> n;
  };

  // Overlap of the canonical pair (i, j).  The hi words of the shifted
  // positions share a binade, so their difference is exact; the lo words add
  // the remaining bits.  delta = (S^2 - d^2) / (S + d) in compensated FP32.
  static __device__ __forceinline__ bool touch(const Params&, const F8& Pi, const F8& Pj,
                                               Geo& g) {
    const float dxh = Pi.hi.x - Pj.hi.x, dyh = Pi.hi.y - Pj.hi.y, dzh = Pi.hi.z - Pj.hi.z;
    const float dxl = Pi.lo.x - Pj.lo.x, dyl = Pi.lo.y - Pj.lo.y, dzl = Pi.lo.z - Pj.lo.z;
    const V3<float> dq = mk(dxh + dxl, dyh + dyl, dzh + dzl);
    const float Sf = (Pi.hi.w + Pi.lo.w) + (Pj.hi.w + Pj.lo.w);
    if (dot(dq, dq) > Sf * Sf * 1.0001f) return false;  // clearly apart
    ff sx = two_prod(dxh, dxh);
    sx.lo = __fmaf_rn(2.f * dxh, dxl, sx.lo);
    ff sy = two_prod(dyh, dyh);
    sy.lo = __fmaf_rn(2.f * dyh, dyl, sy.lo);
    ff sz = two_prod(dzh, dzh);
    sz.lo = __fmaf_rn(2.f * dzh, dzl, sz.lo);
    const ff d2 = ff_add(ff_add(sx, sy), sz);
    ff S = two_sum(Pi.hi.w, Pj.hi.w);
    S.lo += Pi.lo.w + Pj.lo.w;
    S = fast_two_sum(S.hi, S.lo);
    ff S2 = two_prod(S.hi, S.hi);
    S2.lo = __fmaf_rn(2.f * S.hi, S.lo, S2.lo);
    const ff df = ff_add(S2, ff_neg(d2));
    const float num = df.hi + df.lo;
    if (num < 0.f) return false;
    const float dist = sqrtf(d2.hi + d2.lo);
    if (!(dist > 0.f)) return false;
    g.dist = dist;
    g.delta = num / ((S.hi + S.lo) + dist);
    g.n = (1.f / dist) * dq;
    return true;
  }

  // Conservative overlap pre-test (symmetric in its arguments): FP32 centre
  // distance against (R_i + R_j) with a 1e-4 relative margin, far above its
  // rounding error.
  static __device__ __forceinline__ bool near(const F8& a, const F8& b) {
    const V3<float> dq = diff3(a, b);
    const float Sf = (a.hi.w + a.lo.w) + (b.hi.w + b.lo.w);
    return dot(dq, dq) <= Sf * Sf * 1.0001f;
  }

  // Contact law of a canonical pair: if it touches, updates the history and
  // writes the force/torque on the lane's own particle (i if t_is_i, else j)
  // to c6 and returns true.
  static __device__ __forceinline__ bool pair(const Params& p, bool t_is_i, const F8& Pi,
                                              const F8& Pj, const F8& Vi, const F8& Vj,
                                              const F8& Wi, const F8& Wj, const Aux& Ai,
                                              const Aux& Aj, HistM& h, uint32_t stamp_now,
                                              uint32_t stamp_new, float c6[6]) {
    LawOut<float> o;
    if (!pair_law(p, Pi, Pj, Vi, Vj, Wi, Wj, Ai, Aj, h, stamp_now, stamp_new, o))
      return false;
    if (t_is_i) {
      c6[0] = o.f.x; c6[1] = o.f.y; c6[2] = o.f.z;
      c6[3] = o.ti.x; c6[4] = o.ti.y; c6[5] = o.ti.z;
    } else {
      c6[0] = -o.f.x; c6[1] = -o.f.y; c6[2] = -o.f.z;
      c6[3] = o.tj.x; c6[4] = o.tj.y; c6[5] = o.tj.z;
    }
    return true;
  }

  // The law of a canonical pair (i, j): if it touches, updates the history
  // and returns the force on i and the torques on i and j.
  static __device__ __forceinline__ bool pair_law(const Params& p, const F8& Pi, const F8& Pj,
                                                  const F8& Vi, const F8& Vj, const F8& Wi,
                                                  const F8& Wj, const Aux& Ai, const Aux& Aj,
                                                  HistM& h, uint32_t stamp_now, uint32_t stamp_new,
                                                  LawOut<float>& o) {
    Geo g;
    if (!touch(p, Pi, Pj, g)) return false;
    LawConst<float> cpp{p.f_Es_pp, p.f_Gs_pp, p.f_beta, p.f_mu_s, p.f_mu_r, p.f_mu_t, p.f_dt,
                        p.f_cs_cn_pp};
    if (p.n_mat > 0) {  // the mean of the two materials' coefficients
      const float4 a = p.mat_f[__float_as_int(Wi.lo.w)], b = p.mat_f[__float_as_int(Wj.lo.w)];
      cpp.mu_s = (a.x + b.x) * 0.5f;
      cpp.mu_r = (a.y + b.y) * 0.5f;
      cpp.mu_t = (a.z + b.z) * 0.5f;
    }
    const float Ri = Pi.hi.w + Pi.lo.w, Rj = Pj.hi.w + Pj.lo.w;
    const float Rs = 1.f / (Wi.hi.w + Wj.hi.w);  // records carry 1/R and 1/m
    const float ms = 1.f / (Vi.lo.w + Vj.lo.w);
    const float ri = Ri - 0.5f * g.delta, rj = Rj - 0.5f * g.delta;
    V3<float> us = mk(0.f, 0.f, 0.f), ur = us;
    float ut = 0.f;
    if (h.stamp == stamp_now) {
      us = mk(h.us[0], h.us[1], h.us[2]);
      ur = mk(h.ur[0], h.ur[1], h.ur[2]);
      ut = h.ut;
    }
    o = contact_law(cpp, g.n, g.delta, Rs, ms, ri, rj, ri * rj / (ri + rj), diff3(Vi, Vj),
                    sym_sum(ri, sum3(Wi), rj, sum3(Wj)), diff3(Wi, Wj), us, ur, ut);
    h.us[0] = us.x; h.us[1] = us.y; h.us[2] = us.z;
    h.ur[0] = ur.x; h.ur[1] = ur.y; h.ur[2] = ur.z;
    h.ut = ut;
    h.stamp = stamp_new;
    return true;
  }

  // Contact of particle slot t with its m-th element candidate: the FP32
  // closest point as a pre-filter and to pick the nearest feature, then the
  // overlap in compensated FP32 (an element is large compared with the
  // overlap).  If they touch, updates the history and writes the force and
  // torque on the particle to c6.
  static __device__ __forceinline__ bool mesh_contact(const Params& p, const MeshDev& mesh,
                                                      const ListBuf& lb, int t, int m,
                                                      const F8& Pt, const F8& Vt, const F8& Wt,
                                                      uint32_t stamp_now, uint32_t stamp_new,
                                                      float c6[6]) {
    const int n = p.n;
    const float Rt = Pt.hi.w + Pt.lo.w;
    const uint32_t kt = lb.tric[(size_t)m * n + t];
    const V3<float> qf = sum3(Pt);
    const float4 Af = mesh.curf[4 * kt], Bf = mesh.curf[4 * kt + 1],
                 Cf = mesh.curf[4 * kt + 2], Df = mesh.curf[4 * kt + 3];
    const int nvk = (int)Af.w;
    int feat;
    const V3<float> yf = closest_point_element(qf, hi3(Af), hi3(Bf), hi3(Cf), hi3(Df), nvk, feat);
    const V3<float> df = qf - yf;
    const float4 Al = mesh.curl[4 * kt], Bl = mesh.curl[4 * kt + 1];
    const float reachf = Rt + Al.w + p.mesh_prefilter;
    if (dot(df, df) > reachf * reachf) return false;
    float delta;
    V3<float> nh;
    if (!mesh_gap(mesh, kt, feat, Pt, Al, Bl, delta, nh)) return false;
    LawConst<float> cpw{p.f_Es_pw, p.f_Gs_pw, p.f_beta, p.f_mu_s, p.f_mu_r, p.f_mu_t, p.f_dt,
                        p.f_cs_cn_pw};
    if (p.n_mat > 0) {  // the particle's material
      const float4 a = p.mat_f[__float_as_int(Wt.lo.w)];
      cpw.mu_s = a.x;
      cpw.mu_r = a.y;
      cpw.mu_t = a.z;
    }
    const V3<float> Om = mk(p.f_omega[0], p.f_omega[1], p.f_omega[2]);
    // particle centre relative to the rotation axis point, accurately
    const V3<float> rc = mk((Pt.hi.x - p.center_hi[0]) + (Pt.lo.x - p.center_lo[0]),
                            (Pt.hi.y - p.center_hi[1]) + (Pt.lo.y - p.center_lo[1]),
                            (Pt.hi.z - p.center_hi[2]) + (Pt.lo.z - p.center_lo[2]));
    const float ri = Rt - 0.5f * delta;
    const V3<float> vw = cross(Om, rc - ri * nh);
    HistM* hp = &static_cast<HistM*>(lb.hpm)[(size_t)m * n + t];
    const HistM h = *hp;
    V3<float> us = mk(0.f, 0.f, 0.f), ur = us;
    float ut = 0.f;
    if (h.stamp == stamp_now) {
      us = mk(h.us[0], h.us[1], h.us[2]);
      ur = mk(h.ur[0], h.ur[1], h.ur[2]);
      ut = h.ut;
    }
    const V3<float> dv = mk((Vt.hi.x - vw.x) + Vt.lo.x, (Vt.hi.y - vw.y) + Vt.lo.y,
                            (Vt.hi.z - vw.z) + Vt.lo.z);
    const V3<float> om = mk((Wt.hi.x - Om.x) + Wt.lo.x, (Wt.hi.y - Om.y) + Wt.lo.y,
                            (Wt.hi.z - Om.z) + Wt.lo.z);
    const LawOut<float> o = contact_law(cpw, nh, delta, Rt, Vt.hi.w, ri, 0.f, ri, dv,
                                        ri * sum3(Wt), om, us, ur, ut);
    HistM hn;
    hn.us[0] = us.x; hn.us[1] = us.y; hn.us[2] = us.z;
    hn.ur[0] = ur.x; hn.ur[1] = ur.y; hn.ur[2] = ur.z;
    hn.ut = ut;
    hn.stamp = stamp_new;
    *hp = hn;
    c6[0] = o.f.x; c6[1] = o.f.y; c6[2] = o.f.z;
    c6[3] = o.ti.x; c6[4] = o.ti.y; c6[5] = o.ti.z;
    return true;
  }

  // Element contacts (unless the caller took them already: with_mesh false)
  // and integration of particle slot t.
  static __device__ __forceinline__ void finish(const Params& p, const StateBufs& sb,
                                                uint32_t ph, const ListBuf& lb,
                                                const MeshDev& mesh, int t, uint32_t ntc_u,
                                                bool with_mesh, const F8& Pt, const F8& Vt,
                                                const F8& Wt, Acc& sums, uint32_t stamp_now,
                                                uint32_t stamp_new, double* forces,
                                                uint32_t& nmesh, bool& disp, bool& bad) {
    const int ntc = with_mesh ? (int)ntc_u : 0;
    const F8* Q = static_cast<const F8*>(buf_of(sb.Q, ph));
    const float Rt = Pt.hi.w + Pt.lo.w;
    if (Rt == 0.f) {  // inactive (awaiting spawning): carried over unchanged
      static_cast<F8*>(buf_of(sb.P, ph ^ 1u))[t] = Pt;
      static_cast<F8*>(buf_of(sb.V, ph ^ 1u))[t] = Vt;
      static_cast<F8*>(buf_of(sb.W, ph ^ 1u))[t] = Wt;
      static_cast<F8*>(buf_of(sb.Q, ph ^ 1u))[t] = Q[t];
      if (p.record_forces)
        for (int c = 0; c < 6; ++c) forces[6 * (size_t)t + c] = 0.0;
      return;
    }
    Acc3& F = sums.F;
    Acc3& T = sums.T;
    for (int m = 0; m < ntc; ++m) {
      float c6[6];
      if (!mesh_contact(p, mesh, lb, t, m, Pt, Vt, Wt, stamp_now, stamp_new, c6)) continue;
      sums.add(c6);
      ++nmesh;
    }
    // semi-implicit Euler + SPIRAL with compensated (hi, lo) state
    const float mass = Vt.hi.w;
    const float R = Rt;
    const float I = 0.4f * mass * R * R;
    const float ci = p.f_drag / (R * R);
    const float gi = 10.f / 3.f * ci;
    const float dt = p.f_dt;
    const V3<float> v0 = sum3(Vt), w0 = sum3(Wt);
    const float im = Vt.lo.w, iI = 1.f / I;
    const V3<float> a = mk((F.hx + F.lx) * im + p.f_g[0] - ci * v0.x,
                           (F.hy + F.ly) * im + p.f_g[1] - ci * v0.y,
                           (F.hz + F.lz) * im + p.f_g[2] - ci * v0.z);
    const V3<float> al = mk((T.hx + T.lx) * iI - gi * w0.x, (T.hy + T.ly) * iI - gi * w0.y,
                            (T.hz + T.lz) * iI - gi * w0.z);
    F8 Vn = Vt, Pn = Pt, Wn = Wt, Qn = Q[t];
    acc(Vn.hi.x, Vn.lo.x, dt * a.x);
    acc(Vn.hi.y, Vn.lo.y, dt * a.y);
    acc(Vn.hi.z, Vn.lo.z, dt * a.z);
    acc(Pn.hi.x, Pn.lo.x, dt * Vn.hi.x + dt * Vn.lo.x);
    acc(Pn.hi.y, Pn.lo.y, dt * Vn.hi.y + dt * Vn.lo.y);
    acc(Pn.hi.z, Pn.lo.z, dt * Vn.hi.z + dt * Vn.lo.z);
    // orientation: q <- q (cos phi, sin phi w^) (cos th, sin th al^), applied as
    // q + q (cos - 1, sin axis) so the small increment is formed in FP32 and
    // added to the compensated quaternion
    float r[4];
    if (rot_factor(0.5f * dt, w0, r)) {
      const float qh[4] = {Qn.hi.x + Qn.lo.x, Qn.hi.y + Qn.lo.y, Qn.hi.z + Qn.lo.z,
                           Qn.hi.w + Qn.lo.w};
      float dq[4];
      qmul(qh, r, dq);
      acc(Qn.hi.x, Qn.lo.x, dq[0]);
      acc(Qn.hi.y, Qn.lo.y, dq[1]);
      acc(Qn.hi.z, Qn.lo.z, dq[2]);
      acc(Qn.hi.w, Qn.lo.w, dq[3]);
    }
    if (rot_factor((0.5f * dt) * (0.5f * dt), al, r)) {
      const float qh[4] = {Qn.hi.x + Qn.lo.x, Qn.hi.y + Qn.lo.y, Qn.hi.z + Qn.lo.z,
                           Qn.hi.w + Qn.lo.w};
      float dq[4];
      qmul(qh, r, dq);
      acc(Qn.hi.x, Qn.lo.x, dq[0]);
      acc(Qn.hi.y, Qn.lo.y, dq[1]);
      acc(Qn.hi.z, Qn.lo.z, dq[2]);
      acc(Qn.hi.w, Qn.lo.w, dq[3]);
    }
    acc(Wn.hi.x, Wn.lo.x, dt * al.x);
    acc(Wn.hi.y, Wn.lo.y, dt * al.y);
    acc(Wn.hi.z, Wn.lo.z, dt * al.z);
    static_cast<F8*>(buf_of(sb.P, ph ^ 1u))[t] = Pn;
    static_cast<F8*>(buf_of(sb.V, ph ^ 1u))[t] = Vn;
    static_cast<F8*>(buf_of(sb.W, ph ^ 1u))[t] = Wn;
    static_cast<F8*>(buf_of(sb.Q, ph ^ 1u))[t] = Qn;
    if (p.record_forces) {
      double* fo = forces + 6 * (size_t)t;
      fo[0] = (double)F.hx + (double)F.lx;
      fo[1] = (double)F.hy + (double)F.ly;
      fo[2] = (double)F.hz + (double)F.lz;
      fo[3] = (double)T.hx + (double)T.lx;
      fo[4] = (double)T.hy + (double)T.ly;
      fo[5] = (double)T.hz + (double)T.lz;
    }
    bad = !isfinite(Pn.hi.x + Pn.hi.y + Pn.hi.z + Vn.hi.x + Vn.hi.y + Vn.hi.z + Wn.hi.x +
                    Wn.hi.y + Wn.hi.z);
    const float4 pr = lb.posf[t];
    const float ex = (Pn.hi.x - pr.x) + Pn.lo.x, ey = (Pn.hi.y - pr.y) + Pn.lo.y,
                ez = (Pn.hi.z - pr.z) + Pn.lo.z;
    disp = ex * ex + ey * ey + ez * ez >= p.half_skin_trigger * p.half_skin_trigger;
    }
};


// ============================================================================
// DEM_MIXED64: contact law and springs in FP32, state stored and accumulated
// in FP64 (the FP32-force / FP64-position mode)
// ============================================================================

#ifndef DEM_MIXED64_MIN_BLOCKS
#define DEM_MIXED64_MIN_BLOCKS 6
#endif

struct Mixed64Policy {
  static constexpr int kMinBlocks = DEM_MIXED64_MIN_BLOCKS;
  using Rec = D4;
  using Hist = HistM;
  using T = float;
  using Acc = MixedPolicy::Acc;
  using Aux = NoAux;
  static __device__ __forceinline__ Aux aux(const ListBuf&, uint32_t) { return Aux{}; }

  // Conservative pre-test: the offset in FP64, the comparison in FP32 with a
  // 1e-4 relative margin (symmetric in its arguments).
  static __device__ __forceinline__ bool near(const D4& a, const D4& b) {
    const float dx = (float)(a.x - b.x), dy = (float)(a.y - b.y), dz = (float)(a.z - b.z);
    const float S = (float)(a.w + b.w);
    return dx * dx + dy * dy + dz * dz <= S * S * 1.0001f;
  }

  static __device__ __forceinline__ bool pair(const Params& p, bool t_is_i, const D4& Pi,
                                              const D4& Pj, const D4& Vi, const D4& Vj,
                                              const D4& Wi, const D4& Wj, const Aux& Ai,
                                              const Aux& Aj, HistM& h, uint32_t stamp_now,
                                              uint32_t stamp_new, float c6[6]) {
    LawOut<float> o;
    if (!pair_law(p, Pi, Pj, Vi, Vj, Wi, Wj, Ai, Aj, h, stamp_now, stamp_new, o))
      return false;
    if (t_is_i) {
      c6[0] = o.f.x; c6[1] = o.f.y; c6[2] = o.f.z;
      c6[3] = o.ti.x; c6[4] = o.ti.y; c6[5] = o.ti.z;
    } else {
      c6[0] = -o.f.x; c6[1] = -o.f.y; c6[2] = -o.f.z;
      c6[3] = o.tj.x; c6[4] = o.tj.y; c6[5] = o.tj.z;
    }
    return true;
  }

  // The canonical pair (i, j): the offset and S^2 - d^2 = (S - d)(S + d) in
  // FP64 (the overlap is a small difference of two millimetre lengths; the
  // product form keeps it without a double-precision root), then the root and
  // the overlap (S^2 - d^2) / (S + d) in FP32, and everything after that in
  // FP32.  Velocity and spin differences are formed in FP64 before rounding,
  // so they keep their relative accuracy.
  static __device__ __forceinline__ bool pair_law(const Params& p, const D4& Pi, const D4& Pj,
                                                  const D4& Vi, const D4& Vj, const D4& Wi,
                                                  const D4& Wj, const Aux& Ai, const Aux& Aj,
                                                  HistM& h, uint32_t stamp_now, uint32_t stamp_new,
                                                  LawOut<float>& o) {
    const double dx = Pi.x - Pj.x, dy = Pi.y - Pj.y, dz = Pi.z - Pj.z;
    const double d2 = dx * dx + dy * dy + dz * dz;
    const double S = Pi.w + Pj.w;
    const double num = S * S - d2;
    if (!(num >= 0.0)) return false;  // apart
    const float dist = sqrtf((float)d2);
    if (!(dist > 0.f)) return false;
    const float delta = (float)num / ((float)S + dist);
    const float idist = 1.f / dist;
    const V3<float> nh = mk((float)dx * idist, (float)dy * idist, (float)dz * idist);
    LawConst<float> cpp{p.f_Es_pp, p.f_Gs_pp, p.f_beta, p.f_mu_s, p.f_mu_r, p.f_mu_t, p.f_dt,
                        p.f_cs_cn_pp};
    if (p.n_mat > 0) {  // the mean of the two materials' coefficients
      const float4 a = p.mat_f[(int)Wi.w], b = p.mat_f[(int)Wj.w];
      cpp.mu_s = (a.x + b.x) * 0.5f;
      cpp.mu_r = (a.y + b.y) * 0.5f;
      cpp.mu_t = (a.z + b.z) * 0.5f;
    }
    const float Ri = (float)Pi.w, Rj = (float)Pj.w;
    const float mi = (float)Vi.w, mj = (float)Vj.w;
    const float Rs = Ri * Rj / (Ri + Rj), ms = mi * mj / (mi + mj);
    const float ri = Ri - 0.5f * delta, rj = Rj - 0.5f * delta;
    V3<float> us = mk(0.f, 0.f, 0.f), ur = us;
    float ut = 0.f;
    if (h.stamp == stamp_now) {
      us = mk(h.us[0], h.us[1], h.us[2]);
      ur = mk(h.ur[0], h.ur[1], h.ur[2]);
      ut = h.ut;
    }
    const V3<float> wi = mk((float)Wi.x, (float)Wi.y, (float)Wi.z);
    const V3<float> wj = mk((float)Wj.x, (float)Wj.y, (float)Wj.z);
    const V3<float> dv = mk((float)(Vi.x - Vj.x), (float)(Vi.y - Vj.y), (float)(Vi.z - Vj.z));
    const V3<float> om = mk((float)(Wi.x - Wj.x), (float)(Wi.y - Wj.y), (float)(Wi.z - Wj.z));
    o = contact_law(cpp, nh, delta, Rs, ms, ri, rj, ri * rj / (ri + rj), dv,
                    sym_sum(ri, wi, rj, wj), om, us, ur, ut);
    h.us[0] = us.x; h.us[1] = us.y; h.us[2] = us.z;
    h.ur[0] = ur.x; h.ur[1] = ur.y; h.ur[2] = ur.z;
    h.ut = ut;
    h.stamp = stamp_new;
    return true;
  }

  // Particle slot t and its m-th element candidate: the closest point and the
  // overlap in FP64 (an element is large next to the overlap), the law in FP32.
  static __device__ __forceinline__ bool mesh_contact(const Params& p, const MeshDev& mesh,
                                                      const ListBuf& lb, int t, int m,
                                                      const D4& Pt, const D4& Vt, const D4& Wt,
                                                      uint32_t stamp_now, uint32_t stamp_new,
                                                      float c6[6]) {
    const int n = p.n;
    const uint32_t kt = lb.tric[(size_t)m * n + t];
    const V3<double> x = xyz(Pt);
    const D4 A = mesh.cur[4 * kt], B = mesh.cur[4 * kt + 1], C = mesh.cur[4 * kt + 2],
             D = mesh.cur[4 * kt + 3];
    const int nvk = (int)mesh.curf[4 * kt].w;
    const V3<double> pc = closest_point_element(x, xyz(A), xyz(B), xyz(C), xyz(D), nvk);
    const V3<double> d = x - pc;
    const double dist = sqrt(dot(d, d));
    const double deltad = Pt.w + A.w - dist;
    if (deltad < 0.0 || !(dist > 0.0)) return false;
    const float delta = (float)deltad;
    const float idist = 1.f / (float)dist;
    const V3<float> nh = mk((float)d.x * idist, (float)d.y * idist, (float)d.z * idist);
    LawConst<float> cpw{p.f_Es_pw, p.f_Gs_pw, p.f_beta, p.f_mu_s, p.f_mu_r, p.f_mu_t, p.f_dt,
                        p.f_cs_cn_pw};
    if (p.n_mat > 0) {  // the particle's material
      const float4 a = p.mat_f[(int)Wt.w];
      cpw.mu_s = a.x;
      cpw.mu_r = a.y;
      cpw.mu_t = a.z;
    }
    const float Rt = (float)Pt.w;
    const float ri = Rt - 0.5f * delta;
    const V3<float> Om = mk(p.f_omega[0], p.f_omega[1], p.f_omega[2]);
    const V3<float> rc = mk((float)(x.x - p.mesh_center[0]), (float)(x.y - p.mesh_center[1]),
                            (float)(x.z - p.mesh_center[2]));
    const V3<float> vw = cross(Om, rc - ri * nh);
    HistM* hp = &static_cast<HistM*>(lb.hpm)[(size_t)m * n + t];
    const HistM h = *hp;
    V3<float> us = mk(0.f, 0.f, 0.f), ur = us;
    float ut = 0.f;
    if (h.stamp == stamp_now) {
      us = mk(h.us[0], h.us[1], h.us[2]);
      ur = mk(h.ur[0], h.ur[1], h.ur[2]);
      ut = h.ut;
    }
    const V3<float> dv = mk((float)(Vt.x - (double)vw.x), (float)(Vt.y - (double)vw.y),
                            (float)(Vt.z - (double)vw.z));
    const V3<float> wt = mk((float)Wt.x, (float)Wt.y, (float)Wt.z);
    const LawOut<float> o = contact_law(cpw, nh, delta, Rt, (float)Vt.w, ri, 0.f, ri, dv,
                                        ri * wt, wt - Om, us, ur, ut);
    HistM hn;
    hn.us[0] = us.x; hn.us[1] = us.y; hn.us[2] = us.z;
    hn.ur[0] = ur.x; hn.ur[1] = ur.y; hn.ur[2] = ur.z;
    hn.ut = ut;
    hn.stamp = stamp_new;
    *hp = hn;
    c6[0] = o.f.x; c6[1] = o.f.y; c6[2] = o.f.z;
    c6[3] = o.ti.x; c6[4] = o.ti.y; c6[5] = o.ti.z;
    return true;
  }

  // Element contacts (unless taken already) and integration of slot t: the
  // accelerations and the SPIRAL increment in FP32 (from FP32 forces), added
  // to the FP64 velocity, spin and orientation; positions advance in FP64.
  static __device__ __forceinline__ void finish(const Params& p, const StateBufs& sb,
                                                uint32_t ph, const ListBuf& lb,
                                                const MeshDev& mesh, int t, uint32_t ntc_u,
                                                bool with_mesh, const D4& Pt, const D4& Vt,
                                                const D4& Wt, Acc& sums, uint32_t stamp_now,
                                                uint32_t stamp_new, double* forces,
                                                uint32_t& nmesh, bool& disp, bool& bad) {
    const int ntc = with_mesh ? (int)ntc_u : 0;
    const D4* Q = static_cast<const D4*>(buf_of(sb.Q, ph));
    if (Pt.w == 0.0) {  // inactive (awaiting spawning): carried over unchanged
      static_cast<D4*>(buf_of(sb.P, ph ^ 1u))[t] = Pt;
      static_cast<D4*>(buf_of(sb.V, ph ^ 1u))[t] = Vt;
      static_cast<D4*>(buf_of(sb.W, ph ^ 1u))[t] = Wt;
      static_cast<D4*>(buf_of(sb.Q, ph ^ 1u))[t] = Q[t];
      if (p.record_forces)
        for (int c = 0; c < 6; ++c) forces[6 * (size_t)t + c] = 0.0;
      return;
    }
    for (int m = 0; m < ntc; ++m) {
      float c6[6];
      if (!mesh_contact(p, mesh, lb, t, m, Pt, Vt, Wt, stamp_now, stamp_new, c6)) continue;
      sums.add(c6);
      ++nmesh;
    }
    const Acc3& F = sums.F;
    const Acc3& T = sums.T;
    const float R = (float)Pt.w, mass = (float)Vt.w;
    const float I = 0.4f * mass * R * R;
    const float ci = p.f_drag / (R * R), gi = 10.f / 3.f * ci;
    const V3<float> v0 = mk((float)Vt.x, (float)Vt.y, (float)Vt.z);
    const V3<float> w0 = mk((float)Wt.x, (float)Wt.y, (float)Wt.z);
    const float im = 1.f / mass, iI = 1.f / I;
    const V3<float> a = mk((F.hx + F.lx) * im + p.f_g[0] - ci * v0.x,
                           (F.hy + F.ly) * im + p.f_g[1] - ci * v0.y,
                           (F.hz + F.lz) * im + p.f_g[2] - ci * v0.z);
    const V3<float> al = mk((T.hx + T.lx) * iI - gi * w0.x, (T.hy + T.ly) * iI - gi * w0.y,
                            (T.hz + T.lz) * iI - gi * w0.z);
    const double dt = p.dt;
    const V3<double> v = mk(Vt.x + dt * (double)a.x, Vt.y + dt * (double)a.y,
                            Vt.z + dt * (double)a.z);
    const V3<double> x = mk(Pt.x + dt * v.x, Pt.y + dt * v.y, Pt.z + dt * v.z);
    // orientation: q <- q + q (cos phi - 1, sin phi w^), then the same with
    // the angular acceleration; each increment in FP32, the sum in FP64
    const D4 q4 = Q[t];
    double q[4] = {q4.x, q4.y, q4.z, q4.w};
    float r[4];
    for (int pass = 0; pass < 2; ++pass) {
      const bool turn = pass == 0 ? rot_factor(0.5f * p.f_dt, w0, r)
                                  : rot_factor((0.5f * p.f_dt) * (0.5f * p.f_dt), al, r);
      if (!turn) continue;
      const float qf[4] = {(float)q[0], (float)q[1], (float)q[2], (float)q[3]};
      float dq[4];
      qmul(qf, r, dq);
      for (int c = 0; c < 4; ++c) q[c] += (double)dq[c];
    }
    const V3<double> w = mk(Wt.x + dt * (double)al.x, Wt.y + dt * (double)al.y,
                            Wt.z + dt * (double)al.z);
    static_cast<D4*>(buf_of(sb.P, ph ^ 1u))[t] = make_D4(x.x, x.y, x.z, Pt.w);
    static_cast<D4*>(buf_of(sb.V, ph ^ 1u))[t] = make_D4(v.x, v.y, v.z, Vt.w);
    static_cast<D4*>(buf_of(sb.W, ph ^ 1u))[t] = make_D4(w.x, w.y, w.z, Wt.w);
    static_cast<D4*>(buf_of(sb.Q, ph ^ 1u))[t] = make_D4(q[0], q[1], q[2], q[3]);
    if (p.record_forces) {
      double* fo = forces + 6 * (size_t)t;
      fo[0] = (double)F.hx + (double)F.lx;
      fo[1] = (double)F.hy + (double)F.ly;
      fo[2] = (double)F.hz + (double)F.lz;
      fo[3] = (double)T.hx + (double)T.lx;
      fo[4] = (double)T.hy + (double)T.ly;
      fo[5] = (double)T.hz + (double)T.lz;
    }
    bad = !isfinite(x.x + x.y + x.z + v.x + v.y + v.z + w.x + w.y + w.z);
    const float4 pr = lb.posf[t];
    const float ex = (float)(x.x - p.origin[0]) - pr.x, ey = (float)(x.y - p.origin[1]) - pr.y,
                ez = (float)(x.z - p.origin[2]) - pr.z;
    disp = ex * ex + ey * ey + ez * ez >= p.half_skin_trigger * p.half_skin_trigger;
  }
};

}  // namespace

void launch_mesh_pose(cudaStream_t st, const Ctl* ctl, const Params& p, MeshDev mesh, int ahead) {
  if (mesh.nt <= 0) return;
  k_mesh_pose<<<(unsigned)((mesh.nt + kPoseThreads - 1) / kPoseThreads), kPoseThreads, 0, st>>>(
      ctl, p, mesh, ahead);
}

void launch_step(cudaStream_t st, Ctl* ctl, const Params& p, StateBufs sb, Lists L,
                 MeshDev mesh, double* forces) {
  if (p.mixed && p.pair_res)  // one evaluation per pair
    launch_step_pairs<MixedPolicy, MixedPolicy::kMinBlocks, MixedPolicy::kMinBlocks>(
        st, ctl, p, sb, L, mesh, forces);
  else if (p.mixed)
    launch_step_warp<MixedPolicy>(st, ctl, p, sb, L, mesh, forces);
  else if (p.mixed64)
    launch_step_warp<Mixed64Policy>(st, ctl, p, sb, L, mesh, forces);
  else
    launch_step_fp64(st, ctl, p, sb, L, mesh, forces);
}

void launch_set_pose(cudaStream_t st, Ctl* ctl, const Params& p) {
  k_set_pose<<<1, 1, 0, st>>>(ctl, p);
}

void launch_decide(cudaStream_t st, const Ctl* ctl, cudaGraphConditionalHandle h) {
  k_decide<<<1, 1, 0, st>>>(ctl, h);
}

void launch_advance(cudaStream_t st, Ctl* ctl, const Params& p) {
  k_advance<<<1, 1, 0, st>>>(ctl, p);
}

}  // namespace dem
