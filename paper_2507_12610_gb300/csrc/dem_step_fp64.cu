// DEM_FP64 step kernel: contact forces, gather and integration in IEEE double
// precision (arXiv 2507.12610, Sec. 2.1-2.3).  This translation unit is
// compiled without floating-point contraction (--fmad=false), so every product
// and sum is rounded as written, as in a plain double-precision program; the
// kernel is the precision reference of the library.  The structure is the one
// described in dem_step.cu: one thread per particle slot, partners in
// ascending caller index, canonical pair orientation, no atomics on floats.
#include "dem_geom.cuh"
#include "dem_internal.cuh"
#include "dem_law.cuh"
#include "dem_math.cuh"
#include "dem_step_common.cuh"
#include "dem_step_pairs.cuh"
#include "dem_step_warp.cuh"

namespace dem {

namespace {

// ============================================================================
// DEM_FP64
// ============================================================================

#ifndef DEM_FP64_MIN_BLOCKS
#define DEM_FP64_MIN_BLOCKS 4
#endif

struct Fp64Policy {
  static constexpr int kMinBlocks = DEM_FP64_MIN_BLOCKS;  // resident blocks per SM
  using Rec = D4;
  using Hist = HistD;
  using T = double;
  using Aux = D4;  // 1/R, 1/m, 1/I of the particle (ListBuf::inv)
  static __device__ __forceinline__ Aux aux(const ListBuf& lb, uint32_t s) { return lb.inv[s]; }

  struct Acc {
    V3<double> F, T;
    __device__ __forceinline__ void zero() {
      F = mk(0.0, 0.0, 0.0);
      T = F;
    }
    __device__ __forceinline__ void add(const double* c) {
      F = F + mk(c[0], c[1], c[2]);
      T = T + mk(c[3], c[4], c[5]);
    }
    // one component at a time (plain sums: l is not used)
    static __device__ __forceinline__ void add1(double& h, double&, double v) { h = h + v; }
    __device__ __forceinline__ void set(const double* h, const double*) {
      F = mk(h[0], h[1], h[2]);
      T = mk(h[3], h[4], h[5]);
    }
  };

  struct Geo {
    double delta, dist;
    V3<double> d;
  };

  // Overlap of the canonical pair (i, j), as the paper writes it:
  // d = x_i - x_j, delta = R_i + R_j - |d|.
  static __device__ __forceinline__ bool touch(const Params&, const D4& Pi, const D4& Pj,
                                               Geo& g) {
    g.d = mk(Pi.x - Pj.x, Pi.y - Pj.y, Pi.z - Pj.z);
    const double d2 = dot(g.d, g.d);
    const double S = Pi.w + Pj.w;
    if (d2 > S * S * (1.0 + 1e-10)) return false;  // clearly apart
    g.dist = sqrt(d2);
    g.delta = S - g.dist;
    return g.delta >= 0.0 && g.dist > 0.0;
  }

  // Conservative overlap pre-test, symmetric in its arguments (the exact test
  // is touch() in canonical orientation).
  static __device__ __forceinline__ bool near(const D4& a, const D4& b) {
    const V3<double> d = mk(a.x - b.x, a.y - b.y, a.z - b.z);
    const double S = a.w + b.w;
    return dot(d, d) <= S * S * (1.0 + 1e-10);
  }

  static __device__ __forceinline__ bool pair(const Params& p, bool t_is_i, const D4& Pi,
                                              const D4& Pj, const D4& Vi, const D4& Vj,
                                              const D4& Wi, const D4& Wj, const Aux& Ai,
                                              const Aux& Aj, HistD& h, uint32_t stamp_now,
                                              uint32_t stamp_new, double c6[6]) {
    LawOut<double> o;
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
  static __device__ __forceinline__ bool pair_law(const Params& p, const D4& Pi, const D4& Pj,
                                                  const D4& Vi, const D4& Vj, const D4& Wi,
                                                  const D4& Wj, const Aux& Ai, const Aux& Aj,
                                                  HistD& h, uint32_t stamp_now, uint32_t stamp_new,
                                                  LawOut<double>& o) {
    Geo g;
    if (!touch(p, Pi, Pj, g)) return false;
    LawConst<double> cpp{p.Es_pp, p.Gs_pp, p.beta, p.mu_s, p.mu_r, p.mu_t, p.dt, p.cs_cn_pp};
    if (p.n_mat > 0) {  // the mean of the two materials' coefficients
      const D4 a = p.mat_d[(int)Wi.w], b = p.mat_d[(int)Wj.w];
      cpp.mu_s = (a.x + b.x) * 0.5;
      cpp.mu_r = (a.y + b.y) * 0.5;
      cpp.mu_t = (a.z + b.z) * 0.5;
    }
    const V3<double> nh = (1.0 / g.dist) * g.d;
    const double Ri = Pi.w, Rj = Pj.w;
    // the printed forms, in their order of operations: in a settled
    // bed the per-particle torque sums cancel to a small fraction of their
    // terms, so an algebraically equal form (R_i R_j / (R_i + R_j)) would
    // amplify its last-bit differences past the 1e-12 bound; 1/R and 1/m
    // come from the rebuild (the same divisions, done once per particle)
    const double Rs = 1.0 / (Ai.x + Aj.x);
    const double ms = 1.0 / (Ai.y + Aj.y);
    const double ri = Ri - g.delta / 2.0, rj = Rj - g.delta / 2.0;
    V3<double> us = mk(0.0, 0.0, 0.0), ur = us;
    double ut = 0.0;
    if (h.stamp == stamp_now) {
      us = mk(h.us[0], h.us[1], h.us[2]);
      ur = mk(h.ur[0], h.ur[1], h.ur[2]);
      ut = h.ut;
    }
    o = contact_law(cpp, nh, g.delta, Rs, ms, ri, rj, 1.0 / (1.0 / ri + 1.0 / rj), xyz(Vi) - xyz(Vj),
                    ri * xyz(Wi) + rj * xyz(Wj), xyz(Wi) - xyz(Wj), us, ur, ut);
    h.us[0] = us.x; h.us[1] = us.y; h.us[2] = us.z;
    h.ur[0] = ur.x; h.ur[1] = ur.y; h.ur[2] = ur.z;
    h.ut = ut;
    h.stamp = stamp_new;
    h.pad = 0;
    return true;
  }

  // Contact of particle slot t with its m-th element candidate (Sec. 2.2
  // walls, Sec. 3.3 elements): if they touch, updates the history and writes
  // the force and torque on the particle to c6.
  static __device__ __forceinline__ bool mesh_contact(const Params& p, const MeshDev& mesh,
                                                      const ListBuf& lb, int t, int m,
                                                      const D4& Pt, const D4& Vt, const D4& Wt,
                                                      uint32_t stamp_now, uint32_t stamp_new,
                                                      double c6[6]) {
    const int n = p.n;
    const uint32_t kt = lb.tric[(size_t)m * n + t];
    const V3<double> x = xyz(Pt);
    const D4 A = mesh.cur[4 * kt], B = mesh.cur[4 * kt + 1], C = mesh.cur[4 * kt + 2],
             D = mesh.cur[4 * kt + 3];
    const int nvk = (int)mesh.curf[4 * kt].w;
    const V3<double> pc = closest_point_element(x, xyz(A), xyz(B), xyz(C), xyz(D), nvk);
    const V3<double> d = x - pc;
    const double dist = sqrt(dot(d, d));
    const double delta = Pt.w + A.w - dist;
    if (delta < 0.0 || !(dist > 0.0)) return false;
    LawConst<double> cpw{p.Es_pw, p.Gs_pw, p.beta, p.mu_s, p.mu_r, p.mu_t, p.dt, p.cs_cn_pw};
    if (p.n_mat > 0) {  // the particle's material
      const D4 a = p.mat_d[(int)Wt.w];
      cpw.mu_s = a.x;
      cpw.mu_r = a.y;
      cpw.mu_t = a.z;
    }
    const V3<double> Om = mk(p.mesh_omega[0], p.mesh_omega[1], p.mesh_omega[2]);
    const V3<double> ctr = mk(p.mesh_center[0], p.mesh_center[1], p.mesh_center[2]);
    const V3<double> nh = (1.0 / dist) * d;
    const double ri = Pt.w - delta / 2.0;
    const V3<double> xc = x - ri * nh;
    const V3<double> vw = cross(Om, xc - ctr);
    HistD* hp = &static_cast<HistD*>(lb.hpm)[(size_t)m * n + t];
    const HistD h = *hp;
    V3<double> us = mk(0.0, 0.0, 0.0), ur = us;
    double ut = 0.0;
    if (h.stamp == stamp_now) {
      us = mk(h.us[0], h.us[1], h.us[2]);
      ur = mk(h.ur[0], h.ur[1], h.ur[2]);
      ut = h.ut;
    }
    const LawOut<double> o = contact_law(cpw, nh, delta, Pt.w, Vt.w, ri, 0.0, 1.0 / (1.0 / ri),
                                         xyz(Vt) - vw, ri * xyz(Wt), xyz(Wt) - Om, us, ur, ut);
    HistD hn;
    hn.us[0] = us.x; hn.us[1] = us.y; hn.us[2] = us.z;
    hn.ur[0] = ur.x; hn.ur[1] = ur.y; hn.ur[2] = ur.z;
    hn.ut = ut;
    hn.stamp = stamp_new;
    hn.pad = 0;
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
    V3<double>& F = sums.F;
    V3<double>& T = sums.T;
    // particle-element contacts
    for (int m = 0; m < ntc; ++m) {
      double c6[6];
      if (!mesh_contact(p, mesh, lb, t, m, Pt, Vt, Wt, stamp_now, stamp_new, c6)) continue;
      sums.add(c6);
      ++nmesh;
    }
    // semi-implicit Euler + SPIRAL (Sec. 2.3)
    const double R = Pt.w, mass = Vt.w;  // I = 2/5 m R^2
    const double ci = 9.0 * p.eta / (2.0 * p.rho * R * R);
    const double gi = 10.0 / 3.0 * ci;
    V3<double> v = xyz(Vt), w = xyz(Wt), x = xyz(Pt);
    const V3<double> g = mk(p.g[0], p.g[1], p.g[2]);
    const D4 iv = lb.inv[t];  // 1.0 / mass and 1.0 / I, from the rebuild
    const V3<double> a = iv.y * F + g - ci * v;
    const V3<double> al = iv.z * T - gi * w;
    v = v + p.dt * a;
    x = x + p.dt * v;
    const D4 q4 = Q[t];
    double q[4] = {q4.x, q4.y, q4.z, q4.w};
    // q (cos phi, sin phi w^) with phi = dt |w| / 2 (pre-update w), then
    // (cos th, sin th al^) with th = (dt / 2)^2 |al|
    const double hw = p.dt / 2.0;
    double r[4];
    if (rot_factor(hw, w, r)) {
      r[0] += 1.0;
      double o4[4];
      qmul(q, r, o4);
      q[0] = o4[0]; q[1] = o4[1]; q[2] = o4[2]; q[3] = o4[3];
    }
    if (rot_factor(hw * hw, al, r)) {
      r[0] += 1.0;
      double o4[4];
      qmul(q, r, o4);
      q[0] = o4[0]; q[1] = o4[1]; q[2] = o4[2]; q[3] = o4[3];
    }
    w = w + p.dt * al;
    D4* Pn = static_cast<D4*>(buf_of(sb.P, ph ^ 1u));
    D4* Vn = static_cast<D4*>(buf_of(sb.V, ph ^ 1u));
    D4* Wn = static_cast<D4*>(buf_of(sb.W, ph ^ 1u));
    D4* Qn = static_cast<D4*>(buf_of(sb.Q, ph ^ 1u));
    Pn[t] = make_D4(x.x, x.y, x.z, R);
    Vn[t] = make_D4(v.x, v.y, v.z, mass);
    Wn[t] = make_D4(w.x, w.y, w.z, Wt.w);  // .w: material index
    Qn[t] = make_D4(q[0], q[1], q[2], q[3]);
    if (p.record_forces) {
      double* fo = forces + 6 * (size_t)t;
      fo[0] = F.x; fo[1] = F.y; fo[2] = F.z;
      fo[3] = T.x; fo[4] = T.y; fo[5] = T.z;
    }
    bad = !isfinite(x.x + x.y + x.z + v.x + v.y + v.z + w.x + w.y + w.z);
    const float4 pr = lb.posf[t];
    const float ex = (float)(x.x - p.origin[0]) - pr.x, ey = (float)(x.y - p.origin[1]) - pr.y,
                ez = (float)(x.z - p.origin[2]) - pr.z;
    disp = ex * ex + ey * ey + ez * ez >= p.half_skin_trigger * p.half_skin_trigger;
    }
};

}  // namespace

void launch_step_fp64(cudaStream_t st, Ctl* ctl, const Params& p, StateBufs sb, Lists L,
                      MeshDev mesh, double* forces) {
  if (p.pair_res)  // one evaluation per pair: the FP64 pipe bounds this step
    launch_step_pairs<Fp64Policy, Fp64Policy::kMinBlocks, Fp64Policy::kMinBlocks>(
        st, ctl, p, sb, L, mesh, forces);
  else  // both sides evaluate each pair (one kernel)
    launch_step_warp<Fp64Policy>(st, ctl, p, sb, L, mesh, forces);
}

size_t pair_result_bytes() { return sizeof(PairOut<double>); }

}  // namespace dem
