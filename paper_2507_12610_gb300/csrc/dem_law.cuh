// The contact law of arXiv 2507.12610, Sec. 2.2-2.3, for one contact, in
// precision T (double for DEM_FP64, float for DEM_MIXED).
//
// Inputs are already in the canonical orientation: body i is the particle
// with the lower caller index (or the particle of a particle-wall contact),
// n points from body j to body i.  Both particles of a pair evaluate the same
// call with the same inputs, so they obtain bitwise identical results and each
// keeps an identical copy of the pair's friction history.
#pragma once

#include "dem_math.cuh"

namespace dem {

template <typename T>
struct LawConst {
  T Es, Gs;      // effective moduli for this kind of contact (pair or wall)
  T beta;        // damping factor of e_n
  T mu_s, mu_r, mu_t;
  T dt;
  T cs_cn;       // c_s / c_n = sqrt(G* / (5 E*)) (Eqs. cn, cs with k_s / k_n = 6 G* / E*);
                 // used in single precision only
};

template <typename T>
struct LawOut {
  V3<T> f;     // force on i: f_n + f_s
  V3<T> ti;    // torque on i: tau_s + tau_r + tau_t
  V3<T> tj;    // torque on j: r_j f_s x n - tau_r - tau_t (pairs only)
};

__device__ __forceinline__ double vabs(double a) { return fabs(a); }
__device__ __forceinline__ float vabs(float a) { return fabsf(a); }

// Friction spring of mode s or r (Eqs. um .. um_kinetic): project onto the
// tangent plane keeping the length (zero if degenerate), evaluate
// f = -k u - c v, keep it if |f| <= mu |f_n| (static: u += dt v), otherwise
// clip it to mu |f_n| and set u = -(f + c v) / k (kinetic).  A contact that
// slid in the last step meets its bound again within rounding when nothing
// changed, so the test compares the lengths as the printed inequality does
// (the double-precision path then decides exactly as a plain double-precision
// program of the printed equations).
template <typename T>
__device__ __forceinline__ V3<T> spring_vec(V3<T>& u, V3<T> n, V3<T> vm, T k, T c, T mu, T fn,
                                            T dt) {
  const T ulen2 = dot(u, u);
  const V3<T> ut = u - dot(u, n) * n;
  const T utlen2 = dot(ut, ut);
  if (ulen2 > T(0) && utlen2 > T(0)) {
    u = vsqrt(ulen2 / utlen2) * ut;
  } else {
    u = mk(T(0), T(0), T(0));
  }
  V3<T> f = mk(-k * u.x - c * vm.x, -k * u.y - c * vm.y, -k * u.z - c * vm.z);
  const T flen = vnorm(f);
  const T lim = mu * fn;
  if (flen <= lim) {
    u = u + dt * vm;
  } else {
    f = (lim / flen) * f;
    const T ik = T(1) / k;
    u = mk(-(f.x + c * vm.x) * ik, -(f.y + c * vm.y) * ik, -(f.z + c * vm.z) * ik);
  }
  return f;
}

template <typename T>
__device__ __forceinline__ T spring_scalar(T& u, T vm, T k, T c, T mu, T fn, T dt) {
  T f = -k * u - c * vm;
  const T lim = mu * fn;
  if (vabs(f) <= lim) {
    u = u + dt * vm;
  } else {
    f = f > T(0) ? lim : -lim;
    u = -(f + c * vm) / k;
  }
  return f;
}

// One contact.  dv = v_i - v_j (pair) or v_i - v_wall at the contact point
// (wall); rw = r_i w_i + r_j w_j (pair) or r_i w_i (wall), the rotational part
// of the contact velocity; om = w_i - w_j (wall: w_i - Omega).  reff is the
// rolling radius (1/r_i + 1/r_j)^-1 (wall: r_i); rj is unused for walls.  The
// callers form the differences so each precision can do it without
// cancellation.
template <typename T>
__device__ __forceinline__ LawOut<T> contact_law(const LawConst<T>& c, V3<T> n, T delta, T Rs,
                                                 T ms, T ri, T rj, T reff, V3<T> dv, V3<T> rw,
                                                 V3<T> om, V3<T>& us, V3<T>& ur, T& ut) {
  // stiffness and damping (Eqs. ks, cn, cs; k_r = k_n, k_t = k_s, c_r = c_n, c_t = c_s)
  const T a = vsqrt(Rs * delta);
  const T kn = T(4) / T(3) * c.Es * a;
  const T ks = T(8) * c.Gs * a;
  const T cn = vsqrt(T(5) * ms * kn) * c.beta;
  // double precision keeps the printed form (and its rounding);
  // single precision scales c_n by the constant ratio (one root fewer)
  const T cs = sizeof(T) == 8 ? vsqrt(ms * ks / T(6)) * c.beta : cn * c.cs_cn;
  // relative velocity at the contact point
  const V3<T> v = dv + cross(n, rw);
  const V3<T> vn = dot(v, n) * n;
  const V3<T> vs = v - vn;
  const V3<T> vr = reff * cross(om, n);
  const T vt = Rs * dot(om, n);
  // normal force f_n = -k_n u_n - c_n v_n with u_n = -delta n
  const T kd = kn * delta;
  const V3<T> fn = mk(kd * n.x - cn * vn.x, kd * n.y - cn * vn.y, kd * n.z - cn * vn.z);
  const T fnm = vnorm(fn);
  const V3<T> fs = spring_vec(us, n, vs, ks, cs, c.mu_s, fnm, c.dt);
  const V3<T> fr = spring_vec(ur, n, vr, kn, cn, c.mu_r, fnm, c.dt);
  const T ft = spring_scalar(ut, vt, ks, cs, c.mu_t, fnm, c.dt);
  const V3<T> fsxn = cross(fs, n);
  const V3<T> tr = Rs * cross(n, fr);
  const V3<T> tt = (ft * Rs) * n;
  LawOut<T> o;
  o.f = fn + fs;
  o.ti = ri * fsxn + tr + tt;
  o.tj = rj * fsxn - tr - tt;
  return o;
}

}  // namespace dem
