// FP64 reference oracle for the soft-sphere DEM timestep (TEST INFRASTRUCTURE).
//
// This file is test infrastructure, not part of the product path.  Only the
// tests, the smoke check and the CPU-baseline leg of the benchmark load it.
// It shares no code, header, helper or constant with the CUDA library.
//
// It is a plain, slow, literal restatement of the method of arXiv 2507.12610
// ("TinyDEM"), Sec. 2 (particle model) and Sec. 3.2-3.3 (contact bookkeeping),
// in double precision with O(N^2) particle-pair search and O(N*M)
// particle-triangle search.  No cells, no lists, no blocking, no reordering.
//
// Readings of the paper taken here (each one is listed with its reason in the
// design notes of the repository):
//   * Contact-point velocity, Sec. 2.2: the rotational term is taken as
//     n x (r_i w_i + r_j w_j).  The printed minus sign contradicts the contact
//     point kinematics and the sliding-torque relation of Sec. 3.2; the literal
//     sign is available behind `literal_sign` so tests can show the difference.
//   * Degenerate projection of a friction spring (Sec. 2.3): if the spring or
//     its tangential part has zero length, the spring becomes zero.
//   * Coulomb test is inclusive (|f| <= mu |f_n| is static).  Kinetic twisting
//     sets f_t = mu_t |f_n| sign(f_t).
//   * Contact lifetime (Sec. 3.2): a contact exists in a step iff delta >= 0; its
//     history starts at zero and is dropped on the first step with delta < 0.
//   * Mesh elements (Sec. 2.2, 3.3): points, segments, triangles and
//     rectangles, each with a radius R_j >= 0 (rounded edges).  R_j = E_j =
//     m_j = infinity in the contact law, so R* = R_i, m* = m_i; the element
//     radius enters only delta.  Each touching element is an independent
//     contact (ghost collisions are kept, Sec. 3.3).
//   * Rotating mesh (not in the paper, which keeps walls static): the mesh turns
//     rigidly with angular velocity Omega about `mesh_center`; at step n its
//     vertices are the reference vertices rotated by angle |Omega| n dt.  The
//     wall velocity at the contact point x_c = x_i - r_i n is Omega x (x_c - c),
//     and the wall's angular velocity in the rolling/twisting terms is Omega.
//   * Summation order: contributions to a particle are added in ascending
//     partner index, then ascending triangle index (single-evaluation loop
//     over i < j, Sec. 3.2, followed by the mesh loop).
//   * Materials (not in the paper, which has one material): each particle may
//     carry a material index with its own friction coefficients mu_s, mu_r,
//     mu_t (the batched-scenes extension); a pair of particles uses the mean
//     of the two materials' coefficients, a mesh contact the particle's.
//     Without a material table every particle uses the coefficients of the
//     parameters.
//   * Particle spawning (Sec. 3.1, "Particle generation"): every `every` steps
//     (the paper: every step), before the forces of that step, `attempts`
//     attempts in sequence.  An attempt draws a radius uniformly in
//     [r_min, r_max] unless one is carried over from a failed attempt, then a
//     centre uniformly in the spawn box (x, y, z in that order); it is kept
//     unless the sphere overlaps a particle (|x - x_j| < r + R_j) or a mesh
//     element (distance < r + R_k), else its radius carries over.  Kept
//     particles take the next caller index, v0, w0 and the identity
//     orientation, until the capacity n_max is reached.  The uniforms are
//     those of SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) applied to
//     seed + (k + 1) * 0x9E3779B97F4A7C15 for the k-th draw of the run, mapped
//     to [0, 1) by their top 53 bits.
//
// Build: g++ -O2 -ffp-contract=off -fPIC -shared (no fused multiply-add
// contraction, so the oracle gives the same bits on x86-64 and aarch64).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <array>
#include <map>
#include <utility>
#include <vector>

namespace {

struct V3 {
  double x, y, z;
};
inline V3 v3(double x, double y, double z) { return V3{x, y, z}; }
inline V3 operator+(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
inline V3 operator-(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
inline V3 operator-(V3 a) { return v3(-a.x, -a.y, -a.z); }
inline V3 operator*(double s, V3 a) { return v3(s * a.x, s * a.y, s * a.z); }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
  return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }
inline V3 load3(const double* p, int64_t i) { return v3(p[3 * i], p[3 * i + 1], p[3 * i + 2]); }
inline void store3(double* p, int64_t i, V3 a) {
  p[3 * i] = a.x;
  p[3 * i + 1] = a.y;
  p[3 * i + 2] = a.z;
}

}  // namespace

extern "C" {

// Layout must match oracle/oracle.py (ctypes).
struct oracle_params {
  double E, nu, rho, e_n, mu_s, mu_r, mu_t, eta;
  double g[3];
  double dt;
  double mesh_omega[3];
  double mesh_center[3];
  int32_t literal_sign;  // 1: use the printed minus sign in the contact velocity
  int32_t reserved;
};

// Spawning parameters (Sec. 3.1).  Layout must match oracle/oracle.py.
struct oracle_spawn {
  int64_t n_max;             // capacity: particles are never spawned beyond it
  double lo[3], hi[3];       // spawn box corners
  double r_min, r_max;       // radius range
  double v0[3], w0[3];       // initial velocity and angular velocity
  int32_t attempts;          // attempts per spawn event
  int32_t every;             // steps between spawn events (>= 1)
  uint64_t seed;
};

}  // extern "C"

namespace {

// Static friction history of one contact (Table 3): u_s, u_r, u_t.
struct Hist {
  V3 us{0, 0, 0};
  V3 ur{0, 0, 0};
  double ut = 0;
};

// Contact key (Sec. 3.2): (i, j) with i < j for particle pairs; mesh element k
// is labelled by the non-positive index j = -1 - k.
using Key = std::pair<int64_t, int64_t>;

struct Scene {
  oracle_params p;
  int64_t n = 0;   // capacity (rows of the arrays)
  int64_t na = 0;  // active particles: rows 0 .. na-1 (the rest have R = 0)
  std::vector<double> R, x, v, w, q;  // R[n], x/v/w[3n], q[4n] (scalar first)
  std::vector<double> F, T;           // contact force / torque sums of the last step
  int64_t nv = 0, nt = 0;             // vertices, mesh elements
  std::vector<double> vert0;          // reference vertices [3 nv]
  std::vector<int32_t> tri;           // [4 nt] vertex indices, -1 pads (1..4 vertices)
  std::vector<double> tri_radius;     // [nt] element radius
  std::map<Key, Hist> hist;
  // Coulomb ratios (sliding, rolling, twisting) of the contacts of the last
  // step, same keys as hist; test diagnostics only
  std::map<Key, std::array<double, 3>> coulomb;
  int64_t step_count = 0;
  int64_t degenerate = 0;  // contacts skipped because d == 0
  oracle_spawn sp{};       // spawning off while sp.attempts == 0
  std::vector<double> mat_mu;   // [3 n_mat] mu_s, mu_r, mu_t per material (empty: params)
  std::vector<int32_t> mat;     // [n] material index per particle
  uint64_t draws = 0;      // uniforms drawn so far
  double carry = -1.0;     // radius carried over from a failed attempt (< 0: none)
};

// k-th uniform of the spawn stream: SplitMix64 output for counter k, top 53 bits.
double spawn_uniform(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// Damping factor beta(e_n) of Sec. 2.2.
double beta_of(double e_n) {
  if (e_n <= 0.0) return 1.0;  // ln e_n -> -inf
  if (e_n >= 1.0) return 0.0;  // ln e_n -> 0
  const double l = std::log(e_n);
  const double r = M_PI / l;
  return 1.0 / std::sqrt(1.0 + r * r);
}

// Closest point on triangle (a, b, c) to point p: the minimiser of |p - y| over
// the triangle, written out directly.  If the projection of p onto the plane
// lies inside the triangle (all barycentric coordinates >= 0) it is the answer;
// otherwise the minimiser lies on the boundary, i.e. on one of the three edges,
// each of which is handled as a clamped segment projection.
V3 closest_on_segment(V3 p, V3 a, V3 b) {
  V3 ab = b - a;
  double L2 = dot(ab, ab);
  if (L2 <= 0.0) return a;
  double t = dot(p - a, ab) / L2;
  if (t < 0.0) t = 0.0;
  if (t > 1.0) t = 1.0;
  return a + t * ab;
}

V3 closest_on_triangle(V3 p, V3 a, V3 b, V3 c) {
  V3 ab = b - a, ac = c - a;
  V3 nrm = cross(ab, ac);
  double n2 = dot(nrm, nrm);
  if (n2 > 0.0) {
    // projection onto the plane and its barycentric coordinates
    double s = dot(p - a, nrm) / n2;
    V3 y = p - s * nrm;
    // barycentric weights via sub-triangle areas (signed, along nrm)
    double wa = dot(cross(b - y, c - y), nrm) / n2;
    double wb = dot(cross(c - y, a - y), nrm) / n2;
    double wc = dot(cross(a - y, b - y), nrm) / n2;
    if (wa >= 0.0 && wb >= 0.0 && wc >= 0.0) return y;
  }
  V3 c1 = closest_on_segment(p, a, b);
  V3 c2 = closest_on_segment(p, b, c);
  V3 c3 = closest_on_segment(p, c, a);
  double d1 = dot(p - c1, p - c1), d2 = dot(p - c2, p - c2), d3 = dot(p - c3, p - c3);
  V3 best = c1;
  double bd = d1;
  if (d2 < bd) { best = c2; bd = d2; }
  if (d3 < bd) { best = c3; bd = d3; }
  return best;
}

// Closest point on rectangle a, b, c, d (vertices in order, right angles):
// the projection onto its plane if that lies inside, else the nearest point of
// the four edges.
V3 closest_on_rectangle(V3 p, V3 a, V3 b, V3 c, V3 d) {
  V3 u = b - a, w = d - a;
  V3 nrm = cross(u, w);
  double n2 = dot(nrm, nrm);
  if (n2 > 0.0) {
    V3 y = p - (dot(p - a, nrm) / n2) * nrm;
    double s = dot(y - a, u), t = dot(y - a, w);
    if (s >= 0.0 && s <= dot(u, u) && t >= 0.0 && t <= dot(w, w)) return y;
  }
  V3 e[4] = {closest_on_segment(p, a, b), closest_on_segment(p, b, c),
             closest_on_segment(p, c, d), closest_on_segment(p, d, a)};
  V3 best = e[0];
  double bd = dot(p - e[0], p - e[0]);
  for (int k = 1; k < 4; ++k) {
    double dk = dot(p - e[k], p - e[k]);
    if (dk < bd) { best = e[k]; bd = dk; }
  }
  return best;
}

// Closest point of mesh element k (1 to 4 vertices: point, segment, triangle,
// rectangle) to p, with the element's vertices given at the current pose.
V3 closest_on_element(V3 p, const std::vector<V3>& vt, const int32_t* el) {
  int nvk = 0;
  while (nvk < 4 && el[nvk] >= 0) ++nvk;
  switch (nvk) {
    case 1: return vt[el[0]];
    case 2: return closest_on_segment(p, vt[el[0]], vt[el[1]]);
    case 3: return closest_on_triangle(p, vt[el[0]], vt[el[1]], vt[el[2]]);
    default: return closest_on_rectangle(p, vt[el[0]], vt[el[1]], vt[el[2]], vt[el[3]]);
  }
}

// Rodrigues rotation of vector r by angle th about unit axis k.
V3 rotate(V3 r, V3 k, double th) {
  double c = std::cos(th), s = std::sin(th);
  return c * r + s * cross(k, r) + (dot(k, r) * (1.0 - c)) * k;
}

// Friction spring of mode m in {s, r} (Sec. 2.3): project the stored spring
// onto the current tangent plane and restore its length, evaluate
// f = -k u - c v, then apply the Coulomb limit mu |f_n| and update u.
// Coulomb ratio |f| / (mu |f_n|) of a trial force (a diagnostic for tests:
// near 1 the static/kinetic decision is within rounding of either branch).
double coulomb_ratio(double flen, double lim) {
  if (lim > 0.0) return flen / lim;
  return flen > 0.0 ? INFINITY : 0.0;
}

V3 friction_vec(V3& u, V3 n, V3 vm, double k, double c, double mu, double fn_mag, double dt,
                double* ratio = nullptr) {
  // projection back onto the tangent plane, length preserved (zero if degenerate)
  double ulen = norm(u);
  V3 ut = u - dot(u, n) * n;
  double utlen = norm(ut);
  if (ulen > 0.0 && utlen > 0.0)
    u = (ulen / utlen) * ut;
  else
    u = v3(0, 0, 0);
  V3 f = -k * u - c * vm;
  double flen = norm(f);
  if (ratio) *ratio = coulomb_ratio(flen, mu * fn_mag);
  if (flen <= mu * fn_mag) {
    u = u + dt * vm;  // static regime
  } else {
    f = (mu * fn_mag / flen) * f;   // kinetic regime: clip to the Coulomb bound
    u = (-1.0 / k) * (f + c * vm);  // spring set to satisfy Coulomb exactly
  }
  return f;
}

double friction_scalar(double& u, double vm, double k, double c, double mu, double fn_mag, double dt,
                       double* ratio = nullptr) {
  double f = -k * u - c * vm;
  if (ratio) *ratio = coulomb_ratio(std::fabs(f), mu * fn_mag);
  if (std::fabs(f) <= mu * fn_mag) {
    u = u + dt * vm;
  } else {
    f = (f > 0.0 ? 1.0 : -1.0) * mu * fn_mag;
    u = (-1.0 / k) * (f + c * vm);
  }
  return f;
}

struct Coeffs {
  double Es, Gs, Rs, ms;  // effective modulus, shear modulus, radius, mass
  double kn, ks, cn, cs;  // stiffness and damping coefficients
};

// Effective properties and contact coefficients (Sec. 2.2).  All particles
// share E, nu, rho; a wall has E_j = G_j = R_j = m_j = infinity, so the terms
// with 1/inf vanish.
Coeffs contact_coeffs(const oracle_params& p, bool wall, double Ri, double mi, double Rj,
                      double mj, double delta) {
  const double E = p.E, nu = p.nu;
  const double G = E / (2.0 * (1.0 + nu));
  Coeffs k;
  if (wall) {
    k.Es = 1.0 / ((1.0 - nu * nu) / E);
    k.Gs = 1.0 / ((2.0 - nu) / G);
    k.Rs = Ri;
    k.ms = mi;
  } else {
    k.Es = 1.0 / ((1.0 - nu * nu) / E + (1.0 - nu * nu) / E);
    k.Gs = 1.0 / ((2.0 - nu) / G + (2.0 - nu) / G);
    k.Rs = 1.0 / (1.0 / Ri + 1.0 / Rj);
    k.ms = 1.0 / (1.0 / mi + 1.0 / mj);
  }
  const double a = std::sqrt(k.Rs * delta);  // contact radius
  k.kn = 4.0 / 3.0 * k.Es * a;
  k.ks = 8.0 * k.Gs * a;
  const double beta = beta_of(p.e_n);
  k.cn = std::sqrt(5.0 * k.ms * k.kn) * beta;
  k.cs = std::sqrt(k.ms * k.ks / 6.0) * beta;
  return k;
}

struct ContactOut {
  V3 f;      // force on i (f_n + f_s)
  V3 tau_i;  // torque on i (tau_s + tau_r + tau_t)
  V3 tau_j;  // torque on j (r_j f_s x n - tau_r - tau_t); unused for walls
};

// The inelastic Hertz-Mindlin contact law with sliding, rolling and twisting
// friction (Sec. 2.2) and the history update of Sec. 2.3, for body i against
// body j.  For a wall, j is infinitely large, stiff and heavy; its surface
// velocity at the contact point and its angular velocity are given directly.
struct Friction {
  double mu_s, mu_r, mu_t;
};

ContactOut contact_law(const oracle_params& p, const Friction& mu, V3 nhat, double delta,
                       double Ri, double mi, V3 vi, V3 wi,
                       bool wall, double Rj, double mj, V3 vj, V3 wj, V3 vwall,
                       Hist& h, bool literal_sign, double* coul = nullptr) {
  const Coeffs k = contact_coeffs(p, wall, Ri, mi, Rj, mj, delta);
  const double Rs = k.Rs;
  const double kn = k.kn, ks = k.ks, cn = k.cn, cs = k.cs;
  const double kr = kn, cr = cn, kt = ks, ct = cs;
  // distances from the centres to the contact point
  const double ri = Ri - delta / 2.0;
  const double rj = wall ? INFINITY : Rj - delta / 2.0;
  // relative velocity at the contact point and its decomposition
  V3 v;
  if (wall) {
    v = vi - vwall + cross(nhat, ri * wi);
  } else {
    V3 rot = literal_sign ? (ri * wi - rj * wj) : (ri * wi + rj * wj);
    v = vi - vj + cross(nhat, rot);
  }
  const V3 vn = dot(v, nhat) * nhat;
  const V3 vs = v - vn;
  const V3 om = wi - wj;
  const double inv_r = wall ? 1.0 / ri : 1.0 / ri + 1.0 / rj;
  const V3 vr = (1.0 / inv_r) * cross(om, nhat);
  const double vt = Rs * dot(om, nhat);
  // normal force
  const V3 un = -delta * nhat;
  const V3 fn = -kn * un - cn * vn;
  const double fn_mag = norm(fn);
  // friction modes, each independently static or kinetic
  const V3 fs = friction_vec(h.us, nhat, vs, ks, cs, mu.mu_s, fn_mag, p.dt, coul);
  const V3 fr = friction_vec(h.ur, nhat, vr, kr, cr, mu.mu_r, fn_mag, p.dt, coul ? coul + 1 : nullptr);
  const double ft = friction_scalar(h.ut, vt, kt, ct, mu.mu_t, fn_mag, p.dt, coul ? coul + 2 : nullptr);
  // torques
  const V3 tau_s = ri * cross(fs, nhat);
  const V3 tau_r = Rs * cross(nhat, fr);
  const V3 tau_t = (ft * Rs) * nhat;
  ContactOut o;
  o.f = fn + fs;
  o.tau_i = tau_s + tau_r + tau_t;
  if (!wall) o.tau_j = rj * cross(fs, nhat) - tau_r - tau_t;  // Eqs. antisymm_*
  else o.tau_j = v3(0, 0, 0);
  return o;
}

double mass_of(const oracle_params& p, double R) { return 4.0 / 3.0 * M_PI * p.rho * R * R * R; }

// Friction coefficients of particle i's material (the parameters' without a table).
Friction friction_of(const Scene& S, int64_t i) {
  if (S.mat_mu.empty()) return Friction{S.p.mu_s, S.p.mu_r, S.p.mu_t};
  const double* m = &S.mat_mu[3 * (size_t)S.mat[i]];
  return Friction{m[0], m[1], m[2]};
}

// A pair of particles: the mean of the two materials' coefficients.
Friction friction_of_pair(const Scene& S, int64_t i, int64_t j) {
  const Friction a = friction_of(S, i), b = friction_of(S, j);
  return Friction{(a.mu_s + b.mu_s) / 2.0, (a.mu_r + b.mu_r) / 2.0, (a.mu_t + b.mu_t) / 2.0};
}

// Hamilton product (Sec. 2.3).
void qmul(const double* a, const double* b, double* out) {
  double s = a[0] * b[0] - (a[1] * b[1] + a[2] * b[2] + a[3] * b[3]);
  V3 av = v3(a[1], a[2], a[3]), bv = v3(b[1], b[2], b[3]);
  V3 r = a[0] * bv + b[0] * av + cross(av, bv);
  out[0] = s;
  out[1] = r.x;
  out[2] = r.y;
  out[3] = r.z;
}

// Semi-implicit Euler step of one particle (Sec. 2.3): accelerations from the
// contact sums, gravity and Stokes drag; v then x (with the new v); the SPIRAL
// orientation update with the angular velocity before its update; then w.
void integrate_particle(const oracle_params& p, double R, V3 F, V3 T, V3& x, V3& v, V3& w,
                        double* q) {
  const double m = mass_of(p, R);
  const double I = 2.0 / 5.0 * m * R * R;
  const double ci = 9.0 * p.eta / (2.0 * p.rho * R * R);  // Stokes drag rates
  const double gi = 10.0 / 3.0 * ci;
  const V3 g = load3(p.g, 0);
  const V3 a = (1.0 / m) * F + g - ci * v;
  const V3 al = (1.0 / I) * T - gi * w;
  v = v + p.dt * a;
  x = x + p.dt * v;
  // q <- q (cos phi, sin phi w/|w|) (cos theta, sin theta al/|al|), each
  // product only if the rotation vector is non-zero
  const double wn = norm(w);
  if (wn > 0.0) {
    const double phi = p.dt / 2.0 * wn;
    const double r[4] = {std::cos(phi), std::sin(phi) * w.x / wn, std::sin(phi) * w.y / wn,
                         std::sin(phi) * w.z / wn};
    double t[4];
    qmul(q, r, t);
    std::memcpy(q, t, sizeof t);
  }
  const double an = norm(al);
  if (an > 0.0) {
    const double th = (p.dt / 2.0) * (p.dt / 2.0) * an;
    const double r[4] = {std::cos(th), std::sin(th) * al.x / an, std::sin(th) * al.y / an,
                         std::sin(th) * al.z / an};
    double t[4];
    qmul(q, r, t);
    std::memcpy(q, t, sizeof t);
  }
  w = w + p.dt * al;
}

V3 mesh_vertex(const Scene& S, int64_t k) {
  V3 r0 = load3(S.vert0.data(), k);
  V3 Om = load3(S.p.mesh_omega, 0);
  double wm = norm(Om);
  if (!(wm > 0.0)) return r0;
  V3 c = load3(S.p.mesh_center, 0);
  double th = wm * ((double)S.step_count * S.p.dt);
  return c + rotate(r0 - c, (1.0 / wm) * Om, th);
}

// Spawn attempts of one event (Sec. 3.1), in sequence, against the particles
// and mesh at the current step.
void spawn_event(Scene& S) {
  const oracle_spawn& sp = S.sp;
  std::vector<V3> vt(S.nv);
  for (int64_t k = 0; k < S.nv; ++k) vt[k] = mesh_vertex(S, k);
  for (int32_t a = 0; a < sp.attempts && S.na < S.n; ++a) {
    double r = S.carry;
    if (r < 0.0) r = sp.r_min + spawn_uniform(sp.seed, S.draws++) * (sp.r_max - sp.r_min);
    V3 c;
    c.x = sp.lo[0] + spawn_uniform(sp.seed, S.draws++) * (sp.hi[0] - sp.lo[0]);
    c.y = sp.lo[1] + spawn_uniform(sp.seed, S.draws++) * (sp.hi[1] - sp.lo[1]);
    c.z = sp.lo[2] + spawn_uniform(sp.seed, S.draws++) * (sp.hi[2] - sp.lo[2]);
    bool overlap = false;
    for (int64_t j = 0; j < S.na && !overlap; ++j) {
      const V3 d = c - load3(S.x.data(), j);
      const double s = r + S.R[j];
      overlap = dot(d, d) < s * s;
    }
    for (int64_t k = 0; k < S.nt && !overlap; ++k) {
      const V3 d = c - closest_on_element(c, vt, &S.tri[4 * k]);
      const double s = r + S.tri_radius[k];
      overlap = dot(d, d) < s * s;
    }
    if (overlap) {
      S.carry = r;
      continue;
    }
    const int64_t i = S.na++;
    S.R[i] = r;
    store3(S.x.data(), i, c);
    store3(S.v.data(), i, load3(sp.v0, 0));
    store3(S.w.data(), i, load3(sp.w0, 0));
    S.q[4 * i] = 1.0;
    S.q[4 * i + 1] = S.q[4 * i + 2] = S.q[4 * i + 3] = 0.0;
    S.carry = -1.0;
  }
}

// One timestep: contact search and forces at t_n, then integration to t_{n+1}.
void spawn_event(Scene& S);

void step_once(Scene& S) {
  const oracle_params& p = S.p;
  if (S.sp.attempts > 0 && S.step_count % S.sp.every == 0) spawn_event(S);
  const int64_t n = S.na;  // inactive rows take part in nothing
  std::fill(S.F.begin(), S.F.end(), 0.0);
  std::fill(S.T.begin(), S.T.end(), 0.0);
  std::map<Key, Hist> next;
  std::map<Key, std::array<double, 3>> next_coul;

  // particle-particle contacts, each unordered pair evaluated once (i < j)
  for (int64_t i = 0; i < n; ++i) {
    const V3 xi = load3(S.x.data(), i), vi = load3(S.v.data(), i), wi = load3(S.w.data(), i);
    const double Ri = S.R[i], mi = mass_of(p, Ri);
    for (int64_t j = i + 1; j < n; ++j) {
      const V3 xj = load3(S.x.data(), j);
      const V3 d = xi - xj;
      const double dist = norm(d);
      const double delta = Ri + S.R[j] - dist;
      if (delta < 0.0) continue;  // not touching: any history is dropped
      if (!(dist > 0.0)) { ++S.degenerate; continue; }
      const V3 nhat = (1.0 / dist) * d;
      Hist h;
      auto it = S.hist.find(Key(i, j));
      if (it != S.hist.end()) h = it->second;
      const double Rj = S.R[j];
      std::array<double, 3> cr{};
      ContactOut o = contact_law(p, friction_of_pair(S, i, j), nhat, delta, Ri, mi, vi, wi,
                                 false, Rj, mass_of(p, Rj),
                                 load3(S.v.data(), j), load3(S.w.data(), j), v3(0, 0, 0), h,
                                 p.literal_sign != 0, cr.data());
      next_coul[Key(i, j)] = cr;
      store3(S.F.data(), i, load3(S.F.data(), i) + o.f);
      store3(S.F.data(), j, load3(S.F.data(), j) - o.f);
      store3(S.T.data(), i, load3(S.T.data(), i) + o.tau_i);
      store3(S.T.data(), j, load3(S.T.data(), j) + o.tau_j);
      next[Key(i, j)] = h;
    }
  }

  // particle-triangle contacts
  if (S.nt > 0) {
    std::vector<V3> vt(S.nv);
    for (int64_t k = 0; k < S.nv; ++k) vt[k] = mesh_vertex(S, k);
    const V3 Om = load3(p.mesh_omega, 0), c = load3(p.mesh_center, 0);
    for (int64_t i = 0; i < n; ++i) {
      const V3 xi = load3(S.x.data(), i), vi = load3(S.v.data(), i), wi = load3(S.w.data(), i);
      const double Ri = S.R[i], mi = mass_of(p, Ri);
      for (int64_t k = 0; k < S.nt; ++k) {
        const V3 pc = closest_on_element(xi, vt, &S.tri[4 * k]);
        const V3 d = xi - pc;
        const double dist = norm(d);
        const double delta = Ri + S.tri_radius[k] - dist;
        if (delta < 0.0) continue;
        if (!(dist > 0.0)) { ++S.degenerate; continue; }
        const V3 nhat = (1.0 / dist) * d;
        Hist h;
        const Key key(i, -1 - k);
        auto it = S.hist.find(key);
        if (it != S.hist.end()) h = it->second;
        const double ri = Ri - delta / 2.0;
        const V3 xc = xi - ri * nhat;  // contact point
        const V3 vwall = cross(Om, xc - c);
        std::array<double, 3> cr{};
        ContactOut o = contact_law(p, friction_of(S, i), nhat, delta, Ri, mi, vi, wi, true,
                                   INFINITY, INFINITY,
                                   v3(0, 0, 0), Om, vwall, h, false, cr.data());
        store3(S.F.data(), i, load3(S.F.data(), i) + o.f);
        store3(S.T.data(), i, load3(S.T.data(), i) + o.tau_i);
        next[key] = h;
        next_coul[key] = cr;
      }
    }
  }
  S.hist.swap(next);
  S.coulomb.swap(next_coul);

  // semi-implicit Euler with the SPIRAL quaternion update (Sec. 2.3)
  for (int64_t i = 0; i < n; ++i) {
    V3 x = load3(S.x.data(), i), v = load3(S.v.data(), i), w = load3(S.w.data(), i);
    integrate_particle(p, S.R[i], load3(S.F.data(), i), load3(S.T.data(), i), x, v, w, &S.q[4 * i]);
    store3(S.v.data(), i, v);
    store3(S.x.data(), i, x);
    store3(S.w.data(), i, w);
  }
  S.step_count += 1;
}

}  // namespace

extern "C" {

void* oracle_create(const oracle_params* p, int64_t n, const double* R, const double* x,
                    const double* v, const double* w, const double* q, int64_t nv,
                    const double* vert, int64_t nt, const int32_t* tri, const double* tri_radius) {
  Scene* S = new Scene();
  S->p = *p;
  S->n = n;
  S->na = n;
  S->R.assign(R, R + n);
  S->x.assign(x, x + 3 * n);
  S->v.assign(v, v + 3 * n);
  S->w.assign(w, w + 3 * n);
  S->q.assign(q, q + 4 * n);
  S->F.assign(3 * n, 0.0);
  S->T.assign(3 * n, 0.0);
  S->nv = nv;
  S->nt = nt;
  if (nv > 0) S->vert0.assign(vert, vert + 3 * nv);
  if (nt > 0) {
    S->tri.assign(tri, tri + 4 * nt);
    S->tri_radius.assign(tri_radius, tri_radius + nt);
  }
  return S;
}

void oracle_destroy(void* s) { delete static_cast<Scene*>(s); }

// Turn on spawning (Sec. 3.1): rows grow to the capacity sp->n_max; the new
// rows are inactive (R = 0) until spawned.
void oracle_set_spawn(void* s, const oracle_spawn* sp) {
  Scene* S = static_cast<Scene*>(s);
  S->sp = *sp;
  if (S->sp.every < 1) S->sp.every = 1;
  const int64_t cap = sp->n_max > S->n ? sp->n_max : S->n;
  S->R.resize(cap, 0.0);
  S->x.resize(3 * cap, 0.0);
  S->v.resize(3 * cap, 0.0);
  S->w.resize(3 * cap, 0.0);
  S->q.resize(4 * cap, 0.0);
  for (int64_t i = S->n; i < cap; ++i) S->q[4 * i] = 1.0;
  if (!S->mat.empty()) S->mat.resize(cap, 0);  // spawned particles: material 0
  S->F.resize(3 * cap, 0.0);
  S->T.resize(3 * cap, 0.0);
  S->n = cap;
}

int64_t oracle_active(void* s) { return static_cast<Scene*>(s)->na; }

// Friction per material (not in the paper): mu[3k..3k+2] = mu_s, mu_r, mu_t of
// material k; mat[i] = material of particle i (rows beyond n take material 0).
void oracle_set_materials(void* s, int32_t n_mat, const double* mu, const int32_t* mat) {
  Scene* S = static_cast<Scene*>(s);
  S->mat_mu.assign(mu, mu + 3 * (size_t)n_mat);
  S->mat.assign(S->n, 0);
  for (int64_t i = 0; i < S->n; ++i) S->mat[i] = mat ? mat[i] : 0;
}
int64_t oracle_capacity(void* s) { return static_cast<Scene*>(s)->n; }
uint64_t oracle_spawn_draws(void* s) { return static_cast<Scene*>(s)->draws; }

void oracle_read_radii(void* s, double* R) {
  Scene* S = static_cast<Scene*>(s);
  std::memcpy(R, S->R.data(), sizeof(double) * S->n);
}

double oracle_spawn_uniform(uint64_t seed, uint64_t k) { return spawn_uniform(seed, k); }

void oracle_step(void* s, int64_t nsteps) {
  Scene* S = static_cast<Scene*>(s);
  for (int64_t k = 0; k < nsteps; ++k) step_once(*S);
}

void oracle_read_state(void* s, double* x, double* v, double* w, double* q) {
  Scene* S = static_cast<Scene*>(s);
  std::memcpy(x, S->x.data(), sizeof(double) * 3 * S->n);
  std::memcpy(v, S->v.data(), sizeof(double) * 3 * S->n);
  std::memcpy(w, S->w.data(), sizeof(double) * 3 * S->n);
  std::memcpy(q, S->q.data(), sizeof(double) * 4 * S->n);
}

void oracle_read_forces(void* s, double* F, double* T) {
  Scene* S = static_cast<Scene*>(s);
  std::memcpy(F, S->F.data(), sizeof(double) * 3 * S->n);
  std::memcpy(T, S->T.data(), sizeof(double) * 3 * S->n);
}

int64_t oracle_num_contacts(void* s) { return (int64_t) static_cast<Scene*>(s)->hist.size(); }
int64_t oracle_degenerate(void* s) { return static_cast<Scene*>(s)->degenerate; }
int64_t oracle_step_count(void* s) { return static_cast<Scene*>(s)->step_count; }

// Contacts in key order: keys[2k] = i, keys[2k+1] = j (j < 0: triangle -1-j);
// hist[7k..7k+6] = u_s, u_r, u_t.
void oracle_read_contacts(void* s, int64_t* keys, double* hist) {
  Scene* S = static_cast<Scene*>(s);
  int64_t k = 0;
  for (const auto& kv : S->hist) {
    keys[2 * k] = kv.first.first;
    keys[2 * k + 1] = kv.first.second;
    const Hist& h = kv.second;
    double* o = hist + 7 * k;
    o[0] = h.us.x; o[1] = h.us.y; o[2] = h.us.z;
    o[3] = h.ur.x; o[4] = h.ur.y; o[5] = h.ur.z;
    o[6] = h.ut;
    ++k;
  }
}

// Replace the contact history (keys / hist in the layout of oracle_read_contacts).
void oracle_set_contacts(void* s, int64_t m, const int64_t* keys, const double* hist) {
  Scene* S = static_cast<Scene*>(s);
  S->hist.clear();
  for (int64_t k = 0; k < m; ++k) {
    Hist h;
    const double* o = hist + 7 * k;
    h.us = v3(o[0], o[1], o[2]);
    h.ur = v3(o[3], o[4], o[5]);
    h.ut = o[6];
    S->hist[Key(keys[2 * k], keys[2 * k + 1])] = h;
  }
}

void oracle_set_step_count(void* s, int64_t c) { static_cast<Scene*>(s)->step_count = c; }

// Replace the particle state (caller order, n rows of the scene): the tests
// start a step of the oracle from a state taken elsewhere.
void oracle_set_state(void* s, const double* x, const double* v, const double* w,
                      const double* q) {
  Scene* S = static_cast<Scene*>(s);
  std::memcpy(S->x.data(), x, sizeof(double) * 3 * S->n);
  std::memcpy(S->v.data(), v, sizeof(double) * 3 * S->n);
  std::memcpy(S->w.data(), w, sizeof(double) * 3 * S->n);
  std::memcpy(S->q.data(), q, sizeof(double) * 4 * S->n);
}

// Coulomb ratios |f_m| / (mu_m |f_n|) of the trial forces of the last step,
// m = sliding, rolling, twisting, out[3k..3k+2] for the k-th contact in the
// order of oracle_read_contacts (a contact near 1 sits at its Coulomb bound).
void oracle_read_coulomb(void* s, double* out) {
  Scene* S = static_cast<Scene*>(s);
  int64_t k = 0;
  for (const auto& kv : S->coulomb) {
    std::memcpy(out + 3 * k, kv.second.data(), 3 * sizeof(double));
    ++k;
  }
}

// Closest point on a triangle, exposed for tests.
void oracle_closest_on_triangle(const double* p, const double* a, const double* b,
                                const double* c, double* out) {
  V3 r = closest_on_triangle(load3(p, 0), load3(a, 0), load3(b, 0), load3(c, 0));
  store3(out, 0, r);
}

double oracle_beta(double e_n) { return beta_of(e_n); }

// Closest point on a mesh element given by its vertices (nverts = 1..4), for tests.
void oracle_closest_on_element(const double* p, const double* verts, int32_t nverts, double* out) {
  std::vector<V3> vt;
  int32_t el[4] = {-1, -1, -1, -1};
  for (int32_t k = 0; k < nverts && k < 4; ++k) {
    vt.push_back(load3(verts, k));
    el[k] = k;
  }
  store3(out, 0, closest_on_element(load3(p, 0), vt, el));
}

// Contact coefficients for tests: out = {E*, G*, R*, m*, k_n, k_s, c_n, c_s}.
// For a wall (wall != 0) Rj is ignored.
void oracle_contact_coeffs(const oracle_params* p, int32_t wall, double Ri, double Rj,
                           double delta, double* out) {
  const double mi = mass_of(*p, Ri);
  const double mj = wall ? INFINITY : mass_of(*p, Rj);
  Coeffs k = contact_coeffs(*p, wall != 0, Ri, mi, wall ? INFINITY : Rj, mj, delta);
  const double v[8] = {k.Es, k.Gs, k.Rs, k.ms, k.kn, k.ks, k.cn, k.cs};
  std::memcpy(out, v, sizeof v);
}

// One step for a sample of particles, evaluated one by one from a state with
// no contact history (the first step of a run): for each sampled particle the
// contact sums over all other particles (ascending index) and all triangles
// (ascending index), then the integrated state.  Used to check large runs on
// a subset of outputs.  Output rows follow `ids`.
void oracle_sample_first_step(const oracle_params* p, int64_t n, const double* R, const double* x,
                              const double* v, const double* w, const double* q, int64_t nv,
                              const double* vert, int64_t nt, const int32_t* tri,
                              const double* tri_radius, int64_t step_index, int64_t ns,
                              const int64_t* ids, double* F_out, double* T_out, double* x_out,
                              double* v_out, double* w_out, double* q_out) {
  // Build a scene holding only what is needed: all particles (to find
  // partners) but integrate only the sampled ones.
  Scene S;
  S.p = *p;
  S.n = n;
  S.nv = nv;
  S.nt = nt;
  S.step_count = step_index;
  if (nv > 0) S.vert0.assign(vert, vert + 3 * nv);
  if (nt > 0) {
    S.tri.assign(tri, tri + 4 * nt);
    S.tri_radius.assign(tri_radius, tri_radius + nt);
  }
  std::vector<V3> vt(nv);
  for (int64_t k = 0; k < nv; ++k) vt[k] = mesh_vertex(S, k);
  const V3 Om = load3(p->mesh_omega, 0), c = load3(p->mesh_center, 0);
  for (int64_t s = 0; s < ns; ++s) {
    const int64_t i = ids[s];
    const V3 xi = load3(x, i), vi = load3(v, i), wi = load3(w, i);
    const double Ri = R[i], mi = mass_of(*p, Ri);
    V3 F = v3(0, 0, 0), T = v3(0, 0, 0);
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      // evaluate the pair in canonical order (lower index first), as the
      // single-evaluation loop does, and take i's side
      const int64_t lo = i < j ? i : j, hi = i < j ? j : i;
      const V3 d = load3(x, lo) - load3(x, hi);
      const double dist = norm(d);
      const double delta = R[lo] + R[hi] - dist;
      if (delta < 0.0 || !(dist > 0.0)) continue;
      const V3 nhat = (1.0 / dist) * d;
      Hist h;
      ContactOut o = contact_law(*p, Friction{p->mu_s, p->mu_r, p->mu_t}, nhat, delta, R[lo],
                                 mass_of(*p, R[lo]), load3(v, lo),
                                 load3(w, lo), false, R[hi], mass_of(*p, R[hi]), load3(v, hi),
                                 load3(w, hi), v3(0, 0, 0), h, p->literal_sign != 0);
      if (i == lo) {
        F = F + o.f;
        T = T + o.tau_i;
      } else {
        F = F - o.f;
        T = T + o.tau_j;
      }
    }
    for (int64_t k = 0; k < nt; ++k) {
      const V3 pc = closest_on_element(xi, vt, &S.tri[4 * k]);
      const V3 d = xi - pc;
      const double dist = norm(d);
      const double delta = Ri + tri_radius[k] - dist;
      if (delta < 0.0 || !(dist > 0.0)) continue;
      const V3 nhat = (1.0 / dist) * d;
      Hist h;
      const double ri = Ri - delta / 2.0;
      const V3 xc = xi - ri * nhat;
      ContactOut o = contact_law(*p, Friction{p->mu_s, p->mu_r, p->mu_t}, nhat, delta, Ri, mi,
                                 vi, wi, true, INFINITY, INFINITY,
                                 v3(0, 0, 0), Om, cross(Om, xc - c), h, false);
      F = F + o.f;
      T = T + o.tau_i;
    }
    store3(F_out, s, F);
    store3(T_out, s, T);
    // integrate this particle alone (same update as a full step)
    V3 xx = xi, vv = vi, ww = wi;
    double qq[4] = {q[4 * i], q[4 * i + 1], q[4 * i + 2], q[4 * i + 3]};
    integrate_particle(*p, Ri, F, T, xx, vv, ww, qq);
    store3(x_out, s, xx);
    store3(v_out, s, vv);
    store3(w_out, s, ww);
    std::memcpy(q_out + 4 * s, qq, sizeof qq);
  }
}

}  // extern "C"
