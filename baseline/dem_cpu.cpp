// CPU baseline of the DEM timestep in the design of the paper's own program
// (arXiv 2507.12610, Sec. 3 and Sec. 5): double precision, linked cell lists
// over the bounding box of the ensemble rebuilt every step with cells of edge
// 2 R_max, the list built serially and every other loop over particles and
// mesh elements parallelised with OpenMP, each particle pair evaluated once
// (i < j) with the antisymmetry relations of Sec. 3.2, contact history in a
// per-particle list with an "active" flag (Table 3).  It exists to be timed
// beside the GPU library on the same workloads; it shares no code with that
// library or with the test oracle.  Force sums are accumulated with atomic
// additions, so their rounding order depends on thread timing (as the paper
// notes for its parallel runs).
//
// Same physics as the paper: Hertz-Mindlin normal force with the damping of
// Sec. 2.2, sliding/rolling/twisting springs with the Coulomb limits and the
// updates of Sec. 2.3, semi-implicit Euler with the SPIRAL quaternion update,
// Stokes drag.  Readings shared with the rest of the repository: the
// rotational term of the contact velocity is n x (r_i w_i + r_j w_j); a
// contact exists while delta >= 0; mesh elements (points, segments,
// triangles, rectangles with a radius) are walls of infinite radius, modulus
// and mass; a rotating mesh (an extension) has its vertices rotated by
// |Omega| t about an axis and moves with velocity Omega x (p - c).
//
// Build: g++ -O3 -fopenmp -fPIC -shared -std=c++17 dem_cpu.cpp
#include <omp.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

struct Vec {
  double x, y, z;
};
inline Vec vec(double x, double y, double z) { return Vec{x, y, z}; }
inline Vec operator+(Vec a, Vec b) { return vec(a.x + b.x, a.y + b.y, a.z + b.z); }
inline Vec operator-(Vec a, Vec b) { return vec(a.x - b.x, a.y - b.y, a.z - b.z); }
inline Vec operator*(double s, Vec a) { return vec(s * a.x, s * a.y, s * a.z); }
inline double dotp(Vec a, Vec b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline Vec crossp(Vec a, Vec b) {
  return vec(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
inline double len(Vec a) { return std::sqrt(dotp(a, a)); }

}  // namespace

extern "C" {
// Layout must match baseline/dem_cpu.py.
struct dcpu_params {
  double E, nu, rho, e_n, mu_s, mu_r, mu_t, eta;
  double g[3];
  double dt;
  double mesh_omega[3], mesh_center[3];
};
}

namespace {

// One entry of a particle's contact list (Table 3): partner j > i for a
// particle, j = -k <= 0 for mesh element k; springs; active flag psi.
struct Contact {
  int64_t j;
  Vec us, ur;
  double ut;
  bool psi;
};

struct Sim {
  dcpu_params p{};
  int64_t n = 0;
  std::vector<double> R, m;
  std::vector<Vec> x, v, w, F, T;
  std::vector<double> q;  // [4 n], scalar first
  std::vector<std::vector<Contact>> c;
  // mesh
  std::vector<Vec> vref, vcur;
  std::vector<int32_t> el;  // [4 ne], -1 pads
  std::vector<double> erad;
  int64_t ne = 0;
  int64_t steps = 0;
  double rmax = 0;
  // grid (rebuilt every step)
  double lo[3];
  int64_t nc[3];
  double inv_h;
  std::vector<int64_t> head, next;
  std::vector<std::vector<int64_t>> cell_elems;
  // material constants
  double Es_pp, Gs_pp, Es_pw, Gs_pw, beta;
};

double damping_beta(double e) {
  if (e <= 0.0) return 1.0;
  if (e >= 1.0) return 0.0;
  const double l = std::log(e);
  return -l / std::sqrt(l * l + M_PI * M_PI);
}

// Atomic addition of a vector (the partner of a pair may belong to another thread).
inline void add_atomic(Vec& a, Vec b) {
#pragma omp atomic
  a.x += b.x;
#pragma omp atomic
  a.y += b.y;
#pragma omp atomic
  a.z += b.z;
}

// Closest points on the four element kinds (Sec. 3.3): a point is itself;
// a segment clamps the projection parameter; a triangle takes the projection
// onto its plane when that lies on the inner side of all three edges, else the
// nearest clamped projection onto an edge it lies outside of; a rectangle with
// right angles clamps the two edge coordinates.
Vec on_segment(Vec p, Vec a, Vec b) {
  const Vec ab = b - a;
  const double l2 = dotp(ab, ab);
  if (!(l2 > 0.0)) return a;
  const double t = std::min(1.0, std::max(0.0, dotp(p - a, ab) / l2));
  return a + t * ab;
}

Vec on_triangle(Vec p, Vec a, Vec b, Vec c) {
  const Vec nrm = crossp(b - a, c - a);
  const double n2 = dotp(nrm, nrm);
  if (!(n2 > 0.0)) {  // degenerate: the nearest point of the three edges
    const Vec e[3] = {on_segment(p, a, b), on_segment(p, b, c), on_segment(p, c, a)};
    Vec best = e[0];
    for (int k = 1; k < 3; ++k)
      if (dotp(p - e[k], p - e[k]) < dotp(p - best, p - best)) best = e[k];
    return best;
  }
  const Vec y = p - (dotp(p - a, nrm) / n2) * nrm;  // projection onto the plane
  const Vec vtx[3] = {a, b, c};
  bool inside = true;
  Vec best = y;
  double bd = INFINITY;
  for (int k = 0; k < 3; ++k) {
    const Vec s0 = vtx[k], s1 = vtx[(k + 1) % 3];
    if (dotp(crossp(s1 - s0, y - s0), nrm) < 0.0) {  // outside edge k
      inside = false;
      const Vec e = on_segment(p, s0, s1);
      const double de = dotp(p - e, p - e);
      if (de < bd) {
        bd = de;
        best = e;
      }
    }
  }
  return inside ? y : best;
}

Vec on_rectangle(Vec p, Vec a, Vec b, Vec d) {
  const Vec u = b - a, w = d - a;
  const double s = std::min(1.0, std::max(0.0, dotp(p - a, u) / dotp(u, u)));
  const double t = std::min(1.0, std::max(0.0, dotp(p - a, w) / dotp(w, w)));
  return a + s * u + t * w;
}

Vec on_element(const Sim& S, int64_t k, Vec p) {
  const int32_t* e = &S.el[4 * k];
  if (e[1] < 0) return S.vcur[e[0]];
  if (e[2] < 0) return on_segment(p, S.vcur[e[0]], S.vcur[e[1]]);
  if (e[3] < 0) return on_triangle(p, S.vcur[e[0]], S.vcur[e[1]], S.vcur[e[2]]);
  return on_rectangle(p, S.vcur[e[0]], S.vcur[e[1]], S.vcur[e[3]]);
}

// Tangential spring of mode s or r (Sec. 2.3): rotate into the tangent plane
// keeping the length, trial force, Coulomb test, static or kinetic update.
Vec spring(Vec& u, Vec nh, Vec vm, double k, double cdamp, double lim, double dt) {
  const double ul = len(u);
  const Vec ut = u - dotp(u, nh) * nh;
  const double utl = len(ut);
  u = (ul > 0.0 && utl > 0.0) ? (ul / utl) * ut : vec(0, 0, 0);
  Vec f = (-k) * u - cdamp * vm;
  const double fl = len(f);
  if (fl <= lim) {
    u = u + dt * vm;
  } else {
    f = (lim / fl) * f;
    u = (-1.0 / k) * (f + cdamp * vm);
  }
  return f;
}

struct Out {
  Vec f, ti, tj;
};

// The contact law of Sec. 2.2 for body i against body j (or a wall).
Out law(const Sim& S, bool wall, double Ri, double mi, double Rj, double mj, double delta,
        Vec nh, Vec dv, Vec wi, Vec wj, Contact& h) {
  const dcpu_params& p = S.p;
  const double Es = wall ? S.Es_pw : S.Es_pp, Gs = wall ? S.Gs_pw : S.Gs_pp;
  const double Rs = wall ? Ri : Ri * Rj / (Ri + Rj);
  const double ms = wall ? mi : mi * mj / (mi + mj);
  const double a = std::sqrt(Rs * delta);
  const double kn = 4.0 / 3.0 * Es * a, ks = 8.0 * Gs * a;
  const double cn = std::sqrt(5.0 * ms * kn) * S.beta, cs = std::sqrt(ms * ks / 6.0) * S.beta;
  const double ri = Ri - 0.5 * delta;
  const double rj = wall ? 0.0 : Rj - 0.5 * delta;
  const Vec vc = dv + crossp(nh, wall ? ri * wi : ri * wi + rj * wj);
  const Vec vn = dotp(vc, nh) * nh, vs = vc - vn;
  const Vec om = wi - wj;
  const double reff = wall ? ri : ri * rj / (ri + rj);
  const Vec vr = reff * crossp(om, nh);
  const double vt = Rs * dotp(om, nh);
  const Vec fn = (kn * delta) * nh - cn * vn;
  const double fnm = len(fn);
  const Vec fs = spring(h.us, nh, vs, ks, cs, p.mu_s * fnm, p.dt);
  const Vec fr = spring(h.ur, nh, vr, kn, cn, p.mu_r * fnm, p.dt);
  double ft = -ks * h.ut - cs * vt;
  const double limt = p.mu_t * fnm;
  if (std::fabs(ft) <= limt) {
    h.ut += p.dt * vt;
  } else {
    ft = ft > 0.0 ? limt : -limt;
    h.ut = -(ft + cs * vt) / ks;
  }
  const Vec fsn = crossp(fs, nh);
  const Vec tr = Rs * crossp(nh, fr), tt = (ft * Rs) * nh;
  Out o;
  o.f = fn + fs;
  o.ti = ri * fsn + tr + tt;
  o.tj = rj * fsn - tr - tt;
  return o;
}

Contact& find_or_create(std::vector<Contact>& list, int64_t j) {
  for (Contact& e : list)
    if (e.j == j) return e;
  list.push_back(Contact{j, vec(0, 0, 0), vec(0, 0, 0), 0.0, false});
  return list.back();
}

inline int64_t cell_coord(const Sim& S, int a, double xa) {
  int64_t c = (int64_t)std::floor((xa - S.lo[a]) * S.inv_h);
  return std::min(std::max<int64_t>(c, 0), S.nc[a] - 1);
}

void build_cells(Sim& S) {
  double hi[3];
  for (int a = 0; a < 3; ++a) {
    S.lo[a] = INFINITY;
    hi[a] = -INFINITY;
  }
  for (int64_t i = 0; i < S.n; ++i) {
    const double c[3] = {S.x[i].x, S.x[i].y, S.x[i].z};
    for (int a = 0; a < 3; ++a) {
      S.lo[a] = std::min(S.lo[a], c[a]);
      hi[a] = std::max(hi[a], c[a]);
    }
  }
  const double h = 2.0 * S.rmax;
  S.inv_h = 1.0 / h;
  int64_t total = 1;
  for (int a = 0; a < 3; ++a) {
    S.nc[a] = std::max<int64_t>(1, (int64_t)std::floor((hi[a] - S.lo[a]) / h) + 1);
    total *= S.nc[a];
  }
  S.head.assign(total, -1);
  S.next.resize(S.n);
  for (int64_t i = 0; i < S.n; ++i) {  // serial, as in the paper
    const int64_t cx = cell_coord(S, 0, S.x[i].x), cy = cell_coord(S, 1, S.x[i].y),
                  cz = cell_coord(S, 2, S.x[i].z);
    const int64_t cell = (cz * S.nc[1] + cy) * S.nc[0] + cx;
    S.next[i] = S.head[cell];
    S.head[cell] = i;
  }
  // mesh broad phase: each element's bounding box (grown by its radius and
  // R_max) is rasterised into the cells it overlaps
  S.cell_elems.assign(S.ne > 0 ? total : 0, {});
  for (int64_t k = 0; k < S.ne; ++k) {
    double blo[3] = {INFINITY, INFINITY, INFINITY}, bhi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int s = 0; s < 4 && S.el[4 * k + s] >= 0; ++s) {
      const Vec vv = S.vcur[S.el[4 * k + s]];
      const double c[3] = {vv.x, vv.y, vv.z};
      for (int a = 0; a < 3; ++a) {
        blo[a] = std::min(blo[a], c[a]);
        bhi[a] = std::max(bhi[a], c[a]);
      }
    }
    const double grow = S.erad[k] + S.rmax;
    int64_t c0[3], c1[3];
    bool outside = false;
    for (int a = 0; a < 3; ++a) {
      const double l = (blo[a] - grow - S.lo[a]) * S.inv_h, u = (bhi[a] + grow - S.lo[a]) * S.inv_h;
      if (u < 0.0 || l > (double)(S.nc[a] - 1) + 1.0) outside = true;
      c0[a] = std::max<int64_t>(0, (int64_t)std::floor(l));
      c1[a] = std::min<int64_t>(S.nc[a] - 1, (int64_t)std::floor(u));
    }
    if (outside) continue;
    for (int64_t cz = c0[2]; cz <= c1[2]; ++cz)
      for (int64_t cy = c0[1]; cy <= c1[1]; ++cy)
        for (int64_t cx = c0[0]; cx <= c1[0]; ++cx)
          S.cell_elems[(cz * S.nc[1] + cy) * S.nc[0] + cx].push_back(k);
  }
}

void mesh_pose(Sim& S) {
  const Vec Om = vec(S.p.mesh_omega[0], S.p.mesh_omega[1], S.p.mesh_omega[2]);
  const double wn = len(Om);
  if (!(wn > 0.0)) {
    S.vcur = S.vref;
    return;
  }
  const Vec k = (1.0 / wn) * Om, c = vec(S.p.mesh_center[0], S.p.mesh_center[1], S.p.mesh_center[2]);
  const double th = wn * ((double)S.steps * S.p.dt), cs = std::cos(th), sn = std::sin(th);
  S.vcur.resize(S.vref.size());
  for (size_t i = 0; i < S.vref.size(); ++i) {
    const Vec r = S.vref[i] - c;
    S.vcur[i] = c + (cs * r + sn * crossp(k, r) + (dotp(k, r) * (1.0 - cs)) * k);
  }
}

void qprod(const double* a, const double* b, double* o) {
  const double s = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  const double x = a[0] * b[1] + b[0] * a[1] + a[2] * b[3] - a[3] * b[2];
  const double y = a[0] * b[2] + b[0] * a[2] + a[3] * b[1] - a[1] * b[3];
  const double z = a[0] * b[3] + b[0] * a[3] + a[1] * b[2] - a[2] * b[1];
  o[0] = s;
  o[1] = x;
  o[2] = y;
  o[3] = z;
}

void step(Sim& S) {
  const int64_t n = S.n;
  mesh_pose(S);
  build_cells(S);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    S.F[i] = vec(0, 0, 0);
    S.T[i] = vec(0, 0, 0);
  }
  // particle pairs i < j from the 27 neighbouring cells, each evaluated once
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < n; ++i) {
    const Vec xi = S.x[i];
    const int64_t cx = cell_coord(S, 0, xi.x), cy = cell_coord(S, 1, xi.y), cz = cell_coord(S, 2, xi.z);
    for (int64_t dz = -1; dz <= 1; ++dz)
      for (int64_t dy = -1; dy <= 1; ++dy)
        for (int64_t dx = -1; dx <= 1; ++dx) {
          const int64_t X = cx + dx, Y = cy + dy, Z = cz + dz;
          if (X < 0 || Y < 0 || Z < 0 || X >= S.nc[0] || Y >= S.nc[1] || Z >= S.nc[2]) continue;
          for (int64_t j = S.head[(Z * S.nc[1] + Y) * S.nc[0] + X]; j >= 0; j = S.next[j]) {
            if (j <= i) continue;
            const Vec d = xi - S.x[j];
            const double s = S.R[i] + S.R[j];
            const double d2 = dotp(d, d);
            if (d2 > s * s) continue;
            const double dist = std::sqrt(d2);
            const double delta = s - dist;
            if (delta < 0.0 || !(dist > 0.0)) continue;
            Contact& h = find_or_create(S.c[i], j);
            h.psi = true;
            const Vec nh = (1.0 / dist) * d;
            const Out o = law(S, false, S.R[i], S.m[i], S.R[j], S.m[j], delta, nh, S.v[i] - S.v[j],
                              S.w[i], S.w[j], h);
            add_atomic(S.F[i], o.f);
            add_atomic(S.F[j], vec(-o.f.x, -o.f.y, -o.f.z));
            add_atomic(S.T[i], o.ti);
            add_atomic(S.T[j], o.tj);
          }
        }
  }
  // particle-element contacts: the elements listed in the particle's cell
  if (S.ne > 0) {
    const Vec Om = vec(S.p.mesh_omega[0], S.p.mesh_omega[1], S.p.mesh_omega[2]);
    const Vec ctr = vec(S.p.mesh_center[0], S.p.mesh_center[1], S.p.mesh_center[2]);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
      const Vec xi = S.x[i];
      const int64_t cell = (cell_coord(S, 2, xi.z) * S.nc[1] + cell_coord(S, 1, xi.y)) * S.nc[0] +
                           cell_coord(S, 0, xi.x);
      for (int64_t k : S.cell_elems[cell]) {
        const Vec d = xi - on_element(S, k, xi);
        const double dist = len(d);
        const double delta = S.R[i] + S.erad[k] - dist;
        if (delta < 0.0 || !(dist > 0.0)) continue;
        Contact& h = find_or_create(S.c[i], -k);
        h.psi = true;
        const Vec nh = (1.0 / dist) * d;
        const double ri = S.R[i] - 0.5 * delta;
        const Vec vw = crossp(Om, (xi - ri * nh) - ctr);
        const Out o = law(S, true, S.R[i], S.m[i], 0.0, 0.0, delta, nh, S.v[i] - vw, S.w[i], Om, h);
        add_atomic(S.F[i], o.f);
        add_atomic(S.T[i], o.ti);
      }
    }
  }
  // drop contacts that ended, reset the flags; integrate (Sec. 2.3)
  const dcpu_params& p = S.p;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<Contact>& L = S.c[i];
    size_t keep = 0;
    for (size_t e = 0; e < L.size(); ++e)
      if (L[e].psi) {
        L[keep] = L[e];
        L[keep].psi = false;
        ++keep;
      }
    L.resize(keep);
    const double Ri = S.R[i], mi = S.m[i], I = 0.4 * mi * Ri * Ri;
    const double ci = 9.0 * p.eta / (2.0 * p.rho * Ri * Ri), gi = 10.0 / 3.0 * ci;
    const Vec a = (1.0 / mi) * S.F[i] + vec(p.g[0], p.g[1], p.g[2]) - ci * S.v[i];
    const Vec al = (1.0 / I) * S.T[i] - gi * S.w[i];
    S.v[i] = S.v[i] + p.dt * a;
    S.x[i] = S.x[i] + p.dt * S.v[i];
    double* q = &S.q[4 * i];
    const Vec w0 = S.w[i];
    const double wn = len(w0);
    if (wn > 0.0) {
      const double ph = 0.5 * p.dt * wn, sp = std::sin(ph) / wn;
      const double r[4] = {std::cos(ph), sp * w0.x, sp * w0.y, sp * w0.z};
      double o[4];
      qprod(q, r, o);
      std::memcpy(q, o, sizeof o);
    }
    const double an = len(al);
    if (an > 0.0) {
      const double th = 0.25 * p.dt * p.dt * an, st = std::sin(th) / an;
      const double r[4] = {std::cos(th), st * al.x, st * al.y, st * al.z};
      double o[4];
      qprod(q, r, o);
      std::memcpy(q, o, sizeof o);
    }
    S.w[i] = S.w[i] + p.dt * al;
  }
  S.steps += 1;
}

}  // namespace

extern "C" {

void* dcpu_create(const dcpu_params* p, int64_t n, const double* R, const double* x,
                  const double* v, const double* w, const double* q, int64_t nv,
                  const double* vert, int64_t ne, const int32_t* elem, const double* erad) {
  Sim* S = new Sim();
  S->p = *p;
  S->n = n;
  S->R.assign(R, R + n);
  S->m.resize(n);
  S->x.resize(n);
  S->v.resize(n);
  S->w.resize(n);
  S->F.assign(n, vec(0, 0, 0));
  S->T.assign(n, vec(0, 0, 0));
  S->q.assign(q, q + 4 * n);
  S->c.resize(n);
  for (int64_t i = 0; i < n; ++i) {
    S->m[i] = 4.0 / 3.0 * M_PI * p->rho * R[i] * R[i] * R[i];
    S->x[i] = vec(x[3 * i], x[3 * i + 1], x[3 * i + 2]);
    S->v[i] = vec(v[3 * i], v[3 * i + 1], v[3 * i + 2]);
    S->w[i] = vec(w[3 * i], w[3 * i + 1], w[3 * i + 2]);
    S->rmax = std::max(S->rmax, R[i]);
  }
  S->vref.resize(nv);
  for (int64_t k = 0; k < nv; ++k) S->vref[k] = vec(vert[3 * k], vert[3 * k + 1], vert[3 * k + 2]);
  S->ne = ne;
  S->el.assign(elem, elem + 4 * ne);
  S->erad.assign(erad, erad + ne);
  const double E = p->E, nu = p->nu, G = E / (2.0 * (1.0 + nu));
  S->Es_pp = 1.0 / (2.0 * (1.0 - nu * nu) / E);
  S->Gs_pp = 1.0 / (2.0 * (2.0 - nu) / G);
  S->Es_pw = E / (1.0 - nu * nu);
  S->Gs_pw = G / (2.0 - nu);
  S->beta = damping_beta(p->e_n);
  return S;
}

void dcpu_destroy(void* s) { delete static_cast<Sim*>(s); }

void dcpu_step(void* s, int64_t nsteps) {
  Sim* S = static_cast<Sim*>(s);
  for (int64_t k = 0; k < nsteps; ++k) step(*S);
}

void dcpu_read_state(void* s, double* x, double* v, double* w, double* q) {
  Sim* S = static_cast<Sim*>(s);
  for (int64_t i = 0; i < S->n; ++i) {
    const Vec* src[3] = {&S->x[i], &S->v[i], &S->w[i]};
    double* dst[3] = {x, v, w};
    for (int a = 0; a < 3; ++a) {
      dst[a][3 * i] = src[a]->x;
      dst[a][3 * i + 1] = src[a]->y;
      dst[a][3 * i + 2] = src[a]->z;
    }
  }
  std::memcpy(q, S->q.data(), sizeof(double) * 4 * S->n);
}

void dcpu_read_forces(void* s, double* F, double* T) {
  Sim* S = static_cast<Sim*>(s);
  for (int64_t i = 0; i < S->n; ++i) {
    F[3 * i] = S->F[i].x; F[3 * i + 1] = S->F[i].y; F[3 * i + 2] = S->F[i].z;
    T[3 * i] = S->T[i].x; T[3 * i + 1] = S->T[i].y; T[3 * i + 2] = S->T[i].z;
  }
}

int dcpu_threads() { return omp_get_max_threads(); }

}  // extern "C"
