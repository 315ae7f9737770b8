// C ABI of libdem (declared in include/dem.h): scene set-up, memory, the
// per-step launch sequence (captured once into CUDA graphs), read-back,
// save/load.  Host code only; kernels live in dem_rebuild.cu, dem_step.cu and
// dem_scan.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "dem_internal.cuh"

using namespace dem;

namespace {

constexpr int kGraphSteps = 16;  // steps per replay of the long graph

// Device memory of a scene: cudaMalloc, or the caller's allocator
// (dem_scene_create_with_allocator).  Every block is released with the scene.
struct Alloc {
  std::vector<void*> ptrs;
  bool failed = false;
  dem_alloc_fn user_alloc = nullptr;
  dem_free_fn user_free = nullptr;
  void* user_ctx = nullptr;
  template <typename T>
  T* get(size_t count) {
    void* p = nullptr;
    if (failed) return nullptr;  // creation fails anyway; allocate nothing more
    if (count == 0) count = 1;
    const size_t bytes = count * sizeof(T);
    if (user_alloc) {
      p = user_alloc(bytes, user_ctx);
      if (p && (reinterpret_cast<uintptr_t>(p) & 255u) != 0) {  // records need alignment
        user_free(p, user_ctx);
        p = nullptr;
      }
      if (!p) {
        failed = true;
        return nullptr;
      }
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      failed = true;
      cudaGetLastError();
      return nullptr;
    }
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  void release() {
    for (void* p : ptrs) {
      if (user_alloc)
        user_free(p, user_ctx);
      else
        cudaFree(p);
    }
    ptrs.clear();
  }
};

// DEM_FP64_TWO_SIDED=1 in the environment evaluates every pair from both of
// its particles in one kernel (the scheme of DEM_MIXED) instead of once.
bool fp64_two_sided() {
  const char* env = std::getenv("DEM_FP64_TWO_SIDED");
  return env && env[0] == '1';
}

#ifndef DEM_MIXED_PAIRS
#define DEM_MIXED_PAIRS 0
#endif
// Whether the step evaluates each pair once (pair kernel + gather kernel)
// rather than from both sides in one kernel.
bool one_eval_per_pair(const Params& p) {
  if (p.mixed64) return false;
  return p.mixed ? DEM_MIXED_PAIRS != 0 : !fp64_two_sided();
}

bool finite_all(const double* a, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

// The mesh's elements as one table (Sec. 3.3): the triangles, then the rows of
// `elem`; four vertex indices each, -1 for unused slots.
struct ElemTable {
  std::vector<int4> el;
  std::vector<double> rad;
  static int count(const int4& e) {
    return e.w >= 0 ? 4 : (e.z >= 0 ? 3 : (e.y >= 0 ? 2 : 1));
  }
  static int vert(const int4& e, int j) {
    return j == 0 ? e.x : (j == 1 ? e.y : (j == 2 ? e.z : e.w));
  }
};

// Rectangle a-b-c-d with right angles, to the tolerance stated in dem.h.
bool is_rectangle(const double* V, const int4& e) {
  double u[3], w[3], gap[3], uu = 0, ww = 0, uw = 0, gg = 0;
  for (int a = 0; a < 3; ++a) {
    u[a] = V[3 * e.y + a] - V[3 * e.x + a];
    w[a] = V[3 * e.w + a] - V[3 * e.x + a];
    gap[a] = V[3 * e.x + a] + V[3 * e.z + a] - V[3 * e.y + a] - V[3 * e.w + a];
    uu += u[a] * u[a];
    ww += w[a] * w[a];
    uw += u[a] * w[a];
    gg += gap[a] * gap[a];
  }
  if (!(uu > 0) || !(ww > 0)) return false;
  const double lu = std::sqrt(uu), lw = std::sqrt(ww);
  return std::fabs(uw) <= 1e-9 * lu * lw && std::sqrt(gg) <= 1e-9 * (lu + lw);
}

// Build and check the element table; DEM_ERR_INVALID on a bad element.
int gather_elements(const dem_mesh* me, ElemTable& t) {
  t.el.clear();
  t.rad.clear();
  if (!me) return DEM_OK;
  if (me->n_tri < 0 || me->n_elem < 0 || me->n_tri + me->n_elem > 0x7fffffff)
    return DEM_ERR_INVALID;
  const int64_t total = me->n_tri + me->n_elem;
  if (total == 0) return DEM_OK;
  if (!me->vert || me->n_vert < 1 || me->n_vert > 0x7fffffff) return DEM_ERR_INVALID;
  if (me->n_tri > 0 && !me->tri) return DEM_ERR_INVALID;
  if (me->n_elem > 0 && !me->elem) return DEM_ERR_INVALID;
  if (!finite_all(me->vert, 3 * me->n_vert)) return DEM_ERR_INVALID;
  t.el.resize(total);
  t.rad.resize(total);
  for (int64_t k = 0; k < me->n_tri; ++k) {
    t.el[k] = make_int4(me->tri[3 * k], me->tri[3 * k + 1], me->tri[3 * k + 2], -1);
    t.rad[k] = me->tri_radius ? me->tri_radius[k] : 0.0;
    if (t.el[k].x < 0 || t.el[k].y < 0 || t.el[k].z < 0) return DEM_ERR_INVALID;
  }
  for (int64_t k = 0; k < me->n_elem; ++k) {
    const int32_t* r = me->elem + 4 * k;
    int nvk = 0;
    while (nvk < 4 && r[nvk] >= 0) ++nvk;
    if (nvk == 0) return DEM_ERR_INVALID;
    for (int j = nvk; j < 4; ++j)
      if (r[j] != -1) return DEM_ERR_INVALID;
    t.el[me->n_tri + k] = make_int4(r[0], r[1], r[2], r[3]);
    t.rad[me->n_tri + k] = me->elem_radius ? me->elem_radius[k] : 0.0;
  }
  for (int64_t k = 0; k < total; ++k) {
    const int4& e = t.el[k];
    for (int j = 0; j < ElemTable::count(e); ++j)
      if (ElemTable::vert(e, j) >= me->n_vert) return DEM_ERR_INVALID;
    if (ElemTable::count(e) == 4 && !is_rectangle(me->vert, e)) return DEM_ERR_INVALID;
    if (!(t.rad[k] >= 0) || !std::isfinite(t.rad[k])) return DEM_ERR_INVALID;
  }
  return DEM_OK;
}

}  // namespace

struct dem_scene {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  dem_params user{};
  Params p{};
  int64_t n = 0;
  int32_t nv = 0, nt = 0;
  int64_t n_init = 0;     // particles active at creation (the rest await spawning)
  size_t hist_bytes = 0;  // 64 (FP64) or 32 (mixed)
  Ctl* ctl = nullptr;
  StateBufs sb{};
  Lists L{};
  BinBuf bb{};
  MeshDev mesh{};
  double* forces = nullptr;
  double* export_buf = nullptr;  // [13 n] state read-back staging (caller order)
  Alloc mem;
  // step graphs (1 and kGraphSteps steps) for a start at an even / odd step:
  // each captured step passes its kernels the pose buffers of its parity
  cudaGraphExec_t exec1[2] = {nullptr, nullptr}, execG[2] = {nullptr, nullptr};
  int64_t step_host = 0;  // the step the device is at once the queued work ends
  cudaStream_t aux = nullptr;  // captures the conditional rebuild bodies
  // branch of a captured step that computes the next step's mesh pose beside
  // the step kernel (fork and join events)
  cudaStream_t pose_stream = nullptr;
  cudaEvent_t pose_fork = nullptr, pose_join = nullptr;
  bool conditional_graphs = false;
  bool static_mesh = true;
};

namespace {

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return DEM_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? DEM_ERR_NOMEM : DEM_ERR_CUDA;
}

#define DEM_TRY(call)                    \
  do {                                   \
    const int rc_ = cuda_status(call);   \
    if (rc_ != DEM_OK) return rc_;       \
  } while (0)

int validate(const dem_params* pr, const dem_particles* pa, const dem_mesh* me) {
  if (!pr || !pa) return DEM_ERR_INVALID;
  const double sc[] = {pr->E, pr->nu, pr->rho, pr->e_n, pr->mu_s, pr->mu_r, pr->mu_t, pr->eta,
                       pr->g[0], pr->g[1], pr->g[2], pr->dt, pr->mesh_omega[0],
                       pr->mesh_omega[1], pr->mesh_omega[2], pr->mesh_center[0],
                       pr->mesh_center[1], pr->mesh_center[2], pr->skin};
  if (!finite_all(sc, sizeof sc / sizeof sc[0])) return DEM_ERR_INVALID;
  // Table 2, "Requirements"
  if (!(pr->E > 0) || !(pr->nu > -1.0 && pr->nu <= 0.5) || !(pr->rho > 0)) return DEM_ERR_INVALID;
  if (!(pr->e_n >= 0 && pr->e_n <= 1)) return DEM_ERR_INVALID;
  if (pr->mu_s < 0 || pr->mu_r < 0 || pr->mu_t < 0 || pr->eta < 0) return DEM_ERR_INVALID;
  if (!(pr->dt > 0)) return DEM_ERR_INVALID;
  if (pr->precision != DEM_FP64 && pr->precision != DEM_MIXED && pr->precision != DEM_MIXED64)
    return DEM_ERR_INVALID;
  if (pr->max_neighbors > 64 || pr->max_mesh_contacts > 255) return DEM_ERR_INVALID;
  // spawning (Sec. 3.1)
  const bool spawn = pr->spawn_attempts != 0;
  if (pr->spawn_attempts < 0 || pr->spawn_attempts > kSpawnMaxAttempts) return DEM_ERR_INVALID;
  if (pr->step_warps > 0 && pr->step_warps != 4 && pr->step_warps != 8) return DEM_ERR_INVALID;
  if (pr->n_max > (int64_t)0x7fffffff / 2) return DEM_ERR_INVALID;
  if (spawn) {
    const double sp[] = {pr->spawn_lo[0], pr->spawn_lo[1], pr->spawn_lo[2], pr->spawn_hi[0],
                         pr->spawn_hi[1], pr->spawn_hi[2], pr->spawn_r_min, pr->spawn_r_max,
                         pr->spawn_v0[0], pr->spawn_v0[1], pr->spawn_v0[2], pr->spawn_w0[0],
                         pr->spawn_w0[1], pr->spawn_w0[2]};
    if (!finite_all(sp, sizeof sp / sizeof sp[0])) return DEM_ERR_INVALID;
    if (!(pr->spawn_r_min > 0) || !(pr->spawn_r_max >= pr->spawn_r_min)) return DEM_ERR_INVALID;
    for (int a = 0; a < 3; ++a)
      if (!(pr->spawn_lo[a] <= pr->spawn_hi[a])) return DEM_ERR_INVALID;
    if (pr->n_max < 1) return DEM_ERR_INVALID;
  }
  if (pa->n < (spawn ? 0 : 1) || pa->n > (int64_t)0x7fffffff / 2) return DEM_ERR_INVALID;
  if (pa->n > 0 && (!pa->R || !pa->x)) return DEM_ERR_INVALID;
  const int64_t n = pa->n;
  if (pa->n_materials < 0 || pa->n_materials > 65536) return DEM_ERR_INVALID;
  if (pa->n_materials > 0) {
    if (!pa->material_mu || !finite_all(pa->material_mu, 3 * (int64_t)pa->n_materials))
      return DEM_ERR_INVALID;
    for (int64_t k = 0; k < 3 * (int64_t)pa->n_materials; ++k)
      if (pa->material_mu[k] < 0) return DEM_ERR_INVALID;
    if (pa->material)
      for (int64_t i = 0; i < n; ++i)
        if (pa->material[i] < 0 || pa->material[i] >= pa->n_materials) return DEM_ERR_INVALID;
  }
  for (int64_t i = 0; i < n; ++i)
    if (!(pa->R[i] > 0) || !std::isfinite(pa->R[i])) return DEM_ERR_INVALID;
  if (!finite_all(pa->x, 3 * n)) return DEM_ERR_INVALID;
  if (pa->v && !finite_all(pa->v, 3 * n)) return DEM_ERR_INVALID;
  if (pa->w && !finite_all(pa->w, 3 * n)) return DEM_ERR_INVALID;
  if (pa->q && !finite_all(pa->q, 4 * n)) return DEM_ERR_INVALID;
  return DEM_OK;
}

double beta_of(double e_n) {
  if (e_n <= 0.0) return 1.0;
  if (e_n >= 1.0) return 0.0;
  const double l = std::log(e_n);
  const double r = M_PI / l;
  return 1.0 / std::sqrt(1.0 + r * r);
}

// Host-side split of a double into the hi/lo pair used by DEM_MIXED.
inline float int_bits_as_float(int32_t v) {
  float f;
  std::memcpy(&f, &v, sizeof f);
  return f;
}

inline void split(double a, float& hi, float& lo) {
  hi = (float)a;
  lo = (float)(a - (double)hi);
}

// The mesh pose of the step after `step`.  It depends on the step number
// only, so in a capture it is a branch of its own beside the step's kernels
// (joined before the step advances); the pose of the step itself is already
// in its buffer (computed by the previous step, or at upload).
cudaError_t fork_next_pose(dem_scene* s, int64_t step) {
  if (s->static_mesh) return cudaSuccess;
  cudaError_t e = cudaEventRecord(s->pose_fork, s->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->pose_stream, s->pose_fork, 0);
  if (e != cudaSuccess) return e;
  launch_mesh_pose(s->pose_stream, s->ctl, s->p, mesh_at(s->mesh, step + 1), 1);
  return cudaEventRecord(s->pose_join, s->pose_stream);
}
cudaError_t join_next_pose(dem_scene* s) {
  if (s->static_mesh) return cudaSuccess;
  return cudaStreamWaitEvent(s->stream, s->pose_join, 0);
}

// Enqueue one complete step on the stream (inside a capture); `step` is the
// step number it will run at (only its parity matters).
cudaError_t enqueue_step(dem_scene* s, int64_t step) {
  cudaError_t e = fork_next_pose(s, step);
  if (e != cudaSuccess) return e;
  const MeshDev mesh = mesh_at(s->mesh, step);
  launch_rebuild(s->stream, s->ctl, s->p, s->sb, s->L, s->bb, mesh);
  launch_spawn(s->stream, s->ctl, s->p, s->sb, s->bb, mesh);
  launch_step(s->stream, s->ctl, s->p, s->sb, s->L, mesh, s->forces);
  e = join_next_pose(s);
  if (e != cudaSuccess) return e;
  launch_advance(s->stream, s->ctl, s->p);
  return cudaSuccess;
}

// One step inside a stream capture, with the rebuild kernels in the body of a
// conditional (IF) graph node whose condition a one-thread kernel sets from
// ctl->rebuild: steps without a rebuild then launch only the step kernels.
cudaError_t enqueue_step_conditional(dem_scene* s, int64_t step) {
  cudaError_t e = fork_next_pose(s, step);
  if (e != cudaSuccess) return e;
  const MeshDev mesh = mesh_at(s->mesh, step);
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  e = cudaStreamGetCaptureInfo(s->stream, &cs, nullptr, &g, nullptr, nullptr, nullptr);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return e;
  launch_decide(s->stream, s->ctl, h);
  e = cudaStreamGetCaptureInfo(s->stream, &cs, nullptr, &g, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeIf;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &np);
  if (e != cudaSuccess) return e;
  cudaGraph_t body = np.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(s->aux, body, nullptr, nullptr, 0,
                                    cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  launch_rebuild(s->aux, s->ctl, s->p, s->sb, s->L, s->bb, mesh);
  cudaGraph_t body_out = nullptr;
  e = cudaStreamEndCapture(s->aux, &body_out);
  if (e != cudaSuccess) return e;
  e = cudaStreamUpdateCaptureDependencies(s->stream, &node, nullptr, 1,
                                          cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) return e;
  launch_spawn(s->stream, s->ctl, s->p, s->sb, s->bb, mesh);
  launch_step(s->stream, s->ctl, s->p, s->sb, s->L, mesh, s->forces);
  e = join_next_pose(s);
  if (e != cudaSuccess) return e;
  launch_advance(s->stream, s->ctl, s->p);
  return cudaSuccess;
}

// A graph of nsteps steps that starts at a step of parity `odd`.
int build_graph(dem_scene* s, int nsteps, int odd, cudaGraphExec_t* out) {
  // first choice: conditional rebuild bodies; fall back to the plain sequence
  // (rebuild kernels that return at once) if the driver refuses
  // DEM_GRAPH_CONDITIONAL=0 in the environment keeps every rebuild kernel a
  // plain graph node (profilers cannot see kernels of conditional graphs)
  const char* env = std::getenv("DEM_GRAPH_CONDITIONAL");
  const bool allow_cond = !(env && env[0] == '0');
  for (int attempt = 0; attempt < 2; ++attempt) {
    const bool cond = attempt == 0 && s->aux != nullptr && allow_cond;
    cudaGraph_t g = nullptr;
    DEM_TRY(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < nsteps && e == cudaSuccess; ++i) {
      e = cond ? enqueue_step_conditional(s, odd + i) : enqueue_step(s, odd + i);
    }
    const cudaError_t e2 = cudaStreamEndCapture(s->stream, &g);
    if (e == cudaSuccess && e2 == cudaSuccess) {
      e = cudaGraphInstantiate(out, g, 0);
      cudaGraphDestroy(g);
      if (e == cudaSuccess) {
        s->conditional_graphs = cond;
        return DEM_OK;
      }
    } else if (g) {
      cudaGraphDestroy(g);
    }
    cudaGetLastError();
    if (!cond) return cuda_status(e != cudaSuccess ? e : e2);
  }
  return DEM_ERR_CUDA;
}

int read_ctl(dem_scene* s, Ctl* c) {
  DEM_TRY(cudaStreamSynchronize(s->stream));
  DEM_TRY(cudaMemcpy(c, s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  return DEM_OK;
}

// Host copy of the current state records (slot order) and slot -> caller index.
struct HostState {
  std::vector<D4> Pd, Vd, Wd, Qd;
  std::vector<F8> Pm, Vm, Wm, Qm;
  std::vector<uint32_t> gid;
};

int fetch_state(dem_scene* s, const Ctl& c, HostState& h) {
  const int64_t n = s->n;
  const uint32_t ph = c.phase & 1u, lph = c.lphase & 1u;
  h.gid.resize(n);
  DEM_TRY(cudaMemcpy(h.gid.data(), s->L.b[lph].gid, n * 4, cudaMemcpyDeviceToHost));
  if (s->p.mixed) {
    h.Pm.resize(n); h.Vm.resize(n); h.Wm.resize(n); h.Qm.resize(n);
    DEM_TRY(cudaMemcpy(h.Pm.data(), s->sb.P[ph], n * sizeof(F8), cudaMemcpyDeviceToHost));
    DEM_TRY(cudaMemcpy(h.Vm.data(), s->sb.V[ph], n * sizeof(F8), cudaMemcpyDeviceToHost));
    DEM_TRY(cudaMemcpy(h.Wm.data(), s->sb.W[ph], n * sizeof(F8), cudaMemcpyDeviceToHost));
    DEM_TRY(cudaMemcpy(h.Qm.data(), s->sb.Q[ph], n * sizeof(F8), cudaMemcpyDeviceToHost));
  } else {
    h.Pd.resize(n); h.Vd.resize(n); h.Wd.resize(n); h.Qd.resize(n);
    DEM_TRY(cudaMemcpy(h.Pd.data(), s->sb.P[ph], n * sizeof(D4), cudaMemcpyDeviceToHost));
    DEM_TRY(cudaMemcpy(h.Vd.data(), s->sb.V[ph], n * sizeof(D4), cudaMemcpyDeviceToHost));
    DEM_TRY(cudaMemcpy(h.Wd.data(), s->sb.W[ph], n * sizeof(D4), cudaMemcpyDeviceToHost));
    DEM_TRY(cudaMemcpy(h.Qd.data(), s->sb.Q[ph], n * sizeof(D4), cudaMemcpyDeviceToHost));
  }
  return DEM_OK;
}

struct ContactRow {
  int64_t i, j;
  double h[7];
  uint32_t stamp;
};

// Active contacts (written in the last step) in caller indices, sorted by (i, j).
int fetch_contacts(dem_scene* s, const Ctl& c, std::vector<ContactRow>& rows) {
  const int64_t n = s->n;
  const uint32_t lph = c.lphase & 1u;
  const ListBuf& lb = s->L.b[lph];
  std::vector<uint32_t> gid(n), meta(n), offs(n + 1);
  DEM_TRY(cudaMemcpy(gid.data(), lb.gid, n * 4, cudaMemcpyDeviceToHost));
  DEM_TRY(cudaMemcpy(meta.data(), lb.meta, n * 4, cudaMemcpyDeviceToHost));
  DEM_TRY(cudaMemcpy(offs.data(), lb.offs, (n + 1) * 4, cudaMemcpyDeviceToHost));
  int maxnt = 0;
  for (int64_t t = 0; t < n; ++t) maxnt = std::max(maxnt, (int)((meta[t] >> 16) & 0xffu));
  const size_t E = offs[n];
  std::vector<uint32_t> nbr(E), tric((size_t)maxnt * n);
  std::vector<unsigned char> hpp(E * s->hist_bytes), hpm((size_t)maxnt * n * s->hist_bytes);
  if (E) {
    DEM_TRY(cudaMemcpy(nbr.data(), lb.nbr, E * 4, cudaMemcpyDeviceToHost));
    DEM_TRY(cudaMemcpy(hpp.data(), lb.hpp, hpp.size(), cudaMemcpyDeviceToHost));
  }
  if (maxnt) {
    DEM_TRY(cudaMemcpy(tric.data(), lb.tric, tric.size() * 4, cudaMemcpyDeviceToHost));
    DEM_TRY(cudaMemcpy(hpm.data(), lb.hpm, hpm.size(), cudaMemcpyDeviceToHost));
  }
  const uint32_t want = (uint32_t)c.step;  // stamp written by the last completed step
  auto decode = [&](const unsigned char* rec, ContactRow& r) {
    if (s->p.hist32) {
      HistM h;
      std::memcpy(&h, rec, sizeof h);
      for (int q = 0; q < 3; ++q) r.h[q] = h.us[q], r.h[3 + q] = h.ur[q];
      r.h[6] = h.ut;
      r.stamp = h.stamp;
    } else {
      HistD h;
      std::memcpy(&h, rec, sizeof h);
      for (int q = 0; q < 3; ++q) r.h[q] = h.us[q], r.h[3 + q] = h.ur[q];
      r.h[6] = h.ut;
      r.stamp = h.stamp;
    }
  };
  rows.clear();
  for (int64_t t = 0; t < n; ++t) {
    const int nn = (int)(meta[t] & 0xffu), nt = (int)((meta[t] >> 16) & 0xffu);
    const int64_t i = gid[t];
    for (int k = 0; k < nn; ++k) {
      const uint32_t u = nbr[offs[t] + k];
      const int64_t j = gid[u];
      if (j <= i) continue;
      ContactRow r;
      decode(&hpp[((size_t)offs[t] + k) * s->hist_bytes], r);
      if (r.stamp != want || c.step == 0) continue;
      r.i = i;
      r.j = j;
      rows.push_back(r);
    }
    for (int m = 0; m < nt; ++m) {
      ContactRow r;
      decode(&hpm[((size_t)m * n + t) * s->hist_bytes], r);
      if (r.stamp != want || c.step == 0) continue;
      r.i = i;
      r.j = -1 - (int64_t)tric[(size_t)m * n + t];
      rows.push_back(r);
    }
  }
  std::sort(rows.begin(), rows.end(), [](const ContactRow& a, const ContactRow& b) {
    return a.i != b.i ? a.i < b.i : a.j < b.j;
  });
  return DEM_OK;
}

// Install contacts as the "previous list" of every particle (slot = caller
// index) so the next rebuild carries their histories over.
int install_contacts(dem_scene* s, const std::vector<ContactRow>& rows, uint32_t lph,
                     uint32_t stamp) {
  const int64_t n = s->n;
  const ListBuf& lb = s->L.b[lph];
  std::vector<std::vector<std::pair<int64_t, const ContactRow*>>> pp(n), pm(n);
  for (const ContactRow& r : rows) {
    if (r.i < 0 || r.i >= n) return DEM_ERR_INVALID;
    if (r.j >= 0) {
      if (r.j >= n || r.j == r.i) return DEM_ERR_INVALID;
      pp[r.i].push_back({r.j, &r});
      pp[r.j].push_back({r.i, &r});
    } else {
      if (-1 - r.j >= s->nt) return DEM_ERR_INVALID;
      pm[r.i].push_back({-1 - r.j, &r});
    }
  }
  size_t maxnn = 0, maxnt = 0;
  for (int64_t i = 0; i < n; ++i) {
    std::sort(pp[i].begin(), pp[i].end());
    std::sort(pm[i].begin(), pm[i].end());
    maxnn = std::max(maxnn, pp[i].size());
    maxnt = std::max(maxnt, pm[i].size());
  }
  if (maxnn > (size_t)s->p.cap || maxnt > (size_t)s->p.capm) return DEM_ERR_CAPACITY;
  std::vector<uint32_t> meta(n), offs(n + 1), tric(maxnt * n);
  offs[0] = 0;
  for (int64_t i = 0; i < n; ++i) offs[i + 1] = offs[i] + (uint32_t)pp[i].size();
  const size_t E = offs[n];
  std::vector<uint32_t> nbr(E);  // slot = caller index here, so also the partner keys
  std::vector<unsigned char> hpp(E * s->hist_bytes), hpm(maxnt * n * s->hist_bytes);
  auto encode = [&](const ContactRow& r, unsigned char* rec) {
    if (s->p.hist32) {
      HistM h;
      for (int q = 0; q < 3; ++q) h.us[q] = (float)r.h[q], h.ur[q] = (float)r.h[3 + q];
      h.ut = (float)r.h[6];
      h.stamp = stamp;
      std::memcpy(rec, &h, sizeof h);
    } else {
      HistD h;
      for (int q = 0; q < 3; ++q) h.us[q] = r.h[q], h.ur[q] = r.h[3 + q];
      h.ut = r.h[6];
      h.stamp = stamp;
      h.pad = 0;
      std::memcpy(rec, &h, sizeof h);
    }
  };
  for (int64_t i = 0; i < n; ++i) {
    meta[i] = (uint32_t)pp[i].size() | ((uint32_t)pm[i].size() << 16);
    for (size_t k = 0; k < pp[i].size(); ++k) {
      nbr[offs[i] + k] = (uint32_t)pp[i][k].first;
      encode(*pp[i][k].second, &hpp[(offs[i] + k) * s->hist_bytes]);
    }
    for (size_t k = 0; k < pm[i].size(); ++k) {
      tric[k * n + i] = (uint32_t)pm[i][k].first;
      encode(*pm[i][k].second, &hpm[(k * n + i) * s->hist_bytes]);
    }
  }
  std::vector<uint32_t> ident(n);
  for (int64_t i = 0; i < n; ++i) ident[i] = (uint32_t)i;
  DEM_TRY(cudaMemcpy(lb.gid, ident.data(), n * 4, cudaMemcpyHostToDevice));
  DEM_TRY(cudaMemcpy(lb.meta, meta.data(), n * 4, cudaMemcpyHostToDevice));
  DEM_TRY(cudaMemcpy(lb.offs, offs.data(), (n + 1) * 4, cudaMemcpyHostToDevice));
  if (E) {
    DEM_TRY(cudaMemcpy(lb.nbr, nbr.data(), nbr.size() * 4, cudaMemcpyHostToDevice));
    DEM_TRY(cudaMemcpy(lb.ngid, nbr.data(), nbr.size() * 4, cudaMemcpyHostToDevice));
    DEM_TRY(cudaMemcpy(lb.hpp, hpp.data(), hpp.size(), cudaMemcpyHostToDevice));
  }
  if (maxnt) {
    DEM_TRY(cudaMemcpy(lb.tric, tric.data(), tric.size() * 4, cudaMemcpyHostToDevice));
    DEM_TRY(cudaMemcpy(lb.hpm, hpm.data(), hpm.size(), cudaMemcpyHostToDevice));
  }
  return DEM_OK;
}

// Upload a state given in caller order (slot = caller index) into buffer 0,
// reset the control block to (step, lphase 0), and request a rebuild.
// History records of both list buffers to "no contact" (stamp kStampNone in
// every byte pattern 0xff); after this, a record counts only once written.
int clear_histories(dem_scene* s) {
  for (int b = 0; b < 2; ++b) {
    const ListBuf& lb = s->L.b[b];
    DEM_TRY(cudaMemset(lb.hpp, 0xff, (size_t)s->p.cap * s->n * s->hist_bytes));
    if (lb.hpm) DEM_TRY(cudaMemset(lb.hpm, 0xff, (size_t)s->p.capm * s->n * s->hist_bytes));
  }
  // touch masks start clear (the gather clears them again after every step)
  if (s->p.pair_touch) DEM_TRY(cudaMemset(s->p.pair_touch, 0, (size_t)s->n * 8));
  return DEM_OK;
}

int upload_state(dem_scene* s, const double* x, const double* v, const double* w,
                 const double* q, const double* R, const int32_t* mat, int64_t step,
                 int64_t n_active, double spawn_carry, uint64_t spawn_draws) {
  const int64_t n = s->n;
  const double rho = s->p.rho;
  if (s->p.mixed) {
    std::vector<F8> P(n), V(n), W(n), Q(n);
    for (int64_t i = 0; i < n; ++i) {
      const double m = 4.0 / 3.0 * M_PI * rho * R[i] * R[i] * R[i];
      split(x[3 * i] - s->p.origin[0], P[i].hi.x, P[i].lo.x);
      split(x[3 * i + 1] - s->p.origin[1], P[i].hi.y, P[i].lo.y);
      split(x[3 * i + 2] - s->p.origin[2], P[i].hi.z, P[i].lo.z);
      split(R[i], P[i].hi.w, P[i].lo.w);
      split(v ? v[3 * i] : 0.0, V[i].hi.x, V[i].lo.x);
      split(v ? v[3 * i + 1] : 0.0, V[i].hi.y, V[i].lo.y);
      split(v ? v[3 * i + 2] : 0.0, V[i].hi.z, V[i].lo.z);
      V[i].hi.w = (float)m;
      V[i].lo.w = R[i] > 0 ? (float)(1.0 / m) : 0.f;  // inverse mass, for the contact law
      split(w ? w[3 * i] : 0.0, W[i].hi.x, W[i].lo.x);
      split(w ? w[3 * i + 1] : 0.0, W[i].hi.y, W[i].lo.y);
      split(w ? w[3 * i + 2] : 0.0, W[i].hi.z, W[i].lo.z);
      W[i].hi.w = R[i] > 0 ? (float)(1.0 / R[i]) : 0.f;  // inverse radius
      W[i].lo.w = int_bits_as_float(mat ? mat[i] : 0);  // material index (int bits)
      split(q ? q[4 * i] : 1.0, Q[i].hi.x, Q[i].lo.x);
      split(q ? q[4 * i + 1] : 0.0, Q[i].hi.y, Q[i].lo.y);
      split(q ? q[4 * i + 2] : 0.0, Q[i].hi.z, Q[i].lo.z);
      split(q ? q[4 * i + 3] : 0.0, Q[i].hi.w, Q[i].lo.w);
    }
    DEM_TRY(cudaMemcpy(s->sb.P[0], P.data(), n * sizeof(F8), cudaMemcpyHostToDevice));
    DEM_TRY(cudaMemcpy(s->sb.V[0], V.data(), n * sizeof(F8), cudaMemcpyHostToDevice));
    DEM_TRY(cudaMemcpy(s->sb.W[0], W.data(), n * sizeof(F8), cudaMemcpyHostToDevice));
    DEM_TRY(cudaMemcpy(s->sb.Q[0], Q.data(), n * sizeof(F8), cudaMemcpyHostToDevice));
  } else {
    std::vector<D4> P(n), V(n), W(n), Q(n);
    for (int64_t i = 0; i < n; ++i) {
      const double m = 4.0 / 3.0 * M_PI * rho * R[i] * R[i] * R[i];
      P[i] = make_D4(x[3 * i], x[3 * i + 1], x[3 * i + 2], R[i]);
      V[i] = v ? make_D4(v[3 * i], v[3 * i + 1], v[3 * i + 2], m) : make_D4(0, 0, 0, m);
      const double mi = mat ? (double)mat[i] : 0.0;  // material index in .w
      W[i] = w ? make_D4(w[3 * i], w[3 * i + 1], w[3 * i + 2], mi) : make_D4(0, 0, 0, mi);
      Q[i] = q ? make_D4(q[4 * i], q[4 * i + 1], q[4 * i + 2], q[4 * i + 3])
               : make_D4(1, 0, 0, 0);
    }
    DEM_TRY(cudaMemcpy(s->sb.P[0], P.data(), n * sizeof(D4), cudaMemcpyHostToDevice));
    DEM_TRY(cudaMemcpy(s->sb.V[0], V.data(), n * sizeof(D4), cudaMemcpyHostToDevice));
    DEM_TRY(cudaMemcpy(s->sb.W[0], W.data(), n * sizeof(D4), cudaMemcpyHostToDevice));
    DEM_TRY(cudaMemcpy(s->sb.Q[0], Q.data(), n * sizeof(D4), cudaMemcpyHostToDevice));
  }
  std::vector<uint32_t> ident(n);
  for (int64_t i = 0; i < n; ++i) ident[i] = (uint32_t)i;
  for (int b = 0; b < 2; ++b) {
    DEM_TRY(cudaMemcpy(s->L.b[b].gid, ident.data(), n * 4, cudaMemcpyHostToDevice));
    DEM_TRY(cudaMemset(s->L.b[b].meta, 0, n * 4));
    DEM_TRY(cudaMemset(s->L.b[b].offs, 0, (n + 1) * 4));
  }
  {
    const int rc = clear_histories(s);
    if (rc != DEM_OK) return rc;
  }
  Ctl c{};
  c.step = step;
  c.rebuild = 1;
  c.n_active = (uint32_t)n_active;
  c.spawn_carry = spawn_carry;
  c.spawn_draws = spawn_draws;
  DEM_TRY(cudaMemcpy(s->ctl, &c, sizeof c, cudaMemcpyHostToDevice));
  launch_set_pose(s->stream, s->ctl, s->p);  // rotation of this step, on the device
  return DEM_OK;
}

void destroy(dem_scene* s) {
  if (!s) return;
  for (int b = 0; b < 2; ++b) {
    if (s->exec1[b]) cudaGraphExecDestroy(s->exec1[b]);
    if (s->execG[b]) cudaGraphExecDestroy(s->execG[b]);
  }
  if (s->stream) cudaStreamSynchronize(s->stream);
  s->mem.release();
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  if (s->aux) cudaStreamDestroy(s->aux);
  if (s->pose_stream) cudaStreamDestroy(s->pose_stream);
  if (s->pose_fork) cudaEventDestroy(s->pose_fork);
  if (s->pose_join) cudaEventDestroy(s->pose_join);
  delete s;
}

}  // namespace

extern "C" {

const char* dem_status_string(int status) {
  switch (status) {
    case DEM_OK: return "ok";
    case DEM_ERR_INVALID: return "invalid argument";
    case DEM_ERR_CAPACITY: return "list capacity exceeded";
    case DEM_ERR_NONFINITE: return "non-finite particle state";
    case DEM_ERR_TIMEOUT: return "device wait timed out";
    case DEM_ERR_CUDA: return "CUDA error";
    case DEM_ERR_NOMEM: return "out of device memory";
    default: return "unknown status";
  }
}

int dem_scene_create(const dem_params* params, const dem_particles* parts, const dem_mesh* mesh,
                     void* stream, dem_scene** out) {
  return dem_scene_create_with_allocator(params, parts, mesh, stream, nullptr, nullptr, nullptr,
                                         out);
}

int dem_scene_create_with_allocator(const dem_params* params, const dem_particles* parts,
                                    const dem_mesh* mesh, void* stream, dem_alloc_fn alloc,
                                    dem_free_fn release, void* ctx, dem_scene** out) {
  if (!out) return DEM_ERR_INVALID;
  *out = nullptr;
  if ((alloc == nullptr) != (release == nullptr)) return DEM_ERR_INVALID;
  int rc = validate(params, parts, mesh);
  if (rc != DEM_OK) return rc;
  ElemTable et;
  rc = gather_elements(mesh, et);
  if (rc != DEM_OK) return rc;
  dem_scene* s = new (std::nothrow) dem_scene();
  if (!s) return DEM_ERR_NOMEM;
  s->mem.user_alloc = alloc;
  s->mem.user_free = release;
  s->mem.user_ctx = ctx;
  auto fail = [&](int code) {
    destroy(s);
    return code;
  };
  if (cudaGetDevice(&s->device) != cudaSuccess) return fail(DEM_ERR_CUDA);
  if (stream) {
    s->stream = static_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess)
      return fail(DEM_ERR_CUDA);
    s->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&s->aux, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    s->aux = nullptr;
  }
  if (cudaStreamCreateWithFlags(&s->pose_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->pose_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->pose_join, cudaEventDisableTiming) != cudaSuccess)
    return fail(DEM_ERR_CUDA);
  s->user = *params;
  const int64_t n_init = parts->n;  // active at creation; rows n_init .. n-1 await spawning
  const bool spawning = params->spawn_attempts > 0;
  const int64_t n = std::max(n_init, params->n_max);
  s->n = n;
  s->n_init = n_init;
  const bool has_mesh = !et.el.empty();
  s->nt = (int32_t)et.el.size();
  s->nv = has_mesh ? (int32_t)mesh->n_vert : 0;
  Params& p = s->p;
  p.E = params->E;
  p.nu = params->nu;
  p.rho = params->rho;
  p.e_n = params->e_n;
  p.mu_s = params->mu_s;
  p.mu_r = params->mu_r;
  p.mu_t = params->mu_t;
  p.eta = params->eta;
  p.dt = params->dt;
  for (int a = 0; a < 3; ++a) {
    p.g[a] = params->g[a];
    p.mesh_omega[a] = params->mesh_omega[a];
    p.mesh_center[a] = params->mesh_center[a];
  }
  p.beta = beta_of(p.e_n);
  {
    const double E = p.E, nu = p.nu, G = E / (2.0 * (1.0 + nu));
    p.Es_pp = 1.0 / ((1.0 - nu * nu) / E + (1.0 - nu * nu) / E);
    p.Gs_pp = 1.0 / ((2.0 - nu) / G + (2.0 - nu) / G);
    p.Es_pw = 1.0 / ((1.0 - nu * nu) / E);
    p.Gs_pw = 1.0 / ((2.0 - nu) / G);
  }
  p.f_Es_pp = (float)p.Es_pp;
  p.f_Gs_pp = (float)p.Gs_pp;
  p.f_Es_pw = (float)p.Es_pw;
  p.f_Gs_pw = (float)p.Gs_pw;
  p.f_beta = (float)p.beta;
  // c_s / c_n = sqrt(G* / (5 E*)) for either kind of contact (Eqs. cn, cs)
  p.cs_cn_pp = std::sqrt(p.Gs_pp / (5.0 * p.Es_pp));
  p.cs_cn_pw = std::sqrt(p.Gs_pw / (5.0 * p.Es_pw));
  p.f_cs_cn_pp = (float)p.cs_cn_pp;
  p.f_cs_cn_pw = (float)p.cs_cn_pw;
  p.f_mu_s = (float)p.mu_s;
  p.f_mu_r = (float)p.mu_r;
  p.f_mu_t = (float)p.mu_t;
  p.f_dt = (float)p.dt;
  for (int a = 0; a < 3; ++a) {
    p.f_g[a] = (float)p.g[a];
    p.f_omega[a] = (float)p.mesh_omega[a];
  }
  p.f_drag = (float)(9.0 * p.eta / (2.0 * p.rho));
  p.omega_norm = std::sqrt(p.mesh_omega[0] * p.mesh_omega[0] + p.mesh_omega[1] * p.mesh_omega[1] +
                           p.mesh_omega[2] * p.mesh_omega[2]);
  s->static_mesh = !(p.omega_norm > 0.0);
  p.mixed = params->precision == DEM_MIXED ? 1 : 0;
  p.mixed64 = params->precision == DEM_MIXED64 ? 1 : 0;
  p.hist32 = p.mixed || p.mixed64;
  p.record_forces = params->record_forces ? 1 : 0;
  p.n = (int32_t)n;
  p.n_tri = s->nt;
  p.cap = params->max_neighbors > 0 ? params->max_neighbors : 64;
  p.capm = params->max_mesh_contacts > 0 ? params->max_mesh_contacts : 16;
  s->hist_bytes = p.hist32 ? sizeof(HistM) : sizeof(HistD);
  p.step_warps = params->step_warps == 8 ? 8 : 4;
  p.sp_attempts = spawning ? params->spawn_attempts : 0;
  p.sp_every = params->spawn_every > 0 ? params->spawn_every : 1;
  p.sp_seed = params->spawn_seed;
  p.sp_rmin = params->spawn_r_min;
  p.sp_rmax = params->spawn_r_max;
  for (int a = 0; a < 3; ++a) {
    p.sp_lo[a] = params->spawn_lo[a];
    p.sp_hi[a] = params->spawn_hi[a];
    p.sp_v0[a] = params->spawn_v0[a];
    p.sp_w0[a] = params->spawn_w0[a];
  }

  // radii, skin, domain
  double rmax = 0, rmin = INFINITY;
  for (int64_t i = 0; i < n_init; ++i) {
    rmax = std::max(rmax, parts->R[i]);
    rmin = std::min(rmin, parts->R[i]);
  }
  if (spawning) {
    rmax = std::max(rmax, params->spawn_r_max);
    rmin = std::min(rmin, params->spawn_r_min);
  }
  const double skin = params->skin > 0 ? params->skin : 0.25 * rmax;
  double lo[3], hi[3];
  bool user_box = true;
  for (int a = 0; a < 3; ++a)
    if (!(params->domain_lo[a] < params->domain_hi[a])) user_box = false;
  if (user_box) {
    for (int a = 0; a < 3; ++a) lo[a] = params->domain_lo[a], hi[a] = params->domain_hi[a];
  } else {
    for (int a = 0; a < 3; ++a) lo[a] = INFINITY, hi[a] = -INFINITY;
    for (int64_t i = 0; i < n_init; ++i)
      for (int a = 0; a < 3; ++a) {
        lo[a] = std::min(lo[a], parts->x[3 * i + a]);
        hi[a] = std::max(hi[a], parts->x[3 * i + a]);
      }
    if (spawning)
      for (int a = 0; a < 3; ++a) {
        lo[a] = std::min(lo[a], params->spawn_lo[a]);
        hi[a] = std::max(hi[a], params->spawn_hi[a]);
      }
    double mrad = 0;
    if (has_mesh) {
      double rtri = 0;
      for (double r : et.rad) rtri = std::max(rtri, r);
      for (int64_t k = 0; k < mesh->n_vert; ++k)
        for (int a = 0; a < 3; ++a) {
          lo[a] = std::min(lo[a], mesh->vert[3 * k + a] - rtri);
          hi[a] = std::max(hi[a], mesh->vert[3 * k + a] + rtri);
        }
      mrad = rtri;
    }
    if (has_mesh && !s->static_mesh) {
      // a turning mesh: each vertex sweeps a circle about the axis; on axis a
      // that circle spans c_a + s ax_a +- r sqrt(1 - ax_a^2) (s: coordinate
      // along the axis, r: distance from it)
      double ax[3];
      for (int a = 0; a < 3; ++a) ax[a] = p.mesh_omega[a] / p.omega_norm;
      for (int64_t k = 0; k < mesh->n_vert; ++k) {
        double d[3], along = 0, r2 = 0;
        for (int a = 0; a < 3; ++a) {
          d[a] = mesh->vert[3 * k + a] - p.mesh_center[a];
          along += d[a] * ax[a];
        }
        for (int a = 0; a < 3; ++a) {
          const double perp = d[a] - along * ax[a];
          r2 += perp * perp;
        }
        const double r = std::sqrt(r2);
        for (int a = 0; a < 3; ++a) {
          const double half = r * std::sqrt(std::max(0.0, 1.0 - ax[a] * ax[a]));
          const double c = p.mesh_center[a] + along * ax[a];
          lo[a] = std::min(lo[a], c - half - mrad);
          hi[a] = std::max(hi[a], c + half + mrad);
        }
      }
    }
    const double pad = 2.0 * rmax + skin;
    for (int a = 0; a < 3; ++a) lo[a] -= pad, hi[a] += pad;
  }
  // Shifted coordinates X = x - origin, with X in [B, 2B) on each axis (B a
  // power of two), so the hi words of two positions share a binade and their
  // difference is exact.  The frame depends only on the binning box without
  // the skin, so DEM_MIXED rounding does not change with the skin.
  double bmax = 0;
  for (int a = 0; a < 3; ++a) {
    const double flo = lo[a] + (user_box ? 0.0 : skin);
    const double fhi = hi[a] - (user_box ? 0.0 : skin);
    const double ext = std::max(fhi - flo, 1e-300);
    const double B = std::ldexp(1.0, (int)std::ceil(std::log2(ext)));
    p.origin[a] = flo - B;
    p.base[a] = lo[a] - p.origin[a];  // grid corner in shifted coordinates
    bmax = std::max(bmax, B);
  }
  const double ulp_top = std::ldexp(2.0 * bmax, -23);
  const double cut0 = 2.0 * rmax + skin;
  p.list_margin = (float)(4.0 * ulp_top + 1e-6 * cut0);
  const double h = cut0 * (1.0 + 1e-6) + 2.0 * p.list_margin;
  p.h = (float)h;
  p.inv_h = (float)(1.0 / h);
  int64_t ncells = 1;
  for (int a = 0; a < 3; ++a) {
    const int64_t c = std::max<int64_t>(1, (int64_t)std::ceil((hi[a] - lo[a]) / h));
    if (c > (1 << 20)) return fail(DEM_ERR_INVALID);
    p.nc[a] = (int32_t)c;
    ncells *= c;
  }
  if (ncells > ((int64_t)1 << 30)) return fail(DEM_ERR_INVALID);
  p.ncells = ncells;
  p.skin = (float)skin;
  p.half_skin_trigger = (float)(0.5 * skin - 4.0 * ulp_top);
  if (!(p.half_skin_trigger > 0)) return fail(DEM_ERR_INVALID);
  p.rmax = (float)rmax;
  p.mesh_prefilter = (float)(16.0 * ulp_top);
  for (int a = 0; a < 3; ++a) split(p.mesh_center[a] - p.origin[a], p.center_hi[a], p.center_lo[a]);
  p.mesh_rmax = 0;
  if (has_mesh && !s->static_mesh) {
    const double ax[3] = {p.mesh_omega[0] / p.omega_norm, p.mesh_omega[1] / p.omega_norm,
                          p.mesh_omega[2] / p.omega_norm};
    for (int64_t k = 0; k < mesh->n_vert; ++k) {
      double d[3], dd = 0, along = 0;
      for (int a = 0; a < 3; ++a) {
        d[a] = mesh->vert[3 * k + a] - p.mesh_center[a];
        along += d[a] * ax[a];
      }
      for (int a = 0; a < 3; ++a) {
        const double perp = d[a] - along * ax[a];
        dd += perp * perp;
      }
      p.mesh_rmax = std::max(p.mesh_rmax, std::sqrt(dd));
    }
  }

  // device memory
  Alloc& M = s->mem;
  s->ctl = M.get<Ctl>(1);
  const size_t rec = p.mixed ? sizeof(F8) : sizeof(D4);
  for (int b = 0; b < 2; ++b) {
    s->sb.P[b] = M.get<unsigned char>(n * rec);
    s->sb.V[b] = M.get<unsigned char>(n * rec);
    s->sb.W[b] = M.get<unsigned char>(n * rec);
    s->sb.Q[b] = M.get<unsigned char>(n * rec);
    ListBuf& lb = s->L.b[b];
    lb.gid = M.get<uint32_t>(n);
    lb.posf = M.get<float4>(n);
    if (!p.mixed && !p.mixed64) lb.inv = M.get<D4>(n);
    lb.meta = M.get<uint32_t>(n);
    lb.offs = M.get<uint32_t>(n + 1);
    lb.nbr = M.get<uint32_t>((size_t)p.cap * n);
    lb.ngid = M.get<uint32_t>((size_t)p.cap * n);
    lb.hpp = M.get<unsigned char>((size_t)p.cap * n * s->hist_bytes);
    if (one_eval_per_pair(p)) {
      lb.mir = M.get<uint32_t>((size_t)p.cap * n);
      lb.back = M.get<uint8_t>((size_t)p.cap * n);
    }
    if (has_mesh) {
      lb.tric = M.get<uint32_t>((size_t)p.capm * n);
      lb.hpm = M.get<unsigned char>((size_t)p.capm * n * s->hist_bytes);
    }
  }
  s->bb.key = M.get<uint32_t>(n);
  s->bb.local = M.get<uint32_t>(n);
  s->bb.order = M.get<uint32_t>(n);
  // one cell more than the grid: inactive particles (awaiting spawning)
  s->bb.cell_count = M.get<uint32_t>(ncells + 1);
  s->bb.cell_start = M.get<uint32_t>(ncells + 2);
  s->bb.block_sums = M.get<uint32_t>(scan_block_sums_size(std::max<int64_t>(ncells + 1, n)) + 1);
  s->bb.tmp_nbr = M.get<uint32_t>((size_t)p.cap * n);
  s->bb.tmp_gid = M.get<uint32_t>((size_t)p.cap * n);
  s->bb.tmp_hsrc = M.get<uint32_t>((size_t)p.cap * n);
  s->bb.tmp_cnt = M.get<uint32_t>(n);
  s->bb.tmp_offs = M.get<uint32_t>(n + 1);
  if (p.record_forces) s->forces = M.get<double>(6 * (size_t)n);
  s->export_buf = M.get<double>(13 * (size_t)n);
  if (one_eval_per_pair(p)) {  // one evaluation per pair
    p.pair_res = M.get<unsigned char>((size_t)p.cap * n * pair_result_bytes());
    p.pair_touch = M.get<unsigned long long>((size_t)n);
  }
  if (has_mesh) {
    s->bb.tcell_count = M.get<uint32_t>(ncells);
    s->bb.tcell_start = M.get<uint32_t>(ncells + 1);
    s->bb.tcell_overflow = M.get<uint32_t>(2);  // [1]: element lists of a still mesh built
    // capacity: for every element, the cells of a cube around its bounding
    // ball grown by the reach (valid for any pose of a rigid mesh)
    const double reach = rmax + skin + 2.0 * p.list_margin;
    double tcap = 0, max_cells = 1;
    for (int k = 0; k < s->nt; ++k) {
      const int4 e = et.el[k];
      const int nvk = ElemTable::count(e);
      double c[3] = {0, 0, 0};
      for (int j = 0; j < nvk; ++j)
        for (int a = 0; a < 3; ++a) c[a] += mesh->vert[3 * ElemTable::vert(e, j) + a] / nvk;
      double rb = 0;
      for (int j = 0; j < nvk; ++j) {
        double d2 = 0;
        for (int a = 0; a < 3; ++a) {
          const double d = mesh->vert[3 * ElemTable::vert(e, j) + a] - c[a];
          d2 += d * d;
        }
        rb = std::max(rb, std::sqrt(d2));
      }
      const double side = std::ceil(2.0 * (rb + et.rad[k] + reach) / h) + 2.0;
      tcap += std::min((double)ncells, side * side * side);
      // cells the binning kernel walks for this element: its bounding box
      // at the reference pose grown by the reach (a turning element's box
      // changes, which changes only the work per block)
      double cells = 1;
      for (int a = 0; a < 3; ++a) {
        double lo = 1e300, hi = -1e300;
        for (int j = 0; j < nvk; ++j) {
          const double x = mesh->vert[3 * ElemTable::vert(e, j) + a];
          lo = std::min(lo, x);
          hi = std::max(hi, x);
        }
        cells *= std::floor((hi - lo + 2.0 * (et.rad[k] + reach)) / h) + 2.0;
      }
      max_cells = std::max(max_cells, cells);
    }
    // large elements (a floor under a spreading pile) get several blocks each,
    // about 4096 cells per block
    p.tri_chunks = (int32_t)std::min(65535.0, std::max(1.0, std::ceil(max_cells / 4096.0)));
    if (tcap > 2.0e9) return fail(DEM_ERR_NOMEM);
    s->bb.tcap = (uint32_t)tcap + 1024;
    s->bb.tcell_tri = M.get<uint32_t>(s->bb.tcap);
    s->mesh.ref = M.get<D4>(s->nv);
    s->mesh.tri = M.get<int4>(s->nt);
    s->mesh.rad = M.get<double>(s->nt);
    s->mesh.cur = M.get<D4>(4 * (size_t)s->nt);
    s->mesh.curf = M.get<float4>(4 * (size_t)s->nt);
    s->mesh.curl = M.get<float4>(4 * (size_t)s->nt);
    s->mesh.plane = M.get<float4>(2 * (size_t)s->nt);
    s->mesh.nref = M.get<D4>(s->nt);
    s->mesh.cur_odd = M.get<D4>(4 * (size_t)s->nt);
    s->mesh.curf_odd = M.get<float4>(4 * (size_t)s->nt);
    s->mesh.curl_odd = M.get<float4>(4 * (size_t)s->nt);
    s->mesh.plane_odd = M.get<float4>(2 * (size_t)s->nt);
  }
  if (parts->n_materials > 0) {
    p.n_mat = parts->n_materials;
    float4* mf = M.get<float4>(p.n_mat);
    D4* md = M.get<D4>(p.n_mat);
    if (M.failed) return fail(DEM_ERR_NOMEM);
    std::vector<float4> hf(p.n_mat);
    std::vector<D4> hd(p.n_mat);
    for (int k = 0; k < p.n_mat; ++k) {
      const double* m = parts->material_mu + 3 * (size_t)k;
      hf[k] = make_float4((float)m[0], (float)m[1], (float)m[2], 0.f);
      hd[k] = make_D4(m[0], m[1], m[2], 0.0);
    }
    if (cudaMemcpy(mf, hf.data(), p.n_mat * sizeof(float4), cudaMemcpyHostToDevice) ||
        cudaMemcpy(md, hd.data(), p.n_mat * sizeof(D4), cudaMemcpyHostToDevice))
      return fail(DEM_ERR_CUDA);
    p.mat_f = mf;
    p.mat_d = md;
  }
  if (M.failed) return fail(DEM_ERR_NOMEM);
  if (has_mesh && cudaMemset(s->bb.tcell_overflow, 0, 2 * sizeof(uint32_t)) != cudaSuccess)
    return fail(DEM_ERR_CUDA);
  s->mesh.nv = s->nv;
  s->mesh.nt = s->nt;

  if (has_mesh) {
    std::vector<D4> ref(s->nv);
    for (int k = 0; k < s->nv; ++k)
      ref[k] = make_D4(mesh->vert[3 * k], mesh->vert[3 * k + 1], mesh->vert[3 * k + 2], 0);
    // face normals at the reference pose: (V1 - V0) x (V2 - V0), or V3 for the
    // far corner of a rectangle; the pose kernel rotates them with the vertices
    std::vector<D4> nref(s->nt, make_D4(0, 0, 0, 0));
    for (int k = 0; k < s->nt; ++k) {
      const int4 e = et.el[k];
      if (e.z < 0) continue;
      const D4 a = ref[e.x], b = ref[e.y], c = ref[e.w >= 0 ? e.w : e.z];
      const double ux = b.x - a.x, uy = b.y - a.y, uz = b.z - a.z;
      const double vx = c.x - a.x, vy = c.y - a.y, vz = c.z - a.z;
      const double nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
      const double len = std::sqrt(nx * nx + ny * ny + nz * nz);
      if (len > 0.0) nref[k] = make_D4(nx / len, ny / len, nz / len, 0);
    }
    if (cudaMemcpy(s->mesh.ref, ref.data(), s->nv * sizeof(D4), cudaMemcpyHostToDevice) ||
        cudaMemcpy(s->mesh.nref, nref.data(), s->nt * sizeof(D4), cudaMemcpyHostToDevice) ||
        cudaMemcpy(s->mesh.tri, et.el.data(), s->nt * sizeof(int4), cudaMemcpyHostToDevice) ||
        cudaMemcpy(s->mesh.rad, et.rad.data(), s->nt * sizeof(double), cudaMemcpyHostToDevice))
      return fail(DEM_ERR_CUDA);
  }
  // kernels per step: mesh pose, [decide], rebuild (prep, clear, count, 3 scan,
  // scatter, cell sort, permute, [mesh: clear, count, 3 scan, check, clear, fill,
  // sort], list build, 3 scan, compact, end), step, advance -- see dem_get_stats
  {
    // capacity rows: the given particles, then inactive rows (radius 0)
    std::vector<double> R(n, 0.0), x(3 * n, 0.0), v(3 * n, 0.0), w(3 * n, 0.0), q(4 * n, 0.0);
    for (int64_t i = 0; i < n; ++i) q[4 * i] = 1.0;
    for (int64_t i = 0; i < n_init; ++i) {
      R[i] = parts->R[i];
      for (int a = 0; a < 3; ++a) {
        x[3 * i + a] = parts->x[3 * i + a];
        if (parts->v) v[3 * i + a] = parts->v[3 * i + a];
        if (parts->w) w[3 * i + a] = parts->w[3 * i + a];
      }
      if (parts->q)
        for (int a = 0; a < 4; ++a) q[4 * i + a] = parts->q[4 * i + a];
    }
    std::vector<int32_t> mat(n, 0);
    if (parts->material && parts->n_materials > 0)
      for (int64_t i = 0; i < n_init; ++i) mat[i] = parts->material[i];
    rc = upload_state(s, x.data(), v.data(), w.data(), q.data(), R.data(), mat.data(), 0,
                      n_init, -1.0, 0);
  }
  if (rc != DEM_OK) return fail(rc);
  // poses of steps 0 and 1 (a static mesh keeps them)
  s->step_host = 0;
  launch_mesh_pose(s->stream, s->ctl, s->p, mesh_at(s->mesh, 0), 0);
  launch_mesh_pose(s->stream, s->ctl, s->p, mesh_at(s->mesh, 1), 1);
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(DEM_ERR_CUDA);
  // capture and instantiate the step graphs now (1 and kGraphSteps steps,
  // both parities), so that no dem_step call pays for it on the host while
  // the device waits; a failure here leaves them to be built on first use
  for (int odd = 0; odd < 2; ++odd) {
    if (!s->exec1[odd] && build_graph(s, 1, odd, &s->exec1[odd]) != DEM_OK)
      s->exec1[odd] = nullptr;
    if (!s->execG[odd] && build_graph(s, kGraphSteps, odd, &s->execG[odd]) != DEM_OK)
      s->execG[odd] = nullptr;
  }
  cudaGetLastError();
  *out = s;
  return DEM_OK;
}

int dem_step(dem_scene* s, int64_t nsteps) {
  if (!s || nsteps < 0) return DEM_ERR_INVALID;
  if (nsteps == 0) return DEM_OK;
  // graphs are built on first use, per parity of the starting step
  int64_t left = nsteps;
  while (left > 0) {
    const int odd = (int)(s->step_host & 1);
    const int k = left >= kGraphSteps ? kGraphSteps : 1;
    cudaGraphExec_t* ex = k == kGraphSteps ? s->execG : s->exec1;
    if (!ex[odd]) {
      const int rc = build_graph(s, k, odd, &ex[odd]);
      if (rc != DEM_OK) return rc;
    }
    DEM_TRY(cudaGraphLaunch(ex[odd], s->stream));
    left -= k;
    s->step_host += k;
  }
  return DEM_OK;
}

int dem_step_timed(dem_scene* s, int64_t nsteps, double* phase_ms) {
  if (!s || nsteps < 0 || !phase_ms) return DEM_ERR_INVALID;
  cudaEvent_t ev[5];
  for (int i = 0; i < 5; ++i)
    if (cudaEventCreate(&ev[i]) != cudaSuccess) {
      for (int j = 0; j < i; ++j) cudaEventDestroy(ev[j]);
      return DEM_ERR_CUDA;
    }
  int rc = DEM_OK;
  double acc[4] = {0, 0, 0, 0};
  for (int64_t k = 0; k < nsteps && rc == DEM_OK; ++k) {
    // phase by phase on one stream; the pose timed is that of the next step
    const MeshDev mesh = mesh_at(s->mesh, s->step_host);
    cudaEventRecord(ev[0], s->stream);
    if (!s->static_mesh)
      launch_mesh_pose(s->stream, s->ctl, s->p, mesh_at(s->mesh, s->step_host + 1), 1);
    cudaEventRecord(ev[1], s->stream);
    launch_rebuild(s->stream, s->ctl, s->p, s->sb, s->L, s->bb, mesh);
    launch_spawn(s->stream, s->ctl, s->p, s->sb, s->bb, mesh);
    cudaEventRecord(ev[2], s->stream);
    launch_step(s->stream, s->ctl, s->p, s->sb, s->L, mesh, s->forces);
    cudaEventRecord(ev[3], s->stream);
    launch_advance(s->stream, s->ctl, s->p);
    ++s->step_host;
    cudaEventRecord(ev[4], s->stream);
    rc = cuda_status(cudaEventSynchronize(ev[4]));
    for (int i = 0; i < 4 && rc == DEM_OK; ++i) {
      float ms = 0.f;
      rc = cuda_status(cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
      acc[i] += ms;
    }
  }
  for (int i = 0; i < 5; ++i) cudaEventDestroy(ev[i]);
  for (int i = 0; i < 4; ++i) phase_ms[i] += acc[i];
  if (rc != DEM_OK) return rc;
  return dem_synchronize(s);
}

int dem_read_radii(dem_scene* s, double* R) {
  if (!s || !R) return DEM_ERR_INVALID;
  Ctl c;
  int rc = read_ctl(s, &c);
  if (rc != DEM_OK) return rc;
  HostState h;
  rc = fetch_state(s, c, h);
  if (rc != DEM_OK) return rc;
  for (int64_t t = 0; t < s->n; ++t)
    R[h.gid[t]] = s->p.mixed ? (double)h.Pm[t].hi.w + (double)h.Pm[t].lo.w : h.Pd[t].w;
  return (int)c.status;
}

int dem_synchronize(dem_scene* s) {
  if (!s) return DEM_ERR_INVALID;
  Ctl c;
  int rc = read_ctl(s, &c);
  if (rc != DEM_OK) return rc;
  return (int)c.status;
}

int dem_read_state(dem_scene* s, double* x, double* v, double* w, double* q) {
  if (!s) return DEM_ERR_INVALID;
  // converted and put in caller order on the device, then one copy per array
  const int64_t n = s->n;
  launch_export_state(s->stream, s->ctl, s->p, s->sb, s->L, n, s->export_buf);
  DEM_TRY(cudaGetLastError());
  double* const dst[4] = {x, v, w, q};
  for (int k = 0; k < 4; ++k) {
    if (!dst[k]) continue;
    const size_t off = (size_t)(3 * k) * n, len = (size_t)(k == 3 ? 4 : 3) * n;
    DEM_TRY(cudaMemcpyAsync(dst[k], s->export_buf + off, len * sizeof(double),
                            cudaMemcpyDeviceToHost, s->stream));
  }
  Ctl c;
  const int rc = read_ctl(s, &c);
  if (rc != DEM_OK) return rc;
  return (int)c.status;
}

int dem_read_forces(dem_scene* s, double* F, double* T) {
  if (!s || !s->forces) return DEM_ERR_INVALID;
  Ctl c;
  int rc = read_ctl(s, &c);
  if (rc != DEM_OK) return rc;
  const int64_t n = s->n;
  std::vector<double> f(6 * (size_t)n);
  std::vector<uint32_t> gid(n);
  DEM_TRY(cudaMemcpy(f.data(), s->forces, f.size() * 8, cudaMemcpyDeviceToHost));
  DEM_TRY(cudaMemcpy(gid.data(), s->L.b[c.lphase & 1u].gid, n * 4, cudaMemcpyDeviceToHost));
  for (int64_t t = 0; t < n; ++t) {
    const int64_t i = gid[t];
    for (int a = 0; a < 3; ++a) {
      if (F) F[3 * i + a] = f[6 * t + a];
      if (T) T[3 * i + a] = f[6 * t + 3 + a];
    }
  }
  return (int)c.status;
}

int dem_read_contacts(dem_scene* s, int64_t capacity, int64_t* keys, double* hist,
                      int64_t* count) {
  if (!s || !count) return DEM_ERR_INVALID;
  Ctl c;
  int rc = read_ctl(s, &c);
  if (rc != DEM_OK) return rc;
  std::vector<ContactRow> rows;
  rc = fetch_contacts(s, c, rows);
  if (rc != DEM_OK) return rc;
  *count = (int64_t)rows.size();
  if ((int64_t)rows.size() > capacity) return DEM_ERR_CAPACITY;
  for (size_t k = 0; k < rows.size(); ++k) {
    if (keys) keys[2 * k] = rows[k].i, keys[2 * k + 1] = rows[k].j;
    if (hist) std::memcpy(hist + 7 * k, rows[k].h, 7 * sizeof(double));
  }
  return (int)c.status;
}

int dem_get_stats(dem_scene* s, dem_stats* out) {
  if (!s || !out) return DEM_ERR_INVALID;
  Ctl c;
  int rc = read_ctl(s, &c);
  if (rc != DEM_OK) return rc;
  out->steps = c.step;
  out->rebuilds = c.rebuilds;
  out->pair_contacts = c.pair_contacts_last / 2;
  out->mesh_contacts = c.mesh_contacts_last;
  out->list_entries = c.list_entries;
  out->mesh_candidates = c.mesh_candidates;
  out->max_list_len = (int32_t)c.max_list_len;
  out->status = (int32_t)c.status;
  out->active = c.n_active;
  out->capacity = s->n;
  const int32_t rebuild_launches = 15 + (s->nt > 0 ? 9 : 0) + (s->p.pair_res ? 1 : 0);
  const int32_t base = (s->static_mesh ? 0 : 1) + 2 + (s->p.sp_attempts > 0 ? 1 : 0) +
                       (s->p.pair_res ? 1 : 0);
  if (s->conditional_graphs) {
    out->launches_per_step = base + 1;
    out->launches_per_rebuild = rebuild_launches;
  } else {
    out->launches_per_step = base + rebuild_launches;
    out->launches_per_rebuild = 0;
  }
  return DEM_OK;
}

// Save format (little-endian, native struct layout):
//   u64 magic, u64 version (2), i64 n (rows), i64 mesh elements, dem_params,
//   i64 step, i64 active particles, u64 spawn draws, f64 carried spawn radius,
//   n records P, V, W, Q in caller order (D4 or F8 by precision),
//   n radii (double), i64 m, m x (i64 i, i64 j, double h[7]).
static const uint64_t kMagic = 0x4d45445f42503347ull;  // "G3PB_DEM"

int dem_save(dem_scene* s, void* buf, size_t* len) {
  if (!s || !len) return DEM_ERR_INVALID;
  Ctl c;
  int rc = read_ctl(s, &c);
  if (rc != DEM_OK) return rc;
  // a capacity overflow is found while the lists are rebuilt, before the step
  // does any work: the state and contact history of the last completed step
  // are intact, so they can still be saved (and restored into a scene with
  // larger capacities)
  if (c.status && c.status != DEM_ERR_CAPACITY) return (int)c.status;
  HostState h;
  rc = fetch_state(s, c, h);
  if (rc != DEM_OK) return rc;
  std::vector<ContactRow> rows;
  rc = fetch_contacts(s, c, rows);
  if (rc != DEM_OK) return rc;
  const int64_t n = s->n;
  const size_t rec = s->p.mixed ? sizeof(F8) : sizeof(D4);
  const size_t need = 8 * 4 + sizeof(dem_params) + 8 + 24 + 4 * n * rec + 8 * n + 8 +
                      rows.size() * (16 + 56);
  if (!buf) {
    *len = need;
    return DEM_OK;
  }
  if (*len < need) {
    *len = need;
    return DEM_ERR_CAPACITY;
  }
  unsigned char* o = static_cast<unsigned char*>(buf);
  auto put = [&](const void* src, size_t b) {
    std::memcpy(o, src, b);
    o += b;
  };
  const uint64_t ver = 2;
  const int64_t nt = s->nt;
  const int64_t na = c.n_active;
  put(&kMagic, 8);
  put(&ver, 8);
  put(&n, 8);
  put(&nt, 8);
  put(&s->user, sizeof(dem_params));
  put(&c.step, 8);
  put(&na, 8);
  put(&c.spawn_draws, 8);
  put(&c.spawn_carry, 8);
  // records in caller order
  std::vector<unsigned char> tmp(n * rec);
  for (int part = 0; part < 4; ++part) {
    for (int64_t t = 0; t < n; ++t) {
      const int64_t i = h.gid[t];
      const void* src;
      if (s->p.mixed)
        src = part == 0 ? (const void*)&h.Pm[t] : part == 1 ? (const void*)&h.Vm[t]
              : part == 2 ? (const void*)&h.Wm[t] : (const void*)&h.Qm[t];
      else
        src = part == 0 ? (const void*)&h.Pd[t] : part == 1 ? (const void*)&h.Vd[t]
              : part == 2 ? (const void*)&h.Wd[t] : (const void*)&h.Qd[t];
      std::memcpy(&tmp[i * rec], src, rec);
    }
    put(tmp.data(), n * rec);
  }
  std::vector<double> R(n);
  for (int64_t t = 0; t < n; ++t) {
    const int64_t i = h.gid[t];
    R[i] = s->p.mixed ? (double)h.Pm[t].hi.w + (double)h.Pm[t].lo.w : h.Pd[t].w;
  }
  put(R.data(), 8 * n);
  const int64_t m = (int64_t)rows.size();
  put(&m, 8);
  for (const ContactRow& r : rows) {
    put(&r.i, 8);
    put(&r.j, 8);
    put(r.h, 56);
  }
  *len = need;
  return DEM_OK;
}

int dem_load(dem_scene* s, const void* buf, size_t len) {
  if (!s || !buf) return DEM_ERR_INVALID;
  const unsigned char* in = static_cast<const unsigned char*>(buf);
  const unsigned char* end = in + len;
  auto get = [&](void* dst, size_t b) {
    if (in + b > end) return false;
    std::memcpy(dst, in, b);
    in += b;
    return true;
  };
  uint64_t magic, ver;
  int64_t n, nt, step;
  dem_params up;
  if (!get(&magic, 8) || !get(&ver, 8) || !get(&n, 8) || !get(&nt, 8)) return DEM_ERR_INVALID;
  if (magic != kMagic || ver != 2 || n != s->n || nt != s->nt) return DEM_ERR_INVALID;
  int64_t na;
  uint64_t draws;
  double carry;
  if (!get(&up, sizeof up) || !get(&step, 8) || !get(&na, 8) || !get(&draws, 8) ||
      !get(&carry, 8))
    return DEM_ERR_INVALID;
  if (na < 0 || na > n) return DEM_ERR_INVALID;
  if (up.precision != s->user.precision) return DEM_ERR_INVALID;
  const size_t rec = s->p.mixed ? sizeof(F8) : sizeof(D4);
  if (in + 4 * n * rec + 8 * n + 8 > end) return DEM_ERR_INVALID;
  DEM_TRY(cudaStreamSynchronize(s->stream));
  void* dst[4] = {s->sb.P[0], s->sb.V[0], s->sb.W[0], s->sb.Q[0]};
  for (int part = 0; part < 4; ++part) {
    DEM_TRY(cudaMemcpy(dst[part], in, n * rec, cudaMemcpyHostToDevice));
    in += n * rec;
  }
  in += 8 * n;  // radii (already inside the P records)
  int64_t m;
  if (!get(&m, 8) || m < 0) return DEM_ERR_INVALID;
  std::vector<ContactRow> rows(m);
  for (int64_t k = 0; k < m; ++k) {
    if (!get(&rows[k].i, 8) || !get(&rows[k].j, 8) || !get(rows[k].h, 56)) return DEM_ERR_INVALID;
  }
  std::vector<uint32_t> ident(n);
  for (int64_t i = 0; i < n; ++i) ident[i] = (uint32_t)i;
  for (int b = 0; b < 2; ++b) {
    DEM_TRY(cudaMemcpy(s->L.b[b].gid, ident.data(), n * 4, cudaMemcpyHostToDevice));
    DEM_TRY(cudaMemset(s->L.b[b].meta, 0, n * 4));
    DEM_TRY(cudaMemset(s->L.b[b].offs, 0, (n + 1) * 4));
  }
  int rc = clear_histories(s);
  if (rc != DEM_OK) return rc;
  rc = install_contacts(s, rows, 0, (uint32_t)step);
  if (rc != DEM_OK) return rc;
  Ctl c{};
  c.step = step;
  c.rebuild = 1;
  c.n_active = (uint32_t)na;
  c.spawn_draws = draws;
  c.spawn_carry = carry;
  DEM_TRY(cudaMemcpy(s->ctl, &c, sizeof c, cudaMemcpyHostToDevice));
  launch_set_pose(s->stream, s->ctl, s->p);
  s->step_host = step;
  launch_mesh_pose(s->stream, s->ctl, s->p, mesh_at(s->mesh, step), 0);
  launch_mesh_pose(s->stream, s->ctl, s->p, mesh_at(s->mesh, step + 1), 1);
  DEM_TRY(cudaStreamSynchronize(s->stream));
  return DEM_OK;
}

void dem_scene_destroy(dem_scene* s) { destroy(s); }

}  // extern "C"
