// List rebuild: cell binning by counting sort, permutation of the particle
// state into cell order, per-cell triangle lists, and the Verlet list build
// with the pair-key history remap.
//
// The paper rebuilds a linked-cell list every step (Sec. 3.3); here cells are
// only used to rebuild a Verlet list with skin (the extension of Sec. 7), and
// the whole rebuild runs only in steps where the control block asks for it.
// Every kernel returns at once otherwise, so a step is a fixed launch
// sequence that a CUDA graph can replay.
//
// Determinism: particles are ordered by cell and, within a cell, by caller
// index; lists are ordered by partner caller index; triangle lists by triangle
// index.  Atomics are used only on integers (counts and arrival slots) whose
// final values do not depend on thread order, and the within-cell sort removes
// the arrival order.  The result depends only on positions.
#include <algorithm>
#include <cfloat>

#include "dem_geom.cuh"
#include "dem_internal.cuh"
#include "dem_math.cuh"

namespace dem {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ bool rebuilding(const Ctl* ctl) {
  return ctl->rebuild != 0 && ctl->status == 0;
}

__device__ __forceinline__ void set_status(Ctl* ctl, uint32_t code) {
  atomicCAS(&ctl->status, 0u, code);
}

// Shifted float position of slot s in the current dynamic state.
__device__ __forceinline__ float4 posf_of(const Params& p, const void* state, uint32_t s) {
  if (p.mixed) {
    const F8 P = static_cast<const F8*>(state)[s];
    return make_float4(P.hi.x + P.lo.x, P.hi.y + P.lo.y, P.hi.z + P.lo.z, P.hi.w + P.lo.w);
  }
  const D4 P = static_cast<const D4*>(state)[s];
  return make_float4((float)(P.x - p.origin[0]), (float)(P.y - p.origin[1]),
                     (float)(P.z - p.origin[2]), (float)P.w);
}

// 1/R, 1/m and 1/I of a DEM_FP64 particle, each division written as the
// step's law and integrator write it, so with the same bits; zero for a row
// awaiting spawning.  (Only DEM_FP64 keeps them.)
__device__ __forceinline__ D4 inverses(const D4& P, const D4& V) {
  const double R = P.w, mass = V.w;
  if (R == 0.0) return make_D4(0.0, 0.0, 0.0, 0.0);
  const double I = 2.0 / 5.0 * mass * R * R;
  return make_D4(1.0 / R, 1.0 / mass, 1.0 / I, 0.0);
}
__device__ __forceinline__ D4 inverses(const F8&, const F8&) {
  return make_D4(0.0, 0.0, 0.0, 0.0);
}

// The element cell lists are built once, at the first rebuild, in the mesh's
// own frame (the elements at the reference pose), and kept: the mesh is rigid
// and the grid fixed.  A particle looks up the list of the cell that holds its
// position turned back by the mesh's current rotation (distances to the
// elements are the same in both frames).  bb.tcell_overflow[1] marks the lists
// built.  Only the scan of their counts runs again, to the same offsets.
__device__ __forceinline__ bool tcells_kept(const Params&, const BinBuf& bb) {
  return bb.tcell_overflow[1] != 0u;
}

// Vertex slot j of element k at the reference pose, shifted and rounded like
// the pose arrays (unused slots repeat vertex 0); w = the vertex count in slot 0.
__device__ __forceinline__ float4 ref_vertex(const Params& p, const MeshDev& mesh, int4 tv,
                                             int nvk, int j) {
  const int vi = j < nvk ? (j == 0 ? tv.x : (j == 1 ? tv.y : (j == 2 ? tv.z : tv.w))) : tv.x;
  const D4 r = mesh.ref[vi];
  return make_float4((float)(r.x - p.origin[0]), (float)(r.y - p.origin[1]),
                     (float)(r.z - p.origin[2]), j == 0 ? (float)nvk : 0.f);
}

// A shifted position turned back into the mesh's reference frame: the
// rotation by -theta (cos c, sin s) about the axis through the mesh centre.
__device__ __forceinline__ V3<float> to_mesh_frame(const Params& p, V3<float> q, float c,
                                                   float s) {
  const float wn = (float)p.omega_norm;
  const V3<float> ax = mk(p.f_omega[0] / wn, p.f_omega[1] / wn, p.f_omega[2] / wn);
  const V3<float> cen = mk(p.center_hi[0], p.center_hi[1], p.center_hi[2]);
  const V3<float> r = q - cen;
  return cen + (c * r - s * cross(ax, r) + ((1.f - c) * dot(ax, r)) * ax);
}

__global__ void k_clear(const Ctl* ctl, uint32_t* a, int64_t n) {
  if (!rebuilding(ctl)) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = 0u;
}

// k_clear of the element counts, skipped while the lists are kept
__global__ void k_clear_tcells(const Ctl* ctl, Params p, BinBuf bb) {
  if (!rebuilding(ctl) || tcells_kept(p, bb)) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.ncells;
       i += (int64_t)gridDim.x * blockDim.x)
    bb.tcell_count[i] = 0u;
}

// key = cell of each particle; local = its arrival index in the cell.
// Inactive particles (radius 0, awaiting spawning) go to an extra cell after
// the grid that no search visits, in caller order: they are caller indices
// n_active .. n-1, so each one's slot is its caller index.
__global__ void __launch_bounds__(kThreads)
k_bin_count(const Ctl* ctl, Params p, StateBufs sb, BinBuf bb, Lists L) {
  if (!rebuilding(ctl)) return;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.n) return;
  const float4 X = posf_of(p, buf_of(sb.P, ctl->phase & 1u), s);
  if (X.w == 0.f) {
    const uint32_t c = (uint32_t)p.ncells;
    bb.key[s] = c;
    bb.local[s] = list_of(L, ctl->lphase & 1u).gid[s] - ctl->n_active;
    atomicAdd(&bb.cell_count[c], 1u);
    return;
  }
  const uint32_t c = cell_index(p, cell_coords(p, X.x, X.y, X.z));
  bb.key[s] = c;
  bb.local[s] = atomicAdd(&bb.cell_count[c], 1u);
}

__global__ void __launch_bounds__(kThreads)
k_scatter(const Ctl* ctl, Params p, BinBuf bb) {
  if (!rebuilding(ctl)) return;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.n) return;
  bb.order[bb.cell_start[bb.key[s]] + bb.local[s]] = (uint32_t)s;
}

// Within each cell, order the particles by caller index (insertion sort; a
// cell holds a handful of particles).
__global__ void __launch_bounds__(kThreads)
k_cell_sort(const Ctl* ctl, Params p, BinBuf bb, Lists L) {
  if (!rebuilding(ctl)) return;
  const uint32_t* gid_old = list_of(L, ctl->lphase & 1u).gid;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < p.ncells;
       c += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t a = bb.cell_start[c], b = bb.cell_start[c + 1];
    for (uint32_t i = a + 1; i < b; ++i) {
      const uint32_t v = bb.order[i];
      const uint32_t gv = gid_old[v];
      uint32_t j = i;
      while (j > a && gid_old[bb.order[j - 1]] > gv) {
        bb.order[j] = bb.order[j - 1];
        --j;
      }
      bb.order[j] = v;
    }
  }
}

// Move the dynamic state and the per-slot identity into cell order.
template <typename Rec>
__global__ void __launch_bounds__(kThreads)
k_permute(const Ctl* ctl, Params p, BinBuf bb, StateBufs sb, Lists L) {
  if (!rebuilding(ctl)) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.n) return;
  const uint32_t ph = ctl->phase & 1u, lph = ctl->lphase & 1u;
  const Rec* P0 = static_cast<const Rec*>(buf_of(sb.P, ph));
  const Rec* V0 = static_cast<const Rec*>(buf_of(sb.V, ph));
  const Rec* W0 = static_cast<const Rec*>(buf_of(sb.W, ph));
  const Rec* Q0 = static_cast<const Rec*>(buf_of(sb.Q, ph));
  Rec* P1 = static_cast<Rec*>(buf_of(sb.P, ph ^ 1u));
  Rec* V1 = static_cast<Rec*>(buf_of(sb.V, ph ^ 1u));
  Rec* W1 = static_cast<Rec*>(buf_of(sb.W, ph ^ 1u));
  Rec* Q1 = static_cast<Rec*>(buf_of(sb.Q, ph ^ 1u));
  const uint32_t* gid_old = list_of(L, lph).gid;
  uint32_t* gid_new = list_of(L, lph ^ 1u).gid;
  float4* posf_new = list_of(L, lph ^ 1u).posf;
  const uint32_t s = bb.order[t];
  P1[t] = P0[s];
  V1[t] = V0[s];
  W1[t] = W0[s];
  Q1[t] = Q0[s];
  gid_new[t] = gid_old[s];
  posf_new[t] = posf_of(p, P0, s);
  D4* inv_new = list_of(L, lph ^ 1u).inv;
  if (inv_new) inv_new[t] = inverses(P0[s], V0[s]);
}

// ---- triangle cell lists -----------------------------------------------------

// Cells within reach of element k at the reference pose: its bounding box
// grown by the reach R_k + R_max + skin (+ margin), then a conservative
// per-cell test: the cell centre within reach + half the cell diagonal of the
// element.  pass 0 counts, pass 1 fills.  blockIdx.x is the element; its cells are shared by
// the gridDim.y blocks of that element.
__global__ void k_tri_cells(const Ctl* ctl, Params p, MeshDev mesh, BinBuf bb, int pass) {
  if (!rebuilding(ctl) || tcells_kept(p, bb)) return;
  const int k = blockIdx.x;
  if (k >= mesh.nt) return;
  // the reference pose (the lists are in the mesh's frame)
  const int4 tv = mesh.tri[k];
  const int nvk = tv.w >= 0 ? 4 : (tv.z >= 0 ? 3 : (tv.y >= 0 ? 2 : 1));
  const float4 A = ref_vertex(p, mesh, tv, nvk, 0), B = ref_vertex(p, mesh, tv, nvk, 1),
               C = ref_vertex(p, mesh, tv, nvk, 2), D = ref_vertex(p, mesh, tv, nvk, 3);
  const float reach = (float)mesh.rad[k] + p.rmax + p.skin + p.list_margin;
  // unused vertex slots repeat vertex 0, so the box of all four is the element's
  const float3 lo = make_float3(fminf(fminf(A.x, B.x), fminf(C.x, D.x)) - reach,
                                fminf(fminf(A.y, B.y), fminf(C.y, D.y)) - reach,
                                fminf(fminf(A.z, B.z), fminf(C.z, D.z)) - reach);
  const float3 hi = make_float3(fmaxf(fmaxf(A.x, B.x), fmaxf(C.x, D.x)) + reach,
                                fmaxf(fmaxf(A.y, B.y), fmaxf(C.y, D.y)) + reach,
                                fmaxf(fmaxf(A.z, B.z), fmaxf(C.z, D.z)) + reach);
  const int3 c0 = cell_coords(p, lo.x, lo.y, lo.z);
  const int3 c1 = cell_coords(p, hi.x, hi.y, hi.z);
  const int nx = c1.x - c0.x + 1, ny = c1.y - c0.y + 1, nz = c1.z - c0.z + 1;
  const int64_t total = (int64_t)nx * ny * nz;
  const float halfdiag = 0.5f * p.h * 1.7320508f * 1.0001f;
  const float lim = reach + halfdiag;
  const V3<float> a = mk(A.x, A.y, A.z), b = mk(B.x, B.y, B.z), c = mk(C.x, C.y, C.z),
                  dd = mk(D.x, D.y, D.z);
  for (int64_t i = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.y * blockDim.x) {
    const int cx = c0.x + (int)(i % nx);
    const int cy = c0.y + (int)((i / nx) % ny);
    const int cz = c0.z + (int)(i / ((int64_t)nx * ny));
    const V3<float> q = mk((float)p.base[0] + (cx + 0.5f) * p.h,
                           (float)p.base[1] + (cy + 0.5f) * p.h,
                           (float)p.base[2] + (cz + 0.5f) * p.h);
    // boundary cells also hold clamped particles from outside the box:
    // accept them whenever the triangle is within reach of the clamped region
    const bool edge = cx == 0 || cy == 0 || cz == 0 || cx == p.nc[0] - 1 ||
                      cy == p.nc[1] - 1 || cz == p.nc[2] - 1;
    bool hit = edge;
    if (!hit) {
      const V3<float> y = closest_point_element(q, a, b, c, dd, nvk);
      const V3<float> d = q - y;
      hit = dot(d, d) <= lim * lim;
    }
    if (!hit) continue;
    const uint32_t cell = cell_index(p, make_int3(cx, cy, cz));
    if (pass == 0) {
      atomicAdd(&bb.tcell_count[cell], 1u);
    } else {
      const uint32_t pos = bb.tcell_start[cell] + atomicAdd(&bb.tcell_count[cell], 1u);
      if (pos < bb.tcap) bb.tcell_tri[pos] = (uint32_t)k;
    }
  }
}

__global__ void k_tri_cells_check(Ctl* ctl, Params p, BinBuf bb) {
  if (!rebuilding(ctl)) return;
  if (bb.tcell_start[p.ncells] > bb.tcap) {
    *bb.tcell_overflow = bb.tcell_start[p.ncells];
    set_status(ctl, DEM_ERR_CAPACITY);
  }
}

// Order each cell's element list by element index.  One warp per cell: every
// lane ranks its elements against the whole list (indices in a cell are
// distinct, so ranks are a permutation) and writes them to their ranks; a few
// cells (around fan centres) hold a hundred elements or more, which a serial
// insertion sort per cell would make the slowest step of the rebuild.
constexpr int kSortWarps = 8;
constexpr int kSortMax = 512;  // longer lists (not met in practice) sort serially

__global__ void __launch_bounds__(32 * kSortWarps)
k_tri_cell_sort(const Ctl* ctl, Params p, BinBuf bb) {
  __shared__ uint32_t buf_s[kSortWarps][kSortMax];
  if (!rebuilding(ctl) || tcells_kept(p, bb)) return;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint32_t* buf = buf_s[wib];
  const int64_t nw = (int64_t)gridDim.x * kSortWarps;
  for (int64_t c = (int64_t)blockIdx.x * kSortWarps + wib; c < p.ncells; c += nw) {
    const uint32_t a = bb.tcell_start[c], b = min(bb.tcell_start[c + 1], bb.tcap);
    if (b <= a + 1) continue;
    const uint32_t m = b - a;
    if (m > (uint32_t)kSortMax) {
      if (lane == 0)
        for (uint32_t i = a + 1; i < b; ++i) {
          const uint32_t v = bb.tcell_tri[i];
          uint32_t j = i;
          while (j > a && bb.tcell_tri[j - 1] > v) {
            bb.tcell_tri[j] = bb.tcell_tri[j - 1];
            --j;
          }
          bb.tcell_tri[j] = v;
        }
      __syncwarp();
      continue;
    }
    for (uint32_t i = lane; i < m; i += 32) buf[i] = bb.tcell_tri[a + i];
    __syncwarp();
    for (uint32_t i = lane; i < m; i += 32) {
      const uint32_t v = buf[i];
      uint32_t r = 0;
      for (uint32_t j = 0; j < m; ++j) r += buf[j] < v ? 1u : 0u;
      bb.tcell_tri[a + r] = v;
    }
    __syncwarp();
  }
}

// ---- Verlet list build + history remap -----------------------------------------

// History records are never cleared: a record counts only if its stamp is
// the current step, and a record left in a list buffer from an earlier list
// generation carries a stamp of at most the step that generation ended in,
// which is before the current one.  The buffers start filled with kStampNone
// (at creation and at a load).

// For one new slot t: collect the partners within R_t + R_u + skin (float test
// with a conservative margin) from the 27 surrounding cells, sorted by caller
// index, into the temporary fixed-capacity list, and the triangle candidates
// of the particle's cell into its triangle list, carrying each triangle
// contact's history over from the particle's previous list.  The pair list is
// packed into CSR form by k_list_compact once the counts are scanned.
//
// One thread per slot; the candidate positions come through L1 (a block's
// slots are neighbours in cell order, so they read the same cells).  Staging
// the neighbour rows of a block in shared memory first was measured slower
// (the threads of a block that spans two rows of cells wait for each other).
constexpr int kBuildThreads = 128;

template <typename Hist>
__global__ void __launch_bounds__(kBuildThreads)
k_list_build(Ctl* ctl, Params p, BinBuf bb, Lists L, MeshDev mesh) {
  if (!rebuilding(ctl)) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = p.n;
  if (t >= n) return;
  const ListBuf lo = list_of(L, ctl->lphase & 1u);
  const ListBuf ln = list_of(L, (ctl->lphase & 1u) ^ 1u);
  const float4 X = ln.posf[t];
  if (X.w == 0.f) {  // inactive: no list, no mesh candidates
    bb.tmp_cnt[t] = 0u;
    ln.meta[t] = 0u;
    return;
  }
  const int3 c = cell_coords(p, X.x, X.y, X.z);
  const uint32_t gt = ln.gid[t];
  uint32_t cand_g[64];
  uint32_t cand_s[64];
  const int cap = min(p.cap, 64);
  int cnt = 0;
  bool overflow = false;
  // the cells of a row along x are consecutive in the grid, so the three
  // cells x-1 .. x+1 of a neighbour row are one range of slots: 9 ranges
  const int x0 = max(c.x - 1, 0), x1 = min(c.x + 1, p.nc[0] - 1);
  for (int dz = -1; dz <= 1; ++dz) {
    const int cz = c.z + dz;
    if (cz < 0 || cz >= p.nc[2]) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int cy = c.y + dy;
      if (cy < 0 || cy >= p.nc[1]) continue;
      const uint32_t a = bb.cell_start[cell_index(p, make_int3(x0, cy, cz))];
      const uint32_t b = bb.cell_start[cell_index(p, make_int3(x1, cy, cz)) + 1];
      for (uint32_t u = a; u < b; ++u) {
        if (u == (uint32_t)t) continue;
        const float4 Y = ln.posf[u];
        const float ddx = X.x - Y.x, ddy = X.y - Y.y, ddz = X.z - Y.z;
        const float cut = X.w + Y.w + p.skin + p.list_margin;
        if (ddx * ddx + ddy * ddy + ddz * ddz < cut * cut) {
          if (cnt < cap) {
            const uint32_t g = ln.gid[u];
            int j = cnt;
            while (j > 0 && cand_g[j - 1] > g) {
              cand_g[j] = cand_g[j - 1];
              cand_s[j] = cand_s[j - 1];
              --j;
            }
            cand_g[j] = g;
            cand_s[j] = u;
            ++cnt;
          } else {
            overflow = true;
          }
        }
      }
    }
  }
  if (overflow) set_status(ctl, DEM_ERR_CAPACITY);
  int nlow = 0;
  while (nlow < cnt && cand_g[nlow] < gt) ++nlow;
  // the pair history to carry over: both this list and the particle's
  // previous one are sorted by partner caller index, so one merge walk finds
  // each partner's old entry (with one evaluation per pair only the entries
  // of partners with a higher caller index hold records); k_list_compact
  // keeps the record only if the contact touched in the previous step
  const uint32_t s = bb.order[t];
  const uint32_t mo = lo.meta[s];
  const int nn_o = (int)(mo & 0xffu);
  const uint32_t off_o = lo.offs[s];
  const uint32_t stamp_now = (uint32_t)ctl->step;  // records written in the previous step
  const int khist = p.pair_res ? nlow : 0;
  int io = 0;
  for (int k = 0; k < cnt; ++k) {
    const uint32_t g = cand_g[k];
    uint32_t src = kNoHist;
    if (k >= khist) {
      while (io < nn_o && lo.ngid[off_o + io] < g) ++io;
      if (io < nn_o && lo.ngid[off_o + io] == g) src = off_o + (uint32_t)io;
    }
    bb.tmp_nbr[(size_t)k * n + t] = cand_s[k];
    bb.tmp_gid[(size_t)k * n + t] = g;
    bb.tmp_hsrc[(size_t)k * n + t] = src;
  }
  bb.tmp_cnt[t] = (uint32_t)cnt;

  // triangle candidates (fixed capacity per particle), history carried over
  const int nt_o = (int)((mo >> 16) & 0xffu);
  int ntc = 0;
  if (mesh.nt > 0) {
    // the element list of the particle's cell in the mesh's frame
    int3 cm = c;
    if (p.omega_norm > 0.0) {
      const V3<float> qm = to_mesh_frame(p, mk(X.x, X.y, X.z), (float)ctl->rot_c,
                                         (float)ctl->rot_s);
      cm = cell_coords(p, qm.x, qm.y, qm.z);
    }
    const uint32_t cell = cell_index(p, cm);
    const uint32_t a = bb.tcell_start[cell], b = min(bb.tcell_start[cell + 1], bb.tcap);
    const Hist* hpm_o = static_cast<const Hist*>(lo.hpm);
    Hist* hpm_n = static_cast<Hist*>(ln.hpm);
    int ko2 = 0;
    const V3<float> q = mk(X.x, X.y, X.z);
    bool tover = false;
    for (uint32_t i = a; i < b; ++i) {
      const uint32_t k = bb.tcell_tri[i];
      const float4 A = mesh.curf[4 * k], B = mesh.curf[4 * k + 1], C = mesh.curf[4 * k + 2],
                   D = mesh.curf[4 * k + 3];
      const V3<float> y = closest_point_element(q, mk(A.x, A.y, A.z), mk(B.x, B.y, B.z),
                                                mk(C.x, C.y, C.z), mk(D.x, D.y, D.z), (int)A.w);
      const V3<float> d = q - y;
      const float cut = X.w + (float)mesh.rad[k] + p.skin + p.list_margin;
      if (dot(d, d) >= cut * cut) continue;
      if (ntc >= p.capm) {
        tover = true;
        continue;
      }
      ln.tric[(size_t)ntc * n + t] = k;
      while (ko2 < nt_o && lo.tric[(size_t)ko2 * n + s] < k) ++ko2;
      if (ko2 < nt_o && lo.tric[(size_t)ko2 * n + s] == k) {
        const Hist h = hpm_o[(size_t)ko2 * n + s];
        if (h.stamp == stamp_now) hpm_n[(size_t)ntc * n + t] = h;
      }
      ++ntc;
    }
    if (tover) set_status(ctl, DEM_ERR_CAPACITY);
  }
  ln.meta[t] = (uint32_t)cnt | ((uint32_t)nlow << 8) | ((uint32_t)ntc << 16);
  atomicAdd(&ctl->list_entries, (uint32_t)cnt);
  atomicAdd(&ctl->mesh_candidates, (uint32_t)ntc);
  atomicMax(&ctl->max_list_len, (uint32_t)cnt);
}

// Pack the new pair lists into CSR form (offsets from the scan of the counts)
// and copy each pair's friction history record from the previous list where
// k_list_build found one and the contact touched in the previous step.  A
// warp covers the entries of 32 consecutive slots, 32 entries at a time (all
// lanes busy, consecutive entries written by consecutive lanes).
constexpr int kCompactWarps = 4;

__device__ __forceinline__ uint32_t warp_scan_incl(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

template <typename Hist>
__global__ void __launch_bounds__(32 * kCompactWarps)
k_list_compact(Ctl* ctl, Params p, BinBuf bb, Lists L) {
  __shared__ uint32_t seg_s[kCompactWarps][33];
  if (!rebuilding(ctl)) return;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int n = p.n;
  const int w0 = (blockIdx.x * kCompactWarps + wib) * 32;
  if (w0 > n) return;  // the whole warp (no divergence at the shuffles below)
  const int t = w0 + lane;
  const ListBuf lo = list_of(L, ctl->lphase & 1u);
  const ListBuf ln = list_of(L, (ctl->lphase & 1u) ^ 1u);
  uint32_t* seg = seg_s[wib];
  uint32_t cnt = 0;
  if (t <= n) ln.offs[t] = bb.tmp_offs[t];
  if (t < n) cnt = bb.tmp_cnt[t];
  const uint32_t incl = warp_scan_incl(cnt);
  seg[lane + 1] = incl;
  if (lane == 0) seg[0] = 0;
  const uint32_t E = __shfl_sync(full, incl, 31);
  const uint32_t base = bb.tmp_offs[w0 < n ? w0 : n];  // first entry of slot w0
  __syncwarp();
  const Hist* hpp_o = static_cast<const Hist*>(lo.hpp);
  Hist* hpp_n = static_cast<Hist*>(ln.hpp);
  const uint32_t stamp_now = (uint32_t)ctl->step;  // records written in the previous step
  for (uint32_t e0 = 0; e0 < E; e0 += 32) {
    const uint32_t e = e0 + lane;
    if (e >= E) break;
    // the slot owning entry e: largest tl with seg[tl] <= e
    int tl = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1)
      if (seg[tl + step] <= e) tl += step;
    const uint32_t k = e - seg[tl];
    const size_t src = (size_t)k * n + (size_t)(w0 + tl);
    ln.nbr[base + e] = bb.tmp_nbr[src];
    ln.ngid[base + e] = bb.tmp_gid[src];
    const uint32_t hs = bb.tmp_hsrc[src];
    if (hs != kNoHist) {
      const Hist h = hpp_o[hs];
      if (h.stamp == stamp_now) hpp_n[base + e] = h;
    }
  }
}

__global__ void k_rebuild_prep(Ctl* ctl, Params p) {
  if (!rebuilding(ctl)) return;
  if (p.omega_norm > 0.0) {  // the rotation of this step, for the mesh-frame lookups
    const double th = p.omega_norm * ((double)ctl->step * p.dt);
    ctl->rot_c = cos(th);
    ctl->rot_s = sin(th);
  }
  ctl->list_entries = 0;
  ctl->mesh_candidates = 0;
  ctl->max_list_len = 0;
}

__global__ void k_rebuild_end(Ctl* ctl, Params p, BinBuf bb, int nt) {
  if (!rebuilding(ctl)) return;
  if (nt > 0) bb.tcell_overflow[1] = 1u;  // element lists kept
  ctl->phase ^= 1u;
  ctl->lphase ^= 1u;
  ctl->rebuilds += 1;
  ctl->mesh_angle_ref = p.omega_norm * ((double)ctl->step * p.dt);
}

inline unsigned blocks_for(int64_t n, int threads) {
  return (unsigned)((n + threads - 1) / threads);
}

}  // namespace

// For every entry whose partner u has the lower caller index, the index of
// u's entry for the same pair: u's list is sorted by partner caller index, so
// a binary search over its upper entries finds this particle.  That entry of
// u gets, in return, this entry's index k in this particle's list.
__global__ void __launch_bounds__(128)
k_mirror(Ctl* ctl, Params p, Lists L) {
  if (!rebuilding(ctl)) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.n) return;
  const ListBuf ln = list_of(L, (ctl->lphase & 1u) ^ 1u);
  const uint32_t meta = ln.meta[t];
  const uint32_t nlow = (meta >> 8) & 0xffu;
  const uint32_t off = ln.offs[t];
  const uint32_t gt = ln.gid[t];
  for (uint32_t k = 0; k < nlow; ++k) {
    const uint32_t u = ln.nbr[off + k];
    const uint32_t mu = ln.meta[u];
    uint32_t lo = ln.offs[u] + ((mu >> 8) & 0xffu), hi = ln.offs[u] + (mu & 0xffu);
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (ln.gid[ln.nbr[mid]] < gt) lo = mid + 1;
      else hi = mid;
    }
    ln.mir[off + k] = lo;
    ln.back[lo] = (uint8_t)k;
  }
}

void launch_rebuild(cudaStream_t st, Ctl* ctl, const Params& p, StateBufs sb, Lists L,
                    BinBuf bb, MeshDev mesh) {
  const unsigned nb = blocks_for(p.n, kThreads);
  const unsigned gcells = (unsigned)std::min<int64_t>(blocks_for(p.ncells, kThreads), 152 * 16);
  k_rebuild_prep<<<1, 1, 0, st>>>(ctl, p);
  k_clear<<<gcells, kThreads, 0, st>>>(ctl, bb.cell_count, p.ncells + 1);
  k_bin_count<<<nb, kThreads, 0, st>>>(ctl, p, sb, bb, L);
  launch_scan(st, ctl, bb.cell_count, bb.cell_start, p.ncells + 1, bb.block_sums);
  k_scatter<<<nb, kThreads, 0, st>>>(ctl, p, bb);
  k_cell_sort<<<gcells, kThreads, 0, st>>>(ctl, p, bb, L);
  if (p.mixed)
    k_permute<F8><<<nb, kThreads, 0, st>>>(ctl, p, bb, sb, L);
  else
    k_permute<D4><<<nb, kThreads, 0, st>>>(ctl, p, bb, sb, L);
  if (mesh.nt > 0) {
    k_clear_tcells<<<gcells, kThreads, 0, st>>>(ctl, p, bb);
    k_tri_cells<<<dim3((unsigned)mesh.nt, (unsigned)p.tri_chunks), 128, 0, st>>>(ctl, p, mesh, bb, 0);
    launch_scan(st, ctl, bb.tcell_count, bb.tcell_start, p.ncells, bb.block_sums);
    k_tri_cells_check<<<1, 1, 0, st>>>(ctl, p, bb);
    k_clear_tcells<<<gcells, kThreads, 0, st>>>(ctl, p, bb);
    k_tri_cells<<<dim3((unsigned)mesh.nt, (unsigned)p.tri_chunks), 128, 0, st>>>(ctl, p, mesh, bb, 1);
    k_tri_cell_sort<<<152 * 8, 32 * kSortWarps, 0, st>>>(ctl, p, bb);
  }
  const unsigned nb128 = blocks_for(p.n, 128);
  const unsigned nbl = blocks_for(p.n, kBuildThreads);
  const unsigned nbc = blocks_for((int64_t)p.n + 1, 32 * kCompactWarps);
  if (p.hist32)
    k_list_build<HistM><<<nbl, kBuildThreads, 0, st>>>(ctl, p, bb, L, mesh);
  else
    k_list_build<HistD><<<nbl, kBuildThreads, 0, st>>>(ctl, p, bb, L, mesh);
  launch_scan(st, ctl, bb.tmp_cnt, bb.tmp_offs, p.n, bb.block_sums);
  if (p.hist32)
    k_list_compact<HistM><<<nbc, 32 * kCompactWarps, 0, st>>>(ctl, p, bb, L);
  else
    k_list_compact<HistD><<<nbc, 32 * kCompactWarps, 0, st>>>(ctl, p, bb, L);
  if (p.pair_res) k_mirror<<<nb128, 128, 0, st>>>(ctl, p, L);
  k_rebuild_end<<<1, 1, 0, st>>>(ctl, p, bb, mesh.nt);
}

}  // namespace dem
