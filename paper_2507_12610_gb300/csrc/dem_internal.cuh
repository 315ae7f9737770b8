// Internal types shared by the libdem translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dem.h"

namespace dem {

// 32-byte aligned record of four doubles (one DRAM sector per load).
using D4 = double4_32a;
__host__ __device__ __forceinline__ D4 make_D4(double x, double y, double z, double w) {
  return make_double4_32a(x, y, z, w);
}

// ---------------------------------------------------------------------------
// Device control block: one per scene, in device memory.  All per-step
// decisions (rebuild or not, which buffer is current) live here so a step is
// a fixed kernel sequence that can be captured in a CUDA graph.
struct Ctl {
  uint32_t status;      // sticky error code (DEM_OK = 0)
  uint32_t phase;       // index of the current dynamic-state buffer (0/1)
  uint32_t lphase;      // index of the current list/history buffer (0/1)
  uint32_t rebuild;     // 1 while the current step rebuilds the lists
  uint32_t disp_flag;   // set by the step kernel: some particle moved > skin/2
  uint32_t force_rebuild;
  int64_t step;         // steps completed
  int64_t rebuilds;
  double mesh_angle_ref;  // mesh rotation angle at the last rebuild
  double rot_c, rot_s;    // cos / sin of the mesh rotation angle of the current step
  uint32_t pair_contacts;  // touching directed pair entries, this step (accumulating)
  uint32_t mesh_contacts;
  uint32_t pair_contacts_last;  // ... of the last completed step
  uint32_t mesh_contacts_last;
  uint32_t list_entries;     // directed candidate entries of the current list
  uint32_t mesh_candidates;
  uint32_t max_list_len;
  uint32_t n_active;     // particles in the dynamics: caller indices 0 .. n_active-1
  double spawn_carry;    // radius carried over from a failed spawn attempt (< 0: none)
  uint64_t spawn_draws;  // uniforms of the spawn stream drawn so far
};

// Parameters the kernels need, passed by value.
struct Params {
  // material / contact constants (double and float copies)
  double E, nu, rho, e_n, mu_s, mu_r, mu_t, eta, dt;
  double g[3];
  double beta;           // damping factor of e_n (Sec. 2.2)
  double Es_pp, Gs_pp;   // effective moduli particle-particle (same material)
  double Es_pw, Gs_pw;   // particle-wall limits
  double cs_cn_pp, cs_cn_pw;  // c_s / c_n of a pair and of a wall contact
  double mesh_omega[3], mesh_center[3];
  double omega_norm;     // |mesh_omega|
  double mesh_rmax;      // largest vertex distance from the rotation axis
  // binning
  double origin[3];      // shifted coordinates X = x - origin
  double base[3];        // power-of-two offset: domain_lo - origin
  float inv_h;           // 1 / cell edge
  float h;
  int32_t nc[3];         // cells per axis
  int64_t ncells;
  float skin;
  float half_skin_trigger;  // skin/2 minus the float margin
  float list_margin;        // conservative float margin of candidate tests
  float rmax;               // largest particle radius
  float mesh_prefilter;     // float margin before the FP64 triangle geometry (mixed)
  // FP32 copies of the constants for DEM_MIXED (no FP64 conversion in the hot loop)
  float f_Es_pp, f_Gs_pp, f_Es_pw, f_Gs_pw, f_beta, f_mu_s, f_mu_r, f_mu_t, f_dt;
  float f_cs_cn_pp, f_cs_cn_pw;
  float f_g[3], f_omega[3];
  float f_drag;             // 9 eta / (2 rho): Stokes rate c = f_drag / R^2
  float center_hi[3], center_lo[3];  // mesh_center - origin as hi/lo floats
  int32_t n;
  int32_t cap;              // pair-list capacity per particle
  int32_t capm;             // triangle-candidate capacity per particle
  int32_t tri_chunks;       // blocks per element in the element-cell binning
  int32_t n_tri;
  int32_t record_forces;
  int32_t mixed;            // DEM_MIXED: compensated FP32 state records (F8)
  int32_t mixed64;          // DEM_MIXED64: FP64 state records, FP32 contact law
  int32_t hist32;           // friction springs in FP32 (DEM_MIXED, DEM_MIXED64)
  // spawning (n above is the capacity; see Ctl::n_active)
  double sp_lo[3], sp_hi[3];
  double sp_rmin, sp_rmax;
  double sp_v0[3], sp_w0[3];
  uint64_t sp_seed;
  int32_t sp_attempts;      // 0: spawning off
  int32_t sp_every;
  // friction per material (n_mat = 0: the coefficients above); the material
  // index of a particle is in its W record (mixed: lo.w as int bits; FP64: w)
  int32_t step_warps;       // warps per block of the step kernel (4 or 8)
  // DEM_FP64 one-evaluation-per-pair scheme (NULL: both sides evaluate)
  void* pair_res;           // [list capacity] per-entry pair results (DEM_FP64: one
                            // evaluation per pair)
  unsigned long long* pair_touch;  // [n] bit k: list entry k touched in this step
  int32_t n_mat;
  const float4* mat_f;      // [n_mat] mu_s, mu_r, mu_t, 0
  const D4* mat_d;          // [n_mat] mu_s, mu_r, mu_t, 0
};

constexpr int kSpawnMaxAttempts = 1024;

// Dynamic state, double precision: four 32-byte records per particle.
struct StateD {
  D4* P;  // x, y, z (absolute), R
  D4* V;  // v, m
  D4* W;  // w, unused
  D4* Q;  // q0..q3
};

// Dynamic state, compensated single precision (hi + lo pairs).
struct __align__(32) F8 {
  float4 hi, lo;
};
struct StateM {
  F8* P;  // X - origin (shifted, hi/lo), R (hi/lo)
  F8* V;  // v (hi/lo); hi.w = m, lo.w = 1/m
  F8* W;  // w (hi/lo); hi.w = 1/R
  F8* Q;  // q (hi/lo)
};

// Friction history of one contact, in the precision of the contact math.
// stamp = 1 + index of the step that last wrote it; a record is carried into
// step s only if stamp == s, i.e. the contact was touching in step s - 1.
// 32-byte alignment lets a record move as whole 256-bit loads and stores
// instead of one access per field (measured: the mixed step kernel 13 %
// faster, bitwise the same results).
struct __align__(32) HistD {
  double us[3];
  double ur[3];
  double ut;
  uint32_t stamp;
  uint32_t pad;
};
struct __align__(32) HistM {
  float us[3];
  float ur[3];
  float ut;
  uint32_t stamp;
};
static_assert(sizeof(HistD) == 64, "HistD must be 64 bytes");
static_assert(sizeof(HistM) == 32, "HistM must be 32 bytes");

constexpr uint32_t kStampNone = 0xffffffffu;

// Lists and per-slot data valid between two rebuilds (double-buffered by lphase).
struct ListBuf {
  uint32_t* gid;    // [n] caller index of the particle in each slot
  float4* posf;     // [n] shifted position (float) and radius at the rebuild
  uint32_t* meta;   // [n] list length | lower-id count << 8 | triangle count << 16
  uint32_t* offs;   // [n + 1] CSR offsets of the pair entries (slot order)
  uint32_t* nbr;    // [offs[n]] partner slots, ascending partner caller index per particle
  uint32_t* ngid;   // [offs[n]] partner caller indices (the keys of the history remap)
  void* hpp;        // [offs[n]] pair history (HistD or HistM), one record per entry
  uint32_t* tric;   // [capm][n] candidate triangles, ascending
  void* hpm;        // [capm][n] triangle history
  uint32_t* mir;    // [offs[n]] for an entry whose partner has the lower caller index,
                    // the partner's entry for the same pair (one evaluation per pair)
  uint8_t* back;    // [offs[n]] for an entry whose partner has the higher caller index,
                    // the index of this particle in the partner's list
  D4* inv;          // [n] DEM_FP64 only (else null): 1/R, 1/m, 1/I of the particle in
                    // each slot, the divisions of the law done once per rebuild
};

// Per-particle data a policy's contact law reads beside the state records
// (DEM_FP64: the inverses of ListBuf::inv; the other policies: nothing).
struct NoAux {};

// Mesh elements (Sec. 3.3): triangles first, then points, segments and
// rectangles; four vertex slots per element, unused slots repeat vertex 0.
// The pose arrays (cur, curf, curl, plane) hold the pose of an even step, the
// *_odd arrays that of an odd step: the pose of step n + 1 is computed while
// step n runs (it depends on the step number only).  The host passes each
// kernel the view of its step (mesh_at), so kernels index no buffer by the
// step at run time.
struct MeshDev {
  D4* ref;           // [nv] reference vertices (x, y, z, 0)
  int4* tri;         // [nt] vertex indices, -1 for unused slots
  double* rad;       // [nt] element radius
  D4* cur;           // [nt][4] current vertices (absolute); .w of slot 0 = radius
  float4* curf;      // [nt][4] current vertices, shifted (float); .w of slot 0 = vertex count
  float4* curl;      // [nt][4] low words of the shifted vertices (curf + curl = shifted
                     // vertex to ~1e-15); .w of slots 0, 1 = radius (hi, lo)
  float4* plane;     // [nt][2] face plane n.X = c in shifted coordinates, unit n:
                     // (n hi, c hi), (n lo, c lo); zero for points and segments
  D4* nref;          // [nt] unit normal of the face at the reference pose (zero for
                     // points, segments and degenerate faces)
  D4* cur_odd;       // the four pose arrays above, for odd steps
  float4* curf_odd;
  float4* curl_odd;
  float4* plane_odd;
  int32_t nv, nt;
};

constexpr uint32_t kNoHist = 0xffffffffu;  // no history record to carry over

// Binning scratch.
struct BinBuf {
  uint32_t* key;        // [n] cell of each slot (current order)
  uint32_t* local;      // [n] arrival index within its cell
  uint32_t* cell_count; // [ncells]
  uint32_t* cell_start; // [ncells + 1]
  uint32_t* order;      // [n] old slot of each new slot
  uint32_t* block_sums; // scan partials
  uint32_t* tmp_nbr;    // [cap][n] candidates of the list being built (slot order)
  uint32_t* tmp_gid;    // [cap][n] their caller indices
  uint32_t* tmp_hsrc;   // [cap][n] index of the entry's history record in the
                        //   previous list, or kNoHist
  uint32_t* tmp_cnt;    // [n] their counts
  uint32_t* tmp_offs;   // [n + 1] exclusive prefix of the counts
  // triangle cell lists
  uint32_t* tcell_count;  // [ncells]
  uint32_t* tcell_start;  // [ncells + 1]
  uint32_t* tcell_tri;    // [tcap]
  uint32_t tcap;
  uint32_t* tcell_overflow;
};

// Both parities of the double-buffered data.  Kernels pick the current one
// from the control block (ctl->phase for the dynamic state, ctl->lphase for
// lists and histories), so the launch sequence never depends on host state.
// Record type: D4 (DEM_FP64) or F8 (DEM_MIXED).
struct StateBufs {
  void* P[2];
  void* V[2];
  void* W[2];
  void* Q[2];
};
struct Lists {
  ListBuf b[2];
};

// Buffer b (0 or 1) of a double-buffered kernel parameter.  Device code must
// use these instead of indexing the arrays with a run-time value: indexing a
// parameter array that way makes every thread copy the whole parameter to
// local memory first, while a select of two fields keeps it in the constant
// bank.
#ifdef __CUDACC__
__device__ __forceinline__ void* buf_of(void* const (&a)[2], uint32_t b) {
  return b ? a[1] : a[0];
}
size_t pair_result_bytes();  // bytes of one entry's DEM_FP64 pair result

// The mesh with the pose arrays of step `step` (even or odd buffers).
inline MeshDev mesh_at(const MeshDev& m, int64_t step) {
  MeshDev r = m;
  if (step & 1) {
    r.cur = m.cur_odd;
    r.curf = m.curf_odd;
    r.curl = m.curl_odd;
    r.plane = m.plane_odd;
  }
  return r;
}

__device__ __forceinline__ ListBuf list_of(const Lists& L, uint32_t b) {
  ListBuf r;
  r.gid = b ? L.b[1].gid : L.b[0].gid;
  r.posf = b ? L.b[1].posf : L.b[0].posf;
  r.meta = b ? L.b[1].meta : L.b[0].meta;
  r.offs = b ? L.b[1].offs : L.b[0].offs;
  r.nbr = b ? L.b[1].nbr : L.b[0].nbr;
  r.ngid = b ? L.b[1].ngid : L.b[0].ngid;
  r.hpp = b ? L.b[1].hpp : L.b[0].hpp;
  r.tric = b ? L.b[1].tric : L.b[0].tric;
  r.hpm = b ? L.b[1].hpm : L.b[0].hpm;
  r.mir = b ? L.b[1].mir : L.b[0].mir;
  r.back = b ? L.b[1].back : L.b[0].back;
  r.inv = b ? L.b[1].inv : L.b[0].inv;
  return r;
}
#endif

// Kernel launch helpers implemented in the .cu files.
void launch_spawn(cudaStream_t st, Ctl* ctl, const Params& p, StateBufs sb, BinBuf bb,
                  MeshDev mesh);
// The pose of step ctl->step + ahead (ahead 0 or 1) into the pose arrays of
// `mesh` (the view of that step).
void launch_mesh_pose(cudaStream_t st, const Ctl* ctl, const Params& p, MeshDev mesh, int ahead);
void launch_rebuild(cudaStream_t st, Ctl* ctl, const Params& p, StateBufs sb, Lists L,
                    BinBuf bb, MeshDev mesh);
void launch_step(cudaStream_t st, Ctl* ctl, const Params& p, StateBufs sb, Lists L,
                 MeshDev mesh, double* forces);
void launch_advance(cudaStream_t st, Ctl* ctl, const Params& p);
// The current state in caller order as doubles: x[n][3], v[n][3], w[n][3],
// q[n][4] one after another in `out` (13 n doubles, device memory).
void launch_export_state(cudaStream_t st, const Ctl* ctl, const Params& p, StateBufs sb,
                         Lists L, int64_t n, double* out);
// Sets ctl->rot_c / rot_s for the step in the control block.
void launch_set_pose(cudaStream_t st, Ctl* ctl, const Params& p);
// Sets a graph IF-condition from ctl->rebuild (inside a captured graph).
void launch_decide(cudaStream_t st, const Ctl* ctl, cudaGraphConditionalHandle h);

// Scan of a u32 array (exclusive) on the device; early-exits unless ctl->rebuild.
void launch_scan(cudaStream_t st, const Ctl* ctl, const uint32_t* in, uint32_t* out, int64_t n,
                 uint32_t* block_sums);
int64_t scan_block_sums_size(int64_t n);

}  // namespace dem
