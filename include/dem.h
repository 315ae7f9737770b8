/*
 * dem.h -- C ABI of the GB300 soft-sphere DEM timestep library (libdem.so).
 *
 * The library advances a 3D ensemble of frictional spheres and a rigid mesh
 * (triangles, rectangles, segments, points) with the method of arXiv
 * 2507.12610 ("TinyDEM"):
 *   - damped Newton-Euler equations of motion with Stokes drag (Sec. 2.1,
 *     Eqs. translation / rotation),
 *   - the visco-elastic Hertz-Mindlin contact law with Coulomb-limited
 *     sliding, rolling and twisting springs whose history persists for the
 *     life of a contact (Sec. 2.2, Eqs. fn, fs, fr, ft, Coulombs/r/t; Sec. 2.3,
 *     Eqs. um, um_static, fm_kinetic, um_kinetic),
 *   - sphere-mesh element contacts with the wall limits R_j = E_j = m_j = inf
 *     (Sec. 2.2) and one independent contact per touching element (Sec. 3.3),
 *   - semi-implicit Euler integration with the synchronous SPIRAL quaternion
 *     update (Sec. 2.3, Eqs. v, x, w, spiral).
 * Contact search uses cell binning and a Verlet list with skin, the extension
 * suggested in Sec. 7; results do not depend on the skin or rebuild schedule.
 *
 * Conventions for every entry point:
 *   - Host arrays are borrowed for the duration of the call only; the
 *     library owns all device memory it allocates.
 *   - Vectors are row-major [n][3] doubles; quaternions [n][4] doubles with
 *     the scalar part first.  State is always exchanged in the caller's
 *     particle order (index 0..n-1), whatever order the device uses.
 *   - Every call returns a status code (DEM_OK = 0) and never throws.  Device
 *     errors are sticky: once a step fails, later steps do no work and
 *     dem_synchronize() reports the first error.
 *   - A scene is bound to the CUDA device current at creation and to one
 *     stream; calls on one scene must not run concurrently.
 */
#ifndef DEM_H_
#define DEM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define DEM_OK 0
#define DEM_ERR_INVALID 1   /* argument violates the requirements of Table 2 or the layout */
#define DEM_ERR_CAPACITY 2  /* a neighbour or mesh-contact list overflowed its capacity */
#define DEM_ERR_NONFINITE 3 /* a particle state became NaN or infinite */
#define DEM_ERR_TIMEOUT 4   /* reserved for a bounded device wait that gives up; no
                               kernel of this library waits on another (kernel
                               boundaries order the phases), so none returns it */
#define DEM_ERR_CUDA 5      /* a CUDA runtime call failed */
#define DEM_ERR_NOMEM 6     /* device memory allocation failed */

/* precision of the contact arithmetic */
#define DEM_FP64 0  /* everything in IEEE double precision */
#define DEM_MIXED 1 /* contact geometry, forces and springs in FP32; positions,
                       velocities, spins and orientations integrated as
                       compensated double-float pairs (two FP32 words, ~48-bit
                       significand); forces summed with compensated FP32 */
#define DEM_MIXED64 2 /* contact forces, torques and friction springs in FP32
                         (the overlap and the pair offset formed in FP64, then
                         rounded); positions, velocities, spins and
                         orientations stored and accumulated in FP64 */

/* Material, kinetic and numerical parameters.  Physical parameters follow
 * Table 2 of the paper and must satisfy its "Requirements" column:
 * E > 0, nu in (-1, 0.5], rho > 0, e_n in [0, 1], mu_* >= 0, eta >= 0, dt > 0. */
typedef struct dem_params {
  double E;        /* Young's modulus (Pa) */
  double nu;       /* Poisson's ratio */
  double rho;      /* mass density (kg/m^3), shared by all particles */
  double e_n;      /* coefficient of normal restitution */
  double mu_s;     /* sliding friction coefficient */
  double mu_r;     /* rolling friction coefficient */
  double mu_t;     /* twisting friction coefficient */
  double eta;      /* dynamic viscosity of the Stokes drag (Pa s) */
  double g[3];     /* external acceleration (m/s^2) */
  double dt;       /* time step (s) */
  double mesh_omega[3];  /* angular velocity of the rigid mesh (rad/s); the mesh
                            is the reference mesh rotated by |omega| t about the
                            axis through mesh_center (extension: the paper's
                            walls are static) */
  double mesh_center[3]; /* point on the rotation axis (m) */
  double skin;           /* Verlet skin (m); <= 0 selects 0.25 R_max */
  double domain_lo[3];   /* binning box (m); if any lo >= hi the box is the */
  double domain_hi[3];   /*   bounding box of particles and mesh, padded     */
  int32_t precision;     /* DEM_FP64, DEM_MIXED or DEM_MIXED64 */
  int32_t max_neighbors; /* list capacity per particle; <= 0 selects 64 */
  int32_t max_mesh_contacts; /* mesh-element candidate capacity per particle; <= 0: 16 */
  int32_t record_forces; /* nonzero: keep per-particle contact sums for dem_read_forces */
  /* Particle spawning (Sec. 3.1, "Particle generation"), off while
   * spawn_attempts == 0.  The scene holds n_cap = max(n, n_max) particle rows;
   * rows n .. n_cap-1 are inactive (radius 0, no contacts, not integrated)
   * until spawned, in increasing row order.  Every spawn_every steps, before
   * the forces of that step, spawn_attempts attempts run in sequence: a radius
   * uniform in [spawn_r_min, spawn_r_max] (or the radius carried over from the
   * last failed attempt), a centre uniform in the box [spawn_lo, spawn_hi]
   * (x, y, z in that order); the sphere is kept unless it overlaps a particle
   * (|x - x_j| < r + R_j) or a mesh element (distance < r + R_j), with
   * velocity spawn_v0, angular velocity spawn_w0 and the identity
   * orientation.  The k-th uniform of a run is the top 53 bits of SplitMix64
   * (Steele, Lea & Flood 2014) at seed + (k + 1) * 0x9E3779B97F4A7C15.  The
   * paper makes its attempts every step; spawn_every > 1 batches them (each
   * event that keeps a particle costs a list rebuild). */
  int64_t n_max;            /* particle capacity; <= n: no inactive rows */
  double spawn_lo[3];       /* spawn box (m) */
  double spawn_hi[3];
  double spawn_r_min;       /* radius range (m), 0 < r_min <= r_max */
  double spawn_r_max;
  double spawn_v0[3];       /* initial velocity (m/s) */
  double spawn_w0[3];       /* initial angular velocity (rad/s) */
  int32_t spawn_attempts;   /* attempts per spawn event, 0 .. 1024 */
  int32_t spawn_every;      /* steps between spawn events; <= 0 selects 1 */
  uint64_t spawn_seed;
  int32_t step_warps;       /* warps per block of the contact/integration kernel:
                               4 or 8; <= 0 selects 4 (a tuning knob, results do not
                               depend on it) */
  int32_t reserved;
} dem_params;

/* Particles (host arrays, caller order). */
typedef struct dem_particles {
  int64_t n;         /* number of particles, >= 1 (>= 0 with spawning on) */
  const double* R;   /* [n] radii, > 0 */
  const double* x;   /* [n][3] positions */
  const double* v;   /* [n][3] velocities; NULL = zero */
  const double* w;   /* [n][3] angular velocities; NULL = zero */
  const double* q;   /* [n][4] unit quaternions (scalar first); NULL = identity */
  /* Friction per material (extension for batched independent scenes; the
   * paper has one material).  With n_materials > 0 each particle carries the
   * material material[i] (NULL: 0; spawned particles: 0) whose coefficients
   * are material_mu[3 m .. 3 m + 2] = mu_s, mu_r, mu_t, replacing those of
   * dem_params; a particle pair uses the mean of its two materials'
   * coefficients, a mesh contact the particle's.  n_materials = 0: one
   * material, the coefficients of dem_params. */
  int32_t n_materials;        /* 0 .. 65536 */
  const int32_t* material;    /* [n] material index in [0, n_materials) */
  const double* material_mu;  /* [n_materials][3], each >= 0 */
} dem_particles;

/* Rigid mesh in its reference pose (host arrays); may be empty.  Its elements
 * (Sec. 2.2, 3.3) are the triangles of `tri` followed by the rows of `elem`,
 * numbered 0 .. n_tri + n_elem - 1 in that order; a contact with element k has
 * the key j = -1 - k.  Each element has a radius R_j >= 0: the wall is the set
 * of points within R_j of the element (a sphere, a capsule, a rounded plate).
 * Rows of `elem` hold 1 to 4 vertex indices followed by -1 pads:
 *   1 vertex   a point,
 *   2 vertices a segment a-b,
 *   3 vertices a triangle a-b-c,
 *   4 vertices a rectangle a-b-c-d in order around it; its corners must be
 *              right angles (|ab . ad| <= 1e-9 |ab| |ad|, |a + c - b - d| <=
 *              1e-9 (|ab| + |ad|)) and its edges of nonzero length, else
 *              dem_scene_create returns DEM_ERR_INVALID. */
typedef struct dem_mesh {
  int64_t n_vert;
  const double* vert;        /* [n_vert][3] */
  int64_t n_tri;
  const int32_t* tri;        /* [n_tri][3] vertex indices in [0, n_vert) */
  const double* tri_radius;  /* [n_tri] element radius R_j >= 0 (Sec. 3.3); NULL = 0 */
  int64_t n_elem;            /* further elements, numbered after the triangles */
  const int32_t* elem;       /* [n_elem][4] vertex indices in [0, n_vert), -1 pads */
  const double* elem_radius; /* [n_elem] element radius R_j >= 0; NULL = 0 */
} dem_mesh;

typedef struct dem_stats {
  int64_t steps;          /* steps completed */
  int64_t rebuilds;       /* neighbour-list rebuilds performed */
  int64_t pair_contacts;  /* touching particle pairs in the last step */
  int64_t mesh_contacts;  /* touching particle-element pairs in the last step */
  int64_t list_entries;   /* directed candidate entries in the current list */
  int64_t mesh_candidates;/* particle-element candidates in the current list */
  int32_t max_list_len;   /* longest per-particle candidate list */
  int32_t status;         /* sticky device status (DEM_OK if none) */
  int32_t launches_per_step;    /* kernels launched in a step without a list rebuild */
  int32_t launches_per_rebuild; /* additional kernels launched in a step that rebuilds */
  int64_t active;         /* active particles (rows 0 .. active-1); the rest await spawning */
  int64_t capacity;       /* particle rows n_cap */
} dem_stats;

typedef struct dem_scene dem_scene;

/* Create a scene on the current CUDA device.  `stream` is a cudaStream_t (NULL:
 * the library creates its own).  Copies the host arrays to the device (the
 * particle state of Sec. 2.1 / Table 3, the mesh elements of Sec. 3.3) and
 * captures the step sequence into CUDA graphs (1 and 16 steps, for a start
 * at an even and at an odd step), which dem_step replays.
 * Errors: DEM_ERR_INVALID (parameters outside Table 2's requirements, n < 1,
 * non-finite input, bad element), DEM_ERR_NOMEM, DEM_ERR_CUDA. */
int dem_scene_create(const dem_params* params, const dem_particles* particles,
                     const dem_mesh* mesh, void* stream, dem_scene** out);

/* Device memory supplied by the caller (for instance a framework's caching
 * allocator).  alloc returns a block of `bytes` bytes of device memory on the
 * current device, aligned to 256 bytes, or NULL; release returns a block
 * obtained from alloc.  Both get the caller's `ctx`. */
typedef void* (*dem_alloc_fn)(size_t bytes, void* ctx);
typedef void (*dem_free_fn)(void* ptr, void* ctx);

/* dem_scene_create with every device buffer of the scene taken from `alloc`
 * (the library still creates its streams, events and graphs itself).  The
 * blocks are returned through `release` when the scene is destroyed, after its
 * stream has drained, or at once if creation fails; both functions must stay
 * callable until then.  An allocator interface for the scene's memory
 * (ownership stays with the scene; the paper has no counterpart).
 * Errors: as dem_scene_create; DEM_ERR_INVALID if exactly one of alloc and
 * release is NULL (both NULL: cudaMalloc, as dem_scene_create); DEM_ERR_NOMEM
 * if alloc returns NULL or a block that is not 256-byte aligned. */
int dem_scene_create_with_allocator(const dem_params* params, const dem_particles* particles,
                                    const dem_mesh* mesh, void* stream, dem_alloc_fn alloc,
                                    dem_free_fn release, void* ctx, dem_scene** out);

/* Enqueue `nsteps` time steps on the scene's stream and return without
 * waiting.  Each step: mesh pose, rebuild check, (cell binning, Verlet list and
 * history remap when needed: Sec. 3.3 and the Verlet lists suggested in Sec.
 * 7), contact forces (Sec. 2.2), gather and semi-implicit Euler + SPIRAL
 * integration (Sec. 2.3).  Errors found on the device (DEM_ERR_CAPACITY,
 * DEM_ERR_NONFINITE) are sticky and reported by dem_synchronize(); returns
 * DEM_ERR_INVALID (nsteps < 0) or DEM_ERR_CUDA at once. */
int dem_step(dem_scene* s, int64_t nsteps);

/* Like dem_step, but launches each step phase by phase (no CUDA graph) with
 * CUDA events between phases, waits, and adds the elapsed device time of each
 * phase in milliseconds to phase_ms[0..3]: [0] mesh pose, [1] list rebuild
 * (binning, permutation, Verlet list, history remap; its kernels return at
 * once in steps without a rebuild), [2] contact forces + gather + integration,
 * [3] end-of-step bookkeeping.  For measurement; results are identical to
 * dem_step.  Errors: as dem_step, plus the sticky device status. */
int dem_step_timed(dem_scene* s, int64_t nsteps, double* phase_ms);

/* Wait for the scene's stream; return the sticky device status. */
int dem_synchronize(dem_scene* s);

/* Copy the current state (the particle variables x, v, omega, q of Sec. 2.1
 * and Table 3) to host arrays in caller order, n_cap rows (see
 * dem_params.n_max); any pointer may be NULL.  Rows of inactive particles
 * hold zeros and the identity orientation.  The conversion to absolute
 * doubles and the reordering run on the device (into a staging buffer the
 * scene owns); then one copy per array goes to the caller's memory, which
 * may be pageable or pinned (pinned is faster).  Synchronizes the stream. */
int dem_read_state(dem_scene* s, double* x, double* v, double* w, double* q);

/* Particle radii in caller order, n_cap rows (0 for inactive rows).
 * Synchronizes the stream. */
int dem_read_radii(dem_scene* s, double* R);

/* Contact force and torque sums (no gravity or drag) of the last step, [n][3],
 * caller order.  Requires params.record_forces.  Synchronizes. */
int dem_read_forces(dem_scene* s, double* F, double* T);

/* Active contacts of the last step with their friction history (the contact
 * list c of Table 3, Sec. 3.2: partner j, springs u_s, u_r, u_t).  keys[2k] = i,
 * keys[2k+1] = j in caller indices: a particle pair has i < j; a mesh
 * contact has j = -1 - element index (see dem_mesh).  hist[7k..7k+6] = u_s (3), u_r (3), u_t.
 * Rows are sorted by (i, j).  If `capacity` is too small only the count is
 * written and DEM_ERR_CAPACITY is returned.  Synchronizes. */
int dem_read_contacts(dem_scene* s, int64_t capacity, int64_t* keys, double* hist,
                      int64_t* count);

int dem_get_stats(dem_scene* s, dem_stats* out);

/* Serialise the complete scene (parameters, state, contact history of Sec.
 * 3.2 / Table 3, step count) into `buf`, a host buffer of *len bytes; with
 * buf == NULL, writes the required size to *len.  Synchronizes.  Errors: the
 * sticky device status, except DEM_ERR_CAPACITY: an overflowing list is found
 * while the lists are rebuilt, before the step does any work, so the state
 * and history of the last completed step are intact and still saved (regrow:
 * load the blob into a scene created with larger capacities and step on).
 * DEM_ERR_CAPACITY is also returned (with *len set) if *len is too small. */
int dem_save(dem_scene* s, void* buf, size_t* len);

/* Restore a scene saved by dem_save into `s`, which must have the same
 * particle count, mesh and precision (capacities may differ); the next step
 * rebuilds the lists.  Clears the sticky status.  Synchronizes.  Errors:
 * DEM_ERR_INVALID (not a blob of this scene's shape), DEM_ERR_CAPACITY (a
 * particle has more saved contacts than this scene's capacity), DEM_ERR_CUDA. */
int dem_load(dem_scene* s, const void* buf, size_t len);

void dem_scene_destroy(dem_scene* s);

/* Contact force and torque sums of a particle state that has no friction
 * history yet (the first step of a run), for callers that cannot allocate
 * device memory: a real-time loop, where an allocation can stall for an
 * unbounded time, and hosts whose device memory is owned by another allocator
 * (a framework's caching pool) that must stay the only one.  The paper has no
 * counterpart of this entry point; it is a packaging of the library's FP64
 * first-step arithmetic.
 *
 * Inputs and outputs are DEVICE arrays of the caller: R[n], x[n][3], v[n][3],
 * w[n][3] in, F[n][3] and T[n][3] out (contact sums only: no gravity, no drag).
 * Only particle pairs are considered (no mesh).  The cell grid covers
 * params->domain_lo .. domain_hi with cells of edge 2 r_max.  Every particle
 * must lie inside that box and have 0 < R <= r_max, else the call returns
 * DEM_ERR_INVALID; a cell holding more than 64 particles returns
 * DEM_ERR_CAPACITY (both found on the device, after which the remaining
 * kernels return at once and F, T are left unspecified).  Material parameters
 * come from params (precision and list fields are ignored).
 *
 * Memory: nothing is allocated.  Scratch is one fixed device array inside the
 * library (about 3.5 MB, kept by every device that loads the library until
 * the process exits).  Limits: n <= 131072 particles and at most 262144 grid
 * cells; larger requests return DEM_ERR_INVALID without launching anything.
 * More than 64 touching partners of one particle return DEM_ERR_CAPACITY.
 * The first call on a device looks up the array's device address (set-up, no
 * allocation); make that first call before any stream capture.  Every call
 * shares the array and leaves its last contents there; the call clears what
 * must start at zero.  Calls that overlap on the GPU (other streams, other
 * threads) race on the array and must be serialised by the caller.  The call
 * enqueues its kernels on `stream` (a cudaStream_t, NULL = legacy default)
 * and waits for that stream before returning the status. */
int dem_contact_forces_noalloc(const dem_params* params, int64_t n, double r_max,
                               const double* R, const double* x, const double* v,
                               const double* w, double* F, double* T, void* stream);

const char* dem_status_string(int status);

/* Measurement utility (not part of the timestep): the FP64 fused multiply-add
 * throughput of the current device, in FMAs per second, measured with a
 * kernel of 8 blocks of 256 threads per SM, each thread running 8 independent
 * FMA chains of `iters` steps (best of two timed launches after one warm-up,
 * CUDA events on `stream`, a cudaStream_t or NULL).  It is the denominator of
 * the roofline of the DEM_FP64 step, which the FP64 pipe bounds (GB300 runs
 * double precision at about 1/64 of its FP32 rate).  Allocates and frees a
 * small device buffer and synchronizes the stream.  Errors: DEM_ERR_INVALID
 * (iters <= 0 or fma_per_s NULL), DEM_ERR_NOMEM, DEM_ERR_CUDA. */
int dem_probe_fp64_fma(int64_t iters, void* stream, double* fma_per_s);

#ifdef __cplusplus
}
#endif

#endif /* DEM_H_ */
