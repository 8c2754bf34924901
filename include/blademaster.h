/*
 * blademaster.h -- C ABI of the GB300 TLMPM cutting library.
 *
 * One call of bm_step() advances a scene by whole TLMPM substeps of the
 * cutting method of "BladeMaster: Real-Time Robotic Cutting Simulation with
 * Online-Generated Persistent Discontinuities" (arXiv 2609.27342):
 *   (a) side labels from the swept blade band      Sec. III-C, Eq. 3, 4, 6, 7
 *   (b) hyperelastic stress                         Sec. III-B (neo-Hookean)
 *   (c) label-masked P2G on the reference grid      Sec. III-B, Eq. 1, 2
 *   (d) coupled grid update, tool and pair contact  Sec. III-D/E, Eq. 8-16
 *   (e) PIC/FLIP G2P, MUSL re-scatter, F update     Sec. III-B, Eq. 17
 * The problem statement the calls follow: a rigid tool's pose and twist drive
 * each substep and its reaction wrench is returned (Sec. III-A); cuts appear
 * online from blade motion (Sec. III-C); the rigid system may run at a lower
 * rate and receives an interval-averaged wrench (Sec. III-G).
 *
 * Conventions (every call):
 *   - SI units; doubles for tool state, float32 for particle state.
 *   - Return value: BM_OK (0) or a negative bm_status; bm_last_error() gives a
 *     thread-local message for the last failure on the calling thread.
 *   - Handles are owned by the library and released by the matching destroy.
 *   - Device memory comes from the caller's allocator when one is given
 *     (bm_alloc), else from cudaMalloc; all work is enqueued on the stream
 *     given at creation.  One owner per handle: calls on one handle are not
 *     thread-safe.
 *   - Asynchrony: bm_step/bm_batch_step enqueue work and return launch
 *     errors immediately; the device error word (bit set of BM_ERRBIT_*) is
 *     sticky and is read by bm_read_state/bm_scene_info/bm_tool_wrench, which
 *     synchronise the stream.
 *   - Particle arrays crossing the ABI are in the caller's original particle
 *     order, array-of-structs (x: [n][3], F: [n][9] row-major).
 */
#ifndef BLADEMASTER_H
#define BLADEMASTER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BM_MAX_CUTS 32     /* cut-side digits per particle (two 32-bit masks) */
#define BM_MAX_SEGMENTS 16 /* trajectory segments per blade */

typedef enum {
  BM_OK = 0,
  BM_E_INVALID = -1,         /* bad argument or handle */
  BM_E_OOM = -2,             /* allocation failed (caller allocator or cudaMalloc) */
  BM_E_CUDA = -3,            /* CUDA runtime error (message in bm_last_error) */
  BM_E_SLOT_OVERFLOW = -4,   /* logical-grid slots exceeded their capacity */
  BM_E_INVERTED = -5,        /* det F <= 1e-6 met (clamped, simulation continued) */
  BM_E_NONFINITE = -6,       /* NaN/Inf in particle position or velocity */
  BM_E_CONTACT_OVERFLOW = -7,/* pair-contact history or cell capacity exceeded */
  BM_E_TIMEOUT = -8,         /* a bounded device wait gave up */
  BM_E_TOO_MANY_CUTS = -9,   /* cut id outside [0, BM_MAX_CUTS) */
  BM_E_CAPACITY = -10        /* batch pool has no room for the scene */
} bm_status;

/* bits of the sticky device error word (bm_scene_info.error_bits) */
#define BM_ERRBIT_SLOT_OVERFLOW 1u
#define BM_ERRBIT_INVERTED 2u
#define BM_ERRBIT_NONFINITE 4u
#define BM_ERRBIT_CONTACT_OVERFLOW 8u
#define BM_ERRBIT_TOO_MANY_CUTS 16u

typedef struct bm_scene_s *bm_scene_t;
typedef struct bm_batch_s *bm_batch_t;

/* Device allocator callbacks (e.g. PyTorch's caching allocator).  alloc
 * returns a device pointer of at least `bytes` bytes on `stream`, or NULL;
 * free releases it.  Pass NULL for cudaMalloc/cudaFree. */
typedef struct {
  void *(*alloc)(size_t bytes, void *stream, void *ctx);
  void (*free)(void *ptr, void *stream, void *ctx);
  void *ctx;
} bm_alloc;

/* Material, discretisation and contact parameters of one scene.
 * Particle mass m_p = rho V0 and contact radius R_p = s_R V0^(1/3) / 2
 * (Sec. III-E) are uniform over the scene.  Fields marked "<=0 -> default"
 * take the default when non-positive. */
typedef struct {
  double E, nu, rho;         /* Lame: mu = E/(2(1+nu)), lambda = E nu/((1+nu)(1-2nu)) */
  double dx;                 /* reference-grid spacing; node i sits at origin + i dx (Eq. 1) */
  double origin[3];
  double V0;                 /* reference volume per particle V_p^0 */
  double dt;                 /* substep */
  double beta;               /* PIC/FLIP blend (Eq. 17), in [0, 1] */
  double gravity[3];
  int floor_enabled;         /* frictionless half-space z >= floor_z */
  double floor_z;
  double s_R, s_n;           /* contact radius and normal response scales (Sec. III-E) */
  double gamma_k, gamma_c;   /* tangential stiffness / damping ratios (Eq. 12) */
  int pair_contact;          /* material-material contact (Eq. 10-13) */
  double pair_mu_s, pair_mu_d;
  double G_c, zeta;          /* W_th = G_c V0^(2/3) (1 - zeta)/zeta (Eq. 5) */
  double u_min;              /* minimum cut-advance speed (Eq. 5) */
  double b_back, b_lead;     /* band rear / lead extent, <=0 -> dx (Eq. 4) */
  double band_half_width;    /* h_k, <=0 -> 6 dx (Sec. III-D) */
  int tool_contact;          /* 0: the blade only assigns labels */
  int wrench_history;        /* substeps of per-substep wrench kept on device */
  int model;                 /* elastic model: BM_MODEL_NEO_HOOKEAN or BM_MODEL_FIXED_COROTATED */
  double yield_stress;       /* > 0: von Mises plasticity (Pa), radial return of the deviatoric
                                principal Hencky strains of Fe = F Fp^-1; P = P(Fe) Fp^-T */
  double viscosity;          /* > 0: Newtonian viscosity eta (Pa s): J eta (L + L^T) F^-T added
                                to P, L = dF/dt F^-1 from the previous substep */
} bm_scene_desc;

/* Elastic models (first Piola-Kirchhoff stress P(F), Sec. III-B):
 * compressible neo-Hookean, P = mu (F - F^-T) + lambda ln J F^-T;
 * fixed-corotated (the paper's model), P = 2 mu (F - R) + lambda (J - 1) J F^-T
 * with F = R S the polar decomposition.  J <= 1e-6 is clamped and flagged
 * (BM_ERRBIT_INVERTED). */
enum { BM_MODEL_NEO_HOOKEAN = 0, BM_MODEL_FIXED_COROTATED = 1 };

/* A piece of blade trajectory: a world-frame twist (about the tool-frame
 * origin x_B) held for n_steps substeps.  Kinematic tool: the prescribed
 * twist.  Dynamic tool: the servo target.  cut_id >= 0 is the cut (ternary
 * digit k of Eq. 7) this stroke creates; -1 = non-cutting move. */
typedef struct {
  int n_steps;
  int cut_id;
  double v[3], omega[3];
} bm_segment;

/* Planar blade: an oriented box, half-thickness along n, half-length along e,
 * `height` behind the edge along -d (tool-frame axes of Eq. 3).  mass <= 0
 * makes the tool kinematic (w_B = 0, Eq. 15). */
typedef struct {
  double edge_point[3], normal[3], edge_dir[3], front_dir[3]; /* tool frame */
  double half_length, thickness, height;
  double mu_s, mu_d;                                       /* tool friction */
  double mass, inertia[9];                                 /* body frame, row-major */
  double pose_x[3], pose_R[9];                             /* initial pose (tool->world) */
  double servo_gain;                                       /* <=0 -> 1/(10 dt) */
  int rigid_interval;                                      /* substeps per rigid update, >=1 */
  int n_segments;
  bm_segment segments[BM_MAX_SEGMENTS];
} bm_blade_desc;

/* Field ids for bm_read_state / bm_write_state.  Element types:
 *   X, x, v, ut: float32 [n][3];  F: float32 [n][9];  D: float32 [n];
 *   CODE: int64 [n] ternary code c_p of Eq. 7 (read only);
 *   MASK1, MASK2: uint32 [n] -- bit k set <=> digit k is 1 (resp. 2);
 *   PAIR_PARTNER: int32 [n][16], PAIR_U: float32 [n][16][3] (read only,
 *   scenes with material-material contact): the tangential spring history of
 *   Eq. 12 between particle pairs in contact, as the next substep will read
 *   it.  Each pair in contact is listed once, by one of its two particles:
 *   entry k of particle p names the partner q (caller index; -1 ends the
 *   list) and PAIR_U[p][k] is the spring displacement u of p's motion
 *   relative to q (the same pair seen from q has -u). */
enum {
  BM_FIELD_X = 1u << 0,
  BM_FIELD_x = 1u << 1,
  BM_FIELD_v = 1u << 2,
  BM_FIELD_F = 1u << 3,
  BM_FIELD_D = 1u << 4,
  BM_FIELD_UT = 1u << 5,
  BM_FIELD_CODE = 1u << 6,
  BM_FIELD_MASK1 = 1u << 7,
  BM_FIELD_MASK2 = 1u << 8,
  BM_FIELD_PAIR_PARTNER = 1u << 9,
  BM_FIELD_PAIR_U = 1u << 10
};
#define BM_NUM_FIELDS 11

typedef struct {
  int64_t n_particles;
  int64_t n_nodes;           /* reference-grid nodes covering every stencil */
  int64_t n_slots;           /* occupied logical-grid slots (Sec. III-G compact slots) */
  int64_t slot_capacity;
  int64_t step;              /* substeps taken */
  uint32_t error_bits;       /* sticky BM_ERRBIT_* word */
  int grid_lo[3], grid_dim[3];
  int32_t current_cut;       /* id of the cut in progress (the last cut-creating segment), -1 before any */
  int64_t contact_list_builds; /* material-material contact: candidate-list builds so far */
} bm_scene_info;

/* ---- scene ------------------------------------------------------------- */

/* Create a scene from n reference positions X_ref (host, float32 [n][3]).
 * Builds the fixed reference stencil table (Eq. 1: the node-to-particle
 * neighbourhood never changes), sets x = X, v = 0, F = I, D = 0, all codes 0.
 * `alloc` may be NULL.  `stream` is a cudaStream_t (NULL = default stream). */
int bm_scene_create(const bm_scene_desc *desc, const float *X_ref, int64_t n,
                    const bm_alloc *alloc, void *stream, bm_scene_t *out);

/* Attach the scene's blade (one per scene); *blade_id receives 0. */
int bm_add_blade(bm_scene_t s, const bm_blade_desc *b, int *blade_id);

/* Override the tool pose (x_B, row-major R tool->world) and world twist
 * (v_B, omega_B) from the next substep on -- the external rigid-system path of
 * Sec. III-A.  pose = {x[3], R[9]}, twist = {v[3], omega[3]}. */
int bm_set_tool_state(bm_scene_t s, int blade_id, const double pose[12], const double twist[6]);
int bm_get_tool_state(bm_scene_t s, int blade_id, double pose[12], double twist[6]);

/* Advance n_substeps substeps on the scene's stream (one launch per kernel
 * per substep: the plain one-scene-per-launch path). */
int bm_step(bm_scene_t s, int n_substeps);

/* Stop substep of a scene (a serving control; the paper has no counterpart):
 * once the scene has taken `stop_at` substeps it stops advancing -- every
 * kernel of later substeps, alone or in a batch, leaves it untouched until
 * the stop is moved -- so a batch can step its members by whole chunks while
 * each request still ends after exactly its own number of substeps, with
 * the same result as a run of that length alone.  stop_at = -1 (the
 * default) never stops.  A stop at or below the current substep freezes the
 * scene at once.  Synchronises the scene's stream.  Errors: BM_E_INVALID
 * (bad handle, stop_at < -1). */
int bm_scene_set_stop(bm_scene_t s, int64_t stop_at);

/* Copy the fields in field_mask into dst[i] (one pointer per set bit, in bit
 * order).  dst_on_device != 0: dst are device pointers.  Synchronises the
 * stream; returns the error word via bm_scene_info. */
int bm_read_state(bm_scene_t s, uint32_t field_mask, void *const *dst, int dst_on_device);

/* Overwrite fields (x, v, F, D, UT, MASK1, MASK2) from src, same layout.
 * Writing masks rebuilds the logical-grid slots before the next substep. */
int bm_write_state(bm_scene_t s, uint32_t field_mask, const void *const *src, int src_on_device);

/* Interval-averaged reaction wrench {F[3], tau[3]} of the last completed
 * rigid interval (Eq. 16, Sec. III-G); tau about x_B.  Synchronises. */
int bm_tool_wrench(bm_scene_t s, int blade_id, double out[6]);

/* Per-substep reaction wrenches of substeps [first, first+count) (count*6
 * doubles, host).  Only the first desc.wrench_history substeps are kept. */
int bm_wrench_history(bm_scene_t s, int blade_id, int64_t first, int64_t count, double *out);

/* bm_read_state without any device allocation -- this has no counterpart in
 * the paper; it serves callers that must not allocate device memory while the
 * simulation runs: a real-time control loop of the external rigid-body system
 * reading state every tick (cudaMalloc/cudaFree synchronise the device and can
 * stall for milliseconds), or a process whose device memory is already
 * reserved by a framework's caching allocator, where a per-call cudaMalloc
 * can fail.  Same layout and result as bm_read_state with host destinations
 * (dst are host pointers).  The library keeps ONE staging array of 16 MiB
 * in device memory for the life of the process (every GPU that loads the
 * library holds its own copy); each requested field in turn is gathered into
 * it and copied to dst, so each field may be at most 16 MiB: a larger field
 * (e.g. F beyond 466,033 particles) is rejected with BM_E_INVALID before any
 * work is enqueued.  The scene's device (current when it was created) must
 * be the current device, else BM_E_INVALID.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that
 * device current -- make that first call before any stream capture.  All
 * calls share the one array and synchronise the scene's stream before they
 * return; calls from several threads whose GPU work overlaps race on it. */
int bm_read_state_noalloc(bm_scene_t s, uint32_t field_mask, void *const *dst);

int bm_scene_info_get(bm_scene_t s, bm_scene_info *out);
int bm_scene_destroy(bm_scene_t s);

/* ---- checkpoints ---------------------------------------------------------
 * A checkpoint is the scene's complete simulation state in one flat buffer:
 * particle state (x, v, F, D, u_t, side masks; pair-contact history when the
 * scene has pair contact), the tool's pose, twist and rigid-interval
 * accumulators, the current cut, the substep counter, the frame of the next
 * substep, the per-substep wrench history and the sticky error word.
 * Restoring it makes the next substeps reproduce, bit for bit, the ones that
 * followed the save (resume after a failure, and the recomputation between
 * the checkpoints of the adjoint).  The buffer is caller-owned;
 * bm_checkpoint_size gives its size.  It may be restored into the same scene
 * only (same handle, any world: a scene moved into or out of a batch keeps
 * its checkpoints valid).  dst/src are device pointers when *_on_device != 0,
 * else host memory.  Both calls synchronise the scene's stream.  Restore
 * rejects (BM_E_INVALID) a buffer whose header does not match the scene and
 * rebuilds the logical-grid slots for the restored side masks. */
int bm_checkpoint_size(bm_scene_t s, int64_t *bytes);
int bm_checkpoint_save(bm_scene_t s, void *dst, int dst_on_device);
int bm_checkpoint_restore(bm_scene_t s, const void *src, int src_on_device);

/* ---- adjoint of the substep (calibration) ---------------------------------
 * Reverse mode of one substep for gradients of a loss on the per-substep
 * reaction force F_B^n (Eq. 16) with respect to the material (E, nu) and the
 * blade's segment velocities, used with checkpoints: restore the state before
 * substep n (bm_checkpoint_restore) and call bm_adjoint_substep for n in
 * decreasing order.  The discrete decisions of the forward substep are held
 * fixed: codes (Eq. 6-7), contact active sets (Eq. 14-15), stick or slip
 * (Eq. 12), the front band and D release (Eq. 5) and the blade-box face;
 * they are re-taken from the restored state with the forward float32
 * expressions.  With the codes fixed, P2G, the coupling of Eq. 8, the grid
 * update (Eq. 9), G2P (Eq. 17), the MUSL re-scatter and the F update form a
 * fixed linear map; its transpose is applied by per-node gathers in a fixed
 * order (no atomics).  float32 arithmetic, float64 parameter accumulators.
 * Scope: a kinematic blade (mass 0) whose segments and current twist have no
 * angular velocity, rigid interval 1, no material-material contact;
 * anything else is BM_E_INVALID.  Device memory for the adjoint (about 84
 * bytes per particle and 40 per logical-grid slot) comes from the scene's
 * allocator; calls are ordered on the scene's stream. */
typedef struct bm_adjoint_s *bm_adjoint_t;
int bm_adjoint_create(bm_scene_t s, bm_adjoint_t *out);
/* zero the state adjoints and every accumulator */
int bm_adjoint_reset(bm_adjoint_t a);
/* The scene holds the state before substep n (its substep counter says n).
 * force_bar = dL/dF_B^n (host, 3 doubles).  Replaces the state adjoints of
 * the state after the substep by those of the state before it and adds this
 * substep's terms to the parameter accumulators.  Does not change the scene. */
int bm_adjoint_substep(bm_adjoint_t a, const double force_bar[3]);
/* Read (write != 0: overwrite) state adjoints in caller particle order,
 * fields BM_FIELD_x, BM_FIELD_v, BM_FIELD_F, BM_FIELD_UT in increasing bit
 * order (float32, n*3 / n*9 / n*3); buf are device pointers when
 * on_device != 0.  Synchronises. */
int bm_adjoint_state(bm_adjoint_t a, uint32_t field_mask, void *const *buf, int on_device, int write);
/* Accumulated gradients (host, cap >= 7 + 3 * BM_MAX_SEGMENTS doubles):
 * dL/dE, dL/dnu, dL/dmu, dL/dlambda, the adjoint of the tool position at the
 * earliest substep processed (3), then dL/dv of each trajectory segment's
 * linear velocity (3 per segment, BM_MAX_SEGMENTS segments).  Returns the
 * count written.  Synchronises. */
int bm_adjoint_params(bm_adjoint_t a, double *out, int cap);
int bm_adjoint_destroy(bm_adjoint_t a);

/* ---- batches of uneven scenes -------------------------------------------
 * A batch owns packed device pools (particles, nodes, slots) with a fixed
 * capacity.  Scenes moved into it keep their handles; bm_batch_step advances
 * every member scene by n substeps from one CUDA-graph launch per chunk of
 * substeps, with no host work between substeps. */
typedef struct {
  int64_t max_particles;   /* pool capacities */
  int64_t max_nodes;
  int64_t max_slots;       /* <=0 -> 4 x max_nodes */
  int64_t max_bricks;      /* 4x4x4-cell bricks, <=0 -> max_nodes/27 + max_scenes (always enough) */
  int max_scenes;
  int graph_chunk;         /* substeps per captured graph, <=0 -> 16 */
  int node_tile;           /* nodes per CTA of the per-node kernels: 64..512; <=0 -> 128 */
  int pair_contact;        /* reserve pair-contact history for member scenes */
} bm_batch_desc;

int bm_batch_create(const bm_batch_desc *desc, const bm_alloc *alloc, void *stream,
                    bm_batch_t *out);
/* Create a scene (and its blade, when blade != NULL) directly inside the
 * batch pools: the same initial state as bm_scene_create + bm_add_blade,
 * without device allocations of its own.  BM_E_CAPACITY when the pools have
 * no room (nothing is created).  Batch members keep no wrench history. */
int bm_batch_scene_create(bm_batch_t b, const bm_scene_desc *desc, const bm_blade_desc *blade,
                          const float *X_ref, int64_t n, bm_scene_t *out);
/* Move a scene's device state into the batch pools (BM_E_CAPACITY if it
 * does not fit).  The scene's own buffers are released. */
int bm_batch_add(bm_batch_t b, bm_scene_t s);
/* Move a scene out of the batch into buffers of its own. */
int bm_batch_remove(bm_batch_t b, bm_scene_t s);
int bm_batch_step(bm_batch_t b, int n_substeps);
/* Pool needs of a scene with these parameters: particles, reference-grid
 * nodes, 4x4x4-cell bricks and total device bytes (any output may be NULL). */
int bm_scene_footprint(const bm_scene_desc *desc, const float *X_ref, int64_t n,
                       int64_t *particles, int64_t *nodes, int64_t *bricks, int64_t *bytes);
/* Tool state of every member, in membership order (the order of
 * bm_batch_members): states[n][18] = {x_B[3], R[9], v_B[3], omega_B[3]};
 * n must equal the member count.  on_device != 0: a device pointer.
 * Stream-ordered, no synchronisation (the per-substep input of an external
 * rigid-body system, Sec. III-A). */
int bm_batch_set_tool_states(bm_batch_t b, const double *states, int n, int on_device);
/* Interval-averaged wrench of every member, out[n][6] (Eq. 16, Sec. III-G).
 * on_device != 0: a device pointer, stream-ordered; otherwise the call
 * synchronises the stream and fills host memory. */
int bm_batch_tool_wrenches(bm_batch_t b, double *out, int n, int on_device);
/* Member scenes in membership order; returns the member count. */
int bm_batch_members(bm_batch_t b, bm_scene_t *out, int cap);
/* Largest sticky error word over the members (OR of BM_ERRBIT_*); syncs. */
int bm_batch_errors(bm_batch_t b, uint32_t *bits);
/* Profiling hook: run n_substeps eagerly (no graph) with CUDA events around
 * every kernel launch on the batch stream; ms[k] receives the summed device
 * time of kernel k over the run and launches[k] its launch count (cap >= 9
 * entries; names from bm_kernel_name).  Returns the kernel count (>= 0) or
 * a bm_status.  Advances the simulation like bm_batch_step. */
int bm_batch_profile(bm_batch_t b, int n_substeps, double *ms, int *launches, int cap);
const char *bm_kernel_name(int i);
/* Launch shape used by subsequent bm_batch_step calls (set by the
 * autotuner): substeps per captured CUDA graph (1..256), nodes per CTA of the
 * per-node kernels (multiple of 32 in 64..512) and the brick-kernel
 * occupancy variant v in 0..26, one choice per brick kernel: v % 3 for P2G
 * (4, 3 or 2 resident CTAs per SM; 3, 2 or 4 in launch sets with plasticity
 * or viscosity), (v / 3) % 3 for G2P+MUSL (5, 4 or 6) and
 * v / 9 for the F update (7, 5 or 6); fewer CTAs leave more registers per
 * thread, more hide more latency; 0 is every kernel's default.  Results do not
 * depend on any of them: every sum is taken in a fixed order and the
 * variants share their arithmetic.  Synchronises the batch stream; captured
 * graphs are rebuilt on the next step.  BM_E_INVALID on an out-of-range
 * argument (the previous shape stays). */
int bm_batch_set_tiles(bm_batch_t b, int graph_chunk, int node_tile, int brick_variant);
int bm_batch_destroy(bm_batch_t b);

/* ---------------------------------------------------------------------------
 * Reference-grid surface reconstruction (Sec. III-F), for visualisation.
 *
 * The uniform reference grid is the scene's sub-cell particle lattice: with
 * lattice[a] particles per reference cell along axis a the spacing is
 * h_a = dx / lattice[a], and a lattice vertex is material when a particle
 * sits on it (the original boundary is the boundary of the union of the
 * material vertices' voxels).  Links between lattice neighbours are
 * disconnected where the two particles' side codes conflict (the blade's
 * sweep labelled them apart); a disconnected link's Hermite data is the
 * crossing of the lowest conflicting cut's plane with it, the plane being
 * the blade's (n, n . x_e) recorded when that cut began.  In every lattice
 * cell the connected components of material vertices over the connected
 * links are the local regions; each region with a disconnected or boundary
 * link gets one vertex by local dual contouring (the pseudo-inverse
 * minimiser of the quadratic error of its links' Hermite data, relative to
 * their mean, eigenvalues below 0.1 dropped, clamped to the cell), so the two
 * sides of a cut keep separate, coincident faces.  Each (Hermite link,
 * material end) gives a quad over that end's regions in the four cells
 * around the link, split into two triangles wound outward (triangles with a
 * repeated vertex dropped).  Motion is one-way: a vertex carries the code of
 * its region's lowest corner particle and follows that code's logical grid
 * through fixed trilinear weights over the 8 reference nodes around it,
 * each node's displacement being the B-spline-weighted mean of x - X over
 * the particles with exactly that code.
 *
 * Ordering: vertices by cell (lower-corner lattice index, x fastest, from
 * -1), then region (by lowest corner); triangles by link (lower end's
 * lattice index, then axis x, y, z), lower end's quad first.  Integer output
 * is deterministic; positions are float32.
 * ------------------------------------------------------------------------- */
typedef struct bm_surface_s *bm_surface_t;
/* Build the lattice map of a scene (plain or batched).  lattice[3] >= 1.
 * BM_E_INVALID if a particle is off the lattice (more than 1e-3 h from a
 * lattice point), two share a point, or the lattice does not sit at the
 * reference cells' sub-cell centres (every lattice point's stencil base cell
 * must equal its particle's).  The handle keeps device buffers from the
 * scene's allocator and stays valid while the scene lives (also across
 * batch add/remove). */
int bm_surface_create(bm_scene_t s, const int lattice[3], bm_surface_t *out);
/* Rebuild the topology from the scene's current side codes (rebuild != 0)
 * and re-embed every vertex in the current motion field; returns the vertex
 * and triangle counts.  Enqueued on the scene's stream; synchronises to
 * return the counts. */
int bm_surface_update(bm_surface_t f, int rebuild, int64_t *n_vertices, int64_t *n_triangles);
/* Copy the last update's output: vertices [n_vertices][3] current
 * positions, reference [n_vertices][3] reference positions, triangles
 * [n_triangles][3] vertex indices, masks [n_vertices][2] the vertex codes
 * (s1, s2 bit masks).  Any pointer may be NULL.  dst_on_device selects device
 * or host destinations.  Synchronises. */
int bm_surface_read(bm_surface_t f, float *vertices, float *reference, int32_t *triangles,
                    uint32_t *masks, int dst_on_device);
int bm_surface_destroy(bm_surface_t f);

/* Diagnostic: FP32 FMA throughput of the current device, measured by a
 * kernel of independent fused multiply-add chains filling every SM (eight
 * 256-thread blocks per SM), timed with CUDA events on `stream` (NULL: the
 * default stream).  *tflops receives 2 x FMAs / second / 1e12.  The ceiling
 * for the ALU-bound parts of the substep (no tensor cores are involved). */
int bm_fp32_fma_peak(void *stream, double *tflops);

const char *bm_last_error(void);
const char *bm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* BLADEMASTER_H */
