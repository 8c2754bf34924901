// Internal device-side layout of the GB300 TLMPM cutting library.
//
// Memory is organised as "worlds": packed pools of particles, reference-grid
// nodes and logical-grid slots that hold one scene (the plain path) or many
// scenes (a batch).  Every kernel walks a work list of tiles, each tile
// naming its scene, so one code path serves both.
//
// Particle state is structure-of-arrays float32, particles sorted by their
// fixed reference base cell (the TLMPM stencil never changes, Eq. 1), so the
// node-to-particle neighbourhood is a static CSR table (cell_start) and P2G
// is an atomic-free gather in a fixed order: deterministic, bit-identical
// whether a scene runs alone or inside a batch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/blademaster.h"

#define BM_MAXS 16           // logical grids (distinct codes) per node
#define BM_TILE_SLOTS 512    // tile slots cached in shared memory; tiles with more read the pool
#define BM_TILE_NODES 216    // 6 x 6 x 6 nodes touched by a brick of 4 x 4 x 4 base cells
#define BM_BRICK_CELLS 64
#define BM_HIST 16           // pair-contact history entries per particle
#define BM_NBR 64            // pair-contact candidates kept per particle (Verlet list)
#define BM_WRENCH_W 6

struct DevSeg {
  int n_steps, cut_id;
  double v[3], w[3];
};

// One scene, resident in device memory.  Static parameters are written at
// creation; the tool block and counters are updated by kernels.
struct DevScene {
  // ranges inside the world pools
  int p_begin, n_p;
  int node_begin, n_node;
  int cell_begin, n_cell;
  int slot_begin, slot_cap;
  int brick_begin, n_brick;
  int ntile_begin, n_ntile;
  int ppool_begin, ppool_cap;  // brick-tile partial sums (entries)
  int hist_begin;           // wrench history offset (in wrench records)
  int hist_cap;
  int nb[3];                // base-cell grid
  int nn[3];                // node grid = nb + 2
  int nbr[3];               // brick grid = ceil(nb / 4)
  // material / discretisation (float32 for the particle kernels)
  float dx, inv_dx;
  float mp, V0, Rp, dt, beta, g[3], mu, lam;
  int model;                // BM_MODEL_*
  float yield_stress;       // > 0: von Mises projection
  float viscosity;          // > 0: Newtonian viscosity
  float Wth, u_min, b_back, b_lead, h;
  float s_n, gamma_k, gamma_c;
  float pair_mu_s, pair_mu_d;
  float floor_z;
  float pair_h, pair_inv_h;  // pair-contact hash cell size of the last list build
  int pair_vmax_bits;        // max particle speed of this substep (float bits)
  int pair_disp_bits;        // max over particles of displacement since the last list
                             // build + dt |v| (float bits)
  int pair_valid;            // the candidate lists match this scene's pool (0: rebuild)
  int pair_build;            // the lists are rebuilt this substep
  long long pair_builds;     // candidate-list builds so far
  int floor_on, pair_on, tool_contact_on, has_blade;
  // float64 copies used by the exact label path and the tool integrator
  double dt_d, h_d, L_d, b_back_d, b_lead_d;
  double origin_d[3];
  // blade (static)
  double edgeT[3], nT[3], eT[3], dT[3];
  double half_len, half_thick, half_height, mu_s, mu_d;
  double mass, Ib_inv[9], kv;
  int rigid_interval, nseg;
  DevSeg seg[BM_MAX_SEGMENTS];
  // blade (dynamic, float64)
  double xB[3], R[9], vB[3], wB[3];
  double accF[3], accT[3];
  int acc_cnt, cur_cut;
  double lastW[6];
  // frame of the current substep (written by the tool kernel / set-up)
  int cut, reset_D;
  double dxe[3], dn[3], de[3], dd[3], dve[3];
  float fxe[3], fn[3], fe[3], fd[3], fve[3], fc[3], fxB[3], fvB[3], fwB[3];
  float fIinv[9], finv_mass, fmu_s, fmu_d, fhext[3], fL;
  // plane of each cut in the world frame at the substep it began (n, n . x_e),
  // the Hermite data of its faces in the surface reconstruction (Sec. III-F);
  // bit k of cutpl_set marks cut k as recorded
  double cutpl[BM_MAX_CUTS][4];
  unsigned int cutpl_set;
  // counters and flags
  long long step;
  long long stop_at;        // >= 0: the scene stops advancing once step reaches it
  int frozen;               // set by the tool kernel when step reaches stop_at; every
                            // substep kernel then leaves the scene untouched
  unsigned int err;
  int label_pending;
  int need_rebuild;
  int n_slots;
  int pad_[1];
};

struct PPool {
  float *fx[3];
  uint32_t *base;           // packed local base cell: bx | by << 10 | bz << 20
  float *x[3], *v[3], *F[9], *D, *ut[3];
  uint8_t *tflag;           // 0: D and u_t are both zero (P2G then skips their loads); set by
                            // P2G when either becomes nonzero and by any write of either field
  float *Fpi[9];            // inverse plastic deformation Fp^-1 (identity without plasticity)
  float *Fdot[9];           // dF/dt of the last substep (viscosity)
  uint32_t *s1, *s2;        // bit k: digit k == 1 (s1) or == 2 (s2)
  float *J[3];              // pair-contact impulse of this substep (k_pair -> k_p2g_brick)
  uint8_t *pend;            // side digit assigned this substep (0: none), committed by k_fupd
  int *perm;                // pool index -> caller's particle index
  // pair contact
  int *hkey;                // bucket of each particle's current-configuration cell
  int *horder;              // particles ordered by bucket, by pool index inside a bucket
  float4 *hent;             // the same order: position and pool index (int bits in w)
  uint32_t *hbase;          // the same order: packed base cell of the entry's particle
  unsigned long long *hcell;  // per particle: scene and current-configuration cell (cell_key)
  unsigned long long *hentk;  // hent order: the entry's cell key
  int *hist_partner[2];     // pair history (partner pool index, -1 ends), by step parity
  float *hist_u[2];         // [(p * BM_HIST + k) * 3]: tangential spring displacement
  int *nbr;                 // [p * BM_NBR + k]: contact candidates (pool index in bits 0-30;
                            // bit 31: the pair shares a reference stencil)
  uint8_t *nbr_n;           // candidates of each particle
  float *xb[3];             // positions at the last candidate-list build
};

struct NPool {
  int *cell_start;          // per scene n_cell + 1 entries (pool particle indices)
  int *slot_off;            // first slot of each node (pool slot index)
  uint8_t *slot_cnt;        // logical grids at each node
  uint8_t *ncodes;          // distinct codes found at each node by the last recount
  uint8_t *dirty;           // per node: a particle of its stencil gained a label since the last recount
  uint2 *tmp_codes;         // [node * BM_MAXS] scratch for the rebuild
  int *tile_sum;            // per node tile: slots in the tile (scan scratch)
};

struct SPool {
  float4 *vold;             // xyz = v_old (Eq. 9), w = m
  float4 *vnew;             // xyz = v_new (Eq. 9)
  float4 *vstar;            // xyz = v* (MUSL)
  uint2 *code;              // (s1, s2)
};

struct BPool {              // brick-tile partial sums
  float4 *pm;               // [poff[brick] + tile slot]: (sum N, sum N v) / MUSL sum N v
  float4 *pd;               // [poff[brick] + tile slot]: sum (A grad N + N J)
  int *poff;                // first entry of each brick's partial sums (-1: pool overflow)
  int *ptot;                // slots in each brick's tile
  int *tdesc;               // [brick * BM_TILE_NODES]: first tile slot | slot count << 16
  int *tgoff;               // [brick * BM_TILE_NODES]: first pool slot of each tile node
};

struct HashPool {           // pair-contact spatial hash (world-wide table)
  int *bucket_start;        // [n_buckets + 1]: counts, then exclusive offsets
  int *bucket_fill;         // [n_buckets]
  int *block_sum;           // [n_buckets / 1024 + 1]
  int *build;               // some scene rebuilds its candidate lists this substep
  int n_buckets;            // power of two
};

struct World {
  DevScene *scenes;
  PPool P;
  NPool N;
  SPool S;
  BPool B;
  HashPool H;
  double *wpart;            // per brick wrench partials (6 doubles)
  double *whist;            // wrench history records (6 doubles)
};

// brick tiles: x = scene slot, y = pool brick, z = first particle, w = particle count
// node tiles:  x = scene slot, y = first pool node, z = count, w = tile id
struct LaunchSet {
  const int4 *btiles;
  int n_btiles;
  int ppc16;                // some scene has more than 8 particles in a base cell
  const int4 *ntiles;
  int n_ntiles;
  int ntile_size;
  int variant;              // brick-kernel occupancy variant, 0..BM_NUM_VARIANTS-1
  const int *scene_ids;     // scenes in this set
  int n_scenes;
  int any_pair;             // some scene has pair contact
  int any_inelastic;        // some scene has plasticity or viscosity
  int pair_n_particles;     // particles of pair-contact scenes (hash sizing)
};

// surface reconstruction (bm_surface.cu, Sec. III-F) over a scene's sub-cell
// particle lattice; the runtime fills it, the kernels only read the inputs
struct SurfParams {
  int n[3];                  // lattice points per axis
  int nc[3];                 // cells (and link lower ends) per axis: n + 1, lower corners from -1
  long long n_cells;         // nc[0] * nc[1] * nc[2]
  double Xmin[3], h[3];      // lattice point j sits at Xmin + j h
  double origin[3], dx;      // the scene's reference grid
  int lo[3];                 // absolute index of the scene's local base cell 0
  int bmin[3], bmax[3];      // stencil base cells of the first and last lattice point per axis
  const int *jstart[3];      // [B - bmin]: first lattice index whose base cell is >= B
  int *lat;                  // lattice point (x fastest) -> scene-relative pool index, -1 empty
  float *Xr[3];              // scene-relative reference positions
  int p_begin, slot;         // the scene's first pool particle and its record in the world
  int *cell_cnt, *cell_off;  // per cell: vertices, first vertex (n_cells + 1 entries)
  uint32_t *cell_reg;        // per cell: 4 bits per corner, vertex ordinal of its region (15: none)
  int *pt_cnt, *pt_off;      // per link lower end: triangles, first triangle (n_cells + 1)
  int *scan_tmp;             // block sums of the scans
  float *ref[3], *cur[3];    // vertex reference and current positions
  int *anchor;               // vertex anchor particle (scene-relative)
  uint32_t *vmask[2];        // vertex code
  int *tri;                  // [3 * triangles]
};
cudaError_t bm_launch_surface_map(const World &w, const SurfParams &sp, int n, const int *jlin,
                                  const float *Xc, cudaStream_t st);
cudaError_t bm_launch_surface_cells(const World &w, const SurfParams &sp, cudaStream_t st);
cudaError_t bm_launch_surface_vertices(const World &w, const SurfParams &sp, cudaStream_t st);
cudaError_t bm_launch_surface_tri_count(const World &w, const SurfParams &sp, cudaStream_t st);
cudaError_t bm_launch_surface_tris(const World &w, const SurfParams &sp, cudaStream_t st);
cudaError_t bm_launch_surface_embed(const World &w, const SurfParams &sp, int n_vertices, cudaStream_t st);

// kernel launchers (bm_kernels.cu)
#define BM_NUM_KERNELS 19
#define BM_NUM_VARIANTS 27  // 3 occupancy choices for each of the 3 brick kernels
extern const char *const bm_kernel_names[BM_NUM_KERNELS];
cudaError_t bm_kernels_init();  // per device: shared-memory limits of the brick kernels

// adjoint of the substep (bm_adjoint.cu); the work record is opaque here
size_t bm_adj_work_struct_size();
size_t bm_adj_work_alloc_bytes(int64_t n_p, int64_t slot_cap);
void *bm_adj_carve(void *base, int64_t n_p, int64_t slot_cap, int scene_slot, void *out_work);
void bm_adj_set_slot(void *work, int scene_slot);
double *bm_adj_acc(void *work);
cudaError_t bm_launch_adjoint_substep(const World &w, const void *work, const double fbar[3], int n_p,
                                      int n_node, cudaStream_t st);
cudaError_t bm_launch_adjoint_io(const World &w, const void *work, int field, float *buf, int to_work,
                                 int n_p, cudaStream_t st);
cudaError_t bm_launch_substep(const World &w, const LaunchSet &ls, cudaStream_t st);
cudaError_t bm_launch_substep_ev(const World &w, const LaunchSet &ls, cudaStream_t st, cudaEvent_t *ev);
cudaError_t bm_launch_prepare(const World &w, const LaunchSet &ls, cudaStream_t st);
cudaError_t bm_launch_rebuild(const World &w, const LaunchSet &ls, cudaStream_t st, int force);
cudaError_t bm_launch_io(const World &w, int scene_slot, int p_begin, int n, int field, void *buf,
                         int to_device_pool, cudaStream_t st);
cudaError_t bm_launch_code(const World &w, int p_begin, int n, int64_t *out, cudaStream_t st);
