// Host runtime of the GB300 TLMPM cutting library: scene construction (the
// fixed reference stencil table of Eq. 1), packed multi-scene worlds with a
// first-fit range allocator, CUDA-graph capture of batched substeps, state
// I/O, and the C ABI declared in include/blademaster.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "bm_internal.cuh"

// kernels used only here (bm_kernels.cu)
cudaError_t bm_launch_set_tools(const World &w, const int *scene_ids, int n, const double *states,
                                cudaStream_t st);
cudaError_t bm_launch_get_wrenches(const World &w, const int *scene_ids, int n, double *out,
                                   cudaStream_t st);

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

#define CK(call)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(BM_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));          \
  } while (0)

struct Allocator {
  bm_alloc a{};
  bool has = false;
  cudaStream_t st = nullptr;
  void *alloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    if (has) return a.alloc(bytes, (void *)st, a.ctx);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void release(void *p) {
    if (!p) return;
    if (has) a.free(p, (void *)st, a.ctx);
    else cudaFree(p);
  }
};

// first-fit allocator of index ranges inside a pool
struct RangeAlloc {
  int64_t cap = 0;
  std::vector<std::pair<int64_t, int64_t>> fr;  // (begin, length), sorted by begin
  void init(int64_t c) {
    cap = c;
    fr.clear();
    if (c > 0) fr.push_back({0, c});
  }
  int64_t take(int64_t n) {
    if (n <= 0) return 0;
    for (size_t i = 0; i < fr.size(); ++i)
      if (fr[i].second >= n) {
        int64_t b = fr[i].first;
        fr[i].first += n;
        fr[i].second -= n;
        if (fr[i].second == 0) fr.erase(fr.begin() + (long)i);
        return b;
      }
    return -1;
  }
  void give(int64_t b, int64_t n) {
    if (n <= 0) return;
    auto it = std::lower_bound(fr.begin(), fr.end(), std::make_pair(b, (int64_t)0));
    it = fr.insert(it, {b, n});
    size_t i = (size_t)(it - fr.begin());
    if (i + 1 < fr.size() && fr[i].first + fr[i].second == fr[i + 1].first) {
      fr[i].second += fr[i + 1].second;
      fr.erase(fr.begin() + (long)i + 1);
    }
    if (i > 0 && fr[i - 1].first + fr[i - 1].second == fr[i].first) {
      fr[i - 1].second += fr[i].second;
      fr.erase(fr.begin() + (long)i);
    }
  }
};

}  // namespace

struct WorldH;

struct bm_scene_s {
  bm_scene_desc desc{};
  bm_blade_desc blade{};
  bool has_blade = false;
  int64_t n = 0;
  std::vector<float> X;               // caller order, [n][3]
  std::vector<int> cell_start_rel;    // n_cell + 1, relative to the scene's first particle
  int nb[3] = {0, 0, 0}, nn[3] = {0, 0, 0}, lo[3] = {0, 0, 0}, nbr[3] = {0, 0, 0};
  int64_t n_cell = 0, n_node = 0, n_brick = 0, slot_cap = 0, hist_cap = 0, ppool_cap = 0;
  int ppc_max = 0;                    // most particles in one base cell
  WorldH *world = nullptr;
  bool own_world = false;
  int slot = -1;
  int64_t p_begin = 0, cell_begin = 0, node_begin = 0, slot_begin = 0, hist_begin = 0, brick_begin = 0,
          ppool_begin = 0;
  int ntile_begin = 0, n_ntile = 0;
  DevScene tmpl{};                    // static fields (host template)
  // staged fresh state, uploaded when the scene first enters a world
  std::vector<float> h_fx[3];
  std::vector<uint32_t> h_base;
  std::vector<int> h_perm;
  bool fresh = true;
  cudaStream_t home_stream = nullptr;  // stream and allocator given at creation
  bm_alloc home_alloc{};
  bool has_home_alloc = false;
};

struct WorldH {
  Allocator al;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int device = -1;          // device current when the world was created (its memory and stream live there)
  int64_t cap_p = 0, cap_cell = 0, cap_node = 0, cap_slot = 0, cap_hist = 0, cap_brick = 0, cap_ppool = 0;
  int cap_scenes = 0, cap_ntile = 0;
  bool pair = false;
  World w{};
  std::vector<void *> allocs;
  RangeAlloc rp, rcell, rnode, rslot, rhist, rbrick, rppool;
  std::vector<int> free_slots;
  int4 *d_btiles = nullptr, *d_ntiles = nullptr;
  int *d_scene_ids = nullptr, *d_slot_ids = nullptr;
  double *d_stage = nullptr;
  int ntile_size = 128;
  int variant = 0;          // brick-kernel occupancy variant
  int graph_chunk = 16;
  std::vector<bm_scene_s *> members;
  bool tiles_dirty = true;
  int n_btiles = 0, n_ntiles = 0;
  std::map<int, cudaGraphExec_t> graphs;

  template <class T>
  T *get(int64_t count) {
    void *p = al.alloc(sizeof(T) * (size_t)std::max<int64_t>(count, 1));
    if (p) allocs.push_back(p);
    return (T *)p;
  }
  void drop_graphs() {
    for (auto &kv : graphs) cudaGraphExecDestroy(kv.second);
    graphs.clear();
  }
  ~WorldH() {
    drop_graphs();
    if (st) cudaStreamSynchronize(st);
    for (void *p : allocs) al.release(p);
    if (own_stream && st) cudaStreamDestroy(st);
  }
};

struct bm_batch_s {
  WorldH *world = nullptr;
};

namespace {

// A contact-candidate entry moved from pool range [from, ...) to [to, ...):
// the pool index (bits 0-30) is rebased, the shared-stencil flag (bit 31) is
// kept.  Entries beyond a particle's count are never read.
int rebase_candidate(int e, int from, int to) {
  const uint32_t u = (uint32_t)e;
  const uint32_t q = ((u & 0x7fffffffu) - (uint32_t)from + (uint32_t)to) & 0x7fffffffu;
  return (int)((u & 0x80000000u) | q);
}

int world_alloc(WorldH *W) {
  const int64_t P = W->cap_p;
  PPool &pp = W->w.P;
  bool ok = true;
  auto F = [&](float *&ptr, int64_t c) {
    ptr = W->get<float>(c);
    ok &= ptr != nullptr;
  };
  auto U = [&](uint32_t *&ptr, int64_t c) {
    ptr = W->get<uint32_t>(c);
    ok &= ptr != nullptr;
  };
  auto I = [&](int *&ptr, int64_t c) {
    ptr = W->get<int>(c);
    ok &= ptr != nullptr;
  };
  cudaError_t ie = bm_kernels_init();
  if (ie != cudaSuccess) return fail(BM_E_CUDA, std::string("kernel set-up: ") + cudaGetErrorString(ie));
  for (int a = 0; a < 3; ++a) {
    F(pp.fx[a], P);
    F(pp.x[a], P);
    F(pp.v[a], P);
    F(pp.ut[a], P);
    F(pp.J[a], P);
  }
  for (int k = 0; k < 9; ++k) {
    F(pp.F[k], P);
    F(pp.Fpi[k], P);
    F(pp.Fdot[k], P);
  }
  F(pp.D, P);
  pp.tflag = W->get<uint8_t>(P);
  ok &= pp.tflag != nullptr;
  U(pp.base, P);
  U(pp.s1, P);
  U(pp.s2, P);
  I(pp.perm, P);
  pp.pend = W->get<uint8_t>(P);
  ok &= pp.pend != nullptr;
  if (W->pair) {
    I(pp.hkey, P);
    I(pp.horder, P);
    pp.hent = W->get<float4>(P);
    ok &= pp.hent != nullptr;
    U(pp.hbase, P);
    pp.hcell = W->get<unsigned long long>(P);
    pp.hentk = W->get<unsigned long long>(P);
    ok &= pp.hcell && pp.hentk;
    for (int b = 0; b < 2; ++b) {
      I(pp.hist_partner[b], P * BM_HIST);
      F(pp.hist_u[b], P * BM_HIST * 3);
    }
    I(pp.nbr, P * BM_NBR);
    pp.nbr_n = W->get<uint8_t>(P);
    ok &= pp.nbr_n != nullptr;
    for (int a = 0; a < 3; ++a) F(pp.xb[a], P);
    int nb = 1024;
    while (nb < 2 * P && nb < (1 << 28)) nb <<= 1;
    HashPool &H = W->w.H;
    H.n_buckets = nb;
    I(H.bucket_start, (int64_t)nb + 1);
    I(H.bucket_fill, nb);
    I(H.block_sum, nb / 1024 + 1);
    I(H.build, 1);
  }
  NPool &np = W->w.N;
  I(np.cell_start, W->cap_cell);
  I(np.slot_off, W->cap_node);
  np.slot_cnt = W->get<uint8_t>(W->cap_node);
  np.ncodes = W->get<uint8_t>(W->cap_node);
  np.dirty = W->get<uint8_t>(W->cap_node);
  ok &= np.slot_cnt && np.ncodes && np.dirty;
  np.tmp_codes = W->get<uint2>(W->cap_node * BM_MAXS);
  ok &= np.tmp_codes != nullptr;
  I(np.tile_sum, W->cap_ntile);
  SPool &sp = W->w.S;
  sp.vold = W->get<float4>(W->cap_slot);
  sp.vnew = W->get<float4>(W->cap_slot);
  sp.vstar = W->get<float4>(W->cap_slot);
  sp.code = W->get<uint2>(W->cap_slot);
  ok &= sp.vold && sp.vnew && sp.vstar && sp.code;
  BPool &bp = W->w.B;
  bp.pm = W->get<float4>(W->cap_ppool);
  bp.pd = W->get<float4>(W->cap_ppool);
  bp.poff = W->get<int>(W->cap_brick);
  bp.ptot = W->get<int>(W->cap_brick);
  bp.tdesc = W->get<int>(W->cap_brick * BM_TILE_NODES);
  bp.tgoff = W->get<int>(W->cap_brick * BM_TILE_NODES);
  ok &= bp.pm && bp.pd && bp.poff && bp.ptot && bp.tdesc && bp.tgoff;
  W->w.scenes = W->get<DevScene>(W->cap_scenes);
  W->w.wpart = W->get<double>(W->cap_brick * 6);
  W->w.whist = W->get<double>(std::max<int64_t>(W->cap_hist, 1) * 6);
  W->d_btiles = W->get<int4>(W->cap_brick);
  W->d_ntiles = W->get<int4>(W->cap_ntile);
  W->d_scene_ids = W->get<int>(W->cap_scenes);
  W->d_slot_ids = W->get<int>(W->cap_scenes);
  W->d_stage = W->get<double>((int64_t)W->cap_scenes * 18);
  ok &= W->w.scenes && W->w.wpart && W->w.whist && W->d_btiles && W->d_ntiles && W->d_scene_ids &&
        W->d_slot_ids && W->d_stage;
  if (!ok) return fail(BM_E_OOM, "device allocation failed");
  W->rp.init(W->cap_p);
  W->rcell.init(W->cap_cell);
  W->rnode.init(W->cap_node);
  W->rslot.init(W->cap_slot);
  W->rhist.init(W->cap_hist);
  W->rbrick.init(W->cap_brick);
  W->rppool.init(W->cap_ppool);
  W->free_slots.clear();
  for (int i = W->cap_scenes - 1; i >= 0; --i) W->free_slots.push_back(i);
  std::vector<int> ids(W->cap_scenes);
  for (int i = 0; i < W->cap_scenes; ++i) ids[i] = i;
  CK(cudaMemcpy(W->d_slot_ids, ids.data(), sizeof(int) * ids.size(), cudaMemcpyHostToDevice));
  CK(cudaMemset(W->w.wpart, 0, sizeof(double) * (size_t)W->cap_brick * 6));
  return BM_OK;
}

int64_t tiles_for(int64_t n, int tile) { return (n + tile - 1) / tile; }

// assign tile ranges to every member, upload the tile lists and the ranges
int rebuild_tiles(WorldH *W) {
  std::vector<int4> bt, nt;
  std::vector<int> ids;
  for (bm_scene_s *s : W->members) {
    for (int64_t b = 0; b < s->n_brick; ++b) {
      const int first = s->cell_start_rel[(size_t)b * BM_BRICK_CELLS];
      const int last = s->cell_start_rel[(size_t)(b + 1) * BM_BRICK_CELLS];
      bt.push_back(make_int4(s->slot, (int)(s->brick_begin + b), (int)(s->p_begin + first), last - first));
    }
    s->ntile_begin = (int)nt.size();
    for (int64_t b = 0; b < s->n_node; b += W->ntile_size) {
      int c = (int)std::min<int64_t>(W->ntile_size, s->n_node - b);
      nt.push_back(make_int4(s->slot, (int)(s->node_begin + b), c, (int)nt.size()));
    }
    s->n_ntile = (int)nt.size() - s->ntile_begin;
    ids.push_back(s->slot);
  }
  if ((int64_t)bt.size() > W->cap_brick || (int64_t)nt.size() > W->cap_ntile)
    return fail(BM_E_CAPACITY, "tile lists exceed the batch capacity");
  if (!bt.empty()) CK(cudaMemcpy(W->d_btiles, bt.data(), sizeof(int4) * bt.size(), cudaMemcpyHostToDevice));
  if (!nt.empty()) CK(cudaMemcpy(W->d_ntiles, nt.data(), sizeof(int4) * nt.size(), cudaMemcpyHostToDevice));
  if (!ids.empty()) CK(cudaMemcpy(W->d_scene_ids, ids.data(), sizeof(int) * ids.size(), cudaMemcpyHostToDevice));
  for (bm_scene_s *s : W->members) {
    int r[2] = {s->ntile_begin, s->n_ntile};
    CK(cudaMemcpy((char *)(W->w.scenes + s->slot) + offsetof(DevScene, ntile_begin), r, sizeof r,
                  cudaMemcpyHostToDevice));
  }
  W->n_btiles = (int)bt.size();
  W->n_ntiles = (int)nt.size();
  W->tiles_dirty = false;
  W->drop_graphs();
  return BM_OK;
}

// brick tiles of one scene inside the world's list (scenes are listed in order)
int scene_btile_begin(const WorldH *W, const bm_scene_s *s) {
  int b = 0;
  for (const bm_scene_s *m : W->members) {
    if (m == s) return b;
    b += (int)m->n_brick;
  }
  return -1;
}

LaunchSet scene_set(const WorldH *W, const bm_scene_s *s) {
  LaunchSet ls{};
  ls.btiles = W->d_btiles + scene_btile_begin(W, s);
  ls.n_btiles = (int)s->n_brick;
  ls.ppc16 = s->ppc_max > 8;
  ls.ntiles = W->d_ntiles + s->ntile_begin;
  ls.n_ntiles = s->n_ntile;
  ls.ntile_size = W->ntile_size;
  ls.variant = W->variant;
  ls.scene_ids = W->d_slot_ids + s->slot;
  ls.n_scenes = 1;
  ls.any_pair = s->desc.pair_contact;
  ls.any_inelastic = s->desc.yield_stress > 0 || s->desc.viscosity > 0;
  return ls;
}

LaunchSet world_set(const WorldH *W) {
  LaunchSet ls{};
  ls.btiles = W->d_btiles;
  ls.n_btiles = W->n_btiles;
  ls.ntiles = W->d_ntiles;
  ls.n_ntiles = W->n_ntiles;
  ls.ntile_size = W->ntile_size;
  ls.variant = W->variant;
  ls.scene_ids = W->d_scene_ids;
  ls.n_scenes = (int)W->members.size();
  for (auto *s : W->members) {
    ls.any_pair |= s->desc.pair_contact;
    ls.any_inelastic |= s->desc.yield_stress > 0 || s->desc.viscosity > 0;
    ls.ppc16 |= s->ppc_max > 8;
  }
  return ls;
}

void fill_template(bm_scene_s *s) {
  const bm_scene_desc &d = s->desc;
  DevScene &t = s->tmpl;
  std::memset(&t, 0, sizeof t);
  t.stop_at = -1;  // no stop substep: the scene advances with every step call
  t.nb[0] = s->nb[0]; t.nb[1] = s->nb[1]; t.nb[2] = s->nb[2];
  t.nn[0] = s->nn[0]; t.nn[1] = s->nn[1]; t.nn[2] = s->nn[2];
  t.nbr[0] = s->nbr[0]; t.nbr[1] = s->nbr[1]; t.nbr[2] = s->nbr[2];
  t.n_brick = (int)s->n_brick;
  t.n_p = (int)s->n;
  t.n_node = (int)s->n_node;
  t.n_cell = (int)s->n_cell;
  t.slot_cap = (int)s->slot_cap;
  t.hist_cap = (int)s->hist_cap;
  t.dx = (float)d.dx;
  t.inv_dx = (float)(1.0 / d.dx);
  const double mp = d.rho * d.V0;
  t.mp = (float)mp;
  t.V0 = (float)d.V0;
  t.Rp = (float)(d.s_R * std::cbrt(d.V0) / 2.0);
  t.dt = (float)d.dt;
  t.beta = (float)d.beta;
  for (int a = 0; a < 3; ++a) t.g[a] = (float)d.gravity[a];
  t.model = d.model;
  t.yield_stress = (float)d.yield_stress;
  t.viscosity = (float)d.viscosity;
  t.mu = (float)(d.E / (2.0 * (1.0 + d.nu)));
  t.lam = (float)(d.E * d.nu / ((1.0 + d.nu) * (1.0 - 2.0 * d.nu)));
  t.Wth = (float)(d.G_c * std::pow(d.V0, 2.0 / 3.0) * (1.0 - d.zeta) / d.zeta);
  t.u_min = (float)d.u_min;
  t.h_d = d.band_half_width > 0 ? d.band_half_width : 6.0 * d.dx;
  t.b_back_d = d.b_back > 0 ? d.b_back : d.dx;
  t.b_lead_d = d.b_lead > 0 ? d.b_lead : d.dx;
  t.h = (float)t.h_d;
  t.b_back = (float)t.b_back_d;
  t.b_lead = (float)t.b_lead_d;
  t.dt_d = d.dt;
  t.s_n = (float)d.s_n;
  t.gamma_k = (float)d.gamma_k;
  t.gamma_c = (float)d.gamma_c;
  t.pair_mu_s = (float)d.pair_mu_s;
  t.pair_mu_d = (float)d.pair_mu_d;
  t.floor_z = (float)d.floor_z;
  t.pair_h = (float)(3.0 * d.s_R * std::cbrt(d.V0) / 2.0);  // 2 R_p plus an R_p margin
  t.pair_inv_h = (float)(1.0 / (3.0 * d.s_R * std::cbrt(d.V0) / 2.0));
  t.floor_on = d.floor_enabled;
  t.pair_on = d.pair_contact;
  t.tool_contact_on = d.tool_contact;
  for (int a = 0; a < 3; ++a) t.origin_d[a] = d.origin[a];
  t.cur_cut = -1;
  t.cut = -1;
  t.R[0] = t.R[4] = t.R[8] = 1.0;
  if (s->has_blade) {
    const bm_blade_desc &b = s->blade;
    t.has_blade = 1;
    for (int a = 0; a < 3; ++a) {
      t.edgeT[a] = b.edge_point[a];
      t.nT[a] = b.normal[a];
      t.eT[a] = b.edge_dir[a];
      t.dT[a] = b.front_dir[a];
      t.xB[a] = b.pose_x[a];
    }
    for (int k = 0; k < 9; ++k) t.R[k] = b.pose_R[k];
    t.half_len = b.half_length;
    t.L_d = b.half_length;
    t.half_thick = 0.5 * b.thickness;
    t.half_height = 0.5 * b.height;
    t.mu_s = b.mu_s;
    t.mu_d = b.mu_d;
    t.mass = b.mass > 0 ? b.mass : 0.0;
    if (t.mass > 0) {
      const double *A = b.inertia;
      double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                   A[2] * (A[3] * A[7] - A[4] * A[6]);
      t.Ib_inv[0] = (A[4] * A[8] - A[5] * A[7]) / det;
      t.Ib_inv[1] = (A[2] * A[7] - A[1] * A[8]) / det;
      t.Ib_inv[2] = (A[1] * A[5] - A[2] * A[4]) / det;
      t.Ib_inv[3] = (A[5] * A[6] - A[3] * A[8]) / det;
      t.Ib_inv[4] = (A[0] * A[8] - A[2] * A[6]) / det;
      t.Ib_inv[5] = (A[2] * A[3] - A[0] * A[5]) / det;
      t.Ib_inv[6] = (A[3] * A[7] - A[4] * A[6]) / det;
      t.Ib_inv[7] = (A[1] * A[6] - A[0] * A[7]) / det;
      t.Ib_inv[8] = (A[0] * A[4] - A[1] * A[3]) / det;
    }
    t.kv = b.servo_gain > 0 ? b.servo_gain : 1.0 / (10.0 * d.dt);
    t.rigid_interval = b.rigid_interval >= 1 ? b.rigid_interval : 1;
    t.nseg = b.n_segments;
    for (int i = 0; i < b.n_segments; ++i) {
      t.seg[i].n_steps = b.segments[i].n_steps;
      t.seg[i].cut_id = b.segments[i].cut_id;
      for (int a = 0; a < 3; ++a) {
        t.seg[i].v[a] = b.segments[i].v[a];
        t.seg[i].w[a] = b.segments[i].omega[a];
      }
    }
  }
}

// copy the fields of a DevScene that describe where it lives
void set_ranges(const bm_scene_s *s, DevScene &t) {
  t.p_begin = (int)s->p_begin;
  t.node_begin = (int)s->node_begin;
  t.cell_begin = (int)s->cell_begin;
  t.slot_begin = (int)s->slot_begin;
  t.hist_begin = (int)s->hist_begin;
  t.brick_begin = (int)s->brick_begin;
  t.n_brick = (int)s->n_brick;
  t.ppool_begin = (int)s->ppool_begin;
  t.ppool_cap = (int)s->ppool_cap;
  t.ntile_begin = s->ntile_begin;
  t.n_ntile = s->n_ntile;
}

// reserve ranges for s inside W; returns BM_OK or BM_E_CAPACITY
int reserve(WorldH *W, bm_scene_s *s) {
  if (W->free_slots.empty()) return fail(BM_E_CAPACITY, "no free scene slot");
  if (s->desc.pair_contact && !W->pair) return fail(BM_E_CAPACITY, "batch has no pair-contact pools");
  int64_t pb = W->rp.take(s->n);
  int64_t cb = W->rcell.take(s->n_cell + 1);
  int64_t nb = W->rnode.take(s->n_node);
  int64_t sb = W->rslot.take(s->slot_cap);
  int64_t hb = W->rhist.take(s->hist_cap);
  int64_t bb = W->rbrick.take(s->n_brick);
  int64_t qb = W->rppool.take(s->ppool_cap);
  if (pb < 0 || cb < 0 || nb < 0 || sb < 0 || hb < 0 || bb < 0 || qb < 0) {
    if (bb >= 0) W->rbrick.give(bb, s->n_brick);
    if (qb >= 0) W->rppool.give(qb, s->ppool_cap);
    if (pb >= 0) W->rp.give(pb, s->n);
    if (cb >= 0) W->rcell.give(cb, s->n_cell + 1);
    if (nb >= 0) W->rnode.give(nb, s->n_node);
    if (sb >= 0) W->rslot.give(sb, s->slot_cap);
    if (hb >= 0) W->rhist.give(hb, s->hist_cap);
    return fail(BM_E_CAPACITY, "batch pools have no room for the scene");
  }
  s->slot = W->free_slots.back();
  W->free_slots.pop_back();
  s->p_begin = pb;
  s->cell_begin = cb;
  s->node_begin = nb;
  s->slot_begin = sb;
  s->hist_begin = hb;
  s->brick_begin = bb;
  s->ppool_begin = qb;
  return BM_OK;
}

void unreserve(WorldH *W, bm_scene_s *s) {
  W->rp.give(s->p_begin, s->n);
  W->rcell.give(s->cell_begin, s->n_cell + 1);
  W->rnode.give(s->node_begin, s->n_node);
  W->rslot.give(s->slot_cap ? s->slot_begin : 0, s->slot_cap);
  W->rhist.give(s->hist_begin, s->hist_cap);
  W->rbrick.give(s->brick_begin, s->n_brick);
  W->rppool.give(s->ppool_begin, s->ppool_cap);
  W->free_slots.push_back(s->slot);
  s->slot = -1;
}

int upload_cell_start(WorldH *W, bm_scene_s *s) {
  std::vector<int> cs(s->cell_start_rel.size());
  for (size_t i = 0; i < cs.size(); ++i) cs[i] = s->cell_start_rel[i] + (int)s->p_begin;
  CK(cudaMemcpyAsync(W->w.N.cell_start + s->cell_begin, cs.data(), sizeof(int) * cs.size(),
                     cudaMemcpyHostToDevice, W->st));
  CK(cudaStreamSynchronize(W->st));
  return BM_OK;
}

// first placement of a freshly created scene
int place_fresh(WorldH *W, bm_scene_s *s) {
  int rc = reserve(W, s);
  if (rc) return rc;
  const int64_t n = s->n, pb = s->p_begin;
  PPool &P = W->w.P;
  cudaStream_t st = W->st;
  std::vector<float> x3[3];
  for (int a = 0; a < 3; ++a) {
    x3[a].resize(n);
    for (int64_t i = 0; i < n; ++i) x3[a][i] = s->X[3 * (size_t)s->h_perm[i] + a];
  }
  for (int a = 0; a < 3; ++a) {
    CK(cudaMemcpyAsync(P.fx[a] + pb, s->h_fx[a].data(), sizeof(float) * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(P.x[a] + pb, x3[a].data(), sizeof(float) * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(P.v[a] + pb, 0, sizeof(float) * n, st));
    CK(cudaMemsetAsync(P.ut[a] + pb, 0, sizeof(float) * n, st));
  }
  std::vector<float> one((size_t)n, 1.0f);
  for (int k = 0; k < 9; ++k) {
    if (k % 4 == 0) {
      CK(cudaMemcpyAsync(P.F[k] + pb, one.data(), sizeof(float) * n, cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(P.Fpi[k] + pb, one.data(), sizeof(float) * n, cudaMemcpyHostToDevice, st));
    } else {
      CK(cudaMemsetAsync(P.F[k] + pb, 0, sizeof(float) * n, st));
      CK(cudaMemsetAsync(P.Fpi[k] + pb, 0, sizeof(float) * n, st));
    }
    CK(cudaMemsetAsync(P.Fdot[k] + pb, 0, sizeof(float) * n, st));
  }
  CK(cudaMemsetAsync(P.D + pb, 0, sizeof(float) * n, st));
  CK(cudaMemsetAsync(P.tflag + pb, 0, n, st));
  CK(cudaMemsetAsync(P.pend + pb, 0, n, st));
  for (int a = 0; a < 3; ++a) CK(cudaMemsetAsync(P.J[a] + pb, 0, sizeof(float) * n, st));
  CK(cudaMemsetAsync(P.s1 + pb, 0, sizeof(uint32_t) * n, st));
  CK(cudaMemsetAsync(P.s2 + pb, 0, sizeof(uint32_t) * n, st));
  CK(cudaMemcpyAsync(P.base + pb, s->h_base.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(P.perm + pb, s->h_perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
  if (W->pair) {
    for (int b = 0; b < 2; ++b)
      CK(cudaMemsetAsync(P.hist_partner[b] + pb * BM_HIST, 0xff, sizeof(int) * n * BM_HIST, st));
  }
  if (s->hist_cap) CK(cudaMemsetAsync(W->w.whist + s->hist_begin * 6, 0, sizeof(double) * 6 * s->hist_cap, st));
  int r = upload_cell_start(W, s);
  if (r) return r;
  DevScene t = s->tmpl;
  set_ranges(s, t);
  CK(cudaMemcpyAsync(W->w.scenes + s->slot, &t, sizeof t, cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  W->members.push_back(s);
  s->world = W;
  s->fresh = false;
  s->h_fx[0].clear(); s->h_fx[1].clear(); s->h_fx[2].clear();
  s->h_base.clear();
  return BM_OK;
}

int finish_placement(WorldH *W, bm_scene_s *s) {
  int r = rebuild_tiles(W);
  if (r) return r;
  LaunchSet ls = scene_set(W, s);
  CK(bm_launch_rebuild(W->w, ls, W->st, 1));
  CK(bm_launch_prepare(W->w, ls, W->st));
  CK(cudaStreamSynchronize(W->st));
  return BM_OK;
}

WorldH *new_world(const bm_alloc *alloc, cudaStream_t st) {
  WorldH *W = new WorldH();
  if (alloc && alloc->alloc && alloc->free) {
    W->al.a = *alloc;
    W->al.has = true;
  }
  W->al.st = st;
  W->st = st;
  if (cudaGetDevice(&W->device) != cudaSuccess) {
    cudaGetLastError();
    W->device = -1;
  }
  return W;
}

// move s from its world into W (device-to-device copies of the persistent state)
int move_scene(bm_scene_s *s, WorldH *W) {
  WorldH *S = s->world;
  CK(cudaStreamSynchronize(S->st));
  DevScene cur;
  CK(cudaMemcpy(&cur, S->w.scenes + s->slot, sizeof cur, cudaMemcpyDeviceToHost));
  bm_scene_s old = *s;  // ranges in S
  int rc = reserve(W, s);
  if (rc) return rc;
  const int64_t n = s->n;
  const PPool &A = S->w.P;
  PPool &B = W->w.P;
  const int64_t ps = old.p_begin, pd = s->p_begin;
  cudaStream_t st = W->st;
  auto cp = [&](void *dst, const void *src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st);
  };
  for (int a = 0; a < 3; ++a) {
    CK(cp(B.fx[a] + pd, A.fx[a] + ps, sizeof(float) * n));
    CK(cp(B.x[a] + pd, A.x[a] + ps, sizeof(float) * n));
    CK(cp(B.v[a] + pd, A.v[a] + ps, sizeof(float) * n));
    CK(cp(B.ut[a] + pd, A.ut[a] + ps, sizeof(float) * n));
  }
  for (int k = 0; k < 9; ++k) {
    CK(cp(B.F[k] + pd, A.F[k] + ps, sizeof(float) * n));
    CK(cp(B.Fpi[k] + pd, A.Fpi[k] + ps, sizeof(float) * n));
    CK(cp(B.Fdot[k] + pd, A.Fdot[k] + ps, sizeof(float) * n));
  }
  CK(cp(B.D + pd, A.D + ps, sizeof(float) * n));
  CK(cp(B.tflag + pd, A.tflag + ps, n));
  CK(cp(B.base + pd, A.base + ps, sizeof(uint32_t) * n));
  CK(cp(B.s1 + pd, A.s1 + ps, sizeof(uint32_t) * n));
  CK(cp(B.s2 + pd, A.s2 + ps, sizeof(uint32_t) * n));
  CK(cp(B.perm + pd, A.perm + ps, sizeof(int) * n));
  CK(cudaMemsetAsync(B.pend + pd, 0, n, st));
  for (int a = 0; a < 3; ++a) CK(cudaMemsetAsync(B.J[a] + pd, 0, sizeof(float) * n, st));
  if (W->pair) {
    for (int b = 0; b < 2; ++b) {
      if (S->pair) {
        CK(cp(B.hist_partner[b] + pd * BM_HIST, A.hist_partner[b] + ps * BM_HIST, sizeof(int) * n * BM_HIST));
        CK(cp(B.hist_u[b] + pd * BM_HIST * 3, A.hist_u[b] + ps * BM_HIST * 3, sizeof(float) * n * BM_HIST * 3));
      } else {
        CK(cudaMemsetAsync(B.hist_partner[b] + pd * BM_HIST, 0xff, sizeof(int) * n * BM_HIST, st));
      }
    }
    if (S->pair) {  // the contact candidate lists move along (rebased below)
      CK(cp(B.nbr + pd * BM_NBR, A.nbr + ps * BM_NBR, sizeof(int) * n * BM_NBR));
      CK(cp(B.nbr_n + pd, A.nbr_n + ps, n));
      for (int a = 0; a < 3; ++a) CK(cp(B.xb[a] + pd, A.xb[a] + ps, sizeof(float) * n));
    }
  }
  if (s->hist_cap) CK(cp(W->w.whist + s->hist_begin * 6, S->w.whist + old.hist_begin * 6, sizeof(double) * 6 * s->hist_cap));
  CK(cudaStreamSynchronize(st));
  int r = upload_cell_start(W, s);
  if (r) return r;
  // partner indices of the pair history and the contact candidates are pool
  // indices: rebase them
  if (W->pair && S->pair && pd != ps) {
    std::vector<int> h((size_t)n * BM_HIST);
    for (int b = 0; b < 2; ++b) {
      CK(cudaMemcpy(h.data(), B.hist_partner[b] + pd * BM_HIST, sizeof(int) * h.size(), cudaMemcpyDeviceToHost));
      for (auto &q : h)
        if (q >= 0) q = q - (int)ps + (int)pd;
      CK(cudaMemcpy(B.hist_partner[b] + pd * BM_HIST, h.data(), sizeof(int) * h.size(), cudaMemcpyHostToDevice));
    }
    std::vector<int> nb((size_t)n * BM_NBR);
    CK(cudaMemcpy(nb.data(), B.nbr + pd * BM_NBR, sizeof(int) * nb.size(), cudaMemcpyDeviceToHost));
    for (auto &q : nb) q = rebase_candidate(q, (int)ps, (int)pd);
    CK(cudaMemcpy(B.nbr + pd * BM_NBR, nb.data(), sizeof(int) * nb.size(), cudaMemcpyHostToDevice));
  }
  set_ranges(s, cur);
  cur.slot_cap = (int)s->slot_cap;
  cur.label_pending = 0;
  if (!(W->pair && S->pair)) cur.pair_valid = 0;  // no lists came along: build them on the next substep
  CK(cudaMemcpy(W->w.scenes + s->slot, &cur, sizeof cur, cudaMemcpyHostToDevice));
  // leave the old world
  auto &mem = S->members;
  mem.erase(std::remove(mem.begin(), mem.end(), s), mem.end());
  {
    bm_scene_s tmp = old;
    unreserve(S, &tmp);
  }
  S->tiles_dirty = true;
  bool drop_old = s->own_world;
  W->members.push_back(s);
  s->world = W;
  s->own_world = false;
  if (drop_old) delete S;
  else if (!S->members.empty()) {
    int r2 = rebuild_tiles(S);
    if (r2) return r2;
  }
  return finish_placement(W, s);
}

int create_private_world(bm_scene_s *s, const bm_alloc *alloc, cudaStream_t st) {
  WorldH *W = new_world(alloc, st);
  W->cap_p = s->n;
  W->cap_cell = s->n_cell + 1;
  W->cap_node = s->n_node;
  W->cap_slot = s->slot_cap;
  W->cap_hist = s->hist_cap;
  W->cap_scenes = 1;
  W->cap_brick = s->n_brick;
  W->cap_ppool = s->ppool_cap;
  W->cap_ntile = (int)tiles_for(s->n_node, 64) + 1;
  W->pair = s->desc.pair_contact != 0;
  int rc = world_alloc(W);
  if (rc) {
    delete W;
    return rc;
  }
  rc = s->fresh ? place_fresh(W, s) : move_scene(s, W);
  if (rc) return rc;
  s->own_world = true;
  return BM_OK;
}

int validate_desc(const bm_scene_desc *d) {
  if (!d) return fail(BM_E_INVALID, "null scene descriptor");
  if (!(d->dx > 0) || !(d->V0 > 0) || !(d->dt > 0) || !(d->rho > 0) || !(d->E > 0))
    return fail(BM_E_INVALID, "dx, V0, dt, rho and E must be positive");
  if (!(d->nu > -1.0 && d->nu < 0.5)) return fail(BM_E_INVALID, "nu must lie in (-1, 0.5)");
  if (!(d->beta >= 0 && d->beta <= 1)) return fail(BM_E_INVALID, "beta must lie in [0, 1]");
  if (!(d->zeta > 0 && d->zeta < 1)) return fail(BM_E_INVALID, "zeta must lie in (0, 1)");
  if (d->model != BM_MODEL_NEO_HOOKEAN && d->model != BM_MODEL_FIXED_COROTATED)
    return fail(BM_E_INVALID, "unknown elastic model");
  if (!(d->yield_stress >= 0) || !(d->viscosity >= 0))
    return fail(BM_E_INVALID, "yield stress and viscosity must be >= 0");
  return BM_OK;
}

// stencil table: base cell, fractional offset, sort by base cell (Eq. 1)
int build_layout(bm_scene_s *s) {
  const int64_t n = s->n;
  const bm_scene_desc &d = s->desc;
  std::vector<int> b3((size_t)n * 3);
  std::vector<double> f3((size_t)n * 3);
  int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) {
      double xl = ((double)s->X[3 * i + a] - d.origin[a]) / d.dx;
      double fb = std::floor(xl - 0.5);
      if (!std::isfinite(fb) || std::fabs(fb) > 1e8) return fail(BM_E_INVALID, "particle outside the grid range");
      int b = (int)fb;
      b3[3 * i + a] = b;
      f3[3 * i + a] = xl - (double)b;
      lo[a] = std::min(lo[a], b);
      hi[a] = std::max(hi[a], b);
    }
  for (int a = 0; a < 3; ++a) {
    s->lo[a] = lo[a];
    s->nb[a] = hi[a] - lo[a] + 1;
    s->nn[a] = s->nb[a] + 2;
    s->nbr[a] = (s->nb[a] + 3) / 4;
    if (s->nb[a] > 1020) return fail(BM_E_INVALID, "more than 1020 reference cells along an axis");
  }
  // cells are numbered brick-major (bricks of 4x4x4, x-fastest inside), so
  // each brick's particles are one contiguous range
  s->n_brick = (int64_t)s->nbr[0] * s->nbr[1] * s->nbr[2];
  s->n_cell = s->n_brick * BM_BRICK_CELLS;
  s->n_node = (int64_t)s->nn[0] * s->nn[1] * s->nn[2];
  if (s->n_node > (int64_t)1 << 30 || n > (int64_t)1 << 30) return fail(BM_E_INVALID, "scene too large");
  std::vector<int64_t> key((size_t)n);
  std::vector<int> cnt((size_t)s->n_cell + 1, 0);
  for (int64_t i = 0; i < n; ++i) {
    int bx = b3[3 * i] - lo[0], by = b3[3 * i + 1] - lo[1], bz = b3[3 * i + 2] - lo[2];
    int64_t brick = ((int64_t)(bz >> 2) * s->nbr[1] + (by >> 2)) * s->nbr[0] + (bx >> 2);
    key[i] = brick * BM_BRICK_CELLS + (((bz & 3) * 4 + (by & 3)) * 4 + (bx & 3));
    cnt[key[i] + 1]++;
  }
  s->ppc_max = 0;
  for (int64_t c = 0; c < s->n_cell; ++c) s->ppc_max = std::max(s->ppc_max, cnt[c + 1]);
  if (s->ppc_max > 16) return fail(BM_E_INVALID, "more than 16 particles share one reference base cell");
  for (int64_t c = 0; c < s->n_cell; ++c) cnt[c + 1] += cnt[c];
  s->cell_start_rel = cnt;
  std::vector<int> fill((size_t)s->n_cell, 0);
  s->h_perm.assign((size_t)n, 0);
  for (int64_t i = 0; i < n; ++i) s->h_perm[cnt[key[i]] + fill[key[i]]++] = (int)i;  // stable
  for (int a = 0; a < 3; ++a) s->h_fx[a].resize((size_t)n);
  s->h_base.resize((size_t)n);
  for (int64_t j = 0; j < n; ++j) {
    int64_t i = s->h_perm[j];
    for (int a = 0; a < 3; ++a) s->h_fx[a][j] = (float)f3[3 * i + a];
    uint32_t bx = (uint32_t)(b3[3 * i] - lo[0]), by = (uint32_t)(b3[3 * i + 1] - lo[1]),
             bz = (uint32_t)(b3[3 * i + 2] - lo[2]);
    s->h_base[j] = bx | (by << 10) | (bz << 20);
  }
  s->slot_cap = std::max<int64_t>(4 * s->n_node, 64);
  // brick-tile partial sums: a node appears in <= 8 tiles, ~3.4 on average;
  // 6 entries per node covers ~1.8 logical grids per node on average
  s->ppool_cap = std::max<int64_t>(6 * s->n_node, 4096);
  s->hist_cap = d.wrench_history > 0 ? d.wrench_history : 0;
  return BM_OK;
}

bool valid_scene(bm_scene_t s) { return s && s->world; }

}  // namespace

// ============================================================================
// State read without allocation
//
// bm_read_state() gathers a field into a temporary device buffer it
// allocates per call.  The variant below gathers into a fixed staging array
// that lives in the library's own device memory instead, so it never calls
// cudaMalloc/cudaFree.  The array is a file-scope __device__ symbol: every
// GPU that loads the library reserves BM_NOALLOC_STAGE_BYTES for it until the
// process exits.  In host code the symbol name is only a host-side stand-in,
// so its device address is looked up once per device with
// cudaGetSymbolAddress() (with that device current) and passed to the kernel.
// ============================================================================
#define BM_NOALLOC_STAGE_BYTES (16u << 20)  // one 16 MiB array, reused field by field

static __device__ __align__(256) unsigned char bm_noalloc_stage[BM_NOALLOC_STAGE_BYTES];

namespace {

std::mutex g_stage_mu;
std::vector<void *> g_stage_ptr;  // device ordinal -> device address of the array

// set-up, once per device: resolve the array's device address.  `dev` must
// be the current device (the address is that device's copy of the array).
int stage_address(int dev, void **out) {
  std::lock_guard<std::mutex> lk(g_stage_mu);
  if ((int)g_stage_ptr.size() <= dev) g_stage_ptr.resize((size_t)dev + 1, nullptr);
  if (!g_stage_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, bm_noalloc_stage);
    if (e != cudaSuccess || !p)
      return fail(BM_E_CUDA, std::string("cudaGetSymbolAddress(staging array): ") + cudaGetErrorString(e));
    g_stage_ptr[dev] = p;
  }
  *out = g_stage_ptr[dev];
  return BM_OK;
}

// variant of the state gather kernel: pool order -> caller order, into the
// staging array (every element of the used range is written, so nothing in
// the array needs clearing between calls)
__global__ void k_gather_stage(World w, int p_begin, int n, int field, void *stage) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int p = p_begin + i;
  const int o = w.P.perm[p];
  const PPool &P = w.P;
  float *fb = (float *)stage;
  uint32_t *ub = (uint32_t *)stage;
  switch (field) {
    case 1:
      for (int a = 0; a < 3; ++a) fb[3 * o + a] = P.x[a][p];
      break;
    case 2:
      for (int a = 0; a < 3; ++a) fb[3 * o + a] = P.v[a][p];
      break;
    case 3:
      for (int a = 0; a < 9; ++a) fb[9 * o + a] = P.F[a][p];
      break;
    case 4:
      fb[o] = P.D[p];
      break;
    case 5:
      for (int a = 0; a < 3; ++a) fb[3 * o + a] = P.ut[a][p];
      break;
    case 6: {
      const uint32_t s1 = P.s1[p], s2 = P.s2[p];
      int64_t c = 0, pw = 1;
      for (int k = 0; k < BM_MAX_CUTS; ++k) {
        c += (((s1 >> k) & 1u) ? 1 : (((s2 >> k) & 1u) ? 2 : 0)) * pw;
        pw *= 3;
      }
      ((int64_t *)stage)[o] = c;
      break;
    }
    case 7:
      ub[o] = P.s1[p];
      break;
    case 8:
      ub[o] = P.s2[p];
      break;
  }
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

const char *bm_last_error(void) { return g_err.c_str(); }
const char *bm_version(void) { return "blademaster-gb300 0.1 (sm_103a)"; }

int bm_scene_create(const bm_scene_desc *desc, const float *X_ref, int64_t n, const bm_alloc *alloc,
                    void *stream, bm_scene_t *out) {
  if (!out) return fail(BM_E_INVALID, "null output handle");
  *out = nullptr;
  int rc = validate_desc(desc);
  if (rc) return rc;
  if (n <= 0 || !X_ref) return fail(BM_E_INVALID, "need at least one particle");
  bm_scene_s *s = new bm_scene_s();
  s->desc = *desc;
  s->home_stream = (cudaStream_t)stream;
  if (alloc && alloc->alloc && alloc->free) {
    s->home_alloc = *alloc;
    s->has_home_alloc = true;
  }
  s->n = n;
  s->X.assign(X_ref, X_ref + 3 * n);
  rc = build_layout(s);
  if (rc) {
    delete s;
    return rc;
  }
  fill_template(s);
  rc = create_private_world(s, alloc, (cudaStream_t)stream);
  if (rc) {
    if (s->world) delete s->world;
    delete s;
    return rc;
  }
  rc = finish_placement(s->world, s);
  if (rc) {
    delete s->world;
    delete s;
    return rc;
  }
  *out = s;
  return BM_OK;
}

int bm_add_blade(bm_scene_t s, const bm_blade_desc *b, int *blade_id) {
  if (!valid_scene(s) || !b) return fail(BM_E_INVALID, "bad scene or blade");
  if (s->has_blade) return fail(BM_E_INVALID, "one blade per scene");
  if (b->n_segments < 0 || b->n_segments > BM_MAX_SEGMENTS) return fail(BM_E_INVALID, "too many segments");
  for (int i = 0; i < b->n_segments; ++i) {
    if (b->segments[i].cut_id >= BM_MAX_CUTS || b->segments[i].cut_id < -1)
      return fail(BM_E_TOO_MANY_CUTS, "cut id outside [-1, 32)");
    if (b->segments[i].n_steps < 0) return fail(BM_E_INVALID, "negative segment length");
  }
  WorldH *W = s->world;
  CK(cudaStreamSynchronize(W->st));
  DevScene cur;
  CK(cudaMemcpy(&cur, W->w.scenes + s->slot, sizeof cur, cudaMemcpyDeviceToHost));
  s->blade = *b;
  s->has_blade = true;
  fill_template(s);
  DevScene t = s->tmpl;
  set_ranges(s, t);
  t.step = cur.step;
  t.err = cur.err;
  t.n_slots = cur.n_slots;
  t.need_rebuild = cur.need_rebuild;
  t.stop_at = cur.stop_at;
  t.frozen = cur.frozen;
  CK(cudaMemcpy(W->w.scenes + s->slot, &t, sizeof t, cudaMemcpyHostToDevice));
  LaunchSet ls = scene_set(W, s);
  CK(bm_launch_prepare(W->w, ls, W->st));
  CK(cudaStreamSynchronize(W->st));
  if (blade_id) *blade_id = 0;
  return BM_OK;
}

int bm_set_tool_state(bm_scene_t s, int blade_id, const double pose[12], const double twist[6]) {
  if (!valid_scene(s) || !s->has_blade || blade_id != 0 || !pose || !twist)
    return fail(BM_E_INVALID, "bad scene, blade or arguments");
  WorldH *W = s->world;
  double buf[18];
  std::memcpy(buf, pose, sizeof(double) * 12);
  std::memcpy(buf + 12, twist, sizeof(double) * 6);
  CK(cudaMemcpyAsync((char *)(W->w.scenes + s->slot) + offsetof(DevScene, xB), buf, sizeof buf,
                     cudaMemcpyHostToDevice, W->st));
  CK(bm_launch_prepare(W->w, scene_set(W, s), W->st));
  CK(cudaStreamSynchronize(W->st));
  return BM_OK;
}

int bm_get_tool_state(bm_scene_t s, int blade_id, double pose[12], double twist[6]) {
  if (!valid_scene(s) || !s->has_blade || blade_id != 0) return fail(BM_E_INVALID, "bad scene or blade");
  WorldH *W = s->world;
  CK(cudaStreamSynchronize(W->st));
  double buf[18];
  CK(cudaMemcpy(buf, (char *)(W->w.scenes + s->slot) + offsetof(DevScene, xB), sizeof buf,
                cudaMemcpyDeviceToHost));
  if (pose) std::memcpy(pose, buf, sizeof(double) * 12);
  if (twist) std::memcpy(twist, buf + 12, sizeof(double) * 6);
  return BM_OK;
}

int bm_step(bm_scene_t s, int n_substeps) {
  if (!valid_scene(s) || n_substeps < 0) return fail(BM_E_INVALID, "bad scene or step count");
  WorldH *W = s->world;
  if (W->tiles_dirty) {
    int r = rebuild_tiles(W);
    if (r) return r;
  }
  LaunchSet ls = scene_set(W, s);
  for (int k = 0; k < n_substeps; ++k) CK(bm_launch_substep(W->w, ls, W->st));
  return BM_OK;
}

int bm_scene_set_stop(bm_scene_t s, int64_t stop_at) {
  if (!valid_scene(s) || stop_at < -1) return fail(BM_E_INVALID, "bad scene or stop substep");
  WorldH *W = s->world;
  CK(cudaStreamSynchronize(W->st));
  long long step = 0;
  CK(cudaMemcpy(&step, (char *)(W->w.scenes + s->slot) + offsetof(DevScene, step), sizeof step,
                cudaMemcpyDeviceToHost));
  struct {
    long long stop_at;
    int frozen;
  } v{(long long)stop_at, (stop_at >= 0 && step >= stop_at) ? 1 : 0};
  static_assert(offsetof(DevScene, frozen) == offsetof(DevScene, stop_at) + sizeof(long long),
                "stop_at and frozen are adjacent");
  CK(cudaMemcpy((char *)(W->w.scenes + s->slot) + offsetof(DevScene, stop_at), &v,
                sizeof(long long) + sizeof(int), cudaMemcpyHostToDevice));
  return BM_OK;
}

int bm_read_state(bm_scene_t s, uint32_t field_mask, void *const *dst, int dst_on_device) {
  if (!valid_scene(s) || !dst) return fail(BM_E_INVALID, "bad scene or destination");
  WorldH *W = s->world;
  CK(cudaStreamSynchronize(W->st));
  const int64_t n = s->n;
  int j = 0;
  for (int f = 0; f < BM_NUM_FIELDS; ++f) {
    if (!(field_mask & (1u << f))) continue;
    void *d = dst[j++];
    if (!d) return fail(BM_E_INVALID, "null destination pointer");
    if ((f == 9 || f == 10) && !s->desc.pair_contact)
      return fail(BM_E_INVALID, "pair-contact history: the scene has no material-material contact");
    size_t w = (f == 3) ? 9 : (f == 1 || f == 2 || f == 5 || f == 0) ? 3 : (f == 9) ? BM_HIST
             : (f == 10) ? 3 * BM_HIST : 1;
    size_t es = (f == 6) ? 8 : 4;
    size_t bytes = (size_t)n * w * es;
    if (f == 0) {
      CK(cudaMemcpy(d, s->X.data(), bytes, dst_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost));
      continue;
    }
    void *tgt = d;
    void *tmp = nullptr;
    if (!dst_on_device) {
      CK(cudaMalloc(&tmp, bytes));
      tgt = tmp;
    }
    cudaError_t e = (f == 6) ? bm_launch_code(W->w, (int)s->p_begin, (int)n, (int64_t *)tgt, W->st)
                             : bm_launch_io(W->w, s->slot, (int)s->p_begin, (int)n, f, tgt, 0, W->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(W->st);
    if (e == cudaSuccess && tmp) e = cudaMemcpy(d, tmp, bytes, cudaMemcpyDeviceToHost);
    if (tmp) cudaFree(tmp);
    CK(e);
  }
  return BM_OK;
}

int bm_write_state(bm_scene_t s, uint32_t field_mask, const void *const *src, int src_on_device) {
  if (!valid_scene(s) || !src) return fail(BM_E_INVALID, "bad scene or source");
  if (field_mask & (BM_FIELD_X | BM_FIELD_CODE | BM_FIELD_PAIR_PARTNER | BM_FIELD_PAIR_U))
    return fail(BM_E_INVALID, "X, CODE and the pair-contact history are read-only");
  WorldH *W = s->world;
  CK(cudaStreamSynchronize(W->st));
  const int64_t n = s->n;
  int j = 0;
  bool masks = false;
  for (int f = 0; f < BM_NUM_FIELDS; ++f) {
    if (!(field_mask & (1u << f))) continue;
    const void *d = src[j++];
    if (!d) return fail(BM_E_INVALID, "null source pointer");
    size_t w = (f == 3) ? 9 : (f == 1 || f == 2 || f == 5) ? 3 : 1;
    size_t bytes = (size_t)n * w * 4;
    void *buf = (void *)d;
    void *tmp = nullptr;
    if (!src_on_device) {
      CK(cudaMalloc(&tmp, bytes));
      CK(cudaMemcpy(tmp, d, bytes, cudaMemcpyHostToDevice));
      buf = tmp;
    }
    cudaError_t e = bm_launch_io(W->w, s->slot, (int)s->p_begin, (int)n, f, buf, 1, W->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(W->st);
    if (tmp) cudaFree(tmp);
    CK(e);
    if (f == 7 || f == 8) masks = true;
  }
  if (s->desc.pair_contact && (field_mask & BM_FIELD_x)) {  // positions moved: rebuild the contact candidates
    const int zero = 0;
    CK(cudaMemcpy((char *)(W->w.scenes + s->slot) + offsetof(DevScene, pair_valid), &zero, sizeof zero,
                  cudaMemcpyHostToDevice));
  }
  if (masks) {
    CK(bm_launch_rebuild(W->w, scene_set(W, s), W->st, 1));
    CK(cudaStreamSynchronize(W->st));
  }
  return BM_OK;
}

// ---------------------------------------------------------------------------
// checkpoints: a flat buffer with a header, the device scene record and the
// scene's pool ranges, each section 256-byte aligned
// ---------------------------------------------------------------------------
namespace {
const uint64_t kCkMagic = 0x31304b434d4c4242ull;  // "BBLMCK01"
struct CkHeader {
  uint64_t magic;
  int64_t n, p_begin, hist_cap, bytes;
  int32_t pair, pad;
};
size_t ck_align(size_t b) { return (b + 255) & ~size_t(255); }

// (destination offset, pool pointer, bytes) of every section after the scene record
struct CkSection {
  size_t off;
  void *pool;
  size_t bytes;
};

std::vector<CkSection> ck_layout(const bm_scene_s *s, size_t *total) {
  const PPool &P = s->world->w.P;
  const int64_t n = s->n, pb = s->p_begin;
  std::vector<CkSection> v;
  size_t off = ck_align(sizeof(CkHeader)) + ck_align(sizeof(DevScene));
  auto add = [&](void *pool, size_t bytes) {
    v.push_back({off, pool, bytes});
    off += ck_align(bytes);
  };
  for (int a = 0; a < 3; ++a) add(P.x[a] + pb, sizeof(float) * n);
  for (int a = 0; a < 3; ++a) add(P.v[a] + pb, sizeof(float) * n);
  for (int k = 0; k < 9; ++k) add(P.F[k] + pb, sizeof(float) * n);
  for (int k = 0; k < 9; ++k) add(P.Fpi[k] + pb, sizeof(float) * n);
  for (int k = 0; k < 9; ++k) add(P.Fdot[k] + pb, sizeof(float) * n);
  add(P.D + pb, sizeof(float) * n);
  for (int a = 0; a < 3; ++a) add(P.ut[a] + pb, sizeof(float) * n);
  add(P.tflag + pb, n);
  add(P.s1 + pb, sizeof(uint32_t) * n);
  add(P.s2 + pb, sizeof(uint32_t) * n);
  if (s->desc.pair_contact) {
    for (int b = 0; b < 2; ++b) {
      add(P.hist_partner[b] + pb * BM_HIST, sizeof(int) * n * BM_HIST);
      add(P.hist_u[b] + pb * BM_HIST * 3, sizeof(float) * n * BM_HIST * 3);
    }
    // the contact candidate lists and their build positions: a restore then
    // continues with the same lists, so the next substeps repeat bit for bit
    add(P.nbr + pb * BM_NBR, sizeof(int) * n * BM_NBR);
    add(P.nbr_n + pb, n);
    for (int a = 0; a < 3; ++a) add(P.xb[a] + pb, sizeof(float) * n);
  }
  if (s->hist_cap) add(s->world->w.whist + s->hist_begin * 6, sizeof(double) * 6 * s->hist_cap);
  *total = off;
  return v;
}
}  // namespace

int bm_checkpoint_size(bm_scene_t s, int64_t *bytes) {
  if (!valid_scene(s) || !bytes) return fail(BM_E_INVALID, "bad scene or output");
  size_t total = 0;
  ck_layout(s, &total);
  *bytes = (int64_t)total;
  return BM_OK;
}

int bm_checkpoint_save(bm_scene_t s, void *dst, int dst_on_device) {
  if (!valid_scene(s) || !dst) return fail(BM_E_INVALID, "bad scene or destination");
  (void)dst_on_device;  // unified addressing: one copy kind serves both
  WorldH *W = s->world;
  size_t total = 0;
  std::vector<CkSection> secs = ck_layout(s, &total);
  CK(cudaStreamSynchronize(W->st));
  CkHeader h{kCkMagic, s->n, s->p_begin, s->hist_cap, (int64_t)total, s->desc.pair_contact ? 1 : 0, 0};
  char *d = (char *)dst;
  CK(cudaMemcpyAsync(d, &h, sizeof h, cudaMemcpyDefault, W->st));
  CK(cudaMemcpyAsync(d + ck_align(sizeof h), W->w.scenes + s->slot, sizeof(DevScene), cudaMemcpyDefault,
                     W->st));
  for (const CkSection &c : secs) CK(cudaMemcpyAsync(d + c.off, c.pool, c.bytes, cudaMemcpyDefault, W->st));
  CK(cudaStreamSynchronize(W->st));
  return BM_OK;
}

int bm_checkpoint_restore(bm_scene_t s, const void *src, int src_on_device) {
  if (!valid_scene(s) || !src) return fail(BM_E_INVALID, "bad scene or source");
  (void)src_on_device;
  WorldH *W = s->world;
  size_t total = 0;
  std::vector<CkSection> secs = ck_layout(s, &total);
  CK(cudaStreamSynchronize(W->st));
  const char *d = (const char *)src;
  CkHeader h{};
  CK(cudaMemcpy(&h, d, sizeof h, cudaMemcpyDefault));
  if (h.magic != kCkMagic || h.n != s->n || h.hist_cap != s->hist_cap || h.bytes != (int64_t)total ||
      h.pair != (s->desc.pair_contact ? 1 : 0))
    return fail(BM_E_INVALID, "checkpoint does not belong to this scene");
  DevScene sv, cur;
  CK(cudaMemcpy(&sv, d + ck_align(sizeof h), sizeof sv, cudaMemcpyDefault));
  CK(cudaMemcpy(&cur, W->w.scenes + s->slot, sizeof cur, cudaMemcpyDeviceToHost));
  for (const CkSection &c : secs) CK(cudaMemcpyAsync(c.pool, d + c.off, c.bytes, cudaMemcpyDefault, W->st));
  const PPool &P = W->w.P;
  CK(cudaMemsetAsync(P.pend + s->p_begin, 0, s->n, W->st));
  CK(cudaStreamSynchronize(W->st));
  // pair-history partners and contact candidates are pool indices of the
  // world the save was made in
  if (s->desc.pair_contact && h.p_begin != s->p_begin) {
    std::vector<int> q((size_t)s->n * BM_HIST);
    for (int b = 0; b < 2; ++b) {
      int *ptr = P.hist_partner[b] + s->p_begin * BM_HIST;
      CK(cudaMemcpy(q.data(), ptr, sizeof(int) * q.size(), cudaMemcpyDeviceToHost));
      for (auto &v : q)
        if (v >= 0) v = v - (int)h.p_begin + (int)s->p_begin;
      CK(cudaMemcpy(ptr, q.data(), sizeof(int) * q.size(), cudaMemcpyHostToDevice));
    }
    std::vector<int> nb((size_t)s->n * BM_NBR);
    int *np = P.nbr + s->p_begin * BM_NBR;
    CK(cudaMemcpy(nb.data(), np, sizeof(int) * nb.size(), cudaMemcpyDeviceToHost));
    for (auto &v : nb) v = rebase_candidate(v, (int)h.p_begin, (int)s->p_begin);
    CK(cudaMemcpy(np, nb.data(), sizeof(int) * nb.size(), cudaMemcpyHostToDevice));
  }
  set_ranges(s, sv);
  sv.slot_cap = cur.slot_cap;
  sv.label_pending = 0;
  sv.need_rebuild = 0;
  sv.stop_at = cur.stop_at;  // the stop substep is a control of the caller's, not state
  sv.frozen = (sv.stop_at >= 0 && sv.step >= sv.stop_at) ? 1 : 0;
  CK(cudaMemcpy(W->w.scenes + s->slot, &sv, sizeof sv, cudaMemcpyHostToDevice));
  CK(bm_launch_rebuild(W->w, scene_set(W, s), W->st, 1));
  CK(cudaStreamSynchronize(W->st));
  return BM_OK;
}

// ---------------------------------------------------------------------------
// adjoint of the substep
// ---------------------------------------------------------------------------
struct bm_adjoint_s {
  bm_scene_s *s = nullptr;
  Allocator al;
  void *mem = nullptr;
  size_t bytes = 0;
  std::vector<unsigned char> work;  // the kernels' work record (pointers into mem)
};

namespace {
int adjoint_scope(const bm_scene_s *s) {
  if (s->desc.pair_contact) return fail(BM_E_INVALID, "adjoint: material-material contact is not supported");
  if (s->desc.model != BM_MODEL_NEO_HOOKEAN || s->desc.yield_stress > 0 || s->desc.viscosity > 0)
    return fail(BM_E_INVALID, "adjoint: elastic neo-Hookean scenes only");
  if (s->has_blade) {
    if (s->blade.mass > 0) return fail(BM_E_INVALID, "adjoint: the blade must be kinematic (mass 0)");
    if (s->blade.rigid_interval > 1) return fail(BM_E_INVALID, "adjoint: rigid interval must be 1");
    for (int k = 0; k < s->blade.n_segments; ++k)
      for (int r = 0; r < 3; ++r)
        if (s->blade.segments[k].omega[r] != 0.0)
          return fail(BM_E_INVALID, "adjoint: blade segments must not rotate");
  }
  return BM_OK;
}
}  // namespace

int bm_adjoint_create(bm_scene_t s, bm_adjoint_t *out) {
  if (!valid_scene(s) || !out) return fail(BM_E_INVALID, "bad scene or output");
  int rc = adjoint_scope(s);
  if (rc) return rc;
  bm_adjoint_s *a = new bm_adjoint_s();
  a->s = s;
  a->al.a = s->home_alloc;
  a->al.has = s->has_home_alloc;
  a->al.st = s->world->st;
  a->bytes = bm_adj_work_alloc_bytes(s->n, s->slot_cap);
  a->mem = a->al.alloc(a->bytes);
  if (!a->mem) {
    delete a;
    return fail(BM_E_OOM, "adjoint: device allocation failed");
  }
  a->work.resize(bm_adj_work_struct_size());
  bm_adj_carve(a->mem, s->n, s->slot_cap, s->slot, a->work.data());
  *out = a;
  return bm_adjoint_reset(a);
}

int bm_adjoint_reset(bm_adjoint_t a) {
  if (!a || !valid_scene(a->s)) return fail(BM_E_INVALID, "bad adjoint");
  WorldH *W = a->s->world;
  CK(cudaMemsetAsync(a->mem, 0, a->bytes, W->st));
  CK(cudaStreamSynchronize(W->st));
  return BM_OK;
}

int bm_adjoint_substep(bm_adjoint_t a, const double force_bar[3]) {
  if (!a || !valid_scene(a->s) || !force_bar) return fail(BM_E_INVALID, "bad adjoint or force adjoint");
  bm_scene_s *s = a->s;
  int rc = adjoint_scope(s);
  if (rc) return rc;
  WorldH *W = s->world;
  bm_adj_set_slot(a->work.data(), s->slot);
  CK(bm_launch_adjoint_substep(W->w, a->work.data(), force_bar, (int)s->n, (int)s->n_node, W->st));
  return BM_OK;
}

int bm_adjoint_state(bm_adjoint_t a, uint32_t field_mask, void *const *buf, int on_device, int write) {
  if (!a || !valid_scene(a->s) || !buf) return fail(BM_E_INVALID, "bad adjoint or buffers");
  const uint32_t ok = BM_FIELD_x | BM_FIELD_v | BM_FIELD_F | BM_FIELD_UT;
  if (field_mask & ~ok) return fail(BM_E_INVALID, "adjoint fields: x, v, F, UT");
  bm_scene_s *s = a->s;
  WorldH *W = s->world;
  bm_adj_set_slot(a->work.data(), s->slot);
  CK(cudaStreamSynchronize(W->st));
  const uint32_t bits[4] = {BM_FIELD_x, BM_FIELD_v, BM_FIELD_F, BM_FIELD_UT};
  int j = 0;
  for (int f = 0; f < 4; ++f) {
    if (!(field_mask & bits[f])) continue;
    void *d = buf[j++];
    if (!d) return fail(BM_E_INVALID, "null buffer");
    const size_t bytes = sizeof(float) * (size_t)s->n * (f == 2 ? 9 : 3);
    void *dev = d, *tmp = nullptr;
    if (!on_device) {
      CK(cudaMalloc(&tmp, bytes ? bytes : 16));
      if (write) CK(cudaMemcpy(tmp, d, bytes, cudaMemcpyHostToDevice));
      dev = tmp;
    }
    cudaError_t e = bm_launch_adjoint_io(W->w, a->work.data(), f, (float *)dev, write, (int)s->n, W->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(W->st);
    if (e == cudaSuccess && tmp && !write) e = cudaMemcpy(d, tmp, bytes, cudaMemcpyDeviceToHost);
    if (tmp) cudaFree(tmp);
    CK(e);
  }
  return BM_OK;
}

int bm_adjoint_params(bm_adjoint_t a, double *out, int cap) {
  const int need = 7 + 3 * BM_MAX_SEGMENTS;
  if (!a || !valid_scene(a->s) || !out || cap < need) return fail(BM_E_INVALID, "bad adjoint or output");
  bm_scene_s *s = a->s;
  WorldH *W = s->world;
  CK(cudaStreamSynchronize(W->st));
  double acc[5 + 3 * BM_MAX_SEGMENTS];
  CK(cudaMemcpy(acc, bm_adj_acc(a->work.data()), sizeof acc, cudaMemcpyDeviceToHost));
  const double E = s->desc.E, nu = s->desc.nu, Dn = (1.0 + nu) * (1.0 - 2.0 * nu);
  // mu = E / (2 (1 + nu)), lambda = E nu / ((1 + nu)(1 - 2 nu))
  out[0] = acc[0] / (2.0 * (1.0 + nu)) + acc[1] * nu / Dn;
  out[1] = -acc[0] * E / (2.0 * (1.0 + nu) * (1.0 + nu)) + acc[1] * E * (1.0 + 2.0 * nu * nu) / (Dn * Dn);
  out[2] = acc[0];
  out[3] = acc[1];
  for (int k = 0; k < 3 + 3 * BM_MAX_SEGMENTS; ++k) out[4 + k] = acc[2 + k];
  return need;
}

int bm_adjoint_destroy(bm_adjoint_t a) {
  if (!a) return BM_OK;
  if (a->mem) {
    if (a->s && a->s->world) cudaStreamSynchronize(a->s->world->st);
    a->al.release(a->mem);
  }
  delete a;
  return BM_OK;
}

int bm_read_state_noalloc(bm_scene_t s, uint32_t field_mask, void *const *dst) {
  if (!valid_scene(s) || !dst) return fail(BM_E_INVALID, "bad scene or destination");
  WorldH *W = s->world;
  const int64_t n = s->n;
  if (field_mask & (BM_FIELD_PAIR_PARTNER | BM_FIELD_PAIR_U))
    return fail(BM_E_INVALID, "bm_read_state_noalloc: the pair-contact history is read by bm_read_state");
  // size check first: nothing is launched for a request the array cannot hold
  for (int f = 0; f < BM_NUM_FIELDS; ++f) {
    if (!(field_mask & (1u << f)) || f == 0) continue;
    const size_t w = (f == 3) ? 9 : (f == 1 || f == 2 || f == 5) ? 3 : 1;
    const size_t bytes = (size_t)n * w * ((f == 6) ? 8 : 4);
    if (bytes > BM_NOALLOC_STAGE_BYTES)
      return fail(BM_E_INVALID, "bm_read_state_noalloc: field " + std::to_string(f) + " of " +
                                    std::to_string(n) + " particles needs " + std::to_string(bytes) +
                                    " bytes; the staging array holds " +
                                    std::to_string((size_t)BM_NOALLOC_STAGE_BYTES) +
                                    " bytes (one array, reused by each field in turn)");
  }
  // the array's address is per device: the scene's device must be current,
  // or the lookup would name another GPU's copy of the array
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (W->device >= 0 && dev != W->device)
    return fail(BM_E_INVALID, "bm_read_state_noalloc: the scene lives on device " + std::to_string(W->device) +
                                  " but device " + std::to_string(dev) + " is current");
  void *stage = nullptr;
  int rc = stage_address(dev, &stage);
  if (rc) return rc;
  int j = 0;
  for (int f = 0; f < BM_NUM_FIELDS; ++f) {
    if (!(field_mask & (1u << f))) continue;
    void *d = dst[j++];
    if (!d) return fail(BM_E_INVALID, "null destination pointer");
    const size_t w = (f == 3) ? 9 : (f == 1 || f == 2 || f == 5 || f == 0) ? 3 : 1;
    const size_t bytes = (size_t)n * w * ((f == 6) ? 8 : 4);
    if (f == 0) {
      std::memcpy(d, s->X.data(), bytes);
      continue;
    }
    k_gather_stage<<<(unsigned)((n + 255) / 256), 256, 0, W->st>>>(W->w, (int)s->p_begin, (int)n, f, stage);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(d, stage, bytes, cudaMemcpyDeviceToHost, W->st));
    CK(cudaStreamSynchronize(W->st));
  }
  return BM_OK;
}

int bm_scene_info_get(bm_scene_t s, bm_scene_info *out) {
  if (!valid_scene(s) || !out) return fail(BM_E_INVALID, "bad scene");
  WorldH *W = s->world;
  CK(cudaStreamSynchronize(W->st));
  DevScene cur;
  CK(cudaMemcpy(&cur, W->w.scenes + s->slot, sizeof cur, cudaMemcpyDeviceToHost));
  out->n_particles = s->n;
  out->n_nodes = s->n_node;
  out->n_slots = cur.n_slots;
  out->slot_capacity = s->slot_cap;
  out->step = cur.step;
  out->error_bits = cur.err;
  out->current_cut = cur.cur_cut;
  out->contact_list_builds = cur.pair_builds;
  for (int a = 0; a < 3; ++a) {
    out->grid_lo[a] = s->lo[a];
    out->grid_dim[a] = s->nn[a];
  }
  return BM_OK;
}

int bm_tool_wrench(bm_scene_t s, int blade_id, double out[6]) {
  if (!valid_scene(s) || !s->has_blade || blade_id != 0 || !out) return fail(BM_E_INVALID, "bad scene or blade");
  WorldH *W = s->world;
  CK(cudaStreamSynchronize(W->st));
  CK(cudaMemcpy(out, (char *)(W->w.scenes + s->slot) + offsetof(DevScene, lastW), sizeof(double) * 6,
                cudaMemcpyDeviceToHost));
  return BM_OK;
}

int bm_wrench_history(bm_scene_t s, int blade_id, int64_t first, int64_t count, double *out) {
  if (!valid_scene(s) || !s->has_blade || blade_id != 0 || !out || first < 0 || count < 0 ||
      first + count > s->hist_cap)
    return fail(BM_E_INVALID, "bad scene, blade or history range");
  WorldH *W = s->world;
  CK(cudaStreamSynchronize(W->st));
  if (count)
    CK(cudaMemcpy(out, W->w.whist + (s->hist_begin + first) * 6, sizeof(double) * 6 * count,
                  cudaMemcpyDeviceToHost));
  return BM_OK;
}

int bm_scene_destroy(bm_scene_t s) {
  if (!s) return fail(BM_E_INVALID, "null scene");
  WorldH *W = s->world;
  if (W) {
    cudaStreamSynchronize(W->st);
    if (s->own_world) {
      delete W;
    } else {
      auto &mem = W->members;
      mem.erase(std::remove(mem.begin(), mem.end(), s), mem.end());
      unreserve(W, s);
      W->tiles_dirty = true;
    }
  }
  delete s;
  return BM_OK;
}

int bm_scene_footprint(const bm_scene_desc *desc, const float *X_ref, int64_t n, int64_t *particles,
                       int64_t *nodes, int64_t *bricks, int64_t *bytes) {
  int rc = validate_desc(desc);
  if (rc) return rc;
  if (n <= 0 || !X_ref) return fail(BM_E_INVALID, "need at least one particle");
  bm_scene_s s;
  s.desc = *desc;
  s.n = n;
  s.X.assign(X_ref, X_ref + 3 * n);
  rc = build_layout(&s);
  if (rc) return rc;
  if (particles) *particles = n;
  if (nodes) *nodes = s.n_node;
  if (bricks) *bricks = s.n_brick;
  // fx, x, v, u_t, J (3 each); F, Fp^-1, dF/dt (9 each); D; base, masks, perm; pending label;
  // the D / u_t flag;
  // with pair contact: hash key, order, entries with their base cells and cell keys, the double-buffered history,
  // the candidate list and the positions at its build
  const int64_t per_p = 4 * (3 * 5 + 9 * 3 + 1) + 4 * 4 + 1 + 1 +
                        (desc->pair_contact ? (4 + 4 + 16 + 4 + 16 + 2 * BM_HIST * 16 + 4 * BM_NBR + 1 + 12) : 0);
  const int64_t per_node = 4 + 1 + 8 * BM_MAXS + 4 * (3 * 16 + 8) + 6 * 32;
  const int64_t per_brick = 3 * BM_TILE_NODES + 48 + 16 + 8;
  if (bytes) *bytes = n * per_p + s.n_node * per_node + (s.n_cell + 1) * 4 + s.n_brick * per_brick + s.hist_cap * 48;
  return BM_OK;
}

// ---- batches ---------------------------------------------------------------

int bm_batch_create(const bm_batch_desc *desc, const bm_alloc *alloc, void *stream, bm_batch_t *out) {
  if (!desc || !out) return fail(BM_E_INVALID, "null descriptor or output");
  *out = nullptr;
  if (desc->max_particles <= 0 || desc->max_nodes <= 0 || desc->max_scenes <= 0)
    return fail(BM_E_INVALID, "batch capacities must be positive");
  cudaStream_t st = (cudaStream_t)stream;
  bool own = false;
  if (!st) {
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    own = true;
  }
  WorldH *W = new_world(alloc, st);
  W->own_stream = own;
  W->cap_p = desc->max_particles;
  W->cap_node = desc->max_nodes;
  W->cap_slot = desc->max_slots > 0 ? desc->max_slots : 4 * desc->max_nodes;
  W->cap_scenes = desc->max_scenes;
  // a scene's bricks never exceed its nodes / 27 (one brick covers >= 27 nodes)
  W->cap_brick = desc->max_bricks > 0 ? desc->max_bricks : desc->max_nodes / 27 + desc->max_scenes;
  W->cap_cell = W->cap_brick * BM_BRICK_CELLS + desc->max_scenes;
  W->cap_ppool = 6 * desc->max_nodes + 4096 * (int64_t)desc->max_scenes;
  W->cap_hist = 0;
  W->cap_ntile = (int)tiles_for(desc->max_nodes, 64) + desc->max_scenes;
  W->pair = desc->pair_contact != 0;
  W->ntile_size = desc->node_tile > 0 ? desc->node_tile : 128;
  W->graph_chunk = desc->graph_chunk > 0 ? desc->graph_chunk : 16;
  if (W->ntile_size < 64 || W->ntile_size > 512 || W->ntile_size % 32) {
    delete W;
    return fail(BM_E_INVALID, "node tile must be a multiple of 32 in [64, 512]");
  }
  int rc = world_alloc(W);
  if (rc) {
    delete W;
    return rc;
  }
  bm_batch_s *b = new bm_batch_s();
  b->world = W;
  *out = b;
  return BM_OK;
}

int bm_batch_scene_create(bm_batch_t b, const bm_scene_desc *desc, const bm_blade_desc *blade,
                          const float *X_ref, int64_t n, bm_scene_t *out) {
  if (!b || !out) return fail(BM_E_INVALID, "null batch or output handle");
  *out = nullptr;
  int rc = validate_desc(desc);
  if (rc) return rc;
  if (n <= 0 || !X_ref) return fail(BM_E_INVALID, "need at least one particle");
  if (blade) {
    if (blade->n_segments < 0 || blade->n_segments > BM_MAX_SEGMENTS) return fail(BM_E_INVALID, "too many segments");
    for (int i = 0; i < blade->n_segments; ++i)
      if (blade->segments[i].cut_id >= BM_MAX_CUTS || blade->segments[i].cut_id < -1)
        return fail(BM_E_TOO_MANY_CUTS, "cut id outside [-1, 32)");
  }
  WorldH *W = b->world;
  bm_scene_s *s = new bm_scene_s();
  s->desc = *desc;
  s->desc.wrench_history = 0;  // batch pools keep no per-substep wrench history
  s->home_stream = W->st;
  s->n = n;
  s->X.assign(X_ref, X_ref + 3 * n);
  if (blade) {
    s->blade = *blade;
    s->has_blade = true;
  }
  rc = build_layout(s);
  if (!rc) {
    fill_template(s);
    rc = place_fresh(W, s);
  }
  if (rc) {
    delete s;
    return rc;
  }
  rc = finish_placement(W, s);
  if (rc) return rc;
  *out = s;
  return BM_OK;
}

int bm_batch_add(bm_batch_t b, bm_scene_t s) {
  if (!b || !valid_scene(s)) return fail(BM_E_INVALID, "bad batch or scene");
  if (s->world == b->world) return BM_OK;
  if (s->hist_cap) return fail(BM_E_INVALID, "scenes with a wrench history cannot join a batch");
  return move_scene(s, b->world);
}

int bm_batch_remove(bm_batch_t b, bm_scene_t s) {
  if (!b || !valid_scene(s) || s->world != b->world) return fail(BM_E_INVALID, "scene is not in this batch");
  int rc = create_private_world(s, s->has_home_alloc ? &s->home_alloc : nullptr, s->home_stream);
  if (rc) return rc;
  return BM_OK;
}

int bm_batch_set_tiles(bm_batch_t b, int graph_chunk, int node_tile, int brick_variant) {
  if (!b) return fail(BM_E_INVALID, "bad batch");
  if (graph_chunk < 1 || graph_chunk > 256 || node_tile < 64 || node_tile > 512 || node_tile % 32 ||
      brick_variant < 0 || brick_variant >= BM_NUM_VARIANTS)
    return fail(BM_E_INVALID, "graph chunk in [1, 256]; node tile a multiple of 32 in [64, 512]; "
                              "brick variant in [0, 26]");
  WorldH *W = b->world;
  CK(cudaStreamSynchronize(W->st));
  W->graph_chunk = graph_chunk;
  W->ntile_size = node_tile;
  W->variant = brick_variant;
  W->tiles_dirty = true;
  return rebuild_tiles(W);
}

int bm_batch_step(bm_batch_t b, int n_substeps) {
  if (!b || n_substeps < 0) return fail(BM_E_INVALID, "bad batch or step count");
  WorldH *W = b->world;
  if (W->members.empty() || n_substeps == 0) return BM_OK;
  if (W->tiles_dirty) {
    int r = rebuild_tiles(W);
    if (r) return r;
  }
  LaunchSet ls = world_set(W);
  auto graph_for = [&](int k, cudaGraphExec_t *out) -> int {
    auto it = W->graphs.find(k);
    if (it != W->graphs.end()) {
      *out = it->second;
      return BM_OK;
    }
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(W->st, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < k; ++i) {
      cudaError_t e = bm_launch_substep(W->w, ls, W->st);
      if (e != cudaSuccess) {
        cudaStreamEndCapture(W->st, &g);
        return fail(BM_E_CUDA, std::string("capture: ") + cudaGetErrorString(e));
      }
    }
    CK(cudaStreamEndCapture(W->st, &g));
    cudaGraphExec_t ex;
    cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    W->graphs[k] = ex;
    *out = ex;
    return BM_OK;
  };
  const int chunk = W->graph_chunk;
  int full = n_substeps / chunk, rem = n_substeps % chunk;
  cudaGraphExec_t ex;
  if (full) {
    int r = graph_for(chunk, &ex);
    if (r) return r;
    for (int i = 0; i < full; ++i) CK(cudaGraphLaunch(ex, W->st));
  }
  if (rem) {
    int r = graph_for(rem, &ex);
    if (r) return r;
    CK(cudaGraphLaunch(ex, W->st));
  }
  return BM_OK;
}

int bm_batch_profile(bm_batch_t b, int n_substeps, double *ms, int *launches, int cap) {
  if (!b || n_substeps <= 0 || !ms || cap < BM_NUM_KERNELS) return fail(BM_E_INVALID, "bad arguments");
  WorldH *W = b->world;
  if (W->members.empty()) return 0;
  if (W->tiles_dirty) {
    int r = rebuild_tiles(W);
    if (r) return r;
  }
  LaunchSet ls = world_set(W);
  std::vector<cudaEvent_t> ev(2 * BM_NUM_KERNELS);
  for (auto &e : ev) CK(cudaEventCreate(&e));
  for (int k = 0; k < BM_NUM_KERNELS; ++k) {
    ms[k] = 0.0;
    if (launches) launches[k] = 0;
  }
  int rc = BM_OK;
  for (int i = 0; i < n_substeps && rc == BM_OK; ++i) {
    cudaError_t e = bm_launch_substep_ev(W->w, ls, W->st, ev.data());
    if (e == cudaSuccess) e = cudaStreamSynchronize(W->st);
    if (e != cudaSuccess) {
      rc = fail(BM_E_CUDA, std::string("profile: ") + cudaGetErrorString(e));
      break;
    }
    for (int k = 0; k < BM_NUM_KERNELS; ++k) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, ev[2 * k], ev[2 * k + 1]) == cudaSuccess) {
        ms[k] += t;
        if (launches) launches[k] += 1;
      } else {
        cudaGetLastError();  // kernel not launched this substep (its events never recorded)
      }
    }
  }
  for (auto &e : ev) cudaEventDestroy(e);
  return rc ? rc : BM_NUM_KERNELS;
}

const char *bm_kernel_name(int i) {
  return (i >= 0 && i < BM_NUM_KERNELS) ? bm_kernel_names[i] : "";
}

int bm_batch_members(bm_batch_t b, bm_scene_t *out, int cap) {
  if (!b) return fail(BM_E_INVALID, "bad batch");
  int n = (int)b->world->members.size();
  for (int i = 0; i < n && i < cap && out; ++i) out[i] = b->world->members[i];
  return n;
}

int bm_batch_set_tool_states(bm_batch_t b, const double *states, int n, int on_device) {
  if (!b || !states) return fail(BM_E_INVALID, "bad batch or states");
  WorldH *W = b->world;
  if (n != (int)W->members.size()) return fail(BM_E_INVALID, "state count must equal the member count");
  if (W->tiles_dirty) {
    int r = rebuild_tiles(W);
    if (r) return r;
  }
  const double *src = states;
  if (!on_device) {
    CK(cudaMemcpyAsync(W->d_stage, states, sizeof(double) * 18 * (size_t)n, cudaMemcpyHostToDevice, W->st));
    src = W->d_stage;
  }
  CK(bm_launch_set_tools(W->w, W->d_scene_ids, n, src, W->st));
  return BM_OK;
}

int bm_batch_tool_wrenches(bm_batch_t b, double *out, int n, int on_device) {
  if (!b || !out) return fail(BM_E_INVALID, "bad batch or output");
  WorldH *W = b->world;
  if (n != (int)W->members.size()) return fail(BM_E_INVALID, "output count must equal the member count");
  if (W->tiles_dirty) {
    int r = rebuild_tiles(W);
    if (r) return r;
  }
  double *dst = on_device ? out : W->d_stage;
  CK(bm_launch_get_wrenches(W->w, W->d_scene_ids, n, dst, W->st));
  if (!on_device) {
    CK(cudaMemcpyAsync(out, W->d_stage, sizeof(double) * 6 * (size_t)n, cudaMemcpyDeviceToHost, W->st));
    CK(cudaStreamSynchronize(W->st));
  }
  return BM_OK;
}

int bm_batch_errors(bm_batch_t b, uint32_t *bits) {
  if (!b || !bits) return fail(BM_E_INVALID, "bad batch");
  WorldH *W = b->world;
  CK(cudaStreamSynchronize(W->st));
  uint32_t acc = 0;
  for (bm_scene_s *s : W->members) {
    uint32_t e;
    CK(cudaMemcpy(&e, (char *)(W->w.scenes + s->slot) + offsetof(DevScene, err), sizeof e,
                  cudaMemcpyDeviceToHost));
    acc |= e;
  }
  *bits = acc;
  return BM_OK;
}

int bm_batch_destroy(bm_batch_t b) {
  if (!b) return fail(BM_E_INVALID, "bad batch");
  WorldH *W = b->world;
  // member scenes lose their storage: detach them
  for (bm_scene_s *s : W->members) s->world = nullptr;
  delete W;
  delete b;
  return BM_OK;
}

}  // extern "C"

// ============================================================================
// Reference-grid surface reconstruction (Sec. III-F): host side.  The lattice
// map and its tables are built once; each update runs the count / scan /
// write kernels of bm_surface.cu on the scene's current stream.
// ============================================================================
struct bm_surface_s {
  bm_scene_s *scene = nullptr;
  SurfParams sp{};
  Allocator al;
  std::vector<void *> fixed;           // lattice map, tables, per-cell arrays
  void *vbuf = nullptr, *tbuf = nullptr;  // vertex and triangle arrays (grown on demand)
  int64_t vcap = 0, tcap = 0;
  int64_t nv = 0, nt = 0;
  void release_all(cudaStream_t st) {
    if (st) cudaStreamSynchronize(st);
    for (void *p : fixed) al.release(p);
    fixed.clear();
    al.release(vbuf);
    al.release(tbuf);
    vbuf = tbuf = nullptr;
    vcap = tcap = 0;
  }
};

namespace {

template <class T>
T *surf_get(bm_surface_s *f, int64_t count) {
  void *p = f->al.alloc(sizeof(T) * (size_t)std::max<int64_t>(count, 1));
  if (p) f->fixed.push_back(p);
  return (T *)p;
}

// vertex arrays: ref[3], cur[3] floats, anchor int, masks 2 x uint32 (9 words per vertex)
int surf_grow_vertices(bm_surface_s *f, int64_t nv) {
  if (nv <= f->vcap) return BM_OK;
  int64_t cap = std::max<int64_t>(nv + nv / 4, 1024);
  void *b = f->al.alloc(sizeof(uint32_t) * 9 * (size_t)cap);
  if (!b) return fail(BM_E_OOM, "surface vertex arrays");
  f->al.release(f->vbuf);
  f->vbuf = b;
  f->vcap = cap;
  float *fb = (float *)b;
  for (int a = 0; a < 3; ++a) {
    f->sp.ref[a] = fb + (size_t)a * cap;
    f->sp.cur[a] = fb + (size_t)(3 + a) * cap;
  }
  f->sp.anchor = (int *)(fb + (size_t)6 * cap);
  f->sp.vmask[0] = (uint32_t *)(fb + (size_t)7 * cap);
  f->sp.vmask[1] = (uint32_t *)(fb + (size_t)8 * cap);
  return BM_OK;
}

int surf_grow_tris(bm_surface_s *f, int64_t nt) {
  if (nt <= f->tcap) return BM_OK;
  int64_t cap = std::max<int64_t>(nt + nt / 4, 1024);
  void *b = f->al.alloc(sizeof(int) * 3 * (size_t)cap);
  if (!b) return fail(BM_E_OOM, "surface triangle array");
  f->al.release(f->tbuf);
  f->tbuf = b;
  f->tcap = cap;
  f->sp.tri = (int *)b;
  return BM_OK;
}

bool valid_surface(bm_surface_t f) { return f && f->scene && valid_scene(f->scene); }

}  // namespace

extern "C" {

int bm_surface_create(bm_scene_t s, const int lattice[3], bm_surface_t *out) {
  if (!out) return fail(BM_E_INVALID, "null output handle");
  *out = nullptr;
  if (!valid_scene(s) || !lattice) return fail(BM_E_INVALID, "bad scene or lattice");
  for (int a = 0; a < 3; ++a)
    if (lattice[a] < 1 || lattice[a] > 64) return fail(BM_E_INVALID, "lattice counts must lie in [1, 64]");
  const int64_t n = s->n;
  const bm_scene_desc &d = s->desc;
  double h[3], Xmin[3];
  for (int a = 0; a < 3; ++a) {
    h[a] = d.dx / lattice[a];
    Xmin[a] = HUGE_VAL;
  }
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) Xmin[a] = std::min(Xmin[a], (double)s->X[3 * i + a]);
  // lattice index of every particle (caller order)
  std::vector<int64_t> jj((size_t)n * 3);
  int64_t nl[3] = {0, 0, 0};
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) {
      const double X = (double)s->X[3 * i + a];
      const double r = (X - Xmin[a]) / h[a];
      const int64_t j = (int64_t)std::llround(r);
      if (!(std::fabs(Xmin[a] + (double)j * h[a] - X) <= 1e-3 * h[a]) || j < 0 || j > (1 << 20))
        return fail(BM_E_INVALID, "particle off the sub-cell lattice");
      jj[3 * i + a] = j;
      nl[a] = std::max(nl[a], j + 1);
    }
  const int64_t total = nl[0] * nl[1] * nl[2];
  const int64_t ncells = (nl[0] + 1) * (nl[1] + 1) * (nl[2] + 1);
  if (total > ((int64_t)1 << 30) || ncells > ((int64_t)1 << 30))
    return fail(BM_E_INVALID, "surface lattice too large");
  std::vector<int> jlin((size_t)n);
  {
    std::vector<uint8_t> seen((size_t)total, 0);
    for (int64_t i = 0; i < n; ++i) {
      const int64_t lin = (jj[3 * i + 2] * nl[1] + jj[3 * i + 1]) * nl[0] + jj[3 * i];
      if (seen[(size_t)lin]) return fail(BM_E_INVALID, "two particles share a lattice point");
      seen[(size_t)lin] = 1;
      jlin[(size_t)i] = (int)lin;
    }
  }
  // stencil base cell of every lattice coordinate; it must be the particles'
  std::vector<int> base[3], jstart[3];
  int bmin[3], bmax[3];
  for (int a = 0; a < 3; ++a) {
    base[a].resize((size_t)nl[a]);
    for (int64_t j = 0; j < nl[a]; ++j)
      base[a][(size_t)j] = (int)std::floor((Xmin[a] + (double)j * h[a] - d.origin[a]) / d.dx - 0.5);
    bmin[a] = base[a].front();
    bmax[a] = base[a].back();
    for (int64_t j = 1; j < nl[a]; ++j)
      if (base[a][(size_t)j] < base[a][(size_t)j - 1]) return fail(BM_E_INVALID, "lattice not monotone");
    jstart[a].assign((size_t)(bmax[a] - bmin[a] + 2), (int)nl[a]);
    for (int B = bmin[a]; B <= bmax[a] + 1; ++B) {
      int64_t j = 0;
      while (j < nl[a] && base[a][(size_t)j] < B) ++j;
      jstart[a][(size_t)(B - bmin[a])] = (int)j;
    }
  }
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) {
      const double xl = ((double)s->X[3 * i + a] - d.origin[a]) / d.dx;
      if ((int)std::floor(xl - 0.5) != base[a][(size_t)jj[3 * i + a]])
        return fail(BM_E_INVALID, "lattice is not at the reference cells' sub-cell centres");
    }

  bm_surface_s *f = new bm_surface_s();
  f->scene = s;
  f->al.has = s->has_home_alloc;
  f->al.a = s->home_alloc;
  f->al.st = s->home_stream;
  SurfParams &sp = f->sp;
  for (int a = 0; a < 3; ++a) {
    sp.n[a] = (int)nl[a];
    sp.nc[a] = (int)nl[a] + 1;
    sp.Xmin[a] = Xmin[a];
    sp.h[a] = h[a];
    sp.origin[a] = d.origin[a];
    sp.lo[a] = s->lo[a];
    sp.bmin[a] = bmin[a];
    sp.bmax[a] = bmax[a];
  }
  sp.dx = d.dx;
  sp.n_cells = ncells;
  bool ok = true;
  int *js[3];
  for (int a = 0; a < 3; ++a) ok &= (js[a] = surf_get<int>(f, (int64_t)jstart[a].size())) != nullptr;
  ok &= (sp.lat = surf_get<int>(f, total)) != nullptr;
  for (int a = 0; a < 3; ++a) ok &= (sp.Xr[a] = surf_get<float>(f, n)) != nullptr;
  ok &= (sp.cell_cnt = surf_get<int>(f, ncells)) != nullptr;
  ok &= (sp.cell_off = surf_get<int>(f, ncells + 1)) != nullptr;
  ok &= (sp.cell_reg = surf_get<uint32_t>(f, ncells)) != nullptr;
  ok &= (sp.pt_cnt = surf_get<int>(f, ncells)) != nullptr;
  ok &= (sp.pt_off = surf_get<int>(f, ncells + 1)) != nullptr;
  ok &= (sp.scan_tmp = surf_get<int>(f, ncells / 1024 + 2)) != nullptr;
  int *d_jlin = nullptr;
  float *d_X = nullptr;
  if (ok) {
    d_jlin = (int *)f->al.alloc(sizeof(int) * (size_t)n);
    d_X = (float *)f->al.alloc(sizeof(float) * 3 * (size_t)n);
    ok = d_jlin && d_X;
  }
  if (!ok) {
    f->al.release(d_jlin);
    f->al.release(d_X);
    f->release_all(nullptr);
    delete f;
    return fail(BM_E_OOM, "surface buffers");
  }
  for (int a = 0; a < 3; ++a) sp.jstart[a] = js[a];
  WorldH *W = s->world;
  sp.p_begin = (int)s->p_begin;
  sp.slot = s->slot;
  cudaStream_t st = W->st;
  cudaError_t e = cudaSuccess;
  for (int a = 0; a < 3 && e == cudaSuccess; ++a)
    e = cudaMemcpyAsync(js[a], jstart[a].data(), sizeof(int) * jstart[a].size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sp.lat, 0xff, sizeof(int) * (size_t)total, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_jlin, jlin.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_X, s->X.data(), sizeof(float) * 3 * (size_t)n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = bm_launch_surface_map(W->w, sp, (int)n, d_jlin, d_X, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  f->al.release(d_jlin);
  f->al.release(d_X);
  if (e != cudaSuccess) {
    f->release_all(st);
    delete f;
    return fail(BM_E_CUDA, std::string("surface set-up: ") + cudaGetErrorString(e));
  }
  *out = f;
  return BM_OK;
}

int bm_surface_update(bm_surface_t f, int rebuild, int64_t *n_vertices, int64_t *n_triangles) {
  if (!valid_surface(f)) return fail(BM_E_INVALID, "bad surface or its scene has no storage");
  bm_scene_s *s = f->scene;
  WorldH *W = s->world;
  SurfParams &sp = f->sp;
  sp.p_begin = (int)s->p_begin;  // the scene may have moved between worlds
  sp.slot = s->slot;
  cudaStream_t st = W->st;
  if (rebuild || f->vbuf == nullptr) {
    CK(bm_launch_surface_cells(W->w, sp, st));
    int nv = 0;
    CK(cudaMemcpyAsync(&nv, sp.cell_off + sp.n_cells, sizeof nv, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int rc = surf_grow_vertices(f, nv);
    if (rc) return rc;
    CK(bm_launch_surface_vertices(W->w, sp, st));
    CK(bm_launch_surface_tri_count(W->w, sp, st));
    int nt = 0;
    CK(cudaMemcpyAsync(&nt, sp.pt_off + sp.n_cells, sizeof nt, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    rc = surf_grow_tris(f, nt);
    if (rc) return rc;
    CK(bm_launch_surface_tris(W->w, sp, st));
    f->nv = nv;
    f->nt = nt;
  }
  CK(bm_launch_surface_embed(W->w, sp, (int)f->nv, st));
  CK(cudaStreamSynchronize(st));
  if (n_vertices) *n_vertices = f->nv;
  if (n_triangles) *n_triangles = f->nt;
  return BM_OK;
}

int bm_surface_read(bm_surface_t f, float *vertices, float *reference, int32_t *triangles, uint32_t *masks,
                    int dst_on_device) {
  if (!valid_surface(f)) return fail(BM_E_INVALID, "bad surface or its scene has no storage");
  cudaStream_t st = f->scene->world->st;
  CK(cudaStreamSynchronize(st));
  const size_t nv = (size_t)f->nv, nt = (size_t)f->nt;
  const cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  // struct-of-arrays on the device, [n][3] / [n][2] at the ABI
  auto interleave = [&](void *dst, void *const *cols, int ncol, size_t cnt) -> cudaError_t {
    for (int a = 0; a < ncol; ++a) {
      cudaError_t e = cudaMemcpy2DAsync((char *)dst + 4 * a, 4 * (size_t)ncol, cols[a], 4, 4, cnt, kind, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  if (nv && vertices) {
    void *c[3] = {f->sp.cur[0], f->sp.cur[1], f->sp.cur[2]};
    CK(interleave(vertices, c, 3, nv));
  }
  if (nv && reference) {
    void *c[3] = {f->sp.ref[0], f->sp.ref[1], f->sp.ref[2]};
    CK(interleave(reference, c, 3, nv));
  }
  if (nv && masks) {
    void *c[2] = {f->sp.vmask[0], f->sp.vmask[1]};
    CK(interleave(masks, c, 2, nv));
  }
  if (nt && triangles) CK(cudaMemcpyAsync(triangles, f->sp.tri, sizeof(int) * 3 * nt, kind, st));
  CK(cudaStreamSynchronize(st));
  return BM_OK;
}

int bm_surface_destroy(bm_surface_t f) {
  if (!f) return fail(BM_E_INVALID, "null surface");
  cudaStream_t st = (f->scene && f->scene->world) ? f->scene->world->st : nullptr;
  f->release_all(st);
  delete f;
  return BM_OK;
}

}  // extern "C"

// ============================================================================
// Diagnostic: measured FP32 FMA throughput (the ALU roofline's ceiling)
// ============================================================================
namespace {
constexpr int kFmaUnroll = 16;
__global__ void __launch_bounds__(256) k_fma_peak(float *out, int iters, float seed) {
  // eight independent chains per thread keep every FMA pipe busy
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = seed + (float)(threadIdx.x + k);
  const float b = 0.999999f, c = 1e-6f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kFmaUnroll; ++u)
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == 1234.5f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}
}  // namespace

extern "C" int bm_fp32_fma_peak(void *stream, double *tflops) {
  if (!tflops) return fail(BM_E_INVALID, "null output");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256, iters = 4096;
  float *out = nullptr;
  CK(cudaMalloc(&out, sizeof(float) * (size_t)blocks * threads));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  cudaError_t e = cudaSuccess;
  float best = 0.f;
  for (int r = 0; r < 4 && e == cudaSuccess; ++r) {  // first run warms up
    cudaEventRecord(e0, st);
    k_fma_peak<<<blocks, threads, 0, st>>>(out, iters, 1.0f);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r > 0 && ms > 0.f) best = std::max(best, 1.f / ms);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  CK(e);
  const double flop = 2.0 * kFmaUnroll * 8 * (double)iters * blocks * threads;
  *tflops = flop * (double)best * 1e3 / 1e12;
  return BM_OK;
}
