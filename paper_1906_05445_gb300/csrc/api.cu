// api.cu -- host side of the C ABI declared in include/lbm.h.
//
// The context owns every device buffer.  Its state is the post-collision
// array f*(t) (`f[cur]`) plus, in `f[1-cur]`, either f*(t-1) (after a step:
// gathering from it with the current geometry reproduces the pre-collision
// f(t) for queries) or the pre-collision f(t) itself (after an
// initialisation: `prev_local`).  One step (Sec. 2 of Peng, Ayala & Wang):
//   bounce-back: geometry at X(t) (+ refilling) -> sweep -> X += U dt
//   IBM        : X += U dt -> geometry at X(t+1) -> unforced velocity, force,
//                spreading -> sweep
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {
void launch_sweep_f64(SweepOp, int, int, const KArgs &, cudaStream_t);
void launch_sweep_f32(SweepOp, int, int, const KArgs &, cudaStream_t);
void launch_sweep_bf16(SweepOp, int, int, const KArgs &, cudaStream_t);
void launch_sweep_f16(SweepOp, int, int, const KArgs &, cudaStream_t);

bool launch_bulk_group_f32(const KArgs *, int, int, int, cudaStream_t);
bool launch_bulk_group_bf16(const KArgs *, int, int, int, cudaStream_t);
bool launch_bulk_group_f16(const KArgs *, int, int, int, cudaStream_t);

bool launch_bulk_group(const KArgs *as, int n, int lattice, int collision, int precision,
                       cudaStream_t st) {
  switch (precision) {
  case LBM_FP32: return launch_bulk_group_f32(as, n, lattice, collision, st);
  case LBM_FP32_BF16STORE: return launch_bulk_group_bf16(as, n, lattice, collision, st);
  case LBM_FP32_FP16STORE: return launch_bulk_group_f16(as, n, lattice, collision, st);
  default: return false;  // FP64 runs the one-node kernel
  }
}

void launch_sweep(SweepOp op, int lattice, int collision, int precision, const KArgs &a,
                  cudaStream_t st) {
  switch (precision) {
  case LBM_FP64: launch_sweep_f64(op, lattice, collision, a, st); break;
  case LBM_FP32: launch_sweep_f32(op, lattice, collision, a, st); break;
  case LBM_FP32_BF16STORE: launch_sweep_bf16(op, lattice, collision, a, st); break;
  default: launch_sweep_f16(op, lattice, collision, a, st); break;
  }
}
thread_local int g_bulk_kernel = BK_NODE;
}  // namespace lbm

using namespace lbm;

namespace {

constexpr int kHistCap = 4096;          // force records kept (steps)
constexpr double kFp16Scale = (double)(1 << kFp16ScaleLog2);  // FP16 storage keeps (f - w) * 2^10
constexpr int kGeomMargin = 7;          // box margin around a moving solid

struct SolidHost {
  lbm_solid_desc d;
  double c[3];   // centre now
  double cg[3];  // centre of the current geometry
  // free motion: density ratio rho_p / rho_f (0: prescribed), gravity, and
  // the velocities of the previous step (Eq. 23)
  double rho_p = 0, g[3] = {0, 0, 0}, Up[3] = {0, 0, 0}, Omp[3] = {0, 0, 0};
  // Kempe's treatment under IBM (Eq. 24): the inside fluid's momentum and
  // angular momentum at the previous step, once one has been taken
  bool have_Ip = false;
  double Ip[6] = {0, 0, 0, 0, 0, 0};
};

const double PI = 3.14159265358979323846;

}  // namespace

struct lbm_ctx {
  lbm_lattice_desc d;
  int Q = 0, D = 0;
  long long N = 0;
  long long fs = 0;  // direction stride of the distribution arrays (elements)
  int bulk_block = 128;
  int list_block = 256;
  int cache_hints = 0;
  int bulk_mode = 1;
  int bulk_kernel = -1;  // the bulk sweep kernel of the last step (BulkKernel), -1 none yet
  int bulk_vec_words = 0;
  int bulk_vec_packed = -1;
  int ibm_list_thread = 1;  // IBM band nodes: a thread per node in the boundary sweep
  int ibb_list_thread = 0;  // bounce-back boundary nodes too (measured slower: off)
  int coll_mode = 0;  // CM_BGK, CM_MRT or CM_MRT_Q
  cudaStream_t st = 0;
  // auxiliary high-priority stream: the boundary-node sweep and the IBM
  // pre-pass run there, concurrently with the bulk sweep on `st`
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // bumped by every call that changes what a step's launches read (their
  // arguments, buffers or state): a batch's captured graph is then stale
  unsigned long long gen = 0;
  cudaEvent_t ev_grp = nullptr;  // lbm_step_multi: this lattice's stream joins a grouped launch
  // lbm_copy_force_torque_async: the copies run on their own stream, after
  // an event of the step, so that they do not hold up the next step
  cudaStream_t cst = nullptr;
  cudaEvent_t ev_rec = nullptr, ev_cst = nullptr;
  long long copies = 0;
  // uploads (lbm_set_distributions): copies of staging slot k on `cst`,
  // conversions on `st`, each slot reused only after its last conversion
  cudaEvent_t ev_up_start = nullptr, ev_up_copy[2] = {nullptr, nullptr},
              ev_up_conv[2] = {nullptr, nullptr};
  int device = 0;
  size_t ssz = 0;  // storage element size
  size_t tsz = 0;  // compute element size
  void *f[2] = {nullptr, nullptr};
  int cur = 0;
  bool prev_local = true, need_collide = true;
  uint8_t *flags = nullptr, *sid = nullptr;
  int *counts = nullptr;  // 16 ints
  int *list_node = nullptr;
  uint32_t *list_mask = nullptr;
  int *list_link = nullptr;
  double *list_cst = nullptr;
  int list_cap = 0, link_cap = 0, refill_cap = 0;
  int list_count = -1, link_count = -1;  // known after a static build
  long long bulk_nodes = 0;              // plain fluid nodes at the last full build
  void *link_mem = nullptr;
  LinkArrays links{};
  int *link_list = nullptr;
  uint8_t *link_dir = nullptr;
  int *refill_node = nullptr;
  uint8_t *refill_sid = nullptr;
  // moving solids: a second geometry set, built for the next step on its own
  // stream while the current step's kernels run (see prefetch_geometry)
  struct GeomBuf {
    uint8_t *flags = nullptr, *sid = nullptr;
    int *counts = nullptr;
    int *list_node = nullptr;
    uint32_t *list_mask = nullptr;
    int *list_link = nullptr;
    double *list_cst = nullptr;
    void *link_mem = nullptr;
    LinkArrays links{};
    int *link_list = nullptr;
    uint8_t *link_dir = nullptr;
    int *refill_node = nullptr;
    uint8_t *refill_sid = nullptr;
  } spare;
  bool spare_ready = false, prefetched = false, geom_prefetch = true;
  // Eq. 16: pre-collision populations kept at the boundary nodes ([Q][fs],
  // compute type; allocated when the scheme is first selected)
  void *zy_pre = nullptr;
  double *kempe = nullptr;  // [kMaxSolids][6] Eq. 24 sums of the current step
  // domain faces: types and wall velocities, the nodes next to a
  // non-periodic face, and the outflow face's kept populations
  lbm_domain_desc dom{};
  int *face_node = nullptr;
  int nface = 0;
  void *outlet = nullptr;
  int out_face = -1;
  long long out_area = 0;
  double pf_c[kMaxSolids][3] = {};
  // free solids: the solids' state lives in device memory (sol_d[0] the
  // current state, sol_d[1] the centres of the current geometry, free_d the
  // dynamics) and a step moves them there.  The host copy in `solids` is
  // brought up to date on demand (motion_pull) and sent back after a change
  // (motion_push).
  SolidsDev *sol_d = nullptr;
  FreeDev *free_d = nullptr;
  bool host_stale = false, push_needed = true;
  // the force-record slot the next IBM step's motion reads instead of the
  // current one (-1: none); set for the first step of a captured step pair
  int motion_slot = -1;
  cudaStream_t gst = nullptr;
  cudaEvent_t ev_geom = nullptr, ev_gfree = nullptr;
  // IBM
  double *mk_dir = nullptr, *mk_dV = nullptr, *mk_F = nullptr, *mk_dF = nullptr;
  uint8_t *mk_sid = nullptr;
  int4 *mk_base = nullptr;  // stencil table (rebuilt with the geometry)
  void *mk_wts = nullptr;
  bool markers_dirty = false;
  int nmark = 0;
  int mk_start[kMaxSolids + 1] = {0};  // markers of solid k: mk_start[k] .. mk_start[k+1] - 1
  // the forcing loop in one cluster per solid (see ibm.cu), taken with
  // LBM_IBM_CLUSTER=1 where it fits the device (decided when the markers are
  // built); off by default: it measured slower than the warp-per-marker
  // kernels spread over every SM
  bool ibm_cluster = false, ibm_cluster_on = false;
  void *u_band = nullptr, *f_ibm = nullptr;
  // forces
  double *hist = nullptr;
  int slot = 0;
  long long records = 0;
  // queries / residual
  double *qbuf = nullptr;
  size_t qbuf_elems = 0;
  double *u_now = nullptr, *u_snap = nullptr, *red2 = nullptr;
  double last_residual = NAN;
  // host state
  std::vector<SolidHost> solids;
  lbm_scheme_desc scheme{};
  bool geom_dirty = true, restore_geometry = false;
  long long step = 0, launches = 0;
  size_t dev_bytes = 0;
  std::string err;
  // collision constants
  double omega = 0, ds[19] = {0}, s_bulk = 0, nu = 0, inv_scale = 1;
  // timing
  int timing = 0;  // bit k + 1: kernel kind k is timed
  int timing_every = 1;  // time the launches of every n-th step
  struct Pending {
    cudaEvent_t a, b;
    int kind;
    long long nodes;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> free_events;
  double tk_ms[TK_COUNT] = {0};
  long long tk_launch[TK_COUNT] = {0}, tk_nodes[TK_COUNT] = {0};
  std::vector<void *> allocs;
};

namespace {

lbm_status fail(lbm_ctx *c, lbm_status s, const std::string &m) {
  if (c) c->err = m;
  return s;
}

lbm_status cuda_check(lbm_ctx *c, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return LBM_OK;
  return fail(c, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(expr)                                              \
  do {                                                        \
    lbm_status _s = cuda_check(ctx, (expr), #expr);           \
    if (_s != LBM_OK) return _s;                              \
  } while (0)
#define TRY(expr)                                             \
  do {                                                        \
    lbm_status _s = (expr);                                   \
    if (_s != LBM_OK) return _s;                              \
  } while (0)

// allocation fault injection (lbm_debug_fail_allocations_after): the
// number of device allocations still allowed, or -1 for no limit
std::atomic<long long> g_alloc_budget{-1};

lbm_status dalloc(lbm_ctx *ctx, void **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return LBM_OK;
  if (g_alloc_budget.load() >= 0 && g_alloc_budget.fetch_sub(1) <= 0) {
    g_alloc_budget.store(0);
    return fail(ctx, LBM_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) +
                                      " bytes refused by the allocation fault hook");
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(ctx, LBM_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  ctx->dev_bytes += bytes;
  ctx->allocs.push_back(*p);
  return LBM_OK;
}

void dfree(lbm_ctx *ctx, void *p) {
  if (!p) return;
  auto it = std::find(ctx->allocs.begin(), ctx->allocs.end(), p);
  if (it != ctx->allocs.end()) ctx->allocs.erase(it);
  cudaFree(p);
}

bool is_ibb(int s) { return (s >= LBM_BOUNCE_BACK && s <= LBM_YU_QUAD) || s == LBM_ZHAO_YONG; }

// ---- timing helpers (CUDA events on the context's stream)
cudaEvent_t take_event(lbm_ctx *ctx) {
  if (!ctx->free_events.empty()) {
    cudaEvent_t e = ctx->free_events.back();
    ctx->free_events.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

struct Timed {
  lbm_ctx *ctx;
  int kind;
  long long nodes;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  bool on;
  Timed(lbm_ctx *c, int k, long long n, cudaStream_t stream)
      : ctx(c), kind(k), nodes(n), s(stream),
        on(((c->timing >> (k + 1)) & 1) != 0 && c->step % c->timing_every == 0) {
    if (on) {
      a = take_event(ctx);
      cudaEventRecord(a, s);
    }
  }
  ~Timed() {
    if (on) {
      cudaEvent_t b = take_event(ctx);
      cudaEventRecord(b, s);
      ctx->pending.push_back({a, b, kind, nodes});
    }
  }
};

void resolve_timing(lbm_ctx *ctx) {
  for (auto &p : ctx->pending) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      ctx->tk_ms[p.kind] += ms;
      ctx->tk_launch[p.kind] += 1;
      ctx->tk_nodes[p.kind] += p.nodes;
    }
    ctx->free_events.push_back(p.a);
    ctx->free_events.push_back(p.b);
  }
  ctx->pending.clear();
}

bool any_free(const lbm_ctx *ctx);
bool dev_motion(const lbm_ctx *ctx);
bool ibm_cluster_args(const lbm_ctx *ctx, IbmClusterArgs &cl);

// ---- kernel argument assembly
SolidsDev solids_dev(const lbm_ctx *ctx, bool geometry_centres) {
  SolidsDev s{};
  s.n = (int)ctx->solids.size();
  for (int k = 0; k < s.n; k++) {
    const SolidHost &h = ctx->solids[k];
    SolidDev &o = s.s[k];
    o.kind = h.d.kind;
    o.fluid_inside = h.d.fluid_inside;
    o.R = h.d.radius;
    for (int a = 0; a < 3; a++) {
      o.c[a] = geometry_centres ? h.cg[a] : h.c[a];
      o.U[a] = h.d.velocity[a];
      o.Om[a] = h.d.omega[a];
    }
    if (ctx->D == 2) {
      o.c[2] = 0;
      o.U[2] = 0;
      o.Om[0] = o.Om[1] = 0;
    }
    const double rd = ctx->scheme.ibm_retraction;
    o.RL = h.d.fluid_inside ? h.d.radius + rd : h.d.radius - rd;
  }
  return s;
}

KArgs base_args(lbm_ctx *ctx) {
  KArgs a;
  memset(&a, 0, sizeof(a));
  a.nx = ctx->d.nx;
  a.ny = ctx->d.ny;
  a.nz = ctx->D == 2 ? 1 : ctx->d.nz;
  a.N = ctx->N;
  a.fs = ctx->fs;
  a.bulk_block = ctx->bulk_block;
  a.cache_hints = ctx->cache_hints;
  a.bulk_mode = ctx->bulk_mode;
  a.bulk_vec_words = ctx->bulk_vec_words;
  a.bulk_vec_packed = ctx->bulk_vec_packed;
  a.list_thread = (ctx->scheme.scheme == LBM_IBM_DIRECT && ctx->ibm_list_thread) ||
                          ctx->ibb_list_thread ? 1 : 0;
  a.list_block = ctx->list_block;
  a.zy_pre = ctx->scheme.scheme == LBM_ZHAO_YONG ? ctx->zy_pre : nullptr;
  for (int k = 0; k < 6; k++) {
    a.face[k] = ctx->dom.type[k];
    for (int c = 0; c < 3; c++) {
      a.u_face[k][c] = ctx->D == 2 && c == 2 ? 0.0 : ctx->dom.u[k][c];
      a.u_face_f[k][c] = (float)a.u_face[k][c];
    }
  }
  a.face_node = ctx->face_node;
  a.nface = ctx->nface;
  a.outlet = ctx->outlet;
  a.out_face = ctx->out_face;
  a.out_area = ctx->out_area;
  a.flags = ctx->flags;
  a.omega = ctx->omega;
  for (int k = 0; k < 19; k++) a.ds[k] = ctx->ds[k];
  a.s_bulk = ctx->s_bulk;
  a.nu = ctx->nu;
  for (int k = 0; k < 3; k++) a.g[k] = ctx->d.body_force[k];
  if (ctx->D == 2) a.g[2] = 0;
  a.inv_scale = ctx->inv_scale;
  a.omega_f = (float)a.omega;
  for (int k = 0; k < 19; k++) a.ds_f[k] = (float)a.ds[k];
  for (int k = 0; k < 3; k++) a.g_f[k] = (float)a.g[k];
  a.inv_scale_f = (float)a.inv_scale;
  a.list_node = ctx->list_node;
  a.list_mask = ctx->list_mask;
  a.list_link = ctx->list_link;
  a.list_cst = ctx->list_cst;
  a.counts = ctx->counts;
  a.wait_err = ctx->counts + 5;
  a.list_cap = ctx->list_count >= 0 ? std::min(ctx->list_count, ctx->list_cap) : ctx->list_cap;
  a.links = ctx->links;
  a.f_ibm = ctx->f_ibm;
  a.u_band = ctx->u_band;
  a.nsolids = (int)ctx->solids.size();
  a.refill_node = ctx->refill_node;
  a.refill_sid = ctx->refill_sid;
  a.refill_cap = ctx->refill_cap;
  a.solids = solids_dev(ctx, true);
  a.solids_d = dev_motion(ctx) ? ctx->sol_d + 1 : nullptr;
  a.sid = ctx->sid;
  return a;
}

void sweep(lbm_ctx *ctx, SweepOp op, const KArgs &a, cudaStream_t s) {
  launch_sweep(op, ctx->d.lattice, ctx->coll_mode, ctx->d.precision, a, s);
  if (op == OP_BULK_SWEEP) ctx->bulk_kernel = g_bulk_kernel;
  ctx->launches++;
}
void sweep(lbm_ctx *ctx, SweepOp op, const KArgs &a) { sweep(ctx, op, a, ctx->st); }

// ---- geometry
void solid_box(const lbm_ctx *ctx, const SolidHost &s, GeomBox &b) {
  const int n[3] = {ctx->d.nx, ctx->d.ny, ctx->D == 2 ? 1 : ctx->d.nz};
  int o[3], w[3];
  for (int a = 0; a < 3; a++) {
    const bool full = s.d.fluid_inside || (a == 2 && (ctx->D == 2 || s.d.kind == LBM_CYLINDER_Z));
    const double ext = s.d.radius + kGeomMargin + fabs(ctx->scheme.ibm_retraction);
    int lo = (int)floor(s.cg[a] - ext), hi = (int)ceil(s.cg[a] + ext);
    if (full || hi - lo + 1 >= n[a]) {
      o[a] = 0;
      w[a] = n[a];
    } else {
      o[a] = lo;
      w[a] = hi - lo + 1;
    }
  }
  b = {o[0], o[1], o[2], w[0], w[1], w[2]};
}

bool any_free(const lbm_ctx *ctx) {
  for (auto &s : ctx->solids)
    if (s.rho_p > 0) return true;
  return false;
}

bool any_moving(const lbm_ctx *ctx) {
  for (auto &s : ctx->solids)
    if (s.d.velocity[0] != 0 || s.d.velocity[1] != 0 || (ctx->D == 3 && s.d.velocity[2] != 0) ||
        s.rho_p > 0)
      return true;
  return false;
}

// Whether the solids move on the device (a free solid is present).
bool dev_motion(const lbm_ctx *ctx) { return any_free(ctx); }

// Host copy of the solids' state <- device (waits for the stream).
lbm_status motion_pull(lbm_ctx *ctx) {
  if (!ctx->host_stale || !ctx->sol_d) return LBM_OK;
  SolidsDev sd[2];
  FreeDev fd[kMaxSolids];
  CK(cudaMemcpyAsync(sd, ctx->sol_d, sizeof(sd), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(fd, ctx->free_d, sizeof(fd), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  for (size_t k = 0; k < ctx->solids.size(); k++) {
    SolidHost &h = ctx->solids[k];
    for (int a = 0; a < 3; a++) {
      h.c[a] = sd[0].s[k].c[a];
      h.cg[a] = sd[1].s[k].c[a];
      h.d.velocity[a] = sd[0].s[k].U[a];
      h.d.omega[a] = sd[0].s[k].Om[a];
      h.Up[a] = fd[k].Up[a];
      h.Omp[a] = fd[k].Omp[a];
    }
    for (int c = 0; c < 6; c++) h.Ip[c] = fd[k].Ip[c];
    h.have_Ip = fd[k].have_Ip != 0;
  }
  ctx->host_stale = false;
  return LBM_OK;
}

// Device copy of the solids' state <- host (the current state, the
// geometry's centres and the dynamics), ordered on the stream.
lbm_status motion_push(lbm_ctx *ctx) {
  if (!dev_motion(ctx)) {
    ctx->push_needed = false;
    return LBM_OK;
  }
  if (!ctx->sol_d) TRY(dalloc(ctx, (void **)&ctx->sol_d, 2 * sizeof(SolidsDev)));
  if (!ctx->free_d) TRY(dalloc(ctx, (void **)&ctx->free_d, kMaxSolids * sizeof(FreeDev)));
  if (!ctx->kempe) TRY(dalloc(ctx, (void **)&ctx->kempe, sizeof(double) * kMaxSolids * 6));
  SolidsDev sd[2] = {solids_dev(ctx, false), solids_dev(ctx, true)};
  FreeDev fd[kMaxSolids];
  memset(fd, 0, sizeof(fd));
  for (size_t k = 0; k < ctx->solids.size(); k++) {
    const SolidHost &h = ctx->solids[k];
    fd[k].rho_p = h.rho_p;
    for (int a = 0; a < 3; a++) {
      fd[k].g[a] = h.g[a];
      fd[k].Up[a] = h.Up[a];
      fd[k].Omp[a] = h.Omp[a];
    }
    for (int c = 0; c < 6; c++) fd[k].Ip[c] = h.Ip[c];
    fd[k].have_Ip = h.have_Ip ? 1 : 0;
  }
  CK(cudaMemcpyAsync(ctx->sol_d, sd, sizeof(sd), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->free_d, fd, sizeof(fd), cudaMemcpyHostToDevice, ctx->st));
  // the copies read host locals: let them finish before those go
  CK(cudaStreamSynchronize(ctx->st));
  ctx->push_needed = false;
  ctx->host_stale = false;
  return LBM_OK;
}

// Before the host reads or changes the solids: bring its copy up to date,
// and have the device copy sent again before the next kernel reads it.
lbm_status solids_to_host(lbm_ctx *ctx, bool will_change) {
  TRY(motion_pull(ctx));
  if (will_change) ctx->push_needed = true;
  return LBM_OK;
}

// Eq. 24 for every free solid from the current state f*(t) and the forces
// of its collision, into ctx->kempe (FP64, zeroed first).
lbm_status kempe_integrals(lbm_ctx *ctx) {
  if (!ctx->kempe) TRY(dalloc(ctx, (void **)&ctx->kempe, sizeof(double) * kMaxSolids * 6));
  CK(cudaMemsetAsync(ctx->kempe, 0, sizeof(double) * kMaxSolids * 6, ctx->st));
  const int len[3] = {ctx->d.nx, ctx->d.ny, ctx->D == 2 ? 1 : ctx->d.nz};
  for (size_t k = 0; k < ctx->solids.size(); k++) {
    const SolidHost &h = ctx->solids[k];
    if (!(h.rho_p > 0)) continue;
    KArgs a = base_args(ctx);
    a.src = ctx->f[ctx->cur];
    a.solids = solids_dev(ctx, false);
    a.solids_d = ctx->sol_d;  // the current state (free solids move on the device)
    a.kbox_dev = 1;
    a.kempe_out = ctx->kempe + 6 * k;
    a.kempe_solid = (int)k;
    for (int c = 0; c < 3; c++) {
      // every node with a cell corner inside lies within R + 1 of the
      // centre: a box of ceil(2R + 2) + 2 nodes from floor(c - R - 1)
      const bool whole = c >= ctx->D || (c == 2 && h.d.kind == LBM_CYLINDER_Z);
      const int ext = (int)ceil(2.0 * h.d.radius + 2.0) + 2;
      a.kbox[c] = 0;
      a.kbox[3 + c] = (whole || ext >= len[c]) ? len[c] : ext;
    }
    sweep(ctx, OP_KEMPE, a);
  }
  return LBM_OK;
}

double *force_slot(lbm_ctx *ctx, int slot);

// One step of the solids' motion on the device (motion.cu): free solids by
// Newton-Euler from the force record `slot` (this step's momentum exchange
// under bounce-back, the current IBM force under IBM), the others by their
// prescribed velocity.  Nothing is read back.
lbm_status motion_step(lbm_ctx *ctx, int slot) {
  const bool ibm = ctx->scheme.scheme == LBM_IBM_DIRECT;
  const bool kempe = ibm && ctx->scheme.ibm_inertia == LBM_INERTIA_KEMPE;
  if (ctx->push_needed) TRY(motion_push(ctx));
  if (kempe) TRY(kempe_integrals(ctx));
  MotionArgs m;
  memset(&m, 0, sizeof(m));
  m.now = ctx->sol_d;
  m.fr = ctx->free_d;
  m.rec = force_slot(ctx, slot);
  m.kempe = kempe ? ctx->kempe : nullptr;
  m.n = (int)ctx->solids.size();
  m.mode = !ibm ? MM_BOUNCE_BACK
                : kempe ? MM_IBM_KEMPE
                        : ctx->scheme.ibm_inertia == LBM_INERTIA_UHLMANN ? MM_IBM_UHLMANN
                                                                         : MM_IBM_FENG;
  m.dim = ctx->D;
  m.nz = ctx->D == 2 ? 1 : ctx->d.nz;
  for (int k = 0; k < 6; k++) m.face[k] = ctx->dom.type[k];
  m.len[0] = ctx->d.nx;
  m.len[1] = ctx->d.ny;
  m.len[2] = m.nz;
  m.err = ctx->counts + 4;
  launch_motion(m, ctx->st);
  ctx->launches++;
  ctx->host_stale = true;
  CK(cudaGetLastError());
  return LBM_OK;
}

// link records: c0..c4, mw, uw[3], arm[3] in the compute type, then the solid id
size_t link_bytes(const lbm_ctx *ctx, size_t lk) { return (12 * ctx->tsz + 1) * lk + 64; }
void layout_links(const lbm_ctx *ctx, void *mem, size_t lk, LinkArrays &L) {
  char *p = (char *)mem;
  for (int k = 0; k < 5; k++) {
    L.c[k] = p;
    p += ctx->tsz * lk;
  }
  L.mw = p;
  p += ctx->tsz * lk;
  for (int k = 0; k < 3; k++) {
    L.uw[k] = p;
    p += ctx->tsz * lk;
  }
  for (int k = 0; k < 3; k++) {
    L.arm[k] = p;
    p += ctx->tsz * lk;
  }
  L.sid = (uint8_t *)p;
}

lbm_status ensure_list_capacity(lbm_ctx *ctx, int list_cap, int link_cap, int refill_cap) {
  if (list_cap > ctx->list_cap || refill_cap > ctx->refill_cap) {
    dfree(ctx, ctx->list_node);
    dfree(ctx, ctx->list_mask);
    dfree(ctx, ctx->list_link);
    dfree(ctx, ctx->list_cst);
    dfree(ctx, ctx->refill_node);
    dfree(ctx, ctx->refill_sid);
    ctx->list_node = nullptr;
    ctx->list_mask = nullptr;
    ctx->list_link = nullptr;
    ctx->list_cst = nullptr;
    ctx->refill_node = nullptr;
    ctx->refill_sid = nullptr;
    // no capacity until every array exists (a failed allocation leaves the
    // kernels nothing to index)
    ctx->list_cap = ctx->refill_cap = 0;
    const int lc = std::max(list_cap, 1), rc = std::max(refill_cap, 1);
    TRY(dalloc(ctx, (void **)&ctx->list_node, sizeof(int) * lc));
    TRY(dalloc(ctx, (void **)&ctx->list_mask, sizeof(uint32_t) * lc));
    TRY(dalloc(ctx, (void **)&ctx->list_link, sizeof(int) * lc));
    TRY(dalloc(ctx, (void **)&ctx->list_cst, sizeof(double) * 6 * lc));
    TRY(dalloc(ctx, (void **)&ctx->refill_node, sizeof(int) * rc));
    TRY(dalloc(ctx, (void **)&ctx->refill_sid, rc));
    ctx->list_cap = list_cap;
    ctx->refill_cap = refill_cap;
  }
  if (link_cap > ctx->link_cap) {
    dfree(ctx, ctx->link_mem);
    dfree(ctx, ctx->link_list);
    dfree(ctx, ctx->link_dir);
    ctx->link_mem = nullptr;
    ctx->link_list = nullptr;
    ctx->link_dir = nullptr;
    ctx->link_cap = 0;
    const size_t lk = std::max(link_cap, 1);
    TRY(dalloc(ctx, (void **)&ctx->link_list, sizeof(int) * lk));
    TRY(dalloc(ctx, (void **)&ctx->link_dir, lk));
    TRY(dalloc(ctx, &ctx->link_mem, link_bytes(ctx, lk)));
    layout_links(ctx, ctx->link_mem, lk, ctx->links);
    ctx->link_cap = link_cap;
  }
  return LBM_OK;
}

// exchange the current geometry set with the spare one
void swap_geom(lbm_ctx *ctx) {
  auto &b = ctx->spare;
  std::swap(ctx->flags, b.flags);
  std::swap(ctx->sid, b.sid);
  std::swap(ctx->counts, b.counts);
  std::swap(ctx->list_node, b.list_node);
  std::swap(ctx->list_mask, b.list_mask);
  std::swap(ctx->list_link, b.list_link);
  std::swap(ctx->list_cst, b.list_cst);
  std::swap(ctx->link_mem, b.link_mem);
  std::swap(ctx->links, b.links);
  std::swap(ctx->link_list, b.link_list);
  std::swap(ctx->link_dir, b.link_dir);
  std::swap(ctx->refill_node, b.refill_node);
  std::swap(ctx->refill_sid, b.refill_sid);
}

void free_spare(lbm_ctx *ctx) {
  if (!ctx->spare_ready) return;
  if (ctx->gst) cudaStreamSynchronize(ctx->gst);
  auto &b = ctx->spare;
  for (void *p : {(void *)b.flags, (void *)b.sid, (void *)b.counts, (void *)b.list_node,
                  (void *)b.list_mask, (void *)b.list_link, (void *)b.list_cst, b.link_mem,
                  (void *)b.link_list, (void *)b.link_dir, (void *)b.refill_node,
                  (void *)b.refill_sid})
    dfree(ctx, p);
  b = lbm_ctx::GeomBuf{};
  ctx->spare_ready = false;
  ctx->prefetched = false;
}

// the spare geometry set, with the capacities of the current one
lbm_status alloc_spare(lbm_ctx *ctx) {
  if (ctx->spare_ready) return LBM_OK;
  if (!ctx->gst) {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&ctx->gst, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_geom, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_gfree, cudaEventDisableTiming) != cudaSuccess)
      return fail(ctx, LBM_ERR_CUDA, "geometry stream");
  }
  auto &b = ctx->spare;
  const size_t padN = ((ctx->N + 15) / 16) * 16;
  const int lc = std::max(ctx->list_cap, 1), rc = std::max(ctx->refill_cap, 1);
  const size_t lk = std::max(ctx->link_cap, 1);
  TRY(dalloc(ctx, (void **)&b.flags, padN));
  TRY(dalloc(ctx, (void **)&b.sid, 2 * padN));
  TRY(dalloc(ctx, (void **)&b.counts, 16 * sizeof(int)));
  TRY(dalloc(ctx, (void **)&b.list_node, sizeof(int) * lc));
  TRY(dalloc(ctx, (void **)&b.list_mask, sizeof(uint32_t) * lc));
  TRY(dalloc(ctx, (void **)&b.list_link, sizeof(int) * lc));
  TRY(dalloc(ctx, (void **)&b.list_cst, sizeof(double) * 6 * lc));
  TRY(dalloc(ctx, (void **)&b.refill_node, sizeof(int) * rc));
  TRY(dalloc(ctx, (void **)&b.refill_sid, rc));
  TRY(dalloc(ctx, (void **)&b.link_list, sizeof(int) * lk));
  TRY(dalloc(ctx, (void **)&b.link_dir, lk));
  TRY(dalloc(ctx, &b.link_mem, link_bytes(ctx, lk)));
  layout_links(ctx, b.link_mem, lk, b.links);
  ctx->spare_ready = true;
  return LBM_OK;
}

GeomArgs geom_args(lbm_ctx *ctx) {
  GeomArgs g;
  memset(&g, 0, sizeof(g));
  g.nx = ctx->d.nx;
  g.ny = ctx->d.ny;
  g.nz = ctx->D == 2 ? 1 : ctx->d.nz;
  g.N = ctx->N;
  g.lattice = ctx->d.lattice;
  g.scheme = ctx->scheme.scheme;
  g.force_all = ctx->d.force_region == LBM_FORCE_ALL;
  g.solids = solids_dev(ctx, true);
  g.solids_d = dev_motion(ctx) ? ctx->sol_d + 1 : nullptr;
  g.flags = ctx->flags;
  g.sid = ctx->sid;
  g.counts = ctx->counts;
  g.list_node = ctx->list_node;
  g.list_mask = ctx->list_mask;
  g.list_link = ctx->list_link;
  g.list_cst = ctx->list_cst;
  g.link_list = ctx->link_list;
  g.link_dir = ctx->link_dir;
  g.list_cap = ctx->list_cap;
  g.link_cap = ctx->link_cap;
  g.links = ctx->links;
  g.refill_node = ctx->refill_node;
  g.refill_sid = ctx->refill_sid;
  g.refill_cap = ctx->refill_cap;
  g.band_w = 2.0 * sqrt((double)ctx->D) + 1e-6;
  for (int k = 0; k < 6; k++) g.face[k] = ctx->dom.type[k];
  return g;
}

// Solids keep clear of the non-periodic faces:
//  - of a velocity or stress-free face by 1.5 spacings between the surface
//    and the outermost nodes: no node next to the face then has a cut link
//    (links are at most sqrt(2) long), and every IBM delta stencil stays
//    inside the domain.  IBM band nodes next to the face run in the face
//    kernel; bounce-back stencil nodes beyond the face count as missing;
//  - of an outflow face by R + 5 nodes, so that neither a face node nor the
//    inner neighbour its update reads is a boundary or band node.
lbm_status check_clearance(lbm_ctx *ctx) {
  const int len[3] = {ctx->d.nx, ctx->d.ny, ctx->D == 2 ? 1 : ctx->d.nz};
  for (auto &h : ctx->solids)
    for (int a = 0; a < ctx->D; a++) {
      if (ctx->dom.type[2 * a] == LBM_FACE_PERIODIC) continue;
      if (h.d.fluid_inside)
        return fail(ctx, LBM_ERR_UNSUPPORTED, "a fluid-inside solid fills the domain up to its non-periodic faces");
      if (a == 2 && h.d.kind == LBM_CYLINDER_Z)
        return fail(ctx, LBM_ERR_UNSUPPORTED, "a z-cylinder meets the non-periodic z faces");
      const bool conv_lo = ctx->dom.type[2 * a] == LBM_FACE_CONVECTIVE;
      const bool conv_hi = ctx->dom.type[2 * a + 1] == LBM_FACE_CONVECTIVE;
      const double R = h.d.radius;
      const double mlo = conv_lo ? R + 5.0 : R + 1.5, mhi = conv_hi ? R + 5.0 : R + 1.5;
      if (h.c[a] - mlo < 0 || h.c[a] + mhi > len[a] - 1)
        return fail(ctx, LBM_ERR_UNSUPPORTED,
                    "solid too close to a non-periodic face (1.5 nodes from a wall or "
                    "stress-free face, R + 5 from an outflow face)");
    }
  return LBM_OK;
}

void set_boxes(lbm_ctx *ctx, GeomArgs &g, bool full) {
  g.box_dev = 0;
  if (full || ctx->solids.empty()) {
    g.nbox = 1;
    g.box[0] = {0, 0, 0, g.nx, g.ny, g.nz};
  } else if (dev_motion(ctx)) {
    // the centres are in device memory: boxes of a fixed width that covers
    // any position, anchored there by the geometry kernels
    g.nbox = (int)ctx->solids.size();
    g.box_dev = 1;
    const int n[3] = {g.nx, g.ny, g.nz};
    for (int k = 0; k < g.nbox; k++) {
      const SolidHost &h = ctx->solids[k];
      const double ext = h.d.radius + kGeomMargin + fabs(ctx->scheme.ibm_retraction);
      g.box_ext[k] = ext;
      int w[3];
      for (int a = 0; a < 3; a++) {
        const bool whole =
            h.d.fluid_inside || (a == 2 && (ctx->D == 2 || h.d.kind == LBM_CYLINDER_Z));
        const int wa = (int)ceil(2.0 * ext) + 2;
        w[a] = (whole || wa >= n[a]) ? n[a] : wa;
      }
      g.box[k] = {0, 0, 0, w[0], w[1], w[2]};
    }
  } else {
    g.nbox = (int)ctx->solids.size();
    for (int k = 0; k < g.nbox; k++) solid_box(ctx, ctx->solids[k], g.box[k]);
  }
  g.box_offset[0] = 0;
  for (int k = 0; k < g.nbox; k++)
    g.box_offset[k + 1] = g.box_offset[k] + (long long)g.box[k].bx * g.box[k].by * g.box[k].bz;
}

lbm_status build_markers(lbm_ctx *ctx) {
  dfree(ctx, ctx->mk_dir);
  dfree(ctx, ctx->mk_dV);
  dfree(ctx, ctx->mk_F);
  dfree(ctx, ctx->mk_dF);
  dfree(ctx, ctx->mk_sid);
  dfree(ctx, ctx->mk_base);
  dfree(ctx, ctx->mk_wts);
  ctx->mk_dir = ctx->mk_dV = ctx->mk_F = ctx->mk_dF = nullptr;
  ctx->mk_sid = nullptr;
  ctx->mk_base = nullptr;
  ctx->mk_wts = nullptr;
  ctx->nmark = 0;
  if (ctx->scheme.scheme != LBM_IBM_DIRECT || ctx->solids.empty()) return LBM_OK;
  std::vector<double> dx, dy, dz, dV;
  std::vector<uint8_t> ms;
  const double dens = ctx->scheme.ibm_marker_density > 0 ? ctx->scheme.ibm_marker_density : 1.0;
  for (size_t k = 0; k < ctx->solids.size(); k++) {
    ctx->mk_start[k] = (int)dx.size();
    const SolidHost &s = ctx->solids[k];
    const double rd = ctx->scheme.ibm_retraction;
    const double RL = s.d.fluid_inside ? s.d.radius + rd : s.d.radius - rd;
    if (ctx->D == 3 && s.d.kind == LBM_SPHERE) {
      // golden-angle points on the sphere, about `dens` per unit area
      const double area = 4 * PI * RL * RL;
      int n = (int)lround(dens * area);
      if (n < 1) n = 1;
      const double ga = PI * (3 - sqrt(5.0));
      for (int m = 0; m < n; m++) {
        const double z = 1 - (2.0 * m + 1) / n, r = sqrt(1 - z * z);
        dx.push_back(r * cos(ga * m));
        dy.push_back(r * sin(ga * m));
        dz.push_back(z);
        dV.push_back(area / n);
        ms.push_back((uint8_t)k);
      }
    } else {
      // uniform angles on a circle; one ring per z-plane for a cylinder on
      // a 3D lattice (dz holds the plane)
      const double circ = 2 * PI * RL;
      int per = (int)lround(dens * circ);
      if (per < 1) per = 1;
      const int rings = ctx->D == 3 ? ctx->d.nz : 1;
      for (int r = 0; r < rings; r++)
        for (int m = 0; m < per; m++) {
          const double th = 2 * PI * m / per;
          dx.push_back(cos(th));
          dy.push_back(sin(th));
          dz.push_back((double)r);
          dV.push_back(circ / per);
          ms.push_back((uint8_t)k);
        }
    }
  }
  const int n = (int)dx.size();
  ctx->mk_start[ctx->solids.size()] = n;
  std::vector<double> dir(3 * (size_t)n);
  for (int m = 0; m < n; m++) {
    dir[m] = dx[m];
    dir[n + m] = dy[m];
    dir[2 * n + m] = dz[m];
  }
  TRY(dalloc(ctx, (void **)&ctx->mk_dir, sizeof(double) * 3 * n));
  TRY(dalloc(ctx, (void **)&ctx->mk_dV, sizeof(double) * n));
  TRY(dalloc(ctx, (void **)&ctx->mk_F, sizeof(double) * 3 * n));
  TRY(dalloc(ctx, (void **)&ctx->mk_dF, sizeof(double) * 3 * n));
  TRY(dalloc(ctx, (void **)&ctx->mk_sid, n));
  TRY(dalloc(ctx, (void **)&ctx->mk_base, sizeof(int4) * n));
  TRY(dalloc(ctx, &ctx->mk_wts, ctx->tsz * (ctx->D == 3 ? 64 : 16) * (size_t)n));
  CK(cudaMemcpyAsync(ctx->mk_dir, dir.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->mk_dV, dV.data(), sizeof(double) * n, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->mk_sid, ms.data(), n, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  ctx->nmark = n;
  if (!ctx->u_band) {
    TRY(dalloc(ctx, &ctx->u_band, 3 * ctx->tsz * ctx->N));
    CK(cudaMemsetAsync(ctx->u_band, 0, 3 * ctx->tsz * ctx->N, ctx->st));
  }
  if (!ctx->f_ibm) {
    TRY(dalloc(ctx, &ctx->f_ibm, 3 * ctx->tsz * ctx->N));
    CK(cudaMemsetAsync(ctx->f_ibm, 0, 3 * ctx->tsz * ctx->N, ctx->st));
  }
  return LBM_OK;
}

void ibm_prepare(lbm_ctx *ctx);
void ibm_prepare(lbm_ctx *ctx, cudaStream_t s);

lbm_status read_counts(lbm_ctx *ctx, int out[16]) {
  CK(cudaMemcpyAsync(out, ctx->counts, 16 * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return LBM_OK;
}

// Full rebuild over the whole lattice (solids or scheme changed): count the
// boundary nodes and links first, size the lists exactly, then build.
lbm_status rebuild_full(lbm_ctx *ctx) {
  if (ctx) ctx->gen++;
  free_spare(ctx);  // capacities may change; the next moving step prefetches again
  TRY(motion_pull(ctx));
  if (!ctx->restore_geometry)
    for (auto &s : ctx->solids) memcpy(s.cg, s.c, sizeof(s.c));
  ctx->restore_geometry = false;
  TRY(motion_push(ctx));
  TRY(build_markers(ctx));
  GeomArgs g = geom_args(ctx);
  set_boxes(ctx, g, true);
  g.list_cap = g.link_cap = g.refill_cap = 0;
  g.track_new = 0;
  CK(cudaMemsetAsync(ctx->counts, 0, 16 * sizeof(int), ctx->st));
  launch_geometry(g, ctx->d.precision, ctx->st);
  ctx->launches += 4;
  int cnt[16];
  TRY(read_counts(ctx, cnt));
  const bool moving = any_moving(ctx);
  int list_cap = cnt[0], link_cap = cnt[1], refill_cap = 0;
  if (moving) {
    // per-step rebuilds over the solids' boxes: bound by the box volume
    GeomArgs gb = g;
    set_boxes(ctx, gb, false);
    const long long vol = gb.box_offset[gb.nbox];
    const long long lb = std::min<long long>(vol, 2LL * cnt[0] + 4096);
    const long long kb = std::min<long long>((long long)(ctx->Q - 1) * vol, 2LL * cnt[1] + 4096LL * 8);
    list_cap = (int)lb;
    link_cap = (int)kb;
    refill_cap = (int)std::min<long long>(vol, 1 << 20);
  }
  TRY(ensure_list_capacity(ctx, list_cap, link_cap, refill_cap));
  g = geom_args(ctx);
  set_boxes(ctx, g, true);
  g.refill_cap = 0;
  g.track_new = 0;
  CK(cudaMemsetAsync(ctx->counts, 0, 16 * sizeof(int), ctx->st));
  launch_geometry(g, ctx->d.precision, ctx->st);
  ctx->launches += 4;
  TRY(read_counts(ctx, cnt));
  if (cnt[3]) return fail(ctx, LBM_ERR_CAPACITY, "boundary list overflow during rebuild");
  ctx->list_count = moving ? -1 : cnt[0];
  ctx->link_count = moving ? -1 : cnt[1];
  ibm_prepare(ctx);
  {
    IbmClusterArgs cl;
    ctx->ibm_cluster = ctx->ibm_cluster_on && ibm_cluster_args(ctx, cl) &&
                       ibm_cluster_fits(cl, ctx->d.precision);
  }
  {
    std::vector<uint8_t> fl(ctx->N);
    CK(cudaMemcpyAsync(fl.data(), ctx->flags, ctx->N, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    long long b = 0;
    for (long long k = 0; k < ctx->N; k++) b += (fl[k] & ~FL_NOG) == 0;
    ctx->bulk_nodes = b;
  }
  ctx->geom_dirty = false;
  return LBM_OK;
}

// Per-step rebuild over the boxes of the solids (moving geometry).
lbm_status rebuild_boxes(lbm_ctx *ctx) {
  if (dev_motion(ctx)) {
    // the geometry's centres <- the current ones, on the device
    if (ctx->push_needed) TRY(motion_push(ctx));
    CK(cudaMemcpyAsync(ctx->sol_d + 1, ctx->sol_d, sizeof(SolidsDev), cudaMemcpyDeviceToDevice,
                       ctx->st));
  } else {
    for (auto &s : ctx->solids) memcpy(s.cg, s.c, sizeof(s.c));
  }
  GeomArgs g = geom_args(ctx);
  set_boxes(ctx, g, false);
  g.track_new = is_ibb(ctx->scheme.scheme) ? 1 : 0;
  CK(cudaMemsetAsync(ctx->counts, 0, 4 * sizeof(int), ctx->st));
  Timed tm(ctx, TK_GEOM, 0, ctx->st);
  launch_geometry(g, ctx->d.precision, ctx->st);
  ctx->launches += 4;
  ctx->markers_dirty = true;  // marker table: rebuilt by the IBM pre-pass
  return LBM_OK;
}

// Build the next step's geometry (solids at centres `next`) into the spare
// set on the geometry stream.  The spare set was last read by the previous
// step's kernels; ev_gfree, recorded on the main stream at the start of the
// current step, follows them.  The current set is only read here (its
// solid ids are the previous ids of the next build, its flags the starting
// point outside the solids' boxes), so the build overlaps the current step.
lbm_status prefetch_geometry(lbm_ctx *ctx, const double next[][3]) {
  TRY(alloc_spare(ctx));
  const size_t padN = ((ctx->N + 15) / 16) * 16;
  CK(cudaStreamWaitEvent(ctx->gst, ctx->ev_gfree, 0));
  CK(cudaMemcpyAsync(ctx->spare.flags, ctx->flags, padN, cudaMemcpyDeviceToDevice, ctx->gst));
  CK(cudaMemcpyAsync(ctx->spare.sid, ctx->sid, padN, cudaMemcpyDeviceToDevice, ctx->gst));
  CK(cudaMemsetAsync(ctx->spare.counts, 0, 4 * sizeof(int), ctx->gst));
  double saved[kMaxSolids][3];
  for (size_t k = 0; k < ctx->solids.size(); k++) {
    memcpy(saved[k], ctx->solids[k].cg, sizeof(saved[k]));
    memcpy(ctx->solids[k].cg, next[k], sizeof(saved[k]));
    memcpy(ctx->pf_c[k], next[k], sizeof(saved[k]));
  }
  swap_geom(ctx);
  GeomArgs g = geom_args(ctx);
  set_boxes(ctx, g, false);
  swap_geom(ctx);
  for (size_t k = 0; k < ctx->solids.size(); k++)
    memcpy(ctx->solids[k].cg, saved[k], sizeof(saved[k]));
  g.track_new = is_ibb(ctx->scheme.scheme) ? 1 : 0;
  {
    Timed tm(ctx, TK_GEOM, 0, ctx->gst);
    launch_geometry(g, ctx->d.precision, ctx->gst);
  }
  ctx->launches += 4;
  CK(cudaEventRecord(ctx->ev_geom, ctx->gst));
  ctx->prefetched = true;
  return LBM_OK;
}

// Switch to the prefetched geometry if it was built for the centres the
// current step needs (the caller may have moved the solids since).
bool take_prefetched(lbm_ctx *ctx) {
  if (!ctx->prefetched) return false;
  ctx->prefetched = false;
  for (size_t k = 0; k < ctx->solids.size(); k++)
    for (int a = 0; a < 3; a++)
      if (ctx->pf_c[k][a] != ctx->solids[k].c[a]) return false;
  if (cudaStreamWaitEvent(ctx->st, ctx->ev_geom, 0) != cudaSuccess) return false;
  swap_geom(ctx);
  for (auto &sh : ctx->solids) memcpy(sh.cg, sh.c, sizeof(sh.c));
  ctx->markers_dirty = true;  // marker table: rebuilt by the IBM pre-pass
  return true;
}

lbm_status ensure_geometry(lbm_ctx *ctx) {
  // solids moving on the device are checked there, after each move
  if (ctx->nface && !ctx->host_stale) TRY(check_clearance(ctx));
  if (ctx->geom_dirty) return rebuild_full(ctx);
  if (ctx->push_needed) TRY(motion_push(ctx));
  return LBM_OK;
}

double *force_slot(lbm_ctx *ctx, int slot) {
  return ctx->hist + (size_t)slot * kMaxSolids * 6;
}

IbmArgs ibm_args(lbm_ctx *ctx, double *acc) {
  IbmArgs ib;
  memset(&ib, 0, sizeof(ib));
  ib.nx = ctx->d.nx;
  ib.ny = ctx->d.ny;
  ib.nz = ctx->D == 2 ? 1 : ctx->d.nz;
  ib.dim = ctx->D;
  ib.N = ctx->N;
  ib.nmark = ctx->nmark;
  ib.dir = ctx->mk_dir;
  ib.dV = ctx->mk_dV;
  ib.msid = ctx->mk_sid;
  ib.Fm = ctx->mk_F;
  ib.kernel = ctx->scheme.ibm_kernel;
  ib.solids = solids_dev(ctx, true);
  ib.solids_d = dev_motion(ctx) ? ctx->sol_d + 1 : nullptr;
  ib.u_band = ctx->u_band;
  ib.f_ibm = ctx->f_ibm;
  ib.force_acc = acc;
  ib.mk_base = ctx->mk_base;
  ib.mk_wts = ctx->mk_wts;
  return ib;
}

// stencil table of the markers at the geometry centres
void ibm_prepare(lbm_ctx *ctx, cudaStream_t s) {
  ctx->markers_dirty = false;
  if (ctx->scheme.scheme != LBM_IBM_DIRECT || ctx->nmark == 0) return;
  launch_ibm_prepare(ibm_args(ctx, nullptr), ctx->d.precision, s);
  ctx->launches++;
}
void ibm_prepare(lbm_ctx *ctx) { ibm_prepare(ctx, ctx->st); }

// Whether ibm_prepass launches the band-velocity kernel, which clears the
// step's force record before the IBM kernels accumulate into it.
bool ibm_zeroes_record(const lbm_ctx *ctx) {
  const int lc = ctx->list_count >= 0 ? std::min(ctx->list_count, ctx->list_cap) : ctx->list_cap;
  return ctx->scheme.scheme == LBM_IBM_DIRECT && ctx->nmark > 0 && lc > 0;
}

// IBM: unforced velocity at the band, n_it interpolation/force iterations,
// spreading, and the solid's force (into the given record slot).
// whether [o1, o1 + w1) and [o2, o2 + w2) are disjoint on a periodic axis of n
bool disjoint_mod(int o1, int w1, int o2, int w2, int n) {
  if (w1 + w2 > n) return false;
  const int d12 = ((o2 - o1) % n + n) % n, d21 = ((o1 - o2) % n + n) % n;
  return d12 >= w1 && d21 >= w2;
}

// The cluster kernel's boxes: every stencil point of solid k's markers lies
// within [floor(c - R_L) - 1, floor(c + R_L) + 2] per axis; the box is one
// node wider on either side (a whole axis for a z-cylinder's rings or where
// the box would reach round the lattice).
// false where the kernel does not apply: no IBM solids, several solids whose
// boxes may meet (their forcing loops would couple), or a free solid among
// several (its box moves on the device).
bool ibm_cluster_args(const lbm_ctx *ctx, IbmClusterArgs &cl) {
  memset(&cl, 0, sizeof(cl));
  const int ns = (int)ctx->solids.size();
  if (ns < 1 || ctx->nmark == 0 || ctx->scheme.scheme != LBM_IBM_DIRECT) return false;
  const bool dev = dev_motion(ctx);
  if (dev && ns > 1) return false;
  cl.ns = ns;
  cl.dim = ctx->D;
  cl.iters = std::max(1, ctx->scheme.ibm_iters);
  cl.box_dev = dev ? 1 : 0;
  const int n[3] = {ctx->d.nx, ctx->d.ny, ctx->D == 2 ? 1 : ctx->d.nz};
  const int sax = ctx->D == 3 ? 2 : 1;
  for (int k = 0; k <= ns; k++) cl.mk_start[k] = ctx->mk_start[k];
  for (int k = 0; k < ns; k++) {
    const SolidHost &h = ctx->solids[k];
    const double rd = ctx->scheme.ibm_retraction;
    const double RL = h.d.fluid_inside ? h.d.radius + rd : h.d.radius - rd;
    IbmBox &B = cl.box[k];
    // one node of slack on either side of the stencils' reach
    B.ext = RL + 2.0;
    for (int a = 0; a < 3; a++) {
      const bool whole = a >= ctx->D || (a == 2 && h.d.kind == LBM_CYLINDER_Z);
      const int w = (int)ceil(2.0 * RL) + 7;
      if (whole || w >= n[a]) {
        B.o[a] = 0;
        B.w[a] = n[a];
      } else {
        B.o[a] = (int)floor(h.cg[a] - B.ext);
        B.w[a] = w;
      }
    }
    B.h = (B.w[sax] + kIbmClusterSize - 1) / kIbmClusterSize;
    const int cnt = ctx->mk_start[k + 1] - ctx->mk_start[k];
    B.mpc = (cnt + kIbmClusterSize - 1) / kIbmClusterSize;
  }
  for (int i = 0; i < ns; i++)
    for (int j = i + 1; j < ns; j++) {
      bool apart = false;
      for (int a = 0; a < ctx->D && !apart; a++)
        apart = disjoint_mod(cl.box[i].o[a], cl.box[i].w[a], cl.box[j].o[a], cl.box[j].w[a], n[a]);
      if (!apart) return false;
    }
  return true;
}

void ibm_prepass(lbm_ctx *ctx, const void *src, bool local, double *acc, cudaStream_t s) {
  if (ctx->scheme.scheme != LBM_IBM_DIRECT || ctx->nmark == 0) return;
  Timed tm(ctx, TK_IBM, 0, s);
  if (ctx->markers_dirty) ibm_prepare(ctx, s);  // moving solids: every step
  KArgs a = base_args(ctx);
  a.src = src;
  a.local_gather = local ? 1 : 0;
  a.force_acc = acc;  // cleared by the band-velocity kernel
  sweep(ctx, OP_BAND_VEL, a, s);
  IbmArgs ib = ibm_args(ctx, acc);
  const int iters = std::max(1, ctx->scheme.ibm_iters);
  IbmClusterArgs cl;
  if (ctx->ibm_cluster && ibm_cluster_args(ctx, cl)) {
    launch_ibm_cluster(ib, cl, ctx->d.precision, s);
    ctx->launches++;
    return;
  }
  if (iters == 1) {
    ib.first = 1;
    ib.reduce_force = 1;
    launch_ibm_fused(ib, ctx->d.precision, s);
    ctx->launches++;
    return;
  }
  // Eq. 9 iterations: the first is the fused pass; each later one
  // interpolates u~ + f, adds rho0 (U^d - U) to the force, and spreads that
  // increment onto f (the same sum as re-spreading the total force)
  ib.first = 1;
  ib.reduce_force = 0;
  launch_ibm_fused(ib, ctx->d.precision, s);
  ctx->launches++;
  ib.dF = ctx->mk_dF;
  for (int it = 1; it < iters; it++) {
    ib.first = 0;
    ib.use_f = 1;
    launch_ibm_interp(ib, ctx->d.precision, s);
    ib.reduce_force = it == iters - 1;
    launch_ibm_spread(ib, ctx->d.precision, s);
    ctx->launches += 2;
  }
}

// Collide the pre-collision state held in f[1-cur] into f[cur].
lbm_status init_collide(lbm_ctx *ctx) {
  if (ctx) ctx->gen++;
  TRY(ensure_geometry(ctx));
  const int prev = 1 - ctx->cur;
  ctx->slot = (ctx->slot + 1) % kHistCap;
  double *acc = force_slot(ctx, ctx->slot);
  CK(cudaMemsetAsync(acc, 0, sizeof(double) * kMaxSolids * 6, ctx->st));
  ibm_prepass(ctx, ctx->f[prev], true, acc, ctx->st);
  KArgs a = base_args(ctx);
  a.src = ctx->f[prev];
  a.dst = ctx->f[ctx->cur];
  sweep(ctx, OP_LOCAL_INIT, a);
  if (ctx->scheme.scheme == LBM_ZHAO_YONG) sweep(ctx, OP_ZY_SEED, a);
  if (ctx->outlet) sweep(ctx, OP_FACE_SEED, a);
  ctx->need_collide = false;
  ctx->prev_local = true;
  ctx->records = std::min<long long>(ctx->records + 1, kHistCap);
  return LBM_OK;
}

lbm_status prepare(lbm_ctx *ctx) {
  TRY(ensure_geometry(ctx));
  if (ctx->need_collide) TRY(init_collide(ctx));
  return LBM_OK;
}

// One step is step_begin (moving geometry, refill, the auxiliary stream's
// boundary and IBM work), the bulk sweep on the main stream, and step_end
// (join and solid motion); lbm_step_multi runs the bulk sweeps of several
// lattices between their begins and ends as one grouped launch.
struct StepState {
  KArgs a;
  bool ibm = false, moving = false, free_ = false, prefetch = false;
  int nxt = 0;
};

lbm_status step_begin(lbm_ctx *ctx, StepState &ss) {
  const bool moving = any_moving(ctx);
  const bool ibm = ctx->scheme.scheme == LBM_IBM_DIRECT;
  if (moving && ctx->scheme.scheme == LBM_ZHAO_YONG)
    return fail(ctx, LBM_ERR_UNSUPPORTED,
                "Eq. 16 keeps pre-collision values per boundary node: solids must not translate");
  const bool free_ = any_free(ctx);
  // IBM: the force of the previous step's pre-pass moves the free solids;
  // the others move with their prescribed velocity.  With a free solid all
  // of them move on the device (and are checked against the faces there).
  if (ibm && free_) {
    const int ms = ctx->motion_slot >= 0 ? ctx->motion_slot : ctx->slot;
    ctx->motion_slot = -1;
    TRY(motion_step(ctx, ms));
  }
  if (ibm && moving && !free_)
    for (auto &s : ctx->solids)
      for (int a = 0; a < 3; a++) s.c[a] += s.d.velocity[a];
  // free solids' next velocities are not known ahead: no prefetch
  const bool prefetch = moving && ctx->geom_prefetch && !free_;
  if (moving && ctx->nface && !free_) TRY(check_clearance(ctx));
  if (prefetch && ctx->gst) CK(cudaEventRecord(ctx->ev_gfree, ctx->st));
  if (moving && !take_prefetched(ctx)) TRY(rebuild_boxes(ctx));
  if (prefetch && !ctx->gst) {
    // first moving step: the spare set and its stream come into being
    TRY(alloc_spare(ctx));
    CK(cudaEventRecord(ctx->ev_gfree, ctx->st));
  }
  const int cur = ctx->cur, nxt = 1 - ctx->cur;
  KArgs a = base_args(ctx);
  if (moving && is_ibb(ctx->scheme.scheme)) {
    // refill nodes uncovered since the previous geometry (into f*(t))
    a.src = ctx->f[cur];
    a.dst = ctx->f[cur];
    sweep(ctx, OP_REFILL, a);
  }
  ctx->slot = (ctx->slot + 1) % kHistCap;
  double *acc = force_slot(ctx, ctx->slot);
  a = base_args(ctx);
  a.src = ctx->f[cur];
  a.dst = ctx->f[nxt];
  a.force_acc = acc;
  // fork: the boundary nodes (and the IBM pre-pass that feeds them) on the
  // auxiliary stream, the bulk nodes on the main stream; they read the same
  // f*(t) and write disjoint nodes of f*(t+1)
  CK(cudaEventRecord(ctx->ev_fork, ctx->st));
  CK(cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));
  // the IBM band-velocity kernel clears the record itself (one launch fewer
  // on the IBM lattice's critical chain); otherwise a memset does
  if (!ibm_zeroes_record(ctx)) CK(cudaMemsetAsync(acc, 0, sizeof(double) * kMaxSolids * 6, ctx->aux));
  ibm_prepass(ctx, ctx->f[cur], false, acc, ctx->aux);
  {
    Timed tm(ctx, TK_LIST, ctx->list_count >= 0 ? ctx->list_count : 0, ctx->aux);
    sweep(ctx, OP_LIST_SWEEP, a, ctx->aux);
  }
  // nodes next to non-periodic domain faces
  if (ctx->nface) sweep(ctx, OP_FACE_SWEEP, a, ctx->aux);
  ss.a = a;
  ss.ibm = ibm;
  ss.moving = moving;
  ss.free_ = free_;
  ss.prefetch = prefetch;
  ss.nxt = nxt;
  return LBM_OK;
}

void step_bulk(lbm_ctx *ctx, const StepState &ss) {
  Timed tm(ctx, TK_BULK, ctx->bulk_nodes, ctx->st);
  sweep(ctx, OP_BULK_SWEEP, ss.a, ctx->st);
}

lbm_status step_end(lbm_ctx *ctx, const StepState &ss) {
  const bool ibm = ss.ibm, moving = ss.moving, free_ = ss.free_, prefetch = ss.prefetch;
  const int nxt = ss.nxt;
  // join
  CK(cudaEventRecord(ctx->ev_join, ctx->aux));
  CK(cudaStreamWaitEvent(ctx->st, ctx->ev_join, 0));
  ctx->cur = nxt;
  ctx->prev_local = false;
  if (!ibm && moving && !free_)
    for (auto &s : ctx->solids)
      for (int k = 0; k < 3; k++) s.c[k] += s.d.velocity[k];
  // bounce-back: this step's momentum exchange moves the free solids (and
  // the others with them, on the device)
  if (!ibm && free_) TRY(motion_step(ctx, ctx->slot));
  if (prefetch) {
    // the next step's geometry: bounce-back uses the centres just reached,
    // IBM moves first and uses them plus one step
    double next[kMaxSolids][3];
    for (size_t k = 0; k < ctx->solids.size(); k++)
      for (int a = 0; a < 3; a++)
        next[k][a] = ctx->solids[k].c[a] + (ibm ? ctx->solids[k].d.velocity[a] : 0.0);
    TRY(prefetch_geometry(ctx, next));
  }
  ctx->records = std::min<long long>(ctx->records + 1, kHistCap);
  ctx->step++;
  return LBM_OK;
}

lbm_status step_once(lbm_ctx *ctx) {
  StepState ss;
  TRY(step_begin(ctx, ss));
  step_bulk(ctx, ss);
  return step_end(ctx, ss);
}

// The bulk sweeps of the lattices in `idx` (same lattice, collision and
// storage) as grouped launches of up to kMaxGroup lattices on the first
// one's stream; a lattice whose vector shape does not fit runs alone.
lbm_status step_bulk_group(lbm_ctx *const *ctxs, const std::vector<int> &idx,
                           std::vector<StepState> &ss) {
  for (size_t g0 = 0; g0 < idx.size(); g0 += kMaxGroup) {
    const size_t g1 = std::min(idx.size(), g0 + kMaxGroup);
    lbm_ctx *lead = ctxs[idx[g0]];
    lbm_ctx *ctx = lead;  // errors are reported on the group's first lattice
    if (g1 - g0 >= 2) {
      KArgs as[kMaxGroup];
      long long nodes = 0;
      for (size_t k = g0; k < g1; k++) {
        lbm_ctx *c = ctxs[idx[k]];
        as[k - g0] = ss[idx[k]].a;
        nodes += c->bulk_nodes;
        if (c->st != lead->st) {
          CK(cudaEventRecord(c->ev_grp, c->st));
          CK(cudaStreamWaitEvent(lead->st, c->ev_grp, 0));
        }
      }
      bool ok;
      {
        Timed tm(lead, TK_BULK, nodes, lead->st);
        ok = launch_bulk_group(as, (int)(g1 - g0), lead->d.lattice, lead->coll_mode,
                               lead->d.precision, lead->st);
      }
      if (ok) {
        lead->launches++;
        CK(cudaEventRecord(lead->ev_grp, lead->st));
        for (size_t k = g0 + 1; k < g1; k++) {
          lbm_ctx *c = ctxs[idx[k]];
          if (c->st != lead->st) CK(cudaStreamWaitEvent(c->st, lead->ev_grp, 0));
        }
        continue;
      }
    }
    for (size_t k = g0; k < g1; k++) step_bulk(ctxs[idx[k]], ss[idx[k]]);
  }
  return LBM_OK;
}

// ||u - u_snap||_2 / ||u||_2 from the two reduced sums; NaN when either sum
// is not finite (a diverged field must not read as converged), 0 for a
// field at rest.
double residual_of(const double h[2]) {
  if (!std::isfinite(h[0]) || !std::isfinite(h[1])) return NAN;
  return h[1] > 0 ? sqrt(h[0] / h[1]) : 0.0;
}

// The copy stream and its events (asynchronous force copies, uploads).
lbm_status ensure_copy_stream(lbm_ctx *ctx) {
  if (ctx->cst) return LBM_OK;
  cudaStream_t s = nullptr;
  CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  ctx->cst = s;
  for (cudaEvent_t *e : {&ctx->ev_rec, &ctx->ev_cst, &ctx->ev_up_start, &ctx->ev_up_copy[0],
                         &ctx->ev_up_copy[1], &ctx->ev_up_conv[0], &ctx->ev_up_conv[1]})
    CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  return LBM_OK;
}

lbm_status qbuf_ensure(lbm_ctx *ctx, size_t elems) {
  if (elems <= ctx->qbuf_elems) return LBM_OK;
  dfree(ctx, ctx->qbuf);
  ctx->qbuf = nullptr;
  ctx->qbuf_elems = 0;
  TRY(dalloc(ctx, (void **)&ctx->qbuf, elems * sizeof(double)));
  ctx->qbuf_elems = elems;
  return LBM_OK;
}

// Run the query kernels with the given FP64 device outputs (pre-zeroed).
void run_query(lbm_ctx *ctx, KArgs a) {
  a.src = ctx->f[1 - ctx->cur];
  if (ctx->prev_local) {
    a.local_gather = 1;
    sweep(ctx, OP_LOCAL_QUERY, a);
  } else {
    a.local_gather = 0;
    sweep(ctx, OP_BULK_QUERY, a);
    sweep(ctx, OP_LIST_QUERY, a);
    if (ctx->nface) sweep(ctx, OP_FACE_QUERY, a);
  }
}

enum QueryKind { Q_RHO, Q_U, Q_S, Q_STRESS, Q_F, Q_EPS };

// The field into host memory: enqueued on the context's stream, then (wait)
// waited for.
lbm_status query(lbm_ctx *ctx, QueryKind kind, double *host, size_t n, bool wait = true) {
  if (!ctx) return LBM_ERR_ARG;
  const int nc = ctx->D == 2 ? 3 : 6;
  size_t comps = (kind == Q_RHO || kind == Q_EPS) ? 1 : kind == Q_U ? ctx->D : kind == Q_F ? ctx->Q : nc;
  const size_t need = comps * (size_t)ctx->N;
  if (!host || n < need) return fail(ctx, LBM_ERR_ARG, "output buffer too small: need " + std::to_string(need));
  TRY(prepare(ctx));
  TRY(qbuf_ensure(ctx, need));
  CK(cudaMemsetAsync(ctx->qbuf, 0, need * sizeof(double), ctx->st));
  KArgs a = base_args(ctx);
  switch (kind) {
  case Q_RHO: a.out_rho = ctx->qbuf; break;
  case Q_U: a.out_u = ctx->qbuf; break;
  case Q_S: a.out_S = ctx->qbuf; break;
  case Q_STRESS: a.out_stress = ctx->qbuf; break;
  case Q_EPS: a.out_eps = ctx->qbuf; break;
  case Q_F: a.out_f = ctx->qbuf; break;
  }
  run_query(ctx, a);
  CK(cudaMemcpyAsync(host, ctx->qbuf, need * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  if (wait) CK(cudaStreamSynchronize(ctx->st));
  CK(cudaGetLastError());
  return LBM_OK;
}

lbm_status velocity_to(lbm_ctx *ctx, double *dev) {
  CK(cudaMemsetAsync(dev, 0, sizeof(double) * ctx->D * ctx->N, ctx->st));
  KArgs a = base_args(ctx);
  a.out_u = dev;
  run_query(ctx, a);
  return LBM_OK;
}

void set_collision_constants(lbm_ctx *ctx) {
  const lbm_lattice_desc &d = ctx->d;
  ctx->omega = 1.0 / d.tau;
  ctx->nu = (d.tau - 0.5) / 3.0;
  const double sq = 1.0 / (0.5 + (3.0 / 16.0) / (d.tau - 0.5));
  // kinds of the moment rows (see include/lbm.h): c conserved, b energy,
  // e energy square, q energy flux, v stress, p / m ghosts
  const char *k9 = "cbecqcqvv", *k19 = "cbecqcqcqvpvpvvvmmm";
  const char *kind = d.lattice == LBM_D2Q9 ? k9 : k19;
  for (int k = 0; k < 19; k++) ctx->ds[k] = 0;
  ctx->s_bulk = ctx->omega;
  if (d.collision == LBM_MRT) {
    for (int k = 0; k < ctx->Q; k++) {
      double s = kind[k] == 'q' ? sq : ctx->omega;
      if (kind[k] != 'v' && kind[k] != 'c' && d.mrt_rates[k] != 0) s = d.mrt_rates[k];
      if (kind[k] != 'c') ctx->ds[k] = ctx->omega - s;
      if (kind[k] == 'b') ctx->s_bulk = s;
    }
  }
  ctx->inv_scale = d.precision == LBM_FP32_FP16STORE ? 1.0 / kFp16Scale : 1.0;
  // kernel variant: MRT whose only non-BGK moments are the q moments (one
  // common rate, the default) runs a cheaper in-place correction
  ctx->coll_mode = CM_BGK;
  if (d.collision == LBM_MRT) {
    bool q_only = true;
    double dq = 0;
    bool have_q = false;
    for (int k = 0; k < ctx->Q; k++) {
      if (kind[k] == 'q') {
        if (!have_q) {
          dq = ctx->ds[k];
          have_q = true;
        } else if (ctx->ds[k] != dq) {
          q_only = false;
        }
      } else if (ctx->ds[k] != 0) {
        q_only = false;
      }
    }
    ctx->coll_mode = q_only ? (dq != 0 ? CM_MRT_Q : CM_BGK) : CM_MRT;
  }
}

}  // namespace

// ===================================================================== ABI
extern "C" {

void lbm_debug_fail_allocations_after(long long n) { g_alloc_budget.store(n < 0 ? -1 : n); }

const char *lbm_version(void) { return "lbm-gb300 0.1 (sm_103a)"; }

const char *lbm_last_error(const lbm_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

// ---- staging array of lbm_get_velocity_noalloc
//
// 2^20 doubles (8 MiB) compiled into the library, shared by all contexts and
// all calls on a device.  Host code may not take the address of a __device__
// variable directly: lbm_create looks it up once per device, with that
// device current, and caches it.  The lookup also loads this file's module
// (CUDA loads modules lazily), so the 8 MiB is committed on the device by
// its first lbm_create, not by a later query.
static constexpr size_t kNoAllocScratchDoubles = size_t(1) << 20;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];
static constexpr int kNoAllocMaxDevices = 64;
static double *g_noalloc_addr[kNoAllocMaxDevices] = {nullptr};
static std::mutex g_noalloc_mu;

static cudaError_t noalloc_lookup(int dev) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaSuccess;  // the query refuses it
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_addr[dev]) return cudaSuccess;
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e == cudaSuccess) g_noalloc_addr[dev] = (double *)p;
  return e;
}

lbm_status lbm_create(lbm_ctx **out, const lbm_lattice_desc *desc, void *cuda_stream) {
  if (!out || !desc) return LBM_ERR_ARG;
  *out = nullptr;
  const lbm_lattice_desc &d = *desc;
  if (d.lattice != LBM_D2Q9 && d.lattice != LBM_D3Q19) return LBM_ERR_ARG;
  if (d.nx < 1 || d.ny < 1 || (d.lattice == LBM_D3Q19 && d.nz < 1)) return LBM_ERR_ARG;
  if (!(d.tau > 0.5) || !(d.tau < 1e6)) return LBM_ERR_ARG;
  if (d.collision != LBM_BGK && d.collision != LBM_MRT) return LBM_ERR_ARG;
  if (d.precision < LBM_FP64 || d.precision > LBM_FP32_FP16STORE) return LBM_ERR_ARG;
  const long long N = (long long)d.nx * d.ny * (d.lattice == LBM_D2Q9 ? 1 : d.nz);
  if (N > (1LL << 31) - 1) return LBM_ERR_UNSUPPORTED;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return LBM_ERR_CUDA;
  }
  lbm_ctx *ctx = new lbm_ctx();
  ctx->d = d;
  if (d.lattice == LBM_D2Q9) ctx->d.nz = 1;
  ctx->Q = d.lattice == LBM_D2Q9 ? 9 : 19;
  ctx->D = d.lattice == LBM_D2Q9 ? 2 : 3;
  ctx->N = N;
  ctx->st = (cudaStream_t)cuda_stream;
  cudaGetDevice(&ctx->device);
  if (noalloc_lookup(ctx->device) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return LBM_ERR_CUDA;
  }
  {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    // high priority: the boundary and IBM kernels start with the bulk sweep
    // (at the default priority they start late and the join waits on them)
    // LBM_AUX_PRIORITY: 0 lowest, 1 default, 2 highest (the default)
    int prio = hi;
    if (const char *e = getenv("LBM_AUX_PRIORITY")) prio = atoi(e) == 0 ? lo : atoi(e) == 1 ? 0 : hi;
    if (cudaStreamCreateWithPriority(&ctx->aux, cudaStreamNonBlocking, prio) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_grp, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      lbm_destroy(ctx);
      return LBM_ERR_CUDA;
    }
  }
  ctx->ssz = d.precision == LBM_FP64 ? 8 : d.precision == LBM_FP32 ? 4 : 2;
  ctx->tsz = d.precision == LBM_FP64 ? 8 : 4;
  set_collision_constants(ctx);
  // Direction arrays are spaced by an odd number of 128-byte lines beyond a
  // whole number of line pairs, so that the Q read and Q write streams of a
  // warp do not fall on the same cache sets and memory channels when the
  // node count is a power of two.  LBM_DIR_PAD_LINES overrides the padding
  // (0: arrays back to back), LBM_BULK_BLOCK the bulk block width.
  {
    const long long line = 128 / (long long)ctx->ssz;
    long long pad = 1;
    if (const char *e = getenv("LBM_DIR_PAD_LINES")) pad = atoll(e);
    ctx->fs = pad <= 0 ? N : ((N + 2 * line - 1) / (2 * line)) * (2 * line) + pad * line;
    if (const char *e = getenv("LBM_BULK_BLOCK")) {
      const int b = atoi(e);
      if (b >= 32 && b <= 512 && b % 32 == 0) ctx->bulk_block = b;
    }
    if (const char *e = getenv("LBM_CACHE_HINTS")) ctx->cache_hints = atoi(e) & 3;
    if (const char *e = getenv("LBM_LIST_BLOCK")) {
      const int v = atoi(e);
      if (v == 32 || v == 64 || v == 128 || v == 256) ctx->list_block = v;
    }
    if (const char *e = getenv("LBM_BULK_MODE")) ctx->bulk_mode = atoi(e);
    if (const char *e = getenv("LBM_VEC_WORDS")) ctx->bulk_vec_words = atoi(e);
    if (const char *e = getenv("LBM_GEOM_PREFETCH")) ctx->geom_prefetch = atoi(e) != 0;
    if (const char *e = getenv("LBM_VEC_PACKED")) ctx->bulk_vec_packed = atoi(e);
    if (const char *e = getenv("LBM_IBM_LIST_THREAD")) ctx->ibm_list_thread = atoi(e) != 0;
    if (const char *e = getenv("LBM_IBM_CLUSTER")) ctx->ibm_cluster_on = atoi(e) != 0;
    if (const char *e = getenv("LBM_IBB_LIST_THREAD")) ctx->ibb_list_thread = atoi(e) != 0;
    if (const char *e = getenv("LBM_MRT_GENERAL"))
      if (atoi(e) && ctx->coll_mode == CM_MRT_Q) ctx->coll_mode = CM_MRT;
  }
  lbm_status s = LBM_OK;
  const size_t fbytes = (size_t)ctx->Q * ctx->fs * ctx->ssz;
  const size_t padN = ((N + 15) / 16) * 16;
  if ((s = dalloc(ctx, &ctx->f[0], fbytes)) != LBM_OK ||
      (s = dalloc(ctx, &ctx->f[1], fbytes)) != LBM_OK ||
      (s = dalloc(ctx, (void **)&ctx->flags, padN)) != LBM_OK ||
      (s = dalloc(ctx, (void **)&ctx->sid, 2 * padN)) != LBM_OK ||
      (s = dalloc(ctx, (void **)&ctx->counts, 16 * sizeof(int))) != LBM_OK ||
      (s = dalloc(ctx, (void **)&ctx->hist, sizeof(double) * kHistCap * kMaxSolids * 6)) != LBM_OK ||
      (s = dalloc(ctx, (void **)&ctx->red2, 2 * sizeof(double))) != LBM_OK) {
    lbm_destroy(ctx);
    return s;
  }
  cudaMemsetAsync(ctx->flags, 0, padN, ctx->st);
  cudaMemsetAsync(ctx->sid, 0, 2 * padN, ctx->st);
  cudaMemsetAsync(ctx->counts, 0, 16 * sizeof(int), ctx->st);
  cudaMemsetAsync(ctx->hist, 0, sizeof(double) * kHistCap * kMaxSolids * 6, ctx->st);
  // rest state f = w as a pre-collision state, collided on first use
  KArgs a = base_args(ctx);
  a.dst = ctx->f[1];
  a.omega = 1.0;  // rho
  a.g[0] = a.g[1] = a.g[2] = 0;
  sweep(ctx, OP_FILL_EQ, a);
  ctx->cur = 0;
  ctx->need_collide = true;
  ctx->prev_local = true;
  cudaError_t e = cudaStreamSynchronize(ctx->st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    lbm_destroy(ctx);
    return LBM_ERR_CUDA;
  }
  *out = ctx;
  return LBM_OK;
}

void lbm_destroy(lbm_ctx *ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->st);
  if (ctx->aux) {
    cudaStreamSynchronize(ctx->aux);
    cudaStreamDestroy(ctx->aux);
  }
  if (ctx->gst) {
    cudaStreamSynchronize(ctx->gst);
    cudaStreamDestroy(ctx->gst);
  }
  if (ctx->ev_geom) cudaEventDestroy(ctx->ev_geom);
  if (ctx->ev_gfree) cudaEventDestroy(ctx->ev_gfree);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->ev_grp) cudaEventDestroy(ctx->ev_grp);
  if (ctx->cst) {
    cudaStreamSynchronize(ctx->cst);
    cudaStreamDestroy(ctx->cst);
  }
  if (ctx->ev_rec) cudaEventDestroy(ctx->ev_rec);
  if (ctx->ev_cst) cudaEventDestroy(ctx->ev_cst);
  for (cudaEvent_t e : {ctx->ev_up_start, ctx->ev_up_copy[0], ctx->ev_up_copy[1],
                        ctx->ev_up_conv[0], ctx->ev_up_conv[1]})
    if (e) cudaEventDestroy(e);
  for (void *p : ctx->allocs) cudaFree(p);
  for (auto &p : ctx->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : ctx->free_events) cudaEventDestroy(e);
  delete ctx;
}

lbm_status lbm_add_solid(lbm_ctx *ctx, const lbm_solid_desc *solid, int *solid_id) {
  if (ctx) ctx->gen++;
  if (!ctx || !solid) return LBM_ERR_ARG;
  TRY(solids_to_host(ctx, true));
  if ((int)ctx->solids.size() >= kMaxSolids) return fail(ctx, LBM_ERR_CAPACITY, "at most 8 solids");
  if (solid->kind != LBM_SPHERE && solid->kind != LBM_CYLINDER_Z)
    return fail(ctx, LBM_ERR_ARG, "unknown solid kind");
  if (!(solid->radius > 0)) return fail(ctx, LBM_ERR_ARG, "radius must be positive");
  SolidHost h;
  h.d = *solid;
  if (ctx->D == 2) {
    h.d.centre[2] = 0;
    h.d.velocity[2] = 0;
    h.d.omega[0] = h.d.omega[1] = 0;
  }
  memcpy(h.c, h.d.centre, sizeof(h.c));
  memcpy(h.cg, h.d.centre, sizeof(h.cg));
  ctx->solids.push_back(h);
  if (solid_id) *solid_id = (int)ctx->solids.size() - 1;
  ctx->geom_dirty = true;
  return LBM_OK;
}

lbm_status lbm_set_solid_motion(lbm_ctx *ctx, int id, const double centre[3], const double vel[3],
                                const double omega[3]) {
  if (ctx) ctx->gen++;
  if (!ctx || id < 0 || id >= (int)ctx->solids.size()) return LBM_ERR_ARG;
  TRY(solids_to_host(ctx, true));
  SolidHost &h = ctx->solids[id];
  for (int a = 0; a < 3; a++) {
    if (centre) h.c[a] = h.d.centre[a] = centre[a];
    if (vel) h.d.velocity[a] = vel[a];
    if (omega) h.d.omega[a] = omega[a];
  }
  if (ctx->D == 2) {
    h.c[2] = h.d.centre[2] = 0;
    h.d.velocity[2] = 0;
    h.d.omega[0] = h.d.omega[1] = 0;
  }
  // wall velocities are stored with the links: rebuild
  ctx->geom_dirty = true;
  return LBM_OK;
}

lbm_status lbm_set_scheme(lbm_ctx *ctx, const lbm_scheme_desc *scheme) {
  if (ctx) ctx->gen++;
  if (!ctx || !scheme) return LBM_ERR_ARG;
  if (scheme->scheme < LBM_SCHEME_NONE || scheme->scheme > LBM_ZHAO_YONG)
    return fail(ctx, LBM_ERR_ARG, "unknown scheme");
  if (scheme->ibm_iters < 0 || scheme->ibm_retraction < 0 || scheme->ibm_marker_density < 0)
    return fail(ctx, LBM_ERR_ARG, "negative IBM parameter");
  if (scheme->ibm_kernel < LBM_DELTA_PESKIN4 || scheme->ibm_kernel > LBM_DELTA_COSINE4)
    return fail(ctx, LBM_ERR_ARG, "unknown delta-function kernel");
  if (scheme->ibm_inertia < LBM_INERTIA_FENG || scheme->ibm_inertia > LBM_INERTIA_UHLMANN)
    return fail(ctx, LBM_ERR_ARG, "unknown inside-fluid treatment");
  if (scheme->scheme == LBM_IBM_DIRECT && scheme->ibm_inertia == LBM_INERTIA_UHLMANN)
    for (auto &h : ctx->solids)
      if (h.rho_p > 0 && h.rho_p <= 1.0)
        return fail(ctx, LBM_ERR_ARG, "Eq. 22 needs a solid denser than the fluid");
  if (scheme->scheme == LBM_ZHAO_YONG && !ctx->need_collide && !ctx->prev_local)
    return fail(ctx, LBM_ERR_STATE,
                "select Eq. 16 before stepping, or after lbm_init_equilibrium / "
                "lbm_set_distributions (its boundary state starts from a pre-collision state)");
  TRY(solids_to_host(ctx, true));
  if (scheme->scheme == LBM_ZHAO_YONG && !ctx->zy_pre) {
    TRY(dalloc(ctx, &ctx->zy_pre, (size_t)ctx->Q * ctx->fs * ctx->tsz));
    CK(cudaMemsetAsync(ctx->zy_pre, 0, (size_t)ctx->Q * ctx->fs * ctx->tsz, ctx->st));
  }
  ctx->scheme = *scheme;
  ctx->geom_dirty = true;
  for (auto &h : ctx->solids) h.have_Ip = false;
  // the boundary nodes' pre-collision values are seeded by the next
  // initial collision, from the pre-collision state held locally
  if (scheme->scheme == LBM_ZHAO_YONG) ctx->need_collide = true;
  return LBM_OK;
}

lbm_status lbm_init_equilibrium(lbm_ctx *ctx, double rho, const double u[3]) {
  if (ctx) ctx->gen++;
  if (!ctx || !(rho > 0)) return LBM_ERR_ARG;
  TRY(ensure_geometry(ctx));
  KArgs a = base_args(ctx);
  a.dst = ctx->f[1 - ctx->cur];
  a.omega = rho;
  for (int k = 0; k < 3; k++) a.g[k] = u ? u[k] : 0.0;
  if (ctx->D == 2) a.g[2] = 0;
  sweep(ctx, OP_FILL_EQ, a);
  ctx->need_collide = true;
  ctx->prev_local = true;
  return LBM_OK;
}

namespace {

// Upload of full FP64 populations [Q][nodes] into the pre-collision slot
// f[1-cur].  The other array, f[cur], holds nothing that is read again
// before the initial collision rewrites it, so two staging slots of up to
// 2^20 doubles are carved out of it: no device allocation.  Slot k % 2
// takes chunk k (one direction, a run of nodes) on the copy stream; the
// conversion to stored deviations runs on the context's stream after that
// copy, and the copy of chunk k + 2 waits for the conversion of chunk k.
lbm_status upload_f(lbm_ctx *ctx, const double *host_f) {
  TRY(ensure_geometry(ctx));
  TRY(ensure_copy_stream(ctx));
  const long long N = ctx->N;
  const size_t fbytes = (size_t)ctx->Q * ctx->fs * ctx->ssz;
  const long long C = std::max<long long>(
      1, std::min<long long>(1LL << 20, (long long)(fbytes / (2 * sizeof(double)))));
  double *stage[2] = {(double *)ctx->f[ctx->cur], (double *)ctx->f[ctx->cur] + C};
  void *dst = ctx->f[1 - ctx->cur];
  // the staging array is free once the work already on the stream is done
  CK(cudaEventRecord(ctx->ev_up_start, ctx->st));
  CK(cudaStreamWaitEvent(ctx->cst, ctx->ev_up_start, 0));
  long long k = 0;
  for (int i = 0; i < ctx->Q; i++) {
    const double w = ctx->D == 2 ? Lat<0>::w(i) : Lat<1>::w(i);
    for (long long n0 = 0; n0 < N; n0 += C, k++) {
      const int sl = (int)(k & 1);
      const long long len = std::min(C, N - n0);
      if (k >= 2) CK(cudaStreamWaitEvent(ctx->cst, ctx->ev_up_conv[sl], 0));
      CK(cudaMemcpyAsync(stage[sl], host_f + (size_t)i * N + n0, (size_t)len * sizeof(double),
                         cudaMemcpyHostToDevice, ctx->cst));
      CK(cudaEventRecord(ctx->ev_up_copy[sl], ctx->cst));
      CK(cudaStreamWaitEvent(ctx->st, ctx->ev_up_copy[sl], 0));
      UploadArgs u;
      u.src = stage[sl];
      u.dst = (char *)dst + (size_t)i * ctx->fs * ctx->ssz;
      u.flags = ctx->flags;
      u.n0 = n0;
      u.len = len;
      u.w = w;
      u.inv_scale = ctx->inv_scale;
      launch_upload_chunk(u, ctx->d.precision, ctx->st);
      ctx->launches++;
      CK(cudaEventRecord(ctx->ev_up_conv[sl], ctx->st));
    }
  }
  CK(cudaGetLastError());
  ctx->need_collide = true;
  ctx->prev_local = true;
  return LBM_OK;
}

}  // namespace

lbm_status lbm_set_distributions(lbm_ctx *ctx, const double *host_f, size_t n) {
  if (ctx) ctx->gen++;
  if (!ctx || !host_f) return LBM_ERR_ARG;
  if (n < (size_t)ctx->Q * ctx->N) return fail(ctx, LBM_ERR_ARG, "input must hold Q * nodes doubles");
  TRY(upload_f(ctx, host_f));
  CK(cudaStreamSynchronize(ctx->st));
  return LBM_OK;
}

lbm_status lbm_set_distributions_async(lbm_ctx *ctx, const double *host_f, size_t n) {
  if (ctx) ctx->gen++;
  if (!ctx || !host_f) return LBM_ERR_ARG;
  if (n < (size_t)ctx->Q * ctx->N) return fail(ctx, LBM_ERR_ARG, "input must hold Q * nodes doubles");
  return upload_f(ctx, host_f);
}

lbm_status lbm_get_distributions(lbm_ctx *ctx, double *host_f, size_t n) {
  return query(ctx, Q_F, host_f, n);
}

lbm_status lbm_step(lbm_ctx *ctx, int nsteps) {
  if (!ctx || nsteps < 0) return LBM_ERR_ARG;
  TRY(prepare(ctx));
  for (int k = 0; k < nsteps; k++) TRY(step_once(ctx));
  CK(cudaGetLastError());
  return LBM_OK;
}

lbm_status lbm_step_multi(lbm_ctx *const *ctxs, int n, int nsteps) {
  if (!ctxs || n < 1 || nsteps < 0) return LBM_ERR_ARG;
  for (int i = 0; i < n; i++) {
    if (!ctxs[i]) return LBM_ERR_ARG;
    for (int j = 0; j < i; j++)
      if (ctxs[j] == ctxs[i]) return fail(ctxs[i], LBM_ERR_ARG, "a lattice appears twice");
  }
  for (int i = 0; i < n; i++) TRY(prepare(ctxs[i]));
  // lattices that can share a bulk launch: same lattice, collision and storage
  std::vector<std::vector<int>> groups;
  for (int i = 0; i < n; i++) {
    bool placed = false;
    for (auto &g : groups) {
      const lbm_ctx *c = ctxs[g[0]];
      if (c->d.lattice == ctxs[i]->d.lattice && c->coll_mode == ctxs[i]->coll_mode &&
          c->d.precision == ctxs[i]->d.precision && c->device == ctxs[i]->device) {
        g.push_back(i);
        placed = true;
        break;
      }
    }
    if (!placed) groups.push_back({i});
  }
  std::vector<StepState> ss(n);
  for (int k = 0; k < nsteps; k++) {
    for (int i = 0; i < n; i++) TRY(step_begin(ctxs[i], ss[i]));
    for (auto &g : groups) {
      lbm_status st = step_bulk_group(ctxs, g, ss);
      if (st != LBM_OK) return st;
    }
    for (int i = 0; i < n; i++) TRY(step_end(ctxs[i], ss[i]));
  }
  for (int i = 0; i < n; i++) {
    lbm_ctx *ctx = ctxs[i];
    CK(cudaGetLastError());
  }
  return LBM_OK;
}

lbm_status lbm_run_to_steady(lbm_ctx *ctx, double tol, int check_every, int max_steps,
                             int *steps_done, double *residual) {
  if (!ctx || check_every < 1 || max_steps < 0) return LBM_ERR_ARG;
  TRY(prepare(ctx));
  // each buffer on its own: a failed allocation leaves no half-made pair
  if (!ctx->u_now) TRY(dalloc(ctx, (void **)&ctx->u_now, sizeof(double) * ctx->D * ctx->N));
  if (!ctx->u_snap) TRY(dalloc(ctx, (void **)&ctx->u_snap, sizeof(double) * ctx->D * ctx->N));
  TRY(velocity_to(ctx, ctx->u_snap));
  int done = 0;
  double r = INFINITY;
  lbm_status st = LBM_OK;
  while (done < max_steps) {
    const int k = std::min(check_every, max_steps - done);
    for (int j = 0; j < k; j++) TRY(step_once(ctx));
    done += k;
    TRY(velocity_to(ctx, ctx->u_now));
    launch_residual(ctx->u_now, ctx->u_snap, 0, ctx->flags, ctx->N, ctx->D, ctx->red2, ctx->st);
    ctx->launches++;
    double h[2];
    CK(cudaMemcpyAsync(h, ctx->red2, sizeof(h), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    r = residual_of(h);
    ctx->last_residual = r;
    if (!std::isfinite(r)) {
      st = fail(ctx, LBM_ERR_DIVERGED, "non-finite residual");
      break;
    }
    if (r < tol) break;
    std::swap(ctx->u_now, ctx->u_snap);
  }
  if (steps_done) *steps_done = done;
  if (residual) *residual = r;
  return st;
}

lbm_status lbm_get_density(lbm_ctx *ctx, double *o, size_t n) { return query(ctx, Q_RHO, o, n); }
lbm_status lbm_get_velocity(lbm_ctx *ctx, double *o, size_t n) { return query(ctx, Q_U, o, n); }
lbm_status lbm_get_velocity_async(lbm_ctx *ctx, double *o, size_t n) {
  return query(ctx, Q_U, o, n, false);
}
lbm_status lbm_get_strain_rate(lbm_ctx *ctx, double *o, size_t n) { return query(ctx, Q_S, o, n); }
lbm_status lbm_get_stress(lbm_ctx *ctx, double *o, size_t n) { return query(ctx, Q_STRESS, o, n); }
lbm_status lbm_get_dissipation(lbm_ctx *ctx, double *o, size_t n) { return query(ctx, Q_EPS, o, n); }

lbm_status lbm_get_solid_mask(lbm_ctx *ctx, unsigned char *host_out, size_t n) {
  if (!ctx || !host_out || n < (size_t)ctx->N) return LBM_ERR_ARG;
  TRY(prepare(ctx));
  std::vector<uint8_t> fl(ctx->N);
  CK(cudaMemcpyAsync(fl.data(), ctx->flags, ctx->N, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  for (long long k = 0; k < ctx->N; k++) host_out[k] = (fl[k] & FL_SOLID) ? 1 : 0;
  return LBM_OK;
}

lbm_status lbm_get_force_torque(lbm_ctx *ctx, int id, double F[3], double T[3]) {
  if (!ctx || id < 0 || id >= (int)ctx->solids.size()) return LBM_ERR_ARG;
  TRY(prepare(ctx));
  double h[6];
  CK(cudaMemcpyAsync(h, force_slot(ctx, ctx->slot) + 6 * id, sizeof(h), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  CK(cudaGetLastError());
  for (int a = 0; a < 3; a++) {
    if (F) F[a] = h[a];
    if (T) T[a] = h[3 + a];
  }
  return LBM_OK;
}

lbm_status lbm_copy_force_torque_async(lbm_ctx *ctx, int id, double *host_out) {
  if (!ctx || !host_out || id < 0 || id >= (int)ctx->solids.size()) return LBM_ERR_ARG;
  TRY(prepare(ctx));
  TRY(ensure_copy_stream(ctx));
  CK(cudaEventRecord(ctx->ev_rec, ctx->st));
  CK(cudaStreamWaitEvent(ctx->cst, ctx->ev_rec, 0));
  CK(cudaMemcpyAsync(host_out, force_slot(ctx, ctx->slot) + 6 * id, 6 * sizeof(double),
                     cudaMemcpyDeviceToHost, ctx->cst));
  // the record ring holds kHistCap steps: keep the copies well behind it
  if (++ctx->copies % 1024 == 0) {
    CK(cudaEventRecord(ctx->ev_cst, ctx->cst));
    CK(cudaStreamWaitEvent(ctx->st, ctx->ev_cst, 0));
  }
  return LBM_OK;
}

lbm_status lbm_get_force_history(lbm_ctx *ctx, int id, double *host_out, size_t max_steps, size_t *n) {
  if (!ctx || id < 0 || id >= (int)ctx->solids.size() || !n) return LBM_ERR_ARG;
  TRY(prepare(ctx));
  const long long have = std::min<long long>(ctx->records, (long long)max_steps);
  std::vector<double> all((size_t)kHistCap * kMaxSolids * 6);
  CK(cudaMemcpyAsync(all.data(), ctx->hist, all.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  for (long long k = 0; k < have; k++) {
    const int slot = (int)(((ctx->slot - (have - 1 - k)) % kHistCap + kHistCap) % kHistCap);
    if (host_out) memcpy(host_out + 6 * k, &all[((size_t)slot * kMaxSolids + id) * 6], 6 * sizeof(double));
  }
  *n = (size_t)have;
  return LBM_OK;
}

lbm_status lbm_get_residual(lbm_ctx *ctx, double *r) {
  if (!ctx || !r) return LBM_ERR_ARG;
  *r = ctx->last_residual;
  return LBM_OK;
}

lbm_status lbm_set_domain(lbm_ctx *ctx, const lbm_domain_desc *dom) {
  if (ctx) ctx->gen++;
  if (!ctx) return LBM_ERR_ARG;
  TRY(solids_to_host(ctx, false));
  lbm_domain_desc d{};
  if (dom) d = *dom;
  const int len[3] = {ctx->d.nx, ctx->d.ny, ctx->D == 2 ? 1 : ctx->d.nz};
  int conv = -1, open_axes = 0;
  for (int k = 0; k < 6; k++) {
    if (d.type[k] < LBM_FACE_PERIODIC || d.type[k] > LBM_FACE_CONVECTIVE)
      return fail(ctx, LBM_ERR_ARG, "unknown face type");
    for (int c = 0; c < 3; c++)
      if (!(d.u[k][c] == d.u[k][c])) return fail(ctx, LBM_ERR_ARG, "face velocity is NaN");
    if (d.type[k] == LBM_FACE_CONVECTIVE) {
      if (conv >= 0) return fail(ctx, LBM_ERR_ARG, "at most one convective outflow face");
      conv = k;
    }
  }
  for (int a = 0; a < 3; a++) {
    const bool lo = d.type[2 * a] != LBM_FACE_PERIODIC, hi = d.type[2 * a + 1] != LBM_FACE_PERIODIC;
    if (lo != hi) return fail(ctx, LBM_ERR_ARG, "periodic faces come in pairs");
    if (!lo) continue;
    if (a == 2 && ctx->D == 2) return fail(ctx, LBM_ERR_ARG, "a 2D lattice has no z faces");
    if (len[a] < 3) return fail(ctx, LBM_ERR_ARG, "a non-periodic axis needs at least 3 nodes");
    open_axes |= 1 << a;
  }
  if (conv >= 0 && !ctx->need_collide)
    return fail(ctx, LBM_ERR_STATE,
                "an outflow face is set before stepping or right after an initialisation");
  CK(cudaStreamSynchronize(ctx->st));
  // nodes next to a non-periodic face, in node order
  std::vector<int> nodes;
  if (open_axes)
    for (long long n = 0; n < ctx->N; n++) {
      const int x = (int)(n % len[0]), y = (int)((n / len[0]) % len[1]),
                z = (int)(n / ((long long)len[0] * len[1]));
      const int c[3] = {x, y, z};
      bool on = false;
      for (int a = 0; a < 3 && !on; a++)
        on = ((open_axes >> a) & 1) && (c[a] == 0 || c[a] == len[a] - 1);
      if (on) nodes.push_back((int)n);
    }
  dfree(ctx, ctx->face_node);
  dfree(ctx, ctx->outlet);
  ctx->face_node = nullptr;
  ctx->outlet = nullptr;
  ctx->nface = 0;
  ctx->out_face = -1;
  ctx->out_area = 0;
  // periodic until the new faces' arrays exist
  ctx->dom = lbm_domain_desc{};
  ctx->geom_dirty = true;
  if (!nodes.empty()) {
    TRY(dalloc(ctx, (void **)&ctx->face_node, nodes.size() * sizeof(int)));
    CK(cudaMemcpy(ctx->face_node, nodes.data(), nodes.size() * sizeof(int), cudaMemcpyHostToDevice));
    ctx->nface = (int)nodes.size();
  }
  if (conv >= 0) {
    const int a = conv / 2;
    ctx->out_face = conv;
    ctx->out_area = a == 0 ? (long long)len[1] * len[2] : a == 1 ? (long long)len[0] * len[2]
                                                                  : (long long)len[0] * len[1];
    const size_t bytes = (size_t)(ctx->Q + 1) * ctx->out_area * ctx->tsz;
    TRY(dalloc(ctx, &ctx->outlet, bytes));
    CK(cudaMemset(ctx->outlet, 0, bytes));
  }
  ctx->dom = d;
  ctx->geom_dirty = true;
  return LBM_OK;
}

lbm_status lbm_set_solid_dynamics(lbm_ctx *ctx, int id, double density_ratio,
                                  const double gravity[3]) {
  if (ctx) ctx->gen++;
  if (!ctx || id < 0 || id >= (int)ctx->solids.size() || !(density_ratio == density_ratio))
    return LBM_ERR_ARG;
  if (density_ratio > 0 && ctx->scheme.scheme != LBM_IBM_DIRECT && !is_ibb(ctx->scheme.scheme))
    return fail(ctx, LBM_ERR_STATE, "free solids need a bounce-back or IBM scheme (set it first)");
  if (density_ratio > 0 && ctx->scheme.scheme == LBM_ZHAO_YONG)
    return fail(ctx, LBM_ERR_UNSUPPORTED, "Eq. 16 does not take translating solids");
  if (density_ratio > 0 && density_ratio <= 1.0 && ctx->scheme.scheme == LBM_IBM_DIRECT &&
      ctx->scheme.ibm_inertia == LBM_INERTIA_UHLMANN)
    return fail(ctx, LBM_ERR_ARG, "Eq. 22 needs a solid denser than the fluid");
  TRY(solids_to_host(ctx, true));
  SolidHost &h = ctx->solids[id];
  h.rho_p = density_ratio > 0 ? density_ratio : 0;
  h.have_Ip = false;
  for (int a = 0; a < 3; a++) {
    h.g[a] = gravity ? gravity[a] : 0;
    h.Up[a] = h.d.velocity[a];
    h.Omp[a] = h.d.omega[a];
  }
  if (ctx->D == 2) h.g[2] = 0;
  ctx->prefetched = false;
  return LBM_OK;
}

lbm_status lbm_get_solid_velocity(lbm_ctx *ctx, int id, double U[3], double Om[3]) {
  if (!ctx || id < 0 || id >= (int)ctx->solids.size()) return LBM_ERR_ARG;
  TRY(solids_to_host(ctx, false));
  for (int a = 0; a < 3; a++) {
    if (U) U[a] = ctx->solids[id].d.velocity[a];
    if (Om) Om[a] = ctx->solids[id].d.omega[a];
  }
  return LBM_OK;
}

lbm_status lbm_get_solid_centre(lbm_ctx *ctx, int id, double c[3]) {
  if (!ctx || id < 0 || id >= (int)ctx->solids.size() || !c) return LBM_ERR_ARG;
  TRY(solids_to_host(ctx, false));
  memcpy(c, ctx->solids[id].c, 3 * sizeof(double));
  return LBM_OK;
}

lbm_status lbm_get_info(lbm_ctx *ctx, lbm_info *info) {
  if (!ctx || !info) return LBM_ERR_ARG;
  TRY(prepare(ctx));
  int cnt[16];
  TRY(read_counts(ctx, cnt));
  std::vector<uint8_t> fl(ctx->N);
  CK(cudaMemcpy(fl.data(), ctx->flags, ctx->N, cudaMemcpyDeviceToHost));
  long long fluid = 0;
  for (long long k = 0; k < ctx->N; k++) fluid += !(fl[k] & FL_SOLID);
  memset(info, 0, sizeof(*info));
  info->nodes = ctx->N;
  info->fluid_nodes = fluid;
  info->list_nodes = cnt[0];
  info->cut_links = cnt[1];
  info->markers = ctx->nmark;
  info->steps = ctx->step;
  info->kernel_launches = ctx->launches;
  info->device_bytes = (int64_t)ctx->dev_bytes;
  info->num_solids = (int)ctx->solids.size();
  info->precision = ctx->d.precision;
  info->bulk_kernel = ctx->bulk_kernel;
  return LBM_OK;
}

lbm_status lbm_device_field(lbm_ctx *ctx, int which, void **dptr, size_t *bytes,
                            size_t *dir_stride) {
  if (!ctx || !dptr) return LBM_ERR_ARG;
  TRY(prepare(ctx));
  if (dir_stride) *dir_stride = which == LBM_FIELD_F_POST ? (size_t)ctx->fs : 0;
  if (which == LBM_FIELD_F_POST) {
    *dptr = ctx->f[ctx->cur];
    if (bytes) *bytes = (size_t)ctx->Q * ctx->fs * ctx->ssz;
  } else if (which == LBM_FIELD_FLAGS) {
    *dptr = ctx->flags;
    if (bytes) *bytes = (size_t)ctx->N;
  } else {
    return LBM_ERR_ARG;
  }
  return LBM_OK;
}

// ---- checkpoint
namespace {
struct SaveHeader {
  char magic[8];
  int version, lattice, nx, ny, nz, precision, nsolids, prev_local, need_collide, scheme;
  long long step, fs;
  lbm_scheme_desc sch;
};
}  // namespace

lbm_status lbm_save(lbm_ctx *ctx, void *host_buf, size_t *size) {
  if (!ctx || !size) return LBM_ERR_ARG;
  if (ctx->scheme.scheme == LBM_ZHAO_YONG)
    return fail(ctx, LBM_ERR_UNSUPPORTED, "checkpoints do not carry the Eq. 16 boundary state");
  if (ctx->outlet)
    return fail(ctx, LBM_ERR_UNSUPPORTED, "checkpoints do not carry the outflow face's state");
  TRY(solids_to_host(ctx, false));
  const size_t fb = (size_t)ctx->Q * ctx->fs * ctx->ssz;
  const size_t total = sizeof(SaveHeader) + sizeof(SolidHost) * ctx->solids.size() + 2 * fb + ctx->N;
  if (!host_buf) {
    *size = total;
    return LBM_OK;
  }
  if (*size < total) return fail(ctx, LBM_ERR_ARG, "checkpoint buffer too small");
  TRY(ensure_geometry(ctx));
  SaveHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, "LBMGB300", 8);
  h.version = 4;  // 2: delta-function kernel; 3: free motion; 4: inside-fluid treatment
  h.lattice = ctx->d.lattice;
  h.nx = ctx->d.nx;
  h.ny = ctx->d.ny;
  h.nz = ctx->d.nz;
  h.precision = ctx->d.precision;
  h.nsolids = (int)ctx->solids.size();
  h.prev_local = ctx->prev_local;
  h.need_collide = ctx->need_collide;
  h.step = ctx->step;
  h.fs = ctx->fs;
  h.sch = ctx->scheme;
  char *p = (char *)host_buf;
  memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  memcpy(p, ctx->solids.data(), sizeof(SolidHost) * ctx->solids.size());
  p += sizeof(SolidHost) * ctx->solids.size();
  CK(cudaMemcpyAsync(p, ctx->f[ctx->cur], fb, cudaMemcpyDeviceToHost, ctx->st));
  p += fb;
  CK(cudaMemcpyAsync(p, ctx->f[1 - ctx->cur], fb, cudaMemcpyDeviceToHost, ctx->st));
  p += fb;
  CK(cudaMemcpyAsync(p, ctx->sid, ctx->N, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  *size = total;
  return LBM_OK;
}

lbm_status lbm_load(lbm_ctx *ctx, const void *host_buf, size_t size) {
  if (ctx) ctx->gen++;
  if (!ctx || !host_buf || size < sizeof(SaveHeader)) return LBM_ERR_ARG;
  if (ctx->outlet)
    return fail(ctx, LBM_ERR_UNSUPPORTED, "checkpoints do not carry the outflow face's state");
  SaveHeader h;
  memcpy(&h, host_buf, sizeof(h));
  if (memcmp(h.magic, "LBMGB300", 8) != 0 || h.version != 4) return fail(ctx, LBM_ERR_ARG, "not a checkpoint of this version");
  if (h.lattice != ctx->d.lattice || h.nx != ctx->d.nx || h.ny != ctx->d.ny || h.nz != ctx->d.nz ||
      h.precision != ctx->d.precision || h.nsolids < 0 || h.nsolids > kMaxSolids ||
      h.fs != ctx->fs)
    return fail(ctx, LBM_ERR_ARG, "checkpoint does not match this lattice");
  const size_t fb = (size_t)ctx->Q * ctx->fs * ctx->ssz;
  const size_t total = sizeof(SaveHeader) + sizeof(SolidHost) * h.nsolids + 2 * fb + ctx->N;
  if (size < total) return fail(ctx, LBM_ERR_ARG, "checkpoint truncated");
  const char *p = (const char *)host_buf + sizeof(h);
  ctx->solids.assign((const SolidHost *)p, (const SolidHost *)p + h.nsolids);
  ctx->host_stale = false;  // the saved state replaces the device copy
  ctx->push_needed = true;
  p += sizeof(SolidHost) * h.nsolids;
  ctx->scheme = h.sch;
  ctx->cur = 0;
  CK(cudaMemcpyAsync(ctx->f[0], p, fb, cudaMemcpyHostToDevice, ctx->st));
  p += fb;
  CK(cudaMemcpyAsync(ctx->f[1], p, fb, cudaMemcpyHostToDevice, ctx->st));
  p += fb;
  CK(cudaMemcpyAsync(ctx->sid, p, ctx->N, cudaMemcpyHostToDevice, ctx->st));
  const size_t padN = ((ctx->N + 15) / 16) * 16;
  CK(cudaMemcpyAsync(ctx->sid + padN, p, ctx->N, cudaMemcpyHostToDevice, ctx->st));
  ctx->prev_local = h.prev_local;
  ctx->need_collide = h.need_collide;
  ctx->step = h.step;
  ctx->geom_dirty = true;
  ctx->restore_geometry = true;
  TRY(rebuild_full(ctx));
  if (!ctx->need_collide && ctx->scheme.scheme == LBM_IBM_DIRECT) {
    // the IBM force of the current time is recomputed from the restored state
    ctx->slot = (ctx->slot + 1) % kHistCap;
    double *acc = force_slot(ctx, ctx->slot);
    CK(cudaMemsetAsync(acc, 0, sizeof(double) * kMaxSolids * 6, ctx->st));
    ibm_prepass(ctx, ctx->f[1], ctx->prev_local, acc, ctx->st);
  }
  CK(cudaStreamSynchronize(ctx->st));
  return LBM_OK;
}

lbm_status lbm_set_timing(lbm_ctx *ctx, int enable, int every) {
  if (!ctx || every < 1) return LBM_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->st));
  resolve_timing(ctx);
  ctx->timing = enable == 1 ? ~0 : (enable & ~1);
  ctx->timing_every = every;
  for (int k = 0; k < TK_COUNT; k++) {
    ctx->tk_ms[k] = 0;
    ctx->tk_launch[k] = ctx->tk_nodes[k] = 0;
  }
  return LBM_OK;
}

lbm_status lbm_get_kernel_time(lbm_ctx *ctx, int kernel, double *ms, int64_t *launches, int64_t *nodes) {
  if (!ctx || kernel < 0 || kernel >= TK_COUNT) return LBM_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->st));
  resolve_timing(ctx);
  if (ms) *ms = ctx->tk_ms[kernel];
  if (launches) *launches = ctx->tk_launch[kernel];
  if (nodes) *nodes = ctx->tk_nodes[kernel];
  return LBM_OK;
}

// ---- velocity query without device allocation (staging array and its
// per-device address: see the definitions before lbm_create)

lbm_status lbm_get_velocity_noalloc(lbm_ctx *ctx, double *host_out, size_t n) {
  if (!ctx || !host_out) return LBM_ERR_ARG;
  const size_t need = (size_t)ctx->D * (size_t)ctx->N;
  if (n < need) return fail(ctx, LBM_ERR_ARG, "output buffer too small: need " + std::to_string(need));
  if (need > kNoAllocScratchDoubles)
    return fail(ctx, LBM_ERR_CAPACITY,
                "lbm_get_velocity_noalloc stages at most " + std::to_string(kNoAllocScratchDoubles) +
                    " doubles (d * nodes); this lattice needs " + std::to_string(need) +
                    ": use lbm_get_velocity");
  // rebuilding the geometry would allocate: the caller must have stepped or
  // queried the context since its last change
  if (ctx->geom_dirty || (ctx->push_needed && dev_motion(ctx) && !ctx->sol_d))
    return fail(ctx, LBM_ERR_STATE,
                "geometry changed since the last step: call lbm_step or lbm_sync first");
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev != ctx->device)
    return fail(ctx, LBM_ERR_STATE, "make the context's device current before this call");
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(ctx, LBM_ERR_UNSUPPORTED, "device index too large");
  double *scratch = nullptr;
  {
    // cached by lbm_create on this device (the context was created there)
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    scratch = g_noalloc_addr[dev];
  }
  if (!scratch) return fail(ctx, LBM_ERR_STATE, "staging array address not set up on this device");
  if (ctx->need_collide) TRY(init_collide(ctx));  // kernels only, no allocation
  // the array keeps the previous call's values: solid nodes must read 0
  CK(cudaMemsetAsync(scratch, 0, need * sizeof(double), ctx->st));
  KArgs a = base_args(ctx);
  a.out_u = scratch;
  run_query(ctx, a);
  CK(cudaMemcpyAsync(host_out, scratch, need * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  CK(cudaGetLastError());
  return LBM_OK;
}

lbm_status lbm_sync(lbm_ctx *ctx) {
  if (!ctx) return LBM_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->st));
  if (ctx->cst) CK(cudaStreamSynchronize(ctx->cst));
  CK(cudaGetLastError());
  int cnt[16];
  TRY(read_counts(ctx, cnt));
  if (cnt[3]) return fail(ctx, LBM_ERR_CAPACITY, "a boundary or refill list overflowed its capacity");
  if (cnt[4])
    return fail(ctx, LBM_ERR_UNSUPPORTED,
                "a moving solid came too close to a non-periodic face (1.5 nodes from a wall or "
                "stress-free face, R + 5 from an outflow face)");
  if (cnt[5])
    return fail(ctx, LBM_ERR_TIMEOUT,
                "a bulk sweep gave up waiting (one second) for its asynchronous row copies");
  return LBM_OK;
}

}  // extern "C"

// ===================================================================== batch
//
// Many lattices advanced together.  Each lattice keeps its own context; the
// batch gives every context a private stream and captures one step pair
// (even + odd, so that the ping-pong buffers return to their places) of all
// active lattices into a single CUDA graph whose per-lattice chains are
// independent branches.  Replaying the graph advances every lattice two
// steps with one launch; small lattices overlap on the GPU instead of
// queueing behind each other.  Residuals are checked every `check_every`
// steps and converged lattices leave the graph.  Solids that move need a
// geometry rebuild with host-side centres every step: such lattices are
// stepped directly, outside the graph.
struct lbm_batch {
  std::vector<lbm_ctx *> ctx;
  std::vector<cudaStream_t> user_st;   // restored on destroy
  std::vector<cudaStream_t> own_st;    // private stream per lattice
  std::vector<cudaEvent_t> ev_done;
  cudaEvent_t ev_origin = nullptr;
  cudaEvent_t ev_user = nullptr;       // orders the batch after the caller's stream
  cudaStream_t origin = nullptr;       // private stream the graph runs on
  cudaStream_t user = nullptr;         // stream given at creation
  std::vector<char> active;
  std::vector<long long> steps_done;
  std::vector<double> residual;
  cudaGraphExec_t exec = nullptr;
  std::vector<int> graph_cur;          // cur of each lattice when captured
  std::vector<unsigned long long> graph_gen;  // gen of each lattice when captured
  std::vector<long long> pair_launches;  // kernels of one captured step pair
  std::vector<int> graph_slot;           // force-record slot of the pair's 2nd step
  std::vector<char> in_graph;
  long long graph_launches = 0;
  std::string err;
};

namespace {

lbm_status bfail(lbm_batch *b, lbm_status s, const std::string &m) {
  if (b) b->err = m;
  return s;
}

#define BCK(expr)                                                          \
  do {                                                                     \
    cudaError_t _e = (expr);                                               \
    if (_e != cudaSuccess)                                                 \
      return bfail(b, LBM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

// Time the bulk sweep of one lattice for a few block widths and keep the
// fastest (writes go to a scratch buffer: the simulation state is untouched).
lbm_status autotune(lbm_ctx *ctx, void *scratch) {
  const int cand_bulk[3] = {64, 128, 256};
  const int cand_list[3] = {64, 128, 256};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  KArgs a = base_args(ctx);
  a.src = ctx->f[ctx->cur];
  a.dst = scratch;
  a.force_acc = force_slot(ctx, (ctx->slot + kHistCap / 2) % kHistCap);
  float best = 1e30f;
  int best_b = ctx->bulk_block;
  for (int c : cand_bulk) {
    a.bulk_block = c;
    sweep(ctx, OP_BULK_SWEEP, a);  // warm
    cudaEventRecord(e0, ctx->st);
    for (int r = 0; r < 3; r++) sweep(ctx, OP_BULK_SWEEP, a);
    cudaEventRecord(e1, ctx->st);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      best_b = c;
    }
  }
  ctx->bulk_block = best_b;
  best = 1e30f;
  int best_l = ctx->list_block;
  if (a.list_cap > 0)
    for (int c : cand_list) {
      a.list_block = c;
      sweep(ctx, OP_LIST_SWEEP, a);
      cudaEventRecord(e0, ctx->st);
      for (int r = 0; r < 3; r++) sweep(ctx, OP_LIST_SWEEP, a);
      cudaEventRecord(e1, ctx->st);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        best_l = c;
      }
    }
  ctx->list_block = best_l;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // forget the scratch force record written while tuning
  cudaMemsetAsync(a.force_acc, 0, sizeof(double) * kMaxSolids * 6, ctx->st);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

void drop_graph(lbm_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
}

// Whether a lattice's steps can be captured in the batch's graph: static
// solids, or solids that move on the device (a free solid present).  Solids
// with a prescribed motion move on the host, which prefetches their next
// geometry: those lattices step directly.
bool graphable(const lbm_ctx *c) { return !any_moving(c) || dev_motion(c); }

// Capture two steps of every active lattice with static geometry or solids
// moving on the device.
lbm_status capture(lbm_batch *b) {
  drop_graph(b);
  const int n = (int)b->ctx.size();
  b->in_graph.assign(n, 0);
  b->graph_cur.assign(n, 0);
  b->graph_gen.assign(n, 0);
  b->pair_launches.assign(n, 0);
  b->graph_slot.assign(n, 0);
  struct Saved {
    int cur, slot;
    bool prev_local;
    int timing;
    long long step, launches, records;
  };
  std::vector<Saved> saved(n);
  // the device copy of moving solids is sent before the capture (a push
  // waits for its stream)
  for (int i = 0; i < n; i++) {
    lbm_ctx *c = b->ctx[i];
    if (b->active[i] && graphable(c) && c->push_needed) {
      const lbm_status s = motion_push(c);
      if (s != LBM_OK) return bfail(b, s, lbm_last_error(c));
    }
  }
  BCK(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
  BCK(cudaEventRecord(b->ev_origin, b->origin));
  lbm_status st = LBM_OK;
  int members = 0;
  for (int i = 0; i < n && st == LBM_OK; i++) {
    lbm_ctx *c = b->ctx[i];
    if (!b->active[i] || !graphable(c)) continue;
    saved[i] = {c->cur, c->slot, c->prev_local, c->timing, c->step, c->launches, c->records};
    c->timing = 0;
    b->graph_cur[i] = c->cur;
    b->graph_gen[i] = c->gen;
    // a free solid under IBM moves by the record of the step before: in
    // every replay after the first, that is the pair's second record, so
    // the first step reads it there (the current record is copied there
    // before the first replay, below)
    if (c->scheme.scheme == LBM_IBM_DIRECT && dev_motion(c))
      c->motion_slot = (c->slot + 2) % kHistCap;
    cudaStreamWaitEvent(c->st, b->ev_origin, 0);
    st = step_once(c);
    if (st == LBM_OK) st = step_once(c);
    cudaEventRecord(b->ev_done[i], c->st);
    cudaStreamWaitEvent(b->origin, b->ev_done[i], 0);
    b->in_graph[i] = 1;
    members++;
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->origin, &g);
  // capture only recorded the work: put the host-side state back
  for (int i = 0; i < n; i++) {
    if (!b->in_graph[i]) continue;
    lbm_ctx *c = b->ctx[i];
    c->motion_slot = -1;
    if (c->scheme.scheme == LBM_IBM_DIRECT && dev_motion(c))
      cudaMemcpyAsync(force_slot(c, (saved[i].slot + 2) % kHistCap), force_slot(c, saved[i].slot),
                      sizeof(double) * kMaxSolids * 6, cudaMemcpyDeviceToDevice, c->st);
    b->pair_launches[i] = c->launches - saved[i].launches;
    b->graph_slot[i] = c->slot;  // after two captured steps
    c->cur = saved[i].cur;
    c->slot = saved[i].slot;
    c->prev_local = saved[i].prev_local;
    c->timing = saved[i].timing;
    c->step = saved[i].step;
    c->records = saved[i].records;
    c->launches = saved[i].launches;
  }
  if (st != LBM_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  if (members == 0) {
    cudaGraphDestroy(g);
    return LBM_OK;
  }
  // the kernel nodes keep the priorities of the streams they were captured
  // from (the auxiliary stream's boundary and IBM chains run ahead of the
  // bulk sweeps, as when stepped directly); without this flag every node
  // would run at the priority of the stream the graph is launched into
  e = cudaGraphInstantiate(&b->exec, g, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return LBM_OK;
}

// Host bookkeeping of one replayed step pair.  The replay writes the two
// force-record slots that followed the capture-time slot, so the context's
// current slot is the second of them after every replay.
void after_replay(lbm_batch *b) {
  for (size_t i = 0; i < b->ctx.size(); i++) {
    if (!b->in_graph[i]) continue;
    lbm_ctx *c = b->ctx[i];
    c->slot = b->graph_slot[i];
    c->step += 2;
    if (dev_motion(c)) c->host_stale = true;  // the replay moved the solids
    c->prev_local = false;
    c->records = std::min<long long>(c->records + 2, kHistCap);
    c->launches += b->pair_launches[i];
    b->steps_done[i] += 2;
  }
}

bool graph_valid(const lbm_batch *b) {
  if (!b->exec) return false;
  for (size_t i = 0; i < b->ctx.size(); i++) {
    const bool want = b->active[i] && graphable(b->ctx[i]);
    if (want != (bool)b->in_graph[i]) return false;
    if (want && b->ctx[i]->cur != b->graph_cur[i]) return false;
    if (want && b->ctx[i]->gen != b->graph_gen[i]) return false;
  }
  return true;
}

// The batch's private streams start after the work already queued on the
// caller's stream, and the caller's stream waits for all of them at the end.
lbm_status enter(lbm_batch *b) {
  BCK(cudaEventRecord(b->ev_user, b->user));
  for (lbm_ctx *c : b->ctx) BCK(cudaStreamWaitEvent(c->st, b->ev_user, 0));
  return LBM_OK;
}
lbm_status leave(lbm_batch *b) {
  for (size_t i = 0; i < b->ctx.size(); i++) {
    BCK(cudaEventRecord(b->ev_done[i], b->ctx[i]->st));
    BCK(cudaStreamWaitEvent(b->user, b->ev_done[i], 0));
  }
  return LBM_OK;
}

lbm_status batch_advance(lbm_batch *b, int nsteps) {
  const int n = (int)b->ctx.size();
  // a member changed since the last call (geometry, initial state) is brought
  // up to date before any captured step runs; its bumped generation then
  // makes the graph stale
  for (int i = 0; i < n; i++)
    if (b->active[i]) {
      lbm_status s = prepare(b->ctx[i]);
      if (s != LBM_OK) return bfail(b, s, lbm_last_error(b->ctx[i]));
    }
  int done = 0;
  while (done < nsteps) {
    const bool pair = nsteps - done >= 2;
    bool any_static = false;
    for (int i = 0; i < n; i++) any_static |= b->active[i] && graphable(b->ctx[i]);
    if (pair && any_static) {
      if (!graph_valid(b)) {
        // the per-slot bookkeeping in after_replay assumes the capture-time
        // slots; capture again whenever membership or buffer parity changed
        lbm_status s = capture(b);
        if (s != LBM_OK) return s;
      }
      if (b->exec) {
        // the replay follows each lattice's earlier work on its own stream,
        // and later work on those streams (queries, residuals) follows it
        for (int i = 0; i < n; i++) {
          if (!b->in_graph[i]) continue;
          BCK(cudaEventRecord(b->ev_done[i], b->ctx[i]->st));
          BCK(cudaStreamWaitEvent(b->origin, b->ev_done[i], 0));
        }
        BCK(cudaGraphLaunch(b->exec, b->origin));
        BCK(cudaEventRecord(b->ev_origin, b->origin));
        for (int i = 0; i < n; i++)
          if (b->in_graph[i]) BCK(cudaStreamWaitEvent(b->ctx[i]->st, b->ev_origin, 0));
        b->graph_launches++;
        after_replay(b);
      }
      // lattices outside the graph (solids with a prescribed motion) step directly
      for (int i = 0; i < n; i++) {
        if (!b->active[i] || b->in_graph[i]) continue;
        for (int k = 0; k < 2; k++) {
          lbm_status s = step_once(b->ctx[i]);
          if (s != LBM_OK) return bfail(b, s, lbm_last_error(b->ctx[i]));
        }
        b->steps_done[i] += 2;
      }
      done += 2;
    } else {
      for (int i = 0; i < n; i++) {
        if (!b->active[i]) continue;
        lbm_status s = step_once(b->ctx[i]);
        if (s != LBM_OK) return bfail(b, s, lbm_last_error(b->ctx[i]));
        b->steps_done[i] += 1;
      }
      done += 1;
    }
  }
  return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(lbm_batch **out, lbm_ctx *const *ctxs, int n, void *cuda_stream,
                            int autotune_blocks) {
  if (!out || !ctxs || n <= 0) return LBM_ERR_ARG;
  *out = nullptr;
  lbm_batch *b = new lbm_batch();
  b->user = (cudaStream_t)cuda_stream;
  int dev0 = ctxs[0] ? ctxs[0]->device : -1;
  size_t scratch_bytes = 0;
  for (int i = 0; i < n; i++) {
    lbm_ctx *c = ctxs[i];
    if (!c || c->device != dev0) {
      delete b;
      return LBM_ERR_ARG;
    }
    for (int j = 0; j < i; j++)
      if (ctxs[j] == c) {
        delete b;
        return LBM_ERR_ARG;
      }
    lbm_status s = prepare(c);
    if (s != LBM_OK) {
      delete b;
      return s;
    }
    scratch_bytes = std::max<size_t>(scratch_bytes, (size_t)c->Q * c->fs * c->ssz);
  }
  b->ctx.assign(ctxs, ctxs + n);
  b->active.assign(n, 1);
  b->steps_done.assign(n, 0);
  b->residual.assign(n, NAN);
  b->in_graph.assign(n, 0);
  b->graph_cur.assign(n, 0);
  cudaError_t e = cudaEventCreateWithFlags(&b->ev_origin, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_user, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
  for (int i = 0; i < n && e == cudaSuccess; i++) {
    lbm_ctx *c = b->ctx[i];
    cudaStreamSynchronize(c->st);
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    b->user_st.push_back(c->st);
    b->own_st.push_back(s);
    b->ev_done.push_back(ev);
    c->st = s;
  }
  if (e == cudaSuccess && autotune_blocks) {
    void *scratch = nullptr;
    e = cudaMalloc(&scratch, scratch_bytes);
    if (e == cudaSuccess) {
      for (int i = 0; i < n; i++) {
        // lattices of the same shape share the result
        int same = -1;
        for (int j = 0; j < i; j++)
          if (b->ctx[j]->d.nx == b->ctx[i]->d.nx && b->ctx[j]->d.ny == b->ctx[i]->d.ny &&
              b->ctx[j]->d.nz == b->ctx[i]->d.nz && b->ctx[j]->d.precision == b->ctx[i]->d.precision)
            same = j;
        if (same >= 0) {
          b->ctx[i]->bulk_block = b->ctx[same]->bulk_block;
          b->ctx[i]->list_block = b->ctx[same]->list_block;
        } else if (autotune(b->ctx[i], scratch) != LBM_OK) {
          e = cudaErrorUnknown;
          break;
        }
      }
      for (int i = 0; i < n; i++) cudaStreamSynchronize(b->ctx[i]->st);
      cudaFree(scratch);
    }
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    lbm_batch_destroy(b);
    return LBM_ERR_CUDA;
  }
  *out = b;
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch *b) {
  if (!b) return;
  drop_graph(b);
  for (size_t i = 0; i < b->ctx.size(); i++) {
    if (i < b->own_st.size() && b->own_st[i]) {
      cudaStreamSynchronize(b->own_st[i]);
      b->ctx[i]->st = b->user_st[i];
      cudaStreamDestroy(b->own_st[i]);
    }
    if (i < b->ev_done.size() && b->ev_done[i]) cudaEventDestroy(b->ev_done[i]);
  }
  if (b->ev_origin) cudaEventDestroy(b->ev_origin);
  if (b->ev_user) cudaEventDestroy(b->ev_user);
  if (b->origin) {
    cudaStreamSynchronize(b->origin);
    cudaStreamDestroy(b->origin);
  }
  delete b;
}

lbm_status lbm_batch_step(lbm_batch *b, int nsteps) {
  if (!b || nsteps < 0) return LBM_ERR_ARG;
  lbm_status s = enter(b);
  if (s == LBM_OK) s = batch_advance(b, nsteps);
  const lbm_status s2 = leave(b);
  if (s != LBM_OK) return s;
  if (s2 != LBM_OK) return s2;
  BCK(cudaGetLastError());
  return LBM_OK;
}

namespace {

// The stepping loop of lbm_batch_run_to_steady, between enter and leave.
// A lattice whose residual is not finite leaves the loop (LBM_ERR_DIVERGED
// at the end); the others run on to their own residual or max_steps.
lbm_status run_batch_to_steady(lbm_batch *b, double tol, int check_every, int max_steps) {
  const int n = (int)b->ctx.size();
  for (int i = 0; i < n; i++) {
    lbm_ctx *ctx = b->ctx[i];
    TRY(velocity_to(ctx, ctx->u_snap));
  }
  int left = n;
  lbm_status result = LBM_OK;
  while (left > 0) {
    int k = check_every;
    long long most = 0;
    for (int i = 0; i < n; i++)
      if (b->active[i]) most = std::max(most, b->steps_done[i]);
    if (most + k > max_steps) k = (int)(max_steps - most);
    if (k <= 0) break;
    TRY(batch_advance(b, k));
    for (int i = 0; i < n; i++) {
      if (!b->active[i]) continue;
      lbm_ctx *c = b->ctx[i];
      TRY(velocity_to(c, c->u_now));
      launch_residual(c->u_now, c->u_snap, 0, c->flags, c->N, c->D, c->red2, c->st);
      c->launches++;
    }
    for (int i = 0; i < n; i++) {
      if (!b->active[i]) continue;
      lbm_ctx *c = b->ctx[i];
      double h[2];
      BCK(cudaMemcpyAsync(h, c->red2, sizeof(h), cudaMemcpyDeviceToHost, c->st));
      BCK(cudaStreamSynchronize(c->st));
      const double r = residual_of(h);
      b->residual[i] = r;
      c->last_residual = r;
      if (!std::isfinite(r)) {
        b->active[i] = 0;
        left--;
        result = bfail(b, LBM_ERR_DIVERGED, "lattice " + std::to_string(i) + " diverged");
      } else if (r < tol) {
        b->active[i] = 0;
        left--;
      } else {
        std::swap(c->u_now, c->u_snap);
      }
    }
  }
  return result;
}

}  // namespace

lbm_status lbm_batch_run_to_steady(lbm_batch *b, double tol, int check_every, int max_steps,
                                   int64_t *steps_done, double *residual) {
  if (!b || check_every < 1 || max_steps < 0) return LBM_ERR_ARG;
  const int n = (int)b->ctx.size();
  for (int i = 0; i < n; i++) {
    lbm_ctx *c = b->ctx[i];
    {
      lbm_ctx *ctx = c;
      if (!c->u_now) TRY(dalloc(ctx, (void **)&c->u_now, sizeof(double) * c->D * c->N));
      if (!c->u_snap) TRY(dalloc(ctx, (void **)&c->u_snap, sizeof(double) * c->D * c->N));
    }
    b->active[i] = 1;
    b->steps_done[i] = 0;
    b->residual[i] = INFINITY;
  }
  {
    const lbm_status s = enter(b);
    if (s != LBM_OK) return s;
  }
  // every exit from here on passes through leave(): work queued on the
  // caller's stream afterwards stays ordered after the batch's work
  const lbm_status result = run_batch_to_steady(b, tol, check_every, max_steps);
  for (int i = 0; i < n; i++) {
    if (steps_done) steps_done[i] = b->steps_done[i];
    if (residual) residual[i] = b->residual[i];
  }
  const lbm_status s2 = leave(b);
  return result != LBM_OK ? result : s2;
}

lbm_status lbm_batch_info(lbm_batch *b, int i, int *bulk_block, int *list_block, int64_t *graph_launches) {
  if (!b || i < 0 || i >= (int)b->ctx.size()) return LBM_ERR_ARG;
  if (bulk_block) *bulk_block = b->ctx[i]->bulk_block;
  if (list_block) *list_block = b->ctx[i]->list_block;
  if (graph_launches) *graph_launches = b->graph_launches;
  return LBM_OK;
}

const char *lbm_batch_last_error(const lbm_batch *b) { return b ? b->err.c_str() : "null batch"; }

}  // extern "C"
