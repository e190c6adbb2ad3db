// lbm_internal.h -- structures shared by the host API and the kernel
// translation units of the library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lbm.h"

namespace lbm {

constexpr int kMaxSolids = 8;

// Solid state passed to kernels by value (FP64 geometry).
struct SolidDev {
  int kind, fluid_inside;
  double c[3], R, U[3], Om[3];
  double RL;            // marker radius (IBM)
};

struct SolidsDev {
  int n;
  SolidDev s[kMaxSolids];
};

// Cut-link records (SoA, type T = compute type): coefficients c0..c4 of the
// bounce-back rule, the moving-wall term mw = c5 * 6 w_i (e_i.u_w), the wall
// velocity, the lever arm x_w - Y_c, and the solid id.
struct LinkArrays {
  void *c[5];
  void *mw;
  void *uw[3];
  void *arm[3];
  uint8_t *sid;
};

// FP16 storage keeps (f - w_i) * 2^kFp16ScaleLog2.
constexpr int kFp16ScaleLog2 = 10;

// Arguments of every sweep-like kernel (passed by value).
struct KArgs {
  // lattice
  int nx, ny, nz;
  long long N;
  long long fs;     // stride between direction arrays (elements, >= N)
  const void *src;  // distributions read
  void *dst;        // distributions written
  const uint8_t *flags;
  // collision constants in FP64 (FP64 kernels, queries) and the same
  // constants rounded once to FP32 on the host (FP32 kernels never touch
  // FP64 values per node: GB300's FP64 rate is a small fraction of FP32)
  double omega, ds[19], s_bulk, nu;
  double g[3];
  double inv_scale;  // storage scale^-1 (1 except FP16 storage)
  float omega_f, ds_f[19], g_f[3], inv_scale_f;
  // boundary-node list
  const int *list_node;
  const uint32_t *list_mask;
  const int *list_link;
  const int *counts;  // device counters: [0] list nodes, [1] links, [2] refill
  int list_cap;
  const double *list_cst;  // [6][list_cap] state-independent part of Eq. 17
  LinkArrays links;
  // IBM dense fields (type T, [3][N]) and flags
  const void *f_ibm;
  void *u_band;
  // momentum exchange accumulators: [solid][6] doubles (F, T)
  double *force_acc;
  int nsolids;
  // refill
  const int *refill_node;
  const uint8_t *refill_sid;
  int refill_cap;
  SolidsDev solids;
  // device copy of the solids, read instead of `solids` when it is set (free
  // solids: their motion is integrated on the device)
  const SolidsDev *solids_d;
  const uint8_t *sid;
  // query outputs (FP64); unused pointers are null
  double *out_rho, *out_u, *out_S, *out_stress, *out_f;
  double *out_eps;   // dissipation rate 2 nu s_ij s_ij
  int local_gather;  // 1: read src locally (pre-collision state), 0: pull
  int bulk_block;    // threads per block of the bulk sweep (multiple of 32)
  int cache_hints;   // bulk sweep: bit 0 evict-first loads, bit 1 evict-first stores
  int list_block;    // threads per block of the boundary-node sweep (32, 64 or 128)
  int list_thread;   // boundary-node sweep: 1 = a thread per node (IBM band), 0 = a warp per node
  void *zy_pre;      // Eq. 16: T [Q][fs] pre-collision populations at the boundary nodes, or null
  int bulk_mode;       // bulk sweep: 0 one node per thread, 1 vectors of nodes per thread,
                       // 2 vectors fed by bulk copies of row segments (each where nx and
                       // the direction stride allow, else the next simpler one)
  int bulk_vec_words;  // vector sweep: 32-bit words per thread and direction (2 or 4; 0 = 2)
  int bulk_vec_packed; // vector sweep: 1 packed FP32x2 collision of node pairs, 0 node by
                       // node, -1 by storage type
  int *wait_err;       // set to 1 by a kernel whose wait for its asynchronous copies gave up
  // domain faces x-, x+, y-, y+, z-, z+ (LBM_FACE_*), their wall velocities,
  // the nodes next to a non-periodic face, and the outflow face's kept
  // populations and outward velocity (LT [Q + 1][out_area]; out_face -1: none)
  int face[6];
  double u_face[6][3];
  float u_face_f[6][3];
  const int *face_node;
  int nface;
  void *outlet;
  int out_face;
  long long out_area;
  // Eq. 24 for one solid over the box (x0, y0, z0, bx, by, bz) around it:
  // sums of alpha u and alpha r x u added into kempe_out[0..5] (FP64)
  double *kempe_out;
  int kempe_solid;
  int kbox[6];
  int kbox_dev;  // the box origin is floor(c - R - 1) of the device copy's centre
};

#ifdef __CUDACC__
// Solid s of a kernel's arguments: the device copy when there is one.
template <typename A>
__device__ __forceinline__ SolidDev solid_of(const A &a, int s) {
  if (a.solids_d) return a.solids_d->s[s];
  return a.solids.s[s];
}
#endif

// kernel families timed by lbm_set_timing
enum TimedKernel { TK_BULK = 0, TK_LIST = 1, TK_IBM = 2, TK_GEOM = 3, TK_COUNT = 4 };

// Operations of the precision-specific translation units.
enum SweepOp {
  OP_BULK_SWEEP,   // pull + collide + store, plain fluid nodes
  OP_LIST_SWEEP,   // pull + bounce-back + collide + store + Eq. 17
  OP_ZY_SEED,      // Eq. 16: boundary nodes' pre-collision populations from a local state
  OP_BULK_QUERY,   // pull, fields to FP64 outputs
  OP_LIST_QUERY,
  OP_LOCAL_INIT,   // local read of a pre-collision state + collide + store
  OP_LOCAL_QUERY,  // local read of a pre-collision state, fields
  OP_REFILL,       // equilibrium refill of uncovered nodes (+ collide)
  OP_BAND_VEL,     // IBM: unforced velocity at band nodes, zero the IBM force
  OP_FROM_DOUBLE,  // convert a full-f FP64 array (out_f) into deviations (dst)
  OP_FILL_EQ,      // fill dst with equilibrium deviations (g[] = u, omega = rho)
  OP_FACE_SWEEP,   // nodes next to a non-periodic domain face: pull with the face rules + collide
  OP_FACE_QUERY,   // the same nodes, fields
  OP_FACE_SEED,    // outflow face: keep the populations of a state held locally
  OP_KEMPE         // Eq. 24: the fluid momentum inside a solid, from f*(t) and the forces
};

// The bulk sweeps of up to kMaxGroup lattices in one grid (the blocks of
// lattice k start at block_start[k]): short sweeps of several lattices then
// share one launch's ramp-up and tail instead of paying them one after the
// other.
constexpr int kMaxGroup = 8;
struct GroupArgs {
  int n;
  int block_start[kMaxGroup + 1];
  KArgs a[kMaxGroup];
};
// Launches the group when every lattice takes the same vector bulk kernel
// (lattice, collision, storage, vector shape and block size); false, with
// nothing launched, otherwise.
bool launch_bulk_group(const KArgs *as, int n, int lattice, int collision, int precision,
                       cudaStream_t st);

// Launch one operation for the given lattice/collision/precision.  grid
// sizes are chosen by the launcher; counts on the device bound list work.
void launch_sweep(SweepOp op, int lattice, int collision, int precision,
                  const KArgs &a, cudaStream_t st);

// The bulk sweep kernel the calling thread's last OP_BULK_SWEEP launch chose
// (host side): 0 one node per thread, 1 vectors of nodes, 2 vectors fed by
// row-segment copies.
enum BulkKernel { BK_NODE = 0, BK_VEC = 1, BK_ROWS = 2 };
extern thread_local int g_bulk_kernel;

// geometry (geometry.cu)
struct GeomBox {
  int x0, y0, z0, bx, by, bz;
};
struct GeomArgs {
  int nx, ny, nz, lattice, scheme, force_all;
  long long N;
  SolidsDev solids;
  uint8_t *flags;
  uint8_t *sid;
  int *counts;  // [0] list nodes, [1] links, [2] refill nodes, [3] overflow
  int *list_node;
  uint32_t *list_mask;
  int *list_link;
  double *list_cst;
  int *link_list;     // [link_cap] list entry owning each link
  uint8_t *link_dir;  // [link_cap] direction of each link
  int list_cap, link_cap;
  LinkArrays links;
  int *refill_node;
  uint8_t *refill_sid;
  int refill_cap;
  int track_new;  // mark nodes uncovered since the previous geometry
  int face[6];    // domain face types (FL_FACE on the nodes next to a non-periodic face)
  double band_w;  // IBM band half width
  GeomBox box[kMaxSolids];
  int nbox;
  long long box_offset[kMaxSolids + 1];
  // device copy of the solids (see KArgs) and, when box_dev is set, box k is
  // anchored on solid k's centre there: origin floor(c - box_ext[k]) on the
  // axes where its width is below the lattice's
  const SolidsDev *solids_d;
  int box_dev;
  double box_ext[kMaxSolids];
};
void launch_geometry(const GeomArgs &g, int precision, cudaStream_t st);

// IBM (ibm.cu)
struct IbmArgs {
  int nx, ny, nz, dim, nmark;
  long long N;
  const double *dir;  // [3][nmark]
  const double *dV;   // [nmark]
  const uint8_t *msid;
  double *Fm;         // [3][nmark] accumulated marker force density
  SolidsDev solids;
  void *u_band;       // T [3][N]
  void *f_ibm;        // T [3][N]
  int use_f;          // interpolate u_band + f_ibm (iterations > 1)
  int first;          // first iteration: Fm = 0 before adding
  double *force_acc;  // [solid][6]
  int reduce_force;   // accumulate -sum F dV and the torque
  int4 *mk_base;      // [nmark] first stencil node (unwrapped x, y, z) and solid
  void *mk_wts;       // T [nmark][4^dim] delta weights of the stencil points
  int kernel;         // delta-function kernel (LBM_DELTA_*)
  const SolidsDev *solids_d;  // device copy of the solids (see KArgs)
  double *dF;         // [3][nmark] the iteration's force increment, or null: the
                      // interpolation stores it and the spreading adds it to the
                      // force already spread (otherwise the total force is spread)
};
// The whole forcing loop of Sec. 2.1 (n_it iterations of interpolation,
// direct force and spreading) for each solid in one thread-block cluster,
// with the band fields of a box around the solid held in the cluster's
// distributed shared memory (see ibm.cu).
constexpr int kIbmClusterSize = 8;
struct IbmBox {
  int o[3];    // origin (unwrapped); recomputed from the device centre when box_dev
  int w[3];    // widths (the lattice's on a full axis)
  int h;       // planes per block along the slab axis (z in 3D, y in 2D)
  int mpc;     // markers per block
  double ext;  // floor(c - ext) is the origin when box_dev
};
struct IbmClusterArgs {
  int ns;                       // solids, one cluster each
  int mk_start[kMaxSolids + 1]; // markers of solid s: mk_start[s] .. mk_start[s+1] - 1
  IbmBox box[kMaxSolids];
  int iters;
  int box_dev;
  int dim;                      // 2 or 3: the slabs run along y or z
};
// Shared memory bytes per block of the cluster kernel for these boxes.
size_t ibm_cluster_smem(const IbmClusterArgs &cl, int precision);
// Whether clusters of these boxes can be placed on the device (sets the
// kernel's shared-memory limit; not to be called during a stream capture).
bool ibm_cluster_fits(const IbmClusterArgs &cl, int precision);
void launch_ibm_cluster(const IbmArgs &a, const IbmClusterArgs &cl, int precision,
                        cudaStream_t st);
// stencil bases and weights of every marker (after each geometry change)
void launch_ibm_prepare(const IbmArgs &a, int precision, cudaStream_t st);
// interpolation, direct force and spreading in one pass (single iteration)
void launch_ibm_fused(const IbmArgs &a, int precision, cudaStream_t st);
void launch_ibm_interp(const IbmArgs &a, int precision, cudaStream_t st);
void launch_ibm_spread(const IbmArgs &a, int precision, cudaStream_t st);

// chunked upload of FP64 populations (transfer.cu)
struct UploadArgs {
  const double *src;     // staged full populations f_i of nodes n0 .. n0 + len - 1
  void *dst;             // storage array of direction i (element 0 = node 0)
  const uint8_t *flags;  // node flags (solid nodes store 0)
  long long n0, len;
  double w;              // lattice weight w_i
  double inv_scale;      // storage scale^-1 (1 except FP16 storage)
};
void launch_upload_chunk(const UploadArgs &a, int precision, cudaStream_t st);

// solid motion on the device (motion.cu).  Per solid: the density ratio
// rho_p / rho_f (0: prescribed motion), gravity, the velocities of the
// previous step (Eq. 23) and the inside fluid's momentum and angular
// momentum of the previous step (Eq. 24).
struct FreeDev {
  double rho_p, g[3], Up[3], Omp[3], Ip[6];
  int have_Ip;
};
enum MotionMode { MM_BOUNCE_BACK = 0, MM_IBM_FENG = 1, MM_IBM_KEMPE = 2, MM_IBM_UHLMANN = 3 };
struct MotionArgs {
  SolidsDev *now;       // the solids' current state, advanced in place
  FreeDev *fr;          // [kMaxSolids]
  const double *rec;    // force record of the step: [kMaxSolids][F, T]
  const double *kempe;  // [kMaxSolids][6] inside-fluid integrals (MM_IBM_KEMPE)
  int n, mode, dim, nz;
  int face[6];          // domain face types (clearance of free solids)
  int len[3];
  int *err;             // set to 1 when a free solid comes too close to a non-periodic face
};
// One step of motion: free solids by Newton-Euler (Eq. 20 / 23 / 22 / 24),
// the others by their prescribed velocity.
void launch_motion(const MotionArgs &m, cudaStream_t st);

// reductions (reduce.cu)
void launch_residual(const double *u, const double *usnap, long long n,
                     const uint8_t *flags, long long N, int d, double *out2,
                     cudaStream_t st);

}  // namespace lbm
