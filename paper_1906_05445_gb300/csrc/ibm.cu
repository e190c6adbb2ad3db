// ibm.cu -- direct-forcing immersed boundary (Sec. 2.1 of Peng, Ayala &
// Wang): interpolation of the unforced velocity to the Lagrangian markers
// with a regularised delta function (Eqs. 5-6; Peskin's 4-point kernel by
// default, or the 3-point, linear or cosine kernels of Sec. 3.1), the direct force
// F = rho0 (U^d - U~)/dt (Eq. 7), and its spreading back to the lattice as a
// body force (Eq. 8) with atomic accumulation.  One warp per marker: its 4^d
// stencil points are split over the lanes and the interpolated velocity is
// reduced with warp shuffles; the solid's force and torque are reduced per
// block in FP64.
#include <cooperative_groups.h>

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace cg = cooperative_groups;

namespace lbm {

namespace {

// The one-dimensional delta-function kernels compared in Sec. 3.1:
// Peskin's 4-point kernel (Eq. 6, the default), Roma, Peskin & Berger's
// 3-point kernel, the 2-point linear kernel, and the 4-point cosine kernel of
// Appendix B.  Each support lies inside the 4-point window from floor(X) - 1,
// so every kernel uses the same 4^d stencil (points outside the support get
// weight 0).
template <typename T>
__device__ __forceinline__ T phi_k(int kernel, T r) {
  const T a = fabs(r);
  switch (kernel) {
  case LBM_DELTA_ROMA3:
    if (a >= (T)1.5) return (T)0;
    if (a <= (T)0.5) return ((T)1 + sqrt((T)1 - (T)3 * a * a)) / (T)3;
    return ((T)5 - (T)3 * a - sqrt((T)1 - (T)3 * ((T)1 - a) * ((T)1 - a))) / (T)6;
  case LBM_DELTA_LINEAR2:
    return a >= (T)1 ? (T)0 : (T)1 - a;
  case LBM_DELTA_COSINE4:
    return a >= (T)2 ? (T)0 : ((T)1 + cospi(r / (T)2)) / (T)4;
  default:
    if (a >= (T)2) return (T)0;
    if (a >= (T)1) return ((T)5 - (T)2 * a - sqrt((T)-7 + (T)12 * a - (T)4 * a * a)) / (T)8;
    return ((T)3 - (T)2 * a + sqrt((T)1 + (T)4 * a - (T)4 * a * a)) / (T)8;
  }
}

struct Marker {
  double X[3];   // position
  double r[3];   // X - centre (z dropped for cylinders and 2D)
  int s;
};

__device__ __forceinline__ Marker marker(const IbmArgs &a, int m) {
  Marker k;
  k.s = a.msid[m];
  const SolidDev b = solid_of(a, k.s);
  const double dx = a.dir[m], dy = a.dir[a.nmark + m], dz = a.dir[2 * a.nmark + m];
  k.X[0] = b.c[0] + b.RL * dx;
  k.X[1] = b.c[1] + b.RL * dy;
  if (a.dim == 2)
    k.X[2] = 0.0;
  else if (b.kind == LBM_CYLINDER_Z)
    k.X[2] = dz;  // plane of the ring
  else
    k.X[2] = b.c[2] + b.RL * dz;
  k.r[0] = k.X[0] - b.c[0];
  k.r[1] = k.X[1] - b.c[1];
  k.r[2] = (a.dim == 2 || b.kind == LBM_CYLINDER_Z) ? 0.0 : k.X[2] - b.c[2];
  return k;
}

// Stencil of a marker: the 4^d nodes from floor(X) - 1; the marker position
// is FP64, the offsets of the stencil points from it are formed once and the
// per-point arithmetic runs in the compute type.
template <typename T> struct Stencil {
  int ix, iy, iz;  // first stencil node (unwrapped)
  T dx, dy, dz;    // first node - X
};

template <typename T>
__device__ __forceinline__ Stencil<T> stencil_of(const IbmArgs &a, const Marker &k) {
  Stencil<T> st;
  const double bx = floor(k.X[0]) - 1.0, by = floor(k.X[1]) - 1.0;
  const double bz = a.dim == 3 ? floor(k.X[2]) - 1.0 : 0.0;
  st.ix = (int)bx;
  st.iy = (int)by;
  st.iz = (int)bz;
  st.dx = (T)(bx - k.X[0]);
  st.dy = (T)(by - k.X[1]);
  st.dz = a.dim == 3 ? (T)(bz - k.X[2]) : (T)0;
  return st;
}

template <typename T>
__device__ __forceinline__ long long stencil_point(const IbmArgs &a, const Stencil<T> &st,
                                                   int p, T &wgt) {
  const int kx = p & 3, ky = (p >> 2) & 3, kz = p >> 4;
  wgt = phi_k<T>(a.kernel, st.dx + (T)kx) * phi_k<T>(a.kernel, st.dy + (T)ky);
  if (a.dim == 3) wgt *= phi_k<T>(a.kernel, st.dz + (T)kz);
  const int x = wrap(st.ix + kx, a.nx), y = wrap(st.iy + ky, a.ny);
  const int z = a.dim == 3 ? wrap(st.iz + kz, a.nz) : 0;
  return x + (long long)a.nx * (y + (long long)a.ny * z);
}

// Stencil base and the 4^dim weights of every marker, from its FP64
// position (one warp per marker, a lane per stencil point).
template <typename T>
__global__ void __launch_bounds__(128) k_prepare(const IbmArgs a) {
  const int m = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (m >= a.nmark) return;
  const Marker k = marker(a, m);
  const Stencil<T> stc = stencil_of<T>(a, k);
  const int npts = a.dim == 3 ? 64 : 16;
  T *wts = (T *)a.mk_wts + (long long)m * npts;
  for (int p = lane; p < npts; p += 32) {
    const int kx = p & 3, ky = (p >> 2) & 3, kz = p >> 4;
    T wgt = phi_k<T>(a.kernel, stc.dx + (T)kx) * phi_k<T>(a.kernel, stc.dy + (T)ky);
    if (a.dim == 3) wgt *= phi_k<T>(a.kernel, stc.dz + (T)kz);
    wts[p] = wgt;
  }
  if (lane == 0) a.mk_base[m] = make_int4(stc.ix, stc.iy, stc.iz, k.s);
}

__device__ __forceinline__ long long table_node(const IbmArgs &a, int4 b, int p) {
  const int kx = p & 3, ky = (p >> 2) & 3, kz = p >> 4;
  const int x = wrap(b.x + kx, a.nx), y = wrap(b.y + ky, a.ny);
  const int z = a.dim == 3 ? wrap(b.z + kz, a.nz) : 0;
  return x + (long long)a.nx * (y + (long long)a.ny * z);
}

// interpolated velocity of marker m (all lanes get the sum)
template <typename T>
__device__ __forceinline__ void interp_marker(const IbmArgs &a, int m, int lane, int4 b, T U[3]) {
  const int npts = a.dim == 3 ? 64 : 16;
  const T *ub = (const T *)a.u_band, *fi = (const T *)a.f_ibm;
  const T *wts = (const T *)a.mk_wts + (long long)m * npts;
  U[0] = U[1] = U[2] = 0;
  for (int p = lane; p < npts; p += 32) {
    const T wgt = wts[p];
    const long long n = table_node(a, b, p);
    for (int c = 0; c < a.dim; c++) {
      T v = ub[c * a.N + n];
      if (a.use_f) v += fi[c * a.N + n];  // u~ + f dt / rho0, rho0 = 1
      U[c] += wgt * v;
    }
  }
  for (int c = 0; c < 3; c++)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) U[c] += __shfl_xor_sync(0xffffffffu, U[c], o);
}

// desired velocity U + Omega x (X - c) of marker m minus the interpolated one
__device__ __forceinline__ void direct_force(const IbmArgs &a, const Marker &k, const double U[3],
                                             double F[3]) {
  const SolidDev b = solid_of(a, k.s);
  const double Ud[3] = {b.U[0] + b.Om[1] * k.r[2] - b.Om[2] * k.r[1],
                        b.U[1] + b.Om[2] * k.r[0] - b.Om[0] * k.r[2],
                        b.U[2] + b.Om[0] * k.r[1] - b.Om[1] * k.r[0]};
  for (int c = 0; c < 3; c++) F[c] = c < a.dim ? Ud[c] - U[c] : 0.0;  // rho0 (U^d - U~)/dt
}

template <typename T>
__device__ __forceinline__ void spread_marker(const IbmArgs &a, int m, int lane, int4 b,
                                              const double F[3]) {
  const int npts = a.dim == 3 ? 64 : 16;
  const double dV = a.dV[m];
  const T FdV[3] = {(T)(F[0] * dV), (T)(F[1] * dV), (T)(F[2] * dV)};
  const T *wts = (const T *)a.mk_wts + (long long)m * npts;
  T *fi = (T *)a.f_ibm;
  for (int p = lane; p < npts; p += 32) {
    const T wgt = wts[p];
    const long long n = table_node(a, b, p);
    for (int c = 0; c < a.dim; c++) atomicAdd(fi + c * a.N + n, FdV[c] * wgt);
  }
}

// force on the solid, minus the marker forces (Sec. 3.1, Eq. 45), reduced
// per block in FP64
__device__ __forceinline__ void reduce_solid_force(const IbmArgs &a, bool active, int lane,
                                                   int warp, const Marker &k, const double F[3],
                                                   double dV) {
  __shared__ double part[4][6];
  __shared__ int psid[4];
  if (lane == 0) {
    psid[warp] = -1;
    if (active) {
      const double Fs[3] = {-F[0] * dV, -F[1] * dV, -F[2] * dV};
      part[warp][0] = Fs[0];
      part[warp][1] = Fs[1];
      part[warp][2] = Fs[2];
      part[warp][3] = k.r[1] * Fs[2] - k.r[2] * Fs[1];
      part[warp][4] = k.r[2] * Fs[0] - k.r[0] * Fs[2];
      part[warp][5] = k.r[0] * Fs[1] - k.r[1] * Fs[0];
      psid[warp] = k.s;
    }
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int c = threadIdx.x;
    double acc = 0;
    const int s0 = psid[0];
    for (int wi = 0; wi < 4; wi++) {
      if (psid[wi] < 0) continue;
      if (psid[wi] == s0)
        acc += part[wi][c];
      else
        atomicAdd(a.force_acc + 6 * psid[wi] + c, part[wi][c]);
    }
    if (s0 >= 0) atomicAdd(a.force_acc + 6 * s0 + c, acc);
  }
}

template <typename T>
__global__ void __launch_bounds__(128) k_interp(const IbmArgs a) {
  const int m = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (m >= a.nmark) return;  // whole warp exits together
  const int4 b = a.mk_base[m];
  T U[3];
  interp_marker<T>(a, m, lane, b, U);
  if (lane == 0) {
    const Marker k = marker(a, m);
    const double Ud[3] = {(double)U[0], (double)U[1], (double)U[2]};
    double F[3];
    direct_force(a, k, Ud, F);
    for (int c = 0; c < 3; c++) {
      a.Fm[c * a.nmark + m] = (a.first ? 0.0 : a.Fm[c * a.nmark + m]) + F[c];
      if (a.dF) a.dF[c * a.nmark + m] = F[c];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(128) k_spread(const IbmArgs a) {
  const int warp = threadIdx.x >> 5;
  const int m = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  const bool active = m < a.nmark;
  Marker k;
  double F[3] = {0, 0, 0}, dV = 0;
  if (active) {
    k = marker(a, m);
    F[0] = a.Fm[m];
    F[1] = a.Fm[a.nmark + m];
    F[2] = a.Fm[2 * a.nmark + m];
    dV = a.dV[m];
    if (a.dF) {
      // this iteration's increment onto the force already spread
      const double dF[3] = {a.dF[m], a.dF[a.nmark + m], a.dF[2 * a.nmark + m]};
      spread_marker<T>(a, m, lane, a.mk_base[m], dF);
    } else {
      spread_marker<T>(a, m, lane, a.mk_base[m], F);
    }
  }
  if (a.reduce_force) reduce_solid_force(a, active, lane, warp, k, F, dV);
}

// single forcing iteration: interpolate, force, spread and reduce in one
// pass (each warp spreads the force it just computed)
template <typename T>
__global__ void __launch_bounds__(128) k_fused(const IbmArgs a) {
  const int warp = threadIdx.x >> 5;
  const int m = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  const bool active = m < a.nmark;
  Marker k;
  double F[3] = {0, 0, 0}, dV = 0;
  if (active) {
    const int4 b = a.mk_base[m];
    T U[3];
    interp_marker<T>(a, m, lane, b, U);
    k = marker(a, m);
    const double Ud[3] = {(double)U[0], (double)U[1], (double)U[2]};
    direct_force(a, k, Ud, F);
    if (lane == 0)
      for (int c = 0; c < 3; c++) a.Fm[c * a.nmark + m] = F[c];
    dV = a.dV[m];
    spread_marker<T>(a, m, lane, b, F);
  }
  if (a.reduce_force) reduce_solid_force(a, active, lane, warp, k, F, dV);
}

// ---------------------------------------------------------------- cluster
// The forcing loop of one solid in one thread-block cluster of
// kIbmClusterSize blocks.  The box that holds every stencil point of the
// solid's markers is cut into slabs of planes (z in 3D, y in 2D); block r
// keeps slab r of the unforced velocity u~ and of the spread force f in its
// shared memory, so the cluster's distributed shared memory holds both
// fields of the whole box.  Each block takes a contiguous share of the
// markers, a warp per marker:
//   load u~ (f = 0); cluster barrier;
//   n_it times: interpolate u~ + f at the markers (f = 0 in the first pass)
//   from whichever blocks own the stencil points, F += rho0 (U^d - U),
//   barrier; spread the increment of F with shared-memory atomics into the
//   owners' slabs, barrier;
//   store f to the band field; reduce the solid's force and torque (FP64).
// Spreading each iteration's increment onto the field already spread is the
// same sum as re-spreading the total force of Eq. 9 from zero.  The
// barriers are hardware cluster barriers that every thread reaches the same
// number of times.
template <typename T>
struct BoxView {
  int o[3], w[3], h, plane, slab, sax;
};

template <typename T>
__device__ __forceinline__ BoxView<T> box_view(const IbmArgs &a, const IbmClusterArgs &cl,
                                               int s) {
  BoxView<T> v;
  const IbmBox &B = cl.box[s];
  const int n[3] = {a.nx, a.ny, a.nz};
  for (int c = 0; c < 3; c++) {
    v.o[c] = B.o[c];
    v.w[c] = B.w[c];
  }
  if (cl.box_dev) {
    const SolidDev sd = solid_of(a, s);
    for (int c = 0; c < a.dim; c++)
      if (B.w[c] < n[c]) v.o[c] = (int)floor(sd.c[c] - B.ext);
  }
  v.h = B.h;
  v.sax = a.dim == 3 ? 2 : 1;
  v.plane = a.dim == 3 ? v.w[0] * v.w[1] : v.w[0];
  v.slab = v.h * v.plane;
  return v;
}

// box coordinate of an (unwrapped) lattice coordinate along axis c; the
// boxes leave a node of slack beyond every stencil, and the clamp keeps a
// coordinate that rounding might still push out inside the slab arrays
__device__ __forceinline__ int box_coord(int x, int o, int w, int n) {
  if (w >= n) return wrap(x, n);
  const int l = x - o;
  return l < 0 ? 0 : (l >= w ? w - 1 : l);
}

template <typename T, int CS>
__global__ void __launch_bounds__(256) k_ibm_cluster(const IbmArgs a, const IbmClusterArgs cl) {
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  const int s = (int)blockIdx.x / CS;
  extern __shared__ __align__(16) unsigned char ibm_smem[];
  const BoxView<T> v = box_view<T>(a, cl, s);
  T *uS = (T *)ibm_smem;
  T *fS = uS + 3 * v.slab;
  double *dS = (double *)(fS + 3 * v.slab);           // [mpc][3] force increments
  double *red = dS + 3 * cl.box[s].mpc;                // [6] the solid's force, torque
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarp = blockDim.x >> 5;
  const int npl = v.w[v.sax];
  const int p0 = r * v.h;
  const T *ub = (const T *)a.u_band;
  T *fi = (T *)a.f_ibm;
  auto gnode = [&](int i, bool &in) {
    const int pl = i / v.plane, rem = i - pl * v.plane;
    in = p0 + pl < npl;
    int l[3];
    if (a.dim == 3) {
      l[0] = rem % v.w[0];
      l[1] = rem / v.w[0];
      l[2] = p0 + pl;
    } else {
      l[0] = rem;
      l[1] = p0 + pl;
      l[2] = 0;
    }
    const int x = wrap(v.o[0] + l[0], a.nx), y = wrap(v.o[1] + l[1], a.ny);
    const int z = a.dim == 3 ? wrap(v.o[2] + l[2], a.nz) : 0;
    return x + (long long)a.nx * (y + (long long)a.ny * z);
  };
  for (int i = tid; i < v.slab; i += blockDim.x) {
    bool in;
    const long long n = gnode(i, in);
    for (int c = 0; c < 3; c++) {
      uS[c * v.slab + i] = in ? ub[c * a.N + n] : (T)0;
      fS[c * v.slab + i] = (T)0;
    }
  }
  if (tid < 6) red[tid] = 0.0;
  cluster.sync();
  const int npts = a.dim == 3 ? 64 : 16;
  const int mpc = cl.box[s].mpc;
  const int mb = cl.mk_start[s] + r * mpc;
  const int me = min(cl.mk_start[s + 1], mb + mpc);
  // owner block and slot of stencil point p of a marker with base b
  auto where = [&](int4 b, int p, int &owner, int &idx) {
    const int kx = p & 3, ky = (p >> 2) & 3, kz = p >> 4;
    const int lx = box_coord(b.x + kx, v.o[0], v.w[0], a.nx);
    const int ly = box_coord(b.y + ky, v.o[1], v.w[1], a.ny);
    const int lz = a.dim == 3 ? box_coord(b.z + kz, v.o[2], v.w[2], a.nz) : 0;
    const int ls = a.dim == 3 ? lz : ly;
    owner = ls / v.h;
    const int in_plane = a.dim == 3 ? ly * v.w[0] + lx : lx;
    idx = (ls - owner * v.h) * v.plane + in_plane;
  };
  for (int it = 0; it < cl.iters; it++) {
    // interpolation and direct force: every block reads the fields as they
    // stood at the last barrier
    for (int m = mb + wid; m < me; m += nwarp) {
      const int4 b = a.mk_base[m];
      const T *wts = (const T *)a.mk_wts + (long long)m * npts;
      T U[3] = {(T)0, (T)0, (T)0};
      for (int p = lane; p < npts; p += 32) {
        int owner, idx;
        where(b, p, owner, idx);
        const T *ur = cluster.map_shared_rank(uS, owner);
        const T *fr = cluster.map_shared_rank(fS, owner);
        const T wgt = wts[p];
        for (int c = 0; c < a.dim; c++) {
          T val = ur[c * v.slab + idx];
          if (it > 0) val += fr[c * v.slab + idx];  // u~ + f dt / rho0, rho0 = 1
          U[c] += wgt * val;
        }
      }
      for (int c = 0; c < 3; c++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) U[c] += __shfl_xor_sync(0xffffffffu, U[c], o);
      const Marker k = marker(a, m);
      const double Ud[3] = {(double)U[0], (double)U[1], (double)U[2]};
      double F[3];
      direct_force(a, k, Ud, F);
      if (lane == 0)
        for (int c = 0; c < 3; c++) {
          dS[3 * (m - mb) + c] = F[c];
          a.Fm[c * a.nmark + m] = (it == 0 ? 0.0 : a.Fm[c * a.nmark + m]) + F[c];
        }
    }
    cluster.sync();
    // spreading of the increments into the owners' slabs
    for (int m = mb + wid; m < me; m += nwarp) {
      const int4 b = a.mk_base[m];
      const T *wts = (const T *)a.mk_wts + (long long)m * npts;
      const double dV = a.dV[m];
      const T FdV[3] = {(T)(dS[3 * (m - mb)] * dV), (T)(dS[3 * (m - mb) + 1] * dV),
                        (T)(dS[3 * (m - mb) + 2] * dV)};
      for (int p = lane; p < npts; p += 32) {
        int owner, idx;
        where(b, p, owner, idx);
        T *fr = cluster.map_shared_rank(fS, owner);
        const T wgt = wts[p];
        for (int c = 0; c < a.dim; c++) atomicAdd(fr + c * v.slab + idx, FdV[c] * wgt);
      }
    }
    cluster.sync();
  }
  // the spread force of this block's slab to the band field
  for (int i = tid; i < v.slab; i += blockDim.x) {
    bool in;
    const long long n = gnode(i, in);
    if (!in) continue;
    for (int c = 0; c < a.dim; c++) fi[c * a.N + n] = fS[c * v.slab + i];
  }
  // force on the solid: minus the marker forces (Eq. 45), FP64
  for (int m = mb + wid; m < me; m += nwarp) {
    if (lane != 0) continue;
    const Marker k = marker(a, m);
    const double dV = a.dV[m];
    const double Fs[3] = {-a.Fm[m] * dV, -a.Fm[a.nmark + m] * dV, -a.Fm[2 * a.nmark + m] * dV};
    atomicAdd(red + 0, Fs[0]);
    atomicAdd(red + 1, Fs[1]);
    atomicAdd(red + 2, Fs[2]);
    atomicAdd(red + 3, k.r[1] * Fs[2] - k.r[2] * Fs[1]);
    atomicAdd(red + 4, k.r[2] * Fs[0] - k.r[0] * Fs[2]);
    atomicAdd(red + 5, k.r[0] * Fs[1] - k.r[1] * Fs[0]);
  }
  __syncthreads();
  if (tid < 6 && me > mb) atomicAdd(a.force_acc + 6 * s + tid, red[tid]);
}

}  // namespace

void launch_ibm_prepare(const IbmArgs &a, int precision, cudaStream_t st) {
  if (a.nmark <= 0) return;
  const unsigned grid = (unsigned)((32LL * a.nmark + 127) / 128);
  if (precision == LBM_FP64)
    k_prepare<double><<<grid, 128, 0, st>>>(a);
  else
    k_prepare<float><<<grid, 128, 0, st>>>(a);
}

void launch_ibm_fused(const IbmArgs &a, int precision, cudaStream_t st) {
  if (a.nmark <= 0) return;
  const unsigned grid = (unsigned)((32LL * a.nmark + 127) / 128);
  if (precision == LBM_FP64)
    k_fused<double><<<grid, 128, 0, st>>>(a);
  else
    k_fused<float><<<grid, 128, 0, st>>>(a);
}

void launch_ibm_interp(const IbmArgs &a, int precision, cudaStream_t st) {
  if (a.nmark <= 0) return;
  const unsigned grid = (unsigned)((32LL * a.nmark + 127) / 128);
  if (precision == LBM_FP64)
    k_interp<double><<<grid, 128, 0, st>>>(a);
  else
    k_interp<float><<<grid, 128, 0, st>>>(a);
}

void launch_ibm_spread(const IbmArgs &a, int precision, cudaStream_t st) {
  if (a.nmark <= 0) return;
  const unsigned grid = (unsigned)((32LL * a.nmark + 127) / 128);
  if (precision == LBM_FP64)
    k_spread<double><<<grid, 128, 0, st>>>(a);
  else
    k_spread<float><<<grid, 128, 0, st>>>(a);
}

size_t ibm_cluster_smem(const IbmClusterArgs &cl, int precision) {
  const size_t t = precision == LBM_FP64 ? 8 : 4;
  size_t most = 0;
  for (int s = 0; s < cl.ns; s++) {
    const IbmBox &B = cl.box[s];
    const size_t plane = (size_t)B.w[0] * (cl.dim == 3 ? B.w[1] : 1);
    const size_t bytes = 6 * (size_t)B.h * plane * t + 8 * (3 * (size_t)B.mpc + 6) + 16;
    most = bytes > most ? bytes : most;
  }
  return most;
}

template <typename T>
cudaLaunchConfig_t cluster_config(const IbmClusterArgs &cl, size_t smem, cudaStream_t st,
                                  cudaLaunchAttribute *attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(cl.ns * kIbmClusterSize));
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kIbmClusterSize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

template <typename T>
bool cluster_fits_t(const IbmClusterArgs &cl, size_t smem) {
  auto kern = k_ibm_cluster<T, kIbmClusterSize>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) !=
      cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = cluster_config<T>(cl, smem, nullptr, attr);
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return clusters >= 1;
}

bool ibm_cluster_fits(const IbmClusterArgs &cl, int precision) {
  if (cl.ns < 1) return false;
  const size_t smem = ibm_cluster_smem(cl, precision);
  if (smem > 227 * 1024) return false;
  return precision == LBM_FP64 ? cluster_fits_t<double>(cl, smem) : cluster_fits_t<float>(cl, smem);
}

template <typename T>
void launch_cluster_t(const IbmArgs &a, const IbmClusterArgs &cl, size_t smem, cudaStream_t st) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = cluster_config<T>(cl, smem, st, attr);
  cudaLaunchKernelEx(&cfg, k_ibm_cluster<T, kIbmClusterSize>, a, cl);
}

void launch_ibm_cluster(const IbmArgs &a, const IbmClusterArgs &cl, int precision,
                        cudaStream_t st) {
  const size_t smem = ibm_cluster_smem(cl, precision);
  if (precision == LBM_FP64)
    launch_cluster_t<double>(a, cl, smem, st);
  else
    launch_cluster_t<float>(a, cl, smem, st);
}

}  // namespace lbm
