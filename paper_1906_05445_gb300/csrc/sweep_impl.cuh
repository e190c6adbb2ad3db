// sweep_impl.cuh -- the fused pull collide-stream sweep of plain fluid
// nodes (the bulk kernel) and the helpers it shares with the boundary-node,
// query and refill kernels of boundary_impl.cuh.
//
// Pull scheme: array `src` holds post-collision deviations f*(t); node x
// gathers f_i(x, t+1) = f*_i(x - e_i, t), collides (Eq. 1 / Eq. 3 with Guo
// forcing) and writes f*(x, t+1) into `dst`.  Plain fluid nodes (flag 0) run
// in the bulk kernel; nodes with cut links, IBM forcing or no external force
// run from a compacted list in the boundary-node kernel, which replaces the
// pulled value on each cut link by the interpolated bounce-back rule of
// Sec. 2.2 and accumulates the momentum exchange of Eq. 17 in FP64.
#pragma once

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

template <typename T> __device__ __forceinline__ constexpr bool is_f32() {
  return sizeof(T) == 4;
}

template <int LAT, typename T>
__device__ __forceinline__ Coll<T> make_coll(const KArgs &a) {
  Coll<T> c;
  if constexpr (is_f32<T>()) {
    c.omega = a.omega_f;
    c.omc = 1.0f - a.omega_f;
    c.cforce = 1.0f - 0.5f * a.omega_f;
#pragma unroll
    for (int k = 0; k < Lat<LAT>::Q; k++) c.ds[k] = a.ds_f[k];
  } else {
    c.omega = (T)a.omega;
    c.omc = (T)(1.0 - a.omega);
    c.cforce = (T)(1.0 - 0.5 * a.omega);
#pragma unroll
    for (int k = 0; k < Lat<LAT>::Q; k++) c.ds[k] = (T)a.ds[k];
  }
  return c;
}

// body force component and storage scale in the compute type
template <typename T> __device__ __forceinline__ T kg(const KArgs &a, int c) {
  if constexpr (is_f32<T>()) return a.g_f[c];
  else return (T)a.g[c];
}
template <typename T> __device__ __forceinline__ T kisc(const KArgs &a) {
  if constexpr (is_f32<T>()) return a.inv_scale_f;
  else return (T)a.inv_scale;
}

__device__ __forceinline__ void node_xyz(long long n, int nx, int ny, int &x,
                                         int &y, int &z) {
  x = (int)(n % nx);
  long long r = n / nx;
  y = (int)(r % ny);
  z = (int)(r / ny);
}

// Force density at a node: g unless FL_NOG, plus the spread IBM force.
template <typename T, typename LT>
__device__ __forceinline__ void node_force(const KArgs &a, long long n,
                                           uint8_t fl, T &Fx, T &Fy, T &Fz) {
  const bool g = !(fl & FL_NOG);
  Fx = g ? kg<T>(a, 0) : (T)0;
  Fy = g ? kg<T>(a, 1) : (T)0;
  Fz = g ? kg<T>(a, 2) : (T)0;
  if (fl & FL_BAND) {
    const LT *fi = (const LT *)a.f_ibm;
    Fx += (T)fi[n];
    Fy += (T)fi[a.N + n];
    Fz += (T)fi[2 * a.N + n];
  }
}

// Pull the Q populations of node (x, y, z) from src with periodic wrap.
template <int LAT, typename S, typename T, int EVICT_FIRST = 0>
__device__ __forceinline__ void gather_pull(const S *__restrict__ src,
                                            long long fs, int x, int y, int z,
                                            int nx, int ny, int nz, T isc,
                                            T (&f)[Lat<LAT>::Q]) {
  using L = Lat<LAT>;
  const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
  // row offsets of the source rows (y - e_y, z - e_z)
  const long long r[3][3] = {
      {(long long)nx * (ym + (long long)ny * zm), (long long)nx * (y + (long long)ny * zm),
       (long long)nx * (yp + (long long)ny * zm)},
      {(long long)nx * (ym + (long long)ny * z), (long long)nx * (y + (long long)ny * z),
       (long long)nx * (yp + (long long)ny * z)},
      {(long long)nx * (ym + (long long)ny * zp), (long long)nx * (y + (long long)ny * zp),
       (long long)nx * (yp + (long long)ny * zp)}};
  static_for<L::Q>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    // source node x - e_i
    const int sx = L::ex(i) > 0 ? xm : (L::ex(i) < 0 ? xp : x);
    const long long row = r[1 - L::ez(i)][1 - L::ey(i)];
    if constexpr (EVICT_FIRST)
      f[i] = Store<S>::ld_stream(src + (long long)i * fs + row + sx, isc);
    else
      f[i] = Store<S>::ld(src + (long long)i * fs + row + sx, isc);
  });
}

template <int LAT, typename S, typename T>
__device__ __forceinline__ void gather_local(const S *__restrict__ src,
                                             long long fs, long long n, T isc,
                                             T (&f)[Lat<LAT>::Q]) {
  static_for<Lat<LAT>::Q>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    f[i] = Store<S>::ld(src + (long long)i * fs + n, isc);
  });
}

template <int LAT, typename S, typename T, bool STREAM = false>
__device__ __forceinline__ void scatter(S *__restrict__ dst, long long fs,
                                        long long n, T isc,
                                        const T (&f)[Lat<LAT>::Q]) {
  static_for<Lat<LAT>::Q>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    if constexpr (STREAM)
      Store<S>::st_stream(dst + (long long)i * fs + n, f[i], isc);
    else
      Store<S>::st(dst + (long long)i * fs + n, f[i], isc);
  });
}

// ---------------------------------------------------------------- bulk sweep
// one thread per node, nodes in memory order (x fastest) so that every
// direction's loads and stores of a warp are contiguous
template <int LAT, int CM, typename S, typename T, int HINT>
__global__ void __launch_bounds__(512) k_bulk_sweep(const KArgs a) {
  const unsigned n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= (unsigned)a.N) return;
  // plain fluid nodes; nodes inside an IBM solid (FL_NOG) also run here,
  // without the external force, and so do nodes refilled this step (FL_NEW)
  const uint8_t fl = a.flags[n];
  if (fl & (uint8_t)~(FL_NOG | FL_NEW)) return;
  const unsigned yz = n / (unsigned)a.nx;
  const int x = (int)(n - yz * (unsigned)a.nx);
  const int z = (int)(yz / (unsigned)a.ny);
  const int y = (int)(yz - (unsigned)z * (unsigned)a.ny);
  const T isc = kisc<T>(a);
  T f[Lat<LAT>::Q];
  gather_pull<LAT, S, T, (HINT & 1)>((const S *)a.src, a.fs, x, y, z, a.nx, a.ny, a.nz, isc, f);
  const Coll<T> c = make_coll<LAT, T>(a);
  const T gon = (fl & FL_NOG) ? (T)0 : (T)1;
  collide<LAT, CM, T>(f, gon * kg<T>(a, 0), gon * kg<T>(a, 1), gon * kg<T>(a, 2), c);
  scatter<LAT, S, T, (HINT & 2) != 0>((S *)a.dst, a.fs, n, isc, f);
}

}  // namespace lbm
