// sweep_impl.cuh -- the fused pull collide-stream sweep and its relatives,
// instantiated once per storage type by sweep_<precision>.cu.
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
template <int LAT, typename S, typename T>
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

template <int LAT, typename S, typename T>
__device__ __forceinline__ void scatter(S *__restrict__ dst, long long fs,
                                        long long n, T isc,
                                        const T (&f)[Lat<LAT>::Q]) {
  static_for<Lat<LAT>::Q>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    Store<S>::st(dst + (long long)i * fs + n, f[i], isc);
  });
}

// Interpolated bounce-back value of cut link (x_f, i) from post-collision
// deviations (coefficients of Sec. 2.2, precomputed per link):
//   f_i(x_f,t+1) = c0 f*_ib(x_f) + c1 f*_ib(x_ff) + c2 f*_ib(x_fff)
//                + c3 f*_i(x_f) + c4 f*_i(x_ff) + mw.
template <int LAT, typename S, typename T, typename LT>
__device__ __forceinline__ T ibb_value(const KArgs &a, const S *__restrict__ src,
                                       int i, int x, int y, int z, long long n,
                                       int link, T isc, T &fs) {
  using L = Lat<LAT>;
  const int ib = L::opp(i);
  const LT *c0 = (const LT *)a.links.c[0], *c1 = (const LT *)a.links.c[1],
           *c2 = (const LT *)a.links.c[2], *c3 = (const LT *)a.links.c[3],
           *c4 = (const LT *)a.links.c[4], *mw = (const LT *)a.links.mw;
  const long long N = a.fs;
  const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
  fs = Store<S>::ld(src + (long long)ib * N + n, isc);
  T v = (T)c0[link] * fs + (T)mw[link];
  const T k1 = (T)c1[link], k2 = (T)c2[link], k3 = (T)c3[link], k4 = (T)c4[link];
  if (k1 != (T)0 || k2 != (T)0 || k4 != (T)0) {
    const long long nff = wrap(x + ex, a.nx) +
                          (long long)a.nx * (wrap(y + ey, a.ny) + (long long)a.ny * wrap(z + ez, a.nz));
    if (k1 != (T)0) v += k1 * Store<S>::ld(src + (long long)ib * N + nff, isc);
    if (k4 != (T)0) v += k4 * Store<S>::ld(src + (long long)i * N + nff, isc);
    if (k2 != (T)0) {
      const long long nfff = wrap(x + 2 * ex, a.nx) +
                             (long long)a.nx * (wrap(y + 2 * ey, a.ny) +
                                                (long long)a.ny * wrap(z + 2 * ez, a.nz));
      v += k2 * Store<S>::ld(src + (long long)ib * N + nfff, isc);
    }
  }
  if (k3 != (T)0) v += k3 * Store<S>::ld(src + (long long)i * N + n, isc);
  return v;
}

// FP64 outputs of a query at one node from pre-collision deviations f.
template <int LAT, typename T>
__device__ __forceinline__ void write_fields(const KArgs &a, long long n,
                                             const T (&f)[Lat<LAT>::Q], T Fx,
                                             T Fy, T Fz) {
  using L = Lat<LAT>;
  constexpr int Q = L::Q, D = L::D;
  double fd[Q];
  double drho = 0, j[3] = {0, 0, 0};
#pragma unroll
  for (int i = 0; i < Q; i++) {
    fd[i] = (double)f[i];
    drho += fd[i];
    j[0] += L::ex(i) * fd[i];
    j[1] += L::ey(i) * fd[i];
    j[2] += L::ez(i) * fd[i];
  }
  const double F[3] = {(double)Fx, (double)Fy, (double)Fz};
  const double u[3] = {j[0] + 0.5 * F[0], j[1] + 0.5 * F[1], j[2] + 0.5 * F[2]};
  if (a.out_rho) a.out_rho[n] = 1.0 + drho;
  if (a.out_u)
    for (int c = 0; c < D; c++) a.out_u[c * a.N + n] = u[c];
  if (a.out_f)
#pragma unroll
    for (int i = 0; i < Q; i++) a.out_f[(long long)i * a.N + n] = L::w(i) + fd[i];
  if (a.out_S || a.out_stress) {
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double P[3][3];
    for (int p = 0; p < 3; p++)
      for (int q = 0; q < 3; q++) P[p][q] = 0.5 * (F[p] * u[q] + u[p] * F[q]);
#pragma unroll
    for (int i = 0; i < Q; i++) {
      const double neq = fd[i] - feq_dev<LAT, double>(i, drho, u[0], u[1], u[2], uu);
      const int e[3] = {L::ex(i), L::ey(i), L::ez(i)};
      for (int p = 0; p < 3; p++)
        for (int q = 0; q < 3; q++) P[p][q] += neq * e[p] * e[q];
    }
    double tr = 0;
    for (int p = 0; p < D; p++) tr += P[p][p];
    const int nc = D == 2 ? 3 : 6;
    const int ca[6] = {0, 1, D == 2 ? 0 : 2, 0, 1, 0};
    const int cb[6] = {0, 1, D == 2 ? 1 : 2, 1, 2, 2};
    for (int c = 0; c < nc; c++) {
      const int p = ca[c], q = cb[c];
      const double iso = p == q ? tr / D : 0.0;
      const double S = -1.5 * (a.omega * (P[p][q] - iso) + a.s_bulk * iso);
      if (a.out_S) a.out_S[c * a.N + n] = S;
      if (a.out_stress)
        a.out_stress[c * a.N + n] = (p == q ? -(1.0 + drho) / 3.0 : 0.0) + 2.0 * a.nu * S;
    }
  }
}

// ---------------------------------------------------------------- kernels
// one thread per node, nodes in memory order (x fastest) so that every
// direction's loads and stores of a warp are contiguous
template <int LAT, bool MRT, typename S, typename T>
__global__ void __launch_bounds__(512) k_bulk_sweep(const KArgs a) {
  const unsigned n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= (unsigned)a.N) return;
  if (a.flags[n] != 0) return;
  const unsigned yz = n / (unsigned)a.nx;
  const int x = (int)(n - yz * (unsigned)a.nx);
  const int z = (int)(yz / (unsigned)a.ny);
  const int y = (int)(yz - (unsigned)z * (unsigned)a.ny);
  const T isc = kisc<T>(a);
  T f[Lat<LAT>::Q];
  gather_pull<LAT, S, T>((const S *)a.src, a.fs, x, y, z, a.nx, a.ny, a.nz, isc, f);
  const Coll<T> c = make_coll<LAT, T>(a);
  collide<LAT, MRT, T>(f, kg<T>(a, 0), kg<T>(a, 1), kg<T>(a, 2), c);
  scatter<LAT, S, T>((S *)a.dst, a.fs, n, isc, f);
}

template <int LAT, typename S>
__global__ void __launch_bounds__(512) k_bulk_query(const KArgs a) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= a.nx) return;
  const long long n = x + (long long)a.nx * (y + (long long)a.ny * z);
  if (a.flags[n] != 0) return;
  double f[Lat<LAT>::Q];
  gather_pull<LAT, S, double>((const S *)a.src, a.fs, x, y, z, a.nx, a.ny, a.nz,
                              a.inv_scale, f);
  write_fields<LAT, double>(a, n, f, a.g[0], a.g[1], a.g[2]);
}

// Warp-sum of a double.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Boundary-node sweep (MODE 0) or query (MODE 1): one thread per list node.
template <int LAT, bool MRT, typename S, typename T, typename LT, int MODE>
__global__ void __launch_bounds__(64) k_list(const KArgs a) {
  using L = Lat<LAT>;
  constexpr int Q = L::Q;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  int cnt = a.counts[0];
  if (cnt > a.list_cap) cnt = a.list_cap;
  const bool active = t < cnt;
  const T isc = kisc<T>(a);
  const S *__restrict__ src = (const S *)a.src;
  // momentum exchange (Eq. 17) of this thread for solid `sa` (the solid of
  // its first cut link): the state-independent part -2 w_i e_i of every
  // link was summed per node in FP64 when the geometry was built; the part
  // linear in the deviations is formed here in the compute type and the
  // sums are reduced in FP64
  double acc[6] = {0, 0, 0, 0, 0, 0};
  T dacc[6] = {0, 0, 0, 0, 0, 0};
  int sa = -1;
  if (active) {
    const long long n = a.list_node[t];
    const uint32_t mask = a.list_mask[t];
    int link = a.list_link[t];
    int x, y, z;
    node_xyz(n, a.nx, a.ny, x, y, z);
    T f[Q];
    if (a.local_gather)
      gather_local<LAT, S, T>(src, a.fs, n, isc, f);
    else
      gather_pull<LAT, S, T>(src, a.fs, x, y, z, a.nx, a.ny, a.nz, isc, f);
    if (mask && !a.local_gather) {
#pragma unroll
      for (int i = 1; i < Q; i++) {
        if (!((mask >> i) & 1u)) continue;
        T fs;
        const T v = ibb_value<LAT, S, T, LT>(a, src, i, x, y, z, n, link, isc, fs);
        f[i] = v;
        if (MODE == 0) {
          const int s = a.links.sid[link];
          if (sa < 0) sa = s;
          const T e[3] = {(T)L::ex(i), (T)L::ey(i), (T)L::ez(i)};
          const LT *uw0 = (const LT *)a.links.uw[0], *uw1 = (const LT *)a.links.uw[1],
                   *uw2 = (const LT *)a.links.uw[2];
          const LT *ar0 = (const LT *)a.links.arm[0], *ar1 = (const LT *)a.links.arm[1],
                   *ar2 = (const LT *)a.links.arm[2];
          const T uw[3] = {(T)uw0[link], (T)uw1[link], (T)uw2[link]};
          const T r[3] = {(T)ar0[link], (T)ar1[link], (T)ar2[link]};
          if (s == sa) {
            // f*_ib(e_ib - u_w) - f_i(e_i - u_w) = -2 w_i e_i
            //   - d*_ib (e_i + u_w) - d_i (e_i - u_w)   (d: deviations)
            T dp[3];
            for (int c = 0; c < 3; c++) dp[c] = -fs * (e[c] + uw[c]) - v * (e[c] - uw[c]);
            dacc[0] += dp[0];
            dacc[1] += dp[1];
            dacc[2] += dp[2];
            dacc[3] += r[1] * dp[2] - r[2] * dp[1];
            dacc[4] += r[2] * dp[0] - r[0] * dp[2];
            dacc[5] += r[0] * dp[1] - r[1] * dp[0];
          } else {
            // a second solid seen from the same node (narrow gap): full FP64
            const double wi = L::w(i);
            const double fsd = wi + (double)fs, fid = wi + (double)v;
            double dp[3];
            for (int c = 0; c < 3; c++)
              dp[c] = fsd * (-(double)e[c] - (double)uw[c]) - fid * ((double)e[c] - (double)uw[c]);
            const double rr[3] = {(double)r[0], (double)r[1], (double)r[2]};
            atomicAdd(a.force_acc + 6 * s + 0, dp[0]);
            atomicAdd(a.force_acc + 6 * s + 1, dp[1]);
            atomicAdd(a.force_acc + 6 * s + 2, dp[2]);
            atomicAdd(a.force_acc + 6 * s + 3, rr[1] * dp[2] - rr[2] * dp[1]);
            atomicAdd(a.force_acc + 6 * s + 4, rr[2] * dp[0] - rr[0] * dp[2]);
            atomicAdd(a.force_acc + 6 * s + 5, rr[0] * dp[1] - rr[1] * dp[0]);
          }
        }
        link++;
      }
      if (MODE == 0 && sa >= 0)
        for (int c = 0; c < 6; c++) acc[c] = a.list_cst[c * a.list_cap + t] + (double)dacc[c];
    }
    const uint8_t fl = a.flags[n];
    T Fx, Fy, Fz;
    node_force<T, LT>(a, n, fl, Fx, Fy, Fz);
    if (MODE == 0) {
      const Coll<T> c = make_coll<LAT, T>(a);
      collide<LAT, MRT, T>(f, Fx, Fy, Fz, c);
      scatter<LAT, S, T>((S *)a.dst, a.fs, n, isc, f);
    } else {
      write_fields<LAT, T>(a, n, f, Fx, Fy, Fz);
    }
  }
  if (MODE == 0 && a.force_acc) {
    const int lane = threadIdx.x & 31;
    for (int s = 0; s < a.nsolids; s++) {
      if (!__any_sync(0xffffffffu, sa == s)) continue;
      for (int c = 0; c < 6; c++) {
        const double v = warp_sum(sa == s ? acc[c] : 0.0);
        if (lane == 0) atomicAdd(a.force_acc + 6 * s + c, v);
      }
    }
  }
}

// Local read of a pre-collision state: collide into dst (MODE 0) or write
// fields (MODE 1).  One thread per node.
template <int LAT, bool MRT, typename S, typename T, typename LT, int MODE>
__global__ void __launch_bounds__(256) k_local(const KArgs a) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.N) return;
  const uint8_t fl = a.flags[n];
  if (fl & FL_SOLID) return;
  const T isc = kisc<T>(a);
  T f[Lat<LAT>::Q];
  gather_local<LAT, S, T>((const S *)a.src, a.fs, n, isc, f);
  T Fx, Fy, Fz;
  node_force<T, LT>(a, n, fl, Fx, Fy, Fz);
  if (MODE == 0) {
    const Coll<T> c = make_coll<LAT, T>(a);
    collide<LAT, MRT, T>(f, Fx, Fy, Fz, c);
    scatter<LAT, S, T>((S *)a.dst, a.fs, n, isc, f);
  } else {
    write_fields<LAT, T>(a, n, f, Fx, Fy, Fz);
  }
}

// Refill of nodes uncovered by a moving solid: equilibrium at the mean
// density of neighbours fluid before and after the move and at the local
// wall velocity, then the node's collision, written into the current
// post-collision array (src == dst).
template <int LAT, bool MRT, typename S, typename T>
__global__ void __launch_bounds__(128) k_refill(const KArgs a) {
  using L = Lat<LAT>;
  constexpr int Q = L::Q;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  int cnt = a.counts[2];
  if (cnt > a.refill_cap) cnt = a.refill_cap;
  if (t >= cnt) return;
  const long long n = a.refill_node[t];
  const int sidx = a.refill_sid[t];
  int x, y, z;
  node_xyz(n, a.nx, a.ny, x, y, z);
  const S *src = (const S *)a.src;
  const T isc = kisc<T>(a);
  double rs = 0;
  int cntn = 0;
#pragma unroll
  for (int j = 1; j < Q; j++) {
    const long long nb = wrap(x + L::ex(j), a.nx) +
                         (long long)a.nx * (wrap(y + L::ey(j), a.ny) +
                                            (long long)a.ny * wrap(z + L::ez(j), a.nz));
    if (a.sid[nb] != 0 || (a.flags[nb] & FL_NEW)) continue;
    double r = 1.0;
    for (int k = 0; k < Q; k++) r += (double)Store<S>::ld(src + (long long)k * a.fs + nb, isc);
    rs += r;
    cntn++;
  }
  const double rho = cntn ? rs / cntn : 1.0;
  const SolidDev &b = a.solids.s[sidx];
  double r[3] = {x - b.c[0], y - b.c[1], z - b.c[2]};
  r[0] -= a.nx * round(r[0] / a.nx);
  r[1] -= a.ny * round(r[1] / a.ny);
  r[2] = (L::D == 2 || b.kind == 1) ? 0.0 : r[2] - a.nz * round(r[2] / a.nz);
  double uw[3] = {b.U[0] + b.Om[1] * r[2] - b.Om[2] * r[1],
                  b.U[1] + b.Om[2] * r[0] - b.Om[0] * r[2],
                  b.U[2] + b.Om[0] * r[1] - b.Om[1] * r[0]};
  if (L::D == 2) uw[2] = 0;
  const double uu = uw[0] * uw[0] + uw[1] * uw[1] + uw[2] * uw[2];
  T f[Q];
#pragma unroll
  for (int i = 0; i < Q; i++) f[i] = (T)feq_dev<LAT, double>(i, rho - 1.0, uw[0], uw[1], uw[2], uu);
  T Fx, Fy, Fz;
  node_force<T, T>(a, n, a.flags[n], Fx, Fy, Fz);
  const Coll<T> c = make_coll<LAT, T>(a);
  collide<LAT, MRT, T>(f, Fx, Fy, Fz, c);
  scatter<LAT, S, T>((S *)a.dst, a.fs, n, isc, f);
}

// IBM: unforced velocity u~ = (sum f e + g/2)/rho0 at band nodes (the
// external half force only, no IBM half force) and zero the IBM force there.
template <int LAT, typename S, typename T>
__global__ void __launch_bounds__(64) k_band_vel(const KArgs a) {
  using L = Lat<LAT>;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  int cnt = a.counts[0];
  if (cnt > a.list_cap) cnt = a.list_cap;
  if (t >= cnt) return;
  const long long n = a.list_node[t];
  const uint8_t fl = a.flags[n];
  if (!(fl & FL_BAND)) return;
  int x, y, z;
  node_xyz(n, a.nx, a.ny, x, y, z);
  T f[L::Q];
  const T isc = kisc<T>(a);
  if (a.local_gather)
    gather_local<LAT, S, T>((const S *)a.src, a.fs, n, isc, f);
  else
    gather_pull<LAT, S, T>((const S *)a.src, a.fs, x, y, z, a.nx, a.ny, a.nz, isc, f);
  T j[3] = {0, 0, 0};
#pragma unroll
  for (int i = 0; i < L::Q; i++) {
    j[0] += (T)L::ex(i) * f[i];
    j[1] += (T)L::ey(i) * f[i];
    j[2] += (T)L::ez(i) * f[i];
  }
  const bool g = !(fl & FL_NOG);
  T *ub = (T *)a.u_band;
  T *fi = (T *)a.f_ibm;
  for (int c = 0; c < 3; c++) {
    ub[c * a.N + n] = j[c] + (g ? (T)0.5 * kg<T>(a, c) : (T)0);
    fi[c * a.N + n] = (T)0;
  }
}

// Full FP64 f -> stored deviations (solid nodes get 0).
template <int LAT, typename S, typename T>
__global__ void __launch_bounds__(256) k_from_double(const KArgs a) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.N) return;
  const bool solid = a.flags[n] & FL_SOLID;
  const T isc = kisc<T>(a);
#pragma unroll
  for (int i = 0; i < Lat<LAT>::Q; i++) {
    const double v = solid ? 0.0 : a.out_f[(long long)i * a.N + n] - Lat<LAT>::w(i);
    Store<S>::st((S *)a.dst + (long long)i * a.fs + n, (T)v, isc);
  }
}

// Equilibrium deviations at (rho, u): rho in omega, u in g[].
template <int LAT, typename S, typename T>
__global__ void __launch_bounds__(256) k_fill_eq(const KArgs a) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.N) return;
  const double ux = a.g[0], uy = a.g[1], uz = a.g[2];
  const double uu = ux * ux + uy * uy + uz * uz;
  const T isc = kisc<T>(a);
#pragma unroll
  for (int i = 0; i < Lat<LAT>::Q; i++)
    Store<S>::st((S *)a.dst + (long long)i * a.fs + n,
                 (T)feq_dev<LAT, double>(i, a.omega - 1.0, ux, uy, uz, uu), isc);
}

// ---------------------------------------------------------------- launch
inline int div_up(long long a, int b) { return (int)((a + b - 1) / b); }

template <int LAT, bool MRT, typename S, typename T>
void launch_one(SweepOp op, const KArgs &a, cudaStream_t st) {
  const int want = a.bulk_block > 0 ? a.bulk_block : 128;
  const int bx = a.nx >= want ? want : ((a.nx + 31) / 32) * 32;
  const dim3 gbulk(div_up(a.nx, bx), a.ny, a.nz);
  const int lc = a.list_cap > 0 ? a.list_cap : 1;
  switch (op) {
  case OP_BULK_SWEEP:
    k_bulk_sweep<LAT, MRT, S, T><<<div_up(a.N, want), want, 0, st>>>(a);
    break;
  case OP_BULK_QUERY:
    k_bulk_query<LAT, S><<<gbulk, bx, 0, st>>>(a);
    break;
  case OP_LIST_SWEEP:  // small blocks: spread the few boundary nodes over many SMs
    if (a.list_cap > 0) k_list<LAT, MRT, S, T, T, 0><<<div_up(lc, 64), 64, 0, st>>>(a);
    break;
  case OP_LIST_QUERY:
    if (a.list_cap > 0) k_list<LAT, MRT, S, double, T, 1><<<div_up(lc, 64), 64, 0, st>>>(a);
    break;
  case OP_LOCAL_INIT:
    k_local<LAT, MRT, S, T, T, 0><<<div_up(a.N, 256), 256, 0, st>>>(a);
    break;
  case OP_LOCAL_QUERY:
    k_local<LAT, MRT, S, double, T, 1><<<div_up(a.N, 256), 256, 0, st>>>(a);
    break;
  case OP_REFILL:
    if (a.refill_cap > 0) k_refill<LAT, MRT, S, T><<<div_up(a.refill_cap, 128), 128, 0, st>>>(a);
    break;
  case OP_BAND_VEL:
    if (a.list_cap > 0) k_band_vel<LAT, S, T><<<div_up(lc, 64), 64, 0, st>>>(a);
    break;
  case OP_FROM_DOUBLE:
    k_from_double<LAT, S, T><<<div_up(a.N, 256), 256, 0, st>>>(a);
    break;
  case OP_FILL_EQ:
    k_fill_eq<LAT, S, T><<<div_up(a.N, 256), 256, 0, st>>>(a);
    break;
  }
}

template <typename S, typename T>
void launch_precision(SweepOp op, int lattice, int collision, const KArgs &a,
                      cudaStream_t st) {
  if (lattice == LBM_D2Q9) {
    if (collision == LBM_MRT)
      launch_one<0, true, S, T>(op, a, st);
    else
      launch_one<0, false, S, T>(op, a, st);
  } else {
    if (collision == LBM_MRT)
      launch_one<1, true, S, T>(op, a, st);
    else
      launch_one<1, false, S, T>(op, a, st);
  }
}

}  // namespace lbm
