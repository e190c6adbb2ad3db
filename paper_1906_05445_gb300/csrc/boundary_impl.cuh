// boundary_impl.cuh -- the kernels around the bulk sweep: boundary nodes
// (interpolated bounce-back + Eq. 17), queries, local (initial) collisions,
// refilling, the IBM band velocity, conversions, and the launcher of every
// sweep-like operation.  Instantiated once per storage type by
// sweep_<precision>.cu.
#pragma once

#include "sweep_impl.cuh"
#include "sweep_rows.cuh"
#include "sweep_vec.cuh"

namespace lbm {

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
  if (a.zy_pre) {
    // Eq. 16: the post-collision value leaving the wall at x_f (c3), the
    // pre-collision value arriving at x_f from the previous step (c1) and
    // the moving-wall term
    const LT *pre = (const LT *)a.zy_pre;
    return (T)c3[link] * Store<S>::ld(src + (long long)i * N + n, isc) +
           (T)c1[link] * (T)pre[(long long)ib * N + n] + (T)mw[link];
  }
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
  if (a.out_S || a.out_stress || a.out_eps) {
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
    double ss = 0;
    for (int c = 0; c < nc; c++) {
      const int p = ca[c], q = cb[c];
      const double iso = p == q ? tr / D : 0.0;
      const double S = -1.5 * (a.omega * (P[p][q] - iso) + a.s_bulk * iso);
      if (a.out_S) a.out_S[c * a.N + n] = S;
      if (a.out_stress)
        a.out_stress[c * a.N + n] = (p == q ? -(1.0 + drho) / 3.0 : 0.0) + 2.0 * a.nu * S;
      ss += (p == q ? 1.0 : 2.0) * S * S;
    }
    if (a.out_eps) a.out_eps[n] = 2.0 * a.nu * ss;
  }
}

// ---------------------------------------------------------------- kernels
template <int LAT, typename S>
__global__ void __launch_bounds__(512) k_bulk_query(const KArgs a) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= a.nx) return;
  const long long n = x + (long long)a.nx * (y + (long long)a.ny * z);
  const uint8_t fl = a.flags[n];
  if (fl & (uint8_t)~(FL_NOG | FL_NEW)) return;
  double f[Lat<LAT>::Q];
  gather_pull<LAT, S, double>((const S *)a.src, a.fs, x, y, z, a.nx, a.ny, a.nz,
                              a.inv_scale, f);
  const double gon = (fl & FL_NOG) ? 0.0 : 1.0;
  write_fields<LAT, double>(a, n, f, gon * a.g[0], gon * a.g[1], gon * a.g[2]);
}

// Density and velocity only, for FP32 and 16-bit storage: the same moments
// as write_fields (u = sum e_i d_i + F / 2, rho = 1 + sum d_i) summed in FP32
// arithmetic over the stored values, written as FP64.  GB300's FP64 rate
// makes the FP64 sums the query's bound; in FP32 they differ from them by
// about the FP32 rounding of the sums (1e-7 of the largest term), well
// inside the storage's own error.
template <int LAT, typename S>
__global__ void __launch_bounds__(512) k_bulk_query_u(const KArgs a) {
  using L = Lat<LAT>;
  constexpr int Q = L::Q, D = L::D;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= a.nx) return;
  const long long n = x + (long long)a.nx * (y + (long long)a.ny * z);
  const uint8_t fl = a.flags[n];
  if (fl & (uint8_t)~(FL_NOG | FL_NEW)) return;
  float f[Q];
  gather_pull<LAT, S, float>((const S *)a.src, a.fs, x, y, z, a.nx, a.ny, a.nz, a.inv_scale_f, f);
  float drho = 0.f, j[3] = {0.f, 0.f, 0.f};
  static_for<Q>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    drho += f[i];
    if constexpr (L::ex(i) != 0) j[0] += L::ex(i) > 0 ? f[i] : -f[i];
    if constexpr (L::ey(i) != 0) j[1] += L::ey(i) > 0 ? f[i] : -f[i];
    if constexpr (L::ez(i) != 0) j[2] += L::ez(i) > 0 ? f[i] : -f[i];
  });
  const float gon = (fl & FL_NOG) ? 0.f : 1.f;
  if (a.out_rho) a.out_rho[n] = 1.0 + (double)drho;
  if (a.out_u)
    for (int c = 0; c < D; c++) a.out_u[c * a.N + n] = (double)(j[c] + 0.5f * (gon * a.g_f[c]));
}

// Warp-sum of a double.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Boundary-node sweep (MODE 0) or query (MODE 1): one thread per list node.
template <int LAT, int CM, typename S, typename T, typename LT, int MODE>
__global__ void __launch_bounds__(128) k_list(const KArgs a) {
  using L = Lat<LAT>;
  constexpr int Q = L::Q;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  int cnt = a.counts[0];
  if (cnt > a.list_cap) cnt = a.list_cap;
  // IBM band nodes next to a domain face run in the face kernel
  const bool active = t < cnt && !(a.flags[a.list_node[t]] & FL_FACE);
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
    const bool zy_query = MODE == 1 && a.zy_pre && !a.local_gather;
    if (a.local_gather)
      gather_local<LAT, S, T>(src, a.fs, n, isc, f);
    else if (zy_query)  // Eq. 16 keeps the current pre-collision values here
      for (int i = 0; i < Q; i++) f[i] = (T)((const LT *)a.zy_pre)[(long long)i * a.fs + n];
    else
      gather_pull<LAT, S, T>(src, a.fs, x, y, z, a.nx, a.ny, a.nz, isc, f);
    if (mask && !a.local_gather && !zy_query) {
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
    if (MODE == 0 && a.zy_pre)  // the next step's Eq. 16 reads them
      for (int i = 0; i < Q; i++) ((LT *)a.zy_pre)[(long long)i * a.fs + n] = (LT)f[i];
    const uint8_t fl = a.flags[n];
    T Fx, Fy, Fz;
    node_force<T, LT>(a, n, fl, Fx, Fy, Fz);
    if (MODE == 0) {
      const Coll<T> c = make_coll<LAT, T>(a);
      collide<LAT, CM, T>(f, Fx, Fy, Fz, c);
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

// ---------------------------------------------------------------- warp per
// boundary node.  Lane i (< Q) owns direction i: it pulls f_i or rebuilds it
// with the bounce-back rule, the moments and the q-moment correction are
// warp reductions, and each lane writes its own f*_i.  Compared with a thread
// per node this puts Q times more independent loads in flight for the few
// thousand boundary nodes, which otherwise sit on the critical path.

// per-lane direction tables packed into compile-time integers
template <int LAT> __host__ __device__ constexpr unsigned long long pack_dir(int comp) {
  unsigned long long r = 0;
  for (int i = 0; i < Lat<LAT>::Q; i++) {
    const int e = comp == 0 ? Lat<LAT>::ex(i) : comp == 1 ? Lat<LAT>::ey(i) : Lat<LAT>::ez(i);
    r |= (unsigned long long)(e + 1) << (2 * i);
  }
  return r;
}
template <int LAT> __host__ __device__ constexpr unsigned long long pack_opp() {
  unsigned long long r = 0;
  for (int i = 0; i < Lat<LAT>::Q; i++) r |= (unsigned long long)Lat<LAT>::opp(i) << (5 * (i % 12));
  return r;
}
template <int LAT> __host__ __device__ constexpr unsigned long long pack_opp_hi() {
  unsigned long long r = 0;
  for (int i = 12; i < Lat<LAT>::Q; i++) r |= (unsigned long long)Lat<LAT>::opp(i) << (5 * (i - 12));
  return r;
}

template <typename T> __device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Lane-parallel collision (lane = direction, lanes >= Q carry fi = 0): Eq. 1
// / Eq. 3 with Guo forcing as in collide(), the moments and the q moments of
// MRT as warp reductions.  Returns f*_lane.
template <int LAT, int CM, typename T>
__device__ __forceinline__ T collide_lane(const KArgs &a, T fi, bool dir, int ex, int ey,
                                          int ez, int cls, T w, T Fx, T Fy, T Fz) {
  using L = Lat<LAT>;
  const T drho = wsum<T>(fi);
  const T jx = wsum<T>((T)ex * fi), jy = wsum<T>((T)ey * fi), jz = wsum<T>((T)ez * fi);
  const T ux = jx + (T)0.5 * Fx, uy = jy + (T)0.5 * Fy, uz = jz + (T)0.5 * Fz;
  const T uu = ux * ux + uy * uy + uz * uz, uF = ux * Fx + uy * Fy + uz * Fz;
  const T eu = (T)ex * ux + (T)ey * uy + (T)ez * uz;
  const T eF = (T)ex * Fx + (T)ey * Fy + (T)ez * Fz;
  const T feq = w * (drho + (T)3 * eu + (T)4.5 * eu * eu - (T)1.5 * uu);
  const T fb = w * ((T)3 * (eF - uF) + (T)9 * eu * eF);
  const Coll<T> c = make_coll<LAT, T>(a);
  T out = c.omc * fi + c.omega * feq + c.cforce * fb;
  if constexpr (CM == CM_MRT_Q) {
    const T v = dir ? fi - feq + (T)0.5 * fb : (T)0;
    const T qf = L::D == 3 ? (T)(5 * cls - 9) : (T)(3 * cls - 5);
    const T kq = c.ds[4] * (T)(1.0 / mnorm<LAT>(4));
    const T mx = wsum<T>(qf * (T)ex * v), my = wsum<T>(qf * (T)ey * v);
    T corr = qf * ((T)ex * mx + (T)ey * my);
    if (L::D == 3) corr += qf * (T)ez * wsum<T>(qf * (T)ez * v);
    out += kq * corr;
  }
  return out;
}

template <int LAT, int CM, typename S, typename T>
__global__ void __launch_bounds__(256) k_list_warp(const KArgs a) {
  using L = Lat<LAT>;
  constexpr int Q = L::Q;
  constexpr unsigned long long PX = pack_dir<LAT>(0), PY = pack_dir<LAT>(1), PZ = pack_dir<LAT>(2);
  constexpr unsigned long long PO = pack_opp<LAT>(), POH = pack_opp_hi<LAT>();
  __shared__ double part[8][6];
  __shared__ int psid[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t = blockIdx.x * (blockDim.x >> 5) + warp;  // list entry of this warp
  int cnt = a.counts[0];
  if (cnt > a.list_cap) cnt = a.list_cap;
  const bool active = t < cnt && !(a.flags[a.list_node[t]] & FL_FACE);
  const bool dir = lane < Q;
  const T isc = kisc<T>(a);
  const S *__restrict__ src = (const S *)a.src;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  int sa = -1;
  if (active) {
    const long long n = a.list_node[t];
    const uint32_t mask = a.list_mask[t];
    const int lo = a.list_link[t];
    int x, y, z;
    node_xyz(n, a.nx, a.ny, x, y, z);
    const int ex = (int)((PX >> (2 * lane)) & 3ull) - 1;
    const int ey = (int)((PY >> (2 * lane)) & 3ull) - 1;
    const int ez = (int)((PZ >> (2 * lane)) & 3ull) - 1;
    const int cls = ex * ex + ey * ey + ez * ez;
    const T w = cls == 0 ? (T)L::w(0) : (cls == 1 ? (T)L::w(1) : (T)L::w(Q - 1));
    const int ib = lane < 12 ? (int)((PO >> (5 * lane)) & 31ull) : (int)((POH >> (5 * (lane - 12))) & 31ull);
    const bool cut = dir && ((mask >> lane) & 1u);
    T fi = 0, fs = 0;
    int link = 0;
    if (cut) {
      link = lo + __popc(mask & ((1u << lane) - 1u));
      fi = ibb_value<LAT, S, T, T>(a, src, lane, x, y, z, n, link, isc, fs);
      (void)ib;
    } else if (dir) {
      const long long sn = wrap(x - ex, a.nx) +
                           (long long)a.nx * (wrap(y - ey, a.ny) + (long long)a.ny * wrap(z - ez, a.nz));
      fi = Store<S>::ld(src + (long long)lane * a.fs + sn, isc);
    }
    if (a.zy_pre) {
      // every lane has read its Eq. 16 input before any lane replaces it
      __syncwarp();
      if (dir) ((T *)a.zy_pre)[(long long)lane * a.fs + n] = fi;
    }
    const uint8_t fl = a.flags[n];
    T Fx, Fy, Fz;
    node_force<T, T>(a, n, fl, Fx, Fy, Fz);
    const T out = collide_lane<LAT, CM, T>(a, fi, dir, ex, ey, ez, cls, w, Fx, Fy, Fz);
    if (dir) Store<S>::st((S *)a.dst + (long long)lane * a.fs + n, out, isc);
    // Eq. 17 on this node's cut links (first solid: deviation part here,
    // state-independent part from the geometry build)
    const int first = mask ? __ffs(mask) - 1 : -1;
    if (first >= 0) {
      sa = a.links.sid[lo];
      T dp[3] = {0, 0, 0}, tq[3] = {0, 0, 0};
      if (cut) {
        const int s = a.links.sid[link];
        const T *uw0 = (const T *)a.links.uw[0], *uw1 = (const T *)a.links.uw[1],
                *uw2 = (const T *)a.links.uw[2];
        const T *ar0 = (const T *)a.links.arm[0], *ar1 = (const T *)a.links.arm[1],
                *ar2 = (const T *)a.links.arm[2];
        const T uw[3] = {uw0[link], uw1[link], uw2[link]};
        const T r[3] = {ar0[link], ar1[link], ar2[link]};
        const T e[3] = {(T)ex, (T)ey, (T)ez};
        T d[3];
        for (int k = 0; k < 3; k++) d[k] = -fs * (e[k] + uw[k]) - fi * (e[k] - uw[k]);
        if (s == sa) {
          for (int k = 0; k < 3; k++) dp[k] = d[k];
          tq[0] = r[1] * d[2] - r[2] * d[1];
          tq[1] = r[2] * d[0] - r[0] * d[2];
          tq[2] = r[0] * d[1] - r[1] * d[0];
        } else {
          // a second solid seen from this node: full FP64 contribution
          const double wi = (double)w;
          const double fsd = wi + (double)fs, fid = wi + (double)fi;
          double q[3];
          for (int k = 0; k < 3; k++)
            q[k] = fsd * (-(double)e[k] - (double)uw[k]) - fid * ((double)e[k] - (double)uw[k]);
          const double rr[3] = {(double)r[0], (double)r[1], (double)r[2]};
          atomicAdd(a.force_acc + 6 * s + 0, q[0]);
          atomicAdd(a.force_acc + 6 * s + 1, q[1]);
          atomicAdd(a.force_acc + 6 * s + 2, q[2]);
          atomicAdd(a.force_acc + 6 * s + 3, rr[1] * q[2] - rr[2] * q[1]);
          atomicAdd(a.force_acc + 6 * s + 4, rr[2] * q[0] - rr[0] * q[2]);
          atomicAdd(a.force_acc + 6 * s + 5, rr[0] * q[1] - rr[1] * q[0]);
        }
      }
      for (int k = 0; k < 3; k++) {
        acc[k] = a.list_cst[k * a.list_cap + t] + (double)wsum<T>(dp[k]);
        acc[3 + k] = a.list_cst[(3 + k) * a.list_cap + t] + (double)wsum<T>(tq[k]);
      }
    }
  }
  // block reduction of the per-node sums, one FP64 atomic per component
  if (lane == 0) {
    psid[warp] = sa;
    for (int k = 0; k < 6; k++) part[warp][k] = acc[k];
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int k = threadIdx.x, nw = blockDim.x >> 5;
    int s0 = -1;
    for (int wi = 0; wi < nw; wi++)
      if (psid[wi] >= 0) {
        s0 = psid[wi];
        break;
      }
    double sum = 0;
    for (int wi = 0; wi < nw; wi++) {
      if (psid[wi] < 0) continue;
      if (psid[wi] == s0)
        sum += part[wi][k];
      else
        atomicAdd(a.force_acc + 6 * psid[wi] + k, part[wi][k]);
    }
    if (s0 >= 0) atomicAdd(a.force_acc + 6 * s0 + k, sum);
  }
}

template <int LAT, int CM, typename S, typename T>
__device__ __forceinline__ void refill_node_warp(const KArgs &a, int t, int lane) {
  using L = Lat<LAT>;
  constexpr int Q = L::Q;
  constexpr unsigned long long PX = pack_dir<LAT>(0), PY = pack_dir<LAT>(1), PZ = pack_dir<LAT>(2);
  const long long n = a.refill_node[t];
  const int sidx = a.refill_sid[t];
  int x, y, z;
  node_xyz(n, a.nx, a.ny, x, y, z);
  const int ex = (int)((PX >> (2 * lane)) & 3ull) - 1;
  const int ey = (int)((PY >> (2 * lane)) & 3ull) - 1;
  const int ez = (int)((PZ >> (2 * lane)) & 3ull) - 1;
  const bool dir = lane < Q;
  const S *src = (const S *)a.src;
  const T isc = kisc<T>(a);
  double rj = 0;
  int cj = 0;
  if (dir && lane > 0) {
    const long long nb = wrap(x + ex, a.nx) +
                         (long long)a.nx * (wrap(y + ey, a.ny) + (long long)a.ny * wrap(z + ez, a.nz));
    if (a.sid[nb] == 0 && !(a.flags[nb] & FL_NEW)) {
      rj = 1.0;
      for (int k = 0; k < Q; k++) rj += (double)Store<S>::ld(src + (long long)k * a.fs + nb, isc);
      cj = 1;
    }
  }
  const double rs = wsum<double>(rj);
  int cn = cj;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cn += __shfl_xor_sync(0xffffffffu, cn, o);
  const double rho = cn ? rs / cn : 1.0;
  const SolidDev b = solid_of(a, sidx);
  double r[3] = {x - b.c[0], y - b.c[1], z - b.c[2]};
  r[0] -= a.nx * round(r[0] / a.nx);
  r[1] -= a.ny * round(r[1] / a.ny);
  r[2] = (L::D == 2 || b.kind == 1) ? 0.0 : r[2] - a.nz * round(r[2] / a.nz);
  double uw[3] = {b.U[0] + b.Om[1] * r[2] - b.Om[2] * r[1],
                  b.U[1] + b.Om[2] * r[0] - b.Om[0] * r[2],
                  b.U[2] + b.Om[0] * r[1] - b.Om[1] * r[0]};
  if (L::D == 2) uw[2] = 0;
  const int cls = ex * ex + ey * ey + ez * ez;
  const double wd = cls == 0 ? L::w(0) : (cls == 1 ? L::w(1) : L::w(Q - 1));
  const double eu = ex * uw[0] + ey * uw[1] + ez * uw[2];
  const double uu = uw[0] * uw[0] + uw[1] * uw[1] + uw[2] * uw[2];
  const T fi = dir ? (T)(wd * (rho - 1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu)) : (T)0;
  T Fx, Fy, Fz;
  node_force<T, T>(a, n, a.flags[n], Fx, Fy, Fz);
  const T out = collide_lane<LAT, CM, T>(a, fi, dir, ex, ey, ez, cls, (T)wd, Fx, Fy, Fz);
  if (dir) Store<S>::st((S *)a.dst + (long long)lane * a.fs + n, out, isc);
}

// Refill with a warp per uncovered node: lane j sums the density of
// neighbour x + e_j (if it was fluid before and after the move), then lane i
// forms f^eq_i(rho_mean, u_w) and the node's collision runs lane-parallel.
template <int LAT, int CM, typename S, typename T>
__global__ void __launch_bounds__(256) k_refill_warp(const KArgs a) {
  const int lane = threadIdx.x & 31;
  int cnt = a.counts[2];
  if (cnt > a.refill_cap) cnt = a.refill_cap;
  const int stride = gridDim.x * (blockDim.x >> 5);
  for (int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < cnt; t += stride)
    refill_node_warp<LAT, CM, S, T>(a, t, lane);
}


// Local read of a pre-collision state: collide into dst (MODE 0) or write
// fields (MODE 1).  One thread per node.
template <int LAT, int CM, typename S, typename T, typename LT, int MODE>
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
    collide<LAT, CM, T>(f, Fx, Fy, Fz, c);
    scatter<LAT, S, T>((S *)a.dst, a.fs, n, isc, f);
  } else {
    write_fields<LAT, T>(a, n, f, Fx, Fy, Fz);
  }
}

// Refill of nodes uncovered by a moving solid: equilibrium at the mean
// density of neighbours fluid before and after the move and at the local
// wall velocity, then the node's collision, written into the current
// post-collision array (src == dst).
template <int LAT, int CM, typename S, typename T>
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
  const SolidDev b = solid_of(a, sidx);
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
  collide<LAT, CM, T>(f, Fx, Fy, Fz, c);
  scatter<LAT, S, T>((S *)a.dst, a.fs, n, isc, f);
}

// IBM: unforced velocity u~ = (sum f e + g/2)/rho0 at band nodes (the
// external half force only, no IBM half force) and zero the IBM force there.
template <int LAT, typename S, typename T>
__device__ __forceinline__ T face_pull(const KArgs &a, const S *__restrict__ src, int x, int y,
                                       int z, int i, T isc);

template <int LAT, typename S, typename T>
__global__ void __launch_bounds__(64) k_band_vel(const KArgs a) {
  using L = Lat<LAT>;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  // this step's force record, accumulated by the IBM kernels that follow on
  // the same stream, starts at zero
  if (a.force_acc && t < 6 * kMaxSolids) a.force_acc[t] = 0.0;
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
  else if (fl & FL_FACE)  // next to a velocity or stress-free domain face
    for (int i = 0; i < L::Q; i++) f[i] = face_pull<LAT, S, T>(a, (const S *)a.src, x, y, z, i, isc);
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

// Eq. 16: the pre-collision populations of the boundary nodes, read from a
// state held locally (right after an initialisation).
template <int LAT, typename S, typename T>
__global__ void __launch_bounds__(128) k_zy_seed(const KArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  int cnt = a.counts[0];
  if (cnt > a.list_cap) cnt = a.list_cap;
  if (t >= cnt) return;
  const long long n = a.list_node[t];
  const T isc = kisc<T>(a);
  for (int i = 0; i < Lat<LAT>::Q; i++)
    ((T *)a.zy_pre)[(long long)i * a.fs + n] =
        Store<S>::ld((const S *)a.src + (long long)i * a.fs + n, isc);
}

// ---------------------------------------------------------------- domain
// faces (the open box of the uniform flow past a sphere, Sec. 3.4).  A
// non-periodic face lies half a spacing outside the outermost nodes; the
// nodes next to one (flag FL_FACE) run in k_face, a thread per node, which
// pulls like the bulk sweep except on links that leave the domain:
//  - velocity face (plane wall moving with u_f): f_i = f*_ib(x) + 6 w_i e_i.u_f
//    (the moving-wall bounce-back with q = 1/2, rho0 = 1);
//  - stress-free face: specular reflection, f_i = f*_r(x'), r = e_i with the
//    crossed components reversed and x' = x - e_i with x's coordinates on the
//    crossed axes;
//  - convective outflow face (outward normal n): f_i(x, t+1) =
//    [f_i(x, t) + U_o f_i(x - n, t+1)] / (1 + U_o), U_o = max(0, u(x, t).n),
//    from the node's pre-collision populations and velocity kept from the
//    previous step (a.outlet, [Q + 1][face area] in the compute type).
// A velocity face decides a link that crosses two faces, then an outflow
// face, then free slip.

// bit 2a: the low face of axis a is crossed, bit 2a + 1: the high face
template <int LAT>
__device__ __forceinline__ int face_cross(const KArgs &a, int x, int y, int z, int i) {
  using L = Lat<LAT>;
  const int sx = x - L::ex(i), sy = y - L::ey(i), sz = z - L::ez(i);
  int m = 0;
  if (sx < 0 && a.face[0]) m |= 1;
  if (sx >= a.nx && a.face[1]) m |= 2;
  if (sy < 0 && a.face[2]) m |= 4;
  if (sy >= a.ny && a.face[3]) m |= 8;
  if (L::D == 3) {
    if (sz < 0 && a.face[4]) m |= 16;
    if (sz >= a.nz && a.face[5]) m |= 32;
  }
  return m;
}

__device__ __forceinline__ int face_of_type(const KArgs &a, int m, int type) {
  for (int k = 0; k < 6; k++)
    if (((m >> k) & 1) && a.face[k] == type) return k;
  return -1;
}

template <typename T> __device__ __forceinline__ T face_u(const KArgs &a, int k, int c) {
  if constexpr (is_f32<T>()) return a.u_face_f[k][c];
  else return (T)a.u_face[k][c];
}

// f_i(x, t+1) of a link that leaves through velocity / stress-free faces
template <int LAT, typename S, typename T>
__device__ __forceinline__ T face_wall(const KArgs &a, const S *__restrict__ src, int x, int y,
                                       int z, int i, int m, T isc) {
  using L = Lat<LAT>;
  const long long fs = a.fs;
  const int vf = face_of_type(a, m, LBM_FACE_VELOCITY);
  if (vf >= 0) {
    const long long n = x + (long long)a.nx * (y + (long long)a.ny * z);
    const T eu = (T)L::ex(i) * face_u<T>(a, vf, 0) + (T)L::ey(i) * face_u<T>(a, vf, 1) +
                 (T)L::ez(i) * face_u<T>(a, vf, 2);
    return Store<S>::ld(src + (long long)L::opp(i) * fs + n, isc) + (T)(6.0 * L::w(i)) * eu;
  }
  int r[3] = {L::ex(i), L::ey(i), L::ez(i)};
  int p[3] = {x - r[0], y - r[1], z - r[2]};
  const int at[3] = {x, y, z};
#pragma unroll
  for (int c = 0; c < 3; c++)
    if ((m >> (2 * c)) & 3) {
      r[c] = -r[c];
      p[c] = at[c];
    }
  int j = 0;
#pragma unroll
  for (int k = 1; k < L::Q; k++)
    if (L::ex(k) == r[0] && L::ey(k) == r[1] && L::ez(k) == r[2]) j = k;
  const long long ns = wrap(p[0], a.nx) +
                       (long long)a.nx * (wrap(p[1], a.ny) + (long long)a.ny * wrap(p[2], a.nz));
  return Store<S>::ld(src + (long long)j * fs + ns, isc);
}

// f_i(x, t+1) of a node: plain pull, or through velocity / stress-free faces
template <int LAT, typename S, typename T>
__device__ __forceinline__ T face_pull(const KArgs &a, const S *__restrict__ src, int x, int y,
                                       int z, int i, T isc) {
  using L = Lat<LAT>;
  const int m = face_cross<LAT>(a, x, y, z, i);
  if (m) return face_wall<LAT, S, T>(a, src, x, y, z, i, m, isc);
  const long long ns = wrap(x - L::ex(i), a.nx) +
                       (long long)a.nx * (wrap(y - L::ey(i), a.ny) +
                                          (long long)a.ny * wrap(z - L::ez(i), a.nz));
  return Store<S>::ld(src + (long long)i * a.fs + ns, isc);
}

// index of a node of the outflow face in the outlet arrays
__device__ __forceinline__ int outlet_index(const KArgs &a, int x, int y, int z) {
  const int ax = a.out_face >> 1;
  return ax == 0 ? y + a.ny * z : ax == 1 ? x + a.nx * z : x + a.nx * y;
}
__device__ __forceinline__ bool on_outlet(const KArgs &a, int x, int y, int z) {
  if (a.out_face < 0) return false;
  const int ax = a.out_face >> 1, hi = a.out_face & 1;
  const int c = ax == 0 ? x : ax == 1 ? y : z;
  const int len = ax == 0 ? a.nx : ax == 1 ? a.ny : a.nz;
  return c == (hi ? len - 1 : 0);
}

// MODE 0: sweep (src f*(t) -> dst f*(t+1)); MODE 1: query of f(t) from
// src = f*(t - 1); MODE 2: keep the outflow face's populations and velocity
// from a state held locally in src (right after an initialisation).
template <int LAT, int CM, typename S, typename T, typename LT, int MODE>
__global__ void __launch_bounds__(128) k_face(const KArgs a) {
  using L = Lat<LAT>;
  constexpr int Q = L::Q;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.nface) return;
  const long long n = a.face_node[t];
  int x, y, z;
  node_xyz(n, a.nx, a.ny, x, y, z);
  const T isc = kisc<T>(a);
  const S *__restrict__ src = (const S *)a.src;
  const bool out = on_outlet(a, x, y, z);
  const long long A = a.out_area;
  LT *keep = (LT *)a.outlet;
  const int oi = out ? outlet_index(a, x, y, z) : 0;
  const uint8_t fl = a.flags[n];
  T Fx, Fy, Fz;
  node_force<T, LT>(a, n, fl, Fx, Fy, Fz);
  T f[Q];
  if (MODE == 2) {
    if (!out) return;
    gather_local<LAT, S, T>(src, a.fs, n, isc, f);
  } else {
    const int ax = a.out_face >> 1, sg = (a.out_face & 1) ? 1 : -1;
#pragma unroll
    for (int i = 0; i < Q; i++) {
      const int m = face_cross<LAT>(a, x, y, z, i);
      if (m == 0) {
        const long long ns = wrap(x - L::ex(i), a.nx) +
                             (long long)a.nx * (wrap(y - L::ey(i), a.ny) +
                                                (long long)a.ny * wrap(z - L::ez(i), a.nz));
        f[i] = Store<S>::ld(src + (long long)i * a.fs + ns, isc);
      } else if (face_of_type(a, m, LBM_FACE_VELOCITY) < 0 &&
                 face_of_type(a, m, LBM_FACE_CONVECTIVE) >= 0) {
        if (MODE == 1) {
          f[i] = (T)keep[(long long)i * A + oi];  // f_i(x, t), kept by the last step
        } else {
          const int xi = x - (ax == 0 ? sg : 0), yi = y - (ax == 1 ? sg : 0),
                    zi = z - (ax == 2 ? sg : 0);
          const T vin = face_pull<LAT, S, T>(a, src, xi, yi, zi, i, isc);
          T U = (T)keep[(long long)Q * A + oi];
          if (U < (T)0) U = (T)0;
          f[i] = ((T)keep[(long long)i * A + oi] + U * vin) / ((T)1 + U);
        }
      } else {
        f[i] = face_wall<LAT, S, T>(a, src, x, y, z, i, m, isc);
      }
    }
  }
  if (MODE != 1 && out) {
    // this step's pre-collision populations and outward velocity, read by
    // the next step's outflow update
    T j = (T)0;
#pragma unroll
    for (int i = 0; i < Q; i++) keep[(long long)i * A + oi] = (LT)f[i];
    const int ax = a.out_face >> 1;
#pragma unroll
    for (int i = 0; i < Q; i++)
      j += (T)(ax == 0 ? L::ex(i) : ax == 1 ? L::ey(i) : L::ez(i)) * f[i];
    const T Fa = ax == 0 ? Fx : ax == 1 ? Fy : Fz;
    keep[(long long)Q * A + oi] = (LT)(((a.out_face & 1) ? (T)1 : (T)-1) * (j + (T)0.5 * Fa));
  }
  if (MODE == 0) {
    const Coll<T> c = make_coll<LAT, T>(a);
    collide<LAT, CM, T>(f, Fx, Fy, Fz, c);
    scatter<LAT, S, T>((S *)a.dst, a.fs, n, isc, f);
  } else if (MODE == 1) {
    write_fields<LAT, T>(a, n, f, Fx, Fy, Fz);
  }
}

// ---------------------------------------------------------------- Eq. 24
// The fluid momentum and angular momentum inside solid a.kempe_solid at the
// time of the state in src (post-collision f*, so u = sum e f* - F/2 with
// the force of that collision), weighted by the fraction alpha of the cell
// around each node inside the solid (Eq. 25: sum over the cell's corners at
// +-1/2 of -phi H(-phi) over the sum of |phi|, phi the signed distance
// function of Eq. 26 for a sphere, or a circle / z-cylinder).  A thread per
// node of the box around the solid; FP64 sums.
__device__ __forceinline__ double kimage(double d, int L) {
  return d - L * rint(d * (1.0 / L));
}

template <int LAT, typename S, typename T>
__global__ void __launch_bounds__(256) k_kempe(const KArgs a) {
  using L = Lat<LAT>;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int bx = a.kbox[3], by = a.kbox[4], bz = a.kbox[5];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  if (t < (long long)bx * by * bz) {
    const SolidDev b = solid_of(a, a.kempe_solid);
    int o[3] = {a.kbox[0], a.kbox[1], a.kbox[2]};
    if (a.kbox_dev) {
      // every node with a cell corner inside lies within R + 1 of the centre
      const int len[3] = {a.nx, a.ny, a.nz};
      for (int c = 0; c < 3; c++)
        if (a.kbox[3 + c] < len[c]) o[c] = (int)floor(b.c[c] - b.R - 1.0);
    }
    const int x = wrap(o[0] + (int)(t % bx), a.nx);
    const int y = wrap(o[1] + (int)((t / bx) % by), a.ny);
    const int z = wrap(o[2] + (int)(t / ((long long)bx * by)), a.nz);
    const bool flat = L::D == 2 || b.kind == LBM_CYLINDER_Z;
    double num = 0, den = 0;
    for (int c = 0; c < (L::D == 2 ? 4 : 8); c++) {
      const double r0 = kimage(x + ((c & 1) ? 0.5 : -0.5) - b.c[0], a.nx);
      const double r1 = kimage(y + ((c & 2) ? 0.5 : -0.5) - b.c[1], a.ny);
      const double r2 = flat ? 0.0 : kimage(z + ((c & 4) ? 0.5 : -0.5) - b.c[2], a.nz);
      const double phi = sqrt(r0 * r0 + r1 * r1 + r2 * r2) / b.R - 1.0;
      if (phi < 0) num -= phi;
      den += fabs(phi);
    }
    const double al = den > 0 ? num / den : 0.0;
    if (al > 0) {
      const long long n = x + (long long)a.nx * (y + (long long)a.ny * z);
      const T isc = kisc<T>(a);
      T Fx, Fy, Fz;
      node_force<T, T>(a, n, a.flags[n], Fx, Fy, Fz);
      T j[3] = {(T)0, (T)0, (T)0};
#pragma unroll
      for (int i = 1; i < L::Q; i++) {
        const T v = Store<S>::ld((const S *)a.src + (long long)i * a.fs + n, isc);
        j[0] += (T)L::ex(i) * v;
        j[1] += (T)L::ey(i) * v;
        j[2] += (T)L::ez(i) * v;
      }
      const double u[3] = {(double)(j[0] - (T)0.5 * Fx), (double)(j[1] - (T)0.5 * Fy),
                           L::D == 2 ? 0.0 : (double)(j[2] - (T)0.5 * Fz)};
      const double r[3] = {kimage(x - b.c[0], a.nx), kimage(y - b.c[1], a.ny),
                           flat ? 0.0 : kimage(z - b.c[2], a.nz)};
      acc[0] = al * u[0];
      acc[1] = al * u[1];
      acc[2] = al * u[2];
      acc[3] = al * (r[1] * u[2] - r[2] * u[1]);
      acc[4] = al * (r[2] * u[0] - r[0] * u[2]);
      acc[5] = al * (r[0] * u[1] - r[1] * u[0]);
    }
  }
  const int lane = threadIdx.x & 31;
  for (int c = 0; c < 6; c++) {
    const double v = warp_sum(acc[c]);
    if (lane == 0 && v != 0.0) atomicAdd(a.kempe_out + c, v);
  }
}

// ---------------------------------------------------------------- launch
inline int div_up(long long a, int b) { return (int)((a + b - 1) / b); }

// The vector bulk sweep: W words per thread and direction (bulk_vec_words 2
// or 4; 0 = 2) and the node-pair collision packed (bulk_vec_packed 1) or
// node by node (0); -1 picks what measured fastest on the 128^3 sphere
// lattice: 8-byte vectors, node by node for FP32 storage, packed for 16-bit
// storage.  Returns false where nx or the direction stride is not a
// multiple of the V nodes of a vector.
template <int LAT, int CM, typename S, int W>
bool launch_bulk_vec_w(const KArgs &a, int want, bool packed, cudaStream_t st) {
  constexpr int V = W * VecS<S>::per_word;
  if (a.nx % V != 0 || a.fs % V != 0) return false;
  const int nt = (int)(a.N / V);
  const int grid = div_up(nt, want);
  if (packed) k_bulk_vec<LAT, CM, S, W, true><<<grid, want, 0, st>>>(a);
  else k_bulk_vec<LAT, CM, S, W, false><<<grid, want, 0, st>>>(a);
  return true;
}
template <int LAT, int CM, typename S>
bool launch_bulk_vec(const KArgs &a, int want, cudaStream_t st) {
  const bool packed = a.bulk_vec_packed >= 0 ? a.bulk_vec_packed != 0 : sizeof(S) == 2;
  if (a.bulk_vec_words == 4) return launch_bulk_vec_w<LAT, CM, S, 4>(a, want, packed, st);
  return launch_bulk_vec_w<LAT, CM, S, 2>(a, want, packed, st);
}

// The row-copy sweep (bulk_mode 2), built for the default vector shape of
// the storage type only (2 words; node by node for FP32, packed pairs for
// 16-bit storage).  The grid is the resident blocks of all SMs (queried per
// device and shared-memory size), or fewer where the lattice has fewer
// tiles.  Returns false where the lattice, its alignment or the requested
// shape does not fit it.
template <int LAT, int CM, typename S>
bool launch_bulk_rows(const KArgs &a, cudaStream_t st) {
  constexpr int W = 2;
  constexpr int V = W * VecS<S>::per_word;
  constexpr bool kPacked = sizeof(S) == 2;
  const bool packed = a.bulk_vec_packed >= 0 ? a.bulk_vec_packed != 0 : kPacked;
  if (a.bulk_vec_words == 4 || packed != kPacked || !a.wait_err) return false;
  if (a.nx % (32 * V) != 0 || a.N / a.nx >= (1LL << 31) || (a.fs * (long long)sizeof(S)) % 16 != 0 ||
      ((uintptr_t)a.src & 15) != 0 || ((uintptr_t)a.flags & 15) != 0)
    return false;
  // two blocks per SM
  constexpr size_t kSmemLimit = 112 * 1024;
  const RowTiles g = row_tiles<LAT, S, W>(a, kSmemLimit);
  if (g.stage_bytes == 0) return false;
  const size_t smem = 2 * (size_t)g.stage_bytes + 4 * sizeof(uint64_t);
  auto kern = k_bulk_rows<LAT, CM, S, W, kPacked>;
  constexpr int kMaxDev = 64;
  struct Resident {
    size_t smem;
    int blocks;  // 0: not queried, -1: unusable
  };
  static Resident resident[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return false;
  Resident &r = resident[dev];
  if (r.blocks == 0 || r.smem != smem) {
    // the attribute calls are not stream work: allowed inside a capture
    cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
    cudaThreadExchangeStreamCaptureMode(&mode);
    int per_sm = 0, sms = 0;
    const bool ok =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit + 64) ==
            cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRowBlock, smem) ==
            cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess;
    cudaThreadExchangeStreamCaptureMode(&mode);
    r.smem = smem;
    r.blocks = ok && per_sm > 0 ? per_sm * sms : -1;
  }
  if (r.blocks < 0) return false;
  const unsigned grid = (unsigned)std::min<long long>(r.blocks, g.ntiles);
  if (grid == 0) return true;
  kern<<<grid, kRowBlock, smem, st>>>(a, g);
  return true;
}

template <int LAT, int CM, typename S, int W, bool PACKED>
bool launch_group_w(const KArgs *as, int n, int want, cudaStream_t st) {
  constexpr int V = W * VecS<S>::per_word;
  static_assert(sizeof(GroupArgs) <= 32000, "kernel parameter space");
  GroupArgs g;
  g.n = n;
  int blocks = 0;
  for (int k = 0; k < n; k++) {
    if (as[k].nx % V != 0 || as[k].fs % V != 0) return false;
    g.block_start[k] = blocks;
    blocks += div_up(as[k].N / V, want);
    g.a[k] = as[k];
  }
  g.block_start[n] = blocks;
  k_bulk_vec_group<LAT, CM, S, W, PACKED><<<blocks, want, 0, st>>>(g);
  return true;
}

template <int LAT, int CM, typename S>
bool launch_group_t(const KArgs *as, int n, cudaStream_t st) {
  if constexpr (CM == CM_MRT) {
    return false;
  } else {
    const KArgs &a0 = as[0];
    for (int k = 1; k < n; k++)
      if (as[k].bulk_mode != a0.bulk_mode || as[k].bulk_vec_words != a0.bulk_vec_words ||
          as[k].bulk_vec_packed != a0.bulk_vec_packed || as[k].bulk_block != a0.bulk_block)
        return false;
    if (a0.bulk_mode < 1 || n < 1 || n > kMaxGroup) return false;
    // only the default vector shape of the storage type is built grouped (2
    // words; node by node for FP32, packed pairs for 16-bit storage): each
    // grouped variant inlines the update kMaxGroup times
    constexpr bool kPacked = sizeof(S) == 2;
    const bool packed = a0.bulk_vec_packed >= 0 ? a0.bulk_vec_packed != 0 : kPacked;
    if (a0.bulk_vec_words == 4 || packed != kPacked) return false;
    const int want = a0.bulk_block > 0 ? a0.bulk_block : 128;
    return launch_group_w<LAT, CM, S, 2, kPacked>(as, n, want, st);
  }
}

template <typename S>
bool launch_group_precision(const KArgs *as, int n, int lattice, int collision, cudaStream_t st) {
  if (lattice == LBM_D2Q9) {
    if (collision == CM_MRT_Q) return launch_group_t<0, CM_MRT_Q, S>(as, n, st);
    if (collision == CM_BGK) return launch_group_t<0, CM_BGK, S>(as, n, st);
  } else {
    if (collision == CM_MRT_Q) return launch_group_t<1, CM_MRT_Q, S>(as, n, st);
    if (collision == CM_BGK) return launch_group_t<1, CM_BGK, S>(as, n, st);
  }
  return false;
}

template <int LAT, int CM, typename S, typename T>
void launch_one(SweepOp op, const KArgs &a, cudaStream_t st) {
  const int want = a.bulk_block > 0 ? a.bulk_block : 128;
  const int bx = a.nx >= want ? want : ((a.nx + 31) / 32) * 32;
  const dim3 gbulk(div_up(a.nx, bx), a.ny, a.nz);
  const int lc = a.list_cap > 0 ? a.list_cap : 1;
  switch (op) {
  case OP_BULK_SWEEP:
    if constexpr (std::is_same<T, float>::value && CM != CM_MRT) {
      g_bulk_kernel = BK_ROWS;
      if (a.bulk_mode == 2 && launch_bulk_rows<LAT, CM, S>(a, st)) break;
      g_bulk_kernel = BK_VEC;
      if (a.bulk_mode >= 1 && launch_bulk_vec<LAT, CM, S>(a, want, st)) break;
    }
    g_bulk_kernel = BK_NODE;
    switch (a.cache_hints & 3) {
    case 1: k_bulk_sweep<LAT, CM, S, T, 1><<<div_up(a.N, want), want, 0, st>>>(a); break;
    case 2: k_bulk_sweep<LAT, CM, S, T, 2><<<div_up(a.N, want), want, 0, st>>>(a); break;
    case 3: k_bulk_sweep<LAT, CM, S, T, 3><<<div_up(a.N, want), want, 0, st>>>(a); break;
    default: k_bulk_sweep<LAT, CM, S, T, 0><<<div_up(a.N, want), want, 0, st>>>(a);
    }
    break;
  case OP_BULK_QUERY:
    if constexpr (std::is_same<T, float>::value) {
      if (!a.out_S && !a.out_stress && !a.out_eps && !a.out_f) {
        k_bulk_query_u<LAT, S><<<gbulk, bx, 0, st>>>(a);
        break;
      }
    }
    k_bulk_query<LAT, S><<<gbulk, bx, 0, st>>>(a);
    break;
  case OP_LIST_SWEEP:
    if (a.list_cap > 0) {
      if (CM != CM_MRT && !a.list_thread) {
        // a warp per boundary node, list_block / 32 nodes per block
        const int lb = a.list_block >= 64 ? (a.list_block > 256 ? 256 : a.list_block) : 256;
        if constexpr (CM != CM_MRT) k_list_warp<LAT, CM, S, T><<<div_up(lc, lb / 32), lb, 0, st>>>(a);
      } else {
        // general MRT rates, or IBM band nodes (no cut links): a thread per
        // node (small blocks spread the boundary nodes over many SMs)
        const int lb = a.list_block > 0 && a.list_block <= 128 ? a.list_block : 64;
        k_list<LAT, CM, S, T, T, 0><<<div_up(lc, lb), lb, 0, st>>>(a);
      }
    }
    break;
  case OP_ZY_SEED:
    if (a.list_cap > 0 && a.zy_pre) k_zy_seed<LAT, S, T><<<div_up(lc, 128), 128, 0, st>>>(a);
    break;
  case OP_LIST_QUERY:
    if (a.list_cap > 0) k_list<LAT, CM, S, double, T, 1><<<div_up(lc, 64), 64, 0, st>>>(a);
    break;
  case OP_LOCAL_INIT:
    k_local<LAT, CM, S, T, T, 0><<<div_up(a.N, 256), 256, 0, st>>>(a);
    break;
  case OP_LOCAL_QUERY:
    k_local<LAT, CM, S, double, T, 1><<<div_up(a.N, 256), 256, 0, st>>>(a);
    break;
  case OP_REFILL:
    if (a.refill_cap > 0) {
      if constexpr (CM != CM_MRT)
        k_refill_warp<LAT, CM, S, T><<<std::min(div_up(a.refill_cap, 8), 64), 256, 0, st>>>(a);
      else
        k_refill<LAT, CM, S, T><<<div_up(a.refill_cap, 128), 128, 0, st>>>(a);
    }
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
  case OP_FACE_SWEEP:
    if (a.nface > 0) k_face<LAT, CM, S, T, T, 0><<<div_up(a.nface, 128), 128, 0, st>>>(a);
    break;
  case OP_FACE_QUERY:
    if (a.nface > 0) k_face<LAT, CM, S, double, T, 1><<<div_up(a.nface, 128), 128, 0, st>>>(a);
    break;
  case OP_KEMPE: {
    const long long vol = (long long)a.kbox[3] * a.kbox[4] * a.kbox[5];
    if (vol > 0) k_kempe<LAT, S, T><<<div_up(vol, 256), 256, 0, st>>>(a);
    break;
  }
  case OP_FACE_SEED:
    if (a.nface > 0 && a.outlet) k_face<LAT, CM, S, T, T, 2><<<div_up(a.nface, 128), 128, 0, st>>>(a);
    break;
  }
}

// collision: CM_BGK, CM_MRT (general rates) or CM_MRT_Q (only the q moments
// relax at a rate other than 1/tau, the default)
template <typename S, typename T>
void launch_precision(SweepOp op, int lattice, int collision, const KArgs &a,
                      cudaStream_t st) {
  if (lattice == LBM_D2Q9) {
    if (collision == CM_MRT) launch_one<0, CM_MRT, S, T>(op, a, st);
    else if (collision == CM_MRT_Q) launch_one<0, CM_MRT_Q, S, T>(op, a, st);
    else launch_one<0, CM_BGK, S, T>(op, a, st);
  } else {
    if (collision == CM_MRT) launch_one<1, CM_MRT, S, T>(op, a, st);
    else if (collision == CM_MRT_Q) launch_one<1, CM_MRT_Q, S, T>(op, a, st);
    else launch_one<1, CM_BGK, S, T>(op, a, st);
  }
}

}  // namespace lbm
