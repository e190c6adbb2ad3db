// lbm_device.cuh -- device building blocks of the fused collide-stream sweep
// (Peng, Ayala & Wang, arXiv 1906.05445, Eqs. 1-3 with Guo forcing).
//
// Storage holds deviations d_i = f_i - w_i (optionally scaled for FP16), SoA
// [Q][z][y][x].  The compute type T is double for the FP64 build and float
// otherwise.  Everything that depends on the lattice is a compile-time
// constant so that the unrolled loops fold to straight-line arithmetic.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace lbm {

// Compile-time loop: f(std::integral_constant<int, I>) for I = 0..N-1, so
// that lattice tables indexed by I are constant expressions, not run-time
// lookups, whatever the unroller decides.
template <typename F, int... I>
__host__ __device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__host__ __device__ __forceinline__ void static_for(F &&f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// ---------------------------------------------------------------- lattices
// direction order: see include/lbm.h
template <int LAT> struct Lat;

template <> struct Lat<0> {  // D2Q9
  static constexpr int Q = 9, D = 2;
  __host__ __device__ static constexpr int ex(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
  }
  __host__ __device__ static constexpr int ey(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
  }
  __host__ __device__ static constexpr int ez(int) { return 0; }
  __host__ __device__ static constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4 + 1) : ((i - 5 + 2) % 4 + 5));
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
};

template <> struct Lat<1> {  // D3Q19
  static constexpr int Q = 19, D = 3;
  __host__ __device__ static constexpr int ex(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
           : ((i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0);
  }
  __host__ __device__ static constexpr int ey(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
           : ((i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0);
  }
  __host__ __device__ static constexpr int ez(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
           : ((i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0);
  }
  __host__ __device__ static constexpr int opp(int i) {
    return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
};

// Gram-Schmidt moment rows (Lallemand-Luo for D2Q9, d'Humieres et al. for
// D3Q19) as polynomials of e; row order matches lbm_lattice_desc.mrt_rates.
template <int LAT>
__host__ __device__ constexpr int mrow(int k, int i) {
  using L = Lat<LAT>;
  const int x = L::ex(i), y = L::ey(i), z = L::ez(i);
  const int e2 = x * x + y * y + z * z;
  if (LAT == 0) {
    return k == 0 ? 1
         : k == 1 ? -4 + 3 * e2
         : k == 2 ? (8 - 21 * e2 + 9 * e2 * e2) / 2
         : k == 3 ? x
         : k == 4 ? (-5 + 3 * e2) * x
         : k == 5 ? y
         : k == 6 ? (-5 + 3 * e2) * y
         : k == 7 ? x * x - y * y
                  : x * y;
  }
  return k == 0 ? 1
       : k == 1 ? 19 * e2 - 30
       : k == 2 ? (21 * e2 * e2 - 53 * e2 + 24) / 2
       : k == 3 ? x
       : k == 4 ? (5 * e2 - 9) * x
       : k == 5 ? y
       : k == 6 ? (5 * e2 - 9) * y
       : k == 7 ? z
       : k == 8 ? (5 * e2 - 9) * z
       : k == 9 ? 3 * x * x - e2
       : k == 10 ? (3 * e2 - 5) * (3 * x * x - e2)
       : k == 11 ? y * y - z * z
       : k == 12 ? (3 * e2 - 5) * (y * y - z * z)
       : k == 13 ? x * y
       : k == 14 ? y * z
       : k == 15 ? x * z
       : k == 16 ? (y * y - z * z) * x
       : k == 17 ? (z * z - x * x) * y
                 : (x * x - y * y) * z;
}

template <int LAT>
__host__ __device__ constexpr int mnorm(int k) {
  int s = 0;
  for (int i = 0; i < Lat<LAT>::Q; i++) s += mrow<LAT>(k, i) * mrow<LAT>(k, i);
  return s;
}

// moments whose rate is irrelevant (density and momentum)
template <int LAT>
__host__ __device__ constexpr bool conserved(int k) {
  return k == 0 || k == 3 || k == 5 || (LAT == 1 && k == 7);
}

// ---------------------------------------------------------------- storage
template <typename S> struct Store;
// ld/st: default caching; ld_stream/st_stream: evict-first (each element is
// read once and written once per sweep)
template <> struct Store<double> {
  template <typename T> __device__ static T ld(const double *p, T) { return (T)__ldg(p); }
  template <typename T> __device__ static T ld_stream(const double *p, T) { return (T)__ldcs(p); }
  template <typename T> __device__ static void st(double *p, T v, T) { *p = (double)v; }
  template <typename T> __device__ static void st_stream(double *p, T v, T) { __stcs(p, (double)v); }
};
template <> struct Store<float> {
  template <typename T> __device__ static T ld(const float *p, T) { return (T)__ldg(p); }
  template <typename T> __device__ static T ld_stream(const float *p, T) { return (T)__ldcs(p); }
  template <typename T> __device__ static void st(float *p, T v, T) { *p = (float)v; }
  template <typename T> __device__ static void st_stream(float *p, T v, T) { __stcs(p, (float)v); }
};
template <> struct Store<__nv_bfloat16> {
  template <typename T> __device__ static T ld(const __nv_bfloat16 *p, T) {
    return (T)__bfloat162float(__ldg(p));
  }
  template <typename T> __device__ static void st(__nv_bfloat16 *p, T v, T) {
    *p = __float2bfloat16_rn((float)v);
  }
  template <typename T> __device__ static T ld_stream(const __nv_bfloat16 *p, T s) { return ld(p, s); }
  template <typename T> __device__ static void st_stream(__nv_bfloat16 *p, T v, T s) { st(p, v, s); }
};
// FP16 keeps d_i * scale (scale = 2^k) so that deviations stay in the normal
// range; the scale is exact in binary, so it only shifts the exponent.
template <> struct Store<__half> {
  template <typename T> __device__ static T ld(const __half *p, T inv_scale) {
    return (T)__half2float(__ldg(p)) * inv_scale;
  }
  template <typename T> __device__ static void st(__half *p, T v, T inv_scale) {
    *p = __float2half_rn((float)(v / inv_scale));
  }
  template <typename T> __device__ static T ld_stream(const __half *p, T s) { return ld(p, s); }
  template <typename T> __device__ static void st_stream(__half *p, T v, T s) { st(p, v, s); }
};

// ---------------------------------------------------------------- collision
template <typename T> struct Coll {
  T omega;      // 1/tau: rate of the stress moments (and of BGK)
  T omc;        // 1 - omega
  T cforce;     // 1 - omega/2
  T ds[19];     // omega - s_k per moment (0: same as BGK)
};

// Incompressible equilibrium deviation w_i[drho + 3 e.u + 4.5 (e.u)^2 - 1.5 u^2]
template <int LAT, typename T>
__device__ __forceinline__ T feq_dev(int i, T drho, T ux, T uy, T uz, T uu) {
  using L = Lat<LAT>;
  const T eu = (T)L::ex(i) * ux + (T)L::ey(i) * uy + (T)L::ez(i) * uz;
  return (T)L::w(i) * (drho + (T)3 * eu + (T)4.5 * eu * eu - (T)1.5 * uu);
}

// e_i . v with the lattice velocity folded at compile time
template <int LAT, int I, typename T>
__device__ __forceinline__ T edot(T vx, T vy, T vz) {
  using L = Lat<LAT>;
  T r = (T)0;
  if constexpr (L::ex(I) == 1) r += vx;
  if constexpr (L::ex(I) == -1) r -= vx;
  if constexpr (L::ey(I) == 1) r += vy;
  if constexpr (L::ey(I) == -1) r -= vy;
  if constexpr (L::ez(I) == 1) r += vz;
  if constexpr (L::ez(I) == -1) r -= vz;
  return r;
}

// Collide deviations in place: Eq. 1 (BGK) or Eq. 3 (MRT) with Guo forcing,
//   BGK: f* = (1 - omega) f + omega feq + (1 - omega/2) Fbar,
//   Fbar_i = w_i[3 (e_i - u).F + 9 (e_i.u)(e_i.F)].
// Directions come in opposite pairs (e_ib = -e_i), so feq and Fbar split
// into a part even in e (shared by the pair) and an odd part (sign flip):
//   feq  = w[drho - 1.5 u^2 + 4.5 (e.u)^2] +- 3 w (e.u),
//   Fbar = w[9 (e.u)(e.F) - 3 u.F]         +- 3 w (e.F).
// MRT adds, for every moment whose rate s_k differs from omega, the
// correction (omega - s_k) (M_k.(Delta + Fbar/2)) M_ki / |M_k|^2, which
// equals m* = m - S(m - meq) + (I - S/2) M Fbar, f* = M^-1 m* because the
// rows of M are orthogonal.
// collision modes of the kernels
enum : int { CM_BGK = 0, CM_MRT = 1, CM_MRT_Q = 2 };

// q-moment rows (energy flux, odd in e): (5|e|^2 - 9) e_a on D3Q19,
// (3|e|^2 - 5) e_a on D2Q9 (rows 4, 6, 8 / 4, 6 of the basis)
template <int LAT> __host__ __device__ constexpr int qrow(int a, int i) {
  return mrow<LAT>(4 + 2 * a, i);
}

// Sum over the pair leaders i of q_a,i 3 w_i e_i,b: the q moments of the
// pairs' terms -2 A_i + AF_i (A_i = 3 w_i e_i.u, AF_i = 3 w_i e_i.F) are
// sum_b K_ab (F_b - 2 u_b).
template <int LAT> __host__ __device__ constexpr double qk(int a, int b) {
  using L = Lat<LAT>;
  double s = 0;
  for (int i = 1; i < L::Q; i++)
    if (L::opp(i) > i) {
      const int e = b == 0 ? L::ex(i) : (b == 1 ? L::ey(i) : L::ez(i));
      s += qrow<LAT>(a, i) * 3.0 * L::w(i) * e;
    }
  return s;
}

template <int LAT, int CM, typename T>
__device__ __forceinline__ void collide(T (&f)[Lat<LAT>::Q], T Fx, T Fy, T Fz,
                                        const Coll<T> &c) {
  using L = Lat<LAT>;
  constexpr int Q = L::Q;
  constexpr bool MRT = CM == CM_MRT;
  T drho = 0, jx = 0, jy = 0, jz = 0;
  static_for<Q>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    drho += f[i];
    if constexpr (L::ex(i) == 1) jx += f[i];
    if constexpr (L::ex(i) == -1) jx -= f[i];
    if constexpr (L::ey(i) == 1) jy += f[i];
    if constexpr (L::ey(i) == -1) jy -= f[i];
    if constexpr (L::ez(i) == 1) jz += f[i];
    if constexpr (L::ez(i) == -1) jz -= f[i];
  });
  const T ux = jx + (T)0.5 * Fx, uy = jy + (T)0.5 * Fy, uz = jz + (T)0.5 * Fz;
  const T uu = ux * ux + uy * uy + uz * uz;
  const T uF = ux * Fx + uy * Fy + uz * Fz;
  const T base = drho - (T)1.5 * uu;
  const T om = c.omega, omc = c.omc, cf = c.cforce;
  if constexpr (CM != CM_MRT) {
    // BGK, or MRT whose only non-BGK moments are the q moments: update in
    // place pair by pair, grouped for few operations (as the packed pair
    // collision): omega S + cforce SF = w B + A g with B = omega base -
    // 3 cforce u.F and g = 1.5 omega e.u + 3 cforce e.F; omega A + cforce AF
    // = omega A + w (3 cforce e.F); the q moments of Delta + Fbar/2 are
    // sum_i q_a,i (f_i - f_ib) + K (F - 2u) (qk: the pairs' -2A + AF terms)
    T mq[3] = {0, 0, 0};
    const T om15 = om * (T)1.5, cf3 = cf * (T)3;
    const T B = om * base - cf3 * uF;
    f[0] = omc * f[0] + (T)L::w(0) * B;
    const T Ba = (T)L::w(1) * B, Bb = (T)L::w(Q - 1) * B;
    static_for<Q>([&](auto ic) {
      constexpr int i = decltype(ic)::value;
      if constexpr (i > 0 && L::opp(i) > i) {
        constexpr int j = L::opp(i);
        constexpr T w = (T)L::w(i);
        constexpr bool ca = L::w(i) == L::w(1);
        const T eu = edot<LAT, i, T>(ux, uy, uz);
        const T eF = edot<LAT, i, T>(Fx, Fy, Fz);
        const T A = (T)(3.0 * L::w(i)) * eu;
        const T t = cf3 * eF;
        const T P = A * (om15 * eu + t) + (ca ? Ba : Bb);
        const T M = om * A + w * t;
        if constexpr (CM == CM_MRT_Q) {
          const T d = f[i] - f[j];
          static_for<L::D>([&](auto ac) {
            constexpr int ax = decltype(ac)::value;
            constexpr int q = qrow<LAT>(ax, i);
            if constexpr (q != 0) mq[ax] += (T)q * d;
          });
        }
        f[i] = omc * f[i] + P + M;
        f[j] = omc * f[j] + P - M;
      }
    });
    if constexpr (CM == CM_MRT_Q) {
      const T fu[3] = {Fx - (T)2 * ux, Fy - (T)2 * uy, Fz - (T)2 * uz};
      static_for<L::D>([&](auto ac) {
        constexpr int ax = decltype(ac)::value;
        static_for<L::D>([&](auto bc) {
          constexpr int b = decltype(bc)::value;
          constexpr T K = (T)qk<LAT>(ax, b);
          if constexpr (K != (T)0) mq[ax] += K * fu[b];
        });
      });
      // all q rows share one rate: a_a = (omega - s_q) m_q,a / |M_q|^2
      const T k = c.ds[4] * (T)(1.0 / mnorm<LAT>(4));
      T aq[3] = {k * mq[0], k * mq[1], k * mq[2]};
      static_for<Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        static_for<L::D>([&](auto ac) {
          constexpr int ax = decltype(ac)::value;
          constexpr int q = qrow<LAT>(ax, i);
          if constexpr (q != 0) f[i] += (T)q * aq[ax];
        });
      });
    }
    return;
  }
  T out[Q];
  T v[MRT ? Q : 1];
  {
    constexpr T w0 = (T)L::w(0);
    const T S = w0 * base, SF = (T)(-3.0 * L::w(0)) * uF;
    out[0] = omc * f[0] + om * S + cf * SF;
    if constexpr (MRT) v[0] = f[0] - S + (T)0.5 * SF;
  }
  static_for<Q>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    if constexpr (i > 0 && L::opp(i) > i) {
      constexpr int j = L::opp(i);
      constexpr T w = (T)L::w(i);
      const T eu = edot<LAT, i, T>(ux, uy, uz);
      const T eF = edot<LAT, i, T>(Fx, Fy, Fz);
      const T S = w * (base + (T)4.5 * eu * eu);
      const T A = (T)(3.0 * L::w(i)) * eu;
      const T SF = w * ((T)9 * eu * eF - (T)3 * uF);
      const T AF = (T)(3.0 * L::w(i)) * eF;
      const T P = om * S + cf * SF, M = om * A + cf * AF;
      out[i] = omc * f[i] + P + M;
      out[j] = omc * f[j] + P - M;
      if constexpr (MRT) {
        const T hs = (T)0.5 * SF - S, ha = (T)0.5 * AF - A;
        v[i] = f[i] + hs + ha;
        v[j] = f[j] + hs - ha;
      }
    }
  });
  if constexpr (MRT) {
    static_for<Q>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      if constexpr (k > 0 && !conserved<LAT>(k)) {
        const T dk = c.ds[k];
        if (dk != (T)0) {
          T m = 0;
          static_for<Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr int mk = mrow<LAT>(k, i);
            if constexpr (mk == 1) m += v[i];
            else if constexpr (mk == -1) m -= v[i];
            else if constexpr (mk != 0) m += (T)mk * v[i];
          });
          const T a = dk * m * (T)(1.0 / mnorm<LAT>(k));
          static_for<Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr int mk = mrow<LAT>(k, i);
            if constexpr (mk == 1) out[i] += a;
            else if constexpr (mk == -1) out[i] -= a;
            else if constexpr (mk != 0) out[i] += (T)mk * a;
          });
        }
      }
    });
  }
  static_for<Q>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    f[i] = out[i];
  });
}

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ int wrap(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// flag bits of a node
enum : uint8_t {
  FL_SOLID = 1,  // no distributions (inside a solid under bounce-back)
  FL_LIST = 2,   // handled by the boundary-node kernel
  FL_NOG = 4,    // the external body force does not act
  FL_BAND = 8,   // the IBM force may be non-zero
  FL_NEW = 16,   // uncovered by a moving solid; refilled before the sweep
  FL_FACE = 32   // next to a non-periodic domain face (the face kernel)
};

}  // namespace lbm
