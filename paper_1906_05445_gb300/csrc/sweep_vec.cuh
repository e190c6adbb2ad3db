// sweep_vec.cuh -- the bulk sweep with vector loads and stores.
//
// Each thread updates V consecutive nodes of one x-row, held as W 32-bit
// words per direction (W = 2 or 4: 8- or 16-byte accesses; V = W for FP32
// storage, 2W for 16-bit storage).  For the directions with e_x = +-1
// the pulled values are the row shifted by one node: the thread takes the
// missing end node from its neighbour lane's vector (or loads it itself at a
// row or warp edge).  The collision then runs on pairs of nodes in packed
// FP32x2 arithmetic (one instruction for two nodes), with the same pair form
// as `collide` in lbm_device.cuh: Eq. 1 (BGK) or Eq. 3 (MRT) with Guo
// forcing, where MRT differs from BGK only on the energy-flux (q) moments.
//
// Requirements (checked by the launcher, which otherwise runs the one-node
// kernel): nx % V == 0 and a direction stride that is a multiple of V.
#pragma once

#include "sweep_impl.cuh"


namespace lbm {

// ---------------------------------------------------------------- FP32x2
__device__ __forceinline__ float2 bc2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b, exactly as a scalar subtraction (b * -1 is exact)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, bc2(-1.f), a); }

// e_I . v for the first direction of an opposite pair (which has a positive
// component on both lattices' orderings)
template <int LAT, int I>
__device__ __forceinline__ float2 edot2(float2 vx, float2 vy, float2 vz) {
  using L = Lat<LAT>;
  constexpr int a = L::ex(I), b = L::ey(I), c = L::ez(I);
  static_assert(a == 1 || b == 1 || c == 1, "pair leader without a positive component");
  constexpr int first = a == 1 ? 0 : (b == 1 ? 1 : 2);
  float2 r = first == 0 ? vx : (first == 1 ? vy : vz);
  if constexpr (first < 1 && b == 1) r = add2(r, vy);
  if constexpr (first < 2 && c == 1) r = add2(r, vz);
  if constexpr (a == -1) r = sub2(r, vx);
  if constexpr (b == -1) r = sub2(r, vy);
  if constexpr (c == -1) r = sub2(r, vz);
  return r;
}

// sum_a q_a,I v_a over the q-moment rows of direction I
template <int LAT, int I>
__device__ __forceinline__ float2 qdot2(const float2 (&v)[3]) {
  constexpr int q0 = qrow<LAT>(0, I), q1 = qrow<LAT>(1, I);
  constexpr int q2 = Lat<LAT>::D == 3 ? qrow<LAT>(2, I) : 0;
  static_assert(q0 != 0 || q1 != 0 || q2 != 0, "direction without a q component");
  float2 r;
  if constexpr (q0 != 0) r = q0 == 1 ? v[0] : mul2(bc2((float)q0), v[0]);
  if constexpr (q1 != 0) {
    if constexpr (q0 != 0) r = fma2(bc2((float)q1), v[1], r);
    else r = q1 == 1 ? v[1] : mul2(bc2((float)q1), v[1]);
  }
  if constexpr (q2 != 0) {
    if constexpr (q0 != 0 || q1 != 0) r = fma2(bc2((float)q2), v[2], r);
    else r = q2 == 1 ? v[2] : mul2(bc2((float)q2), v[2]);
  }
  return r;
}

// Collide two nodes at once (lane x and lane y of every float2): BGK, or MRT
// whose only non-BGK rates are those of the q moments.  Same algebra as
// `collide`: feq and Fbar split into parts even and odd in e over each
// opposite pair (i, j),
//   S  = w[drho - 1.5 u^2 + 4.5 (e.u)^2],  A  = 3 w (e.u),
//   SF = w[9 (e.u)(e.F) - 3 u.F],           AF = 3 w (e.F),
//   f_i* = (1 - omega) f_i + omega (S + A) + (1 - omega/2)(SF + AF),
//   f_j* = (1 - omega) f_j + omega (S - A) + (1 - omega/2)(SF - AF),
// and the q-moment correction (omega - s_q) m_q M_q,i / |M_q|^2 with m_q the
// q moments of Delta + Fbar/2, i.e. of f_i - f_j - 2A + AF over the pairs.
// Grouped for few operations:
//   P = omega S + cforce SF = w B + A g,  B = omega (drho - 1.5 u^2) - 3 cforce u.F,
//       g = 1.5 omega e.u + 3 cforce e.F,
//   M = omega A + cforce AF = omega A + w (3 cforce e.F),
//   m_q,a = sum_i q_a,i (f_i - f_j) + sum_b K_ab (F_b - 2 u_b)   (qk above).
// With SL > 0 the populations and the force come in units of 2^-SL (FP16
// storage's scaled deviations) and the results go out in them: everything
// but the terms quadratic in u and F is linear, and those take their
// constants times 2^-SL.  Every operation then gives 2^SL times its unscaled
// result exactly (power-of-two scaling commutes with rounding), so the
// stored values equal those of colliding the unscaled deviations.
template <int LAT, int CM, int SL = 0>
__device__ __forceinline__ void collide_x2(float2 (&f)[Lat<LAT>::Q], float2 Fx, float2 Fy,
                                           float2 Fz, const Coll<float> &c) {
  using L = Lat<LAT>;
  constexpr int Q = L::Q;
  static_assert(CM != CM_MRT, "general MRT rates run in the one-node kernel");
  constexpr float wa = (float)L::w(1), wb = (float)L::w(Q - 1);
  constexpr float kInv = 1.0f / (float)(1 << SL);  // exact
  constexpr float kS = (float)(1 << SL);
  float2 drho = f[0];
  float2 jx = bc2(0.f), jy = bc2(0.f), jz = bc2(0.f);
  float2 mq[3] = {bc2(0.f), bc2(0.f), bc2(0.f)};  // sum_i q_a,i (f_i - f_j)
  static_for<Q>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    if constexpr (i > 0 && L::opp(i) > i) {
      constexpr int j = L::opp(i);
      static_assert(L::w(i) == L::w(1) || L::w(i) == L::w(Q - 1), "two weight classes");
      drho = add2(drho, add2(f[i], f[j]));
      const float2 d = sub2(f[i], f[j]);
      if constexpr (L::ex(i) == 1) jx = add2(jx, d);
      if constexpr (L::ex(i) == -1) jx = sub2(jx, d);
      if constexpr (L::ey(i) == 1) jy = add2(jy, d);
      if constexpr (L::ey(i) == -1) jy = sub2(jy, d);
      if constexpr (L::ez(i) == 1) jz = add2(jz, d);
      if constexpr (L::ez(i) == -1) jz = sub2(jz, d);
      if constexpr (CM == CM_MRT_Q) {
        static_for<L::D>([&](auto ac) {
          constexpr int ax = decltype(ac)::value;
          constexpr int q = qrow<LAT>(ax, i);
          if constexpr (q == 1) mq[ax] = add2(mq[ax], d);
          else if constexpr (q == -1) mq[ax] = sub2(mq[ax], d);
          else if constexpr (q != 0) mq[ax] = fma2(bc2((float)q), d, mq[ax]);
        });
      }
    }
  });
  const float2 half = bc2(0.5f);
  const float2 ux = fma2(half, Fx, jx), uy = fma2(half, Fy, jy), uz = fma2(half, Fz, jz);
  const float2 uu = fma2(uz, uz, fma2(uy, uy, mul2(ux, ux)));
  const float2 uF = fma2(uz, Fz, fma2(uy, Fy, mul2(ux, Fx)));
  const float2 base = fma2(bc2(-1.5f * kInv), uu, drho);
  const float2 om = bc2(c.omega), omc = bc2(c.omc);
  // the constants of the terms quadratic in u and F carry 2^-SL: 1.5 omega,
  // 3 cforce (each the power-of-two multiple of its unscaled rounding)
  const float om15 = c.omega * (1.5f * kInv), cf3 = c.cforce * (3.f * kInv);
  const float2 B = fma2(bc2(-cf3), uF, mul2(om, base));
  {
    constexpr float w0 = (float)L::w(0);
    f[0] = fma2(omc, f[0], mul2(bc2(w0), B));
  }
  const float2 Ba = mul2(bc2(wa), B), Bb = mul2(bc2(wb), B);
  static_for<Q>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    if constexpr (i > 0 && L::opp(i) > i) {
      constexpr int j = L::opp(i);
      constexpr bool ca = L::w(i) == L::w(1);
      constexpr float w = (float)L::w(i), w3 = (float)(3.0 * L::w(i));
      const float2 eu = edot2<LAT, i>(ux, uy, uz);
      const float2 eF = edot2<LAT, i>(Fx, Fy, Fz);
      const float2 A = mul2(bc2(w3), eu);
      const float2 t = mul2(bc2(cf3), eF);     // 3 cforce e.F (times 2^-SL)
      const float2 g = fma2(bc2(om15), eu, t);  // 1.5 omega e.u + 3 cforce e.F
      const float2 P = fma2(A, g, ca ? Ba : Bb);
      const float2 M = fma2(om, A, mul2(bc2(w * kS), t));
      f[i] = fma2(omc, f[i], add2(P, M));
      f[j] = fma2(omc, f[j], sub2(P, M));
    }
  });
  if constexpr (CM == CM_MRT_Q) {
    // the pairs' -2 A + AF terms of the q moments, then the correction: all q
    // rows share one rate; the rows are odd in e, so the opposite direction
    // of a pair gets the negative correction
    const float2 fu[3] = {fma2(bc2(-2.f), ux, Fx), fma2(bc2(-2.f), uy, Fy), fma2(bc2(-2.f), uz, Fz)};
    static_for<L::D>([&](auto ac) {
      constexpr int ax = decltype(ac)::value;
      static_for<L::D>([&](auto bc) {
        constexpr int b = decltype(bc)::value;
        constexpr float K = (float)qk<LAT>(ax, b);
        if constexpr (K != 0.f) mq[ax] = fma2(bc2(K), fu[b], mq[ax]);
      });
    });
    const float2 k = bc2(c.ds[4] * (float)(1.0 / mnorm<LAT>(4)));
    const float2 aq[3] = {mul2(k, mq[0]), mul2(k, mq[1]), mul2(k, mq[2])};
    static_for<Q>([&](auto ic) {
      constexpr int i = decltype(ic)::value;
      if constexpr (i > 0 && L::opp(i) > i) {
        constexpr int j = L::opp(i);
        const float2 cq = qdot2<LAT, i>(aq);
        f[i] = add2(f[i], cq);
        f[j] = sub2(f[j], cq);
      }
    });
  }
}

// ---------------------------------------------------------------- storage
// W words of a direction's vector; node k of the vector is word k (FP32) or
// the low (k even) / high (k odd) half of word k / 2 (16-bit).
template <int W> struct Words {
  uint32_t w[W];
};
template <int W> __device__ __forceinline__ Words<W> ld_words(const void *p) {
  Words<W> r;
  if constexpr (W == 4) {
    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
    r.w[0] = v.x, r.w[1] = v.y, r.w[2] = v.z, r.w[3] = v.w;
  } else {
    static_assert(W == 2, "8- or 16-byte vectors");
    const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
    r.w[0] = v.x, r.w[1] = v.y;
  }
  return r;
}
template <int W> __device__ __forceinline__ void st_words(void *p, const Words<W> &r) {
  if constexpr (W == 4) {
    *reinterpret_cast<uint4 *>(p) = make_uint4(r.w[0], r.w[1], r.w[2], r.w[3]);
  } else {
    *reinterpret_cast<uint2 *>(p) = make_uint2(r.w[0], r.w[1]);
  }
}

// high half of a, low half of b
__device__ __forceinline__ uint32_t join16(uint32_t a, uint32_t b) {
  return __byte_perm(a, b, 0x5432);
}

template <typename S> struct VecS;
template <> struct VecS<float> {
  static constexpr int per_word = 1;
  static constexpr int kScaleLog2 = 0;  // stored values are the deviations
  // the end node fetched from outside the vector, as the word the shift
  // below expects
  __device__ static uint32_t left_word(const float *p) { return __float_as_uint(__ldg(p)); }
  __device__ static uint32_t right_word(const float *p) { return __float_as_uint(__ldg(p)); }
  // shift by one node: e_x = +1 pulls from x - 1, e_x = -1 from x + 1
  template <int W> __device__ static void shift_in_left(Words<W> &v, uint32_t l) {
#pragma unroll
    for (int k = W - 1; k > 0; k--) v.w[k] = v.w[k - 1];
    v.w[0] = l;
  }
  template <int W> __device__ static void shift_in_right(Words<W> &v, uint32_t r) {
#pragma unroll
    for (int k = 0; k < W - 1; k++) v.w[k] = v.w[k + 1];
    v.w[W - 1] = r;
  }
  // pair p (nodes 2p, 2p + 1) as float2, and back
  template <int W> __device__ static float2 get(const Words<W> &v, int p, float2) {
    return make_float2(__uint_as_float(v.w[2 * p]), __uint_as_float(v.w[2 * p + 1]));
  }
  template <int W> __device__ static void put(Words<W> &v, int p, float2 f, float2) {
    v.w[2 * p] = __float_as_uint(f.x);
    v.w[2 * p + 1] = __float_as_uint(f.y);
  }
  template <int W> __device__ static void store_node(float *p, const Words<W> &v, int k) {
    *p = __uint_as_float(v.w[k]);
  }
};

template <typename H> struct VecS16 {
  static constexpr int per_word = 2;
  static constexpr int kScaleLog2 = 0;
  __device__ static uint32_t ld16(const H *p) {
    return (uint32_t)__ldg(reinterpret_cast<const unsigned short *>(p));
  }
  // node x0 - 1 in the high half, node x0 + V in the low half
  __device__ static uint32_t left_word(const H *p) { return ld16(p) << 16; }
  __device__ static uint32_t right_word(const H *p) { return ld16(p); }
  template <int W> __device__ static void shift_in_left(Words<W> &v, uint32_t l) {
#pragma unroll
    for (int k = W - 1; k > 0; k--) v.w[k] = join16(v.w[k - 1], v.w[k]);
    v.w[0] = join16(l, v.w[0]);
  }
  template <int W> __device__ static void shift_in_right(Words<W> &v, uint32_t r) {
#pragma unroll
    for (int k = 0; k < W - 1; k++) v.w[k] = join16(v.w[k], v.w[k + 1]);
    v.w[W - 1] = join16(v.w[W - 1], r);
  }
  template <int W> __device__ static void store_node(H *p, const Words<W> &v, int k) {
    const uint32_t w = v.w[k >> 1];
    *reinterpret_cast<unsigned short *>(p) = (unsigned short)((k & 1) ? (w >> 16) : (w & 0xffffu));
  }
};

template <> struct VecS<__nv_bfloat16> : VecS16<__nv_bfloat16> {
  template <int W> __device__ static float2 get(const Words<W> &v, int p, float2) {
    const uint32_t w = v.w[p];
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
  }
  template <int W> __device__ static void put(Words<W> &v, int p, float2 f, float2) {
    const __nv_bfloat162 h = __float22bfloat162_rn(f);
    v.w[p] = *reinterpret_cast<const uint32_t *>(&h);
  }
};

// FP16 holds deviations times 2^k (k = kFp16ScaleLog2): get multiplies by
// inv_scale = 2^-k, put by scale = 2^k (both exact); get_scaled / put_scaled
// keep the scaled units, for the packed collision that works in them
template <> struct VecS<__half> : VecS16<__half> {
  static constexpr int kScaleLog2 = kFp16ScaleLog2;
  template <int W> __device__ static float2 get_scaled(const Words<W> &v, int p) {
    const uint32_t w = v.w[p];
    return __half22float2(*reinterpret_cast<const __half2 *>(&w));
  }
  template <int W> __device__ static void put_scaled(Words<W> &v, int p, float2 f) {
    const __half2 h = __float22half2_rn(f);
    v.w[p] = *reinterpret_cast<const uint32_t *>(&h);
  }
  template <int W> __device__ static float2 get(const Words<W> &v, int p, float2 inv_scale) {
    return mul2(get_scaled(v, p), inv_scale);
  }
  template <int W> __device__ static void put(Words<W> &v, int p, float2 f, float2 scale) {
    put_scaled(v, p, mul2(f, scale));
  }
};

// flag bytes of V consecutive nodes (V = 2, 4 or 8, aligned), as words
template <int V> __device__ __forceinline__ void ld_flags(const uint8_t *p, uint32_t (&f)[(V + 3) / 4]) {
  if constexpr (V == 8) {
    const uint2 w = *reinterpret_cast<const uint2 *>(p);
    f[0] = w.x;
    f[1] = w.y;
  } else if constexpr (V == 4) {
    f[0] = *reinterpret_cast<const uint32_t *>(p);
  } else {
    f[0] = *reinterpret_cast<const uint16_t *>(p);
  }
}

// ---------------------------------------------------------------- kernel
// The second half of a vector update: collide the V pulled nodes of a
// thread (v, their flag bytes fl) and store the plain fluid ones at n0.  A
// node is updated when its flag byte has no bit but FL_NOG / FL_NEW; the
// other nodes of a vector (boundary-list nodes, solid nodes) are computed but
// not stored, since the boundary-node kernel writes them.
template <int LAT, int CM, typename S, int W, bool PACKED>
__device__ __forceinline__ void vec_collide_store(const KArgs &a, Words<W> (&v)[Lat<LAT>::Q],
                                                  const uint32_t (&fl)[(W * VecS<S>::per_word + 3) / 4],
                                                  unsigned n0, bool valid) {
  using L = Lat<LAT>;
  using VS = VecS<S>;
  constexpr int Q = L::Q, V = W * VS::per_word, NP = V / 2;
  static_assert(V % 2 == 0, "nodes are collided in pairs");
  constexpr uint32_t kOther = (uint8_t)~(FL_NOG | FL_NEW);
  auto flag = [&](int k) { return (fl[k >> 2] >> (8 * (k & 3))) & 0xffu; };
  bool all = valid, any = false;
#pragma unroll
  for (int k = 0; k < V; k++) {
    const bool u = (flag(k) & kOther) == 0;
    all = all && u;
    any = any || u;
  }
  any = any && valid;
  const Coll<float> c = make_coll<LAT, float>(a);
  // the packed collision of FP16 storage runs in its scaled units (the host
  // sets a.inv_scale_f = 2^-SL for it); the rest unscale on load
  constexpr int SL = PACKED ? VS::kScaleLog2 : 0;
  const float2 isc = bc2(a.inv_scale_f), sc = bc2(1.0f / a.inv_scale_f);
  constexpr float kF = (float)(1 << SL);  // force in the same units (exact)
  const float gx = a.g_f[0] * kF, gy = a.g_f[1] * kF, gz = a.g_f[2] * kF;
  static_for<NP>([&](auto pc) {
    constexpr int p = decltype(pc)::value;
    float2 f[Q];
    static_for<Q>([&](auto ic) {
      constexpr int i = decltype(ic)::value;
      if constexpr (SL != 0) f[i] = VS::get_scaled(v[i], p);
      else f[i] = VS::get(v[i], p, isc);
    });
    const float g0 = (flag(2 * p) & FL_NOG) ? 0.f : 1.f;
    const float g1 = (flag(2 * p + 1) & FL_NOG) ? 0.f : 1.f;
    if constexpr (PACKED) {
      collide_x2<LAT, CM, SL>(f, make_float2(g0 * gx, g1 * gx), make_float2(g0 * gy, g1 * gy),
                              make_float2(g0 * gz, g1 * gz), c);
    } else {
      float fa[Q], fb[Q];
      static_for<Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        fa[i] = f[i].x;
        fb[i] = f[i].y;
      });
      collide<LAT, CM, float>(fa, g0 * gx, g0 * gy, g0 * gz, c);
      collide<LAT, CM, float>(fb, g1 * gx, g1 * gy, g1 * gz, c);
      static_for<Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        f[i] = make_float2(fa[i], fb[i]);
      });
    }
    static_for<Q>([&](auto ic) {
      constexpr int i = decltype(ic)::value;
      if constexpr (SL != 0) VS::put_scaled(v[i], p, f[i]);
      else VS::put(v[i], p, f[i], sc);
    });
  });
  S *dst = (S *)a.dst;
  if (all) {
    static_for<Q>([&](auto ic) {
      constexpr int i = decltype(ic)::value;
      st_words<W>(dst + (long long)i * a.fs + n0, v[i]);
    });
  } else if (any) {
#pragma unroll
    for (int k = 0; k < V; k++) {
      if (flag(k) & kOther) continue;
      static_for<Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        VS::store_node(dst + (long long)i * a.fs + n0 + k, v[i], k);
      });
    }
  }
}

// Thread t updates the vector of nodes [V t, V t + V), pulling the shifted
// rows straight from global memory.  Every lane of the warp calls this
// (threads past the end with t >= nt), for the shuffles.
template <int LAT, int CM, typename S, int W, bool PACKED>
__device__ __forceinline__ void bulk_vec_update(const KArgs &a, unsigned t, unsigned nt) {
  using L = Lat<LAT>;
  using VS = VecS<S>;
  constexpr int Q = L::Q, V = W * VS::per_word;
  const bool valid = t < nt;
  // threads past the end still take part in the lane shuffles (on node 0)
  const unsigned n0 = valid ? t * V : 0u;
  const unsigned yz = n0 / (unsigned)a.nx;
  const int x0 = (int)(n0 - yz * (unsigned)a.nx);
  const int z = (int)(yz / (unsigned)a.ny);
  const int y = (int)(yz - (unsigned)z * (unsigned)a.ny);
  uint32_t fl[(V + 3) / 4];
  ld_flags<V>(a.flags + n0, fl);
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
  // source rows (y - e_y, z - e_z)
  const unsigned r[3][3] = {
      {(unsigned)nx * (ym + (unsigned)ny * zm), (unsigned)nx * (y + (unsigned)ny * zm),
       (unsigned)nx * (yp + (unsigned)ny * zm)},
      {(unsigned)nx * (ym + (unsigned)ny * z), (unsigned)nx * (y + (unsigned)ny * z),
       (unsigned)nx * (yp + (unsigned)ny * z)},
      {(unsigned)nx * (ym + (unsigned)ny * zp), (unsigned)nx * (y + (unsigned)ny * zp),
       (unsigned)nx * (yp + (unsigned)ny * zp)}};
  const int lane = threadIdx.x & 31;
  // the neighbour lane holds the adjacent vector of the same row
  const bool lnb = lane != 0 && x0 != 0;
  const bool rnb = lane != 31 && x0 + V != nx;
  const int xl = x0 == 0 ? nx - 1 : x0 - 1, xr = x0 + V == nx ? 0 : x0 + V;
  const S *src = (const S *)a.src;
  Words<W> v[Q];
  uint32_t edge[Q];
  static_for<Q>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    const S *row = src + (long long)i * a.fs + r[1 - L::ez(i)][1 - L::ey(i)];
    v[i] = ld_words<W>(row + x0);
    edge[i] = 0u;
    if constexpr (L::ex(i) == 1) {
      if (!lnb) edge[i] = VS::left_word(row + xl);
    } else if constexpr (L::ex(i) == -1) {
      if (!rnb) edge[i] = VS::right_word(row + xr);
    }
  });
  static_for<Q>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    if constexpr (L::ex(i) == 1) {
      const uint32_t sw = __shfl_up_sync(0xffffffffu, v[i].w[W - 1], 1);
      VS::shift_in_left(v[i], lnb ? sw : edge[i]);
    } else if constexpr (L::ex(i) == -1) {
      const uint32_t sw = __shfl_down_sync(0xffffffffu, v[i].w[0], 1);
      VS::shift_in_right(v[i], rnb ? sw : edge[i]);
    }
  });
  vec_collide_store<LAT, CM, S, W, PACKED>(a, v, fl, n0, valid);
}


// One thread per vector.  (A persistent grid walking the lattice measured
// slower: it holds more registers and leaves the boundary kernels less room;
// so did one that kept the next vector's loads in flight through a cp.async
// ring in shared memory.)  The 8-byte 16-bit kernels are held to 128
// registers, 4 blocks of 128 per SM (130 unbounded: 3 blocks); the FP32
// node-by-node kernel to 64, 8 blocks of 128 per SM (88 unbounded: 5 blocks),
// whose extra warps hide more of the boundary kernel's share of the SMs.
template <int LAT, int CM, typename S, int W, bool PACKED>
__global__ void __launch_bounds__(256, (sizeof(S) == 2 && W == 2) ? 2 : ((sizeof(S) == 4 && W == 2 && !PACKED) ? 4 : 0))
    k_bulk_vec(const KArgs a) {
  constexpr int V = W * VecS<S>::per_word;
  bulk_vec_update<LAT, CM, S, W, PACKED>(a, blockIdx.x * blockDim.x + threadIdx.x,
                                         (unsigned)a.N / V);
}

// The same update for several lattices in one grid: block b belongs to the
// last lattice k with block_start[k] <= b.
// Each lattice gets its own inlined copy of the update, so that its
// arguments stay constant-bank operands (indexing the argument array by a
// run-time k holds them in registers: 92 instead of 80, one block per SM
// fewer).
// Register limits near the single-lattice kernel's: 80 for the FP32
// node-by-node variant (6 blocks of 128 per SM), 128 for the 2-word 16-bit
// ones; 4-word vectors are left unbounded.
template <int LAT, int CM, typename S, int W, bool PACKED>
__global__ void __launch_bounds__(256, W == 4 ? 1 : (sizeof(S) == 4 && !PACKED) ? 3 : 2)
    k_bulk_vec_group(const __grid_constant__ GroupArgs g) {
  constexpr int V = W * VecS<S>::per_word;
  const int b = (int)blockIdx.x;
  static_for<kMaxGroup>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    if (k < g.n && b >= g.block_start[k] && b < g.block_start[k + 1])
      bulk_vec_update<LAT, CM, S, W, PACKED>(
          g.a[k], (unsigned)(b - g.block_start[k]) * blockDim.x + threadIdx.x, (unsigned)g.a[k].N / V);
  });
}

}  // namespace lbm
