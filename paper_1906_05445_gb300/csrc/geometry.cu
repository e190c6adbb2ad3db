// geometry.cu -- solid/fluid flags, the compacted boundary-node list and the
// cut-link records of the interpolated bounce-back schemes (Sec. 2.2,
// Fig. 1): for a fluid node x_f and a direction i whose upstream node
// x_b = x_f - e_i is solid, the wall fraction q = |x_f - x_w| / |x_f - x_b|
// is the first crossing of the segment from x_f towards x_b with the solid's
// surface (FP64), and the rule's coefficients are stored per link.
//
// Work is done over boxes (the bounding boxes of the solids, or the whole
// lattice) in four passes: flags (reads the previous solid ids; a node
// uncovered since the last build is marked FL_NEW until the next one), list
// (claims each node once, appends list entries, cut links and refill
// entries), links (one thread per cut link) and commit (previous ids <- new
// ids).
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr uint8_t FL_CLAIM = 0x80;

// nearest periodic image; the reciprocal replaces a division (the two can
// only disagree for a separation within an ulp of half the period, where
// both images are equally far and the solid tests below do not change)
__device__ __forceinline__ double mimage(double d, int L) {
  return d - L * round(d * (1.0 / L));
}

// separation of node (x,y,z) from the solid's axis/centre, nearest image;
// z is dropped on 2D lattices and for cylinders along z
__device__ __forceinline__ void rel(const GeomArgs &g, const SolidDev &b, int x,
                                    int y, int z, double r[3]) {
  r[0] = mimage(x - b.c[0], g.nx);
  r[1] = mimage(y - b.c[1], g.ny);
  r[2] = (g.lattice == LBM_D2Q9 || b.kind == LBM_CYLINDER_Z) ? 0.0 : mimage(z - b.c[2], g.nz);
}

__device__ __forceinline__ double norm2(const double r[3]) {
  // explicit rounding (no contraction) so that the solid test is reproducible
  return __dadd_rn(__dadd_rn(__dmul_rn(r[0], r[0]), __dmul_rn(r[1], r[1])),
                   __dmul_rn(r[2], r[2]));
}

__device__ __forceinline__ bool inside(const GeomArgs &g, const SolidDev &b,
                                       int x, int y, int z) {
  double r[3];
  rel(g, b, x, y, z, r);
  const double r2 = norm2(r), R2 = __dmul_rn(b.R, b.R);
  return b.fluid_inside ? r2 >= R2 : r2 <= R2;
}

__device__ __forceinline__ long long box_node(const GeomArgs &g, long long t,
                                              int &x, int &y, int &z) {
  int b = 0;
  while (b + 1 < g.nbox && t >= g.box_offset[b + 1]) b++;
  const long long l = t - g.box_offset[b];
  const GeomBox &B = g.box[b];
  const int i = (int)(l % B.bx);
  const int j = (int)((l / B.bx) % B.by);
  const int k = (int)(l / ((long long)B.bx * B.by));
  int x0 = B.x0, y0 = B.y0, z0 = B.z0;
  if (g.box_dev) {
    // anchored on the solid's centre in device memory
    const SolidDev s = solid_of(g, b);
    const double e = g.box_ext[b];
    if (B.bx < g.nx) x0 = (int)floor(s.c[0] - e);
    if (B.by < g.ny) y0 = (int)floor(s.c[1] - e);
    if (B.bz < g.nz) z0 = (int)floor(s.c[2] - e);
  }
  x = wrap(x0 + i, g.nx);
  y = wrap(y0 + j, g.ny);
  z = wrap(z0 + k, g.nz);
  return x + (long long)g.nx * (y + (long long)g.ny * z);
}

// whether (x, y, z) lies inside the domain across its non-periodic faces
__device__ __forceinline__ bool in_domain(const GeomArgs &g, int x, int y, int z) {
  return !((g.face[0] && x < 0) || (g.face[1] && x >= g.nx) || (g.face[2] && y < 0) ||
           (g.face[3] && y >= g.ny) || (g.face[4] && z < 0) || (g.face[5] && z >= g.nz));
}

// byte-wise atomic OR on the flag array (4-byte aligned, padded)
__device__ __forceinline__ uint8_t flag_or(uint8_t *flags, long long n, uint8_t bits) {
  unsigned int *w = (unsigned int *)(flags + (n & ~3LL));
  const int sh = 8 * (int)(n & 3);
  const unsigned int old = atomicOr(w, ((unsigned int)bits) << sh);
  return (uint8_t)(old >> sh);
}

__global__ void k_geom_flags(const GeomArgs g, uint8_t *sid_new) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.box_offset[g.nbox]) return;
  int x, y, z;
  const long long n = box_node(g, t, x, y, z);
  int s_in = 0;
  if (g.scheme != LBM_SCHEME_NONE)
    for (int s = 0; s < g.solids.n; s++)
      if (inside(g, solid_of(g, s), x, y, z)) {
        s_in = s + 1;
        break;
      }
  uint8_t fl = 0;
  const bool ibb =
      (g.scheme >= LBM_BOUNCE_BACK && g.scheme <= LBM_YU_QUAD) || g.scheme == LBM_ZHAO_YONG;
  if (ibb) {
    if (s_in)
      fl |= FL_SOLID;
    else if (g.track_new && g.sid[n] != 0)
      fl |= FL_NEW;
  } else if (g.scheme == LBM_IBM_DIRECT) {
    if (s_in && !g.force_all) fl |= FL_NOG;
    for (int s = 0; s < g.solids.n; s++) {
      // | |r| - R_L | <= band_w, without the square root
      double r[3];
      const SolidDev b = solid_of(g, s);
      rel(g, b, x, y, z, r);
      const double r2 = norm2(r), RL = b.RL;
      const double lo = RL - g.band_w, hi = RL + g.band_w;
      if (r2 <= hi * hi && (lo <= 0 || r2 >= lo * lo)) fl |= FL_BAND;
    }
  }
  if ((g.face[0] && x == 0) || (g.face[1] && x == g.nx - 1) || (g.face[2] && y == 0) ||
      (g.face[3] && y == g.ny - 1) || (g.face[4] && z == 0) || (g.face[5] && z == g.nz - 1))
    fl |= FL_FACE;
  g.flags[n] = fl;
  sid_new[n] = (uint8_t)s_in;
}

// Warp-aggregated append: every lane of the warp calls it (want may be 0);
// returns the lane's first slot in the counter's list.
__device__ __forceinline__ int warp_append(int *counter, int want) {
  const int lane = threadIdx.x & 31;
  int incl = want;  // inclusive prefix over the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  int base = 0;
  if (lane == 31 && total > 0) base = atomicAdd(counter, total);
  base = __shfl_sync(0xffffffffu, base, 31);
  return base + incl - want;
}

// Node pass: cut-link masks, list entries and refill entries.  Every thread
// of the grid reaches the warp-wide appends (no early return).
template <int LAT>
__global__ void __launch_bounds__(256) k_geom_list(const GeomArgs g, const uint8_t *sid_new) {
  using L = Lat<LAT>;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = t < g.box_offset[g.nbox];
  int x = 0, y = 0, z = 0;
  long long n = 0;
  uint8_t fl = FL_SOLID;
  if (valid) {
    n = box_node(g, t, x, y, z);
    fl = g.flags[n];
  }
  const bool ibb =
      (g.scheme >= LBM_BOUNCE_BACK && g.scheme <= LBM_YU_QUAD) || g.scheme == LBM_ZHAO_YONG;
  uint32_t mask = 0;
  if (valid && !(fl & FL_SOLID) && ibb) {
#pragma unroll
    for (int i = 1; i < L::Q; i++) {
      const long long src = wrap(x - L::ex(i), g.nx) +
                            (long long)g.nx * (wrap(y - L::ey(i), g.ny) +
                                               (long long)g.ny * wrap(z - L::ez(i), g.nz));
      if (sid_new[src]) mask |= 1u << i;
    }
  }
  // IBM: only band nodes need the spread force; nodes inside the solid
  // that are not in the band run in the bulk sweep without external force
  bool listed = valid && !(fl & FL_SOLID) && (ibb ? mask != 0 : (fl & FL_BAND) != 0);
  bool refill = valid && !(fl & FL_SOLID) && (fl & FL_NEW) != 0;
  // claim the node once even if it lies in several boxes
  if ((listed || refill) && (flag_or(g.flags, n, FL_CLAIM) & FL_CLAIM)) listed = refill = false;
  const int r = warp_append(&g.counts[2], refill ? 1 : 0);
  if (refill) {
    if (r < g.refill_cap) {
      g.refill_node[r] = (int)n;
      g.refill_sid[r] = (uint8_t)(g.sid[n] - 1);
    } else {
      atomicOr(&g.counts[3], 1);
    }
  }
  const int nl = listed ? __popc(mask) : 0;
  const int idx = warp_append(&g.counts[0], listed ? 1 : 0);
  const int lo = warp_append(&g.counts[1], nl);
  if (!listed) return;
  flag_or(g.flags, n, FL_LIST);
  if (idx >= g.list_cap || lo + nl > g.link_cap) {
    atomicOr(&g.counts[3], 1);
    return;
  }
  g.list_node[idx] = (int)n;
  g.list_mask[idx] = mask;
  g.list_link[idx] = lo;
  for (int c = 0; c < 6; c++) g.list_cst[(long long)c * g.list_cap + idx] = 0.0;
  int link = lo;
  for (int i = 1; i < L::Q; i++) {
    if (!((mask >> i) & 1u)) continue;
    g.link_list[link] = idx;
    g.link_dir[link] = (uint8_t)i;
    link++;
  }
}

// Bounce-back coefficients in the compute type (FP64 build: FP64).
template <typename T>
__device__ int ibb_rule_t(int scheme, T q, bool ff, bool fff, T c[6]) {
  for (int k = 0; k < 6; k++) c[k] = (T)0;
  if (scheme == LBM_ZHAO_YONG) {
    // Eq. 16 (single node, no fallback): c3 weighs the post-collision value
    // leaving the wall at x_f, c1 the pre-collision value arriving at x_f
    // (read from the previous step), c5 the moving-wall term
    const T d = (T)1 / ((T)1 + (T)2 * q);
    c[3] = (T)2 * q * d;
    c[1] = d;
    c[5] = d;
    return scheme;
  }
  int s = scheme;
  if (s == LBM_BOUZIDI_QUAD && !(ff && fff)) s = LBM_BOUZIDI_LIN;
  if (s == LBM_YU_QUAD && !(ff && fff)) s = LBM_YU_LIN;
  if ((s == LBM_BOUZIDI_LIN || s == LBM_YU_LIN) && !ff) s = LBM_BOUNCE_BACK;
  const T one = (T)1, two = (T)2, tq = two * q;
  if (s == LBM_BOUZIDI_QUAD) {
    if (q < (T)0.5) {  // virtual point 1 - 2q between x_f and x_ff
      c[0] = q * (tq + one);
      c[1] = (one + tq) * (one - tq);
      c[2] = -q * (one - tq);
      c[5] = one;
    } else {           // bounce first, then interpolate x_t, x_ff, x_fff
      c[0] = one / (q * (tq + one));
      c[5] = c[0];
      c[3] = (tq - one) / q;
      c[4] = (one - tq) / (tq + one);
    }
  } else if (s == LBM_BOUZIDI_LIN) {
    if (q < (T)0.5) {
      c[0] = tq;
      c[1] = one - tq;
      c[5] = one;
    } else {
      c[0] = one / tq;
      c[5] = c[0];
      c[3] = (tq - one) / tq;
    }
  } else if (s == LBM_YU_QUAD) {
    const T wall = two / ((one + q) * (two + q));
    c[0] = q / (two + q);                                // wall * q(q+1)/2
    c[1] = two * (one - q) / (two + q);                  // wall * (1+q)(1-q)
    c[2] = -q * (one - q) / ((one + q) * (two + q));     // wall * -q(1-q)/2
    c[3] = two * q / (one + q);
    c[4] = -q / (two + q);
    c[5] = wall;
  } else if (s == LBM_YU_LIN) {
    const T wall = one / (one + q);
    c[0] = q * wall;
    c[1] = (one - q) * wall;
    c[3] = q * wall;
    c[5] = wall;
  } else {
    s = LBM_BOUNCE_BACK;
    c[0] = one;
    c[5] = one;
  }
  return s;
}

// Link pass: one thread per cut link -- wall fraction (FP64), rule
// coefficients, wall velocity, lever arm, and the node's state-independent
// part of Eq. 17 (-2 w_i e_i for links to the node's first solid).
template <int LAT, typename T>
__global__ void __launch_bounds__(128) k_geom_links(const GeomArgs g, const uint8_t *sid_new) {
  using L = Lat<LAT>;
  const int link = blockIdx.x * blockDim.x + threadIdx.x;
  int cnt = g.counts[1];
  if (cnt > g.link_cap) cnt = g.link_cap;
  if (link >= cnt) return;
  const int idx = g.link_list[link];
  const int i = g.link_dir[link];
  const long long n = g.list_node[idx];
  const uint32_t mask = g.list_mask[idx];
  const int x = (int)(n % g.nx), y = (int)((n / g.nx) % g.ny), z = (int)(n / ((long long)g.nx * g.ny));
  const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
  const long long src = wrap(x - ex, g.nx) +
                        (long long)g.nx * (wrap(y - ey, g.ny) + (long long)g.ny * wrap(z - ez, g.nz));
  const int s = sid_new[src] - 1;
  const SolidDev b = solid_of(g, s);
  double r[3];
  rel(g, b, x, y, z, r);
  const bool flat = g.lattice == LBM_D2Q9 || b.kind == LBM_CYLINDER_Z;
  const double d[3] = {(double)-ex, (double)-ey, flat ? 0.0 : (double)-ez};
  const int A = (int)(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  const double B = 2.0 * (r[0] * d[0] + r[1] * d[1] + r[2] * d[2]);
  const double C = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] - b.R * b.R;
  double q = 0.5;
  if (A > 0) {
    double disc = B * B - 4.0 * A * C;
    if (disc < 0) disc = 0;
    const double h = A == 1 ? 0.5 : (A == 2 ? 0.25 : 1.0 / 6.0);  // 1 / (2A)
    q = b.fluid_inside ? (-B + sqrt(disc)) * h : (-B - sqrt(disc)) * h;
  }
  if (q > 1.0) q = 1.0;
  if (q < 1e-12) q = 1e-12;
  const long long nff = wrap(x + ex, g.nx) +
                        (long long)g.nx * (wrap(y + ey, g.ny) + (long long)g.ny * wrap(z + ez, g.nz));
  const long long nfff = wrap(x + 2 * ex, g.nx) +
                         (long long)g.nx * (wrap(y + 2 * ey, g.ny) + (long long)g.ny * wrap(z + 2 * ez, g.nz));
  // a stencil node beyond a non-periodic domain face does not exist
  const bool ff = sid_new[nff] == 0 && in_domain(g, x + ex, y + ey, z + ez);
  const bool fff = ff && sid_new[nfff] == 0 && in_domain(g, x + 2 * ex, y + 2 * ey, z + 2 * ez);
  T c[6];
  ibb_rule_t<T>(g.scheme, (T)q, ff, fff, c);
  // wall point relative to the centre and the wall velocity there
  const T arm[3] = {(T)(r[0] - q * ex), (T)(r[1] - q * ey), flat ? (T)0 : (T)(r[2] - q * ez)};
  T uw[3] = {(T)b.U[0] + (T)b.Om[1] * arm[2] - (T)b.Om[2] * arm[1],
             (T)b.U[1] + (T)b.Om[2] * arm[0] - (T)b.Om[0] * arm[2],
             (T)b.U[2] + (T)b.Om[0] * arm[1] - (T)b.Om[1] * arm[0]};
  if (g.lattice == LBM_D2Q9) uw[2] = (T)0;
  const T eu = (T)ex * uw[0] + (T)ey * uw[1] + (T)ez * uw[2];
  for (int k = 0; k < 5; k++) ((T *)g.links.c[k])[link] = c[k];
  ((T *)g.links.mw)[link] = c[5] * (T)(6.0 * L::w(i)) * eu;  // c5 * 2 rho0 w_i e.u / cs2
  for (int k = 0; k < 3; k++) {
    ((T *)g.links.uw[k])[link] = uw[k];
    ((T *)g.links.arm[k])[link] = arm[k];
  }
  g.links.sid[link] = (uint8_t)s;
  // the node's first cut link decides which solid its constant part goes to
  const int first = __ffs(mask) - 1;
  const long long src0 = wrap(x - L::ex(first), g.nx) +
                         (long long)g.nx * (wrap(y - L::ey(first), g.ny) +
                                            (long long)g.ny * wrap(z - L::ez(first), g.nz));
  if (sid_new[src0] - 1 == s) {
    const double w2 = -2.0 * L::w(i);
    const double p[3] = {w2 * ex, w2 * ey, w2 * ez};
    const double am[3] = {(double)arm[0], (double)arm[1], (double)arm[2]};
    double *cst = g.list_cst;
    const long long lc = g.list_cap;
    atomicAdd(cst + 0 * lc + idx, p[0]);
    atomicAdd(cst + 1 * lc + idx, p[1]);
    atomicAdd(cst + 2 * lc + idx, p[2]);
    atomicAdd(cst + 3 * lc + idx, am[1] * p[2] - am[2] * p[1]);
    atomicAdd(cst + 4 * lc + idx, am[2] * p[0] - am[0] * p[2]);
    atomicAdd(cst + 5 * lc + idx, am[0] * p[1] - am[1] * p[0]);
  }
}

__global__ void k_geom_commit(const GeomArgs g, const uint8_t *sid_new) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.box_offset[g.nbox]) return;
  int x, y, z;
  const long long n = box_node(g, t, x, y, z);
  g.sid[n] = sid_new[n];
  g.flags[n] &= (uint8_t)~FL_CLAIM;
}

}  // namespace

// sid_new lives right after sid in the same allocation (N bytes each, padded)
void launch_geometry(const GeomArgs &g, int precision, cudaStream_t st) {
  const long long total = g.box_offset[g.nbox];
  if (total <= 0) return;
  const int bs = 256;
  const unsigned grid = (unsigned)((total + bs - 1) / bs);
  uint8_t *sid_new = g.sid + ((g.N + 15) / 16) * 16;
  k_geom_flags<<<grid, bs, 0, st>>>(g, sid_new);
  const bool dbl = precision == LBM_FP64;
  if (g.lattice == LBM_D2Q9)
    k_geom_list<0><<<grid, bs, 0, st>>>(g, sid_new);
  else
    k_geom_list<1><<<grid, bs, 0, st>>>(g, sid_new);
  // one thread per link, up to the link capacity (the count is on the device)
  if (g.link_cap > 0) {
    const unsigned lg = (unsigned)((g.link_cap + 127) / 128);
    if (g.lattice == LBM_D2Q9) {
      if (dbl) k_geom_links<0, double><<<lg, 128, 0, st>>>(g, sid_new);
      else k_geom_links<0, float><<<lg, 128, 0, st>>>(g, sid_new);
    } else {
      if (dbl) k_geom_links<1, double><<<lg, 128, 0, st>>>(g, sid_new);
      else k_geom_links<1, float><<<lg, 128, 0, st>>>(g, sid_new);
    }
  }
  k_geom_commit<<<grid, bs, 0, st>>>(g, sid_new);
}

}  // namespace lbm
