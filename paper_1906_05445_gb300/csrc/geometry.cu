// geometry.cu -- solid/fluid flags, the compacted boundary-node list and the
// cut-link records of the interpolated bounce-back schemes (Sec. 2.2,
// Fig. 1): for a fluid node x_f and a direction i whose upstream node
// x_b = x_f - e_i is solid, the wall fraction q = |x_f - x_w| / |x_f - x_b|
// is the first crossing of the segment from x_f towards x_b with the solid's
// surface (FP64), and the rule's coefficients are stored per link.
//
// Work is done over boxes (the bounding boxes of the solids, or the whole
// lattice) in three passes: flags (reads the previous solid ids), list
// (claims each node once, appends list entries, links and refill entries),
// commit (previous ids <- new ids).
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr uint8_t FL_CLAIM = 0x80;

__device__ __forceinline__ double mimage(double d, int L) { return d - L * round(d / L); }

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
  x = wrap(B.x0 + i, g.nx);
  y = wrap(B.y0 + j, g.ny);
  z = wrap(B.z0 + k, g.nz);
  return x + (long long)g.nx * (y + (long long)g.ny * z);
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
      if (inside(g, g.solids.s[s], x, y, z)) {
        s_in = s + 1;
        break;
      }
  uint8_t fl = 0;
  const bool ibb = g.scheme >= LBM_BOUNCE_BACK && g.scheme <= LBM_YU_QUAD;
  if (ibb) {
    if (s_in)
      fl |= FL_SOLID;
    else if (g.track_new && g.sid[n] != 0)
      fl |= FL_NEW;
  } else if (g.scheme == LBM_IBM_DIRECT) {
    if (s_in && !g.force_all) fl |= FL_NOG;
    for (int s = 0; s < g.solids.n; s++) {
      double r[3];
      rel(g, g.solids.s[s], x, y, z, r);
      const double dist = sqrt(norm2(r));
      if (fabs(dist - g.solids.s[s].RL) <= g.band_w) fl |= FL_BAND;
    }
  }
  g.flags[n] = fl;
  sid_new[n] = (uint8_t)s_in;
}

// Bounce-back coefficients of Sec. 2.2 (Eq. 9, Eq. 11, Eqs. 12-14 and their
// two-point forms) with the fallback quadratic -> linear -> Eq. 9 when the
// interpolation nodes x_ff / x_fff are not fluid.  Returns the rule used.
__device__ int ibb_rule(int scheme, double q, bool ff, bool fff, double c[6]) {
  for (int k = 0; k < 6; k++) c[k] = 0.0;
  int s = scheme;
  if (s == LBM_BOUZIDI_QUAD && !(ff && fff)) s = LBM_BOUZIDI_LIN;
  if (s == LBM_YU_QUAD && !(ff && fff)) s = LBM_YU_LIN;
  if ((s == LBM_BOUZIDI_LIN || s == LBM_YU_LIN) && !ff) s = LBM_BOUNCE_BACK;
  const double tq = 2.0 * q;
  if (s == LBM_BOUZIDI_QUAD) {
    if (q < 0.5) {  // virtual point 1 - 2q between x_f and x_ff
      c[0] = q * (tq + 1.0);
      c[1] = (1.0 + tq) * (1.0 - tq);
      c[2] = -q * (1.0 - tq);
      c[5] = 1.0;
    } else {        // bounce first, then interpolate x_t, x_ff, x_fff
      c[0] = 1.0 / (q * (tq + 1.0));
      c[5] = c[0];
      c[3] = (tq - 1.0) / q;
      c[4] = (1.0 - tq) / (tq + 1.0);
    }
  } else if (s == LBM_BOUZIDI_LIN) {
    if (q < 0.5) {
      c[0] = tq;
      c[1] = 1.0 - tq;
      c[5] = 1.0;
    } else {
      c[0] = 1.0 / tq;
      c[5] = c[0];
      c[3] = (tq - 1.0) / tq;
    }
  } else if (s == LBM_YU_QUAD) {
    const double wall = 2.0 / ((1.0 + q) * (2.0 + q));
    c[0] = q / (2.0 + q);                              // wall * q(q+1)/2
    c[1] = 2.0 * (1.0 - q) / (2.0 + q);                // wall * (1+q)(1-q)
    c[2] = -q * (1.0 - q) / ((1.0 + q) * (2.0 + q));   // wall * -q(1-q)/2
    c[3] = 2.0 * q / (1.0 + q);
    c[4] = -q / (2.0 + q);
    c[5] = wall;
  } else if (s == LBM_YU_LIN) {
    const double wall = 1.0 / (1.0 + q);
    c[0] = q * wall;
    c[1] = (1.0 - q) * wall;
    c[3] = q * wall;
    c[5] = wall;
  } else {
    s = LBM_BOUNCE_BACK;
    c[0] = 1.0;
    c[5] = 1.0;
  }
  return s;
}

template <int LAT, typename T>
__global__ void k_geom_list(const GeomArgs g, const uint8_t *sid_new) {
  using L = Lat<LAT>;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.box_offset[g.nbox]) return;
  int x, y, z;
  const long long n = box_node(g, t, x, y, z);
  const uint8_t fl = g.flags[n];
  if (fl & FL_SOLID) return;
  const bool ibb = g.scheme >= LBM_BOUNCE_BACK && g.scheme <= LBM_YU_QUAD;
  uint32_t mask = 0;
  if (ibb) {
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
  const bool listed = ibb ? mask != 0 : (fl & FL_BAND) != 0;
  const bool refill = (fl & FL_NEW) != 0;
  if (!listed && !refill) return;
  // claim the node once even if it lies in several boxes
  if (flag_or(g.flags, n, FL_CLAIM) & FL_CLAIM) return;
  if (refill) {
    const int r = atomicAdd(&g.counts[2], 1);
    if (r < g.refill_cap) {
      g.refill_node[r] = (int)n;
      g.refill_sid[r] = (uint8_t)(g.sid[n] - 1);
    } else {
      atomicOr(&g.counts[3], 1);
    }
  }
  if (!listed) return;
  flag_or(g.flags, n, FL_LIST);
  const int nl = __popc(mask);
  const int idx = atomicAdd(&g.counts[0], 1);
  const int lo = nl ? atomicAdd(&g.counts[1], nl) : 0;
  if (idx >= g.list_cap || lo + nl > g.link_cap) {
    atomicOr(&g.counts[3], 1);
    return;
  }
  g.list_node[idx] = (int)n;
  g.list_mask[idx] = mask;
  g.list_link[idx] = lo;
  int link = lo;
  // state-independent part of the momentum exchange, -2 w_i e_i per cut link
  // to the node's first solid, and its torque (FP64)
  double cst[6] = {0, 0, 0, 0, 0, 0};
  int first_solid = -1;
  for (int i = 1; i < L::Q; i++) {
    if (!((mask >> i) & 1u)) continue;
    const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
    const long long src = wrap(x - ex, g.nx) +
                          (long long)g.nx * (wrap(y - ey, g.ny) + (long long)g.ny * wrap(z - ez, g.nz));
    const int s = sid_new[src] - 1;
    const SolidDev &b = g.solids.s[s];
    double r[3];
    rel(g, b, x, y, z, r);
    const bool flat = g.lattice == LBM_D2Q9 || b.kind == LBM_CYLINDER_Z;
    const double d[3] = {(double)-ex, (double)-ey, flat ? 0.0 : (double)-ez};
    const double A = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double B = 2.0 * (r[0] * d[0] + r[1] * d[1] + r[2] * d[2]);
    const double C = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] - b.R * b.R;
    double q = 0.5;
    if (A > 0) {
      double disc = B * B - 4.0 * A * C;
      if (disc < 0) disc = 0;
      q = b.fluid_inside ? (-B + sqrt(disc)) / (2.0 * A) : (-B - sqrt(disc)) / (2.0 * A);
    }
    if (q > 1.0) q = 1.0;
    if (q < 1e-12) q = 1e-12;
    const long long nff = wrap(x + ex, g.nx) +
                          (long long)g.nx * (wrap(y + ey, g.ny) + (long long)g.ny * wrap(z + ez, g.nz));
    const long long nfff = wrap(x + 2 * ex, g.nx) +
                           (long long)g.nx * (wrap(y + 2 * ey, g.ny) +
                                              (long long)g.ny * wrap(z + 2 * ez, g.nz));
    const bool ff = sid_new[nff] == 0;
    const bool fff = ff && sid_new[nfff] == 0;
    double c[6];
    const int used = ibb_rule(g.scheme, q, ff, fff, c);
    atomicAdd(&g.counts[4 + used], 1);
    // wall point relative to the centre and the wall velocity there
    const double arm[3] = {r[0] - q * ex, r[1] - q * ey, flat ? 0.0 : r[2] - q * ez};
    double uw[3] = {b.U[0] + b.Om[1] * arm[2] - b.Om[2] * arm[1],
                    b.U[1] + b.Om[2] * arm[0] - b.Om[0] * arm[2],
                    b.U[2] + b.Om[0] * arm[1] - b.Om[1] * arm[0]};
    if (g.lattice == LBM_D2Q9) uw[2] = 0;
    const double eu = ex * uw[0] + ey * uw[1] + ez * uw[2];
    for (int k = 0; k < 5; k++) ((T *)g.links.c[k])[link] = (T)c[k];
    ((T *)g.links.mw)[link] = (T)(c[5] * 6.0 * L::w(i) * eu);  // c5 * 2 rho0 w_i e.u / cs2
    for (int k = 0; k < 3; k++) {
      ((T *)g.links.uw[k])[link] = (T)uw[k];
      ((T *)g.links.arm[k])[link] = (T)arm[k];
    }
    g.links.sid[link] = (uint8_t)s;
    if (first_solid < 0) first_solid = s;
    if (s == first_solid) {
      const double p[3] = {-2.0 * L::w(i) * ex, -2.0 * L::w(i) * ey, -2.0 * L::w(i) * ez};
      cst[0] += p[0];
      cst[1] += p[1];
      cst[2] += p[2];
      cst[3] += arm[1] * p[2] - arm[2] * p[1];
      cst[4] += arm[2] * p[0] - arm[0] * p[2];
      cst[5] += arm[0] * p[1] - arm[1] * p[0];
    }
    link++;
  }
  for (int c = 0; c < 6; c++) g.list_cst[(long long)c * g.list_cap + idx] = cst[c];
}

__global__ void k_geom_commit(const GeomArgs g, const uint8_t *sid_new) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.box_offset[g.nbox]) return;
  int x, y, z;
  const long long n = box_node(g, t, x, y, z);
  g.sid[n] = sid_new[n];
  g.flags[n] &= (uint8_t)~FL_CLAIM;
}

__global__ void k_clear_new(uint8_t *flags, const int *counts, const int *node, int cap) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  int cnt = counts[2];
  if (cnt > cap) cnt = cap;
  if (t >= cnt) return;
  flags[node[t]] &= (uint8_t)~FL_NEW;
}

}  // namespace

void launch_clear_new(uint8_t *flags, const int *counts, const int *node, int cap,
                      cudaStream_t st) {
  if (cap <= 0) return;
  k_clear_new<<<(cap + 127) / 128, 128, 0, st>>>(flags, counts, node, cap);
}

// sid_new lives right after sid in the same allocation (N bytes each, padded)
void launch_geometry(const GeomArgs &g, int precision, cudaStream_t st) {
  const long long total = g.box_offset[g.nbox];
  if (total <= 0) return;
  const int bs = 256;
  const unsigned grid = (unsigned)((total + bs - 1) / bs);
  uint8_t *sid_new = g.sid + ((g.N + 15) / 16) * 16;
  k_geom_flags<<<grid, bs, 0, st>>>(g, sid_new);
  const bool dbl = precision == LBM_FP64;
  if (g.lattice == LBM_D2Q9) {
    if (dbl) k_geom_list<0, double><<<grid, bs, 0, st>>>(g, sid_new);
    else k_geom_list<0, float><<<grid, bs, 0, st>>>(g, sid_new);
  } else {
    if (dbl) k_geom_list<1, double><<<grid, bs, 0, st>>>(g, sid_new);
    else k_geom_list<1, float><<<grid, bs, 0, st>>>(g, sid_new);
  }
  k_geom_commit<<<grid, bs, 0, st>>>(g, sid_new);
}

}  // namespace lbm
