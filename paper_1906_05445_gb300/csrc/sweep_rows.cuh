// sweep_rows.cuh -- the bulk sweep fed by bulk asynchronous copies.
//
// The same update as the vector sweep (Eqs. 1-3 with Guo forcing on pairs
// of nodes, sweep_vec.cuh), with another way of getting the pulled values
// to the threads.  A block owns a tile of TR consecutive x-rows (whole rows)
// and walks the lattice's tiles with a stride of the grid size.  For each
// tile, lanes of all the block's warps issue the copies (cp.async.bulk,
// global -> shared, completed on an mbarrier): for direction i the tile's
// source rows (y - e_y, z - e_z) are consecutive in memory except where the
// tile wraps in y or z, so each direction takes one copy of TR rows (two or
// three at a wrap), and the tile's flag bytes take one more.  The x-shift of
// e_x = +-1 then reads the neighbouring value from the same row in shared
// memory, wrapping at the row's ends (periodic x), so there is no halo.
// Two stages per block: a warp releases a stage (a second mbarrier) once
// the values it needs are in registers, and the warps refill it with the
// tile after next as soon as every warp has, so that both stages are in
// flight while the block collides.  The collided values are stored straight
// from registers.
//
// Requirements (checked by the launcher, which otherwise runs the vector
// kernel): nx a multiple of the 32 V nodes of a warp's vectors, two stages
// within the shared memory of a block, and the direction stride, the
// distributions and the flags 16-byte aligned.
#pragma once

#include "sweep_vec.cuh"

namespace lbm {

// ---------------------------------------------------------------- PTX
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count)
               : "memory");
}
// make the initialised barriers visible to the copy engine
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// one arrival that also raises the barrier's expected byte count
__device__ __forceinline__ void mbar_arrive_expect(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *b, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity` of the barrier, for one second at most.
constexpr uint64_t kCopyWaitNs = 1000000000ull;
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity) {
  if (mbar_test(b, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_test(b, parity))
    if (global_ns() - t0 > kCopyWaitNs) return false;
  return true;
}
// bytes (a multiple of 16) from global src to shared dst (both 16-byte
// aligned), completing on barrier b
__device__ __forceinline__ void bulk_copy_in(void *dst, const void *src, uint32_t bytes,
                                             uint64_t *b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(b))
      : "memory");
}
// order this thread's earlier shared-memory accesses before later copies
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---------------------------------------------------------------- layout
// A stage holds, for each direction i, the tile's TR source rows back to
// back (row t at i * TR * row_bytes + t * row_bytes), then the tile's TR * nx
// flag bytes.  Sizes depend on nx and are set by the launcher.
struct RowTiles {
  int rows;          // rows per tile (TR)
  int row_bytes;     // nx * sizeof(S), a multiple of 256
  int stage_bytes;   // Q * TR * row_bytes + TR * nx, rounded up to 16
  int flag_offset;   // Q * TR * row_bytes
  unsigned nrows;    // ny * nz
  unsigned ntiles;   // ceil(nrows / TR)
};

// This warp's share of the copies of tile tl into a stage.  The copies are
// Q + 1 items (direction i's rows, then the flags); item m belongs to warp
// m % nwarps and is issued by its lane m / nwarps, so that no warp issues
// more than a few (an issue costs tens of cycles of the issuing thread).
// Each warp raises the stage's `full` barrier by its own bytes with its one
// arrival.  Every lane of the warp calls this.
template <int LAT, typename S>
__device__ __forceinline__ void issue_tile(const KArgs &a, const RowTiles &g, unsigned tl,
                                           uint8_t *stage, uint64_t *full, int warp, int nwarps,
                                           int lane) {
  using L = Lat<LAT>;
  constexpr int Q = L::Q;
  const unsigned r0 = tl * (unsigned)g.rows;
  const int nr = (int)min((unsigned)g.rows, g.nrows - r0);
  uint32_t bytes = 0;
  for (int m = warp; m <= Q; m += nwarps) bytes += (uint32_t)nr * (uint32_t)(m < Q ? g.row_bytes : a.nx);
  if (lane == 0) mbar_arrive_expect(full, bytes);
  __syncwarp();
  const int m = warp + lane * nwarps;
  if (m < Q) {
    const int i = m;
    const int ey = L::ey(i), ez = L::ez(i);
    // source row of tile row t
    auto srow = [&](int t) {
      const unsigned r = r0 + (unsigned)t;
      const int z = (int)(r / (unsigned)a.ny), y = (int)(r - (unsigned)z * (unsigned)a.ny);
      int ys = y - ey, zs = z - ez;
      ys = ys < 0 ? ys + a.ny : (ys >= a.ny ? ys - a.ny : ys);
      zs = zs < 0 ? zs + a.nz : (zs >= a.nz ? zs - a.nz : zs);
      return (long long)zs * a.ny + ys;
    };
    const uint8_t *src = (const uint8_t *)a.src + (long long)i * a.fs * (long long)sizeof(S);
    uint8_t *slot = stage + (size_t)i * g.rows * g.row_bytes;
    // the shared memory being refilled was read by ordinary loads
    fence_async_smem();
    int t = 0;
    long long s0 = srow(0);
    while (t < nr) {
      int t1 = t + 1;
      long long s1 = 0;
      while (t1 < nr && (s1 = srow(t1)) == s0 + (t1 - t)) t1++;
      bulk_copy_in(slot + (size_t)t * g.row_bytes, src + s0 * g.row_bytes,
                   (uint32_t)(t1 - t) * (uint32_t)g.row_bytes, full);
      t = t1;
      s0 = s1;
    }
  } else if (m == Q) {
    fence_async_smem();
    bulk_copy_in(stage + g.flag_offset, a.flags + (size_t)r0 * a.nx, (uint32_t)(nr * a.nx), full);
  }
}

// Collide and store the vectors of a tile held in a stage: thread j of the
// block takes vectors j, j + blockDim.x, ... of the tile (row-major).  Each
// warp releases the stage (one arrival on `empty`) as soon as its last
// vector is in registers, before colliding it, so that the refill overlaps
// the collision.
template <int LAT, int CM, typename S, int W, bool PACKED>
__device__ __forceinline__ void update_tile(const KArgs &a, const RowTiles &g, unsigned tl,
                                            const uint8_t *stage, uint64_t *empty, int lane) {
  using L = Lat<LAT>;
  using VS = VecS<S>;
  constexpr int Q = L::Q, V = W * VS::per_word;
  const unsigned r0 = tl * (unsigned)g.rows;
  const int nr = (int)min((unsigned)g.rows, g.nrows - r0);
  const int vpr = a.nx / V;            // vectors per row, a multiple of 32
  const int nwords = g.row_bytes / 4;  // words per row
  const int nvec = nr * vpr;
  if ((int)threadIdx.x - lane >= nvec) {  // a warp without vectors in this tile
    if (lane == 0) mbar_arrive(empty);
    return;
  }
  for (int j = threadIdx.x; j < nvec; j += blockDim.x) {
    const int t = j / vpr, xv = j - t * vpr;
    const int w0 = W * xv;
    const int wl = w0 == 0 ? nwords - 1 : w0 - 1, wr = w0 + W == nwords ? 0 : w0 + W;
    Words<W> v[Q];
    static_for<Q>([&](auto ic) {
      constexpr int i = decltype(ic)::value;
      const uint32_t *row =
          reinterpret_cast<const uint32_t *>(stage + ((size_t)i * g.rows + t) * g.row_bytes);
      if constexpr (W == 4) {
        const uint4 q = *reinterpret_cast<const uint4 *>(row + w0);
        v[i].w[0] = q.x, v[i].w[1] = q.y, v[i].w[2] = q.z, v[i].w[3] = q.w;
      } else {
        const uint2 q = *reinterpret_cast<const uint2 *>(row + w0);
        v[i].w[0] = q.x, v[i].w[1] = q.y;
      }
      // the word before (after) the vector, wrapped in the row, holds node
      // x0 - 1 (x0 + V): in its high (low) half for 16-bit storage
      if constexpr (L::ex(i) == 1) VS::shift_in_left(v[i], row[wl]);
      else if constexpr (L::ex(i) == -1) VS::shift_in_right(v[i], row[wr]);
    });
    uint32_t fl[(V + 3) / 4];
    ld_flags<V>(stage + g.flag_offset + (size_t)t * a.nx + V * xv, fl);
    // the same pass count for every lane of a warp (vpr is a multiple of 32);
    // the arrival releases the lanes' shared-memory reads above
    if (j + (int)blockDim.x >= nvec) {
      __syncwarp();
      if (lane == 0) mbar_arrive(empty);
    }
    const unsigned n0 = (r0 + (unsigned)t) * (unsigned)a.nx + (unsigned)(V * xv);
    vec_collide_store<LAT, CM, S, W, PACKED>(a, v, fl, n0, true);
  }
}

// 8 warps per block; 16-bit storage is held to 128 registers (2 blocks per
// SM).  A wait that runs out (one second) sets a.wait_err and ends the warp,
// which first waits (again a second at most) for the stages it filled that
// nobody consumed.
constexpr int kRowBlock = 256;
template <int LAT, int CM, typename S, int W, bool PACKED>
__global__ void __launch_bounds__(kRowBlock, sizeof(S) == 2 ? 2 : 0)
    k_bulk_rows(const KArgs a, const RowTiles g) {
  extern __shared__ __align__(128) uint8_t rows_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  uint64_t *full = reinterpret_cast<uint64_t *>(rows_smem + 2 * (size_t)g.stage_bytes);
  uint64_t *empty = full + 2;
  if (threadIdx.x == 0) {
    for (int b = 0; b < 4; b++) mbar_init(full + b, nwarps);  // full[0..1], empty[0..1]
    mbar_init_fence();
  }
  __syncthreads();
  const unsigned stride = gridDim.x;
  unsigned tl = blockIdx.x;
  if (tl < g.ntiles) issue_tile<LAT, S>(a, g, tl, rows_smem, full, warp, nwarps, lane);
  for (int k = 0; tl < g.ntiles; tl += stride, k++) {
    const int s = k & 1;
    bool ok = true, issued = false;
    if (tl + stride < g.ntiles) {
      // stage s ^ 1 last held tile k - 1: every warp must have released it
      if (k > 0) ok = __all_sync(0xffffffffu, mbar_wait(empty + (s ^ 1), ((k - 1) >> 1) & 1));
      if (ok) {
        issue_tile<LAT, S>(a, g, tl + stride, rows_smem + (s ^ 1) * (size_t)g.stage_bytes,
                           full + (s ^ 1), warp, nwarps, lane);
        issued = true;
      }
    }
    bool have = false;
    if (ok) have = ok = __all_sync(0xffffffffu, mbar_wait(full + s, (k >> 1) & 1));
    if (!ok) {
      if (lane == 0) atomicOr(a.wait_err, 1);
      // the stages this warp helped fill that nobody consumed
      if (!have) mbar_wait(full + s, (k >> 1) & 1);
      if (issued) mbar_wait(full + (s ^ 1), ((k + 1) >> 1) & 1);
      return;
    }
    update_tile<LAT, CM, S, W, PACKED>(a, g, tl, rows_smem + s * (size_t)g.stage_bytes,
                                       empty + s, lane);
  }
}

// Tile shape for a lattice: as many rows as one pass of the block's threads
// covers (at least one).  stage_bytes = 0 where it does not fit.
template <int LAT, typename S, int W>
RowTiles row_tiles(const KArgs &a, size_t smem_limit) {
  constexpr int Q = Lat<LAT>::Q, V = W * VecS<S>::per_word;
  RowTiles g{};
  const int vpr = a.nx / V;
  g.rows = vpr >= kRowBlock ? 1 : kRowBlock / vpr;
  g.row_bytes = a.nx * (int)sizeof(S);
  g.flag_offset = Q * g.rows * g.row_bytes;
  g.stage_bytes = ((g.flag_offset + g.rows * a.nx + 15) / 16) * 16;
  g.nrows = (unsigned)(a.N / a.nx);
  g.ntiles = (g.nrows + g.rows - 1) / g.rows;
  if (2 * (size_t)g.stage_bytes + 4 * sizeof(uint64_t) > smem_limit) g.stage_bytes = 0;
  return g;
}

}  // namespace lbm
