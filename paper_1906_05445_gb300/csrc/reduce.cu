// reduce.cu -- FP64 reductions of the steady-state residual
// r = ||u^n - u^(n-K)||_2 / ||u^n||_2 over nodes that carry distributions.
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

namespace {

__global__ void __launch_bounds__(256) k_residual(const double *u, const double *us,
                                                  const uint8_t *flags, long long N,
                                                  int d, double *out2) {
  __shared__ double sh[2][8];
  double num = 0, den = 0;
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    if (flags[n] & FL_SOLID) continue;
    for (int c = 0; c < d; c++) {
      const double a = u[c * N + n], b = us[c * N + n];
      num += (a - b) * (a - b);
      den += a * a;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_down_sync(0xffffffffu, num, o);
    den += __shfl_down_sync(0xffffffffu, den, o);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sh[0][w] = num;
    sh[1][w] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) {
      a += sh[0][k];
      b += sh[1][k];
    }
    atomicAdd(out2, a);
    atomicAdd(out2 + 1, b);
  }
}

}  // namespace

void launch_residual(const double *u, const double *usnap, long long, const uint8_t *flags,
                     long long N, int d, double *out2, cudaStream_t st) {
  cudaMemsetAsync(out2, 0, 2 * sizeof(double), st);
  long long blocks = (N + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;  // a few waves over the 152 SMs
  k_residual<<<(unsigned)blocks, 256, 0, st>>>(u, usnap, flags, N, d, out2);
}

}  // namespace lbm
