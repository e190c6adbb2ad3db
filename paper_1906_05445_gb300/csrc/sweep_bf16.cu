// sweep_bf16.cu -- sweep kernels with __nv_bfloat16 storage and float arithmetic.
#include "boundary_impl.cuh"

namespace lbm {
void launch_sweep_bf16(SweepOp op, int lattice, int collision, const KArgs &a,
                        cudaStream_t st) {
  launch_precision<__nv_bfloat16, float>(op, lattice, collision, a, st);
}
}  // namespace lbm
