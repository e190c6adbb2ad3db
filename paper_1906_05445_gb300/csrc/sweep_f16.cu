// sweep_f16.cu -- sweep kernels with __half storage and float arithmetic.
#include "boundary_impl.cuh"

namespace lbm {
void launch_sweep_f16(SweepOp op, int lattice, int collision, const KArgs &a,
                        cudaStream_t st) {
  launch_precision<__half, float>(op, lattice, collision, a, st);
}
}  // namespace lbm
