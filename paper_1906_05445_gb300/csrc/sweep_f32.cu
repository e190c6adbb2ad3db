// sweep_f32.cu -- sweep kernels with float storage and float arithmetic.
#include "boundary_impl.cuh"

namespace lbm {
void launch_sweep_f32(SweepOp op, int lattice, int collision, const KArgs &a,
                        cudaStream_t st) {
  launch_precision<float, float>(op, lattice, collision, a, st);
}
bool launch_bulk_group_f32(const KArgs *as, int n, int lattice, int collision,
                             cudaStream_t st) {
  return launch_group_precision<float>(as, n, lattice, collision, st);
}
}  // namespace lbm
