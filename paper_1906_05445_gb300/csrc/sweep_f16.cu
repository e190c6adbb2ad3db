// sweep_f16.cu -- sweep kernels with __half storage and float arithmetic.
#include "boundary_impl.cuh"

namespace lbm {
void launch_sweep_f16(SweepOp op, int lattice, int collision, const KArgs &a,
                        cudaStream_t st) {
  launch_precision<__half, float>(op, lattice, collision, a, st);
}
bool launch_bulk_group_f16(const KArgs *as, int n, int lattice, int collision,
                             cudaStream_t st) {
  return launch_group_precision<__half>(as, n, lattice, collision, st);
}
}  // namespace lbm
