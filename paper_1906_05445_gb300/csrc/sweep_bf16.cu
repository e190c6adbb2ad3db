// sweep_bf16.cu -- sweep kernels with __nv_bfloat16 storage and float arithmetic.
#include "boundary_impl.cuh"

namespace lbm {
void launch_sweep_bf16(SweepOp op, int lattice, int collision, const KArgs &a,
                        cudaStream_t st) {
  launch_precision<__nv_bfloat16, float>(op, lattice, collision, a, st);
}
bool launch_bulk_group_bf16(const KArgs *as, int n, int lattice, int collision,
                             cudaStream_t st) {
  return launch_group_precision<__nv_bfloat16>(as, n, lattice, collision, st);
}
}  // namespace lbm
