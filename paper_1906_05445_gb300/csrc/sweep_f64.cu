// sweep_f64.cu -- sweep kernels with double storage and double arithmetic.
#include "boundary_impl.cuh"

namespace lbm {
void launch_sweep_f64(SweepOp op, int lattice, int collision, const KArgs &a,
                        cudaStream_t st) {
  launch_precision<double, double>(op, lattice, collision, a, st);
}
}  // namespace lbm
