// Instantiations of the band sweeps (sf_sweep.cuh) for the plain SGM (constant P2, no uniqueness filter).
#include "sf_sweep.cuh"

namespace sf {
namespace fused {

cudaError_t launch_sweep_plain(const SweepArgs& a, int mode, cudaStream_t s) {
  return sweep_launch<false>(a, mode, s);
}

}  // namespace fused
}  // namespace sf
