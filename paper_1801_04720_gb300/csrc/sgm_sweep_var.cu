// Instantiations of the band sweeps (sf_sweep.cuh) for the SGM variants compiled in (intensity-adaptive P2 of the SGM cited in
// Sec. 3.1, uniqueness filter of the winners).
#include "sf_sweep.cuh"

namespace sf {
namespace fused {

cudaError_t launch_sweep_variants(const SweepArgs& a, int mode, cudaStream_t s) {
  return sweep_launch<true>(a, mode, s);
}

}  // namespace fused
}  // namespace sf
