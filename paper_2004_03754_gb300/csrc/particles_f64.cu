// particles_f64.cu -- the particle kernels of libpic for FP64 fields.
#include "particle_kernels.cuh"

namespace pic {
PIC_PARTICLE_INST(double)
}  // namespace pic
