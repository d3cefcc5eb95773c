// particles_f32.cu -- the particle kernels of libpic for FP32 fields.
#include "particle_kernels.cuh"

namespace pic {
PIC_PARTICLE_INST(float)
}  // namespace pic
