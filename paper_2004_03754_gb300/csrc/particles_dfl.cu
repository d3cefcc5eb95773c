// particles_dfl.cu -- the particle kernels of libpic for compensated FP32-pair fields.
#include "particle_kernels.cuh"

namespace pic {
PIC_PARTICLE_INST(dfl)
}  // namespace pic
