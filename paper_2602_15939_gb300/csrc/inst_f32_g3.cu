// Particle kernels for precision f32, template geometry 3 (2D x-y with 32 x 32-cell tiles).
#define INST_T float
#define INST_G 3
#define INST_NAME lookup_f32_g3
#include "inst.inc"
