// Particle kernels for precision f32, template geometry 4 (2D x-z with 32 x 32-cell tiles).
#define INST_T float
#define INST_G 4
#define INST_NAME lookup_f32_g4
#include "inst.inc"
