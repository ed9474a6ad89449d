// Particle kernels for precision f32, template geometry 6 (2D x-z with 8 x 8-cell tiles).
#define INST_T float
#define INST_G 6
#define INST_NAME lookup_f32_g6
#include "inst.inc"
