// Particle kernels for precision f32, template geometry 5 (2D x-y with 8 x 8-cell tiles).
#define INST_T float
#define INST_G 5
#define INST_NAME lookup_f32_g5
#include "inst.inc"
