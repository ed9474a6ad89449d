// Particle kernels for precision f32, template geometry 7 (3D with 4 x 4 x 4-cell tiles).
#define INST_T float
#define INST_G 7
#define INST_NAME lookup_f32_g7
#include "inst.inc"
