// Particle kernels for precision f32, geometry 2 (0: 3D, 1: 2D x-y, 2: 2D x-z).
#define INST_T float
#define INST_G 2
#define INST_NAME lookup_f32_g2
#include "inst.inc"
