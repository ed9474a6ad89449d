// Particle kernels for precision f32, geometry 1 (0: 3D, 1: 2D x-y, 2: 2D x-z).
#define INST_T float
#define INST_G 1
#define INST_NAME lookup_f32_g1
#include "inst.inc"
