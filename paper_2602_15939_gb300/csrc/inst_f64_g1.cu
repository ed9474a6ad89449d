// Particle kernels for precision f64, geometry 1 (0: 3D, 1: 2D x-y, 2: 2D x-z).
#define INST_T double
#define INST_G 1
#define INST_NAME lookup_f64_g1
#include "inst.inc"
