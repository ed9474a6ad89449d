// Particle kernels for precision f64, geometry 0 (0: 3D, 1: 2D x-y, 2: 2D x-z).
#define INST_T double
#define INST_G 0
#define INST_NAME lookup_f64_g0
#include "inst.inc"
