// Particle kernels for precision f64, template geometry 5 (2D x-y with 8 x 8-cell tiles).
#define INST_T double
#define INST_G 5
#define INST_NAME lookup_f64_g5
#include "inst.inc"
