// Particle kernels for precision f64, template geometry 6 (2D x-z with 8 x 8-cell tiles).
#define INST_T double
#define INST_G 6
#define INST_NAME lookup_f64_g6
#include "inst.inc"
