// Particle kernels for precision f64, template geometry 7 (3D with 4 x 4 x 4-cell tiles).
#define INST_T double
#define INST_G 7
#define INST_NAME lookup_f64_g7
#include "inst.inc"
