// dispatch.h -- host-side lookup of the templated particle kernels.  Each
// instantiation unit (inst_<prec>_g<geom>.cu) compiles the tile and loose
// kernels of one precision and template geometry for both shape orders and
// every (pusher, escape) pair a box uses.
#pragma once

namespace pic {

struct KernelSet {
    const void* tile[7];  // one per TILE_VARIANTS entry
    const void* loose;
    const void* batch;    // batched launch, variant batch_tile_variant
};

KernelSet lookup_f32_g0(int ord, int push, int esc);
KernelSet lookup_f32_g1(int ord, int push, int esc);
KernelSet lookup_f32_g2(int ord, int push, int esc);
KernelSet lookup_f32_g3(int ord, int push, int esc);
KernelSet lookup_f32_g4(int ord, int push, int esc);
KernelSet lookup_f32_g5(int ord, int push, int esc);
KernelSet lookup_f32_g6(int ord, int push, int esc);
KernelSet lookup_f32_g7(int ord, int push, int esc);
KernelSet lookup_f64_g0(int ord, int push, int esc);
KernelSet lookup_f64_g1(int ord, int push, int esc);
KernelSet lookup_f64_g2(int ord, int push, int esc);
KernelSet lookup_f64_g5(int ord, int push, int esc);
KernelSet lookup_f64_g6(int ord, int push, int esc);
KernelSet lookup_f64_g7(int ord, int push, int esc);

// geom: the template geometry (Geom: 3 and 4 are the 2D planes with 32 x 32
// tiles, FP32 only; 5 and 6 with 8 x 8 tiles; 7 is 3D with 4 x 4 x 4 tiles)
inline KernelSet lookup_kernels(bool fp64, int geom, int ord, int push, int esc) {
    if (!fp64) {
        if (geom == 0) return lookup_f32_g0(ord, push, esc);
        if (geom == 1) return lookup_f32_g1(ord, push, esc);
        if (geom == 3) return lookup_f32_g3(ord, push, esc);
        if (geom == 4) return lookup_f32_g4(ord, push, esc);
        if (geom == 5) return lookup_f32_g5(ord, push, esc);
        if (geom == 6) return lookup_f32_g6(ord, push, esc);
        if (geom == 7) return lookup_f32_g7(ord, push, esc);
        return lookup_f32_g2(ord, push, esc);
    }
    if (geom == 0) return lookup_f64_g0(ord, push, esc);
    if (geom == 1) return lookup_f64_g1(ord, push, esc);
    if (geom == 5) return lookup_f64_g5(ord, push, esc);
    if (geom == 6) return lookup_f64_g6(ord, push, esc);
    if (geom == 7) return lookup_f64_g7(ord, push, esc);
    return lookup_f64_g2(ord, push, esc);
}

}  // namespace pic
