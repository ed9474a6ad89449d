// common.cuh -- shared device-side definitions of libpic (CUDA, sm_103a).
//
// Grid arrays are padded with guard cells on every active axis: GL = 2 on the
// low side and at least GR = 3 on the high side (the x pitch is rounded up so
// that rows start on 16-byte boundaries, as TMA requires).  The 2D ignorable
// axis has extent 1 and no guards.  Particles are stored per species in SoA
// arrays, grouped by tile; see particle.cuh.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pic {

constexpr int GL = 2;  // low guard cells
constexpr int GR = 3;  // high guard cells (deposits reach node n+2)

// geometry kinds: which axes are active.  G2XY_W / G2XZ_W and G2XY_S /
// G2XZ_S are the 2D planes again, with 32 x 32- and 8 x 8-cell particle
// tiles instead of 16 x 16, and G3D_S is 3D with 4 x 4 x 4 tiles instead of
// 8 x 8 x 8 (template geometries: the grid and field code is that of the
// plain geometry).
enum Geom : int { G3D = 0, G2XY = 1, G2XZ = 2, G2XY_W = 3, G2XZ_W = 4, G2XY_S = 5, G2XZ_S = 6, G3D_S = 7 };
constexpr int N_TGEOM = 8;
__host__ __device__ constexpr int plane_of(int G) {
    return (G == G2XY_W || G == G2XY_S) ? G2XY : ((G == G2XZ_W || G == G2XZ_S) ? G2XZ : (G == G3D_S ? G3D : G));
}
// particle tile side in cells (per active axis) of a template geometry
__host__ __device__ constexpr int tile_side(int G) {
    return G == G3D_S ? 4 : ((G == G3D || G == G2XY_S || G == G2XZ_S) ? 8 : ((G == G2XY_W || G == G2XZ_W) ? 32 : 16));
}
// the template geometry of a geometry (G3D, G2XY, G2XZ) with tiles of `side` cells
__host__ __device__ constexpr int tgeom_of(int geom, int side) {
    return geom == G3D ? (side == 4 ? G3D_S : G3D)
           : side == 32 ? (geom == G2XY ? G2XY_W : G2XZ_W)
           : side == 8 ? (geom == G2XY ? G2XY_S : G2XZ_S) : geom;
}
// template geometries with kernels for a precision (32 x 32 tiles: FP32 only)
__host__ __device__ constexpr bool tgeom_built(int tg, bool fp64) { return !(fp64 && (tg == G2XY_W || tg == G2XZ_W)); }
// particle pusher kinds
enum Push : int { PUSH_BORIS = 0, PUSH_KSB = 1, PUSH_KEB = 2, PUSH_SXE = 3 /* shearing + expanding */ };
// escape kinds (leaky box)
enum Esc : int { ESC_NONE = 0, ESC_DISP = 1, ESC_PROB = 2 };

// device error word bits
enum : int {
    ERRB_TMA_TIMEOUT = 1,
    ERRB_NONFINITE = 2,
    ERRB_LOOSE_OVERFLOW = 4,
    ERRB_BAD_CELL = 8,
    ERRB_J_RANGE = 16,  // a fixed-point current sum reached half its range
    ERRB_SMEM_ALIGN = 32,  // a TMA destination in shared memory was not 128-byte aligned (copy skipped)
    ERRB_BATCH = 64,       // a batched launch met an inconsistent work item (skipped)
};

template <int G> struct GeomT {
    static constexpr int P = plane_of(G);
    static constexpr bool AX = true;
    static constexpr bool AY = (P != G2XZ);
    static constexpr bool AZ = (P != G2XY);
    static constexpr int IGN = (P == G2XY) ? 2 : ((P == G2XZ) ? 1 : -1);  // ignorable axis
};

// Padded grid geometry (element offsets).  cell (i,j,k) -> index
// ((k+gz)*py + (j+gy))*px + (i+gx).
struct Grid {
    int nx, ny, nz;     // physical cells
    int px, py, pz;     // padded extents
    int gx, gy, gz;     // low guards per axis (0 on an ignorable axis)
    long long cstride;  // elements per component (px*py*pz)
    __host__ __device__ long long idx(int i, int j, int k) const {
        return ((long long)(k + gz) * py + (j + gy)) * px + (i + gx);
    }
};

// Coefficients of one Yee curl update: out_c <- a_c out_c + b_c curl(s (.) in)_c + g_c J_c.
struct Coef3 { double a[3], b[3], g[3], s[3]; };

// Per-step, time-dependent scalars, kept in device memory so that a captured
// CUDA graph of a step stays valid from one step to the next.  ctx_kernel
// fills it at the start of every step from the step counter next_step.
struct StepCtx {
    long long next_step;  // the step the next ctx_kernel starts (written by the host on pic_set_step)
    long long step;       // n of the step in progress (fields at t^n = n)
    int dys_i[3];         // shearing shift Dy_s mod ny at t, t+1/2, t+1: integer part
    double dys_f[3];      //                                               fractional part
    double inv_lh[3];     // 1 / l_i(t + 1/2) (expanding box)
    double lh[3];         // l_i(t + 1/2)
    float f_dys_f[3];     // the same three in FP32, for the FP32 particle path
    float f_inv_lh[3];
    float f_lh[3];
    Coef3 curl[3];        // curl updates of the step: B half, E full, B half
    // shearing + expanding box (ones for the shearing box): the shear flow in
    // the expanding coordinates, (l_1/l_2)(t + 1/2); l_1(t), which turns xi_x
    // into the physical radial coordinate; X^ = ell L^{-1} X at t (pre) and
    // back with L / ell at t + 1 (post); the midpoint right-hand sides' curl
    // factors l_a^2 / ell and the factors (l_2/l_1)^2, (l_2/l_3)^2 of the
    // -V d_x E^_y and -V d_z E^_y terms, all at t + 1/2
    double sxe_vf, sxe_l0x;
    float f_sxe_vf, f_sxe_l0x;
    double sxe_pre[3], sxe_post[3], sxe_sig[3];
    double sxe_rx, sxe_rz;
};

// Constants ctx_kernel needs (fixed for a handle).
struct CtxConst {
    int box;        // 1 shearing, 2 expanding, 4 shearing + expanding, other: static
    int ny;
    double sO_Lx;   // s Omega0 nx: Dy_s(t) = sO_Lx t mod ny
    double rate[3]; // l_i(t) = exp(rate_i t)
    double c;
};

__device__ inline void ctx_update(StepCtx* ctx, const CtxConst& k);

__global__ inline void ctx_kernel(StepCtx* ctx, CtxConst k) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    ctx_update(ctx, k);
}

// Fill the context of the step that starts now (one thread).
__device__ inline void ctx_update(StepCtx* ctx, const CtxConst& k) {
    const long long n = ctx->next_step;
    ctx->step = n;
    ctx->next_step = n + 1;
    const double t = (double)n;
    for (int w = 0; w < 3; ++w) {
        double d = 0.0;
        const double tw = t + 0.5 * w;
        if (k.box == 1 || k.box == 4) {
            // shearing box: Dy_s = s Omega0 Lx t; with expansion the faces slide
            // apart along xi_y at s Omega0 nx l_1/l_2: Dxi_s = s Omega0 nx int_0^t l_1/l_2
            double I = tw;
            if (k.box == 4) {
                const double dr = k.rate[0] - k.rate[1];
                I = dr == 0.0 ? tw : expm1(dr * tw) / dr;
            }
            d = fmod(k.sO_Lx * I, (double)k.ny);
            if (d < 0.0) d += (double)k.ny;
        }
        double fl = floor(d);
        int di = (int)fl;
        ctx->dys_f[w] = d - fl;
        ctx->f_dys_f[w] = (float)(d - fl);
        ctx->dys_i[w] = k.ny > 0 ? di % k.ny : 0;
    }
    double l0[3], lh[3], l1[3];
    for (int a = 0; a < 3; ++a) {
        const bool ex = k.box == 2 || k.box == 4;
        l0[a] = ex ? exp(k.rate[a] * t) : 1.0;
        lh[a] = ex ? exp(k.rate[a] * (t + 0.5)) : 1.0;
        l1[a] = ex ? exp(k.rate[a] * (t + 1.0)) : 1.0;
        ctx->inv_lh[a] = 1.0 / lh[a];
        ctx->f_inv_lh[a] = (float)(1.0 / lh[a]);
        ctx->lh[a] = lh[a];
        ctx->f_lh[a] = (float)lh[a];
    }
    const double e0 = l0[0] * l0[1] * l0[2], eh = lh[0] * lh[1] * lh[2], e1 = l1[0] * l1[1] * l1[2];
    ctx->sxe_vf = lh[0] / lh[1];
    ctx->sxe_l0x = l0[0];
    ctx->f_sxe_vf = (float)ctx->sxe_vf;
    ctx->f_sxe_l0x = (float)l0[0];
    for (int a = 0; a < 3; ++a) {
        ctx->sxe_pre[a] = e0 / l0[a];
        ctx->sxe_post[a] = l1[a] / e1;
        ctx->sxe_sig[a] = lh[a] * lh[a] / eh;
    }
    ctx->sxe_rx = (lh[1] / lh[0]) * (lh[1] / lh[0]);
    ctx->sxe_rz = (lh[1] / lh[2]) * (lh[1] / lh[2]);
    const double FOUR_PI = 12.566370614359172;
    // B^{n+1/2}: B' = ell L^-1 B at t^n, minus (c/2) curl(L E), back with L at n+1/2
    // E^{n+1}:   E' + c curl(L B^{n+1/2}) - 4 pi (ell J'), back with L at n+1
    // B^{n+1}:   B'^{n+1/2} - (c/2) curl(L E^{n+1}), back with L at n+1
    for (int a = 0; a < 3; ++a) {
        ctx->curl[0].a[a] = (lh[a] / eh) * (e0 / l0[a]);
        ctx->curl[0].b[a] = -0.5 * k.c * (lh[a] / eh);
        ctx->curl[0].g[a] = 0.0;
        ctx->curl[0].s[a] = l0[a];
        ctx->curl[1].a[a] = (l1[a] / e1) * (e0 / l0[a]);
        ctx->curl[1].b[a] = k.c * (l1[a] / e1);
        ctx->curl[1].g[a] = -FOUR_PI * (l1[a] / e1);
        ctx->curl[1].s[a] = lh[a];
        ctx->curl[2].a[a] = (l1[a] / e1) * (eh / lh[a]);
        ctx->curl[2].b[a] = -0.5 * k.c * (l1[a] / e1);
        ctx->curl[2].g[a] = 0.0;
        ctx->curl[2].s[a] = l1[a];
    }
}

// ---- packed cell index --------------------------------------------------
// 3D: i in bits 0..10, j in 11..21, k in 22..31 (nx, ny <= 2048, nz <= 1024).
// 2D: first active axis in bits 0..15, second in 16..31 (<= 65536 cells each).
template <int G> struct CellPack {
    static constexpr int P = plane_of(G);
    __host__ __device__ static int pack(int i, int j, int k) {
        if (P == G3D) return (int)((unsigned)i | ((unsigned)j << 11) | ((unsigned)k << 22));
        if (P == G2XY) return (int)((unsigned)i | ((unsigned)j << 16));
        return (int)((unsigned)i | ((unsigned)k << 16));
    }
    __host__ __device__ static void unpack(int c, int& i, int& j, int& k) {
        unsigned u = (unsigned)c;
        if (P == G3D) { i = u & 2047u; j = (u >> 11) & 2047u; k = u >> 22; }
        else if (P == G2XY) { i = u & 65535u; j = u >> 16; k = 0; }
        else { i = u & 65535u; k = u >> 16; j = 0; }
    }
};

// ---- Philox4x32-10 (Salmon et al., SC'11) --------------------------------
struct U4 { uint32_t x[4]; };

__host__ __device__ inline U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                             uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
        uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
        uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
#else
        uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
        uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += W0; k1 += W1;
    }
    U4 r; r.x[0] = c0; r.x[1] = c1; r.x[2] = c2; r.x[3] = c3;
    return r;
}

// stream tags (third counter word)
constexpr uint32_t TAG_ESCAPE = 0x45534350u;  // escape decision
constexpr uint32_t TAG_ENERGY = 0x494E4A54u;  // reinjection energy attempts
constexpr uint32_t TAG_DIRECT = 0x44495243u;  // reinjection direction
constexpr uint32_t TAG_LOADPOS = 0x4C504F53u; // loader: position in cell
constexpr uint32_t TAG_LOADNOI = 0x4C4E4F49u; // loader: Gaussian noise

__host__ __device__ inline U4 draw(uint32_t id, uint32_t seed, long long step, uint32_t tag, uint32_t w3) {
    unsigned long long s = (unsigned long long)step;
    return philox4x32_10((uint32_t)s, (uint32_t)(s >> 32), tag, w3, id, seed);
}

__host__ __device__ inline double u01(uint32_t v) { return ((double)v + 0.5) * (1.0 / 4294967296.0); }

// Isotropic Maxwell-Juettner momentum (u = c gamma beta) at temperature theta.
// Kinetic energy e = gamma - 1 has density ~ (1+e) sqrt(e(e+2)) exp(-e/theta),
// dominated by (sqrt2 e^1/2 + e + sqrt2 e^3/2 + e^2) exp(-e/theta) because
// sqrt(e+2) <= sqrt2 + sqrt(e): draw from that Gamma mixture, accept with
// probability sqrt(e+2)/(sqrt2 + sqrt e) >= 1/sqrt2.  At most 64 attempts
// (the 64th draw is kept).  Computed in FP64 in every precision mode.
__host__ __device__ inline void sample_mj(uint32_t id, uint32_t seed, long long step, double theta,
                                          double c, double& ux, double& uy, double& uz) {
    const double SQ2 = 1.4142135623730951, SQPI = 1.7724538509055159;
    double w0 = SQ2 * (0.5 * SQPI) * theta * sqrt(theta);
    double w1 = theta * theta;
    double w2 = SQ2 * (0.75 * SQPI) * theta * theta * sqrt(theta);
    double w3 = 2.0 * theta * theta * theta;
    double wsum = w0 + w1 + w2 + w3;
    double e = 0.0;
    for (int a = 0; a < 64; ++a) {
        U4 r0 = draw(id, seed, step, TAG_ENERGY, 2u * (uint32_t)a);
        U4 r1 = draw(id, seed, step, TAG_ENERGY, 2u * (uint32_t)a + 1u);
        double pick = u01(r0.x[0]) * wsum;
        double x1 = -log(u01(r0.x[1]));
        double x2 = -log(u01(r0.x[2]));
        double x3 = -log(u01(r0.x[3]));
        double cb = cos(6.283185307179586 * u01(r1.x[1]));
        double hg = -log(u01(r1.x[0])) * cb * cb;
        if (pick < w0) e = theta * (x1 + hg);
        else if (pick < w0 + w1) e = theta * (x1 + x2);
        else if (pick < w0 + w1 + w2) e = theta * (x1 + x2 + hg);
        else e = theta * (x1 + x2 + x3);
        if (u01(r1.x[2]) < sqrt(e + 2.0) / (SQ2 + sqrt(e))) break;
    }
    U4 rd = draw(id, seed, step, TAG_DIRECT, 0u);
    double mu = 2.0 * u01(rd.x[0]) - 1.0;
    double phi = 6.283185307179586 * u01(rd.x[1]);
    double um = c * sqrt(e * (e + 2.0));
    double st = sqrt(1.0 - mu * mu);
    ux = um * st * cos(phi);
    uy = um * st * sin(phi);
    uz = um * mu;
}

// ---- PTX wrappers: mbarrier and TMA ----------------------------------------
__device__ inline uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ inline void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Orders this thread's earlier generic-proxy accesses of shared memory (and,
// after a barrier, those of the threads it synchronised with) before later
// async-proxy (TMA) writes to the same addresses.
__device__ inline void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ inline void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ inline bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: returns false if the phase did not complete within `limit` polls.
__device__ inline bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}

__device__ inline void tma_load_4d(void* dst, const CUtensorMap* map, int x, int y, int z, int w, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
        : "memory");
}

template <class T> __device__ inline void atomic_add_shared(T* p, T v) { atomicAdd(p, v); }

// Add v to the shared int32 word at shared-window address a (no return).
__device__ inline void red_shared(uint32_t a, int v) {
    asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

__device__ inline void red_shared(uint32_t a, double v) {
    asm volatile("red.shared.add.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}

// Add v to the shared word at shared-window address a unless v is zero, as a
// predicated reduction: no branch, so a warp whose lanes differ in which
// contributions vanish still issues a single instruction per word.
__device__ inline void red_shared_nz(uint32_t a, int v) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.s32 p, %1, 0;\n\t@p red.shared.add.s32 [%0], %1;\n\t}" ::"r"(a), "r"(v)
                 : "memory");
}
__device__ inline void red_shared_nz(uint32_t a, double v) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.neu.f64 p, %1, 0d0000000000000000;\n\t@p red.shared.add.f64 [%0], %1;\n\t}" ::"r"(a),
                 "d"(v)
                 : "memory");
}

template <class T> __device__ inline void red_add_global(T* p, T v) { atomicAdd(p, v); }

template <class T> __device__ inline T t_floor(T x);
template <> __device__ inline float t_floor<float>(float x) { return floorf(x); }
template <> __device__ inline double t_floor<double>(double x) { return floor(x); }
template <class T> __device__ inline T t_sqrt(T x);
template <> __device__ inline float t_sqrt<float>(float x) { return sqrtf(x); }
template <> __device__ inline double t_sqrt<double>(double x) { return sqrt(x); }
// Reciprocal and reciprocal square root of the path's arithmetic type: FP64
// divides and takes the square root exactly rounded; FP32 uses the correctly
// rounded reciprocal and the hardware reciprocal square root (about 2 ulp),
// far inside the FP32 path's 1e-6 budget and without the division sequence.
template <class T> __device__ inline T t_rcp(T x);
template <> __device__ inline float t_rcp<float>(float x) { return __frcp_rn(x); }
template <> __device__ inline double t_rcp<double>(double x) { return 1.0 / x; }
template <class T> __device__ inline T t_rsqrt(T x);
template <> __device__ inline float t_rsqrt<float>(float x) { return rsqrtf(x); }
template <> __device__ inline double t_rsqrt<double>(double x) { return 1.0 / sqrt(x); }
template <class T> __device__ inline T t_abs(T x);
template <> __device__ inline float t_abs<float>(float x) { return fabsf(x); }
template <> __device__ inline double t_abs<double>(double x) { return fabs(x); }

}  // namespace pic
