// particle.cuh -- the fused particle step of libpic (CUDA, sm_103a).
//
// One CTA owns one tile of cells.  It stages the tile's E and B (plus guard
// cells) into shared memory with two TMA copies, then, for every particle of
// every species in the tile:
//   gather E, B at x^n (shape order 1 or 2, each component at its own Yee
//   location) -> push (Boris; KSB-OA Boris-like, Sec. 2.2; KEB modified Boris,
//   Sec. 3.2) -> position update (two-stage for the shearing box) ->
//   charge-conserving (Esirkepov) current into a shared-memory J tile ->
//   leaky-box escape test and reinjection (Sec. 4.1) -> write the particle to
//   its slot in the tile-sorted output buffer.
// Particles that stay in the tile are packed at the front of the tile's slot
// range (warp-aggregated shared-memory counter); particles that move to a
// neighbouring tile are appended at the back of that tile's range through a
// global counter.  A particle whose destination tile has no free slot goes to
// a "loose" list handled by loose_kernel (global-memory gather and atomics),
// which re-inserts it as soon as room appears.  After all particles, the J
// tile is added to the global (guarded) J array with one atomic per non-zero
// point.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace pic {

// ---- kernel arguments --------------------------------------------------------

template <class T> struct PView {
    int* cell;
    T* o[3];   // in-cell offsets of the active axes (o[2] unused in 2D)
    T* u[3];
    uint32_t* id;
    T* dr[3];  // leaky-box displacement (null otherwise)
};

template <class T> struct SpecStep {
    PView<T> in, out;      // tile-sorted buffers
    PView<T> lin, lout;    // loose lists
    const int* stay_in;    // [ntiles]
    int* arr_in;           // [ntiles], zeroed by the kernel after reading
    int* stay_out;         // [ntiles]
    int* arr_out;          // [ntiles], must be zero on entry
    const int* lcount_in;  // loose count of lin
    int* lcount_out;       // loose count of lout (atomic)
    long long tcap;        // slots per tile
    long long lcap;        // loose-list capacity
    T qdt2m;               // q dt / (2 m)
    T qdt2mc;              // q dt / (2 m c)
    T q;                   // macro charge
};

constexpr int MAXSP = 4;

template <class T> struct SpecPack { SpecStep<T> s[MAXSP]; };

struct Tiling {
    int tx, ty, tz;     // tile extent (cells) per axis, 1 on the ignorable axis
    int ntx, nty, ntz;  // tiles per axis
    int ntiles;
    int bx, by, bz;     // staged field box (elements)
    int xalign;         // TMA x quantum (elements)
    int jx, jy, jz;     // shared J box (points)
};

// FP32 copies of the FP64 step constants below (the time-dependent ones are
// refreshed by with_ctx from the device context): the FP32 particle path
// reads them from the parameter bank, with no FP64 conversion per particle.
struct StepPF {
    float c, inv_c, inv_c2, sO, Omega0, half_nx, l_esc, dys_end_f;
    float Lam[3], im[3], Lt[3], inv_lh[3], lh[3];
    float sxe_vf, sxe_l0x;
};

// The step constant of the path's arithmetic type: FP64 or its FP32 copy.
template <class T> __device__ inline T pk(double d, float f);
template <> __device__ inline float pk<float>(double, float f) { return f; }
template <> __device__ inline double pk<double>(double d, float) { return d; }

struct StepP {
    double c;
    double inv_c;       // 1 / c
    double inv_c2;      // 1 / c^2
    long long step;
    int nsp;
    int keb_exact;
    // shearing box
    double sO;          // s Omega0
    double Omega0;
    double half_nx;     // box centre
    int dys_end_i;      // floor of Dy_s(t^{n+1}) mod ny
    double dys_end_f;   // fractional part
    // expanding box
    double Lam[3];      // -(dt/2) L^{-1} dL/dt
    double keb_im[3];   // 1 / (1 - Lambda_ii)
    double keb_Lt[3];   // (1 + Lambda_ii) / (1 - Lambda_ii)
    double inv_lh[3];   // 1 / l_i(t^{n+1/2})
    double lh[3];       // l_i(t^{n+1/2})
    // shearing + expanding box: (l_1/l_2)(t^{n+1/2}) and l_1(t^n)
    double sxe_vf, sxe_l0x;
    // leaky box
    double l_esc;
    uint32_t esc_thresh;
    uint32_t seed;
    double theta_inj;
    int esc_dims;
    int* err;
    unsigned long long* counters;  // [0] escaped, [1] superluminal
    // FP32 path: fixed-point current accumulation in shared memory.  A
    // contribution v is added as round(v * fx_scale) to an int32 word; one
    // unit is worth fx_unit = 1 / fx_scale.  The range 2^31 fx_unit is 16x
    // the current of the mean density moving coherently at c, and at least
    // 512 c q_max, so a single contribution (|v| <= c q) stays below 2^22 units.
    float fx_scale;
    double fx_unit;
    StepPF f;
};

// ---- shapes --------------------------------------------------------------------
// Weights on ORD+1 consecutive grid points starting at cell + off, for a
// particle at offset o in [0,1) of that cell: node-centred ("n") or
// half-staggered ("s") quantities.
template <class T, int ORD> struct Shape;

template <class T> struct Shape<T, 1> {
    __device__ static void node(T o, int& off, T w[2]) { off = 0; w[0] = T(1) - o; w[1] = o; }
    __device__ static void stag(T o, int& off, T w[2]) {
        T f;
        if (o >= T(0.5)) { off = 0; f = o - T(0.5); } else { off = -1; f = o + T(0.5); }
        w[0] = T(1) - f; w[1] = f;
    }
    // node shape of a position x (relative to the cell origin, -1 <= x < 2) on
    // the 3-node window starting at node wb: weights (1-f, f) at floor(x) and
    // floor(x)+1, placed at window index k = floor(x) - wb (0 or 1)
    __device__ static void window(T x, int wb, T w[4]) {
        const T fl = t_floor<T>(x);
        const T f = x - fl;
        const bool k = ((int)fl - wb) != 0;
        w[0] = k ? T(0) : T(1) - f;
        w[1] = k ? T(1) - f : f;
        w[2] = k ? f : T(0);
        w[3] = T(0);
    }
};

template <class T> struct Shape<T, 2> {
    __device__ static void q3(T d, T w[3]) {
        T a = T(0.5) - d, b = T(0.5) + d;
        w[0] = T(0.5) * a * a; w[1] = T(0.75) - d * d; w[2] = T(0.5) * b * b;
    }
    __device__ static void node(T o, int& off, T w[3]) {
        T d;
        if (o >= T(0.5)) { off = 0; d = o - T(1); } else { off = -1; d = o; }
        q3(d, w);
    }
    __device__ static void stag(T o, int& off, T w[3]) { off = -1; q3(o - T(0.5), w); }
    // node shape of a position x on the 4-node window starting at node wb: the
    // three weights q3(x - n) around the nearest node n, placed at window
    // index k = n - 1 - wb (0 or 1)
    __device__ static void window(T x, int wb, T w[4]) {
        const T n = t_floor<T>(x + T(0.5));
        T q[3];
        q3(x - n, q);
        const bool k = ((int)n - 1 - wb) != 0;
        w[0] = k ? T(0) : q[0];
        w[1] = k ? q[0] : q[1];
        w[2] = k ? q[1] : q[2];
        w[3] = k ? q[2] : T(0);
    }
};

// ---- field and current accessors -------------------------------------------------
// Fields and currents are addressed by a linear index: cell (i,j,k) of an
// accessor's box is i + j*SY + k*SZ and component c adds c*SC.  The shared-
// memory boxes of a tile have compile-time strides (fixed tile shape per
// geometry), so every stencil offset is an immediate; the global padded
// arrays (loose particles) use runtime strides.

template <int G> struct TileDims {
    static constexpr int TX = tile_side(G);
    static constexpr int TY = GeomT<G>::AY ? tile_side(G) : 1;
    static constexpr int TZ = GeomT<G>::AZ ? tile_side(G) : 1;
    static constexpr int BX = TX + 4;
    static constexpr int BY = GeomT<G>::AY ? TY + 4 : 1;
    static constexpr int BZ = GeomT<G>::AZ ? TZ + 4 : 1;
    static constexpr int JX = TX + 5;
    static constexpr int JY = GeomT<G>::AY ? TY + 5 : 1;
    static constexpr int JZ = GeomT<G>::AZ ? TZ + 5 : 1;
    static constexpr int FB = BX * BY * BZ;
    static constexpr int JB = JX * JY * JZ;
};

// Shared-memory field boxes: E and B, 3 components each, [comp][bz][by][bx].
template <class T, int G> struct SmemFields {
    using D = TileDims<G>;
    static constexpr int SY = D::BX, SZ = D::BX * D::BY, SC = D::FB;
    const T* e;
    const T* b;
    __device__ T at(int comp, int idx) const { return comp < 3 ? e[comp * SC + idx] : b[(comp - 3) * SC + idx]; }
};

// Global padded fields (index = padded linear index).
template <class T> struct GlobalFields {
    const T* e;
    const T* b;
    long long SY, SZ, SC;
    __device__ T at(int comp, long long idx) const {
        return comp < 3 ? __ldg(e + comp * SC + idx) : __ldg(b + (comp - 3) * SC + idx);
    }
};

// Shared-memory current box of a tile.  FP32: one int32 fixed-point word per
// point (native integer shared atomics); values arrive pre-multiplied by the
// fixed-point scale and are rounded to the nearest unit.  Integer addition is
// exact modulo 2^32, so only the tile's final sum per point must fit (checked
// at the flush).  FP64: one double per point.
// Every add is made (no branch); trash(base) is the base that exact-zero
// contributions are sent to (see deposit): word `lane` of the box, so the
// lanes of a warp hit distinct banks.  All trash addresses lie inside the box.
template <class T, int G> struct SmemJ;

// The contribution added is a * b.  FP32 converts it to the nearest integer
// unit with the 1.5 * 2^23 trick (one FMA and one integer subtract, exact
// round-to-nearest for |a b| < 2^22 units, which the unit choice guarantees).
template <int G> struct SmemJ<float, G> {
    using D = TileDims<G>;
    static constexpr int SY = D::JX, SZ = D::JX * D::JY, SC = D::JB;
    static_assert(31 + 3 * (1 + (GeomT<G>::AY ? SY : 0) + (GeomT<G>::AZ ? SZ : 0)) < SC,
                  "trash words of the last component stay inside the box");
    uint32_t j;  // shared-window address of the box
    int tw;      // trash word: exact zeros go here (a word of the first 32)
    __device__ SmemJ(int* p, int trash_word) : j(smem_u32(p)), tw(trash_word) {}
    __device__ int trash(int) const { return tw; }
    __device__ void add(int comp, int idx, float a, float b) const {
        const int iv = __float_as_int(fmaf(a, b, 12582912.0f)) - 0x4B400000;
        red_shared(j + 4u * (uint32_t)(comp * SC + idx), iv);
    }
    // word: component offset comp * SC already added
    __device__ void add_w(int word, float a, float b) const {
        const int iv = __float_as_int(fmaf(a, b, 12582912.0f)) - 0x4B400000;
        red_shared(j + 4u * (uint32_t)word, iv);
    }
};

template <int G> struct SmemJ<double, G> {
    using D = TileDims<G>;
    static constexpr int SY = D::JX, SZ = D::JX * D::JY, SC = D::JB;
    static_assert(31 + 3 * (1 + (GeomT<G>::AY ? SY : 0) + (GeomT<G>::AZ ? SZ : 0)) < SC,
                  "trash words of the last component stay inside the box");
    uint32_t j;
    int tw;
    __device__ SmemJ(double* p, int trash_word) : j(smem_u32(p)), tw(trash_word) {}
    __device__ int trash(int) const { return tw; }
    __device__ void add(int comp, int idx, double a, double b) const {
        red_shared(j + 8u * (uint32_t)(comp * SC + idx), a * b);
    }
};

// Global padded current (loose particles).  FP32: the int32 fixed-point
// array the tiles flush into (same units and rounding as the shared box);
// FP64: doubles.
template <class T> struct GlobalJ;

template <> struct GlobalJ<float> {
    int* J;
    long long SY, SZ, SC;
    __device__ long long trash(long long base) const { return base; }  // exact zeros are skipped below
    __device__ void add(int comp, long long idx, float a, float b) const {
        const int iv = __float_as_int(fmaf(a, b, 12582912.0f)) - 0x4B400000;
        if (iv != 0) atomicAdd(J + comp * SC + idx, iv);
    }
};

template <> struct GlobalJ<double> {
    double* J;
    long long SY, SZ, SC;
    __device__ long long trash(long long base) const { return base; }
    __device__ void add(int comp, long long idx, double a, double b) const {
        const double v = a * b;
        if (v != 0.0) red_add_global(J + comp * SC + idx, v);
    }
};

// word type of the current accumulators: int32 fixed point (FP32), double (FP64)
template <class T> using JWord = typename std::conditional<sizeof(T) == 4, int, double>::type;

// ---- gather ------------------------------------------------------------------------
// cidx: linear index of the particle's cell in the accessor's box; o: offsets.
template <class T, int G, int ORD, class F, class I>
__device__ inline void gather(const F& fa, I cidx, const T o[3], T Ep[3], T Bp[3]) {
    using GT = GeomT<G>;
    constexpr int NP = ORD + 1;
    T wn[3][NP], ws[3][NP];
    int offn[3] = {0, 0, 0}, offs[3] = {0, 0, 0};
    Shape<T, ORD>::node(o[0], offn[0], wn[0]);
    Shape<T, ORD>::stag(o[0], offs[0], ws[0]);
    if (GT::AY) { Shape<T, ORD>::node(o[1], offn[1], wn[1]); Shape<T, ORD>::stag(o[1], offs[1], ws[1]); }
    if (GT::AZ) { Shape<T, ORD>::node(o[2], offn[2], wn[2]); Shape<T, ORD>::stag(o[2], offs[2], ws[2]); }
    // components: E x,y,z then B x,y,z; staggered (1) or node-centred (0) per axis
    constexpr bool ST[6][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {0, 1, 1}, {1, 0, 1}, {1, 1, 0}};
    T out[6];
#pragma unroll
    for (int comp = 0; comp < 6; ++comp) {
        const T* wx = ST[comp][0] ? ws[0] : wn[0];
        const int ox = ST[comp][0] ? offs[0] : offn[0];
        T acc = T(0);
        if (GT::AY && GT::AZ) {
            const T* wy = ST[comp][1] ? ws[1] : wn[1];
            const T* wz = ST[comp][2] ? ws[2] : wn[2];
            const I b0 = cidx + ox + (ST[comp][1] ? offs[1] : offn[1]) * fa.SY + (ST[comp][2] ? offs[2] : offn[2]) * fa.SZ;
#pragma unroll
            for (int c = 0; c < NP; ++c)
#pragma unroll
                for (int b = 0; b < NP; ++b) {
                    T row = T(0);
#pragma unroll
                    for (int a = 0; a < NP; ++a) row += wx[a] * fa.at(comp, b0 + a + b * fa.SY + c * fa.SZ);
                    acc += (wy[b] * wz[c]) * row;
                }
        } else {
            constexpr int A2 = GT::AY ? 1 : 2;  // second active axis
            const T* w2 = ST[comp][A2] ? ws[A2] : wn[A2];
            const auto s2 = A2 == 1 ? fa.SY : fa.SZ;
            const I b0 = cidx + ox + (ST[comp][A2] ? offs[A2] : offn[A2]) * s2;
#pragma unroll
            for (int b = 0; b < NP; ++b) {
                T row = T(0);
#pragma unroll
                for (int a = 0; a < NP; ++a) row += wx[a] * fa.at(comp, b0 + a + b * s2);
                acc += w2[b] * row;
            }
        }
        out[comp] = acc;
    }
    Ep[0] = out[0]; Ep[1] = out[1]; Ep[2] = out[2];
    Bp[0] = out[3]; Bp[1] = out[4]; Bp[2] = out[5];
}

// FP32 gather from the shared-memory boxes with packed two-wide FP32
// arithmetic.  E_k and B_k are staggered oppositely on every axis (E_k is
// half-staggered along k only, B_k along the other two), so with the node
// and staggered shape weights of each axis held as one pair (node, stag) --
// or its swap (stag, node) -- every weight, row and accumulator of the pair
// (E_k, B_k) is one packed register: each fused multiply-add does the work of
// two, with the rounding of the scalar form.  Same weights, stencils and
// summation order as gather().
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2swap(float2 v) { return make_float2(v.y, v.x); }

template <int ORD> struct Shape2;
template <> struct Shape2<1> {
    // (node, stag) weights of one axis at offset o, and the start offsets
    __device__ static void pair(float o, int& offn, int& offs, float2 w[2]) {
        offn = 0;
        const bool hi = o >= 0.5f;
        offs = hi ? 0 : -1;
        const float2 f = f2(o, hi ? o - 0.5f : o + 0.5f);
        w[0] = __fadd2_rn(f2(1.0f, 1.0f), f2(-f.x, -f.y));
        w[1] = f;
    }
};
template <> struct Shape2<2> {
    __device__ static void pair(float o, int& offn, int& offs, float2 w[3]) {
        const bool hi = o >= 0.5f;
        offn = hi ? 0 : -1;
        offs = -1;
        const float2 d = f2(hi ? o - 1.0f : o, o - 0.5f);
        const float2 half = f2(0.5f, 0.5f);
        const float2 a = __fadd2_rn(half, f2(-d.x, -d.y)), bb = __fadd2_rn(half, d);
        w[0] = __fmul2_rn(half, __fmul2_rn(a, a));
        w[1] = __ffma2_rn(f2(-d.x, -d.y), d, f2(0.75f, 0.75f));
        w[2] = __fmul2_rn(half, __fmul2_rn(bb, bb));
    }
};

template <int G, int ORD>
__device__ __forceinline__ void gather_packed(const SmemFields<float, G>& fa, int cidx, const float o[3], float Ep[3],
                                              float Bp[3]) {
    using GT = GeomT<G>;
    using FA = SmemFields<float, G>;
    constexpr int NP = ORD + 1;
    float2 w[3][NP];  // (node, stag) per axis
    int offn[3] = {0, 0, 0}, offs[3] = {0, 0, 0};
    Shape2<ORD>::pair(o[0], offn[0], offs[0], w[0]);
    if (GT::AY) Shape2<ORD>::pair(o[1], offn[1], offs[1], w[1]);
    if (GT::AZ) Shape2<ORD>::pair(o[2], offn[2], offs[2], w[2]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        // E_k: staggered along k (weights .y of axis k, .x elsewhere); B_k the opposite
        float2 wk[3][NP];
        int bE = cidx, bB = cidx;
        constexpr int SS[3] = {1, FA::SY, FA::SZ};
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const bool act = ax == 0 || (ax == 1 && GT::AY) || (ax == 2 && GT::AZ);
            if (!act) continue;
#pragma unroll
            for (int m = 0; m < NP; ++m) wk[ax][m] = ax == k ? f2swap(w[ax][m]) : w[ax][m];
            bE += (ax == k ? offs[ax] : offn[ax]) * SS[ax];
            bB += (ax == k ? offn[ax] : offs[ax]) * SS[ax];
        }
        float2 acc = f2(0.0f, 0.0f);
        if (GT::AY && GT::AZ) {
#pragma unroll
            for (int c = 0; c < NP; ++c)
#pragma unroll
                for (int b = 0; b < NP; ++b) {
                    const int off = b * FA::SY + c * FA::SZ;
                    float2 row = f2(0.0f, 0.0f);
#pragma unroll
                    for (int a = 0; a < NP; ++a)
                        row = __ffma2_rn(wk[0][a], f2(fa.e[k * FA::SC + bE + off + a], fa.b[k * FA::SC + bB + off + a]), row);
                    acc = __ffma2_rn(__fmul2_rn(wk[1][b], wk[2][c]), row, acc);
                }
        } else {
            constexpr int A2 = GT::AY ? 1 : 2;
            constexpr int S2 = A2 == 1 ? FA::SY : FA::SZ;
#pragma unroll
            for (int b = 0; b < NP; ++b) {
                float2 row = f2(0.0f, 0.0f);
#pragma unroll
                for (int a = 0; a < NP; ++a)
                    row = __ffma2_rn(wk[0][a], f2(fa.e[k * FA::SC + bE + b * S2 + a], fa.b[k * FA::SC + bB + b * S2 + a]), row);
                acc = __ffma2_rn(wk[A2][b], row, acc);
            }
        }
        Ep[k] = acc.x;
        Bp[k] = acc.y;
    }
}

// ---- pushers ------------------------------------------------------------------------

template <class T> __device__ inline void cross(const T a[3], const T b[3], T r[3]) {
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}
template <class T> __device__ inline T dot(const T a[3], const T b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// nu x t + (nu x t) x t, divided by 1 + t^2, times k: the rotation part of
// the Boris (k = 2) and half-Boris (k = 1) operators of Sec. 2.2.
template <class T> __device__ inline void rot(const T nu[3], const T t[3], T k_over_den, T out[3]) {
    T a[3], b[3];
    cross(nu, t, a);
    cross(a, t, b);
    out[0] = nu[0] + k_over_den * (a[0] + b[0]);
    out[1] = nu[1] + k_over_den * (a[1] + b[1]);
    out[2] = nu[2] + k_over_den * (a[2] + b[2]);
}

// Standard Boris push with gamma at u^-.
template <class T> __device__ inline void push_boris(T u[3], const T E[3], const T B[3], T qdt2m, T qdt2mc, T inv_c2) {
    T eps[3] = {qdt2m * E[0], qdt2m * E[1], qdt2m * E[2]};
    T um[3] = {u[0] + eps[0], u[1] + eps[1], u[2] + eps[2]};
    T ig = t_rsqrt<T>(T(1) + dot(um, um) * inv_c2);  // 1 / gamma^-
    T tau[3] = {qdt2mc * B[0] * ig, qdt2mc * B[1] * ig, qdt2mc * B[2] * ig};
    T up[3];
    rot(um, tau, T(2) * t_rcp<T>(T(1) + dot(tau, tau)), up);
    u[0] = up[0] + eps[0]; u[1] = up[1] + eps[1]; u[2] = up[2] + eps[2];
}

// Shearing-box (KSB-OA) push of Sec. 2.2.  xc: x^n from the box centre.
template <class T>
__device__ inline void push_ksb(T u[3], const T E[3], const T B[3], T qdt2m, T qdt2mc, T inv_c, T inv_c2, T sO, T Om,
                                T xc) {
    T eps[3] = {qdt2m * E[0], qdt2m * E[1], qdt2m * E[2]};
    T um[3] = {u[0] + eps[0], u[1] + eps[1], u[2] + eps[2]};
    T a1 = sO * T(0.5);
    T a2 = sO * xc * inv_c;
    const T ic2 = inv_c2;
    // gbar: root >= 1 of g^3 - A g - C = 0 (the Lorentz-factor relation of Sec. 2.2)
    T u2 = dot(um, um), ue = dot(um, eps);
    T A = T(1) + (u2 + T(2) * a1 * um[0] * um[1]) * ic2;
    T Cc = T(2) * a2 * ue * um[1] * ic2;
    const T g2m = T(1) + u2 * ic2;  // (gamma^-)^2
    const T igm = t_rsqrt<T>(g2m);
    const T gm = g2m * igm;
    T g = gm + (a1 * um[0] * um[1] * gm + a2 * ue * um[1]) * ic2 * (igm * igm);
    // Newton: converged for FP64, two corrections for FP32 (quadratic convergence
    // from an O(Omega0^2)-accurate start)
    const int NIT = sizeof(T) == 8 ? 8 : 2;
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
        T f = (g * g - A) * g - Cc;
        T df = T(3) * g * g - A;
        g -= sizeof(T) == 8 ? f / df : f * t_rcp<T>(df);
    }
    T ig = t_rcp<T>(g);
    const T igc = ig * inv_c;
    T et[3] = {eps[0] * igc, eps[1] * igc, eps[2] * igc};
    T tt[3] = {qdt2mc * B[0] * ig, qdt2mc * B[1] * ig, qdt2mc * B[2] * ig + Om};
    T den = t_rcp<T>(T(1) + dot(tt, tt));
    T S2[3] = {a1 + a2 * et[0], a2 * et[1], a2 * et[2]};
    // R(e_y) and g = S2 . R(e_y)
    T ey[3] = {T(0), T(1), T(0)}, Rey[3];
    rot(ey, tt, den, Rey);
    T gg = dot(S2, Rey);
    // w = B(u-) + R(S u-) ; S v = (S2.v) e_y, so R(S v) = (S2.v) R(e_y)
    T w[3];
    rot(um, tt, T(2) * den, w);
    T su = dot(S2, um);
    w[0] += su * Rey[0]; w[1] += su * Rey[1]; w[2] += su * Rey[2];
    T sw = dot(S2, w) * t_rcp<T>(T(1) - gg);
    u[0] = w[0] + sw * Rey[0] + eps[0];
    u[1] = w[1] + sw * Rey[1] + eps[1];
    u[2] = w[2] + sw * Rey[2] + eps[2];
}

// Expanding-box modified Boris push of Sec. 3.2 (diagonal Lambda), or the
// direct 3x3 solve of its defining equation when exact != 0.
template <class T>
__device__ inline void push_keb(T u[3], const T E[3], const T B[3], T qdt2m, T qdt2mc, T inv_c2, const T Lam[3],
                                const T im[3], const T Lt[3], bool exact) {
    T eps[3] = {qdt2m * E[0], qdt2m * E[1], qdt2m * E[2]};
    T um[3] = {u[0] + eps[0], u[1] + eps[1], u[2] + eps[2]};
    T lu[3] = {(T(1) + Lam[0]) * um[0], (T(1) + Lam[1]) * um[1], (T(1) + Lam[2]) * um[2]};
    T ig = t_rsqrt<T>(T(1) + dot(lu, lu) * inv_c2);  // 1 / gbar
    T tau[3] = {qdt2mc * B[0] * ig, qdt2mc * B[1] * ig, qdt2mc * B[2] * ig};
    T up[3];
    if (!exact) {
        T tt[3], a[3], ax[3], bx[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            tt[i] = tau[i] * im[i];
            a[i] = (T(1) + Lt[i]) * um[i];
        }
        T den = t_rcp<T>(T(1) + dot(tt, tt));
        cross(a, tt, ax);
        cross(ax, tt, bx);
#pragma unroll
        for (int i = 0; i < 3; ++i) up[i] = Lt[i] * um[i] + (ax[i] + bx[i]) * den;
    } else {
        // (I - Lambda - T) u+ = (I + Lambda + T) u-, T v = v x tau
        T r[3];
        cross(um, tau, r);
#pragma unroll
        for (int i = 0; i < 3; ++i) r[i] += (T(1) + Lam[i]) * um[i];
        T M[3][3] = {{T(1) - Lam[0], -tau[2], tau[1]}, {tau[2], T(1) - Lam[1], -tau[0]}, {-tau[1], tau[0], T(1) - Lam[2]}};
        T det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
        T id = T(1) / det;
#pragma unroll
        for (int col = 0; col < 3; ++col) {
            T A_[3][3];
#pragma unroll
            for (int rr = 0; rr < 3; ++rr)
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) A_[rr][cc] = (cc == col) ? r[rr] : M[rr][cc];
            T d = A_[0][0] * (A_[1][1] * A_[2][2] - A_[1][2] * A_[2][1]) - A_[0][1] * (A_[1][0] * A_[2][2] - A_[1][2] * A_[2][0]) +
                  A_[0][2] * (A_[1][0] * A_[2][1] - A_[1][1] * A_[2][0]);
            up[col] = d * id;
        }
    }
    u[0] = up[0] + eps[0]; u[1] = up[1] + eps[1]; u[2] = up[2] + eps[2];
}

// Shearing + expanding box push: the discrete momentum equation of Sec. 2.2
// with the expansion term of Sec. 3.2 added,
//   (I - Lambda - T - S) u+ = (I + Lambda + T + S) u-,
// T v = v x tt, S v = (S_2 . v) e_y, gbar from the Lambda-corrected cubic
// gbar^3 - A gbar - C = 0 (A with ((I + Lambda) u-)^2), solved by Newton from
// the expanding box's Lorentz factor; the 3x3 system by Cramer's rule.  xc:
// the physical radial coordinate l_1 (xi_x - nx/2) at t^n.
template <class T>
__device__ inline void push_sxe(T u[3], const T E[3], const T B[3], T qdt2m, T qdt2mc, T inv_c, T inv_c2, T sO, T Om,
                                T xc, const T Lam[3]) {
    T eps[3] = {qdt2m * E[0], qdt2m * E[1], qdt2m * E[2]};
    T um[3] = {u[0] + eps[0], u[1] + eps[1], u[2] + eps[2]};
    const T a1 = sO * T(0.5), a2 = sO * xc * inv_c;
    T lu[3] = {(T(1) + Lam[0]) * um[0], (T(1) + Lam[1]) * um[1], (T(1) + Lam[2]) * um[2]};
    const T l2 = dot(lu, lu) * inv_c2;
    const T A = T(1) + l2 + T(2) * a1 * um[0] * um[1] * inv_c2;
    const T Cc = T(2) * a2 * dot(um, eps) * um[1] * inv_c2;
    T g = t_sqrt<T>(T(1) + l2);
    const int NIT = sizeof(T) == 8 ? 8 : 2;
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
        T f = (g * g - A) * g - Cc;
        T df = T(3) * g * g - A;
        g -= sizeof(T) == 8 ? f / df : f * t_rcp<T>(df);
    }
    const T ig = t_rcp<T>(g), igc = ig * inv_c;
    const T tt[3] = {qdt2mc * B[0] * ig, qdt2mc * B[1] * ig, qdt2mc * B[2] * ig + Om};
    const T S2[3] = {a1 + a2 * eps[0] * igc, a2 * eps[1] * igc, a2 * eps[2] * igc};
    // K = Lambda + T + S: (K v)_r = Lambda_r v_r + (v x tt)_r + [r = y] S_2 . v
    T K[3][3] = {{Lam[0], tt[2], -tt[1]}, {-tt[2], Lam[1], tt[0]}, {tt[1], -tt[0], Lam[2]}};
    K[1][0] += S2[0];
    K[1][1] += S2[1];
    K[1][2] += S2[2];
    T M[3][3], r[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        r[i] = um[i] + K[i][0] * um[0] + K[i][1] * um[1] + K[i][2] * um[2];
#pragma unroll
        for (int k = 0; k < 3; ++k) M[i][k] = (i == k ? T(1) : T(0)) - K[i][k];
    }
    const T c00 = M[1][1] * M[2][2] - M[1][2] * M[2][1];
    const T c01 = M[1][2] * M[2][0] - M[1][0] * M[2][2];
    const T c02 = M[1][0] * M[2][1] - M[1][1] * M[2][0];
    const T det = M[0][0] * c00 + M[0][1] * c01 + M[0][2] * c02;
    const T idet = sizeof(T) == 8 ? T(1) / det : t_rcp<T>(det);
    // Cramer: column k replaced by r
    const T x0 = r[0] * c00 + M[0][1] * (M[1][2] * r[2] - r[1] * M[2][2]) + M[0][2] * (r[1] * M[2][1] - M[1][1] * r[2]);
    const T x1 = M[0][0] * (r[1] * M[2][2] - M[1][2] * r[2]) + r[0] * c01 + M[0][2] * (M[1][0] * r[2] - r[1] * M[2][0]);
    const T x2 = M[0][0] * (M[1][1] * r[2] - r[1] * M[2][1]) + M[0][1] * (r[1] * M[2][0] - M[1][0] * r[2]) + r[0] * c02;
    u[0] = x0 * idet + eps[0];
    u[1] = x1 * idet + eps[1];
    u[2] = x2 * idet + eps[2];
}

// ---- charge-conserving deposit (Esirkepov) -------------------------------------------
// The particle moves from x0 = o (offsets in its start cell) to x1 = o + d,
// |d| < 1 per axis.  With S0, S1 the node shapes on a window of ORD+2 nodes
// starting at node wb (relative to the start cell), W_x = dS_x * F_yz with
// F_yz = S0y S0z + dSy S0z / 2 + S0y dSz / 2 + dSy dSz / 3, so the running
// sum J_x(l + 1/2) = -q sum_{l' <= l} W_x(l') = -q CS_x(l) F_yz: an outer
// product of ORD+1 running sums and (ORD+2)^2 weights per component.  On the
// 2D ignorable axis the current is q v F of the two active axes.  qs is the
// charge times the accumulator's value scale; cidx the start cell's linear
// index in the accumulator's box.
// First window node of axis a relative to the start cell: the lowest node
// either shape touches (order 1: floor of the lower end point; order 2: one
// below the lower nearest node).
template <class T, int ORD> __device__ inline int window_base(T o, T x1) {
    if (ORD == 1) return x1 < T(0) ? -1 : 0;
    const int n0 = o >= T(0.5) ? 1 : 0;
    const int n1 = (int)t_floor<T>(x1 + T(0.5));
    return (n0 < n1 ? n0 : n1) - 1;
}

// The last window node of an axis (index ORD+1) carries shape weight only when
// the particle changes its nearest node (order 2) or its cell (order 1) on
// that axis ("crosses"); otherwise every contribution that involves it is an
// exact zero: the weights there are exactly 0, and the running sum that
// reaches it is set to exactly 0 (the shape sums of both end points are 1, so
// only rounding is dropped).  Such contributions are not added where they
// belong: they go, unconditionally, to the accumulator's trash base, which
// for the shared box is a word of the box chosen by lane (distinct banks
// across a warp; adding an exact zero changes nothing).  So no add is skipped
// by a branch.  The global accumulator skips zeros itself.
template <class T, int G, int ORD, class JA, class I>
__device__ inline void deposit(const JA& ja, I cidx, const T o[3], const T d[3], T qs) {
    using GT = GeomT<G>;
    constexpr int NW = ORD + 2;  // window nodes
    T S0[3][4], DS[3][4], CS[3][4];
    int wb[3] = {0, 0, 0};
    int crm = 0;  // bit a: the particle crosses on axis a
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if ((a == 1 && !GT::AY) || (a == 2 && !GT::AZ)) continue;
        const T x1 = o[a] + d[a];
        bool cr;
        if (ORD == 1) {
            const int f1 = (int)t_floor<T>(x1);
            cr = f1 != 0;
            wb[a] = f1 < 0 ? -1 : 0;
        } else {
            const int n0 = o[a] >= T(0.5) ? 1 : 0;
            const int n1 = (int)t_floor<T>(x1 + T(0.5));
            cr = n0 != n1;
            wb[a] = (n0 < n1 ? n0 : n1) - 1;
        }
        crm |= cr ? (1 << a) : 0;
        T S1[4];
        Shape<T, ORD>::window(o[a], wb[a], S0[a]);
        Shape<T, ORD>::window(x1, wb[a], S1);
        T run = T(0);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            DS[a][m] = S1[m] - S0[a][m];
            run += DS[a][m];
            CS[a][m] = -qs * run;
        }
        if (!cr) CS[a][NW - 2] = T(0);
    }
    // F_ab[m][n] = S0a[m] S0b[n] + dSa[m] S0b[n]/2 + S0a[m] dSb[n]/2 + dSa[m] dSb[n]/3
    //            = S0a[m] A_b[n] + dSa[m] Q_b[n],  A = S0 + dS/2,  Q = S0/2 + dS/3
    const T third = T(1) / T(3);
    T A[3][4], Q[3][4];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            A[a][m] = S0[a][m] + T(0.5) * DS[a][m];
            Q[a][m] = T(0.5) * S0[a][m] + third * DS[a][m];
        }
    const I base = cidx + wb[0] + wb[1] * ja.SY + wb[2] * ja.SZ;
    // bs[k]: base of the adds that touch the last node on the axes of bit set k
    const I trash = ja.trash(base);
    I bs[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) bs[k] = (k & ~crm) ? trash : base;
    constexpr int LX = NW - 2, LN = NW - 1;  // last current index, last node index
    if (GT::AY && GT::AZ) {
        // The outermost loop of each component stays rolled: this full-window
        // path runs only for the queued crossing particles, and unrolled it
        // would crowd the particle loop out of the instruction cache.  Values
        // indexed by the rolled counter are picked by selects (an indexed
        // register array would go to local memory).
        auto pick = [](const T* v, int i) -> T { return i == 0 ? v[0] : (i == 1 ? v[1] : (i == 2 ? v[2] : v[3])); };
#pragma unroll 1
        for (int n = 0; n < NW; ++n) {
            const T az = pick(A[2], n), qz = pick(Q[2], n);
            const I noff = (I)n * ja.SZ;
            const bool nl = n == LN;
#pragma unroll
            for (int m = 0; m < NW; ++m) {
                const T fyz = S0[1][m] * az + DS[1][m] * qz;
#pragma unroll
                for (int l = 0; l < NW - 1; ++l) {
                    const int kl = (l == LX ? 1 : 0) | (m == LN ? 2 : 0);
                    const I bb = nl ? bs[kl | 4] : bs[kl];
                    ja.add(0, bb + noff + l + m * ja.SY, CS[0][l], fyz);
                }
            }
        }
#pragma unroll 1
        for (int n = 0; n < NW; ++n) {
            const T az = pick(A[2], n), qz = pick(Q[2], n);
            const I noff = (I)n * ja.SZ;
            const bool nl = n == LN;
#pragma unroll
            for (int l = 0; l < NW; ++l) {
                const T fxz = S0[0][l] * az + DS[0][l] * qz;
#pragma unroll
                for (int m = 0; m < NW - 1; ++m) {
                    const int kl = (l == LN ? 1 : 0) | (m == LX ? 2 : 0);
                    const I bb = nl ? bs[kl | 4] : bs[kl];
                    ja.add(1, bb + noff + l + m * ja.SY, CS[1][m], fxz);
                }
            }
        }
#pragma unroll 1
        for (int m = 0; m < NW; ++m) {
            const T ay = pick(A[1], m), qy = pick(Q[1], m);
            const I moff = (I)m * ja.SY;
            const bool ml = m == LN;
#pragma unroll
            for (int l = 0; l < NW; ++l) {
                const T fxy = S0[0][l] * ay + DS[0][l] * qy;
#pragma unroll
                for (int n = 0; n < NW - 1; ++n) {
                    const int kl = (l == LN ? 1 : 0) | (n == LX ? 4 : 0);
                    const I bb = ml ? bs[kl | 2] : bs[kl];
                    ja.add(2, bb + moff + l + n * ja.SZ, CS[2][n], fxy);
                }
            }
        }
    } else {
        constexpr int A2 = GT::AY ? 1 : 2;  // second active axis
        constexpr int IG = GT::AY ? 2 : 1;  // ignorable axis
        constexpr int C2 = GT::AY ? 1 : 2;  // current component along A2
        constexpr int B2 = 1 << A2;         // crossing bit of A2
        const auto s2 = A2 == 1 ? ja.SY : ja.SZ;
#pragma unroll
        for (int m = 0; m < NW; ++m) {
#pragma unroll
            for (int l = 0; l < NW - 1; ++l) {
                const int k = (l == LX ? 1 : 0) | (m == LN ? B2 : 0);
                ja.add(0, bs[k] + l + m * s2, CS[0][l], A[A2][m]);
            }
        }
#pragma unroll
        for (int l = 0; l < NW; ++l) {
#pragma unroll
            for (int m = 0; m < NW - 1; ++m) {
                const int k = (l == LN ? 1 : 0) | (m == LX ? B2 : 0);
                ja.add(C2, bs[k] + l + m * s2, CS[A2][m], A[0][l]);
            }
        }
        // out-of-plane component: q v_ign F(x, a2)
        const T qv = qs * d[IG];
#pragma unroll
        for (int m = 0; m < NW; ++m)
#pragma unroll
            for (int l = 0; l < NW; ++l) {
                const int k = (l == LN ? 1 : 0) | (m == LN ? B2 : 0);
                ja.add(IG, bs[k] + l + m * s2, qv, S0[0][l] * A[A2][m] + DS[0][l] * Q[A2][m]);
            }
    }
}

// Base word of the core window of a particle that crosses no boundary: its
// cell (order 1), or the node below its nearest node (order 2), per axis.
template <class T, int G, int ORD, class I, class S>
__device__ __forceinline__ I core_base(I cidx, const T o[3], S sy, S sz) {
    using GT = GeomT<G>;
    if (ORD == 1) return cidx;
    I b = cidx - (o[0] >= T(0.5) ? 0 : 1);
    if (GT::AY) b -= (o[1] >= T(0.5) ? 0 : 1) * sy;
    if (GT::AZ) b -= (o[2] >= T(0.5) ? 0 : 1) * sz;
    return b;
}

// Core deposit: the part of the current of a particle that crosses no
// boundary (order 2: keeps its nearest node, order 1: keeps its cell, on every
// axis), on the window of ORD+1 nodes that holds both of its shapes: (ORD)
// running sums times (ORD+1)^2 weights per component.  It equals deposit() for
// such a particle (the words deposit() adds beyond this window are exact
// zeros).  A crossing particle passes cross = true: its contributions are set
// to exact zeros and sent to the trash base, and deposit() must be called for
// it separately.
template <class T, int G, int ORD, class JA, class I>
__device__ inline void deposit_core(const JA& ja, I cidx, const T o[3], const T d[3], T qs, bool cross) {
    using GT = GeomT<G>;
    constexpr int NC = ORD + 1;  // core window nodes
    const T qz = cross ? T(0) : qs;
    T S0[3][3], DS[3][3], CS[3][2];
    int wb[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if ((a == 1 && !GT::AY) || (a == 2 && !GT::AZ)) continue;
        const T x1 = o[a] + d[a];
        wb[a] = ORD == 1 ? 0 : (o[a] >= T(0.5) ? 0 : -1);  // start node (non-crossing particle)
        T w0[4], w1[4];
        Shape<T, ORD>::window(o[a], wb[a], w0);
        Shape<T, ORD>::window(x1, wb[a], w1);
        T run = T(0);
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            S0[a][m] = w0[m];
            DS[a][m] = w1[m] - w0[m];
            run += DS[a][m];
            if (m < NC - 1) CS[a][m] = -qz * run;
        }
    }
    const T third = T(1) / T(3);
    T A[3][3], Q[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            A[a][m] = S0[a][m] + T(0.5) * DS[a][m];
            Q[a][m] = T(0.5) * S0[a][m] + third * DS[a][m];
        }
    const I b = cross ? ja.trash(cidx) : core_base<T, G, ORD>(cidx, o, ja.SY, ja.SZ);
    if (GT::AY && GT::AZ) {
#pragma unroll
        for (int n = 0; n < NC; ++n)
#pragma unroll
            for (int m = 0; m < NC; ++m) {
                const T fyz = S0[1][m] * A[2][n] + DS[1][m] * Q[2][n];
#pragma unroll
                for (int l = 0; l < NC - 1; ++l) ja.add(0, b + l + m * ja.SY + n * ja.SZ, CS[0][l], fyz);
            }
#pragma unroll
        for (int n = 0; n < NC; ++n)
#pragma unroll
            for (int l = 0; l < NC; ++l) {
                const T fxz = S0[0][l] * A[2][n] + DS[0][l] * Q[2][n];
#pragma unroll
                for (int m = 0; m < NC - 1; ++m) ja.add(1, b + l + m * ja.SY + n * ja.SZ, CS[1][m], fxz);
            }
#pragma unroll
        for (int m = 0; m < NC; ++m)
#pragma unroll
            for (int l = 0; l < NC; ++l) {
                const T fxy = S0[0][l] * A[1][m] + DS[0][l] * Q[1][m];
#pragma unroll
                for (int n = 0; n < NC - 1; ++n) ja.add(2, b + l + m * ja.SY + n * ja.SZ, CS[2][n], fxy);
            }
    } else {
        constexpr int A2 = GT::AY ? 1 : 2;
        constexpr int IG = GT::AY ? 2 : 1;
        constexpr int C2 = GT::AY ? 1 : 2;
        const auto s2 = A2 == 1 ? ja.SY : ja.SZ;
#pragma unroll
        for (int m = 0; m < NC; ++m)
#pragma unroll
            for (int l = 0; l < NC - 1; ++l) ja.add(0, b + l + m * s2, CS[0][l], A[A2][m]);
#pragma unroll
        for (int l = 0; l < NC; ++l)
#pragma unroll
            for (int m = 0; m < NC - 1; ++m) ja.add(C2, b + l + m * s2, CS[A2][m], A[0][l]);
        const T qv = qz * d[IG];
#pragma unroll
        for (int m = 0; m < NC; ++m)
#pragma unroll
            for (int l = 0; l < NC; ++l) ja.add(IG, b + l + m * s2, qv, S0[0][l] * A[A2][m] + DS[0][l] * Q[A2][m]);
    }
}

// Does the move o -> o + d cross a boundary on some active axis (see deposit_core)?
template <class T, int G, int ORD> __device__ inline bool crosses(const T o[3], const T d[3]) {
    using GT = GeomT<G>;
    bool c = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if ((a == 1 && !GT::AY) || (a == 2 && !GT::AZ)) continue;
        const T x1 = o[a] + d[a];
        if (ORD == 1) c |= t_floor<T>(x1) != T(0);
        else c |= t_floor<T>(x1 + T(0.5)) != (o[a] >= T(0.5) ? T(1) : T(0));
    }
    return c;
}

// Bit a set: the move o -> o + d crosses a boundary on axis a (see deposit_core).
template <class T, int G, int ORD> __device__ inline int cross_mask(const T o[3], const T d[3]) {
    using GT = GeomT<G>;
    int m = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if ((a == 1 && !GT::AY) || (a == 2 && !GT::AZ)) continue;
        const T x1 = o[a] + d[a];
        bool c;
        if (ORD == 1) c = t_floor<T>(x1) != T(0);
        else c = t_floor<T>(x1 + T(0.5)) != (o[a] >= T(0.5) ? T(1) : T(0));
        m |= c ? (1 << a) : 0;
    }
    return m;
}

// 3D deposit of a particle that crosses on axis a only (it keeps its nearest
// node, order 2, or its cell, order 1, on the other two).  Its current lives
// on the ORD+2 window nodes along a and the ORD+1 core nodes along the other
// axes: (ORD+1)^3 + 2 ORD (ORD+2)(ORD+1) adds (order 2: 27 + 24 + 24 = 75,
// against the full window's 144, whose other adds are exact zeros for such a
// particle).  The axes are taken in the cyclic order (a, a+1, a+2), with the
// strides and component offsets picked per lane.  Same Esirkepov weights as
// deposit(): F_bc = S0_b A_c + dS_b Q_c, symmetric in b and c.
template <class T, int ORD, class JA>
__device__ inline void deposit_1axis(const JA& ja, int cidx, const T o[3], const T d[3], T qs, int a) {
    constexpr int NW = ORD + 2, NC = ORD + 1;
    const int b = a == 2 ? 0 : a + 1, c = a == 0 ? 2 : a - 1;
    auto pick3 = [](const T* v, int i) -> T { return i == 0 ? v[0] : (i == 1 ? v[1] : v[2]); };
    auto stride = [](int i) -> int { return i == 0 ? 1 : (i == 1 ? JA::SY : JA::SZ); };
    const T oa = pick3(o, a), ob = pick3(o, b), oc = pick3(o, c);
    const T xa1 = oa + pick3(d, a), xb1 = ob + pick3(d, b), xc1 = oc + pick3(d, c);
    const int sa = stride(a), sb = stride(b), sc = stride(c);
    // axis a: the window of the full deposit
    const int wba = window_base<T, ORD>(oa, xa1);
    T S0a[4], S1a[4], DSa[4], CSa[NW - 1];
    Shape<T, ORD>::window(oa, wba, S0a);
    Shape<T, ORD>::window(xa1, wba, S1a);
    {
        T run = T(0);
#pragma unroll
        for (int m = 0; m < NW; ++m) {
            DSa[m] = S1a[m] - S0a[m];
            run += DSa[m];
            if (m < NW - 1) CSa[m] = -qs * run;
        }
    }
    // axes b and c: the core windows
    const int wbb = ORD == 1 ? 0 : (ob >= T(0.5) ? 0 : -1);
    const int wbc = ORD == 1 ? 0 : (oc >= T(0.5) ? 0 : -1);
    T S0b[NC], DSb[NC], CSb[NC - 1], S0c[NC], DSc[NC], CSc[NC - 1];
    {
        T w0[4], w1[4];
        Shape<T, ORD>::window(ob, wbb, w0);
        Shape<T, ORD>::window(xb1, wbb, w1);
        T run = T(0);
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            S0b[m] = w0[m];
            DSb[m] = w1[m] - w0[m];
            run += DSb[m];
            if (m < NC - 1) CSb[m] = -qs * run;
        }
        Shape<T, ORD>::window(oc, wbc, w0);
        Shape<T, ORD>::window(xc1, wbc, w1);
        run = T(0);
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            S0c[m] = w0[m];
            DSc[m] = w1[m] - w0[m];
            run += DSc[m];
            if (m < NC - 1) CSc[m] = -qs * run;
        }
    }
    const T third = T(1) / T(3);
    T Aa[NW], Qa[NW], Ab[NC], Qb[NC], Ac[NC], Qc[NC];
#pragma unroll
    for (int m = 0; m < NW; ++m) {
        Aa[m] = S0a[m] + T(0.5) * DSa[m];
        Qa[m] = T(0.5) * S0a[m] + third * DSa[m];
    }
#pragma unroll
    for (int m = 0; m < NC; ++m) {
        Ab[m] = S0b[m] + T(0.5) * DSb[m];
        Qb[m] = T(0.5) * S0b[m] + third * DSb[m];
        Ac[m] = S0c[m] + T(0.5) * DSc[m];
        Qc[m] = T(0.5) * S0c[m] + third * DSc[m];
    }
    const int base = cidx + wba * sa + wbb * sb + wbc * sc;
    const int wa = base + a * JA::SC, wb = base + b * JA::SC, wc = base + c * JA::SC;
    // The outermost loop of each component stays rolled (instruction cache, as
    // in deposit()); the values it indexes are picked by selects.
    // (windows of NC = ORD+1 nodes on b and c, NW = ORD+2 on a)
    auto pickc = [](const T* v, int i) -> T { return NC == 2 ? (i == 0 ? v[0] : v[NC - 1]) : (i == 0 ? v[0] : (i == 1 ? v[1] : v[NC - 1])); };
    auto pickw = [](const T* v, int i) -> T {
        return NW == 3 ? (i == 0 ? v[0] : (i == 1 ? v[1] : v[NW - 1])) : (i == 0 ? v[0] : (i == 1 ? v[1] : (i == 2 ? v[2] : v[NW - 1])));
    };
    // J_a: running sums along a times F_bc
#pragma unroll 1
    for (int m = 0; m < NC; ++m) {
        const T s0 = pickc(S0b, m), ds = pickc(DSb, m);
        const int mo = wa + m * sb;
#pragma unroll
        for (int n = 0; n < NC; ++n) {
            const T f = s0 * Ac[n] + ds * Qc[n];
            const int off = mo + n * sc;
#pragma unroll
            for (int l = 0; l < NW - 1; ++l) ja.add_w(off + l * sa, CSa[l], f);
        }
    }
    // J_b: running sums along b times F_ac
#pragma unroll 1
    for (int l = 0; l < NW; ++l) {
        const T s0 = pickw(S0a, l), ds = pickw(DSa, l);
        const int lo = wb + l * sa;
#pragma unroll
        for (int n = 0; n < NC; ++n) {
            const T f = s0 * Ac[n] + ds * Qc[n];
            const int off = lo + n * sc;
#pragma unroll
            for (int m = 0; m < NC - 1; ++m) ja.add_w(off + m * sb, CSb[m], f);
        }
    }
    // J_c: running sums along c times F_ab
#pragma unroll 1
    for (int l = 0; l < NW; ++l) {
        const T s0 = pickw(S0a, l), ds = pickw(DSa, l);
        const int lo = wc + l * sa;
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            const T f = s0 * Ab[m] + ds * Qb[m];
            const int off = lo + m * sb;
#pragma unroll
            for (int n = 0; n < NC - 1; ++n) ja.add_w(off + n * sc, CSc[n], f);
        }
    }
}

// ---- one particle ---------------------------------------------------------------------

template <class T> struct Particle {
    int ci, cj, ck;  // physical cell
    T o[3];
    T u[3];
    uint32_t id;
    T dr[3];
};

template <class T, int G> __device__ inline void load_particle(const PView<T>& v, long long s, bool leaky, Particle<T>& p) {
    using GT = GeomT<G>;
    CellPack<G>::unpack(v.cell[s], p.ci, p.cj, p.ck);
    p.o[0] = v.o[0][s];
    p.o[1] = GT::AY ? v.o[1][s] : T(0.5);
    p.o[2] = GT::AZ ? v.o[GT::AY ? 2 : 1][s] : T(0.5);
    p.u[0] = v.u[0][s]; p.u[1] = v.u[1][s]; p.u[2] = v.u[2][s];
    p.id = v.id[s];
    if (leaky) { p.dr[0] = v.dr[0][s]; p.dr[1] = v.dr[1][s]; p.dr[2] = v.dr[2][s]; }
    else { p.dr[0] = p.dr[1] = p.dr[2] = T(0); }
}

template <class T, int G> __device__ inline void store_particle(const PView<T>& v, long long s, bool leaky, const Particle<T>& p) {
    using GT = GeomT<G>;
    v.cell[s] = CellPack<G>::pack(p.ci, p.cj, p.ck);
    v.o[0][s] = p.o[0];
    if (GT::AY) v.o[1][s] = p.o[1];
    if (GT::AZ) v.o[GT::AY ? 2 : 1][s] = p.o[2];
    v.u[0][s] = p.u[0]; v.u[1][s] = p.u[1]; v.u[2][s] = p.u[2];
    v.id[s] = p.id;
    if (leaky) { v.dr[0][s] = p.dr[0]; v.dr[1][s] = p.dr[1]; v.dr[2][s] = p.dr[2]; }
}

// Normalise offset o (possibly outside [0,1)) into [0,1), moving the cell.
template <class T> __device__ inline void renorm(T& o, int& c) {
    T f = t_floor<T>(o);
    int df = (int)f;
    o -= f;
    if (o >= T(1)) { o = T(0); df += 1; }  // -tiny + 1 rounded up to 1
    c += df;
}

// Gather and push one particle: p.u becomes u^{n+1/2}; d is the displacement
// of the position update in cells (comoving for the expanding box; for the
// shearing box the comoving move x^n -> x' of Sec. 2.2).  FA: field accessor;
// fidx: the start cell's linear index in the accessor's box.
template <class T, int G, int ORD, int PUSH, class FA, class I>
__device__ inline void push_particle(Particle<T>& p, const FA& fa, I fidx, const SpecStep<T>& S, const StepP& P,
                                     T d[3]) {
    T E[3], B[3];
    if constexpr (std::is_same<FA, SmemFields<float, G>>::value) gather_packed<G, ORD>(fa, fidx, p.o, E, B);
    else gather<T, G, ORD>(fa, fidx, p.o, E, B);
    const T inv_c2 = pk<T>(P.inv_c2, P.f.inv_c2);
    if (PUSH == PUSH_KSB) {
        const T xc0 = (T(p.ci) - pk<T>(P.half_nx, P.f.half_nx)) + p.o[0];  // exact: integer and half-integer
        push_ksb<T>(p.u, E, B, S.qdt2m, S.qdt2mc, pk<T>(P.inv_c, P.f.inv_c), inv_c2, pk<T>(P.sO, P.f.sO),
                    pk<T>(P.Omega0, P.f.Omega0), xc0);
    } else if (PUSH == PUSH_SXE) {
        const T xi0 = (T(p.ci) - pk<T>(P.half_nx, P.f.half_nx)) + p.o[0];
        const T Lam[3] = {pk<T>(P.Lam[0], P.f.Lam[0]), pk<T>(P.Lam[1], P.f.Lam[1]), pk<T>(P.Lam[2], P.f.Lam[2])};
        push_sxe<T>(p.u, E, B, S.qdt2m, S.qdt2mc, pk<T>(P.inv_c, P.f.inv_c), inv_c2, pk<T>(P.sO, P.f.sO),
                    pk<T>(P.Omega0, P.f.Omega0), xi0 * pk<T>(P.sxe_l0x, P.f.sxe_l0x), Lam);
    } else if (PUSH == PUSH_KEB) {
        const T Lam[3] = {pk<T>(P.Lam[0], P.f.Lam[0]), pk<T>(P.Lam[1], P.f.Lam[1]), pk<T>(P.Lam[2], P.f.Lam[2])};
        const T im[3] = {pk<T>(P.keb_im[0], P.f.im[0]), pk<T>(P.keb_im[1], P.f.im[1]), pk<T>(P.keb_im[2], P.f.im[2])};
        const T Lt[3] = {pk<T>(P.keb_Lt[0], P.f.Lt[0]), pk<T>(P.keb_Lt[1], P.f.Lt[1]), pk<T>(P.keb_Lt[2], P.f.Lt[2])};
        push_keb<T>(p.u, E, B, S.qdt2m, S.qdt2mc, inv_c2, Lam, im, Lt, P.keb_exact != 0);
    } else {
        push_boris<T>(p.u, E, B, S.qdt2m, S.qdt2mc, inv_c2);
    }
    T ig = t_rsqrt<T>(T(1) + dot(p.u, p.u) * inv_c2);  // 1 / gamma^{n+1/2}
    d[0] = p.u[0] * ig; d[1] = p.u[1] * ig; d[2] = p.u[2] * ig;
    if (PUSH == PUSH_KEB || PUSH == PUSH_SXE) {
        d[0] *= pk<T>(P.inv_lh[0], P.f.inv_lh[0]);
        d[1] *= pk<T>(P.inv_lh[1], P.f.inv_lh[1]);
        d[2] *= pk<T>(P.inv_lh[2], P.f.inv_lh[2]);
    }
    if (!(d[0] == d[0]) || !(d[1] == d[1]) || !(d[2] == d[2])) {
        atomicOr(P.err, ERRB_NONFINITE);
        d[0] = d[1] = d[2] = T(0);
    }
}

// Move a pushed particle by d (p still holds its start position): the leaky
// displacement, the shearing-box second stage and superluminal count, the
// cell update, periodic and shearing-periodic wraps, and the leaky escape
// and reinjection.  Afterwards p holds the particle at t^{n+1}.
template <class T, int G, int PUSH, int ESC>
__device__ inline void move_particle(Particle<T>& p, const T d[3], const StepP& P, const Grid& g) {
    using GT = GeomT<G>;
    if (ESC == ESC_DISP) { p.dr[0] += d[0]; p.dr[1] += d[1]; p.dr[2] += d[2]; }
    T nx_ = p.o[0] + d[0];
    T ny_ = p.o[1] + d[1];
    T nz_ = p.o[2] + d[2];
    if (PUSH == PUSH_KSB) {
        // x^{n+1} = x' - s Omega0 (x' + x^n)/2 dt e_y (Sec. 2.2)
        const T c = pk<T>(P.c, P.f.c);
        const T sO = pk<T>(P.sO, P.f.sO);
        const T half_nx = pk<T>(P.half_nx, P.f.half_nx);
        const T xc0 = (T(p.ci) - half_nx) + p.o[0];
        const T xc1 = (T(p.ci) - half_nx) + nx_;
        const T vs = sO * (xc1 + xc0) * T(0.5);
        {
            // superluminal effective velocity u'/gamma' + v_s (counted, not corrected)
            T vy = d[1] - sO * xc0;
            if (d[0] * d[0] + vy * vy + d[2] * d[2] >= c * c) atomicAdd(P.counters + 1, 1ull);
        }
        ny_ -= vs;
    } else if (PUSH == PUSH_SXE) {
        // in the expanding coordinates the shear flow moves xi_y at v_{s,y} / l_2:
        // xi^{n+1}_y = xi'_y - s Omega0 (l_1/l_2)(t^{n+1/2}) (xi'_x + xi^n_x)/2 dt
        const T c = pk<T>(P.c, P.f.c);
        const T sO = pk<T>(P.sO, P.f.sO);
        const T vf = pk<T>(P.sxe_vf, P.f.sxe_vf);
        const T half_nx = pk<T>(P.half_nx, P.f.half_nx);
        const T xc0 = (T(p.ci) - half_nx) + p.o[0];
        const T xc1 = (T(p.ci) - half_nx) + nx_;
        {
            // physical velocity u'/gamma' + v_s (d is the xi displacement L^{-1} u'/gamma')
            const T lx = pk<T>(P.lh[0], P.f.lh[0]), ly = pk<T>(P.lh[1], P.f.lh[1]), lz = pk<T>(P.lh[2], P.f.lh[2]);
            const T vx = d[0] * lx, vz = d[2] * lz;
            const T vy = d[1] * ly - sO * xc0 * pk<T>(P.sxe_l0x, P.f.sxe_l0x);
            if (vx * vx + vy * vy + vz * vz >= c * c) atomicAdd(P.counters + 1, 1ull);
        }
        ny_ -= sO * vf * (xc1 + xc0) * T(0.5);
    }
    p.o[0] = nx_; renorm(p.o[0], p.ci);
    if (GT::AY) { p.o[1] = ny_; renorm(p.o[1], p.cj); } else { p.o[1] = T(0.5); }
    if (GT::AZ) { p.o[2] = nz_; renorm(p.o[2], p.ck); } else { p.o[2] = T(0.5); }
    // periodic / shearing-periodic wrap
    if (p.ci >= g.nx) {
        p.ci -= g.nx;
        if ((PUSH == PUSH_KSB || PUSH == PUSH_SXE) && GT::AY) {
            p.cj += P.dys_end_i;
            p.o[1] += pk<T>(P.dys_end_f, P.f.dys_end_f);
            renorm(p.o[1], p.cj);
        }
    } else if (p.ci < 0) {
        p.ci += g.nx;
        if ((PUSH == PUSH_KSB || PUSH == PUSH_SXE) && GT::AY) {
            p.cj -= P.dys_end_i;
            p.o[1] -= pk<T>(P.dys_end_f, P.f.dys_end_f);
            renorm(p.o[1], p.cj);
        }
    }
    if (GT::AY) {
        if (p.cj >= g.ny) p.cj -= g.ny;
        if (p.cj >= g.ny) p.cj -= g.ny;
        if (p.cj < 0) p.cj += g.ny;
        if (p.cj < 0) p.cj += g.ny;
    }
    if (GT::AZ) { if (p.ck >= g.nz) p.ck -= g.nz; else if (p.ck < 0) p.ck += g.nz; }

    if (ESC != ESC_NONE) {
        bool esc;
        if (ESC == ESC_DISP) {
            T m = t_abs<T>(p.dr[0]);
            T ay = t_abs<T>(p.dr[1]);
            m = ay > m ? ay : m;
            if (P.esc_dims == 3) { T az = t_abs<T>(p.dr[2]); m = az > m ? az : m; }
            esc = m >= pk<T>(P.l_esc, P.f.l_esc);
        } else {
            U4 r = draw(p.id, P.seed, P.step, TAG_ESCAPE, 0u);
            esc = r.x[0] < P.esc_thresh;
        }
        if (esc) {
            double ux, uy, uz;
            sample_mj(p.id, P.seed, P.step, P.theta_inj, P.c, ux, uy, uz);
            p.u[0] = T(ux); p.u[1] = T(uy); p.u[2] = T(uz);
            p.dr[0] = p.dr[1] = p.dr[2] = T(0);
            atomicAdd(P.counters, 1ull);
        }
    }
}

// Push, deposit and move one particle: FA/fidx as for
// push_particle, JA: current accumulator, jidx: the start cell's linear index
// in its box.
template <class T, int G, int ORD, int PUSH, int ESC, class FA, class JA, class I>
__device__ inline void advance_particle(Particle<T>& p, const FA& fa, I fidx, const JA& ja, I jidx, T qs,
                                        const SpecStep<T>& S, const StepP& P, const Grid& g) {
    T d[3];
    push_particle<T, G, ORD, PUSH>(p, fa, fidx, S, P, d);
    deposit<T, G, ORD>(ja, jidx, p.o, d, qs);  // current from the (comoving) move x^n -> x^n + d
    move_particle<T, G, PUSH, ESC>(p, d, P, g);
}


// The per-step scalars of a step come from the device-resident context.
__device__ inline StepP with_ctx(const StepP& P0, const StepCtx* ctx) {
    StepP P = P0;
    P.step = ctx->step;
    P.dys_end_i = ctx->dys_i[2];
    P.dys_end_f = ctx->dys_f[2];
    P.inv_lh[0] = ctx->inv_lh[0];
    P.inv_lh[1] = ctx->inv_lh[1];
    P.inv_lh[2] = ctx->inv_lh[2];
    P.f.dys_end_f = ctx->f_dys_f[2];
    P.f.inv_lh[0] = ctx->f_inv_lh[0];
    P.f.inv_lh[1] = ctx->f_inv_lh[1];
    P.f.inv_lh[2] = ctx->f_inv_lh[2];
    for (int a = 0; a < 3; ++a) {
        P.lh[a] = ctx->lh[a];
        P.f.lh[a] = ctx->f_lh[a];
    }
    P.sxe_vf = ctx->sxe_vf;
    P.sxe_l0x = ctx->sxe_l0x;
    P.f.sxe_vf = ctx->f_sxe_vf;
    P.f.sxe_l0x = ctx->f_sxe_l0x;
    return P;
}

template <int G> __device__ inline int tile_of(const Tiling& tl, int ci, int cj, int ck) {
    using GT = GeomT<G>;
    using D = TileDims<G>;
    const int a = ci / D::TX;  // compile-time powers of two: shifts
    const int b = GT::AY ? cj / D::TY : 0;
    const int cc = GT::AZ ? ck / D::TZ : 0;
    return a + tl.ntx * (b + tl.nty * cc);
}

// Put a particle that left its tile into the arrival range (the back of the
// slot range) of tile `dest`.  Slots below the tile's start-of-step count may
// be taken by its stayers, so the k-th arrival (slot tcap-1-k) is valid only
// above it; otherwise the particle joins the loose list.  Failed claims
// over-count arr_out; finalize_kernel clamps it to the valid range.
template <class T, int G>
__device__ inline void place_mover(const Particle<T>& p, int dest, const SpecStep<T>& S, const StepP& P, bool leaky) {
    int cnt_in = S.stay_in[dest] + S.arr_in[dest];
    int k = atomicAdd(S.arr_out + dest, 1);
    long long rel = S.tcap - 1 - k;
    if (rel >= cnt_in) {
        store_particle<T, G>(S.out, (long long)dest * S.tcap + rel, leaky, p);
        return;
    }
    int l = atomicAdd(S.lcount_out, 1);
    if (l < S.lcap) store_particle<T, G>(S.lout, l, leaky, p);
    else atomicOr(P.err, ERRB_LOOSE_OVERFLOW);
}

constexpr int TPB = 256;  // threads per CTA of the loose kernel
constexpr long long TMA_WAIT_LIMIT = 1ll << 24;

// Tile-kernel variants: threads per CTA, the order of the stayers' write,
// and the number of copies of the shared current box.
//
// Shared-memory atomics of a warp cost about one pass per lane on the busiest
// bank, whether those lanes add to one word or to several (only a warp whose
// 32 lanes all add to one word is merged into one pass).  "stable" variants
// write each chunk's stayers in input order (a CTA-wide prefix over the warps'
// counts, one barrier per chunk), which keeps the cell grouping of the device
// loader longer; the others let warps claim output ranges in any order (no
// barrier).  jc > 1: copies of the current box 32/jc banks apart, each lane's
// particle dealt onto a copy so that the warp's adds spread over the banks
// (pick_copy); the flush sums the copies.  Particle states and FP32 currents
// are the same in all variants (exact integer sums).
struct TileVariant { int nt, stable, jc; };
constexpr int N_TILE_VARIANTS = 7;
constexpr TileVariant TILE_VARIANTS[N_TILE_VARIANTS] = {{256, 0, 1}, {512, 0, 1}, {512, 1, 1}, {256, 1, 1},
                                                        {256, 0, 2}, {256, 1, 2}, {512, 0, 4}};

// Variant (index) used when the choice is left to the library (measured on
// GB300: 512 threads with four current boxes for 3D FP32 tiles, 512 threads
// with one otherwise), and the one batched launches use (the same: for a
// batch of 16 3D FP32 boxes the four-copy variant also beat two copies at
// 256 threads, 1.31e10 against 1.24e10 particle-steps/s).
constexpr int default_tile_variant(bool fp64, int geom) { return (!fp64 && plane_of(geom) == G3D) ? 6 : 1; }
constexpr int batch_tile_variant(bool fp64, int geom) { return default_tile_variant(fp64, geom); }

// Dynamic shared memory: E box, B box (each 128-byte aligned, the TMA
// destinations), the J box (int32 for FP32, double for FP64), the mbarrier,
// small counters, and for stable variants two buffers of per-warp stayer
// counts.
// The copy of the shared current box a lane's particle adds into, with JC
// copies placed 32/JC banks apart (copy stride = 32/JC mod 32 words).  All
// adds of a warp instruction go to (each lane's base word + one common
// offset), so two lanes conflict whenever their base words share a bank, and
// for particles spread over a tile that is random: about 3.5 lanes on the
// busiest bank.  The lanes whose base banks share a residue mod 32/JC are
// dealt round-robin onto that residue's JC banks (copy = slot - bank / (32/JC)
// mod JC), so no bank takes more than ceil(lanes of the residue / JC): about
// 2.7 lanes with 2 copies, 2.1 with 4.  Lanes of the same cell fall apart the
// same way.  Lanes that are not dealt (crossing particles, which add only
// exact zeros here, and idle lanes) use copy 0 and trash word `lane`; the
// trash word of a dealt lane is the word of its copy whose bank is `lane`, so
// the exact zeros of a warp still land on 32 distinct banks.  FP64 words span
// two banks: its copies are chosen by lane parity.
template <class T, int G, int JC, int JCS>
__device__ __forceinline__ SmemJ<T, G> pick_copy(JWord<T>* sJ, int lane, bool deal, int base) {
    if constexpr (JC == 1) {
        return SmemJ<T, G>(sJ, lane);
    } else if constexpr (sizeof(JWord<T>) != 4) {
        return SmemJ<T, G>(sJ + (lane % JC) * JCS, lane);
    } else {
        constexpr int OFF = 32 / JC;
        static_assert(JC * OFF == 32 && JCS % 32 == OFF, "copies 32/JC banks apart");
        const int bank = base & 31;
        const int key = bank & (OFF - 1);
        unsigned same = __ballot_sync(0xffffffffu, deal);
#pragma unroll
        for (int k = 1; k < OFF; k <<= 1) {
            const unsigned bk = __ballot_sync(0xffffffffu, (key & k) != 0);
            same &= (key & k) ? bk : ~bk;
        }
        const int slot = __popc(same & ((1u << lane) - 1u)) & (JC - 1);
        const int c = deal ? ((slot - bank / OFF) & (JC - 1)) : 0;
        return SmemJ<T, G>(sJ + c * JCS, (lane - OFF * c) & 31);
    }
}

// 3D FP32 tiles queue crossing particles in two queues per warp: those that
// cross on one axis (deposit_1axis) and the rest (the full window).
template <class T, int G> __host__ __device__ constexpr bool split_queue() { return sizeof(T) == 4 && plane_of(G) == G3D; }

template <class T, int G, int NT, int STABLE, int JC> struct SmemLayout {
    static constexpr int FB = TileDims<G>::FB, JB = TileDims<G>::JB;
    static constexpr int QCAP = 64;  // entries of a warp's crossing-particle queue
    static constexpr int NQ = split_queue<T, G>() ? 2 : 1;  // queues per warp
    // copy stride in words: a multiple of 32 plus 32/JC (copy k is 32k/JC banks over)
    static constexpr int JCS = JC == 1 ? 3 * JB : ((3 * JB + 31) / 32) * 32 + 32 / JC;
    static constexpr size_t off_B = ((size_t)3 * FB * sizeof(T) + 127) & ~(size_t)127;
    static constexpr size_t off_J = (off_B + (size_t)3 * FB * sizeof(T) + 127) & ~(size_t)127;
    // queue k of warp w: offsets/moves at off_q + k QBYTES_OD + w QCAP 6 sizeof(T),
    // cells at off_qc + k QBYTES_C + w QCAP 4
    static constexpr size_t QBYTES_OD = (size_t)(NT / 32) * QCAP * 6 * sizeof(T);
    static constexpr size_t QBYTES_C = (size_t)(NT / 32) * QCAP * 4;
    static constexpr size_t off_q = (off_J + (size_t)JC * JCS * sizeof(T) + 15) & ~(size_t)15;
    static constexpr size_t off_qc = off_q + NQ * QBYTES_OD;
    static constexpr size_t off_bar = (off_qc + NQ * QBYTES_C + 15) & ~(size_t)15;
    static constexpr size_t off_wc = off_bar + 16 + 4 * (MAXSP + 2);
    static constexpr size_t bytes = off_wc + (STABLE ? 2 * (NT / 32) * 4 : 0);
};

// The fused particle step for tile t of one box (see the file header), made
// by a CTA of NT threads whose mbarrier is initialised; parity: the phase of
// its next use.  STABLE: order-preserving stayer write; JC: current copies.
// Returns false (error bit set) if the tile's fields did not arrive.  Ends
// with a barrier, so the CTA may go on to another tile.
template <class T, int G, int ORD, int PUSH, int ESC, int NT, int STABLE, int JC>
__device__ __forceinline__ bool tile_body(const CUtensorMap* tmE, const CUtensorMap* tmB, const Grid& g, const Tiling& tl,
                                          const StepP& P, const SpecPack<T>& SP, JWord<T>* __restrict__ J, const int t,
                                          const uint32_t parity) {
    using GT = GeomT<G>;
    constexpr bool LEAKY = (ESC == ESC_DISP);
    using D = TileDims<G>;
    using L = SmemLayout<T, G, NT, STABLE, JC>;
    constexpr int NW = NT / 32;
    using JW = JWord<T>;
    extern __shared__ __align__(128) unsigned char smem[];
    T* sE = reinterpret_cast<T*>(smem);
    T* sB = reinterpret_cast<T*>(smem + L::off_B);
    JW* sJ = reinterpret_cast<JW*>(smem + L::off_J);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::off_bar);
    int* s_cnt = reinterpret_cast<int*>(smem + L::off_bar + 16);
    int* s_ok = s_cnt + MAXSP;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ti = t % tl.ntx, tj = (t / tl.ntx) % tl.nty, tk = t / (tl.ntx * tl.nty);
    const int t0x = ti * D::TX, t0y = tj * D::TY, t0z = tk * D::TZ;
    // padded coordinate of physical t0 - 2 is t0 (GL = 2); TX is a multiple of the TMA x quantum
    const int xs = t0x;
    const int ys = GT::AY ? t0y : 0;
    const int zs = GT::AZ ? t0z : 0;

    // tensor copies need 128-byte aligned shared destinations: check, and
    // report instead of copying if the layout ever breaks that
    if (((smem_u32(sE) | smem_u32(sB)) & 127u) != 0u) {
        if (tid == 0) atomicOr(P.err, ERRB_SMEM_ALIGN);
        __syncthreads();
        return false;
    }
    if (tid == 0) {
        // a CTA that runs several tiles read the previous tile's boxes with
        // ordinary loads (all done: the previous tile ended with a barrier)
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar, (uint32_t)(6 * L::FB * sizeof(T)));
        tma_load_4d(sE, tmE, xs, ys, zs, 0, bar);
        tma_load_4d(sB, tmB, xs, ys, zs, 0, bar);
    }
    for (int i = tid; i < JC * L::JCS; i += NT) sJ[i] = JW(0);
    if (tid < MAXSP) s_cnt[tid] = 0;
    if (tid == 0) {
        const bool ok = mbar_wait_bounded(bar, parity, TMA_WAIT_LIMIT);
        // on a timeout the copies may still be writing this CTA's shared
        // memory: wait for them once more (bounded) before the CTA may leave
        if (!ok) mbar_wait_bounded(bar, parity, TMA_WAIT_LIMIT);
        s_ok[0] = ok ? 1 : 0;
    }
    __syncthreads();
    if (!s_ok[0]) {
        if (tid == 0) atomicOr(P.err, ERRB_TMA_TIMEOUT);
        return false;
    }

    const SmemFields<T, G> fa{sE, sB};
    using FA = SmemFields<T, G>;
    using JA = SmemJ<T, G>;
    const T vscale = sizeof(T) == 4 ? T(P.fx_scale) : T(1);
    // index-space origins (physical cell of local index 0)
    const int fox = xs - 2, foy = GT::AY ? t0y - 2 : 0, foz = GT::AZ ? t0z - 2 : 0;
    const int jox = t0x - 2, joy = GT::AY ? t0y - 2 : 0, joz = GT::AZ ? t0z - 2 : 0;
    T* q_od = reinterpret_cast<T*>(smem + L::off_q) + (size_t)warp * 6 * L::QCAP;  // this warp's queue:
    int* q_cell = reinterpret_cast<int*>(smem + L::off_qc) + warp * L::QCAP;        // start offsets, moves, cells
    int qn = 0;                                                                     // entries (warp-uniform)
    // 3D FP32: a second queue for particles that cross on one axis only (the
    // axis rides in the cell word's top bits), deposited by deposit_1axis
    constexpr bool SPLIT = split_queue<T, G>();
    T* q1_od = reinterpret_cast<T*>(smem + L::off_q + (SPLIT ? L::QBYTES_OD : 0)) + (size_t)warp * 6 * L::QCAP;
    int* q1_cell = reinterpret_cast<int*>(smem + L::off_qc + (SPLIT ? L::QBYTES_C : 0)) + warp * L::QCAP;
    int qn1 = 0;
    int* s_wc = reinterpret_cast<int*>(smem + L::off_wc);  // [2][NW] stayer counts (stable variants)
    int wcb = 0;                                            // their buffer for the current chunk

    for (int s = 0; s < P.nsp; ++s) {
        const SpecStep<T>& S = SP.s[s];
        const int nst = S.stay_in[t], nar = S.arr_in[t];
        const int n = nst + nar;
        const long long base = (long long)t * S.tcap;
        const T qs = S.q * vscale;
        int run = 0;  // stayers written so far (stable variants)
        // full deposit of queue entry e by this lane (have: the lane holds an
        // entry; every lane of the warp calls it; lanes read their entries
        // before any write)
        auto queued_deposit = [&](int e, bool have) {
            T oe[3] = {T(0), T(0), T(0)}, de[3] = {T(0), T(0), T(0)};
            int ce = 0;
            if (have) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    oe[a] = q_od[a * L::QCAP + e];
                    de[a] = q_od[(3 + a) * L::QCAP + e];
                }
                ce = q_cell[e];
            }
            int wbase = ce + window_base<T, ORD>(oe[0], oe[0] + de[0]);
            if (GT::AY) wbase += window_base<T, ORD>(oe[1], oe[1] + de[1]) * JA::SY;
            if (GT::AZ) wbase += window_base<T, ORD>(oe[2], oe[2] + de[2]) * JA::SZ;
            const JA jq = pick_copy<T, G, JC, L::JCS>(sJ, lane, have, wbase);
            if (have) deposit<T, G, ORD>(jq, ce, oe, de, qs);
        };
        // the same for the single-axis queue
        auto queued_deposit1 = [&](int e, bool have) {
            T oe[3] = {T(0), T(0), T(0)}, de[3] = {T(0), T(0), T(0)};
            int cw = 0;
            if (have) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    oe[a] = q1_od[a * L::QCAP + e];
                    de[a] = q1_od[(3 + a) * L::QCAP + e];
                }
                cw = q1_cell[e];
            }
            const int ce = cw & 0x0FFFFFFF, ax = (int)((unsigned)cw >> 28);
            int wbase = ce + window_base<T, ORD>(oe[0], oe[0] + de[0]);
            if (GT::AY) wbase += window_base<T, ORD>(oe[1], oe[1] + de[1]) * JA::SY;
            if (GT::AZ) wbase += window_base<T, ORD>(oe[2], oe[2] + de[2]) * JA::SZ;
            const JA jq = pick_copy<T, G, JC, L::JCS>(sJ, lane, have, wbase);
            if constexpr (SPLIT) {
                if (have) deposit_1axis<T, ORD>(jq, ce, oe, de, qs, ax);
            }
        };
        for (int i0 = 0; i0 < n; i0 += NT) {
            const int i = i0 + tid;
            const bool valid = i < n;
            Particle<T> p;
            int dest = -1;
            bool cross = false, cross1 = false;  // crosses on some axis / on exactly one
            int cax = 0;                        // that one axis
            int jidx = 0;
            T o0[3], d[3];
            int cbase = 0;  // base word of the core deposit
            if (valid) {
                const long long slot = i < nst ? base + i : base + S.tcap - nar + (i - nst);
                load_particle<T, G>(S.in, slot, LEAKY, p);
                const int fidx = (p.ci - fox) + (GT::AY ? (p.cj - foy) * FA::SY : 0) + (GT::AZ ? (p.ck - foz) * FA::SZ : 0);
                jidx = (p.ci - jox) + (GT::AY ? (p.cj - joy) * JA::SY : 0) + (GT::AZ ? (p.ck - joz) * JA::SZ : 0);
                push_particle<T, G, ORD, PUSH>(p, fa, fidx, S, P, d);
                if constexpr (SPLIT) {
                    const int cm = cross_mask<T, G, ORD>(p.o, d);
                    cross = cm != 0;
                    cross1 = cm == 1 || cm == 2 || cm == 4;
                    cax = cm == 1 ? 0 : (cm == 2 ? 1 : 2);
                } else {
                    cross = crosses<T, G, ORD>(p.o, d);
                }
                cbase = core_base<T, G, ORD>(jidx, p.o, JA::SY, JA::SZ);
            }
            const JA ja = pick_copy<T, G, JC, L::JCS>(sJ, lane, valid && !cross, cbase);
            if (valid) {
                deposit_core<T, G, ORD>(ja, jidx, p.o, d, qs, cross);
                o0[0] = p.o[0]; o0[1] = p.o[1]; o0[2] = p.o[2];
                move_particle<T, G, PUSH, ESC>(p, d, P, g);
                dest = tile_of<G>(tl, p.ci, p.cj, p.ck);
            }
            // crossing particles join the warp's queue; their full deposit is
            // made 32 at a time, every lane adding real contributions
            const bool crossf = cross && !cross1;  // to the full-window queue
            const unsigned qm = __ballot_sync(0xffffffffu, crossf);
            if constexpr (SPLIT) {
                const unsigned q1m = __ballot_sync(0xffffffffu, cross1);
                if (cross1) {
                    const int pos = qn1 + __popc(q1m & ((1u << lane) - 1u));
                    q1_cell[pos] = jidx | (cax << 28);
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        q1_od[a * L::QCAP + pos] = o0[a];
                        q1_od[(3 + a) * L::QCAP + pos] = d[a];
                    }
                }
                qn1 += __popc(q1m);
            }
            if (crossf) {
                const int pos = qn + __popc(qm & ((1u << lane) - 1u));
                q_cell[pos] = jidx;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    q_od[a * L::QCAP + pos] = o0[a];
                    q_od[(3 + a) * L::QCAP + pos] = d[a];
                }
            }
            qn += __popc(qm);
            const bool stay = valid && dest == t;
            const unsigned m = __ballot_sync(0xffffffffu, stay);
            int wb = 0;
            if (STABLE) {
                // this warp's stayers go after those of the chunk's lower warps
                int* wc = s_wc + wcb * NW;
                if (lane == 0) wc[warp] = __popc(m);
                __syncthreads();
                const int cw = lane < NW ? wc[lane] : 0;
                int incl = cw;
#pragma unroll
                for (int sh = 1; sh < 32; sh <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, incl, sh);
                    if (lane >= sh) incl += v;
                }
                wb = run + __shfl_sync(0xffffffffu, incl - cw, warp);
                run += __shfl_sync(0xffffffffu, incl, 31);
                wcb ^= 1;
            } else {
                if (lane == 0 && m) wb = atomicAdd(&s_cnt[s], __popc(m));
                wb = __shfl_sync(0xffffffffu, wb, 0);
            }
            if (stay) store_particle<T, G>(S.out, base + wb + __popc(m & ((1u << lane) - 1u)), LEAKY, p);
            else if (valid) place_mover<T, G>(p, dest, S, P, LEAKY);
            if (SPLIT && qn1 >= 32) {
                __syncwarp();
                queued_deposit1(lane, true);
                const int rest = qn1 - 32;
                int c = 0;
                T od[6];
                if (lane < rest) {
                    c = q1_cell[32 + lane];
#pragma unroll
                    for (int k = 0; k < 6; ++k) od[k] = q1_od[k * L::QCAP + 32 + lane];
                }
                __syncwarp();
                if (lane < rest) {
                    q1_cell[lane] = c;
#pragma unroll
                    for (int k = 0; k < 6; ++k) q1_od[k * L::QCAP + lane] = od[k];
                }
                __syncwarp();
                qn1 = rest;
            }
            if (qn >= 32) {
                __syncwarp();
                queued_deposit(lane, true);
                // move the remaining entries (qn - 32 < 32) to the front
                const int rest = qn - 32;
                int c = 0;
                T od[6];
                if (lane < rest) {
                    c = q_cell[32 + lane];
#pragma unroll
                    for (int k = 0; k < 6; ++k) od[k] = q_od[k * L::QCAP + 32 + lane];
                }
                __syncwarp();
                if (lane < rest) {
                    q_cell[lane] = c;
#pragma unroll
                    for (int k = 0; k < 6; ++k) q_od[k * L::QCAP + lane] = od[k];
                }
                __syncwarp();
                qn = rest;
            }
        }
        // the species' remaining queue (charge qs)
        __syncwarp();
        if (qn > 0) queued_deposit(lane, lane < qn);  // qn is warp-uniform
        if (SPLIT && qn1 > 0) {
            __syncwarp();
            queued_deposit1(lane, lane < qn1);
        }
        qn1 = 0;
        __syncwarp();
        qn = 0;
        if (STABLE && tid == 0) s_cnt[s] = run;
    }

    __syncthreads();
    // flush the J tile into the global accumulator (integer adds for FP32, so
    // the result does not depend on the order tiles finish in): padded index
    // of local point (a,b,c) is (t0x + a, t0y + b, t0z + c)
    for (int idx = tid; idx < 3 * L::JB; idx += NT) {
        JW v = sJ[idx];
#pragma unroll
        for (int k = 1; k < JC; ++k) v += sJ[k * L::JCS + idx];  // FP32: exact mod 2^32
        if (v == JW(0)) continue;
        const int comp = idx / L::JB;
        const int r = idx - comp * L::JB;
        const int a = r % D::JX;
        const int b = (r / D::JX) % D::JY;
        const int c = r / (D::JX * D::JY);
        const int pi = jox + g.gx + a, pj = joy + g.gy + b, pk = joz + g.gz + c;
        if (pi >= g.px || pj >= g.py || pk >= g.pz) continue;  // beyond a ragged last tile: never deposited
        atomicAdd(J + (long long)comp * g.cstride + ((long long)pk * g.py + pj) * g.px + pi, v);
    }
    if (tid < P.nsp) SP.s[tid].stay_out[t] = s_cnt[tid];
    __syncthreads();
    return true;
}

template <class T, int G, int NT, int STABLE, int JC> __device__ __forceinline__ void init_tile_barrier() {
    using L = SmemLayout<T, G, NT, STABLE, JC>;
    extern __shared__ __align__(128) unsigned char smem[];
    if (threadIdx.x == 0) {
        mbar_init(reinterpret_cast<uint64_t*>(smem + L::off_bar), 1);
        fence_mbar_init();
    }
    __syncthreads();
}

// One box: one CTA per tile.
template <class T, int G, int ORD, int PUSH, int ESC, int NT, int STABLE, int JC>
__global__ void __launch_bounds__(NT, NT == 1024 || JC >= 4 ? 1 : (NT == 512 ? 2 : 3)) tile_kernel(const __grid_constant__ CUtensorMap tmE,
                                                   const __grid_constant__ CUtensorMap tmB, Grid g, Tiling tl,
                                                   StepP P0, SpecPack<T> SP, JWord<T>* __restrict__ J,
                                                   const StepCtx* __restrict__ ctx) {
    init_tile_barrier<T, G, NT, STABLE, JC>();
    const StepP P = with_ctx(P0, ctx);
    tile_body<T, G, ORD, PUSH, ESC, NT, STABLE, JC>(&tmE, &tmB, g, tl, P, SP, J, blockIdx.x, 0u);
}

// A batch of boxes of one kind (precision, geometry, order, pusher, escape
// rule) in one persistent launch: the tiles of all boxes form one work list,
// box b owning items [first[b], first[b+1]) (boxes in decreasing particles per
// tile), and every CTA claims its next item from a counter (zero at launch),
// so CTAs that drew light tiles take more of them.  The boxes' descriptors,
// tensor maps included, are kernel parameters.
template <class T> struct BoxDesc {
    CUtensorMap tmE, tmB;
    Grid g;
    Tiling tl;
    StepP P0;
    SpecPack<T> SP;
    JWord<T>* J;
    const StepCtx* ctx;
};
constexpr int BATCH_PARAM_BYTES = 32000;  // kernel parameters allow 32,764 bytes
template <class T> struct BatchArgs {
    static constexpr int MAXB = (BATCH_PARAM_BYTES - 64) / (int)sizeof(BoxDesc<T>);
    BoxDesc<T> box[MAXB];
    int first[MAXB + 1];
    int nbox;
    int* next;  // work counter of this launch
};

template <class T, int G, int ORD, int PUSH, int ESC, int NT, int STABLE, int JC>
__global__ void __launch_bounds__(NT, NT == 1024 || JC >= 4 ? 1 : (NT == 512 ? 2 : 3)) batch_tile_kernel(
    const __grid_constant__ BatchArgs<T> A) {
    init_tile_barrier<T, G, NT, STABLE, JC>();
    // the claimed item goes through the layout's spare word (no static
    // shared variable: it would shift the dynamic area the tensor copies
    // address off its 128-byte alignment)
    using L = SmemLayout<T, G, NT, STABLE, JC>;
    extern __shared__ __align__(128) unsigned char smem[];
    int* s_item = reinterpret_cast<int*>(smem + L::off_bar + 16) + MAXSP + 1;
    if (A.nbox < 1 || A.nbox > BatchArgs<T>::MAXB || A.next == nullptr) return;
    uint32_t parity = 0;
    int b = 0;
    const int nwork = A.first[A.nbox];
    for (;;) {
        if (threadIdx.x == 0) *s_item = atomicAdd(A.next, 1);
        __syncthreads();
        const int w = *s_item;
        __syncthreads();
        if (w >= nwork) break;
        while (b < A.nbox && w >= A.first[b + 1]) ++b;  // a CTA's items increase
        const int t = b < A.nbox ? w - A.first[b] : -1;
        if (w < 0 || b >= A.nbox || t < 0 || t >= A.box[b < A.nbox ? b : 0].tl.ntiles) {
            if (threadIdx.x == 0) atomicOr(A.box[0].P0.err, ERRB_BATCH);
            break;
        }
        const BoxDesc<T>& B = A.box[b];
        // tensor maps must sit on 64-byte boundaries
        if ((reinterpret_cast<uintptr_t>(&B.tmE) | reinterpret_cast<uintptr_t>(&B.tmB)) & 63u) {
            if (threadIdx.x == 0) atomicOr(A.box[0].P0.err, ERRB_BATCH);
            break;
        }
        const StepP P = with_ctx(B.P0, B.ctx);
        if (!tile_body<T, G, ORD, PUSH, ESC, NT, STABLE, JC>(&B.tmE, &B.tmB, B.g, B.tl, P, B.SP, B.J, t, parity))
            return;
        parity ^= 1;
    }
}

// Loose particles: the same per-particle step with fields read from global
// memory and the current added with global atomics; afterwards each particle
// is inserted into its tile like any mover, or stays loose.
template <class T, int G, int ORD, int PUSH, int ESC>
__global__ void __launch_bounds__(TPB) loose_kernel(Grid g, Tiling tl, StepP P0, SpecPack<T> SP,
                                                    const T* __restrict__ E, const T* __restrict__ B,
                                                    JWord<T>* __restrict__ J, const StepCtx* __restrict__ ctx) {
    using GT = GeomT<G>;
    const StepP P = with_ctx(P0, ctx);
    constexpr bool LEAKY = (ESC == ESC_DISP);
    const long long SY = g.px, SZ = (long long)g.px * g.py;
    const GlobalFields<T> fa{E, B, SY, SZ, g.cstride};
    const GlobalJ<T> ja{J, SY, SZ, g.cstride};
    for (int s = 0; s < P.nsp; ++s) {
        const SpecStep<T>& S = SP.s[s];
        long long n = *S.lcount_in;
        if (n > S.lcap) n = S.lcap;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
            Particle<T> p;
            load_particle<T, G>(S.lin, i, LEAKY, p);
            const long long cidx = (long long)(p.ci + g.gx) + (GT::AY ? (long long)(p.cj + g.gy) * SY : 0) +
                                   (GT::AZ ? (long long)(p.ck + g.gz) * SZ : 0);
            const T qs = sizeof(T) == 4 ? T(S.q * P.fx_scale) : S.q;
            advance_particle<T, G, ORD, PUSH, ESC>(p, fa, cidx, ja, cidx, qs, S, P, g);
            place_mover<T, G>(p, tile_of<G>(tl, p.ci, p.cj, p.ck), S, P, LEAKY);
        }
    }
}

}  // namespace pic
