// fields.cuh -- grid kernels of libpic: Yee curl updates (standard and
// expanding box), the shearing-box implicit-midpoint sweep, guard-cell fill
// and current fold with the shearing-periodic shift, the shearing-box
// current advection, and FP64 reductions.  All kernels work on padded
// component arrays (see common.cuh); one thread per grid point.
#pragma once

#include "common.cuh"

namespace pic {

// Launch shape of the grid kernels: x (or the fastest index) over the
// threads of a block and over blockIdx.x, the other two indices over
// blockIdx.y and blockIdx.z, so no thread divides an index.
constexpr int CELL_THREADS = 128;
inline dim3 cell_grid(long long nfast, long long ny, long long nz) {
    return dim3((unsigned)((nfast + CELL_THREADS - 1) / CELL_THREADS), (unsigned)ny, (unsigned)nz);
}

// ---- Yee curl updates ------------------------------------------------------------------
// out_c <- alpha_c out_c + beta_c curl(sigma (.) in)_c + gam_c J_c over interior cells.
// CURL_E: curl of an E-located field, result at B locations; else curl of a
// B-located field, result at E locations.  The ignorable 2D axis contributes no
// differences.  Standard Yee: alpha = 1, sigma = 1; expanding box: the
// transforms X' = ell L^-1 X folded into alpha, beta, gam, sigma (Sec. 3.2).
template <class T, int G, bool CURL_E>
__device__ __forceinline__ void curl_update_body(const Grid& g, const T* __restrict__ in, T* __restrict__ out,
                                                 const T* __restrict__ J, const StepCtx* __restrict__ ctx, int which,
                                                 int i, int j, int k) {
    using GT = GeomT<G>;
    const Coef3 cf = ctx->curl[which];
    {
        long long c0 = g.idx(i, j, k);
        const long long sx = 1, sy = g.px, sz = (long long)g.px * g.py, cs = g.cstride;
        const T* X = in;
        const T* Y = in + cs;
        const T* Z = in + 2 * cs;
        T s0 = T(cf.s[0]), s1 = T(cf.s[1]), s2 = T(cf.s[2]);
        T cu[3];
        if (CURL_E) {
            // (curl E)_x = dy Ez - dz Ey, (curl E)_y = dz Ex - dx Ez, (curl E)_z = dx Ey - dy Ex, forward differences
            T dyEz = GT::AY ? s2 * (Z[c0 + sy] - Z[c0]) : T(0);
            T dzEy = GT::AZ ? s1 * (Y[c0 + sz] - Y[c0]) : T(0);
            T dzEx = GT::AZ ? s0 * (X[c0 + sz] - X[c0]) : T(0);
            T dxEz = s2 * (Z[c0 + sx] - Z[c0]);
            T dxEy = s1 * (Y[c0 + sx] - Y[c0]);
            T dyEx = GT::AY ? s0 * (X[c0 + sy] - X[c0]) : T(0);
            cu[0] = dyEz - dzEy;
            cu[1] = dzEx - dxEz;
            cu[2] = dxEy - dyEx;
        } else {
            // backward differences
            T dyBz = GT::AY ? s2 * (Z[c0] - Z[c0 - sy]) : T(0);
            T dzBy = GT::AZ ? s1 * (Y[c0] - Y[c0 - sz]) : T(0);
            T dzBx = GT::AZ ? s0 * (X[c0] - X[c0 - sz]) : T(0);
            T dxBz = s2 * (Z[c0] - Z[c0 - sx]);
            T dxBy = s1 * (Y[c0] - Y[c0 - sx]);
            T dyBx = GT::AY ? s0 * (X[c0] - X[c0 - sy]) : T(0);
            cu[0] = dyBz - dzBy;
            cu[1] = dzBx - dxBz;
            cu[2] = dxBy - dyBx;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            T v = T(cf.a[c]) * out[c * cs + c0] + T(cf.b[c]) * cu[c];
            if (J) v += T(cf.g[c]) * J[c * cs + c0];
            out[c * cs + c0] = v;
        }
    }
}

template <class T, int G, bool CURL_E>
__global__ void curl_update_kernel(Grid g, const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ J,
                                   const StepCtx* __restrict__ ctx, int which) {
    // launch: cell_grid(nx, ny, nz)
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nx) return;
    curl_update_body<T, G, CURL_E>(g, in, out, J, ctx, which, i, blockIdx.y, blockIdx.z);
}

// ---- shearing-box implicit-midpoint sweep ---------------------------------------------
// X_out = X_n + dt F((X_n + X_k)/2), F the right-hand sides of the KSB-OA
// field equations (Sec. 2.1) with V(x) = -s Omega0 (x - nx/2):
//   F_B  = -c curl E' - V dy B - s Omega0 Bx e_y
//   F_Ex = c (curl B)_x - 4 pi J'_x + V dy E'_x - V dx E'_y
//   F_Ey = c (curl B)_y - 4 pi J'_y - V dy E'_y - V (dx E'_x + dz E'_z)
//   F_Ez = c (curl B)_z - 4 pi J'_z + V dy E'_z - V dz E'_y
// The advection term of each component is upwinded for its own transport
// velocity (V in the B and E'_y rows, -V in the E'_x and E'_z rows); the
// other V-terms are centred and averaged in y onto the component's location;
// Bx in the By row is the mean of its four neighbours.  Guards of X_n and X_k
// hold the shearing-periodic images at t^{n+1/2}.
//
// The shearing + expanding box sweeps the expanding-frame fields X^ = ell
// L^{-1} X (Sec. 3.1) with the factors of its coordinates from the step
// context: curls of (l_a^2 / ell) X^_a, the shear flow and shear term times
// l_1/l_2, the -V d_x E^_y and -V d_z E^_y terms times (l_2/l_1)^2 and
// (l_2/l_3)^2, all at t^{n+1/2}.  For the shearing box these are ones.
template <class T, int G>
__global__ void ksb_sweep_kernel(Grid g, const T* __restrict__ En, const T* __restrict__ Bn, const T* __restrict__ Ek,
                                 const T* __restrict__ Bk, const T* __restrict__ J, T* __restrict__ Eo, T* __restrict__ Bo,
                                 double c_, double sO_, double half_nx, const StepCtx* __restrict__ ctx) {
    using GT = GeomT<G>;
    const T c = T(c_), sO = T(sO_ * ctx->sxe_vf);
    const T sg0 = T(ctx->sxe_sig[0]), sg1 = T(ctx->sxe_sig[1]), sg2 = T(ctx->sxe_sig[2]);
    const T rx = T(ctx->sxe_rx), rz = T(ctx->sxe_rz);
    const T FOUR_PI = T(12.566370614359172);
    const long long sx = 1, sy = GT::AY ? g.px : 0, sz = GT::AZ ? (long long)g.px * g.py : 0, cs = g.cstride;
    // launch: cell_grid(nx, ny, nz)
    {
        const int i = blockIdx.x * blockDim.x + threadIdx.x;
        if (i >= g.nx) return;
        const int j = blockIdx.y, k = blockIdx.z;
        long long c0 = g.idx(i, j, k);
        // midpoint fields
        auto ME = [&](int comp, long long off) -> T { return T(0.5) * (En[comp * cs + c0 + off] + Ek[comp * cs + c0 + off]); };
        auto MB = [&](int comp, long long off) -> T { return T(0.5) * (Bn[comp * cs + c0 + off] + Bk[comp * cs + c0 + off]); };
        // x - nx/2 at nodes and half-points: exact in either precision
        const T VN = -sO * (T(i) - T(half_nx));
        const T VH = -sO * ((T(i) + T(0.5)) - T(half_nx));
        // curls (ignorable-axis differences vanish because its stride is 0)
        T curlEx = sg2 * (ME(2, sy) - ME(2, 0)) - sg1 * (ME(1, sz) - ME(1, 0));
        T curlEy = sg0 * (ME(0, sz) - ME(0, 0)) - sg2 * (ME(2, sx) - ME(2, 0));
        T curlEz = sg1 * (ME(1, sx) - ME(1, 0)) - sg0 * (ME(0, sy) - ME(0, 0));
        T curlBx = sg2 * (MB(2, 0) - MB(2, -sy)) - sg1 * (MB(1, 0) - MB(1, -sz));
        T curlBy = sg0 * (MB(0, 0) - MB(0, -sz)) - sg2 * (MB(2, 0) - MB(2, -sx));
        T curlBz = sg1 * (MB(1, 0) - MB(1, -sx)) - sg0 * (MB(0, 0) - MB(0, -sy));
        auto upB = [&](int comp, T v) -> T { return v > T(0) ? MB(comp, 0) - MB(comp, -sy) : MB(comp, sy) - MB(comp, 0); };
        auto upE = [&](int comp, T v) -> T { return v > T(0) ? ME(comp, 0) - ME(comp, -sy) : ME(comp, sy) - ME(comp, 0); };
        T bx4 = T(0.25) * (MB(0, 0) + MB(0, sx) + MB(0, -sy) + MB(0, sx - sy));
        T FBx = -c * curlEx - VN * upB(0, VN);
        T FBy = -c * curlEy - VH * upB(1, VH) - sO * bx4;
        T FBz = -c * curlEz - VH * upB(2, VH);
        T dxEy = T(0.5) * ((ME(1, sx) - ME(1, 0)) + (ME(1, sx - sy) - ME(1, -sy)));
        T divxz = T(0.5) * ((ME(0, 0) - ME(0, -sx)) + (ME(0, sy) - ME(0, sy - sx)) + (ME(2, 0) - ME(2, -sz)) +
                            (ME(2, sy) - ME(2, sy - sz)));
        T dzEy = T(0.5) * ((ME(1, sz) - ME(1, 0)) + (ME(1, sz - sy) - ME(1, -sy)));
        T FEx = c * curlBx - FOUR_PI * J[c0] + VH * upE(0, -VH) - VH * (rx * dxEy);
        T FEy = c * curlBy - FOUR_PI * J[cs + c0] - VN * upE(1, VN) - VN * divxz;
        T FEz = c * curlBz - FOUR_PI * J[2 * cs + c0] + VN * upE(2, -VN) - VN * (rz * dzEy);
        Eo[c0] = En[c0] + FEx;
        Eo[cs + c0] = En[cs + c0] + FEy;
        Eo[2 * cs + c0] = En[2 * cs + c0] + FEz;
        Bo[c0] = Bn[c0] + FBx;
        Bo[cs + c0] = Bn[cs + c0] + FBy;
        Bo[2 * cs + c0] = Bn[2 * cs + c0] + FBz;
    }
}

// ---- guard fill -----------------------------------------------------------------------
// Axis passes: x first (interior y, z rows; with the shear shift dys for the
// shearing box: the ghost at (i >= nx, j) is the interior value at
// (i - nx, j + dys), linearly interpolated, and at (i < 0, j) the one at
// (i + nx, j - dys)), then y over all padded x, then z over all padded x, y.
// The shift is (dys_i, dys_f), or ctx->dys_*[which] when ctx is given.
template <class T, int G>
__device__ __forceinline__ void fill_x_body(const Grid& g, T* F, int dys_i, double dys_f, int j, int k, int zs) {
    using GT = GeomT<G>;
    const int nguard = g.px - g.nx;  // gx low + the rest high
    {
        const int comp = zs / nguard, gi = zs - comp * nguard;
        int i = gi < g.gx ? gi - g.gx : g.nx + (gi - g.gx);  // physical ghost index
        int w = i < 0 ? -1 : 1;
        int is = i - w * g.nx;
        T* Fc = F + (long long)comp * g.cstride;
        T v;
        if (GT::AY && (dys_i != 0 || dys_f != 0.0)) {
            // y + w dys = j + w (dys_i + dys_f)
            int m;
            double f;
            if (w > 0) { m = dys_i; f = dys_f; }
            else { m = -dys_i; f = -dys_f; if (f < 0.0) { f += 1.0; m -= 1; } }
            int j0 = j + m, j1 = j0 + 1;
            j0 %= g.ny; if (j0 < 0) j0 += g.ny;
            j1 %= g.ny; if (j1 < 0) j1 += g.ny;
            v = T(1.0 - f) * Fc[g.idx(is, j0, k)] + T(f) * Fc[g.idx(is, j1, k)];
        } else {
            v = Fc[g.idx(is, j, k)];
        }
        Fc[g.idx(i, j, k)] = v;
    }
}

template <class T, int G>
__global__ void fill_x_kernel(Grid g, T* F, int ncomp, int dys_i, double dys_f, const StepCtx* __restrict__ ctx, int which) {
    if (ctx) {
        dys_i = ctx->dys_i[which];
        dys_f = ctx->dys_f[which];
    }
    // launch: cell_grid(ny, nz, ncomp * nguard)
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= g.ny) return;
    fill_x_body<T, G>(g, F, dys_i, dys_f, j, blockIdx.y, blockIdx.z);
}

template <class T>
__device__ __forceinline__ void fill_y_body(const Grid& g, T* F, int pi, int k, int zs) {
    const int nguard = g.py - g.ny;
    const int comp = zs / nguard, gj = zs - comp * nguard;
    int j = gj < g.gy ? gj - g.gy : g.ny + (gj - g.gy);
    int js = j < 0 ? j + g.ny : j - g.ny;
    T* Fc = F + (long long)comp * g.cstride;
    long long row = (long long)(k + g.gz) * g.py;
    Fc[(row + j + g.gy) * g.px + pi] = Fc[(row + js + g.gy) * g.px + pi];
}

template <class T>
__global__ void fill_y_kernel(Grid g, T* F, int ncomp) {
    // launch: cell_grid(px, nz, ncomp * nguard)
    const int pi = blockIdx.x * blockDim.x + threadIdx.x;
    if (pi >= g.px) return;
    fill_y_body<T>(g, F, pi, blockIdx.y, blockIdx.z);
}

template <class T>
__device__ __forceinline__ void fill_z_body(const Grid& g, T* F, int pi, int pj, int zs) {
    const int nguard = g.pz - g.nz;
    const long long plane = (long long)g.px * g.py;
    const long long pp = (long long)pj * g.px + pi;
    const int comp = zs / nguard, gk = zs - comp * nguard;
    int k = gk < g.gz ? gk - g.gz : g.nz + (gk - g.gz);
    int ks = k < 0 ? k + g.nz : k - g.nz;
    T* Fc = F + (long long)comp * g.cstride;
    Fc[(long long)(k + g.gz) * plane + pp] = Fc[(long long)(ks + g.gz) * plane + pp];
}

template <class T>
__global__ void fill_z_kernel(Grid g, T* F, int ncomp) {
    // launch: cell_grid(px, py, ncomp * nguard)
    const int pi = blockIdx.x * blockDim.x + threadIdx.x;
    if (pi >= g.px) return;
    fill_z_body<T>(g, F, pi, blockIdx.y, blockIdx.z);
}

// One-pass guard fill of the three components of F for boxes without a
// shear shift: every guard point takes the interior value at its periodic
// image in all axes at once, so the x, y and z guards need no ordering and
// one launch does what the three axis passes do (the same values: a copy).
// Guard points are enumerated in three regions: the z-guard planes (all
// padded x, y), then the y-guard rows of interior planes (all padded x),
// then the x-guard columns of interior rows.
template <class T, int G>
__device__ __forceinline__ void fill_all_point(const Grid& g, T* F, long long q) {
    using GT = GeomT<G>;
    const long long nzr = GT::AZ ? (long long)(g.pz - g.nz) * g.py * g.px : 0;
    const long long nyr = GT::AY ? (long long)g.nz * (g.py - g.ny) * g.px : 0;
    const long long nxr = (long long)g.nz * g.ny * (g.px - g.nx);
    const long long per = nzr + nyr + nxr;
    const int comp = (int)(q / per);
    long long r = q - comp * per;
    int pi, pj, pk;  // padded coordinates of the guard point
    if (r < nzr) {
        const long long plane = (long long)g.py * g.px;
        const int b = (int)(r / plane);
        const long long rr = r - b * plane;
        pk = b < g.gz ? b : g.nz + b;  // low guards, then high guards after the interior
        pj = (int)(rr / g.px);
        pi = (int)(rr - (long long)pj * g.px);
    } else if ((r -= nzr) < nyr) {
        const long long row = (long long)(g.py - g.ny) * g.px;
        pk = (int)(r / row) + g.gz;
        const long long rr = r - (long long)(pk - g.gz) * row;
        const int b = (int)(rr / g.px);
        pj = b < g.gy ? b : g.ny + b;
        pi = (int)(rr - (long long)b * g.px);
    } else {
        r -= nyr;
        const int nxg = g.px - g.nx;
        const long long col = (long long)g.ny * nxg;
        pk = (int)(r / col) + g.gz;
        const long long rr = r - (long long)(pk - g.gz) * col;
        pj = (int)(rr / nxg) + g.gy;
        const int b = (int)(rr - (long long)(pj - g.gy) * nxg);
        pi = b < g.gx ? b : g.nx + b;
    }
    // physical coordinates and their periodic images
    auto img = [](int p, int lo, int n) {
        int v = p - lo;
        v %= n;
        if (v < 0) v += n;
        return v + lo;
    };
    const int si = img(pi, g.gx, g.nx);
    const int sj = GT::AY ? img(pj, g.gy, g.ny) : pj;
    const int sk = GT::AZ ? img(pk, g.gz, g.nz) : pk;
    T* Fc = F + (long long)comp * g.cstride;
    Fc[((long long)pk * g.py + pj) * g.px + pi] = Fc[((long long)sk * g.py + sj) * g.px + si];
}

template <class T, int G> __host__ __device__ inline long long fill_all_count(const Grid& g) {
    using GT = GeomT<G>;
    const long long nzr = GT::AZ ? (long long)(g.pz - g.nz) * g.py * g.px : 0;
    const long long nyr = GT::AY ? (long long)g.nz * (g.py - g.ny) * g.px : 0;
    return 3 * (nzr + nyr + (long long)g.nz * g.ny * (g.px - g.nx));
}

template <class T, int G>
__global__ void fill_all_kernel(Grid g, T* F) {
    const long long n = fill_all_count<T, G>(g);
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        fill_all_point<T, G>(g, F, q);
}

// ---- current fold (adjoint of the fill) ------------------------------------------------
// Pull form: each interior point near a boundary adds the guard values that
// map onto it.  Order z, y (over all padded x), then x with the shear shift at
// t^{n+1/2}: a guard value at (i >= nx, j) belongs at (i - nx, j + dys), split
// (1 - f, f) between rows floor and floor + 1; at (i < 0, j) at (i + nx, j - dys).
template <class T>
__device__ __forceinline__ void fold_z_body(const Grid& g, T* F, int pi, int pj, int zs) {
    const long long plane = (long long)g.px * g.py;
    const int band = g.pz - g.nz;  // receiving interior planes: k in [0, gzh) and [nz - gz, nz)
    const int gzh = g.pz - g.gz - g.nz;  // high guards
    const long long pp = (long long)pj * g.px + pi;
    const int comp = zs / band, b = zs - comp * band;
    T* Fc = F + (long long)comp * g.cstride;
    int k;  // receiving interior plane
    T add = T(0);
    if (b < gzh) {
        k = b;  // from high guard nz + b
        add += Fc[(long long)(g.nz + b + g.gz) * plane + pp];
    } else {
        k = g.nz - g.gz + (b - gzh);  // from low guard k - nz
        add += Fc[(long long)(k - g.nz + g.gz) * plane + pp];
    }
    Fc[(long long)(k + g.gz) * plane + pp] += add;
}

template <class T>
__global__ void fold_z_kernel(Grid g, T* F) {
    // launch: cell_grid(px, py, 3 * band)
    const int pi = blockIdx.x * blockDim.x + threadIdx.x;
    if (pi >= g.px) return;
    fold_z_body<T>(g, F, pi, blockIdx.y, blockIdx.z);
}

template <class T>
__device__ __forceinline__ void fold_y_body(const Grid& g, T* F, int pi, int k, int zs) {
    const int band = g.py - g.ny;
    const int gyh = g.py - g.gy - g.ny;
    {
        const int comp = zs / band, b = zs - comp * band;
        T* Fc = F + (long long)comp * g.cstride;
        long long row = (long long)(k + g.gz) * g.py;
        int j;
        T add;
        if (b < gyh) { j = b; add = Fc[(row + g.ny + b + g.gy) * g.px + pi]; }
        else { j = g.ny - g.gy + (b - gyh); add = Fc[(row + j - g.ny + g.gy) * g.px + pi]; }
        Fc[(row + j + g.gy) * g.px + pi] += add;
    }
}

template <class T>
__global__ void fold_y_kernel(Grid g, T* F) {
    // launch: cell_grid(px, nz, 3 * band)
    const int pi = blockIdx.x * blockDim.x + threadIdx.x;
    if (pi >= g.px) return;
    fold_y_body<T>(g, F, pi, blockIdx.y, blockIdx.z);
}

template <class T, int G>
__device__ __forceinline__ void fold_x_body(const Grid& g, T* F, const StepCtx* __restrict__ ctx, int which, int j, int k,
                                            int zs) {
    using GT = GeomT<G>;
    const int dys_i = ctx->dys_i[which];
    const double dys_f = ctx->dys_f[which];
    const int band = g.px - g.nx;
    const int gxh = g.px - g.gx - g.nx;
    const bool sh = GT::AY && (dys_i != 0 || dys_f != 0.0);
    {
        const int comp = zs / band, b = zs - comp * band;
        T* Fc = F + (long long)comp * g.cstride;
        int i, is, w;  // receiving interior column, source ghost column, side
        if (b < gxh) { i = b; is = g.nx + b; w = 1; }
        else { i = g.nx - g.gx + (b - gxh); is = i - g.nx; w = -1; }
        T add;
        if (sh) {
            // sources: ghost rows js with floor(js + w dys) = j (weight 1-f) or j - 1 (weight f)
            int m;
            double f;
            if (w > 0) { m = dys_i; f = dys_f; }
            else { m = -dys_i; f = -dys_f; if (f < 0.0) { f += 1.0; m -= 1; } }
            int ja = j - m, jb = j - m - 1;
            ja %= g.ny; if (ja < 0) ja += g.ny;
            jb %= g.ny; if (jb < 0) jb += g.ny;
            add = T(1.0 - f) * Fc[g.idx(is, ja, k)] + T(f) * Fc[g.idx(is, jb, k)];
        } else {
            add = Fc[g.idx(is, j, k)];
        }
        Fc[g.idx(i, j, k)] += add;
    }
}

template <class T, int G>
__global__ void fold_x_kernel(Grid g, T* F, const StepCtx* __restrict__ ctx, int which) {
    // launch: cell_grid(ny, nz, 3 * band)
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= g.ny) return;
    fold_x_body<T, G>(g, F, ctx, which, j, blockIdx.y, blockIdx.z);
}

// Shearing box: advect J' along y by v_{s,y} dt / 2 = -s Omega0 x dt / 2 per x
// column (x of each component's location from the box centre), linear
// interpolation, periodic in y: Jn(j) = (1-f) J(j0) + f J(j0+1), j - d = j0 + f.
constexpr int ADVECT_ROWS = 8;  // y rows per thread: the column's shift is computed once
template <class T>
__global__ void ksb_advect_kernel(Grid g, const T* __restrict__ Jin, T* __restrict__ Jout, double sO_, double half_nx,
                                  const StepCtx* __restrict__ ctx) {
    // the shearing + expanding box advects along xi_y by v_{s,y} dt / (2 l_2):
    // the shear times (l_1/l_2)(t^{n+1/2}) (one for the shearing box)
    const double sO = sO_ * ctx->sxe_vf;
    // launch: cell_grid(nx, ceil(ny / ADVECT_ROWS), 3 * nz)
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nx) return;
    const int comp = blockIdx.z / g.nz, k = blockIdx.z - comp * g.nz;
    // the column moves by d = -s Omega0 xc / 2; row j takes y = j - d = j + m + f, 0 <= f < 1
    const double xc = (double)i + (comp == 0 ? 0.5 : 0.0) - half_nx;
    const double md = sO * xc * 0.5;  // -d
    const double fl = floor(md);
    const T f = T(md - fl);
    int m = (int)fmod(fl, (double)g.ny);
    if (m < 0) m += g.ny;
    const T* Jc = Jin + (long long)comp * g.cstride;
    T* Jo = Jout + (long long)comp * g.cstride;
    const int j0 = blockIdx.y * ADVECT_ROWS;
#pragma unroll 4
    for (int jj = 0; jj < ADVECT_ROWS; ++jj) {
        const int j = j0 + jj;
        if (j >= g.ny) break;
        int ja = j + m;
        if (ja >= g.ny) ja -= g.ny;
        int jb = ja + 1;
        if (jb >= g.ny) jb -= g.ny;
        Jo[g.idx(i, j, k)] = (T(1) - f) * Jc[g.idx(i, ja, k)] + f * Jc[g.idx(i, jb, k)];
    }
}

// Component-wise scaling of a padded 3-component field (guards included) by
// ctx->sxe_pre (which = 0: X^ = ell L^{-1} X at t^n) or ctx->sxe_post (which
// = 1: back to X = L X^ / ell at t^{n+1}).  Launch: cell_grid(cstride, 1, 3).
template <class T>
__global__ void scale3_kernel(T* F, long long cstride, const StepCtx* __restrict__ ctx, int which) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= cstride) return;
    const int comp = blockIdx.z;
    const double f = which == 0 ? ctx->sxe_pre[comp] : ctx->sxe_post[comp];
    F[comp * cstride + q] = T((double)F[comp * cstride + q] * f);
}

// FP32 current: fixed-point int32 sums -> float, flagging sums that reached
// half of the int32 range (the only place a wrap could show).
__global__ void fixed_to_float_kernel(long long n, const int* __restrict__ src, float* __restrict__ dst, double unit,
                                      int* err) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int v = src[q];
        if (v > (1 << 30) || v < -(1 << 30)) atomicOr(err, ERRB_J_RANGE);
        dst[q] = (float)((double)v * unit);
    }
}

// ---- batched grid kernels -----------------------------------------------------------------
// The grid work of many boxes of one kind in one launch each: box b's
// blocks are blockIdx.z in [zoff[b], zoff[b+1]) (its slabs along the launch's
// z index), x and y cover the largest box and blocks beyond a box's own
// extent return.  The bodies are the single-box kernels', so results are the
// same bit for bit.  Descriptors and offset tables live in device memory
// (fixed for the life of a batch).
template <class T> struct FieldBox {
    Grid g;
    T* E;
    T* B;
    T* J;         // the current the field update reads (the folded one)
    int* Jint;    // FP32: the fixed-point current (null in FP64)
    StepCtx* ctx;
    int* err;
    double fx_unit;
    CtxConst cc;
};

__device__ __forceinline__ int box_of_z(const int* __restrict__ zoff, int n, int z) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (zoff[mid] <= z) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Start of a step for every box: the step context and the current reset.
// Launch: grid (any, n); block row b serves box b.
template <class T>
__global__ void multi_pre_kernel(const FieldBox<T>* __restrict__ fb, int n) {
    const int b = blockIdx.y;
    if (b >= n) return;
    const FieldBox<T>& f = fb[b];
    if (blockIdx.x == 0 && threadIdx.x == 0) ctx_update(f.ctx, f.cc);
    const long long m = 3ll * f.g.cstride;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < m; q += (long long)gridDim.x * blockDim.x) {
        if (sizeof(T) == 4) f.Jint[q] = 0;
        else f.J[q] = T(0);
    }
}

// FP32 current: fixed point -> float for every box.  Launch: grid (any, n).
__global__ inline void multi_fixed_to_float_kernel(const FieldBox<float>* __restrict__ fb, int n) {
    const int b = blockIdx.y;
    if (b >= n) return;
    const FieldBox<float>& f = fb[b];
    const long long m = 3ll * f.g.cstride;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < m; q += (long long)gridDim.x * blockDim.x) {
        const int v = f.Jint[q];
        if (v > (1 << 30) || v < -(1 << 30)) atomicOr(f.err, ERRB_J_RANGE);
        f.J[q] = (float)((double)v * f.fx_unit);
    }
}

// which field: 0 E, 1 B, 2 J
template <class T> __device__ __forceinline__ T* field_of(const FieldBox<T>& f, int which) {
    return which == 0 ? f.E : (which == 1 ? f.B : f.J);
}

template <class T, int G, bool CURL_E>
__global__ void multi_curl_kernel(const FieldBox<T>* __restrict__ fb, const int* __restrict__ zoff, int n, int which) {
    const int b = box_of_z(zoff, n, blockIdx.z);
    const FieldBox<T>& f = fb[b];
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z - zoff[b];
    if (i >= f.g.nx || j >= f.g.ny) return;
    curl_update_body<T, G, CURL_E>(f.g, CURL_E ? f.E : f.B, CURL_E ? f.B : f.E, CURL_E ? nullptr : f.J, f.ctx, which, i, j,
                                   k);
}

// One-pass guard fill (fill_all_point) of field `which` for every box.
// Launch: grid (any, n); block row b serves box b.
template <class T, int G>
__global__ void multi_fill_all_kernel(const FieldBox<T>* __restrict__ fb, int n, int which) {
    const int b = blockIdx.y;
    if (b >= n) return;
    const FieldBox<T>& f = fb[b];
    const long long m = fill_all_count<T, G>(f.g);
    T* F = field_of(f, which);
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < m; q += (long long)gridDim.x * blockDim.x)
        fill_all_point<T, G>(f.g, F, q);
}

template <class T>
__global__ void multi_fold_z_kernel(const FieldBox<T>* __restrict__ fb, const int* __restrict__ zoff, int n) {
    const int b = box_of_z(zoff, n, blockIdx.z);
    const FieldBox<T>& f = fb[b];
    const int pi = blockIdx.x * blockDim.x + threadIdx.x, pj = blockIdx.y;
    if (pi >= f.g.px || pj >= f.g.py) return;
    fold_z_body<T>(f.g, f.J, pi, pj, blockIdx.z - zoff[b]);
}

template <class T>
__global__ void multi_fold_y_kernel(const FieldBox<T>* __restrict__ fb, const int* __restrict__ zoff, int n) {
    const int b = box_of_z(zoff, n, blockIdx.z);
    const FieldBox<T>& f = fb[b];
    const int pi = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (pi >= f.g.px || k >= f.g.nz) return;
    fold_y_body<T>(f.g, f.J, pi, k, blockIdx.z - zoff[b]);
}

template <class T, int G>
__global__ void multi_fold_x_kernel(const FieldBox<T>* __restrict__ fb, const int* __restrict__ zoff, int n) {
    const int b = box_of_z(zoff, n, blockIdx.z);
    const FieldBox<T>& f = fb[b];
    const int j = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (j >= f.g.ny || k >= f.g.nz) return;
    fold_x_body<T, G>(f.g, f.J, f.ctx, 1, j, k, blockIdx.z - zoff[b]);
}

// ---- host <-> padded layout -----------------------------------------------------------
template <class T>
__global__ void scatter_field_kernel(Grid g, const double* __restrict__ src, T* __restrict__ dst) {
    long long n = 3ll * g.nx * g.ny * g.nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        int i = (int)(q % g.nx);
        long long r = q / g.nx;
        int j = (int)(r % g.ny);
        r /= g.ny;
        int k = (int)(r % g.nz);
        int comp = (int)(r / g.nz);
        dst[(long long)comp * g.cstride + g.idx(i, j, k)] = T(src[q]);
    }
}

template <class T>
__global__ void gather_field_kernel(Grid g, const T* __restrict__ src, double* __restrict__ dst) {
    long long n = 3ll * g.nx * g.ny * g.nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        int i = (int)(q % g.nx);
        long long r = q / g.nx;
        int j = (int)(r % g.ny);
        r /= g.ny;
        int k = (int)(r % g.nz);
        int comp = (int)(r / g.nz);
        dst[q] = (double)src[(long long)comp * g.cstride + g.idx(i, j, k)];
    }
}

template <class T>
__global__ void uniform_field_kernel(Grid g, T* dst, double v0, double v1, double v2) {
    long long n = 3ll * g.cstride;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        int comp = (int)(q / g.cstride);
        dst[q] = T(comp == 0 ? v0 : (comp == 1 ? v1 : v2));
    }
}

// ---- FP64 reductions -------------------------------------------------------------------
// Sum of squares of each component over interior cells: block partials in
// `partial` ([gridDim.x][3]), then one block adds them (deterministic order).
template <class T>
__global__ void sumsq_partial_kernel(Grid g, const T* __restrict__ F, double* __restrict__ partial) {
    __shared__ double red[3][32];
    double acc[3] = {0.0, 0.0, 0.0};
    long long n = (long long)g.nx * g.ny * g.nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        int i = (int)(q % g.nx);
        long long r = q / g.nx;
        int j = (int)(r % g.ny);
        int k = (int)(r / g.ny);
        long long c0 = g.idx(i, j, k);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double v = (double)F[c * g.cstride + c0];
            acc[c] += v * v;
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double v = acc[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
        partial[blockIdx.x * 3 + threadIdx.x] = s;
    }
}

__global__ void sum_partials_kernel(const double* __restrict__ partial, int nblocks, int width, double* __restrict__ out) {
    // one thread per output column, sequential over blocks: deterministic
    int c = threadIdx.x;
    if (c >= width) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partial[b * width + c];
    out[c] = s;
}

}  // namespace pic
