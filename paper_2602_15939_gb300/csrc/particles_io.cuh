// particles_io.cuh -- loading, re-binning and read-back of tile-sorted
// particles, plus per-step counter bookkeeping and the kinetic-energy sum.
// None of this is on the per-step hot path except finalize_kernel.
#pragma once

#include "particle.cuh"

namespace pic {

// Wrap an absolute coordinate into [0, n) and split it into cell + offset.
template <class T> __device__ inline void split_coord(double x, int n, int& c, T& o) {
    double w = x - floor(x / (double)n) * (double)n;
    if (w >= (double)n) w -= (double)n;
    if (w < 0.0) w = 0.0;
    double f = floor(w);
    c = (int)f;
    if (c >= n) c = n - 1;
    double r = w - f;
    o = T(r);
    if (o >= T(1)) { o = T(0); c += 1; if (c >= n) c = 0; }
}

// Tile counters of a load, one atomic per group of lanes with the same tile
// (loaded particles usually come in cell or tile order, so most of a warp
// shares one counter).  Returns the lane's slot: the counter's old value
// plus the lane's rank in its group.
__device__ __forceinline__ int tile_count_add(int* __restrict__ count, int t) {
    const unsigned act = __activemask();
    const unsigned grp = __match_any_sync(act, t);
    const int lane = (int)(threadIdx.x & 31u);
    const int leader = __ffs(grp) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count + t, __popc(grp));
    base = __shfl_sync(grp, base, leader);
    return base + __popc(grp & ((1u << lane) - 1u));
}

// Pass 1 of a load: per particle, its tile; per tile, a count.
template <class T, int G>
__global__ void load_bin_kernel(long long n, const double* __restrict__ x, Tiling tl, Grid g, int* __restrict__ count) {
    using GT = GeomT<G>;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        int ci, cj = 0, ck = 0;
        T o;
        split_coord<T>(x[3 * q + 0], g.nx, ci, o);
        if (GT::AY) split_coord<T>(x[3 * q + 1], g.ny, cj, o);
        if (GT::AZ) split_coord<T>(x[3 * q + 2], g.nz, ck, o);
        tile_count_add(count, tile_of<G>(tl, ci, cj, ck));
    }
}

// Pass 2: write each particle to a slot of its tile (order within a tile is
// arbitrary).
template <class T, int G>
__global__ void load_scatter_kernel(long long n, long long q0, const double* __restrict__ x, const double* __restrict__ u,
                                    const uint32_t* __restrict__ id, const double* __restrict__ dr, Tiling tl, Grid g,
                                    int* __restrict__ fill, long long tcap, PView<T> v, bool has_dr) {
    // particles q0 + q of the caller's arrays (x, u, id, dr hold q = 0..n-1)
    using GT = GeomT<G>;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        Particle<T> p;
        p.cj = 0; p.ck = 0;
        split_coord<T>(x[3 * q + 0], g.nx, p.ci, p.o[0]);
        if (GT::AY) split_coord<T>(x[3 * q + 1], g.ny, p.cj, p.o[1]); else p.o[1] = T(0.5);
        if (GT::AZ) split_coord<T>(x[3 * q + 2], g.nz, p.ck, p.o[2]); else p.o[2] = T(0.5);
        p.u[0] = T(u[3 * q]); p.u[1] = T(u[3 * q + 1]); p.u[2] = T(u[3 * q + 2]);
        p.id = id ? id[q] : (uint32_t)(q0 + q);
        if (has_dr) {
            p.dr[0] = dr ? T(dr[3 * q]) : T(0);
            p.dr[1] = dr ? T(dr[3 * q + 1]) : T(0);
            p.dr[2] = dr ? T(dr[3 * q + 2]) : T(0);
        }
        const int t = tile_of<G>(tl, p.ci, p.cj, p.ck);
        const int s = tile_count_add(fill, t);
        store_particle<T, G>(v, (long long)t * tcap + s, has_dr, p);
    }
}

// Device Maxwellian loader: slot r of tile t holds particle r of the tile's
// cells in order, ppc per cell.  blockIdx.x is the tile; the gridDim.y CTAs
// of a tile share its particles (small boxes still fill the GPU).  Positions uniform in the cell, momenta
// Maxwell-Juettner(theta) + drift + Gaussian noise (Box-Muller), all from
// Philox keyed on (id, seed).
template <class T, int G>
__global__ void maxwellian_kernel(Tiling tl, Grid g, int ppc, double theta, double c, double dx_, double dy_, double dz_,
                                  double noise, uint32_t seed, uint32_t id_base, long long tcap, PView<T> v, bool has_dr,
                                  int* __restrict__ count) {
    using GT = GeomT<G>;
    const int t = blockIdx.x;
    const int ti = t % tl.ntx, tj = (t / tl.ntx) % tl.nty, tk = t / (tl.ntx * tl.nty);
    const int t0x = ti * tl.tx, t0y = tj * tl.ty, t0z = tk * tl.tz;
    const int ex = min(tl.tx, g.nx - t0x), ey = GT::AY ? min(tl.ty, g.ny - t0y) : 1, ez = GT::AZ ? min(tl.tz, g.nz - t0z) : 1;
    const int ncell = ex * ey * ez;
    const int n = ncell * ppc;
    for (int r = blockIdx.y * blockDim.x + threadIdx.x; r < n; r += blockDim.x * gridDim.y) {
        int lc = r / ppc, pc = r % ppc;
        int a = lc % ex, b = (lc / ex) % ey, cc = lc / (ex * ey);
        Particle<T> p;
        p.ci = t0x + a; p.cj = GT::AY ? t0y + b : 0; p.ck = GT::AZ ? t0z + cc : 0;
        long long cell_lin = ((long long)p.ck * g.ny + p.cj) * g.nx + p.ci;
        p.id = id_base + (uint32_t)(cell_lin * ppc + pc);
        U4 rp = draw(p.id, seed, 0, TAG_LOADPOS, 0u);
        p.o[0] = T(u01(rp.x[0]));
        p.o[1] = GT::AY ? T(u01(rp.x[1])) : T(0.5);
        p.o[2] = GT::AZ ? T(u01(rp.x[2])) : T(0.5);
        if (p.o[0] >= T(1)) p.o[0] = T(0);
        if (p.o[1] >= T(1)) p.o[1] = T(0);
        if (p.o[2] >= T(1)) p.o[2] = T(0);
        double ux = 0.0, uy = 0.0, uz = 0.0;
        if (theta > 0.0) sample_mj(p.id, seed, 0, theta, c, ux, uy, uz);
        ux += dx_; uy += dy_; uz += dz_;
        if (noise > 0.0) {
            U4 rn = draw(p.id, seed, 0, TAG_LOADNOI, 0u);
            double r1 = sqrt(-2.0 * log(u01(rn.x[0]))), r2 = sqrt(-2.0 * log(u01(rn.x[2])));
            double a1 = 6.283185307179586 * u01(rn.x[1]), a2 = 6.283185307179586 * u01(rn.x[3]);
            ux += noise * r1 * cos(a1);
            uy += noise * r1 * sin(a1);
            uz += noise * r2 * cos(a2);
        }
        p.u[0] = T(ux); p.u[1] = T(uy); p.u[2] = T(uz);
        p.dr[0] = p.dr[1] = p.dr[2] = T(0);
        store_particle<T, G>(v, (long long)t * tcap + r, has_dr, p);
    }
    if (threadIdx.x == 0 && blockIdx.y == 0) count[t] = n;
}

// Copy tile t's particles (front and back segments) to double arrays at
// offset off[t]: absolute positions, momenta, ids, displacements.
template <class T, int G>
__global__ void compact_kernel(Tiling tl, Grid g, PView<T> v, const int* __restrict__ stay, const int* __restrict__ arr,
                               long long tcap, const long long* __restrict__ off, int t_first, long long o_first, bool has_dr,
                               double* __restrict__ x, double* __restrict__ u, uint32_t* __restrict__ id,
                               double* __restrict__ dr) {
    // tiles t_first + blockIdx.x; output index off[t] - o_first + i
    const int t = t_first + blockIdx.x;
    const int nst = stay[t], nar = arr[t];
    const long long base = (long long)t * tcap;
    for (int i = threadIdx.x; i < nst + nar; i += blockDim.x) {
        long long slot = i < nst ? base + i : base + tcap - nar + (i - nst);
        Particle<T> p;
        load_particle<T, G>(v, slot, has_dr, p);
        long long o = off[t] - o_first + i;
        if (x) {
            x[3 * o + 0] = (double)p.ci + (double)p.o[0];
            x[3 * o + 1] = (double)p.cj + (double)p.o[1];
            x[3 * o + 2] = (double)p.ck + (double)p.o[2];
        }
        if (u) { u[3 * o] = (double)p.u[0]; u[3 * o + 1] = (double)p.u[1]; u[3 * o + 2] = (double)p.u[2]; }
        if (id) id[o] = p.id;
        if (dr) {
            dr[3 * o] = has_dr ? (double)p.dr[0] : 0.0;
            dr[3 * o + 1] = has_dr ? (double)p.dr[1] : 0.0;
            dr[3 * o + 2] = has_dr ? (double)p.dr[2] : 0.0;
        }
    }
}

template <class T, int G>
__global__ void compact_loose_kernel(PView<T> v, const int* __restrict__ lcount, long long lcap, long long off0, bool has_dr,
                                     double* __restrict__ x, double* __restrict__ u, uint32_t* __restrict__ id,
                                     double* __restrict__ dr) {
    long long n = *lcount;
    if (n > lcap) n = lcap;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        Particle<T> p;
        load_particle<T, G>(v, i, has_dr, p);
        long long o = off0 + i;
        if (x) {
            x[3 * o + 0] = (double)p.ci + (double)p.o[0];
            x[3 * o + 1] = (double)p.cj + (double)p.o[1];
            x[3 * o + 2] = (double)p.ck + (double)p.o[2];
        }
        if (u) { u[3 * o] = (double)p.u[0]; u[3 * o + 1] = (double)p.u[1]; u[3 * o + 2] = (double)p.u[2]; }
        if (id) id[o] = p.id;
        if (dr) {
            dr[3 * o] = has_dr ? (double)p.dr[0] : 0.0;
            dr[3 * o + 1] = has_dr ? (double)p.dr[1] : 0.0;
            dr[3 * o + 2] = has_dr ? (double)p.dr[2] : 0.0;
        }
    }
}

// Particles whose id is remainder mod modulus (a fixed subset that can be
// followed from step to step), appended in any order up to max_out.
template <class T, int G>
__global__ void sample_kernel(Tiling tl, PView<T> v, const int* __restrict__ stay, const int* __restrict__ arr, long long tcap,
                              PView<T> lv, const int* __restrict__ lcount, long long lcap, uint32_t modulus,
                              uint32_t remainder, bool has_dr, long long max_out, unsigned long long* __restrict__ count,
                              double* __restrict__ x, double* __restrict__ u, uint32_t* __restrict__ id,
                              double* __restrict__ dr) {
    for (int t = blockIdx.x; t < tl.ntiles + 1; t += gridDim.x) {
        const bool loose = t == tl.ntiles;
        long long n;
        int nst = 0, nar = 0;
        if (loose) {
            n = *lcount;
            if (n > lcap) n = lcap;
        } else {
            nst = stay[t];
            nar = arr[t];
            n = nst + nar;
        }
        const long long base = (long long)t * tcap;
        for (long long i = threadIdx.x; i < n; i += blockDim.x) {
            const long long slot = loose ? i : (i < nst ? base + i : base + tcap - nar + (i - nst));
            const PView<T>& src = loose ? lv : v;
            const uint32_t pid = src.id[slot];
            if (pid % modulus != remainder) continue;
            const unsigned long long o = atomicAdd(count, 1ull);
            if ((long long)o >= max_out) continue;
            Particle<T> p;
            load_particle<T, G>(src, slot, has_dr, p);
            x[3 * o + 0] = (double)p.ci + (double)p.o[0];
            x[3 * o + 1] = (double)p.cj + (double)p.o[1];
            x[3 * o + 2] = (double)p.ck + (double)p.o[2];
            u[3 * o] = (double)p.u[0];
            u[3 * o + 1] = (double)p.u[1];
            u[3 * o + 2] = (double)p.u[2];
            id[o] = p.id;
            dr[3 * o] = has_dr ? (double)p.dr[0] : 0.0;
            dr[3 * o + 1] = has_dr ? (double)p.dr[1] : 0.0;
            dr[3 * o + 2] = has_dr ? (double)p.dr[2] : 0.0;
        }
    }
}

// After the particle kernels of a step: clamp each tile's arrival count to
// the claims that got a slot (failed claims over-count), clamp the loose
// count to the list capacity, and zero the counters of the consumed buffer,
// which the next step writes.
// occ_max keeps the largest tile occupancy since it was last reset, occ_loose
// the loose count after the step (the library's capacity check reads them).
__global__ void finalize_kernel(int ntiles, long long tcap, const int* __restrict__ stay_in, int* __restrict__ arr_in,
                                       int* __restrict__ arr_out, int* __restrict__ lcount_in, int* __restrict__ lcount_out,
                                       long long lcap, int* err, int* __restrict__ occ_max,
                                       int* __restrict__ occ_loose) {
    int mx = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x) {
        const int cnt = stay_in[t] + arr_in[t];
        mx = max(mx, cnt);
        int room = (int)(tcap - cnt);
        if (arr_out[t] > room) arr_out[t] = room;
        arr_in[t] = 0;
    }
    for (int sh = 16; sh > 0; sh >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, sh));
    if ((threadIdx.x & 31) == 0 && mx > 0) atomicMax(occ_max, mx);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int lc = *lcount_out;
        if (lc > lcap) { atomicOr(err, ERRB_LOOSE_OVERFLOW); lc = (int)lcap; *lcount_out = lc; }
        *occ_loose = lc;
        *lcount_in = 0;
    }
}

// Re-lay tile-sorted particles out with another capacity per tile: tile t's
// stayers and arrivals in buffer `in` (capacity tcap_in) become the first
// stay_out[t] slots of tile t in `out` (capacity tcap_out).
template <class T, int G>
// stay_in and stay_out may be the same array (a re-layout within one buffer
// pair), so neither is declared __restrict__.
__global__ void regrow_kernel(PView<T> in, PView<T> out, const int* stay_in, const int* __restrict__ arr_in,
                              long long tcap_in, long long tcap_out, int* stay_out, bool has_dr) {
    const int t = blockIdx.x;
    const int nst = stay_in[t], nar = arr_in[t], n = nst + nar;
    const long long bi = (long long)t * tcap_in, bo = (long long)t * tcap_out;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const long long slot = i < nst ? bi + i : bi + tcap_in - nar + (i - nst);
        Particle<T> p;
        load_particle<T, G>(in, slot, has_dr, p);
        store_particle<T, G>(out, bo + i, has_dr, p);
    }
    __syncthreads();  // stay_in may be stay_out: every thread has read it
    if (threadIdx.x == 0) stay_out[t] = n;
}

// Regroup: tile t's particles of one buffer (stayers, then arrivals) are
// written to the front of its range in the other buffer, ordered by cell (a
// counting sort in shared memory; the order within a cell is arbitrary).  A
// warp of the particle kernel then holds the particles of one or two cells:
// its gathers read few distinct words (lanes reading one word share a pass)
// and its adds spread over the current copies.  The order decays as particles
// change cells, so the library repeats this every few steps.  Each array is
// copied in its own pass (coalesced writes; the scattered reads stay within
// the tile's range of that array, which L2 holds).  Shared memory: one counter
// per cell and 4 bytes per slot (tcap < 65536).
constexpr int RG_THREADS = 512;
constexpr int RG_UNROLL = 8;

template <int G> __host__ __device__ constexpr int tile_cells() { return TileDims<G>::TX * TileDims<G>::TY * TileDims<G>::TZ; }

template <class T, int G>
__global__ void __launch_bounds__(RG_THREADS) regroup_kernel(Tiling tl, PView<T> in, PView<T> out, const int* __restrict__ stay_in,
                                                             const int* __restrict__ arr_in, int* __restrict__ stay_out,
                                                             long long tcap, bool has_dr) {
    using GT = GeomT<G>;
    using D = TileDims<G>;
    constexpr int NCELL = tile_cells<G>();
    static_assert(NCELL % 32 == 0 && NCELL <= 1024, "one warp scans the cell counters");
    extern __shared__ __align__(16) unsigned char smem[];
    int* cnt = reinterpret_cast<int*>(smem);                       // [NCELL]
    uint16_t* key = reinterpret_cast<uint16_t*>(cnt + NCELL);      // [tcap] local cell of input i
    uint16_t* src = key + tcap;                                    // [tcap] input index of output j
    const int t = blockIdx.x;
    const int nst = stay_in[t], nar = arr_in[t], n = nst + nar;
    const long long base = (long long)t * tcap;
    const int ti = t % tl.ntx, tj = (t / tl.ntx) % tl.nty, tk = t / (tl.ntx * tl.nty);
    const int t0x = ti * D::TX, t0y = tj * D::TY, t0z = tk * D::TZ;
    auto slot = [&](int i) -> long long { return i < nst ? base + i : base + tcap - nar + (i - nst); };
    for (int c = threadIdx.x; c < NCELL; c += RG_THREADS) cnt[c] = 0;
    __syncthreads();
    // RG_UNROLL independent loads per thread at a time: one tile's CTA must
    // keep many loads in flight for the copy to run near HBM speed
    for (int i0 = threadIdx.x; i0 < n; i0 += RG_THREADS * RG_UNROLL) {
        int w[RG_UNROLL];
#pragma unroll
        for (int u = 0; u < RG_UNROLL; ++u) {
            const int i = i0 + u * RG_THREADS;
            w[u] = i < n ? in.cell[slot(i)] : 0;
        }
#pragma unroll
        for (int u = 0; u < RG_UNROLL; ++u) {
            const int i = i0 + u * RG_THREADS;
            if (i >= n) break;
            int ci, cj, ck;
            CellPack<G>::unpack(w[u], ci, cj, ck);
            int lc = ci - t0x;
            if (GT::AY) lc += (cj - t0y) * D::TX;
            if (GT::AZ) lc += (ck - t0z) * D::TX * D::TY;
            lc = min(max(lc, 0), NCELL - 1);  // a tile's range holds only its own cells
            key[i] = (uint16_t)lc;
            atomicAdd(&cnt[lc], 1);
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // exclusive prefix of the counters, NCELL / 32 per lane
        constexpr int PER = NCELL / 32;
        const int lane = threadIdx.x;
        int loc = 0;
#pragma unroll
        for (int k = 0; k < PER; ++k) loc += cnt[lane * PER + k];
        int incl = loc;
#pragma unroll
        for (int sh = 1; sh < 32; sh <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, sh);
            if (lane >= sh) incl += v;
        }
        int run = incl - loc;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int c = cnt[lane * PER + k];
            cnt[lane * PER + k] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += RG_THREADS) src[atomicAdd(&cnt[key[i]], 1)] = (uint16_t)i;
    __syncthreads();
    auto copy = [&](const auto* a_in, auto* a_out) {
        for (int j0 = threadIdx.x; j0 < n; j0 += RG_THREADS * RG_UNROLL) {
            typename std::remove_pointer<decltype(a_out)>::type v[RG_UNROLL];
#pragma unroll
            for (int u = 0; u < RG_UNROLL; ++u) {
                const int j = j0 + u * RG_THREADS;
                if (j < n) v[u] = a_in[slot(src[j])];
            }
#pragma unroll
            for (int u = 0; u < RG_UNROLL; ++u) {
                const int j = j0 + u * RG_THREADS;
                if (j < n) a_out[base + j] = v[u];
            }
        }
    };
    copy(in.cell, out.cell);
    copy(in.o[0], out.o[0]);
    if (GT::AY) copy(in.o[1], out.o[1]);
    if (GT::AZ) copy(in.o[GT::AY ? 2 : 1], out.o[GT::AY ? 2 : 1]);
    copy(in.u[0], out.u[0]);
    copy(in.u[1], out.u[1]);
    copy(in.u[2], out.u[2]);
    copy(in.id, out.id);
    if (has_dr) {
        copy(in.dr[0], out.dr[0]);
        copy(in.dr[1], out.dr[1]);
        copy(in.dr[2], out.dr[2]);
    }
    if (threadIdx.x == 0) stay_out[t] = n;
}

// Copy the first *count_in entries of a loose list (at most lcap_in).
// count_in and count_out may be the same word (the count is rewritten with
// the value every block reads), so neither is declared __restrict__.
template <class T, int G>
__global__ void copy_loose_kernel(PView<T> in, PView<T> out, const int* count_in, long long lcap_in,
                                  int* count_out, bool has_dr) {
    long long n = *count_in;
    if (n > lcap_in) n = lcap_in;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        Particle<T> p;
        load_particle<T, G>(in, i, has_dr, p);
        store_particle<T, G>(out, i, has_dr, p);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *count_out = (int)n;
}

// Sum of m c^2 (gamma - 1) over the tile-sorted particles and the loose list.
template <class T, int G>
__global__ void kinetic_kernel(Tiling tl, PView<T> v, const int* __restrict__ stay, const int* __restrict__ arr, long long tcap,
                               PView<T> lv, const int* __restrict__ lcount, long long lcap, double c, double m,
                               double* __restrict__ partial) {
    // gamma - 1 = (u/c)^2 / (gamma + 1) per particle in the particles' own
    // precision (no cancellation; FP64 division and square root per particle
    // would cost far more than the pass's memory traffic on this part), summed
    // in FP64; m c^2 is applied once per block
    __shared__ double red[32];
    double acc = 0.0;
    const T ic2 = T(1.0 / (c * c));
    auto term = [&](T ux, T uy, T uz) {
        const T u2 = (ux * ux + uy * uy + uz * uz) * ic2;
        return (double)(u2 / (t_sqrt<T>(T(1) + u2) + T(1)));
    };
    for (int t = blockIdx.x; t < tl.ntiles + 1; t += gridDim.x) {
        if (t < tl.ntiles) {
            const int nst = stay[t], nar = arr[t], n = nst + nar;
            const long long base = (long long)t * tcap;
            auto slot = [&](int i) -> long long { return i < nst ? base + i : base + tcap - nar + (i - nst); };
            // four particles per thread at a time: enough loads in flight to stream u at HBM speed
            constexpr int K = 4;
            for (int i0 = threadIdx.x; i0 < n; i0 += K * blockDim.x) {
                T ux[K], uy[K], uz[K];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const int i = i0 + k * blockDim.x;
                    if (i < n) {
                        const long long sl = slot(i);
                        ux[k] = v.u[0][sl];
                        uy[k] = v.u[1][sl];
                        uz[k] = v.u[2][sl];
                    }
                }
#pragma unroll
                for (int k = 0; k < K; ++k)
                    if (i0 + k * blockDim.x < n) acc += term(ux[k], uy[k], uz[k]);
            }
        } else {
            long long n = *lcount;
            if (n > lcap) n = lcap;
            for (long long i = threadIdx.x; i < n; i += blockDim.x) acc += term(lv.u[0][i], lv.u[1][i], lv.u[2][i]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        partial[blockIdx.x] = m * c * c * s;
    }
}

}  // namespace pic
