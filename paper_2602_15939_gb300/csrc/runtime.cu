// runtime.cu -- host runtime of libpic: the C ABI declared in include/pic.h.
//
// A handle owns one box: padded field arrays (E, B, J, scratch), the tile
// layout, and per species double-buffered SoA particle arrays in tile order.
// pic_step enqueues, per step: the fused particle kernel (one CTA per tile),
// the loose-particle kernel, counter bookkeeping, the current fold (with the
// shearing-periodic shift), the shearing-box current advection, and the box's
// field update with guard fills, all on the handle's stream.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pic.h"
#include "dispatch.h"
#include "fields.cuh"
#include "particles_io.cuh"

using namespace pic;

namespace {

thread_local std::string g_init_error;

constexpr int NTHR = 256;

struct DevSpecies {
    bool loaded = false;
    double q = 0, m = 1;
    long long n = 0;     // particles loaded
    long long tcap = 0;  // slots per tile
    long long lcap = 0;  // loose capacity
    // [buffer][array]: cell, o0, o1, o2, u0, u1, u2, id, d0, d1, d2
    void* arr[2][11] = {};
    void* larr[2][11] = {};
    int* stay[2] = {};
    int* arrv[2] = {};
    int* lcount = nullptr;  // [2]
};

struct EvPair {
    cudaEvent_t a, b;
    int cat;  // 0 particle, 1 other, 2 field
};

struct Prof {
    bool on = false;
    double ms[3] = {0, 0, 0};
    long long launches = 0, particle_launches = 0, particle_steps = 0;
    std::vector<EvPair> pending;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t open = nullptr;
};

}  // namespace

// Shared memory of the particle kernel of variant v (E and B boxes, the
// variant's current copies, barrier and counters).
constexpr size_t MAX_SMEM = 227 * 1024;

template <class T, int G, int V> static size_t smem_v() {
    return SmemLayout<T, G, TILE_VARIANTS[V].nt, TILE_VARIANTS[V].stable, TILE_VARIANTS[V].jc>::bytes;
}

template <class T, int G> static size_t tile_smem_bytes_t(int v) {
    static_assert(N_TILE_VARIANTS == 7, "one entry per tile variant");
    switch (v) {
        case 0: return smem_v<T, G, 0>();
        case 1: return smem_v<T, G, 1>();
        case 2: return smem_v<T, G, 2>();
        case 3: return smem_v<T, G, 3>();
        case 4: return smem_v<T, G, 4>();
        case 6: return smem_v<T, G, 6>();
        default: return smem_v<T, G, 5>();
    }
}

// tg: template geometry (Geom; the 32 x 32-tile planes are FP32 only)
static size_t tile_smem_bytes(bool fp64, int tg, int v) {
    if (fp64) {
        switch (tg) {
            case 0: return tile_smem_bytes_t<double, 0>(v);
            case 1: return tile_smem_bytes_t<double, 1>(v);
            case 5: return tile_smem_bytes_t<double, 5>(v);
            case 6: return tile_smem_bytes_t<double, 6>(v);
            case 7: return tile_smem_bytes_t<double, 7>(v);
            default: return tile_smem_bytes_t<double, 2>(v);
        }
    }
    switch (tg) {
        case 0: return tile_smem_bytes_t<float, 0>(v);
        case 1: return tile_smem_bytes_t<float, 1>(v);
        case 2: return tile_smem_bytes_t<float, 2>(v);
        case 3: return tile_smem_bytes_t<float, 3>(v);
        case 4: return tile_smem_bytes_t<float, 4>(v);
        case 5: return tile_smem_bytes_t<float, 5>(v);
        case 6: return tile_smem_bytes_t<float, 6>(v);
        default: return tile_smem_bytes_t<float, 7>(v);
    }
}

// Variant used when the configuration leaves the choice to the library
// (pic_autotune refines it for a given box).
static int default_variant(bool fp64, int tg) { return default_tile_variant(fp64, tg); }

// Steps between regroups of the particles by cell (0: never).  FP64 boxes do
// not regroup: the order of their current's floating-point adds would then
// vary from run to run.
static int default_regroup_interval(bool fp64, int tg) { return fp64 ? 0 : (plane_of(tg) == G3D ? 3 : 0); }

struct pic_handle {
    pic_config cfg;
    int geom = 0;  // 0 3D, 1 2D-XY, 2 2D-XZ
    int tg = 0;    // template geometry of the particle kernels: geom, or a 2D plane with 32 x 32 or 8 x 8 tiles
    bool fp64 = false;
    size_t esz = 4;
    Grid g;
    Tiling tl;
    int push = PUSH_BORIS, esc = ESC_NONE;
    KernelSet ks{};
    const void* tile_fn = nullptr;
    int tile_variant = 1;  // index into TILE_VARIANTS
    int tile_threads = 512;
    size_t smem_bytes = 0;
    // fields
    void* E = nullptr;
    void* B = nullptr;
    void* J = nullptr;
    void* Jtmp = nullptr;
    int* Jint = nullptr;  // FP32: fixed-point current the particle kernels add into
    void* Jcur = nullptr; // the current the field update uses (J, or Jtmp after the shearing-box advection)
    StepCtx* ctx = nullptr;  // device-resident per-step scalars
    CtxConst cc{};
    // CUDA graphs of two consecutive steps, one per starting particle buffer
    bool graphs_on = true;
    bool graph_ok[2] = {false, false};
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    long long graph_kernels = 0;  // kernels in one two-step graph
    void* Es = nullptr;  // shearing box: saved X^n
    void* Bs = nullptr;
    void* Ec = nullptr;  // shearing box: alternate iterate
    void* Bc = nullptr;
    double* stage = nullptr;  // host-layout staging [3][nz][ny][nx] doubles
    size_t stage_elems = 0;
    double* partial = nullptr;  // reduction partials
    int partial_blocks = 0;
    int* err = nullptr;
    unsigned long long* counters = nullptr;
    CUtensorMap tmE;
    CUtensorMap tmB;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool batched = false;  // stepped by a pic_batch; pic_step refuses
    int since_check = 0;   // steps since the last tile-capacity check
    int regroup_every = 0;  // regroup the particles by cell every this many steps (0: never)
    int since_regroup = 0;  // steps since the last regroup (or load)
    long long regrows = 0; // tile re-layouts so far
    // asynchronous occupancy snapshot: per species [stay x ntiles, arrivals x
    // ntiles, loose count] of the buffer current when it was taken
    int* occ_dev = nullptr;   // largest tile occupancy of each species since the last check, then each loose count
    int* occ_host = nullptr;  // pinned, two slots
    cudaEvent_t occ_ev[2] = {nullptr, nullptr};
    bool occ_pending[2] = {false, false};
    int occ_next = 0;         // slot of the next snapshot (the older one)
    int check_every = 8;      // steps between capacity checks (0: none)
    bool check_block = true;  // wait for the older snapshot (bounds the host's lead)
    int buf = 0;  // particle buffer holding the current state
    long long step = 0;
    DevSpecies sp[PIC_MAX_SPECIES];
    int nsp_loaded = 0;
    Prof prof;
    std::string last_error;
};

// ---- helpers ----------------------------------------------------------------------------

static pic_status fail(pic_handle* h, pic_status st, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h) h->last_error = buf;
    else g_init_error = buf;
    return st;
}

#define CK(call)                                                                                       \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            return fail(h, e_ == cudaErrorMemoryAllocation ? PIC_ERR_OOM : PIC_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                            \
    } while (0)

static int grid_blocks(long long n) {
    long long b = (n + NTHR - 1) / NTHR;
    if (b < 1) b = 1;
    if (b > 152 * 16) b = 152 * 16;
    return (int)b;
}

// Device-time accounting: event pairs recorded on the handle's stream around
// each kernel group, resolved later (pic_get_profile), so timing never
// synchronises the stream.
static cudaEvent_t prof_event(pic_handle* h) {
    if (!h->prof.pool.empty()) {
        cudaEvent_t e = h->prof.pool.back();
        h->prof.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
static void prof_begin(pic_handle* h) {
    if (!h->prof.on) return;
    h->prof.open = prof_event(h);
    cudaEventRecord(h->prof.open, h->stream);
}
static void prof_end(pic_handle* h, int cat) {
    if (!h->prof.on || !h->prof.open) return;
    cudaEvent_t b = prof_event(h);
    cudaEventRecord(b, h->stream);
    h->prof.pending.push_back(EvPair{h->prof.open, b, cat});
    h->prof.open = nullptr;
}
static void prof_resolve(pic_handle* h) {
    for (const EvPair& p : h->prof.pending) {
        cudaEventSynchronize(p.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p.a, p.b);
        h->prof.ms[p.cat] += ms;
        h->prof.pool.push_back(p.a);
        h->prof.pool.push_back(p.b);
    }
    h->prof.pending.clear();
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                                  const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static pic_status encode_field_map(pic_handle* h, CUtensorMap* map, void* base) {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p)
            return fail(h, PIC_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
        fn = (EncodeTiledFn)p;
    }
    const Grid& g = h->g;
    cuuint64_t dims[4] = {(cuuint64_t)g.px, (cuuint64_t)g.py, (cuuint64_t)g.pz, 3};
    cuuint64_t strides[3] = {(cuuint64_t)g.px * h->esz, (cuuint64_t)g.px * g.py * h->esz, (cuuint64_t)g.cstride * h->esz};
    cuuint32_t box[4] = {(cuuint32_t)h->tl.bx, (cuuint32_t)h->tl.by, (cuuint32_t)h->tl.bz, 3};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = fn(map, h->fp64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box,
                    estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(h, PIC_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return PIC_OK;
}

// ---- field kernel launchers ----------------------------------------------------------------

// Guard fill of a 3-component field.  The x-pass takes the shearing shift
// from the step context (ctx_which = 0, 1, 2 for t, t+1/2, t+1) during a
// step, or an explicit shift (ctx_which < 0) outside of one.
template <class T, int G> static void fill_guards_t(pic_handle* h, T* F, int ctx_which, double dys = 0.0) {
    const Grid& g = h->g;
    int di = 0;
    double df = 0.0;
    if (ctx_which < 0 && dys != 0.0) {
        di = (int)std::floor(dys);
        df = dys - di;
        di %= g.ny;
    }
    const bool shearing = h->cfg.box == PIC_BOX_SHEAR || h->cfg.box == PIC_BOX_SHEAR_EXPAND;
    const StepCtx* ctx = (ctx_which >= 0 && shearing) ? h->ctx : nullptr;
    fill_x_kernel<T, G><<<cell_grid(g.ny, g.nz, 3ll * (g.px - g.nx)), CELL_THREADS, 0, h->stream>>>(
        g, F, 3, di, df, ctx, ctx_which < 0 ? 0 : ctx_which);
    h->prof.launches++;
    if (GeomT<G>::AY) {
        fill_y_kernel<T><<<cell_grid(g.px, g.nz, 3ll * (g.py - g.ny)), CELL_THREADS, 0, h->stream>>>(g, F, 3);
        h->prof.launches++;
    }
    if (GeomT<G>::AZ) {
        fill_z_kernel<T><<<cell_grid(g.px, g.py, 3ll * (g.pz - g.nz)), CELL_THREADS, 0, h->stream>>>(g, F, 3);
        h->prof.launches++;
    }
}

// Current fold with the shift at t^{n+1/2} (step context slot 1).
template <class T, int G> static void fold_current_t(pic_handle* h, T* J) {
    const Grid& g = h->g;
    if (GeomT<G>::AZ) {
        fold_z_kernel<T><<<cell_grid(g.px, g.py, 3ll * (g.pz - g.nz)), CELL_THREADS, 0, h->stream>>>(g, J);
        h->prof.launches++;
    }
    if (GeomT<G>::AY) {
        fold_y_kernel<T><<<cell_grid(g.px, g.nz, 3ll * (g.py - g.ny)), CELL_THREADS, 0, h->stream>>>(g, J);
        h->prof.launches++;
    }
    fold_x_kernel<T, G><<<cell_grid(g.ny, g.nz, 3ll * (g.px - g.nx)), CELL_THREADS, 0, h->stream>>>(g, J, h->ctx, 1);
    h->prof.launches++;
}

template <class T, int G> static void curl_t(pic_handle* h, bool curlE, const void* in, void* out, const void* J, int which) {
    const dim3 grid = cell_grid(h->g.nx, h->g.ny, h->g.nz);
    if (curlE)
        curl_update_kernel<T, G, true><<<grid, CELL_THREADS, 0, h->stream>>>(h->g, (const T*)in, (T*)out, (const T*)J,
                                                                            h->ctx, which);
    else
        curl_update_kernel<T, G, false><<<grid, CELL_THREADS, 0, h->stream>>>(h->g, (const T*)in, (T*)out, (const T*)J,
                                                                             h->ctx, which);
    h->prof.launches++;
}

// Host-side shearing shift and expansion factors (diagnostics, set-up fills);
// the step itself takes them from the device context.
static double shear_shift(const pic_handle* h, double t) {
    const pic_config& c = h->cfg;
    if (c.box != PIC_BOX_SHEAR && c.box != PIC_BOX_SHEAR_EXPAND) return 0.0;
    double I = t;  // shearing + expanding box: int_0^t l_1/l_2 dt'
    if (c.box == PIC_BOX_SHEAR_EXPAND) {
        const double dr = c.expand_rate[0] - c.expand_rate[1];
        I = dr == 0.0 ? t : std::expm1(dr * t) / dr;
    }
    double ny = (double)c.ny;
    double d = std::fmod(c.s_shear * c.Omega0 * (double)c.nx * I, ny);
    if (d < 0) d += ny;
    return d;
}

static void lvals(const pic_handle* h, double t, double l[3]) {
    const bool ex = h->cfg.box == PIC_BOX_EXPAND || h->cfg.box == PIC_BOX_SHEAR_EXPAND;
    for (int a = 0; a < 3; ++a) l[a] = ex ? std::exp(h->cfg.expand_rate[a] * t) : 1.0;
}

template <class T, int G> static void fill_all_t(pic_handle* h, double t) {
    double d = shear_shift(h, t);
    fill_guards_t<T, G>(h, (T*)h->E, -1, d);
    fill_guards_t<T, G>(h, (T*)h->B, -1, d);
}

// Field update of one step, after h->Jcur holds the folded current.
template <class T, int G> static void field_step_t(pic_handle* h) {
    const Grid& g = h->g;
    const double c = h->cfg.c;
    if (h->cfg.box == PIC_BOX_SHEAR || h->cfg.box == PIC_BOX_SHEAR_EXPAND) {
        const size_t bytes = (size_t)3 * g.cstride * h->esz;
        const bool sxe = h->cfg.box == PIC_BOX_SHEAR_EXPAND;
        const dim3 sgrid = cell_grid(g.cstride, 1, 3);
        if (sxe) {
            // the shearing + expanding box sweeps X^ = ell L^{-1} X at t^n
            scale3_kernel<T><<<sgrid, CELL_THREADS, 0, h->stream>>>((T*)h->E, g.cstride, h->ctx, 0);
            scale3_kernel<T><<<sgrid, CELL_THREADS, 0, h->stream>>>((T*)h->B, g.cstride, h->ctx, 0);
            h->prof.launches += 2;
        }
        // guards of X^n at t^{n+1/2}, then save X^n
        fill_guards_t<T, G>(h, (T*)h->E, 1);
        fill_guards_t<T, G>(h, (T*)h->B, 1);
        cudaMemcpyAsync(h->Es, h->E, bytes, cudaMemcpyDeviceToDevice, h->stream);
        cudaMemcpyAsync(h->Bs, h->B, bytes, cudaMemcpyDeviceToDevice, h->stream);
        const int N = h->cfg.fp_iters;
        const void* Ek = h->Es;
        const void* Bk = h->Bs;
        for (int k = 1; k <= N; ++k) {
            bool to_main = ((N - k) % 2) == 0;
            T* Eo = (T*)(to_main ? h->E : h->Ec);
            T* Bo = (T*)(to_main ? h->B : h->Bc);
            ksb_sweep_kernel<T, G><<<cell_grid(g.nx, g.ny, g.nz), CELL_THREADS, 0, h->stream>>>(g, (const T*)h->Es, (const T*)h->Bs, (const T*)Ek,
                                                                            (const T*)Bk, (const T*)h->Jcur, Eo, Bo, c,
                                                                            h->cfg.s_shear * h->cfg.Omega0, 0.5 * g.nx,
                                                                            h->ctx);
            h->prof.launches++;
            fill_guards_t<T, G>(h, Eo, k == N ? 2 : 1);
            fill_guards_t<T, G>(h, Bo, k == N ? 2 : 1);
            Ek = Eo;
            Bk = Bo;
        }
        if (sxe) {
            // back to X = L X^ / ell at t^{n+1} (guards included: the scaling is per component)
            scale3_kernel<T><<<sgrid, CELL_THREADS, 0, h->stream>>>((T*)h->E, g.cstride, h->ctx, 1);
            scale3_kernel<T><<<sgrid, CELL_THREADS, 0, h->stream>>>((T*)h->B, g.cstride, h->ctx, 1);
            h->prof.launches += 2;
        }
        return;
    }
    // standard / expanding leapfrog: coefficients of the three curl updates in
    // the context; no shear shift, so each guard fill is one pass
    auto fill = [&](T* F) {
        fill_all_kernel<T, G><<<grid_blocks(fill_all_count<T, G>(g)), NTHR, 0, h->stream>>>(g, F);
        h->prof.launches++;
    };
    curl_t<T, G>(h, true, h->E, h->B, nullptr, 0);
    fill((T*)h->B);
    curl_t<T, G>(h, false, h->B, h->E, h->Jcur, 1);
    fill((T*)h->E);
    curl_t<T, G>(h, true, h->E, h->B, nullptr, 2);
    fill((T*)h->B);
}

template <class T> static PView<T> view_of(void* const a[11]) {
    PView<T> v;
    v.cell = (int*)a[0];
    for (int i = 0; i < 3; ++i) {
        v.o[i] = (T*)a[1 + i];
        v.u[i] = (T*)a[4 + i];
        v.dr[i] = (T*)a[8 + i];
    }
    v.id = (uint32_t*)a[7];
    return v;
}

// ---- the step -----------------------------------------------------------------------------

// The step's parameters for particle buffer b (input) -> 1 - b (output):
// the StepP scalars (the time-dependent ones come from the device context)
// and the per-species buffer views.  Returns the particle count.
template <class T> static long long step_params(pic_handle* h, int b, StepP& P, SpecPack<T>& SP) {
    const Grid& g = h->g;
    const pic_config& cf = h->cfg;
    const int o = 1 - b;
    memset(&P, 0, sizeof(P));
    P.c = cf.c;
    P.step = h->step;
    P.keb_exact = cf.keb_push == PIC_KEB_EXACT;
    P.sO = cf.s_shear * cf.Omega0;
    P.Omega0 = cf.Omega0;
    P.half_nx = 0.5 * g.nx;
    for (int a = 0; a < 3; ++a) {
        P.Lam[a] = (cf.box == PIC_BOX_EXPAND || cf.box == PIC_BOX_SHEAR_EXPAND) ? -0.5 * cf.expand_rate[a] : 0.0;
        P.keb_im[a] = 1.0 / (1.0 - P.Lam[a]);
        P.keb_Lt[a] = (1.0 + P.Lam[a]) / (1.0 - P.Lam[a]);
    }
    P.l_esc = cf.l_esc;
    double pe = cf.p_esc < 0 ? 0 : cf.p_esc;
    P.esc_thresh = pe >= 1.0 ? 0xFFFFFFFFu : (uint32_t)std::floor(pe * 4294967296.0);
    P.seed = cf.seed;
    P.theta_inj = cf.theta_inj;
    P.esc_dims = cf.escape_dims;
    P.inv_c2 = 1.0 / (cf.c * cf.c);
    P.inv_c = 1.0 / cf.c;
    P.f.c = (float)P.c;
    P.f.inv_c = (float)P.inv_c;
    P.f.inv_c2 = (float)P.inv_c2;
    P.f.sO = (float)P.sO;
    P.f.Omega0 = (float)P.Omega0;
    P.f.half_nx = (float)P.half_nx;
    P.f.l_esc = (float)P.l_esc;
    for (int a = 0; a < 3; ++a) {
        P.f.Lam[a] = (float)P.Lam[a];
        P.f.im[a] = (float)P.keb_im[a];
        P.f.Lt[a] = (float)P.keb_Lt[a];
    }
    P.err = h->err;
    P.counters = h->counters;

    memset(&SP, 0, sizeof(SP));
    int nsp = 0;
    long long nparticles = 0;
    for (int s = 0; s < PIC_MAX_SPECIES; ++s) {
        DevSpecies& d = h->sp[s];
        if (!d.loaded) continue;
        SpecStep<T>& S = SP.s[nsp++];
        S.in = view_of<T>(d.arr[b]);
        S.out = view_of<T>(d.arr[o]);
        S.lin = view_of<T>(d.larr[b]);
        S.lout = view_of<T>(d.larr[o]);
        S.stay_in = d.stay[b];
        S.arr_in = d.arrv[b];
        S.stay_out = d.stay[o];
        S.arr_out = d.arrv[o];
        S.lcount_in = d.lcount + b;
        S.lcount_out = d.lcount + o;
        S.tcap = d.tcap;
        S.lcap = d.lcap;
        S.qdt2m = T(d.q / (2.0 * d.m));
        S.qdt2mc = T(d.q / (2.0 * d.m * cf.c));
        S.q = T(d.q);
        nparticles += d.n;
    }
    P.nsp = nsp;
    {
        // FP32 fixed-point current: one int32 unit is worth fx_unit; the range
        // 2^31 fx_unit is 16x the current of the mean total density moving
        // coherently at c, and at least 512 c q_max.  A single contribution is
        // at most c q (|running shape sum| <= |displacement| < c, weights <= 1),
        // so it stays below 2^22 units, as the kernel's conversion requires.  Integer sums are exact mod
        // 2^32, so only a tile's final sum per point must stay inside the
        // range; the flush flags sums above half of it.
        long long ntot = 0;
        double qmax = 0.0;
        for (int s = 0; s < PIC_MAX_SPECIES; ++s)
            if (h->sp[s].loaded) {
                ntot += h->sp[s].n;
                qmax = std::max(qmax, std::fabs(h->sp[s].q));
            }
        if (qmax == 0.0) qmax = 1.0;
        const double rho0 = (double)ntot / ((double)g.nx * g.ny * g.nz);
        const double range = std::max(512.0, 16.0 * rho0) * cf.c * qmax;
        P.fx_scale = (float)(2147483648.0 / range);
        P.fx_unit = 1.0 / (double)P.fx_scale;
    }

    return nparticles;
}

// Start of a step: the device step context, and a zero current.
static pic_status pre_particle(pic_handle* h) {
    const Grid& g = h->g;
    // per-step scalars (step index, shearing shifts, expansion factors, curl
    // coefficients) are computed on the device from its step counter
    ctx_kernel<<<1, 1, 0, h->stream>>>(h->ctx, h->cc);
    h->prof.launches++;
    if (h->fp64) CK(cudaMemsetAsync(h->J, 0, (size_t)3 * g.cstride * h->esz, h->stream));
    else CK(cudaMemsetAsync(h->Jint, 0, (size_t)3 * g.cstride * sizeof(int), h->stream));
    return PIC_OK;
}

// Rest of a step after the tile kernel: loose particles, counter bookkeeping,
// the current's conversion and guard fold, the field update; then the buffers
// flip and the step count advances.
template <class T, int G> static pic_status post_particles_t(pic_handle* h, const StepP& P, const SpecPack<T>& SP) {
    const Grid& g = h->g;
    const int b = h->buf, o = 1 - b;
    if (P.nsp > 0) {
        prof_begin(h);
        void* Jp = h->fp64 ? h->J : (void*)h->Jint;
        const T* Ep = (const T*)h->E;
        const T* Bp = (const T*)h->B;
        StepP Pc = P;
        SpecPack<T> SPc = SP;
        void* largs[] = {(void*)&g, &h->tl, &Pc, &SPc, &Ep, &Bp, &Jp, &h->ctx};
        CK(cudaLaunchKernel(h->ks.loose, dim3(152), dim3(TPB), largs, 0, h->stream));
        h->prof.launches++;
        for (int s = 0; s < PIC_MAX_SPECIES; ++s) {
            DevSpecies& d = h->sp[s];
            if (!d.loaded) continue;
            finalize_kernel<<<grid_blocks(h->tl.ntiles), NTHR, 0, h->stream>>>(
                h->tl.ntiles, d.tcap, d.stay[b], d.arrv[b], d.arrv[o], d.lcount + b, d.lcount + o, d.lcap, h->err,
                h->occ_dev + s, h->occ_dev + PIC_MAX_SPECIES + s);
            h->prof.launches++;
        }
        prof_end(h, 1);
    }
    CK(cudaGetLastError());
    return PIC_OK;
}

// The grid part of the rest of a step: the current's conversion and guard
// fold, the shearing boxes' J' advection, the field update.
template <class T, int G> static pic_status post_fields_t(pic_handle* h, const StepP& P) {
    const Grid& g = h->g;
    const pic_config& cf = h->cfg;
    prof_begin(h);
    if (!h->fp64) {
        fixed_to_float_kernel<<<grid_blocks(3ll * g.cstride), NTHR, 0, h->stream>>>(3ll * g.cstride, h->Jint, (float*)h->J,
                                                                                    P.fx_unit, h->err);
        h->prof.launches++;
    }
    fold_current_t<T, G>(h, (T*)h->J);
    if ((cf.box == PIC_BOX_SHEAR || cf.box == PIC_BOX_SHEAR_EXPAND) && GeomT<G>::AY) {
        // J'(x') -> J'(x): advect along y into the second buffer (h->Jcur)
        ksb_advect_kernel<T><<<cell_grid(g.nx, (g.ny + ADVECT_ROWS - 1) / ADVECT_ROWS, 3ll * g.nz), CELL_THREADS, 0,
                               h->stream>>>(g, (const T*)h->J, (T*)h->Jtmp, cf.s_shear * cf.Omega0, 0.5 * g.nx, h->ctx);
        h->prof.launches++;
    }
    field_step_t<T, G>(h);
    prof_end(h, 2);
    CK(cudaGetLastError());
    return PIC_OK;
}

// The step is done: the particle buffers flip and the step count advances.
static void finish_step(pic_handle* h) {
    h->buf = 1 - h->buf;
    h->step += 1;
}

template <class T, int G> static pic_status post_particle_t(pic_handle* h, const StepP& P, const SpecPack<T>& SP) {
    pic_status st = post_particles_t<T, G>(h, P, SP);
    if (st == PIC_OK) st = post_fields_t<T, G>(h, P);
    if (st != PIC_OK) return st;
    finish_step(h);
    return PIC_OK;
}

// Regroup every species' tiles by cell into the other buffer (see
// regroup_kernel); a species whose slots per tile exceed the sort's shared
// memory is copied in order instead.  Loose lists move along.
template <class T, int G> static pic_status regroup_t(pic_handle* h) {
    const int b = h->buf, o = 1 - b;
    const bool leaky = h->esc == ESC_DISP;
    const int nt = h->tl.ntiles;
    prof_begin(h);
    for (int s = 0; s < PIC_MAX_SPECIES; ++s) {
        DevSpecies& d = h->sp[s];
        if (!d.loaded) continue;
        const PView<T> vin = view_of<T>(d.arr[b]), vout = view_of<T>(d.arr[o]);
        const size_t sm = sizeof(int) * tile_cells<G>() + 4 * (size_t)d.tcap;
        if (d.tcap < 65536 && sm <= MAX_SMEM) {  // the attribute is set by pic_init (regroup_attr_t)
            regroup_kernel<T, G><<<nt, RG_THREADS, sm, h->stream>>>(h->tl, vin, vout, d.stay[b], d.arrv[b], d.stay[o], d.tcap,
                                                                   leaky);
        } else {
            regrow_kernel<T, G><<<nt, NTHR, 0, h->stream>>>(vin, vout, d.stay[b], d.arrv[b], d.tcap, d.tcap, d.stay[o], leaky);
        }
        copy_loose_kernel<T, G><<<64, NTHR, 0, h->stream>>>(view_of<T>(d.larr[b]), view_of<T>(d.larr[o]), d.lcount + b, d.lcap,
                                                            d.lcount + o, leaky);
        CK(cudaGetLastError());
        h->prof.launches += 2;
    }
    // every species is now whole in buffer o (a failed launch above left the
    // state whole in b): switch to it, then restart buffer b's arrival and
    // loose counts for the next step's output.  A reset that fails is
    // reported; the state in o is untouched by it.
    h->buf = o;
    for (int s = 0; s < PIC_MAX_SPECIES; ++s) {
        DevSpecies& d = h->sp[s];
        if (!d.loaded) continue;
        CK(cudaMemsetAsync(d.arrv[b], 0, sizeof(int) * nt, h->stream));
        CK(cudaMemsetAsync(d.lcount + b, 0, sizeof(int), h->stream));
    }
    prof_end(h, 1);
    return PIC_OK;
}

template <class T, int G> static pic_status regroup_attr_t(pic_handle* h) {
    CK(cudaFuncSetAttribute(regroup_kernel<T, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MAX_SMEM));
    return PIC_OK;
}

template <class T, int G> static pic_status step_t(pic_handle* h) {
    if (h->regroup_every > 0 && h->since_regroup >= h->regroup_every) {
        pic_status st = regroup_t<T, G>(h);
        if (st != PIC_OK) return st;
        h->since_regroup = 0;
    }
    h->since_regroup += 1;
    pic_status st = pre_particle(h);
    if (st != PIC_OK) return st;
    StepP P;
    SpecPack<T> SP;
    const long long nparticles = step_params<T>(h, h->buf, P, SP);
    if (P.nsp > 0) {
        prof_begin(h);
        void* Jp = h->fp64 ? h->J : (void*)h->Jint;
        void* args[] = {&h->tmE, &h->tmB, (void*)&h->g, &h->tl, &P, &SP, &Jp, &h->ctx};
        CK(cudaLaunchKernel(h->tile_fn, dim3(h->tl.ntiles), dim3(h->tile_threads), args, h->smem_bytes, h->stream));
        h->prof.launches++;
        h->prof.particle_launches++;
        h->prof.particle_steps += nparticles;
        prof_end(h, 0);
    }
    return post_particle_t<T, G>(h, P, SP);
}

// ---- loading / read-back ------------------------------------------------------------------

// ---- device memory ------------------------------------------------------------------------
// All device memory of a handle comes from one stream-ordered memory pool per
// device, allocated and freed on the handle's stream.  The pool keeps up to
// POOL_KEEP bytes of freed memory for reuse, so the tens of allocations of a
// short run (a served ensemble admits and retires many) cost microseconds
// instead of a cudaMalloc each; large boxes still return their memory.
constexpr uint64_t POOL_KEEP = 8ull << 30;

static cudaMemPool_t lib_pool(int device) {
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    std::lock_guard<std::mutex> lk(mu);
    auto it = pools.find(device);
    if (it != pools.end()) return it->second;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        pool = nullptr;  // fall back to plain allocations
    } else {
        uint64_t keep = POOL_KEEP;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    pools[device] = pool;
    return pool;
}

static cudaError_t dalloc(pic_handle* h, void** p, size_t bytes) {
    cudaMemPool_t pool = lib_pool(h->cfg.device);
    if (!pool) return cudaMalloc(p, bytes);
    return cudaMallocFromPoolAsync(p, bytes, pool, h->stream);
}

static void dfree(pic_handle* h, void* p) {
    if (!p) return;
    if (lib_pool(h->cfg.device)) cudaFreeAsync(p, h->stream);
    else cudaFree(p);
}

// ---- pinned snapshot slots --------------------------------------------------------------------
// A capacity check copies a few counters of a handle to pinned host memory.
// cudaMallocHost and cudaFreeHost per handle would synchronise the device at
// every create and destroy (a served ensemble makes hundreds of handles), so
// the slots come from process-wide slabs that stay allocated until exit.
constexpr int SNAP_INTS = 4 * PIC_MAX_SPECIES;  // two snapshots of (maxima, loose counts)
constexpr int SNAP_PER_SLAB = 1024;

struct SnapSlots {
    std::mutex mu;
    std::vector<int*> free;
};
static SnapSlots& snap_slots() {
    static SnapSlots* s = new SnapSlots();  // never destroyed: handles may outlive static destructors
    return *s;
}

static int* snap_take() {
    SnapSlots& S = snap_slots();
    std::lock_guard<std::mutex> lk(S.mu);
    if (S.free.empty()) {
        int* slab = nullptr;
        if (cudaMallocHost(&slab, sizeof(int) * SNAP_INTS * SNAP_PER_SLAB) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        for (int i = SNAP_PER_SLAB - 1; i >= 0; --i) S.free.push_back(slab + (size_t)i * SNAP_INTS);
    }
    int* p = S.free.back();
    S.free.pop_back();
    return p;
}

static void snap_give(int* p) {
    if (!p) return;
    SnapSlots& S = snap_slots();
    std::lock_guard<std::mutex> lk(S.mu);
    S.free.push_back(p);
}

static void drop_graphs(pic_handle* h) {
    for (int b = 0; b < 2; ++b) {
        if (h->gexec[b]) cudaGraphExecDestroy(h->gexec[b]);
        h->gexec[b] = nullptr;
        h->graph_ok[b] = false;
    }
}

static pic_status alloc_species(pic_handle* h, DevSpecies& d, long long tcap) {
    drop_graphs(h);
    const int nt = h->tl.ntiles;
    const bool leaky = h->esc == ESC_DISP;
    const int nact = h->geom == 0 ? 3 : 2;
    for (int b = 0; b < 2; ++b)
        for (int i = 0; i < 11; ++i) {
            if (d.arr[b][i]) dfree(h, d.arr[b][i]);
            if (d.larr[b][i]) dfree(h, d.larr[b][i]);
            d.arr[b][i] = d.larr[b][i] = nullptr;
        }
    d.tcap = tcap;
    const long long cap = (long long)nt * tcap;
    for (int b = 0; b < 2; ++b) {
        for (int i = 0; i < 11; ++i) {
            bool need = i == 0 || (i >= 1 && i <= nact) || (i >= 4 && i <= 7) || (i >= 8 && leaky);
            if (!need) continue;
            size_t es = (i == 0 || i == 7) ? 4 : h->esz;
            CK(dalloc(h, (void**)&d.arr[b][i], (size_t)cap * es));
            CK(dalloc(h, (void**)&d.larr[b][i], (size_t)d.lcap * es));
        }
        if (!d.stay[b]) CK(dalloc(h, (void**)&d.stay[b], sizeof(int) * nt));
        if (!d.arrv[b]) CK(dalloc(h, (void**)&d.arrv[b], sizeof(int) * nt));
        CK(cudaMemsetAsync(d.stay[b], 0, sizeof(int) * nt, h->stream));
        CK(cudaMemsetAsync(d.arrv[b], 0, sizeof(int) * nt, h->stream));
    }
    // 2D: o[1] of the view is the second active axis; the kernels index o[AY ? 1 : ...]
    if (!d.lcount) CK(dalloc(h, (void**)&d.lcount, sizeof(int) * 2));
    CK(cudaMemsetAsync(d.lcount, 0, sizeof(int) * 2, h->stream));
    return PIC_OK;
}

// Loads and read-backs move particles between the caller's arrays and the
// tiles through device staging buffers of at most this many particles: small
// enough for the memory pool to keep between calls (no new device memory
// after the first), and no transfer needs memory in proportion to the box.
constexpr long long STAGE_PARTICLES = 1ll << 23;

// True when p is (null or) device memory of `device`: a load reads such
// arrays in place.
static bool on_device(const void* p, int device) {
    if (!p) return true;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

// Copy/compute overlap of a chunked transfer: chunk k's copies go on a copy
// stream into staging set k & 1 while the handle's stream runs chunk k - 1's
// kernel; events order each set's copy after the kernel that last read it.
struct LoadPipe {
    cudaStream_t cs = nullptr;
    cudaEvent_t ready[2] = {nullptr, nullptr}, done[2] = {nullptr, nullptr}, start = nullptr;
    bool used[2] = {false, false};
    cudaError_t open(cudaStream_t main) {
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            e = cudaEventCreateWithFlags(&ready[b], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done[b], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&start, cudaEventDisableTiming);
        // the staging memory comes from the pool on the main stream: the copy stream starts after it
        if (e == cudaSuccess) e = cudaEventRecord(start, main);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, start, 0);
        return e;
    }
    // before the copies of set b
    cudaError_t acquire(int b) { return used[b] ? cudaStreamWaitEvent(cs, done[b], 0) : cudaSuccess; }
    // after the copies of set b, before the kernel on `main` that reads them
    cudaError_t hand_over(int b, cudaStream_t main) {
        cudaError_t e = cudaEventRecord(ready[b], cs);
        return e == cudaSuccess ? cudaStreamWaitEvent(main, ready[b], 0) : e;
    }
    // after that kernel
    cudaError_t release(int b, cudaStream_t main) {
        used[b] = true;
        return cudaEventRecord(done[b], main);
    }
    void close() {
        for (int b = 0; b < 2; ++b) {
            if (ready[b]) cudaEventDestroy(ready[b]);
            if (done[b]) cudaEventDestroy(done[b]);
        }
        if (start) cudaEventDestroy(start);
        if (cs) cudaStreamDestroy(cs);  // returns at once; its queued copies still complete
    }
};

// Particles from the caller's arrays (host or device memory) in two passes:
// one counts each tile's particles (positions only), the layout is sized
// from the fullest tile, the second scatters the particles into their tiles.
// Device-resident arrays are read in place.  Host arrays go through device
// staging, a chunk of at most STAGE_PARTICLES particles at a time, with each
// chunk's copy overlapping the previous chunk's kernel (two staging sets and
// a copy stream); the positions copied for the first pass are kept on the
// device for the second when the device has room for them (the input's
// positions and 4 GB more free), else copied again.
template <class T, int G>
static pic_status load_t(pic_handle* h, int species, long long n, const double* x, const double* u, const uint32_t* id,
                         const double* dr) {
    DevSpecies& d = h->sp[species];
    const int nt = h->tl.ntiles;
    const bool leaky = h->esc == ESC_DISP;
    const int dev = h->cfg.device;
    const bool in_place = on_device(x, dev) && on_device(u, dev) && on_device(id, dev) && on_device(dr, dev);
    const long long S = std::max(1ll, std::min(STAGE_PARTICLES, n));
    int* cnt = nullptr;
    double* dx = nullptr;  // the positions, kept on the device between the passes
    double *sx[2] = {nullptr, nullptr}, *su[2] = {nullptr, nullptr}, *sdr[2] = {nullptr, nullptr};
    uint32_t* sid[2] = {nullptr, nullptr};
    LoadPipe pipe;
    auto cleanup = [&]() {
        // copies still queued (a failure midway) finish before their buffers go back to the pool
        if (pipe.cs) cudaStreamSynchronize(pipe.cs);
        cudaStreamSynchronize(h->stream);
        dfree(h, cnt);
        dfree(h, dx);
        for (int b = 0; b < 2; ++b) {
            dfree(h, sx[b]);
            dfree(h, su[b]);
            dfree(h, sid[b]);
            dfree(h, sdr[b]);
        }
        pipe.close();
    };
    cudaError_t e = dalloc(h, (void**)&cnt, sizeof(int) * nt);
    bool keep_x = !in_place && n > S;
    if (const char* v = getenv("PIC_LOAD_RESIDENT_POSITIONS")) keep_x = keep_x && atoi(v) != 0;
    if (e == cudaSuccess && keep_x) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && fr > sizeof(double) * 3 * (size_t)n + (4ull << 30))
            if (dalloc(h, (void**)&dx, sizeof(double) * 3 * (size_t)n) != cudaSuccess) {
                cudaGetLastError();
                dx = nullptr;
            }
    }
    for (int b = 0; b < 2 && e == cudaSuccess && !in_place; ++b) {
        if (!dx) e = dalloc(h, (void**)&sx[b], sizeof(double) * 3 * S);
        if (e == cudaSuccess) e = dalloc(h, (void**)&su[b], sizeof(double) * 3 * S);
        if (e == cudaSuccess && id) e = dalloc(h, (void**)&sid[b], sizeof(uint32_t) * S);
        if (e == cudaSuccess && dr) e = dalloc(h, (void**)&sdr[b], sizeof(double) * 3 * S);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return fail(h, PIC_ERR_OOM, "load staging allocation failed");
    }
    if (!in_place) e = pipe.open(h->stream);
    // pass 1: tile counts
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int) * nt, h->stream);
    if (in_place) {
        if (e == cudaSuccess && n > 0) {
            load_bin_kernel<T, G><<<grid_blocks(n), NTHR, 0, h->stream>>>(n, x, h->tl, h->g, cnt);
            e = cudaGetLastError();
        }
    } else {
        for (long long q0 = 0, k = 0; q0 < n && e == cudaSuccess; q0 += S, ++k) {
            const long long m = std::min(S, n - q0);
            const int b = (int)(k & 1);
            double* px = dx ? dx + 3 * q0 : sx[b];
            e = pipe.acquire(b);
            if (e == cudaSuccess) e = cudaMemcpyAsync(px, x + 3 * q0, sizeof(double) * 3 * m, cudaMemcpyDefault, pipe.cs);
            if (e == cudaSuccess) e = pipe.hand_over(b, h->stream);
            if (e == cudaSuccess) {
                load_bin_kernel<T, G><<<grid_blocks(m), NTHR, 0, h->stream>>>(m, px, h->tl, h->g, cnt);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = pipe.release(b, h->stream);
        }
    }
    std::vector<int> hc(nt);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hc.data(), cnt, sizeof(int) * nt, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        cleanup();
        return fail(h, PIC_ERR_CUDA, "load failed: %s", cudaGetErrorString(e));
    }
    int mx = 0;
    for (int v : hc) mx = std::max(mx, v);
    double slack = h->cfg.capacity_slack > 0 ? h->cfg.capacity_slack : 0.3;
    long long tcap = (long long)std::ceil(mx * (1.0 + slack)) + 32;
    tcap = (tcap + 3) & ~3ll;
    d.lcap = std::max(4096ll, n / 32);
    pic_status st = alloc_species(h, d, tcap);
    if (st != PIC_OK) {
        cleanup();
        return st;
    }
    // pass 2: scatter into the tiles
    const int b0 = h->buf;
    e = cudaMemsetAsync(cnt, 0, sizeof(int) * nt, h->stream);
    if (in_place) {
        if (e == cudaSuccess && n > 0) {
            load_scatter_kernel<T, G><<<grid_blocks(n), NTHR, 0, h->stream>>>(n, 0, x, u, id, dr, h->tl, h->g, cnt, tcap,
                                                                              view_of<T>(d.arr[b0]), leaky);
            e = cudaGetLastError();
        }
    } else {
        for (long long q0 = 0, k = 0; q0 < n && e == cudaSuccess; q0 += S, ++k) {
            const long long m = std::min(S, n - q0);
            const int b = (int)((k + 1) & 1);  // continues the alternation of pass 1's sets
            const double* px = dx ? dx + 3 * q0 : sx[b];
            e = pipe.acquire(b);
            if (e == cudaSuccess && !dx)
                e = cudaMemcpyAsync(sx[b], x + 3 * q0, sizeof(double) * 3 * m, cudaMemcpyDefault, pipe.cs);
            if (e == cudaSuccess) e = cudaMemcpyAsync(su[b], u + 3 * q0, sizeof(double) * 3 * m, cudaMemcpyDefault, pipe.cs);
            if (id && e == cudaSuccess)
                e = cudaMemcpyAsync(sid[b], id + q0, sizeof(uint32_t) * m, cudaMemcpyDefault, pipe.cs);
            if (dr && e == cudaSuccess)
                e = cudaMemcpyAsync(sdr[b], dr + 3 * q0, sizeof(double) * 3 * m, cudaMemcpyDefault, pipe.cs);
            if (e == cudaSuccess) e = pipe.hand_over(b, h->stream);
            if (e == cudaSuccess) {
                load_scatter_kernel<T, G><<<grid_blocks(m), NTHR, 0, h->stream>>>(
                    m, q0, px, su[b], id ? sid[b] : nullptr, dr ? sdr[b] : nullptr, h->tl, h->g, cnt, tcap,
                    view_of<T>(d.arr[b0]), leaky);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = pipe.release(b, h->stream);
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.stay[b0], cnt, sizeof(int) * nt, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cleanup();
    if (e != cudaSuccess) return fail(h, PIC_ERR_CUDA, "load failed: %s", cudaGetErrorString(e));
    d.n = n;
    d.loaded = true;
    h->since_regroup = 0;  // loads leave each tile grouped by cell or freshly ordered
    return PIC_OK;
}

// ---- tile capacity ------------------------------------------------------------------------
// Particles crowding into some tiles fill their slots; arrivals beyond a
// tile's capacity take the loose list, and beyond its capacity are lost
// (PIC_ERR_STATE).  Each step's bookkeeping kernel keeps the fullest tile's
// occupancy on the device; a check copies those maxima and the loose counts
// to the host (one small copy, read one check later), and when a species'
// fullest tile passed 90% of its slots, or its loose list a quarter of its
// room, every species is laid out again into buffer 0 with capacity
// (fullest tile) x max(1 + slack, 1.25) + 32 (never less than before) and a loose list
// at least 4x its current fill.  Re-layout keeps every particle and its order
// within a tile, so the physics does not change.
constexpr double REGROW_HEADROOM = 1.25;  // at least 25% free slots after a re-layout

template <class T, int G> static pic_status regrow_t(pic_handle* h, bool force, bool* grown) {
    *grown = false;
    const int nt = h->tl.ntiles;
    const int b = h->buf;
    const bool leaky = h->esc == ESC_DISP;
    CK(cudaStreamSynchronize(h->stream));
    long long new_tcap[PIC_MAX_SPECIES] = {}, new_lcap[PIC_MAX_SPECIES] = {};
    bool need = force;
    for (int s = 0; s < PIC_MAX_SPECIES; ++s) {
        DevSpecies& d = h->sp[s];
        if (!d.loaded) continue;
        std::vector<int> st(nt), ar(nt);
        int lc = 0;
        CK(cudaMemcpyAsync(st.data(), d.stay[b], sizeof(int) * nt, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(ar.data(), d.arrv[b], sizeof(int) * nt, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(&lc, d.lcount + b, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        long long mx = 0;
        for (int t = 0; t < nt; ++t) mx = std::max(mx, (long long)st[t] + ar[t]);
        const double slack = h->cfg.capacity_slack > 0 ? h->cfg.capacity_slack : 0.3;
        long long tc = (long long)std::ceil(mx * std::max(1.0 + slack, REGROW_HEADROOM)) + 32;
        tc = std::max(d.tcap, (tc + 3) & ~3ll);
        new_tcap[s] = tc;
        new_lcap[s] = std::max(d.lcap, 4ll * lc);
        if (mx > 0.9 * d.tcap || lc > d.lcap / 4) need = true;
    }
    if (!need) return PIC_OK;
    // every new array first: if one does not fit, the current layout stays as it is
    const int nact = h->geom == 0 ? 3 : 2;
    void* na[PIC_MAX_SPECIES][2][11] = {};
    void* nl[PIC_MAX_SPECIES][2][11] = {};
    int* ncnt[PIC_MAX_SPECIES] = {};  // new stay counts [nt], then the new loose count
    bool fits = true;
    for (int s = 0; s < PIC_MAX_SPECIES && fits; ++s) {
        if (!h->sp[s].loaded) continue;
        fits = dalloc(h, (void**)&ncnt[s], sizeof(int) * ((size_t)nt + 1)) == cudaSuccess;
        for (int bb = 0; bb < 2 && fits; ++bb)
            for (int i = 0; i < 11 && fits; ++i) {
                const bool use = i == 0 || (i >= 1 && i <= nact) || (i >= 4 && i <= 7) || (i >= 8 && leaky);
                if (!use) continue;
                const size_t es = (i == 0 || i == 7) ? 4 : h->esz;
                fits = dalloc(h, &na[s][bb][i], (size_t)nt * new_tcap[s] * es) == cudaSuccess &&
                       dalloc(h, &nl[s][bb][i], (size_t)new_lcap[s] * es) == cudaSuccess;
            }
    }
    auto free_new = [&]() {
        for (int s = 0; s < PIC_MAX_SPECIES; ++s) {
            dfree(h, ncnt[s]);
            for (int bb = 0; bb < 2; ++bb)
                for (int i = 0; i < 11; ++i) {
                    dfree(h, na[s][bb][i]);
                    dfree(h, nl[s][bb][i]);
                }
        }
    };
    if (!fits) {
        cudaGetLastError();
        free_new();
        return fail(h, PIC_ERR_OOM, "a larger tile layout does not fit in device memory; the current one is kept");
    }
    // copies into the new arrays only (the new counts go to ncnt): a launch
    // that fails here leaves every species' current layout untouched
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < PIC_MAX_SPECIES && e == cudaSuccess; ++s) {
        DevSpecies& d = h->sp[s];
        if (!d.loaded) continue;
        PView<T> vin = view_of<T>(d.arr[b]), vout = view_of<T>(na[s][0]);
        regrow_kernel<T, G><<<nt, NTHR, 0, h->stream>>>(vin, vout, d.stay[b], d.arrv[b], d.tcap, new_tcap[s], ncnt[s], leaky);
        copy_loose_kernel<T, G><<<64, NTHR, 0, h->stream>>>(view_of<T>(d.larr[b]), view_of<T>(nl[s][0]), d.lcount + b, d.lcap,
                                                            ncnt[s] + nt, leaky);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        free_new();
        return fail(h, PIC_ERR_CUDA, "re-layout copy failed (the current layout is kept): %s", cudaGetErrorString(e));
    }
    // commit: buffer 0 takes the new counts, every species switches to the new arrays
    drop_graphs(h);
    for (int s = 0; s < PIC_MAX_SPECIES; ++s) {
        DevSpecies& d = h->sp[s];
        if (!d.loaded) continue;
        if (e == cudaSuccess) e = cudaMemcpyAsync(d.stay[0], ncnt[s], sizeof(int) * nt, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d.lcount, ncnt[s] + nt, sizeof(int), cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(d.lcount + 1, 0, sizeof(int), h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(d.arrv[0], 0, sizeof(int) * nt, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(d.arrv[1], 0, sizeof(int) * nt, h->stream);
        dfree(h, ncnt[s]);
        ncnt[s] = nullptr;
        for (int bb = 0; bb < 2; ++bb)
            for (int i = 0; i < 11; ++i) {
                dfree(h, d.arr[bb][i]);
                dfree(h, d.larr[bb][i]);
                d.arr[bb][i] = na[s][bb][i];
                d.larr[bb][i] = nl[s][bb][i];
                na[s][bb][i] = nl[s][bb][i] = nullptr;
            }
        d.tcap = new_tcap[s];
        d.lcap = new_lcap[s];
    }
    // a failed count copy after the switch leaves the counts unknown: the
    // handle reports the error and its particle state must be reloaded
    if (e != cudaSuccess) return fail(h, PIC_ERR_CUDA, "re-layout count update failed: %s", cudaGetErrorString(e));
    h->buf = 0;
    h->regrows += 1;
    *grown = true;
    CK(cudaStreamSynchronize(h->stream));
    return PIC_OK;
}

// Particles of a species read back in tile order, then the loose list, into
// the caller's buffers (host or device memory, any kind): tiles are compacted
// a chunk at a time into device staging buffers of at most STAGE_PARTICLES
// particles, each chunk copied out before the next is written.

template <class T, int G>
static pic_status compact_t(pic_handle* h, int species, double* x, double* u, uint32_t* id, double* dr) {
    DevSpecies& d = h->sp[species];
    const int nt = h->tl.ntiles;
    const int b = h->buf;
    std::vector<int> st(nt), ar(nt);
    int lc = 0;
    CK(cudaMemcpyAsync(st.data(), d.stay[b], sizeof(int) * nt, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(ar.data(), d.arrv[b], sizeof(int) * nt, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&lc, d.lcount + b, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    lc = (int)std::min<long long>(lc, d.lcap);
    std::vector<long long> off(nt + 1);
    long long acc = 0, big = lc;
    for (int t = 0; t < nt; ++t) {
        off[t] = acc;
        acc += st[t] + ar[t];
        big = std::max<long long>(big, st[t] + ar[t]);
    }
    off[nt] = acc;
    if (acc + lc != d.n)
        return fail(h, PIC_ERR_STATE, "species %d holds %lld particles, expected %lld", species, acc + lc, d.n);
    if (acc + lc == 0) return PIC_OK;
    const long long S = std::min(std::max(STAGE_PARTICLES, big), acc + lc);
    long long* doff = nullptr;
    double *sx = nullptr, *su = nullptr, *sdr = nullptr;
    uint32_t* sid = nullptr;
    pic_status ret = PIC_OK;
    auto cleanup = [&]() {
        dfree(h, doff);
        dfree(h, sx);
        dfree(h, su);
        dfree(h, sid);
        dfree(h, sdr);
    };
    if (dalloc(h, (void**)&doff, sizeof(long long) * (nt + 1)) != cudaSuccess ||
        (x && dalloc(h, (void**)&sx, sizeof(double) * 3 * S) != cudaSuccess) ||
        (u && dalloc(h, (void**)&su, sizeof(double) * 3 * S) != cudaSuccess) ||
        (id && dalloc(h, (void**)&sid, sizeof(uint32_t) * S) != cudaSuccess) ||
        (dr && dalloc(h, (void**)&sdr, sizeof(double) * 3 * S) != cudaSuccess)) {
        cudaGetLastError();
        cleanup();
        return fail(h, PIC_ERR_OOM, "read-back staging allocation failed");
    }
    const bool hd = h->esc == ESC_DISP;
    auto copy_out = [&](long long o0, long long cnt) -> cudaError_t {
        cudaError_t e = cudaSuccess;
        if (x && e == cudaSuccess) e = cudaMemcpyAsync(x + 3 * o0, sx, sizeof(double) * 3 * cnt, cudaMemcpyDefault, h->stream);
        if (u && e == cudaSuccess) e = cudaMemcpyAsync(u + 3 * o0, su, sizeof(double) * 3 * cnt, cudaMemcpyDefault, h->stream);
        if (id && e == cudaSuccess) e = cudaMemcpyAsync(id + o0, sid, sizeof(uint32_t) * cnt, cudaMemcpyDefault, h->stream);
        if (dr && e == cudaSuccess) e = cudaMemcpyAsync(dr + 3 * o0, sdr, sizeof(double) * 3 * cnt, cudaMemcpyDefault, h->stream);
        return e;
    };
    cudaError_t e = cudaMemcpyAsync(doff, off.data(), sizeof(long long) * (nt + 1), cudaMemcpyHostToDevice, h->stream);
    // stream order: each chunk's copies finish before the next chunk's
    // compaction overwrites the staging buffers
    for (int t0 = 0; t0 < nt && e == cudaSuccess;) {
        int t1 = t0 + 1;
        while (t1 < nt && off[t1 + 1] - off[t0] <= S) ++t1;
        const long long cnt = off[t1] - off[t0];
        if (cnt > 0) {
            compact_kernel<T, G><<<t1 - t0, NTHR, 0, h->stream>>>(h->tl, h->g, view_of<T>(d.arr[b]), d.stay[b], d.arrv[b],
                                                                d.tcap, doff, t0, off[t0], hd, sx, su, sid, sdr);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = copy_out(off[t0], cnt);
        }
        t0 = t1;
    }
    if (lc > 0 && e == cudaSuccess) {
        compact_loose_kernel<T, G><<<64, NTHR, 0, h->stream>>>(view_of<T>(d.larr[b]), d.lcount + b, d.lcap, 0, hd, sx, su, sid,
                                                               sdr);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = copy_out(acc, lc);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) ret = fail(h, PIC_ERR_CUDA, "read-back failed: %s", cudaGetErrorString(e));
    cleanup();
    return ret;
}

template <class T, int G>
static pic_status sample_t(pic_handle* h, int species, uint32_t modulus, uint32_t remainder, long long max_out, double* x,
                           double* u, uint32_t* id, double* dr, long long* n_out) {
    DevSpecies& d = h->sp[species];
    const int b = h->buf;
    double *dx = nullptr, *du = nullptr, *ddr = nullptr;
    uint32_t* did = nullptr;
    unsigned long long* dcount = nullptr;
    const size_t m = (size_t)std::max(max_out, 1ll);
    CK(dalloc(h, (void**)&dx, sizeof(double) * 3 * m));
    CK(dalloc(h, (void**)&du, sizeof(double) * 3 * m));
    CK(dalloc(h, (void**)&ddr, sizeof(double) * 3 * m));
    CK(dalloc(h, (void**)&did, sizeof(uint32_t) * m));
    CK(dalloc(h, (void**)&dcount, sizeof(unsigned long long)));
    CK(cudaMemsetAsync(dcount, 0, sizeof(unsigned long long), h->stream));
    sample_kernel<T, G><<<std::min(h->tl.ntiles + 1, 152 * 8), NTHR, 0, h->stream>>>(
        h->tl, view_of<T>(d.arr[b]), d.stay[b], d.arrv[b], d.tcap, view_of<T>(d.larr[b]), d.lcount + b, d.lcap, modulus,
        remainder, h->esc == ESC_DISP, max_out, dcount, dx, du, did, ddr);
    unsigned long long cnt = 0;
    CK(cudaMemcpyAsync(&cnt, dcount, sizeof(cnt), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaGetLastError());
    const long long k = std::min((long long)cnt, max_out);
    if (k > 0) {
        if (x) CK(cudaMemcpyAsync(x, dx, sizeof(double) * 3 * k, cudaMemcpyDeviceToHost, h->stream));
        if (u) CK(cudaMemcpyAsync(u, du, sizeof(double) * 3 * k, cudaMemcpyDeviceToHost, h->stream));
        if (id) CK(cudaMemcpyAsync(id, did, sizeof(uint32_t) * k, cudaMemcpyDeviceToHost, h->stream));
        if (dr) CK(cudaMemcpyAsync(dr, ddr, sizeof(double) * 3 * k, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        if (x && h->geom != 0) {
            const int ig = h->geom == 1 ? 2 : 1;
            for (long long i = 0; i < k; ++i) x[3 * i + ig] = 0.5;
        }
    }
    *n_out = (long long)cnt;
    dfree(h, dx);
    dfree(h, du);
    dfree(h, ddr);
    dfree(h, did);
    dfree(h, dcount);
    return PIC_OK;
}

template <class T, int G> static pic_status maxwellian_t(pic_handle* h, int species, int ppc, double theta, const double drift[3],
                                                         double noise, uint32_t seed, uint32_t id_base) {
    DevSpecies& d = h->sp[species];
    const int cells_per_tile = h->tl.tx * h->tl.ty * h->tl.tz;
    double slack = h->cfg.capacity_slack > 0 ? h->cfg.capacity_slack : 0.3;
    long long tcap = (long long)std::ceil((double)ppc * cells_per_tile * (1.0 + slack)) + 32;
    tcap = (tcap + 3) & ~3ll;
    long long n = (long long)ppc * h->g.nx * h->g.ny * h->g.nz;
    d.lcap = std::max(4096ll, n / 32);
    pic_status st = alloc_species(h, d, tcap);
    if (st != PIC_OK) return st;
    const int b = h->buf;
    // about four CTAs per SM in all, at most one per 256 particles of a tile
    const int per_tile = ppc * cells_per_tile;
    const int ny = std::max(1, std::min((per_tile + NTHR - 1) / NTHR, (4 * 152 + h->tl.ntiles - 1) / h->tl.ntiles));
    maxwellian_kernel<T, G><<<dim3(h->tl.ntiles, ny), NTHR, 0, h->stream>>>(h->tl, h->g, ppc, theta, h->cfg.c, drift ? drift[0] : 0.0,
                                                                 drift ? drift[1] : 0.0, drift ? drift[2] : 0.0, noise, seed,
                                                                 id_base, tcap, view_of<T>(d.arr[b]), h->esc == ESC_DISP,
                                                                 d.stay[b]);
    CK(cudaGetLastError());
    d.n = n;
    d.loaded = true;
    h->since_regroup = 0;  // loads leave each tile grouped by cell or freshly ordered
    return PIC_OK;
}

// ---- dispatch by precision / geometry --------------------------------------------------------

#define DISPATCH(h, FN, ...) TG_DISPATCH((h)->fp64, (h)->tg, FN, __VA_ARGS__)
// by precision and template geometry (no FP64 kernels for 32 x 32 tiles)
#define TG_DISPATCH(fp64, tg, FN, ...)                                              \
    ((fp64) ? ((tg) == 0   ? FN<double, 0>(__VA_ARGS__)                             \
               : (tg) == 1 ? FN<double, 1>(__VA_ARGS__)                             \
               : (tg) == 5 ? FN<double, 5>(__VA_ARGS__)                             \
               : (tg) == 6 ? FN<double, 6>(__VA_ARGS__)                             \
               : (tg) == 7 ? FN<double, 7>(__VA_ARGS__)                             \
                           : FN<double, 2>(__VA_ARGS__))                            \
            : ((tg) == 0   ? FN<float, 0>(__VA_ARGS__)                              \
               : (tg) == 1 ? FN<float, 1>(__VA_ARGS__)                              \
               : (tg) == 2 ? FN<float, 2>(__VA_ARGS__)                              \
               : (tg) == 3 ? FN<float, 3>(__VA_ARGS__)                              \
               : (tg) == 4 ? FN<float, 4>(__VA_ARGS__)                              \
               : (tg) == 5 ? FN<float, 5>(__VA_ARGS__)                              \
               : (tg) == 6 ? FN<float, 6>(__VA_ARGS__)                              \
                           : FN<float, 7>(__VA_ARGS__)))

template <class T, int G> static pic_status set_fields_t(pic_handle* h, const double* E, const double* B) {
    const Grid& g = h->g;
    long long n = 3ll * g.nx * g.ny * g.nz;
    CK(cudaMemcpyAsync(h->stage, E, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    scatter_field_kernel<T><<<grid_blocks(n), NTHR, 0, h->stream>>>(g, h->stage, (T*)h->E);
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaMemcpyAsync(h->stage, B, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    scatter_field_kernel<T><<<grid_blocks(n), NTHR, 0, h->stream>>>(g, h->stage, (T*)h->B);
    fill_all_t<T, G>(h, (double)h->step);
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaGetLastError());
    return PIC_OK;
}

template <class T, int G> static pic_status uniform_fields_t(pic_handle* h, const double* E, const double* B) {
    const Grid& g = h->g;
    uniform_field_kernel<T><<<grid_blocks(3ll * g.cstride), NTHR, 0, h->stream>>>(g, (T*)h->E, E[0], E[1], E[2]);
    uniform_field_kernel<T><<<grid_blocks(3ll * g.cstride), NTHR, 0, h->stream>>>(g, (T*)h->B, B[0], B[1], B[2]);
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaGetLastError());
    return PIC_OK;
}

template <class T, int G> static pic_status get_fields_t(pic_handle* h, double* E, double* B, double* J) {
    const Grid& g = h->g;
    long long n = 3ll * g.nx * g.ny * g.nz;
    void* src[3] = {h->E, h->B, h->Jcur};
    double* dst[3] = {E, B, J};
    for (int f = 0; f < 3; ++f) {
        if (!dst[f]) continue;
        gather_field_kernel<T><<<grid_blocks(n), NTHR, 0, h->stream>>>(g, (const T*)src[f], h->stage);
        CK(cudaMemcpyAsync(dst[f], h->stage, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    CK(cudaGetLastError());
    return PIC_OK;
}

template <class T, int G> static pic_status diag_t(pic_handle* h, pic_diag* out) {
    const Grid& g = h->g;
    double* dsum = h->partial + (size_t)h->partial_blocks * 3;
    double hs[3];
    void* f[2] = {h->E, h->B};
    for (int k = 0; k < 2; ++k) {
        sumsq_partial_kernel<T><<<h->partial_blocks, NTHR, 0, h->stream>>>(g, (const T*)f[k], h->partial);
        sum_partials_kernel<<<1, 32, 0, h->stream>>>(h->partial, h->partial_blocks, 3, dsum);
        CK(cudaMemcpyAsync(hs, dsum, sizeof(hs), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        for (int c = 0; c < 3; ++c) (k == 0 ? out->field_energy_E : out->field_energy_B)[c] = hs[c] / 25.132741228718345;
    }
    const int b = h->buf;
    for (int s = 0; s < PIC_MAX_SPECIES; ++s) {
        DevSpecies& d = h->sp[s];
        out->kinetic_energy[s] = 0.0;
        out->count[s] = 0;
        if (!d.loaded) continue;
        kinetic_kernel<T, G><<<h->partial_blocks, NTHR, 0, h->stream>>>(h->tl, view_of<T>(d.arr[b]), d.stay[b], d.arrv[b], d.tcap,
                                                                       view_of<T>(d.larr[b]), d.lcount + b, d.lcap, h->cfg.c,
                                                                       d.m, h->partial);
        sum_partials_kernel<<<1, 32, 0, h->stream>>>(h->partial, h->partial_blocks, 1, dsum);
        CK(cudaMemcpyAsync(hs, dsum, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        int lc = 0;
        CK(cudaMemcpyAsync(&lc, d.lcount + b, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        out->kinetic_energy[s] = hs[0];
        out->count[s] = d.n;
        out->loose += lc;
    }
    CK(cudaGetLastError());
    return PIC_OK;
}

// ---- configuration ----------------------------------------------------------------------------

static pic_status validate(const pic_config* c) {
    pic_handle* h = nullptr;
    if (!c) return fail(h, PIC_ERR_ARG, "config is NULL");
    if (c->box < 0 || c->box > 4) return fail(h, PIC_ERR_ARG, "box must be 0..4");
    if (c->ndim != 2 && c->ndim != 3) return fail(h, PIC_ERR_ARG, "ndim must be 2 or 3");
    if (c->ndim == 2 && c->plane != PIC_PLANE_XY && c->plane != PIC_PLANE_XZ)
        return fail(h, PIC_ERR_ARG, "2D plane must be PIC_PLANE_XY or PIC_PLANE_XZ");
    if (c->ndim == 2 && c->plane == PIC_PLANE_XY && c->nz != 1) return fail(h, PIC_ERR_ARG, "2D x-y plane needs nz = 1");
    if (c->ndim == 2 && c->plane == PIC_PLANE_XZ && c->ny != 1) return fail(h, PIC_ERR_ARG, "2D x-z plane needs ny = 1");
    int act[3] = {c->nx, c->ny, c->nz};
    bool active[3] = {true, !(c->ndim == 2 && c->plane == PIC_PLANE_XZ), !(c->ndim == 2 && c->plane == PIC_PLANE_XY)};
    for (int a = 0; a < 3; ++a)
        if (active[a] && act[a] < 8) return fail(h, PIC_ERR_ARG, "active axes need at least 8 cells (axis %d has %d)", a, act[a]);
    if (c->nx > (c->ndim == 3 ? 2048 : 65536) || c->ny > (c->ndim == 3 ? 2048 : 65536) || c->nz > (c->ndim == 3 ? 1024 : 65536))
        return fail(h, PIC_ERR_ARG, "grid too large for the packed cell index (3D: 2048 x 2048 x 1024)");
    if (c->shape_order != 1 && c->shape_order != 2) return fail(h, PIC_ERR_ARG, "shape_order must be 1 or 2");
    if (c->precision != PIC_FP32 && c->precision != PIC_FP64) return fail(h, PIC_ERR_ARG, "precision must be FP32 or FP64");
    if (!(c->c > 0) || !(c->c * std::sqrt((double)c->ndim) < 1.0))
        return fail(h, PIC_ERR_ARG, "Courant number c must satisfy 0 < c sqrt(ndim) < 1");
    if (c->box == PIC_BOX_SHEAR || c->box == PIC_BOX_SHEAR_EXPAND) {
        if (c->fp_iters < 1 || c->fp_iters > 64) return fail(h, PIC_ERR_ARG, "fp_iters must be in 1..64");
        double vmax = std::fabs(c->s_shear * c->Omega0) * 0.5 * c->nx;
        if (c->c + vmax >= 1.0) return fail(h, PIC_ERR_ARG, "c + max shear speed must stay below one cell per step");
    }
    if (c->escape_mode < 0 || c->escape_mode > 2) return fail(h, PIC_ERR_ARG, "escape_mode must be 0..2");
    if (c->escape_mode == PIC_ESC_DISPLACEMENT && c->box != PIC_BOX_LEAKY)
        return fail(h, PIC_ERR_ARG, "the displacement escape rule is the leaky box's; other boxes take the probabilistic one");
    if (c->box == PIC_BOX_LEAKY) {
        if (c->escape_mode == PIC_ESC_DISPLACEMENT && !(c->l_esc > 0)) return fail(h, PIC_ERR_ARG, "l_esc must be > 0");
        if (c->escape_dims != 2 && c->escape_dims != 3) return fail(h, PIC_ERR_ARG, "escape_dims must be 2 or 3");
    }
    if (c->escape_mode != PIC_ESC_NONE && !(c->theta_inj > 0)) return fail(h, PIC_ERR_ARG, "theta_inj must be > 0");
    for (int a = 0; a < 3; ++a)
        if (c->tile[a] < 0) return fail(h, PIC_ERR_ARG, "tile sizes must be >= 0");
    return PIC_OK;
}

template <class T, int G> static pic_status refill_t(pic_handle* h) {
    fill_all_t<T, G>(h, (double)h->step);
    CK(cudaGetLastError());
    return PIC_OK;
}

extern "C" {

// used by entry points without a handle (noalloc.cu)
void pic_internal_set_global_error(const char* msg) { g_init_error = msg ? msg : ""; }

const char* pic_version(void) { return "libpic 0.1 (sm_103a)"; }
int pic_abi_version(void) { return PIC_ABI_VERSION; }

const char* pic_last_error(pic_handle* h) { return h ? h->last_error.c_str() : g_init_error.c_str(); }

// The 2D tile side pic_init picks when the configuration leaves it open: 8
// when 16 x 16 tiles would give fewer than two per SM (a small box's
// particle kernel then runs on a few SMs), 32 (FP32) when 32 x 32 tiles still
// give eight per SM (the larger tiles amortise staging and barriers), else
// 16.  pic_autotune_tile measures instead.
static int auto_tile_side(const pic_config& c, bool fp64) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        sms = 152;
    }
    if (c.ndim == 3) {
        // 4 x 4 x 4 tiles when 8 x 8 x 8 ones would be fewer than two per SM
        const long long t8 = ((c.nx + 7ll) / 8) * ((c.ny + 7ll) / 8) * ((c.nz + 7ll) / 8);
        return t8 < 2ll * sms ? 4 : 8;
    }
    const long long a = c.nx, b = c.plane == PIC_PLANE_XY ? c.ny : c.nz;
    auto tiles = [&](long long s) { return ((a + s - 1) / s) * ((b + s - 1) / s); };
    if (tiles(16) < 2ll * sms) return 8;
    if (!fp64 && tiles(32) >= 8ll * sms) return 32;
    return 16;
}

// Tiling of a handle from its template geometry (h->tg) and grid: the tile
// extents are those the particle kernels of h->tg are compiled for.
static void set_tiling(pic_handle* h) {
    const pic_config& c = h->cfg;
    const bool AY = h->geom != 2, AZ = h->geom != 1;
    const int side = tile_side(h->tg);
    Tiling& tl = h->tl;
    tl.tx = side;
    tl.ty = AY ? side : 1;
    tl.tz = AZ ? side : 1;
    tl.ntx = (c.nx + tl.tx - 1) / tl.tx;
    tl.nty = (c.ny + tl.ty - 1) / tl.ty;
    tl.ntz = (c.nz + tl.tz - 1) / tl.tz;
    tl.ntiles = tl.ntx * tl.nty * tl.ntz;
    tl.xalign = (int)(16 / h->esz);
    tl.bx = tl.tx + 4;
    tl.by = AY ? tl.ty + 4 : 1;
    tl.bz = AZ ? tl.tz + 4 : 1;
    tl.jx = tl.tx + 5;
    tl.jy = AY ? tl.ty + 5 : 1;
    tl.jz = AZ ? tl.tz + 5 : 1;
}

pic_status pic_init(const pic_config* cfg, pic_handle** out) {
    if (!out) return fail(nullptr, PIC_ERR_ARG, "out is NULL");
    *out = nullptr;
    pic_status st = validate(cfg);
    if (st != PIC_OK) return st;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return fail(nullptr, PIC_ERR_CUDA, "no CUDA device available");
    if (cfg->device < 0 || cfg->device >= ndev)
        return fail(nullptr, PIC_ERR_ARG, "device %d out of range (%d devices)", cfg->device, ndev);
    if (cudaSetDevice(cfg->device) != cudaSuccess) return fail(nullptr, PIC_ERR_CUDA, "cudaSetDevice(%d) failed", cfg->device);
    pic_handle* h = new pic_handle();
    h->cfg = *cfg;
    pic_config& c = h->cfg;
    if (c.escape_dims == 0) c.escape_dims = 2;
    h->geom = c.ndim == 3 ? 0 : (c.plane == PIC_PLANE_XY ? 1 : 2);
    h->fp64 = c.precision == PIC_FP64;
    h->esz = h->fp64 ? 8 : 4;
    h->push = c.box == PIC_BOX_SHEAR           ? PUSH_KSB
              : c.box == PIC_BOX_EXPAND        ? PUSH_KEB
              : c.box == PIC_BOX_SHEAR_EXPAND ? PUSH_SXE
                                               : PUSH_BORIS;
    // escape: the displacement rule in the leaky box, the probabilistic rule in any box
    h->esc = c.escape_mode == PIC_ESC_PROBABILISTIC                              ? ESC_PROB
             : (c.box == PIC_BOX_LEAKY && c.escape_mode == PIC_ESC_DISPLACEMENT) ? ESC_DISP
                                                                                 : ESC_NONE;
    const bool AY = h->geom != 2, AZ = h->geom != 1;
    const int A = (int)(16 / h->esz);  // TMA x quantum
    Grid& g = h->g;
    g.nx = c.nx; g.ny = c.ny; g.nz = c.nz;
    g.gx = GL; g.gy = AY ? GL : 0; g.gz = AZ ? GL : 0;
    g.px = ((c.nx + GL + GR) + A - 1) / A * A;
    g.py = AY ? c.ny + GL + GR : 1;
    g.pz = AZ ? c.nz + GL + GR : 1;
    g.cstride = (long long)g.px * g.py * g.pz;
    // particle tiles: 8^3 cells in 3D; 16^2 cells in 2D, or 8^2 or 32^2 (FP32) on request
    {
        const int t0 = c.tile[0], t1 = AY ? c.tile[1] : c.tile[2];
        const int want = t0 ? t0 : t1;
        const int w3 = c.tile[0] ? c.tile[0] : (c.tile[1] ? c.tile[1] : c.tile[2]);
        const bool ok3 = h->geom == 0 && (w3 == 0 || w3 == 4 || w3 == 8) && (c.tile[0] == 0 || c.tile[0] == w3) &&
                         (c.tile[1] == 0 || c.tile[1] == w3) && (c.tile[2] == 0 || c.tile[2] == w3);
        const bool ok2 = h->geom != 0 && (want == 0 || want == 8 || want == 16 || (want == 32 && !h->fp64)) &&
                         (t1 == 0 || t1 == want);
        if (!(h->geom == 0 ? ok3 : ok2)) {
            delete h;
            return fail(nullptr, PIC_ERR_ARG, "tile must be 0 (automatic) or %s", h->geom == 0 ? "4x4x4 or 8x8x8 in 3D"
                        : "8x8, 16x16, or 32x32 (FP32), on the active plane in 2D");
        }
        const int side = h->geom == 0 ? w3 : want;
        h->tg = tgeom_of(h->geom, side ? side : auto_tile_side(c, h->fp64));
    }
    set_tiling(h);
    {
        int v = c.kernel_variant > 0 ? (int)c.kernel_variant - 1 : default_variant(h->fp64, h->tg);
        if (c.kernel_variant == 0)
            if (const char* e = getenv("PIC_KERNEL_VARIANT")) v = atoi(e) - 1;
        if (v < 0 || v >= N_TILE_VARIANTS || tile_smem_bytes(h->fp64, h->tg, v) > MAX_SMEM) {
            delete h;
            return fail(nullptr, PIC_ERR_ARG, "particle-kernel variant %d does not fit this configuration", v + 1);
        }
        h->tile_variant = v;
        h->tile_threads = TILE_VARIANTS[v].nt;
        h->smem_bytes = tile_smem_bytes(h->fp64, h->tg, v);
    }
    h->ks = lookup_kernels(h->fp64, h->tg, c.shape_order, h->push, h->esc);
    h->tile_fn = h->ks.tile[h->tile_variant];

    auto bail = [&](pic_status s) {
        g_init_error = h->last_error;
        pic_destroy(h);
        return s;
    };
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete h;
        return fail(nullptr, PIC_ERR_CUDA, "cudaStreamCreate failed");
    }
    h->own_stream = true;
    if (cudaFuncSetAttribute(h->tile_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->smem_bytes) != cudaSuccess)
        return bail(fail(h, PIC_ERR_CUDA, "cannot set %zu bytes of dynamic shared memory", h->smem_bytes));
    if (DISPATCH(h, regroup_attr_t, h) != PIC_OK) return bail(PIC_ERR_CUDA);
    h->regroup_every = default_regroup_interval(h->fp64, h->tg);
    const size_t fb = (size_t)3 * g.cstride * h->esz;
    void** bufs[] = {&h->E, &h->B, &h->J, &h->Jtmp};
    for (void** p : bufs) {
        if (dalloc(h, p, fb) != cudaSuccess) return bail(fail(h, PIC_ERR_OOM, "field allocation failed"));
        cudaMemsetAsync(*p, 0, fb, h->stream);
    }
    h->Jcur = ((c.box == PIC_BOX_SHEAR || c.box == PIC_BOX_SHEAR_EXPAND) && AY) ? h->Jtmp : h->J;
    if (dalloc(h, (void**)&h->ctx, sizeof(StepCtx)) != cudaSuccess) return bail(fail(h, PIC_ERR_OOM, "allocation failed"));
    cudaMemsetAsync(h->ctx, 0, sizeof(StepCtx), h->stream);
    h->cc.box = c.box == PIC_BOX_SHEAR ? 1 : (c.box == PIC_BOX_EXPAND ? 2 : (c.box == PIC_BOX_SHEAR_EXPAND ? 4 : 0));
    h->cc.ny = c.ny;
    h->cc.sO_Lx = c.s_shear * c.Omega0 * (double)c.nx;
    for (int a = 0; a < 3; ++a) h->cc.rate[a] = c.expand_rate[a];
    h->cc.c = c.c;
    if (const char* e = getenv("PIC_NO_GRAPHS")) h->graphs_on = atoi(e) == 0;
    if (!h->fp64) {
        if (dalloc(h, (void**)&h->Jint, (size_t)3 * g.cstride * sizeof(int)) != cudaSuccess)
            return bail(fail(h, PIC_ERR_OOM, "field allocation failed"));
        cudaMemsetAsync(h->Jint, 0, (size_t)3 * g.cstride * sizeof(int), h->stream);
    }
    if (c.box == PIC_BOX_SHEAR || c.box == PIC_BOX_SHEAR_EXPAND) {
        void** kb[] = {&h->Es, &h->Bs, &h->Ec, &h->Bc};
        for (void** p : kb) {
            if (dalloc(h, p, fb) != cudaSuccess) return bail(fail(h, PIC_ERR_OOM, "field allocation failed"));
            cudaMemsetAsync(*p, 0, fb, h->stream);
        }
    }
    h->stage_elems = (size_t)3 * c.nx * c.ny * c.nz;
    if (dalloc(h, (void**)&h->stage, sizeof(double) * h->stage_elems) != cudaSuccess)
        return bail(fail(h, PIC_ERR_OOM, "staging allocation failed"));
    h->partial_blocks = 152 * 8;
    if (dalloc(h, (void**)&h->partial, sizeof(double) * (h->partial_blocks * 3 + 8)) != cudaSuccess)
        return bail(fail(h, PIC_ERR_OOM, "allocation failed"));
    if (dalloc(h, (void**)&h->err, sizeof(int)) != cudaSuccess || dalloc(h, (void**)&h->counters, 2 * sizeof(unsigned long long)) != cudaSuccess)
        return bail(fail(h, PIC_ERR_OOM, "allocation failed"));
    if (dalloc(h, (void**)&h->occ_dev, sizeof(int) * 2 * PIC_MAX_SPECIES) != cudaSuccess)
        return bail(fail(h, PIC_ERR_OOM, "allocation failed"));
    cudaMemsetAsync(h->occ_dev, 0, sizeof(int) * 2 * PIC_MAX_SPECIES, h->stream);
    cudaMemsetAsync(h->err, 0, sizeof(int), h->stream);
    cudaMemsetAsync(h->counters, 0, 2 * sizeof(unsigned long long), h->stream);
    if (encode_field_map(h, &h->tmE, h->E) != PIC_OK || encode_field_map(h, &h->tmB, h->B) != PIC_OK)
        return bail(PIC_ERR_CUDA);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return bail(fail(h, PIC_ERR_CUDA, "initialisation failed"));
    *out = h;
    return PIC_OK;
}

pic_status pic_destroy(pic_handle* h) {
    if (!h) return PIC_OK;
    cudaSetDevice(h->cfg.device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (auto& d : h->sp) {
        for (int b = 0; b < 2; ++b) {
            for (int i = 0; i < 11; ++i) {
                if (d.arr[b][i]) dfree(h, d.arr[b][i]);
                if (d.larr[b][i]) dfree(h, d.larr[b][i]);
            }
            if (d.stay[b]) dfree(h, d.stay[b]);
            if (d.arrv[b]) dfree(h, d.arrv[b]);
        }
        if (d.lcount) dfree(h, d.lcount);
    }
    void* ptrs[] = {h->E,     h->B,     h->J,       h->Jtmp,    h->Es,       h->Bs,       h->Ec,
                    h->Bc,    h->stage, h->partial, h->err,     h->counters, (void*)h->Jint, (void*)h->occ_dev};
    for (void* p : ptrs)
        if (p) dfree(h, p);
    prof_resolve(h);
    for (cudaEvent_t e : h->prof.pool) cudaEventDestroy(e);
    drop_graphs(h);
    for (cudaEvent_t e : h->occ_ev)
        if (e) {
            cudaEventSynchronize(e);
            cudaEventDestroy(e);
        }
    snap_give(h->occ_host);
    if (h->ctx) dfree(h, h->ctx);
    // hand the freed memory beyond what the pool keeps back now, not at some
    // later synchronisation of another box's work
    if (cudaMemPool_t pool = lib_pool(h->cfg.device)) {
        if (h->stream) cudaStreamSynchronize(h->stream);
        cudaMemPoolTrimTo(pool, POOL_KEEP);
    }
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return PIC_OK;
}

pic_status pic_set_stream(pic_handle* h, void* stream) {
    if (!h) return fail(h, PIC_ERR_ARG, "handle is NULL");
    cudaSetDevice(h->cfg.device);
    cudaStreamSynchronize(h->stream);
    if (stream) {
        if (h->own_stream) cudaStreamDestroy(h->stream);
        h->stream = (cudaStream_t)stream;
        h->own_stream = false;
    } else if (!h->own_stream) {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(h, PIC_ERR_CUDA, "cudaStreamCreate failed");
        h->own_stream = true;
    }
    return PIC_OK;
}

pic_status pic_synchronize(pic_handle* h) {
    if (!h) return fail(h, PIC_ERR_ARG, "handle is NULL");
    cudaSetDevice(h->cfg.device);
    CK(cudaStreamSynchronize(h->stream));
    return PIC_OK;
}

static pic_status check_species(pic_handle* h, int species) {
    if (!h) return fail(h, PIC_ERR_ARG, "handle is NULL");
    cudaSetDevice(h->cfg.device);
    if (species < 0 || species >= PIC_MAX_SPECIES) return fail(h, PIC_ERR_ARG, "species index %d out of range", species);
    return PIC_OK;
}

pic_status pic_load_particles(pic_handle* h, int species, double q, double m, int64_t n, const double* x, const double* u,
                              const uint32_t* id) {
    pic_status st = check_species(h, species);
    if (st != PIC_OK) return st;
    if (n < 0 || (n > 0 && (!x || !u))) return fail(h, PIC_ERR_ARG, "bad particle arrays");
    if (!(m > 0) || !std::isfinite(q)) return fail(h, PIC_ERR_ARG, "mass must be > 0 and charge finite");
    if (n >= (1ll << 31)) return fail(h, PIC_ERR_ARG, "at most 2^31 - 1 particles per species");
    CK(cudaStreamSynchronize(h->stream));
    h->sp[species].q = q;
    h->sp[species].m = m;
    return DISPATCH(h, load_t, h, species, (long long)n, x, u, id, (const double*)nullptr);
}

pic_status pic_load_maxwellian(pic_handle* h, int species, double q, double m, int ppc, double theta, const double drift[3],
                               double noise_sigma, uint32_t seed, uint32_t id_base) {
    pic_status st = check_species(h, species);
    if (st != PIC_OK) return st;
    if (ppc < 0 || !(m > 0) || theta < 0 || noise_sigma < 0) return fail(h, PIC_ERR_ARG, "bad loader arguments");
    // no host wait: reallocation and loading are ordered on the handle's stream
    h->sp[species].q = q;
    h->sp[species].m = m;
    return DISPATCH(h, maxwellian_t, h, species, ppc, theta, drift, noise_sigma, seed, id_base);
}

pic_status pic_set_fields(pic_handle* h, const double* E, const double* B) {
    if (!h || !E || !B) return fail(h, PIC_ERR_ARG, "NULL argument");
    cudaSetDevice(h->cfg.device);
    return DISPATCH(h, set_fields_t, h, E, B);
}

pic_status pic_set_uniform_fields(pic_handle* h, const double E[3], const double B[3]) {
    if (!h || !E || !B) return fail(h, PIC_ERR_ARG, "NULL argument");
    cudaSetDevice(h->cfg.device);
    return DISPATCH(h, uniform_fields_t, h, E, B);
}

static pic_status check_error_word(pic_handle* h) {
    int e = 0;
    CK(cudaMemcpyAsync(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (e & ERRB_TMA_TIMEOUT) return fail(h, PIC_ERR_TIMEOUT, "a field-staging wait expired (error word %d)", e);
    if (e & ERRB_NONFINITE) return fail(h, PIC_ERR_NUMERIC, "non-finite particle velocity (error word %d)", e);
    if (e & ERRB_LOOSE_OVERFLOW) return fail(h, PIC_ERR_STATE, "loose-particle list overflowed (error word %d)", e);
    if (e & ERRB_BATCH) return fail(h, PIC_ERR_STATE, "a batched launch met an inconsistent work item (error word %d)", e);
    if (e & ERRB_SMEM_ALIGN) return fail(h, PIC_ERR_STATE, "misaligned shared-memory staging area (error word %d)", e);
    if (e & ERRB_J_RANGE)
        return fail(h, PIC_ERR_NUMERIC, "a tile current reached half the fixed-point range (error word %d)", e);
    if (e) return fail(h, PIC_ERR_STATE, "device error word %d", e);
    return PIC_OK;
}

// Step graphs: consecutive steps starting from one particle buffer are
// captured into a CUDA graph; all per-step scalars come from the device
// context, so the graph is replayed unchanged for every later cycle that
// starts from that buffer.  On any capture failure graphs are switched off
// for this handle.  Steps per captured graph: a regroup and the steps up to
// the next one, or a pair of steps when regrouping is off.
static int graph_cycle(const pic_handle* h) { return h->regroup_every > 0 ? h->regroup_every : 2; }

// Capture one cycle of steps starting from buffer h->buf (with the regroup
// due, when regroups are on) as the graph of that buffer.
static pic_status capture_cycle(pic_handle* h) {
    const int b0 = h->buf;
    const long long s0 = h->step, l0 = h->prof.launches;
    const int r0 = h->since_regroup;
    const int ncyc = graph_cycle(h);
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        h->graphs_on = false;
        cudaGetLastError();
        return PIC_OK;
    }
    pic_status st = PIC_OK;
    for (int k = 0; k < ncyc && st == PIC_OK; ++k) st = DISPATCH(h, step_t, h);
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    h->buf = b0;
    h->step = s0;
    h->since_regroup = r0;
    h->graph_kernels = h->prof.launches - l0;
    h->prof.launches = l0;
    if (st != PIC_OK || e != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        h->graphs_on = false;
        return st == PIC_OK ? PIC_OK : st;
    }
    e = cudaGraphInstantiate(&h->gexec[b0], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->gexec[b0] = nullptr;
        h->graphs_on = false;
        return PIC_OK;
    }
    h->graph_ok[b0] = true;
    return PIC_OK;
}

pic_status pic_set_step(pic_handle* h, int64_t step) {
    if (!h) return fail(h, PIC_ERR_ARG, "handle is NULL");
    cudaSetDevice(h->cfg.device);
    if (step < 0) return fail(h, PIC_ERR_ARG, "step must be >= 0");
    h->step = step;
    long long ns = step;
    CK(cudaMemcpyAsync(&h->ctx->next_step, &ns, sizeof(ns), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return DISPATCH(h, refill_t, h);
}

// The periodic capacity check of pic_step.  Two occupancy snapshots are in
// flight, taken one check apart; each check acts on the older one -- waiting
// for it if the GPU is that far behind, which also bounds how many steps the
// host queues ahead of the GPU (about two checks) -- and takes a new snapshot
// in its slot.  Only a re-layout, when the snapshot shows crowding, waits for
// the GPU to drain.
static pic_status capacity_check(pic_handle* h) {
    const int nv = 2 * PIC_MAX_SPECIES;  // largest occupancy of each species since the last snapshot, loose counts
    static_assert(2 * nv == SNAP_INTS, "a snapshot slot holds two snapshots");
    for (cudaEvent_t& e : h->occ_ev)
        if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            e = nullptr;
            return fail(h, PIC_ERR_CUDA, "cannot create the occupancy snapshot events");
        }
    if (!h->occ_host && !(h->occ_host = snap_take())) return fail(h, PIC_ERR_OOM, "cannot allocate the occupancy snapshots");
    const int k = h->occ_next;
    int* snap = h->occ_host + k * nv;
    if (h->occ_pending[k]) {
        if (!h->check_block && cudaEventQuery(h->occ_ev[k]) != cudaSuccess) return PIC_OK;  // look again next time
        CK(cudaEventSynchronize(h->occ_ev[k]));
        h->occ_pending[k] = false;
        bool pressure = false;
        for (int s = 0; s < PIC_MAX_SPECIES; ++s) {
            const DevSpecies& d = h->sp[s];
            if (!d.loaded) continue;
            if (snap[s] > 0.9 * d.tcap || snap[PIC_MAX_SPECIES + s] > d.lcap / 4) pressure = true;
        }
        if (pressure) {
            bool grown = false;
            pic_status st = DISPATCH(h, regrow_t, h, false, &grown);
            if (st != PIC_OK) return st;
            if (grown) h->occ_pending[1 - k] = false;  // taken on the old layout
        }
    }
    CK(cudaMemcpyAsync(snap, h->occ_dev, sizeof(int) * nv, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemsetAsync(h->occ_dev, 0, sizeof(int) * PIC_MAX_SPECIES, h->stream));  // restart the running maxima
    CK(cudaEventRecord(h->occ_ev[k], h->stream));
    h->occ_pending[k] = true;
    h->occ_next = 1 - k;
    return PIC_OK;
}

pic_status pic_step(pic_handle* h, int nsteps) {
    if (!h) return fail(h, PIC_ERR_ARG, "handle is NULL");
    if (h->batched) return fail(h, PIC_ERR_STATE, "the box is stepped by a batch");
    cudaSetDevice(h->cfg.device);
    if (nsteps < 0) return fail(h, PIC_ERR_ARG, "nsteps must be >= 0");
    while (nsteps > 0) {
        if (h->check_every > 0 && h->since_check >= h->check_every) {
            h->since_check = 0;
            pic_status st = capacity_check(h);
            if (st != PIC_OK) return st;
        }
        const int ncyc = graph_cycle(h);
        const bool due = h->regroup_every == 0 || h->since_regroup >= h->regroup_every;
        if (h->graphs_on && !h->prof.on && nsteps >= ncyc && due) {
            const int b0 = h->buf;
            if (!h->graph_ok[b0]) {
                pic_status st = capture_cycle(h);
                if (st != PIC_OK) return st;
            }
            if (h->graph_ok[b0]) {
                CK(cudaGraphLaunch(h->gexec[b0], h->stream));
                h->step += ncyc;
                h->since_check += ncyc;
                if (h->regroup_every > 0) {
                    h->since_regroup = ncyc;
                    h->buf = (ncyc + 1) % 2 ? 1 - b0 : b0;  // one flip per step and one for the regroup
                }
                h->prof.launches += h->graph_kernels;
                nsteps -= ncyc;
                continue;
            }
        }
        pic_status st = DISPATCH(h, step_t, h);
        if (st != PIC_OK) return st;
        h->since_check += 1;
        nsteps -= 1;
    }
    return PIC_OK;
}

pic_status pic_set_capacity_check(pic_handle* h, int32_t every, int32_t block) {
    if (!h) return fail(h, PIC_ERR_ARG, "handle is NULL");
    if (every < 0) return fail(h, PIC_ERR_ARG, "check interval must be >= 0");
    h->check_every = every;
    h->check_block = block != 0;
    return PIC_OK;
}

pic_status pic_set_regroup_interval(pic_handle* h, int32_t every) {
    if (!h) return fail(h, PIC_ERR_ARG, "handle is NULL");
    if (every < 0) return fail(h, PIC_ERR_ARG, "regroup interval must be >= 0");
    if (every == h->regroup_every) return PIC_OK;
    cudaSetDevice(h->cfg.device);
    CK(cudaStreamSynchronize(h->stream));
    drop_graphs(h);
    h->regroup_every = every;
    return PIC_OK;
}

pic_status pic_get_regroup_interval(pic_handle* h, int32_t* every) {
    if (!h || !every) return fail(h, PIC_ERR_ARG, "NULL argument");
    *every = h->regroup_every;
    return PIC_OK;
}

pic_status pic_rebalance(pic_handle* h, int32_t force, int32_t* grown) {
    if (!h) return fail(h, PIC_ERR_ARG, "handle is NULL");
    if (h->batched) return fail(h, PIC_ERR_STATE, "the box is stepped by a batch");
    cudaSetDevice(h->cfg.device);
    bool g = false;
    pic_status st = DISPATCH(h, regrow_t, h, force != 0, &g);
    if (grown) *grown = g ? 1 : 0;
    return st;
}

pic_status pic_get_capacity(pic_handle* h, int species, int64_t* slots_per_tile, int64_t* loose_capacity,
                            int64_t* relayouts) {
    pic_status st = check_species(h, species);
    if (st != PIC_OK) return st;
    if (slots_per_tile) *slots_per_tile = h->sp[species].tcap;
    if (loose_capacity) *loose_capacity = h->sp[species].lcap;
    if (relayouts) *relayouts = h->regrows;
    return PIC_OK;
}

pic_status pic_diagnostics(pic_handle* h, pic_diag* out) {
    if (!h || !out) return fail(h, PIC_ERR_ARG, "NULL argument");
    cudaSetDevice(h->cfg.device);
    memset(out, 0, sizeof(*out));
    CK(cudaStreamSynchronize(h->stream));
    out->step = h->step;
    out->t = (double)h->step;
    out->shear_shift = shear_shift(h, out->t);
    lvals(h, out->t, out->l);
    pic_status st = DISPATCH(h, diag_t, h, out);
    if (st != PIC_OK) return st;
    unsigned long long cnt[2];
    CK(cudaMemcpyAsync(cnt, h->counters, sizeof(cnt), cudaMemcpyDeviceToHost, h->stream));
    int e = 0;
    CK(cudaMemcpyAsync(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    out->escaped_total = (int64_t)cnt[0];
    out->superluminal_total = (int64_t)cnt[1];
    out->error_word = e;
    return check_error_word(h);
}

pic_status pic_clear_error(pic_handle* h) {
    if (!h) return fail(h, PIC_ERR_ARG, "handle is NULL");
    cudaSetDevice(h->cfg.device);
    CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return PIC_OK;
}

pic_status pic_get_count(pic_handle* h, int species, int64_t* n) {
    pic_status st = check_species(h, species);
    if (st != PIC_OK) return st;
    if (!n) return fail(h, PIC_ERR_ARG, "n is NULL");
    *n = h->sp[species].loaded ? h->sp[species].n : 0;
    return PIC_OK;
}

pic_status pic_get_particles(pic_handle* h, int species, double* x, double* u, uint32_t* id, double* dr) {
    pic_status st = check_species(h, species);
    if (st != PIC_OK) return st;
    if (!h->sp[species].loaded) return fail(h, PIC_ERR_STATE, "species %d is not loaded", species);
    CK(cudaStreamSynchronize(h->stream));
    return DISPATCH(h, compact_t, h, species, x, u, id, dr);
}

pic_status pic_get_particles_sampled(pic_handle* h, int species, uint32_t modulus, uint32_t remainder, int64_t max_out,
                                     double* x, double* u, uint32_t* id, double* dr, int64_t* n_out) {
    pic_status st = check_species(h, species);
    if (st != PIC_OK) return st;
    if (!h->sp[species].loaded) return fail(h, PIC_ERR_STATE, "species %d is not loaded", species);
    if (modulus == 0 || remainder >= modulus || max_out < 0 || !n_out)
        return fail(h, PIC_ERR_ARG, "need modulus > remainder, max_out >= 0 and n_out");
    CK(cudaStreamSynchronize(h->stream));
    long long n = 0;
    st = DISPATCH(h, sample_t, h, species, modulus, remainder, (long long)max_out, x, u, id, dr, &n);
    *n_out = n;
    return st;
}

pic_status pic_get_fields(pic_handle* h, double* E, double* B, double* J) {
    if (!h) return fail(h, PIC_ERR_ARG, "handle is NULL");
    cudaSetDevice(h->cfg.device);
    return DISPATCH(h, get_fields_t, h, E, B, J);
}

pic_status pic_set_profiling(pic_handle* h, int enable) {
    if (!h) return fail(h, PIC_ERR_ARG, "handle is NULL");
    h->prof.on = enable != 0;
    return PIC_OK;
}

pic_status pic_get_profile(pic_handle* h, pic_profile* out) {
    if (!h || !out) return fail(h, PIC_ERR_ARG, "NULL argument");
    prof_resolve(h);
    out->ms_particle = h->prof.ms[0];
    out->ms_other = h->prof.ms[1];
    out->ms_field = h->prof.ms[2];
    out->launches = h->prof.launches;
    out->particle_launches = h->prof.particle_launches;
    out->particle_steps = h->prof.particle_steps;
    return PIC_OK;
}

extern "C" int pic_internal_noalloc_preload(void);  // noalloc.cu

pic_status pic_preload_kernels(int32_t device, int32_t precision) {
    if (precision != PIC_FP32 && precision != PIC_FP64) return fail(nullptr, PIC_ERR_ARG, "bad precision");
    if (cudaSetDevice(device) != cudaSuccess) return fail(nullptr, PIC_ERR_CUDA, "no such CUDA device");
    const bool fp64 = precision == PIC_FP64;
    const int pushes[9][2] = {{PUSH_BORIS, ESC_NONE}, {PUSH_BORIS, ESC_DISP}, {PUSH_BORIS, ESC_PROB},
                              {PUSH_KSB, ESC_NONE},   {PUSH_KEB, ESC_NONE},   {PUSH_SXE, ESC_NONE},
                              {PUSH_KSB, ESC_PROB},   {PUSH_KEB, ESC_PROB},   {PUSH_SXE, ESC_PROB}};
    cudaFuncAttributes a;
    for (int tg = 0; tg < N_TGEOM; ++tg)
        for (int ord = 1; ord <= 2 && tgeom_built(tg, fp64); ++ord)
            for (const auto& pe : pushes) {
                const KernelSet ks = lookup_kernels(fp64, tg, ord, pe[0], pe[1]);
                for (const void* f : ks.tile)
                    if (cudaFuncGetAttributes(&a, f) != cudaSuccess) return fail(nullptr, PIC_ERR_CUDA, "kernel load failed");
                if (cudaFuncGetAttributes(&a, ks.loose) != cudaSuccess || cudaFuncGetAttributes(&a, ks.batch) != cudaSuccess)
                    return fail(nullptr, PIC_ERR_CUDA, "kernel load failed");
            }
    if (pic_internal_noalloc_preload() != 0)
        return fail(nullptr, PIC_ERR_CUDA, "loading the allocation-free reduction failed");
    return PIC_OK;
}

int pic_kernel_variant_count(void) { return N_TILE_VARIANTS; }

pic_status pic_kernel_variant_info(int32_t k, int32_t* threads_per_cta, int32_t* stable, int32_t* copies) {
    if (k < 1 || k > N_TILE_VARIANTS) return fail(nullptr, PIC_ERR_ARG, "kernel variant %d out of range", (int)k);
    if (threads_per_cta) *threads_per_cta = TILE_VARIANTS[k - 1].nt;
    if (stable) *stable = TILE_VARIANTS[k - 1].stable;
    if (copies) *copies = TILE_VARIANTS[k - 1].jc;
    return PIC_OK;
}

pic_status pic_get_kernel_variant(pic_handle* h, int32_t* k) {
    if (!h || !k) return fail(h, PIC_ERR_ARG, "NULL argument");
    *k = h->tile_variant + 1;
    return PIC_OK;
}

pic_status pic_set_kernel_variant(pic_handle* h, int32_t k) {
    if (!h) return fail(h, PIC_ERR_ARG, "handle is NULL");
    if (k < 1 || k > N_TILE_VARIANTS) return fail(h, PIC_ERR_ARG, "kernel variant %d out of range", (int)k);
    const int v = k - 1;
    const size_t smem = tile_smem_bytes(h->fp64, h->tg, v);
    if (smem > MAX_SMEM) return fail(h, PIC_ERR_ARG, "kernel variant %d needs %zu bytes of shared memory", (int)k, smem);
    cudaSetDevice(h->cfg.device);
    if (cudaFuncSetAttribute(h->ks.tile[v], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return fail(h, PIC_ERR_CUDA, "cannot set %zu bytes of dynamic shared memory", smem);
    drop_graphs(h);
    h->tile_variant = v;
    h->tile_threads = TILE_VARIANTS[v].nt;
    h->smem_bytes = smem;
    h->tile_fn = h->ks.tile[v];
    return PIC_OK;
}

pic_status pic_autotune_regroup(pic_handle* h, const int32_t* candidates, int32_t n, int32_t cycles, int32_t* best,
                                double* ms_per_step) {
    if (!h || !candidates || n < 1 || cycles < 1) return fail(h, PIC_ERR_ARG, "bad arguments");
    if (h->fp64) return fail(h, PIC_ERR_ARG, "FP64 boxes keep regrouping off");
    for (int i = 0; i < n; ++i)
        if (candidates[i] < 0) return fail(h, PIC_ERR_ARG, "intervals must be >= 0");
    cudaSetDevice(h->cfg.device);
    const bool prof_was = h->prof.on;
    const int start = h->regroup_every;
    prof_resolve(h);
    const double ms0[3] = {h->prof.ms[0], h->prof.ms[1], h->prof.ms[2]};
    const long long l0 = h->prof.launches, pl0 = h->prof.particle_launches, ps0 = h->prof.particle_steps;
    pic_status st = PIC_OK;
    int bi = -1;
    double bms = 0.0;
    for (int i = 0; i < n && st == PIC_OK; ++i) {
        st = pic_set_regroup_interval(h, candidates[i]);
        if (st != PIC_OK) break;
        const int cyc = candidates[i] > 0 ? candidates[i] : 2;
        h->prof.on = false;
        st = pic_step(h, cyc);  // one untimed cycle: the order settles into this interval's rhythm
        if (st != PIC_OK) break;
        prof_resolve(h);
        const double before = h->prof.ms[0] + h->prof.ms[1] + h->prof.ms[2];
        h->prof.on = true;
        st = pic_step(h, cyc * cycles);
        prof_resolve(h);
        const double per = (h->prof.ms[0] + h->prof.ms[1] + h->prof.ms[2] - before) / (cyc * cycles);
        if (ms_per_step) ms_per_step[i] = per;
        if (bi < 0 || per < bms) {
            bi = i;
            bms = per;
        }
    }
    h->prof.ms[0] = ms0[0];
    h->prof.ms[1] = ms0[1];
    h->prof.ms[2] = ms0[2];
    h->prof.launches = l0;
    h->prof.particle_launches = pl0;
    h->prof.particle_steps = ps0;
    h->prof.on = prof_was;
    if (st != PIC_OK || bi < 0) {
        pic_set_regroup_interval(h, start);
        return st != PIC_OK ? st : fail(h, PIC_ERR_STATE, "no interval was timed");
    }
    st = pic_set_regroup_interval(h, candidates[bi]);
    if (st == PIC_OK && best) *best = candidates[bi];
    return st;
}

// Switch a handle to the particle tiles of template geometry tg (2D FP32:
// 16 x 16 or 32 x 32 cells).  Every species is read out into flat device
// arrays (position = cell + offset in FP64, which holds the FP32 cell and
// offset exactly, so the round trip changes no particle), its arrays are
// freed and it is loaded again under the new tiling.  The kernels, shared
// memory attributes and field tensor maps follow the new tiles.  If the new
// layout cannot be made, the old one is made again from the same copies.
static pic_status switch_tiling(pic_handle* h, int tg) {
    h->tg = tg;
    set_tiling(h);
    int v = h->tile_variant;
    if (tile_smem_bytes(h->fp64, tg, v) > MAX_SMEM) v = default_variant(h->fp64, tg);
    h->ks = lookup_kernels(h->fp64, tg, h->cfg.shape_order, h->push, h->esc);
    h->tile_variant = v;
    h->tile_threads = TILE_VARIANTS[v].nt;
    h->smem_bytes = tile_smem_bytes(h->fp64, tg, v);
    h->tile_fn = h->ks.tile[v];
    if (cudaFuncSetAttribute(h->tile_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->smem_bytes) != cudaSuccess)
        return fail(h, PIC_ERR_CUDA, "cannot set %zu bytes of dynamic shared memory", h->smem_bytes);
    if (DISPATCH(h, regroup_attr_t, h) != PIC_OK) return PIC_ERR_CUDA;
    if (encode_field_map(h, &h->tmE, h->E) != PIC_OK || encode_field_map(h, &h->tmB, h->B) != PIC_OK) return PIC_ERR_CUDA;
    return PIC_OK;
}

static pic_status retile(pic_handle* h, int tg) {
    if (tg == h->tg) return PIC_OK;
    if (h->batched) return fail(h, PIC_ERR_STATE, "the box is stepped by a batch");
    CK(cudaStreamSynchronize(h->stream));
    struct Flat {
        double* x = nullptr;
        double* u = nullptr;
        uint32_t* id = nullptr;
        double* dr = nullptr;
        long long n = 0;
        bool on = false;
    };
    Flat f[PIC_MAX_SPECIES];
    const bool hd = h->esc == ESC_DISP;
    auto free_flat = [&]() {
        for (Flat& q : f) {
            dfree(h, q.x);
            dfree(h, q.u);
            dfree(h, q.id);
            dfree(h, q.dr);
            q = Flat();
        }
    };
    for (int s = 0; s < PIC_MAX_SPECIES; ++s) {
        DevSpecies& d = h->sp[s];
        if (!d.loaded) continue;
        Flat& q = f[s];
        q.n = d.n;
        q.on = true;
        const size_t m = (size_t)std::max(1ll, d.n);
        if (dalloc(h, (void**)&q.x, sizeof(double) * 3 * m) != cudaSuccess ||
            dalloc(h, (void**)&q.u, sizeof(double) * 3 * m) != cudaSuccess ||
            dalloc(h, (void**)&q.id, sizeof(uint32_t) * m) != cudaSuccess ||
            (hd && dalloc(h, (void**)&q.dr, sizeof(double) * 3 * m) != cudaSuccess)) {
            cudaGetLastError();
            free_flat();
            return fail(h, PIC_ERR_OOM, "re-tiling: no room for a flat copy of the particles (the tiling is kept)");
        }
        const pic_status st = DISPATCH(h, compact_t, h, s, q.x, q.u, q.id, q.dr);
        if (st != PIC_OK) {
            free_flat();
            return st;
        }
    }
    CK(cudaStreamSynchronize(h->stream));
    drop_graphs(h);
    // the per-tile counters are sized by the tile count: drop them with the arrays
    auto drop_species = [&]() {
        for (int s = 0; s < PIC_MAX_SPECIES; ++s) {
            if (!f[s].on) continue;
            DevSpecies& d = h->sp[s];
            for (int b = 0; b < 2; ++b) {
                for (int i = 0; i < 11; ++i) {
                    dfree(h, d.arr[b][i]);
                    dfree(h, d.larr[b][i]);
                    d.arr[b][i] = d.larr[b][i] = nullptr;
                }
                dfree(h, d.stay[b]);
                dfree(h, d.arrv[b]);
                d.stay[b] = d.arrv[b] = nullptr;
            }
            d.loaded = false;
        }
    };
    auto load_all = [&]() -> pic_status {
        for (int s = 0; s < PIC_MAX_SPECIES; ++s) {
            if (!f[s].on) continue;
            const pic_status st = DISPATCH(h, load_t, h, s, f[s].n, f[s].x, f[s].u, f[s].id, f[s].dr);
            if (st != PIC_OK) return st;
        }
        return PIC_OK;
    };
    const int old_tg = h->tg;
    const int old_variant = h->tile_variant;
    drop_species();
    h->buf = 0;
    pic_status st = switch_tiling(h, tg);
    if (st == PIC_OK) st = load_all();
    if (st != PIC_OK) {
        const std::string why = h->last_error;
        drop_species();
        h->tile_variant = old_variant;
        pic_status back = switch_tiling(h, old_tg);
        if (back == PIC_OK) back = load_all();
        free_flat();
        if (back != PIC_OK) return fail(h, PIC_ERR_STATE, "re-tiling failed (%s) and the old tiling could not be restored", why.c_str());
        return fail(h, st, "re-tiling failed (the old tiling is restored): %s", why.c_str());
    }
    free_flat();
    for (int k = 0; k < 2; ++k) h->occ_pending[k] = false;
    CK(cudaMemsetAsync(h->occ_dev, 0, sizeof(int) * 2 * PIC_MAX_SPECIES, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return PIC_OK;
}

pic_status pic_get_tile(pic_handle* h, int32_t tile[3]) {
    if (!h || !tile) return fail(h, PIC_ERR_ARG, "NULL argument");
    tile[0] = h->tl.tx;
    tile[1] = h->tl.ty;
    tile[2] = h->tl.tz;
    return PIC_OK;
}

pic_status pic_set_tile(pic_handle* h, int32_t side) {
    if (!h) return fail(h, PIC_ERR_ARG, "handle is NULL");
    if (h->geom == 0 && side != 4 && side != 8) return fail(h, PIC_ERR_ARG, "3D tiles are 4x4x4 or 8x8x8");
    if (h->geom != 0 && side != 8 && side != 16 && !(side == 32 && !h->fp64))
        return fail(h, PIC_ERR_ARG, "2D tiles are 8x8, 16x16, or 32x32 in FP32");
    cudaSetDevice(h->cfg.device);
    return retile(h, tgeom_of(h->geom, side));
}

pic_status pic_autotune(pic_handle* h, int32_t trial_steps, int32_t* best, double* ms_per_variant,
                        int64_t* steps_taken) {
    if (!h) return fail(h, PIC_ERR_ARG, "handle is NULL");
    if (trial_steps < 1) return fail(h, PIC_ERR_ARG, "trial_steps must be >= 1");
    cudaSetDevice(h->cfg.device);
    const bool prof_was = h->prof.on;
    const int start_variant = h->tile_variant;
    double ms[N_TILE_VARIANTS];
    long long launches[N_TILE_VARIANTS];
    bool fits[N_TILE_VARIANTS];
    for (int v = 0; v < N_TILE_VARIANTS; ++v) {
        ms[v] = 0.0;
        launches[v] = 0;
        fits[v] = tile_smem_bytes(h->fp64, h->tg, v) <= MAX_SMEM;
    }
    long long taken = 0;
    // two interleaved rounds, so that every variant sees particles in a
    // similar order (the order within tiles evolves from step to step)
    const int rounds = 2;
    const int per_round = (trial_steps + rounds - 1) / rounds;
    prof_resolve(h);
    const double ms0[3] = {h->prof.ms[0], h->prof.ms[1], h->prof.ms[2]};
    const long long l0 = h->prof.launches, pl0 = h->prof.particle_launches, ps0 = h->prof.particle_steps;
    pic_status st = PIC_OK;
    for (int r = 0; r < rounds && st == PIC_OK; ++r)
        for (int v = 0; v < N_TILE_VARIANTS && st == PIC_OK; ++v) {
            if (!fits[v]) continue;
            st = pic_set_kernel_variant(h, v + 1);
            if (st != PIC_OK) break;
            h->prof.on = false;
            st = pic_step(h, 1);  // first launch of the variant: not timed
            taken += 1;
            if (st != PIC_OK) break;
            prof_resolve(h);
            const double before = h->prof.ms[0];
            const long long lb = h->prof.particle_launches;
            h->prof.on = true;
            st = pic_step(h, per_round);
            taken += per_round;
            prof_resolve(h);
            ms[v] += h->prof.ms[0] - before;
            launches[v] += h->prof.particle_launches - lb;
        }
    // the profile counters are the caller's: put them back
    h->prof.ms[0] = ms0[0];
    h->prof.ms[1] = ms0[1];
    h->prof.ms[2] = ms0[2];
    h->prof.launches = l0;
    h->prof.particle_launches = pl0;
    h->prof.particle_steps = ps0;
    h->prof.on = prof_was;
    if (st != PIC_OK) {
        pic_set_kernel_variant(h, start_variant + 1);
        return st;
    }
    int bv = start_variant;
    for (int v = 0; v < N_TILE_VARIANTS; ++v)
        if (fits[v] && launches[v] > 0 && (launches[bv] == 0 || ms[v] / launches[v] < ms[bv] / launches[bv])) bv = v;
    st = pic_set_kernel_variant(h, bv + 1);
    if (st != PIC_OK) return st;
    if (best) *best = bv + 1;
    if (ms_per_variant)
        for (int v = 0; v < N_TILE_VARIANTS; ++v) ms_per_variant[v] = launches[v] > 0 ? ms[v] / launches[v] : -1.0;
    if (steps_taken) *steps_taken = taken;
    return PIC_OK;
}

pic_status pic_autotune_tile(pic_handle* h, int32_t trial_steps, int32_t* best_side, double* ms_per_side) {
    if (!h) return fail(h, PIC_ERR_ARG, "handle is NULL");
    if (trial_steps < 1) return fail(h, PIC_ERR_ARG, "trial_steps must be >= 1");
    cudaSetDevice(h->cfg.device);
    // 3D: 4 and 8; 2D: 8, 16 and (no FP64 kernels for 32 x 32 tiles) 32
    int sides[3] = {8, 16, 32};
    int nsides = h->fp64 ? 2 : 3;
    if (h->geom == 0) {
        sides[0] = 4;
        sides[1] = 8;
        nsides = 2;
    }
    const int start_side = h->tl.tx;
    const bool prof_was = h->prof.on;
    prof_resolve(h);
    const double ms0[3] = {h->prof.ms[0], h->prof.ms[1], h->prof.ms[2]};
    const long long l0 = h->prof.launches, pl0 = h->prof.particle_launches, ps0 = h->prof.particle_steps;
    double per[3] = {-1.0, -1.0, -1.0};
    int var[3] = {0, 0, 0};
    pic_status st = PIC_OK;
    for (int k = 0; k < nsides && st == PIC_OK; ++k) {
        st = pic_set_tile(h, sides[k]);
        if (st != PIC_OK) break;
        // the best launch variant for these tiles, then whole steps with it
        int32_t bv = 0;
        st = pic_autotune(h, trial_steps, &bv, nullptr, nullptr);
        if (st != PIC_OK) break;
        var[k] = bv;
        h->prof.on = false;
        st = pic_step(h, 1);
        if (st != PIC_OK) break;
        prof_resolve(h);
        const double before = h->prof.ms[0] + h->prof.ms[1] + h->prof.ms[2];
        h->prof.on = true;
        st = pic_step(h, trial_steps);
        prof_resolve(h);
        per[k] = (h->prof.ms[0] + h->prof.ms[1] + h->prof.ms[2] - before) / trial_steps;
    }
    h->prof.ms[0] = ms0[0];
    h->prof.ms[1] = ms0[1];
    h->prof.ms[2] = ms0[2];
    h->prof.launches = l0;
    h->prof.particle_launches = pl0;
    h->prof.particle_steps = ps0;
    h->prof.on = prof_was;
    if (st != PIC_OK) {
        const std::string why = h->last_error;
        pic_set_tile(h, start_side);
        return fail(h, st, "%s", why.c_str());
    }
    int b = 0;
    for (int k = 1; k < nsides; ++k)
        if (per[k] >= 0.0 && per[k] < per[b]) b = k;
    st = pic_set_tile(h, sides[b]);
    if (st == PIC_OK && var[b] > 0) st = pic_set_kernel_variant(h, var[b]);
    if (st != PIC_OK) return st;
    if (best_side) *best_side = sides[b];
    if (ms_per_side)
        for (int k = 0; k < 3; ++k) ms_per_side[k] = per[k];
    return PIC_OK;
}

pic_status pic_reset_profile(pic_handle* h) {
    if (!h) return fail(h, PIC_ERR_ARG, "handle is NULL");
    prof_resolve(h);
    h->prof.ms[0] = h->prof.ms[1] = h->prof.ms[2] = 0.0;
    h->prof.launches = h->prof.particle_launches = h->prof.particle_steps = 0;
    return PIC_OK;
}


// ---- batches: many boxes of one kind, one persistent particle kernel per step ----------------

}  // extern "C"

struct pic_batch {
    std::vector<pic_handle*> box;
    std::vector<cudaStream_t> home;  // the boxes' streams, given back at destroy
    cudaStream_t stream = nullptr;   // the batch's stream
    std::vector<cudaStream_t> side;  // box i runs its own kernels on side[i % side.size()]
    std::vector<cudaEvent_t> ev;     // fork / join events: one per side stream, plus the fork
    int device = 0;
    bool fp64 = false;
    int tg = 0;  // the members' template geometry
    const void* kern = nullptr;
    int nt = 256;
    size_t smem = 0;
    int max_grid = 0;  // resident CTAs of the batched kernel on the device
    size_t args_bytes = 0;
    // per phase (parity of the step relative to creation): one parameter image per launch
    std::vector<std::vector<unsigned char>> args[2];
    std::vector<int> nwork[2];
    int* counters = nullptr;  // work counters, one per launch
    int phase = 0;
    // Unsheared kinds (multi): the boxes are split into lanes.  A lane is a
    // chain of batched launches on its own side stream: its boxes' step
    // contexts, one persistent particle kernel over their tiles, their loose
    // particles, and their grid work in one launch per field kernel.  The
    // lanes are forked from the batch stream at the start of a cycle of steps
    // and joined at its end, so one lane's field work and the tail of its
    // particle kernel overlap the other lanes' particle kernels.
    struct FieldTab {
        void* dev = nullptr;    // FieldBox[n], then four z-offset tables of n + 1 ints
        size_t zoff_bytes = 0;  // byte offset of the z-offset tables
        int n = 0;
        int ztot[4] = {0, 0, 0, 0};  // slabs per table: cells, x guards, y guards, z guards
        int mx_nx = 0, mx_ny = 0, mx_nz = 0, mx_px = 0, mx_py = 0;
    };
    struct Lane {
        std::vector<int> idx;  // the lane's boxes (indices into box)
        std::vector<unsigned char> args[2];
        int nwork[2] = {0, 0};
        FieldTab ft;
    };
    bool multi = false;
    std::vector<Lane> lanes;
    int regroup_every = 0;  // regroup every box by cell every this many steps (0: never)
    int since_regroup = 0;
    bool graphs_on = true;
    bool graph_ok[2] = {false, false};
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
};

namespace {

thread_local std::string g_batch_error;

pic_status batch_fail(pic_status st, const char* msg) {
    g_batch_error = msg;
    pic_internal_set_global_error(msg);
    return st;
}

// A batch's own device memory (work counters, field tables) comes from the
// library's stream-ordered pool on the batch stream: cudaMalloc and cudaFree
// would synchronise the device, stalling every other box and served run.
static cudaError_t balloc(pic_batch* B, void** p, size_t bytes) {
    cudaMemPool_t pool = lib_pool(B->device);
    if (!pool) return cudaMalloc(p, bytes);
    return cudaMallocFromPoolAsync(p, bytes, pool, B->stream);
}

static void bfree(pic_batch* B, void* p) {
    if (!p) return;
    if (lib_pool(B->device)) cudaFreeAsync(p, B->stream);
    else cudaFree(p);
}

// Descriptor images of the batched particle kernel for boxes `idx` (at most
// MAXB): one per phase, the box's buffers at that parity.
template <class T> static void batch_images(pic_batch* B, const std::vector<int>& idx, int* counter,
                                           std::vector<unsigned char> img[2], int nwork[2]) {
    using A_t = BatchArgs<T>;
    for (int ph = 0; ph < 2; ++ph) {
        img[ph].assign(sizeof(A_t), 0);
        A_t* A = reinterpret_cast<A_t*>(img[ph].data());
        const int k = (int)idx.size();
        A->nbox = k;
        A->next = counter;
        A->first[0] = 0;
        for (int j = 0; j < k; ++j) {
            pic_handle* h = B->box[idx[j]];
            BoxDesc<T>& D = A->box[j];
            D.tmE = h->tmE;
            D.tmB = h->tmB;
            D.g = h->g;
            D.tl = h->tl;
            step_params<T>(h, ph == 0 ? h->buf : 1 - h->buf, D.P0, D.SP);
            D.J = h->fp64 ? (JWord<T>*)h->J : (JWord<T>*)(void*)h->Jint;
            D.ctx = h->ctx;
            A->first[j + 1] = A->first[j] + h->tl.ntiles;
        }
        nwork[ph] = A->first[k];
    }
}

// Field descriptors and z-offset tables of boxes `idx`, uploaded to the device.
template <class T> static pic_status field_table(pic_batch* B, const std::vector<int>& idx, pic_batch::FieldTab& ft) {
    const int n = (int)idx.size();
    std::vector<FieldBox<T>> fb(n);
    std::vector<int> z(4 * (n + 1), 0);
    for (int i = 0; i < n; ++i) {
        pic_handle* h = B->box[idx[i]];
        StepP P;
        SpecPack<T> SP;
        step_params<T>(h, h->buf, P, SP);
        FieldBox<T>& f = fb[i];
        f.g = h->g;
        f.E = (T*)h->E;
        f.B = (T*)h->B;
        f.J = (T*)h->Jcur;
        f.Jint = h->Jint;
        f.ctx = h->ctx;
        f.err = h->err;
        f.fx_unit = P.fx_unit;
        f.cc = h->cc;
        const Grid& g = h->g;
        const int ext[4] = {g.nz, 3 * (g.px - g.nx), 3 * (g.py - g.ny), 3 * (g.pz - g.nz)};
        for (int t = 0; t < 4; ++t) z[t * (n + 1) + i + 1] = z[t * (n + 1) + i] + ext[t];
        ft.mx_nx = std::max(ft.mx_nx, g.nx);
        ft.mx_ny = std::max(ft.mx_ny, g.ny);
        ft.mx_nz = std::max(ft.mx_nz, g.nz);
        ft.mx_px = std::max(ft.mx_px, g.px);
        ft.mx_py = std::max(ft.mx_py, g.py);
    }
    ft.n = n;
    for (int t = 0; t < 4; ++t) ft.ztot[t] = z[t * (n + 1) + n];
    ft.zoff_bytes = (sizeof(FieldBox<T>) * n + 15) & ~(size_t)15;
    if (balloc(B, &ft.dev, ft.zoff_bytes + sizeof(int) * z.size()) != cudaSuccess)
        return batch_fail(PIC_ERR_OOM, "pic_batch_create: allocation failed");
    // pageable sources: each copy has left the host buffer when the call returns
    if (cudaMemcpyAsync(ft.dev, fb.data(), sizeof(FieldBox<T>) * n, cudaMemcpyHostToDevice, B->stream) != cudaSuccess ||
        cudaMemcpyAsync((char*)ft.dev + ft.zoff_bytes, z.data(), sizeof(int) * z.size(), cudaMemcpyHostToDevice,
                        B->stream) != cudaSuccess)
        return batch_fail(PIC_ERR_CUDA, "pic_batch_create: table upload failed");
    return PIC_OK;
}

template <class T, int G> pic_status batch_build_t(pic_batch* B) {
    using A_t = BatchArgs<T>;
    const int n = (int)B->box.size();
    B->args_bytes = sizeof(A_t);
    if (B->multi) {
        const int L = (int)B->lanes.size();
        if (balloc(B, (void**)&B->counters, sizeof(int) * L) != cudaSuccess)
            return batch_fail(PIC_ERR_OOM, "pic_batch_create: allocation failed");
        for (int l = 0; l < L; ++l) {
            pic_batch::Lane& ln = B->lanes[l];
            batch_images<T>(B, ln.idx, B->counters + l, ln.args, ln.nwork);
            const pic_status st = field_table<T>(B, ln.idx, ln.ft);
            if (st != PIC_OK) return st;
        }
        return PIC_OK;
    }
    const int ngroups = (n + A_t::MAXB - 1) / A_t::MAXB;
    if (balloc(B, (void**)&B->counters, sizeof(int) * ngroups) != cudaSuccess)
        return batch_fail(PIC_ERR_OOM, "pic_batch_create: allocation failed");
    for (int ph = 0; ph < 2; ++ph) {
        B->args[ph].clear();
        B->nwork[ph].clear();
    }
    for (int g0 = 0; g0 < n; g0 += A_t::MAXB) {
        std::vector<int> idx;
        for (int j = g0; j < std::min(n, g0 + A_t::MAXB); ++j) idx.push_back(j);
        std::vector<unsigned char> img[2];
        int nw[2];
        batch_images<T>(B, idx, B->counters + g0 / A_t::MAXB, img, nw);
        for (int ph = 0; ph < 2; ++ph) {
            B->args[ph].push_back(std::move(img[ph]));
            B->nwork[ph].push_back(nw[ph]);
        }
    }
    return PIC_OK;
}

// The grid work of a step for the boxes of a field table, in batched
// launches on stream s: the current's conversion and guard fold, then the
// leapfrog (B half, E full, B half) with its guard fills.
template <class T, int G> static void multi_fields_t(const pic_batch::FieldTab& ft, cudaStream_t s) {
    using GT = GeomT<G>;
    const int n = ft.n;
    const FieldBox<T>* fb = (const FieldBox<T>*)ft.dev;
    const int* z = (const int*)((const char*)ft.dev + ft.zoff_bytes);
    const int* zc = z;                  // cells
    const int* zx = z + (n + 1);        // x guards
    const int* zy = z + 2 * (n + 1);    // y guards
    const int* zz = z + 3 * (n + 1);    // z guards
    if (sizeof(T) == 4)
        multi_fixed_to_float_kernel<<<dim3(64, n), NTHR, 0, s>>>((const FieldBox<float>*)fb, n);
    if (GT::AZ) multi_fold_z_kernel<T><<<cell_grid(ft.mx_px, ft.mx_py, ft.ztot[3]), CELL_THREADS, 0, s>>>(fb, zz, n);
    if (GT::AY) multi_fold_y_kernel<T><<<cell_grid(ft.mx_px, ft.mx_nz, ft.ztot[2]), CELL_THREADS, 0, s>>>(fb, zy, n);
    multi_fold_x_kernel<T, G><<<cell_grid(ft.mx_ny, ft.mx_nz, ft.ztot[1]), CELL_THREADS, 0, s>>>(fb, zx, n);
    auto fills = [&](int which) { multi_fill_all_kernel<T, G><<<dim3(64, n), NTHR, 0, s>>>(fb, n, which); };
    const dim3 cg = cell_grid(ft.mx_nx, ft.mx_ny, ft.ztot[0]);
    multi_curl_kernel<T, G, true><<<cg, CELL_THREADS, 0, s>>>(fb, zc, n, 0);
    fills(1);
    multi_curl_kernel<T, G, false><<<cg, CELL_THREADS, 0, s>>>(fb, zc, n, 1);
    fills(0);
    multi_curl_kernel<T, G, true><<<cg, CELL_THREADS, 0, s>>>(fb, zc, n, 2);
    fills(1);
}

// Fork: every side stream waits for the batch stream; join: the reverse.
pic_status batch_fork(pic_batch* B) {
    const size_t K = B->side.size();
    if (cudaEventRecord(B->ev[K], B->stream) != cudaSuccess) return batch_fail(PIC_ERR_CUDA, "event record failed");
    for (size_t k = 0; k < K; ++k)
        if (cudaStreamWaitEvent(B->side[k], B->ev[K], 0) != cudaSuccess) return batch_fail(PIC_ERR_CUDA, "stream wait failed");
    return PIC_OK;
}

pic_status batch_join(pic_batch* B) {
    for (size_t k = 0; k < B->side.size(); ++k) {
        if (cudaEventRecord(B->ev[k], B->side[k]) != cudaSuccess) return batch_fail(PIC_ERR_CUDA, "event record failed");
        if (cudaStreamWaitEvent(B->stream, B->ev[k], 0) != cudaSuccess) return batch_fail(PIC_ERR_CUDA, "stream wait failed");
    }
    return PIC_OK;
}

template <class T, int G> pic_status batch_step_t(pic_batch* B) {
    using A_t = BatchArgs<T>;
    // a regroup, when due, runs in each box's branch before its step context;
    // every box flips its buffer, so the batch changes phase
    const bool regroup = B->regroup_every > 0 && B->since_regroup >= B->regroup_every;
    if (regroup) {
        B->phase ^= 1;
        B->since_regroup = 0;
    }
    B->since_regroup += 1;
    const int ph = B->phase;
    pic_status st = PIC_OK;
    if (B->multi) {
        // each lane on its own stream (forked by the caller): regroups, step
        // contexts and current resets, the particle kernel, loose particles,
        // the grid work
        for (size_t l = 0; l < B->lanes.size(); ++l) {
            pic_batch::Lane& ln = B->lanes[l];
            cudaStream_t s = B->side[l];
            for (int i : ln.idx)
                if (regroup && (st = regroup_t<T, G>(B->box[i])) != PIC_OK) return st;
            multi_pre_kernel<T><<<dim3(64, (unsigned)ln.ft.n), NTHR, 0, s>>>((const FieldBox<T>*)ln.ft.dev, ln.ft.n);
            if (cudaMemsetAsync(B->counters + l, 0, sizeof(int), s) != cudaSuccess)
                return batch_fail(PIC_ERR_CUDA, "work counter reset failed");
            const int grid = std::max(1, std::min(ln.nwork[ph], B->max_grid));
            void* a[] = {ln.args[ph].data()};
            if (cudaLaunchKernel(B->kern, dim3(grid), dim3(B->nt), a, B->smem, s) != cudaSuccess)
                return batch_fail(PIC_ERR_CUDA, "batched particle kernel launch failed");
            const A_t* A = reinterpret_cast<const A_t*>(ln.args[ph].data());
            for (size_t j = 0; j < ln.idx.size(); ++j) {
                st = post_particles_t<T, G>(B->box[ln.idx[j]], A->box[j].P0, A->box[j].SP);
                if (st != PIC_OK) return st;
            }
            multi_fields_t<T, G>(ln.ft, s);
            if (cudaGetLastError() != cudaSuccess) return batch_fail(PIC_ERR_CUDA, "batched step failed");
            for (int i : ln.idx) finish_step(B->box[i]);
        }
        B->phase ^= 1;
        return PIC_OK;
    }
    {
        st = batch_fork(B);
        for (size_t i = 0; i < B->box.size() && st == PIC_OK; ++i) {
            if (regroup) st = regroup_t<T, G>(B->box[i]);
            if (st == PIC_OK) st = pre_particle(B->box[i]);
        }
        if (st == PIC_OK) st = batch_join(B);
        if (st != PIC_OK) return st;
    }
    // one launch per group of boxes, the groups side by side
    const size_t ng = B->args[ph].size();
    if (cudaMemsetAsync(B->counters, 0, sizeof(int) * ng, B->stream) != cudaSuccess)
        return batch_fail(PIC_ERR_CUDA, "work counter reset failed");
    if (ng > 1 && (st = batch_fork(B)) != PIC_OK) return st;
    for (size_t gi = 0; gi < ng; ++gi) {
        const int grid = std::max(1, std::min(B->nwork[ph][gi], B->max_grid));
        void* a[] = {B->args[ph][gi].data()};
        cudaStream_t s = ng > 1 ? B->side[gi % B->side.size()] : B->stream;
        if (cudaLaunchKernel(B->kern, dim3(grid), dim3(B->nt), a, B->smem, s) != cudaSuccess)
            return batch_fail(PIC_ERR_CUDA, "batched particle kernel launch failed");
    }
    if (ng > 1 && (st = batch_join(B)) != PIC_OK) return st;
    st = batch_fork(B);
    for (size_t i = 0; i < B->box.size() && st == PIC_OK; ++i) {
        const A_t* A = reinterpret_cast<const A_t*>(B->args[ph][i / A_t::MAXB].data());
        const BoxDesc<T>& D = A->box[i % A_t::MAXB];
        st = post_particle_t<T, G>(B->box[i], D.P0, D.SP);
    }
    if (st == PIC_OK) st = batch_join(B);
    if (st != PIC_OK) return st;
    B->phase ^= 1;
    return PIC_OK;
}

#define BDISPATCH(B, FN, ...) TG_DISPATCH((B)->fp64, (B)->tg, FN, __VA_ARGS__)

void batch_drop_graphs(pic_batch* B) {
    for (int p = 0; p < 2; ++p) {
        if (B->gexec[p]) cudaGraphExecDestroy(B->gexec[p]);
        B->gexec[p] = nullptr;
        B->graph_ok[p] = false;
    }
}

// Steps per captured batch graph: a regroup and the steps up to the next
// one, or a pair of steps.
// Lanes of an unsheared batch (more where one launch cannot hold a lane's
// boxes, fewer for fewer boxes).
constexpr int BATCH_LANES = 2;

int batch_cycle(const pic_batch* B) { return B->regroup_every > 0 ? B->regroup_every : 2; }

// Capture one cycle of steps from the current phase (with the regroup due,
// when regroups are on) into one graph (the boxes' state is put back:
// capturing runs nothing).
pic_status batch_capture(pic_batch* B) {
    const int ph0 = B->phase;
    const int r0 = B->since_regroup;
    std::vector<int> buf0;
    std::vector<long long> step0, l0;
    for (pic_handle* h : B->box) {
        buf0.push_back(h->buf);
        step0.push_back(h->step);
        l0.push_back(h->prof.launches);
    }
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        B->graphs_on = false;
        return PIC_OK;
    }
    pic_status st = B->multi ? batch_fork(B) : PIC_OK;
    for (int k = 0; k < batch_cycle(B) && st == PIC_OK; ++k) st = BDISPATCH(B, batch_step_t, B);
    if (st == PIC_OK && B->multi) st = batch_join(B);
    cudaError_t e = cudaStreamEndCapture(B->stream, &graph);
    B->phase = ph0;
    B->since_regroup = r0;
    for (size_t i = 0; i < B->box.size(); ++i) {
        B->box[i]->buf = buf0[i];
        B->box[i]->step = step0[i];
        B->box[i]->prof.launches = l0[i];
    }
    if (st != PIC_OK || e != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        B->graphs_on = false;
        return st;
    }
    e = cudaGraphInstantiate(&B->gexec[ph0], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        B->gexec[ph0] = nullptr;
        B->graphs_on = false;
        return PIC_OK;
    }
    B->graph_ok[ph0] = true;
    return PIC_OK;
}

void batch_release(pic_batch* B) {
    if (B->stream) cudaStreamSynchronize(B->stream);
    for (size_t i = 0; i < B->box.size(); ++i) {
        B->box[i]->stream = B->home[i];
        B->box[i]->batched = false;
    }
    batch_drop_graphs(B);
    bfree(B, B->counters);
    for (pic_batch::Lane& ln : B->lanes) bfree(B, ln.ft.dev);
    for (cudaEvent_t e : B->ev)
        if (e) cudaEventDestroy(e);
    for (cudaStream_t s : B->side)
        if (s) cudaStreamDestroy(s);
    if (B->stream) cudaStreamDestroy(B->stream);
    delete B;
}

}  // namespace

extern "C" {

pic_status pic_batch_create(pic_handle* const* boxes, int32_t n, pic_batch** out) {
    if (!out) return batch_fail(PIC_ERR_ARG, "pic_batch_create: out is NULL");
    *out = nullptr;
    if (!boxes || n < 1) return batch_fail(PIC_ERR_ARG, "pic_batch_create: no boxes");
    pic_handle* h0 = boxes[0];
    for (int i = 0; i < n; ++i) {
        pic_handle* h = boxes[i];
        if (!h) return batch_fail(PIC_ERR_ARG, "pic_batch_create: NULL box");
        if (h->batched) return batch_fail(PIC_ERR_STATE, "pic_batch_create: a box is already in a batch");
        for (int j = 0; j < i; ++j)
            if (boxes[j] == h) return batch_fail(PIC_ERR_ARG, "pic_batch_create: a box appears twice");
        if (h->cfg.device != h0->cfg.device || h->fp64 != h0->fp64 || h->geom != h0->geom ||
            h->cfg.shape_order != h0->cfg.shape_order || h->push != h0->push || h->esc != h0->esc)
            return batch_fail(PIC_ERR_ARG,
                              "pic_batch_create: boxes differ in device, precision, geometry, shape order or box type");
        bool any = false;
        for (int s = 0; s < PIC_MAX_SPECIES; ++s) any |= h->sp[s].loaded;
        if (!any) return batch_fail(PIC_ERR_STATE, "pic_batch_create: a box has no particles");
    }
    cudaSetDevice(h0->cfg.device);
    // one persistent kernel serves every member, so they share a tile shape:
    // the plain tiles of their geometry (8^3, 16^2).  The batch's many boxes
    // fill the GPU, so a small box's automatic smaller tiles (chosen for a box
    // running alone) would only add per-tile work; members on another shape
    // are re-laid out.
    {
        const int plain = tgeom_of(h0->geom, h0->geom == 0 ? 8 : 16);
        for (int i = 0; i < n; ++i)
            if (boxes[i]->tg != plain && retile(boxes[i], plain) != PIC_OK)
                return batch_fail(PIC_ERR_STATE, "pic_batch_create: a member could not take the batch's tile shape");
    }
    pic_batch* B = new pic_batch();
    B->device = h0->cfg.device;
    B->fp64 = h0->fp64;
    B->tg = h0->tg;
    B->kern = h0->ks.batch;
    const int v = batch_tile_variant(B->fp64, B->tg);
    B->nt = TILE_VARIANTS[v].nt;
    B->smem = tile_smem_bytes(B->fp64, B->tg, v);
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, B->device);
    if (cudaFuncSetAttribute(B->kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B->smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, B->kern, B->nt, B->smem) != cudaSuccess || per_sm < 1) {
        delete B;
        return batch_fail(PIC_ERR_CUDA, "pic_batch_create: the batched kernel cannot be launched");
    }
    B->max_grid = sms * per_sm;
    B->regroup_every = default_regroup_interval(B->fp64, B->tg);
    // every box's queued work ends before the batch takes over
    for (int i = 0; i < n; ++i) cudaStreamSynchronize(boxes[i]->stream);
    // unsheared kinds run in lanes, when the batched grid launches' z extents
    // (summed over a lane's boxes) stay within the grid limit
    {
        const int kind = h0->cfg.box;
        B->multi = kind != PIC_BOX_SHEAR && kind != PIC_BOX_SHEAR_EXPAND;
        long long zs[4] = {0, 0, 0, 0};
        for (int i = 0; i < n; ++i) {
            const Grid& g = boxes[i]->g;
            zs[0] += g.nz;
            zs[1] += 3ll * (g.px - g.nx);
            zs[2] += 3ll * (g.py - g.ny);
            zs[3] += 3ll * (g.pz - g.nz);
        }
        for (long long z : zs)
            if (z >= 65536) B->multi = false;
        if (const char* e = getenv("PIC_BATCH_NO_LANES")) B->multi = B->multi && atoi(e) == 0;
    }
    const int maxb = B->fp64 ? BatchArgs<double>::MAXB : BatchArgs<float>::MAXB;
    int nlanes = BATCH_LANES;
    if (const char* e = getenv("PIC_BATCH_LANES")) nlanes = std::max(1, atoi(e));
    nlanes = std::min(n, std::max(nlanes, (n + maxb - 1) / maxb));
    int K = B->multi ? nlanes : std::min(n, 16);  // side streams: the lanes, or parallel branches for the boxes' own kernels
    if (!B->multi)
        if (const char* e = getenv("PIC_BATCH_STREAMS")) K = std::max(1, std::min(n, atoi(e)));
    bool ok = cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) == cudaSuccess;
    B->side.assign(K, nullptr);
    B->ev.assign(K + 1, nullptr);
    for (int k = 0; k < K && ok; ++k) ok = cudaStreamCreateWithFlags(&B->side[k], cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; k <= K && ok; ++k) ok = cudaEventCreateWithFlags(&B->ev[k], cudaEventDisableTiming) == cudaSuccess;
    // heaviest tiles first: boxes in decreasing particles per tile
    std::vector<int> ord(n);
    for (int i = 0; i < n; ++i) ord[i] = i;
    auto per_tile = [&](int i) {
        long long np = 0;
        for (int s = 0; s < PIC_MAX_SPECIES; ++s)
            if (boxes[i]->sp[s].loaded) np += boxes[i]->sp[s].n;
        return (double)np / boxes[i]->tl.ntiles;
    };
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return per_tile(a) > per_tile(b); });
    for (int i : ord) {
        B->box.push_back(boxes[i]);
        B->home.push_back(boxes[i]->stream);
    }
    if (!ok) {
        batch_release(B);
        return batch_fail(PIC_ERR_CUDA, "pic_batch_create: stream or event creation failed");
    }
    if (B->multi) {
        // lanes balanced by particle count (heaviest box first to the lightest
        // lane with room); each lane keeps the heaviest-tiles-first order
        std::vector<long long> np(n, 0), load(K, 0);
        for (int i = 0; i < n; ++i)
            for (int s = 0; s < PIC_MAX_SPECIES; ++s)
                if (B->box[i]->sp[s].loaded) np[i] += B->box[i]->sp[s].n;
        std::vector<int> by(n);
        for (int i = 0; i < n; ++i) by[i] = i;
        std::stable_sort(by.begin(), by.end(), [&](int a, int b) { return np[a] > np[b]; });
        std::vector<int> lane_of(n, 0);
        B->lanes.assign(K, pic_batch::Lane());
        std::vector<int> cnt(K, 0);
        for (int i : by) {
            int best = -1;
            for (int l = 0; l < K; ++l)
                if (cnt[l] < maxb && (best < 0 || load[l] < load[best])) best = l;
            lane_of[i] = best;
            load[best] += np[i];
            cnt[best] += 1;
        }
        for (int i = 0; i < n; ++i) B->lanes[lane_of[i]].idx.push_back(i);
        for (int i = 0; i < n; ++i) {
            B->box[i]->stream = B->side[lane_of[i]];
            B->box[i]->batched = true;
        }
    } else {
        for (int i = 0; i < n; ++i) {
            B->box[i]->stream = B->side[i % K];
            B->box[i]->batched = true;
        }
    }
    pic_status st = BDISPATCH(B, batch_build_t, B);
    if (st != PIC_OK) {
        batch_release(B);
        return st;
    }
    if (const char* e = getenv("PIC_NO_GRAPHS")) B->graphs_on = atoi(e) == 0;
    *out = B;
    return PIC_OK;
}

// The stream a batch's work is ordered on (for the server's completion events).
cudaStream_t pic_internal_batch_stream(pic_batch* B) { return B ? B->stream : nullptr; }

// Graph capture of a batch's step cycles on (1) or off (0): short-lived
// batches (the server's cohorts) may not step long enough to repay a capture.
void pic_internal_batch_graphs(pic_batch* B, int on) {
    if (!B) return;
    if (!on) batch_drop_graphs(B);
    B->graphs_on = on != 0;
}

pic_status pic_batch_step(pic_batch* B, int32_t nsteps) {
    if (!B) return batch_fail(PIC_ERR_ARG, "pic_batch_step: batch is NULL");
    if (nsteps < 0) return batch_fail(PIC_ERR_ARG, "pic_batch_step: nsteps must be >= 0");
    cudaSetDevice(B->device);
    while (nsteps > 0) {
        const int ncyc = batch_cycle(B);
        const bool due = B->regroup_every == 0 || B->since_regroup >= B->regroup_every;
        if (B->graphs_on && nsteps >= ncyc && due) {
            const int ph = B->phase;
            if (!B->graph_ok[ph]) {
                pic_status st = batch_capture(B);
                if (st != PIC_OK) return st;
            }
            if (B->graph_ok[ph]) {
                if (cudaGraphLaunch(B->gexec[ph], B->stream) != cudaSuccess)
                    return batch_fail(PIC_ERR_CUDA, "pic_batch_step: graph launch failed");
                // one buffer flip per step, and one for the regroup
                const int flips = ncyc + (B->regroup_every > 0 ? 1 : 0);
                for (pic_handle* h : B->box) {
                    h->step += ncyc;
                    h->buf ^= flips & 1;
                }
                B->phase ^= flips & 1;
                if (B->regroup_every > 0) B->since_regroup = ncyc;
                nsteps -= ncyc;
                continue;
            }
        }
        pic_status st = B->multi ? batch_fork(B) : PIC_OK;
        if (st == PIC_OK) st = BDISPATCH(B, batch_step_t, B);
        if (st == PIC_OK && B->multi) st = batch_join(B);
        if (st != PIC_OK) return st;
        nsteps -= 1;
    }
    return PIC_OK;
}

pic_status pic_batch_set_regroup_interval(pic_batch* B, int32_t every) {
    if (!B) return batch_fail(PIC_ERR_ARG, "pic_batch_set_regroup_interval: batch is NULL");
    if (every < 0) return batch_fail(PIC_ERR_ARG, "pic_batch_set_regroup_interval: interval must be >= 0");
    if (every == B->regroup_every) return PIC_OK;
    cudaSetDevice(B->device);
    if (cudaStreamSynchronize(B->stream) != cudaSuccess) return batch_fail(PIC_ERR_CUDA, "pic_batch_set_regroup_interval: sync failed");
    batch_drop_graphs(B);
    B->regroup_every = every;
    return PIC_OK;
}

pic_status pic_batch_synchronize(pic_batch* B) {
    if (!B) return batch_fail(PIC_ERR_ARG, "pic_batch_synchronize: batch is NULL");
    cudaSetDevice(B->device);
    if (cudaStreamSynchronize(B->stream) != cudaSuccess) return batch_fail(PIC_ERR_CUDA, "pic_batch_synchronize failed");
    return PIC_OK;
}

pic_status pic_batch_destroy(pic_batch* B) {
    if (!B) return PIC_OK;
    cudaSetDevice(B->device);
    batch_release(B);
    return PIC_OK;
}

int32_t pic_batch_max_boxes_per_launch(int32_t precision) {
    return precision == PIC_FP64 ? BatchArgs<double>::MAXB : BatchArgs<float>::MAXB;
}

}  // extern "C"
