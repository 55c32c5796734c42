// Parallel-beam strip-area projector (A of Eq. porj_matd_rel / Eq. recon).
//
// A_{(v,c),i} = area(unit pixel i intersect the unit-width strip of bin c at
// view v).  It is the integral over the bin of the pixel's trapezoidal
// footprint, so it has a closed form (footprint_cdf in proj.cu).  The weights
// are evaluated once per call (pixel-to-bin offset in FP64, the footprint
// integral in FP32) into two tables:
//   forward  [Nv][N][Nc] lines: along the image axis most parallel to the
//            rays, 4 candidate pixels per line (a strip crosses at most 4),
//   backward [Nv][N*N]: 3 candidate bins per pixel (a footprint spans <= 3),
// both from the one compiled strip_area routine on equal inputs, so A^T is the
// exact transpose of A.  The two gathers apply each weight to a vector of Wl values per
// pixel / ray (all slices and subspace channels at once), so every access is
// a contiguous, vectorised read of Wl floats.
#pragma once

#include "common.cuh"

namespace fhr {

struct ProjTables {
    float4 *fw;        // [Nv][N][Nc] weights of candidates s0..s0+3 (per view, line, ray)
    int *fws;          // [Nv][N][Nc] s0
    uint8_t *rowmaj;   // [Nv] 1: lines are image rows (|cos| >= |sin|)
    float4 *bk;        // [Nv][N*N] {w0, w1, w2, c0}
    int *fspan;        // [Nv][ray blocks of 32][N] first pixel of the staged run (proj_tma.cuh)
    int *bspan;        // [Nv][8 x 8 tiles] first bin of the staged slab
};

// a += w * x on two lanes at once (the packed FP32 FMA of sm_100 and later; each
// lane is rounded as a separate fmaf, so the bits are the same)
__device__ __forceinline__ void fma2(float &a0, float &a1, float w, float x0, float x1) {
    const float2 r = __ffma2_rn(make_float2(w, w), make_float2(x0, x1), make_float2(a0, a1));
    a0 = r.x;
    a1 = r.y;
}

template <int VW>
struct VecF;
template <>
struct VecF<4> {
    using T = float4;
    __device__ __forceinline__ static float4 ld(const float *p) { return *reinterpret_cast<const float4 *>(p); }
    __device__ __forceinline__ static float4 ldca(const float *p) { return __ldca(reinterpret_cast<const float4 *>(p)); }
    __device__ __forceinline__ static void st(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
    __device__ __forceinline__ static void fma(float4 &a, float w, float4 x) {
        fma2(a.x, a.y, w, x.x, x.y);
        fma2(a.z, a.w, w, x.z, x.w);
    }
    __device__ __forceinline__ static float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ __forceinline__ static float get(const float4 &v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }
    __device__ __forceinline__ static void set(float4 &v, int e, float f) {
        if (e == 0) v.x = f; else if (e == 1) v.y = f; else if (e == 2) v.z = f; else v.w = f;
    }
};
template <>
struct VecF<2> {
    using T = float2;
    __device__ __forceinline__ static float2 ld(const float *p) { return *reinterpret_cast<const float2 *>(p); }
    __device__ __forceinline__ static float2 ldca(const float *p) { return __ldca(reinterpret_cast<const float2 *>(p)); }
    __device__ __forceinline__ static void st(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
    __device__ __forceinline__ static void fma(float2 &a, float w, float2 x) {
        a.x = fmaf(w, x.x, a.x); a.y = fmaf(w, x.y, a.y);
    }
    __device__ __forceinline__ static float2 zero() { return make_float2(0.f, 0.f); }
    __device__ __forceinline__ static float get(const float2 &v, int e) { return e == 0 ? v.x : v.y; }
    __device__ __forceinline__ static void set(float2 &v, int e, float f) {
        if (e == 0) v.x = f; else v.y = f;
    }
};
template <>
struct VecF<1> {
    using T = float;
    __device__ __forceinline__ static float ld(const float *p) { return *p; }
    __device__ __forceinline__ static float ldca(const float *p) { return __ldca(p); }
    __device__ __forceinline__ static void st(float *p, float v) { *p = v; }
    __device__ __forceinline__ static void fma(float &a, float w, float x) { a = fmaf(w, x, a); }
    __device__ __forceinline__ static float zero() { return 0.f; }
    __device__ __forceinline__ static float get(const float &v, int) { return v; }
    __device__ __forceinline__ static void set(float &v, int, float f) { v = f; }
};

// Load of a vector.  COH: the same launch wrote it before a grid-wide
// barrier (release/acquire fences), so it must be an ordinary coherent load
// (ld.global.ca), never the read-only non-coherent path the compiler may pick
// for const restrict pointers.
template <int VW, bool COH>
__device__ __forceinline__ typename VecF<VW>::T ldv(const float *p) {
    if constexpr (COH) return VecF<VW>::ldca(p);
    else return VecF<VW>::ld(p);
}

// sum over lines and candidates of A * x[pixel][w] for one ray (item = (v, c)),
// the G groups of VW values at w0 + g gs (one table read serves all groups).
template <int VW, int G, bool COH = false>
__device__ __forceinline__ void forward_at(const float *__restrict__ x, const ProjTables &t, int N, int Nc, int Wl,
                                           int item, int w0, int gs, typename VecF<VW>::T (&acc)[G]) {
    using VF = VecF<VW>;
    const int v = item / Nc, c = item - v * Nc;
    const bool rows = t.rowmaj[v] != 0;
    const float4 *fw = t.fw + (size_t)v * N * Nc + c;
    const int *fs = t.fws + (size_t)v * N * Nc + c;
    const int lstride = rows ? N : 1;     // pixel index = l * lstride + q * qstride
    const int qstride = rows ? 1 : N;
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = VF::zero();
    const float *xc = x + w0;
    for (int l = 0; l < N; ++l) {
        const float4 w = __ldg(fw + (size_t)l * Nc);
        const int s0 = __ldg(fs + (size_t)l * Nc);
        const float *xp = xc + (size_t)(l * lstride + s0 * qstride) * Wl;
        const size_t qs = (size_t)qstride * Wl;
        if (w.x != 0.f) {
#pragma unroll
            for (int g = 0; g < G; ++g) VF::fma(acc[g], w.x, ldv<VW, COH>(xp + g * gs));
        }
        if (w.y != 0.f) {
#pragma unroll
            for (int g = 0; g < G; ++g) VF::fma(acc[g], w.y, ldv<VW, COH>(xp + qs + g * gs));
        }
        if (w.z != 0.f) {
#pragma unroll
            for (int g = 0; g < G; ++g) VF::fma(acc[g], w.z, ldv<VW, COH>(xp + 2 * qs + g * gs));
        }
        if (w.w != 0.f) {
#pragma unroll
            for (int g = 0; g < G; ++g) VF::fma(acc[g], w.w, ldv<VW, COH>(xp + 3 * qs + g * gs));
        }
    }
}

// Gathers over a vector of Wl values per pixel / ray run in channel chunks of
// Wc values (Wc | Wl, VW | Wc), chunk-major over the grid: the blocks resident
// at one time touch one chunk of the image / sinogram, which stays in L2 when
// the whole does not.  Thread = (item, G groups of VW values); the CH = Wc /
// (VW G) threads of an item take VW values each per group, so that group g of
// the item is the contiguous run w0 + g gs (gs = CH VW) across those threads
// and every load instruction of a warp reads whole sectors once.
struct GatherIdx {
    int item, w0, gs;
    bool ok;
};

template <int VW, int G>
__device__ __forceinline__ GatherIdx gather_idx(int items, int Wl, int Wc) {
    const int CH = Wc / (VW * G);
    const int ipb = blockDim.x / CH;
    const int bpc = (items + ipb - 1) / ipb;   // blocks per chunk
    const int chunk = blockIdx.x / bpc;
    GatherIdx r;
    r.item = (blockIdx.x - chunk * bpc) * ipb + threadIdx.x / CH;
    r.w0 = chunk * Wc + (threadIdx.x % CH) * VW;
    r.gs = CH * VW;
    r.ok = threadIdx.x < ipb * CH && r.item < items && r.w0 < Wl;
    return r;
}

// y[v][c][w] = sum over lines and candidates of A * x[pixel][w].
// With V non-null the output is the residual V - A x.
template <int VW, int G>
__global__ void __launch_bounds__(1024) proj_fwd_kernel(const float *__restrict__ x, float *__restrict__ y,
                                                        const float *__restrict__ V, ProjTables t, int N, int Nc,
                                                        int Nv, int Wl, int Wc) {
    using VF = VecF<VW>;
    const GatherIdx gi = gather_idx<VW, G>(Nv * Nc, Wl, Wc);
    if (!gi.ok) return;
    const int item = gi.item;
    typename VF::T acc[G];
    forward_at<VW, G>(x, t, N, Nc, Wl, item, gi.w0, gi.gs, acc);
    float *yo = y + (size_t)item * Wl + gi.w0;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        if (V) {
            typename VF::T vv = VF::ld(V + (size_t)item * Wl + gi.w0 + g * gi.gs);
#pragma unroll
            for (int e = 0; e < VW; ++e) VF::set(acc[g], e, VF::get(vv, e) - VF::get(acc[g], e));
        }
        VF::st(yo + g * gi.gs, acc[g]);
    }
}

// x[pixel][w] = sum over views and candidate bins of A * y[v][c][w], for the
// G groups of VW values at w0 + g gs.
template <int VW, int G, bool COH = false>
__device__ __forceinline__ void backproject_at(const float *__restrict__ y, const ProjTables &t, int N, int Nc,
                                               int Nv, int Wl, int pix, int w0, int gs,
                                               typename VecF<VW>::T (&acc)[G]) {
    using VF = VecF<VW>;
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = VF::zero();
    const float *yc = y + w0;
    const size_t NN = (size_t)N * N;
    for (int v = 0; v < Nv; ++v) {
        const float4 w = __ldg(t.bk + v * NN + pix);
        const float *yr = yc + ((size_t)v * Nc + (int)w.w) * Wl;
        if (w.x != 0.f) {
#pragma unroll
            for (int g = 0; g < G; ++g) VF::fma(acc[g], w.x, ldv<VW, COH>(yr + g * gs));
        }
        if (w.y != 0.f) {
#pragma unroll
            for (int g = 0; g < G; ++g) VF::fma(acc[g], w.y, ldv<VW, COH>(yr + Wl + g * gs));
        }
        if (w.z != 0.f) {
#pragma unroll
            for (int g = 0; g < G; ++g) VF::fma(acc[g], w.z, ldv<VW, COH>(yr + 2 * (size_t)Wl + g * gs));
        }
    }
}

template <int VW, int G>
__global__ void __launch_bounds__(1024) proj_bwd_kernel(const float *__restrict__ y, float *__restrict__ x,
                                                        ProjTables t, int N, int Nc, int Nv, int Wl, int Wc) {
    using VF = VecF<VW>;
    const GatherIdx gi = gather_idx<VW, G>(N * N, Wl, Wc);
    if (!gi.ok) return;
    typename VF::T acc[G];
    backproject_at<VW, G>(y, t, N, Nc, Nv, Wl, gi.item, gi.w0, gi.gs, acc);
#pragma unroll
    for (int g = 0; g < G; ++g) VF::st(x + (size_t)gi.item * Wl + gi.w0 + g * gi.gs, acc[g]);
}

// Launch shape for the gathers: chunks of Wc values (the whole vector unless
// the larger of the image / sinogram slabs exceeds kGatherSlab bytes), CH =
// Wc / (VW G) threads per item, items per block so that a block holds about
// `target` threads, and the grid = chunks x blocks per chunk.
// 64 MB measured best on the 256^3 volume's gathers (N = 256, Wl = 1536: chunks of
// 192 values): forward + update 12.1 ms against 13.0 at 32 MB, 12.3 at 128 MB and 15.5
// unchunked
constexpr size_t kGatherSlab = (size_t)64 << 20;
// groups per thread: the forward gather gains up to 4 (0.341 -> 0.287 ms on the
// 128^2 x 64 slice / K = 5 shape), the fused backward + update is best at 2
constexpr int kGatherMaxGFwd = 4, kGatherMaxGBwd = 2;
// the fused backward + update is held to 48 registers (five 256-thread blocks per SM:
// 0.393 -> 0.355 ms on that shape), so its blocks have at most 256 threads
constexpr int kUpdateThreads = 256, kUpdateMinBlocks = 5;

struct GatherShape {
    int vw, g, wc, ch, ipb, threads;   // g: groups of vw values per thread
    unsigned blocks(int items, int Wl) const {
        const int bpc = (items + ipb - 1) / ipb;
        return (unsigned)(bpc * (Wl / wc));
    }
};

static inline GatherShape gather_shape(int Wl, size_t slab_values, int max_g, int max_threads = 1024,
                                       int target = 256) {
    GatherShape g;
    g.vw = (Wl % 4 == 0) ? 4 : 1;
    g.wc = Wl;
    // halve the chunk while the slab of one chunk exceeds the L2 budget (keeping VW | Wc | Wl)
    while (slab_values * (size_t)g.wc * sizeof(float) > kGatherSlab && g.wc % (2 * g.vw) == 0 && g.wc / 2 >= 32)
        g.wc /= 2;
    // up to max_g groups per thread share each table read where the chunk allows it
    g.g = 1;
    if (g.vw == 4) {
        if (max_g >= 4 && g.wc % 16 == 0) g.g = 4;
        else if (max_g >= 2 && g.wc % 8 == 0) g.g = 2;
    }
    // an item's threads: halve the chunk down to `target` where it divides, and never
    // more than the kernel's block limit (else the largest chunk of whole vectors that
    // fits, one group)
    while (g.wc / (g.vw * g.g) > target && g.wc % (2 * g.vw * g.g) == 0) g.wc /= 2;
    if (g.wc / (g.vw * g.g) > max_threads) {
        g.g = 1;
        for (int c = std::min(Wl, max_threads * g.vw); c >= g.vw; --c)
            if (Wl % c == 0 && c % g.vw == 0) {
                g.wc = c;
                break;
            }
    }
    g.ch = g.wc / (g.vw * g.g);
    g.ipb = std::max(1, target / g.ch);
    g.threads = g.ipb * g.ch;
    return g;
}

// values per channel of the larger of the image and the sinogram
static inline size_t gather_slab_values(const fhr_geom *g) {
    return std::max((size_t)g->N * g->N, (size_t)g->Nv * g->Nc);
}

void proj_tables_carve(Carve &c, int N, int Nc, int Nv, ProjTables *t);
fhr_status proj_build_tables(fhr_ctx *ctx, const fhr_geom *g, const ProjTables &t);
// status: the device status word that the staged gathers report to (may be null)
fhr_status proj_forward(fhr_ctx *ctx, const fhr_geom *g, const ProjTables &t, int Wl, const float *x, float *y,
                        const float *V, int *status = nullptr);
fhr_status proj_backward(fhr_ctx *ctx, const fhr_geom *g, const ProjTables &t, int Wl, const float *y, float *x,
                         int *status = nullptr);
fhr_status check_geom(fhr_ctx *ctx, const fhr_geom *g, int Wl);

}  // namespace fhr
