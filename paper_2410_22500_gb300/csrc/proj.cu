// Projector tables, launches and the standalone projector entry points.
#include "proj_tma.cuh"

namespace fhr {

// Cumulative integral of a unit pixel's footprint seen along (cos, sin): a
// trapezoid of area 1, flat top of height 1/hi for |s| <= (hi - lo)/2, linear to
// 0 at |s| = (hi + lo)/2 (hi = max(|cos|, |sin|), lo = min).  FP32: the argument
// is a small offset (|s| < 2) computed in FP64 by the caller.
__device__ __forceinline__ float footprint_cdf(float s, float hi, float lo) {
    const float t2 = 0.5f * (hi + lo), t1 = 0.5f * (hi - lo);
    if (s <= -t2) return 0.f;
    if (s >= t2) return 1.f;
    if (s <= -t1) return (s + t2) * (s + t2) / (2.f * hi * lo);
    if (s <= t1) return lo / (2.f * hi) + (s + t1) / hi;
    return 1.f - (t2 - s) * (t2 - s) / (2.f * hi * lo);
}

// area of pixel (px, py) inside the unit strip centred at uc, direction (c, s):
// the pixel's position along the detector in FP64, the footprint integral in FP32.
// Results below 2^-22 (the rounding level of the FP32 integral) are returned as
// 0, so a pixel / bin pair that only touches stays exactly 0 in both tables,
// whichever candidate ranges they scan.  Not inlined: both tables call the one
// compiled instance, so equal inputs give equal bits.
__device__ __noinline__ float strip_area(double c, double s, double px, double py, double uc) {
    const float a = fabsf((float)c), b = fabsf((float)s);
    const float hi = fmaxf(a, b), lo = fminf(a, b);
    const float d = (float)(uc - fma(px, c, py * s));
    const float w = footprint_cdf(d + 0.5f, hi, lo) - footprint_cdf(d - 0.5f, hi, lo);
    return w < 0x1p-22f ? 0.f : w;
}

__device__ __forceinline__ void view_dir(const double *angles, int v, int Nv, double *c, double *s) {
    const double th = angles ? angles[v] : (double)v * (3.141592653589793 / (double)Nv);
    sincos(th, s, c);
}

// forward table: one thread per (v, line, c); layout [Nv][N][Nc] so that the
// rays of one view read consecutive entries for each line
__global__ void proj_table_fw(const double *angles, int N, int Nc, int Nv, ProjTables t) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)Nv * Nc * N) return;
    const int c = (int)(idx % Nc);
    const int l = (int)((idx / Nc) % N);
    const int v = (int)(idx / ((int64_t)N * Nc));
    double cs, sn;
    view_dir(angles, v, Nv, &cs, &sn);
    const double h = 0.5 * (N - 1);
    const double uc = c - 0.5 * (Nc - 1);
    const double half = 0.5 + 0.5 * (fabs(cs) + fabs(sn));
    const bool rows = fabs(cs) >= fabs(sn);
    double center, R;
    if (rows) {
        const double py = l - h;
        center = (uc - py * sn) / cs + h;
        R = half / fabs(cs);
    } else {
        const double px = l - h;
        center = (uc - px * cs) / sn + h;
        R = half / fabs(sn);
    }
    int s0 = (int)floor(center - R) + 1;
    s0 = max(0, min(s0, N - 4));
    float w[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int q = s0 + m;
        const double px = rows ? q - h : l - h;
        const double py = rows ? l - h : q - h;
        w[m] = strip_area(cs, sn, px, py, uc);
    }
    t.fw[idx] = make_float4(w[0], w[1], w[2], w[3]);
    t.fws[idx] = s0;
    if (c == 0 && l == 0) t.rowmaj[v] = rows ? 1 : 0;
}

// backward table: one thread per (v, pixel)
__global__ void proj_table_bk(const double *angles, int N, int Nc, int Nv, ProjTables t) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)Nv * N * N) return;
    const int pix = (int)(idx % ((int64_t)N * N));
    const int v = (int)(idx / ((int64_t)N * N));
    const int iy = pix / N, ix = pix % N;
    double cs, sn;
    view_dir(angles, v, Nv, &cs, &sn);
    const double h = 0.5 * (N - 1);
    const double px = ix - h, py = iy - h;
    const double u0 = px * cs + py * sn;
    const double half = 0.5 + 0.5 * (fabs(cs) + fabs(sn));
    int c0 = (int)floor(u0 + 0.5 * (Nc - 1) - half) + 1;
    c0 = max(0, min(c0, Nc - 3));
    float w[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) w[m] = strip_area(cs, sn, px, py, (c0 + m) - 0.5 * (Nc - 1));
    t.bk[idx] = make_float4(w[0], w[1], w[2], (float)c0);
}

void proj_tables_carve(Carve &c, int N, int Nc, int Nv, ProjTables *t) {
    ProjTables tt;
    tt.fw = c.take<float4>((size_t)Nv * Nc * N);
    tt.fws = c.take<int>((size_t)Nv * Nc * N);
    tt.rowmaj = c.take<uint8_t>((size_t)Nv);
    tt.bk = c.take<float4>((size_t)Nv * N * N);
    const int64_t NTX = cdiv(N, kTmaTile);
    // the run table of either forward block shape: groups x 2 sweeps x ray blocks x lines
    tt.fspan = c.take<int>((size_t)Nv * 2 * cdiv(Nc, 16) * N);
    tt.bspan = c.take<int>((size_t)Nv * NTX * NTX);
    if (t) *t = tt;
}

fhr_status check_geom(fhr_ctx *ctx, const fhr_geom *g, int Wl) {
    FHR_ARG(g, "geometry is null");
    FHR_ARG(g->N >= 4, "N must be >= 4");
    FHR_ARG(g->Nc >= 3, "Nc must be >= 3");
    FHR_ARG(g->Nv >= 1 && g->Nr >= 1, "Nv and Nr must be positive");
    FHR_ARG((int64_t)g->N * g->N < (1ll << 31) && (int64_t)g->Nv * g->Nc < (1ll << 31), "geometry too large");
    FHR_ARG(Wl >= 1 && Wl <= 4096 && (Wl % 4 == 0 || Wl <= 1024), "Wl must be 1..1024, or a multiple of 4 up to 4096");
    return FHR_OK;
}

fhr_status proj_build_tables(fhr_ctx *ctx, const fhr_geom *g, const ProjTables &t) {
    const int64_t nf = (int64_t)g->Nv * g->Nc * g->N, nb = (int64_t)g->Nv * g->N * g->N;
    proj_table_fw<<<(unsigned)cdiv(nf, 256), 256, 0, ctx->stream>>>(g->angles, g->N, g->Nc, g->Nv, t);
    FHR_LAUNCHED();
    proj_table_bk<<<(unsigned)cdiv(nb, 256), 256, 0, ctx->stream>>>(g->angles, g->N, g->Nc, g->Nv, t);
    FHR_LAUNCHED();
    const int vg = tma_fwd_vg(g), rb = vg == 4 ? 16 : kTmaRays;
    const int64_t ns = cdiv(g->Nv, vg) * 2 * cdiv(g->Nc, rb) * g->N;
    proj_span_fw<<<(unsigned)cdiv(ns, 256), 256, 0, ctx->stream>>>(t, g->N, g->Nc, g->Nv, vg, rb, t.fspan);
    FHR_LAUNCHED();
    const int64_t nt = (int64_t)g->Nv * cdiv(g->N, kTmaTile) * cdiv(g->N, kTmaTile);
    proj_span_bk<<<(unsigned)cdiv(nt, 256), 256, 0, ctx->stream>>>(t, g->N, g->Nc, g->Nv, t.bspan);
    FHR_LAUNCHED();
    return FHR_OK;
}

template <template <int, int> class Launch, typename... A>
static fhr_status gather_dispatch(const GatherShape &s, A... args) {
    if (s.vw == 4 && s.g == 4) return Launch<4, 4>::run(s, args...);
    if (s.vw == 4 && s.g == 2) return Launch<4, 2>::run(s, args...);
    if (s.vw == 4) return Launch<4, 1>::run(s, args...);
    return Launch<1, 1>::run(s, args...);
}

template <int VW, int G>
struct FwdLaunch {
    static fhr_status run(const GatherShape &s, fhr_ctx *ctx, const fhr_geom *g, const ProjTables &t, int Wl,
                          const float *x, float *y, const float *V) {
        FHR_TIMED(TM_PROJ_FWD, (proj_fwd_kernel<VW, G><<<s.blocks(g->Nv * g->Nc, Wl), s.threads, 0, ctx->stream>>>(
                                    x, y, V, t, g->N, g->Nc, g->Nv, Wl, s.wc)));
        return FHR_OK;
    }
};

template <int VW, int G>
struct BwdLaunch {
    static fhr_status run(const GatherShape &s, fhr_ctx *ctx, const fhr_geom *g, const ProjTables &t, int Wl,
                          const float *y, float *x) {
        FHR_TIMED(TM_PROJ_BWD, (proj_bwd_kernel<VW, G><<<s.blocks(g->N * g->N, Wl), s.threads, 0, ctx->stream>>>(
                                    y, x, t, g->N, g->Nc, g->Nv, Wl, s.wc)));
        return FHR_OK;
    }
};

fhr_status proj_forward(fhr_ctx *ctx, const fhr_geom *g, const ProjTables &t, int Wl, const float *x, float *y,
                        const float *V, int *status) {
    if (tma_gathers_ok(g, Wl)) return tma_forward(ctx, g, t, Wl, x, y, V, status);
    const GatherShape s = gather_shape(Wl, gather_slab_values(g), kGatherMaxGFwd);
    return gather_dispatch<FwdLaunch>(s, ctx, g, t, Wl, x, y, V);
}

fhr_status proj_backward(fhr_ctx *ctx, const fhr_geom *g, const ProjTables &t, int Wl, const float *y, float *x,
                         int *status) {
    if (tma_gathers_ok(g, Wl)) return tma_backward(ctx, g, t, Wl, y, x, nullptr, status);
    const GatherShape s = gather_shape(Wl, gather_slab_values(g), kGatherMaxGBwd);
    return gather_dispatch<BwdLaunch>(s, ctx, g, t, Wl, y, x);
}

static size_t proj_ws(const fhr_geom *g, ProjTables *t, void *base) {
    Carve c(base);
    c.take<int>(kStatusBytes / sizeof(int));
    proj_tables_carve(c, g->N, g->Nc, g->Nv, t);
    return c.size();
}

}  // namespace fhr

using namespace fhr;

extern "C" fhr_status fhr_projector_workspace_size(fhr_ctx *ctx, const fhr_geom *g, size_t *bytes) {
    if (!ctx) return FHR_ERR_ARG;
    FHR_TRY(check_geom(ctx, g, 1));
    FHR_ARG(bytes, "bytes is null");
    *bytes = proj_ws(g, nullptr, nullptr);
    return FHR_OK;
}

static fhr_status proj_common(fhr_ctx *ctx, const fhr_geom *g, int Wl, const void *in, void *out, void *ws,
                              size_t ws_bytes, ProjTables *t) {
    FHR_TRY(check_geom(ctx, g, Wl));
    FHR_ARG(in && out && ws, "null pointer argument");
    FHR_ARG(aligned(ws, 256), "workspace must be 256-byte aligned");
    FHR_ARG(Wl % 4 != 0 || (aligned(in, 16) && aligned(out, 16)), "x and y must be 16-byte aligned when Wl % 4 == 0");
    const size_t need = proj_ws(g, t, ws);
    FHR_ARG(ws_bytes >= need, "workspace too small: %zu < %zu bytes", ws_bytes, need);
    FHR_CUDA(cudaSetDevice(ctx->device));
    return proj_build_tables(ctx, g, *t);
}

extern "C" fhr_status fhr_project(fhr_ctx *ctx, const fhr_geom *g, int Wl, const float *x, float *y, void *ws,
                                  size_t ws_bytes) {
    if (!ctx) return FHR_ERR_ARG;
    ProjTables t;
    FHR_TRY(proj_common(ctx, g, Wl, x, y, ws, ws_bytes, &t));
    return proj_forward(ctx, g, t, Wl, x, y, nullptr, (int *)ws);
}

extern "C" fhr_status fhr_backproject(fhr_ctx *ctx, const fhr_geom *g, int Wl, const float *y, float *x, void *ws,
                                      size_t ws_bytes) {
    if (!ctx) return FHR_ERR_ARG;
    ProjTables t;
    FHR_TRY(proj_common(ctx, g, Wl, y, x, ws, ws_bytes, &t));
    return proj_backward(ctx, g, t, Wl, y, x, (int *)ws);
}
