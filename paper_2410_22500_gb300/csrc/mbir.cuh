// Shared pieces of the MBIR update (Eq. recon, SQS with the qGGMRF prior).
#pragma once

#include "proj.cuh"

namespace fhr {

constexpr int kMbirMaxK = 8;

struct MbirChan {
    float inv_sv2[kMbirMaxK];   // 1 / sigma_v^2
    float c0[kMbirMaxK];        // 1 / (T^(2-p) sigma_x^2)
    float inv_tsx[kMbirMaxK];   // 1 / (T sigma_x)
    float sv[kMbirMaxK], sx[kMbirMaxK];
};

// Explicit per-channel sigmas (kernel argument).
struct SigmaArgs {
    float sv[kMbirMaxK], sx[kMbirMaxK];
};

// Blocks of the sigma reduction; fixed, so every caller sums in the same order.
constexpr int kSigBlocks = 128;

struct MbirPrior {
    float e;        // 2 - p
    float c1;       // (2 - p) / p
    float beta;
    float b_edge, b_diag, b_slice;
    float T, p;
};

// PTX approximations (PTX ISA: lg2.approx and ex2.approx within about 2^-22
// relative, rcp.approx within 1 ulp); the influence weight below only scales
// the prior's surrogate curvature, so these errors stay near 1e-6 of it.
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// rho'(d)/d of the qGGMRF potential with q = 2:
//   c0 / (1 + u) * (1 + c1 / (1 + u)),  u = (|d| / (T sx))^(2 - p)
// (a = 0 gives u = 0 through ex2(-inf) = 0; e = 0 gives u = 1)
__device__ __forceinline__ float qggmrf_infl(float d, float c0, float inv_tsx, float e, float c1) {
    const float a = fabsf(d) * inv_tsx;
    const float u = e == 0.f ? 1.f : ex2_approx(e * lg2_approx(a));
    const float r = rcp_approx(1.f + u);
    return c0 * r * (1.f + c1 * r);
}

// SQS update of one (pixel, VW values from w0) given bp, the back-projected
// residual: x+ = max(0, z - g/d) with the qGGMRF prior over the 8 in-plane
// and (Nr > 1) 2 inter-slice neighbours; with znext, also the momentum point.
// COH: e, z and xprev were written earlier in the same launch.
template <int VW, bool COH>
__device__ __forceinline__ void mbir_update_group(const typename VecF<VW>::T &bp, const float *__restrict__ z,
                                                  const float *__restrict__ xprev, float *__restrict__ xnew,
                                                  float *__restrict__ znext, const float *__restrict__ dA,
                                                  const MbirChan *__restrict__ chp, const MbirPrior &pr, float mom_a,
                                                  int N, int Nc, int Nv, int Nr, int K, int Wl, int pix, int w0) {
    using VF = VecF<VW>;
    const int iy = pix / N, ix = pix % N;
    const size_t base = (size_t)pix * Wl + w0;
    const typename VF::T zc = ldv<VW, COH>(z + base);
    const float da = dA[pix];
    float g[VW], d[VW];
#pragma unroll
    for (int q = 0; q < VW; ++q) {
        const int j = (w0 + q) % K;
        g[q] = -VF::get(bp, q) * chp->inv_sv2[j];
        d[q] = da * chp->inv_sv2[j];
    }
    if (pr.beta != 0.f) {
        const int dy8[8] = {-1, 1, 0, 0, -1, -1, 1, 1};
        const int dx8[8] = {0, 0, -1, 1, -1, 1, -1, 1};
        // neighbours outside the image read the pixel itself with weight 0 (adds exact
        // zeros), so no load sits behind a branch
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            const int yy = iy + dy8[n], xx = ix + dx8[n];
            const bool in = yy >= 0 && yy < N && xx >= 0 && xx < N;
            const float b = in ? pr.beta * (n < 4 ? pr.b_edge : pr.b_diag) : 0.f;
            const typename VF::T zn = ldv<VW, COH>(z + ((size_t)(in ? yy : iy) * N + (in ? xx : ix)) * Wl + w0);
#pragma unroll
            for (int q = 0; q < VW; ++q) {
                const int j = (w0 + q) % K;
                const float dl = VF::get(zc, q) - VF::get(zn, q);
                const float wt = qggmrf_infl(dl, chp->c0[j], chp->inv_tsx[j], pr.e, pr.c1);
                g[q] = fmaf(b * dl, wt, g[q]);
                d[q] = fmaf(2.f * b, wt, d[q]);
            }
        }
        if (Nr > 1) {
            // slices r - 1 and r + 1 of the same channel (w -+ K); missing ones read the
            // value itself with weight 0
            float zlo[VW], zhi[VW];
#pragma unroll
            for (int q = 0; q < VW; ++q) {
                const int w = w0 + q, r = w / K;
                zlo[q] = ldv<1, COH>(z + (size_t)pix * Wl + (r > 0 ? w - K : w));
                zhi[q] = ldv<1, COH>(z + (size_t)pix * Wl + (r < Nr - 1 ? w + K : w));
            }
#pragma unroll
            for (int q = 0; q < VW; ++q) {
                const int w = w0 + q;
                const int j = w % K, r = w / K;
                const float b = pr.beta * pr.b_slice;
                const float zq = VF::get(zc, q);
                {
                    const float bl = r > 0 ? b : 0.f;
                    const float dl = zq - zlo[q];
                    const float wt = qggmrf_infl(dl, chp->c0[j], chp->inv_tsx[j], pr.e, pr.c1);
                    g[q] = fmaf(bl * dl, wt, g[q]);
                    d[q] = fmaf(2.f * bl, wt, d[q]);
                }
                {
                    const float bh = r < Nr - 1 ? b : 0.f;
                    const float dl = zq - zhi[q];
                    const float wt = qggmrf_infl(dl, chp->c0[j], chp->inv_tsx[j], pr.e, pr.c1);
                    g[q] = fmaf(bh * dl, wt, g[q]);
                    d[q] = fmaf(2.f * bh, wt, d[q]);
                }
            }
        }
    }
    typename VF::T xn;
#pragma unroll
    for (int q = 0; q < VW; ++q) {
        const float zq = VF::get(zc, q);
        VF::set(xn, q, d[q] > 0.f ? fmaxf(0.f, zq - __fdiv_rn(g[q], d[q])) : zq);
    }
    VF::st(xnew + base, xn);
    if (znext) {
        const typename VF::T xp = ldv<VW, COH>(xprev + base);
        typename VF::T zz;
#pragma unroll
        for (int q = 0; q < VW; ++q) {
            const float a = VF::get(xn, q);
            VF::set(zz, q, fmaxf(0.f, fmaf(mom_a, a - VF::get(xp, q), a)));
        }
        VF::st(znext + base, zz);
    }
}


// SQS update of one pixel for the G groups of VW values at w0 + g gs: one
// backward gather (shared table reads), then the update of each group.
template <int VW, int G, bool COH = false>
__device__ __forceinline__ void mbir_update_at(const float *__restrict__ e, const float *__restrict__ z,
                                               const float *__restrict__ xprev, float *__restrict__ xnew,
                                               float *__restrict__ znext, const ProjTables &t,
                                               const float *__restrict__ dA, const MbirChan *__restrict__ chp,
                                               const MbirPrior &pr, float mom_a, int N, int Nc, int Nv, int Nr, int K,
                                               int Wl, int pix, int w0, int gs) {
    typename VecF<VW>::T bp[G];
    backproject_at<VW, G, COH>(e, t, N, Nc, Nv, Wl, pix, w0, gs, bp);
#pragma unroll
    for (int g = 0; g < G; ++g)
        mbir_update_group<VW, COH>(bp[g], z, xprev, xnew, znext, dA, chp, pr, mom_a, N, Nc, Nv, Nr, K, Wl, pix,
                                   w0 + g * gs);
}

}  // namespace fhr
