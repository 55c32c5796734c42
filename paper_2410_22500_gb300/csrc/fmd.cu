// Semi-supervised fast material decomposition (Algorithm 2 after the
// reconstruction), from the subspace reconstruction x^s [Nx][Ns], user
// region labels and the subspace spectra D^s [Nk][Ns]:
//   T[i][j] = mean of x^s_{n,j} over region i          (Eq. trans_mat)
//   x^m_n   = argmin_{x >= 0} || x^s_n - T^T x ||^2     (Eq. mat_recon_nmf)
//   D^m     = D^s T^T                                   (Eq. sub_mat_rel_basis)
// Region sums: one block per voxel range, one thread per (region, channel),
// voxels in order, then a fixed-order sum of the block partials in FP64.  The
// per-voxel problems: one thread each, Lawson-Hanson active sets on the normal
// equations (T T^T) x = T x^s_n in FP64 (at most 8 materials), with the inverse of
// every principal block of T T^T formed once per call.
#include "common.cuh"

namespace fhr {

constexpr int kFmdMaxM = 8;
constexpr int kFmdMaxS = 16;
constexpr int kFmdBlocks = 2048;
constexpr int kFmdInvSmem = 2304;   // subset inverses kept in shared memory (FP64 + FP32: 27 KB, Nm <= 6)

__global__ void fmd_region_partials(const float *__restrict__ xs, const uint8_t *__restrict__ lab, int64_t Nx, int Ns,
                                    int Nm, double *part, long long *cnt) {
    // a lane per (region i, channel j) pair p, G warps covering the P pairs, and the
    // block's voxel range split into R = 4 / G sub-ranges walked in voxel order; the
    // sub-range sums are combined in order (deterministic)
    __shared__ double ssum[4][kFmdMaxM * kFmdMaxS];
    __shared__ long long scnt[4][kFmdMaxM * kFmdMaxS];
    const int P = Nm * Ns, G = (P + 31) / 32, R = 4 / G;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = w / G, p = (w % G) * 32 + lane;
    const int i = p / Ns, j = p % Ns;
    const int64_t per = (Nx + gridDim.x - 1) / gridDim.x;
    const int64_t lo = min(Nx, (int64_t)blockIdx.x * per), hi = min(Nx, lo + per);
    const int64_t sub = (hi - lo + R - 1) / R;
    double s = 0.0;
    long long c = 0;
    if (q < R && p < P) {
        const int64_t a = min(hi, lo + q * sub), b = min(hi, a + sub);
        // eight voxels per step, their loads issued together; summed in voxel order
        constexpr int U = 8;
        for (int64_t n0 = a; n0 < b; n0 += U) {
            int lb[U];
            float v[U];
#pragma unroll
            for (int k = 0; k < U; ++k) lb[k] = n0 + k < b ? lab[n0 + k] : 0;
#pragma unroll
            for (int k = 0; k < U; ++k) v[k] = lb[k] == i + 1 ? xs[(n0 + k) * Ns + j] : 0.f;
#pragma unroll
            for (int k = 0; k < U; ++k)
                if (lb[k] == i + 1) {
                    s += (double)v[k];
                    ++c;
                }
        }
        ssum[q][p] = s;
        scnt[q][p] = c;
    }
    __syncthreads();
    if (threadIdx.x < P) {
        const int pp = threadIdx.x;
        double t = 0.0;
        long long n = 0;
        for (int r = 0; r < R; ++r) {
            t += ssum[r][pp];
            n += scnt[r][pp];
        }
        part[(size_t)blockIdx.x * P + pp] = t;
        if (pp % Ns == 0) cnt[(size_t)blockIdx.x * Nm + pp / Ns] = n;
    }
}

// T[i][j] from the block partials, one warp per (region i, channel j): lanes take
// the blocks in a fixed stride, then a fixed shuffle tree (deterministic); FP32
// and FP64 copies; a status when a region is empty
__global__ void fmd_finish_T(const double *part, const long long *cnt, int nb, int Ns, int Nm, double *T64,
                             float *T, int *status) {
    const int t = blockIdx.x, lane = threadIdx.x;
    const int i = t / Ns, j = t % Ns;
    double s = 0.0;
    long long c = 0;
    for (int b = lane; b < nb; b += 32) {
        s += part[((size_t)b * Nm + i) * Ns + j];
        c += cnt[(size_t)b * Nm + i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
        const double v = c > 0 ? s / (double)c : 0.0;
        if (c == 0 && j == 0) report(status, FHR_ERR_ARG);
        T64[t] = v;
        T[t] = (float)v;
    }
}

// G = T T^T (FP64)
__global__ void fmd_gram(const double *T64, int Ns, int Nm, double *G) {
    const int t = threadIdx.x;
    if (t >= Nm * Nm) return;
    const int a = t / Nm, b = t % Nm;
    double g = 0.0;
    for (int j = 0; j < Ns; ++j) g += T64[a * Ns + j] * T64[b * Ns + j];
    G[t] = g;
}

__global__ void fmd_spectra(const float *__restrict__ D, const double *__restrict__ T64, int Nk, int Ns, int Nm,
                            float *Dm) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)Nk * Nm) return;
    const int k = (int)(idx / Nm), i = (int)(idx % Nm);
    double s = 0.0;
    for (int j = 0; j < Ns; ++j) s += (double)D[(size_t)k * Ns + j] * T64[i * Ns + j];
    Dm[idx] = (float)s;
}

// Every active set P of the per-voxel problems shares G = T T^T, so the inverse of
// each principal block G_PP (at most 2^8 of them) is formed once, in FP64, one
// thread per subset: Cholesky of G_PP, then its inverse embedded in an Nm x Nm
// block with zeros outside P.  inv[P * Nm * Nm] = NaN marks a block that is not
// positive definite.
__global__ void fmd_subset_inverses(const double *__restrict__ Gg, int Nm, double *inv, float *invf) {
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= (1 << Nm)) return;
    double *out = inv + (size_t)P * Nm * Nm;
    float *outf = invf + (size_t)P * Nm * Nm;
    for (int i = 0; i < Nm * Nm; ++i) out[i] = 0.0;
    int idx[kFmdMaxM], m = 0;
    for (int i = 0; i < Nm; ++i)
        if (P >> i & 1) idx[m++] = i;
    double L[kFmdMaxM * kFmdMaxM];
    for (int r = 0; r < m; ++r) {
        for (int c = 0; c <= r; ++c) {
            double s = Gg[idx[r] * Nm + idx[c]];
            for (int k = 0; k < c; ++k) s -= L[r * kFmdMaxM + k] * L[c * kFmdMaxM + k];
            if (r == c) {
                if (!(s > 0.0)) {
                    out[0] = nan("");
                    for (int i = 0; i < Nm * Nm; ++i) outf[i] = i == 0 ? nanf("") : 0.f;
                    return;
                }
                L[r * kFmdMaxM + r] = sqrt(s);
            } else {
                L[r * kFmdMaxM + c] = s / L[c * kFmdMaxM + c];
            }
        }
    }
    // column e of the inverse: L y = e_e, then L^T z = y
    for (int e = 0; e < m; ++e) {
        double y[kFmdMaxM], z[kFmdMaxM];
        for (int r = 0; r < m; ++r) {
            double s = r == e ? 1.0 : 0.0;
            for (int k = 0; k < r; ++k) s -= L[r * kFmdMaxM + k] * y[k];
            y[r] = s / L[r * kFmdMaxM + r];
        }
        for (int r = m - 1; r >= 0; --r) {
            double s = y[r];
            for (int k = r + 1; k < m; ++k) s -= L[k * kFmdMaxM + r] * z[k];
            z[r] = s / L[r * kFmdMaxM + r];
        }
        for (int r = 0; r < m; ++r) out[idx[r] * Nm + idx[e]] = z[r];
    }
    for (int i = 0; i < Nm * Nm; ++i) outf[i] = (float)out[i];
}

// z = G_PP^-1 b_P (zero outside P) from the table; false if G_PP is not positive definite
template <typename R>
__device__ __forceinline__ bool fmd_solve(const R *inv, const R *b, int Nm, unsigned P, R *z) {
    const R *S = inv + (size_t)P * Nm * Nm;
    if (isnan(S[0])) return false;
    for (int i = 0; i < Nm; ++i) {
        R s = 0;
        if (P >> i & 1u)
            for (int k = 0; k < Nm; ++k)
                if (P >> k & 1u) s = fma(S[i * Nm + k], b[k], s);
        z[i] = s;
    }
    return true;
}

// Lawson-Hanson active-set NNLS on the normal equations G x = b in precision R;
// returns the final passive set, x holds the solution
template <typename R>
__device__ unsigned fmd_lh(const R *G, const R *inv, const R *b, int Nm, R tol, R *x) {
    R z[kFmdMaxM];
    for (int i = 0; i < Nm; ++i) x[i] = 0;
    unsigned P = 0;
    for (int outer = 0; outer < 3 * kFmdMaxM; ++outer) {
        // w = b - G x: the most violated coordinate outside P enters
        int t = -1;
        R best = tol;
        for (int i = 0; i < Nm; ++i) {
            R s = b[i];
            for (int k = 0; k < Nm; ++k) s -= G[i * Nm + k] * x[k];
            if (!(P >> i & 1u) && s > best) {
                best = s;
                t = i;
            }
        }
        if (t < 0) break;
        P |= 1u << t;
        for (int inner = 0; inner < 3 * kFmdMaxM; ++inner) {
            if (!fmd_solve<R>(inv, b, Nm, P, z)) {
                P &= ~(1u << t);
                break;
            }
            bool feasible = true;
            for (int i = 0; i < Nm; ++i)
                if ((P >> i & 1u) && z[i] <= 0) feasible = false;
            if (feasible) {
                for (int i = 0; i < Nm; ++i) x[i] = z[i];
                break;
            }
            R alpha = 1;
            for (int i = 0; i < Nm; ++i)
                if ((P >> i & 1u) && z[i] <= 0) alpha = fmin(alpha, x[i] / (x[i] - z[i]));
            for (int i = 0; i < Nm; ++i) {
                x[i] += alpha * (z[i] - x[i]);
                if ((P >> i & 1u) && x[i] <= 0) {
                    x[i] = 0;
                    P &= ~(1u << i);
                }
            }
        }
    }
    return P;
}

// Per voxel: the passive set is searched in FP32, then the solution on that set is
// formed in FP64 and accepted only if it satisfies the NNLS optimality conditions in
// FP64 (positive on the set, w = b - G x <= tol off it); otherwise the search is
// repeated in FP64.  The result is the FP64 Lawson-Hanson solution either way.
__global__ void fmd_nnls(const float *__restrict__ xs, const double *__restrict__ T64, const double *__restrict__ Gg,
                         const double *__restrict__ inv_g, const float *__restrict__ inv_f, int64_t Nx, int Ns, int Nm,
                         float *xm) {
    extern __shared__ double fmd_sm[];   // the subset inverses (FP64, then FP32), when they fit
    __shared__ double G[kFmdMaxM * kFmdMaxM], T[kFmdMaxM * kFmdMaxS];
    __shared__ float Gf[kFmdMaxM * kFmdMaxM], Tf[kFmdMaxM * kFmdMaxS];
    for (int i = threadIdx.x; i < Nm * Nm; i += blockDim.x) {
        G[i] = Gg[i];
        Gf[i] = (float)Gg[i];
    }
    for (int i = threadIdx.x; i < Nm * Ns; i += blockDim.x) {
        T[i] = T64[i];
        Tf[i] = (float)T64[i];
    }
    const int ninv = (1 << Nm) * Nm * Nm;
    const bool in_smem = ninv <= kFmdInvSmem;
    float *fsm = reinterpret_cast<float *>(fmd_sm + ninv);
    if (in_smem)
        for (int i = threadIdx.x; i < ninv; i += blockDim.x) {
            fmd_sm[i] = inv_g[i];
            fsm[i] = inv_f[i];
        }
    const double *inv = in_smem ? fmd_sm : inv_g;
    const float *invf = in_smem ? fsm : inv_f;
    __syncthreads();
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= Nx) return;
    float v[kFmdMaxS];
    for (int j = 0; j < Ns; ++j) v[j] = xs[n * Ns + j];
    double b[kFmdMaxM], x[kFmdMaxM];
    float bf[kFmdMaxM], xf[kFmdMaxM];
    double bn = 0.0;
    float bnf = 0.f;
    for (int i = 0; i < Nm; ++i) {
        double s = 0.0;
        float sf = 0.f;
        for (int j = 0; j < Ns; ++j) {
            s += T[i * Ns + j] * (double)v[j];
            sf = fmaf(Tf[i * Ns + j], v[j], sf);
        }
        b[i] = s;
        bf[i] = sf;
        bn = fmax(bn, fabs(s));
        bnf = fmaxf(bnf, fabsf(sf));
    }
    double gmax = 0.0;
    for (int i = 0; i < Nm * Nm; ++i) gmax = fmax(gmax, fabs(G[i]));
    const double tol = 1e-13 * fmax(bn, 1e-300) * fmax(1.0, gmax);
    const float tolf = 1e-5f * fmaxf(bnf, 1e-30f) * fmaxf(1.f, (float)gmax);
    const unsigned P = fmd_lh<float>(Gf, invf, bf, Nm, tolf, xf);
    bool ok = fmd_solve<double>(inv, b, Nm, P, x);
    for (int i = 0; i < Nm && ok; ++i) {
        if (P >> i & 1u) {
            ok = x[i] > 0.0;
        } else {
            double w = b[i];
            for (int k = 0; k < Nm; ++k) w -= G[i * Nm + k] * x[k];
            ok = w <= tol;
        }
    }
    if (!ok) fmd_lh<double>(G, inv, b, Nm, tol, x);
    for (int i = 0; i < Nm; ++i) xm[n * Nm + i] = (float)x[i];
}

struct FmdWs {
    int *status;
    double *part, *T64, *G, *inv;
    float *invf;
    long long *cnt;
};

static size_t carve_fmd(void *base, int Ns, int Nm, FmdWs *w) {
    Carve c(base);
    FmdWs t;
    t.status = c.take<int>(kStatusBytes / sizeof(int));
    t.part = c.take<double>((size_t)kFmdBlocks * Nm * Ns);
    t.cnt = c.take<long long>((size_t)kFmdBlocks * Nm);
    t.T64 = c.take<double>((size_t)Nm * Ns);
    t.G = c.take<double>((size_t)Nm * Nm);
    t.inv = c.take<double>((size_t)(1 << Nm) * Nm * Nm);
    t.invf = c.take<float>((size_t)(1 << Nm) * Nm * Nm);
    if (w) *w = t;
    return c.size();
}

static fhr_status check_fmd(fhr_ctx *ctx, int64_t Nx, int Ns, int Nm, int Nk) {
    FHR_ARG(Nx > 0 && Nk > 0, "Nx and Nk must be positive");
    FHR_ARG(Ns >= 1 && Ns <= kFmdMaxS, "Ns must be 1..%d", kFmdMaxS);
    FHR_ARG(Nm >= 1 && Nm <= kFmdMaxM && Nm <= Ns, "Nm must be 1..min(8, Ns)");
    return FHR_OK;
}

}  // namespace fhr

using namespace fhr;

extern "C" fhr_status fhr_fmd_workspace_size(fhr_ctx *ctx, int64_t Nx, int Ns, int Nm, int Nk, size_t *bytes) {
    if (!ctx) return FHR_ERR_ARG;
    FHR_TRY(check_fmd(ctx, Nx, Ns, Nm, Nk));
    FHR_ARG(bytes, "bytes is null");
    *bytes = carve_fmd(nullptr, Ns, Nm, nullptr);
    return FHR_OK;
}

extern "C" fhr_status fhr_fmd(fhr_ctx *ctx, int64_t Nx, int Ns, int Nm, int Nk, const float *xs,
                              const uint8_t *labels, const float *D, float *T, float *xm, float *Dm, void *ws,
                              size_t ws_bytes) {
    if (!ctx) return FHR_ERR_ARG;
    FHR_TRY(check_fmd(ctx, Nx, Ns, Nm, Nk));
    FHR_ARG(xs && labels && D && T && xm && Dm && ws, "null pointer argument");
    FHR_ARG(aligned(ws, 256), "workspace must be 256-byte aligned");
    FmdWs w;
    const size_t need = carve_fmd(ws, Ns, Nm, &w);
    FHR_ARG(ws_bytes >= need, "workspace too small: %zu < %zu bytes", ws_bytes, need);
    FHR_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    cudaEvent_t *ev = timer_begin(ctx, TM_FMD);   // the whole decomposition, when profiling
    FHR_CUDA(cudaMemsetAsync(w.status, 0, kStatusBytes, st));
    fmd_region_partials<<<kFmdBlocks, kFmdMaxM * kFmdMaxS, 0, st>>>(xs, labels, Nx, Ns, Nm, w.part, w.cnt);
    FHR_LAUNCHED();
    fmd_finish_T<<<Nm * Ns, 32, 0, st>>>(w.part, w.cnt, kFmdBlocks, Ns, Nm, w.T64, T, w.status);
    FHR_LAUNCHED();
    fmd_gram<<<1, kFmdMaxM * kFmdMaxM, 0, st>>>(w.T64, Ns, Nm, w.G);
    FHR_LAUNCHED();
    fmd_spectra<<<(unsigned)cdiv((int64_t)Nk * Nm, 256), 256, 0, st>>>(D, w.T64, Nk, Ns, Nm, Dm);
    FHR_LAUNCHED();
    fmd_subset_inverses<<<(unsigned)cdiv(1 << Nm, 64), 64, 0, st>>>(w.G, Nm, w.inv, w.invf);
    FHR_LAUNCHED();
    const int ninv = (1 << Nm) * Nm * Nm;
    const size_t smem = ninv <= kFmdInvSmem ? (size_t)ninv * (sizeof(double) + sizeof(float)) : 0;
    fmd_nnls<<<(unsigned)cdiv(Nx, 128), 128, smem, st>>>(xs, w.T64, w.G, w.inv, w.invf, Nx, Ns, Nm, xm);
    FHR_LAUNCHED();
    if (ev) cudaEventRecord(ev[1], st);
    return FHR_OK;
}
