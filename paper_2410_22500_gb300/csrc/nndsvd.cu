// NNDSVD initialisation (the start named in Sec. III; Boutsidis & Gallopoulos
// 2008) on the device.
//
// The top-K singular triplets of P come from a randomised subspace iteration
// that reuses the fused pass kernel in projection mode: with an orthonormal
// Nk x L basis Q in place of D, one pass gives Z = P^T P Q and H = Q^T P^T P Q.
// Z is re-orthonormalised by two rounds of Cholesky-QR in double precision.
// After the last round H is diagonalised (cyclic Jacobi, double precision) and
// the Ritz vectors V = Q U give the wavelength-side singular vectors; one
// more pass stores the pixel-side vectors u_i = P v_i / s_i into W.  Then the
// NNDSVD rule picks, per component, the positive or negative parts.
#include <math.h>

#include "nmf_internal.h"

namespace fhr {

constexpr int kColThreads = 256;

struct NnState {
    double Rinv[kMaxK * kMaxK];   // inverse Cholesky factor of the last Gram
    double sig[kMaxK];            // singular values s_i
    double U[kMaxK * kMaxK];      // eigenvectors of H (columns), sorted
    int L, K;
    float wmul[kMaxK], dmul[kMaxK];
    int sign[kMaxK];              // 0: absolute value (first component), +1 / -1 part
};

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

// Gaussian start matrix Omega [Nk][L] (Box-Muller on two splitmix64 uniforms)
__global__ void nn_random(double *Q, int Nk, int L, uint64_t seed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Nk * L) return;
    const uint64_t a = splitmix64(seed * 0x100000001b3ull + 2ull * i);
    const uint64_t b = splitmix64(seed * 0x100000001b3ull + 2ull * i + 1ull);
    const double u1 = ((a >> 11) + 1.0) * (1.0 / 9007199254740993.0);
    const double u2 = (b >> 11) * (1.0 / 9007199254740992.0);
    Q[i] = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

// Partial Gram Z^T Z over a block of rows; the last block forms the inverse
// Cholesky factor Rinv (Z = Q R, Q = Z Rinv).
__global__ void nn_colgram(const double *Z, int Nk, int L, double *part, unsigned *counter, NnState *st,
                           int *status) {
    __shared__ double sh[kColThreads];
    __shared__ bool last;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double z[kMaxK];
    for (int s = 0; s < L; ++s) z[s] = k < Nk ? Z[(size_t)k * L + s] : 0.0;
    for (int s = 0; s < L; ++s)
        for (int t = 0; t <= s; ++t) {
            sh[threadIdx.x] = z[s] * z[t];
            __syncthreads();
            for (int o = blockDim.x / 2; o > 0; o >>= 1) {
                if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
                __syncthreads();
            }
            if (threadIdx.x == 0) part[(size_t)blockIdx.x * kMaxK * kMaxK + s * kMaxK + t] = sh[0];
            __syncthreads();
        }
    __threadfence();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    double G[kMaxK][kMaxK], R[kMaxK][kMaxK], Ri[kMaxK][kMaxK];
    for (int s = 0; s < L; ++s)
        for (int t = 0; t <= s; ++t) {
            double a = 0.0;
            for (unsigned b = 0; b < gridDim.x; ++b) a += part[(size_t)b * kMaxK * kMaxK + s * kMaxK + t];
            G[s][t] = G[t][s] = a;
        }
    // Cholesky G = R^T R (R upper triangular); a column that has collapsed is
    // replaced by a tiny diagonal so the basis stays finite
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j) R[i][j] = 0.0;
    double scale = 0.0;
    for (int i = 0; i < L; ++i) scale = fmax(scale, G[i][i]);
    for (int j = 0; j < L; ++j) {
        double d = G[j][j];
        for (int k2 = 0; k2 < j; ++k2) d -= R[k2][j] * R[k2][j];
        if (!(d > 1e-28 * scale)) d = 1e-28 * scale + 1e-300;
        R[j][j] = sqrt(d);
        for (int i = j + 1; i < L; ++i) {
            double a = G[j][i];
            for (int k2 = 0; k2 < j; ++k2) a -= R[k2][j] * R[k2][i];
            R[j][i] = a / R[j][j];
        }
    }
    // Ri = R^{-1} (upper triangular back substitution)
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j) Ri[i][j] = 0.0;
    for (int j = 0; j < L; ++j) {
        Ri[j][j] = 1.0 / R[j][j];
        for (int i = j - 1; i >= 0; --i) {
            double a = 0.0;
            for (int k2 = i + 1; k2 <= j; ++k2) a += R[i][k2] * Ri[k2][j];
            Ri[i][j] = -a / R[i][i];
        }
    }
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j) {
            st->Rinv[i * kMaxK + j] = Ri[i][j];
            if (!isfinite(Ri[i][j])) report(status, FHR_ERR_NONFINITE);
        }
    *counter = 0u;
}

// Q = Z Rinv, row by row
__global__ void nn_apply_rinv(const double *Z, double *Q, int Nk, int L, const NnState *st) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nk) return;
    double z[kMaxK];
    for (int s = 0; s < L; ++s) z[s] = Z[(size_t)k * L + s];
    for (int j = 0; j < L; ++j) {
        double a = 0.0;
        for (int s = 0; s <= j; ++s) a += z[s] * st->Rinv[s * kMaxK + j];
        Q[(size_t)k * L + j] = a;
    }
}

// Pass state for projection mode: D = basis as given, W scale set by `wsc`.
__global__ void nn_pass_state(NmfState *st, int L, const NnState *nn, int use_inv_sigma) {
    const int t = threadIdx.x;
    if (t < kMaxK) {
        st->invn[t] = 1.0;
        float w = 1.f;
        if (use_inv_sigma && t < nn->K) w = nn->sig[t] > 0.0 ? (float)(1.0 / nn->sig[t]) : 0.f;
        st->wscale[t] = w;
        st->invdiag[t] = 0.f;
        st->Gdiag[t] = 0.f;
    }
    for (int i = t; i < kMaxK * kMaxK; i += blockDim.x) st->G[i] = 0.f;
}

// Rayleigh-Ritz: H = GW64 (L x L) -> eigenpairs by cyclic Jacobi, sorted descending.
__global__ void nn_rayleigh_ritz(const double *H64, int L, int K, NnState *st, int *status) {
    if (threadIdx.x != 0) return;
    double A[kMaxK][kMaxK], Vv[kMaxK][kMaxK];
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j) {
            A[i][j] = 0.5 * (H64[i * L + j] + H64[j * L + i]);
            Vv[i][j] = i == j ? 1.0 : 0.0;
        }
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < L; ++i)
            for (int j = 0; j < L; ++j) {
                tot += A[i][j] * A[i][j];
                if (i != j) off += A[i][j] * A[i][j];
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < L - 1; ++p)
            for (int q = p + 1; q < L; ++q) {
                if (A[p][q] == 0.0) continue;
                const double th = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < L; ++k) {
                    const double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < L; ++k) {
                    const double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < L; ++k) {
                    const double vkp = Vv[k][p], vkq = Vv[k][q];
                    Vv[k][p] = c * vkp - s * vkq;
                    Vv[k][q] = s * vkp + c * vkq;
                }
            }
    }
    int order[kMaxK];
    for (int i = 0; i < L; ++i) order[i] = i;
    for (int i = 0; i < L; ++i)
        for (int j = i + 1; j < L; ++j)
            if (A[order[j]][order[j]] > A[order[i]][order[i]]) {
                const int tmp = order[i];
                order[i] = order[j];
                order[j] = tmp;
            }
    for (int i = 0; i < K; ++i) {
        const double lam = A[order[i]][order[i]];
        st->sig[i] = lam > 0.0 ? sqrt(lam) : 0.0;
        for (int r = 0; r < L; ++r) st->U[r * kMaxK + i] = Vv[r][order[i]];
        if (!isfinite(st->sig[i])) report(status, FHR_ERR_NONFINITE);
    }
    st->L = L;
    st->K = K;
}

// Ritz vectors: Vk[k][i] = sum_r Q[k][r] U[r][i]  (stored [Nk][K] as the pass's D)
__global__ void nn_ritz_vectors(const double *Q, int Nk, int L, int K, const NnState *st, double *Vk) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nk) return;
    for (int i = 0; i < K; ++i) {
        double a = 0.0;
        for (int r = 0; r < L; ++r) a += Q[(size_t)k * L + r] * st->U[r * kMaxK + i];
        Vk[(size_t)k * K + i] = a;
    }
}

// Norms of the positive and negative parts of u_i (columns of W, over Np) and
// of v_i (over Nk); the last block applies the NNDSVD choice.
__global__ void nn_split_norms(const float *W, int64_t Np, const double *Vk, int Nk, int K, double *part,
                               unsigned *counter, NnState *st) {
    __shared__ double sh[2 * kMaxK][33];
    __shared__ bool last;
    double sp[kMaxK], sn[kMaxK];
    for (int i = 0; i < K; ++i) sp[i] = sn[i] = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < Np; j += (int64_t)gridDim.x * blockDim.x)
        for (int i = 0; i < K; ++i) {
            const double u = W[j * K + i];
            if (u > 0) sp[i] += u * u;
            else sn[i] += u * u;
        }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = 0; i < 2 * K; ++i) {
        double v = i < K ? sp[i] : sn[i - K];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[i][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 2 * K) {
        double a = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += sh[threadIdx.x][w];
        part[(size_t)blockIdx.x * 2 * kMaxK + threadIdx.x] = a;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    for (int i = 0; i < K; ++i) {
        double up = 0.0, un = 0.0, vp = 0.0, vn = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) {
            up += part[(size_t)b * 2 * kMaxK + i];
            un += part[(size_t)b * 2 * kMaxK + K + i];
        }
        for (int k = 0; k < Nk; ++k) {
            const double v = Vk[(size_t)k * K + i];
            if (v > 0) vp += v * v;
            else vn += v * v;
        }
        up = sqrt(up); un = sqrt(un); vp = sqrt(vp); vn = sqrt(vn);
        const double s = st->sig[i];
        if (i == 0) {
            st->sign[i] = 0;
            st->wmul[i] = (float)sqrt(s);
            st->dmul[i] = (float)sqrt(s);
            continue;
        }
        const double mp = up * vp, mn = un * vn;
        const bool pos = mp >= mn;
        const double m = pos ? mp : mn;
        st->sign[i] = pos ? 1 : -1;
        if (m > 0.0) {
            const double lam = sqrt(s * m);
            st->wmul[i] = (float)(lam / (pos ? up : un));
            st->dmul[i] = (float)(lam / (pos ? vp : vn));
        } else {
            st->wmul[i] = st->dmul[i] = 0.f;
        }
    }
    *counter = 0u;
}

__device__ __forceinline__ float nn_part(double x, int sign) {
    if (sign == 0) return (float)fabs(x);
    return (float)(sign > 0 ? fmax(x, 0.0) : fmax(-x, 0.0));
}

__global__ void nn_apply_split(float *W, int64_t Np, const double *Vk, int Nk, int K, const NnState *st, float *D) {
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = i0; j < Np * K; j += stride) {
        const int i = (int)(j % K);
        W[j] = nn_part(W[j], st->sign[i]) * st->wmul[i];
    }
    for (int64_t j = i0; j < (int64_t)Nk * K; j += stride) {
        const int i = (int)(j % K);
        D[j] = nn_part(Vk[j], st->sign[i]) * st->dmul[i];
    }
}

struct NnWs {
    float *Qpart, *Gpart, *ssqpart;
    double *Z64, *H64, *ssq64, *Q64, *Vk, *part;
    unsigned *counter;
    NmfState *pst;
    NnState *nst;
};

size_t carve_nndsvd(Carve &c, int64_t Np, int Nk, int L, int K, int grid, void *out) {
    NnWs t;
    t.counter = c.take<unsigned>(4);
    t.pst = c.take<NmfState>(1);
    t.nst = c.take<NnState>(1);
    t.Qpart = c.take<float>((size_t)grid * Nk * L);
    t.Gpart = c.take<float>((size_t)grid * L * L);
    t.ssqpart = c.take<float>((size_t)grid);
    t.Z64 = c.take<double>((size_t)Nk * L);
    t.H64 = c.take<double>((size_t)L * L);
    t.ssq64 = c.take<double>(1);
    t.Q64 = c.take<double>((size_t)Nk * L);
    t.Vk = c.take<double>((size_t)Nk * K);
    const int nb = (int)cdiv(Nk, kColThreads);
    t.part = c.take<double>((size_t)std::max(nb, 256) * kMaxK * kMaxK);
    (void)Np;
    if (out) *(NnWs *)out = t;
    return c.size();
}

int nndsvd_L(int K, int Nk) { return std::min(std::min(kMaxK, K + 2), Nk); }

// reduction kernel shared with the decomposition
__global__ void nmf_reduce(const float *Qpart, const float *Gpart, const float *ssqpart, int grid, int nval, int K,
                           double *Q64, double *GW64, double *ssq64, int want_ssq);

fhr_status nndsvd_run(fhr_ctx *ctx, const fhr_nmf_params *p, const void *P, float *D, float *W, void *region,
                      int *status) {
    const int K = p->K, Nk = p->Nk, L = nndsvd_L(K, Nk);
    PassConfig cfgL, cfgK;
    FHR_TRY(pass_config(ctx, L, Nk, p->ldP, p->p_dtype, &cfgL));
    FHR_TRY(pass_config(ctx, K, Nk, p->ldP, p->p_dtype, &cfgK));
    const int grid = std::max(cfgL.grid, cfgK.grid);
    Carve c(region);
    NnWs w;
    carve_nndsvd(c, p->Np, Nk, L, K, grid, &w);
    cudaStream_t st = ctx->stream;
    FHR_CUDA(cudaMemsetAsync(w.counter, 0, 4 * sizeof(unsigned), st));
    const int nb = (int)cdiv(Nk, kColThreads);
    const int q = p->power_iters > 0 ? p->power_iters : 8;

    nn_random<<<(unsigned)cdiv((int64_t)Nk * L, 256), 256, 0, st>>>(w.Z64, Nk, L, p->seed);
    FHR_LAUNCHED();
    nn_pass_state<<<1, 64, 0, st>>>(w.pst, L, w.nst, 0);
    FHR_LAUNCHED();

    PassArgs a;
    a.P = P;
    a.Np = p->Np;
    a.Nk = Nk;
    a.ldP = p->ldP;
    a.st = w.pst;
    a.W = W;
    a.Qpart = w.Qpart;
    a.Gpart = w.Gpart;
    a.ssqpart = w.ssqpart;
    a.status = status;
    a.want_ssq = 0;

    auto orthonormalise = [&](void) -> fhr_status {
        for (int round = 0; round < 2; ++round) {   // Cholesky-QR twice
            nn_colgram<<<nb, kColThreads, 0, st>>>(w.Z64, Nk, L, w.part, w.counter, w.nst, status);
            FHR_LAUNCHED();
            nn_apply_rinv<<<nb, kColThreads, 0, st>>>(w.Z64, w.Q64, Nk, L, w.nst);
            FHR_LAUNCHED();
            if (round == 0) FHR_CUDA(cudaMemcpyAsync(w.Z64, w.Q64, sizeof(double) * Nk * L, cudaMemcpyDeviceToDevice, st));
        }
        return FHR_OK;
    };

    FHR_TRY(orthonormalise());
    const int nval = Nk * L;
    for (int it = 0; it <= q; ++it) {
        // Z = P^T P Q, H = Q^T P^T P Q
        a.D64 = w.Q64;
        a.mode = PASS_PROJECT;
        FHR_TRY(launch_pass(ctx, cfgL, a));
        nmf_reduce<<<(unsigned)cdiv(nval, 32) + 1, 256, 0, st>>>(w.Qpart, w.Gpart, w.ssqpart, cfgL.grid, nval, L,
                                                                 w.Z64, w.H64, w.ssq64, 0);
        FHR_LAUNCHED();
        if (it < q) FHR_TRY(orthonormalise());
    }
    nn_rayleigh_ritz<<<1, 32, 0, st>>>(w.H64, L, K, w.nst, status);
    FHR_LAUNCHED();
    nn_ritz_vectors<<<nb, kColThreads, 0, st>>>(w.Q64, Nk, L, K, w.nst, w.Vk);
    FHR_LAUNCHED();
    // u_i = P v_i / s_i into W
    nn_pass_state<<<1, 64, 0, st>>>(w.pst, K, w.nst, 1);
    FHR_LAUNCHED();
    a.D64 = w.Vk;
    a.mode = PASS_PROJECT_STORE;
    FHR_TRY(launch_pass(ctx, cfgK, a));
    nn_split_norms<<<256, 256, 0, st>>>(W, p->Np, w.Vk, Nk, K, w.part, w.counter, w.nst);
    FHR_LAUNCHED();
    nn_apply_split<<<ctx->sm_count * 4, 256, 0, st>>>(W, p->Np, w.Vk, Nk, K, w.nst, D);
    FHR_LAUNCHED();
    return FHR_OK;
}

}  // namespace fhr

namespace fhr {
fhr_status nndsvd_ws_size(fhr_ctx *ctx, const fhr_nmf_params *p, size_t *bytes) {
    const int K = p->K, Nk = p->Nk, L = nndsvd_L(K, Nk);
    PassConfig cfgL, cfgK;
    FHR_TRY(pass_config(ctx, L, Nk, p->ldP, p->p_dtype, &cfgL));
    FHR_TRY(pass_config(ctx, K, Nk, p->ldP, p->p_dtype, &cfgK));
    Carve c(nullptr);
    *bytes = carve_nndsvd(c, p->Np, Nk, L, K, std::max(cfgL.grid, cfgK.grid), nullptr);
    return FHR_OK;
}
}  // namespace fhr
