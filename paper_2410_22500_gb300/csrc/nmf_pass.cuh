// Fused one-pass NMF kernel (fast HALS, Sec. III / Eq. sub_extract_solve).
//
// One launch streams P = [Np][ldP] exactly once.  Each CTA is persistent and
// owns tiles of ROWS pixel rows, fetched by a producer warp with 1-D bulk
// copies (cp.async.bulk, mbarrier completion) into a ring of shared-memory
// stages.  For every tile the consumer threads
//   1. form r_j = D^T p_j for each pixel j of the tile (each thread owns fixed
//      16-byte columns of bins and keeps D for them in registers; partial sums
//      are reduced across lanes with a butterfly reduce-scatter and across
//      warps through shared memory),
//   2. update the pixel's K coefficients (HALS V half-step, Gauss-Seidel over
//      the K coordinates, in ROWS threads), or, in projection mode, take w = r,
//   3. accumulate Q += p_j w_j^T (Nk x K, registers of the column owners) and
//      G_W += w_j w_j^T, re-reading the tile from shared memory.
// Per-CTA partials (FP32) of Q, G_W and ||P||^2 are written at the end and
// reduced across CTAs in double precision by the update kernels.
#pragma once

#include "common.cuh"

namespace fhr {

constexpr int kPassRows = 8;       // pixel rows per tile
constexpr int kMaxK = 8;

enum PassMode { PASS_HALS = 0, PASS_PROJECT = 1, PASS_PROJECT_STORE = 2 };

// Iteration state published by the D-update kernel for the next pass.
struct NmfState {
    double invn[kMaxK];        // normalised D = D64 * invn (column-wise)
    float wscale[kMaxK];       // true W = W buffer * wscale (column-wise)
    float G[kMaxK * kMaxK];    // (normalised D)^T (normalised D)
    float invdiag[kMaxK];      // 1 / G[s][s] (0 when G[s][s] == 0)
    float Gdiag[kMaxK];        // G[s][s]
};

struct PassArgs {
    const void *P;             // [Np][ldP]
    int64_t Np;
    int Nk, ldP;
    const double *D64;         // [Nk][K] (unnormalised)
    const NmfState *st;
    float *W;                  // [Np][K]
    float *Qpart;              // [grid][Nk][K]
    float *Gpart;              // [grid][K*K]
    float *ssqpart;            // [grid]
    int *status;
    int mode;
    int stages;
};

template <typename TP>
struct Vec16;
template <>
struct Vec16<float> {
    static constexpr int N = 4;
    __device__ __forceinline__ static void load(const float *s, float *x) {
        float4 v = *reinterpret_cast<const float4 *>(s);
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    }
};
template <>
struct Vec16<__nv_bfloat16> {
    static constexpr int N = 8;
    __device__ __forceinline__ static void load(const __nv_bfloat16 *s, float *x) {
        uint4 v = *reinterpret_cast<const uint4 *>(s);
        const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            x[2 * i] = __uint_as_float(u[i] << 16);
            x[2 * i + 1] = __uint_as_float(u[i] & 0xffff0000u);
        }
    }
};

// ---- butterfly reduce-scatter of N values across the 32 lanes of a warp.
// After the call lane l holds in v[0..final_count) the warp sums of original
// indices i + base(l), base(l) = sum over steps of (lane bit ? half : 0).
template <int N>
struct Half {
    static constexpr int H = (N + 1) / 2;
};

template <int N, int OFF>
__device__ __forceinline__ void bfly_step(float *v, int lane, int &base, int &cnt) {
    constexpr int H = Half<N>::H;
    const bool up = (lane & OFF) != 0;
#pragma unroll
    for (int i = 0; i < H; ++i) {
        float lo = v[i];
        float hi = (i + H < N) ? v[i + H] : 0.f;
        float send = up ? lo : hi;
        float keep = up ? hi : lo;
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, OFF);
    }
    // the lower lane keeps entries [0, H) of the previous array, the upper lane
    // [H, 2H); only the first `cnt` entries of a lane's array are real values
    if (up) {
        base += H;
        cnt = cnt > H ? cnt - H : 0;
    } else {
        cnt = cnt < H ? cnt : H;
    }
}

template <int N>
struct Bfly {
    static constexpr int N1 = Half<N>::H, N2 = Half<N1>::H, N3 = Half<N2>::H, N4 = Half<N3>::H,
                         N5 = Half<N4>::H;
    static constexpr int FINAL = N5;
    // After run(), final value i < cnt of this lane is the warp sum of original
    // index base + i; every original index is held by exactly one lane.
    __device__ __forceinline__ static void run(float *v, int lane, int &base, int &cnt) {
        base = 0;
        cnt = N;
        bfly_step<N, 16>(v, lane, base, cnt);
        bfly_step<N1, 8>(v, lane, base, cnt);
        bfly_step<N2, 4>(v, lane, base, cnt);
        bfly_step<N3, 2>(v, lane, base, cnt);
        bfly_step<N4, 1>(v, lane, base, cnt);
    }
};

__device__ __forceinline__ bool bar_red_or(int id, int nthreads, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %3, 0;\n\t"
        "bar.red.or.pred p, %1, %2, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"(id), "r"(nthreads), "r"((uint32_t)pred)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void bar_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <int K, int CPT, typename TP>
__global__ void __launch_bounds__(256, 1) nmf_pass_kernel(PassArgs a) {
    constexpr int VEC = Vec16<TP>::N;
    constexpr int ROWS = kPassRows;
    constexpr int V = ROWS * K;
    using BF = Bfly<V>;

    const int NT = blockDim.x - 32;          // consumer threads
    const int NW = NT / 32;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int ncol = a.ldP / VEC;
    const int S = a.stages;
    const int64_t ntiles = (a.Np + ROWS - 1) / ROWS;

    extern __shared__ __align__(128) unsigned char smem[];
    const size_t stage_bytes = (size_t)ROWS * a.ldP * sizeof(TP);
    TP *tiles = reinterpret_cast<TP *>(smem);
    float *red = reinterpret_cast<float *>(smem + S * stage_bytes);      // [NW][V]
    float *wnew = red + NW * V;                                           // [ROWS][K]
    float *gsm = wnew + ROWS * K;                                         // G[K][K]
    float *invd = gsm + K * K;                                            // [K]
    float *wsc = invd + K;                                                // [K]
    float *gwacc = wsc + K;                                               // [ROWS][K*K]
    uint64_t *full = reinterpret_cast<uint64_t *>(
        (reinterpret_cast<uintptr_t>(gwacc + ROWS * K * K) + 7) & ~uintptr_t(7));
    uint64_t *empty = full + S;

    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], NT);
        }
        fence_mbar_init();
    }
    for (int i = tid; i < K * K; i += blockDim.x) gsm[i] = a.st->G[(i / K) * kMaxK + i % K];
    if (tid < K) {
        invd[tid] = a.st->invdiag[tid];
        wsc[tid] = a.st->wscale[tid];
    }
    __syncthreads();

    if (warp == NW) {
        // ---------------- producer warp
        if (lane == 0) {
            int64_t i = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
                const int s = (int)(i % S);
                if (i >= S) {
                    if (!mbar_wait_bounded(&empty[s], (uint32_t)(((i / S) - 1) & 1))) {
                        ok = false;
                        report(a.status, FHR_ERR_TIMEOUT);
                        break;
                    }
                }
                const int64_t r0 = tile * ROWS;
                const int rows = (int)((a.Np - r0) < ROWS ? (a.Np - r0) : ROWS);
                const uint32_t bytes = (uint32_t)(rows * (size_t)a.ldP * sizeof(TP));
                mbar_arrive_expect_tx(&full[s], bytes);
                bulk_g2s(reinterpret_cast<unsigned char *>(tiles) + s * stage_bytes,
                         reinterpret_cast<const TP *>(a.P) + r0 * a.ldP, bytes, &full[s]);
            }
            // drain: every issued copy must land before the CTA exits
            const int64_t issued = i;
            for (int64_t j = (issued > S ? issued - S : 0); j < issued; ++j) {
                const int s = (int)(j % S);
                if (!mbar_wait_bounded(&full[s], (uint32_t)((j / S) & 1))) {
                    report(a.status, FHR_ERR_TIMEOUT);
                }
            }
            (void)ok;
        }
        return;
    }

    // ---------------- consumers
    float Dr[CPT][VEC][K];
    float Qr[CPT][VEC][K];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        const int col = tid + c * NT;
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            const int k = col * VEC + e;
#pragma unroll
            for (int s = 0; s < K; ++s) {
                Qr[c][e][s] = 0.f;
                Dr[c][e][s] = (col < ncol && k < a.Nk) ? (float)(a.D64[(size_t)k * K + s] * a.st->invn[s]) : 0.f;
            }
        }
    }
    float ssq = 0.f;
    // G_W partials live in shared memory, one K x K block per update thread
    if (tid < ROWS) {
        for (int j = 0; j < K * K; ++j) gwacc[tid * K * K + j] = 0.f;
    }

    int64_t i = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
        const int s_ = (int)(i % S);
        const int64_t r0 = tile * ROWS;
        const int rows = (int)((a.Np - r0) < ROWS ? (a.Np - r0) : ROWS);
        // the pixel-update threads fetch the old coefficients early
        float wold[K];
        if (a.mode == PASS_HALS && tid < rows) {
#pragma unroll
            for (int s = 0; s < K; ++s) wold[s] = a.W[(r0 + tid) * K + s];
        }
        const bool ok = mbar_wait_bounded(&full[s_], (uint32_t)((i / S) & 1));
        const TP *tl = tiles + (size_t)s_ * ROWS * a.ldP;

        // ---- phase 1: r = D^T p (partial over this thread's columns)
        float rp[V];
#pragma unroll
        for (int j = 0; j < V; ++j) rp[j] = 0.f;
        if (ok) {
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int col = tid + c * NT;
                if (col < ncol) {
#pragma unroll
                    for (int row = 0; row < ROWS; ++row) {
                        if (row < rows) {
                            float x[VEC];
                            Vec16<TP>::load(tl + (size_t)row * a.ldP + col * VEC, x);
#pragma unroll
                            for (int e = 0; e < VEC; ++e) {
                                ssq = fmaf(x[e], x[e], ssq);
#pragma unroll
                                for (int s = 0; s < K; ++s) rp[row * K + s] = fmaf(x[e], Dr[c][e][s], rp[row * K + s]);
                            }
                        }
                    }
                }
            }
        }
        int base, cnt;
        BF::run(rp, lane, base, cnt);
#pragma unroll
        for (int j = 0; j < BF::FINAL; ++j)
            if (j < cnt) red[warp * V + base + j] = rp[j];
        const bool bad = bar_red_or(1, NT, !ok);
        if (bad) {
            report(a.status, FHR_ERR_TIMEOUT);
            break;
        }

        // ---- phase 2: per-pixel coefficient update
        if (tid < rows) {
            float r[K], w[K];
#pragma unroll
            for (int s = 0; s < K; ++s) {
                float acc = 0.f;
                for (int wp = 0; wp < NW; ++wp) acc += red[wp * V + tid * K + s];
                r[s] = acc;
            }
            if (a.mode == PASS_HALS) {
#pragma unroll
                for (int s = 0; s < K; ++s) w[s] = wold[s] * wsc[s];
#pragma unroll
                for (int s = 0; s < K; ++s) {
                    if (invd[s] != 0.f) {
                        float g = r[s];
#pragma unroll
                        for (int t = 0; t < K; ++t) g = fmaf(-gsm[s * K + t], w[t], g);
                        w[s] = fmaxf(0.f, w[s] + __fdiv_rn(g, gsm[s * K + s]));
                    }
                }
#pragma unroll
                for (int s = 0; s < K; ++s) a.W[(r0 + tid) * K + s] = w[s];
            } else {
#pragma unroll
                for (int s = 0; s < K; ++s) w[s] = r[s];
                if (a.mode == PASS_PROJECT_STORE) {
#pragma unroll
                    for (int s = 0; s < K; ++s) a.W[(r0 + tid) * K + s] = w[s] * wsc[s];
                }
            }
            float *gwt = gwacc + tid * K * K;
#pragma unroll
            for (int s = 0; s < K; ++s) {
                wnew[tid * K + s] = w[s];
#pragma unroll
                for (int t = 0; t < K; ++t) gwt[s * K + t] = fmaf(w[s], w[t], gwt[s * K + t]);
            }
        }
        bar_sync(1, NT);

        // ---- phase 3: Q += p w^T over this thread's columns
#pragma unroll
        for (int row = 0; row < ROWS; ++row) {
            if (row < rows) {
                float wv[K];
#pragma unroll
                for (int s = 0; s < K; ++s) wv[s] = wnew[row * K + s];
#pragma unroll
                for (int c = 0; c < CPT; ++c) {
                    const int col = tid + c * NT;
                    if (col < ncol) {
                        float x[VEC];
                        Vec16<TP>::load(tl + (size_t)row * a.ldP + col * VEC, x);
#pragma unroll
                        for (int e = 0; e < VEC; ++e)
#pragma unroll
                            for (int s = 0; s < K; ++s) Qr[c][e][s] = fmaf(x[e], wv[s], Qr[c][e][s]);
                    }
                }
            }
        }
        mbar_arrive(&empty[s_]);
    }

    // ---- per-CTA partials
    const int g = blockIdx.x;
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        const int col = tid + c * NT;
        if (col < ncol) {
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const int k = col * VEC + e;
                if (k < a.Nk) {
#pragma unroll
                    for (int s = 0; s < K; ++s) a.Qpart[((size_t)g * a.Nk + k) * K + s] = Qr[c][e][s];
                }
            }
        }
    }
    // ||P||^2: warp then CTA reduction
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ssq += __shfl_xor_sync(0xffffffffu, ssq, o);
    if (lane == 0) red[warp] = ssq;
    bar_sync(1, NT);
    for (int i = tid; i < K * K; i += NT) {   // K*K may exceed the consumer count
        float acc = 0.f;
        for (int r = 0; r < ROWS; ++r) acc += gwacc[r * K * K + i];
        a.Gpart[(size_t)g * K * K + i] = acc;
    }
    if (tid == 0) {
        float acc = 0.f;
        for (int wp = 0; wp < NW; ++wp) acc += red[wp];
        a.ssqpart[g] = acc;
    }
}

}  // namespace fhr
