// Fused one-pass NMF kernel (fast HALS, Sec. III / Eq. sub_extract_solve).
//
// One launch streams P = [Np][ldP] exactly once.  Each CTA is persistent and
// owns tiles of ROWS pixel rows.  Three warp roles share a ring of
// shared-memory stages:
//   producer warp   1-D bulk copies (cp.async.bulk, mbarrier completion) of
//                   whole tiles (ROWS contiguous rows of P) into the ring;
//   consumer warps  each thread owns fixed 16-byte columns of bins;
//                   phase 1 (tile t): partial r_j = D^T p_j over its columns
//                   (D read from shared memory once per column and tile),
//                   reduced across lanes by a butterfly reduce-scatter and
//                   handed to the update warp through shared memory;
//                   phase 3 (tile t-1): Q += p_j w_j^T over its columns (Q in
//                   registers for the whole launch), then the stage is freed;
//   update warp     for tile t, as soon as its r is complete: the HALS V
//                   half-step of the ROWS pixels (Gauss-Seidel over the K
//                   coordinates), or w = r in projection mode; G_W += w w^T.
// The update of tile t overlaps phase 1 of tile t+1, so no CTA-wide barrier
// sits on the per-tile path; all hand-offs are mbarriers with bounded waits.
// Per-CTA partials (FP32) of Q, G_W and ||P||^2 are written at the end and
// reduced across CTAs in double precision by the update kernels.
#pragma once

#include "common.cuh"

namespace fhr {

constexpr int kPassRows = 4;       // pixel rows per tile
constexpr int kMaxK = 8;

enum PassMode { PASS_HALS = 0, PASS_PROJECT = 1, PASS_PROJECT_STORE = 2, PASS_GIVEN_W = 3 };

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
    int want_ssq;              // accumulate ||P||^2 (first pass only)
    int K;                     // columns of D / W (set by the launcher)
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

// Explicit shared-space accesses (32-bit shared addresses): keeps every tile,
// dictionary and hand-off access an LDS/STS whatever the compiler can prove.
__device__ __forceinline__ float4 lds_f4(uint32_t a) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ uint4 lds_u4(uint32_t a) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts_f32(uint32_t a, float v) {
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v));
}

template <typename TP>
struct LdsVec;
template <>
struct LdsVec<float> {
    __device__ __forceinline__ static void load(uint32_t a, float *x) {
        const float4 v = lds_f4(a);
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    }
};
template <>
struct LdsVec<__nv_bfloat16> {
    __device__ __forceinline__ static void load(uint32_t a, float *x) {
        const uint4 v = lds_u4(a);
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


template <int K>
struct KPad {
    static constexpr int P = (2 * K + 3) / 4 * 4;   // w rows: K pairs {w, w}, padded to whole float4s
};

// Shared-memory layout of the pass kernel (host and device agree on it).
struct PassSmem {
    size_t tiles, dsm, red, wnew, gsm, invd, wsc, gwacc, ssq, bars, total;
};

__host__ __device__ inline PassSmem pass_smem_layout(int K, int NW, int ldP, int esize, int stages) {
    const int ROWS = kPassRows, V = ROWS * K, KP = (2 * K + 3) / 4 * 4;
    PassSmem L;
    size_t o = 0;
    auto take = [&](size_t bytes, size_t align) {
        o = (o + align - 1) / align * align;
        size_t r = o;
        o += bytes;
        return r;
    };
    L.tiles = take((size_t)stages * ROWS * ldP * esize, 128);
    L.dsm = take((size_t)ldP * K * sizeof(float), 16);
    L.red = take((size_t)2 * NW * V * sizeof(float), 16);
    L.wnew = take((size_t)2 * ROWS * KP * sizeof(float), 16);
    L.gsm = take((size_t)K * K * sizeof(float), 16);
    L.invd = take((size_t)K * sizeof(float), 16);
    L.wsc = take((size_t)K * sizeof(float), 16);
    L.gwacc = take((size_t)ROWS * K * K * sizeof(float), 16);
    L.ssq = take((size_t)(NW + 1) * sizeof(float), 16);
    L.bars = take((size_t)(2 * stages + 4) * sizeof(uint64_t), 8);
    L.total = (o + 127) / 128 * 128;
    return L;
}

// Two CTAs per SM need <= 128 registers per thread; variants whose register
// state (Q, partial r, one column of D) fits are compiled for that.
template <int K, int CPT, typename TP>
struct PassOcc {
    static constexpr int VEC = Vec16<TP>::N;
    static constexpr int MINB = (CPT * VEC * K + VEC * K + 2 * kPassRows * K <= 100) ? 2 : 1;
};

template <int K, int CPT, typename TP>
__global__ void __launch_bounds__(256, (PassOcc<K, CPT, TP>::MINB)) nmf_pass_kernel(PassArgs a) {
    constexpr int VEC = Vec16<TP>::N;
    constexpr int ROWS = kPassRows;
    constexpr int V = ROWS * K;
    constexpr int KP = KPad<K>::P;
    using BF = Bfly<V>;

    const int NT = blockDim.x - 64;          // consumer threads; then the update warp, then the producer
    const int NW = NT / 32;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int ncol = a.ldP / VEC;
    const int S = a.stages;
    const int64_t ntiles = (a.Np + ROWS - 1) / ROWS;
    const int64_t my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    extern __shared__ __align__(128) unsigned char smem[];
    const PassSmem Lyt = pass_smem_layout(K, NW, a.ldP, (int)sizeof(TP), S);
    TP *tiles = reinterpret_cast<TP *>(smem + Lyt.tiles);
    float *dsm = reinterpret_cast<float *>(smem + Lyt.dsm);       // [ldP][K] normalised D
    float *red = reinterpret_cast<float *>(smem + Lyt.red);       // [2][NW][V]
    float *wnew = reinterpret_cast<float *>(smem + Lyt.wnew);     // [2][ROWS][KP]
    float *gsm = reinterpret_cast<float *>(smem + Lyt.gsm);       // [K][K]
    float *invd = reinterpret_cast<float *>(smem + Lyt.invd);     // [K]
    float *wsc = reinterpret_cast<float *>(smem + Lyt.wsc);       // [K]
    float *gwacc = reinterpret_cast<float *>(smem + Lyt.gwacc);   // [ROWS][K*K]
    float *ssqs = reinterpret_cast<float *>(smem + Lyt.ssq);      // [NW]
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + Lyt.bars);
    uint64_t *empty = full + S;
    uint64_t *redfull = empty + S;      // [2] consumers -> update warp
    uint64_t *wready = redfull + 2;     // [2] update warp -> consumers

    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], NT);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&redfull[i], NT);
            mbar_init(&wready[i], 1);
        }
        fence_mbar_init();
    }
    // dictionary (normalised, FP32) in pair layout: for each 16-byte column of
    // bins and each pair of bins (2q, 2q+1) in it, K pairs {d[2q][s], d[2q+1][s]}
    for (int i = tid; i < a.ldP * K; i += blockDim.x) {
        const int col = i / (VEC * K), rem = i % (VEC * K);
        const int q = rem / (2 * K), s2 = rem % (2 * K), sc = s2 >> 1, half = s2 & 1;
        const int k = col * VEC + 2 * q + half;
        dsm[i] = k < a.Nk ? (float)(a.D64[(size_t)k * K + sc] * a.st->invn[sc]) : 0.f;
    }
    for (int i = tid; i < K * K; i += blockDim.x) gsm[i] = a.st->G[(i / K) * kMaxK + i % K];
    for (int i = tid; i < ROWS * K * K; i += blockDim.x) gwacc[i] = 0.f;
    if (tid < K) {
        invd[tid] = a.st->invdiag[tid];
        wsc[tid] = a.st->wscale[tid];
    }
    __syncthreads();

    if (warp == NW + 1) {
        // ---------------- producer warp
        if (lane == 0) {
            // stage index and ring parity advance incrementally (no 64-bit division per tile)
            int s = 0;
            uint32_t par = 0;          // parity of the ring pass that stage s is on
            int64_t i = 0;
            int64_t r0 = (int64_t)blockIdx.x * ROWS;
            const int64_t rstep = (int64_t)gridDim.x * ROWS;
            for (; i < my_tiles; ++i, r0 += rstep) {
                if (i >= S && !mbar_wait_bounded(&empty[s], par ^ 1u)) {
                    report(a.status, FHR_ERR_TIMEOUT);
                    break;
                }
                const int rows = (int)((a.Np - r0) < ROWS ? (a.Np - r0) : ROWS);
                const uint32_t bytes = (uint32_t)(rows * (size_t)a.ldP * sizeof(TP));
                mbar_arrive_expect_tx(&full[s], bytes);
                bulk_g2s(tiles + (size_t)s * ROWS * a.ldP, reinterpret_cast<const TP *>(a.P) + r0 * a.ldP, bytes,
                         &full[s]);
                // the ring holds only a few tiles per CTA: ask L2 for the tiles after it
                // so their DRAM latency is paid before the ring reaches them
                const int64_t rp = r0 + (int64_t)S * rstep;
                if (rp < a.Np) {
                    const int prow = (int)((a.Np - rp) < ROWS ? (a.Np - rp) : ROWS);
                    bulk_prefetch_l2(reinterpret_cast<const TP *>(a.P) + rp * a.ldP,
                                     (uint32_t)(prow * (size_t)a.ldP * sizeof(TP)));
                }
                if (++s == S) {
                    s = 0;
                    par ^= 1u;
                }
            }
            // drain: every issued copy must land before the CTA exits
            for (int64_t j = (i > S ? i - S : 0); j < i; ++j)
                if (!mbar_wait_bounded(&full[(int)(j % S)], (uint32_t)((j / S) & 1))) report(a.status, FHR_ERR_TIMEOUT);
        }
        return;
    }

    if (warp == NW) {
        // ---------------- update warp: lanes < rows update one pixel each
        float wold[K], wnext[K];
        auto fetch = [&](int64_t i, float *dst) {
            const int64_t r0 = (blockIdx.x + i * gridDim.x) * ROWS;
            if ((a.mode == PASS_HALS || a.mode == PASS_GIVEN_W) && i < my_tiles && r0 + lane < a.Np && lane < ROWS) {
#pragma unroll
                for (int s = 0; s < K; ++s) dst[s] = a.W[(r0 + lane) * K + s];
            }
        };
        fetch(0, wnext);
        for (int64_t i = 0; i < my_tiles; ++i) {
            const int b = (int)(i & 1);
            const int64_t r0 = (blockIdx.x + i * gridDim.x) * ROWS;
            const int rows = (int)((a.Np - r0) < ROWS ? (a.Np - r0) : ROWS);
#pragma unroll
            for (int s = 0; s < K; ++s) wold[s] = wnext[s];
            fetch(i + 1, wnext);   // prefetch the next tile's coefficients
            if (!mbar_wait_bounded(&redfull[b], (uint32_t)((i >> 1) & 1))) {
                report(a.status, FHR_ERR_TIMEOUT);
                break;
            }
            if (lane < rows) {
                float r[K], w[K];
#pragma unroll
                for (int s = 0; s < K; ++s) {
                    float acc = 0.f;
                    for (int wp = 0; wp < NW; ++wp) acc += red[(b * NW + wp) * V + lane * K + s];
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
                    for (int s = 0; s < K; ++s) a.W[(r0 + lane) * K + s] = w[s];
                } else if (a.mode == PASS_GIVEN_W) {
                    // W held fixed: only P^T W and W^T W are accumulated
#pragma unroll
                    for (int s = 0; s < K; ++s) w[s] = wold[s] * wsc[s];
                } else {
#pragma unroll
                    for (int s = 0; s < K; ++s) w[s] = r[s];
                    if (a.mode == PASS_PROJECT_STORE) {
#pragma unroll
                        for (int s = 0; s < K; ++s) a.W[(r0 + lane) * K + s] = w[s] * wsc[s];
                    }
                }
                float *wn = wnew + (b * ROWS + lane) * KP;
#pragma unroll
                for (int s = 0; s < KP; ++s) wn[s] = s < 2 * K ? w[s >> 1] : 0.f;
                float *gwt = gwacc + lane * K * K;
#pragma unroll
                for (int s = 0; s < K; ++s)
#pragma unroll
                    for (int t = 0; t < K; ++t) gwt[s * K + t] = fmaf(w[s], w[t], gwt[s * K + t]);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&wready[b]);
        }
    } else {
        // ---------------- consumer warps
        constexpr int EP = VEC / 2;   // bin pairs per 16-byte column
        float2 Q2[CPT][EP][K];        // {Q[2q][s], Q[2q+1][s]} for the owned columns
#pragma unroll
        for (int c = 0; c < CPT; ++c)
#pragma unroll
            for (int q = 0; q < EP; ++q)
#pragma unroll
                for (int s = 0; s < K; ++s) Q2[c][q][s] = make_float2(0.f, 0.f);
        float2 ssq2 = make_float2(0.f, 0.f);
        const uint32_t sb = smem_u32(smem);
        const uint32_t row_bytes = (uint32_t)(a.ldP * sizeof(TP));
        const uint32_t stage_bytes = ROWS * row_bytes;
        const uint32_t tiles_a = sb + (uint32_t)Lyt.tiles;
        const uint32_t dsm_a = sb + (uint32_t)Lyt.dsm;
        const uint32_t wnew_a = sb + (uint32_t)Lyt.wnew;
        const uint32_t red_a = sb + (uint32_t)Lyt.red;
        bool ok = true;
        // stage / parity of the tile in phase 1 (cur) and of the one in phase 3 (prev),
        // advanced incrementally (no 64-bit division per tile)
        int s_cur = 0, s_prev = 0;
        uint32_t par_cur = 0;
        int64_t r0_cur = (int64_t)blockIdx.x * ROWS, r0_prev = 0;
        const int64_t rstep = (int64_t)gridDim.x * ROWS;
        for (int64_t i = 0; i <= my_tiles && ok; ++i) {
            if (i < my_tiles) {
                const int s_ = s_cur;
                const int b = (int)(i & 1);
                const int64_t r0 = r0_cur;
                const int rows = (int)((a.Np - r0) < ROWS ? (a.Np - r0) : ROWS);
                if (!mbar_wait_bounded(&full[s_], par_cur)) {
                    ok = false;
                    break;
                }
                const uint32_t tl = tiles_a + s_ * stage_bytes;
                // ---- phase 1: partial r = D^T p over this thread's columns; even and
                // odd bins of each pair accumulate in the two halves of a float2
                float2 acc[ROWS][K];
#pragma unroll
                for (int row = 0; row < ROWS; ++row)
#pragma unroll
                    for (int s = 0; s < K; ++s) acc[row][s] = make_float2(0.f, 0.f);
#pragma unroll
                for (int c = 0; c < CPT; ++c) {
                    const int col = tid + c * NT;
                    if (col < ncol) {
                        float2 d[EP][K];
#pragma unroll
                        for (int f = 0; f < EP * K / 2; ++f) {
                            const float4 v = lds_f4(dsm_a + (uint32_t)(col * VEC * K + 4 * f) * 4u);
                            d[(2 * f) / K][(2 * f) % K] = make_float2(v.x, v.y);
                            d[(2 * f + 1) / K][(2 * f + 1) % K] = make_float2(v.z, v.w);
                        }
                        if (EP * K % 2) {   // odd pair count: the last pair sits alone in a float4
                            const float4 v = lds_f4(dsm_a + (uint32_t)(col * VEC * K + 2 * (EP * K - 1)) * 4u);
                            d[EP - 1][K - 1] = make_float2(v.x, v.y);
                        }
                        const uint32_t ca = tl + (uint32_t)(col * VEC * sizeof(TP));
#pragma unroll
                        for (int row = 0; row < ROWS; ++row) {
                            if (rows == ROWS || row < rows) {
                                float x[VEC];
                                LdsVec<TP>::load(ca + row * row_bytes, x);
#pragma unroll
                                for (int q = 0; q < EP; ++q) {
                                    const float2 xp = make_float2(x[2 * q], x[2 * q + 1]);
#pragma unroll
                                    for (int s = 0; s < K; ++s) acc[row][s] = __ffma2_rn(xp, d[q][s], acc[row][s]);
                                    if (a.want_ssq) ssq2 = __ffma2_rn(xp, xp, ssq2);
                                }
                            }
                        }
                    }
                }
                float rp[V];
#pragma unroll
                for (int row = 0; row < ROWS; ++row)
#pragma unroll
                    for (int s = 0; s < K; ++s) rp[row * K + s] = acc[row][s].x + acc[row][s].y;
                int base, cnt;
                BF::run(rp, lane, base, cnt);
                const uint32_t rw = red_a + (uint32_t)((b * NW + warp) * V) * 4u;
#pragma unroll
                for (int j = 0; j < BF::FINAL; ++j)
                    if (j < cnt) sts_f32(rw + (uint32_t)(base + j) * 4u, rp[j]);
                mbar_arrive(&redfull[b]);
            }
            // ---- phase 3 of the previous tile: Q += p w^T, then free its stage
            if (i >= 1) {
                const int64_t j = i - 1;
                const int b = (int)(j & 1);
                if (!mbar_wait_bounded(&wready[b], (uint32_t)((j >> 1) & 1))) {
                    ok = false;
                    break;
                }
                const int64_t r0 = r0_prev;
                const int rows = (int)((a.Np - r0) < ROWS ? (a.Np - r0) : ROWS);
                const uint32_t tl = tiles_a + (uint32_t)s_prev * stage_bytes;
#pragma unroll
                for (int row = 0; row < ROWS; ++row) {
                    if (rows == ROWS || row < rows) {
                        float2 wd[K];   // {w_s, w_s}
#pragma unroll
                        for (int f = 0; f < KP / 4; ++f) {
                            const float4 v = lds_f4(wnew_a + (uint32_t)((b * ROWS + row) * KP + 4 * f) * 4u);
                            if (2 * f < K) wd[2 * f] = make_float2(v.x, v.y);
                            if (2 * f + 1 < K) wd[2 * f + 1] = make_float2(v.z, v.w);
                        }
#pragma unroll
                        for (int c = 0; c < CPT; ++c) {
                            const int col = tid + c * NT;
                            if (col < ncol) {
                                float x[VEC];
                                LdsVec<TP>::load(tl + row * row_bytes + (uint32_t)(col * VEC * sizeof(TP)), x);
#pragma unroll
                                for (int q = 0; q < EP; ++q) {
                                    const float2 xp = make_float2(x[2 * q], x[2 * q + 1]);
#pragma unroll
                                    for (int s = 0; s < K; ++s) Q2[c][q][s] = __ffma2_rn(xp, wd[s], Q2[c][q][s]);
                                }
                            }
                        }
                    }
                }
                mbar_arrive(&empty[s_prev]);
            }
            s_prev = s_cur;
            r0_prev = r0_cur;
            r0_cur += rstep;
            if (++s_cur == S) {
                s_cur = 0;
                par_cur ^= 1u;
            }
        }
        if (!ok) report(a.status, FHR_ERR_TIMEOUT);

        // per-CTA partials of Q
        const int g = blockIdx.x;
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int col = tid + c * NT;
            if (col < ncol) {
#pragma unroll
                for (int q = 0; q < EP; ++q)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int k = col * VEC + 2 * q + h;
                        if (k < a.Nk) {
#pragma unroll
                            for (int s = 0; s < K; ++s)
                                a.Qpart[((size_t)g * a.Nk + k) * K + s] = h ? Q2[c][q][s].y : Q2[c][q][s].x;
                        }
                    }
            }
        }
        float ssq = ssq2.x + ssq2.y;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ssq += __shfl_xor_sync(0xffffffffu, ssq, o);
        if (lane == 0) ssqs[warp] = ssq;
    }

    // consumers and the update warp meet once at the end
    bar_sync(1, NT + 32);
    if (warp == NW) {
        for (int i = lane; i < K * K; i += 32) {
            float acc = 0.f;
            for (int r = 0; r < ROWS; ++r) acc += gwacc[r * K * K + i];
            a.Gpart[(size_t)blockIdx.x * K * K + i] = acc;
        }
        if (lane == 0 && a.want_ssq) {
            float acc = 0.f;
            for (int wp = 0; wp < NW; ++wp) acc += ssqs[wp];
            a.ssqpart[blockIdx.x] = acc;
        }
    }
}

}  // namespace fhr
