// Signal-to-noise ratios of the reconstructions, Eq. (snr_fhr) and Eq.
// (snr_fmd) (Sec. V-B), over user regions of interest.
//
// The regions are small next to the volume, so the voxels they hold are first
// listed in voxel order (a count per segment, an ordered scan, then an ordered
// write), and only their rows of x are read.  The sums per (region, channel)
// are FP64 and taken in one fixed order (list segments in turn, voxels in
// order inside each), so the result does not depend on the launch.
#include <math.h>

#include "common.cuh"

namespace fhr {

constexpr int kSnrSeg = 16384;        // voxels per compaction segment (one block of 1024 threads)
constexpr int kSnrListSegs = 64;      // segments of the region list in the sums
constexpr int kSnrChan = 128;         // channels per block in the sums
constexpr int kSnrMaxRegions = 16;
constexpr int kRoiBackground = FHR_ROI_BACKGROUND;

__global__ void __launch_bounds__(1024) snr_count(const uint8_t *__restrict__ roi, int64_t Nx, int Nm,
                                                  int *__restrict__ cnt) {
    __shared__ int wsum[32];
    const int64_t a = (int64_t)blockIdx.x * kSnrSeg;
    int c = 0;
    for (int i = threadIdx.x; i < kSnrSeg; i += blockDim.x) {
        const int64_t n = a + i;
        if (n < Nx) {
            const int r = roi[n];
            c += (r == kRoiBackground || (r >= 1 && r <= Nm)) ? 1 : 0;
        }
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
        cnt[blockIdx.x] = t;
    }
}

// exclusive scan of the per-segment counts (one block; chunk sums then offsets)
__global__ void __launch_bounds__(1024) snr_scan(const int *__restrict__ cnt, int nseg, int *__restrict__ off,
                                                 int *__restrict__ total) {
    __shared__ int part[1024];
    const int per = (nseg + blockDim.x - 1) / blockDim.x;
    const int a = threadIdx.x * per, b = min(nseg, a + per);
    int s = 0;
    for (int i = a; i < b; ++i) s += cnt[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const int v = part[t];
            part[t] = run;
            run += v;
        }
        *total = run;
    }
    __syncthreads();
    int run = part[threadIdx.x];
    for (int i = a; i < b; ++i) {
        off[i] = run;
        run += cnt[i];
    }
}

// the region voxels of each segment, in voxel order, at the segment's offset
__global__ void __launch_bounds__(1024) snr_write(const uint8_t *__restrict__ roi, int64_t Nx, int Nm,
                                                  const int *__restrict__ off, int *__restrict__ list,
                                                  uint8_t *__restrict__ lab) {
    __shared__ int wcount[32];
    __shared__ int base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) base = off[blockIdx.x];
    __syncthreads();
    const int64_t a = (int64_t)blockIdx.x * kSnrSeg;
    for (int i0 = 0; i0 < kSnrSeg; i0 += blockDim.x) {
        const int64_t n = a + i0 + threadIdx.x;
        int r = 0;
        bool in = false;
        if (i0 + (int)threadIdx.x < kSnrSeg && n < Nx) {
            r = roi[n];
            in = r == kRoiBackground || (r >= 1 && r <= Nm);
        }
        const unsigned m = __ballot_sync(0xffffffffu, in);
        if (lane == 0) wcount[warp] = __popc(m);
        __syncthreads();
        int before = base;
        for (int w = 0; w < warp; ++w) before += wcount[w];
        if (in) {
            const int at = before + __popc(m & ((1u << lane) - 1u));
            list[at] = (int)n;
            lab[at] = (uint8_t)r;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int w = 0; w < nw; ++w) t += wcount[w];
            base += t;
        }
        __syncthreads();
    }
}

// per (list segment, region or background, channel): FP64 sums of x, and of x^2
// over the background; thread = channel, every thread of a block walks the same
// voxel, so the branch on its label is uniform
__global__ void __launch_bounds__(kSnrChan) snr_sums(const float *__restrict__ x, int C, const int *__restrict__ list,
                                                     const uint8_t *__restrict__ lab, const int *__restrict__ total,
                                                     int Nm, double *__restrict__ part,
                                                     long long *__restrict__ pcnt) {
    const int c = blockIdx.x * kSnrChan + threadIdx.x;
    const int seg = blockIdx.y;
    const int tot = *total;
    const int a = (int)((int64_t)tot * seg / kSnrListSegs), b = (int)((int64_t)tot * (seg + 1) / kSnrListSegs);
    double s[kSnrMaxRegions], bs = 0.0, bq = 0.0;
    long long n[kSnrMaxRegions + 1];
#pragma unroll
    for (int r = 0; r < kSnrMaxRegions; ++r) {
        s[r] = 0.0;
        n[r] = 0;
    }
    n[kSnrMaxRegions] = 0;
    for (int i = a; i < b; ++i) {
        const int r = lab[i];
        const float v = c < C ? x[(size_t)list[i] * C + c] : 0.f;
        if (r == kRoiBackground) {
            bs += (double)v;
            bq = fma((double)v, (double)v, bq);
            ++n[kSnrMaxRegions];
        } else {
#pragma unroll
            for (int q = 0; q < kSnrMaxRegions; ++q)
                if (q == r - 1) {
                    s[q] += (double)v;
                    ++n[q];
                }
        }
    }
    if (c < C) {
        const size_t stride = (size_t)(Nm + 2) * C;
        double *o = part + (size_t)seg * stride;
        for (int r = 0; r < Nm; ++r) o[(size_t)r * C + c] = s[r];
        o[(size_t)Nm * C + c] = bs;
        o[(size_t)(Nm + 1) * C + c] = bq;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int r = 0; r < Nm; ++r) pcnt[(size_t)seg * (Nm + 1) + r] = n[r];
        pcnt[(size_t)seg * (Nm + 1) + Nm] = n[kSnrMaxRegions];
    }
}

// means, background deviations and the average of the (mean / deviation)^2 terms
__global__ void __launch_bounds__(256) snr_finish(const double *__restrict__ part, const long long *__restrict__ pcnt,
                                                  int C, int Nm, int mode, double *__restrict__ out,
                                                  int *__restrict__ status) {
    __shared__ double red[256];
    __shared__ long long cnt[kSnrMaxRegions + 1];
    if (threadIdx.x <= Nm) {
        long long t = 0;
        for (int seg = 0; seg < kSnrListSegs; ++seg) t += pcnt[(size_t)seg * (Nm + 1) + threadIdx.x];
        cnt[threadIdx.x] = t;
    }
    __syncthreads();
    bool empty = false;
    for (int r = 0; r <= Nm; ++r) empty |= cnt[r] == 0;
    if (empty) {
        if (threadIdx.x == 0) {
            report(status, FHR_ERR_ARG);
            *out = nan("");
        }
        return;
    }
    const size_t stride = (size_t)(Nm + 2) * C;
    const double nb = (double)cnt[Nm];
    double acc = 0.0;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        double bs = 0.0, bq = 0.0;
        for (int seg = 0; seg < kSnrListSegs; ++seg) {
            bs += part[seg * stride + (size_t)Nm * C + c];
            bq += part[seg * stride + (size_t)(Nm + 1) * C + c];
        }
        const double bm = bs / nb;
        const double sd = sqrt(fmax(bq / nb - bm * bm, 0.0));
        for (int m = 0; m < Nm; ++m) {
            if (mode == FHR_SNR_FMD && c != m) continue;
            double s = 0.0;
            for (int seg = 0; seg < kSnrListSegs; ++seg) s += part[seg * stride + (size_t)m * C + c];
            const double q = (s / (double)cnt[m]) / sd;
            acc = fma(q, q, acc);
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double terms = mode == FHR_SNR_FMD ? (double)Nm : (double)Nm * (double)C;
        const double v = 10.0 * log10(red[0] / terms);
        if (!isfinite(v)) report(status, FHR_ERR_NONFINITE);
        *out = v;
    }
}

struct SnrWs {
    int *status, *cnt, *off, *total, *list;
    uint8_t *lab;
    double *part;
    long long *pcnt;
};

static size_t carve_snr(void *base, int64_t Nx, int C, int Nm, SnrWs *w) {
    Carve c(base);
    SnrWs t;
    const int64_t nseg = cdiv(Nx, kSnrSeg);
    t.status = c.take<int>(kStatusBytes / sizeof(int));
    t.cnt = c.take<int>((size_t)nseg);
    t.off = c.take<int>((size_t)nseg);
    t.total = c.take<int>(1);
    t.list = c.take<int>((size_t)Nx);
    t.lab = c.take<uint8_t>((size_t)Nx);
    t.part = c.take<double>((size_t)kSnrListSegs * (Nm + 2) * C);
    t.pcnt = c.take<long long>((size_t)kSnrListSegs * (Nm + 1));
    if (w) *w = t;
    return c.size();
}

static fhr_status check_snr(fhr_ctx *ctx, int64_t Nx, int C, int Nm, int mode) {
    FHR_ARG(Nx >= 1 && Nx < ((int64_t)1 << 31), "Nx must be 1..2^31-1");
    FHR_ARG(C >= 1 && C <= (1 << 20), "C must be 1..2^20");
    FHR_ARG(Nm >= 1 && Nm <= kSnrMaxRegions, "Nm must be 1..16");
    FHR_ARG(mode == FHR_SNR_FMD || mode == FHR_SNR_FHR, "mode must be FHR_SNR_FMD or FHR_SNR_FHR");
    FHR_ARG(mode != FHR_SNR_FMD || C >= Nm, "Eq. snr_fmd reads channel m of region m: C >= Nm");
    return FHR_OK;
}

}  // namespace fhr

using namespace fhr;

extern "C" fhr_status fhr_snr_workspace_size(fhr_ctx *ctx, int64_t Nx, int C, int Nm, int mode, size_t *bytes) {
    if (!ctx) return FHR_ERR_ARG;
    FHR_TRY(check_snr(ctx, Nx, C, Nm, mode));
    FHR_ARG(bytes, "bytes is null");
    *bytes = carve_snr(nullptr, Nx, C, Nm, nullptr);
    return FHR_OK;
}

extern "C" fhr_status fhr_snr(fhr_ctx *ctx, int64_t Nx, int C, int Nm, int mode, const float *x, const uint8_t *roi,
                              double *snr_db, void *ws, size_t ws_bytes) {
    if (!ctx) return FHR_ERR_ARG;
    FHR_TRY(check_snr(ctx, Nx, C, Nm, mode));
    FHR_ARG(x && roi && snr_db && ws, "null pointer argument");
    FHR_ARG(aligned(ws, 256), "workspace must be 256-byte aligned");
    SnrWs w;
    const size_t need = carve_snr(ws, Nx, C, Nm, &w);
    FHR_ARG(ws_bytes >= need, "workspace too small: %zu < %zu bytes", ws_bytes, need);
    FHR_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    FHR_CUDA(cudaMemsetAsync(w.status, 0, kStatusBytes, st));
    const int nseg = (int)cdiv(Nx, kSnrSeg);
    snr_count<<<nseg, 1024, 0, st>>>(roi, Nx, Nm, w.cnt);
    FHR_LAUNCHED();
    snr_scan<<<1, 1024, 0, st>>>(w.cnt, nseg, w.off, w.total);
    FHR_LAUNCHED();
    snr_write<<<nseg, 1024, 0, st>>>(roi, Nx, Nm, w.off, w.list, w.lab);
    FHR_LAUNCHED();
    snr_sums<<<dim3((unsigned)cdiv(C, kSnrChan), kSnrListSegs), kSnrChan, 0, st>>>(x, C, w.list, w.lab, w.total, Nm,
                                                                                   w.part, w.pcnt);
    FHR_LAUNCHED();
    snr_finish<<<1, 256, 0, st>>>(w.part, w.pcnt, C, Nm, mode, snr_db, w.status);
    FHR_LAUNCHED();
    return FHR_OK;
}
