// Batched MBIR: every subspace channel and slice of many independent problems
// of uneven size (Eq. recon for each) in ONE persistent cooperative launch,
// replayed from a CUDA graph.  Each iteration is two grid-wide phases over a
// flat list of work items (problem, range of rays / range of pixels):
//   phase F: e = V - A z for every ray of every problem;
//   phase B: the backward gather fused with the SQS update for every pixel;
// separated by grid barriers whose waits are bounded (FHR_ERR_TIMEOUT).
// The tile (rays or pixels per work item, in units of one block-wide sweep)
// is chosen by an autotuner that times the candidates on the actual batch.
#include <math.h>

#include <algorithm>
#include <vector>

#include "mbir.cuh"

namespace fhr {

__global__ void mbir_sigma_kernel(const float *sino, int64_t rows, int K, double *part, unsigned *counter,
                                  float snr_db, int Nc, float T, float p, MbirChan *out);
__global__ void mbir_set_chan(SigmaArgs s, int K, float T, float p, MbirChan *out);
__global__ void fill_kernel(float *x, int64_t n, float v);

struct BatchProb {
    int N, Nc, Nv, Nr, K, Wl;
    int vw;   // values of the channel vector per thread in the gathers
    ProjTables t;
    const float *sino;
    float *e, *buf[4], *dA;
    MbirChan *chan;
};

struct BatchItem {
    int q, start, count;
};

struct BatchArgs {
    const BatchProb *probs;
    const BatchItem *fitems, *bitems;
    int nf, nb, iters, momentum;
    const float *mom;       // [iters] momentum coefficients
    MbirPrior pr;
    unsigned *bar;          // [2]: arrival count, generation
    unsigned *ctr;          // [2 * iters]: next work item of each phase
    int *status;
};

constexpr int kBatchThreads = 256;

// Grid-wide barrier for a co-resident grid; the wait gives up after kWaitLimitNs.
__device__ bool grid_barrier(unsigned *bar, int *status) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned *gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u) + 1u;
        if (arrived == gridDim.x) {
            bar[0] = 0u;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const uint64_t t0 = globaltimer_ns();
            for (uint32_t n = 1; *gen == g; ++n) {
                if ((n & 255u) == 0 && globaltimer_ns() - t0 > kWaitLimitNs) {
                    report(status, FHR_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Values per thread for a problem's Wl (all Wl values of a pixel / ray are
// one contiguous vector): the widest of 4, 2, 1 that is at most the requested
// width (0: no limit) and divides Wl; host and device agree on this split.
// A width that would need more than a block's threads for one vector is widened.
__host__ __device__ inline int batch_vw(int Wl, int req = 0) {
    const int lim = req > 0 ? req : 4;
    int vw = (lim >= 4 && Wl % 4 == 0) ? 4 : ((lim >= 2 && Wl % 2 == 0) ? 2 : 1);
    while (vw < 4 && Wl / vw > kBatchThreads && Wl % (2 * vw) == 0) vw *= 2;
    return vw;
}
__host__ __device__ inline int batch_sweep(int Wl, int vw) { return kBatchThreads / (Wl / vw); }

template <int VW>
__device__ __forceinline__ void batch_forward(const BatchItem &item, const BatchProb &P, const float *z) {
    using VF = VecF<VW>;
    const int CH = P.Wl / VW, sweep = kBatchThreads / CH;
    const int tid = threadIdx.x, ch = tid % CH;
    if (tid >= sweep * CH) return;
    for (int r = tid / CH; r < item.count; r += sweep) {
        const int row = item.start + r;
        typename VF::T axs[1];
        forward_at<VW, 1, true>(z, P.t, P.N, P.Nc, P.Wl, row, ch * VW, VW, axs);
        typename VF::T ax = axs[0];
        const size_t o = (size_t)row * P.Wl + ch * VW;
        const typename VF::T v = VF::ld(P.sino + o);
#pragma unroll
        for (int e = 0; e < VW; ++e) VF::set(ax, e, VF::get(v, e) - VF::get(ax, e));
        VF::st(P.e + o, ax);
    }
}

template <int VW>
__device__ __forceinline__ void batch_update(const BatchItem &item, const BatchProb &P, const float *xprev,
                                             const float *z, float *xnew, float *znext, const MbirPrior &pr,
                                             float mom) {
    const int CH = P.Wl / VW, sweep = kBatchThreads / CH;
    const int tid = threadIdx.x, ch = tid % CH;
    if (tid >= sweep * CH) return;
    for (int r = tid / CH; r < item.count; r += sweep)
        mbir_update_at<VW, 1, true>(P.e, z, xprev, xnew, znext, P.t, P.dA, P.chan, pr, mom, P.N, P.Nc, P.Nv, P.Nr, P.K,
                                    P.Wl, item.start + r, ch * VW, VW);
}

// Next work item of a phase: items are taken in list order (largest first)
// from a per-phase counter, so uneven items balance across the grid.
__device__ __forceinline__ int next_item(unsigned *ctr) {
    __shared__ int idx;
    __syncthreads();
    if (threadIdx.x == 0) idx = (int)atomicAdd(ctr, 1u);
    __syncthreads();
    return idx;
}

__global__ void __launch_bounds__(kBatchThreads, 65536 / (kBatchThreads * 64)) mbir_batch_kernel(BatchArgs a) {
    for (int it = 0; it < a.iters; ++it) {
        const int par = it & 1;
        // ---- phase F: residual e = V - A z
        for (int f = next_item(a.ctr + 2 * it); f < a.nf; f = next_item(a.ctr + 2 * it)) {
            const BatchItem item = a.fitems[f];
            const BatchProb &P = a.probs[item.q];
            const float *z = a.momentum ? P.buf[1 + 2 * par] : P.buf[par];
            const int vw = P.vw;
            if (vw == 4) batch_forward<4>(item, P, z);
            else if (vw == 2) batch_forward<2>(item, P, z);
            else batch_forward<1>(item, P, z);
        }
        if (!grid_barrier(a.bar, a.status)) return;
        // ---- phase B: backward gather + SQS update (+ momentum)
        for (int b = next_item(a.ctr + 2 * it + 1); b < a.nb; b = next_item(a.ctr + 2 * it + 1)) {
            const BatchItem item = a.bitems[b];
            const BatchProb &P = a.probs[item.q];
            float *xprev = nullptr, *z, *xnew, *znext = nullptr;
            if (a.momentum) {
                xprev = P.buf[2 * par];
                z = P.buf[1 + 2 * par];
                xnew = P.buf[2 * (1 - par)];
                znext = P.buf[1 + 2 * (1 - par)];
            } else {
                z = P.buf[par];
                xnew = P.buf[1 - par];
            }
            const int vw = P.vw;
            if (vw == 4) batch_update<4>(item, P, xprev, z, xnew, znext, a.pr, a.mom[it]);
            else if (vw == 2) batch_update<2>(item, P, xprev, z, xnew, znext, a.pr, a.mom[it]);
            else batch_update<1>(item, P, xprev, z, xnew, znext, a.pr, a.mom[it]);
        }
        if (!grid_barrier(a.bar, a.status)) return;
    }
}

// ---------------------------------------------------------------- host
struct BatchWs {
    int *status;
    unsigned *bar;
    unsigned *counter;
    double *sig_part;
    BatchProb *dprobs;
    BatchItem *items;
    float *mom;
    unsigned *ctr;
    char *per;   // per-problem region
};

static size_t prob_bytes(const fhr_problem &q, int K) {
    Carve c(nullptr);
    fhr_geom g{q.N, q.Nr, q.Nc, q.Nv, q.angles};
    const int Wl = q.Nr * K;
    proj_tables_carve(c, g.N, g.Nc, g.Nv, nullptr);
    c.take<MbirChan>(1);
    c.take<float>((size_t)q.N * q.N);                 // dA
    c.take<float>((size_t)q.Nv * q.Nc * Wl);          // e
    for (int i = 0; i < 4; ++i) c.take<float>((size_t)q.N * q.N * Wl);
    return c.size();
}

// rays / pixels per work item; at least one whenever the problem passed check_batch
// (batch_vw widens vw until a vector fits a block)
static int64_t tile_rows(int Wl, int vw, int tile) { return (int64_t)tile * std::max(1, batch_sweep(Wl, vw)); }

static size_t carve_batch(void *base, int nprob, const fhr_problem *probs, const fhr_batch_params *p, int tile,
                          int vw_req, BatchWs *w, std::vector<BatchItem> *fi, std::vector<BatchItem> *bi) {
    Carve c(base);
    BatchWs t{};
    t.status = c.take<int>(kStatusBytes / sizeof(int));
    t.bar = c.take<unsigned>(4);
    t.counter = c.take<unsigned>(4);
    t.sig_part = c.take<double>((size_t)kSigBlocks * 2 * kMbirMaxK);
    t.dprobs = c.take<BatchProb>((size_t)nprob);
    // work items: enough room for the smallest tile (1 sweep at the narrowest width the
    // problem takes: batch_vw(Wl, 1), widened when Wl exceeds a block's threads)
    int64_t nitems = 0;
    for (int q = 0; q < nprob; ++q) {
        const int Wl = probs[q].Nr * probs[q].K;
        const int64_t tr = tile_rows(Wl, batch_vw(Wl, 1), 1);
        nitems += cdiv((int64_t)probs[q].Nv * probs[q].Nc, tr);
        nitems += cdiv((int64_t)probs[q].N * probs[q].N, tr);
    }
    t.items = c.take<BatchItem>((size_t)nitems);
    t.mom = c.take<float>((size_t)std::max(1, p->iters));
    t.ctr = c.take<unsigned>((size_t)2 * std::max(1, p->iters));
    t.per = c.take<char>(0);
    size_t per_total = 0;
    for (int q = 0; q < nprob; ++q) per_total += prob_bytes(probs[q], probs[q].K) + 256;
    c.take<char>(per_total);
    if (w) *w = t;
    if (fi && bi) {
        fi->clear();
        bi->clear();
        for (int q = 0; q < nprob; ++q) {
            const int Wl = probs[q].Nr * probs[q].K;
            const int64_t tr = tile_rows(Wl, batch_vw(Wl, vw_req), tile);
            const int64_t nr = (int64_t)probs[q].Nv * probs[q].Nc, npx = (int64_t)probs[q].N * probs[q].N;
            for (int64_t s = 0; s < nr; s += tr) fi->push_back({q, (int)s, (int)std::min<int64_t>(tr, nr - s)});
            for (int64_t s = 0; s < npx; s += tr) bi->push_back({q, (int)s, (int)std::min<int64_t>(tr, npx - s)});
        }
        // largest items first (work per item ~ block sweeps x gather length x values per thread)
        auto cost = [&](const BatchItem &it, bool fwd) {
            const fhr_problem &b = probs[it.q];
            const int Wl = b.Nr * b.K, vw = batch_vw(Wl, vw_req), sw = batch_sweep(Wl, vw);
            return (int64_t)((it.count + sw - 1) / sw) * (fwd ? b.N : b.Nv + 9) * vw;
        };
        std::stable_sort(fi->begin(), fi->end(),
                         [&](const BatchItem &x, const BatchItem &y) { return cost(x, true) > cost(y, true); });
        std::stable_sort(bi->begin(), bi->end(),
                         [&](const BatchItem &x, const BatchItem &y) { return cost(x, false) > cost(y, false); });
    }
    return c.size();
}

static fhr_status check_batch(fhr_ctx *ctx, int nprob, const fhr_problem *probs, const fhr_batch_params *p) {
    FHR_ARG(nprob >= 1 && probs && p, "need at least one problem and params");
    FHR_ARG(p->iters >= 0, "iters < 0");
    if (p->q != 2.f) return set_error(ctx, FHR_ERR_UNSUPPORTED, "only q = 2 is implemented");
    FHR_ARG(p->p >= 1.f && p->p <= 2.f && p->T > 0.f && p->beta >= 0.f, "bad prior parameters");
    for (int q = 0; q < nprob; ++q) {
        const fhr_problem &b = probs[q];
        FHR_ARG(b.K >= 1 && b.K <= kMbirMaxK, "problem %d: K must be 1..8", q);
        fhr_geom g{b.N, b.Nr, b.Nc, b.Nv, b.angles};
        FHR_TRY(check_geom(ctx, &g, b.Nr * b.K));
        FHR_ARG(b.Nr * b.K / batch_vw(b.Nr * b.K) <= kBatchThreads,
                "problem %d: Nr*K must be <= %d in a batch (<= %d when a multiple of 4)", q, kBatchThreads,
                4 * kBatchThreads);
        FHR_ARG(b.sino && b.xs, "problem %d: null sinogram or volume", q);
        FHR_ARG(aligned(b.sino, 4 * (size_t)batch_vw(b.Nr * b.K)), "problem %d: sinogram not aligned to %d bytes", q,
                4 * batch_vw(b.Nr * b.K));
        FHR_ARG((b.Nr > 1) == (probs[0].Nr > 1), "a batch mixes 2-D and 3-D problems");
        if (b.sigma_v[0] > 0.f && b.sigma_x[0] > 0.f)
            for (int j = 0; j < b.K; ++j)
                FHR_ARG(b.sigma_v[j] > 0.f && b.sigma_x[j] > 0.f, "problem %d: sigmas must be positive", q);
    }
    return FHR_OK;
}

static fhr_status batch_run(fhr_ctx *ctx, int nprob, const fhr_problem *probs, const fhr_batch_params *p, int tile,
                            int vw_req, void *ws, size_t ws_bytes, bool write_back, float *ms_out) {
    FHR_TRY(check_batch(ctx, nprob, probs, p));
    FHR_ARG(ws && aligned(ws, 256), "workspace must be non-null and 256-byte aligned");
    FHR_ARG(tile >= 1 && tile <= 64, "tile must be 1..64");
    FHR_ARG(vw_req == 0 || vw_req == 1 || vw_req == 2 || vw_req == 4, "vw must be 0, 1, 2 or 4");
    BatchWs w;
    std::vector<BatchItem> fi, bi;
    const size_t need = carve_batch(ws, nprob, probs, p, tile, vw_req, &w, &fi, &bi);
    FHR_ARG(ws_bytes >= need, "workspace too small: %zu < %zu bytes", ws_bytes, need);
    {   // the item lists must fit the array carved for them (sized for the smallest tile)
        int64_t cap = 0;
        for (int q = 0; q < nprob; ++q) {
            const int Wl = probs[q].Nr * probs[q].K;
            const int64_t tr = tile_rows(Wl, batch_vw(Wl, 1), 1);
            cap += cdiv((int64_t)probs[q].Nv * probs[q].Nc, tr) + cdiv((int64_t)probs[q].N * probs[q].N, tr);
        }
        if ((int64_t)(fi.size() + bi.size()) > cap)
            return set_error(ctx, FHR_ERR_ARG, "internal: %zu work items for room of %lld", fi.size() + bi.size(),
                             (long long)cap);
    }
    FHR_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    FHR_CUDA(cudaMemsetAsync(w.status, 0, kStatusBytes, st));
    FHR_CUDA(cudaMemsetAsync(w.bar, 0, 4 * sizeof(unsigned), st));
    FHR_CUDA(cudaMemsetAsync(w.ctr, 0, sizeof(unsigned) * 2 * (size_t)std::max(1, p->iters), st));
    FHR_CUDA(cudaMemsetAsync(w.counter, 0, 4 * sizeof(unsigned), st));

    // per-problem set-up: tables, sigmas, A^T A 1, starting point
    std::vector<BatchProb> hp((size_t)nprob);
    MbirPrior pr;
    pr.p = p->p;
    pr.T = p->T;
    pr.e = 2.f - p->p;
    pr.c1 = (2.f - p->p) / p->p;
    pr.beta = p->beta;
    char *cur = w.per;
    for (int q = 0; q < nprob; ++q) {
        const fhr_problem &b = probs[q];
        fhr_geom g{b.N, b.Nr, b.Nc, b.Nv, b.angles};
        BatchProb &P = hp[(size_t)q];
        P.N = b.N; P.Nc = b.Nc; P.Nv = b.Nv; P.Nr = b.Nr; P.K = b.K; P.Wl = b.Nr * b.K;
        P.vw = batch_vw(P.Wl, vw_req);
        Carve c(cur);
        proj_tables_carve(c, g.N, g.Nc, g.Nv, &P.t);
        P.chan = c.take<MbirChan>(1);
        P.dA = c.take<float>((size_t)b.N * b.N);
        P.e = c.take<float>((size_t)b.Nv * b.Nc * P.Wl);
        for (int i = 0; i < 4; ++i) P.buf[i] = c.take<float>((size_t)b.N * b.N * P.Wl);
        P.sino = b.sino;
        cur += round_up(c.size(), 256) + 256;
        FHR_TRY(proj_build_tables(ctx, &g, P.t));
        if (b.sigma_v[0] > 0.f && b.sigma_x[0] > 0.f) {
            SigmaArgs s;
            for (int j = 0; j < kMbirMaxK; ++j) {
                s.sv[j] = j < b.K ? b.sigma_v[j] : 1.f;
                s.sx[j] = j < b.K ? b.sigma_x[j] : 1.f;
            }
            mbir_set_chan<<<1, 32, 0, st>>>(s, b.K, p->T, p->p, P.chan);
        } else {
            mbir_sigma_kernel<<<kSigBlocks, 256, 0, st>>>(b.sino, (int64_t)b.Nv * b.Nc * b.Nr, b.K, w.sig_part, w.counter,
                                                   p->snr_db, b.Nc, p->T, p->p, P.chan);
        }
        FHR_LAUNCHED();
        fill_kernel<<<64, 256, 0, st>>>(P.buf[0], (int64_t)b.N * b.N, 1.f);
        FHR_LAUNCHED();
        FHR_TRY(proj_forward(ctx, &g, P.t, 1, P.buf[0], P.e, nullptr));
        FHR_TRY(proj_backward(ctx, &g, P.t, 1, P.e, P.dA));
        const size_t xb = sizeof(float) * (size_t)b.N * b.N * P.Wl;
        FHR_CUDA(cudaMemcpyAsync(P.buf[0], b.xs, xb, cudaMemcpyDeviceToDevice, st));
        if (p->momentum) FHR_CUDA(cudaMemcpyAsync(P.buf[1], b.xs, xb, cudaMemcpyDeviceToDevice, st));
    }
    // the weights' normalisation depends on the slice count; one batch shares Nr
    const double r2 = 1.0 / sqrt(2.0);
    const double z = 4.0 + 4.0 * r2 + (probs[0].Nr > 1 ? 2.0 : 0.0);
    pr.b_edge = (float)(1.0 / z);
    pr.b_diag = (float)(r2 / z);
    pr.b_slice = (float)(1.0 / z);
    std::vector<float> mom((size_t)std::max(1, p->iters), 0.f);
    double tk = 1.0;
    for (int i = 0; i < p->iters; ++i) {
        const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tk * tk));
        mom[(size_t)i] = p->momentum ? (float)((tk - 1.0) / tn) : 0.f;
        tk = tn;
    }
    // small host tables travel with the stream (pageable copies are staged by the runtime)
    std::vector<BatchItem> items(fi);
    items.insert(items.end(), bi.begin(), bi.end());
    FHR_CUDA(cudaMemcpyAsync(w.dprobs, hp.data(), sizeof(BatchProb) * hp.size(), cudaMemcpyHostToDevice, st));
    FHR_CUDA(cudaMemcpyAsync(w.items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice, st));
    FHR_CUDA(cudaMemcpyAsync(w.mom, mom.data(), sizeof(float) * mom.size(), cudaMemcpyHostToDevice, st));

    if (p->iters > 0) {
        BatchArgs a;
        a.probs = w.dprobs;
        a.fitems = w.items;
        a.nf = (int)fi.size();
        a.bitems = w.items + fi.size();
        a.nb = (int)bi.size();
        a.iters = p->iters;
        a.momentum = p->momentum;
        a.mom = w.mom;
        a.pr = pr;
        a.bar = w.bar;
        a.ctr = w.ctr;
        a.status = w.status;
        int per_sm = 0;
        FHR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mbir_batch_kernel, kBatchThreads, 0));
        if (per_sm < 1) return set_error(ctx, FHR_ERR_UNSUPPORTED, "batch kernel does not fit an SM");
        const int grid = std::min(ctx->sm_count * per_sm, std::max(a.nf, a.nb));
        // one persistent cooperative launch, replayed from a CUDA graph
        cudaGraph_t graph;
        cudaGraphExec_t exec;
        FHR_CUDA(cudaGraphCreate(&graph, 0));
        void *args[] = {&a};
        cudaKernelNodeParams kp{};
        kp.func = (void *)mbir_batch_kernel;
        kp.gridDim = dim3(grid);
        kp.blockDim = dim3(kBatchThreads);
        kp.sharedMemBytes = 0;
        kp.kernelParams = args;
        cudaGraphNode_t node;
        FHR_CUDA(cudaGraphAddKernelNode(&node, graph, nullptr, 0, &kp));
        cudaLaunchAttributeValue coop{};
        coop.cooperative = 1;
        FHR_CUDA(cudaGraphKernelNodeSetAttribute(node, cudaLaunchAttributeCooperative, &coop));
        FHR_CUDA(cudaGraphInstantiate(&exec, graph, 0));
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (ms_out) {
            FHR_CUDA(cudaEventCreate(&e0));
            FHR_CUDA(cudaEventCreate(&e1));
            FHR_CUDA(cudaEventRecord(e0, st));
        }
        FHR_CUDA(cudaGraphLaunch(exec, st));
        ++ctx->launches;
        if (ms_out) {
            FHR_CUDA(cudaEventRecord(e1, st));
            FHR_CUDA(cudaEventSynchronize(e1));
            FHR_CUDA(cudaEventElapsedTime(ms_out, e0, e1));
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
        }
        FHR_CUDA(cudaGraphExecDestroy(exec));
        FHR_CUDA(cudaGraphDestroy(graph));
    }
    if (write_back) {
        const int fin = p->iters & 1;
        for (int q = 0; q < nprob; ++q) {
            const BatchProb &P = hp[(size_t)q];
            const float *src = p->momentum ? P.buf[2 * fin] : P.buf[fin];
            FHR_CUDA(cudaMemcpyAsync(probs[q].xs, src, sizeof(float) * (size_t)P.N * P.N * P.Wl,
                                     cudaMemcpyDeviceToDevice, st));
        }
    }
    return FHR_OK;
}

}  // namespace fhr

using namespace fhr;

extern "C" fhr_status fhr_reconstruct_batch_workspace_size(fhr_ctx *ctx, int nprob, const fhr_problem *probs,
                                                           const fhr_batch_params *p, size_t *bytes) {
    if (!ctx) return FHR_ERR_ARG;
    FHR_TRY(check_batch(ctx, nprob, probs, p));
    FHR_ARG(bytes, "bytes is null");
    *bytes = carve_batch(nullptr, nprob, probs, p, 1, 1, nullptr, nullptr, nullptr);
    return FHR_OK;
}

extern "C" fhr_status fhr_reconstruct_batch(fhr_ctx *ctx, int nprob, const fhr_problem *probs,
                                            const fhr_batch_params *p, void *ws, size_t ws_bytes) {
    if (!ctx) return FHR_ERR_ARG;
    FHR_ARG(p, "params is null");
    return batch_run(ctx, nprob, probs, p, p->tile > 0 ? p->tile : 2, p->vw, ws, ws_bytes, true, nullptr);
}

extern "C" fhr_status fhr_reconstruct_batch_autotune(fhr_ctx *ctx, int nprob, const fhr_problem *probs,
                                                     const fhr_batch_params *p, void *ws, size_t ws_bytes,
                                                     int *best_tile, int *best_vw) {
    if (!ctx) return FHR_ERR_ARG;
    FHR_ARG(p && best_tile && best_vw, "null argument");
    FHR_TRY(check_batch(ctx, nprob, probs, p));
    fhr_batch_params q = *p;
    q.iters = p->iters > 0 ? std::min(p->iters, 4) : 4;
    float best = 1e30f;
    int bt = 2, bv = 0;
    const int tiles[] = {1, 2, 4, 8, 16};
    std::vector<int> prev;   // the per-problem widths of the last width tried
    for (int vw : {4, 2, 1}) {
        std::vector<int> eff((size_t)nprob);
        for (int k = 0; k < nprob; ++k) eff[(size_t)k] = batch_vw(probs[k].Nr * probs[k].K, vw);
        if (eff == prev) continue;   // no problem takes this width: same shapes as the last
        prev = eff;
        for (int t : tiles) {
            float ms = 0.f;
            FHR_TRY(batch_run(ctx, nprob, probs, &q, t, vw, ws, ws_bytes, false, &ms));
            if (ms < best) {
                best = ms;
                bt = t;
                bv = vw;
            }
        }
    }
    *best_tile = bt;
    *best_vw = bv;
    return FHR_OK;
}
