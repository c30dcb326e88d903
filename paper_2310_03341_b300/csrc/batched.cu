// Batched solve of independent Hermitian blocks of uneven size (the kz
// blocks of a tube geometry, where kz is a good quantum number and the 3-D
// BdG matrix splits into H_kz = H_perp + (kz^2/2) tau_z, tau_z = +1 on u and
// -1 on v; paper, section "Theoretical Framework", on the symmetry-reduced
// problems).
//
// A pool of worker contexts, each with its own workspace arena, stream and
// is driven by one host thread per worker; blocks are taken
// largest first from a shared counter, so the small latency-bound solves of
// different blocks overlap on the device.  The band width of each block size
// is chosen by an autotuner: the first blocks of a size class are solved one
// after the other with each candidate width and timed with CUDA events; the
// fastest width is cached in the calling context for that (precision,
// order) and used for every later block of that size.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <thread>

#include "internal.h"

namespace bdg {

static int env_workers() {
    const char *v = getenv("BDG_BATCH_WORKERS");
    int k = v ? atoi(v) : 6;
    return std::max(1, std::min(k, 16));
}

static int ensure_workers(bdg_ctx *ctx, int k) {
    while ((int)ctx->workers.size() < k) {
        bdg_ctx *wk = nullptr;
        int rc = bdg_create(ctx->device, &wk);
        if (rc) return bdg_fail(ctx, rc, "bdg_heev_batched: worker context creation failed");
        // the workers inherit the tuning knobs of the calling context
        wk->band_fp32 = ctx->band_fp32;
        wk->band_fp64 = ctx->band_fp64;
        wk->bt2_group = ctx->bt2_group;
        wk->use_tc = ctx->use_tc;
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            bdg_destroy(wk);
            return bdg_fail(ctx, BDG_ECUDA, "bdg_heev_batched: stream creation failed");
        }
        ctx->workers.push_back(wk);
        ctx->worker_streams.push_back(s);
    }
    return BDG_OK;
}

void batch_destroy(bdg_ctx *ctx) {
    for (size_t i = 0; i < ctx->workers.size(); ++i) {
        cudaStreamSynchronize(ctx->worker_streams[i]);
        cudaStreamDestroy(ctx->worker_streams[i]);
        bdg_destroy(ctx->workers[i]);
    }
    ctx->workers.clear();
    ctx->worker_streams.clear();
}

// candidate band widths for a block of order n (each must leave n > 2b)
static std::vector<int> band_candidates(int prec, int64_t n) {
    std::vector<int> c;
    const int base[] = {16, 32, 64};
    for (int b : base) {
        if (prec == BDG_PREC_FP64 && b > 32) continue;   // FP64 windows of b = 64 exceed shared memory
        if (n > 4 * b) c.push_back(b);
    }
    return c;
}

}  // namespace bdg

extern "C" int bdg_heev_batched(bdg_ctx *ctx, int nblocks, const int64_t *sizes, double2 *const *A,
                                double *const *w, double2 *const *Z, int prec, cudaStream_t stream) {
    using namespace bdg;
    if (!ctx) return BDG_EINVAL;
    if (nblocks < 0 || (nblocks > 0 && (!sizes || !A || !w || !Z)))
        return bdg_fail(ctx, BDG_EINVAL, "bdg_heev_batched: bad arguments");
    for (int i = 0; i < nblocks; ++i)
        if (sizes[i] < 1 || !A[i] || !w[i] || !Z[i])
            return bdg_fail(ctx, BDG_EINVAL, "bdg_heev_batched: block %d: bad arguments", i);
    if (nblocks == 0) return BDG_OK;
    cudaSetDevice(ctx->device);
    ctx->err[0] = 0;
    const int base_prec = prec & ~BDG_HEEV_PH;
    const int K = std::min(env_workers(), nblocks);
    int rc = ensure_workers(ctx, K);
    if (rc) return rc;
    for (bdg_ctx *wk : ctx->workers) wk->wait_cycles = ctx->wait_cycles;
    // the batch starts after the work already queued on the caller's stream
    cudaEvent_t start_ev;
    BDG_CUDA_TRY(ctx, cudaEventCreateWithFlags(&start_ev, cudaEventDisableTiming));
    BDG_CUDA_TRY(ctx, cudaEventRecord(start_ev, stream));
    for (int k = 0; k < K; ++k) BDG_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->worker_streams[k], start_ev, 0));
    cudaEventDestroy(start_ev);

    // largest first
    std::vector<int> order(nblocks);
    for (int i = 0; i < nblocks; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sizes[a] > sizes[b]; });

    auto solve = [&](int wid, int i, int band) -> int {
        bdg_ctx *wk = ctx->workers[wid];
        wk->band_override = band;
        const int64_t n = sizes[i];
        int r = bdg_heev(wk, n, A[i], n, w[i], Z[i], n, prec, ctx->worker_streams[wid]);
        wk->band_override = 0;
        return r;
    };

    // ---- autotuning pre-pass on worker 0: size classes not seen before
    std::vector<char> done(nblocks, 0);
    {
        size_t pos = 0;
        while (pos < order.size()) {
            const int64_t n = sizes[order[pos]];
            size_t end = pos;
            while (end < order.size() && sizes[order[end]] == n) ++end;
            const auto key = std::make_pair(base_prec, n);
            std::vector<int> cand = band_candidates(base_prec, n);
            if (!ctx->batch_band.count(key) && cand.size() > 1 && end - pos >= cand.size() + 1) {
                float best = 1e30f;
                int best_b = cand[0];
                cudaEvent_t e0, e1;
                BDG_CUDA_TRY(ctx, cudaEventCreate(&e0));
                BDG_CUDA_TRY(ctx, cudaEventCreate(&e1));
                for (size_t c = 0; c < cand.size(); ++c) {
                    const int i = order[pos + c];
                    cudaEventRecord(e0, ctx->worker_streams[0]);
                    int r = solve(0, i, cand[c]);
                    cudaEventRecord(e1, ctx->worker_streams[0]);
                    if (r) {
                        cudaEventDestroy(e0);
                        cudaEventDestroy(e1);
                        return bdg_fail(ctx, r, "bdg_heev_batched: block %d (n=%lld): %s", i, (long long)n,
                                        bdg_last_error(ctx->workers[0]));
                    }
                    cudaEventSynchronize(e1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms < best) { best = ms; best_b = cand[c]; }
                    done[pos + c] = 1;
                }
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                ctx->batch_band[key] = best_b;
            }
            pos = end;
        }
    }

    // ---- concurrent phase
    std::atomic<size_t> next(0);
    std::mutex mu;
    int first_rc = BDG_OK;
    auto worker = [&](int wid) {
        cudaSetDevice(ctx->device);
        for (;;) {
            size_t p = next.fetch_add(1);
            if (p >= order.size()) break;
            if (done[p]) continue;
            {
                std::lock_guard<std::mutex> lk(mu);
                if (first_rc) break;
            }
            const int i = order[p];
            const auto key = std::make_pair(base_prec, sizes[i]);
            int band = 0;
            {
                std::lock_guard<std::mutex> lk(mu);
                auto it = ctx->batch_band.find(key);
                if (it != ctx->batch_band.end()) band = it->second;
            }
            int r = solve(wid, i, band);
            if (r) {
                std::lock_guard<std::mutex> lk(mu);
                if (!first_rc) {
                    first_rc = r;
                    bdg_fail(ctx, r, "bdg_heev_batched: block %d (n=%lld): %s", i, (long long)sizes[i],
                             bdg_last_error(ctx->workers[wid]));
                }
                break;
            }
        }
    };
    std::vector<std::thread> th;
    for (int k = 1; k < K; ++k) th.emplace_back(worker, k);
    worker(0);
    for (auto &t : th) t.join();
    // the caller's stream continues after every block is solved
    for (int k = 0; k < K; ++k) {
        cudaEvent_t ev;
        BDG_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        BDG_CUDA_TRY(ctx, cudaEventRecord(ev, ctx->worker_streams[k]));
        BDG_CUDA_TRY(ctx, cudaStreamWaitEvent(stream, ev, 0));
        cudaEventDestroy(ev);
    }
    return first_rc;
}
