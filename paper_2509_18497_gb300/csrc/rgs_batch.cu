// rgs_solve_batched: many traced scenes of uneven size (surfel count, SH degree, rays per
// surfel, bounce count) solved together.
//
// The direct terms are formed per scene; then every bounce of every scene runs in ONE
// persistent kernel.  Its blocks take work items (scene, receiver, 3-column tile) from a
// queue per bounce level: level b holds the items of every scene that runs at least b
// bounces, so small scenes fill the gaps of large ones.  Between levels the blocks meet at
// a grid barrier (the launch is cooperative, so all blocks are resident); every wait is
// bounded and a wait that runs out sets an error flag (RGS_ERR_TIMEOUT) and ends the
// kernel instead of hanging.  The launches of a batch are captured once into a CUDA graph
// and replayed on later calls with the same arguments; the number of resident blocks per
// SM is chosen by timing the candidates on the first call (autotuning).
#include <map>
#include <mutex>
#include <vector>

#include "rgs_bounce_body.cuh"

namespace {

struct BatchSceneDev {
    SceneDev sc;
    RaysDev rays;
    int C, nc, nb, prec;
    float *iters, *Q;
    __nv_bfloat16 *iters16;
    long long A, A16;
    double *norm2;
};

__device__ __forceinline__ unsigned ld_volatile(const unsigned *p) { return *(const volatile unsigned *)p; }
__device__ __forceinline__ int ld_volatile(const int *p) { return *(const volatile int *)p; }

template <int NC, class SL>
__device__ __forceinline__ void batch_item(const BatchSceneDev &S, int b, int i, int col0, float *red) {
    const bool rows16 = S.prec != RGS_FP32 && !(S.prec == RGS_BF16_FP32ACC_RESCORR && b == S.nb);
    const float *Bprev = S.iters + S.A * (b - 1);
    __nv_bfloat16 *Bout16 = S.prec != RGS_FP32 ? S.iters16 + S.A16 * b : nullptr;
    if constexpr (sizeof(typename SL::T) == 2) {
        (void)rows16;
        bounce_receiver<NC, 3, SL>(S.sc, S.rays, S.C, S.iters16 + S.A16 * (b - 1), Bprev, S.iters, S.Q + S.A * (b - 1),
                                   S.iters + S.A * b, Bout16, S.norm2 + b, i, col0, red);
    } else {
        bounce_receiver<NC, 3, SL>(S.sc, S.rays, S.C, Bprev, Bprev, S.iters, S.Q + S.A * (b - 1), S.iters + S.A * b,
                                   Bout16, S.norm2 + b, i, col0, red);
    }
}

__global__ void __launch_bounds__(BOUNCE_THREADS) k_bounce_persistent(const BatchSceneDev *__restrict__ scenes,
                                                                     int count, const long long *__restrict__ level_off,
                                                                     int maxnb, unsigned long long *counters,
                                                                     unsigned *barrier, int spin_limit, int *err) {
    __shared__ float red[(BOUNCE_THREADS / 32) * 4 * 4 * 3]; // largest G * KPL * CT (nc = 16)
    __shared__ long long s_item;
    __shared__ int s_abort;
    for (int b = 1; b <= maxnb; ++b) {
        const long long *off = level_off + (size_t)b * (count + 1);
        const long long total = off[count];
        while (true) {
            if (threadIdx.x == 0) s_item = (long long)atomicAdd(&counters[b], 1ull);
            __syncthreads();
            const long long item = s_item;
            __syncthreads();
            if (item >= total) break;
            int s = 0;
            while (s + 1 < count && off[s + 1] <= item) ++s;
            const BatchSceneDev &S = scenes[s];
            const long long local = item - off[s];
            const int T = S.C / 3;
            const int i = (int)(local / T), col0 = (int)(local % T) * 3;
            const bool rows16 = S.prec != RGS_FP32 && !(S.prec == RGS_BF16_FP32ACC_RESCORR && b == S.nb);
            switch (S.nc) {
            case 1: rows16 ? batch_item<1, SliceH<1>>(S, b, i, col0, red) : batch_item<1, Slice<1>>(S, b, i, col0, red); break;
            case 4: rows16 ? batch_item<4, SliceH<4>>(S, b, i, col0, red) : batch_item<4, Slice<4>>(S, b, i, col0, red); break;
            case 9: rows16 ? batch_item<9, SliceH<9>>(S, b, i, col0, red) : batch_item<9, Slice<9>>(S, b, i, col0, red); break;
            default: rows16 ? batch_item<16, SliceH<16>>(S, b, i, col0, red) : batch_item<16, Slice<16>>(S, b, i, col0, red);
            }
        }
        if (b == maxnb) break;
        // grid barrier between bounce levels, with a bounded wait
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(barrier, 1u);
            const unsigned target = gridDim.x * (unsigned)b;
            bool ok = true;
            int polls = 0;
            while (ld_volatile(barrier) < target) {
                if (++polls >= spin_limit || ld_volatile(err)) {
                    ok = false;
                    break;
                }
                __nanosleep(128);
            }
            if (!ok) atomicExch(err, 1);
            __threadfence();
            s_abort = (!ok || ld_volatile(err)) ? 1 : 0;
        }
        __syncthreads();
        if (s_abort) return;
    }
}

// ------------------------------------------------------------------ host side
struct Plan {
    std::vector<BatchSceneDev> host;
    BatchSceneDev *d_scenes = nullptr;
    long long *d_level_off = nullptr;
    unsigned long long *d_counters = nullptr;
    unsigned *d_barrier = nullptr;
    int *d_err = nullptr;
    int maxnb = 0, count = 0;
    int blocks = 0;         // persistent grid size (autotuned)
    cudaGraphExec_t exec = nullptr;
    bool graph_failed = false;
};

std::mutex g_plan_mu;
std::map<std::vector<const void *>, Plan *> g_plans;

template <int NC>
void enqueue_make_S(rgs_transport *t, const float *E, cudaStream_t st, bool bf16);

rgs_status enqueue_batch(Plan &P, const std::vector<rgs_transport *> &ts, const float *const *E, float *const *B_out,
                         int spin_limit, cudaStream_t st) {
    const size_t L = (size_t)(P.maxnb + 1);
    RGS_CUDA(cudaMemsetAsync(P.d_counters, 0, sizeof(unsigned long long) * L, st));
    RGS_CUDA(cudaMemsetAsync(P.d_barrier, 0, sizeof(unsigned), st));
    RGS_CUDA(cudaMemsetAsync(P.d_err, 0, sizeof(int), st));
    for (int s = 0; s < P.count; ++s) {
        rgs_transport *t = ts[s];
        RGS_CUDA(cudaMemsetAsync(t->norm2, 0, sizeof(double) * (RGS_MAX_BOUNCES + 1), st));
        const bool bf16 = P.host[s].prec != RGS_FP32;
        switch (t->nc) {
        case 1: enqueue_make_S<1>(t, E ? E[s] : nullptr, st, bf16); break;
        case 4: enqueue_make_S<4>(t, E ? E[s] : nullptr, st, bf16); break;
        case 9: enqueue_make_S<9>(t, E ? E[s] : nullptr, st, bf16); break;
        default: enqueue_make_S<16>(t, E ? E[s] : nullptr, st, bf16);
        }
    }
    RGS_LAUNCH("batch make_S");
    if (P.maxnb > 0) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(P.blocks);
        cfg.blockDim = dim3(BOUNCE_THREADS);
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        ProfScope ps_("k_bounce_persistent", st);
        RGS_CUDA(cudaLaunchKernelEx(&cfg, k_bounce_persistent, (const BatchSceneDev *)P.d_scenes, P.count,
                                    (const long long *)P.d_level_off, P.maxnb, P.d_counters, P.d_barrier, spin_limit,
                                    P.d_err));
    }
    for (int s = 0; s < P.count; ++s)
        if (B_out && B_out[s]) {
            rgs_status r = rgs_get_iterate_impl(ts[s], P.host[s].nb, B_out[s], st);
            if (r != RGS_OK) return r;
        }
    return RGS_OK;
}

} // namespace

namespace {
template <int NC> __global__ void k_make_S_b(int n, int C, const int *__restrict__ uid, const float *__restrict__ E,
                                             const float *__restrict__ D, float *S, __nv_bfloat16 *S16) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * C * NC) return;
    const int k = (int)(idx % NC);
    const size_t ic = idx / NC;
    const int c = (int)(ic % C);
    const int i = (int)(ic / C);
    const float e = E ? E[((size_t)uid[i] * NC + k) * 3 + (c % 3)] : 0.f;
    const float v = e + D[idx];
    S[idx] = v;
    if (S16) S16[ic * bf16_stride<NC>() + k] = __float2bfloat16_rn(v);
}
template <int NC> void enqueue_make_S(rgs_transport *t, const float *E, cudaStream_t st, bool bf16) {
    const size_t tot = t->arr();
    ProfScope ps_("k_make_S", st);
    k_make_S_b<NC><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(t->n, t->C, t->sc->uid, E, t->D, t->iters,
                                                                  bf16 ? t->iters16 : nullptr);
}
} // namespace

rgs_status rgs_solve_prepare(rgs_transport *t, int nb, int precision, cudaStream_t st);

rgs_status rgs_solve_batched_impl(rgs_transport *const *tsp, int count, const float *const *E, const int32_t *nbs,
                                  const rgs_batch_opts *opts, float *const *B_out, double *norms, cudaStream_t st) {
    const int precision = opts ? opts->precision : RGS_FP32;
    const bool use_graph = opts ? opts->use_graph != 0 : true;
    const bool autotune = opts ? opts->autotune != 0 : true;
    const int spin_limit = (opts && opts->spin_limit > 0) ? opts->spin_limit : (1 << 24);
    std::vector<rgs_transport *> ts(tsp, tsp + count);
    rgs_status r;
    for (int s = 0; s < count; ++s)
        if ((r = rgs_solve_prepare(ts[s], nbs[s], precision, st)) != RGS_OK) return r;

    // plan: keyed by every pointer and size the launches bake in
    std::vector<const void *> key;
    key.push_back((const void *)(size_t)precision);
    key.push_back((const void *)(size_t)spin_limit);
    for (int s = 0; s < count; ++s) {
        key.push_back(ts[s]);
        key.push_back((const void *)(size_t)ts[s]->n);
        key.push_back((const void *)(size_t)ts[s]->nd);
        key.push_back((const void *)(size_t)ts[s]->C);
        key.push_back(ts[s]->sc->P);
        key.push_back(ts[s]->sc->nodes);
        key.push_back(ts[s]->off);
        key.push_back(ts[s]->dir);
        key.push_back(ts[s]->Q);
        key.push_back(ts[s]->iters);
        key.push_back(ts[s]->iters16);
        key.push_back(ts[s]->rec_ja);
        key.push_back((const void *)(size_t)nbs[s]);
        key.push_back(E ? E[s] : nullptr);
        key.push_back(B_out ? B_out[s] : nullptr);
    }
    std::lock_guard<std::mutex> lk(g_plan_mu);
    Plan *P = g_plans.count(key) ? g_plans[key] : nullptr;
    const bool fresh = (P == nullptr);
    if (fresh) {
        P = new Plan();
        P->count = count;
        for (int s = 0; s < count; ++s) P->maxnb = std::max(P->maxnb, (int)nbs[s]);
        for (int s = 0; s < count; ++s) {
            rgs_transport *t = ts[s];
            BatchSceneDev b;
            b.sc = t->sc->dev();
            b.rays = t->rays();
            b.C = t->C;
            b.nc = t->nc;
            b.nb = nbs[s];
            b.prec = precision;
            b.iters = t->iters;
            b.Q = t->Q;
            b.iters16 = t->iters16;
            b.A = (long long)t->arr();
            b.A16 = (long long)t->n * t->C * (t->nc >= 9 ? 16 : t->nc);
            b.norm2 = t->norm2;
            P->host.push_back(b);
        }
        std::vector<long long> off((size_t)(P->maxnb + 1) * (count + 1), 0);
        for (int b = 1; b <= P->maxnb; ++b)
            for (int s = 0; s < count; ++s)
                off[(size_t)b * (count + 1) + s + 1] =
                    off[(size_t)b * (count + 1) + s] + (nbs[s] >= b ? (long long)ts[s]->n * (ts[s]->C / 3) : 0);
        if ((r = dev_alloc(&P->d_scenes, (size_t)count)) != RGS_OK) return r;
        if ((r = dev_alloc(&P->d_level_off, off.size())) != RGS_OK) return r;
        if ((r = dev_alloc(&P->d_counters, (size_t)P->maxnb + 1)) != RGS_OK) return r;
        if ((r = dev_alloc(&P->d_barrier, 1)) != RGS_OK) return r;
        if ((r = dev_alloc(&P->d_err, 1)) != RGS_OK) return r;
        RGS_CUDA(cudaMemcpyAsync(P->d_scenes, P->host.data(), sizeof(BatchSceneDev) * count, cudaMemcpyHostToDevice, st));
        RGS_CUDA(cudaMemcpyAsync(P->d_level_off, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice, st));
        // resident blocks per SM: the occupancy limit, or the fastest of the candidates
        int dev = 0, sms = 0, occ = 0;
        RGS_CUDA(cudaGetDevice(&dev));
        RGS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        RGS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bounce_persistent, BOUNCE_THREADS, 0));
        if (occ < 1) {
            rgs_set_error("rgs_solve_batched: the persistent kernel cannot be resident");
            return RGS_ERR_CUDA;
        }
        P->blocks = sms * occ;
        if (autotune && P->maxnb > 0 && occ > 1) {
            cudaEvent_t e0, e1;
            RGS_CUDA(cudaEventCreate(&e0));
            RGS_CUDA(cudaEventCreate(&e1));
            float best = 1e30f;
            int best_blocks = P->blocks;
            for (int per = occ; per >= 1; per = (per > 2 ? per / 2 : per - 1)) {
                P->blocks = sms * per;
                RGS_CUDA(cudaEventRecord(e0, st));
                if ((r = enqueue_batch(*P, ts, E, B_out, spin_limit, st)) != RGS_OK) return r;
                RGS_CUDA(cudaEventRecord(e1, st));
                RGS_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                RGS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) {
                    best = ms;
                    best_blocks = P->blocks;
                }
            }
            P->blocks = best_blocks;
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
        }
        g_plans[key] = P;
    }
    bool launched = false;
    if (use_graph && !P->graph_failed) {
        if (!P->exec) {
            cudaGraph_t graph = nullptr;
            cudaStreamCaptureStatus cs;
            bool ok = cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone &&
                      cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                rgs_status er = enqueue_batch(*P, ts, E, B_out, spin_limit, st);
                ok = (cudaStreamEndCapture(st, &graph) == cudaSuccess) && er == RGS_OK;
                ok = ok && cudaGraphInstantiate(&P->exec, graph, 0) == cudaSuccess;
                if (graph) cudaGraphDestroy(graph);
            }
            if (!ok) { // capture not possible here: launch directly from now on
                cudaGetLastError();
                P->graph_failed = true;
                P->exec = nullptr;
            }
        }
        if (P->exec) {
            ProfScope ps_("batch_graph", st);
            RGS_CUDA(cudaGraphLaunch(P->exec, st));
            launched = true;
        }
    }
    if (!launched && (r = enqueue_batch(*P, ts, E, B_out, spin_limit, st)) != RGS_OK) return r;
    // device-side timeouts are reported after the batch
    int err = 0;
    RGS_CUDA(cudaMemcpyAsync(&err, P->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (norms) {
        for (int s = 0; s < count; ++s) {
            double nrm[RGS_MAX_BOUNCES + 1];
            RGS_CUDA(cudaMemcpyAsync(nrm, ts[s]->norm2, sizeof nrm, cudaMemcpyDeviceToHost, st));
            RGS_CUDA(cudaStreamSynchronize(st));
            for (int b = 0; b < RGS_MAX_BOUNCES; ++b)
                norms[(size_t)s * RGS_MAX_BOUNCES + b] = b < nbs[s] ? sqrt(nrm[b + 1]) : 0.0;
        }
    }
    RGS_CUDA(cudaStreamSynchronize(st));
    for (int s = 0; s < count; ++s) {
        ts[s]->nb_last = err ? -1 : nbs[s];
        ts[s]->prec_last = precision;
    }
    if (err) {
        rgs_set_error("rgs_solve_batched: a bounded wait of the inter-bounce grid barrier ran out (limit %d polls)",
                      spin_limit);
        return RGS_ERR_TIMEOUT;
    }
    return RGS_OK;
}

void rgs_batch_plans_release(void) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    for (auto &kv : g_plans) {
        Plan *P = kv.second;
        if (P->exec) cudaGraphExecDestroy(P->exec);
        dev_free(P->d_scenes);
        dev_free(P->d_level_off);
        dev_free(P->d_counters);
        dev_free(P->d_barrier);
        dev_free(P->d_err);
        delete P;
    }
    g_plans.clear();
}

// drops every cached batch plan that refers to transport t (called when t is destroyed)
void rgs_batch_forget(const rgs_transport *t) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    for (auto it = g_plans.begin(); it != g_plans.end();) {
        bool uses = false;
        for (const void *k : it->first)
            if (k == (const void *)t) uses = true;
        if (uses) {
            Plan *P = it->second;
            if (P->exec) cudaGraphExecDestroy(P->exec);
            dev_free(P->d_scenes);
            dev_free(P->d_level_off);
            dev_free(P->d_counters);
            dev_free(P->d_barrier);
            dev_free(P->d_err);
            delete P;
            it = g_plans.erase(it);
        } else {
            ++it;
        }
    }
}
