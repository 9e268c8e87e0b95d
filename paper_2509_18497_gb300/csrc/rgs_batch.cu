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
#include <array>
#include <map>
#include <memory>
#include <type_traits>
#include <mutex>
#include <vector>

#include "rgs_bounce_body.cuh"

namespace {

struct BatchSceneDev {
    SceneDev sc;
    RaysDev rays;
    int C, nc, nb, prec;
    // item shape of the levels that gather BF16 rows (16) and FP32 rows (32):
    // 0 = 3-column tiles (4 lanes per ray), 1 = 32-column tiles (lane per column)
    int wide16, wide32;
    int tiles16, tiles32; // column tiles per receiver for each shape
    float *iters, *Q;
    __nv_bfloat16 *iters16;
    long long A, A16;
    double *norm2;
};
static_assert(sizeof(BatchSceneDev) % 4 == 0, "descriptor is copied as 32-bit words");

__device__ __forceinline__ unsigned ld_volatile(const unsigned *p) { return *(const volatile unsigned *)p; }
__device__ __forceinline__ int ld_volatile(const int *p) { return *(const volatile int *)p; }

// one (receiver, column tile) item of bounce b: gathers rows of B^(b-1) (BF16 copies or FP32)
template <int NC, bool ROWS16, bool WIDE>
__device__ __forceinline__ void batch_item(const BatchSceneDev &S, int b, int i, int tile, float *red) {
    const float *Bprev = S.iters + S.A * (b - 1);
    __nv_bfloat16 *Bout16 = S.prec != RGS_FP32 ? S.iters16 + S.A16 * b : nullptr;
    using T = typename std::conditional<ROWS16, __nv_bfloat16, float>::type;
    const T *Bg;
    if constexpr (ROWS16) Bg = S.iters16 + S.A16 * (b - 1);
    else Bg = Bprev;
    if constexpr (WIDE) {
        bounce_receiver_mc<NC, T>(S.sc, S.rays, S.C, Bg, Bprev, S.iters, S.Q + S.A * (b - 1), S.iters + S.A * b,
                                  Bout16, S.norm2 + b, i, tile, red);
    } else {
        using SL = typename std::conditional<ROWS16, SliceH<NC>, Slice<NC>>::type;
        bounce_receiver<NC, 3, SL>(S.sc, S.rays, S.C, Bg, Bprev, S.iters, S.Q + S.A * (b - 1), S.iters + S.A * b,
                                   Bout16, S.norm2 + b, i, tile * 3, red);
    }
}

template <int NC>
__device__ __forceinline__ void batch_item_nc(const BatchSceneDev &S, int b, bool rows16, bool wide, int i, int tile,
                                              float *red) {
    if (wide) {
        if (rows16) batch_item<NC, true, true>(S, b, i, tile, red);
        else batch_item<NC, false, true>(S, b, i, tile, red);
    } else {
        if (rows16) batch_item<NC, true, false>(S, b, i, tile, red);
        else batch_item<NC, false, false>(S, b, i, tile, red);
    }
}

// Levels b0..b1 of every scene.  Items of a level are numbered scene by scene
// (level_off[b][s] .. level_off[b][s+1]) and, within a scene, tile-major: neighbouring
// items are neighbouring receivers (Morton order) of one column tile, whose rays gather
// largely the same source rows (measured faster than receiver-major for the per-scene
// kernels, whose grids use the same order).
template <int MINB>
__global__ void __launch_bounds__(BOUNCE_THREADS, MINB) k_bounce_persistent(const BatchSceneDev *__restrict__ scenes,
                                                                        int count, const long long *__restrict__ level_off,
                                                                        int b0, int b1, int force32,
                                                                        unsigned long long *counters,
                                                                        unsigned *barrier, int spin_limit, int *err) {
    __shared__ float red[MC_WARPS * 16 * 32]; // the larger of the two bodies' scratch
    __shared__ long long s_item;
    __shared__ BatchSceneDev s_scene;
    __shared__ int s_abort;
    for (int b = b0; b <= b1; ++b) {
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
            // the scene's descriptor in shared memory: its fields are read where used instead
            // of being held in registers across the item
            if (threadIdx.x < sizeof(BatchSceneDev) / 4)
                reinterpret_cast<int *>(&s_scene)[threadIdx.x] = reinterpret_cast<const int *>(scenes + s)[threadIdx.x];
            __syncthreads();
            const BatchSceneDev &S = s_scene;
            const bool rows16 =
                !force32 && S.prec != RGS_FP32 && !(S.prec == RGS_BF16_FP32ACC_RESCORR && b == S.nb);
            const bool wide = rows16 ? S.wide16 : S.wide32;
            const long long local = item - off[s];
            const int tile = (int)(local / S.sc.n), i = (int)(local - (long long)tile * S.sc.n);
            switch (S.nc) {
            case 1: batch_item_nc<1>(S, b, rows16, wide, i, tile, red); break;
            case 4: batch_item_nc<4>(S, b, rows16, wide, i, tile, red); break;
            case 9: batch_item_nc<9>(S, b, rows16, wide, i, tile, red); break;
            default: batch_item_nc<16>(S, b, rows16, wide, i, tile, red);
            }
        }
        if (b == b1) break;
        // grid barrier between bounce levels, with a bounded wait
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(barrier, 1u);
            const unsigned target = gridDim.x * (unsigned)(b - b0 + 1);
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
    int minb = 3;           // kernel instance: registers for 2 or 3 resident blocks per SM (autotuned)
    // item-shape policy of the BF16-row and FP32-row levels per bucket of scenes with equal
    // (nc, C, rays per surfel) (autotuned): 0 = 3-column items, 1 = wide_bounce's choice,
    // 2 = 32-column items wherever C >= kWideMinCols
    std::vector<int> bucket;            // per scene
    std::vector<std::array<int, 3>> bkey; // per bucket: nc, C, rays per surfel
    std::vector<int> pol16, pol32;      // per bucket
    bool tuned = false;
    cudaGraphExec_t exec = nullptr;
    bool graph_failed = false;
    ~Plan() {
        if (exec) cudaGraphExecDestroy(exec);
        dev_free(d_scenes);
        dev_free(d_level_off);
        dev_free(d_counters);
        dev_free(d_barrier);
        dev_free(d_err);
    }
};

std::mutex g_plan_mu;
std::map<std::vector<const void *>, Plan *> g_plans;
bool policy_wide(int pol, int C, bool rows16);
std::vector<int32_t> g_last_plan; // the plan of the last rgs_solve_batched call (rgs_batch_last_plan)

void note_plan(const Plan &P) {
    g_last_plan.clear();
    g_last_plan.push_back(P.blocks);
    g_last_plan.push_back(P.minb);
    g_last_plan.push_back(P.tuned ? 1 : 0);
    g_last_plan.push_back((int32_t)P.bkey.size());
    for (size_t k = 0; k < P.bkey.size(); ++k) {
        const int C = P.bkey[k][1];
        g_last_plan.push_back(P.bkey[k][0]);
        g_last_plan.push_back(C);
        g_last_plan.push_back(P.bkey[k][2]);
        g_last_plan.push_back(P.pol16[k]);
        g_last_plan.push_back(P.pol32[k]);
        g_last_plan.push_back(policy_wide(P.pol16[k], C, true) ? 32 : 3);
        g_last_plan.push_back(policy_wide(P.pol32[k], C, false) ? 32 : 3);
    }
}

template <int NC>
void enqueue_make_S(rgs_transport *t, const float *E, cudaStream_t st, bool bf16);

// columns from which policy 2 gives a scene 32-column items
constexpr int kWideMinCols = 6;

bool policy_wide(int pol, int C, bool rows16) {
    return pol == 0 ? false : (pol == 1 ? wide_bounce(C, rows16) : C >= kWideMinCols);
}

// item shapes of every scene under the plan's policies, the level offsets they imply, and
// their upload
rgs_status upload_shape(Plan &P, cudaStream_t st, bool force32 = false) {
    const int count = P.count;
    for (int s = 0; s < count; ++s) {
        BatchSceneDev &b = P.host[s];
        b.wide16 = policy_wide(P.pol16[P.bucket[s]], b.C, true) ? 1 : 0;
        b.wide32 = policy_wide(P.pol32[P.bucket[s]], b.C, false) ? 1 : 0;
        b.tiles16 = b.wide16 ? (b.C + 31) / 32 : b.C / 3;
        b.tiles32 = b.wide32 ? (b.C + 31) / 32 : b.C / 3;
    }
    std::vector<long long> off((size_t)(P.maxnb + 1) * (count + 1), 0);
    for (int b = 1; b <= P.maxnb; ++b)
        for (int s = 0; s < count; ++s) {
            const BatchSceneDev &h = P.host[s];
            const bool rows16 =
                !force32 && h.prec != RGS_FP32 && !(h.prec == RGS_BF16_FP32ACC_RESCORR && b == h.nb);
            const long long items = h.nb >= b ? (long long)h.sc.n * (rows16 ? h.tiles16 : h.tiles32) : 0;
            off[(size_t)b * (count + 1) + s + 1] = off[(size_t)b * (count + 1) + s] + items;
        }
    RGS_CUDA(cudaMemcpyAsync(P.d_scenes, P.host.data(), sizeof(BatchSceneDev) * count, cudaMemcpyHostToDevice, st));
    RGS_CUDA(cudaMemcpyAsync(P.d_level_off, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice, st));
    RGS_CUDA(cudaStreamSynchronize(st)); // the host vectors are released on return
    return RGS_OK;
}

// S = E + D per scene (plain launches, before the graph)
rgs_status enqueue_make_S_all(Plan &P, const std::vector<rgs_transport *> &ts, const float *const *E, cudaStream_t st) {
    for (int s = 0; s < P.count; ++s) {
        rgs_transport *t = ts[s];
        const bool bf16 = P.host[s].prec != RGS_FP32;
        switch (t->nc) {
        case 1: enqueue_make_S<1>(t, E ? E[s] : nullptr, st, bf16); break;
        case 4: enqueue_make_S<4>(t, E ? E[s] : nullptr, st, bf16); break;
        case 9: enqueue_make_S<9>(t, E ? E[s] : nullptr, st, bf16); break;
        default: enqueue_make_S<16>(t, E ? E[s] : nullptr, st, bf16);
        }
    }
    RGS_LAUNCH("batch make_S");
    return RGS_OK;
}

// counter and norm resets and the persistent kernel: the part captured into the graph
rgs_status enqueue_core(Plan &P, const std::vector<rgs_transport *> &ts, int spin_limit, cudaStream_t st,
                        int level0 = 0, int level1 = 0, bool force32 = false) {
    const size_t L = (size_t)(P.maxnb + 1);
    RGS_CUDA(cudaMemsetAsync(P.d_counters, 0, sizeof(unsigned long long) * L, st));
    RGS_CUDA(cudaMemsetAsync(P.d_barrier, 0, sizeof(unsigned), st));
    RGS_CUDA(cudaMemsetAsync(P.d_err, 0, sizeof(int), st));
    for (int s = 0; s < P.count; ++s)
        RGS_CUDA(cudaMemsetAsync(ts[s]->norm2, 0, sizeof(double) * (RGS_MAX_BOUNCES + 1), st));
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
        const int b0 = level0 > 0 ? level0 : 1, b1 = level1 > 0 ? level1 : P.maxnb;
        if (P.minb == 2)
            RGS_CUDA(cudaLaunchKernelEx(&cfg, k_bounce_persistent<2>, (const BatchSceneDev *)P.d_scenes, P.count,
                                        (const long long *)P.d_level_off, b0, b1, force32 ? 1 : 0, P.d_counters, P.d_barrier,
                                        spin_limit, P.d_err));
        else
            RGS_CUDA(cudaLaunchKernelEx(&cfg, k_bounce_persistent<3>, (const BatchSceneDev *)P.d_scenes, P.count,
                                        (const long long *)P.d_level_off, b0, b1, force32 ? 1 : 0, P.d_counters, P.d_barrier,
                                        spin_limit, P.d_err));
    }
    return RGS_OK;
}

// B^(n) of every scene to the caller's layout (plain launches, after the graph)
rgs_status enqueue_outputs(Plan &P, const std::vector<rgs_transport *> &ts, float *const *B_out, cudaStream_t st) {
    for (int s = 0; s < P.count; ++s)
        if (B_out && B_out[s]) {
            rgs_status r = rgs_get_iterate_impl(ts[s], P.host[s].nb, B_out[s], st);
            if (r != RGS_OK) return r;
        }
    return RGS_OK;
}

rgs_status enqueue_batch(Plan &P, const std::vector<rgs_transport *> &ts, const float *const *E, float *const *B_out,
                         int spin_limit, cudaStream_t st) {
    rgs_status r;
    if ((r = enqueue_make_S_all(P, ts, E, st)) != RGS_OK) return r;
    {
        ProfScope ps_("k_bounce_persistent", st);
        if ((r = enqueue_core(P, ts, spin_limit, st)) != RGS_OK) return r;
    }
    return enqueue_outputs(P, ts, B_out, st);
}

// library-owned stream the batch graphs are captured on (capture is not possible on the
// legacy or per-thread default streams a caller may pass); created once per device
cudaStream_t capture_stream() {
    static cudaStream_t streams[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        streams[dev] = nullptr;
    }
    return streams[dev];
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


rgs_status rgs_solve_batched_impl(rgs_transport *const *tsp, int count, const float *const *E, const int32_t *nbs,
                                  const rgs_batch_opts *opts, float *const *B_out, double *norms, cudaStream_t st) {
    const int precision = opts ? opts->precision : RGS_FP32;
    const bool use_graph = opts ? opts->use_graph != 0 : true;
    const bool autotune = opts ? opts->autotune != 0 : true;
    const int spin_limit = (opts && opts->spin_limit > 0) ? opts->spin_limit : (1 << 24);
    std::vector<rgs_transport *> ts(tsp, tsp + count);
    rgs_status r;
    for (int s = 0; s < count; ++s)
        if ((r = rgs_solve_prepare(ts[s], nbs[s], precision, 0, st)) != RGS_OK) return r;

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
    std::unique_ptr<Plan> owner; // a new plan is freed if its set-up fails
    if (fresh) {
        owner.reset(new Plan());
        P = owner.get();
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
            const std::array<int, 3> bk = {t->nc, t->C, t->nd};
            int k = 0;
            while (k < (int)P->bkey.size() && P->bkey[k] != bk) ++k;
            if (k == (int)P->bkey.size()) P->bkey.push_back(bk);
            P->bucket.push_back(k);
        }
        const int nbk = (int)P->bkey.size();
        P->pol16.assign(nbk, 1);
        P->pol32.assign(nbk, 1);
        if ((r = dev_alloc(&P->d_scenes, (size_t)count)) != RGS_OK) return r;
        if ((r = dev_alloc(&P->d_level_off, (size_t)(P->maxnb + 1) * (count + 1))) != RGS_OK) return r;
        if ((r = dev_alloc(&P->d_counters, (size_t)P->maxnb + 1)) != RGS_OK) return r;
        if ((r = dev_alloc(&P->d_barrier, 1)) != RGS_OK) return r;
        if ((r = dev_alloc(&P->d_err, 1)) != RGS_OK) return r;
        int dev = 0, sms = 0, occ2 = 0, occ3 = 0;
        RGS_CUDA(cudaGetDevice(&dev));
        RGS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        RGS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, k_bounce_persistent<2>, BOUNCE_THREADS, 0));
        RGS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ3, k_bounce_persistent<3>, BOUNCE_THREADS, 0));
        if (occ2 < 1 || occ3 < 1) {
            rgs_set_error("rgs_solve_batched: the persistent kernel cannot be resident");
            return RGS_ERR_CUDA;
        }
        auto configure = [&](const std::vector<int> &pol16, const std::vector<int> &pol32, int minb,
                             bool force32) -> rgs_status {
            P->pol16 = pol16;
            P->pol32 = pol32;
            P->minb = minb;
            P->blocks = sms * (minb == 2 ? occ2 : occ3);
            return upload_shape(*P, st, force32);
        };
        const std::vector<int> ones(nbk, 1);
        if ((r = configure(ones, ones, 3, false)) != RGS_OK) return r; // default: the measured crossovers, 3 blocks/SM
        if (autotune && P->maxnb > 0) {
            // Time bounce level 1 per candidate and keep the fastest: first the item-shape policy
            // of the rows level 1 gathers (BF16 in the batched modes) with the kernel occupancy,
            // then, for the residual-corrected mode, the policy of its FP32-row level, timed as
            // level 1 gathering FP32 rows.  S must exist for level 1.
            if ((r = enqueue_make_S_all(*P, ts, E, st)) != RGS_OK) return r;
            cudaEvent_t e0, e1;
            RGS_CUDA(cudaEventCreate(&e0));
            RGS_CUDA(cudaEventCreate(&e1));
            auto time_level1 = [&](const std::vector<int> &pol16, const std::vector<int> &pol32, int minb,
                                   bool force32, float *ms) -> rgs_status {
                rgs_status q;
                if ((q = configure(pol16, pol32, minb, force32)) != RGS_OK) return q;
                RGS_CUDA(cudaEventRecord(e0, st));
                if ((q = enqueue_core(*P, ts, spin_limit, st, 1, 1, force32)) != RGS_OK) return q;
                RGS_CUDA(cudaEventRecord(e1, st));
                RGS_CUDA(cudaEventSynchronize(e1));
                RGS_CUDA(cudaEventElapsedTime(ms, e0, e1));
                return RGS_OK;
            };
            // 1. one policy for every bucket, with the kernel occupancy; 2. each bucket's policy
            // in turn with the others held (coordinate descent, when scenes differ in nc, C or
            // rays per surfel); the level being tuned gathers BF16 rows in the batched modes
            const bool bf16 = precision != RGS_FP32;
            std::vector<int> p16 = ones, p32 = ones;
            std::vector<int> &tuned = bf16 ? p16 : p32;
            float best = 1e30f;
            int best_pol = 1, best_minb = 3;
            for (int pol = 0; pol <= 2 && r == RGS_OK; ++pol)
                for (int minb = 2; minb <= 3 && r == RGS_OK; ++minb) {
                    float ms = 0.f;
                    std::fill(tuned.begin(), tuned.end(), pol);
                    r = time_level1(p16, p32, minb, false, &ms);
                    if (r == RGS_OK && ms < best) {
                        best = ms;
                        best_pol = pol;
                        best_minb = minb;
                    }
                }
            std::fill(tuned.begin(), tuned.end(), best_pol);
            auto refine = [&](std::vector<int> &pols, bool force32, float &cur) {
                if (nbk < 2) return;
                for (int k = 0; k < nbk && r == RGS_OK; ++k) {
                    const int keep = pols[k];
                    for (int pol = 0; pol <= 2 && r == RGS_OK; ++pol) {
                        if (pol == keep) continue;
                        const int prev = pols[k];
                        pols[k] = pol;
                        float ms = 0.f;
                        r = time_level1(p16, p32, best_minb, force32, &ms);
                        if (r == RGS_OK && ms < cur) cur = ms;
                        else pols[k] = prev;
                    }
                }
            };
            refine(tuned, false, best);
            if (r == RGS_OK && precision == RGS_BF16_FP32ACC_RESCORR) {
                // the FP32-row level (the corrected bounce), timed as level 1 gathering FP32 rows
                float best32 = 1e30f;
                int bp32 = 1;
                for (int pol = 0; pol <= 2 && r == RGS_OK; ++pol) {
                    float ms = 0.f;
                    std::fill(p32.begin(), p32.end(), pol);
                    r = time_level1(p16, p32, best_minb, true, &ms);
                    if (r == RGS_OK && ms < best32) {
                        best32 = ms;
                        bp32 = pol;
                    }
                }
                std::fill(p32.begin(), p32.end(), bp32);
                refine(p32, true, best32);
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (r != RGS_OK) return r;
            if ((r = configure(p16, p32, best_minb, false)) != RGS_OK) return r;
            P->tuned = true;
        }
        g_plans[key] = owner.release();
    }
    note_plan(*P);
    bool launched = false;
    if (use_graph && !P->graph_failed) {
        if (!P->exec) { // capture the core once, on the library's own stream
            cudaGraph_t graph = nullptr;
            cudaStream_t cs = capture_stream();
            bool ok = cs && cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                rgs_status er = enqueue_core(*P, ts, spin_limit, cs);
                ok = (cudaStreamEndCapture(cs, &graph) == cudaSuccess) && er == RGS_OK;
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
            if ((r = enqueue_make_S_all(*P, ts, E, st)) != RGS_OK) return r;
            {
                ProfScope ps_("k_bounce_persistent", st); // the graph: resets + the persistent kernel
                RGS_CUDA(cudaGraphLaunch(P->exec, st));
            }
            if ((r = enqueue_outputs(*P, ts, B_out, st)) != RGS_OK) return r;
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
        ts[s]->tc_used = false;
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
    for (auto &kv : g_plans) delete kv.second;
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
            delete it->second;
            it = g_plans.erase(it);
        } else {
            ++it;
        }
    }
}

extern "C" int32_t rgs_batch_last_plan(int32_t *out, int32_t n) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    if (g_last_plan.empty()) return -1;
    if (n > 0 && !out) return -1;
    for (int32_t q = 0; q < n && q < (int32_t)g_last_plan.size(); ++q) out[q] = g_last_plan[q];
    return (int32_t)g_last_plan.size();
}
