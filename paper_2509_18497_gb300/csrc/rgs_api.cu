// C ABI entry points of librgs (declared in include/rgs.h): argument checks, handle
// lifetime and error reporting.  The GPU work lives in rgs_scene.cu, rgs_trace.cu,
// rgs_solve.cu and rgs_adjoint.cu.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "rgs_internal.cuh"

static thread_local char g_err[512] = "";

void rgs_set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

rgs_status rgs_cuda_fail(cudaError_t e, const char *what) {
    rgs_set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    cudaGetLastError(); // clear a sticky launch error where possible
    return e == cudaErrorMemoryAllocation ? RGS_ERR_OOM : RGS_ERR_CUDA;
}

static cudaStream_t S(void *stream) { return reinterpret_cast<cudaStream_t>(stream); }

// ---------------------------------------------------------------- allocation sizes
namespace {
std::mutex g_alloc_mu;
std::unordered_map<void *, size_t> g_alloc_sizes;
} // namespace

void rgs_alloc_note(void *p, size_t bytes) {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc_sizes[p] = bytes;
}

size_t rgs_alloc_forget(void *p) {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    auto it = g_alloc_sizes.find(p);
    if (it == g_alloc_sizes.end()) return 0;
    const size_t b = it->second;
    g_alloc_sizes.erase(it);
    return b;
}

// ---------------------------------------------------------------- workspace pool
namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mempool_mu;
cudaMemPool_t g_mempool[kMaxDevices] = {};

rgs_status device_pool(cudaMemPool_t *out) {
    int dev = 0;
    RGS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        rgs_set_error("device ordinal %d out of range", dev);
        return RGS_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_mempool_mu);
    if (!g_mempool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        RGS_CUDA(cudaMemPoolCreate(&p, &props));
        unsigned long long keep = ~0ull; // keep freed blocks reserved for the next call
        RGS_CUDA(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep));
        g_mempool[dev] = p;
    }
    *out = g_mempool[dev];
    return RGS_OK;
}
} // namespace

rgs_status pool_alloc_bytes(void **p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    cudaMemPool_t pool = nullptr;
    rgs_status r = device_pool(&pool);
    if (r != RGS_OK) return r;
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, st);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        rgs_set_error("workspace allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? RGS_ERR_OOM : RGS_ERR_CUDA;
    }
    return RGS_OK;
}

size_t pool_available_bytes() {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaMemPool_t pool = nullptr;
    if (device_pool(&pool) != RGS_OK) return free_b;
    unsigned long long reserved = 0, used = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) != cudaSuccess ||
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess) {
        cudaGetLastError();
        return free_b;
    }
    return free_b + (size_t)(reserved > used ? reserved - used : 0);
}

void pool_free(void *p, cudaStream_t st) {
    if (p && cudaFreeAsync(p, st) != cudaSuccess) cudaGetLastError();
}

// ---------------------------------------------------------------- launch profiler
namespace {
struct ProfRec {
    int name;
    cudaEvent_t a, b;
};
std::atomic<long long> g_launches{0};
std::atomic<bool> g_prof_on{false};
std::mutex g_prof_mu;
std::vector<std::string> g_names;
std::vector<ProfRec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t pool_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}
} // namespace

ProfScope::ProfScope(const char *name, cudaStream_t s) : st(s) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_prof_on.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    int id = -1;
    for (size_t q = 0; q < g_names.size(); ++q)
        if (g_names[q] == name) id = (int)q;
    if (id < 0) {
        g_names.emplace_back(name);
        id = (int)g_names.size() - 1;
    }
    ProfRec r{id, pool_event(), pool_event()};
    if (!r.a || !r.b) return;
    cudaEventRecord(r.a, st);
    g_recs.push_back(r);
    rec = (int)g_recs.size() - 1;
}

ProfScope::~ProfScope() {
    if (rec < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (rec < (int)g_recs.size()) cudaEventRecord(g_recs[rec].b, st);
}

extern "C" {

int32_t rgs_abi_version(void) { return RGS_ABI_VERSION; }

void rgs_profile_enable(int32_t on) { g_prof_on.store(on != 0); }

int64_t rgs_launch_count(void) { return g_launches.load(); }

void rgs_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &r : g_recs) {
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
}

int32_t rgs_profile_report(rgs_kernel_time *out, int32_t max) {
    if (!out && max > 0) {
        rgs_set_error("rgs_profile_report: NULL output array with max = %d", max);
        return -1;
    }
    std::lock_guard<std::mutex> lk(g_prof_mu);
    std::vector<double> ms(g_names.size(), 0.0);
    std::vector<long long> cnt(g_names.size(), 0);
    for (auto &r : g_recs) {
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess) {
            rgs_set_error("rgs_profile_report: %s", cudaGetErrorString(e));
            cudaGetLastError();
            return -1;
        }
        ms[r.name] += t;
        cnt[r.name] += 1;
    }
    for (size_t q = 0; q < g_names.size() && (int)q < max; ++q) {
        memset(out[q].name, 0, sizeof out[q].name);
        strncpy(out[q].name, g_names[q].c_str(), sizeof out[q].name - 1);
        out[q].launches = cnt[q];
        out[q].total_ms = ms[q];
    }
    return (int32_t)g_names.size();
}

const char *rgs_last_error(void) { return g_err; }

const char *rgs_status_string(rgs_status s) {
    switch (s) {
    case RGS_OK: return "ok";
    case RGS_ERR_ARG: return "invalid argument";
    case RGS_ERR_CUDA: return "CUDA error";
    case RGS_ERR_OOM: return "out of device memory";
    case RGS_ERR_CAPACITY: return "capacity exceeded";
    case RGS_ERR_NONFINITE: return "non-finite input";
    case RGS_ERR_TIMEOUT: return "device wait timed out";
    case RGS_ERR_STATE: return "call out of order";
    }
    return "unknown status";
}

rgs_status rgs_build_scene(const rgs_surfels *surfels, const rgs_build_opts *opts, void *stream, rgs_scene **inout) {
    g_err[0] = 0;
    if (!surfels || !inout) {
        rgs_set_error("rgs_build_scene: NULL argument");
        return RGS_ERR_ARG;
    }
    const rgs_surfels &s = *surfels;
    if (s.n < 1 || s.n > (1 << 28)) {
        rgs_set_error("rgs_build_scene: n = %d outside [1, 2^28]", s.n);
        return RGS_ERR_ARG;
    }
    if (s.sh_degree < 0 || s.sh_degree > RGS_MAX_SH_DEGREE) {
        rgs_set_error("rgs_build_scene: sh_degree = %d outside [0, %d]", s.sh_degree, RGS_MAX_SH_DEGREE);
        return RGS_ERR_ARG;
    }
    if (!s.p || !s.tu || !s.tv || !s.s || !s.o || !s.ad || !s.k || !s.as || !s.shin) {
        rgs_set_error("rgs_build_scene: NULL surfel array");
        return RGS_ERR_ARG;
    }
    if (opts && opts->alpha_model != RGS_ALPHA_GAUSS && opts->alpha_model != RGS_ALPHA_DISC &&
        opts->alpha_model != RGS_ALPHA_GFSGS) {
        rgs_set_error("rgs_build_scene: unknown alpha model %d", opts->alpha_model);
        return RGS_ERR_ARG;
    }
    rgs_scene *sc = *inout;
    bool created = false;
    if (!sc) {
        sc = new (std::nothrow) rgs_scene();
        if (!sc) return RGS_ERR_OOM;
        created = true;
        cudaGetDevice(&sc->device);
    }
    rgs_status r = rgs_scene_build_impl(sc, surfels, opts, S(stream));
    if (r != RGS_OK) {
        if (created) rgs_destroy_scene(sc);
        return r;
    }
    *inout = sc;
    return RGS_OK;
}

rgs_status rgs_trace_transport(rgs_scene *scene, const rgs_lights *lights, const rgs_trace_opts *opts, void *stream,
                               rgs_transport **inout) {
    g_err[0] = 0;
    if (!scene || !opts || !inout) {
        rgs_set_error("rgs_trace_transport: NULL argument");
        return RGS_ERR_ARG;
    }
    if (opts->nd < 32 || opts->nd > 4096 || opts->nd % 32 != 0) {
        rgs_set_error("rgs_trace_transport: nd = %d must be a multiple of 32 in [32, 4096]", opts->nd);
        return RGS_ERR_ARG;
    }
    if ((long long)scene->n * opts->nd >= (1ll << 31)) {
        rgs_set_error("rgs_trace_transport: n * nd = %lld rays exceeds 2^31", (long long)scene->n * opts->nd);
        return RGS_ERR_ARG;
    }
    if (lights && (lights->n_lights < 0 || lights->n_lights > 4096 ||
                   (lights->n_lights > 0 && (!lights->pos || !lights->intensity)))) {
        rgs_set_error("rgs_trace_transport: invalid lights");
        return RGS_ERR_ARG;
    }
    if (opts->hit_capacity < 0) {
        rgs_set_error("rgs_trace_transport: negative hit capacity");
        return RGS_ERR_ARG;
    }
    rgs_transport *t = *inout;
    bool created = false;
    if (!t) {
        t = new (std::nothrow) rgs_transport();
        if (!t) return RGS_ERR_OOM;
        created = true;
    }
    t->sc = scene;
    rgs_status r = rgs_trace_impl(t, lights, opts, S(stream));
    if (r != RGS_OK) {
        if (created) rgs_destroy_transport(t);
        else t->nb_last = -1;
        return r;
    }
    *inout = t;
    return RGS_OK;
}

rgs_status rgs_trace_pairs(rgs_scene *scene, const rgs_lights *lights, const rgs_pair_opts *opts, void *stream,
                           rgs_transport **inout) {
    g_err[0] = 0;
    if (!scene || !inout) {
        rgs_set_error("rgs_trace_pairs: NULL argument");
        return RGS_ERR_ARG;
    }
    if (lights && (lights->n_lights < 0 || lights->n_lights > 4096 ||
                   (lights->n_lights > 0 && (!lights->pos || !lights->intensity)))) {
        rgs_set_error("rgs_trace_pairs: invalid lights");
        return RGS_ERR_ARG;
    }
    rgs_transport *t = *inout;
    bool created = false;
    if (!t) {
        t = new (std::nothrow) rgs_transport();
        if (!t) return RGS_ERR_OOM;
        created = true;
    }
    t->sc = scene;
    rgs_status r = rgs_trace_pairs_impl(t, lights, opts ? opts->lambda : nullptr, S(stream));
    if (r != RGS_OK) {
        if (created) rgs_destroy_transport(t);
        else t->nb_last = -1;
        return r;
    }
    *inout = t;
    return RGS_OK;
}

static rgs_status adjoint_pairs_checked(const char *fn, rgs_transport *t, const float *dL_dB, float *dL_dE,
                                        float *dL_dalbedo, float *dL_dopacity, float *dL_dlambda, float *dL_dp,
                                        float *dL_ds, float *dL_dtu, float *dL_dtv, void *stream) {
    g_err[0] = 0;
    if (!t || !dL_dB) {
        rgs_set_error("%s: NULL argument", fn);
        return RGS_ERR_ARG;
    }
    if (t->kind != RGS_KIND_PAIRS) {
        rgs_set_error("%s: not a center-to-center transport", fn);
        return RGS_ERR_ARG;
    }
    if (t->nb_last < 0) {
        rgs_set_error("%s: no rgs_solve on this transport since it was traced", fn);
        return RGS_ERR_STATE;
    }
    return rgs_adjoint_pairs_impl(t, dL_dB, dL_dE, dL_dalbedo, dL_dopacity, dL_dlambda, dL_dp, dL_ds, dL_dtu, dL_dtv,
                                  S(stream));
}

rgs_status rgs_adjoint_pairs(rgs_transport *t, const float *dL_dB, float *dL_dE, float *dL_dalbedo,
                             float *dL_dopacity, float *dL_dlambda, void *stream) {
    return adjoint_pairs_checked("rgs_adjoint_pairs", t, dL_dB, dL_dE, dL_dalbedo, dL_dopacity, dL_dlambda, nullptr,
                                 nullptr, nullptr, nullptr, stream);
}

rgs_status rgs_adjoint_pairs_geometry(rgs_transport *t, const float *dL_dB, float *dL_dE, float *dL_dalbedo,
                                      float *dL_dopacity, float *dL_dlambda, float *dL_dp, float *dL_ds,
                                      float *dL_dtu, float *dL_dtv, void *stream) {
    return adjoint_pairs_checked("rgs_adjoint_pairs_geometry", t, dL_dB, dL_dE, dL_dalbedo, dL_dopacity, dL_dlambda,
                                 dL_dp, dL_ds, dL_dtu, dL_dtv, stream);
}

rgs_status rgs_solve(rgs_transport *t, const float *E, int32_t n_bounces, int32_t precision, float *B_out,
                     rgs_solve_stats *stats, void *stream) {
    g_err[0] = 0;
    if (!t || !t->sc) {
        rgs_set_error("rgs_solve: NULL transport");
        return RGS_ERR_ARG;
    }
    if (n_bounces < 0 || n_bounces > RGS_MAX_BOUNCES) {
        rgs_set_error("rgs_solve: n_bounces = %d outside [0, %d]", n_bounces, RGS_MAX_BOUNCES);
        return RGS_ERR_ARG;
    }
    if (precision != RGS_FP32 && precision != RGS_BF16_FP32ACC && precision != RGS_BF16_FP32ACC_RESCORR) {
        rgs_set_error("rgs_solve: unknown precision %d", precision);
        return RGS_ERR_ARG;
    }
    if (t->kind == RGS_KIND_NONE) {
        rgs_set_error("rgs_solve: transport was not traced");
        return RGS_ERR_STATE;
    }
    return rgs_solve_impl(t, E, n_bounces, precision, B_out, stats, S(stream));
}

rgs_status rgs_adjoint(rgs_transport *t, const float *dL_dB, float *dL_dE, float *dL_dalbedo, float *dL_dopacity,
                       void *stream) {
    g_err[0] = 0;
    if (!t || !dL_dB) {
        rgs_set_error("rgs_adjoint: NULL argument");
        return RGS_ERR_ARG;
    }
    if (t->nb_last < 0) {
        rgs_set_error("rgs_adjoint: no rgs_solve on this transport since it was traced");
        return RGS_ERR_STATE;
    }
    return rgs_adjoint_impl(t, dL_dB, dL_dE, dL_dalbedo, dL_dopacity, S(stream));
}

rgs_status rgs_adjoint_geometry(rgs_transport *t, const float *dL_dB, float *dL_dE, float *dL_dalbedo,
                                float *dL_dopacity, float *dL_dp, float *dL_ds, float *dL_dtu, float *dL_dtv,
                                void *stream) {
    g_err[0] = 0;
    if (!t || !dL_dB) {
        rgs_set_error("rgs_adjoint_geometry: NULL argument");
        return RGS_ERR_ARG;
    }
    if (t->nb_last < 0) {
        rgs_set_error("rgs_adjoint_geometry: no rgs_solve on this transport since it was traced");
        return RGS_ERR_STATE;
    }
    return rgs_adjoint_impl(t, dL_dB, dL_dE, dL_dalbedo, dL_dopacity, S(stream), dL_dp, dL_ds, dL_dtu, dL_dtv);
}

rgs_status rgs_solve_batched(rgs_transport *const *ts, int32_t count, const float *const *E,
                             const int32_t *n_bounces, const rgs_batch_opts *opts, float *const *B_out,
                             double *residual_norms, void *stream) {
    g_err[0] = 0;
    if (!ts || !n_bounces || count < 1 || count > 4096) {
        rgs_set_error("rgs_solve_batched: need 1..4096 transports and their bounce counts");
        return RGS_ERR_ARG;
    }
    const int precision = opts ? opts->precision : RGS_FP32;
    if (precision != RGS_FP32 && precision != RGS_BF16_FP32ACC && precision != RGS_BF16_FP32ACC_RESCORR) {
        rgs_set_error("rgs_solve_batched: unknown precision %d", precision);
        return RGS_ERR_ARG;
    }
    for (int s = 0; s < count; ++s) {
        if (!ts[s] || !ts[s]->sc) {
            rgs_set_error("rgs_solve_batched: transport %d is NULL", s);
            return RGS_ERR_ARG;
        }
        if (ts[s]->kind == RGS_KIND_NONE) {
            rgs_set_error("rgs_solve_batched: transport %d was not traced", s);
            return RGS_ERR_STATE;
        }
        if (ts[s]->kind != RGS_KIND_HEMISPHERE) {
            rgs_set_error("rgs_solve_batched: transport %d is a center-to-center transport (solve it with rgs_solve)", s);
            return RGS_ERR_ARG;
        }
        if (n_bounces[s] < 0 || n_bounces[s] > RGS_MAX_BOUNCES) {
            rgs_set_error("rgs_solve_batched: n_bounces[%d] = %d outside [0, %d]", s, n_bounces[s], RGS_MAX_BOUNCES);
            return RGS_ERR_ARG;
        }
        for (int q = 0; q < s; ++q)
            if (ts[q] == ts[s]) {
                rgs_set_error("rgs_solve_batched: transport %d appears twice", s);
                return RGS_ERR_ARG;
            }
    }
    return rgs_solve_batched_impl(ts, count, E, n_bounces, opts, B_out, residual_norms, S(stream));
}

rgs_status rgs_get_iterate(rgs_transport *t, int32_t b, float *out, void *stream) {
    g_err[0] = 0;
    if (!t || !out) {
        rgs_set_error("rgs_get_iterate: NULL argument");
        return RGS_ERR_ARG;
    }
    if (t->nb_last < 0) {
        rgs_set_error("rgs_get_iterate: no rgs_solve on this transport");
        return RGS_ERR_STATE;
    }
    if (b < 0 || b > t->nb_last) {
        rgs_set_error("rgs_get_iterate: b = %d outside [0, %d]", b, t->nb_last);
        return RGS_ERR_ARG;
    }
    return rgs_get_iterate_impl(t, b, out, S(stream));
}

rgs_status rgs_set_checkpointing(rgs_transport *t, int32_t stride) {
    if (!t) {
        rgs_set_error("rgs_set_checkpointing: NULL transport");
        return RGS_ERR_ARG;
    }
    if (stride < -1 || stride > RGS_MAX_BOUNCES) {
        rgs_set_error("rgs_set_checkpointing: stride %d outside [-1, %d]", stride, RGS_MAX_BOUNCES);
        return RGS_ERR_ARG;
    }
    t->ckpt_req = stride;
    return RGS_OK;
}

rgs_status rgs_set_tensor_cores(rgs_transport *t, int32_t mode) {
    if (!t || mode < -1 || mode > 3) {
        rgs_set_error("rgs_set_tensor_cores: NULL transport or mode outside [-1, 3]");
        return RGS_ERR_ARG;
    }
    t->tc_mode = mode;
    return RGS_OK;
}

rgs_status rgs_set_wait_limit(rgs_transport *t, int64_t ns) {
    if (!t || ns < 0) {
        rgs_set_error("rgs_set_wait_limit: NULL transport or negative limit");
        return RGS_ERR_ARG;
    }
    t->tc_wait_ns = ns ? (unsigned long long)ns : 4000000000ull;
    return RGS_OK;
}

rgs_status rgs_set_memory_budget(rgs_transport *t, int64_t bytes) {
    if (!t || bytes < 0) {
        rgs_set_error("rgs_set_memory_budget: NULL transport or negative budget");
        return RGS_ERR_ARG;
    }
    t->mem_budget = bytes;
    return RGS_OK;
}

rgs_status rgs_trim_workspace(void) {
    int dev = 0;
    RGS_CUDA(cudaGetDevice(&dev));
    cudaMemPool_t p = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mempool_mu);
        if (dev >= 0 && dev < kMaxDevices) p = g_mempool[dev];
    }
    if (!p) return RGS_OK;
    RGS_CUDA(cudaDeviceSynchronize());
    RGS_CUDA(cudaMemPoolTrimTo(p, 0));
    return RGS_OK;
}

rgs_status rgs_transport_info_get(const rgs_transport *t, rgs_transport_info *info) {
    if (!t || !info) {
        rgs_set_error("rgs_transport_info_get: NULL argument");
        return RGS_ERR_ARG;
    }
    info->n = t->n;
    info->sh_degree = t->L;
    info->nc = t->nc;
    info->n_cols = t->C;
    info->nd = t->nd;
    info->n_lights = t->nl;
    info->n_hits = t->n_hits;
    info->n_hit_slots = t->n_slots;
    info->n_full_rays = t->n_full;
    info->device_bytes = t->device_bytes;
    return RGS_OK;
}

void rgs_destroy_transport(rgs_transport *t) {
    if (!t) return;
    cudaDeviceSynchronize();
    rgs_batch_forget(t);
    dev_free(t->lpos);
    dev_free(t->lint);
    dev_free(t->rec_ja);
    dev_free(t->off);
    dev_free(t->ray_ctr);
    dev_free(t->cnt);
    dev_free(t->counter);
    dev_free(t->flags);
    dev_free(t->src_off);
    dev_free(t->src_cnt);
    dev_free(t->cursor);
    dev_free(t->scan_tmp);
    dev_free(t->D);
    dev_free(t->iters);
    dev_free(t->Q);
    dev_free(t->iters16);
    dev_free(t->norm2);
    dev_free(t->Pg);
    dev_free(t->dop);
    dev_free(t->dir);
    dev_free(t->pair_off);
    dev_free(t->pair_rec);
    dev_free(t->chunk_off);
    dev_free(t->chunk_cnt);
    dev_free(t->chunk_tmp);
    dev_free(t->lam);
    dev_free(t->aarea);
    dev_free(t->daarea);
    rgs_tc_free(t);
    rgs_mc_free(t);
    delete t;
}

void rgs_destroy_scene(rgs_scene *s) {
    if (!s) return;
    cudaDeviceSynchronize();
    dev_free(s->P);
    dev_free(s->N4);
    dev_free(s->FU);
    dev_free(s->FV);
    dev_free(s->GS);
    dev_free(s->cl);
    dev_free(s->kk);
    dev_free(s->uid);
    dev_free(s->inv);
    dev_free(s->nodes);
    dev_free(s->boxes);
    dev_free(s->parent);
    dev_free(s->visit);
    dev_free(s->keys);
    dev_free(s->keys_alt);
    dev_free(s->vals);
    dev_free(s->vals_alt);
    dev_free(s->hist);
    dev_free(s->bounds);
    dev_free(s->eps_plane);
    dev_free(s->flags);
    delete s;
}

} // extern "C"
