// Bounce iteration (rgs_solve): B^(0) = S = E + D, B^(k) = S + K B^(k-1).
//
// k_bounce is the gather/projection of Eq. final-radiosity in its ray-factored form:
// one CTA per receiver i and column tile; each thread owns rays of i and, per ray,
// gathers the stored hits' radiance x_r[c] = sum_h a_rh Y(-d_r) . B_{j_h}[c]; the CTA then
// projects Q_i[c][k] = (pi/nd) sum_r Y_k(R_i d_r) x_r[c] and writes Q^(k-1),
// B^(k) = S + o_i c_i (x) Q and the FP64 partial sum of (B^(k) - B^(k-1))^2.
#include <algorithm>
#include <vector>

#include "rgs_bounce_body.cuh"

namespace {


// internal [N][C][NC] <- user [N][nc][3] emission broadcast over the columns, plus D;
// optionally also the BF16 copy (rows of bf16_stride<NC>)
template <int NC>
__global__ void k_make_S(int n, int C, const int *__restrict__ uid, const float *__restrict__ E,
                         const float *__restrict__ D, float *S, __nv_bfloat16 *S16) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * C * NC) return;
    const int k = (int)(idx % NC);
    const size_t ic = idx / NC;
    const int c = (int)(ic % C);
    const int i = (int)(ic / C);
    float e = E ? E[((size_t)uid[i] * NC + k) * 3 + (c % 3)] : 0.f;
    const float v = e + D[idx];
    S[idx] = v;
    if (S16) S16[ic * bf16_stride<NC>() + k] = __float2bfloat16_rn(v);
}

// internal [N][C][NC] -> user [N][nc][C]
template <int NC>
__global__ void k_to_user(int n, int C, const int *__restrict__ uid, const float *__restrict__ X, float *Y) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * C * NC) return;
    const int k = (int)(idx % NC);
    const size_t ic = idx / NC;
    const int c = (int)(ic % C);
    const int i = (int)(ic / C);
    Y[((size_t)uid[i] * NC + k) * C + c] = X[idx];
}

template <int NC, int CT, class SL>
__global__ void RGS_BOUNCE_LB k_bounce(SceneDev sc, RaysDev rays, int C,
                                                          const typename SL::T *__restrict__ Bg,
                                                          const float *__restrict__ Bprev, const float *__restrict__ S,
                                                          float *__restrict__ Qout, float *__restrict__ Bout,
                                                          __nv_bfloat16 *__restrict__ Bout16, double *norm2) {
    __shared__ float red[(BOUNCE_THREADS / 32) * SL::G * SL::KPL * CT];
    bounce_receiver<NC, CT, SL>(sc, rays, C, Bg, Bprev, S, Qout, Bout, Bout16, norm2, blockIdx.x, blockIdx.y * CT, red);
}

template <int NC>
rgs_status launch_bounce(const rgs_transport *t, SceneDev sd, RaysDev rd, bool bf16_rows, const float *Bprev,
                         const __nv_bfloat16 *Bprev16, const float *S, float *Q, float *Bout, __nv_bfloat16 *Bout16,
                         double *norm2, cudaStream_t st) {
    dim3 grid(t->n, t->C / 3);
    if (bf16_rows) {
        ProfScope ps_("k_bounce", st);
        k_bounce<NC, 3, SliceH<NC>><<<grid, BOUNCE_THREADS, 0, st>>>(sd, rd, t->C, Bprev16, Bprev, S, Q, Bout, Bout16, norm2);
    } else {
        ProfScope ps_("k_bounce", st);
        k_bounce<NC, 3, Slice<NC>><<<grid, BOUNCE_THREADS, 0, st>>>(sd, rd, t->C, Bprev, Bprev, S, Q, Bout, Bout16, norm2);
    }
    RGS_LAUNCH("bounce");
    return RGS_OK;
}

template <int NC>
void launch_make_S(const rgs_transport *t, const float *E, float *S, __nv_bfloat16 *S16, cudaStream_t st) {
    size_t tot = t->arr();
    { ProfScope ps_("k_make_S", st); k_make_S<NC><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(t->n, t->C, t->sc->uid, E, t->D, S, S16); }
}
template <int NC>
void launch_to_user(const rgs_transport *t, const float *X, float *Y, cudaStream_t st) {
    size_t tot = t->arr();
    { ProfScope ps_("k_to_user", st); k_to_user<NC><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(t->n, t->C, t->sc->uid, X, Y); }
}

} // namespace

// the batched modes on the tensor cores (rgs_tc.cu): B^(0) = S, then per bounce the pair-tile
// contraction reading the blocked BF16 copy of B^(b-1) (and its low part in the correction
// bounce) and writing Q^(b-1), B^(b), its row-layout BF16 copy and the next blocked copy
rgs_status run_solve_tc(rgs_transport *t, const float *E, int nb, int precision, cudaStream_t st) {
    const size_t A = t->arr();
    rgs_status r;
    launch_make_S<16>(t, E, t->iters, t->iters16, st);
    RGS_LAUNCH("make_S");
    if ((r = rgs_tc_prepare(t, st)) != RGS_OK) return r;
    if ((r = rgs_tc_reset_flags(t, st)) != RGS_OK) return r;
    const bool rescorr = precision == RGS_BF16_FP32ACC_RESCORR;
    if ((r = rgs_tc_load_blk(t, t->iters, 0, rescorr && nb == 1, st)) != RGS_OK) return r;
    for (int b = 1; b <= nb; ++b) {
        const bool split = rescorr && b == nb;
        const bool want_lo = rescorr && b == nb - 1;
        if ((r = rgs_tc_bounce(t, (b - 1) & 1, b & 1, split, want_lo, t->iters + A * (b - 1), t->iters,
                               t->Q + A * (b - 1), t->iters + A * b, t->iters16 + A * b, t->norm2 + b, st)) != RGS_OK)
            return r;
    }
    t->tc_used = true;
    return rgs_tc_check(t, st);
}

template <int NC>
rgs_status run_solve(rgs_transport *t, const float *E, int nb, int precision, cudaStream_t st) {
    const size_t A = t->arr();
    t->tc_used = false;
    if constexpr (NC == 16)
        if (nb >= 1 && rgs_tc_eligible(t, precision)) return run_solve_tc(t, E, nb, precision, st);
    const size_t A16 = (size_t)t->n * t->C * bf16_stride<NC>();
    const bool bf16 = precision != RGS_FP32;
    SceneDev sd = t->sc->dev();
    RaysDev rd = t->rays();
    __nv_bfloat16 *I16 = bf16 ? t->iters16 : nullptr;
    launch_make_S<NC>(t, E, t->iters, I16, st); // B^(0) = S lives in slot 0 in every mode
    RGS_LAUNCH("make_S");
    for (int b = 1; b <= nb; ++b) {
        // RESCORR: the last bounce gathers the FP32 rows (one residual-correction sweep)
        const bool rows16 = bf16 && !(precision == RGS_BF16_FP32ACC_RESCORR && b == nb);
        const int sp = t->slot(b - 1), so = t->slot(b);
        rgs_status r;
        if (t->kind == RGS_KIND_PAIRS)
            r = pairs_bounce<NC>(t, rows16, t->iters + A * sp, bf16 ? I16 + A16 * sp : nullptr, t->iters,
                                 t->Q + A * (b - 1), t->iters + A * so, bf16 ? I16 + A16 * so : nullptr, t->norm2 + b, st);
        else
            r = (wide_bounce(t->C, rows16) ? mc_bounce<NC> : launch_bounce<NC>)(
                t, sd, rd, rows16, t->iters + A * sp, bf16 ? I16 + A16 * sp : nullptr, t->iters,
                t->Q + A * (t->stride ? 0 : b - 1), t->iters + A * so, bf16 ? I16 + A16 * so : nullptr, t->norm2 + b, st);
        if (r != RGS_OK) return r;
    }
    return RGS_OK;
}

template <int NC>
rgs_status run_recompute(rgs_transport *t, int c, int e, float *const *B, __nv_bfloat16 *const *B16, float *const *Q,
                         double *norm2, cudaStream_t st) {
    const size_t A = t->arr();
    const size_t A16 = (size_t)t->n * t->C * bf16_stride<NC>();
    const bool bf16 = t->prec_last != RGS_FP32;
    SceneDev sd = t->sc->dev();
    RaysDev rd = t->rays();
    for (int b = c + 1; b <= e; ++b) {
        const bool rows16 = bf16 && !(t->prec_last == RGS_BF16_FP32ACC_RESCORR && b == t->nb_last);
        const int k = b - c - 1;
        const float *Bp = k == 0 ? t->iters + A * t->slot(c) : B[k - 1];
        const __nv_bfloat16 *Bp16 = !bf16 ? nullptr : (k == 0 ? t->iters16 + A16 * t->slot(c) : B16[k - 1]);
        rgs_status r = (wide_bounce(t->C, rows16) ? mc_bounce<NC> : launch_bounce<NC>)(
            t, sd, rd, rows16, Bp, Bp16, t->iters, Q[k], B[k], bf16 ? B16[k] : nullptr, norm2 + b, st);
        if (r != RGS_OK) return r;
    }
    return RGS_OK;
}

rgs_status rgs_recompute(rgs_transport *t, int c, int e, float *const *B, __nv_bfloat16 *const *B16, float *const *Q,
                         double *norm2, cudaStream_t st) {
    switch (t->nc) {
    case 1: return run_recompute<1>(t, c, e, B, B16, Q, norm2, st);
    case 4: return run_recompute<4>(t, c, e, B, B16, Q, norm2, st);
    case 9: return run_recompute<9>(t, c, e, B, B16, Q, norm2, st);
    default: return run_recompute<16>(t, c, e, B, B16, Q, norm2, st);
    }
}

static size_t bf16_row(int nc) { return nc >= 9 ? 16 : (size_t)nc; }

int rgs_auto_stride(const rgs_transport *t, int nb, int precision) {
    if (nb <= 1) return 0;
    const double A = 4.0 * t->arr();
    const double A16 = precision != RGS_FP32 ? 2.0 * t->n * t->C * bf16_row(t->nc) : 0.0;
    const double rays = (double)t->n * t->nd;
    const double fwd = (nb + 1) * (A + A16) + nb * A;
    const double adj = (nb + 2) * A + 8.0 * t->n_hits + 4.0 * t->n_slots + rays * (wide_adjoint(t->C) ? 128 : 16);
    const double held = t->iters_cap * A + t->q_cap * A + t->iters16_cap * A16;
    double room = 0.95 * ((double)pool_available_bytes() + held);
    if (t->mem_budget > 0) room = std::min(room, (double)t->mem_budget - ((double)t->device_bytes - held));
    if (fwd + adj <= room) return 0;
    int s = 1;
    while (s * s < nb) ++s;
    return s;
}

// iterate buffers for nb bounces at the given precision and checkpoint stride
rgs_status rgs_solve_prepare(rgs_transport *t, int nb, int precision, int stride, cudaStream_t st) {
    rgs_status r;
    const size_t A = t->arr();
    t->nb_last = -1; // set again once the new iterates are complete
    if (nb <= 1) stride = 0; // nothing to save
    const int n_ckpt = stride ? (nb - 1) / stride + 1 : 0;
    const int n_it = stride ? n_ckpt + 2 : nb + 1;
    const int n_q = stride ? 1 : (nb > 0 ? nb : 1);
    // checkpointing sizes the buffers exactly (memory is what it is for); otherwise they only grow
    if (n_it > t->iters_cap || (stride && n_it != t->iters_cap)) {
        t->iters_cap = 0;
        if ((r = dev_alloc(&t->iters, A * n_it, &t->device_bytes)) != RGS_OK) return r;
        t->iters_cap = n_it;
    }
    if (n_q > t->q_cap || (stride && n_q != t->q_cap)) {
        t->q_cap = 0;
        if ((r = dev_alloc(&t->Q, A * n_q, &t->device_bytes)) != RGS_OK) return r;
        t->q_cap = n_q;
    }
    if (precision != RGS_FP32 && (n_it > t->iters16_cap || (stride && n_it != t->iters16_cap))) {
        const size_t A16 = (size_t)t->n * t->C * bf16_row(t->nc);
        t->iters16_cap = 0;
        if ((r = dev_alloc(&t->iters16, A16 * n_it, &t->device_bytes)) != RGS_OK) return r;
        RGS_CUDA(cudaMemsetAsync(t->iters16, 0, sizeof(__nv_bfloat16) * A16 * n_it, st)); // row padding stays 0
        t->iters16_cap = n_it;
    }
    if (!t->norm2 && (r = dev_alloc(&t->norm2, RGS_MAX_BOUNCES + 1, &t->device_bytes)) != RGS_OK) return r;
    t->stride = stride;
    t->n_ckpt = n_ckpt;
    return RGS_OK;
}

rgs_status rgs_solve_impl(rgs_transport *t, const float *E, int nb, int precision, float *B_out,
                          rgs_solve_stats *stats, cudaStream_t st) {
    rgs_status r;
    const size_t A = t->arr();
    // the center-to-center adjoint keeps every iterate (its pairs are few next to the rays)
    const int stride = t->kind == RGS_KIND_PAIRS ? 0 : (t->ckpt_req < 0 ? rgs_auto_stride(t, nb, precision) : t->ckpt_req);
    if ((r = rgs_solve_prepare(t, nb, precision, stride, st)) != RGS_OK) return r;
    RGS_CUDA(cudaMemsetAsync(t->norm2, 0, sizeof(double) * (RGS_MAX_BOUNCES + 1), st));
    switch (t->nc) {
    case 1: r = run_solve<1>(t, E, nb, precision, st); break;
    case 4: r = run_solve<4>(t, E, nb, precision, st); break;
    case 9: r = run_solve<9>(t, E, nb, precision, st); break;
    default: r = run_solve<16>(t, E, nb, precision, st);
    }
    if (r != RGS_OK) return r;
    t->nb_last = nb;
    t->prec_last = precision;
    if (B_out) {
        const float *X = t->iters + A * t->slot(nb);
        switch (t->nc) {
        case 1: launch_to_user<1>(t, X, B_out, st); break;
        case 4: launch_to_user<4>(t, X, B_out, st); break;
        case 9: launch_to_user<9>(t, X, B_out, st); break;
        default: launch_to_user<16>(t, X, B_out, st);
        }
        RGS_LAUNCH("to_user");
    }
    if (stats) {
        double nrm[RGS_MAX_BOUNCES + 1];
        RGS_CUDA(cudaMemcpyAsync(nrm, t->norm2, sizeof nrm, cudaMemcpyDeviceToHost, st));
        RGS_CUDA(cudaStreamSynchronize(st));
        stats->n_bounces = nb;
        stats->n_cols = t->C;
        for (int b = 0; b < RGS_MAX_BOUNCES; ++b) stats->residual_norm[b] = (b < nb) ? sqrt(nrm[b + 1]) : 0.0;
        stats->n_hits = t->n_hits;
        stats->n_hit_slots = t->n_slots;
        stats->n_full_rays = t->n_full;
    }
    return RGS_OK;
}

// B^(b) in the user layout; an iterate that a checkpointed solve did not keep is
// recomputed from the checkpoint below it into pooled scratch.
rgs_status rgs_get_iterate_impl(rgs_transport *t, int b, float *out, cudaStream_t st) {
    const size_t A = t->arr();
    const float *X = nullptr;
    float *tmp[2] = {nullptr, nullptr}, *q = nullptr;
    __nv_bfloat16 *tmp16[2] = {nullptr, nullptr};
    double *nrm = nullptr;
    rgs_status r = RGS_OK;
    if (t->is_stored(b)) {
        X = t->iters + A * t->slot(b);
    } else {
        const int c = (b / t->stride) * t->stride;
        const size_t A16 = (size_t)t->n * t->C * bf16_row(t->nc);
        const bool bf16 = t->prec_last != RGS_FP32;
        std::vector<float *> B, Qv;
        std::vector<__nv_bfloat16 *> B16;
        for (int k = 0; k < 2 && r == RGS_OK; ++k) {
            r = pool_alloc(&tmp[k], A, st);
            if (r == RGS_OK && bf16) {
                r = pool_alloc(&tmp16[k], A16, st);
                if (r == RGS_OK && cudaMemsetAsync(tmp16[k], 0, sizeof(__nv_bfloat16) * A16, st) != cudaSuccess)
                    r = rgs_cuda_fail(cudaGetLastError(), "memset");
            }
        }
        if (r == RGS_OK) r = pool_alloc(&q, A, st);
        if (r == RGS_OK) r = pool_alloc(&nrm, RGS_MAX_BOUNCES + 1, st);
        if (r == RGS_OK) {
            for (int k = 0; k < b - c; ++k) {
                B.push_back(tmp[k & 1]);
                B16.push_back(tmp16[k & 1]);
                Qv.push_back(q);
            }
            r = rgs_recompute(t, c, b, B.data(), B16.data(), Qv.data(), nrm, st);
            X = tmp[(b - c - 1) & 1];
        }
    }
    if (r == RGS_OK) {
        switch (t->nc) {
        case 1: launch_to_user<1>(t, X, out, st); break;
        case 4: launch_to_user<4>(t, X, out, st); break;
        case 9: launch_to_user<9>(t, X, out, st); break;
        default: launch_to_user<16>(t, X, out, st);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) r = rgs_cuda_fail(e, "get_iterate");
    }
    for (int k = 0; k < 2; ++k) {
        pool_release(tmp[k], st);
        pool_release(tmp16[k], st);
    }
    pool_release(q, st);
    pool_release(nrm, st);
    return r;
}
