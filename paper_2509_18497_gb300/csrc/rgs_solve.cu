// Bounce iteration (rgs_solve): B^(0) = S = E + D, B^(k) = S + K B^(k-1).
//
// k_bounce is the gather/projection of Eq. final-radiosity in its ray-factored form:
// one CTA per receiver i and column tile; each thread owns rays of i and, per ray,
// gathers the stored hits' radiance x_r[c] = sum_h a_rh Y(-d_r) . B_{j_h}[c]; the CTA then
// projects Q_i[c][k] = (pi/nd) sum_r Y_k(R_i d_r) x_r[c] and writes Q^(k-1),
// B^(k) = S + o_i c_i (x) Q and the FP64 partial sum of (B^(k) - B^(k-1))^2.
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
__global__ void __launch_bounds__(BOUNCE_THREADS) k_bounce(SceneDev sc, RaysDev rays, int C,
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

template <int NC>
rgs_status run_solve(rgs_transport *t, const float *E, int nb, int precision, cudaStream_t st) {
    const size_t A = t->arr();
    const size_t A16 = (size_t)t->n * t->C * bf16_stride<NC>();
    const bool bf16 = precision != RGS_FP32;
    SceneDev sd = t->sc->dev();
    RaysDev rd = t->rays();
    __nv_bfloat16 *I16 = bf16 ? t->iters16 : nullptr;
    launch_make_S<NC>(t, E, t->iters, I16, st);
    RGS_LAUNCH("make_S");
    for (int b = 1; b <= nb; ++b) {
        // RESCORR: the last bounce gathers the FP32 rows (one residual-correction sweep)
        const bool rows16 = bf16 && !(precision == RGS_BF16_FP32ACC_RESCORR && b == nb);
        rgs_status r =
            (t->C >= RGS_MC_MIN_COLS ? mc_bounce<NC> : launch_bounce<NC>)(
                t, sd, rd, rows16, t->iters + A * (b - 1), bf16 ? I16 + A16 * (b - 1) : nullptr, t->iters,
                t->Q + A * (b - 1), t->iters + A * b, bf16 ? I16 + A16 * b : nullptr, t->norm2 + b, st);
        if (r != RGS_OK) return r;
    }
    return RGS_OK;
}

// iterate buffers for nb bounces at the given precision (kept for the adjoint)
rgs_status rgs_solve_prepare(rgs_transport *t, int nb, int precision, cudaStream_t st) {
    rgs_status r;
    const size_t A = t->arr();
    if (nb + 1 > t->iters_cap) {
        if ((r = dev_alloc(&t->iters, A * (nb + 1), &t->device_bytes)) != RGS_OK) return r;
        if ((r = dev_alloc(&t->Q, A * (nb > 0 ? nb : 1), &t->device_bytes)) != RGS_OK) return r;
        t->iters_cap = nb + 1;
    }
    if (precision != RGS_FP32 && nb + 1 > t->iters16_cap) {
        const size_t A16 = (size_t)t->n * t->C * (t->nc >= 9 ? 16 : t->nc);
        if ((r = dev_alloc(&t->iters16, A16 * (nb + 1), &t->device_bytes)) != RGS_OK) return r;
        RGS_CUDA(cudaMemsetAsync(t->iters16, 0, sizeof(__nv_bfloat16) * A16 * (nb + 1), st)); // row padding stays 0
        t->iters16_cap = nb + 1;
    }
    if (!t->norm2 && (r = dev_alloc(&t->norm2, RGS_MAX_BOUNCES + 1, &t->device_bytes)) != RGS_OK) return r;
    return RGS_OK;
}

rgs_status rgs_solve_impl(rgs_transport *t, const float *E, int nb, int precision, float *B_out,
                          rgs_solve_stats *stats, cudaStream_t st) {
    rgs_status r;
    const size_t A = t->arr();
    if ((r = rgs_solve_prepare(t, nb, precision, st)) != RGS_OK) return r;
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
        switch (t->nc) {
        case 1: launch_to_user<1>(t, t->iters + A * nb, B_out, st); break;
        case 4: launch_to_user<4>(t, t->iters + A * nb, B_out, st); break;
        case 9: launch_to_user<9>(t, t->iters + A * nb, B_out, st); break;
        default: launch_to_user<16>(t, t->iters + A * nb, B_out, st);
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

rgs_status rgs_get_iterate_impl(rgs_transport *t, int b, float *out, cudaStream_t st) {
    const size_t A = t->arr();
    switch (t->nc) {
    case 1: launch_to_user<1>(t, t->iters + A * b, out, st); break;
    case 4: launch_to_user<4>(t, t->iters + A * b, out, st); break;
    case 9: launch_to_user<9>(t, t->iters + A * b, out, st); break;
    default: launch_to_user<16>(t, t->iters + A * b, out, st);
    }
    RGS_LAUNCH("get_iterate");
    return RGS_OK;
}
