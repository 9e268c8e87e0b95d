// Bounce iteration (rgs_solve): B^(0) = S = E + D, B^(k) = S + K B^(k-1).
//
// k_bounce is the gather/projection of Eq. final-radiosity in its ray-factored form:
// one CTA per receiver i and column tile; each thread owns rays of i and, per ray,
// gathers the stored hits' radiance x_r[c] = sum_h a_rh Y(-d_r) . B_{j_h}[c]; the CTA then
// projects Q_i[c][k] = (pi/nd) sum_r Y_k(R_i d_r) x_r[c] and writes Q^(k-1),
// B^(k) = S + o_i c_i (x) Q and the FP64 partial sum of (B^(k) - B^(k-1))^2.
#include "rgs_internal.cuh"

namespace {

constexpr int BOUNCE_THREADS = 256;

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
    constexpr int G = SL::G, KPL = SL::KPL, GROUPS = BOUNCE_THREADS / G, RS = SL::STRIDE;
    const int i = blockIdx.x;
    const int col0 = blockIdx.y * CT;
    const int nd = rays.nd;
    const int grp = threadIdx.x / G, g = threadIdx.x % G;
    const float3 n = f3(sc.N4[i]);
    float acc[KPL][CT];
#pragma unroll
    for (int m = 0; m < KPL; ++m)
#pragma unroll
        for (int c = 0; c < CT; ++c) acc[m][c] = 0.f;

    for (int q = grp; q < nd; q += GROUPS) {
        const long long r = (long long)i * nd + q;
        const float3 d = f3(rays.dir[r]);
        float yo[KPL], yi[KPL];
        {
            float Y[NC];
            sh_eval<NC>(neg3(d), Y);
            SL::pick(Y, g, yo);
            sh_eval<NC>(reflect_n(n, d), Y);
            SL::pick(Y, g, yi);
        }
        const int cnt = rays.cnt[r];
        const long long base = rays.off[r];
        float x[CT];
#pragma unroll
        for (int c = 0; c < CT; ++c) x[c] = 0.f;
#pragma unroll 4
        for (int h = 0; h < cnt; ++h) {
            const int2 ja = __ldg(&rays.rec_ja[base + h]);
            const float a = __int_as_float(ja.y);
            const typename SL::T *Bj = Bg + ((size_t)ja.x * C + col0) * RS;
#pragma unroll
            for (int c = 0; c < CT; ++c) {
                float v[KPL];
                SL::load(Bj + c * RS, g, v);
                float s = 0.f;
#pragma unroll
                for (int m = 0; m < KPL; ++m) s += yo[m] * v[m];
                x[c] += a * s;
            }
        }
#pragma unroll
        for (int c = 0; c < CT; ++c) {
            const float xc = SL::group_sum(x[c]);
#pragma unroll
            for (int m = 0; m < KPL; ++m) acc[m][c] += yi[m] * xc;
        }
    }
    // reduce over the groups: lanes with equal g within the warp, then across warps
    __shared__ float red[BOUNCE_THREADS / 32][G][KPL * CT];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int m = 0; m < KPL; ++m)
#pragma unroll
        for (int c = 0; c < CT; ++c) {
            float v = acc[m][c];
#pragma unroll
            for (int off = G; off < 32; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane < G) red[warp][lane][m * CT + c] = v;
        }
    __syncthreads();
    double dsq = 0.0;
    const float w = 3.14159265358979f / (float)nd;
    for (int e = threadIdx.x; e < NC * CT; e += BOUNCE_THREADS) {
        const int k = e / CT, c = e - k * CT;
        int gg = 0, mm = 0;
#pragma unroll
        for (int g2 = 0; g2 < G; ++g2)
#pragma unroll
            for (int m2 = 0; m2 < KPL; ++m2)
                if (SL::k(g2, m2) == k) {
                    gg = g2;
                    mm = m2;
                }
        float v = 0.f;
        for (int q = 0; q < BOUNCE_THREADS / 32; ++q) v += red[q][gg][mm * CT + c];
        const int col = col0 + c;
        const float Q = w * v;
        const size_t idx = ((size_t)i * C + col) * NC + k;
        Qout[idx] = Q;
        const float oc = sc.P[i].w * sc.cl[(size_t)i * 12 + band_of(k) * 3 + (col % 3)];
        const float b = S[idx] + oc * Q;
        Bout[idx] = b;
        if (Bout16) Bout16[((size_t)i * C + col) * bf16_stride<NC>() + k] = __float2bfloat16_rn(b);
        const double df = (double)b - (double)Bprev[idx];
        dsq += df * df;
    }
    // FP64 residual norm: warp reduce, one atomic per warp with work
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) dsq += __shfl_xor_sync(0xffffffffu, dsq, off);
    if (lane == 0 && warp * 32 < NC * CT) atomicAdd(norm2, dsq);
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

rgs_status rgs_solve_impl(rgs_transport *t, const float *E, int nb, int precision, float *B_out,
                          rgs_solve_stats *stats, cudaStream_t st) {
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
