// Adjoint (rgs_adjoint): exact gradients of L(B^(n)) for the truncated bounce series.
//
//   v^(0) = dL/dB^(n),  v^(a) = K^T v^(a-1)   (Eq. final_dL_dE: the same paths with the
//                                              decay reversed, propagating gradients)
//   u = sum_a v^(a) = dL/dS,   P_i[l][ch] = sum_{k in l, light} (sum_{a<n} v^(a) Q^(n-1-a) + u Dgeo)
//
// k_adj_bounce gathers K^T v over the records grouped by source surfel j:
//   (K^T v)_j[c][k] = sum_{hits e on j} a_e Y_k(-d_e) y_e[c],
//   y_e[c] = (pi/nd) o_i sum_k' c_{i,l(k'),ch} Y_k'(R_i d_e) v_i[c][k']      (i = receiver of e)
// k_hemi_opacity_bwd / k_shadow_bwd run the compositing backward of every hemisphere and
// shadow ray (dL/dalpha_h = T_h (g_h - R_h), dL/dT = -prod of the other (1 - alpha)).
#include "rgs_internal.cuh"

namespace {

constexpr int ADJ_THREADS = 128;

// user [N][nc][C] -> internal [N][C][NC]
template <int NC>
__global__ void k_from_user(int n, int C, const int *__restrict__ uid, const float *__restrict__ X, float *Y) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * C * NC) return;
    const int k = (int)(idx % NC);
    const size_t ic = idx / NC;
    const int c = (int)(ic % C);
    const int i = (int)(ic / C);
    Y[idx] = X[((size_t)uid[i] * NC + k) * C + c];
}

// P_i[l][ch] += sum_{c, k in l} X[i][c][k] * Y[i][c][k]   (one thread per surfel)
template <int NC>
__global__ void k_pair_accum(int n, int C, const float *__restrict__ X, const float *__restrict__ Y, float *P) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float acc[4][3] = {};
    for (int c = 0; c < C; ++c) {
        const size_t b = ((size_t)i * C + c) * NC;
#pragma unroll
        for (int k = 0; k < NC; ++k) acc[band_of(k)][c % 3] += X[b + k] * Y[b + k];
    }
    for (int l = 0; l < 4; ++l)
        for (int ch = 0; ch < 3; ++ch) P[(size_t)i * 12 + l * 3 + ch] += acc[l][ch];
}

template <int NC, int CT>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_bounce(SceneDev sc, RaysDev rays, int C,
                                                           const long long *__restrict__ src_off,
                                                           const int2 *__restrict__ tr, const float *__restrict__ vin,
                                                           float *__restrict__ vout, float *__restrict__ u) {
    const int j = blockIdx.x;
    const int col0 = blockIdx.y * CT;
    const int nd = rays.nd;
    const float w = 3.14159265358979f / (float)nd;
    float acc[NC][CT];
#pragma unroll
    for (int k = 0; k < NC; ++k)
#pragma unroll
        for (int c = 0; c < CT; ++c) acc[k][c] = 0.f;
    const long long e0 = src_off[j], e1 = src_off[j + 1];
    for (long long e = e0 + threadIdx.x; e < e1; e += ADJ_THREADS) {
        const int2 ent = __ldg(&tr[e]);
        const int r = ent.x;
        const float a = __int_as_float(ent.y);
        const int i = r / nd, q = r - i * nd;
        const float3 n = f3(__ldg(&sc.N4[i]));
        const float3 d = ray_dir(rays.seed, __ldg(&sc.uid[i]), q, rays.na, rays.nbs, f3(__ldg(&sc.FU[i])),
                                 f3(__ldg(&sc.FV[i])), n);
        float Yo[NC], Yi[NC];
        sh_eval<NC>(neg3(d), Yo);
        sh_eval<NC>(reflect_n(n, d), Yi);
        const float oi = __ldg(&sc.P[i].w) * w;
        const float *vi = vin + ((size_t)i * C + col0) * NC;
#pragma unroll
        for (int c = 0; c < CT; ++c) {
            const int ch = (col0 + c) % 3;
            float y = 0.f;
#pragma unroll
            for (int k = 0; k < NC; ++k) y += __ldg(&sc.cl[(size_t)i * 12 + band_of(k) * 3 + ch]) * Yi[k] * __ldg(&vi[c * NC + k]);
            y *= oi * a;
#pragma unroll
            for (int k = 0; k < NC; ++k) acc[k][c] += Yo[k] * y;
        }
    }
    __shared__ float red[ADJ_THREADS / 32][NC * CT];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < NC; ++k)
#pragma unroll
        for (int c = 0; c < CT; ++c) {
            float v = acc[k][c];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0) red[warp][k * CT + c] = v;
        }
    __syncthreads();
    for (int e = threadIdx.x; e < NC * CT; e += ADJ_THREADS) {
        float v = 0.f;
        for (int q = 0; q < ADJ_THREADS / 32; ++q) v += red[q][e];
        const int k = e / CT, c = e - k * CT;
        const size_t idx = ((size_t)j * C + col0 + c) * NC + k;
        vout[idx] = v;
        u[idx] += v;
    }
}

// Shadow rays: dL/dT_L = q = sum_{k,ch} u_i[L,ch][k] o_i c_{i,l,ch} Y_k(R_i w) I cos/r^2,
// dT/dalpha_m = -prod_{m' != m} (1 - alpha_m'); also adds u (x) Dgeo to P.
template <int NC>
__global__ void k_shadow_bwd(SceneDev sc, int nl, const float *__restrict__ lpos, const float *__restrict__ lint, int C,
                             const float *__restrict__ u, float *P, float *dop) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= sc.n * nl) return;
    const int i = tid / nl, lt = tid - i * nl;
    const float4 Pi = sc.P[i];
    const float3 o = f3(Pi), n = f3(sc.N4[i]);
    const float3 l = make_float3(lpos[3 * lt] - o.x, lpos[3 * lt + 1] - o.y, lpos[3 * lt + 2] - o.z);
    const float r = sqrtf(dot3(l, l));
    const float3 w = (1.f / r) * l;
    const float cs = dot3(n, w);
    if (!(cs > 0.f)) return;
    const float eps = *sc.eps_plane;
    float Tnz = 1.f;
    int nzero = 0;
    auto pass1 = [&](int j) {
        float t, g;
        if (!hit_surfel(sc, j, i, o, w, r, eps, t, g)) return;
        const float om = 1.f - __ldg(&sc.P[j].w) * g;
        if (om == 0.f) ++nzero;
        else Tnz *= om;
    };
    bvh_traverse(sc, o, w, r, pass1);
    const float T = nzero ? 0.f : Tnz;
    float Y[NC];
    sh_eval<NC>(reflect_n(n, w), Y);
    const float pre = cs / (r * r);
    const float *ui = u + ((size_t)i * C + lt * 3) * NC;
    float qv = 0.f;
    float acc[4][3] = {};
    for (int ch = 0; ch < 3; ++ch) {
        const float I = lint[3 * lt + ch];
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const float uy = ui[ch * NC + k] * Y[k] * I * pre;
            qv += uy * sc.cl[(size_t)i * 12 + band_of(k) * 3 + ch];
            acc[band_of(k)][ch] += uy * T;
        }
    }
    for (int b = 0; b < 4; ++b)
        for (int ch = 0; ch < 3; ++ch)
            if (acc[b][ch] != 0.f) atomicAdd(&P[(size_t)i * 12 + b * 3 + ch], acc[b][ch]);
    qv *= Pi.w;
    if (qv == 0.f || nzero > 1) return;
    auto pass2 = [&](int j) {
        float t, g;
        if (!hit_surfel(sc, j, i, o, w, r, eps, t, g)) return;
        const float om = 1.f - __ldg(&sc.P[j].w) * g;
        float others;
        if (nzero == 0) others = Tnz / om;
        else others = (om == 0.f) ? Tnz : 0.f;
        if (others != 0.f) atomicAdd(&dop[j], -qv * others * g);
    };
    bvh_traverse(sc, o, w, r, pass2);
}

// Hemisphere rays: g_h = sum_{a<n} sum_c y^(a)[c] Y(-d).B^(n-1-a)_{j_h}[c], then back to front
// R_{h-1} = alpha_h g_h + (1 - alpha_h) R_h and dL/do_{j_h} += T_h (g_h - R_h) G_h.
template <int NC, int CT>
__global__ void __launch_bounds__(128) k_hemi_opacity_bwd(SceneDev sc, RaysDev rays, int C, int nb, size_t A,
                                                          const float *__restrict__ V, const float *__restrict__ Bit,
                                                          float *dop) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int n_rays = sc.n * rays.nd;
    if (r >= n_rays) return;
    const int cnt = rays.cnt[r];
    if (cnt == 0) return;
    const int col0 = blockIdx.y * CT;
    const int i = r / rays.nd, q = r - i * rays.nd;
    const float3 n = f3(sc.N4[i]);
    const float3 d = ray_dir(rays.seed, sc.uid[i], q, rays.na, rays.nbs, f3(sc.FU[i]), f3(sc.FV[i]), n);
    float Yo[NC], Yi[NC];
    sh_eval<NC>(neg3(d), Yo);
    sh_eval<NC>(reflect_n(n, d), Yi);
    const float w = 3.14159265358979f / (float)rays.nd;
    const float oi = sc.P[i].w * w;
    const long long base = rays.warp_base[r >> 5] + (r & 31);
    float g[RGS_HMAX];
    for (int h = 0; h < cnt; ++h) g[h] = 0.f;
    for (int a = 0; a < nb; ++a) {
        float y[CT];
        const float *vi = V + A * a + ((size_t)i * C + col0) * NC;
#pragma unroll
        for (int c = 0; c < CT; ++c) {
            const int ch = (col0 + c) % 3;
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < NC; ++k) s += sc.cl[(size_t)i * 12 + band_of(k) * 3 + ch] * Yi[k] * vi[c * NC + k];
            y[c] = oi * s;
        }
        const float *Bb = Bit + A * (nb - 1 - a);
        for (int h = 0; h < cnt; ++h) {
            const int j = __ldg(&rays.rec_ja[base + (long long)h * 32]).x;
            const float *Bj = Bb + ((size_t)j * C + col0) * NC;
            float acc = 0.f;
#pragma unroll
            for (int c = 0; c < CT; ++c) {
                float s = 0.f;
#pragma unroll
                for (int k = 0; k < NC; ++k) s += Yo[k] * __ldg(&Bj[c * NC + k]);
                acc += y[c] * s;
            }
            g[h] += acc;
        }
    }
    // transmittance in front of each hit, then the back-to-front recurrence
    float Th[RGS_HMAX];
    float T = 1.f;
    for (int h = 0; h < cnt; ++h) {
        Th[h] = T;
        const int j = __ldg(&rays.rec_ja[base + (long long)h * 32]).x;
        T *= 1.f - __ldg(&sc.P[j].w) * __ldg(&rays.rec_g[base + (long long)h * 32]);
    }
    float R = 0.f;
    for (int h = cnt - 1; h >= 0; --h) {
        const int j = __ldg(&rays.rec_ja[base + (long long)h * 32]).x;
        const float G = __ldg(&rays.rec_g[base + (long long)h * 32]);
        const float alpha = __ldg(&sc.P[j].w) * G;
        const float da = Th[h] * (g[h] - R);
        if (da != 0.f) atomicAdd(&dop[j], da * G);
        R = alpha * g[h] + (1.f - alpha) * R;
    }
}

template <int NC>
__global__ void k_finalize(SceneDev sc, int C, const float *__restrict__ u, const float *__restrict__ P,
                           const float *__restrict__ kk, const float *__restrict__ dop_acc, float *dE, float *dad,
                           float *dop) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sc.n) return;
    const int ui = sc.uid[i];
    const float *Pi = P + (size_t)i * 12;
    if (dE) {
        for (int k = 0; k < NC; ++k)
            for (int ch = 0; ch < 3; ++ch) {
                float s = 0.f;
                for (int c = ch; c < C; c += 3) s += u[((size_t)i * C + c) * NC + k];
                dE[((size_t)ui * NC + k) * 3 + ch] = s;
            }
    }
    const float o = sc.P[i].w;
    if (dad)
        for (int ch = 0; ch < 3; ++ch) dad[(size_t)ui * 3 + ch] = 4.f * kk[i] * o * Pi[ch];
    if (dop) {
        float s = dop_acc[i];
        for (int q = 0; q < 12; ++q) s += sc.cl[(size_t)i * 12 + q] * Pi[q];
        dop[ui] = s;
    }
}

template <int NC>
rgs_status run_adjoint(rgs_transport *t, const float *g, float *dE, float *dad, float *dopo, cudaStream_t st) {
    const int n = t->n, C = t->C, nb = t->nb_last;
    const size_t A = t->arr();
    SceneDev sd = t->sc->dev();
    RaysDev rd = t->rays();
    const unsigned ga = (unsigned)((A + 255) / 256);
    // v^(0) = g (internal layout), u = v^(0), P = 0, dop = 0
    { ProfScope ps_("k_from_user", st); k_from_user<NC><<<ga, 256, 0, st>>>(n, C, t->sc->uid, g, t->v); }
    RGS_CUDA(cudaMemcpyAsync(t->u, t->v, sizeof(float) * A, cudaMemcpyDeviceToDevice, st));
    RGS_CUDA(cudaMemsetAsync(t->Pg, 0, sizeof(float) * 12 * (size_t)n, st));
    RGS_CUDA(cudaMemsetAsync(t->dop, 0, sizeof(float) * (size_t)n, st));
    RGS_LAUNCH("adjoint init");
    const unsigned gn = (unsigned)((n + 127) / 128);
    if (nb >= 1) { ProfScope ps_("k_pair_accum", st); k_pair_accum<NC><<<gn, 128, 0, st>>>(n, C, t->v, t->Q + A * (nb - 1), t->Pg); }
    for (int a = 1; a <= nb; ++a) {
        dim3 grid(n, C / 3);
        { ProfScope ps_("k_adj_bounce", st); k_adj_bounce<NC, 3><<<grid, ADJ_THREADS, 0, st>>>(sd, rd, C, t->src_off, t->tr, t->v + A * (a - 1),
                                                           t->v + A * a, t->u); }
        RGS_LAUNCH("adjoint bounce");
        if (a <= nb - 1) { ProfScope ps_("k_pair_accum", st); k_pair_accum<NC><<<gn, 128, 0, st>>>(n, C, t->v + A * a, t->Q + A * (nb - 1 - a), t->Pg); }
    }
    if (t->nl > 0) {
        const int nth = n * t->nl;
        { ProfScope ps_("k_shadow_bwd", st); k_shadow_bwd<NC><<<(nth + 127) / 128, 128, 0, st>>>(sd, t->nl, t->lpos, t->lint, C, t->u, t->Pg, t->dop); }
        RGS_LAUNCH("shadow backward");
    }
    if (nb >= 1 && dopo) {
        const long long n_rays = (long long)n * t->nd;
        dim3 grid((unsigned)((n_rays + 127) / 128), C / 3);
        { ProfScope ps_("k_hemi_opacity_bwd", st); k_hemi_opacity_bwd<NC, 3><<<grid, 128, 0, st>>>(sd, rd, C, nb, A, t->v, t->iters, t->dop); }
        RGS_LAUNCH("hemisphere opacity backward");
    }
    { ProfScope ps_("k_finalize", st); k_finalize<NC><<<gn, 128, 0, st>>>(sd, C, t->u, t->Pg, t->sc->kk, t->dop, dE, dad, dopo); }
    RGS_LAUNCH("finalize");
    return RGS_OK;
}

} // namespace

rgs_status rgs_adjoint_impl(rgs_transport *t, const float *g, float *dE, float *dad, float *dop, cudaStream_t st) {
    rgs_status r;
    const int nb = t->nb_last;
    const size_t A = t->arr();
    if (nb + 1 > t->v_cap) {
        if ((r = dev_alloc(&t->v, A * (nb + 1), &t->device_bytes)) != RGS_OK) return r;
        if ((r = dev_alloc(&t->u, A, &t->device_bytes)) != RGS_OK) return r;
        t->v_cap = nb + 1;
    }
    if (t->n > t->pg_cap) {
        if ((r = dev_alloc(&t->Pg, (size_t)t->n * 12, &t->device_bytes)) != RGS_OK) return r;
        if ((r = dev_alloc(&t->dop, (size_t)t->n, &t->device_bytes)) != RGS_OK) return r;
        t->pg_cap = t->n;
    }
    switch (t->nc) {
    case 1: return run_adjoint<1>(t, g, dE, dad, dop, st);
    case 4: return run_adjoint<4>(t, g, dE, dad, dop, st);
    case 9: return run_adjoint<9>(t, g, dE, dad, dop, st);
    default: return run_adjoint<16>(t, g, dE, dad, dop, st);
    }
}
