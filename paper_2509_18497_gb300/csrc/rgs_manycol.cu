// Many right-hand sides (many lights): kernels with one lane per column.
//
// With C columns the per-hit work of the gather is a row of C x nc coefficients of the
// source surfel.  The 3-column kernels (rgs_solve.cu, rgs_adjoint.cu) would re-read every
// hit record once per 3-column tile; here a warp takes one ray (or one transposed entry) at
// a time and its 32 lanes take 32 consecutive columns, so each hit is read once per
// 32-column tile and every row load is one contiguous 512-byte (BF16) or 1-KiB (FP32)
// warp access.  Which layout a launch uses is decided per kernel family by wide_bounce,
// wide_opacity and wide_adjoint (rgs_internal.cuh).
#include "rgs_bounce_body.cuh"

namespace {

// ------------------------------------------------------------------ forward bounce
template <int NC, class T>
__global__ void RGS_MCB_LB k_bounce_mc(SceneDev sc, RaysDev rays, int C, const T *__restrict__ Bg,
                                                         const float *__restrict__ Bprev, const float *__restrict__ S,
                                                         float *__restrict__ Qout, float *__restrict__ Bout,
                                                         __nv_bfloat16 *__restrict__ Bout16, double *norm2) {
    __shared__ float red[MC_WARPS * NC * 32];
    bounce_receiver_mc<NC, T>(sc, rays, C, Bg, Bprev, S, Qout, Bout, Bout16, norm2, blockIdx.x, blockIdx.y, red);
}

// ------------------------------------------------------------------ adjoint
// y_r[c] = (pi/nd) o_i sum_k' c_{i,l(k'),ch} Y_k'(R_i d_r) v_i[c][k'] for the 32 columns of
// tile `ct`, stored as dy[r*32 + lane]
template <int NC>
__global__ void __launch_bounds__(MC_THREADS) k_adj_ray_mc(SceneDev sc, RaysDev rays, int C, int ct,
                                                          const float *__restrict__ vin, float *dy) {
    const int i = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int col = ct * 32 + lane;
    const bool live = col < C;
    const int nd = rays.nd;
    const float3 n = f3(sc.N4[i]);
    float cv[NC]; // c_{i,l(k),ch(col)} * v_i[col][k] * o_i pi/nd
    {
        const float oi = alpha_center(sc, i) * (3.14159265358979f / (float)nd);
        float v[NC];
        if (live) load_col<NC>(vin + ((size_t)i * C + col) * NC, v);
#pragma unroll
        for (int k = 0; k < NC; ++k)
            cv[k] = live ? oi * __ldg(&sc.cl[(size_t)i * 12 + band_of(k) * 3 + col % 3]) * v[k] : 0.f;
    }
    for (int q = warp; q < nd; q += MC_WARPS) {
        const long long r = (long long)i * nd + q;
        const float3 d = f3(rays.dir[r]);
        float Yi[NC];
        sh_eval<NC>(reflect_n(n, d), Yi);
        float y = 0.f;
#pragma unroll
        for (int k = 0; k < NC; ++k) y += cv[k] * Yi[k];
        dy[r * 32 + lane] = y;
    }
}

// (K^T v)_j[c][k] = sum_{entries e on j} a_e Y_k(-d_e) y_e[c], one CTA per source j
template <int NC>
__global__ void RGS_MC_LB k_adj_src_mc(RaysDev rays, int C, int ct,
                                                          const long long *__restrict__ src_off,
                                                          const int2 *__restrict__ tr, const float *__restrict__ dy,
                                                          float *__restrict__ vout, float *__restrict__ u, int j0,
                                                          long long ebase) {
    const int j = j0 + blockIdx.x; // sources j0 .. of this index part; its entries start at ebase
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float acc[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) acc[k] = 0.f;
    const long long e0 = src_off[j] - ebase, e1 = src_off[j + 1] - ebase;
    for (long long e = e0 + warp; e < e1; e += MC_WARPS) {
        const int2 ent = __ldg(&tr[e]);
        const float4 d4 = __ldg(&rays.dir[ent.x]);
        float Yo[NC];
        sh_eval<NC>(make_float3(-d4.x, -d4.y, -d4.z), Yo);
        const float y = __int_as_float(ent.y) * __ldg(&dy[(long long)ent.x * 32 + lane]);
#pragma unroll
        for (int k = 0; k < NC; ++k) acc[k] += Yo[k] * y;
    }
    __shared__ float red[MC_WARPS][NC][32];
#pragma unroll
    for (int k = 0; k < NC; ++k) red[warp][k][lane] = acc[k];
    __syncthreads();
    for (int e = threadIdx.x; e < NC * 32; e += MC_THREADS) {
        const int k = e >> 5, c = e & 31;
        const int cc = ct * 32 + c;
        if (cc >= C) continue;
        float v = 0.f;
#pragma unroll
        for (int q = 0; q < MC_WARPS; ++q) v += red[q][k][c];
        const size_t idx = ((size_t)j * C + cc) * NC + k;
        vout[idx] = v;
        u[idx] += v;
    }
}

// opacity backward: per hit g_h (partial over this column tile and iterate chunk)
// accumulated into gh[slot]; a warp per ray, lanes over columns
template <int NC, int NA, class T>
__global__ void RGS_MC_LB k_opacity_g_mc(SceneDev sc, RaysDev rays, int C, int ct, int na,
                                                            OpaSet<T, NA> it, float *gh, bool first) {
    constexpr int RS = row_stride<NC, T>();
    constexpr bool COOP = sizeof(T) == 4 && NC == 16; // whole-tile reads (TileDot)
    const int warp_g = (int)((blockIdx.x * (size_t)MC_THREADS + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const int n_rays = sc.n * rays.nd;
    if (warp_g >= n_rays) return; // whole warps
    const int r = warp_g;
    const int cnt = rays.cnt[r];
    if (cnt == 0) return;
    int own = lane; // the tile column whose terms this lane forms
    if constexpr (COOP) own = TileDot<T, NC>::own(lane);
    const int col = ct * 32 + own;
    const bool live = col < C;
    const int colc = live ? col : C - 1;
    const int ncols = min(32, C - ct * 32);
    const int i = r / rays.nd;
    const float3 n = f3(sc.N4[i]);
    const float3 d = f3(rays.dir[r]);
    float Yo[NC], y[NA];
    {
        float Yi[NC];
        sh_eval<NC>(neg3(d), Yo);
        sh_eval<NC>(reflect_n(n, d), Yi);
        const float oi = alpha_center(sc, i) * (3.14159265358979f / (float)rays.nd);
#pragma unroll
        for (int aa = 0; aa < NA; ++aa) {
            float s = 0.f;
            if (aa < na && live) {
                float v[NC];
                load_col<NC>(it.v[aa] + ((size_t)i * C + col) * NC, v);
#pragma unroll
                for (int k = 0; k < NC; ++k) s += __ldg(&sc.cl[(size_t)i * 12 + band_of(k) * 3 + col % 3]) * Yi[k] * v[k];
            }
            y[aa] = oi * s;
        }
    }
    const long long base = rays.off[r];
    [[maybe_unused]] float ys[4]; // this lane's quarter of Y(-d) (TileDot)
    if constexpr (COOP) TileDot<T, NC>::pick(Yo, lane, ys);
    for (int h = 0; h < cnt; ++h) {
        const int j = __ldg(&rays.rec_ja[base + h]).x;
        float acc = 0.f;
#pragma unroll
        for (int aa = 0; aa < NA; ++aa) {
            if (aa < na) {
                float s = 0.f;
                if constexpr (COOP) {
                    s = TileDot<T, NC>::dot(it.b[aa] + ((size_t)j * C + ct * 32) * RS, ncols, lane, ys);
                } else {
                    float v[NC];
                    load_col<NC>(it.b[aa] + ((size_t)j * C + colc) * RS, v);
#pragma unroll
                    for (int k = 0; k < NC; ++k) s += Yo[k] * v[k];
                }
                acc += y[aa] * s;
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) gh[base + h] = first ? acc : gh[base + h] + acc;
    }
}

} // namespace

// ------------------------------------------------------------------ launchers
template <int NC>
rgs_status mc_bounce(const rgs_transport *t, SceneDev sd, RaysDev rd, bool rows16, const float *Bprev,
                     const __nv_bfloat16 *Bprev16, const float *S, float *Q, float *Bout, __nv_bfloat16 *Bout16,
                     double *norm2, cudaStream_t st) {
    dim3 grid(t->n, (t->C + 31) / 32);
    if (rows16) {
        ProfScope ps_("k_bounce_mc", st);
        k_bounce_mc<NC, __nv_bfloat16><<<grid, MC_THREADS, 0, st>>>(sd, rd, t->C, Bprev16, Bprev, S, Q, Bout, Bout16, norm2);
    } else {
        ProfScope ps_("k_bounce_mc", st);
        k_bounce_mc<NC, float><<<grid, MC_THREADS, 0, st>>>(sd, rd, t->C, Bprev, Bprev, S, Q, Bout, Bout16, norm2);
    }
    RGS_LAUNCH("bounce_mc");
    return RGS_OK;
}

template <int NC>
rgs_status mc_adjoint_bounce(rgs_transport *t, SceneDev sd, RaysDev rd, const float *vin, float *vout, int j0, int j1,
                             long long ebase, cudaStream_t st) {
    for (int ct = 0; ct * 32 < t->C; ++ct) {
        { ProfScope ps_("k_adj_ray_mc", st); k_adj_ray_mc<NC><<<t->n, MC_THREADS, 0, st>>>(sd, rd, t->C, ct, vin, t->dy_mc); }
        { ProfScope ps_("k_adj_src_mc", st); k_adj_src_mc<NC><<<j1 - j0, MC_THREADS, 0, st>>>(rd, t->C, ct, t->src_off, t->tr, t->dy_mc, vout, t->u, j0, ebase); }
    }
    RGS_LAUNCH("adjoint bounce mc");
    return RGS_OK;
}

template <int NC>
rgs_status mc_opacity(rgs_transport *t, SceneDev sd, RaysDev rd, int na, const float *const *v, const float *const *Bf,
                      const __nv_bfloat16 *const *Bh, bool first, cudaStream_t st) {
    constexpr int NA = 4;
    const long long n_rays = (long long)t->n * t->nd;
    const unsigned grid = (unsigned)((n_rays * 32 + MC_THREADS - 1) / MC_THREADS);
    OpaSet<float, NA> sf = {};
    OpaSet<__nv_bfloat16, NA> sh = {};
    for (int a = 0; a < na; ++a) {
        sf.v[a] = sh.v[a] = v[a];
        sf.b[a] = Bf[a];
        sh.b[a] = Bh ? Bh[a] : nullptr;
    }
    for (int ct = 0; ct * 32 < t->C; ++ct) {
        if (Bh) {
            ProfScope ps_("k_opacity_g_mc", st);
            k_opacity_g_mc<NC, NA, __nv_bfloat16><<<grid, MC_THREADS, 0, st>>>(sd, rd, t->C, ct, na, sh, t->gh, first && ct == 0);
        } else {
            ProfScope ps_("k_opacity_g_mc", st);
            k_opacity_g_mc<NC, NA, float><<<grid, MC_THREADS, 0, st>>>(sd, rd, t->C, ct, na, sf, t->gh, first && ct == 0);
        }
    }
    RGS_LAUNCH("opacity mc");
    return RGS_OK;
}

#define RGS_MC_INSTANTIATE(NC)                                                                                         \
    template rgs_status mc_bounce<NC>(const rgs_transport *, SceneDev, RaysDev, bool, const float *,                   \
                                      const __nv_bfloat16 *, const float *, float *, float *, __nv_bfloat16 *,         \
                                      double *, cudaStream_t);                                                         \
    template rgs_status mc_adjoint_bounce<NC>(rgs_transport *, SceneDev, RaysDev, const float *, float *, int, int,    \
                                              long long, cudaStream_t);                                                \
    template rgs_status mc_opacity<NC>(rgs_transport *, SceneDev, RaysDev, int, const float *const *,                 \
                                       const float *const *, const __nv_bfloat16 *const *, bool, cudaStream_t);
RGS_MC_INSTANTIATE(1)
RGS_MC_INSTANTIATE(4)
RGS_MC_INSTANTIATE(9)
RGS_MC_INSTANTIATE(16)
