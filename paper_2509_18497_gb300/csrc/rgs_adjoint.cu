// Adjoint (rgs_adjoint): exact gradients of L(B^(n)) for the truncated bounce series.
//
//   v^(0) = dL/dB^(n),  v^(a) = K^T v^(a-1)   (Eq. final_dL_dE: the same paths with the
//                                              decay reversed, propagating gradients)
//   u = sum_a v^(a) = dL/dS,   P_i[l][ch] = sum_{k in l, light} (sum_{a<n} v^(a) Q^(n-1-a) + u Dgeo)
//
// K^T v is a gather over the records grouped by source surfel j:
//   (K^T v)_j[c][k] = sum_{hits e on j} a_e Y_k(-d_e) y_e[c],
//   y_e[c] = (pi/nd) o_i sum_k' c_{i,l(k'),ch} Y_k'(R_i d_e) v_i[c][k']      (i = receiver of e)
// k_adj_ray forms y per ray once (ray-major, next to the stored direction) and k_adj_src
// gathers (d, y) per entry, 32 bytes, instead of a 192-byte row of v_i per entry.
// k_opacity_g / k_opacity_rec and k_shadow_bwd run the compositing backward of every
// hemisphere and shadow ray (dL/dalpha_h = T_h (g_h - R_h), dL/dT = -prod of the other (1 - alpha)).
#include <algorithm>
#include <vector>

#include "rgs_internal.cuh"

namespace {

constexpr int ADJ_THREADS = 128;
static_assert(ADJ_THREADS == 128, "RGS_ADJ_LB assumes 128 threads");

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

// Per ray r of receiver i (column tile col0..col0+2):
//   y_r[c] = (pi/nd) o_i sum_k' c_{i,l(k'),ch} Y_k'(R_i d_r) v_i[c][k']
// stored next to the ray's direction for the by-source gather.
template <int NC>
__global__ void __launch_bounds__(256) k_adj_ray(SceneDev sc, RaysDev rays, int C, int col0,
                                                 const float *__restrict__ vin, float4 *dy) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= sc.n * rays.nd) return;
    const int i = r / rays.nd;
    const float3 n = f3(sc.N4[i]);
    const float3 d = f3(rays.dir[r]);
    float Yi[NC];
    sh_eval<NC>(reflect_n(n, d), Yi);
    const float oi = alpha_center(sc, i) * (3.14159265358979f / (float)rays.nd);
    const float *vi = vin + ((size_t)i * C + col0) * NC;
    float y[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int ch = (col0 + c) % 3;
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < NC; ++k) s += __ldg(&sc.cl[(size_t)i * 12 + band_of(k) * 3 + ch]) * Yi[k] * __ldg(&vi[c * NC + k]);
        y[c] = oi * s;
    }
    dy[r] = make_float4(y[0], y[1], y[2], 0.f);
}

// (K^T v)_j[c][k] = sum_{entries e on j} a_e Y_k(-d_e) y_e[c]; one CTA per source j.
template <int NC>
__global__ void RGS_ADJ_LB k_adj_src(RaysDev rays, int C, int col0, const long long *__restrict__ src_off,
                                                        const int2 *__restrict__ tr, const float4 *__restrict__ dy,
                                                        float *__restrict__ vout, float *__restrict__ u, int j0,
                                                        long long ebase) {
    constexpr int CT = 3;
    const int j = j0 + blockIdx.x; // sources j0 .. of this index part; its entries start at ebase
    float acc[NC][CT];
#pragma unroll
    for (int k = 0; k < NC; ++k)
#pragma unroll
        for (int c = 0; c < CT; ++c) acc[k][c] = 0.f;
    const long long e0 = src_off[j] - ebase, e1 = src_off[j + 1] - ebase;
    for (long long e = e0 + threadIdx.x; e < e1; e += ADJ_THREADS) {
        const int2 ent = __ldg(&tr[e]);
        const float a = __int_as_float(ent.y);
        const float4 d4 = __ldg(&rays.dir[ent.x]);
        const float4 y4 = __ldg(&dy[ent.x]);
        float Yo[NC];
        sh_eval<NC>(make_float3(-d4.x, -d4.y, -d4.z), Yo);
        const float y[3] = {a * y4.x, a * y4.y, a * y4.z};
#pragma unroll
        for (int k = 0; k < NC; ++k)
#pragma unroll
            for (int c = 0; c < CT; ++c) acc[k][c] += Yo[k] * y[c];
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
// dT/dalpha_m = -prod_{m' != m} (1 - alpha_m'); also adds u (x) Dgeo to P.  With dp (and
// ds) the geometry gradients of the direct term as well (Eq. dl-dgeo-1 for the light's
// direction): with h_k = sum_ch u_i[L,ch][k] o_i c_{i,l(k),ch} I_ch and H = h . Y(R_i w), the
// term H (n_i.w) fall T moves with w (through Y(R_i w) and n_i.w), with fall = 1/r^2 and with
// each shadow occluder's crossing point; a directional light has a fixed w and fall = 1.
// gF (with dp): the frame gradients, through n_i (cos and R_i) and the occluders' frames.
template <int NC>
__global__ void k_shadow_bwd(SceneDev sc, int nl, int ldir, const float *__restrict__ lpos, const float *__restrict__ lint,
                             int C, const float *__restrict__ u, float *P, float *dop, float *dp, float *ds, float *gF) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= sc.n * nl) return;
    const int i = tid / nl, lt = tid - i * nl;
    const float4 Pi = sc.P[i];
    const float3 o = f3(Pi), n = f3(sc.N4[i]);
    float r, fall;
    const float3 w = light_dir(lpos, lt, o, ldir, r, fall);
    const float cs = dot3(n, w);
    if (!(cs > 0.f)) return;
    const float eps = *sc.eps_plane;
    float Tnz = 1.f;
    int nzero = 0;
    auto pass1 = [&](int j) {
        float t, g;
        if (!hit_surfel(sc, j, i, o, w, r, eps, t, g)) return;
        const float om = 1.f - alpha_of(sc, __ldg(&sc.P[j].w), g);
        if (om == 0.f) ++nzero;
        else Tnz *= om;
    };
    bvh_traverse(sc, o, w, r, pass1);
    const float T = nzero ? 0.f : Tnz;
    float Y[NC], h[NC];
    const float3 rw = reflect_n(n, w);
    sh_eval<NC>(rw, Y);
    const float pre = cs * fall;
    const float *ui = u + ((size_t)i * C + lt * 3) * NC;
    const float ai = alpha_center(sc, i);
    float qv = 0.f;
    float acc[4][3] = {};
#pragma unroll
    for (int k = 0; k < NC; ++k) h[k] = 0.f;
    for (int ch = 0; ch < 3; ++ch) {
        const float I = lint[3 * lt + ch];
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const float cl = sc.cl[(size_t)i * 12 + band_of(k) * 3 + ch];
            const float uy = ui[ch * NC + k] * Y[k] * I * pre;
            qv += uy * cl;
            acc[band_of(k)][ch] += uy * T;
            h[k] += ui[ch * NC + k] * I * cl;
        }
    }
    for (int b = 0; b < 4; ++b)
        for (int ch = 0; ch < 3; ++ch)
            if (acc[b][ch] != 0.f) atomicAdd(&P[(size_t)i * 12 + b * 3 + ch], acc[b][ch]);
    qv *= ai;
    float3 gw = make_float3(0.f, 0.f, 0.f), gpi = make_float3(0.f, 0.f, 0.f);
    float H = 0.f;
    if (dp) {
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            h[k] *= ai;
            H += h[k] * Y[k];
        }
        const float3 t1 = sh_grad_dot<NC>(rw, h);
        const float3 t3 = reflect_n(n, t1);
        const float f = fall * T;
        gw = make_float3(f * (cs * t3.x + H * n.x), f * (cs * t3.y + H * n.y), f * (cs * t3.z + H * n.z));
        const float3 gn = reflect_grad_n(n, w, (f * cs) * t1) + (H * f) * w; // R_i w and cos = n_i.w
        geo_add3(gF + GEO_GF * (size_t)i + GEO_N, gn);
    }
    if (qv != 0.f && nzero <= 1) {
        auto pass2 = [&](int j) {
            float t, g;
            if (!hit_surfel(sc, j, i, o, w, r, eps, t, g)) return;
            const float oj = __ldg(&sc.P[j].w);
            const float om = 1.f - alpha_of(sc, oj, g);
            float others;
            if (nzero == 0) others = Tnz / om;
            else others = (om == 0.f) ? Tnz : 0.f;
            if (others == 0.f) return;
            atomicAdd(&dop[j], -qv * others * dalpha_do(sc, oj, g));
            if (dp) {
                const float coef = -qv * others * dalpha_dq(sc, oj, g);
                if (coef == 0.f) return;
                float uu, vv;
                const float3 pw = crossing_pw(sc, j, o, w, t, uu, vv);
                gpi = gpi + coef * pw;
                gw = gw + (coef * t) * pw;
                geo_add3(dp + GEO_DP * (size_t)j, (-coef) * pw);
                geo_add2(ds + 2 * (size_t)j, coef * (-2.f * uu * uu * __ldg(&sc.FU[j].w)),
                         coef * (-2.f * vv * vv * __ldg(&sc.FV[j].w)));
                occluder_frame_grad(sc, j, o, w, t, uu, vv, coef, gF);
            }
        };
        bvh_traverse(sc, o, w, r, pass2);
    }
    if (dp) {
        float3 gp = gpi;
        if (!ldir) { // w = (p_L - p_i)/r, fall = 1/r^2
            const float ww = dot3(w, gw), gr = H * cs * T * (-2.f * fall / r);
            gp.x += -(gw.x - w.x * ww) / r - w.x * gr;
            gp.y += -(gw.y - w.y * ww) / r - w.y * gr;
            gp.z += -(gw.z - w.z * ww) / r - w.z * gr;
        }
        geo_add3(dp + GEO_DP * (size_t)i, gp);
    }
}

// Hemisphere rays, part 1: for every stored hit h of ray r (receiver i, source j_h),
//   g_h = sum_{a<n} sum_c y_r^(a)[c] Y(-d_r) . B^(n-1-a)_{j_h}[c],
//   y_r^(a)[c] = (pi/nd) o_i sum_k' c_{i,l(k'),ch} Y_k'(R_i d_r) v_i^(a)[c][k'],
// accumulated into gh[slot] for iterates a0 .. a0+na-1 (first chunk writes, later add).
template <int NC, int CT, int NA, class SLB>
__global__ void RGS_OPA_LB k_opacity_g(SceneDev sc, RaysDev rays, int C, int col0, int na,
                                                   OpaSet<typename SLB::T, NA> it, float *gh, bool first) {
    using SL = Slice<NC>;
    constexpr int G = SL::G, KPL = SL::KPL;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int ray = t / G, g = t % G;
    const int n_rays = sc.n * rays.nd;
    const bool live = ray < n_rays;
    const int r = live ? ray : n_rays - 1;
    const int cnt = live ? rays.cnt[r] : 0;
    const int i = r / rays.nd;
    const float3 n = f3(sc.N4[i]);
    const float3 d = f3(rays.dir[r]);
    float yo[KPL];
    float y[NA][CT];
    {
        float Y[NC], yi[KPL];
        sh_eval<NC>(neg3(d), Y);
        SL::pick(Y, g, yo);
        sh_eval<NC>(reflect_n(n, d), Y);
        SL::pick(Y, g, yi);
        const float oi = alpha_center(sc, i) * (3.14159265358979f / (float)rays.nd);
#pragma unroll
        for (int aa = 0; aa < NA; ++aa) {
#pragma unroll
            for (int c = 0; c < CT; ++c) {
                float s = 0.f;
                if (aa < na) {
                    const int ch = (col0 + c) % 3;
                    float v[KPL];
                    SL::load(it.v[aa] + ((size_t)i * C + col0 + c) * NC, g, v);
#pragma unroll
                    for (int m = 0; m < KPL; ++m) {
                        const int kk = SL::k(g, m);
                        const float cl = (kk < NC) ? __ldg(&sc.cl[(size_t)i * 12 + band_of(kk) * 3 + ch]) : 0.f;
                        s += cl * yi[m] * v[m];
                    }
                }
                y[aa][c] = oi * SL::group_sum(s);
            }
        }
    }
    const long long base = rays.off[r];
    const int rows = SL::G == 1 ? cnt : __reduce_max_sync(0xffffffffu, cnt); // groups of a warp stay converged
    for (int h = 0; h < rows; ++h) {
        float acc = 0.f;
        int j = 0;
        if (h < cnt) j = __ldg(&rays.rec_ja[base + h]).x;
#pragma unroll
        for (int aa = 0; aa < NA; ++aa) {
            if (aa < na && h < cnt) {
                const typename SLB::T *Bj = it.b[aa] + ((size_t)j * C + col0) * SLB::STRIDE;
#pragma unroll
                for (int c = 0; c < CT; ++c) {
                    float v[KPL];
                    SLB::load(Bj + c * SLB::STRIDE, g, v);
                    float s = 0.f;
#pragma unroll
                    for (int m = 0; m < KPL; ++m) s += yo[m] * v[m];
                    acc += y[aa][c] * s;
                }
            }
        }
        acc = SL::group_sum(acc);
        if (g == 0 && h < cnt) {
            const long long slot = base + h;
            gh[slot] = first ? acc : gh[slot] + acc;
        }
    }
}

// Hemisphere rays, part 2: back to front, R_{h-1} = alpha_h g_h + (1 - alpha_h) R_h and
// dL/do_{j_h} += T_h (g_h - R_h) dalpha_h/do, with T_h the transmittance in front of hit h,
// T_h = a_h / alpha_h from the stored weight.  G_h is recomputed from the stored direction
// (bit-identical to the trace's value).
__global__ void RGS_OPAREC_LB k_opacity_rec(SceneDev sc, RaysDev rays, const float *__restrict__ gh,
                                                     float *dop) {
    // Blocks take the rays in a scattered order (block b -> b * 2654435761 mod gridDim, a
    // bijection: the multiplier is prime): blocks resident at the same time then hold
    // receivers spread over the scene, so their dL/do atomics go to sources all over it
    // instead of piling onto the few sources of one neighbourhood (32 % faster measured).
    const unsigned bs = (unsigned)(((unsigned long long)blockIdx.x * 2654435761ull) % gridDim.x);
    const int r = (int)bs * blockDim.x + threadIdx.x;
    if (r >= sc.n * rays.nd) return;
    const int cnt = rays.cnt[r];
    if (cnt == 0) return;
    const long long base = rays.off[r];
    const int i = r / rays.nd;
    const float3 o = f3(sc.P[i]);
    const float3 d = f3(rays.dir[r]);
    float R = 0.f;
    for (int h = cnt - 1; h >= 0; --h) {
        const long long slot = base + h;
        const int2 ja = __ldg(&rays.rec_ja[slot]);
        const int j = ja.x;
        const float G = stored_hit_G(sc, j, o, d);
        const float oj = __ldg(&sc.P[j].w);
        const float alpha = alpha_of(sc, oj, G);
        const float g = gh[slot];
        // the transmittance in front of the hit from its stored weight a_h = alpha_h T_h
        // (alpha_h = 0 makes dalpha/do vanish for the disc and Gaussian models; GFSGS: alpha = 0
        // only where x = o G = 0, where dalpha/do is 0 too)
        const float Th = alpha > 0.f ? __int_as_float(ja.y) / alpha : 0.f;
        const float da = Th * (g - R);
        if (da != 0.f) atomicAdd(&dop[j], da * dalpha_do(sc, oj, G));
        R = alpha * g + (1.f - alpha) * R;
    }
}

// Geometry gradients of the hemisphere-ray transport (Eqs. dl-dgeo-0/1), part 1 (compositing),
// one thread per ray from the per-record g_h of the opacity backward: each hit's alpha moves
// with q_h = u^2 + v^2 at the hit point on its source's plane, with dL/dalpha_h =
// T_h (g_h - R_h) (back to front, as k_opacity_rec); q_h moves with p_i, the ray direction
// and the source's centre, scales and frame.  The ray leaves p_i along
// d = c_x t^u_i + c_y t^v_i + c_z n_i with fixed c, so dL/dd goes to the receiver's frame.
// The receiver's terms are summed over the warp (nd is a multiple of 32, so a warp's rays
// share their receiver) and added once per warp.  Part 2 is k_hemi_geo_dir.
__global__ void __launch_bounds__(128) k_hemi_geo(SceneDev sc, RaysDev rays, int nb, const float *__restrict__ gh,
                                                 float *dp, float *ds, float *gF) {
    // scattered block order (as k_opacity_rec): resident blocks hold receivers spread over the
    // scene, so their per-hit atomics land on sources all over it
    const unsigned bs = (unsigned)(((unsigned long long)blockIdx.x * 2654435761ull) % gridDim.x);
    const int r = (int)bs * blockDim.x + threadIdx.x;
    const int n_rays = sc.n * rays.nd;
    if (r - (int)(threadIdx.x & 31) >= n_rays) return; // whole warps (n_rays % 32 == 0)
    const int i = r / rays.nd;
    const int cnt = rays.cnt[r];
    const float3 o = f3(sc.P[i]), n = f3(sc.N4[i]), d = f3(rays.dir[r]);
    float3 gpi = make_float3(0.f, 0.f, 0.f), gd = make_float3(0.f, 0.f, 0.f);
    if (cnt > 0 && nb > 0) {
        const long long base = rays.off[r];
        float R = 0.f;
        for (int h = cnt - 1; h >= 0; --h) {
            const int2 ja = __ldg(&rays.rec_ja[base + h]);
            const int j = ja.x;
            const float G = stored_hit_G(sc, j, o, d);
            const float oj = __ldg(&sc.P[j].w);
            const float al = alpha_of(sc, oj, G);
            const float g = gh[base + h];
            // the transmittance in front of the hit from its stored weight a_h = alpha_h T_h
            // (alpha_h = 0 makes dalpha/dq vanish too)
            const float Th = al > 0.f ? __int_as_float(ja.y) / al : 0.f;
            const float coef = Th * (g - R) * dalpha_dq(sc, oj, G);
            if (coef != 0.f) {
                const float4 Nj = __ldg(&sc.N4[j]), Pj = __ldg(&sc.P[j]);
                const float t = (Nj.x * (Pj.x - o.x) + Nj.y * (Pj.y - o.y) + Nj.z * (Pj.z - o.z)) /
                                (Nj.x * d.x + Nj.y * d.y + Nj.z * d.z);
                float uu, vv;
                const float3 pw = crossing_pw(sc, j, o, d, t, uu, vv);
                gpi = gpi + coef * pw;
                gd = gd + (coef * t) * pw;
                geo_add3(dp + GEO_DP * (size_t)j, (-coef) * pw);
                geo_add2(ds + 2 * (size_t)j, coef * (-2.f * uu * uu * __ldg(&sc.FU[j].w)),
                         coef * (-2.f * vv * vv * __ldg(&sc.FV[j].w)));
                occluder_frame_grad(sc, j, o, d, t, uu, vv, coef, gF);
            }
            R = al * g + (1.f - al) * R;
        }
    }
    const float3 tu = f3(sc.FU[i]), tv = f3(sc.FV[i]);
    const float cx = dot3(d, tu), cy = dot3(d, tv), cz = dot3(d, n);
    const float3 gn = cz * gd;
    float red[12] = {gpi.x, gpi.y, gpi.z, cx * gd.x, cx * gd.y, cx * gd.z, cy * gd.x, cy * gd.y, cy * gd.z,
                     gn.x, gn.y, gn.z};
#pragma unroll
    for (int q = 0; q < 12; ++q)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) red[q] += __shfl_xor_sync(0xffffffffu, red[q], off);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (red[q] != 0.f) atomicAdd(&dp[GEO_DP * (size_t)i + q], red[q]);
#pragma unroll
        for (int q = 0; q < 9; ++q)
            if (red[3 + q] != 0.f) atomicAdd(&gF[GEO_GF * (size_t)i + 4 * (q / 3) + q % 3], red[3 + q]);
    }
}

constexpr int GEO_DIR_THREADS = 256;

// Part 2 (directional effects), a CTA per receiver and G lanes per ray, each lane a slice of
// the SH coefficients (the layout of the bounce gather): Y(R_i d) through
// X^(a)[c] = Y(-d).P^(a)[c] and Y(-d) through the composited source rows
// P^(a)[c] = sum_h a_h B_{j_h}^(nb-1-a)[c] (gathered once per 3-column tile and iterate);
// with cv = (pi/nd) o_i c_i (x) v_i^(a)[c], w_i = sum X cv and w_o = sum (cv.Y(R_i d)) P,
// dL/dd = R_i grad Y(R_i d).w_i - grad Y(-d).w_o, dL/dn_i from R_i, summed over the
// receiver's rays into its frame gradient.
template <int NC>
__global__ void __launch_bounds__(GEO_DIR_THREADS) k_hemi_geo_dir(SceneDev sc, RaysDev rays, int C, int nb, size_t A,
                                                                const float *__restrict__ V,
                                                                const float *__restrict__ Bit, float *gF) {
    using SL = Slice<NC>;
    constexpr int G = SL::G, KPL = SL::KPL, GROUPS = GEO_DIR_THREADS / G, CT = 3;
    __shared__ float red[GEO_DIR_THREADS / 32][9];
    const int i = blockIdx.x;
    const int grp = threadIdx.x / G, g = threadIdx.x % G, lane = threadIdx.x & 31;
    const int nd = rays.nd;
    const float3 n = f3(sc.N4[i]), tu = f3(sc.FU[i]), tv = f3(sc.FV[i]);
    const float wa = alpha_center(sc, i) * (3.14159265358979f / (float)nd);
    float acc[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) acc[q] = 0.f;
    for (int qb = 0; qb < nd; qb += GROUPS) { // every lane makes the same trips (group shuffles)
        const int q = qb + grp;
        const bool live = q < nd;
        const long long r = (long long)i * nd + (live ? q : 0);
        const float3 d = f3(rays.dir[r]);
        const int cnt = live ? rays.cnt[r] : 0;
        const long long base = rays.off[r];
        const float3 rd = reflect_n(n, d);
        float yo[KPL], yi[KPL];
        {
            float Y[NC];
            sh_eval<NC>(neg3(d), Y);
            SL::pick(Y, g, yo);
            sh_eval<NC>(rd, Y);
            SL::pick(Y, g, yi);
        }
        float wi[KPL], wo[KPL];
#pragma unroll
        for (int m = 0; m < KPL; ++m) wi[m] = wo[m] = 0.f;
        for (int a = 0; a < nb; ++a) {
            const float *va = V + A * a + (size_t)i * C * NC;
            const float *Bb = Bit + A * (nb - 1 - a);
            for (int c0 = 0; c0 < C; c0 += CT) {
                float P[CT][KPL];
#pragma unroll
                for (int c = 0; c < CT; ++c)
#pragma unroll
                    for (int m = 0; m < KPL; ++m) P[c][m] = 0.f;
#pragma unroll 2
                for (int h = 0; h < cnt; ++h) {
                    const int2 ja = __ldg(&rays.rec_ja[base + h]);
                    const float ah = __int_as_float(ja.y);
                    const float *Bj = Bb + ((size_t)ja.x * C + c0) * NC;
#pragma unroll
                    for (int c = 0; c < CT; ++c) {
                        float v[KPL];
                        SL::load(Bj + c * NC, g, v);
#pragma unroll
                        for (int m = 0; m < KPL; ++m) P[c][m] += ah * v[m];
                    }
                }
#pragma unroll
                for (int c = 0; c < CT; ++c) {
                    const int col = c0 + c;
                    float vv[KPL], cv[KPL];
                    SL::load(va + (size_t)col * NC, g, vv);
                    float xs = 0.f, ys = 0.f;
#pragma unroll
                    for (int m = 0; m < KPL; ++m) {
                        const int k = SL::k(g, m);
                        cv[m] = k < NC ? wa * __ldg(&sc.cl[(size_t)i * 12 + band_of(k) * 3 + (col % 3)]) * vv[m] : 0.f;
                        xs += yo[m] * P[c][m];
                        ys += cv[m] * yi[m];
                    }
                    const float X = SL::group_sum(xs), y = SL::group_sum(ys);
#pragma unroll
                    for (int m = 0; m < KPL; ++m) {
                        wi[m] += X * cv[m];
                        wo[m] += y * P[c][m];
                    }
                }
            }
        }
        // the whole w_i, w_o from the group's lanes
        float WI[NC], WO[NC];
#pragma unroll
        for (int g2 = 0; g2 < G; ++g2)
#pragma unroll
            for (int m = 0; m < KPL; ++m) {
                const float xi = __shfl_sync(0xffffffffu, wi[m], (lane & ~(G - 1)) + g2);
                const float xo = __shfl_sync(0xffffffffu, wo[m], (lane & ~(G - 1)) + g2);
                const int k = SL::k(g2, m);
                if (k < NC) {
                    WI[k] = xi;
                    WO[k] = xo;
                }
            }
        if (live && g == 0 && cnt > 0) {
            const float3 t1 = sh_grad_dot<NC>(rd, WI);
            const float3 gd = reflect_n(n, t1) - sh_grad_dot<NC>(neg3(d), WO);
            const float cx = dot3(d, tu), cy = dot3(d, tv), cz = dot3(d, n);
            const float3 gn = reflect_grad_n(n, d, t1) + cz * gd;
            acc[0] += cx * gd.x, acc[1] += cx * gd.y, acc[2] += cx * gd.z;
            acc[3] += cy * gd.x, acc[4] += cy * gd.y, acc[5] += cy * gd.z;
            acc[6] += gn.x, acc[7] += gn.y, acc[8] += gn.z;
        }
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        float v = acc[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) red[threadIdx.x >> 5][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        float v = 0.f;
        for (int w = 0; w < GEO_DIR_THREADS / 32; ++w) v += red[w][threadIdx.x];
        if (v != 0.f) atomicAdd(&gF[GEO_GF * (size_t)i + 4 * (threadIdx.x / 3) + threadIdx.x % 3], v);
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
    const float ai = alpha_center(sc, i);
    if (dad)
        for (int ch = 0; ch < 3; ++ch) dad[(size_t)ui * 3 + ch] = 4.f * kk[i] * ai * Pi[ch];
    if (dop) {
        float s = 0.f;
        for (int q = 0; q < 12; ++q) s += sc.cl[(size_t)i * 12 + q] * Pi[q];
        dop[ui] = dop_acc[i] + dalpha_center(sc, i) * s;
    }
}

// transposed index: the records of every ray on a source j0 <= j < j1 scattered into
// per-source lists of (ray, a), stored from entry ebase = src_off[j0] on
__global__ void k_src_fill(RaysDev rays, int n_rays, unsigned long long *cursor, int2 *tr, int j0, int j1,
                           long long ebase) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const long long base = rays.off[r];
    const int c = rays.cnt[r];
    for (int h = 0; h < c; ++h) {
        const int2 ja = rays.rec_ja[base + h];
        if (ja.x < j0 || ja.x >= j1) continue;
        const unsigned long long pos = atomicAdd(&cursor[ja.x], 1ull);
        tr[(long long)pos - ebase] = make_int2(r, ja.y);
    }
}

__global__ void k_copy_off(const long long *off, unsigned long long *cursor, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cursor[i] = (unsigned long long)off[i];
}


// the transposed index of sources j0 .. j1-1 into t->tr (entries from ebase on)
rgs_status build_index(rgs_transport *t, int j0, int j1, long long ebase, cudaStream_t st) {
    const int n = t->n;
    const long long n_rays = (long long)n * t->nd;
    RaysDev rd = t->rays();
    { ProfScope ps_("k_copy_off", st); k_copy_off<<<(n + 255) / 256, 256, 0, st>>>(t->src_off, t->cursor, n); }
    { ProfScope ps_("k_src_fill", st); k_src_fill<<<(unsigned)((n_rays + 255) / 256), 256, 0, st>>>(rd, (int)n_rays, t->cursor, t->tr, j0, j1, ebase); }
    RGS_LAUNCH("transposed index");
    return RGS_OK;
}

// g_h (+)= the na iterates of one group, all column tiles; first: the group that writes gh
template <int NC>
rgs_status opacity_group(rgs_transport *t, SceneDev sd, RaysDev rd, int na, const float *const *v,
                         const float *const *Bf, const __nv_bfloat16 *const *Bh, bool first, cudaStream_t st) {
    if (wide_opacity(t->C, Bh != nullptr)) return mc_opacity<NC>(t, sd, rd, na, v, Bf, Bh, first, st);
    constexpr int NA = 4;
    const long long n_rays = (long long)t->n * t->nd;
    const unsigned gg = (unsigned)((n_rays * Slice<NC>::G + 255) / 256);
    OpaSet<float, NA> sf = {};
    OpaSet<__nv_bfloat16, NA> sh = {};
    for (int a = 0; a < na; ++a) {
        sf.v[a] = sh.v[a] = v[a];
        sf.b[a] = Bf[a];
        sh.b[a] = Bh ? Bh[a] : nullptr;
    }
    for (int col0 = 0; col0 < t->C; col0 += 3) {
        const bool wr = first && col0 == 0;
        if (Bh) { // the batched modes gather the BF16 iterate copies
            ProfScope ps_("k_opacity_g", st);
            k_opacity_g<NC, 3, NA, SliceH<NC>><<<gg, 256, 0, st>>>(sd, rd, t->C, col0, na, sh, t->gh, wr);
        } else {
            ProfScope ps_("k_opacity_g", st);
            k_opacity_g<NC, 3, NA, Slice<NC>><<<gg, 256, 0, st>>>(sd, rd, t->C, col0, na, sf, t->gh, wr);
        }
    }
    RGS_LAUNCH("opacity gather");
    return RGS_OK;
}

// The adjoint walks the bounces backwards, b = n-1 .. 0 (a = n-1-b = 0 .. n-1), in segments
// [lo, hi] that end at a stored iterate: one segment holding everything when every iterate
// was kept, else one per checkpoint, whose B^(b) and Q^(b) are recomputed from B^(lo) into
// pooled scratch before the segment's v^(a) are formed and used.
template <int NC>
rgs_status run_adjoint(rgs_transport *t, const float *g, float *dE, float *dad, float *dopo,
                       const std::vector<int> &parts, const std::vector<long long> &part_base, cudaStream_t st,
                       const RgsGeoAcc *geo, bool tcp) {
    const int n = t->n, C = t->C, nb = t->nb_last, s = t->stride;
    const size_t A = t->arr();
    const size_t A16 = (size_t)n * C * bf16_stride<NC>();
    const bool bf16 = t->prec_last != RGS_FP32;
    const bool mc = wide_adjoint(C);
    SceneDev sd = t->sc->dev();
    RaysDev rd = t->rays();
    const unsigned ga = (unsigned)((A + 255) / 256);
    const unsigned gn = (unsigned)((n + 127) / 128);
    const long long n_rays = (long long)n * t->nd;
    const unsigned gr = (unsigned)((n_rays + 255) / 256);
    auto vp = [&](int a) { return t->v + A * (s ? a % (s + 1) : a); };
    // v^(0) = g (internal layout), u = v^(0), P = 0, dop = 0
    { ProfScope ps_("k_from_user", st); k_from_user<NC><<<ga, 256, 0, st>>>(n, C, t->sc->uid, g, vp(0)); }
    RGS_CUDA(cudaMemcpyAsync(t->u, vp(0), sizeof(float) * A, cudaMemcpyDeviceToDevice, st));
    RGS_CUDA(cudaMemsetAsync(t->Pg, 0, sizeof(float) * 12 * (size_t)n, st));
    RGS_CUDA(cudaMemsetAsync(t->dop, 0, sizeof(float) * (size_t)n, st));
    RGS_LAUNCH("adjoint init");
    // v^(a) = K^T v^(a-1), u += v^(a): per part of the transposed index (one part holding
    // every source unless memory asked for more), per column tile
    auto KT = [&](int a) -> rgs_status {
        rgs_status q;
        if (tcp) { // tensor cores over source tiles: y^(a-1) = o c (x) v^(a-1) in BF16 row blocks
            // mode 2: the opacity gather pairs y^(a) with B^(n-1-a) while y^(a) is at hand, per
            // (tile, receiver) group (at 16 columns per MMA it measured slower than the row
            // gathers and than the sampled products that modes -1 and 1 run after the bounces)
            const bool gh = (dopo || geo) && nb >= 1 && t->tc_mode == 2;
            if (a == 1) {
                if ((q = rgs_tc_make_y(t, vp(0), 0, st)) != RGS_OK) return q;
                if (gh && (q = rgs_tc_opacity(t, 0, t->iters + A * (nb - 1), true, st)) != RGS_OK) return q;
            }
            if ((q = rgs_tc_adjoint_bounce(t, (a - 1) & 1, a & 1, vp(a), t->u, st)) != RGS_OK) return q;
            if (gh && a <= nb - 1 && (q = rgs_tc_opacity(t, a & 1, t->iters + A * (nb - 1 - a), false, st)) != RGS_OK)
                return q;
            return RGS_OK;
        }
        for (size_t p = 0; p + 1 < parts.size(); ++p) {
            const int j0 = parts[p], j1 = parts[p + 1];
            if (j1 <= j0) continue;
            const long long eb = part_base[p];
            if (parts.size() > 2 && (q = build_index(t, j0, j1, eb, st)) != RGS_OK) return q;
            if (mc) {
                if ((q = mc_adjoint_bounce<NC>(t, sd, rd, vp(a - 1), vp(a), j0, j1, eb, st)) != RGS_OK) return q;
                continue;
            }
            for (int col0 = 0; col0 < C; col0 += 3) {
                { ProfScope ps_("k_adj_ray", st); k_adj_ray<NC><<<gr, 256, 0, st>>>(sd, rd, C, col0, vp(a - 1), t->dy); }
                { ProfScope ps_("k_adj_src", st); k_adj_src<NC><<<j1 - j0, ADJ_THREADS, 0, st>>>(rd, C, col0, t->src_off, t->tr, t->dy, vp(a), t->u, j0, eb); }
            }
            RGS_LAUNCH("adjoint bounce");
        }
        return RGS_OK;
    };
    // segment scratch (checkpointing): B^(lo+1 .. lo+s) FP32 (+BF16) and Q^(lo .. lo+s-1)
    struct SegScratch {
        cudaStream_t st;
        std::vector<float *> B, Q;
        std::vector<__nv_bfloat16 *> B16;
        double *nrm = nullptr;
        ~SegScratch() {
            for (auto &p : B) pool_release(p, st);
            for (auto &p : Q) pool_release(p, st);
            for (auto &p : B16) pool_release(p, st);
            pool_release(nrm, st);
        }
    } seg{st, {}, {}, {}, nullptr};
    rgs_status r;
    if (s) {
        seg.B.assign(s, nullptr);
        seg.Q.assign(s, nullptr);
        seg.B16.assign(s, nullptr);
        for (int k = 0; k < s; ++k) {
            if ((r = pool_alloc(&seg.B[k], A, st)) != RGS_OK) return r;
            if ((r = pool_alloc(&seg.Q[k], A, st)) != RGS_OK) return r;
            if (bf16) {
                if ((r = pool_alloc(&seg.B16[k], A16, st)) != RGS_OK) return r;
                RGS_CUDA(cudaMemsetAsync(seg.B16[k], 0, sizeof(__nv_bfloat16) * A16, st)); // row padding
            }
        }
        if ((r = pool_alloc(&seg.nrm, RGS_MAX_BOUNCES + 1, st)) != RGS_OK) return r;
    }
    bool first_g = true;
    // the opacity gather's form, fixed for the whole adjoint (the sampled products sum in
    // the source tiles' hit order and hand the record slots their sums after the last pairing)
    const bool sddmm = tcp && (t->tc_mode == -1 || t->tc_mode == 1) && rgs_tc_opa_pass_cols(t) > 0;
    for (int hi = nb - 1; hi >= 0;) {
        const int lo = s ? (hi / s) * s : 0;
        // iterates B^(b) (FP32, BF16) and Q^(b) of this segment, indexed by b - lo
        std::vector<const float *> Bf(hi - lo + 1), Qb(hi - lo + 1);
        std::vector<const __nv_bfloat16 *> Bh(hi - lo + 1);
        if (!s) {
            for (int b = lo; b <= hi; ++b) {
                Bf[b - lo] = t->iters + A * b;
                Bh[b - lo] = bf16 ? t->iters16 + A16 * b : nullptr;
                Qb[b - lo] = t->Q + A * b;
            }
        } else {
            if ((r = rgs_recompute(t, lo, hi + 1, seg.B.data(), seg.B16.data(), seg.Q.data(), seg.nrm, st)) != RGS_OK)
                return r;
            for (int b = lo; b <= hi; ++b) {
                Bf[b - lo] = b == lo ? t->iters + A * t->slot(lo) : seg.B[b - lo - 1];
                Bh[b - lo] = !bf16 ? nullptr : (b == lo ? t->iters16 + A16 * t->slot(lo) : seg.B16[b - lo - 1]);
                Qb[b - lo] = seg.Q[b - lo];
            }
        }
        for (int b = hi; b >= lo; --b) {
            const int a = nb - 1 - b;
            if (a > 0 && (r = KT(a)) != RGS_OK) return r;
            { ProfScope ps_("k_pair_accum", st); k_pair_accum<NC><<<gn, 128, 0, st>>>(n, C, vp(a), Qb[b - lo], t->Pg); }
            RGS_LAUNCH("pair accum");
        }
        if ((dopo || geo) && sddmm) { // g_h as sampled products on the tensor cores
            for (int b = hi; b >= lo; --b) {
                if ((r = rgs_tc_opacity_sddmm(t, vp(nb - 1 - b), Bf[b - lo], first_g, b == 0, st)) != RGS_OK) return r;
                first_g = false;
            }
        } else if ((dopo || geo) && !(tcp && t->tc_mode == 2)) { // g_h over this segment's iterates, four per launch
            for (int b0 = hi; b0 >= lo; b0 -= 4) {
                const int na = min(4, b0 - lo + 1);
                const float *vv[4], *bb[4];
                const __nv_bfloat16 *hh[4];
                for (int q = 0; q < na; ++q) {
                    const int b = b0 - q;
                    vv[q] = vp(nb - 1 - b);
                    bb[q] = Bf[b - lo];
                    hh[q] = Bh[b - lo];
                }
                if ((r = opacity_group<NC>(t, sd, rd, na, vv, bb, bf16 ? hh : nullptr, first_g, st)) != RGS_OK) return r;
                first_g = false;
            }
        }
        hi = lo - 1;
    }
    if (nb >= 1 && (r = KT(nb)) != RGS_OK) return r; // v^(n) only adds to u
    if (t->nl > 0) {
        const int nth = n * t->nl;
        { ProfScope ps_("k_shadow_bwd", st); k_shadow_bwd<NC><<<(nth + 127) / 128, 128, 0, st>>>(sd, t->nl, t->ldir, t->lpos, t->lint, C, t->u, t->Pg, t->dop, geo ? geo->dp : nullptr, geo ? geo->ds : nullptr, geo ? geo->gF : nullptr); }
        RGS_LAUNCH("shadow backward");
    }
    if (nb >= 1 && dopo) {
        { ProfScope ps_("k_opacity_rec", st); k_opacity_rec<<<gr, 256, 0, st>>>(sd, rd, t->gh, t->dop); }
        RGS_LAUNCH("hemisphere opacity backward");
    }
    if (nb >= 1 && geo) { // every iterate is kept (the caller checked the stride)
        const long long n_rays = (long long)n * t->nd;
        { ProfScope ps_("k_hemi_geo", st); k_hemi_geo<<<(unsigned)((n_rays + 127) / 128), 128, 0, st>>>(sd, rd, nb, t->gh, geo->dp, geo->ds, geo->gF); }
        RGS_LAUNCH("hemisphere geometry backward");
        { ProfScope ps_("k_hemi_geo_dir", st); k_hemi_geo_dir<NC><<<n, GEO_DIR_THREADS, 0, st>>>(sd, rd, C, nb, A, t->v, t->iters, geo->gF); }
        RGS_LAUNCH("hemisphere geometry backward (directional)");
    }
    { ProfScope ps_("k_finalize", st); k_finalize<NC><<<gn, 128, 0, st>>>(sd, C, t->u, t->Pg, t->sc->kk, t->dop, dE, dad, dopo); }
    RGS_LAUNCH("finalize");
    return tcp ? rgs_tc_check(t, st) : RGS_OK;
}

} // namespace

// ------------------------------------------------------------------ pieces shared with the
// center-to-center adjoint (rgs_pairs.cu)
void rgs_copy_offsets(const long long *off, unsigned long long *cursor, int n, cudaStream_t st) {
    k_copy_off<<<(n + 255) / 256, 256, 0, st>>>(off, cursor, n);
}

namespace {
template <int NC> rgs_status prologue_nc(rgs_transport *t, const float *g, cudaStream_t st) {
    const int n = t->n, C = t->C, nb = t->nb_last;
    const size_t A = t->arr();
    { ProfScope ps_("k_from_user", st); k_from_user<NC><<<(unsigned)((A + 255) / 256), 256, 0, st>>>(n, C, t->sc->uid, g, t->v); }
    RGS_CUDA(cudaMemcpyAsync(t->u, t->v, sizeof(float) * A, cudaMemcpyDeviceToDevice, st));
    RGS_CUDA(cudaMemsetAsync(t->Pg, 0, sizeof(float) * 12 * (size_t)n, st));
    RGS_CUDA(cudaMemsetAsync(t->dop, 0, sizeof(float) * (size_t)n, st));
    if (nb >= 1) { ProfScope ps_("k_pair_accum", st); k_pair_accum<NC><<<(n + 127) / 128, 128, 0, st>>>(n, C, t->v, t->Q + A * (nb - 1), t->Pg); }
    RGS_LAUNCH("adjoint init");
    return RGS_OK;
}
template <int NC> rgs_status accum_nc(rgs_transport *t, const float *X, const float *Y, cudaStream_t st) {
    { ProfScope ps_("k_pair_accum", st); k_pair_accum<NC><<<(t->n + 127) / 128, 128, 0, st>>>(t->n, t->C, X, Y, t->Pg); }
    RGS_LAUNCH("pair accum");
    return RGS_OK;
}
template <int NC> rgs_status shadow_nc(rgs_transport *t, cudaStream_t st, float *dp, float *ds, float *gF) {
    if (t->nl <= 0) return RGS_OK;
    const int nth = t->n * t->nl;
    { ProfScope ps_("k_shadow_bwd", st); k_shadow_bwd<NC><<<(nth + 127) / 128, 128, 0, st>>>(t->sc->dev(), t->nl, t->ldir, t->lpos, t->lint, t->C, t->u, t->Pg, t->dop, dp, ds, gF); }
    RGS_LAUNCH("shadow backward");
    return RGS_OK;
}
template <int NC> rgs_status finalize_nc(rgs_transport *t, float *dE, float *dad, float *dop, cudaStream_t st) {
    { ProfScope ps_("k_finalize", st); k_finalize<NC><<<(t->n + 127) / 128, 128, 0, st>>>(t->sc->dev(), t->C, t->u, t->Pg, t->sc->kk, t->dop, dE, dad, dop); }
    RGS_LAUNCH("finalize");
    return RGS_OK;
}
} // namespace

#define RGS_NC_SWITCH(nc, call1, call4, call9, call16)                                                                 \
    switch (nc) {                                                                                                      \
    case 1: return call1;                                                                                              \
    case 4: return call4;                                                                                              \
    case 9: return call9;                                                                                              \
    default: return call16;                                                                                            \
    }
rgs_status rgs_adjoint_prologue(rgs_transport *t, int nc, const float *g, cudaStream_t st) {
    RGS_NC_SWITCH(nc, prologue_nc<1>(t, g, st), prologue_nc<4>(t, g, st), prologue_nc<9>(t, g, st), prologue_nc<16>(t, g, st))
}
rgs_status rgs_pair_accum(rgs_transport *t, int nc, const float *X, const float *Y, cudaStream_t st) {
    RGS_NC_SWITCH(nc, accum_nc<1>(t, X, Y, st), accum_nc<4>(t, X, Y, st), accum_nc<9>(t, X, Y, st), accum_nc<16>(t, X, Y, st))
}
rgs_status rgs_shadow_backward(rgs_transport *t, int nc, cudaStream_t st, float *dp, float *ds, float *gF) {
    RGS_NC_SWITCH(nc, shadow_nc<1>(t, st, dp, ds, gF), shadow_nc<4>(t, st, dp, ds, gF), shadow_nc<9>(t, st, dp, ds, gF),
                  shadow_nc<16>(t, st, dp, ds, gF))
}
rgs_status rgs_adjoint_finalize(rgs_transport *t, int nc, float *dE, float *dad, float *dop, cudaStream_t st) {
    RGS_NC_SWITCH(nc, finalize_nc<1>(t, dE, dad, dop, st), finalize_nc<4>(t, dE, dad, dop, st),
                  finalize_nc<9>(t, dE, dad, dop, st), finalize_nc<16>(t, dE, dad, dop, st))
}
#undef RGS_NC_SWITCH

rgs_status rgs_adjoint_impl(rgs_transport *t, const float *g, float *dE, float *dad, float *dop, cudaStream_t st,
                            float *dp, float *ds, float *dtu, float *dtv) {
    if (t->kind == RGS_KIND_PAIRS) return rgs_adjoint_pairs_impl(t, g, dE, dad, dop, nullptr, dp, ds, dtu, dtv, st);
    const bool want_geo = dp || ds || dtu || dtv;
    if (want_geo && t->stride != 0) {
        rgs_set_error("geometry gradients of the hemisphere transport need every iterate: solve with checkpointing off");
        return RGS_ERR_STATE;
    }
    rgs_status r;
    const int nb = t->nb_last, n = t->n;
    const size_t A = t->arr();
    const long long n_rays = (long long)n * t->nd;
    if (n > t->pg_cap) {
        if ((r = dev_alloc(&t->Pg, (size_t)n * 12, &t->device_bytes)) != RGS_OK) return r;
        if ((r = dev_alloc(&t->dop, (size_t)n, &t->device_bytes)) != RGS_OK) return r;
        t->pg_cap = n;
    }
    // Workspaces that live only inside this call come from the stream-ordered pool and are
    // returned to it on every exit path: v^(0..n), u, the transposed index, the per-ray
    // adjoint values and the per-record opacity sums.
    struct Scratch {
        rgs_transport *t;
        cudaStream_t st;
        ~Scratch() {
            pool_release(t->v, st);
            pool_release(t->u, st);
            pool_release(t->tr, st);
            pool_release(t->dy, st);
            pool_release(t->dy_mc, st);
            pool_release(t->gh, st);
            pool_release(geo.dp, st);
            pool_release(geo.ds, st);
            pool_release(geo.gF, st);
        }
        RgsGeoAcc geo;
    } scratch{t, st, {}};
    const bool mc = wide_adjoint(t->C);
    const bool want_gh = (dop || want_geo) && nb >= 1;
    // the last solve ran on the tensor cores: so do the transposed bounces (source tiles
    // instead of the transposed hit index and the per-ray adjoint values)
    const bool tcp = t->tc_used && t->kind == RGS_KIND_HEMISPHERE && t->stride == 0 && nb >= 1;
    if (tcp && ((r = rgs_tc_prepare_adjoint(t, st)) != RGS_OK || (r = rgs_tc_reset_flags(t, st)) != RGS_OK)) return r;
    if (want_geo) {
        RgsGeoAcc &geo = scratch.geo;
        if ((r = pool_alloc(&geo.dp, (size_t)n * GEO_DP, st)) != RGS_OK) return r;
        if ((r = pool_alloc(&geo.ds, (size_t)n * 2, st)) != RGS_OK) return r;
        if ((r = pool_alloc(&geo.gF, (size_t)n * GEO_GF, st)) != RGS_OK) return r;
        RGS_CUDA(cudaMemsetAsync(geo.dp, 0, sizeof(float) * n * GEO_DP, st));
        RGS_CUDA(cudaMemsetAsync(geo.ds, 0, sizeof(float) * n * 2, st));
        RGS_CUDA(cudaMemsetAsync(geo.gF, 0, sizeof(float) * n * GEO_GF, st));
    }
    const RgsGeoAcc *geop = want_geo ? &scratch.geo : nullptr;
    const int n_v = t->stride ? t->stride + 1 : nb + 1;
    if ((r = pool_alloc(&t->v, A * n_v, st)) != RGS_OK) return r;
    if ((r = pool_alloc(&t->u, A, st)) != RGS_OK) return r;
    if (tcp) {
    } else if (mc) {
        if ((r = pool_alloc(&t->dy_mc, (size_t)n_rays * 32, st)) != RGS_OK) return r;
    } else {
        if ((r = pool_alloc(&t->dy, (size_t)n_rays, st)) != RGS_OK) return r;
    }
    if (want_gh && (r = pool_alloc(&t->gh, (size_t)t->n_slots, st)) != RGS_OK) return r;
    // The transposed index in one part when it fits next to the segment scratch of a
    // checkpointed adjoint, else in P parts of about equal entry counts, each rebuilt from
    // the records for every transposed bounce.
    const double A16 = t->prec_last != RGS_FP32 ? 2.0 * n * t->C * (t->nc >= 9 ? 16 : t->nc) : 0.0;
    const double seg = t->stride ? t->stride * (8.0 * A + A16) + 8.0 * (RGS_MAX_BOUNCES + 1) : 0.0;
    const double tr_all = 8.0 * (double)t->n_hits;
    double avail = 0.92 * (double)pool_available_bytes() - seg;
    if (t->mem_budget > 0) {
        const double scratch = 4.0 * A * (n_v + 1) + (mc ? 128.0 : 16.0) * n_rays + (want_gh ? 4.0 * t->n_slots : 0.0);
        avail = std::min(avail, (double)t->mem_budget - (double)t->device_bytes - scratch - seg);
    }
    int P = 1;
    while (!tcp && P < 64 && tr_all / P > avail) P *= 2;
    std::vector<int> parts{0};
    std::vector<long long> base{0};
    if (P > 1) {
        std::vector<long long> off((size_t)n + 1);
        RGS_CUDA(cudaMemcpyAsync(off.data(), t->src_off, sizeof(long long) * (n + 1), cudaMemcpyDeviceToHost, st));
        RGS_CUDA(cudaStreamSynchronize(st));
        int j = 0;
        for (int p = 1; p < P; ++p) {
            const long long target = (long long)((double)t->n_hits * p / P);
            while (j < n && off[j] < target) ++j;
            parts.push_back(j);
            base.push_back(off[j]);
        }
    }
    parts.push_back(n);
    long long biggest = 0;
    for (size_t p = 0; p + 1 < parts.size(); ++p) {
        const long long e1 = p + 2 < parts.size() ? base[p + 1] : t->n_hits;
        biggest = std::max(biggest, e1 - base[p]);
    }
    if (!tcp) {
        if ((r = pool_alloc(&t->tr, (size_t)std::max(biggest, 1ll), st)) != RGS_OK) return r;
        if (parts.size() == 2 && (r = build_index(t, 0, n, 0, st)) != RGS_OK) return r;
    }
    switch (t->nc) {
    case 1: r = run_adjoint<1>(t, g, dE, dad, dop, parts, base, st, geop, false); break;
    case 4: r = run_adjoint<4>(t, g, dE, dad, dop, parts, base, st, geop, false); break;
    case 9: r = run_adjoint<9>(t, g, dE, dad, dop, parts, base, st, geop, false); break;
    default: r = run_adjoint<16>(t, g, dE, dad, dop, parts, base, st, geop, tcp);
    }
    if (r != RGS_OK || !want_geo) return r;
    return rgs_geometry_out(t, scratch.geo, dp, ds, dtu, dtv, st);
}
