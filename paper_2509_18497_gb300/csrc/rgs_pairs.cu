// Center-to-center transport (Sec. 8, the approximated forward rendering equation):
//
//   B_i = E_i + sum_j f_i(w) (Y(w)^T B_j) V_ji,
//   V_ji = lambda_j (int alpha_j dx) prod_k (1 - alpha_k) |n_i.w| |n_j.w| / |p_i - p_j|^2,
//
// one segment per pair of surfel centres instead of hemisphere rays; f_i absorbs
// alpha_i(p_i) = o_i, so with d = (p_j - p_i)/r the pair adds o_i c_i (x) Y(R_i d) V_ji
// Y(-d)^T B_j to the receiver, exactly the hemisphere gather with one "hit" of weight V_ji
// per direction and no pi/nd.  Sources count when they lie more than eps_plane in front
// of the receiver's plane; the segment's occluders follow the hemisphere-ray hit rules and
// must lie more than eps_plane from the source's end too; int alpha_j is closed-form.
//
// Storage: the pairs of receiver i are contiguous (pair_off[i] .. pair_off[i+1]), each one
// record (j, bits of V_ji), sources in increasing internal (Morton) index, so that a warp's 32
// segments leave one centre towards neighbouring sources.  A count pass sizes
// every (receiver, 256-source chunk) block exactly; the fill pass traces each front pair's
// segment and writes its record at the chunk's offset plus its rank in the block.
#include <algorithm>
#include <vector>

#include "rgs_bounce_body.cuh"

namespace {

constexpr int PCH = 256;      // sources per block of the count / fill passes
constexpr int PAIR_THREADS = 128;

// Ein(x) = int_0^x (1 - e^{-y}) / y dy in FP32: for x <= 2 its power series
// sum (-1)^{k+1} x^k / (k k!) (terms below 2^-24 of the sum after k = 14); beyond,
// ln x + gamma + E1(x) with E1 from the continued fraction of Abramowitz & Stegun 5.1.22,
// E1(x) = e^{-x} / (x + 1/(1 + 1/(x + 2/(1 + 2/(x + ...))))), evaluated from depth 12 upwards
// (the truncation is below 1.2e-7 relative from x = 2 on).  Within 2.3e-7 of the exact value.
__device__ float ein_f(float x) {
    if (!(x > 0.f)) return 0.f;
    if (x <= 2.f) {
        float term = x, sum = x;
#pragma unroll
        for (int k = 2; k <= 16; ++k) {
            term *= -x / (float)k;
            sum += term / (float)k;
        }
        return sum;
    }
    float tail = 0.f;
#pragma unroll
    for (int m = 12; m >= 1; --m) tail = (float)m / (1.f + (float)m / (x + tail));
    return logf(x) + 0.5772157f + expf(-x) / (x + tail);
}

// int alpha_j dx over the tangent plane and its derivative in o_j, per surfel: the
// Gaussian truncated at 3 sigma 2 pi s^u s^v o (1 - e^{-9/2}), the disc pi s^u s^v o, and
// App. E's GFSGS closed form (2 pi / 3.4) s^u s^v Ein(0.03279 o^3.4), whose derivative
// is 2 pi s^u s^v alpha_j(p_j) / o.
__global__ void k_alpha_area(SceneDev sc, float *aarea, float *daarea) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= sc.n) return;
    const float su = 1.f / sc.FU[j].w, sv = 1.f / sc.FV[j].w, o = sc.P[j].w;
    const float two_pi = 6.2831853f;
    float A, dA;
    if (sc.alpha_model == RGS_ALPHA_GFSGS) {
        const float x = o > 0.f ? 0.03279f * powf(o, 3.4f) : 0.f;
        A = two_pi / 3.4f * su * sv * ein_f(x);
        dA = o > 0.f ? two_pi * su * sv * (-expm1f(-x)) / o : 0.f;
    } else {
        const float unit = (sc.alpha_model == RGS_ALPHA_DISC) ? 0.5f * two_pi * su * sv
                                                              : two_pi * su * sv * (1.f - expf(-4.5f));
        A = o * unit;
        dA = unit;
    }
    aarea[j] = A;
    daarea[j] = dA;
}

// source j in front of receiver i: n_i.(p_j - p_i) > eps (explicitly rounded, so the count
// and the fill pass agree bit for bit)
__device__ __forceinline__ bool pair_front(const SceneDev &sc, float3 pi, float3 ni, int j, float eps, float3 &dv) {
    const float4 Pj = __ldg(&sc.P[j]);
    dv = make_float3(__fsub_rn(Pj.x, pi.x), __fsub_rn(Pj.y, pi.y), __fsub_rn(Pj.z, pi.z));
    const float h = __fmaf_rn(ni.z, dv.z, __fmaf_rn(ni.y, dv.y, __fmul_rn(ni.x, dv.x)));
    return h > eps;
}

__device__ __forceinline__ float3 unit_dir(float3 dv, float &r) {
    r = sqrtf(dv.x * dv.x + dv.y * dv.y + dv.z * dv.z);
    const float inv = 1.f / r;
    return make_float3(dv.x * inv, dv.y * inv, dv.z * inv);
}

// occluder k of the segment i -> j (t in (0, r)): a regular hit that is not the source and
// whose plane is more than eps from the source's centre
__device__ __forceinline__ bool pair_occluder(const SceneDev &sc, int k, int i, int j, float3 o, float3 d, float r,
                                              float3 pj, float eps, float &g, float &t) {
    if (k == j) return false;
    if (!hit_surfel(sc, k, i, o, d, r, eps, t, g)) return false;
    const float4 Nk = __ldg(&sc.N4[k]);
    const float4 Pk = __ldg(&sc.P[k]);
    const float e = Nk.x * (pj.x - Pk.x) + Nk.y * (pj.y - Pk.y) + Nk.z * (pj.z - Pk.z);
    return fabsf(e) > eps;
}

__global__ void __launch_bounds__(PCH) k_pair_count(SceneDev sc, int n, int chunks, int *chunk_cnt, int *src_cnt) {
    const int blk = blockIdx.x;
    const int i = blk / chunks, c = blk - i * chunks;
    const int j = c * PCH + threadIdx.x;
    const float eps = *sc.eps_plane;
    const float3 pi = f3(sc.P[i]), ni = f3(sc.N4[i]);
    float3 dv;
    const bool front = j < n && j != i && pair_front(sc, pi, ni, j, eps, dv);
    const int cnt = __syncthreads_count(front);
    if (threadIdx.x == 0) chunk_cnt[blk] = cnt;
    if (front) atomicAdd(&src_cnt[j], 1);
}

__global__ void __launch_bounds__(PCH) k_pair_fill(SceneDev sc, int n, int chunks, const long long *__restrict__ chunk_off,
                                                   const float *__restrict__ lam, const float *__restrict__ aarea,
                                                   int2 *rec, int *flags) {
    __shared__ int warp_base[PCH / 32];
    const int blk = blockIdx.x;
    const int i = blk / chunks, c = blk - i * chunks;
    const int j = c * PCH + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float eps = *sc.eps_plane;
    const float3 pi = f3(sc.P[i]), ni = f3(sc.N4[i]);
    float3 dv;
    const bool front = j < n && j != i && pair_front(sc, pi, ni, j, eps, dv);
    // rank of this pair in the block (sources in increasing order)
    const unsigned bal = __ballot_sync(0xffffffffu, front);
    if (lane == 0) warp_base[warp] = __popc(bal);
    __syncthreads();
    int base = 0;
    for (int w = 0; w < warp; ++w) base += warp_base[w];
    if (!front) return;
    const int rank = base + __popc(bal & ((1u << lane) - 1u));
    float r;
    const float3 d = unit_dir(dv, r);
    const float3 pj = f3(sc.P[j]);
    float T = 1.f;
    auto visit = [&](int k) {
        float g, t;
        if (pair_occluder(sc, k, i, j, pi, d, r, pj, eps, g, t)) T *= 1.f - alpha_of(sc, __ldg(&sc.P[k].w), g);
    };
    if (!bvh_traverse(sc, pi, d, r, visit)) atomicAdd(&flags[FLAG_STACK], 1);
    const float3 nj = f3(sc.N4[j]);
    const float geo = fabsf(dot3(ni, d)) * fabsf(dot3(nj, d)) / (r * r);
    const float V = __ldg(&lam[j]) * __ldg(&aarea[j]) * T * geo;
    rec[chunk_off[blk] + rank] = make_int2(j, __float_as_int(V));
}

__global__ void k_pair_off(const long long *chunk_off, int chunks, int n, long long *pair_off) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) pair_off[i] = chunk_off[(size_t)i * chunks];
}

// lambda in internal order (1 where the caller gives none)
__global__ void k_lam_in(int n, const int *__restrict__ uid, const float *__restrict__ lam_user, float *lam) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) lam[i] = lam_user ? lam_user[uid[i]] : 1.f;
}

// ------------------------------------------------------------------ bounce
// One receiver and one 3-column tile: G lanes per pair, each a slice of the coefficients.
template <int NC, int CT, class SL>
__global__ void RGS_BOUNCE_LB k_bounce_pairs(SceneDev sc, const long long *__restrict__ pair_off,
                                             const int2 *__restrict__ rec, int C, const typename SL::T *__restrict__ Bg,
                                             const float *__restrict__ Bprev, const float *__restrict__ S,
                                             float *__restrict__ Qout, float *__restrict__ Bout,
                                             __nv_bfloat16 *__restrict__ Bout16, double *norm2) {
    __shared__ float red[(BOUNCE_THREADS / 32) * SL::G * SL::KPL * CT];
    constexpr int G = SL::G, KPL = SL::KPL, GROUPS = BOUNCE_THREADS / G, RS = SL::STRIDE;
    const int i = blockIdx.x, col0 = blockIdx.y * CT;
    const int grp = threadIdx.x / G, g = threadIdx.x % G;
    const float3 pi = f3(sc.P[i]), ni = f3(sc.N4[i]);
    float acc[KPL][CT];
#pragma unroll
    for (int m = 0; m < KPL; ++m)
#pragma unroll
        for (int c = 0; c < CT; ++c) acc[m][c] = 0.f;
    const long long e0 = pair_off[i], e1 = pair_off[i + 1];
    // every lane makes the same number of trips (the group sums shuffle across the warp);
    // a group past the receiver's last pair contributes zero
    for (long long eb = e0; eb < e1; eb += GROUPS) {
        const long long e = eb + grp;
        const bool live = e < e1;
        const int2 jv = __ldg(&rec[live ? e : e1 - 1]);
        const float V = live ? __int_as_float(jv.y) : 0.f;
        const float4 Pj = __ldg(&sc.P[jv.x]);
        float r;
        const float3 d = unit_dir(make_float3(Pj.x - pi.x, Pj.y - pi.y, Pj.z - pi.z), r);
        float yo[KPL], yi[KPL];
        {
            float Y[NC];
            sh_eval<NC>(neg3(d), Y);
            SL::pick(Y, g, yo);
            sh_eval<NC>(reflect_n(ni, d), Y);
            SL::pick(Y, g, yi);
        }
        const typename SL::T *Bj = Bg + ((size_t)jv.x * C + col0) * RS;
#pragma unroll
        for (int c = 0; c < CT; ++c) {
            float v[KPL];
            SL::load(Bj + c * RS, g, v);
            float s = 0.f;
#pragma unroll
            for (int m = 0; m < KPL; ++m) s += yo[m] * v[m];
            const float xc = V * SL::group_sum(s);
#pragma unroll
            for (int m = 0; m < KPL; ++m) acc[m][c] += yi[m] * xc;
        }
    }
    bounce_epilogue<NC, CT, SL>(sc, C, acc, 1.f, Bprev, S, Qout, Bout, Bout16, norm2, i, col0, red);
}

// ------------------------------------------------------------------ adjoint
// transposed index: for every pair (i -> j) the entry (i, bits of V) in source j's list
__global__ void k_pair_src_fill(int n, const long long *__restrict__ pair_off, const int2 *__restrict__ rec,
                                unsigned long long *cursor, int2 *tr) {
    const int i = blockIdx.x;
    for (long long e = pair_off[i] + threadIdx.x; e < pair_off[i + 1]; e += blockDim.x) {
        const int2 jv = rec[e];
        const unsigned long long pos = atomicAdd(&cursor[jv.x], 1ull);
        tr[pos] = make_int2(i, jv.y);
    }
}

// (K^T v)_j[c][k] = sum_{pairs i -> j} V_ji Y_k(-d) y_i[c],
// y_i[c] = o_i sum_k' c_{i,l(k'),ch} Y_k'(R_i d) v_i[c][k']; one CTA per source, all tiles
template <int NC>
__global__ void __launch_bounds__(PAIR_THREADS) k_adj_src_pairs(SceneDev sc, int C, const long long *__restrict__ src_off,
                                                               const int2 *__restrict__ tr, const float *__restrict__ vin,
                                                               float *__restrict__ vout, float *__restrict__ u) {
    constexpr int CT = 3;
    __shared__ float red[PAIR_THREADS / 32][NC * CT];
    const int j = blockIdx.x;
    const float4 Pj = __ldg(&sc.P[j]);
    const long long e0 = src_off[j], e1 = src_off[j + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int col0 = 0; col0 < C; col0 += CT) {
        float acc[NC][CT];
#pragma unroll
        for (int k = 0; k < NC; ++k)
#pragma unroll
            for (int c = 0; c < CT; ++c) acc[k][c] = 0.f;
        for (long long e = e0 + threadIdx.x; e < e1; e += PAIR_THREADS) {
            const int2 iv = __ldg(&tr[e]);
            const int i = iv.x;
            const float V = __int_as_float(iv.y);
            const float4 Pi = __ldg(&sc.P[i]);
            const float ai = alpha_center(sc, i);
            float r;
            const float3 d = unit_dir(make_float3(Pj.x - Pi.x, Pj.y - Pi.y, Pj.z - Pi.z), r);
            float Yi[NC], Yo[NC];
            sh_eval<NC>(reflect_n(f3(sc.N4[i]), d), Yi);
            sh_eval<NC>(neg3(d), Yo);
            const float *vi = vin + ((size_t)i * C + col0) * NC;
#pragma unroll
            for (int c = 0; c < CT; ++c) {
                const int ch = (col0 + c) % 3;
                float s = 0.f;
#pragma unroll
                for (int k = 0; k < NC; ++k) s += __ldg(&sc.cl[(size_t)i * 12 + band_of(k) * 3 + ch]) * Yi[k] * __ldg(&vi[c * NC + k]);
                const float y = V * ai * s;
#pragma unroll
                for (int k = 0; k < NC; ++k) acc[k][c] += Yo[k] * y;
            }
        }
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
        for (int q = threadIdx.x; q < NC * CT; q += PAIR_THREADS) {
            float v = 0.f;
            for (int w = 0; w < PAIR_THREADS / 32; ++w) v += red[w][q];
            const int k = q / CT, c = q - k * CT;
            const size_t idx = ((size_t)j * C + col0 + c) * NC + k;
            vout[idx] = v;
            u[idx] += v;
        }
        __syncthreads();
    }
}

// g_e = dL/dV_ji of every pair e = (i -> j), summed over the bounces:
//   g = o_i sum_{a<n} sum_c (c_i (x) Y(R_i d) . v_i^(a)[c]) (Y(-d) . B_j^(n-1-a)[c]).
// GEO: also the directional effects of Eq. dl-dgeo-1, the derivative of the pair's term in
// its direction d through Y(R_i d) and Y(-d):
//   gq_e = V_ji o_i (R_i sum_k wi_k grad Y_k(R_i d) - sum_k wo_k grad Y_k(-d)),
//   wi_k = sum_{a,c} (Y(-d) . B_j[c]) c_{i,l(k),ch} v_i[c][k],  wo_k = sum_{a,c} y_c B_j[c][k],
// and the receiver normal's share through R_i d, added to gF[i] (dL/dn_i).
template <int NC, bool GEO>
__global__ void __launch_bounds__(PAIR_THREADS) k_pair_g(SceneDev sc, int C, int nb, const long long *__restrict__ pair_off,
                                                        const int2 *__restrict__ rec, size_t A,
                                                        const float *__restrict__ V, const float *__restrict__ Bit,
                                                        float *gpair, float4 *gq, float *gF) {
    const int i = blockIdx.x;
    const float4 Pi = __ldg(&sc.P[i]);
    const float3 pi = f3(Pi), ni = f3(sc.N4[i]);
    [[maybe_unused]] float3 gn = make_float3(0.f, 0.f, 0.f);
    for (long long e = pair_off[i] + threadIdx.x; e < pair_off[i + 1]; e += PAIR_THREADS) {
        const int2 jv = __ldg(&rec[e]);
        const int j = jv.x;
        const float4 Pj = __ldg(&sc.P[j]);
        float r;
        const float3 d = unit_dir(make_float3(Pj.x - pi.x, Pj.y - pi.y, Pj.z - pi.z), r);
        float Yi[NC], Yo[NC];
        const float3 rd = reflect_n(ni, d);
        sh_eval<NC>(rd, Yi);
        sh_eval<NC>(neg3(d), Yo);
        float wi[GEO ? NC : 1], wo[GEO ? NC : 1];
        if constexpr (GEO) {
#pragma unroll
            for (int k = 0; k < NC; ++k) wi[k] = wo[k] = 0.f;
        }
        float g = 0.f;
        for (int a = 0; a < nb; ++a) {
            const float *va = V + A * a + (size_t)i * C * NC;
            const float *Bb = Bit + A * (nb - 1 - a) + (size_t)j * C * NC;
            for (int c = 0; c < C; ++c) {
                const int ch = c % 3;
                float cv[NC], bv[NC];
                float y = 0.f, s = 0.f;
#pragma unroll
                for (int k = 0; k < NC; ++k) {
                    cv[k] = __ldg(&sc.cl[(size_t)i * 12 + band_of(k) * 3 + ch]) * __ldg(&va[c * NC + k]);
                    bv[k] = __ldg(&Bb[c * NC + k]);
                    y += cv[k] * Yi[k];
                    s += Yo[k] * bv[k];
                }
                g += y * s;
                if constexpr (GEO) {
#pragma unroll
                    for (int k = 0; k < NC; ++k) {
                        wi[k] += s * cv[k];
                        wo[k] += y * bv[k];
                    }
                }
            }
        }
        const float ai = alpha_center(sc, i);
        gpair[e] = g * ai;
        if constexpr (GEO) {
            const float3 t1 = sh_grad_dot<NC>(rd, wi);
            const float3 t3 = reflect_n(ni, t1);
            const float3 t2 = sh_grad_dot<NC>(neg3(d), wo);
            const float f = __int_as_float(jv.y) * ai;
            gq[e] = make_float4(f * (t3.x - t2.x), f * (t3.y - t2.y), f * (t3.z - t2.z), 0.f);
            gn = gn + reflect_grad_n(ni, d, f * t1);
        }
    }
    if constexpr (GEO) { // every thread of the block has receiver i: one atomic per warp
        float red[3] = {gn.x, gn.y, gn.z};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) red[q] += __shfl_xor_sync(0xffffffffu, red[q], off);
            if ((threadIdx.x & 31) == 0 && red[q] != 0.f) atomicAdd(&gF[GEO_GF * (size_t)i + GEO_N + q], red[q]);
        }
    }
}

// Source-side gradients of every pair, laid out as the fill pass (one block per receiver
// and 256-source chunk, a thread per source, so a warp's segments leave one centre towards
// neighbouring sources):
//   dL/dlambda_j += g A_j T geo,  dL/do_j += g lambda_j (A_j/o_j) T geo,
//   dL/do_k += -g lambda_j A_j geo prod_{m != k}(1 - alpha_m) G_k for the segment's occluders
// (the segment is traced again: once for T and the zero factors, once for the occluders).
// With dp (and ds) also the geometry gradients of Eqs. dl-dgeo-0/1: the decay term
// V = lambda_j A_j T geo through geo = (n_i.d)|n_j.d|/r^2, through A_j (proportional to
// s^u_j s^v_j) and through every occluder's crossing point and scales, plus the directional
// part gq from k_pair_g; d = (p_j - p_i)/r moves with (I - d d^T)/r (dp_j - dp_i).
template <bool GEO>
__global__ void __launch_bounds__(PCH) k_pair_grad(SceneDev sc, int n, int chunks, const long long *__restrict__ chunk_off,
                                                   const float *__restrict__ lam, const float *__restrict__ aarea,
                                                   const float *__restrict__ daarea, const float *__restrict__ gpair,
                                                   const float4 *__restrict__ gq, float *dop, float *dlam, float *dp,
                                                   float *ds, float *gF, int *flags) {
    __shared__ int warp_base[PCH / 32];
    const int blk = blockIdx.x;
    const int i = blk / chunks, c = blk - i * chunks;
    const int j = c * PCH + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float eps = *sc.eps_plane;
    const float3 pi = f3(sc.P[i]), ni = f3(sc.N4[i]);
    float3 dv;
    const bool front = j < n && j != i && pair_front(sc, pi, ni, j, eps, dv);
    const unsigned bal = __ballot_sync(0xffffffffu, front);
    if (lane == 0) warp_base[warp] = __popc(bal);
    __syncthreads();
    int base = 0;
    for (int w = 0; w < warp; ++w) base += warp_base[w];
    // the receiver's own position and normal terms are summed over the warp (all 32 lanes
    // share receiver i) and added once per warp
    float3 dpi = make_float3(0.f, 0.f, 0.f), gni = make_float3(0.f, 0.f, 0.f);
    auto body = [&]() {
        if (!front) return;
        const long long e = chunk_off[blk] + base + __popc(bal & ((1u << lane) - 1u));
        const float g = gpair[e];
        const float4 gs = GEO ? gq[e] : make_float4(0.f, 0.f, 0.f, 0.f);
        if (g == 0.f && gs.x == 0.f && gs.y == 0.f && gs.z == 0.f) return;
        float r;
        const float3 d = unit_dir(dv, r);
        const float3 pj = f3(sc.P[j]), nj = f3(sc.N4[j]);
        const float Aj = __ldg(&aarea[j]), dAj = __ldg(&daarea[j]), lj = __ldg(&lam[j]);
        const float nid = dot3(ni, d), njd = dot3(nj, d);
        const float geo = fabsf(nid) * fabsf(njd) / (r * r);
        float Tnz = 1.f;
        int nzero = 0;
        auto pass1 = [&](int k) {
            float gk, tk;
            if (!pair_occluder(sc, k, i, j, pi, d, r, pj, eps, gk, tk)) return;
            const float om = 1.f - alpha_of(sc, __ldg(&sc.P[k].w), gk);
            if (om == 0.f) ++nzero;
            else Tnz *= om;
        };
        if (!bvh_traverse(sc, pi, d, r, pass1)) atomicAdd(&flags[FLAG_STACK], 1);
        const float T = nzero ? 0.f : Tnz;
        if (dlam) atomicAdd(&dlam[j], g * Aj * T * geo);
        if (dop && T != 0.f) atomicAdd(&dop[j], g * lj * dAj * T * geo);
        float3 gd = make_float3(gs.x, gs.y, gs.z), gpi = make_float3(0.f, 0.f, 0.f);
        float gr = 0.f;
        if constexpr (GEO) {
            const float f = g * lj * Aj * T / (r * r), sj = njd >= 0.f ? 1.f : -1.f;
            gd = gd + f * (fabsf(njd) * ni + (fabsf(nid) * sj) * nj);
            gr = g * lj * Aj * T * (-2.f * geo / r);
            const float fs = g * lj * T * geo * Aj;
            geo_add2(ds + 2 * (size_t)j, fs * __ldg(&sc.FU[j].w), fs * __ldg(&sc.FV[j].w));
            // normals through geo: d geo/d n_i = |n_j.d| d / r^2, d geo/d n_j = (n_i.d) sgn(n_j.d) d / r^2
            const float fi = f * fabsf(njd), fj = f * fabsf(nid) * sj;
            gni = gni + fi * d;
            geo_add3(gF + GEO_GF * (size_t)j + GEO_N, fj * d);
        }
        if ((dop || GEO) && nzero <= 1 && g != 0.f) {
            const float q = -g * lj * Aj * geo;
            auto pass2 = [&](int k) {
                float gk, tk;
                if (!pair_occluder(sc, k, i, j, pi, d, r, pj, eps, gk, tk)) return;
                const float ok = __ldg(&sc.P[k].w);
                const float om = 1.f - alpha_of(sc, ok, gk);
                float others;
                if (nzero == 0) others = Tnz / om;
                else others = (om == 0.f) ? Tnz : 0.f;
                if (others == 0.f) return;
                if (dop) atomicAdd(&dop[k], q * others * dalpha_do(sc, ok, gk));
                if constexpr (GEO) {
                    const float coef = q * others * dalpha_dq(sc, ok, gk);
                    if (coef == 0.f) return;
                    float uu, vv;
                    const float3 pw = crossing_pw(sc, k, pi, d, tk, uu, vv);
                    gpi = gpi + coef * pw;
                    gd = gd + (coef * tk) * pw;
                    geo_add3(dp + GEO_DP * (size_t)k, (-coef) * pw);
                    geo_add2(ds + 2 * (size_t)k, coef * (-2.f * uu * uu * __ldg(&sc.FU[k].w)),
                             coef * (-2.f * vv * vv * __ldg(&sc.FV[k].w)));
                    occluder_frame_grad(sc, k, pi, d, tk, uu, vv, coef, gF);
                }
            };
            bvh_traverse(sc, pi, d, r, pass2);
        }
        if constexpr (GEO) {
            const float dd = dot3(d, gd);
            const float3 gp = make_float3((gd.x - d.x * dd) / r + d.x * gr, (gd.y - d.y * dd) / r + d.y * gr,
                                          (gd.z - d.z * dd) / r + d.z * gr);
            geo_add3(dp + GEO_DP * (size_t)j, gp);
            dpi = gpi - gp;
        }
    };
    body();
    if constexpr (!GEO) return;
    float red[6] = {dpi.x, dpi.y, dpi.z, gni.x, gni.y, gni.z};
#pragma unroll
    for (int q = 0; q < 6; ++q)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) red[q] += __shfl_xor_sync(0xffffffffu, red[q], off);
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            if (red[q] != 0.f) atomicAdd(&dp[GEO_DP * (size_t)i + q], red[q]);
            if (red[3 + q] != 0.f) atomicAdd(&gF[GEO_GF * (size_t)i + GEO_N + q], red[3 + q]);
        }
    }
}

// geometry gradients back to the caller's order; the frame's (dL/dt^u, dL/dt^v, dL/dn)
// carried back through the Gram-Schmidt construction of Eq. G: n = t^u x t^v,
// t^v = b'/|b'| with b' = tv - (t^u.tv) t^u, t^u = tu/|tu| (GS holds |tu|, |b'|, t^u.tv)
__global__ void k_geo_out(SceneDev sc, const float4 *__restrict__ GS, int n, const int *__restrict__ uid,
                          const float *__restrict__ dp_acc, const float *__restrict__ ds_acc,
                          const float *__restrict__ gF, float *dp, float *ds, float *dtu, float *dtv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int o = uid[i];
    if (dp)
        for (int a = 0; a < 3; ++a) dp[3 * o + a] = dp_acc[GEO_DP * (size_t)i + a];
    if (ds)
        for (int a = 0; a < 2; ++a) ds[2 * o + a] = ds_acc[2 * i + a];
    if (!dtu && !dtv) return;
    const float3 tu = f3(sc.FU[i]), tv = f3(sc.FV[i]);
    const float4 gs = GS[i];
    const float *g = gF + GEO_GF * (size_t)i;
    const float3 Gn = make_float3(g[GEO_N], g[GEO_N + 1], g[GEO_N + 2]);
    const float3 cu = make_float3(tv.y * Gn.z - tv.z * Gn.y, tv.z * Gn.x - tv.x * Gn.z, tv.x * Gn.y - tv.y * Gn.x);
    const float3 cv = make_float3(Gn.y * tu.z - Gn.z * tu.y, Gn.z * tu.x - Gn.x * tu.z, Gn.x * tu.y - Gn.y * tu.x);
    float3 Gu = make_float3(g[GEO_TU] + cu.x, g[GEO_TU + 1] + cu.y, g[GEO_TU + 2] + cu.z);
    const float3 Gv = make_float3(g[GEO_TV] + cv.x, g[GEO_TV + 1] + cv.y, g[GEO_TV + 2] + cv.z);
    const float vg = dot3(tv, Gv);
    const float3 gb = (1.f / gs.y) * (Gv - vg * tv);
    const float3 b = gs.y * tv + gs.z * tu;
    const float ugb = dot3(tu, gb);
    Gu = Gu - (gs.z * gb + ugb * b);
    const float ug = dot3(tu, Gu);
    const float3 du = (1.f / gs.x) * (Gu - ug * tu), dv = gb - ugb * tu;
    if (dtu) {
        dtu[3 * o] = du.x;
        dtu[3 * o + 1] = du.y;
        dtu[3 * o + 2] = du.z;
    }
    if (dtv) {
        dtv[3 * o] = dv.x;
        dtv[3 * o + 1] = dv.y;
        dtv[3 * o + 2] = dv.z;
    }
}

__global__ void k_lam_out(int n, const int *__restrict__ uid, const float *__restrict__ dlam, float *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[uid[i]] = dlam[i];
}

} // namespace

// ------------------------------------------------------------------ host side
rgs_status rgs_trace_pairs_impl(rgs_transport *t, const rgs_lights *L, const float *lambda, cudaStream_t st) {
    rgs_status r;
    t->kind = RGS_KIND_PAIRS;
    rgs_tc_invalidate(t);
    rgs_mc_free(t);
    t->tc_used = false;
    t->nd = 0;
    if ((r = rgs_transport_common(t, L, st)) != RGS_OK) return r;
    const int n = t->n;
    const int chunks = (n + PCH - 1) / PCH;
    const long long nchunk = (long long)n * chunks;
    if (nchunk >= (1ll << 31)) {
        rgs_set_error("rgs_trace_pairs: %d surfels give too many (receiver, source-chunk) blocks", n);
        return RGS_ERR_ARG;
    }
    if (nchunk > t->chunk_cap) {
        if ((r = dev_alloc(&t->chunk_cnt, (size_t)nchunk, &t->device_bytes)) != RGS_OK) return r;
        if ((r = dev_alloc(&t->chunk_off, (size_t)nchunk + 1, &t->device_bytes)) != RGS_OK) return r;
        t->chunk_tmp_cap = rgs_scan_tmp_size((int)nchunk);
        if ((r = dev_alloc(&t->chunk_tmp, (size_t)t->chunk_tmp_cap, &t->device_bytes)) != RGS_OK) return r;
        t->chunk_cap = nchunk;
    }
    if (n > t->lam_cap) {
        if ((r = dev_alloc(&t->lam, (size_t)n, &t->device_bytes)) != RGS_OK) return r;
        if ((r = dev_alloc(&t->aarea, (size_t)n, &t->device_bytes)) != RGS_OK) return r;
        if ((r = dev_alloc(&t->daarea, (size_t)n, &t->device_bytes)) != RGS_OK) return r;
        if ((r = dev_alloc(&t->pair_off, (size_t)n + 1, &t->device_bytes)) != RGS_OK) return r;
        t->lam_cap = n;
    }
    SceneDev sd = t->sc->dev();
    { ProfScope ps_("k_lam_in", st); k_lam_in<<<(n + 255) / 256, 256, 0, st>>>(n, t->sc->uid, lambda, t->lam); }
    { ProfScope ps_("k_alpha_area", st); k_alpha_area<<<(n + 255) / 256, 256, 0, st>>>(sd, t->aarea, t->daarea); }
    RGS_CUDA(cudaMemsetAsync(t->flags, 0, sizeof(int) * FLAG_COUNT, st));
    RGS_CUDA(cudaMemsetAsync(t->src_cnt, 0, sizeof(int) * n, st));
    { ProfScope ps_("k_pair_count", st); k_pair_count<<<(unsigned)nchunk, PCH, 0, st>>>(sd, n, chunks, t->chunk_cnt, t->src_cnt); }
    RGS_LAUNCH("pair count");
    if ((r = rgs_scan_counts(t->chunk_cnt, t->chunk_off, (int)nchunk, t->chunk_tmp, t->chunk_tmp_cap, st)) != RGS_OK)
        return r;
    long long total = 0;
    RGS_CUDA(cudaMemcpyAsync(&total, t->chunk_off + nchunk, sizeof total, cudaMemcpyDeviceToHost, st));
    RGS_CUDA(cudaStreamSynchronize(st));
    if (total > t->pair_cap) {
        if ((r = dev_alloc(&t->pair_rec, (size_t)total, &t->device_bytes)) != RGS_OK) return r;
        t->pair_cap = total;
    }
    t->n_pairs = total;
    t->n_hits = total;
    t->n_slots = total;
    t->n_full = 0;
    { ProfScope ps_("k_pair_fill", st); k_pair_fill<<<(unsigned)nchunk, PCH, 0, st>>>(sd, n, chunks, t->chunk_off, t->lam, t->aarea, t->pair_rec, t->flags); }
    { ProfScope ps_("k_pair_off", st); k_pair_off<<<(n + 256) / 256, 256, 0, st>>>(t->chunk_off, chunks, n, t->pair_off); }
    RGS_LAUNCH("pair fill");
    if ((r = rgs_direct_term(t, st)) != RGS_OK) return r;
    // per-source counts -> offsets of the transposed index (filled by the adjoint)
    if ((r = rgs_scan_counts(t->src_cnt, t->src_off, n, t->scan_tmp, t->scan_tmp_cap, st)) != RGS_OK) return r;
    int flags[FLAG_COUNT];
    RGS_CUDA(cudaMemcpyAsync(flags, t->flags, sizeof flags, cudaMemcpyDeviceToHost, st));
    RGS_CUDA(cudaStreamSynchronize(st));
    if (flags[FLAG_STACK]) {
        rgs_set_error("BVH traversal stack overflow on %d segments", flags[FLAG_STACK]);
        return RGS_ERR_CAPACITY;
    }
    return RGS_OK;
}

template <int NC>
rgs_status pairs_bounce(const rgs_transport *t, bool rows16, const float *Bprev, const __nv_bfloat16 *Bprev16,
                        const float *S, float *Q, float *Bout, __nv_bfloat16 *Bout16, double *norm2, cudaStream_t st) {
    dim3 grid(t->n, t->C / 3);
    SceneDev sd = t->sc->dev();
    if (rows16) {
        ProfScope ps_("k_bounce_pairs", st);
        k_bounce_pairs<NC, 3, SliceH<NC>><<<grid, BOUNCE_THREADS, 0, st>>>(sd, t->pair_off, t->pair_rec, t->C, Bprev16,
                                                                         Bprev, S, Q, Bout, Bout16, norm2);
    } else {
        ProfScope ps_("k_bounce_pairs", st);
        k_bounce_pairs<NC, 3, Slice<NC>><<<grid, BOUNCE_THREADS, 0, st>>>(sd, t->pair_off, t->pair_rec, t->C, Bprev, Bprev,
                                                                        S, Q, Bout, Bout16, norm2);
    }
    RGS_LAUNCH("bounce pairs");
    return RGS_OK;
}
template rgs_status pairs_bounce<1>(const rgs_transport *, bool, const float *, const __nv_bfloat16 *, const float *,
                                    float *, float *, __nv_bfloat16 *, double *, cudaStream_t);
template rgs_status pairs_bounce<4>(const rgs_transport *, bool, const float *, const __nv_bfloat16 *, const float *,
                                    float *, float *, __nv_bfloat16 *, double *, cudaStream_t);
template rgs_status pairs_bounce<9>(const rgs_transport *, bool, const float *, const __nv_bfloat16 *, const float *,
                                    float *, float *, __nv_bfloat16 *, double *, cudaStream_t);
template rgs_status pairs_bounce<16>(const rgs_transport *, bool, const float *, const __nv_bfloat16 *, const float *,
                                     float *, float *, __nv_bfloat16 *, double *, cudaStream_t);

// the transposed pair index: for every source j its entries (receiver i, bits of V_ji) at
// src_off[j] .. src_off[j+1] of tr (entry order within a source unspecified)
rgs_status rgs_pairs_transpose(rgs_transport *t, int2 *tr, cudaStream_t st) {
    const int n = t->n;
    { ProfScope ps_("k_copy_off", st); rgs_copy_offsets(t->src_off, t->cursor, n, st); }
    { ProfScope ps_("k_pair_src_fill", st); k_pair_src_fill<<<n, 256, 0, st>>>(n, t->pair_off, t->pair_rec, t->cursor, tr); }
    RGS_LAUNCH("pair transposed index");
    return RGS_OK;
}

namespace {
struct GeoAcc : RgsGeoAcc { // with the pairs' directional derivatives (all or none)
    float4 *gq = nullptr;
};

template <int NC>
rgs_status run_adjoint_pairs(rgs_transport *t, const float *g, float *dE, float *dad, float *dopo, float *dlam_acc,
                             const GeoAcc &geo, cudaStream_t st) {
    const int n = t->n, C = t->C, nb = t->nb_last;
    const size_t A = t->arr();
    SceneDev sd = t->sc->dev();
    rgs_status r;
    if ((r = rgs_adjoint_prologue(t, NC, g, st)) != RGS_OK) return r;
    for (int a = 1; a <= nb; ++a) {
        { ProfScope ps_("k_adj_src_pairs", st); k_adj_src_pairs<NC><<<n, PAIR_THREADS, 0, st>>>(sd, C, t->src_off, t->tr, t->v + A * (a - 1), t->v + A * a, t->u); }
        RGS_LAUNCH("adjoint pairs");
        if (a <= nb - 1 && (r = rgs_pair_accum(t, NC, t->v + A * a, t->Q + A * (nb - 1 - a), st)) != RGS_OK) return r;
    }
    if ((r = rgs_shadow_backward(t, NC, st, geo.dp, geo.ds, geo.gF)) != RGS_OK) return r;
    if (nb >= 1 && (dopo || dlam_acc || geo.dp)) {
        const int chunks = (n + PCH - 1) / PCH;
        if (geo.dp) {
            ProfScope ps_("k_pair_g", st);
            k_pair_g<NC, true><<<n, PAIR_THREADS, 0, st>>>(sd, C, nb, t->pair_off, t->pair_rec, A, t->v, t->iters, t->gh, geo.gq, geo.gF);
        } else {
            ProfScope ps_("k_pair_g", st);
            k_pair_g<NC, false><<<n, PAIR_THREADS, 0, st>>>(sd, C, nb, t->pair_off, t->pair_rec, A, t->v, t->iters, t->gh, nullptr, nullptr);
        }
        if (geo.dp) {
            ProfScope ps_("k_pair_grad", st);
            k_pair_grad<true><<<(unsigned)((long long)n * chunks), PCH, 0, st>>>(sd, n, chunks, t->chunk_off, t->lam, t->aarea, t->daarea, t->gh, geo.gq, dopo ? t->dop : nullptr, dlam_acc, geo.dp, geo.ds, geo.gF, t->flags);
        } else {
            ProfScope ps_("k_pair_grad", st);
            k_pair_grad<false><<<(unsigned)((long long)n * chunks), PCH, 0, st>>>(sd, n, chunks, t->chunk_off, t->lam, t->aarea, t->daarea, t->gh, nullptr, dopo ? t->dop : nullptr, dlam_acc, nullptr, nullptr, nullptr, t->flags);
        }
        RGS_LAUNCH("pair backward");
    }
    return rgs_adjoint_finalize(t, NC, dE, dad, dopo, st);
}
} // namespace

rgs_status rgs_adjoint_pairs_impl(rgs_transport *t, const float *g, float *dE, float *dad, float *dop, float *dlam,
                                  float *dp, float *ds, float *dtu, float *dtv, cudaStream_t st) {
    rgs_status r;
    const int nb = t->nb_last, n = t->n;
    const size_t A = t->arr();
    if (n > t->pg_cap) {
        if ((r = dev_alloc(&t->Pg, (size_t)n * 12, &t->device_bytes)) != RGS_OK) return r;
        if ((r = dev_alloc(&t->dop, (size_t)n, &t->device_bytes)) != RGS_OK) return r;
        t->pg_cap = n;
    }
    float *dlam_acc = nullptr;
    GeoAcc geo;
    const bool want_geo = dp || ds || dtu || dtv;
    struct Scratch {
        rgs_transport *t;
        cudaStream_t st;
        float **dl;
        GeoAcc *geo;
        ~Scratch() {
            pool_release(t->v, st);
            pool_release(t->u, st);
            pool_release(t->tr, st);
            pool_release(t->gh, st);
            pool_release(*dl, st);
            pool_release(geo->dp, st);
            pool_release(geo->ds, st);
            pool_release(geo->gq, st);
            pool_release(geo->gF, st);
        }
    } scratch{t, st, &dlam_acc, &geo};
    if ((r = pool_alloc(&t->v, A * (nb + 1), st)) != RGS_OK) return r;
    if ((r = pool_alloc(&t->u, A, st)) != RGS_OK) return r;
    if ((r = pool_alloc(&t->tr, (size_t)std::max(t->n_pairs, 1ll), st)) != RGS_OK) return r;
    if ((dop || dlam || want_geo) && nb >= 1 && (r = pool_alloc(&t->gh, (size_t)std::max(t->n_pairs, 1ll), st)) != RGS_OK)
        return r; // g per pair
    if (dlam) {
        if ((r = pool_alloc(&dlam_acc, (size_t)n, st)) != RGS_OK) return r;
        RGS_CUDA(cudaMemsetAsync(dlam_acc, 0, sizeof(float) * n, st));
    }
    if (want_geo) {
        if ((r = pool_alloc(&geo.dp, (size_t)n * GEO_DP, st)) != RGS_OK) return r;
        if ((r = pool_alloc(&geo.ds, (size_t)n * 2, st)) != RGS_OK) return r;
        if ((r = pool_alloc(&geo.gq, (size_t)std::max(t->n_pairs, 1ll), st)) != RGS_OK) return r;
        if ((r = pool_alloc(&geo.gF, (size_t)n * GEO_GF, st)) != RGS_OK) return r;
        RGS_CUDA(cudaMemsetAsync(geo.dp, 0, sizeof(float) * n * GEO_DP, st));
        RGS_CUDA(cudaMemsetAsync(geo.ds, 0, sizeof(float) * n * 2, st));
        RGS_CUDA(cudaMemsetAsync(geo.gF, 0, sizeof(float) * n * GEO_GF, st));
    }
    if ((r = rgs_pairs_transpose(t, t->tr, st)) != RGS_OK) return r;
    RGS_CUDA(cudaMemsetAsync(t->flags, 0, sizeof(int) * FLAG_COUNT, st));
    switch (t->nc) {
    case 1: r = run_adjoint_pairs<1>(t, g, dE, dad, dop, dlam_acc, geo, st); break;
    case 4: r = run_adjoint_pairs<4>(t, g, dE, dad, dop, dlam_acc, geo, st); break;
    case 9: r = run_adjoint_pairs<9>(t, g, dE, dad, dop, dlam_acc, geo, st); break;
    default: r = run_adjoint_pairs<16>(t, g, dE, dad, dop, dlam_acc, geo, st);
    }
    if (r != RGS_OK) return r;
    if (dlam) {
        { ProfScope ps_("k_lam_out", st); k_lam_out<<<(n + 255) / 256, 256, 0, st>>>(n, t->sc->uid, dlam_acc, dlam); }
        RGS_LAUNCH("lambda gradient");
    }
    if (want_geo) return rgs_geometry_out(t, geo, dp, ds, dtu, dtv, st);
    return RGS_OK;
}

rgs_status rgs_geometry_out(rgs_transport *t, const RgsGeoAcc &acc, float *dp, float *ds, float *dtu, float *dtv,
                            cudaStream_t st) {
    const int n = t->n;
    { ProfScope ps_("k_geo_out", st); k_geo_out<<<(n + 255) / 256, 256, 0, st>>>(t->sc->dev(), t->sc->GS, n, t->sc->uid, acc.dp, acc.ds, acc.gF, dp, ds, dtu, dtv); }
    RGS_LAUNCH("geometry gradients");
    return RGS_OK;
}
