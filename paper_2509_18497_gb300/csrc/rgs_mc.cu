// The Monte-Carlo TD(0) solver of Sec. 7 (Alg. 1) with next-event estimation by weighted
// reservoir sampling and the variance-driven receiver selection of App. "Monte-Carlo Solver
// Details", on the center-to-center transport (rgs_mc_solve, rgs_mc_estimate, rgs_mc_groups), and
// the shooting (progressive refinement) solver of the same section (rgs_prog_refine).
//
// Step t = 1..T draws N estimates.  Draw q's receiver is a = q while t <= 8, afterwards a
// draw with replacement with probability proportional to each receiver's tracked variance
// (an FP64 scan of the variances in caller order and a binary search of the draw's uniform).
// Its next event is one of a's pairs, picked by a single-item weighted reservoir (Chao's
// scheme) streamed over a's pairs in caller order of the source (the transport stores them in
// internal order; a per-receiver sorted copy, cached with the transport, gives the caller
// order), with proxy weights
//     w_b = geo_ab (sum_c lum(c) |Y(-d)^T Bhat_b[c]| + floor),  floor = 1e-9 (1 + mean lum),
// or, with K-means groups, first a group by its proxy (mean centre, mean normal, the sum of
// its members' means; zero for a group holding none of a's sources), then a pair inside it.
// The estimate delta = S_a + (1/p_b) K_ab Bhat_b updates the receiver's FP64 sums
// S += delta, S2 += delta^2, D += 1; every draw of a step reads the previous step's means
// Bhat = S / D (the running mean is TD(0) with learning rate 1/(t+1)).
//
// GPU form: one 128-thread block per draw.  The reservoir's running sum over a chunk of 128
// candidates is a block-wide FP64 inclusive scan, so every candidate's keep decision
// u_k W_k < w_k is taken in parallel; the kept candidate is the last one whose decision holds.
// The uniforms are SplitMix64 outputs keyed by (seed, step, draw, stream) -- stream 0 the
// receiver selection, 1000 + k the k-th candidate, draw q + 2^30 for the group stage -- so a
// draw is reproducible from its key alone.  K-means (Lloyd's iterations on centre and normal,
// FP64) runs once per (transport, group count) and is cached.
#include <algorithm>
#include <vector>

#include "rgs_internal.cuh"

struct rgs_mc_cache {
    int G = 0;            // groups of the cached K-means result (0: none)
    int *assign = nullptr; // [n] internal order
    double *gc = nullptr, *gn = nullptr; // [G][3]
    long long bytes = 0;
    int2 *rec = nullptr; // [n_pairs] the transport's pair records, each receiver's by caller index of the source
    long long rec_bytes = 0;
};

namespace {

constexpr int MT = 128;      // threads per draw
constexpr int MC_GMAX = 1024; // most K-means groups
constexpr unsigned long long MC_GROUP_DRAW = 0x40000000ull;

__device__ __forceinline__ double mc_uniform(unsigned long long seed, unsigned long long t, unsigned long long q,
                                             unsigned long long stream) {
    const unsigned long long k = splitmix64(splitmix64(splitmix64(seed) + t) + q) + stream;
    return (double)(splitmix64(k) >> 11) * (1.0 / 9007199254740992.0); // 53 bits in [0, 1)
}
// Rec. 709 luminance weight of column c (columns are RGB triples per light)
__device__ __forceinline__ float lum_w(int c) {
    const int ch = c % 3;
    return ch == 0 ? 0.2126f : (ch == 1 ? 0.7152f : 0.0722f);
}

// inclusive FP64 scan over the block (MT threads); sh: MT / 32 doubles.  Ends synchronised.
__device__ __forceinline__ double block_scan(double v, double *sh, double &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) sh[warp] = v;
    __syncthreads();
    double base = 0.0;
    total = 0.0;
#pragma unroll
    for (int w = 0; w < MT / 32; ++w) {
        if (w < warp) base += sh[w];
        total += sh[w];
    }
    __syncthreads();
    return base + v;
}

// Single-item weighted reservoir over candidates 0..count-1 in order: candidate k (weight
// wf(k) > 0) replaces the kept one when u_k W_k < w_k, W_k the running sum.  Returns the
// kept index (-1 if none), the total weight and the kept weight (to every thread).
template <class WF>
__device__ long long reservoir(long long count, WF &&wf, unsigned long long seed, int t, unsigned long long q,
                               double &tot, double &wkept, double *sh_scan, long long *sh_pick, double *sh_w) {
    double carry = 0.0;
    long long mine = -1;
    double mine_w = 0.0;
    for (long long base = 0; base < count; base += MT) {
        const long long k = base + threadIdx.x;
        const double w = k < count ? (double)wf(k) : 0.0;
        double chunk;
        const double W = carry + block_scan(w, sh_scan, chunk);
        if (w > 0.0 && mc_uniform(seed, (unsigned long long)t, q, 1000ull + (unsigned long long)k) * W < w) {
            mine = k;
            mine_w = w;
        }
        carry += chunk;
    }
    // the last kept candidate: block-wide maximum of the per-thread last keeps
    long long best = mine;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = max(best, (long long)__shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) sh_pick[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long b = -1;
        for (int w = 0; w < MT / 32; ++w) b = max(b, sh_pick[w]);
        sh_pick[0] = b;
    }
    __syncthreads();
    const long long pick = sh_pick[0];
    if (pick >= 0 && mine == pick) *sh_w = mine_w;
    __syncthreads();
    wkept = pick >= 0 ? *sh_w : 0.0;
    tot = carry;
    __syncthreads();
    return pick;
}

struct McArgs {
    SceneDev sc;
    int n, C;
    const long long *pair_off;
    const int2 *rec;
    const float *S;    // [n][C][NC] internal
    const float *Bhat; // [n][C][NC] internal
    const double *lum_acc; // sum over Bhat of lum(c) |Bhat|, for the floor
    // groups (G = 0: flat)
    int G;
    const int *assign;
    const double *gc, *gn, *Bsum; // [G][3], [G][3], [G][C][NC]
    unsigned long long seed;
    int t;
    int n_draws;
    const int *recv; // caller receiver of each draw (null: draw q -> receiver q)
    // solve: the receivers' FP64 sums; estimate: per-draw outputs
    double *SB, *SB2, *D;
    long long *pick_out;
    double *p_out;
    float *delta_out; // [n_draws][nc][C] caller layout
    int *bad;         // count of draws whose receiver index is out of range
};

// sort keys of the pair records: the caller index of the source
__global__ void k_mc_rec_keys(long long n_pairs, const int2 *__restrict__ rec, const int *__restrict__ uid,
                              uint32_t *key, uint2 *val) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n_pairs;
         e += (long long)gridDim.x * blockDim.x) {
        const int2 r = rec[e];
        key[e] = (uint32_t)__ldg(&uid[r.x]);
        val[e] = make_uint2((uint32_t)r.x, (uint32_t)r.y);
    }
}

template <int NC>
__device__ __forceinline__ float row_lum(const float *Y, const float *X, int C) {
    float lum = 0.f;
    for (int c = 0; c < C; ++c) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < NC; ++k) s += Y[k] * __ldg(X + (size_t)c * NC + k);
        lum += lum_w(c) * fabsf(s);
    }
    return lum;
}

template <int NC>
__global__ void __launch_bounds__(MT) k_mc_draw(McArgs A) {
    __shared__ double sh_scan[MT / 32];
    __shared__ long long sh_pick[MT / 32];
    __shared__ double sh_w;
    __shared__ unsigned has[MC_GMAX / 32];
    __shared__ float wg[MC_GMAX];
    __shared__ float Yo[NC], Yi[NC];
    __shared__ float sh_V;
    __shared__ int sh_j;
    const int q = blockIdx.x;
    if (q >= A.n_draws) return;
    const SceneDev &sc = A.sc;
    const int ac = A.recv ? A.recv[q] : q; // caller index of the receiver
    if (ac < 0 || ac >= A.n) { // the whole block leaves: no estimate for this draw
        if (threadIdx.x == 0) {
            if (A.bad) atomicAdd(A.bad, 1);
            if (A.pick_out) A.pick_out[q] = -1;
            if (A.p_out) A.p_out[q] = 0.0;
        }
        return;
    }
    const int i = __ldg(&sc.inv[ac]);
    const long long e0 = A.pair_off[i], np = A.pair_off[i + 1] - e0;
    const float3 pa = f3(sc.P[i]), na = f3(sc.N4[i]);
    const float fl = (float)(1e-9 * (1.0 + *A.lum_acc / (double)A.n));
    const int C = A.C;
    // the flat proxy of a's k-th pair (0 outside the group gsel when one is given)
    auto pair_w = [&](long long k, int gsel) -> float {
        const int2 jv = __ldg(&A.rec[e0 + k]);
        if (gsel >= 0 && __ldg(&A.assign[jv.x]) != gsel) return 0.f;
        const float3 pj = f3(sc.P[jv.x]), nj = f3(sc.N4[jv.x]);
        float3 d = make_float3(pj.x - pa.x, pj.y - pa.y, pj.z - pa.z);
        const float r2 = dot3(d, d), r = sqrtf(r2);
        d = (1.f / r) * d;
        const float geo = fabsf(dot3(na, d)) * fabsf(dot3(nj, d)) / r2;
        float Y[NC];
        sh_eval<NC>(neg3(d), Y);
        return geo * (row_lum<NC>(Y, A.Bhat + (size_t)jv.x * C * NC, C) + fl);
    };
    double tot = 0.0, wk = 0.0, p = 0.0;
    long long pick = -1;
    if (A.G == 0) {
        pick = reservoir(np, [&](long long k) { return pair_w(k, -1); }, A.seed, A.t, (unsigned long long)q, tot, wk,
                         sh_scan, sh_pick, &sh_w);
        if (pick >= 0) p = wk / tot;
    } else {
        const int G = A.G;
        for (int w = threadIdx.x; w < MC_GMAX / 32; w += MT) has[w] = 0u;
        __syncthreads();
        for (long long k = threadIdx.x; k < np; k += MT) {
            const int g = __ldg(&A.assign[__ldg(&A.rec[e0 + k]).x]);
            atomicOr(&has[g >> 5], 1u << (g & 31));
        }
        __syncthreads();
        for (int g = threadIdx.x; g < G; g += MT) {
            float w = 0.f;
            if (has[g >> 5] >> (g & 31) & 1u) {
                double wv[3] = {A.gc[g * 3] - pa.x, A.gc[g * 3 + 1] - pa.y, A.gc[g * 3 + 2] - pa.z};
                const double r2 = wv[0] * wv[0] + wv[1] * wv[1] + wv[2] * wv[2] + 1e-24, r = sqrt(r2);
                for (int a = 0; a < 3; ++a) wv[a] /= r;
                float Y[NC];
                sh_eval<NC>(make_float3((float)-wv[0], (float)-wv[1], (float)-wv[2]), Y);
                double lum = 0.0;
                const double *X = A.Bsum + (size_t)g * C * NC;
                for (int c = 0; c < C; ++c) {
                    double s = 0.0;
#pragma unroll
                    for (int k = 0; k < NC; ++k) s += (double)Y[k] * X[(size_t)c * NC + k];
                    lum += (double)lum_w(c) * fabs(s);
                }
                const double geo = fabs(na.x * wv[0] + na.y * wv[1] + na.z * wv[2]) *
                                   fabs(A.gn[g * 3] * wv[0] + A.gn[g * 3 + 1] * wv[1] + A.gn[g * 3 + 2] * wv[2]) / r2;
                w = (float)((geo + 1e-12) * (lum + (double)fl));
            }
            wg[g] = w;
        }
        __syncthreads();
        double totg = 0.0, wgk = 0.0;
        const long long gsel = reservoir(G, [&](long long g) { return wg[g]; }, A.seed, A.t,
                                         (unsigned long long)q + MC_GROUP_DRAW, totg, wgk, sh_scan, sh_pick, &sh_w);
        if (gsel >= 0) {
            pick = reservoir(np, [&](long long k) { return pair_w(k, (int)gsel); }, A.seed, A.t, (unsigned long long)q,
                             tot, wk, sh_scan, sh_pick, &sh_w);
            if (pick >= 0) p = wgk / totg * (wk / tot);
        }
    }
    // delta = S_a + (1/p) o_a c_a (x) Y(R_a d) V_ba Y(-d)^T Bhat_b
    if (threadIdx.x == 0) {
        sh_j = -1;
        if (pick >= 0 && p > 0.0) {
            const int2 jv = __ldg(&A.rec[e0 + pick]);
            const float3 pj = f3(sc.P[jv.x]);
            float3 d = make_float3(pj.x - pa.x, pj.y - pa.y, pj.z - pa.z);
            d = (1.f / sqrtf(dot3(d, d))) * d;
            sh_eval<NC>(neg3(d), Yo);
            sh_eval<NC>(reflect_n(na, d), Yi);
            sh_V = __int_as_float(jv.y);
            sh_j = jv.x;
        }
    }
    __syncthreads();
    const int j = sh_j;
    const float scale = j >= 0 ? (float)((double)sh_V / p) : 0.f;
    const float oa = alpha_center(sc, i);
    for (int e = threadIdx.x; e < C * NC; e += MT) {
        const int c = e / NC, k = e - c * NC;
        const size_t idx = (size_t)i * C * NC + e;
        float v = __ldg(&A.S[idx]);
        if (j >= 0) {
            const float *Bj = A.Bhat + ((size_t)j * C + c) * NC;
            float sv = 0.f;
#pragma unroll
            for (int kk = 0; kk < NC; ++kk) sv += Yo[kk] * __ldg(Bj + kk);
            v += oa * sc.cl[(size_t)i * 12 + band_of(k) * 3 + (c % 3)] * Yi[k] * scale * sv;
        }
        if (A.SB) {
            atomicAdd(&A.SB[idx], (double)v);
            atomicAdd(&A.SB2[idx], (double)v * (double)v);
        } else {
            A.delta_out[((size_t)q * NC + k) * C + c] = v;
        }
    }
    if (threadIdx.x == 0) {
        if (A.SB) atomicAdd(&A.D[i], 1.0);
        if (A.pick_out) A.pick_out[q] = pick;
        if (A.p_out) A.p_out[q] = p;
    }
}

// sum over the means of lum(c) |Bhat| (the proposal's floor)
__global__ void k_mc_lum(size_t M, int C, int NC, const float *__restrict__ Bhat, double *acc) {
    double s = 0.0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < M; e += (size_t)gridDim.x * blockDim.x)
        s += (double)lum_w((int)((e / NC) % C)) * fabs((double)Bhat[e]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(acc, s);
}

// Bhat = S / D where D > 0
__global__ void k_mc_mean(size_t M, int R, const double *__restrict__ SB, const double *__restrict__ D, float *Bhat) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= M) return;
    const double d = D[e / R];
    if (d > 0.0) Bhat[e] = (float)(SB[e] / d);
}

// tracked variance of every receiver, caller order: sum_k S2/D - (S/D)^2, clamped, + 1e-30
__global__ void k_mc_var(int n, int R, const int *__restrict__ inv, const double *__restrict__ SB,
                         const double *__restrict__ SB2, const double *__restrict__ D, double *var) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    const int i = inv[a];
    const double d = D[i];
    double v = 0.0;
    for (int k = 0; k < R; ++k) {
        const double m = SB[(size_t)i * R + k] / d;
        v += SB2[(size_t)i * R + k] / d - m * m;
    }
    var[a] = (v > 0.0 ? v : 0.0) + 1e-30;
}

// inclusive FP64 prefix sums of n values by one block, chunk after chunk
__global__ void __launch_bounds__(MT) k_mc_scan(int n, const double *__restrict__ x, double *cum) {
    __shared__ double sh[MT / 32];
    double carry = 0.0;
    for (int base = 0; base < n; base += MT) {
        const int k = base + threadIdx.x;
        double chunk;
        const double v = carry + block_scan(k < n ? x[k] : 0.0, sh, chunk);
        if (k < n) cum[k] = v;
        carry += chunk;
    }
}

// draw q's receiver: the first a with u * total < cum[a] (the last one if rounding leaves none)
__global__ void k_mc_select(int n, const double *__restrict__ cum, unsigned long long seed, int t, int *recv) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const double u = mc_uniform(seed, (unsigned long long)t, (unsigned long long)q, 0ull) * cum[n - 1];
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (u < cum[mid]) hi = mid;
        else lo = mid + 1;
    }
    recv[q] = lo;
}

// ---------------------------------------------------------------- K-means (FP64)
// feature of internal surfel i: (p, ext/2 n)
__device__ __forceinline__ void km_feat(const SceneDev &sc, int i, double ext, double *f) {
    const float4 P = sc.P[i], N = sc.N4[i];
    f[0] = P.x;
    f[1] = P.y;
    f[2] = P.z;
    f[3] = 0.5 * ext * N.x;
    f[4] = 0.5 * ext * N.y;
    f[5] = 0.5 * ext * N.z;
}
__global__ void k_km_init(SceneDev sc, int n, int G, const double *ext, double *cen) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= G) return;
    km_feat(sc, sc.inv[(int)((long long)k * n / G)], *ext, cen + 6 * k);
}
__global__ void k_km_assign(SceneDev sc, int n, int G, const double *ext, const double *__restrict__ cen, int *assign,
                            int *changed, double *acc, int *cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double f[6];
    km_feat(sc, i, *ext, f);
    int best = 0;
    double bd = 1e300;
    for (int k = 0; k < G; ++k) {
        double dd = 0.0;
#pragma unroll
        for (int a = 0; a < 6; ++a) dd += (f[a] - cen[6 * k + a]) * (f[a] - cen[6 * k + a]);
        if (dd < bd) {
            bd = dd;
            best = k;
        }
    }
    if (assign[i] != best) *changed = 1;
    assign[i] = best;
    atomicAdd(&cnt[best], 1);
#pragma unroll
    for (int a = 0; a < 6; ++a) atomicAdd(&acc[6 * best + a], f[a]);
}
__global__ void k_km_update(int G, const double *__restrict__ acc, const int *__restrict__ cnt, double *cen) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 6 * G) return;
    const int k = e / 6;
    if (cnt[k]) cen[e] = acc[e] / cnt[k];
}
// the scene's largest extent over the axes (at least 1e-12)
__global__ void k_km_extent(SceneDev sc, int n, double *ext) {
    __shared__ float lo[3][256], hi[3][256];
    float l[3] = {INFINITY, INFINITY, INFINITY}, h[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float4 P = sc.P[i];
        l[0] = fminf(l[0], P.x), l[1] = fminf(l[1], P.y), l[2] = fminf(l[2], P.z);
        h[0] = fmaxf(h[0], P.x), h[1] = fmaxf(h[1], P.y), h[2] = fmaxf(h[2], P.z);
    }
    for (int a = 0; a < 3; ++a) lo[a][threadIdx.x] = l[a], hi[a][threadIdx.x] = h[a];
    __syncthreads();
    if (threadIdx.x == 0) {
        double e = 1e-12;
        for (int a = 0; a < 3; ++a) {
            float mn = INFINITY, mx = -INFINITY;
            for (int k = 0; k < (int)blockDim.x; ++k) mn = fminf(mn, lo[a][k]), mx = fmaxf(mx, hi[a][k]);
            e = fmax(e, (double)mx - (double)mn);
        }
        *ext = e;
    }
}
// group centres (mean p) and normals (normalised mean n, 0 if degenerate)
__global__ void k_km_groups(SceneDev sc, int n, int G, const int *__restrict__ assign, double *acc, int *cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 P = sc.P[i], N = sc.N4[i];
    const int g = assign[i];
    atomicAdd(&cnt[g], 1);
    atomicAdd(&acc[6 * g + 0], (double)P.x);
    atomicAdd(&acc[6 * g + 1], (double)P.y);
    atomicAdd(&acc[6 * g + 2], (double)P.z);
    atomicAdd(&acc[6 * g + 3], (double)N.x);
    atomicAdd(&acc[6 * g + 4], (double)N.y);
    atomicAdd(&acc[6 * g + 5], (double)N.z);
}
__global__ void k_km_finish(int G, const double *__restrict__ acc, const int *__restrict__ cnt, double *gc, double *gn) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const double c = cnt[g];
    const double *a = acc + 6 * g;
    const double ln = sqrt(a[3] * a[3] + a[4] * a[4] + a[5] * a[5]);
    for (int q = 0; q < 3; ++q) {
        gc[3 * g + q] = c > 0 ? a[q] / c : 0.0;
        gn[3 * g + q] = ln > 1e-12 ? a[3 + q] / ln : 0.0;
    }
}
__global__ void k_km_to_user(int n, const int *__restrict__ uid, const int *__restrict__ assign, int *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[uid[i]] = assign[i];
}

template <int NC>
__global__ void k_mc_group_sums(int n, int C, const int *__restrict__ assign, const float *__restrict__ Bhat,
                                double *Bsum) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t R = (size_t)C * NC;
    if (e >= (size_t)n * R) return;
    const float v = Bhat[e];
    if (v != 0.f) atomicAdd(&Bsum[(size_t)assign[e / R] * R + e % R], (double)v);
}

// internal [N][C][NC] <-> user [N][nc][C]
template <int NC>
__global__ void k_mc_from_user(int n, int C, const int *__restrict__ uid, const float *__restrict__ X, float *Y) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * C * NC) return;
    const int k = (int)(idx % NC);
    const size_t ic = idx / NC;
    const int c = (int)(ic % C), i = (int)(ic / C);
    Y[idx] = X[((size_t)uid[i] * NC + k) * C + c];
}
template <int NC>
__global__ void k_mc_to_user(int n, int C, const int *__restrict__ uid, const float *__restrict__ X, float *Y) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * C * NC) return;
    const int k = (int)(idx % NC);
    const size_t ic = idx / NC;
    const int c = (int)(ic % C), i = (int)(ic / C);
    Y[((size_t)uid[i] * NC + k) * C + c] = X[idx];
}
// S = E + D (E user [N][nc][3] broadcast over the lights; D the direct term, internal)
template <int NC>
__global__ void k_mc_make_S(int n, int C, const int *__restrict__ uid, const float *__restrict__ E,
                            const float *__restrict__ D, float *S) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * C * NC) return;
    const int k = (int)(idx % NC);
    const size_t ic = idx / NC;
    const int c = (int)(ic % C), i = (int)(ic / C);
    S[idx] = (E ? E[((size_t)uid[i] * NC + k) * 3 + (c % 3)] : 0.f) + D[idx];
}
__global__ void k_mc_visits(int n, const int *__restrict__ uid, const double *__restrict__ D, float *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[uid[i]] = (float)D[i];
}

// ---------------------------------------------------------------- progressive refinement
// Sec. 7's shooting solver: each shot takes the surfel whose unshot radiance dB has the
// largest luminance (sum over its coefficients and columns of lum(c) |dB|, ties to the lower
// caller index) and sends it to every receiver that has it as a source:
// dB_a += K_a,best dB_best, Bhat_a += the same, then dB_best = 0.
constexpr int PR_T = 256;
struct LumIdx {
    double v;
    int idx; // caller index (n: none)
};
__device__ __forceinline__ LumIdx lum_better(LumIdx a, LumIdx b) {
    return (b.v > a.v || (b.v == a.v && b.idx < a.idx)) ? b : a;
}
__device__ __forceinline__ LumIdx lum_warp(LumIdx x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        LumIdx y;
        y.v = __shfl_xor_sync(0xffffffffu, x.v, o);
        y.idx = __shfl_xor_sync(0xffffffffu, x.idx, o);
        x = lum_better(x, y);
    }
    return x;
}
__device__ __forceinline__ LumIdx lum_block(LumIdx x, LumIdx *sh) {
    x = lum_warp(x);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        x = threadIdx.x < PR_T / 32 ? sh[threadIdx.x] : LumIdx{0.0, 0x7fffffff};
        x = lum_warp(x);
    }
    return x; // valid in thread 0
}
// per-block brightest unshot surfel (luminance > 0 only)
__global__ void __launch_bounds__(PR_T) k_pr_argmax(int n, int C, int NC, const int *__restrict__ uid,
                                                   const float *__restrict__ dB, LumIdx *part) {
    __shared__ LumIdx sh[PR_T / 32];
    LumIdx best{0.0, 0x7fffffff};
    const int i = blockIdx.x * PR_T + threadIdx.x;
    if (i < n) {
        double l = 0.0;
        const float *x = dB + (size_t)i * C * NC;
        for (int e = 0; e < C * NC; ++e) l += (double)lum_w(e / NC) * fabs((double)x[e]);
        if (l > 0.0) best = LumIdx{l, uid[i]};
    }
    best = lum_block(best, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = best;
}
// the shot: the brightest surfel (internal index to *shot_i, -1 if nothing is left), its
// unshot radiance copied to shot and cleared in dB
__global__ void __launch_bounds__(PR_T) k_pr_pick(int nparts, int R, const int *__restrict__ inv,
                                                 const LumIdx *__restrict__ part, float *dB, float *shot, int *shot_i) {
    __shared__ LumIdx sh[PR_T / 32];
    __shared__ int sel;
    LumIdx best{0.0, 0x7fffffff};
    for (int b = threadIdx.x; b < nparts; b += PR_T) best = lum_better(best, part[b]);
    best = lum_block(best, sh);
    if (threadIdx.x == 0) {
        sel = best.v > 0.0 ? inv[best.idx] : -1;
        *shot_i = sel;
    }
    __syncthreads();
    if (sel < 0) return;
    for (int e = threadIdx.x; e < R; e += PR_T) {
        shot[e] = dB[(size_t)sel * R + e];
        dB[(size_t)sel * R + e] = 0.f;
    }
}
// a warp per receiver of the shot's source: dB_a += K_a,j shot, Bhat_a += the same
template <int NC>
__global__ void __launch_bounds__(PR_T) k_pr_scatter(SceneDev sc, int C, const long long *__restrict__ src_off,
                                                    const int2 *__restrict__ tr, const int *__restrict__ shot_i,
                                                    const float *__restrict__ shot, float *dB, float *Bhat) {
    const int j = *shot_i;
    if (j < 0) return;
    const long long e0 = src_off[j], e1 = src_off[j + 1];
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (PR_T / 32);
    const float3 pj = f3(sc.P[j]);
    for (long long e = e0 + blockIdx.x * (PR_T / 32) + (threadIdx.x >> 5); e < e1; e += warps) {
        const int2 iv = tr[e];
        const int a = iv.x;
        const float V = __int_as_float(iv.y);
        const float3 pa = f3(sc.P[a]), na = f3(sc.N4[a]);
        float3 d = make_float3(pj.x - pa.x, pj.y - pa.y, pj.z - pa.z);
        d = (1.f / sqrtf(dot3(d, d))) * d;
        float Yo[NC], Yi[NC];
        sh_eval<NC>(neg3(d), Yo);
        sh_eval<NC>(reflect_n(na, d), Yi);
        const float oa = alpha_center(sc, a);
        for (int c = lane; c < C; c += 32) {
            float sv = 0.f;
#pragma unroll
            for (int k = 0; k < NC; ++k) sv += Yo[k] * shot[c * NC + k];
            const float x = V * sv;
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                const size_t idx = ((size_t)a * C + c) * NC + k;
                const float v = oa * sc.cl[(size_t)a * 12 + band_of(k) * 3 + (c % 3)] * Yi[k] * x;
                dB[idx] += v;
                Bhat[idx] += v;
            }
        }
    }
}

inline unsigned nblk(size_t m, int b) { return (unsigned)((m + b - 1) / b); }

// pooled scratch of one call, returned at its end
struct Scratch {
    cudaStream_t st;
    std::vector<void *> ptrs;
    template <class T> rgs_status get(T **p, size_t count) {
        rgs_status r = pool_alloc(p, count, st);
        if (r == RGS_OK) ptrs.push_back(*p);
        return r;
    }
    ~Scratch() {
        for (void *p : ptrs) pool_free(p, st);
    }
};

rgs_status check_pairs(const rgs_transport *t, const char *what) {
    if (!t) {
        rgs_set_error("%s: NULL transport", what);
        return RGS_ERR_ARG;
    }
    if (t->kind != RGS_KIND_PAIRS) {
        rgs_set_error("%s: the Monte-Carlo solver runs on the center-to-center transport (rgs_trace_pairs)", what);
        return t->kind == RGS_KIND_NONE ? RGS_ERR_STATE : RGS_ERR_ARG;
    }
    return RGS_OK;
}

// K-means groups of t's surfels (cached per group count)
rgs_status ensure_groups(rgs_transport *t, int G, cudaStream_t st) {
    if (G == 0) return RGS_OK;
    if (!t->mc) t->mc = new rgs_mc_cache();
    rgs_mc_cache *m = t->mc;
    if (m->G == G) return RGS_OK;
    m->G = 0;
    rgs_status r;
    const int n = t->n;
    long long acct = m->bytes; // a reallocation takes the old blocks' sizes off
    if ((r = dev_alloc(&m->assign, (size_t)n, &acct)) != RGS_OK) return r;
    if ((r = dev_alloc(&m->gc, (size_t)3 * G, &acct)) != RGS_OK) return r;
    if ((r = dev_alloc(&m->gn, (size_t)3 * G, &acct)) != RGS_OK) return r;
    t->device_bytes += acct - m->bytes;
    m->bytes = acct;
    Scratch s{st};
    double *ext, *cen, *acc;
    int *cnt, *changed;
    if ((r = s.get(&ext, 1)) != RGS_OK || (r = s.get(&cen, (size_t)6 * G)) != RGS_OK ||
        (r = s.get(&acc, (size_t)6 * G)) != RGS_OK || (r = s.get(&cnt, (size_t)G)) != RGS_OK ||
        (r = s.get(&changed, 1)) != RGS_OK)
        return r;
    const SceneDev sd = t->sc->dev();
    { ProfScope ps_("k_km_extent", st); k_km_extent<<<1, 256, 0, st>>>(sd, n, ext); }
    RGS_LAUNCH("k-means extent");
    { ProfScope ps_("k_km_init", st); k_km_init<<<nblk(G, 128), 128, 0, st>>>(sd, n, G, ext, cen); }
    RGS_LAUNCH("k-means init");
    RGS_CUDA(cudaMemsetAsync(m->assign, 0xff, sizeof(int) * n, st)); // -1: unassigned
    for (int it = 0; it < 50; ++it) {
        RGS_CUDA(cudaMemsetAsync(changed, 0, sizeof(int), st));
        RGS_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * 6 * G, st));
        RGS_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * G, st));
        { ProfScope ps_("k_km_assign", st); k_km_assign<<<nblk(n, 128), 128, 0, st>>>(sd, n, G, ext, cen, m->assign, changed, acc, cnt); }
        RGS_LAUNCH("k-means assign");
        { ProfScope ps_("k_km_update", st); k_km_update<<<nblk(6 * G, 128), 128, 0, st>>>(G, acc, cnt, cen); }
        RGS_LAUNCH("k-means update");
        int ch = 0;
        RGS_CUDA(cudaMemcpyAsync(&ch, changed, sizeof(int), cudaMemcpyDeviceToHost, st));
        RGS_CUDA(cudaStreamSynchronize(st));
        if (!ch) break;
    }
    RGS_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * 6 * G, st));
    RGS_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * G, st));
    { ProfScope ps_("k_km_groups", st); k_km_groups<<<nblk(n, 128), 128, 0, st>>>(sd, n, G, m->assign, acc, cnt); }
    RGS_LAUNCH("k-means groups");
    { ProfScope ps_("k_km_finish", st); k_km_finish<<<nblk(G, 128), 128, 0, st>>>(G, acc, cnt, m->gc, m->gn); }
    RGS_LAUNCH("k-means finish");
    m->G = G;
    return RGS_OK;
}

// the caller-ordered copy of t's pair records (cached)
rgs_status ensure_caller_rec(rgs_transport *t, cudaStream_t st) {
    if (!t->mc) t->mc = new rgs_mc_cache();
    rgs_mc_cache *m = t->mc;
    const long long np = t->n_pairs;
    if (m->rec || np == 0) return RGS_OK;
    rgs_status r;
    long long acct = 0;
    if ((r = dev_alloc(&m->rec, (size_t)np, &acct)) != RGS_OK) return r;
    t->device_bytes += acct;
    m->rec_bytes = acct;
    Scratch s{st};
    uint32_t *k0, *k1;
    uint2 *v0;
    if ((r = s.get(&k0, (size_t)np)) != RGS_OK || (r = s.get(&k1, (size_t)np)) != RGS_OK ||
        (r = s.get(&v0, (size_t)np)) != RGS_OK)
        return r;
    const SceneDev sd = t->sc->dev();
    { ProfScope ps_("k_mc_rec_keys", st); k_mc_rec_keys<<<std::min<long long>((np + 255) / 256, 4096), 256, 0, st>>>(np, t->pair_rec, sd.uid, k0, v0); }
    RGS_LAUNCH("mc pair keys");
    // caller indices below 2^24 take three passes (the result in the odd buffers), else four
    uint2 *v1 = reinterpret_cast<uint2 *>(m->rec);
    if (t->n <= (1 << 24)) return rgs_seg_sort(t->pair_off, t->n, 3, k0, v0, k1, v1, st);
    if ((r = rgs_seg_sort(t->pair_off, t->n, 4, k0, v0, k1, v1, st)) != RGS_OK) return r;
    RGS_CUDA(cudaMemcpyAsync(v1, v0, sizeof(uint2) * np, cudaMemcpyDeviceToDevice, st));
    return RGS_OK;
}

// per-step inputs shared by the solve and the estimate: the floor's sum and the group sums
template <int NC>
rgs_status step_inputs(rgs_transport *t, const float *Bhat, double *lum_acc, double *Bsum, int G, cudaStream_t st) {
    const size_t M = t->arr();
    RGS_CUDA(cudaMemsetAsync(lum_acc, 0, sizeof(double), st));
    { ProfScope ps_("k_mc_lum", st); k_mc_lum<<<std::min<unsigned>(nblk(M, 256), 1024u), 256, 0, st>>>(M, t->C, NC, Bhat, lum_acc); }
    RGS_LAUNCH("mc floor");
    if (G > 0) {
        RGS_CUDA(cudaMemsetAsync(Bsum, 0, sizeof(double) * G * t->C * NC, st));
        { ProfScope ps_("k_mc_group_sums", st); k_mc_group_sums<NC><<<nblk(M, 256), 256, 0, st>>>(t->n, t->C, t->mc->assign, Bhat, Bsum); }
        RGS_LAUNCH("mc group sums");
    }
    return RGS_OK;
}

McArgs base_args(rgs_transport *t, int G, const float *S, const float *Bhat, const double *lum_acc, const double *Bsum,
                 unsigned long long seed) {
    McArgs A{};
    A.sc = t->sc->dev();
    A.n = t->n;
    A.C = t->C;
    A.pair_off = t->pair_off;
    A.rec = t->mc && t->mc->rec ? t->mc->rec : t->pair_rec; // the caller-ordered copy (none: no pairs)
    A.S = S;
    A.Bhat = Bhat;
    A.lum_acc = lum_acc;
    A.G = G;
    A.assign = G ? t->mc->assign : nullptr;
    A.gc = G ? t->mc->gc : nullptr;
    A.gn = G ? t->mc->gn : nullptr;
    A.Bsum = Bsum;
    A.seed = seed;
    return A;
}

template <int NC>
rgs_status mc_solve_nc(rgs_transport *t, const float *E, const float *S_in, int T, unsigned long long seed, int G,
                       float *B_out, float *visits, cudaStream_t st) {
    rgs_status r;
    const int n = t->n, C = t->C, R = C * NC;
    const size_t M = t->arr();
    if ((r = ensure_groups(t, G, st)) != RGS_OK || (r = ensure_caller_rec(t, st)) != RGS_OK) return r;
    Scratch s{st};
    float *S, *Bhat;
    double *SB, *SB2, *D, *var, *cum, *lum_acc, *Bsum = nullptr;
    int *recv;
    if ((r = s.get(&S, M)) != RGS_OK || (r = s.get(&Bhat, M)) != RGS_OK || (r = s.get(&SB, M)) != RGS_OK ||
        (r = s.get(&SB2, M)) != RGS_OK || (r = s.get(&D, (size_t)n)) != RGS_OK || (r = s.get(&var, (size_t)n)) != RGS_OK ||
        (r = s.get(&cum, (size_t)n)) != RGS_OK || (r = s.get(&recv, (size_t)n)) != RGS_OK ||
        (r = s.get(&lum_acc, 1)) != RGS_OK || (G && (r = s.get(&Bsum, (size_t)G * R)) != RGS_OK))
        return r;
    if (S_in) {
        ProfScope ps_("k_mc_from_user", st);
        k_mc_from_user<NC><<<nblk(M, 256), 256, 0, st>>>(n, C, t->sc->uid, S_in, S);
    } else {
        ProfScope ps_("k_mc_make_S", st);
        k_mc_make_S<NC><<<nblk(M, 256), 256, 0, st>>>(n, C, t->sc->uid, E, t->D, S);
    }
    RGS_LAUNCH("mc source");
    RGS_CUDA(cudaMemsetAsync(Bhat, 0, sizeof(float) * M, st));
    RGS_CUDA(cudaMemsetAsync(SB, 0, sizeof(double) * M, st));
    RGS_CUDA(cudaMemsetAsync(SB2, 0, sizeof(double) * M, st));
    RGS_CUDA(cudaMemsetAsync(D, 0, sizeof(double) * n, st));
    McArgs A = base_args(t, G, S, Bhat, lum_acc, Bsum, seed);
    A.n_draws = n;
    A.SB = SB;
    A.SB2 = SB2;
    A.D = D;
    for (int step = 1; step <= T; ++step) {
        if (step > 8) {
            { ProfScope ps_("k_mc_var", st); k_mc_var<<<nblk(n, 128), 128, 0, st>>>(n, R, t->sc->inv, SB, SB2, D, var); }
            RGS_LAUNCH("mc variance");
            { ProfScope ps_("k_mc_scan", st); k_mc_scan<<<1, MT, 0, st>>>(n, var, cum); }
            RGS_LAUNCH("mc variance scan");
            { ProfScope ps_("k_mc_select", st); k_mc_select<<<nblk(n, 128), 128, 0, st>>>(n, cum, seed, step, recv); }
            RGS_LAUNCH("mc receivers");
        }
        if ((r = step_inputs<NC>(t, Bhat, lum_acc, Bsum, G, st)) != RGS_OK) return r;
        A.t = step;
        A.recv = step > 8 ? recv : nullptr;
        { ProfScope ps_("k_mc_draw", st); k_mc_draw<NC><<<n, MT, 0, st>>>(A); }
        RGS_LAUNCH("mc draws");
        { ProfScope ps_("k_mc_mean", st); k_mc_mean<<<nblk(M, 256), 256, 0, st>>>(M, R, SB, D, Bhat); }
        RGS_LAUNCH("mc means");
    }
    { ProfScope ps_("k_mc_to_user", st); k_mc_to_user<NC><<<nblk(M, 256), 256, 0, st>>>(n, C, t->sc->uid, Bhat, B_out); }
    RGS_LAUNCH("mc output");
    if (visits) {
        { ProfScope ps_("k_mc_visits", st); k_mc_visits<<<nblk(n, 128), 128, 0, st>>>(n, t->sc->uid, D, visits); }
        RGS_LAUNCH("mc visits");
    }
    return RGS_OK;
}

template <int NC>
rgs_status mc_estimate_nc(rgs_transport *t, const float *E, const float *Bhat_user, unsigned long long seed, int step,
                          int G, int n_draws, const int *recv, long long *pick, double *p, float *delta,
                          cudaStream_t st) {
    rgs_status r;
    const int n = t->n, C = t->C, R = C * NC;
    const size_t M = t->arr();
    if ((r = ensure_groups(t, G, st)) != RGS_OK || (r = ensure_caller_rec(t, st)) != RGS_OK) return r;
    Scratch s{st};
    float *S, *Bhat;
    double *lum_acc, *Bsum = nullptr;
    int *bad;
    if ((r = s.get(&S, M)) != RGS_OK || (r = s.get(&Bhat, M)) != RGS_OK || (r = s.get(&lum_acc, 1)) != RGS_OK ||
        (r = s.get(&bad, 1)) != RGS_OK || (G && (r = s.get(&Bsum, (size_t)G * R)) != RGS_OK))
        return r;
    RGS_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
    { ProfScope ps_("k_mc_make_S", st); k_mc_make_S<NC><<<nblk(M, 256), 256, 0, st>>>(n, C, t->sc->uid, E, t->D, S); }
    RGS_LAUNCH("mc source");
    { ProfScope ps_("k_mc_from_user", st); k_mc_from_user<NC><<<nblk(M, 256), 256, 0, st>>>(n, C, t->sc->uid, Bhat_user, Bhat); }
    RGS_LAUNCH("mc means");
    if ((r = step_inputs<NC>(t, Bhat, lum_acc, Bsum, G, st)) != RGS_OK) return r;
    McArgs A = base_args(t, G, S, Bhat, lum_acc, Bsum, seed);
    A.t = step;
    A.n_draws = n_draws;
    A.recv = recv;
    A.pick_out = pick;
    A.p_out = p;
    A.delta_out = delta;
    A.bad = bad;
    if (n_draws > 0) {
        ProfScope ps_("k_mc_draw", st);
        k_mc_draw<NC><<<n_draws, MT, 0, st>>>(A);
    }
    RGS_LAUNCH("mc draws");
    int nbad = 0;
    RGS_CUDA(cudaMemcpyAsync(&nbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    RGS_CUDA(cudaStreamSynchronize(st));
    if (nbad) {
        rgs_set_error("rgs_mc_estimate: %d draws name a receiver outside [0, N)", nbad);
        return RGS_ERR_ARG;
    }
    return RGS_OK;
}

template <int NC>
rgs_status prog_refine_nc(rgs_transport *t, const float *E, int shots, float *Bhat_out, float *dB_out, cudaStream_t st) {
    rgs_status r;
    const int n = t->n, C = t->C, R = C * NC;
    const size_t M = t->arr();
    const int nparts = (int)nblk(n, PR_T);
    Scratch s{st};
    float *dB, *Bhat, *shot;
    LumIdx *part;
    int *shot_i;
    int2 *tr;
    if ((r = s.get(&dB, M)) != RGS_OK || (r = s.get(&Bhat, M)) != RGS_OK || (r = s.get(&shot, (size_t)R)) != RGS_OK ||
        (r = s.get(&part, (size_t)nparts)) != RGS_OK || (r = s.get(&shot_i, 1)) != RGS_OK ||
        (r = s.get(&tr, (size_t)std::max(t->n_pairs, 1ll))) != RGS_OK)
        return r;
    if ((r = rgs_pairs_transpose(t, tr, st)) != RGS_OK) return r;
    { ProfScope ps_("k_mc_make_S", st); k_mc_make_S<NC><<<nblk(M, 256), 256, 0, st>>>(n, C, t->sc->uid, E, t->D, Bhat); }
    RGS_LAUNCH("shooting source");
    RGS_CUDA(cudaMemcpyAsync(dB, Bhat, sizeof(float) * M, cudaMemcpyDeviceToDevice, st));
    const SceneDev sd = t->sc->dev();
    for (int m = 0; m < shots; ++m) {
        { ProfScope ps_("k_pr_argmax", st); k_pr_argmax<<<nparts, PR_T, 0, st>>>(n, C, NC, t->sc->uid, dB, part); }
        RGS_LAUNCH("shooting argmax");
        { ProfScope ps_("k_pr_pick", st); k_pr_pick<<<1, PR_T, 0, st>>>(nparts, R, t->sc->inv, part, dB, shot, shot_i); }
        RGS_LAUNCH("shooting pick");
        { ProfScope ps_("k_pr_scatter", st); k_pr_scatter<NC><<<256, PR_T, 0, st>>>(sd, C, t->src_off, tr, shot_i, shot, dB, Bhat); }
        RGS_LAUNCH("shooting scatter");
    }
    { ProfScope ps_("k_mc_to_user", st); k_mc_to_user<NC><<<nblk(M, 256), 256, 0, st>>>(n, C, t->sc->uid, Bhat, Bhat_out); }
    { ProfScope ps_("k_mc_to_user", st); k_mc_to_user<NC><<<nblk(M, 256), 256, 0, st>>>(n, C, t->sc->uid, dB, dB_out); }
    RGS_LAUNCH("shooting output");
    return RGS_OK;
}

} // namespace

void rgs_mc_free(rgs_transport *t) {
    if (!t || !t->mc) return;
    dev_free(t->mc->assign);
    dev_free(t->mc->gc);
    dev_free(t->mc->gn);
    dev_free(t->mc->rec);
    t->device_bytes -= t->mc->bytes + t->mc->rec_bytes;
    delete t->mc;
    t->mc = nullptr;
}

extern "C" rgs_status rgs_mc_solve(rgs_transport *t, const float *E, const float *S_in, int32_t steps, uint64_t seed,
                                   int32_t groups, float *B_out, float *visits, void *stream) {
    rgs_status r = check_pairs(t, "rgs_mc_solve");
    if (r != RGS_OK) return r;
    if (!B_out || steps < 0 || groups < 0 || groups > MC_GMAX || groups > t->n) {
        rgs_set_error("rgs_mc_solve: NULL B_out, negative steps or groups outside [0, min(%d, N)]", MC_GMAX);
        return RGS_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    switch (t->nc) {
    case 1: return mc_solve_nc<1>(t, E, S_in, steps, seed, groups, B_out, visits, st);
    case 4: return mc_solve_nc<4>(t, E, S_in, steps, seed, groups, B_out, visits, st);
    case 9: return mc_solve_nc<9>(t, E, S_in, steps, seed, groups, B_out, visits, st);
    default: return mc_solve_nc<16>(t, E, S_in, steps, seed, groups, B_out, visits, st);
    }
}

extern "C" rgs_status rgs_mc_estimate(rgs_transport *t, const float *E, const float *Bhat, uint64_t seed, int32_t step,
                                      int32_t groups, int32_t n_draws, const int32_t *recv, int64_t *pick, double *p,
                                      float *delta, void *stream) {
    rgs_status r = check_pairs(t, "rgs_mc_estimate");
    if (r != RGS_OK) return r;
    if (!Bhat || !pick || !p || !delta || step < 1 || n_draws < 0 || (!recv && n_draws > t->n) || groups < 0 ||
        groups > MC_GMAX || groups > t->n) {
        rgs_set_error("rgs_mc_estimate: NULL output, step < 1, n_draws outside [0, N] without receivers, or groups "
                      "outside [0, min(%d, N)]",
                      MC_GMAX);
        return RGS_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    long long *pk = reinterpret_cast<long long *>(pick);
    switch (t->nc) {
    case 1: return mc_estimate_nc<1>(t, E, Bhat, seed, step, groups, n_draws, recv, pk, p, delta, st);
    case 4: return mc_estimate_nc<4>(t, E, Bhat, seed, step, groups, n_draws, recv, pk, p, delta, st);
    case 9: return mc_estimate_nc<9>(t, E, Bhat, seed, step, groups, n_draws, recv, pk, p, delta, st);
    default: return mc_estimate_nc<16>(t, E, Bhat, seed, step, groups, n_draws, recv, pk, p, delta, st);
    }
}

extern "C" rgs_status rgs_mc_groups(rgs_transport *t, int32_t groups, int32_t *assign, void *stream) {
    rgs_status r = check_pairs(t, "rgs_mc_groups");
    if (r != RGS_OK) return r;
    if (!assign || groups < 1 || groups > MC_GMAX || groups > t->n) {
        rgs_set_error("rgs_mc_groups: NULL assign or groups outside [1, min(%d, N)]", MC_GMAX);
        return RGS_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if ((r = ensure_groups(t, groups, st)) != RGS_OK) return r;
    { ProfScope ps_("k_km_to_user", st); k_km_to_user<<<nblk(t->n, 128), 128, 0, st>>>(t->n, t->sc->uid, t->mc->assign, assign); }
    RGS_LAUNCH("k-means output");
    return RGS_OK;
}

extern "C" rgs_status rgs_prog_refine(rgs_transport *t, const float *E, int32_t shots, float *Bhat_out, float *dB_out,
                                      void *stream) {
    rgs_status r = check_pairs(t, "rgs_prog_refine");
    if (r != RGS_OK) return r;
    if (!Bhat_out || !dB_out || shots < 0) {
        rgs_set_error("rgs_prog_refine: NULL output or negative shot count");
        return RGS_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    switch (t->nc) {
    case 1: return prog_refine_nc<1>(t, E, shots, Bhat_out, dB_out, st);
    case 4: return prog_refine_nc<4>(t, E, shots, Bhat_out, dB_out, st);
    case 9: return prog_refine_nc<9>(t, E, shots, Bhat_out, dB_out, st);
    default: return prog_refine_nc<16>(t, E, shots, Bhat_out, dB_out, st);
    }
}
