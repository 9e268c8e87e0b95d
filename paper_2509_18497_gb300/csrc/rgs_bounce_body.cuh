// Bounce gather/projection for one receiver and one column tile (the body of k_bounce and
// of the persistent batch kernel): CTA-wide, BOUNCE_THREADS threads, red = shared scratch of
// (BOUNCE_THREADS/32) * G * KPL * CT floats.
#pragma once
#include "rgs_internal.cuh"

#define BOUNCE_THREADS 256

// many-column (lane-per-column) layout: a warp takes one ray at a time and its 32 lanes take
// 32 consecutive columns of one tile
constexpr int MC_WARPS = 8;
constexpr int MC_THREADS = MC_WARPS * 32;
static_assert(MC_THREADS == BOUNCE_THREADS, "the batch kernel runs both bodies in one block");
static_assert(BOUNCE_THREADS == 256, "RGS_BOUNCE_LB and RGS_MC_LB assume 256 threads");

// the NC coefficients of one column of a row (FP32 rows of NC floats, BF16 rows padded)
template <int NC> __device__ __forceinline__ void load_col(const float *__restrict__ p, float *v) {
    if constexpr (NC % 4 == 0) {
#pragma unroll
        for (int q = 0; q < NC / 4; ++q) {
            const float4 f = __ldg(reinterpret_cast<const float4 *>(p) + q);
            v[4 * q] = f.x;
            v[4 * q + 1] = f.y;
            v[4 * q + 2] = f.z;
            v[4 * q + 3] = f.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < NC; ++k) v[k] = __ldg(p + k);
    }
}
template <int NC> __device__ __forceinline__ void load_col(const __nv_bfloat16 *__restrict__ p, float *v) {
    if constexpr (NC >= 9) { // padded to 16
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const uint4 w = __ldg(reinterpret_cast<const uint4 *>(p) + q);
            const unsigned u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int k0 = 8 * q + 2 * m;
                if (k0 < NC) v[k0] = __uint_as_float(u[m] << 16);
                if (k0 + 1 < NC) v[k0 + 1] = __uint_as_float(u[m] & 0xffff0000u);
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < NC; ++k) v[k] = __bfloat162float(p[k]);
    }
}
template <int NC, class T> constexpr int row_stride() {
    return sizeof(T) == 2 ? ((NC >= 9) ? 16 : NC) : NC;
}

// Dot products of Y with the 32 columns of one FP32 source row tile (nc = 16: 64 B per
// column, 2 KB per tile), read as four contiguous 512-B warp requests, a lane taking 16 B
// (a quarter of one column).  Each lane forms its partial dot products with its quarter of
// Y, and a reduce-scatter over the 4 lanes holding each column leaves lane l with the
// whole dot product of tile column own(l).  A 64-B column row per lane at a 64-B stride
// costs the L1 about twice the wavefronts for the same bytes (measured: the FP32 form of
// the 300- and 1,536-column workloads 6 % and 25 % faster).  For BF16 rows (32 B per
// column) the same scheme measured 3-7 % slower than a row per lane and is not used.
// Columns past the tile's `ncols` live ones read the last live column (their results are
// not used).  All 32 lanes take part (the shuffles use the full mask).
template <class T, int NC> struct TileDot;

template <int NC> struct TileDot<float, NC> {
    static_assert(NC == 16, "FP32 tiles of 16 coefficients per column");
    static constexpr int KPL = 4;
    __device__ static int own(int lane) {
        const int g = lane & 3;
        return 8 * (2 * (g & 1) + (g >> 1)) + (lane >> 2);
    }
    __device__ static void pick(const float *Y, int lane, float (&y)[KPL]) {
        const int g = lane & 3;
#pragma unroll
        for (int m = 0; m < KPL; ++m) {
            float v = Y[m];
            v = g == 1 ? Y[4 + m] : v;
            v = g == 2 ? Y[8 + m] : v;
            v = g == 3 ? Y[12 + m] : v;
            y[m] = v;
        }
    }
    // tile: the tile's first column in source row j; ncols: its live columns (1..32)
    __device__ static float dot(const float *__restrict__ tile, int ncols, int lane, const float (&y)[KPL]) {
        const int g = lane & 3, a = lane >> 2;
        float p[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = min(8 * q + a, ncols - 1);
            const float4 f = __ldg(reinterpret_cast<const float4 *>(tile + c * 16) + g);
            p[q] = y[0] * f.x + y[1] * f.y + y[2] * f.z + y[3] * f.w;
        }
        const bool b0 = (g & 1) != 0, b1 = (g & 2) != 0;
        const float r0 = __shfl_xor_sync(0xffffffffu, b0 ? p[0] : p[2], 1);
        const float r1 = __shfl_xor_sync(0xffffffffu, b0 ? p[1] : p[3], 1);
        const float s0 = (b0 ? p[2] : p[0]) + r0, s1 = (b0 ? p[3] : p[1]) + r1;
        const float r = __shfl_xor_sync(0xffffffffu, b1 ? s0 : s1, 2);
        return (b1 ? s1 : s0) + r;
    }
};


template <int NC, int CT, class SL>
__device__ __forceinline__ void bounce_epilogue(const SceneDev &sc, int C, const float (&acc)[SL::KPL][CT], float w,
                                                const float *__restrict__ Bprev, const float *__restrict__ S,
                                                float *__restrict__ Qout, float *__restrict__ Bout,
                                                __nv_bfloat16 *__restrict__ Bout16, double *norm2, int i, int col0,
                                                float *red);

template <int NC, int CT, class SL>
__device__ __forceinline__ void bounce_receiver(const SceneDev &sc, const RaysDev &rays, int C,
                                                const typename SL::T *__restrict__ Bg, const float *__restrict__ Bprev,
                                                const float *__restrict__ S, float *__restrict__ Qout,
                                                float *__restrict__ Bout, __nv_bfloat16 *__restrict__ Bout16,
                                                double *norm2, int i, int col0, float *red) {

    constexpr int G = SL::G, KPL = SL::KPL, GROUPS = BOUNCE_THREADS / G, RS = SL::STRIDE;
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
    bounce_epilogue<NC, CT, SL>(sc, C, acc, 3.14159265358979f / (float)nd, Bprev, S, Qout, Bout, Bout16, norm2, i, col0,
                                red);
}

// Reduction of the per-thread projections acc over the CTA and the bounce update of one
// (receiver, column tile): Q = w * sum, B = S + o_i c_i (x) Q, its BF16 copy, and the FP64
// partial of ||B - Bprev||^2.  Ends with __syncthreads (red is reused).
template <int NC, int CT, class SL>
__device__ __forceinline__ void bounce_epilogue(const SceneDev &sc, int C, const float (&acc)[SL::KPL][CT], float w,
                                                const float *__restrict__ Bprev, const float *__restrict__ S,
                                                float *__restrict__ Qout, float *__restrict__ Bout,
                                                __nv_bfloat16 *__restrict__ Bout16, double *norm2, int i, int col0,
                                                float *red) {
    constexpr int G = SL::G, KPL = SL::KPL;
    // reduce over the groups: lanes with equal g within the warp, then across warps
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int m = 0; m < KPL; ++m)
#pragma unroll
        for (int c = 0; c < CT; ++c) {
            float v = acc[m][c];
#pragma unroll
            for (int off = G; off < 32; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane < G) red[(warp * G + lane) * (KPL * CT) + m * CT + c] = v;
        }
    __syncthreads();
    double dsq = 0.0;
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
        for (int q = 0; q < BOUNCE_THREADS / 32; ++q) v += red[(q * G + gg) * (KPL * CT) + mm * CT + c];
        const int col = col0 + c;
        const float Q = w * v;
        const size_t idx = ((size_t)i * C + col) * NC + k;
        Qout[idx] = Q;
        const float oc = alpha_center(sc, i) * sc.cl[(size_t)i * 12 + band_of(k) * 3 + (col % 3)];
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
    __syncthreads(); // red is reused by the caller's next receiver
}

// Lane-per-column bounce for one receiver and one 32-column tile (the body of k_bounce_mc and
// of the persistent batch kernel's wide items); red = shared scratch of MC_WARPS * NC * 32 floats.
template <int NC, class T>
__device__ __forceinline__ void bounce_receiver_mc(const SceneDev &sc, const RaysDev &rays, int C,
                                                   const T *__restrict__ Bg, const float *__restrict__ Bprev,
                                                   const float *__restrict__ S, float *__restrict__ Qout,
                                                   float *__restrict__ Bout, __nv_bfloat16 *__restrict__ Bout16,
                                                   double *norm2, int i, int tile, float *red) {
    constexpr int RS = row_stride<NC, T>();
    constexpr bool COOP = sizeof(T) == 4 && NC == 16; // whole-tile reads (TileDot)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int own = lane; // the tile column whose sums this lane keeps
    if constexpr (COOP) own = TileDot<T, NC>::own(lane);
    const int col = tile * 32 + own;
    const bool live = col < C;
    const int colc = live ? col : C - 1;
    const int ncols = min(32, C - tile * 32);
    const int nd = rays.nd;
    const float3 n = f3(sc.N4[i]);
    float acc[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) acc[k] = 0.f;
    for (int q = warp; q < nd; q += MC_WARPS) {
        const long long r = (long long)i * nd + q;
        const float3 d = f3(rays.dir[r]);
        float Yo[NC];
        sh_eval<NC>(neg3(d), Yo);
        const int cnt = rays.cnt[r];
        const long long base = rays.off[r];
        float x = 0.f;
        if constexpr (COOP) {
            float ys[TileDot<T, NC>::KPL];
            TileDot<T, NC>::pick(Yo, lane, ys);
#pragma unroll 2
            for (int h = 0; h < cnt; ++h) {
                const int2 ja = __ldg(&rays.rec_ja[base + h]);
                x += __int_as_float(ja.y) * TileDot<T, NC>::dot(Bg + ((size_t)ja.x * C + tile * 32) * RS, ncols, lane, ys);
            }
        } else {
#pragma unroll 2
            for (int h = 0; h < cnt; ++h) {
                const int2 ja = __ldg(&rays.rec_ja[base + h]);
                float v[NC];
                load_col<NC>(Bg + ((size_t)ja.x * C + colc) * RS, v);
                float s = 0.f;
#pragma unroll
                for (int k = 0; k < NC; ++k) s += Yo[k] * v[k];
                x += __int_as_float(ja.y) * s;
            }
        }
        float Yi[NC];
        sh_eval<NC>(reflect_n(n, d), Yi);
#pragma unroll
        for (int k = 0; k < NC; ++k) acc[k] += Yi[k] * x;
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) red[(warp * NC + k) * 32 + own] = acc[k];
    __syncthreads();
    double dsq = 0.0;
    const float w = 3.14159265358979f / (float)nd;
    for (int e = threadIdx.x; e < NC * 32; e += MC_THREADS) {
        const int k = e >> 5, c = e & 31;
        const int cc = tile * 32 + c;
        if (cc >= C) continue;
        float v = 0.f;
#pragma unroll
        for (int q = 0; q < MC_WARPS; ++q) v += red[(q * NC + k) * 32 + c];
        const float Q = w * v;
        const size_t idx = ((size_t)i * C + cc) * NC + k;
        Qout[idx] = Q;
        const float b = S[idx] + alpha_center(sc, i) * sc.cl[(size_t)i * 12 + band_of(k) * 3 + (cc % 3)] * Q;
        Bout[idx] = b;
        if (Bout16) Bout16[((size_t)i * C + cc) * ((NC >= 9) ? 16 : NC) + k] = __float2bfloat16_rn(b);
        const double df = (double)b - (double)Bprev[idx];
        dsq += df * df;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) dsq += __shfl_xor_sync(0xffffffffu, dsq, off);
    if (lane == 0) atomicAdd(norm2, dsq);
    __syncthreads(); // red is reused by the caller's next receiver
}
