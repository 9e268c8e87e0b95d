// Internal definitions shared by the CUDA translation units of librgs (not part of the ABI).
//
// Data layout in HBM (all arrays in the library's internal Morton order of the surfels):
//   P[j]  = (p.xyz, o)          N4[j] = (n.xyz, 0)
//   FU[j] = (t^u.xyz, 1/s^u)    FV[j] = (t^v.xyz, 1/s^v)        64 B read per intersection test
//   cl[j] = c_{j,l,ch} as [4][3] floats (bands beyond L are zero)
//   uid[j] = caller index of internal surfel j (ray seeds and depth-tie order use it)
//   radiosity-like arrays (S, B^(b), Q^(b), v^(a), u): [N][C][NC] float, SH index innermost
//   hit records: contiguous per ray, hit h of ray r at off[r] + h (exactly sized, in depth
//                order): rec_ja = (source j, bits of a_rh); G is recomputed where needed
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rgs.h" // include/ is on the include path (build.py)

#define RGS_HMAX 96           // per-ray hit buffer; when full the nearest RGS_HMAX hits are kept
#define RGS_T_EPS 1e-6f       // compositing stops once the transmittance is below this
#define RGS_STACK 64          // BVH traversal stack depth (tree depth is bounded by 32 + log2 N)

// Launch bounds of the gather kernels: with RGS_<KERNEL>_MINB defined, the register budget
// is sized for that many resident blocks per SM (these latency-bound kernels gain from more
// resident warps as long as nothing spills); undefined, the compiler's default budget.
// Build-time knobs, set from measurements on GB300 (50,000-surfel bowl, 1 and 16 lights):
// 5 blocks for the 3-column bounce (-9 %, despite a few spilled registers) and 4 for the
// lane-per-column bounce (-18 %); the opacity and adjoint gathers keep the default (tighter
// budgets measured slower).
#define RGS_LB_(threads, minb) __launch_bounds__(threads, minb)
#ifndef RGS_BOUNCE_MINB
#define RGS_BOUNCE_MINB 5
#endif
#ifndef RGS_MCB_MINB
#define RGS_MCB_MINB 4
#endif
#define RGS_MCB_LB RGS_LB_(256, RGS_MCB_MINB)
#ifdef RGS_BOUNCE_MINB
#define RGS_BOUNCE_LB RGS_LB_(256, RGS_BOUNCE_MINB)
#else
#define RGS_BOUNCE_LB __launch_bounds__(256)
#endif
#ifdef RGS_OPA_MINB
#define RGS_OPA_LB RGS_LB_(256, RGS_OPA_MINB)
#else
#define RGS_OPA_LB __launch_bounds__(256)
#endif
#ifdef RGS_OPAREC_MINB
#define RGS_OPAREC_LB RGS_LB_(256, RGS_OPAREC_MINB)
#else
#define RGS_OPAREC_LB __launch_bounds__(256)
#endif
#ifdef RGS_ADJ_MINB
#define RGS_ADJ_LB RGS_LB_(128, RGS_ADJ_MINB)
#else
#define RGS_ADJ_LB __launch_bounds__(128)
#endif
#ifdef RGS_MC_MINB
#define RGS_MC_LB RGS_LB_(256, RGS_MC_MINB)
#else
#define RGS_MC_LB __launch_bounds__(256)
#endif

// ------------------------------------------------------------------ error flags
enum {
    FLAG_CAPACITY = 0,  // hit-record slots exhausted (warps that could not store)
    FLAG_FULL_RAYS = 1, // rays whose full RGS_HMAX buffer ended above the transmittance cut
    FLAG_STACK = 2,     // traversal stack overflow (the ray then misses the rest of the tree)
    FLAG_NONFINITE = 3,
    FLAG_TC_TIMEOUT = 4, // a bounded wait of the tensor-core contraction ran out (5, 6: where)
    FLAG_COUNT = 8
};

// ------------------------------------------------------------------ BVH node
// Internal node of a binary LBVH; stores both children's boxes. A child index c >= 0
// is an internal node, c < 0 is the leaf (surfel) ~c.
struct __align__(16) BvhNode {
    float4 a; // l.lo.x l.lo.y l.lo.z l.hi.x
    float4 b; // l.hi.y l.hi.z r.lo.x r.lo.y
    float4 c; // r.lo.z r.hi.x r.hi.y r.hi.z
    int4 d;   // left, right, 0, 0
};

struct SceneDev {
    int n, L, alpha_model;
    float cutoff2;
    const float4 *P, *N4, *FU, *FV;
    const float *cl; // [n][4][3]
    const int *uid; // caller index of internal surfel i
    const int *inv; // internal index of caller surfel k
    const BvhNode *nodes;
    const float *eps_plane; // device scalar
};

struct RaysDev {
    int nd, na, nbs; // rays per surfel, strata n_a x n_b
    unsigned long long seed;
    const int2 *rec_ja;
    const long long *off; // first record of each ray
    const int *cnt;
    const float4 *dir; // per-ray direction (xyz), written by the trace
};

// ------------------------------------------------------------------ small math
__device__ __forceinline__ float3 f3(float4 v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 neg3(float3 a) { return make_float3(-a.x, -a.y, -a.z); }

// Light lt seen from o: the unit direction w towards it, its distance r (infinite for a
// directional light, whose lpos is the direction towards it) and the falloff 1/r^2 (1 for a
// directional light: Sec. 5.1 puts such lights far away without the inverse-square falloff)
__device__ __forceinline__ float3 light_dir(const float *__restrict__ lpos, int lt, float3 o, int ldir, float &r,
                                           float &fall) {
    const float3 l = ldir ? make_float3(lpos[3 * lt], lpos[3 * lt + 1], lpos[3 * lt + 2])
                          : make_float3(lpos[3 * lt] - o.x, lpos[3 * lt + 1] - o.y, lpos[3 * lt + 2] - o.z);
    const float len = sqrtf(l.x * l.x + l.y * l.y + l.z * l.z);
    r = ldir ? INFINITY : len;
    fall = ldir ? 1.f : 1.f / (len * len);
    const float inv = 1.f / len;
    return make_float3(l.x * inv, l.y * inv, l.z * inv);
}

// mirror of d about the normal n: R d = 2 (n.d) n - d (places the Phong lobe, Eq. sh-brdf)
__device__ __forceinline__ float3 reflect_n(float3 n, float3 d) {
    float s = 2.f * dot3(n, d);
    return make_float3(s * n.x - d.x, s * n.y - d.y, s * n.z - d.z);
}

// Real orthonormal SH up to degree 3, Condon-Shortley phase, index l*l + l + m,
// as Cartesian polynomials of a unit vector.  Constants are the normalisations
// K = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times sqrt(2) for m != 0, folded with
// the polynomial's integer factors.
template <int NC>
__device__ __forceinline__ void sh_eval(float3 v, float *Y) {
    const float x = v.x, y = v.y, z = v.z;
    Y[0] = 0.28209479177387814f; // 1/(2 sqrt(pi))
    if (NC > 1) {
        const float c1 = 0.4886025119029199f; // sqrt(3/(4 pi))
        Y[1] = -c1 * y;
        Y[2] = c1 * z;
        Y[3] = -c1 * x;
    }
    if (NC > 4) {
        const float c21 = 1.0925484305920792f; // (1/2) sqrt(15/pi)
        const float c20 = 0.31539156525252005f; // (1/4) sqrt(5/pi)
        const float c22 = 0.5462742152960396f; // (1/4) sqrt(15/pi)
        Y[4] = c21 * x * y;
        Y[5] = -c21 * y * z;
        Y[6] = c20 * (3.f * z * z - 1.f);
        Y[7] = -c21 * x * z;
        Y[8] = c22 * (x * x - y * y);
    }
    if (NC > 9) {
        const float c33 = 0.5900435899266435f;  // (1/4) sqrt(35/(2 pi))
        const float c32a = 2.890611442640554f;  // (1/2) sqrt(105/pi)
        const float c31 = 0.4570457994644658f;  // (1/4) sqrt(21/(2 pi))
        const float c30 = 0.3731763325901154f;  // (1/4) sqrt(7/pi)
        const float c32b = 1.445305721320277f;  // (1/4) sqrt(105/pi)
        const float zz5 = 5.f * z * z;
        Y[9] = -c33 * y * (3.f * x * x - y * y);
        Y[10] = c32a * x * y * z;
        Y[11] = -c31 * y * (zz5 - 1.f);
        Y[12] = c30 * z * (zz5 - 3.f);
        Y[13] = -c31 * x * (zz5 - 1.f);
        Y[14] = c32b * z * (x * x - y * y);
        Y[15] = -c33 * x * (x * x - 3.f * y * y);
    }
}

// sum_k coef[k] grad Y_k(v): the gradient of sh_eval's polynomials (their tangential part is
// the derivative along the sphere, the only part the geometry gradients use)
template <int NC>
__device__ __forceinline__ float3 sh_grad_dot(float3 v, const float *coef) {
    const float x = v.x, y = v.y, z = v.z;
    float gx = 0.f, gy = 0.f, gz = 0.f;
    if (NC > 1) {
        const float c1 = 0.4886025119029199f;
        gy -= c1 * coef[1];
        gz += c1 * coef[2];
        gx -= c1 * coef[3];
    }
    if (NC > 4) {
        const float c21 = 1.0925484305920792f, c20 = 0.31539156525252005f, c22 = 0.5462742152960396f;
        gx += c21 * y * coef[4];
        gy += c21 * x * coef[4];
        gy -= c21 * z * coef[5];
        gz -= c21 * y * coef[5];
        gz += 6.f * c20 * z * coef[6];
        gx -= c21 * z * coef[7];
        gz -= c21 * x * coef[7];
        gx += 2.f * c22 * x * coef[8];
        gy -= 2.f * c22 * y * coef[8];
    }
    if (NC > 9) {
        const float c33 = 0.5900435899266435f, c32a = 2.890611442640554f, c31 = 0.4570457994644658f;
        const float c30 = 0.3731763325901154f, c32b = 1.445305721320277f;
        const float zz5 = 5.f * z * z;
        gx -= 6.f * c33 * x * y * coef[9];
        gy -= 3.f * c33 * (x * x - y * y) * coef[9];
        gx += c32a * y * z * coef[10];
        gy += c32a * x * z * coef[10];
        gz += c32a * x * y * coef[10];
        gy -= c31 * (zz5 - 1.f) * coef[11];
        gz -= 10.f * c31 * y * z * coef[11];
        gz += c30 * (3.f * zz5 - 3.f) * coef[12];
        gx -= c31 * (zz5 - 1.f) * coef[13];
        gz -= 10.f * c31 * x * z * coef[13];
        gx += 2.f * c32b * x * z * coef[14];
        gy -= 2.f * c32b * y * z * coef[14];
        gz += c32b * (x * x - y * y) * coef[14];
        gx -= 3.f * c33 * (x * x - y * y) * coef[15];
        gy += 6.f * c33 * x * y * coef[15];
    }
    return make_float3(gx, gy, gz);
}

__host__ __device__ constexpr int band_of(int k) { return k == 0 ? 0 : (k < 4 ? 1 : (k < 9 ? 2 : 3)); }

// Cooperative row slices for the gathers: G lanes share one ray (or one transposed entry)
// and lane g owns the KPL contiguous coefficients k = KPL*g + m of every row.  nc = 16, 9:
// 4 lanes x 4 coefficients (the 4 lanes read one contiguous row per load); nc <= 4: one
// lane per ray, the whole row.  Slice reads FP32 rows (float4 where aligned), SliceH reads
// BF16 copies whose rows are padded to 16 (nc >= 9) so every lane loads 8 aligned bytes.
template <int NC> struct Slice {
    using T = float;
    static constexpr int G = (NC >= 9) ? 4 : 1;
    static constexpr int KPL = (NC >= 9) ? 4 : NC;
    static constexpr int STRIDE = NC; // floats per row
    __device__ static constexpr int k(int g, int m) { return KPL * g + m; }
    // this lane's KPL entries of the row `row` (zero where k >= NC)
    __device__ static void load(const float *__restrict__ row, int g, float *v) {
        if constexpr (NC % 4 == 0) {
            const float4 q4 = __ldg(reinterpret_cast<const float4 *>(row) + g);
            v[0] = q4.x;
            v[1] = q4.y;
            v[2] = q4.z;
            v[3] = q4.w;
        } else {
#pragma unroll
            for (int m = 0; m < KPL; ++m) {
                const int kk = k(g, m);
                v[m] = (kk < NC) ? __ldg(row + kk) : 0.f;
            }
        }
    }
    // select this lane's entries of a full NC-vector held in registers (no dynamic indexing)
    __device__ static void pick(const float *full, int g, float *v) {
#pragma unroll
        for (int m = 0; m < KPL; ++m) {
            float x = 0.f;
#pragma unroll
            for (int kk = 0; kk < NC; ++kk)
                if (kk == k(g, m)) x = full[kk];
            v[m] = x;
        }
    }
    // sum over the G lanes of a group (lanes g = 0..G-1 are consecutive)
    __device__ static float group_sum(float x) {
#pragma unroll
        for (int off = 1; off < G; off <<= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        return x;
    }
};

template <int NC> struct SliceH {
    using T = __nv_bfloat16;
    static constexpr int G = Slice<NC>::G;
    static constexpr int KPL = Slice<NC>::KPL;
    static constexpr int STRIDE = (NC >= 9) ? 16 : NC; // bf16 per row
    __device__ static constexpr int k(int g, int m) { return KPL * g + m; }
    __device__ static void load(const __nv_bfloat16 *__restrict__ row, int g, float *v) {
        if constexpr (KPL == 4) {
            const uint2 q = __ldg(reinterpret_cast<const uint2 *>(row) + g);
            v[0] = __uint_as_float(q.x << 16);
            v[1] = __uint_as_float(q.x & 0xffff0000u);
            v[2] = __uint_as_float(q.y << 16);
            v[3] = __uint_as_float(q.y & 0xffff0000u);
        } else {
#pragma unroll
            for (int m = 0; m < KPL; ++m) v[m] = __bfloat162float(row[k(g, m)]);
        }
    }
    __device__ static void pick(const float *full, int g, float *v) { Slice<NC>::pick(full, g, v); }
    __device__ static float group_sum(float x) { return Slice<NC>::group_sum(x); }
};

template <int NC> constexpr int bf16_stride() { return (NC >= 9) ? 16 : NC; }

// ------------------------------------------------------------------ ray generation
// SplitMix64 output function (Steele, Lea & Flood 2014) applied to a counter.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
// 24-bit uniform in [0,1); key = ((seed*2^32 + i)*2^12 + r)*2 + dim (exact in float)
__device__ __forceinline__ float jitter(unsigned long long seed, unsigned i, unsigned r, unsigned dim) {
    unsigned long long key = ((((seed << 32) + (unsigned long long)i) << 12) + (unsigned long long)r) * 2ull + dim;
    return (float)(unsigned)(splitmix64(key) >> 40) * (1.0f / 16777216.0f);
}

// Ray q of a surfel with caller index uid and frame (tu, tv, n): stratified cosine-weighted
// direction on the front hemisphere (App. B, Omega = {w_I . n < 0}); weight pi/nd.
__device__ __forceinline__ float3 ray_dir(unsigned long long seed, int uid, int q, int na, int nbs, float3 tu, float3 tv,
                                          float3 n) {
    int a = q / nbs, b = q - a * nbs;
    float u1 = ((float)a + jitter(seed, (unsigned)uid, (unsigned)q, 0u)) / (float)na;
    float u2 = ((float)b + jitter(seed, (unsigned)uid, (unsigned)q, 1u)) / (float)nbs;
    float rr = sqrtf(u1), cz = sqrtf(fmaxf(0.f, 1.f - u1));
    float sn, cs;
    sincospif(2.f * u2, &sn, &cs);
    return (rr * cs) * tu + (rr * sn) * tv + cz * n;
}

// ------------------------------------------------------------------ intersection
// Squared local radius u^2 + v^2 of the point o + t d on the plane of surfel j (Eq. G),
// with explicitly rounded operations so that every call site computes identical bits
// (the trace recomputes it after sorting instead of storing it).
__device__ __forceinline__ float surfel_r2(const SceneDev &sc, int j, float3 o, float3 d, float t) {
    const float4 Pj = __ldg(&sc.P[j]);
    const float wx = __fsub_rn(Pj.x, o.x), wy = __fsub_rn(Pj.y, o.y), wz = __fsub_rn(Pj.z, o.z);
    const float qx = __fmaf_rn(t, d.x, -wx), qy = __fmaf_rn(t, d.y, -wy), qz = __fmaf_rn(t, d.z, -wz); // x - p_j
    const float4 U = __ldg(&sc.FU[j]);
    const float4 V = __ldg(&sc.FV[j]);
    const float u = __fmul_rn(__fmaf_rn(qz, U.z, __fmaf_rn(qy, U.y, __fmul_rn(qx, U.x))), U.w);
    const float v = __fmul_rn(__fmaf_rn(qz, V.z, __fmaf_rn(qy, V.y, __fmul_rn(qx, V.x))), V.w);
    return __fmaf_rn(v, v, __fmul_rn(u, u));
}

__device__ __forceinline__ float surfel_G(const SceneDev &sc, float r2) {
    return (sc.alpha_model == RGS_ALPHA_DISC) ? 1.f : expf(-0.5f * r2);
}

// Opacity of a hit with Gaussian value G on a surfel of opacity parameter o, and its
// derivative in o: o G for the Gaussian and disc models; App. E's GFSGS form
// 1 - exp(-0.03279 (o G)^3.4) otherwise (o is then the unbounded parameter g).
__device__ __forceinline__ float alpha_of(const SceneDev &sc, float o, float G) {
    if (sc.alpha_model == RGS_ALPHA_GFSGS) {
        const float x = o * G;
        return x > 0.f ? -expm1f(-0.03279f * powf(x, 3.4f)) : 0.f;
    }
    return o * G;
}
// d alpha / d q of a hit at squared local radius q = u^2 + v^2 (G = exp(-q/2)): -o G / 2
// for the Gaussian, 0 inside the disc, -1.7 p e^{-p} for GFSGS with p = 0.03279 (o G)^3.4
__device__ __forceinline__ float dalpha_dq(const SceneDev &sc, float o, float G) {
    if (sc.alpha_model == RGS_ALPHA_DISC) return 0.f;
    if (sc.alpha_model == RGS_ALPHA_GFSGS) {
        const float x = o * G;
        if (!(x > 0.f)) return 0.f;
        const float p = 0.03279f * powf(x, 3.4f);
        return -1.7f * p * expf(-p);
    }
    return -0.5f * o * G;
}
// Crossing of the segment o + t d (t given) with the plane of surfel k: P_k^T grad_x q with
// P_k = I - d n_k^T / (n_k.d) (the projector onto plane k along d), and u, v; a move of o,
// d or p_k changes q by pw . (do + t dd - dp_k) and s^u_k by dq = -2 u^2 / s^u_k.
__device__ __forceinline__ float3 crossing_pw(const SceneDev &sc, int k, float3 o, float3 d, float t, float &u,
                                              float &v) {
    const float4 Pk = __ldg(&sc.P[k]), Nk = __ldg(&sc.N4[k]), U = __ldg(&sc.FU[k]), V = __ldg(&sc.FV[k]);
    const float3 q = make_float3(o.x + t * d.x - Pk.x, o.y + t * d.y - Pk.y, o.z + t * d.z - Pk.z);
    u = (q.x * U.x + q.y * U.y + q.z * U.z) * U.w;
    v = (q.x * V.x + q.y * V.y + q.z * V.z) * V.w;
    const float a = 2.f * u * U.w, b = 2.f * v * V.w;
    float3 g = make_float3(a * U.x + b * V.x, a * U.y + b * V.y, a * U.z + b * V.z);
    const float s = (d.x * g.x + d.y * g.y + d.z * g.z) / (Nk.x * d.x + Nk.y * d.y + Nk.z * d.z);
    g.x -= Nk.x * s;
    g.y -= Nk.y * s;
    g.z -= Nk.z * s;
    return g;
}
// Geometry-gradient accumulators (scratch of the geometry adjoints, in internal order): dp
// [n][GEO_DP] (x, y, z, unused), ds [n][2] and gF [n][GEO_GF] (dL/dt^u at GEO_TU, dL/dt^v at
// GEO_TV, dL/dn at GEO_N, three floats each), so that each 3-vector is one 16-byte (and each
// scale pair one 8-byte) vector atomic.
constexpr int GEO_DP = 4, GEO_GF = 12, GEO_TU = 0, GEO_TV = 4, GEO_N = 8;
__device__ __forceinline__ void geo_add3(float *base, float3 v) {
    atomicAdd(reinterpret_cast<float4 *>(base), make_float4(v.x, v.y, v.z, 0.f));
}
__device__ __forceinline__ void geo_add2(float *base, float x, float y) {
    atomicAdd(reinterpret_cast<float2 *>(base), make_float2(x, y));
}
// Frame gradients of an occluder k crossed at o + t d (u, v from crossing_pw), scaled by
// coef = dL/dq, added to gF[k] = (dL/dt^u, dL/dt^v, dL/dn): q = u^2 + v^2 with
// u = (x - p_k).t^u_k / s^u_k moves with t^u_k by 2 u (x - p_k) / s^u_k, and with n_k through
// t = n_k.(p_k - o)/(n_k.d) by -(grad_x q . d)/(n_k.d) (x - p_k).
__device__ __forceinline__ void occluder_frame_grad(const SceneDev &sc, int k, float3 o, float3 d, float t, float u,
                                                    float v, float coef, float *gF) {
    const float4 Pk = __ldg(&sc.P[k]), Nk = __ldg(&sc.N4[k]), U = __ldg(&sc.FU[k]), V = __ldg(&sc.FV[k]);
    const float3 xm = make_float3(o.x + t * d.x - Pk.x, o.y + t * d.y - Pk.y, o.z + t * d.z - Pk.z);
    const float a = 2.f * u * U.w, b = 2.f * v * V.w;
    const float gxd = a * (U.x * d.x + U.y * d.y + U.z * d.z) + b * (V.x * d.x + V.y * d.y + V.z * d.z);
    const float fn = -gxd / (Nk.x * d.x + Nk.y * d.y + Nk.z * d.z);
    float *g = gF + GEO_GF * (size_t)k;
    geo_add3(g + GEO_TU, (coef * a) * xm);
    geo_add3(g + GEO_TV, (coef * b) * xm);
    geo_add3(g + GEO_N, (coef * fn) * xm);
}
// dL/dn of a term gR . Y(R w) with R w = 2 (n.w) n - w: 2 ((n.gR) w + (n.w) gR)
__device__ __forceinline__ float3 reflect_grad_n(float3 n, float3 w, float3 gR) {
    const float ng = dot3(n, gR), nw = dot3(n, w);
    return make_float3(2.f * (ng * w.x + nw * gR.x), 2.f * (ng * w.y + nw * gR.y), 2.f * (ng * w.z + nw * gR.z));
}
__device__ __forceinline__ float dalpha_do(const SceneDev &sc, float o, float G) {
    if (sc.alpha_model == RGS_ALPHA_GFSGS) {
        const float x = o * G;
        if (!(x > 0.f)) return 0.f;
        const float p = 0.03279f * powf(x, 3.4f);
        return expf(-p) * 3.4f * p / o;
    }
    return G;
}
// the receiver's own alpha_i(p_i) (kappa_i a Dirac at the centre: G = 1) and its derivative
__device__ __forceinline__ float alpha_center(const SceneDev &sc, int i) { return alpha_of(sc, __ldg(&sc.P[i].w), 1.f); }
__device__ __forceinline__ float dalpha_center(const SceneDev &sc, int i) {
    return dalpha_do(sc, __ldg(&sc.P[i].w), 1.f);
}

// Ray o + t d against the plane of surfel j (Eq. G). Returns true with t and r2 when the
// hit is accepted: j != self, |n_j.(p_j - o)| > eps, 0 < t < tmax, inside the cutoff.
__device__ __forceinline__ bool hit_surfel_t(const SceneDev &sc, int j, int self, float3 o, float3 d, float tmax,
                                             float eps, float &t_out, float &r2_out) {
    if (j == self) return false;
    const float4 Nj = __ldg(&sc.N4[j]);
    const float den = __fmaf_rn(Nj.z, d.z, __fmaf_rn(Nj.y, d.y, __fmul_rn(Nj.x, d.x)));
    if (fabsf(den) < 1e-12f) return false;
    const float4 Pj = __ldg(&sc.P[j]);
    const float h = __fmaf_rn(Nj.z, __fsub_rn(Pj.z, o.z),
                              __fmaf_rn(Nj.y, __fsub_rn(Pj.y, o.y), __fmul_rn(Nj.x, __fsub_rn(Pj.x, o.x))));
    if (fabsf(h) <= eps) return false;
    const float t = __fdiv_rn(h, den);
    if (!(t > 0.f) || !(t < tmax)) return false;
    const float r2 = surfel_r2(sc, j, o, d, t);
    if (r2 > sc.cutoff2) return false;
    t_out = t;
    r2_out = r2;
    return true;
}

// G of a hit that the trace stored (ray o + t d on surfel j), recomputed with the same
// rounding as hit_surfel_t, so it equals the value the compositing used bit for bit.
__device__ __forceinline__ float stored_hit_G(const SceneDev &sc, int j, float3 o, float3 d) {
    const float4 Nj = __ldg(&sc.N4[j]);
    const float den = __fmaf_rn(Nj.z, d.z, __fmaf_rn(Nj.y, d.y, __fmul_rn(Nj.x, d.x)));
    const float4 Pj = __ldg(&sc.P[j]);
    const float h = __fmaf_rn(Nj.z, __fsub_rn(Pj.z, o.z),
                              __fmaf_rn(Nj.y, __fsub_rn(Pj.y, o.y), __fmul_rn(Nj.x, __fsub_rn(Pj.x, o.x))));
    return surfel_G(sc, surfel_r2(sc, j, o, d, __fdiv_rn(h, den)));
}

__device__ __forceinline__ bool hit_surfel(const SceneDev &sc, int j, int self, float3 o, float3 d, float tmax,
                                           float eps, float &t_out, float &g_out) {
    float r2;
    if (!hit_surfel_t(sc, j, self, o, d, tmax, eps, t_out, r2)) return false;
    g_out = surfel_G(sc, r2);
    return true;
}

// slab test of the box [lo, hi] against the segment (0, tmax); NaNs from 0*inf are ignored
__device__ __forceinline__ bool slab(float lox, float loy, float loz, float hix, float hiy, float hiz, float3 o,
                                     float3 inv, float tmax) {
    float tx0 = (lox - o.x) * inv.x, tx1 = (hix - o.x) * inv.x;
    float ty0 = (loy - o.y) * inv.y, ty1 = (hiy - o.y) * inv.y;
    float tz0 = (loz - o.z) * inv.z, tz1 = (hiz - o.z) * inv.z;
    float tmin = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.f));
    float tmx = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tmax));
    return tmin <= tmx;
}

// slab test returning the entry distance (clamped to 0) of a hit box
__device__ __forceinline__ bool slab_t(float lox, float loy, float loz, float hix, float hiy, float hiz, float3 o,
                                       float3 inv, float tmax, float &tnear) {
    float tx0 = (lox - o.x) * inv.x, tx1 = (hix - o.x) * inv.x;
    float ty0 = (loy - o.y) * inv.y, ty1 = (hiy - o.y) * inv.y;
    float tz0 = (loz - o.z) * inv.z, tz1 = (hiz - o.z) * inv.z;
    float tmin = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.f));
    float tmx = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tmax));
    tnear = tmin;
    return tmin <= tmx;
}

// Nearer-first traversal for rays that need all hits in depth order: children are
// visited in order of their entry distance, so hits arrive almost sorted and the
// per-ray insertion sort does little work.  Leaves are tested as soon as they are
// reached (postponing them to test all lanes' leaves together was measured slower here:
// lanes holding a leaf idled while the others searched).  Calls f(j) for every surfel
// whose box the ray crosses; returns false if the stack overflowed.
template <class F>
__device__ __forceinline__ bool bvh_traverse_ordered(const SceneDev &sc, float3 o, float3 d, F &&f) {
    if (sc.n == 1) {
        f(0);
        return true;
    }
    const float3 inv = make_float3(1.f / d.x, 1.f / d.y, 1.f / d.z);
    int stack[RGS_STACK];
    int sp = 0;
    int node = 0;
    bool ok = true;
    while (true) {
        const BvhNode nd = sc.nodes[node];
        int cn = nd.d.x, cf = nd.d.y; // near / far child
        float tn, tf;
        bool hn = slab_t(nd.a.x, nd.a.y, nd.a.z, nd.a.w, nd.b.x, nd.b.y, o, inv, INFINITY, tn);
        bool hf = slab_t(nd.b.z, nd.b.w, nd.c.x, nd.c.y, nd.c.z, nd.c.w, o, inv, INFINITY, tf);
        if (hn && hf && tf < tn) {
            const int tc = cn;
            cn = cf;
            cf = tc;
        }
        if (hn && cn < 0) {
            f(~cn);
            hn = false;
        }
        if (hf && cf < 0) {
            f(~cf);
            hf = false;
        }
        if (hn && hf) {
            if (sp < RGS_STACK) stack[sp++] = cf;
            else ok = false;
            node = cn;
        } else if (hn) {
            node = cn;
        } else if (hf) {
            node = cf;
        } else {
            if (sp == 0) break;
            node = stack[--sp];
        }
    }
    return ok;
}

// Visits every surfel whose box the segment (0, tmax) crosses and calls f(j).
// Returns false if the stack overflowed (then part of the tree was skipped).
template <class F>
__device__ __forceinline__ bool bvh_traverse(const SceneDev &sc, float3 o, float3 d, float tmax, F &&f) {
    if (sc.n == 1) {
        f(0);
        return true;
    }
    const float3 inv = make_float3(1.f / d.x, 1.f / d.y, 1.f / d.z);
    int stack[RGS_STACK];
    int sp = 0;
    int node = 0;
    bool ok = true;
    while (true) {
        const BvhNode nd = sc.nodes[node];
        const int cl = nd.d.x, cr = nd.d.y;
        bool hl = slab(nd.a.x, nd.a.y, nd.a.z, nd.a.w, nd.b.x, nd.b.y, o, inv, tmax);
        bool hr = slab(nd.b.z, nd.b.w, nd.c.x, nd.c.y, nd.c.z, nd.c.w, o, inv, tmax);
        if (hl && cl < 0) {
            f(~cl);
            hl = false;
        }
        if (hr && cr < 0) {
            f(~cr);
            hr = false;
        }
        if (hl && hr) {
            if (sp < RGS_STACK) stack[sp++] = cr;
            else ok = false;
            node = cl;
        } else if (hl) {
            node = cl;
        } else if (hr) {
            node = cr;
        } else {
            if (sp == 0) break;
            node = stack[--sp];
        }
    }
    return ok;
}

// ------------------------------------------------------------------ host-side handles
struct rgs_scene {
    int device = 0;
    int n = 0, cap = 0, L = 0, nc = 1, alpha_model = 0;
    float4 *P = nullptr, *N4 = nullptr, *FU = nullptr, *FV = nullptr;
    float4 *GS = nullptr; // Gram-Schmidt record of the frame inputs: |tu|, |tv - (t^u.tv) t^u|, t^u.tv
    float *cl = nullptr, *kk = nullptr;
    int *uid = nullptr, *inv = nullptr;
    BvhNode *nodes = nullptr;
    float *boxes = nullptr; // [2n-1][6]
    int *parent = nullptr, *visit = nullptr;
    unsigned *keys = nullptr, *keys_alt = nullptr;
    int *vals = nullptr, *vals_alt = nullptr;
    int *hist = nullptr;
    int hist_cap = 0;
    int *bounds = nullptr; // 6 ordered ints
    float *eps_plane = nullptr;
    int *flags = nullptr;
    SceneDev dev() const {
        SceneDev s;
        s.n = n;
        s.L = L;
        s.alpha_model = alpha_model;
        s.cutoff2 = (alpha_model == RGS_ALPHA_DISC) ? 1.f : 9.f;
        s.P = P;
        s.N4 = N4;
        s.FU = FU;
        s.FV = FV;
        s.cl = cl;
        s.uid = uid;
        s.inv = inv;
        s.nodes = nodes;
        s.eps_plane = eps_plane;
        return s;
    }
};

enum { RGS_KIND_NONE = 0, RGS_KIND_HEMISPHERE = 1, RGS_KIND_PAIRS = 2 };

// tensor-core contraction state of a transport (rgs_tc.cu): pair tiles and BF16 row blocks
struct rgs_tc_state;
// Monte-Carlo solver state of a transport (rgs_mc.cu): the cached K-means groups
struct rgs_mc_cache;
// the batched modes take the tensor-core contraction from this many columns on (automatic mode)
#define RGS_TC_MIN_COLS 96

struct rgs_transport {
    rgs_scene *sc = nullptr;
    int kind = RGS_KIND_NONE; // which trace built it: hemisphere rays or center-to-center pairs
    int n = 0, L = 0, nc = 1;
    int nd = 0, na = 1, nbs = 1;
    unsigned long long seed = 0;
    int nl = 0, C = 3;
    int ldir = 0; // directional lights (lpos = directions towards them)
    float *lpos = nullptr, *lint = nullptr;
    int lcap = 0;
    // center-to-center pairs: receiver i's pairs at pair_off[i] .. pair_off[i+1], each
    // (source j, bits of V_ji); chunk_off: first pair of each (receiver, 256-source chunk)
    long long *pair_off = nullptr;
    int2 *pair_rec = nullptr;
    long long pair_cap = 0, n_pairs = 0;
    long long *chunk_off = nullptr;
    int *chunk_cnt = nullptr;
    long long chunk_cap = 0;
    long long *chunk_tmp = nullptr;
    int chunk_tmp_cap = 0;
    float *lam = nullptr; // lambda in internal order
    float *aarea = nullptr, *daarea = nullptr; // int alpha_j dx and its derivative in o_j
    int lam_cap = 0;
    // hemisphere hit records
    long long cap_slots = 0;
    int2 *rec_ja = nullptr;
    long long *off = nullptr; // per-ray first record
    int *cnt = nullptr;
    unsigned *ray_ctr = nullptr; // persistent trace: next ray to fetch
    int num_sms = 0;
    float4 *dir = nullptr; // per-ray direction
    // adjoint scratch (dy, dy_mc, tr, v, u, gh): taken from the workspace pool at the start
    // of rgs_adjoint and returned at its end; null outside that call
    float4 *dy = nullptr;  // adjoint: per-ray (y[0..2], 0) for the current column tile
    float *dy_mc = nullptr; // adjoint, many columns: per-ray y of one 32-column tile
    long long rays_cap = 0;
    unsigned long long *counter = nullptr;
    int *flags = nullptr;
    long long n_hits = 0, n_slots = 0, n_full = 0;
    // transposed index (records grouped by source surfel)
    long long *src_off = nullptr;
    int *src_cnt = nullptr;
    unsigned long long *cursor = nullptr;
    int2 *tr = nullptr; // (ray id, bits of a), for the sources of the current index part
    int src_cap = 0;      // surfels allocated in src_off / src_cnt / cursor
    long long *scan_tmp = nullptr;
    int scan_tmp_cap = 0;
    // direct term D [N][C][NC]
    float *D = nullptr;
    long long nc_cap = 0; // capacity (floats) of one [N][C][NC] array
    // iterates.  stride 0: iters holds B^(0..nb) at slot b and Q holds Q^(0..nb-1).
    // stride s >= 1 (checkpointing): slots 0..n_ckpt-1 hold the checkpoints B^(0), B^(s), ...
    // (every multiple of s below nb), slots n_ckpt and n_ckpt+1 the running iterate by parity
    // of b, and Q one scratch array; the adjoint recomputes the rest from the checkpoints.
    int nb_last = -1;
    int ckpt_req = 0;   // rgs_set_checkpointing: 0 store all, s >= 1 every s-th, -1 automatic
    long long mem_budget = 0; // rgs_set_memory_budget: bytes this transport may hold with its scratch (0: none)
    int stride = 0;     // checkpoint stride of the last solve
    int n_ckpt = 0;     // checkpoints stored by the last solve
    int iters_cap = 0;  // number of [N][C][NC] arrays allocated in iters
    int q_cap = 0;      // number of arrays allocated in Q
    float *iters = nullptr;
    float *Q = nullptr;
    __nv_bfloat16 *iters16 = nullptr; // BF16 copies of the iters slots, rows padded to bf16_stride<NC>
    int iters16_cap = 0;
    int prec_last = 0;      // precision of the last solve
    double *norm2 = nullptr; // [RGS_MAX_BOUNCES + 1]
    // forward slot of B^(b) for the last solve
    int slot(int b) const {
        if (!stride) return b;
        if (b % stride == 0 && b / stride < n_ckpt) return b / stride;
        return n_ckpt + (b & 1);
    }
    bool is_stored(int b) const { return !stride || b == nb_last || (b % stride == 0 && b / stride < n_ckpt); }
    // adjoint workspace
    float *v = nullptr; // v^(0..nb), or a ring of stride + 1 arrays when checkpointing
    float *u = nullptr;
    float *Pg = nullptr;  // [N][4][3]
    float *dop = nullptr; // [N]
    int pg_cap = 0;       // surfels allocated in Pg / dop
    float *gh = nullptr;  // per hit-record slot: dL/d(weight) accumulated over the bounces
    long long device_bytes = 0;
    // tensor-core contraction (batched modes): -1 automatic (many columns), 0 off, 1 always
    int tc_mode = -1;
    unsigned long long tc_wait_ns = 4000000000ull; // limit of each pipeline wait (rgs_set_wait_limit)
    bool tc_used = false; // the last solve ran on the tensor-core path
    rgs_tc_state *tc = nullptr;
    rgs_mc_cache *mc = nullptr;
    RaysDev rays() const {
        RaysDev r;
        r.nd = nd;
        r.na = na;
        r.nbs = nbs;
        r.seed = seed;
        r.rec_ja = rec_ja;
        r.off = off;
        r.cnt = cnt;
        r.dir = dir;
        return r;
    }
    size_t arr() const { return (size_t)n * C * nc; }
};

// ------------------------------------------------------------------ host helpers (rgs_api.cu)
// Brackets exactly one kernel launch: counts it and, while profiling is enabled, records
// CUDA events before and after it on its stream (rgs_profile_report reads them).
struct ProfScope {
    ProfScope(const char *name, cudaStream_t st);
    ~ProfScope();
    int rec = -1;
    cudaStream_t st;
};
void rgs_set_error(const char *fmt, ...);
rgs_status rgs_cuda_fail(cudaError_t e, const char *what);
#define RGS_CUDA(call)                                                                                                 \
    do {                                                                                                               \
        cudaError_t e_ = (call);                                                                                       \
        if (e_ != cudaSuccess) return rgs_cuda_fail(e_, #call);                                                        \
    } while (0)
#define RGS_LAUNCH(what)                                                                                               \
    do {                                                                                                               \
        cudaError_t e_ = cudaGetLastError();                                                                           \
        if (e_ != cudaSuccess) return rgs_cuda_fail(e_, what);                                                         \
    } while (0)

// sizes of the library's live cudaMalloc blocks (rgs_api.cu), so that reallocation keeps
// each handle's device_bytes equal to what it holds
void rgs_alloc_note(void *p, size_t bytes);
size_t rgs_alloc_forget(void *p);

template <class T>
rgs_status dev_alloc(T **p, size_t count, long long *acct = nullptr) {
    if (*p) {
        const size_t old = rgs_alloc_forget(*p);
        if (acct) *acct -= (long long)old;
        cudaFree(*p);
        *p = nullptr;
    }
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        rgs_set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
        return RGS_ERR_OOM;
    }
    rgs_alloc_note(*p, count * sizeof(T));
    if (acct) *acct += (long long)(count * sizeof(T));
    return RGS_OK;
}
template <class T> void dev_free(T *&p) {
    if (p) {
        rgs_alloc_forget(p);
        cudaFree(p);
    }
    p = nullptr;
}

// Stream-ordered scratch from a library-owned memory pool (one per device, created on
// first use, memory kept reserved between calls until rgs_trim_workspace).  Used for the
// workspaces that live only inside one call (adjoint), so that transports that run one
// after another on a stream share the same memory.
rgs_status pool_alloc_bytes(void **p, size_t bytes, cudaStream_t st);
// device memory a pool allocation could get now: free memory plus what the pool holds unused
size_t pool_available_bytes();
void pool_free(void *p, cudaStream_t st);
template <class T> rgs_status pool_alloc(T **p, size_t count, cudaStream_t st) {
    *p = nullptr;
    return pool_alloc_bytes(reinterpret_cast<void **>(p), (count ? count : 1) * sizeof(T), st);
}
template <class T> void pool_release(T *&p, cudaStream_t st) {
    if (p) pool_free(p, st);
    p = nullptr;
}

// Column layout of the gathers.  The 3-column kernels (4 lanes share a ray, each lane a
// slice of the coefficients of 3 columns) re-read the hit records and re-evaluate the SH
// per 3-column tile; the lane-per-column kernels (rgs_manycol.cu) read them once per
// 32-column tile but leave lanes idle when C is not a multiple of 32, and load a full
// column row per lane (32 bytes BF16, 64 bytes FP32).  Crossovers measured on GB300 with
// SH degree 3 and 50,000 surfels: the bounce on BF16 rows from 18 columns, on FP32 rows
// from 64; the opacity gather on BF16 rows from 12, on FP32 rows from 64; the adjoint
// (FP32) when one 32-column tile costs less than 26.5 three-column passes would.
__host__ __device__ inline bool wide_bounce(int C, bool rows16) { return C >= (rows16 ? 18 : 64); }
__host__ __device__ inline bool wide_opacity(int C, bool rows16) { return C >= (rows16 ? 12 : 64); }
__host__ __device__ inline bool wide_adjoint(int C) { return 2 * C > 53 * ((C + 31) / 32); }
template <int NC>
rgs_status mc_bounce(const rgs_transport *t, SceneDev sd, RaysDev rd, bool rows16, const float *Bprev,
                     const __nv_bfloat16 *Bprev16, const float *S, float *Q, float *Bout, __nv_bfloat16 *Bout16,
                     double *norm2, cudaStream_t st);
// K^T for the sources j0 .. j1-1, whose transposed entries start at ebase in t->tr
template <int NC>
rgs_status mc_adjoint_bounce(rgs_transport *t, SceneDev sd, RaysDev rd, const float *vin, float *vout, int j0, int j1,
                             long long ebase, cudaStream_t st);
// per-launch set of up to NA adjoint iterates v^(a) and the matching B^(n-1-a) (FP32 or BF16)
template <class T, int NA> struct OpaSet {
    const float *v[NA];
    const T *b[NA];
};
// g_h += sum over the na iterates of the set, for every column (first: write instead of add)
template <int NC>
rgs_status mc_opacity(rgs_transport *t, SceneDev sd, RaysDev rd, int na, const float *const *v, const float *const *Bf,
                      const __nv_bfloat16 *const *Bh, bool first, cudaStream_t st);

// tensor-core contraction (rgs_tc.cu)
bool rgs_tc_eligible(const rgs_transport *t, int precision);
rgs_status rgs_tc_prepare(rgs_transport *t, cudaStream_t st);
rgs_status rgs_tc_prepare_adjoint(rgs_transport *t, cudaStream_t st);
rgs_status rgs_tc_load_blk(rgs_transport *t, const float *x, int slot, bool lo, cudaStream_t st);
rgs_status rgs_tc_bounce(rgs_transport *t, int in, int out, bool split, bool want_lo, const float *Bprev,
                         const float *S, float *Q, float *Bout, __nv_bfloat16 *Bout16, double *norm2, cudaStream_t st);
rgs_status rgs_tc_make_y(rgs_transport *t, const float *v, int slot, cudaStream_t st);
rgs_status rgs_tc_adjoint_bounce(rgs_transport *t, int in, int out, float *vout, float *u, cudaStream_t st);
rgs_status rgs_tc_opacity(rgs_transport *t, int slot, const float *Bsrc, bool first, cudaStream_t st);
// the adjoint's source tiles' hits (built by rgs_tc_prepare_adjoint): per tile [hoff[t], hoff[t+1]),
// per hit its direction (source slot in the weight's 3 low bits), record slot and ray
// per hit its direction (source slot in the weight's 3 low bits), record slot and ray, and a
// per-hit float buffer in the same order
struct RgsTcAdjHits {
    int ntiles;
    long long n_hits;
    const long long *hoff;
    const float4 *hd;
    const uint32_t *hslot, *hray;
    float *gt;
};
bool rgs_tc_adj_hits(const rgs_transport *t, RgsTcAdjHits *out);
// the opacity gather of one adjoint pairing as a sampled product on the tensor cores (rgs_tc_opa.cu)
rgs_status rgs_tc_opacity_sddmm(rgs_transport *t, const float *v, const float *B, bool first, bool last,
                                cudaStream_t st);
int rgs_tc_opa_pass_cols(const rgs_transport *t);
rgs_status rgs_tc_check(rgs_transport *t, cudaStream_t st); // RGS_ERR_TIMEOUT if a bounded wait ran out
rgs_status rgs_tc_reset_flags(rgs_transport *t, cudaStream_t st);
// drops the Monte-Carlo solver's cached K-means groups (rgs_mc.cu)
void rgs_mc_free(rgs_transport *t);
void rgs_tc_invalidate(rgs_transport *t);
void rgs_tc_free(rgs_transport *t);

// entry points implemented per translation unit
rgs_status rgs_scene_build_impl(rgs_scene *s, const rgs_surfels *in, const rgs_build_opts *o, cudaStream_t st);
rgs_status rgs_trace_impl(rgs_transport *t, const rgs_lights *L, const rgs_trace_opts *o, cudaStream_t st);
rgs_status rgs_solve_impl(rgs_transport *t, const float *E, int nb, int precision, float *B_out,
                          rgs_solve_stats *stats, cudaStream_t st);
rgs_status rgs_adjoint_impl(rgs_transport *t, const float *g, float *dE, float *dad, float *dop, cudaStream_t st,
                            float *dp = nullptr, float *ds = nullptr, float *dtu = nullptr, float *dtv = nullptr);
// internal-order accumulators of the geometry gradients: dL/dp [n][3], dL/ds [n][2] and the
// orthonormal frame's (dL/dt^u, dL/dt^v, dL/dn) [n][9]
struct RgsGeoAcc {
    float *dp = nullptr, *ds = nullptr, *gF = nullptr;
};
// the accumulators back to the caller's order, the frame's through Gram-Schmidt (Eq. G)
rgs_status rgs_geometry_out(rgs_transport *t, const RgsGeoAcc &acc, float *dp, float *ds, float *dtu, float *dtv,
                            cudaStream_t st);
rgs_status rgs_get_iterate_impl(rgs_transport *t, int b, float *out, cudaStream_t st);
rgs_status rgs_solve_prepare(rgs_transport *t, int nb, int precision, int stride, cudaStream_t st);
// B^(b) for b in (c, e] from the stored checkpoint or iterate B^(c), with Q^(b-1); outputs are
// indexed by b - c - 1 (B, B16) and b - c - 1 (Q).  Uses the precision of the last solve.
rgs_status rgs_recompute(rgs_transport *t, int c, int e, float *const *B, __nv_bfloat16 *const *B16,
                         float *const *Q, double *norm2, cudaStream_t st);
// stride the automatic checkpoint mode picks for nb bounces at this precision
int rgs_auto_stride(const rgs_transport *t, int nb, int precision);
rgs_status rgs_solve_batched_impl(rgs_transport *const *ts, int count, const float *const *E, const int32_t *nbs,
                                  const rgs_batch_opts *opts, float *const *B_out, double *norms, cudaStream_t st);
void rgs_batch_forget(const rgs_transport *t);
// device-wide exclusive scan of int counts into int64 offsets (offsets[n] = total)
rgs_status rgs_scan_counts(const int *cnt, long long *off, int n, long long *tmp, int tmp_cap, cudaStream_t st);
// light copies and per-surfel buffers shared by both transports; the direct term
rgs_status rgs_transport_common(rgs_transport *t, const rgs_lights *L, cudaStream_t st);
rgs_status rgs_direct_term(rgs_transport *t, cudaStream_t st);
// center-to-center transport (rgs_pairs.cu)
rgs_status rgs_trace_pairs_impl(rgs_transport *t, const rgs_lights *L, const float *lambda, cudaStream_t st);
template <int NC>
rgs_status pairs_bounce(const rgs_transport *t, bool rows16, const float *Bprev, const __nv_bfloat16 *Bprev16,
                        const float *S, float *Q, float *Bout, __nv_bfloat16 *Bout16, double *norm2, cudaStream_t st);
rgs_status rgs_adjoint_pairs_impl(rgs_transport *t, const float *g, float *dE, float *dad, float *dop, float *dlam,
                                  float *dp, float *ds, float *dtu, float *dtv, cudaStream_t st);
// adjoint pieces shared by both transports (rgs_adjoint.cu): v^(0) = dL/dB, u = v^(0),
// P = v^(0) Q^(n-1), dop = 0; P += X Y; the shadow-ray backward; the outputs
rgs_status rgs_adjoint_prologue(rgs_transport *t, int nc, const float *g, cudaStream_t st);
rgs_status rgs_pair_accum(rgs_transport *t, int nc, const float *X, const float *Y, cudaStream_t st);
rgs_status rgs_shadow_backward(rgs_transport *t, int nc, cudaStream_t st, float *dp = nullptr, float *ds = nullptr,
                               float *gF = nullptr);
rgs_status rgs_adjoint_finalize(rgs_transport *t, int nc, float *dE, float *dad, float *dop, cudaStream_t st);
void rgs_copy_offsets(const long long *off, unsigned long long *cursor, int n, cudaStream_t st);
// stable sort of every segment [seg[s], seg[s+1]) of (key, value) by the low 8 * passes bits of
// the key (one 8-bit pass each, one block per segment; rgs_tc.cu); the result lands in (k1, v1)
// for an odd pass count, in (k0, v0) for an even one
rgs_status rgs_seg_sort(const long long *seg, int nseg, int passes, uint32_t *k0, uint2 *v0, uint32_t *k1, uint2 *v1,
                        cudaStream_t st);
// center-to-center transport: fills the transposed pair index tr [n_pairs] (rgs_pairs.cu)
rgs_status rgs_pairs_transpose(rgs_transport *t, int2 *tr, cudaStream_t st);
int rgs_scan_tmp_size(int n);
