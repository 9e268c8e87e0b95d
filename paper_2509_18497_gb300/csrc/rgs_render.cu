// Image formation (rgs_render / rgs_render_adjoint): Eq. L_I for the rays of a pinhole camera
// over a solved radiance B -- what the paper's tile rasterizer draws from the surfels'
// outgoing SH radiance (Sec. 5.3, end) -- and its transpose, the dL/dB a loss on the image
// hands to rgs_adjoint (Sec. 6, opening).
//
//  k_render_trace : one thread per pixel.  The pixel ray o + t d meets the surfels in depth
//                   order under the transport's hit rules (eps_plane, the cutoff, tie runs;
//                   no surfel excluded), composited a_h = alpha_h prod_{k<h} (1 - alpha_k)
//                   until the transmittance is below RGS_T_EPS; records (j, a_h) per pixel.
//  k_render_shade : a warp per pixel, a lane per column: I[c] = sum_h a_h Y(-d)^T B_j[c].
//  k_render_adj   : a warp per pixel, a lane per column: dB_j[c][k] += a_h Y_k(-d) dI[c].
#include "rgs_bounce_body.cuh"

namespace {

constexpr int RN_THREADS = 128;

// pixel (x, y) (y down) of a W x H pinhole camera cam = {o, forward, up} with vertical field
// of view fov: right = forward x up, the true up = right x forward, the pixel's centre
__device__ __forceinline__ float3 pixel_dir(const float *cam, int W, int H, float fov, int x, int y) {
    const float3 f = make_float3(cam[3], cam[4], cam[5]), u0 = make_float3(cam[6], cam[7], cam[8]);
    const float lf = sqrtf(dot3(f, f));
    const float3 fn = (1.f / lf) * f;
    float3 r = make_float3(fn.y * u0.z - fn.z * u0.y, fn.z * u0.x - fn.x * u0.z, fn.x * u0.y - fn.y * u0.x);
    r = (1.f / sqrtf(dot3(r, r))) * r;
    const float3 u = make_float3(r.y * fn.z - r.z * fn.y, r.z * fn.x - r.x * fn.z, r.x * fn.y - r.y * fn.x);
    const float th = tanf(0.5f * fov);
    const float sx = (2.f * (x + 0.5f) / (float)W - 1.f) * th * (float)W / (float)H;
    const float sy = (1.f - 2.f * (y + 0.5f) / (float)H) * th;
    float3 d = fn + sx * r + sy * u;
    return (1.f / sqrtf(dot3(d, d))) * d;
}

struct Cam {
    float v[9];
};

// The composited hits of one pixel ray, nearest first: emit(h, j, a_h) for h = 0, 1, ...
// until the transmittance falls below RGS_T_EPS.  Hits are gathered RGS_HMAX at a time: each
// pass keeps the RGS_HMAX nearest hits beyond the previous pass's last composited one, so a
// ray composites any number of hits.  A full buffer's last run of near-equal depths may
// continue past the buffer, so it is left to the next pass (a run is never split, unless one
// run alone fills the buffer).  Returns false if the traversal stack overflowed.
template <class F>
__device__ bool render_ray(const SceneDev &sc, float3 o, float3 d, float eps, F &&emit) {
    unsigned long long key[RGS_HMAX];
    unsigned long long lower = 0ull;
    bool have_lower = false, ok = true;
    float T = 1.f;
    int out = 0;
    while (true) {
        int nh = 0;
        auto visit = [&](int j) {
            float t, r2;
            if (!hit_surfel_t(sc, j, -1, o, d, INFINITY, eps, t, r2)) return;
            const unsigned long long k = ((unsigned long long)__float_as_uint(t) << 32) | (unsigned)j;
            if (have_lower && k <= lower) return;
            if (nh < RGS_HMAX) {
                key[nh++] = k;
                return;
            }
            int far = 0; // keep the RGS_HMAX nearest
            for (int m = 1; m < RGS_HMAX; ++m)
                if (key[m] > key[far]) far = m;
            if (k < key[far]) key[far] = k;
        };
        ok = bvh_traverse_ordered(sc, o, d, visit) && ok;
        for (int a = 1; a < nh; ++a) { // depth order
            const unsigned long long k = key[a];
            int b = a - 1;
            while (b >= 0 && key[b] > k) {
                key[b + 1] = key[b];
                --b;
            }
            key[b + 1] = k;
        }
        auto tkey = [&](int m) { return __uint_as_float((unsigned)(key[m] >> 32)); };
        auto same_run = [&](int m) { // hit m + 1 continues the run of hit m
            const float tm = tkey(m);
            return tkey(m + 1) - tm <= 1e-6f * fmaxf(1.f, tm);
        };
        const bool full = nh == RGS_HMAX;
        int limit = nh;
        if (full) {
            int s0 = nh - 1;
            while (s0 > 0 && same_run(s0 - 1)) --s0;
            if (s0 > 0) limit = s0;
        }
        for (int k0 = 0; k0 < limit;) { // runs of near-equal depth by caller index
            int e = k0;
            while (e + 1 < limit && same_run(e)) ++e;
            for (int a = k0 + 1; a <= e; ++a) {
                const unsigned long long k = key[a];
                const int uk = sc.uid[(int)(unsigned)k];
                int b = a - 1;
                while (b >= k0 && sc.uid[(int)(unsigned)key[b]] > uk) {
                    key[b + 1] = key[b];
                    --b;
                }
                key[b + 1] = k;
            }
            k0 = e + 1;
        }
        unsigned long long last = 0ull;
        for (int h = 0; h < limit && T >= RGS_T_EPS; ++h) {
            const int j = (int)(unsigned)key[h];
            const float G = surfel_G(sc, surfel_r2(sc, j, o, d, tkey(h)));
            const float alpha = alpha_of(sc, __ldg(&sc.P[j].w), G);
            emit(out++, j, alpha * T);
            T *= 1.f - alpha;
            last = max(last, key[h]);
        }
        if (!full || T < RGS_T_EPS) break;
        lower = last; // every key up to the composited ones (the run order may differ from key order)
        have_lower = true;
    }
    return ok;
}

// pass 0 counts every pixel's composited hits; pass 1 writes them (j, a_h) at the pixel's offset
template <bool FILL>
__global__ void __launch_bounds__(RN_THREADS) k_render_trace(SceneDev sc, Cam cam, int W, int H, float fov,
                                                            int *cnt, const long long *__restrict__ off, int2 *rec,
                                                            float4 *pdir, int *flags) {
    const int pix = blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= W * H) return;
    const int x = pix % W, y = pix / W;
    const float3 o = make_float3(cam.v[0], cam.v[1], cam.v[2]);
    const float3 d = pixel_dir(cam.v, W, H, fov, x, y);
    const float eps = *sc.eps_plane;
    int n = 0;
    bool ok;
    if (FILL) {
        int2 *r = rec + off[pix];
        ok = render_ray(sc, o, d, eps, [&](int h, int j, float a) {
            r[h] = make_int2(j, __float_as_int(a));
            n = h + 1;
        });
    } else {
        ok = render_ray(sc, o, d, eps, [&](int h, int, float) { n = h + 1; });
        pdir[pix] = make_float4(d.x, d.y, d.z, 0.f);
        cnt[pix] = n;
    }
    if (!ok && !FILL) atomicAdd(&flags[FLAG_STACK], 1);
}

// internal [N][C][NC] <- user [N][nc][C]
template <int NC>
__global__ void k_render_from_user(int n, int C, const int *__restrict__ uid, const float *__restrict__ X, float *Y) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * C * NC) return;
    const int k = (int)(idx % NC);
    const size_t ic = idx / NC;
    const int c = (int)(ic % C);
    const int i = (int)(ic / C);
    Y[idx] = X[((size_t)uid[i] * NC + k) * C + c];
}
// user [N][nc][C] <- internal [N][C][NC]
template <int NC>
__global__ void k_render_to_user(int n, int C, const int *__restrict__ uid, const float *__restrict__ X, float *Y) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * C * NC) return;
    const int k = (int)(idx % NC);
    const size_t ic = idx / NC;
    const int c = (int)(ic % C);
    const int i = (int)(ic / C);
    Y[((size_t)uid[i] * NC + k) * C + c] = X[idx];
}

template <int NC>
__global__ void __launch_bounds__(RN_THREADS) k_render_shade(int npix, int C, const int2 *__restrict__ rec,
                                                            const long long *__restrict__ off, const float4 *__restrict__ pdir,
                                                            const float *__restrict__ B, float *img) {
    const int pix = (int)(((size_t)blockIdx.x * RN_THREADS + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (pix >= npix) return;
    const float4 d4 = pdir[pix];
    float Yo[NC];
    sh_eval<NC>(make_float3(-d4.x, -d4.y, -d4.z), Yo);
    const long long h0 = off[pix], h1 = off[pix + 1];
    if constexpr (NC == 16) {
        // 32-column tiles of each source row read as four contiguous 512-B warp requests, every
        // lane ending with the dot product of one tile column (TileDot)
        float ys[4];
        TileDot<float, 16>::pick(Yo, lane, ys);
        const int own = TileDot<float, 16>::own(lane);
        for (int c0 = 0; c0 < C; c0 += 32) {
            const int ncols = min(32, C - c0);
            float acc = 0.f;
            for (long long h = h0; h < h1; ++h) {
                const int2 ja = __ldg(&rec[h]);
                acc += __int_as_float(ja.y) * TileDot<float, 16>::dot(B + ((size_t)ja.x * C + c0) * 16, ncols, lane, ys);
            }
            if (own < ncols) img[(size_t)pix * C + c0 + own] = acc;
        }
    } else {
        for (int c = lane; c < C; c += 32) {
            float acc = 0.f;
            for (long long h = h0; h < h1; ++h) {
                const int2 ja = __ldg(&rec[h]);
                const float *row = B + ((size_t)ja.x * C + c) * NC;
                float s = 0.f;
#pragma unroll
                for (int k = 0; k < NC; ++k) s += Yo[k] * __ldg(row + k);
                acc += __int_as_float(ja.y) * s;
            }
            img[(size_t)pix * C + c] = acc;
        }
    }
}

template <int NC>
__global__ void __launch_bounds__(RN_THREADS) k_render_adj(int npix, int C, const int2 *__restrict__ rec,
                                                          const long long *__restrict__ off, const float4 *__restrict__ pdir,
                                                          const float *__restrict__ dimg, float *dB) {
    const int pix = (int)(((size_t)blockIdx.x * RN_THREADS + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (pix >= npix) return;
    const float4 d4 = pdir[pix];
    float Yo[NC];
    sh_eval<NC>(make_float3(-d4.x, -d4.y, -d4.z), Yo);
    const long long h0 = off[pix], h1 = off[pix + 1];
    for (int c = lane; c < C; c += 32) {
        const float g = dimg[(size_t)pix * C + c];
        if (g == 0.f) continue;
        for (long long h = h0; h < h1; ++h) {
            const int2 ja = __ldg(&rec[h]);
            const float ga = __int_as_float(ja.y) * g;
            float *row = dB + ((size_t)ja.x * C + c) * NC;
            if constexpr (NC % 4 == 0) { // rows of NC floats start on 16-byte boundaries
#pragma unroll
                for (int q = 0; q < NC / 4; ++q)
                    atomicAdd(reinterpret_cast<float4 *>(row) + q,
                              make_float4(ga * Yo[4 * q], ga * Yo[4 * q + 1], ga * Yo[4 * q + 2], ga * Yo[4 * q + 3]));
            } else {
#pragma unroll
                for (int k = 0; k < NC; ++k) atomicAdd(row + k, ga * Yo[k]);
            }
        }
    }
}

struct RenderScratch {
    cudaStream_t st;
    int2 *rec = nullptr;
    int *cnt = nullptr;
    long long *off = nullptr, *scan_tmp = nullptr;
    float4 *pdir = nullptr;
    float *X = nullptr;
    int *flag = nullptr;
    ~RenderScratch() {
        pool_release(flag, st);
        pool_release(rec, st);
        pool_release(cnt, st);
        pool_release(off, st);
        pool_release(scan_tmp, st);
        pool_release(pdir, st);
        pool_release(X, st);
    }
};

rgs_status check_args(const rgs_transport *t, const float *in, const float *cam, int W, int H, float fov,
                      const float *out, const char *what) {
    if (!t || !in || !cam || !out) {
        rgs_set_error("%s: NULL argument", what);
        return RGS_ERR_ARG;
    }
    if (t->kind == RGS_KIND_NONE) {
        rgs_set_error("%s: the transport has not been traced", what);
        return RGS_ERR_STATE;
    }
    if (W <= 0 || H <= 0 || (long long)W * H > (1ll << 26) || !(fov > 0.f && fov < 3.14159f)) {
        rgs_set_error("%s: image %d x %d or field of view %g out of range", what, W, H, (double)fov);
        return RGS_ERR_ARG;
    }
    for (int q = 0; q < 9; ++q)
        if (!isfinite(cam[q])) {
            rgs_set_error("%s: non-finite camera", what);
            return RGS_ERR_NONFINITE;
        }
    return RGS_OK;
}

// traces every pixel twice into pooled scratch: the counts (and directions), their offsets,
// then the exactly sized records
rgs_status render_trace(rgs_transport *t, const float *cam, int W, int H, float fov, RenderScratch &s) {
    rgs_status r;
    const int npix = W * H;
    const int tmp_cap = rgs_scan_tmp_size(npix);
    if ((r = pool_alloc(&s.cnt, (size_t)npix, s.st)) != RGS_OK) return r;
    if ((r = pool_alloc(&s.off, (size_t)npix + 1, s.st)) != RGS_OK) return r;
    if ((r = pool_alloc(&s.scan_tmp, (size_t)tmp_cap, s.st)) != RGS_OK) return r;
    if ((r = pool_alloc(&s.pdir, (size_t)npix, s.st)) != RGS_OK) return r;
    if ((r = pool_alloc(&s.flag, (size_t)FLAG_COUNT, s.st)) != RGS_OK) return r;
    RGS_CUDA(cudaMemsetAsync(s.flag, 0, sizeof(int) * FLAG_COUNT, s.st));
    Cam c;
    for (int q = 0; q < 9; ++q) c.v[q] = cam[q];
    const SceneDev sd = t->sc->dev();
    const unsigned blocks = (npix + RN_THREADS - 1) / RN_THREADS;
    {
        ProfScope ps_("k_render_trace", s.st);
        k_render_trace<false><<<blocks, RN_THREADS, 0, s.st>>>(sd, c, W, H, fov, s.cnt, nullptr, nullptr, s.pdir, s.flag);
    }
    RGS_LAUNCH("render trace (count)");
    if ((r = rgs_scan_counts(s.cnt, s.off, npix, s.scan_tmp, tmp_cap, s.st)) != RGS_OK) return r;
    long long total = 0;
    int stack_overflows = 0;
    RGS_CUDA(cudaMemcpyAsync(&total, s.off + npix, sizeof total, cudaMemcpyDeviceToHost, s.st));
    RGS_CUDA(cudaMemcpyAsync(&stack_overflows, s.flag + FLAG_STACK, sizeof(int), cudaMemcpyDeviceToHost, s.st));
    RGS_CUDA(cudaStreamSynchronize(s.st));
    if (stack_overflows) {
        rgs_set_error("render: BVH traversal stack overflow on %d pixel rays", stack_overflows);
        return RGS_ERR_CAPACITY;
    }
    if ((r = pool_alloc(&s.rec, (size_t)total, s.st)) != RGS_OK) return r;
    if (total > 0) {
        ProfScope ps_("k_render_trace", s.st);
        k_render_trace<true><<<blocks, RN_THREADS, 0, s.st>>>(sd, c, W, H, fov, nullptr, s.off, s.rec, nullptr, s.flag);
    }
    RGS_LAUNCH("render trace (fill)");
    return RGS_OK;
}

template <int NC>
rgs_status render_nc(rgs_transport *t, const float *B, const float *cam, int W, int H, float fov, float *img,
                     cudaStream_t st) {
    rgs_status r;
    RenderScratch s{st};
    const size_t A = (size_t)t->n * t->C * NC;
    if ((r = pool_alloc(&s.X, A, st)) != RGS_OK) return r;
    {
        ProfScope ps_("k_render_from_user", st);
        k_render_from_user<NC><<<(unsigned)((A + 255) / 256), 256, 0, st>>>(t->n, t->C, t->sc->uid, B, s.X);
    }
    RGS_LAUNCH("render from user");
    if ((r = render_trace(t, cam, W, H, fov, s)) != RGS_OK) return r;
    const int npix = W * H;
    {
        ProfScope ps_("k_render_shade", st);
        k_render_shade<NC><<<(unsigned)(((size_t)npix * 32 + RN_THREADS - 1) / RN_THREADS), RN_THREADS, 0, st>>>(
            npix, t->C, s.rec, s.off, s.pdir, s.X, img);
    }
    RGS_LAUNCH("render shade");
    return RGS_OK;
}

template <int NC>
rgs_status render_adjoint_nc(rgs_transport *t, const float *dimg, const float *cam, int W, int H, float fov,
                             float *dB, cudaStream_t st) {
    rgs_status r;
    RenderScratch s{st};
    const size_t A = (size_t)t->n * t->C * NC;
    if ((r = pool_alloc(&s.X, A, st)) != RGS_OK) return r;
    RGS_CUDA(cudaMemsetAsync(s.X, 0, sizeof(float) * A, st));
    if ((r = render_trace(t, cam, W, H, fov, s)) != RGS_OK) return r;
    const int npix = W * H;
    {
        ProfScope ps_("k_render_adj", st);
        k_render_adj<NC><<<(unsigned)(((size_t)npix * 32 + RN_THREADS - 1) / RN_THREADS), RN_THREADS, 0, st>>>(
            npix, t->C, s.rec, s.off, s.pdir, dimg, s.X);
    }
    RGS_LAUNCH("render adjoint");
    {
        ProfScope ps_("k_render_to_user", st);
        k_render_to_user<NC><<<(unsigned)((A + 255) / 256), 256, 0, st>>>(t->n, t->C, t->sc->uid, s.X, dB);
    }
    RGS_LAUNCH("render to user");
    return RGS_OK;
}

} // namespace

extern "C" rgs_status rgs_render(rgs_transport *t, const float *B, const float *cam, int32_t W, int32_t H, float fov,
                                 float *img, void *stream) {
    rgs_status r = check_args(t, B, cam, W, H, fov, img, "rgs_render");
    if (r != RGS_OK) return r;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    switch (t->nc) {
    case 1: return render_nc<1>(t, B, cam, W, H, fov, img, st);
    case 4: return render_nc<4>(t, B, cam, W, H, fov, img, st);
    case 9: return render_nc<9>(t, B, cam, W, H, fov, img, st);
    default: return render_nc<16>(t, B, cam, W, H, fov, img, st);
    }
}

extern "C" rgs_status rgs_render_adjoint(rgs_transport *t, const float *dL_dimg, const float *cam, int32_t W,
                                         int32_t H, float fov, float *dL_dB, void *stream) {
    rgs_status r = check_args(t, dL_dimg, cam, W, H, fov, dL_dB, "rgs_render_adjoint");
    if (r != RGS_OK) return r;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    switch (t->nc) {
    case 1: return render_adjoint_nc<1>(t, dL_dimg, cam, W, H, fov, dL_dB, st);
    case 4: return render_adjoint_nc<4>(t, dL_dimg, cam, W, H, fov, dL_dB, st);
    case 9: return render_adjoint_nc<9>(t, dL_dimg, cam, W, H, fov, dL_dB, st);
    default: return render_adjoint_nc<16>(t, dL_dimg, cam, W, H, fov, dL_dB, st);
    }
}
