// Transport tracing (rgs_trace_transport).
//
//  k_trace_hemi : one thread per hemisphere ray (App. B); a warp is 32 consecutive rays
//                 of one surfel.  Hits are collected during BVH traversal, put in depth
//                 order (near-equal depths by caller index), alpha-composited (Eq. L_I)
//                 and stored as warp-interleaved records (coalesced 256-B rows).
//  k_direct     : one thread per (surfel, light) shadow ray; transmittance product and
//                 the direct term D (Sec. 5.2) for every column of that light.
//  k_src_*      : the same records grouped by source surfel (transposed index) for the
//                 adjoint's gather form of K^T.
#include <algorithm>

#include "rgs_internal.cuh"

#ifndef RGS_TRACE_PATCH_A
#define RGS_TRACE_PATCH_A 8
#endif
#ifndef RGS_TRACE_MINB
#define RGS_TRACE_MINB 12 // resident 128-thread blocks per SM the register budget is sized for (measured best)
#endif

namespace {

// One thread per hemisphere ray; the 32 rays of a warp belong to one surfel.
// Hits are kept as one 64-bit key each, (bits of t) << 32 | j: t > 0, so the unsigned key
// order is the depth order and ties of exactly equal t fall back to the internal index
// (such ties are always re-ordered inside their run).  After compositing, the warp
// allocates exactly its rays' kept hits with one atomic (prefix sum over the lanes) and
// every ray stores its records contiguously.
__global__ void __launch_bounds__(128, RGS_TRACE_MINB) k_trace_hemi(SceneDev sc, RaysDev rays, int n_rays, long long cap_slots,
                                                       unsigned long long *slot_ctr, int2 *rec_ja,
                                                       long long *off_out, int *cnt_out, float4 *dir_out,
                                                       int *src_cnt, int *flags, int pa) {
    const unsigned FULL = 0xffffffffu;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid - (int)(threadIdx.x & 31) >= n_rays) return; // whole warps only (n_rays % 32 == 0)
    const int lane = threadIdx.x & 31;
    // the warps of surfel i take patches of pa x (32 / pa) strata (elevation x azimuth) of its
    // na x nbs grid, so that a warp's rays leave in similar directions; pa = 0: 32 consecutive rays
    const int i = tid / rays.nd;
    int q = tid - i * rays.nd;
    if (pa > 0) {
        const int pb = 32 / pa, w = q >> 5, per_row = rays.nbs / pb;
        const int a = (w / per_row) * pa + lane / pb, b = (w % per_row) * pb + lane % pb;
        q = a * rays.nbs + b;
    }
    const int r = i * rays.nd + q; // the ray this thread traces (outputs are indexed by ray)
    const float3 o = f3(sc.P[i]);
    const float3 d = ray_dir(rays.seed, sc.uid[i], q, rays.na, rays.nbs, f3(sc.FU[i]), f3(sc.FV[i]), f3(sc.N4[i]));
    dir_out[r] = make_float4(d.x, d.y, d.z, 0.f);
    const float eps = *sc.eps_plane;

    unsigned long long key[RGS_HMAX];
    int H = 0;
    bool full = false;
    auto visit = [&](int j) {
        float t, r2;
        if (!hit_surfel_t(sc, j, i, o, d, INFINITY, eps, t, r2)) return;
        const unsigned long long k = ((unsigned long long)__float_as_uint(t) << 32) | (unsigned)j;
        if (H < RGS_HMAX) {
            key[H++] = k;
            return;
        }
        full = true; // keep the RGS_HMAX nearest: replace the farthest if this one is nearer
        int far = 0;
        for (int m = 1; m < RGS_HMAX; ++m)
            if (key[m] > key[far]) far = m;
        if (k < key[far]) key[far] = k;
    };
    if (!bvh_traverse_ordered(sc, o, d, visit)) atomicAdd(&flags[FLAG_STACK], 1);

    for (int a = 1; a < H; ++a) { // insertion sort by key (hits arrive almost sorted)
        const unsigned long long k = key[a];
        int b = a - 1;
        while (b >= 0 && key[b] > k) {
            key[b + 1] = key[b];
            --b;
        }
        key[b + 1] = k;
    }
    for (int k0 = 0; k0 < H;) { // runs of near-equal depth are ordered by caller index
        int e = k0;
        float te = __uint_as_float((unsigned)(key[e] >> 32));
        while (e + 1 < H) {
            const float tn = __uint_as_float((unsigned)(key[e + 1] >> 32));
            if (tn - te > 1e-6f * fmaxf(1.f, te)) break;
            ++e;
            te = tn;
        }
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
    // composite: a_h = alpha_h prod_{k<h} (1 - alpha_k); stop below RGS_T_EPS
    int kept = 0;
    {
        float T = 1.f;
        for (; kept < H; ++kept) {
            if (T < RGS_T_EPS) break;
            const int j = (int)(unsigned)key[kept];
            T *= 1.f - alpha_of(sc, __ldg(&sc.P[j].w),
                                surfel_G(sc, surfel_r2(sc, j, o, d, __uint_as_float((unsigned)(key[kept] >> 32)))));
        }
        // a full buffer only loses something if the transmittance is still above the cut
        if (full && kept == H && T >= RGS_T_EPS) atomicAdd(&flags[FLAG_FULL_RAYS], 1);
    }
    // warp-aggregated, exactly sized record allocation
    int incl = kept;
#pragma unroll
    for (int offs = 1; offs < 32; offs <<= 1) {
        const int v = __shfl_up_sync(FULL, incl, offs);
        if (lane >= offs) incl += v;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    unsigned long long sbase = 0;
    if (lane == 31 && total > 0) sbase = atomicAdd(slot_ctr, (unsigned long long)total);
    sbase = __shfl_sync(FULL, sbase, 31);
    const unsigned long long mine = sbase + (unsigned long long)(incl - kept);
    const bool fits = mine + (unsigned long long)kept <= (unsigned long long)cap_slots;
    off_out[r] = (long long)mine;
    cnt_out[r] = fits ? kept : 0;
    if (!fits) {
        atomicAdd(&flags[FLAG_CAPACITY], 1);
        return;
    }
    float T = 1.f;
    for (int h = 0; h < kept; ++h) {
        const int j = (int)(unsigned)key[h];
        const float G = surfel_G(sc, surfel_r2(sc, j, o, d, __uint_as_float((unsigned)(key[h] >> 32))));
        const float alpha = alpha_of(sc, __ldg(&sc.P[j].w), G);
        rec_ja[mine + h] = make_int2(j, __float_as_int(alpha * T));
        T *= 1.f - alpha;
        atomicAdd(&src_cnt[j], 1); // transposed-index histogram
    }
}

// Direct term (Sec. 5.2): D_i[L*3+ch][k] = o_i c_{i,l(k),ch} Y_k(R_i w) I_{L,ch} (n_i.w)/r^2 T
// (no 1/r^2 and a shadow ray to infinity for a directional light)
template <int NC>
__global__ void k_direct(SceneDev sc, int nl, int ldir, const float *__restrict__ lpos, const float *__restrict__ lint,
                         int C, float *D, int *flags) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= sc.n * nl) return;
    const int i = tid / nl, lt = tid - i * nl;
    const float4 Pi = sc.P[i];
    const float3 o = f3(Pi), n = f3(sc.N4[i]);
    float r, fall;
    const float3 w = light_dir(lpos, lt, o, ldir, r, fall);
    const float cs = dot3(n, w);
    float *Dout = D + ((size_t)i * C + lt * 3) * NC;
    if (!(cs > 0.f)) {
        for (int q = 0; q < 3 * NC; ++q) Dout[q] = 0.f;
        return;
    }
    const float eps = *sc.eps_plane;
    float T = 1.f;
    auto visit = [&](int j) {
        float t, g;
        if (hit_surfel(sc, j, i, o, w, r, eps, t, g)) T *= 1.f - alpha_of(sc, __ldg(&sc.P[j].w), g);
    };
    if (!bvh_traverse(sc, o, w, r, visit)) atomicAdd(&flags[FLAG_STACK], 1);
    float Y[NC];
    sh_eval<NC>(reflect_n(n, w), Y);
    const float pre = alpha_center(sc, i) * cs * fall * T;
    for (int ch = 0; ch < 3; ++ch) {
        const float I = lint[3 * lt + ch];
        for (int k = 0; k < NC; ++k) Dout[ch * NC + k] = sc.cl[(size_t)i * 12 + band_of(k) * 3 + ch] * Y[k] * I * pre;
    }
}

} // namespace

static int strata_a(int nd) {
    int na = 1;
    while ((2 * na) * (2 * na) <= nd) na *= 2;
    return na;
}

// Shared by both transports: the light copies, the per-surfel buffers (flags, D, the
// per-source counts and offsets of the transposed index) sized for the scene.
rgs_status rgs_transport_common(rgs_transport *t, const rgs_lights *L, cudaStream_t st) {
    rgs_scene *sc = t->sc;
    const int n = sc->n;
    t->n = n;
    t->L = sc->L;
    t->nc = sc->nc;
    t->nl = L ? L->n_lights : 0;
    t->ldir = (L && L->directional) ? 1 : 0;
    t->C = 3 * (t->nl > 0 ? t->nl : 1);
    t->nb_last = -1;
    rgs_status r;
    if (t->nl > t->lcap) {
        if ((r = dev_alloc(&t->lpos, 3 * (size_t)t->nl, &t->device_bytes)) != RGS_OK) return r;
        if ((r = dev_alloc(&t->lint, 3 * (size_t)t->nl, &t->device_bytes)) != RGS_OK) return r;
        t->lcap = t->nl;
    }
    if (t->nl > 0) {
        RGS_CUDA(cudaMemcpyAsync(t->lpos, L->pos, sizeof(float) * 3 * t->nl, cudaMemcpyDeviceToDevice, st));
        RGS_CUDA(cudaMemcpyAsync(t->lint, L->intensity, sizeof(float) * 3 * t->nl, cudaMemcpyDeviceToDevice, st));
    }
    if (!t->counter && (r = dev_alloc(&t->counter, 1, &t->device_bytes)) != RGS_OK) return r;
    if (!t->flags && (r = dev_alloc(&t->flags, FLAG_COUNT, &t->device_bytes)) != RGS_OK) return r;
    const long long arr = (long long)n * t->C * t->nc;
    if (arr > t->nc_cap) {
        if ((r = dev_alloc(&t->D, (size_t)arr, &t->device_bytes)) != RGS_OK) return r;
        t->nc_cap = arr;
        t->iters_cap = 0; // iterate buffers are sized by the array size: force regrowth
        t->q_cap = 0;
        t->iters16_cap = 0;
    }
    if (n > t->src_cap) {
        if ((r = dev_alloc(&t->src_off, (size_t)n + 1, &t->device_bytes)) != RGS_OK) return r;
        if ((r = dev_alloc(&t->src_cnt, (size_t)n, &t->device_bytes)) != RGS_OK) return r;
        if ((r = dev_alloc(&t->cursor, (size_t)n, &t->device_bytes)) != RGS_OK) return r;
        t->scan_tmp_cap = rgs_scan_tmp_size(n);
        if ((r = dev_alloc(&t->scan_tmp, (size_t)t->scan_tmp_cap, &t->device_bytes)) != RGS_OK) return r;
        t->src_cap = n;
    }
    return RGS_OK;
}

// D = o c (x) Y(R w) I cos / r^2 T for every (surfel, light), or 0 without lights
rgs_status rgs_direct_term(rgs_transport *t, cudaStream_t st) {
    SceneDev sd = t->sc->dev();
    if (t->nl > 0) {
        const int nth = t->n * t->nl;
        switch (t->nc) {
        case 1: { ProfScope ps_("k_direct", st); k_direct<1><<<(nth + 127) / 128, 128, 0, st>>>(sd, t->nl, t->ldir, t->lpos, t->lint, t->C, t->D, t->flags); } break;
        case 4: { ProfScope ps_("k_direct", st); k_direct<4><<<(nth + 127) / 128, 128, 0, st>>>(sd, t->nl, t->ldir, t->lpos, t->lint, t->C, t->D, t->flags); } break;
        case 9: { ProfScope ps_("k_direct", st); k_direct<9><<<(nth + 127) / 128, 128, 0, st>>>(sd, t->nl, t->ldir, t->lpos, t->lint, t->C, t->D, t->flags); } break;
        default: { ProfScope ps_("k_direct", st); k_direct<16><<<(nth + 127) / 128, 128, 0, st>>>(sd, t->nl, t->ldir, t->lpos, t->lint, t->C, t->D, t->flags); }
        }
        RGS_LAUNCH("direct");
    } else {
        RGS_CUDA(cudaMemsetAsync(t->D, 0, sizeof(float) * t->arr(), st));
    }
    return RGS_OK;
}

rgs_status rgs_trace_impl(rgs_transport *t, const rgs_lights *L, const rgs_trace_opts *o, cudaStream_t st) {
    rgs_scene *sc = t->sc;
    const int n = sc->n;
    rgs_status r;
    t->kind = RGS_KIND_HEMISPHERE;
    rgs_tc_invalidate(t);
    rgs_mc_free(t);
    t->tc_used = false;
    t->nd = o->nd;
    t->na = strata_a(o->nd);
    t->nbs = o->nd / t->na;
    t->seed = o->seed;
    if ((r = rgs_transport_common(t, L, st)) != RGS_OK) return r;
    const long long n_rays = (long long)n * o->nd;
    // per-ray arrays
    if (n_rays > t->rays_cap) {
        if ((r = dev_alloc(&t->cnt, (size_t)n_rays, &t->device_bytes)) != RGS_OK) return r;
        if ((r = dev_alloc(&t->dir, (size_t)n_rays, &t->device_bytes)) != RGS_OK) return r;
        if ((r = dev_alloc(&t->off, (size_t)n_rays, &t->device_bytes)) != RGS_OK) return r;
        t->rays_cap = n_rays;
    }

    long long want = o->hit_capacity > 0 ? o->hit_capacity : (t->cap_slots > 0 ? t->cap_slots : n_rays * 24);
    if (o->hit_capacity <= 0 && t->cap_slots == 0) {
        // first trace of a large transport: rather than reserve a guess of 24 slots per ray,
        // let the first pass only count (no slots: every warp's store is refused, the
        // counter still adds up) and reserve what it needs
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) cudaGetLastError();
        if ((double)want * sizeof(int2) > 0.25 * (double)free_b) want = 0;
    }
    SceneDev sd = sc->dev();
    // warp patch of the strata grid: the largest pa <= RGS_TRACE_PATCH_A dividing na with
    // 32 / pa dividing nbs; none (0) keeps 32 consecutive rays per warp
    int pa = 0;
    for (int c = RGS_TRACE_PATCH_A; c >= 1 && !pa; c >>= 1)
        if (t->na % c == 0 && 32 % c == 0 && t->nbs % (32 / c) == 0) pa = c;
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (want > t->cap_slots) {
            if ((r = dev_alloc(&t->rec_ja, (size_t)want, &t->device_bytes)) != RGS_OK) return r;
            t->cap_slots = want;
        }
        RGS_CUDA(cudaMemsetAsync(t->counter, 0, sizeof(unsigned long long), st));
        RGS_CUDA(cudaMemsetAsync(t->flags, 0, sizeof(int) * FLAG_COUNT, st));
        RGS_CUDA(cudaMemsetAsync(t->src_cnt, 0, sizeof(int) * n, st));
        RaysDev rd = t->rays();
        const int TB = 128;
        { ProfScope ps_("k_trace_hemi", st); k_trace_hemi<<<(unsigned)((n_rays + TB - 1) / TB), TB, 0, st>>>(sd, rd, (int)n_rays, t->cap_slots, t->counter, t->rec_ja, t->off, t->cnt, t->dir, t->src_cnt, t->flags, pa); }
        RGS_LAUNCH("trace_hemi");
        unsigned long long used = 0;
        int flags[FLAG_COUNT];
        RGS_CUDA(cudaMemcpyAsync(&used, t->counter, sizeof used, cudaMemcpyDeviceToHost, st));
        RGS_CUDA(cudaMemcpyAsync(flags, t->flags, sizeof flags, cudaMemcpyDeviceToHost, st));
        RGS_CUDA(cudaStreamSynchronize(st));
        t->n_slots = (long long)used;
        t->n_full = flags[FLAG_FULL_RAYS];
        if (flags[FLAG_STACK]) {
            rgs_set_error("BVH traversal stack overflow on %d rays", flags[FLAG_STACK]);
            return RGS_ERR_CAPACITY;
        }
        if (!flags[FLAG_CAPACITY]) break;
        if (o->hit_capacity > 0 || attempt == 1) {
            rgs_set_error("hit-record capacity %lld slots too small (%llu needed)", t->cap_slots, used);
            return RGS_ERR_CAPACITY;
        }
        const unsigned long long slack = used > (1ull << 30) ? used / 32 : used / 8; // for later re-traces
        want = (long long)(used + slack + 1024);
    }

    if ((r = rgs_direct_term(t, st)) != RGS_OK) return r;

    // per-source hit counts -> offsets of the transposed index (filled by rgs_adjoint)
    if ((r = rgs_scan_counts(t->src_cnt, t->src_off, n, t->scan_tmp, t->scan_tmp_cap, st)) != RGS_OK) return r;
    long long total = 0;
    RGS_CUDA(cudaMemcpyAsync(&total, t->src_off + n, sizeof total, cudaMemcpyDeviceToHost, st));
    RGS_CUDA(cudaStreamSynchronize(st));
    t->n_hits = total;
    return RGS_OK;
}
