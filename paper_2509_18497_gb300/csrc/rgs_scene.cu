// Scene build (rgs_build_scene): frames (Eq. G), BRDF coefficients (Eq. brdf, App. A),
// Morton order of the surfel centres and a binary LBVH over the cutoff ellipses.
//
// The BVH follows the linear construction of Karras (HPG 2012): sorted 30-bit Morton
// codes, one internal node per adjacent pair found from common prefixes, then a
// bottom-up box refit with one atomic arrival counter per node.  The sort is a
// stable 4-pass LSD radix sort written here (no library sort).
#include <stdio.h>

#include "rgs_internal.cuh"

namespace {

constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 8; // keys per thread per tile -> 2048-key tiles
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;

__device__ __forceinline__ int f2ord(float f) {
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ord2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void k_init_bounds(int *b) {
    if (threadIdx.x < 3) b[threadIdx.x] = 0x7fffffff;
    else if (threadIdx.x < 6) b[threadIdx.x] = (int)0x80000000;
}

__global__ void k_bounds(const float *__restrict__ p, int n, int *bounds) {
    __shared__ int smin[3], smax[3];
    if (threadIdx.x < 3) {
        smin[threadIdx.x] = 0x7fffffff;
        smax[threadIdx.x] = (int)0x80000000;
    }
    __syncthreads();
    int lo[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, hi[3] = {(int)0x80000000, (int)0x80000000, (int)0x80000000};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int a = 0; a < 3; ++a) {
            int v = f2ord(p[3 * (size_t)i + a]);
            lo[a] = min(lo[a], v);
            hi[a] = max(hi[a], v);
        }
    for (int a = 0; a < 3; ++a) {
        atomicMin(&smin[a], lo[a]);
        atomicMax(&smax[a], hi[a]);
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        atomicMin(&bounds[threadIdx.x], smin[threadIdx.x]);
        atomicMax(&bounds[3 + threadIdx.x], smax[threadIdx.x]);
    }
}

__device__ __forceinline__ unsigned expand_bits(unsigned v) { // 10 bits -> every third bit
    v = (v * 0x00010001u) & 0xFF0000FFu;
    v = (v * 0x00000101u) & 0x0F00F00Fu;
    v = (v * 0x00000011u) & 0xC30C30C3u;
    v = (v * 0x00000005u) & 0x49249249u;
    return v;
}

__global__ void k_morton(const float *__restrict__ p, int n, const int *bounds, unsigned *keys, int *vals,
                         float *eps_plane) {
    float lo[3], ext[3];
    float diag2 = 0.f;
    for (int a = 0; a < 3; ++a) {
        lo[a] = ord2f(bounds[a]);
        float hi = ord2f(bounds[3 + a]);
        ext[a] = fmaxf(hi - lo[a], 1e-30f);
        diag2 += (hi - lo[a]) * (hi - lo[a]);
    }
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *eps_plane = 1e-5f * sqrtf(diag2);
    if (i >= n) return;
    unsigned q[3];
    for (int a = 0; a < 3; ++a) {
        float u = (p[3 * (size_t)i + a] - lo[a]) / ext[a];
        q[a] = (unsigned)fminf(fmaxf(u * 1024.f, 0.f), 1023.f);
    }
    keys[i] = (expand_bits(q[0]) << 2) | (expand_bits(q[1]) << 1) | expand_bits(q[2]);
    vals[i] = i;
}

// ---------------------------------------------------------------- radix sort (stable LSD)
__global__ void k_radix_hist(const unsigned *__restrict__ keys, int n, int shift, int nblocks, int *hist) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int base = blockIdx.x * SORT_TILE;
    for (int it = 0; it < SORT_ITEMS; ++it) {
        int i = base + it * SORT_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x]; // digit-major
}

// exclusive scan of m ints in place, single block of 1024 threads
__global__ void k_scan_single(int *a, int m) {
    __shared__ int s[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < m; base += 1024) {
        int i = base + threadIdx.x;
        int v = i < m ? a[i] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            int t = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < m) a[i] = carry + s[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += s[1023];
        __syncthreads();
    }
}

__global__ void k_radix_scatter(const unsigned *__restrict__ kin, const int *__restrict__ vin, unsigned *kout,
                                int *vout, int n, int shift, int nblocks, const int *__restrict__ hist) {
    __shared__ int run[256];    // running offset of each digit within this tile
    __shared__ int wcnt[8][256]; // per-warp digit counts of the current chunk
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    run[threadIdx.x] = hist[threadIdx.x * nblocks + blockIdx.x];
    int base = blockIdx.x * SORT_TILE;
    for (int it = 0; it < SORT_ITEMS; ++it) {
        for (int w = 0; w < 8; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        int i = base + it * SORT_THREADS + threadIdx.x;
        bool valid = i < n;
        unsigned key = valid ? kin[i] : 0u;
        int dig = valid ? (int)((key >> shift) & 255u) : 256 + lane; // invalid lanes get unique dummies
        unsigned peers = __match_any_sync(0xffffffffu, dig);
        int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wcnt[warp][dig] = __popc(peers);
        __syncthreads();
        if (valid) {
            int off = run[dig];
            for (int w = 0; w < warp; ++w) off += wcnt[w][dig];
            kout[off + rank] = key;
            vout[off + rank] = vin[i];
        }
        __syncthreads();
        int tot = 0;
        for (int w = 0; w < 8; ++w) tot += wcnt[w][threadIdx.x];
        run[threadIdx.x] += tot;
        __syncthreads();
    }
}

// ---------------------------------------------------------------- surfel gather
__global__ void k_gather(rgs_surfels in, int n, int L, int alpha_model, const int *__restrict__ perm, float4 *P,
                         float4 *N4, float4 *FU, float4 *FV, float4 *GS, float *cl, float *kk, int *uid, int *inv,
                         float *boxes, int *flags) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int i = perm[k];
    uid[k] = i;
    inv[i] = k;
    float3 p = make_float3(in.p[3 * i], in.p[3 * i + 1], in.p[3 * i + 2]);
    float3 a = make_float3(in.tu[3 * i], in.tu[3 * i + 1], in.tu[3 * i + 2]);
    float3 b = make_float3(in.tv[3 * i], in.tv[3 * i + 1], in.tv[3 * i + 2]);
    // Gram-Schmidt, n = tu x tv (Eq. G)
    float la = sqrtf(dot3(a, a));
    a = (1.f / la) * a;
    const float pr = dot3(a, b);
    b = b - pr * a;
    float lb = sqrtf(dot3(b, b));
    b = (1.f / lb) * b;
    GS[k] = make_float4(la, lb, pr, 0.f);
    float3 nn = make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
    float su = in.s[2 * i], sv = in.s[2 * i + 1];
    float o = in.o[i];
    P[k] = make_float4(p.x, p.y, p.z, o);
    N4[k] = make_float4(nn.x, nn.y, nn.z, 0.f);
    FU[k] = make_float4(a.x, a.y, a.z, 1.f / su);
    FV[k] = make_float4(b.x, b.y, b.z, 1.f / sv);
    // BRDF coefficients (App. A): c_0 = 4 k a^d + (1-k) a^s, c_l = (1-k) a^s rho_l(s)
    float kd = in.k[i], s = in.shin[i];
    float rho[4] = {1.f, (s + 1.f) / (s + 2.f), s / (s + 3.f), (s + 1.f) * (s - 1.f) / ((s + 2.f) * (s + 4.f))};
    for (int l = 0; l < 4; ++l)
        for (int ch = 0; ch < 3; ++ch) {
            float ad = in.ad[3 * i + ch], as = in.as[3 * i + ch];
            float c = (l == 0) ? 4.f * kd * ad + (1.f - kd) * as : (1.f - kd) * as * rho[l];
            cl[(size_t)k * 12 + l * 3 + ch] = (l <= L) ? c : 0.f;
        }
    kk[k] = kd;
    // leaf box: cutoff ellipse of radius 3 (or 1 for the disc model), padded
    float rad = (alpha_model == RGS_ALPHA_DISC) ? 1.f : 3.f;
    float e[3] = {rad * sqrtf(su * su * a.x * a.x + sv * sv * b.x * b.x),
                  rad * sqrtf(su * su * a.y * a.y + sv * sv * b.y * b.y),
                  rad * sqrtf(su * su * a.z * a.z + sv * sv * b.z * b.z)};
    float pc[3] = {p.x, p.y, p.z};
    float *bx = boxes + (size_t)(n - 1 + k) * 6;
    for (int q = 0; q < 3; ++q) {
        float pad = e[q] * 1e-4f + 1e-6f * (fabsf(pc[q]) + e[q]);
        bx[q] = pc[q] - e[q] - pad;
        bx[3 + q] = pc[q] + e[q] + pad;
    }
    bool bad = !(isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(la) && la > 0.f && isfinite(lb) &&
                 lb > 0.f && isfinite(su) && su > 0.f && isfinite(sv) && sv > 0.f && isfinite(o) && isfinite(kd) &&
                 isfinite(s));
    for (int ch = 0; ch < 3; ++ch) bad |= !(isfinite(in.ad[3 * i + ch]) && isfinite(in.as[3 * i + ch]));
    if (bad) atomicAdd(&flags[FLAG_NONFINITE], 1);
}

// ---------------------------------------------------------------- Karras hierarchy
__device__ __forceinline__ int delta(const unsigned *keys, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    unsigned a = keys[i], b = keys[j];
    if (a != b) return __clz(a ^ b);
    return 32 + __clz((unsigned)i ^ (unsigned)j);
}

__global__ void k_karras(const unsigned *__restrict__ keys, int n, BvhNode *nodes, int *parent, int *visit) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    visit[i] = 0;
    int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = delta(keys, n, i, i - d);
    int lmax = 2;
    while (delta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = delta(keys, n, i, j);
    int s = 0, step = l;
    do {
        step = (step + 1) >> 1;
        if (delta(keys, n, i, i + (s + step) * d) > dnode) s += step;
    } while (step > 1);
    int gamma = i + s * d + min(d, 0);
    int left = (min(i, j) == gamma) ? ~gamma : gamma;
    int right = (max(i, j) == gamma + 1) ? ~(gamma + 1) : gamma + 1;
    nodes[i].d = make_int4(left, right, 0, 0);
    // parent array over all 2n-1 nodes: internal x -> x, leaf k -> n-1+k
    parent[left < 0 ? (n - 1 + ~left) : left] = i;
    parent[right < 0 ? (n - 1 + ~right) : right] = i;
}

// bottom-up refit: each leaf walks up; the second visitor of a node computes its box
__global__ void k_refit(int n, const BvhNode *__restrict__ nodes, const int *__restrict__ parent, int *visit,
                        float *boxes) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int x = parent[n - 1 + k];
    while (true) {
        __threadfence();
        if (atomicAdd(&visit[x], 1) == 0) return; // first arrival: the sibling will finish
        __threadfence();
        int4 c = nodes[x].d;
        const volatile float *bl = boxes + (size_t)(c.x < 0 ? (n - 1 + ~c.x) : c.x) * 6;
        const volatile float *br = boxes + (size_t)(c.y < 0 ? (n - 1 + ~c.y) : c.y) * 6;
        volatile float *bx = boxes + (size_t)x * 6;
        for (int q = 0; q < 3; ++q) {
            bx[q] = fminf(bl[q], br[q]);
            bx[3 + q] = fmaxf(bl[3 + q], br[3 + q]);
        }
        if (x == 0) return;
        x = parent[x];
    }
}

__global__ void k_pack(int n, BvhNode *nodes, const float *__restrict__ boxes) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int4 c = nodes[i].d;
    const float *bl = boxes + (size_t)(c.x < 0 ? (n - 1 + ~c.x) : c.x) * 6;
    const float *br = boxes + (size_t)(c.y < 0 ? (n - 1 + ~c.y) : c.y) * 6;
    nodes[i].a = make_float4(bl[0], bl[1], bl[2], bl[3]);
    nodes[i].b = make_float4(bl[4], bl[5], br[0], br[1]);
    nodes[i].c = make_float4(br[2], br[3], br[4], br[5]);
}

// ---------------------------------------------------------------- int -> int64 scan
constexpr int SCAN_BLOCK = 1024, SCAN_ITEMS = 4, SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

__global__ void k_scan_tiles(const int *__restrict__ cnt, long long *off, int n, long long *tile_sum) {
    __shared__ long long s[SCAN_BLOCK];
    int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    long long v[SCAN_ITEMS], t = 0;
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        v[q] = (base + q < n) ? cnt[base + q] : 0;
        t += v[q];
    }
    s[threadIdx.x] = t;
    __syncthreads();
    for (int o = 1; o < SCAN_BLOCK; o <<= 1) {
        long long x = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
        __syncthreads();
        s[threadIdx.x] += x;
        __syncthreads();
    }
    long long run = s[threadIdx.x] - t;
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        if (base + q < n) off[base + q] = run;
        run += v[q];
    }
    if (threadIdx.x == SCAN_BLOCK - 1) tile_sum[blockIdx.x] = s[SCAN_BLOCK - 1];
}

__global__ void k_scan_sums(long long *a, int m, long long *total_out) {
    __shared__ long long s[SCAN_BLOCK];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < m; base += SCAN_BLOCK) {
        int i = base + threadIdx.x;
        long long v = i < m ? a[i] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < SCAN_BLOCK; o <<= 1) {
            long long x = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
            __syncthreads();
            s[threadIdx.x] += x;
            __syncthreads();
        }
        if (i < m) a[i] = carry + s[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == SCAN_BLOCK - 1) carry += s[SCAN_BLOCK - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total_out = carry;
}

__global__ void k_scan_add(long long *off, int n, const long long *tile_off) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) off[i] += tile_off[i / SCAN_TILE];
}

} // namespace

int rgs_scan_tmp_size(int n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

rgs_status rgs_scan_counts(const int *cnt, long long *off, int n, long long *tmp, int tmp_cap, cudaStream_t st) {
    int tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles + 1 > tmp_cap) {
        rgs_set_error("scan workspace too small");
        return RGS_ERR_CAPACITY;
    }
    if (tiles > 0) {
        { ProfScope ps_("k_scan_tiles", st); k_scan_tiles<<<tiles, SCAN_BLOCK, 0, st>>>(cnt, off, n, tmp); }
        { ProfScope ps_("k_scan_sums", st); k_scan_sums<<<1, SCAN_BLOCK, 0, st>>>(tmp, tiles, off + n); }
        { ProfScope ps_("k_scan_add", st); k_scan_add<<<(n + 255) / 256, 256, 0, st>>>(off, n, tmp); }
    } else {
        RGS_CUDA(cudaMemsetAsync(off, 0, sizeof(long long), st));
    }
    RGS_LAUNCH("scan");
    return RGS_OK;
}

rgs_status rgs_scene_build_impl(rgs_scene *s, const rgs_surfels *in, const rgs_build_opts *o, cudaStream_t st) {
    const int n = in->n;
    if (n > s->cap) { // (re)allocate everything sized by n
        long long acct = 0;
        rgs_status r;
#define ALLOC(ptr, cnt)                                                                                                \
    if ((r = dev_alloc(&s->ptr, (size_t)(cnt), &acct)) != RGS_OK) {                                                   \
        s->cap = 0;                                                                                                    \
        return r;                                                                                                      \
    }
        ALLOC(P, n) ALLOC(N4, n) ALLOC(FU, n) ALLOC(FV, n) ALLOC(GS, n) ALLOC(cl, (size_t)n * 12) ALLOC(kk, n) ALLOC(uid, n)
        ALLOC(inv, n) ALLOC(nodes, n > 1 ? n - 1 : 1) ALLOC(boxes, (size_t)(2 * n - 1) * 6) ALLOC(parent, 2 * n)
        ALLOC(visit, n) ALLOC(keys, n) ALLOC(keys_alt, n) ALLOC(vals, n) ALLOC(vals_alt, n)
#undef ALLOC
        s->hist_cap = 256 * ((n + SORT_TILE - 1) / SORT_TILE);
        if ((r = dev_alloc(&s->hist, (size_t)s->hist_cap)) != RGS_OK) return r;
        if (!s->bounds && (r = dev_alloc(&s->bounds, 6)) != RGS_OK) return r;
        if (!s->eps_plane && (r = dev_alloc(&s->eps_plane, 1)) != RGS_OK) return r;
        if (!s->flags && (r = dev_alloc(&s->flags, FLAG_COUNT)) != RGS_OK) return r;
        s->cap = n;
    }
    s->n = n;
    s->L = in->sh_degree;
    s->nc = (in->sh_degree + 1) * (in->sh_degree + 1);
    s->alpha_model = o ? o->alpha_model : RGS_ALPHA_GAUSS;
    RGS_CUDA(cudaMemsetAsync(s->flags, 0, sizeof(int) * FLAG_COUNT, st));

    { ProfScope ps_("k_init_bounds", st); k_init_bounds<<<1, 32, 0, st>>>(s->bounds); }
    int nb = min((n + 255) / 256, 1024);
    { ProfScope ps_("k_bounds", st); k_bounds<<<nb, 256, 0, st>>>(in->p, n, s->bounds); }
    { ProfScope ps_("k_morton", st); k_morton<<<(n + 255) / 256, 256, 0, st>>>(in->p, n, s->bounds, s->keys, s->vals, s->eps_plane); }
    RGS_LAUNCH("morton");
    // 4 x 8-bit stable LSD passes; the result lands back in keys/vals
    int tiles = (n + SORT_TILE - 1) / SORT_TILE;
    unsigned *ka = s->keys, *kb = s->keys_alt;
    int *va = s->vals, *vb = s->vals_alt;
    for (int pass = 0; pass < 4; ++pass) {
        int shift = pass * 8;
        { ProfScope ps_("k_radix_hist", st); k_radix_hist<<<tiles, SORT_THREADS, 0, st>>>(ka, n, shift, tiles, s->hist); }
        { ProfScope ps_("k_scan_single", st); k_scan_single<<<1, 1024, 0, st>>>(s->hist, 256 * tiles); }
        { ProfScope ps_("k_radix_scatter", st); k_radix_scatter<<<tiles, SORT_THREADS, 0, st>>>(ka, va, kb, vb, n, shift, tiles, s->hist); }
        unsigned *tk = ka;
        ka = kb;
        kb = tk;
        int *tv = va;
        va = vb;
        vb = tv;
    }
    RGS_LAUNCH("radix sort");
    // after an even number of passes ka == keys, va == vals
    { ProfScope ps_("k_gather", st); k_gather<<<(n + 127) / 128, 128, 0, st>>>(*in, n, s->L, s->alpha_model, va, s->P, s->N4, s->FU, s->FV, s->GS, s->cl,
                                              s->kk, s->uid, s->inv, s->boxes, s->flags); }
    RGS_LAUNCH("gather");
    if (n > 1) {
        { ProfScope ps_("k_karras", st); k_karras<<<(n - 1 + 255) / 256, 256, 0, st>>>(ka, n, s->nodes, s->parent, s->visit); }
        { ProfScope ps_("k_refit", st); k_refit<<<(n + 255) / 256, 256, 0, st>>>(n, s->nodes, s->parent, s->visit, s->boxes); }
        { ProfScope ps_("k_pack", st); k_pack<<<(n - 1 + 255) / 256, 256, 0, st>>>(n, s->nodes, s->boxes); }
        RGS_LAUNCH("bvh");
    }
    if (o && o->check_finite) {
        int flags[FLAG_COUNT];
        RGS_CUDA(cudaMemcpyAsync(flags, s->flags, sizeof flags, cudaMemcpyDeviceToHost, st));
        RGS_CUDA(cudaStreamSynchronize(st));
        if (flags[FLAG_NONFINITE]) {
            rgs_set_error("%d surfels have non-finite or degenerate parameters", flags[FLAG_NONFINITE]);
            return RGS_ERR_NONFINITE;
        }
    }
    return RGS_OK;
}
