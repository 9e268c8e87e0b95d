// The adjoint's opacity gather on the tensor cores as a sampled dense-dense product (many
// right-hand sides; the opacity term of the adjoint, Sec. 6 and Eq. final_dL_dE).
//
// For a pairing (v^(a), B^(b)) every stored hit h (ray r of receiver i, source j) takes
//     g_h (+)= sum_c y_r[c] s_h[c],
//     y_r[c] = (pi/nd) o_i sum_k c_{i,l(k),ch(c)} Y_k(R_i d_r) v_i[c][k]   (one row per ray),
//     s_h[c] = sum_m Y_m(-d_r) B_j[c][m],
// that is g_h = sum_m Y_m(-d_r) W_h[m] with W_h[m] = sum_c y_r[c] B_j[c][m]: a product of the
// hits' y rows with their source's rows, of which only the (hit, own source) entries are kept.
// y is formed once per ray (BF16, in passes of at most 320 columns), then per source tile
// (8 consecutive sources, the adjoint's hit tiles) and block of 128 of its hits
//     D[h][(sigma, m)] = sum_c y_{r_h}[c] B_{8t+sigma}[c][m]          (128 x 128, K = columns)
// runs on tcgen05 (M = N = 128, K = 16 per MMA, FP32 accumulator in TMEM): A is the block's
// 128 y rows, gathered into shared memory by cp.async, B the tile's 8 source rows, converted
// to BF16 once per tile and kept in shared memory for all its blocks.  The epilogue keeps
// the 16 entries of each hit's own source and finishes g_h = Y(-d)^T D[h][(sigma_h, .)].
// The tensor work per hit is 8x the kept part (all 8 sources of the tile are formed), but
// at 128 x 128 x 16 per instruction it stays below the cost of gathering the y rows, 2 bytes
// per hit and column, which bounds the kernel (the SM's L1/TEX data pipe).  The sums stay in
// the tiles' hit order (coalesced) and reach the record slots after the last pairing.
//
// Roles (one persistent CTA per SM, source tiles round-robin):
//   warps 0..3   epilogue (TMEM lane quarters 0..3: one hit row per thread)
//   warp  4      TMEM owner and MMA issuer (one lane)
//   warps 5..12  producers in 4 groups of 2 warps: group q copies the block's 128 y rows of
//                every stage s = q (mod 4) of a ring of 64-column stages; all 8 load the
//                tile's source rows
// Every mbarrier wait is bounded; a wait that runs out sets the transport's error flag and
// every role leaves its loop (the host then reports RGS_ERR_TIMEOUT).
#include <algorithm>

#include "rgs_internal.cuh"
#include "rgs_tc.cuh"

namespace {

constexpr int OP_EPI = 4;                   // epilogue warps
constexpr int OP_MW = 4;                    // the MMA warp
constexpr int OP_P0 = 5;                    // first producer warp
constexpr int OP_NP = 8;                    // producer warps
constexpr int OP_THREADS = (OP_P0 + OP_NP) * 32;
constexpr int OP_ROWS = 128;                // hits per block (the MMA's M)
constexpr int OP_SC = 64;                   // columns per stage (pass widths are multiples of it)
constexpr int OP_NST = 8;                   // most stages in the ring
constexpr int OP_NG = 4;                    // producer groups (stage s belongs to group s mod OP_NG)
constexpr int OP_WPG = OP_NP / OP_NG;       // warps per group
constexpr int OP_RPT = 8 / OP_WPG;          // 16-row groups per thread
constexpr int OP_KW_MAX = 320;              // columns per pass
constexpr uint64_t OP_DRAIN_NS = 1000000000ull;

struct OpaArgs {
    int ntiles, n, C, c0, kw; // this pass's columns [c0, c0 + kw), kw a multiple of 64
    int nst;                  // stages in the ring (64 columns of the block's 128 rows each)
    const long long *hoff;    // [ntiles + 1] hits of each source tile
    const float4 *hd;         // per hit: direction d, weight (source slot sigma in its 3 low bits)
    const uint32_t *hray;     // per hit: its ray
    const __nv_bfloat16 *yr;  // [n_rays][kw] y of every ray, this pass's columns (pads 0)
    const float *Bsrc;        // B^(b), FP32 [n][C][16]
    float *gt;                // per hit, in tile order: g_h (the record slots receive it at the end)
    int first;                // write g_h instead of adding to it
    int *flags;
    unsigned long long wait_ns;
};

__device__ __forceinline__ bool op_aborted(const int *f) { return *(volatile const int *)f != 0; }

// where = warp * 16 + wait site; the first failure's site and block count are kept
__device__ __forceinline__ void op_fail(const OpaArgs &g, int *abort_flag, int where, long long count) {
    atomicExch(abort_flag, 1);
    if (atomicAdd(&g.flags[FLAG_TC_TIMEOUT], 1) == 0) {
        g.flags[FLAG_TC_TIMEOUT + 1] = where;
        g.flags[FLAG_TC_TIMEOUT + 2] = (int)count;
    }
}

// 16 bytes global -> shared, allocating in L1: the two lanes that copy the two halves of a
// 32-byte sector then share one sector fetch (the L2-only form fetched the sector twice)
__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *gptr) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(gptr) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// 32 lanes x 32 consecutive 32-bit TMEM columns into registers (warp-collective)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
                   "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
                   "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

// a warp-uniform bounded wait by lane 0, its outcome broadcast
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    bool ok = true;
    if ((threadIdx.x & 31) == 0) ok = tc::bar_wait(bar, parity, limit_ns);
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok;
}

__global__ void __launch_bounds__(OP_THREADS, 1) k_tc_opa(OpaArgs g) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_full[OP_NST], bar_empty[OP_NST];
    __shared__ __align__(8) uint64_t bar_dfull[2], bar_dempty[2], bar_bfull, bar_bfree, bar_drain;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int spb = g.kw / OP_SC;                // stages per block
    constexpr int sc = OP_SC, ksteps = OP_SC / 16; // columns and K = 16 steps of a stage
    constexpr uint32_t stage_bytes = (uint32_t)sc * OP_ROWS * 2u;
    const int nst = g.nst;
    unsigned char *btile = smem + (size_t)nst * stage_bytes;
    if (threadIdx.x == 0) {
        for (int s = 0; s < nst; ++s) {
            tc::bar_init(&bar_full[s], OP_WPG);
            tc::bar_init(&bar_empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::bar_init(&bar_dfull[b], 1);
            tc::bar_init(&bar_dempty[b], OP_EPI);
        }
        tc::bar_init(&bar_bfull, OP_NP);
        tc::bar_init(&bar_bfree, 1);
        tc::bar_init(&bar_drain, 1);
        abort_flag = 0;
        tc::bar_init_fence();
    }
    if (warp == OP_MW) tc::tmem_alloc(&tmem_slot, 256);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp >= OP_P0) {
        // ------------------------------------------------------------ producers
        // groups of OP_WPG warps own every OP_NG-th stage: a group copies its stage's rows, waits
        // for its own copies, makes them visible to the tensor core and signals, while the
        // other groups' stages are in flight (with one group whose threads kept several stages
        // in flight, the proxy fence before each signal took 46 % of the producers' time, as
        // if it waited for the later stages' copies too)
        const int p = warp - OP_P0, grp = p / OP_WPG, wig = p % OP_WPG;
        const int hl = lane & 15, half = lane >> 4;
        const uint32_t sbase = tc::smem_addr(smem);
        uint32_t srow[OP_RPT];
#pragma unroll
        for (int q = 0; q < OP_RPT; ++q) {
            const int row = 16 * (wig + OP_WPG * q) + hl; // this thread's rows of the block's 128
            srow[q] = (uint32_t)(row >> 3) * 256u + (uint32_t)half * 128u + (uint32_t)(row & 7) * 16u;
        }
        long long gs = 0; // stages of every group so far
        int tl = 0;       // tiles with hits seen
        for (int t = blockIdx.x; t < g.ntiles && !op_aborted(&abort_flag); t += gridDim.x) {
            const long long h0 = g.hoff[t], nh = g.hoff[t + 1] - h0;
            if (nh <= 0) continue;
            // the tile's source rows, once the previous tile's MMAs are done
            if (tl > 0 && !warp_wait(&bar_bfree, (uint32_t)((tl - 1) & 1), g.wait_ns)) {
                if (lane == 0) op_fail(g, &abort_flag, 16 * warp + 1, gs);
                break;
            }
            {
                // element (n = sigma * 16 + m, c) at (c / 16) * 4096 + (n / 8) * 256 + ((c / 8) % 2) * 128
                // + (n % 8) * 16 + (c % 8) * 2: the K-major core-matrix layout, 16 columns per 4 KB
                const int ntask = OP_ROWS * (g.kw / 8);
                for (int q = p * 32 + lane; q < ntask; q += OP_NP * 32) {
                    const int n = q & 127, cg = q >> 7;
                    const int sigma = n >> 4, m = n & 15;
                    const int src = t * 8 + sigma;
                    float x[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int c = g.c0 + cg * 8 + u;
                        x[u] = (src < g.n && c < g.C) ? __ldg(&g.Bsrc[((size_t)src * g.C + c) * 16 + m]) : 0.f;
                    }
                    const uint4 v = make_uint4(tc::pack_bf16(x[0], x[1]), tc::pack_bf16(x[2], x[3]),
                                               tc::pack_bf16(x[4], x[5]), tc::pack_bf16(x[6], x[7]));
                    tc::sts128(tc::smem_addr(btile) + (uint32_t)(cg >> 1) * 4096u + (uint32_t)(n >> 3) * 256u +
                                   (uint32_t)(cg & 1) * 128u + (uint32_t)(n & 7) * 16u,
                               v);
                }
                tc::fence_async_smem();
                __syncwarp();
                if (lane == 0) tc::bar_arrive(&bar_bfull);
            }
            ++tl;
            uint32_t ray_next[OP_RPT];
#pragma unroll
            for (int q = 0; q < OP_RPT; ++q) {
                const int row = 16 * (wig + OP_WPG * q) + hl;
                ray_next[q] = row < nh ? __ldg(&g.hray[h0 + row]) : 0u;
            }
            for (long long b0 = 0; b0 < nh && !op_aborted(&abort_flag); b0 += OP_ROWS) {
                uint32_t ray[OP_RPT];
#pragma unroll
                for (int q = 0; q < OP_RPT; ++q) {
                    const int row = 16 * (wig + OP_WPG * q) + hl;
                    ray[q] = ray_next[q];
                    if (b0 + OP_ROWS + row < nh) ray_next[q] = __ldg(&g.hray[h0 + b0 + OP_ROWS + row]); // the next block's
                }
                bool ok = true;
                for (int st = 0; st < spb; ++st, ++gs) {
                    if ((int)(gs % OP_NG) != grp) continue;
                    const int s = (int)(gs % nst);
                    if (!warp_wait(&bar_empty[s], (uint32_t)(((gs / nst) & 1) ^ 1), g.wait_ns)) {
                        if (lane == 0) op_fail(g, &abort_flag, 16 * warp + 2, gs);
                        ok = false;
                        break;
                    }
                    const uint32_t dst = sbase + (uint32_t)s * stage_bytes;
#pragma unroll
                    for (int q = 0; q < OP_RPT; ++q) {
                        const int row = 16 * (wig + OP_WPG * q) + hl;
                        if (b0 + row < nh) {
                            const __nv_bfloat16 *src = g.yr + (size_t)ray[q] * g.kw + half * 8 + st * sc;
#pragma unroll
                            for (int ks = 0; ks < ksteps; ++ks) cp_async16(dst + srow[q] + (uint32_t)ks * 4096u, src + ks * 16);
                        }
                    }
                    cp_async_commit();
                    cp_async_wait<0>();
                    tc::fence_async_smem();
                    __syncwarp();
                    if (lane == 0) tc::bar_arrive(&bar_full[s]);
                }
                if (!ok) break;
            }
        }
        cp_async_wait<0>();
    } else if (warp == OP_MW) {
        // ------------------------------------------------------------ MMA issuer
        long long gs = 0, bc = 0;
        int tl = 0;
        const uint32_t id = tc::idesc_bf16(OP_ROWS, 128);
        const uint32_t sbase = tc::smem_addr(smem), bbase = tc::smem_addr(btile);
        for (int t = blockIdx.x; t < g.ntiles && !op_aborted(&abort_flag); t += gridDim.x) {
            const long long nh = g.hoff[t + 1] - g.hoff[t];
            if (nh <= 0) continue;
            if (lane == 0) {
                bool ok = tc::bar_wait(&bar_bfull, (uint32_t)(tl & 1), g.wait_ns);
                if (!ok) op_fail(g, &abort_flag, 16 * warp + 3, bc);
                tc::fence_after();
                for (long long b0 = 0; b0 < nh && ok && !op_aborted(&abort_flag); b0 += OP_ROWS, ++bc) {
                    const int buf = (int)(bc & 1);
                    if (bc >= 2 && !tc::bar_wait(&bar_dempty[buf], (uint32_t)(((bc >> 1) - 1) & 1), g.wait_ns)) {
                        op_fail(g, &abort_flag, 16 * warp + 4, bc);
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    const uint32_t d = tmem + (uint32_t)(buf * 128);
                    for (int st = 0; st < spb; ++st, ++gs) {
                        const int s = (int)(gs % nst);
                        if (!tc::bar_wait(&bar_full[s], (uint32_t)((gs / nst) & 1), g.wait_ns)) {
                            op_fail(g, &abort_flag, 16 * warp + 5, bc);
                            ok = false;
                            break;
                        }
                        tc::fence_after();
                        for (int ks = 0; ks < ksteps; ++ks)
                            tc::mma_bf16(d, tc::sdesc(sbase + (uint32_t)s * stage_bytes + (uint32_t)ks * 4096u),
                                         tc::sdesc(bbase + (uint32_t)(st * ksteps + ks) * 4096u), id,
                                         (st | ks) ? 1u : 0u);
                        tc::mma_commit(&bar_empty[s]);
                    }
                    if (!ok) break;
                    tc::mma_commit(&bar_dfull[buf]);
                }
                tc::mma_commit(&bar_bfree);
            }
            __syncwarp();
            bc = __shfl_sync(0xffffffffu, bc, 0);
            gs = __shfl_sync(0xffffffffu, gs, 0);
            ++tl;
        }
        if (lane == 0) {
            tc::mma_commit(&bar_drain);
            tc::bar_wait(&bar_drain, 0u, OP_DRAIN_NS);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        const int quarter = warp; // TMEM lanes 32 quarter .. 32 quarter + 31
        const int row = quarter * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
        long long bc = 0;
        // a block's hit data (direction and, when adding, the running g_h, both in the tile's
        // hit order) is fetched one block ahead, so that its latency overlaps the previous block
        struct Hit {
            float4 d4;
            float gold;
        };
        auto fetch = [&](long long e, bool valid) {
            Hit x{make_float4(0.f, 0.f, 1.f, 0.f), 0.f};
            if (valid) {
                x.d4 = __ldg(&g.hd[e]);
                if (!g.first) x.gold = g.gt[e];
            }
            return x;
        };
        for (int t = blockIdx.x; t < g.ntiles && !op_aborted(&abort_flag); t += gridDim.x) {
            const long long h0 = g.hoff[t], nh = g.hoff[t + 1] - h0;
            if (nh <= 0) continue;
            bool ok = true;
            Hit nxt = fetch(h0 + row, row < nh);
            for (long long b0 = 0; b0 < nh && !op_aborted(&abort_flag); b0 += OP_ROWS, ++bc) {
                const int buf = (int)(bc & 1);
                const bool valid = b0 + row < nh;
                const Hit cur = nxt;
                if (b0 + OP_ROWS < nh) nxt = fetch(h0 + b0 + OP_ROWS + row, b0 + OP_ROWS + row < nh);
                const int sigma = (int)(__float_as_uint(cur.d4.w) & 7u);
                float Yo[16];
                sh_eval<16>(make_float3(-cur.d4.x, -cur.d4.y, -cur.d4.z), Yo);
                if (!warp_wait(&bar_dfull[buf], (uint32_t)((bc >> 1) & 1), g.wait_ns)) {
                    if (lane == 0) op_fail(g, &abort_flag, 16 * warp + 6, bc);
                    ok = false;
                    break;
                }
                tc::fence_after();
                float val = 0.f;
#pragma unroll 1
                for (int sg = 0; sg < 8; sg += 2) {
                    float P[32];
                    tmem_ld32(trow + (uint32_t)(buf * 128 + sg * 16), P);
                    float s0 = 0.f, s1 = 0.f;
#pragma unroll
                    for (int m = 0; m < 16; ++m) {
                        s0 = fmaf(Yo[m], P[m], s0);
                        s1 = fmaf(Yo[m], P[16 + m], s1);
                    }
                    val = (sg == sigma) ? s0 : ((sg + 1 == sigma) ? s1 : val);
                }
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::bar_arrive(&bar_dempty[buf]);
                if (valid) g.gt[h0 + b0 + row] = g.first ? val : cur.gold + val;
            }
            if (!ok) break;
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == OP_MW) tc::tmem_dealloc(tmem, 256);
}

// y_r[c] for the pass columns [c0, c0 + kw) of every ray of receiver i (one block each):
// (pi/nd) o_i sum_k c_{i,l(k),ch(c)} Y_k(R_i d_r) v_i[c][k], BF16, columns past C zero.  A
// thread holds one column pair's 2 x 16 factors in registers and walks the receiver's rays,
// whose Y(R_i d) the block first tabulates in shared memory.
constexpr int YR_MAX_RAYS = 512;
__global__ void __launch_bounds__(OP_KW_MAX / 2) k_tc_opa_y(SceneDev sc, RaysDev rays, int C, int c0, int kw,
                                                             const float *__restrict__ v, __nv_bfloat16 *yr) {
    __shared__ __align__(16) float Ysh[YR_MAX_RAYS][16];
    const int i = blockIdx.x, nd = rays.nd;
    const float3 n = f3(sc.N4[i]);
    for (int q = threadIdx.x; q < nd; q += blockDim.x) {
        float Y[16];
        sh_eval<16>(reflect_n(n, f3(rays.dir[(size_t)i * nd + q])), Y);
#pragma unroll
        for (int k = 0; k < 16; ++k) Ysh[q][k] = Y[k];
    }
    const int cp = threadIdx.x, c = 2 * cp; // this thread's columns c0 + c, c0 + c + 1
    const bool live = c < kw;
    float u0[16], u1[16];
    {
        const float w = alpha_center(sc, i) * (3.14159265358979f / (float)nd);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int ca = c0 + c, cb = ca + 1;
            u0[k] = (live && ca < C) ? w * __ldg(&sc.cl[(size_t)i * 12 + band_of(k) * 3 + ca % 3]) * __ldg(&v[((size_t)i * C + ca) * 16 + k]) : 0.f;
            u1[k] = (live && cb < C) ? w * __ldg(&sc.cl[(size_t)i * 12 + band_of(k) * 3 + cb % 3]) * __ldg(&v[((size_t)i * C + cb) * 16 + k]) : 0.f;
        }
    }
    __syncthreads();
    if (!live) return;
    __nv_bfloat16 *out = yr + (size_t)i * nd * kw + c;
    for (int q = 0; q < nd; ++q) {
        const float4 *Yq = reinterpret_cast<const float4 *>(Ysh[q]);
        float y0 = 0.f, y1 = 0.f;
#pragma unroll
        for (int k4 = 0; k4 < 4; ++k4) {
            const float4 yk = Yq[k4];
            y0 = fmaf(u0[4 * k4], yk.x, fmaf(u0[4 * k4 + 1], yk.y, fmaf(u0[4 * k4 + 2], yk.z, fmaf(u0[4 * k4 + 3], yk.w, y0))));
            y1 = fmaf(u1[4 * k4], yk.x, fmaf(u1[4 * k4 + 1], yk.y, fmaf(u1[4 * k4 + 2], yk.z, fmaf(u1[4 * k4 + 3], yk.w, y1))));
        }
        *reinterpret_cast<__nv_bfloat162 *>(out + (size_t)q * kw) = __floats2bfloat162_rn(y0, y1);
    }
}

// the record slots receive the tile-ordered sums
__global__ void k_tc_opa_scatter(long long H, const uint32_t *__restrict__ hslot, const float *__restrict__ gt,
                                 float *gh) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < H; e += (long long)gridDim.x * blockDim.x)
        gh[__ldg(&hslot[e])] = __ldg(&gt[e]);
}

} // namespace

// columns per pass that the y buffer may take (a multiple of 64, at most 320; 0: none fits):
// at most 30 % of the free device memory (48 GB at most) and, under a memory budget, half
// of what the budget leaves beside the transport's own buffers
int rgs_tc_opa_pass_cols(const rgs_transport *t) {
    const long long n_rays = (long long)t->n * t->nd;
    const int full = std::min(OP_KW_MAX, (t->C + OP_SC - 1) / OP_SC * OP_SC);
    double budget = std::min(0.3 * (double)pool_available_bytes(), 48e9);
    if (t->mem_budget > 0) budget = std::min(budget, 0.5 * (double)(t->mem_budget - t->device_bytes));
    int kw = (int)(budget / (2.0 * (double)std::max(n_rays, 1ll)) / OP_SC) * OP_SC;
    return t->nd > YR_MAX_RAYS ? 0 : std::min(full, kw);
}

// g_h (+)= the pairing of v (FP32 adjoint iterate) with B (FP32 iterate) over every hit of the
// adjoint's source tiles, summed in the tiles' hit order; first: the first pairing, which
// writes the sums; last: the last one, after which the record slots receive them
rgs_status rgs_tc_opacity_sddmm(rgs_transport *t, const float *v, const float *B, bool first, bool last,
                                cudaStream_t st) {
    RgsTcAdjHits h{};
    if (!rgs_tc_adj_hits(t, &h)) {
        rgs_set_error("tensor-core opacity gather: the adjoint's hit tiles are not built");
        return RGS_ERR_STATE;
    }
    if (t->nd > YR_MAX_RAYS) {
        rgs_set_error("tensor-core opacity gather: more than %d rays per surfel", YR_MAX_RAYS);
        return RGS_ERR_ARG;
    }
    const int kw = rgs_tc_opa_pass_cols(t);
    if (kw < OP_SC) {
        rgs_set_error("tensor-core opacity gather: no memory for one 64-column pass of y");
        return RGS_ERR_OOM;
    }
    static int num_sms = 0, optin = 0;
    if (!num_sms) {
        int dev = 0;
        RGS_CUDA(cudaGetDevice(&dev));
        RGS_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
        RGS_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    }
    cudaFuncAttributes fa{};
    RGS_CUDA(cudaFuncGetAttributes(&fa, k_tc_opa));
    // stages of 64 columns x 128 rows, as many as fit (at most 8) beside the tile's source
    // rows (kw x 256 bytes)
    const size_t stage_bytes = (size_t)OP_SC * OP_ROWS * 2, room = (size_t)optin - fa.sharedSizeBytes - 256;
    int nst = (int)std::min<size_t>(OP_NST, room > (size_t)kw * 256 ? (room - (size_t)kw * 256) / stage_bytes : 0);
    nst -= nst % OP_NG; // a stage slot keeps its producer group
    if (nst < OP_NG) {
        rgs_set_error("tensor-core opacity gather: %d columns per pass leave no room for the stage ring", kw);
        return RGS_ERR_ARG;
    }
    const size_t smem = (size_t)nst * stage_bytes + (size_t)kw * 256;
    RGS_CUDA(cudaFuncSetAttribute(k_tc_opa, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long long n_rays = (long long)t->n * t->nd;
    __nv_bfloat16 *yr = nullptr;
    rgs_status r;
    if ((r = pool_alloc(&yr, (size_t)n_rays * kw, st)) != RGS_OK) return r;
    struct Rel {
        __nv_bfloat16 *p;
        cudaStream_t st;
        ~Rel() { pool_release(p, st); }
    } rel{yr, st};
    const SceneDev sd = t->sc->dev();
    const RaysDev rd = t->rays();
    OpaArgs a{};
    a.ntiles = h.ntiles;
    a.n = t->n;
    a.C = t->C;
    a.kw = kw;
    a.hoff = h.hoff;
    a.hd = h.hd;
    a.hray = h.hray;
    a.yr = yr;
    a.Bsrc = B;
    a.gt = h.gt;
    a.flags = t->flags;
    a.wait_ns = t->tc_wait_ns;
    a.nst = nst;
    const int grid = std::max(1, std::min(h.ntiles, num_sms));
    for (int c0 = 0; c0 < t->C; c0 += kw) {
        { ProfScope ps_("k_tc_opa_y", st); k_tc_opa_y<<<t->n, (kw / 2 + 31) / 32 * 32, 0, st>>>(sd, rd, t->C, c0, kw, v, yr); }
        RGS_LAUNCH("opacity gather: y rows");
        a.c0 = c0;
        a.first = (first && c0 == 0) ? 1 : 0;
        { ProfScope ps_("k_tc_opa", st); k_tc_opa<<<grid, OP_THREADS, smem, st>>>(a); }
        RGS_LAUNCH("tensor-core opacity gather");
    }
    if (last) {
        ProfScope ps_("k_tc_opa_scatter", st);
        k_tc_opa_scatter<<<(unsigned)std::min<long long>((h.n_hits + 255) / 256, 8192), 256, 0, st>>>(h.n_hits, h.hslot, h.gt, t->gh);
        RGS_LAUNCH("opacity gather: record slots");
    }
    return RGS_OK;
}
