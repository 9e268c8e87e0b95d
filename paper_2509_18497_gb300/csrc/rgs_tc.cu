// Tensor-core bounce contraction (many right-hand sides, Eq. final-radiosity; Sec. 7):
//   Q_i = sum_j G_ij B_j,   G_ij = sum_{r, h : j_h = j} a_rh Y(R_i d_r) Y(-d_r)^T   (16 x 16)
// and its transpose for the adjoint (Eq. final_dL_dE):
//   (K^T v)_j = sum_i G_ij^T y_i,   y_i = o_i c_i (x) v_i.
//
// The stored hit records are regrouped once per transport into "pair tiles": 8 consecutive
// receivers (Morton order) and, for each source j any of them sees, the hits of that
// (tile, source) group, sorted by receiver and ray.  Per group the CTA
//   * bulk-copies the source's BF16 row block (C columns x 16 coefficients, stored in the
//     core-matrix layout of rgs_tc.cuh) from global into shared memory (TMA engine),
//   * forms the 8 receivers' 16 x 16 blocks G_ij as one 128 x 16 operand from the group's
//     hits (FP32, rounded to BF16; rows of receivers that do not see j are zero),
//   * issues D[128 x C] += A[128 x 16] * B_j^T with tcgen05 (accumulator in TMEM).
// After the tile's last group D holds Q^T of its 8 receivers (rows = receiver x SH
// coefficient), and the epilogue forms B = S + o c (x) (pi/nd) Q, its BF16 copies and the FP64
// residual norm.  The adjoint is the same kernel over "source tiles" (8 consecutive
// sources, groups = receivers seeing them) with the roles of Y(R_i d) and Y(-d) swapped.
// The residual-correction bounce splits both operands into BF16 high and low parts and
// accumulates the three products hi*hi + hi*lo + lo*hi (FP32-level accuracy).
//
// Roles (one persistent CTA per SM, tiles assigned round-robin):
//   warp 0      producer: group list, bulk copies of source rows into a ring of stages
//   warp 1      TMEM owner and MMA issuer (one elected lane)
//   warps 2..9  operand builders (one group each, round-robin) and epilogue (TMEM -> HBM)
// Every wait on an mbarrier is bounded; a wait that runs out sets an error flag and the
// kernel returns (the host reports RGS_ERR_TIMEOUT), so a broken partner cannot hang the GPU.
#include <algorithm>
#include <vector>

#include "rgs_internal.cuh"
#include "rgs_tc.cuh"

namespace {

constexpr int TC_R = 8;           // receivers (or sources) per tile: 8 x 16 coefficients = M 128
constexpr int TC_NB = 16;         // builder warps (as many as stages take part)
constexpr int TC_NP = 2;           // producer warps (each owns every TC_NP-th stage)
constexpr int TC_THREADS = (TC_NP + 1 + TC_NB) * 32; // producers, the MMA warp, the builders
constexpr int TC_GPS_MAX = 4;      // groups per pipeline stage
constexpr int TC_CT_STAGES = 4;    // pipeline stages of the contraction
constexpr int TC_MAX_STAGES = 16;  // one per builder
constexpr int TC_HCAP = 20;        // hit records per group (longer (tile, source) runs are split)
constexpr int TC_CHUNK = 512;     // columns per pass (TMEM holds 512 FP32 columns)
constexpr uint64_t TC_DRAIN_NS = 1000000000ull; // wait for in-flight copies and MMAs at exit

// ------------------------------------------------------------------ SH as monomials
// Y_k(v) = sum_q TC_SH[k][q] m_q(v) with the 20 monomials of degree <= 3
// (1, x, y, z, xy, yz, zz, xz, xx, yy, xxy, yyy, xyz, yzz, zzz, xzz, xxz, yyz, xxx, xyy):
// the real orthonormal SH with the Condon-Shortley phase (the polynomials of sh_eval), so
// that a lane can evaluate "its" coefficient k with the same instructions as every other.
__device__ const float TC_SH[16][20] = {
    {0.28209479177387814f},
    {0, 0, -0.4886025119029199f},
    {0, 0, 0, 0.4886025119029199f},
    {0, -0.4886025119029199f},
    {0, 0, 0, 0, 1.0925484305920792f},
    {0, 0, 0, 0, 0, -1.0925484305920792f},
    {-0.31539156525252005f, 0, 0, 0, 0, 0, 3.f * 0.31539156525252005f},
    {0, 0, 0, 0, 0, 0, 0, -1.0925484305920792f},
    {0, 0, 0, 0, 0, 0, 0, 0, 0.5462742152960396f, -0.5462742152960396f},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, -3.f * 0.5900435899266435f, 0.5900435899266435f},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 2.890611442640554f},
    {0, 0, 0.4570457994644658f, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, -5.f * 0.4570457994644658f},
    {0, 0, 0, -3.f * 0.3731763325901154f, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 5.f * 0.3731763325901154f},
    {0, 0.4570457994644658f, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, -5.f * 0.4570457994644658f},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1.445305721320277f, -1.445305721320277f},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, -0.5900435899266435f, 3.f * 0.5900435899266435f},
};

__device__ __forceinline__ float sh_mono(const float (&cf)[20], float3 v) {
    const float x = v.x, y = v.y, z = v.z;
    const float xx = x * x, yy = y * y, zz = z * z, xy = x * y, yz = y * z, xz = x * z;
    float s = cf[0];
    s = fmaf(cf[1], x, s);
    s = fmaf(cf[2], y, s);
    s = fmaf(cf[3], z, s);
    s = fmaf(cf[4], xy, s);
    s = fmaf(cf[5], yz, s);
    s = fmaf(cf[6], zz, s);
    s = fmaf(cf[7], xz, s);
    s = fmaf(cf[8], xx, s);
    s = fmaf(cf[9], yy, s);
    s = fmaf(cf[10], xx * y, s);
    s = fmaf(cf[11], yy * y, s);
    s = fmaf(cf[12], xy * z, s);
    s = fmaf(cf[13], y * zz, s);
    s = fmaf(cf[14], z * zz, s);
    s = fmaf(cf[15], x * zz, s);
    s = fmaf(cf[16], xx * z, s);
    s = fmaf(cf[17], yy * z, s);
    s = fmaf(cf[18], xx * x, s);
    s = fmaf(cf[19], x * yy, s);
    return s;
}

// ------------------------------------------------------------------ kernel arguments
struct TcArgs {
    int adjoint;   // 0: forward over receiver tiles, 1: transpose over source tiles
    int split;     // 1: hi/lo operands, three MMAs per column piece
    int n, C, Cp, nd, ntiles, nchunks, stages, stage_shift, gps;
    uint32_t stage_bytes, rows_bytes, a_bytes; // a stage; the rows and the operand of one of its groups
    const long long *hoff; // [ntiles + 1] first hit of each tile
    const long long *goff; // [ntiles + 1] first group of each tile
    const int2 *grp;       // per group: (other entity, first hit relative to its tile)
    const float4 *hd;      // per hit: ray direction d, weight a (tile slot p in a's 3 low bits)
    const __nv_bfloat16 *rows_hi, *rows_lo; // [n][Cp x 16] blocked BF16 rows of the other entities
    const float4 *N4, *P;
    const float *cl;
    int alpha_model;
    float w; // pi / nd
    // forward epilogue
    const float *S, *Bprev;
    float *Qout, *Bout;
    __nv_bfloat16 *Bout16;           // row layout copy (stride 16 per column)
    __nv_bfloat16 *Bblk, *Bblk_lo;   // blocked copies (lo: optional)
    double *norm2;
    // adjoint epilogue
    float *vout, *u;
    __nv_bfloat16 *yblk;
    int *flags;
    unsigned long long wait_ns; // limit of every pipeline wait
};

struct __align__(16) StageMeta {
    float4 nrm; // adjoint: the group's receiver normal
    int other, cnt;
};

__device__ __forceinline__ float alpha_at(int model, float o) {
    if (model == RGS_ALPHA_GFSGS) return o > 0.f ? -expm1f(-0.03279f * powf(o, 3.4f)) : 0.f;
    return o;
}

__device__ __forceinline__ bool aborted(const int *f) { return *(volatile const int *)f != 0; }

// pipeline stages an item's groups [g0, g1) fill, gps groups each
__device__ __forceinline__ long long stage_uses(long long g0, long long g1, int gps) { return (g1 - g0 + gps - 1) / gps; }

// where = role * 16 + wait site (1 producer empty, 2 mma dempty, 3 mma afull/rows, 4 builder
// hits, 5 builder dfull); the first failure's site and group count are kept for the message
__device__ __forceinline__ void tc_fail(const TcArgs &g, int *abort_flag, int where, long long gcount) {
    atomicExch(abort_flag, 1);
    if (atomicAdd(&g.flags[FLAG_TC_TIMEOUT], 1) == 0) {
        g.flags[FLAG_TC_TIMEOUT + 1] = where;
        g.flags[FLAG_TC_TIMEOUT + 2] = (int)gcount;
    }
}

// ------------------------------------------------------------------ the contraction kernel
// A stage holds GPS consecutive groups of one item (their source rows, their operands and
// their hit records, copied with one bulk copy), so that every barrier handshake, bulk
// hit copy and MMA commit is shared by GPS groups: the single issuing thread's per-group
// cost, not the tensor work, bounds a pipeline of 16-column-deep (K = 16) products.
// Roles: warps 0 .. TC_NP - 1 produce (all bulk copies; stage s belongs to warp s mod TC_NP:
// a copy's issue costs its thread a few hundred cycles), warp TC_NP owns the TMEM and issues
// the MMAs (one lane), the next TC_NB warps build operands (builder b = s * GPS + j builds slot j of
// every use of stage s, so every use of a stage is awaited by the same warps and a parity
// wait can never see a phase two uses old) and drain the accumulator.  Per stage: `hits`
// (records and metadata), `rows` (awaited by the MMA only), `afull` (GPS builders done),
// `empty` (MMAs done).
constexpr int TC_MW = TC_NP;     // the MMA warp
constexpr int TC_B0 = TC_NP + 1; // first builder warp
struct __align__(16) SlotMeta {
    float4 nrm; // adjoint: the group's receiver normal
    int other, cnt, hoff, pad;
};
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_contract(TcArgs g) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_hits[TC_CT_STAGES], bar_rows[TC_CT_STAGES], bar_afull[TC_CT_STAGES],
        bar_empty[TC_CT_STAGES];
    __shared__ __align__(8) uint64_t bar_dfull, bar_dempty, bar_drain;
    __shared__ SlotMeta meta[TC_CT_STAGES][TC_GPS_MAX];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ float sh_tab[16][20];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = g.stages, SS = g.stage_shift, GPS = g.gps;
    const int items = g.ntiles * g.nchunks;
    for (int q = threadIdx.x; q < 16 * 20; q += blockDim.x) (&sh_tab[0][0])[q] = (&TC_SH[0][0])[q];

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            tc::bar_init(&bar_hits[s], 1);
            tc::bar_init(&bar_rows[s], 1);
            tc::bar_init(&bar_afull[s], GPS);
            tc::bar_init(&bar_empty[s], 1);
        }
        tc::bar_init(&bar_dfull, 1);
        tc::bar_init(&bar_dempty, TC_NB);
        tc::bar_init(&bar_drain, 1);
        abort_flag = 0;
        tc::bar_init_fence();
    }
    if (warp == TC_MW) tc::tmem_alloc(&tmem_slot, 512);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t slot_rows = g.rows_bytes, slot_a = g.a_bytes; // per group of a stage
    const uint32_t a_off = (uint32_t)GPS * slot_rows;            // the operands after the rows
    const uint32_t h_off = a_off + (uint32_t)GPS * slot_a;       // then the hit records
    // the operands start as zeros: a builder then only clears the rows it wrote last time
    for (uint32_t q = threadIdx.x; q < (uint32_t)S * (GPS * slot_a / 16u); q += blockDim.x) {
        const uint32_t s = q / (GPS * slot_a / 16u), w = q - s * (GPS * slot_a / 16u);
        reinterpret_cast<uint4 *>(smem + (size_t)s * g.stage_bytes + a_off)[w] = make_uint4(0u, 0u, 0u, 0u);
    }
    tc::fence_async_smem();
    __syncthreads();

    if (warp < TC_NP) {
        // ---------------------------------------------------------- producers (stage s: warp s mod TC_NP)
        long long su = 0; // stage uses so far (stage su mod S, its use su >> SS)
        for (int it = blockIdx.x; it < items && !aborted(&abort_flag); it += gridDim.x) {
            const int t = it / g.nchunks, ch = it - t * g.nchunks;
            const int c0 = ch * TC_CHUNK;
            const int cw = min(TC_CHUNK, g.Cp - c0);
            const uint32_t rbytes = (uint32_t)cw * 32u;
            const long long g0 = g.goff[t], g1 = g.goff[t + 1];
            const long long hb = g.hoff[t];
            const int tile_hits = (int)(g.hoff[t + 1] - hb);
            for (long long gb = g0; gb < g1 && !aborted(&abort_flag); gb += 32) {
                const int m = (int)min(32ll, g1 - gb);
                int2 e = make_int2(0, 0);
                int next = tile_hits;
                float4 nrm = make_float4(0.f, 0.f, 1.f, 0.f);
                if (lane < m) {
                    e = __ldg(&g.grp[gb + lane]);
                    if (gb + lane + 1 < g1) next = __ldg(&g.grp[gb + lane + 1]).y;
                    if (g.adjoint) nrm = __ldg(&g.N4[e.x]);
                }
                // the batch in stage-sized chunks (a chunk never leaves its item)
                for (int q0 = 0; q0 < m; q0 += GPS, ++su) {
                    const int s = (int)(su & (S - 1));
                    if (s % TC_NP != warp) continue; // another producer's stage
                    const uint32_t ph = (uint32_t)((su >> SS) & 1);
                    bool ok = true;
                    if (lane == 0 && !tc::bar_wait(&bar_empty[s], ph ^ 1u, g.wait_ns)) {
                        tc_fail(g, &abort_flag, 16 * warp + 1, su);
                        ok = false;
                    }
                    ok = __shfl_sync(0xffffffffu, ok, 0);
                    if (!ok) break;
                    // lanes j < GPS describe slot j; lane 0 issues the copies
                    const int nin = min(GPS, m - q0);
                    const int first0 = __shfl_sync(0xffffffffu, e.y, q0);
                    int jo = 0, jc = -1, jf = 0;
                    float4 jn = make_float4(0.f, 0.f, 1.f, 0.f);
                    {
                        const int src = min(q0 + (lane < GPS ? lane : 0), 31);
                        jo = __shfl_sync(0xffffffffu, e.x, src);
                        jf = __shfl_sync(0xffffffffu, e.y, src);
                        const int jn_ = __shfl_sync(0xffffffffu, next, src);
                        jn.x = __shfl_sync(0xffffffffu, nrm.x, src);
                        jn.y = __shfl_sync(0xffffffffu, nrm.y, src);
                        jn.z = __shfl_sync(0xffffffffu, nrm.z, src);
                        jc = jn_ - jf;
                    }
                    const int last = __shfl_sync(0xffffffffu, next, q0 + nin - 1);
                    unsigned char *st = smem + (size_t)s * g.stage_bytes;
                    if (lane < GPS) {
                        SlotMeta sm;
                        sm.nrm = jn;
                        sm.other = jo;
                        sm.cnt = lane < nin ? jc : -1;
                        sm.hoff = jf - first0;
                        sm.pad = 0;
                        meta[s][lane] = sm;
                    }
                    __syncwarp();
                    if (lane == 0) {
                        const uint32_t hbytes = (uint32_t)(last - first0) * 16u;
                        tc::bar_arrive_tx(&bar_hits[s], hbytes);
                        tc::bulk_g2s(st + h_off, g.hd + hb + first0, hbytes, &bar_hits[s]);
                        tc::bar_arrive_tx(&bar_rows[s], (uint32_t)nin * rbytes * (g.split ? 2u : 1u));
                    }
                    if (lane < nin) { // one lane per group of the chunk issues its row copies
                        const size_t rb = (size_t)jo * (size_t)g.Cp * 16 + (size_t)c0 * 16;
                        unsigned char *dst = st + (size_t)lane * slot_rows;
                        tc::bulk_g2s(dst, g.rows_hi + rb, rbytes, &bar_rows[s]);
                        if (g.split) tc::bulk_g2s(dst + rbytes, g.rows_lo + rb, rbytes, &bar_rows[s]);
                    }
                    __syncwarp();
                }
                if (aborted(&abort_flag)) break;
            }
        }
        // no bulk copy may still be writing into this CTA's shared memory when it exits: wait
        // (bounded) for the last fill of every stage
        if (lane == 0)
            for (long long q = su - 1; q >= 0 && q >= su - S; --q) {
                if ((int)(q & (S - 1)) % TC_NP != warp) continue;
                tc::bar_wait(&bar_rows[q & (S - 1)], (uint32_t)((q >> SS) & 1), TC_DRAIN_NS);
                tc::bar_wait(&bar_hits[q & (S - 1)], (uint32_t)((q >> SS) & 1), TC_DRAIN_NS);
            }
        __syncwarp();
    } else if (warp == TC_MW) {
        // ---------------------------------------------------------- MMA issuer
        long long su = 0;
        int tl = 0;
        for (int it = blockIdx.x; it < items && !aborted(&abort_flag); it += gridDim.x, ++tl) {
            const int t = it / g.nchunks, ch = it - t * g.nchunks;
            const int cw = min(TC_CHUNK, g.Cp - ch * TC_CHUNK);
            const long long g0 = g.goff[t], g1 = g.goff[t + 1];
            const long long nst = stage_uses(g0, g1, GPS);
            if (lane == 0) {
                bool ok = true;
                if (tl > 0 && !tc::bar_wait(&bar_dempty, (uint32_t)((tl - 1) & 1), g.wait_ns)) {
                    tc_fail(g, &abort_flag, 16 * warp + 2, su);
                    ok = false;
                }
                tc::fence_after();
                const uint32_t rbytes = (uint32_t)cw * 32u;
                uint32_t acc0 = 0u;
                for (long long k = 0; k < nst && ok; ++k, ++su) {
                    const int s = (int)(su & (S - 1));
                    const uint32_t ph = (uint32_t)((su >> SS) & 1);
                    if (!tc::bar_wait(&bar_afull[s], ph, g.wait_ns) || !tc::bar_wait(&bar_rows[s], ph, g.wait_ns)) {
                        tc_fail(g, &abort_flag, 16 * warp + 3, su);
                        ok = false;
                        break;
                    }
                    const uint32_t st = tc::smem_addr(smem + (size_t)s * g.stage_bytes);
                    const int nin = (int)min((long long)GPS, (g1 - g0) - k * GPS);
                    for (int j = 0; j < nin; ++j) {
                        const uint32_t rows = st + (uint32_t)j * slot_rows;
                        const uint32_t A = st + a_off + (uint32_t)j * slot_a;
                        for (int c = 0; c < cw; c += 256) {
                            const int N = min(256, cw - c);
                            const uint32_t id = tc::idesc_bf16(128, N);
                            const uint32_t d = tmem + (uint32_t)c;
                            const uint64_t da = tc::sdesc(A), db = tc::sdesc(rows + (uint32_t)c * 32u);
                            tc::mma_bf16(d, da, db, id, acc0);
                            if (g.split) {
                                tc::mma_bf16(d, da, tc::sdesc(rows + rbytes + (uint32_t)c * 32u), id, 1u);
                                tc::mma_bf16(d, tc::sdesc(A + 4096u), db, id, 1u);
                            }
                        }
                        acc0 = 1u;
                    }
                    tc::mma_commit(&bar_empty[s]);
                }
                tc::mma_commit(&bar_dfull); // after a failure the other roles give up on their own waits
            }
            __syncwarp();
            su = __shfl_sync(0xffffffffu, su, 0);
        }
        // every MMA this thread issued has completed before the TMEM is freed
        if (lane == 0) {
            tc::mma_commit(&bar_drain);
            tc::bar_wait(&bar_drain, 0u, TC_DRAIN_NS);
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------- builders + epilogue
        const int b = warp - TC_B0;
        const int bs = b / GPS, bj = b - bs * GPS; // the stage and slot this warp builds
        const int k = lane & 15;
        // this lane's SH coefficients from the CTA's shared copy of the table (a divergent
        // read of constant memory would serialise the lanes every time it is re-read)
        float cf[20];
#pragma unroll
        for (int q = 0; q < 20; ++q) cf[q] = sh_tab[k][q];
        unsigned prev_written = 0u; // rows (tile slots) of this half written by the buffer's last use
        long long su = 0;
        int tl = 0;
        for (int it = blockIdx.x; it < items && !aborted(&abort_flag); it += gridDim.x, ++tl) {
            const int t = it / g.nchunks, ch = it - t * g.nchunks;
            const int c0 = ch * TC_CHUNK;
            const int cw = min(TC_CHUNK, g.Cp - c0);
            const long long g0 = g.goff[t], g1 = g.goff[t + 1];
            const long long nst = stage_uses(g0, g1, GPS);
            // forward: lane p < 8 holds the item's receiver p's normal
            float4 tn = make_float4(0.f, 0.f, 1.f, 0.f);
            if (!g.adjoint && lane < TC_R && t * TC_R + lane < g.n) tn = __ldg(&g.N4[t * TC_R + lane]);
            // this warp's uses: those of stage bs among the item's stage uses su .. su + nst - 1
            const long long k0 = (long long)((bs - (int)(su & (S - 1)) + S) & (S - 1));
            for (long long kk = k0; bs < S && kk < nst && !aborted(&abort_flag); kk += S) {
                const long long u = su + kk;
                const int s = bs;
                const uint32_t ph = (uint32_t)((u >> SS) & 1);
                bool ok = true;
                if (lane == 0) ok = tc::bar_wait(&bar_hits[s], ph, g.wait_ns);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                __syncwarp(); // lane 0's acquire of the stage covers the warp's reads of it
                if (!ok) {
                    if (lane == 0) tc_fail(g, &abort_flag, 16 * warp + 4, u);
                    break;
                }
                const SlotMeta mt = meta[s][bj];
                if (mt.cnt >= 0) {
                    unsigned char *st = smem + (size_t)s * g.stage_bytes;
                    const uint32_t A = tc::smem_addr(st + a_off + (size_t)bj * slot_a);
                    const float4 *hits = reinterpret_cast<const float4 *>(st + h_off) + mt.hoff;
                    const float3 ngrp = f3(mt.nrm);
                    // half-warp hf takes the group's hits whose tile slot p has parity hf, so the
                    // halves never share a row; lane k of a half forms row (p, k): sum over its hits
                    // of a X_k Z^T, X = Y(R d) (forward) or Y(-d) (adjoint), Z the other one
                    const int hf = lane >> 4;
                    float acc[16];
#pragma unroll
                    for (int m = 0; m < 16; ++m) acc[m] = 0.f;
                    int cur = -1;
                    unsigned written = 0;
                    auto flush = [&](int p) {
                        uint4 h0, h1;
                        h0.x = tc::pack_bf16(acc[0], acc[1]);
                        h0.y = tc::pack_bf16(acc[2], acc[3]);
                        h0.z = tc::pack_bf16(acc[4], acc[5]);
                        h0.w = tc::pack_bf16(acc[6], acc[7]);
                        h1.x = tc::pack_bf16(acc[8], acc[9]);
                        h1.y = tc::pack_bf16(acc[10], acc[11]);
                        h1.z = tc::pack_bf16(acc[12], acc[13]);
                        h1.w = tc::pack_bf16(acc[14], acc[15]);
                        const uint32_t off = tc::blk_off(p * 16 + k, 0);
                        tc::sts128(A + off, h0);
                        tc::sts128(A + off + 128u, h1);
                        if (g.split) {
                            float r[16];
#pragma unroll
                            for (int m = 0; m < 16; ++m) r[m] = acc[m] - __bfloat162float(__float2bfloat16_rn(acc[m]));
                            uint4 l0, l1;
                            l0.x = tc::pack_bf16(r[0], r[1]);
                            l0.y = tc::pack_bf16(r[2], r[3]);
                            l0.z = tc::pack_bf16(r[4], r[5]);
                            l0.w = tc::pack_bf16(r[6], r[7]);
                            l1.x = tc::pack_bf16(r[8], r[9]);
                            l1.y = tc::pack_bf16(r[10], r[11]);
                            l1.z = tc::pack_bf16(r[12], r[13]);
                            l1.w = tc::pack_bf16(r[14], r[15]);
                            tc::sts128(A + 4096u + off, l0);
                            tc::sts128(A + 4096u + off + 128u, l1);
                        }
                        written |= 1u << p;
                    };
                    // the slots' parities, 32 hits at a time: lane e holds hit e's parity bit
                    for (int base = 0; base < mt.cnt; base += 32) {
                        const int m_here = min(32, mt.cnt - base);
                        const bool odd = lane < m_here && (__float_as_uint(hits[base + lane].w) & 1u);
                        const unsigned odd_m = __ballot_sync(0xffffffffu, odd);
                        const unsigned all_m = m_here == 32 ? 0xffffffffu : ((1u << m_here) - 1u);
                        unsigned mine = hf ? odd_m : (all_m & ~odd_m); // this half's hits in the window
                        const int n_mine = __popc(mine);
                        const int n_iter = max(__popc(odd_m), __popc(all_m & ~odd_m));
                        for (int it2 = 0; it2 < n_iter; ++it2) {
                            const bool have = it2 < n_mine;
                            const int e = have ? __ffs(mine) - 1 : 0;
                            if (have) mine &= mine - 1;
                            const float4 rec = hits[base + e];
                            const uint32_t abits = __float_as_uint(rec.w);
                            const int p = (int)(abits & 7u);
                            const float a = have ? __uint_as_float(abits & ~7u) : 0.f;
                            const float3 d = make_float3(rec.x, rec.y, rec.z);
                            float3 nrm = ngrp;
                            if (!g.adjoint)
                                nrm = make_float3(__shfl_sync(0xffffffffu, tn.x, p), __shfl_sync(0xffffffffu, tn.y, p),
                                                  __shfl_sync(0xffffffffu, tn.z, p));
                            const float3 rd = reflect_n(nrm, d), md = make_float3(-d.x, -d.y, -d.z);
                            const float X = sh_mono(cf, g.adjoint ? md : rd);
                            float Z[16];
                            sh_eval<16>(g.adjoint ? rd : md, Z);
                            if (have && p != cur) {
                                if (cur >= 0) flush(cur);
#pragma unroll
                                for (int m = 0; m < 16; ++m) acc[m] = 0.f;
                                cur = p;
                            }
                            const float ax = a * X;
#pragma unroll
                            for (int m = 0; m < 16; ++m) acc[m] = fmaf(ax, Z[m], acc[m]);
                        }
                    }
                    if (cur >= 0) flush(cur);
                    // rows this half wrote in the buffer's last use and not now go back to zero
                    const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
                    unsigned stale = prev_written & ~written;
                    prev_written = written;
                    while (stale) {
                        const int p = __ffs(stale) - 1;
                        stale &= stale - 1;
                        const uint32_t off = tc::blk_off(p * 16 + k, 0);
                        tc::sts128(A + off, z4);
                        tc::sts128(A + off + 128u, z4);
                        if (g.split) {
                            tc::sts128(A + 4096u + off, z4);
                            tc::sts128(A + 4096u + off + 128u, z4);
                        }
                    }
                    tc::fence_async_smem();
                }
                __syncwarp();
                if (lane == 0) tc::bar_arrive(&bar_afull[s]);
            }
            su += nst;
            if (aborted(&abort_flag)) break;
            // ------------------------------------------------------ epilogue of the item
            bool ok = true;
            if (lane == 0) ok = tc::bar_wait(&bar_dfull, (uint32_t)(tl & 1), g.wait_ns);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            __syncwarp();
            tc::fence_after();
            if (!ok) {
                if (lane == 0) tc_fail(g, &abort_flag, 16 * warp + 5, su);
                break;
            }
            const bool empty = (g1 == g0);
            const int quarter = warp & 3, part = b >> 2; // TC_NB / 4 warps share a TMEM lane quarter
            const int row = quarter * 32 + lane;
            const int p = row >> 4, kr = row & 15;
            const int e_ent = t * TC_R + p;
            const bool live = e_ent < g.n;
            const float oe = live ? alpha_at(g.alpha_model, __ldg(&g.P[e_ent].w)) : 0.f;
            double dsq = 0.0;
            for (int cb = part * 16; cb < cw; cb += 16 * (TC_NB / 4)) {
                float v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)cb, v);
                if (!live) continue;
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int c = c0 + cb + q;
                    if (c >= g.C) break;
                    const float val = empty ? 0.f : v[q] * g.w;
                    const size_t idx = ((size_t)e_ent * g.C + c) * 16 + kr;
                    const float oc = oe * __ldg(&g.cl[(size_t)e_ent * 12 + band_of(kr) * 3 + (c % 3)]);
                    const size_t bidx = (size_t)e_ent * g.Cp * 16 + tc::blk_off(c, kr) / 2;
                    if (!g.adjoint) {
                        g.Qout[idx] = val;
                        const float bb = g.S[idx] + oc * val;
                        g.Bout[idx] = bb;
                        const __nv_bfloat16 bh = __float2bfloat16_rn(bb);
                        if (g.Bout16) g.Bout16[idx] = bh;
                        g.Bblk[bidx] = bh;
                        if (g.Bblk_lo) g.Bblk_lo[bidx] = __float2bfloat16_rn(bb - __bfloat162float(bh));
                        const double df = (double)bb - (double)g.Bprev[idx];
                        dsq += df * df;
                    } else {
                        g.vout[idx] = val;
                        g.u[idx] += val;
                        g.yblk[bidx] = __float2bfloat16_rn(oc * val);
                    }
                }
            }
            if (!g.adjoint) {
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) dsq += __shfl_xor_sync(0xffffffffu, dsq, off);
                if (lane == 0) atomicAdd(g.norm2, dsq);
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::bar_arrive(&bar_dempty);
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == TC_MW) tc::tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------------ opacity gather (adjoint)
// The per-hit sums of the opacity backward, g_h += sum over columns of y_r^(a) . s_h^(b) with
// y_r = (pi/nd) Y(R_i d)^T y_i^(a) and s_h = Y(-d)^T B_j^(b) (y = o c (x) v), regrouped per
// (receiver i, source j) pair:  g_h = (pi/nd) Y(R_i d)^T P_ij Y(-d),  P_ij[k][m] =
// sum_c y_i[c][k] B_j[c][m].  Over the adjoint's source tiles: the tile's 8 sources' rows
// B^(b) sit in TMEM as a 128 x C BF16 operand (rows = source x coefficient m); per group
// (receiver i) the receiver's BF16 y^(a) rows are bulk-copied into shared memory and read as
// an MN-major C x 16 operand, so C/16 MMAs leave D2[(sigma, m)][k] = P_{i sigma}[k][m] in TMEM;
// then the warps of one quad (one per TMEM lane quarter: sources 2q, 2q + 1) read their
// quarter and finish g_h for the group's hits on those sources.
struct TcOpaArgs {
    int n, C, Cp, nd, ntiles, stages;
    uint32_t stage_bytes, rows_bytes, tmem_cols;
    const long long *hoff, *goff;
    const int2 *grp;
    const float4 *hd;
    const uint32_t *hslot;          // per hit: its record slot (the compositing order of its ray)
    const __nv_bfloat16 *yblk;      // y^(a) of every receiver, blocked BF16 rows
    const float *Bsrc;              // B^(b), FP32 [N][C][16]
    const float4 *N4;
    float w;
    float *gh;
    int first;                      // write g_h instead of adding to it
    int *flags;
    unsigned long long wait_ns;
};

constexpr int TO_PROD = 2, TO_MMA = 2, TO_C0 = 3, TO_NC = 16, TO_QUADS = TO_NC / 4;
constexpr int TO_THREADS = (TO_C0 + TO_NC) * 32;

__device__ __forceinline__ void to_fail(const TcOpaArgs &g, int *abort_flag, int where, long long gcount) {
    atomicExch(abort_flag, 1);
    if (atomicAdd(&g.flags[FLAG_TC_TIMEOUT], 1) == 0) {
        g.flags[FLAG_TC_TIMEOUT + 1] = where;
        g.flags[FLAG_TC_TIMEOUT + 2] = (int)gcount;
    }
}

__global__ void __launch_bounds__(TO_THREADS, 1) k_tc_opacity(TcOpaArgs g) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_hits[TC_MAX_STAGES], bar_rows[TC_MAX_STAGES], bar_empty[TC_MAX_STAGES];
    __shared__ __align__(8) uint64_t bar_d2full[TO_QUADS], bar_d2empty[TO_QUADS], bar_a2full, bar_a2empty, bar_drain;
    __shared__ StageMeta meta[TC_MAX_STAGES];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ __align__(16) float ybuf_all[TO_NC][32];
    __shared__ float sh_tab[16][20];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = g.stages, SS = (S == 16) ? 4 : 3; // 16 or 8 stages
    for (int q = threadIdx.x; q < 16 * 20; q += blockDim.x) (&sh_tab[0][0])[q] = (&TC_SH[0][0])[q];
    const int a2cols = g.Cp / 2;                 // BF16 pairs per TMEM column
    const int d2col0 = (a2cols + 15) & ~15;      // D2 slots after the A2 operand

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            tc::bar_init(&bar_hits[s], 1);
            tc::bar_init(&bar_rows[s], 1);
            tc::bar_init(&bar_empty[s], 1 + 4); // the MMAs (rows free) and the quad's 4 warps (hits read)
        }
        for (int q = 0; q < TO_QUADS; ++q) {
            tc::bar_init(&bar_d2full[q], 1);
            tc::bar_init(&bar_d2empty[q], 4);
        }
        tc::bar_init(&bar_a2full, TO_NC);
        tc::bar_init(&bar_a2empty, 1);
        tc::bar_init(&bar_drain, 1);
        abort_flag = 0;
        tc::bar_init_fence();
    }
    if (warp == TO_MMA) tc::tmem_alloc(&tmem_slot, g.tmem_cols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_slot;
    const int items = g.ntiles;

    if (warp < TO_PROD) {
        // ---------------------------------------------------------- producers
        long long gc = 0;
        const uint32_t rbytes = (uint32_t)g.Cp * 32u;
        for (int t = blockIdx.x; t < items && !aborted(&abort_flag); t += gridDim.x) {
            const long long g0 = g.goff[t], g1 = g.goff[t + 1];
            const long long hb = g.hoff[t];
            const int tile_hits = (int)(g.hoff[t + 1] - hb);
            for (long long gb = g0; gb < g1 && !aborted(&abort_flag); gb += 32) {
                const int m = (int)min(32ll, g1 - gb);
                int2 e = make_int2(0, 0);
                int next = tile_hits;
                float4 nrm = make_float4(0.f, 0.f, 1.f, 0.f);
                if (lane < m) {
                    e = __ldg(&g.grp[gb + lane]);
                    if (gb + lane + 1 < g1) next = __ldg(&g.grp[gb + lane + 1]).y;
                    nrm = __ldg(&g.N4[e.x]);
                }
                for (int q = 0; q < m; ++q) {
                    const long long gq = gc + (gb - g0) + q;
                    if ((int)(gq % TO_PROD) != warp) continue;
                    const int other = __shfl_sync(0xffffffffu, e.x, q);
                    const int first = __shfl_sync(0xffffffffu, e.y, q);
                    const int cnt = __shfl_sync(0xffffffffu, next, q) - first;
                    float4 nq;
                    nq.x = __shfl_sync(0xffffffffu, nrm.x, q);
                    nq.y = __shfl_sync(0xffffffffu, nrm.y, q);
                    nq.z = __shfl_sync(0xffffffffu, nrm.z, q);
                    nq.w = __int_as_float(first); // the group's first hit, relative to the tile
                    if (lane == 0) {
                        const int s = (int)(gq & (S - 1));
                        const uint32_t ph = (uint32_t)((gq >> SS) & 1);
                        if (!tc::bar_wait(&bar_empty[s], ph ^ 1u, g.wait_ns)) {
                            to_fail(g, &abort_flag, 16 * warp + 1, gq);
                        } else {
                            meta[s].nrm = nq;
                            meta[s].other = other;
                            meta[s].cnt = cnt;
                            unsigned char *st = smem + (size_t)s * g.stage_bytes;
                            const uint32_t hbytes = (uint32_t)cnt * 16u;
                            tc::bar_arrive_tx(&bar_hits[s], hbytes);
                            tc::bulk_g2s(st + g.rows_bytes, g.hd + hb + first, hbytes, &bar_hits[s]);
                            tc::bar_arrive_tx(&bar_rows[s], rbytes);
                            tc::bulk_g2s(st, g.yblk + (size_t)other * (size_t)g.Cp * 16, rbytes, &bar_rows[s]);
                        }
                    }
                    __syncwarp();
                    if (aborted(&abort_flag)) break;
                }
            }
            gc += g1 - g0;
        }
        if (lane == 0) {
            long long seen = 0;
            for (long long q = gc - 1; q >= 0 && seen < S / TO_PROD; --q) {
                if ((int)(q % TO_PROD) != warp) continue;
                ++seen;
                tc::bar_wait(&bar_rows[q & (S - 1)], (uint32_t)((q >> SS) & 1), TC_DRAIN_NS);
                tc::bar_wait(&bar_hits[q & (S - 1)], (uint32_t)((q >> SS) & 1), TC_DRAIN_NS);
            }
        }
        __syncwarp();
    } else if (warp == TO_MMA) {
        // ---------------------------------------------------------- MMA issuer
        long long gc = 0;
        long long quse[TO_QUADS] = {0, 0, 0, 0};
        int tl = 0;
        for (int t = blockIdx.x; t < items && !aborted(&abort_flag); t += gridDim.x, ++tl) {
            const long long g0 = g.goff[t], g1 = g.goff[t + 1];
            if (lane == 0) {
                bool ok = tc::bar_wait(&bar_a2full, (uint32_t)(tl & 1), g.wait_ns);
                if (!ok) to_fail(g, &abort_flag, 16 * warp + 2, gc);
                tc::fence_after();
                for (long long q = g0; q < g1 && ok && !aborted(&abort_flag); ++q, ++gc) {
                    const int s = (int)(gc & (S - 1));
                    const uint32_t ph = (uint32_t)((gc >> SS) & 1);
                    const int Q = (int)(gc % TO_QUADS);
                    if (!tc::bar_wait(&bar_rows[s], ph, g.wait_ns) ||
                        (quse[Q] > 0 && !tc::bar_wait(&bar_d2empty[Q], (uint32_t)((quse[Q] - 1) & 1), g.wait_ns))) {
                        to_fail(g, &abort_flag, 16 * warp + 3, gc);
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    const uint32_t rows = tc::smem_addr(smem + (size_t)s * g.stage_bytes);
                    const uint32_t d = tmem + (uint32_t)(d2col0 + 16 * Q);
                    const uint32_t id = tc::idesc_bf16(128, 16) | (1u << 16); // B MN-major
                    for (int kk = 0; kk < g.Cp / 16; ++kk)
                        tc::mma_bf16_ta(d, tmem + (uint32_t)(kk * 8), tc::sdesc_mn(rows + (uint32_t)kk * 512u), id,
                                        kk > 0 ? 1u : 0u);
                    tc::mma_commit(&bar_empty[s]);
                    tc::mma_commit(&bar_d2full[Q]);
                    ++quse[Q];
                }
                tc::mma_commit(&bar_a2empty);
            }
            __syncwarp();
            gc = __shfl_sync(0xffffffffu, gc, 0);
            for (int Q = 0; Q < TO_QUADS; ++Q) quse[Q] = __shfl_sync(0xffffffffu, quse[Q], 0);
        }
        if (lane == 0) {
            tc::mma_commit(&bar_drain);
            tc::bar_wait(&bar_drain, 0u, TC_DRAIN_NS);
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------- A2 loaders + consumers
        const int cwp = warp - TO_C0;            // 0..15
        const int Q = cwp >> 2;                  // quad
        const int quarter = warp & 3;            // TMEM lane quarter: sources 2 quarter, 2 quarter + 1
        const int part = cwp >> 2;               // column share of the A2 load within the quarter
        const int k = lane & 15;
        // this lane's SH coefficients from the CTA's shared copy of the table (a divergent
        // read of constant memory would serialise the lanes every time it is re-read)
        float cf[20];
#pragma unroll
        for (int q = 0; q < 20; ++q) cf[q] = sh_tab[k][q];
        float *ybuf = ybuf_all[cwp];
        long long gc = 0, use = 0;
        int tl = 0;
        for (int t = blockIdx.x; t < items && !aborted(&abort_flag); t += gridDim.x, ++tl) {
            const long long g0 = g.goff[t], g1 = g.goff[t + 1];
            // A2: lane (sigma, m) of this quarter holds B^(b)[sigma][c][m] for every c, BF16 pairs
            if (tl > 0) {
                bool ok = true;
                if (lane == 0) ok = tc::bar_wait(&bar_a2empty, (uint32_t)((tl - 1) & 1), g.wait_ns);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                __syncwarp();
                tc::fence_after();
                if (!ok) {
                    if (lane == 0) to_fail(g, &abort_flag, 16 * warp + 6, gc);
                    break;
                }
            }
            {
                const int row = quarter * 32 + lane;
                const int src = t * TC_R + (row >> 4), m = row & 15;
                const bool live = src < g.n;
                for (int j0 = part * 8; j0 < a2cols; j0 += 8 * 4) {
                    uint32_t r[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int c = 2 * (j0 + q);
                        float x0 = 0.f, x1 = 0.f;
                        if (live && c < g.C) x0 = __ldg(&g.Bsrc[((size_t)src * g.C + c) * 16 + m]);
                        if (live && c + 1 < g.C) x1 = __ldg(&g.Bsrc[((size_t)src * g.C + c + 1) * 16 + m]);
                        r[q] = tc::pack_bf16(x0, x1);
                    }
                    tc::tmem_st8(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)j0, r);
                }
                tc::tmem_st_wait();
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::bar_arrive(&bar_a2full);
            }
            // this quad's groups of the item: CTA-wide index gq = Q (mod 4)
            const long long qfirst = g0 + (long long)((Q - (int)(gc % TO_QUADS) + TO_QUADS) % TO_QUADS);
            for (long long q = qfirst; q < g1 && !aborted(&abort_flag); q += TO_QUADS, ++use) {
                const long long gq = gc + (q - g0);
                const int s = (int)(gq & (S - 1));
                const uint32_t ph = (uint32_t)((gq >> SS) & 1);
                bool ok = true;
                if (lane == 0)
                    ok = tc::bar_wait(&bar_hits[s], ph, g.wait_ns) && tc::bar_wait(&bar_d2full[Q], (uint32_t)(use & 1), g.wait_ns);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                __syncwarp();
                tc::fence_after();
                if (!ok) {
                    if (lane == 0) to_fail(g, &abort_flag, 16 * warp + 4, gq);
                    break;
                }
                float P[16]; // P[k] of this lane's (sigma, m) row
                tc::tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(d2col0 + 16 * Q), P);
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::bar_arrive(&bar_d2empty[Q]);
                const int cnt = meta[s].cnt;
                const float3 nrm = f3(meta[s].nrm);
                const long long h0 = g.hoff[t] + __float_as_int(meta[s].nrm.w);
                const float4 *hits = reinterpret_cast<const float4 *>(smem + (size_t)s * g.stage_bytes + g.rows_bytes);
                const int mysig = 2 * quarter + (lane >> 4);
                for (int e = 0; e < cnt; ++e) {
                    const float4 rec = hits[e];
                    const uint32_t abits = __float_as_uint(rec.w);
                    const int sig = (int)(abits & 7u);
                    if ((sig >> 1) != quarter) continue; // another quarter's source
                    const float3 d = make_float3(rec.x, rec.y, rec.z);
                    // lanes 0..15: Y_k(R_i d); lanes 16..31: Y_k(-d)
                    const float3 v = (lane < 16) ? reflect_n(nrm, d) : make_float3(-d.x, -d.y, -d.z);
                    ybuf[lane] = sh_mono(cf, v);
                    __syncwarp();
                    float tsum = 0.f;
#pragma unroll
                    for (int kk = 0; kk < 16; ++kk) tsum = fmaf(ybuf[kk], P[kk], tsum);
                    float val = (sig == mysig) ? tsum * ybuf[16 + (lane & 15)] : 0.f;
#pragma unroll
                    for (int off = 8; off > 0; off >>= 1) val += __shfl_xor_sync(0xffffffffu, val, off);
                    __syncwarp();
                    if (lane == (sig & 1) * 16) {
                        const uint32_t slot = __ldg(&g.hslot[h0 + e]);
                        const float add = g.w * val;
                        g.gh[slot] = g.first ? add : g.gh[slot] + add;
                    }
                }
                __syncwarp();
                if (lane == 0) tc::bar_arrive(&bar_empty[s]);
            }
            gc += g1 - g0;
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == TO_MMA) tc::tmem_dealloc(tmem, g.tmem_cols);
}

// ------------------------------------------------------------------ pair-tile construction
// hits per receiver tile (forward): the sum of the counts of its rays
__global__ void k_tc_tile_count_fwd(const int *__restrict__ cnt, int n, int nd, int ntiles, int *tcount) {
    const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (t >= ntiles) return;
    const long long r0 = (long long)t * TC_R * nd, r1 = (long long)min(n, (t + 1) * TC_R) * nd;
    int s = 0;
    for (long long r = r0 + lane; r < r1; r += 32) s += cnt[r];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) tcount[t] = s;
}
// hits per source tile (adjoint): from the per-source offsets of the trace
__global__ void k_tc_tile_count_adj(const long long *__restrict__ src_off, int n, int ntiles, int *tcount) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    tcount[t] = (int)(src_off[min(n, (t + 1) * TC_R)] - src_off[t * TC_R]);
}

// forward: the tile's hits in ray order, key = j << 12 | rho << 9 | q, payload (a, h)
__global__ void __launch_bounds__(256) k_tc_gather_fwd(RaysDev rays, int n, const long long *__restrict__ hoff,
                                                       uint32_t *key, uint2 *pay) {
    const int t = blockIdx.x;
    const int nd = rays.nd;
    const long long r0 = (long long)t * TC_R * nd, r1 = (long long)min(n, (t + 1) * TC_R) * nd;
    __shared__ int wsum[8];
    long long pos = hoff[t];
    for (long long rb = r0; rb < r1; rb += 256) {
        const long long r = rb + threadIdx.x;
        const int c = (r < r1) ? rays.cnt[r] : 0;
        // block exclusive scan of c
        int incl = c;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += v;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        int before = 0, total = 0;
        for (int q = 0; q < 8; ++q) {
            if (q < w) before += wsum[q];
            total += wsum[q];
        }
        const long long out = pos + before + (incl - c);
        if (c > 0) {
            const long long base = rays.off[r];
            const int rl = (int)(r - r0);
            const uint32_t lo = (uint32_t)(((rl / nd) << 9) | (rl % nd));
            for (int h = 0; h < c; ++h) {
                const int2 ja = rays.rec_ja[base + h];
                key[out + h] = ((uint32_t)ja.x << 12) | lo;
                pay[out + h] = make_uint2((uint32_t)ja.y, (uint32_t)h);
            }
        }
        pos += total;
        __syncthreads();
    }
}

// adjoint: every hit to its source tile (unordered), key = i << 12 | sigma << 9 | q
__global__ void __launch_bounds__(256) k_tc_scatter_adj(RaysDev rays, long long n_rays, unsigned long long *cursor,
                                                        uint32_t *key, uint2 *pay) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const int c = rays.cnt[r];
    const long long base = rays.off[r];
    const int nd = rays.nd;
    const int i = (int)(r / nd), q = (int)(r - (long long)i * nd);
    for (int h = 0; h < c; ++h) {
        const int2 ja = rays.rec_ja[base + h];
        const unsigned long long at = atomicAdd(&cursor[ja.x / TC_R], 1ull);
        key[at] = ((uint32_t)i << 12) | ((uint32_t)(ja.x % TC_R) << 9) | (uint32_t)q;
        pay[at] = make_uint2((uint32_t)ja.y, (uint32_t)h);
    }
}

__global__ void k_tc_cursor(const long long *__restrict__ hoff, int ntiles, unsigned long long *cursor) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ntiles) cursor[t] = (unsigned long long)hoff[t];
}

// one stable pass of a segmented LSD radix sort (one block per segment): elements of
// segment t move by their digit (key >> shift) & 255, keeping their order within a digit
constexpr int SORT_THREADS = 1024;
__global__ void __launch_bounds__(SORT_THREADS) k_tc_sort_pass(const long long *__restrict__ seg, int shift,
                                                                const uint32_t *__restrict__ kin,
                                                                const uint2 *__restrict__ pin, uint32_t *kout,
                                                                uint2 *pout) {
    __shared__ int base[256];
    __shared__ int tot[256];
    __shared__ int wcnt[SORT_THREADS / 32][256];
    const long long s0 = seg[blockIdx.x], s1 = seg[blockIdx.x + 1];
    const int n = (int)(s1 - s0);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid < 256) base[tid] = 0;
    __syncthreads();
    for (int e = tid; e < n; e += SORT_THREADS) atomicAdd(&base[(kin[s0 + e] >> shift) & 255u], 1);
    __syncthreads();
    if (tid == 0) {
        int run = 0;
        for (int d = 0; d < 256; ++d) {
            const int c = base[d];
            base[d] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int c0 = 0; c0 < n; c0 += SORT_THREADS) {
        for (int q = tid; q < (SORT_THREADS / 32) * 256; q += SORT_THREADS) (&wcnt[0][0])[q] = 0;
        __syncthreads();
        const int e = c0 + tid;
        const bool valid = e < n;
        uint32_t kv = 0;
        uint2 pv = make_uint2(0u, 0u);
        int d = 256; // sentinel for lanes past the end
        if (valid) {
            kv = kin[s0 + e];
            pv = pin[s0 + e];
            d = (int)((kv >> shift) & 255u);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wcnt[w][d] = __popc(peers);
        __syncthreads();
        if (tid < 256) {
            int run = 0;
            for (int q = 0; q < SORT_THREADS / 32; ++q) {
                const int c = wcnt[q][tid];
                wcnt[q][tid] = run;
                run += c;
            }
            tot[tid] = run;
        }
        __syncthreads();
        if (valid) {
            const int at = base[d] + wcnt[w][d] + rank;
            kout[s0 + at] = kv;
            pout[s0 + at] = pv;
        }
        __syncthreads();
        if (tid < 256) base[tid] += tot[tid];
        __syncthreads();
    }
}

// groups per segment: each run of equal key >> 12 (one source, or one receiver) in pieces of
// at most TC_HCAP hits
__global__ void __launch_bounds__(256) k_tc_group_count(const long long *__restrict__ seg, const uint32_t *__restrict__ key,
                                                        int *gcount, unsigned long long *pairs) {
    const long long s0 = seg[blockIdx.x], s1 = seg[blockIdx.x + 1];
    int c = 0, pc = 0;
    for (long long e = s0 + threadIdx.x; e < s1; e += blockDim.x) {
        // distinct (other entity, tile slot) pairs: runs of equal key >> 9
        pc += (e == s0 || (key[e] >> 9) != (key[e - 1] >> 9)) ? 1 : 0;
        if (e != s0 && (key[e] >> 12) == (key[e - 1] >> 12)) continue;
        long long f = e + 1;
        while (f < s1 && (key[f] >> 12) == (key[e] >> 12)) ++f;
        c += (int)((f - e + TC_HCAP - 1) / TC_HCAP);
    }
    __shared__ int red[8];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) pc += __shfl_xor_sync(0xffffffffu, pc, off);
    if ((threadIdx.x & 31) == 0 && pc) atomicAdd(pairs, (unsigned long long)pc);
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
        gcount[blockIdx.x] = s;
    }
}

// the group list (other entity, first hit relative to the tile) and the per-hit records:
// direction d and weight a, with the hit's tile slot p in the 3 low mantissa bits of a
// (a relative change below 1e-6)
__global__ void __launch_bounds__(256) k_tc_finish(const long long *__restrict__ seg, const long long *__restrict__ goff,
                                                   const uint32_t *__restrict__ key, const uint2 *__restrict__ pay,
                                                   const float4 *__restrict__ dir, const long long *__restrict__ off,
                                                   int nd, int adjoint, int2 *grp, float4 *hd, uint32_t *hslot,
                                                   uint32_t *hray) {
    const int t = blockIdx.x;
    const long long s0 = seg[t], s1 = seg[t + 1];
    for (long long e = s0 + threadIdx.x; e < s1; e += blockDim.x) {
        const uint32_t kv = key[e];
        const uint2 pv = pay[e];
        const int other = (int)(kv >> 12), p = (int)((kv >> 9) & 7u), q = (int)(kv & 511u);
        const int recv = adjoint ? other : t * TC_R + p;
        const long long r = (long long)recv * nd + q;
        const float4 d = dir[r];
        hd[e] = make_float4(d.x, d.y, d.z, __uint_as_float((pv.x & ~7u) | (uint32_t)p));
        if (hslot) hslot[e] = (uint32_t)(off[r] + pv.y); // the record slot of the hit (its ray's h-th)
        if (hray) hray[e] = (uint32_t)r;
    }
    // groups: one warp walks the runs in 32-element windows
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        long long gi = goff[t];
        long long start = s0;
        auto emit = [&](long long a, long long b) { // the run [a, b) in pieces of TC_HCAP
            for (long long x = a; x < b; x += TC_HCAP) {
                if (lane == 0) grp[gi] = make_int2((int)(key[a] >> 12), (int)(x - s0));
                ++gi;
            }
        };
        for (long long e0 = s0; e0 < s1; e0 += 32) {
            const long long e = e0 + lane;
            const bool head = e < s1 && e != s0 && (key[e] >> 12) != (key[e - 1] >> 12);
            unsigned hm = __ballot_sync(0xffffffffu, head);
            while (hm) {
                const int l = __ffs(hm) - 1;
                hm &= hm - 1;
                emit(start, e0 + l);
                start = e0 + l;
            }
        }
        if (s1 > s0) emit(start, s1);
    }
}

// y = o c (x) v in the blocked BF16 layout (the adjoint's first right-hand side)
__global__ void k_tc_make_y(int n, int C, int Cp, int alpha_model, const float4 *__restrict__ P,
                            const float *__restrict__ cl, const float *__restrict__ v, __nv_bfloat16 *yblk) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * C * 16) return;
    const int k = (int)(idx & 15);
    const size_t ic = idx >> 4;
    const int c = (int)(ic % C);
    const int i = (int)(ic / C);
    const float o = alpha_at(alpha_model, P[i].w);
    const float y = o * cl[(size_t)i * 12 + band_of(k) * 3 + (c % 3)] * v[idx];
    yblk[(size_t)i * Cp * 16 + tc::blk_off(c, k) / 2] = __float2bfloat16_rn(y);
}
// x in the blocked BF16 layout, hi and (optionally) lo parts
__global__ void k_tc_to_blk(int n, int C, int Cp, const float *__restrict__ x, __nv_bfloat16 *hi, __nv_bfloat16 *lo) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * C * 16) return;
    const int k = (int)(idx & 15);
    const size_t ic = idx >> 4;
    const int c = (int)(ic % C);
    const int i = (int)(ic / C);
    const float v = x[idx];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const size_t b = (size_t)i * Cp * 16 + tc::blk_off(c, k) / 2;
    hi[b] = h;
    if (lo) lo[b] = __float2bfloat16_rn(v - __bfloat162float(h));
}

} // namespace

// ------------------------------------------------------------------ host side
struct TcPairs {
    int ntiles = 0;
    long long n_hits = 0, n_groups = 0, n_pairs = 0;
    long long *hoff = nullptr, *goff = nullptr;
    int2 *grp = nullptr;
    float4 *hd = nullptr;
    uint32_t *hslot = nullptr; // source tiles: each hit's record slot (the opacity gather writes g_h there)
    uint32_t *hray = nullptr;  // source tiles: each hit's ray (the opacity gather reads its y row)
    float *gt = nullptr;       // source tiles: the opacity gather's per-hit sums in this order
};

struct rgs_tc_state {
    TcPairs fwd, adj;
    bool fwd_ok = false, adj_ok = false;
    long long bytes = 0;
    int Cp = 0;
    __nv_bfloat16 *blk[3] = {nullptr, nullptr, nullptr}; // ping, pong, lo
    long long blk_cap = 0;
};

namespace {

void pairs_free(TcPairs &p) {
    dev_free(p.hoff);
    dev_free(p.goff);
    dev_free(p.grp);
    dev_free(p.hd);
    dev_free(p.hslot);
    dev_free(p.hray);
    dev_free(p.gt);
    p = TcPairs{};
}

// builds one pair-tile structure (forward: receiver tiles; adjoint: source tiles)
rgs_status build_pairs(rgs_transport *t, bool adjoint, TcPairs &P, cudaStream_t st) {
    rgs_status r;
    const int n = t->n, nd = t->nd;
    const int ntiles = (n + TC_R - 1) / TC_R;
    const long long H = t->n_hits;
    RaysDev rd = t->rays();
    pairs_free(P);
    P.ntiles = ntiles;
    P.n_hits = H;
    int *tcount = nullptr;
    uint32_t *kA = nullptr, *kB = nullptr;
    uint2 *pA = nullptr, *pB = nullptr;
    unsigned long long *cur = nullptr;
    long long *scan_tmp = nullptr;
    struct Tmp {
        cudaStream_t st;
        int **tc;
        uint32_t **ka, **kb;
        uint2 **pa, **pb;
        unsigned long long **cu;
        long long **sc;
        ~Tmp() {
            pool_release(*tc, st);
            pool_release(*ka, st);
            pool_release(*kb, st);
            pool_release(*pa, st);
            pool_release(*pb, st);
            pool_release(*cu, st);
            pool_release(*sc, st);
        }
    } tmp{st, &tcount, &kA, &kB, &pA, &pB, &cur, &scan_tmp};
    const int scan_cap = rgs_scan_tmp_size(ntiles);
    if ((r = pool_alloc(&tcount, (size_t)ntiles + 1, st)) != RGS_OK) return r;
    unsigned long long *cur_pairs = nullptr;
    struct PairsTmp {
        cudaStream_t st;
        unsigned long long **p;
        ~PairsTmp() { pool_release(*p, st); }
    } ptmp{st, &cur_pairs};
    if ((r = pool_alloc(&cur_pairs, 1, st)) != RGS_OK) return r;
    if ((r = pool_alloc(&scan_tmp, (size_t)scan_cap, st)) != RGS_OK) return r;
    if ((r = pool_alloc(&kA, (size_t)std::max(H, 1ll), st)) != RGS_OK) return r;
    if ((r = pool_alloc(&kB, (size_t)std::max(H, 1ll), st)) != RGS_OK) return r;
    if ((r = pool_alloc(&pA, (size_t)std::max(H, 1ll), st)) != RGS_OK) return r;
    if ((r = pool_alloc(&pB, (size_t)std::max(H, 1ll), st)) != RGS_OK) return r;
    if ((r = dev_alloc(&P.hoff, (size_t)ntiles + 1)) != RGS_OK) return r;
    if ((r = dev_alloc(&P.goff, (size_t)ntiles + 1)) != RGS_OK) return r;
    if ((r = dev_alloc(&P.hd, (size_t)std::max(H, 1ll))) != RGS_OK) return r;
    if (adjoint && (r = dev_alloc(&P.hslot, (size_t)std::max(H, 1ll))) != RGS_OK) return r;
    if (adjoint && (r = dev_alloc(&P.hray, (size_t)std::max(H, 1ll))) != RGS_OK) return r;
    if (adjoint && (r = dev_alloc(&P.gt, (size_t)std::max(H, 1ll))) != RGS_OK) return r;
    if (!adjoint) {
        { ProfScope ps_("k_tc_tile_count", st); k_tc_tile_count_fwd<<<(ntiles + 7) / 8, 256, 0, st>>>(t->cnt, n, nd, ntiles, tcount); }
    } else {
        { ProfScope ps_("k_tc_tile_count", st); k_tc_tile_count_adj<<<(ntiles + 255) / 256, 256, 0, st>>>(t->src_off, n, ntiles, tcount); }
    }
    RGS_LAUNCH("tc tile count");
    if ((r = rgs_scan_counts(tcount, P.hoff, ntiles, scan_tmp, scan_cap, st)) != RGS_OK) return r;
    int passes_lo;
    if (!adjoint) {
        { ProfScope ps_("k_tc_gather", st); k_tc_gather_fwd<<<ntiles, 256, 0, st>>>(rd, n, P.hoff, kA, pA); }
        passes_lo = 12; // ray order already sorts the low 12 bits (rho, q); sort j stably
    } else {
        if ((r = pool_alloc(&cur, (size_t)ntiles, st)) != RGS_OK) return r;
        { ProfScope ps_("k_tc_cursor", st); k_tc_cursor<<<(ntiles + 255) / 256, 256, 0, st>>>(P.hoff, ntiles, cur); }
        const long long n_rays = (long long)n * nd;
        { ProfScope ps_("k_tc_scatter", st); k_tc_scatter_adj<<<(unsigned)((n_rays + 255) / 256), 256, 0, st>>>(rd, n_rays, cur, kA, pA); }
        passes_lo = 0; // arbitrary order: sort all 32 bits
    }
    RGS_LAUNCH("tc gather");
    // LSD passes of 8 bits from passes_lo up to bit 32 (keys: entity < 2^20 above bit 12)
    uint32_t *kin = kA, *kout = kB;
    uint2 *pin = pA, *pout = pB;
    for (int shift = passes_lo; shift < 32; shift += 8) {
        { ProfScope ps_("k_tc_sort_pass", st); k_tc_sort_pass<<<ntiles, SORT_THREADS, 0, st>>>(P.hoff, shift, kin, pin, kout, pout); }
        std::swap(kin, kout);
        std::swap(pin, pout);
    }
    RGS_LAUNCH("tc sort");
    RGS_CUDA(cudaMemsetAsync(cur_pairs, 0, sizeof(unsigned long long), st));
    { ProfScope ps_("k_tc_group_count", st); k_tc_group_count<<<ntiles, 256, 0, st>>>(P.hoff, kin, tcount, cur_pairs); }
    RGS_LAUNCH("tc group count");
    if ((r = rgs_scan_counts(tcount, P.goff, ntiles, scan_tmp, scan_cap, st)) != RGS_OK) return r;
    long long ng = 0;
    unsigned long long np = 0;
    RGS_CUDA(cudaMemcpyAsync(&ng, P.goff + ntiles, sizeof(long long), cudaMemcpyDeviceToHost, st));
    RGS_CUDA(cudaMemcpyAsync(&np, cur_pairs, sizeof(np), cudaMemcpyDeviceToHost, st));
    RGS_CUDA(cudaStreamSynchronize(st));
    P.n_groups = ng;
    P.n_pairs = (long long)np;
    if ((r = dev_alloc(&P.grp, (size_t)std::max(ng, 1ll))) != RGS_OK) return r;
    { ProfScope ps_("k_tc_finish", st); k_tc_finish<<<ntiles, 256, 0, st>>>(P.hoff, P.goff, kin, pin, t->dir, t->off, nd, adjoint ? 1 : 0, P.grp, P.hd, P.hslot, P.hray); }
    RGS_LAUNCH("tc finish");
    return RGS_OK;
}

int g_num_sms = 0;
uint32_t g_smem_budget = 0;

rgs_status launch_contract(const rgs_transport *t, TcArgs a, cudaStream_t st) {
    if (!g_num_sms) {
        int dev = 0;
        RGS_CUDA(cudaGetDevice(&dev));
        RGS_CUDA(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    const int cw = std::min(TC_CHUNK, a.Cp);
    a.nchunks = (a.Cp + TC_CHUNK - 1) / TC_CHUNK;
    a.rows_bytes = (uint32_t)cw * 32u * (a.split ? 2u : 1u);
    a.a_bytes = 4096u * (a.split ? 2u : 1u);
    // the dynamic shared memory a CTA may opt into, less the kernel's static barriers and buffers
    if (!g_smem_budget) {
        int dev = 0, optin = 0;
        RGS_CUDA(cudaGetDevice(&dev));
        RGS_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        cudaFuncAttributes fa{};
        RGS_CUDA(cudaFuncGetAttributes(&fa, k_tc_contract));
        g_smem_budget = (uint32_t)(optin - (int)fa.sharedSizeBytes - 256);
    }
    const uint32_t budget = g_smem_budget;
    // four stages of as many groups as fit (up to four: the builder warps are stages x groups)
    a.stages = TC_CT_STAGES;
    a.stage_shift = 2;
    a.gps = 0;
    for (int gps = TC_GPS_MAX; gps >= 1 && !a.gps; gps /= 2) {
        const uint32_t sb = ((uint32_t)gps * (a.rows_bytes + a.a_bytes + TC_HCAP * 16u) + 127u) & ~127u;
        if ((uint32_t)a.stages * sb <= budget) {
            a.gps = gps;
            a.stage_bytes = sb;
        }
    }
    if (!a.gps) {
        rgs_set_error("tensor-core contraction: a stage of %u-byte rows exceeds shared memory", a.rows_bytes);
        return RGS_ERR_ARG;
    }
    const size_t smem = std::max<size_t>((size_t)a.stages * a.stage_bytes, 120u * 1024u);
    RGS_CUDA(cudaFuncSetAttribute(k_tc_contract, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int items = a.ntiles * a.nchunks;
    const int grid = std::max(1, std::min(items, g_num_sms));
    {
        ProfScope ps_(a.adjoint ? "k_tc_adjoint" : "k_tc_bounce", st);
        k_tc_contract<<<grid, TC_THREADS, smem, st>>>(a);
    }
    RGS_LAUNCH("tensor-core contraction");
    return RGS_OK;
}

} // namespace

rgs_status rgs_seg_sort(const long long *seg, int nseg, int passes, uint32_t *k0, uint2 *v0, uint32_t *k1, uint2 *v1,
                        cudaStream_t st) {
    if (nseg <= 0) return RGS_OK;
    for (int p = 0; p < passes; ++p) {
        ProfScope ps_("k_tc_sort_pass", st);
        if (p % 2 == 0) k_tc_sort_pass<<<nseg, SORT_THREADS, 0, st>>>(seg, 8 * p, k0, v0, k1, v1);
        else k_tc_sort_pass<<<nseg, SORT_THREADS, 0, st>>>(seg, 8 * p, k1, v1, k0, v0);
    }
    RGS_LAUNCH("segmented sort");
    return RGS_OK;
}

void rgs_tc_free(rgs_transport *t) {
    if (!t->tc) return;
    pairs_free(t->tc->fwd);
    pairs_free(t->tc->adj);
    for (auto &b : t->tc->blk) dev_free(b);
    delete t->tc;
    t->tc = nullptr;
}

// clears the contraction's failure record before a solve or an adjoint on the tensor cores
rgs_status rgs_tc_reset_flags(rgs_transport *t, cudaStream_t st) {
    RGS_CUDA(cudaMemsetAsync(t->flags + FLAG_TC_TIMEOUT, 0, 3 * sizeof(int), st));
    return RGS_OK;
}

rgs_status rgs_tc_check(rgs_transport *t, cudaStream_t st) {
    int f[3] = {0, 0, 0};
    RGS_CUDA(cudaMemcpyAsync(f, t->flags + FLAG_TC_TIMEOUT, sizeof f, cudaMemcpyDeviceToHost, st));
    RGS_CUDA(cudaStreamSynchronize(st));
    if (f[0]) {
        rgs_set_error("tensor-core contraction: %d bounded waits ran out (first: role %d, site %d, group %d)", f[0],
                      f[1] / 16, f[1] % 16, f[2]);
        return RGS_ERR_TIMEOUT;
    }
    return RGS_OK;
}

bool rgs_tc_adj_hits(const rgs_transport *t, RgsTcAdjHits *out) {
    if (!t->tc || !t->tc->adj_ok) return false;
    const TcPairs &P = t->tc->adj;
    *out = RgsTcAdjHits{P.ntiles, P.n_hits, P.hoff, P.hd, P.hslot, P.hray, P.gt};
    return true;
}

void rgs_tc_invalidate(rgs_transport *t) {
    if (!t->tc) return;
    t->tc->fwd_ok = t->tc->adj_ok = false;
}

bool rgs_tc_eligible(const rgs_transport *t, int precision) {
    if (t->tc_mode == 0) return false; // disabled by the caller
    if (t->kind != RGS_KIND_HEMISPHERE || t->nc != 16 || precision == RGS_FP32) return false;
    if (t->n > (1 << 20) || t->nd > 512 || t->n_hits <= 0 || t->n_slots >= (1ll << 32)) return false;
    if (t->tc_mode < 0 && t->C < RGS_TC_MIN_COLS) return false; // automatic: many right-hand sides only
    if (2 * ((t->C + 15) / 16) * 8 + 64 > 512 && t->tc_mode == 2) return false; // opacity operand in TMEM
    if (t->stride != 0) return false; // the adjoint reads every iterate of this path
    // memory: two structures of 16-28 B per hit, three blocked BF16 arrays, sort scratch of 24 B per hit
    const double need = 48.0 * t->n_hits + 24.0 * t->n_hits + 3.0 * 2.0 * t->n * (double)((t->C + 15) & ~15) * 16;
    return need < 0.8 * (double)pool_available_bytes();
}

// the forward structure and the blocked BF16 buffers (built once per trace)
rgs_status rgs_tc_prepare(rgs_transport *t, cudaStream_t st) {
    rgs_status r;
    if (!t->tc) t->tc = new rgs_tc_state();
    rgs_tc_state &s = *t->tc;
    const int Cp = (t->C + 15) & ~15; // MMA pieces of N = 16k columns
    const long long need = (long long)t->n * Cp * 16;
    if (need > s.blk_cap || s.Cp != Cp) {
        for (auto &b : s.blk)
            if ((r = dev_alloc(&b, (size_t)need, &t->device_bytes)) != RGS_OK) return r;
        s.blk_cap = need;
        s.Cp = Cp;
        for (auto &b : s.blk) RGS_CUDA(cudaMemsetAsync(b, 0, sizeof(__nv_bfloat16) * need, st)); // padding columns stay 0
    }
    if (!s.fwd_ok) {
        if ((r = build_pairs(t, false, s.fwd, st)) != RGS_OK) return r;
        s.fwd_ok = true;
    }
    return RGS_OK;
}

rgs_status rgs_tc_prepare_adjoint(rgs_transport *t, cudaStream_t st) {
    rgs_status r;
    if ((r = rgs_tc_prepare(t, st)) != RGS_OK) return r;
    if (!t->tc->adj_ok) {
        if ((r = build_pairs(t, true, t->tc->adj, st)) != RGS_OK) return r;
        t->tc->adj_ok = true;
    }
    return RGS_OK;
}

// B^(0) = S into the blocked buffer `slot` (hi) and, with lo, its low part
rgs_status rgs_tc_load_blk(rgs_transport *t, const float *x, int slot, bool lo, cudaStream_t st) {
    rgs_tc_state &s = *t->tc;
    const size_t tot = t->arr();
    { ProfScope ps_("k_tc_to_blk", st); k_tc_to_blk<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(t->n, t->C, s.Cp, x, s.blk[slot], lo ? s.blk[2] : nullptr); }
    RGS_LAUNCH("to blocked");
    return RGS_OK;
}

// one forward bounce on the tensor cores: reads blk[in] (and blk[2] as lo when split),
// writes Q, B (FP32), B16 (row layout, optional), blk[out] and, with want_lo, blk[2]
rgs_status rgs_tc_bounce(rgs_transport *t, int in, int out, bool split, bool want_lo, const float *Bprev,
                         const float *S, float *Q, float *Bout, __nv_bfloat16 *Bout16, double *norm2, cudaStream_t st) {
    rgs_tc_state &s = *t->tc;
    TcArgs a{};
    a.adjoint = 0;
    a.split = split ? 1 : 0;
    a.n = t->n;
    a.C = t->C;
    a.Cp = s.Cp;
    a.nd = t->nd;
    a.ntiles = s.fwd.ntiles;
    a.hoff = s.fwd.hoff;
    a.goff = s.fwd.goff;
    a.grp = s.fwd.grp;
    a.hd = s.fwd.hd;
    a.rows_hi = s.blk[in];
    a.rows_lo = split ? s.blk[2] : nullptr;
    a.N4 = t->sc->N4;
    a.P = t->sc->P;
    a.cl = t->sc->cl;
    a.alpha_model = t->sc->alpha_model;
    a.w = 3.14159265358979f / (float)t->nd;
    a.S = S;
    a.Bprev = Bprev;
    a.Qout = Q;
    a.Bout = Bout;
    a.Bout16 = Bout16;
    a.Bblk = s.blk[out];
    a.Bblk_lo = want_lo ? s.blk[2] : nullptr;
    a.norm2 = norm2;
    a.flags = t->flags;
    a.wait_ns = t->tc_wait_ns;
    return launch_contract(t, a, st);
}

// y^(0) = o c (x) v^(0) into blk[slot]
rgs_status rgs_tc_make_y(rgs_transport *t, const float *v, int slot, cudaStream_t st) {
    rgs_tc_state &s = *t->tc;
    const size_t tot = t->arr();
    { ProfScope ps_("k_tc_make_y", st); k_tc_make_y<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(t->n, t->C, s.Cp, t->sc->alpha_model, t->sc->P, t->sc->cl, v, s.blk[slot]); }
    RGS_LAUNCH("make y");
    return RGS_OK;
}

// one transposed bounce: v_out = K^T v_in from y_in = blk[in]; u += v_out; y_out = blk[out]
rgs_status rgs_tc_adjoint_bounce(rgs_transport *t, int in, int out, float *vout, float *u, cudaStream_t st) {
    rgs_tc_state &s = *t->tc;
    TcArgs a{};
    a.adjoint = 1;
    a.split = 0;
    a.n = t->n;
    a.C = t->C;
    a.Cp = s.Cp;
    a.nd = t->nd;
    a.ntiles = s.adj.ntiles;
    a.hoff = s.adj.hoff;
    a.goff = s.adj.goff;
    a.grp = s.adj.grp;
    a.hd = s.adj.hd;
    a.rows_hi = s.blk[in];
    a.N4 = t->sc->N4;
    a.P = t->sc->P;
    a.cl = t->sc->cl;
    a.alpha_model = t->sc->alpha_model;
    a.w = 3.14159265358979f / (float)t->nd;
    a.vout = vout;
    a.u = u;
    a.yblk = s.blk[out];
    a.flags = t->flags;
    a.wait_ns = t->tc_wait_ns;
    return launch_contract(t, a, st);
}

// counts of the pair tiles (for throughput reports): receiver tiles, their groups and
// distinct (receiver, source) pairs, stored hits, source tiles and their groups; zeros for
// a structure not built yet
extern "C" rgs_status rgs_contraction_info(const rgs_transport *t, int64_t *out, int32_t n) {
    if (!t || !out || n < 6) {
        rgs_set_error("rgs_contraction_info: NULL argument or fewer than 6 entries");
        return RGS_ERR_ARG;
    }
    for (int q = 0; q < n; ++q) out[q] = 0;
    if (!t->tc) return RGS_OK;
    const rgs_tc_state &s = *t->tc;
    if (s.fwd_ok) {
        out[0] = s.fwd.ntiles;
        out[1] = s.fwd.n_groups;
        out[2] = s.fwd.n_pairs;
        out[3] = s.fwd.n_hits;
    }
    if (s.adj_ok) {
        out[4] = s.adj.ntiles;
        out[5] = s.adj.n_groups;
    }
    return RGS_OK;
}

// the opacity gather of one adjoint pairing: g_h (+)= the sums of y^(a) (blk[slot]) against B^(b)
// (FP32 Bsrc) over the source tiles; first: write instead of add
rgs_status rgs_tc_opacity(rgs_transport *t, int slot, const float *Bsrc, bool first, cudaStream_t st) {
    rgs_tc_state &s = *t->tc;
    if (!g_num_sms) {
        int dev = 0;
        RGS_CUDA(cudaGetDevice(&dev));
        RGS_CUDA(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    TcOpaArgs a{};
    a.n = t->n;
    a.C = t->C;
    a.Cp = s.Cp;
    a.nd = t->nd;
    a.ntiles = s.adj.ntiles;
    a.hoff = s.adj.hoff;
    a.goff = s.adj.goff;
    a.grp = s.adj.grp;
    a.hd = s.adj.hd;
    a.hslot = s.adj.hslot;
    a.yblk = s.blk[slot];
    a.Bsrc = Bsrc;
    a.N4 = t->sc->N4;
    a.w = 3.14159265358979f / (float)t->nd;
    a.gh = t->gh;
    a.first = first ? 1 : 0;
    a.flags = t->flags;
    a.wait_ns = t->tc_wait_ns;
    a.rows_bytes = (uint32_t)s.Cp * 32u;
    a.stage_bytes = (a.rows_bytes + TC_HCAP * 16u + 127u) & ~127u;
    const uint32_t need_cols = (uint32_t)(((s.Cp / 2 + 15) & ~15) + 16 * TO_QUADS);
    a.tmem_cols = need_cols <= 256 ? 256u : 512u;
    if (need_cols > 512) {
        rgs_set_error("tensor-core opacity gather: %d columns do not fit tensor memory", t->C);
        return RGS_ERR_ARG;
    }
    int optin = 0, dev = 0;
    RGS_CUDA(cudaGetDevice(&dev));
    RGS_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa{};
    RGS_CUDA(cudaFuncGetAttributes(&fa, k_tc_opacity));
    const uint32_t budget = (uint32_t)(optin - (int)fa.sharedSizeBytes - 256);
    a.stages = (16u * a.stage_bytes <= budget) ? 16 : 8;
    if ((uint32_t)a.stages * a.stage_bytes > budget) {
        rgs_set_error("tensor-core opacity gather: stages of %u bytes exceed shared memory", a.stage_bytes);
        return RGS_ERR_ARG;
    }
    const size_t smem = std::max<size_t>((size_t)a.stages * a.stage_bytes, 120u * 1024u);
    RGS_CUDA(cudaFuncSetAttribute(k_tc_opacity, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = std::max(1, std::min(a.ntiles, g_num_sms));
    {
        ProfScope ps_("k_tc_opacity", st);
        k_tc_opacity<<<grid, TO_THREADS, smem, st>>>(a);
    }
    RGS_LAUNCH("tensor-core opacity gather");
    return RGS_OK;
}
