/*
 * rgs.h — C ABI of the GB300 light-transport library for Gaussian surfels
 * (adapted radiosity; "Differentiable Light Transport with Gaussian Surfels via
 * Adapted Radiosity", arXiv 2509.18497).
 *
 * The library computes, on one GPU, the outgoing radiance of every surfel held as
 * spherical-harmonic (SH) coefficients per RGB channel, under point lights, with
 * global illumination, and the gradients of a loss with respect to the surfels'
 * emission, diffuse albedo and opacity, and (rgs_adjoint_geometry) their centres, scales
 * and frames:
 *
 *   rgs_build_scene      surfel frames, BRDF coefficients, Morton order, BVH  (Eq. G, Eq. brdf, App. A)
 *   rgs_trace_transport  hemisphere rays with alpha compositing (Eq. L_I, App. B) and the
 *                        direct term from shadow rays (Sec. 5.2 direct-illumination equation)
 *   rgs_solve            bounce iteration B <- S + K B (Eq. final-radiosity; Sec. 7 hybrid solver:
 *                        direct term first, then a fixed number of bounces)
 *   rgs_adjoint          transposed bounces and parameter gradients (Eq. final_dL_dE,
 *                        Eq. final-dl-dbrdf, Eq. dl-dgeo-0 restricted to opacity)
 *   rgs_adjoint_geometry the same with the geometry gradients of Eqs. dl-dgeo-0/1
 *                        (centres, scales, frames) for either transport
 *   rgs_trace_pairs      the center-to-center approximation (Sec. 8) in place of the
 *                        hemisphere rays, and rgs_adjoint_pairs with its lambda gradient
 *                        (rgs_adjoint_pairs_geometry: with the position, scale and
 *                        frame gradients of Eqs. dl-dgeo-0/1 as well)
 *
 * CONVENTIONS (all entry points)
 *  - Every pointer documented "device" must point to memory of the current CUDA device;
 *    "host" pointers to host memory.  Arrays are dense, row-major, float32 unless stated.
 *  - The caller owns every array it passes in or receives results in; the library never
 *    frees caller memory.  The library owns the opaque handles and their workspace.
 *  - All GPU work is enqueued on `stream` (a cudaStream_t; NULL = legacy default stream).
 *    Entry points that report data to the host (hit counts, residual norms, status flags
 *    raised on the device) synchronise `stream` before returning; this is stated per call.
 *  - No C++ exception crosses this boundary.  Every call returns an rgs_status; the text
 *    of the last error on the calling thread is available from rgs_last_error().
 *  - Handles are not thread-safe: one handle is used by one host thread at a time.
 *  - Indexing: surfels are numbered 0..N-1 in the caller's order everywhere in the ABI.
 *    SH coefficients are ordered Y00, Y1-1, Y10, Y11, Y2-2, ... (index l*l + l + m), real,
 *    orthonormal, with the Condon-Shortley phase (Y1-1 = -c y, Y10 = c z, Y11 = -c x).
 *  - Right-hand sides ("columns"): C = 3 * max(NL, 1).  Column c = light * 3 + channel:
 *    light `light` alone plus the emission E.  With no lights there is one condition
 *    (emission only).
 *  - Radiosity arrays B and dL/dB are [N][nc][C] with nc = (L+1)^2.
 */
#ifndef RGS_H
#define RGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RGS_MAX_SH_DEGREE 3  /* L in [0, 3]: nc in {1, 4, 9, 16} */
#define RGS_MAX_BOUNCES 64
#define RGS_ABI_VERSION 1

typedef enum rgs_status {
    RGS_OK = 0,
    RGS_ERR_ARG = 1,       /* invalid argument (NULL pointer, size out of range, bad enum) */
    RGS_ERR_CUDA = 2,      /* a CUDA runtime call failed; see rgs_last_error() */
    RGS_ERR_OOM = 3,       /* device allocation failed */
    RGS_ERR_CAPACITY = 4,  /* a fixed-size buffer was too small (reported, never overrun) */
    RGS_ERR_NONFINITE = 5, /* an input holds NaN or Inf (only when checking is enabled) */
    RGS_ERR_TIMEOUT = 6,   /* a bounded device-side wait gave up */
    RGS_ERR_STATE = 7      /* call out of order (e.g. adjoint before solve) */
} rgs_status;

typedef enum rgs_alpha_model {
    RGS_ALPHA_GAUSS = 0, /* alpha = o * exp(-(u^2+v^2)/2) for u^2+v^2 <= 9 (3-sigma cutoff) */
    RGS_ALPHA_DISC = 1,  /* alpha = o for u^2+v^2 <= 1, else 0 (closed-sphere furnace test) */
    RGS_ALPHA_GFSGS = 2  /* App. E: alpha = 1 - exp(-0.03279 (o exp(-(u^2+v^2)/2))^3.4) for u^2+v^2 <= 9,
                            o the unbounded opacity parameter g; the receiver's own alpha_i(p_i)
                            (the o_i factor of the other models) is 1 - exp(-0.03279 o_i^3.4) */
} rgs_alpha_model;

/* Precision of the bounce gathers (the batched form of the contraction).  Every mode
 * accumulates in FP32 and keeps FP32 iterates; the BF16 modes gather BF16 copies of the
 * iterate rows (half the bytes per hit).  RESCORR runs bounces 1..n-1 on BF16 rows and the
 * last bounce on FP32 rows: one FP32 residual-correction sweep that damps the BF16 error by
 * the spectral radius of K. */
typedef enum rgs_precision {
    RGS_FP32 = 0,
    RGS_BF16_FP32ACC = 1,
    RGS_BF16_FP32ACC_RESCORR = 2
} rgs_precision;

typedef struct rgs_scene rgs_scene;         /* opaque: surfels in Morton order + BVH */
typedef struct rgs_transport rgs_transport; /* opaque: hit records, direct term, iterates */

/* Surfel parameters, caller order, all device pointers (Sec. 3.1, Eq. G; Sec. 5.1, Eq. brdf):
 *   p[N][3]   centre p_i                tu[N][3], tv[N][3]  tangent directions t^u, t^v
 *   s[N][2]   scales (s^u, s^v) > 0     o[N]                opacity in [0, 1]
 *   ad[N][3]  diffuse albedo a^d        k[N]                diffuse/specular blend k
 *   as[N][3]  specular albedo a^s       shin[N]             Phong shininess s >= 0
 * The normal is n = t^u x t^v after Gram-Schmidt orthonormalisation of (t^u, t^v). */
typedef struct rgs_surfels {
    int32_t n;         /* N >= 1 */
    int32_t sh_degree; /* L in [0, RGS_MAX_SH_DEGREE] */
    const float *p, *tu, *tv, *s, *o, *ad, *k, *as, *shin;
} rgs_surfels;

typedef struct rgs_build_opts {
    int32_t alpha_model;  /* rgs_alpha_model */
    int32_t check_finite; /* nonzero: reject NaN/Inf inputs with RGS_ERR_NONFINITE (synchronises) */
} rgs_build_opts;

/* Point lights (Sec. 5.1 "Lighting", Sec. 5.3): infinitesimal emitters sampled at their
 * centre, isotropic, intensity I (RGB) so that the received radiance is I / r^2.
 * Directional lights (directional != 0; Sec. 5.1: "far away" point lights without the
 * inverse-square falloff, and the 16 x 32 environment map of Sec. 9 as such lights): pos
 * is the direction towards the light (any length), intensity the irradiance it gives a
 * surface facing it, no 1/r^2, and shadow rays run to infinity.
 * Device pointers pos[NL][3], intensity[NL][3]; NL may be 0.  All lights of a call are of
 * one kind. */
typedef struct rgs_lights {
    int32_t n_lights;
    int32_t directional;
    const float *pos;
    const float *intensity;
} rgs_lights;

typedef struct rgs_trace_opts {
    int32_t nd;           /* hemisphere rays per surfel: multiple of 32 in [32, 4096] */
    int32_t reserved0;
    uint64_t seed;        /* jitter seed of the stratified directions */
    int64_t hit_capacity; /* hit-record slots to reserve; 0 = automatic (grown on demand) */
} rgs_trace_opts;

/* Options of the center-to-center transport (rgs_trace_pairs). */
typedef struct rgs_pair_opts {
    const float *lambda; /* device [N]: the per-surfel scale lambda_j of Sec. 8, or NULL (all 1) */
} rgs_pair_opts;

typedef struct rgs_solve_stats {
    int32_t n_bounces;
    int32_t n_cols;
    double residual_norm[RGS_MAX_BOUNCES]; /* FP64 ||B^(k) - B^(k-1)||_2 over all columns */
    int64_t n_hits;          /* stored hemisphere hit records */
    int64_t n_hit_slots;     /* reserved record slots actually used (with warp padding) */
    int64_t n_full_rays;     /* rays truncated: their nearest-hit buffer filled before the
                                transmittance fell below the compositing cut */
} rgs_solve_stats;

typedef struct rgs_transport_info {
    int32_t n, sh_degree, nc, n_cols, nd, n_lights;
    int64_t n_hits, n_hit_slots, n_full_rays; /* center-to-center: pairs, pairs, 0 */
    int64_t device_bytes; /* device memory held by the transport handle (not counting the shared
                             workspace pool that rgs_adjoint and rgs_get_iterate draw from) */
} rgs_transport_info;

/* ---------------------------------------------------------------- entry points */

/* Builds (or rebuilds in place) the scene: orthonormal frames and normals (Eq. G), the
 * BRDF coefficients c_{i,l,ch} of the diffuse + Phong mixture (Eq. brdf; App. A: l = 0:
 * 4 k a^d + (1-k) a^s, l >= 1: (1-k) a^s rho_l(s)), the Morton order of the centres and
 * a BVH over the surfels' cutoff ellipses.
 *   surfels : host struct of device pointers (read only during the call's GPU work).
 *   opts    : host, may be NULL (Gaussian model, no finite check).
 *   inout   : host; *inout == NULL creates a handle, otherwise the handle is rebuilt and
 *             its buffers reused when large enough (no allocation in steady state).
 * Asynchronous unless opts->check_finite is set.  Errors: RGS_ERR_ARG, RGS_ERR_OOM,
 * RGS_ERR_CUDA, RGS_ERR_NONFINITE.  On error *inout keeps its previous value. */
rgs_status rgs_build_scene(const rgs_surfels *surfels, const rgs_build_opts *opts, void *stream, rgs_scene **inout);

/* Traces N * nd stratified cosine-weighted hemisphere rays from the surfel centres over
 * their front hemispheres (App. B; weight pi/nd), alpha-composites the hits in depth order
 * (Eq. L_I) and stores per-ray hit records (source surfel, compositing weight: 8 bytes
 * per hit); traces the N * NL shadow rays of the direct term (Sec. 5.2) and forms
 * S = E + D (E added in rgs_solve).  Rays start at the surfel centre (kappa_i = Dirac),
 * a surfel never hits itself (Sec. 5.1) nor planes within eps = 1e-5 * (bounding-box
 * diagonal) of the ray origin; compositing stops once the transmittance drops below 1e-6.
 *   scene  : built scene.  lights: host struct of device pointers (copied during the call).
 *   opts   : host.  inout: as in rgs_build_scene.
 * Synchronises `stream` (the record count decides the buffer size).  Errors: RGS_ERR_ARG,
 * RGS_ERR_OOM, RGS_ERR_CUDA, RGS_ERR_CAPACITY (opts->hit_capacity too small). */
rgs_status rgs_trace_transport(rgs_scene *scene, const rgs_lights *lights, const rgs_trace_opts *opts, void *stream,
                               rgs_transport **inout);

/* Center-to-center transport (Sec. 8, the approximated forward rendering equation): one
 * segment per pair of surfel centres instead of hemisphere rays,
 *   (K B)_i = o_i c_i (x) sum_j Y(R_i d) V_ji Y(-d)^T B_j,   d = (p_j - p_i)/|p_j - p_i|,
 *   V_ji = lambda_j (int alpha_j dx) T_ij |n_i.d| |n_j.d| / |p_j - p_i|^2,
 * over the sources j lying more than eps_plane in front of receiver i's plane.  T_ij is the
 * product of (1 - alpha_k) over the surfels k != i, j the open segment meets under the
 * hemisphere-ray hit rules whose plane lies more than eps_plane from p_j as well.
 * int alpha_j dx = 2 pi s^u s^v o (1 - e^{-9/2}) (Gaussian to 3 sigma), pi s^u s^v o
 * (disc) or, for the GFSGS model, App. E's closed form (2 pi / 3.4) s^u s^v Ein(c) with
 * c = 0.03279 o^3.4 and Ein(c) = int_0^c (1 - e^{-y}) / y dy.  The direct term is that of rgs_trace_transport.  The result is a transport
 * handle that rgs_solve, rgs_get_iterate and rgs_adjoint accept (every iterate is kept;
 * rgs_solve_batched does not take it).  Cost: N^2 front tests and one segment trace per
 * front pair; memory 8 bytes per pair.
 *   opts : host, may be NULL (lambda = 1).  Other arguments as rgs_trace_transport.
 * Synchronises `stream` (the pair count decides the buffer size).  Errors: RGS_ERR_ARG,
 * RGS_ERR_OOM, RGS_ERR_CUDA, RGS_ERR_CAPACITY (traversal stack). */
rgs_status rgs_trace_pairs(rgs_scene *scene, const rgs_lights *lights, const rgs_pair_opts *opts, void *stream,
                           rgs_transport **inout);

/* rgs_adjoint for a center-to-center transport, with the gradient of L with respect to
 * lambda as well:  dL/dlambda_j = sum over pairs (i -> j) of g_ij V_ji / lambda_j, where
 * g_ij = dL/dV_ji; dL/do adds the source term through int alpha_j and the occluders of
 * every pair's segment.  dL_dlambda: device [N] or NULL; the rest as rgs_adjoint.
 * Asynchronous.  Errors: RGS_ERR_ARG (not a center-to-center transport), RGS_ERR_STATE,
 * RGS_ERR_OOM, RGS_ERR_CUDA. */
rgs_status rgs_adjoint_pairs(rgs_transport *t, const float *dL_dB, float *dL_dE, float *dL_dalbedo,
                             float *dL_dopacity, float *dL_dlambda, void *stream);

/* rgs_adjoint_pairs with the geometry gradients as well (Sec. 6, Eqs. dl-dgeo-0 and
 * dl-dgeo-1, App. C), with respect to the surfel centres, scales and frame inputs:
 *   - the decay term V_ji = lambda_j A_j T_ij |n_i.d| |n_j.d| / r^2 of every pair moves with
 *     p_i and p_j (d = (p_j - p_i)/r and r), with s^u_j, s^v_j (A_j is proportional to
 *     s^u_j s^v_j) and with the centre and scales of every occluder k of its segment
 *     (alpha_k is taken where the segment crosses k's plane);
 *   - the directional effects Y(R_i d) (receiver's BRDF lobe) and Y(-d) (source's
 *     radiance) move with d;
 *   - the direct term moves with p_i (the light direction, cos and 1/r^2 of a point light)
 *     and with its shadow occluders;
 *   - the normals enter geo, the lobe R_i and the direct term's cos, and every occluder's
 *     frame (t^u, t^v, n) its crossing point; the orthonormal frame's gradients are carried
 *     back through the Gram-Schmidt construction of rgs_build_scene (Eq. G) to the tu, tv
 *     the caller passed (unnormalised inputs are fine).
 * Discrete events (the front and eps_plane tests, the 3-sigma cutoff) are held fixed, so
 * this is the derivative of the smooth piece the scene lies on.
 *   dL_dp : device [N][3] (dL/dp_i, caller order) or NULL.
 *   dL_ds : device [N][2] (dL/ds^u_i, dL/ds^v_i) or NULL.
 *   dL_dtu, dL_dtv : device [N][3] (dL/dtu_i, dL/dtv_i of the frame inputs) or NULL.
 *   the rest as rgs_adjoint_pairs (every output may be NULL).
 * Asynchronous.  Errors as rgs_adjoint_pairs. */
rgs_status rgs_adjoint_pairs_geometry(rgs_transport *t, const float *dL_dB, float *dL_dE, float *dL_dalbedo,
                                      float *dL_dopacity, float *dL_dlambda, float *dL_dp, float *dL_ds,
                                      float *dL_dtu, float *dL_dtv, void *stream);

/* rgs_adjoint with the geometry gradients as well (Sec. 6, Eqs. dl-dgeo-0/1, App. C),
 * for either transport (a center-to-center transport gives what rgs_adjoint_pairs_geometry
 * gives, without dL/dlambda).  For the hemisphere rays (rgs_trace_transport):
 *   - every stored hit's alpha moves with its point on the source's plane, which moves with
 *     the receiver's centre p_i, the ray's direction and the source's centre, scales and
 *     frame (the hit set and depth order are held fixed); the compositing weights pass the
 *     derivative on as in the opacity gradient;
 *   - the directional effects Y(R_i d) and Y(-d) of every ray move with its direction;
 *   - each ray leaves p_i along a direction fixed in the receiver's frame (its stratum and
 *     jitter), so the frame's gradient collects the ray directions';
 *   - the direct term as in rgs_adjoint_pairs_geometry.
 * The hemisphere form needs every iterate: it returns RGS_ERR_STATE after a checkpointed
 * solve (rgs_set_checkpointing with a stride other than 0).
 *   dL_dp, dL_ds, dL_dtu, dL_dtv : device [N][3], [N][2], [N][3], [N][3] (caller order), or
 *   NULL; the rest as rgs_adjoint.
 * Asynchronous.  Errors: RGS_ERR_ARG, RGS_ERR_STATE, RGS_ERR_OOM, RGS_ERR_CUDA. */
rgs_status rgs_adjoint_geometry(rgs_transport *t, const float *dL_dB, float *dL_dE, float *dL_dalbedo,
                                float *dL_dopacity, float *dL_dp, float *dL_ds, float *dL_dtu, float *dL_dtv,
                                void *stream);

/* Runs B^(0) = S = E + D, B^(k) = S + K B^(k-1) for k = 1..n_bounces with
 * (K B)_i = o_i c_i (x) sum_r (pi/nd) Y(R_i d_r) sum_h a_rh Y(-d_r)^T B_{j_h}
 * (Eq. final-radiosity with the hemisphere integral taken by the traced rays;
 * R_i d = 2 (n_i.d) n_i - d places the Phong lobe, Eq. sh-brdf) and keeps every
 * iterate for rgs_adjoint.
 *   E      : device [N][nc][3] emission coefficients, or NULL for zero emission.
 *   B_out  : device [N][nc][C], receives B^(n_bounces).
 *   stats  : host, may be NULL; if given, the stream is synchronised and the FP64
 *            residual norms per bounce are written.
 * Errors: RGS_ERR_ARG (n_bounces outside [0, RGS_MAX_BOUNCES], unknown precision),
 * RGS_ERR_CUDA, RGS_ERR_OOM. */
rgs_status rgs_solve(rgs_transport *t, const float *E, int32_t n_bounces, int32_t precision, float *B_out,
                     rgs_solve_stats *stats, void *stream);

/* Exact gradients of a loss L(B^(n)) for the last rgs_solve (the truncated series; the
 * paper's Eq. final_dL_dE / final-dl-dbrdf are its n -> infinity limit):
 *   v^(0) = dL/dB, v^(a) = K^T v^(a-1), u = sum_a v^(a) = dL/dS
 *   dL/dE[i][k][ch]  = sum over lights of u                                 (device [N][nc][3])
 *   dL/da^d[i][ch]   = 4 k_i alpha_i sum_{light} ( sum_a v^(a) Q^(n-1-a) + u Dgeo )_00  (device [N][3]),
 *                      alpha_i = alpha_i(p_i): o_i, or 1 - exp(-0.03279 o_i^3.4) for GFSGS
 *   dL/do[i]         = receiver factor + backward through the compositing of every
 *                      hemisphere and shadow ray that hits surfel i           (device [N])
 * Each output may be NULL (not computed).  dL_dB: device [N][nc][C].
 * K^T is a gather over the hit records grouped by source surfel; that transposed index is
 * built at the start of every call, in the workspace pool (see rgs_trim_workspace) with
 * the call's other scratch, and returned to the pool at its end.  After a checkpointed
 * solve (rgs_set_checkpointing) the iterates between checkpoints are recomputed here.
 * Asynchronous.  Errors: RGS_ERR_STATE (no prior rgs_solve), RGS_ERR_ARG, RGS_ERR_OOM,
 * RGS_ERR_CUDA. */
rgs_status rgs_adjoint(rgs_transport *t, const float *dL_dB, float *dL_dE, float *dL_dalbedo, float *dL_dopacity,
                       void *stream);

typedef struct rgs_batch_opts {
    int32_t precision;  /* rgs_precision, for every scene of the batch */
    int32_t use_graph;  /* nonzero: capture the batch's launches into a CUDA graph on the first call with
                           these arguments and replay the graph on later calls */
    int32_t autotune;   /* nonzero: on the first call, time the candidate numbers of resident blocks per SM
                           of the persistent kernel and keep the fastest */
    int32_t spin_limit; /* polls of each inter-bounce grid-barrier wait before the kernel gives up with
                           RGS_ERR_TIMEOUT; 0 = default (about a second) */
} rgs_batch_opts;

/* Solves `count` traced transports together -- scenes of uneven surfel count, SH degree, rays
 * per surfel and bounce count (the batching of right-hand sides and scenes; Sec. 7 hybrid solver,
 * Eq. final-radiosity per scene).  S = E + D is formed per scene; then every bounce of every scene
 * runs in one persistent cooperative kernel whose blocks take (scene, receiver, 3-column tile)
 * items from one queue per bounce level, with a bounded grid barrier between levels.  Each
 * transport keeps its iterates, so rgs_adjoint and rgs_get_iterate work per scene afterwards.
 *   ts        : host array of count traced transports (distinct).
 *   E         : host array of count device pointers [N_s][nc_s][3] (entries may be NULL), or NULL.
 *   n_bounces : host array of count bounce counts in [0, RGS_MAX_BOUNCES].
 *   opts      : host, may be NULL (FP32, graph, autotune, default wait limit).
 *   B_out     : host array of count device pointers [N_s][nc_s][C_s] (entries may be NULL), or NULL.
 *   residual_norms : host [count][RGS_MAX_BOUNCES] FP64 norms per bounce, or NULL.
 * Launch plans (device descriptors, graph, tuned shape) are cached per argument set; the first
 * call with new arguments also runs the autotuning candidates.  Synchronises `stream` (the
 * device-side timeout flag is read back).  Errors: RGS_ERR_ARG, RGS_ERR_STATE (untraced
 * transport), RGS_ERR_OOM, RGS_ERR_CUDA, RGS_ERR_TIMEOUT (a barrier wait ran out; the iterates
 * of the batch are then invalid, the context stays usable). */
rgs_status rgs_solve_batched(rgs_transport *const *ts, int32_t count, const float *const *E,
                             const int32_t *n_bounces, const rgs_batch_opts *opts, float *const *B_out,
                             double *residual_norms, void *stream);

/* The plan of the last rgs_solve_batched call (host-only, no device work): writes up to n
 * values to out and returns how many there are (-1 if no batched solve ran yet, or out is
 * NULL with n > 0).  Layout: [0] persistent blocks, [1] the kernel instance (2 or 3 resident
 * blocks per SM), [2] 1 if the plan was autotuned, [3] the number of buckets K (scenes with
 * equal nc, C and rays per surfel), then per bucket seven values: nc, C, rays per surfel,
 * the item-shape policy of its BF16-row and of its FP32-row levels (0 = 3-column items,
 * 1 = the measured crossover, 2 = 32-column items from 6 columns) and the item widths they
 * give (3 or 32 columns).  The autotuner times bounce level 1 for one policy shared by every
 * bucket with either kernel instance, then each bucket's policy in turn with the others
 * held, and in the corrected mode the same for the FP32-row level. */
int32_t rgs_batch_last_plan(int32_t *out, int32_t n);

/* Copies iterate B^(b) (0 <= b <= last n_bounces) of the last rgs_solve to the device
 * array out [N][nc][C].  An iterate that a checkpointed solve did not keep is recomputed
 * from the checkpoint below it (bit-identical to the solve's value) in pooled scratch.
 * Asynchronous.  Errors: RGS_ERR_STATE, RGS_ERR_ARG, RGS_ERR_OOM, RGS_ERR_CUDA. */
rgs_status rgs_get_iterate(rgs_transport *t, int32_t b, float *out, void *stream);

/* Iterate storage of the following rgs_solve calls on t (bounce-iterate checkpointing):
 *   stride = 0 : keep every B^(b) and Q^(b) for the adjoint (default, fastest adjoint);
 *   stride = s >= 1 : keep only the checkpoints B^(0), B^(s), B^(2s), ... below n_bounces and
 *                two running iterates; rgs_adjoint recomputes the others segment by segment
 *                from the checkpoint below them (one extra forward pass, bit-identical
 *                iterates), holding s iterates at a time;
 *   stride = -1 : automatic -- every iterate is kept when the solve's and the adjoint's
 *                buffers fit in free device memory, else s = ceil(sqrt(n_bounces)).
 * rgs_solve_batched always keeps every iterate.  Host-only.  Errors: RGS_ERR_ARG
 * (stride < -1 or > RGS_MAX_BOUNCES). */
rgs_status rgs_set_checkpointing(rgs_transport *t, int32_t stride);

/* Device-memory budget of t: the bytes its own buffers and the pooled scratch of its calls
 * may take (0 = no budget: the device's free memory decides).  It steers the two memory
 * choices the library makes on its own: the automatic checkpoint stride (stride -1 of
 * rgs_set_checkpointing) and the number of parts rgs_adjoint splits the transposed hit
 * index into (8 bytes per hit; each part is rebuilt from the records for every transposed
 * bounce, so more parts cost time, not accuracy).  Buffers the solve needs regardless are
 * allocated even above the budget.  Host-only.  Errors: RGS_ERR_ARG. */
rgs_status rgs_set_memory_budget(rgs_transport *t, int64_t bytes);

/* Which contraction the batched precision modes (RGS_BF16_FP32ACC, RGS_BF16_FP32ACC_RESCORR)
 * of the following rgs_solve / rgs_adjoint calls on a hemisphere transport with SH degree 3
 * use (Eq. final-radiosity; the many-light batching of Sec. 7):
 *   mode = -1 : automatic (default) -- the tensor-core form when C >= 96 columns and its
 *               buffers fit in free device memory, else the row-gather kernels;
 *   mode =  0 : always the row-gather kernels;
 *   mode =  1 : the tensor-core form whenever it applies (any C; still not for checkpointed
 *               solves, SH degree < 3, more than 2^20 surfels or 512 rays per surfel);
 *   mode =  2 : as 1, with the adjoint's opacity gather as per (source tile, receiver) group
 *               products (C / 16 products of 128 x 16 x 16 against the tile's sources' rows
 *               held in tensor memory; C <= 768): correct, but slower than mode 1's form;
 *   mode =  3 : as 1, with the adjoint's opacity gather as row gathers on the CUDA cores.
 * Modes -1 and 1 run the adjoint's opacity gather (g_h = sum_c y_r[c] (Y(-d)^T B_j[c]) per
 * stored hit, y_r = (pi/nd) o_i c_i (x) Y(R_i d_r)^T v_i per ray) as sampled products on the
 * tensor cores: the rays' y rows are formed once (BF16, at most 320 columns per pass; the
 * buffer takes 2 bytes per ray and column of a pass, sized to free device memory and to
 * half of what rgs_set_memory_budget leaves beside the transport's buffers), and per
 * tile of 8 sources and block of 128 of its hits a 128 x 128 product of the hits' gathered
 * y rows with the 8 sources' BF16 rows keeps each hit's own 16 entries.  Where no pass fits
 * in memory they fall back to mode 3's row gathers.
 * The tensor-core form regroups the hit records once per trace into tiles of 8 consecutive
 * receivers, and per tile into the sources they see; per (tile, source) it forms the 8
 * receivers' 16 x 16 transport blocks G_ij = sum_{r,h: j_h = j} a_rh Y(R_i d_r) Y(-d_r)^T as a
 * 128 x 16 BF16 operand and multiplies it with the source's BF16 rows (copied into shared
 * memory by the bulk-copy engine) on the tcgen05 tensor cores, FP32 accumulation in tensor
 * memory.  RGS_BF16_FP32ACC_RESCORR's last bounce splits both operands into BF16 high and low
 * parts (three products, FP32-level accuracy).  rgs_adjoint then runs the transposed bounces
 * the same way over tiles of 8 sources (y = o c (x) v rounded to BF16), with FP32 outputs.
 * Extra device memory: about 48 bytes per stored hit and three BF16 copies of an iterate.
 * Host-only.  Errors: RGS_ERR_ARG (NULL transport, mode outside [-1, 3]). */
rgs_status rgs_set_tensor_cores(rgs_transport *t, int32_t mode);

/* Sizes of the tensor-core contraction's pair tiles for t (built by the first solve or
 * adjoint that used the tensor-core form after the trace), written to out[0..5] (host):
 * receiver tiles, their (tile, source) groups, distinct (receiver, source) pairs, stored hits,
 * source tiles, their (tile, receiver) groups; zeros where a structure is not built.  One
 * 16 x 16 transport block per pair is the algorithmic work of a bounce (2 * 256 * C flops
 * per pair); every group costs one 128 x C x 16 MMA.  Host-only.  Errors: RGS_ERR_ARG
 * (NULL t or out, n < 6). */
rgs_status rgs_contraction_info(const rgs_transport *t, int64_t *out, int32_t n);

/* Limit, in nanoseconds, of every wait inside the tensor-core contraction's pipeline (a
 * role waiting for a stage of source rows, an operand, a finished accumulator; 0 = default,
 * 4 s).  A wait that runs out makes every role of the kernel stop, wait (for at most a
 * second) for its own copies and MMAs in flight, free its tensor memory and return; the
 * solve or adjoint then returns RGS_ERR_TIMEOUT (the results are invalid, the context stays
 * usable).  The library's service watchdog for the contraction; its tests set a tiny limit.
 * Host-only.  Errors: RGS_ERR_ARG (NULL transport, negative limit). */
rgs_status rgs_set_wait_limit(rgs_transport *t, int64_t ns);

/* Image formation, Eq. L_I for the rays of a pinhole camera (what the paper draws with its
 * tile rasterizer from the surfels' outgoing radiance, Sec. 5.3): each pixel's ray
 * o + t d meets the surfels of t's scene in depth order under the transport's hit rules
 * (the eps_plane plane test, the Gaussian's cutoff, runs of near-equal depth ordered by caller
 * index; no surfel excluded), composited with a_h = alpha_h prod_{k<h} (1 - alpha_k) until the
 * transmittance falls below 1e-6 (any number of hits), and
 *     img[y][x][c] = sum_h a_h Y(-d)^T B_{j_h}[:, c].
 * cam: HOST float[9] = {o[3], forward[3], up[3]}; right = forward x up (normalised), the true
 * up = right x forward; fov is the vertical field of view in radians (0, pi); pixel (x, y),
 * y pointing down, is sampled at its centre.  B: device float [N][nc][C] in caller order (the
 * layout rgs_solve writes); img: device float [H][W][C], fully written.  Device buffers are
 * the caller's; pooled scratch (40 bytes per pixel and 8 per composited hit) is returned
 * before the call ends.  Every pixel ray is traced twice (count, then fill).  Synchronises
 * `stream` once (the record count and the traversal's overflow check).  Errors: RGS_ERR_ARG (NULL
 * pointer, W or H <= 0, W*H > 2^26, fov outside (0, pi)), RGS_ERR_NONFINITE (camera),
 * RGS_ERR_STATE (t not traced), RGS_ERR_CAPACITY (traversal stack), RGS_ERR_OOM,
 * RGS_ERR_CUDA. */
rgs_status rgs_render(rgs_transport *t, const float *B, const float *cam, int32_t W, int32_t H, float fov,
                      float *img, void *stream);

/* The transpose of rgs_render: dL_dB[j][k][c] = sum over pixels and their hits h on surfel j of
 * a_h Y_k(-d) dL_dimg[y][x][c] -- the dL/dB that a loss on the image hands to rgs_adjoint.
 * dL_dimg: device float [H][W][C]; dL_dB: device float [N][nc][C] in caller order, fully
 * written (overwritten, not accumulated).  Sums are formed with atomic adds, so the last bits
 * may differ from run to run.  Same camera, scratch, synchronisation and errors as
 * rgs_render. */
rgs_status rgs_render_adjoint(rgs_transport *t, const float *dL_dimg, const float *cam, int32_t W, int32_t H,
                              float fov, float *dL_dB, void *stream);

/* The Monte-Carlo TD(0) solver of Sec. 7 (Alg. 1) on a center-to-center transport (traced
 * by rgs_trace_pairs), with next-event estimation by weighted reservoir sampling and the
 * variance-driven receiver selection of App. "Monte-Carlo Solver Details":
 *   step t = 1..steps draws N estimates; draw q's receiver is a = q for t <= 8, afterwards a
 *   draw with replacement with probability proportional to the receivers' tracked variances
 *   (sum over coefficients of S2/D - (S/D)^2, plus 1e-30); its next event is one pair
 *   (a <- b) picked with probability p_b proportional to the proxy
 *     w_b = geo_ab (sum_c lum(c) |Y(-d)^T Bhat_b[:, c]| + floor),
 *   geo = |n_a.d||n_b.d|/r^2, lum the Rec. 709 weights (0.2126, 0.7152, 0.0722) of each
 *   column's colour channel, floor = 1e-9 (1 + sum of lum |Bhat| / N); with groups > 0 the
 *   surfels are first grouped by K-means on centre and normal and the pick is a group by
 *   its proxy, then a pair of a inside it (p_b the product).  The estimate
 *   delta = S_a + (1/p_b) K_ab Bhat_b enters a's FP64 sums (S += delta, S2 += delta^2,
 *   D += 1); Bhat = S / D after every step, and every draw reads the previous step's means.
 * Random numbers: u = (SplitMix64(k) >> 11) * 2^-53 with
 * k = SplitMix64(SplitMix64(SplitMix64(seed) + t) + q) + stream, stream 0 for the receiver
 * selection and 1000 + k for the k-th candidate of a reservoir (the group stage uses draw
 * q + 2^30); a's candidates are its pairs in increasing caller index of the source (the
 * order rgs_trace_pairs stores them in) or the groups in index order.
 * E: device [N][nc][3] or NULL (no emission); S_in: device [N][nc][C] or NULL -- when given
 * it replaces S = E + D (the direct term), e.g. the unshot radiance of a shooting solver.
 * B_out: device [N][nc][C], the means after `steps` steps (zero for a receiver never
 * visited); visits: device float [N] or NULL, each receiver's estimate count.  Scratch:
 * about 24 bytes per entry of B from the workspace pool.  Synchronises `stream` per K-means
 * iteration the first time a group count is used on t.  Errors: RGS_ERR_ARG (NULL t or
 * B_out, a hemisphere transport, steps < 0, groups outside [0, min(1024, N)]),
 * RGS_ERR_STATE (t not traced), RGS_ERR_OOM, RGS_ERR_CUDA. */
rgs_status rgs_mc_solve(rgs_transport *t, const float *E, const float *S_in, int32_t steps, uint64_t seed,
                        int32_t groups, float *B_out, float *visits, void *stream);

/* One step's next-event estimates for given means, the building block of rgs_mc_solve:
 * draw q (0 <= q < n_draws) uses the keys (seed, step, q), receiver recv[q] (device int32
 * [n_draws], caller indices; NULL: receiver q, then n_draws <= N) and the means Bhat
 * (device [N][nc][C]).  Writes pick[q] (device int64: the picked pair's index among the
 * receiver's pairs in increasing caller index of the source, -1 if the receiver has none),
 * p[q] (device double: its probability, 0 without a pick) and delta (device float
 * [n_draws][nc][C], S_a + K_ab Bhat_b / p_b with S = E + D).  Synchronises `stream` (the
 * check of recv).  Errors: RGS_ERR_ARG (NULL pointers, step < 1, n_draws < 0, n_draws > N
 * without recv, a receiver outside [0, N), groups outside [0, min(1024, N)]), RGS_ERR_STATE,
 * RGS_ERR_OOM, RGS_ERR_CUDA. */
rgs_status rgs_mc_estimate(rgs_transport *t, const float *E, const float *Bhat, uint64_t seed, int32_t step,
                           int32_t groups, int32_t n_draws, const int32_t *recv, int64_t *pick, double *p,
                           float *delta, void *stream);

/* The K-means groups the solver's grouped proposal uses (App. "Monte-Carlo Solver
 * Details"): Lloyd's iterations in FP64 on the features (p, (extent / 2) n), extent the
 * scene's largest side, from the surfels with caller indices floor(k N / groups), until no
 * assignment changes (at most 50).  assign: device int32 [N], caller order.  The result is
 * cached on t until its next trace.  Errors: as rgs_mc_solve, groups in [1, min(1024, N)]. */
rgs_status rgs_mc_groups(rgs_transport *t, int32_t groups, int32_t *assign, void *stream);

/* Progressive refinement (the shooting solver of Sec. 7) on a center-to-center transport:
 * Bhat = dB = S = E + D, then `shots` times the surfel whose unshot radiance has the largest
 * luminance (sum over its coefficients and columns of lum(c) |dB|, the Rec. 709 weights of
 * each column's channel; ties to the lower caller index) sends it to every receiver a that
 * has it as a source, dB_a += K_a,b dB_b and Bhat_a += K_a,b dB_b, and its dB is cleared;
 * once no unshot radiance is left the remaining shots do nothing.  The remaining problem
 * B^r = dB + K B^r is again the full transport, so B = Bhat + B^r - dB exactly: running
 * rgs_mc_solve with S_in = dB and combining gives the paper's hybrid solver.  Bhat_out,
 * dB_out: device [N][nc][C].  Three launches per shot.  Errors: RGS_ERR_ARG (NULL t or
 * output, shots < 0, a hemisphere transport), RGS_ERR_STATE, RGS_ERR_OOM, RGS_ERR_CUDA. */
rgs_status rgs_prog_refine(rgs_transport *t, const float *E, int32_t shots, float *Bhat_out, float *dB_out,
                           void *stream);

/* Workspace pool: the per-call scratch of rgs_adjoint (the transposed hit index, 8 bytes per
 * hit; per-hit opacity sums, 4 bytes; v^(a) and u; per-ray adjoint values) and of
 * rgs_get_iterate comes from one stream-ordered memory pool per device, so transports used
 * one after another on a stream share it.  The pool keeps its memory reserved between calls;
 * this returns the unused part to the device.  Synchronises the current device.
 * Errors: RGS_ERR_CUDA. */
rgs_status rgs_trim_workspace(void);

/* FP64 residual norm ||x - y||_2 of two device float arrays of n elements, written to the
 * device double *norm_out -- the same quantity rgs_solve reports per bounce, for two
 * iterates the caller holds.  The paper has no counterpart: this is a library service.
 *
 * It allocates no device memory, for callers that cannot: a host application that has
 * reserved its whole device-memory budget and passes the library only buffers it owns,
 * or a latency-critical loop that must not pay cudaMalloc's device-wide synchronisation.
 * Its scratch (one FP64 partial per 8192-element block, 8192 blocks = 64 KiB) is a static
 * device array inside librgs.so that every GPU loading the library keeps until exit.
 *   x, y     : device float arrays, n elements each (caller-owned, read only).
 *   n        : 0 <= n <= 8192 * 8192 = 67,108,864; larger n returns RGS_ERR_ARG; n = 0
 *              writes 0.
 *   norm_out : device double (caller-owned), written on `stream`.
 * x, y and norm_out must live on the current device; the kernels run there.
 * The first call on each device looks up the scratch's device address (with that device
 * current) and caches it for the life of the process; make that first call before any
 * stream capture, and do not use this entry point after a device reset (cudaDeviceReset
 * reloads the library's device image and leaves the cached address stale).  All calls share
 * the one scratch array, which keeps the last call's contents (each call writes every slot
 * it reads, so nothing needs clearing); calls that overlap on the GPU -- on different
 * streams, or from different host threads -- race on it and must be serialised.
 * Asynchronous.  Errors: RGS_ERR_ARG, RGS_ERR_CUDA. */
rgs_status rgs_residual_norm_noalloc(const float *x, const float *y, int64_t n, double *norm_out, void *stream);

/* Fills *info (host).  Synchronises nothing.  Errors: RGS_ERR_ARG. */
rgs_status rgs_transport_info_get(const rgs_transport *t, rgs_transport_info *info);

/* Release handles (NULL is accepted).  Synchronises the device. */
void rgs_destroy_transport(rgs_transport *t);
void rgs_destroy_scene(rgs_scene *s);

/* ---------------------------------------------------------------- profiling
 * Per-kernel timing for roofline reports.  While enabled, every kernel the library
 * launches is bracketed by two CUDA events recorded on the stream it is launched on;
 * rgs_profile_report synchronises those events and returns, per kernel name, the
 * number of launches and their summed device time.  rgs_launch_count counts every
 * kernel launched by the library since it was loaded (enabled or not). */
typedef struct rgs_kernel_time {
    char name[32];
    int64_t launches;
    double total_ms;
} rgs_kernel_time;

void rgs_profile_enable(int32_t on);
void rgs_profile_reset(void);
/* Writes up to max entries to out (host); returns the number of kernel names seen, or -1
 * if out is NULL with max > 0 or an event could not be read (see rgs_last_error).
 * Synchronises on the events. */
int32_t rgs_profile_report(rgs_kernel_time *out, int32_t max);
int64_t rgs_launch_count(void);

const char *rgs_status_string(rgs_status s);
const char *rgs_last_error(void); /* thread-local message of the last failing call */
int32_t rgs_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RGS_H */
