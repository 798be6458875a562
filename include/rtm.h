/*
 * librtm -- C ABI of the GB300 (sm_103a) RTM hot path.
 *
 * The method: reverse time migration as the paper describes it (Sec. I):
 * pressure waves are simulated forward from the source and backward from the
 * recorded data, and the two wavefields are correlated into an image. The
 * solver applies a high-order stencil to a 3D block in every time step
 * (Sec. II). The paper gives no formulas; the discrete method implemented
 * here is:
 *
 *   L u       = sum over x, y, z of [a0 u + sum_{k=1..r} a_k (u_{+k} + u_{-k})] / dx^2
 *               (2r-order central weights, zero ghost cells outside the padded grid)
 *   u^{n+1}   = g (2 u^n + c L u^n) - g^2 u^{n-1},   c = v^2 dt^2,  g = gx gy gz
 *   u^{n+1}[s]  += c[s] w(n dt) / dx^3,   w = Ricker(f0, t0)
 *   d[n][j]   = u^{n+1}[rec_j]
 *   mu^m      = g (2 mu^{m+1} + c L mu^{m+1}) - g^2 mu^{m+2},  m = nt..1  (mu^{nt+1} = mu^{nt+2} = 0)
 *   mu^m[rec_j] += c g r^{m-1}_j / dx^3
 *   I(x)     += u^m(x) mu^m(x)    on the model region, for m % image_every == 0
 *
 * with a sponge g_a(d) = exp(-(0.015 (nb - d))^2) for cells at distance
 * d < nb from an outer face and 1 elsewhere. The backward recursion is the
 * exact transpose of the forward one in the scaled variable
 * mu = C G lambda / dx^3, so the same kernel runs in both directions.
 *
 * Conventions for every call:
 *  - Grids are float32, C order [z][y][x], x contiguous (the x-innermost
 *    loop order the paper settles on in Sec. III).
 *  - The model grid is nx * ny * nz. The padded (computational) grid adds nb
 *    sponge cells on all six faces: NX = nx + 2 nb, etc. NX must be a
 *    multiple of 4 so that every row starts on a 16-byte boundary.
 *  - Every array argument is caller-owned memory. Pointers named d_* are
 *    device pointers, h_* host pointers. The library never allocates device
 *    memory and never frees caller memory: all scratch lives in the caller's
 *    workspace (the paper's lesson of passing pointers instead of copying
 *    data, Sec. III). Device pointers must be 16-byte aligned; the workspace
 *    256-byte aligned.
 *  - Calls are asynchronous on the given stream (NULL = legacy default
 *    stream) unless stated otherwise. Host-side argument checks run before any
 *    launch and return RTM_ERR_INVALID without touching the device.
 *    Device-side checks (receiver coordinates out of range, bounded waits)
 *    write a status word in the workspace; rtm_check() reads and clears it.
 *    rtm_forward and rtm_shot clear it when they start, so it reports the
 *    device-side errors of the pipeline started by the latest forward pass.
 *  - On any error the thread-local message of rtm_last_error() says why.
 */
#ifndef RTM_H
#define RTM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *rtm_stream; /* the same handle as cudaStream_t */

typedef enum {
    RTM_OK = 0,
    RTM_ERR_INVALID = 1,     /* an argument is out of range */
    RTM_ERR_CFL = 2,         /* dt above the leapfrog stability limit */
    RTM_ERR_WORKSPACE = 3,   /* workspace missing, too small or misaligned */
    RTM_ERR_CUDA = 4,        /* a CUDA runtime call failed */
    RTM_ERR_TIMEOUT = 5,     /* a bounded device-side wait ran out */
    RTM_ERR_NUMERIC = 6,     /* non-finite or non-positive model values, or a
                                run whose fields hold non-finite values */
    RTM_ERR_UNSUPPORTED = 7, /* e.g. a stencil radius other than 4 or 8 */
    RTM_ERR_STATE = 8        /* workspace prepared for another purpose */
} rtm_status;

enum { RTM_STORE_ALL = 0, RTM_STORE_CKPT = 1, RTM_STORE_LEARNED = 2, RTM_STORE_REVOLVE = 3,
       RTM_STORE_BOUNDARY = 4, RTM_STORE_DECIMATED = 5 };
enum { RTM_VEL_V = 0, RTM_VEL_V2 = 1 };

typedef struct {
    int32_t nx, ny, nz;     /* model grid */
    int32_t nb;             /* sponge width (cells, each face) */
    int32_t radius;         /* stencil radius r: 4 (8th order) or 8 (16th order) */
    int32_t nt;             /* time steps */
    double dx;              /* grid spacing (m) */
    double dt;              /* time step (s) */
    double f0;              /* Ricker peak frequency (Hz) */
    double t0;              /* Ricker delay (s) */
    int32_t src_x, src_y, src_z; /* source, model coordinates in [-nb, n + nb) */
    int32_t nrec;           /* receivers */
    int32_t storage;        /* RTM_STORE_ALL: keep every imaging snapshot;
                               RTM_STORE_CKPT: checkpoints + segment recompute;
                               RTM_STORE_LEARNED: an 8x autoencoder latent per
                               imaging snapshot (the *_learned calls);
                               RTM_STORE_REVOLVE: binomial checkpointing in a
                               fixed number of slots (imaging only);
                               RTM_STORE_BOUNDARY: the model region's boundary
                               band of every state, the source wavefield
                               recovered by reverse time stepping (imaging
                               only; model sides above 2 radius);
                               RTM_STORE_DECIMATED: the non-learned 8x scheme
                               beside learned storage: every other model
                               sample per axis of each imaging snapshot, kept
                               in float32 ([(nz+1)/2][(ny+1)/2][(nx+1)/2]) and
                               rebuilt by linear interpolation along each
                               axis (the last odd sample copies its left
                               neighbour) before the imaging step (imaging
                               only; rtm_forward / rtm_backward_image /
                               rtm_shot) */
    int32_t ckpt_every;     /* steps per checkpoint segment (RTM_STORE_CKPT);
                               number of checkpoint slots (RTM_STORE_REVOLVE);
                               exact window (RTM_STORE_LEARNED,
                               RTM_STORE_DECIMATED): the imaging snapshots of
                               steps 1..ckpt_every are recomputed from the
                               zero initial state in the backward call
                               instead of being coded (0: none) */
    int32_t image_every;    /* image at steps m with m % image_every == 0 (>= 1) */
    int32_t want_grad;      /* 1: prepare the workspace for rtm_grad instead of imaging */
} rtm_params;

/* Per-kernel-class device time, filled when timing is enabled. */
typedef struct {
    int64_t launches;       /* kernel launches of this library since the last reset */
    int64_t stencil_launches[7];  /* per stencil mode: fwd, fwd+snap, bwd+image,
                                     fwd+Lu, bwd+grad, batched, reverse */
    double stencil_ms[7];   /* summed CUDA-event time per stencil mode */
    double stencil_bytes[7];/* summed algorithmic bytes per stencil mode */
} rtm_stats;

/* Library version string. */
const char *rtm_version(void);

/* Thread-local description of the last error returned on this thread. */
const char *rtm_last_error(void);

/* Host-only argument checks of a parameter block (no device access). */
rtm_status rtm_validate(const rtm_params *p);

/* Workspace bytes that rtm_forward / rtm_backward_image / rtm_shot / rtm_grad
 * need for p (0 if p is invalid). The same workspace must be passed to the
 * forward call and to the backward call that consumes its snapshots or
 * checkpoints. A checkpointed backward call recomputes each segment in place
 * in its checkpoint slot, so one forward call feeds one backward call;
 * store-all and learned storage may be imaged more than once. */
size_t rtm_workspace_size(const rtm_params *p);

/* Model preparation (the padded coefficient grid).
 *   d_vel  [nz][ny][nx] velocity (vel_kind RTM_VEL_V, m/s) or squared
 *          velocity (RTM_VEL_V2, m^2/s^2) on the model grid.
 *   d_c    [NZ][NY][NX] out: c = v^2 dt^2, each padded cell copying the
 *          nearest model cell.
 *   d_ws   any workspace of at least 256 bytes (its status block holds the
 *          reduction words).
 * Computes max v on the device and SYNCHRONISES the stream to check the
 * leapfrog stability limit vmax dt / dx <= 2 / sqrt(3 |S(pi)|) with
 * S(theta) = a0 + 2 sum_k a_k cos(k theta) (0.4529 for r = 4, 0.4237 for
 * r = 8): RTM_ERR_CFL if violated, RTM_ERR_NUMERIC if a value is not finite
 * and positive. */
rtm_status rtm_model_prep(const rtm_params *p, const float *d_vel, int32_t vel_kind,
                          float *d_c, void *d_ws, size_t ws_bytes, rtm_stream stream);

/* Forward modelling from zero initial fields.
 *   d_c     [NZ][NY][NX] coefficient grid from rtm_model_prep.
 *   d_rec   [nrec][3] int32 receiver model coordinates (x, y, z), each in
 *           [-nb, n + nb); receivers outside are skipped and flagged.
 *   d_data  [nt][nrec] out: d[n][j] = u^{n+1}[rec_j]; may be NULL.
 *   d_ws    workspace of rtm_workspace_size(p) bytes; receives the imaging
 *           snapshots (RTM_STORE_ALL) or the checkpoints (RTM_STORE_CKPT).
 *   d_u_last [2][NZ][NY][NX] out: u^{nt-1}, u^{nt}; may be NULL. */
rtm_status rtm_forward(const rtm_params *p, const float *d_c, const int32_t *d_rec,
                       float *d_data, void *d_ws, size_t ws_bytes, float *d_u_last,
                       rtm_stream stream);

/* Receiver propagation backward in time with the zero-lag imaging condition
 * fused into the backward stencil. Needs a preceding rtm_forward with the same
 * p, d_c, d_rec and d_ws on the same stream (want_grad = 0).
 *   d_rdata   [nt][nrec] data injected at the receivers (RTM: the recorded data).
 *   d_image   [nz][ny][nx] model grid, ACCUMULATED (+=), so shots sum.
 *   d_src_adj [nt] out: mu^{n+1}[s] / g_s, the transpose of the forward map
 *             evaluated on d_rdata (for dot-product tests); may be NULL. */
rtm_status rtm_backward_image(const rtm_params *p, const float *d_c, const int32_t *d_rec,
                              const float *d_rdata, void *d_ws, size_t ws_bytes,
                              float *d_image, float *d_src_adj, rtm_stream stream);

/* One RTM shot: rtm_forward then rtm_backward_image of d_dobs.
 *   d_data  [nt][nrec] out: the modelled data; may be NULL. */
rtm_status rtm_shot(const rtm_params *p, const float *d_c, const int32_t *d_rec,
                    const float *d_dobs, float *d_data, void *d_ws, size_t ws_bytes,
                    float *d_image, rtm_stream stream);

/* Gradient of J = 1/2 ||d - d_obs||^2 with respect to v^2 on the model grid,
 * given the residual d - d_obs. Needs a preceding rtm_forward with the same
 * p (want_grad = 1), d_c, d_rec and d_ws on the same stream.
 *   d_resid   [nt][nrec] residual r = d - d_obs.
 *   d_grad_v2 [nz][ny][nx] out (overwritten): dJ/d(v^2)
 *             = dt^2 * fold(dx^3 / c * sum_n mu^{n+1} (L u^n + [s] w^n / (dx^3 g_s))),
 *             fold = transpose of the edge padding. */
rtm_status rtm_grad(const rtm_params *p, const float *d_c, const int32_t *d_rec,
                    const float *d_resid, void *d_ws, size_t ws_bytes, float *d_grad_v2,
                    rtm_stream stream);

/* Learned storage (p->storage == RTM_STORE_LEARNED, model sides multiples of
 * 4): the forward pass encodes each imaging snapshot u^m (m % image_every ==
 * 0) into a bfloat16 latent in the workspace right after the stencil writes
 * it; the backward pass decodes it just before the backward stencil that
 * images with it. No checkpoints, no recompute. d_ae_params: the codec's
 * RTM_AE_NPARAMS float32 parameters (see rtm_ae_encode). Otherwise as
 * rtm_forward / rtm_backward_image / rtm_shot. */
rtm_status rtm_forward_learned(const rtm_params *p, const float *d_c, const int32_t *d_rec,
                               float *d_data, const float *d_ae_params, void *d_ws,
                               size_t ws_bytes, rtm_stream stream);
rtm_status rtm_backward_image_learned(const rtm_params *p, const float *d_c, const int32_t *d_rec,
                                      const float *d_rdata, const float *d_ae_params, void *d_ws,
                                      size_t ws_bytes, float *d_image, rtm_stream stream);
rtm_status rtm_shot_learned(const rtm_params *p, const float *d_c, const int32_t *d_rec,
                            const float *d_dobs, const float *d_ae_params, void *d_ws,
                            size_t ws_bytes, float *d_image, rtm_stream stream);

/* Copy the stored imaging snapshot u^m (m a multiple of image_every) of a
 * store-all imaging workspace, after rtm_forward, into d_out [nz][ny][nx]. */
rtm_status rtm_snapshot(const rtm_params *p, const void *d_ws, size_t ws_bytes, int32_t m,
                        float *d_out, rtm_stream stream);

/* Misfit: d_resid[i] = d_data[i] - d_obs[i]; *d_J = 1/2 sum d_resid^2
 * accumulated in float64 (overwritten). d_resid may be NULL. */
rtm_status rtm_misfit(const float *d_data, const float *d_obs, int64_t n, float *d_resid,
                      double *d_J, rtm_stream stream);

/* Workspace bytes for rtm_shot_host: rtm_workspace_size(p) plus device room
 * for the velocity, coefficients, receivers, data and image. */
size_t rtm_host_workspace_size(const rtm_params *p);

/* One RTM shot from HOST buffers, end to end: copies h_vel [nz][ny][nx],
 * h_rec [nrec][3] and h_dobs [nt][nrec] to the device workspace, prepares the
 * model, runs the shot and copies the image [nz][ny][nx] back into h_image
 * (overwritten). The observed data are copied on a private stream after the
 * velocity and receivers, while the model is prepared and the source is
 * propagated; the receiver pass waits for them. Pinned host memory makes
 * the copies asynchronous. Returns after the stream has been synchronised. */
rtm_status rtm_shot_host(const rtm_params *p, const float *h_vel, int32_t vel_kind,
                         const int32_t *h_rec, const float *h_dobs, float *h_image,
                         void *d_ws, size_t ws_bytes, rtm_stream stream);

/* Synchronise the stream, read and clear the device status word of the
 * workspace: RTM_OK, RTM_ERR_INVALID (a receiver out of range was skipped),
 * RTM_ERR_TIMEOUT (a bounded wait ran out), RTM_ERR_NUMERIC (the post-run
 * scan found a NaN or an infinity: every forward pass scans its newest
 * state u^nt, every receiver pass its image or gradient accumulator) or
 * RTM_ERR_CUDA. The first error recorded wins. */
rtm_status rtm_check(void *d_ws, size_t ws_bytes, rtm_stream stream);

/* ---- learned snapshot compression (tensor cores) ------------------------
 * A 4-layer 3D convolutional autoencoder compresses a float32 snapshot
 * [nz][ny][nx] (every side a multiple of 4) 8x, into a bfloat16 latent
 * [nz/4][ny/4][nx/4][16] plus one float32 scale (the snapshot's rms):
 *   x0 = s / rms(s); h1 = LeakyReLU(conv 1->32, kernel 2, stride 2);
 *   latent = conv 32->16 (kernel 3, stride 2, padding 1);
 *   g1 = LeakyReLU(transposed conv 16->32, kernel 4, stride 2, padding 1);
 *   s_hat = rms(s) * transposed conv 32->1 (kernel 2, stride 2).
 * Every convolution (forward, data gradient, weight gradient) runs as an
 * implicit GEMM on tcgen05 tensor cores (bfloat16 operands, float32
 * accumulation in tensor memory). The paper has no learned part; the codec
 * stands in for the recompute of the source wavefield in the imaging
 * condition. Parameters: RTM_AE_NPARAMS float32 in the order W1[32][2][2][2],
 * b1[32], W2[16][3][3][3][32], b2[16], W3[32][4][4][4][16], b3[32],
 * W4[2][2][2][32], b4[1]. Strides sy, sz are in elements (x contiguous). */
#define RTM_AE_NPARAMS 47185
size_t rtm_ae_param_count(void);
/* Workspace bytes for the codec calls on an nx * ny * nz volume (0 if a side
 * is not a positive multiple of 4). Its first word is a status word that
 * rtm_check reads. */
size_t rtm_ae_workspace_size(int32_t nx, int32_t ny, int32_t nz);
/* d_latent [nz/4][ny/4][nx/4][16] bfloat16 out; d_scale [1] out (may be NULL). */
rtm_status rtm_ae_encode(const float *d_params, const float *d_snap, int64_t sy, int64_t sz,
                         int32_t nx, int32_t ny, int32_t nz, uint16_t *d_latent, float *d_scale,
                         void *d_ws, size_t ws_bytes, rtm_stream stream);
/* d_out [nz][ny][nx] (strided) out = scale * decoder(latent); d_scale may be
 * NULL (scale 1). */
rtm_status rtm_ae_decode(const float *d_params, const uint16_t *d_latent, const float *d_scale,
                         float *d_out, int64_t sy, int64_t sz, int32_t nx, int32_t ny,
                         int32_t nz, void *d_ws, size_t ws_bytes, rtm_stream stream);
/* One training step on d_batch [batch][nz][ny][nx] (dense): the mean over
 * the batch of mean((y - x0)^2) in normalised units goes to *d_loss (float64),
 * its gradient (hand-written backward through every layer, gradient
 * operands rounded to bfloat16 for the tensor cores) to d_grad if not NULL,
 * then Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected at step >= 1,
 * gradient scaled to a global L2 norm of at most 1) updates d_params in
 * place unless lr <= 0. */
rtm_status rtm_ae_train_step(float *d_params, float *d_adam_m, float *d_adam_v, int32_t step,
                             float lr, const float *d_batch, int32_t batch, int32_t nx,
                             int32_t ny, int32_t nz, double *d_loss, float *d_grad, void *d_ws,
                             size_t ws_bytes, rtm_stream stream);
/* Inference decoder used by rtm_ae_decode and the learned-storage backward
 * pass: 0 automatic (the z-marching kernel: latent planes loaded by TMA and
 * read in place by the tensor cores, D1 and D2 fused, one persistent CTA per
 * SM; the GEMM-engine decoder when the driver has no tensor-map encoder),
 * 1 the GEMM-engine decoder, 2 the z-marching kernel where it can run.
 * Both give the same values. Process-wide; returns RTM_ERR_INVALID for other
 * values. */
rtm_status rtm_ae_set_decoder(int32_t which);
/* Inference encoder used by rtm_ae_encode and the learned-storage forward
 * pass: 0 automatic (the z-marching kernel: snapshot planes loaded by TMA,
 * E1 and E2 on the tensor cores with h1 kept in shared memory, one
 * persistent CTA per SM; the GEMM-engine encoder when the driver has no
 * tensor-map encoder or the snapshot rows are not 16-byte aligned), 1 the
 * GEMM-engine encoder, 2 the z-marching kernel where it can run. Both give
 * the same values. Process-wide; returns RTM_ERR_INVALID for other values. */
rtm_status rtm_ae_set_encoder(int32_t which);
/* The tensor-core engine under the codec, exposed for checking: C[M][N] =
 * A[M][K] * B[N][K]^T, bfloat16 in, float32 out, K a multiple of 32, N 16 or
 * 32. A bounded wait that runs out writes RTM_ERR_TIMEOUT to *d_status. */
rtm_status rtm_ae_gemm_bf16(const uint16_t *d_A, const uint16_t *d_B, float *d_C, int32_t M,
                            int32_t K, int32_t N, int32_t *d_status, rtm_stream stream);

/* ---- binomial checkpointing (RTM_STORE_REVOLVE) ----------------------------
 * The receiver pass needs the source wavefield at the imaging steps in
 * reverse order. With s = p->ckpt_every slots, each holding a leapfrog pair
 * (2 padded fields), the backward call recomputes the source states from the
 * zero initial state and the slots along the schedule with the fewest
 * forward steps T(n, s), n = nt / image_every imaging steps:
 *   T(0, s) = 0, T(n, 0) = n (n + 1) / 2,
 *   T(n, s) = min_{1 <= c <= n} [c + T(n - c, s - 1) + T(c - 1, s)],
 * in units of image_every forward steps (the recursion of binomial, or
 * revolve, checkpointing; the forward call stores nothing and only models
 * the data). Memory: s slots + one snapshot slab, independent of nt. The
 * planning table is O(n^2 s) host work, refused beyond n^2 s = 2e9.
 *
 * rtm_revolve_cost: T(n, s) in image_every-step units (-1 over the limit).
 * rtm_revolve_schedule: the action list into h_actions (host memory, 4
 * int32 per action: op, a, b, c; op 0 restore slot a (-1: zero state) holding
 * state b, 1 advance from state a to state b (c = 1: write the snapshot at
 * the end), 2 store state b in slot a, 3 deliver state a (b = -1: the working
 * pair, b >= 0: from slot b), 4 free slot a). Returns the number of actions;
 * if that exceeds max_actions nothing is written; -1 over the limit. */
int64_t rtm_revolve_cost(int32_t nstates, int32_t slots);
int32_t rtm_revolve_schedule(int32_t nstates, int32_t slots, int32_t *h_actions,
                             int32_t max_actions);

/* ---- boundary storage (RTM_STORE_BOUNDARY) ---------------------------------
 * The receiver pass needs the source wavefield at the imaging steps in
 * reverse order (Sec. I). Inside the model region the sponge factor is
 * exactly 1, so the forward update u^{n+1} = 2u^n + c L u^n - u^{n-1} (+ the
 * source term) can be solved for u^{n-1}: the same arithmetic with the two
 * time levels swapped. rtm_forward keeps, for every state u^1 .. u^{nt-2},
 * the model region's band of cells within r of one of its faces (their
 * stencils reach into the sponge); the backward call starts from the last
 * two states the forward call leaves in the workspace and steps the source
 * field back in time next to the receiver field, one reverse step (model
 * region only) per time step, taking the band cells from storage. No
 * recompute pass and no snapshot slab; imaging reads the recovered field in
 * place. Band storage per state:
 *   2r nx ny + 2r (nz - 2r) nx + 2r (nz - 2r)(ny - 2r) floats
 * (z-face planes, then y-face rows, then x-face cells). Needs nx, ny, nz >
 * 2r; imaging only (want_grad = 0). The recovered field carries FP32
 * rounding of the reverse steps (about 1e-6 relative over hundreds of
 * steps); the receiver field and the source trace are those of the other
 * storage modes bit for bit. rtm_backward_image must follow the rtm_forward
 * of the same shot with nothing in between that writes the workspace. */

/* ---- imaging-condition variants -------------------------------------------
 * The paper forms the image by zero-lag cross-correlation of the source and
 * receiver wavefields (Sec. I) and says nothing about post-processing; these
 * are the two standard companions of that condition.
 *
 * rtm_backward_image_illum: rtm_backward_image (or, with storage =
 * RTM_STORE_LEARNED and d_ae_params given, rtm_backward_image_learned) that
 * also accumulates the source illumination d_illum[z][y][x] += sum over the
 * imaging steps m of u^m(x)^2, from the same snapshots the image uses
 * (decoded ones in learned storage). d_illum: model grid [nz][ny][nx], float32,
 * caller-owned, added to.
 *
 * rtm_image_filter: on the model grid [nz][ny][nx], d_normalized (if not NULL)
 * = image / (illum + eps_rel * max(illum)), eps_rel > 0 (the maximum is
 * reduced on the device into the status block of d_ws, which must be an RTM
 * workspace of at least 256 bytes); d_laplacian (if not NULL) = -L image with
 * the 2r-order star of p->radius divided by dx^2 and zero outside the model
 * grid (suppresses the low-wavenumber backscatter of zero-lag imaging).
 * Only p->nx, ny, nz, radius and dx are read. Outputs must not alias the
 * inputs. */
rtm_status rtm_backward_image_illum(const rtm_params *p, const float *d_c, const int32_t *d_rec,
                                    const float *d_rdata, const float *d_ae_params, void *d_ws,
                                    size_t ws_bytes, float *d_image, float *d_illum,
                                    rtm_stream stream);
rtm_status rtm_image_filter(const rtm_params *p, const float *d_image, const float *d_illum,
                            float eps_rel, float *d_normalized, float *d_laplacian, void *d_ws,
                            size_t ws_bytes, rtm_stream stream);

/* ---- batched shots on uneven apertures (one persistent launch per wave) ----
 * Each shot runs a full RTM (forward modelling with checkpoints every
 * p->ckpt_every steps, segment recompute, receiver propagation with zero-lag
 * imaging every p->image_every steps) on its own aperture of a common model,
 * padded by p->nb sponge cells, receivers at every (x, y) of the aperture at
 * depth rec_z. All shots of a wave run inside ONE cooperative persistent
 * kernel launch: blocks take (phase step, shot, tile) work items from an
 * atomic queue and wait (bounded) for the previous phase step of the same
 * shot, so uneven apertures balance dynamically. Waves are consecutive shots
 * whose buffers fit budget_bytes (0: one wave); the call captures every
 * wave's model preparation, persistent launch and image stack into one CUDA
 * graph, launches it and synchronises the stream.
 *   p: nx, ny, nz = the full model; radius, nb, nt, dx, dt, f0, t0,
 *      ckpt_every, image_every as for one shot; storage = RTM_STORE_CKPT.
 *   d_vel   [nz][ny][nx] velocity of the full model (m/s).
 *   d_dobs  per-shot data [nt][ny_s][nx_s], concatenated in shot order.
 *   d_data  modelled data in the same layout, or NULL.
 *   d_image [nz][ny][nx] of the full model, ACCUMULATED: each shot adds its
 *           image at its aperture, in shot order (deterministic).
 *   zchunk  z planes per work item (0: per wave, the tallest slab that gives
 *           every phase step at least three items per resident block).
 * The work items march their tiles with TMA plane loads when the driver
 * provides tensor maps and rtm_set_tuning has not selected the vector-load
 * variant (1) for the radius; both kernels give the same image within the
 * wavefield tolerance. */
typedef struct {
    int32_t ox, oy, oz;          /* aperture origin in the full model */
    int32_t nx, ny, nz;          /* aperture size */
    int32_t src_x, src_y, src_z; /* source, aperture coordinates */
    int32_t rec_z;               /* receiver plane depth, aperture coordinates */
} rtm_aperture;
size_t rtm_batch_workspace_size(const rtm_params *p, int32_t nshots, const rtm_aperture *h_shots,
                                size_t budget_bytes);
/* Bound (seconds of SM clock at its base rate, default 20) of every
 * inter-block wait of the persistent batch kernel. A wait that runs out sets
 * an abort flag that every block sees, the launch ends without hanging, the
 * status word reads RTM_ERR_TIMEOUT (rtm_check) and rtm_batch returns it.
 * poison_shot >= 0 makes that shot's first work item wait for a count that
 * is never reached: a host-injected failure for testing the timeout path
 * (-1: off). */
rtm_status rtm_batch_set_wait(double seconds, int32_t poison_shot);
rtm_status rtm_batch(const rtm_params *p, int32_t nshots, const rtm_aperture *h_shots,
                     const float *d_vel, const float *d_dobs, float *d_data, float *d_image,
                     void *d_ws, size_t ws_bytes, size_t budget_bytes, int32_t zchunk,
                     rtm_stream stream);

/* Size of the static device scratch of rtm_forward_noalloc: 24 MiB. */
#define RTM_NOALLOC_SCRATCH_BYTES (24u << 20)

/* Forward modelling without any device allocation and without a workspace.
 * (The paper has no counterpart; this is a deployment convenience.)
 *
 * For callers that cannot call cudaMalloc or hand out a workspace: code that
 * runs inside a host application owning every device allocation, plugins that
 * may not touch the process's allocator, or callers that must keep the
 * device's memory footprint fixed. They pass only the inputs and outputs,
 * exactly as for rtm_forward (d_c, d_rec, d_data [nt][nrec] or NULL,
 * d_u_last [2][NZ][NY][NX] or NULL).
 *
 * The scratch (the two wavefields, the wavelet, the sponge profiles and a
 * status word) is a file-scope static device array of
 * RTM_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds until
 * the process exits. Problems whose two padded fields plus tables do not fit
 * (about 2.9 M padded points, e.g. 104^3 fits) are rejected with
 * RTM_ERR_WORKSPACE and a message naming the sizes; nothing is allocated,
 * freed or copied to host memory by this call.
 *
 * The first call on each device looks the scratch's device address up
 * (cudaGetSymbolAddress with that device current); make that first call
 * before capturing the stream into a CUDA graph. All calls share the one
 * array, which keeps the previous call's contents: each call clears what must
 * start at zero. Calls whose execution overlaps on the GPU (other streams or
 * threads) race on the array and must be serialised by the caller. It stores
 * no snapshots or checkpoints, so it cannot feed rtm_backward_image; receivers
 * outside the padded grid get zero traces and are not reported (there is no
 * workspace for rtm_check). It does not update rtm_stats. It always runs the
 * 16-byte vector-load stencil kernel (the plane-load variant of
 * rtm_set_tuning does not apply); the forward slab height set by
 * rtm_set_tuning or rtm_set_tuning_mode (mode 0) does.
 * A failed CUDA call returns RTM_ERR_CUDA with its message in
 * rtm_last_error(). */
rtm_status rtm_forward_noalloc(const rtm_params *p, const float *d_c, const int32_t *d_rec,
                               float *d_data, float *d_u_last, rtm_stream stream);

/* ---- off-grid source and receivers ---------------------------------------
 * The paper's time step includes "interpolation where necessary" (Sec. II).
 * Here a source or receiver may sit between grid points: it is spread over
 * the grid with Kaiser-windowed sinc weights (Hicks 2002): along each axis a
 * point at xi (cells) weighs grid point i by
 *   sinc(i - xi) I0(b sqrt(1 - ((i - xi) / 4)^2)) / I0(b),  |i - xi| <= 4,
 * b = 4.14, on its 8 nearest points (a single point of weight 1 where xi is
 * a grid point); a tap's weight is the product of its three axis weights.
 * The source adds c w^n / dx^3 times each tap weight to u^{n+1}; a receiver
 * records the weighted sum of u^{n+1} over its taps; the receiver pass
 * injects c g r / dx^3 times each tap weight (the exact transpose). */
typedef struct rtm_point_taps {
    int32_t i0, j0, k0;     /* padded index of the first tap along x, y, z */
    int32_t nx, ny, nz;     /* taps along x, y, z: 1 .. 8 (taps outside the padded
                               grid are left out) */
    float wx[8], wy[8], wz[8];  /* the axis weights of those taps */
    int32_t reserved[2];
} rtm_point_taps;               /* 128 bytes */

/* Tap tables of a source at h_src_xyz[3] and nrec receivers at
 * h_rec_xyz[nrec][3], model coordinates in cells (x, y, z; fractional; the
 * padded position is the model one plus nb), computed on the host in double
 * precision and stored in float. h_out[0] is the source, h_out[1 + j]
 * receiver j. Host only. Returns 1 + nrec (entries written only if
 * out_count >= 1 + nrec), or 0 if a position lies outside the padded grid
 * or p is invalid. */
size_t rtm_offgrid_taps(const rtm_params *p, const double *h_src_xyz, int32_t nrec,
                        const double *h_rec_xyz, rtm_point_taps *h_out, size_t out_count);

/* rtm_forward and rtm_shot with the source and the p->nrec receivers of a
 * device tap table d_taps[1 + nrec] (from rtm_offgrid_taps) instead of
 * p->src_* and integer receiver coordinates. Storage: every imaging storage
 * of rtm_shot (store-all, checkpoints, binomial, boundary, decimated); not
 * the gradient. The receiver injection of the backward pass adds with
 * atomics where taps of neighbouring receivers overlap, so its sums are not
 * ordered. A tap outside the padded grid (a corrupted table) is skipped and
 * sets RTM_ERR_INVALID in the status word. Costs up to 512 taps per point
 * and step in the small kernels. */
rtm_status rtm_forward_offgrid(const rtm_params *p, const float *d_c,
                               const rtm_point_taps *d_taps, float *d_data, void *d_ws,
                               size_t ws_bytes, float *d_u_last, rtm_stream stream);
rtm_status rtm_shot_offgrid(const rtm_params *p, const float *d_c, const rtm_point_taps *d_taps,
                            const float *d_dobs, float *d_data, void *d_ws, size_t ws_bytes,
                            float *d_image, rtm_stream stream);

/* ---- X-Y domain decomposition of one shot ----------------------------------
 * The paper's distributed time step (Sec. II): the padded grid is split in x
 * and y into px x py subdomains, each holding its owned block plus an r-wide
 * halo on its four x-y faces. Every step applies the stencil to the bands of
 * tiles along the faces that have a neighbour first, packs the r-wide strips
 * the neighbours need, exchanges them on a communication stream (the
 * dedicated communication thread of Sec. III) while the interior is
 * computed, and unpacks them into the neighbours' halos before the next
 * step. All subdomains of a call live on the calling GPU; a strip's exchange
 * is a device copy between pack and unpack buffers.
 *
 * Partition: x boundaries at multiples of 4 cells (as even as possible),
 * y boundaries as even as possible; every part at least r (and 4 in x) wide.
 * rtm_decomp_plan (host only, no device access) writes 8 int32 per subdomain
 * (index j * px + i) into h_out: owned padded x0, x1, y0, y1 and the
 * neighbour across the W (x-), E (x+), S (y-), N (y+) face, -1 at the grid's
 * outer faces; returns px * py (h_out untouched if more than max_sub), or -1
 * if p or the decomposition is invalid (rtm_last_error says why). */
int32_t rtm_decomp_plan(const rtm_params *p, int32_t px, int32_t py, int32_t *h_out,
                        int32_t max_sub);

/* Workspace bytes of rtm_forward_decomposed (0 if invalid): the subdomains'
 * local fields, coefficients and profiles, pack and unpack buffers, strip
 * descriptors and per-subdomain receiver lists and traces. */
size_t rtm_decomp_workspace_size(const rtm_params *p, int32_t px, int32_t py);

/* Forward modelling (source injection, propagation, receiver gather) on the
 * decomposition: d_c [NZ][NY][NX] as for rtm_forward (copied into the
 * subdomains' local arrays at the start), d_rec [nrec][3] device array (read
 * back to the host once to assign receivers to subdomains: the call
 * synchronises the stream before its first launch), d_data [nt][nrec] or
 * NULL, d_u_last [2][NZ][NY][NX] or NULL. storage must be RTM_STORE_ALL or
 * RTM_STORE_CKPT (nothing is stored; no snapshots or checkpoints for a
 * backward call) and want_grad 0. Needs the TMA stencil (tuning variant 2 or
 * 3 gives the tile; otherwise 8-row tiles). The results equal rtm_forward's
 * with the same tile bit for bit. A receiver outside the padded grid gets a
 * zero trace and sets RTM_ERR_INVALID in the status word (rtm_check on
 * d_ws); the post-run scan of u^nt applies. The call creates and destroys
 * streams and events of its own: up to eight compute streams (subdomain k
 * on stream k % 8, so that the subdomains' launches overlap) and the
 * communication stream; the caller's stream waits for all of them before
 * the call returns. */
rtm_status rtm_forward_decomposed(const rtm_params *p, int32_t px, int32_t py, const float *d_c,
                                  const int32_t *d_rec, float *d_data, void *d_ws,
                                  size_t ws_bytes, float *d_u_last, rtm_stream stream);

/* Stencil tuning: z extent of the slab one thread block marches through
 * (0 = automatic) and the plane-load path and tile (0 = automatic: TMA
 * where the driver provides tensor maps; 1 = 16-byte vector loads through
 * registers; 2 = TMA bulk tensor copies into shared-memory rings, 16-row
 * tiles of 256 threads; 3 = the same with 8-row tiles of 128 threads and
 * 4-point vectors at both radii, five blocks per SM at radius 4, four at
 * radius 8). Applies to later
 * calls on every thread, to every kernel mode on the padded grid (the
 * allocation-free forward call takes the slab height only); the
 * reverse step of boundary storage, which covers the model region, sizes
 * its slabs for that region. The batched multi-shot kernel (rtm_batch)
 * takes its plane-load path and tile from the same variant and its slab
 * height from its own argument. */
rtm_status rtm_set_tuning(int32_t radius, int32_t zchunk, int32_t variant);

/* Slab height of one stencil mode at a radius (0 = the radius's general
 * slab height), set after rtm_set_tuning (which clears these): mode 0
 * forward step (and the learned forward step that sums squares), 1 forward +
 * snapshot, 2 backward + imaging, 3 forward + L u, 4 backward + gradient,
 * 6 reverse step of boundary storage. The modes move different bytes per
 * point, so their best slab heights differ; the autotuner sets them from
 * the per-mode timings of its trials. Applies to the single-shot calls. */
rtm_status rtm_set_tuning_mode(int32_t radius, int32_t mode, int32_t zchunk);

/* Host-injected wait failure for testing the timeout path of the kernels
 * with mbarrier rings: kernel RTM_STALL_STENCIL (the TMA stencil's plain
 * forward step with 8-row tiles, tuning variant 3, as a separate kernel
 * instance: the others carry no code for it) or RTM_STALL_ENCODER (the
 * z-marching codec encoder); plane >= 0 arms a
 * one-shot stall of that kernel's next launch: block 0's copy of the plane
 * `plane` planes before the last one it copies (0: the last; the encoder
 * takes 0-2) expects 16 bytes more than it delivers, so the bounded wait
 * for it runs out after about 2 s; the block raises its abort flag, waits
 * (bounded) for every copy it issued and leaves, and the call's status word
 * reads RTM_ERR_TIMEOUT (rtm_check). Every copy lands, and no later copy
 * reuses the stalled ring slot (a wait for a later phase of a barrier whose
 * phase never completes would pass at once); nothing faults. -1 disarms.
 * Returns RTM_ERR_INVALID for an unknown kernel. */
#define RTM_STALL_STENCIL 0
#define RTM_STALL_ENCODER 1
rtm_status rtm_set_test_stall(int32_t kernel, int32_t plane);

/* Enable (1) or disable (0) per-launch CUDA-event timing of the stencil
 * kernels. While enabled, each API call synchronises its stream on return. */
rtm_status rtm_set_timing(int32_t enable);
rtm_status rtm_stats_get(rtm_stats *out);
rtm_status rtm_stats_reset(void);

#ifdef __cplusplus
}
#endif

#endif /* RTM_H */
