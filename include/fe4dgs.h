/*
 * fe4dgs.h -- C ABI of the GB300 (sm_103a) FE-4DGS rasterization library.
 *
 * One differentiable tile-rasterization pass of FeatureEndo-4DGS
 * (arXiv 2503.06161): per-Gaussian deformation query (Sec. 3.2, Eq. 4-6),
 * EWA projection (Sec. 3.3, Sigma' = J W Sigma W^T J^T), SH colour
 * (Sec. 3.1), (tile, depth) binning and sort (the tile-based rasterization
 * of 3DGS the paper builds on, Sec. 2.1), and front-to-back blending of
 * colour, a D-channel semantic feature and depth in one pass (Sec. 3.3,
 * Eq. 7-8), plus the reverse pass of all of it.
 *
 * Conventions shared by every entry point:
 *  - Every array pointer is a DEVICE pointer owned by the caller, except
 *    where "host" is written.  The library never frees caller memory and
 *    allocates no device memory: scratch space is the caller's workspace.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *    default stream).  A return of FE_OK means the work was enqueued;
 *    device-side conditions (duplicate-list overflow, a bounded wait that
 *    gave up, non-finite input) are recorded in the workspace and read
 *    back with fe_read_stats().
 *  - Arrays are row-major and densely packed, float32 unless stated;
 *    bfloat16 arrays hold raw 16-bit patterns.
 *  - Pixel (x, y) covers [x, x+1) x [y, y+1); its centre is (x+0.5, y+0.5).
 *  - No entry point throws; each returns an fe_status.
 */
#ifndef FE4DGS_H
#define FE4DGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FE_OK = 0,
  FE_ERR_INVALID_ARG = 1,   /* NULL pointer, negative size, bad tile shape, ... */
  FE_ERR_CUDA = 2,          /* a CUDA runtime call failed (launch, memset, ...) */
  FE_ERR_WORKSPACE = 3,     /* workspace too small, or (stats) duplicate capacity exceeded */
  FE_ERR_UNSUPPORTED = 4,   /* D, plane channels, SH degree or tile shape not compiled in */
  FE_ERR_NONFINITE = 5,     /* (stats) a non-finite Gaussian parameter was seen */
  FE_ERR_TIMEOUT = 6,       /* (stats) a bounded device-side wait gave up */
  FE_ERR_STATE = 7          /* backward called on a workspace without a matching forward */
} fe_status;

/* Pinhole camera (Sec. 3.3).  u = fx * x/z + cx, v = fy * y/z + cy for the
 * camera-space point (x, y, z) = world_to_cam * (X, Y, Z, 1).  Gaussians
 * with z <= znear are culled. */
typedef struct {
  int width, height;        /* image size in pixels, both >= 1 */
  float fx, fy, cx, cy;
  float world_to_cam[16];   /* host array, row-major 4x4 rigid transform */
  float campos[3];          /* host array, camera centre in world space (SH view direction) */
  float znear;
} fe_camera;

/* Canonical Gaussians (Sec. 3.1, Eq. 1-2) with a D-channel semantic
 * feature z (Sec. 3.2-3.3).  Opacity o = sigmoid(logit); scale s = exp(log_scale);
 * rotation from the quaternion (w, x, y, z) after normalisation. */
typedef struct {
  int P;                    /* number of Gaussians, >= 0 */
  int D;                    /* feature channels: 16, 32, 64, 128 or 256 (256 runs the compositing
                               kernels as two passes over 128-channel halves) */
  int sh_degree;            /* 0..3; sh always holds 16 coefficients per channel */
  int sh_bf16;              /* 1: sh holds bfloat16, else float32 */
  int feat_bf16;            /* 1: feat holds bfloat16, else float32 */
  const float *means;       /* [P,3] */
  const float *log_scales;  /* [P,3] */
  const float *quats;       /* [P,4] (w, x, y, z), any non-zero length */
  const float *opacity_logits; /* [P] */
  const void *sh;           /* [P,16,3] coefficient-major: sh[g][k][channel] */
  const void *feat;         /* [P,D] */
} fe_gaussians;

/* FST deformation field (Sec. 3.2, Eq. 4 and 6; Appendix A), single
 * resolution: six planes xy, xz, yz, xt, yt, zt sampled bilinearly at the
 * Gaussian's normalised (x, y, z, t) (grid corners at -1 and +1, positions
 * clamped to the border), multiplied elementwise into f[C], then
 * h1 = relu(W1 f + b1), h2 = relu(W2 h1 + b2), delta = Wh h2 + bh with
 * delta = (d_mu[3], d_q[4], d_s[3], d_o[1]) applied as
 * mu + d_mu (+ noise_scale * t * noise), normalise(q + d_q), log_s + d_s,
 * logit + d_o.  The MLP and its reverse run on the tensor cores with FP32
 * accuracy: each operand as three BF16 terms, six term products per layer
 * accumulated in FP32. */
typedef struct {
  int C;                    /* plane channels: 32 or 64 */
  int R;                    /* plane resolution (R x R), >= 2 */
  const float *planes;      /* [6,R,R,C] channels-last; plane k index [i][j] with i along
                               the first coordinate of the pair, j along the second */
  const float *w1, *b1;     /* [64,C], [64] */
  const float *w2, *b2;     /* [64,64], [64] */
  const float *wh, *bh;     /* [11,64], [11] */
  float bbox_min[3], bbox_max[3]; /* host arrays: scene box mapped to [-1,1]^3 */
  const float *noise;       /* [P,3] or NULL */
  float noise_scale;
} fe_deform;

typedef struct {
  int tile_w, tile_h;       /* tile shape; tile_w * tile_h == 256, each in {8,16,32} */
  float bg[3];              /* background colour added as bg * T_final */
  int64_t max_dups;         /* capacity of the (Gaussian, tile) list; 0 = 16 * P + 4096 */
  int forward_only;         /* 1: workspace without backward storage */
  int accumulate_grads;     /* backward: 1 = add the gradients to the fe_grads buffers (e.g. a
                               sum over views rendered one after another); 0 = overwrite */
  void *const *events;      /* profiling: NULL, or host array of 8 cudaEvent_t (NULL entries
                               skipped) recorded on the stream at stage boundaries:
                               forward [0] start [1] after deform+projection [2] after
                               binning [3] after compositing; backward [4] start [5] after
                               the compositing reverse [6] after the feature-gradient sum
                               [7] after the per-Gaussian reverse */
  int fwd_batch;            /* Gaussians per shared-memory batch of the compositing forward:
                               0 = the default for D (128 up to D = 32, 64 at D = 64, 32 at
                               D = 128), else 32, 64 or 128 (128 only up to D = 64); the
                               images do not depend on it */
  int wait_polls;           /* bound of each staging wait of the compositing kernels, in
                               polls: 0 = the default (2^20); a negative value makes every
                               such wait give up at once -- a test hook for the timeout path:
                               the launch still waits (with its own bound) for the copies it
                               issued, records FE_ERR_TIMEOUT and returns */
} fe_opts;

/* Render outputs (Eq. 7-8 plus depth): rgb [3,H,W] planar = sum w c + bg T;
 * depth [H,W] = sum w z_cam (not normalised); alpha [H,W] = 1 - T_final;
 * feat [H*W, D] channels-last = sum w z.  feat_bf16 (optional, NULL = not
 * written; 16-byte aligned): the same map rounded to bf16 (nearest even),
 * the operand layout of the decoder. */
typedef struct {
  float *rgb, *depth, *alpha, *feat;
  void *feat_bf16;
} fe_outputs;

/* Upstream gradients, same shapes as fe_outputs; any may be NULL (= zero). */
typedef struct {
  const float *rgb, *depth, *alpha, *feat;
} fe_output_grads;

/* Parameter gradients (overwritten, or added to when fe_opts.accumulate_grads
 * is set; float32 even for bfloat16 storage):
 * means [P,3], log_scales [P,3], quats [P,4], opacity_logits [P],
 * sh [P,16,3], feat [P,D].  Deformation-network weight gradients are not
 * produced (the canonical mean receives the gradient through the grid). */
typedef struct {
  float *means, *log_scales, *quats, *opacity_logits, *sh, *feat;
} fe_grads;

/* Host-side view of the workspace header, filled by fe_read_stats(). */
typedef struct {
  int64_t num_dups;         /* K: (Gaussian, tile) pairs of the last forward */
  int64_t capacity;         /* duplicate capacity of this workspace */
  int64_t num_visible;      /* Gaussians in front of znear with a non-empty rect */
  uint32_t device_errors;   /* bit 0 overflow, bit 1 timeout, bit 2 non-finite */
  int32_t has_forward;      /* 1 after a forward on this workspace */
} fe_stats;

/* Bytes of workspace for P Gaussians, D channels, a width x height image
 * and opts (NULL = defaults).  It includes, for any deformation field the
 * forward may be given (HexPlane channels C <= 64), the deformation state
 * (64 B per Gaussian) and the HexPlane features split into three BF16
 * terms for the tensor-core MLP (384 B per Gaussian).  Returns
 * FE_ERR_UNSUPPORTED for a tile shape or D that is not compiled in, or for
 * more than 8192 tiles. */
fe_status fe_workspace_size(int P, int D, int width, int height, const fe_opts *opts, size_t *bytes);

/* Forward pass (Sec. 3.2-3.3): deform (deform may be NULL: static scene)
 * at time t, project, colour, bin, sort and composite.  The workspace (at
 * least fe_workspace_size bytes, 256-byte aligned, device memory) receives
 * the state the backward pass needs; it must not be modified in between.
 * All output pointers are required. */
fe_status fe_render_forward(const fe_gaussians *g, const fe_deform *deform, const fe_camera *cam, float t,
                            const fe_opts *opts, void *workspace, size_t workspace_bytes,
                            const fe_outputs *out, void *stream);

/* Reverse pass of fe_render_forward: same g, deform, cam, t, opts and
 * workspace as the forward that preceded it on this stream.  Replays
 * transmittance from T_final (no per-pixel lists), reduces per tile in a
 * fixed order and sums per-(tile, Gaussian) partials in a fixed order:
 * deterministic, no floating-point atomics. */
fe_status fe_render_backward(const fe_gaussians *g, const fe_deform *deform, const fe_camera *cam, float t,
                             const fe_opts *opts, void *workspace, size_t workspace_bytes,
                             const fe_output_grads *grad_out, const fe_grads *grads, void *stream);

/* Integer stage alone (tile-based binning of 3DGS, Sec. 2.1): given
 * projected centres uv [P,2], integer radii [P] (<= 0: culled) and depths
 * [P] (float32), build the tile lists sorted by (tile, depth), ties by
 * index, in the workspace.  A Gaussian covers the pixels whose centre lies
 * in the square of half-side r around (u, v); its pixel rect is
 * [ceil(u-(r+0.5)), floor(u+(r-0.5))] x [ceil(v-(r+0.5)), floor(v+(r-0.5))]
 * in binary32, clamped to the image.  Read the result with fe_debug_dump. */
fe_status fe_tile_bin(int P, const float *uv, const int *radius, const float *depth, int width, int height,
                      const fe_opts *opts, void *workspace, size_t workspace_bytes, void *stream);

/* Synchronous: wait for `stream`, then copy the workspace header to host. */
fe_status fe_read_stats(const void *workspace, size_t workspace_bytes, int P, int D, int width, int height,
                        const fe_opts *opts, fe_stats *stats, void *stream);

/* Pair counts of the last forward's compositing, for the roofline: visits
 * (pixel, list entry) pairs a pixel evaluated before stopping, contrib the
 * pairs that were blended.  counts: device array of 2 uint64 (overwritten).
 * Re-runs the compositing on the same workspace (outputs are not written). */
fe_status fe_count_pairs(const fe_gaussians *g, const fe_camera *cam, const fe_opts *opts, void *workspace,
                         size_t workspace_bytes, uint64_t *counts, void *stream);

/* Copy forward state out for parity tests; any pointer may be NULL.
 * keys [cap] u64 = (tile << 32) | bits(depth), gauss [cap] u32 (sorted
 * Gaussian index per list entry), ranges [tiles,2] u32 (start, end),
 * n_contrib [H*W] u32, t_final [H*W] f32, uv [P,2], conic [P,3]
 * (inverse of the dilated 2D covariance), opacity [P], depth [P],
 * rgb [P,3] (clamped), radius [P] i32, touched [P] u32.  Entries past the
 * last forward's K are left untouched. */
fe_status fe_debug_dump(const void *workspace, size_t workspace_bytes, int P, int D, int width, int height,
                        const fe_opts *opts, uint64_t *keys, uint32_t *gauss, uint32_t *ranges,
                        uint32_t *n_contrib, float *t_final, float *uv, float *conic, float *opacity,
                        float *depth, float *rgb, int32_t *radius, uint32_t *touched, void *stream);

/* Per-pixel L1 loss (Sec. 3.3, Eq. 10 form: mean over `rows` pixels of the
 * L1 norm over the channels) of pred against target, both [n] float32 with
 * n = rows * channels in any layout.  Writes grad [n] = sign(pred - target)
 * / rows (sign(0) = 0) and *loss (one device float) = sum |pred - target|
 * / rows.  scratch: device array of at least 1024 floats for the per-block
 * partial sums; summation order is fixed, so the result is deterministic. */
fe_status fe_l1_loss_grad(const float *pred, const float *target, int64_t n, int64_t rows, float *grad,
                          float *loss, float *scratch, void *stream);

/* Allocation-free form of fe_l1_loss_grad, for callers that cannot
 * allocate device memory even for 4 KiB of scratch -- for example a plug-in
 * whose host application owns every device allocation, or a latency-bound
 * loop in which a cudaMalloc (which synchronises the device) is not
 * acceptable.  The paper has no counterpart: this is a deployment variant.
 * Same inputs, outputs and layout as fe_l1_loss_grad except that the
 * per-block partial sums live in a 64 KiB array inside the library (one
 * per GPU that loads it, kept until the process exits); n may be at most
 * 33,554,432 elements (16384 blocks of 2048), else FE_ERR_WORKSPACE is
 * returned and nothing is launched.  Every call looks up that array's
 * device address on the current device (a host-side lookup); the first
 * lookup on a device may load the library's device code, so make the first
 * call on each device before any stream capture.  Every call shares the array: calls whose
 * work overlaps on the GPU (different streams, or other threads) race and
 * must be ordered by the caller.  No device memory is allocated or freed. */
fe_status fe_l1_loss_grad_noalloc(const float *pred, const float *target, int64_t n, int64_t rows, float *grad,
                                  float *loss, void *stream);

/* ------------------------------------------------------------------------
 * Semantic decoder (Sec. 3.3): a pointwise (1x1) convolution of the
 * rendered feature map from D to 256 channels,
 *     out[p][c] = sum_d feat[p][d] * weight[c][d] + bias[c],
 * with BF16 operands and FP32 accumulation on the tensor cores.  The map is
 * channels-last, as fe_render_forward writes it; the decoder applies no
 * spatial upsampling.
 * ------------------------------------------------------------------------ */
typedef struct {
  int64_t HW;               /* pixels (rows of feat), 0 <= HW < 2^31 - 128 */
  int D;                    /* feature channels: 16, 32, 64 or 128 (else FE_ERR_UNSUPPORTED); 16 runs
                               the 32-channel kernel on tiles the tensor maps zero-fill past channel
                               16; 128 runs as two launches over the output channels 0-127 and
                               128-255 (the second adds its share of d_feat to the first's) */
  const void *feat;         /* [HW, D] bf16, row-major, 16-byte aligned */
  const void *weight;       /* [256, D] bf16, row-major, 16-byte aligned */
  const float *bias;        /* [256] float32 */
} fe_decoder_args;

/* Bytes of device workspace for the decoder calls: a 256-byte header whose
 * first word collects device error bits, then per-CTA partial sums of the
 * loss and of the weight and bias gradients.  0 for an unsupported D. */
size_t fe_decoder_workspace_size(int64_t HW, int D);

/* out [HW, 256] float32 (16-byte aligned) = the decoder applied to feat.
 * Asynchronous on `stream`; the caller owns every buffer. */
fe_status fe_decode_forward(const fe_decoder_args *args, float *out, void *workspace, size_t workspace_bytes,
                            void *stream);

/* Decoder, L1 feature loss (Eq. 10) and its reverse pass in one launch; the
 * 256-channel output is never written to memory.  With S[p][c] =
 * sign(out[p][c] - target[p][c]) (sign(0) = 0):
 *     *loss        = scale * sum_{p,c} |out - target|
 *     d_feat[p][d] = scale * sum_c S[p][c] weight[c][d]     [HW, D] float32
 *     d_weight[c][d] = scale * sum_p S[p][c] feat[p][d]    [256, D] float32
 *     d_bias[c]    = scale * sum_p S[p][c]                 [256] float32
 * scale = 1/HW gives Eq. 10 (mean over pixels of the L1 norm over
 * channels).  target: [HW, 256] row-major, bf16 if target_bf16 else
 * float32, 16-byte aligned.  loss, d_weight, d_bias are device pointers;
 * every output is overwritten.  Sums over pixels run in a fixed order, so
 * results are bitwise reproducible.  Asynchronous on `stream`. */
fe_status fe_decode_l1(const fe_decoder_args *args, const void *target, int target_bf16, float scale, float *loss,
                       float *d_feat, float *d_weight, float *d_bias, void *workspace, size_t workspace_bytes,
                       void *stream);

/* Reads the device error bits of the last decoder call on this workspace
 * (2 = a pipeline wait timed out).  Synchronises `stream`. */
fe_status fe_decoder_read_errors(const void *workspace, uint32_t *err, void *stream);

/* ------------------------------------------------------------------------
 * Adam (the optimiser the paper trains with, Sec. 4.1), with bias
 * correction, on FP32 master parameters:
 *     m <- b1 m + (1 - b1) g;   v <- b2 v + (1 - b2) g^2
 *     p <- p - lr * (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps)
 * ------------------------------------------------------------------------ */
typedef struct {
  float *param;             /* [n] FP32 master, updated in place */
  const float *grad;        /* [n] */
  float *m, *v;             /* [n] first and second moments, updated in place (start at 0) */
  void *param_bf16;         /* optional [n] bf16 copy written from the updated param (nearest
                               even), e.g. the SH / feature storage the renderer reads; NULL = none */
  int64_t n;                /* elements, >= 0 */
  float lr;                 /* learning rate of this group */
} fe_adam_group;

/* One Adam step over 1..8 parameter groups in a single launch.  step >= 1
 * is the 1-based step count of the bias correction; 0 <= b1, b2 < 1,
 * eps >= 0.  param, grad, m, v: device pointers, 16-byte aligned;
 * param_bf16 8-byte aligned.  Asynchronous on `stream`. */
fe_status fe_adam_step(const fe_adam_group *groups, int ngroups, int step, float beta1, float beta2, float eps,
                       void *stream);

/* dst[i] = ((srcs[0][i] + srcs[1][i]) + srcs[2][i]) + ... in this fixed
 * order (e.g. gradients of views rendered on separate streams, combined
 * reproducibly).  srcs: host array of 1..8 device pointers; dst and every
 * source float32 [n], 16-byte aligned; dst may alias srcs[0].  Asynchronous
 * on `stream`.  The paper has no counterpart: a batching utility. */
fe_status fe_sum_f32(float *dst, const float *const *srcs, int nsrc, int64_t n, void *stream);

/* ------------------------------------------------------------------------
 * Full FST deformation module (Sec. 3.2, Eq. 4-6; Appendix A).
 *
 * Each Gaussian's canonical centre mu and the time t are encoded by a
 * multi-resolution HexPlane: coordinates are normalised to [-1, 1] by the
 * scene box (t in [0, 1] -> [-1, 1]); level l (0 <= l < levels) holds six
 * planes xy, xz, yz, xt, yt, zt with FE_FST_CHANNELS channels, spatial axes
 * of rs << l nodes and a time axis of rt nodes (grid corners at +-1,
 * positions clamped to the border, bilinear sampling); a level's feature is
 * the channel-wise product of its six samples and f is the concatenation
 * of the levels' features (levels * 32 values).  The decoder MLP F_out
 * (width 64, depth 8: Linear(f) then seven ReLU -> Linear(64, 64)) gives h;
 * each branch g in (mu, R, S, o) applies ReLU -> Linear(64, 32),
 * ReLU -> Linear(32, 32) giving h_g and ReLU -> Linear(32, d_g) giving the
 * offset (d_g = 3, 4, 3, 1: Eq. 4); the semantic updater F_feat applies
 * ReLU -> Linear(128, 64), ReLU -> Linear(64, D) to [h_mu, h_R, h_S, h_o],
 * giving dz (Eq. 5).  The deformed Gaussian (Eq. 6) in the renderer's
 * parameterisation: mu + d_mu, q + d_R (normalised by the renderer),
 * log s + d_S, opacity logit + d_o, z + dz.
 *
 * Parameter layout.  planes: level-major, then plane-major in the order
 * above, each [R_a][R_b][32] float32 (channels innermost; R_a, R_b the node
 * counts of the plane's two axes).  mlp: one float32 array holding, for
 * each linear layer in the order F_out 0..7, branch mu (E1, E2, head),
 * branch R, branch S, branch o, F_feat (Z1, Z2), its weight [out][in]
 * row-major followed by its bias [out].
 * ------------------------------------------------------------------------ */
#define FE_FST_WIDTH 64
#define FE_FST_DEPTH 8
#define FE_FST_CHANNELS 32
#define FE_FST_MAX_LEVELS 4

typedef struct {
  int levels;            /* 1..4 */
  int rs, rt;            /* base spatial node count (level l: rs << l) and time node count, >= 2 */
  int D;                 /* semantic channels of dz: 16, 32, 64 or 128 */
  const float *planes;   /* device, fe_fst_plane_floats(levels, rs, rt) floats, 16-byte aligned */
  const float *mlp;      /* device, fe_fst_mlp_floats(levels, D) floats, 16-byte aligned */
  float bbox_min[3], bbox_max[3];   /* scene box of the coordinate normalisation */
  int exact_planes;      /* reverse: 0 = plane gradients summed with float atomics (fast; the
                            last bits depend on the order of the additions); 1 = summed exactly
                            in fixed point, bitwise reproducible (workspace with_backward = 2;
                            about twice the reverse's time) */
} fe_fst;

/* Float counts of the plane and MLP arrays (0 for invalid arguments). */
int64_t fe_fst_plane_floats(int levels, int rs, int rt);
int64_t fe_fst_mlp_floats(int levels, int D);

/* Device workspace of fe_fst_forward / fe_fst_backward for P Gaussians and
 * planes of levels x (rs, rt) nodes.  with_backward = 0: forward only
 * (inference; the HexPlane features, 0.5 KB per Gaussian at 4 levels); 1:
 * the forward also keeps the per-Gaussian activations the reverse pass
 * reads, and the reverse's own per-Gaussian buffers (about 5.1 KB per
 * Gaussian at 4 levels in all) and per-block partial sums of the weight
 * gradients; 2: as 1, plus the exact plane-gradient accumulators that
 * fe_fst.exact_planes = 1 needs (16 bytes per plane float).  The first 4
 * bytes of the workspace hold the reverse's error bits (1: an exact
 * plane-gradient term of magnitude >= 2^23 was clamped). */
fe_status fe_fst_workspace_size(int P, int levels, int rs, int rt, int D, int with_backward, size_t *bytes);

/* Deformation of P Gaussians at time t.  Inputs (device, canonical, the
 * fe_gaussians layouts): means [P,3], quats [P,4], log_scales [P,3],
 * opacity_logits [P], feat [P,D] (bf16 if feat_bf16, else float32).
 * Outputs (device, caller-owned, overwritten): the deformed arrays in the
 * same layouts, feat_t in the same type as feat (bf16 outputs rounded to
 * nearest even).  Outputs must not alias inputs.  With with_backward the
 * workspace (fe_fst_workspace_size with with_backward = 1) keeps the state
 * fe_fst_backward needs; it must not be touched in between.  Asynchronous
 * on `stream`. */
fe_status fe_fst_forward(const fe_fst *fst, int P, const float *means, const float *quats, const float *log_scales,
                         const float *opacity_logits, const void *feat, int feat_bf16, float t, float *means_t,
                         float *quats_t, float *log_scales_t, float *opacity_logits_t, void *feat_t,
                         void *workspace, size_t workspace_bytes, int with_backward, void *stream);

/* Reverse pass of the last fe_fst_forward (with_backward = 1, same fst, P,
 * means and t).  Inputs: the gradients of the loss with respect to the
 * deformed arrays (device float32, layouts as above; d_feat_t [P,D]) --
 * e.g. the fe_grads of a render of the deformed Gaussians; d_feat_t 16-byte
 * aligned.  Because the
 * offsets are added, these are also the gradients of the offsets and of
 * the canonical quats, log_scales, opacity logits and features.  Outputs
 * (device float32, overwritten):
 *   d_means   [P,3]  d_means_t plus the path through the HexPlane
 *                    coordinates (may alias d_means_t);
 *   d_planes         like planes: with fst->exact_planes, every Gaussian's
 *                    terms summed exactly (96-bit fixed point, resolution
 *                    2^-72, |sum| < 2^23, integer atomics whose order does
 *                    not matter), then rounded once to float32 -- bitwise
 *                    reproducible; otherwise summed with float atomics (the
 *                    last bits depend on the order of the additions);
 *   d_mlp            like mlp: per-block partial sums reduced in a fixed
 *                    order (reproducible bit for bit).
 * Asynchronous on `stream`. */
fe_status fe_fst_backward(const fe_fst *fst, int P, const float *means, float t, const float *d_means_t,
                          const float *d_quats_t, const float *d_log_scales_t, const float *d_opacity_logits_t,
                          const float *d_feat_t, float *d_means, float *d_planes, float *d_mlp, void *workspace,
                          size_t workspace_bytes, void *stream);

/* Total-variation smoothness of the planes (the L_TV term of Eq. 11): for
 * every plane of the first `levels` levels, the mean over its nodes and
 * channels of the squared difference of neighbouring nodes along each of
 * its two axes, summed over planes and axes, times `weight`.  Writes the
 * weighted loss to *loss (one device float) and ADDS weight * dL_TV/dplanes
 * to d_planes (so it composes with fe_fst_backward's plane gradients);
 * d_planes must not overlap the planes (FE_ERR_INVALID_ARG).
 * scratch: device array of at least 1024 floats.  Deterministic.
 * Asynchronous on `stream`. */
fe_status fe_fst_tv(const fe_fst *fst, float weight, float *loss, float *d_planes, float *scratch, void *stream);

/* ------------------------------------------------------------------------
 * Adaptive density control.  The paper trains with densification, pruning
 * and opacity resets (its appendix hyperparameter table gives the
 * percent-dense fraction and the reset / prune intervals) without stating
 * the procedure; these entry points implement the adaptive density control
 * of the 3D Gaussian splatting lineage it builds on:
 *   statistics  per Gaussian, the sum over the views in which it touched a
 *               tile of |(dL/du W/2, dL/dv H/2)| -- the gradient of the loss
 *               with respect to its projected centre in normalised device
 *               coordinates -- and the number of such views;
 *   densify     a Gaussian whose mean statistic is >= grad_thresh is cloned
 *               (an identical copy appended) when its largest scale
 *               exp(log_scale) is <= dense_scale, and otherwise split: it is
 *               replaced by two Gaussians with centres mu + R(q) (s * n_i),
 *               n_i the caller's N(0, I3) draws, and scales s / 1.6, the
 *               other parameters copied;
 *   prune       Gaussians with sigmoid(opacity logit) < min_opacity, and
 *               their copies, are dropped;
 *   order       surviving originals in index order, then clones in index
 *               order, then split children (two per parent, parent order);
 *   reset       opacity logits capped at logit(max_opacity).
 * ------------------------------------------------------------------------ */

/* After fe_render_backward on `workspace` (same P, D, width, height, opts):
 * accum[g] += |(dL/du W/2, dL/dv H/2)| and count[g] += 1 for every Gaussian
 * that touched a tile in that view.  accum float32 [P], count int32 [P],
 * device, caller-owned (zero them to start).  Asynchronous on `stream`. */
fe_status fe_screen_grad_stats(const void *workspace, size_t workspace_bytes, int P, int D, int width, int height,
                               const fe_opts *opts, float *accum, int32_t *count, void *stream);

#define FE_ATTR_COPY 0        /* copied to survivors, clones and split children */
#define FE_ATTR_MEANS 1       /* [P][3] float32: children get mu + R(q)(s * n_i) */
#define FE_ATTR_LOG_SCALES 2  /* [P][3] float32: children get log_scale + log(1 / 1.6) */
#define FE_ATTR_STATE 3       /* optimiser state: survivors keep it, new Gaussians get 0 */

typedef struct {
  const void *src;   /* device, [P][width] elements */
  void *dst;         /* device, [capacity][width] elements, must not alias src */
  int width;         /* elements per Gaussian, >= 1 */
  int elem_bytes;    /* 4 (float32) or 2 (bf16; FE_ATTR_COPY and FE_ATTR_STATE only) */
  int role;          /* FE_ATTR_* */
} fe_attr;

typedef struct {
  int P;
  const float *means, *log_scales, *quats, *opacity_logits;  /* device: the decision inputs */
  const float *accum;                /* device [P]: statistics from fe_screen_grad_stats */
  const int32_t *count;              /* device [P] */
  const float *normals;              /* device [P][2][3]: N(0,1) draws for split children */
  float grad_thresh, dense_scale, min_opacity;
  const fe_attr *attrs;              /* host array of nattrs descriptors (1..32) */
  int nattrs;
  int64_t capacity;                  /* rows of every dst; must be >= 2 P */
} fe_densify_args;

/* Device workspace of fe_densify for P Gaussians (pass it 16-byte aligned). */
size_t fe_densify_workspace_size(int P);

/* Writes every attribute's densified rows to its dst and the new Gaussian
 * count to *new_P (one device int64).  The result is deterministic (fixed
 * scan order).  FE_ERR_INVALID_ARG for NULL pointers, unaligned float
 * arrays, a workspace that is not 16-byte aligned or capacity < 2 P;
 * FE_ERR_WORKSPACE for a small workspace.
 * Asynchronous on `stream`. */
fe_status fe_densify(const fe_densify_args *args, int64_t *new_P, void *workspace, size_t workspace_bytes,
                     void *stream);

/* logits[g] = min(logits[g], log(max_opacity / (1 - max_opacity))), g < P,
 * 0 < max_opacity < 1.  Asynchronous on `stream`. */
fe_status fe_reset_opacity(float *logits, int64_t P, float max_opacity, void *stream);

/* ------------------------------------------------------------------------
 * Batched form: V views of one deforming scene, each with its own time t,
 * camera and resolution (e.g. the timestamps and viewpoints of one training
 * batch), rendered in one call (Sec. 3.3: the same single rasterization
 * pass per view), and their reverse pass with the parameter gradients
 * summed over the views.  The per-Gaussian stages of each view
 * (deformation, projection, colour, binning; in the reverse, the sums of
 * the partial rows and the per-Gaussian chain rule) run on up to four
 * helper streams forked from `stream` and joined back to it (views dealt
 * round-robin: view v on helper v mod S, S = min(4, V)); the compositing of
 * ALL views runs on `stream` as one persistent launch -- as many blocks as
 * fit on the GPU, each taking (view, tile) work items from a device counter
 * until none are left -- and so does the compositing reverse.  Images are
 * bitwise those of fe_render_forward on each view with the same options;
 * the gradients are those of fe_render_backward on each view, summed in a
 * fixed order: helper i adds views i, i + S, i + 2S, ... in that order, then
 * the S sums are added in helper order (for V <= 4: plain view order).
 * The helper streams and their events are created by the first batched
 * call on a device (make it before any stream capture); calls on one device
 * serialise their enqueueing on a lock, and the whole call can be captured
 * into a CUDA graph.
 * ------------------------------------------------------------------------ */
#define FE_MAX_VIEWS 32

typedef struct {
  int V;                    /* number of views, 1..FE_MAX_VIEWS */
  const fe_camera *cams;    /* host array [V] */
  const float *t;           /* host array [V]: time of each view */
  const fe_opts *opts;      /* host array [V]: tile shape, background and list capacity of each
                               view.  forward_only, accumulate_grads (first view: add to the
                               gradient buffers instead of overwriting them), fwd_batch and
                               wait_polls are taken from opts[0] for the whole batch, and so
                               are the profiling events, here: forward [0] start [1] after
                               every view's deformation, projection and binning [2] after
                               the batched compositing; backward [4] start [5] after the
                               batched compositing reverse [7] after every view's
                               per-Gaussian reverse. */
} fe_batch;

/* Bytes of workspace for a batch: a 256-byte batch header, then one
 * fe_workspace_size region per view (256-byte aligned), then (with the
 * backward and more than one view) one float32 gradient set per helper
 * stream (P x (3 + 3 + 4 + 1 + 48 + D) floats, each array 256-byte aligned). */
fe_status fe_batch_workspace_size(int P, int D, const fe_batch *b, size_t *bytes);

/* Forward pass of every view of the batch.  out: host array [V] of the
 * views' outputs (as fe_render_forward's).  The workspace (at least
 * fe_batch_workspace_size bytes, 256-byte aligned) keeps each view's state
 * for fe_render_batch_backward.  Asynchronous on `stream`. */
fe_status fe_render_batch(const fe_gaussians *g, const fe_deform *deform, const fe_batch *b, void *workspace,
                          size_t workspace_bytes, const fe_outputs *out, void *stream);

/* Reverse pass of the last fe_render_batch on this workspace (same g,
 * deform, b).  grad_out: host array [V] of the views' upstream gradients.
 * grads receives the sum over views of each view's parameter gradients in
 * the fixed order above (overwritten, unless opts[0].accumulate_grads: then
 * the sum is added to it).  Deterministic.  Asynchronous on `stream`. */
fe_status fe_render_batch_backward(const fe_gaussians *g, const fe_deform *deform, const fe_batch *b,
                                   void *workspace, size_t workspace_bytes, const fe_output_grads *grad_out,
                                   const fe_grads *grads, void *stream);

/* Synchronous: per-view statistics of the last batch call (host array [V]).
 * Returns the first non-OK status of the views (FE_ERR_TIMEOUT,
 * FE_ERR_WORKSPACE or FE_ERR_NONFINITE as fe_read_stats). */
fe_status fe_batch_read_stats(const void *workspace, size_t workspace_bytes, int P, int D, const fe_batch *b,
                              fe_stats *stats, void *stream);

/* Measured single-precision FMA throughput: runs an FMA-chain kernel over
 * the whole GPU for `iters` iterations per thread and writes FLOP/s
 * (2 per FMA) to *flops (host).  Synchronous; used for the FP32 roofline. */
fe_status fe_probe_fp32_peak(int iters, double *flops, void *stream);

const char *fe_status_string(fe_status s);

#ifdef __cplusplus
}
#endif

#endif /* FE4DGS_H */
