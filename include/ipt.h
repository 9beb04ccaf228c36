/*
 * ipt.h -- C ABI of the GB300 inverse path tracer.
 *
 * Inverse Path Tracing (Azinovic, Li, Kaplanyan, Niessner, CVPR 2019) recovers
 * per-object materials and emission of a triangle-mesh scene from images with
 * known camera poses, by nesting a differentiable Monte Carlo path tracer in
 * stochastic gradient descent (Sec. 3, Fig. 2).  The problem statement gives
 * the shape of this interface: geometry, segmentation, camera poses and images
 * go in; the unknowns Theta = {M, L} (Sec. 3.2) are optimised and come out.
 *
 * Conventions shared by every call:
 *   - Every call returns an ipt_status; nothing throws across the ABI.
 *   - Host pointers are read during the call and copied; the caller keeps
 *     ownership.  Device pointers must stay valid until the work queued on the
 *     context's stream has finished; the library never frees them.
 *   - Device work is queued on the context's CUDA stream.  Calls that return
 *     host data (loss, parameters) synchronise that stream first.
 *   - Argument errors are reported as IPT_ERR_INVALID_ARG before anything is
 *     launched.  Errors found on the device set a status word that the next
 *     synchronising call returns: a traversal stack overflow as IPT_ERR_CUDA,
 *     a non-finite loss or gradient met by an Adam step as IPT_ERR_NONFINITE,
 *     a bounded wait for the tensor cores that gave up (radiance-cache
 *     training) as IPT_ERR_TIMEOUT.
 *   - Non-finite guard: every Adam step (ipt_adam_step, ipt_step,
 *     ipt_batch_step per member, ipt_disney_step) first checks, on the device,
 *     the gradient it is given and, for the context's own gradient, the loss
 *     that came with it.  On a NaN or infinity it skips the update: the
 *     parameters, Adam moments and Adam step count stay those of the last good
 *     step (the iteration counter of ipt_step still advances, so the next step
 *     draws new samples), and IPT_ERR_NONFINITE is reported.
 *   - ipt_last_error_detail gives a one-line description of the last error.
 *   - A context is bound to one device and one stream and is not thread-safe.
 *
 * Parameters (Sec. 4.1, Sec. 4.2): one row of 10 floats per segment (object),
 *   [kd_r, kd_g, kd_b, ks_r, ks_g, ks_b, roughness, e_r, e_g, e_b],
 *   row-major S x 10.  f_r = kd/pi + ks * D G2 / (4 |n.wi| |n.wo|), GGX with
 *   alpha = max(roughness^2, 1e-4), height-correlated Smith G2, no Fresnel.
 *   Emitted radiance is emission_scale * e * profile, with the profile
 *   (w . n)_+ of Sec. 4.3 (or a uniform front-face profile).
 */
#ifndef IPT_H_
#define IPT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IPT_OK = 0,
  IPT_ERR_INVALID_ARG = 1,
  IPT_ERR_OUT_OF_MEMORY = 2,
  IPT_ERR_CUDA = 3,
  IPT_ERR_TIMEOUT = 4,
  IPT_ERR_NONFINITE = 5,
  IPT_ERR_NOT_READY = 6
} ipt_status;

typedef struct ipt_ctx ipt_ctx;

/* ipt_options.flags bits. */
#define IPT_FLAG_KERNEL_TIMING 1 /* time every launch with CUDA events on the context stream */
#define IPT_FLAG_COUNTERS 2      /* count rays, BVH node visits and triangle tests */
#define IPT_FLAG_OWN_STREAM 4    /* create and own a non-blocking stream, ignoring .stream */

/* Kernel ids reported by ipt_kernel_times. */
typedef enum {
  IPT_KERNEL_PREPARE = 0,
  IPT_KERNEL_FORWARD = 1,
  IPT_KERNEL_ADJOINT = 2,
  IPT_KERNEL_FINALIZE = 3,
  IPT_KERNEL_ADAM = 4,
  IPT_KERNEL_TRACE = 5,
  IPT_KERNEL_PHILOX = 6,
  /* wavefront integrator stages */
  IPT_KERNEL_WF_CAMERA = 7,
  IPT_KERNEL_WF_CLOSEST = 8,
  IPT_KERNEL_WF_SHADOW = 9,
  IPT_KERNEL_WF_SHADE = 10,
  IPT_KERNEL_WF_ADJ_A = 11,
  IPT_KERNEL_WF_ADJ_CONNECT = 12,
  IPT_KERNEL_WF_ADJ_B = 13,
  IPT_KERNEL_WF_REDUCE = 14,
  IPT_KERNEL_BATCH_STEP = 15, /* one replay of a batch's iteration graph */
  /* radiance cache */
  IPT_KERNEL_CACHE_INFER = 16,   /* queries of the forward pass */
  IPT_KERNEL_CACHE_VJP = 17,     /* queries of the adjoint pass, with input gradients */
  IPT_KERNEL_CACHE_RECORDS = 18, /* training-record targets */
  IPT_KERNEL_CACHE_GRAD = 19,    /* training forward + backward */
  IPT_KERNEL_CACHE_ADAM = 20,    /* optimizer step on weights and hash table */
  IPT_KERNEL_WF_SORT = 21,       /* reordering of secondary closest-hit rays */
  IPT_KERNEL_COUNT = 22
} ipt_kernel_id;

/* device: CUDA device ordinal.  stream: the cudaStream_t every call queues
 * its work on (NULL = the legacy default stream), unless flags has
 * IPT_FLAG_OWN_STREAM.  seed: Philox key for all sample sets. */
typedef struct {
  int32_t device;
  void* stream;
  uint64_t seed;
  int32_t flags; /* IPT_FLAG_* bits */
} ipt_options;

/* Integrator configuration of a context (picked per workload by the autotuner
 * in paper_1903_07145_gb300/autotune.py; every configuration traces
 * identical paths).
 *   integrator: 0 = megakernel (one thread per path, every stage inline),
 *     1 = wavefront (chunks of path slots; persistent traversal kernels over
 *     compacted ray queues).
 *   wavefront_slots: path slots per wavefront chunk (0 = 1 << 20); rounded
 *     down to whole pixels.  The context keeps 162 bytes of device memory
 *     per slot, and once it has run an adjoint 52 + 40 D more (D: the
 *     largest max_depth its adjoints have used; the Disney model's adjoint
 *     adds 32 D + 64); the buffers are allocated on first use and grow, never
 *     shrink, while the context lives.
 *   trace_steps: refill point of the persistent traversal kernels (0 = 16).
 *     4- and 8-wide BVHs: a warp fetches new rays once this many of its 32
 *     lanes are idle (values above 32 act as 32).  Binary BVH: node visits
 *     per refill round.
 *   blocks_per_sm: persistent blocks per SM for the wavefront kernels (0 =
 *     as many as fit).
 *   bvh_width: BVH the traversal walks (every integrator, and
 *     ipt_trace_rays): 2 = binary nodes with float boxes, 4 = 4-wide nodes
 *     with 8-bit child boxes visited nearest first, 8 = 8-wide nodes with
 *     8-bit child boxes whose children sit in slots by octant and are
 *     visited in the ray's octant order (0 = 4).  All three give the same
 *     closest hits up to exact ties.
 *   sort_cells, sort_dirs: wavefront launches reorder each secondary
 *     closest-hit queue (after the first vertex) by bin before tracing it:
 *     origin cell (sort_cells^3 boxes of the ray's scene's bounding box)
 *     and direction cell (the cube-map face of the direction's dominant
 *     axis, split into sort_dirs x sort_dirs squares; 0: the origin cell
 *     alone).  sort_cells = 0 traces in queue order.  The bins of one scene,
 *     6 sort_dirs^2 sort_cells^3 (sort_cells^3 without directions), must not
 *     exceed 8192; a chunk of a batch keeps its scenes' bins apart and
 *     coarsens the grid (fewer cells, then fewer directions) until they fit
 *     8192 together.  The order changes no result.  The context keeps 6
 *     more bytes of device memory per slot for it. */
typedef struct {
  int32_t integrator;
  uint32_t wavefront_slots;
  uint32_t trace_steps;
  uint32_t blocks_per_sm;
  uint32_t bvh_width;
  uint32_t sort_cells;
  uint32_t sort_dirs;
} ipt_config;

/* Pinhole camera.  cam_to_world is row-major 3x4; its columns are the
 * camera's right, up and backward axes and its position (the camera looks
 * down its -z axis; image row 0 is the top).  Pixel j integrates a box filter
 * over its own footprint (h_j in Eq. 1). */
typedef struct {
  float cam_to_world[12];
  float fov_y_deg;
  uint32_t width;
  uint32_t height;
} ipt_camera;

/* Per-call tracing options.
 *   spp_r, spp_d: samples per pixel of the residual image and of the
 *     derivative estimate; the two use independent sample sets (Sec. 3.3),
 *     unless gradcheck_same_set is non-zero.
 *   max_depth: number of scattering events (1 = direct light only, App. A.3).
 *   loss: 0 = L2, 1 = L1 (Eq. 3).
 *   nee, mis: light sampling and its MIS with BRDF sampling (App. A.2).
 *   emission_profile: 0 = (w.n)_+ (Sec. 4.3), 1 = uniform over the front face.
 *   pixel_batch: 0 = every pixel of every view.  B > 0 = a stochastic batch
 *     of B pixels drawn per iteration uniformly, with replacement, from all
 *     pixels of all views (Sec. 4.5 uses B = 8); see ipt_pick_pixels for the
 *     draw.  Batch entry b traces its pixel with the sample counters
 *     b*spp .. b*spp+spp-1 of each set, and the loss and its gradient are
 *     normalised by the 3B entry-channels, so the batch loss is an unbiased
 *     estimate of the full-image loss.  Accepted by ipt_loss_grad, ipt_step
 *     and ipt_batch_step (every other call requires 0), on either integrator
 *     (batches of scenes: wavefront); not with the radiance cache.
 *     B * max(spp_r, spp_d) must stay below 2^32. */
typedef struct {
  uint32_t spp_r;
  uint32_t spp_d;
  uint32_t max_depth;
  int32_t loss;
  int32_t nee;
  int32_t mis;
  int32_t emission_profile;
  int32_t gradcheck_same_set;
  uint32_t pixel_batch;
} ipt_trace_opts;

/* Adam (Sec. 4.5: Adam, learning rate 5e-3) plus the L1 emission regulariser
 * of Sec. 4.4 with weight l1_emission; after the update kd, ks are clamped
 * to [0,1], roughness to [0.02,1], emission to >= 0. */
typedef struct {
  float lr;
  float beta1;
  float beta2;
  float eps;
  float l1_emission;
} ipt_adam_opts;

/* Sample-set ids for ipt_render / ipt_backward. */
#define IPT_SET_RESIDUAL 0u
#define IPT_SET_DERIVATIVE 1u
#define IPT_SET_TARGET 2u
#define IPT_SET_CACHE 3u
#define IPT_SET_PICK 4u /* the pixel-batch draw (ipt_pick_pixels) */

/* Create a context on opt->device.  *out receives the handle.  Fails with
 * IPT_ERR_CUDA if the device cannot be used. */
ipt_status ipt_create(ipt_ctx** out, const ipt_options* opt);

/* Set or read the integrator configuration (see ipt_config).  Setting it
 * may release wavefront buffers; they are re-created on first use. */
ipt_status ipt_config_set(ipt_ctx* ctx, const ipt_config* cfg);
ipt_status ipt_config_get(const ipt_ctx* ctx, ipt_config* cfg);

/* Release every device buffer the context owns.  NULL is accepted. */
ipt_status ipt_destroy(ipt_ctx* ctx);

/* Static string for a status code. */
const char* ipt_status_string(ipt_status s);

/* Copy the last error message (NUL-terminated, truncated to n bytes). */
ipt_status ipt_last_error_detail(const ipt_ctx* ctx, char* buf, size_t n);

/* Scene geometry (Sec. 4.2): n_vert positions (host, n_vert x 3), optional
 * per-vertex normals (host, n_vert x 3, NULL = geometric normals; when given
 * they are interpolated with barycentrics), n_tri index triples (host), a
 * segment id per triangle (host, each < n_seg).  Builds the BVH (binned SAH)
 * and the per-segment light-selection tables, uploads everything and returns
 * the scene's id.  Errors: non-finite coordinates, out-of-range index or
 * segment id, zero triangles, degenerate (zero-area) triangles. */
ipt_status ipt_scene_upload(ipt_ctx* ctx, const float* pos, uint32_t n_vert, const float* nrm,
                            const uint32_t* idx, uint32_t n_tri, const uint32_t* tri_seg,
                            uint32_t n_seg, float emission_scale, int32_t* scene_id);

/* Camera poses and (optionally) the captured images I_C (Sec. 3.2, 3.4).
 * cams: host array of n_views cameras.  target_rgb: linear RGB, the views'
 * W*H*3 float images concatenated in view order; host or device according to
 * target_on_device; NULL keeps no target.  Copied into the context. */
ipt_status ipt_views_set(ipt_ctx* ctx, int32_t scene, const ipt_camera* cams, uint32_t n_views,
                         const float* target_rgb, int32_t target_on_device);

/* Replace the targets only (same layout as ipt_views_set). */
ipt_status ipt_targets_set(ipt_ctx* ctx, int32_t scene, const float* target_rgb,
                           int32_t target_on_device);

/* Parameters Theta: host S x 10 floats (layout above).  free_mask: host
 * S x 10 bytes, non-zero = optimised (NULL = all free).  Resets the Adam
 * moments and step counter. */
ipt_status ipt_params_set(ipt_ctx* ctx, int32_t scene, const float* params,
                          const uint8_t* free_mask);

/* Copy the current parameters to host memory (S x 10 floats). */
ipt_status ipt_params_get(ipt_ctx* ctx, int32_t scene, float* params_out);

/* Device pointer of the context's S x 10 parameter buffer (valid until the
 * scene is destroyed). */
ipt_status ipt_params_device(ipt_ctx* ctx, int32_t scene, float** params_dev);

/* Forward render (Eq. 1-2) of one view (view >= 0) or all views (view = -1,
 * images concatenated in view order): per-pixel mean over `spp` samples of
 * sample set `set` at iteration `iteration`, and optionally the per-pixel
 * mean of squares (for standard errors).  params / sampling_params: device
 * S x 10 (NULL = the context's parameters; sampling_params NULL = params).
 * Sampling decisions (lobe choice, light selection, MIS weights) use
 * sampling_params; BRDF values and emission use params.  rgb_out, msq_out:
 * device float arrays of pixels x 3 (msq_out may be NULL). */
ipt_status ipt_render(ipt_ctx* ctx, int32_t scene, int32_t view, const ipt_trace_opts* opts,
                      uint32_t set, uint32_t spp, uint64_t iteration, const float* params,
                      const float* sampling_params, float* rgb_out, float* msq_out);

/* Vector-Jacobian product of the rendered images (Eq. 5-6): grad_out (device
 * S x 10, overwritten) = sum over all pixels of all views and channels of
 * grad_image * d(mean over spp_d samples of set `set`)/d(params), with pdfs,
 * MIS weights and light selection held at sampling_params.  grad_image:
 * device, all views concatenated, pixels x 3. */
ipt_status ipt_backward(ipt_ctx* ctx, int32_t scene, const ipt_trace_opts* opts, uint32_t set,
                        uint64_t iteration, const float* params, const float* sampling_params,
                        const float* grad_image, float* grad_out);

/* One gradient evaluation of the nested SGD (Sec. 3.2-3.4): render the
 * residual set with spp_r, compare with the targets (L2 or L1, normalised by
 * the number of pixel-channels N), and trace the derivative set with spp_d
 * to accumulate dE/dTheta.  loss_out (host, may be NULL) receives E; grad_out
 * (device S x 10, may be NULL to keep the gradient in the context). */
ipt_status ipt_loss_grad(ipt_ctx* ctx, int32_t scene, const ipt_trace_opts* opts,
                         uint64_t iteration, double* loss_out, float* grad_out);

/* The part of ipt_loss_grad that belongs to pixels [pix_begin, pix_begin +
 * pix_count) of the concatenated views, for sharding one scene over several
 * devices (each pixel's residual and derivative samples stay on one shard).
 * Both the loss and the gradient are normalised by n_total_pixels (the pixel
 * count of all shards together), so the shards' results add up to the
 * unsharded ones.  grad_out: device S x 10 (required); loss_out: host, may be
 * NULL.  Errors: an empty range or one beyond the views. */
ipt_status ipt_loss_grad_shard(ipt_ctx* ctx, int32_t scene, const ipt_trace_opts* opts,
                               uint64_t iteration, uint64_t pix_begin, uint64_t pix_count,
                               uint64_t n_total_pixels, double* loss_out, float* grad_out);

/* Adam step on the context's parameters (Sec. 4.5) with grad (device S x 10;
 * NULL = the gradient left by ipt_loss_grad). */
ipt_status ipt_adam_step(ipt_ctx* ctx, int32_t scene, const float* grad,
                         const ipt_adam_opts* adam);

/* ipt_loss_grad followed by ipt_adam_step; the iteration counter lives on
 * the device and advances by one.  loss_out (host, may be NULL) receives the
 * loss of this step and makes the call synchronous. */
ipt_status ipt_step(ipt_ctx* ctx, int32_t scene, const ipt_trace_opts* opts,
                    const ipt_adam_opts* adam, double* loss_out);

/* Closest-hit ray casting (the paper's Embree queries, App. E): n rays,
 * device arrays orig and dir (n x 3 floats), optional skip triangle per ray
 * (device int32, -1 = none), t in (0, inf).  Outputs (device, n each):
 * original triangle id or -1, t, barycentrics u, v with hit point
 * (1-u-v) p0 + u p1 + v p2.  Any output but tri_out may be NULL. */
ipt_status ipt_trace_rays(ipt_ctx* ctx, int32_t scene, uint32_t n, const float* orig,
                          const float* dir, const int32_t* skip, int32_t* tri_out, float* t_out,
                          float* u_out, float* v_out);

/* The pixel batch of one iteration (Sec. 4.5: each optimisation step draws
 * its B pixels uniformly over every pixel of every view): ids_out[b] (device, `batch`
 * entries) receives the global pixel id (views concatenated in order, row
 * major within a view) of entry b, floor(x * N / 2^32), where N is the
 * scene's pixel count and x the first word of Philox4x32-10 at the scene's
 * key (seed_lo, seed_hi ^ scene) and counter
 * (b, 0, (IPT_SET_PICK << 24) | (iteration & 0xFFFFFF), 0).  This is the draw
 * ipt_loss_grad and ipt_step make when opts->pixel_batch = batch. */
ipt_status ipt_pick_pixels(ipt_ctx* ctx, int32_t scene, uint32_t batch, uint64_t iteration, uint32_t* ids_out);

/* Philox4x32-10 (Salmon et al., SC'11), the counter-based generator behind
 * every random decision: out[4i..4i+3] = philox(ctr[4i..4i+3], key[2i..2i+1]).
 * All arrays on the device. */
ipt_status ipt_philox(ipt_ctx* ctx, uint32_t n, const uint32_t* ctr, const uint32_t* key,
                      uint32_t* out);

/* Wait for the context's stream and return any device-side error. */
ipt_status ipt_synchronize(ipt_ctx* ctx);

/* Scene statistics: triangles, segments, BVH inner nodes, BVH depth,
 * views, total pixels.  Any pointer may be NULL. */
ipt_status ipt_scene_info(ipt_ctx* ctx, int32_t scene, uint32_t* n_tri, uint32_t* n_seg,
                          uint32_t* n_nodes, uint32_t* bvh_depth, uint32_t* n_views,
                          uint64_t* n_pixels);

/* Per-kernel device time (requires IPT_FLAG_KERNEL_TIMING): total_ms and
 * launches are arrays of IPT_KERNEL_COUNT entries (either may be NULL),
 * accumulated since the last reset.  Synchronises the context's stream. */
ipt_status ipt_kernel_times(ipt_ctx* ctx, double* total_ms, uint64_t* launches, int32_t reset);

/* Traversal counters (requires IPT_FLAG_COUNTERS), accumulated since the
 * last reset: out[0] closest-hit rays, out[1] shadow rays, out[2] BVH
 * inner-node visits and out[3] triangle tests of closest-hit rays, out[4]
 * node visits and out[5] triangle tests of shadow rays (out has 6 entries).
 * Synchronises the context's stream. */
ipt_status ipt_counters_read(ipt_ctx* ctx, uint64_t* out, int32_t reset);

/* Batches: several scenes optimised together (independent problems; each
 * keeps its own parameters, Adam state and loss).  Every stage of an
 * iteration is one launch over the concatenated pixels of all member
 * scenes, and ipt_batch_step replays the whole iteration as one CUDA graph
 * (captured on first use and again whenever the options or the context
 * configuration change).  A scene gives the same paths in a batch as alone.
 *
 * ipt_batch_create: scenes (host array of n scene ids, each with views,
 * targets and parameters set) -> *batch_id.  Copies each member's current
 * parameters and free mask; Adam state and the iteration counter start at 0.
 * Errors: unknown or repeated scene, missing views or targets, n == 0 or
 * more than 4096 members. */
ipt_status ipt_batch_create(ipt_ctx* ctx, const int32_t* scenes, uint32_t n, int32_t* batch_id);

/* One nested-SGD iteration of every member (residual set, derivative set,
 * per-member loss and Adam step).  losses_out: host array of n (may be NULL;
 * then the call does not wait for the GPU). */
ipt_status ipt_batch_step(ipt_ctx* ctx, int32_t batch, const ipt_trace_opts* opts,
                          const ipt_adam_opts* adam, double* losses_out);

/* Current parameters of member `member` (0-based position in the batch):
 * host S x 10 floats. */
ipt_status ipt_batch_params_get(ipt_ctx* ctx, int32_t batch, uint32_t member, float* params_out);

/* Which members take part in the batch's next steps (active[k] != 0 for
 * member k; host array of one byte per member; all members start active).
 * An inactive member traces nothing and keeps its parameters and Adam
 * moments as they are; its loss reads 0.  This lets a serving loop retire
 * scenes that have finished (or hold some back) without rebuilding the
 * batch; Adam's bias correction counts the batch's iterations, so a member
 * made active again continues with the batch's step count.  The next step
 * recaptures the graph when the set changed. */
ipt_status ipt_batch_set_active(ipt_ctx* ctx, int32_t batch, const uint8_t* active);

/* Release a batch (its member scenes stay). */
ipt_status ipt_batch_destroy(ipt_ctx* ctx, int32_t batch);

/* ipt_backward without any device allocation (the paper has no counterpart;
 * this is an interface convenience).  Same arguments, result and errors as
 * ipt_backward, for callers that may not allocate device memory at the point
 * of the call: code that runs under CUDA stream capture (where cudaMalloc is
 * not a stream operation), real-time loops and embedders that own the device
 * memory budget.  Inputs and outputs are still the caller's.  The only scratch,
 * an FP64 S x 10 gradient accumulator, is a file-scope __device__ array sized
 * for at most 1024 segments (80 KiB, held by every device that loads the
 * library until the process exits); a scene with more segments is rejected
 * with IPT_ERR_INVALID_ARG.  The first call with each context looks the
 * array's address on the context's device up (cudaGetSymbolAddress) and keeps
 * it in the context; make that first call before any stream capture.  A
 * device reset ends every context, and with it the kept address: create a
 * new context after one.  The array is cleared at the start of every call,
 * and all calls share it: calls whose work overlaps on the GPU (other
 * streams, other contexts on the same device) race on it.  It always runs the
 * plain estimator on the megakernel integrator (a scene's radiance cache is
 * not used), whatever ipt_config_set selected.  With IPT_FLAG_KERNEL_TIMING
 * its launches are timed like ipt_backward's (prepare, adjoint, finalize);
 * the CUDA events this takes are host objects, not device memory. */
ipt_status ipt_backward_noalloc(ipt_ctx* ctx, int32_t scene, const ipt_trace_opts* opts, uint32_t set,
                                uint64_t iteration, const float* params, const float* sampling_params,
                                const float* grad_image, float* grad_out);

/* ---------------------------------------------------------------------------
 * Learned radiance cache (the paper has none: its estimator traces every path
 * to max_depth, Sec. 3.1; this is an optional acceleration of that
 * estimator).  Paths end at vertex b_term (0 = the camera ray's hit): the
 * emission found there is kept, and instead of next-event estimation and
 * continuation the cache's prediction of the reflected radiance at that
 * vertex, times the path throughput, is added.  The prediction is a small
 * network: a multiresolution hash-grid encoding of the position (Mueller et
 * al., SIGGRAPH 2022: 16 levels x 2 features, 2^19 entries per level,
 * resolutions 16..2048 over the scene's bounding box), spherical harmonics of
 * degrees 0..3 of the direction towards the previous vertex and of the
 * oriented shading normal, and the terminal segment's kd, ks and roughness
 * (input of 80 values, the last 9 zero), then 80 -> 64 -> 64 -> 64 -> 64 ->
 * 16 with ReLU, no biases, the first 3 outputs being RGB.  It runs on BF16
 * tensor cores with FP32 accumulation.
 *
 * Gradients: the adjoint pass chains the cache's derivative with respect to
 * the terminal segment's kd, ks and roughness into that segment's gradient,
 * and the prediction into the earlier vertices' Eq. 6 terms.  What the
 * reflected radiance owes to other segments' parameters is not seen: the
 * cached gradient is biased, and ipt_cache_bias measures by how much.
 *
 * Training (self-supervised, in ipt_step or ipt_cache_train): train_spp
 * full-length paths per pixel from a fourth independent sample set
 * (IPT_SET_CACHE) record, at vertex b_term, the inputs and the reflected
 * radiance they gather after it (next-event estimation at b_term and every
 * later contribution, with unit throughput at b_term).  The records are
 * split into train_steps minibatches, each one step of Adam on the relative
 * L2 loss mean((y - t)^2 / (y^2 + 0.01)) (the denominator held constant)
 * over the weights and the hash table.
 *
 * A cache belongs to one scene and serves that scene's ipt_render,
 * ipt_backward, ipt_loss_grad(_shard) and ipt_step calls while active; the
 * megakernel integrator and batches do not use it (the cached passes always
 * run on the wavefront integrator).
 * ------------------------------------------------------------------------- */

/* Number of FP32 network weights: W1 (80 x 64), W2..W4 (64 x 64), W5
 * (64 x 16), each row-major with the input index first, concatenated. */
#define IPT_CACHE_WEIGHTS 18432u
/* Hash-table size in floats: [16 levels][2^19 entries][2 features]. */
#define IPT_CACHE_TABLE_FLOATS (16u * 524288u * 2u)

typedef struct {
  int32_t enabled;          /* 1: the scene's passes use the cached estimator */
  uint32_t b_term;          /* vertex where paths end in the cache; >= 1, and
                               < max_depth to have any effect */
  uint32_t train_spp;       /* training paths per pixel; 0: max(1, spp_r / 16) */
  uint32_t train_steps;     /* Adam steps per training pass (1..64) */
  uint32_t record_capacity; /* records kept per training pass (others dropped) */
  float lr, beta1, beta2, eps; /* Adam on weights and table */
  float bias_threshold;     /* ipt_cache_bias turns the cache off above this
                               relative bias (0: never) */
  uint64_t init_seed;       /* weights: uniform +-sqrt(6 / fan_in); table:
                               uniform +-1e-4 */
} ipt_cache_opts;

typedef struct {
  int32_t active;           /* the cached estimator is in use */
  int32_t fell_back;        /* turned off by ipt_cache_bias */
  uint32_t records;         /* training paths that reached b_term in the last
                               pass (may exceed record_capacity) */
  uint32_t pad;
  uint64_t train_steps;     /* Adam steps taken */
  double last_loss;         /* mean relative L2 over the last pass's records */
  double image_bias;        /* last ipt_cache_bias results, -1: not measured */
  double grad_bias;
  float lo[3], hi[3];       /* box mapped to the grid's unit cube */
  int32_t res[16];          /* grid resolution of each level */
} ipt_cache_stats;

/* Create (or reconfigure) the scene's cache.  The first call allocates and
 * initialises the network from init_seed; later calls change the options and
 * keep the weights.  enabled = 0 turns the cached estimator off (the state is
 * kept).  Errors: b_term == 0, train_steps outside 1..64, record_capacity 0,
 * non-positive lr or eps, beta outside [0, 1). */
ipt_status ipt_cache_configure(ipt_ctx* ctx, int32_t scene, const ipt_cache_opts* opts);

/* Replace the weights (host, IPT_CACHE_WEIGHTS floats) and/or the hash table
 * (host, IPT_CACHE_TABLE_FLOATS floats); NULL keeps that part.  Adam state is
 * cleared.  Requires a configured cache. */
ipt_status ipt_cache_weights_set(ipt_ctx* ctx, int32_t scene, const float* weights, const float* table);

/* Copy the weights and/or the hash table to host arrays (NULL skips). */
ipt_status ipt_cache_weights_get(ipt_ctx* ctx, int32_t scene, float* weights, float* table);

/* Evaluate the network on n rows given directly (all device arrays):
 * x01 (n x 3, positions in the unit cube, clamped to [0, 1]), dir and nrm
 * (n x 3, unit vectors), params7 (n x 7: kd rgb, ks rgb, roughness).
 * rgb_out (n x 3) receives the prediction.  With upstream (n x 3, nullable)
 * and dparams_out (n x 7, nullable) both given, dparams_out receives
 * upstream . d(prediction) / d(params7) per row. */
ipt_status ipt_cache_eval(ipt_ctx* ctx, int32_t scene, uint32_t n, const float* x01, const float* dir,
                          const float* nrm, const float* params7, const float* upstream, float* rgb_out,
                          float* dparams_out);

/* Relative-L2 loss of n rows against target (n x 3, device) and its
 * gradient, without a step: *loss_out (host, nullable) receives the mean over
 * rows and channels; grad_weights (device, IPT_CACHE_WEIGHTS, nullable) and
 * grad_table (device, IPT_CACHE_TABLE_FLOATS, nullable) receive the
 * gradients of that mean. */
ipt_status ipt_cache_grad(ipt_ctx* ctx, int32_t scene, uint32_t n, const float* x01, const float* dir,
                          const float* nrm, const float* params7, const float* target, double* loss_out,
                          float* grad_weights, float* grad_table);

/* One training pass for `iteration`: record the training paths (set
 * IPT_SET_CACHE, opts->max_depth, nee, mis, profile; spp from the cache
 * options) and take train_steps Adam steps.  ipt_step calls this after the
 * gradient passes while the cache is active. */
ipt_status ipt_cache_train(ipt_ctx* ctx, int32_t scene, const ipt_trace_opts* opts, uint64_t iteration);

/* Records of the last training pass: *n_out receives how many are kept
 * (<= record_capacity); records (host, nullable, capacity >= *n_out x 16
 * floats) receives per record [path id = scene pixel * train_spp + sample,
 * segment, x (3, world), direction (3), normal (3), target (3), 0, 0, 0].
 * Record order is not deterministic. */
ipt_status ipt_cache_records(ipt_ctx* ctx, int32_t scene, uint32_t* n_out, float* records);

ipt_status ipt_cache_status(ipt_ctx* ctx, int32_t scene, ipt_cache_stats* out);

/* Bias of the cached estimator against the plain one, both with the sample
 * sets of `iteration` at `spp` samples per pixel (common random numbers up to
 * the cache vertex): image_bias = ||I_cache - I_plain|| / ||I_plain|| over all
 * views (set 0); grad_bias the same for the loss gradients (residual and
 * derivative sets at spp samples each; needs targets; -1 without).  opts
 * gives max_depth, loss, nee, mis and profile.  When bias_threshold > 0 and either
 * exceeds it, the cache is turned off (stats.fell_back = 1).  Outputs are
 * host pointers (nullable). */
ipt_status ipt_cache_bias(ipt_ctx* ctx, int32_t scene, const ipt_trace_opts* opts, uint32_t spp,
                          uint64_t iteration, double* image_bias, double* grad_bias);

/* Checkpoint of a scene's optimisation (to resume a run of the nested SGD of
 * Sec. 3 later or elsewhere): its parameters, free mask, Adam moments and
 * step count, its iteration counter and, when it has a radiance cache, the
 * cache's weights, hash table, their Adam moments and step count and its
 * on/off state, and, when Disney parameters are set (ipt_disney_params_set),
 * their blocks, free mask, Adam moments, step count and iteration (restored
 * into the target scene's Disney state, which a load creates if needed).
 * Host memory, the library's own layout: a 64-byte header
 * ("IPTCKPT1", version, segment count, counters, flags) followed by the
 * arrays.  Save: with buf == NULL, *n receives the size in bytes; with a
 * buffer, *n must hold at least that size and receives the bytes written.
 * Load: the checkpoint must come from a scene with the same number of
 * segments, and a checkpoint with cache state needs a configured cache
 * (ipt_cache_configure) on the target scene; the cache's options are not part
 * of the checkpoint.  Batches (ipt_batch_*) keep their own state and are not
 * covered.  Errors: IPT_ERR_INVALID_ARG for a short buffer, a wrong magic,
 * version or size, or a segment-count or cache mismatch, before any state
 * changes. */
ipt_status ipt_checkpoint_save(ipt_ctx* ctx, int32_t scene, void* buf, size_t* n);
ipt_status ipt_checkpoint_load(ipt_ctx* ctx, int32_t scene, const void* buf, size_t n);

/* Disney material model (Sec. 4.1: a base colour and ten further values,
 * all in [0, 1]; Burley 2012 with linear base colour), on the integrator
 * ipt_config_set selects (both build the same paths).  Its parameter block per
 * segment is 16 floats: base colour r, g, b (0-2), subsurface (3), metallic
 * (4), specular (5), specular tint (6), roughness (7), anisotropic (8), sheen
 * (9), sheen tint (10), clearcoat (11), clearcoat gloss (12), emission r, g, b
 * (13-15).  Anisotropy is measured in the tangent frame whose first axis is
 * the hit triangle's first edge (vertex 1 - vertex 0) made orthogonal to the
 * shading normal.  Paths, light selection, sample sets, the random-number
 * slots, pixel batches and the losses are those of the Lambert + GGX calls;
 * the sampler mixes cosine-weighted diffuse, visible anisotropic GGX normals
 * and GTR1 clearcoat normals with lobe weights (1 - metallic) lum(base),
 * (1 - metallic) 0.08 specular + metallic lum(base) and clearcoat / 4.
 * These blocks live beside the scene's 10-value parameters (which the other
 * calls keep using); batches, checkpoints and the radiance cache do not
 * include them.  Errors: as the corresponding Lambert + GGX call; calls other
 * than ipt_disney_params_set fail until the blocks are set. */
#define IPT_DISNEY_VALUES 16u

/* Host S x 16 parameters and (NULL = all free) S x 16 free mask; resets the
 * Adam moments, step counter and iteration. */
ipt_status ipt_disney_params_set(ipt_ctx* ctx, int32_t scene, const float* params, const uint8_t* free_mask);
ipt_status ipt_disney_params_get(ipt_ctx* ctx, int32_t scene, float* params_out);

/* As ipt_render; sampling_params (device S x 16, nullable) replaces the
 * parameters the sampler and light selection use. */
ipt_status ipt_disney_render(ipt_ctx* ctx, int32_t scene, int32_t view, const ipt_trace_opts* opts, uint32_t set,
                             uint32_t spp, uint64_t iteration, const float* sampling_params, float* rgb_out,
                             float* msq_out);

/* As ipt_loss_grad; grad_out: device S x 16 floats, nullable. */
ipt_status ipt_disney_loss_grad(ipt_ctx* ctx, int32_t scene, const ipt_trace_opts* opts, uint64_t iteration,
                                double* loss_out, float* grad_out);

/* As ipt_step: loss and gradient at the scene's Disney iteration counter,
 * then Adam with the material values clamped to [0, 1] (roughness to
 * [0.02, 1]) and emission kept >= 0 under the L1 term. */
ipt_status ipt_disney_step(ipt_ctx* ctx, int32_t scene, const ipt_trace_opts* opts, const ipt_adam_opts* adam,
                           double* loss_out);

/* Measurement support (not part of the method).  Achievable bandwidth, in
 * GB/s (1e9 bytes), of random 64-byte line gathers over a device buffer of
 * `bytes` bytes on `device`: each line read with two 256-bit read-only loads
 * (as the traversal reads a node), four independent gathers in flight per
 * thread, 8 blocks of 256 threads per SM, about 10 ms per timed run, best of
 * three timed runs after a warm-up.
 * This is the access pattern of BVH traversal, and with the size of a
 * scene's node and triangle arrays the denominator of its roofline.  The
 * buffer is allocated and freed inside the call.  Errors: bytes < 64 KiB or
 * above 2^32 lines, out of memory, CUDA failures. */
ipt_status ipt_probe_gather(int32_t device, uint64_t bytes, double* gbs_out);

/* Build check (not part of the method): the binary version (major * 10 +
 * minor of the SM architecture, 103 for sm_103a) and PTX version the device
 * runs the library's kernels from, as cudaFuncGetAttributes reports them for
 * one of its kernels on `device`.  Either output may be NULL, not both.
 * Errors: IPT_ERR_CUDA when the device cannot load the kernels (for example a
 * GPU other than compute capability 10.3). */
ipt_status ipt_build_info(int32_t device, int32_t* binary_version, int32_t* ptx_version);

#ifdef __cplusplus
}
#endif

#endif /* IPT_H_ */
