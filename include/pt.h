/*
 * pt.h -- C ABI of the GB300 (sm_103a) neural path tracer.
 *
 * The library implements the data-parallel hot path of "Towards Neural Path
 * Tracing in SRAM" (Pupilli 2023): a Monte Carlo path tracer without light
 * sampling whose environment light is an HDR neural image field (NIF), an
 * MLP over Fourier-encoded equirect coordinates (Sections 3.1 and 3.2), with
 * the sampling loop alternating between tracing and batched network
 * inference (Section 3.3).
 *
 * Conventions for every entry point:
 *  - Pointers named d_* are CUDA device pointers owned by the caller; the
 *    library never frees them.  Pointers without the prefix are host memory,
 *    read during the call only.  Objects the library creates (pt_ctx,
 *    pt_scene, pt_nif, pt_cache) own their device memory and are released by
 *    the matching pt_destroy_* call.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls taking a stream are asynchronous and stream-ordered:
 *    they return after enqueueing work.  Device-side failures (stack or queue
 *    overflow, non-finite radiance, a bounded wait that gave up) set bits in
 *    the context's device error word and are reported by pt_check().  No
 *    kernel traps or asserts.
 *  - Calls that create objects from host arrays (pt_create_scene,
 *    pt_load_nif, pt_create_cache) copy them on a stream of the context's own
 *    that does not wait for other streams, and return once the copy is
 *    complete: they do not wait for renders still running, so the next
 *    scene or network can be built while the GPU works.  The pt_destroy_*
 *    calls free device memory with cudaFree, which waits for the device.
 *  - Every call returns a pt_status; on failure pt_last_error() describes it.
 *    No exception or exit() crosses this boundary.
 *  - A context is used by one host thread at a time.
 *
 * Scene conventions: global primitive IDs number spheres first, then quads,
 * then triangles.  Closest hits take the smallest t > 0; equal t goes to the
 * smaller ID.  Materials are rows of 8 floats [albedo r, g, b, roughness,
 * ior, emission r, g, b] with type 0 Lambertian, 1 GGX metal (F0 = albedo,
 * alpha = roughness^2), 2 dielectric (tint 1).
 */
#ifndef PT_H
#define PT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define PT_API __attribute__((visibility("default")))
#else
#define PT_API
#endif

typedef enum pt_status {
    PT_OK = 0,
    PT_EINVAL = 1,        /* invalid argument or inconsistent description */
    PT_ENOMEM = 2,        /* host or device allocation failed */
    PT_ECUDA = 3,         /* a CUDA runtime call failed */
    PT_EDEVICE = 4,       /* a kernel set bits in the device error word */
    PT_EUNSUPPORTED = 5,  /* valid request this build does not implement */
    PT_EIO = 6            /* a checkpoint file could not be written, read or verified */
} pt_status;

/* arithmetic of the neural image field's hidden layers */
typedef enum pt_precision {
    PT_FP32 = 0,          /* FP32 CUDA-core arithmetic (the accuracy reference path) */
    PT_BF16 = 1,          /* BF16 operands on tcgen05 tensor cores, FP32 accumulation */
    PT_FP8E4M3 = 2        /* FP8 E4M3 operands on tcgen05 tensor cores, FP32 accumulation */
} pt_precision;

/* bits of the device error word (pt_check) */
#define PT_ERR_STACK_OVERFLOW 0x1u   /* BVH traversal stack exhausted */
#define PT_ERR_QUEUE_OVERFLOW 0x2u   /* a ray or escape queue exceeded its capacity */
#define PT_ERR_NONFINITE      0x4u   /* a non-finite radiance value was produced */
#define PT_ERR_TIMEOUT        0x8u   /* a bounded device wait gave up */
#define PT_ERR_ITER_CAP       0x10u  /* traversal exceeded its iteration cap */
#define PT_ERR_BAD_NODE       0x20u  /* traversal met a node reference outside the node array */
#define PT_ERR_UNREADABLE     0x80000000u  /* pt_device_error_bits could not read the word */

typedef struct pt_ctx pt_ctx;
typedef struct pt_scene pt_scene;
typedef struct pt_nif pt_nif;
typedef struct pt_cache pt_cache;

/* ------------------------------------------------------------------------ */
/* Context                                                                   */
/* ------------------------------------------------------------------------ */

/* Create a context on CUDA device `device` (made current for the calling
   thread).  *out receives the handle; release it with pt_destroy.  It also
   resolves, once per device, the fixed scratch array of pt_render_noalloc
   (about 43 MiB that the driver reserves for the library's lifetime). */
PT_API pt_status pt_create(pt_ctx** out, int device);
PT_API void pt_destroy(pt_ctx* ctx);

/* Text of the last failure on this context ("" if none); valid until the
   next call on the context.  ctx may be NULL for failures of pt_create. */
PT_API const char* pt_last_error(const pt_ctx* ctx);

/* Synchronise `stream`, then read and clear the device error word into
   *bits (may be NULL).  Returns PT_EDEVICE if any bit was set, PT_ECUDA if
   the stream reported a CUDA error. */
PT_API pt_status pt_check(pt_ctx* ctx, void* stream, uint32_t* bits);

/* The context's device error word without clearing it: waits for all work
   on the context's device (cudaDeviceSynchronize), then returns the PT_ERR_*
   bits set since the last pt_check.  Returns PT_ERR_UNREADABLE alone when
   ctx is NULL or the word cannot be read (a CUDA failure). */
PT_API uint32_t pt_device_error_bits(pt_ctx* ctx);

/* ------------------------------------------------------------------------ */
/* Scenes (Section 3.1.1: the scene description is replicated per core and  */
/* serialised into one binary chunk; here it is one device arena holding     */
/* packed BVH nodes and primitive arrays).                                   */
/* ------------------------------------------------------------------------ */
typedef struct pt_scene_desc {
    int64_t n_spheres;
    const float* spheres;      /* [n_spheres][4]: centre x, y, z, radius */
    const int32_t* sphere_mat; /* [n_spheres] material index */
    int64_t n_quads;
    const float* quads;        /* [n_quads][5]: plane position p, lo_u, hi_u, lo_v, hi_v */
    const int32_t* quad_axis;  /* [n_quads] plane normal axis a; u = (a+1)%3, v = (a+2)%3 */
    const int32_t* quad_mat;
    int64_t n_verts;
    const float* verts;        /* [n_verts][3] */
    int64_t n_tris;
    const int32_t* tris;       /* [n_tris][3] vertex indices */
    const int32_t* tri_mat;
    int64_t n_mats;
    const int32_t* mat_type;   /* [n_mats] 0 Lambertian, 1 GGX metal, 2 dielectric */
    const float* mats;         /* [n_mats][8] see file header */
    float camera[10];          /* eye[3], target[3], up[3], vertical fov in degrees */
    int32_t env_is_nif;        /* 1: environment = NIF passed at render; 0: constant env_rgb */
    float env_rgb[3];
    int32_t node_format;       /* pt_node_format: the BVH node form traversal reads (0 = automatic) */
} pt_scene_desc;

/* BVH node forms (all hold the same tree; every form's child boxes contain
   the exact fp32 boxes, so every form finds the same closest hits):
   PACKED  48 bytes per node: both children as fp32 origin + fp16 extent
           rounded up (Section 3.1.4);
   DECODED 64 bytes per node: the packed boxes decoded to fp32 bounds;
   QUANT8  32 bytes per node: both children on an 8-bit grid of the node
           (origin + 8-bit codes, lo rounded down, hi up; the paper's
           quarter-precision outlook, Section 5); needs fewer than 2^24
           nodes and primitives (PT_EUNSUPPORTED otherwise).
   AUTO    DECODED for trees up to 48 MiB in that form, else PACKED. */
typedef enum { PT_NODES_AUTO = 0, PT_NODES_PACKED = 1, PT_NODES_DECODED = 2, PT_NODES_QUANT8 = 3 } pt_node_format;

typedef struct pt_scene_info {
    int64_t n_prims;
    int64_t n_nodes;           /* interior BVH nodes (leaves hold one primitive, stored in the parent) */
    int64_t node_bytes;        /* device bytes of the packed node array */
    int64_t prim_bytes;        /* device bytes of primitive data */
    int32_t bvh_depth;         /* longest root-to-leaf path */
    int32_t has_emission;
    int32_t node_format;       /* pt_node_format the traversal reads (never AUTO) */
    int32_t reserved;
    int64_t traversed_node_bytes;  /* device bytes of the node form the traversal reads */
} pt_scene_info;

/* Build the BVH on the host (binned SAH, one primitive per leaf, child boxes
   stored with fp32 origin and fp16 extent rounded so the box never shrinks,
   Section 3.1.4), pack it for 128-bit loads and upload.  Host arrays are
   read during the call only.  Fails with PT_EINVAL on out-of-range indices,
   non-finite coordinates or extents beyond the fp16 range. */
PT_API pt_status pt_create_scene(pt_ctx* ctx, const pt_scene_desc* desc, pt_scene** out);
PT_API void pt_destroy_scene(pt_scene* scene);
PT_API pt_status pt_scene_get_info(const pt_scene* scene, pt_scene_info* info);

/* The scene builder's BVH step alone, on the host (no context, no device):
   binned SAH over n primitive boxes lo[i][3], hi[i][3] with centroids at
   the box centres, one primitive per leaf, children's boxes packed as in
   pt_create_scene (12 uint32 per node: w[0..2] left fp32 origin, w[3..5]
   right fp32 origin, w[6..8] the six fp16 extents rounded up (left x, y, z,
   right x, y, z, two per word, low half first), w[9] left and w[10] right
   child reference (bit 31 set: primitive index), w[11] 0).  nodes: host
   [cap][12] (cap >= n - 1), *n_nodes the count written, *root the root
   reference (bit 31 set when n == 1; 0xFFFFFFFF when n == 0), *depth the
   tree depth.  PT_EINVAL for n < 0, a NULL output, cap too small,
   non-finite bounds or an inverted box (lo > hi on some axis);
   PT_EUNSUPPORTED when an extent exceeds the fp16 range. */
PT_API pt_status pt_build_bvh_host(int64_t n, const float* lo, const float* hi, uint32_t* nodes, int64_t cap,
                                   int64_t* n_nodes, uint32_t* root, int32_t* depth);

/* The quantised node form (PT_NODES_QUANT8) of a packed tree, on the host
   (no context, no device): nodes [n_nodes][12] as pt_build_bvh_host writes
   them, out [n_nodes][8] uint32 in the same order with the same child
   references: w[0..2] the node's grid origin (fp32 bits, per-axis minimum of
   the two children's decoded boxes); w[3] bits 0-7 the biased exponent e,
   bits 8-9 / 10-11 / 12-13 the axis offsets d_x, d_y, d_z, bit 14 / 15 the
   left / right child is a primitive, bits 16-31 the left reference's low 16
   bits; w[4] bits 0-7 the left reference's high 8 bits, bits 8-31 the right
   reference; w[5..7] twelve 8-bit codes (lo_l xyz, hi_l xyz, lo_r xyz, hi_r
   xyz, low byte first).  A bound on axis a decodes in fp32 as origin_a +
   q * 2^(e - 127 - d_a) (exact product, one rounding to nearest) and
   contains the decoded fp16-extent box: lo codes rounded down, hi codes up.
   PT_EINVAL for a NULL buffer; PT_EUNSUPPORTED when a reference or
   primitive ID needs more than 24 bits. */
PT_API pt_status pt_quantize_bvh_host(int64_t n_nodes, const uint32_t* nodes, uint32_t* out);

/* Copy the packed BVH back to the host for inspection: nodes as 12 uint32
   per node (see the packing in the library source), root reference in
   *root.  Either buffer may be NULL; sizes come from pt_scene_get_info. */
PT_API pt_status pt_scene_download_bvh(pt_ctx* ctx, const pt_scene* scene, uint32_t* nodes, uint32_t* root);

/* ------------------------------------------------------------------------ */
/* Neural image field (Section 3.2): (u, v) -> F Gaussian Fourier           */
/* frequencies as [sin 2 pi Bx (F), cos 2 pi Bx (F)] -> L dense ReLU layers  */
/* of width H -> linear layer to 3 -> fixed 3x3 colour matrix M -> exp.     */
/* ------------------------------------------------------------------------ */
typedef struct pt_nif_desc {
    int32_t n_freq;            /* F (2F <= 128) */
    int32_t hidden;            /* H (1..256) */
    int32_t n_hidden_layers;   /* L (1..8) */
    const float* params;       /* host, flat: B[F][2], then per layer W[out][in], b[out], then M[3][3] */
    int32_t skip_after;        /* 0: plain MLP.  s in [1, L - 1] (needs H > 2F): hidden layer s has H - 2F
                                  outputs and hidden layer s + 1 takes them followed by the 2F Fourier
                                  features (the paper's network: F = 20, H = 128, L = 4, s = 2, Section
                                  3.2).  Trained with FP32 GEMMs. */
} pt_nif_desc;

/* Upload FP32 master weights and build the BF16 operand image of the
   tensor-core kernel where one exists for the shape: F = 64 without a skip
   layer and H = 128, 1 <= L <= 5 (the weights stay resident in shared memory
   beside three 128-row tile slots for L <= 3, two for L = 4, one for L = 5;
   from L = 6 they do not fit, and only the FP32 path serves), H = 64 or 32,
   1 <= L <= 8 (four slots), H = 256, L = 1 (two slots); and the paper's
   network F = 20, H = 128, L = 4, skip_after = 2 (three slots).  The FP8
   image (F = 64, H = 128, L = 3 only) is built on first use, see
   pt_nif_fp8_scales.  PT_EUNSUPPORTED outside 2F <= 128, H <= 256,
   1 <= L <= 8; PT_EINVAL for a bad skip layer. */
PT_API pt_status pt_load_nif(pt_ctx* ctx, const pt_nif_desc* desc, pt_nif** out);
PT_API void pt_destroy_nif(pt_nif* nif);
/* number of floats in the flat layout */
PT_API int64_t pt_nif_param_count(const pt_nif* nif);
/* Download the current FP32 master weights in the flat layout (host buffer
   of pt_nif_param_count floats).  Synchronises the context's device. */
PT_API pt_status pt_nif_get_params(pt_ctx* ctx, const pt_nif* nif, float* params);

/* Evaluate the NIF at n coordinates: d_uv [n][2] float -> d_rgb [n][3]
   float, in the requested precision.  PT_EUNSUPPORTED for BF16 on a shape
   without a tensor-core kernel (see pt_load_nif), and for FP8 other than
   F = 64, H = 128, L = 3. */
PT_API pt_status pt_nif_eval(pt_ctx* ctx, const pt_nif* nif, int32_t precision, int64_t n, const float* d_uv,
                             float* d_rgb, void* stream);

/* FP8 E4M3 quantisation of the tensor-core NIF (PT_FP8E4M3): scales[0..3]
   are the activation scales of the features and of hidden layers 1..3
   (value = scale x E4M3 code).  Features use 1/448; hidden layers use their
   maximum over the FP32 network on a 32 x 32 grid of (u, v) pixel centres,
   divided by 448.  Weights use one scale per output row (row max / 448).
   PT_EUNSUPPORTED for shapes other than F = 64, H = 128, L = 3.  The FP8
   image (and with it these scales) is built on its first use after loading or
   after the weights change: that call synchronises the device and runs the
   calibration on the host. */
PT_API pt_status pt_nif_fp8_scales(const pt_nif* nif, float* scales);

/* Replace the FP32 master weights (host, flat layout of pt_nif_desc) and
   rebuild the derived layouts.  Synchronises `stream`. */
PT_API pt_status pt_nif_set_params(pt_ctx* ctx, pt_nif* nif, const float* params, void* stream);

/* ------------------------------------------------------------------------ */
/* NIF training (Section 3.2.1): uniform (u, v) samples, bilinear sub-pixel */
/* lookup of the HDR image, target log(max(rgb, 1e-6)), Huber loss on the   */
/* colour-matrix output, Adam on the FP32 master weights (B and M fixed).   */
/* ------------------------------------------------------------------------ */
typedef struct pt_train_cfg {
    int64_t steps;             /* Adam steps in this call */
    int64_t batch;             /* samples per step */
    float lr, beta1, beta2, eps;  /* Adam (Kingma & Ba) with bias correction */
    float huber_delta;         /* Huber loss threshold (the paper uses 1e-3) */
    uint32_t seed;             /* Philox key (seed, 1); counter (sample, global step, 0, 0) */
    int32_t precision;         /* GEMMs: PT_FP32 (CUDA cores) or PT_BF16 (tcgen05: BF16 operands, FP32
                                  accumulation; activations, gradients and master weights stay FP32) */
} pt_train_cfg;

/* Train for cfg->steps steps on d_sky, an equirect HDR image [h][w][3] float
   (row 0 = zenith, pixel centres at ((i + 0.5)/w, (j + 0.5)/h), u wraps, v
   clamps).  d_losses (nullable) receives the mean Huber loss of each step.
   Adam moments and the global step count persist in the pt_nif across calls,
   so calls continue one run.  The FP32 and tensor-core layouts are rebuilt
   at the end of the call.  FP32 arithmetic (or BF16 GEMM operands with
   cfg->precision = PT_BF16), loss sums in FP64, deterministic in both.
   PT_EUNSUPPORTED for hidden widths above 128 and for BF16 GEMMs on a shape
   whose weights do not stay resident or with a skip layer. */
PT_API pt_status pt_train_nif(pt_ctx* ctx, pt_nif* nif, const float* d_sky, int32_t w, int32_t h,
                              const pt_train_cfg* cfg, float* d_losses, void* stream);

/* Loss and gradient of one batch without updating: d_uv [n][2], d_target
   [n][3] (log space, compared with the colour-matrix output) -> d_grad
   (nullable; trainable part of the flat layout: per layer W then b) and
   *d_loss (nullable device double, mean Huber loss over n x 3).  precision
   as in pt_train_cfg. */
PT_API pt_status pt_nif_loss_grad(pt_ctx* ctx, pt_nif* nif, int64_t n, const float* d_uv, const float* d_target,
                                  float delta, int32_t precision, float* d_grad, double* d_loss, void* stream);

/* ------------------------------------------------------------------------ */
/* Rendering (Section 3.1: paths without light sampling; radiance gathered   */
/* at emitters and at escapes, where the NIF is queried; Section 3.3).       */
/* ------------------------------------------------------------------------ */
/* Scheduling of a chunk's paths (Section 3.1).  Both schedules compute the
   same paths bit for bit (same Philox counters, traversal and shading); only
   the order of the NIF escape and cache query queues differs.
   WAVEFRONT: one traversal and one shading launch per vertex, with compacted
   queues between vertices (throughput for large chunks).  The camera rays of
   a whole image (no pixel list, width % 8 == 0, height % 4 == 0) walk the
   upper tree as warp packets of 8 x 4 pixels: the same hits, but the
   traversal work of pt_last_render_work follows the packets' visiting order.
   PATHS: one launch in which each thread follows whole paths (latency for
   chunks that fit in one resident wave: a call pays for its slowest path once
   instead of for the slowest ray of every vertex).
   AUTO: PATHS when the chunk fits in one resident wave of the path kernel,
   else WAVEFRONT. */
typedef enum { PT_SCHED_AUTO = 0, PT_SCHED_WAVEFRONT = 1, PT_SCHED_PATHS = 2 } pt_schedule;

typedef struct pt_render_cfg {
    int32_t width, height;     /* image size; pixel index = y * width + x */
    int32_t spp;               /* samples (paths) per pixel */
    int32_t max_depth;         /* surface interactions per path; rays leaving vertex max_depth are not traced */
    uint32_t seed;             /* Philox key word 0 (key word 1 = stream tag 0) */
    int32_t rr;                /* 1: Russian roulette from vertex rr_start, continue prob min(1, max tp) */
    int32_t rr_start;
    int32_t precision;         /* pt_precision of the NIF at escapes */
    int64_t chunk_slots;       /* paths per wavefront chunk; 0 = automatic; rounded to whole samples */
    int32_t first_sample;      /* sample index of the first path per pixel (Philox counter word 1 =
                                  first_sample + s): disjoint ranges render independent sample sets */
    int32_t schedule;          /* pt_schedule: how the paths of a chunk are scheduled (same results) */
    int32_t cache_vertex;      /* pt_render with a radiance cache: paths end in the cache at this vertex
                                  (>= 2); 0 without a cache.  pt_render_pixels and pt_render_noalloc
                                  need 0; pt_render_cached takes its own argument (0 here or equal) */
} pt_render_cfg;

/* Render the image (Section 3.3: paths traced through the scene, escapes
   shaded by the NIF): d_image [height][width][3] float, caller-owned device
   memory, the mean over spp paths of each pixel.  Path (pixel p, sample s)
   draws Philox-4x32-10 words with key (seed, 0) and counter (p,
   first_sample + s, k, 0) at vertex k (k = 0 for the camera jitter).  `nif`
   is required when the scene's environment is a NIF and ignored otherwise.
   `cache` (nullable): a radiance cache on the same device; with it, paths
   that reach vertex cfg->cache_vertex (>= 2) end there with the cache's
   prediction of the radiance leaving that vertex (the same paths and image
   as pt_render_cached over all pixels).  PT_EINVAL when cache and
   cfg->cache_vertex do not go together (a cache needs cache_vertex >= 2,
   no cache needs 0).  Asynchronous on `stream`; device-side failures are
   reported through the error word (pt_check, pt_device_error_bits). */
PT_API pt_status pt_render(pt_ctx* ctx, const pt_scene* scene, const pt_nif* nif, const pt_cache* cache,
                           const pt_render_cfg* cfg, float* d_image, void* stream);

/* Render all spp paths of a list of pixels.  d_pixels: [n_pix] int64 pixel
   indices (NULL = all width*height pixels in order).  Outputs: d_pixel_rgb
   [n_pix][3] mean radiance; d_slot_rgb (nullable) [spp][n_pix][3] radiance
   of each path; d_hit_ids (nullable) [spp][n_pix][max_depth] int32 primitive
   hit at each vertex, -1 for an escape, -2 when not traced. */
PT_API pt_status pt_render_pixels(pt_ctx* ctx, const pt_scene* scene, const pt_nif* nif, const pt_render_cfg* cfg,
                                  int64_t n_pix, const int64_t* d_pixels, float* d_pixel_rgb, float* d_slot_rgb,
                                  int32_t* d_hit_ids, void* stream);

/* Statistics of the last pt_render / pt_render_pixels call on this context
   (valid after pt_check): rays traced per vertex and escapes shaded by the
   NIF.  counts: [max_depth + 1] int64 -> counts[k-1] = rays traced at vertex
   k, counts[max_depth] = NIF evaluations; with n >= max_depth + 2,
   counts[max_depth + 1] = radiance-cache queries (pt_render_cached). */
PT_API pt_status pt_last_render_counts(pt_ctx* ctx, int64_t* counts, int32_t n);

/* Kernels this library has launched in this process (all contexts and
   threads), each kernel of a replayed CUDA graph included: the difference
   across a region of work is the number of the library's kernels it ran.
   Library copies and memsets are not kernels and are not counted. */
PT_API pt_status pt_kernel_launches(uint64_t* count);

/* Schedule the last render's last chunk ran with: PT_SCHED_WAVEFRONT or
   PT_SCHED_PATHS (PT_SCHED_AUTO before the first render).  A replayed
   render reports the schedule it was captured with, which is the same. */
PT_API pt_status pt_last_render_schedule(pt_ctx* ctx, int32_t* schedule);

/* Traversal work of the last render (valid after pt_check): work[0] BVH
   node fetches (each tests the two child boxes), work[1] sphere, work[2]
   quad, work[3] triangle intersection tests, summed over rays (a node that a
   warp packet visits counts once for each lane whose ray entered it).
   Writes min(n, 4) values. */
PT_API pt_status pt_last_render_work(pt_ctx* ctx, int64_t* work, int32_t n);

/* Kernel timing.  While enabled, the library records a CUDA event pair on
   the launching stream around each of its kernel launches and accumulates
   the device time per kernel kind: 0 traversal (k_trace of each wavefront
   vertex, or the whole path-per-thread launch k_paths, which also shades),
   1 NIF evaluation, 2 sample reduction, 3 other (training and utilities),
   4 radiance-cache queries, 5 wavefront shading and compaction (k_bounce).
   pt_profile_read synchronises the device, writes up to n kinds of total
   milliseconds and launch counts (either pointer may be NULL) and resets
   the totals. */
#define PT_KIND_TRACE 0
#define PT_KIND_NIF 1
#define PT_KIND_REDUCE 2
#define PT_KIND_OTHER 3
#define PT_KIND_CACHE 4    /* radiance-cache queries */
#define PT_KIND_SHADE 5    /* wavefront shading step */
#define PT_N_KINDS 6
PT_API pt_status pt_profile_enable(pt_ctx* ctx, int32_t enable);
PT_API pt_status pt_profile_read(pt_ctx* ctx, double* ms, int64_t* launches, int32_t n);

/* Measurement helper (the paper has no counterpart): the FP32 FMA rate of
   the current device, the denominator of the traversal roofline.  Launches
   one kernel on `stream` in which every thread of 8 resident 256-thread
   blocks per SM runs 8 independent chains of `iters` dependent FMAs;
   *flop receives the FLOPs it performs (2 per FMA), to be divided by the
   launch's event-timed duration.  d_sink: one caller-owned device float,
   never written for the values used.  PT_EINVAL for iters < 1 or NULL
   pointers. */
PT_API pt_status pt_microbench_ffma(int64_t iters, float* d_sink, double* flop, void* stream);

/* Measurement helper (the paper has no counterpart): the L2 read bandwidth
   of the current device, the denominator of the large tree's L2 traffic.
   Launches one kernel on `stream` in which 8 resident 256-thread blocks per
   SM read the caller's device buffer d_buf (bytes, 16-byte aligned; pick it
   well inside L2, e.g. 48 MiB) `reps` times over in 16-byte words with
   loads that bypass L1; *bytes_read receives the bytes read (bytes rounded
   down to 16 x reps), to be divided by the event-timed duration of a launch
   after a warm-up launch has brought the buffer into L2.  d_sink: one
   caller-owned device word, never written in practice.  PT_EINVAL for a
   NULL pointer, an unaligned buffer, bytes < 16 or reps < 1. */
PT_API pt_status pt_microbench_l2_read(const void* d_buf, int64_t bytes, int32_t reps, uint32_t* d_sink,
                                       double* bytes_read, void* stream);

/* ------------------------------------------------------------------------ */
/* Building blocks of the same path, exposed for testing and for callers    */
/* that stream their own rays (Section 3.1.2).                               */
/* ------------------------------------------------------------------------ */

/* Philox-4x32-10 (Salmon et al. 2011): d_ctr [n][4] counters with key
   (seed, tag) -> d_out [n][4] words. */
PT_API pt_status pt_philox(pt_ctx* ctx, uint32_t seed, uint32_t tag, int64_t n, const uint32_t* d_ctr,
                           uint32_t* d_out, void* stream);

/* Camera rays of slots [first_slot, first_slot + n) where slot = s * W * H +
   p: d_org, d_dir [n][3] float (directions unit length). */
PT_API pt_status pt_primary_rays(pt_ctx* ctx, const pt_scene* scene, const pt_render_cfg* cfg, int64_t first_slot,
                                 int64_t n, float* d_org, float* d_dir, void* stream);

/* Closest hit of n rays through the packed BVH: d_org, d_dir [n][3] float
   (directions need not be normalised for triangles and quads; spheres
   assume unit length) -> d_t [n] (INFINITY on a miss), d_prim [n] int32
   (-1 on a miss). */
PT_API pt_status pt_trace_rays(pt_ctx* ctx, const pt_scene* scene, int64_t n, const float* d_org, const float* d_dir,
                               float* d_t, int32_t* d_prim, void* stream);

/* ------------------------------------------------------------------------ */
/* Neural radiance cache (Mueller et al. 2021; Section 2.1 cites it as the  */
/* way to end paths early).  A path that hits at the cache vertex stops     */
/* there and takes tp * max(cache(x, wo, n), 0) as the rest of its          */
/* radiance.  Inputs: position normalised to the box [lo, hi] and encoded   */
/* as sin/cos(2^j pi p) for j < n_freq per axis, then wo (unit vector to    */
/* the previous vertex) and n (geometric normal facing wo), both raw.       */
/* Network: n_hidden_layers x FC-hidden ReLU, then FC-3 (linear).  FP32.    */
/* ------------------------------------------------------------------------ */
typedef struct pt_cache_desc {
    int32_t n_freq;            /* J: frequencies per axis (1..15) */
    int32_t hidden;            /* must be 64 */
    int32_t n_hidden_layers;   /* L: 1..7 */
    const float* params;       /* host: W0 [hidden][6J+6], b0, W1 [hidden][hidden], b1, ..., WL [3][hidden], bL
                                  (PyTorch Linear layout, layers in order) */
    float lo[3], hi[3];        /* position box (hi > lo per axis) */
} pt_cache_desc;

/* Create a cache on the context's device; parameters are copied. */
PT_API pt_status pt_create_cache(pt_ctx* ctx, const pt_cache_desc* desc, pt_cache** out);
PT_API void pt_destroy_cache(pt_cache* cache);
PT_API int64_t pt_cache_param_count(const pt_cache* cache);
/* host copy of / replacement for the flat FP32 parameters (pt_cache_desc layout); set_params resets Adam */
PT_API pt_status pt_cache_get_params(pt_ctx* ctx, const pt_cache* cache, float* params);
PT_API pt_status pt_cache_set_params(pt_ctx* ctx, pt_cache* cache, const float* params, void* stream);

/* Raw network outputs (no clamp) for d_q [n][9] = x, wo, n -> d_out [n][3].
   precision PT_FP32 (FP32 throughout) or PT_BF16 (tcgen05 tensor cores: BF16
   inputs, weights and activations, FP32 accumulation and biases; needs
   n_freq = 12, hidden = 64, 5 hidden layers, else PT_EUNSUPPORTED). */
PT_API pt_status pt_cache_eval(pt_ctx* ctx, const pt_cache* cache, int32_t precision, int64_t n, const float* d_q,
                               float* d_out, void* stream);

/* Relative L2 loss (y - t)^2 / (sg(y)^2 + 0.01), sg() holding the
   prediction constant in the gradient, averaged over all n x 3 entries;
   rows with d_mask[i] == 0 (d_mask nullable) contribute zero.  d_q [n][9],
   d_target [n][3] -> d_grad (nullable, flat layout) and *d_loss (nullable
   device double).  Nothing is updated.  precision: the GEMMs, PT_FP32 (CUDA
   cores) or PT_BF16 (tcgen05, BF16 operands, FP32 accumulation). */
PT_API pt_status pt_cache_loss_grad(pt_ctx* ctx, pt_cache* cache, int64_t n, const float* d_q, const float* d_target,
                                    const int32_t* d_mask, int32_t precision, float* d_grad, double* d_loss,
                                    void* stream);

typedef struct pt_cache_train_cfg {
    int32_t width, height;     /* image whose pixels the training paths start from */
    int32_t n_train;           /* training paths per frame (2^16) */
    int32_t max_depth;         /* their depth (plain path tracing, no cache) */
    int32_t rec_vertex;        /* the vertex whose suffix radiance is the target (the cache vertex) */
    uint32_t seed;             /* Philox key word 0 */
    uint32_t frame;            /* frame index */
    int32_t precision;         /* NIF precision at the training paths' escapes */
    float lr, beta1, beta2, eps;  /* Adam */
    int32_t train_precision;   /* the network's training GEMMs: PT_FP32 or PT_BF16 (tcgen05) */
} pt_cache_train_cfg;

/* One online training step of a frame.  Pixel i of the n_train training
   paths is word 0 of Philox (key (seed, 2), counter (i, frame, 0, 0)) modulo
   width*height; path i is that pixel's render path with sample index
   2^30 + frame (key (seed, 0); renders whose sample indices stay below 2^30
   never share a stream with it), traced to max_depth without the cache.
   A path that hits at rec_vertex gives the sample (x, wo, n) -> (L_path -
   L_before) / tp, the radiance it gathered from that vertex on divided by
   the throughput reaching it; other paths are masked out.  Then one Adam
   step on the relative L2 loss of pt_cache_loss_grad.  d_loss (nullable
   device float) receives the loss.  Adam's moments and step count persist
   in the cache. */
PT_API pt_status pt_train_cache(pt_ctx* ctx, const pt_scene* scene, const pt_nif* nif, pt_cache* cache,
                                const pt_cache_train_cfg* cfg, float* d_loss, void* stream);

/* pt_render_pixels with a radiance cache at vertex cache_vertex (cache and
   cache_vertex >= 2 together, or NULL and 0; the cache runs in BF16 on the
   tensor cores when cfg->precision is not PT_FP32 and its shape allows, else
   in FP32) and, when rec_vertex > 0,
   vertex records d_rec [spp][n_pix][16] of each path at rec_vertex: x[3],
   wo[3], n[3], throughput[3], radiance gathered before the vertex[3], valid
   (1.0 when the path hit there, else 0.0). */
PT_API pt_status pt_render_cached(pt_ctx* ctx, const pt_scene* scene, const pt_nif* nif, const pt_cache* cache,
                                  int32_t cache_vertex, int32_t rec_vertex, const pt_render_cfg* cfg, int64_t n_pix,
                                  const int64_t* d_pixels, float* d_pixel_rgb, float* d_slot_rgb, float* d_rec,
                                  int32_t* d_hit_ids, void* stream);

/* ------------------------------------------------------------------------ */
/* Rendering without device allocation.  The paper has no counterpart: this */
/* serves callers that may not allocate device memory at render time (a host */
/* application that owns all GPU memory through its own pool, or a real-time */
/* loop that must stay off the driver's allocator).                         */
/* ------------------------------------------------------------------------ */

/* Same image as pt_render with precision PT_FP32, but every byte of wavefront
   scratch comes from one fixed array compiled into the library (about 43 MiB
   per GPU, held until the process exits); the call makes no cudaMalloc,
   cudaFree or other allocating call.  Limits: at most 262144 pixels per
   frame (one sample of the frame must fit the array) and the FP32 network;
   larger frames return PT_EINVAL, other precisions PT_EUNSUPPORTED.
   The scene's device must be current.  The array's device address is
   looked up by pt_create on that device (which is when the driver loads
   and reserves the array, also under lazy module loading), so the render
   call itself only reads it; no object of this library survives a
   cudaDeviceReset.  All calls share the array and it keeps the last
   call's contents (the call clears what must start at zero), so calls whose
   GPU work overlaps race: serialise them on one stream.  d_err (nullable,
   caller-owned device word) receives the PT_ERR_* bits the kernels set;
   without it they are discarded.  No context is needed; failures are
   reported by the return code only.  It always runs the wavefront schedule
   (cfg->schedule is not read; the image is the same either way). */
PT_API pt_status pt_render_noalloc(const pt_scene* scene, const pt_nif* nif, const pt_render_cfg* cfg,
                                   float* d_image, uint32_t* d_err, void* stream);

/* ------------------------------------------------------------------------ */
/* Checkpoints: the trained NIF (Section 3.2.1, weights saved after training */
/* and loaded by the renderer) and per-frame snapshots of the radiance cache. */
/* A checkpoint is one little-endian binary file:                           */
/*   bytes  0-7   magic "PTCKPT01"                                           */
/*          8-11  uint32 kind: 1 = NIF, 2 = radiance cache                   */
/*         12-15  uint32 version (1)                                         */
/*         16-31  int32 dims[4]: NIF (n_freq, hidden, n_hidden_layers,       */
/*                skip_after),                                               */
/*                cache (n_freq, hidden, n_hidden_layers, 0)                 */
/*         32-55  float box[6]: cache lo[3], hi[3]; zeros for a NIF          */
/*         56-63  int64 n_params (the flat FP32 layout of pt_nif_desc /      */
/*                pt_cache_desc)                                             */
/*         64-71  int64 n_adam: entries of each Adam moment, 0 when training */
/*                has not started (NIF: the trainable part; cache: all)      */
/*         72-79  int64 adam_t: Adam steps taken (also the NIF's Philox     */
/*                step counter)                                              */
/*   then float params[n_params], float m[n_adam], float v[n_adam], and a   */
/*   uint64 FNV-1a hash of every preceding byte.                             */
/* Loading a checkpoint restores the object and its training state, so      */
/* training resumed from it continues the run bit-exactly.                   */
/* ------------------------------------------------------------------------ */
typedef struct pt_checkpoint_info {
    int32_t kind;              /* 1 NIF, 2 radiance cache */
    int32_t version;
    int32_t dims[4];
    float lo[3], hi[3];        /* cache box (zeros for a NIF) */
    int64_t n_params, n_adam, adam_t;
} pt_checkpoint_info;

/* Write `nif` (weights and, once training started, Adam state) to `path`.
   Synchronises `stream` first; PT_EIO when the file cannot be written. */
PT_API pt_status pt_save_nif(pt_ctx* ctx, const pt_nif* nif, const char* path, void* stream);
/* Create a NIF from a checkpoint (as pt_load_nif, plus the training state).
   PT_EIO for a missing, truncated or corrupted file (hash mismatch), PT_EINVAL
   for a checkpoint of another kind or an unknown version. */
PT_API pt_status pt_load_nif_file(pt_ctx* ctx, const char* path, pt_nif** out);
/* The same for a radiance cache (pt_create_cache plus its training state). */
PT_API pt_status pt_save_cache(pt_ctx* ctx, const pt_cache* cache, const char* path, void* stream);
PT_API pt_status pt_load_cache_file(pt_ctx* ctx, const char* path, pt_cache** out);
/* Read and verify a checkpoint's header and hash without a device or
   context (host only). */
PT_API pt_status pt_checkpoint_read_info(const char* path, pt_checkpoint_info* out);

/* Failure-path self-test of the device waits (no fault involved): one CTA
   waits, with the same bounded mbarrier wait the tensor-core kernels use, on
   a barrier nothing arrives on.  After `seconds` (0 < seconds <= 2) the wait
   gives up, sets PT_ERR_TIMEOUT in the context's error word (reported by the
   next pt_check) and the kernel returns; the context stays usable.
   *waited_s (nullable) receives the time the device waited.  Synchronises
   `stream`. */
PT_API pt_status pt_selftest_wait_timeout(pt_ctx* ctx, double seconds, double* waited_s, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PT_H */
