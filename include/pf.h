/*
 * pf.h -- C ABI of the Photon Field Networks hot path on B300 (sm_103a).
 *
 * Method: "Photon Field Networks for Dynamic Real-Time Volumetric Global
 * Illumination" (Bauer, Wu, Ma; arXiv 2304.07338).  The four calls of the hot
 * path follow the paper's statement of the problem:
 *   pf_build_photon_cache  -- multi-phase photon tracing (Algorithm 1, Sec. 3.2)
 *                             binned into per-(light, g) photon caches;
 *   pf_train_field         -- training samples, radiance estimates and log
 *                             targets (Sec. 3.3), field MLP (Sec. 3.4) trained
 *                             with Adam on the relative MSE (Sec. 3.5);
 *   pf_render_neural       -- volumetric path tracing with the field standing
 *                             in for indirect light (Algorithm 2, Sec. 3.6);
 *   pf_render_pathtraced   -- the plain multi-bounce path tracer the paper
 *                             compares against (Sec. 4.3).
 *
 * Conventions
 *   Memory.  Arguments named *_dev are device pointers on the context's device;
 *     *_host are host pointers.  Volumes, transfer functions and output
 *     images belong to the caller.  pf_cache and pf_field objects belong to the
 *     library and are released with pf_cache_free / pf_field_free.  The
 *     library allocates its own scratch (grown on demand, kept in the context).
 *   Streams.  Every call is ordered on the context's stream.  Calls return
 *     after enqueueing their kernels unless they write host memory (those
 *     synchronise the stream first).  pf_sync waits for the stream.
 *     pf_train_field also uses a second stream of the context internally and
 *     joins it back before returning.
 *   Threads.  A context (and the caches and fields made with it) is used by
 *     one host thread at a time; separate contexts may run concurrently.
 *   Errors.  Every call returns a pf_status and never aborts.  pf_last_error
 *     gives a message.  Device loops carry iteration limits; a kernel that
 *     hits one records it in a device error word, which the next synchronising
 *     call reports as PF_ERR_TIMEOUT (or PF_ERR_NUMERIC for a non-finite
 *     value where none is allowed).
 *   Volumes.  Scalar density on [0,1]^3, x-fastest, voxel (i,j,k) centred at
 *     ((i+1/2)/nx, (j+1/2)/ny, (k+1/2)/nz); trilinear interpolation with
 *     clamp-to-edge inside the box and zero outside.  The transfer function
 *     is a linear RGBA table over density [0,1]: sigma_t = sigma_scale *
 *     alpha(d), albedo = albedo * rgb(d).
 *   Random numbers.  Philox4x32-10 (Salmon et al., SC'11), key = seed, counter
 *     = (item, tag << 24 | sub, block).  Results are reproducible bit for bit
 *     for a given seed, independent of launch configuration.
 */
#ifndef PF_H_
#define PF_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PF_OK = 0,
  PF_ERR_INVALID_ARG = 1,
  PF_ERR_OOM = 2,
  PF_ERR_CUDA = 3,
  PF_ERR_TIMEOUT = 4,
  PF_ERR_UNSUPPORTED = 5,
  PF_ERR_NUMERIC = 6
} pf_status;

typedef struct pf_ctx pf_ctx;      /* one device + one stream + scratch */
typedef struct pf_cache pf_cache;  /* photon records, CSR, caches (device) */
typedef struct pf_field pf_field;  /* field weights, Adam state (device) */

typedef enum { PF_F32 = 0, PF_F16 = 1, PF_U8 = 2 } pf_dtype;
typedef enum { PF_PREC_F32 = 0, PF_PREC_BF16 = 1, PF_PREC_F16 = 2, PF_PREC_FP8 = 3 } pf_prec;
typedef enum { PF_LIGHT_DIRECTIONAL = 0, PF_LIGHT_POINT = 1 } pf_light_kind;

/* Scalar volume + transfer function (Algorithm 1: Volume, TransferFunction). */
typedef struct {
  int nx, ny, nz;
  int dtype;                /* pf_dtype; u8 density = value / 255 */
  const void* data_dev;     /* nx*ny*nz voxels, x fastest, caller-owned */
  float sigma_scale;        /* sigma_t = sigma_scale * alpha(d) */
  float albedo;             /* single-scattering albedo = albedo * rgb(d) */
  const float* tf_lut_dev;  /* tf_n x 4 RGBA rows over d in [0,1], tf_n >= 2 */
  int tf_n;
  float majorant;           /* global max of sigma_t (informational; 0 = unknown) */
  const float* brick_majorants_dev; /* brick majorants from pf_volume_brick_majorants, or NULL:
                                       the tracers then compute them into context scratch */
  int brick;                /* majorant brick edge in voxels: power of two, 0 = 8 */
  int brick_primary;        /* brick edge for the free flight of the neural renderer's camera
                               rays: 0 = brick, else a power-of-two multiple of brick; that
                               grid is the brick grid max-pooled over groups of bricks (camera
                               rays cross the whole volume and rarely collide, so fewer, looser
                               bricks cost less; shadow rays keep the tight grid) */
  int brick_shadow;         /* brick edge walked by the neural renderer's shadow rays: 0 = brick,
                               else a power-of-two multiple of brick; the rays cross that
                               max-pooled grid and thin its tentative collisions (one more
                               uniform each) to the brick grid's majorants, so the ratio-tracking
                               estimate is that of the brick grid at the cost of a coarser walk */
  const void* tiled_dev;    /* optional copy of the voxels in 4x4x4 tiles from pf_volume_tile
                               (same values, same dtype): a trilinear lookup then touches about
                               two cache lines instead of four; NULL reads data_dev */
} pf_volume;

/* Light source.  Directional: v = unit direction towards the light, rgb =
 * irradiance.  Point: v = position, rgb = intensity (irradiance at distance r
 * is rgb / r^2).  Light arrays are host memory, at most PF_MAX_LIGHTS. */
typedef struct { int kind; float v[3]; float rgb[3]; } pf_light;
#define PF_MAX_LIGHTS 16

/* Pinhole camera (Algorithm 2 input `camera`); row 0 is the top row.  The
 * renderers refuse (PF_ERR_INVALID_ARG) a camera with a non-finite eye, at
 * or up, eye == at, or up parallel to at - eye, and fovy_deg outside (0, 180). */
typedef struct { float eye[3], at[3], up[3]; float fovy_deg; int width, height; } pf_camera;

/* Photon field (Sec. 3.4): 6-D query (x, y, z, theta', phi', g) with theta',
 * phi' the outgoing direction in normalised spherical coordinates, an input
 * encoding, n_hidden ReLU layers of width `hidden` (32, 64 or 128) without
 * bias, a linear 3-wide output predicting L' (the log-encoded radiance,
 * Sec. 3.3.2), and decode L = 10^(-psi L').  prec selects the hidden layers'
 * arithmetic.
 * Encodings:
 *   PF_ENC_FREQUENCY  sin / cos of 2^k pi v, k < in_freqs, for all six inputs
 *                     (12 * in_freqs features);
 *   PF_ENC_HASHGRID   the paper's multiresolution hash grids (Sec. 3.4, after
 *                     Mueller et al. 2022): a 3-D grid over the position and
 *                     a 2-D grid over (theta', phi'), each with hash_levels
 *                     levels of hash_features features; level l has
 *                     N_l = floor(hash_base_res * hash_scale^l) cells per axis
 *                     (hash_scale^l as repeated FP64 products) and a table of
 *                     min((N_l + 1)^d, 2^hash_log2_size) entries, indexed
 *                     densely (x fastest) when the vertices fit and else by
 *                     (xor of v_k pi_k, pi = 1, 2654435761, 805459861, 32-bit)
 *                     mod 2^hash_log2_size; the cell is i = min(floor(p),
 *                     N_l - 1) with p = clamp(v, 0, 1) * N_l in float32, and
 *                     the features are multilinear in the corners; g enters
 *                     raw.  MLP input: [position levels, direction levels, g]
 *                     (2 L F + 1).  The tables follow the MLP weights in the
 *                     flat parameter vector (see pf_field_num_params), each
 *                     level on an 8-float boundary, initialised to
 *                     (2u - 1) 1e-4 (Philox tag 4, item 64 + 16 grid + level).
 *                     f32 / bf16 / f16 fields; SIMT kernels. */
enum { PF_ENC_FREQUENCY = 0, PF_ENC_HASHGRID = 1 };
typedef struct {
  int in_freqs;
  int hidden;
  int n_hidden;
  int prec;                 /* pf_prec */
  float psi;
  uint64_t seed;            /* Kaiming-uniform initialisation */
  int encoding;             /* PF_ENC_FREQUENCY (0) or PF_ENC_HASHGRID */
  int hash_levels;          /* [1, 16] */
  int hash_features;        /* 1, 2, 4 or 8 */
  int hash_log2_size;       /* [4, 24] */
  int hash_base_res;        /* [1, 65536] */
  float hash_scale;         /* [1, 4]; N_l must stay <= 2^22 */
} pf_field_desc;

/* Training (Sec. 3.5.1): Adam(beta1, beta2, eps), learning rate lr decayed by
 * `decay` every `decay_every` steps from step ceil(decay_start_frac*steps).
 * Targets (Sec. 3.3.1): PF_TARGET_CELL, the estimate over the query's cache
 * cell (pf_estimate_targets), or PF_TARGET_KNN, the phase-selective K-nearest
 * estimate (pf_estimate_targets_knn) with K = knn_k and the staggered radius
 * schedule of Sec. 3.5.2: stage i (of knn_stages, 1..8) starts at step
 * ceil(knn_stage_begin[i] * steps) and caps the search radius at
 * knn_radius[i] (box units, in (0, 2]); knn_stage_begin[0] = 0 and the
 * starts do not decrease.  A zero-initialised tail (target 0) keeps the cell
 * estimate. */
enum { PF_TARGET_CELL = 0, PF_TARGET_KNN = 1 };
#define PF_MAX_KNN_STAGES 8
typedef struct {
  int steps;
  int batch;
  float lr, beta1, beta2, eps;
  float decay, decay_start_frac;
  int decay_every;
  uint64_t seed;
  int target;               /* PF_TARGET_CELL or PF_TARGET_KNN */
  int knn_k;                /* K, in [1, 2^20] */
  int knn_stages;
  float knn_stage_begin[PF_MAX_KNN_STAGES];
  float knn_radius[PF_MAX_KNN_STAGES];
} pf_train_desc;

/* Totals of a photon cache.  tally = emitted, escaped, absorbed, truncated
 * (bounce cap) and Russian-roulette net power, three channels each (FP64). */
typedef struct {
  int64_t n_photons, n_records, n_keys, n_occupied;
  int res, n_lights, n_g, max_bounces;
  double tally[15];
} pf_cache_info_t;

/* ---------------------------------------------------------------- context */
/* Create a context on `device` using `cuda_stream` (a cudaStream_t; NULL =
 * legacy default stream). */
pf_status pf_create(pf_ctx** out, int device, void* cuda_stream);
pf_status pf_destroy(pf_ctx* ctx);
pf_status pf_set_stream(pf_ctx* ctx, void* cuda_stream);
const char* pf_last_error(const pf_ctx* ctx);
/* Work counters for measurement (not part of the method): while set, the
 * renderers add the number of density lookups they perform to
 * counters_dev[0], the neural renderer adds its valid samples (= field
 * queries) to counters_dev[1] and the lookups of its next-event pass (the
 * shadow rays, tracking mode) to counters_dev[2] (u64[4], caller-owned,
 * device memory).  NULL switches them off. */
pf_status pf_set_counters(pf_ctx* ctx, uint64_t* counters_dev);
/* Per-stage timing for measurement (not part of the method).  While enabled,
 * each stage's kernels are bracketed by CUDA events on the context's stream.
 * pf_stage_times synchronises, returns the accumulated milliseconds and
 * launch counts of the first n stages since the last call, and resets them. */
enum { PF_STAGE_CAMERA = 0, PF_STAGE_FIELD = 1, PF_STAGE_COMPOSE = 2, PF_STAGE_PATH = 3, PF_STAGE_TRAIN = 4,
       PF_STAGE_PHOTONS = 5, PF_STAGE_NEE = 6, PF_NUM_STAGES = 7 };
pf_status pf_stage_timing(pf_ctx* ctx, int enable);
pf_status pf_stage_times(pf_ctx* ctx, double* ms_host, int* launches_host, int n);
/* Wait for the context's stream; report any device-side error word. */
pf_status pf_sync(pf_ctx* ctx);

/* Global majorant: sigma_scale times the largest transfer-function alpha
 * over densities [0, max voxel], times (1 + 2^-10).  Synchronises; writes one
 * float to out_host. */
pf_status pf_volume_majorant(pf_ctx* ctx, const pf_volume* vol, float* out_host);
/* Voxels rearranged into 4x4x4 tiles for the tracers' gathers: tile
 * (I, J, K) (I fastest over ceil(nx/4) x ceil(ny/4) x ceil(nz/4) tiles)
 * holds voxels (4I + a, 4J + b, 4K + c) at element 16c + 4b + a, so each
 * z-slice of a tile is 16 consecutive elements (32 bytes for f16); voxels
 * past the volume's extent are zero and never read.  out_dev: that many
 * tiles x 64 elements of the volume's dtype, caller-owned; set the result as
 * vol->tiled_dev. */
pf_status pf_volume_tile(pf_ctx* ctx, const pf_volume* vol, void* out_dev);
/* Brick majorants used by delta and ratio tracking (regular tracking over a
 * piecewise-constant majorant).  With B = vol->brick, brick (i,j,k) covers
 * voxels [Bi, Bi+B) per axis (region between the planes Bi/n and B(i+1)/n,
 * the last brick cut by the box); its majorant is
 * sigma_scale times the largest TF alpha over the density range of the
 * voxels trilinear interpolation can reach there (the brick plus a one-voxel
 * apron, and density 0 for bricks on the box boundary), times (1 + 2^-10).
 * out_dev: ceil(nx/B)*ceil(ny/B)*ceil(nz/B) floats, x fastest.  Tracing walks
 * the bricks with an incremental DDA and spends each tentative collision's
 * optical-depth budget brick by brick. */
pf_status pf_volume_brick_majorants(pf_ctx* ctx, const pf_volume* vol, float* out_dev);

/* ---------------------------------------------------------------- photon caches */
/* Multi-phase photon tracing (Algorithm 1; Sec. 3.2) on the GPU.
 * photons_per_light_per_g photons are traced for every light and every g in
 * g_set (host array); photon p belongs to light p / (n_g*N) and phase
 * (p / N) % n_g.  Directional lights emit from a sqrt(3)-wide square one unit
 * upstream of the box centre, point lights isotropically.  Delta tracking
 * over the brick majorants; at real interaction j the photon is recorded
 * if j >= 2 (incoming direction, power before this vertex's albedo, cache
 * bin floor(cache_res * x)), then scaled by the albedo, stopped at
 * j == max_bounces, scattered by Henyey-Greenstein, and, for j >= 3 and
 * use_rr != 0, Russian-rouletted with q = min(1, max_c P_c / max_c P_emit).
 * Float arithmetic is IEEE single precision without contraction and with
 * the library's own logarithm and sine/cosine, so bins and counts are
 * reproducible on any IEEE machine.  cache_res must be a power of two in
 * [1, 256]; the record count is bounded by n_photons * (max_bounces - 1).
 * The result is library-owned; free it with pf_cache_free. */
pf_status pf_build_photon_cache(pf_ctx* ctx, const pf_volume* vol, const pf_light* lights, int n_lights,
                                const float* g_set, int n_g, uint64_t photons_per_light_per_g,
                                int max_bounces, int cache_res, uint64_t seed, int use_rr, pf_cache** out);
/* Synchronises; fills *out. */
pf_status pf_cache_info(pf_ctx* ctx, const pf_cache* cache, pf_cache_info_t* out);
/* Copies cache contents to caller buffers (each nullable):
 *   counts_dev   [n_keys] u32   records per key, key = (l*n_g + gi)*res^3 + bin
 *   flux_dev     [n_keys*3] f32 per-key power sums (FP64 accumulation)
 *   rec_key_dev  [n_records] u32, rec_id_dev [n_records] u32 (photon id << 4 | slot,
 *                slot = interaction index - 2), rec_dir_dev [n_records*3] f32,
 *                rec_phi_dev [n_records*3] f32, rec_pos_dev [n_records*3] f32
 *                (interaction position) -- the records grouped by key (CSR
 *                order; order inside a key is unspecified)
 *   occupied_dev [n_occupied] u32 cells with records and sigma > 0, ascending
 *   cell_sigma_dev [res^3] f32   mean sigma_t of the voxel centres in each cell */
pf_status pf_cache_export(pf_ctx* ctx, const pf_cache* cache, uint32_t* counts_dev, float* flux_dev,
                          uint32_t* rec_key_dev, uint32_t* rec_id_dev, float* rec_dir_dev, float* rec_phi_dev,
                          float* rec_pos_dev, uint32_t* occupied_dev, float* cell_sigma_dev);
pf_status pf_cache_free(pf_cache* cache);

/* ---------------------------------------------------------------- training samples */
/* Training queries (Sec. 3.3): cell uniform over the occupied cells, position
 * uniform in the cell, outgoing direction uniform on the sphere, g uniform
 * over the cache's g set.  q_dev [B*6] f32 = (x, y, z, theta', phi', g). */
pf_status pf_sample_queries(pf_ctx* ctx, const pf_cache* cache, int64_t B, int step, uint64_t seed, float* q_dev);
/* Radiance estimate per query (Sec. 3.3.1 estimator with the cache cell as
 * the gather region): L_s = sum_l sum_{records of (l, g, cell(x))}
 * p_g(dir . w) Phi / (V_cell * sigma_cell); then L' = -log10(L_s)/psi if
 * L_s > 10^-psi else 1 (Sec. 3.3.2).  ls_dev, lp_dev [B*3] f32, nullable. */
pf_status pf_estimate_targets(pf_ctx* ctx, const pf_cache* cache, const float* q_dev, int64_t B, float psi,
                              float* ls_dev, float* lp_dev);
/* Phase-selective k-nearest-neighbour radiance estimate per query (Sec. 3.3.1:
 * the adaptive-radius estimator over the photons of the query's phase g only,
 * from every light, K nearest, search radius capped at r_max):
 *   L_s = sum_{K nearest} p_g(dir_n . w) Phi_n / ((4/3) pi r^3 sigma_cell(x)),
 * "nearest" ordering records by (d2, record id) with the float32 squared
 * distance d2 = ((x_n - x)^2 + (y_n - y)^2) + (z_n - z)^2, each operation
 * rounded; records with d2 > r_max^2 (float32 product) are never used.
 * r = sqrt(d2) of the K-th record when at least K lie within r_max, else r_max.
 * sigma_cell(x) = mean sigma_t of the query's cache cell (the normaliser of
 * the cell estimate); L_s = 0 when sigma_cell or r is 0.  Then the log
 * encoding of pf_estimate_targets.  K in [1, 2^20], r_max in (0, 2] (box
 * units).  ls_dev, lp_dev [B*3] f32; k_dev [B] i32 (records used) and r_dev
 * [B] f32 (radius); all nullable. */
pf_status pf_estimate_targets_knn(pf_ctx* ctx, const pf_cache* cache, const float* q_dev, int64_t B, int K,
                                  float r_max, float psi, float* ls_dev, float* lp_dev, int32_t* k_dev,
                                  float* r_dev);

/* ---------------------------------------------------------------- photon field */
/* Create a field with seeded Kaiming-uniform weights (layer l, element e:
 * u from Philox tag 4, item l, block e/4, lane e%4; w = (2u-1) sqrt(6/fan_in)). */
pf_status pf_field_create(pf_ctx* ctx, const pf_field_desc* desc, pf_field** out);
pf_status pf_field_free(pf_field* field);
/* Number of float parameters: layers [hidden x n_in], (n_hidden-1) x
 * [hidden x hidden], [3 x hidden], each row-major [out][in], concatenated
 * (n_in = 12*in_freqs, or 2*L*F + 1 for hash grids); for hash grids then,
 * from the next multiple of 8, the position grid's level tables and the
 * direction grid's, each [entries][F] rounded up to 8 floats. */
int64_t pf_field_num_params(const pf_field* field);
pf_status pf_field_get_weights(pf_ctx* ctx, const pf_field* field, float* dst_dev);
pf_status pf_field_set_weights(pf_ctx* ctx, pf_field* field, const float* src_dev);
/* fp8 fields: per-layer power-of-two scales s = 2^ceil(log2(amax/448)), with
 * amax = max|W| for the weights and max|layer input| over B calibration
 * queries (unquantised pass) for the activations; codes = e4m3(x / s). */
pf_status pf_field_calibrate_fp8(pf_ctx* ctx, pf_field* field, const float* q_dev, int64_t B);
/* Frequency encoding gamma (Sec. 3.4) of B field queries, as the tensor-core
 * fields form it for their first layer (before the operand rounding):
 * out_dev [B][12 F] = for input d = 0..5 (x, y, z, theta', phi', g), for
 * k = 0..F-1: sin(2^k pi v_d), cos(2^k pi v_d), float32.  Sine and cosine are
 * the library's own float32 steps: at k = 0, 4, 8, ... a turn-based
 * evaluation of frac(2^(k-1) v_d), in between the double-angle formulas
 * (every feature within 6e-6 of the exact value for |v| <= 1).
 * q_dev [B*6] and out_dev are device pointers (caller-owned); F = in_freqs in
 * 1..16.  B = 0 is a no-op; B < 0, a NULL pointer or F out of range is
 * PF_ERR_INVALID_ARG.  Enqueued on the context's stream. */
pf_status pf_field_encode(pf_ctx* ctx, const float* q_dev, int64_t B, int in_freqs, float* out_dev);
/* Field forward pass: out_dev [B*3] = L' predictions for queries q_dev [B*6]. */
pf_status pf_field_forward(pf_ctx* ctx, const pf_field* field, const float* q_dev, int64_t B, float* out_dev);
/* Field backward pass: dw_dev [n_params] = sum_b (dL'_b/dW)^T dy_b (f32, bf16
 * and f16 fields). */
pf_status pf_field_backward(pf_ctx* ctx, const pf_field* field, const float* q_dev, const float* dy_dev,
                            int64_t B, float* dw_dev);
/* The training loss (Sec. 3.5.1, relative MSE (yhat - y)^2 / (y^2 + 0.01)
 * on L', averaged over the batch and the three outputs) of B queries q_dev
 * [B*6] against targets_dev [B*3] (L'), and its gradient dw_dev [n_params]
 * -- the step pf_train_field takes before Adam.  The backward pass runs with
 * loss scaling: on dy = 2 (yhat - y) / (y^2 + 0.01), 3B times the gradient
 * of the mean, so that the gradients rounded to a 16-bit field precision
 * stay in its normal range; the float32 sums are multiplied by 1/(3B).
 * loss_host (nullable): the loss; synchronises when given. */
pf_status pf_field_loss_gradient(pf_ctx* ctx, const pf_field* field, const float* q_dev, const float* targets_dev,
                                 int64_t B, float* dw_dev, float* loss_host);
/* One Adam step (Sec. 3.5.1) on the field's master weights with gradient
 * grad_dev [n_params]; t = the field's step counter + 1. */
pf_status pf_field_adam(pf_ctx* ctx, pf_field* field, const float* grad_dev, float lr, float beta1, float beta2,
                        float eps);
/* Field training (Sec. 3.3-3.5): per step, fresh queries (step index as the
 * Philox sub-stream), targets from the cache (cell or KNN estimate, with the
 * step's radius), forward, relative MSE
 * (yhat-y)^2/(y^2+0.01) averaged over batch and channels, backward, Adam.
 * loss_host [steps] (nullable) receives the loss of every step; synchronises
 * at the end. */
pf_status pf_train_field(pf_ctx* ctx, const pf_cache* cache, const pf_train_desc* desc, pf_field* field,
                         float* loss_host);

/* ---------------------------------------------------------------- rendering */
/* Neural volumetric path tracing (Algorithm 2): per pixel and sample,
 * RayGeneration (jittered pinhole ray, box test), VolumeSampling (first
 * interaction), DirectIllumination (NEE towards every light), field query at
 * the interaction with w = -ray direction, decode, and Compose
 * L = 1/spp sum_k albedo_k (L_d,k + L_i,k).  step_vox in [0.05, 64] selects ray
 * marching with step step_vox voxels (stratified inverse-CDF free flight,
 * marched shadow transmittance); step_vox == 0 selects delta tracking and
 * ratio-tracking shadow rays.  field == NULL renders direct light only.
 * out_rgb_dev [H*W*3] f32. */
pf_status pf_render_neural(pf_ctx* ctx, const pf_volume* vol, const pf_light* lights, int n_lights, float g,
                           const pf_camera* cam, int spp, float step_vox, uint64_t seed, const pf_field* field,
                           float* out_rgb_dev);
/* Ray marching with the photon field at every step (Sec. 3.6: the field
 * replaces the multiple-scattering term in ray marching as in path tracing).
 * Per pixel and sample: a jittered pinhole ray (Philox tag 1, block 0: pixel
 * jitter, march offset u); segments of step_vox voxels ([t0 + s h,
 * min(t0 + (s+1) h, t1))) sampled at fraction u; weight a_s = exp(-tau_s)
 * (1 - exp(-sigma_s len_s)) with tau_s the optical depth before the segment;
 * L = sum_s a_s albedo_s (L_d + L_i) with L_d towards every light by a marched
 * shadow ray (jitter: lane l % 4 of block 4 s + l / 4 of Philox tag 6, item
 * pixel, sub sample) and L_i = 10^(-psi L') from the field at (x_s, -d, g)
 * (no field: L_i = 0); the pixel is the mean over its samples.  Every
 * segment with sigma > 0 asks one field query: the call counts them first,
 * then renders in chunks of whole pixels whose queries fit a buffer of 2^23
 * (or one pixel's worth); synchronises once.  step_vox in [0.05, 64].
 * out_rgb_dev [H*W*3] f32. */
pf_status pf_render_raymarched(pf_ctx* ctx, const pf_volume* vol, const pf_light* lights, int n_lights, float g,
                               const pf_camera* cam, int spp, float step_vox, uint64_t seed, const pf_field* field,
                               float* out_rgb_dev);
/* Plain multi-bounce path tracer (the paper's baseline): delta tracking,
 * next-event estimation with ratio tracking at every real interaction,
 * Henyey-Greenstein continuation, at most max_bounces interactions, Russian
 * roulette from the third (use_rr).  out_rgb_dev [H*W*3] f32. */
pf_status pf_render_pathtraced(pf_ctx* ctx, const pf_volume* vol, const pf_light* lights, int n_lights, float g,
                               const pf_camera* cam, int spp, int max_bounces, uint64_t seed, int use_rr,
                               float* out_rgb_dev);

/* Allocation-free variant of pf_render_pathtraced (the paper has no
 * counterpart; it is a deployment aid).  Some callers cannot allocate device
 * memory when they render: an application that reserved its whole device
 * budget up front, a plug-in whose host forbids allocation inside the frame
 * loop, or code that must not risk the device-wide synchronisation that
 * cudaMalloc / cudaFree can cause.  This entry point needs no pf_ctx and
 * calls no allocator: its scratch is a file-scope device array of 48 MiB that
 * every GPU loading the library holds until the process exits, which bounds
 * the image to about 2.09 million pixels (1920x1080 fits); larger images are
 * rejected with PF_ERR_INVALID_ARG.  The caller passes the inputs, a stream
 * of the current device and the output image; vol->brick_majorants_dev must
 * be set (an input, e.g. from pf_volume_brick_majorants).  It accepts exactly the
 * volumes and lights pf_render_pathtraced accepts (the same checks).  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the
 * process, so make that first call before any stream capture, and do not
 * call this entry point on a device after cudaDeviceReset there (the module
 * may then be loaded at another address).  All calls
 * share the array and it keeps the last call's contents (each call resets
 * what it needs); calls that overlap on the GPU race.  Synchronises the
 * stream and reports an iteration-limit hit as PF_ERR_TIMEOUT; err_msg
 * (nullable, err_len bytes) receives a message.  Results equal
 * pf_render_pathtraced's bit for bit. */
pf_status pf_render_pathtraced_noalloc(const pf_volume* vol, const pf_light* lights, int n_lights, float g,
                                       const pf_camera* cam, int spp, int max_bounces, uint64_t seed, int use_rr,
                                       void* cuda_stream, float* out_rgb_dev, char* err_msg, int err_len);

/* sqrt(sum (a-b)^2 / n) accumulated in FP64 on the device; synchronises. */
pf_status pf_image_rmse(pf_ctx* ctx, const float* a_dev, const float* b_dev, int64_t n, double* out_host);

#ifdef __cplusplus
}
#endif
#endif
