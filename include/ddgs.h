/*
 * ddgs.h -- C ABI of the GB300 (sm_103a) DDGS-CT DRR splatting library.
 *
 * Renders a digitally reconstructed radiograph (DRR) from a cloud of 3D
 * Gaussians (DDGS-CT, Sec. 3.1-3.2 and Appendix A) and differentiates it with
 * respect to every Gaussian parameter, the shared radiosity bases and the
 * per-view source/detector pose (Sec. 3.1 "differentiable", Sec. 4.3 pose
 * registration).
 *
 * Conventions
 *   - All array pointers in the structs and calls are DEVICE pointers
 *     (cudaMalloc / torch CUDA tensors) unless a comment says "host". They are
 *     owned by the caller and must stay valid until the stream reaches the
 *     end of the call's work. The library owns only a workspace.
 *   - Every call is asynchronous on the given stream (a cudaStream_t passed as
 *     void*; NULL = legacy default stream) unless stated otherwise.
 *   - No call aborts, throws or prints. Each returns a ddgs_status. Errors
 *     found while kernels run (capacity overflow in the no-sync mode, a
 *     non-finite input) are latched in the workspace and returned by
 *     ddgs_sync_status(); a synchronising render reports a non-finite input
 *     itself.
 *   - Feature dimension k (1..32, default 8) and harmonic degree L (1..3,
 *     default 1; k_L = L(L+2)) per cloud: k = 8, L = 1 is the paper's
 *     evaluation setting (Sec. 4.1); Table 2 uses L = 3, Table 5 k = 1..32.
 *
 * Geometry (the paper fixes cone-beam X-ray imaging but not its
 * parameterisation; this is the library's reading). The X-ray source is the
 * camera origin; the pose [R | t] maps world to camera coordinates; the
 * detector is the plane z = sdd with pixel pitch (pitch_u, pitch_v); pixel
 * (row i, col j) has centre (j + 1/2, i + 1/2) in pixel units; the principal
 * point is (W/2 + off_u, H/2 + off_v).
 */
#ifndef DDGS_H
#define DDGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DDGS_FEAT_DIM 8   /* default k: features per Gaussian (Sec. 4.1) */
#define DDGS_SH_DIM 3     /* default k_L = L(L+2) at L = 1 (Sec. 3.2, after Eq. 3) */
#define DDGS_MAX_FEAT_DIM 32
#define DDGS_MAX_SH_DEGREE 3

typedef enum {
  DDGS_OK = 0,
  DDGS_ERR_INVALID_ARG = 1,   /* a null pointer, negative size, bad tile ... */
  DDGS_ERR_CAPACITY = 2,      /* no-sync mode: pairs exceeded the reserved capacity */
  DDGS_ERR_NONFINITE = 3,     /* an input parameter (Gaussian, basis, pose or
                                 detector entry) was NaN or infinite */
  DDGS_ERR_TIMEOUT = 4,       /* reserved: a bounded device wait gave up */
  DDGS_ERR_CUDA = 5,          /* a CUDA runtime call failed (see ddgs_last_cuda_error) */
  DDGS_ERR_UNSUPPORTED = 6,   /* e.g. no sm_103 device */
  DDGS_ERR_OUT_OF_MEMORY = 7  /* workspace growth failed */
} ddgs_status;

/* A cloud of n Gaussians g_i = {mu_i, Sigma_i, alpha_i, f_i} (Sec. 3.1).
 * Sigma_i = R(q_i) diag(exp(log_s_i))^2 R(q_i)^T; alpha_i = sigmoid(logit_i).
 * Gaussians [0, n_iso) are isotropic, [n_iso, n) direction-dependent; the two
 * sets are distinct Gaussians (Sec. 3.2, Eq. 3) rendered jointly (App. A.2). */
typedef struct {
  int64_t n;
  int64_t n_iso;
  const float *means;          /* [n][3] world coordinates */
  const float *log_scales;     /* [n][3] */
  const float *quats;          /* [n][4] (w, x, y, z), any non-zero norm */
  const float *opacity_logits; /* [n] */
  const float *feat_iso;       /* [n_iso][k] f_iso (Eq. 3); may be NULL if n_iso == 0 */
  const void *feat_dir;        /* [n - n_iso][k] f_dir (Eq. 3); float32 or bfloat16 */
  int32_t feat_dir_bf16;       /* 0: feat_dir is float32, 1: bfloat16 */
  const float *b_iso;          /* [k] shared isotropic basis b_iso (Eq. 3) */
  const float *B_dir;          /* [k_L][k] shared direction basis B_dir (Eq. 3), row-major;
                                  rows ordered by degree l = 1..L, order m = -l..l */
  int32_t feat_dim;            /* k, 1..32 (0 = 8); rows of 8 must be 16-byte aligned */
  int32_t sh_degree;           /* L, 1..3 (0 = 1) */
  int32_t entangled;           /* 1: every Gaussian carries both terms of Eq. 3,
                                  c = sigmoid(b_iso . f + Y(d) . B_dir f) (the
                                  direct-entangled ablation of Table 3); f is the
                                  Gaussian's row of feat_iso or feat_dir */
  int32_t per_pixel;           /* 1: Y is evaluated at the direction of each pixel's
                                  ray (source to pixel centre) instead of the
                                  source-to-mean direction; needs L = 1 */
} ddgs_gaussians;

/* n_views cone-beam views sharing one detector size. */
typedef struct {
  int32_t n_views;
  int32_t height, width;       /* detector pixels (rows, columns); host values */
  const float *world_to_cam;   /* [n_views][3][4] rigid pose (R | t), row-major */
  const float *detector;       /* [n_views][5]: sdd, pitch_u, pitch_v, off_u, off_v */
} ddgs_views;

/* Cutoffs and tiling. The paper states none of them (Eq. 1 sums over all
 * Gaussians); these are the usual 3D Gaussian splatting choices. */
typedef struct {
  int32_t tile;      /* tile edge in pixels: 8, 16 or 32 */
  float dilation;    /* added to the 2D covariance diagonal, pixels^2 (e.g. 0.3) */
  float near_plane;  /* Gaussians with camera z <= near_plane are culled; z >= sdd too */
  float alpha_min;   /* sigma below this is skipped (e.g. 1/255) */
  float alpha_max;   /* sigma = min(alpha_max, alpha G) (e.g. 0.99) */
  float t_min;       /* the walk stops before T would drop below this (e.g. 1e-4) */
  float q_max;       /* Mahalanobis cutoff q <= q_max (e.g. 9) */
  int32_t no_sync;   /* 0: a render may synchronise the stream once to size the
                        workspace; 1: never synchronise (CUDA-graph capture):
                        capacities come from ddgs_workspace_reserve and an
                        overflow is latched as DDGS_ERR_CAPACITY */
  int32_t batch_depth; /* list entries a rasteriser block stages per round:
                          128, 256 or 512; 32: every warp streams its own
                          8 x 4 pixel region's list 32 entries at a time, with
                          no block-wide staging (other values = 256) */
} ddgs_config;

/* Gradient outputs of ddgs_render_backward. Every pointer may be NULL (that
 * gradient is skipped). Layouts equal the inputs', always float32; outputs
 * are overwritten, not accumulated. */
typedef struct {
  float *means, *log_scales, *quats, *opacity_logits;
  float *feat_iso, *feat_dir;
  float *b_iso, *B_dir;
  float *world_to_cam;         /* [n_views][3][4]: dL/d(pose entries) */
} ddgs_grads;

typedef struct ddgs_workspace ddgs_workspace;

/* Workspace (infrastructure; no passage of the paper defines it): the
 * per-(view, Gaussian) projections, the depth-ordered tile lists that Eq. 1's
 * product over nearer Gaussians needs (Sec. 3.1), their counters, the
 * request/view tables and the device status word, on the device that is
 * current at creation; a call that uses the workspace while another device is
 * current returns DDGS_ERR_INVALID_ARG. Owned by the library between create
 * and destroy (destroy accepts NULL). One workspace serves one render at a
 * time; ddgs_render_backward reads what the preceding ddgs_render left. A
 * CUDA graph that captured calls on a workspace stays valid while no call
 * with another batch layout (counts, view sizes, tile) or a larger size runs
 * on that workspace. Create returns DDGS_ERR_OUT_OF_MEMORY or DDGS_ERR_CUDA
 * on failure, with *ws set to NULL. */
ddgs_status ddgs_workspace_create(ddgs_workspace **ws);
ddgs_status ddgs_workspace_destroy(ddgs_workspace *ws);

/* Grow the workspace so that renders of up to `records` (= views x
 * Gaussians), `pairs` (Gaussian-tile overlaps) and `tiles` (= views x tiles
 * per view) never reallocate. Synchronises the device. Required before
 * no_sync renders. */
ddgs_status ddgs_workspace_reserve(ddgs_workspace *ws, int64_t records,
                                   int64_t pairs, int64_t tiles);

/* Forward rendering, Eq. 1 of the paper with the radiosity of Eq. 3:
 *   C(p) = sum_j c_j sigma_j prod_{l<j} (1 - sigma_l),
 *   sigma_j = min(alpha_max, alpha_j exp(-q_j / 2)),
 *   q_j = (p - mu-hat_j)^T Sigma-hat_j^-1 (p - mu-hat_j),
 * over the Gaussians whose q <= q_max and sigma >= alpha_min, in ascending
 * camera depth of their means (ties: ascending index), isotropic and
 * direction-dependent Gaussians in one list (App. A.2), stopping before the
 * transmittance would drop below t_min. mu-hat, Sigma-hat are the perspective
 * projection of the mean and the Jacobian projection of Sigma (+ dilation).
 * Radiosity (Eq. 3): c = sigmoid(b_iso . f) for isotropic Gaussians and
 * c = sigmoid(Y_1..L(d) . B_dir f) for direction-dependent ones, with d the
 * unit direction from the source to the mean in world coordinates and Y the
 * real spherical harmonics of degrees 1..L (Y_1(d) = sqrt(3/(4 pi)) (-d_y,
 * d_z, -d_x)). With g->entangled every Gaussian uses both terms; with
 * g->per_pixel d is the pixel ray's direction, so c varies across a
 * Gaussian's footprint. A per_pixel render with cfg->no_sync needs the
 * workspace to have held a per_pixel render before (its extra per-record
 * storage is allocated then).
 * Outputs (device, [n_views][height][width], overwritten):
 *   image   C(p) (background 0, no log transform; App. A.1)
 *   t_final transmittance after the last Gaussian added
 *   n_last  1 + position, in the pixel's tile list, of the last Gaussian
 *           added (0 if none); needed by the backward pass.
 * Synchronises the stream once (to size the tile lists) unless cfg->no_sync.
 * Pairs are limited to 2^31 - 1 per render (DDGS_ERR_CAPACITY beyond).
 * A NaN or infinite input (Gaussian parameter, basis entry, pose or detector
 * entry) makes a synchronising call return DDGS_ERR_NONFINITE after writing
 * its outputs as the kernels computed them (such a Gaussian is culled when its
 * geometry is not finite, and otherwise reaches the image); with
 * cfg->no_sync the status is latched for ddgs_sync_status(). */
ddgs_status ddgs_render(const ddgs_gaussians *g, const ddgs_views *v,
                        const ddgs_config *cfg, ddgs_workspace *ws,
                        float *image, float *t_final, uint32_t *n_last,
                        void *stream);

/* Backward pass of ddgs_render (Sec. 3.1: the rasterisation is
 * differentiable; Sec. 4.3: back-propagation to the pose). Given dL/dC
 * ([n_views][height][width]) and the t_final / n_last of the forward call,
 * writes dL/d(every input) into the non-NULL fields of *out. The blending
 * state is recomputed from the sorted lists, walking each pixel back to front
 * (T_before = T_after / (1 - sigma)). Must follow the ddgs_render that filled
 * ws, with the same g, v and cfg (a different g->per_pixel is rejected). */
ddgs_status ddgs_render_backward(const ddgs_gaussians *g, const ddgs_views *v,
                                 const ddgs_config *cfg, ddgs_workspace *ws,
                                 const float *dL_dimage, const float *t_final,
                                 const uint32_t *n_last, const ddgs_grads *out,
                                 void *stream);

/* ddgs_render (Eq. 1 with Eq. 3) with no device allocation at all. (The
 * paper has no counterpart for the allocation rule: this serves callers that may not allocate device memory while
 * they run -- a registration loop whose memory is fixed at start-up, code
 * running inside another runtime's allocator, a process whose device memory a
 * caching allocator owns.) Same inputs, outputs and results as ddgs_render;
 * its scratch is one static device array of about 37 MiB that every GPU
 * loading this library holds until the process exits. Limits per call:
 * n_views * n <= 262144 records, n_views <= 1024, n_views * tiles per view
 * <= 65536 tiles and at most 1048576 (Gaussian, tile) pairs; larger renders return
 * DDGS_ERR_CAPACITY (the pair count is known only after the projection, so
 * that case returns after synchronising the stream, with the outputs left
 * unwritten). Calls no cudaMalloc, cudaFree or any other allocating routine.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture. The call synchronises the stream once to read the pair count.
 * Every call on a device shares the array and each clears what must start at
 * zero; calls whose GPU work overlaps (other streams or host threads) race.
 * g->per_pixel is not supported here (DDGS_ERR_INVALID_ARG). */
ddgs_status ddgs_render_static(const ddgs_gaussians *g, const ddgs_views *v,
                               const ddgs_config *cfg, float *image,
                               float *t_final, uint32_t *n_last, void *stream);

/* A batch of independent requests rendered by one sequence of launches: many
 * candidate poses of one patient, or many patients at once (Sec. 4.3's
 * registration renders many poses; a serving system renders many clouds).
 * Request r has its own cloud, its own bases and its own views; every view has
 * its own detector size. Device arrays are concatenated over the requests in
 * order; the counts and sizes are host arrays. */
typedef struct {
  int32_t n_requests;              /* R */
  const int64_t *gaussian_counts;  /* host [R]: N_r */
  const int64_t *iso_counts;       /* host [R]: the first iso_counts[r] of request r are isotropic */
  const int32_t *view_counts;      /* host [R]: V_r */
  const int32_t *heights, *widths; /* host [V], V = sum V_r: detector pixels of each view */
  const float *means;              /* [N][3], N = sum N_r, request order */
  const float *log_scales;         /* [N][3] */
  const float *quats;              /* [N][4] (w, x, y, z), 16-byte aligned */
  const float *opacity_logits;     /* [N] */
  const float *feat_iso;           /* [sum iso_counts][8], request order, 16-byte aligned */
  const void *feat_dir;            /* [N - sum iso_counts][8], float32 or bfloat16 */
  int32_t feat_dir_bf16;
  const float *b_iso;              /* [R][k] */
  const float *B_dir;              /* [R][k_L][k] */
  const float *world_to_cam;       /* [V][3][4], views in request order */
  const float *detector;           /* [V][5] */
  int32_t feat_dim;                /* k for every request, 1..32 (0 = 8) */
  int32_t sh_degree;               /* L for every request, 1..3 (0 = 1) */
  int32_t entangled, per_pixel;    /* Eq. 3 variants, as in ddgs_gaussians */
} ddgs_batch;

/* ddgs_render over a batch (same rule, Eq. 1 and Eq. 3, per view). Outputs are
 * concatenated per view: view v occupies H_v * W_v floats, row-major, after
 * the views before it. Each request's Gaussians are sorted and blended only
 * in its own views. */
ddgs_status ddgs_render_batched(const ddgs_batch *b, const ddgs_config *cfg,
                                ddgs_workspace *ws, float *image, float *t_final,
                                uint32_t *n_last, void *stream);

/* ddgs_render_backward over a batch: the gradients of Eq. 1 and Eq. 3
 * (Sec. 3.1's differentiable rasteriser; Sec. 4.3's gradient to the pose) for
 * every request. Gradient layouts follow the batch's
 * arrays: per-Gaussian fields [N][...], b_iso [R][k], B_dir [R][k_L][k],
 * world_to_cam [V][3][4]. Must follow the ddgs_render_batched that filled ws
 * with the same batch. */
ddgs_status ddgs_render_batched_backward(const ddgs_batch *b, const ddgs_config *cfg,
                                         ddgs_workspace *ws, const float *dL_dimage,
                                         const float *t_final, const uint32_t *n_last,
                                         const ddgs_grads *out, void *stream);

/* Per-view mean L1 loss of the registration objective (Sec. 4.3 compares the
 * rendering at a predicted pose with the target image; the l1 term of Eq. 2)
 * and its gradient. image [n_views][hw]; target [hw] (shared by all views)
 * or [n_views][hw] (target_per_view = 1). Writes loss [n_views] and
 * dL_dimage [n_views][hw] = sign(image - target) / hw. */
ddgs_status ddgs_l1_loss(const float *image, const float *target,
                         int32_t target_per_view, int32_t n_views, int64_t hw,
                         float *loss, float *dL_dimage, void *stream);

/* ---- initialisation: radiodensity-aware dual sampling (RADS, Sec. 3.3) ---- */

/* A CT volume: integer radiodensities (HU) on a regular grid. */
typedef struct {
  int32_t nx, ny, nz;   /* voxels along x (fastest), y, z; nx * ny * nz * 3 < 2^32 */
  const int16_t *hu;    /* device [nz][ny][nx], 16-byte aligned */
  float spacing[3];     /* voxel size along x, y, z (mm) */
  float origin[3];      /* world position of voxel (0, 0, 0)'s centre (mm) */
} ddgs_volume;

/* Initial point cloud of Sec. 3.3, with the sizes of Sec. 4.1 (n1 = 15000,
 * n2 = 10000):
 *   P^mc  marching-cubes points at the isolevel (min + max) / 2 of the volume:
 *         on every grid edge whose end voxels lie on opposite sides of it (a
 *         voxel is above when 2 HU > min + max), the point at the linear
 *         interpolation t = (level - HU_0) / (HU_1 - HU_0) along the edge.
 *         min(n1, crossings) of them are kept uniformly without replacement:
 *         edge e (= 3 * voxel + axis, voxel = (z ny + y) nx + x, axis 0/1/2 =
 *         +x/+y/+z neighbour) has the key (splitmix64(seed, e) >> 32) << 32 | e
 *         and the smallest keys win; kept points are written in edge order.
 *   P^dw  n2 voxel centres drawn independently with probability proportional
 *         to HU - min: draw j maps u = splitmix64(~seed, j) to the target
 *         floor(u * W / 2^64) (W the total weight) and takes the voxel whose
 *         cumulative-weight interval holds it. No draws if W = 0.
 * splitmix64(s, i) is output number i + 1 of SplitMix64 (Steele, Lea and
 * Flood 2014) seeded with s. Scales follow the 3D Gaussian splatting default:
 * log_s = log sqrt(max(mean squared distance to the 3 nearest other points,
 * 1e-7)), the same on the three axes.
 * Outputs (device, caller-owned, at least n1 + n2 rows): means [][3] (P^mc
 * kept, then P^dw in draw order, packed), log_scales [][3]; optional
 * kept_edges [n1] and draw_voxels [n2] (int64 edge ids / voxel indices, may
 * be NULL). counts (host [3]): points of P^mc kept, points of P^dw, crossings
 * found. The cloud has counts[0] + counts[1] points; Sec. 3.3 makes the first
 * counts[0] + counts[1] - counts[1] / 2 isotropic and the rest direction-
 * dependent. Synchronises the stream (to size the crossing list). */
ddgs_status ddgs_rads(const ddgs_volume *vol, int32_t n1, int32_t n2, uint64_t seed,
                      ddgs_workspace *ws, float *means, float *log_scales,
                      int64_t *kept_edges, int64_t *draw_voxels, int64_t *counts,
                      void *stream);

/* Number of (Gaussian, tile) pairs of the last render, read from the host
 * mirror written by that render (valid after the stream has synchronised;
 * infrastructure, no counterpart in the paper). */
ddgs_status ddgs_workspace_pairs(const ddgs_workspace *ws, int64_t *pairs);

/* Per-request timing of the last batched render + backward on this workspace
 * (measurement support, no counterpart in the paper). Synchronises the stream;
 * writes to host arrays of n_requests entries the nanoseconds (%globaltimer)
 * from the start of the render's first kernel to the end of the request's
 * last forward-raster tile (fwd_ns) and last backward-raster tile (bwd_ns);
 * 0 where that pass did not run. Either pointer may be NULL. */
ddgs_status ddgs_request_times(const ddgs_workspace *ws, uint64_t *fwd_ns, uint64_t *bwd_ns,
                               void *stream);

/* Copy the binning of the last render (the per-tile depth order of Eq. 1's
 * product, Sec. 3.1) into caller buffers (device):
 * tiles_touched [n_views][n], keys [pairs] ((global tile << 32) | depth bits,
 * global tile = view * tiles_per_view + row * tiles_x + col), vals [pairs]
 * (Gaussian index), ranges [n_views * tiles_per_view][2] ([start, end),
 * (0, 0) when empty). Any pointer may be NULL. */
ddgs_status ddgs_debug_binning(const ddgs_workspace *ws, uint32_t *tiles_touched,
                               uint64_t *keys, uint32_t *vals, uint32_t *ranges,
                               void *stream);

/* Synchronise the stream, then return and clear the status latched by
 * kernels since the last call: DDGS_OK; DDGS_ERR_CAPACITY when a no_sync
 * render had more pairs than the reserved capacity (the tile lists that did
 * not fit were left empty); else DDGS_ERR_NONFINITE when a render's inputs
 * held a NaN or infinite value not already reported by a synchronising
 * render. Infrastructure, no counterpart in the paper. */
ddgs_status ddgs_sync_status(ddgs_workspace *ws, void *stream);

/* Floats of a cloud: n * (3 + 4 + 3 + 1 + k) + k + k_L * k, i.e. 19 per
 * Gaussian and a 32-float shared basis at k = 8, L = 1 (Sec. 4.2). Host only. */
int64_t ddgs_parameter_count(int64_t n, int32_t k, int32_t L);

/* Human-readable name of a status; the last CUDA error string. Host only. */
const char *ddgs_status_string(ddgs_status s);
const char *ddgs_last_cuda_error(void);

/* 1 if a device of compute capability 10.3 is current and usable. Host only. */
int32_t ddgs_device_supported(void);

/* ---- tracing (no counterpart in the paper; measurement support) ----
 * Number of kernels this library has launched in this process. Host only. */
int64_t ddgs_kernel_launches(void);

/* When enabled, every kernel launch is bracketed by two CUDA events recorded
 * on the launch's own stream (not inside CUDA-graph capture). Host only. */
ddgs_status ddgs_profiler_enable(int32_t on);

/* Wait for the recorded events, then write per kernel id the summed device
 * time in milliseconds and the launch count (arrays of max_kernels entries,
 * host memory), set *n_kernels to the number of kernel ids, and reset. */
ddgs_status ddgs_profiler_collect(int32_t max_kernels, double *total_ms,
                                  int64_t *launches, int32_t *n_kernels);

/* Name of a kernel id reported by ddgs_profiler_collect ("" if out of range). */
const char *ddgs_profiler_kernel_name(int32_t id);

#ifdef __cplusplus
}
#endif
#endif /* DDGS_H */
