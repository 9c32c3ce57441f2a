/*
 * vgicp.h -- C ABI of the GB300 (sm_103a) VGICP factor-linearization library.
 *
 * The library computes, on one GPU, the voxelized-GICP matching cost factor of
 * arXiv 2202.00242 ("Globally Consistent and Tightly Coupled 3D LiDAR Inertial
 * Mapping"), Sec. III-A:
 *
 *   e^M = sum_{p_k in P_i} d_k^T (C'_k + R C_k R^T)^-1 d_k          (Eqs. 2-3)
 *   d_k = mu'_k - (R mu_k + t),
 *
 * where (mu'_k, C'_k) is the Gaussian of the voxel of the target map P_j that
 * contains T mu_k, and its linearization into a Hessian factor (Sec. III-A, last
 * paragraph: the factor is re-linearized at every optimizer iteration):
 *
 *   J_k = d d_k / d xi = [ R [mu_k]x , -R ]   for T <- T Exp(xi), xi = [omega; v]
 *   H = sum J_k^T W_k J_k,  b = sum J_k^T W_k d_k,  err = sum d_k^T W_k d_k,
 *   W_k = (C'_k + R C_k R^T)^-1 held at the linearization point,
 *   so err(xi) ~ err + 2 b^T xi + xi^T H xi and the Gauss-Newton step is -H^-1 b.
 *
 * Conventions shared by every entry point:
 *   - All functions return an int status (VGICP_OK or a negative code) and set a
 *     thread-local message readable with vgicp_last_error_string().
 *   - Pointers are DEVICE pointers unless the parameter is marked "host".
 *     The caller owns every input and output buffer; the library owns handles.
 *   - Every call takes a cudaStream_t and is asynchronous on it unless stated
 *     ("synchronizes").  Argument errors are reported synchronously.  Device-side
 *     build errors (key range, hash probe limit) are recorded in the map and read
 *     by vgicp_voxelmap_status(), which synchronizes the stream.
 *   - Point clouds are float32 AoS: points n x 3 (x, y, z), covariances n x 6
 *     upper triangles (xx, xy, xz, yy, yz, zz).  Both arrays must be 4-byte
 *     aligned; 16-byte alignment of the base is recommended.
 *   - Poses are host binary64 row-major 4x4 matrices T_target_source mapping
 *     source coordinates into the target frame.
 *   - A factor result is 43 doubles: H (36, row-major, symmetric), b (6), err (1).
 */
#ifndef VGICP_H
#define VGICP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same underlying type as cudaStream_t; 0 is the legacy default stream. */
typedef struct CUstream_st* vgicp_stream_t;

enum {
  VGICP_OK = 0,
  VGICP_ERR_INVALID_ARG = -1, /* bad pointer, size, option or pose */
  VGICP_ERR_OOM = -2,         /* device allocation failed */
  VGICP_ERR_HASH_FULL = -3,   /* a voxel could not be inserted within max_probe slots */
  VGICP_ERR_KEY_RANGE = -4,   /* |floor(x / r)| does not fit the 21-bit key field */
  VGICP_ERR_CUDA = -5         /* a CUDA runtime call failed (message has details) */
};

/* Message of the last failing call on this host thread ("" if none). */
const char* vgicp_last_error_string(void);

/* Library version, e.g. 10000 for 1.0.0. */
int vgicp_version(void);

/* Number of CUDA kernels this library has launched in the process so far
 * (all threads, all devices); for accounting in benchmarks. */
int64_t vgicp_launch_count(void);

/* Fault injection for tests of error handling (no counterpart in the paper):
 * the next `count` device allocations the library would make fail with
 * VGICP_ERR_OOM, without calling the allocator, exactly as a real out-of-memory
 * would; count = 0 cancels.  Applies to all threads and devices.  A negative
 * count is VGICP_ERR_INVALID_ARG. */
int vgicp_test_fail_allocations(int32_t count);

/* Fault injection for tests of the staged kernel's bounded waits (no
 * counterpart in the paper).  Arms the next launch of the staged kernel
 * (variant 2) only: in every CTA the producer withholds its tile number `tile`
 * (0-based; neither its copies nor its arrivals are issued), and every mbarrier
 * wait of that launch gives up after limit_ns (0 < limit_ns <= 2e9) instead of
 * 2 s.  The consumers' wait for the withheld tile then runs out, the launch
 * sets its status word (that call's outputs become NaN, inliers -1), each
 * producer waits for its copies in flight, and the kernel returns; the context
 * stays usable.  A CTA with fewer tiles withholds nothing. */
int vgicp_test_expire_waits(int32_t tile, int64_t limit_ns);

/* ------------------------------------------------------------------------ */
/* Voxel maps (Sec. III-A: the target cloud P_j is split into voxels, and each
 * voxel keeps one Gaussian formed from the means and covariances of the points
 * that fall inside it).
 *
 * Voxel key of a point x: k = floor((double)x / resolution) per axis, computed
 * exactly as in binary64 (a point on a face belongs to the voxel above it).
 * Each voxel stores N, mu' = (sum mu_p) / N and C' = (sum C_p) / N, the sums
 * taken in binary64 in ascending point index and rounded once to float32.
 * Voxels are numbered 0..V-1 in order of first appearance in the cloud.       */
/* ------------------------------------------------------------------------ */

typedef struct vgicp_map vgicp_map;

typedef struct {
  int32_t max_probe;       /* linear-probe limit of the hash table; 0 = 64 */
  int32_t capacity_factor; /* build-table capacity = next pow2 >= factor * n; 0 = 2 */
} vgicp_map_opts;

/* Build the voxel map of one target cloud.  points: n x 3, covs: n x 6 (device,
 * read during the call's kernels only; symmetric positive semi-definite, as the
 * regularised k-nearest-neighbour covariances are).  resolution > 0.  n >= 0 (an empty map
 * is valid).  *out receives a new handle.  The call synchronizes the stream once,
 * after counting the voxels, to size the lookup table (next pow2 >= max(16 V,
 * 2 n) slots of 64 B); the rest is asynchronous: check vgicp_voxelmap_status()
 * before relying on the contents. */
int vgicp_build_voxelmap(const float* points, const float* covs, int64_t n, double resolution,
                         const vgicp_map_opts* opts, vgicp_stream_t stream, vgicp_map** out);

/* Build n_maps voxel maps at once from concatenated clouds: map m is built from
 * rows offsets[m] .. offsets[m+1]-1 of points/covs.  offsets: host, n_maps + 1
 * non-decreasing entries starting at 0.  out: host array of n_maps handles.
 * The maps share one allocation (freed when the last handle is destroyed) and
 * one set of build kernels. */
int vgicp_build_voxelmaps(const float* points, const float* covs, const int64_t* offsets,
                          int32_t n_maps, double resolution, const vgicp_map_opts* opts,
                          vgicp_stream_t stream, vgicp_map** out);

/* Rebuild maps in place from new clouds of the same sizes.  maps must be all
 * handles of one vgicp_build_voxelmaps() call (or the single handle of
 * vgicp_build_voxelmap()), in their original order.  No allocation and no
 * synchronization: each lookup table keeps the region of the first build (at
 * least 2 n slots), so clouds with more voxels run at a higher load factor,
 * never above 1/2.  A rebuild empties only the table slots the previous build's
 * voxels occupy (recorded by that build), so successive builds of one batch
 * must be ordered: issue them on one stream, or synchronize between them. */
int vgicp_rebuild_voxelmaps(vgicp_map* const* maps, int32_t n_maps, const float* points,
                            const float* covs, vgicp_stream_t stream);

/* Release a handle (and the storage when it is the last handle of its batch).
 * The caller must ensure no queued kernel still reads the map. */
int vgicp_destroy_voxelmap(vgicp_map* map);

/* Synchronizes stream; returns the device-side build status of the map's batch
 * (VGICP_OK, VGICP_ERR_HASH_FULL or VGICP_ERR_KEY_RANGE). */
int vgicp_voxelmap_status(const vgicp_map* map, vgicp_stream_t stream);

/* Synchronizes stream.  num_voxels: V of this map; capacity: hash slots. */
int vgicp_voxelmap_info(const vgicp_map* map, vgicp_stream_t stream, int64_t* num_voxels,
                        int64_t* capacity);

/* Synchronizes stream.  Copies the voxels (first-appearance order) to host
 * arrays of at least max_voxels rows: keys V x 3 (int64), counts V (int32),
 * means V x 3 and covs V x 6 (float32).  Any output may be NULL. */
int vgicp_voxelmap_export(const vgicp_map* map, vgicp_stream_t stream, int64_t max_voxels,
                          int64_t* keys, int32_t* counts, float* means, float* covs);

/* Copies the map's voxel-grouped cloud (the cloud a map-as-source factor reads,
 * Sec. III-F): its n rows with the points of each voxel contiguous and in
 * ascending input index, the voxels in Morton order within chunks of the map's
 * voxels.  points: device n x 3, covs: device n x 6 (either may be NULL);
 * asynchronous on stream. */
int vgicp_voxelmap_grouped_cloud(const vgicp_map* map, vgicp_stream_t stream, float* points,
                                 float* covs);

/* ------------------------------------------------------------------------ */
/* Linearization (Eqs. 2-3 and the Hessian factor of Sec. III-A).             */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t neighbours; /* 1: the voxel containing T mu (the paper's lookup);
                         27: every occupied voxel of the 3x3x3 block around it,
                         one independent term each; 0 = 1 */
  int32_t tile;       /* source points per work item; 0 = automatic */
  int32_t grid;       /* CTAs of the persistent launch; 0 = automatic */
  int32_t variant;    /* 1-neighbour kernel: 0 = automatic, 1 = one point per thread,
                         2 = shared-memory staged (bulk asynchronous copies),
                         3 = per-warp hit compaction (terms evaluated in full
                             warps from a shared-memory queue); the debug outputs
                             corr_out / qkey_out always use kernel 1 */
  int32_t* corr_out;  /* optional device, n_src (single factor only): index of the
                         point's own voxel (first-appearance numbering) or -1 */
  int32_t* qkey_out;  /* optional device, n_src x 3 (single factor only): key of T mu */
  void* kernel_start; /* optional cudaEvent_t recorded on the stream just before the
                         linearize kernel is launched (for timing) */
  void* kernel_stop;  /* optional cudaEvent_t recorded just after it */
} vgicp_lin_opts;

/* Linearize one factor.  T_target_source: host, 16 doubles.  out: device, 43
 * doubles (H 36, b 6, err 1).  inliers: device, 1 int64 = number of source
 * points whose voxel is occupied (the overlap rate of Sec. III-D times n_src).
 * n_src = 0 gives zeros.  opts may be NULL. */
int vgicp_linearize(const vgicp_map* map, const float* src_points, const float* src_covs,
                    int64_t n_src, const double* T_target_source, double* out, int64_t* inliers,
                    const vgicp_lin_opts* opts, vgicp_stream_t stream);

/* vgicp_linearize without any device allocation (the paper has no counterpart:
 * this serves callers that may not allocate device memory once running, such as
 * a real-time loop whose GPU memory is fixed at start-up, or a plugin handed a
 * stream by a framework that forbids allocations on it).  Same arguments and
 * results as vgicp_linearize.  Its scratch (per-item partial sums and a status
 * word) is one fixed array in device memory that exists on every GPU that loads
 * the library, until the process exits, so no call allocates or frees.
 *   - Limit: at most 4096 work items per call, i.e. n_src <= 4096 * item size
 *     (automatic item size up to 16384 points: n_src up to 67,108,864); larger
 *     calls return VGICP_ERR_INVALID_ARG with a message and launch nothing.
 *   - The first call on a device looks up the array's device address (once per
 *     device, with that device current); make that first call before any
 *     stream capture.
 *   - All calls share the array and it keeps the last call's contents (the
 *     status word is cleared by each call).  Calls whose kernels overlap on the
 *     GPU (different streams without ordering, or concurrent host threads) race
 *     on it and give wrong results: serialize them, e.g. on one stream. */
int vgicp_linearize_noalloc(const vgicp_map* map, const float* src_points,
                            const float* src_covs, int64_t n_src, const double* T_target_source,
                            double* out, int64_t* inliers, const vgicp_lin_opts* opts,
                            vgicp_stream_t stream);

/* A source cloud for batched calls (device pointers), or a voxel map whose own
 * cloud is the source: when `map` is non-null, points/covs/n are ignored and the
 * map's cloud is read in the voxel-grouped order its build produced (points of
 * one voxel contiguous), which makes neighbouring source points look up
 * neighbouring target voxels.  The sum over points does not depend on the
 * order; the float32 rounding does, within the library's tolerance.  Results
 * are undefined if that map's build reported an error. */
typedef struct {
  const float* points; /* n x 3 */
  const float* covs;   /* n x 6 */
  int64_t n;
  const vgicp_map* map;
} vgicp_cloud;

/* Linearize n_pairs independent factors in one persistent launch (Sec. III-F:
 * a factor for every overlapping submap pair).  maps: host array of n_maps
 * handles; sources: host array of n_sources clouds; pairs: host n_pairs x 2
 * int32 (map index, source index); poses: host n_pairs x 16 doubles.  out:
 * device n_pairs x 43; inliers: device n_pairs.  Work is split into tiles of
 * opts->tile points so that uneven clouds balance across the GPU. */
int vgicp_linearize_batched(vgicp_map* const* maps, int32_t n_maps, const vgicp_cloud* sources,
                            int32_t n_sources, const int32_t* pairs, int64_t n_pairs,
                            const double* poses, double* out, int64_t* inliers,
                            const vgicp_lin_opts* opts, vgicp_stream_t stream);

/* Cost and gradient of n_pairs factors (same arguments as
 * vgicp_linearize_batched), for differentiable use of Eq. 2 with respect to
 * the right perturbation xi = [omega; v] of each pose:
 *   mode 1: err only;
 *   mode 2: gradient 2 J^T W d with W held at the pose (= 2 b, the
 *           Gauss-Newton gradient) and err;
 *   mode 3: the exact gradient, which adds for each omega_i the change of
 *           W = (C' + R C R^T)^-1 with the rotation, -u^T (dM/domega_i) u with
 *           u = W d, and err.
 * out: device n_pairs x 7 doubles (gradient 6, err 1); inliers as before.
 * Runs the one-point-per-thread kernel. */
int vgicp_evaluate_batched(vgicp_map* const* maps, int32_t n_maps, const vgicp_cloud* sources,
                           int32_t n_sources, const int32_t* pairs, int64_t n_pairs,
                           const double* poses, int32_t mode, double* out, int64_t* inliers,
                           const vgicp_lin_opts* opts, vgicp_stream_t stream);

/* The backward pass of the differentiable factor (Sec. III-A: the gradient of
 * Eq. 2 with respect to the pose increment): the gradient of each factor's err,
 * 2 J^T W d with W held (exact = 0, the Gauss-Newton gradient, twice the b of
 * vgicp_linearize), or the exact gradient (exact = 1).  vgicp_evaluate_batched
 * with mode 2 or 3; same arguments, out: device n_pairs x 7 (gradient 6, err 1).
 * For poses composed on the device and the incoming gradient applied there, see
 * vgicp_plan_evaluate. */
int vgicp_backward_batched(vgicp_map* const* maps, int32_t n_maps, const vgicp_cloud* sources,
                           int32_t n_sources, const int32_t* pairs, int64_t n_pairs,
                           const double* poses, int32_t exact, double* out, int64_t* inliers,
                           const vgicp_lin_opts* opts, vgicp_stream_t stream);

/* Host binary64 pose algebra for optimizers (no device work; never fails on
 * finite input except solve6 on a non positive definite system).
 *   vgicp_se3_exp: T (row-major 4x4) = Exp(xi), xi = [omega; v].
 *   vgicp_se3_right_jacobian: J (row-major 6x6) with
 *     Exp(xi + d) = Exp(xi) Exp(J d) + O(|d|^2).
 *   vgicp_pose_mul: C = A B (4x4, C may alias A or B).
 *   vgicp_solve6: xi = -(H + lambda diag(H))^-1 b by Cholesky (lambda >= 0;
 *     0 gives the Gauss-Newton step of err ~ err + 2 b^T xi + xi^T H xi). */
int vgicp_se3_exp(const double* xi, double* T);
int vgicp_se3_right_jacobian(const double* xi, double* J);
int vgicp_pose_mul(const double* A, const double* B, double* C);
int vgicp_solve6(const double* H, const double* b, double lambda, double* xi);

/* Binary form of a matching-cost factor, which constrains the two poses T_i
 * (source) and T_j (target) (Sec. III-A).  Input: the factor's H (6x6), b (6)
 * in the right perturbation xi of T = T_j^-1 T_i (as vgicp_linearize returns them)
 * and T (4x4).  With right perturbations of the world poses, T_i <- T_i Exp(d_i)
 * and T_j <- T_j Exp(d_j), xi = d_i - Ad(T^-1) d_j to first order, so over
 * [d_i; d_j]: H2 = A^T H A (12x12) and b2 = A^T b (12) with A = [I, -Ad(T^-1)]
 * (Ad of [omega; v] twists).  All host binary64, row-major. */
int vgicp_binary_factor(const double* H, const double* b, const double* T, double* H2,
                        double* b2);

/* Overlap rate (Sec. III-D: the fraction of a frame's points that fall within a
 * voxel of the other frame; keyframes, submaps and global factors are created
 * from it, Sec. III-D to III-F).  For each pair, inliers[p] (device, n_pairs) =
 * the number of source points whose transformed voxel is occupied in the target
 * map; the rate is inliers[p] / n_src.  Same factor description as
 * vgicp_linearize_batched; lookups only (the source covariances are not read).
 * opts: tile, grid; neighbours must be 0 or 1.  A nonzero device status gives
 * inliers = -1. */
int vgicp_overlap_batched(vgicp_map* const* maps, int32_t n_maps, const vgicp_cloud* sources,
                          int32_t n_sources, const int32_t* pairs, int64_t n_pairs,
                          const double* poses, int64_t* inliers, const vgicp_lin_opts* opts,
                          vgicp_stream_t stream);

/* Point covariances from the k nearest neighbours (Sec. III-C: each point is a
 * Gaussian whose covariance comes from its neighbouring points), regularised as
 * in GICP: the sample covariance of the k neighbours (the point itself
 * included, ties broken by lower index, squared distances formed in binary64)
 * has its eigenvalues, in decreasing order, replaced by (1, 1, eps).
 * points: device, the concatenated clouds (offsets: host, n_clouds + 1, from 0,
 * non-decreasing); neighbours are searched within each cloud.  k in [1, 32];
 * eps in (0, 1]; cell: grid cell size of the search (0 = per cloud from its
 * bounding box).  covs_out: device n x 6 (xx xy xz yy yz zz).  nbr_out: optional
 * device n x k int32, the neighbours in (distance, index) order as cloud-local
 * indices, -1 past the cloud's size.  Allocates scratch on the stream and
 * synchronizes it (to report VGICP_ERR_KEY_RANGE / VGICP_ERR_HASH_FULL). */
int vgicp_estimate_covariances(const float* points, const int64_t* offsets, int32_t n_clouds,
                               int32_t k, double eps, double cell, int32_t* nbr_out,
                               float* covs_out, vgicp_stream_t stream);

/* Voxel-grid downsampling with timestamp averaging (Sec. III-C: the input
 * clouds are downsampled by a voxel grid whose voxels average the timestamps
 * of their points as well as their positions; a point whose time lies far from
 * its voxel's goes to another, new voxel so the first and last points of a scan
 * are not fused).  Reading: a point's voxel is floor(p / resolution); the voxel's
 * reference time is that of its first point (index order); a point whose time
 * differs from it by more than `split` (e.g. a tenth of the scan duration)
 * belongs to the voxel's second output voxel.  Output voxels are numbered in
 * order of first appearance, cloud by cloud; each is the mean of its points'
 * positions and times (binary64 mean rounded to float32).
 * points: device n x 3; times: device n or NULL (no split, no times out);
 * offsets: host n_clouds + 1 (from 0, non-decreasing).  out_points: device,
 * room for n x 3; out_times: device n or NULL; out_counts: device n or NULL
 * (points per output voxel); out_offsets: host n_clouds + 1 (cloud c's output
 * voxels are out_offsets[c] .. out_offsets[c + 1] - 1).  Allocates scratch on
 * the stream and synchronizes it. */
int vgicp_downsample(const float* points, const float* times, const int64_t* offsets,
                     int32_t n_clouds, double resolution, double split, float* out_points,
                     float* out_times, int32_t* out_counts, int64_t* out_offsets,
                     vgicp_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Admission: factor sets larger than device memory (host-only planning).      */
/* ------------------------------------------------------------------------ */

/* Upper bound of the device bytes a voxel map of n_points occupies (all its
 * buffers; the lookup table counted at V = n), for admission budgets. */
int64_t vgicp_voxelmap_bytes(int64_t n_points, const vgicp_map_opts* opts);

/* Assigns every pair to a batch whose working set (its target maps and source
 * clouds, counted once each) fits in budget bytes.  Greedy over the pairs in
 * (target, source) order, which keeps the pairs of one target together.
 * map_bytes: host n_maps; src_bytes: host n_sources, or ignored when
 * src_is_map != 0 (each source is the map of the same index, counted once).
 * batch_of_pair: host n_pairs output; *n_batches: output.  A pair whose own
 * working set exceeds the budget is an error. */
int vgicp_admission_schedule(const int64_t* map_bytes, int32_t n_maps, const int64_t* src_bytes,
                             int32_t n_sources, const int32_t* pairs, int64_t n_pairs,
                             int64_t budget, int32_t src_is_map, int32_t* batch_of_pair,
                             int32_t* n_batches);

/* ------------------------------------------------------------------------ */
/* Plans: a fixed factor set linearized at every optimizer iteration          */
/* (Sec. III-A re-linearizes each factor per iteration; Sec. III-F links every */
/* overlapping submap pair).  The work list is built once, the launch shape   */
/* can be chosen by timing candidates (autotune), and one linearization is    */
/* captured in a CUDA graph replayed with new poses.                          */
/* ------------------------------------------------------------------------ */

typedef struct vgicp_plan vgicp_plan;

/* Same factor description as vgicp_linearize_batched (maps, sources, pairs are
 * host arrays; sources may reference maps).  opts: neighbours, tile (points
 * per work item, 0 = default 16384, else >= 2048), variant, grid.  Allocates
 * the plan's device and pinned host buffers.  The maps and source clouds must
 * outlive the plan. */
int vgicp_plan_create(vgicp_map* const* maps, int32_t n_maps, const vgicp_cloud* sources,
                      int32_t n_sources, const int32_t* pairs, int64_t n_pairs,
                      const vgicp_lin_opts* opts, vgicp_stream_t stream, vgicp_plan** out);

/* Synchronizes.  Times each kernel variant (1-neighbour: 1, 2, 3) with work items
 * of 4096, 8192, 16384 and 32768 points on these poses (host, n_pairs x 16) and
 * keeps the fastest; results then depend (within float32 rounding) on that
 * choice, and are deterministic for it. */
int vgicp_plan_autotune(vgicp_plan* plan, const double* poses, vgicp_stream_t stream);

/* Linearize all factors at poses (host, n_pairs x 16 doubles, read during the
 * call).  out: device n_pairs x 43, inliers: device n_pairs (either may be NULL;
 * results are copied there after the graph).  kernel_start/kernel_stop:
 * optional cudaEvent_t recorded on the stream around the graph launch (status
 * reset, linearize kernel, per-pair reduction).  The first call captures the
 * graph. */
int vgicp_plan_execute(vgicp_plan* plan, const double* poses, double* out, int64_t* inliers,
                       void* kernel_start, void* kernel_stop, vgicp_stream_t stream);

/* Differentiable evaluation (Sec. III-A: the matching cost as a function of the
 * pose, differentiated for a gradient-based optimizer).  Every factor p is
 * evaluated at T_p = T0_p Exp(xi_p), composed on the device in binary64, with
 * the one-point-per-thread kernel and the plan's work list; nothing is copied
 * to or from the host and the call does not synchronize.
 *   base_poses: device, n_pairs x 16 doubles (row-major T0_p, finite rigid).
 *   xi:         device, n_pairs x 6 doubles ([omega; v]), or NULL for xi = 0.
 *   mode 1: err only; 2: gradient with W held, 2 J^T W d; 3: exact gradient
 *           (adds the change of W with the rotation); see vgicp_evaluate_batched.
 *   grad_scale: device, n_pairs doubles, or NULL (= 1): the gradient of factor p
 *           is multiplied by grad_scale[p] (the incoming gradient of a
 *           reverse-mode pass).
 *   out: device, n_pairs x 7 doubles: [0..5] the gradient with respect to xi_p,
 *        J_r(xi_p)^T g (modes 2, 3; g when xi is NULL), times grad_scale; [6] err.
 *   inliers: device n_pairs, or NULL.
 * A base pose that is not a finite rigid transform, or a non-finite xi, makes
 * every output of the call NaN (inliers -1).  Calls on one plan, including
 * vgicp_plan_execute, must be ordered on one stream: they share the plan's
 * pose descriptors. */
int vgicp_plan_evaluate(vgicp_plan* plan, const double* base_poses, const double* xi,
                        int32_t mode, const double* grad_scale, double* out, int64_t* inliers,
                        vgicp_stream_t stream);

/* Current launch shape: kernel variant, points per work item, CTAs, work items. */
int vgicp_plan_info(const vgicp_plan* plan, int32_t* variant, int32_t* item_points,
                    int32_t* grid, int64_t* n_items);

/* Waits for the device to finish using the plan, then releases it. */
int vgicp_plan_destroy(vgicp_plan* plan);

#ifdef __cplusplus
}
#endif

#endif /* VGICP_H */
