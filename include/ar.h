/*
 * ar.h -- C ABI of the GB300 abstract-rendering library (libar).
 *
 * Abstract rendering of Gaussian-splat scenes (Li, Ji, Zhong, Zhang, Mitra,
 * arXiv 2503.00308): for a scene, a nominal camera and a box of camera poses
 * split into cells, compute for every cell and pixel a lower and an upper RGB
 * bound that contain the colour GSplat (Algorithm 1) renders at EVERY pose of
 * the cell -- the abstract rendering problem stated at the end of Sec. 2.2 --
 * by the AbstractSplat construction of Sec. 3.3: linear bounds over the pose
 * variables pushed through Algorithm 1, MatrixInv (Algorithm 3) for the conic,
 * and BlendInd (Algorithm 4) for the blend.
 *
 * Conventions shared by every entry point
 *   - Status: every call returns AR_OK (0) or one of the AR_E* codes below and
 *     never throws across the boundary; ar_last_error() gives the message of
 *     the calling thread's last failure.
 *   - Camera frame: OpenCV (x right, y down, z forward).  A nominal pose is a
 *     world->camera rotation R_wc (row-major 3x3) and the camera centre t in
 *     world coordinates, so a world point X maps to R_wc (X - t).
 *   - Pose cells: a box over delta = (tx, ty, tz, rx, ry, rz).  (tx, ty, tz) is
 *     a world-frame offset of the camera centre (metres); (rx, ry, rz) are XYZ
 *     Euler angles (radians) of a rotation R_d = Rx(rx) Ry(ry) Rz(rz) applied in
 *     the camera frame, so the perturbed camera has R_wc' = R_d^T R_wc and
 *     t' = t + (tx, ty, tz).  lo[k] <= hi[k]; lo == hi (a point) is legal.
 *   - Pixels: centre of pixel (px, py) is (px + 0.5, py + 0.5); outputs are
 *     row-major [n_cells][height][width][3] float32 in [0, 1].
 *   - Rendering semantics bounded (Algorithm 1 with the usual splatting
 *     conventions that the paper leaves open): Gaussians with depth <= near_plane
 *     are dropped, effective opacities below 1/255 are zero, the background is
 *     black, colours are degree-0 RGB, the blend is BlendInd/BlendSort.
 *   - Soundness: for every pose in cell c, pixel p and channel k,
 *       out_lower[c][p][k] <= GSplat(scene, pose, p)[k] <= out_upper[c][p][k].
 *   - Streams: `cuda_stream` is a cudaStream_t (NULL = legacy default stream).
 *     Device outputs are written asynchronously on that stream.
 *   - Threads: one ar_scene must not be used by two threads at the same time.
 */
#ifndef AR_H
#define AR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AR_OK 0
#define AR_EINVAL 1    /* bad argument: null pointer, size, NaN, lo > hi, ... */
#define AR_ENOMEM 2    /* device or host allocation failed / over the budget */
#define AR_EAGAIN 3    /* serving: request queue full, try again */
#define AR_ETIMEOUT 4  /* serving: a bounded wait ran out */
#define AR_EDEVICE 5   /* CUDA error (message from the runtime) */
#define AR_ECANCELED 6 /* serving: the request was cancelled */

typedef struct ar_intrinsics {
    int32_t width, height;      /* image size in pixels, 1..16384 each */
    float fx, fy, cx, cy;       /* pinhole K = [[fx, 0, cx], [0, fy, cy]] (Sec. 2.2) */
    float near_plane;           /* depth below which Gaussians are dropped, > 0 */
} ar_intrinsics;

typedef struct ar_nominal_pose {
    double R_wc[9];             /* world -> camera rotation, row-major */
    double t[3];                /* camera centre, world frame */
} ar_nominal_pose;

typedef struct ar_pose_box {
    double lo[6], hi[6];        /* bounds of (tx, ty, tz, rx, ry, rz) */
} ar_pose_box;

typedef struct ar_scene ar_scene;
typedef struct ar_server ar_server;

/* Per-render counters and stage times (ms; timed with CUDA events on the
 * render stream when profiling is on, else -1). */
typedef struct ar_render_stats {
    int64_t n_records;          /* (Gaussian, cell) pairs that reach the image */
    int64_t n_entries;          /* (Gaussian, cell, tile) bin entries (2 events each) */
    int64_t n_triples;          /* (pixel, Gaussian, cell) triples inside a screen box */
    int64_t n_fallback;         /* (Gaussian, cell) pairs where MatrixInv's assertion failed
                                   even on the split pieces of the cell, so that the opacity is
                                   bounded by [0, o] (among the pairs whose records were built) */
    int32_t n_launches;         /* kernels launched by the render */
    int32_t tile;               /* tile edge used (pixels) */
    int32_t m_vars;             /* pose variables carried by the linear forms */
    float ms_prep, ms_bin, ms_render, ms_total;
    int64_t n_evaluated;        /* per-pixel opacity relaxations evaluated (triples the sweep
                                   reached before each pixel's bounds were settled; MatrixInv
                                   fallbacks, which are constant, are not counted) */
    int64_t n_reevaluated;      /* evaluations repeated at an upper depth endpoint because the
                                   lower endpoint's result had left the per-pixel ring */
    int64_t n_built;            /* pairs whose record value part (the per-pixel forms, MatrixInv
                                   included) was built: the FP32 renderer builds only the pairs
                                   its tiles can reach before their pixels stop */
    int64_t n_restarted;        /* (cell, tile) sweeps abandoned because they reached entries
                                   beyond their window of built records, then swept again */
    float ms_build;             /* record value parts built on demand (included in neither
                                   ms_prep nor ms_render; ms_render is the per-pixel sweep) */
    int64_t n_split;            /* (Gaussian, cell) pairs whose MatrixInv held only after the
                                   cell was split into pieces (Sec. 3.1, adjustment (2); among
                                   the pairs whose records were built) */
    int64_t n_fp64;             /* opacity evaluations taken again in FP64 because their m
                                   interval was too wide for FP32 (ar_scene_set_fp64_alpha) */
    int64_t n_fp64_segments;    /* (cell, tile) sweeps that met such an evaluation and were
                                   swept again by the FP64-capable instance of the renderer */
    int64_t n_graph_replays;    /* cell batches whose binning and render were replayed from a
                                   captured CUDA graph (ar_scene_set_graphs) */
    int32_t chunk;              /* events per staged chunk of the per-pixel sweep (autotuned
                                   with tile = 0, else 16) */
} ar_render_stats;

/* Create a scene from n Gaussians <uw, Mw, o, c> (Sec. 2.2).  Mw is given by
 * a per-axis log-scale and a rotation quaternion (w, x, y, z): Mw = R(q)
 * diag(exp(logscale)), any square-root factor of the covariance being
 * allowed by the footnote of Sec. 2.2.
 *   uw3[n][3], logscale3[n][3], quat4[n][4], opacity[n] in [0, 1), rgb3[n][3]
 *   in [0, 1]: float32, row-major.  device_ptrs = 0: host arrays; 1: device
 *   arrays on the current device.  The arrays are copied; the caller keeps
 *   ownership.  n = 0 is legal (renders black).  The scene lives on the
 *   current CUDA device and owns its device memory until ar_scene_destroy.
 * Errors: AR_EINVAL (null pointers with n > 0, n < 0, non-finite values,
 * opacity outside [0, 1), colour outside [0, 1], zero quaternion),
 * AR_ENOMEM, AR_EDEVICE. */
int ar_scene_create(const float *uw3, const float *logscale3, const float *quat4,
                    const float *opacity, const float *rgb3, int64_t n, int device_ptrs,
                    ar_scene **out);

/* Release a scene and all its device memory (synchronises the device). */
int ar_scene_destroy(ar_scene *scene);

/* Abstract-render n_cells pose cells (AbstractSplat, Sec. 3.3, with the input
 * partitioning of Sec. 4.2 batched into one call): per cell, per pixel, RGB
 * lower and upper bounds.
 *   cells[n_cells] (host memory), n_cells >= 1.
 *   tile: 0 = choose, else 8 or 16 (screen tile edge of the binning; the
 *   bounds do not depend on it beyond 2e-5: a pixel stops sweeping once what
 *   is left of its tile's list can move its bounds by less than 1e-5, and
 *   widens them by that much).  With 0, the first call for a given image
 *   size and number of pose variables times the pipeline on its first eight
 *   cells for each (tile edge, events per staged chunk of the sweep) of
 *   (16, 16), (16, 8), (16, 32), (8, 16) and keeps the fastest for the scene
 *   (autotuner; ar_render_stats.tile and .chunk report the choice).  An
 *   explicit tile sweeps in chunks of 16.
 *   out_lower, out_upper: device pointers, float32 [n_cells][H][W][3] each,
 *   owned by the caller.
 * Work is enqueued on cuda_stream; the call returns after the last launch is
 * enqueued (it synchronises once with the stream to size the tile bins).
 * Errors: AR_EINVAL (null pointers, bad intrinsics or cells, tile not in
 * {0, 8, 16}), AR_ENOMEM (workspace), AR_EDEVICE. */
int ar_render_abstract(ar_scene *scene, const ar_intrinsics *intr, const ar_nominal_pose *pose,
                       const ar_pose_box *cells, int32_t n_cells, int32_t tile,
                       float *out_lower, float *out_upper, void *cuda_stream);

/* Same as ar_render_abstract with HOST output buffers host_lower /
 * host_upper ([n_cells][H][W][3] float32 each).  When both are page-locked
 * host memory mapped into the device (cudaHostAlloc, or cudaHostRegister on a
 * unified-addressing system), the render kernel stores the bounds into them
 * directly, so the device-to-host transfer overlaps the render.  Any other
 * host memory gets the bounds computed into scene-owned device memory and
 * copied after the render.  The results are identical either way.  Returns
 * after the bounds are in host memory; on an error the buffers' contents are
 * undefined. */
int ar_render_abstract_host(ar_scene *scene, const ar_intrinsics *intr, const ar_nominal_pose *pose,
                            const ar_pose_box *cells, int32_t n_cells, int32_t tile,
                            float *host_lower, float *host_upper, void *cuda_stream);

/* ar_render_abstract without any allocation.  The paper has no counterpart:
 * this entry point exists for callers that may not allocate memory while
 * they run (a real-time loop or embedded verifier that fixes its memory up
 * front, or a host under a strict GPU memory budget where cudaMalloc would
 * stall or fail).  It computes the same bounds with the same kernels, but
 * places every per-call buffer in one 64 MiB array compiled into libar
 * instead of growing the scene's workspace, and calls neither cudaMalloc,
 * cudaFree nor any other allocating routine.
 *   - Every GPU that loads libar holds the 64 MiB array until the process
 *     exits.  Requests whose buffers need more (roughly: many cells x
 *     Gaussians, or many tile entries) fail with AR_ENOMEM and a message
 *     naming the limit; the outputs are then left untouched.
 *   - Each call looks up the array's device address on the scene's device;
 *     the first call on a device may load the library's device code there
 *     (the one-time set-up), so make that first call before any stream
 *     capture.
 *   - tile = 0 takes the tile edge and sweep chunk the scene's autotuner
 *     chose for this image size and number of pose variables in an earlier
 *     ar_render_abstract call, else 16 and 16; this entry point does not time
 *     candidates itself.  With the same tile argument, after the same tuning,
 *     the bounds are bit-identical to ar_render_abstract's.
 *   - All calls share the array and it keeps the last call's contents: two
 *     calls that overlap on the GPU (different streams or threads without
 *     ordering) race and corrupt each other's results.  Serialise them.
 *   - The call synchronises once with cuda_stream (to read two counters),
 *     like ar_render_abstract.
 * Arguments, output layout and other errors as for ar_render_abstract. */
int ar_render_abstract_noalloc(ar_scene *scene, const ar_intrinsics *intr, const ar_nominal_pose *pose,
                               const ar_pose_box *cells, int32_t n_cells, int32_t tile,
                               float *out_lower, float *out_upper, void *cuda_stream);

/* Union of the bounds of several pose cells (Sec. 5: the bounds of a camera
 * set partitioned into subsets are the subsets' bounds, joined).
 *   in_lower, in_upper: DEVICE [n_cells][height][width][3] float32, as
 *     ar_render_abstract writes them.
 *   out_lower, out_upper: DEVICE [height][width][3] float32; out_lower gets
 *     the elementwise minimum of in_lower over the cells, out_upper the
 *     maximum of in_upper.  The outputs must not overlap the inputs or each
 *     other.
 * Enqueued on cuda_stream (no synchronisation).  One kernel launch, bound by
 * HBM bandwidth.  Errors: AR_EINVAL (null pointers, n_cells < 1, sizes out of
 * range, overlapping buffers), AR_EDEVICE. */
int ar_bounds_union(const float *in_lower, const float *in_upper, int32_t n_cells, int32_t width, int32_t height,
                    float *out_lower, float *out_upper, void *cuda_stream);

/* Bounds of one pose box over all its poses, from a partition of the box
 * (Sec. 5): the box is cut into parts[k] equal pieces along pose dimension k
 * (dimension 0 varying fastest), the pieces are rendered as cells, in chunks
 * of at most 64, and their bounds are joined as by ar_bounds_union.  Finer
 * partitions give tighter bounds (Sec. 5) at proportional cost.
 *   box: one pose box (the checks of ar_render_abstract's cells apply).
 *   parts: 6 entries >= 1 whose product is at most 2^24; a dimension with
 *     lo = hi takes 1.
 *   out_lower, out_upper: DEVICE [height][width][3] float32.
 * Piece k of n along a dimension is [lo + w k / n, lo + w (k + 1) / n], with
 * w = hi - lo, and the last piece ends at hi exactly, so the pieces cover the
 * box.  The scene's blend mode applies.  Chunk buffers come from the scene's
 * workspace.  Synchronises with cuda_stream once per chunk (as
 * ar_render_abstract does); the stats of ar_last_render_stats describe the
 * last chunk.  Errors as for ar_render_abstract, and AR_EINVAL for bad parts;
 * after an error the outputs' contents are undefined. */
int ar_render_abstract_partitioned(ar_scene *scene, const ar_intrinsics *intr, const ar_nominal_pose *pose,
                                   const ar_pose_box *box, const int32_t *parts, int32_t tile, float *out_lower,
                                   float *out_upper, void *cuda_stream);

/* Piece `index` of the partition used by ar_render_abstract_partitioned
 * (dimension 0 varying fastest), written to *out.  Host only: no CUDA call.
 * Errors: AR_EINVAL (null pointers, parts < 1 or more than 2^24 pieces,
 * index outside [0, prod parts)). */
int ar_partition_piece(const ar_pose_box *box, const int32_t *parts, int64_t index, ar_pose_box *out);

/* Bounds of one pose box from an adaptive partition (Sec. 5 partitions the
 * camera set to tighten the bounds; here the pieces whose bounds stay loose
 * are the ones cut further).  Round 0 renders the box.  Each of the next
 * `rounds` rounds cuts the looser half of the current pieces, ranked by the
 * mean width of their bounds (sum over pixels and channels of upper - lower,
 * ties by index), each into two halves along the pose dimension where the
 * piece is widest relative to the box, and renders the new set of pieces.
 * The outputs are the intersection over the rounds of each round's union of
 * its pieces' bounds: sound, because every round's union bounds every pose of
 * the box, and never looser than the box's own bounds.
 *   box: one pose box (the checks of ar_render_abstract's cells apply).
 *   rounds: 0..12.  Pieces per round: 1, 2, 3, 5, 8, 12, ... (n + ceil(n/2)).
 *   out_lower, out_upper: DEVICE [height][width][3] float32.
 *   leaves (optional, host, leaves_cap entries): the last round's pieces, in
 *     order; n_leaves (optional) gets their number.
 * Rendering goes through ar_render_abstract in chunks of at most 64 pieces;
 * the scene's blend mode applies.  Synchronises with cuda_stream once per
 * chunk.  Errors as for ar_render_abstract, and AR_EINVAL for bad rounds or
 * leaves arguments; after an error the outputs' contents are undefined. */
int ar_render_abstract_refined(ar_scene *scene, const ar_intrinsics *intr, const ar_nominal_pose *pose,
                               const ar_pose_box *box, int32_t rounds, int32_t tile, float *out_lower,
                               float *out_upper, ar_pose_box *leaves, int32_t leaves_cap, int32_t *n_leaves,
                               void *cuda_stream);

/* Plain comparison path: the same bounds computed one cell per launch
 * sequence in FP64 with directed rounding, without cell batching.  Same
 * arguments and output layout as ar_render_abstract. */
int ar_render_abstract_plain_fp64(ar_scene *scene, const ar_intrinsics *intr,
                                  const ar_nominal_pose *pose, const ar_pose_box *cells,
                                  int32_t n_cells, int32_t tile, float *out_lower,
                                  float *out_upper, void *cuda_stream);

/* Concrete GSplat render (Algorithm 1, blended as BlendInd, Algorithm 4:
 * Gaussians of equal depth do not occlude each other) at n_poses poses, for
 * checking the abstract bounds on the device.  deltas: host, [n_poses][6]
 * (tx, ty, tz, rx, ry, rz) relative to the nominal pose, as in ar_pose_box;
 * out: device, [n_poses][H][W][3] float32, each value the FP64 colour
 * clipped to [0, 1] and rounded to nearest.  Computed in FP64 with the same
 * 1/255 cutoff, near plane and frustum guard band as the abstract render;
 * a pixel stops once its transmittance is below 1e-13 (the colour left out
 * is below that).  One pose per pipeline pass (projection, binning, blend);
 * uses the scene's workspace, so it must not overlap a render of the same
 * scene.  AR_EINVAL for bad arguments or non-finite deltas. */
int ar_render_concrete(ar_scene *scene, const ar_intrinsics *intr, const ar_nominal_pose *pose,
                       const double *deltas, int32_t n_poses, float *out, void *cuda_stream);

/* Scene-parameter boxes (Sec. 4.5, abstract rendering of sets of scenes):
 * per Gaussian, an interval for its mean (uw_lo3/uw_hi3, [n][3], world
 * frame), its opacity (opacity_lo/hi, [n], 0 <= lo <= hi < 1) and its colour
 * (rgb_lo3/rgb_hi3, [n][3], 0 <= lo <= hi <= 1).  Host arrays, copied.  A
 * NULL pair keeps that parameter at the scene's nominal value (all NULL:
 * back to the nominal scene).  The boxes need not contain the nominal values.
 * Later abstract renders bound GSplat over every pose of each cell and every
 * scene whose Gaussians take any parameters in their boxes, independently of
 * one another.  The mean's box enters the projection as an interval; the
 * opacity box as o_lo in the lower opacity forms and cutoff and o_hi in the
 * upper ones; the colour box as c_lo in the lower colour sum and c_hi in the
 * upper one.  (ar_render_concrete keeps rendering the nominal scene.)
 * Synchronous; must not overlap a render of the scene.  AR_EINVAL for a half
 * given pair, a non-finite value or lo > hi. */
int ar_scene_set_boxes(ar_scene *scene, const float *uw_lo3, const float *uw_hi3, const float *opacity_lo,
                       const float *opacity_hi, const float *rgb_lo3, const float *rgb_hi3);

/* Test and diagnosis hook: the decision part of every (Gaussian, cell)
 * record of one pose cell, as the batched renderer computes it (Algorithm 1
 * lines 2-7 with set-valued variables: depth, near-plane class, depth key,
 * pixel box; the frustum guard band).  out: host, [n][10] doubles per
 * Gaussian: valid, straddle, k_lo, k_hi, px0, px1, py0, py1, mu_x, mu_y
 * (all 0 where the pair reaches no pixel; mu is the pixel centre the pixel
 * stage expands around).  The decisions are taken in FP64 in the order of the
 * oracle's steps, so they are bit-identical to a plain FP64 implementation.
 * Synchronous (default stream); uses the scene's workspace, so it must not
 * overlap a render of the same scene.  AR_EINVAL for bad arguments.  (out =
 * NULL only leaves the records of the cell in the scene's workspace.) */
int ar_debug_records(ar_scene *scene, const ar_intrinsics *intr, const ar_nominal_pose *pose,
                     const ar_pose_box *cell, double *out);

/* Test and diagnosis hook: the per-pixel effective-opacity relaxation
 * (Algorithm 1 lines 9-10 relaxed, Table 2's Exp) of n (Gaussian, pixel)
 * pairs of one pose cell, as the batched renderer evaluates them: the record
 * of Gaussian gi[t] on the cell is built as the renderer builds it, then
 * evaluated at pixel (px[t], py[t]) in FP32 (precision 0), in FP32 and again
 * in FP64 where the FP32 deviation estimate alone exceeds the scene's
 * ar_scene_set_fp64_alpha threshold (precision 1; the renderer also weights it
 * by the pixel's transmittance), or always in FP64 as well (precision 2).
 * Precision 3 is precision 0 with the chain to the Mahalanobis term taken by
 * scalar directed-rounding steps in place of the renderer's packed (-lo, hi)
 * pairs: the outputs are the same bit for bit, which a test checks.
 * out: host, [n][40] doubles per pair: the lower opacity form (coefficients of
 * the 6 pose dimensions tx..rz over the cell normalised to [-1, 1], then the
 * constant), the upper form (7), the radii bounding the sums of the
 * coefficients' magnitudes of the two forms, a_lo, a_hi, the FP32 deviation
 * estimate, m_lo, m_hi, the record's W entries as 6 (lo, hi) intervals, its
 * S, R_x, R_y as (lo, hi), and flags (1 valid, 2 FP64 taken, 4 MatrixInv
 * fallback); all 0 where the Gaussian reaches no pixel on the cell.
 * Synchronous; uses the scene's workspace and allocates a few small device
 * buffers.  AR_EINVAL for bad arguments or a pair out of range. */
int ar_debug_alpha(ar_scene *scene, const ar_intrinsics *intr, const ar_nominal_pose *pose,
                   const ar_pose_box *cell, int32_t n, const int64_t *gi, const int32_t *px, const int32_t *py,
                   int32_t precision, double *out);

/* Test hook: the events per staged chunk (8, 16 or 32) of the FP32 sweep at
 * tile 16 for the scene's renders with an explicit tile (0: back to 16), so
 * that the autotuner's other candidates can be checked for parity.
 * AR_EINVAL for a null scene or another value. */
int ar_debug_set_chunk(ar_scene *scene, int32_t chunk);

/* Test hook: a cell batch whose (Gaussian, cell, tile) entries reach `cap`
 * is split into two halves and rendered again (the bins index entries with
 * 32 bits, so the library's own cap is 2^32 - 2^20, which cap = 0 restores);
 * a lower cap exercises the split.  The bounds do not change.  AR_EINVAL for
 * a null scene or a cap outside [0, 2^32 - 2^20]. */
int ar_debug_set_entry_cap(ar_scene *scene, int64_t cap);

/* Test hook: the depth prefix of the binning's first phase for the scene's
 * renders.  Each (cell, tile) list first holds only the entries of the cell's
 * first ceil(E / 2^shift) depth-sorted endpoint events (E: the cell's
 * events); a segment whose sweep needs more is binned again with its full
 * list before the second windowed round.  shift = 0 bins every list in full
 * in one phase, shift = -1 (the default) learns the shift per workspace from
 * where the previous render's segments stopped.  The bounds do not depend on
 * it.  AR_EINVAL for a null scene or a shift outside [-1, 8]. */
int ar_debug_set_prefix(ar_scene *scene, int32_t shift);

/* Test hook: the cull before the FP64 decision part of the (Gaussian, cell)
 * records.  With it on, a first pass drops, from FP32 enclosures of the
 * FP64 values, the pairs certainly behind the near plane or outside the
 * frustum guard band (the outcome the FP64 chain reaches for them) and lists
 * the others, over which the FP64 chain then runs.  mode 1: always, 0: never,
 * -1 (the default): while the previous render of the workspace found fewer
 * than 3/4 of its pairs reaching a pixel.  ar_debug_records culls unless
 * mode is 0.  The records do not depend on it.  AR_EINVAL for a null scene
 * or another mode. */
int ar_debug_set_cull(ar_scene *scene, int32_t mode);

/* Test hooks, host only (no CUDA call): the two sizes a scene's next render
 * learns from the sweep statistics of its previous one.
 * ar_debug_learned_prefix: the depth prefix of the first binning phase (each
 * cell's first 2^-shift of its sorted events; 0 = one phase).  weights[64]
 * and counts[64]: over 64 equal buckets of each cell's depth order, the
 * summed full-list lengths and the number of the segments whose sweep
 * stopped in the bucket; n_entries, n_events: the tile entries and the depth
 * events of the render to come.  The shift minimises, over 0..6, the entries
 * the first phase sorts (n_entries 2^-shift), plus the full lists of the
 * segments that stopped past the prefix (scaled from the previous render),
 * the events of a second phase if there is one, and 12000 entries per
 * restarted segment; empty statistics give 3.  Result in *shift.
 * ar_debug_learned_window: the first round's record window (entries of a
 * segment whose records are built before its first sweep) from hist[256],
 * the segments by the entries they swept, in buckets of 32: the end of the
 * bucket that holds the 99.5th percentile plus one bucket, clamped to
 * [128, 4096]; an empty histogram gives 512.  Result in *window.
 * AR_EINVAL for null pointers. */
int ar_debug_learned_prefix(const uint64_t *weights, const uint32_t *counts, uint64_t n_entries, uint64_t n_events,
                            int32_t *shift);
int ar_debug_learned_window(const uint32_t *hist, uint32_t *window);

/* Device-memory limit (bytes, >= 1 MiB) for the scene's render workspace.
 * ar_render_abstract splits the cells of a call into batches whose
 * per-(Gaussian, cell) records take about a third of this limit, and runs the
 * pipeline once per batch (the bounds are the same as in one batch).
 * Default 64 GiB. */
int ar_set_workspace_limit(ar_scene *scene, int64_t bytes);

/* Stage timing with CUDA events on the render stream (on = 1) or off (0). */
int ar_set_profiling(ar_scene *scene, int on);

/* Blend of the scene's abstract renders (ar_render_abstract, _host, _noalloc
 * and serving; the plain FP64 path always uses AR_BLEND_INTERVAL):
 *   AR_BLEND_INTERVAL (default): BlendInd of Algorithm 4 with Prod bounded by
 *     interval products.
 *   AR_BLEND_RELATIONAL: the same, except that the transmittance of the upper
 *     bound is kept as an affine form in the pose, a McCormick product of the
 *     front Gaussians' opacity forms taken in depth order.  The extra term it
 *     adds is never positive, so every upper bound is at most the interval
 *     one (tighter where the cell is small enough that the bounds are not
 *     saturated); the lower bounds are the same.  Where the constants of
 *     the interval blend's upper terms alone reach 1 in every channel, the
 *     upper bound is 1 in both modes (the sweep stops there).  A Gaussian
 *     whose lower depth key equals the upper key of one absorbed earlier in
 *     its group of equal keys takes the interval term.
 * The mode applies to renders issued after the call.  AR_EINVAL for a null
 * scene or an unknown mode. */
#define AR_BLEND_INTERVAL 0
#define AR_BLEND_RELATIONAL 1
int ar_scene_set_blend(ar_scene *scene, int32_t mode);

/* Precision of the per-pixel opacity relaxation (Algorithm 1 lines 9-10 with
 * Table 2's Exp; FP64 in choosing the tangent and secant points of the Exp
 * relaxation where FP32 cannot carry them).  The FP32 renderer evaluates each
 * (pixel, Gaussian, cell) triple in FP32 with outward rounding and estimates
 * how far single precision moves the opacity bounds: the Mahalanobis term m
 * is a small difference of terms of magnitude about |m_lo| + |m_hi|, so the
 * estimate is 16 u (|m_lo| + |m_hi|) (a_lo + a_hi [m_lo > 0]) with u = 2^-24.
 * It is weighted by how far the pixel's bounds can still move with this
 * Gaussian's opacity: T_hi (the running upper transmittance) unless the upper
 * bound has already reached 1 in every channel, plus T_lo (the running lower
 * transmittance).  Where the weighted estimate exceeds `threshold`, the triple
 * is evaluated again in FP64 from the same record (the m interval, the Exp
 * points and the opacity forms) and the result is narrowed to FP32 outward.
 * Both results are sound; the FP64 one is within the record's own FP32
 * storage error of the FP64 oracle.  threshold = 0 takes every evaluation
 * with a nonzero estimate in FP64 (slow); a huge value none.  The decision
 * depends only on the pixel's own sweep, so it is the same for every tile
 * size and cell batching.  Default AR_FP64_ALPHA_DEFAULT.  Applies to ar_render_abstract, _host, _noalloc,
 * the partitioned and refined renders and serving; the count is
 * ar_render_stats.n_fp64.  AR_EINVAL for a null scene or a negative or NaN
 * threshold. */
#define AR_FP64_ALPHA_DEFAULT 1e-4f
int ar_scene_set_fp64_alpha(ar_scene *scene, float threshold);

/* CUDA graphs for repeated renders (on = 1, the default; 0 = off).  After the
 * one host synchronisation of a cell batch (which reads how many pairs and
 * tile entries it has, to size its buffers), everything else the batch
 * enqueues -- the binning and the windowed rounds of record build and render,
 * some forty kernels and memsets -- depends on the host only through those
 * sizes, the workspace's buffers and the call's parameters.  With graphs on,
 * that phase is captured once per such key (on a private stream, then
 * launched on cuda_stream) and later batches with the same key replay the
 * graph instead of enqueueing it again; up to 32 graphs are kept per
 * workspace.  The key includes the output buffers' addresses, the first
 * window the workspace has learned and the stage-timing switch, so renders
 * that reuse their output buffers replay from the second or third call on.  The bounds are bit-identical either way.  If a capture fails,
 * the scene falls back to enqueueing and turns graphs off.  Applies to
 * ar_render_abstract, _host, the partitioned and refined renders and serving
 * (not to the plain FP64 path or the no-allocation entry point, which
 * allocate nothing for graphs).  AR_EINVAL for a null scene or on not 0/1. */
int ar_scene_set_graphs(ar_scene *scene, int32_t on);

/* Counters and stage times of the scene's last render (synchronises its stream). */
int ar_last_render_stats(ar_scene *scene, ar_render_stats *stats);

/* ---- serving: continuous batching of abstract-render requests ----------
 * (The paper has no counterpart: it renders one query at a time.)
 * A server owns n_slots slots; each is a host worker thread with its own
 * non-blocking CUDA stream and workspace, so requests in different slots run
 * their whole pipelines concurrently on the device.  Submitted requests wait
 * in a FIFO (up to 1024); a slot that frees up admits the oldest request whose
 * workspace estimate fits the budget next to what the other slots hold, or a
 * later one that fits while leaving room for the oldest (backfilling).
 * Idle slots' workspaces are released when the oldest request does not fit.
 * Every slot has a high- and a low-priority CUDA stream: requests of at most 4
 * cells run on the high-priority one, larger ones on the other, and the
 * slots launch each batch's first per-pixel sweep as one CTA per (cell, tile)
 * segment, so that a small request's work is scheduled on the SMs a large
 * request's CTAs free as they finish, instead of after the large request.
 * Results are bit-identical to ar_render_abstract of the same request. */

/* hbm_budget_bytes: workspace budget (>= 1 MiB) shared by the slots, beside
 * the scenes and the callers' output buffers; n_slots: concurrent requests
 * (1..64).  The server uses the current CUDA device.  AR_EINVAL for bad
 * arguments, AR_EDEVICE if a stream cannot be created. */
int ar_serve_create(int64_t hbm_budget_bytes, int32_t n_slots, ar_server **out);

/* Drops queued requests (their tickets become unknown), waits for running
 * ones to finish, then frees the server's streams and workspaces. */
int ar_serve_destroy(ar_server *server);

/* Submit one request (non-blocking).  The scene must live on the server's
 * device and outlive the request; intrinsics, pose and cells are copied;
 * out_lower/out_upper are device buffers as for ar_render_abstract (tile
 * chosen automatically) and must not be touched until the ticket is done.
 * Returns AR_EAGAIN when the queue is full (try again later), AR_EINVAL for
 * bad arguments (validated as for ar_render_abstract).  *ticket identifies
 * the request. */
int ar_serve_submit(ar_server *server, ar_scene *scene, const ar_intrinsics *intr,
                    const ar_nominal_pose *pose, const ar_pose_box *cells, int32_t n_cells,
                    float *out_lower, float *out_upper, uint64_t *ticket);

/* Timeout of the server's requests in ms, measured from submission (0: none,
 * the default).  A request still queued when it expires is completed with
 * AR_ETIMEOUT without running.  A running one whose GPU work has not finished
 * when it expires (a host watchdog polls the slot's stream) is completed with
 * AR_ETIMEOUT at once; its outputs are then undefined, and the slot waits for
 * that work to drain before it admits another request.  Applies to requests
 * admitted or polled after the call.  AR_EINVAL for a null server or a
 * negative or NaN timeout. */
int ar_serve_set_timeout(ar_server *server, double timeout_ms);

/* Cancel a ticket.  A queued request leaves the queue at once and completes
 * with AR_ECANCELED (its outputs untouched); a running one completes with
 * AR_ECANCELED when its GPU work ends (its outputs may have been written); a
 * completed one keeps its status.  The ticket is retired by ar_serve_poll as
 * usual.  AR_EINVAL for a null server or an unknown or retired ticket. */
int ar_serve_cancel(ar_server *server, uint64_t ticket);

/* Poll a ticket: *done = 1 once its outputs are complete; then *latency_ms is
 * the submit-to-completion wall time, the ticket is retired, and the return
 * value is the request's own status (AR_OK, or the code its render failed
 * with, the message in ar_last_error).  *done = 0 (and *latency_ms = -1) while
 * it waits or runs.  AR_EINVAL for an unknown or retired ticket. */
int ar_serve_poll(ar_server *server, uint64_t ticket, int *done, double *latency_ms);

/* Message of the calling thread's last failure ("" if none).  The pointer
 * stays valid until the thread's next libar call. */
const char *ar_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* AR_H */
