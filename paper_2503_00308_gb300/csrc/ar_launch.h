// ar_launch.h -- host launchers of the per-M kernels (instantiated for the
// numbers of pose variables M in {1, 4, 6} carried by the linear forms).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ar {

struct CallConst;
struct PixBox;

struct RenderLaunch {
    float *recs;                      // FP32 records
    const double *recs64 = nullptr;   // FP64 records (plain renderer only)
    const PixBox *boxes;
    const uint32_t *seg_start, *seg_end, *seg_order, *ent_ev, *ev_val;
    // full-list lengths where the lists are depth prefixes (the first binning
    // phase), else null; a segment whose sweep needs more than its prefix is
    // abandoned like one that leaves its window
    const uint32_t *seg_total = nullptr;
    const uint32_t *cell_ev = nullptr;  // [n_cells + 1] first sorted event of each cell (for sweep_hist's depth part)
    // windowed rounds (FP32 renderer): segments active[0, *n_active) are swept;
    // one that needs entries beyond `window` is appended to next_active
    const uint32_t *active = nullptr, *n_active = nullptr;
    uint32_t *next_active = nullptr, *n_next = nullptr;
    uint32_t window = 0xffffffffu;
    uint32_t *sweep_hist = nullptr;   // optional [256]: completed segments by entries swept / 32, then (with
                                      // cell_ev) [64] 64-bit: their full lengths by where in the cell's
                                      // depth order they stopped, and [64] their counts
    const uint64_t *ev_key;
    int W, H, ntx, n_tiles, n_cells;
    int64_t n_gauss;
    float k_open;                     // 1 / (1 - largest opacity), rounded up
    float fp64_dev = 3.0e38f;         // opacity evaluations whose FP32 deviation estimate exceeds this
                                      // are taken again in FP64 (pixel_alpha_fp64)
    float *out_lo, *out_hi;
    unsigned long long *counters;     // optional: [0] opacity evaluations, [1] re-evaluations,
                                      // [5] segments abandoned for a wider window ([2]-[4]: record build),
                                      // [6] evaluations taken again in FP64, [7] segments swept again for them
    unsigned int *work;               // segment counter of the persistent grid (zeroed by the launcher)
    int rel = 0;                      // 1: relational upper transmittance (AR_BLEND_RELATIONAL)
    int ch = 16;                      // events per staged chunk of the FP32 sweep (8, 16 or 32 at tile 16)
    // interleave: the first round's FP32 sweep (whose active list is all n_seg
    // segments) launches one CTA per segment (direct) instead of persistent
    // CTAs, so that work on a higher-priority stream can take SMs as they free
    int interleave = 0, direct = 0;
    // precision: the FP32 sweep (f64 = 0) appends a segment that needs an FP64
    // evaluation to precise[*n_precise], with the mask of the pixels that do in
    // precise_mask[slot * (TS * TS / 32 + 1) ...] (then a flag word); the f64 = 1 instance sweeps them
    int f64 = 0;
    uint32_t *precise = nullptr, *n_precise = nullptr, *precise_mask = nullptr;
};

size_t cell_data_bytes(int M);
int rec_width(int M);
int launch_cell_prep(int M, const double *lo, const double *hi, const CallConst &cc, void *cells, cudaStream_t st);
// list, count (optional): cull the certain drops first and run the FP64
// decision chain over the list of the other pairs (cull_kernel)
int launch_record_prep(int M, const double *vN, const void *gp,
                       const CallConst &cc, const void *cells, int TS, float *recs, PixBox *boxes, double *keys,
                       unsigned long long *counters, cudaStream_t st, uint32_t *list = nullptr,
                       uint32_t *count = nullptr);
int launch_render(int M, int TS, const RenderLaunch &a, cudaStream_t st);
int launch_record_prep64(int M, const double *vN, const void *gp,
                         const CallConst &cc, const void *cells, int TS, double *recs, PixBox *boxes, double *keys,
                         unsigned long long *counters, cudaStream_t st);
int launch_render_plain(int M, int TS, const RenderLaunch &a, cudaStream_t st);
// union of the bounds of n_cells cells of n floats each (k_union.cu); acc: fold
// the current outputs in too
int launch_bounds_union(const float *lo, const float *hi, int n_cells, size_t n, float *out_lo, float *out_hi,
                        bool acc, cudaStream_t st);
// out = out intersected with [lo, hi] elementwise (k_union.cu)
int launch_bounds_intersect(const float *lo, const float *hi, size_t n, float *out_lo, float *out_hi, cudaStream_t st);
// part[c * blocks + b] = partial sum of (hi - lo) over cell c (k_union.cu); the
// host adds the partials in order, so the sums are deterministic
int launch_width_partials(const float *lo, const float *hi, int n_cells, size_t n, int blocks, double *part,
                          cudaStream_t st);
// value parts of the records listed in work[0, *count); counters: [0] fallbacks, [1] built, [2] split.
// split_list (list_cap >= *count entries), split_count and khigh_count (zeroed by the caller): pairs whose
// MatrixInv fails on the cell are split by a warp each in a second kernel, pairs whose Taylor order exceeds
// the default are finished in a third (listed from the back of split_list).
int launch_record_build(int M, const double *vN, const CallConst &cc, const void *cells, int64_t n_gauss,
                        const uint32_t *work, const uint32_t *count, float *recs, unsigned long long *counters,
                        uint32_t *split_list, uint32_t *split_count, uint32_t list_cap, uint32_t *khigh_count,
                        cudaStream_t st);
// concrete render (k_concrete.cu)
size_t concrete_pose_bytes();
int concrete_rec_width();
int launch_concrete_pose(const double *delta, const CallConst &cc, void *pose, cudaStream_t st);
int launch_concrete_prep(const float *uw, const double *Mw, const double *tau, const float *opac, const float *rgb,
                         const CallConst &cc, const void *pose, int TS, double *recs, PixBox *boxes, double *keys,
                         unsigned long long *counters, cudaStream_t st);
int launch_concrete_render(const double *recs, const PixBox *boxes, const uint32_t *seg_start, const uint32_t *seg_end,
                           const uint32_t *ent_ev, const uint32_t *ev_val, const uint64_t *ev_key, int W, int H,
                           int ntx, int n_tiles, float *out, cudaStream_t st);
int launch_scene_prep(const float *logscale, const float *quat, const float *opacity, int64_t n, double *Mw,
                      double *tau, cudaStream_t st);
int launch_pose_prep(const float *uw_lo, const float *uw_hi, const double *Mw, int64_t n, const CallConst &cc,
                     double *vN, cudaStream_t st);
int launch_gparam(const float *o_lo, const float *o_hi, const float *c_lo, const float *c_hi, int64_t n, void *gp,
                  cudaStream_t st);

}  // namespace ar
