// ar_host.h -- host-side device-memory helpers of libar.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "ar.h"

namespace ar {

// Grow-only device buffer.
struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    int ensure(size_t bytes);  // AR_OK or AR_ENOMEM (sets the thread's error message)
    void release();
    template <class T> T *as() const { return (T *)p; }
};

// A captured post-sync phase of a cell batch (binning and the windowed
// rounds), keyed by everything its launches depend on.
struct GraphEntry {
    std::vector<uint64_t> key;
    cudaGraphExec_t exec;
    int launches;        // kernels it launches
    uint64_t last_use;
};
constexpr size_t kMaxGraphs = 32;  // cached graphs per workspace (least recently used goes)

// Everything one render needs besides the scene itself.  A scene owns one
// workspace; a server owns one per slot so that concurrent requests never
// share buffers.
struct Workspace {
    DevBuf cells_lohi, cells, vN, recs, boxes, keys, counters;
    DevBuf evk0, evk1, evv0, evv1, ents0, ents1, ente0, ente1;
    DevBuf ua, ub, uc, ud, hist, scan, segs, sege, segk0, segk1, segv0, segv1, work;
    DevBuf clist;                              // pairs left by the cull (then their count)
    bool cull_on = true;                       // the last render found culling worth it
    DevBuf segt, cellev, bwords, smask, ssat;  // two-phase binning: full-list lengths, cell event ranges,
                                               // counts, active mask and its summed-area tables
    DevBuf state, wlist, act0, act1, words, slist;  // windowed rounds: pair states, build list, active segments
    DevBuf plist, pmask;                     // segments swept again with FP64 evaluations, their pixel masks
    DevBuf whist;                            // [256] sweep-length histogram of the current render, then
                                             // [64] 64-bit: full-list entries by where the segments stopped
    uint32_t *h_whist = nullptr;             // page-locked copy of the last render's histogram
    bool whist_pending = false;              // h_whist holds a render not yet learned from
    uint32_t w0 = 512;                       // first window of the windowed rounds
    int prefix_shift = 3;                    // depth prefix of the first binning phase: 1 / 2^shift of the events
    DevBuf out_lo, out_hi;      // staged outputs of ar_render_abstract_host
    DevBuf part_lo, part_hi;    // chunk outputs of ar_render_abstract_partitioned / _refined
    DevBuf lvl_lo, lvl_hi;      // one refinement round's union (ar_render_abstract_refined)
    DevBuf wpart;               // partial width sums of the refinement's pieces
    unsigned long long *h_counters = nullptr;  // page-locked
    std::vector<cudaEvent_t> evs;              // 9 per cell batch (stage timing)
    int n_batches = 0;                         // cell batches of the last render
    int64_t fallback_prep = 0;                 // MatrixInv fallbacks counted by the record kernel
    int64_t split_prep = 0;                    // MatrixInv input splits counted by the record kernel
    int64_t built_prep = 0;                    // records built completely by the record kernel
    std::vector<GraphEntry> graphs;            // captured batch phases (see render_batch)
    uint64_t graph_clock = 0, graph_hits = 0;
    cudaStream_t cap_stream = nullptr;         // private stream the captures are taken on
    bool interleave = false;                   // server slots: the first sweep in one CTA per segment
    void release();
    size_t bytes() const;
    void append_pointers(std::vector<uint64_t> &key) const;  // every buffer's address, for graph keys
};

int set_last_error(int code, const char *msg);  // sets ar_last_error() for this thread

int validate_call(const ar_intrinsics *in, const ar_nominal_pose *pose, const ar_pose_box *cells, int32_t n_cells,
                  int32_t tile);
struct RenderLaunch;
struct CallConst;
struct TunedTile {
    int W, H, M, TS, CH;  // key (image size, pose variables) -> tile edge, events per staged chunk
};
// The FP32 render of one batch in windowed rounds (see render_kernel):
// demand -> build -> render per round, windows w0, 8192, then unlimited.
// state [n_pairs] (zeroed here), wlist [n_pairs], act0/act1 [n_seg], words [8];
// build_counters: [0] fallbacks, [1] records built, [2] splits (optional);
// split_list [n_pairs]: pairs whose MatrixInv needs input splitting, which a
// second kernel finishes with a warp each; precise_list [n_seg]: segments that
// meet an opacity evaluation needing FP64, swept again by the FP64-capable
// render instance in the same round, and precise_mask [n_seg * TS * TS / 32]
// the pixels of each that do.
// rebin / first: the binning of a two-phase render, whose second phase runs
// between the first and the second round (null: one phase, lists complete)
struct BinArgs;
struct BinOut;
int run_windowed_render(int M, int TS, RenderLaunch rl, const CallConst &cc, const void *cells, const double *vN,
                        uint64_t n_pairs, uint64_t n_seg, uint32_t *state, uint32_t *wlist, uint32_t *act0,
                        uint32_t *act1, uint32_t *words, unsigned long long *build_counters, cudaStream_t st,
                        int *launches, cudaEvent_t *ev, uint32_t w0, uint32_t *split_list, uint32_t *precise_list,
                        uint32_t *precise_mask, const BinArgs *rebin = nullptr, const BinOut *first = nullptr);
// Depth prefix of the next render's first binning phase, from the stop
// histograms of an earlier render (64 buckets of full-list entries, and of
// segments, by where in its cell's depth order a segment stopped): the shift
// s in [0, 6] that minimises the entries sorted, n_entries / 2^s plus the
// entries of the segments that stop beyond the prefix, plus n_events for the
// second phase's pass over the events if any does, plus a fixed cost per
// restarted segment.
int learned_prefix_shift(const unsigned long long *hist64, const uint32_t *count64, uint64_t n_entries,
                         uint64_t n_events);
// First window from the sweep histogram of an earlier render: the smallest
// multiple of 32 entries that covers 99.5 % of its segments, in [128, 4096].
uint32_t learned_window(const uint32_t *hist256);
int render_core(ar_scene *s, Workspace &ws, const ar_intrinsics *in, const ar_nominal_pose *pose,
                const ar_pose_box *cells, int32_t n_cells, int32_t tile, float *out_lo, float *out_hi,
                cudaStream_t st, bool profiling, ar_render_stats *stats, bool plain = false,
                int64_t ws_limit = 0, int chunk = 0);

}  // namespace ar

// A scene: the Gaussians on one device plus the workspace of its renders.
struct ar_scene {
    int device = 0;
    int64_t n = 0;
    float *uw = nullptr, *ls = nullptr, *quat = nullptr, *opac = nullptr, *rgb = nullptr;
    double *Mw = nullptr, *tau = nullptr;
    // scene-parameter boxes (Sec. 4.5) of the abstract render: the mean's box
    // (both pointers at uw without boxes) and the opacity and colour boxes as
    // GParam; boxbuf owns the box arrays once they are set
    const float *uw_lo = nullptr, *uw_hi = nullptr;
    void *gp = nullptr;
    float *boxbuf = nullptr;
    float k_open = 1.f;  // 1 / (1 - largest upper opacity), rounded up (bounds skipped lower-sum terms)
    int64_t ws_limit = int64_t(64) << 30;  // workspace limit that sizes the cell batches
    ar::Workspace ws;
    bool profiling = false;
    int blend = AR_BLEND_INTERVAL;  // blend of the abstract renders (ar_scene_set_blend)
    bool graphs = true;             // replay repeated batch phases as CUDA graphs (ar_scene_set_graphs)
    int chunk = 0;                  // sweep chunk for explicit tiles (0: 16; ar_debug_set_chunk)
    // a cell batch with this many tile entries or more is split in two (the
    // 32-bit entry indices; lowered by ar_debug_set_entry_cap for tests)
    uint64_t entry_cap = (1ull << 32) - (1ull << 20);
    // depth prefix of the first binning phase: -1 learned per workspace, else
    // the shift (0: one phase); set by ar_debug_set_prefix for tests
    int prefix_force = -1;
    // culling of the certain drops before the FP64 decision chain: -1 chosen
    // per workspace, 0 off, 1 on; set by ar_debug_set_cull for tests
    int cull_force = -1;
    float fp64_dev = AR_FP64_ALPHA_DEFAULT;  // FP64 re-evaluation threshold (ar_scene_set_fp64_alpha)
    ar_render_stats stats;
    cudaStream_t stats_stream = nullptr;
    // tile edges chosen by the autotuner, per (width, height, pose variables)
    std::mutex tune_mu;
    std::vector<ar::TunedTile> tuned;
};
