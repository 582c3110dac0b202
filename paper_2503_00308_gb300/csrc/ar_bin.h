// ar_bin.h -- host interface of the binning / sorting stage.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ar {

struct PixBox;

struct BinArgs {
    const PixBox *boxes;     // [n_pairs] pixel boxes, x0 < 0 = absent
    const double *keys;      // [n_pairs][2] depth-key interval
    uint64_t n_pairs;        // n_cells * n_gauss
    uint64_t n_gauss;
    int n_cells;
    uint64_t n_events;       // 2 * pairs present
    uint64_t n_entries;      // sum over events of tiles met
    int TS, ntx, n_tiles;
    uint64_t n_segments;     // n_cells * n_tiles
    uint64_t *ev_key[2];     // [n_events] x2
    uint32_t *ev_val[2];     // [n_events] x2
    uint32_t *ent_seg[2];    // [n_entries] x2
    uint32_t *ent_ev[2];     // [n_entries] x2
    uint32_t *u32_a, *u32_b, *u32_c, *u32_d;  // scratch, >= max(n_pairs, n_events) words each
    uint32_t *hist;          // >= radix_hist_words(max(n_events, n_entries))
    uint32_t *scan_tmp;      // >= scan_temp_words(largest scanned length)
    uint32_t *seg_start, *seg_end;  // [n_segments]
    uint32_t *seg_k[2], *seg_v[2];  // [n_segments] x2 each: segment order by length
    // Two-phase binning (prefix_shift > 0): the first phase bins only each
    // cell's first ceil(E / 2^prefix_shift) depth-sorted events (E: the
    // cell's events), and seg_total receives the lengths of the full lists;
    // run_rebin bins the full lists of the segments that need them.
    int prefix_shift = 0;
    uint32_t *cell_ev = nullptr;    // [n_cells + 1] first sorted event of each cell
    uint32_t *pref_start = nullptr; // [n_cells + 1] first index of each cell's prefix events (compacted)
    uint32_t *seg_total = nullptr;  // [n_segments]
    uint32_t *words = nullptr;      // [4] counts known on the device only (entries of each phase, prefix events)
    uint32_t *mask = nullptr;       // [(n_segments + 31) / 32] active segments of the second phase
    uint32_t *sat = nullptr;        // [n_cells][(nty + 1) (ntx + 1)] their summed-area tables
};

struct BinOut {
    const uint64_t *ev_key;  // sorted event keys
    const uint32_t *ev_val;  // sorted event values: 2 * pair + (upper endpoint)
    const uint32_t *ent_seg; // entries sorted by segment
    const uint32_t *ent_ev;  // entry -> sorted event index
    const uint32_t *seg_order;  // segments, longest first
    const uint32_t *seg_total;  // full-list lengths, or null: the lists are complete (seg_end - seg_start)
};

size_t scan_temp_words(uint64_t n);
size_t radix_hist_words(uint64_t n);
void exclusive_scan(const uint32_t *in, uint32_t *out, uint64_t n, uint32_t *tmp, cudaStream_t st, int *launches);
int run_binning(const BinArgs &a, BinOut &o, cudaStream_t st, int *launches);
// The second phase: complete lists for the segments active[0, *n_active)
// (a device count), sorted as run_binning sorts them, in place of the first
// phase's lists (the other segments' bounds become empty); o.seg_order lists
// the active segments again, longest first.
int run_rebin(const BinArgs &a, const BinOut &first, const uint32_t *active, const uint32_t *n_active, BinOut &o,
              cudaStream_t st, int *launches);

// Windowed rounds of the renderer.  launch_demand claims (state 0 -> 1) the
// pairs whose lower endpoints lie in the first `window` entries of the
// active segments and lists them in work (count is incremented); the grid is
// sized from max_active, the count of active segments is read on the device.
void launch_set_u32(uint32_t *p, uint32_t v, cudaStream_t st);
void launch_demand(const uint32_t *active, const uint32_t *n_active, uint32_t max_active, const uint32_t *seg_start,
                   const uint32_t *seg_end, const uint32_t *ent_ev, const uint32_t *ev_val, uint32_t window,
                   uint32_t *state, uint32_t *work, uint32_t *count, cudaStream_t st);

}  // namespace ar
