// k_bin.cu -- screen-tile binning of (Gaussian, cell) pairs and depth-key
// ordering of their endpoint events (the tile-based batching of Sec. 4,
// "AbstractSplat on GPUs").
//
// Pipeline (all on the render stream):
//   1. flags/scan   : compact the (cell, Gaussian) pairs that reach the image;
//   2. events       : two per pair (lower / upper depth-key endpoint), keyed by
//                     the order-preserving bits of the FP64 key;
//   3. sort         : stable LSD radix sort by key, then stably by cell;
//   4. entries      : each event is copied to every tile its pixel box meets,
//                     in sorted-event order (cell-major), keyed by tile and cell;
//   5. sort         : stable LSD radix sort by tile (keeps the cell-major key
//                     order inside, so every (cell, tile) segment is contiguous);
//   6. bounds       : [start, end) of every segment.
#include "ar_bin.h"
#include "ar_common.cuh"

namespace ar {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;  // items per block
constexpr uint32_t kDevGrid = 152u * 8u;          // blocks of a pass whose count is on the device

// ------------------------------------------------------------------ scan
constexpr int SC_THREADS = 256;
constexpr int SC_IPT = 8;
constexpr int SC_TILE = SC_THREADS * SC_IPT;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *s_warp, uint32_t &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = (lane < SC_THREADS / 32) ? s_warp[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += y;
        }
        if (lane < SC_THREADS / 32) s_warp[lane] = w;
    }
    __syncthreads();
    total = s_warp[SC_THREADS / 32 - 1];
    uint32_t excl = x - v + (warp > 0 ? s_warp[warp - 1] : 0);
    __syncthreads();
    return excl;
}

// The length of a scanned array known on the device only: mul ceil(*p /
// div) words, at most the host's bound (p null: the host's length).
struct DevLen {
    const uint32_t *p = nullptr;
    uint32_t mul = 1, div = 1;
};
__device__ __forceinline__ uint32_t dev_len(DevLen d, uint32_t n)
{
    if (!d.p) return n;
    const uint64_t w = (uint64_t)d.mul * (((uint64_t)*d.p + d.div - 1) / d.div);
    return w < n ? (uint32_t)w : n;
}

__global__ void __launch_bounds__(SC_THREADS) scan_sums_kernel(const uint32_t *__restrict__ in, uint32_t n,
                                                               uint32_t *__restrict__ sums, DevLen dl)
{
    __shared__ uint32_t s_warp[32];
    n = dev_len(dl, n);
    const uint64_t base = (uint64_t)blockIdx.x * SC_TILE + (uint64_t)threadIdx.x * SC_IPT;
    uint32_t t = 0;
#pragma unroll
    for (int i = 0; i < SC_IPT; ++i)
        if (base + i < n) t += in[base + i];
    uint32_t total;
    block_exclusive_scan(t, s_warp, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SC_THREADS) scan_apply_kernel(const uint32_t *__restrict__ in, uint32_t n,
                                                                const uint32_t *__restrict__ offs,
                                                                uint32_t *__restrict__ out, DevLen dl)
{
    __shared__ uint32_t s_warp[32];
    n = dev_len(dl, n);
    if ((uint64_t)blockIdx.x * SC_TILE >= n) return;  // uniform over the block
    const uint64_t base = (uint64_t)blockIdx.x * SC_TILE + (uint64_t)threadIdx.x * SC_IPT;
    uint32_t v[SC_IPT];
    uint32_t t = 0;
#pragma unroll
    for (int i = 0; i < SC_IPT; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0u;
        t += v[i];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan(t, s_warp, total) + (offs ? offs[blockIdx.x] : 0u);
#pragma unroll
    for (int i = 0; i < SC_IPT; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

size_t scan_temp_words(uint64_t n)
{
    size_t w = 0;
    while (n > (uint64_t)SC_TILE) {
        n = (n + SC_TILE - 1) / SC_TILE;
        w += 2 * n;
    }
    return w + 2;
}

// exclusive scan of n words (in may equal out); tmp from scan_temp_words.
// dl: the length on the device (n its bound); the words past it are neither
// read nor written.
static void exclusive_scan_dl(const uint32_t *in, uint32_t *out, uint64_t n, uint32_t *tmp, cudaStream_t st,
                              int *launches, DevLen dl)
{
    if (n == 0) return;
    const uint64_t nb = (n + SC_TILE - 1) / SC_TILE;
    if (nb == 1) {
        scan_apply_kernel<<<1, SC_THREADS, 0, st>>>(in, (uint32_t)n, nullptr, out, dl);
        ++*launches;
        return;
    }
    uint32_t *sums = tmp, *offs = tmp + nb;
    scan_sums_kernel<<<(unsigned)nb, SC_THREADS, 0, st>>>(in, (uint32_t)n, sums, dl);
    ++*launches;
    exclusive_scan_dl(sums, offs, nb, tmp + 2 * nb, st, launches, DevLen{});
    scan_apply_kernel<<<(unsigned)nb, SC_THREADS, 0, st>>>(in, (uint32_t)n, offs, out, dl);
    ++*launches;
}

void exclusive_scan(const uint32_t *in, uint32_t *out, uint64_t n, uint32_t *tmp, cudaStream_t st, int *launches)
{
    exclusive_scan_dl(in, out, n, tmp, st, launches, DevLen{});
}

// ------------------------------------------------------------ radix sort
// Digits of RB bits (NB = 2^RB buckets, RB <= 8).  A sort of `bits` key bits
// takes ceil(bits / 8) passes of equal digits, so that no pass spends buckets
// on bits beyond the key: fewer buckets give longer digit runs per block and
// fuller store sectors in the scatter.
// digit of an item: key bits [shift, shift + RB), or, with CELL, bits of the
// cell of the event's pair (val = 2 pair + end, pair = cell n_gauss + g)
template <class K, int RB, bool CELL>
__device__ __forceinline__ uint32_t rs_digit(K key, uint32_t val, int shift, uint64_t n_gauss)
{
    constexpr uint32_t NB = 1u << RB;
    if (CELL) return (uint32_t)(((uint64_t)(val >> 1) / n_gauss) >> shift) & (NB - 1u);
    return (uint32_t)(key >> shift) & (NB - 1u);
}

// Both kernels of a pass take the item count n from the host, or (n_dev
// non-null) the smaller of n and *n_dev, a count known only on the device
// (the grid is then sized for n and each block loops over tiles).
template <class K, int RB, bool CELL>
__global__ void __launch_bounds__(RS_THREADS) rs_hist_kernel(const K *__restrict__ keys,
                                                             const uint32_t *__restrict__ vals, uint32_t n,
                                                             int shift, uint64_t n_gauss,
                                                             uint32_t *__restrict__ hist, uint32_t nblocks,
                                                             const uint32_t *__restrict__ n_dev)
{
    constexpr uint32_t NB = 1u << RB;
    __shared__ uint32_t h[NB];
    // with a device count, the histogram's columns are its blocks alone
    if (n_dev) {
        n = min(n, *n_dev);
        nblocks = (n + RS_TILE - 1) / RS_TILE;
    }
    for (uint32_t blk = blockIdx.x; blk < nblocks; blk += gridDim.x) {
        if (threadIdx.x < NB) h[threadIdx.x] = 0;
        __syncthreads();
        const uint64_t base = (uint64_t)blk * RS_TILE;
        // the counts do not depend on which thread reads which item: each thread
        // reads RS_ROUNDS consecutive items with 16-byte loads where the tile is
        // whole (the arrays are 16-byte aligned), else one by one
        const uint64_t i0 = base + (uint64_t)threadIdx.x * RS_ROUNDS;
        if (CELL) {
            static_assert(RS_ROUNDS % 4 == 0, "whole vectors per thread");
            uint32_t v[RS_ROUNDS];
            if (base + RS_TILE <= n) {
#pragma unroll
                for (int q = 0; q < RS_ROUNDS / 4; ++q)
                    reinterpret_cast<uint4 *>(v)[q] = reinterpret_cast<const uint4 *>(vals + i0)[q];
#pragma unroll
                for (int r = 0; r < RS_ROUNDS; ++r)
                    atomicAdd(&h[rs_digit<K, RB, true>(0, v[r], shift, n_gauss)], 1u);
            } else {
#pragma unroll
                for (int r = 0; r < RS_ROUNDS; ++r)
                    if (i0 + r < n) atomicAdd(&h[rs_digit<K, RB, true>(0, vals[i0 + r], shift, n_gauss)], 1u);
            }
        } else {
            constexpr int PER16 = 16 / (int)sizeof(K);
            static_assert(RS_ROUNDS % PER16 == 0, "whole vectors per thread");
            K v[RS_ROUNDS];
            if (base + RS_TILE <= n) {
#pragma unroll
                for (int q = 0; q < RS_ROUNDS / PER16; ++q)
                    reinterpret_cast<uint4 *>(v)[q] = reinterpret_cast<const uint4 *>(keys + i0)[q];
#pragma unroll
                for (int r = 0; r < RS_ROUNDS; ++r) atomicAdd(&h[rs_digit<K, RB, false>(v[r], 0, shift, 0)], 1u);
            } else {
#pragma unroll
                for (int r = 0; r < RS_ROUNDS; ++r)
                    if (i0 + r < n) atomicAdd(&h[rs_digit<K, RB, false>(keys[i0 + r], 0, shift, 0)], 1u);
            }
        }
        __syncthreads();
        if (threadIdx.x < NB) hist[(uint64_t)threadIdx.x * nblocks + blk] = h[threadIdx.x];
        __syncthreads();  // h is cleared for the next tile
    }
}

// Scatter of one radix pass.  Each block ranks its RS_TILE items by digit
// (stable: warps in order, rounds in order, lanes in order), reorders them by
// digit in shared memory, then writes every digit run to its global offset
// with consecutive threads on consecutive addresses.
template <class K, int RB, bool CELL>
__global__ void __launch_bounds__(RS_THREADS) rs_scatter_kernel(const K *__restrict__ kin,
                                                                const uint32_t *__restrict__ vin,
                                                                K *__restrict__ kout, uint32_t *__restrict__ vout,
                                                                uint32_t n, int shift, uint64_t n_gauss,
                                                                const uint32_t *__restrict__ offs,
                                                                uint32_t nblocks, const uint32_t *__restrict__ n_dev)
{
    constexpr uint32_t NB = 1u << RB;
    static_assert(NB <= RS_THREADS, "one thread per digit");
    __shared__ uint32_t wcnt[RS_WARPS][NB];
    __shared__ uint32_t dstart[NB];   // block-local start of each digit run
    __shared__ uint32_t gbase[NB];    // global start of each digit run of this block
    __shared__ uint32_t s_warp[RS_WARPS];
    __shared__ K s_key[RS_TILE];
    __shared__ uint32_t s_val[RS_TILE];
    if (n_dev) {
        n = min(n, *n_dev);
        nblocks = (n + RS_TILE - 1) / RS_TILE;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t ltmask = (1u << lane) - 1u;
    for (uint32_t blk = blockIdx.x; blk < nblocks; blk += gridDim.x) {
        const uint64_t blk0 = (uint64_t)blk * RS_TILE;
        if (blk0 >= n) break;  // uniform over the block; later tiles are empty too
        for (int i = threadIdx.x; i < RS_WARPS * (int)NB; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
        __syncthreads();
        const uint64_t base = blk0 + (uint64_t)warp * (RS_ROUNDS * 32);
        K key[RS_ROUNDS];
        uint32_t val[RS_ROUNDS], dig[RS_ROUNDS], rank[RS_ROUNDS];
        // all loads first, so that they are in flight together
#pragma unroll
        for (int r = 0; r < RS_ROUNDS; ++r) {
            const uint64_t i = base + (uint64_t)r * 32 + lane;
            const bool ok = i < n;
            key[r] = ok ? kin[i] : (K)0;
            val[r] = ok ? vin[i] : 0u;
            dig[r] = ok ? rs_digit<K, RB, CELL>(key[r], val[r], shift, n_gauss) : NB;
        }
#pragma unroll
        for (int r = 0; r < RS_ROUNDS; ++r) {
            const bool ok = dig[r] < NB;
            // lanes with the same digit, by one ballot per digit bit (bit RB marks
            // the lanes past the end, so that they match only one another)
            uint32_t peers = 0xffffffffu;
#pragma unroll
            for (int b = 0; b <= RB; ++b) {
                const bool bit = (dig[r] >> b) & 1u;
                const uint32_t m = __ballot_sync(0xffffffffu, bit);
                peers &= bit ? m : ~m;
            }
            uint32_t before = 0;
            if (ok) before = wcnt[warp][dig[r]];
            rank[r] = before + __popc(peers & ltmask);
            __syncwarp();
            if (ok && lane == __ffs(peers) - 1) wcnt[warp][dig[r]] = before + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        {
            // per digit (threads 0..NB-1): warp prefix, block total, then the
            // block-local start
            const int d = threadIdx.x;
            uint32_t run = 0;
            if (d < (int)NB) {
#pragma unroll
                for (int w = 0; w < RS_WARPS; ++w) {
                    const uint32_t t = wcnt[w][d];
                    wcnt[w][d] = run;
                    run += t;
                }
            }
            uint32_t x = run;  // inclusive scan of the totals over the digits
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) s_warp[warp] = x;
            __syncthreads();
            if (d < (int)NB) {
                uint32_t wpre = 0;
                for (int w = 0; w < warp; ++w) wpre += s_warp[w];
                dstart[d] = wpre + x - run;
                gbase[d] = offs[(uint64_t)d * nblocks + blk];
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < RS_ROUNDS; ++r) {
            if (dig[r] < NB) {
                const uint32_t lp = dstart[dig[r]] + wcnt[warp][dig[r]] + rank[r];
                s_key[lp] = key[r];
                s_val[lp] = val[r];
            }
        }
        __syncthreads();
        const uint32_t cnt = n - blk0 < (uint64_t)RS_TILE ? (uint32_t)(n - blk0) : (uint32_t)RS_TILE;
        for (uint32_t j = threadIdx.x; j < cnt; j += RS_THREADS) {
            const K k = s_key[j];
            const uint32_t v = s_val[j];
            const uint32_t d = rs_digit<K, RB, CELL>(k, v, shift, n_gauss);
            const uint32_t pos = gbase[d] + (j - dstart[d]);
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();  // the shared arrays are rewritten for the next tile
    }
}

size_t radix_hist_words(uint64_t n)
{
    const uint64_t nb = (n + RS_TILE - 1) / RS_TILE;
    return 256 * nb;
}

// n_dev: see rs_hist_kernel; n is then an upper bound, and the grid is at
// most a few blocks per SM
template <class K, int RB, bool CELL = false>
static void radix_pass(const K *ka, const uint32_t *va, K *kb, uint32_t *vb, uint64_t n, int shift, uint32_t *hist,
                       uint32_t *scan_tmp, cudaStream_t st, int *launches, uint64_t n_gauss = 0,
                       const uint32_t *n_dev = nullptr)
{
    const uint32_t nb = (uint32_t)((n + RS_TILE - 1) / RS_TILE);
    const uint32_t grid = n_dev ? (nb < kDevGrid ? nb : kDevGrid) : nb;
    rs_hist_kernel<K, RB, CELL><<<grid, RS_THREADS, 0, st>>>(ka, va, (uint32_t)n, shift, n_gauss, hist, nb, n_dev);
    ++*launches;
    DevLen dl;
    if (n_dev) dl = DevLen{n_dev, 1u << RB, (uint32_t)RS_TILE};
    exclusive_scan_dl(hist, hist, ((uint64_t)1 << RB) * nb, scan_tmp, st, launches, dl);
    rs_scatter_kernel<K, RB, CELL><<<grid, RS_THREADS, 0, st>>>(ka, va, kb, vb, (uint32_t)n, shift, n_gauss, hist, nb,
                                                                n_dev);
    ++*launches;
}

// Stable sort of the events (keys, vals) by the cell of their pair, bits
// [0, bits) of it, in passes of at most 8 bits; returns 1 if the result
// ended in the alt buffers.
static int radix_sort_cells(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, uint64_t n,
                            int bits, uint64_t n_gauss, uint32_t *hist, uint32_t *scan_tmp, cudaStream_t st,
                            int *launches)
{
    if (n == 0 || bits <= 0) return 0;
    const int passes = (bits + 7) / 8;
    const int rb = (bits + passes - 1) / passes;
    uint64_t *ka = keys, *kb = keys_alt;
    uint32_t *va = vals, *vb = vals_alt;
    int flips = 0;
    for (int p = 0, shift = 0; p < passes; ++p, shift += rb) {
        switch (rb) {
        case 1: case 2: case 3: case 4:
            radix_pass<uint64_t, 4, true>(ka, va, kb, vb, n, shift, hist, scan_tmp, st, launches, n_gauss); break;
        case 5: radix_pass<uint64_t, 5, true>(ka, va, kb, vb, n, shift, hist, scan_tmp, st, launches, n_gauss); break;
        case 6: radix_pass<uint64_t, 6, true>(ka, va, kb, vb, n, shift, hist, scan_tmp, st, launches, n_gauss); break;
        case 7: radix_pass<uint64_t, 7, true>(ka, va, kb, vb, n, shift, hist, scan_tmp, st, launches, n_gauss); break;
        default: radix_pass<uint64_t, 8, true>(ka, va, kb, vb, n, shift, hist, scan_tmp, st, launches, n_gauss); break;
        }
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
        flips ^= 1;
    }
    return flips;
}

// Stable LSD sort of (keys, vals) on key bits [shift0, shift0 + bits): the
// fewest passes of at most 8 bits, with equal digits (at least 4 bits: the
// key bits above shift0 + bits must then be zero, as they are for every
// caller).  Uses the alt buffers; returns 1 if the result ended in the alt
// buffers.  n_dev: the count on the device, n its upper bound (radix_pass).
template <class K>
static int radix_sort(K *keys, uint32_t *vals, K *keys_alt, uint32_t *vals_alt, uint64_t n, int bits,
                      uint32_t *hist, uint32_t *scan_tmp, cudaStream_t st, int *launches, int shift0 = 0,
                      const uint32_t *n_dev = nullptr)
{
    if (n == 0 || bits <= 0) return 0;
    const int passes = (bits + 7) / 8;
    const int rb = (bits + passes - 1) / passes;
    K *ka = keys, *kb = keys_alt;
    uint32_t *va = vals, *vb = vals_alt;
    int flips = 0;
    for (int p = 0, shift = shift0; p < passes; ++p, shift += rb) {
        switch (rb) {
        case 1: case 2: case 3: case 4: radix_pass<K, 4>(ka, va, kb, vb, n, shift, hist, scan_tmp, st, launches, 0, n_dev); break;
        case 5: radix_pass<K, 5>(ka, va, kb, vb, n, shift, hist, scan_tmp, st, launches, 0, n_dev); break;
        case 6: radix_pass<K, 6>(ka, va, kb, vb, n, shift, hist, scan_tmp, st, launches, 0, n_dev); break;
        case 7: radix_pass<K, 7>(ka, va, kb, vb, n, shift, hist, scan_tmp, st, launches, 0, n_dev); break;
        default: radix_pass<K, 8>(ka, va, kb, vb, n, shift, hist, scan_tmp, st, launches, 0, n_dev); break;
        }
        K *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
        flips ^= 1;
    }
    return flips;
}

// -------------------------------------------------------------- binning
__global__ void valid_flags_kernel(const PixBox *__restrict__ boxes, uint64_t n, uint32_t *__restrict__ flags)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i < n) flags[i] = boxes[i].x0 >= 0 ? 1u : 0u;
}

__global__ void emit_events_kernel(const PixBox *__restrict__ boxes, const double *__restrict__ keys,
                                   const uint32_t *__restrict__ pos, uint64_t n, uint64_t *__restrict__ ev_key,
                                   uint32_t *__restrict__ ev_val)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n || boxes[i].x0 < 0) return;
    const uint32_t p = pos[i];
    ev_key[2 * p] = key_bits(keys[2 * i]);
    ev_key[2 * p + 1] = key_bits(keys[2 * i + 1]);
    ev_val[2 * p] = (uint32_t)(2 * i);
    ev_val[2 * p + 1] = (uint32_t)(2 * i + 1);
}

__device__ __forceinline__ void tile_rect(const PixBox &b, int TS, int &tx0, int &tx1, int &ty0, int &ty1)
{
    tx0 = b.x0 / TS; tx1 = b.x1 / TS; ty0 = b.y0 / TS; ty1 = b.y1 / TS;
}

// First sorted event of every cell (cell c holds [cell_ev[c], cell_ev[c + 1])):
// from the exclusive scan pos of the pairs' presence flags, cell c's events
// start at 2 pos[c n_gauss].
__global__ void cell_events_kernel(const uint32_t *__restrict__ pos, uint64_t n_gauss, int n_cells, uint32_t ne,
                                   uint32_t *__restrict__ cell_ev)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c > n_cells) return;
    cell_ev[c] = c < n_cells ? 2u * pos[(uint64_t)c * n_gauss] : ne;
}

// The depth prefix of a cell: its first ceil(E / 2^shift) sorted events, E
// the cell's events (shift = 0: all of them).  Sorted event e of cell `cell`
// lies in it when this holds.
__device__ __forceinline__ bool in_prefix(uint64_t e, uint32_t cell, const uint32_t *__restrict__ cell_ev, int shift)
{
    if (!shift) return true;
    const uint32_t c0 = cell_ev[cell], ec = cell_ev[cell + 1] - c0;
    return e - c0 < (((uint64_t)ec + (1u << shift) - 1u) >> shift);
}

__global__ void tile_counts_kernel(const uint32_t *__restrict__ ev_val, uint64_t ne,
                                   const PixBox *__restrict__ boxes, int TS, uint64_t n_gauss,
                                   const uint32_t *__restrict__ cell_ev, int shift, uint32_t *__restrict__ cnt)
{
    const uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const uint32_t ri = ev_val[e] >> 1;
    int tx0, tx1, ty0, ty1;
    tile_rect(boxes[ri], TS, tx0, tx1, ty0, ty1);
    cnt[e] = in_prefix(e, (uint32_t)(ri / n_gauss), cell_ev, shift) ? (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1))
                                                                      : 0u;
}

// *word = cnt[n - 1] before an in-place exclusive scan of cnt, then (add)
// the scan's last value: the total
__global__ void scan_last_kernel(const uint32_t *__restrict__ v, uint64_t n, uint32_t *__restrict__ word, int add,
                                 DevLen dl)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const uint32_t m = dev_len(dl, (uint32_t)n);
        *word = (add ? *word : 0u) + (m ? v[m - 1] : 0u);
    }
}

// The first phase's events as one index range: the prefix events of cell c
// are pref_start[c] .. pref_start[c + 1] - 1 (one block; *n_pre: their total)
__global__ void __launch_bounds__(SC_THREADS) prefix_ranges_kernel(const uint32_t *__restrict__ cell_ev, int n_cells,
                                                                   int shift, uint32_t *__restrict__ pref_start,
                                                                   uint32_t *__restrict__ n_pre)
{
    __shared__ uint32_t s_warp[32];
    uint32_t carry = 0;
    for (int c0 = 0; c0 < n_cells; c0 += SC_THREADS) {
        const int c = c0 + (int)threadIdx.x;
        uint32_t p = 0;
        if (c < n_cells) {
            const uint32_t ec = cell_ev[c + 1] - cell_ev[c];
            p = (uint32_t)(((uint64_t)ec + (1u << shift) - 1u) >> shift);
        }
        uint32_t total;
        const uint32_t first = carry + block_exclusive_scan(p, s_warp, total);
        if (c < n_cells) pref_start[c] = first;
        carry += total;
    }
    if (threadIdx.x == 0) {
        pref_start[n_cells] = carry;
        *n_pre = carry;
    }
}

// The prefix events' tile counts, in the compacted index i < *n_pre, and the
// sorted event each index stands for (evmap)
__global__ void prefix_counts_kernel(const uint32_t *__restrict__ ev_val, uint64_t ne,
                                     const PixBox *__restrict__ boxes, int TS, const uint32_t *__restrict__ cell_ev,
                                     const uint32_t *__restrict__ pref_start, int n_cells,
                                     const uint32_t *__restrict__ n_pre, uint32_t *__restrict__ cnt,
                                     uint32_t *__restrict__ evmap)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= ne || i >= *n_pre) return;
    int lo = 0, hi = n_cells;  // the cell c with pref_start[c] <= i < pref_start[c + 1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pref_start[mid] <= i) lo = mid; else hi = mid;
    }
    const uint32_t e = cell_ev[lo] + (uint32_t)(i - pref_start[lo]);
    int tx0, tx1, ty0, ty1;
    tile_rect(boxes[ev_val[e] >> 1], TS, tx0, tx1, ty0, ty1);
    cnt[i] = (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
    evmap[i] = e;
}

// Entry counts of the segments' full lists, as 2D difference marks per cell:
// each present pair adds 2 (its two events) at the corner of its tile
// rectangle and subtracts it past the right and the bottom edge (adding it
// back past both); marks past the grid's last column or row are dropped, as
// no prefix sum reaches them.  tot: [n_cells][n_tiles], zeroed first.  One
// block takes MARK_PAIRS pairs of one cell (blockIdx.y) and gathers their
// marks in shared memory (SMEM; else straight into tot).
constexpr int MARK_PAIRS = 16384;
constexpr int kMarkSmemTiles = 12288;  // 48 KB of shared marks
template <bool SMEM>
__global__ void __launch_bounds__(256) seg_marks_kernel(const PixBox *__restrict__ boxes, uint64_t n_gauss, int TS,
                                                        int ntx, int nty, uint32_t *__restrict__ tot)
{
    extern __shared__ uint32_t s_m[];
    const int n_tiles = ntx * nty;
    const uint64_t c = blockIdx.y, g0 = (uint64_t)blockIdx.x * MARK_PAIRS;
    const uint64_t g1 = min(g0 + (uint64_t)MARK_PAIRS, n_gauss);
    uint32_t *t = tot + c * (uint64_t)n_tiles;
    uint32_t *m = SMEM ? s_m : t;
    if (SMEM) {
        for (int i = threadIdx.x; i < n_tiles; i += blockDim.x) s_m[i] = 0u;
        __syncthreads();
    }
    const PixBox *bc = boxes + c * n_gauss;
    for (uint64_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
        const PixBox b = bc[g];
        if (b.x0 < 0) continue;
        int tx0, tx1, ty0, ty1;
        tile_rect(b, TS, tx0, tx1, ty0, ty1);
        const bool right = tx1 + 1 < ntx, below = ty1 + 1 < nty;
        atomicAdd(&m[ty0 * ntx + tx0], 2u);
        if (right) atomicAdd(&m[ty0 * ntx + tx1 + 1], 0u - 2u);
        if (below) {
            atomicAdd(&m[(ty1 + 1) * ntx + tx0], 0u - 2u);
            if (right) atomicAdd(&m[(ty1 + 1) * ntx + tx1 + 1], 2u);
        }
    }
    if (SMEM) {
        __syncthreads();
        for (int i = threadIdx.x; i < n_tiles; i += blockDim.x)
            if (s_m[i]) atomicAdd(&t[i], s_m[i]);
    }
}

// prefix sums of the marks (modulo 2^32) along each row (cols = 0: one
// thread per (cell, row)) or each column (cols = 1: per (cell, column))
__global__ void seg_prefix_kernel(uint32_t *__restrict__ tot, int n_cells, int ntx, int nty, int cols)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const int lines = cols ? ntx : nty, len = cols ? nty : ntx;
    if (i >= (uint64_t)n_cells * (uint64_t)lines) return;
    const uint64_t c = i / (uint64_t)lines;
    const int l = (int)(i % (uint64_t)lines);
    uint32_t *t = tot + c * (uint64_t)ntx * (uint64_t)nty;
    const int step = cols ? ntx : 1;
    uint32_t *p = t + (cols ? l : l * ntx);
    uint32_t run = 0;
    for (int k = 0; k < len; ++k, p += step) {
        run += *p;
        *p = run;
    }
}

// The second binning phase's input: the active segments as a bit mask
// (zeroed first), and per event the tiles of its box whose segment is active.
__global__ void active_mask_kernel(const uint32_t *__restrict__ active, const uint32_t *__restrict__ n_active,
                                   uint32_t *__restrict__ mask)
{
    const uint32_t na = *n_active;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < na; i += gridDim.x * blockDim.x)
        atomicOr(&mask[active[i] >> 5], 1u << (active[i] & 31u));
}

__device__ __forceinline__ bool seg_active(const uint32_t *__restrict__ mask, uint64_t seg)
{
    return (mask[seg >> 5] >> (seg & 31u)) & 1u;
}

// Per cell, a summed-area table of the active tiles ([n_cells][(nty + 1) x
// (ntx + 1)], the first row and column 0; sat zeroed first, then prefix sums
// along its rows and columns): the active tiles of any tile rectangle in four
// lookups.
__global__ void sat_fill_kernel(const uint32_t *__restrict__ mask, int n_cells, int ntx, int nty,
                                uint32_t *__restrict__ sat)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t n_tiles = (uint64_t)ntx * (uint64_t)nty;
    if (i >= (uint64_t)n_cells * n_tiles) return;
    const uint64_t c = i / n_tiles;
    const int t = (int)(i % n_tiles), y = t / ntx, x = t % ntx;
    if (seg_active(mask, i)) sat[c * (uint64_t)(ntx + 1) * (nty + 1) + (uint64_t)(y + 1) * (ntx + 1) + (x + 1)] = 1u;
}

__device__ __forceinline__ uint32_t sat_rect(const uint32_t *__restrict__ s, int w, int tx0, int tx1, int ty0, int ty1)
{
    return s[(ty1 + 1) * w + tx1 + 1] - s[ty0 * w + tx1 + 1] - s[(ty1 + 1) * w + tx0] + s[ty0 * w + tx0];
}

__global__ void events_if_active_kernel(const uint32_t *__restrict__ n_active, uint32_t ne, uint32_t *__restrict__ out)
{
    if (threadIdx.x == 0) *out = *n_active ? ne : 0u;
}

// (no segment active: nothing is written, and the scan reads nothing)
__global__ void masked_counts_kernel(const uint32_t *__restrict__ ev_val, uint64_t ne,
                                     const PixBox *__restrict__ boxes, int TS, int ntx, int nty, uint64_t n_gauss,
                                     const uint32_t *__restrict__ sat, const uint32_t *__restrict__ n_active,
                                     uint32_t *__restrict__ cnt)
{
    const uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (e >= ne || *n_active == 0) return;
    const uint32_t ri = ev_val[e] >> 1;
    int tx0, tx1, ty0, ty1;
    tile_rect(boxes[ri], TS, tx0, tx1, ty0, ty1);
    cnt[e] = sat_rect(sat + (ri / n_gauss) * (uint64_t)(ntx + 1) * (nty + 1), ntx + 1, tx0, tx1, ty0, ty1);
}

// Entry keys: (tile << cb) | cell when cb >= 0 (the entries of one cell are
// contiguous and in key order, so a stable sort on the tile bits alone leaves
// every (cell, tile) segment contiguous and in key order), else the segment
// cell * n_tiles + tile.
__device__ __forceinline__ uint32_t entry_key(uint32_t cell, uint32_t tile, int cb, int n_tiles)
{
    return cb >= 0 ? ((tile << cb) | cell) : cell * (uint32_t)n_tiles + tile;
}
__device__ __forceinline__ uint32_t entry_segment(uint32_t key, int cb, int n_tiles)
{
    return cb >= 0 ? (key & ((1u << cb) - 1u)) * (uint32_t)n_tiles + (key >> cb) : key;
}

// Each warp owns 32 consecutive events, whose entries form one contiguous
// range of the output (off is their exclusive scan).  The lanes stride over
// that range, so every store instruction writes 32 consecutive words; each
// lane finds the event of its entry by a binary search over the warp's 32
// offsets (shuffles).  Launch with a multiple of 32 threads per block.
// With evmap, the items are the first phase's prefix events in their
// compacted index (*n_map of them, evmap: the sorted event of each), else the
// sorted events themselves.
__global__ void emit_entries_kernel(const uint32_t *__restrict__ ev_val, uint64_t ne,
                                    const PixBox *__restrict__ boxes, int TS, int ntx, int n_tiles, int cb,
                                    uint64_t n_gauss, const uint32_t *__restrict__ evmap,
                                    const uint32_t *__restrict__ n_map, const uint32_t *__restrict__ off,
                                    uint32_t *__restrict__ ent_seg, uint32_t *__restrict__ ent_ev)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    if (evmap) ne = min(ne, (uint64_t)*n_map);
    const uint64_t e0 = ((blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5) * 32u;
    if (e0 >= ne) return;  // uniform across the warp
    const uint64_t item = e0 + (uint64_t)lane;
    uint32_t myoff = 0xffffffffu, myend = 0, cell = 0, myev = 0;
    int tx0 = 0, ty0 = 0, tw = 1;
    if (item < ne) {
        myev = evmap ? evmap[item] : (uint32_t)item;
        const uint32_t ri = ev_val[myev] >> 1;
        cell = (uint32_t)(ri / n_gauss);
        int tx1, ty1;
        tile_rect(boxes[ri], TS, tx0, tx1, ty0, ty1);
        tw = tx1 - tx0 + 1;
        myoff = off[item];
        myend = myoff + (uint32_t)(tw * (ty1 - ty0 + 1));
    }
    const uint32_t start = __shfl_sync(full, myoff, 0);
    uint32_t end = myend;
#pragma unroll
    for (int d = 16; d; d >>= 1) end = max(end, __shfl_xor_sync(full, end, d));
    for (uint32_t b = start; b < end; b += 32u) {
        const uint32_t o = b + (uint32_t)lane;
        int j = 0;  // last lane whose offset is <= o (offsets ascend; idle lanes hold ~0)
#pragma unroll
        for (int step = 16; step; step >>= 1) {
            const int cand = j + step;
            const uint32_t oc = __shfl_sync(full, myoff, cand & 31);
            if (cand < 32 && oc <= o) j = cand;
        }
        const uint32_t oj = __shfl_sync(full, myoff, j);
        const uint32_t cj = __shfl_sync(full, cell, j);
        const int x0 = __shfl_sync(full, tx0, j), y0 = __shfl_sync(full, ty0, j), w = __shfl_sync(full, tw, j);
        const uint32_t evj = __shfl_sync(full, myev, j);
        if (o < end) {
            const uint32_t k = o - oj;
            const uint32_t ty = (uint32_t)y0 + k / (uint32_t)w, tx = (uint32_t)x0 + k % (uint32_t)w;
            ent_seg[o] = entry_key(cj, ty * (uint32_t)ntx + tx, cb, n_tiles);
            ent_ev[o] = evj;
        }
    }
}

// The second phase's entries: each event writes, one thread per event, its
// tiles whose segment is active, from off[e] on (off: the exclusive scan of
// masked_counts_kernel's counts).
__global__ void masked_emit_kernel(const uint32_t *__restrict__ ev_val, uint64_t ne, const PixBox *__restrict__ boxes,
                                   int TS, int ntx, int nty, int cb, uint64_t n_gauss,
                                   const uint32_t *__restrict__ mask, const uint32_t *__restrict__ sat,
                                   const uint32_t *__restrict__ n_active, const uint32_t *__restrict__ off,
                                   uint32_t *__restrict__ ent_seg, uint32_t *__restrict__ ent_ev)
{
    const uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (e >= ne || *n_active == 0) return;
    const int n_tiles = ntx * nty;
    const uint32_t ri = ev_val[e] >> 1;
    const uint32_t cell = (uint32_t)(ri / n_gauss);
    const uint64_t s0 = (uint64_t)cell * (uint64_t)n_tiles;
    int tx0, tx1, ty0, ty1;
    tile_rect(boxes[ri], TS, tx0, tx1, ty0, ty1);
    if (!sat_rect(sat + cell * (uint64_t)(ntx + 1) * (nty + 1), ntx + 1, tx0, tx1, ty0, ty1)) return;
    uint32_t j = off[e];
    for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx) {
            const uint32_t tile = (uint32_t)(ty * ntx + tx);
            if (seg_active(mask, s0 + tile)) {
                ent_seg[j] = entry_key(cell, tile, cb, n_tiles);
                ent_ev[j] = (uint32_t)e;
                ++j;
            }
        }
}

// key = ~length so that an ascending stable sort puts the longest first
__global__ void seg_len_kernel(const uint32_t *__restrict__ start, const uint32_t *__restrict__ end, uint64_t n,
                               uint32_t *__restrict__ key, uint32_t *__restrict__ val)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    key[i] = ~(end[i] - start[i]);
    val[i] = (uint32_t)i;
}

__global__ void seg_bounds_kernel(const uint32_t *__restrict__ key, uint64_t n, int cb, int n_tiles,
                                  uint32_t *__restrict__ start, uint32_t *__restrict__ end,
                                  const uint32_t *__restrict__ n_dev)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (n_dev && *n_dev < n) n = *n_dev;
    if (i >= n) return;
    const uint32_t k = key[i];
    const uint32_t s = entry_segment(k, cb, n_tiles);
    if (i == 0 || key[i - 1] != k) start[s] = (uint32_t)i;
    if (i == n - 1 || key[i + 1] != k) end[s] = (uint32_t)(i + 1);
}

// Packed keys come out of the tile sort in ascending order (tile, then cell),
// so each segment's range is found by two binary searches over the keys.
__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t *__restrict__ a, uint32_t n, uint32_t v)
{
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}
__global__ void seg_bounds_search_kernel(const uint32_t *__restrict__ key, uint32_t n, int cb, int n_cells,
                                         int n_tiles, uint32_t *__restrict__ start, uint32_t *__restrict__ end,
                                         const uint32_t *__restrict__ n_dev)
{
    const uint64_t sg = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (n_dev && *n_dev < n) n = *n_dev;
    if (sg >= (uint64_t)n_cells * (uint64_t)n_tiles) return;
    const uint32_t cell = (uint32_t)(sg / (uint64_t)n_tiles), tile = (uint32_t)(sg % (uint64_t)n_tiles);
    const uint32_t k = (tile << cb) | cell;
    const uint32_t b = lower_bound_u32(key, n, k);
    start[sg] = b;
    end[sg] = (b < n && key[b] == k) ? (k == 0xffffffffu ? n : lower_bound_u32(key, n, k + 1u)) : b;
}

__global__ void iota_kernel(uint32_t *__restrict__ p, uint64_t n)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i < n) p[i] = (uint32_t)i;
}

static inline unsigned blocks_for(uint64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// The entries' stable sort by tile (packed keys: the tile bits above cb) or
// by segment, then the segment bounds; n_dev: the entries' count when it is
// known on the device only (n_entries bounds it).  Returns the buffer
// holding the result.
static int sort_entries(const BinArgs &a, bool packed, int cb, int tb, const uint32_t *n_dev, cudaStream_t st,
                        int *launches)
{
    const int T = 256;
    int h;
    if (packed) {
        h = radix_sort<uint32_t>(a.ent_seg[0], a.ent_ev[0], a.ent_seg[1], a.ent_ev[1], a.n_entries, tb, a.hist,
                                 a.scan_tmp, st, launches, cb, n_dev);
    } else {
        int bits = 0;
        while ((1ull << bits) < a.n_segments) ++bits;
        h = radix_sort<uint32_t>(a.ent_seg[0], a.ent_ev[0], a.ent_seg[1], a.ent_ev[1], a.n_entries, bits, a.hist,
                                 a.scan_tmp, st, launches, 0, n_dev);
    }
    const uint32_t *keys = a.ent_seg[h];
    if (packed) {
        seg_bounds_search_kernel<<<blocks_for(a.n_segments, T), T, 0, st>>>(keys, (uint32_t)a.n_entries, cb, a.n_cells,
                                                                            a.n_tiles, a.seg_start, a.seg_end, n_dev);
        ++*launches;
    } else {
        cudaMemsetAsync(a.seg_start, 0, sizeof(uint32_t) * a.n_segments, st);
        cudaMemsetAsync(a.seg_end, 0, sizeof(uint32_t) * a.n_segments, st);
        if (a.n_entries) {
            seg_bounds_kernel<<<blocks_for(a.n_entries, T), T, 0, st>>>(keys, a.n_entries, -1, a.n_tiles, a.seg_start,
                                                                         a.seg_end, n_dev);
            ++*launches;
        }
    }
    return h;
}

int run_binning(const BinArgs &a, BinOut &o, cudaStream_t st, int *launches)
{
    const int T = 256;
    // 1. compact the pairs that reach the image
    valid_flags_kernel<<<blocks_for(a.n_pairs, T), T, 0, st>>>(a.boxes, a.n_pairs, a.u32_a);
    ++*launches;
    exclusive_scan(a.u32_a, a.u32_a, a.n_pairs, a.scan_tmp, st, launches);
    // 2. events
    emit_events_kernel<<<blocks_for(a.n_pairs, T), T, 0, st>>>(a.boxes, a.keys, a.u32_a, a.n_pairs, a.ev_key[0],
                                                                 a.ev_val[0]);
    ++*launches;
    const uint64_t ne = a.n_events;
    o.seg_total = nullptr;
    if (ne == 0) {
        o.ev_key = a.ev_key[0];
        o.ev_val = a.ev_val[0];
        o.ent_seg = a.ent_seg[0];
        o.ent_ev = a.ent_ev[0];
        cudaMemsetAsync(a.seg_start, 0, sizeof(uint32_t) * a.n_segments, st);
        cudaMemsetAsync(a.seg_end, 0, sizeof(uint32_t) * a.n_segments, st);
        iota_kernel<<<blocks_for(a.n_segments, T), T, 0, st>>>(a.seg_v[0], a.n_segments);
        ++*launches;
        o.seg_order = a.seg_v[0];
        return cudaGetLastError() == cudaSuccess ? 0 : 1;
    }
    // the first phase bins only each cell's depth prefix (see in_prefix): the
    // cells' event ranges, while the presence scan is at hand (also wanted by
    // the renderer's stop histogram when there is one phase)
    const bool prefix = a.prefix_shift > 0 && a.cell_ev;
    if (a.cell_ev) {
        cell_events_kernel<<<blocks_for((uint64_t)a.n_cells + 1, T), T, 0, st>>>(a.u32_a, a.n_gauss, a.n_cells,
                                                                                  (uint32_t)ne, a.cell_ev);
        ++*launches;
    }
    // 3. sort by key bits, then stably by cell
    int f = radix_sort<uint64_t>(a.ev_key[0], a.ev_val[0], a.ev_key[1], a.ev_val[1], ne, 64, a.hist, a.scan_tmp,
                                 st, launches);
    uint64_t *evk = a.ev_key[f];
    uint32_t *evv = a.ev_val[f];
    if (a.n_cells > 1) {
        // stably by cell, the digits taken from the pair index in the value
        int bits = 0;
        while ((1ull << bits) < (uint64_t)a.n_cells) ++bits;
        const int g = radix_sort_cells(evk, evv, a.ev_key[f ^ 1], a.ev_val[f ^ 1], ne, bits, a.n_gauss, a.hist,
                                       a.scan_tmp, st, launches);
        evk = a.ev_key[f ^ g];
        evv = a.ev_val[f ^ g];
    }
    o.ev_key = evk;
    o.ev_val = evv;
    const int nty = a.n_tiles / a.ntx;
    if (prefix) {
        // the lengths of the segments' full lists
        cudaMemsetAsync(a.seg_total, 0, sizeof(uint32_t) * a.n_segments, st);
        const dim3 mg((unsigned)((a.n_gauss + MARK_PAIRS - 1) / MARK_PAIRS), (unsigned)a.n_cells);
        if (a.n_tiles <= kMarkSmemTiles)
            seg_marks_kernel<true><<<mg, T, sizeof(uint32_t) * a.n_tiles, st>>>(a.boxes, a.n_gauss, a.TS, a.ntx, nty,
                                                                                 a.seg_total);
        else
            seg_marks_kernel<false><<<mg, T, 0, st>>>(a.boxes, a.n_gauss, a.TS, a.ntx, nty, a.seg_total);
        seg_prefix_kernel<<<blocks_for((uint64_t)a.n_cells * nty, T), T, 0, st>>>(a.seg_total, a.n_cells, a.ntx, nty, 0);
        seg_prefix_kernel<<<blocks_for((uint64_t)a.n_cells * a.ntx, T), T, 0, st>>>(a.seg_total, a.n_cells, a.ntx, nty,
                                                                                    1);
        *launches += 3;
        o.seg_total = a.seg_total;
    }
    // 4. entries per tile.  The first phase counts its prefix events alone,
    // in their compacted index (words[2] of them; evmap: the sorted event of
    // each), and the count of its entries is then known on the device only.
    const uint32_t *n_dev = nullptr, *evmap = nullptr;
    if (prefix) {
        prefix_ranges_kernel<<<1, SC_THREADS, 0, st>>>(a.cell_ev, a.n_cells, a.prefix_shift, a.pref_start,
                                                       a.words + 2);
        prefix_counts_kernel<<<blocks_for(ne, T), T, 0, st>>>(evv, ne, a.boxes, a.TS, a.cell_ev, a.pref_start,
                                                              a.n_cells, a.words + 2, a.u32_a, a.u32_b);
        const DevLen dl{a.words + 2, 1, 1};
        scan_last_kernel<<<1, 32, 0, st>>>(a.u32_a, ne, a.words, 0, dl);
        exclusive_scan_dl(a.u32_a, a.u32_a, ne, a.scan_tmp, st, launches, dl);
        scan_last_kernel<<<1, 32, 0, st>>>(a.u32_a, ne, a.words, 1, dl);
        *launches += 4;
        n_dev = a.words;
        evmap = a.u32_b;
    } else {
        tile_counts_kernel<<<blocks_for(ne, T), T, 0, st>>>(evv, ne, a.boxes, a.TS, a.n_gauss, a.cell_ev, 0, a.u32_a);
        ++*launches;
        exclusive_scan(a.u32_a, a.u32_a, ne, a.scan_tmp, st, launches);
    }
    // entry keys: tile bits above cell bits when both fit in 32 bits
    int cb = 0, tb = 0;
    while ((1ull << cb) < (uint64_t)a.n_cells) ++cb;
    while ((1ull << tb) < (uint64_t)a.n_tiles) ++tb;
    if (tb == 0) tb = 1;
    const bool packed = cb + tb <= 32;
    emit_entries_kernel<<<blocks_for(ne, T), T, 0, st>>>(evv, ne, a.boxes, a.TS, a.ntx, a.n_tiles, packed ? cb : -1,
                                                          a.n_gauss, evmap, prefix ? a.words + 2 : nullptr, a.u32_a,
                                                          a.ent_seg[0],
                                                          a.ent_ev[0]);
    ++*launches;
    // 5-6. stable sort by tile, segment bounds
    const int h = sort_entries(a, packed, cb, tb, n_dev, st, launches);
    o.ent_seg = a.ent_seg[h];
    o.ent_ev = a.ent_ev[h];
    // 7. schedule: segments by decreasing length (load balance of the render)
    seg_len_kernel<<<blocks_for(a.n_segments, T), T, 0, st>>>(a.seg_start, a.seg_end, a.n_segments, a.seg_k[0],
                                                               a.seg_v[0]);
    ++*launches;
    int q = radix_sort<uint32_t>(a.seg_k[0], a.seg_v[0], a.seg_k[1], a.seg_v[1], a.n_segments, 32, a.hist,
                                 a.scan_tmp, st, launches);
    o.seg_order = a.seg_v[q];
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

// keys ~len[seg] of the listed segments, so that an ascending sort puts the
// longest first
__global__ void active_keys_kernel(const uint32_t *__restrict__ active, const uint32_t *__restrict__ n_active,
                                   const uint32_t *__restrict__ len, uint32_t *__restrict__ key,
                                   uint32_t *__restrict__ val)
{
    const uint32_t na = *n_active;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < na; i += gridDim.x * blockDim.x) {
        key[i] = ~len[active[i]];
        val[i] = active[i];
    }
}

int run_rebin(const BinArgs &a, const BinOut &first, const uint32_t *active, const uint32_t *n_active, BinOut &o,
              cudaStream_t st, int *launches)
{
    const int T = 256;
    const uint64_t ne = a.n_events;
    o = first;
    if (ne == 0) return 0;
    const int nty = a.n_tiles / a.ntx;
    cudaMemsetAsync(a.mask, 0, sizeof(uint32_t) * ((a.n_segments + 31) / 32), st);
    cudaMemsetAsync(a.sat, 0, sizeof(uint32_t) * (size_t)a.n_cells * (a.ntx + 1) * (nty + 1), st);
    const uint64_t mg = blocks_for(a.n_segments, T);
    active_mask_kernel<<<(unsigned)(mg < kDevGrid ? mg : kDevGrid), T, 0, st>>>(active, n_active, a.mask);
    sat_fill_kernel<<<blocks_for(a.n_segments, T), T, 0, st>>>(a.mask, a.n_cells, a.ntx, nty, a.sat);
    seg_prefix_kernel<<<blocks_for((uint64_t)a.n_cells * (nty + 1), T), T, 0, st>>>(a.sat, a.n_cells, a.ntx + 1,
                                                                                    nty + 1, 0);
    seg_prefix_kernel<<<blocks_for((uint64_t)a.n_cells * (a.ntx + 1), T), T, 0, st>>>(a.sat, a.n_cells, a.ntx + 1,
                                                                                      nty + 1, 1);
    // the events' count, or 0 when no segment is active (nothing is then read)
    events_if_active_kernel<<<1, 32, 0, st>>>(n_active, (uint32_t)ne, a.words + 3);
    const DevLen dl{a.words + 3, 1, 1};
    masked_counts_kernel<<<blocks_for(ne, T), T, 0, st>>>(first.ev_val, ne, a.boxes, a.TS, a.ntx, nty, a.n_gauss,
                                                           a.sat, n_active, a.u32_a);
    scan_last_kernel<<<1, 32, 0, st>>>(a.u32_a, ne, a.words + 1, 0, dl);
    *launches += 7;
    exclusive_scan_dl(a.u32_a, a.u32_a, ne, a.scan_tmp, st, launches, dl);
    scan_last_kernel<<<1, 32, 0, st>>>(a.u32_a, ne, a.words + 1, 1, dl);
    int cb = 0, tb = 0;
    while ((1ull << cb) < (uint64_t)a.n_cells) ++cb;
    while ((1ull << tb) < (uint64_t)a.n_tiles) ++tb;
    if (tb == 0) tb = 1;
    const bool packed = cb + tb <= 32;
    masked_emit_kernel<<<blocks_for(ne, T), T, 0, st>>>(first.ev_val, ne, a.boxes, a.TS, a.ntx, nty, packed ? cb : -1,
                                                         a.n_gauss, a.mask, a.sat, n_active, a.u32_a, a.ent_seg[0],
                                                         a.ent_ev[0]);
    *launches += 2;
    const int h = sort_entries(a, packed, cb, tb, a.words + 1, st, launches);
    o.ent_seg = a.ent_seg[h];
    o.ent_ev = a.ent_ev[h];
    // the active segments, longest full list first (the first phase's order
    // is no longer needed: its buffers are reused)
    active_keys_kernel<<<(unsigned)(mg < kDevGrid ? mg : kDevGrid), T, 0, st>>>(active, n_active, a.seg_total,
                                                                               a.seg_k[0], a.seg_v[0]);
    ++*launches;
    const int q = radix_sort<uint32_t>(a.seg_k[0], a.seg_v[0], a.seg_k[1], a.seg_v[1], a.n_segments, 32, a.hist,
                                       a.scan_tmp, st, launches, 0, n_active);
    o.seg_order = a.seg_v[q];
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

// ------------------------------------------------------------ windowed rounds
__global__ void set_u32_kernel(uint32_t *p, uint32_t v) { *p = v; }

// For each active segment, the lower endpoints among its first `window`
// entries: every pair not yet claimed (state 0 -> 1) is appended to work.
// One block per active segment (grid-stride over the active list).
__global__ void __launch_bounds__(256) demand_kernel(const uint32_t *__restrict__ active,
                                                     const uint32_t *__restrict__ n_active,
                                                     const uint32_t *__restrict__ seg_start,
                                                     const uint32_t *__restrict__ seg_end,
                                                     const uint32_t *__restrict__ ent_ev,
                                                     const uint32_t *__restrict__ ev_val, uint32_t window,
                                                     uint32_t *__restrict__ state, uint32_t *__restrict__ work,
                                                     uint32_t *__restrict__ count)
{
    const uint32_t na = *n_active;
    const int lane = threadIdx.x & 31;
    for (uint32_t a = blockIdx.x; a < na; a += gridDim.x) {
        const uint32_t seg = active[a];
        const uint32_t b0 = seg_start[seg], b1 = seg_end[seg];
        const uint32_t e1 = (b1 - b0 > window) ? b0 + window : b1;
        for (uint32_t i0 = b0; i0 < e1; i0 += blockDim.x) {
            const uint32_t i = i0 + threadIdx.x;
            bool claim = false;
            uint32_t p = 0;
            if (i < e1) {
                const uint32_t v = ev_val[ent_ev[i]];
                p = v >> 1;
                claim = !(v & 1u) && state[p] == 0u && atomicCAS(&state[p], 0u, 1u) == 0u;
            }
            const unsigned m = __ballot_sync(0xffffffffu, claim);
            if (m) {
                const int leader = __ffs(m) - 1;
                uint32_t at = 0;
                if (lane == leader) at = atomicAdd(count, (uint32_t)__popc(m));
                at = __shfl_sync(0xffffffffu, at, leader);
                if (claim) work[at + __popc(m & ((1u << lane) - 1u))] = p;
            }
        }
    }
}

void launch_set_u32(uint32_t *p, uint32_t v, cudaStream_t st) { set_u32_kernel<<<1, 1, 0, st>>>(p, v); }

void launch_demand(const uint32_t *active, const uint32_t *n_active, uint32_t max_active, const uint32_t *seg_start,
                   const uint32_t *seg_end, const uint32_t *ent_ev, const uint32_t *ev_val, uint32_t window,
                   uint32_t *state, uint32_t *work, uint32_t *count, cudaStream_t st)
{
    unsigned grid = max_active < 152u * 16u ? max_active : 152u * 16u;
    if (grid == 0) grid = 1;
    demand_kernel<<<grid, 256, 0, st>>>(active, n_active, seg_start, seg_end, ent_ev, ev_val, window, state, work,
                                        count);
}

}  // namespace ar
