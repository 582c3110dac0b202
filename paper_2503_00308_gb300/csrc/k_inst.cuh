// k_inst.cuh -- instantiation of the per-M kernels; included once per M by
// k_m1.cu, k_m4.cu, k_m6.cu with AR_M defined.
#include "ar_launch.h"
#include "k_prep.cuh"
#include "k_render.cuh"

#define AR_CAT2(a, b) a##b
#define AR_CAT(a, b) AR_CAT2(a, b)

namespace ar {

size_t AR_CAT(cell_data_bytes_m, AR_M)() { return sizeof(CellData<AR_M>); }
int AR_CAT(rec_width_m, AR_M)() { return Rec<AR_M>::WIDTH; }
int AR_CAT(rec_scalar_offset_m, AR_M)() { return Rec<AR_M>::SC; }

int AR_CAT(launch_cell_prep_m, AR_M)(const double *lo, const double *hi, const CallConst &cc, void *cells,
                                     cudaStream_t st)
{
    const int T = 64;
    cell_prep_kernel<AR_M><<<(cc.n_cells + T - 1) / T, T, 0, st>>>(lo, hi, cc, (CellData<AR_M> *)cells);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int AR_CAT(launch_record_prep_m, AR_M)(const double *vN, const void *gp,
                                       const CallConst &cc, const void *cells, int TS, float *recs,
                                       PixBox *boxes, double *keys, unsigned long long *counters,
                                       cudaStream_t st, uint32_t *list, uint32_t *count)
{
    const int T = 128;
    const CellData<AR_M> *cd = (const CellData<AR_M> *)cells;
    const unsigned gb = (unsigned)((cc.n_gauss + T - 1) / T);
    // all cells of a range of Gaussians together (their vN rows stay in L2),
    // where the grid's y can hold the Gaussian blocks
    const int cf = gb <= 65535u ? 1 : 0;
    const dim3 grid = cf ? dim3((unsigned)cc.n_cells, gb) : dim3(gb, (unsigned)cc.n_cells);
    // decision part only: the value parts are built by the renderer on demand
    if (!list) {
        record_prep_kernel<AR_M, float, false><<<grid, T, 0, st>>>(vN, (const GParam *)gp, cc, cd, TS, recs, boxes,
                                                                   keys, counters, cf);
        return cudaGetLastError() == cudaSuccess ? 0 : 1;
    }
    if (cudaMemsetAsync(count, 0, sizeof(uint32_t), st) != cudaSuccess) return 1;
    cull_kernel<AR_M><<<grid, T, 0, st>>>(vN, (const GParam *)gp, cc, cd, boxes, list, count, cf);
    const uint64_t pairs = (uint64_t)cc.n_gauss * (uint64_t)cc.n_cells;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t lg = (pairs + T - 1) / T;
    if (lg > (uint64_t)sms * 32u) lg = (uint64_t)sms * 32u;
    record_prep_list_kernel<AR_M, float, false><<<(unsigned)(lg ? lg : 1), T, 0, st>>>(
        vN, (const GParam *)gp, cc, cd, TS, recs, boxes, keys, counters, list, count);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int AR_CAT(launch_record_prep64_m, AR_M)(const double *vN, const void *gp,
                                         const CallConst &cc, const void *cells, int TS, double *recs,
                                         PixBox *boxes, double *keys, unsigned long long *counters,
                                         cudaStream_t st)
{
    const int T = 128;
    dim3 grid((unsigned)((cc.n_gauss + T - 1) / T), (unsigned)cc.n_cells);
    record_prep_kernel<AR_M, double><<<grid, T, 0, st>>>(vN, (const GParam *)gp, cc, (const CellData<AR_M> *)cells,
                                                         TS, recs, boxes, keys, counters, 0);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

template <int TS>
static int launch_render_plain_ts(const RenderLaunch &a, cudaStream_t st)
{
    const uint32_t nseg = (uint32_t)a.n_cells * (uint32_t)a.n_tiles;
    render_plain_kernel<AR_M, TS, 32><<<nseg, TS * TS, 0, st>>>(a.recs64, a.boxes, a.seg_start, a.seg_end, a.ent_ev,
                                                                a.ev_val, a.ev_key, a.W, a.H, a.ntx, a.n_tiles,
                                                                a.n_gauss, a.out_lo, a.out_hi);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int AR_CAT(launch_render_plain_m, AR_M)(int TS, const RenderLaunch &a, cudaStream_t st)
{
    return TS == 16 ? launch_render_plain_ts<16>(a, st) : launch_render_plain_ts<8>(a, st);
}

template <int TS, bool REL, bool F64, int CH = 16>
static int launch_render_ts(const RenderLaunch &a, cudaStream_t st)
{
    // double-buffered chunks of CH events (16 unless the autotuner picks 8 or
    // 32 for the FP32 sweep at tile 16: the exit vote, taken once per chunk,
    // stops a tile sooner with short chunks, while long chunks take fewer
    // barriers) and a ring of 4 (rings of 3-8 measured: 4 keeps the ring's
    // shared memory small)
    constexpr int RING = 4;
    typedef RenderShape<TS, F64> SH;
    typedef RenderSmem<AR_M, TS, CH, RING, SH::NTH, SH::NBUF> SM;
    auto kern = render_kernel<AR_M, TS, CH, RING, REL, F64>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::BYTES) != cudaSuccess)
        return 1;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SH::NTH, SM::BYTES) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const uint32_t nseg = (uint32_t)a.n_cells * (uint32_t)a.n_tiles;
    // work items: segments, or for the FP64 instance (segment, group of 32 pixels)
    const uint64_t items = (uint64_t)nseg * (F64 ? (uint64_t)(TS * TS / 32) : 1u);
    uint32_t grid = (uint32_t)(sms * per_sm);
    if (grid > items) grid = (uint32_t)items;
    // direct launches (a.direct: the active list holds all nseg segments) take
    // one CTA per segment
    if (a.direct) grid = nseg;
    if (cudaMemsetAsync(a.work, 0, sizeof(unsigned int), st) != cudaSuccess) return 1;
    kern<<<grid, SH::NTH, SM::BYTES, st>>>(a.recs, a.boxes, a.seg_start, a.seg_end, a.seg_total, a.cell_ev,
                                           a.active, a.n_active,
                                           a.window,
                                           a.next_active, a.n_next, a.precise, a.n_precise, a.precise_mask, a.sweep_hist,
                                           a.ent_ev, a.ev_val,
                                           a.ev_key, a.W, a.H, a.ntx, a.n_tiles, a.n_gauss, a.k_open, a.fp64_dev, a.out_lo,
                                           a.out_hi, a.counters, a.work, a.direct);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int AR_CAT(launch_record_build_m, AR_M)(const double *vN, const CallConst &cc, const void *cells, int64_t n_gauss,
                                        const uint32_t *work, const uint32_t *count, float *recs,
                                        unsigned long long *counters, uint32_t *split_list, uint32_t *split_count,
                                        uint32_t list_cap, uint32_t *khigh_count, cudaStream_t st)
{
    auto kern = record_build_kernel<AR_M>;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
    kern<<<sms * per_sm, 128, 0, st>>>(vN, cc.fx, cc.fy, cc.cx, cc.cy, (const CellData<AR_M> *)cells, n_gauss, work,
                                       count, recs, counters, split_list, split_count, list_cap, khigh_count);
    if (cudaGetLastError() != cudaSuccess) return 1;
    // the deferred pairs (the counts stay on the device): splits one warp
    // each, high orders one thread each, grid-stride
    split_build_kernel<AR_M><<<sms, 128, 0, st>>>(vN, cc.fx, cc.fy, cc.cx, cc.cy, (const CellData<AR_M> *)cells,
                                                 n_gauss, split_list, split_count, recs, counters);
    if (cudaGetLastError() != cudaSuccess) return 1;
    auto kh = khigh_build_kernel<AR_M>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kh, 128, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
    kh<<<sms * per_sm, 128, 0, st>>>(vN, cc.fx, cc.fy, cc.cx, cc.cy, (const CellData<AR_M> *)cells, n_gauss,
                                     split_list, list_cap, khigh_count, recs, counters);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int AR_CAT(launch_debug_alpha_m, AR_M)(const float *recs, int n, const int64_t *gi, const int32_t *px,
                                       const int32_t *py, int precision, float fp64_dev, double *out,
                                       cudaStream_t st)
{
    debug_alpha_kernel<AR_M><<<(n + 63) / 64, 64, 0, st>>>(recs, n, gi, px, py, precision, fp64_dev, out);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int AR_CAT(launch_render_m, AR_M)(int TS, const RenderLaunch &a, cudaStream_t st)
{
    if (a.f64) {
        if (a.rel) return TS == 16 ? launch_render_ts<16, true, true>(a, st) : launch_render_ts<8, true, true>(a, st);
        return TS == 16 ? launch_render_ts<16, false, true>(a, st) : launch_render_ts<8, false, true>(a, st);
    }
    if (TS == 8) return a.rel ? launch_render_ts<8, true, false>(a, st) : launch_render_ts<8, false, false>(a, st);
    if (a.ch == 8) return a.rel ? launch_render_ts<16, true, false, 8>(a, st) : launch_render_ts<16, false, false, 8>(a, st);
    if (a.ch == 32)
        return a.rel ? launch_render_ts<16, true, false, 32>(a, st) : launch_render_ts<16, false, false, 32>(a, st);
    return a.rel ? launch_render_ts<16, true, false>(a, st) : launch_render_ts<16, false, false>(a, st);
}

}  // namespace ar
