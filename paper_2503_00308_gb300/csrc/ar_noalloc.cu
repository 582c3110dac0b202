// ar_noalloc.cu -- ar_render_abstract_noalloc: the abstract render with every
// per-call buffer carved from one fixed device array, so that the call itself
// never allocates device or host memory.
//
// Who needs it: callers that must not allocate while they run -- a real-time
// control loop or an embedded verifier that sizes all of its memory up front
// and treats a late cudaMalloc as a failure, or a host that shares the GPU
// under a strict memory budget where cudaMalloc/cudaFree would synchronise the
// device or fail unpredictably.  ar_render_abstract grows a per-scene
// workspace with cudaMalloc; this variant instead uses a 64 MiB array that is
// part of the library image (every GPU that loads libar reserves it until the
// process exits) and rejects requests whose buffers do not fit in it.
//
// The kernels and their launchers are the ones ar_render_abstract uses; only
// the placement of their buffers differs.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "ar.h"
#include "ar_bin.h"
#include "ar_common.cuh"
#include "ar_host.h"
#include "ar_launch.h"

namespace ar {

constexpr size_t kNoallocScratchBytes = size_t(64) << 20;  // the stated maximum: 64 MiB
constexpr int kMaxDevices = 64;

// The scratch array.  In host code `g_noalloc_scratch` names a host-side
// stand-in, not device memory: kernels must be given the address that
// cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of the scratch array on the current device, looked up on
// every call (with that device current) so that no address outlives a device
// reset or a re-created context.  Once the library's module is loaded on the
// device the lookup allocates nothing; the first call on a device may load
// it, which is the set-up the first call does.
static int scratch_base(int device, unsigned char **out)
{
    if (device < 0 || device >= kMaxDevices) return set_last_error(AR_EDEVICE, "device index out of range");
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return set_last_error(AR_EDEVICE, "cudaGetSymbolAddress of the no-allocation scratch array failed");
    }
    *out = (unsigned char *)p;
    return AR_OK;
}

// Bump allocator over the scratch array (256-byte alignment).
struct Arena {
    unsigned char *base;
    size_t used = 0;
    bool over = false;
    template <class T> T *take(size_t count)
    {
        size_t off = (used + 255) & ~size_t(255);
        size_t bytes = count * sizeof(T);
        if (off + bytes > kNoallocScratchBytes) {
            over = true;
            return nullptr;
        }
        used = off + bytes;
        return (T *)(base + off);
    }
};

static int too_big(const char *what, size_t used)
{
    static thread_local char msg[256];
    snprintf(msg, sizeof msg,
             "ar_render_abstract_noalloc: %s need more than the %zu MiB scratch (at least %zu bytes); "
             "use fewer cells, Gaussians or pixels per call, or ar_render_abstract",
             what, kNoallocScratchBytes >> 20, used);
    return set_last_error(AR_ENOMEM, msg);
}

}  // namespace ar

using namespace ar;

#define NA_CK(call)                                                                   \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) return set_last_error(AR_EDEVICE, cudaGetErrorString(e_)); \
    } while (0)

int ar_render_abstract_noalloc(ar_scene *s, const ar_intrinsics *in, const ar_nominal_pose *pose,
                               const ar_pose_box *cells, int32_t n_cells, int32_t tile, float *out_lower,
                               float *out_upper, void *stream)
{
    if (!s) return set_last_error(AR_EINVAL, "scene is null");
    int r = validate_call(in, pose, cells, n_cells, tile);
    if (r) return r;
    if (!out_lower || !out_upper) return set_last_error(AR_EINVAL, "null output");
    cudaStream_t st = (cudaStream_t)stream;
    NA_CK(cudaSetDevice(s->device));
    unsigned char *base = nullptr;
    if ((r = scratch_base(s->device, &base))) return r;
    const int W = in->width, H = in->height;
    const size_t out_words = (size_t)n_cells * W * H * 3;
    if (s->n == 0) {
        NA_CK(cudaMemsetAsync(out_lower, 0, out_words * sizeof(float), st));
        NA_CK(cudaMemsetAsync(out_upper, 0, out_words * sizeof(float), st));
        return AR_OK;
    }
    CallConst cc;
    std::memset(&cc, 0, sizeof cc);
    int m_active = 0;
    for (int k = 0; k < MAXV; ++k) {
        bool act = false;
        for (int c = 0; c < n_cells; ++c) act = act || cells[c].hi[k] > cells[c].lo[k];
        cc.m_slot[k] = act ? m_active++ : -1;
    }
    const int M = m_active <= 1 ? 1 : (m_active <= 4 ? 4 : 6);
    // tile = 0: the tile edge and chunk the scene's autotuner chose for this
    // image size and number of pose variables, if an earlier
    // ar_render_abstract call tuned them; else 16 and 16 (this entry point
    // does not time candidates itself)
    int TS = tile, CH = 16;
    if (TS == 0) {
        TS = 16;
        std::lock_guard<std::mutex> lock(s->tune_mu);
        for (const TunedTile &t : s->tuned)
            if (t.W == W && t.H == H && t.M == M) {
                TS = t.TS;
                CH = t.CH;
            }
    }
    cc.W = W; cc.H = H;
    cc.fx = in->fx; cc.fy = in->fy; cc.cx = in->cx; cc.cy = in->cy; cc.near_plane = in->near_plane;
    std::memcpy(cc.R0, pose->R_wc, sizeof cc.R0);
    std::memcpy(cc.t0, pose->t, sizeof cc.t0);
    cc.n_cells = n_cells;
    cc.n_gauss = s->n;
    const uint64_t n_pairs = (uint64_t)n_cells * (uint64_t)s->n;
    const int ntx = (W + TS - 1) / TS, nty = (H + TS - 1) / TS, n_tiles = ntx * nty;
    const uint64_t n_seg = (uint64_t)n_cells * n_tiles;

    // buffers whose sizes are known before the records are built
    Arena A{base};
    double *d_lo = A.take<double>((size_t)MAXV * n_cells), *d_hi = A.take<double>((size_t)MAXV * n_cells);
    void *cellbuf = A.take<unsigned char>(cell_data_bytes(M) * n_cells);
    double *vN = A.take<double>((size_t)VN_STRIDE * s->n);
    float *recs = A.take<float>((size_t)rec_width(M) * n_pairs);
    PixBox *boxes = A.take<PixBox>(n_pairs);
    double *keys = A.take<double>(2 * n_pairs);
    unsigned long long *counters = A.take<unsigned long long>(8);
    uint32_t *seg_start = A.take<uint32_t>(n_seg), *seg_end = A.take<uint32_t>(n_seg);
    uint32_t *seg_k0 = A.take<uint32_t>(n_seg), *seg_k1 = A.take<uint32_t>(n_seg);
    uint32_t *seg_v0 = A.take<uint32_t>(n_seg), *seg_v1 = A.take<uint32_t>(n_seg);
    unsigned int *work = A.take<unsigned int>(64);
    uint32_t *state = A.take<uint32_t>(n_pairs), *wlist = A.take<uint32_t>(n_pairs);
    uint32_t *slist = A.take<uint32_t>(n_pairs);
    uint32_t *act0 = A.take<uint32_t>(n_seg), *act1 = A.take<uint32_t>(n_seg), *words = A.take<uint32_t>(8);
    uint32_t *plist = A.take<uint32_t>(n_seg), *pmask = A.take<uint32_t>(n_seg * (TS * TS / 32 + 1));
    if (A.over) return too_big("the per-(Gaussian, cell) records", A.used);

    // pose cells: lo and hi rows straight from the caller's array (no staging copy)
    NA_CK(cudaMemcpy2DAsync(d_lo, MAXV * sizeof(double), cells[0].lo, sizeof(ar_pose_box), MAXV * sizeof(double),
                            n_cells, cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpy2DAsync(d_hi, MAXV * sizeof(double), cells[0].hi, sizeof(ar_pose_box), MAXV * sizeof(double),
                            n_cells, cudaMemcpyHostToDevice, st));
    // the counters keep the previous call's values: clear them
    NA_CK(cudaMemsetAsync(counters, 0, 8 * sizeof(unsigned long long), st));
    if (launch_pose_prep(s->uw_lo, s->uw_hi, s->Mw, s->n, cc, vN, st) || launch_cell_prep(M, d_lo, d_hi, cc, cellbuf, st) ||
        launch_record_prep(M, vN, s->gp, cc, cellbuf, TS, recs, boxes, keys, counters, st))
        return set_last_error(AR_EDEVICE, cudaGetErrorString(cudaGetLastError()));
    unsigned long long hc[4] = {0, 0, 0, 0};
    NA_CK(cudaMemcpyAsync(hc, counters, sizeof hc, cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    const uint64_t ne = 2 * hc[2], nent = 2 * hc[3];

    // buffers sized by the counts
    const uint64_t nsc = n_pairs > ne ? n_pairs : ne;
    const uint64_t nsort = ne > nent ? ne : nent;
    const uint64_t hist_words = radix_hist_words(nsort > n_seg ? nsort : n_seg) + 64;
    const uint64_t scan_len = nsc > hist_words ? nsc : hist_words;
    BinArgs ba;
    ba.boxes = boxes;
    ba.keys = keys;
    ba.n_pairs = n_pairs;
    ba.n_gauss = (uint64_t)s->n;
    ba.n_cells = n_cells;
    ba.n_events = ne;
    ba.n_entries = nent;
    ba.TS = TS; ba.ntx = ntx; ba.n_tiles = n_tiles;
    ba.n_segments = n_seg;
    for (int i = 0; i < 2; ++i) {
        ba.ev_key[i] = A.take<uint64_t>(ne + 1);
        ba.ev_val[i] = A.take<uint32_t>(ne + 1);
        ba.ent_seg[i] = A.take<uint32_t>(nent + 1);
        ba.ent_ev[i] = A.take<uint32_t>(nent + 1);
    }
    ba.u32_a = A.take<uint32_t>(nsc + 1);
    ba.u32_b = A.take<uint32_t>(nsc + 1);
    ba.u32_c = A.take<uint32_t>(nsc + 1);
    ba.u32_d = A.take<uint32_t>(nsc + 1);
    ba.hist = A.take<uint32_t>(hist_words);
    ba.scan_tmp = A.take<uint32_t>(scan_temp_words(scan_len) + 64);
    ba.seg_start = seg_start;
    ba.seg_end = seg_end;
    ba.seg_k[0] = seg_k0; ba.seg_k[1] = seg_k1;
    ba.seg_v[0] = seg_v0; ba.seg_v[1] = seg_v1;
    if (A.over) return too_big("the depth-sorted tile bins", A.used);
    int launches = 0;
    BinOut bo;
    if (run_binning(ba, bo, st, &launches)) return set_last_error(AR_EDEVICE, cudaGetErrorString(cudaGetLastError()));
    RenderLaunch rl;
    rl.recs = recs;
    rl.boxes = boxes;
    rl.seg_start = seg_start;
    rl.seg_end = seg_end;
    rl.seg_order = bo.seg_order;
    rl.work = work;
    rl.ent_ev = bo.ent_ev;
    rl.ev_val = bo.ev_val;
    rl.ev_key = bo.ev_key;
    rl.W = W; rl.H = H; rl.ntx = ntx; rl.n_tiles = n_tiles; rl.n_cells = n_cells;
    rl.n_gauss = s->n;
    rl.k_open = s->k_open;
    rl.rel = s->blend == AR_BLEND_RELATIONAL;
    rl.fp64_dev = s->fp64_dev;
    rl.ch = CH;
    rl.out_lo = out_lower;
    rl.out_hi = out_upper;
    rl.counters = nullptr;
    return run_windowed_render(M, TS, rl, cc, cellbuf, vN, n_pairs, n_seg, state, wlist, act0, act1, words, nullptr,
                               st, &launches, nullptr, 512u, slist, plist, pmask);
}
