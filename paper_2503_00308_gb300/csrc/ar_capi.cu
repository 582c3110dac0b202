// ar_capi.cu -- host implementation of the libar C ABI (include/ar.h).
//
// A scene owns its Gaussians on the device (FP32 inputs plus the FP64
// covariance factors Mw and cutoff exponents tau) and a grow-only workspace
// that keeps the per-(Gaussian, cell) records, the depth-ordered tile bins and
// the sort buffers resident between calls.  A render is one pass of:
//   pose prep -> cell prep -> record prep -> (one counter read-back) ->
//   binning (radix sorts) -> per-pixel render,
// all enqueued on the caller's stream.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ar.h"
#include "ar_bin.h"
#include "ar_common.cuh"
#include "ar_launch.h"
#include "ar_host.h"

namespace ar {
// NVTX range over a host scope (the enqueue of a render stage; a profiler's
// CUDA trace lines the kernels up under it).  Header-only NVTX 3: no library
// is linked, and the calls cost nothing without a tool attached.
struct NvtxRange {
    bool open = true;
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    void end()
    {
        if (open) nvtxRangePop();
        open = false;
    }
    ~NvtxRange() { end(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
// stage events of one cell batch: start, after prep, after binning, then per
// windowed round: after the record build, after the render
constexpr int kEventsPerBatch = 10;
// the renderer's histograms: 256 sweep lengths, then 64 64-bit stop depths
// weighted by full-list length, then 64 stop depths by segment count
constexpr int kHistWords = 256 + 2 * 64 + 64;
// device counters of one cell batch: opacity evaluations, re-evaluations,
// MatrixInv fallbacks and records built (record build), MatrixInv input
// splits (record build), segments restarted (render), evaluations taken
// again in FP64 (render), segments swept again for them (render)
constexpr int kCountersPerBatch = 8;
// render_batch's answer for a batch with more tile entries than 32-bit
// indices reach (not an AR_ code: render_core splits the batch)
constexpr int kSplitBatch = 1000;
}  // namespace ar

namespace ar {
size_t cell_data_bytes_m1();
size_t cell_data_bytes_m4();
size_t cell_data_bytes_m6();
int rec_width_m1();
int rec_width_m4();
int rec_width_m6();
int rec_scalar_offset_m1();
int rec_scalar_offset_m4();
int rec_scalar_offset_m6();
int launch_cell_prep_m1(const double *, const double *, const CallConst &, void *, cudaStream_t);
int launch_cell_prep_m4(const double *, const double *, const CallConst &, void *, cudaStream_t);
int launch_cell_prep_m6(const double *, const double *, const CallConst &, void *, cudaStream_t);
int launch_record_prep_m1(const double *, const void *, const CallConst &, const void *, int, float *, PixBox *,
                          double *, unsigned long long *, cudaStream_t, uint32_t *, uint32_t *);
int launch_record_prep_m4(const double *, const void *, const CallConst &, const void *, int, float *, PixBox *,
                          double *, unsigned long long *, cudaStream_t, uint32_t *, uint32_t *);
int launch_record_prep_m6(const double *, const void *, const CallConst &, const void *, int, float *, PixBox *,
                          double *, unsigned long long *, cudaStream_t, uint32_t *, uint32_t *);
int launch_render_m1(int, const RenderLaunch &, cudaStream_t);
int launch_render_m4(int, const RenderLaunch &, cudaStream_t);
int launch_render_m6(int, const RenderLaunch &, cudaStream_t);
int launch_record_prep64_m1(const double *, const void *, const CallConst &,
                            const void *, int, double *, PixBox *, double *, unsigned long long *, cudaStream_t);
int launch_record_prep64_m4(const double *, const void *, const CallConst &,
                            const void *, int, double *, PixBox *, double *, unsigned long long *, cudaStream_t);
int launch_record_prep64_m6(const double *, const void *, const CallConst &,
                            const void *, int, double *, PixBox *, double *, unsigned long long *, cudaStream_t);
int launch_record_build_m1(const double *, const CallConst &, const void *, int64_t, const uint32_t *,
                           const uint32_t *, float *, unsigned long long *, uint32_t *, uint32_t *, uint32_t, uint32_t *,
                           cudaStream_t);
int launch_record_build_m4(const double *, const CallConst &, const void *, int64_t, const uint32_t *,
                           const uint32_t *, float *, unsigned long long *, uint32_t *, uint32_t *, uint32_t, uint32_t *,
                           cudaStream_t);
int launch_record_build_m6(const double *, const CallConst &, const void *, int64_t, const uint32_t *,
                           const uint32_t *, float *, unsigned long long *, uint32_t *, uint32_t *, uint32_t, uint32_t *,
                           cudaStream_t);
int launch_debug_alpha_m1(const float *, int, const int64_t *, const int32_t *, const int32_t *, int, float, double *,
                          cudaStream_t);
int launch_debug_alpha_m4(const float *, int, const int64_t *, const int32_t *, const int32_t *, int, float, double *,
                          cudaStream_t);
int launch_debug_alpha_m6(const float *, int, const int64_t *, const int32_t *, const int32_t *, int, float, double *,
                          cudaStream_t);
static int launch_debug_alpha(int M, const float *recs, int n, const int64_t *gi, const int32_t *px, const int32_t *py,
                              int precision, float fp64_dev, double *out, cudaStream_t st)
{
    if (M == 1) return launch_debug_alpha_m1(recs, n, gi, px, py, precision, fp64_dev, out, st);
    if (M == 4) return launch_debug_alpha_m4(recs, n, gi, px, py, precision, fp64_dev, out, st);
    return launch_debug_alpha_m6(recs, n, gi, px, py, precision, fp64_dev, out, st);
}
int launch_render_plain_m1(int, const RenderLaunch &, cudaStream_t);
int launch_render_plain_m4(int, const RenderLaunch &, cudaStream_t);
int launch_render_plain_m6(int, const RenderLaunch &, cudaStream_t);

size_t cell_data_bytes(int M)
{
    return M == 1 ? cell_data_bytes_m1() : (M == 4 ? cell_data_bytes_m4() : cell_data_bytes_m6());
}
int rec_width(int M) { return M == 1 ? rec_width_m1() : (M == 4 ? rec_width_m4() : rec_width_m6()); }
// offset of the scalar fields (o, tau, colour, flags, mu) within a record
static int rec_scalar_offset(int M)
{
    return M == 1 ? rec_scalar_offset_m1() : (M == 4 ? rec_scalar_offset_m4() : rec_scalar_offset_m6());
}
int launch_cell_prep(int M, const double *lo, const double *hi, const CallConst &cc, void *cells, cudaStream_t st)
{
    return M == 1 ? launch_cell_prep_m1(lo, hi, cc, cells, st)
                  : (M == 4 ? launch_cell_prep_m4(lo, hi, cc, cells, st) : launch_cell_prep_m6(lo, hi, cc, cells, st));
}
int launch_record_prep(int M, const double *vN, const void *gp,
                       const CallConst &cc, const void *cells, int TS, float *recs, PixBox *boxes, double *keys,
                       unsigned long long *counters, cudaStream_t st, uint32_t *list, uint32_t *count)
{
    if (M == 1) return launch_record_prep_m1(vN, gp, cc, cells, TS, recs, boxes, keys, counters, st, list, count);
    if (M == 4) return launch_record_prep_m4(vN, gp, cc, cells, TS, recs, boxes, keys, counters, st, list, count);
    return launch_record_prep_m6(vN, gp, cc, cells, TS, recs, boxes, keys, counters, st, list, count);
}
int launch_render(int M, int TS, const RenderLaunch &a, cudaStream_t st)
{
    return M == 1 ? launch_render_m1(TS, a, st) : (M == 4 ? launch_render_m4(TS, a, st) : launch_render_m6(TS, a, st));
}
int launch_record_prep64(int M, const double *vN, const void *gp,
                         const CallConst &cc, const void *cells, int TS, double *recs, PixBox *boxes, double *keys,
                         unsigned long long *counters, cudaStream_t st)
{
    if (M == 1) return launch_record_prep64_m1(vN, gp, cc, cells, TS, recs, boxes, keys, counters, st);
    if (M == 4) return launch_record_prep64_m4(vN, gp, cc, cells, TS, recs, boxes, keys, counters, st);
    return launch_record_prep64_m6(vN, gp, cc, cells, TS, recs, boxes, keys, counters, st);
}
int launch_record_build(int M, const double *vN, const CallConst &cc, const void *cells, int64_t n_gauss,
                        const uint32_t *work, const uint32_t *count, float *recs, unsigned long long *counters,
                        uint32_t *split_list, uint32_t *split_count, uint32_t list_cap, uint32_t *khigh_count,
                        cudaStream_t st)
{
    if (M == 1)
        return launch_record_build_m1(vN, cc, cells, n_gauss, work, count, recs, counters, split_list, split_count,
                                      list_cap, khigh_count, st);
    if (M == 4)
        return launch_record_build_m4(vN, cc, cells, n_gauss, work, count, recs, counters, split_list, split_count,
                                      list_cap, khigh_count, st);
    return launch_record_build_m6(vN, cc, cells, n_gauss, work, count, recs, counters, split_list, split_count,
                                  list_cap, khigh_count, st);
}
int launch_render_plain(int M, int TS, const RenderLaunch &a, cudaStream_t st)
{
    return M == 1 ? launch_render_plain_m1(TS, a, st)
                  : (M == 4 ? launch_render_plain_m4(TS, a, st) : launch_render_plain_m6(TS, a, st));
}
}  // namespace ar

using namespace ar;

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;

static int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(call)                                                                                     \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return fail(AR_EDEVICE, "%s: %s", #call, cudaGetErrorString(e_));     \
    } while (0)

const char *ar_last_error(void) { return g_err.c_str(); }

namespace ar {
int set_last_error(int code, const char *msg)
{
    g_err = msg;
    return code;
}
}  // namespace ar

// --------------------------------------------------------------- buffers
namespace ar {

int DevBuf::ensure(size_t bytes)
{
    if (bytes <= cap) return AR_OK;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    size_t want = bytes + bytes / 4 + 256;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        return fail(AR_ENOMEM, "device allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
    }
    cap = want;
    return AR_OK;
}

void DevBuf::release()
{
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
}

void Workspace::append_pointers(std::vector<uint64_t> &key) const
{
    const DevBuf *all[] = {&cells_lohi, &cells, &vN, &recs, &boxes, &keys, &counters, &evk0, &evk1, &evv0, &evv1,
                           &ents0, &ents1, &ente0, &ente1, &ua, &ub, &uc, &ud, &hist, &scan, &segs, &sege, &segt, &cellev, &bwords, &smask, &ssat, &clist,
                           &segk0, &segk1, &segv0, &segv1, &work, &state, &wlist, &act0, &act1, &words,
                           &slist, &plist, &pmask, &whist};
    for (const DevBuf *b : all) key.push_back((uint64_t)(uintptr_t)b->p);
}

void Workspace::release()
{
    for (GraphEntry &g : graphs) cudaGraphExecDestroy(g.exec);
    graphs.clear();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    cap_stream = nullptr;
    DevBuf *all[] = {&cells_lohi, &cells, &vN, &recs, &boxes, &keys, &counters, &evk0, &evk1, &evv0, &evv1,
                     &ents0, &ents1, &ente0, &ente1, &ua, &ub, &uc, &ud, &hist, &scan, &segs, &sege, &segt, &cellev, &bwords, &smask, &ssat, &clist, &segk0,
                     &segk1, &segv0, &segv1, &work, &state, &wlist, &act0, &act1, &words, &slist, &plist, &pmask, &whist, &out_lo,
                     &out_hi, &part_lo, &part_hi, &lvl_lo, &lvl_hi, &wpart};
    for (DevBuf *b : all) b->release();
    if (h_whist) cudaFreeHost(h_whist);
    h_whist = nullptr;
    whist_pending = false;
    if (h_counters) cudaFreeHost(h_counters);
    h_counters = nullptr;
    for (cudaEvent_t e : evs) cudaEventDestroy(e);
    evs.clear();
}

size_t Workspace::bytes() const
{
    const DevBuf *all[] = {&cells_lohi, &cells, &vN, &recs, &boxes, &keys, &counters, &evk0, &evk1, &evv0, &evv1,
                           &ents0, &ents1, &ente0, &ente1, &ua, &ub, &uc, &ud, &hist, &scan, &segs, &sege, &segt, &cellev, &bwords, &smask, &ssat, &clist,
                           &segk0, &segk1, &segv0, &segv1, &work, &state, &wlist, &act0, &act1, &words,
                           &slist, &plist, &pmask, &whist, &out_lo, &out_hi, &part_lo, &part_hi, &lvl_lo, &lvl_hi, &wpart};
    size_t s = 0;
    for (const DevBuf *b : all) s += b->cap;
    return s;
}

}  // namespace ar


static bool finite3(const float *v, int64_t n, int k)
{
    for (int64_t i = 0; i < n * k; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

int ar_scene_create(const float *uw3, const float *logscale3, const float *quat4, const float *opacity,
                    const float *rgb3, int64_t n, int device_ptrs, ar_scene **out)
{
    if (!out) return fail(AR_EINVAL, "out is null");
    *out = nullptr;
    if (n < 0) return fail(AR_EINVAL, "n < 0");
    if (n > ((int64_t)1 << 30)) return fail(AR_EINVAL, "n > 2^30 Gaussians");
    if (n > 0 && (!uw3 || !logscale3 || !quat4 || !opacity || !rgb3)) return fail(AR_EINVAL, "null array");
    std::vector<float> h_uw, h_ls, h_q, h_o, h_c;
    const float *src[5] = {uw3, logscale3, quat4, opacity, rgb3};
    const int width[5] = {3, 3, 4, 1, 3};
    std::vector<float> *dst[5] = {&h_uw, &h_ls, &h_q, &h_o, &h_c};
    for (int a = 0; a < 5; ++a) {
        dst[a]->resize((size_t)n * width[a]);
        if (n == 0) continue;
        if (device_ptrs) {
            cudaError_t e = cudaMemcpy(dst[a]->data(), src[a], sizeof(float) * n * width[a], cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return fail(AR_EINVAL, "cannot read device array %d: %s", a, cudaGetErrorString(e));
        } else {
            std::memcpy(dst[a]->data(), src[a], sizeof(float) * n * width[a]);
        }
    }
    for (int a = 0; a < 5; ++a)
        if (!finite3(dst[a]->data(), n, width[a])) return fail(AR_EINVAL, "non-finite value in input array %d", a);
    for (int64_t i = 0; i < n; ++i) {
        if (!(h_o[i] >= 0.f && h_o[i] < 1.f)) return fail(AR_EINVAL, "opacity[%lld] outside [0, 1)", (long long)i);
        for (int k = 0; k < 3; ++k)
            if (!(h_c[3 * i + k] >= 0.f && h_c[3 * i + k] <= 1.f))
                return fail(AR_EINVAL, "rgb[%lld] outside [0, 1]", (long long)i);
        const float *q = &h_q[4 * i];
        if (q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3] == 0.f)
            return fail(AR_EINVAL, "quaternion %lld is zero", (long long)i);
        for (int k = 0; k < 3; ++k)
            if (!(std::fabs(h_ls[3 * i + k]) < 40.f)) return fail(AR_EINVAL, "log-scale %lld out of range", (long long)i);
    }
    ar_scene *s = new ar_scene();
    cudaGetDevice(&s->device);
    s->n = n;
    {
        double omax = 0.0;
        for (int64_t i = 0; i < n; ++i) omax = std::fmax(omax, (double)h_o[i]);
        s->k_open = (float)(1.0 / (1.0 - omax)) * 1.0001f + 1e-6f;
    }
    std::memset(&s->stats, 0, sizeof s->stats);
    if (n > 0) {
        float **dp[5] = {&s->uw, &s->ls, &s->quat, &s->opac, &s->rgb};
        for (int a = 0; a < 5; ++a) {
            if (cudaMalloc(dp[a], sizeof(float) * n * width[a]) != cudaSuccess ||
                cudaMemcpy(*dp[a], dst[a]->data(), sizeof(float) * n * width[a], cudaMemcpyHostToDevice) != cudaSuccess) {
                cudaGetLastError();
                ar_scene_destroy(s);
                return fail(AR_ENOMEM, "scene upload failed");
            }
        }
        if (cudaMalloc(&s->Mw, sizeof(double) * 9 * n) != cudaSuccess ||
            cudaMalloc(&s->tau, sizeof(double) * n) != cudaSuccess) {
            cudaGetLastError();
            ar_scene_destroy(s);
            return fail(AR_ENOMEM, "scene allocation failed");
        }
        if (cudaMalloc(&s->gp, sizeof(GParam) * n) != cudaSuccess) {
            cudaGetLastError();
            ar_scene_destroy(s);
            return fail(AR_ENOMEM, "scene allocation failed");
        }
        s->uw_lo = s->uw;
        s->uw_hi = s->uw;
        if (launch_scene_prep(s->ls, s->quat, s->opac, n, s->Mw, s->tau, 0) ||
            launch_gparam(s->opac, s->opac, s->rgb, s->rgb, n, s->gp, 0) || cudaDeviceSynchronize() != cudaSuccess) {
            const char *m = cudaGetErrorString(cudaGetLastError());
            ar_scene_destroy(s);
            return fail(AR_EDEVICE, "scene preprocessing failed: %s", m);
        }
    }
    *out = s;
    return AR_OK;
}

int ar_scene_set_boxes(ar_scene *s, const float *uw_lo3, const float *uw_hi3, const float *opacity_lo,
                       const float *opacity_hi, const float *rgb_lo3, const float *rgb_hi3)
{
    if (!s) return fail(AR_EINVAL, "scene is null");
    if (!uw_lo3 != !uw_hi3 || !opacity_lo != !opacity_hi || !rgb_lo3 != !rgb_hi3)
        return fail(AR_EINVAL, "a box needs both its lower and its upper array");
    const int64_t n = s->n;
    if (n == 0) return AR_OK;
    CK(cudaSetDevice(s->device));
    // host copies of the nominal values fill the parameters without a box
    std::vector<float> nom_uw((size_t)3 * n), nom_o((size_t)n), nom_c((size_t)3 * n);
    CK(cudaMemcpy(nom_uw.data(), s->uw, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(nom_o.data(), s->opac, sizeof(float) * n, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(nom_c.data(), s->rgb, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost));
    // layout of the box buffer: uw_lo 3n, uw_hi 3n, o_lo n, o_hi n, c_lo 3n, c_hi 3n
    std::vector<float> h((size_t)14 * n);
    float *ul = h.data(), *uh = ul + 3 * n, *ol = uh + 3 * n, *oh = ol + n, *cl = oh + n, *ch = cl + 3 * n;
    for (int64_t i = 0; i < 3 * n; ++i) {
        ul[i] = uw_lo3 ? uw_lo3[i] : nom_uw[i];
        uh[i] = uw_hi3 ? uw_hi3[i] : nom_uw[i];
        cl[i] = rgb_lo3 ? rgb_lo3[i] : nom_c[i];
        ch[i] = rgb_hi3 ? rgb_hi3[i] : nom_c[i];
        if (!std::isfinite(ul[i]) || !std::isfinite(uh[i]) || !(ul[i] <= uh[i]))
            return fail(AR_EINVAL, "mean box %lld: not finite or lo > hi", (long long)(i / 3));
        if (!(cl[i] >= 0.f && cl[i] <= ch[i] && ch[i] <= 1.f))
            return fail(AR_EINVAL, "colour box %lld outside 0 <= lo <= hi <= 1", (long long)(i / 3));
    }
    double omax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        ol[i] = opacity_lo ? opacity_lo[i] : nom_o[i];
        oh[i] = opacity_hi ? opacity_hi[i] : nom_o[i];
        if (!(ol[i] >= 0.f && ol[i] <= oh[i] && oh[i] < 1.f))
            return fail(AR_EINVAL, "opacity box %lld outside 0 <= lo <= hi < 1", (long long)i);
        omax = std::fmax(omax, (double)oh[i]);
    }
    float *buf = nullptr;
    if (cudaMalloc(&buf, sizeof(float) * h.size()) != cudaSuccess) {
        cudaGetLastError();
        return fail(AR_ENOMEM, "box allocation failed");
    }
    if (cudaMemcpy(buf, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        launch_gparam(buf + 6 * n, buf + 7 * n, buf + 8 * n, buf + 11 * n, n, s->gp, 0) ||
        cudaDeviceSynchronize() != cudaSuccess) {
        const char *m = cudaGetErrorString(cudaGetLastError());
        cudaFree(buf);
        return fail(AR_EDEVICE, "box upload failed: %s", m);
    }
    if (s->boxbuf) cudaFree(s->boxbuf);
    s->boxbuf = buf;
    s->uw_lo = buf;
    s->uw_hi = buf + 3 * n;
    s->k_open = (float)(1.0 / (1.0 - omax)) * 1.0001f + 1e-6f;
    return AR_OK;
}

int ar_scene_destroy(ar_scene *s)
{
    if (!s) return fail(AR_EINVAL, "scene is null");
    cudaSetDevice(s->device);
    cudaDeviceSynchronize();
    void *ptrs[] = {s->uw, s->ls, s->quat, s->opac, s->rgb, s->Mw, s->tau, s->gp, s->boxbuf};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    s->ws.release();
    delete s;
    return AR_OK;
}

int ar_set_workspace_limit(ar_scene *s, int64_t bytes)
{
    if (!s) return fail(AR_EINVAL, "scene is null");
    if (bytes < (int64_t)1 << 20) return fail(AR_EINVAL, "workspace limit below 1 MiB");
    s->ws_limit = bytes;
    return AR_OK;
}

int ar_set_profiling(ar_scene *s, int on)
{
    if (!s) return fail(AR_EINVAL, "scene is null");
    s->profiling = on != 0;
    return AR_OK;
}

int ar_scene_set_blend(ar_scene *s, int32_t mode)
{
    if (!s) return fail(AR_EINVAL, "scene is null");
    if (mode != AR_BLEND_INTERVAL && mode != AR_BLEND_RELATIONAL) return fail(AR_EINVAL, "unknown blend mode %d", mode);
    s->blend = mode;
    return AR_OK;
}

int ar_debug_set_cull(ar_scene *s, int32_t mode)
{
    if (!s) return fail(AR_EINVAL, "scene is null");
    if (mode < -1 || mode > 1) return fail(AR_EINVAL, "mode must be -1, 0 or 1");
    s->cull_force = mode;
    return AR_OK;
}

int ar_debug_learned_prefix(const uint64_t *weights, const uint32_t *counts, uint64_t n_entries, uint64_t n_events,
                            int32_t *shift)
{
    if (!weights || !counts || !shift) return fail(AR_EINVAL, "null argument");
    static_assert(sizeof(unsigned long long) == sizeof(uint64_t), "64-bit histogram words");
    *shift = learned_prefix_shift(reinterpret_cast<const unsigned long long *>(weights), counts, n_entries, n_events);
    return AR_OK;
}

int ar_debug_learned_window(const uint32_t *hist, uint32_t *window)
{
    if (!hist || !window) return fail(AR_EINVAL, "null argument");
    *window = learned_window(hist);
    return AR_OK;
}

int ar_debug_set_prefix(ar_scene *s, int32_t shift)
{
    if (!s) return fail(AR_EINVAL, "scene is null");
    if (shift < -1 || shift > 8) return fail(AR_EINVAL, "shift must be -1 or in [0, 8]");
    s->prefix_force = shift;
    return AR_OK;
}

int ar_debug_set_entry_cap(ar_scene *s, int64_t cap)
{
    if (!s) return fail(AR_EINVAL, "scene is null");
    const int64_t top = (int64_t)((1ull << 32) - (1ull << 20));
    if (cap < 0 || cap > top) return fail(AR_EINVAL, "cap must be in [0, 2^32 - 2^20]");
    s->entry_cap = cap ? (uint64_t)cap : (uint64_t)top;
    return AR_OK;
}

int ar_debug_set_chunk(ar_scene *s, int32_t chunk)
{
    if (!s) return fail(AR_EINVAL, "scene is null");
    if (chunk != 0 && chunk != 8 && chunk != 16 && chunk != 32) return fail(AR_EINVAL, "chunk must be 0, 8, 16 or 32");
    s->chunk = chunk;
    return AR_OK;
}

int ar_scene_set_graphs(ar_scene *s, int32_t on)
{
    if (!s) return fail(AR_EINVAL, "scene is null");
    if (on != 0 && on != 1) return fail(AR_EINVAL, "on must be 0 or 1");
    s->graphs = on != 0;
    return AR_OK;
}

int ar_scene_set_fp64_alpha(ar_scene *s, float threshold)
{
    if (!s) return fail(AR_EINVAL, "scene is null");
    if (!(threshold >= 0.f)) return fail(AR_EINVAL, "threshold must be >= 0 (not NaN)");
    s->fp64_dev = threshold;
    return AR_OK;
}

// ---------------------------------------------------------------- render
namespace ar {

int validate_call(const ar_intrinsics *in, const ar_nominal_pose *pose, const ar_pose_box *cells, int32_t n_cells,
                  int32_t tile)
{
    if (!in || !pose || !cells) return fail(AR_EINVAL, "null argument");
    if (n_cells < 1 || n_cells > 65535) return fail(AR_EINVAL, "n_cells must be in [1, 65535]");
    if (in->width < 1 || in->height < 1 || in->width > 16384 || in->height > 16384)
        return fail(AR_EINVAL, "image size out of range");
    const float f[5] = {in->fx, in->fy, in->cx, in->cy, in->near_plane};
    for (float v : f)
        if (!std::isfinite(v)) return fail(AR_EINVAL, "non-finite intrinsics");
    if (!(in->fx > 0 && in->fy > 0 && in->near_plane > 0)) return fail(AR_EINVAL, "fx, fy, near_plane must be > 0");
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(pose->R_wc[i])) return fail(AR_EINVAL, "non-finite rotation");
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(pose->t[i])) return fail(AR_EINVAL, "non-finite camera centre");
    for (int c = 0; c < n_cells; ++c)
        for (int k = 0; k < MAXV; ++k) {
            const double lo = cells[c].lo[k], hi = cells[c].hi[k];
            if (!std::isfinite(lo) || !std::isfinite(hi) || lo > hi)
                return fail(AR_EINVAL, "cell %d dimension %d: need finite lo <= hi", c, k);
            if (k >= 3 && (hi - lo) > 0.5) return fail(AR_EINVAL, "cell %d: rotation width above 0.5 rad", c);
        }
    if (tile != 0 && tile != 8 && tile != 16) return fail(AR_EINVAL, "tile must be 0, 8 or 16");
    return AR_OK;
}

#define RK(x)                      \
    do {                           \
        int r_ = (x);              \
        if (r_) return r_;         \
    } while (0)

// Sizes the binning buffers of the workspace and (run) runs the binning of
// n_pairs (cell, Gaussian) pairs with ne events and nent (event, tile) entries.
// shift > 0: the first phase of a two-phase binning (BinArgs), whose
// arguments ba_out receives for the second; the renderer's own binning
// (cell_ev) also passes a non-null ba_out with shift 0.
static int bin_pairs(Workspace &ws, const PixBox *boxes, const double *keys, uint64_t n_pairs, uint64_t n_gauss,
                     int n_cells, uint64_t ne, uint64_t nent, int TS, int ntx, int n_tiles, cudaStream_t st,
                     BinOut &bo, int &launches, bool run = true, int shift = 0, BinArgs *ba_out = nullptr)
{
    const uint64_t n_seg = (uint64_t)n_cells * n_tiles;
    const uint64_t nsc = n_pairs > ne ? n_pairs : ne;
    const uint64_t nsort = ne > nent ? ne : nent;
    const uint64_t hist_words = radix_hist_words(nsort > n_seg ? nsort : n_seg) + 64;
    uint64_t scan_len = nsc > hist_words ? nsc : hist_words;
    RK(ws.evk0.ensure(sizeof(uint64_t) * (ne + 1)));
    RK(ws.evk1.ensure(sizeof(uint64_t) * (ne + 1)));
    RK(ws.evv0.ensure(sizeof(uint32_t) * (ne + 1)));
    RK(ws.evv1.ensure(sizeof(uint32_t) * (ne + 1)));
    RK(ws.ents0.ensure(sizeof(uint32_t) * (nent + 1)));
    RK(ws.ents1.ensure(sizeof(uint32_t) * (nent + 1)));
    RK(ws.ente0.ensure(sizeof(uint32_t) * (nent + 1)));
    RK(ws.ente1.ensure(sizeof(uint32_t) * (nent + 1)));
    RK(ws.ua.ensure(sizeof(uint32_t) * (nsc + 1)));
    RK(ws.ub.ensure(sizeof(uint32_t) * (nsc + 1)));
    RK(ws.uc.ensure(sizeof(uint32_t) * (nsc + 1)));
    RK(ws.ud.ensure(sizeof(uint32_t) * (nsc + 1)));
    RK(ws.hist.ensure(sizeof(uint32_t) * hist_words));
    RK(ws.scan.ensure(sizeof(uint32_t) * (scan_temp_words(scan_len) + 64)));
    RK(ws.segs.ensure(sizeof(uint32_t) * n_seg));
    RK(ws.sege.ensure(sizeof(uint32_t) * n_seg));
    RK(ws.segk0.ensure(sizeof(uint32_t) * n_seg));
    RK(ws.segk1.ensure(sizeof(uint32_t) * n_seg));
    RK(ws.segv0.ensure(sizeof(uint32_t) * n_seg));
    RK(ws.segv1.ensure(sizeof(uint32_t) * n_seg));
    RK(ws.work.ensure(256));
    if (ba_out) {
        RK(ws.cellev.ensure(sizeof(uint32_t) * 2 * (n_cells + 1)));
        RK(ws.bwords.ensure(sizeof(uint32_t) * 4));
    }
    if (shift > 0) {
        RK(ws.segt.ensure(sizeof(uint32_t) * n_seg));
        RK(ws.smask.ensure(sizeof(uint32_t) * ((n_seg + 31) / 32 + 1)));
        RK(ws.ssat.ensure(sizeof(uint32_t) * (uint64_t)n_cells * (ntx + 1) * (n_tiles / ntx + 1)));
    }
    if (!run) return AR_OK;
    BinArgs ba;
    ba.boxes = boxes;
    ba.keys = keys;
    ba.n_pairs = n_pairs;
    ba.n_gauss = n_gauss;
    ba.n_cells = n_cells;
    ba.n_events = ne;
    ba.n_entries = nent;
    ba.TS = TS; ba.ntx = ntx; ba.n_tiles = n_tiles;
    ba.n_segments = n_seg;
    ba.ev_key[0] = ws.evk0.as<uint64_t>(); ba.ev_key[1] = ws.evk1.as<uint64_t>();
    ba.ev_val[0] = ws.evv0.as<uint32_t>(); ba.ev_val[1] = ws.evv1.as<uint32_t>();
    ba.ent_seg[0] = ws.ents0.as<uint32_t>(); ba.ent_seg[1] = ws.ents1.as<uint32_t>();
    ba.ent_ev[0] = ws.ente0.as<uint32_t>(); ba.ent_ev[1] = ws.ente1.as<uint32_t>();
    ba.u32_a = ws.ua.as<uint32_t>(); ba.u32_b = ws.ub.as<uint32_t>();
    ba.u32_c = ws.uc.as<uint32_t>(); ba.u32_d = ws.ud.as<uint32_t>();
    ba.hist = ws.hist.as<uint32_t>();
    ba.scan_tmp = ws.scan.as<uint32_t>();
    ba.seg_start = ws.segs.as<uint32_t>();
    ba.seg_end = ws.sege.as<uint32_t>();
    ba.seg_k[0] = ws.segk0.as<uint32_t>(); ba.seg_k[1] = ws.segk1.as<uint32_t>();
    ba.seg_v[0] = ws.segv0.as<uint32_t>(); ba.seg_v[1] = ws.segv1.as<uint32_t>();
    if (ba_out) {
        ba.cell_ev = ws.cellev.as<uint32_t>();
        ba.pref_start = ba.cell_ev + (n_cells + 1);
        ba.words = ws.bwords.as<uint32_t>();
    }
    if (shift > 0) {
        ba.prefix_shift = shift;
        ba.seg_total = ws.segt.as<uint32_t>();
        ba.mask = ws.smask.as<uint32_t>();
        ba.sat = ws.ssat.as<uint32_t>();
    }
    if (ba_out) *ba_out = ba;
    if (run_binning(ba, bo, st, &launches))
        return fail(AR_EDEVICE, "binning: %s", cudaGetErrorString(cudaGetLastError()));
    return AR_OK;
}

static uint32_t float_bits(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, sizeof u);
    return u;
}
static uint64_t double_bits(double d)
{
    uint64_t u;
    std::memcpy(&u, &d, sizeof u);
    return u;
}

// A stage-timing event on q.  While q is being captured, the record becomes an
// external event node of the graph, so that every replay records the event
// (an ordinary record during capture would only order the graph's nodes).
static cudaError_t record_stage(cudaEvent_t e, cudaStream_t q)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(q, &cs) != cudaSuccess) return cudaGetLastError();
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, q, cudaEventRecordExternal)
                                               : cudaEventRecord(e, q);
}

static int enqueue_rest(ar_scene *s, Workspace &ws, const CallConst &cc, int M, int TS, int CH, float *out_lo, float *out_hi,
                        cudaStream_t q, bool profiling, int batch, cudaEvent_t *ev, uint64_t n_pairs, uint64_t n_seg,
                        uint64_t ne, uint64_t nent, int ntx, int n_tiles, bool plain, int shift, int &launches);

// One batch of cells through the whole pipeline.  cc describes the batch
// (n_cells = cells in the batch, slots shared by every batch of the call).
// plain: FP64 records and the plain FP64 renderer instead of the FP32 ones.
static int render_batch(ar_scene *s, Workspace &ws, const CallConst &cc, int M, int TS, int CH, const double *d_lo,
                        const double *d_hi, float *out_lo, float *out_hi, cudaStream_t st, bool profiling,
                        int batch, ar_render_stats &rs, int &launches, bool plain)
{
    const int W = cc.W, H = cc.H, n_cells = cc.n_cells;
    const uint64_t n_pairs = (uint64_t)n_cells * (uint64_t)s->n;
    const int ntx = (W + TS - 1) / TS, nty = (H + TS - 1) / TS, n_tiles = ntx * nty;
    const uint64_t n_seg = (uint64_t)n_cells * n_tiles;
    RK(ws.cells.ensure(cell_data_bytes(M) * n_cells));
    RK(ws.recs.ensure((plain ? sizeof(double) : sizeof(float)) * rec_width(M) * n_pairs));
    RK(ws.boxes.ensure(sizeof(PixBox) * n_pairs));
    RK(ws.keys.ensure(sizeof(double) * 2 * n_pairs));

    cudaEvent_t *ev = &ws.evs[kEventsPerBatch * batch];
    NvtxRange batch_range("ar.cell_batch");
    if (profiling) CK(cudaEventRecord(ev[0], st));
    CK(cudaMemsetAsync(ws.counters.p, 0, sizeof(unsigned long long) * 8, st));
    // the certain drops culled first where the last render found many
    const bool cull = !plain && (s->cull_force >= 0 ? s->cull_force == 1 : ws.cull_on);
    if (cull) RK(ws.clist.ensure(sizeof(uint32_t) * (n_pairs + 1)));
    NvtxRange prep_range("ar.prep: cells and (Gaussian, cell) decisions");
    if (launch_cell_prep(M, d_lo, d_hi, cc, ws.cells.p, st)) return fail(AR_EDEVICE, "cell_prep launch");
    const int rp = plain ? launch_record_prep64(M, ws.vN.as<double>(), s->gp, cc, ws.cells.p, TS,
                                                ws.recs.as<double>(), ws.boxes.as<PixBox>(), ws.keys.as<double>(),
                                                ws.counters.as<unsigned long long>(), st)
                         : launch_record_prep(M, ws.vN.as<double>(), s->gp, cc, ws.cells.p, TS,
                                              ws.recs.as<float>(), ws.boxes.as<PixBox>(), ws.keys.as<double>(),
                                              ws.counters.as<unsigned long long>(), st,
                                              cull ? ws.clist.as<uint32_t>() : nullptr,
                                              cull ? ws.clist.as<uint32_t>() + n_pairs : nullptr);
    if (rp) return fail(AR_EDEVICE, "record_prep launch: %s", cudaGetErrorString(cudaGetLastError()));
    launches += 2;
    if (profiling) CK(cudaEventRecord(ev[1], st));
    CK(cudaMemcpyAsync(ws.h_counters, ws.counters.p, sizeof(unsigned long long) * 5, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    prep_range.end();
    const unsigned long long n_valid = ws.h_counters[2];
    const uint64_t ne = 2 * n_valid, nent = 2 * ws.h_counters[3];
    // culling pays where many pairs reach no pixel: here fewer than 3/4 do
    if (!plain) ws.cull_on = n_valid * 4 < n_pairs * 3;
    if (ws.whist_pending) {
        // the previous render's histograms arrived with this synchronisation
        ws.w0 = learned_window(ws.h_whist);
        ws.prefix_shift = learned_prefix_shift(reinterpret_cast<const unsigned long long *>(ws.h_whist + 256),
                                               ws.h_whist + 384, nent, ne);
        ws.whist_pending = false;
    }
    // the depth prefix of the first binning phase (0: one phase)
    const int shift = plain ? 0 : (s->prefix_force >= 0 ? s->prefix_force : ws.prefix_shift);
    if (nent >= s->entry_cap) return kSplitBatch;  // the caller splits the batch
    rs.n_records += (int64_t)n_valid;
    rs.n_triples += (int64_t)ws.h_counters[0];
    rs.n_fallback += (int64_t)ws.h_counters[1];
    rs.n_split += (int64_t)ws.h_counters[4];
    rs.n_entries += (int64_t)(nent / 2);
    // every buffer of the rest of the batch, sized before any of it is enqueued
    BinOut bo;
    BinArgs sized;
    RK(bin_pairs(ws, ws.boxes.as<PixBox>(), ws.keys.as<double>(), n_pairs, (uint64_t)s->n, n_cells, ne, nent, TS, ntx,
                 n_tiles, st, bo, launches, false, shift, plain ? nullptr : &sized));
    if (!plain) {
        RK(ws.state.ensure(sizeof(uint32_t) * n_pairs));
        RK(ws.wlist.ensure(sizeof(uint32_t) * n_pairs));
        RK(ws.act0.ensure(sizeof(uint32_t) * n_seg));
        RK(ws.act1.ensure(sizeof(uint32_t) * n_seg));
        RK(ws.words.ensure(sizeof(uint32_t) * 8));
        RK(ws.slist.ensure(sizeof(uint32_t) * n_pairs));
        RK(ws.plist.ensure(sizeof(uint32_t) * n_seg));
        RK(ws.pmask.ensure(sizeof(uint32_t) * n_seg * (TS * TS / 32 + 1)));  // pixel mask + a flag per slot
    }
    // The rest of the batch (binning, then the windowed rounds of build and
    // render) depends on the host only through the sizes read above, so with
    // graphs on it is captured once per sizes, buffers and parameters and
    // replayed as one CUDA graph: a repeated render of the same shape
    // launches one graph instead of some forty kernels and memsets.
    std::vector<uint64_t> key;
    if (s->graphs && !plain) {
        const uint64_t head[] = {(uint64_t)M, (uint64_t)TS, (uint64_t)CH, (uint64_t)n_cells, n_pairs, ne, nent, (uint64_t)n_tiles,
                                 (uint64_t)ntx, (uint64_t)W, (uint64_t)H, (uint64_t)s->n, ws.w0,
                                 (uint64_t)s->blend, (uint64_t)float_bits(s->fp64_dev), (uint64_t)float_bits(s->k_open),
                                 (uint64_t)profiling, (uint64_t)ws.interleave, (uint64_t)batch, (uint64_t)(uintptr_t)out_lo,
                                 (uint64_t)(uintptr_t)out_hi, (uint64_t)(uintptr_t)d_lo, (uint64_t)shift};
        key.assign(head, head + sizeof head / sizeof head[0]);
        ws.append_pointers(key);
        for (int k = 0; k < kEventsPerBatch; ++k) key.push_back((uint64_t)(uintptr_t)ev[k]);
        // the call constants the launches take by value (named fields: no padding bytes)
        const float fc[5] = {cc.fx, cc.fy, cc.cx, cc.cy, cc.near_plane};
        for (float f : fc) key.push_back(float_bits(f));
        for (int i = 0; i < 9; ++i) key.push_back(double_bits(cc.R0[i]));
        for (int i = 0; i < 3; ++i) key.push_back(double_bits(cc.t0[i]));
        for (int k = 0; k < MAXV; ++k) key.push_back((uint64_t)(int64_t)cc.m_slot[k]);
        key.push_back((uint64_t)cc.n_gauss);
        for (GraphEntry &g : ws.graphs)
            if (g.key == key) {
                CK(cudaGraphLaunch(g.exec, st));
                g.last_use = ++ws.graph_clock;
                launches += g.launches;
                ++ws.graph_hits;
                ++rs.n_graph_replays;
                return AR_OK;
            }
    }
    cudaStream_t q = st;  // the stream the rest is enqueued on (the capture stream while capturing)
    bool capturing = false;
    if (!key.empty()) {
        if (!ws.cap_stream) CK(cudaStreamCreateWithFlags(&ws.cap_stream, cudaStreamNonBlocking));
        if (cudaStreamBeginCapture(ws.cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            q = ws.cap_stream;
            capturing = true;
        } else {
            cudaGetLastError();
        }
    }
    const int launches0 = launches;
    const int rc = enqueue_rest(s, ws, cc, M, TS, CH, out_lo, out_hi, q, profiling, batch, ev, n_pairs, n_seg, ne, nent,
                                ntx, n_tiles, plain, shift, launches);
    if (capturing) {
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(ws.cap_stream, &graph);
        cudaGraphExec_t exec = nullptr;
        if (rc == AR_OK && e == cudaSuccess && graph &&
            cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess && exec) {
            cudaGraphDestroy(graph);
            if (ws.graphs.size() >= kMaxGraphs) {
                size_t old = 0;
                for (size_t i = 1; i < ws.graphs.size(); ++i)
                    if (ws.graphs[i].last_use < ws.graphs[old].last_use) old = i;
                cudaGraphExecDestroy(ws.graphs[old].exec);
                ws.graphs.erase(ws.graphs.begin() + (long)old);
            }
            ws.graphs.push_back(GraphEntry{key, exec, launches - launches0, ++ws.graph_clock});
            CK(cudaGraphLaunch(exec, st));
            return AR_OK;
        }
        // capture failed (a call that cannot be captured): run uncaptured from now on
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        s->graphs = false;
        RK(rc);
        launches = launches0;
        return enqueue_rest(s, ws, cc, M, TS, CH, out_lo, out_hi, st, profiling, batch, ev, n_pairs, n_seg, ne, nent, ntx,
                            n_tiles, plain, shift, launches);
    }
    return rc;
}

// The part of a batch after the host has read its sizes: binning, then the
// render (windowed rounds, or the plain FP64 renderer), enqueued on q.
static int enqueue_rest(ar_scene *s, Workspace &ws, const CallConst &cc, int M, int TS, int CH, float *out_lo, float *out_hi,
                        cudaStream_t q, bool profiling, int batch, cudaEvent_t *ev, uint64_t n_pairs, uint64_t n_seg,
                        uint64_t ne, uint64_t nent, int ntx, int n_tiles, bool plain, int shift, int &launches)
{
    const int W = cc.W, H = cc.H, n_cells = cc.n_cells;
    BinOut bo;
    BinArgs ba;
    {
        NvtxRange r("ar.bin: depth-sorted tile bins");
        RK(bin_pairs(ws, ws.boxes.as<PixBox>(), ws.keys.as<double>(), n_pairs, (uint64_t)s->n, n_cells, ne, nent, TS,
                     ntx, n_tiles, q, bo, launches, true, shift, plain ? nullptr : &ba));
    }
    if (profiling) CK(record_stage(ev[2], q));
    RenderLaunch rl;
    rl.recs = ws.recs.as<float>();
    rl.recs64 = ws.recs.as<double>();
    rl.boxes = ws.boxes.as<PixBox>();
    rl.seg_start = ws.segs.as<uint32_t>();
    rl.seg_end = ws.sege.as<uint32_t>();
    rl.seg_order = bo.seg_order;
    rl.work = ws.work.as<unsigned int>();
    rl.ent_ev = bo.ent_ev;
    rl.ev_val = bo.ev_val;
    rl.ev_key = bo.ev_key;
    rl.seg_total = bo.seg_total;
    rl.cell_ev = plain ? nullptr : ba.cell_ev;
    rl.W = W; rl.H = H; rl.ntx = ntx; rl.n_tiles = n_tiles; rl.n_cells = n_cells;
    rl.n_gauss = s->n;
    rl.k_open = s->k_open;
    rl.rel = s->blend == AR_BLEND_RELATIONAL;
    rl.fp64_dev = s->fp64_dev;
    rl.ch = CH;
    rl.interleave = ws.interleave ? 1 : 0;
    rl.out_lo = out_lo;
    rl.out_hi = out_hi;
    rl.counters = ws.counters.as<unsigned long long>() + 8 + kCountersPerBatch * batch;
    if (plain) {
        if (profiling) CK(record_stage(ev[3], q));
        if (launch_render_plain(M, TS, rl, q))
            return fail(AR_EDEVICE, "render launch: %s", cudaGetErrorString(cudaGetLastError()));
        ++launches;
        if (profiling)
            for (int k = 4; k < kEventsPerBatch; ++k) CK(record_stage(ev[k], q));
    } else {
        rl.sweep_hist = ws.whist.as<uint32_t>();
        RK(run_windowed_render(M, TS, rl, cc, ws.cells.p, ws.vN.as<double>(), n_pairs, n_seg, ws.state.as<uint32_t>(),
                               ws.wlist.as<uint32_t>(), ws.act0.as<uint32_t>(), ws.act1.as<uint32_t>(),
                               ws.words.as<uint32_t>(), rl.counters + 2, q, &launches,
                               profiling ? ev + 3 : nullptr, ws.w0, ws.slist.as<uint32_t>(), ws.plist.as<uint32_t>(),
                               ws.pmask.as<uint32_t>(), bo.seg_total ? &ba : nullptr, &bo));
    }
    return AR_OK;
}

// the cost of a segment's restart (its prefix swept twice) in sorted
// entries: on object300k a restart cost about 183 ns of render time and the
// tile binning about 14 ps per entry
constexpr double kRestartEntries = 12000.0;

int learned_prefix_shift(const unsigned long long *h, const uint32_t *hc, uint64_t n_entries, uint64_t n_events)
{
    unsigned long long tot = 0, segs = 0;
    for (int b = 0; b < 64; ++b) {
        tot += h[b];
        segs += hc[b];
    }
    if (tot == 0 || segs == 0) return 3;
    int best = 0;
    double best_cost = (double)n_entries;
    for (int sh = 1; sh <= 6; ++sh) {
        unsigned long long beyond = 0, beyond_n = 0;  // buckets at or past the prefix, 2^-sh of the events
        for (int b = 64 >> sh; b < 64; ++b) {
            beyond += h[b];
            beyond_n += hc[b];
        }
        const double scale = (double)n_entries / (double)tot;  // the earlier render's lengths to this one's
        const double cost = (double)n_entries * std::ldexp(1.0, -sh) + scale * (double)beyond +
                            (beyond_n ? (double)n_events : 0.0) + kRestartEntries * scale * (double)beyond_n;
        if (cost < best_cost) {
            best_cost = cost;
            best = sh;
        }
    }
    return best;
}

uint32_t learned_window(const uint32_t *hist256)
{
    uint64_t total = 0;
    for (int b = 0; b < 256; ++b) total += hist256[b];
    if (total == 0) return 512u;
    const uint64_t keep = total - total / 200;  // 99.5 %
    uint64_t run = 0;
    int b = 0;
    for (; b < 256; ++b) {
        run += hist256[b];
        if (run >= keep) break;
    }
    uint32_t w = 32u * (uint32_t)(b + 2);  // the bucket's end plus one chunk of margin
    if (w < 128u) w = 128u;
    if (w > 4096u) w = 4096u;
    return w;
}

int run_windowed_render(int M, int TS, RenderLaunch rl, const CallConst &cc, const void *cells, const double *vN,
                        uint64_t n_pairs, uint64_t n_seg, uint32_t *state, uint32_t *wlist, uint32_t *act0,
                        uint32_t *act1, uint32_t *words, unsigned long long *build_counters, cudaStream_t st,
                        int *launches, cudaEvent_t *ev, uint32_t w0, uint32_t *split_list, uint32_t *precise_list,
                        uint32_t *precise_mask, const BinArgs *rebin, const BinOut *first)
{
    // two phases: a segment restarts in the second round mostly because its
    // depth prefix ran out, so that round keeps the first window
    const bool two = rebin && first && first->seg_total;
    const uint32_t kWindow[3] = {w0, two ? w0 : (w0 < 8192u ? 8192u : 0xffffffffu), 0xffffffffu};
    const uint32_t *round1_order = nullptr;
    uint32_t *act[2] = {act0, act1};
    CK(cudaMemsetAsync(state, 0, sizeof(uint32_t) * n_pairs, st));
    launch_set_u32(words + 1, (uint32_t)n_seg, st);
    ++*launches;
    static const char *kRoundName[3] = {"ar.round 0: build + render", "ar.round 1: build + render",
                                        "ar.round 2: build + render"};
    for (int r = 0; r < 3; ++r) {
        NvtxRange round_range(kRoundName[r]);
        uint32_t *cur_n = words + 1 + (r & 1), *nxt_n = words + 1 + ((r + 1) & 1);
        const uint32_t *cur = r == 0 ? rl.seg_order : (r == 1 && round1_order ? round1_order : act[(r - 1) & 1]);
        CK(cudaMemsetAsync(words, 0, sizeof(uint32_t), st));
        CK(cudaMemsetAsync(nxt_n, 0, sizeof(uint32_t), st));
        CK(cudaMemsetAsync(words + 3, 0, 2 * sizeof(uint32_t), st));
        launch_demand(cur, cur_n, (uint32_t)n_seg, rl.seg_start, rl.seg_end, rl.ent_ev, rl.ev_val, kWindow[r], state,
                      wlist, words, st);
        if (launch_record_build(M, vN, cc, cells, rl.n_gauss, wlist, words, rl.recs, build_counters, split_list,
                                words + 3, (uint32_t)n_pairs, words + 4, st))
            return fail(AR_EDEVICE, "record build launch: %s", cudaGetErrorString(cudaGetLastError()));
        *launches += 2;
        if (ev) CK(record_stage(ev[2 * r], st));
        rl.active = cur;
        rl.n_active = cur_n;
        rl.window = kWindow[r];
        rl.next_active = act[r & 1];
        rl.n_next = nxt_n;
        rl.precise = precise_list;
        rl.n_precise = words + 5;
        rl.precise_mask = precise_mask;
        CK(cudaMemsetAsync(words + 5, 0, sizeof(uint32_t), st));
        rl.f64 = 0;
        rl.direct = rl.interleave && r == 0;
        if (launch_render(M, TS, rl, st))
            return fail(AR_EDEVICE, "render launch: %s", cudaGetErrorString(cudaGetLastError()));
        // the segments where some pixel met an evaluation needing FP64, swept
        // again from their start for those pixels by the FP64-capable
        // instance (window abandons go to the same next list)
        RenderLaunch rp = rl;
        rp.active = precise_list;
        rp.n_active = words + 5;
        rp.f64 = 1;
        rp.direct = 0;
        if (launch_render(M, TS, rp, st))
            return fail(AR_EDEVICE, "render launch: %s", cudaGetErrorString(cudaGetLastError()));
        if (ev) CK(record_stage(ev[2 * r + 1], st));
        *launches += 6;
        if (r == 0) {
            // the second binning phase: full lists for the segments that
            // left the first round (a window or their depth prefix ran out)
            if (two) {
                NvtxRange rebin_range("ar.bin: full lists of the segments left");
                BinOut full;
                if (run_rebin(*rebin, *first, act[0], words + 2, full, st, launches))
                    return fail(AR_EDEVICE, "second binning phase: %s", cudaGetErrorString(cudaGetLastError()));
                rl.ent_ev = full.ent_ev;
                round1_order = full.seg_order;
            }
            if (ev) CK(record_stage(ev[6], st));
        }
    }
    return AR_OK;
}

// The autotuner: for tile = 0, the first render of a scene at a given image
// size and number of pose variables times the whole pipeline on the first
// eight cells of the call for each candidate (tile edge, events per staged
// chunk): (16, 16), (16, 8), (16, 32), (8, 16).  Each candidate runs three
// times and keeps the faster of the last two, so that workspace growth and
// graph capture are not counted; the fastest is kept for every later render
// with the same key.
// Other tile edges and chunks move the bounds only by the early stop's 2e-5.
static const int kTuneCand[4][2] = {{16, 16}, {16, 8}, {16, 32}, {8, 16}};
static int tuned_tile(ar_scene *s, Workspace &ws, const ar_intrinsics *in, const ar_nominal_pose *pose,
                      const ar_pose_box *cells, int32_t n_cells, float *out_lo, float *out_hi, cudaStream_t st,
                      int64_t ws_limit, int *TS, int *CH)
{
    int m_active = 0;
    for (int k = 0; k < MAXV; ++k) {
        bool act = false;
        for (int c = 0; c < n_cells; ++c) act = act || cells[c].hi[k] > cells[c].lo[k];
        m_active += act;
    }
    const int M = m_active <= 1 ? 1 : (m_active <= 4 ? 4 : 6);
    std::lock_guard<std::mutex> lock(s->tune_mu);
    for (const TunedTile &t : s->tuned)
        if (t.W == in->width && t.H == in->height && t.M == M) {
            *TS = t.TS;
            *CH = t.CH;
            return AR_OK;
        }
    const int32_t k = n_cells < 8 ? n_cells : 8;
    float best = 0.f;
    int bi = 0;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int r = AR_OK;
    for (int c = 0; c < 4 && r == AR_OK; ++c)
        for (int rep = 0; rep < 3 && r == AR_OK; ++rep) {
            CK(cudaEventRecord(e0, st));
            r = render_core(s, ws, in, pose, cells, k, kTuneCand[c][0], out_lo, out_hi, st, false, nullptr, false,
                            ws_limit, kTuneCand[c][1]);
            CK(cudaEventRecord(e1, st));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (r == AR_ENOMEM && c > 0) {  // a candidate that does not fit is not chosen
                r = AR_OK;
                break;
            }
            if (rep >= 1 && ((c == 0 && rep == 1) || ms < best)) {
                best = ms;
                bi = c;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    RK(r);
    s->tuned.push_back(TunedTile{in->width, in->height, M, kTuneCand[bi][0], kTuneCand[bi][1]});
    *TS = kTuneCand[bi][0];
    *CH = kTuneCand[bi][1];
    return AR_OK;
}

// The per-call constants of a render; returns the number of pose variables
// the forms carry (1, 4 or 6): the active variables of the call, taken over
// all cells so that every batch agrees on the form slots.
static int call_const(const ar_scene *s, const ar_intrinsics *in, const ar_nominal_pose *pose,
                      const ar_pose_box *cells, int32_t n_cells, CallConst &cc)
{
    std::memset(&cc, 0, sizeof cc);
    int m_active = 0;
    for (int k = 0; k < MAXV; ++k) {
        bool act = false;
        for (int c = 0; c < n_cells; ++c) act = act || cells[c].hi[k] > cells[c].lo[k];
        cc.m_slot[k] = act ? m_active++ : -1;
    }
    cc.W = in->width; cc.H = in->height;
    cc.fx = in->fx; cc.fy = in->fy; cc.cx = in->cx; cc.cy = in->cy; cc.near_plane = in->near_plane;
    std::memcpy(cc.R0, pose->R_wc, sizeof cc.R0);
    std::memcpy(cc.t0, pose->t, sizeof cc.t0);
    cc.n_gauss = s->n;
    cc.n_cells = n_cells;
    return m_active <= 1 ? 1 : (m_active <= 4 ? 4 : 6);
}

int render_core(ar_scene *s, Workspace &ws, const ar_intrinsics *in, const ar_nominal_pose *pose,
                const ar_pose_box *cells, int32_t n_cells, int32_t tile, float *out_lo, float *out_hi,
                cudaStream_t st, bool profiling, ar_render_stats *stats, bool plain, int64_t ws_limit, int chunk)
{
    RK(validate_call(in, pose, cells, n_cells, tile));
    if (!out_lo || !out_hi) return fail(AR_EINVAL, "null output");
    CK(cudaSetDevice(s->device));
    int tuned_ch = (tile != 0 && s->chunk) ? s->chunk : 16;
    if (tile == 0 && !plain && s->n > 0)
        RK(tuned_tile(s, ws, in, pose, cells, n_cells, out_lo, out_hi, st, ws_limit, &tile, &tuned_ch));
    const int W = in->width, H = in->height;
    const int TS = tile ? tile : 16;
    // events per staged chunk of the FP32 sweep: the tuner's choice with tile
    // = 0, else 16 (the FP64 instance always stages 16)
    const int CH = plain ? 16 : (chunk ? chunk : (TS == 16 ? tuned_ch : 16));
    const size_t out_words = (size_t)n_cells * W * H * 3;
    ar_render_stats rs;
    std::memset(&rs, 0, sizeof rs);
    rs.tile = TS;
    rs.chunk = CH;
    rs.ms_prep = rs.ms_bin = rs.ms_render = rs.ms_total = rs.ms_build = -1.f;
    CallConst cc;
    const int M = call_const(s, in, pose, cells, n_cells, cc);
    rs.m_vars = M;
    if (s->n == 0) {
        CK(cudaMemsetAsync(out_lo, 0, out_words * sizeof(float), st));
        CK(cudaMemsetAsync(out_hi, 0, out_words * sizeof(float), st));
        ws.n_batches = 0;
        if (stats) *stats = rs;
        return AR_OK;
    }
    // cells per batch: the records of a batch stay within the workspace limit
    // (about a third of the workspace goes to records), and pairs below 2^31
    const size_t rec_bytes = (plain ? sizeof(double) : sizeof(float)) * rec_width(M) + 64;
    const size_t per_cell = rec_bytes * (size_t)s->n;
    const int64_t limit = ws_limit > 0 ? ws_limit : s->ws_limit;
    int64_t per_batch = (int64_t)((limit / 3) / (per_cell ? per_cell : 1));
    const int64_t pair_cap = (int64_t)(((1ull << 31) - 1) / (uint64_t)s->n);
    if (per_batch > pair_cap) per_batch = pair_cap;
    if (per_batch < 1) per_batch = 1;
    if (per_batch > n_cells) per_batch = n_cells;
    if (plain) per_batch = 1;  // the plain path: one cell per launch sequence
    const int n_batches = (int)((n_cells + per_batch - 1) / per_batch);
    // a batch whose tile entries would not fit 32-bit indices is split in two
    // (see below): room for that many more batches' counters and events
    const int max_batches = 2 * n_batches + 16;
    const int ntx = (W + TS - 1) / TS, nty = (H + TS - 1) / TS;
    if ((uint64_t)per_batch * (uint64_t)ntx * (uint64_t)nty >= (1ull << 31))
        return fail(AR_EINVAL, "too many (cell, tile) segments");
    if (!ws.h_counters) CK(cudaMallocHost(&ws.h_counters, 8 * sizeof(unsigned long long)));
    while ((int)ws.evs.size() < kEventsPerBatch * max_batches) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        ws.evs.push_back(e);
    }
    RK(ws.cells_lohi.ensure(sizeof(double) * 12 * n_cells));
    RK(ws.vN.ensure(sizeof(double) * VN_STRIDE * s->n));
    RK(ws.counters.ensure(sizeof(unsigned long long) * (8 + kCountersPerBatch * max_batches)));
    {
        std::vector<double> lohi((size_t)12 * n_cells);
        for (int c = 0; c < n_cells; ++c)
            for (int k = 0; k < MAXV; ++k) {
                lohi[(size_t)MAXV * c + k] = cells[c].lo[k];
                lohi[(size_t)MAXV * n_cells + (size_t)MAXV * c + k] = cells[c].hi[k];
            }
        CK(cudaMemcpyAsync(ws.cells_lohi.p, lohi.data(), sizeof(double) * lohi.size(), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));  // the host vector is released on return
    }
    const double *d_lo = ws.cells_lohi.as<double>(), *d_hi = d_lo + (size_t)MAXV * n_cells;
    RK(ws.whist.ensure(sizeof(uint32_t) * kHistWords));
    if (!ws.h_whist) CK(cudaMallocHost(&ws.h_whist, sizeof(uint32_t) * kHistWords));
    CK(cudaMemsetAsync(ws.whist.p, 0, sizeof(uint32_t) * kHistWords, st));
    CK(cudaMemsetAsync(ws.counters.as<unsigned long long>() + 8, 0, sizeof(unsigned long long) * kCountersPerBatch * max_batches, st));
    int launches = 0;
    NvtxRange call_range(plain ? "ar.render_abstract_plain_fp64" : "ar.render_abstract");
    if (launch_pose_prep(s->uw_lo, s->uw_hi, s->Mw, s->n, cc, ws.vN.as<double>(), st)) return fail(AR_EDEVICE, "pose_prep launch");
    ++launches;
    std::vector<std::pair<int, int>> batches;  // (first cell, cells)
    for (int c0 = 0; c0 < n_cells; c0 += (int)per_batch)
        batches.push_back({c0, (int)(c0 + per_batch <= n_cells ? per_batch : n_cells - c0)});
    for (size_t b = 0; b < batches.size(); ++b) {
        const int c0 = batches[b].first, nb = batches[b].second;
        CallConst cb = cc;
        cb.n_cells = nb;
        const size_t off = (size_t)c0 * W * H * 3;
        const int r = render_batch(s, ws, cb, M, TS, CH, d_lo + (size_t)MAXV * c0, d_hi + (size_t)MAXV * c0,
                                   out_lo + off, out_hi + off, st, profiling, (int)b, rs, launches, plain);
        if (r == kSplitBatch) {
            // more tile entries than 32-bit indices reach (its record prep ran,
            // nothing else was enqueued): the batch goes again as two halves
            if (nb == 1 || (int)batches.size() >= max_batches)
                return fail(AR_ENOMEM, "a cell's tile entries exceed the 32-bit index range");
            batches[b].second = nb / 2;
            batches.insert(batches.begin() + (long)b + 1, {c0 + nb / 2, nb - nb / 2});
            --b;
            continue;
        }
        RK(r);
    }
    if (!plain) {
        // for the next render's first window (read after its first synchronisation)
        CK(cudaMemcpyAsync(ws.h_whist, ws.whist.p, sizeof(uint32_t) * kHistWords, cudaMemcpyDeviceToHost, st));
        ws.whist_pending = true;
    }
    ws.n_batches = (int)batches.size();
    ws.fallback_prep = rs.n_fallback;
    ws.split_prep = rs.n_split;
    ws.built_prep = plain ? rs.n_records : 0;
    rs.n_launches = launches;
    if (stats) *stats = rs;
    return AR_OK;
}

int finish_stats(Workspace &ws, cudaStream_t st, bool profiling, ar_render_stats &rs)
{
    CK(cudaStreamSynchronize(st));
    if (ws.n_batches > 0 && ws.counters.p) {
        std::vector<unsigned long long> ev(kCountersPerBatch * ws.n_batches);
        CK(cudaMemcpy(ev.data(), ws.counters.as<unsigned long long>() + 8, sizeof(unsigned long long) * ev.size(),
                      cudaMemcpyDeviceToHost));
        rs.n_evaluated = rs.n_reevaluated = 0;
        rs.n_fallback = ws.fallback_prep;
        rs.n_built = ws.built_prep;
        rs.n_split = ws.split_prep;
        rs.n_restarted = 0;
        rs.n_fp64 = 0;
        rs.n_fp64_segments = 0;
        for (int b = 0; b < ws.n_batches; ++b) {
            const unsigned long long *c = &ev[(size_t)kCountersPerBatch * b];
            rs.n_evaluated += (int64_t)c[0];
            rs.n_reevaluated += (int64_t)c[1];
            rs.n_fallback += (int64_t)c[2];
            rs.n_built += (int64_t)c[3];
            rs.n_split += (int64_t)c[4];
            rs.n_restarted += (int64_t)c[5];
            rs.n_fp64 += (int64_t)c[6];
            rs.n_fp64_segments += (int64_t)c[7];
        }
    }
    if (profiling && ws.n_batches > 0) {
        rs.ms_prep = rs.ms_bin = rs.ms_render = rs.ms_build = 0.f;
        for (int b = 0; b < ws.n_batches; ++b) {
            float t;
            const cudaEvent_t *e = &ws.evs[kEventsPerBatch * b];
            CK(cudaEventElapsedTime(&t, e[0], e[1])); rs.ms_prep += t;
            CK(cudaEventElapsedTime(&t, e[1], e[2])); rs.ms_bin += t;
            // e[9]: the end of the second binning phase, after round 0
            CK(cudaEventElapsedTime(&t, e[4], e[9])); rs.ms_bin += t;
            for (int r = 0; r < 3; ++r) {
                CK(cudaEventElapsedTime(&t, r == 1 ? e[9] : e[2 + 2 * r], e[3 + 2 * r])); rs.ms_build += t;
                CK(cudaEventElapsedTime(&t, e[3 + 2 * r], e[4 + 2 * r])); rs.ms_render += t;
            }
        }
        CK(cudaEventElapsedTime(&rs.ms_total, ws.evs[0], ws.evs[kEventsPerBatch * (ws.n_batches - 1) + 8]));
    }
    return AR_OK;
}

}  // namespace ar

int ar_render_abstract(ar_scene *s, const ar_intrinsics *in, const ar_nominal_pose *pose, const ar_pose_box *cells,
                       int32_t n_cells, int32_t tile, float *out_lower, float *out_upper, void *stream)
{
    if (!s) return fail(AR_EINVAL, "scene is null");
    cudaStream_t st = (cudaStream_t)stream;
    int r = render_core(s, s->ws, in, pose, cells, n_cells, tile, out_lower, out_upper, st, s->profiling, &s->stats);
    s->stats_stream = st;
    return r;
}

// Device address of a host buffer of `bytes` bytes when its first and last
// byte are page-locked host memory mapped into `device`'s address space (one
// contiguous mapping), else null.  Pageable memory and device memory give null.
static float *mapped_host(float *p, size_t bytes, int device)
{
    if (!p || bytes == 0) return nullptr;
    cudaPointerAttributes a, b;
    char *last = (char *)p + (bytes - 1);
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess || cudaPointerGetAttributes(&b, last) != cudaSuccess) {
        cudaGetLastError();  // not a CUDA-known pointer: clear the error, use the copy path
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer || !b.devicePointer)
        return nullptr;
    if ((char *)b.devicePointer - (char *)a.devicePointer != (ptrdiff_t)(bytes - 1)) return nullptr;
    int dev_ok = 0;
    if (cudaDeviceGetAttribute(&dev_ok, cudaDevAttrCanMapHostMemory, device) != cudaSuccess || !dev_ok) return nullptr;
    return (float *)a.devicePointer;
}

int ar_render_abstract_host(ar_scene *s, const ar_intrinsics *in, const ar_nominal_pose *pose,
                            const ar_pose_box *cells, int32_t n_cells, int32_t tile, float *host_lower,
                            float *host_upper, void *stream)
{
    if (!s) return fail(AR_EINVAL, "scene is null");
    if (!host_lower || !host_upper) return fail(AR_EINVAL, "null output");
    RK(validate_call(in, pose, cells, n_cells, tile));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = sizeof(float) * 3 * (size_t)in->width * in->height * n_cells;
    CK(cudaSetDevice(s->device));
    // Page-locked, mapped buffers are written by the render kernel itself:
    // it only stores to its outputs, once per finished (cell, tile) segment,
    // so the transfer to the host runs while the render does instead of after
    // it.  Both ends of both buffers must lie in mapped host memory.
    float *map_lo = mapped_host(host_lower, bytes, s->device), *map_hi = mapped_host(host_upper, bytes, s->device);
    if (map_lo && map_hi && s->n > 0) {
        RK(render_core(s, s->ws, in, pose, cells, n_cells, tile, map_lo, map_hi, st, s->profiling, &s->stats));
        s->stats_stream = st;
        CK(cudaStreamSynchronize(st));
        return AR_OK;
    }
    RK(s->ws.out_lo.ensure(bytes));
    RK(s->ws.out_hi.ensure(bytes));
    RK(render_core(s, s->ws, in, pose, cells, n_cells, tile, s->ws.out_lo.as<float>(), s->ws.out_hi.as<float>(), st,
                   s->profiling, &s->stats));
    s->stats_stream = st;
    CK(cudaMemcpyAsync(host_lower, s->ws.out_lo.p, bytes, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(host_upper, s->ws.out_hi.p, bytes, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return AR_OK;
}

// true if [a, a + na) and [b, b + nb) (in floats) overlap
static bool overlaps(const float *a, size_t na, const float *b, size_t nb)
{
    const uintptr_t a0 = (uintptr_t)a, a1 = a0 + na * sizeof(float);
    const uintptr_t b0 = (uintptr_t)b, b1 = b0 + nb * sizeof(float);
    return a0 < b1 && b0 < a1;
}

int ar_bounds_union(const float *in_lower, const float *in_upper, int32_t n_cells, int32_t width, int32_t height,
                    float *out_lower, float *out_upper, void *stream)
{
    if (!in_lower || !in_upper || !out_lower || !out_upper) return fail(AR_EINVAL, "null argument");
    if (n_cells < 1) return fail(AR_EINVAL, "n_cells must be >= 1");
    if (width < 1 || height < 1 || width > 16384 || height > 16384) return fail(AR_EINVAL, "image size out of range");
    const size_t n = (size_t)3 * width * height, nin = n * (size_t)n_cells;
    if (overlaps(out_lower, n, in_lower, nin) || overlaps(out_lower, n, in_upper, nin) ||
        overlaps(out_upper, n, in_lower, nin) || overlaps(out_upper, n, in_upper, nin) ||
        overlaps(out_lower, n, out_upper, n))
        return fail(AR_EINVAL, "overlapping buffers");
    if (launch_bounds_union(in_lower, in_upper, n_cells, n, out_lower, out_upper, false, (cudaStream_t)stream))
        return fail(AR_EDEVICE, "bounds_union launch: %s", cudaGetErrorString(cudaGetLastError()));
    return AR_OK;
}

int ar_partition_piece(const ar_pose_box *box, const int32_t *parts, int64_t index, ar_pose_box *out)
{
    if (!box || !parts || !out) return fail(AR_EINVAL, "null argument");
    int64_t total = 1;
    for (int k = 0; k < MAXV; ++k) {
        if (parts[k] < 1) return fail(AR_EINVAL, "parts[%d] must be >= 1", k);
        total *= parts[k];
        if (total > (int64_t)1 << 24) return fail(AR_EINVAL, "more than 2^24 pieces");
    }
    if (index < 0 || index >= total) return fail(AR_EINVAL, "piece index out of range");
    int64_t r = index;  // multi-index, dimension 0 fastest
    for (int k = 0; k < MAXV; ++k) {
        const int64_t P = parts[k], i = r % P;
        r /= P;
        const double lo = box->lo[k], hi = box->hi[k], w = hi - lo;
        out->lo[k] = i == 0 ? lo : lo + w * (double)i / (double)P;
        out->hi[k] = i + 1 == P ? hi : lo + w * (double)(i + 1) / (double)P;
    }
    return AR_OK;
}

int ar_render_abstract_partitioned(ar_scene *s, const ar_intrinsics *in, const ar_nominal_pose *pose,
                                   const ar_pose_box *box, const int32_t *parts, int32_t tile, float *out_lower,
                                   float *out_upper, void *stream)
{
    if (!s || !parts) return fail(AR_EINVAL, "null argument");
    if (!out_lower || !out_upper) return fail(AR_EINVAL, "null output");
    RK(validate_call(in, pose, box, 1, tile));
    int64_t total = 1;
    for (int k = 0; k < MAXV; ++k) {
        if (parts[k] < 1) return fail(AR_EINVAL, "parts[%d] must be >= 1", k);
        if (parts[k] > 1 && !(box->hi[k] > box->lo[k])) return fail(AR_EINVAL, "parts[%d] > 1 on a point dimension", k);
        total *= parts[k];
        if (total > (int64_t)1 << 24) return fail(AR_EINVAL, "more than 2^24 pieces");
    }
    const size_t n = (size_t)3 * in->width * in->height;
    if (overlaps(out_lower, n, out_upper, n)) return fail(AR_EINVAL, "overlapping outputs");
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(s->device));
    // chunks of at most 64 pieces, and at most 2 GiB of chunk images
    int64_t chunk = 64;
    while (chunk > 1 && (size_t)chunk * n * sizeof(float) > ((size_t)1 << 30)) chunk /= 2;
    if (chunk > total) chunk = total;
    RK(s->ws.part_lo.ensure(sizeof(float) * n * (size_t)chunk));
    RK(s->ws.part_hi.ensure(sizeof(float) * n * (size_t)chunk));
    std::vector<ar_pose_box> cells((size_t)chunk);
    for (int64_t c0 = 0; c0 < total; c0 += chunk) {
        const int64_t nb = c0 + chunk <= total ? chunk : total - c0;
        for (int64_t q = 0; q < nb; ++q) RK(ar_partition_piece(box, parts, c0 + q, &cells[(size_t)q]));
        RK(render_core(s, s->ws, in, pose, cells.data(), (int32_t)nb, tile, s->ws.part_lo.as<float>(),
                       s->ws.part_hi.as<float>(), st, s->profiling, &s->stats));
        s->stats_stream = st;
        if (launch_bounds_union(s->ws.part_lo.as<float>(), s->ws.part_hi.as<float>(), (int)nb, n, out_lower, out_upper,
                                c0 > 0, st))
            return fail(AR_EDEVICE, "bounds_union launch: %s", cudaGetErrorString(cudaGetLastError()));
    }
    return AR_OK;
}

int ar_render_abstract_refined(ar_scene *s, const ar_intrinsics *in, const ar_nominal_pose *pose,
                               const ar_pose_box *box, int32_t rounds, int32_t tile, float *out_lower,
                               float *out_upper, ar_pose_box *leaves, int32_t leaves_cap, int32_t *n_leaves,
                               void *stream)
{
    if (!s) return fail(AR_EINVAL, "scene is null");
    if (!out_lower || !out_upper) return fail(AR_EINVAL, "null output");
    if (leaves_cap < 0 || (leaves_cap > 0 && !leaves)) return fail(AR_EINVAL, "bad leaves buffer");
    if (rounds < 0 || rounds > 12) return fail(AR_EINVAL, "rounds must be in [0, 12]");
    RK(validate_call(in, pose, box, 1, tile));
    const size_t n = (size_t)3 * in->width * in->height;
    if (overlaps(out_lower, n, out_upper, n)) return fail(AR_EINVAL, "overlapping outputs");
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(s->device));
    int64_t chunk = 64;
    while (chunk > 1 && (size_t)chunk * n * sizeof(float) > ((size_t)1 << 30)) chunk /= 2;
    const int PB = 64;  // partial sums per piece
    RK(s->ws.part_lo.ensure(sizeof(float) * n * (size_t)chunk));
    RK(s->ws.part_hi.ensure(sizeof(float) * n * (size_t)chunk));
    RK(s->ws.lvl_lo.ensure(sizeof(float) * n));
    RK(s->ws.lvl_hi.ensure(sizeof(float) * n));
    RK(s->ws.wpart.ensure(sizeof(double) * (size_t)chunk * PB));
    float *plo = s->ws.part_lo.as<float>(), *phi = s->ws.part_hi.as<float>();
    float *llo = s->ws.lvl_lo.as<float>(), *lhi = s->ws.lvl_hi.as<float>();
    std::vector<ar_pose_box> cur(1, *box);
    std::vector<double> width, part((size_t)chunk * PB);
    for (int r = 0; r <= rounds; ++r) {
        const int64_t L = (int64_t)cur.size();
        width.assign((size_t)L, 0.0);
        for (int64_t c0 = 0; c0 < L; c0 += chunk) {
            const int64_t nb = c0 + chunk <= L ? chunk : L - c0;
            RK(render_core(s, s->ws, in, pose, &cur[(size_t)c0], (int32_t)nb, tile, plo, phi, st, s->profiling,
                           &s->stats));
            s->stats_stream = st;
            if (launch_bounds_union(plo, phi, (int)nb, n, llo, lhi, c0 > 0, st))
                return fail(AR_EDEVICE, "bounds_union launch: %s", cudaGetErrorString(cudaGetLastError()));
            if (r < rounds) {  // the pieces' mean widths choose the next splits
                if (launch_width_partials(plo, phi, (int)nb, n, PB, s->ws.wpart.as<double>(), st))
                    return fail(AR_EDEVICE, "width launch: %s", cudaGetErrorString(cudaGetLastError()));
                CK(cudaMemcpyAsync(part.data(), s->ws.wpart.p, sizeof(double) * (size_t)nb * PB,
                                   cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                for (int64_t q = 0; q < nb; ++q) {
                    double w = 0.0;
                    for (int b = 0; b < PB; ++b) w += part[(size_t)q * PB + b];
                    width[(size_t)(c0 + q)] = w;
                }
            }
        }
        if (r == 0) {
            CK(cudaMemcpyAsync(out_lower, llo, sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(out_upper, lhi, sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
        } else if (launch_bounds_intersect(llo, lhi, n, out_lower, out_upper, st)) {
            return fail(AR_EDEVICE, "intersect launch: %s", cudaGetErrorString(cudaGetLastError()));
        }
        if (r == rounds) break;
        // split the looser half of the pieces (ties by index), each in two
        // halves along its widest pose dimension relative to the box
        std::vector<int64_t> order((size_t)L);
        for (int64_t i = 0; i < L; ++i) order[(size_t)i] = i;
        std::stable_sort(order.begin(), order.end(),
                         [&](int64_t a, int64_t b) { return width[(size_t)a] > width[(size_t)b]; });
        std::vector<char> split((size_t)L, 0);
        for (int64_t i = 0; i < (L + 1) / 2; ++i) split[(size_t)order[(size_t)i]] = 1;
        std::vector<ar_pose_box> next;
        next.reserve((size_t)(L + (L + 1) / 2));
        for (int64_t i = 0; i < L; ++i) {
            const ar_pose_box &c = cur[(size_t)i];
            int kbest = -1;
            double best = 0.0;
            for (int k = 0; k < MAXV; ++k) {
                const double bw = box->hi[k] - box->lo[k];
                if (!(bw > 0.0)) continue;
                const double rel = (c.hi[k] - c.lo[k]) / bw;
                if (rel > best) { best = rel; kbest = k; }
            }
            if (!split[(size_t)i] || kbest < 0) { next.push_back(c); continue; }
            const double mid = c.lo[kbest] + (c.hi[kbest] - c.lo[kbest]) / 2.0;
            ar_pose_box a = c, b = c;
            a.hi[kbest] = mid;
            b.lo[kbest] = mid;
            next.push_back(a);
            next.push_back(b);
        }
        cur.swap(next);
    }
    if (n_leaves) *n_leaves = (int32_t)cur.size();
    for (int64_t i = 0; i < (int64_t)cur.size() && i < leaves_cap; ++i) leaves[i] = cur[(size_t)i];
    return AR_OK;
}

int ar_last_render_stats(ar_scene *s, ar_render_stats *out)
{
    if (!s || !out) return fail(AR_EINVAL, "null argument");
    RK(finish_stats(s->ws, s->stats_stream, s->profiling, s->stats));
    *out = s->stats;
    return AR_OK;
}

int ar_render_abstract_plain_fp64(ar_scene *s, const ar_intrinsics *in, const ar_nominal_pose *pose,
                                  const ar_pose_box *cells, int32_t n_cells, int32_t tile, float *out_lower,
                                  float *out_upper, void *stream)
{
    if (!s) return fail(AR_EINVAL, "scene is null");
    cudaStream_t st = (cudaStream_t)stream;
    int r = render_core(s, s->ws, in, pose, cells, n_cells, tile, out_lower, out_upper, st, s->profiling, &s->stats,
                        true);
    s->stats_stream = st;
    return r;
}

int ar_render_concrete(ar_scene *s, const ar_intrinsics *in, const ar_nominal_pose *pose, const double *deltas,
                       int32_t n_poses, float *out, void *stream)
{
    if (!s) return fail(AR_EINVAL, "scene is null");
    if (!deltas || !out) return fail(AR_EINVAL, "null argument");
    if (n_poses < 1) return fail(AR_EINVAL, "n_poses must be >= 1");
    // the intrinsics and pose checks of the abstract render, on a point cell
    ar_pose_box pt;
    for (int k = 0; k < MAXV; ++k) pt.lo[k] = pt.hi[k] = 0.0;
    RK(validate_call(in, pose, &pt, 1, 16));
    for (int64_t i = 0; i < (int64_t)n_poses * MAXV; ++i)
        if (!std::isfinite(deltas[i])) return fail(AR_EINVAL, "non-finite pose delta");
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(s->device));
    Workspace &ws = s->ws;
    const int W = in->width, H = in->height, TS = 16;
    const int ntx = (W + TS - 1) / TS, nty = (H + TS - 1) / TS, n_tiles = ntx * nty;
    const size_t img = (size_t)W * H * 3;
    if (s->n == 0) {
        CK(cudaMemsetAsync(out, 0, sizeof(float) * img * n_poses, st));
        return AR_OK;
    }
    CallConst cc;
    std::memset(&cc, 0, sizeof cc);
    cc.W = W; cc.H = H;
    cc.fx = in->fx; cc.fy = in->fy; cc.cx = in->cx; cc.cy = in->cy; cc.near_plane = in->near_plane;
    std::memcpy(cc.R0, pose->R_wc, sizeof cc.R0);
    std::memcpy(cc.t0, pose->t, sizeof cc.t0);
    cc.n_cells = 1;
    cc.n_gauss = s->n;
    const uint64_t n = (uint64_t)s->n;
    if (!ws.h_counters) CK(cudaMallocHost(&ws.h_counters, 8 * sizeof(unsigned long long)));
    RK(ws.cells_lohi.ensure(sizeof(double) * MAXV * n_poses));
    RK(ws.cells.ensure(concrete_pose_bytes()));
    RK(ws.recs.ensure(sizeof(double) * concrete_rec_width() * n));
    RK(ws.boxes.ensure(sizeof(PixBox) * n));
    RK(ws.keys.ensure(sizeof(double) * 2 * n));
    RK(ws.counters.ensure(sizeof(unsigned long long) * 8));
    CK(cudaMemcpyAsync(ws.cells_lohi.p, deltas, sizeof(double) * MAXV * n_poses, cudaMemcpyHostToDevice, st));
    int launches = 0;
    for (int p = 0; p < n_poses; ++p) {
        float *o = out + img * p;
        CK(cudaMemsetAsync(ws.counters.p, 0, sizeof(unsigned long long) * 8, st));
        if (launch_concrete_pose(ws.cells_lohi.as<double>() + (size_t)MAXV * p, cc, ws.cells.p, st) ||
            launch_concrete_prep(s->uw, s->Mw, s->tau, s->opac, s->rgb, cc, ws.cells.p, TS, ws.recs.as<double>(),
                                 ws.boxes.as<PixBox>(), ws.keys.as<double>(), ws.counters.as<unsigned long long>(),
                                 st))
            return fail(AR_EDEVICE, "concrete prep launch: %s", cudaGetErrorString(cudaGetLastError()));
        CK(cudaMemcpyAsync(ws.h_counters, ws.counters.p, sizeof(unsigned long long) * 5, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const uint64_t ne = 2 * ws.h_counters[2], nent = 2 * ws.h_counters[3];
        if (ne == 0) {
            CK(cudaMemsetAsync(o, 0, sizeof(float) * img, st));
            continue;
        }
        if (nent >= (1ull << 32) - (1ull << 20)) return fail(AR_ENOMEM, "too many tile entries for one pose");
        BinOut bo;
        RK(bin_pairs(ws, ws.boxes.as<PixBox>(), ws.keys.as<double>(), n, n, 1, ne, nent, TS, ntx, n_tiles, st, bo,
                     launches));
        if (launch_concrete_render(ws.recs.as<double>(), ws.boxes.as<PixBox>(), ws.segs.as<uint32_t>(),
                                   ws.sege.as<uint32_t>(), bo.ent_ev, bo.ev_val, bo.ev_key, W, H, ntx, n_tiles, o, st))
            return fail(AR_EDEVICE, "concrete render launch: %s", cudaGetErrorString(cudaGetLastError()));
    }
    return AR_OK;
}

int ar_debug_records(ar_scene *s, const ar_intrinsics *in, const ar_nominal_pose *pose, const ar_pose_box *cell,
                     double *out)
{
    if (!s) return fail(AR_EINVAL, "null argument");
    RK(validate_call(in, pose, cell, 1, 16));
    CK(cudaSetDevice(s->device));
    if (s->n == 0) return AR_OK;
    Workspace &ws = s->ws;
    CallConst cc;
    const int M = call_const(s, in, pose, cell, 1, cc);
    const int64_t n = s->n;
    cudaStream_t st = 0;
    RK(ws.cells_lohi.ensure(sizeof(double) * 2 * MAXV));
    RK(ws.vN.ensure(sizeof(double) * VN_STRIDE * n));
    RK(ws.cells.ensure(cell_data_bytes(M)));
    RK(ws.recs.ensure(sizeof(float) * rec_width(M) * n));
    RK(ws.boxes.ensure(sizeof(PixBox) * n));
    RK(ws.keys.ensure(sizeof(double) * 2 * n));
    RK(ws.counters.ensure(sizeof(unsigned long long) * 8));
    double lohi[2 * MAXV];
    for (int k = 0; k < MAXV; ++k) { lohi[k] = cell->lo[k]; lohi[MAXV + k] = cell->hi[k]; }
    CK(cudaMemcpy(ws.cells_lohi.p, lohi, sizeof lohi, cudaMemcpyHostToDevice));
    CK(cudaMemset(ws.counters.p, 0, sizeof(unsigned long long) * 8));
    const double *d_lo = ws.cells_lohi.as<double>(), *d_hi = d_lo + MAXV;
    if (launch_pose_prep(s->uw_lo, s->uw_hi, s->Mw, s->n, cc, ws.vN.as<double>(), st) ||
        launch_cell_prep(M, d_lo, d_hi, cc, ws.cells.p, st) ||
        (s->cull_force != 0 && ws.clist.ensure(sizeof(uint32_t) * (cc.n_gauss + 1)) != AR_OK) ||
        launch_record_prep(M, ws.vN.as<double>(), s->gp, cc, ws.cells.p, 16, ws.recs.as<float>(),
                           ws.boxes.as<PixBox>(), ws.keys.as<double>(), ws.counters.as<unsigned long long>(), st,
                           s->cull_force != 0 ? ws.clist.as<uint32_t>() : nullptr,
                           s->cull_force != 0 ? ws.clist.as<uint32_t>() + cc.n_gauss : nullptr))
        return fail(AR_EDEVICE, "record prep launch: %s", cudaGetErrorString(cudaGetLastError()));
    if (!out) return AR_OK;  // (ar_debug_alpha: the device records are what it needs)
    const int w = rec_width(M);
    std::vector<PixBox> boxes((size_t)n);
    std::vector<double> keys((size_t)2 * n);
    std::vector<float> recs((size_t)w * n);
    CK(cudaMemcpy(boxes.data(), ws.boxes.p, sizeof(PixBox) * n, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(keys.data(), ws.keys.p, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(recs.data(), ws.recs.p, sizeof(float) * w * n, cudaMemcpyDeviceToHost));
    const int sc = rec_scalar_offset(M);
    for (int64_t g = 0; g < n; ++g) {
        double *o = out + 10 * g;
        const PixBox &b = boxes[(size_t)g];
        const bool valid = b.x0 >= 0;
        for (int k = 0; k < 10; ++k) o[k] = 0.0;
        if (!valid) continue;
        const float *r = &recs[(size_t)w * g];
        uint32_t flags;
        std::memcpy(&flags, &r[sc + 6], sizeof flags);
        o[0] = 1.0;
        o[1] = (flags & 2u) ? 1.0 : 0.0;
        o[2] = keys[2 * g];
        o[3] = keys[2 * g + 1];
        o[4] = b.x0; o[5] = b.x1; o[6] = b.y0; o[7] = b.y1;
        o[8] = r[sc + 7];
        o[9] = r[sc + 8];
    }
    return AR_OK;
}

int ar_debug_alpha(ar_scene *s, const ar_intrinsics *in, const ar_nominal_pose *pose, const ar_pose_box *cell,
                   int32_t n, const int64_t *gi, const int32_t *px, const int32_t *py, int32_t precision, double *out)
{
    constexpr int OW = 42, W_OUT = 40;
    if (!s || !out || (n > 0 && (!gi || !px || !py))) return fail(AR_EINVAL, "null argument");
    if (n < 0 || n > (1 << 20)) return fail(AR_EINVAL, "n must be in [0, 2^20]");
    if (precision < 0 || precision > 3) return fail(AR_EINVAL, "precision must be 0, 1, 2 or 3");
    for (int32_t t = 0; t < n; ++t)
        if (gi[t] < 0 || gi[t] >= s->n || px[t] < 0 || py[t] < 0 || px[t] >= in->width || py[t] >= in->height)
            return fail(AR_EINVAL, "triple %d out of range", t);
    RK(ar_debug_records(s, in, pose, cell, nullptr));
    if (n == 0) return AR_OK;
    Workspace &ws = s->ws;
    CallConst cc;
    const int M = call_const(s, in, pose, cell, 1, cc);
    // the value parts of the listed pairs (cell 0: pair index = Gaussian index);
    // pairs that reach no pixel keep their decision part only
    std::vector<PixBox> boxes((size_t)s->n);
    CK(cudaMemcpy(boxes.data(), ws.boxes.p, sizeof(PixBox) * s->n, cudaMemcpyDeviceToHost));
    std::vector<uint32_t> work;
    for (int32_t t = 0; t < n; ++t)
        if (boxes[(size_t)gi[t]].x0 >= 0) work.push_back((uint32_t)gi[t]);
    std::sort(work.begin(), work.end());
    work.erase(std::unique(work.begin(), work.end()), work.end());
    const uint32_t nw = (uint32_t)work.size();
    uint32_t *d_work = nullptr, *d_words = nullptr, *d_list = nullptr;
    int64_t *d_gi = nullptr;
    int32_t *d_px = nullptr, *d_py = nullptr;
    double *d_out = nullptr;
    int rc = AR_OK;
    auto cleanup = [&]() {
        cudaFree(d_work); cudaFree(d_words); cudaFree(d_list); cudaFree(d_gi); cudaFree(d_px); cudaFree(d_py);
        cudaFree(d_out);
    };
    if (cudaMalloc(&d_work, sizeof(uint32_t) * (nw + 1)) != cudaSuccess ||
        cudaMalloc(&d_words, sizeof(uint32_t) * 8) != cudaSuccess ||
        cudaMalloc(&d_list, sizeof(uint32_t) * (nw + 1)) != cudaSuccess ||
        cudaMalloc(&d_gi, sizeof(int64_t) * n) != cudaSuccess || cudaMalloc(&d_px, sizeof(int32_t) * n) != cudaSuccess ||
        cudaMalloc(&d_py, sizeof(int32_t) * n) != cudaSuccess ||
        cudaMalloc(&d_out, sizeof(double) * OW * n) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return fail(AR_ENOMEM, "debug buffers");
    }
    uint32_t words[8] = {nw, 0, 0, 0, 0, 0, 0, 0};
    if (cudaMemcpy(d_work, work.data(), sizeof(uint32_t) * nw, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_words, words, sizeof words, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_gi, gi, sizeof(int64_t) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_px, px, sizeof(int32_t) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_py, py, sizeof(int32_t) * n, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = fail(AR_EDEVICE, "debug copies: %s", cudaGetErrorString(cudaGetLastError()));
    if (rc == AR_OK && nw > 0 &&
        launch_record_build(M, ws.vN.as<double>(), cc, ws.cells.p, s->n, d_work, d_words, ws.recs.as<float>(), nullptr,
                            d_list, d_words + 3, nw, d_words + 4, 0))
        rc = fail(AR_EDEVICE, "record build launch: %s", cudaGetErrorString(cudaGetLastError()));
    if (rc == AR_OK &&
        launch_debug_alpha(M, ws.recs.as<float>(), n, d_gi, d_px, d_py, precision, s->fp64_dev, d_out, 0))
        rc = fail(AR_EDEVICE, "debug launch: %s", cudaGetErrorString(cudaGetLastError()));
    std::vector<double> h((size_t)OW * n);
    if (rc == AR_OK && cudaMemcpy(h.data(), d_out, sizeof(double) * OW * n, cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = fail(AR_EDEVICE, "debug read-back: %s", cudaGetErrorString(cudaGetLastError()));
    cleanup();
    if (rc != AR_OK) return rc;
    // coefficients by pose dimension (slot order -> dimension order)
    for (int32_t t = 0; t < n; ++t) {
        const double *g = &h[(size_t)OW * t];
        double *o = out + (size_t)W_OUT * t;
        for (int k = 0; k < W_OUT; ++k) o[k] = 0.0;
        if (boxes[(size_t)gi[t]].x0 < 0) continue;
        for (int k = 0; k < MAXV; ++k) {
            const int sl = cc.m_slot[k];
            o[k] = sl >= 0 ? g[sl] : 0.0;
            o[7 + k] = sl >= 0 ? g[7 + sl] : 0.0;
        }
        o[6] = g[6];
        o[13] = g[13];
        for (int k = 14; k < 21; ++k) o[k] = g[k];   // rL rU alo ahi dev mlo mhi
        for (int k = 21; k < 39; ++k) o[k] = g[k];   // W, S, Rx, Ry intervals
        o[39] = 1.0 + 2.0 * g[40] + 4.0 * (((uint32_t)g[39] & 1u) != 0);  // valid, FP64 taken, fallback
    }
    return AR_OK;
}
