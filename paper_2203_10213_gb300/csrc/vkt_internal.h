// vkt_internal.h -- host-side structures shared by the runtime and the kernel launchers.
#pragma once

#include <utility>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "vkt.h"

#define VKT_VOLUME_MAGIC 0x564B5456u   // "VKTV"
#define VKT_FILTER_MAGIC 0x564B5446u   // "VKTF"

struct vktStructuredVolume_impl {
    uint32_t magic;
    void* data;          // device pointer
    int owning;          // 1: cudaMalloc'ed by Create, freed by Destroy
    int32_t dims[3];
    vktDataFormat format;
    float cell[3];
    float lo, hi;
};

struct vktFilter_impl {
    uint32_t magic;
    int32_t k;
    int separable;
    float w[VKT_MAX_FILTER_SIZE * VKT_MAX_FILTER_SIZE * VKT_MAX_FILTER_SIZE];  // dense, x fastest
    float g[3][VKT_MAX_FILTER_SIZE];   // separable vectors (x, y, z)
};

namespace vkt {

// An NVTX range named after a public call, open for the call's host-side duration (a
// profiler's timeline shows each call and the launches it enqueues; without a tool attached
// the push and pop return at once).
struct CallRange {
    explicit CallRange(const char* name) { nvtxRangePushA(name); }
    ~CallRange() { nvtxRangePop(); }
    CallRange(const CallRange&) = delete;
    CallRange& operator=(const CallRange&) = delete;
};

// One filter application as the kernels see it.
struct Job {
    // every member starts at zero, so a job left partly unset filters the whole volume
    const void* src = nullptr;
    void* dst = nullptr;
    int nx = 0, ny = 0, nz = 0;
    int sfmt = 0, dfmt = 0;     // vktDataFormat values
    // Epilogue: the kernels accumulate acc = sum w * q over stored source values q and
    // write a0 + a1*acc (float dst), or clamp(rint(a0 + a1*acc), 0, qmax) (integer dst).
    float a0 = 0.f, a1 = 0.f, qmax = 0.f;
    // Compensated accumulation (integer destinations, direct and separable paths): set when
    // an FP32 error bound does not keep the code within 5e-4 LSB of exact; a0lo/a1lo carry
    // the low halves of a0/a1 as double-float pairs.
    int comp = 0;
    float a0lo = 0.f, a1lo = 0.f;
    // Output region of interest (Sec. 3.2, "range" algorithms): when roi is set, only voxels
    // in [rx0, rx1) x [ry0, ry1) x [rz0, rz1) (cell coordinates) are written; the taps still
    // read the real neighbours, clamped at the volume's faces.  Otherwise the whole volume.
    int roi = 0;
    int rx0 = 0, ry0 = 0, rz0 = 0, rx1 = 0, ry1 = 0, rz1 = 0;
    // A batch of nvol volumes with equal dims and formats filtered by one launch (direct
    // path): volume v's source starts vs_src voxels after src, its destination vs_dst voxels
    // after dst.
    int nvol = 1;
    int64_t vs_src = 0, vs_dst = 0;
    // Planes per z chunk of a brick (direct and separable paths); 0: the launcher's rule.
    // The chunking changes no result, only the launch shape (the autotuner sets it).
    int zchunk = 0;
};

// the output region of a job as [x0, x1) x [y0, y1) x [z0, z1)
inline void job_region(const Job& j, int& x0, int& y0, int& z0, int& x1, int& y1, int& z1)
{
    if (j.roi) {
        x0 = j.rx0; y0 = j.ry0; z0 = j.rz0;
        x1 = j.rx1; y1 = j.ry1; z1 = j.rz1;
    } else {
        x0 = y0 = z0 = 0;
        x1 = j.nx; y1 = j.ny; z1 = j.nz;
    }
}

// Planes per z chunk for a grid of `tiles` column tiles (over all volumes of a batch, and
// all kernel planes of the weight gradient) of ez planes each: about 8 CTAs per SM in total,
// with chunks of at least 8 planes while that still gives at least one CTA per SM; smaller
// jobs take shorter chunks (down to one plane, read with its halo planes from L2) until
// there are about two CTAs per SM.
inline int zchunk_for(long tiles, int ez, int sms)
{
    tiles = tiles < 1 ? 1 : tiles;
    const long target = static_cast<long>(sms) * 8;
    const long cap8 = ez / 8 < 1 ? 1 : ez / 8;
    long chunks = (target + tiles - 1) / tiles;
    if (tiles * cap8 >= sms) {
        chunks = chunks < cap8 ? chunks : cap8;
    } else {
        const long two = (2L * sms + tiles - 1) / tiles;
        chunks = chunks < ez ? chunks : ez;
        chunks = chunks < two ? chunks : two;
    }
    chunks = chunks < 1 ? 1 : chunks;
    return static_cast<int>((ez + chunks - 1) / chunks);
}

// z planes per CTA for `tiles` column tiles over ez planes, with `slots` CTAs resident at
// once (SMs x CTAs per SM) and r halo planes on each side of a chunk: the chunk count whose
// launch takes the least estimated time, waves x (planes per chunk + 2r), at least 8 planes
// per chunk; ties go to fewer chunks (less halo).
inline int zchunk_waves(long tiles, int ez, long slots, int r)
{
    slots = slots < 1 ? 1 : slots;
    const long cap = ez / 8 < 1 ? 1 : ez / 8;
    long best_cost = -1;
    int best = ez;
    for (long chunks = 1; chunks <= cap; ++chunks) {
        const long z = (ez + chunks - 1) / chunks;
        const long real = (ez + z - 1) / z;
        const long waves = (tiles * real + slots - 1) / slots;
        const long cost = waves * (z + 2 * r);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = static_cast<int>(z);
        }
    }
    return best;
}

// The z chunk of a z-marching kernel (direct, adjoint): the wave-aware choice while chunks of
// at least 8 planes still give every SM a CTA, else the short chunks of zchunk_for.
inline int zchunk_direct(long tiles, int ez, int sms, int per_sm, int r)
{
    tiles = tiles < 1 ? 1 : tiles;
    const long cap8 = ez / 8 < 1 ? 1 : ez / 8;
    if (tiles * cap8 >= sms) return zchunk_waves(tiles, ez, static_cast<long>(sms) * per_sm, r);
    return zchunk_for(tiles, ez, sms);
}

// Launches `kern` with programmatic stream serialization: the kernel may start while the
// previous kernel on the stream finishes, and must call grid_dependency_wait() before it
// touches global memory.
template <typename... Params, typename... Args>
cudaError_t launch_pdl(void (*kern)(Params...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t stream, Args&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// bits of the device status word (Ctx::status), reported by vktSynchronize
constexpr unsigned STATUS_TIMEOUT = 1u;   // a bounded device wait gave up
constexpr unsigned STATUS_CONFIG = 2u;    // a kernel found its launch inconsistent with its build

struct Ctx {
    cudaStream_t stream;
    int debug;
    unsigned* status;   // device status word of the current device
    int device;         // the current device and its SM count
    int sms;
};

// Sets `kern`'s dynamic shared memory limit to `smem` and returns its resident CTAs per SM
// at `threads` threads (at least 1), once per (device, kernel, smem); later calls read the
// remembered answer instead of asking the driver again.
vktError prepare_kernel(const Ctx& ctx, const void* kern, int threads, size_t smem, int* per_sm);

// Kernel launchers (each returns VKT_NO_ERROR or a launch error).  launch_direct takes
// the compensated kernels when job.comp is set (launch_direct_comp).
vktError launch_direct(const Job& job, const float* w, int k, const Ctx& ctx);
vktError launch_direct_comp(const Job& job, const float* w, int k, const Ctx& ctx);
// dL/dsrc of the clamped correlation (float32 gy in job.src, gx in job.dst): every voxel of
// gx is written (the main launch), then the shell outside the volume is added to the face
// voxels (a second, small launch).
vktError launch_adjoint(const Job& job, const float* w, int k, const Ctx& ctx);
// dL/dw summed over nvol volumes of equal dims (volume v of x at x + v vs_x, of gy at
// gy + v vs_gy): per-CTA FP32 partial sums into `partials` (capacity `cap` floats), then
// one FP64 reduction over all of them into gw (k^3 floats).  `partials` is caller-provided
// scratch of weight_grad_scratch_floats(..., nvol) floats.
vktError launch_weight_grad(const float* x, const float* gy, int nx, int ny, int nz, int k,
                            float* partials, size_t cap, float* gw, const Ctx& ctx, int nvol = 1,
                            int64_t vs_x = 0, int64_t vs_gy = 0);
size_t weight_grad_scratch_floats(int nx, int ny, int nz, int k, int nvol = 1);
// The partial sums only (no reduction), for volumes that are not evenly spaced: one launch
// per volume into its own slice, then reduce_weight_grad once over all slices.
vktError launch_weight_grad_partials(const float* x, const float* gy, int nx, int ny, int nz,
                                     int k, float* partials, const Ctx& ctx);
vktError reduce_weight_grad(const float* partials, size_t nspatial, int k, float* gw,
                            const Ctx& ctx);
vktError launch_separable(const Job& job, const float* gx, const float* gy, const float* gz,
                          int k, const Ctx& ctx);

// Tensor-core path: VKT_NO_ERROR if it can evaluate this triple, else why not.
vktError tensor_available(const vktStructuredVolume_impl* dst, const vktStructuredVolume_impl* src,
                          const vktFilter_impl* f);
vktError launch_tensor(const Job& job, const float* w, int k, const Ctx& ctx);

// Whether a separable filter into an integer destination needs compensated accumulation.
bool separable_needs_comp(const vktStructuredVolume_impl* dst, const vktStructuredVolume_impl* src,
                          const vktFilter_impl* f);
// The same for the direct path with the filter's dense weights.
bool direct_needs_comp(const vktStructuredVolume_impl* dst, const vktStructuredVolume_impl* src,
                       const vktFilter_impl* f);

// Volumes whose data lie evenly spaced, `stride` voxels apart (one volume: stride 0).
bool evenly_spaced(int32_t n, const vktStructuredVolume* v, int64_t* stride);
// The one-launch form of a batch that shares one filter over equal, evenly spaced volumes
// (direct path); *handled is false when the batch does not qualify.
vktError apply_filter_multi(int32_t n, vktStructuredVolume* dst, vktStructuredVolume* src,
                            vktFilter* filters, bool* handled);

// Helpers provided by the runtime.
vktError get_context(Ctx* ctx);
void count_launches(unsigned n);
void uncount_launches(unsigned n);   // launches that were captured into a graph, not run
vktError from_cuda(cudaError_t e);
// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link).
bool encode_tensor_map_3d(void* map /* CUtensorMap* */, int fmt, const void* base, int nx,
                          int ny, int nz, int boxx, int boxy, int boxz);
// The same as a 4-D map (x, y, z, volume) of nvol >= 1 volumes of nx x ny x nz voxels,
// vstride voxels apart (vstride >= nx ny nz and a multiple of 16 bytes; 0 for one volume).
// nvol == 0 gives the 3-D map of encode_tensor_map_3d.
bool encode_tensor_map(void* map, int fmt, const void* base, int nx, int ny, int nz, int nvol,
                       int64_t vstride, int boxx, int boxy, int boxz);

// Autotuner (vkt_tune.cu).  A choice for one call shape: the evaluation path and the z
// chunk of the CUDA-core paths (0: the rule), or for a batch its brick z extent and its
// persistent grid's CTAs per SM (0: as many as fit).
struct TuneChoice {
    int path = 0;
    int zchunk = 0;
    float ms = 0.f;
};
bool autotune_enabled();
bool autotune_lookup(const char* key, TuneChoice* c);
void autotune_store(const char* key, const TuneChoice& c);
// Whether work enqueued on `stream` now would be captured into a graph (no timing then).
bool stream_capturing(cudaStream_t stream);
// Times run(candidate) for every candidate on `stream` and returns the fastest in *best
// (VKT_ERROR_UNSUPPORTED when none ran); candidate 0 is the rule.  Two passes over the
// candidates, each launching a candidate once untimed and three times between CUDA events;
// a candidate's time is its faster pass (interleaving the passes keeps a drift of the
// clocks or of the memory system from favouring one candidate), and the rule stays the
// choice unless another candidate is more than 2 % faster.  Synchronises the stream.
template <class Run>
vktError autotune_time(const TuneChoice* cand, int n, Run run, cudaStream_t stream, TuneChoice* best)
{
    constexpr int MAXC = 16;
    if (n < 1 || n > MAXC) return VKT_ERROR_INVALID_VALUE;
    cudaEvent_t ev[2];
    if (cudaEventCreate(&ev[0]) != cudaSuccess) return from_cuda(cudaGetLastError());
    if (cudaEventCreate(&ev[1]) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return from_cuda(cudaGetLastError());
    }
    float t[MAXC];
    bool ran[MAXC];
    for (int i = 0; i < n; ++i) {
        t[i] = 0.f;
        ran[i] = false;
    }
    vktError err = VKT_NO_ERROR;
    for (int pass = 0; pass < 2 && err == VKT_NO_ERROR; ++pass) {
        for (int i = 0; i < n; ++i) {
            if (pass == 1 && !ran[i]) continue;
            if (run(cand[i]) != VKT_NO_ERROR) continue;
            cudaEventRecord(ev[0], stream);
            vktError e2 = VKT_NO_ERROR;
            for (int r = 0; r < 3 && e2 == VKT_NO_ERROR; ++r) e2 = run(cand[i]);
            cudaEventRecord(ev[1], stream);
            if (cudaEventSynchronize(ev[1]) != cudaSuccess) {
                err = from_cuda(cudaGetLastError());
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[0], ev[1]);
            if (e2 != VKT_NO_ERROR) continue;
            ms *= 1.f / 3.f;
            t[i] = ran[i] ? (ms < t[i] ? ms : t[i]) : ms;
            ran[i] = true;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (err != VKT_NO_ERROR) return err;
    int b = -1;
    for (int i = 0; i < n; ++i)
        if (ran[i] && (b < 0 || t[i] < t[b])) b = i;
    if (b < 0) return VKT_ERROR_UNSUPPORTED;
    if (ran[0] && t[b] > 0.98f * t[0]) b = 0;   // the rule unless clearly slower
    *best = cand[b];
    best->ms = t[b];
    return VKT_NO_ERROR;
}

}  // namespace vkt
