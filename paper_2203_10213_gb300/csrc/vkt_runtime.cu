// vkt_runtime.cu -- the C ABI of vkt.h: handles, thread-local execution policy, argument
// validation, the value-mapping epilogue constants and the choice of evaluation path.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <new>
#include <string>
#include <vector>

#include "vkt_internal.h"

namespace vkt {

namespace {

thread_local vktExecutionPolicy t_policy = {nullptr, 0, 0, VKT_PATH_AUTO};
std::atomic<uint64_t> g_launches{0};

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
unsigned* g_status[MAX_DEVICES] = {};
int g_sms[MAX_DEVICES] = {};
// for prepare_kernel: (device, kernel, dynamic shared memory) -> resident CTAs per SM, and
// (device, kernel) -> the largest dynamic shared memory limit set so far (the limit is never
// lowered: a smaller setting would refuse a later launch that needs the larger one)
std::map<std::tuple<int, const void*, size_t>, int> g_prepared;
std::map<std::pair<int, const void*>, size_t> g_smem_limit;

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;
bool g_encode_tried = false;

bool valid(const vktStructuredVolume_impl* v) { return v && v->magic == VKT_VOLUME_MAGIC; }
bool valid(const vktFilter_impl* f) { return f && f->magic == VKT_FILTER_MAGIC; }

int fmt_bytes(vktDataFormat f) { return f == vktDataFormatUint8 ? 1 : (f == vktDataFormatUint16 ? 2 : 4); }
double fmt_qmax(vktDataFormat f) { return f == vktDataFormatUint8 ? 255.0 : 65535.0; }
bool fmt_valid(int f) { return f >= vktDataFormatUint8 && f <= vktDataFormatFloat32; }

uint64_t volume_bytes(const vktStructuredVolume_impl* v)
{
    return static_cast<uint64_t>(v->dims[0]) * v->dims[1] * v->dims[2] * fmt_bytes(v->format);
}

vktError check_device()
{
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        cudaGetLastError();
        return VKT_ERROR_NO_DEVICE;
    }
    return VKT_NO_ERROR;
}

vktError check_volume_args(int32_t dx, int32_t dy, int32_t dz, vktDataFormat format, float sx,
                           float sy, float sz, float lo, float hi)
{
    if (dx < 1 || dy < 1 || dz < 1) return VKT_ERROR_INVALID_VALUE;
    if (!fmt_valid(format)) return VKT_ERROR_INVALID_VALUE;
    if (!(sx > 0.f) || !(sy > 0.f) || !(sz > 0.f)) return VKT_ERROR_INVALID_VALUE;
    if (!std::isfinite(lo) || !std::isfinite(hi)) return VKT_ERROR_INVALID_VALUE;
    if (format != vktDataFormatFloat32 && lo == hi) return VKT_ERROR_INVALID_VALUE;
    return VKT_NO_ERROR;
}

vktError check_filter_size(int32_t k)
{
    if (k < 1 || k > VKT_MAX_FILTER_SIZE || (k & 1) == 0) return VKT_ERROR_UNSUPPORTED;
    return VKT_NO_ERROR;
}

void dense_from_separable(vktFilter_impl* f)
{
    const int k = f->k;
    for (int c = 0; c < k; ++c)
        for (int b = 0; b < k; ++b)
            for (int a = 0; a < k; ++a)
                f->w[(c * k + b) * k + a] = static_cast<float>(
                    static_cast<double>(f->g[2][c]) * f->g[1][b] * f->g[0][a]);
}

bool overlaps(const vktStructuredVolume_impl* a, const vktStructuredVolume_impl* b)
{
    const char* pa = static_cast<const char*>(a->data);
    const char* pb = static_cast<const char*>(b->data);
    return pa < pb + volume_bytes(b) && pb < pa + volume_bytes(a);
}

// Epilogue constants of one (dst, src, filter-sum) triple.  The kernels accumulate over
// stored values q (codes for integer sources); the mapped result is
//   v = lo_s * W + s_s * acc,   W = sum of the weights, s_s = (hi_s - lo_s)/(2^N - 1)
// and an integer destination stores clamp(rint((v - lo_d) * (2^M - 1)/(hi_d - lo_d))).
// a0 + a1 * acc is that destination value (or code); the low halves give double-float pairs.
void epilogue(const vktStructuredVolume_impl* dst, const vktStructuredVolume_impl* src,
              double wsum, Job* job)
{
    double ls = 0.0, ss = 1.0;
    if (src->format != vktDataFormatFloat32) {
        ls = src->lo;
        ss = (static_cast<double>(src->hi) - src->lo) / fmt_qmax(src->format);
    }
    double a0, a1;
    if (dst->format == vktDataFormatFloat32) {
        a0 = ls * wsum;
        a1 = ss;
        job->qmax = 0.f;
    } else {
        const double sd = fmt_qmax(dst->format) / (static_cast<double>(dst->hi) - dst->lo);
        a0 = (ls * wsum - dst->lo) * sd;
        a1 = ss * sd;
        job->qmax = static_cast<float>(fmt_qmax(dst->format));
    }
    job->a0 = static_cast<float>(a0);
    job->a1 = static_cast<float>(a1);
    job->a0lo = static_cast<float>(a0 - static_cast<double>(job->a0));
    job->a1lo = static_cast<float>(a1 - static_cast<double>(job->a1));
    job->comp = 0;
}

}  // namespace

vktError get_context(Ctx* ctx)
{
    vktError err = check_device();
    if (err != VKT_NO_ERROR) return err;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return from_cuda(e);
    if (dev < 0 || dev >= MAX_DEVICES) return VKT_ERROR_UNSUPPORTED;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_status[dev]) {
            unsigned* p = nullptr;
            e = cudaMalloc(&p, 16);
            if (e != cudaSuccess) return from_cuda(e);
            e = cudaMemset(p, 0, 16);
            if (e != cudaSuccess) {
                cudaFree(p);
                return from_cuda(e);
            }
            g_status[dev] = p;
        }
        if (g_sms[dev] <= 0) {
            int n = 0;
            e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return from_cuda(e);
            g_sms[dev] = n > 0 ? n : 1;
        }
        ctx->status = g_status[dev];
        ctx->sms = g_sms[dev];
    }
    ctx->device = dev;
    ctx->stream = static_cast<cudaStream_t>(t_policy.stream);
    ctx->debug = t_policy.debug;
    return VKT_NO_ERROR;
}

vktError prepare_kernel(const Ctx& ctx, const void* kern, int threads, size_t smem, int* per_sm)
{
    const auto key = std::make_tuple(ctx.device, kern, smem);
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        auto it = g_prepared.find(key);
        if (it != g_prepared.end()) {
            *per_sm = it->second;
            return VKT_NO_ERROR;
        }
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    size_t& limit = g_smem_limit[std::make_pair(ctx.device, kern)];
    if (smem > limit) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   static_cast<int>(smem));
        if (e != cudaSuccess) return from_cuda(e);
        limit = smem;
    }
    int n = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 1;
    }
    g_prepared[key] = n;
    *per_sm = n;
    return VKT_NO_ERROR;
}

// Whether a separable filter into an integer destination needs compensated accumulation:
// an FP32 evaluation of the three passes (3k + 4 roundings, each at most 2^-24 of a value
// bounded by sum|gx| sum|gy| sum|gz| max|v|) must stay below 5e-4 of a destination code, or
// a rounding decision outside the 1e-3 LSB tie window could flip.  A float32 source has no
// known bound on |v| and always takes the compensated path.
bool separable_needs_comp(const vktStructuredVolume_impl* dst, const vktStructuredVolume_impl* src,
                          const vktFilter_impl* f)
{
    if (dst->format == vktDataFormatFloat32) return false;
    if (src->format == vktDataFormatFloat32) return true;
    double s[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i < f->k; ++i) s[a] += std::fabs(static_cast<double>(f->g[a][i]));
    const double vmax = std::max(std::fabs(static_cast<double>(src->lo)), std::fabs(static_cast<double>(src->hi)));
    const double sd = fmt_qmax(dst->format) / std::fabs(static_cast<double>(dst->hi) - dst->lo);
    const double bound = (3.0 * f->k + 4.0) * std::ldexp(1.0, -24) * s[0] * s[1] * s[2] * vmax * sd;
    return bound >= 5e-4;
}

// Whether a dense filter into an integer destination needs compensated accumulation.  The
// direct kernel sums t = sum_d w_d q_d over stored source values q (codes, |q| <= Qs) in
// k^3 FP32 additions, then forms the code a0 + a1 t with one fma (a1 = (hi_s - lo_s)/Qs * sd,
// sd = qmax_d / (hi_d - lo_d), both rounded to float32).  With u = 2^-24 the code's error is
// at most u sd ((k^3 + 1) sum|w| |hi_s - lo_s| + |lo_s| sum|w| + |lo_d|) + u (qmax_d + 1):
// the sum's k^3 roundings and the rounding of a1 (each relative to sum|w| Qs, scaled by
// a1), the rounding of a0, and the fma's own.  Below 5e-4 of a code, a rounding decision
// outside the 1e-3 LSB tie window cannot flip; otherwise the kernel accumulates Dot2
// pairs.  A float32 source has no known bound on |q| and always takes the compensated
// kernel.
bool direct_needs_comp(const vktStructuredVolume_impl* dst, const vktStructuredVolume_impl* src,
                       const vktFilter_impl* f)
{
    if (dst->format == vktDataFormatFloat32) return false;
    if (src->format == vktDataFormatFloat32) return true;
    const int kkk = f->k * f->k * f->k;
    double sw = 0.0;
    for (int i = 0; i < kkk; ++i) sw += std::fabs(static_cast<double>(f->w[i]));
    const double srange = std::fabs(static_cast<double>(src->hi) - src->lo);
    const double qd = fmt_qmax(dst->format);
    const double sd = qd / std::fabs(static_cast<double>(dst->hi) - dst->lo);
    const double u = std::ldexp(1.0, -24);
    const double bound = u * sd * ((kkk + 1.0) * sw * srange +
                                   std::fabs(static_cast<double>(src->lo)) * sw +
                                   std::fabs(static_cast<double>(dst->lo))) +
                         u * (qd + 1.0);
    return bound >= 5e-4;
}

// Volumes b = 0..n-1 whose data lie `stride` voxels apart (data[b] = data[0] + b stride,
// stride >= the volume's size): one launch can then address them all.  One volume is evenly
// spaced with stride 0.
bool evenly_spaced(int32_t n, const vktStructuredVolume* v, int64_t* stride)
{
    *stride = 0;
    if (n <= 1) return true;
    const int es = fmt_bytes(v[0]->format);
    const intptr_t d = static_cast<const char*>(v[1]->data) - static_cast<const char*>(v[0]->data);
    if (d <= 0 || d % es != 0 || static_cast<uint64_t>(d) < volume_bytes(v[0])) return false;
    for (int32_t b = 2; b < n; ++b)
        if (static_cast<const char*>(v[b]->data) - static_cast<const char*>(v[0]->data) !=
            static_cast<intptr_t>(d) * b)
            return false;
    *stride = d / es;
    return true;
}

void count_launches(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void uncount_launches(unsigned n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }

vktError from_cuda(cudaError_t e)
{
    switch (e) {
    case cudaSuccess: return VKT_NO_ERROR;
    case cudaErrorMemoryAllocation: cudaGetLastError(); return VKT_ERROR_OUT_OF_MEMORY;
    case cudaErrorNoDevice:
    case cudaErrorInsufficientDriver: cudaGetLastError(); return VKT_ERROR_NO_DEVICE;
    default: cudaGetLastError(); return VKT_ERROR_CUDA;
    }
}

bool encode_tensor_map_3d(void* map, int fmt, const void* base, int nx, int ny, int nz,
                          int boxx, int boxy, int boxz)
{
    return encode_tensor_map(map, fmt, base, nx, ny, nz, 0, 0, boxx, boxy, boxz);
}

bool encode_tensor_map(void* map, int fmt, const void* base, int nx, int ny, int nz, int nvol,
                       int64_t vstride, int boxx, int boxy, int boxz)
{
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_encode_tried) {
            g_encode_tried = true;
            void* fn = nullptr;
            cudaDriverEntryPointQueryResult q;
            if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                 cudaEnableDefault, &q) == cudaSuccess &&
                q == cudaDriverEntryPointSuccess)
                g_encode = reinterpret_cast<EncodeTiledFn>(fn);
            cudaGetLastError();
        }
    }
    if (!g_encode) return false;
    const int es = fmt == vktDataFormatUint8 ? 1 : (fmt == vktDataFormatUint16 ? 2 : 4);
    if (reinterpret_cast<uintptr_t>(base) % 16 != 0) return false;
    if ((static_cast<uint64_t>(nx) * es) % 16 != 0) return false;
    if (boxx > 256 || boxy > 256 || boxz > 256 || (boxx * es) % 16 != 0) return false;
    const CUtensorMapDataType dt = fmt == vktDataFormatUint8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                   : fmt == vktDataFormatUint16 ? CU_TENSOR_MAP_DATA_TYPE_UINT16
                                                                : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    // nvol > 0: a 4-D map whose fourth dimension counts nvol volumes vstride voxels apart
    // (one volume: vstride 0 stands for the volume's own size); nvol == 0: a 3-D map
    const int rank = nvol > 0 ? 4 : 3;
    if (rank == 4 && nvol == 1 && vstride == 0) vstride = static_cast<int64_t>(nx) * ny * nz;
    if (rank == 4 && ((vstride * es) % 16 != 0 || vstride < static_cast<int64_t>(nx) * ny * nz))
        return false;
    cuuint64_t dims[4] = {static_cast<cuuint64_t>(nx), static_cast<cuuint64_t>(ny),
                          static_cast<cuuint64_t>(nz),
                          static_cast<cuuint64_t>(nvol > 0 ? nvol : 1)};
    cuuint64_t strides[3] = {static_cast<cuuint64_t>(nx) * es,
                             static_cast<cuuint64_t>(nx) * ny * es,
                             static_cast<cuuint64_t>(vstride) * es};
    cuuint32_t box[4] = {static_cast<cuuint32_t>(boxx), static_cast<cuuint32_t>(boxy),
                         static_cast<cuuint32_t>(boxz), 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = g_encode(static_cast<CUtensorMap*>(map), dt, rank, const_cast<void*>(base), dims,
                          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace vkt

using namespace vkt;

extern "C" {

vktError vktSetThreadExecutionPolicy(vktExecutionPolicy policy)
{
    if (policy.path < VKT_PATH_AUTO || policy.path > VKT_PATH_TENSOR) return VKT_ERROR_INVALID_VALUE;
    t_policy = policy;
    return VKT_NO_ERROR;
}

vktError vktGetThreadExecutionPolicy(vktExecutionPolicy* policy)
{
    if (!policy) return VKT_ERROR_INVALID_VALUE;
    *policy = t_policy;
    return VKT_NO_ERROR;
}

const char* vktGetErrorString(vktError error)
{
    switch (error) {
    case VKT_NO_ERROR: return "no error";
    case VKT_ERROR_INVALID_VALUE: return "invalid value";
    case VKT_ERROR_INVALID_HANDLE: return "invalid handle";
    case VKT_ERROR_DIMS_MISMATCH: return "volume dims mismatch";
    case VKT_ERROR_UNSUPPORTED: return "unsupported filter size, format or path";
    case VKT_ERROR_OUT_OF_MEMORY: return "out of device memory";
    case VKT_ERROR_NO_DEVICE: return "no CUDA device";
    case VKT_ERROR_CUDA: return "CUDA error";
    case VKT_ERROR_DEVICE_TIMEOUT: return "a bounded device wait timed out";
    default: return "unknown error";
    }
}

vktError vktSynchronize(void)
{
    Ctx ctx;
    vktError err = get_context(&ctx);
    if (err != VKT_NO_ERROR) return err;
    cudaError_t e = cudaStreamSynchronize(ctx.stream);
    if (e != cudaSuccess) return from_cuda(e);
    unsigned st = 0;
    e = cudaMemcpyAsync(&st, ctx.status, sizeof(st), cudaMemcpyDeviceToHost, ctx.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx.stream);
    if (e != cudaSuccess) return from_cuda(e);
    if (st != 0) {
        e = cudaMemsetAsync(ctx.status, 0, sizeof(st), ctx.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx.stream);
        if (e != cudaSuccess) return from_cuda(e);
        return (st & STATUS_TIMEOUT) ? VKT_ERROR_DEVICE_TIMEOUT : VKT_ERROR_CUDA;
    }
    return VKT_NO_ERROR;
}

vktError vktGetLaunchCount(uint64_t* count)
{
    if (!count) return VKT_ERROR_INVALID_VALUE;
    *count = g_launches.load();
    return VKT_NO_ERROR;
}

// ------------------------------------------------------------------ volumes

static vktError create_volume(vktStructuredVolume* volume, void* devPtr, int owning, int32_t dx,
                              int32_t dy, int32_t dz, vktDataFormat format, float sx, float sy,
                              float sz, float lo, float hi)
{
    if (!volume) return VKT_ERROR_INVALID_VALUE;
    *volume = nullptr;
    vktError err = check_volume_args(dx, dy, dz, format, sx, sy, sz, lo, hi);
    if (err != VKT_NO_ERROR) return err;
    if (!owning && (!devPtr || reinterpret_cast<uintptr_t>(devPtr) % fmt_bytes(format) != 0))
        return VKT_ERROR_INVALID_VALUE;
    if (!owning && check_device() == VKT_NO_ERROR) {
        // a view must wrap device memory of the current device (or managed memory): host
        // memory, or an address no allocation covers, is refused here, before any kernel
        // could be launched on it
        cudaPointerAttributes attr;
        if (cudaPointerGetAttributes(&attr, devPtr) != cudaSuccess) {
            cudaGetLastError();
            return VKT_ERROR_INVALID_VALUE;
        }
        int dev = -1;
        if (cudaGetDevice(&dev) != cudaSuccess) {
            cudaGetLastError();
            return VKT_ERROR_NO_DEVICE;
        }
        const bool on_device = attr.type == cudaMemoryTypeDevice && attr.device == dev;
        if (!on_device && attr.type != cudaMemoryTypeManaged) return VKT_ERROR_INVALID_VALUE;
    }
    auto* v = new (std::nothrow) vktStructuredVolume_impl;
    if (!v) return VKT_ERROR_OUT_OF_MEMORY;
    v->magic = VKT_VOLUME_MAGIC;
    v->dims[0] = dx;
    v->dims[1] = dy;
    v->dims[2] = dz;
    v->format = format;
    v->cell[0] = sx;
    v->cell[1] = sy;
    v->cell[2] = sz;
    v->lo = lo;
    v->hi = hi;
    v->owning = owning;
    v->data = devPtr;
    if (owning) {
        err = check_device();
        if (err == VKT_NO_ERROR) {
            cudaError_t e = cudaMalloc(&v->data, volume_bytes(v));
            if (e == cudaSuccess) e = cudaMemset(v->data, 0, volume_bytes(v));
            err = from_cuda(e);
        }
        if (err != VKT_NO_ERROR) {
            if (v->data) cudaFree(v->data);
            v->magic = 0;
            delete v;
            return err;
        }
    }
    *volume = v;
    return VKT_NO_ERROR;
}

vktError vktStructuredVolumeCreate(vktStructuredVolume* volume, int32_t dx, int32_t dy,
                                   int32_t dz, vktDataFormat format, float sx, float sy,
                                   float sz, float lo, float hi)
{
    return create_volume(volume, nullptr, 1, dx, dy, dz, format, sx, sy, sz, lo, hi);
}

vktError vktStructuredVolumeCreateView(vktStructuredVolume* volume, void* devPtr, int32_t dx,
                                       int32_t dy, int32_t dz, vktDataFormat format, float sx,
                                       float sy, float sz, float lo, float hi)
{
    return create_volume(volume, devPtr, 0, dx, dy, dz, format, sx, sy, sz, lo, hi);
}

vktError vktStructuredVolumeDestroy(vktStructuredVolume volume)
{
    if (!valid(volume)) return VKT_ERROR_INVALID_HANDLE;
    vktError err = VKT_NO_ERROR;
    if (volume->owning && volume->data) err = from_cuda(cudaFree(volume->data));
    volume->magic = 0;
    delete volume;
    return err;
}

vktError vktStructuredVolumeGetDims(vktStructuredVolume v, int32_t* dx, int32_t* dy, int32_t* dz)
{
    if (!valid(v)) return VKT_ERROR_INVALID_HANDLE;
    if (!dx || !dy || !dz) return VKT_ERROR_INVALID_VALUE;
    *dx = v->dims[0];
    *dy = v->dims[1];
    *dz = v->dims[2];
    return VKT_NO_ERROR;
}

vktError vktStructuredVolumeGetDataFormat(vktStructuredVolume v, vktDataFormat* format)
{
    if (!valid(v)) return VKT_ERROR_INVALID_HANDLE;
    if (!format) return VKT_ERROR_INVALID_VALUE;
    *format = v->format;
    return VKT_NO_ERROR;
}

vktError vktStructuredVolumeGetCellSize(vktStructuredVolume v, float* sx, float* sy, float* sz)
{
    if (!valid(v)) return VKT_ERROR_INVALID_HANDLE;
    if (!sx || !sy || !sz) return VKT_ERROR_INVALID_VALUE;
    *sx = v->cell[0];
    *sy = v->cell[1];
    *sz = v->cell[2];
    return VKT_NO_ERROR;
}

vktError vktStructuredVolumeGetVoxelMapping(vktStructuredVolume v, float* lo, float* hi)
{
    if (!valid(v)) return VKT_ERROR_INVALID_HANDLE;
    if (!lo || !hi) return VKT_ERROR_INVALID_VALUE;
    *lo = v->lo;
    *hi = v->hi;
    return VKT_NO_ERROR;
}

vktError vktStructuredVolumeSetVoxelMapping(vktStructuredVolume v, float lo, float hi)
{
    if (!valid(v)) return VKT_ERROR_INVALID_HANDLE;
    if (!std::isfinite(lo) || !std::isfinite(hi)) return VKT_ERROR_INVALID_VALUE;
    if (v->format != vktDataFormatFloat32 && lo == hi) return VKT_ERROR_INVALID_VALUE;
    v->lo = lo;
    v->hi = hi;
    return VKT_NO_ERROR;
}

vktError vktStructuredVolumeGetData(vktStructuredVolume v, void** devPtr)
{
    if (!valid(v)) return VKT_ERROR_INVALID_HANDLE;
    if (!devPtr) return VKT_ERROR_INVALID_VALUE;
    *devPtr = v->data;
    return VKT_NO_ERROR;
}

vktError vktStructuredVolumeGetSizeInBytes(vktStructuredVolume v, uint64_t* bytes)
{
    if (!valid(v)) return VKT_ERROR_INVALID_HANDLE;
    if (!bytes) return VKT_ERROR_INVALID_VALUE;
    *bytes = volume_bytes(v);
    return VKT_NO_ERROR;
}

vktError vktStructuredVolumeSetData(vktStructuredVolume v, const void* hostPtr)
{
    if (!valid(v)) return VKT_ERROR_INVALID_HANDLE;
    if (!hostPtr) return VKT_ERROR_INVALID_VALUE;
    vktError err = check_device();
    if (err != VKT_NO_ERROR) return err;
    return from_cuda(cudaMemcpyAsync(v->data, hostPtr, volume_bytes(v), cudaMemcpyHostToDevice,
                                     static_cast<cudaStream_t>(t_policy.stream)));
}

vktError vktStructuredVolumeCopyToHost(vktStructuredVolume v, void* hostPtr)
{
    if (!valid(v)) return VKT_ERROR_INVALID_HANDLE;
    if (!hostPtr) return VKT_ERROR_INVALID_VALUE;
    vktError err = check_device();
    if (err != VKT_NO_ERROR) return err;
    return from_cuda(cudaMemcpyAsync(hostPtr, v->data, volume_bytes(v), cudaMemcpyDeviceToHost,
                                     static_cast<cudaStream_t>(t_policy.stream)));
}

// ------------------------------------------------------------------ filters

static vktFilter_impl* new_filter(int32_t k)
{
    auto* f = new (std::nothrow) vktFilter_impl;
    if (!f) return nullptr;
    memset(f, 0, sizeof(*f));
    f->magic = VKT_FILTER_MAGIC;
    f->k = k;
    return f;
}

vktError vktFilterCreate(vktFilter* filter, int32_t k, const float* hostWeights)
{
    if (!filter) return VKT_ERROR_INVALID_VALUE;
    *filter = nullptr;
    vktError err = check_filter_size(k);
    if (err != VKT_NO_ERROR) return err;
    vktFilter_impl* f = new_filter(k);
    if (!f) return VKT_ERROR_OUT_OF_MEMORY;
    if (hostWeights) memcpy(f->w, hostWeights, sizeof(float) * k * k * k);
    *filter = f;
    return VKT_NO_ERROR;
}

vktError vktFilterCreateSeparable(vktFilter* filter, int32_t k, const float* wx, const float* wy,
                                  const float* wz)
{
    if (!filter) return VKT_ERROR_INVALID_VALUE;
    *filter = nullptr;
    vktError err = check_filter_size(k);
    if (err != VKT_NO_ERROR) return err;
    if (!wx || !wy || !wz) return VKT_ERROR_INVALID_VALUE;
    vktFilter_impl* f = new_filter(k);
    if (!f) return VKT_ERROR_OUT_OF_MEMORY;
    f->separable = 1;
    memcpy(f->g[0], wx, sizeof(float) * k);
    memcpy(f->g[1], wy, sizeof(float) * k);
    memcpy(f->g[2], wz, sizeof(float) * k);
    dense_from_separable(f);
    *filter = f;
    return VKT_NO_ERROR;
}

vktError vktFilterCreateGaussian(vktFilter* filter, int32_t k, float sigma)
{
    if (!filter) return VKT_ERROR_INVALID_VALUE;
    *filter = nullptr;
    vktError err = check_filter_size(k);
    if (err != VKT_NO_ERROR) return err;
    if (!(sigma > 0.f) || !std::isfinite(sigma)) return VKT_ERROR_INVALID_VALUE;
    // sampled Gaussian at integer offsets, normalised by its FP64 sum
    const int r = (k - 1) / 2;
    double e[VKT_MAX_FILTER_SIZE], s = 0.0;
    const double sg = sigma;
    for (int i = 0; i < k; ++i) {
        const double d = static_cast<double>(i - r);
        e[i] = std::exp(-d * d / (2.0 * sg * sg));
        s += e[i];
    }
    float g[VKT_MAX_FILTER_SIZE];
    for (int i = 0; i < k; ++i) g[i] = static_cast<float>(e[i] / s);
    return vktFilterCreateSeparable(filter, k, g, g, g);
}

vktError vktFilterSetWeights(vktFilter f, const float* hostWeights)
{
    if (!valid(f)) return VKT_ERROR_INVALID_HANDLE;
    if (!hostWeights) return VKT_ERROR_INVALID_VALUE;
    memcpy(f->w, hostWeights, sizeof(float) * f->k * f->k * f->k);
    f->separable = 0;
    return VKT_NO_ERROR;
}

vktError vktFilterNormalize(vktFilter f)
{
    if (!valid(f)) return VKT_ERROR_INVALID_HANDLE;
    const int k = f->k;
    if (f->separable) {
        double sums[3];
        for (int a = 0; a < 3; ++a) {
            double s = 0.0;
            for (int i = 0; i < k; ++i) s += f->g[a][i];
            if (s == 0.0 || !std::isfinite(s)) return VKT_ERROR_INVALID_VALUE;
            sums[a] = s;
        }
        for (int a = 0; a < 3; ++a)
            for (int i = 0; i < k; ++i) f->g[a][i] = static_cast<float>(f->g[a][i] / sums[a]);
        dense_from_separable(f);
        return VKT_NO_ERROR;
    }
    double s = 0.0;
    for (int i = 0; i < k * k * k; ++i) s += f->w[i];
    if (s == 0.0 || !std::isfinite(s)) return VKT_ERROR_INVALID_VALUE;
    for (int i = 0; i < k * k * k; ++i) f->w[i] = static_cast<float>(f->w[i] / s);
    return VKT_NO_ERROR;
}

vktError vktFilterGetSize(vktFilter f, int32_t* k)
{
    if (!valid(f)) return VKT_ERROR_INVALID_HANDLE;
    if (!k) return VKT_ERROR_INVALID_VALUE;
    *k = f->k;
    return VKT_NO_ERROR;
}

vktError vktFilterIsSeparable(vktFilter f, int32_t* separable)
{
    if (!valid(f)) return VKT_ERROR_INVALID_HANDLE;
    if (!separable) return VKT_ERROR_INVALID_VALUE;
    *separable = f->separable;
    return VKT_NO_ERROR;
}

vktError vktFilterGetWeights(vktFilter f, float* hostWeights)
{
    if (!valid(f)) return VKT_ERROR_INVALID_HANDLE;
    if (!hostWeights) return VKT_ERROR_INVALID_VALUE;
    memcpy(hostWeights, f->w, sizeof(float) * f->k * f->k * f->k);
    return VKT_NO_ERROR;
}

vktError vktFilterGetSeparableWeights(vktFilter f, float* wx, float* wy, float* wz)
{
    if (!valid(f)) return VKT_ERROR_INVALID_HANDLE;
    if (!wx || !wy || !wz) return VKT_ERROR_INVALID_VALUE;
    if (!f->separable) return VKT_ERROR_UNSUPPORTED;
    memcpy(wx, f->g[0], sizeof(float) * f->k);
    memcpy(wy, f->g[1], sizeof(float) * f->k);
    memcpy(wz, f->g[2], sizeof(float) * f->k);
    return VKT_NO_ERROR;
}

vktError vktFilterDestroy(vktFilter f)
{
    if (!valid(f)) return VKT_ERROR_INVALID_HANDLE;
    f->magic = 0;
    delete f;
    return VKT_NO_ERROR;
}

// ------------------------------------------------------------------ ApplyFilter

// The autotuner's key of a single-volume call: filter size and kind, formats, the
// compensated mode, region or whole volume, and the extent filtered, each axis rounded up to
// a power of two (a size class), plus the SM count of the device.
static std::string tune_key(const vktStructuredVolume_impl* dst, const vktStructuredVolume_impl* src,
                            const vktFilter_impl* f, const int32_t* ext, bool roi, bool tensor_ok)
{
    auto cls = [](int v) {
        int c = 1;
        while (c < v) c <<= 1;
        return c;
    };
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    char buf[160];
    std::snprintf(buf, sizeof(buf), "filter k%d %s s%d d%d %s %dx%dx%d sm%d", f->k,
                  f->separable ? "separable" : (tensor_ok ? "dense-tc" : "dense"),
                  static_cast<int>(src->format),
                  static_cast<int>(dst->format), roi ? "range" : "volume", cls(ext[0]), cls(ext[1]),
                  cls(ext[2]), sms);
    return buf;
}

// ApplyFilter on the whole volume (box == nullptr) or on the region
// [box[0], box[3]) x [box[1], box[4]) x [box[2], box[5]) (validated by the caller).
//
// Path and launch shape: a forced policy path is used as given, with the launchers' rules.
// Under VKT_PATH_AUTO the fixed rule is separable for separable filters, tensor cores for
// dense k >= 5 float32 volumes that a tensor map describes (whole volumes), else direct;
// with the autotuner enabled, the first call of each call shape (tune_key) instead times
// the candidates -- the rule's path and, for dense filters the tensor path could also
// evaluate, the other one; for the CUDA-core paths three brick z extents (the rule's, and
// about 16 and 4 chunks per volume) -- on the policy stream and keeps the fastest.  A
// separable filter keeps its separable path (the batch computes the same bits).  No timing
// happens while the stream is being captured into a graph: the rule is used instead.
static vktError apply_filter(vktStructuredVolume dst, vktStructuredVolume src, vktFilter filter,
                             const int32_t* box)
{
    Ctx ctx;
    vktError err = get_context(&ctx);
    if (err != VKT_NO_ERROR) return err;

    const int k = filter->k;
    const bool auto_path = t_policy.path == VKT_PATH_AUTO;
    int path = t_policy.path;
    const bool tensor_ok = !box && k >= 5 && tensor_available(dst, src, filter) == VKT_NO_ERROR;
    if (auto_path) {
        if (filter->separable)
            path = VKT_PATH_SEPARABLE;
        else if (tensor_ok)
            path = VKT_PATH_TENSOR;
        else
            path = VKT_PATH_DIRECT;
    }
    if (path == VKT_PATH_SEPARABLE && !filter->separable) return VKT_ERROR_UNSUPPORTED;
    if (path == VKT_PATH_TENSOR) {
        if (box) return VKT_ERROR_UNSUPPORTED;   // the tensor-core path filters whole volumes
        err = tensor_available(dst, src, filter);
        if (err != VKT_NO_ERROR) return err;
    }

    Job base{};
    if (box) {
        base.roi = 1;
        base.rx0 = box[0];
        base.ry0 = box[1];
        base.rz0 = box[2];
        base.rx1 = box[3];
        base.ry1 = box[4];
        base.rz1 = box[5];
    }
    base.src = src->data;
    base.dst = dst->data;
    base.nx = src->dims[0];
    base.ny = src->dims[1];
    base.nz = src->dims[2];
    base.sfmt = src->format;
    base.dfmt = dst->format;
    // the job of one path: epilogue constants from that path's weight sum, compensated mode
    auto job_for = [&](int p, int zchunk) {
        Job job = base;
        double wsum = 0.0;
        if (p == VKT_PATH_SEPARABLE) {
            double sv[3] = {0.0, 0.0, 0.0};
            for (int a = 0; a < 3; ++a)
                for (int i = 0; i < k; ++i) sv[a] += filter->g[a][i];
            wsum = sv[0] * sv[1] * sv[2];
        } else {
            for (int i = 0; i < k * k * k; ++i) wsum += filter->w[i];
        }
        epilogue(dst, src, wsum, &job);
        if (p == VKT_PATH_SEPARABLE) job.comp = separable_needs_comp(dst, src, filter) ? 1 : 0;
        if (p == VKT_PATH_DIRECT) job.comp = direct_needs_comp(dst, src, filter) ? 1 : 0;
        job.zchunk = zchunk;
        return job;
    };
    auto launch = [&](int p, int zchunk) {
        const Job job = job_for(p, zchunk);
        if (p == VKT_PATH_SEPARABLE)
            return launch_separable(job, filter->g[0], filter->g[1], filter->g[2], k, ctx);
        if (p == VKT_PATH_TENSOR) return launch_tensor(job, filter->w, k, ctx);
        return launch_direct(job, filter->w, k, ctx);
    };

    int zchunk = 0;
    if (auto_path && autotune_enabled()) {
        const int32_t ext[3] = {box ? box[3] - box[0] : base.nx, box ? box[4] - box[1] : base.ny,
                                box ? box[5] - box[2] : base.nz};
        const std::string key = tune_key(dst, src, filter, ext, box != nullptr, tensor_ok);
        TuneChoice c;
        if (autotune_lookup(key.c_str(), &c)) {
            // a choice read from a file is used only where it can evaluate this call
            const bool usable = (c.path == VKT_PATH_SEPARABLE && filter->separable) ||
                                (c.path == VKT_PATH_TENSOR && tensor_ok) ||
                                c.path == VKT_PATH_DIRECT;
            if (usable) {
                path = c.path;
                zchunk = std::max(0, c.zchunk);
            }
        } else if (!stream_capturing(ctx.stream)) {
            // candidate 0 is the rule (its path, the launcher's z chunks); the tuner keeps
            // it unless another candidate is clearly faster
            TuneChoice cand[8];
            int n = 0;
            cand[n].path = path;
            cand[n++].zchunk = 0;
            const int ez = ext[2];
            const int zs[2] = {std::max(1, (ez + 15) / 16), std::max(1, (ez + 3) / 4)};
            const int cpath = filter->separable ? VKT_PATH_SEPARABLE : VKT_PATH_DIRECT;
            for (int i = 0; i < 2; ++i) {
                if (i > 0 && zs[i] == zs[i - 1]) continue;
                cand[n].path = cpath;
                cand[n++].zchunk = zs[i];
            }
            if (path == VKT_PATH_TENSOR) {   // the other path at its rule's z chunks
                cand[n].path = cpath;
                cand[n++].zchunk = 0;
            }
            err = autotune_time(cand, n, [&](const TuneChoice& t) { return launch(t.path, t.zchunk); },
                                ctx.stream, &c);
            if (err != VKT_NO_ERROR) return err;
            autotune_store(key.c_str(), c);
            if (ctx.debug & VKT_DEBUG_LOG)
                fprintf(stderr, "[vkt] autotune %s: %d candidates, path=%d zchunk=%d %.4f ms\n",
                        key.c_str(), n, c.path, c.zchunk, c.ms);
            path = c.path;
            zchunk = c.zchunk;
        }
    }

    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (t_policy.printTimes) {
        cudaEventCreate(&ev[0]);
        cudaEventCreate(&ev[1]);
        cudaEventRecord(ev[0], ctx.stream);
    }
    err = launch(path, zchunk);
    if (t_policy.printTimes) {
        cudaEventRecord(ev[1], ctx.stream);
        cudaEventSynchronize(ev[1]);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        fprintf(stderr, "[vkt] ApplyFilter%s %dx%dx%d k=%d path=%d: %.3f ms\n",
                box ? "Range" : "", base.nx, base.ny, base.nz, k, path, ms);
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
    }
    return err;
}

// A batch of n triples that share one dense (or direct-forced) filter, with equal dims,
// formats and value ranges: the direct path takes one launch over all n volumes when
// sources and destinations are evenly spaced (else one launch per volume), the tensor path
// one launch per volume; no graph is built, so a filter whose weights change from call to
// call (a training step) costs no recapture.  Sets *handled when the batch qualifies (and
// returns the launches' error); otherwise the caller builds its general batch.
}  // extern "C"

vktError vkt::apply_filter_multi(int32_t n, vktStructuredVolume* dst, vktStructuredVolume* src,
                                 vktFilter* filters, bool* handled)
{
    *handled = false;
    const vktFilter_impl* f = filters[0];
    for (int32_t i = 1; i < n; ++i) {
        if (filters[i] != f) return VKT_NO_ERROR;
        for (int a = 0; a < 3; ++a)
            if (src[i]->dims[a] != src[0]->dims[a]) return VKT_NO_ERROR;
        if (src[i]->format != src[0]->format || dst[i]->format != dst[0]->format ||
            src[i]->lo != src[0]->lo || src[i]->hi != src[0]->hi || dst[i]->lo != dst[0]->lo ||
            dst[i]->hi != dst[0]->hi)
            return VKT_NO_ERROR;
    }
    int path = t_policy.path;
    if (path == VKT_PATH_AUTO) {
        if (f->separable) return VKT_NO_ERROR;   // the persistent separable batch
        path = (f->k >= 5 && tensor_available(dst[0], src[0], f) == VKT_NO_ERROR) ? VKT_PATH_TENSOR
                                                                                  : VKT_PATH_DIRECT;
    }
    if (path == VKT_PATH_SEPARABLE) return VKT_NO_ERROR;
    if (path == VKT_PATH_TENSOR) {
        const vktError te = tensor_available(dst[0], src[0], f);
        if (te != VKT_NO_ERROR) {
            *handled = true;
            return te;
        }
    }
    int64_t ss = 0, sd = 0;
    const bool even = evenly_spaced(n, src, &ss) && evenly_spaced(n, dst, &sd);
    *handled = true;
    Ctx ctx;
    vktError err = get_context(&ctx);
    if (err != VKT_NO_ERROR) return err;
    Job job{};
    job.nx = src[0]->dims[0];
    job.ny = src[0]->dims[1];
    job.nz = src[0]->dims[2];
    job.sfmt = src[0]->format;
    job.dfmt = dst[0]->format;
    double wsum = 0.0;
    for (int i = 0; i < f->k * f->k * f->k; ++i) wsum += f->w[i];
    epilogue(dst[0], src[0], wsum, &job);
    if (path == VKT_PATH_DIRECT) {
        job.comp = direct_needs_comp(dst[0], src[0], f) ? 1 : 0;
        if (even) {
            job.src = src[0]->data;
            job.dst = dst[0]->data;
            job.nvol = n;
            job.vs_src = ss;
            job.vs_dst = sd;
            return launch_direct(job, f->w, f->k, ctx);
        }
    }
    for (int32_t i = 0; i < n && err == VKT_NO_ERROR; ++i) {
        job.src = src[i]->data;
        job.dst = dst[i]->data;
        err = path == VKT_PATH_TENSOR ? launch_tensor(job, f->w, f->k, ctx)
                                      : launch_direct(job, f->w, f->k, ctx);
    }
    return err;
}

extern "C" {

static vktError check_filter_args(vktStructuredVolume dst, vktStructuredVolume src,
                                  vktFilter filter)
{
    if (!valid(dst) || !valid(src) || !valid(filter)) return VKT_ERROR_INVALID_HANDLE;
    if (dst->dims[0] != src->dims[0] || dst->dims[1] != src->dims[1] ||
        dst->dims[2] != src->dims[2])
        return VKT_ERROR_DIMS_MISMATCH;
    if (overlaps(dst, src)) return VKT_ERROR_INVALID_VALUE;
    return VKT_NO_ERROR;
}

vktError vktApplyFilterSV(vktStructuredVolume dst, vktStructuredVolume src, vktFilter filter)
{
    vkt::CallRange nvtx_range("vktApplyFilterSV");
    const vktError err = check_filter_args(dst, src, filter);
    if (err != VKT_NO_ERROR) return err;
    return apply_filter(dst, src, filter, nullptr);
}

vktError vktApplyFilterRangeSV(vktStructuredVolume dst, vktStructuredVolume src,
                               vktFilter filter, int32_t firstX, int32_t firstY, int32_t firstZ,
                               int32_t lastX, int32_t lastY, int32_t lastZ)
{
    vkt::CallRange nvtx_range("vktApplyFilterRangeSV");
    const vktError err = check_filter_args(dst, src, filter);
    if (err != VKT_NO_ERROR) return err;
    const int32_t box[6] = {firstX, firstY, firstZ, lastX, lastY, lastZ};
    for (int a = 0; a < 3; ++a)
        if (box[a] < 0 || box[a] > box[a + 3] || box[a + 3] > src->dims[a])
            return VKT_ERROR_INVALID_VALUE;
    if (box[0] == box[3] || box[1] == box[4] || box[2] == box[5]) {
        // an empty region writes nothing; the device is still required, as for any call
        Ctx ctx;
        return get_context(&ctx);
    }
    return apply_filter(dst, src, filter, box);
}

vktError vktApplyFilterBackwardSV(vktStructuredVolume gradSrc, float* gradWeights,
                                  vktStructuredVolume gradDst, vktStructuredVolume src,
                                  vktFilter filter)
{
    vkt::CallRange nvtx_range("vktApplyFilterBackwardSV");
    if (!valid(gradDst) || !valid(src) || !valid(filter)) return VKT_ERROR_INVALID_HANDLE;
    if (gradSrc && !valid(gradSrc)) return VKT_ERROR_INVALID_HANDLE;
    if (src->format != vktDataFormatFloat32 || gradDst->format != vktDataFormatFloat32 ||
        (gradSrc && gradSrc->format != vktDataFormatFloat32))
        return VKT_ERROR_UNSUPPORTED;
    for (int a = 0; a < 3; ++a) {
        if (gradDst->dims[a] != src->dims[a]) return VKT_ERROR_DIMS_MISMATCH;
        if (gradSrc && gradSrc->dims[a] != src->dims[a]) return VKT_ERROR_DIMS_MISMATCH;
    }
    if (gradSrc && (overlaps(gradSrc, gradDst) || overlaps(gradSrc, src)))
        return VKT_ERROR_INVALID_VALUE;
    if (reinterpret_cast<uintptr_t>(gradWeights) % 4 != 0) return VKT_ERROR_INVALID_VALUE;
    Ctx ctx;
    vktError err = get_context(&ctx);
    if (err != VKT_NO_ERROR) return err;
    const int k = filter->k;
    const int nx = src->dims[0], ny = src->dims[1], nz = src->dims[2];
    if (gradSrc) {
        // the adjoint writes every voxel, then adds the shell outside the volume to the faces
        Job job{};
        job.src = gradDst->data;
        job.dst = gradSrc->data;
        job.nx = nx;
        job.ny = ny;
        job.nz = nz;
        job.sfmt = vktDataFormatFloat32;
        job.dfmt = vktDataFormatFloat32;
        job.a0 = 0.f;
        job.a1 = 1.f;
        job.qmax = 0.f;
        err = launch_adjoint(job, filter->w, k, ctx);
        if (err != VKT_NO_ERROR) return err;
    }
    if (gradWeights) {
        // per-CTA partial sums live in stream-ordered scratch for the duration of the call
        const size_t cap = weight_grad_scratch_floats(nx, ny, nz, k);
        float* partials = nullptr;
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&partials), cap * sizeof(float),
                                        ctx.stream);
        if (e != cudaSuccess) return from_cuda(e);
        err = launch_weight_grad(static_cast<const float*>(src->data),
                                 static_cast<const float*>(gradDst->data), nx, ny, nz, k, partials,
                                 cap, gradWeights, ctx);
        e = cudaFreeAsync(partials, ctx.stream);
        if (err == VKT_NO_ERROR && e != cudaSuccess) err = from_cuda(e);
    }
    return err;
}

// The volumes a batch call writes must not overlap one another, nor any volume it reads.
static bool writes_disjoint(int32_t n, const vktStructuredVolume* w, const vktStructuredVolume* r1,
                            const vktStructuredVolume* r2)
{
    struct Span {
        uintptr_t lo, hi;
    };
    std::vector<Span> d;
    d.reserve(n);
    for (int32_t i = 0; i < n; ++i) {
        const uintptr_t lo = reinterpret_cast<uintptr_t>(w[i]->data);
        d.push_back({lo, lo + volume_bytes(w[i])});
    }
    std::sort(d.begin(), d.end(), [](const Span& a, const Span& b) { return a.lo < b.lo; });
    for (size_t i = 1; i < d.size(); ++i)
        if (d[i].lo < d[i - 1].hi) return false;
    for (const vktStructuredVolume* r : {r1, r2}) {
        for (int32_t j = 0; j < n; ++j) {
            const uintptr_t lo = reinterpret_cast<uintptr_t>(r[j]->data);
            const uintptr_t hi = lo + volume_bytes(r[j]);
            auto it = std::lower_bound(d.begin(), d.end(), hi,
                                       [](const Span& s, uintptr_t v) { return s.lo < v; });
            if (it != d.begin() && (it - 1)->hi > lo) return false;
        }
    }
    return true;
}

vktError vktApplyFilterBackwardBatchSV(int32_t n, vktStructuredVolume* gradSrcs, float* gradWeights,
                                       vktStructuredVolume* gradDsts, vktStructuredVolume* srcs,
                                       vktFilter filter)
{
    vkt::CallRange nvtx_range("vktApplyFilterBackwardBatchSV");
    if (n < 1 || !gradDsts || !srcs) return VKT_ERROR_INVALID_VALUE;
    if (!valid(filter)) return VKT_ERROR_INVALID_HANDLE;
    for (int32_t b = 0; b < n; ++b) {
        if (!valid(gradDsts[b]) || !valid(srcs[b])) return VKT_ERROR_INVALID_HANDLE;
        if (gradSrcs && !valid(gradSrcs[b])) return VKT_ERROR_INVALID_HANDLE;
        if (srcs[b]->format != vktDataFormatFloat32 || gradDsts[b]->format != vktDataFormatFloat32 ||
            (gradSrcs && gradSrcs[b]->format != vktDataFormatFloat32))
            return VKT_ERROR_UNSUPPORTED;
        for (int a = 0; a < 3; ++a) {
            if (srcs[b]->dims[a] != srcs[0]->dims[a] || gradDsts[b]->dims[a] != srcs[0]->dims[a])
                return VKT_ERROR_DIMS_MISMATCH;
            if (gradSrcs && gradSrcs[b]->dims[a] != srcs[0]->dims[a]) return VKT_ERROR_DIMS_MISMATCH;
        }
    }
    if (gradSrcs && !writes_disjoint(n, gradSrcs, gradDsts, srcs)) return VKT_ERROR_INVALID_VALUE;
    if (reinterpret_cast<uintptr_t>(gradWeights) % 4 != 0) return VKT_ERROR_INVALID_VALUE;
    Ctx ctx;
    vktError err = get_context(&ctx);
    if (err != VKT_NO_ERROR) return err;
    const int k = filter->k;
    const int nx = srcs[0]->dims[0], ny = srcs[0]->dims[1], nz = srcs[0]->dims[2];
    int64_t s_x = 0, s_gy = 0, s_gx = 0;
    const bool even_x = evenly_spaced(n, srcs, &s_x);
    const bool even_gy = evenly_spaced(n, gradDsts, &s_gy);
    const bool even_gx = gradSrcs && evenly_spaced(n, gradSrcs, &s_gx);
    if (gradSrcs) {
        // the adjoint writes every voxel, then adds the shell outside the volume to the faces
        Job job{};
        job.nx = nx;
        job.ny = ny;
        job.nz = nz;
        job.sfmt = vktDataFormatFloat32;
        job.dfmt = vktDataFormatFloat32;
        job.a0 = 0.f;
        job.a1 = 1.f;
        job.qmax = 0.f;
        if (even_gy && even_gx) {
            // the whole batch in one launch
            job.src = gradDsts[0]->data;
            job.dst = gradSrcs[0]->data;
            job.nvol = n;
            job.vs_src = s_gy;
            job.vs_dst = s_gx;
            err = launch_adjoint(job, filter->w, k, ctx);
        } else {
            for (int32_t b = 0; b < n && err == VKT_NO_ERROR; ++b) {
                job.src = gradDsts[b]->data;
                job.dst = gradSrcs[b]->data;
                err = launch_adjoint(job, filter->w, k, ctx);
            }
        }
        if (err != VKT_NO_ERROR) return err;
    }
    if (gradWeights) {
        // every volume's per-CTA partial sums in one stream-ordered scratch, reduced together
        const bool one = even_x && even_gy;
        const size_t per = weight_grad_scratch_floats(nx, ny, nz, k, 1);
        const size_t cap = one ? weight_grad_scratch_floats(nx, ny, nz, k, n) : per * n;
        float* partials = nullptr;
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&partials), cap * sizeof(float),
                                        ctx.stream);
        if (e != cudaSuccess) return from_cuda(e);
        if (one) {
            err = launch_weight_grad(static_cast<const float*>(srcs[0]->data),
                                     static_cast<const float*>(gradDsts[0]->data), nx, ny, nz, k,
                                     partials, cap, gradWeights, ctx, n, s_x, s_gy);
        } else {
            for (int32_t b = 0; b < n && err == VKT_NO_ERROR; ++b)
                err = launch_weight_grad_partials(static_cast<const float*>(srcs[b]->data),
                                                  static_cast<const float*>(gradDsts[b]->data), nx,
                                                  ny, nz, k, partials + per * b, ctx);
            if (err == VKT_NO_ERROR)
                err = reduce_weight_grad(partials, per * n / (static_cast<size_t>(k) * k * k), k,
                                         gradWeights, ctx);
        }
        e = cudaFreeAsync(partials, ctx.stream);
        if (err == VKT_NO_ERROR && e != cudaSuccess) err = from_cuda(e);
    }
    return err;
}

}  // extern "C"
