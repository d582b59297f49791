// vkt_backward.cu -- gradients of the float32 clamped correlation y = C_w x:
//   dL/dx : exact adjoint, evaluated by the direct kernel in adjoint mode (vkt_direct.cuh);
//   dL/dw[c][b][a] = sum_i gy(i) x(clamp(i + (a-r, b-r, c-r))), evaluated here.
//
// Weight gradient: CTA (c, x tile, y tile, z chunk) owns one kernel plane offset c and a
// 64 x 32 x zchunk brick of output positions i.  It streams the x planes z + c - r (TMA into
// a ring of raw float32 stages that the FMAs read directly, clamp-to-edge applied by row
// index and, at the x faces, by patching the columns outside the volume in place) and the
// gy planes z, and accumulates the k^2 sums over (b, a) in registers: k^2 FMAs per voxel
// per CTA, k^3 over the k CTAs that share a tile.  The CTA reduces its sums (warp
// shuffles, then shared memory) to one FP32 partial per tap; a second kernel adds the
// partials of all CTAs in FP64 and writes float32 dL/dw.
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "vkt_internal.h"
#include "vkt_tile.cuh"

namespace vkt {
namespace {

constexpr int NT = 256;
constexpr int BX = 16, BY = 16, RX = 4, RY = 2;
constexpr int TX = BX * RX, TY = BY * RY;
constexpr int STAGES = 4;

struct WgArgs {
    const float* x;
    const float* gy;
    float* partials;     // [nspatial][k^3], nspatial = volumes x chunks x tiles_y x tiles_x
    int nx, ny, nz;
    int tiles_x, tiles_y, zchunk, chunks;
    int64_t vs_x, vs_gy; // voxels from one volume of the batch to the next
    int use_tma;
    unsigned* status;
};

template <int K>
constexpr size_t wgrad_smem_bytes()
{
    using Geo = Brick<K, TX, TY>;
    return 128 + static_cast<size_t>(STAGES) * Geo::raw_bytes(FMT_F32) +
           static_cast<size_t>(NT / 32) * K * K * sizeof(float);
}

// The FMAs read the raw float32 stage as delivered (no float tile): a window row is read as
// NQ aligned float4s from the thread's column 4 tx on, and window element a of output x is
// raw column 4 tx + x + a + XA - r.  Rows are clamped through the row each window row reads;
// columns outside the volume (zero-filled by the tensor map) are overwritten with the face
// column in the tiles at the x faces.  A stage is refilled only after the CTA barrier that
// follows the FMAs reading it, so STAGES - 1 planes are in flight.
template <int K>
__global__ void __launch_bounds__(NT)
    k_wgrad(const __grid_constant__ CUtensorMap tmap, const WgArgs p)
{
    using Geo = Brick<K, TX, TY>;
    constexpr int R = Geo::R, FH = Geo::FH;
    constexpr int XA = 4;                                  // float32 x halo of the raw tile
    constexpr int RW = Geo::raw_w(FMT_F32);                // TX + 2 XA floats per raw row
    constexpr int NW = RX + K - 1;                         // window row length
    constexpr int NQ = (NW + XA - R + 3) / 4;              // float4 loads per window row
    static_assert(RX * (BX - 1) + 4 * NQ <= RW, "window loads stay inside the raw row");
    __builtin_assume(threadIdx.x < NT);   // every launch has NT threads
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    constexpr int rawb = Geo::raw_bytes(FMT_F32);
    constexpr uint32_t txb = Geo::raw_tx(FMT_F32);
    unsigned char* raw = smem + 128;
    float* red = reinterpret_cast<float*>(raw + STAGES * rawb);

    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const int tx = tid % BX, ty = tid / BX;
    const int c = blockIdx.x % K;
    const int xt = blockIdx.x / K;
    const int x0 = xt * TX, y0 = blockIdx.y * TY;
    // blockIdx.z = volume * chunks + z chunk
    const int vol = static_cast<int>(blockIdx.z) / p.chunks;
    const int zc0 = (static_cast<int>(blockIdx.z) - vol * p.chunks) * p.zchunk;
    const float* xv = p.x + vol * p.vs_x;
    const float* gyv = p.gy + vol * p.vs_gy;
    const int zc1 = min(zc0 + p.zchunk, p.nz);
    const int nplanes = max(zc1 - zc0, 0);

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
        if (p.use_tma) prefetch_tensor_map(&tmap);
    }
    __syncthreads();
    grid_dependency_wait();   // programmatic launch: the previous kernel's writes are visible
    launch_dependents();
    int issued = 0;
    // x plane paired with gy plane z is clamp(z + c - r)
    auto issue = [&](int q) {
        const int s = q % STAGES;
        mbar_arrive_expect_tx(&bars[s], txb);
        tma_load_4d(raw + s * rawb, &tmap, &bars[s], x0 - XA, y0 - R,
                    clampi(zc0 + q + c - R, 0, p.nz - 1), vol);
        ++issued;
    };
    if (p.use_tma && tid == 0)
        for (int q = 0; q < STAGES - 1 && q < nplanes; ++q) issue(q);

    // raw offset of each window row of this thread (rows clamped to the volume)
    int rowoff[RY + K - 1];
#pragma unroll
    for (int j = 0; j < RY + K - 1; ++j)
        rowoff[j] = (clampi(y0 - R + ty * RY + j, 0, p.ny - 1) - (y0 - R)) * RW + tx * RX;
    // tensor-map stages at the x faces: raw columns [0, lfix) lie left of x = 0 and take
    // column XA (x = 0); columns [rfix, RW) lie right of nx - 1 and take column rfix - 1;
    // only the raw rows inside the volume, [ry0, ry1), are ever read
    const int lfix = max(0, XA - x0);
    const int rfix = min(RW, p.nx - x0 + XA);
    const int ry0 = max(0, R - y0), ry1 = min(FH, p.ny - y0 + R);
    const bool edge = p.use_tma && (lfix > 0 || rfix < RW);
    auto fix_faces = [&](float* rf) {
        const int nr = RW - rfix, per = lfix + nr;
        for (int e = tid; e < (ry1 - ry0) * per; e += NT) {
            const int r = ry0 + e / per, k = e % per;
            float* row = rf + r * RW;
            if (k < lfix)
                row[k] = row[XA];
            else
                row[rfix + k - lfix] = row[rfix - 1];
        }
        fence_proxy_async();   // a later tensor-map load refills these bytes
    };

    float acc[K][K];
#pragma unroll
    for (int b = 0; b < K; ++b)
#pragma unroll
        for (int a = 0; a < K; ++a) acc[b][a] = 0.f;

    const int ox = x0 + tx * RX;
    // gy block of this thread in plane z (zero outside the volume so it adds nothing)
    auto load_g = [&](int z, float (&g)[RY][RX]) {
#pragma unroll
        for (int i = 0; i < RY; ++i) {
            const int oy = y0 + ty * RY + i;
            const int64_t row = (static_cast<int64_t>(z) * p.ny + oy) * p.nx;
#pragma unroll
            for (int x = 0; x < RX; ++x)
                g[i][x] = (oy < p.ny && ox + x < p.nx) ? __ldg(gyv + row + ox + x) : 0.f;
        }
    };
    // the block of the next plane is loaded before the FMAs of this one (its latency hides
    // behind them)
    float g[RY][RX];
    if (nplanes > 0) load_g(zc0, g);
    bool failed = false;
    for (int it = 0; it < nplanes; ++it) {
        const int s = it % STAGES;
        const int z = zc0 + it;
        unsigned char* rs = raw + s * rawb;
        bool ok = true;
        if (p.use_tma) {
            ok = mbar_wait(&bars[s], (it / STAGES) & 1);
            if (ok && edge) fix_faces(reinterpret_cast<float*>(rs));
        } else {
            fill_raw_plain<Geo, NT>(rs, xv, FMT_F32, p.nx, p.ny, p.nz, x0, y0, z + c - R, tid);
        }
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        // every thread is past the FMAs of plane it - 1: its stage takes plane it + STAGES - 1
        if (p.use_tma && tid == 0 && it + STAGES - 1 < nplanes) issue(it + STAGES - 1);
        float gn[RY][RX];
        if (it + 1 < nplanes) load_g(z + 1, gn);
        const float* rf = reinterpret_cast<const float*>(rs);
#pragma unroll
        for (int j = 0; j < RY + K - 1; ++j) {
            float q[4 * NQ];
#pragma unroll
            for (int n = 0; n < NQ; ++n) {
                const float4 t = *reinterpret_cast<const float4*>(rf + rowoff[j] + 4 * n);
                q[4 * n] = t.x;
                q[4 * n + 1] = t.y;
                q[4 * n + 2] = t.z;
                q[4 * n + 3] = t.w;
            }
#pragma unroll
            for (int i = 0; i < RY; ++i) {
                const int b = j - i;
                if (b < 0 || b >= K) continue;
#pragma unroll
                for (int a = 0; a < K; ++a)
#pragma unroll
                    for (int x = 0; x < RX; ++x)
                        acc[b][a] = fmaf(g[i][x], q[x + a + XA - R], acc[b][a]);
            }
        }
        if (it + 1 < nplanes) {
#pragma unroll
            for (int i = 0; i < RY; ++i)
#pragma unroll
                for (int x = 0; x < RX; ++x) g[i][x] = gn[i][x];
        }
    }
    if (failed) {
        if (tid == 0) {
            atomicOr(p.status, STATUS_TIMEOUT);
            for (int q = issued - 1; q >= 0 && q >= issued - STAGES; --q)
                mbar_wait(&bars[q % STAGES], (q / STAGES) & 1);
        }
        __syncthreads();
        return;
    }
    // CTA reduction of the K*K sums: warps, then shared memory
#pragma unroll
    for (int b = 0; b < K; ++b)
#pragma unroll
        for (int a = 0; a < K; ++a) {
            float v = acc[b][a];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp * K * K + b * K + a] = v;
        }
    __syncthreads();
    const int spatial = (blockIdx.z * p.tiles_y + blockIdx.y) * p.tiles_x + xt;
    for (int t = tid; t < K * K; t += NT) {
        float v = 0.f;
        for (int w = 0; w < NT / 32; ++w) v += red[w * K * K + t];
        p.partials[static_cast<int64_t>(spatial) * K * K * K + c * K * K + t] = v;
    }
}

// dL/dw[d] = sum over CTAs of partials[cta][d], in FP64; one warp per tap.  `failed`
// (may be null): a status word that the partial-sum kernel of this call set when a bounded
// wait of one of its CTAs timed out; that CTA wrote no partials, so the sums would mix in
// stale scratch, and gw is filled with NaN instead.
__global__ void k_wgrad_reduce(const float* partials, int nspatial, int kkk, float* gw,
                               const unsigned* failed)
{
    grid_dependency_wait();   // programmatic launch: the partial sums are written
    const int d = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    if (d >= kkk) return;
    if (failed && (*failed & STATUS_TIMEOUT)) {
        if (lane == 0) gw[d] = __int_as_float(0x7fc00000);
        return;
    }
    double s = 0.0;
    for (int i = lane; i < nspatial; i += 32) s += static_cast<double>(partials[static_cast<int64_t>(i) * kkk + d]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) gw[d] = static_cast<float>(s);
}

struct Geometry {
    int tiles_x, tiles_y, chunks, zchunk;
};

// CTAs: k kernel planes x tiles_x x tiles_y x chunks per volume, the z chunks chosen by
// zchunk_for over all volumes' tiles (at least 8 planes per chunk unless the job is too
// small for one CTA per SM).
Geometry geometry(int nx, int ny, int nz, int k, int nvol = 1)
{
    Geometry g;
    g.tiles_x = (nx + TX - 1) / TX;
    g.tiles_y = (ny + TY - 1) / TY;
    int sms = 152, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long xyc = static_cast<long>(g.tiles_x) * g.tiles_y * k * std::max(nvol, 1);
    g.zchunk = zchunk_for(xyc, nz, sms);
    g.chunks = (nz + g.zchunk - 1) / g.zchunk;
    return g;
}

// The partial-sum kernel over nvol volumes (vs_x, vs_gy voxels apart) into `partials`.
template <int K>
vktError launch_wg_partials(const float* x, const float* gy, int nx, int ny, int nz, int nvol,
                            int64_t vs_x, int64_t vs_gy, const Geometry& g, float* partials,
                            unsigned* status, cudaStream_t stream, int debug)
{
    using Geo = Brick<K, TX, TY>;
    if (static_cast<long>(g.chunks) * nvol > 65535) return VKT_ERROR_UNSUPPORTED;
    WgArgs a;
    a.x = x;
    a.gy = gy;
    a.partials = partials;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.tiles_x = g.tiles_x;
    a.tiles_y = g.tiles_y;
    a.zchunk = g.zchunk;
    a.chunks = g.chunks;
    a.vs_x = vs_x;
    a.vs_gy = vs_gy;
    a.status = status;
    alignas(64) CUtensorMap map;
    a.use_tma = encode_tensor_map(&map, FMT_F32, x, nx, ny, nz, nvol, vs_x, Geo::raw_w(FMT_F32),
                                  Geo::FH, 1)
                    ? 1
                    : 0;
    if (!a.use_tma) memset(&map, 0, sizeof(map));
    const size_t smem = wgrad_smem_bytes<K>();
    cudaError_t e = cudaFuncSetAttribute(k_wgrad<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return from_cuda(e);
    if (debug & VKT_DEBUG_LOG)
        fprintf(stderr, "[vkt] wgrad k=%d grid=(%d,%d,%d) zchunk=%d volumes=%d tma=%d\n", K,
                g.tiles_x * K, g.tiles_y, g.chunks * nvol, g.zchunk, nvol, a.use_tma);
    e = launch_pdl(k_wgrad<K>, dim3(g.tiles_x * K, g.tiles_y, g.chunks * nvol), dim3(NT), smem,
                   stream, map, a);
    count_launches(1);
    if (e != cudaSuccess) return from_cuda(e);
    return from_cuda(cudaGetLastError());
}

void launch_reduce(const float* partials, size_t nspatial, int k, float* gw, const unsigned* failed,
                   cudaStream_t stream)
{
    const int kkk = k * k * k;
    launch_pdl(k_wgrad_reduce, dim3((kkk + 7) / 8), dim3(256), 0, stream, partials,
               static_cast<int>(nspatial), kkk, gw, failed);
    count_launches(1);
}

template <int K>
vktError launch_wg(const float* x, const float* gy, int nx, int ny, int nz, float* partials,
                   size_t cap, float* gw, const Ctx& ctx, int nvol, int64_t vs_x, int64_t vs_gy)
{
    const Geometry g = geometry(nx, ny, nz, K, nvol);
    const size_t nspatial = static_cast<size_t>(g.tiles_x) * g.tiles_y * g.chunks * nvol;
    if (nspatial * K * K * K > cap) return VKT_ERROR_INVALID_VALUE;
    vktError err = launch_wg_partials<K>(x, gy, nx, ny, nz, nvol, vs_x, vs_gy, g, partials,
                                         ctx.status, ctx.stream, ctx.debug);
    if (err != VKT_NO_ERROR) return err;
    launch_reduce(partials, nspatial, K, gw, nullptr, ctx.stream);
    return from_cuda(cudaGetLastError());
}

}  // namespace

size_t weight_grad_scratch_floats(int nx, int ny, int nz, int k, int nvol)
{
    const Geometry g = geometry(nx, ny, nz, k, nvol);
    return static_cast<size_t>(g.tiles_x) * g.tiles_y * g.chunks * std::max(nvol, 1) * k * k * k;
}

vktError launch_weight_grad(const float* x, const float* gy, int nx, int ny, int nz, int k,
                            float* partials, size_t cap, float* gw, const Ctx& ctx, int nvol,
                            int64_t vs_x, int64_t vs_gy)
{
    nvol = std::max(nvol, 1);
    switch (k) {
    case 1: return launch_wg<1>(x, gy, nx, ny, nz, partials, cap, gw, ctx, nvol, vs_x, vs_gy);
    case 3: return launch_wg<3>(x, gy, nx, ny, nz, partials, cap, gw, ctx, nvol, vs_x, vs_gy);
    case 5: return launch_wg<5>(x, gy, nx, ny, nz, partials, cap, gw, ctx, nvol, vs_x, vs_gy);
    case 7: return launch_wg<7>(x, gy, nx, ny, nz, partials, cap, gw, ctx, nvol, vs_x, vs_gy);
    case 9: return launch_wg<9>(x, gy, nx, ny, nz, partials, cap, gw, ctx, nvol, vs_x, vs_gy);
    default: return VKT_ERROR_UNSUPPORTED;
    }
}

vktError launch_weight_grad_partials(const float* x, const float* gy, int nx, int ny, int nz,
                                     int k, float* partials, const Ctx& ctx)
{
    const Geometry g = geometry(nx, ny, nz, k, 1);
    switch (k) {
    case 1: return launch_wg_partials<1>(x, gy, nx, ny, nz, 1, 0, 0, g, partials, ctx.status, ctx.stream, ctx.debug);
    case 3: return launch_wg_partials<3>(x, gy, nx, ny, nz, 1, 0, 0, g, partials, ctx.status, ctx.stream, ctx.debug);
    case 5: return launch_wg_partials<5>(x, gy, nx, ny, nz, 1, 0, 0, g, partials, ctx.status, ctx.stream, ctx.debug);
    case 7: return launch_wg_partials<7>(x, gy, nx, ny, nz, 1, 0, 0, g, partials, ctx.status, ctx.stream, ctx.debug);
    case 9: return launch_wg_partials<9>(x, gy, nx, ny, nz, 1, 0, 0, g, partials, ctx.status, ctx.stream, ctx.debug);
    default: return VKT_ERROR_UNSUPPORTED;
    }
}

vktError reduce_weight_grad(const float* partials, size_t nspatial, int k, float* gw, const Ctx& ctx)
{
    launch_reduce(partials, nspatial, k, gw, nullptr, ctx.stream);
    return from_cuda(cudaGetLastError());
}

}  // namespace vkt

// ------------------------------------------------------------------ allocation-free variant
//
// For callers that cannot let the library allocate device memory (see vkt.h): the per-CTA
// partial sums of the weight gradient live in this fixed array instead of stream-ordered
// scratch, and the kernels' status word lives next to it.  Host code must not pass these
// names to a kernel (on the host they name a stand-in, not a device address): their device
// addresses are looked up once per device with cudaGetSymbolAddress.

#include <mutex>

static __device__ __align__(256) float g_noalloc_partials[VKT_NOALLOC_SCRATCH_FLOATS];
static __device__ __align__(256) unsigned g_noalloc_status[4];

namespace {

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
float* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
unsigned* g_noalloc_status_ptr[NOALLOC_MAX_DEVICES] = {};

// device addresses of the scratch array and status word on the current device
vktError noalloc_scratch(float** partials, unsigned** status)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return vkt::from_cuda(e);
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return VKT_ERROR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        void* q = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return vkt::from_cuda(e);
        e = cudaGetSymbolAddress(&q, g_noalloc_status);
        if (e != cudaSuccess) return vkt::from_cuda(e);
        g_noalloc_ptr[dev] = static_cast<float*>(p);
        g_noalloc_status_ptr[dev] = static_cast<unsigned*>(q);
    }
    *partials = g_noalloc_ptr[dev];
    *status = g_noalloc_status_ptr[dev];
    return VKT_NO_ERROR;
}

// the weight-gradient kernels over the fixed scratch
template <int K>
vktError launch_wg_noalloc(const float* x, const float* gy, int nx, int ny, int nz,
                           float* partials, unsigned* status, float* gw, cudaStream_t stream,
                           int debug)
{
    using namespace vkt;
    // geometry() adds z chunks only while the grid is under about 8 CTAs per SM (two per
    // SM for small volumes), so a volume with more than one chunk needs fewer than
    // 16 x SMs x k^2 partial sums; only single-chunk volumes of many column tiles can
    // exceed the scratch
    const Geometry g = geometry(nx, ny, nz, K);
    const size_t nspatial = static_cast<size_t>(g.tiles_x) * g.tiles_y * g.chunks;
    if (nspatial * K * K * K > VKT_NOALLOC_SCRATCH_FLOATS) return VKT_ERROR_INVALID_VALUE;
    // the call's own status word starts at zero in stream order (a memset allocates nothing)
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(unsigned), stream);
    if (e != cudaSuccess) return from_cuda(e);
    vktError err = launch_wg_partials<K>(x, gy, nx, ny, nz, 1, 0, 0, g, partials, status, stream,
                                         debug);
    if (err != VKT_NO_ERROR) return err;
    launch_reduce(partials, nspatial, K, gw, status, stream);
    return from_cuda(cudaGetLastError());
}

}  // namespace

extern "C" vktError vktApplyFilterWeightGradNoAllocSV(float* gradWeights, vktStructuredVolume gradDst,
                                                      vktStructuredVolume src, vktFilter filter)
{
    vkt::CallRange nvtx_range("vktApplyFilterWeightGradNoAllocSV");
    if (!gradDst || gradDst->magic != VKT_VOLUME_MAGIC || !src || src->magic != VKT_VOLUME_MAGIC ||
        !filter || filter->magic != VKT_FILTER_MAGIC)
        return VKT_ERROR_INVALID_HANDLE;
    if (!gradWeights || reinterpret_cast<uintptr_t>(gradWeights) % 4 != 0) return VKT_ERROR_INVALID_VALUE;
    if (src->format != vktDataFormatFloat32 || gradDst->format != vktDataFormatFloat32)
        return VKT_ERROR_UNSUPPORTED;
    for (int a = 0; a < 3; ++a)
        if (gradDst->dims[a] != src->dims[a]) return VKT_ERROR_DIMS_MISMATCH;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return VKT_ERROR_NO_DEVICE;
    }
    float* partials = nullptr;
    unsigned* status = nullptr;
    vktError err = noalloc_scratch(&partials, &status);
    if (err != VKT_NO_ERROR) return err;
    vktExecutionPolicy pol;
    vktGetThreadExecutionPolicy(&pol);
    cudaStream_t stream = static_cast<cudaStream_t>(pol.stream);
    const float* x = static_cast<const float*>(src->data);
    const float* gy = static_cast<const float*>(gradDst->data);
    const int nx = src->dims[0], ny = src->dims[1], nz = src->dims[2];
    const int dbg = pol.debug;
    switch (filter->k) {
    case 1: return launch_wg_noalloc<1>(x, gy, nx, ny, nz, partials, status, gradWeights, stream, dbg);
    case 3: return launch_wg_noalloc<3>(x, gy, nx, ny, nz, partials, status, gradWeights, stream, dbg);
    case 5: return launch_wg_noalloc<5>(x, gy, nx, ny, nz, partials, status, gradWeights, stream, dbg);
    case 7: return launch_wg_noalloc<7>(x, gy, nx, ny, nz, partials, status, gradWeights, stream, dbg);
    case 9: return launch_wg_noalloc<9>(x, gy, nx, ny, nz, partials, status, gradWeights, stream, dbg);
    default: return VKT_ERROR_UNSUPPORTED;
    }
}

