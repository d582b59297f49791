// vkt_clahe.cu -- CLAHE-3D (Sec. 4.1, "Case Study: CLAHE-3D": contrast limited adaptive
// histogram equalisation by brick decomposition, local histograms with a maximum cut-off,
// and linear interpolation of the local results), as three kernels on uint8 volumes:
//   k_clahe_hist  one CTA per brick: 256-bin histogram of the brick's codes (a sub-histogram
//                 per warp in shared memory, then one global add per bin);
//   k_clahe_lut   one CTA per brick, one thread per bin: clip at the limit, hand the excess
//                 back evenly (E / 256 to every bin, the remainder one each to every
//                 step-th bin), prefix sum, equalised mapping lut[q] = (255 cdf[q] + N/2) / N;
//   k_clahe_map   one thread per voxel: trilinear blend of the 8 nearest bricks' mappings of
//                 its code at brick coordinate t = (x + 0.5) / s - 0.5 per axis (clamped to
//                 the brick grid), rounded half to even.
// The brick size s = dims / bricks must be whole.  Histograms and mappings live in
// stream-ordered scratch for the duration of the call.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "vkt_internal.h"

namespace vkt {
namespace {

constexpr int NT = 256;
constexpr int NWARP = NT / 32;

struct ClaheGeo {
    int nx, ny, nz;
    int nbx, nby, nbz;
    int sx, sy, sz;
};

__global__ void __launch_bounds__(NT) k_clahe_hist(const uint8_t* __restrict__ src, ClaheGeo g,
                                                   unsigned* __restrict__ hist)
{
    __shared__ unsigned sh[NWARP][256];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < NWARP * 256; i += NT) (&sh[0][0])[i] = 0u;
    __syncthreads();
    const int b = blockIdx.x;
    const int bx = b % g.nbx, by = (b / g.nbx) % g.nby, bz = b / (g.nbx * g.nby);
    const int x0 = bx * g.sx, y0 = by * g.sy, z0 = bz * g.sz;
    const int rows = g.sy * g.sz;
    for (int r = warp; r < rows; r += NWARP) {
        const int z = z0 + r / g.sy, y = y0 + r % g.sy;
        const uint8_t* row = src + (static_cast<int64_t>(z) * g.ny + y) * g.nx + x0;
        for (int x = lane; x < g.sx; x += 32) atomicAdd(&sh[warp][__ldg(row + x)], 1u);
    }
    __syncthreads();
    unsigned c = 0;
#pragma unroll
    for (int w = 0; w < NWARP; ++w) c += sh[w][tid];
    hist[static_cast<int64_t>(b) * 256 + tid] = c;
}

__global__ void __launch_bounds__(256) k_clahe_lut(const unsigned* __restrict__ hist, int64_t n,
                                                   int64_t limit, uint8_t* __restrict__ luts)
{
    __shared__ int64_t red[8];
    __shared__ int64_t scan[256];
    const int i = threadIdx.x, warp = i >> 5, lane = i & 31;
    const int64_t b = blockIdx.x;
    int64_t h = hist[b * 256 + i];
    if (limit > 0) {
        // excess over the limit, summed over the 256 bins
        int64_t e = h > limit ? h - limit : 0;
        h -= e;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        if (lane == 0) red[warp] = e;
        __syncthreads();
        int64_t excess = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) excess += red[w];
        const int64_t add = excess / 256, rem = excess - add * 256;
        h += add;
        if (rem > 0) {
            const int64_t step = max(int64_t(1), int64_t(256) / rem);
            if (i % step == 0 && i / step < rem) h += 1;
        }
    }
    // inclusive prefix sum over the bins (Hillis-Steele in shared memory)
    scan[i] = h;
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {
        const int64_t v = i >= o ? scan[i - o] : 0;
        __syncthreads();
        scan[i] += v;
        __syncthreads();
    }
    const int64_t v = (255 * scan[i] + n / 2) / n;
    luts[b * 256 + i] = static_cast<uint8_t>(v > 255 ? 255 : v);
}

__device__ __forceinline__ void brick_coord(int x, int s, int nb, float inv_s, int& b0, int& b1,
                                            float& w)
{
    const float t = (static_cast<float>(x) + 0.5f) * inv_s - 0.5f;
    const float f = floorf(t);
    w = t - f;
    const int i = static_cast<int>(f);
    b0 = min(max(i, 0), nb - 1);
    b1 = min(max(i + 1, 0), nb - 1);
    (void)s;
}

__global__ void __launch_bounds__(NT) k_clahe_map(const uint8_t* __restrict__ src, ClaheGeo g,
                                                  const uint8_t* __restrict__ luts,
                                                  uint8_t* __restrict__ dst)
{
    const int x = blockIdx.x * NT + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    int x0, x1, y0, y1, z0, z1;
    float wx, wy, wz;
    brick_coord(x, g.sx, g.nbx, 1.0f / g.sx, x0, x1, wx);
    brick_coord(y, g.sy, g.nby, 1.0f / g.sy, y0, y1, wy);
    brick_coord(z, g.sz, g.nbz, 1.0f / g.sz, z0, z1, wz);
    const int64_t i = (static_cast<int64_t>(z) * g.ny + y) * g.nx + x;
    const int q = __ldg(src + i);
    auto L = [&](int bz, int by, int bx) {
        return static_cast<float>(__ldg(luts + ((static_cast<int64_t>(bz) * g.nby + by) * g.nbx + bx) * 256 + q));
    };
    const float c00 = L(z0, y0, x0) * (1.f - wx) + L(z0, y0, x1) * wx;
    const float c01 = L(z0, y1, x0) * (1.f - wx) + L(z0, y1, x1) * wx;
    const float c10 = L(z1, y0, x0) * (1.f - wx) + L(z1, y0, x1) * wx;
    const float c11 = L(z1, y1, x0) * (1.f - wx) + L(z1, y1, x1) * wx;
    const float c0 = c00 * (1.f - wy) + c01 * wy;
    const float c1 = c10 * (1.f - wy) + c11 * wy;
    const float v = c0 * (1.f - wz) + c1 * wz;
    dst[i] = static_cast<uint8_t>(fminf(fmaxf(rintf(v), 0.f), 255.f));
}

bool valid_volume(const vktStructuredVolume_impl* v) { return v && v->magic == VKT_VOLUME_MAGIC; }

}  // namespace
}  // namespace vkt

using namespace vkt;

extern "C" vktError vktClahe3DSV(vktStructuredVolume dst, vktStructuredVolume src, int32_t bricksX,
                                 int32_t bricksY, int32_t bricksZ, float clipLimit)
{
    if (!valid_volume(dst) || !valid_volume(src)) return VKT_ERROR_INVALID_HANDLE;
    if (dst->dims[0] != src->dims[0] || dst->dims[1] != src->dims[1] || dst->dims[2] != src->dims[2])
        return VKT_ERROR_DIMS_MISMATCH;
    if (src->format != vktDataFormatUint8 || dst->format != vktDataFormatUint8)
        return VKT_ERROR_UNSUPPORTED;
    const int nb[3] = {bricksX, bricksY, bricksZ};
    for (int a = 0; a < 3; ++a)
        if (nb[a] < 1 || src->dims[a] % nb[a] != 0) return VKT_ERROR_INVALID_VALUE;
    if (!(clipLimit == clipLimit)) return VKT_ERROR_INVALID_VALUE;   // NaN
    const uint64_t bytes = static_cast<uint64_t>(src->dims[0]) * src->dims[1] * src->dims[2];
    {
        const char* a = static_cast<const char*>(dst->data);
        const char* b = static_cast<const char*>(src->data);
        if (a < b + bytes && b < a + bytes) return VKT_ERROR_INVALID_VALUE;
    }
    Ctx ctx;
    vktError err = get_context(&ctx);
    if (err != VKT_NO_ERROR) return err;

    ClaheGeo g;
    g.nx = src->dims[0];
    g.ny = src->dims[1];
    g.nz = src->dims[2];
    g.nbx = bricksX;
    g.nby = bricksY;
    g.nbz = bricksZ;
    g.sx = g.nx / bricksX;
    g.sy = g.ny / bricksY;
    g.sz = g.nz / bricksZ;
    const int64_t nbricks = static_cast<int64_t>(bricksX) * bricksY * bricksZ;
    if (nbricks > 0x7fffffff || g.ny > 65535 || g.nz > 65535) return VKT_ERROR_UNSUPPORTED;
    const int64_t n = static_cast<int64_t>(g.sx) * g.sy * g.sz;
    int64_t limit = 0;   // no clipping
    if (clipLimit > 0.f) {
        limit = static_cast<int64_t>(std::floor(static_cast<double>(clipLimit) * static_cast<double>(n) / 256.0));
        limit = std::max<int64_t>(limit, 1);
    }
    unsigned* hist = nullptr;
    uint8_t* luts = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&hist), nbricks * 256 * sizeof(unsigned), ctx.stream);
    if (e != cudaSuccess) return from_cuda(e);
    e = cudaMallocAsync(reinterpret_cast<void**>(&luts), nbricks * 256, ctx.stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(hist, ctx.stream);
        return from_cuda(e);
    }
    const uint8_t* s = static_cast<const uint8_t*>(src->data);
    k_clahe_hist<<<static_cast<unsigned>(nbricks), NT, 0, ctx.stream>>>(s, g, hist);
    k_clahe_lut<<<static_cast<unsigned>(nbricks), 256, 0, ctx.stream>>>(hist, n, limit, luts);
    const dim3 grid((g.nx + NT - 1) / NT, g.ny, g.nz);
    k_clahe_map<<<grid, NT, 0, ctx.stream>>>(s, g, luts, static_cast<uint8_t*>(dst->data));
    count_launches(3);
    e = cudaGetLastError();
    if (ctx.debug & VKT_DEBUG_LOG)
        fprintf(stderr, "[vkt] clahe3d %dx%dx%d bricks %dx%dx%d (%dx%dx%d voxels) limit=%lld\n", g.nx,
                g.ny, g.nz, bricksX, bricksY, bricksZ, g.sx, g.sy, g.sz, static_cast<long long>(limit));
    const cudaError_t e1 = cudaFreeAsync(hist, ctx.stream);
    const cudaError_t e2 = cudaFreeAsync(luts, ctx.stream);
    if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2;
    return from_cuda(e);
}
