// vkt_bricks.cu -- BrickDecompose (Sec. 3.2, "domain decomposition algorithms": a volume is
// split into subgrids, optionally with ghost cells for interpolation).
//
// Brick (kx, ky, kz) covers the source voxels [o, o + s) with o = (kx bx, ky by, kz bz) and
// s = min(b, dims - o) per axis, and is stored as a volume of s + 2 g voxels per axis whose
// voxel (i, j, k) is the source voxel clamp(o - g + (i, j, k)): ghost cells inside the volume
// copy the neighbouring bricks' voxels, ghost cells beyond a face repeat the face voxel (the
// clamp-to-edge rule of ApplyFilter).  One launch copies every brick: a CTA takes a run of
// brick rows, a warp four rows at a time, the lanes consecutive x (coalesced reads and
// writes).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "vkt_internal.h"

namespace vkt {
namespace {

constexpr int NT = 256;
constexpr int MIN_ROWS_PER_CTA = 64;

struct BrickDesc {
    void* dst;
    int ox, oy, oz;      // source origin of the brick's interior
    int dx, dy, dz;      // stored dims (interior + 2 ghost)
};

bool valid_volume(const vktStructuredVolume_impl* v) { return v && v->magic == VKT_VOLUME_MAGIC; }

int elem_bytes(vktDataFormat f) { return f == vktDataFormatUint8 ? 1 : (f == vktDataFormatUint16 ? 2 : 4); }

__device__ __forceinline__ int clampd(int v, int lo, int hi) { return min(max(v, lo), hi); }

// T: the voxel's storage type as an unsigned integer of its size (bit-exact copies).  A warp
// copies RP brick rows at a time, its lanes consecutive x; a lane issues its RP x EPL loads
// before its stores (brick rows are short, so the reads in flight come from several rows).
constexpr int RP = 4, EPL = 3;

template <typename T>
__global__ void __launch_bounds__(NT)
    k_bricks(const T* __restrict__ src, int nx, int ny, int nz, const BrickDesc* __restrict__ bricks,
             int ghost, int rows_per_cta)
{
    const BrickDesc b = bricks[blockIdx.y];
    const int rows = b.dy * b.dz;
    const int r0 = blockIdx.x * rows_per_cta;
    if (r0 >= rows) return;
    const int r1 = min(rows, r0 + rows_per_cta);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* dst = static_cast<T*>(b.dst);
    // dst columns [0, left) repeat source column 0, [right, dx) column nx-1; in between
    // they are one contiguous span of the source row (plain indexing, no clamps)
    const int sx0 = b.ox - ghost;
    const int left = clampd(-sx0, 0, b.dx);
    const int right = clampd(nx - sx0, left, b.dx);
    const int n = right - left;
    for (int rb = r0 + warp * RP; rb < r1; rb += (NT / 32) * RP) {
        const T* s[RP];
        T* d[RP];
#pragma unroll
        for (int q = 0; q < RP; ++q) {
            const int r = min(rb + q, r1 - 1);
            const int k = r / b.dy, j = r - k * b.dy;
            const int sz = clampd(b.oz - ghost + k, 0, nz - 1);
            const int sy = clampd(b.oy - ghost + j, 0, ny - 1);
            const T* srow = src + (static_cast<int64_t>(sz) * ny + sy) * nx;
            T* drow = dst + static_cast<int64_t>(r) * b.dx;
            if (rb + q < r1) {
                for (int i = lane; i < left; i += 32) drow[i] = __ldg(srow);
                for (int i = right + lane; i < b.dx; i += 32) drow[i] = __ldg(srow + nx - 1);
            }
            s[q] = srow + sx0 + left;
            d[q] = drow + left;
        }
        const int nq = min(RP, r1 - rb);
        for (int c0 = lane; c0 < n; c0 += 32 * EPL) {
            T v[RP][EPL];
#pragma unroll
            for (int q = 0; q < RP; ++q)
#pragma unroll
                for (int e = 0; e < EPL; ++e)
                    if (c0 + 32 * e < n) v[q][e] = __ldg(s[q] + c0 + 32 * e);
#pragma unroll
            for (int q = 0; q < RP; ++q) {
                if (q >= nq) break;
#pragma unroll
                for (int e = 0; e < EPL; ++e)
                    if (c0 + 32 * e < n) d[q][c0 + 32 * e] = v[q][e];
            }
        }
    }
}

int bricks_along(int n, int b) { return (n + b - 1) / b; }

}  // namespace
}  // namespace vkt

using namespace vkt;

extern "C" {

vktError vktBrickDecomposeCountSV(int32_t* countX, int32_t* countY, int32_t* countZ,
                                  vktStructuredVolume volume, int32_t brickX, int32_t brickY,
                                  int32_t brickZ)
{
    if (!valid_volume(volume)) return VKT_ERROR_INVALID_HANDLE;
    if (!countX || !countY || !countZ || brickX < 1 || brickY < 1 || brickZ < 1)
        return VKT_ERROR_INVALID_VALUE;
    *countX = bricks_along(volume->dims[0], brickX);
    *countY = bricks_along(volume->dims[1], brickY);
    *countZ = bricks_along(volume->dims[2], brickZ);
    return VKT_NO_ERROR;
}

vktError vktBrickDecomposeSV(vktStructuredVolume* bricks, int32_t numBricks,
                             vktStructuredVolume volume, int32_t brickX, int32_t brickY,
                             int32_t brickZ, int32_t ghost)
{
    if (!valid_volume(volume)) return VKT_ERROR_INVALID_HANDLE;
    if (!bricks || brickX < 1 || brickY < 1 || brickZ < 1 || ghost < 0)
        return VKT_ERROR_INVALID_VALUE;
    const int nx = volume->dims[0], ny = volume->dims[1], nz = volume->dims[2];
    const int b[3] = {brickX, brickY, brickZ};
    const int cx = bricks_along(nx, brickX), cy = bricks_along(ny, brickY), cz = bricks_along(nz, brickZ);
    if (static_cast<int64_t>(cx) * cy * cz != numBricks) return VKT_ERROR_INVALID_VALUE;
    const int es = elem_bytes(volume->format);
    const char* s0 = static_cast<const char*>(volume->data);
    const uint64_t sbytes = static_cast<uint64_t>(nx) * ny * nz * es;
    std::vector<BrickDesc> desc(static_cast<size_t>(numBricks));
    int max_rows = 0;
    for (int kz = 0; kz < cz; ++kz)
        for (int ky = 0; ky < cy; ++ky)
            for (int kx = 0; kx < cx; ++kx) {
                const size_t i = (static_cast<size_t>(kz) * cy + ky) * cx + kx;
                const vktStructuredVolume_impl* v = bricks[i];
                if (!valid_volume(v)) return VKT_ERROR_INVALID_HANDLE;
                if (v->format != volume->format) return VKT_ERROR_INVALID_VALUE;
                const int o[3] = {kx * b[0], ky * b[1], kz * b[2]};
                const int n[3] = {nx, ny, nz};
                BrickDesc& d = desc[i];
                int dd[3];
                for (int a = 0; a < 3; ++a) dd[a] = std::min(b[a], n[a] - o[a]) + 2 * ghost;
                if (v->dims[0] != dd[0] || v->dims[1] != dd[1] || v->dims[2] != dd[2])
                    return VKT_ERROR_DIMS_MISMATCH;
                const char* p = static_cast<const char*>(v->data);
                const uint64_t bytes = static_cast<uint64_t>(dd[0]) * dd[1] * dd[2] * es;
                if (p < s0 + sbytes && s0 < p + bytes) return VKT_ERROR_INVALID_VALUE;
                d.dst = v->data;
                d.ox = o[0];
                d.oy = o[1];
                d.oz = o[2];
                d.dx = dd[0];
                d.dy = dd[1];
                d.dz = dd[2];
                max_rows = std::max(max_rows, dd[1] * dd[2]);
            }
    Ctx ctx;
    vktError err = get_context(&ctx);
    if (err != VKT_NO_ERROR) return err;
    // the brick table lives in stream-ordered scratch for the duration of the call
    BrickDesc* dtab = nullptr;
    const size_t tbytes = desc.size() * sizeof(BrickDesc);
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&dtab), tbytes, ctx.stream);
    if (e != cudaSuccess) return from_cuda(e);
    e = cudaMemcpyAsync(dtab, desc.data(), tbytes, cudaMemcpyHostToDevice, ctx.stream);
    // rows per CTA: enough that the grid is a few waves (short brick rows make small CTAs
    // latency-bound), at least MIN_ROWS_PER_CTA
    int sms = 152;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess)
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    const int64_t total_rows = static_cast<int64_t>(max_rows) * numBricks;
    const int64_t want = std::max<int64_t>(MIN_ROWS_PER_CTA, total_rows / (static_cast<int64_t>(sms) * 32));
    const int rows_per_cta = static_cast<int>(std::min<int64_t>(want, max_rows));
    const int gx = (max_rows + rows_per_cta - 1) / rows_per_cta;
    int launches = 0;
    // at most 65535 bricks per launch (grid y)
    for (int first = 0; e == cudaSuccess && first < numBricks; first += 65535) {
        const int nb = std::min(65535, numBricks - first);
        const dim3 grid(gx, nb);
        if (es == 1)
            k_bricks<uint8_t><<<grid, NT, 0, ctx.stream>>>(static_cast<const uint8_t*>(volume->data),
                                                           nx, ny, nz, dtab + first, ghost,
                                                            rows_per_cta);
        else if (es == 2)
            k_bricks<uint16_t><<<grid, NT, 0, ctx.stream>>>(static_cast<const uint16_t*>(volume->data),
                                                            nx, ny, nz, dtab + first, ghost,
                                                            rows_per_cta);
        else
            k_bricks<uint32_t><<<grid, NT, 0, ctx.stream>>>(static_cast<const uint32_t*>(volume->data),
                                                            nx, ny, nz, dtab + first, ghost,
                                                            rows_per_cta);
        e = cudaGetLastError();
        ++launches;
    }
    count_launches(launches);
    if (ctx.debug & VKT_DEBUG_LOG)
        fprintf(stderr, "[vkt] brick-decompose %d bricks (%dx%dx%d, ghost %d) grid=(%d,%d) launches=%d\n",
                numBricks, brickX, brickY, brickZ, ghost, gx, std::min(numBricks, 65535), launches);
    const cudaError_t ef = cudaFreeAsync(dtab, ctx.stream);
    if (e == cudaSuccess) e = ef;
    return from_cuda(e);
}

}  // extern "C"
