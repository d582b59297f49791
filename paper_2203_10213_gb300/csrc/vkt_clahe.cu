// vkt_clahe.cu -- CLAHE-3D (Sec. 4.1, "Case Study: CLAHE-3D": contrast limited adaptive
// histogram equalisation by brick decomposition, local histograms with a maximum cut-off,
// and linear interpolation of the local results), as three kernels on uint8 volumes:
//   k_clahe_hist  one CTA per brick: 256-bin histogram of the brick's codes (a sub-histogram
//                 per warp in shared memory, then one global add per bin; 16- or 4-byte
//                 loads where the rows allow, one add for a word of equal codes);
//   k_clahe_lut   one CTA per brick, one thread per bin: clip at the limit, hand the excess
//                 back evenly (E / 256 to every bin, the remainder one each to every
//                 step-th bin), prefix sum, equalised mapping lut[q] = (255 cdf[q] + N/2) / N;
//   k_clahe_map   one thread per voxel: trilinear blend of the 8 nearest bricks' mappings of
//                 its code at brick coordinate t = (x + 0.5) / s - 0.5 per axis (clamped to
//                 the brick grid), rounded half to even (k_clahe_map_cells: the same blend
//                 by cells between brick centres, their mappings staged in shared memory).
// The brick size s = dims / bricks must be whole.  Histograms and mappings live in
// stream-ordered scratch for the duration of the call.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <type_traits>

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

// VEC: bytes a lane reads at once (1, 4 or 16; the brick rows and the volume's rows are
// multiples of VEC long).  A 4-byte word of equal codes (the CT volume's uniform regions)
// counts with one atomic add of 4 instead of four adds to the same bin.
__device__ __forceinline__ void hist_word(unsigned* h, uint32_t w)
{
    const uint32_t b0 = w & 0xffu;
    if (w == b0 * 0x01010101u) {
        atomicAdd(&h[b0], 4u);
    } else {
        atomicAdd(&h[b0], 1u);
        atomicAdd(&h[(w >> 8) & 0xffu], 1u);
        atomicAdd(&h[(w >> 16) & 0xffu], 1u);
        atomicAdd(&h[w >> 24], 1u);
    }
}

template <int VEC>
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
    unsigned* h = sh[warp];
    if constexpr (VEC == 1) {
        const int rows = g.sy * g.sz;
        for (int r = warp; r < rows; r += NWARP) {
            const int z = z0 + r / g.sy, y = y0 + r % g.sy;
            const uint8_t* row = src + (static_cast<int64_t>(z) * g.ny + y) * g.nx + x0;
            for (int x = lane; x < g.sx; x += 32) atomicAdd(&h[__ldg(row + x)], 1u);
        }
    } else {
        // items: (row, VEC-byte group), groups fastest; a thread loads HU items before
        // counting them
        constexpr int HU = 4;
        using V = typename std::conditional<VEC == 4, uint32_t, uint4>::type;
        const int gpr = g.sx / VEC;
        const int items = gpr * g.sy * g.sz;
        for (int i0 = tid; i0 < items; i0 += HU * NT) {
            V v[HU];
#pragma unroll
            for (int u = 0; u < HU; ++u) {
                const int it = i0 + u * NT;
                if (it < items) {
                    const int r = it / gpr, gi = it - r * gpr;
                    const int z = z0 + r / g.sy, y = y0 + r % g.sy;
                    const uint8_t* p = src + (static_cast<int64_t>(z) * g.ny + y) * g.nx + x0 + gi * VEC;
                    v[u] = __ldg(reinterpret_cast<const V*>(p));
                }
            }
#pragma unroll
            for (int u = 0; u < HU; ++u) {
                if (i0 + u * NT >= items) break;
                if constexpr (VEC == 4) {
                    hist_word(h, v[u]);
                } else {
                    const uint4 w = v[u];
                    if (w.x == w.y && w.x == w.z && w.x == w.w && w.x == (w.x & 0xffu) * 0x01010101u) {
                        atomicAdd(&h[w.x & 0xffu], 16u);
                    } else {
                        hist_word(h, w.x);
                        hist_word(h, w.y);
                        hist_word(h, w.z);
                        hist_word(h, w.w);
                    }
                }
            }
        }
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

// The same blend by cells: along an axis, the voxels between two neighbouring brick centres
// share their pair of bricks (b0, b1) = (clamp(i), clamp(i + 1)), cell i covering the x with
// floor((x + 0.5) / s - 0.5) = i, i.e. [s i + s/2, s (i + 1) + s/2) (integer division, cut
// to the volume; i = -1 and i = nb - 1 are the half cells at the faces).  A CTA takes one
// cell (a z slab of it), stages its 8 mappings interleaved (tab[q] = the 8 codes of q, as
// floats) in shared memory, and blends each voxel from two 16-byte shared loads.  Each voxel still
// computes its brick coordinates as k_clahe_map does and takes the global mappings if float
// rounding puts it in a neighbouring cell, so the results are the same bits.
__device__ __forceinline__ void cell_range(int i, int s, int nb, int n, int& lo, int& hi)
{
    lo = i < 0 ? 0 : min(n, s * i + s / 2);
    hi = i + 1 < nb ? min(n, s * (i + 1) + s / 2) : n;
}

// Off: the type of voxel offsets (32 bits for volumes under 2^32 voxels)
template <typename Off>
__global__ void __launch_bounds__(NT, 4) k_clahe_map_cells(const uint8_t* __restrict__ src, ClaheGeo g,
                                                        const uint8_t* __restrict__ luts,
                                                        uint8_t* __restrict__ dst, int tz)
{
    __shared__ float4 tab[256][2];   // q -> (z0: y0x0 y0x1 y1x0 y1x1), (z1: ...)
    const int ncx = g.nbx + 1, ncy = g.nby + 1;
    const int c = blockIdx.x;
    const int ci = c % ncx - 1, cj = (c / ncx) % ncy - 1, ck = c / (ncx * ncy) - 1;
    int X0, X1, Y0, Y1, Z0, Z1;
    cell_range(ci, g.sx, g.nbx, g.nx, X0, X1);
    cell_range(cj, g.sy, g.nby, g.ny, Y0, Y1);
    cell_range(ck, g.sz, g.nbz, g.nz, Z0, Z1);
    const int zlo = Z0 + static_cast<int>(blockIdx.y) * tz, zhi = min(Z1, zlo + tz);
    if (X0 >= X1 || Y0 >= Y1 || zlo >= zhi) return;
    const int bx0 = min(max(ci, 0), g.nbx - 1), bx1 = min(max(ci + 1, 0), g.nbx - 1);
    const int by0 = min(max(cj, 0), g.nby - 1), by1 = min(max(cj + 1, 0), g.nby - 1);
    const int bz0 = min(max(ck, 0), g.nbz - 1), bz1 = min(max(ck + 1, 0), g.nbz - 1);
    const int nby = g.nby, nbx = g.nbx;
    auto G = [luts, nby, nbx](int bz, int by, int bx, int q) {
        return static_cast<uint32_t>(__ldg(luts + static_cast<int64_t>((bz * nby + by) * nbx + bx) * 256 + q));
    };
    {
        const int q = threadIdx.x;   // NT == 256 entries
        auto F = [&](int bz, int by, int bx) { return static_cast<float>(G(bz, by, bx, q)); };
        tab[q][0] = make_float4(F(bz0, by0, bx0), F(bz0, by0, bx1), F(bz0, by1, bx0), F(bz0, by1, bx1));
        tab[q][1] = make_float4(F(bz1, by0, bx0), F(bz1, by0, bx1), F(bz1, by1, bx0), F(bz1, by1, bx1));
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float isx = 1.0f / g.sx, isy = 1.0f / g.sy, isz = 1.0f / g.sz;
    // lanes over x (one x per lane for cells up to 32 wide), then z, then RU consecutive
    // rows y per warp whose codes are loaded before they are blended
    constexpr int RU = 4;
    for (int x = X0 + lane; x < X1; x += 32) {
        int x0, x1;
        float wx;
        brick_coord(x, g.sx, g.nbx, isx, x0, x1, wx);
        const bool xm = x0 == bx0 && x1 == bx1;
        for (int z = zlo; z < zhi; ++z) {
            int z0, z1;
            float wz;
            brick_coord(z, g.sz, g.nbz, isz, z0, z1, wz);
            const bool zm = xm && z0 == bz0 && z1 == bz1;
            const Off plane = static_cast<Off>(z) * g.ny;
            for (int yb = Y0 + warp * RU; yb < Y1; yb += NWARP * RU) {
                int qv[RU];
#pragma unroll
                for (int u = 0; u < RU; ++u) {
                    const int y = min(yb + u, Y1 - 1);
                    qv[u] = __ldg(src + (plane + y) * g.nx + x);
                }
#pragma unroll
                for (int u = 0; u < RU; ++u) {
                    const int y = yb + u;
                    if (y < Y1) {
                        int y0, y1;
                        float wy;
                        brick_coord(y, g.sy, g.nby, isy, y0, y1, wy);
                        const int q = qv[u];
                        float l000, l001, l010, l011, l100, l101, l110, l111;
                        if (zm && y0 == by0 && y1 == by1) {
                            const float4 e0 = tab[q][0], e1 = tab[q][1];
                            l000 = e0.x;
                            l001 = e0.y;
                            l010 = e0.z;
                            l011 = e0.w;
                            l100 = e1.x;
                            l101 = e1.y;
                            l110 = e1.z;
                            l111 = e1.w;
                        } else {
                            // float rounding put the voxel in a neighbouring cell
                            const uint8_t* pq = luts + q;
                            auto Lg = [&](int bz, int by, int bx) {
                                return static_cast<float>(
                                    __ldg(pq + static_cast<int64_t>((bz * nby + by) * nbx + bx) * 256));
                            };
                            l000 = Lg(z0, y0, x0);
                            l001 = Lg(z0, y0, x1);
                            l010 = Lg(z0, y1, x0);
                            l011 = Lg(z0, y1, x1);
                            l100 = Lg(z1, y0, x0);
                            l101 = Lg(z1, y0, x1);
                            l110 = Lg(z1, y1, x0);
                            l111 = Lg(z1, y1, x1);
                        }
                        const float c00 = l000 * (1.f - wx) + l001 * wx;
                        const float c01 = l010 * (1.f - wx) + l011 * wx;
                        const float c10 = l100 * (1.f - wx) + l101 * wx;
                        const float c11 = l110 * (1.f - wx) + l111 * wx;
                        const float c0 = c00 * (1.f - wy) + c01 * wy;
                        const float c1 = c10 * (1.f - wy) + c11 * wy;
                        const float v = c0 * (1.f - wz) + c1 * wz;
                        dst[(plane + y) * g.nx + x] = static_cast<uint8_t>(fminf(fmaxf(rintf(v), 0.f), 255.f));
                    }
                }
            }
        }
    }
}

bool valid_volume(const vktStructuredVolume_impl* v) { return v && v->magic == VKT_VOLUME_MAGIC; }

}  // namespace
}  // namespace vkt

using namespace vkt;

extern "C" vktError vktClahe3DSV(vktStructuredVolume dst, vktStructuredVolume src, int32_t bricksX,
                                 int32_t bricksY, int32_t bricksZ, float clipLimit)
{
    vkt::CallRange nvtx_range("vktClahe3DSV");
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
    // widest loads the rows allow (brick rows and volume rows multiples of the width, the
    // data 16-byte aligned)
    const bool al16 = (reinterpret_cast<uintptr_t>(s) & 15) == 0;
    const int vec = (al16 && g.sx % 16 == 0 && g.nx % 16 == 0) ? 16
                    : ((reinterpret_cast<uintptr_t>(s) & 3) == 0 && g.sx % 4 == 0 && g.nx % 4 == 0) ? 4 : 1;
    if (vec == 16)
        k_clahe_hist<16><<<static_cast<unsigned>(nbricks), NT, 0, ctx.stream>>>(s, g, hist);
    else if (vec == 4)
        k_clahe_hist<4><<<static_cast<unsigned>(nbricks), NT, 0, ctx.stream>>>(s, g, hist);
    else
        k_clahe_hist<1><<<static_cast<unsigned>(nbricks), NT, 0, ctx.stream>>>(s, g, hist);
    k_clahe_lut<<<static_cast<unsigned>(nbricks), 256, 0, ctx.stream>>>(hist, n, limit, luts);
    // cells of at least 2048 voxels amortise staging their mappings; smaller bricks blend
    // voxel by voxel from the global mappings
    const int64_t cells = static_cast<int64_t>(bricksX + 1) * (bricksY + 1) * (bricksZ + 1);
    const bool by_cells = n >= 2048 && cells <= 0x7fffffff;
    if (by_cells) {
        const int tz = std::max(1, 16384 / (g.sx * g.sy));
        const dim3 grid(static_cast<unsigned>(cells), (g.sz + tz - 1) / tz);
        if (bytes <= 0xffffffffull)
            k_clahe_map_cells<uint32_t><<<grid, NT, 0, ctx.stream>>>(s, g, luts, static_cast<uint8_t*>(dst->data), tz);
        else
            k_clahe_map_cells<int64_t><<<grid, NT, 0, ctx.stream>>>(s, g, luts, static_cast<uint8_t*>(dst->data), tz);
    } else {
        const dim3 grid((g.nx + NT - 1) / NT, g.ny, g.nz);
        k_clahe_map<<<grid, NT, 0, ctx.stream>>>(s, g, luts, static_cast<uint8_t*>(dst->data));
    }
    count_launches(3);
    e = cudaGetLastError();
    if (ctx.debug & VKT_DEBUG_LOG)
        fprintf(stderr, "[vkt] clahe3d %dx%dx%d bricks %dx%dx%d (%dx%dx%d voxels) limit=%lld blend=%s\n",
                g.nx, g.ny, g.nz, bricksX, bricksY, bricksZ, g.sx, g.sy, g.sz,
                static_cast<long long>(limit), by_cells ? "cells" : "voxels");
    if (ctx.debug & VKT_DEBUG_LOG) fprintf(stderr, "[vkt] clahe3d histogram loads of %d bytes\n", vec);
    const cudaError_t e1 = cudaFreeAsync(hist, ctx.stream);
    const cudaError_t e2 = cudaFreeAsync(luts, ctx.stream);
    if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2;
    return from_cuda(e);
}
